// Step planner: an estimate of every partition's work, made before the kinetic kernel
// starts, so that the partitions are handed out longest-first (the kinetic launch lasts
// as long as its busiest warp), and, with the learned proposal, the proposal's guess for
// every move computed at once instead of inside each move.
//
// This is this library's scheduling extension of Fig. 4's parallel loop over the blocks
// (the paper takes the blocks in no particular order); it never changes the
// triangulation, only which warp takes which partition when, and where the locate of a
// move looks first.
//
//   k_plan      one thread per move: walk the moved point's star (its degree k), and
//               with the network compute the move's 32 features and evaluate the
//               network (the same features and the same FP32 operation order as the
//               warp-level evaluation inside a move, so the guess is the same when the
//               star has not changed meanwhile); the move's estimated cost (k + 8, plus
//               the predicted cavity size 2^out17 with the network) is added to its
//               partition's total.
//               With the network on the tensor cores the features go to a buffer
//               instead and k_mlp_tc<1> evaluates all moves' rows as dense products.
//   k_order     counting sort of the partitions by their estimated cost, largest
//               first (64 logarithmic classes; the order inside a class is the order in
//               which the atomics arrive, which only affects scheduling).
#pragma once

namespace kd {

constexpr int PLAN_ORDER = 1;    // kdt_config.plan bit: hand out partitions by estimated work
constexpr int PLAN_NETWORK = 2;  // ... bit: evaluate the proposal for all moves in the planner
constexpr int PLAN_TENSOR = 4;   // ... bit: with PLAN_NETWORK, evaluate it on the tensor cores
constexpr int PLAN_THREADS = 256;
constexpr int PLAN_CLASSES = 64;

// Star of p in ccw order from pt_tri[p]: link vertices into L (up to KMAX), returns the
// degree, -1 for a hull point (a ghost in the link) or an inconsistent read, -2 for a
// degree above KMAX.  Reads only: the store is not being written while the planner runs.
__device__ __forceinline__ int plan_star(const Dev &d, int p, int *L)
{
    const int t0 = __ldcg(d.pt_tri + p);
    if (t0 < 0 || t0 >= d.cap) return -1;
    int t = t0, k = 0;
    for (int guard = 0; guard <= KMAX; ++guard) {
        const int4 v = __ldcg(d.tv + t);
        const int4 nb = __ldcg(d.tn + t);
        if (!(v.w & ALIVE)) return -1;
        const int i = v.x == p ? 0 : (v.y == p ? 1 : (v.z == p ? 2 : -1));
        if (i < 0) return -1;
        const int a = comp(v, (i + 1) % 3);
        if (a == KDT_GHOST) return -1;
        if (k == KMAX) return -2;
        L[k++] = a;
        const int nx = comp(nb, (i + 1) % 3) >> 2;
        if (nx == t0) return k >= 3 ? k : -1;
        if (nx < 0 || nx >= d.cap) return -1;
        t = nx;
    }
    return -2;
}

// The network's guess for one row of features x (the argmax of the 17 slot logits,
// lowest index on ties) and its output 17 (predicted log2 of the cavity size).  W holds
// the parameters as FP32 (shared memory); every sum runs in the order of
// mlp_warp_forward.
__device__ __forceinline__ int plan_network(const float *W, const float *x, float &out17)
{
    float h1[MLP_H];
#pragma unroll
    for (int u = 0; u < MLP_H; ++u) {
        float a = W[OFF_B1 + u];
        const float *r = W + OFF_W1 + u * MLP_IN;
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) a = fmaf(r[k], x[k], a);
        h1[u] = fmaxf(a, 0.f);
    }
    float out[MLP_OUT];
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) out[o] = W[OFF_B3 + o];
    // eight hidden units at a time: eight independent sums in flight (each unit's sum
    // and the outputs' sums over the units keep their order)
    constexpr int UB = 8;
    for (int u0 = 0; u0 < MLP_H; u0 += UB) {
        float c[UB];
#pragma unroll
        for (int j = 0; j < UB; ++j) c[j] = W[OFF_B2 + u0 + j];
#pragma unroll
        for (int k = 0; k < MLP_H; ++k)
#pragma unroll
            for (int j = 0; j < UB; ++j) c[j] = fmaf(W[OFF_W2 + (u0 + j) * MLP_H + k], h1[k], c[j]);
#pragma unroll
        for (int j = 0; j < UB; ++j) {
            const float g = fmaxf(c[j], 0.f);
#pragma unroll
            for (int o = 0; o < MLP_OUT; ++o) out[o] = fmaf(W[OFF_W3 + o * MLP_H + u0 + j], g, out[o]);
        }
    }
    int best = 0;
    float bv = out[0];
#pragma unroll
    for (int o = 1; o < MLP_SLOTS; ++o)
        if (out[o] > bv) {
            bv = out[o];
            best = o;
        }
    out17 = out[MLP_SLOTS];
    return best;
}

// The 32 features of a move of p (at po, link L of degree k) to q, as move_feature
// defines them (every operation correctly rounded FP32, sums in the same order);
// returns false when no wedge holds the move direction.
__device__ __forceinline__ bool plan_features(const Dev &d, const int *L, int k, int2 po, int2 q, float *x)
{
    const long long dx = (long long)q.x - po.x, dy = (long long)q.y - po.y;
    int j0 = -1, hits = 0;
    int2 first = __ldcg(d.xy + L[0]), a = first;
    for (int j = 0; j < k; ++j) {
        const int2 b = j + 1 == k ? first : __ldcg(d.xy + L[j + 1]);
        const long long ax = (long long)a.x - po.x, ay = (long long)a.y - po.y;
        const long long bx = (long long)b.x - po.x, by = (long long)b.y - po.y;
        if (ax * dy - ay * dx >= 0 && dx * by - dy * bx > 0) {
            j0 = j;
            ++hits;
        }
        a = b;
    }
    if (hits != 1) return false;
    const float fdx = __int2float_rn(q.x - po.x), fdy = __int2float_rn(q.y - po.y);
    const float s = __fsqrt_rn(__fadd_rn(__fmul_rn(fdx, fdx), __fmul_rn(fdy, fdy)));
    const float ux = __fdiv_rn(fdx, s), uy = __fdiv_rn(fdy, s);
    float R = 0.f;
    for (int r = 0; r < k; ++r) {
        const int j = j0 + r >= k ? j0 + r - k : j0 + r;
        const int2 v = __ldcg(d.xy + L[j]);
        const float rx = __int2float_rn(v.x - po.x), ry = __int2float_rn(v.y - po.y);
        R = __fadd_rn(R, __fsqrt_rn(__fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry))));
    }
    R = __fdiv_rn(R, __int2float_rn(k));
    x[0] = __fdiv_rn(s, R);
    x[1] = __fdiv_rn(__int2float_rn(k), 16.0f);
#pragma unroll
    for (int r = 0; r < 15; ++r) {
        float f0 = 0.f, f1 = 0.f;
        if (r < k) {
            const int j = j0 + r >= k ? j0 + r - k : j0 + r;
            const int2 v = __ldcg(d.xy + L[j]);
            const float rx = __int2float_rn(v.x - po.x), ry = __int2float_rn(v.y - po.y);
            f0 = __fdiv_rn(__fadd_rn(__fmul_rn(rx, ux), __fmul_rn(ry, uy)), R);
            f1 = __fdiv_rn(__fsub_rn(__fmul_rn(ry, ux), __fmul_rn(rx, uy)), R);
        }
        x[2 + 2 * r] = f0;
        x[3 + 2 * r] = f1;
    }
    return true;
}

// One thread per move i < m (m from the step's control words in a graph launch):
// pguess[p] = the network's guess (0 .. 16, -1 = none) when mlp is set; pcost[cell of
// the move's partition] += its estimated cost when pcost is set.  With feat set (the
// network evaluated on the tensor cores afterwards, k_mlp_tc<1>) the move's features go
// to feat[i][0..31] and its partition to part[i] (-1: no features, no guess), pguess[p]
// is set to -1 and the cost here leaves out the network's part.
__global__ void __launch_bounds__(PLAN_THREADS) k_plan(Dev d, const int3 *gmoves, const int2 *old_xy, int m, Inst I,
                                                       int bits, const unsigned short *mlp, signed char *pguess,
                                                       float *pcost, float *feat, int *part)
{
    __shared__ float W[MLP_PARAMS];
    if (d.ctl) m = __ldcg(d.ctl);
    const int first = blockIdx.x * blockDim.x;
    if (first >= m) return;  // (uniform per block, before the barrier)
    if (mlp) {
        for (int i = threadIdx.x; i < MLP_PARAMS; i += blockDim.x) W[i] = __uint_as_float((unsigned)__ldg(mlp + i) << 16);
        __syncthreads();
    }
    int L[KMAX];
    for (int i = first + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int3 mv = gmoves[i];
        const int p = mv.x;
        const int2 po = old_xy[i], q = make_int2(mv.y, mv.z);
        const int k = plan_star(d, p, L);
        float cost = 8.f + (k > 0 ? (float)k : (k == -2 ? 4.f * KMAX : 8.f));
        int guess = -1;
        bool featured = false;
        float x[MLP_IN];
        if ((mlp || feat) && k > 0) featured = plan_features(d, L, k, po, q, x);
        if (featured && mlp) {
            float o17 = 0.f;
            guess = plan_network(W, x, o17);
            cost += exp2f(fminf(fmaxf(o17, 0.f), 10.f));
        }
        if (pguess) pguess[p] = (signed char)guess;
        int cell = -1;
        if (pcost || feat) {
            const int inst = I.ninst > 1 ? csr_find(I.moff, I.ninst + 1, i) : 0;
            cell = partition_of(I, inst, bits, po);
        }
        if (pcost) atomicAdd(pcost + cell, cost);
        if (feat) {
            if (featured) {
                float4 *f4 = reinterpret_cast<float4 *>(feat + (long long)i * MLP_IN);
#pragma unroll
                for (int c = 0; c < MLP_IN / 4; ++c) f4[c] = make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
            }
            part[i] = featured ? cell : -1;
        }
    }
}

__device__ __forceinline__ int plan_class(float c)
{
    if (!(c > 0.f)) return 0;
    return min(PLAN_CLASSES - 1, 1 + (int)(4.f * log2f(1.f + c)));
}

// phase 0: classes' sizes into hist[0 .. 63]; phase 1: order[] = partitions by class,
// largest class first (cursor = hist[64 .. 127], zero before phase 0).  Partitions are
// visited with the scattering stride (Inst.stride), so that inside a class neighbouring
// partitions are rarely next to each other.
__global__ void k_order(const float *pcost, int ncells, int *hist, int *order, int phase, int stride)
{
    __shared__ int start[PLAN_CLASSES];
    if (phase == 1) {
        if (threadIdx.x == 0) {
            int run = 0;
            for (int c = PLAN_CLASSES - 1; c >= 0; --c) {
                start[c] = run;
                run += __ldcg(hist + c);
            }
        }
        __syncthreads();
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ncells; j += gridDim.x * blockDim.x) {
        const int i = stride > 1 ? (int)(((long long)j * stride) % ncells) : j;
        const int c = plan_class(pcost[i]);
        if (phase == 0) {
            atomicAdd(hist + c, 1);
        } else {
            const int pos = start[c] + atomicAdd(hist + PLAN_CLASSES + c, 1);
            if (pos < ncells) order[pos] = i;
        }
    }
}

}  // namespace kd
