// Learned locate proposal: a small network that guesses, from the shape of the hole a
// deletion leaves, which of its triangles will hold the moved point's new position.
// It is this library's extension of the locate step (paper, Section IV: a walk finds
// the triangle that holds the point to insert); the paper has no learned component.
// A guess is only a starting point: the exact test decides, so results never depend
// on the network.
//
// Network: 32 inputs -> 64 (ReLU) -> 64 (ReLU) -> 18 outputs; outputs 0..16 are the
// logits of the landing slot (16 = "beyond"), output 17 predicts log2 of the cavity
// size.  Parameters (7442, BF16, one flat array): W1 [64][32] (row = output unit),
// b1 [64], W2 [64][64], b2 [64], W3 [18][64], b3 [18].  Products and sums are FP32.
//
// Kernels here:
//   mlp_warp_forward   one warp evaluates the network for one input row (used inside
//                      the kinetic kernel and by k_mlp_forward),
//   k_mlp_grad         forward + backward of the mean loss over a batch of rows
//                      (cross-entropy of the slot + lam * squared error of out17 against
//                      log2(cavity size)), per-block partial gradients,
//   k_mlp_reduce       fixed-order sum of the partials (deterministic),
//   k_mlp_adam         Adam (Kingma and Ba, 2015) on FP32 master parameters, writing
//                      their BF16 rounding for the network.
#pragma once
#include <cuda_bf16.h>
#include <math_constants.h>

namespace kd {

constexpr int MLP_IN = 32, MLP_H = 64, MLP_OUT = 18, MLP_SLOTS = 17, MLP_BEYOND = 16;
constexpr int OFF_W1 = 0, OFF_B1 = 2048, OFF_W2 = 2112, OFF_B2 = 6208, OFF_W3 = 6272, OFF_B3 = 7424;
constexpr int MLP_PARAMS = 7442;

__device__ __forceinline__ float bf_lo(unsigned u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(unsigned u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ float bf_at(const unsigned short *w, int i)
{
    return __uint_as_float((unsigned)__ldg(w + i) << 16);
}

// One row through the network on one warp: lane l holds input l; lane o < 18 gets
// output o.  Every offset of the layout is even, so rows are read as BF16 pairs.
__device__ __forceinline__ float mlp_warp_forward(const unsigned short *w, float x, int lane)
{
    const unsigned FULLM = 0xffffffffu;
    const unsigned *w32 = reinterpret_cast<const unsigned *>(w);
    float a0 = bf_at(w, OFF_B1 + lane), a1 = bf_at(w, OFF_B1 + lane + 32);
    const unsigned *r0 = w32 + (OFF_W1 + lane * MLP_IN) / 2;
    const unsigned *r1 = w32 + (OFF_W1 + (lane + 32) * MLP_IN) / 2;
#pragma unroll
    for (int kk = 0; kk < MLP_IN / 2; ++kk) {
        float x0 = __shfl_sync(FULLM, x, 2 * kk), x1 = __shfl_sync(FULLM, x, 2 * kk + 1);
        unsigned u0 = __ldg(r0 + kk), u1 = __ldg(r1 + kk);
        a0 = fmaf(bf_lo(u0), x0, a0);
        a0 = fmaf(bf_hi(u0), x1, a0);
        a1 = fmaf(bf_lo(u1), x0, a1);
        a1 = fmaf(bf_hi(u1), x1, a1);
    }
    const float h0 = fmaxf(a0, 0.f), h1 = fmaxf(a1, 0.f);  // units lane, lane + 32
    float c0 = bf_at(w, OFF_B2 + lane), c1 = bf_at(w, OFF_B2 + lane + 32);
    const unsigned *s0 = w32 + (OFF_W2 + lane * MLP_H) / 2;
    const unsigned *s1 = w32 + (OFF_W2 + (lane + 32) * MLP_H) / 2;
#pragma unroll
    for (int kk = 0; kk < MLP_H / 2; ++kk) {
        const float src = kk < 16 ? h0 : h1;
        const int l = (2 * kk) & 31;
        float y0 = __shfl_sync(FULLM, src, l), y1 = __shfl_sync(FULLM, src, l + 1);
        unsigned u0 = __ldg(s0 + kk), u1 = __ldg(s1 + kk);
        c0 = fmaf(bf_lo(u0), y0, c0);
        c0 = fmaf(bf_hi(u0), y1, c0);
        c1 = fmaf(bf_lo(u1), y0, c1);
        c1 = fmaf(bf_hi(u1), y1, c1);
    }
    const float g0 = fmaxf(c0, 0.f), g1 = fmaxf(c1, 0.f);
    const int o = lane < MLP_OUT ? lane : 0;
    float e = bf_at(w, OFF_B3 + o);
    const unsigned *t0 = w32 + (OFF_W3 + o * MLP_H) / 2;
#pragma unroll
    for (int kk = 0; kk < MLP_H / 2; ++kk) {
        const float src = kk < 16 ? g0 : g1;
        const int l = (2 * kk) & 31;
        float z0 = __shfl_sync(FULLM, src, l), z1 = __shfl_sync(FULLM, src, l + 1);
        unsigned u = __ldg(t0 + kk);
        e = fmaf(bf_lo(u), z0, e);
        e = fmaf(bf_hi(u), z1, e);
    }
    return e;
}

// Arg-max of the 17 slot logits held by lanes 0..16 (lowest index on ties).
__device__ __forceinline__ int mlp_argmax_slot(float out, int lane)
{
    float v = lane < MLP_SLOTS ? out : -CUDART_INF_F;
    int idx = lane;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        float v2 = __shfl_xor_sync(0xffffffffu, v, off);
        int i2 = __shfl_xor_sync(0xffffffffu, idx, off);
        if (v2 > v || (v2 == v && i2 < idx)) {
            v = v2;
            idx = i2;
        }
    }
    return idx;
}

// Batched forward pass: one warp per row, outputs (rows x 18).
__global__ void k_mlp_forward(const unsigned short *w, const float *x, long long rows, float *out)
{
    const int lane = threadIdx.x & 31;
    long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (; row < rows; row += nw) {
        float o = mlp_warp_forward(w, x[row * MLP_IN + lane], lane);
        if (lane < MLP_OUT) out[row * MLP_OUT + lane] = o;
    }
}

// ---------------------------------------------------------------- training

constexpr int GT = 32;             // rows per tile
constexpr int GTHREADS = 256;      // threads per block
constexpr int GPER = (MLP_PARAMS + GTHREADS - 1) / GTHREADS;  // parameters per thread (30)

struct MlpSmem {
    float w[MLP_PARAMS];            // the BF16 parameters as FP32
    float x[GT][MLP_IN];
    float z1[GT][MLP_H];            // pre-activations (ReLU masks)
    float h1[GT][MLP_H];
    float z2[GT][MLP_H];
    float h2[GT][MLP_H];
    float dout[GT][MLP_OUT];
    float dz2[GT][MLP_H];
    float dz1[GT][MLP_H];
    float loss[GT];
};

// Forward + backward of the mean loss over `rows` rows (row r of the batch is input
// row idx[r], or r when idx is null).  Block b accumulates the gradient of its tiles
// in registers (thread t owns parameters t, t + 256, ...) and writes it to
// partial[b][.]; its loss sum goes to partial_loss[b].  Labels: (slot, cavity size)
// per row.  Gradients are those of the mean (every row's term is divided by rows).
__global__ void __launch_bounds__(GTHREADS) k_mlp_grad(const unsigned short *wb, const float *x, const int *labels,
                                                       const long long *idx, long long rows, float lam,
                                                       float *partial, float *partial_loss)
{
    extern __shared__ float smem_raw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem_raw);
    const int tid = threadIdx.x;
    for (int i = tid; i < MLP_PARAMS; i += GTHREADS) S.w[i] = __uint_as_float((unsigned)wb[i] << 16);
    float acc[GPER];
#pragma unroll
    for (int i = 0; i < GPER; ++i) acc[i] = 0.f;
    float lsum = 0.f;
    const float inv_rows = 1.0f / (float)rows;
    const float *W1 = S.w + OFF_W1, *B1 = S.w + OFF_B1, *W2 = S.w + OFF_W2, *B2 = S.w + OFF_B2;
    const float *W3 = S.w + OFF_W3, *B3 = S.w + OFF_B3;
    const long long ntiles = (rows + GT - 1) / GT;
    __syncthreads();
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long r0 = tile * GT;
        const int nr = (int)(rows - r0 < GT ? rows - r0 : GT);
        // inputs (zero past the last row)
        for (int i = tid; i < GT * MLP_IN; i += GTHREADS) {
            int r = i / MLP_IN, c = i - r * MLP_IN;
            float v = 0.f;
            if (r < nr) {
                long long row = idx ? idx[r0 + r] : r0 + r;
                v = x[row * MLP_IN + c];
            }
            S.x[r][c] = v;
        }
        __syncthreads();
        // layer 1
        for (int i = tid; i < GT * MLP_H; i += GTHREADS) {
            int r = i / MLP_H, n = i - r * MLP_H;
            float a = B1[n];
            for (int c = 0; c < MLP_IN; ++c) a = fmaf(W1[n * MLP_IN + c], S.x[r][c], a);
            S.z1[r][n] = a;
            S.h1[r][n] = fmaxf(a, 0.f);
        }
        __syncthreads();
        // layer 2
        for (int i = tid; i < GT * MLP_H; i += GTHREADS) {
            int r = i / MLP_H, n = i - r * MLP_H;
            float a = B2[n];
            for (int c = 0; c < MLP_H; ++c) a = fmaf(W2[n * MLP_H + c], S.h1[r][c], a);
            S.z2[r][n] = a;
            S.h2[r][n] = fmaxf(a, 0.f);
        }
        __syncthreads();
        // layer 3 (into dout, turned into the output gradient below)
        for (int i = tid; i < GT * MLP_OUT; i += GTHREADS) {
            int r = i / MLP_OUT, o = i - r * MLP_OUT;
            float a = B3[o];
            for (int c = 0; c < MLP_H; ++c) a = fmaf(W3[o * MLP_H + c], S.h2[r][c], a);
            S.dout[r][o] = a;
        }
        __syncthreads();
        // loss and output gradient: one thread per row
        if (tid < GT) {
            const int r = tid;
            if (r < nr) {
                long long row = idx ? idx[r0 + r] : r0 + r;
                int slot = labels[2 * row];
                float target = log2f((float)labels[2 * row + 1]);
                float mx = S.dout[r][0];
                for (int o = 1; o < MLP_SLOTS; ++o) mx = fmaxf(mx, S.dout[r][o]);
                float se = 0.f;
                for (int o = 0; o < MLP_SLOTS; ++o) se += expf(S.dout[r][o] - mx);
                float lse = mx + logf(se);
                float res = S.dout[r][MLP_SLOTS] - target;
                S.loss[r] = (lse - S.dout[r][slot]) + lam * res * res;
                for (int o = 0; o < MLP_SLOTS; ++o) {
                    float pr = expf(S.dout[r][o] - lse);
                    S.dout[r][o] = (pr - (o == slot ? 1.f : 0.f)) * inv_rows;
                }
                S.dout[r][MLP_SLOTS] = 2.f * lam * res * inv_rows;
            } else {
                S.loss[r] = 0.f;
                for (int o = 0; o < MLP_OUT; ++o) S.dout[r][o] = 0.f;
            }
        }
        __syncthreads();
        if (tid == 0)
            for (int r = 0; r < GT; ++r) lsum += S.loss[r];
        // back through layer 3 and the second ReLU
        for (int i = tid; i < GT * MLP_H; i += GTHREADS) {
            int r = i / MLP_H, n = i - r * MLP_H;
            float a = 0.f;
            for (int o = 0; o < MLP_OUT; ++o) a = fmaf(W3[o * MLP_H + n], S.dout[r][o], a);
            S.dz2[r][n] = S.z2[r][n] > 0.f ? a : 0.f;
        }
        __syncthreads();
        // back through layer 2 and the first ReLU
        for (int i = tid; i < GT * MLP_H; i += GTHREADS) {
            int r = i / MLP_H, n = i - r * MLP_H;
            float a = 0.f;
            for (int m = 0; m < MLP_H; ++m) a = fmaf(W2[m * MLP_H + n], S.dz2[r][m], a);
            S.dz1[r][n] = S.z1[r][n] > 0.f ? a : 0.f;
        }
        __syncthreads();
        // parameter gradients of this tile, summed over its rows
#pragma unroll
        for (int j = 0; j < GPER; ++j) {
            const int pidx = tid + j * GTHREADS;
            if (pidx >= MLP_PARAMS) continue;
            float g = 0.f;
            if (pidx < OFF_B1) {
                int n = pidx / MLP_IN, c = pidx - n * MLP_IN;
                for (int r = 0; r < GT; ++r) g = fmaf(S.dz1[r][n], S.x[r][c], g);
            } else if (pidx < OFF_W2) {
                int n = pidx - OFF_B1;
                for (int r = 0; r < GT; ++r) g += S.dz1[r][n];
            } else if (pidx < OFF_B2) {
                int q = pidx - OFF_W2, n = q / MLP_H, c = q - n * MLP_H;
                for (int r = 0; r < GT; ++r) g = fmaf(S.dz2[r][n], S.h1[r][c], g);
            } else if (pidx < OFF_W3) {
                int n = pidx - OFF_B2;
                for (int r = 0; r < GT; ++r) g += S.dz2[r][n];
            } else if (pidx < OFF_B3) {
                int q = pidx - OFF_W3, o = q / MLP_H, c = q - o * MLP_H;
                for (int r = 0; r < GT; ++r) g = fmaf(S.dout[r][o], S.h2[r][c], g);
            } else {
                int o = pidx - OFF_B3;
                for (int r = 0; r < GT; ++r) g += S.dout[r][o];
            }
            acc[j] += g;
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < GPER; ++j) {
        const int pidx = tid + j * GTHREADS;
        if (pidx < MLP_PARAMS) partial[(long long)blockIdx.x * MLP_PARAMS + pidx] = acc[j];
    }
    if (tid == 0) partial_loss[blockIdx.x] = lsum;
}

// grad[i] = sum over blocks of partial[b][i] in block order; loss likewise (divided by rows).
__global__ void k_mlp_reduce(const float *partial, const float *partial_loss, int nblocks, long long rows, float *grad,
                             float *loss)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_PARAMS) {
        float g = 0.f;
        for (int b = 0; b < nblocks; ++b) g += partial[(long long)b * MLP_PARAMS + i];
        grad[i] = g;
    }
    if (i == 0 && loss) {
        float l = 0.f;
        for (int b = 0; b < nblocks; ++b) l += partial_loss[b];
        *loss = l / (float)rows;
    }
}

// Adam step t (bias corrections bc1 = 1 - beta1^t, bc2 = 1 - beta2^t from the host).
__global__ void k_mlp_adam(float *master, const float *grad, float *m, float *v, int n, float lr, float beta1,
                           float beta2, float eps, float bc1, float bc2, unsigned short *wbf16)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float g = grad[i];
    float mi = beta1 * m[i] + (1.f - beta1) * g;
    float vi = beta2 * v[i] + (1.f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    float mh = mi / bc1, vh = vi / bc2;
    float p = master[i] - lr * mh / (sqrtf(vh) + eps);
    master[i] = p;
    if (wbf16) wbf16[i] = __bfloat16_as_ushort(__float2bfloat16_rn(p));
}

}  // namespace kd
