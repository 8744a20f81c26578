// The learned proposal's network on the fifth-generation tensor cores (tcgen05): a
// batch of rows goes through the three layers as dense products, 128 rows per tile,
// operands staged in shared memory, accumulators in tensor memory (TMEM).
//
// Precision.  The weights are BF16 already, so a layer's product W x is exact in FP32
// once x is: every activation x is written as hi + lo, two BF16 values (hi = x rounded
// to BF16, lo = the rest rounded again), |x - hi - lo| <= 2^-16 |x|, and the layer is
// two BF16 products accumulated in FP32 (x_hi W^T + x_lo W^T).  A layer's error is
// then at most about 2^-16 of sum_k |w_k| |x_k| plus the FP32 accumulation; the
// bias, the ReLU and the next split run per row in FP32 on the CUDA cores.
//
// One CTA of 128 threads per tile (a persistent loop over tiles): thread r owns row r
// of the tile, which is TMEM lane r of every accumulator (M = 128).  One elected
// thread issues the MMAs and commits them to an mbarrier; every wait is bounded
// (about a second), after which the CTA counts the failure (*fails), leaves its
// results marked (NaN outputs, no guesses), frees its TMEM and returns.
//
//   k_mlp_tc<0>   outputs of rows x (rows x 32 FP32) to out (rows x 18),
//   k_mlp_tc<1>   the step planner's form: the features k_plan wrote for each move,
//                 the guess (argmax of the 17 slot logits, lowest index on ties) to
//                 pguess[point] and the predicted cavity size to its partition's cost.
#pragma once
#include <cuda_bf16.h>

namespace kd {

// ---------------------------------------------------------------- primitives

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor for an operand tile in the canonical K-major layout
// without swizzling: core matrices of 8 rows x 16 bytes (128 contiguous bytes), `lbo`
// bytes between core matrices adjacent along K, `sbo` bytes between groups of 8 rows.
// Fields: start address >> 4 (bits 0-13), lbo >> 4 (16-29), sbo >> 4 (32-45), the
// descriptor version 1 (bits 46-48), base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ unsigned long long tc_sdesc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B
// (bits 7-9 and 10-12 = 1), dense, no negation, both operands K-major (bits 15, 16 =
// 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr unsigned tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

// D (TMEM) = A B^T (+ D when acc): A M x 16, B N x 16, BF16, issued by one thread.
__device__ __forceinline__ void tc_mma(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// The mbarrier at `bar` receives one arrival when every MMA this thread issued so far
// has completed.
__device__ __forceinline__ void tc_commit(unsigned bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor cores' reads
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// whole warp: allocate `cols` TMEM columns (a power of two >= 32), address to smem
__device__ __forceinline__ void tmem_alloc(unsigned dst, unsigned cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(unsigned taddr, unsigned cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (the warp's 32 lanes), the
// load completed before the values are used.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float *v)
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` to complete; false after about 2^31 cycles.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity)
{
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) return false;
        __nanosleep(64);
    }
    return true;
}

// Eight FP32 values as BF16 hi and lo parts (x = hi + lo + O(2^-16 x)), each packed
// into 16 bytes in element order.
__device__ __forceinline__ void split8(const float *v, uint4 &hi, uint4 &lo)
{
    unsigned h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat16 a0 = __float2bfloat16_rn(v[2 * i]), a1 = __float2bfloat16_rn(v[2 * i + 1]);
        const __nv_bfloat16 b0 = __float2bfloat16_rn(v[2 * i] - __bfloat162float(a0));
        const __nv_bfloat16 b1 = __float2bfloat16_rn(v[2 * i + 1] - __bfloat162float(a1));
        h[i] = (unsigned)__bfloat16_as_ushort(a0) | ((unsigned)__bfloat16_as_ushort(a1) << 16);
        l[i] = (unsigned)__bfloat16_as_ushort(b0) | ((unsigned)__bfloat16_as_ushort(b1) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Byte offset of BF16 element (r, k) in a K-major tile of K columns (K a multiple of
// 8): core matrix (r / 8, k / 8) at (r / 8) * 16K + (k / 8) * 128, so lbo = 128 and
// sbo = 16K.
__host__ __device__ constexpr unsigned tc_off(int r, int k, int K)
{
    return (unsigned)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// ---------------------------------------------------------------- the network

constexpr int TC_M = 128;        // rows per tile = TMEM lanes = threads
constexpr int TC_N3 = 32;        // the 18 outputs padded to a multiple of 16 (N of layer 3)
constexpr unsigned TC_COLS = 128;  // TMEM columns: layer 1 at 0-63, layer 2 at 64-127, layer 3 at 0-31
// shared-memory layout (bytes from a 1024-aligned base)
constexpr unsigned TCS_W1 = 0;                                  // B of layer 1: 64 x 32
constexpr unsigned TCS_W2 = TCS_W1 + MLP_H * MLP_IN * 2;        // B of layer 2: 64 x 64
constexpr unsigned TCS_W3 = TCS_W2 + MLP_H * MLP_H * 2;         // B of layer 3: 32 x 64 (rows >= 18 zero)
constexpr unsigned TCS_XH = TCS_W3 + TC_N3 * MLP_H * 2;         // A of layer 1, hi and lo: 128 x 32
constexpr unsigned TCS_XL = TCS_XH + TC_M * MLP_IN * 2;
constexpr unsigned TCS_HH = TCS_XL + TC_M * MLP_IN * 2;         // A of layers 2 and 3: 128 x 64
constexpr unsigned TCS_HL = TCS_HH + TC_M * MLP_H * 2;
constexpr unsigned TCS_BIAS = TCS_HL + TC_M * MLP_H * 2;        // b1, b2, b3 as FP32 (160 floats)
constexpr unsigned TCS_BAR = TCS_BIAS + 160 * 4;                // the mbarrier
constexpr unsigned TCS_TMEM = TCS_BAR + 8;                      // the TMEM base address
constexpr unsigned TCS_BYTES = TCS_TMEM + 8 + 1024;             // + alignment of the base
static_assert(TCS_BAR % 8 == 0, "mbarrier alignment");
static_assert(TCS_HL + TC_M * MLP_H * 2 <= (1u << 18), "descriptor address range");

// Row `row` (K values as BF16 bit patterns at src, 4-byte aligned) of a weight matrix
// into a K-major B tile.
__device__ __forceinline__ void tc_stage_wrow(unsigned char *tile, const unsigned short *src, int row, int K)
{
    const unsigned *s32 = reinterpret_cast<const unsigned *>(src);
    for (int j = 0; j < K / 8; ++j) {
        uint4 c = make_uint4(__ldg(s32 + 4 * j), __ldg(s32 + 4 * j + 1), __ldg(s32 + 4 * j + 2), __ldg(s32 + 4 * j + 3));
        *reinterpret_cast<uint4 *>(tile + tc_off(row, 8 * j, K)) = c;
    }
}

// 16 values of this thread's row as hi / lo chunks at column c0 of the K-column A tiles.
__device__ __forceinline__ void tc_put16(unsigned char *S, unsigned hiofs, unsigned loofs, int r, int c0, int K,
                                         const float *v)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint4 a, b;
        split8(v + 8 * h, a, b);
        *reinterpret_cast<uint4 *>(S + hiofs + tc_off(r, c0 + 8 * h, K)) = a;
        *reinterpret_cast<uint4 *>(S + loofs + tc_off(r, c0 + 8 * h, K)) = b;
    }
}

// All threads: shared-memory writes visible to the tensor cores, TMEM reads before this
// point ordered before MMAs issued after it.
__device__ __forceinline__ void tc_handoff()
{
    fence_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// One layer on the tensor cores: D = A_hi B^T + A_lo B^T over K (multiple of 16), one
// thread issuing; the commit arrives on `bar`.
__device__ __forceinline__ void tc_layer(unsigned d, unsigned ahi, unsigned alo, unsigned b, int K, unsigned idesc,
                                         unsigned bar)
{
    const unsigned sbo = (unsigned)K * 16;
#pragma unroll 1
    for (int s = 0; s < K / 16; ++s) {
        const unsigned long long bd = tc_sdesc(b + 256u * s, 128, sbo);
        tc_mma(d, tc_sdesc(ahi + 256u * s, 128, sbo), bd, idesc, s > 0);
        tc_mma(d, tc_sdesc(alo + 256u * s, 128, sbo), bd, idesc, 1);
    }
    tc_commit(bar);
}

template <int MODE>
__global__ void __launch_bounds__(TC_M) k_mlp_tc(const unsigned short *w, const float *x, long long rows,
                                                 const int *ctl_rows, float *out, const int *ppart,
                                                 const int3 *gmoves, signed char *pguess, float *pcost,
                                                 unsigned long long *fails)
{
    extern __shared__ unsigned char tc_raw[];
    unsigned char *S = tc_raw + ((1024u - (smem_addr(tc_raw) & 1023u)) & 1023u);
    if (ctl_rows) rows = __ldcg(ctl_rows);
    const long long ntiles = (rows + TC_M - 1) / TC_M;
    if ((long long)blockIdx.x >= ntiles) return;  // uniform per block, before any barrier
    const int tid = threadIdx.x, warp = tid >> 5;
    const unsigned base = smem_addr(S), bar = base + TCS_BAR;
    float *bias = reinterpret_cast<float *>(S + TCS_BIAS);
    if (warp == 0) tmem_alloc(base + TCS_TMEM, TC_COLS);
    if (tid == 0) mbar_init(bar, 1);
    // weights (B operands, row = output unit) and biases, once per CTA
    if (tid < MLP_H) {
        tc_stage_wrow(S + TCS_W1, w + OFF_W1 + tid * MLP_IN, tid, MLP_IN);
        tc_stage_wrow(S + TCS_W2, w + OFF_W2 + tid * MLP_H, tid, MLP_H);
        bias[tid] = __uint_as_float((unsigned)__ldg(w + OFF_B1 + tid) << 16);
        bias[64 + tid] = __uint_as_float((unsigned)__ldg(w + OFF_B2 + tid) << 16);
    } else if (tid < MLP_H + TC_N3) {
        const int o = tid - MLP_H;
        if (o < MLP_OUT) {
            tc_stage_wrow(S + TCS_W3, w + OFF_W3 + o * MLP_H, o, MLP_H);
            bias[128 + o] = __uint_as_float((unsigned)__ldg(w + OFF_B3 + o) << 16);
        } else {
            for (int j = 0; j < MLP_H / 8; ++j)
                *reinterpret_cast<uint4 *>(S + TCS_W3 + tc_off(o, 8 * j, MLP_H)) = make_uint4(0, 0, 0, 0);
            bias[128 + o] = 0.f;
        }
    }
    tc_handoff();
    const unsigned t0 = *reinterpret_cast<volatile unsigned *>(S + TCS_TMEM);
    const unsigned trow = t0 + ((unsigned)(warp * 32) << 16);  // this warp's 32 lanes
    const unsigned ID64 = tc_idesc(TC_M, MLP_H), ID32 = tc_idesc(TC_M, TC_N3);
    unsigned phase = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long g = tile * TC_M + tid;  // this thread's row
        bool live = g < rows;
        if (MODE == 1 && live) live = __ldcg(ppart + g) >= 0;
        {
            float v[MLP_IN];
#pragma unroll
            for (int c = 0; c < MLP_IN; ++c) v[c] = live ? __ldcg(x + g * MLP_IN + c) : 0.f;
            tc_put16(S, TCS_XH, TCS_XL, tid, 0, MLP_IN, v);
            tc_put16(S, TCS_XH, TCS_XL, tid, 16, MLP_IN, v + 16);
        }
        tc_handoff();
        // layer 1: 128 x 64 at columns 0..63
        if (tid == 0) tc_layer(t0, base + TCS_XH, base + TCS_XL, base + TCS_W1, MLP_IN, ID64, bar);
        ok = __syncthreads_and(mbar_wait_bounded(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
#pragma unroll 1
        for (int c0 = 0; c0 < MLP_H; c0 += 16) {
            float v[16];
            tmem_ld16(trow + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + bias[c0 + j], 0.f);
            tc_put16(S, TCS_HH, TCS_HL, tid, c0, MLP_H, v);
        }
        tc_handoff();
        // layer 2: 128 x 64 at columns 64..127
        if (tid == 0) tc_layer(t0 + 64, base + TCS_HH, base + TCS_HL, base + TCS_W2, MLP_H, ID64, bar);
        ok = __syncthreads_and(mbar_wait_bounded(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
#pragma unroll 1
        for (int c0 = 0; c0 < MLP_H; c0 += 16) {
            float v[16];
            tmem_ld16(trow + 64 + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + bias[64 + c0 + j], 0.f);
            tc_put16(S, TCS_HH, TCS_HL, tid, c0, MLP_H, v);  // layer 2 has read h1
        }
        tc_handoff();
        // layer 3: 128 x 32 at columns 0..31 (layer 1's values were read)
        if (tid == 0) tc_layer(t0, base + TCS_HH, base + TCS_HL, base + TCS_W3, MLP_H, ID32, bar);
        ok = __syncthreads_and(mbar_wait_bounded(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
        float o[TC_N3];
        tmem_ld16(trow, o);
        tmem_ld16(trow + 16, o + 16);
#pragma unroll
        for (int j = 0; j < MLP_OUT; ++j) o[j] += bias[128 + j];
        if (live) {
            if (MODE == 0) {
#pragma unroll
                for (int j = 0; j < MLP_OUT; ++j) out[g * MLP_OUT + j] = o[j];
            } else {
                int best = 0;
                float bv = o[0];
#pragma unroll
                for (int j = 1; j < MLP_SLOTS; ++j)
                    if (o[j] > bv) {
                        bv = o[j];
                        best = j;
                    }
                pguess[gmoves[g].x] = (signed char)best;
                if (pcost) atomicAdd(pcost + __ldcg(ppart + g), exp2f(fminf(fmaxf(o[MLP_SLOTS], 0.f), 10.f)));
            }
        }
        tc_fence_before();
        __syncthreads();  // this tile's TMEM reads before the next tile's MMAs
        tc_fence_after();
    }
    if (!ok) {
        if (tid == 0) atomicAdd(fails, 1ull);
        if (MODE == 0)  // every row of this CTA's tiles marked
            for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                const long long g = tile * TC_M + tid;
                if (g < rows)
                    for (int j = 0; j < MLP_OUT; ++j) out[g * MLP_OUT + j] = __int_as_float(0x7fc00000);
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_free(t0, TC_COLS);
    }
}

}  // namespace kd

namespace kd {

// ---------------------------------------------------------------- training

// Forward + backward of the mean loss of k_mlp_grad on the tensor cores, 128 rows per
// tile, one CTA per SM looping over tiles.  Per tile: the three layers forward, then
// back through layer 3 (dH2 = dOut W3) and layer 2 (dH1 = dZ2 W2), each with the
// activations split into three BF16 parts (hi + mid + lo, to 2^-24 of |x|) against the
// exact BF16 weights: a split into two leaves pre-activations near zero on the other
// side of the ReLU often enough to move the weight gradients by about 1e-2 of their
// size, three keep them within FP32 rounding.  Then the tile's weight gradients,
// summed over its rows, are added to two accumulators that stay in TMEM over all the
// CTA's tiles:
//   G_a [128 x 112] += [dZ1 | dZ2]^T [X | H1 | 1]: rows 0-63 hold gW1 (columns 0-31)
//                      and gb1 (column 96), rows 64-127 gW2 (columns 32-95) and gb2;
//   G_b [128 x 32]  += [H2_hi | H2_lo]^T dOut: gW3^T = rows 0-63 + rows 64-127.
// In these two the rows of the batch are the contraction dimension, so their operands
// are read in the MN-major layout from the same tiles the row-wise products read
// K-major.  A product of two FP32 operands takes three BF16 products (hi hi + hi lo +
// lo hi, with hi and mid as the two parts; G_b's A holds them as separate rows, so it
// takes two).  gb3 and the loss
// are summed on the CUDA cores in a fixed order, so the result repeats bit for bit.
// Block b writes partial[b][.] and partial_loss[b] as k_mlp_grad does.

// tiles (bytes from a 1024-aligned base); the column count of each sets its row stride
constexpr unsigned TG_DZH = 0;                 // [dZ1 | dZ2] 128 x 128, hi
constexpr unsigned TG_DZL = TG_DZH + 32768;    // ... mid
constexpr unsigned TG_XH = TG_DZL + 32768;     // [X | H1 | 1 0 ... 0] 128 x 112, hi
constexpr unsigned TG_XL = TG_XH + 28672;      // ... mid (the constant columns zero)
constexpr unsigned TG_H2 = TG_XL + 28672;      // [H2 hi | H2 mid] 128 x 128
constexpr unsigned TG_DOH = TG_H2 + 32768;     // dOut 128 x 32 (columns 18-31 zero), hi
constexpr unsigned TG_DOL = TG_DOH + 8192;     // ... mid
constexpr unsigned TG_LO = TG_DOL + 8192;      // the lo parts of the current product's A: 128 x 64
constexpr unsigned TG_W1 = TG_LO + 16384;      // B of layer 1: 64 x 32
constexpr unsigned TG_W2 = TG_W1 + 4096;       // B of layer 2: 64 x 64
constexpr unsigned TG_W3 = TG_W2 + 8192;       // B of layer 3: 32 x 64 (rows >= 18 zero)
constexpr unsigned TG_W3T = TG_W3 + 4096;      // B of dH2 = dOut W3: 64 x 32, (u, o) = W3[o][u]
constexpr unsigned TG_W2T = TG_W3T + 4096;     // B of dH1 = dZ2 W2: 64 x 64, (c, u) = W2[u][c]
constexpr unsigned TG_BIAS = TG_W2T + 8192;    // b1, b2, b3 (160 floats)
constexpr unsigned TG_RED = TG_BIAS + 640;     // per warp: 18 column sums of dOut, the loss (4 x 20 floats)
constexpr unsigned TG_BAR = TG_RED + 320;
constexpr unsigned TG_TMEM = TG_BAR + 8;
constexpr unsigned TG_BYTES = TG_TMEM + 8 + 1024;
constexpr unsigned TG_COLS = 256;              // TMEM: products at 0-63, G_a at 64-175, G_b at 176-207
constexpr unsigned TG_GA = 64, TG_GB = 176;
static_assert(TG_BAR % 8 == 0 && TG_BYTES <= 227 * 1024, "training tile layout");

// D = A B^T for an A and a B both read K-major: K / 16 steps of three MMAs (A's hi,
// mid and lo parts against B); hi and mid rows `asbo` bytes apart per 8, lo rows 1024
// (the 64-column lo tile), B's `bsbo`.
__device__ __forceinline__ void tc_rows(unsigned d, unsigned ahi, unsigned amid, unsigned asbo, unsigned alo,
                                        unsigned b, unsigned bsbo, int K, unsigned idesc)
{
#pragma unroll 1
    for (int s = 0; s < K / 16; ++s) {
        const unsigned long long bd = tc_sdesc(b + 256u * s, 128, bsbo);
        tc_mma(d, tc_sdesc(ahi + 256u * s, 128, asbo), bd, idesc, s > 0);
        tc_mma(d, tc_sdesc(amid + 256u * s, 128, asbo), bd, idesc, 1);
        tc_mma(d, tc_sdesc(alo + 256u * s, 128, 1024), bd, idesc, 1);
    }
}

// Sixteen values of this thread's row split into hi, mid and lo BF16 parts: hi and mid
// at column c0 of the K-column tiles at hiofs / midofs, lo at column c0 - lo0 of the
// 64-column lo tile.
__device__ __forceinline__ void tc_put16x3(unsigned char *S, unsigned hiofs, unsigned midofs, int r, int c0, int K,
                                           int lo0, const float *v)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float rest[8];
        uint4 a, b, c, unused;
        split8(v + 8 * h, a, b);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const unsigned wa = (&a.x)[i >> 1], wb = (&b.x)[i >> 1];
            const float fa = __uint_as_float((i & 1 ? wa & 0xffff0000u : wa << 16));
            const float fb = __uint_as_float((i & 1 ? wb & 0xffff0000u : wb << 16));
            rest[i] = (v[8 * h + i] - fa) - fb;  // exact: what hi + mid leave
        }
        split8(rest, c, unused);
        *reinterpret_cast<uint4 *>(S + hiofs + tc_off(r, c0 + 8 * h, K)) = a;
        *reinterpret_cast<uint4 *>(S + midofs + tc_off(r, c0 + 8 * h, K)) = b;
        *reinterpret_cast<uint4 *>(S + TG_LO + tc_off(r, c0 - lo0 + 8 * h, 64)) = c;
    }
}

// the instruction descriptor with both operands MN-major
__host__ __device__ constexpr unsigned tc_idesc_mn(int M, int N) { return tc_idesc(M, N) | (1u << 15) | (1u << 16); }

// MN-major descriptor of a tile whose rows (the contraction dimension here) are
// `rs` bytes apart per 8: core matrices adjacent along K are rs apart (lbo), along
// M / N 128 bytes (sbo).
__device__ __forceinline__ unsigned long long tc_mn(unsigned addr, unsigned rs) { return tc_sdesc(addr, rs, 128); }

__global__ void __launch_bounds__(TC_M) k_mlp_grad_tc(const unsigned short *w, const float *x, const int *labels,
                                                      const long long *idx, long long rows, float lam,
                                                      float *partial, float *partial_loss,
                                                      unsigned long long *fails)
{
    extern __shared__ unsigned char tc_raw[];
    unsigned char *S = tc_raw + ((1024u - (smem_addr(tc_raw) & 1023u)) & 1023u);
    const long long ntiles = (rows + TC_M - 1) / TC_M;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned base = smem_addr(S), bar = base + TG_BAR;
    float *bias = reinterpret_cast<float *>(S + TG_BIAS);
    float *red = reinterpret_cast<float *>(S + TG_RED);
    if (warp == 0) tmem_alloc(base + TG_TMEM, TG_COLS);
    if (tid == 0) mbar_init(bar, 1);
    // weights: the forward B operands (row = output unit) and the two transposed ones
    if (tid < MLP_H) {
        tc_stage_wrow(S + TG_W1, w + OFF_W1 + tid * MLP_IN, tid, MLP_IN);
        tc_stage_wrow(S + TG_W2, w + OFF_W2 + tid * MLP_H, tid, MLP_H);
        bias[tid] = __uint_as_float((unsigned)__ldg(w + OFF_B1 + tid) << 16);
        bias[64 + tid] = __uint_as_float((unsigned)__ldg(w + OFF_B2 + tid) << 16);
        // W2T row c = tid: (c, u) = W2[u][c]; W3T row u = tid: (u, o) = W3[o][u]
        for (int j = 0; j < MLP_H / 8; ++j) {
            unsigned short e[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) e[i] = __ldg(w + OFF_W2 + (8 * j + i) * MLP_H + tid);
            *reinterpret_cast<uint4 *>(S + TG_W2T + tc_off(tid, 8 * j, MLP_H)) =
                make_uint4(e[0] | (unsigned)e[1] << 16, e[2] | (unsigned)e[3] << 16, e[4] | (unsigned)e[5] << 16,
                           e[6] | (unsigned)e[7] << 16);
        }
        for (int j = 0; j < TC_N3 / 8; ++j) {
            unsigned short e[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int o = 8 * j + i;
                e[i] = o < MLP_OUT ? __ldg(w + OFF_W3 + o * MLP_H + tid) : (unsigned short)0;
            }
            *reinterpret_cast<uint4 *>(S + TG_W3T + tc_off(tid, 8 * j, TC_N3)) =
                make_uint4(e[0] | (unsigned)e[1] << 16, e[2] | (unsigned)e[3] << 16, e[4] | (unsigned)e[5] << 16,
                           e[6] | (unsigned)e[7] << 16);
        }
    } else if (tid < MLP_H + TC_N3) {
        const int o = tid - MLP_H;
        if (o < MLP_OUT) {
            tc_stage_wrow(S + TG_W3, w + OFF_W3 + o * MLP_H, o, MLP_H);
            bias[128 + o] = __uint_as_float((unsigned)__ldg(w + OFF_B3 + o) << 16);
        } else {
            for (int j = 0; j < MLP_H / 8; ++j)
                *reinterpret_cast<uint4 *>(S + TG_W3 + tc_off(o, 8 * j, MLP_H)) = make_uint4(0, 0, 0, 0);
            bias[128 + o] = 0.f;
        }
    }
    // the constant columns 96-111 of [X | H1 | 1]: a one in column 96 (hi), zeros
    {
        const uint4 one = make_uint4(0x3F80u, 0, 0, 0), zero = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4 *>(S + TG_XH + tc_off(tid, 96, 112)) = one;
        *reinterpret_cast<uint4 *>(S + TG_XH + tc_off(tid, 104, 112)) = zero;
        *reinterpret_cast<uint4 *>(S + TG_XL + tc_off(tid, 96, 112)) = zero;
        *reinterpret_cast<uint4 *>(S + TG_XL + tc_off(tid, 104, 112)) = zero;
    }
    tc_handoff();
    const unsigned t0 = *reinterpret_cast<volatile unsigned *>(S + TG_TMEM);
    const unsigned trow = t0 + ((unsigned)(warp * 32) << 16);
    const unsigned ID64 = tc_idesc(TC_M, MLP_H), ID32 = tc_idesc(TC_M, TC_N3);
    const unsigned IDA = tc_idesc_mn(TC_M, 112), IDB = tc_idesc_mn(TC_M, TC_N3);
    const float inv_rows = 1.0f / (float)rows;
    unsigned phase = 0;
    bool ok = true, first = true;
    float lsum = 0.f, gb3 = 0.f;  // (gb3: thread o < 18)
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long g = tile * TC_M + tid;
        const bool live = g < rows;
        const long long row = live ? (idx ? idx[g] : g) : 0;
        {
            float v[MLP_IN];
#pragma unroll
            for (int c = 0; c < MLP_IN; ++c) v[c] = live ? __ldg(x + row * MLP_IN + c) : 0.f;
            tc_put16x3(S, TG_XH, TG_XL, tid, 0, 112, 0, v);
            tc_put16x3(S, TG_XH, TG_XL, tid, 16, 112, 0, v + 16);
        }
        tc_handoff();
        // layer 1 -> columns 0-63; h1 into columns 32-95 of [X | H1 | 1]
        if (tid == 0) {
            tc_rows(t0, base + TG_XH, base + TG_XL, 1792, base + TG_LO, base + TG_W1, 512, MLP_IN, ID64);
            tc_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait_bounded(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
        unsigned long long m1 = 0, m2 = 0;  // ReLU masks of this row
#pragma unroll 1
        for (int c0 = 0; c0 < MLP_H; c0 += 16) {
            float v[16];
            tmem_ld16(trow + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float z = v[j] + bias[c0 + j];
                if (z > 0.f) m1 |= 1ull << (c0 + j);
                v[j] = fmaxf(z, 0.f);
            }
            tc_put16x3(S, TG_XH, TG_XL, tid, 32 + c0, 112, 32, v);
        }
        tc_handoff();
        // layer 2 -> columns 0-63; h2 into [H2 hi | H2 lo]
        if (tid == 0) {
            tc_rows(t0, base + TG_XH + 512, base + TG_XL + 512, 1792, base + TG_LO, base + TG_W2, 1024, MLP_H, ID64);
            tc_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait_bounded(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
#pragma unroll 1
        for (int c0 = 0; c0 < MLP_H; c0 += 16) {
            float v[16];
            tmem_ld16(trow + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float z = v[j] + bias[64 + c0 + j];
                if (z > 0.f) m2 |= 1ull << (c0 + j);
                v[j] = fmaxf(z, 0.f);
            }
            tc_put16x3(S, TG_H2, TG_H2 + 1024, tid, c0, 128, 0, v);
        }
        tc_handoff();
        // layer 3 -> columns 0-31; the loss and dOut of this row
        if (tid == 0) {
            tc_rows(t0, base + TG_H2, base + TG_H2 + 1024, 2048, base + TG_LO, base + TG_W3, 1024, MLP_H, ID32);
            tc_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait_bounded(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
        float o[TC_N3];
        tmem_ld16(trow, o);
        tmem_ld16(trow + 16, o + 16);
        float loss = 0.f;
        if (live) {
#pragma unroll
            for (int j = 0; j < MLP_OUT; ++j) o[j] += bias[128 + j];
            const int slot = labels[2 * row];
            const float target = log2f((float)labels[2 * row + 1]);
            float mx = o[0];
#pragma unroll
            for (int j = 1; j < MLP_SLOTS; ++j) mx = fmaxf(mx, o[j]);
            float se = 0.f;
#pragma unroll
            for (int j = 0; j < MLP_SLOTS; ++j) se += expf(o[j] - mx);
            const float lse = mx + logf(se);
            const float res = o[MLP_SLOTS] - target;
            float oslot = 0.f;
#pragma unroll
            for (int j = 0; j < MLP_SLOTS; ++j)
                if (j == slot) oslot = o[j];
            loss = (lse - oslot) + lam * res * res;
#pragma unroll
            for (int j = 0; j < MLP_SLOTS; ++j) o[j] = (expf(o[j] - lse) - (j == slot ? 1.f : 0.f)) * inv_rows;
            o[MLP_SLOTS] = 2.f * lam * res * inv_rows;
        } else {
#pragma unroll
            for (int j = 0; j < MLP_OUT; ++j) o[j] = 0.f;
        }
#pragma unroll
        for (int j = MLP_OUT; j < TC_N3; ++j) o[j] = 0.f;
        tc_put16x3(S, TG_DOH, TG_DOL, tid, 0, TC_N3, 0, o);
        tc_put16x3(S, TG_DOH, TG_DOL, tid, 16, TC_N3, 0, o + 16);
        // the tile's gb3 and loss: per warp by a fixed shuffle tree, then warps in order
#pragma unroll
        for (int j = 0; j < MLP_OUT; ++j) {
            float v = o[j];
#pragma unroll
            for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) red[warp * 20 + j] = v;
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, off);
        if (lane == 0) red[warp * 20 + 18] = loss;
        tc_handoff();
        if (tid < MLP_OUT) gb3 += ((red[tid] + red[20 + tid]) + red[40 + tid]) + red[60 + tid];
        if (tid == 0) lsum += ((red[18] + red[38]) + red[58]) + red[78];
        // dH2 = dOut W3 -> columns 0-63; dZ2 into columns 64-127 of [dZ1 | dZ2]
        if (tid == 0) {
            tc_rows(t0, base + TG_DOH, base + TG_DOL, 512, base + TG_LO, base + TG_W3T, 512, TC_N3, ID64);
            tc_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait_bounded(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
#pragma unroll 1
        for (int c0 = 0; c0 < MLP_H; c0 += 16) {
            float v[16];
            tmem_ld16(trow + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = (m2 >> (c0 + j)) & 1ull ? v[j] : 0.f;
            tc_put16x3(S, TG_DZH, TG_DZL, tid, 64 + c0, 128, 64, v);
        }
        tc_handoff();
        // dH1 = dZ2 W2 -> columns 0-63; dZ1 into columns 0-63 of [dZ1 | dZ2]
        if (tid == 0) {
            tc_rows(t0, base + TG_DZH + 1024, base + TG_DZL + 1024, 2048, base + TG_LO, base + TG_W2T, 1024, MLP_H,
                    ID64);
            tc_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait_bounded(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
#pragma unroll 1
        for (int c0 = 0; c0 < MLP_H; c0 += 16) {
            float v[16];
            tmem_ld16(trow + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = (m1 >> (c0 + j)) & 1ull ? v[j] : 0.f;
            tc_put16(S, TG_DZH, TG_DZL, tid, c0, 128, v);
        }
        tc_handoff();
        // the tile's weight gradients into G_a and G_b (rows of the tile = K, 8 steps)
        if (tid == 0) {
#pragma unroll 1
            for (int s = 0; s < TC_M / 16; ++s) {
                const unsigned acc = first && s == 0 ? 0u : 1u;
                const unsigned long long ah = tc_mn(base + TG_DZH + 4096u * s, 2048);
                const unsigned long long al = tc_mn(base + TG_DZL + 4096u * s, 2048);
                const unsigned long long bh = tc_mn(base + TG_XH + 3584u * s, 1792);
                const unsigned long long bl = tc_mn(base + TG_XL + 3584u * s, 1792);
                tc_mma(t0 + TG_GA, ah, bh, IDA, acc);
                tc_mma(t0 + TG_GA, ah, bl, IDA, 1);
                tc_mma(t0 + TG_GA, al, bh, IDA, 1);
                const unsigned long long h2 = tc_mn(base + TG_H2 + 4096u * s, 2048);
                tc_mma(t0 + TG_GB, h2, tc_mn(base + TG_DOH + 1024u * s, 512), IDB, acc);
                tc_mma(t0 + TG_GB, h2, tc_mn(base + TG_DOL + 1024u * s, 512), IDB, 1);
            }
            tc_commit(bar);
        }
        first = false;
        ok = __syncthreads_and(mbar_wait_bounded(bar, phase));  // before the tiles are rewritten
        phase ^= 1;
        if (!ok) break;
        tc_fence_after();
    }
    if (ok) {
        float *out = partial + (long long)blockIdx.x * MLP_PARAMS;
        float *tmp = reinterpret_cast<float *>(S + TG_DZH);  // the tiles are free now
        if (first) {  // no tile: zero gradients
            for (int i = tid; i < MLP_PARAMS; i += TC_M) out[i] = 0.f;
        } else {
            float v[16];
            // G_a row tid: gW1 / gb1 (rows 0-63) or gW2 / gb2 (rows 64-127)
            const int u = tid & 63;
#pragma unroll 1
            for (int c0 = 0; c0 < 112; c0 += 16) {
                tmem_ld16(trow + TG_GA + c0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = c0 + j;
                    if (tid < 64) {
                        if (c < MLP_IN) out[OFF_W1 + u * MLP_IN + c] = v[j];
                    } else if (c >= 32 && c < 96) {
                        out[OFF_W2 + u * MLP_H + (c - 32)] = v[j];
                    }
                    if (c == 96) out[(tid < 64 ? OFF_B1 : OFF_B2) + u] = v[j];
                }
            }
            // G_b: gW3[o][u] = row u + row 64 + u
            float gbv[TC_N3];
            tmem_ld16(trow + TG_GB, gbv);
            tmem_ld16(trow + TG_GB + 16, gbv + 16);
            if (tid >= 64)
                for (int j = 0; j < MLP_OUT; ++j) tmp[u * MLP_OUT + j] = gbv[j];
            __syncthreads();
            if (tid < 64)
                for (int j = 0; j < MLP_OUT; ++j) out[OFF_W3 + j * MLP_H + u] = gbv[j] + tmp[u * MLP_OUT + j];
            if (tid < MLP_OUT) out[OFF_B3 + tid] = gb3;
        }
        if (tid == 0) partial_loss[blockIdx.x] = lsum;
    } else {  // the gradient and the loss marked NaN
        for (int i = tid; i < MLP_PARAMS; i += TC_M) partial[(long long)blockIdx.x * MLP_PARAMS + i] = __int_as_float(0x7fc00000);
        if (tid == 0) {
            partial_loss[blockIdx.x] = __int_as_float(0x7fc00000);
            atomicAdd(fails, 1ull);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_free(t0, TG_COLS);
    }
}

}  // namespace kd
