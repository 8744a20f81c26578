// Kernels of the kinetic Delaunay library.  Included once, by kdt.cu.
//
//   step:    k_intake_link -> k_kinetic (last warp: deferred points, certification of
//            global-path writes) (-> k_fixup / k_certify until no violation)
//   build:   k_range / k_bbox -> k_hilbert -> scan -> k_place_order -> k_third -> k_init
//            -> k_insert_level (one launch per level) -> k_certify_all (-> k_fixup ...)
//   export:  k_exp_count -> scan -> k_exp_place -> k_exp_sortseg
#pragma once
#include "kdt_local.cuh"

namespace kd {

constexpr int WPB = 4;  // warps per block of the warp-per-item kernels
constexpr int DEV_DUP_ID = 10;  // a move id repeated within one step (found at intake)
constexpr int DEV_FAR = 11;     // a move went farther than the rebuild rule allows (found at intake):
                                // not an error; the step is done as a rebuild

// small device block of scalars
enum Slot : int {
    S_STATUS = 0, S_DIRTY = 1, S_VIOL = 2, S_TRIS = 3, S_DEFER = 4, S_THIRD = 5,
    S_MINX = 6, S_MINY = 7, S_MAXX = 8, S_MAXY = 9, S_TOTAL = 10, S_BAD = 11, S_ALIVE = 12,
    S_WRAPS = 13, S_FAILPT = 14, S_DONE = 15, S_CERTPEND = 16, S_TICKET = 17, S_DNEXT = 18,
    S_DRUN = 19,  // warps running a move taken from the deferred list (kinetic launch)
    S_FAR = 20,   // moves beyond the displacement rule's bound (intake)
    S_NCELLS = 21, // partitions of this step (quad-tree re-divided at every step)
    S_NUM = 22
};

// Instance tables (one instance for kdt_build; many for kdt_build_batch).  Every
// instance is its own triangulation in one shared store: global point ids
// pofs[i] .. pofs[i+1]-1, partitions cofs[i] .. cofs[i+1]-1 (grid[i] per side).
struct Inst {
    const int *pofs;
    const int *cofs;
    const int *grid;
    // quad-tree partitions (one instance): the leaf of every fine cell of side
    // 2^qshift of the square at (qx0, qy0), qF x qF fine cells; null = the grid
    const int *qmap;
    int qx0, qy0, qshift, qF;
    const int *moff;  // per step: the moves of instance i are moff[i] .. moff[i+1]-1
    const int *tofs;  // triangle slots of instance i: tofs[i] .. tofs[i+1]-1
    const int *order; // the order in which the kinetic kernel takes the partitions (the
                      // step planner's, longest first), or null: index order
    int *qhist;       // quad-tree re-divided at every step: points per fine cell, kept
                      // current by the intake; null otherwise
    const int *ncells_dyn;  // ... and this step's number of leaves (else the launch's count)
    int stride;       // without a planned order: ticket k takes partition k * stride mod the
                      // partition count (a stride coprime with it, near the golden ratio of
                      // it), so partitions taken at the same time lie far apart; 0 or 1:
                      // index order
    int ninst;
};

// Partition of a position of instance `inst`: its grid cell, or the quad-tree leaf of
// its fine cell (positions outside the square clamped into it).
__device__ __forceinline__ int partition_of(const Inst &I, int inst, int bits, int2 o)
{
    if (I.qmap) {
        int fx = (int)max(0ll, min((long long)I.qF - 1, ((long long)o.x - I.qx0) >> I.qshift));
        int fy = (int)max(0ll, min((long long)I.qF - 1, ((long long)o.y - I.qy0) >> I.qshift));
        return I.qmap[fy * I.qF + fx];
    }
    const int G = I.grid[inst];
    const int cx = (int)(((long long)o.x * G) >> bits);
    const int cy = (int)(((long long)o.y * G) >> bits);
    return I.cofs[inst] + cy * G + cx;
}

// fine cell (row-major) of a position in the quad-tree's square, clamped into it
__device__ __forceinline__ int qt_fine(const Inst &I, int2 o)
{
    int fx = (int)max(0ll, min((long long)I.qF - 1, ((long long)o.x - I.qx0) >> I.qshift));
    int fy = (int)max(0ll, min((long long)I.qF - 1, ((long long)o.y - I.qy0) >> I.qshift));
    return fy * I.qF + fx;
}

// ---- the quad-tree re-divided at every step (kdt_config.quadtree = 2), on the GPU.
// Depth-first order of the leaves with children (low x, low y), (high x, low y), (low x,
// high y), (high x, high y) is the order of their first fine cell's Morton index with x
// in the low bit of every two-bit digit.
__device__ __forceinline__ unsigned qt_morton(unsigned x, unsigned y)
{
    unsigned m = 0;
    for (int b = 0; b < 16; ++b) m |= (((x >> b) & 1u) << (2 * b)) | (((y >> b) & 1u) << (2 * b + 1));
    return m;
}

// one level of the count pyramid: dst (w x w, row-major) from src (2w x 2w)
__global__ void k_qt_level(const int *src, int *dst, int w)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w * w; i += gridDim.x * blockDim.x) {
        const int y = i / w, x = i - y * w, s = 2 * w;
        dst[i] = src[(2 * y) * s + 2 * x] + src[(2 * y) * s + 2 * x + 1] + src[(2 * y + 1) * s + 2 * x] +
                 src[(2 * y + 1) * s + 2 * x + 1];
    }
}

// every fine cell: the level of its leaf (the first level from the whole square down
// whose square holds at most T points, or the floor D) into lev[morton], and
// flag[morton] = 1 iff the cell is the first of its leaf.  Level l of the pyramid
// (2^l x 2^l) starts at pyr + (4^l - 1) / 3; level D is qhist.
__global__ void k_qt_leaf(const int *pyr, int D, int T, int *flag, unsigned char *lev)
{
    const int F = 1 << D;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F * F; f += gridDim.x * blockDim.x) {
        const int fy = f >> D, fx = f & (F - 1);
        int l = 0;
        for (; l < D; ++l) {
            const int c = pyr[((1 << (2 * l)) - 1) / 3 + ((fy >> (D - l)) << l) + (fx >> (D - l))];
            if (c <= T) break;
        }
        const unsigned m = qt_morton((unsigned)fx, (unsigned)fy);
        lev[m] = (unsigned char)l;
        flag[m] = (m & ((1u << (2 * (D - l))) - 1u)) == 0u ? 1 : 0;
    }
}

// qmap (row-major) = the depth-first number of each fine cell's leaf: the exclusive
// prefix count of leaf starts at its leaf's first cell
__global__ void k_qt_map(const int *pre, const unsigned char *lev, int D, int *qmap)
{
    const int F = 1 << D;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F * F; f += gridDim.x * blockDim.x) {
        const int fy = f >> D, fx = f & (F - 1);
        const unsigned m = qt_morton((unsigned)fx, (unsigned)fy);
        const int l = lev[m];
        qmap[f] = pre[m & ~((1u << (2 * (D - l))) - 1u)];
    }
}

// points per fine cell of the quad-tree's square (the first division is made on the host)
__global__ void k_qt_hist(const int2 *xy, int n, int x0, int y0, int shift, int F, int *hist)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int2 p = xy[i];
        int fx = (int)max(0ll, min((long long)F - 1, ((long long)p.x - x0) >> shift));
        int fy = (int)max(0ll, min((long long)F - 1, ((long long)p.y - y0) >> shift));
        atomicAdd(hist + fy * F + fx, 1);
    }
}


// The warp's handle and its shared state (counters zero, claims none, random state
// from `seed`, instance = the points [d.rlo, d.rlo + d.rn)).
static_assert(C_NUM <= 32, "one lane clears each counter");
// k_kinetic runs six 128-thread blocks per SM, set by its registers (up to 80 a thread:
// fewer spills of the inlined move path than at 72, which measured 0.1125 against
// 0.118 ms per launch on the 1e6-point step).  The shared memory would allow seven:
// 7 x (static shared memory, rounded up to 128 bytes, + 1 KB reserved per block) fits
// the SM's 228 KB; keeping that bound leaves the choice open.
static_assert(WPB * sizeof(WarpShared) + sizeof(Dev) <= 32256, "k_kinetic's shared memory must allow 7 blocks per SM");

__device__ __forceinline__ Warp make_warp(WarpShared *sh, int token, unsigned seed, const Dev &d)
{
    Warp w;
    w.sh = sh;
    w.lane = threadIdx.x & 31;
    w.token = token;
    if (w.lane < C_NUM) sh->cnt[w.lane] = 0;
    if (w.lane == 0) {
        unsigned r = seed * 2654435761u + 0x9E3779B9u;
        sh->rng = r ? r : 1u;
        sh->ncl = 0;
        sh->cyc_max = 0;
        sh->rlo = d.rlo;
        sh->rn = d.rn;
        sh->clbig = 0;
    }
    __syncwarp();
    return w;
}

// One copy of the launch's Dev per block in shared memory: device functions take it
// by reference, which a kernel parameter cannot give without a per-thread copy in
// local memory.
#define KD_BLOCK_DEV(param)                                           \
    __shared__ Dev kd_block_dev;                                      \
    if (threadIdx.x == 0) {                                           \
        kd_block_dev = (param);                                       \
        if ((param).ctl) kd_block_dev.stamp = __ldcg((param).ctl + 1); \
    }                                                                 \
    __syncthreads();                                                  \
    const Dev &d = kd_block_dev

// ------------------------------------------------------------------ scan

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// exclusive scan of one tile; tile totals to tile_sums
__global__ void k_scan_tile(const int *in, int *out, int n, int *tile_sums)
{
    __shared__ int ws[SCAN_THREADS / 32];
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int y = lane < SCAN_THREADS / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int z = __shfl_up_sync(FULL, y, o);
            if (lane >= o) y += z;
        }
        if (lane < SCAN_THREADS / 32) ws[lane] = y;
    }
    __syncthreads();
    int run = x - s + (wid > 0 ? ws[wid - 1] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == SCAN_THREADS - 1) tile_sums[blockIdx.x] = run;
}

// exclusive scan of the tile totals in one block; grand total to *total
__global__ void k_scan_sums(int *tile_sums, int ntiles, int *total)
{
    __shared__ int ws[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < ntiles; base += blockDim.x) {
        int i = base + threadIdx.x;
        int s = i < ntiles ? tile_sums[i] : 0;
        int x = s;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int y = lane < (int)(blockDim.x / 32) ? ws[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int z = __shfl_up_sync(FULL, y, o);
                if (lane >= o) y += z;
            }
            ws[lane] = y;
        }
        __syncthreads();
        int excl = carry + x - s + (wid > 0 ? ws[wid - 1] : 0);
        if (i < ntiles) tile_sums[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + s;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_add(int *out, int n, const int *tile_sums)
{
    int add = tile_sums[blockIdx.x];
    int base = blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x)
        if (base + i < n) out[base + i] += add;
}

// ------------------------------------------------------------------ step: intake

// The moves of a step, read from the control block when the step is a graph launch
// (ctl[2..3] hold the pointer), else from the argument.
__device__ __forceinline__ const int3 *step_moves(const Dev &d, const int3 *moves)
{
    if (!d.ctl) return moves;
    unsigned lo = (unsigned)__ldcg(d.ctl + 2), hi = (unsigned)__ldcg(d.ctl + 3);
    return reinterpret_cast<const int3 *>(((unsigned long long)hi << 32) | lo);
}

// Start of a step: the scalars zero, every partition's move list empty, every deferred
// entry -1 (one launch instead of three copies of memset).
__global__ void k_step_clear(int *scal, int nscal, int *head, int ncells, int4 *deferred, int ndef)
{
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(ncells, ndef); i += stride) {
        if (i < nscal) scal[i] = 0;
        if (i < ncells) head[i] = -1;
        if (i < ndef) deferred[i] = make_int4(-1, -1, -1, -1);
    }
}

// An invalid move stops the step; it wins over the displacement rule's DEV_FAR, so
// the host never rebuilds from an invalid move list.
__device__ __forceinline__ void intake_fail(int *status, int code)
{
    if (atomicCAS(status, 0, code) == DEV_FAR) atomicCAS(status, DEV_FAR, code);
}

// Intake and per-partition bucketing in one pass: validate each move (A2), stamp the
// moved id, remember the old position, and push the move onto the list of the
// partition that owns the point (its cell at the start of the step, Section III
// blocks): next[i] = previous head of the cell's list.  With far2 > 0 (the rebuild
// rule of kdt_config.rebuild_displacement) a move whose squared displacement exceeds
// far2 x its partition's d_local^2 (dloc2; INT64_MAX = unknown or an empty partition)
// is counted, and the
// step becomes a rebuild (DEV_FAR stops the kinetic kernel before it changes anything).
__global__ void k_intake_link(Dev d, const int3 *moves, int m, Inst I, int bits, int *head, int *next,
                              int2 *old_xy, int3 *gmoves, const unsigned long long *dloc2, double far2)
{
    if (d.ctl) {
        m = __ldcg(d.ctl);
        d.stamp = __ldcg(d.ctl + 1);
    }
    moves = step_moves(d, moves);
    long long lim = 1ll << bits;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int inst = I.ninst > 1 ? csr_find(I.moff, I.ninst + 1, i) : 0;
        int p0 = I.pofs[inst], ni = I.pofs[inst + 1] - p0;
        int3 mv = moves[i];
        if (mv.x < 0 || mv.x >= ni) {
            intake_fail(d.status, DEV_ARG);
            continue;
        }
        if (mv.y < 0 || mv.z < 0 || mv.y >= lim || mv.z >= lim) {
            intake_fail(d.status, DEV_RANGE);
            continue;
        }
        int g = p0 + mv.x;
        int prev = atomicExch(d.pt_stamp + g, d.stamp);
        if (prev == d.stamp) {
            intake_fail(d.status, DEV_DUP_ID);
            continue;
        }
        int2 o = d.xy[g];
        old_xy[i] = o;
        gmoves[i] = make_int3(g, mv.y, mv.z);
        const int cell = partition_of(I, inst, bits, o);
        if (I.qhist) {
            // the re-divided quad-tree counts points at their positions after the step
            atomicSub(I.qhist + qt_fine(I, o), 1);
            atomicAdd(I.qhist + qt_fine(I, make_int2(mv.y, mv.z)), 1);
        }
        if (far2 > 0.0 && dloc2) {
            const long long dx = (long long)mv.y - o.x, dy = (long long)mv.z - o.y;
            const unsigned long long dl = dloc2[cell];
            if (dl < (unsigned long long)LLONG_MAX && (double)(dx * dx + dy * dy) > far2 * (double)dl) {
                atomicAdd(d.status + S_FAR, 1);
                atomicCAS(d.status, 0, DEV_FAR);
            }
        }
        next[i] = atomicExch(head + cell, i);
    }
}

// ------------------------------------------------------------------ step: kinetic

// One warp per partition (Fig. 4's parallel loop over the blocks): for each of the
// block's moved points, Delete (Section IV), Update the coordinate, Insert at the
// new position (walk, split, Lawson flips).  The new block of a point that crosses a
// partition border follows from its new position; all blocks share one
// triangulation in HBM, so the hand-off of Fig. 4 is an ownership change, not a
// message.  A point whose target is still occupied by a point that has not moved
// yet is deferred.  The last warp to finish inserts the deferred points and
// certifies the triangles written on the global-memory path.
__device__ __noinline__ void step_tail(Warp w, const Dev &d, Inst I, int4 *deferred, int *defer_count,
                                       int defer_cap, int *viol, int viol_cap);

// Entries of the deferred list: (p, s0, s1, hint) = an insertion left to the end of the
// step (s0 >= 0); (p, DQ_MOVE - pass, qx, qy) = a whole move left for later, pass
// counting how often it was left; (p, DQ_HUGE, qx, qy) = the move of a point of degree
// above KMAX, for the first warp that runs out of partitions; DQ_DONE once a warp has
// taken it.
constexpr int DQ_MOVE = -2, DQ_HUGE = -50, DQ_DONE = -100, DQ_PASSES = 3;

// Global-path writes the last warp certifies itself; a longer list goes to the whole GPU.
constexpr int TAIL_CERTIFY = 64;

// Append an entry.  The list is cleared to -1 before every step and the point id is
// written last (after a fence), so a warp that takes a reserved but unwritten entry
// sees -1 there and waits for it (read_deferred).
__device__ __forceinline__ void push_deferred(Warp w, const Dev &d, int4 *deferred, int *defer_count, int defer_cap,
                                              int4 e)
{
    if (w.lane == 0) {
        int pos = atomicAdd(defer_count, 1);
        if (pos < defer_cap) {
            int *f = reinterpret_cast<int *>(deferred + pos);
            f[1] = e.y;
            f[2] = e.z;
            f[3] = e.w;
            __threadfence();
            atomicExch(f, e.x);
        } else {
            atomicCAS(d.status, 0, DEV_CAPACITY);
        }
    }
    cnt_add(w, C_DEFERRED, 1);
    __syncwarp();
}

// Entry j once its writer has published it (bounded wait); x = -1 if it never appeared.
__device__ __forceinline__ int4 read_deferred(Warp w, const int4 *deferred, int j)
{
    const int *f = reinterpret_cast<const int *>(deferred + j);
    int4 e = make_int4(-1, 0, 0, 0);
    if (w.lane == 0) {
        int x = -1;
        for (int spin = 0; spin < (1 << 20); ++spin) {
            x = __ldcg(f);
            if (x != -1) break;
        }
        __threadfence();
        e = make_int4(x, __ldcg(f + 1), __ldcg(f + 2), __ldcg(f + 3));
    }
    return bcast4(e, 0);
}

// One move of p to q (Fig. 4: Delete, Update, Insert): the staged move, else the
// global-memory path.  may_give_up: a move whose claims keep failing returns MV_BIG
// untouched, one whose point has a degree above KMAX MV_HUGE; otherwise claims are
// retried and a high-degree point is moved with its star in the warp's global scratch.
// rc: 0, MV_BIG, MV_HUGE, INS_DEFER / MV_DEFER (p deleted and placed, its insertion
// left to the end of the step with spares s0, s1 and hint), or an error.
struct MoveOut {
    int rc, s0, s1, hint;
};

__device__ __forceinline__ MoveOut run_move(Warp w, const Dev &d, int p, int2 q, bool may_give_up)
{
    MoveOut o;
    int s0 = -1, s1 = -1, hint = -1;
    long long c0 = clock64();
    int rc = move_point(w, d, p, q, s0, s1, hint, may_give_up);
    const bool big = (rc == MV_BIG || rc == MV_HUGE) && !may_give_up;
    if (big) {
        // a degree above KMAX: the star goes to the warp's global scratch.  A short
        // move that keeps every triangle of the star valid changes p's position (and
        // flips the star's edges that stop being Delaunay); otherwise p is deleted and
        // inserted again.  Its claims are patient.
        long long cb = clock64();
        Warp wb = w;
        wb.token |= TOK_PATIENT;
        rc = move_in_place_big(wb, d, p, q);
        const long long ci = clock64();
        dev_count(w, d, C_CYC_BIG_INPLACE, (unsigned long long)(ci - cb));
        if (rc == 1) {
            rc = 0;
            dev_count(w, d, C_BIG_INPLACE, 1);
        } else if (rc == 0) {
            rc = delete_point_big(wb, d, p, s0, s1, hint);
            dev_count(w, d, C_CYC_BIG_DELETE, (unsigned long long)(clock64() - ci));
            if (rc == 0) rc = MV_GLOBAL;
        }
        dev_count(w, d, C_BIG_MOVES, 1);
    }
    if (rc == MV_GLOBAL) {
        cnt_add(w, C_MV_GLOBAL, 1);
        if (w.lane == 0) {
            d.xy[p] = q;
            __threadfence();
        }
        __syncwarp();
        const long long cg = clock64();
        // p is deleted and must be inserted: its claims are patient (they wait, bounded,
        // for slots other warps hold instead of releasing everything and walking again)
        Warp wi = w;
        wi.token |= TOK_PATIENT;
        rc = insert_staged(wi, d, p, q, hint, s0, s1, true);
        if (rc == INS_GLOBAL) rc = insert_point(wi, d, p, q, hint, s0, s1, true);
        const unsigned long long gc = (unsigned long long)(clock64() - cg);
        dev_count(w, d, C_CYC_GLOBAL_INS, gc);
        if (w.lane == 0 && d.counters) atomicMax(d.counters + C_GLOBAL_INS_MAX, gc);
    }
    unsigned cy = (unsigned)((clock64() - c0) >> 6);
    if (!may_give_up) {
        // a move run without giving up: the high-degree ones' whole time (in place,
        // or deletion + insertion), and the longest of all such moves
        if (w.lane == 0 && d.counters) atomicMax(d.counters + C_BIG_MAX, (unsigned long long)cy << 6);
        if (big) dev_count(w, d, C_CYC_BIG, (unsigned long long)cy << 6);
    }
    cnt_add(w, C_CYC_MOVE, cy);
    if (w.lane == 0 && cy > w.sh->cyc_max) w.sh->cyc_max = cy;
    o.rc = rc;
    o.s0 = s0;
    o.s1 = s1;
    o.hint = hint;
    return o;
}

// Record a move's outcome: deferred work goes to the list, an error to the status.
// Returns false when the warp must stop.
__device__ __forceinline__ bool settle_move(Warp w, const Dev &d, int rc, int p, int2 q, int pass, int s0, int s1,
                                            int hint, int4 *deferred, int *defer_count, int defer_cap)
{
    if (rc == MV_BIG || rc == MV_HUGE) {
        push_deferred(w, d, deferred, defer_count, defer_cap,
                      make_int4(p, rc == MV_HUGE ? DQ_HUGE : DQ_MOVE - pass, q.x, q.y));
        return true;
    }
    if (rc == MV_DEFER || rc == INS_DEFER) {
        push_deferred(w, d, deferred, defer_count, defer_cap, make_int4(p, s0, s1, hint));
        return true;
    }
    if (rc) {
        if (rc > 0 && w.lane == 0 && atomicCAS(d.status, 0, rc) == 0) d.status[S_FAILPT] = p;
        return false;
    }
    return true;
}

// A warp stops running a move taken from the deferred list; the entries it pushed
// were counted first.
__device__ __noinline__ void drain_stop(Warp w, const Dev &d)
{
    if (w.lane == 0) {
        __threadfence();
        atomicSub(d.status + S_DRUN, 1);
    }
    __syncwarp();
}

// A move taken from the deferred list: j < 0 when there is none to take (stop
// draining), skip when the entry is not this phase's work.
struct Drained {
    int j, p, pass;
    int2 q;
    bool skip, huge;
};

// Reserve the next entry of the deferred list with one atomic add (a compare-and-swap
// loop on one word costs entries x contenders atomics when thousands of warps drain at
// once).  An entry reserved before it was pushed is waited for while a warp may still
// push one (one is still on its partitions: a warp leaves them with the one ticket it
// takes beyond the last; or one is on a move from the list); one pushed after all of
// them stopped is left to the last warp.  A taken move counts as running (S_DRUN)
// until drain_stop.
__device__ __noinline__ Drained take_deferred(Warp w, const Dev &d, int4 *deferred, const int *defer_count,
                                              int defer_cap, int items, int nw)
{
    Drained t;
    t.j = -1;
    t.skip = false;
    t.huge = false;
    t.p = -1;
    t.pass = 0;
    t.q = make_int2(0, 0);
    if (read_status(d)) return t;
    int j = -1;
    if (w.lane == 0) {
        if (__ldcg(d.status + S_DNEXT) < min(__ldcg(defer_count), defer_cap)) {
            const int r = atomicAdd(d.status + S_DNEXT, 1);
            for (int spin = 0; spin < (1 << 16) && r < defer_cap; ++spin) {
                if (r < min(__ldcg(defer_count), defer_cap)) {
                    j = r;
                    break;
                }
                if (__ldcg(d.status + S_TICKET) - items >= nw && __ldcg(d.status + S_DRUN) == 0) break;
                __nanosleep(256);
            }
            if (j >= 0) atomicAdd(d.status + S_DRUN, 1);
        }
    }
    t.j = __shfl_sync(FULL, j, 0);
    if (t.j < 0) return t;
    int4 e = read_deferred(w, deferred, t.j);
    // an unpublished entry, an insertion (for the end), a taken entry, or a move left
    // too often: the last warp takes those
    bool skip = e.x < 0 || e.y > DQ_MOVE || e.y <= DQ_DONE;
    t.huge = !skip && e.y == DQ_HUGE;
    t.skip = skip || (!t.huge && DQ_MOVE - e.y >= DQ_PASSES);
    if (t.skip) {
        drain_stop(w, d);
        return t;
    }
    if (w.lane == 0) deferred[t.j].y = DQ_DONE;
    __syncwarp();
    t.pass = t.huge ? 0 : DQ_MOVE - e.y + 1;
    dev_count(w, d, C_DRAIN_MOVES, 1);
    t.p = e.x;
    t.q = make_int2(e.z, e.w);
    return t;
}

// timeline notes of a drained move (debug)
__device__ __noinline__ void drained_done(Warp w, const Dev &d, int rc, bool huge, long long cycles)
{
    if (d.timeline && d.counters && w.lane == 0) {
        atomicMax(d.counters + (huge ? C_TH : C_TDM), global_ns());
        atomicMax(d.counters + C_DRAINED_MAX, (unsigned long long)cycles);
        if (rc == MV_BIG) atomicAdd(d.counters + C_REDEFER, 1ull);
    }
}

// The kinetic kernel, compiled for two occupancies: MINB = 6 blocks per SM (up to 80
// registers a thread, the default) or 7 (up to 72: more warps in flight, more spills of
// the inlined move path); kdt_config.kinetic_blocks_per_sm chooses.
template <int MINB>
__global__ void __launch_bounds__(WPB * 32, MINB) k_kinetic(Dev dp, const int3 *moves, const int *head,
                                                            const int *next, Inst I, int ncells, int wpp,
                                                            int4 *deferred, int *defer_count, int defer_cap,
                                                            int *viol, int viol_cap)
{
    KD_BLOCK_DEV(dp);
    __shared__ WarpShared shs[WPB];
    int wib = threadIdx.x >> 5;
    int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    int nw = gridDim.x * (blockDim.x >> 5);
    Warp w = make_warp(&shs[wib], gw + 1, gw + 17 * d.stamp, d);
    const bool tl = d.timeline && d.counters;
    if (tl && gw == 0 && w.lane == 0) d.counters[C_T0] = global_ns();
    const int items = (I.ncells_dyn ? __ldcg(I.ncells_dyn) : ncells) * wpp;
    // One loop, one move per iteration: first the moves of the (partition, share) work
    // items the warp takes from a ticket; when those are gone, the whole moves left
    // so far (drained in parallel with the warps still busy; each may be left again,
    // DQ_PASSES times, before the last warp runs it when nothing else competes).
    int i = -1, kk = -1, sub = 0, c = 0;  // position in the current partition's list
    bool tickets = true;
    while (true) {
        int p, pass = 0;
        bool huge = false;  // a high-degree point's move, run without giving up
        int2 q;
        if (tickets) {
            // next move of this work item (every wpp-th of the partition's list)
            if (i >= 0) i = __shfl_sync(FULL, __ldcg(next + i), 0);
            while (i >= 0 && ++kk % wpp != sub) i = __shfl_sync(FULL, __ldcg(next + i), 0);
            if (i < 0) {
                if (read_status(d)) break;
                int t = 0;
                if (w.lane == 0) t = atomicAdd(d.status + S_TICKET, 1);
                t = __shfl_sync(FULL, t, 0);
                if (t >= items) {
                    tickets = false;
                    if (tl && w.lane == 0) atomicMax(d.counters + C_TT, global_ns());
                    // nothing was left for later so far: this warp is done
                    if (__shfl_sync(FULL, w.lane == 0 ? __ldcg(defer_count) : 0, 0) == 0) break;
                    continue;
                }
                c = t / wpp;
                sub = t - c * wpp;
                if (I.order) c = __ldcg(I.order + c);
                else if (I.stride > 1) c = (int)(((long long)c * I.stride) % ncells);
                kk = -1;
                i = __shfl_sync(FULL, __ldcg(head + c), 0);
                int inst = I.ninst > 1 ? csr_find(I.cofs, I.ninst + 1, c) : 0;
                set_instance(w, I.pofs[inst], I.pofs[inst + 1] - I.pofs[inst]);
                while (i >= 0 && ++kk % wpp != sub) i = __shfl_sync(FULL, __ldcg(next + i), 0);
                if (i < 0) continue;
            }
            int3 mv = moves[i];
            p = mv.x;
            q = make_int2(mv.y, mv.z);
        } else {
            const Drained t = take_deferred(w, d, deferred, defer_count, defer_cap, items, nw);
            if (t.j < 0) break;
            if (t.skip) continue;
            huge = t.huge;
            pass = t.pass;
            p = t.p;
            q = t.q;
            int inst = I.ninst > 1 ? csr_find(I.pofs, I.ninst + 1, p) : 0;
            set_instance(w, I.pofs[inst], I.pofs[inst + 1] - I.pofs[inst]);
        }
        const long long cm = tl ? clock64() : 0;
        MoveOut o = run_move(w, d, p, q, !huge);
        if (!tickets) drained_done(w, d, o.rc, huge, tl ? clock64() - cm : 0);
        if (!settle_move(w, d, o.rc, p, q, pass, o.s0, o.s1, o.hint, deferred, defer_count, defer_cap)) {
            if (!tickets) drain_stop(w, d);
            break;
        }
        if (!tickets) drain_stop(w, d);
    }
    // the last warp to finish does the tail work
    int done = 0;
    __syncwarp();
    if (w.lane == 0) {
        if (tl) atomicMax(d.counters + C_TD, global_ns());
        __threadfence();
        done = atomicAdd(d.status + S_DONE, 1);
    }
    done = __shfl_sync(FULL, done, 0);
    if (done == nw - 1) {
        __threadfence();
        step_tail(w, d, I, deferred, defer_count, defer_cap, viol, viol_cap);
        if (tl && w.lane == 0) {
            unsigned long long t0 = __ldcg(d.counters + C_T0), tt = __ldcg(d.counters + C_TT);
            unsigned long long td = __ldcg(d.counters + C_TD), now = global_ns();
            if (t0 && tt >= t0) d.counters[C_SPAN_TICKETS] += tt - t0;
            if (t0 && td >= t0) d.counters[C_SPAN_DRAIN] += td - t0;
            if (t0 && now >= t0) d.counters[C_SPAN_ALL] += now - t0;
            unsigned long long th = __ldcg(d.counters + C_TH), tdm = __ldcg(d.counters + C_TDM);
            if (t0 && th >= t0) d.counters[C_SPAN_HUGE] += th - t0;
            if (t0 && tdm >= t0) d.counters[C_SPAN_DRAINED] += tdm - t0;
            d.counters[C_TT] = 0;
            d.counters[C_TD] = 0;
            d.counters[C_TH] = 0;
            d.counters[C_TDM] = 0;
        }
    }
    flush_counters(w, d);
}

// ------------------------------------------------------------------ hull winding

// 0 for directions with angle in [0, pi), 1 for [pi, 2 pi)
__device__ __forceinline__ int dir_half(long long dx, long long dy) { return (dy < 0 || (dy == 0 && dx < 0)) ? 1 : 0; }

// is direction a strictly before direction b in counter-clockwise angle from +x?
__device__ __forceinline__ bool dir_less(long long ax, long long ay, long long bx, long long by)
{
    int ha = dir_half(ax, ay), hb = dir_half(bx, by);
    if (ha != hb) return ha < hb;
    return ax * by - ay * bx > 0;
}

// Does the hull turn "wrap" past angle 0 at the vertex between this ghost's hull edge
// and the next one?  Summed over the hull, a valid triangulation wraps exactly once:
// with every triangle counter-clockwise and every edge locally Delaunay, the ghost
// cycle winding once makes the surface a degree-1 cover of the plane, i.e. a
// triangulation, and then Lawson's lemma makes it the Delaunay triangulation.
__device__ int hull_wrap(const Dev &d, const int4 &v, const int4 &nb)
{
    int g = v.x == KDT_GHOST ? 0 : (v.y == KDT_GHOST ? 1 : (v.z == KDT_GHOST ? 2 : -1));
    if (g < 0) return 0;
    int u = comp(v, (g + 1) % 3), vv = comp(v, (g + 2) % 3);  // hull edge vv -> u
    int4 nv = __ldcg(d.tv + (comp(nb, (g + 2) % 3) >> 2));
    int ng = nv.x == KDT_GHOST ? 0 : (nv.y == KDT_GHOST ? 1 : (nv.z == KDT_GHOST ? 2 : -1));
    if (ng < 0) return 100;  // not a ghost: inconsistent
    int y = comp(nv, (ng + 1) % 3);                            // next hull edge u -> y
    int2 pu = __ldcg(d.xy + u), pv = __ldcg(d.xy + vv), py = __ldcg(d.xy + y);
    return dir_less((long long)py.x - pu.x, (long long)py.y - pu.y, (long long)pu.x - pv.x,
                    (long long)pu.y - pv.y)
               ? 1
               : 0;
}

// ------------------------------------------------------------------ certification

__device__ void certify_one(const Dev &d, int t, int *viol, int *viol_count, int viol_cap, unsigned *ex,
                            unsigned *ti)
{
    int4 v = __ldcg(d.tv + t);
    if (!(v.w & ALIVE)) return;
    int4 nb = __ldcg(d.tn + t);
    if (v.x >= 0 && v.y >= 0 && v.z >= 0) {
        if (orient2d(__ldcg(d.xy + v.x), __ldcg(d.xy + v.y), __ldcg(d.xy + v.z)) <= 0) {
            atomicCAS(d.status, 0, DEV_INTERNAL);
            return;
        }
    }
    for (int e = 0; e < 3; ++e) {
        int r = check_edge(d, t, v, nb, e, ex, ti);
        if (r < 0) {
            atomicCAS(d.status, 0, DEV_INTERNAL);
            return;
        }
        if (r > 0) {
            int pos = atomicAdd(viol_count, 1);
            if (pos < viol_cap) viol[pos] = (t << 2) | e;
        }
    }
}

// Tail of a step (one warp, after every other warp finished): insert the deferred
// points, then certify the triangles written on the global-memory path (the staged
// path certified its own).  A long dirty list is left to the host.
__device__ __noinline__ void step_tail(Warp w, const Dev &d, Inst I, int4 *deferred, int *defer_count,
                                       int defer_cap, int *viol, int viol_cap)
{
    if (read_status(d)) return;
    const long long c0 = clock64();
    // Every other warp has finished, so every entry is published.  The lanes read 32
    // entries at a time and the warp runs the ones with work in list order; entries
    // appended meanwhile are read when the scan reaches them.  Pass 0: whole moves not
    // taken yet (left by the last warps), run without giving up (an insertion onto a
    // point still to be inserted is deferred again); pass 1: the deferred insertions.
    for (int pass = 0; pass < 2; ++pass) {
        int scanned = 0;
        while (true) {
            if (read_status(d)) return;
            int cnt = min(__shfl_sync(FULL, __ldcg(defer_count), 0), defer_cap);
            if (scanned >= cnt) break;
            int j = scanned + w.lane;
            int4 e = j < cnt ? __ldcg(deferred + j) : make_int4(-1, 0, 0, 0);
            bool todo = e.x >= 0 && (pass == 0 ? (e.y <= DQ_MOVE && e.y > DQ_DONE) : e.y >= 0);
            unsigned tm = __ballot_sync(FULL, todo);
            scanned = min(scanned + 32, cnt);
            while (tm) {
                const int src = __ffs(tm) - 1;
                tm &= tm - 1u;
                int4 ei = bcast4(e, src);
                if (pass == 0) {
                    if (w.lane == 0) deferred[j - w.lane + src].y = DQ_DONE;
                    __syncwarp();
                    int p = ei.x;
                    int2 q = make_int2(ei.z, ei.w);
                    int inst = I.ninst > 1 ? csr_find(I.pofs, I.ninst + 1, p) : 0;
                    set_instance(w, I.pofs[inst], I.pofs[inst + 1] - I.pofs[inst]);
                    MoveOut o = run_move(w, d, p, q, false);
                    dev_count(w, d, C_TAIL_MOVES, 1);
                    if (o.rc == MV_BIG || o.rc == MV_HUGE) o.rc = DEV_INTERNAL;  // never returned without giving up
                    if (!settle_move(w, d, o.rc, p, q, DQ_PASSES, o.s0, o.s1, o.hint, deferred, defer_count,
                                     defer_cap))
                        return;
                } else {
                    int2 q = __ldcg(d.xy + ei.x);
                    q = bcast2(q, 0);
                    int inst = I.ninst > 1 ? csr_find(I.pofs, I.ninst + 1, ei.x) : 0;
                    set_instance(w, I.pofs[inst], I.pofs[inst + 1] - I.pofs[inst]);
                    int rc = insert_staged(w, d, ei.x, q, ei.w, ei.y, ei.z, false);
                    if (rc == INS_GLOBAL) rc = insert_point(w, d, ei.x, q, ei.w, ei.y, ei.z, false);
                    if (rc) {
                        if (rc > 0 && w.lane == 0 && atomicCAS(d.status, 0, rc) == 0) d.status[S_FAILPT] = ei.x;
                        return;
                    }
                }
            }
        }
        __threadfence();
    }
    dev_count(w, d, C_CYC_TAIL, (unsigned long long)(clock64() - c0));
    __threadfence();
    int hi = __shfl_sync(FULL, __ldcg(d.dirty_count), 0);
    if (hi > TAIL_CERTIFY) {
        // a longer list is certified by the whole GPU (k_certify_step, the next node)
        if (w.lane == 0) d.status[S_CERTPEND] = 1;
        return;
    }
    unsigned ex = 0, ti = 0;
    for (int i = w.lane; i < hi; i += 32)
        certify_one(d, d.dirty[i], viol, d.status + S_VIOL, viol_cap, &ex, &ti);
}

// certify the dirty slots [lo, *dirty_count) (the slots written in this step)
// The step's certification of the triangles written on the global-memory path when the
// last warp left the list to the whole GPU (S_CERTPEND); a no-op otherwise.
__global__ void k_certify_step(Dev d, int *viol, int *viol_count, int viol_cap)
{
    if (__ldcg(d.status + S_CERTPEND) == 0 || __ldcg(d.status) != 0) return;
    int hi = __ldcg(d.dirty_count);
    if (hi > d.dirty_cap) return;  // overflowed: the host certifies every slot
    unsigned ex = 0, ti = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x)
        certify_one(d, d.dirty[i], viol, viol_count, viol_cap, &ex, &ti);
}

__global__ void k_certify(Dev d, int lo, int *viol, int *viol_count, int viol_cap)
{
    int hi = *d.dirty_count;
    if (hi > d.dirty_cap) hi = d.dirty_cap;
    unsigned ex = 0, ti = 0;
    for (int i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x)
        certify_one(d, d.dirty[i], viol, viol_count, viol_cap, &ex, &ti);
}

// certify every slot (after a build, or when the dirty list overflowed)
__global__ void k_certify_all(Dev d, int s0, int nslots, int *viol, int *viol_count, int viol_cap, int *wraps)
{
    unsigned ex = 0, ti = 0;
    for (int t = s0 + blockIdx.x * blockDim.x + threadIdx.x; t < s0 + nslots; t += gridDim.x * blockDim.x) {
        certify_one(d, t, viol, viol_count, viol_cap, &ex, &ti);
        int4 v = __ldcg(d.tv + t);
        if ((v.w & ALIVE) && (v.x < 0 || v.y < 0 || v.z < 0)) {
            int wr = hull_wrap(d, v, __ldcg(d.tn + t));
            if (wr) atomicAdd(wraps, wr);
        }
    }
}

// Lawson repair of the edges the certification rejected (general flip algorithm:
// every flip queues the four outer edges of its quadrilateral).
__global__ void __launch_bounds__(WPB * 32) k_fixup(Dev dp, const int *viol, int nviol)
{
    KD_BLOCK_DEV(dp);
    __shared__ WarpShared shs[WPB];
    int wib = threadIdx.x >> 5;
    int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    int nw = gridDim.x * (blockDim.x >> 5);
    Warp w = make_warp(&shs[wib], gw + 1, gw + 31 * d.stamp + 5, d);
    for (int j = gw; j < nviol; j += nw) {
        if (read_status(d)) break;
        int r = viol[j];
        if (w.lane == 0) w.sh->stack[0] = make_int2(r >> 2, r & 3);
        __syncwarp();
        lawson(w, d, 1, -2, false);
    }
    flush_counters(w, d);
}

// ------------------------------------------------------------------ build

__global__ void k_range(const int2 *xy, int n, int bits, int *status, int *bbox)
{
    long long lim = 1ll << bits;
    int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int2 p = xy[i];
        if (p.x < 0 || p.y < 0 || p.x >= lim || p.y >= lim) atomicCAS(status, 0, DEV_RANGE);
        mnx = min(mnx, p.x);
        mny = min(mny, p.y);
        mxx = max(mxx, p.x);
        mxy = max(mxy, p.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mnx = min(mnx, __shfl_xor_sync(FULL, mnx, o));
        mny = min(mny, __shfl_xor_sync(FULL, mny, o));
        mxx = max(mxx, __shfl_xor_sync(FULL, mxx, o));
        mxy = max(mxy, __shfl_xor_sync(FULL, mxy, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(bbox + 0, mnx);
        atomicMin(bbox + 1, mny);
        atomicMax(bbox + 2, mxx);
        atomicMax(bbox + 3, mxy);
    }
}

// Hilbert index of cell (x, y) in a 2^k x 2^k grid (the rotate-and-accumulate
// construction of the Hilbert curve).
__device__ __forceinline__ unsigned hilbert_d(int k, unsigned x, unsigned y)
{
    unsigned nside = 1u << k, dsum = 0;
    for (unsigned s = nside >> 1; s > 0; s >>= 1) {
        unsigned rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        dsum += s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = nside - 1 - x;
                y = nside - 1 - y;
            }
            unsigned t = x;
            x = y;
            y = t;
        }
    }
    return dsum;
}

__global__ void k_hilbert(const int2 *xy, int n, const int *bbox, int k, int shift, unsigned *key, int *hist)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int2 p = xy[i];
    unsigned cx = (unsigned)(p.x - bbox[0]) >> shift, cy = (unsigned)(p.y - bbox[1]) >> shift;
    unsigned lim = (1u << k) - 1;
    cx = min(cx, lim);
    cy = min(cy, lim);
    unsigned h = hilbert_d(k, cx, cy);
    key[i] = h;
    atomicAdd(hist + h, 1);
}

__global__ void k_place_order(int n, const unsigned *key, const int *off, int *fill, int *order, int base)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned h = key[i];
    order[off[h] + atomicAdd(fill + h, 1)] = base + i;
}

// first j >= 2 with orient(order[0], order[1], order[j]) != 0
__global__ void k_third(const int2 *xy, int n, const int *order, int *third)
{
    int2 a = xy[order[0]], b = xy[order[1]];
    for (int j = 2 + blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        if (orient2d(a, b, xy[order[j]]) != 0) atomicMin(third, j);
}

// The first triangle (a, b, c) and its three ghosts (c,b,inf), (a,c,inf), (b,a,inf).
__global__ void k_init(Dev d, const int *order, const int *third, int *tri_count, int s0)
{
    int a = order[0], b = order[1], c = order[*third];
    if (orient2d(d.xy[a], d.xy[b], d.xy[c]) < 0) {
        int t = b;
        b = c;
        c = t;
    }
    const int G = KDT_GHOST;
    const int t0 = s0, t1 = s0 + 1, t2 = s0 + 2, t3 = s0 + 3;
    d.tv[t0] = make_int4(a, b, c, ALIVE);
    d.tn[t0] = make_int4((t1 << 2) | 2, (t2 << 2) | 2, (t3 << 2) | 2, 0);
    d.tv[t1] = make_int4(c, b, G, ALIVE);
    d.tn[t1] = make_int4((t3 << 2) | 1, (t2 << 2) | 0, (t0 << 2) | 0, 0);
    d.tv[t2] = make_int4(a, c, G, ALIVE);
    d.tn[t2] = make_int4((t1 << 2) | 1, (t3 << 2) | 0, (t0 << 2) | 1, 0);
    d.tv[t3] = make_int4(b, a, G, ALIVE);
    d.tn[t3] = make_int4((t2 << 2) | 1, (t1 << 2) | 0, (t0 << 2) | 2, 0);
    d.pt_tri[a] = t0;
    d.pt_tri[b] = t0;
    d.pt_tri[c] = t0;
    *tri_count = s0 + 4;
}

// Insert the points at sorted positions (2j+1) * 2^level, each starting its walk at
// the triangle of its Hilbert predecessor (2j) * 2^level, already inserted.
__global__ void __launch_bounds__(WPB * 32) k_insert_level(Dev dp, const int *order, int level, int items,
                                                           int *tri_count, int nloc, int slot_end)
{
    KD_BLOCK_DEV(dp);
    __shared__ WarpShared shs[WPB];
    int wib = threadIdx.x >> 5;
    int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    int nw = gridDim.x * (blockDim.x >> 5);
    Warp w = make_warp(&shs[wib], gw + 1, gw * 7 + level * 1315423911u, d);
    // each warp takes a contiguous run of the level's points: runs are far apart along
    // the Hilbert curve, so the insertions in flight at any moment rarely share a cavity
    const int per = (items + nw - 1) / nw;
    const int jend = min(items, (gw + 1) * per);
    for (int j = gw * per; j < jend; ++j) {
        if (read_status(d)) break;
        long long i = ((long long)(2 * j + 1)) << level;
        if (i >= nloc) continue;
        int v = order[i];
        if (__shfl_sync(FULL, __ldcg(d.pt_tri + v), 0) >= 0) continue;  // one of the first three
        int parent = order[i - (1ll << level)];
        int start = __shfl_sync(FULL, __ldcg(d.pt_tri + parent), 0);
        if (start < 0) start = 0;
        int s = 0;
        if (w.lane == 0) s = atomicAdd(tri_count, 2);
        s = __shfl_sync(FULL, s, 0);
        if (s + 1 >= slot_end) {
            set_status(d, DEV_INTERNAL);
            break;
        }
        int2 q = d.xy[v];
        int rc = insert_staged(w, d, v, q, start, s, s + 1, false);
        if (rc == INS_GLOBAL) rc = insert_point(w, d, v, q, start, s, s + 1, false);
        if (rc) {
            if (rc > 0) set_status(d, rc);
            break;
        }
    }
    flush_counters(w, d);
}

// ------------------------------------------------------------------ batched build
//
// All instances of a batch built by one set of launches: per-instance bounding boxes,
// Hilbert keys offset by instance (so one counting sort orders every instance's points
// inside its own range of `order`), per-instance first triangles, and one launch per
// insertion level whose items are every instance's points of that level, back to back.

// bounding box of every instance (bbox[4 i .. 4 i + 3]) and the range check
__global__ void k_range_batch(const int2 *xy, int n, const int *pofs, int ninst, int bits, int *status, int *bbox)
{
    const long long lim = 1ll << bits;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int2 p = xy[i];
        if (p.x < 0 || p.y < 0 || p.x >= lim || p.y >= lim) atomicCAS(status, 0, DEV_RANGE);
        int *b = bbox + 4 * csr_find(pofs, ninst + 1, i);
        atomicMin(b + 0, p.x);
        atomicMin(b + 1, p.y);
        atomicMax(b + 2, p.x);
        atomicMax(b + 3, p.y);
    }
}

// Hilbert key of every point over its instance's grid (2^hk[i] cells a side, cell side
// 2^hshift[i] from the instance's minimum corner), offset by hbase[i] (the instances'
// grids one after another)
__global__ void k_hilbert_batch(const int2 *xy, int n, const int *pofs, int ninst, const int *bbox, const int *hk,
                                const int *hshift, const unsigned *hbase, unsigned *key, int *hist)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int inst = csr_find(pofs, ninst + 1, i);
        const int k = hk[inst], shift = hshift[inst];
        const int2 p = xy[i];
        unsigned cx = (unsigned)(p.x - bbox[4 * inst]) >> shift, cy = (unsigned)(p.y - bbox[4 * inst + 1]) >> shift;
        const unsigned lim = (1u << k) - 1;
        cx = min(cx, lim);
        cy = min(cy, lim);
        const unsigned h = hbase[inst] + hilbert_d(k, cx, cy);
        key[i] = h;
        atomicAdd(hist + h, 1);
    }
}

// per instance: the first position j >= 2 of its order whose point is not collinear
// with its first two (third[i], instance-local)
__global__ void k_third_batch(const int2 *xy, int n, const int *order, const int *pofs, int ninst, int *third)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int inst = csr_find(pofs, ninst + 1, j);
        const int p0 = pofs[inst];
        if (j - p0 < 2) continue;
        if (orient2d(xy[order[p0]], xy[order[p0 + 1]], xy[order[j]]) != 0) atomicMin(third + inst, j - p0);
    }
}

// per instance: its first triangle and three ghosts at its first slots (as k_init)
__global__ void k_init_batch(Dev d, const int *order, const int *third, const int *pofs, const int *tofs, int ninst,
                             int *tri_count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ninst; i += gridDim.x * blockDim.x) {
        const int p0 = pofs[i], s0 = tofs[i];
        int a = order[p0], b = order[p0 + 1], c = order[p0 + third[i]];
        if (orient2d(d.xy[a], d.xy[b], d.xy[c]) < 0) {
            int t = b;
            b = c;
            c = t;
        }
        const int G = KDT_GHOST;
        const int t0 = s0, t1 = s0 + 1, t2 = s0 + 2, t3 = s0 + 3;
        d.tv[t0] = make_int4(a, b, c, ALIVE);
        d.tn[t0] = make_int4((t1 << 2) | 2, (t2 << 2) | 2, (t3 << 2) | 2, 0);
        d.tv[t1] = make_int4(c, b, G, ALIVE);
        d.tn[t1] = make_int4((t3 << 2) | 1, (t2 << 2) | 0, (t0 << 2) | 0, 0);
        d.tv[t2] = make_int4(a, c, G, ALIVE);
        d.tn[t2] = make_int4((t1 << 2) | 1, (t3 << 2) | 0, (t0 << 2) | 1, 0);
        d.tv[t3] = make_int4(b, a, G, ALIVE);
        d.tn[t3] = make_int4((t2 << 2) | 1, (t1 << 2) | 0, (t0 << 2) | 2, 0);
        d.pt_tri[a] = t0;
        d.pt_tri[b] = t0;
        d.pt_tri[c] = t0;
        tri_count[i] = s0 + 4;
    }
}

// One insertion level of every instance: items lvoff[i] .. lvoff[i+1]-1 are instance
// i's points at its sorted positions (2j+1) * 2^level (as k_insert_level); each warp
// takes a contiguous run of the items, so its insertions are far apart along their
// instance's Hilbert curve.
__global__ void __launch_bounds__(WPB * 32) k_insert_level_batch(Dev dp, const int *order, int level, int items,
                                                                 const int *lvoff, const int *pofs, const int *tofs,
                                                                 int ninst, int *tri_count)
{
    KD_BLOCK_DEV(dp);
    __shared__ WarpShared shs[WPB];
    int wib = threadIdx.x >> 5;
    int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    int nw = gridDim.x * (blockDim.x >> 5);
    Warp w = make_warp(&shs[wib], gw + 1, gw * 7 + level * 1315423911u, d);
    const int per = (items + nw - 1) / nw;
    const int gend = min(items, (gw + 1) * per);
    int cur = -1, p0 = 0, nloc = 0;
    for (int g = gw * per; g < gend; ++g) {
        if (read_status(d)) break;
        const int inst = csr_find(lvoff, ninst + 1, g);
        if (inst != cur) {
            cur = inst;
            p0 = pofs[inst];
            nloc = pofs[inst + 1] - p0;
            set_instance(w, p0, nloc);
        }
        const int j = g - lvoff[inst];
        long long i = ((long long)(2 * j + 1)) << level;
        if (i >= nloc) continue;
        int v = order[p0 + i];
        if (__shfl_sync(FULL, __ldcg(d.pt_tri + v), 0) >= 0) continue;  // one of the first three
        int parent = order[p0 + i - (1ll << level)];
        int start = __shfl_sync(FULL, __ldcg(d.pt_tri + parent), 0);
        if (start < 0) start = tofs[inst];
        int s = 0;
        if (w.lane == 0) s = atomicAdd(tri_count + inst, 2);
        s = __shfl_sync(FULL, s, 0);
        if (s + 1 >= tofs[inst + 1]) {
            set_status(d, DEV_INTERNAL);
            break;
        }
        int2 q = d.xy[v];
        int rc = insert_staged(w, d, v, q, start, s, s + 1, false);
        if (rc == INS_GLOBAL) rc = insert_point(w, d, v, q, start, s, s + 1, false);
        if (rc) {
            if (rc > 0) set_status(d, rc);
            break;
        }
    }
    flush_counters(w, d);
}

// ------------------------------------------------------------------ export

__device__ __forceinline__ bool finite_alive(const int4 &v)
{
    return (v.w & ALIVE) && v.x >= 0 && v.y >= 0 && v.z >= 0;
}

__global__ void k_exp_count(TriHalf tv, int nslots, int *cnt, int idbase)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nslots; t += gridDim.x * blockDim.x) {
        int4 v = tv[t];
        if (!finite_alive(v)) continue;
        atomicAdd(cnt + min(v.x, min(v.y, v.z)) - idbase, 1);
    }
}

// rotate so the smallest id comes first (keeps the counter-clockwise order)
__global__ void k_exp_place(TriHalf tv, int nslots, const int *off, int *fill, int3 *out, int idbase)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nslots; t += gridDim.x * blockDim.x) {
        int4 v = tv[t];
        if (!finite_alive(v)) continue;
        int3 r;
        if (v.x < v.y && v.x < v.z) r = make_int3(v.x, v.y, v.z);
        else if (v.y < v.z) r = make_int3(v.y, v.z, v.x);
        else r = make_int3(v.z, v.x, v.y);
        r.x -= idbase;
        r.y -= idbase;
        r.z -= idbase;
        out[off[r.x] + atomicAdd(fill + r.x, 1)] = r;
    }
}

// sort each first-vertex segment by (second, third): segments are short (<= degree)
__global__ void k_exp_sortseg(int n, const int *off, const int *cnt, int3 *out)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        int c = cnt[a];
        if (c < 2) continue;
        int3 *s = out + off[a];
        for (int i = 1; i < c; ++i) {
            int3 x = s[i];
            int j = i - 1;
            while (j >= 0 && (s[j].y > x.y || (s[j].y == x.y && s[j].z > x.z))) {
                s[j + 1] = s[j];
                --j;
            }
            s[j + 1] = x;
        }
    }
}

// ------------------------------------------------------------------ verifier

__global__ void k_verify(Dev d, Inst I, int nslots, int *bad, int *alive, int *wraps)
{
    unsigned ex = 0, ti = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nslots; t += gridDim.x * blockDim.x) {
        int4 v = __ldcg(d.tv + t);
        if (!(v.w & ALIVE)) continue;
        atomicAdd(alive, 1);
        int4 nb = __ldcg(d.tn + t);
        int ghosts = (v.x < 0) + (v.y < 0) + (v.z < 0);
        if (ghosts > 1 || (v.x == v.y || v.y == v.z || v.x == v.z)) {
            atomicAdd(bad, 1);
            continue;
        }
        if (I.ninst > 1) {
            // every vertex and neighbour of a triangle belongs to the instance of its slot
            int inst = csr_find(I.tofs, I.ninst + 1, t);
            int plo = I.pofs[inst], phi = I.pofs[inst + 1], slo = I.tofs[inst], shi = I.tofs[inst + 1];
            bool own = true;
            for (int e = 0; e < 3; ++e) {
                int id = e == 0 ? v.x : (e == 1 ? v.y : v.z);
                int r = (e == 0 ? nb.x : (e == 1 ? nb.y : nb.z)) >> 2;
                own = own && (id == KDT_GHOST || (id >= plo && id < phi)) && r >= slo && r < shi;
            }
            if (!own) {
                atomicAdd(bad, 1);
                continue;
            }
        }
        if (ghosts == 0 && orient2d(d.xy[v.x], d.xy[v.y], d.xy[v.z]) <= 0) atomicAdd(bad, 1);
        if (nb.w != 0) atomicAdd(bad, 1);  // a claim left behind
        for (int e = 0; e < 3; ++e)
            if (check_edge(d, t, v, nb, e, &ex, &ti) != 0) atomicAdd(bad, 1);
        if (ghosts == 1) {
            int wr = hull_wrap(d, v, nb);
            if (wr) atomicAdd(wraps, wr);
        }
    }
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d.n; p += gridDim.x * blockDim.x) {
        int t = d.pt_tri[p];
        if (t < 0 || t >= nslots) {
            atomicAdd(bad, 1);
            continue;
        }
        int4 v = d.tv[t];
        if (!(v.w & ALIVE) || (v.x != p && v.y != p && v.z != p)) atomicAdd(bad, 1);
    }
}

// ------------------------------------------------------------------ misc

__global__ void k_set_positions(int2 *xy, const int3 *moves, int m)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) xy[moves[i].x] = make_int2(moves[i].y, moves[i].z);
}

__global__ void k_restore_positions(int2 *xy, const int3 *moves, const int2 *old_xy, int m)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) xy[moves[i].x] = old_xy[i];
}

__global__ void k_fill_int(int *p, int n, int v)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_predicates(const int2 *xy, const int4 *quads, int m, int4 *out, int use_filter)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int4 q = quads[i];
    int2 a = xy[q.x], b = xy[q.y], c = xy[q.z], dd = xy[q.w];
    unsigned ex = 0, ti = 0;
    out[i] = make_int4(orient2d(a, b, c), incircle_exact(a, b, c, dd), incircle_filter(a, b, c, dd),
                       incircle_sos(q.x, q.y, q.z, q.w, a, b, c, dd, use_filter != 0, &ex, &ti));
}

}  // namespace kd
