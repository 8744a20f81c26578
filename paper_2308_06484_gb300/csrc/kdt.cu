// C-ABI and host orchestration of the GB300 kinetic Delaunay library.
// The declarations, argument conventions and error behaviour are in include/kdt.h.
//
// A handle holds one or more independent instances in one store: instance i owns
// the global point ids pofs[i] .. pofs[i+1]-1, the triangle slots tofs[i] ..
// tofs[i+1]-1 (2 n_i - 2 of them) and the partitions cofs[i] .. cofs[i+1]-1.  Each
// instance is its own triangulation (its own sphere with the shared vertex at
// infinity), so every kernel works on the whole store at once; only builds and
// exports go instance by instance.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <new>
#include <vector>

#include "../../include/kdt.h"
#include "kdt_kernels.cuh"
#include "kdt_dcalc.cuh"
#include "kdt_plan.cuh"
#include "kdt_tc.cuh"

using namespace kd;

namespace {

constexpr int ABI_VERSION = 7;

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// the partition sizes and warps per partition the autotuner tries
constexpr int TUNE_PPP[3] = {128, 256, 512};
constexpr int TUNE_WPP[3] = {1, 2, 4};
constexpr int TUNE_STEPS = 1;  // timed steps per configuration

}  // namespace

struct kdt {
    int device = 0;
    cudaStream_t stream = nullptr;
    kdt_config cfg{};
    int64_t n = 0;  // points (all instances)
    int cap = 0;    // triangle slots (all instances)
    bool built = false;
    int stamp = 0;
    // instances
    int ninst = 0;
    std::vector<int> pofs, tofs, cofs, igrid;  // host copies
    int *d_pofs = nullptr, *d_cofs = nullptr, *d_grid = nullptr, *d_tofs = nullptr;
    int *d_moff = nullptr, *h_moff = nullptr;  // move offsets: ctl + 4 and hctl + 4
    int ncells = 0;          // partitions (all instances)
    int stride = 1;          // the scattering stride of the partitions (Inst.stride)
    int ncells_cap = 0;      // entries of the per-partition arrays (more than ncells when the
                             // quad-tree is re-divided at every step: one per fine cell)
    int ppp = 256;           // points per partition in use
    int wpp = 1;             // warps per partition in use
    // state
    int2 *xy = nullptr;
    int *pt_tri = nullptr;
    int *pt_stamp = nullptr;
    int4 *tri = nullptr;  // 2 x cap int4: the 32-byte triangle records (TriHalf)
    int *scal = nullptr;                     // S_NUM device scalars
    unsigned long long *counters = nullptr;  // C_SLOTS
    int *dirty = nullptr;
    int dirty_cap = 0;
    int *viol = nullptr;
    int viol_cap = 0;
    // step buffers
    int mcap = 0;
    int3 *moves = nullptr;   // host moves copied in
    int3 *gmoves = nullptr;  // moves with global ids (written by the intake)
    int2 *old_xy = nullptr;
    int *next = nullptr;     // per-partition move lists
    int *head = nullptr;
    int4 *deferred = nullptr;
    int *scan_tmp = nullptr;
    int scan_tmp_cap = 0;
    // build / export temporaries (kept between calls)
    Buf key, bord, hist, hoff, exp_cnt, exp_off, exp_fill, exp_out;
    Buf btab, blev;  // batched build: per-instance tables, per-level item offsets
    // d-calculation: neighbour lists, results, running minimum (per N)
    Buf nb_deg, nb_off, nb_list, dc_dist, dc_cmin, dc_scal;
    int64_t d2_run = INT64_MAX;
    int d_n = 0;
    // the displacement rule (kdt_config.rebuild_displacement): running per-partition
    // d_local^2 (INT64_MAX = unknown), valid since the partitions were last set
    unsigned long long *dloc2 = nullptr;
    bool dloc_valid = false;
    // step planner (kdt_config.plan): per-partition cost estimates, the order of the
    // partitions, class sizes and cursors, and the network's guess per point
    float *pcost = nullptr;
    int *order = nullptr;
    int *ohist = nullptr;
    signed char *pguess = nullptr;
    // the network on the tensor cores (kdt_config.plan bit 2): every move's features and
    // its partition (-1: no features), written by the planner
    float *pfeat = nullptr;
    int *ppart = nullptr;
    // quad-tree partitions (kdt_config.quadtree): leaf of every fine cell, the square
    int *qmap = nullptr;
    int qx0 = 0, qy0 = 0, qshift = 0, qF = 0, qleaves = 0, qleaf_side_lg = 0, qD = 0;
    // re-divided at every step (kdt_config.quadtree = 2): points per fine cell, the count
    // pyramid above it, and per fine cell (Morton order) the leaf-start flags, their
    // prefix counts and the leaf levels
    int *qhist = nullptr, *qpyr = nullptr, *qflag = nullptr, *qpre = nullptr;
    unsigned char *qlev = nullptr;
    // graph-launched step: control words (moves, stamp, moves address) followed by the
    // move offsets of the instances, copied in one piece each step, and the graph
    int *ctl = nullptr;   // device
    int *hctl = nullptr;  // pinned host
    cudaStream_t cstream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_gen = -1;  // buffer generation the graph was captured for
    int gen = 0;         // bumped whenever step buffers or tables change
    // autotuner state: configuration index being timed, accumulated times
    int tune_idx = -1;
    int tune_done = 0;
    int tune_count = 0;
    double tune_ms[9] = {0};
    // host side
    int *hscal = nullptr;  // pinned copy of the scalars
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
    kdt_stats stats{};
    // learned locate proposal and its training rows (kdt_mlp.cuh)
    unsigned short *mlp_w = nullptr;  // library copy of the proposal's BF16 parameters
    bool prop_on = false;
    float *trace_x = nullptr;         // caller's buffers
    int *trace_y = nullptr;
    int trace_cap = 0;
    int *trace_count = nullptr;       // device counter
    float *mlp_part = nullptr;        // per-block partial gradients of k_mlp_grad
    int mlp_part_blocks = 0;
    // per-warp global scratch of the kinetic launch for deletions of degree > KMAX
    int *big = nullptr;
    long long big_warps = 0;
};

namespace {

#define CK(call)                                    \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return KDT_ERR_CUDA; \
    } while (0)

int dev_to_abi(int s)
{
    switch (s) {
    case DEV_OK: return KDT_OK;
    case DEV_RETRY: return KDT_ERR_RETRY_EXHAUSTED;
    case DEV_DEGREE: return KDT_ERR_RETRY_EXHAUSTED;
    case DEV_DUPLICATE: return KDT_ERR_DUPLICATE;
    case DEV_DUP_ID: return KDT_ERR_DUPLICATE;
    case DEV_DEGENERATE: return KDT_ERR_DEGENERATE;
    case DEV_ARG: return KDT_ERR_ARG;
    case DEV_RANGE: return KDT_ERR_RANGE;
    default: return KDT_ERR_INTERNAL;
    }
}

// Where a caller's pointer points: host memory (pageable or pinned), memory the
// handle's GPU reads directly (its own device memory, or managed memory), or device
// memory of another GPU, which every entry point rejects with KDT_ERR_ARG before
// launching anything (without peer access a kernel touching it would fault).
enum PtrKind { PTR_HOST = 0, PTR_DEV = 1, PTR_FOREIGN = 2 };

PtrKind ptr_kind(const void *p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return PTR_HOST;
    }
    if (a.type == cudaMemoryTypeManaged) return PTR_DEV;
    if (a.type == cudaMemoryTypeDevice) return a.device == device ? PTR_DEV : PTR_FOREIGN;
    return PTR_HOST;
}

// true iff p is memory the handle's GPU reads directly (see ptr_kind)
bool on_device(const kdt *h, const void *p) { return ptr_kind(p, h->device) == PTR_DEV; }

// true iff p is device memory of another GPU
bool foreign(const kdt *h, const void *p) { return p && ptr_kind(p, h->device) == PTR_FOREIGN; }

int grow(Buf &b, size_t bytes)
{
    if (b.bytes >= bytes) return 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) return KDT_ERR_CUDA;
    b.bytes = bytes;
    return 0;
}

template <class T>
int dalloc(T **p, size_t count)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T)) == cudaSuccess ? 0 : KDT_ERR_CUDA;
}

void free_buf(Buf &b)
{
    if (b.p) cudaFree(b.p);
    b = Buf();
}

int sm_count(int device)
{
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v > 0 ? v : 1;
}

Dev make_dev(kdt *h)
{
    Dev d;
    d.xy = h->xy;
    d.pt_tri = h->pt_tri;
    d.tv = TriHalf{h->tri};
    d.tn = TriHalf{h->tri + 1};
    d.n = (int)h->n;
    d.cap = h->cap;
    d.status = h->scal + S_STATUS;
    d.dirty = h->dirty;
    d.dirty_count = h->scal + S_DIRTY;
    d.dirty_cap = h->dirty_cap;
    d.pt_stamp = h->pt_stamp;
    d.stamp = h->stamp;
    d.counters = h->counters;
    d.use_filter = h->cfg.filter;
    d.retry_cap = h->cfg.retry_cap;
    d.ctl = nullptr;
    d.viol = h->viol;
    d.viol_count = h->scal + S_VIOL;
    d.viol_cap = h->viol_cap;
    d.rlo = 0;
    d.rn = (int)std::max<int64_t>(h->n, 1);
    d.mlp = h->prop_on ? h->mlp_w : nullptr;
    d.pguess = h->prop_on && (h->cfg.plan & PLAN_NETWORK) ? h->pguess : nullptr;
    d.trace_x = h->trace_x;
    d.trace_y = h->trace_y;
    d.trace_count = h->trace_count;
    d.trace_cap = h->trace_cap;
    d.big = nullptr;  // set for the kinetic launch only (enqueue_step)
    d.variant = h->cfg.variant;
    d.timeline = (h->cfg.debug >> 1) & 1;
    return d;
}

Inst make_inst(kdt *h)
{
    Inst I;
    I.pofs = h->d_pofs;
    I.cofs = h->d_cofs;
    I.grid = h->d_grid;
    I.tofs = h->d_tofs;
    I.moff = h->d_moff;
    I.ninst = h->ninst;
    I.qmap = h->qmap;
    I.qx0 = h->qx0;
    I.qy0 = h->qy0;
    I.qshift = h->qshift;
    I.qF = h->qF;
    I.order = (h->cfg.plan & PLAN_ORDER) ? h->order : nullptr;
    I.qhist = h->qhist;
    I.stride = h->cfg.partition_order == 0 && !h->qhist ? h->stride : 1;
    I.ncells_dyn = h->qhist ? h->scal + S_NCELLS : nullptr;
    return I;
}

// exclusive scan of n ints; *total receives the sum
int scan(kdt *h, const int *in, int *out, int n, int *total, cudaStream_t st)
{
    int tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles < 1) tiles = 1;
    if (tiles + 1 > h->scan_tmp_cap) {
        int c = tiles + 1024;
        if (dalloc(&h->scan_tmp, (size_t)c)) return KDT_ERR_CUDA;
        h->scan_tmp_cap = c;
        h->gen++;  // a captured step graph may hold the old pointer
    }
    k_scan_tile<<<tiles, SCAN_THREADS, 0, st>>>(in, out, n, h->scan_tmp);
    k_scan_sums<<<1, 1024, 0, st>>>(h->scan_tmp, tiles, total);
    k_scan_add<<<tiles, SCAN_THREADS, 0, st>>>(out, n, h->scan_tmp);
    h->stats.kernel_launches += 3;
    CK(cudaGetLastError());
    return 0;
}

int sync_scalars(kdt *h)
{
    CK(cudaMemcpyAsync(h->hscal, h->scal, S_NUM * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return 0;
}

int warp_grid(kdt *h, long long items, int per_sm_blocks)
{
    long long blocks = (items + WPB - 1) / WPB;
    long long lim = (long long)sm_count(h->device) * per_sm_blocks;
    if (blocks > lim) blocks = lim;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

int thread_grid(kdt *h, long long items, int threads)
{
    long long blocks = (items + threads - 1) / threads;
    long long lim = (long long)sm_count(h->device) * 32;
    if (blocks > lim) blocks = lim;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

// blocks of the kinetic kernel that fit on the GPU at once (persistent launch)
int kinetic_blocks(kdt *h)
{
    int per_sm = 0;
    const bool seven = h->cfg.kinetic_blocks_per_sm == 7;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, seven ? k_kinetic<7> : k_kinetic<6>, WPB * 32, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 4;
    return sm_count(h->device) * per_sm;
}

// Certify slots [s0, s0 + nslots) (or the dirty list when !full), then repair until
// no violation is left.  A full pass must see `wraps` hull windings (one per
// instance in the range).  Returns a CUDA/ABI error; the device status goes to
// *dev_status.
int certify_and_repair(kdt *h, bool full, int s0, int nslots, int wraps, int *dev_status)
{
    Dev d = make_dev(h);
    if (full && d.retry_cap < 4096) d.retry_cap = 4096;
    int lo = 0;
    for (int round = 0; round < 64; ++round) {
        CK(cudaMemsetAsync(h->scal + S_VIOL, 0, sizeof(int), h->stream));
        CK(cudaMemsetAsync(h->scal + S_WRAPS, 0, sizeof(int), h->stream));
        if (full) {
            k_certify_all<<<thread_grid(h, nslots, 256), 256, 0, h->stream>>>(d, s0, nslots, h->viol, h->scal + S_VIOL,
                                                                             h->viol_cap, h->scal + S_WRAPS);
        } else {
            k_certify<<<thread_grid(h, 65536, 256), 256, 0, h->stream>>>(d, lo, h->viol, h->scal + S_VIOL,
                                                                        h->viol_cap);
        }
        h->stats.kernel_launches++;
        CK(cudaGetLastError());
        if (sync_scalars(h)) return KDT_ERR_CUDA;
        *dev_status = h->hscal[S_STATUS];
        if (*dev_status) return 0;
        int nv = h->hscal[S_VIOL];
        h->stats.violations += nv;
        if (nv == 0) {
            // every edge is locally Delaunay; after a full pass each hull winds once
            if (full && h->hscal[S_WRAPS] != wraps) *dev_status = DEV_INTERNAL;
            return 0;
        }
        if (nv > h->viol_cap) nv = h->viol_cap;  // the rest is found again next round
        int dirty_before = h->hscal[S_DIRTY];
        lo = dirty_before;
        k_fixup<<<warp_grid(h, nv, 16), WPB * 32, 0, h->stream>>>(d, h->viol, nv);
        h->stats.kernel_launches++;
        CK(cudaGetLastError());
        if (sync_scalars(h)) return KDT_ERR_CUDA;
        *dev_status = h->hscal[S_STATUS];
        if (*dev_status) return 0;
        if (!full && h->hscal[S_DIRTY] > h->dirty_cap) {
            full = true;
            s0 = 0;
            nslots = h->cap;
            wraps = h->ninst;
        }
    }
    *dev_status = DEV_INTERNAL;
    return 0;
}

// Build the triangulation of instance i from the positions in h->xy: Hilbert order
// over a grid on its bounding box, the first non-degenerate triangle, then parallel
// insertion level by level (positions (2j+1) * 2^level walk from position 2j * 2^level),
// then certification and repair.  Returns an ABI code.
int rebuild_instance(kdt *h, int i)
{
    const int p0 = h->pofs[i], n = h->pofs[i + 1] - p0;
    const int s0 = h->tofs[i], capi = h->tofs[i + 1] - s0;
    cudaStream_t st = h->stream;
    Dev d = make_dev(h);
    d.dirty_cap = 0;  // the build certifies every slot of the instance instead
    if (d.retry_cap < 32768) d.retry_cap = 32768;  // the step's cap does not apply to builds
    d.rlo = p0;
    d.rn = n;
    CK(cudaMemsetAsync(h->scal, 0, S_NUM * sizeof(int), st));
    int init_bbox[4] = {INT_MAX, INT_MAX, INT_MIN, INT_MIN};
    CK(cudaMemcpyAsync(h->scal + S_MINX, init_bbox, sizeof init_bbox, cudaMemcpyHostToDevice, st));
    int third0 = INT_MAX;
    CK(cudaMemcpyAsync(h->scal + S_THIRD, &third0, sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->tri + 2 * (size_t)s0, 0, 2 * (size_t)capi * sizeof(int4), st));
    k_fill_int<<<thread_grid(h, n, 256), 256, 0, st>>>(h->pt_tri + p0, n, -1);
    k_range<<<thread_grid(h, n, 256), 256, 0, st>>>(h->xy + p0, n, h->cfg.domain_bits, h->scal + S_STATUS,
                                                    h->scal + S_MINX);
    h->stats.kernel_launches += 2;
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    if (h->hscal[S_STATUS]) return dev_to_abi(h->hscal[S_STATUS]);
    int k = 1;
    while ((1ll << (2 * k)) < (long long)n && k < 14) ++k;
    long long span = (long long)std::max(h->hscal[S_MAXX] - h->hscal[S_MINX], h->hscal[S_MAXY] - h->hscal[S_MINY]) + 1;
    int shift = 0;
    while ((span >> shift) > (1ll << k)) ++shift;
    size_t ncell = (size_t)1 << (2 * k);
    if (grow(h->key, (size_t)n * 4) || grow(h->bord, (size_t)n * 4) || grow(h->hist, ncell * 4) ||
        grow(h->hoff, ncell * 4))
        return KDT_ERR_CUDA;
    unsigned *key = (unsigned *)h->key.p;
    int *order = (int *)h->bord.p, *hist = (int *)h->hist.p, *hoff = (int *)h->hoff.p;
    CK(cudaMemsetAsync(hist, 0, ncell * 4, st));
    k_hilbert<<<(n + 255) / 256, 256, 0, st>>>(h->xy + p0, n, h->scal + S_MINX, k, shift, key, hist);
    h->stats.kernel_launches++;
    if (scan(h, hist, hoff, (int)ncell, h->scal + S_TOTAL, st)) return KDT_ERR_CUDA;
    CK(cudaMemsetAsync(hist, 0, ncell * 4, st));
    k_place_order<<<(n + 255) / 256, 256, 0, st>>>(n, key, hoff, hist, order, p0);
    k_third<<<thread_grid(h, n, 256), 256, 0, st>>>(h->xy, n, order, h->scal + S_THIRD);
    h->stats.kernel_launches += 2;
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    if (h->hscal[S_THIRD] == INT_MAX) return KDT_ERR_DEGENERATE;
    k_init<<<1, 1, 0, st>>>(d, order, h->scal + S_THIRD, h->scal + S_TRIS, s0);
    h->stats.kernel_launches++;
    int K = 0;
    while ((1ll << (K + 1)) < (long long)n) ++K;
    long long inserted = 3;
    for (int lev = K; lev >= 0; --lev) {
        long long items = ((long long)n - 1 + (1ll << lev)) >> (lev + 1);  // odd multiples of 2^lev below n
        if (items <= 0) continue;
        // about 16 triangles of room per concurrent insertion: more warps than that only
        // collide on the same cavities (claims fail, back off, retry)
        long long conc = inserted / 8;
        if (conc < 8) conc = 8;
        if (h->cfg.build_warps > 0) conc = h->cfg.build_warps;
        long long warps = items < conc ? items : conc;
        int blocks = warp_grid(h, warps, 64), threads = WPB * 32;
        if (h->cfg.build_warps > 0 && h->cfg.build_warps < WPB) {
            blocks = 1;
            threads = 32 * h->cfg.build_warps;
        }
        k_insert_level<<<blocks, threads, 0, st>>>(d, order, lev, (int)items, h->scal + S_TRIS, n, s0 + capi);
        h->stats.kernel_launches++;
        CK(cudaGetLastError());
        inserted += items;
    }
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    if (h->hscal[S_STATUS]) return dev_to_abi(h->hscal[S_STATUS]);
    if (h->hscal[S_TRIS] != s0 + capi) return KDT_ERR_INTERNAL;
    int ds = 0;
    if (certify_and_repair(h, true, s0, capi, 1, &ds)) return KDT_ERR_CUDA;
    if (ds) return dev_to_abi(ds);
    return KDT_OK;
}

// Build the triangulations of every instance of a batch from the positions in h->xy in
// one set of launches (the steps of rebuild_instance, each over all instances at once;
// see the batched build kernels).  Returns an ABI code, or BATCH_TOO_WIDE (nothing
// built) when the instances' Hilbert grids together exceed 2^31 cells.
constexpr int BATCH_TOO_WIDE = 1;

int rebuild_batch(kdt *h)
{
    const int ni = h->ninst, n = (int)h->n;
    cudaStream_t st = h->stream;
    Dev d = make_dev(h);
    d.dirty_cap = 0;
    if (d.retry_cap < 32768) d.retry_cap = 32768;
    // per-instance tables: bbox (4), hk, hshift, hbase (ni + 1), third, tri_count
    const size_t tab_ints = 4 * (size_t)ni + 5 * (size_t)ni + 1;
    if (grow(h->btab, tab_ints * sizeof(int))) return KDT_ERR_CUDA;
    int *bbox = (int *)h->btab.p, *hk = bbox + 4 * ni, *hsh = hk + ni, *third = hsh + ni, *tcount = third + ni;
    unsigned *hbase = (unsigned *)(tcount + ni);
    std::vector<int> hb(4 * (size_t)ni);
    for (int i = 0; i < ni; ++i) {
        hb[4 * i] = INT_MAX;
        hb[4 * i + 1] = INT_MAX;
        hb[4 * i + 2] = INT_MIN;
        hb[4 * i + 3] = INT_MIN;
    }
    CK(cudaMemsetAsync(h->scal, 0, S_NUM * sizeof(int), st));
    CK(cudaMemcpyAsync(bbox, hb.data(), hb.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->tri, 0, 2 * (size_t)h->cap * sizeof(int4), st));
    k_fill_int<<<thread_grid(h, n, 256), 256, 0, st>>>(h->pt_tri, n, -1);
    k_range_batch<<<thread_grid(h, n, 256), 256, 0, st>>>(h->xy, n, h->d_pofs, ni, h->cfg.domain_bits,
                                                          h->scal + S_STATUS, bbox);
    h->stats.kernel_launches += 2;
    CK(cudaMemcpyAsync(hb.data(), bbox, hb.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    if (h->hscal[S_STATUS]) return dev_to_abi(h->hscal[S_STATUS]);
    // Hilbert grids per instance (as rebuild_instance), laid one after another
    std::vector<int> kk(ni), sh(ni), th(ni, INT_MAX);
    std::vector<unsigned> base(ni + 1, 0);
    int Kmax = 0;
    for (int i = 0; i < ni; ++i) {
        const int nn = h->pofs[i + 1] - h->pofs[i];
        int k = 1;
        while ((1ll << (2 * k)) < (long long)nn && k < 14) ++k;
        long long span = (long long)std::max(hb[4 * i + 2] - hb[4 * i], hb[4 * i + 3] - hb[4 * i + 1]) + 1;
        int shift = 0;
        while ((span >> shift) > (1ll << k)) ++shift;
        kk[i] = k;
        sh[i] = shift;
        if ((unsigned long long)base[i] + (1ull << (2 * k)) > 0x7fffffffull) return BATCH_TOO_WIDE;
        base[i + 1] = base[i] + (1u << (2 * k));
        int K = 0;
        while ((1ll << (K + 1)) < (long long)nn) ++K;
        Kmax = std::max(Kmax, K);
    }
    const size_t ncell = base[ni];
    if (grow(h->key, (size_t)n * 4) || grow(h->bord, (size_t)n * 4) || grow(h->hist, ncell * 4) ||
        grow(h->hoff, ncell * 4))
        return KDT_ERR_CUDA;
    unsigned *key = (unsigned *)h->key.p;
    int *order = (int *)h->bord.p, *hist = (int *)h->hist.p, *hoff = (int *)h->hoff.p;
    CK(cudaMemcpyAsync(hk, kk.data(), ni * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(hsh, sh.data(), ni * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(hbase, base.data(), (ni + 1) * sizeof(unsigned), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(third, th.data(), ni * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(hist, 0, ncell * 4, st));
    k_hilbert_batch<<<thread_grid(h, n, 256), 256, 0, st>>>(h->xy, n, h->d_pofs, ni, bbox, hk, hsh, hbase, key, hist);
    h->stats.kernel_launches++;
    if (scan(h, hist, hoff, (int)ncell, h->scal + S_TOTAL, st)) return KDT_ERR_CUDA;
    CK(cudaMemsetAsync(hist, 0, ncell * 4, st));
    k_place_order<<<(n + 255) / 256, 256, 0, st>>>(n, key, hoff, hist, order, 0);
    k_third_batch<<<thread_grid(h, n, 256), 256, 0, st>>>(h->xy, n, order, h->d_pofs, ni, third);
    h->stats.kernel_launches += 2;
    CK(cudaMemcpyAsync(th.data(), third, ni * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < ni; ++i)
        if (th[i] == INT_MAX) return KDT_ERR_DEGENERATE;
    k_init_batch<<<thread_grid(h, ni, 128), 128, 0, st>>>(d, order, third, h->d_pofs, h->d_tofs, ni, tcount);
    h->stats.kernel_launches++;
    // the items of every level: instance i's positions (2j+1) * 2^level below n_i
    std::vector<int> lv((size_t)(Kmax + 1) * (ni + 1), 0);
    for (int lev = 0; lev <= Kmax; ++lev) {
        int *o = lv.data() + (size_t)lev * (ni + 1);
        for (int i = 0; i < ni; ++i) {
            const long long nn = h->pofs[i + 1] - h->pofs[i];
            const long long items = (nn - 1 + (1ll << lev)) >> (lev + 1);
            o[i + 1] = o[i] + (int)std::max(0ll, items);
        }
    }
    if (grow(h->blev, lv.size() * sizeof(int))) return KDT_ERR_CUDA;
    CK(cudaMemcpyAsync(h->blev.p, lv.data(), lv.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    std::vector<long long> inserted(ni, 3);
    for (int lev = Kmax; lev >= 0; --lev) {
        const int *o = lv.data() + (size_t)lev * (ni + 1);
        const int items = o[ni];
        if (items <= 0) continue;
        // about 16 triangles of room per concurrent insertion in every instance
        long long conc = 0;
        for (int i = 0; i < ni; ++i)
            if (o[i + 1] > o[i]) conc += std::max(8ll, inserted[i] / 8);
        if (h->cfg.build_warps > 0) conc = h->cfg.build_warps;
        long long warps = std::min<long long>(items, conc);
        k_insert_level_batch<<<warp_grid(h, warps, 64), WPB * 32, 0, st>>>(
            d, order, lev, items, (const int *)h->blev.p + (size_t)lev * (ni + 1), h->d_pofs, h->d_tofs, ni, tcount);
        h->stats.kernel_launches++;
        CK(cudaGetLastError());
        for (int i = 0; i < ni; ++i) inserted[i] += o[i + 1] - o[i];
    }
    std::vector<int> tc(ni);
    CK(cudaMemcpyAsync(tc.data(), tcount, ni * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    if (h->hscal[S_STATUS]) return dev_to_abi(h->hscal[S_STATUS]);
    for (int i = 0; i < ni; ++i)
        if (tc[i] != h->tofs[i + 1]) return KDT_ERR_INTERNAL;
    int ds = 0;
    if (certify_and_repair(h, true, 0, h->cap, ni, &ds)) return KDT_ERR_CUDA;
    if (ds) return dev_to_abi(ds);
    return KDT_OK;
}

int rebuild_all(kdt *h)
{
    h->built = false;
    h->stamp++;
    int rc = h->ninst > 1 && h->cfg.batch_build ? rebuild_batch(h) : BATCH_TOO_WIDE;
    if (rc != BATCH_TOO_WIDE && rc != KDT_OK) return rc;
    if (rc == BATCH_TOO_WIDE) {
        for (int i = 0; i < h->ninst; ++i) {
            const int ri = rebuild_instance(h, i);
            if (ri) return ri;
        }
    }
    h->built = true;
    h->stats.rebuilds++;
    return KDT_OK;
}

int ensure_moves(kdt *h, int64_t m)
{
    if (m <= h->mcap) return 0;
    int c = (int)std::max<int64_t>(m, 1024);
    if (dalloc(&h->moves, c) || dalloc(&h->gmoves, c) || dalloc(&h->old_xy, c) || dalloc(&h->next, c) ||
        dalloc(&h->deferred, c))
        return KDT_ERR_CUDA;
    if ((h->cfg.plan & PLAN_TENSOR) && (dalloc(&h->pfeat, (size_t)c * MLP_IN) || dalloc(&h->ppart, c)))
        return KDT_ERR_CUDA;
    h->mcap = c;
    long long dc = 64ll * c + 4096;
    if (dc > (1ll << 30)) dc = 1ll << 30;
    if (dalloc(&h->dirty, (size_t)dc)) return KDT_ERR_CUDA;
    h->dirty_cap = (int)dc;
    h->gen++;
    return 0;
}

// partitions of every instance for `ppp` points per partition (or the configured
// grid for a single instance), uploaded with the instance tables
int set_partitions(kdt *h, int ppp)
{
    h->ppp = ppp;
    h->cofs.assign(h->ninst + 1, 0);
    h->igrid.assign(h->ninst, 1);
    long long cells = 0;
    if (h->qmap) {
        // the quad-tree's leaves (one instance)
        h->igrid[0] = 0;
        h->cofs[0] = 0;
        cells = h->qleaves;
    }
    for (int i = 0; i < h->ninst && !h->qmap; ++i) {
        int ni = h->pofs[i + 1] - h->pofs[i];
        int G;
        if (h->ninst == 1 && h->cfg.grid > 0) {
            G = h->cfg.grid;
        } else {
            G = (int)std::lround(std::sqrt((double)ni / (double)ppp));
            G = std::max(1, std::min(G, 4096));
        }
        h->igrid[i] = G;
        h->cofs[i] = (int)cells;
        cells += (long long)G * G;
    }
    if (cells > INT_MAX / 8) return KDT_ERR_ARG;
    h->cofs[h->ninst] = (int)cells;
    h->ncells = (int)cells;
    // a stride near the golden ratio of the partition count, coprime with it
    long long stride = std::max(1ll, std::llround(0.6180339887498949 * (double)cells));
    while (std::gcd(stride, cells) != 1) ++stride;
    h->stride = (int)stride;
    // a quad-tree re-divided at every step has at most one leaf per fine cell
    const long long cap = h->qhist ? (long long)h->qF * h->qF : cells;
    h->ncells_cap = (int)cap;
    if (dalloc(&h->head, (size_t)cap) || dalloc(&h->d_cofs, h->ninst + 1) || dalloc(&h->d_grid, h->ninst) ||
        dalloc(&h->dloc2, (size_t)cap) || dalloc(&h->pcost, (size_t)cap) || dalloc(&h->order, (size_t)cap))
        return KDT_ERR_CUDA;
    k_fill_u64<<<thread_grid(h, cap, 256), 256, 0, h->stream>>>(h->dloc2, cap, (unsigned long long)INT64_MAX);
    h->stats.kernel_launches++;
    h->dloc_valid = false;
    CK(cudaMemcpy(h->d_cofs, h->cofs.data(), (h->ninst + 1) * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_grid, h->igrid.data(), h->ninst * sizeof(int), cudaMemcpyHostToDevice));
    h->gen++;
    return 0;
}

void drop_graph(kdt *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    h->graph_gen = -1;
}

void free_state(kdt *h)
{
    drop_graph(h);
    h->gen++;
    void *ps[] = {h->xy, h->pt_tri, h->pt_stamp, h->tri, h->viol, h->moves, h->gmoves, h->old_xy,
                  h->next, h->head, h->deferred, h->dirty, h->scan_tmp, h->d_pofs, h->d_cofs, h->d_grid,
                  h->ctl, h->d_tofs, h->qmap, h->dloc2, h->pcost, h->order, h->ohist, h->pguess,
                  h->qhist, h->qpyr, h->qflag, h->qpre, h->qlev, h->pfeat, h->ppart};
    for (void *p : ps)
        if (p) cudaFree(p);
    if (h->hctl) cudaFreeHost(h->hctl);
    h->ctl = nullptr;
    h->hctl = nullptr;
    h->xy = nullptr; h->pt_tri = nullptr; h->pt_stamp = nullptr; h->tri = nullptr;
    h->viol = nullptr; h->moves = nullptr; h->gmoves = nullptr; h->old_xy = nullptr; h->next = nullptr;
    h->head = nullptr; h->deferred = nullptr; h->dirty = nullptr; h->scan_tmp = nullptr;
    h->d_pofs = nullptr; h->d_cofs = nullptr; h->d_grid = nullptr; h->d_moff = nullptr; h->h_moff = nullptr;
    h->d_tofs = nullptr;
    h->qmap = nullptr;
    h->qhist = nullptr;
    h->qpyr = nullptr;
    h->qflag = nullptr;
    h->qpre = nullptr;
    h->qlev = nullptr;
    h->dloc2 = nullptr;
    h->dloc_valid = false;
    h->pcost = nullptr;
    h->order = nullptr;
    h->ohist = nullptr;
    h->pguess = nullptr;
    h->pfeat = nullptr;
    h->ppart = nullptr;
    h->qleaves = 0;
    h->mcap = 0; h->dirty_cap = 0; h->scan_tmp_cap = 0;
    Buf *bs[] = {&h->key, &h->bord, &h->hist, &h->hoff, &h->exp_cnt, &h->exp_off, &h->exp_fill, &h->exp_out,
                 &h->btab, &h->blev,
                 &h->nb_deg, &h->nb_off, &h->nb_list, &h->dc_dist, &h->dc_cmin, &h->dc_scal};
    for (Buf *b : bs) free_buf(*b);
    h->n = 0;
    h->cap = 0;
    h->ninst = 0;
    h->built = false;
    h->tune_idx = -1;
    h->tune_done = 0;
}

// state for instances with point offsets `offs` (host, n_inst + 1 entries)
int alloc_state(kdt *h, const int64_t *offs, int n_inst)
{
    h->ninst = n_inst;
    h->pofs.assign(n_inst + 1, 0);
    h->tofs.assign(n_inst + 1, 0);
    for (int i = 0; i <= n_inst; ++i) {
        h->pofs[i] = (int)offs[i];
        h->tofs[i] = (int)(2 * offs[i] - 2 * i);
    }
    h->n = offs[n_inst];
    h->cap = h->tofs[n_inst];
    h->built = false;
    if (dalloc(&h->xy, h->n) || dalloc(&h->pt_tri, h->n) || dalloc(&h->pt_stamp, h->n) || dalloc(&h->tri, 2 * (size_t)h->cap) || dalloc(&h->d_pofs, n_inst + 1) || dalloc(&h->ctl, 4 + n_inst + 1) ||
        dalloc(&h->d_tofs, n_inst + 1) || dalloc(&h->pguess, h->n) || dalloc(&h->ohist, 2 * PLAN_CLASSES))
        return KDT_ERR_CUDA;
    if (cudaMallocHost(&h->hctl, (4 + n_inst + 1) * sizeof(int)) != cudaSuccess) return KDT_ERR_CUDA;
    h->d_moff = h->ctl + 4;
    h->h_moff = h->hctl + 4;
    CK(cudaMemcpy(h->d_pofs, h->pofs.data(), (n_inst + 1) * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_tofs, h->tofs.data(), (n_inst + 1) * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemsetAsync(h->pt_stamp, 0, h->n * sizeof(int), h->stream));
    h->viol_cap = std::max(4096, h->cap);
    if (dalloc(&h->viol, (size_t)h->viol_cap)) return KDT_ERR_CUDA;
    int ppp = h->cfg.points_per_partition > 0 ? h->cfg.points_per_partition : 256;
    h->wpp = h->cfg.warps_per_partition > 0 ? h->cfg.warps_per_partition : 1;
    h->tune_idx = h->cfg.autotune ? 0 : -1;
    h->tune_done = 0;
    h->tune_count = 0;
    for (double &x : h->tune_ms) x = 0.0;
    return set_partitions(h, ppp);
}

void add_counters(kdt *h)
{
    unsigned long long c[C_SLOTS];
    if (cudaMemcpy(c, h->counters, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess) return;
    cudaMemset(h->counters, 0, sizeof c);
    kdt_stats &s = h->stats;
    s.flips += c[C_FLIPS];
    s.retries += c[C_RETRIES];
    s.walk_steps += c[C_WALK_STEPS];
    s.exact_incircle += c[C_EXACT];
    s.sos_ties += c[C_TIES];
    s.deferred += c[C_DEFERRED];
    s.fixup_flips += c[C_FIX_FLIPS];
    s.deleted_degree_sum += c[C_DEG_DEL];
    s.stack_drops += c[C_STACK_DROP];
    s.edge_splits += c[C_SPLIT_EDGE];
    s.ghost_splits += c[C_SPLIT_GHOST];
    s.deletes += c[C_DELETES];
    s.inserts += c[C_INSERTS];
    s.flip_tests += c[C_FLIP_TESTS];
    s.staged_to_global += c[C_MV_GLOBAL];
    s.cycles_move += (int64_t)c[C_CYC_MOVE] << 6;
    if ((int64_t)(c[C_CYC_MAX] << 6) > s.cycles_move_max) s.cycles_move_max = (int64_t)(c[C_CYC_MAX] << 6);
    s.cycles_gather += (int64_t)c[C_CYC_GATHER] << 6;
    s.cycles_claim += (int64_t)c[C_CYC_CLAIM] << 6;
    s.cycles_local += (int64_t)c[C_CYC_LOCAL] << 6;
    s.cycles_writeback += (int64_t)c[C_CYC_WB] << 6;
    s.cycles_ear += (int64_t)c[C_CYC_EAR] << 6;
    s.cycles_lawson += (int64_t)c[C_CYC_LAWSON] << 6;
    s.cycles_certify += (int64_t)c[C_CYC_CERT] << 6;
    s.proposal_moves += c[C_PROP_MOVES];
    s.tensor_timeouts += (int64_t)c[C_TC_FAIL];
    s.proposal_hits += c[C_PROP_HITS];
    s.trace_rows += c[C_TRACE_ROWS];
    s.tail_moves += c[C_TAIL_MOVES];
    s.cycles_tail += (int64_t)c[C_CYC_TAIL];
    s.big_moves += c[C_BIG_MOVES];
    s.cycles_big += (int64_t)c[C_CYC_BIG];
    s.drain_moves += c[C_DRAIN_MOVES];
    s.span_tickets_ns += (int64_t)c[C_SPAN_TICKETS];
    s.span_drain_ns += (int64_t)c[C_SPAN_DRAIN];
    s.span_kernel_ns += (int64_t)c[C_SPAN_ALL];
    s.span_huge_ns += (int64_t)c[C_SPAN_HUGE];
    s.span_drained_ns += (int64_t)c[C_SPAN_DRAINED];
    if ((int64_t)c[C_DRAINED_MAX] > s.cycles_drained_max) s.cycles_drained_max = (int64_t)c[C_DRAINED_MAX];
    s.redeferred += (int64_t)c[C_REDEFER];
    s.big_in_place += (int64_t)c[C_BIG_INPLACE];
    s.cycles_big_in_place += (int64_t)c[C_CYC_BIG_INPLACE];
    s.cycles_big_delete += (int64_t)c[C_CYC_BIG_DELETE];
    s.cycles_big_insert += (int64_t)c[C_CYC_BIG] - (int64_t)c[C_CYC_BIG_INPLACE] - (int64_t)c[C_CYC_BIG_DELETE];
    if ((int64_t)c[C_BIG_MAX] > s.cycles_unyielding_max) s.cycles_unyielding_max = (int64_t)c[C_BIG_MAX];
    s.cycles_global_insert += (int64_t)c[C_CYC_GLOBAL_INS];
    if ((int64_t)c[C_GLOBAL_INS_MAX] > s.cycles_global_insert_max)
        s.cycles_global_insert_max = (int64_t)c[C_GLOBAL_INS_MAX];
}

// Undo a step that failed after it started: restore the old positions and rebuild.
int roll_back(kdt *h, int m)
{
    k_restore_positions<<<(m + 255) / 256, 256, 0, h->stream>>>(h->xy, h->gmoves, h->old_xy, m);
    h->stats.kernel_launches++;
    return rebuild_all(h);
}

int verify_state(kdt *h, int64_t *bad)
{
    Dev d = make_dev(h);
    CK(cudaMemsetAsync(h->scal + S_BAD, 0, 3 * sizeof(int), h->stream));
    k_verify<<<thread_grid(h, std::max<int64_t>(h->cap, h->n), 256), 256, 0, h->stream>>>(
        d, make_inst(h), h->cap, h->scal + S_BAD, h->scal + S_ALIVE, h->scal + S_WRAPS);
    h->stats.kernel_launches++;
    CK(cudaGetLastError());
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    int64_t b = h->hscal[S_BAD];
    if (h->hscal[S_ALIVE] != h->cap) b += 1;
    if (h->hscal[S_WRAPS] != h->ninst) b += 1;  // every hull winds exactly once
    *bad = b;
    return 0;
}

// Issue one step's kernels on `st`: intake + per-partition lists, the kinetic kernel
// (whose last warp inserts deferred points and certifies global-path writes), and the
// copy of the status scalars to the host.  With from_ctl the kernels read m, the
// stamp and the moves' address from h->ctl, so the sequence can be captured once
// into a CUDA graph.
// warps of the kinetic launch
void kinetic_shape(kdt *h, int *blocks, int *threads)
{
    int kblocks = kinetic_blocks(h), kthreads = WPB * 32;
    if (h->cfg.kinetic_warps > 0) {
        kblocks = (h->cfg.kinetic_warps + WPB - 1) / WPB;
        if (h->cfg.kinetic_warps < WPB) kthreads = 32 * h->cfg.kinetic_warps;
    }
    *blocks = kblocks;
    *threads = kthreads;
}

// The global scratch for deletions of degree above KMAX: BIG_INTS ints per warp of the
// kinetic launch, allocated before the first step (outside any graph capture).
int ensure_big(kdt *h)
{
    int kb = 0, kt = 0;
    kinetic_shape(h, &kb, &kt);
    long long warps = (long long)kb * (kt / 32);
    if (warps <= h->big_warps) return 0;
    if (h->big) cudaFree(h->big);
    h->big = nullptr;
    h->big_warps = 0;
    if (cudaMalloc(&h->big, (size_t)warps * BIG_INTS * sizeof(int)) != cudaSuccess) return KDT_ERR_CUDA;
    h->big_warps = warps;
    h->gen++;  // a captured step graph holds the old Dev
    return 0;
}

// kdt_d_values without the argument checks (also run by a step whose displacement rule
// needs d_local)
int d_values_impl(kdt *h, int N, int64_t *dist2, int64_t *cell_min2, kdt_dinfo *info);

// f^2 of the displacement rule, 0 when it is off
double far2(const kdt *h)
{
    const double f = h->cfg.rebuild_displacement;
    return f > 0.0 && !h->qhist ? f * f : 0.0;  // (partitions that change every step keep no d_local)
}

// CTAs of the tensor-core network for `rows` rows: one per 128-row tile, at most three
// per SM (66 KB of shared memory and 128 TMEM columns each)
int tc_grid(const kdt *h, long long rows)
{
    const long long tiles = std::max(1ll, (rows + TC_M - 1) / TC_M);
    return (int)std::min<long long>(tiles, 3ll * sm_count(h->device));
}

int enqueue_step(kdt *h, cudaStream_t st, const Dev &d, const int3 *mp, int mi, bool from_ctl)
{
    int cap = from_ctl ? h->mcap : mi;
    Inst I = make_inst(h);
    // the step's control words and move offsets, from pinned host memory (a captured
    // copy reads them when the graph runs)
    CK(cudaMemcpyAsync(h->ctl, h->hctl, (4 + h->ninst + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    // scalars zero, partition lists empty, deferred entries -1: one kernel
    k_step_clear<<<thread_grid(h, std::max<long long>(h->ncells_cap, 4ll * h->mcap), 256), 256, 0, st>>>(
        h->scal, S_NUM, h->head, h->ncells_cap, h->deferred, h->mcap);
    if (h->qhist) {
        // Fig. 4's Quad-treeDvision at the start of the step, from the points per fine
        // cell the intakes keep current: count pyramid, every fine cell's leaf, leaves
        // numbered depth-first (a scan in Morton order); their number goes to S_NCELLS
        const int D = h->qD, F = 1 << D;
        for (int l = D - 1; l >= 0; --l) {
            const int *src = l == D - 1 ? h->qhist : h->qpyr + ((1 << (2 * (l + 1))) - 1) / 3;
            k_qt_level<<<thread_grid(h, 1ll << (2 * l), 256), 256, 0, st>>>(src, h->qpyr + ((1 << (2 * l)) - 1) / 3,
                                                                         1 << l);
        }
        k_qt_leaf<<<thread_grid(h, (long long)F * F, 256), 256, 0, st>>>(h->qpyr, D, h->ppp, h->qflag, h->qlev);
        if (scan(h, h->qflag, h->qpre, F * F, h->scal + S_NCELLS, st)) return KDT_ERR_CUDA;
        k_qt_map<<<thread_grid(h, (long long)F * F, 256), 256, 0, st>>>(h->qpre, h->qlev, D, h->qmap);
    }
    k_intake_link<<<thread_grid(h, cap, 256), 256, 0, st>>>(d, mp, mi, I, h->cfg.domain_bits, h->head, h->next,
                                                            h->old_xy, h->gmoves, h->dloc2, far2(h));
    const bool net = h->prop_on && (h->cfg.plan & PLAN_NETWORK), ordered = (h->cfg.plan & PLAN_ORDER) != 0;
    const bool tensor = net && (h->cfg.plan & PLAN_TENSOR);
    if (net || ordered) {
        // the planner: estimated work per partition and / or the network's guesses,
        // then (ordered) the partitions in order of decreasing estimate
        if (ordered) {
            CK(cudaMemsetAsync(h->pcost, 0, (size_t)h->ncells_cap * sizeof(float), st));
            CK(cudaMemsetAsync(h->ohist, 0, 2 * PLAN_CLASSES * sizeof(int), st));
        }
        int pblocks = (int)std::min<long long>(((long long)cap + PLAN_THREADS - 1) / PLAN_THREADS,
                                               8ll * sm_count(h->device));
        k_plan<<<std::max(pblocks, 1), PLAN_THREADS, 0, st>>>(d, h->gmoves, h->old_xy, mi, I, h->cfg.domain_bits,
                                                             net && !tensor ? h->mlp_w : nullptr,
                                                             net ? h->pguess : nullptr, ordered ? h->pcost : nullptr,
                                                             tensor ? h->pfeat : nullptr, tensor ? h->ppart : nullptr);
        if (tensor)
            k_mlp_tc<1><<<tc_grid(h, cap), TC_M, TCS_BYTES, st>>>(h->mlp_w, h->pfeat, mi, from_ctl ? h->ctl : nullptr,
                                                                  nullptr, h->ppart, h->gmoves, h->pguess,
                                                                  ordered ? h->pcost : nullptr,
                                                                  h->counters + C_TC_FAIL);
    }
    if (ordered) {
        const int ostride = h->qhist || h->cfg.partition_order ? 1 : h->stride;
        k_order<<<thread_grid(h, h->ncells_cap, 256), 256, 0, st>>>(h->pcost, h->ncells_cap, h->ohist, h->order, 0,
                                                                    ostride);
        k_order<<<thread_grid(h, h->ncells_cap, 256), 256, 0, st>>>(h->pcost, h->ncells_cap, h->ohist, h->order, 1,
                                                                    ostride);
    }
    // inside a capture an event record must be an external node to keep its timestamp
    unsigned evflags = from_ctl ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (h->cfg.timing) CK(cudaEventRecordWithFlags(h->ev0, st, evflags));
    int kblocks = 0, kthreads = 0;
    kinetic_shape(h, &kblocks, &kthreads);
    Dev dk = d;
    dk.big = h->big;
    auto kin = h->cfg.kinetic_blocks_per_sm == 7 ? k_kinetic<7> : k_kinetic<6>;
    kin<<<kblocks, kthreads, 0, st>>>(dk, h->gmoves, h->head, h->next, I, h->ncells, h->wpp, h->deferred,
                                            h->scal + S_DEFER, h->mcap, h->viol, h->viol_cap);
    if (h->cfg.timing) CK(cudaEventRecordWithFlags(h->ev1, st, evflags));
    k_certify_step<<<thread_grid(h, 4096, 256), 256, 0, st>>>(d, h->viol, h->scal + S_VIOL, h->viol_cap);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->hscal, h->scal, S_NUM * sizeof(int), cudaMemcpyDeviceToHost, st));
    return 0;
}

// After the step kernels: repair the violations they recorded (general Lawson) and
// certify what the repair wrote, until nothing is left.  Returns a CUDA/ABI error;
// the device status goes to *ds.
int repair_step(kdt *h, int *ds)
{
    cudaStream_t st = h->stream;
    *ds = 0;
    int nv = h->hscal[S_VIOL];
    if (h->hscal[S_DIRTY] > h->dirty_cap) return certify_and_repair(h, true, 0, h->cap, h->ninst, ds);
    if (nv == 0) return 0;
    Dev d = make_dev(h);
    h->stats.violations += nv;
    for (int round = 0; round < 64; ++round) {
        if (nv > h->viol_cap) nv = h->viol_cap;
        int dirty_before = h->hscal[S_DIRTY];
        k_fixup<<<warp_grid(h, nv, 16), WPB * 32, 0, st>>>(d, h->viol, nv);
        h->stats.kernel_launches++;
        CK(cudaGetLastError());
        if (sync_scalars(h)) return KDT_ERR_CUDA;
        *ds = h->hscal[S_STATUS];
        if (*ds) return 0;
        if (h->hscal[S_DIRTY] > h->dirty_cap) return certify_and_repair(h, true, 0, h->cap, h->ninst, ds);
        CK(cudaMemsetAsync(h->scal + S_VIOL, 0, sizeof(int), st));
        k_certify<<<thread_grid(h, 65536, 256), 256, 0, st>>>(d, dirty_before, h->viol, h->scal + S_VIOL,
                                                             h->viol_cap);
        h->stats.kernel_launches++;
        if (sync_scalars(h)) return KDT_ERR_CUDA;
        *ds = h->hscal[S_STATUS];
        nv = h->hscal[S_VIOL];
        if (*ds || nv == 0) return 0;
        h->stats.violations += nv;
    }
    *ds = DEV_INTERNAL;
    return 0;
}

// Autotuner: the first TUNE_STEPS steps of every (points per partition, warps per
// partition) pair are timed with events around the step; then the pair with the
// least time per move is kept.  Results do not depend on the pair.  A single instance with a configured
// grid tunes the warps per partition only.
bool tune_fixed_grid(const kdt *h) { return h->ninst == 1 && (h->cfg.grid > 0 || h->qmap); }

int autotune_before(kdt *h)
{
    if (h->tune_idx < 0 || h->tune_done) return 0;
    int ppp = tune_fixed_grid(h) ? h->ppp : TUNE_PPP[h->tune_idx / 3];
    if (ppp != h->ppp) {
        int rc = set_partitions(h, ppp);
        if (rc) return rc;
    }
    h->wpp = TUNE_WPP[h->tune_idx % 3];
    return 0;
}

int autotune_after(kdt *h, float ms, int64_t m)
{
    if (h->tune_idx < 0 || h->tune_done) return 0;
    h->tune_ms[h->tune_idx] += (double)ms / (double)(m > 0 ? m : 1);
    if (++h->tune_count < TUNE_STEPS) return 0;
    h->tune_count = 0;
    ++h->tune_idx;
    int last = tune_fixed_grid(h) ? 3 : 9;
    if (h->tune_idx < last) return 0;
    int best = 0;
    for (int k = 1; k < last; ++k)
        if (h->tune_ms[k] < h->tune_ms[best]) best = k;
    h->tune_done = 1;
    int ppp = tune_fixed_grid(h) ? h->ppp : TUNE_PPP[best / 3];
    if (ppp != h->ppp) {
        int rc = set_partitions(h, ppp);
        if (rc) return rc;
    }
    h->wpp = TUNE_WPP[best % 3];
    h->stats.tuned_points_per_partition = h->ppp;
    h->stats.tuned_warps_per_partition = h->wpp;
    return 0;
}

// One step of every instance: moves (instance-local ids, host or device) with CSR
// offsets moff (host, ninst + 1 entries).
int step_core(kdt *h, const kdt_move *moves, const int64_t *moff, int64_t m);
int qt_recount(kdt *h);

// One step; with the quad-tree re-divided at every step, a step that did not finish on the
// kinetic path (an error, a rebuild) has the points per fine cell counted again.
int step_impl(kdt *h, const kdt_move *moves, const int64_t *moff, int64_t m)
{
    const int64_t rebuilds = h->stats.rebuilds;
    const int rc = step_core(h, moves, moff, m);
    if (h->qhist && (rc != KDT_OK || h->stats.rebuilds != rebuilds)) {
        const int rr = qt_recount(h);
        if (rr) return rr;
    }
    return rc;
}

int step_core(kdt *h, const kdt_move *moves, const int64_t *moff, int64_t m)
{
    if (m == 0) return KDT_OK;
    if (m > h->n) return KDT_ERR_DUPLICATE;  // some id must repeat (or be out of range)
    CK(cudaSetDevice(h->device));
    const PtrKind mk = ptr_kind(moves, h->device);
    if (mk == PTR_FOREIGN) return KDT_ERR_ARG;
    int rc = ensure_moves(h, m);
    if (rc) return rc;
    cudaStream_t st = h->stream;
    const int mi = (int)m;
    const int3 *mp = (const int3 *)moves;
    if (mk != PTR_DEV) {
        CK(cudaMemcpyAsync(h->moves, moves, (size_t)m * sizeof(int3), cudaMemcpyHostToDevice, st));
        mp = h->moves;
    }
    for (int i = 0; i <= h->ninst; ++i) h->h_moff[i] = (int)moff[i];
    h->stamp++;
    Dev d = make_dev(h);
    bool large = h->cfg.fallback && (double)m > (double)h->cfg.rebuild_ratio * (double)h->n;
    if (large) {
        // a step this large is cheaper as a rebuild (Abstract: "if the points move so
        // far, it's better to rebuild the triangulation")
        CK(cudaMemcpyAsync(h->ctl, h->hctl, (4 + h->ninst + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(h->scal, 0, S_NUM * sizeof(int), st));
        CK(cudaMemsetAsync(h->head, 0xff, (size_t)h->ncells_cap * sizeof(int), st));
        k_intake_link<<<thread_grid(h, mi, 256), 256, 0, st>>>(d, mp, mi, make_inst(h), h->cfg.domain_bits, h->head,
                                                               h->next, h->old_xy, h->gmoves, nullptr, 0.0);
        h->stats.kernel_launches++;
        if (sync_scalars(h)) return KDT_ERR_CUDA;
        if (h->hscal[S_STATUS]) return dev_to_abi(h->hscal[S_STATUS]);
        k_set_positions<<<(mi + 255) / 256, 256, 0, st>>>(h->xy, h->gmoves, mi);
        h->stats.kernel_launches++;
        rc = rebuild_all(h);
        if (rc) {
            int rr = roll_back(h, mi);
            return rr ? rr : rc;
        }
        h->stats.steps++;
        h->stats.moves += m;
        return KDT_OK;
    }
    rc = autotune_before(h);
    if (rc) return rc;
    rc = ensure_big(h);
    if (rc) return rc;
    if (h->qhist && h->scan_tmp_cap < (h->qF * h->qF + SCAN_TILE - 1) / SCAN_TILE + 1) {
        // the step graph scans every fine cell: its scan scratch must exist before capture
        const int c = (h->qF * h->qF + SCAN_TILE - 1) / SCAN_TILE + 1024;
        if (dalloc(&h->scan_tmp, (size_t)c)) return KDT_ERR_CUDA;
        h->scan_tmp_cap = c;
        h->gen++;
    }
    if (far2(h) > 0.0 && !h->dloc_valid) {
        // the displacement rule needs d_local: compute it (a failure, e.g. an instance
        // with too few points, leaves the rule inactive for this step)
        kdt_dinfo info;
        if (d_values_impl(h, h->d_n > 0 ? h->d_n : 1, nullptr, nullptr, &info) == KDT_ERR_CUDA) return KDT_ERR_CUDA;
    }
    d = make_dev(h);
    bool timed = h->cfg.timing || (h->tune_idx >= 0 && !h->tune_done);
    if (h->cfg.use_graph) {
        // one graph launch per step
        if (h->graph_gen != h->gen) {
            drop_graph(h);
            Dev dg = d;
            dg.ctl = h->ctl;
            CK(cudaStreamBeginCapture(h->cstream, cudaStreamCaptureModeThreadLocal));
            int er = enqueue_step(h, h->cstream, dg, nullptr, 0, true);
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamEndCapture(h->cstream, &g);
            if (er || ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return KDT_ERR_CUDA;
            }
            h->graph = g;
            CK(cudaGraphInstantiate(&h->gexec, h->graph, 0));
            h->graph_gen = h->gen;
        }
        h->hctl[0] = mi;
        h->hctl[1] = h->stamp;
        unsigned long long pa = (unsigned long long)(uintptr_t)mp;
        h->hctl[2] = (int)(unsigned)(pa & 0xffffffffu);
        h->hctl[3] = (int)(unsigned)(pa >> 32);
        if (timed) CK(cudaEventRecord(h->ev2, st));
        CK(cudaGraphLaunch(h->gexec, st));
        if (timed) CK(cudaEventRecord(h->ev3, st));
    } else {
        if (timed) CK(cudaEventRecord(h->ev2, st));
        if (enqueue_step(h, st, d, mp, mi, false)) return KDT_ERR_CUDA;
        if (timed) CK(cudaEventRecord(h->ev3, st));
    }
    h->stats.kernel_launches += 4 + ((h->cfg.plan & PLAN_ORDER) ? 2 : 0) +
                                ((h->cfg.plan & PLAN_ORDER) || (h->prop_on && (h->cfg.plan & PLAN_NETWORK)) ? 1 : 0) +
                                (h->prop_on && (h->cfg.plan & PLAN_NETWORK) && (h->cfg.plan & PLAN_TENSOR) ? 1 : 0) +
                                (h->qhist ? h->qD + 5 : 0);
    CK(cudaStreamSynchronize(st));
    if (h->qhist) h->ncells = h->qleaves = h->hscal[S_NCELLS];
    if (timed) {
        float ms = 0.f;
        if (h->cfg.timing && cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) {
            h->stats.kinetic_kernel_ms += ms;
            h->stats.kinetic_kernel_timed++;
        }
        if (cudaEventElapsedTime(&ms, h->ev2, h->ev3) == cudaSuccess) {
            if (h->cfg.timing) h->stats.step_graph_ms += ms;
            rc = autotune_after(h, ms, m);
            if (rc) return rc;
        }
    }
    int s = h->hscal[S_STATUS];
    if (s == DEV_ARG || s == DEV_RANGE || s == DEV_DUP_ID) return dev_to_abi(s);  // intake: nothing modified
    if (s == DEV_FAR) {
        // a move went farther than the displacement rule allows: the kinetic kernel
        // stopped before changing anything; triangulate the final positions again
        h->stats.far_rebuilds++;
        k_set_positions<<<(mi + 255) / 256, 256, 0, st>>>(h->xy, h->gmoves, mi);
        h->stats.kernel_launches++;
        rc = rebuild_all(h);
        if (rc) {
            int rr = roll_back(h, mi);
            return rr ? rr : rc;
        }
        h->stats.steps++;
        h->stats.moves += m;
        return KDT_OK;
    }
    if (s == 0) {
        int ds = 0;
        if (repair_step(h, &ds)) return KDT_ERR_CUDA;
        s = ds;
    }
    if (s) {
        // the step failed while running: finish it by a full rebuild of the final
        // positions (the certified fallback); if those are invalid, roll back
        h->stats.fallbacks++;
        h->stats.last_fallback_reason = s;
        h->stats.last_fallback_point = h->hscal[S_FAILPT];
        if (h->cfg.debug & 1) {
            h->built = true;  // keep the failed state for kdt_export_store
            return dev_to_abi(s);
        }
        bool allow = h->cfg.fallback || s == DEV_DUPLICATE || s == DEV_DEGENERATE;
        int rc2 = KDT_ERR_RETRY_EXHAUSTED;
        if (allow) {
            k_set_positions<<<(mi + 255) / 256, 256, 0, st>>>(h->xy, h->gmoves, mi);
            h->stats.kernel_launches++;
            rc2 = rebuild_all(h);
        }
        if (rc2) {
            int rr = roll_back(h, mi);
            if (rr) return rr;
            return allow ? rc2 : dev_to_abi(s);
        }
    }
    h->stats.steps++;
    h->stats.moves += m;
    if (h->cfg.verify) {
        int64_t bad = 0;
        int vr = verify_state(h, &bad);
        if (vr) return vr;
        if (bad) return KDT_ERR_INTERNAL;
    }
    return KDT_OK;
}

// canonical export of slots [s0, s0 + nslots) whose point ids are idbase .. idbase + np - 1
int export_range(kdt *h, int s0, int nslots, int idbase, int np, int32_t *out, int64_t cap, int64_t *n_tri)
{
    cudaStream_t st = h->stream;
    if (grow(h->exp_cnt, (size_t)np * 4) || grow(h->exp_off, (size_t)np * 4) || grow(h->exp_fill, (size_t)np * 4))
        return KDT_ERR_CUDA;
    int *cnt = (int *)h->exp_cnt.p, *off = (int *)h->exp_off.p, *fill = (int *)h->exp_fill.p;
    CK(cudaMemsetAsync(cnt, 0, (size_t)np * 4, st));
    k_exp_count<<<thread_grid(h, nslots, 256), 256, 0, st>>>(TriHalf{h->tri + 2 * (size_t)s0}, nslots, cnt, idbase);
    h->stats.kernel_launches++;
    if (scan(h, cnt, off, np, h->scal + S_TOTAL, st)) return KDT_ERR_CUDA;
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    int64_t total = h->hscal[S_TOTAL];
    *n_tri = total;
    if (total > cap) return KDT_ERR_CAPACITY;
    bool dev_out = total > 0 && on_device(h, out);
    int3 *dst;
    if (dev_out) {
        dst = (int3 *)out;
    } else {
        if (grow(h->exp_out, (size_t)std::max<int64_t>(total, 1) * sizeof(int3))) return KDT_ERR_CUDA;
        dst = (int3 *)h->exp_out.p;
    }
    CK(cudaMemsetAsync(fill, 0, (size_t)np * 4, st));
    k_exp_place<<<thread_grid(h, nslots, 256), 256, 0, st>>>(TriHalf{h->tri + 2 * (size_t)s0}, nslots, off, fill, dst, idbase);
    k_exp_sortseg<<<thread_grid(h, np, 256), 256, 0, st>>>(np, off, cnt, dst);
    h->stats.kernel_launches += 2;
    CK(cudaGetLastError());
    if (!dev_out && total > 0)
        CK(cudaMemcpyAsync(out, dst, (size_t)total * sizeof(int3), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return KDT_OK;
}

// The quad-tree of Section III (Data structure) over the current positions of the
// single instance: the square of side 2^lg (the smallest power of two >= the larger
// extent) at the points' minimum corner, divided into four recursively until a square
// holds at most ppp points or has the side of a fine cell (2^lg / 2^D, D = min(11,
// lg)).  The points per fine cell are counted on the GPU; the division runs on the
// host over the count pyramid; every fine cell gets its leaf's number (depth-first,
// children low-x low-y, high-x low-y, low-x high-y, high-x high-y).
int build_quadtree(kdt *h)
{
    cudaStream_t st = h->stream;
    const int n = (int)h->n;
    int init_bbox[4] = {INT_MAX, INT_MAX, INT_MIN, INT_MIN};
    CK(cudaMemsetAsync(h->scal, 0, S_NUM * sizeof(int), st));
    CK(cudaMemcpyAsync(h->scal + S_MINX, init_bbox, sizeof init_bbox, cudaMemcpyHostToDevice, st));
    k_range<<<thread_grid(h, n, 256), 256, 0, st>>>(h->xy, n, h->cfg.domain_bits, h->scal + S_STATUS,
                                                    h->scal + S_MINX);
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    const int x0 = h->hscal[S_MINX], y0 = h->hscal[S_MINY];
    const long long ext = std::max((long long)h->hscal[S_MAXX] - x0, (long long)h->hscal[S_MAXY] - y0) + 1;
    int lg = 0;
    while ((1ll << lg) < ext) ++lg;
    const int D = std::min(11, lg), F = 1 << D;
    if (grow(h->hist, (size_t)F * F * sizeof(int))) return KDT_ERR_CUDA;
    CK(cudaMemsetAsync(h->hist.p, 0, (size_t)F * F * sizeof(int), st));
    k_qt_hist<<<thread_grid(h, n, 256), 256, 0, st>>>(h->xy, n, x0, y0, lg - D, F, (int *)h->hist.p);
    h->stats.kernel_launches += 2;
    std::vector<std::vector<long long>> lev(D + 1);
    {
        std::vector<int> fine((size_t)F * F);
        CK(cudaMemcpyAsync(fine.data(), h->hist.p, fine.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        lev[D].assign(fine.begin(), fine.end());
    }
    for (int l = D - 1; l >= 0; --l) {
        const int w = 1 << l, wc = 2 << l;
        lev[l].assign((size_t)w * w, 0);
        for (int y = 0; y < w; ++y)
            for (int x = 0; x < w; ++x)
                lev[l][(size_t)y * w + x] = lev[l + 1][(size_t)(2 * y) * wc + 2 * x] +
                                            lev[l + 1][(size_t)(2 * y) * wc + 2 * x + 1] +
                                            lev[l + 1][(size_t)(2 * y + 1) * wc + 2 * x] +
                                            lev[l + 1][(size_t)(2 * y + 1) * wc + 2 * x + 1];
    }
    std::vector<int> qmap((size_t)F * F, -1);
    int leaves = 0, largest = D;
    const long long T = h->ppp;
    auto divide = [&](auto &&self, int l, int x, int y) -> void {
        if (lev[l][(size_t)y * (1 << l) + x] <= T || l == D) {
            const int id = leaves++, span = 1 << (D - l);
            largest = std::min(largest, l);
            for (int fy = y * span; fy < (y + 1) * span; ++fy)
                for (int fx = x * span; fx < (x + 1) * span; ++fx) qmap[(size_t)fy * F + fx] = id;
            return;
        }
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) self(self, l + 1, 2 * x + cx, 2 * y + cy);
    };
    divide(divide, 0, 0, 0);
    if (dalloc(&h->qmap, qmap.size())) return KDT_ERR_CUDA;
    CK(cudaMemcpy(h->qmap, qmap.data(), qmap.size() * sizeof(int), cudaMemcpyHostToDevice));
    h->qx0 = x0;
    h->qy0 = y0;
    h->qshift = lg - D;
    h->qF = F;
    h->qleaves = leaves;
    h->qleaf_side_lg = lg - largest;  // log2 of the side of the largest leaf
    h->qD = D;
    if (h->cfg.quadtree == 2) {
        // re-divided at every step: keep the points per fine cell, and the scratch of the
        // division on the GPU
        const size_t f2 = (size_t)F * F;
        if (dalloc(&h->qhist, f2) || dalloc(&h->qpyr, std::max<size_t>(1, (f2 - 1) / 3)) ||
            dalloc(&h->qflag, f2) || dalloc(&h->qpre, f2) || dalloc(&h->qlev, f2))
            return KDT_ERR_CUDA;
        CK(cudaMemcpyAsync(h->qhist, h->hist.p, f2 * sizeof(int), cudaMemcpyDeviceToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    return set_partitions(h, h->ppp);
}

// Points per fine cell of the re-divided quad-tree counted again from the positions
// (after a step that did not finish on the kinetic path).
int qt_recount(kdt *h)
{
    const size_t f2 = (size_t)h->qF * h->qF;
    CK(cudaMemsetAsync(h->qhist, 0, f2 * sizeof(int), h->stream));
    k_qt_hist<<<thread_grid(h, h->n, 256), 256, 0, h->stream>>>(h->xy, (int)h->n, h->qx0, h->qy0, h->qshift, h->qF,
                                                               h->qhist);
    h->stats.kernel_launches++;
    CK(cudaStreamSynchronize(h->stream));
    return 0;
}

int build_impl(kdt *h, const int32_t *xy, const int64_t *offs, int n_inst)
{
    CK(cudaSetDevice(h->device));
    if (foreign(h, xy)) return KDT_ERR_ARG;
    free_state(h);
    int rc = alloc_state(h, offs, n_inst);
    if (rc) {
        free_state(h);
        return rc;
    }
    CK(cudaMemcpyAsync(h->xy, xy, (size_t)h->n * sizeof(int2),
                       on_device(h, xy) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    rc = rebuild_all(h);
    if (rc == 0 && h->cfg.quadtree && h->ninst == 1) rc = build_quadtree(h);
    return rc;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

int kdt_version(void) { return ABI_VERSION; }

int64_t kdt_stats_size(void) { return (int64_t)sizeof(kdt_stats); }

int64_t kdt_config_size(void) { return (int64_t)sizeof(kdt_config); }

const char *kdt_error_string(int code)
{
    switch (code) {
    case KDT_OK: return "ok";
    case KDT_ERR_ARG: return "bad argument";
    case KDT_ERR_RANGE: return "coordinate out of range";
    case KDT_ERR_DUPLICATE: return "duplicate point or repeated move id";
    case KDT_ERR_DEGENERATE: return "degenerate input (n < 3 or all points collinear)";
    case KDT_ERR_CAPACITY: return "output buffer too small";
    case KDT_ERR_RETRY_EXHAUSTED: return "conflict retries exhausted";
    case KDT_ERR_CUDA: return "CUDA runtime error";
    case KDT_ERR_INTERNAL: return "internal consistency check failed";
    case KDT_ERR_STATE: return "call out of order";
    case KDT_ERR_TOO_LARGE: return "more points than the allocation-free export serves";
    default: return "unknown error";
    }
}

int kdt_default_config(kdt_config *cfg)
{
    if (!cfg) return KDT_ERR_ARG;
    memset(cfg, 0, sizeof *cfg);
    cfg->grid = 0;
    cfg->domain_bits = 28;
    cfg->retry_cap = 4096;
    cfg->fallback = 1;
    cfg->rebuild_ratio = 0.25f;
    cfg->filter = 1;
    cfg->verify = 0;
    cfg->timing = 0;
    cfg->warps_per_block = WPB;
    cfg->use_graph = 1;
    cfg->points_per_partition = 0;
    cfg->warps_per_partition = 0;
    cfg->autotune = 0;
    cfg->variant = 0;
    cfg->batch_build = 1;
    return KDT_OK;
}

int kdt_create(kdt **out, const kdt_config *cfg, int device, void *cuda_stream)
{
    if (!out) return KDT_ERR_ARG;
    *out = nullptr;
    kdt_config c;
    if (cfg) c = *cfg;
    else kdt_default_config(&c);
    if (c.domain_bits <= 0 || c.domain_bits > 28 || c.grid < 0 || c.grid > 4096 || c.retry_cap < 0 ||
        c.points_per_partition < 0 || c.warps_per_partition < 0 || c.warps_per_partition > 32 ||
        c.variant < 0 || c.variant > 2 || c.quadtree < 0 || c.quadtree > 2 ||
        !(c.rebuild_displacement >= 0.0f) || c.rebuild_displacement > 1e9f || c.plan < 0 || c.plan > 7 ||
        c.batch_build < 0 || c.batch_build > 1 ||
        (c.kinetic_blocks_per_sm != 0 && c.kinetic_blocks_per_sm != 6 && c.kinetic_blocks_per_sm != 7) ||
        c.partition_order < 0 || c.partition_order > 1)
        return KDT_ERR_ARG;
    if (c.retry_cap == 0) c.retry_cap = 4096;
    if (cudaSetDevice(device) != cudaSuccess) return KDT_ERR_CUDA;
    kdt *h = new (std::nothrow) kdt();
    if (!h) return KDT_ERR_ARG;
    h->device = device;
    h->stream = (cudaStream_t)cuda_stream;
    h->cfg = c;
    if (cudaMalloc(&h->scal, S_NUM * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->counters, C_SLOTS * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&h->hscal, S_NUM * sizeof(int)) != cudaSuccess ||

        cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
        cudaEventCreate(&h->ev2) != cudaSuccess || cudaEventCreate(&h->ev3) != cudaSuccess) {
        kdt_destroy(h);
        return KDT_ERR_CUDA;
    }
    cudaMemset(h->scal, 0, S_NUM * sizeof(int));
    cudaMemset(h->counters, 0, C_SLOTS * sizeof(unsigned long long));
    if (cudaFuncSetAttribute(k_mlp_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_BYTES) != cudaSuccess) {
        kdt_destroy(h);
        return KDT_ERR_CUDA;
    }
    *out = h;
    return KDT_OK;
}

int kdt_destroy(kdt *h)
{
    if (!h) return KDT_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    free_state(h);
    if (h->scal) cudaFree(h->scal);
    if (h->counters) cudaFree(h->counters);
    if (h->mlp_w) cudaFree(h->mlp_w);
    if (h->trace_count) cudaFree(h->trace_count);
    if (h->mlp_part) cudaFree(h->mlp_part);
    if (h->big) cudaFree(h->big);
    if (h->hscal) cudaFreeHost(h->hscal);
    if (h->cstream) cudaStreamDestroy(h->cstream);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev2) cudaEventDestroy(h->ev2);
    if (h->ev3) cudaEventDestroy(h->ev3);
    delete h;
    return KDT_OK;
}

int64_t kdt_num_points(const kdt *h) { return h && h->built ? h->n : 0; }

int32_t kdt_num_instances(const kdt *h) { return h && h->built ? h->ninst : 0; }

int64_t kdt_num_cells(const kdt *h) { return h && h->built ? h->ncells : 0; }

int kdt_build(kdt *h, const int32_t *xy, int64_t n)
{
    if (!h || !xy || n < 0 || n > (1ll << 28)) return KDT_ERR_ARG;
    if (n < 3) return KDT_ERR_DEGENERATE;
    h->d2_run = INT64_MAX;
    int64_t offs[2] = {0, n};
    return build_impl(h, xy, offs, 1);
}

int kdt_build_batch(kdt *h, const int32_t *xy, const int64_t *offsets, int32_t n_inst)
{
    if (!h || !xy || !offsets || n_inst < 1 || n_inst > (1 << 20)) return KDT_ERR_ARG;
    if (offsets[0] != 0) return KDT_ERR_ARG;
    for (int i = 0; i < n_inst; ++i) {
        if (offsets[i + 1] < offsets[i]) return KDT_ERR_ARG;
        if (offsets[i + 1] - offsets[i] < 3) return KDT_ERR_DEGENERATE;
    }
    if (offsets[n_inst] > (1ll << 28)) return KDT_ERR_ARG;
    if (h->cfg.quadtree) return KDT_ERR_ARG;  // quad-tree partitions: one instance
    h->d2_run = INT64_MAX;
    return build_impl(h, xy, offsets, n_inst);
}

int kdt_rebuild(kdt *h)
{
    if (!h) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    CK(cudaSetDevice(h->device));
    return rebuild_all(h);
}

int kdt_step(kdt *h, const kdt_move *moves, int64_t m)
{
    if (!h || m < 0 || (m > 0 && !moves)) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    if (h->ninst != 1) return KDT_ERR_STATE;  // batched handles step with kdt_step_batch
    int64_t moff[2] = {0, m};
    return step_impl(h, moves, moff, m);
}

int kdt_step_batch(kdt *h, const kdt_move *moves, const int64_t *move_offsets, int32_t n_inst)
{
    if (!h || !move_offsets || n_inst < 0) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    if (n_inst != h->ninst) return KDT_ERR_ARG;
    if (move_offsets[0] != 0) return KDT_ERR_ARG;
    for (int i = 0; i < n_inst; ++i)
        if (move_offsets[i + 1] < move_offsets[i]) return KDT_ERR_ARG;
    int64_t m = move_offsets[n_inst];
    if (m > 0 && !moves) return KDT_ERR_ARG;
    return step_impl(h, moves, move_offsets, m);
}

int kdt_export_triangles(kdt *h, int32_t *out, int64_t cap, int64_t *n_tri)
{
    if (!h || !n_tri || cap < 0 || (cap > 0 && !out)) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    CK(cudaSetDevice(h->device));
    return export_range(h, 0, h->cap, 0, (int)h->n, out, cap, n_tri);
}

int kdt_export_triangles_inst(kdt *h, int32_t inst, int32_t *out, int64_t cap, int64_t *n_tri)
{
    if (!h || !n_tri || cap < 0 || (cap > 0 && !out)) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    if (inst < 0 || inst >= h->ninst) return KDT_ERR_ARG;
    CK(cudaSetDevice(h->device));
    int s0 = h->tofs[inst], p0 = h->pofs[inst];
    return export_range(h, s0, h->tofs[inst + 1] - s0, p0, h->pofs[inst + 1] - p0, out, cap, n_tri);
}

int kdt_export_points(kdt *h, int32_t *xy, int64_t cap_points)
{
    if (!h || !xy || cap_points < 0) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    if (cap_points < h->n) return KDT_ERR_CAPACITY;
    CK(cudaSetDevice(h->device));
    if (foreign(h, xy)) return KDT_ERR_ARG;
    CK(cudaMemcpyAsync(xy, h->xy, (size_t)h->n * sizeof(int2),
                       on_device(h, xy) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return KDT_OK;
}

int kdt_d_values(kdt *h, int32_t N, int64_t *dist2, int64_t *cell_min2, kdt_dinfo *info)
{
    if (!h || !info || N < 1 || N > DC_MAX_N) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    CK(cudaSetDevice(h->device));
    if (foreign(h, dist2) || foreign(h, cell_min2)) return KDT_ERR_ARG;
    return d_values_impl(h, N, dist2, cell_min2, info);
}

}  // extern "C"

namespace {

int d_values_impl(kdt *h, int N, int64_t *dist2, int64_t *cell_min2, kdt_dinfo *info)
{
    for (int i = 0; i < h->ninst; ++i)
        if (h->pofs[i + 1] - h->pofs[i] <= N) return KDT_ERR_ARG;
    cudaStream_t st = h->stream;
    const int n = (int)h->n;
    // neighbour lists (CSR) from the live triangles
    if (grow(h->nb_deg, (size_t)n * sizeof(int)) || grow(h->nb_off, (size_t)(n + 1) * sizeof(int)) ||
        grow(h->dc_scal, 4 * sizeof(unsigned long long)))
        return KDT_ERR_CUDA;
    int *deg = (int *)h->nb_deg.p, *off = (int *)h->nb_off.p;
    CK(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(int), st));
    k_nbr_count<<<thread_grid(h, h->cap, 256), 256, 0, st>>>(TriHalf{h->tri}, h->cap, deg);
    if (scan(h, deg, off, n, off + n, st)) return KDT_ERR_CUDA;
    int total = 0;
    CK(cudaMemcpyAsync(&total, off + n, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (grow(h->nb_list, (size_t)std::max(total, 1) * sizeof(int))) return KDT_ERR_CUDA;
    CK(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(int), st));  // now the fill positions
    k_nbr_fill<<<thread_grid(h, h->cap, 256), 256, 0, st>>>(TriHalf{h->tri}, h->cap, off, deg, (int *)h->nb_list.p);
    // the N-th nearest neighbours and their minima
    const bool dist_dev = dist2 && on_device(h, dist2);
    const bool cmin_dev = cell_min2 && on_device(h, cell_min2);
    long long *dd = nullptr;
    unsigned long long *cm = nullptr;
    if (dist2) {
        if (dist_dev) {
            dd = (long long *)dist2;
        } else {
            if (grow(h->dc_dist, (size_t)n * sizeof(long long))) return KDT_ERR_CUDA;
            dd = (long long *)h->dc_dist.p;
        }
    }
    // per-partition minima: into the caller's device buffer, else the handle's (they
    // also feed the displacement rule's running d_local^2)
    if (cmin_dev) {
        cm = (unsigned long long *)cell_min2;
    } else {
        if (grow(h->dc_cmin, (size_t)std::max(h->ncells, 1) * sizeof(long long))) return KDT_ERR_CUDA;
        cm = (unsigned long long *)h->dc_cmin.p;
    }
    k_fill_u64<<<thread_grid(h, h->ncells, 256), 256, 0, st>>>(cm, h->ncells, (unsigned long long)INT64_MAX);
    unsigned long long *sc = (unsigned long long *)h->dc_scal.p;  // [0] minimum, [1] largest degree
    unsigned long long init[2] = {(unsigned long long)INT64_MAX, 0ull};
    CK(cudaMemcpyAsync(sc, init, sizeof init, cudaMemcpyHostToDevice, st));
    k_nth_nn<<<thread_grid(h, n, 128), 128, 0, st>>>(h->xy, off, (const int *)h->nb_list.p, n, N, make_inst(h),
                                                    h->cfg.domain_bits, dd, cm, sc, (int *)(sc + 1));
    const int restart = !h->dloc_valid || h->d_n != N;
    k_merge_min_u64<<<thread_grid(h, h->ncells, 256), 256, 0, st>>>(h->dloc2, cm, h->ncells, restart);
    h->dloc_valid = true;
    h->stats.kernel_launches += 8;
    CK(cudaGetLastError());
    if (dist2 && !dist_dev)
        CK(cudaMemcpyAsync(dist2, dd, (size_t)n * sizeof(long long), cudaMemcpyDeviceToHost, st));
    if (cell_min2 && !cmin_dev)
        CK(cudaMemcpyAsync(cell_min2, cm, (size_t)h->ncells * sizeof(long long), cudaMemcpyDeviceToHost, st));
    unsigned long long res[2];
    CK(cudaMemcpyAsync(res, sc, sizeof res, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h->d_n != N) {
        h->d_n = N;
        h->d2_run = INT64_MAX;
    }
    info->min2 = (int64_t)res[0];
    if (info->min2 < h->d2_run) h->d2_run = info->min2;
    info->d2 = h->d2_run;
    info->max_degree = (int64_t)(int)(unsigned)res[1];
    info->cells = h->ncells;
    info->spread = 0.0;
    if (h->ninst == 1 && h->d2_run > 0) {
        const double side = h->qmap ? (double)(1ll << h->qleaf_side_lg)
                                    : (double)(1ll << h->cfg.domain_bits) / (double)h->igrid[0];
        info->spread = side * std::sqrt(2.0) / std::sqrt((double)h->d2_run);
    }
    return KDT_OK;
}

}  // namespace

extern "C" {

int kdt_verify(kdt *h, int64_t *bad)
{
    if (!h || !bad) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    CK(cudaSetDevice(h->device));
    return verify_state(h, bad);
}

int kdt_get_stats(const kdt *h, kdt_stats *out)
{
    if (!h || !out) return KDT_ERR_ARG;
    kdt *hm = const_cast<kdt *>(h);  // the device counters are merged in lazily
    cudaSetDevice(hm->device);
    cudaStreamSynchronize(hm->stream);
    add_counters(hm);
    *out = h->stats;
    return KDT_OK;
}

int kdt_reset_stats(kdt *h)
{
    if (!h) return KDT_ERR_ARG;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    add_counters(h);
    int64_t tp = h->stats.tuned_points_per_partition, tw = h->stats.tuned_warps_per_partition;
    memset(&h->stats, 0, sizeof h->stats);
    h->stats.tuned_points_per_partition = tp;
    h->stats.tuned_warps_per_partition = tw;
    return KDT_OK;
}

int kdt_export_store(kdt *h, int32_t *tv, int32_t *tn, int32_t *pt_tri, int64_t cap_slots)
{
    if (!h || cap_slots < 0) return KDT_ERR_ARG;
    if (h->n == 0) return KDT_ERR_STATE;
    if (cap_slots < h->cap) return KDT_ERR_CAPACITY;
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    // the two halves of the 32-byte records, each as a dense cap x 4 array
    if (tv) CK(cudaMemcpy2D(tv, sizeof(int4), h->tri, 2 * sizeof(int4), sizeof(int4), (size_t)h->cap,
                            cudaMemcpyDeviceToHost));
    if (tn) CK(cudaMemcpy2D(tn, sizeof(int4), h->tri + 1, 2 * sizeof(int4), sizeof(int4), (size_t)h->cap,
                            cudaMemcpyDeviceToHost));
    if (pt_tri) CK(cudaMemcpy(pt_tri, h->pt_tri, (size_t)h->n * sizeof(int), cudaMemcpyDeviceToHost));
    return KDT_OK;
}

int kdt_eval_predicates(const int32_t *xy, const int32_t *quads, int64_t m, int32_t *out, int use_filter,
                        void *cuda_stream)
{
    if (m < 0 || (m > 0 && (!xy || !quads || !out))) return KDT_ERR_ARG;
    if (m == 0) return KDT_OK;
    if (m > INT_MAX) return KDT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    k_predicates<<<(int)((m + 255) / 256), 256, 0, st>>>((const int2 *)xy, (const int4 *)quads, (int)m,
                                                        (int4 *)out, use_filter);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return KDT_OK;
}

}  // extern "C"

// ====================================================================== allocation-free export
//
// The scratch of kdt_export_triangles_noalloc: counts (reused as fill cursors) and
// offsets per point, then scan partial sums and the grand total.  Host code must not
// use the symbol's name as a device address: the address is looked up per device
// with cudaGetSymbolAddress and cached.
namespace {

constexpr int NOALLOC_TILES = KDT_NOALLOC_MAX_POINTS / SCAN_TILE + 8;
constexpr size_t NOALLOC_WORDS = 2 * (size_t)KDT_NOALLOC_MAX_POINTS + 1024;
static_assert(NOALLOC_TILES + 1 <= 1024, "tile sums must fit the reserved tail");

static __device__ __align__(256) int g_noalloc_scratch[NOALLOC_WORDS];

constexpr int NOALLOC_MAX_DEVICES = 64;
int *g_noalloc_ptr[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mutex;

// device address of the scratch on `device` (which must be current); nullptr on error
int *noalloc_scratch(int device)
{
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_noalloc_ptr[device] = (int *)p;
    }
    return g_noalloc_ptr[device];
}

}  // namespace

extern "C" int kdt_export_triangles_noalloc(kdt *h, int32_t *out, int64_t cap, int64_t *n_tri)
{
    if (!h || !n_tri || cap < 0 || (cap > 0 && !out)) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    if (h->n > KDT_NOALLOC_MAX_POINTS) return KDT_ERR_TOO_LARGE;
    CK(cudaSetDevice(h->device));
    if (cap > 0 && !on_device(h, out)) return KDT_ERR_ARG;
    int *scratch = noalloc_scratch(h->device);
    if (!scratch) return KDT_ERR_CUDA;
    cudaStream_t st = h->stream;
    const int n = (int)h->n;
    int *cnt = scratch;                                   // counts, then fill cursors
    int *off = scratch + KDT_NOALLOC_MAX_POINTS;          // exclusive offsets
    int *tiles = scratch + 2 * (size_t)KDT_NOALLOC_MAX_POINTS;  // scan partial sums
    int *total = tiles + 1023;                            // grand total
    const int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    CK(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int), st));
    k_exp_count<<<thread_grid(h, h->cap, 256), 256, 0, st>>>(TriHalf{h->tri}, h->cap, cnt, 0);
    k_scan_tile<<<ntiles, SCAN_THREADS, 0, st>>>(cnt, off, n, tiles);
    k_scan_sums<<<1, 1024, 0, st>>>(tiles, ntiles, total);
    k_scan_add<<<ntiles, SCAN_THREADS, 0, st>>>(off, n, tiles);
    h->stats.kernel_launches += 4;
    CK(cudaGetLastError());
    int tot = 0;
    CK(cudaMemcpyAsync(&tot, total, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *n_tri = tot;
    if (tot > cap) return KDT_ERR_CAPACITY;
    CK(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int), st));
    k_exp_place<<<thread_grid(h, h->cap, 256), 256, 0, st>>>(TriHalf{h->tri}, h->cap, off, cnt, (int3 *)out, 0);
    k_exp_sortseg<<<thread_grid(h, n, 256), 256, 0, st>>>(n, off, cnt, (int3 *)out);
    h->stats.kernel_launches += 2;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return KDT_OK;
}


// ------------------------------------------------------------------ learned proposal

extern "C" {

int kdt_set_trace(kdt *h, float *features, int32_t *labels, int64_t cap)
{
    if (!h || cap < 0 || (cap > 0 && (!features || !labels)) || cap > INT_MAX) return KDT_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (cap > 0 && (!on_device(h, features) || !on_device(h, labels))) return KDT_ERR_ARG;
    if (!h->trace_count && cudaMalloc(&h->trace_count, sizeof(int)) != cudaSuccess) return KDT_ERR_CUDA;
    CK(cudaMemsetAsync(h->trace_count, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->trace_x = cap > 0 ? features : nullptr;
    h->trace_y = cap > 0 ? labels : nullptr;
    h->trace_cap = (int)cap;
    h->gen++;  // a captured step graph holds the old Dev
    return KDT_OK;
}

int kdt_trace_count(kdt *h, int64_t *rows)
{
    if (!h || !rows) return KDT_ERR_ARG;
    *rows = 0;
    if (!h->trace_count) return KDT_OK;
    CK(cudaSetDevice(h->device));
    int c = 0;
    CK(cudaMemcpyAsync(&c, h->trace_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *rows = std::min<int64_t>(c, h->trace_cap);
    return KDT_OK;
}

int kdt_set_proposal(kdt *h, const uint16_t *params_bf16)
{
    if (!h) return KDT_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (foreign(h, params_bf16)) return KDT_ERR_ARG;
    if (!params_bf16) {
        h->prop_on = false;
        h->gen++;
        return KDT_OK;
    }
    if (!h->mlp_w && cudaMalloc(&h->mlp_w, MLP_PARAMS * sizeof(uint16_t)) != cudaSuccess) return KDT_ERR_CUDA;
    CK(cudaMemcpyAsync(h->mlp_w, params_bf16, MLP_PARAMS * sizeof(uint16_t),
                       on_device(h, params_bf16) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->prop_on = true;
    h->gen++;
    return KDT_OK;
}

int kdt_mlp_forward(kdt *h, const uint16_t *params_bf16, const float *x, int64_t rows, float *out)
{
    if (!h || rows < 0 || (rows > 0 && (!params_bf16 || !x || !out))) return KDT_ERR_ARG;
    if (rows == 0) return KDT_OK;
    CK(cudaSetDevice(h->device));
    if (!on_device(h, params_bf16) || !on_device(h, x) || !on_device(h, out)) return KDT_ERR_ARG;
    if (((uintptr_t)params_bf16 & 3) != 0) return KDT_ERR_ARG;  // read as BF16 pairs
    long long warps = rows < (1ll << 22) ? rows : (1ll << 22);
    int blocks = (int)((warps * 32 + 255) / 256);
    k_mlp_forward<<<blocks, 256, 0, h->stream>>>((const unsigned short *)params_bf16, x, rows, out);
    h->stats.kernel_launches++;
    CK(cudaGetLastError());
    return KDT_OK;
}

int kdt_mlp_forward_tc(kdt *h, const uint16_t *params_bf16, const float *x, int64_t rows, float *out)
{
    if (!h || rows < 0 || (rows > 0 && (!params_bf16 || !x || !out))) return KDT_ERR_ARG;
    if (rows == 0) return KDT_OK;
    CK(cudaSetDevice(h->device));
    if (!on_device(h, params_bf16) || !on_device(h, x) || !on_device(h, out)) return KDT_ERR_ARG;
    if (((uintptr_t)params_bf16 & 3) != 0) return KDT_ERR_ARG;  // weight rows read as BF16 pairs
    k_mlp_tc<0><<<tc_grid(h, rows), TC_M, TCS_BYTES, h->stream>>>((const unsigned short *)params_bf16, x, rows,
                                                                  nullptr, out, nullptr, nullptr, nullptr, nullptr,
                                                                  h->counters + C_TC_FAIL);
    h->stats.kernel_launches++;
    CK(cudaGetLastError());
    return KDT_OK;
}

// per-block partial gradients for `blocks` blocks (kept between calls)
static int ensure_mlp_part(kdt *h, int blocks)
{
    if (blocks > h->mlp_part_blocks) {
        if (h->mlp_part) cudaFree(h->mlp_part);
        h->mlp_part = nullptr;
        h->mlp_part_blocks = 0;
        if (cudaMalloc(&h->mlp_part, (size_t)blocks * (MLP_PARAMS + 1) * sizeof(float)) != cudaSuccess)
            return KDT_ERR_CUDA;
        h->mlp_part_blocks = blocks;
    }
    return KDT_OK;
}

int kdt_mlp_loss_grad(kdt *h, const uint16_t *params_bf16, const float *x, const int32_t *labels,
                      const int64_t *index, int64_t rows, float lam, float *grad, float *loss)
{
    if (!h || rows <= 0 || !params_bf16 || !x || !labels || !grad) return KDT_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (!on_device(h, params_bf16) || !on_device(h, x) || !on_device(h, labels) || !on_device(h, grad) ||
        (loss && !on_device(h, loss)) || (index && !on_device(h, index)))
        return KDT_ERR_ARG;
    long long tiles = (rows + GT - 1) / GT;
    int blocks = (int)std::min<long long>(tiles, 2ll * sm_count(h->device));
    if (int rc = ensure_mlp_part(h, blocks)) return rc;
    const size_t smem = sizeof(MlpSmem);
    CK(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    float *part_loss = h->mlp_part + (size_t)h->mlp_part_blocks * MLP_PARAMS;
    k_mlp_grad<<<blocks, GTHREADS, smem, h->stream>>>((const unsigned short *)params_bf16, x, (const int *)labels,
                                                     (const long long *)index, rows, lam, h->mlp_part, part_loss);
    k_mlp_reduce<<<(MLP_PARAMS + 255) / 256, 256, 0, h->stream>>>(h->mlp_part, part_loss, blocks, rows, grad, loss);
    h->stats.kernel_launches += 2;
    CK(cudaGetLastError());
    return KDT_OK;
}

int kdt_mlp_loss_grad_tc(kdt *h, const uint16_t *params_bf16, const float *x, const int32_t *labels,
                         const int64_t *index, int64_t rows, float lam, float *grad, float *loss)
{
    if (!h || rows <= 0 || !params_bf16 || !x || !labels || !grad) return KDT_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (!on_device(h, params_bf16) || !on_device(h, x) || !on_device(h, labels) || !on_device(h, grad) ||
        (loss && !on_device(h, loss)) || (index && !on_device(h, index)))
        return KDT_ERR_ARG;
    if (((uintptr_t)params_bf16 & 3) != 0) return KDT_ERR_ARG;  // weight rows read as BF16 pairs
    const int blocks = (int)std::min<long long>((rows + TC_M - 1) / TC_M, sm_count(h->device));
    if (int rc = ensure_mlp_part(h, blocks)) return rc;
    float *part_loss = h->mlp_part + (size_t)h->mlp_part_blocks * MLP_PARAMS;
    k_mlp_grad_tc<<<blocks, TC_M, TG_BYTES, h->stream>>>((const unsigned short *)params_bf16, x, (const int *)labels,
                                                        (const long long *)index, rows, lam, h->mlp_part, part_loss,
                                                        h->counters + C_TC_FAIL);
    k_mlp_reduce<<<(MLP_PARAMS + 255) / 256, 256, 0, h->stream>>>(h->mlp_part, part_loss, blocks, rows, grad, loss);
    h->stats.kernel_launches += 2;
    CK(cudaGetLastError());
    return KDT_OK;
}

int kdt_mlp_adam(kdt *h, float *master, const float *grad, float *m, float *v, int64_t t, float lr, float beta1,
                 float beta2, float eps, uint16_t *params_bf16)
{
    if (!h || !master || !grad || !m || !v || t < 1) return KDT_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (!on_device(h, master) || !on_device(h, grad) || !on_device(h, m) || !on_device(h, v) ||
        (params_bf16 && !on_device(h, params_bf16)))
        return KDT_ERR_ARG;
    double bc1 = 1.0 - std::pow((double)beta1, (double)t), bc2 = 1.0 - std::pow((double)beta2, (double)t);
    k_mlp_adam<<<(MLP_PARAMS + 255) / 256, 256, 0, h->stream>>>(master, grad, m, v, MLP_PARAMS, lr, beta1, beta2, eps,
                                                                (float)bc1, (float)bc2,
                                                                (unsigned short *)params_bf16);
    h->stats.kernel_launches++;
    CK(cudaGetLastError());
    return KDT_OK;
}

}  // extern "C"
