// C-ABI and host orchestration of the GB300 kinetic Delaunay library.
// The declarations, argument conventions and error behaviour are in include/kdt.h.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/kdt.h"
#include "kdt_kernels.cuh"

using namespace kd;

namespace {

constexpr int ABI_VERSION = 1;

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct kdt {
    int device = 0;
    cudaStream_t stream = nullptr;
    kdt_config cfg{};
    int grid = 1;  // partitions per side in use
    int64_t n = 0;
    int cap = 0;  // triangle slots (2n - 2)
    bool built = false;
    int stamp = 0;
    // state
    int2 *xy = nullptr;
    int *pt_tri = nullptr;
    int *pt_stamp = nullptr;
    int4 *tv = nullptr;
    int4 *tn = nullptr;
    int *scal = nullptr;                       // S_NUM device scalars
    unsigned long long *counters = nullptr;    // C_NUM
    int *dirty = nullptr;
    int dirty_cap = 0;
    int *viol = nullptr;
    int viol_cap = 0;
    // step buffers
    int mcap = 0;
    int3 *moves = nullptr;
    int2 *old_xy = nullptr;
    int *move_cell = nullptr;
    int *order = nullptr;
    int4 *deferred = nullptr;
    int ncells = 0;
    int *cell_cnt = nullptr, *cell_off = nullptr, *cell_fill = nullptr;
    int *scan_tmp = nullptr;
    int scan_tmp_cap = 0;
    // build / export temporaries (kept between calls)
    Buf key, bord, hist, hoff, exp_cnt, exp_off, exp_fill, exp_out, in_xy;
    // graph-launched step: control words (moves, stamp) and the captured graph
    int *ctl = nullptr;    // device
    int *hctl = nullptr;   // pinned host
    cudaStream_t cstream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_gen = -1;    // buffer generation the graph was captured for
    int gen = 0;           // bumped whenever step buffers are (re)allocated
    // host side
    int *hscal = nullptr;  // pinned copy of the scalars
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
    kdt_stats stats{};
};

namespace {

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
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

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

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
    d.tv = h->tv;
    d.tn = h->tn;
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
    return d;
}

// exclusive scan in place (or out of place) of n ints; *total receives the sum
int scan(kdt *h, const int *in, int *out, int n, int *total, cudaStream_t st)
{
    int tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles < 1) tiles = 1;
    if (tiles + 1 > h->scan_tmp_cap) {
        int c = tiles + 1024;
        if (dalloc(&h->scan_tmp, (size_t)c)) return KDT_ERR_CUDA;
        h->scan_tmp_cap = c;
        h->gen++;  // a captured step graph holds the old pointer
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

// Certify (dirty range or everything), then repair until no violation is left.
// Returns a device status (0 fine).
int certify_and_repair(kdt *h, bool all, int *dev_status)
{
    Dev d = make_dev(h);
    if (all && d.retry_cap < 4096) d.retry_cap = 4096;
    bool full = all;
    int lo = 0;
    for (int round = 0; round < 64; ++round) {
        CK(cudaMemsetAsync(h->scal + S_VIOL, 0, sizeof(int), h->stream));
        CK(cudaMemsetAsync(h->scal + S_WRAPS, 0, sizeof(int), h->stream));
        if (full) {
            k_certify_all<<<thread_grid(h, h->cap, 256), 256, 0, h->stream>>>(
                d, h->cap, h->viol, h->scal + S_VIOL, h->viol_cap, h->scal + S_WRAPS);
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
            // every edge is locally Delaunay; after a full pass the hull must also wind once
            if (full && h->hscal[S_WRAPS] != 1) *dev_status = DEV_INTERNAL;
            return 0;
        }
        if (nv > h->viol_cap) nv = h->viol_cap;  // the rest is found again next round
        int dirty_before = h->hscal[S_DIRTY];
        full = all || dirty_before > h->dirty_cap;
        lo = dirty_before;
        k_fixup<<<warp_grid(h, nv, 16), WPB * 32, 0, h->stream>>>(d, h->viol, nv);
        h->stats.kernel_launches++;
        CK(cudaGetLastError());
        if (sync_scalars(h)) return KDT_ERR_CUDA;
        *dev_status = h->hscal[S_STATUS];
        if (*dev_status) return 0;
        if (!full && h->hscal[S_DIRTY] > h->dirty_cap) full = true;
    }
    *dev_status = DEV_INTERNAL;
    return 0;
}

// Build the triangulation of the positions already in h->xy (kdt_build, kdt_rebuild
// and the step fallback).  Returns an ABI code.
int rebuild_positions(kdt *h)
{
    const int n = (int)h->n;
    cudaStream_t st = h->stream;
    h->built = false;
    h->stamp++;
    Dev d = make_dev(h);
    d.dirty_cap = 0;  // the build certifies every slot instead
    if (d.retry_cap < 4096) d.retry_cap = 4096;  // the step's cap does not apply to builds
    CK(cudaMemsetAsync(h->scal, 0, S_NUM * sizeof(int), st));
    int init_bbox[4] = {INT_MAX, INT_MAX, INT_MIN, INT_MIN};
    CK(cudaMemcpyAsync(h->scal + S_MINX, init_bbox, sizeof init_bbox, cudaMemcpyHostToDevice, st));
    int third0 = INT_MAX;
    CK(cudaMemcpyAsync(h->scal + S_THIRD, &third0, sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->tv, 0, (size_t)h->cap * sizeof(int4), st));
    CK(cudaMemsetAsync(h->tn, 0, (size_t)h->cap * sizeof(int4), st));
    k_fill_int<<<thread_grid(h, n, 256), 256, 0, st>>>(h->pt_tri, n, -1);
    k_range<<<thread_grid(h, n, 256), 256, 0, st>>>(h->xy, n, h->cfg.domain_bits, h->scal + S_STATUS,
                                                    h->scal + S_MINX);
    h->stats.kernel_launches += 2;
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    if (h->hscal[S_STATUS]) return dev_to_abi(h->hscal[S_STATUS]);
    // spatial order: cells of a 2^k x 2^k grid over the bounding box, Hilbert order
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
    k_hilbert<<<(n + 255) / 256, 256, 0, st>>>(h->xy, n, h->scal + S_MINX, k, shift, key, hist);
    h->stats.kernel_launches++;
    if (scan(h, hist, hoff, (int)ncell, h->scal + S_TOTAL, st)) return KDT_ERR_CUDA;
    CK(cudaMemsetAsync(hist, 0, ncell * 4, st));
    k_place_order<<<(n + 255) / 256, 256, 0, st>>>(n, key, hoff, hist, order);
    k_third<<<thread_grid(h, n, 256), 256, 0, st>>>(h->xy, n, order, h->scal + S_THIRD);
    h->stats.kernel_launches += 2;
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    if (h->hscal[S_THIRD] == INT_MAX) return KDT_ERR_DEGENERATE;
    k_init<<<1, 1, 0, st>>>(d, order, h->scal + S_THIRD, h->scal + S_TRIS);
    h->stats.kernel_launches++;
    // levels: sorted index i is inserted at level ctz(i), highest level first
    int K = 0;
    while ((1ll << (K + 1)) < (long long)n) ++K;
    long long inserted = 3;
    for (int lev = K; lev >= 0; --lev) {
        long long items = ((long long)n - 1 + (1ll << lev)) >> (lev + 1);  // odd multiples of 2^lev below n
        if (items <= 0) continue;
        long long conc = inserted / 8;
        if (conc < 64) conc = 64;
        if (h->cfg.build_warps > 0) conc = h->cfg.build_warps;
        long long warps = items < conc ? items : conc;
        int blocks = warp_grid(h, warps, 64), threads = WPB * 32;
        if (h->cfg.build_warps > 0 && h->cfg.build_warps < WPB) {
            blocks = 1;
            threads = 32 * h->cfg.build_warps;
        }
        k_insert_level<<<blocks, threads, 0, st>>>(d, order, lev, (int)items, h->scal + S_TRIS);
        h->stats.kernel_launches++;
        CK(cudaGetLastError());
        inserted += items;
    }
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    if (h->hscal[S_STATUS]) return dev_to_abi(h->hscal[S_STATUS]);
    if (h->hscal[S_TRIS] != h->cap) return KDT_ERR_INTERNAL;
    int ds = 0;
    if (certify_and_repair(h, true, &ds)) return KDT_ERR_CUDA;
    if (ds) return dev_to_abi(ds);
    h->built = true;
    h->stats.rebuilds++;
    return KDT_OK;
}

int ensure_moves(kdt *h, int64_t m)
{
    if (m <= h->mcap) return 0;
    int c = (int)std::max<int64_t>(m, 1024);
    if (dalloc(&h->moves, c) || dalloc(&h->old_xy, c) || dalloc(&h->move_cell, c) || dalloc(&h->order, c) ||
        dalloc(&h->deferred, c))
        return KDT_ERR_CUDA;
    h->mcap = c;
    long long dc = 64ll * c + 4096;
    if (dc > (1ll << 30)) dc = 1ll << 30;
    if (dalloc(&h->dirty, (size_t)dc)) return KDT_ERR_CUDA;
    h->dirty_cap = (int)dc;
    h->gen++;
    return 0;
}

int alloc_state(kdt *h, int64_t n)
{
    h->n = n;
    h->cap = (int)(2 * n - 2);
    h->built = false;
    if (dalloc(&h->xy, n) || dalloc(&h->pt_tri, n) || dalloc(&h->pt_stamp, n) || dalloc(&h->tv, h->cap) ||
        dalloc(&h->tn, h->cap))
        return KDT_ERR_CUDA;
    CK(cudaMemsetAsync(h->pt_stamp, 0, n * sizeof(int), h->stream));
    h->viol_cap = std::max(4096, h->cap);
    if (dalloc(&h->viol, (size_t)h->viol_cap)) return KDT_ERR_CUDA;
    int G = h->cfg.grid;
    if (G <= 0) {
        G = 1;
        while ((long long)G * G * 256 < n && G < 4096) G *= 2;
    }
    h->grid = G;
    h->ncells = G * G;
    if (dalloc(&h->cell_cnt, h->ncells) || dalloc(&h->cell_off, h->ncells) || dalloc(&h->cell_fill, h->ncells))
        return KDT_ERR_CUDA;
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
    void *ps[] = {h->xy, h->pt_tri, h->pt_stamp, h->tv, h->tn, h->viol, h->moves, h->old_xy, h->move_cell,
                  h->order, h->deferred, h->dirty, h->cell_cnt, h->cell_off, h->cell_fill, h->scan_tmp};
    for (void *p : ps)
        if (p) cudaFree(p);
    h->xy = nullptr; h->pt_tri = nullptr; h->pt_stamp = nullptr; h->tv = nullptr; h->tn = nullptr;
    h->viol = nullptr; h->moves = nullptr; h->old_xy = nullptr; h->move_cell = nullptr; h->order = nullptr;
    h->deferred = nullptr; h->dirty = nullptr; h->cell_cnt = nullptr; h->cell_off = nullptr;
    h->cell_fill = nullptr; h->scan_tmp = nullptr;
    h->mcap = 0; h->dirty_cap = 0; h->scan_tmp_cap = 0;
    Buf *bs[] = {&h->key, &h->bord, &h->hist, &h->hoff, &h->exp_cnt, &h->exp_off, &h->exp_fill, &h->exp_out,
                 &h->in_xy};
    for (Buf *b : bs) free_buf(*b);
    h->n = 0;
    h->cap = 0;
    h->built = false;
}

void add_counters(kdt *h)
{
    unsigned long long c[C_NUM + 1];
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
}

// Undo a step that failed after it started: restore the old positions and rebuild.
int roll_back(kdt *h, const int3 *mp, int m)
{
    k_restore_positions<<<(m + 255) / 256, 256, 0, h->stream>>>(h->xy, mp, h->old_xy, m);
    h->stats.kernel_launches++;
    return rebuild_positions(h);
}

int verify_state(kdt *h, int64_t *bad)
{
    Dev d = make_dev(h);
    CK(cudaMemsetAsync(h->scal + S_BAD, 0, 3 * sizeof(int), h->stream));
    k_verify<<<thread_grid(h, std::max<int64_t>(h->cap, h->n), 256), 256, 0, h->stream>>>(
        d, h->cap, h->scal + S_BAD, h->scal + S_ALIVE, h->scal + S_WRAPS);
    h->stats.kernel_launches++;
    CK(cudaGetLastError());
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    int64_t b = h->hscal[S_BAD];
    if (h->hscal[S_ALIVE] != h->cap) b += 1;
    if (h->hscal[S_WRAPS] != 1) b += 1;  // the hull must wind exactly once
    *bad = b;
    return 0;
}

// Issue one step's kernels on `st`: intake, per-partition counting sort, the kinetic
// kernel, deferred insertions, certification, and the copy of the status scalars to
// the host.  With from_ctl the grids do not depend on m (the kernels read m and the
// stamp from h->ctl), so the sequence can be captured once into a CUDA graph.
int enqueue_step(kdt *h, cudaStream_t st, const Dev &d, const int3 *mp, int mi, bool from_ctl)
{
    int cap = from_ctl ? h->mcap : mi;
    CK(cudaMemsetAsync(h->scal, 0, S_NUM * sizeof(int), st));
    CK(cudaMemsetAsync(h->cell_cnt, 0xff, (size_t)h->ncells * sizeof(int), st));  // empty lists
    k_intake_link<<<thread_grid(h, cap, 256), 256, 0, st>>>(d, mp, mi, h->grid, h->cfg.domain_bits, h->cell_cnt,
                                                            h->move_cell, h->old_xy);
    // inside a capture an event record must be an external node to keep its timestamp
    unsigned evflags = from_ctl ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (h->cfg.timing) CK(cudaEventRecordWithFlags(h->ev0, st, evflags));
    int kblocks = warp_grid(h, h->ncells, 64), kthreads = WPB * 32;
    if (h->cfg.kinetic_warps > 0) {
        kblocks = (h->cfg.kinetic_warps + WPB - 1) / WPB;
        if (h->cfg.kinetic_warps < WPB) kthreads = 32 * h->cfg.kinetic_warps;
    }
    k_kinetic<<<kblocks, kthreads, 0, st>>>(d, mp, h->cell_cnt, h->move_cell, h->ncells, h->deferred,
                                            h->scal + S_DEFER, h->mcap, h->viol, h->viol_cap);
    if (h->cfg.timing) CK(cudaEventRecordWithFlags(h->ev1, st, evflags));
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->hscal, h->scal, S_NUM * sizeof(int), cudaMemcpyDeviceToHost, st));
    return 0;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

int kdt_version(void) { return ABI_VERSION; }

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
    return KDT_OK;
}

int kdt_create(kdt **out, const kdt_config *cfg, int device, void *cuda_stream)
{
    if (!out) return KDT_ERR_ARG;
    *out = nullptr;
    kdt_config c;
    if (cfg) c = *cfg;
    else kdt_default_config(&c);
    if (c.domain_bits <= 0 || c.domain_bits > 28 || c.grid < 0 || c.grid > 4096 || c.retry_cap < 0)
        return KDT_ERR_ARG;
    if (c.retry_cap == 0) c.retry_cap = 4096;
    if (cudaSetDevice(device) != cudaSuccess) return KDT_ERR_CUDA;
    kdt *h = new (std::nothrow) kdt();
    if (!h) return KDT_ERR_ARG;
    h->device = device;
    h->stream = (cudaStream_t)cuda_stream;
    h->cfg = c;
    if (cudaMalloc(&h->scal, S_NUM * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->counters, (C_NUM + 1) * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&h->hscal, S_NUM * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->ctl, 4 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&h->hctl, 4 * sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
        cudaEventCreate(&h->ev2) != cudaSuccess || cudaEventCreate(&h->ev3) != cudaSuccess) {
        kdt_destroy(h);
        return KDT_ERR_CUDA;
    }
    cudaMemset(h->scal, 0, S_NUM * sizeof(int));
    cudaMemset(h->counters, 0, (C_NUM + 1) * sizeof(unsigned long long));
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
    if (h->hscal) cudaFreeHost(h->hscal);
    if (h->ctl) cudaFree(h->ctl);
    if (h->hctl) cudaFreeHost(h->hctl);
    if (h->cstream) cudaStreamDestroy(h->cstream);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev2) cudaEventDestroy(h->ev2);
    if (h->ev3) cudaEventDestroy(h->ev3);
    delete h;
    return KDT_OK;
}

int64_t kdt_num_points(const kdt *h) { return h && h->built ? h->n : 0; }

int kdt_build(kdt *h, const int32_t *xy, int64_t n)
{
    if (!h || !xy || n < 0 || n > (1ll << 28)) return KDT_ERR_ARG;
    if (n < 3) return KDT_ERR_DEGENERATE;
    CK(cudaSetDevice(h->device));
    free_state(h);
    int rc = alloc_state(h, n);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->xy, xy, (size_t)n * sizeof(int2),
                       is_device_ptr(xy) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    rc = rebuild_positions(h);
    return rc;
}

int kdt_rebuild(kdt *h)
{
    if (!h) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    CK(cudaSetDevice(h->device));
    int rc = rebuild_positions(h);
    return rc;
}

int kdt_step(kdt *h, const kdt_move *moves, int64_t m)
{
    if (!h || m < 0 || (m > 0 && !moves)) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    if (m == 0) return KDT_OK;
    if (m > h->n) return KDT_ERR_DUPLICATE;  // some id must repeat (or be out of range)
    CK(cudaSetDevice(h->device));
    int rc = ensure_moves(h, m);
    if (rc) return rc;
    cudaStream_t st = h->stream;
    const int mi = (int)m;
    // device moves are read in place; host moves are copied in first
    const int3 *mp = (const int3 *)moves;
    if (!is_device_ptr(moves)) {
        CK(cudaMemcpyAsync(h->moves, moves, (size_t)m * sizeof(int3), cudaMemcpyHostToDevice, st));
        mp = h->moves;
    }
    h->stamp++;
    Dev d = make_dev(h);
    bool large = h->cfg.fallback && (double)m > (double)h->cfg.rebuild_ratio * (double)h->n;
    if (large) {
        // a step this large is cheaper as a rebuild (Abstract: "if the points move so
        // far, it's better to rebuild the triangulation")
        CK(cudaMemsetAsync(h->scal, 0, S_NUM * sizeof(int), st));
        CK(cudaMemsetAsync(h->cell_cnt, 0, (size_t)h->ncells * sizeof(int), st));
        k_intake<<<(mi + 255) / 256, 256, 0, st>>>(d, mp, mi, h->grid, h->cfg.domain_bits, h->cell_cnt,
                                                   h->old_xy, h->move_cell);
        h->stats.kernel_launches++;
        if (sync_scalars(h)) return KDT_ERR_CUDA;
        if (h->hscal[S_STATUS]) return dev_to_abi(h->hscal[S_STATUS]);
        k_set_positions<<<(mi + 255) / 256, 256, 0, st>>>(h->xy, mp, mi);
        h->stats.kernel_launches++;
        rc = rebuild_positions(h);
        if (rc) {
            int rr = roll_back(h, mp, mi);
            return rr ? rr : rc;
        }
        h->stats.steps++;
        h->stats.moves += m;
        return KDT_OK;
    }
    if (h->cfg.use_graph) {
        // one graph launch per step: the kernels read m and the stamp from ctl
        if (h->graph_gen != h->gen) {
            drop_graph(h);
            // nothing may allocate while capturing: size the scan scratch first
            if (scan(h, h->cell_cnt, h->cell_off, h->ncells, h->scal + S_TOTAL, st)) return KDT_ERR_CUDA;
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
        if (h->cfg.timing) CK(cudaEventRecord(h->ev2, st));
        CK(cudaMemcpyAsync(h->ctl, h->hctl, 4 * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaGraphLaunch(h->gexec, st));
        if (h->cfg.timing) CK(cudaEventRecord(h->ev3, st));
        h->stats.kernel_launches += 2;
        CK(cudaStreamSynchronize(st));
    } else {
        if (enqueue_step(h, st, d, mp, mi, false)) return KDT_ERR_CUDA;
        h->stats.kernel_launches += 2;
        CK(cudaStreamSynchronize(st));
    }
    if (h->hscal[S_CERTPEND] && !h->hscal[S_STATUS]) {
        // a long dirty list (global-path writes): certify it here, appending to the
        // violations the kinetic kernel already recorded
        k_certify<<<thread_grid(h, h->hscal[S_DIRTY], 256), 256, 0, st>>>(d, 0, h->viol, h->scal + S_VIOL,
                                                                          h->viol_cap);
        h->stats.kernel_launches++;
        if (sync_scalars(h)) return KDT_ERR_CUDA;
    }
    if (h->cfg.timing) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) {
            h->stats.kinetic_kernel_ms += ms;
            h->stats.kinetic_kernel_timed++;
        }
        if (h->cfg.use_graph && cudaEventElapsedTime(&ms, h->ev2, h->ev3) == cudaSuccess)
            h->stats.step_graph_ms += ms;
    }
    int s = h->hscal[S_STATUS];
    if (s == DEV_ARG || s == DEV_RANGE || s == DEV_DUP_ID) {
        // found at intake: nothing was modified
        return dev_to_abi(s);
    }
    if (s == 0) {
        int nv = h->hscal[S_VIOL];
        bool overflow = h->hscal[S_DIRTY] > h->dirty_cap;
        if (nv > 0 || overflow) {
            int ds = 0;
            if (overflow) {
                if (certify_and_repair(h, true, &ds)) return KDT_ERR_CUDA;
            } else {
                // repair the violations already found, then certify what the repair wrote
                h->stats.violations += nv;
                if (nv > h->viol_cap) nv = h->viol_cap;
                int dirty_before = h->hscal[S_DIRTY];
                k_fixup<<<warp_grid(h, nv, 16), WPB * 32, 0, st>>>(d, h->viol, nv);
                h->stats.kernel_launches++;
                CK(cudaGetLastError());
                if (sync_scalars(h)) return KDT_ERR_CUDA;
                ds = h->hscal[S_STATUS];
                if (!ds) {
                    // certify the slots written by the repair (dirty range after dirty_before)
                    Dev d2 = make_dev(h);
                    bool all = h->hscal[S_DIRTY] > h->dirty_cap;
                    if (all) {
                        if (certify_and_repair(h, true, &ds)) return KDT_ERR_CUDA;
                    } else {
                        for (int round = 0; round < 64; ++round) {
                            CK(cudaMemsetAsync(h->scal + S_VIOL, 0, sizeof(int), st));
                            k_certify<<<thread_grid(h, 65536, 256), 256, 0, st>>>(d2, dirty_before, h->viol,
                                                                                 h->scal + S_VIOL, h->viol_cap);
                            h->stats.kernel_launches++;
                            if (sync_scalars(h)) return KDT_ERR_CUDA;
                            ds = h->hscal[S_STATUS];
                            int nv2 = h->hscal[S_VIOL];
                            if (ds || nv2 == 0) break;
                            h->stats.violations += nv2;
                            if (nv2 > h->viol_cap) nv2 = h->viol_cap;
                            dirty_before = h->hscal[S_DIRTY];
                            k_fixup<<<warp_grid(h, nv2, 16), WPB * 32, 0, st>>>(d2, h->viol, nv2);
                            h->stats.kernel_launches++;
                            if (sync_scalars(h)) return KDT_ERR_CUDA;
                            ds = h->hscal[S_STATUS];
                            if (ds) break;
                            if (h->hscal[S_DIRTY] > h->dirty_cap) {
                                if (certify_and_repair(h, true, &ds)) return KDT_ERR_CUDA;
                                break;
                            }
                        }
                    }
                }
            }
            s = ds;
        }
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
            k_set_positions<<<(mi + 255) / 256, 256, 0, st>>>(h->xy, mp, mi);
            h->stats.kernel_launches++;
            rc2 = rebuild_positions(h);
        }
        if (rc2) {
            int rr = roll_back(h, mp, mi);
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
        if (bad) {
            return KDT_ERR_INTERNAL;
        }
    }
    return KDT_OK;
}

int kdt_export_triangles(kdt *h, int32_t *out, int64_t cap, int64_t *n_tri)
{
    if (!h || !n_tri || cap < 0 || (cap > 0 && !out)) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    CK(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    const int n = (int)h->n;
    if (grow(h->exp_cnt, (size_t)n * 4) || grow(h->exp_off, (size_t)n * 4) || grow(h->exp_fill, (size_t)n * 4))
        return KDT_ERR_CUDA;
    int *cnt = (int *)h->exp_cnt.p, *off = (int *)h->exp_off.p, *fill = (int *)h->exp_fill.p;
    CK(cudaMemsetAsync(cnt, 0, (size_t)n * 4, st));
    k_exp_count<<<thread_grid(h, h->cap, 256), 256, 0, st>>>(h->tv, h->cap, cnt);
    h->stats.kernel_launches++;
    if (scan(h, cnt, off, n, h->scal + S_TOTAL, st)) return KDT_ERR_CUDA;
    if (sync_scalars(h)) return KDT_ERR_CUDA;
    int64_t total = h->hscal[S_TOTAL];
    *n_tri = total;
    if (total > cap) return KDT_ERR_CAPACITY;
    bool dev_out = is_device_ptr(out);
    int3 *dst;
    if (dev_out) {
        dst = (int3 *)out;
    } else {
        if (grow(h->exp_out, (size_t)std::max<int64_t>(total, 1) * sizeof(int3))) return KDT_ERR_CUDA;
        dst = (int3 *)h->exp_out.p;
    }
    CK(cudaMemsetAsync(fill, 0, (size_t)n * 4, st));
    k_exp_place<<<thread_grid(h, h->cap, 256), 256, 0, st>>>(h->tv, h->cap, off, fill, dst);
    k_exp_sortseg<<<thread_grid(h, n, 256), 256, 0, st>>>(n, off, cnt, dst);
    h->stats.kernel_launches += 2;
    CK(cudaGetLastError());
    if (!dev_out && total > 0)
        CK(cudaMemcpyAsync(out, dst, (size_t)total * sizeof(int3), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return KDT_OK;
}

int kdt_export_points(kdt *h, int32_t *xy, int64_t cap_points)
{
    if (!h || !xy || cap_points < 0) return KDT_ERR_ARG;
    if (!h->built) return KDT_ERR_STATE;
    if (cap_points < h->n) return KDT_ERR_CAPACITY;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpyAsync(xy, h->xy, (size_t)h->n * sizeof(int2),
                       is_device_ptr(xy) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return KDT_OK;
}

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
    memset(&h->stats, 0, sizeof h->stats);
    return KDT_OK;
}

int kdt_export_store(kdt *h, int32_t *tv, int32_t *tn, int32_t *pt_tri, int64_t cap_slots)
{
    if (!h || cap_slots < 0) return KDT_ERR_ARG;
    if (h->n == 0) return KDT_ERR_STATE;
    if (cap_slots < h->cap) return KDT_ERR_CAPACITY;
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    if (tv) CK(cudaMemcpy(tv, h->tv, (size_t)h->cap * sizeof(int4), cudaMemcpyDeviceToHost));
    if (tn) CK(cudaMemcpy(tn, h->tn, (size_t)h->cap * sizeof(int4), cudaMemcpyDeviceToHost));
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
    if (cap > 0 && !is_device_ptr(out)) return KDT_ERR_ARG;
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
    k_exp_count<<<thread_grid(h, h->cap, 256), 256, 0, st>>>(h->tv, h->cap, cnt);
    k_scan_tile<<<ntiles, SCAN_THREADS, 0, st>>>(cnt, off, n, tiles);
    k_scan_sums<<<1, 1024, 0, st>>>(tiles, ntiles, total);
    k_scan_add<<<ntiles, SCAN_THREADS, 0, st>>>(off, n, tiles);
    CK(cudaGetLastError());
    int tot = 0;
    CK(cudaMemcpyAsync(&tot, total, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *n_tri = tot;
    if (tot > cap) return KDT_ERR_CAPACITY;
    CK(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int), st));
    k_exp_place<<<thread_grid(h, h->cap, 256), 256, 0, st>>>(h->tv, h->cap, off, cnt, (int3 *)out);
    k_exp_sortseg<<<thread_grid(h, n, 256), 256, 0, st>>>(n, off, cnt, (int3 *)out);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return KDT_OK;
}

