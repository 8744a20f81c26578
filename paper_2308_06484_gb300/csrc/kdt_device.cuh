// Device-side triangle store and the warp-cooperative operations of the kinetic
// update: star deletion (paper, Section IV "Insertion and Deletion", the simple
// deletion it prefers), walk + split + Lawson flips for insertion (Section IV,
// insertion; the result equals Bowyer-Watson's), and the claim protocol that lets
// partitions ("blocks", Fig. 4) work in parallel on one shared triangulation.
//
// Store (structure of arrays, 32 B per triangle, ghosts included, 2n-2 slots):
//   tv[t] = int4(v0, v1, v2, flags)   vertices counter-clockwise; KDT_GHOST = infinity;
//                                      flags bit 0 = alive
//   tn[t] = int4(n0, n1, n2, owner)   n_i = (neighbour << 2) | edge index in the
//                                      neighbour, across the edge opposite v_i;
//                                      owner = claim token (0 = free)
//   xy[p] = int2 position, pt_tri[p] = an incident live triangle (-1 while p is
//   deleted inside a step).
//
// Execution model.  One warp runs one operation.  Control flow is warp-uniform:
// every lane computes the same sequential logic on the same values, global reads
// are done by one or several lanes and broadcast with shuffles, global writes are
// issued by lane 0, and lane-parallel sections (claims, loads, ear tests) combine
// through ballots.  Claims are taken with atomicCAS on the owner word, never waited
// for while holding others (release all, back off, retry), so no deadlock exists;
// every retry loop is capped and reports KDT_DEV_RETRY on exhaustion.
#pragma once
#include "kdt_predicates.cuh"

namespace kd {

constexpr unsigned FULL = 0xffffffffu;
constexpr int KMAX = 64;               // largest vertex degree a deletion handles
constexpr int MAXC = 2 * KMAX + 16;    // claims one warp may hold
constexpr int STACK = 48;              // Lawson flip stack per warp
constexpr int WALK_CAP = 1 << 12;      // steps before a walk restarts
constexpr int WALK_RESTARTS = 1024;    // restarts before point location gives up
constexpr int ALIVE = 1;
constexpr int LM = 64;                 // triangles a staged region holds

// device status codes (first error wins); mapped to the C-ABI codes on the host
enum DevStatus : int {
    DEV_OK = 0,
    DEV_RETRY = 1,        // claim retries exhausted
    DEV_DEGREE = 2,       // vertex degree above KMAX
    DEV_DUPLICATE = 3,    // a point would coincide with another
    DEV_DEGENERATE = 4,   // a deletion would leave all points collinear
    DEV_INTERNAL = 5,     // inconsistent store (never expected)
    DEV_WALK = 6,         // point location failed (never expected)
    DEV_ARG = 7,          // a move failed validation (id / range / repeated id)
    DEV_RANGE = 8,
    DEV_CAPACITY = 9,     // a work list overflowed
};

// Results of the insertion routines besides 0 (done) and a DevStatus error (> 0):
// negative, so they never collide with a status.
constexpr int INS_DEFER = -10;   // q lies on a vertex still moving in this step
constexpr int INS_GLOBAL = -11;  // (staged insertion) the caller must use the global path
constexpr int DEL_BUSY = -12;    // (deletion) claims kept failing: nothing was changed
constexpr int DEL_HUGE = -13;    // (deletion) the degree grew above the star arrays: nothing was changed
// Claim losses after which a move stops competing and is left for later (taken again by
// a warp out of partitions, finally by the last warp when no other warp runs): an
// operation with a large footprint (whose star shares long thin triangles with many
// neighbours) can otherwise keep losing against the small ones around it.
constexpr int DEFER_AFTER = 16;

enum Counter : int {
    C_FLIPS = 0, C_RETRIES, C_WALK_STEPS, C_EXACT, C_TIES, C_DEFERRED, C_VIOL, C_FIX_FLIPS,
    C_DEG_DEL, C_STACK_DROP, C_SPLIT_EDGE, C_SPLIT_GHOST, C_DELETES, C_INSERTS, C_FLIP_TESTS,
    C_MV_GLOBAL, C_CYC_MOVE, C_CYC_GATHER, C_CYC_CLAIM, C_CYC_LOCAL, C_CYC_WB,
    C_CYC_EAR, C_CYC_LAWSON, C_CYC_CERT, C_PROP_MOVES, C_PROP_HITS, C_TRACE_ROWS,
    C_NUM,
    C_CYC_MAX = C_NUM,  // a second device slot, updated with atomicMax
    // device-only slots for rare events, added straight to global memory (dev_count)
    C_TAIL_MOVES, C_CYC_TAIL, C_BIG_MOVES, C_CYC_BIG, C_DRAIN_MOVES,
    // high-degree moves: done in place, and the cycles of the in-place attempts and of
    // the deletions (C_CYC_BIG is their whole time, insertion included); the longest move
    // run without giving up (atomicMax)
    C_BIG_INPLACE, C_CYC_BIG_INPLACE, C_CYC_BIG_DELETE, C_BIG_MAX,
    // insertions on the global-memory path after a deletion: cycles, and the longest one
    C_CYC_GLOBAL_INS, C_GLOBAL_INS_MAX,
    // timeline of a kinetic launch (global timer, ns): its start, the latest end of a
    // warp's partitions and of its drain; summed spans from the start
    C_T0, C_TT, C_TD, C_SPAN_TICKETS, C_SPAN_DRAIN, C_SPAN_ALL,
    C_TH, C_TDM, C_SPAN_HUGE, C_SPAN_DRAINED, C_DRAINED_MAX, C_REDEFER,
    // CTAs of the tensor-core network kernels that gave up waiting for their products
    C_TC_FAIL,
    C_SLOTS
};

// One half of the triangle store.  A triangle is one 32-byte record: its vertex half
// (tv: three point ids, the alive flag) at an even int4 slot and its neighbour half (tn:
// three (slot << 2 | edge) references, the claim owner word) right after it, so both
// halves of a triangle come from one DRAM sector.  tv[t] / tv + t reach record t's
// vertex half, tn[t] / tn + t its neighbour half.
struct TriHalf {
    int4 *p;  // this half of record 0
    __host__ __device__ __forceinline__ int4 &operator[](long long t) const { return p[2 * t]; }
    __host__ __device__ __forceinline__ int4 *operator+(long long t) const { return p + 2 * t; }
};

struct Dev {
    // (pointers first, then 32-bit fields: no padding, the struct is copied into every
    // block's shared memory)
    int2 *xy;
    int *pt_tri;
    TriHalf tv;
    TriHalf tn;
    int *status;
    int *dirty;          // slots written in this step (for certification)
    int *dirty_count;
    int *pt_stamp;       // step stamp of points moved in this step
    const int *ctl;      // graph-launched steps: ctl[0] = moves, ctl[1] = stamp,
                         // ctl[2..3] = the moves' device address
    int *viol;           // edges found not locally Delaunay: (slot << 2) | edge
    int *viol_count;
    unsigned long long *counters;
    // learned locate proposal (kdt_mlp.cuh) and its training rows; null = off
    const unsigned short *mlp;  // network parameters, BF16
    const signed char *pguess;  // the step planner's guess per point (0..16, -1 none), or null:
                                // the move evaluates the network itself
    float *trace_x;             // features, trace_cap x 32
    int *trace_y;               // (slot, cavity size) per row
    int *trace_count;           // rows written (may exceed trace_cap: later rows dropped)
    // per-warp global scratch for the deletion of a point of degree above KMAX: set for
    // the kinetic launch only (BIG_INTS ints per warp of that launch), else null
    int *big;
    int n;
    int cap;
    int dirty_cap;
    int stamp;
    int viol_cap;
    int rlo, rn;         // the points of the instance being worked on (walk restarts)
    int use_filter;
    int retry_cap;
    int trace_cap;
    int variant;         // 1: try a move in place before delete + insert (kdt_config.variant)
    int timeline;        // record the kinetic launch's timeline (the C_T* / C_SPAN* slots)
};

constexpr int KBIG = 1024;                  // largest degree the global deletion handles
constexpr int BIG_INTS = 9 * KBIG + 64;     // S, I, L, ON, T, LX (2), claims (2 KBIG + 64)

// The star arrays of a deletion: in the warp's shared block (degree <= KMAX) or in its
// global scratch (degree <= KBIG).
struct Star {
    int *S;    // star triangle slots, counter-clockwise around p
    int *I;    // index of p in each
    int *L;    // link vertices
    int *ON;   // outer refs across the link edges
    int *T;    // scratch (the ring's slots for the claims)
    int2 *LX;  // link coordinates
    int cap;
};

struct WarpShared {
    int cl[MAXC];          // claimed slots
    int S[KMAX];           // star slots
    int I[KMAX];           // index of the centre in each star triangle
    int L[KMAX];           // link vertices (ccw)
    int ON[KMAX];          // outer refs across link edges
    int2 LX[KMAX];         // link coordinates
    int2 stack[STACK];     // flip stack: (slot, edge)
    int tmp[64];
    // staged region of a fused move (kdt_local.cuh)
    int lslot[LM];         // global slot of each staged triangle
    int4 lv[LM];           // its vertices and flags
    int4 ln[LM];           // its neighbour refs (global: slot << 2 | edge)
    int4 lnl[LM];          // the same neighbours as staged indices (-1: not staged)
    int2 lp[LM][3];        // coordinates of its three vertices
    int EO[KMAX];          // staged outer ref (index << 2 | edge) of each link edge
    // per-warp state every lane reads; only lane 0 writes it (then a warp barrier)
    unsigned cnt[C_NUM];   // event counters, flushed at the end of the kernel
    unsigned cyc_max;      // longest single move (cycles / 64)
    unsigned rng;          // xorshift state
    int ncl;               // claims held (cl[0 .. ncl-1])
    int rlo, rn;           // the points of the instance being worked on
    unsigned earbad;       // ears found invalid in the current clipping round
    int clbig;             // claims go to the warp's global scratch (a large star) instead of cl
};

__device__ __forceinline__ Star star_shared(WarpShared *sh)
{
    Star A;
    A.S = sh->S;
    A.I = sh->I;
    A.L = sh->L;
    A.ON = sh->ON;
    A.T = sh->tmp;
    A.LX = sh->LX;
    A.cap = KMAX;
    return A;
}

__device__ __forceinline__ Star star_big(int *b)
{
    Star A;
    A.S = b;
    A.I = b + KBIG;
    A.L = b + 2 * KBIG;
    A.ON = b + 3 * KBIG;
    A.T = b + 4 * KBIG;
    A.LX = reinterpret_cast<int2 *>(b + 5 * KBIG);
    A.cap = KBIG;
    return A;
}

// A warp's handle, passed by value: its shared block, its lane and its claim token.
// Everything mutable lives in the shared block, so no per-lane copy of warp state
// exists (each lane would otherwise hold an identical copy in local memory).
struct Warp {
    WarpShared *sh;
    int lane;
    int token;
};

__device__ __forceinline__ void cnt_add(const Warp w, int i, unsigned v)
{
    if (w.lane == 0) w.sh->cnt[i] += v;
}

// This warp's global scratch for stars above KMAX (only the kinetic launch has one;
// BIG_INTS ints per warp of the launch), or null.
__device__ __forceinline__ int *warp_big(const Dev &d)
{
    if (!d.big) return nullptr;
    size_t gw = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    return d.big + gw * BIG_INTS;
}

// The claim list in use and its capacity.
__device__ __forceinline__ int *claim_list_of(const Warp &w, const Dev &d)
{
    return w.sh->clbig ? warp_big(d) + 7 * KBIG : w.sh->cl;
}

__device__ __forceinline__ int claim_cap(const Warp &w) { return w.sh->clbig ? 2 * KBIG + 64 : MAXC; }

// next value of the warp's random state (uniform across the warp)
__device__ __forceinline__ unsigned warp_rand(const Warp w)
{
    unsigned s = w.sh->rng;
    s ^= s << 13;
    s ^= s >> 17;
    s ^= s << 5;
    __syncwarp();
    if (w.lane == 0) w.sh->rng = s;
    __syncwarp();
    return s;
}

// the instance whose points are [lo, lo + n) (walk restarts, of_instance)
__device__ __forceinline__ void set_instance(const Warp w, int lo, int n)
{
    __syncwarp();
    if (w.lane == 0) {
        w.sh->rlo = lo;
        w.sh->rn = n;
    }
    __syncwarp();
}

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ int4 bcast4(int4 v, int src)
{
    v.x = __shfl_sync(FULL, v.x, src);
    v.y = __shfl_sync(FULL, v.y, src);
    v.z = __shfl_sync(FULL, v.z, src);
    v.w = __shfl_sync(FULL, v.w, src);
    return v;
}

__device__ __forceinline__ int2 bcast2(int2 v, int src)
{
    v.x = __shfl_sync(FULL, v.x, src);
    v.y = __shfl_sync(FULL, v.y, src);
    return v;
}

__device__ __forceinline__ int comp(const int4 &v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }

__device__ __forceinline__ void set_status(const Dev &d, int code)
{
    atomicCAS(d.status, 0, code);
}

__device__ __forceinline__ int read_status(const Dev &d) { return __shfl_sync(FULL, __ldcg(d.status), 0); }

// Load tv[t] and tn[t] together (lanes 0 and 1) and broadcast.
// A slot outside the store (an unclaimed read can see the transient -1 neighbour of
// a triangle another warp is writing) reads as a dead triangle.
// Vertex id of the warp's current instance (or the ghost).
__device__ __forceinline__ bool of_instance(const Warp w, int id)
{
    return id == KDT_GHOST || (unsigned)(id - w.sh->rlo) < (unsigned)w.sh->rn;
}

__device__ __forceinline__ void load_tri(const Warp w, const Dev &d, int t, int4 &v, int4 &nb)
{
    int4 x = make_int4(0, 0, 0, 0);
    bool in = t >= 0 && t < d.cap;
    if (in && w.lane == 0) x = __ldcg(d.tv + t);
    else if (in && w.lane == 1) x = __ldcg(d.tn + t);
    v = bcast4(x, 0);
    nb = bcast4(x, 1);
}

// Coordinates of up to 4 vertices (ghost -> (0,0), never used) in one round trip.
__device__ __forceinline__ void load_xy4(const Warp w, const Dev &d, int a, int b, int c, int e,
                                         int2 &pa, int2 &pb, int2 &pc, int2 &pe)
{
    int id = w.lane == 0 ? a : (w.lane == 1 ? b : (w.lane == 2 ? c : (w.lane == 3 ? e : KDT_GHOST)));
    int2 x = make_int2(0, 0);
    if (id >= 0) x = __ldcg(d.xy + id);
    pa = bcast2(x, 0);
    pb = bcast2(x, 1);
    pc = bcast2(x, 2);
    pe = bcast2(x, 3);
}

__device__ __forceinline__ void backptr(const Dev &d, int ref, int val)
{
    reinterpret_cast<int *>(d.tn + (ref >> 2))[ref & 3] = val;
}

__device__ __forceinline__ void dirty_push(const Dev &d, int t)
{
    int pos = atomicAdd(d.dirty_count, 1);
    if (pos < d.dirty_cap) d.dirty[pos] = t;
}

__device__ __forceinline__ void backoff(Warp w, int attempt)
{
    unsigned lim = 32u << (attempt < 7 ? attempt : 7);  // up to ~4 us
    unsigned ns = 16 + (warp_rand(w) % lim);
    if (w.lane == 0) __nanosleep(ns);
    __syncwarp();
    cnt_add(w, C_RETRIES, 1);
}

__device__ __forceinline__ void flush_counters(Warp w, const Dev &d)
{
    if (w.lane == 0 && d.counters) {
        for (int i = 0; i < C_NUM; ++i)
            if (w.sh->cnt[i]) atomicAdd(d.counters + i, (unsigned long long)w.sh->cnt[i]);
        if (w.sh->cyc_max) atomicMax(d.counters + C_CYC_MAX, (unsigned long long)w.sh->cyc_max);
    }
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// a rare event, counted straight into the device slot
__device__ __forceinline__ void dev_count(const Warp w, const Dev &d, int i, unsigned long long v)
{
    if (w.lane == 0 && d.counters) atomicAdd(d.counters + i, v);
}

// ------------------------------------------------------------------ certification

// Is edge e of live triangle t locally Delaunay?  Also checks that the adjacency is
// reciprocal and the triangle counter-clockwise.  Returns 0 (fine), 1 (not locally
// Delaunay), -1 (store inconsistent).
__device__ int check_edge(const Dev &d, int t, const int4 &v, const int4 &nb, int e, unsigned *ex,
                          unsigned *ti)
{
    int ref = comp(nb, e);
    int U = ref >> 2, f = ref & 3;
    if (U < 0 || U >= d.cap || f > 2) return -1;
    int4 uv = __ldcg(d.tv + U);
    int4 un = __ldcg(d.tn + U);
    if (!(uv.w & ALIVE) || comp(un, f) != ((t << 2) | e)) return -1;
    int a = comp(v, (e + 1) % 3), b = comp(v, (e + 2) % 3);
    if (comp(uv, (f + 1) % 3) != b || comp(uv, (f + 2) % 3) != a) return -1;
    int dd = comp(uv, f);
    int2 z = make_int2(0, 0);
    int2 p0 = v.x >= 0 ? __ldcg(d.xy + v.x) : z;
    int2 p1 = v.y >= 0 ? __ldcg(d.xy + v.y) : z;
    int2 p2 = v.z >= 0 ? __ldcg(d.xy + v.z) : z;
    int2 pd = dd >= 0 ? __ldcg(d.xy + dd) : z;
    return conflict(v.x, v.y, v.z, p0, p1, p2, dd, pd, d.use_filter, ex, ti) ? 1 : 0;
}

// largest k in [0, cnt) with off[k] <= x (CSR offsets, off[cnt] = total)
__device__ __forceinline__ int csr_find(const int *off, int cnt, int x)
{
    int lo = 0, hi = cnt - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------ claims

// Claim tokens with this bit are "patient": the warp is on a move that must not keep
// losing (the star of a high-degree point, claimed whole).  A patient
// claim waits (bounded) for a slot another warp holds, unless the holder is patient
// too and has the smaller token; then it fails like any claim.  Other claims never
// wait while holding slots, and patient waits only go from a smaller to a larger
// token, so no cycle of waiting warps can form.
constexpr int TOK_PATIENT = 1 << 30;
constexpr int PATIENCE = 1 << 13;  // tries per slot (back-off up to ~1 us: < 10 ms)

// A patient claim of `slot` that found it held by `old`: wait for it (see above).
// Returns the last owner word seen (0 or token: claimed).
__device__ __noinline__ int claim_wait(const Dev &d, int slot, int token, int old)
{
    for (int it = 0; it < PATIENCE; ++it) {
        if ((old & TOK_PATIENT) && old < token) break;
        __nanosleep(32u << (it < 5 ? it : 5));
        old = atomicCAS(&d.tn[slot].w, 0, token);
        if (old == 0 || old == token) break;
    }
    return old;
}

// Try to claim the slots lane j holds in `mine` (j < m).  Returns true when every
// slot is now owned by this warp.  Newly taken slots are appended to the claim
// list either way; the caller releases everything on failure.
template <bool PATIENT = false>
__device__ __forceinline__ bool claim_lanes(Warp w, const Dev &d, int mine, int m)
{
    bool ok = true, added = false;
    if (w.lane < m && mine >= d.cap) ok = false;  // never a slot: fail the claim, touch nothing
    if (w.lane < m && mine >= 0 && mine < d.cap) {
        int old = atomicCAS(&d.tn[mine].w, 0, w.token);
        if (PATIENT && old != 0 && old != w.token) old = claim_wait(d, mine, w.token, old);
        ok = (old == 0) || (old == w.token);
        added = (old == 0);
    }
    unsigned am = __ballot_sync(FULL, added);
    unsigned om = __ballot_sync(FULL, ok);
    int held = w.sh->ncl;
    if (added) claim_list_of(w, d)[held + __popc(am & ((1u << w.lane) - 1))] = mine;
    __syncwarp();
    if (w.lane == 0) w.sh->ncl = held + __popc(am);
    __threadfence();
    __syncwarp();
    return om == FULL;
}

// Claim a list (any length; the caller keeps ncl + m <= the claim list's capacity).
template <bool PATIENT = false>
__device__ __forceinline__ bool claim_list(Warp w, const Dev &d, const int *list, int m)
{
    bool all = true;
    for (int base = 0; base < m; base += 32) {
        int j = base + w.lane;
        int mine = j < m ? list[j] : -1;
        all = claim_lanes<PATIENT>(w, d, mine, m - base < 32 ? m - base : 32) && all;
        if (!all) break;
    }
    return all;
}

// claim_list, patient when the warp's token says so (the global-memory deletions and
// in-place moves of a high-degree point's star, the insertions that finish a move on the
// global-memory path)
__device__ __forceinline__ bool claim_star_list(Warp w, const Dev &d, const int *list, int m)
{
    return (w.token & TOK_PATIENT) ? claim_list<true>(w, d, list, m) : claim_list<false>(w, d, list, m);
}

// claim_lanes, patient when the warp's token says so
__device__ __forceinline__ bool claim_lanes_tok(Warp w, const Dev &d, int mine, int m)
{
    return (w.token & TOK_PATIENT) ? claim_lanes<true>(w, d, mine, m) : claim_lanes<false>(w, d, mine, m);
}

__device__ __forceinline__ void release_all(Warp w, const Dev &d)
{
    __syncwarp();
    if (w.lane == 0) {
        __threadfence();  // our writes are visible before any owner word clears
        const int *cl = claim_list_of(w, d);
        for (int i = 0; i < w.sh->ncl; ++i) atomicExch(&d.tn[cl[i]].w, 0);
        w.sh->ncl = 0;
    }
    __syncwarp();
}

// release_all for a long claim list (a star gathered whole): all lanes clear words
__device__ __forceinline__ void release_star(Warp w, const Dev &d)
{
    __threadfence();  // every lane's writes are visible before any owner word clears
    __syncwarp();
    const int n = w.sh->ncl;
    const int *cl = claim_list_of(w, d);
    for (int i = w.lane; i < n; i += 32) atomicExch(&d.tn[cl[i]].w, 0);
    __syncwarp();
    if (w.lane == 0) w.sh->ncl = 0;
    __syncwarp();
}

// ------------------------------------------------------------------ walk

enum Where : int { W_INSIDE = 0, W_EDGE = 1, W_VERTEX = 2, W_GHOST = 3, W_FAIL = -1 };

// Visibility walk (exact orient2d) from slot `t` towards q.  Returns the slot where
// it stopped; `where` classifies q there, `e` is the edge for W_EDGE, `vtx` the
// coinciding vertex for W_VERTEX.  Reads are unclaimed; callers re-check after
// claiming.  A random start edge breaks ties so walks cannot cycle forever in the
// non-Delaunay states other warps may leave transiently.
struct WalkResult {
    int t;      // slot where the walk stopped, -1 when it gave up
    int where;  // Where
    int e;      // edge for W_EDGE
    int vtx;    // coinciding vertex for W_VERTEX
};

__device__ __noinline__ WalkResult walk(Warp w, const Dev &d, int t, int2 q)
{
    WalkResult res;
    res.t = -1;
    res.where = W_FAIL;
    res.e = 0;
    res.vtx = -1;
    for (int steps = 0; steps < WALK_CAP; ++steps) {
        cnt_add(w, C_WALK_STEPS, 1);
        if (t < 0 || t >= d.cap) return res;
        int4 v, nb;
        load_tri(w, d, t, v, nb);
        if (!(v.w & ALIVE)) return res;
        // The walk reads without claims: a triangle being written can pair its new
        // vertices with old neighbour words (zero in a fresh slot, i.e. slot 0).  In a
        // batch every instance covers the same coordinate domain, so such a reference
        // can lead into another instance's triangulation, where the geometry alone
        // would accept a location.  A triangle with a vertex outside the instance
        // ends the walk (the caller restarts).
        if (!of_instance(w, v.x) || !of_instance(w, v.y) || !of_instance(w, v.z)) return res;
        int2 p0, p1, p2, pz;
        load_xy4(w, d, v.x, v.y, v.z, KDT_GHOST, p0, p1, p2, pz);
        int g = v.x == KDT_GHOST ? 0 : (v.y == KDT_GHOST ? 1 : (v.z == KDT_GHOST ? 2 : -1));
        if (g >= 0) {
            int2 pu = g == 0 ? p1 : (g == 1 ? p2 : p0);
            int2 pv = g == 0 ? p2 : (g == 1 ? p0 : p1);
            if (orient2d(pu, pv, q) > 0) {
                res.where = W_GHOST;
                res.t = t;
                return res;
            }
            t = comp(nb, g) >> 2;  // across the finite edge
            continue;
        }
        int o0 = orient2d(p1, p2, q), o1 = orient2d(p2, p0, q), o2 = orient2d(p0, p1, q);
        // the edge tried first varies with the slot, the step count and the warp (a
        // hash, uniform across the warp), so walks cannot cycle
        unsigned h = (unsigned)t * 0x9E3779B1u ^ (unsigned)(steps + 1) * 0x85EBCA77u ^ (unsigned)w.token * 0xC2B2AE3Du;
        h ^= h >> 15;
        h *= 0x2C1B3C6Du;
        h ^= h >> 12;
        unsigned r = h % 3;
        int nxt = -1;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int i = (int)((r + k) % 3);
            int oi = i == 0 ? o0 : (i == 1 ? o1 : o2);
            if (oi < 0 && nxt < 0) nxt = i;
        }
        if (nxt >= 0) {
            t = comp(nb, nxt) >> 2;
            continue;
        }
        int zeros = (o0 == 0) + (o1 == 0) + (o2 == 0);
        if (zeros == 0) {
            res.where = W_INSIDE;
        } else if (zeros == 1) {
            res.where = W_EDGE;
            res.e = o0 == 0 ? 0 : (o1 == 0 ? 1 : 2);
        } else {
            res.where = W_VERTEX;
            // the vertex shared by the two zero edges
            res.vtx = o0 != 0 ? v.x : (o1 != 0 ? v.y : v.z);
        }
        res.t = t;
        return res;
    }
    return res;
}

// ------------------------------------------------------------------ writes

// Write the fan of m triangles (q, W[k], W[k+1]) into slots X[k]; O[k] is the
// outer reference across edge (W[k], W[k+1]).  Used by the 1->3 and 2->4 splits.
__device__ void write_fan(Warp w, const Dev &d, int q, const int *W, const int *O, const int *X, int m)
{
    if (w.lane == 0) {
        for (int k = 0; k < m; ++k) {
            int kn = (k + 1) % m, kp = (k + m - 1) % m;
            d.tv[X[k]] = make_int4(q, W[k], W[kn], ALIVE);
            d.tn[X[k]] = make_int4(O[k], (X[kn] << 2) | 2, (X[kp] << 2) | 1, w.token);
        }
        for (int k = 0; k < m; ++k) {
            backptr(d, O[k], (X[k] << 2) | 0);
            if (W[k] >= 0) d.pt_tri[W[k]] = X[k];
            dirty_push(d, X[k]);
        }
        d.pt_tri[q] = X[0];
    }
    __syncwarp();
}

// Flip the edge opposite vertex e of slot T (apex p).  U is the neighbour across it
// (its apex at index f is d).  Before:  T = (p, a, b),  U = (b, a, d).
// After:  T = (p, a, d),  U = (p, d, b).  All four outer back-pointers are rewritten.
__device__ void do_flip(Warp w, const Dev &d, int T, int e, const int4 &tv_, const int4 &tn_, int U,
                        int f, const int4 &uv, const int4 &un)
{
    if (w.lane == 0) {
        int p = comp(tv_, e), a = comp(tv_, (e + 1) % 3), b = comp(tv_, (e + 2) % 3);
        int dd = comp(uv, f);
        int nt_a = comp(tn_, (e + 1) % 3), nt_b = comp(tn_, (e + 2) % 3);
        int nu_b = comp(un, (f + 1) % 3), nu_a = comp(un, (f + 2) % 3);
        d.tv[T] = make_int4(p, a, dd, ALIVE);
        d.tn[T] = make_int4(nu_b, (U << 2) | 2, nt_b, w.token);
        d.tv[U] = make_int4(p, dd, b, ALIVE);
        d.tn[U] = make_int4(nu_a, nt_a, (T << 2) | 1, w.token);
        backptr(d, nu_b, (T << 2) | 0);
        backptr(d, nt_b, (T << 2) | 2);
        backptr(d, nu_a, (U << 2) | 0);
        backptr(d, nt_a, (U << 2) | 1);
        if (p >= 0) d.pt_tri[p] = T;
        if (a >= 0) d.pt_tri[a] = T;
        if (dd >= 0) d.pt_tri[dd] = T;
        if (b >= 0) d.pt_tri[b] = U;
        dirty_push(d, T);
        dirty_push(d, U);
    }
    __syncwarp();
}

// ------------------------------------------------------------------ Lawson flips

// Process the flip stack.  insertion_mode: only entries whose apex is still `p` are
// valid and a flip pushes the two edges opposite p (Lawson after an insertion);
// otherwise (general repair) any apex is accepted and the four outer edges are
// pushed.  Tests are made on unclaimed reads; only an indicated flip is claimed and
// re-checked.  An edge that cannot be settled here is left to the certification
// pass that follows every step, so correctness never depends on this stack.
__device__ __noinline__ int lawson(Warp w, const Dev &d, int top, int p, bool insertion_mode)
{
    WarpShared *sh = w.sh;
    int attempts = 0;
    while (top > 0) {
        if (read_status(d)) return top;
        int2 ent = sh->stack[top - 1];
        __syncwarp();
        --top;
        int T = ent.x, e = ent.y;
        int4 v, nb;
        load_tri(w, d, T, v, nb);
        if (!(v.w & ALIVE)) continue;
        int apex = comp(v, e);
        if (insertion_mode && apex != p) continue;
        int ref = comp(nb, e);
        int U = ref >> 2, f = ref & 3;
        int4 uv, un;
        load_tri(w, d, U, uv, un);
        if (!(uv.w & ALIVE)) continue;
        int a = comp(v, (e + 1) % 3), b = comp(v, (e + 2) % 3), dd = comp(uv, f);
        if (comp(uv, (f + 1) % 3) != b || comp(uv, (f + 2) % 3) != a) continue;  // stale read
        int2 pp, pa, pb, pd;
        load_xy4(w, d, apex, a, b, dd, pp, pa, pb, pd);
        cnt_add(w, C_FLIP_TESTS, 1);
        // coordinates in the triangle's stored rotation (apex at index e)
        int2 pv0 = e == 0 ? pp : (e == 1 ? pb : pa);
        int2 pv1 = e == 1 ? pp : (e == 2 ? pb : pa);
        int2 pv2 = e == 2 ? pp : (e == 0 ? pb : pa);
        unsigned ex = 0, ti = 0;
        bool cf = conflict(v.x, v.y, v.z, pv0, pv1, pv2, dd, pd, d.use_filter, &ex, &ti);
        cnt_add(w, C_EXACT, ex);
        cnt_add(w, C_TIES, ti);
        if (!cf) continue;
        // claim the quad and its four outer neighbours, then re-check
        int mine = -1;
        if (w.lane == 0) mine = T;
        else if (w.lane == 1) mine = U;
        else if (w.lane == 2) mine = comp(nb, (e + 1) % 3) >> 2;
        else if (w.lane == 3) mine = comp(nb, (e + 2) % 3) >> 2;
        else if (w.lane == 4) mine = comp(un, (f + 1) % 3) >> 2;
        else if (w.lane == 5) mine = comp(un, (f + 2) % 3) >> 2;
        bool ok = claim_lanes_tok(w, d, mine, 6);
        if (ok) {
            int4 v2, nb2, uv2, un2;
            load_tri(w, d, T, v2, nb2);
            load_tri(w, d, U, uv2, un2);
            ok = v2.x == v.x && v2.y == v.y && v2.z == v.z && (v2.w & ALIVE) && nb2.x == nb.x &&
                 nb2.y == nb.y && nb2.z == nb.z && uv2.x == uv.x && uv2.y == uv.y && uv2.z == uv.z &&
                 (uv2.w & ALIVE) && un2.x == un.x && un2.y == un.y && un2.z == un.z;
            if (ok) {
                do_flip(w, d, T, e, v2, nb2, U, f, uv2, un2);
                cnt_add(w, insertion_mode ? C_FLIPS : C_FIX_FLIPS, 1);
                release_all(w, d);
                // push follow-up edges
                int add = insertion_mode ? 2 : 4;
                if (top + add > STACK) {
                    cnt_add(w, C_STACK_DROP, 1);
                    continue;
                }
                if (w.lane == 0) {
                    sh->stack[top] = make_int2(T, 0);
                    sh->stack[top + 1] = make_int2(U, 0);
                    if (!insertion_mode) {
                        sh->stack[top + 2] = make_int2(T, 2);
                        sh->stack[top + 3] = make_int2(U, 1);
                    }
                }
                __syncwarp();
                top += add;
                attempts = 0;
                continue;
            }
        }
        release_all(w, d);
        // contention or a stale read: retry this edge later
        if (++attempts > d.retry_cap) {
            cnt_add(w, C_STACK_DROP, 1);
            attempts = 0;
            continue;
        }
        backoff(w, attempts);
        if (w.lane == 0) sh->stack[top] = ent;
        __syncwarp();
        ++top;
    }
    return 0;
}

// ------------------------------------------------------------------ insertion

// Insertion outside the hull (Section IV insertion; the ghost part of the Bowyer-
// Watson cavity).  The hull edges visible from q form one chain x_0 -> ... -> x_k;
// its ghosts, the finite triangles behind them, the two ghosts at its ends and the
// two spare slots are claimed together, and the chain is replaced in one fan
// (q, x_k, x_{k-1}), ..., (q, x_1, x_0), (q, x_0, inf), (q, inf, x_k).  Doing it in
// one claimed operation keeps the hull convex whenever nothing is claimed, so no
// other warp can ever mistake a pocket of a half-repaired hull for the outside.
// Returns 0 when written, 1 to retry (contention or stale reads), or an error.
__device__ __noinline__ int insert_outside(Warp w, const Dev &d, int p, int2 q, int V0, int spare0, int spare1, int &m_out)
{
    WarpShared *sh = w.sh;
    const int KCH = 60;
    // ghost (u, v, inf) at slot t: g = index of inf, u = v[g+1], v = v[g+2]; hull edge v -> u.
    // backward neighbour (hull edge ending at v): edge index g+1; forward (from u): g+2.
    int cur = V0, eb_ref = -1;
    for (int s = 0;; ++s) {
        if (s > KCH) return 1;  // a transient loop, or a chain longer than KCH (retry budget decides)
        int4 v, nb;
        load_tri(w, d, cur, v, nb);
        int g = v.x == KDT_GHOST ? 0 : (v.y == KDT_GHOST ? 1 : (v.z == KDT_GHOST ? 2 : -1));
        if (!(v.w & ALIVE) || g < 0) return 1;
        int br = comp(nb, (g + 1) % 3);
        int4 bv, bn;
        load_tri(w, d, br >> 2, bv, bn);
        int bg = bv.x == KDT_GHOST ? 0 : (bv.y == KDT_GHOST ? 1 : (bv.z == KDT_GHOST ? 2 : -1));
        if (!(bv.w & ALIVE) || bg < 0) return 1;
        int2 pu, pv, pz, pz2;
        load_xy4(w, d, comp(bv, (bg + 1) % 3), comp(bv, (bg + 2) % 3), KDT_GHOST, KDT_GHOST, pu, pv, pz, pz2);
        if (orient2d(pu, pv, q) <= 0) {
            eb_ref = br;
            break;
        }
        cur = br >> 2;
    }
    // forward from the first visible ghost, recording the chain in ccw order
    int k = 0, ef_ref = -1;
    while (true) {
        if (k >= KCH) return 1;
        int4 v, nb;
        load_tri(w, d, cur, v, nb);
        int g = v.x == KDT_GHOST ? 0 : (v.y == KDT_GHOST ? 1 : (v.z == KDT_GHOST ? 2 : -1));
        if (!(v.w & ALIVE) || g < 0) return 1;
        if (w.lane == 0) {
            sh->S[k] = cur;
            sh->L[k] = comp(v, (g + 2) % 3);      // x_k = v (start of the hull edge)
            sh->L[k + 1] = comp(v, (g + 1) % 3);  // x_{k+1} = u
            sh->ON[k] = comp(nb, g);              // finite triangle behind the hull edge
            sh->I[k] = comp(nb, (g + 2) % 3);     // forward ref
        }
        __syncwarp();
        ++k;
        int fr = comp(nb, (g + 2) % 3);
        int4 fv, fn;
        load_tri(w, d, fr >> 2, fv, fn);
        int fg = fv.x == KDT_GHOST ? 0 : (fv.y == KDT_GHOST ? 1 : (fv.z == KDT_GHOST ? 2 : -1));
        if (!(fv.w & ALIVE) || fg < 0) return 1;
        int2 pu, pv, pz, pz2;
        load_xy4(w, d, comp(fv, (fg + 1) % 3), comp(fv, (fg + 2) % 3), KDT_GHOST, KDT_GHOST, pu, pv, pz, pz2);
        if (orient2d(pu, pv, q) <= 0) {
            ef_ref = fr;
            break;
        }
        cur = fr >> 2;
        if (cur == sh->S[0]) return 1;  // wrapped around: stale reads
    }
    // claim: chain ghosts, finite triangles behind them, end ghosts, spares
    int *cand = reinterpret_cast<int *>(sh->LX);
    if (w.lane == 0) {
        for (int j = 0; j < k; ++j) {
            cand[2 * j] = sh->S[j];
            cand[2 * j + 1] = sh->ON[j] >> 2;
        }
        cand[2 * k] = eb_ref >> 2;
        cand[2 * k + 1] = ef_ref >> 2;
        cand[2 * k + 2] = spare0;
        cand[2 * k + 3] = spare1;
    }
    __syncwarp();
    bool ok = claim_star_list(w, d, cand, 2 * k + 4);
    if (ok) {
        // re-check the chain under the claims
        bool good = true;
        for (int j = w.lane; j < k; j += 32) {
            int4 v = __ldcg(d.tv + sh->S[j]);
            int4 nb = __ldcg(d.tn + sh->S[j]);
            int g = v.x == KDT_GHOST ? 0 : (v.y == KDT_GHOST ? 1 : (v.z == KDT_GHOST ? 2 : -1));
            good = good && (v.w & ALIVE) && g >= 0 && comp(v, (g + 2) % 3) == sh->L[j] &&
                   comp(v, (g + 1) % 3) == sh->L[j + 1] && comp(nb, g) == sh->ON[j] &&
                   comp(nb, (g + 2) % 3) == sh->I[j] &&
                   (j + 1 == k ? comp(nb, (g + 2) % 3) == ef_ref : (comp(nb, (g + 2) % 3) >> 2) == sh->S[j + 1]) &&
                   (j == 0 ? comp(nb, (g + 1) % 3) == eb_ref : true);
            if (good) {
                int2 pu = __ldcg(d.xy + sh->L[j + 1]), pv = __ldcg(d.xy + sh->L[j]);
                good = orient2d(pu, pv, q) > 0;
            }
        }
        if (w.lane < 2) {
            int ref = w.lane == 0 ? eb_ref : ef_ref;
            int4 v = __ldcg(d.tv + (ref >> 2));
            int g = v.x == KDT_GHOST ? 0 : (v.y == KDT_GHOST ? 1 : (v.z == KDT_GHOST ? 2 : -1));
            good = good && (v.w & ALIVE) && g >= 0;
            if (good) {
                int2 pu = __ldcg(d.xy + comp(v, (g + 1) % 3)), pv = __ldcg(d.xy + comp(v, (g + 2) % 3));
                good = orient2d(pu, pv, q) <= 0;
            }
        }
        ok = __all_sync(FULL, good);
    }
    if (!ok) {
        release_all(w, d);
        return 1;
    }
    // fan: W = (x_k, ..., x_0, inf) in tmp, outer refs (F_{k-1}, ..., F_0, E_b, E_f) in I
    // (the forward refs are no longer needed), slots = the chain's own slots + spares in S
    int m = k + 2;
    int *W = sh->tmp, *Ow = sh->I, *Xw = sh->S;
    if (w.lane == 0) {
        for (int j = 0; j < k; ++j) W[j] = sh->L[k - j];
        W[k] = sh->L[0];
        W[k + 1] = KDT_GHOST;
        for (int j = 0; j < k; ++j) Ow[j] = sh->ON[k - 1 - j];
        Ow[k] = eb_ref;
        Ow[k + 1] = ef_ref;
        Xw[k] = spare0;
        Xw[k + 1] = spare1;
    }
    __syncwarp();
    write_fan(w, d, p, W, Ow, Xw, m);
    cnt_add(w, C_SPLIT_GHOST, 1);
    cnt_add(w, C_INSERTS, 1);
    release_all(w, d);
    m_out = m;
    return 0;
}

// Insert point p (its coordinates already in xy[p]) starting the walk at `start`.
// spare0 / spare1 are two dead slots owned by the caller (a deletion's leftovers or
// fresh slots during a build).  Returns 0, INS_DEFER (p lands on a vertex that is
// still moving in this step), or a DevStatus error.
__device__ __noinline__ int insert_point(Warp w, const Dev &d, int p, int2 q, int start, int spare0, int spare1,
                            bool allow_defer)
{
    WarpShared *sh = w.sh;
    if (spare0 < 0 || spare0 >= d.cap || spare1 < 0 || spare1 >= d.cap) return DEV_INTERNAL;
    int t = start, walk_fail = 0;
    for (int attempt = 0;; ++attempt) {
        if (attempt > d.retry_cap) return DEV_RETRY;
        if (read_status(d)) return -1;
        WalkResult wr = walk(w, d, t, q);
        int tt = wr.t, where = wr.where, e = wr.e, vtx = wr.vtx;
        if (tt < 0) {
            if (++walk_fail > WALK_RESTARTS) return DEV_WALK;
            // restart from the hint, then from the triangle of a random present point
            if (attempt & 1) {
                t = start;
            } else {
                int r = w.sh->rlo + (int)(warp_rand(w) % (unsigned)w.sh->rn);
                t = __shfl_sync(FULL, __ldcg(d.pt_tri + r), 0);
                if (t < 0) t = start;
            }
            backoff(w, attempt);
            continue;
        }
        if (where == W_VERTEX) {
            int st = __shfl_sync(FULL, __ldcg(d.pt_stamp + vtx), 0);
            if (allow_defer && st == d.stamp) return INS_DEFER;
            return DEV_DUPLICATE;
        }
        if (where == W_GHOST) {
            int m = 0;
            int r = insert_outside(w, d, p, q, tt, spare0, spare1, m);
            if (r == 1) {
                t = tt;
                backoff(w, attempt);
                continue;
            }
            if (r) return r;
            if (w.lane == 0)
                for (int j = 0; j < m; ++j) sh->stack[j] = make_int2(sh->S[j], 0);
            __syncwarp();
            lawson(w, d, m, p, true);
            return DEV_OK;
        }
        int4 v, nb;
        load_tri(w, d, tt, v, nb);
        int U = -1, f = 0;
        int4 uv = make_int4(0, 0, 0, 0), un = make_int4(0, 0, 0, 0);
        if (where == W_EDGE) {
            U = comp(nb, e) >> 2;
            f = comp(nb, e) & 3;
            load_tri(w, d, U, uv, un);
        }
        // claim: the triangle(s) split, their outer neighbours, the spare slots
        int mine = -1;
        switch (w.lane) {
        case 0: mine = tt; break;
        case 1: mine = spare0; break;
        case 2: mine = spare1; break;
        case 3: mine = where == W_EDGE ? comp(nb, (e + 1) % 3) >> 2 : nb.x >> 2; break;
        case 4: mine = where == W_EDGE ? comp(nb, (e + 2) % 3) >> 2 : nb.y >> 2; break;
        case 5: mine = where == W_EDGE ? U : nb.z >> 2; break;
        case 6: mine = where == W_EDGE ? comp(un, (f + 1) % 3) >> 2 : -1; break;
        case 7: mine = where == W_EDGE ? comp(un, (f + 2) % 3) >> 2 : -1; break;
        default: break;
        }
        bool ok = claim_lanes_tok(w, d, mine, 8);
        if (ok) {
            // re-read under the claims and re-classify
            int4 v2, nb2;
            load_tri(w, d, tt, v2, nb2);
            ok = (v2.w & ALIVE) && v2.x == v.x && v2.y == v.y && v2.z == v.z && nb2.x == nb.x &&
                 nb2.y == nb.y && nb2.z == nb.z;
            if (ok && where == W_EDGE) {
                int4 uv2, un2;
                load_tri(w, d, U, uv2, un2);
                ok = (uv2.w & ALIVE) && uv2.x == uv.x && uv2.y == uv.y && uv2.z == uv.z &&
                     un2.x == un.x && un2.y == un.y && un2.z == un.z;
            }
            if (ok) {
                int2 p0, p1, p2, pz;
                load_xy4(w, d, v.x, v.y, v.z, KDT_GHOST, p0, p1, p2, pz);
                int g = v.x == KDT_GHOST ? 0 : (v.y == KDT_GHOST ? 1 : (v.z == KDT_GHOST ? 2 : -1));
                if (g >= 0) {
                    int2 pu = g == 0 ? p1 : (g == 1 ? p2 : p0);
                    int2 pv = g == 0 ? p2 : (g == 1 ? p0 : p1);
                    ok = where == W_GHOST && orient2d(pu, pv, q) > 0;
                } else {
                    int o0 = orient2d(p1, p2, q), o1 = orient2d(p2, p0, q), o2 = orient2d(p0, p1, q);
                    int zeros = (o0 == 0) + (o1 == 0) + (o2 == 0);
                    ok = o0 >= 0 && o1 >= 0 && o2 >= 0 &&
                         ((where == W_INSIDE && zeros == 0) ||
                          (where == W_EDGE && zeros == 1 && comp(make_int4(o0, o1, o2, 0), e) == 0));
                }
            }
        }
        if (!ok) {
            release_all(w, d);
            t = tt;
            backoff(w, attempt);
            continue;
        }
        // split
        int *W = sh->tmp, *O = sh->tmp + 8, *X = sh->tmp + 16;
        int m;
        if (w.lane == 0) {
            if (where == W_EDGE) {
                int a = comp(v, e), b = comp(v, (e + 1) % 3), c = comp(v, (e + 2) % 3);
                int dd = comp(uv, f);
                W[0] = a; W[1] = b; W[2] = dd; W[3] = c;
                O[0] = comp(nb, (e + 2) % 3);   // (a, b)
                O[1] = comp(un, (f + 1) % 3);   // (b, d): u = (d, c, b), edge opposite c
                O[2] = comp(un, (f + 2) % 3);   // (d, c): edge opposite b
                O[3] = comp(nb, (e + 1) % 3);   // (c, a)
                X[0] = tt; X[1] = U; X[2] = spare0; X[3] = spare1;
            } else {
                W[0] = v.x; W[1] = v.y; W[2] = v.z;
                O[0] = nb.z; O[1] = nb.x; O[2] = nb.y;
                X[0] = tt; X[1] = spare0; X[2] = spare1;
            }
        }
        m = where == W_EDGE ? 4 : 3;
        __syncwarp();
        write_fan(w, d, p, W, O, X, m);
        if (where == W_EDGE) cnt_add(w, C_SPLIT_EDGE, 1);
        if (where == W_GHOST) cnt_add(w, C_SPLIT_GHOST, 1);
        cnt_add(w, C_INSERTS, 1);
        release_all(w, d);
        if (w.lane == 0)
            for (int k = 0; k < m; ++k) sh->stack[k] = make_int2(X[k], 0);
        __syncwarp();
        lawson(w, d, m, p, true);
        return DEV_OK;
    }
}

// ------------------------------------------------------------------ deletion

// Gather the star of p counter-clockwise from pt_tri[p] into A (S/I/L/ON).  Returns k,
// or -1 when the reads are inconsistent (another warp is working there), -2 when
// the degree exceeds A.cap.  The star is walked in both directions at once (the
// next triangle counter-clockwise and the next clockwise are loaded in the same
// round trip), so a star of k triangles costs about k/2 dependent loads.  The
// clockwise part is kept at the top of the arrays and moved into place at the end.
__device__ __noinline__ int gather_star(Warp w, const Dev &d, int p, Star A)
{
    const int cap = A.cap;
    int t0 = __ldcg(d.pt_tri + p);
    t0 = __shfl_sync(FULL, t0, 0);
    if (t0 < 0 || t0 >= d.cap) return -1;
    int nf = 0, nbk = 0;   // entries counter-clockwise after t0, clockwise before it
    int tf = t0, tb = -1;  // triangles to load this round (-1: none)
    while (true) {
        // lanes 0, 1: tf (vertices, neighbours); lanes 2, 3: tb
        int4 x = make_int4(0, 0, 0, 0);
        int tl = w.lane < 2 ? tf : (w.lane < 4 ? tb : -1);
        if (tl >= 0 && tl < d.cap) x = (w.lane & 1) ? __ldcg(d.tn + tl) : __ldcg(d.tv + tl);
        int4 fv = bcast4(x, 0), fn = bcast4(x, 1), bv = bcast4(x, 2), bn = bcast4(x, 3);
        // forward triangle (t0 itself in the first round)
        if (!(fv.w & ALIVE)) return -1;
        int If = fv.x == p ? 0 : (fv.y == p ? 1 : (fv.z == p ? 2 : -1));
        if (If < 0) return -1;
        if (nf + nbk + 1 > cap) return -2;
        if (w.lane == 0) {
            A.S[nf] = tf;
            A.I[nf] = If;
            A.L[nf] = comp(fv, (If + 1) % 3);
            A.ON[nf] = comp(fn, If);
        }
        ++nf;
        int fnext = comp(fn, (If + 1) % 3) >> 2;
        if (tb < 0) {
            // first round: t0; its clockwise neighbour starts the other direction
            int fprev = comp(fn, (If + 2) % 3) >> 2;
            if (fnext == t0) break;  // a star of one triangle (never valid: rejected by k < 3)
            if (fnext < 0 || fnext >= d.cap || fprev < 0 || fprev >= d.cap) return -1;
            if (fnext == fprev) {    // two triangles
                tf = fnext;
                int4 y = make_int4(0, 0, 0, 0);
                if (w.lane < 2) y = (w.lane & 1) ? __ldcg(d.tn + tf) : __ldcg(d.tv + tf);
                int4 v2 = bcast4(y, 0), n2 = bcast4(y, 1);
                if (!(v2.w & ALIVE)) return -1;
                int I2 = v2.x == p ? 0 : (v2.y == p ? 1 : (v2.z == p ? 2 : -1));
                if (I2 < 0) return -1;
                if (w.lane == 0) {
                    A.S[nf] = tf;
                    A.I[nf] = I2;
                    A.L[nf] = comp(v2, (I2 + 1) % 3);
                    A.ON[nf] = comp(n2, I2);
                }
                ++nf;
                break;
            }
            tf = fnext;
            tb = fprev;
            continue;
        }
        // backward triangle
        if (tb == tf) break;  // both directions reached the same triangle: stored once
        if (!(bv.w & ALIVE)) return -1;
        int Ib = bv.x == p ? 0 : (bv.y == p ? 1 : (bv.z == p ? 2 : -1));
        if (Ib < 0) return -1;
        if (nf + nbk + 1 > cap) return -2;
        if (w.lane == 0) {
            int at = cap - 1 - nbk;
            A.S[at] = tb;
            A.I[at] = Ib;
            A.L[at] = comp(bv, (Ib + 1) % 3);
            A.ON[at] = comp(bn, Ib);
        }
        ++nbk;
        int bprev = comp(bn, (Ib + 2) % 3) >> 2;
        if (fnext == tb) break;  // the forward direction continues into the backward part
        if (bprev == tf) break;  // (the same meeting seen from the other side)
        if (fnext < 0 || fnext >= d.cap || bprev < 0 || bprev >= d.cap) return -1;
        if (fnext == bprev) {
            // one triangle left between them: load it forward in the next round
            tf = fnext;
            tb = fnext;
            continue;
        }
        tf = fnext;
        tb = bprev;
    }
    __syncwarp();
    // move the clockwise part (top of the arrays, last found first) after the rest, in
    // chunks of 32 in increasing order (a destination never lies above its source)
    for (int c0 = 0; c0 < nbk; c0 += 32) {
        int i = c0 + w.lane;
        int src = cap - nbk + i;
        bool mv = i < nbk;
        int cS = 0, cI = 0, cL = 0, cO = 0;
        if (mv) {
            cS = A.S[src];
            cI = A.I[src];
            cL = A.L[src];
            cO = A.ON[src];
        }
        __syncwarp();
        if (mv) {
            A.S[nf + i] = cS;
            A.I[nf + i] = cI;
            A.L[nf + i] = cL;
            A.ON[nf + i] = cO;
        }
        __syncwarp();
    }
    return nf + nbk;
}

// The same walk with the star in the warp's shared block (degree <= KMAX), written with
// direct shared-memory accesses: this is the hot path of every staged move.
__device__ __forceinline__ int gather_star(Warp w, const Dev &d, int p)
{
    WarpShared *sh = w.sh;
    int t0 = __ldcg(d.pt_tri + p);
    t0 = __shfl_sync(FULL, t0, 0);
    if (t0 < 0 || t0 >= d.cap) return -1;
    int nf = 0, nbk = 0;
    int tf = t0, tb = -1;
    while (true) {
        int4 x = make_int4(0, 0, 0, 0);
        int tl = w.lane < 2 ? tf : (w.lane < 4 ? tb : -1);
        if (tl >= 0 && tl < d.cap) x = (w.lane & 1) ? __ldcg(d.tn + tl) : __ldcg(d.tv + tl);
        int4 fv = bcast4(x, 0), fn = bcast4(x, 1), bv = bcast4(x, 2), bn = bcast4(x, 3);
        if (!(fv.w & ALIVE)) return -1;
        int If = fv.x == p ? 0 : (fv.y == p ? 1 : (fv.z == p ? 2 : -1));
        if (If < 0) return -1;
        if (nf + nbk + 1 > KMAX) return -2;
        if (w.lane == 0) {
            sh->S[nf] = tf;
            sh->I[nf] = If;
            sh->L[nf] = comp(fv, (If + 1) % 3);
            sh->ON[nf] = comp(fn, If);
        }
        ++nf;
        int fnext = comp(fn, (If + 1) % 3) >> 2;
        if (tb < 0) {
            int fprev = comp(fn, (If + 2) % 3) >> 2;
            if (fnext == t0) break;
            if (fnext < 0 || fnext >= d.cap || fprev < 0 || fprev >= d.cap) return -1;
            if (fnext == fprev) {
                tf = fnext;
                int4 y = make_int4(0, 0, 0, 0);
                if (w.lane < 2) y = (w.lane & 1) ? __ldcg(d.tn + tf) : __ldcg(d.tv + tf);
                int4 v2 = bcast4(y, 0), n2 = bcast4(y, 1);
                if (!(v2.w & ALIVE)) return -1;
                int I2 = v2.x == p ? 0 : (v2.y == p ? 1 : (v2.z == p ? 2 : -1));
                if (I2 < 0) return -1;
                if (w.lane == 0) {
                    sh->S[nf] = tf;
                    sh->I[nf] = I2;
                    sh->L[nf] = comp(v2, (I2 + 1) % 3);
                    sh->ON[nf] = comp(n2, I2);
                }
                ++nf;
                break;
            }
            tf = fnext;
            tb = fprev;
            continue;
        }
        if (tb == tf) break;
        if (!(bv.w & ALIVE)) return -1;
        int Ib = bv.x == p ? 0 : (bv.y == p ? 1 : (bv.z == p ? 2 : -1));
        if (Ib < 0) return -1;
        if (nf + nbk + 1 > KMAX) return -2;
        if (w.lane == 0) {
            int at = KMAX - 1 - nbk;
            sh->S[at] = tb;
            sh->I[at] = Ib;
            sh->L[at] = comp(bv, (Ib + 1) % 3);
            sh->ON[at] = comp(bn, Ib);
        }
        ++nbk;
        int bprev = comp(bn, (Ib + 2) % 3) >> 2;
        if (fnext == tb) break;
        if (bprev == tf) break;
        if (fnext < 0 || fnext >= d.cap || bprev < 0 || bprev >= d.cap) return -1;
        if (fnext == bprev) {
            tf = fnext;
            tb = fnext;
            continue;
        }
        tf = fnext;
        tb = bprev;
    }
    __syncwarp();
    // move the clockwise part (at most KMAX/2 = 32 entries: one lane each) after the rest
    int k = nf + nbk;
    int src = KMAX - nbk + w.lane;
    int cS = 0, cI = 0, cL = 0, cO = 0;
    bool mv = w.lane < nbk;
    if (mv) {
        cS = sh->S[src];
        cI = sh->I[src];
        cL = sh->L[src];
        cO = sh->ON[src];
    }
    __syncwarp();
    if (mv) {
        sh->S[nf + w.lane] = cS;
        sh->I[nf + w.lane] = cI;
        sh->L[nf + w.lane] = cL;
        sh->ON[nf + w.lane] = cO;
    }
    __syncwarp();
    return k;
}

// A word another lane of the warp may have updated (shared or global memory)
__device__ __forceinline__ int vload(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

// Bit i of a bit set spread over the warp (lane c holds bits 32c .. 32c+31); every
// lane must take part.
__device__ __forceinline__ bool bit_of(unsigned words, int i)
{
    return (__shfl_sync(FULL, words, i >> 5) >> (i & 31)) & 1u;
}

// One test of ear i (L[i], L[i+1], L[i+2]) of the current link polygon of m vertices:
// t = 0 fails a finite ear that is not counter-clockwise; t >= 1 fails it when
// vertex i+2+t conflicts with it (the conditions ear_valid checks, one per call).
__device__ __forceinline__ bool ear_test_fails(const int *EL, const int2 *EX, int m, int i, int t, const Dev &d,
                                               unsigned *exact_calls, unsigned *ties)
{
    int i1 = i + 1 == m ? 0 : i + 1, i2 = i1 + 1 == m ? 0 : i1 + 1;
    int x = EL[i], y = EL[i1], z = EL[i2];
    int2 px = EX[i], py = EX[i1], pz = EX[i2];
    int g = x == KDT_GHOST ? 0 : (y == KDT_GHOST ? 1 : (z == KDT_GHOST ? 2 : -1));
    if (t == 0) return g < 0 && orient2d(px, py, pz) <= 0;
    int j = i + 2 + t;
    if (j >= m) j -= m;
    int wv = EL[j];
    if (wv == KDT_GHOST) return false;
    if (g >= 0) {
        int2 gu = g == 0 ? py : (g == 1 ? pz : px);
        int2 gv = g == 0 ? pz : (g == 1 ? px : py);
        return ghost_conflict(gu, gv, EX[j]);
    }
    return incircle_sos(x, y, z, wv, px, py, pz, EX[j], d.use_filter, exact_calls, ties) > 0;
}

// Delete p on the global-memory path: claim its star and the ring of outer
// neighbours, re-triangulate the star-shaped hole by Delaunay ears (the simple
// deletion the paper prefers, Section IV) written straight to the store, release.
// The star lives in A: the warp's shared block, or its global scratch for a degree
// above KMAX (the claims then go to the scratch's claim list).  Each round tests every
// (ear, remaining vertex) pair on its own lane and clips all valid, pairwise
// non-adjacent ears.  On success the two slots the hole no longer needs are returned
// dead in spare0/spare1 and `hint` is a new triangle next to p's old position.
__device__ __noinline__ int delete_point_in(Warp w, const Dev &d, int p, int &spare0, int &spare1, int &hint,
                                            Star A, bool may_give_up)
{
    int busy = 0;
    for (int attempt = 0;; ++attempt) {
        if (attempt > d.retry_cap) return DEV_RETRY;
        if (read_status(d)) return -1;
        // an unclaimed walk around p can run round a transient loop while another warp
        // is writing p's triangles: treat every failed gather as contention, and report
        // a real degree overflow only when it persists for the whole retry budget
        int k = gather_star(w, d, p, A);
        // a degree above the shared arrays (it can grow after the caller looked): the
        // warp's global scratch takes it, if the launch has one
        if (k == -2 && A.cap < KBIG && d.big) return DEL_HUGE;
        if (k == -2 && attempt == d.retry_cap) return DEV_DEGREE;
        if (k < 3) {
            backoff(w, attempt);
            continue;
        }
        // claim the star and the outer ring
        for (int i = w.lane; i < k; i += 32) A.T[i] = A.ON[i] >> 2;
        __syncwarp();
        bool ok = claim_star_list(w, d, A.S, k);
        if (ok) ok = claim_star_list(w, d, A.T, k);
        if (ok) {
            // validate the gathered star under the claims (one parallel pass)
            bool good = true;
            for (int i = w.lane; i < k; i += 32) {
                int4 v = __ldcg(d.tv + A.S[i]);
                int4 nb = __ldcg(d.tn + A.S[i]);
                int I = A.I[i];
                good = good && (v.w & ALIVE) && comp(v, I) == p && comp(v, (I + 1) % 3) == A.L[i] &&
                       comp(nb, I) == A.ON[i] && (comp(nb, (I + 1) % 3) >> 2) == A.S[i + 1 == k ? 0 : i + 1];
            }
            ok = __all_sync(FULL, good);
        }
        if (!ok) {
            release_star(w, d);
            if (may_give_up && ++busy >= DEFER_AFTER) return DEL_BUSY;
            backoff(w, attempt);
            continue;
        }
        // link coordinates
        for (int i = w.lane; i < k; i += 32) {
            int lv = A.L[i];
            A.LX[i] = lv >= 0 ? __ldcg(d.xy + lv) : make_int2(0, 0);
        }
        __syncwarp();
        // degenerate check: a hull vertex whose finite link is collinear and whose
        // ring has no finite triangle would leave only collinear points behind
        int gpos = -1;
        for (int i = 0; i < k; ++i)
            if (A.L[i] == KDT_GHOST) gpos = i;
        if (gpos >= 0) {
            int f0 = (gpos + 1) % k, f1 = (gpos + 2) % k;
            bool col = true;
            for (int i = w.lane; i < k; i += 32)
                if (i != gpos && orient2d(A.LX[f0], A.LX[f1], A.LX[i]) != 0) col = false;
            col = __all_sync(FULL, col);
            if (col) {
                bool finite_ring = false;
                for (int i = w.lane; i < k; i += 32) {
                    if (A.L[i] == KDT_GHOST || A.L[i + 1 == k ? 0 : i + 1] == KDT_GHOST) continue;
                    int4 ov = __ldcg(d.tv + (A.ON[i] >> 2));
                    if (ov.x != KDT_GHOST && ov.y != KDT_GHOST && ov.z != KDT_GHOST) finite_ring = true;
                }
                if (!__any_sync(FULL, finite_ring)) {
                    release_star(w, d);
                    return DEV_DEGENERATE;
                }
            }
        }
        // Ear clipping over the link polygon (L, ON, LX).  T[i] counts the failed tests
        // of ear i (L[i], L[i+1], L[i+2]): its orientation, and one per other link
        // vertex in conflict with it, so the valid ears are those with T[i] == 0.  A
        // round clips every valid ear no neighbour of which is clipped (each valid ear is
        // a triangle of the hole's unique triangulation).  Removing vertices only removes
        // conflicts from an ear whose three vertices stay consecutive, so such an ear
        // loses the clipped vertices it conflicted with, and only the ears next to a
        // clipped one are tested in full again: O(m^2) tests for the whole hole, not per
        // round (a point beside a straight lattice row has hundreds of collinear link
        // vertices and loses about one ear per round).  I lists the ears to test, then
        // the clipped ears; lane c holds the bits of ears 32c .. 32c+31 in word registers.
        int m = k, newc = 0, nt = k;
        for (int i = w.lane; i < m; i += 32) {
            A.T[i] = 0;
            A.I[i] = i;
        }
        __syncwarp();
        while (m > 3) {
            unsigned ex = 0, ti = 0;
            {
                const long long npair = (long long)nt * (m - 2);
                for (long long base = 0; base < npair; base += 32) {
                    long long idx = base + w.lane;
                    if (idx < npair) {
                        int r = (int)(idx / (m - 2)), t = (int)(idx - (long long)r * (m - 2));
                        int i = A.I[r];
                        if (ear_test_fails(A.L, A.LX, m, i, t, d, &ex, &ti)) atomicAdd(A.T + i, 1);
                    }
                }
            }
            __syncwarp();
            // greedy choice in index order, keeping >= 3 vertices (warp-uniform on ballots)
            const int nch = (m + 31) >> 5;
            unsigned pw = 0;
            int ns = 0;
            {
                bool prev = false, first = false;
                for (int c = 0; c < nch; ++c) {
                    int idx = (c << 5) + w.lane;
                    unsigned vm = __ballot_sync(FULL, idx < m && vload(A.T + idx) == 0);
                    unsigned pm = 0;
                    int last = -2;
                    while (vm && ns < m - 3) {
                        int b = __ffs(vm) - 1;
                        vm &= vm - 1u;
                        int i = (c << 5) + b;
                        if (b == 0 ? prev : last == b - 1) continue;
                        if (i == m - 1 && first) continue;
                        pm |= 1u << b;
                        last = b;
                        ++ns;
                        if (i == 0) first = true;
                    }
                    prev = (pm >> 31) & 1u;
                    if (w.lane == c) pw = pm;
                }
            }
            if (ns == 0) {
                // cannot happen for a valid star; leave the store to the fallback
                release_star(w, d);
                return DEV_INTERNAL;
            }
            // the clipped ears in index order
            for (int c = 0, at = 0; c < nch; ++c) {
                unsigned pm = __shfl_sync(FULL, pw, c);
                if ((pm >> w.lane) & 1u) A.I[at + __popc(pm & ((1u << w.lane) - 1u))] = (c << 5) + w.lane;
                at += __popc(pm);
            }
            __syncwarp();
            // lane r writes the r-th clipped ear into slot S[newc + r]
            for (int r = w.lane; r < ns; r += 32) {
                int i = A.I[r], i1 = i + 1 == m ? 0 : i + 1, i2 = i1 + 1 == m ? 0 : i1 + 1;
                int X = A.S[newc + r];
                int Li = A.L[i], Li1 = A.L[i1], Li2 = A.L[i2];
                int oi = A.ON[i], oi1 = A.ON[i1];
                d.tv[X] = make_int4(Li, Li1, Li2, ALIVE);
                d.tn[X] = make_int4(oi1, -1, oi, w.token);
                backptr(d, oi1, (X << 2) | 0);
                backptr(d, oi, (X << 2) | 2);
                if (Li >= 0) d.pt_tri[Li] = X;
                if (Li1 >= 0) d.pt_tri[Li1] = X;
                if (Li2 >= 0) d.pt_tri[Li2] = X;
                dirty_push(d, X);
                A.ON[i] = (X << 2) | 1;
            }
            __syncwarp();
            // an invalid ear whose vertices all stay loses the clipped vertices (the
            // middles of the clipped ears) that conflict with it
            {
                const long long npair = (long long)m * ns;
                for (long long base = 0; base < npair; base += 32) {
                    long long idx = base + w.lane;
                    const bool act = idx < npair;
                    int e = act ? (int)(idx / ns) : 0, r = act ? (int)(idx - (long long)e * ns) : 0;
                    int em = e == 0 ? m - 1 : e - 1, e1 = e + 1 == m ? 0 : e + 1;
                    // (shuffles: every lane takes part)
                    bool pem = bit_of(pw, em), pe = bit_of(pw, e), pe1 = bit_of(pw, e1);
                    if (act && !pem && !pe && !pe1 && vload(A.T + e) > 0) {
                        int v = A.I[r] + 1 == m ? 0 : A.I[r] + 1;
                        int t = v - e - 2;
                        if (t < 0) t += m;
                        if (ear_test_fails(A.L, A.LX, m, e, t, d, &ex, &ti)) atomicAdd(A.T + e, -1);
                    }
                }
            }
            __syncwarp();
            cnt_add(w, C_EXACT, __reduce_add_sync(FULL, ex));
            cnt_add(w, C_TIES, __reduce_add_sync(FULL, ti));
            // drop the clipped ears' middle vertices (vertex j goes when ear j-1 was
            // clipped), in chunks of 32 in increasing order; the ear at a kept vertex j is
            // new when ear j or ear j+1 was clipped, and is listed for the full tests
            int kept = 0, nlist = 0;
            for (int c0 = 0; c0 < m; c0 += 32) {
                int j = c0 + w.lane;
                int jm = j == 0 ? m - 1 : j - 1, j1 = j + 1 >= m ? j + 1 - m : j + 1;
                bool pj = bit_of(pw, j < m ? j : 0), pjm = bit_of(pw, j < m ? jm : 0),
                     pj1 = bit_of(pw, j < m ? j1 : 0);
                bool keep = j < m && !pjm;
                bool fresh = keep && (pj || pj1);
                unsigned km = __ballot_sync(FULL, keep);
                unsigned fm = __ballot_sync(FULL, fresh);
                int nj = kept + __popc(km & ((1u << w.lane) - 1u));
                int lv = 0, onv = 0, tv = 0;
                int2 xv = make_int2(0, 0);
                if (keep) {
                    lv = A.L[j];
                    onv = A.ON[j];
                    xv = A.LX[j];
                    tv = fresh ? 0 : vload(A.T + j);
                }
                __syncwarp();
                if (keep) {
                    A.L[nj] = lv;
                    A.ON[nj] = onv;
                    A.LX[nj] = xv;
                    A.T[nj] = tv;
                }
                if (fresh) A.I[nlist + __popc(fm & ((1u << w.lane) - 1u))] = nj;
                __syncwarp();
                kept += __popc(km);
                nlist += __popc(fm);
            }
            m -= ns;
            newc += ns;
            nt = nlist;
        }
        {
            int X = A.S[newc++];
            if (w.lane == 0) {
                d.tv[X] = make_int4(A.L[0], A.L[1], A.L[2], ALIVE);
                d.tn[X] = make_int4(A.ON[1], A.ON[2], A.ON[0], w.token);
                backptr(d, A.ON[1], (X << 2) | 0);
                backptr(d, A.ON[2], (X << 2) | 1);
                backptr(d, A.ON[0], (X << 2) | 2);
                for (int c = 0; c < 3; ++c)
                    if (A.L[c] >= 0) d.pt_tri[A.L[c]] = X;
                dirty_push(d, X);
            }
        }
        // the two slots left over
        spare0 = A.S[k - 2];
        spare1 = A.S[k - 1];
        hint = A.S[0];
        if (w.lane == 0) {
            d.tv[spare0].w = 0;
            d.tv[spare1].w = 0;
            d.pt_tri[p] = -1;
        }
        cnt_add(w, C_DEG_DEL, k);
        cnt_add(w, C_DELETES, 1);
        release_star(w, d);
        return DEV_OK;
    }
}

__device__ __forceinline__ int delete_point(Warp w, const Dev &d, int p, int &spare0, int &spare1, int &hint,
                                            bool may_give_up = false)
{
    return delete_point_in(w, d, p, spare0, spare1, hint, star_shared(w.sh), may_give_up);
}

// Move p to q in place (no deletion): when every triangle around p stays counter-
// clockwise with p at q, the star is still a triangulation of the same star-shaped
// link polygon, so the whole triangulation stays valid; edges not in the star keep
// their triangles and their vertices' positions, so by the Delaunay lemma only the
// star's edges (the spokes p-v_i and the link edges v_i-v_{i+1}) can fail to be locally
// Delaunay.  If none fails, only p's coordinate changes.  Otherwise, with `flip`, the
// failing edges are flipped (Lawson's algorithm from a valid triangulation reaches
// the unique Delaunay triangulation; the kinetic move-and-flip of the related work
// in Section II) and their triangles go to the dirty list, so the certification that
// ends every step settles anything the flip stack drops.  Exact SoS predicates decide,
// as everywhere.  Only for an interior p.  Returns 1 (moved), 0 (not so: the caller
// deletes and inserts), or a DevStatus error.  The star and its claims live in A and
// the current claim list (the caller provides room for 2k claims).
__device__ __noinline__ int move_in_place(Warp w, const Dev &d, int p, int2 q, Star A, bool flip)
{
    for (int attempt = 0;; ++attempt) {
        if (attempt > d.retry_cap) return DEV_RETRY;
        if (read_status(d)) return -1;
        int k = gather_star(w, d, p, A);
        if (k == -2) return 0;  // beyond even the scratch: leave it to the deletion
        if (k < 3) {
            backoff(w, attempt);
            continue;
        }
        for (int i = w.lane; i < k; i += 32) A.T[i] = A.ON[i] >> 2;
        __syncwarp();
        bool ok = claim_star_list(w, d, A.S, k);
        if (ok) ok = claim_star_list(w, d, A.T, k);
        if (ok) {
            bool good = true;
            for (int i = w.lane; i < k; i += 32) {
                int4 v = __ldcg(d.tv + A.S[i]);
                int4 nb = __ldcg(d.tn + A.S[i]);
                int I = A.I[i];
                good = good && (v.w & ALIVE) && comp(v, I) == p && comp(v, (I + 1) % 3) == A.L[i] &&
                       comp(nb, I) == A.ON[i] && (comp(nb, (I + 1) % 3) >> 2) == A.S[i + 1 == k ? 0 : i + 1];
            }
            ok = __all_sync(FULL, good);
        }
        if (!ok) {
            release_star(w, d);
            backoff(w, attempt);
            continue;
        }
        bool hull = false;
        for (int i = w.lane; i < k; i += 32) {
            int lv = A.L[i];
            hull = hull || lv == KDT_GHOST;
            A.LX[i] = lv >= 0 ? __ldcg(d.xy + lv) : make_int2(0, 0);
        }
        if (__any_sync(FULL, hull)) {
            release_star(w, d);
            return 0;
        }
        __syncwarp();
        bool ccw = true;
        unsigned ex = 0, ti = 0;
        // T[i]: bit 0 = spoke p-L[i] fails, bit 1 = link edge L[i]-L[i+1] fails
        for (int i = w.lane; i < k; i += 32) {
            int i0 = i == 0 ? k - 1 : i - 1, i1 = i + 1 == k ? 0 : i + 1;
            int a = A.L[i0], b = A.L[i], c = A.L[i1];
            int2 pa = A.LX[i0], pb = A.LX[i], pc = A.LX[i1];
            // triangle (p, b, c) counter-clockwise with p at q
            ccw = ccw && orient2d(q, pb, pc) > 0;
            // spoke p-b: c outside the circle of (p, a, b)
            int fails = conflict(p, a, b, q, pa, pb, c, pc, d.use_filter, &ex, &ti) ? 1 : 0;
            // link edge b-c: the apex across it outside the circle of (p, b, c)
            int ref = A.ON[i];
            int4 ov = __ldcg(d.tv + (ref >> 2));
            int r = comp(ov, ref & 3);
            int2 pr = r >= 0 ? __ldcg(d.xy + r) : make_int2(0, 0);
            if (conflict(p, b, c, q, pb, pc, r, pr, d.use_filter, &ex, &ti)) fails |= 2;
            A.T[i] = fails;
        }
        cnt_add(w, C_EXACT, __reduce_add_sync(FULL, ex));
        cnt_add(w, C_TIES, __reduce_add_sync(FULL, ti));
        ccw = __all_sync(FULL, ccw);
        __syncwarp();
        bool del = true;
        for (int i = w.lane; i < k; i += 32) del = del && A.T[i] == 0;
        del = __all_sync(FULL, del);
        if (!ccw || (!del && !flip)) {
            release_star(w, d);
            return 0;
        }
        if (w.lane == 0) {
            d.xy[p] = q;
            __threadfence();
        }
        __syncwarp();
        if (del) {
            release_star(w, d);
            return 1;
        }
        // the failing edges onto the flip stack (triangle i = (p, L[i], L[i+1]) holds p
        // at index I[i]: the link edge is opposite p, the spoke p-L[i] opposite
        // L[i+1]); their triangles (both sides of a spoke) to the dirty list
        int top = 0;
        for (int c0 = 0; c0 < k; c0 += 32) {
            int i = c0 + w.lane;
            int f = i < k ? A.T[i] : 0;
            if (f) {
                int im = i == 0 ? k - 1 : i - 1;
                dirty_push(d, A.S[i]);
                if (f & 1) dirty_push(d, A.S[im]);
            }
            unsigned sm = __ballot_sync(FULL, f & 1), lm = __ballot_sync(FULL, (f & 2) != 0);
            int lt = __popc(sm & ((1u << w.lane) - 1u)) + __popc(lm & ((1u << w.lane) - 1u));
            if (f & 1 && top + lt < STACK) w.sh->stack[top + lt] = make_int2(A.S[i], (A.I[i] + 2) % 3);
            if (f & 2 && top + lt + (f & 1) < STACK) w.sh->stack[top + lt + (f & 1)] = make_int2(A.S[i], A.I[i]);
            top += __popc(sm) + __popc(lm);
        }
        if (top > STACK) {
            cnt_add(w, C_STACK_DROP, 1);
            top = STACK;
        }
        __syncwarp();
        release_star(w, d);
        lawson(w, d, top, -2, false);
        return 1;
    }
}

// Delete a point of degree above KMAX with the star in the warp's global scratch (and
// its claims in the scratch's claim list).  DEV_DEGREE when there is no scratch.
__device__ __noinline__ int delete_point_big(Warp w, const Dev &d, int p, int &spare0, int &spare1, int &hint)
{
    int *big = warp_big(d);
    if (!big) return DEV_DEGREE;
    __syncwarp();
    if (w.lane == 0) w.sh->clbig = 1;
    __syncwarp();
    int rc = delete_point_in(w, d, p, spare0, spare1, hint, star_big(big), false);
    __syncwarp();
    if (w.lane == 0) w.sh->clbig = 0;
    __syncwarp();
    return rc;
}

// move_in_place with the star in the warp's global scratch (degree above KMAX), with
// flips when the move keeps the star valid but not Delaunay.
__device__ __noinline__ int move_in_place_big(Warp w, const Dev &d, int p, int2 q)
{
    int *big = warp_big(d);
    if (!big) return 0;
    __syncwarp();
    if (w.lane == 0) w.sh->clbig = 1;
    __syncwarp();
    int rc = move_in_place(w, d, p, q, star_big(big), true);
    __syncwarp();
    if (w.lane == 0) w.sh->clbig = 0;
    __syncwarp();
    return rc;
}

}  // namespace kd
