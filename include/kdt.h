/*
 * kdt.h — C ABI of the GB300 kinetic Delaunay library (libkdt.so).
 *
 * The library maintains the Delaunay triangulation of a set of moving points in the
 * plane on one GPU.  It follows the problem statement of the paper "A parallel
 * algorithm for Delaunay triangulation of moving points on the plane":
 *   - input: a point set with x and y coordinates (Section I) whose triangulation
 *     satisfies the Delaunay constraints (the input of Fig. 4);
 *   - at each time step some points move (Section III, movepoint_i) and the
 *     triangulation is repaired by deleting each moved point and inserting it at its
 *     new position (Section IV; the Update, Delete and Insert steps of Fig. 4);
 *   - output: the Delaunay triangulation after every time step (the output of Fig. 4
 *     at the end of each step).
 * The triangulation is the unique one defined by the empty-circumcircle property
 * (Section I); ties between cocircular points are broken by Simulation of Simplicity
 * (a smaller point id gets a larger lifting perturbation), so results are
 * bit-reproducible.
 *
 * Conventions for every function:
 *   - Return 0 on success or a negative KDT_ERR_* code; kdt_error_string() names it.
 *   - Pointers marked "host or device" may point to host memory (pageable or pinned)
 *     or to device memory of the handle's GPU; the library detects which and copies
 *     as needed.  Device memory of any other GPU is rejected with KDT_ERR_ARG before
 *     anything is launched (managed memory is accepted).  The caller keeps ownership
 *     of every buffer it passes; the library copies inputs in before returning and
 *     never keeps a caller pointer.
 *   - The library owns all device state of a handle (allocated in kdt_create /
 *     kdt_build, freed in kdt_destroy).  Handles are independent; no global state.
 *   - Coordinates are int32 in [0, 2^domain_bits) with domain_bits <= 28.
 *   - All work is issued on the handle's CUDA stream; every call below is complete
 *     (stream-synchronous) when it returns unless stated otherwise.
 *   - On an error detected before a step starts modifying the state, the state is
 *     unchanged.  On an error found while a step runs (duplicate target, degenerate
 *     configuration), the step is rolled back: positions are restored and the
 *     triangulation is rebuilt, so the state is again unchanged.
 */
#ifndef KDT_H
#define KDT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------------ */
#define KDT_OK 0
#define KDT_ERR_ARG (-1)             /* bad argument (NULL, n < 0, id out of range, ...) */
#define KDT_ERR_RANGE (-2)           /* a coordinate outside [0, 2^domain_bits)           */
#define KDT_ERR_DUPLICATE (-3)       /* coincident points, or one id moved twice in a step */
#define KDT_ERR_DEGENERATE (-4)      /* n < 3 or all points collinear                      */
#define KDT_ERR_CAPACITY (-5)        /* an output buffer is too small (*n_tri still set)   */
#define KDT_ERR_RETRY_EXHAUSTED (-6) /* conflict retries exhausted and fallback disabled   */
#define KDT_ERR_CUDA (-7)            /* a CUDA runtime call failed                         */
#define KDT_ERR_INTERNAL (-8)        /* an internal consistency check failed               */
#define KDT_ERR_STATE (-9)           /* call out of order (e.g. kdt_step before kdt_build) */
#define KDT_ERR_TOO_LARGE (-10)      /* more points than kdt_export_triangles_noalloc serves */

/* ---- types -------------------------------------------------------------------- */
typedef struct kdt kdt; /* opaque handle, owned by the library */

/* One moved point: the point's id and its new absolute position (Section III,
 * movepoint_i; Lemma 1 moves are axis-aligned, but any target is accepted). */
typedef struct {
    int32_t id, x, y;
} kdt_move;

/* Configuration (kdt_default_config fills the defaults).  The paper's only
 * parameters are the block layout (Section III, Data structure) and N of the
 * d-calculation; the rest are implementation choices. */
typedef struct {
    int32_t grid;          /* G: G x G equal-area partitions over [0,2^domain_bits)^2; 0 = auto
                              (about 256 points per partition)                              */
    int32_t domain_bits;   /* B <= 28: coordinates lie in [0, 2^B)                           */
    int32_t retry_cap;     /* claim retries per operation before giving up (default 4096)   */
    int32_t fallback;      /* 1: on retry exhaustion / large steps do a full GPU rebuild
                              (default); 0: return KDT_ERR_RETRY_EXHAUSTED instead          */
    float rebuild_ratio;   /* m / n above which a step is done as a full rebuild (0.25)     */
    int32_t filter;        /* 1: FP32 filter in front of the exact incircle (default)       */
    int32_t verify;        /* 1: run the full GPU verifier after every step (tests)         */
    int32_t timing;        /* 1: time the kinetic kernel with CUDA events (kdt_stats)       */
    int32_t warps_per_block; /* kinetic kernel launch shape (default 4)                      */
    int32_t build_warps;   /* warps inserting concurrently during a build (0 = auto)         */
    int32_t kinetic_warps; /* warps moving points concurrently in a step (0 = one per cell)  */
    int32_t debug;         /* bit 0: on an in-step failure keep the failed state (no
                              fallback, no roll-back) so kdt_export_store can inspect it;
                              bit 1: record the kinetic launch's timeline (span_* stats)     */
    int32_t use_graph;     /* 1: launch each step as one captured CUDA graph (default)       */
    int32_t points_per_partition; /* partition size of batched instances (0 = 256)           */
    int32_t warps_per_partition;  /* warps sharing one partition's moves (0 = 1)             */
    int32_t autotune;      /* 1: time the first steps over points per partition {128, 256,
                              512} x warps per partition {1, 2, 4} and keep the fastest       */
    int32_t variant;       /* 0: every move deletes and re-inserts the point (the paper's
                              method, default).  1: first test whether the point can move
                              in place: every triangle of its star stays counter-clockwise
                              and every edge of the star stays locally Delaunay at the new
                              position (a safe-region test in the spirit of the paper's
                              related work [6]); if so only the position changes, else
                              delete + insert.  2: move and flip (the kinetic approach of
                              the related work [4]): a move that keeps every triangle of
                              the star counter-clockwise only changes the position, and
                              the star's edges that stop being locally Delaunay are
                              flipped by the step's certification and repair; else delete
                              + insert.  The triangulation is the same in every case.       */
    int32_t quadtree;      /* 1: partitions are the leaves of the paper's quad-tree (Section
                              III, Data structure) instead of the grid: the square of side
                              S (a power of two >= the points' larger extent) at the points'
                              minimum corner is divided into four, recursively, until every
                              square holds at most points_per_partition points (256 if 0) or
                              has side S / 2^11; blocks are numbered depth-first (children
                              low-x low-y, high-x low-y, low-x high-y, high-x high-y).  Built
                              by kdt_build from the initial positions; a moved point's block
                              is the leaf holding its current position (clamped into the
                              square).  2: as 1, and the division is made again at the start
                              of every step from the current positions (Fig. 4 runs the
                              division inside its time loop), on the GPU, within the square
                              of the build (positions outside it are clamped into it); the
                              number of partitions then changes from step to step
                              (kdt_num_cells gives the last step's), and the displacement rule
                              below is inactive.  Single-instance handles only
                              (kdt_build_batch returns KDT_ERR_ARG).  Scheduling only: the
                              triangulation is the same.                                     */
    float rebuild_displacement; /* f; 0 = off (default).  The rebuild rule of the paper's
                              abstract (points that move far are cheaper to triangulate
                              again) with Section III's d as the yardstick: before a step
                              changes anything, every move's squared displacement |q - p|^2
                              is compared with f^2 * d_local^2, where d_local^2 is the
                              running minimum of the N-th nearest-neighbour squared
                              distance over the move's partition (the per-partition minima
                              of kdt_d_values, kept over its calls since the partitions
                              were last set, N of the last call).  If any move exceeds it
                              the step is done as a certified GPU rebuild of the final
                              positions (kdt_stats.far_rebuilds).  With f > 0 a step that
                              finds no d values computes them first (N = 1, or the N of the
                              last call).  The triangulation is the same either way.      */
    int32_t plan;          /* step planner, two bits (scheduling only; the triangulation is the
                              same).  Bit 0 (1): before the moves start, every move's star is
                              walked (its degree k), each partition's work is estimated as
                              the sum over its moves of k + 8 (plus the network's predicted
                              cavity size 2^out17 with bit 1 and a proposal), and the
                              partitions are handed out largest estimate first (64
                              logarithmic classes).  Bit 1 (2): with a proposal set
                              (kdt_set_proposal) the network is evaluated for all moves at
                              once by the planner instead of inside each move; its guess is
                              the locate's first candidate.  Bit 2 (4), with bit 1: the
                              planner evaluates the network on the tensor cores (as
                              kdt_mlp_forward_tc does) instead of one thread per move.
                              0 (default): none.                                            */
    int32_t batch_build;   /* 1 (default): the instances of a batch are (re)built together,
                              one set of launches for all of them; 0: one instance after
                              another.  The triangulations are the same.                    */
    int32_t kinetic_blocks_per_sm; /* 0 or 6 (default): the kinetic kernel compiled for six
                              128-thread blocks per SM (up to 80 registers a thread); 7: for
                              seven (up to 72 registers, more warps in flight).  Scheduling
                              only.                                                          */
    int32_t partition_order; /* 0 (default): without a planned order the kinetic kernel takes
                              the partitions scattered, ticket k -> partition k * s mod the
                              count (s coprime with the count, near 0.618 of it), so that
                              partitions worked on at the same time are rarely neighbours
                              (fewer claim conflicts on the triangles they share); 1: index
                              order.  Scheduling only.                                       */
} kdt_config;

/* Counters since creation (or kdt_reset_stats). */
typedef struct {
    int64_t steps, moves, rebuilds, fallbacks, kernel_launches;
    int64_t flips, retries, walk_steps, exact_incircle, sos_ties, deferred;
    int64_t violations, fixup_flips, deleted_degree_sum, stack_drops, edge_splits;
    int64_t ghost_splits, deletes, inserts, flip_tests;
    double kinetic_kernel_ms; /* sum of event-timed kinetic kernel durations (timing = 1) */
    int64_t kinetic_kernel_timed; /* launches included in kinetic_kernel_ms               */
    int64_t last_fallback_reason; /* internal status that triggered the last fallback     */
    int64_t last_fallback_point;  /* point whose operation reported it (-1 if unknown)     */
    int64_t staged_to_global;     /* moves that left the staged region (long / hull moves)  */
    int64_t cycles_move;          /* SM cycles summed over moved points (kinetic kernel)   */
    int64_t cycles_move_max;      /* longest single move, cycles                            */
    int64_t cycles_gather, cycles_claim, cycles_local, cycles_writeback; /* phase sums    */
    double step_graph_ms;         /* event-timed control copy + step graph (timing = 1)     */
    int64_t tuned_points_per_partition, tuned_warps_per_partition; /* autotuner choice   */
    int64_t cycles_ear, cycles_lawson, cycles_certify; /* parts of cycles_local             */
    int64_t proposal_moves;       /* staged moves located with the learned proposal on      */
    int64_t proposal_hits;        /* ... whose proposed hole triangle held the new position */
    int64_t trace_rows;           /* training rows written (kdt_set_trace)                  */
    int64_t tail_moves;           /* moves the last warp of a step ran alone                */
    int64_t cycles_tail;          /* SM cycles of those last-warp tails                      */
    int64_t big_moves;            /* moves of points of degree above 64 (star in scratch)    */
    int64_t cycles_big;           /* SM cycles of those moves                                */
    int64_t drain_moves;          /* moves taken again from the list of moves left for later */
    int64_t span_tickets_ns;      /* kinetic launches (global timer, summed; debug bit 1):  */
                                  /* start to the                                           */
    int64_t span_drain_ns;        /* last warp out of partitions, to the last warp out of   */
    int64_t span_kernel_ns;       /* the moves left for later, to the end of the step tail  */
    int64_t span_huge_ns;         /* ... start to the end of the last high-degree move      */
    int64_t span_drained_ns;      /* ... start to the end of the last other drained move    */
    int64_t cycles_drained_max;   /* longest move taken from the list, cycles (debug bit 1) */
    int64_t redeferred;           /* drained moves left for later again (debug bit 1)       */
    int64_t far_rebuilds;         /* steps done as a rebuild because a move went farther
                                     than rebuild_displacement * d_local                  */
    int64_t big_in_place;         /* moves of points of degree above 64 done in place      */
    int64_t cycles_big_in_place;  /* SM cycles of their in-place attempts                  */
    int64_t cycles_big_delete;    /* ... of their deletions (when not in place)            */
    int64_t cycles_big_insert;    /* ... of the insertions that followed those deletions   */
    int64_t cycles_unyielding_max; /* longest move run without giving up (a high-degree
                                     move, or a move taken again from the list), cycles   */
    int64_t cycles_global_insert; /* SM cycles of insertions finished on the global-memory path
                                     after a deletion (moves that left the staged region)  */
    int64_t cycles_global_insert_max; /* the longest of those, cycles                       */
    int64_t tensor_timeouts;      /* CTAs of the tensor-core network kernels that gave up
                                     waiting for their products (after about a second):
                                     planner guesses left out (the step stays exact),
                                     kdt_mlp_*_tc results NaN                              */
} kdt_stats;

/* ---- lifecycle ------------------------------------------------------------------ */

/* Fill *cfg with the defaults. */
int kdt_default_config(kdt_config *cfg);

/* Create a handle on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  cfg may be NULL (defaults).
 * *out receives the handle.  Errors: KDT_ERR_ARG, KDT_ERR_CUDA. */
int kdt_create(kdt **out, const kdt_config *cfg, int device, void *cuda_stream);

/* Release every resource of the handle.  NULL is accepted. */
int kdt_destroy(kdt *h);

/* ---- the method ------------------------------------------------------------------ */

/* Build the Delaunay triangulation of n distinct points xy[2*i], xy[2*i+1]
 * (host or device) from scratch on the GPU: the triangulated point set that Fig. 4
 * starts from, divided into the blocks of Section III.  Replaces any
 * previous state.  Errors: KDT_ERR_ARG (NULL, n > 2^28), KDT_ERR_RANGE,
 * KDT_ERR_DUPLICATE, KDT_ERR_DEGENERATE (n < 3 or all collinear), KDT_ERR_CUDA. */
int kdt_build(kdt *h, const int32_t *xy, int64_t n);

/* One time step (Fig. 4 loop body) of a single-instance handle: the m moves (host or
 * device; distinct ids) are
 * applied simultaneously and the triangulation of the new positions is restored:
 * per partition, each moved point is deleted from the triangulation and inserted at
 * its new position (Section IV).  The result does not depend on the order of the
 * moves.  m = 0 is a no-op.  Errors (state unchanged): KDT_ERR_ARG (id out of range),
 * KDT_ERR_RANGE, KDT_ERR_DUPLICATE (repeated id, or a target coinciding with
 * another final position), KDT_ERR_DEGENERATE (all final positions collinear),
 * KDT_ERR_RETRY_EXHAUSTED (only with fallback = 0), KDT_ERR_STATE, KDT_ERR_CUDA. */
int kdt_step(kdt *h, const kdt_move *moves, int64_t m);

/* Batched instances (many independent point sets advanced by one step launch; the
 * paper's blocks of one data set generalised to blocks of many data sets).  xy holds
 * the points of all instances back to back; offsets (host, n_inst + 1 entries,
 * offsets[0] = 0) delimits them, every instance having at least 3 points.  Each
 * instance gets its own triangulation; point ids inside an instance are local
 * (0 .. n_i - 1) in the step and per-instance export calls, global (offsets[i] + local)
 * in kdt_export_triangles / kdt_export_points.  Errors as kdt_build. */
int kdt_build_batch(kdt *h, const int32_t *xy, const int64_t *offsets, int32_t n_inst);

/* One time step of every instance of a batched handle: moves (host or device) with
 * instance-local ids, move_offsets (host, n_inst + 1 entries) delimiting each
 * instance's moves.  Errors as kdt_step. */
int kdt_step_batch(kdt *h, const kdt_move *moves, const int64_t *move_offsets, int32_t n_inst);

/* Canonical triangle list of one instance, with instance-local ids (as
 * kdt_export_triangles for a single instance). */
int kdt_export_triangles_inst(kdt *h, int32_t inst, int32_t *out, int64_t cap, int64_t *n_tri);

/* Number of instances of the current state (0 before a build). */
int32_t kdt_num_instances(const kdt *h);

/* Rebuild the triangulation of the current positions from scratch on the GPU (the
 * full-rebuild comparator; the same code is the fallback of kdt_step). */
int kdt_rebuild(kdt *h);

/* Export the triangulation (what Fig. 4 returns after each time step) as the canonical list:
 * every finite triangle counter-clockwise, rotated so its smallest id comes first,
 * rows sorted lexicographically; 3 int32 per row into out (host or device, capacity
 * `cap` rows).  *n_tri receives the row count (2n - 2 - h, h = hull points) even when
 * the buffer is too small (KDT_ERR_CAPACITY).  out may be NULL with cap = 0 to query. */
int kdt_export_triangles(kdt *h, int32_t *out, int64_t cap, int64_t *n_tri);

/* Copy the current positions (2 int32 per point) into xy (host or device). */
int kdt_export_points(kdt *h, int32_t *xy, int64_t cap_points);

/* Export without allocating (the paper has no counterpart; this serves callers).
 * kdt_export_triangles grows its own device scratch and staging buffers on first use
 * and whenever the point count grows, so it calls cudaMalloc.  Some callers cannot
 * allow that: an application that reserved the whole device memory budget for its
 * own pool before creating the handle, or a per-step output loop that must not take
 * the CUDA driver's allocation path.  This entry point produces the same canonical list
 * (same order, same rows) and allocates nothing: its scratch (per-vertex counts and
 * offsets, scan partial sums) is one file-scope device array of
 * KDT_NOALLOC_MAX_POINTS * 8 + 4 KiB bytes (about 8 MiB), which every GPU that
 * loads the library holds until the process exits.
 *   out:   DEVICE pointer (this handle's GPU), capacity `cap` rows of 3 int32; a host
 *          pointer is rejected with KDT_ERR_ARG (copying to it would need staging).
 *   n_tri: receives the row count, also on KDT_ERR_CAPACITY.
 * Errors: KDT_ERR_TOO_LARGE when the handle holds more than KDT_NOALLOC_MAX_POINTS
 * points (nothing is launched); KDT_ERR_CAPACITY, KDT_ERR_ARG, KDT_ERR_STATE,
 * KDT_ERR_CUDA.
 * The first call on a device looks the scratch array's device address up
 * (cudaGetSymbolAddress, with that device current) and caches it for the life of the
 * process; make that first call before any stream capture.  A cudaDeviceReset of that
 * device discards the array with the context, so do not call this entry point after
 * one.  All calls share the one array, so calls that
 * overlap on the GPU (other handles' streams, other host threads) race; serialise
 * them.  Each call clears what must start at zero. */
#define KDT_NOALLOC_MAX_POINTS (1 << 20)
int kdt_export_triangles_noalloc(kdt *h, int32_t *out, int64_t cap, int64_t *n_tri);

/* ---- d-calculation (Section III "Notation and definitions"; Section IV) ------------
 * For a constant N (1 <= N <= 16, N < the smallest instance's point count): for every
 * point p, dist_p^2 = the squared distance to its N-th nearest other point of its own
 * instance (exact int64); the minimum of dist_p^2 over the points of each partition
 * (the partitions of the steps: grid cell (x * G >> domain_bits, y * G >> domain_bits),
 * row-major, instances one after another, or the quad-tree leaf) and over all points,
 * mindistance(P)^2; and
 * d^2 = the minimum of mindistance^2 over the calls since the last kdt_build /
 * kdt_build_batch with the same N (the paper's d = min over the time steps; a call
 * with another N starts the minimum again).  The N-th nearest neighbour is found on
 * the triangulation (exact: see kdt_dcalc.cuh); nothing in the state changes.
 *   dist2:     n int64 (host or device), or NULL;
 *   cell_min2: one int64 per partition (host or device; INT64_MAX for an empty cell),
 *              or NULL;
 *   info:      host, required.
 * Errors: KDT_ERR_ARG (N out of range, info NULL), KDT_ERR_STATE (not built),
 * KDT_ERR_CUDA.  Allocates device scratch (neighbour lists, ~28 bytes per point). */
typedef struct {
    int64_t min2;     /* mindistance(P)^2 of this call                                     */
    int64_t d2;       /* d^2: the running minimum (see above)                              */
    double spread;    /* N-spread of a block, Delta_N(P_i) = diam(P_i) / d with diam(P_i)
                         the grid cell's diagonal (one instance on the grid; the largest
                         leaf's for the quad-tree; 0 for a batch)                           */
    int64_t max_degree; /* largest vertex degree met (the search's fan-out)                */
    int64_t cells;    /* partitions (entries of cell_min2)                                 */
} kdt_dinfo;
int kdt_d_values(kdt *h, int32_t N, int64_t *dist2, int64_t *cell_min2, kdt_dinfo *info);

/* Partitions of the current state (grid cells or quad-tree leaves: the entries of
 * kdt_d_values' cell_min2; 0 before a build). */
int64_t kdt_num_cells(const kdt *h);

/* Full GPU verifier: every triangle alive and counter-clockwise, adjacency
 * reciprocal, every edge locally Delaunay (SoS), 2n - 2 triangles with ghosts, every
 * point's incident-triangle pointer valid.  *bad receives the number of failures. */
int kdt_verify(kdt *h, int64_t *bad);

/* Number of points of the current state (0 before kdt_build). */
int64_t kdt_num_points(const kdt *h);

/* Counters. */
int kdt_get_stats(const kdt *h, kdt_stats *out);
int kdt_reset_stats(kdt *h);

/* Human-readable name of an error code. */
const char *kdt_error_string(int code);

/* ABI version (incremented on any incompatible change). */
int kdt_version(void);

/* sizeof(kdt_stats) and sizeof(kdt_config) as this library was built (a binding
 * checks its own layouts against them). */
int64_t kdt_stats_size(void);
int64_t kdt_config_size(void);

/* ---- diagnostics ---------------------------------------------------------------- */

/* Copy the raw triangle store into host buffers (diagnostics): tv and tn receive
 * 4 int32 per slot (cap_slots >= 2n - 2; see the store layout in the design notes),
 * pt_tri n int32.  Any pointer may be NULL to skip it. */
int kdt_export_store(kdt *h, int32_t *tv, int32_t *tn, int32_t *pt_tri, int64_t cap_slots);

/* Evaluate the device predicates on m quadruples of point indices (Section I,
 * empty-circumcircle test).  xy: device, 2 int32 per point; quads: device, 4 int32
 * (a, b, c, d) per row; out: device, 4 int32 per row receiving
 *   orient2d(a,b,c), exact incircle sign, FP32-filter verdict (0 = uncertain),
 *   SoS incircle sign (filter as selected by use_filter).
 * Runs on `cuda_stream` and synchronizes it.  Used by the parity tests. */
int kdt_eval_predicates(const int32_t *xy, const int32_t *quads, int64_t m, int32_t *out,
                        int use_filter, void *cuda_stream);

/* ---- learned locate proposal (this library's extension; the paper has none) ------
 *
 * The paper locates the new position of a moved point by a walk (Section IV,
 * insertion).  Here the staged kinetic move first tests the hole triangle a small
 * network proposes, then (on a miss) every staged triangle; the exact tests decide,
 * so the triangulation never depends on the network.  A training row describes one
 * move of an interior point p to q on the triangulation in force when the move starts:
 *
 *   link    v_0..v_{k-1}: the neighbours of p, counter-clockwise;
 *   j0      the one j whose half-open wedge [dir(v_j - p), dir(v_{j+1} - p)) holds
 *           d = q - p; rotated index r(v_j) = (j - j0) mod k;
 *   hole    the k - 2 triangles that replace p's star when p is deleted; each is named
 *           by its rotated vertex indices sorted ascending, and the names sorted
 *           lexicographically give the ranks;
 *   slot    the lowest rank of a hole triangle whose closed region holds q, or 16
 *           ("beyond") when none does or that rank is 16 or more;
 *   cavity  the number of triangles the insertion of q destroys (Bowyer-Watson);
 *   features (32 FP32, every operation correctly rounded): f0 = |d| / R, f1 = k / 16,
 *           f[2+2r] = <v_{j0+r} - p, u> / R and f[3+2r] = <v_{j0+r} - p, n> / R for
 *           r = 0..14 (0 for r >= k), u = d / |d|, n = u turned a quarter
 *           counter-clockwise, R = mean |v_j - p| summed in rotated order.
 *
 * Network: 32 -> 64 (ReLU) -> 64 (ReLU) -> 18; outputs 0..16 are slot logits, output
 * 17 predicts log2(cavity).  Parameters: KDT_MLP_PARAMS BF16 values in the order
 * W1 [64][32] (row = output unit), b1 [64], W2 [64][64], b2 [64], W3 [18][64], b3 [18];
 * products and sums in FP32.  Loss of a batch: mean over rows of
 * cross-entropy(logits, slot) + lam * (out17 - log2(cavity))^2. */
#define KDT_MLP_IN 32
#define KDT_MLP_HIDDEN 64
#define KDT_MLP_OUT 18
#define KDT_MLP_SLOTS 17
#define KDT_MLP_PARAMS 7442

/* Record a training row for every staged move of an interior point in the following
 * steps: features (device, cap x 32 FP32) and labels (device, cap x 2 int32: slot,
 * cavity).  The caller owns both buffers and keeps them alive while recording; rows
 * past cap are dropped.  Resets the row count.  cap = 0 (NULL buffers) stops. */
int kdt_set_trace(kdt *h, float *features, int32_t *labels, int64_t cap);

/* Rows recorded since kdt_set_trace (at most cap).  Synchronizes the handle's stream. */
int kdt_trace_count(kdt *h, int64_t *rows);

/* Use the network with these parameters (KDT_MLP_PARAMS BF16 values, host or device;
 * copied) as the locate proposal of later steps; NULL turns the proposal off. */
int kdt_set_proposal(kdt *h, const uint16_t *params_bf16);

/* Network outputs for rows inputs: x (device, rows x 32) -> out (device, rows x 18).
 * params_bf16: device, 4-byte aligned.  Asynchronous on the handle's stream (a handle
 * needs no triangulation for the kdt_mlp_* calls). */
int kdt_mlp_forward(kdt *h, const uint16_t *params_bf16, const float *x, int64_t rows, float *out);

/* The same outputs computed on the tensor cores (tcgen05, 128 rows per tile): every
 * activation is split into two BF16 parts (x = hi + lo to 2^-16 of |x|) and each layer
 * is the two BF16 products with the BF16 weights, accumulated in FP32, so an output is
 * within about 3 * 2^-15 of the magnitude sum_k |w_k| |x_k| propagated through the
 * layers of kdt_mlp_forward's value (not bit-identical: the accumulation order is the
 * hardware's).  Same arguments as kdt_mlp_forward; asynchronous.  Rows of a CTA whose
 * products did not complete within about a second are NaN (counted in
 * kdt_stats.tensor_timeouts). */
int kdt_mlp_forward_tc(kdt *h, const uint16_t *params_bf16, const float *x, int64_t rows, float *out);

/* Mean loss (device scalar, may be NULL) and its gradient with respect to the BF16
 * parameters' values (device, KDT_MLP_PARAMS FP32) over a batch: batch row r is input
 * row index[r] (device int64) or r when index is NULL; labels as kdt_set_trace writes
 * them.  Summation order is fixed, so results repeat exactly.  Asynchronous. */
int kdt_mlp_loss_grad(kdt *h, const uint16_t *params_bf16, const float *x, const int32_t *labels,
                      const int64_t *index, int64_t rows, float lam, float *grad, float *loss);

/* The same loss and gradient computed on the tensor cores (tcgen05, 128 rows per
 * tile): in the forward and backward products every activation is split into three
 * BF16 parts (to 2^-24 of its value) against the BF16 weights, and the weight
 * gradients are products over the batch rows whose FP32 operands are split into two
 * parts (three BF16 products per pair), all accumulated in FP32.  Not bit-identical
 * to kdt_mlp_loss_grad (the hardware's accumulation order); within the tolerance its
 * test uses (1e-3 of each tensor's largest entry, and of every entry above 5 % of it).
 * The summation order is fixed, so results repeat exactly.  Same arguments as
 * kdt_mlp_loss_grad (params_bf16 4-byte aligned); asynchronous.  If a CTA's products
 * did not complete within about a second the gradient and loss are NaN (counted in
 * kdt_stats.tensor_timeouts). */
int kdt_mlp_loss_grad_tc(kdt *h, const uint16_t *params_bf16, const float *x, const int32_t *labels,
                         const int64_t *index, int64_t rows, float lam, float *grad, float *loss);

/* One Adam step t >= 1 (Kingma and Ba, 2015) on FP32 master parameters with moments m
 * and v (device, KDT_MLP_PARAMS each, updated in place); params_bf16 (device, may be
 * NULL) receives the masters rounded to BF16 (nearest, ties to even).  Asynchronous. */
int kdt_mlp_adam(kdt *h, float *master, const float *grad, float *m, float *v, int64_t t, float lr,
                 float beta1, float beta2, float eps, uint16_t *params_bf16);

#ifdef __cplusplus
}
#endif

#endif /* KDT_H */
