// d-calculation (Section III "Notation and definitions"; Section IV, the sub-algorithm
// d-calculation): for a constant N, every point's distance to its N-th nearest
// neighbour, its minimum per block and over all blocks (mindistance), and the block
// N-spread that follows from it.
//
// The N-th nearest neighbour is found on the triangulation itself.  Order the other
// points by (squared distance to p, id).  The k-th of them, q, is a Delaunay neighbour
// of p or of one of the k-1 before it: grow a circle through q with its centre moving
// from q towards p; the first point it meets lies strictly inside the disk of radius
// |pq| around p, hence before q, and the empty circle through q and that point makes
// them adjacent (when several points are met at once, q is adjacent to one of them in
// every triangulation of that Delaunay face).  So taking the k nearest one at a time,
// each time from the neighbours of p and of the points already taken (the expansion of
// Dickerson, Drysdale and Sack for k nearest neighbours), is exact, and a candidate
// list of N entries suffices.  Distances are exact int64 squares.
#pragma once

#include "kdt_kernels.cuh"

namespace kd {

constexpr int DC_MAX_N = 16;  // largest N a call may ask for

// Neighbour counts from the live triangles: every edge u -> v of a triangle in
// counter-clockwise order gives u the neighbour v.  An interior edge is seen once from
// each side and a hull edge once from its finite triangle and once from its ghost, so
// every neighbour is counted exactly once.
__global__ void k_nbr_count(TriHalf tv, int nslots, int *deg)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nslots; t += gridDim.x * blockDim.x) {
        int4 v = tv[t];
        if (!(v.w & ALIVE)) continue;
        if (v.x >= 0 && v.y >= 0) atomicAdd(deg + v.x, 1);
        if (v.y >= 0 && v.z >= 0) atomicAdd(deg + v.y, 1);
        if (v.z >= 0 && v.x >= 0) atomicAdd(deg + v.z, 1);
    }
}

// The same edges written into the lists (off: exclusive scan of the counts; cur:
// zeroed fill positions).  The order inside a list does not matter.
__global__ void k_nbr_fill(TriHalf tv, int nslots, const int *off, int *cur, int *nbr)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nslots; t += gridDim.x * blockDim.x) {
        int4 v = tv[t];
        if (!(v.w & ALIVE)) continue;
        if (v.x >= 0 && v.y >= 0) nbr[off[v.x] + atomicAdd(cur + v.x, 1)] = v.y;
        if (v.y >= 0 && v.z >= 0) nbr[off[v.y] + atomicAdd(cur + v.y, 1)] = v.z;
        if (v.z >= 0 && v.x >= 0) nbr[off[v.z] + atomicAdd(cur + v.z, 1)] = v.x;
    }
}

__device__ __forceinline__ long long dist2_of(int2 a, int2 b)
{
    long long dx = (long long)a.x - b.x, dy = (long long)a.y - b.y;
    return dx * dx + dy * dy;
}

// One thread per point: the N nearest, one at a time, from the neighbour lists (see
// the header).  bd/bi hold the best candidates in (distance, id) order; entries
// 0 .. e-1 are the points taken so far.  Writes dist2[p] (if asked), the minimum of
// its partition (cell_min, if asked) and of all points (gmin); the largest degree met
// goes to max_deg.
__global__ void k_nth_nn(const int2 *xy, const int *off, const int *nbr, int n, int N, Inst I, int bits,
                         long long *dist2, unsigned long long *cell_min, unsigned long long *gmin, int *max_deg)
{
    long long best = LLONG_MAX;
    int mdeg = 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int2 pp = xy[p];
        long long bd[DC_MAX_N];
        int bi[DC_MAX_N];
        int cnt = 0;
        int src = p;
        for (int e = 0; e < N; ++e) {
            // add the neighbours of src (p, then the point taken last)
            const int lo = off[src], hi = off[src + 1];
            mdeg = max(mdeg, hi - lo);
            for (int k = lo; k < hi; ++k) {
                const int w = nbr[k];
                if (w == p) continue;
                const long long dw = dist2_of(pp, xy[w]);
                if (cnt == N && (dw > bd[N - 1] || (dw == bd[N - 1] && w >= bi[N - 1]))) continue;
                bool seen = false;
                for (int j = 0; j < cnt; ++j) seen = seen || bi[j] == w;
                if (seen) continue;
                int j = cnt < N ? cnt : N - 1;  // the slot freed at the end
                while (j > 0 && (bd[j - 1] > dw || (bd[j - 1] == dw && bi[j - 1] > w))) {
                    bd[j] = bd[j - 1];
                    bi[j] = bi[j - 1];
                    --j;
                }
                bd[j] = dw;
                bi[j] = w;
                if (cnt < N) ++cnt;
            }
            if (e == cnt) break;  // fewer than N other points reachable (cannot happen for n > N)
            src = bi[e];          // the (e+1)-th nearest: expand it next
        }
        const long long v = cnt == N ? bd[N - 1] : LLONG_MAX;
        if (dist2) dist2[p] = v;
        if (cell_min) {
            const int inst = I.ninst > 1 ? csr_find(I.pofs, I.ninst + 1, p) : 0;
            atomicMin(cell_min + partition_of(I, inst, bits, pp), (unsigned long long)v);
        }
        best = min(best, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        best = min(best, (long long)__shfl_xor_sync(FULL, (unsigned long long)best, o));
        mdeg = max(mdeg, __shfl_xor_sync(FULL, mdeg, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(gmin, (unsigned long long)best);
        atomicMax(max_deg, mdeg);
    }
}

// run[c] = min(run[c], cur[c]) (or cur[c] when restart): the running per-partition
// d_local^2 of the displacement rule
__global__ void k_merge_min_u64(unsigned long long *run, const unsigned long long *cur, long long n, int restart)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        run[i] = restart ? cur[i] : min(run[i], cur[i]);
}

__global__ void k_fill_u64(unsigned long long *a, long long n, unsigned long long v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = v;
}

}  // namespace kd
