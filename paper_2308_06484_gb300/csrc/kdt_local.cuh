// Fused kinetic move of one point in a claimed, shared-memory staged region.
//
// The paper's per-block update (Fig. 4: Update, Delete, Insert; Section IV) touches
// the star of the moved point p and, for a short move, the star of its new position
// q, which overlaps it.  This operation claims p's star and the ring of triangles
// around it in one batch, copies them into the warp's shared memory (vertices,
// neighbours as global refs and as staged indices, and the coordinates of every
// vertex, so no lookup is needed later), and there
//   1. deletes p by Delaunay ears (the simple deletion Section IV prefers): every
//      (ear, vertex) test of a round runs on its own lane, and all valid ears no two
//      of which are neighbours are clipped in the same round,
//   2. locates q among the staged triangles (one triangle per lane),
//   3. inserts q by Bowyer-Watson (the insertion Section IV names): the conflict
//      test of every staged triangle on its own lane gives the cavity, which is
//      grown past the region (claiming and staging) only when it reaches its edge;
//      q is joined to the cavity boundary in the cavity's entries and two spares,
//   4. certifies every edge of every new triangle against its staged neighbour,
// then writes every modified triangle back and releases the claims.  Global memory
// sees one claim batch, one validation pass and one write-back instead of a round
// trip per ear and per flip.  When q is not inside the staged region (a long move,
// a move outside the hull) or a claim needed later fails, the work done so far is
// written back (a valid triangulation) and the caller continues on the global path.
//
// Staged values every lane computes identically are written to shared memory by all
// lanes (same value, same address); only lane-parallel writes are followed by a
// warp barrier.
#pragma once
#include "kdt_device.cuh"
#include "kdt_mlp.cuh"

namespace kd {

// outcome of move_point
// (0, negative: none of them a DevStatus, which are all positive)
// MV_BIG: p's claims kept failing; MV_HUGE: p's degree is above what the shared arrays
// hold (KMAX).  Nothing was done in either case: the move is left for later, when
// fewer warps compete for claims (MV_HUGE then takes the warp's global scratch).
enum MoveResult : int { MV_DONE = 0, MV_DEFER = -20, MV_GLOBAL = -21, MV_BIG = -22, MV_HUGE = -23, MV_ABORT = -1 };

struct Region {
    int cnt;                   // staged triangles
    unsigned long long dirty;  // modified staged triangles
    unsigned long long vchg;   // staged triangles whose vertices changed
};

__device__ __forceinline__ int local_find(const WarpShared *sh, int cnt, int slot)
{
    int idx = -1;
    for (int base = 0; base < cnt; base += 32) {
        int j = base + (threadIdx.x & 31);
        bool hit = j < cnt && sh->lslot[j] == slot;
        unsigned b = __ballot_sync(FULL, hit);
        if (b) {
            idx = base + __ffs(b) - 1;
            break;
        }
    }
    return idx;
}

__device__ __forceinline__ int ic(const int4 &v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }

// neighbour of staged triangle j across edge e: staged index and global ref (uniform write)
__device__ __forceinline__ void set_nb(WarpShared *sh, int j, int e, int lj, int gref)
{
    reinterpret_cast<int *>(&sh->lnl[j])[e] = lj;
    reinterpret_cast<int *>(&sh->ln[j])[e] = gref;
}

__device__ __forceinline__ int gref_of(const WarpShared *sh, int lref)
{
    return (sh->lslot[lref >> 2] << 2) | (lref & 3);
}

// Claim and stage one more triangle, read under the claim (so no validation is
// needed), with its vertex coordinates and its links to the staged triangles.
// Returns its staged index, or -1 when the claim fails or space runs out.
// (`cnt` staged so far; a new entry gets index cnt, and the caller counts it)
__device__ __noinline__ int ensure_local(Warp w, const Dev &d, int cnt, int slot)
{
    WarpShared *sh = w.sh;
    int j = local_find(sh, cnt, slot);
    if (j >= 0) return j;
    if (cnt >= LM || w.sh->ncl >= claim_cap(w) || slot < 0 || slot >= d.cap) return -1;
    int mine = w.lane == 0 ? slot : -1;
    if (!claim_lanes_tok(w, d, mine, 1)) return -1;
    int4 v, nb;
    load_tri(w, d, slot, v, nb);
    if (!(v.w & ALIVE)) return -1;
    int2 p0, p1, p2, pz;
    load_xy4(w, d, v.x, v.y, v.z, KDT_GHOST, p0, p1, p2, pz);
    j = cnt++;
    sh->lslot[j] = slot;
    sh->lv[j] = v;
    sh->ln[j] = nb;
    sh->lp[j][0] = p0;
    sh->lp[j][1] = p1;
    sh->lp[j][2] = p2;
    for (int e = 0; e < 3; ++e) {
        int r = ic(nb, e);
        int k = local_find(sh, cnt, r >> 2);
        reinterpret_cast<int *>(&sh->lnl[j])[e] = k;
        if (k >= 0) reinterpret_cast<int *>(&sh->lnl[k])[r & 3] = j;
    }
    __syncwarp();
    return j;
}

// make sure the neighbour of staged j across edge e is staged; its staged index or -1
__device__ __forceinline__ int nb_staged(Warp w, const Dev &d, Region &R, int j, int e)
{
    int k = ic(w.sh->lnl[j], e);
    if (k >= 0) return k;
    k = ensure_local(w, d, R.cnt, ic(w.sh->ln[j], e) >> 2);
    if (k == R.cnt) ++R.cnt;
    return k;
}

// Certify the finished region before it is written: every edge of a triangle whose
// vertices changed, tested against the staged triangle across it (all of them are
// staged and were claimed while they were read and modified).  Triangles whose
// vertices did not change only got new neighbour references: their edges keep the
// state they had.  An edge whose far side is not staged is left to the step's
// certification of the dirty list.  Returns true when every edge could be tested
// here (violations go to the violation list for the host's repair pass).
__device__ __forceinline__ bool certify_staged(Warp w, const Dev &d, const Region &R)
{
    WarpShared *sh = w.sh;
    unsigned ex = 0, ti = 0;
    bool far = false;
    for (int idx = w.lane; idx < 3 * R.cnt; idx += 32) {
        int j = idx / 3, e = idx - 3 * j;
        if (!((R.vchg >> j) & 1ull)) continue;
        int4 v = sh->lv[j];
        if (!(v.w & ALIVE)) continue;
        int k = ic(sh->lnl[j], e);
        if (k < 0) {
            far = true;
            continue;
        }
        // test each shared edge once: from the lower staged index when both changed
        if (((R.vchg >> k) & 1ull) && k < j) continue;
        int f = ic(sh->ln[j], e) & 3;
        int dd = ic(sh->lv[k], f);
        if (conflict(v.x, v.y, v.z, sh->lp[j][0], sh->lp[j][1], sh->lp[j][2], dd, sh->lp[k][f], d.use_filter,
                     &ex, &ti)) {
            int pos = atomicAdd(d.viol_count, 1);
            if (pos < d.viol_cap) d.viol[pos] = (sh->lslot[j] << 2) | e;
        }
    }
    cnt_add(w, C_EXACT, __reduce_add_sync(FULL, ex));
    cnt_add(w, C_TIES, __reduce_add_sync(FULL, ti));
    return !__any_sync(FULL, far);
}

// Write every modified staged triangle back (lane-parallel), update pt_tri of their
// vertices, release all claims, then (unless the caller certified the region on its
// staged copy) certify the written triangles against global memory.
__device__ void write_back(Warp w, const Dev &d, Region R, bool certified = false)
{
    WarpShared *sh = w.sh;
    __syncwarp();
    unsigned long long m = R.dirty;
    for (int j0 = 0; j0 < R.cnt; j0 += 32) {
        int j = j0 + w.lane;
        if (j < R.cnt && ((m >> j) & 1ull)) {
            int slot = sh->lslot[j];
            int4 v = sh->lv[j], n = sh->ln[j];
            n.w = w.token;
            d.tv[slot] = v;
            d.tn[slot] = n;
            if (v.w & ALIVE) {
                if (v.x >= 0) d.pt_tri[v.x] = slot;
                if (v.y >= 0) d.pt_tri[v.y] = slot;
                if (v.z >= 0) d.pt_tri[v.z] = slot;
            }
        }
    }
    __syncwarp();
    __threadfence();
    release_all(w, d);
    if (certified) return;
    // certify what was written: an edge whose far side changes later is certified
    // again by the operation that changes it, so the last writer of every edge checks
    // it against final data.  A transiently inconsistent read goes to the dirty list,
    // which is certified once the step is quiescent.
    unsigned ex = 0, ti = 0;
    for (int j = w.lane; j < R.cnt; j += 32) {
        if (!((m >> j) & 1ull)) continue;
        int4 v = sh->lv[j];
        if (!(v.w & ALIVE)) continue;
        int slot = sh->lslot[j];
        int4 n = sh->ln[j];
        for (int e = 0; e < 3; ++e) {
            int r = check_edge(d, slot, v, n, e, &ex, &ti);
            if (r > 0) {
                int pos = atomicAdd(d.viol_count, 1);
                if (pos < d.viol_cap) d.viol[pos] = (slot << 2) | e;
            } else if (r < 0) {
                dirty_push(d, slot);
            }
        }
    }
    __syncwarp();
}

// Locate q in staged triangle j: -1 not inside, 0 inside, 1 on edge (*e), 2 on a vertex
// (*vtx), 3 strictly outside a ghost's hull edge.
__device__ __forceinline__ int locate_in(const WarpShared *sh, int j, int2 q, int *e, int *vtx)
{
    int4 v = sh->lv[j];
    if (!(v.w & ALIVE)) return -1;
    int2 p0 = sh->lp[j][0], p1 = sh->lp[j][1], p2 = sh->lp[j][2];
    if (v.x == KDT_GHOST) return orient2d(p1, p2, q) > 0 ? 3 : -1;
    if (v.y == KDT_GHOST) return orient2d(p2, p0, q) > 0 ? 3 : -1;
    if (v.z == KDT_GHOST) return orient2d(p0, p1, q) > 0 ? 3 : -1;
    int o0 = orient2d(p1, p2, q), o1 = orient2d(p2, p0, q), o2 = orient2d(p0, p1, q);
    if (o0 < 0 || o1 < 0 || o2 < 0) return -1;
    int zeros = (o0 == 0) + (o1 == 0) + (o2 == 0);
    if (zeros == 0) return 0;
    if (zeros == 1) {
        *e = o0 == 0 ? 0 : (o1 == 0 ? 1 : 2);
        return 1;
    }
    *vtx = o0 != 0 ? v.x : (o1 != 0 ? v.y : v.z);
    return 2;
}

// ---- Bowyer-Watson insertion on a staged region

enum BwResult : int { BW_OK = 0, BW_CLAIM = 1, BW_FULL = 2, BW_BAD = 3 };

// Stage every not-yet-staged neighbour of the cavity triangles (C) at once: claim them
// together, read them under the claims, link them to the staged triangles both ways, and
// add those in conflict with q to C.  Repeats until the cavity's boundary is staged.
__device__ __forceinline__ int bw_grow(Warp w, const Dev &d, Region &R, int p, int2 q, unsigned long long &C)
{
    WarpShared *sh = w.sh;
    int *need = sh->tmp;  // the slots to stage this round
    while (true) {
        int nneed = 0;
        for (int base = 0; base < 3 * R.cnt; base += 32) {
            int idx = base + w.lane;
            int j = idx / 3, e = idx - 3 * j;
            bool nd = idx < 3 * R.cnt && ((C >> j) & 1ull) && ic(sh->lnl[j], e) < 0;
            unsigned bm = __ballot_sync(FULL, nd);
            int pos = nneed + __popc(bm & ((1u << w.lane) - 1u));
            if (nd && pos < 64) need[pos] = ic(sh->ln[j], e) >> 2;
            nneed += __popc(bm);
        }
        if (nneed == 0) return BW_OK;
        if (nneed > 64) return BW_FULL;
        __syncwarp();
        // distinct slots, in first-seen order
        int mine = w.lane < nneed ? need[w.lane] : -1;
        int mine2 = w.lane + 32 < nneed ? need[w.lane + 32] : -1;
        bool keep = mine >= 0, keep2 = mine2 >= 0;
        for (int t = 0; t < nneed; ++t) {
            int o = need[t];
            if (t < w.lane && o == mine) keep = false;
            if (t < w.lane + 32 && o == mine2) keep2 = false;
        }
        if (mine < 0 || mine >= d.cap) keep = false;
        if (mine2 < 0 || mine2 >= d.cap) keep2 = false;
        unsigned k1 = __ballot_sync(FULL, keep), k2 = __ballot_sync(FULL, keep2);
        const int nu = __popc(k1) + __popc(k2);
        if (R.cnt + nu > LM || w.sh->ncl + nu > claim_cap(w)) return BW_FULL;
        __syncwarp();
        if (keep) need[__popc(k1 & ((1u << w.lane) - 1u))] = mine;
        if (keep2) need[__popc(k1) + __popc(k2 & ((1u << w.lane) - 1u))] = mine2;
        __syncwarp();
        if (!claim_star_list(w, d, need, nu)) return BW_CLAIM;
        // read the new triangles under their claims, then their vertices' coordinates
        const int base0 = R.cnt, cnt1 = R.cnt + nu;
        for (int i = w.lane; i < nu; i += 32) {
            int j = base0 + i, slot = need[i];
            int4 v = __ldcg(d.tv + slot), nb = __ldcg(d.tn + slot);
            sh->lslot[j] = slot;
            sh->lv[j] = v;
            sh->ln[j] = nb;
            int2 z = make_int2(0, 0);
            sh->lp[j][0] = v.x >= 0 ? __ldcg(d.xy + v.x) : z;
            sh->lp[j][1] = v.y >= 0 ? __ldcg(d.xy + v.y) : z;
            sh->lp[j][2] = v.z >= 0 ? __ldcg(d.xy + v.z) : z;
        }
        __syncwarp();
        bool bad = false;
        for (int i = w.lane; i < nu; i += 32) {
            int j = base0 + i;
            int4 nb = sh->ln[j];
            bad = bad || !(sh->lv[j].w & ALIVE);
            int lk[3] = {-1, -1, -1};
            for (int t = 0; t < cnt1; ++t) {
                int sl = sh->lslot[t];
                if (lk[0] < 0 && sl == (nb.x >> 2)) lk[0] = t;
                if (lk[1] < 0 && sl == (nb.y >> 2)) lk[1] = t;
                if (lk[2] < 0 && sl == (nb.z >> 2)) lk[2] = t;
            }
            sh->lnl[j] = make_int4(lk[0], lk[1], lk[2], 0);
            if (lk[0] >= 0) reinterpret_cast<int *>(&sh->lnl[lk[0]])[nb.x & 3] = j;
            if (lk[1] >= 0) reinterpret_cast<int *>(&sh->lnl[lk[1]])[nb.y & 3] = j;
            if (lk[2] >= 0) reinterpret_cast<int *>(&sh->lnl[lk[2]])[nb.z & 3] = j;
        }
        if (__any_sync(FULL, bad)) return BW_BAD;
        __syncwarp();
        // conflicts of the new triangles
        unsigned ex = 0, ti = 0;
        for (int base = base0; base < cnt1; base += 32) {
            int j = base + w.lane;
            bool c = false;
            if (j < cnt1) {
                int4 v = sh->lv[j];
                c = conflict(v.x, v.y, v.z, sh->lp[j][0], sh->lp[j][1], sh->lp[j][2], p, q, d.use_filter, &ex, &ti);
            }
            C |= (unsigned long long)__ballot_sync(FULL, c) << base;
        }
        cnt_add(w, C_EXACT, __reduce_add_sync(FULL, ex));
        cnt_add(w, C_TIES, __reduce_add_sync(FULL, ti));
        R.cnt = cnt1;
    }
}

// Insert p at q into the staged region by Bowyer-Watson (the insertion Section IV
// names): the cavity is every triangle whose circumcircle holds q (SoS incircle, the
// ghost rule for ghosts), tested one staged triangle per lane; it is connected and
// star-shaped from q, so staging the cavity's neighbours until none is missing gives
// its whole boundary.  q is joined to every boundary edge; the new triangles reuse the
// cavity's entries and the two dead entries X0, X1.  tj: a staged triangle holding q.
__device__ __forceinline__ int bw_insert(Warp w, const Dev &d, Region &R, int p, int2 q, int tj, int X0, int X1,
                                         int &ncav_out)
{
    WarpShared *sh = w.sh;
    unsigned long long C = 0;
    {
        unsigned ex = 0, ti = 0;
        for (int base = 0; base < R.cnt; base += 32) {
            int j = base + w.lane;
            bool c = false;
            if (j < R.cnt && sh->lslot[j] >= 0) {
                int4 v = sh->lv[j];
                c = (v.w & ALIVE) && conflict(v.x, v.y, v.z, sh->lp[j][0], sh->lp[j][1], sh->lp[j][2], p, q,
                                              d.use_filter, &ex, &ti);
            }
            C |= (unsigned long long)__ballot_sync(FULL, c) << base;
        }
        cnt_add(w, C_EXACT, __reduce_add_sync(FULL, ex));
        cnt_add(w, C_TIES, __reduce_add_sync(FULL, ti));
    }
    if (!((C >> tj) & 1ull)) return BW_BAD;  // q's triangle always conflicts
    int g = bw_grow(w, d, R, p, q, C);
    if (g != BW_OK) return g;
    const int ncav = __popcll(C);
    // boundary edges (a -> b, counter-clockwise around the cavity) into S (a), I (b),
    // L (outer staged ref), LX (coordinates of a)
    int nbd = 0;
    for (int base = 0; base < 3 * R.cnt; base += 32) {
        int idx = base + w.lane;
        int j = idx / 3, e = idx - 3 * j;
        int kn = idx < 3 * R.cnt ? ic(sh->lnl[j], e) : -1;
        bool b = idx < 3 * R.cnt && ((C >> j) & 1ull) && kn >= 0 && !((C >> kn) & 1ull);
        unsigned bm = __ballot_sync(FULL, b);
        int pos = nbd + __popc(bm & ((1u << w.lane) - 1u));
        if (b && pos < KMAX) {
            int4 v = sh->lv[j];
            int e1 = e == 2 ? 0 : e + 1, e2 = e == 0 ? 2 : e - 1;
            sh->S[pos] = ic(v, e1);
            sh->I[pos] = ic(v, e2);
            sh->L[pos] = (kn << 2) | (ic(sh->ln[j], e) & 3);
            sh->LX[pos] = sh->lp[j][e1];
        }
        nbd += __popc(bm);
    }
    if (nbd != ncav + 2 || nbd > KMAX) return BW_BAD;
    __syncwarp();
    // The cavity must be a disk seen from q: each boundary vertex starts and ends one
    // edge, and every finite boundary edge has q on its inner side.  Only a region that
    // is not Delaunay (concurrent work not yet certified) can fail this; the caller then
    // inserts by split and Lawson flips, which need no such property.  Checked for every
    // edge before anything is written.
    for (int b0 = 0; b0 < nbd; b0 += 32) {
        int b = b0 + w.lane;
        bool bad = false;
        if (b < nbd) {
            int a = sh->S[b], bb = sh->I[b], nx = -1, nnx = 0, npv = 0;
            for (int c = 0; c < nbd; ++c) {
                if (sh->S[c] == bb) {
                    nx = c;
                    ++nnx;
                }
                if (sh->I[c] == a) ++npv;
            }
            bad = nnx != 1 || npv != 1;
            if (!bad && a != KDT_GHOST && bb != KDT_GHOST) bad = orient2d(q, sh->LX[b], sh->LX[nx]) <= 0;
        }
        if (__any_sync(FULL, bad)) return BW_BAD;
    }
    // lane b joins q to boundary edge b; its neighbours are the edges that end at a
    // (previous) and start at b (next)
    unsigned long long dmask = 0, vmask = 0;
    for (int b0 = 0; b0 < nbd; b0 += 32) {
        int b = b0 + w.lane;
        int a = 0, bb = 0, ol = 0, nx = -1, pv = -1;
        int2 pa = make_int2(0, 0);
        if (b < nbd) {
            a = sh->S[b];
            bb = sh->I[b];
            ol = sh->L[b];
            pa = sh->LX[b];
            for (int c = 0; c < nbd; ++c) {
                if (sh->S[c] == bb) nx = c;
                if (sh->I[c] == a) pv = c;
            }
        }
        // staged entry of boundary edge c: the c-th cavity triangle, then X0, X1
        auto entry = [&](int c) -> int {
            if (c >= ncav) return c == ncav ? X0 : X1;
            unsigned lo = (unsigned)C, hi = (unsigned)(C >> 32);
            int nlo = __popc(lo);
            return c < nlo ? (int)__fns(lo, 0, c + 1) : 32 + (int)__fns(hi, 0, c - nlo + 1);
        };
        int x = -1, xn = -1, xp = -1;
        int2 pb = make_int2(0, 0);
        if (b < nbd) {
            x = entry(b);
            xn = entry(nx);
            xp = entry(pv);
            pb = sh->LX[nx];
        }
        int sx = b < nbd ? sh->lslot[x] : 0, sxn = b < nbd ? sh->lslot[xn] : 0, sxp = b < nbd ? sh->lslot[xp] : 0;
        __syncwarp();
        if (b < nbd) {
            sh->lv[x] = make_int4(p, a, bb, ALIVE);
            sh->lp[x][0] = q;
            sh->lp[x][1] = pa;
            sh->lp[x][2] = pb;
            set_nb(sh, x, 0, ol >> 2, gref_of(sh, ol));
            set_nb(sh, x, 1, xn, (sxn << 2) | 2);
            set_nb(sh, x, 2, xp, (sxp << 2) | 1);
            set_nb(sh, ol >> 2, ol & 3, x, (sx << 2) | 0);
            dmask |= (1ull << x) | (1ull << (ol >> 2));
            vmask |= 1ull << x;
        }
    }
    dmask |= __shfl_xor_sync(FULL, dmask, 16);
    dmask |= __shfl_xor_sync(FULL, dmask, 8);
    dmask |= __shfl_xor_sync(FULL, dmask, 4);
    dmask |= __shfl_xor_sync(FULL, dmask, 2);
    dmask |= __shfl_xor_sync(FULL, dmask, 1);
    vmask |= __shfl_xor_sync(FULL, vmask, 16);
    vmask |= __shfl_xor_sync(FULL, vmask, 8);
    vmask |= __shfl_xor_sync(FULL, vmask, 4);
    vmask |= __shfl_xor_sync(FULL, vmask, 2);
    vmask |= __shfl_xor_sync(FULL, vmask, 1);
    R.dirty |= dmask;
    R.vchg |= vmask;
    __syncwarp();
    cnt_add(w, C_INSERTS, 1);
    cnt_add(w, C_FLIPS, (unsigned)(ncav - 1));  // the Lawson flips of the same insertion
    ncav_out = ncav;
    return BW_OK;
}

// ---- features of a move for the learned proposal and its training rows
//
// For an interior p with link v_0..v_{k-1} (counter-clockwise, in L / LX):
//   j0: the one j whose half-open wedge [dir(v_j - p), dir(v_{j+1} - p)) holds the
//       move direction d = q - p (exact integer cross products); -1 if none is found;
//   feature (lane l): f0 = |d| / R, f1 = k / 16, and for r = 0..14 the link vertex
//       v_{j0+r} relative to p in the frame (u, n) of the move (u = d / |d|, n = u
//       turned a quarter counter-clockwise), divided by R = mean |v_j - p| summed in
//       the order r = 0..k-1: f[2+2r] = <v - p, u> / R, f[3+2r] = <v - p, n> / R,
//       0 for r >= k.  Every operation is a correctly rounded FP32 operation.
__device__ __forceinline__ int move_wedge(const WarpShared *sh, int k, int2 po, int2 q, int lane)
{
    long long dx = (long long)q.x - po.x, dy = (long long)q.y - po.y;
    bool hit = false;
    if (lane < k) {
        int2 a = sh->LX[lane], b = sh->LX[lane + 1 == k ? 0 : lane + 1];
        long long ax = (long long)a.x - po.x, ay = (long long)a.y - po.y;
        long long bx = (long long)b.x - po.x, by = (long long)b.y - po.y;
        hit = ax * dy - ay * dx >= 0 && dx * by - dy * bx > 0;
    }
    unsigned bm = __ballot_sync(FULL, hit);
    return __popc(bm) == 1 ? __ffs(bm) - 1 : -1;
}

__device__ __forceinline__ float move_feature(const WarpShared *sh, int k, int j0, int2 po, int2 q, int lane)
{
    float dx = __int2float_rn(q.x - po.x), dy = __int2float_rn(q.y - po.y);
    float s = __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
    float ux = __fdiv_rn(dx, s), uy = __fdiv_rn(dy, s);
    float R = 0.f;
    for (int r = 0; r < k; ++r) {
        int j = j0 + r >= k ? j0 + r - k : j0 + r;
        int2 v = sh->LX[j];
        float rx = __int2float_rn(v.x - po.x), ry = __int2float_rn(v.y - po.y);
        R = __fadd_rn(R, __fsqrt_rn(__fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry))));
    }
    R = __fdiv_rn(R, __int2float_rn(k));
    if (lane == 0) return __fdiv_rn(s, R);
    if (lane == 1) return __fdiv_rn(__int2float_rn(k), 16.0f);
    int r = (lane - 2) >> 1;
    if (r >= k) return 0.f;
    int j = j0 + r >= k ? j0 + r - k : j0 + r;
    int2 v = sh->LX[j];
    float rx = __int2float_rn(v.x - po.x), ry = __int2float_rn(v.y - po.y);
    float num = (lane & 1) == 0 ? __fadd_rn(__fmul_rn(rx, ux), __fmul_rn(ry, uy))
                                : __fsub_rn(__fmul_rn(ry, ux), __fmul_rn(rx, uy));
    return __fdiv_rn(num, R);
}

// Rank of hole triangle `lane` (< k - 2; the others get a large value): its vertices'
// rotated link indices (link position - j0 mod k, link order saved in L0) sorted
// ascending name it, and the names sorted lexicographically give the ranks.
__device__ __forceinline__ int hole_rank(const WarpShared *sh, const int *L0, int k, int j0, int lane)
{
    int key = 1 << 30;
    if (lane < k - 2) {
        int4 v = sh->lv[lane];
        int ra = 0, rb = 0, rc = 0;
        for (int i = 0; i < k; ++i) {
            int r = i - j0 < 0 ? i - j0 + k : i - j0;
            if (L0[i] == v.x) ra = r;
            if (L0[i] == v.y) rb = r;
            if (L0[i] == v.z) rc = r;
        }
        int lo = min(ra, min(rb, rc)), hi = max(ra, max(rb, rc)), mid = ra + rb + rc - lo - hi;
        key = (lo << 12) | (mid << 6) | hi;
    }
    int rank = 0;
    for (int t = 0; t < k - 2; ++t) {
        int kt = __shfl_sync(FULL, key, t);
        rank += kt < key;
    }
    return lane < k - 2 ? rank : 1 << 30;
}

// Move p to q: delete p and insert it at q in one claimed region.  On MV_GLOBAL the
// deletion is written back and the caller inserts p at q with insert_point starting
// at `hint` with the spares (s0, s1); on MV_DEFER likewise but q is still occupied by
// a point that moves later in this step.
__device__ int move_point(Warp w, const Dev &d, int p, int2 q, int &s0, int &s1, int &hint, bool may_give_up = true)
{
    WarpShared *sh = w.sh;
    int claim_fail = 0;
    for (int attempt = 0;; ++attempt) {
        if (attempt > d.retry_cap) return DEV_RETRY;
        if (read_status(d)) return MV_ABORT;
        long long t0 = clock64();
        int k = gather_star(w, d, p);
        long long t1 = clock64();
        cnt_add(w, C_CYC_GATHER, (unsigned)((t1 - t0) >> 6));
        if (k == -2 && d.big) return MV_HUGE;
        if (k == -2 && attempt == d.retry_cap) return DEV_DEGREE;
        if (k < 3 || 2 * k + 8 > LM) {
            if (k >= 3) {
                // a star too large to stage: take the plain global path (or leave the
                // whole move for later when its claims keep failing or its degree grew
                // past the shared arrays)
                int rc = delete_point(w, d, p, s0, s1, hint, may_give_up && d.big != nullptr);
                if (rc == DEL_BUSY) return MV_BIG;
                if (rc == DEL_HUGE) return MV_HUGE;
                return rc ? rc : MV_GLOBAL;
            }
            backoff(w, attempt);
            continue;
        }
        // speculative read of the star and the ring (one round trip), then claim both
        Region R;
        R.cnt = 2 * k;
        R.dirty = 0;
        R.vchg = 0;
        // (an unclaimed gather can read a neighbour word another warp holds and has not
        // finished, e.g. -1: such a slot is kept out of range and fails validation)
        bool inrange = true;
        for (int i = w.lane; i < 2 * k; i += 32) {
            int slot = i < k ? sh->S[i] : (sh->ON[i - k] >> 2);
            bool in = slot >= 0 && slot < d.cap;
            inrange = inrange && in;
            sh->lslot[i] = in ? slot : -1;
            sh->lv[i] = in ? __ldcg(d.tv + slot) : make_int4(0, 0, 0, 0);
            sh->ln[i] = in ? __ldcg(d.tn + slot) : make_int4(-1, -1, -1, 0);
        }
        __syncwarp();
        bool ok = __all_sync(FULL, inrange) && claim_list(w, d, sh->lslot, 2 * k);
        if (ok) {
            // validate under the claims and load every vertex's coordinates (one pass)
            bool good = true;
            for (int i = w.lane; i < 2 * k; i += 32) {
                int slot = sh->lslot[i];  // in range (checked above)
                int4 v = __ldcg(d.tv + slot), nb = __ldcg(d.tn + slot);
                int4 v0 = sh->lv[i], n0 = sh->ln[i];
                good = good && v.x == v0.x && v.y == v0.y && v.z == v0.z && v.w == v0.w && nb.x == n0.x &&
                       nb.y == n0.y && nb.z == n0.z && (v.w & ALIVE);
                if (i < k) {
                    int I = sh->I[i];
                    good = good && ic(v, I) == p && ic(v, (I + 1) % 3) == sh->L[i] && ic(nb, I) == sh->ON[i] &&
                           (ic(nb, (I + 1) % 3) >> 2) == sh->S[(i + 1) % k];
                }
                int2 z = make_int2(0, 0);
                sh->lp[i][0] = v.x >= 0 ? __ldcg(d.xy + v.x) : z;
                sh->lp[i][1] = v.y >= 0 ? __ldcg(d.xy + v.y) : z;
                sh->lp[i][2] = v.z >= 0 ? __ldcg(d.xy + v.z) : z;
            }
            ok = __all_sync(FULL, good);
        }
        if (!ok) {
            release_all(w, d);
            if (may_give_up && d.big && ++claim_fail >= DEFER_AFTER) return MV_BIG;
            backoff(w, attempt);
            continue;
        }
        long long t2 = clock64();
        cnt_add(w, C_CYC_CLAIM, (unsigned)((t2 - t1) >> 6));
        // a ring triangle adjacent to two link edges is staged once: later copies get
        // an unused negative slot id so that lookups find the first one
        for (int i = w.lane; i < k; i += 32) {
            int slot = sh->lslot[k + i];
            for (int j = 0; j < i; ++j)
                if (sh->lslot[k + j] == slot) sh->lslot[k + i] = -2 - i;
        }
        __syncwarp();
        // staged neighbour indices, link coordinates and outer refs of the link edges
        for (int i = w.lane; i < 2 * k; i += 32) {
            int4 nb = sh->ln[i];
            int l0 = -1, l1 = -1, l2 = -1;
            for (int t = 0; t < 2 * k; ++t) {
                int s = sh->lslot[t];
                if (l0 < 0 && s == (nb.x >> 2)) l0 = t;
                if (l1 < 0 && s == (nb.y >> 2)) l1 = t;
                if (l2 < 0 && s == (nb.z >> 2)) l2 = t;
            }
            sh->lnl[i] = make_int4(l0, l1, l2, 0);
            if (i < k) {
                int I = sh->I[i];
                sh->LX[i] = sh->lp[i][(I + 1) % 3];
                // the outer triangle of link edge i: the neighbour of star triangle i across I
                int o = I == 0 ? l0 : (I == 1 ? l1 : l2);
                sh->EO[i] = (o << 2) | (sh->ON[i] & 3);
            }
        }
        __syncwarp();
        // ---- degenerate check (as in delete_point)
        int gpos = -1;
        for (int i = 0; i < k; ++i)
            if (sh->L[i] == KDT_GHOST) gpos = i;
        if (gpos >= 0) {
            int f0 = (gpos + 1) % k, f1 = (gpos + 2) % k;
            bool col = true;
            for (int i = 0; i < k; ++i)
                if (i != gpos && orient2d(sh->LX[f0], sh->LX[f1], sh->LX[i]) != 0) col = false;
            if (col) {
                bool finite_ring = false;
                for (int i = 0; i < k; ++i) {
                    if (sh->L[i] == KDT_GHOST || sh->L[(i + 1) % k] == KDT_GHOST) continue;
                    int4 ov = sh->lv[sh->EO[i] >> 2];
                    if (ov.x != KDT_GHOST && ov.y != KDT_GHOST && ov.z != KDT_GHOST) finite_ring = true;
                }
                if (!finite_ring) {
                    release_all(w, d);
                    return DEV_DEGENERATE;
                }
            }
        }
        // ---- variants (kdt_config.variant).  1: a move that keeps every triangle of the
        // star counter-clockwise and every edge of the star (spokes p-v_i, link edges
        // v_i-v_{i+1} against the staged ring apex) locally Delaunay at q changes only
        // p's position: every other edge keeps its triangles and their vertices, so the
        // triangulation stays Delaunay (Delaunay lemma) and nothing is written.  2 (move
        // and flip): a move that keeps the star counter-clockwise also changes only p's
        // position, and the star's triangles go to the dirty list: the certification
        // that ends the step finds the star edges that stopped being Delaunay and the
        // repair (general Lawson flips) settles them.
        if (d.variant >= 1 && gpos < 0) {
            bool ccw = true, del = true;
            unsigned ex = 0, ti = 0;
            for (int i = w.lane; i < k; i += 32) {
                int i0 = i == 0 ? k - 1 : i - 1, i1 = i + 1 == k ? 0 : i + 1;
                int a = sh->L[i0], b = sh->L[i], c = sh->L[i1];
                int2 pa = sh->LX[i0], pb = sh->LX[i], pc = sh->LX[i1];
                int eo = sh->EO[i];
                int o = eo >> 2, f = eo & 3;
                int r = ic(sh->lv[o], f);
                int2 pr = sh->lp[o][f];
                const bool turn = orient2d(q, pb, pc) > 0;
                ccw = ccw && turn;
                del = del && turn && !conflict(p, a, b, q, pa, pb, c, pc, d.use_filter, &ex, &ti) &&
                      !conflict(p, b, c, q, pb, pc, r, pr, d.use_filter, &ex, &ti);
            }
            cnt_add(w, C_EXACT, __reduce_add_sync(FULL, ex));
            cnt_add(w, C_TIES, __reduce_add_sync(FULL, ti));
            ccw = __all_sync(FULL, ccw);
            del = __all_sync(FULL, del);
            if (del || (ccw && d.variant == 2)) {
                if (w.lane == 0) {
                    d.xy[p] = q;
                    __threadfence();
                }
                if (!del)
                    for (int i = w.lane; i < k; i += 32) dirty_push(d, sh->S[i]);
                __syncwarp();
                release_all(w, d);
                cnt_add(w, C_CYC_LOCAL, (unsigned)((clock64() - t2) >> 6));
                return MV_DONE;
            }
        }
        // ---- learned proposal / training rows: the move's features (interior p only);
        // the link order is kept in I for the hole ranks (I is not needed any more)
        const bool learn = (d.mlp != nullptr || d.trace_x != nullptr) && gpos < 0;
        float feat = 0.f;
        int j0 = -1;
        if (learn) {
            int2 po = sh->lp[0][sh->I[0]];  // p's position before the move
            j0 = move_wedge(sh, k, po, q, w.lane);
            // the features feed a training row, or the network when the planner did not
            // evaluate it for this step
            if (j0 >= 0 && (d.trace_x || !d.pguess)) feat = move_feature(sh, k, j0, po, q, w.lane);
            __syncwarp();
            for (int i = w.lane; i < k; i += 32) sh->I[i] = sh->L[i];
            __syncwarp();
        }
        // ---- 1. delete p: Delaunay ears over the link, into the star's staged entries
        long long te0 = clock64();
        int m = k, newc = 0;
        while (m > 3) {
            // Every (ear i, test t) pair on its own lane: t = 0 is the ear's orientation,
            // t >= 1 the conflict of vertex i+2+t with the ear (SoS incircle, or the
            // ghost rule for an ear through infinity).
            const unsigned allm = m == 32 ? FULL : ((1u << m) - 1u);
            if (w.lane == 0) sh->earbad = 0u;
            __syncwarp();
            unsigned ex = 0, ti = 0;
            const int npair = m * (m - 2);
            for (int base = 0; base < npair; base += 32) {
                int idx = base + w.lane;
                if (idx < npair) {
                    int i = idx / (m - 2), t = idx - i * (m - 2);
                    if (ear_test_fails(sh->L, sh->LX, m, i, t, d, &ex, &ti)) atomicOr(&sh->earbad, 1u << i);
                }
            }
            __syncwarp();
            unsigned good = ~sh->earbad & allm;
            cnt_add(w, C_EXACT, __reduce_add_sync(FULL, ex));
            cnt_add(w, C_TIES, __reduce_add_sync(FULL, ti));
            if (!good) {
                release_all(w, d);
                return DEV_INTERNAL;
            }
            // Clip every valid ear no neighbour of which is clipped too (each valid ear is
            // a triangle of the hole's unique triangulation), keeping 3 vertices or more.
            unsigned sel = 0;
            int ns = 0;
            for (int i = 0; i < m && ns < m - 3; ++i) {
                if (!((good >> i) & 1u)) continue;
                int ip = i == 0 ? m - 1 : i - 1;
                if ((sel >> ip) & 1u) continue;
                if (i == m - 1 && (sel & 1u)) continue;
                sel |= 1u << i;
                ++ns;
            }
            // lane r builds the r-th clipped ear into staged entry newc + r
            unsigned long long dmask = 0, vmask = 0;
            {
                int r = w.lane, i = -1;
                int X = newc + r, eo_i = 0, eo_i1 = 0, Li = 0, Li1 = 0, Li2 = 0, sX = 0;
                int2 Xi = make_int2(0, 0), Xi1 = Xi, Xi2 = Xi;
                if (r < ns) {
                    i = (int)__fns(sel, 0, r + 1);
                    int i1 = i + 1 == m ? 0 : i + 1, i2 = i1 + 1 == m ? 0 : i1 + 1;
                    eo_i = sh->EO[i];
                    eo_i1 = sh->EO[i1];
                    Li = sh->L[i];
                    Li1 = sh->L[i1];
                    Li2 = sh->L[i2];
                    Xi = sh->LX[i];
                    Xi1 = sh->LX[i1];
                    Xi2 = sh->LX[i2];
                    sX = sh->lslot[X];
                }
                __syncwarp();  // every lane has read before any lane writes
                if (r < ns) {
                    sh->lv[X] = make_int4(Li, Li1, Li2, ALIVE);
                    sh->lp[X][0] = Xi;
                    sh->lp[X][1] = Xi1;
                    sh->lp[X][2] = Xi2;
                    set_nb(sh, X, 0, eo_i1 >> 2, gref_of(sh, eo_i1));
                    set_nb(sh, X, 1, -1, -1);  // the new diagonal: set when it is consumed
                    set_nb(sh, X, 2, eo_i >> 2, gref_of(sh, eo_i));
                    set_nb(sh, eo_i1 >> 2, eo_i1 & 3, X, (sX << 2) | 0);
                    set_nb(sh, eo_i >> 2, eo_i & 3, X, (sX << 2) | 2);
                    sh->EO[i] = (X << 2) | 1;
                    dmask = (1ull << X) | (1ull << (eo_i >> 2)) | (1ull << (eo_i1 >> 2));
                    vmask = 1ull << X;
                }
            }
            dmask |= __shfl_xor_sync(FULL, dmask, 16);
            dmask |= __shfl_xor_sync(FULL, dmask, 8);
            dmask |= __shfl_xor_sync(FULL, dmask, 4);
            dmask |= __shfl_xor_sync(FULL, dmask, 2);
            dmask |= __shfl_xor_sync(FULL, dmask, 1);
            vmask |= __shfl_xor_sync(FULL, vmask, 16);
            vmask |= __shfl_xor_sync(FULL, vmask, 8);
            vmask |= __shfl_xor_sync(FULL, vmask, 4);
            vmask |= __shfl_xor_sync(FULL, vmask, 2);
            vmask |= __shfl_xor_sync(FULL, vmask, 1);
            R.dirty |= dmask;
            R.vchg |= vmask;
            __syncwarp();
            // drop the clipped ears' middle vertices from the link
            {
                unsigned removed = ((sel << 1) | (sel >> (m - 1))) & allm;
                int j = w.lane;
                bool keep = j < m && !((removed >> j) & 1u);
                int nj = j - __popc(removed & ((1u << j) - 1u));
                int lv = 0, eov = 0;
                int2 xv = make_int2(0, 0);
                if (keep) {
                    lv = sh->L[j];
                    eov = sh->EO[j];
                    xv = sh->LX[j];
                }
                __syncwarp();
                if (keep) {
                    sh->L[nj] = lv;
                    sh->EO[nj] = eov;
                    sh->LX[nj] = xv;
                }
                __syncwarp();
            }
            m -= ns;
            newc += ns;
        }
        {
            int X = newc++;
            int e0 = sh->EO[0], e1 = sh->EO[1], e2 = sh->EO[2];
            int L0 = sh->L[0], L1 = sh->L[1], L2 = sh->L[2];
            int2 P0 = sh->LX[0], P1 = sh->LX[1], P2 = sh->LX[2];
            int sX = sh->lslot[X];
            __syncwarp();
            sh->lv[X] = make_int4(L0, L1, L2, ALIVE);
            sh->lp[X][0] = P0;
            sh->lp[X][1] = P1;
            sh->lp[X][2] = P2;
            set_nb(sh, X, 0, e1 >> 2, gref_of(sh, e1));
            set_nb(sh, X, 1, e2 >> 2, gref_of(sh, e2));
            set_nb(sh, X, 2, e0 >> 2, gref_of(sh, e0));
            set_nb(sh, e1 >> 2, e1 & 3, X, (sX << 2) | 0);
            set_nb(sh, e2 >> 2, e2 & 3, X, (sX << 2) | 1);
            set_nb(sh, e0 >> 2, e0 & 3, X, (sX << 2) | 2);
            R.dirty |= (1ull << X) | (1ull << (e0 >> 2)) | (1ull << (e1 >> 2)) | (1ull << (e2 >> 2));
            R.vchg |= 1ull << X;
        }
        // spares: staged entries k-2, k-1 (dead)
        const int X0 = k - 2, X1 = k - 1;
        sh->lv[X0] = make_int4(0, 0, 0, 0);
        sh->lv[X1] = make_int4(0, 0, 0, 0);
        sh->lnl[X0] = make_int4(-1, -1, -1, 0);
        sh->lnl[X1] = make_int4(-1, -1, -1, 0);
        if (w.lane == 0) d.pt_tri[p] = -1;
        R.dirty |= (1ull << X0) | (1ull << X1);
        cnt_add(w, C_DEG_DEL, k);
        cnt_add(w, C_DELETES, 1);
        s0 = sh->lslot[X0];
        s1 = sh->lslot[X1];
        hint = sh->lslot[0];
        cnt_add(w, C_CYC_EAR, (unsigned)((clock64() - te0) >> 6));
        // Update (Fig. 4): p takes its new position
        if (w.lane == 0) d.xy[p] = q;
        __syncwarp();
        // ---- 2. locate q among the staged triangles (first the proposed one)
        int where = -1, tvtx = -1, tj = -1;
        int rank = 1 << 30, slot = MLP_BEYOND;
        if (learn && j0 >= 0) {
            rank = hole_rank(sh, sh->I, k, j0, w.lane);
            int e = 0, vt = -1;
            int r = w.lane < k - 2 ? locate_in(sh, w.lane, q, &e, &vt) : -1;
            // training label: the lowest-ranked hole triangle holding q (closed)
            int lab = (r == 0 || r == 1) ? rank : 1 << 30;
#pragma unroll
            for (int off = 16; off; off >>= 1) lab = min(lab, __shfl_xor_sync(FULL, lab, off));
            slot = lab < MLP_BEYOND ? lab : MLP_BEYOND;
            if (d.mlp) {
                int guess = d.pguess ? (int)__ldcg(d.pguess + p)
                                     : mlp_argmax_slot(mlp_warp_forward(d.mlp, feat, w.lane), w.lane);
                cnt_add(w, C_PROP_MOVES, 1);
                unsigned bm = __ballot_sync(FULL, guess < MLP_BEYOND && rank == guess && (r == 0 || r == 1));
                if (bm) {
                    int src = __ffs(bm) - 1;
                    tj = src;
                    where = __shfl_sync(FULL, r, src);
                    cnt_add(w, C_PROP_HITS, 1);
                }
            }
        }
        for (int base = 0; base < R.cnt && tj < 0; base += 32) {
            int j = base + w.lane;
            int e = 0, vt = -1;
            int r = j < R.cnt && sh->lslot[j] >= 0 ? locate_in(sh, j, q, &e, &vt) : -1;
            // a finite hit; a ghost hit (outside the hull) goes to the global path
            unsigned bm = __ballot_sync(FULL, r >= 0 && r <= 2);
            if (bm) {
                int src = __ffs(bm) - 1;
                tj = base + src;
                where = __shfl_sync(FULL, r, src);
                tvtx = __shfl_sync(FULL, vt, src);
            }
        }
        if (tj < 0) {
            // not in the staged region (or outside the hull): finish on the global path
            write_back(w, d, R);
            return MV_GLOBAL;
        }
        if (where == 2) {
            write_back(w, d, R);
            int st = __shfl_sync(FULL, __ldcg(d.pt_stamp + tvtx), 0);
            if (st == d.stamp) return MV_DEFER;
            return DEV_DUPLICATE;
        }
        // ---- 3. Bowyer-Watson insertion of q (Section IV names it for insertion)
        long long tl0 = clock64();
        int ncav = 0;
        int bw = bw_insert(w, d, R, p, q, tj, X0, X1, ncav);
        if (bw != BW_OK) {
            // the deletion is written; the insertion continues on the global path
            write_back(w, d, R);
            return MV_GLOBAL;
        }
        if (learn && j0 >= 0 && d.trace_x) {
            int row = 0;
            if (w.lane == 0) row = atomicAdd(d.trace_count, 1);
            row = __shfl_sync(FULL, row, 0);
            if (row < d.trace_cap) {
                d.trace_x[(long long)row * MLP_IN + w.lane] = feat;
                if (w.lane == 0) {
                    d.trace_y[2ll * row] = slot;
                    d.trace_y[2ll * row + 1] = ncav;
                }
                cnt_add(w, C_TRACE_ROWS, 1);
            }
        }
        if (where == 1) cnt_add(w, C_SPLIT_EDGE, 1);
        cnt_add(w, C_CYC_LAWSON, (unsigned)((clock64() - tl0) >> 6));
        const int left = 0;
        long long tc0 = clock64();
        bool certified = left == 0 && certify_staged(w, d, R);
        cnt_add(w, C_CYC_CERT, (unsigned)((clock64() - tc0) >> 6));
        long long t3 = clock64();
        cnt_add(w, C_CYC_LOCAL, (unsigned)((t3 - t2) >> 6));
        write_back(w, d, R, certified);
        cnt_add(w, C_CYC_WB, (unsigned)((clock64() - t3) >> 6));
        return MV_DONE;
    }
}

}  // namespace kd

namespace kd {

// Insert p (xy[p] already holds q) by Bowyer-Watson on a staged region: a walk finds
// a triangle holding q; it and the two spare slots are claimed and staged, the cavity
// is grown and replaced as in the staged move, certified on the staged copy and
// written back.  spare0 / spare1: two dead slots the caller owns (a deletion's
// leftovers, or fresh slots during a build).  Returns 0, INS_DEFER (q lies on a
// vertex that is still moving in this step), INS_GLOBAL (the cavity outgrew a staged
// region, or the region is not Delaunay: the caller uses the global-memory
// insertion), or a DevStatus error.
__device__ __noinline__ int insert_staged(Warp w, const Dev &d, int p, int2 q, int start, int spare0, int spare1,
                                          bool allow_defer)
{
    WarpShared *sh = w.sh;
    if (spare0 < 0 || spare0 >= d.cap || spare1 < 0 || spare1 >= d.cap) return DEV_INTERNAL;
    int t = start, walk_fail = 0, cavity_fail = 0;
    for (int attempt = 0;; ++attempt) {
        if (attempt > d.retry_cap) return DEV_RETRY;
        if (read_status(d)) return -1;
        WalkResult wr = walk(w, d, t, q);
        if (wr.t < 0) {
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
        if (wr.where == W_VERTEX) {
            int st = __shfl_sync(FULL, __ldcg(d.pt_stamp + wr.vtx), 0);
            if (allow_defer && st == d.stamp) return INS_DEFER;
            return DEV_DUPLICATE;
        }
        // claim the triangle and the spares; read the triangle under its claim
        if (w.lane == 0) {
            sh->tmp[0] = wr.t;
            sh->tmp[1] = spare0;
            sh->tmp[2] = spare1;
        }
        __syncwarp();
        bool ok = claim_star_list(w, d, sh->tmp, 3);
        Region R;
        R.cnt = 3;
        R.dirty = (1ull << 1) | (1ull << 2);
        R.vchg = 0;
        if (ok) {
            if (w.lane < 3) {
                int slot = sh->tmp[w.lane];
                int4 v = make_int4(0, 0, 0, 0), nb = make_int4(-1, -1, -1, 0);
                int2 z = make_int2(0, 0), p0 = z, p1 = z, p2 = z;
                if (w.lane == 0) {
                    v = __ldcg(d.tv + slot);
                    nb = __ldcg(d.tn + slot);
                    p0 = v.x >= 0 ? __ldcg(d.xy + v.x) : z;
                    p1 = v.y >= 0 ? __ldcg(d.xy + v.y) : z;
                    p2 = v.z >= 0 ? __ldcg(d.xy + v.z) : z;
                }
                sh->lslot[w.lane] = slot;
                sh->lv[w.lane] = v;
                sh->ln[w.lane] = nb;
                sh->lnl[w.lane] = make_int4(-1, -1, -1, 0);
                sh->lp[w.lane][0] = p0;
                sh->lp[w.lane][1] = p1;
                sh->lp[w.lane][2] = p2;
            }
            __syncwarp();
            // it must still hold q (a finite triangle) or see q outside its hull edge
            int e = 0, vt = -1;
            int r = locate_in(sh, 0, q, &e, &vt);
            ok = r == 0 || r == 1 || r == 3;
        }
        if (!ok) {
            release_all(w, d);
            backoff(w, attempt);
            t = wr.t;
            continue;
        }
        int ncav = 0;
        int bw = bw_insert(w, d, R, p, q, 0, 1, 2, ncav);
        if (bw == BW_FULL || bw == BW_BAD) {
            release_all(w, d);
            return INS_GLOBAL;
        }
        if (bw != BW_OK) {
            // a cavity claim lost a race.  A large cavity (a point beside long, thin
            // triangles whose circles are huge) overlaps many other operations and can
            // keep losing; after a few losses the insertion by split and Lawson flips,
            // which claims a few triangles at a time, takes over.
            release_all(w, d);
            if (++cavity_fail >= (allow_defer ? 4 : 32)) return INS_GLOBAL;  // (4 during a step)
            backoff(w, attempt);
            t = wr.t;
            continue;
        }
        if (wr.where == W_EDGE) cnt_add(w, C_SPLIT_EDGE, 1);
        if (wr.where == W_GHOST) cnt_add(w, C_SPLIT_GHOST, 1);
        bool certified = certify_staged(w, d, R);
        write_back(w, d, R, certified);
        return 0;
    }
}

}  // namespace kd
