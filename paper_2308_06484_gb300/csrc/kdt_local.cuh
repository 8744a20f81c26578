// Fused kinetic move of one point in a claimed, shared-memory staged region.
//
// The paper's per-block update (Fig. 4: Update, Delete, Insert; Section IV) touches
// the star of the moved point p and, for a short move, the star of its new position
// q, which overlaps it.  This operation claims p's star and the ring of triangles
// around it in one batch, copies them into the warp's shared memory (vertices,
// neighbours as global refs and as staged indices, and the coordinates of every
// vertex, so no lookup is needed later), and there
//   1. deletes p by Delaunay ears (the simple deletion Section IV prefers),
//   2. locates q among the staged triangles,
//   3. splits the containing triangle (1->3, or 2->4 when q is on an edge),
//   4. runs the Lawson flips of the edges opposite q with the flip stack in shared
//      memory, claiming and staging further triangles only when a flip reaches
//      outside the region,
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

namespace kd {

// outcome of move_point
enum MoveResult : int { MV_DONE = 0, MV_DEFER = 1, MV_GLOBAL = 2, MV_ABORT = -1 };

struct Region {
    int cnt;                   // staged triangles
    unsigned long long dirty;  // modified staged triangles
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
__device__ __noinline__ int ensure_local(Warp &w, const Dev &d, Region &R, int slot)
{
    WarpShared *sh = w.sh;
    int j = local_find(sh, R.cnt, slot);
    if (j >= 0) return j;
    if (R.cnt >= LM || w.ncl >= MAXC || slot < 0 || slot >= d.cap) return -1;
    int mine = w.lane == 0 ? slot : -1;
    if (!claim_lanes(w, d, mine, 1)) return -1;
    int4 v, nb;
    load_tri(w, d, slot, v, nb);
    if (!(v.w & ALIVE)) return -1;
    int2 p0, p1, p2, pz;
    load_xy4(w, d, v.x, v.y, v.z, KDT_GHOST, p0, p1, p2, pz);
    j = R.cnt++;
    sh->lslot[j] = slot;
    sh->lv[j] = v;
    sh->ln[j] = nb;
    sh->lp[j][0] = p0;
    sh->lp[j][1] = p1;
    sh->lp[j][2] = p2;
    for (int e = 0; e < 3; ++e) {
        int r = ic(nb, e);
        int k = local_find(sh, R.cnt, r >> 2);
        reinterpret_cast<int *>(&sh->lnl[j])[e] = k;
        if (k >= 0) reinterpret_cast<int *>(&sh->lnl[k])[r & 3] = j;
    }
    __syncwarp();
    return j;
}

// make sure the neighbour of staged j across edge e is staged; its staged index or -1
__device__ __forceinline__ int nb_staged(Warp &w, const Dev &d, Region &R, int j, int e)
{
    int k = ic(w.sh->lnl[j], e);
    if (k >= 0) return k;
    return ensure_local(w, d, R, ic(w.sh->ln[j], e) >> 2);
}

// Write every modified staged triangle back (lane-parallel), update pt_tri of their
// vertices, release all claims, then certify the written triangles.
__device__ void write_back(Warp &w, const Dev &d, Region &R)
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
    R.dirty = 0;
    release_all(w, d);
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

// Staged fan around q: triangles (q, W[k], W[k+1]) into staged entries X[k]; OL[k] is
// the staged ref (index << 2 | edge) of the outer neighbour across (W[k], W[k+1]).
__device__ void local_fan(WarpShared *sh, Region &R, int q, int2 pq, const int *W, const int2 *WX,
                          const int *OL, const int *X, int m)
{
    for (int k = 0; k < m; ++k) {
        int kn = k + 1 == m ? 0 : k + 1, kp = k == 0 ? m - 1 : k - 1;
        int x = X[k], o = OL[k];
        sh->lv[x] = make_int4(q, W[k], W[kn], ALIVE);
        sh->lp[x][0] = pq;
        sh->lp[x][1] = WX[k];
        sh->lp[x][2] = WX[kn];
        set_nb(sh, x, 0, o >> 2, gref_of(sh, o));
        set_nb(sh, x, 1, X[kn], (sh->lslot[X[kn]] << 2) | 2);
        set_nb(sh, x, 2, X[kp], (sh->lslot[X[kp]] << 2) | 1);
        set_nb(sh, o >> 2, o & 3, x, (sh->lslot[x] << 2) | 0);
        R.dirty |= (1ull << x) | (1ull << (o >> 2));
    }
}

// Lawson flips of the edges opposite p on the staged region (stack entries: staged
// index, edge).  Triangles a flip needs beyond the region are claimed and staged; if
// that fails, the remaining stack is handed back with *top_out > 0.
__device__ void local_lawson(Warp &w, const Dev &d, Region &R, int p, int top, int *top_out)
{
    WarpShared *sh = w.sh;
    while (top > 0) {
        int2 ent = sh->stack[top - 1];
        --top;
        int T = ent.x, e = ent.y;
        int4 v = sh->lv[T];
        if (!(v.w & ALIVE) || ic(v, e) != p) continue;
        int U = nb_staged(w, d, R, T, e);
        if (U < 0) {
            __syncwarp();
            sh->stack[top] = ent;
            *top_out = top + 1;
            return;
        }
        int f = ic(sh->ln[T], e) & 3;
        int4 uv = sh->lv[U];
        int e1 = e == 2 ? 0 : e + 1, e2 = e == 0 ? 2 : e - 1;
        int f1 = f == 2 ? 0 : f + 1, f2 = f == 0 ? 2 : f - 1;
        int a = ic(v, e1), b = ic(v, e2), dd = ic(uv, f);
        int2 pp = sh->lp[T][e], pa = sh->lp[T][e1], pb = sh->lp[T][e2], pd = sh->lp[U][f];
        w.cnt[C_FLIP_TESTS]++;
        // the test is on the triangle in its stored rotation
        int2 q0 = sh->lp[T][0], q1 = sh->lp[T][1], q2 = sh->lp[T][2];
        if (!conflict(v.x, v.y, v.z, q0, q1, q2, dd, pd, d.use_filter, &w.cnt[C_EXACT], &w.cnt[C_TIES]))
            continue;
        // the four outer neighbours get new back-pointers: stage them
        int Ta = nb_staged(w, d, R, T, e1), Tb = nb_staged(w, d, R, T, e2);
        int Ub = Ta >= 0 && Tb >= 0 ? nb_staged(w, d, R, U, f1) : -1;
        int Ua = Ub >= 0 ? nb_staged(w, d, R, U, f2) : -1;
        if (Ua < 0) {
            __syncwarp();
            sh->stack[top] = ent;
            *top_out = top + 1;
            return;
        }
        int ga = ic(sh->ln[T], e1), gb = ic(sh->ln[T], e2);    // nt_a, nt_b
        int hb = ic(sh->ln[U], f1), ha = ic(sh->ln[U], f2);    // nu_b, nu_a
        int sT = sh->lslot[T], sU = sh->lslot[U];
        __syncwarp();  // every lane has read T, U and the entry before any lane writes
        // T = (p, a, d), U = (p, d, b)
        sh->lv[T] = make_int4(p, a, dd, ALIVE);
        sh->lp[T][0] = pp;
        sh->lp[T][1] = pa;
        sh->lp[T][2] = pd;
        sh->lv[U] = make_int4(p, dd, b, ALIVE);
        sh->lp[U][0] = pp;
        sh->lp[U][1] = pd;
        sh->lp[U][2] = pb;
        set_nb(sh, T, 0, Ub, hb);
        set_nb(sh, T, 1, U, (sU << 2) | 2);
        set_nb(sh, T, 2, Tb, gb);
        set_nb(sh, U, 0, Ua, ha);
        set_nb(sh, U, 1, Ta, ga);
        set_nb(sh, U, 2, T, (sT << 2) | 1);
        set_nb(sh, Ub, hb & 3, T, (sT << 2) | 0);
        set_nb(sh, Tb, gb & 3, T, (sT << 2) | 2);
        set_nb(sh, Ua, ha & 3, U, (sU << 2) | 0);
        set_nb(sh, Ta, ga & 3, U, (sU << 2) | 1);
        R.dirty |= (1ull << T) | (1ull << U) | (1ull << Ta) | (1ull << Tb) | (1ull << Ua) | (1ull << Ub);
        w.cnt[C_FLIPS]++;
        if (top + 2 > STACK) {
            w.cnt[C_STACK_DROP]++;
            continue;
        }
        sh->stack[top] = make_int2(T, 0);
        sh->stack[top + 1] = make_int2(U, 0);
        top += 2;
    }
    *top_out = 0;
}

// Move p to q: delete p and insert it at q in one claimed region.  On MV_GLOBAL the
// deletion is written back and the caller inserts p at q with insert_point starting
// at `hint` with the spares (s0, s1); on MV_DEFER likewise but q is still occupied by
// a point that moves later in this step.
__device__ int move_point(Warp &w, const Dev &d, int p, int2 q, int &s0, int &s1, int &hint)
{
    WarpShared *sh = w.sh;
    for (int attempt = 0;; ++attempt) {
        if (attempt > d.retry_cap) return DEV_RETRY;
        if (read_status(d)) return MV_ABORT;
        long long t0 = clock64();
        int k = gather_star(w, d, p);
        long long t1 = clock64();
        w.cnt[C_CYC_GATHER] += (unsigned)((t1 - t0) >> 6);
        if (k == -2 && attempt == d.retry_cap) return DEV_DEGREE;
        if (k < 3 || 2 * k + 8 > LM) {
            if (k >= 3) {
                // a star too large to stage: take the plain global path
                int rc = delete_point(w, d, p, s0, s1, hint);
                return rc ? rc : MV_GLOBAL;
            }
            backoff(w, attempt);
            continue;
        }
        // speculative read of the star and the ring (one round trip), then claim both
        Region R;
        R.cnt = 2 * k;
        R.dirty = 0;
        for (int i = w.lane; i < 2 * k; i += 32) {
            int slot = i < k ? sh->S[i] : (sh->ON[i - k] >> 2);
            sh->lslot[i] = slot;
            sh->lv[i] = __ldcg(d.tv + slot);
            sh->ln[i] = __ldcg(d.tn + slot);
        }
        __syncwarp();
        bool ok = claim_list(w, d, sh->lslot, 2 * k);
        if (ok) {
            // validate under the claims and load every vertex's coordinates (one pass)
            bool good = true;
            for (int i = w.lane; i < 2 * k; i += 32) {
                int slot = sh->lslot[i];
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
            backoff(w, attempt);
            continue;
        }
        long long t2 = clock64();
        w.cnt[C_CYC_CLAIM] += (unsigned)((t2 - t1) >> 6);
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
        // ---- 1. delete p: Delaunay ears over the link, into the star's staged entries
        int m = k, newc = 0;
        while (m > 3) {
            int chosen = -1;
            unsigned ex = 0, ti = 0;
            for (int base = 0; base < m && chosen < 0; base += 32) {
                int i = base + w.lane;
                bool v = i < m && ear_valid(sh->L, sh->LX, m, i, d, &ex, &ti);
                unsigned bm = __ballot_sync(FULL, v);
                if (bm) chosen = base + __ffs(bm) - 1;
            }
            w.cnt[C_EXACT] += __reduce_add_sync(FULL, ex);
            w.cnt[C_TIES] += __reduce_add_sync(FULL, ti);
            if (chosen < 0) {
                release_all(w, d);
                return DEV_INTERNAL;
            }
            int i = chosen, i1 = i + 1 == m ? 0 : i + 1, i2 = i1 + 1 == m ? 0 : i1 + 1;
            int X = newc++;  // staged index == star position
            int eo_i = sh->EO[i], eo_i1 = sh->EO[i1];
            int Li = sh->L[i], Li1 = sh->L[i1], Li2 = sh->L[i2];
            int2 Xi = sh->LX[i], Xi1 = sh->LX[i1], Xi2 = sh->LX[i2];
            int sX = sh->lslot[X];
            __syncwarp();  // every lane has read before any lane writes
            sh->lv[X] = make_int4(Li, Li1, Li2, ALIVE);
            sh->lp[X][0] = Xi;
            sh->lp[X][1] = Xi1;
            sh->lp[X][2] = Xi2;
            set_nb(sh, X, 0, eo_i1 >> 2, gref_of(sh, eo_i1));
            set_nb(sh, X, 1, -1, -1);  // the new diagonal: set when it is consumed
            set_nb(sh, X, 2, eo_i >> 2, gref_of(sh, eo_i));
            set_nb(sh, eo_i1 >> 2, eo_i1 & 3, X, (sX << 2) | 0);
            set_nb(sh, eo_i >> 2, eo_i & 3, X, (sX << 2) | 2);
            R.dirty |= (1ull << X) | (1ull << (eo_i >> 2)) | (1ull << (eo_i1 >> 2));
            sh->EO[i] = (X << 2) | 1;
            __syncwarp();
            // remove element i1 (shift the tail down by one)
            int lv = 0, eov = 0;
            int2 xv = make_int2(0, 0);
            int j = w.lane;
            bool mv = j >= i1 && j < m - 1;
            if (mv) {
                lv = sh->L[j + 1];
                eov = sh->EO[j + 1];
                xv = sh->LX[j + 1];
            }
            bool mv2 = j + 32 >= i1 && j + 32 < m - 1;
            int lv2 = 0, eov2 = 0;
            int2 xv2 = make_int2(0, 0);
            if (mv2) {
                lv2 = sh->L[j + 33];
                eov2 = sh->EO[j + 33];
                xv2 = sh->LX[j + 33];
            }
            __syncwarp();
            if (mv) {
                sh->L[j] = lv;
                sh->EO[j] = eov;
                sh->LX[j] = xv;
            }
            if (mv2) {
                sh->L[j + 32] = lv2;
                sh->EO[j + 32] = eov2;
                sh->LX[j + 32] = xv2;
            }
            __syncwarp();
            --m;
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
        }
        // spares: staged entries k-2, k-1 (dead)
        const int X0 = k - 2, X1 = k - 1;
        sh->lv[X0] = make_int4(0, 0, 0, 0);
        sh->lv[X1] = make_int4(0, 0, 0, 0);
        sh->lnl[X0] = make_int4(-1, -1, -1, 0);
        sh->lnl[X1] = make_int4(-1, -1, -1, 0);
        if (w.lane == 0) d.pt_tri[p] = -1;
        R.dirty |= (1ull << X0) | (1ull << X1);
        w.cnt[C_DEG_DEL] += k;
        w.cnt[C_DELETES]++;
        s0 = sh->lslot[X0];
        s1 = sh->lslot[X1];
        hint = sh->lslot[0];
        // Update (Fig. 4): p takes its new position
        if (w.lane == 0) d.xy[p] = q;
        __syncwarp();
        // ---- 2. locate q among the staged triangles
        int where = -1, te = 0, tvtx = -1, tj = -1;
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
                te = __shfl_sync(FULL, e, src);
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
        // ---- 3. split (staged); every triangle whose refs change must be staged
        int4 v = sh->lv[tj];
        int *W = sh->tmp, *OL = sh->tmp + 8, *Xs = sh->tmp + 16;
        int2 *WX = reinterpret_cast<int2 *>(sh->tmp + 24);
        int mf;
        bool okf;
        if (where == 1) {
            int e = te, e1 = (e + 1) % 3, e2 = (e + 2) % 3;
            int Uj = nb_staged(w, d, R, tj, e);
            int f = ic(sh->ln[tj], e) & 3, f1 = (f + 1) % 3, f2 = (f + 2) % 3;
            okf = Uj >= 0 && nb_staged(w, d, R, tj, e1) >= 0 && nb_staged(w, d, R, tj, e2) >= 0 &&
                  nb_staged(w, d, R, Uj, f1) >= 0 && nb_staged(w, d, R, Uj, f2) >= 0;
            if (okf) {
                int4 uv = sh->lv[Uj];
                W[0] = ic(v, e);  WX[0] = sh->lp[tj][e];
                W[1] = ic(v, e1); WX[1] = sh->lp[tj][e1];
                W[2] = ic(uv, f); WX[2] = sh->lp[Uj][f];
                W[3] = ic(v, e2); WX[3] = sh->lp[tj][e2];
                // outer staged refs: (a,b) t opp c; (b,d) u opp c; (d,c) u opp b; (c,a) t opp b
                OL[0] = (ic(sh->lnl[tj], e2) << 2) | (ic(sh->ln[tj], e2) & 3);
                OL[1] = (ic(sh->lnl[Uj], f1) << 2) | (ic(sh->ln[Uj], f1) & 3);
                OL[2] = (ic(sh->lnl[Uj], f2) << 2) | (ic(sh->ln[Uj], f2) & 3);
                OL[3] = (ic(sh->lnl[tj], e1) << 2) | (ic(sh->ln[tj], e1) & 3);
                Xs[0] = tj; Xs[1] = Uj; Xs[2] = X0; Xs[3] = X1;
                w.cnt[C_SPLIT_EDGE]++;
            }
            mf = 4;
        } else {
            okf = nb_staged(w, d, R, tj, 0) >= 0 && nb_staged(w, d, R, tj, 1) >= 0 &&
                  nb_staged(w, d, R, tj, 2) >= 0;
            if (okf) {
                W[0] = v.x; W[1] = v.y; W[2] = v.z;
                WX[0] = sh->lp[tj][0]; WX[1] = sh->lp[tj][1]; WX[2] = sh->lp[tj][2];
                OL[0] = (sh->lnl[tj].z << 2) | (sh->ln[tj].z & 3);
                OL[1] = (sh->lnl[tj].x << 2) | (sh->ln[tj].x & 3);
                OL[2] = (sh->lnl[tj].y << 2) | (sh->ln[tj].y & 3);
                Xs[0] = tj; Xs[1] = X0; Xs[2] = X1;
            }
            mf = 3;
        }
        if (!okf) {
            write_back(w, d, R);
            return MV_GLOBAL;
        }
        local_fan(sh, R, p, q, W, WX, OL, Xs, mf);
        w.cnt[C_INSERTS]++;
        // ---- 4. Lawson flips of the edges opposite q
        __syncwarp();
        for (int j = 0; j < mf; ++j) sh->stack[j] = make_int2(Xs[j], 0);
        int left = 0;
        local_lawson(w, d, R, p, mf, &left);
        // convert what is left to global (slot, edge) entries before the region goes
        __syncwarp();
        for (int j = w.lane; j < left; j += 32) {
            int2 en = sh->stack[j];
            sh->stack[j] = make_int2(sh->lslot[en.x], en.y);
        }
        __syncwarp();
        long long t3 = clock64();
        w.cnt[C_CYC_LOCAL] += (unsigned)((t3 - t2) >> 6);
        write_back(w, d, R);
        w.cnt[C_CYC_WB] += (unsigned)((clock64() - t3) >> 6);
        if (left > 0) lawson(w, d, left, p, true);
        return MV_DONE;
    }
}

}  // namespace kd
