// Fused kinetic move of one point in a claimed, shared-memory staged region.
//
// The paper's per-block update (Fig. 4: Update, Delete, Insert; Section IV) touches
// the star of the moved point p and, for a short move, the star of its new position
// q, which overlaps it.  This operation claims p's star and the ring of triangles
// around it in one batch, copies them (and their vertices' coordinates) into the
// warp's shared memory, and there
//   1. deletes p by Delaunay ears (the simple deletion Section IV prefers),
//   2. locates q among the staged triangles,
//   3. splits the containing triangle (1->3, or 2->4 when q is on an edge),
//   4. runs the Lawson flips of the edges opposite q, claiming and staging further
//      triangles only when a flip reaches outside the region,
// then writes every modified triangle back and releases the claims.  Global memory
// sees one claim batch, one validation pass and one write-back instead of a round
// trip per ear and per flip.  When q is not inside the staged region (a long move,
// a move outside the hull) or a claim needed later fails, the work done so far is
// written back (a valid triangulation) and the caller continues on the global path.
#pragma once
#include "kdt_device.cuh"

namespace kd {

// outcome of move_point
enum MoveResult : int { MV_DONE = 0, MV_DEFER = 1, MV_GLOBAL = 2, MV_ABORT = -1 };

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

__device__ __forceinline__ int vtx_find(const WarpShared *sh, int cnt, int id)
{
    int idx = -1;
    for (int base = 0; base < cnt; base += 32) {
        int j = base + (threadIdx.x & 31);
        bool hit = j < cnt && sh->vid[j] == id;
        unsigned b = __ballot_sync(FULL, hit);
        if (b) {
            idx = base + __ffs(b) - 1;
            break;
        }
    }
    return idx;
}

struct Region {
    int cnt;             // staged triangles
    int vcnt;            // staged vertices
    unsigned long long dirty;  // modified staged triangles
};

__device__ __forceinline__ int2 vxy_of(const WarpShared *sh, const Region &R, int id)
{
    if (id < 0) return make_int2(0, 0);
    int j = vtx_find(sh, R.vcnt, id);
    return j >= 0 ? sh->vxy[j] : make_int2(0, 0);
}

// stage the vertices of triangle v that are not yet known (one round trip)
__device__ bool stage_vertices(Warp &w, const Dev &d, Region &R, int4 v)
{
    WarpShared *sh = w.sh;
    int ids[3] = {v.x, v.y, v.z};
    for (int c = 0; c < 3; ++c) {
        int id = ids[c];
        if (id < 0) continue;
        if (vtx_find(sh, R.vcnt, id) >= 0) continue;
        if (R.vcnt >= LV) return false;
        int2 x = make_int2(0, 0);
        if (w.lane == 0) x = __ldcg(d.xy + id);
        x = bcast2(x, 0);
        if (w.lane == 0) {
            sh->vid[R.vcnt] = id;
            sh->vxy[R.vcnt] = x;
        }
        __syncwarp();
        R.vcnt++;
    }
    return true;
}

// Claim and stage one more triangle (read under the claim, so no validation is
// needed).  Returns its staged index, or -1 when the claim fails or space runs out.
__device__ int ensure_local(Warp &w, const Dev &d, Region &R, int slot)
{
    WarpShared *sh = w.sh;
    int j = local_find(sh, R.cnt, slot);
    if (j >= 0) return j;
    if (R.cnt >= LM || w.ncl >= MAXC) return -1;
    int mine = w.lane == 0 ? slot : -1;
    if (!claim_lanes(w, d, mine, 1)) return -1;
    int4 v, nb;
    load_tri(w, d, slot, v, nb);
    if (!(v.w & ALIVE)) return -1;
    if (w.lane == 0) {
        sh->lslot[R.cnt] = slot;
        sh->lv[R.cnt] = v;
        sh->ln[R.cnt] = nb;
    }
    __syncwarp();
    j = R.cnt++;
    if (!stage_vertices(w, d, R, v)) return -1;
    return j;
}

// set component e of the neighbour refs of the staged triangle with global ref `ref`
__device__ __forceinline__ bool set_local_backptr(Warp &w, Region &R, int ref, int val)
{
    WarpShared *sh = w.sh;
    int j = local_find(sh, R.cnt, ref >> 2);
    if (j < 0) return false;
    if (w.lane == 0) {
        int4 n = sh->ln[j];
        int e = ref & 3;
        if (e == 0) n.x = val;
        else if (e == 1) n.y = val;
        else n.z = val;
        sh->ln[j] = n;
    }
    __syncwarp();
    R.dirty |= 1ull << j;
    return true;
}

// Write every modified staged triangle back (lane-parallel), update pt_tri of their
// vertices, append them to the dirty list with one atomic, then release all claims.
__device__ void write_back(Warp &w, const Dev &d, Region &R)
{
    WarpShared *sh = w.sh;
    unsigned long long m = R.dirty;
    int nd = __popcll(m);
    int base = 0;
    if (nd > 0 && w.lane == 0) base = atomicAdd(d.dirty_count, nd);
    base = __shfl_sync(FULL, base, 0);
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
            int pos = base + __popcll(m & ((1ull << j) - 1ull));
            if (pos < d.dirty_cap) d.dirty[pos] = slot;
        }
    }
    __syncwarp();
    __threadfence();
    R.dirty = 0;
    release_all(w, d);
}

// Ear validity on the staged link (same rule as ear_valid).
__device__ bool ear_ok(const WarpShared *sh, int m, int i, const Dev &d, unsigned *ex, unsigned *ti)
{
    return ear_valid(sh->L, sh->LX, m, i, d, ex, ti);
}

// Locate q in staged triangle j: -1 not inside, 0 inside, 1 on edge (*e), 2 on a vertex
// (*vtx), 3 strictly outside a ghost's hull edge.
__device__ __forceinline__ int locate_in(const WarpShared *sh, const Region &R, int j, int2 q, int *e, int *vtx)
{
    int4 v = sh->lv[j];
    if (!(v.w & ALIVE)) return -1;
    int g = v.x == KDT_GHOST ? 0 : (v.y == KDT_GHOST ? 1 : (v.z == KDT_GHOST ? 2 : -1));
    // coordinates through the staged vertex table (lane-local search)
    int2 p[3];
    int ids[3] = {v.x, v.y, v.z};
    for (int c = 0; c < 3; ++c) {
        p[c] = make_int2(0, 0);
        if (ids[c] < 0) continue;
        for (int t = 0; t < R.vcnt; ++t)
            if (sh->vid[t] == ids[c]) {
                p[c] = sh->vxy[t];
                break;
            }
    }
    if (g >= 0) {
        int2 pu = p[(g + 1) % 3], pv = p[(g + 2) % 3];
        return orient2d(pu, pv, q) > 0 ? 3 : -1;
    }
    int o0 = orient2d(p[1], p[2], q), o1 = orient2d(p[2], p[0], q), o2 = orient2d(p[0], p[1], q);
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

// Staged fan around q: triangles (q, W[k], W[k+1]) into staged entries X[k]; O[k]
// is the global ref of the outer neighbour across (W[k], W[k+1]) (staged).
__device__ bool local_fan(Warp &w, Region &R, int q, const int *W, const int *O, const int *X, int m)
{
    WarpShared *sh = w.sh;
    if (w.lane == 0) {
        for (int k = 0; k < m; ++k) {
            int kn = (k + 1) % m, kp = (k + m - 1) % m;
            sh->lv[X[k]] = make_int4(q, W[k], W[kn], ALIVE);
            sh->ln[X[k]] = make_int4(O[k], (sh->lslot[X[kn]] << 2) | 2, (sh->lslot[X[kp]] << 2) | 1, 0);
        }
    }
    __syncwarp();
    for (int k = 0; k < m; ++k) {
        R.dirty |= 1ull << X[k];
        if (!set_local_backptr(w, R, O[k], (sh->lslot[X[k]] << 2) | 0)) return false;
    }
    return true;
}

// Lawson flips of the edges opposite p on the staged region.  Entries are (staged
// index, edge).  A flip whose quadrilateral or outer ring leaves the region stages
// the missing triangles first; if that fails the remaining stack is returned to the
// caller (converted to global slots) with *top_out > 0.
__device__ void local_lawson(Warp &w, const Dev &d, Region &R, int p, int top, int *top_out, bool *aborted)
{
    WarpShared *sh = w.sh;
    *aborted = false;
    while (top > 0) {
        int2 ent = sh->stack[top - 1];
        __syncwarp();
        --top;
        int T = ent.x, e = ent.y;
        int4 v = sh->lv[T], nb = sh->ln[T];
        if (!(v.w & ALIVE) || comp(v, e) != p) continue;
        int ref = comp(nb, e);
        int U = ensure_local(w, d, R, ref >> 2);
        if (U < 0) {
            // push the entry back and hand the rest to the global path
            if (w.lane == 0) sh->stack[top] = ent;
            __syncwarp();
            *top_out = top + 1;
            *aborted = true;
            return;
        }
        int f = ref & 3;
        int4 uv = sh->lv[U], un = sh->ln[U];
        int a = comp(v, (e + 1) % 3), b = comp(v, (e + 2) % 3), dd = comp(uv, f);
        int2 pv[3];
        pv[e] = vxy_of(sh, R, p);
        pv[(e + 1) % 3] = vxy_of(sh, R, a);
        pv[(e + 2) % 3] = vxy_of(sh, R, b);
        int2 pd = vxy_of(sh, R, dd);
        w.cnt[C_FLIP_TESTS]++;
        if (!conflict(v.x, v.y, v.z, pv[0], pv[1], pv[2], dd, pd, d.use_filter, &w.cnt[C_EXACT], &w.cnt[C_TIES]))
            continue;
        // stage the four outer neighbours (back-pointers change)
        int nt_a = comp(nb, (e + 1) % 3), nt_b = comp(nb, (e + 2) % 3);
        int nu_b = comp(un, (f + 1) % 3), nu_a = comp(un, (f + 2) % 3);
        bool ok = ensure_local(w, d, R, nt_a >> 2) >= 0 && ensure_local(w, d, R, nt_b >> 2) >= 0 &&
                  ensure_local(w, d, R, nu_a >> 2) >= 0 && ensure_local(w, d, R, nu_b >> 2) >= 0;
        if (!ok) {
            if (w.lane == 0) sh->stack[top] = ent;
            __syncwarp();
            *top_out = top + 1;
            *aborted = true;
            return;
        }
        int sT = sh->lslot[T], sU = sh->lslot[U];
        if (w.lane == 0) {
            sh->lv[T] = make_int4(p, a, dd, ALIVE);
            sh->ln[T] = make_int4(nu_b, (sU << 2) | 2, nt_b, 0);
            sh->lv[U] = make_int4(p, dd, b, ALIVE);
            sh->ln[U] = make_int4(nu_a, nt_a, (sT << 2) | 1, 0);
        }
        __syncwarp();
        R.dirty |= (1ull << T) | (1ull << U);
        set_local_backptr(w, R, nu_b, (sT << 2) | 0);
        set_local_backptr(w, R, nt_b, (sT << 2) | 2);
        set_local_backptr(w, R, nu_a, (sU << 2) | 0);
        set_local_backptr(w, R, nt_a, (sU << 2) | 1);
        w.cnt[C_FLIPS]++;
        if (top + 2 > STACK) {
            w.cnt[C_STACK_DROP]++;
            continue;
        }
        if (w.lane == 0) {
            sh->stack[top] = make_int2(T, 0);
            sh->stack[top + 1] = make_int2(U, 0);
        }
        __syncwarp();
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
        R.vcnt = 0;
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
            // validate under the claims; stage the vertex coordinates in the same pass
            bool good = true;
            for (int i = w.lane; i < 2 * k; i += 32) {
                int slot = sh->lslot[i];
                int4 v = __ldcg(d.tv + slot), nb = __ldcg(d.tn + slot);
                int4 v0 = sh->lv[i], n0 = sh->ln[i];
                good = good && v.x == v0.x && v.y == v0.y && v.z == v0.z && v.w == v0.w && nb.x == n0.x &&
                       nb.y == n0.y && nb.z == n0.z && (v.w & ALIVE);
                if (i < k) {
                    int I = sh->I[i];
                    good = good && comp(v, I) == p && comp(v, (I + 1) % 3) == sh->L[i] && comp(nb, I) == sh->ON[i] &&
                           (comp(nb, (I + 1) % 3) >> 2) == sh->S[(i + 1) % k];
                }
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
        // vertex table: link vertices (coordinates into LX too) and ring apexes
        for (int i = w.lane; i < k; i += 32) {
            int lv = sh->L[i];
            int2 x = lv >= 0 ? __ldcg(d.xy + lv) : make_int2(0, 0);
            sh->LX[i] = x;
            sh->vid[i] = lv;
            sh->vxy[i] = x;
            int4 rv = sh->lv[k + i];
            int ap = comp(rv, sh->ON[i] & 3);
            sh->vid[k + i] = ap;
            sh->vxy[k + i] = ap >= 0 ? __ldcg(d.xy + ap) : make_int2(0, 0);
        }
        __syncwarp();
        R.vcnt = 2 * k;
        // ring duplicates (a triangle adjacent to two link edges) keep their first copy:
        // point later copies at an unused slot id so lookups find the first one
        for (int i = w.lane; i < k; i += 32) {
            int slot = sh->lslot[k + i];
            for (int j = 0; j < i; ++j)
                if (sh->lslot[k + j] == slot) sh->lslot[k + i] = -2 - i;
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
                    int4 ov = sh->lv[k + i];
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
                bool v = i < m && ear_ok(sh, m, i, d, &ex, &ti);
                unsigned bm = __ballot_sync(FULL, v);
                if (bm) chosen = base + __ffs(bm) - 1;
            }
            w.cnt[C_EXACT] += __reduce_add_sync(FULL, ex);
            w.cnt[C_TIES] += __reduce_add_sync(FULL, ti);
            if (chosen < 0) {
                release_all(w, d);
                return DEV_INTERNAL;
            }
            int i = chosen, i1 = (i + 1) % m, i2 = (i + 2) % m;
            int X = newc++;  // staged index == star position
            int sX = sh->S[X];
            int on_i = sh->ON[i], on_i1 = sh->ON[i1];
            if (w.lane == 0) {
                sh->lv[X] = make_int4(sh->L[i], sh->L[i1], sh->L[i2], ALIVE);
                sh->ln[X] = make_int4(on_i1, -1, on_i, 0);
                sh->ON[i] = (sX << 2) | 1;
            }
            __syncwarp();
            R.dirty |= 1ull << X;
            set_local_backptr(w, R, on_i1, (sX << 2) | 0);
            set_local_backptr(w, R, on_i, (sX << 2) | 2);
            // remove element i1
            int lv = 0, onv = 0;
            int2 xv = make_int2(0, 0);
            int j = w.lane;
            bool mv = j >= i1 && j < m - 1;
            if (mv) {
                lv = sh->L[j + 1];
                onv = sh->ON[j + 1];
                xv = sh->LX[j + 1];
            }
            bool mv2 = j + 32 >= i1 && j + 32 < m - 1;
            int lv2 = 0, onv2 = 0;
            int2 xv2 = make_int2(0, 0);
            if (mv2) {
                lv2 = sh->L[j + 33];
                onv2 = sh->ON[j + 33];
                xv2 = sh->LX[j + 33];
            }
            __syncwarp();
            if (mv) {
                sh->L[j] = lv;
                sh->ON[j] = onv;
                sh->LX[j] = xv;
            }
            if (mv2) {
                sh->L[j + 32] = lv2;
                sh->ON[j + 32] = onv2;
                sh->LX[j + 32] = xv2;
            }
            __syncwarp();
            --m;
        }
        {
            int X = newc++;
            int sX = sh->S[X];
            int on0 = sh->ON[0], on1 = sh->ON[1], on2 = sh->ON[2];
            if (w.lane == 0) {
                sh->lv[X] = make_int4(sh->L[0], sh->L[1], sh->L[2], ALIVE);
                sh->ln[X] = make_int4(on1, on2, on0, 0);
            }
            __syncwarp();
            R.dirty |= 1ull << X;
            set_local_backptr(w, R, on1, (sX << 2) | 0);
            set_local_backptr(w, R, on2, (sX << 2) | 1);
            set_local_backptr(w, R, on0, (sX << 2) | 2);
        }
        // spares: staged entries k-2, k-1 (dead)
        int X0 = k - 2, X1 = k - 1;
        if (w.lane == 0) {
            sh->lv[X0] = make_int4(0, 0, 0, 0);
            sh->lv[X1] = make_int4(0, 0, 0, 0);
            d.pt_tri[p] = -1;
        }
        __syncwarp();
        R.dirty |= (1ull << X0) | (1ull << X1);
        w.cnt[C_DEG_DEL] += k;
        w.cnt[C_DELETES]++;
        s0 = sh->S[X0];
        s1 = sh->S[X1];
        hint = sh->S[0];
        // Update (Fig. 4): p takes its new position
        if (w.lane == 0) d.xy[p] = q;
        // q joins the vertex table
        if (w.lane == 0) {
            sh->vid[R.vcnt] = p;
            sh->vxy[R.vcnt] = q;
        }
        __syncwarp();
        R.vcnt++;
        // ---- 2. locate q among the staged triangles
        int where = -1, te = 0, tvtx = -1, tj = -1;
        for (int base = 0; base < R.cnt && tj < 0; base += 32) {
            int j = base + w.lane;
            int e = 0, vt = -1;
            int r = j < R.cnt && sh->lslot[j] >= 0 ? locate_in(sh, R, j, q, &e, &vt) : -1;
            // prefer a finite hit; a ghost hit (outside the hull) goes to the global path
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
        // ---- 3. split (staged); make sure every triangle whose refs change is staged
        int4 v = sh->lv[tj], nb = sh->ln[tj];
        int *W = sh->tmp, *O = sh->tmp + 8, *Xs = sh->tmp + 16;
        int mf;
        bool okf = true;
        if (where == 1) {
            int e = te;
            int Uj = ensure_local(w, d, R, comp(nb, e) >> 2);
            okf = Uj >= 0;
            int4 uv = make_int4(0, 0, 0, 0), un = make_int4(0, 0, 0, 0);
            int f = comp(nb, e) & 3;
            if (okf) {
                uv = sh->lv[Uj];
                un = sh->ln[Uj];
                okf = ensure_local(w, d, R, comp(nb, (e + 1) % 3) >> 2) >= 0 &&
                      ensure_local(w, d, R, comp(nb, (e + 2) % 3) >> 2) >= 0 &&
                      ensure_local(w, d, R, comp(un, (f + 1) % 3) >> 2) >= 0 &&
                      ensure_local(w, d, R, comp(un, (f + 2) % 3) >> 2) >= 0;
            }
            if (okf && w.lane == 0) {
                int a = comp(v, e), b = comp(v, (e + 1) % 3), c = comp(v, (e + 2) % 3), dd = comp(uv, f);
                W[0] = a; W[1] = b; W[2] = dd; W[3] = c;
                O[0] = comp(nb, (e + 2) % 3);
                O[1] = comp(un, (f + 1) % 3);
                O[2] = comp(un, (f + 2) % 3);
                O[3] = comp(nb, (e + 1) % 3);
                Xs[0] = tj; Xs[1] = Uj; Xs[2] = X0; Xs[3] = X1;
            }
            mf = 4;
            if (okf) w.cnt[C_SPLIT_EDGE]++;
        } else {
            okf = ensure_local(w, d, R, nb.x >> 2) >= 0 && ensure_local(w, d, R, nb.y >> 2) >= 0 &&
                  ensure_local(w, d, R, nb.z >> 2) >= 0;
            if (okf && w.lane == 0) {
                W[0] = v.x; W[1] = v.y; W[2] = v.z;
                O[0] = nb.z; O[1] = nb.x; O[2] = nb.y;
                Xs[0] = tj; Xs[1] = X0; Xs[2] = X1;
            }
            mf = 3;
        }
        __syncwarp();
        if (!okf) {
            write_back(w, d, R);
            return MV_GLOBAL;
        }
        // the spare entries get slots s0, s1 already (lslot of X0 / X1)
        if (!local_fan(w, R, p, W, O, Xs, mf)) {
            // a needed neighbour was not staged (cannot happen after ensure_local)
            write_back(w, d, R);
            return DEV_INTERNAL;
        }
        w.cnt[C_INSERTS]++;
        // ---- 4. Lawson flips of the edges opposite q
        if (w.lane == 0)
            for (int j = 0; j < mf; ++j) sh->stack[j] = make_int2(Xs[j], 0);
        __syncwarp();
        int left = 0;
        bool aborted = false;
        local_lawson(w, d, R, p, mf, &left, &aborted);
        // convert what is left to global (slot, edge) entries before the region goes
        if (left > 0 && w.lane == 0)
            for (int j = 0; j < left; ++j) sh->stack[j] = make_int2(sh->lslot[sh->stack[j].x], sh->stack[j].y);
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
