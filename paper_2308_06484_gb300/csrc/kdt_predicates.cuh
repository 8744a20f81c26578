// Exact geometric predicates for the kinetic Delaunay path (device side).
//
// The Delaunay property (paper, Section I: the circumcircle of a triangle holds no
// point but its own vertices) is decided by two signs:
//   orient2d(a,b,c)  = sign det[[ax,ay,1],[bx,by,1],[cx,cy,1]]      (int64, exact)
//   incircle(a,b,c,d) = sign of the lifted 4x4 determinant            (__int128, exact)
// behind an FP32 filter whose sign is only used when a proven error bound certifies
// it.  Section I's uniqueness claim needs general position; ties (four cocircular
// points) are broken by Simulation of Simplicity on the lifting map: point i's lifted
// height gets +eps_i with eps decreasing as the id grows, so the sign of a zero
// determinant is the sign of the z-cofactor of the smallest id.
//
// Coordinates lie in [0, 2^28): a difference fits 29 bits, a product of two
// differences 57 bits, the incircle determinant |det| < 3 * 2^114.
#pragma once
#include <cstdint>

#define KDT_GHOST (-1)

namespace kd {

__device__ __forceinline__ int sgn64(long long v) { return (v > 0) - (v < 0); }

// orient2d: +1 when a, b, c turn counter-clockwise.
__device__ __forceinline__ int orient2d(int2 a, int2 b, int2 c)
{
    long long d = (long long)(b.x - a.x) * (long long)(c.y - a.y) -
                  (long long)(b.y - a.y) * (long long)(c.x - a.x);
    return sgn64(d);
}

// q strictly inside the open segment uv, given u, v, q collinear.
__device__ __forceinline__ bool strictly_between(int2 u, int2 v, int2 q)
{
    long long d1 = (long long)(q.x - u.x) * (v.x - u.x) + (long long)(q.y - u.y) * (v.y - u.y);
    long long d2 = (long long)(q.x - v.x) * (u.x - v.x) + (long long)(q.y - v.y) * (u.y - v.y);
    return d1 > 0 && d2 > 0;
}

// Exact sign of the incircle determinant of d against (a,b,c):
//   det rows (x_i - x_d, y_i - y_d, (x_i - x_d)^2 + (y_i - y_d)^2), i = a, b, c,
// positive iff d is strictly inside the circle of counter-clockwise (a,b,c).
__device__ __forceinline__ int incircle_exact(int2 a, int2 b, int2 c, int2 d)
{
    long long adx = a.x - d.x, ady = a.y - d.y;
    long long bdx = b.x - d.x, bdy = b.y - d.y;
    long long cdx = c.x - d.x, cdy = c.y - d.y;
    long long al = adx * adx + ady * ady;  // < 2^57
    long long bl = bdx * bdx + bdy * bdy;
    long long cl = cdx * cdx + cdy * cdy;
    long long ma = bdx * cdy - cdx * bdy;  // < 2^57 in magnitude
    long long mb = cdx * ady - adx * cdy;
    long long mc = adx * bdy - bdx * ady;
    __int128 det = (__int128)al * ma + (__int128)bl * mb + (__int128)cl * mc;
    return (det > 0) - (det < 0);
}

// FP32 filter for the same determinant.  Differences are exact int32 values rounded
// once to float (relative error <= u = 2^-24).  Every later operation is an explicit
// round-to-nearest op (no contraction), so standard forward error analysis gives
//   |det_f - det| <= ~12 u * perm,   perm = sum_i lift_i * (|m_i,1| + |m_i,2|),
// and the computed perm_f is within ~10 u of perm.  The filter certifies the sign
// when |det_f| > 64 u * perm_f; otherwise it returns 0 and the exact path decides.
__device__ __forceinline__ int incircle_filter(int2 a, int2 b, int2 c, int2 d)
{
    float adx = __int2float_rn(a.x - d.x), ady = __int2float_rn(a.y - d.y);
    float bdx = __int2float_rn(b.x - d.x), bdy = __int2float_rn(b.y - d.y);
    float cdx = __int2float_rn(c.x - d.x), cdy = __int2float_rn(c.y - d.y);
    float al = __fadd_rn(__fmul_rn(adx, adx), __fmul_rn(ady, ady));
    float bl = __fadd_rn(__fmul_rn(bdx, bdx), __fmul_rn(bdy, bdy));
    float cl = __fadd_rn(__fmul_rn(cdx, cdx), __fmul_rn(cdy, cdy));
    float a1 = __fmul_rn(bdx, cdy), a2 = __fmul_rn(cdx, bdy);
    float b1 = __fmul_rn(cdx, ady), b2 = __fmul_rn(adx, cdy);
    float c1 = __fmul_rn(adx, bdy), c2 = __fmul_rn(bdx, ady);
    float det = __fadd_rn(__fadd_rn(__fmul_rn(al, __fsub_rn(a1, a2)), __fmul_rn(bl, __fsub_rn(b1, b2))),
                          __fmul_rn(cl, __fsub_rn(c1, c2)));
    float perm = __fadd_rn(__fadd_rn(__fmul_rn(al, __fadd_rn(fabsf(a1), fabsf(a2))),
                                     __fmul_rn(bl, __fadd_rn(fabsf(b1), fabsf(b2)))),
                           __fmul_rn(cl, __fadd_rn(fabsf(c1), fabsf(c2))));
    float bound = perm * 0x1p-18f;  // 64 u, exact scaling by a power of two
    if (det > bound) return 1;
    if (det < -bound) return -1;
    return 0;
}

// Unperturbed sign; use_filter selects the filtered path.  *exact_calls counts how
// often the exact path ran (filter misses).
__device__ __forceinline__ int incircle_raw(int2 a, int2 b, int2 c, int2 d, bool use_filter,
                                            unsigned *exact_calls)
{
    if (use_filter) {
        int f = incircle_filter(a, b, c, d);
        if (f) return f;
    }
    ++*exact_calls;
    return incircle_exact(a, b, c, d);
}

// The exact sign, and when it is zero the Simulation-of-Simplicity answer: the sign of
// the first non-zero z-cofactor in increasing id order (row a: +orient(b,c,d), row b:
// -orient(a,c,d), row c: +orient(a,b,d), row d: -orient(a,b,c)).  Out of line: the
// filter decides most tests, and one copy of this slow path keeps the inlined code of
// every caller small.  Returns the sign, plus 8 when the tie-break decided.
__device__ __noinline__ int incircle_sos_exact(int ia, int ib, int ic, int id, int2 a, int2 b, int2 c, int2 d)
{
    int s = incircle_exact(a, b, c, d);
    if (s) return s;
    int ids[4] = {ia, ib, ic, id};
    int done = 0;
    for (int k = 0; k < 4; ++k) {
        int best = -1;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (!((done >> i) & 1) && (best < 0 || ids[i] < ids[best])) best = i;
        done |= 1 << best;
        int cof;
        switch (best) {
        case 0: cof = orient2d(b, c, d); break;
        case 1: cof = -orient2d(a, c, d); break;
        case 2: cof = orient2d(a, b, d); break;
        default: cof = -orient2d(a, b, c); break;
        }
        if (cof) return cof + 8;
    }
    return 8;
}

// Simulation-of-Simplicity incircle: rows a, b, c, d with ids ia..id (the filter, then
// incircle_sos_exact).
__device__ __forceinline__ int incircle_sos(int ia, int ib, int ic, int id, int2 a, int2 b,
                                            int2 c, int2 d, bool use_filter, unsigned *exact_calls,
                                            unsigned *ties)
{
    if (use_filter) {
        int f = incircle_filter(a, b, c, d);
        if (f) return f;
    }
    ++*exact_calls;
    int r = incircle_sos_exact(ia, ib, ic, id, a, b, c, d);
    if (r >= 7) {
        ++*ties;
        return r - 8;
    }
    return r;
}

// Conflict of a ghost triangle (u, v, inf), stored counter-clockwise: the outside of
// the hull is to the left of u->v.  q conflicts iff it is strictly left of u->v or on
// the open segment uv.
__device__ __forceinline__ bool ghost_conflict(int2 u, int2 v, int2 q)
{
    int o = orient2d(u, v, q);
    if (o) return o > 0;
    return strictly_between(u, v, q);
}

// Does the circumcircle of triangle (v0,v1,v2) (one vertex may be the ghost) contain
// point q?  The Bowyer-Watson / Lawson conflict test, generalised to ghosts.
__device__ __forceinline__ bool conflict(int v0, int v1, int v2, int2 p0, int2 p1, int2 p2, int q,
                                         int2 pq, bool use_filter, unsigned *exact_calls,
                                         unsigned *ties)
{
    if (q == KDT_GHOST) return false;  // infinity is never inside a finite circle
    if (v0 == KDT_GHOST) return ghost_conflict(p1, p2, pq);
    if (v1 == KDT_GHOST) return ghost_conflict(p2, p0, pq);
    if (v2 == KDT_GHOST) return ghost_conflict(p0, p1, pq);
    return incircle_sos(v0, v1, v2, q, p0, p1, p2, pq, use_filter, exact_calls, ties) > 0;
}

}  // namespace kd
