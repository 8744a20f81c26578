/*
 * Delaunay triangulation oracle — plain, slow, single-threaded C.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline / reference leg may load this library.  The product path (the CUDA
 * library and its Python binding) never links, loads or calls it, and it shares no
 * code, header, table or helper with that path.
 *
 * What it computes (paper, Section I, definition of the DT; Section IV "Insertion
 * and Deletion", Bowyer-Watson insertion; Fig. 4, the triangulation it outputs after
 * every time step): for a set P of distinct integer points, the unique Delaunay
 * triangulation, as a canonical sorted list of triangles.  The kinetic method of the
 * paper reaches the same triangulation by deletions and insertions; the oracle does
 * not replay them, it rebuilds from scratch (the DT is a function of the positions
 * only, Section III: "only the DT after each time step is completely valid").
 *
 * Readings of the paper (all listed in the design notes):
 *  - Uniqueness (Section I) only holds in general position.  Ties (four cocircular
 *    points) are broken by Simulation of Simplicity on the lifting map: the lifted
 *    height x^2+y^2 of point i gets an infinitesimal eps_i added, with
 *    eps_0 >> eps_1 >> ... (a smaller point id means a larger perturbation).
 *    Coordinates are never perturbed.
 *  - "Circumcircle includes only the vertices" leaves points on the circle open;
 *    the same perturbation decides them.
 *  - The hull is handled with a vertex at infinity (ghost triangles).  A ghost
 *    (u, v, inf) stored counter-clockwise has the outside of the hull to the left of
 *    u->v.  A point q conflicts with it iff q is strictly left of u->v, or on the
 *    line strictly inside the segment uv.
 *
 * Coordinates must lie in [0, 2^28): differences fit 29 bits, orient2d fits int64
 * and the 3x3 incircle determinant fits __int128 (|det| < 3 * 2^114).
 *
 * Every function cites the passage it follows.  All arithmetic deciding the
 * triangulation is exact integer arithmetic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

#define ORC_GHOST (-1)

/* Return codes shared by the oracle's entry points (not by the CUDA library). */
#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_RANGE (-2)
#define ORC_ERR_DUPLICATE (-3)
#define ORC_ERR_DEGENERATE (-4)
#define ORC_ERR_CAPACITY (-5)
#define ORC_ERR_NOMEM (-6)
#define ORC_ERR_INTERNAL (-7)

#define COORD_LIMIT (1 << 28)

static inline int64_t px(const int32_t *xy, int32_t v) { return (int64_t)xy[2 * (int64_t)v]; }
static inline int64_t py(const int32_t *xy, int32_t v) { return (int64_t)xy[2 * (int64_t)v + 1]; }

/* ---------------------------------------------------------------------------
 * Predicates (Section I: the empty-circumcircle definition of the DT).
 * ------------------------------------------------------------------------- */

/* Sign of det[[ax,ay,1],[bx,by,1],[cx,cy,1]]: +1 when a,b,c turn counter-clockwise. */
int oracle_orient2d(const int32_t *xy, int32_t a, int32_t b, int32_t c)
{
    int64_t d = (px(xy, b) - px(xy, a)) * (py(xy, c) - py(xy, a)) -
                (py(xy, b) - py(xy, a)) * (px(xy, c) - px(xy, a));
    return (d > 0) - (d < 0);
}

/* Sign of the unperturbed incircle determinant of d against (a,b,c):
 * det of the rows (x_i - x_d, y_i - y_d, (x_i - x_d)^2 + (y_i - y_d)^2), i = a,b,c.
 * For counter-clockwise (a,b,c) it is positive iff d is strictly inside the
 * circumcircle.  It equals the 4x4 determinant of the lifted rows (x, y, x^2+y^2, 1)
 * of a, b, c, d in that order. */
int oracle_incircle_raw(const int32_t *xy, int32_t a, int32_t b, int32_t c, int32_t d)
{
    int64_t adx = px(xy, a) - px(xy, d), ady = py(xy, a) - py(xy, d);
    int64_t bdx = px(xy, b) - px(xy, d), bdy = py(xy, b) - py(xy, d);
    int64_t cdx = px(xy, c) - px(xy, d), cdy = py(xy, c) - py(xy, d);
    i128 alift = (i128)adx * adx + (i128)ady * ady;
    i128 blift = (i128)bdx * bdx + (i128)bdy * bdy;
    i128 clift = (i128)cdx * cdx + (i128)cdy * cdy;
    i128 m_a = (i128)bdx * cdy - (i128)cdx * bdy;
    i128 m_b = (i128)cdx * ady - (i128)adx * cdy;
    i128 m_c = (i128)adx * bdy - (i128)bdx * ady;
    i128 det = alift * m_a + blift * m_b + clift * m_c;
    return (det > 0) - (det < 0);
}

/* Simulation-of-Simplicity incircle (reading of the uniqueness claim, Section I).
 * With z_i = x_i^2 + y_i^2 + eps_i and eps decreasing with the point id, the
 * perturbed 4x4 determinant is D + sum_i eps_i * C_i, where C_i is the cofactor of
 * the z entry of row i.  When D == 0 its sign is the sign of the cofactor of the
 * smallest id whose cofactor is non-zero:
 *   row a: +orient(b,c,d)   row b: -orient(a,c,d)
 *   row c: +orient(a,b,d)   row d: -orient(a,b,c)
 * Returns +1 (d inside), -1 (d outside), or 0 only for fully degenerate input
 * (e.g. four collinear points), which a triangulation never asks. */
int oracle_incircle_sos(const int32_t *xy, int32_t a, int32_t b, int32_t c, int32_t d)
{
    int s = oracle_incircle_raw(xy, a, b, c, d);
    if (s != 0)
        return s;
    int32_t ids[4] = {a, b, c, d};
    int cof[4];
    cof[0] = oracle_orient2d(xy, b, c, d);
    cof[1] = -oracle_orient2d(xy, a, c, d);
    cof[2] = oracle_orient2d(xy, a, b, d);
    cof[3] = -oracle_orient2d(xy, a, b, c);
    /* visit rows in increasing id order */
    int used[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; ++k) {
        int best = -1;
        for (int i = 0; i < 4; ++i)
            if (!used[i] && (best < 0 || ids[i] < ids[best]))
                best = i;
        used[best] = 1;
        if (cof[best] != 0)
            return cof[best];
    }
    return 0;
}

/* q strictly inside the open segment uv, given that u, v, q are collinear. */
static int strictly_between(const int32_t *xy, int32_t u, int32_t v, int32_t q)
{
    int64_t d1 = (px(xy, q) - px(xy, u)) * (px(xy, v) - px(xy, u)) +
                 (py(xy, q) - py(xy, u)) * (py(xy, v) - py(xy, u));
    int64_t d2 = (px(xy, q) - px(xy, v)) * (px(xy, u) - px(xy, v)) +
                 (py(xy, q) - py(xy, v)) * (py(xy, u) - py(xy, v));
    return d1 > 0 && d2 > 0;
}

/* Bowyer-Watson conflict test (Section IV, Insertion): does the circumcircle of
 * triangle (v0,v1,v2) (counter-clockwise) contain q?  A ghost triangle's "circle"
 * is the open half-plane outside its hull edge plus the open hull segment. */
static int conflicts(const int32_t *xy, const int32_t *tv, int32_t q)
{
    int g = -1;
    for (int i = 0; i < 3; ++i)
        if (tv[i] == ORC_GHOST)
            g = i;
    if (g < 0)
        return oracle_incircle_sos(xy, tv[0], tv[1], tv[2], q) > 0;
    int32_t u = tv[(g + 1) % 3], v = tv[(g + 2) % 3];
    int o = oracle_orient2d(xy, u, v, q);
    if (o != 0)
        return o > 0;
    return strictly_between(xy, u, v, q);
}

/* ---------------------------------------------------------------------------
 * A counter-based generator (splitmix64, Steele, Lea and Flood 2014), used only to
 * draw the oracle's own insertion order.  The result does not depend on it.
 * ------------------------------------------------------------------------- */
static uint64_t splitmix64(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ---------------------------------------------------------------------------
 * Bowyer-Watson triangulation (Section IV, Insertion, reference [13]).
 * ------------------------------------------------------------------------- */
typedef struct {
    const int32_t *xy;
    int64_t n;
    int32_t *tv;   /* 3 vertices per triangle, counter-clockwise; ORC_GHOST = infinity */
    int32_t *tn;   /* tn[3t+i]: triangle across the edge opposite vertex i */
    int64_t nt;    /* triangles in use */
    int64_t cap;
    int32_t *vtri; /* vtri[v]: some live triangle incident to v */
    int64_t *stamp;
    int32_t *start_of; /* scratch: new triangle whose boundary edge starts at a vertex */
    /* locate hint: a uniform grid over the bounding box, last inserted vertex per cell */
    int64_t gx0, gy0, gshift;
    int64_t gdim;
    int32_t *grid;
    int32_t last_tri;
    /* growable work lists */
    int32_t *cav;
    int64_t cav_cap;
    int32_t *bnd; /* triples (t, i, outside) */
    int64_t bnd_cap;
} bw_t;

static int is_ghost_tri(const bw_t *s, int32_t t)
{
    const int32_t *v = s->tv + 3 * (int64_t)t;
    return v[0] == ORC_GHOST || v[1] == ORC_GHOST || v[2] == ORC_GHOST;
}

static int64_t vslot(const bw_t *s, int32_t v) { return v == ORC_GHOST ? s->n : (int64_t)v; }

static int64_t grid_cell(const bw_t *s, int32_t v)
{
    int64_t cx = (px(s->xy, v) - s->gx0) >> s->gshift;
    int64_t cy = (py(s->xy, v) - s->gy0) >> s->gshift;
    if (cx >= s->gdim) cx = s->gdim - 1;
    if (cy >= s->gdim) cy = s->gdim - 1;
    return cy * s->gdim + cx;
}

/* Visibility walk from triangle t towards q.  Returns a triangle in conflict with q
 * (the triangle holding q, or a ghost whose hull edge q sees strictly). */
static int32_t locate(bw_t *s, int32_t t, int32_t q)
{
    const int32_t *xy = s->xy;
    int64_t steps = 0, limit = 4 * s->nt + 64;
    while (steps++ < limit) {
        const int32_t *v = s->tv + 3 * (int64_t)t;
        if (is_ghost_tri(s, t)) {
            if (conflicts(xy, v, q))
                return t;
            int g = v[0] == ORC_GHOST ? 0 : (v[1] == ORC_GHOST ? 1 : 2);
            t = s->tn[3 * (int64_t)t + g]; /* across the finite edge */
            continue;
        }
        int moved = 0;
        for (int i = 0; i < 3; ++i) {
            if (oracle_orient2d(xy, v[(i + 1) % 3], v[(i + 2) % 3], q) < 0) {
                t = s->tn[3 * (int64_t)t + i];
                moved = 1;
                break;
            }
        }
        if (!moved)
            return t;
    }
    /* never expected; a linear scan is still correct (the cavity is connected) */
    for (int64_t u = 0; u < s->nt; ++u)
        if (conflicts(xy, s->tv + 3 * u, q))
            return (int32_t)u;
    return -1;
}

static int grow(void **p, int64_t *cap, int64_t need, size_t elem)
{
    if (need <= *cap)
        return 0;
    int64_t nc = *cap ? *cap : 64;
    while (nc < need)
        nc *= 2;
    void *q = realloc(*p, (size_t)nc * elem);
    if (!q)
        return -1;
    *p = q;
    *cap = nc;
    return 0;
}

/* find the edge of triangle o whose endpoints are (b, a) in o's orientation */
static int edge_index(const bw_t *s, int32_t o, int32_t a, int32_t b)
{
    const int32_t *v = s->tv + 3 * (int64_t)o;
    for (int j = 0; j < 3; ++j)
        if (v[(j + 1) % 3] == b && v[(j + 2) % 3] == a)
            return j;
    return -1;
}

/* Insert q: grow the conflict region from a located triangle, remove it, and join
 * every boundary edge to q (Bowyer-Watson, Section IV). */
static int bw_insert(bw_t *s, int32_t q, int64_t it)
{
    int32_t t0 = -1;
    int64_t cell = grid_cell(s, q);
    int32_t hint = s->grid[cell];
    if (hint >= 0)
        t0 = s->vtri[hint];
    if (t0 < 0)
        t0 = s->last_tri;
    int32_t seed = locate(s, t0, q);
    if (seed < 0)
        return ORC_ERR_INTERNAL;

    int64_t ncav = 0, nbnd = 0;
    if (grow((void **)&s->cav, &s->cav_cap, 1, sizeof(int32_t)))
        return ORC_ERR_NOMEM;
    s->cav[ncav++] = seed;
    s->stamp[seed] = it;
    for (int64_t k = 0; k < ncav; ++k) {
        int32_t t = s->cav[k];
        for (int i = 0; i < 3; ++i) {
            int32_t o = s->tn[3 * (int64_t)t + i];
            if (s->stamp[o] == it)
                continue;
            if (conflicts(s->xy, s->tv + 3 * (int64_t)o, q)) {
                s->stamp[o] = it;
                if (grow((void **)&s->cav, &s->cav_cap, ncav + 1, sizeof(int32_t)))
                    return ORC_ERR_NOMEM;
                s->cav[ncav++] = o;
            } else {
                if (grow((void **)&s->bnd, &s->bnd_cap, 3 * (nbnd + 1), sizeof(int32_t)))
                    return ORC_ERR_NOMEM;
                s->bnd[3 * nbnd] = t;
                s->bnd[3 * nbnd + 1] = i;
                s->bnd[3 * nbnd + 2] = o;
                ++nbnd;
            }
        }
    }
    if (nbnd != ncav + 2)
        return ORC_ERR_INTERNAL; /* the cavity of a triangulated sphere is a disk */
    if (s->nt + 2 > s->cap)
        return ORC_ERR_INTERNAL;

    /* slots: the cavity's own, then two fresh ones */
    int32_t *newt = (int32_t *)malloc((size_t)nbnd * sizeof(int32_t));
    int32_t *ea = (int32_t *)malloc((size_t)nbnd * sizeof(int32_t));
    int32_t *eb = (int32_t *)malloc((size_t)nbnd * sizeof(int32_t));
    if (!newt || !ea || !eb) {
        free(newt); free(ea); free(eb);
        return ORC_ERR_NOMEM;
    }
    for (int64_t k = 0; k < nbnd; ++k) {
        int32_t t = s->bnd[3 * k], i = s->bnd[3 * k + 1];
        ea[k] = s->tv[3 * (int64_t)t + (i + 1) % 3];
        eb[k] = s->tv[3 * (int64_t)t + (i + 2) % 3];
        newt[k] = k < ncav ? s->cav[k] : (int32_t)(s->nt++);
    }
    for (int64_t k = 0; k < nbnd; ++k) {
        int32_t N = newt[k], o = s->bnd[3 * k + 2];
        int32_t *v = s->tv + 3 * (int64_t)N;
        v[0] = ea[k];
        v[1] = eb[k];
        v[2] = q;
        s->tn[3 * (int64_t)N + 2] = o;
        int j = edge_index(s, o, ea[k], eb[k]);
        if (j < 0) {
            free(newt); free(ea); free(eb);
            return ORC_ERR_INTERNAL;
        }
        s->tn[3 * (int64_t)o + j] = N;
        s->start_of[vslot(s, ea[k])] = N;
    }
    for (int64_t k = 0; k < nbnd; ++k) {
        int32_t N = newt[k];
        int32_t M = s->start_of[vslot(s, eb[k])]; /* new triangle (eb, c, q) */
        s->tn[3 * (int64_t)N + 0] = M;             /* N's edge (eb, q) ...     */
        s->tn[3 * (int64_t)M + 1] = N;             /* ... is M's edge (q, eb)  */
        for (int i = 0; i < 3; ++i) {
            int32_t w = s->tv[3 * (int64_t)N + i];
            if (w != ORC_GHOST)
                s->vtri[w] = N;
        }
    }
    for (int64_t k = 0; k < nbnd; ++k)
        s->start_of[vslot(s, ea[k])] = -1;
    s->last_tri = newt[0];
    s->grid[grid_cell(s, q)] = q;
    free(newt); free(ea); free(eb);
    return ORC_OK;
}

static int cmp_tri(const void *pa, const void *pb)
{
    const int32_t *a = (const int32_t *)pa, *b = (const int32_t *)pb;
    for (int i = 0; i < 3; ++i) {
        if (a[i] < b[i]) return -1;
        if (a[i] > b[i]) return 1;
    }
    return 0;
}

static int cmp_key(const void *pa, const void *pb)
{
    uint64_t a = *(const uint64_t *)pa, b = *(const uint64_t *)pb;
    return (a > b) - (a < b);
}

/* Input checks shared by the oracle's entry points: range and distinctness. */
static int check_points(const int32_t *xy, int64_t n)
{
    if (!xy || n < 0)
        return ORC_ERR_ARG;
    for (int64_t i = 0; i < 2 * n; ++i)
        if (xy[i] < 0 || xy[i] >= COORD_LIMIT)
            return ORC_ERR_RANGE;
    uint64_t *key = (uint64_t *)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    if (!key)
        return ORC_ERR_NOMEM;
    for (int64_t i = 0; i < n; ++i)
        key[i] = ((uint64_t)(uint32_t)xy[2 * i] << 32) | (uint32_t)xy[2 * i + 1];
    qsort(key, (size_t)n, sizeof(uint64_t), cmp_key);
    int dup = 0;
    for (int64_t i = 1; i < n; ++i)
        if (key[i] == key[i - 1])
            dup = 1;
    free(key);
    return dup ? ORC_ERR_DUPLICATE : ORC_OK;
}

/* Canonical form of the output (Fig. 4, the triangulation after a step): every finite
 * triangle counter-clockwise and rotated so its smallest id comes first; the list
 * sorted lexicographically.  It has 2n - 2 - h rows, h = points on the hull
 * boundary (collinear ones included). */
static int64_t emit_canonical(const bw_t *s, int32_t *out, int64_t cap, int64_t *n_tri)
{
    int64_t cnt = 0;
    for (int64_t t = 0; t < s->nt; ++t)
        if (!is_ghost_tri(s, (int32_t)t))
            ++cnt;
    *n_tri = cnt;
    if (cnt > cap || (cnt > 0 && !out))
        return ORC_ERR_CAPACITY;
    int64_t k = 0;
    for (int64_t t = 0; t < s->nt; ++t) {
        if (is_ghost_tri(s, (int32_t)t))
            continue;
        const int32_t *v = s->tv + 3 * t;
        int r = 0;
        if (v[1] < v[r]) r = 1;
        if (v[2] < v[r]) r = 2;
        out[3 * k] = v[r];
        out[3 * k + 1] = v[(r + 1) % 3];
        out[3 * k + 2] = v[(r + 2) % 3];
        ++k;
    }
    qsort(out, (size_t)cnt, 3 * sizeof(int32_t), cmp_tri);
    return ORC_OK;
}

/* Connect the neighbour fields of a small set of triangles by matching edges. */
static void link_small(bw_t *s, const int32_t *ts, int m)
{
    for (int x = 0; x < m; ++x)
        for (int i = 0; i < 3; ++i) {
            const int32_t *v = s->tv + 3 * (int64_t)ts[x];
            int32_t a = v[(i + 1) % 3], b = v[(i + 2) % 3];
            for (int y = 0; y < m; ++y) {
                if (y == x) continue;
                int j = edge_index(s, ts[y], a, b);
                if (j >= 0)
                    s->tn[3 * (int64_t)ts[x] + i] = ts[y];
            }
        }
}

/* DT of n distinct points (Section I definition, Section IV Bowyer-Watson).
 * out receives the canonical list (3 ids per row), n_tri its length.
 * The seed only chooses the insertion order; the output does not depend on it. */
int oracle_delaunay(const int32_t *xy, int64_t n, uint64_t seed, int32_t *out, int64_t cap,
                    int64_t *n_tri)
{
    if (!n_tri)
        return ORC_ERR_ARG;
    *n_tri = 0;
    int rc = check_points(xy, n);
    if (rc)
        return rc;
    if (n < 3)
        return ORC_ERR_DEGENERATE;

    bw_t s;
    memset(&s, 0, sizeof s);
    s.xy = xy;
    s.n = n;
    s.cap = 2 * n - 2 + 8;
    s.tv = (int32_t *)malloc((size_t)s.cap * 3 * sizeof(int32_t));
    s.tn = (int32_t *)malloc((size_t)s.cap * 3 * sizeof(int32_t));
    s.stamp = (int64_t *)malloc((size_t)s.cap * sizeof(int64_t));
    s.vtri = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    s.start_of = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    /* grid hint: about two points per cell */
    int64_t minx = px(xy, 0), miny = py(xy, 0), maxx = minx, maxy = miny;
    for (int64_t i = 1; i < n; ++i) {
        if (px(xy, i) < minx) minx = px(xy, i);
        if (px(xy, i) > maxx) maxx = px(xy, i);
        if (py(xy, i) < miny) miny = py(xy, i);
        if (py(xy, i) > maxy) maxy = py(xy, i);
    }
    int64_t span = (maxx - minx > maxy - miny ? maxx - minx : maxy - miny) + 1;
    int64_t want = 1;
    while (want * want * 2 < n) want *= 2;
    s.gshift = 0;
    while ((span >> s.gshift) > want) s.gshift++;
    s.gdim = (span >> s.gshift) + 1;
    s.gx0 = minx;
    s.gy0 = miny;
    s.grid = (int32_t *)malloc((size_t)(s.gdim * s.gdim) * sizeof(int32_t));
    if (!s.tv || !s.tn || !s.stamp || !s.vtri || !s.start_of || !order || !s.grid) {
        rc = ORC_ERR_NOMEM;
        goto done;
    }
    for (int64_t i = 0; i < s.cap; ++i) s.stamp[i] = -1;
    for (int64_t i = 0; i < n; ++i) s.vtri[i] = -1;
    for (int64_t i = 0; i <= n; ++i) s.start_of[i] = -1;
    for (int64_t i = 0; i < s.gdim * s.gdim; ++i) s.grid[i] = -1;

    /* random insertion order (Fisher-Yates) */
    uint64_t st = seed;
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)(splitmix64(&st) % (uint64_t)(i + 1));
        int32_t tmp = order[i]; order[i] = order[j]; order[j] = tmp;
    }
    /* first triangle: the first two points and the first point not collinear with them */
    int32_t a = order[0], b = order[1], c = -1;
    int64_t ci = -1;
    for (int64_t i = 2; i < n; ++i)
        if (oracle_orient2d(xy, a, b, order[i]) != 0) {
            c = order[i];
            ci = i;
            break;
        }
    if (c < 0) {
        rc = ORC_ERR_DEGENERATE; /* all points collinear: no triangle exists */
        goto done;
    }
    if (oracle_orient2d(xy, a, b, c) < 0) {
        int32_t tmp = b; b = c; c = tmp;
    }
    {
        int32_t init[4][3] = {{a, b, c}, {c, b, ORC_GHOST}, {a, c, ORC_GHOST}, {b, a, ORC_GHOST}};
        int32_t ts[4] = {0, 1, 2, 3};
        for (int t = 0; t < 4; ++t)
            for (int i = 0; i < 3; ++i)
                s.tv[3 * t + i] = init[t][i];
        s.nt = 4;
        link_small(&s, ts, 4);
        s.vtri[a] = 0; s.vtri[b] = 0; s.vtri[c] = 0;
        s.last_tri = 0;
        s.grid[grid_cell(&s, a)] = a;
        s.grid[grid_cell(&s, b)] = b;
        s.grid[grid_cell(&s, c)] = c;
    }
    for (int64_t i = 2; i < n; ++i) {
        if (i == ci)
            continue;
        rc = bw_insert(&s, order[i], i);
        if (rc)
            goto done;
    }
    if (s.nt != 2 * n - 2) {
        rc = ORC_ERR_INTERNAL;
        goto done;
    }
    rc = (int)emit_canonical(&s, out, cap, n_tri);
done:
    free(s.tv); free(s.tn); free(s.stamp); free(s.vtri); free(s.start_of);
    free(s.grid); free(s.cav); free(s.bnd); free(order);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Certifier: is a given triangle list the SoS Delaunay triangulation of P?
 *
 * Used where a full Bowyer-Watson comparison is too slow.  It checks properties
 * that together characterise the DT (Section I definition; Lawson's lemma that a
 * triangulation whose every interior edge is locally Delaunay is the DT):
 *   1. ids in range, every triangle strictly counter-clockwise;
 *   2. every directed edge used once; interior edges paired;
 *   3. the unpaired edges form one closed boundary cycle that turns left or goes
 *      straight at every vertex and winds exactly once (a convex polygon);
 *   4. every point is a vertex, and T = 2n - 2 - h (Euler, h = boundary vertices);
 *   5. every interior edge is locally Delaunay under the SoS incircle.
 * Returns 0 when all hold, else the number of the first failed property; detail[0]
 * receives the offending triangle or edge index.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint64_t key; /* (a << 32) | b for the directed edge a->b */
    int64_t tri;
    int32_t opp;
} dedge_t;

static int cmp_dedge(const void *pa, const void *pb)
{
    uint64_t a = ((const dedge_t *)pa)->key, b = ((const dedge_t *)pb)->key;
    return (a > b) - (a < b);
}

static int64_t find_dedge(const dedge_t *e, int64_t m, uint64_t key)
{
    int64_t lo = 0, hi = m - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (e[mid].key == key) return mid;
        if (e[mid].key < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* half-plane index of a direction: 0 for angles in [0, pi), 1 for [pi, 2 pi) */
static int dir_half(int64_t dx, int64_t dy) { return (dy < 0 || (dy == 0 && dx < 0)) ? 1 : 0; }

/* is direction (ax,ay) strictly before (bx,by) in counter-clockwise angle from +x? */
static int dir_less(int64_t ax, int64_t ay, int64_t bx, int64_t by)
{
    int ha = dir_half(ax, ay), hb = dir_half(bx, by);
    if (ha != hb) return ha < hb;
    return ax * by - ay * bx > 0;
}

int oracle_check_dt(const int32_t *xy, int64_t n, const int32_t *tris, int64_t T, int64_t *detail)
{
    int64_t dummy;
    if (!detail) detail = &dummy;
    *detail = -1;
    if (!xy || n < 3 || (T > 0 && !tris))
        return 1;
    /* 1 */
    for (int64_t t = 0; t < T; ++t) {
        for (int i = 0; i < 3; ++i)
            if (tris[3 * t + i] < 0 || tris[3 * t + i] >= n) { *detail = t; return 1; }
        if (oracle_orient2d(xy, tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]) <= 0) { *detail = t; return 1; }
    }
    /* 2 */
    int64_t m = 3 * T;
    dedge_t *e = (dedge_t *)malloc((size_t)(m ? m : 1) * sizeof(dedge_t));
    char *used = (char *)calloc((size_t)n, 1);
    int32_t *bnext = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!e || !used || !bnext) { free(e); free(used); free(bnext); return 2; }
    for (int64_t t = 0; t < T; ++t)
        for (int i = 0; i < 3; ++i) {
            int32_t a = tris[3 * t + (i + 1) % 3], b = tris[3 * t + (i + 2) % 3];
            e[3 * t + i].key = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
            e[3 * t + i].tri = t;
            e[3 * t + i].opp = tris[3 * t + i];
            used[tris[3 * t + i]] = 1;
        }
    qsort(e, (size_t)m, sizeof(dedge_t), cmp_dedge);
    int rc = 0;
    for (int64_t k = 1; k < m; ++k)
        if (e[k].key == e[k - 1].key) { *detail = e[k].tri; rc = 2; goto out; }
    /* 3 and 5 */
    for (int64_t v = 0; v < n; ++v) bnext[v] = -1;
    int64_t nb = 0;
    int32_t bstart = -1;
    for (int64_t k = 0; k < m; ++k) {
        int32_t a = (int32_t)(e[k].key >> 32), b = (int32_t)(e[k].key & 0xffffffffu);
        uint64_t twin = ((uint64_t)(uint32_t)b << 32) | (uint32_t)a;
        int64_t j = find_dedge(e, m, twin);
        if (j < 0) {
            if (bnext[a] != -1) { *detail = e[k].tri; rc = 3; goto out; }
            bnext[a] = b;
            ++nb;
            bstart = a;
        } else if (a < b) {
            /* interior edge: the far vertex must lie outside the near circle */
            const int32_t *t = tris + 3 * e[k].tri;
            if (oracle_incircle_sos(xy, t[0], t[1], t[2], e[j].opp) >= 0) { *detail = e[k].tri; rc = 5; goto out; }
        }
    }
    if (nb < 3) { rc = 3; goto out; }
    {
        /* one cycle through all boundary edges, convex, winding once */
        int64_t steps = 0, wraps = 0;
        int32_t v = bstart;
        do {
            int32_t w = bnext[v];
            if (w < 0) { *detail = v; rc = 3; goto out; }
            int32_t x = bnext[w];
            if (x < 0) { *detail = w; rc = 3; goto out; }
            int o = oracle_orient2d(xy, v, w, x);
            if (o < 0) { *detail = w; rc = 3; goto out; }
            if (o == 0 && !strictly_between(xy, v, x, w)) { *detail = w; rc = 3; goto out; }
            int64_t d1x = px(xy, w) - px(xy, v), d1y = py(xy, w) - py(xy, v);
            int64_t d2x = px(xy, x) - px(xy, w), d2y = py(xy, x) - py(xy, w);
            if (dir_less(d2x, d2y, d1x, d1y)) ++wraps;
            v = w;
            if (++steps > nb) { rc = 3; goto out; }
        } while (v != bstart);
        if (steps != nb || wraps != 1) { *detail = steps; rc = 3; goto out; }
    }
    /* 4 */
    for (int64_t v = 0; v < n; ++v)
        if (!used[v]) { *detail = v; rc = 4; goto out; }
    if (T != 2 * n - 2 - nb) { *detail = T; rc = 4; goto out; }
out:
    free(e); free(used); free(bnext);
    return rc;
}

/* Library identity for the loader tests. */
int oracle_version(void) { return 1; }
