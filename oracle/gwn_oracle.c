/*
 * CPU oracle for generalized winding numbers of triangle meshes.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library never does, and the two
 * share no source.
 *
 * What it computes (citations are to the paper, arXiv 2605.01536):
 *
 *   oracle_direct     w(q) = (1/4pi) * sum_T Area(T), the signed solid-angle sum
 *                     (Sec. 3.1, Eqs. 1-2), each area by the van Oosterom-Strackee
 *                     formula on unit vectors (Sec. 3.3), in FP64 with a
 *                     double-double accumulator (the ground-truth protocol of
 *                     Sec. 5.2).
 *   oracle_chi        the signed number of crossings of the ray q + t(0,0,1),
 *                     t > 0, with the mesh (Sec. 3.2), a crossing counting the sign
 *                     of (0,0,1).n.  Every predicate is evaluated exactly on the
 *                     FP32 inputs with the symbolic perturbation
 *                     q_eps = q + (e1, e2, e3), e3 << e2 << e1 (Supp. S2.1).
 *   oracle_boundary   the oriented boundary edges dM: interior edges cancel in
 *                     pairs (Sec. 4.1, Eq. 9); an undirected edge {u,v} with net
 *                     multiplicity m = #(u->v) - #(v->u) contributes |m| copies.
 *   oracle_antipodal  w(q) = chi + (1/4pi) sum_{(a,b) in dM} Area(A, B, x1),
 *                     x1 = -(0,0,1) (Eq. 9, Algorithm 1 with the fixed direction of
 *                     Supp. S2.1), FP64 areas, double-double accumulation; where the
 *                     area's atan2 is on its branch cut (denominator < 0) the sign of
 *                     the numerator is the exact perturbed sign of the same 2-D edge
 *                     predicate the crossing test uses (Supp. S2.1, last paragraph).
 *
 *   oracle_gradient   grad w(q) = (1/4pi) sum_{(a,b) in dM} (c_n g_n + c_d g_d)
 *                     (Supp. S4, Algorithm 3) for an arbitrary antipode x1: the
 *                     crossing count is piecewise constant, so only the boundary
 *                     terms carry a gradient.  FP64, double-double accumulation.
 *
 *   oracle_chi_fixed, oracle_antipodal_fixed
 *                     the same with the predicates decided on the inputs snapped to
 *                     a 30-bit fixed-point grid over the mesh's bounding box
 *                     (Supp. S2.1), in 128-bit integers.
 *
 * Exact arithmetic: every FP32 value is an integer multiple of 2^-149, so the
 * predicates are evaluated on big integers (the inputs scaled by 2^149) with a
 * fixed-width sign-magnitude integer type written below.  No floating-point
 * filter is used anywhere in this file.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI_D 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Double-double accumulation (Knuth's TwoSum, then renormalisation).         */
/* ------------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd_t;

static void dd_add(dd_t *s, double x)
{
    double a = s->hi;
    double sum = a + x;
    double bv = sum - a;
    double av = sum - bv;
    double err = (a - av) + (x - bv);
    double lo = s->lo + err;
    double hi = sum + lo;
    s->lo = lo - (hi - sum);
    s->hi = hi;
}

static double dd_value(const dd_t *s) { return s->hi + s->lo; }

/* ------------------------------------------------------------------------ */
/* Fixed-width signed big integers.                                          */
/* An FP32 input scaled by 2^149 has at most 277 bits (9 limbs); the largest  */
/* expression below is a sum of products of three differences (<= 28 limbs). */
/* ------------------------------------------------------------------------ */
#define NL 32
typedef struct { int s; int n; uint32_t m[NL]; } big;  /* value = s * sum m[i] 2^(32i) */

static void big_zero(big *r) { r->s = 0; r->n = 0; }

static void big_trim(big *r)
{
    while (r->n > 0 && r->m[r->n - 1] == 0) r->n--;
    if (r->n == 0) r->s = 0;
}

/* exact integer value of f * 2^149 */
static big big_from_f32(float f)
{
    big r;
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t E = (u >> 23) & 0xffu, M = u & 0x7fffffu;
    uint64_t mant = (E == 0) ? M : (M | 0x800000u);
    int shift = (E == 0) ? 0 : (int)E - 1;
    memset(r.m, 0, sizeof r.m);
    r.n = 0;
    r.s = 0;
    if (mant == 0) return r;
    int limb = shift / 32, bit = shift % 32;
    uint64_t v = mant << bit;
    r.m[limb] = (uint32_t)v;
    r.m[limb + 1] = (uint32_t)(v >> 32);
    r.n = limb + 2;
    r.s = (u >> 31) ? -1 : 1;
    big_trim(&r);
    return r;
}

static int mag_cmp(const big *a, const big *b)
{
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int i = a->n - 1; i >= 0; --i)
        if (a->m[i] != b->m[i]) return a->m[i] < b->m[i] ? -1 : 1;
    return 0;
}

static void mag_add(big *r, const big *a, const big *b)
{
    int n = a->n > b->n ? a->n : b->n;
    uint64_t c = 0;
    for (int i = 0; i < n; ++i) {
        uint64_t t = c + (i < a->n ? a->m[i] : 0) + (i < b->n ? b->m[i] : 0);
        r->m[i] = (uint32_t)t;
        c = t >> 32;
    }
    if (n >= NL) {
        if (c) { fprintf(stderr, "oracle bigint overflow\n"); abort(); }
        r->n = n;
        return;
    }
    r->m[n] = (uint32_t)c;
    r->n = n + 1;
}

/* |a| >= |b| */
static void mag_sub(big *r, const big *a, const big *b)
{
    int64_t br = 0;
    for (int i = 0; i < a->n; ++i) {
        int64_t t = (int64_t)a->m[i] - (i < b->n ? b->m[i] : 0) - br;
        br = t < 0;
        r->m[i] = (uint32_t)(t + (br ? ((int64_t)1 << 32) : 0));
    }
    r->n = a->n;
}

static big big_add(const big *a, const big *b)
{
    big r;
    if (a->s == 0) return *b;
    if (b->s == 0) return *a;
    if (a->s == b->s) {
        mag_add(&r, a, b);
        r.s = a->s;
    } else {
        int c = mag_cmp(a, b);
        if (c == 0) { big_zero(&r); return r; }
        if (c > 0) { mag_sub(&r, a, b); r.s = a->s; }
        else       { mag_sub(&r, b, a); r.s = b->s; }
    }
    big_trim(&r);
    return r;
}

static big big_sub(const big *a, const big *b)
{
    big nb = *b;
    nb.s = -nb.s;
    return big_add(a, &nb);
}

static big big_mul(const big *a, const big *b)
{
    big r;
    if (a->s == 0 || b->s == 0) { big_zero(&r); return r; }
    int n = a->n + b->n;
    if (n > NL) { fprintf(stderr, "oracle bigint overflow\n"); abort(); }
    memset(r.m, 0, sizeof(uint32_t) * (size_t)n);
    for (int i = 0; i < a->n; ++i) {
        uint64_t c = 0;
        for (int j = 0; j < b->n; ++j) {
            uint64_t t = (uint64_t)a->m[i] * b->m[j] + r.m[i + j] + c;
            r.m[i + j] = (uint32_t)t;
            c = t >> 32;
        }
        r.m[i + b->n] = (uint32_t)c;
    }
    r.n = n;
    r.s = a->s * b->s;
    big_trim(&r);
    return r;
}

static int sgn_f(float a, float b) { return (a > b) - (a < b); }   /* sign(a - b), exact */

/* ------------------------------------------------------------------------ */
/* Predicates (Supp. S2.1).                                                  */
/* ------------------------------------------------------------------------ */

/* Real part of the 2-D edge classification of (x, y) against the projected edge
 * p_i -> p_j:  (x - x_i)(y_i - y_j) + (y - y_i)(x_j - x_i).  Exact. */
static int edge_real_sign(float x, float y, float xi, float yi, float xj, float yj)
{
    big X = big_from_f32(x), Y = big_from_f32(y);
    big Xi = big_from_f32(xi), Yi = big_from_f32(yi);
    big Xj = big_from_f32(xj), Yj = big_from_f32(yj);
    big d1 = big_sub(&X, &Xi), d2 = big_sub(&Yi, &Yj);
    big d3 = big_sub(&Y, &Yi), d4 = big_sub(&Xj, &Xi);
    big t1 = big_mul(&d1, &d2), t2 = big_mul(&d3, &d4);
    big s = big_add(&t1, &t2);
    return s.s;
}

/* Sign of the perturbed classification
 *   (x + e1 - x_i)(y_i - y_j) + (y + e2 - y_i)(x_j - x_i)
 * taken in the order: real part, e1 coefficient (y_i - y_j), e2 coefficient
 * (x_j - x_i).  0 only for an edge whose projection is a single point. */
int oracle_edge_sos(float x, float y, float xi, float yi, float xj, float yj)
{
    int s = edge_real_sign(x, y, xi, yi, xj, yj);
    if (s) return s;
    s = sgn_f(yi, yj);
    if (s) return s;
    return sgn_f(xj, xi);
}

/* Perturbed sign of n.(a - q_eps), n = (b - a) x (c - a): the real part
 * n.(a - q) first, then the coefficients of e1, e2, e3: -n_x, -n_y, -n_z. */
int oracle_plane_sos(const float *q, const float *a, const float *b, const float *c)
{
    big A[3], B[3], C[3], Q[3];
    for (int k = 0; k < 3; ++k) {
        A[k] = big_from_f32(a[k]); B[k] = big_from_f32(b[k]);
        C[k] = big_from_f32(c[k]); Q[k] = big_from_f32(q[k]);
    }
    big u[3], v[3], w[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = big_sub(&B[k], &A[k]);      /* b - a */
        v[k] = big_sub(&C[k], &A[k]);      /* c - a */
        w[k] = big_sub(&A[k], &Q[k]);      /* a - q */
    }
    big n[3];
    for (int k = 0; k < 3; ++k) {
        int i = (k + 1) % 3, j = (k + 2) % 3;
        big p1 = big_mul(&u[i], &v[j]), p2 = big_mul(&u[j], &v[i]);
        n[k] = big_sub(&p1, &p2);
    }
    big acc;
    big_zero(&acc);
    for (int k = 0; k < 3; ++k) {
        big p = big_mul(&n[k], &w[k]);
        acc = big_add(&acc, &p);
    }
    if (acc.s) return acc.s;
    for (int k = 0; k < 3; ++k)
        if (n[k].s) return -n[k].s;
    return 0;
}

/* Signed crossing of the ray q_eps + t(0,0,1), t > 0, with triangle (a,b,c):
 * +1 / -1 = sign of the triangle's normal z component when hit, else 0. */
int oracle_tri_crossing(const float *q, const float *a, const float *b, const float *c)
{
    /* exact early out: outside the closed xy bounding box -> not hit */
    float xmin = fminf(a[0], fminf(b[0], c[0])), xmax = fmaxf(a[0], fmaxf(b[0], c[0]));
    float ymin = fminf(a[1], fminf(b[1], c[1])), ymax = fmaxf(a[1], fmaxf(b[1], c[1]));
    if (q[0] < xmin || q[0] > xmax || q[1] < ymin || q[1] > ymax) return 0;
    int s0 = oracle_edge_sos(q[0], q[1], a[0], a[1], b[0], b[1]);
    int s1 = oracle_edge_sos(q[0], q[1], b[0], b[1], c[0], c[1]);
    int s2 = oracle_edge_sos(q[0], q[1], c[0], c[1], a[0], a[1]);
    if (s0 == 0 || s1 == 0 || s2 == 0) return 0;   /* projected edge is a point */
    if (s0 != s1 || s1 != s2) return 0;            /* projected query outside */
    int side = oracle_plane_sos(q, a, b, c);
    return side == s0 ? s0 : 0;                    /* plane above the query */
}

/* ------------------------------------------------------------------------ */
/* Exported batch entry points.                                              */
/* ------------------------------------------------------------------------ */

/* ------------------------------------------------------------------------ */
/* Fixed-point variant of the predicates (Supp. S2.1: inputs snapped to a     */
/* 30-bit grid, perturbed signs decided in integer arithmetic).  The frame:   */
/* c = centre of the vertices' bounding box, e = the smallest exponent with   */
/* max |v - c| 2^-e <= 2^29 (from frexp), X = rint((x - c) 2^-e) computed in  */
/* FP64 (exact for FP32 x near the mesh) and clamped to [-2^62, 2^62].        */
/* ------------------------------------------------------------------------ */
typedef struct { double c[3]; double scale; int e; } qframe_t;

static void qframe_from_vertices(const float *V, int64_t nv, qframe_t *f)
{
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, half = 0.0;
    for (int d = 0; d < 3; ++d) {
        lo[d] = INFINITY;
        hi[d] = -INFINITY;
    }
    for (int64_t i = 0; i < nv; ++i)
        for (int d = 0; d < 3; ++d) {
            const double v = (double)V[3 * i + d];
            if (v < lo[d]) lo[d] = v;
            if (v > hi[d]) hi[d] = v;
        }
    for (int d = 0; d < 3; ++d) {
        f->c[d] = nv > 0 ? 0.5 * (lo[d] + hi[d]) : 0.0;
        if (nv > 0) {
            const double a = hi[d] - f->c[d], b = f->c[d] - lo[d];
            if (a > half) half = a;
            if (b > half) half = b;
        }
    }
    int k = 0;
    if (half > 0.0) frexp(half, &k);
    f->e = half > 0.0 ? k - 29 : 0;
    f->scale = ldexp(1.0, -f->e);
}

static long long qsnap(float v, double c, double scale)
{
    double t = ((double)v - c) * scale;
    const double lim = 4611686018427387904.0;   /* 2^62 */
    if (t > lim) t = lim;
    if (t < -lim) t = -lim;
    return llrint(t);
}

static int sgn128(__int128 v) { return (v > 0) - (v < 0); }

/* (x + e1 - xi)(yi - yj) + (y + e2 - yi)(xj - xi): real part, then e1, e2 */
static int edge_sos_fixed(long long x, long long y, long long xi, long long yi, long long xj, long long yj)
{
    const __int128 f = (__int128)(x - xi) * (yi - yj) + (__int128)(y - yi) * (xj - xi);
    if (f != 0) return sgn128(f);
    if (yi != yj) return yi > yj ? 1 : -1;
    return (xj > xi) - (xj < xi);
}

/* n . (a - q_eps), n = (b - a) x (c - a): det[a - q, b - q, c - q], then the
 * e1, e2, e3 coefficients -n_x, -n_y, -n_z.  Called only with q's projection
 * inside the triangle, where |x, y differences| < 2^31 and the products fit. */
static int plane_sos_fixed(const long long *q, const long long *a, const long long *b, const long long *c)
{
    __int128 u[3], v[3], w[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = (__int128)a[k] - q[k];
        v[k] = (__int128)b[k] - q[k];
        w[k] = (__int128)c[k] - q[k];
    }
    const __int128 d = u[0] * (v[1] * w[2] - v[2] * w[1]) + u[1] * (v[2] * w[0] - v[0] * w[2]) +
                       u[2] * (v[0] * w[1] - v[1] * w[0]);
    if (d != 0) return sgn128(d);
    const __int128 nx = (__int128)(b[1] - a[1]) * (c[2] - a[2]) - (__int128)(b[2] - a[2]) * (c[1] - a[1]);
    if (nx != 0) return -sgn128(nx);
    const __int128 ny = (__int128)(b[2] - a[2]) * (c[0] - a[0]) - (__int128)(b[0] - a[0]) * (c[2] - a[2]);
    if (ny != 0) return -sgn128(ny);
    const __int128 nz = (__int128)(b[0] - a[0]) * (c[1] - a[1]) - (__int128)(b[1] - a[1]) * (c[0] - a[0]);
    return -sgn128(nz);
}

static int tri_crossing_fixed(const long long *q, const long long *a, const long long *b, const long long *c)
{
    long long zmax = a[2];
    if (b[2] > zmax) zmax = b[2];
    if (c[2] > zmax) zmax = c[2];
    if (q[2] >= zmax) return 0;                    /* the whole triangle at or below q_eps */
    const int s0 = edge_sos_fixed(q[0], q[1], a[0], a[1], b[0], b[1]);
    const int s1 = edge_sos_fixed(q[0], q[1], b[0], b[1], c[0], c[1]);
    const int s2 = edge_sos_fixed(q[0], q[1], c[0], c[1], a[0], a[1]);
    if (s0 == 0 || s0 != s1 || s1 != s2) return 0;
    return plane_sos_fixed(q, a, b, c) == s0 ? s0 : 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* chi with the fixed-point predicates (bits = 30) */
void oracle_chi_fixed(const float *V, int64_t nv, const int32_t *F, int64_t nt,
                      const float *Q, int64_t nq, int32_t *chi)
{
    qframe_t f;
    qframe_from_vertices(V, nv, &f);
    long long *S = (long long *)malloc(sizeof(long long) * 3 * (nv > 0 ? nv : 1));
    for (int64_t i = 0; i < nv; ++i)
        for (int d = 0; d < 3; ++d) S[3 * i + d] = qsnap(V[3 * i + d], f.c[d], f.scale);
    #pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < nq; ++i) {
        long long q[3];
        for (int d = 0; d < 3; ++d) q[d] = qsnap(Q[3 * i + d], f.c[d], f.scale);
        int32_t c = 0;
        for (int64_t t = 0; t < nt; ++t)
            c += tri_crossing_fixed(q, S + 3 * (int64_t)F[3 * t], S + 3 * (int64_t)F[3 * t + 1],
                                    S + 3 * (int64_t)F[3 * t + 2]);
        chi[i] = c;
    }
    free(S);
}

void oracle_chi(const float *V, int64_t nv, const int32_t *F, int64_t nt,
                const float *Q, int64_t nq, int32_t *chi)
{
    (void)nv;
    #pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < nq; ++i) {
        const float *q = Q + 3 * i;
        int32_t c = 0;
        for (int64_t t = 0; t < nt; ++t)
            c += oracle_tri_crossing(q, V + 3 * (int64_t)F[3 * t], V + 3 * (int64_t)F[3 * t + 1],
                                     V + 3 * (int64_t)F[3 * t + 2]);
        chi[i] = c;
    }
}

/* Signed area of the spherical triangle with unit vertices v0, v1, v2
 * (van Oosterom-Strackee, Sec. 3.3). */
static double vos_area(const double *v0, const double *v1, const double *v2, double *num_out, double *den_out)
{
    double cx = v1[1] * v2[2] - v1[2] * v2[1];
    double cy = v1[2] * v2[0] - v1[0] * v2[2];
    double cz = v1[0] * v2[1] - v1[1] * v2[0];
    double num = v0[0] * cx + v0[1] * cy + v0[2] * cz;
    double den = 1.0 + (v0[0] * v1[0] + v0[1] * v1[1] + v0[2] * v1[2])
                     + (v0[0] * v2[0] + v0[1] * v2[1] + v0[2] * v2[2])
                     + (v1[0] * v2[0] + v1[1] * v2[1] + v1[2] * v2[2]);
    if (num_out) *num_out = num;
    if (den_out) *den_out = den;
    return 2.0 * atan2(num, den);
}

static void unit_from(const float *v, const float *q, double *u)
{
    double d0 = (double)v[0] - (double)q[0];
    double d1 = (double)v[1] - (double)q[1];
    double d2 = (double)v[2] - (double)q[2];
    double l = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    u[0] = d0 / l; u[1] = d1 / l; u[2] = d2 / l;
}

void oracle_direct(const float *V, int64_t nv, const int32_t *F, int64_t nt,
                   const float *Q, int64_t nq, double *w)
{
    (void)nv;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nq; ++i) {
        const float *q = Q + 3 * i;
        dd_t acc = {0.0, 0.0};
        for (int64_t t = 0; t < nt; ++t) {
            double a[3], b[3], c[3];
            unit_from(V + 3 * (int64_t)F[3 * t], q, a);
            unit_from(V + 3 * (int64_t)F[3 * t + 1], q, b);
            unit_from(V + 3 * (int64_t)F[3 * t + 2], q, c);
            dd_add(&acc, vos_area(a, b, c, NULL, NULL));
        }
        w[i] = dd_value(&acc) / (4.0 * PI_D);
    }
}

/* Solid angle of a single triangle seen from q (for the closed-form tests). */
double oracle_triangle_area(const float *a, const float *b, const float *c, const float *q)
{
    double A[3], B[3], C[3];
    unit_from(a, q, A); unit_from(b, q, B); unit_from(c, q, C);
    return vos_area(A, B, C, NULL, NULL);
}

/* ---- boundary extraction ---- */
typedef struct { int64_t key; int32_t sgn; } hedge_t;

static int hedge_cmp(const void *x, const void *y)
{
    const hedge_t *a = x, *b = y;
    return (a->key > b->key) - (a->key < b->key);
}

/* Writes the oriented boundary edges (pairs of vertex indices) sorted by the
 * undirected key (min, max); returns their number.  `out` must hold 2*3*nt ints. */
int64_t oracle_boundary(const int32_t *F, int64_t nt, int64_t nv, int32_t *out)
{
    hedge_t *h = malloc(sizeof(hedge_t) * (size_t)(3 * nt > 0 ? 3 * nt : 1));
    int64_t nh = 0;
    for (int64_t t = 0; t < nt; ++t)
        for (int e = 0; e < 3; ++e) {
            int64_t u = F[3 * t + e], v = F[3 * t + (e + 1) % 3];
            if (u == v) continue;   /* an edge from a vertex to itself is a zero chain */
            int64_t lo = u < v ? u : v, hi = u < v ? v : u;
            h[nh].key = lo * nv + hi;
            h[nh].sgn = (u < v) ? 1 : -1;
            ++nh;
        }
    qsort(h, (size_t)nh, sizeof(hedge_t), hedge_cmp);
    int64_t nb = 0;
    for (int64_t i = 0; i < nh;) {
        int64_t j = i, m = 0;
        while (j < nh && h[j].key == h[i].key) m += h[j++].sgn;
        int64_t lo = h[i].key / nv, hi = h[i].key % nv;
        for (int64_t r = 0; r < (m > 0 ? m : -m); ++r) {
            out[2 * nb] = (int32_t)(m > 0 ? lo : hi);
            out[2 * nb + 1] = (int32_t)(m > 0 ? hi : lo);
            ++nb;
        }
        i = j;
    }
    free(h);
    return nb;
}

/* q lies on the closed segment [a, b] (exactly). */
static int on_segment(const float *q, const float *a, const float *b)
{
    for (int k = 0; k < 3; ++k) {
        float lo = fminf(a[k], b[k]), hi = fmaxf(a[k], b[k]);
        if (q[k] < lo || q[k] > hi) return 0;
    }
    /* (b - a) x (q - a) == 0 */
    big A[3], B[3], Q[3], u[3], v[3];
    for (int k = 0; k < 3; ++k) {
        A[k] = big_from_f32(a[k]); B[k] = big_from_f32(b[k]); Q[k] = big_from_f32(q[k]);
        u[k] = big_sub(&B[k], &A[k]); v[k] = big_sub(&Q[k], &A[k]);
    }
    for (int k = 0; k < 3; ++k) {
        int i = (k + 1) % 3, j = (k + 2) % 3;
        big p1 = big_mul(&u[i], &v[j]), p2 = big_mul(&u[j], &v[i]);
        big c = big_sub(&p1, &p2);
        if (c.s) return 0;
    }
    return 1;
}

/* Limit of the boundary term of the edge (u, v) when u lies exactly on the
 * query's vertical ray (u - q = (0, 0, h), h > 0) and the query is perturbed by
 * (e1, e2, e3): the unit vector to u tends to (-e1/h, -e2/h, 1), which gives
 * Area = 2 atan2(r_y, -r_x) with r = v - q; for r_y == 0 the e2 order decides:
 * -2pi for r_x > 0 and 0 for r_x < 0.  Sets *bad when r_x == r_y == 0. */
static double apex_limit(const float *v, const float *q, int *bad)
{
    double rx = (double)v[0] - (double)q[0];
    double ry = (double)v[1] - (double)q[1];
    if (v[1] != q[1]) return 2.0 * atan2(ry, -rx);
    if (v[0] > q[0]) return -2.0 * PI_D;
    if (v[0] < q[0]) return 0.0;
    *bad = 1;
    return 0.0;
}

/* flags: bit 0 = the query lies on the boundary curve (w undefined there);
 *        bit 1 = a boundary edge is vertical and on the query's vertical line
 *                (no perturbation order resolves its term; term taken as 0). */
static void antipodal_core(const float *V, int64_t nv, const int32_t *E, int64_t nb,
                           const float *Q, int64_t nq, const int32_t *chi,
                           double *w, int32_t *flags, const qframe_t *qf)
{
    (void)nv;
    const double x1[3] = {0.0, 0.0, -1.0};
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nq; ++i) {
        const float *q = Q + 3 * i;
        dd_t acc = {0.0, 0.0};
        int fl = 0;
        for (int64_t e = 0; e < nb; ++e) {
            const float *a = V + 3 * (int64_t)E[2 * e];
            const float *b = V + 3 * (int64_t)E[2 * e + 1];
            if (on_segment(q, a, b)) { fl |= 1; continue; }
            int a_up = (a[0] == q[0] && a[1] == q[1]);
            int b_up = (b[0] == q[0] && b[1] == q[1]);
            double term;
            if (a_up && b_up) {            /* vertical edge on the query's line */
                fl |= 2;
                term = 0.0;
            } else if (a_up && a[2] > q[2]) {
                int bad = 0;
                term = apex_limit(b, q, &bad);
                if (bad) fl |= 2;
            } else if (b_up && b[2] > q[2]) {
                int bad = 0;
                term = -apex_limit(a, q, &bad);
                if (bad) fl |= 2;
            } else {
                double A[3], B[3], num, den;
                unit_from(a, q, A);
                unit_from(b, q, B);
                term = vos_area(A, B, x1, &num, &den);
                if (den < 0.0) {
                    /* branch cut of atan2: the numerator x1.(A x B) has the sign of
                     * minus the perturbed 2-D edge classification of a -> b */
                    int s = qf ? -edge_sos_fixed(qsnap(q[0], qf->c[0], qf->scale), qsnap(q[1], qf->c[1], qf->scale),
                                                 qsnap(a[0], qf->c[0], qf->scale), qsnap(a[1], qf->c[1], qf->scale),
                                                 qsnap(b[0], qf->c[0], qf->scale), qsnap(b[1], qf->c[1], qf->scale))
                               : -oracle_edge_sos(q[0], q[1], a[0], a[1], b[0], b[1]);
                    term = 2.0 * atan2(fabs(num), den);
                    if (s < 0) term = -term;
                }
            }
            dd_add(&acc, term);
        }
        w[i] = (double)chi[i] + dd_value(&acc) / (4.0 * PI_D);
        flags[i] = fl;
    }
}

/* ------------------------------------------------------------------------ */
/* Gradient of w with respect to the query point (Supp. S4, Algorithm 3).    */
/* For each boundary edge (a, b), with r0 = a - p, r1 = b - p, l = |r|,      */
/* v = r / l:                                                                */
/*   n   = x1 . (r0 x r1)                       (the VOS numerator)          */
/*   d   = l0 l1 + l1 x1.r0 + l0 x1.r1 + r0.r1  (the VOS denominator)        */
/*   c_n = 2 d / (n^2 + d^2),  c_d = -2 n / (n^2 + d^2)                      */
/*         (2 atan2(n, d) differentiated by n and by d)                      */
/*   g_n = -(r1 x x1 + x1 x r0)                 (dn / dp)                    */
/*   t1  = l1 (x1 + v1 + (1 + x1.v1) v0),  t2 = l0 (x1 + v0 + (1 + x1.v0) v1) */
/*   g_d = -(t1 + t2)                           (dd / dp)                    */
/* and grad w = (1/4pi) sum (c_n g_n + c_d g_d).                             */
/* Also returned per query (for error bounds): sum |term| and                */
/* sum |term| / rho, rho = sqrt(n^2 + d^2) / (l0 l1), the modulus of the     */
/* VOS pair for unit vectors.  flags bit 0: q on a boundary segment; bit 1:  */
/* a term with rho = 0 (an endpoint in direction -x1 or the two endpoints    */
/* opposite), skipped.                                                       */
/* ------------------------------------------------------------------------ */
static void cross3(const double *a, const double *b, double *r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

void oracle_gradient(const float *V, int64_t nv, const int32_t *E, int64_t nb,
                     const float *Q, int64_t nq, const double *x1,
                     double *grad, double *abs_sum, double *cond_sum, int32_t *flags)
{
    (void)nv;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nq; ++i) {
        const float *q = Q + 3 * i;
        dd_t acc[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        double sabs = 0.0, scond = 0.0;
        int fl = 0;
        for (int64_t e = 0; e < nb; ++e) {
            const float *a = V + 3 * (int64_t)E[2 * e];
            const float *b = V + 3 * (int64_t)E[2 * e + 1];
            if (on_segment(q, a, b)) { fl |= 1; continue; }
            double r0[3], r1[3], v0[3], v1[3];
            for (int k = 0; k < 3; ++k) {
                r0[k] = (double)a[k] - (double)q[k];
                r1[k] = (double)b[k] - (double)q[k];
            }
            const double l0 = sqrt(dot3(r0, r0)), l1 = sqrt(dot3(r1, r1));
            for (int k = 0; k < 3; ++k) {
                v0[k] = r0[k] / l0;
                v1[k] = r1[k] / l1;
            }
            double c01[3];
            cross3(r0, r1, c01);
            const double n = dot3(x1, c01);
            const double d = l0 * l1 + l1 * dot3(x1, r0) + l0 * dot3(x1, r1) + dot3(r0, r1);
            const double m2 = n * n + d * d;
            const double rho = sqrt(m2) / (l0 * l1);
            if (!(rho > 0.0)) { fl |= 2; continue; }
            const double cn = 2.0 * d / m2, cd = -2.0 * n / m2;
            double t_a[3], t_b[3], gn[3], gd[3];
            cross3(r1, x1, t_a);
            cross3(x1, r0, t_b);
            for (int k = 0; k < 3; ++k) gn[k] = -(t_a[k] + t_b[k]);
            const double x1v1 = dot3(x1, v1), x1v0 = dot3(x1, v0);
            for (int k = 0; k < 3; ++k) {
                const double t1 = l1 * (x1[k] + v1[k] + (1.0 + x1v1) * v0[k]);
                const double t2 = l0 * (x1[k] + v0[k] + (1.0 + x1v0) * v1[k]);
                gd[k] = -(t1 + t2);
            }
            double mag = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double term = cn * gn[k] + cd * gd[k];
                dd_add(&acc[k], term);
                mag += term * term;
            }
            mag = sqrt(mag);
            sabs += mag;
            scond += mag / rho;
        }
        for (int k = 0; k < 3; ++k) grad[3 * i + k] = dd_value(&acc[k]) / (4.0 * PI_D);
        abs_sum[i] = sabs / (4.0 * PI_D);
        cond_sum[i] = scond / (4.0 * PI_D);
        flags[i] = fl;
    }
}

void oracle_antipodal(const float *V, int64_t nv, const int32_t *E, int64_t nb,
                      const float *Q, int64_t nq, const int32_t *chi,
                      double *w, int32_t *flags)
{
    antipodal_core(V, nv, E, nb, Q, nq, chi, w, flags, NULL);
}

/* the antipodal w with the branch-cut signs taken on the snapped integers (bits = 30) */
void oracle_antipodal_fixed(const float *V, int64_t nv, const int32_t *E, int64_t nb,
                            const float *Q, int64_t nq, const int32_t *chi,
                            double *w, int32_t *flags)
{
    qframe_t f;
    qframe_from_vertices(V, nv, &f);
    antipodal_core(V, nv, E, nb, Q, nq, chi, w, flags, &f);
}
