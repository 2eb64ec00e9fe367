/*
 * ivm_oracle.c -- CPU oracle for the inter-visibility matrix, the per-snapshot
 * inter-visibility table and the image-tree path sets.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * definition that the CUDA library is compared against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It shares
 * no code, header, table or helper with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Everything is brute force: every sample pair against every triangle of the
 * scene, no acceleration structure, exact __int128 arithmetic throughout.
 *
 * The definition (paper sections in brackets):
 *
 *  1. Scale.  Coordinates (integer cm) are multiplied by 2s, s = samples per
 *     side, so that every sample point is an integer.  Facet f is the
 *     parallelogram {o + a u + b v : a, b in [0,1]}; its outward normal is
 *     n_f = u x v.  It is split into triangles A = (o, o+u, o+u+v) and
 *     B = (o, o+u+v, o+v) [the scene's faces are triangulated, Sec. IV-B].
 *     Samples are the s*s cell centres p_ab = 2s o + (2a+1) u + (2b+1) v.
 *  2. Facing.  front(x, f) <=> n_f . (x - 2s o_f) > 0.  Only the outward
 *     side of a face can be visible, and an angle of 180 degrees or more
 *     counts as not visible [Sec. II-B, Eq. (2)], hence the strict sign.
 *  3. Occlusion ("intersection judgment") [Abstract; Sec. I contributions;
 *     Sec. II-B: the reference face reaches the aim face with no other
 *     obstacle; Sec. III-A: blockage by nearby buildings].
 *     blocked(P, Q) <=> some triangle of the scene meets the OPEN segment
 *     {P + l (Q - P) : 0 < l < 1}; triangles are CLOSED (touching blocks).
 *  4. Matrix [Sec. II].  M_ij = [i != j] and there are samples p_a of i and
 *     q_b of j with front(q_b, i), front(p_a, j) and not blocked(p_a, q_b).
 *     Partial visibility counts as visible [Sec. III-A, Fig. 4].  The Tx is
 *     not involved [Sec. II-B: Tx-to-reference-face visibility is assumed].
 *  5. Table [Sec. III-B/C, Table II].  vis_X[t][j] = front(X_t, j) and some
 *     sample q_b of j has not blocked(X_t, q_b), for X in {Tx, Rx};
 *     los[t] = not blocked(Tx_t, Rx_t) (1 when Tx_t = Rx_t).
 *  6. Image tree [Sec. II intro; Sec. III-B, Table II rows are (parent =
 *     transmitter, reference face, aim face); Sec. III-C].  Order-k paths are
 *     (f1..fk) with vis_Tx[f1], M[f_m][f_m+1] for every hop, vis_Rx[fk].
 *     Order 0 is the direct path (los).  Paths are enumerated by depth-first
 *     search; the summary per (snapshot, order) is the path count and two
 *     fingerprints sum over paths of prod_m h_c(m, f_m) mod 2^64 with
 *     h_c(m, f) = splitmix64(seed_c ^ (m << 32) ^ f) | 1.
 *  7. Traditional per-snapshot method [Sec. IV-B, brute-force image tree per
 *     location]: the same path sets with every hop's visibility recomputed
 *     from geometry at every snapshot, no cached matrix.
 *  8. Blockage [Sec. III-C, Tables III-IV, "Blockage" column]: the first
 *     facet the segment from a source point to facet j's centre sample
 *     (a = b = floor(s/2)) meets, i.e. the hit with the smallest parameter l
 *     in (0,1) (the infimum of the hit parameters, 0 when the segment starts
 *     inside a coplanar facet); ties go to the lower facet index.  The
 *     visibility ranges themselves (runs of a table bit along the route,
 *     Tables III-IV) are read off the table in oracle/__init__.py.
 *  9. Edges [Sec. I and II: the matrix lists visible faces and edges;
 *     Sec. III-B: first-order diffraction uses the edge closest to the
 *     receiver].  Edge e = segment A -> B (cm) has s samples at the cell
 *     centres p_a = 2s A + (2a+1)(B - A), a in [0, s).  vis_X[t][e] = some
 *     sample p_a has not blocked(X_t, p_a); the nearest visible edge of X_t is
 *     the visible edge with the sample closest to X_t (squared distance over
 *     all of its samples, ties to the lower edge index), -1 if none.
 * 10. Edges as rows and columns of the matrix [Sec. I and II: per face or
 *     edge, the visible faces and edges].  Edge e also names the two facets
 *     meeting at it; a point reaches e from outside its building only when it
 *     is strictly in front of one of them (ext).  fe[i][e]: some sample p of
 *     facet i and sample q of e with front(q, i), ext(p, e) and not
 *     blocked(p, q); ee[e][g]: e != g and samples q of e, r of g with
 *     ext(r, e), ext(q, g) and not blocked(q, r).
 *
 * 11. Grid mode.  The same matrix and table entries, each decided by the
 *     same triangle test on the same triangles; a segment is only tested
 *     against the triangles an exact xy grid cannot rule out (see the grid
 *     section below for why no hit is missed).  It is the reference for
 *     scenes too large for brute force and is checked bit for bit against
 *     brute force on smaller ones.
 *
 * Bit layout of rows: bit j of a row is word j >> 5, bit j & 31 (LSB first);
 * W = ceil(N / 32) words per row; padding bits are 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* ---------------------------------------------------------------- vectors */

typedef struct { i128 x, y, z; } V;

static V mk(i128 x, i128 y, i128 z) { V r = {x, y, z}; return r; }
static V sub(V a, V b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static V add(V a, V b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static V scl(i128 k, V a) { return mk(k * a.x, k * a.y, k * a.z); }
static i128 dot(V a, V b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static V cross(V a, V b)
{
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static int sgn(i128 v) { return (v > 0) - (v < 0); }
static int veq(V a, V b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

/* orient3d(a, b, c, d) = det[b - a, c - a, d - a] */
static i128 orient3d(V a, V b, V c, V d)
{
    return dot(sub(b, a), cross(sub(c, a), sub(d, a)));
}

/* ---------------------------------------------------------------- facets */

typedef struct {
    V o, u, v;        /* unscaled, cm */
    V n;              /* u x v, outward */
    V O;              /* 2s o, scaled */
    V tri[2][3];      /* triangles A and B, scaled */
} Facet;

static Facet facet_of(const int32_t *r, int s)
{
    Facet f;
    i128 k = 2 * (i128)s;
    f.o = mk(r[0], r[1], r[2]);
    f.u = mk(r[3], r[4], r[5]);
    f.v = mk(r[6], r[7], r[8]);
    f.n = cross(f.u, f.v);
    f.O = scl(k, f.o);
    V a = f.O, b = scl(k, add(f.o, f.u)), c = scl(k, add(add(f.o, f.u), f.v)),
      d = scl(k, add(f.o, f.v));
    f.tri[0][0] = a; f.tri[0][1] = b; f.tri[0][2] = c;   /* A = (o, o+u, o+u+v) */
    f.tri[1][0] = a; f.tri[1][1] = c; f.tri[1][2] = d;   /* B = (o, o+u+v, o+v) */
    return f;
}

static Facet *load_facets(const int32_t *facets, int32_t n, int s)
{
    Facet *F = (Facet *)malloc(sizeof(Facet) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; i++) F[i] = facet_of(facets + 10 * (size_t)i, s);
    return F;
}

static V sample(const Facet *f, int s, int a, int b)
{
    return add(f->O, add(scl(2 * a + 1, f->u), scl(2 * b + 1, f->v)));
}

/* step 2: strict facing */
static int front(V x, const Facet *f) { return dot(f->n, sub(x, f->O)) > 0; }

/* ------------------------------------------------ step 3: segment vs triangle */

/* a/b < c/d for b, d > 0 */
static int frac_lt(i128 a, i128 b, i128 c, i128 d) { return a * d < c * b; }
static int frac_le(i128 a, i128 b, i128 c, i128 d) { return a * d <= c * b; }

/* Coplanar case: P, Q and the triangle lie in one plane.  The set of
 * l in [0,1] with P + l d inside the closed triangle is an interval [lo, hi];
 * it is found by clipping against the three edge half-planes in the
 * projection that drops the normal's dominant axis.  The open segment meets
 * the triangle iff lo <= hi, lo < 1 and hi > 0. */
static int coplanar_clip(V P, V Q, V A, V B, V C, i128 *lo_num, i128 *lo_den);

static int coplanar_hit(V P, V Q, V A, V B, V C)
{
    i128 ln, ld;
    return coplanar_clip(P, Q, A, B, C, &ln, &ld);
}

/* The coplanar test of coplanar_hit; also returns the clip interval's lower
 * end lo = lo_num / lo_den (lo_den > 0, lo >= 0). */
static int coplanar_clip(V P, V Q, V A, V B, V C, i128 *lo_num, i128 *lo_den)
{
    V n = cross(sub(B, A), sub(C, A));
    i128 ax = n.x < 0 ? -n.x : n.x, ay = n.y < 0 ? -n.y : n.y, az = n.z < 0 ? -n.z : n.z;
    int drop = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    i128 p[3][2], pp[2], dd[2];
    V T[3] = {A, B, C};
    V d = sub(Q, P);
    for (int i = 0; i < 3; i++) {
        i128 c3[3] = {T[i].x, T[i].y, T[i].z};
        int m = 0;
        for (int k = 0; k < 3; k++) if (k != drop) p[i][m++] = c3[k];
    }
    {
        i128 c3[3] = {P.x, P.y, P.z}, e3[3] = {d.x, d.y, d.z};
        int m = 0;
        for (int k = 0; k < 3; k++) if (k != drop) { pp[m] = c3[k]; dd[m] = e3[k]; m++; }
    }
    /* orientation of the projected triangle */
    i128 area = (p[1][0] - p[0][0]) * (p[2][1] - p[0][1]) - (p[1][1] - p[0][1]) * (p[2][0] - p[0][0]);
    int sig = sgn(area);
    if (sig == 0) return 0;   /* degenerate triangle: never produced by valid facets */
    i128 lo_n = 0, lo_d = 1, hi_n = 1, hi_d = 1;
    for (int e = 0; e < 3; e++) {
        const i128 *a = p[e], *b = p[(e + 1) % 3];
        i128 ex = b[0] - a[0], ey = b[1] - a[1];
        /* inside <=> sig * cross2(edge, X - a) >= 0 with X = P + l d */
        i128 alpha = sig * (ex * (pp[1] - a[1]) - ey * (pp[0] - a[0]));
        i128 beta = sig * (ex * dd[1] - ey * dd[0]);
        if (beta > 0) {            /* l >= -alpha / beta */
            if (frac_lt(lo_n, lo_d, -alpha, beta)) { lo_n = -alpha; lo_d = beta; }
        } else if (beta < 0) {     /* l <= alpha / (-beta) */
            if (frac_lt(alpha, -beta, hi_n, hi_d)) { hi_n = alpha; hi_d = -beta; }
        } else if (alpha < 0) {
            return 0;
        }
    }
    *lo_num = lo_n;
    *lo_den = lo_d;
    return frac_le(lo_n, lo_d, hi_n, hi_d) && frac_lt(lo_n, lo_d, 1, 1) && frac_lt(0, 1, hi_n, hi_d);
}

/* Open segment PQ against closed triangle ABC. */
static int seg_hits_tri(V P, V Q, V A, V B, V C)
{
    if (veq(P, Q)) return 0;                 /* empty open segment */
    int oP = sgn(orient3d(A, B, C, P));
    int oQ = sgn(orient3d(A, B, C, Q));
    if (oP != 0 && oP == oQ) return 0;       /* same strict side */
    if ((oP == 0) != (oQ == 0)) return 0;    /* touches the plane only at an endpoint */
    if (oP != 0) {                           /* strictly opposite sides */
        int e1 = sgn(orient3d(P, Q, A, B));
        int e2 = sgn(orient3d(P, Q, B, C));
        int e3 = sgn(orient3d(P, Q, C, A));
        return (e1 >= 0 && e2 >= 0 && e3 >= 0) || (e1 <= 0 && e2 <= 0 && e3 <= 0);
    }
    return coplanar_hit(P, Q, A, B, C);
}

static i128 gcd128(i128 a, i128 b)
{
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b) { i128 t = a % b; a = b; b = t; }
    return a;
}

/* step 8: the first facet the open segment P -> Q meets, or -1.  A crossing
 * of triangle ABC's plane is at l = oP / (oP - oQ), oP and oQ the sides of P
 * and Q against the plane (normal divided by the gcd of its components, so
 * that the cross-multiplied comparisons stay within 128 bits); a coplanar hit
 * starts at the clip interval's lower end. */
static int32_t first_blocker(const Facet *F, int32_t n, V P, V Q)
{
    int32_t best = -1;
    i128 bn = 1, bd = 1;
    for (int32_t k = 0; k < n; k++)
        for (int t = 0; t < 2; t++) {
            V A = F[k].tri[t][0], B = F[k].tri[t][1], C = F[k].tri[t][2];
            if (!seg_hits_tri(P, Q, A, B, C)) continue;
            V nr = cross(sub(B, A), sub(C, A));
            i128 g = gcd128(gcd128(nr.x, nr.y), nr.z);
            nr = mk(nr.x / g, nr.y / g, nr.z / g);
            i128 oP = dot(nr, sub(P, A)), oQ = dot(nr, sub(Q, A));
            i128 ln = 0, ld = 1;
            if (oP == 0 && oQ == 0) {
                coplanar_clip(P, Q, A, B, C, &ln, &ld);
            } else {
                ln = oP;
                ld = oP - oQ;
                if (ld < 0) { ln = -ln; ld = -ld; }
            }
            if (best < 0 || frac_lt(ln, ld, bn, bd)) { best = k; bn = ln; bd = ld; }
        }
    return best;
}

static int blocked(const Facet *F, int32_t n, V P, V Q)
{
    for (int32_t k = 0; k < n; k++)
        for (int t = 0; t < 2; t++)
            if (seg_hits_tri(P, Q, F[k].tri[t][0], F[k].tri[t][1], F[k].tri[t][2])) return 1;
    return 0;
}

/* step 4, one ordered pair */
static int pair_visible(const Facet *F, int32_t n, int s, int32_t i, int32_t j)
{
    if (i == j) return 0;
    for (int a0 = 0; a0 < s; a0++)
        for (int a1 = 0; a1 < s; a1++) {
            V p = sample(&F[i], s, a0, a1);
            if (!front(p, &F[j])) continue;
            for (int b0 = 0; b0 < s; b0++)
                for (int b1 = 0; b1 < s; b1++) {
                    V q = sample(&F[j], s, b0, b1);
                    if (!front(q, &F[i])) continue;
                    if (!blocked(F, n, p, q)) return 1;
                }
        }
    return 0;
}

/* step 5, one (point, facet) entry */
static int point_sees(const Facet *F, int32_t n, int s, V X, int32_t j)
{
    if (!front(X, &F[j])) return 0;
    for (int b0 = 0; b0 < s; b0++)
        for (int b1 = 0; b1 < s; b1++)
            if (!blocked(F, n, X, sample(&F[j], s, b0, b1))) return 1;
    return 0;
}

static V point_of(const int32_t *p, int s)
{
    return scl(2 * (i128)s, mk(p[0], p[1], p[2]));
}

/* ------------------------------------------------------------- public API */

#define OR_EXPORT __attribute__((visibility("default")))

OR_EXPORT int32_t oracle_words(int32_t n) { return (n + 31) / 32; }

/* Predicate on scaled integer points (for the predicate tests). */
OR_EXPORT int oracle_seg_hits_tri(const int64_t *P, const int64_t *Q, const int64_t *A,
                                  const int64_t *B, const int64_t *C)
{
    return seg_hits_tri(mk(P[0], P[1], P[2]), mk(Q[0], Q[1], Q[2]), mk(A[0], A[1], A[2]),
                        mk(B[0], B[1], B[2]), mk(C[0], C[1], C[2]));
}

/* blocked(P, Q) against a whole scene; P, Q are scaled (x 2s) points. */
OR_EXPORT int oracle_blocked(const int32_t *facets, int32_t n, int32_t s, const int64_t *P,
                             const int64_t *Q)
{
    Facet *F = load_facets(facets, n, s);
    int r = blocked(F, n, mk(P[0], P[1], P[2]), mk(Q[0], Q[1], Q[2]));
    free(F);
    return r;
}

/* Single entries, for sampled checks at sizes where whole rows are too slow:
 * M_ij, vis of the point X (cm, unscaled) towards facet j, and the direct
 * segment between two points (cm). */
OR_EXPORT int oracle_pair_visible(const int32_t *facets, int32_t n, int32_t s, int32_t i, int32_t j)
{
    Facet *F = load_facets(facets, n, s);
    int r = pair_visible(F, n, s, i, j);
    free(F);
    return r;
}

OR_EXPORT int oracle_point_sees(const int32_t *facets, int32_t n, int32_t s, const int32_t *X,
                                int32_t j)
{
    Facet *F = load_facets(facets, n, s);
    int r = point_sees(F, n, s, point_of(X, s), j);
    free(F);
    return r;
}

OR_EXPORT int oracle_los(const int32_t *facets, int32_t n, int32_t s, const int32_t *A,
                         const int32_t *B)
{
    Facet *F = load_facets(facets, n, s);
    int r = !blocked(F, n, point_of(A, s), point_of(B, s));
    free(F);
    return r;
}

/* step 8 on scaled points P, Q; and from the source point X (cm) to the
 * centre sample of facet j. */
OR_EXPORT int32_t oracle_first_blocker_pts(const int32_t *facets, int32_t n, int32_t s,
                                           const int64_t *P, const int64_t *Q)
{
    Facet *F = load_facets(facets, n, s);
    int32_t r = first_blocker(F, n, mk(P[0], P[1], P[2]), mk(Q[0], Q[1], Q[2]));
    free(F);
    return r;
}

OR_EXPORT int32_t oracle_first_blocker(const int32_t *facets, int32_t n, int32_t s,
                                       const int32_t *X, int32_t j)
{
    Facet *F = load_facets(facets, n, s);
    int32_t r = first_blocker(F, n, point_of(X, s), sample(&F[j], s, s / 2, s / 2));
    free(F);
    return r;
}

/* step 9: edge rows for snapshots [t0, t1): table is (t1 - t0) x 2 x WE words
 * (WE = ceil(ne / 32)), nearest is (t1 - t0) x 2 edge indices. */
OR_EXPORT void oracle_edge_table(const int32_t *facets, int32_t n, int32_t s,
                                 const int32_t *edges, int32_t ne, const int32_t *tx,
                                 const int32_t *rx, int64_t t0, int64_t t1, uint32_t *table,
                                 int32_t *nearest)
{
    int32_t WE = oracle_words(ne);
    Facet *F = load_facets(facets, n, s);
    memset(table, 0, sizeof(uint32_t) * (size_t)WE * 2 * (size_t)(t1 - t0));
    for (int64_t t = t0; t < t1; t++) {
        V X[2] = {point_of(tx + 3 * t, s), point_of(rx + 3 * t, s)};
        for (int side = 0; side < 2; side++) {
            uint32_t *row = table + ((size_t)(t - t0) * 2 + side) * WE;
            int32_t best = -1;
            i128 bd = 0;
            for (int32_t e = 0; e < ne; e++) {
                const int32_t *E = edges + 6 * (size_t)e;
                V A = scl(2 * (i128)s, mk(E[0], E[1], E[2]));
                V d = sub(mk(E[3], E[4], E[5]), mk(E[0], E[1], E[2]));
                int vis = 0;
                i128 emin = 0;
                for (int a = 0; a < s; a++) {
                    V p = add(A, scl(2 * a + 1, d));
                    V r = sub(p, X[side]);
                    if (a == 0 || dot(r, r) < emin) emin = dot(r, r);
                    if (!vis && !blocked(F, n, X[side], p)) vis = 1;
                }
                if (!vis) continue;
                row[e >> 5] |= 1u << (e & 31);
                if (best < 0 || emin < bd) { best = e; bd = emin; }
            }
            nearest[(t - t0) * 2 + side] = best;
        }
    }
    free(F);
}

/* step 10: edges as rows and columns of the matrix.  Edge e (A -> B, cm)
 * has s samples q_b = 2s A + (2b+1)(B - A) and two adjacent facets f1, f2
 * (edge_faces[2e], edge_faces[2e+1]); a point P reaches the edge from outside
 * its building only when it is strictly in front of f1 or f2 (ext).
 *   fe[i][e] = exists facet sample p, edge sample q: front(q, i), ext(p, e),
 *              not blocked(p, q);
 *   ee[e][g] = e != g and exists q on e, r on g: ext(r, e), ext(q, g),
 *              not blocked(q, r).
 * Rows [fe0, fe1) of fe and [ee0, ee1) of ee, WE = ceil(ne / 32) words each. */
static V edge_sample(const int32_t *E, int s, int b)
{
    V A = scl(2 * (i128)s, mk(E[0], E[1], E[2]));
    return add(A, scl(2 * b + 1, sub(mk(E[3], E[4], E[5]), mk(E[0], E[1], E[2]))));
}

static int ext(V P, const Facet *F, const int32_t *ef, int32_t e)
{
    return front(P, &F[ef[2 * e]]) || front(P, &F[ef[2 * e + 1]]);
}

OR_EXPORT void oracle_edge_matrix_rows(const int32_t *facets, int32_t n, int32_t s,
                                       const int32_t *edges, const int32_t *edge_faces,
                                       int32_t ne, int32_t fe0, int32_t fe1, uint32_t *fe,
                                       int32_t ee0, int32_t ee1, uint32_t *ee)
{
    int32_t WE = oracle_words(ne);
    Facet *F = load_facets(facets, n, s);
    memset(fe, 0, sizeof(uint32_t) * (size_t)WE * (size_t)(fe1 - fe0));
    memset(ee, 0, sizeof(uint32_t) * (size_t)WE * (size_t)(ee1 - ee0));
    for (int32_t i = fe0; i < fe1; i++)
        for (int32_t e = 0; e < ne; e++) {
            int vis = 0;
            for (int b = 0; b < s && !vis; b++) {
                V q = edge_sample(edges + 6 * (size_t)e, s, b);
                if (!front(q, &F[i])) continue;
                for (int a0 = 0; a0 < s && !vis; a0++)
                    for (int a1 = 0; a1 < s && !vis; a1++) {
                        V p = sample(&F[i], s, a0, a1);
                        if (ext(p, F, edge_faces, e) && !blocked(F, n, p, q)) vis = 1;
                    }
            }
            if (vis) fe[(size_t)(i - fe0) * WE + (e >> 5)] |= 1u << (e & 31);
        }
    for (int32_t e = ee0; e < ee1; e++)
        for (int32_t g = 0; g < ne; g++) {
            if (g == e) continue;
            int vis = 0;
            for (int b = 0; b < s && !vis; b++) {
                V q = edge_sample(edges + 6 * (size_t)e, s, b);
                if (!ext(q, F, edge_faces, g)) continue;
                for (int c = 0; c < s && !vis; c++) {
                    V r = edge_sample(edges + 6 * (size_t)g, s, c);
                    if (ext(r, F, edge_faces, e) && !blocked(F, n, q, r)) vis = 1;
                }
            }
            if (vis) ee[(size_t)(e - ee0) * WE + (g >> 5)] |= 1u << (g & 31);
        }
    free(F);
}

/* Number of sample pairs (p_a on i, q_b on j) that satisfy the three
 * conditions of step 4 (for the hand-counted partial-blocker scene). */
OR_EXPORT int64_t oracle_pair_free_count(const int32_t *facets, int32_t n, int32_t s, int32_t i,
                                         int32_t j)
{
    Facet *F = load_facets(facets, n, s);
    int64_t cnt = 0;
    for (int a0 = 0; a0 < s; a0++)
        for (int a1 = 0; a1 < s; a1++) {
            V p = sample(&F[i], s, a0, a1);
            if (!front(p, &F[j])) continue;
            for (int b0 = 0; b0 < s; b0++)
                for (int b1 = 0; b1 < s; b1++) {
                    V q = sample(&F[j], s, b0, b1);
                    if (front(q, &F[i]) && !blocked(F, n, p, q)) cnt++;
                }
        }
    free(F);
    return cnt;
}

/* Rows [row0, row1) of the matrix: out is (row1 - row0) x W words. */
OR_EXPORT void oracle_matrix_rows(const int32_t *facets, int32_t n, int32_t s, int32_t row0,
                                  int32_t row1, uint32_t *out)
{
    int32_t W = oracle_words(n);
    Facet *F = load_facets(facets, n, s);
    memset(out, 0, sizeof(uint32_t) * (size_t)W * (size_t)(row1 - row0));
    for (int32_t i = row0; i < row1; i++)
        for (int32_t j = 0; j < n; j++)
            if (pair_visible(F, n, s, i, j))
                out[(size_t)(i - row0) * W + (j >> 5)] |= 1u << (j & 31);
    free(F);
}

/* Snapshots [t0, t1) of the table: table is (t1 - t0) x 2 x W (Tx row, Rx
 * row), los is (t1 - t0) bytes.  tx, rx are the full [S][3] arrays (cm). */
OR_EXPORT void oracle_table(const int32_t *facets, int32_t n, int32_t s, const int32_t *tx,
                            const int32_t *rx, int64_t t0, int64_t t1, uint32_t *table,
                            uint8_t *los)
{
    int32_t W = oracle_words(n);
    Facet *F = load_facets(facets, n, s);
    memset(table, 0, sizeof(uint32_t) * (size_t)W * 2 * (size_t)(t1 - t0));
    for (int64_t t = t0; t < t1; t++) {
        V X[2] = {point_of(tx + 3 * t, s), point_of(rx + 3 * t, s)};
        uint32_t *row = table + (size_t)(t - t0) * 2 * W;
        for (int side = 0; side < 2; side++)
            for (int32_t j = 0; j < n; j++)
                if (point_sees(F, n, s, X[side], j))
                    row[side * W + (j >> 5)] |= 1u << (j & 31);
        los[t - t0] = (uint8_t)!blocked(F, n, X[0], X[1]);
    }
    free(F);
}

/* ------------------------------------------ grid mode: the same definition
 *
 * The full-size reference for scenes too large for brute force.  It decides
 * exactly what blocked(), pair_visible() and point_sees() decide, with the
 * same seg_hits_tri() on the same triangles; only the set of triangles a
 * segment is tested against is narrowed first, to those that can possibly
 * meet it:
 *
 *  - An xy grid of nx * ny square cells of width w (scaled units) covers the
 *    scene.  Cell (cx, cy) holds every triangle whose closed xy bounding box
 *    meets the cell's column cx and row cy, where the column of a coordinate
 *    x is floor((x - gx0) / w) clamped to [0, nx - 1] (rows alike).
 *  - A segment visits, column by column, every cell the column's part of
 *    the closed segment can lie in: for column c the part has x in [xa, xb]
 *    (xa = the segment's smallest x in its first column, else the column's
 *    left edge; xb alike), so y lies between y(xa) and y(xb), and the rows
 *    from cell(min) to cell(max) are visited.  y(x) is a fraction of
 *    integers and is floored exactly.
 *  - Why nothing is missed: a point X where the segment meets a triangle
 *    lies in that triangle's bounding box, so its cell holds the triangle;
 *    X lies on the segment, in column cell(X.x), between that column's xa
 *    and xb, so its row is among those visited.
 *  - Each triangle is tested once per segment (a per-call stamp), and only
 *    if its 3D bounding box meets the segment's (a disjoint box cannot hold
 *    a point of the segment).
 */

typedef struct {
    const Facet *F;
    int32_t n_tri;
    i128 gx0, gy0, w;
    int32_t nx, ny;
    int32_t *start;        /* nx * ny + 1 offsets into ids */
    int32_t *ids;          /* triangle ids: 2 * facet + t */
    i128 (*box)[6];        /* per triangle: min x, y, z, max x, y, z */
    uint32_t *stamp;
    uint32_t epoch;
} Grid;

static i128 floordiv(i128 a, i128 b)   /* b > 0 */
{
    i128 q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

static int32_t cell_of(i128 x, i128 x0, i128 w, int32_t m)
{
    i128 c = floordiv(x - x0, w);
    if (c < 0) c = 0;
    if (c > m - 1) c = m - 1;
    return (int32_t)c;
}

static i128 min3(i128 a, i128 b, i128 c) { i128 m = a < b ? a : b; return m < c ? m : c; }
static i128 max3(i128 a, i128 b, i128 c) { i128 m = a > b ? a : b; return m > c ? m : c; }

static void grid_build(Grid *g, const Facet *F, int32_t n)
{
    memset(g, 0, sizeof *g);
    g->F = F;
    g->n_tri = 2 * n;
    g->box = malloc(sizeof(i128[6]) * (size_t)(g->n_tri > 0 ? g->n_tri : 1));
    i128 lo[2] = {0, 0}, hi[2] = {0, 0};
    for (int32_t k = 0; k < g->n_tri; k++) {
        const V *T = F[k / 2].tri[k % 2];
        i128 *b = g->box[k];
        b[0] = min3(T[0].x, T[1].x, T[2].x); b[3] = max3(T[0].x, T[1].x, T[2].x);
        b[1] = min3(T[0].y, T[1].y, T[2].y); b[4] = max3(T[0].y, T[1].y, T[2].y);
        b[2] = min3(T[0].z, T[1].z, T[2].z); b[5] = max3(T[0].z, T[1].z, T[2].z);
        for (int a = 0; a < 2; a++) {
            if (k == 0 || b[a] < lo[a]) lo[a] = b[a];
            if (k == 0 || b[3 + a] > hi[a]) hi[a] = b[3 + a];
        }
    }
    /* about one cell per facet, at most 1024 per axis */
    int32_t m = 1;
    while ((int64_t)m * m < n && m < 1024) m++;
    i128 span = hi[0] - lo[0] > hi[1] - lo[1] ? hi[0] - lo[0] : hi[1] - lo[1];
    g->w = span / m + 1;
    g->gx0 = lo[0];
    g->gy0 = lo[1];
    g->nx = g->ny = m;
    int32_t nc = g->nx * g->ny;
    g->start = calloc((size_t)nc + 1, sizeof(int32_t));
    for (int pass = 0; pass < 2; pass++) {
        int32_t *fill = pass ? calloc((size_t)nc, sizeof(int32_t)) : NULL;
        for (int32_t k = 0; k < g->n_tri; k++) {
            const i128 *b = g->box[k];
            int32_t c0 = cell_of(b[0], g->gx0, g->w, g->nx), c1 = cell_of(b[3], g->gx0, g->w, g->nx);
            int32_t r0 = cell_of(b[1], g->gy0, g->w, g->ny), r1 = cell_of(b[4], g->gy0, g->w, g->ny);
            for (int32_t c = c0; c <= c1; c++)
                for (int32_t r = r0; r <= r1; r++) {
                    int32_t cell = c * g->ny + r;
                    if (pass == 0) g->start[cell + 1]++;
                    else g->ids[g->start[cell] + fill[cell]++] = k;
                }
        }
        if (pass == 0) {
            for (int32_t c = 0; c < nc; c++) g->start[c + 1] += g->start[c];
            g->ids = malloc(sizeof(int32_t) * (size_t)(g->start[nc] > 0 ? g->start[nc] : 1));
        } else {
            free(fill);
        }
    }
    g->stamp = calloc((size_t)(g->n_tri > 0 ? g->n_tri : 1), sizeof(uint32_t));
}

static void grid_free(Grid *g)
{
    free(g->start); free(g->ids); free(g->box); free(g->stamp);
}

/* Calls visit(g, k, P, Q, arg) for every candidate triangle k of the closed
 * segment PQ (each once), in columns and rows ordered from P towards Q;
 * stops when visit returns nonzero and returns that value. */
typedef int (*grid_visit)(Grid *g, int32_t k, V P, V Q, void *arg);

static int grid_walk(Grid *g, V P, V Q, grid_visit visit, void *arg)
{
    if (++g->epoch == 0) {                     /* stamps wrapped: start over */
        memset(g->stamp, 0, sizeof(uint32_t) * (size_t)g->n_tri);
        g->epoch = 1;
    }
    i128 sb[6] = {P.x < Q.x ? P.x : Q.x, P.y < Q.y ? P.y : Q.y, P.z < Q.z ? P.z : Q.z,
                  P.x > Q.x ? P.x : Q.x, P.y > Q.y ? P.y : Q.y, P.z > Q.z ? P.z : Q.z};
    i128 dx = Q.x - P.x, dy = Q.y - P.y;
    int32_t cP = cell_of(P.x, g->gx0, g->w, g->nx), cQ = cell_of(Q.x, g->gx0, g->w, g->nx);
    int32_t c0 = cP < cQ ? cP : cQ, c1 = cP < cQ ? cQ : cP;
    int cstep = cP <= cQ ? 1 : -1;
    for (int32_t c = cP;; c += cstep) {
        i128 xa = (c == c0) ? sb[0] : g->gx0 + (i128)c * g->w;
        i128 xb = (c == c1) ? sb[3] : g->gx0 + (i128)(c + 1) * g->w;
        int32_t r0, r1;
        if (dx == 0) {
            r0 = cell_of(sb[1], g->gy0, g->w, g->ny);
            r1 = cell_of(sb[4], g->gy0, g->w, g->ny);
        } else {
            /* y(x) = P.y + (x - P.x) dy / dx = num / den, den > 0 */
            i128 den = dx > 0 ? dx : -dx, sg = dx > 0 ? 1 : -1;
            i128 na = sg * (P.y * dx + (xa - P.x) * dy), nb = sg * (P.y * dx + (xb - P.x) * dy);
            i128 nlo = na < nb ? na : nb, nhi = na < nb ? nb : na;
            /* row of y = floor((y - gy0) / w) = floor((num - gy0 den) / (w den)) */
            i128 rl = floordiv(nlo - g->gy0 * den, g->w * den);
            i128 rh = floordiv(nhi - g->gy0 * den, g->w * den);
            if (rl < 0) rl = 0;
            if (rl > g->ny - 1) rl = g->ny - 1;
            if (rh < 0) rh = 0;
            if (rh > g->ny - 1) rh = g->ny - 1;
            r0 = (int32_t)rl;
            r1 = (int32_t)rh;
        }
        int rstep = dy >= 0 ? 1 : -1;
        int32_t rs = rstep > 0 ? r0 : r1, re = rstep > 0 ? r1 : r0;
        for (int32_t r = rs;; r += rstep) {
            int32_t cell = c * g->ny + r;
            for (int32_t q = g->start[cell]; q < g->start[cell + 1]; q++) {
                int32_t k = g->ids[q];
                if (g->stamp[k] == g->epoch) continue;
                g->stamp[k] = g->epoch;
                const i128 *b = g->box[k];
                if (b[0] > sb[3] || b[3] < sb[0] || b[1] > sb[4] || b[4] < sb[1] ||
                    b[2] > sb[5] || b[5] < sb[2])
                    continue;
                int v = visit(g, k, P, Q, arg);
                if (v) return v;
            }
            if (r == re) break;
        }
        if (c == cQ) break;
    }
    return 0;
}

static int visit_hit(Grid *g, int32_t k, V P, V Q, void *arg)
{
    const V *T = g->F[k / 2].tri[k % 2];
    return seg_hits_tri(P, Q, T[0], T[1], T[2]);
}

/* blocked() with the candidates of the grid */
static int blocked_grid(Grid *g, V P, V Q) { return grid_walk(g, P, Q, visit_hit, NULL); }

static int pair_visible_grid(Grid *g, int s, int32_t i, int32_t j)
{
    const Facet *F = g->F;
    if (i == j) return 0;
    for (int a0 = 0; a0 < s; a0++)
        for (int a1 = 0; a1 < s; a1++) {
            V p = sample(&F[i], s, a0, a1);
            if (!front(p, &F[j])) continue;
            for (int b0 = 0; b0 < s; b0++)
                for (int b1 = 0; b1 < s; b1++) {
                    V q = sample(&F[j], s, b0, b1);
                    if (!front(q, &F[i])) continue;
                    if (!blocked_grid(g, p, q)) return 1;
                }
        }
    return 0;
}

static int point_sees_grid(Grid *g, int s, V X, int32_t j)
{
    const Facet *F = g->F;
    if (!front(X, &F[j])) return 0;
    for (int b0 = 0; b0 < s; b0++)
        for (int b1 = 0; b1 < s; b1++)
            if (!blocked_grid(g, X, sample(&F[j], s, b0, b1))) return 1;
    return 0;
}

/* Grid mode of oracle_matrix_rows: the listed rows (n_rows of them), out is
 * n_rows x W words. */
OR_EXPORT void oracle_matrix_rows_grid(const int32_t *facets, int32_t n, int32_t s,
                                       const int32_t *rows, int32_t n_rows, uint32_t *out)
{
    int32_t W = oracle_words(n);
    Facet *F = load_facets(facets, n, s);
    Grid g;
    grid_build(&g, F, n);
    memset(out, 0, sizeof(uint32_t) * (size_t)W * (size_t)n_rows);
    for (int32_t k = 0; k < n_rows; k++) {
        int32_t i = rows[k];
        for (int32_t j = 0; j < n; j++)
            if (pair_visible_grid(&g, s, i, j)) out[(size_t)k * W + (j >> 5)] |= 1u << (j & 31);
    }
    grid_free(&g);
    free(F);
}

/* Grid mode of oracle_table: the listed snapshots, table is n_snaps x 2 x W,
 * los is n_snaps bytes; tx, rx are the full [S][3] arrays (cm). */
OR_EXPORT void oracle_table_grid(const int32_t *facets, int32_t n, int32_t s, const int32_t *tx,
                                 const int32_t *rx, const int64_t *snaps, int64_t n_snaps,
                                 uint32_t *table, uint8_t *los)
{
    int32_t W = oracle_words(n);
    Facet *F = load_facets(facets, n, s);
    Grid g;
    grid_build(&g, F, n);
    memset(table, 0, sizeof(uint32_t) * (size_t)W * 2 * (size_t)n_snaps);
    for (int64_t k = 0; k < n_snaps; k++) {
        int64_t t = snaps[k];
        V X[2] = {point_of(tx + 3 * t, s), point_of(rx + 3 * t, s)};
        uint32_t *row = table + (size_t)k * 2 * W;
        for (int side = 0; side < 2; side++)
            for (int32_t j = 0; j < n; j++)
                if (point_sees_grid(&g, s, X[side], j))
                    row[side * W + (j >> 5)] |= 1u << (j & 31);
        los[k] = (uint8_t)!blocked_grid(&g, X[0], X[1]);
    }
    grid_free(&g);
    free(F);
}

/* The grid's candidate set of the segment PQ (scaled points): marks[k] = 1
 * for every triangle k = 2 * facet + t that grid_walk would test (before the
 * 3D box check), for the test that the candidates cover every hit. */
static int visit_mark(Grid *g, int32_t k, V P, V Q, void *arg)
{
    ((uint8_t *)arg)[k] = 1;
    return 0;
}

OR_EXPORT void oracle_grid_candidates(const int32_t *facets, int32_t n, int32_t s,
                                      const int64_t *P, const int64_t *Q, uint8_t *marks)
{
    Facet *F = load_facets(facets, n, s);
    Grid g;
    grid_build(&g, F, n);
    memset(marks, 0, (size_t)2 * n);
    grid_walk(&g, mk(P[0], P[1], P[2]), mk(Q[0], Q[1], Q[2]), visit_mark, marks);
    grid_free(&g);
    free(F);
}

/* ------------------------------------------------------- step 6: image tree */

static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static const uint64_t FP_SEED[2] = {0x243F6A8885A308D3ull, 0x13198A2E03707344ull};

OR_EXPORT uint64_t oracle_splitmix64(uint64_t x) { return splitmix64(x); }

OR_EXPORT uint64_t oracle_fp_weight(int32_t c, int32_t m, int32_t f)
{
    return splitmix64(FP_SEED[c] ^ ((uint64_t)(uint32_t)m << 32) ^ (uint64_t)(uint32_t)f) | 1ull;
}

static int bit(const uint32_t *row, int32_t j) { return (row[j >> 5] >> (j & 31)) & 1u; }

typedef struct {
    const uint32_t *M, *tx_row, *rx_row;
    int32_t n, W, k, t;
    int32_t path[32];
    uint64_t count, fp[2];
    int32_t *paths;        /* nullable */
    int64_t cap, *n_paths;
    int32_t K;
    /* traditional mode: recompute hops from geometry */
    const Facet *F;
    int s;
} Dfs;

static void emit(Dfs *d)
{
    uint64_t w0 = 1, w1 = 1;
    for (int m = 1; m <= d->k; m++) {
        w0 *= oracle_fp_weight(0, m, d->path[m - 1]);
        w1 *= oracle_fp_weight(1, m, d->path[m - 1]);
    }
    d->count += 1;
    d->fp[0] += w0;
    d->fp[1] += w1;
    if (d->n_paths) {
        int64_t idx = (*d->n_paths)++;
        if (d->paths && idx < d->cap) {
            int32_t *rec = d->paths + (size_t)idx * (d->K + 2);
            rec[0] = d->t;
            rec[1] = d->k;
            for (int m = 0; m < d->K; m++) rec[2 + m] = m < d->k ? d->path[m] : -1;
        }
    }
}

static int hop(Dfs *d, int32_t f, int32_t g)
{
    if (d->F) return pair_visible(d->F, d->n, d->s, f, g);
    return bit(d->M + (size_t)f * d->W, g);
}

static void dfs(Dfs *d, int depth)
{
    if (depth == d->k) {
        if (bit(d->rx_row, d->path[depth - 1])) emit(d);
        return;
    }
    for (int32_t g = 0; g < d->n; g++) {
        if (depth == 0) {
            if (!bit(d->tx_row, g)) continue;
        } else if (!hop(d, d->path[depth - 1], g)) {
            continue;
        }
        d->path[depth] = g;
        dfs(d, depth + 1);
    }
}

/* Image-tree summaries for snapshots [t0, t1): summary is (t1-t0) x (K+1) x 3
 * u64 {count, fp0, fp1}; M is N x W; table is the full S x 2 x W; los is S.
 * If n_paths is non-null, paths are counted into *n_paths (not reset here)
 * and the first cap are written as records (t, k, f1..fK, -1 padded). */
OR_EXPORT void oracle_tree(const uint32_t *M, const uint32_t *table, const uint8_t *los,
                           int32_t n, int64_t t0, int64_t t1, int32_t K, uint64_t *summary,
                           int32_t *paths, int64_t cap, int64_t *n_paths)
{
    int32_t W = oracle_words(n);
    for (int64_t t = t0; t < t1; t++) {
        uint64_t *sm = summary + (size_t)(t - t0) * (K + 1) * 3;
        Dfs d;
        memset(&d, 0, sizeof d);
        d.M = M; d.n = n; d.W = W; d.t = (int32_t)t; d.K = K;
        d.tx_row = table + (size_t)t * 2 * W;
        d.rx_row = d.tx_row + W;
        d.paths = paths; d.cap = cap; d.n_paths = n_paths;
        /* order 0: the direct path */
        sm[0] = sm[1] = sm[2] = los[t] ? 1 : 0;
        if (n_paths && los[t]) {
            d.k = 0;
            emit(&d);
            d.count = 0; d.fp[0] = d.fp[1] = 0;
        }
        for (int k = 1; k <= K; k++) {
            d.k = k; d.count = 0; d.fp[0] = d.fp[1] = 0;
            dfs(&d, 0);
            sm[3 * k + 0] = d.count;
            sm[3 * k + 1] = d.fp[0];
            sm[3 * k + 2] = d.fp[1];
        }
    }
}

/* Step 7: the same summaries, with nothing cached: for each snapshot the Tx
 * and Rx rows are computed from geometry, and every hop's visibility is
 * recomputed from geometry when the search reaches it. */
OR_EXPORT void oracle_traditional(const int32_t *facets, int32_t n, int32_t s, const int32_t *tx,
                                  const int32_t *rx, int64_t t0, int64_t t1, int32_t K,
                                  uint64_t *summary)
{
    int32_t W = oracle_words(n);
    Facet *F = load_facets(facets, n, s);
    uint32_t *rows = (uint32_t *)calloc((size_t)2 * W, sizeof(uint32_t));
    for (int64_t t = t0; t < t1; t++) {
        V X[2] = {point_of(tx + 3 * t, s), point_of(rx + 3 * t, s)};
        memset(rows, 0, sizeof(uint32_t) * 2 * W);
        for (int side = 0; side < 2; side++)
            for (int32_t j = 0; j < n; j++)
                if (point_sees(F, n, s, X[side], j)) rows[side * W + (j >> 5)] |= 1u << (j & 31);
        uint64_t *sm = summary + (size_t)(t - t0) * (K + 1) * 3;
        int l = !blocked(F, n, X[0], X[1]);
        sm[0] = sm[1] = sm[2] = (uint64_t)l;
        Dfs d;
        memset(&d, 0, sizeof d);
        d.n = n; d.W = W; d.t = (int32_t)t; d.K = K;
        d.tx_row = rows; d.rx_row = rows + W;
        d.F = F; d.s = s;
        for (int k = 1; k <= K; k++) {
            d.k = k; d.count = 0; d.fp[0] = d.fp[1] = 0;
            dfs(&d, 0);
            sm[3 * k + 0] = d.count;
            sm[3 * k + 1] = d.fp[0];
            sm[3 * k + 2] = d.fp[1];
        }
    }
    free(rows);
    free(F);
}
