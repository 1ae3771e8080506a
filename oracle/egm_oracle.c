/*
 * Brute-force CPU oracle for exact epipolar-guided matching.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no source with
 * the CUDA path and is deliberately slow: it evaluates the paper's plain
 * definition of the candidate set for every (query, reference) pair.
 *
 * What it computes (paper, Sec. 3 "Guided Matching"):
 *   - the epipolar line of query i:       l_i = F p~_i^1 = (a, b, c)
 *   - the point-to-line distance (Eq. 3): dist = |a x + b y + c| / sqrt(a^2 + b^2)
 *   - the candidate set (Eq. 4):          C_i = { j : dist(l_i, p_j^2) <= eps_j }
 *     (eps_j is the tolerance of image-2 keypoint j; a scalar eps is the
 *      broadcast case, Algorithm 1)
 *   - descriptor matching restricted to C_i (Sec. 4.3): exhaustive distance
 *     over the candidates, best and second best by (distance, index) with the
 *     lower index winning ties, and Lowe's ratio test with tau = num/den
 *     (tau = 0.8 in Sec. 5.1) applied to distances, not squared distances.
 *
 * Floating point: FP64 throughout.  This file must be compiled with
 * -ffp-contract=off so that every expression is evaluated as written, left to
 * right, with one rounding per operation and no fused multiply-add.
 *
 * Pins (all in tests/test_oracle_pins.py, none of them re-types these
 * formulas): the rectified pose reduces the set to |y2 - y1| <= eps (checked
 * against a sorted range query); forward motion gives radial lines whose
 * distance is r |sin(theta - alpha)| (polar closed form); noise-free true
 * correspondences of a random pose sit at distance ~0 (fixes F versus F^T);
 * hand-built tiny scenes with hand-written expected sets; eps = infinity
 * reduces matching to exhaustive nearest neighbour (checked against an
 * independent numpy argsort); exact rational ratio tests on small integers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_DESC_U8_L2 0
#define ORACLE_DESC_F32_L2 1
#define ORACLE_DESC_BIN 2

#define ORACLE_FLAG_HAS_BEST 1
#define ORACLE_FLAG_RATIO_PASS 2
#define ORACLE_FLAG_NO_SECOND 4
#define ORACLE_FLAG_DEGENERATE_LINE 8

/* Width of the band around the tolerance boundary, in pixels, whose pairs are
 * listed apart from the bit-exact comparison. */
#define ORACLE_BOUNDARY_BAND 1e-9

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* l = F * (x, y, 1)^T, F row-major (Sec. 3). */
static void epipolar_line(const double *F, double x, double y, double l[3]) {
    l[0] = F[0] * x + F[1] * y + F[2];
    l[1] = F[3] * x + F[4] * y + F[5];
    l[2] = F[6] * x + F[7] * y + F[8];
}

/* Eq. 3 with the norm sqrt(a^2 + b^2) passed in. */
static double line_distance(const double l[3], double norm, double x, double y) {
    return fabs(l[0] * x + l[1] * y + l[2]) / norm;
}

static double eps_of(const double *eps2, double eps_scalar, int64_t j) {
    return eps2 ? eps2[j] : eps_scalar;
}

double oracle_point_line_distance(const double *F, double x1, double y1, double x2, double y2) {
    double l[3];
    epipolar_line(F, x1, y1, l);
    double norm = sqrt(l[0] * l[0] + l[1] * l[1]);
    return line_distance(l, norm, x2, y2);
}

/*
 * Candidate sets in CSR form, ascending j within each row.
 *   pass 1 (idx == NULL): writes counts[i] (and bcounts[i], the number of
 *                         boundary pairs |dist - eps| < 1e-9) and returns 0.
 *   pass 2 (idx != NULL): offsets[m+1] / boffsets[m+1] from pass 1's counts;
 *                         writes candidate indices and boundary indices.
 * degenerate[i] = 1 where a^2 + b^2 == 0 (that query's set is empty).
 */
int oracle_candidates(int64_t m, const double *xy1, int64_t n, const double *xy2,
                      const double *F, const double *eps2, double eps_scalar,
                      int64_t *counts, int64_t *bcounts,
                      const int64_t *offsets, int32_t *idx,
                      const int64_t *boffsets, int32_t *bidx,
                      uint8_t *degenerate) {
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < m; i++) {
        double l[3];
        epipolar_line(F, xy1[2 * i], xy1[2 * i + 1], l);
        double norm = sqrt(l[0] * l[0] + l[1] * l[1]);
        int64_t k = 0, kb = 0;
        if (norm == 0.0) {
            if (degenerate) degenerate[i] = 1;
        } else {
            if (degenerate) degenerate[i] = 0;
            for (int64_t j = 0; j < n; j++) {
                double d = line_distance(l, norm, xy2[2 * j], xy2[2 * j + 1]);
                double e = eps_of(eps2, eps_scalar, j);
                if (d <= e) {
                    if (idx) idx[offsets[i] + k] = (int32_t)j;
                    k++;
                }
                if (fabs(d - e) < ORACLE_BOUNDARY_BAND) {
                    if (bidx) bidx[boffsets[i] + kb] = (int32_t)j;
                    kb++;
                }
            }
        }
        if (counts) counts[i] = k;
        if (bcounts) bcounts[i] = kb;
    }
    return 0;
}

/* Exact squared L2 distance of two uint8 vectors (Sec. 4.3). */
static int64_t dist_u8(const uint8_t *q, const uint8_t *r, int dim) {
    int64_t s = 0;
    for (int k = 0; k < dim; k++) {
        int64_t d = (int64_t)q[k] - (int64_t)r[k];
        s += d * d;
    }
    return s;
}

/* Hamming distance of two bit strings of `bytes` bytes. */
static int64_t dist_bin(const uint8_t *q, const uint8_t *r, int bytes) {
    int64_t s = 0;
    for (int k = 0; k < bytes; k++) {
        unsigned v = (unsigned)(q[k] ^ r[k]);
        while (v) {
            s += v & 1u;
            v >>= 1;
        }
    }
    return s;
}

/* Squared L2 distance of two float vectors, accumulated in FP64. */
static double dist_f32(const float *q, const float *r, int dim) {
    double s = 0.0;
    for (int k = 0; k < dim; k++) {
        double d = (double)q[k] - (double)r[k];
        s += d * d;
    }
    return s;
}

/* (d, j) < (d1, j1) in lexicographic order. */
static int lex_less(double d, int64_t j, double d1, int64_t j1) {
    return d < d1 || (d == d1 && j < j1);
}

/*
 * Guided matching (Algorithm 1, "select best by descriptor"): for each query,
 * exhaustive descriptor distances over its candidate set, best / second best
 * by (distance, index), Lowe's ratio test with tau = ratio_num / ratio_den on
 * distances (squared distances compared with tau^2; Hamming counts compared
 * with tau).  exclude_boundary = 1 drops the pairs with |dist - eps| < 1e-9.
 *
 * Distances reported: squared L2 for the L2 kinds, the bit count for binary.
 * A missing best / second is index -1 with distance +inf.
 */
int oracle_match(int64_t m, const double *xy1, int64_t n, const double *xy2,
                 const double *F, const double *eps2, double eps_scalar,
                 int kind, int dim, const void *desc1, const void *desc2,
                 int ratio_num, int ratio_den, int exclude_boundary,
                 int32_t *best, int32_t *second, double *best_d, double *second_d,
                 uint8_t *flags, int64_t *ncand) {
    int row = kind == ORACLE_DESC_U8_L2 ? dim : kind == ORACLE_DESC_BIN ? dim / 8 : dim * 4;
    const uint8_t *d1b = (const uint8_t *)desc1;
    const uint8_t *d2b = (const uint8_t *)desc2;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < m; i++) {
        double l[3];
        epipolar_line(F, xy1[2 * i], xy1[2 * i + 1], l);
        double norm = sqrt(l[0] * l[0] + l[1] * l[1]);
        double b1 = INFINITY, b2 = INFINITY;
        int64_t j1 = -1, j2 = -1, k = 0;
        uint8_t fl = 0;
        if (norm == 0.0) {
            fl |= ORACLE_FLAG_DEGENERATE_LINE;
        } else {
            for (int64_t j = 0; j < n; j++) {
                double d = line_distance(l, norm, xy2[2 * j], xy2[2 * j + 1]);
                double e = eps_of(eps2, eps_scalar, j);
                if (!(d <= e)) continue;
                if (exclude_boundary && fabs(d - e) < ORACLE_BOUNDARY_BAND) continue;
                k++;
                double dd;
                const uint8_t *q = d1b + (size_t)i * row;
                const uint8_t *r = d2b + (size_t)j * row;
                if (kind == ORACLE_DESC_U8_L2)
                    dd = (double)dist_u8(q, r, dim);
                else if (kind == ORACLE_DESC_BIN)
                    dd = (double)dist_bin(q, r, row);
                else
                    dd = dist_f32((const float *)q, (const float *)r, dim);
                if (lex_less(dd, j, b1, j1)) {
                    b2 = b1;
                    j2 = j1;
                    b1 = dd;
                    j1 = j;
                } else if (lex_less(dd, j, b2, j2)) {
                    b2 = dd;
                    j2 = j;
                }
            }
        }
        if (j1 >= 0) {
            fl |= ORACLE_FLAG_HAS_BEST;
            int pass;
            if (j2 < 0) {
                fl |= ORACLE_FLAG_NO_SECOND;
                pass = 1;
            } else if (kind == ORACLE_DESC_U8_L2) {
                /* sqrt(D1) < (num/den) sqrt(D2)  <=>  D1 den^2 < D2 num^2, exact in int64 */
                int64_t D1 = (int64_t)b1, D2 = (int64_t)b2;
                pass = D1 * ratio_den * ratio_den < D2 * ratio_num * ratio_num;
            } else if (kind == ORACLE_DESC_BIN) {
                int64_t H1 = (int64_t)b1, H2 = (int64_t)b2;
                pass = H1 * ratio_den < H2 * ratio_num;
            } else {
                pass = b1 * ((double)ratio_den * ratio_den) < b2 * ((double)ratio_num * ratio_num);
            }
            if (pass) fl |= ORACLE_FLAG_RATIO_PASS;
        }
        best[i] = (int32_t)j1;
        second[i] = (int32_t)j2;
        best_d[i] = b1;
        second_d[i] = b2;
        flags[i] = fl;
        if (ncand) ncand[i] = k;
    }
    return 0;
}
