/*
 * CPU baseline: the paper's own method on the host cores.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY: the benchmark times it beside the
 * brute-force oracle as a fair CPU reference (the paper's data structure,
 * multithreaded), and the tests check it against the oracle.  It shares no
 * source with the CUDA path or with the oracle.
 *
 * What it computes (paper, Sec. 4.1-4.4 and Algorithm 1):
 *   - the epipole e = null(F^T) (Algorithm 1, preprocessing), as the cross
 *     product of the two columns of F whose cross product is largest;
 *   - per image-2 keypoint, the angle theta_j = atan2(y_j - y_e, x_j - x_e)
 *     and angular radius delta_j = asin(eps_j / ||p_j - e||) (Sec. 4.2),
 *     folded into [0, pi) and split in two where it wraps (Sec. 4.4,
 *     "Discontinuity"); keypoints within eps of the epipole get [0, pi]
 *     (Sec. 4.4, "Keypoints near the epipole");
 *   - a centred segment tree over the intervals (Sec. 4.4, "Segment Tree
 *     Structure"): each node splits at the median of its intervals'
 *     midpoints, keeps the intervals containing the split in a bucket with
 *     their smallest start and largest end, and passes the intervals wholly
 *     left / right of it to its children; stored flat;
 *   - per query, the angle alpha_i of its line from the epipole and a stab
 *     of the tree (Sec. 4.2), then descriptor matching over the candidates
 *     (Sec. 4.3): best and second by (distance, index), ratio test.
 *
 * Two modes:
 *   exact = 0  the paper's method as described: alpha_i is the direction from
 *              the epipole to the point of the line closest to the image
 *              centre (Sec. 4.2) and a candidate is any interval containing
 *              it, with no distance test.  Sets equal the definition up to
 *              floating-point effects at the tolerance boundary.
 *   exact = 1  the same tree with every interval widened by a pad that covers
 *              the rounding of the angles and the distance of each line from
 *              the computed epipole, alpha_i the line's own direction, and
 *              the point-to-line test of Eq. 3 / Eq. 4 on every candidate
 *              (FP64, evaluated as written; compile with -ffp-contract=off).
 *              Sets equal the brute-force definition.
 * An epipole farther than 10^6 image diagonals from the image centre (or at
 * infinity) switches to a parallel key: the offset of each keypoint along the
 * normal of the epipole direction, interval [key - eps, key + eps] (the paper
 * never meets this case, Sec. 6).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ST_DESC_U8_L2 0
#define ST_DESC_F32_L2 1
#define ST_DESC_BIN 2

#define ST_FLAG_HAS_BEST 1
#define ST_FLAG_RATIO_PASS 2
#define ST_FLAG_NO_SECOND 4
#define ST_FLAG_DEGENERATE_LINE 8

typedef struct {
    double lo, hi;
    int32_t j;
} Interval;

typedef struct {
    double split, min_lo, max_hi;
    int64_t b0, b1;        /* bucket: items[b0 .. b1) */
    int32_t left, right;   /* child node indices, -1 if none */
} Node;

typedef struct {
    Interval *items;
    Node *nodes;
    int64_t nitems, nnodes;
    int32_t root;
    /* frame */
    int parallel;
    double ex, ey;         /* epipole (angular mode) */
    double nx, ny;         /* normal of the epipole direction (parallel mode) */
    double cx, cy;         /* image centre */
} Index;

int segtree_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- geometry */

static void line_of(const double *F, double x, double y, double l[3]) {
    l[0] = F[0] * x + F[1] * y + F[2];
    l[1] = F[3] * x + F[4] * y + F[5];
    l[2] = F[6] * x + F[7] * y + F[8];
}

/* e with F^T e = 0: orthogonal to every column of F. */
static void epipole(const double *F, double e[3]) {
    double col[3][3];
    e[0] = e[1] = e[2] = 0.0;
    for (int c = 0; c < 3; c++)
        for (int r = 0; r < 3; r++) col[c][r] = F[3 * r + c];
    double bestn = -1.0;
    for (int a = 0; a < 3; a++)
        for (int b = a + 1; b < 3; b++) {
            double v[3] = {col[a][1] * col[b][2] - col[a][2] * col[b][1],
                           col[a][2] * col[b][0] - col[a][0] * col[b][2],
                           col[a][0] * col[b][1] - col[a][1] * col[b][0]};
            double nn = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            if (nn > bestn) {
                bestn = nn;
                memcpy(e, v, sizeof v);
            }
        }
    double s = sqrt(bestn);
    if (s > 0.0)
        for (int k = 0; k < 3; k++) e[k] /= s;
}

static double fold_pi(double a) {
    if (a < 0.0) a += M_PI;
    if (a >= M_PI) a -= M_PI;
    if (a < 0.0 || a >= M_PI) a = 0.0;
    return a;
}

/* ---------------------------------------------------------------- tree */

static double nth_smallest(double *v, int64_t n, int64_t k) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        double p = v[lo + (hi - lo) / 2];
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (v[i] < p) i++;
            while (v[j] > p) j--;
            if (i <= j) {
                double t = v[i];
                v[i] = v[j];
                v[j] = t;
                i++;
                j--;
            }
        }
        if (k <= j)
            hi = j;
        else if (k >= i)
            lo = i;
        else
            break;
    }
    return v[k];
}

static void swap_iv(Interval *a, Interval *b) {
    Interval t = *a;
    *a = *b;
    *b = t;
}

/* Builds the subtree over items[lo, hi); returns its node index or -1.
 * Subtrees of more than 2048 intervals are built as parallel tasks; each
 * uses the scratch range [lo, hi) and takes its node index atomically. */
static int32_t build_node(Index *ix, int64_t lo, int64_t hi, double *scratch) {
    if (lo >= hi) return -1;
    int64_t cnt = hi - lo;
    double *sc = scratch + lo;
    for (int64_t k = 0; k < cnt; k++) sc[k] = 0.5 * (ix->items[lo + k].lo + ix->items[lo + k].hi);
    double c = nth_smallest(sc, cnt, cnt / 2);
    /* three-way partition: [lo, a) left of c, [a, b) containing c, [b, hi) right */
    int64_t a = lo, k = lo, b = hi;
    while (k < b) {
        Interval *it = &ix->items[k];
        if (it->hi < c)
            swap_iv(it, &ix->items[a++]), k++;
        else if (it->lo > c)
            swap_iv(it, &ix->items[--b]);
        else
            k++;
    }
    int64_t id64;
#pragma omp atomic capture
    id64 = ix->nnodes++;
    int32_t id = (int32_t)id64;
    Node *nd = &ix->nodes[id];
    nd->split = c;
    nd->b0 = a;
    nd->b1 = b;
    nd->min_lo = INFINITY;
    nd->max_hi = -INFINITY;
    for (int64_t t = a; t < b; t++) {
        if (ix->items[t].lo < nd->min_lo) nd->min_lo = ix->items[t].lo;
        if (ix->items[t].hi > nd->max_hi) nd->max_hi = ix->items[t].hi;
    }
    int32_t l, r;
    if (cnt > 2048) {
#pragma omp task shared(l)
        l = build_node(ix, lo, a, scratch);
        r = build_node(ix, b, hi, scratch);
#pragma omp taskwait
    } else {
        l = build_node(ix, lo, a, scratch);
        r = build_node(ix, b, hi, scratch);
    }
    ix->nodes[id].left = l;
    ix->nodes[id].right = r;
    return id;
}

/* Calls emit(j) for every interval containing q. */
#define STAB(ix, q, EMIT)                                                      \
    do {                                                                       \
        int32_t nd_ = (ix)->root;                                              \
        while (nd_ >= 0) {                                                     \
            const Node *N_ = &(ix)->nodes[nd_];                                \
            if ((q) >= N_->min_lo && (q) <= N_->max_hi)                        \
                for (int64_t t_ = N_->b0; t_ < N_->b1; t_++) {                 \
                    const Interval *I_ = &(ix)->items[t_];                     \
                    if (I_->lo <= (q) && (q) <= I_->hi) EMIT(I_->j);           \
                }                                                              \
            if ((q) < N_->split)                                               \
                nd_ = N_->left;                                                \
            else if ((q) > N_->split)                                          \
                nd_ = N_->right;                                               \
            else                                                               \
                break;                                                         \
        }                                                                      \
    } while (0)

static double eps_at(const double *eps2, double eps_scalar, int64_t j) { return eps2 ? eps2[j] : eps_scalar; }

/*
 * The index over the references.  In exact mode the intervals are widened by
 * `pad` pixels plus 1e-13 of the keypoint's distance from the epipole (angle
 * rounding); `pad` covers the lines' distance from the computed epipole
 * (angular) or the deviation of their normals from the common one times the
 * image radius (parallel).
 */
static int build_index(Index *ix, int64_t m, const double *xy1, int64_t n, const double *xy2, const double *F,
                       const double *eps2, double eps_scalar, int width, int height, int exact) {
    memset(ix, 0, sizeof *ix);
    ix->cx = 0.5 * width;
    ix->cy = 0.5 * height;
    double e[3];
    epipole(F, e);
    if (e[0] == 0.0 && e[1] == 0.0 && e[2] == 0.0) return -2;  /* rank of F below 2 */
    double diag = sqrt((double)width * width + (double)height * height);
    double far = hypot(e[0] - e[2] * ix->cx, e[1] - e[2] * ix->cy);
    ix->parallel = !(far <= 1e6 * diag * fabs(e[2]));
    if (ix->parallel) {
        double dn = hypot(e[0], e[1]);
        ix->nx = -e[1] / dn;
        ix->ny = e[0] / dn;
    } else {
        ix->ex = e[0] / e[2];
        ix->ey = e[1] / e[2];
    }
    double pad = 0.0;
    if (exact) {
        double worst = 0.0, R = 0.0;
        int64_t i;
#pragma omp parallel for reduction(max : worst) schedule(static)
        for (i = 0; i < m; i++) {
            double l[3];
            line_of(F, xy1[2 * i], xy1[2 * i + 1], l);
            double nn = hypot(l[0], l[1]);
            if (!(nn > 0.0)) continue;
            double v;
            if (ix->parallel) {
                /* 1 - |cos| of the angle between the line normal and the common one, as a sine */
                double cr = (l[0] * ix->ny - l[1] * ix->nx) / nn;
                v = fabs(cr);
            } else {
                v = fabs(l[0] * ix->ex + l[1] * ix->ey + l[2]) / nn;
            }
            if (v > worst) worst = v;
        }
        if (ix->parallel) {
            for (int64_t j = 0; j < n; j++) {
                double r = hypot(xy2[2 * j] - ix->cx, xy2[2 * j + 1] - ix->cy);
                if (r > R) R = r;
            }
            pad = worst * R * 1.01 + 1e-6;
        } else {
            pad = worst * 1.000001 + 1e-6;
        }
    }
    /* up to two intervals per keypoint in slots 2j, 2j + 1, then compacted */
    Interval *tmp = (Interval *)malloc(sizeof(Interval) * (size_t)(2 * n + 1));
    uint8_t *cnt = (uint8_t *)malloc((size_t)n + 1);
    ix->items = (Interval *)malloc(sizeof(Interval) * (size_t)(2 * n + 1));
    if (!tmp || !cnt || !ix->items) {
        free(tmp);
        free(cnt);
        return -1;
    }
    int64_t j;
#pragma omp parallel for schedule(static)
    for (j = 0; j < n; j++) {
        double x = xy2[2 * j], y = xy2[2 * j + 1], eps = eps_at(eps2, eps_scalar, j);
        Interval *o = tmp + 2 * j;
        cnt[j] = 1;
        if (ix->parallel) {
            double key = ix->nx * (x - ix->cx) + ix->ny * (y - ix->cy);
            double w = eps + pad + (exact ? 1e-13 * fabs(key) + 1e-9 : 0.0);
            o[0] = (Interval){key - w, key + w, (int32_t)j};
            continue;
        }
        double dx = x - ix->ex, dy = y - ix->ey;
        double d = hypot(dx, dy);
        double r = exact ? eps + pad + 1e-13 * d : eps;
        if (d <= r) {
            o[0] = (Interval){0.0, M_PI, (int32_t)j};
            continue;
        }
        double th = fold_pi(atan2(dy, dx));
        double de = asin(r / d);
        double lo = th - de, hi = th + de;
        if (lo < 0.0) {
            o[0] = (Interval){lo + M_PI, M_PI, (int32_t)j};
            o[1] = (Interval){0.0, hi, (int32_t)j};
            cnt[j] = 2;
        } else if (hi > M_PI) {
            o[0] = (Interval){lo, M_PI, (int32_t)j};
            o[1] = (Interval){0.0, hi - M_PI, (int32_t)j};
            cnt[j] = 2;
        } else {
            o[0] = (Interval){lo, hi, (int32_t)j};
        }
    }
    int64_t k = 0;
    for (j = 0; j < n; j++)
        for (int t = 0; t < cnt[j]; t++) ix->items[k++] = tmp[2 * j + t];
    free(tmp);
    free(cnt);
    ix->nitems = k;
    ix->nodes = (Node *)malloc(sizeof(Node) * (size_t)(k + 1));
    double *scratch = (double *)malloc(sizeof(double) * (size_t)(k + 1));
    if (!ix->nodes || !scratch) {
        free(scratch);
        return -1;
    }
    int32_t root = -1;
#pragma omp parallel
#pragma omp single
    root = build_node(ix, 0, k, scratch);
    ix->root = root;
    free(scratch);
    return 0;
}

static void free_index(Index *ix) {
    free(ix->items);
    free(ix->nodes);
}

/* The query key of line l (a, b, c); returns 0 for a degenerate line. */
static int query_key(const Index *ix, const double l[3], int exact, double *q) {
    double nn = hypot(l[0], l[1]);
    if (!(nn > 0.0)) return 0;
    if (ix->parallel) {
        double s = l[0] * ix->nx + l[1] * ix->ny >= 0.0 ? 1.0 : -1.0;
        /* signed offset of the line from the centre along its own normal */
        *q = -s * (l[0] * ix->cx + l[1] * ix->cy + l[2]) / nn;
        return 1;
    }
    if (!exact) {
        /* the point of the line closest to the image centre (Sec. 4.2) */
        double t = (l[0] * ix->cx + l[1] * ix->cy + l[2]) / (nn * nn);
        double qx = ix->cx - t * l[0], qy = ix->cy - t * l[1];
        double dx = qx - ix->ex, dy = qy - ix->ey;
        if (hypot(dx, dy) > 1e-9 * (1.0 + hypot(ix->ex, ix->ey))) {
            *q = fold_pi(atan2(dy, dx));
            return 1;
        }
    }
    *q = fold_pi(atan2(-l[0], l[1]));  /* the line's direction (b, -a) */
    return 1;
}

/* ---------------------------------------------------------------- descriptors */

static int64_t dist_u8(const uint8_t *q, const uint8_t *r, int dim) {
    int32_t s = 0;
    for (int k = 0; k < dim; k++) {
        int32_t d = (int32_t)q[k] - (int32_t)r[k];
        s += d * d;
    }
    return s;
}

static int64_t dist_bin(const uint8_t *q, const uint8_t *r, int bytes) {
    int64_t s = 0;
    int k = 0;
    for (; k + 8 <= bytes; k += 8) {
        uint64_t a, b;
        memcpy(&a, q + k, 8);
        memcpy(&b, r + k, 8);
        s += __builtin_popcountll(a ^ b);
    }
    for (; k < bytes; k++) s += __builtin_popcount((unsigned)(q[k] ^ r[k]));
    return s;
}

static double dist_f32(const float *q, const float *r, int dim) {
    double s = 0.0;
    for (int k = 0; k < dim; k++) {
        double d = (double)q[k] - (double)r[k];
        s += d * d;
    }
    return s;
}

/* ---------------------------------------------------------------- entry points */

/*
 * Candidate sets in CSR form, ascending j: pass 1 (idx NULL) writes counts[m];
 * pass 2 writes idx at offsets[m + 1] taken from pass 1.
 */
int segtree_candidates(int64_t m, const double *xy1, int64_t n, const double *xy2, const double *F,
                       const double *eps2, double eps_scalar, int width, int height, int exact, int64_t *counts,
                       const int64_t *offsets, int32_t *idx) {
    Index ix;
    if (build_index(&ix, m, xy1, n, xy2, F, eps2, eps_scalar, width, height, exact) != 0) return -1;
    int64_t i;
#pragma omp parallel
    {
        uint8_t *seen = (uint8_t *)calloc((size_t)n + 1, 1);
#pragma omp for schedule(dynamic, 32)
        for (i = 0; i < m; i++) {
            double l[3], q;
            line_of(F, xy1[2 * i], xy1[2 * i + 1], l);
            int64_t k = 0;
            if (query_key(&ix, l, exact, &q)) {
                double nn = sqrt(l[0] * l[0] + l[1] * l[1]);
#define EMIT_C(j)                                                                                   \
    do {                                                                                            \
        int32_t j_ = (j);                                                                           \
        if (exact && !(fabs(l[0] * xy2[2 * j_] + l[1] * xy2[2 * j_ + 1] + l[2]) / nn <=             \
                       eps_at(eps2, eps_scalar, j_)))                                               \
            break;                                                                                  \
        seen[j_] = 1;                                                                               \
    } while (0)
                STAB(&ix, q, EMIT_C);
#undef EMIT_C
                for (int64_t j = 0; j < n; j++)
                    if (seen[j]) {
                        if (idx) idx[offsets[i] + k] = (int32_t)j;
                        k++;
                        seen[j] = 0;
                    }
            }
            if (counts) counts[i] = k;
        }
        free(seen);
    }
    free_index(&ix);
    return 0;
}

/*
 * Matching (Algorithm 1, "select best by descriptor"): outputs as the
 * oracle's (best / second by (distance, index), squared L2 or bit counts,
 * ratio test tau = ratio_num / ratio_den on distances).  seconds[0..1]
 * receive the wall time of the index build and of the matching.
 */
int segtree_match(int64_t m, const double *xy1, int64_t n, const double *xy2, const double *F, const double *eps2,
                  double eps_scalar, int width, int height, int exact, int kind, int dim, const void *desc1,
                  const void *desc2, int ratio_num, int ratio_den, int32_t *best, int32_t *second,
                  double *best_d, double *second_d, uint8_t *flags, int64_t *ncand, double *seconds) {
    int row = kind == ST_DESC_U8_L2 ? dim : kind == ST_DESC_BIN ? dim / 8 : dim * 4;
    const uint8_t *d1b = (const uint8_t *)desc1, *d2b = (const uint8_t *)desc2;
#ifdef _OPENMP
    double t0 = omp_get_wtime();
#endif
    Index ix;
    if (build_index(&ix, m, xy1, n, xy2, F, eps2, eps_scalar, width, height, exact) != 0) return -1;
#ifdef _OPENMP
    double t1 = omp_get_wtime();
#endif
    int64_t i;
#pragma omp parallel for schedule(dynamic, 32)
    for (i = 0; i < m; i++) {
        double l[3], q;
        line_of(F, xy1[2 * i], xy1[2 * i + 1], l);
        double b1 = INFINITY, b2 = INFINITY;
        int64_t j1 = -1, j2 = -1, k = 0;
        uint8_t fl = 0;
        if (!query_key(&ix, l, exact, &q)) {
            fl |= ST_FLAG_DEGENERATE_LINE;
        } else {
            double nn = sqrt(l[0] * l[0] + l[1] * l[1]);
            const uint8_t *qd = d1b + (size_t)i * row;
#define EMIT_M(j)                                                                                   \
    do {                                                                                            \
        int64_t j_ = (j);                                                                           \
        if (exact && !(fabs(l[0] * xy2[2 * j_] + l[1] * xy2[2 * j_ + 1] + l[2]) / nn <=             \
                       eps_at(eps2, eps_scalar, j_)))                                               \
            break;                                                                                  \
        k++;                                                                                        \
        const uint8_t *r_ = d2b + (size_t)j_ * row;                                                 \
        double dd = kind == ST_DESC_U8_L2 ? (double)dist_u8(qd, r_, dim)                            \
                    : kind == ST_DESC_BIN ? (double)dist_bin(qd, r_, row)                           \
                                          : dist_f32((const float *)qd, (const float *)r_, dim);    \
        if (dd < b1 || (dd == b1 && j_ < j1)) {                                                     \
            b2 = b1, j2 = j1, b1 = dd, j1 = j_;                                                     \
        } else if (j_ != j1 && (dd < b2 || (dd == b2 && j_ < j2))) {                                \
            b2 = dd, j2 = j_;                                                                       \
        }                                                                                           \
    } while (0)
            STAB(&ix, q, EMIT_M);
#undef EMIT_M
        }
        if (j1 >= 0) {
            fl |= ST_FLAG_HAS_BEST;
            int pass;
            if (j2 < 0) {
                fl |= ST_FLAG_NO_SECOND;
                pass = 1;
            } else if (kind == ST_DESC_U8_L2) {
                int64_t D1 = (int64_t)b1, D2 = (int64_t)b2;
                pass = D1 * ratio_den * ratio_den < D2 * ratio_num * ratio_num;
            } else if (kind == ST_DESC_BIN) {
                pass = (int64_t)b1 * ratio_den < (int64_t)b2 * ratio_num;
            } else {
                pass = b1 * ((double)ratio_den * ratio_den) < b2 * ((double)ratio_num * ratio_num);
            }
            if (pass) fl |= ST_FLAG_RATIO_PASS;
        }
        best[i] = (int32_t)j1;
        second[i] = (int32_t)j2;
        best_d[i] = b1;
        second_d[i] = b2;
        flags[i] = fl;
        if (ncand) ncand[i] = k;
    }
#ifdef _OPENMP
    double t2 = omp_get_wtime();
    if (seconds) seconds[0] = t1 - t0, seconds[1] = t2 - t1;
#else
    if (seconds) seconds[0] = seconds[1] = 0.0;
#endif
    free_index(&ix);
    return 0;
}
