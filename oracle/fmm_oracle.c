/*
 * fmm_oracle.c -- plain, slow, FP64 CPU oracle for the shift-free 2D FMM.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * library in paper_2009_00767_gb300/csrc.
 *
 * What it computes (Kajima, "Summation of certain locally bilinear forms and
 * its applications to the Fast Multipole Method", arXiv 2009.00767):
 *
 *   phi(z_i) = sum_{j != i} q_j log|z_i - z_j|      (the 2D log potential)
 *
 * three ways:
 *   oracle_direct      the O(N^2) definition itself;
 *   oracle_shiftfree   the paper's shift-free scheme (Sec. 2.2.1, upward pass
 *                      U-bar-1/U-bar-2 and downward pass D-bar-1/D-bar-2):
 *                      per level k = 2..l the multipole moments of every square
 *                      are formed straight from the particles (no M2M), each
 *                      square's interaction list is converted to a local
 *                      expansion (M2L), and that local expansion is evaluated
 *                      straight at the particles (no L2L); the near field of
 *                      the own and eight adjacent finest squares is summed
 *                      directly (Sec. 2.1, E-2);
 *   oracle_classical   Greengard's scheme as the paper recalls it (Sec. 2.1,
 *                      U-1, U-2, D-1, D-2, E-1, E-2): leaf multipoles, M2M
 *                      shifts up, M2L, L2L shifts down, leaf evaluation.
 *
 * The vectors v of Sec. 2.2.1 are realised as complex multipole moments of
 * order p (coefficients 0..p) and the bilinear forms B as the multipole-to-
 * local conversion of Greengard's 2D expansions (the paper's ref. [101]).
 * This oracle works in UNSCALED form: moments about the box centre c are
 *   a_0 = sum q_j,  a_m = -(1/m) sum q_j (z_j - c)^m,
 * and the far field of a box is Re[a_0 log(z - c) + sum_m a_m (z - c)^-m].
 *
 * Tree (Sec. 2.1 items 1-5): the computation box is the square [0,box]^2 at
 * level 0; every level-k square splits into four at level k+1, down to level
 * l.  A particle's finest square is (ix, iy) = (floor(x 2^l / box),
 * floor(y 2^l / box)), both evaluated in FP64 in that order and clamped to
 * [0, 2^l - 1]; its level-k square is (ix >> (l-k), iy >> (l-k)).  The
 * interaction list of a level-k square (k >= 2) is the set of children of its
 * parent's neighbours (and of its parent) that are not adjacent to it.
 * Squares are indexed row-major here (bx + by * 2^k).
 *
 * Readings where the paper is silent: j = i and coincident pairs (r^2 == 0)
 * contribute 0; the interaction lists of ALL levels 2..l are converted (the
 * text's "k < l" would drop the finest level's well-separated pairs).
 *
 * Force field (Sec. 3: the paper's timings cover "potential and force
 * fields"): E = -grad phi.  With phi = Re f(z), f analytic, grad phi =
 * (Re f', -Im f'), so E = (-Re f'(z), Im f'(z)); oracle_direct_field is the
 * definition, E_i = -sum_{j != i, r > 0} q_j (z_i - z_j) / |z_i - z_j|^2, and
 * oracle_shiftfree_field differentiates the same method term by term (each
 * level's local expansion, sum_l l b_l (z - c)^(l-1), plus the near field).
 *
 * Loops over independent outputs carry OpenMP pragmas; no reduction crosses
 * threads, so results do not depend on the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { ORACLE_OK = 0, ORACLE_ERR_ARG = 1, ORACLE_ERR_OUT_OF_BOX = 2, ORACLE_ERR_NOMEM = 3 };

/* ------------------------------------------------------------------------ */
/* threads                                                                   */
/* ------------------------------------------------------------------------ */

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* binomial coefficients C(n, r) by Pascal's rule, n <= ORACLE_MAXBINOM      */
/* ------------------------------------------------------------------------ */

#define ORACLE_MAXP 64
#define ORACLE_MAXBINOM (2 * ORACLE_MAXP + 2)

static double binom_table[ORACLE_MAXBINOM + 1][ORACLE_MAXBINOM + 1];
static int binom_ready = 0;

/* The table is filled once, serially, before any OpenMP region can read it: every public
 * entry point that reaches an expansion calls binom_init() first, and the library
 * constructor fills it at load time. */
static void binom_init(void) {
    if (binom_ready) return;
    for (int n = 0; n <= ORACLE_MAXBINOM; ++n) {
        for (int r = 0; r <= ORACLE_MAXBINOM; ++r) binom_table[n][r] = 0.0;
        binom_table[n][0] = 1.0;
        for (int r = 1; r <= n; ++r)
            binom_table[n][r] = binom_table[n - 1][r - 1] + (r <= n - 1 ? binom_table[n - 1][r] : 0.0);
    }
    binom_ready = 1;
}

__attribute__((constructor)) static void oracle_init(void) { binom_init(); }

double oracle_binom(int n, int r) {
    binom_init();
    if (n < 0 || r < 0 || r > n || n > ORACLE_MAXBINOM) return 0.0;
    return binom_table[n][r];
}

/* ------------------------------------------------------------------------ */
/* Greengard's 2D expansions, unscaled (the paper's ref. [101])             */
/* ------------------------------------------------------------------------ */

/* P2M: moments a[0..p] about centre c of charges q at z (U-1 / U-bar-1). */
static void p2m_accumulate(cplx c, cplx z, double q, int p, cplx *a) {
    cplx d = z - c;
    cplx dm = 1.0;
    a[0] += q;
    for (int m = 1; m <= p; ++m) {
        dm *= d;
        a[m] -= q * dm / (double)m;
    }
}

/* Far field of moments a[] about c at the point z: Re[a0 log(z-c) + sum a_m (z-c)^-m]. */
static double multipole_eval(const cplx *a, int p, cplx c, cplx z) {
    cplx d = z - c;
    cplx inv = 1.0 / d;
    cplx acc = 0.0;
    for (int m = p; m >= 1; --m) acc = (acc + a[m]) * inv;   /* Horner in 1/d */
    return creal(a[0] * clog(d) + acc);
}

/* M2L: moments a[] about c_s to local coefficients b[] about c_t, z0 = c_s - c_t
 * (D-1 / D-bar-1).  With u = z - c_t and z - c_s = -z0 (1 - u/z0):
 *   b_0 = a_0 log(-z0) + sum_{k>=1} a_k (-1)^k z0^-k
 *   b_l = -a_0 / (l z0^l) + z0^-l sum_{k>=1} a_k (-1)^k z0^-k C(l+k-1, k-1)   (l >= 1)
 * The result is ADDED to b[]. */
static void m2l_accumulate(const cplx *a, int p, cplx z0, cplx *b) {
    cplx inv = 1.0 / z0;
    cplx ak_over[ORACLE_MAXP + 1];          /* a_k (-1)^k z0^-k */
    cplx ip = 1.0;
    for (int k = 1; k <= p; ++k) {
        ip *= inv;
        ak_over[k] = a[k] * ip * ((k & 1) ? -1.0 : 1.0);
    }
    cplx b0 = a[0] * clog(-z0);
    for (int k = 1; k <= p; ++k) b0 += ak_over[k];
    b[0] += b0;
    cplx il = 1.0;
    for (int l = 1; l <= p; ++l) {
        il *= inv;                           /* z0^-l */
        cplx s = -a[0] / (double)l;
        for (int k = 1; k <= p; ++k) s += ak_over[k] * binom_table[l + k - 1][k - 1];
        b[l] += s * il;
    }
}

/* L2P: Re sum_l b_l (z - c)^l (E-1). */
static double local_eval(const cplx *b, int p, cplx c, cplx z) {
    cplx u = z - c;
    cplx acc = 0.0;
    for (int l = p; l >= 0; --l) acc = acc * u + b[l];
    return creal(acc);
}

/* M2M: child moments a[] about c_c to parent moments about c_p, z0 = c_c - c_p (U-2).
 *   b_0 = a_0,  b_l = -a_0 z0^l / l + sum_{k=1}^{l} a_k z0^(l-k) C(l-1, k-1).  Added to b[]. */
static void m2m_accumulate(const cplx *a, int p, cplx z0, cplx *b) {
    cplx zp[ORACLE_MAXP + 1];
    zp[0] = 1.0;
    for (int m = 1; m <= p; ++m) zp[m] = zp[m - 1] * z0;
    b[0] += a[0];
    for (int l = 1; l <= p; ++l) {
        cplx s = -a[0] * zp[l] / (double)l;
        for (int k = 1; k <= l; ++k) s += a[k] * zp[l - k] * binom_table[l - 1][k - 1];
        b[l] += s;
    }
}

/* L2L: parent local a[] about c_p re-centred at the child centre c_c, z0 = c_c - c_p (D-2).
 * sum_k a_k (u + z0)^k with u = z - c_c gives b_l = sum_{k>=l} a_k C(k, l) z0^(k-l).  Added to b[]. */
static void l2l_accumulate(const cplx *a, int p, cplx z0, cplx *b) {
    cplx zp[ORACLE_MAXP + 1];
    zp[0] = 1.0;
    for (int m = 1; m <= p; ++m) zp[m] = zp[m - 1] * z0;
    for (int l = 0; l <= p; ++l) {
        cplx s = 0.0;
        for (int k = l; k <= p; ++k) s += a[k] * binom_table[k][l] * zp[k - l];
        b[l] += s;
    }
}

/* Exposed single-step expansions, for unit checks of each formula. */
void oracle_p2m(int n, const double *xy, const double *q, double cx, double cy, int p, double *a_out) {
    cplx a[ORACLE_MAXP + 1];
    for (int m = 0; m <= p; ++m) a[m] = 0.0;
    for (int j = 0; j < n; ++j) p2m_accumulate(cx + I * cy, xy[2 * j] + I * xy[2 * j + 1], q[j], p, a);
    for (int m = 0; m <= p; ++m) { a_out[2 * m] = creal(a[m]); a_out[2 * m + 1] = cimag(a[m]); }
}

static void unpack(const double *in, int p, cplx *out) {
    for (int m = 0; m <= p; ++m) out[m] = in[2 * m] + I * in[2 * m + 1];
}
static void pack(const cplx *in, int p, double *out) {
    for (int m = 0; m <= p; ++m) { out[2 * m] = creal(in[m]); out[2 * m + 1] = cimag(in[m]); }
}

double oracle_multipole_eval(const double *a_in, int p, double cx, double cy, double x, double y) {
    cplx a[ORACLE_MAXP + 1];
    unpack(a_in, p, a);
    return multipole_eval(a, p, cx + I * cy, x + I * y);
}

void oracle_m2l(const double *a_in, int p, double z0x, double z0y, double *b_out) {
    binom_init();
    cplx a[ORACLE_MAXP + 1], b[ORACLE_MAXP + 1];
    unpack(a_in, p, a);
    for (int m = 0; m <= p; ++m) b[m] = 0.0;
    m2l_accumulate(a, p, z0x + I * z0y, b);
    pack(b, p, b_out);
}

double oracle_local_eval(const double *b_in, int p, double cx, double cy, double x, double y) {
    cplx b[ORACLE_MAXP + 1];
    unpack(b_in, p, b);
    return local_eval(b, p, cx + I * cy, x + I * y);
}

void oracle_m2m(const double *a_in, int p, double z0x, double z0y, double *b_out) {
    binom_init();
    cplx a[ORACLE_MAXP + 1], b[ORACLE_MAXP + 1];
    unpack(a_in, p, a);
    for (int m = 0; m <= p; ++m) b[m] = 0.0;
    m2m_accumulate(a, p, z0x + I * z0y, b);
    pack(b, p, b_out);
}

void oracle_l2l(const double *a_in, int p, double z0x, double z0y, double *b_out) {
    binom_init();
    cplx a[ORACLE_MAXP + 1], b[ORACLE_MAXP + 1];
    unpack(a_in, p, a);
    for (int m = 0; m <= p; ++m) b[m] = 0.0;
    l2l_accumulate(a, p, z0x + I * z0y, b);
    pack(b, p, b_out);
}

/* ------------------------------------------------------------------------ */
/* direct sum: the definition                                                */
/* ------------------------------------------------------------------------ */

static double pair_term(double xi, double yi, double xj, double yj, double qj) {
    double dx = xi - xj, dy = yi - yj;
    double r2 = dx * dx + dy * dy;
    if (r2 > 0.0) return qj * 0.5 * log(r2);   /* log|z| = (1/2) log r^2 */
    return 0.0;                                 /* coincident: reading, contributes 0 */
}

/* phi at targets[t] (indices into the particle list), t < n_targets. */
int oracle_direct_targets(int64_t n, const double *xy, const double *q,
                          int64_t n_targets, const int64_t *targets, double *phi) {
    if (n < 0 || n_targets < 0) return ORACLE_ERR_ARG;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_targets; ++t) {
        int64_t i = targets[t];
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i) s += pair_term(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1], q[j]);
        phi[t] = s;
    }
    return ORACLE_OK;
}

int oracle_direct(int64_t n, const double *xy, const double *q, double *phi) {
    if (n < 0) return ORACLE_ERR_ARG;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i) s += pair_term(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1], q[j]);
        phi[i] = s;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* the tree                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int levels, p;
    double box;
    int64_t n;
    int side;            /* 2^l finest squares per side */
    int *ix, *iy;        /* finest square of each particle */
    int64_t *start;      /* CSR over finest squares, row-major: leaf (x, y) -> x + y*side */
    int64_t *order;      /* particle indices grouped by finest square */
} tree_t;

static void tree_free(tree_t *t) {
    free(t->ix); free(t->iy); free(t->start); free(t->order);
}

static int finest_coord(double x, int levels, double box) {
    double f = floor(x * (double)(1 << levels) / box);
    int side = 1 << levels;
    if (f < 0.0) return 0;
    if (f > (double)(side - 1)) return side - 1;
    return (int)f;
}

/* The finest square of each particle by the rule above (Sec. 2.1 items 1-4 with the
 * floor/clamp reading for points on an edge or on x = box): ix[i], iy[i] in [0, 2^l - 1]. */
int oracle_finest_squares(int64_t n, const double *xy, int levels, double box, int *ix, int *iy) {
    if (n < 0 || levels < 0 || levels > 12 || !(box > 0.0)) return ORACLE_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) {
        ix[i] = finest_coord(xy[2 * i], levels, box);
        iy[i] = finest_coord(xy[2 * i + 1], levels, box);
    }
    return ORACLE_OK;
}

static int tree_build(tree_t *t, int64_t n, const double *xy, int levels, int p, double box) {
    memset(t, 0, sizeof(*t));
    if (n < 0 || levels < 0 || levels > 12 || p < 1 || p > ORACLE_MAXP || !(box > 0.0)) return ORACLE_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) {
        double x = xy[2 * i], y = xy[2 * i + 1];
        if (!(x >= 0.0 && x <= box && y >= 0.0 && y <= box)) return ORACLE_ERR_OUT_OF_BOX;
    }
    t->levels = levels; t->p = p; t->box = box; t->n = n;
    t->side = 1 << levels;
    int64_t nleaf = (int64_t)t->side * t->side;
    t->ix = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    t->iy = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    t->start = calloc((size_t)nleaf + 1, sizeof(int64_t));
    t->order = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!t->ix || !t->iy || !t->start || !t->order) { tree_free(t); return ORACLE_ERR_NOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        t->ix[i] = finest_coord(xy[2 * i], levels, box);
        t->iy[i] = finest_coord(xy[2 * i + 1], levels, box);
        t->start[(int64_t)t->ix[i] + (int64_t)t->iy[i] * t->side + 1]++;
    }
    for (int64_t b = 0; b < nleaf; ++b) t->start[b + 1] += t->start[b];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)nleaf);
    if (!fill) { tree_free(t); return ORACLE_ERR_NOMEM; }
    for (int64_t b = 0; b < nleaf; ++b) fill[b] = t->start[b];
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = (int64_t)t->ix[i] + (int64_t)t->iy[i] * t->side;
        t->order[fill[b]++] = i;
    }
    free(fill);
    return ORACLE_OK;
}

static cplx box_centre(int bx, int by, int k, double box) {
    double s = box / (double)(1 << k);
    return (bx + 0.5) * s + I * ((by + 0.5) * s);
}

/* Interaction list of level-k square (bx, by), k >= 2: children of the parent's
 * 3x3 neighbourhood that are not adjacent to (bx, by).  Returns the count. */
static int interaction_list(int bx, int by, int k, int *sx, int *sy) {
    int side = 1 << k, cnt = 0;
    int px = bx >> 1, py = by >> 1;
    for (int qy = py - 1; qy <= py + 1; ++qy)
        for (int qx = px - 1; qx <= px + 1; ++qx) {
            if (qx < 0 || qy < 0 || qx >= (side >> 1) || qy >= (side >> 1)) continue;
            for (int c = 0; c < 4; ++c) {
                int cx = 2 * qx + (c & 1), cy = 2 * qy + (c >> 1);
                if (abs(cx - bx) <= 1 && abs(cy - by) <= 1) continue;   /* adjacent or itself */
                sx[cnt] = cx; sy[cnt] = cy; ++cnt;
            }
        }
    return cnt;
}

int oracle_interaction_list(int bx, int by, int k, int *sx, int *sy) {
    if (k < 2) return 0;
    return interaction_list(bx, by, k, sx, sy);
}

/* Multipole moments of every level-k square, straight from the particles. */
static cplx *moments_from_particles(const tree_t *t, const double *xy, const double *q, int k) {
    int side = 1 << k, p = t->p, sh = t->levels - k;
    cplx *a = calloc((size_t)side * side * (p + 1), sizeof(cplx));
    if (!a) return NULL;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int b = 0; b < side * side; ++b) {
        int bx = b % side, by = b / side;
        cplx c = box_centre(bx, by, k, t->box);
        cplx *ab = a + (size_t)b * (p + 1);
        /* the square covers finest squares [bx<<sh, (bx+1)<<sh) x [by<<sh, (by+1)<<sh) */
        for (int ly = by << sh; ly < (by + 1) << sh; ++ly)
            for (int lx = bx << sh; lx < (bx + 1) << sh; ++lx) {
                int64_t leaf = (int64_t)lx + (int64_t)ly * t->side;
                for (int64_t s = t->start[leaf]; s < t->start[leaf + 1]; ++s) {
                    int64_t j = t->order[s];
                    p2m_accumulate(c, xy[2 * j] + I * xy[2 * j + 1], q[j], p, ab);
                }
            }
    }
    return a;
}

/* Local expansion of every level-k square from its interaction list (D-1 / D-bar-1). */
static cplx *locals_from_interaction_lists(const tree_t *t, const cplx *a, int k) {
    int side = 1 << k, p = t->p;
    cplx *b = calloc((size_t)side * side * (p + 1), sizeof(cplx));
    if (!b) return NULL;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int tb = 0; tb < side * side; ++tb) {
        int bx = tb % side, by = tb / side;
        int sx[27], sy[27];
        int cnt = interaction_list(bx, by, k, sx, sy);
        cplx ct = box_centre(bx, by, k, t->box);
        for (int s = 0; s < cnt; ++s) {
            cplx cs = box_centre(sx[s], sy[s], k, t->box);
            m2l_accumulate(a + (size_t)(sx[s] + sy[s] * side) * (p + 1), p, cs - ct, b + (size_t)tb * (p + 1));
        }
    }
    return b;
}

/* Near field (E-2): own finest square and its (up to) eight neighbours, directly. */
static void near_field(const tree_t *t, const double *xy, const double *q, double *phi) {
    int side = t->side;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < t->n; ++i) {
        double s = 0.0;
        for (int ny = t->iy[i] - 1; ny <= t->iy[i] + 1; ++ny)
            for (int nx = t->ix[i] - 1; nx <= t->ix[i] + 1; ++nx) {
                if (nx < 0 || ny < 0 || nx >= side || ny >= side) continue;
                int64_t leaf = (int64_t)nx + (int64_t)ny * side;
                for (int64_t r = t->start[leaf]; r < t->start[leaf + 1]; ++r) {
                    int64_t j = t->order[r];
                    if (j != i) s += pair_term(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1], q[j]);
                }
            }
        phi[i] += s;
    }
}

/* ------------------------------------------------------------------------ */
/* force field E = -grad phi                                                  */
/* ------------------------------------------------------------------------ */

/* grad phi contribution at (xi, yi) of a charge qj at (xj, yj): qj (z_i - z_j) / r^2; 0 at r = 0 */
static void pair_grad(double xi, double yi, double xj, double yj, double qj, double *gx, double *gy) {
    double dx = xi - xj, dy = yi - yj;
    double r2 = dx * dx + dy * dy;
    if (r2 > 0.0) { *gx += qj * dx / r2; *gy += qj * dy / r2; }
}

/* E at targets[t]: E[2t] = Ex, E[2t+1] = Ey. */
int oracle_direct_field_targets(int64_t n, const double *xy, const double *q,
                                int64_t n_targets, const int64_t *targets, double *E) {
    if (n < 0 || n_targets < 0) return ORACLE_ERR_ARG;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_targets; ++t) {
        int64_t i = targets[t];
        double gx = 0.0, gy = 0.0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i) pair_grad(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1], q[j], &gx, &gy);
        E[2 * t] = -gx;
        E[2 * t + 1] = -gy;
    }
    return ORACLE_OK;
}

int oracle_direct_field(int64_t n, const double *xy, const double *q, double *E) {
    if (n < 0) return ORACLE_ERR_ARG;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double gx = 0.0, gy = 0.0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i) pair_grad(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1], q[j], &gx, &gy);
        E[2 * i] = -gx;
        E[2 * i + 1] = -gy;
    }
    return ORACLE_OK;
}

/* f'(z) of a local expansion about c: sum_{l>=1} l b_l (z - c)^(l-1) */
static cplx local_eval_deriv(const cplx *b, int p, cplx c, cplx z) {
    cplx u = z - c;
    cplx acc = 0.0;
    for (int l = p; l >= 1; --l) acc = acc * u + (double)l * b[l];
    return acc;
}

double oracle_local_eval_deriv(const double *b_in, int p, double cx, double cy, double x, double y, double *im) {
    cplx b[ORACLE_MAXP + 1];
    for (int m = 0; m <= p; ++m) b[m] = b_in[2 * m] + I * b_in[2 * m + 1];
    cplx d = local_eval_deriv(b, p, cx + I * cy, x + I * y);
    *im = cimag(d);
    return creal(d);
}

/* ------------------------------------------------------------------------ */
/* shift-free FMM (Sec. 2.2.1)                                               */
/* ------------------------------------------------------------------------ */

/* phi_far_level (optional, may be NULL): [levels+1][n] far field per level. */
int oracle_shiftfree_levels(int64_t n, const double *xy, const double *q, int levels, int p, double box,
                            double *phi, double *phi_far_level) {
    binom_init();
    tree_t t;
    int rc = tree_build(&t, n, xy, levels, p, box);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i) phi[i] = 0.0;
    if (phi_far_level)
        for (int64_t i = 0; i < (int64_t)(levels + 1) * n; ++i) phi_far_level[i] = 0.0;
    for (int k = 2; k <= levels; ++k) {
        /* U-bar: the level-k vectors (moments) summed straight from the particles */
        cplx *a = moments_from_particles(&t, xy, q, k);
        if (!a) { tree_free(&t); return ORACLE_ERR_NOMEM; }
        /* D-bar-1: the level-k linear forms from the interaction lists */
        cplx *b = locals_from_interaction_lists(&t, a, k);
        free(a);
        if (!b) { tree_free(&t); return ORACLE_ERR_NOMEM; }
        /* D-bar-2 by linearity: each level's form evaluated at the particle and added */
        int sh = levels - k, side = 1 << k;
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            int bx = t.ix[i] >> sh, by = t.iy[i] >> sh;
            double v = local_eval(b + (size_t)(bx + by * side) * (p + 1), p, box_centre(bx, by, k, box),
                                  xy[2 * i] + I * xy[2 * i + 1]);
            phi[i] += v;
            if (phi_far_level) phi_far_level[(int64_t)k * n + i] = v;
        }
        free(b);
    }
    near_field(&t, xy, q, phi);
    tree_free(&t);
    return ORACLE_OK;
}

int oracle_shiftfree(int64_t n, const double *xy, const double *q, int levels, int p, double box, double *phi) {
    return oracle_shiftfree_levels(n, xy, q, levels, p, box, phi, NULL);
}

/* ------------------------------------------------------------------------ */
/* classical Greengard FMM with shifts (Sec. 2.1)                            */
/* ------------------------------------------------------------------------ */

/* The shift-free FMM with the field: phi as oracle_shiftfree, and E = -grad phi from the same
 * local expansions (differentiated) and the same near field (E[2i] = Ex, E[2i+1] = Ey). */
int oracle_shiftfree_field(int64_t n, const double *xy, const double *q, int levels, int p, double box,
                           double *phi, double *E) {
    binom_init();
    tree_t t;
    int rc = tree_build(&t, n, xy, levels, p, box);
    if (rc) return rc;
    double *gx = calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *gy = calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!gx || !gy) { free(gx); free(gy); tree_free(&t); return ORACLE_ERR_NOMEM; }
    for (int64_t i = 0; i < n; ++i) phi[i] = 0.0;
    for (int k = 2; k <= levels; ++k) {
        cplx *a = moments_from_particles(&t, xy, q, k);
        if (!a) { free(gx); free(gy); tree_free(&t); return ORACLE_ERR_NOMEM; }
        cplx *b = locals_from_interaction_lists(&t, a, k);
        free(a);
        if (!b) { free(gx); free(gy); tree_free(&t); return ORACLE_ERR_NOMEM; }
        int sh = levels - k, side = 1 << k;
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            int bx = t.ix[i] >> sh, by = t.iy[i] >> sh;
            const cplx *bl = b + (size_t)(bx + by * side) * (p + 1);
            cplx c = box_centre(bx, by, k, box), z = xy[2 * i] + I * xy[2 * i + 1];
            phi[i] += local_eval(bl, p, c, z);
            cplx d = local_eval_deriv(bl, p, c, z);     /* grad = (Re f', -Im f') */
            gx[i] += creal(d);
            gy[i] -= cimag(d);
        }
        free(b);
    }
    near_field(&t, xy, q, phi);
    int side = t.side;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double sx = 0.0, sy = 0.0;
        for (int ny = t.iy[i] - 1; ny <= t.iy[i] + 1; ++ny)
            for (int nx = t.ix[i] - 1; nx <= t.ix[i] + 1; ++nx) {
                if (nx < 0 || ny < 0 || nx >= side || ny >= side) continue;
                int64_t leaf = (int64_t)nx + (int64_t)ny * side;
                for (int64_t r = t.start[leaf]; r < t.start[leaf + 1]; ++r) {
                    int64_t j = t.order[r];
                    if (j != i) pair_grad(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1], q[j], &sx, &sy);
                }
            }
        E[2 * i] = -(gx[i] + sx);
        E[2 * i + 1] = -(gy[i] + sy);
    }
    free(gx);
    free(gy);
    tree_free(&t);
    return ORACLE_OK;
}

int oracle_classical(int64_t n, const double *xy, const double *q, int levels, int p, double box, double *phi) {
    binom_init();
    tree_t t;
    int rc = tree_build(&t, n, xy, levels, p, box);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i) phi[i] = 0.0;
    if (levels >= 2) {
        cplx **a = calloc((size_t)levels + 1, sizeof(cplx *));
        cplx **loc = calloc((size_t)levels + 1, sizeof(cplx *));
        if (!a || !loc) { free(a); free(loc); tree_free(&t); return ORACLE_ERR_NOMEM; }
        /* U-1: finest-level multipoles from the particles */
        a[levels] = moments_from_particles(&t, xy, q, levels);
        if (!a[levels]) rc = ORACLE_ERR_NOMEM;
        /* U-2: shift children to parents, levels l-1 .. 2 */
        for (int k = levels - 1; k >= 2 && !rc; --k) {
            int side = 1 << k;
            a[k] = calloc((size_t)side * side * (p + 1), sizeof(cplx));
            if (!a[k]) { rc = ORACLE_ERR_NOMEM; break; }
            for (int b = 0; b < side * side; ++b) {
                int bx = b % side, by = b / side;
                cplx cp = box_centre(bx, by, k, box);
                for (int c = 0; c < 4; ++c) {
                    int cx = 2 * bx + (c & 1), cy = 2 * by + (c >> 1);
                    cplx cc = box_centre(cx, cy, k + 1, box);
                    m2m_accumulate(a[k + 1] + (size_t)(cx + cy * 2 * side) * (p + 1), p, cc - cp,
                                   a[k] + (size_t)b * (p + 1));
                }
            }
        }
        /* D-1: interaction-list conversion at every level 2..l */
        for (int k = 2; k <= levels && !rc; ++k) {
            loc[k] = locals_from_interaction_lists(&t, a[k], k);
            if (!loc[k]) rc = ORACLE_ERR_NOMEM;
        }
        /* D-2: Psi = 0 above level 2; shift each parent's local to its children and add */
        for (int k = 3; k <= levels && !rc; ++k) {
            int side = 1 << k;
            for (int b = 0; b < side * side; ++b) {
                int bx = b % side, by = b / side;
                int px = bx >> 1, py = by >> 1;
                cplx cp = box_centre(px, py, k - 1, box);
                cplx cc = box_centre(bx, by, k, box);
                l2l_accumulate(loc[k - 1] + (size_t)(px + py * (side >> 1)) * (p + 1), p, cc - cp,
                               loc[k] + (size_t)b * (p + 1));
            }
        }
        /* E-1: evaluate the finest-level local expansions at the particles */
        if (!rc) {
            int side = t.side;
            for (int64_t i = 0; i < n; ++i)
                phi[i] += local_eval(loc[levels] + (size_t)(t.ix[i] + t.iy[i] * side) * (p + 1), p,
                                     box_centre(t.ix[i], t.iy[i], levels, box), xy[2 * i] + I * xy[2 * i + 1]);
        }
        for (int k = 0; k <= levels; ++k) { free(a[k]); free(loc[k]); }
        free(a); free(loc);
        if (rc) { tree_free(&t); return rc; }
    }
    /* E-2 */
    near_field(&t, xy, q, phi);
    tree_free(&t);
    return ORACLE_OK;
}
