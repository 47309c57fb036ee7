/*
 * lagrange_oracle.c -- plain, slow, FP64 CPU oracle for the paper's own realisation of the
 * shift-free FMM: charges fixed in position at Lagrange nodes (arXiv 2009.00767, Appendix,
 * STEP1-STEP5, Eq. 1-2, with the summation scheme of Sec. 2.2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this file:
 * only the tests, the smoke check and the benchmark's CPU baseline do.  It shares no code,
 * header, table or constant with the CUDA library in paper_2009_00767_gb300/csrc.
 *
 * What it computes, for D = 2 (the log potential) and D = 3 (the Coulomb potential):
 *
 *   phi(c_i) = sum_{j != i} q_j K(c_i, c_j),   K = log|r| (D = 2) or 1/|r| (D = 3),
 *
 * three ways:
 *   oracle_lag_direct    the definition;
 *   oracle_lag_literal   the paper's steps in its order and notation: the vector v_c of a
 *                        charge is its image under h_{m^0} (the 16 or 64 charges at the root
 *                        box's nodes, STEP2); U-bar-1 sums them per finest square and U-bar-2
 *                        up the tree with no shift; D-bar-1 forms the dual vectors
 *                        sum_{m_i in IL(m)} B_{m_i,m}(v_{m_i}, .) with B's matrix
 *                        M_{m_i}^T M_b M_m (STEP3-STEP5) formed explicitly per pair; D-bar-2
 *                        adds each square's dual vector to its children's; F(v) = L_{m^l}(v);
 *   oracle_lag_node      the same bilinear forms with the change of basis M_m applied on the
 *                        particle side: the node charges of a square, M_m v_m, are formed
 *                        straight from its particles at every level as sum_c h_m(c) (STEP4:
 *                        M_m h_{m^0}(c) = h_m(c) exactly, since both sides interpolate a
 *                        polynomial of degree < n per axis), the node-to-node matrix M_b of
 *                        every interaction-list pair is applied to them, and the potential at
 *                        a charge is sum over levels of h_m(c) . (node potentials of m).  In
 *                        exact arithmetic it equals oracle_lag_literal; in FP64 it does not
 *                        lose the digits that M_m's large entries cost the literal form
 *                        (Sec. 4, Discussion (3)).
 *
 * Readings where the paper is silent or its figures are missing (Fig. 3, Fig. 4):
 *   * nodes: n = 4 per axis; in a square (cube) of side s centred at c the node coordinates
 *     per axis are c + (s/5) a_i with a = {-2, -1, 1, 2} -- Eq. 2's node values for the
 *     paper's box of side 5, scaled with the square;
 *   * f_i(x) = prod_{j != i} (x - a_j) / (a_i - a_j) (Eq. 1, its garbled "g_i(a_i)" read as
 *     g(a_i)), with x the charge's local coordinate (position - c) / (s/5);
 *   * h_m(c) = q_c f_i(x) f_j(y) [f_k(z)] on node (i, j[, k]), node index i + 4j + 16k;
 *   * the root box is [0, box]^D with its nodes at box/2 + (box/5) a_i; a charge's finest
 *     square is floor(x 2^l / box) per axis in FP64, clamped to [0, 2^l - 1];
 *   * interaction list of a level-k square (k >= 2): the children of its parent and of the
 *     parent's neighbours that are not adjacent to it (up to 27 in 2D, 189 in 3D); the near
 *     field is the own and adjacent finest squares (Sec. 2.1, E-2), j = i excluded and
 *     coincident pairs contributing 0;
 *   * the dual vectors of all levels 2..l are summed (as in the complex-moment oracle).
 *
 * kernel = 1 replaces K by a fixed polynomial of degree 3 per axis in the difference of the
 * two positions.  Lagrange interpolation on 4 nodes reproduces it exactly (Eq. 1), so both
 * FMM forms then equal the direct sum up to rounding: that is the pin of the two forms.
 * skip_level >= 2 leaves that level's far field out (a planted mistake for the pins).
 *
 * Loops over independent outputs carry OpenMP pragmas; no reduction crosses threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LAG_OK 0
#define LAG_ERR_ARG 1
#define LAG_ERR_OUT_OF_BOX 2
#define LAG_ERR_NOMEM 3
#define LAG_N 4

static const double lag_a[LAG_N] = {-2.0, -1.0, 1.0, 2.0};

/* Eq. 1: the Lagrange basis f_i on the nodes a, at local coordinate x. */
void oracle_lag_weights1(double x, double *w) {
    for (int i = 0; i < LAG_N; ++i) {
        double num = 1.0, den = 1.0;
        for (int j = 0; j < LAG_N; ++j) {
            if (j == i) continue;
            num *= x - lag_a[j];
            den *= lag_a[i] - lag_a[j];
        }
        w[i] = num / den;
    }
}

static int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

/* Number of nodes d = n^D. */
static int nodes_of(int dim) { return dim == 2 ? 16 : 64; }

/* STEP2: the weights f_i(x) f_j(y) [f_k(z)] of a point in the square (level, cell[]) of the
 * box [0, box]^dim, unit charge.  w has d entries. */
static void node_weights(int dim, int level, const int *cell, double box, const double *pos, double *w) {
    double s = box / (double)(1 << level);
    double wa[3][LAG_N];
    for (int a = 0; a < dim; ++a) {
        double c = ((double)cell[a] + 0.5) * s;
        oracle_lag_weights1((pos[a] - c) / (s / 5.0), wa[a]);
    }
    int d = nodes_of(dim);
    for (int j = 0; j < d; ++j) {
        int i0 = j % LAG_N, i1 = (j / LAG_N) % LAG_N, i2 = j / (LAG_N * LAG_N);
        double v = wa[0][i0] * wa[1][i1];
        if (dim == 3) v *= wa[2][i2];
        w[j] = v;
    }
}

/* STEP1: the position of node j of the square (level, cell[]). */
static void node_pos(int dim, int level, const int *cell, double box, int j, double *pos) {
    double s = box / (double)(1 << level);
    int ii[3] = {j % LAG_N, (j / LAG_N) % LAG_N, j / (LAG_N * LAG_N)};
    for (int a = 0; a < dim; ++a) pos[a] = ((double)cell[a] + 0.5) * s + (s / 5.0) * lag_a[ii[a]];
}

/* The test polynomial of kernel 1: degree 3 per axis, not symmetric under r -> -r. */
static double poly_kernel(int dim, const double *r) {
    double x = r[0], y = r[1], z = dim == 3 ? r[2] : 0.0;
    double v = 1.0 + 0.3 * x - 0.2 * y + 0.1 * x * x * y - 0.05 * x * x * x + 0.07 * y * y * y * x * x
               + 0.02 * x * x * x * y * y * y;
    if (dim == 3) v += 0.4 * z - 0.03 * z * z * z * x + 0.01 * x * y * z * z * z;
    return v;
}

/* The pairwise interaction K(a, b) of a unit charge at b seen at a (0 for coincident points). */
static double kernel_eval(int dim, int kernel, const double *a, const double *b) {
    double r[3] = {0.0, 0.0, 0.0}, r2 = 0.0;
    for (int k = 0; k < dim; ++k) {
        r[k] = a[k] - b[k];
        r2 += r[k] * r[k];
    }
    if (kernel == 1) return poly_kernel(dim, r);
    if (r2 == 0.0) return 0.0;
    return dim == 2 ? 0.5 * log(r2) : 1.0 / sqrt(r2);
}

static int finest_coord(double x, int levels, double box) {
    double f = floor(x * (double)(1 << levels) / box);
    int side = 1 << levels;
    if (f < 0.0) return 0;
    if (f > (double)(side - 1)) return side - 1;
    return (int)f;
}

static int check_args(int dim, int kernel, int64_t n, const double *pos, int levels, double box) {
    if ((dim != 2 && dim != 3) || (kernel != 0 && kernel != 1) || n < 0 || levels < 0 || !(box > 0.0))
        return LAG_ERR_ARG;
    if ((dim == 2 && levels > 8) || (dim == 3 && levels > 5)) return LAG_ERR_ARG;
    for (int64_t i = 0; i < n * dim; ++i)
        if (!(pos[i] >= 0.0 && pos[i] <= box)) return LAG_ERR_OUT_OF_BOX;
    return LAG_OK;
}

/* The definition: phi_i = sum_{j != i} q_j K(c_i, c_j). */
int oracle_lag_direct(int dim, int kernel, int64_t n, const double *pos, const double *q, double *phi) {
    if ((dim != 2 && dim != 3) || (kernel != 0 && kernel != 1) || n < 0) return LAG_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i) acc += q[j] * kernel_eval(dim, kernel, pos + i * dim, pos + j * dim);
        phi[i] = acc;
    }
    return LAG_OK;
}

/* The definition at chosen targets only. */
int oracle_lag_direct_targets(int dim, int kernel, int64_t n, const double *pos, const double *q, int64_t nt,
                              const int64_t *tgt, double *phi) {
    if ((dim != 2 && dim != 3) || (kernel != 0 && kernel != 1) || n < 0 || nt < 0) return LAG_ERR_ARG;
    for (int64_t t = 0; t < nt; ++t)
        if (tgt[t] < 0 || tgt[t] >= n) return LAG_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = tgt[t];
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i) acc += q[j] * kernel_eval(dim, kernel, pos + i * dim, pos + j * dim);
        phi[t] = acc;
    }
    return LAG_OK;
}

/* ------------------------------------------------------------------------------ the tree */

typedef struct {
    int dim, levels, d;
    double box;
    int64_t n;
    int *cell;        /* [n][dim] finest cell of every charge */
    int64_t *start;   /* [nleaf + 1] charges of each finest square, in order[] */
    int64_t *order;
} lag_tree;

static void tree_free(lag_tree *t) {
    free(t->cell);
    free(t->start);
    free(t->order);
}

static int64_t cell_index(int dim, int level, const int *c) {
    int64_t side = (int64_t)1 << level, idx = 0;
    for (int a = dim - 1; a >= 0; --a) idx = idx * side + c[a];
    return idx;
}

static void cell_coords(int dim, int level, int64_t idx, int *c) {
    int64_t side = (int64_t)1 << level;
    for (int a = 0; a < dim; ++a) {
        c[a] = (int)(idx % side);
        idx /= side;
    }
}

static int tree_build(lag_tree *t, int dim, int64_t n, const double *pos, int levels, double box) {
    memset(t, 0, sizeof(*t));
    t->dim = dim; t->levels = levels; t->box = box; t->n = n; t->d = nodes_of(dim);
    int64_t nleaf = ipow((int64_t)1 << levels, dim);
    t->cell = malloc(sizeof(int) * (size_t)(n > 0 ? n * dim : 1));
    t->start = calloc((size_t)nleaf + 1, sizeof(int64_t));
    t->order = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!t->cell || !t->start || !t->order) { tree_free(t); return LAG_ERR_NOMEM; }
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < dim; ++a) t->cell[i * dim + a] = finest_coord(pos[i * dim + a], levels, box);
    for (int64_t i = 0; i < n; ++i) t->start[cell_index(dim, levels, t->cell + i * dim) + 1]++;
    for (int64_t b = 0; b < nleaf; ++b) t->start[b + 1] += t->start[b];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)nleaf);
    if (!fill) { tree_free(t); return LAG_ERR_NOMEM; }
    memcpy(fill, t->start, sizeof(int64_t) * (size_t)nleaf);
    for (int64_t i = 0; i < n; ++i) t->order[fill[cell_index(dim, levels, t->cell + i * dim)]++] = i;
    free(fill);
    return LAG_OK;
}

/* The level-k square of charge i. */
static void cell_at(const lag_tree *t, int64_t i, int k, int *c) {
    for (int a = 0; a < t->dim; ++a) c[a] = t->cell[i * t->dim + a] >> (t->levels - k);
}

/* Sec. 2.1 item 5: the interaction list of square m at level k >= 2.  Returns the count and
 * writes the members' indices. */
static int interaction_list(int dim, int k, const int *m, int64_t *out) {
    int side = 1 << k, cnt = 0;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        int p = m[a] >> 1;
        lo[a] = 2 * (p - 1) < 0 ? 0 : 2 * (p - 1);
        hi[a] = 2 * (p + 1) + 1 > side - 1 ? side - 1 : 2 * (p + 1) + 1;
    }
    int c[3] = {0, 0, 0};
    for (c[2] = (dim == 3 ? lo[2] : 0); c[2] <= (dim == 3 ? hi[2] : 0); ++c[2])
        for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
            for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0]) {
                int cheb = 0;
                for (int a = 0; a < dim; ++a) {
                    int dd = abs(c[a] - m[a]);
                    if (dd > cheb) cheb = dd;
                }
                if (cheb >= 2) out[cnt++] = cell_index(dim, k, c);
            }
    return cnt;
}

/* Sec. 2.1 E-2: the near field of charge i, its own and the adjacent finest squares. */
static double near_field(const lag_tree *t, int kernel, const double *pos, const double *q, int64_t i) {
    int dim = t->dim, side = 1 << t->levels;
    const int *m = t->cell + i * dim;
    double acc = 0.0;
    int o[3] = {0, 0, 0};
    for (o[2] = (dim == 3 ? -1 : 0); o[2] <= (dim == 3 ? 1 : 0); ++o[2])
        for (o[1] = -1; o[1] <= 1; ++o[1])
            for (o[0] = -1; o[0] <= 1; ++o[0]) {
                int c[3] = {0, 0, 0}, inside = 1;
                for (int a = 0; a < dim; ++a) {
                    c[a] = m[a] + o[a];
                    if (c[a] < 0 || c[a] >= side) inside = 0;
                }
                if (!inside) continue;
                int64_t b = cell_index(dim, t->levels, c);
                for (int64_t s = t->start[b]; s < t->start[b + 1]; ++s) {
                    int64_t j = t->order[s];
                    if (j != i) acc += q[j] * kernel_eval(dim, kernel, pos + i * dim, pos + j * dim);
                }
            }
    return acc;
}

/* STEP4: M_m, column l = h_m(p_l) for a unit charge at the root box's node p_l.  M is d x d,
 * row-major (M[j * d + l] = weight of m's node j for p_l). */
int oracle_lag_matrix_M(int dim, int level, const int *cell, double box, double *M) {
    if ((dim != 2 && dim != 3) || level < 0 || !(box > 0.0)) return LAG_ERR_ARG;
    int d = nodes_of(dim), root[3] = {0, 0, 0};
    double *w = malloc(sizeof(double) * (size_t)d);
    if (!w) return LAG_ERR_NOMEM;
    for (int l = 0; l < d; ++l) {
        double p[3];
        node_pos(dim, 0, root, box, l, p);
        node_weights(dim, level, cell, box, p, w);
        for (int j = 0; j < d; ++j) M[j * d + l] = w[j];
    }
    free(w);
    return LAG_OK;
}

/* STEP2 as a standalone: the unit-charge weights of a point in the square (level, cell). */
int oracle_lag_weights(int dim, int level, const int *cell, double box, const double *pos, double *w) {
    if ((dim != 2 && dim != 3) || level < 0 || !(box > 0.0)) return LAG_ERR_ARG;
    node_weights(dim, level, cell, box, pos, w);
    return LAG_OK;
}

/* ------------------------------------------------------------------ the paper's literal form */

int oracle_lag_literal(int dim, int kernel, int64_t n, const double *pos, const double *q, int levels, double box,
                       int skip_level, double *phi) {
    int rc = check_args(dim, kernel, n, pos, levels, box);
    if (rc) return rc;
    lag_tree t;
    if ((rc = tree_build(&t, dim, n, pos, levels, box))) return rc;
    const int d = t.d, root[3] = {0, 0, 0};
    /* per level: v (U-bar) and u (D-bar), d doubles per square */
    double *v[9] = {0}, *u[9] = {0};
    int64_t ncell[9];
    for (int k = 0; k <= levels; ++k) {
        ncell[k] = ipow((int64_t)1 << k, dim);
        v[k] = calloc((size_t)(ncell[k] * d), sizeof(double));
        u[k] = calloc((size_t)(ncell[k] * d), sizeof(double));
        if (!v[k] || !u[k]) { rc = LAG_ERR_NOMEM; goto done; }
    }
    /* STEP2 / U-bar-1: v_c = h_{m^0}(c); v of a finest square = sum of its charges' v_c */
    {
        double *w = malloc(sizeof(double) * (size_t)d);
        if (!w) { rc = LAG_ERR_NOMEM; goto done; }
        for (int64_t i = 0; i < n; ++i) {
            node_weights(dim, 0, root, box, pos + i * dim, w);
            int64_t b = cell_index(dim, levels, t.cell + i * dim);
            for (int j = 0; j < d; ++j) v[levels][b * d + j] += q[i] * w[j];
        }
        free(w);
    }
    /* U-bar-2: v of a level-k square = sum of its children's, no shift */
    for (int k = levels - 1; k >= 0; --k)
        for (int64_t b = 0; b < ncell[k + 1]; ++b) {
            int c[3];
            cell_coords(dim, k + 1, b, c);
            for (int a = 0; a < dim; ++a) c[a] >>= 1;
            int64_t pb = cell_index(dim, k, c);
            for (int j = 0; j < d; ++j) v[k][pb * d + j] += v[k + 1][b * d + j];
        }
    /* D-bar-1: u~_m = sum_{m_i in IL(m)} B_{m_i,m}^T v_{m_i}, B = M_{m_i}^T M_b M_m (STEP5) */
    for (int k = 2; k <= levels; ++k) {
        if (k == skip_level) continue;
#pragma omp parallel
        {
            double *Mi = malloc(sizeof(double) * (size_t)(d * d)), *Mm = malloc(sizeof(double) * (size_t)(d * d));
            double *Mb = malloc(sizeof(double) * (size_t)(d * d)), *T = malloc(sizeof(double) * (size_t)(d * d));
            double *B = malloc(sizeof(double) * (size_t)(d * d));
            int64_t il[189];
            if (Mi && Mm && Mb && T && B) {
#pragma omp for schedule(dynamic, 1)
                for (int64_t mb = 0; mb < ncell[k]; ++mb) {
                    int m[3];
                    cell_coords(dim, k, mb, m);
                    oracle_lag_matrix_M(dim, k, m, box, Mm);
                    int cnt = interaction_list(dim, k, m, il);
                    for (int e = 0; e < cnt; ++e) {
                        int mi[3];
                        cell_coords(dim, k, il[e], mi);
                        oracle_lag_matrix_M(dim, k, mi, box, Mi);
                        /* STEP3: M_b[i][j] = phi(c_1^i, c_2^j), node i of m_i, node j of m */
                        for (int i = 0; i < d; ++i) {
                            double pi[3];
                            node_pos(dim, k, mi, box, i, pi);
                            for (int j = 0; j < d; ++j) {
                                double pj[3];
                                node_pos(dim, k, m, box, j, pj);
                                Mb[i * d + j] = kernel_eval(dim, kernel, pj, pi);
                            }
                        }
                        /* T = M_b M_m, B = M_{m_i}^T T */
                        for (int i = 0; i < d; ++i)
                            for (int l = 0; l < d; ++l) {
                                double s = 0.0;
                                for (int j = 0; j < d; ++j) s += Mb[i * d + j] * Mm[j * d + l];
                                T[i * d + l] = s;
                            }
                        for (int a = 0; a < d; ++a)
                            for (int l = 0; l < d; ++l) {
                                double s = 0.0;
                                for (int i = 0; i < d; ++i) s += Mi[i * d + a] * T[i * d + l];
                                B[a * d + l] = s;
                            }
                        /* the linear form B(v_{m_i}, .) as a dual vector */
                        const double *vi = v[k] + il[e] * d;
                        for (int l = 0; l < d; ++l) {
                            double s = 0.0;
                            for (int a = 0; a < d; ++a) s += vi[a] * B[a * d + l];
                            u[k][mb * d + l] += s;
                        }
                    }
                }
            } else {
#pragma omp critical
                rc = LAG_ERR_NOMEM;
            }
            free(Mi); free(Mm); free(Mb); free(T); free(B);
        }
        if (rc) goto done;
    }
    /* D-bar-2: L_{m^{k+1}} = L~_{m^{k+1}} + L_{m^k}, top down (levels 0 and 1 have none) */
    for (int k = 1; k <= levels; ++k)
        for (int64_t b = 0; b < ncell[k]; ++b) {
            int c[3];
            cell_coords(dim, k, b, c);
            for (int a = 0; a < dim; ++a) c[a] >>= 1;
            int64_t pb = cell_index(dim, k - 1, c);
            for (int j = 0; j < d; ++j) u[k][b * d + j] += u[k - 1][pb * d + j];
        }
    /* F(v) = L_{m^l}(v) for the charge's own v_c (unit charge), plus the near field */
#pragma omp parallel
    {
        double *w = malloc(sizeof(double) * (size_t)d);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            node_weights(dim, 0, root, box, pos + i * dim, w);
            int64_t b = cell_index(dim, levels, t.cell + i * dim);
            double far = 0.0;
            for (int j = 0; j < d; ++j) far += u[levels][b * d + j] * w[j];
            phi[i] = far + near_field(&t, kernel, pos, q, i);
        }
        free(w);
    }
done:
    for (int k = 0; k <= levels; ++k) { free(v[k]); free(u[k]); }
    tree_free(&t);
    return rc;
}

/* ----------------------------------------------------------- the node-charge (change of basis) form */

int oracle_lag_node(int dim, int kernel, int64_t n, const double *pos, const double *q, int levels, double box,
                    int skip_level, double *phi) {
    int rc = check_args(dim, kernel, n, pos, levels, box);
    if (rc) return rc;
    lag_tree t;
    if ((rc = tree_build(&t, dim, n, pos, levels, box))) return rc;
    const int d = t.d;
    double *Q[9] = {0}, *psi[9] = {0};
    int64_t ncell[9];
    for (int k = 2; k <= levels; ++k) {
        ncell[k] = ipow((int64_t)1 << k, dim);
        Q[k] = calloc((size_t)(ncell[k] * d), sizeof(double));
        psi[k] = calloc((size_t)(ncell[k] * d), sizeof(double));
        if (!Q[k] || !psi[k]) { rc = LAG_ERR_NOMEM; goto done; }
    }
    /* node charges M_m v_m = sum_{c in m} h_m(c), every level straight from the charges */
    {
        double *w = malloc(sizeof(double) * (size_t)d);
        if (!w) { rc = LAG_ERR_NOMEM; goto done; }
        for (int k = 2; k <= levels; ++k)
            for (int64_t i = 0; i < n; ++i) {
                int c[3];
                cell_at(&t, i, k, c);
                node_weights(dim, k, c, box, pos + i * dim, w);
                int64_t b = cell_index(dim, k, c);
                for (int j = 0; j < d; ++j) Q[k][b * d + j] += q[i] * w[j];
            }
        free(w);
    }
    /* node potentials of m: psi_m[j] = sum_{m_i in IL(m)} sum_i M_b[i][j] Q_{m_i}[i] */
    for (int k = 2; k <= levels; ++k) {
        if (k == skip_level) continue;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t mb = 0; mb < ncell[k]; ++mb) {
            int m[3];
            int64_t il[189];
            cell_coords(dim, k, mb, m);
            int cnt = interaction_list(dim, k, m, il);
            for (int e = 0; e < cnt; ++e) {
                int mi[3];
                cell_coords(dim, k, il[e], mi);
                for (int j = 0; j < d; ++j) {
                    double pj[3], s = 0.0;
                    node_pos(dim, k, m, box, j, pj);
                    for (int i = 0; i < d; ++i) {
                        double pi[3];
                        node_pos(dim, k, mi, box, i, pi);
                        s += kernel_eval(dim, kernel, pj, pi) * Q[k][il[e] * d + i];
                    }
                    psi[k][mb * d + j] += s;
                }
            }
        }
    }
    /* phi_far(c) = sum_k h_{m_k}(c) . psi_{m_k}, plus the near field */
#pragma omp parallel
    {
        double *w = malloc(sizeof(double) * (size_t)d);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            double far = 0.0;
            for (int k = 2; k <= levels; ++k) {
                int c[3];
                cell_at(&t, i, k, c);
                node_weights(dim, k, c, box, pos + i * dim, w);
                int64_t b = cell_index(dim, k, c);
                for (int j = 0; j < d; ++j) far += w[j] * psi[k][b * d + j];
            }
            phi[i] = far + near_field(&t, kernel, pos, q, i);
        }
        free(w);
    }
done:
    for (int k = 2; k <= levels; ++k) { free(Q[k]); free(psi[k]); }
    tree_free(&t);
    return rc;
}

/* The finest cell of every charge by the rule above (for bit-exact binning checks). */
int oracle_lag_cells(int dim, int64_t n, const double *pos, int levels, double box, int *cell) {
    if ((dim != 2 && dim != 3) || n < 0 || levels < 0 || levels > 12 || !(box > 0.0)) return LAG_ERR_ARG;
    for (int64_t i = 0; i < n * dim; ++i) cell[i] = finest_coord(pos[i], levels, box);
    return LAG_OK;
}
