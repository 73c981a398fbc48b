/* Oracle of the phylogenetic Brownian prior (Section 2.2, Eq. 2) by its dense
 * definition, in long double.
 *
 * TEST INFRASTRUCTURE: used only by the tests and the bench's CPU legs.
 *
 * z ~ N(0, sigma^2 V) with V_ij = root_var + (root-to-MRCA time of tips i
 * and j): the time from the root to a node is the sum of the branch lengths
 * on its root path.  With short tip branches V is badly conditioned (the
 * information sits in differences V_ii - V_ij of a few 1e-7 between entries
 * near 1), so V is built and factored in long double: a plain Cholesky
 * V = L L^T, then
 *   log N(z; 0, sigma^2 V) = -M/2 log(2 pi sigma^2) - sum_i log L_ii - 1/2 |L^-1 z|^2 / sigma^2,
 *   (sigma^2 V)^-1 z = L^-T L^-1 z / sigma^2,
 *   ((sigma^2 V)^-1)_ij = sum_k (L^-1)_ki (L^-1)_kj / sigma^2.
 *
 * Tree encoding: nodes 0..M-1 are the tips, M..2M-2 internal, parent[v] = -1
 * at the root, length[v] = branch length from v to its parent.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef long double ld;

/* time from the root to every node, and every node's depth in edges */
static int root_times(int64_t nn, const int64_t *parent, const double *length, ld *tr, int64_t *depth) {
    for (int64_t v = 0; v < nn; ++v) {
        ld acc = 0.0L;
        int64_t d = 0, u = v;
        while (parent[u] >= 0) {
            acc += (ld)length[u];
            u = parent[u];
            if (++d > nn) return -1; /* a cycle */
        }
        tr[v] = acc;
        depth[v] = d;
    }
    return 0;
}

static int64_t mrca(const int64_t *parent, const int64_t *depth, int64_t a, int64_t b) {
    while (depth[a] > depth[b]) a = parent[a];
    while (depth[b] > depth[a]) b = parent[b];
    while (a != b) {
        a = parent[a];
        b = parent[b];
    }
    return a;
}

/* V (row-major, M x M, long double) into v; returns 0 or -1 for a malformed tree */
static int build_cov(int64_t m, const int64_t *parent, const double *length, double root_var, ld *v) {
    const int64_t nn = 2 * m - 1;
    ld *tr = malloc(sizeof(ld) * nn);
    int64_t *depth = malloc(sizeof(int64_t) * nn);
    if (!tr || !depth || root_times(nn, parent, length, tr, depth) != 0) {
        free(tr);
        free(depth);
        return -1;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = i; j < m; ++j) {
            const ld s = (ld)root_var + tr[mrca(parent, depth, i, j)];
            v[i * m + j] = s;
            v[j * m + i] = s;
        }
    free(tr);
    free(depth);
    return 0;
}

/* in place: lower triangle of a becomes L with a = L L^T; -1 if not positive definite */
static int cholesky(int64_t m, ld *a) {
    for (int64_t j = 0; j < m; ++j) {
        ld d = a[j * m + j];
        for (int64_t k = 0; k < j; ++k) d -= a[j * m + k] * a[j * m + k];
        if (!(d > 0.0L)) return -1;
        const ld ljj = sqrtl(d);
        a[j * m + j] = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < m; ++i) {
            ld s = a[i * m + j];
            for (int64_t k = 0; k < j; ++k) s -= a[i * m + k] * a[j * m + k];
            a[i * m + j] = s / ljj;
        }
    }
    return 0;
}

int tree_oracle_cov(int64_t m, const int64_t *parent, const double *length, double root_var, double *out) {
    ld *v = malloc(sizeof(ld) * m * m);
    if (!v) return -1;
    if (build_cov(m, parent, length, root_var, v) != 0) {
        free(v);
        return -1;
    }
    for (int64_t k = 0; k < m * m; ++k) out[k] = (double)v[k];
    free(v);
    return 0;
}

/* Outputs (any may be NULL): logdens[1], pz[m], pdiag[m], prec[m*m] (the full (sigma^2 V)^-1). */
int tree_oracle_prior(int64_t m, const int64_t *parent, const double *length, double root_var, double sigma2,
                      const double *z, double *logdens, double *pz, double *pdiag, double *prec) {
    ld *a = malloc(sizeof(ld) * m * m);
    ld *w = malloc(sizeof(ld) * m);
    if (!a || !w) {
        free(a);
        free(w);
        return -1;
    }
    if (build_cov(m, parent, length, root_var, a) != 0 || cholesky(m, a) != 0) {
        free(a);
        free(w);
        return -1;
    }
    const ld s2 = (ld)sigma2;
    if (z && (logdens || pz)) {
        /* w = L^-1 z */
        for (int64_t i = 0; i < m; ++i) {
            ld s = (ld)z[i];
            for (int64_t k = 0; k < i; ++k) s -= a[i * m + k] * w[k];
            w[i] = s / a[i * m + i];
        }
        if (logdens) {
            ld quad = 0.0L, logdet_half = 0.0L;
            for (int64_t i = 0; i < m; ++i) {
                quad += w[i] * w[i];
                logdet_half += logl(a[i * m + i]);
            }
            const ld log_2pi = 1.837877066409345483560659472811235279722794947275566825634L;
            *logdens = (double)(-0.5L * (ld)m * (log_2pi + logl(s2)) - logdet_half - 0.5L * quad / s2);
        }
        if (pz) {
            /* x = L^-T w */
            for (int64_t i = m - 1; i >= 0; --i) {
                ld s = w[i];
                for (int64_t k = i + 1; k < m; ++k) s -= a[k * m + i] * w[k];
                w[i] = s / a[i * m + i];
            }
            for (int64_t i = 0; i < m; ++i) pz[i] = (double)(w[i] / s2);
        }
    }
    if (pdiag || prec) {
        /* columns of L^-1: column c has rows c..m-1; (V^-1)_ij = sum_k Linv[k][i] Linv[k][j] */
        ld *li = calloc((size_t)(m * m), sizeof(ld)); /* li[k*m + c] = (L^-1)_{kc} */
        if (!li) {
            free(a);
            free(w);
            return -1;
        }
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t c = 0; c < m; ++c) {
            for (int64_t i = c; i < m; ++i) {
                ld s = (i == c) ? 1.0L : 0.0L;
                for (int64_t k = c; k < i; ++k) s -= a[i * m + k] * li[k * m + c];
                li[i * m + c] = s / a[i * m + i];
            }
        }
        if (pdiag) {
            for (int64_t c = 0; c < m; ++c) {
                ld s = 0.0L;
                for (int64_t k = c; k < m; ++k) s += li[k * m + c] * li[k * m + c];
                pdiag[c] = (double)(s / s2);
            }
        }
        if (prec) {
#pragma omp parallel for schedule(dynamic, 8)
            for (int64_t i = 0; i < m; ++i)
                for (int64_t j = i; j < m; ++j) {
                    ld s = 0.0L;
                    for (int64_t k = j; k < m; ++k) s += li[k * m + i] * li[k * m + j];
                    prec[i * m + j] = prec[j * m + i] = (double)(s / s2);
                }
        }
        free(li);
    }
    free(a);
    free(w);
    return 0;
}
