// The phylogenetic Brownian prior on the sequenced log-rates (Section 2.2,
// Eq. 2) in O(M) by message passing on the tree (the dynamic programme of
// Section 2.3.1), with no M x M matrix.
//
// z ~ N(0, sigma^2 V), V_ij = tau0 + (length of the root path shared by tips i
// and j).  Post-order (independent contrasts): for an internal node v with
// children a, b and extended branch lengths l_a = len_a + d_a, l_b = len_b + d_b,
//     s_v = l_a + l_b,   m_v = (m_a l_b + m_b l_a) / s_v,   d_v = l_a l_b / s_v,
//     u_v = m_a - m_b,
// with m = z and d = 0 at the tips.  Then
//     z^T V^-1 z = sum_v u_v^2 / s_v + m_root^2 / (d_root + tau0),
//     log |V|    = sum_v log s_v + log(d_root + tau0).
// Pre-order, the adjoint of the quadratic form (halved): G_root = m_root /
// (d_root + tau0) and, for each internal v,
//     G_a = (l_b / s_v) G_v + u_v / s_v,   G_b = (l_a / s_v) G_v - u_v / s_v,
// so that G at tip i is (V^-1 z)_i.  The same sweep gives diag(V^-1): with
// D_root = 1 / (d_root + tau0) and
//     D_a = 1 / s_v + (l_b / s_v)^2 D_v,   D_b = 1 / s_v + (l_a / s_v)^2 D_v,
// D at tip i is (V^-1)_ii (the quadratic form's Hessian is the sum of squared
// contrast gradients, and each contrast above a node sees that node's m
// through the product of the l_other / s factors on the way up).
// One block sweeps the internal nodes level by level, children before parents.
// FP64 division is costly on this part and the block runs on one SM, so each
// node takes one reciprocal 1/s_v in the upward sweep and keeps it for the
// downward one; the logarithms of log |V| are taken only when the density is
// requested.
#include <stdlib.h>
#include <string.h>

#include "hawkes_internal.cuh"

namespace hk {

constexpr int TREE_THREADS = 1024;

// plan layout (int32): [0] levels L, [1] m, then parent[2m-1], ca[2m-1], cb[2m-1],
// order[m-1] (internal nodes, level 1 first), offs[L+1] (start of each level in order)
struct TreePlan {
    int levels, m;
    const int *parent, *ca, *cb, *order, *offs;
};

__host__ __device__ inline TreePlan tree_plan_view(const int *p) {
    TreePlan t;
    t.levels = p[0];
    t.m = p[1];
    const int nn = 2 * t.m - 1;
    t.parent = p + 2;
    t.ca = t.parent + nn;
    t.cb = t.ca + nn;
    t.order = t.cb + nn;
    t.offs = t.order + (t.m - 1);
    return t;
}

// Trees of up to TREE_SMEM_MAX_TIPS tips run with every array staged in shared
// memory (the sweeps are a chain of dependent loads per level, which shared
// memory serves in a few cycles); larger trees use the caller's scratch.
constexpr int TREE_SMEM_MAX_TIPS = 1860;  // dynamic + the static 8 KB reduction buffer <= 227 KB

__host__ __device__ inline size_t tree_smem_bytes(int64_t m) {
    // 6 doubles (mu, dl, gb, dd, 1/s, length) and 2 ints (children) per node,
    // then the level order (m - 1) and the level offsets (at most m)
    return (size_t)(2 * m - 1) * (6 * sizeof(double) + 2 * sizeof(int)) + (size_t)(2 * m) * sizeof(int) + 64;
}

// STAGED: the plan and lengths are copied into shared memory and the state
// arrays live there; otherwise mu, dl, gb, dd, is are the global scratch
// (2m-1 doubles each; is_v = 1 / s_v).
template <bool STAGED>
__global__ void __launch_bounds__(TREE_THREADS)
    tree_prior_kernel(int64_t m_arg, const int *__restrict__ plan, const double *__restrict__ len_g, double tau0,
                      double sigma2, const double *__restrict__ z, double *mu, double *dl, double *gb, double *dd,
                      double *is, double *__restrict__ logdens, double *__restrict__ pz, double *__restrict__ pdiag) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char tree_smem[];
    __shared__ double sh[TREE_THREADS];
    TreePlan T = tree_plan_view(plan);
    const int m = T.m;
    if ((int64_t)m != m_arg || T.levels < 1 || T.levels > m - 1) {  // a plan for another tree: touch no scratch
        for (int64_t i = threadIdx.x; i < m_arg; i += TREE_THREADS) {
            if (pz) pz[i] = NAN;
            if (pdiag) pdiag[i] = NAN;
        }
        if (logdens && threadIdx.x == 0) *logdens = NAN;
        return;
    }
    const int nn = 2 * m - 1;
    const double *len = len_g;
    if (STAGED) {
        double *base = reinterpret_cast<double *>(tree_smem);
        mu = base;
        dl = mu + nn;
        gb = dl + nn;
        dd = gb + nn;
        is = dd + nn;
        double *len_s = is + nn;
        int *ca = reinterpret_cast<int *>(len_s + nn), *cb = ca + nn, *order = cb + nn, *offs = order + (m - 1);
        for (int v = threadIdx.x; v < nn; v += TREE_THREADS) {
            len_s[v] = len_g[v];
            ca[v] = T.ca[v];
            cb[v] = T.cb[v];
        }
        for (int k = threadIdx.x; k < m - 1; k += TREE_THREADS) order[k] = T.order[k];
        for (int k = threadIdx.x; k <= T.levels; k += TREE_THREADS) offs[k] = T.offs[k];
        len = len_s;
        T.ca = ca;
        T.cb = cb;
        T.order = order;
        T.offs = offs;
    }
    for (int i = threadIdx.x; i < m; i += TREE_THREADS) {
        mu[i] = z[i];
        dl[i] = 0.0;
    }
    __syncthreads();
    const bool want_density = logdens != nullptr;
    double quad = 0.0, logdet = 0.0;
    for (int L = 0; L < T.levels; ++L) {
        for (int k = T.offs[L] + threadIdx.x; k < T.offs[L + 1]; k += TREE_THREADS) {
            const int v = T.order[k], a = T.ca[v], b = T.cb[v];
            const double la = len[a] + dl[a], lb = len[b] + dl[b], s = la + lb, r = 1.0 / s;
            const double u = mu[a] - mu[b];
            mu[v] = (mu[a] * lb + mu[b] * la) * r;
            dl[v] = la * lb * r;
            is[v] = r;
            if (want_density) {
                quad += u * u * r;
                logdet += log(s);
            }
        }
        __syncthreads();
    }
    const int root = T.order[m - 2];
    const double droot = dl[root] + tau0;
    if (want_density) {
        quad = block_sum<TREE_THREADS>(quad, sh);
        logdet = block_sum<TREE_THREADS>(logdet, sh);
    }
    if (threadIdx.x == 0) {
        const double ir = 1.0 / droot;
        gb[root] = mu[root] * ir;
        dd[root] = ir;
        if (want_density) {
            quad += mu[root] * mu[root] / droot;
            logdet += log(droot);
            const double LOG_2PI = 1.8378770664093454836;
            *logdens = -0.5 * (double)m * (LOG_2PI + log(sigma2)) - 0.5 * logdet - 0.5 * quad / sigma2;
        }
    }
    __syncthreads();
    for (int L = T.levels - 1; L >= 0; --L) {
        for (int k = T.offs[L] + threadIdx.x; k < T.offs[L + 1]; k += TREE_THREADS) {
            const int v = T.order[k], a = T.ca[v], b = T.cb[v];
            const double r = is[v], la = len[a] + dl[a], lb = len[b] + dl[b];
            const double uu = (mu[a] - mu[b]) * r, g = gb[v], D = dd[v];
            const double fa = lb * r, fb = la * r;
            gb[a] = fa * g + uu;
            gb[b] = fb * g - uu;
            dd[a] = r + fa * fa * D;
            dd[b] = r + fb * fb * D;
        }
        __syncthreads();
    }
    const double is2 = 1.0 / sigma2;
    for (int i = threadIdx.x; i < m; i += TREE_THREADS) {
        if (pz) pz[i] = gb[i] * is2;        // (sigma^2 V)^-1 z
        if (pdiag) pdiag[i] = dd[i] * is2;  // diag((sigma^2 V)^-1)
    }
}

cudaError_t launch_tree_prior(int64_t m, const int *plan, const double *len, double tau0, double sigma2,
                              const double *z, double *scratch, double *logdens, double *pz, double *pdiag,
                              cudaStream_t s) {
    const int64_t nn = 2 * m - 1;
    double *mu = scratch, *dl = mu + nn, *gb = dl + nn, *dd = gb + nn, *is = dd + nn;
    if (m <= TREE_SMEM_MAX_TIPS) {
        const size_t bytes = tree_smem_bytes(m);
        // the opt-in limit is a per-function, per-device attribute: set once per device
        // (outside any stream capture, since the first launch on a device is eager)
        static int attr_set[64] = {0};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
        if (dev < 0 || dev >= 64 || !attr_set[dev]) {
            const cudaError_t e = cudaFuncSetAttribute(tree_prior_kernel<true>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)tree_smem_bytes(TREE_SMEM_MAX_TIPS));
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) attr_set[dev] = 1;
        }
        launch_pdl(tree_prior_kernel<true>, 1, TREE_THREADS, bytes, s, m, plan, len, tau0, sigma2, z, mu, dl, gb, dd, is,
                                                               logdens, pz, pdiag);
    } else {
        launch_pdl(tree_prior_kernel<false>, 1, TREE_THREADS, 0, s, m, plan, len, tau0, sigma2, z, mu, dl, gb, dd, is,
                                                            logdens, pz, pdiag);
    }
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Tree-structured HMC mass matrix on the sequenced log-rates (Section 2.3.2's
// preconditioner, widened from a diagonal to the phylogenetic prior's full
// precision).  Inside the rate block [z0, z0 + m) of a k-dimensional state
//     M_z = diag(d) + (sigma^2 V)^-1,     d >= 0 (the likelihood's curvature),
// and M = diag(1 / minv) elsewhere.  M_z^-1 p is the posterior mean of the
// tips of a Brownian motion on the tree (prior N(0, sigma^2 V)) that receives
// Gaussian evidence in information form, precision d_i and information p_i,
// at tip i.  An upward sweep folds each node's evidence into a message to its
// parent across the branch of variance s = sigma^2 len:
//     J_v = d_v (tip) or J'_a + J'_b,   h_v = p_v (tip) or h'_a + h'_b,
//     r_v = 1 / (1 + s_v J_v),  J'_v = J_v r_v,  h'_v = h_v r_v,
// (the root's branch is the root variance, s = sigma^2 root_var, to a parent
// fixed at 0); the downward sweep gives the means
//     X_root = s_root h_root r_root,   X_c = X_parent r_c + (s_c r_c) h_c,
// and X at the tips is M_z^-1 p.  1 + s J >= 1, so the sweeps stay well
// conditioned however small the branches (V's condition number reaches ~1e9
// on coalescent trees).  The precisions J, hence r and s r, do not depend on
// p: tree_mass_factor_kernel computes them once per change of d (one
// reciprocal per node), and each velocity then takes an addition and a
// multiply per node up and a multiply and a multiply-add per branch down,
// no division.
//
// Optional coupling of the first nc <= 8 coordinates (the globals) with the
// rate block: M = [[A, B^T], [B, M_z]] with A (nc x nc) and B (m x nc).  With
// U = M_z^-1 B and S = A - B^T U (both supplied by the caller in cpl: U row
// by row, then S^-1, then the lower Cholesky factor of S), the Schur
// complement gives
//     x_g = S^-1 (p_g - U^T p_z),   x_z = M_z^-1 p_z - U x_g,
// one tree sweep as before plus nc dot products; and p ~ N(0, M) is p_z as
// before, then p_g = U^T p_z + chol(S) xi_g (p_g given p_z is N(U^T p_z, S)).
constexpr int TMASS_SMEM_MAX_TIPS = 2048;
constexpr int TMASS_MAX_COUPLED = HAWKES_TREE_MASS_MAX_COUPLED;

__host__ __device__ inline size_t tmass_smem_bytes(int64_t m) {
    // 4 doubles (r, s r, own h, message h / mean X) and 2 ints (children) per
    // node, then the level order (m - 1) and the level offsets (at most m)
    return (size_t)(2 * m - 1) * (4 * sizeof(double) + 2 * sizeof(int)) + (size_t)(2 * m) * sizeof(int) + 64;
}

// fac[0, nn) = r_v, fac[nn, 2 nn) = s_v r_v for every node; J is scratch (nn).
__global__ void __launch_bounds__(TREE_THREADS)
    tree_mass_factor_kernel(int64_t m_arg, const int *__restrict__ plan, const double *__restrict__ len,
                            double tau0, double sigma2, const double *__restrict__ dlik, double *__restrict__ fac,
                            double *__restrict__ J) {
    pdl_wait();
    const TreePlan T = tree_plan_view(plan);
    const int m = T.m;
    if ((int64_t)m != m_arg || T.levels < 1 || T.levels > m - 1) {  // a plan for another tree
        for (int64_t v = threadIdx.x; v < 2 * (2 * m_arg - 1); v += TREE_THREADS) fac[v] = NAN;
        return;
    }
    const int nn = 2 * m - 1;
    double *R = fac, *SR = fac + nn;
    for (int i = threadIdx.x; i < m; i += TREE_THREADS) {
        const double dv = dlik[i];
        const double d = dv > 0.0 ? dv : 0.0;  // negative or NaN curvature counts as none
        const double sv = sigma2 * len[i];
        const double r = 1.0 / fma(sv, d, 1.0);
        J[i] = d * r;
        R[i] = r;
        SR[i] = sv * r;
    }
    __syncthreads();
    const int root = T.order[m - 2];
    for (int L = 0; L < T.levels; ++L) {
        for (int j = T.offs[L] + threadIdx.x; j < T.offs[L + 1]; j += TREE_THREADS) {
            const int v = T.order[j];
            const double Jv = J[T.ca[v]] + J[T.cb[v]];
            const double sv = sigma2 * (v == root ? tau0 : len[v]);
            const double r = 1.0 / fma(sv, Jv, 1.0);
            J[v] = Jv * r;
            R[v] = r;
            SR[v] = sv * r;
        }
        __syncthreads();
    }
}

template <bool STAGED>
__global__ void __launch_bounds__(TREE_THREADS)
    tree_mass_velocity_kernel(int64_t m_arg, const int *__restrict__ plan, const double *__restrict__ fac,
                              int nc, const double *__restrict__ cpl, int64_t k, int64_t z0,
                              const double *__restrict__ minv, const double *__restrict__ p,
                              double *__restrict__ vel, double *__restrict__ q, double eps,
                              double *__restrict__ kinetic, double *H, double *HA) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char tree_smem[];
    __shared__ double sh[TREE_THREADS];
    __shared__ double s_c[TMASS_MAX_COUPLED], s_xg[TMASS_MAX_COUPLED];
    TreePlan T = tree_plan_view(plan);
    const int m = T.m;
    if ((int64_t)m != m_arg || T.levels < 1 || T.levels > m - 1) {  // a plan for another tree: touch no scratch
        for (int64_t i = threadIdx.x; i < k; i += TREE_THREADS) {
            if (vel) vel[i] = NAN;
            if (q) q[i] = NAN;
        }
        if (kinetic && threadIdx.x == 0) *kinetic = NAN;
        return;
    }
    const int nn = 2 * m - 1;
    const double *R = fac, *SR = fac + nn;
    if (STAGED) {
        double *base = reinterpret_cast<double *>(tree_smem);
        double *R_s = base, *SR_s = R_s + nn;
        H = SR_s + nn;
        HA = H + nn;
        int *ca = reinterpret_cast<int *>(HA + nn), *cb = ca + nn, *order = cb + nn, *offs = order + (m - 1);
        for (int v = threadIdx.x; v < nn; v += TREE_THREADS) {
            R_s[v] = fac[v];
            SR_s[v] = fac[nn + v];
            ca[v] = T.ca[v];
            cb[v] = T.cb[v];
        }
        for (int j = threadIdx.x; j < m - 1; j += TREE_THREADS) order[j] = T.order[j];
        for (int j = threadIdx.x; j <= T.levels; j += TREE_THREADS) offs[j] = T.offs[j];
        R = R_s;
        SR = SR_s;
        T.ca = ca;
        T.cb = cb;
        T.order = order;
        T.offs = offs;
        __syncthreads();
    }
    double kin = 0.0;
    // coordinates outside the rate block and the coupled set: the diagonal mass
    for (int64_t i = threadIdx.x; i < k; i += TREE_THREADS) {
        if ((i >= z0 && i < z0 + m) || i < nc) continue;
        const double v = minv[i] * p[i];
        if (vel) vel[i] = v;
        if (q) q[i] += eps * v;
        kin += p[i] * v;
    }
    for (int i = threadIdx.x; i < m; i += TREE_THREADS) {
        const double h = p[z0 + i];
        HA[i] = h;
        H[i] = h * R[i];
    }
    if (nc > 0) {  // c = U^T p_z (the barrier inside also orders the tips' writes above)
        double cv[TMASS_MAX_COUPLED];
#pragma unroll
        for (int j = 0; j < TMASS_MAX_COUPLED; ++j) cv[j] = 0.0;
        for (int i = threadIdx.x; i < m; i += TREE_THREADS) {
            const double pz = p[z0 + i];
#pragma unroll
            for (int j = 0; j < TMASS_MAX_COUPLED; ++j)
                if (j < nc) cv[j] = fma(cpl[(size_t)i * nc + j], pz, cv[j]);
        }
        const double c = block_sum_multi<TREE_THREADS, TMASS_MAX_COUPLED>(cv, sh);
        if (threadIdx.x < nc) s_c[threadIdx.x] = c;
    }
    __syncthreads();
    const int root = T.order[m - 2];
    for (int L = 0; L < T.levels; ++L) {
        for (int j = T.offs[L] + threadIdx.x; j < T.offs[L + 1]; j += TREE_THREADS) {
            const int v = T.order[j];
            const double hv = H[T.ca[v]] + H[T.cb[v]];
            HA[v] = hv;
            H[v] = hv * R[v];
        }
        __syncthreads();
    }
    // downward: the means X overwrite the messages H (no longer needed)
    if (threadIdx.x == 0) H[root] = SR[root] * HA[root];
    __syncthreads();
    for (int L = T.levels - 1; L >= 0; --L) {
        for (int j = T.offs[L] + threadIdx.x; j < T.offs[L + 1]; j += TREE_THREADS) {
            const int v = T.order[j], a = T.ca[v], b = T.cb[v];
            const double xv = H[v];
            H[a] = fma(xv, R[a], SR[a] * HA[a]);
            H[b] = fma(xv, R[b], SR[b] * HA[b]);
        }
        __syncthreads();
    }
    if (nc > 0) {  // x_g = S^-1 (p_g - U^T p_z), by threads 0..nc-1
        const double *Sinv = cpl + (size_t)m * nc;
        if (threadIdx.x < nc) {
            const int j = threadIdx.x;
            double x = 0.0;
            for (int l = 0; l < nc; ++l) x = fma(Sinv[j * nc + l], p[l] - s_c[l], x);
            s_xg[j] = x;
            if (vel) vel[j] = x;
            if (q) q[j] += eps * x;
            kin += p[j] * x;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < m; i += TREE_THREADS) {
        double v = H[i];
        for (int j = 0; j < nc; ++j) v = fma(-cpl[(size_t)i * nc + j], s_xg[j], v);  // x_z = M_z^-1 p_z - U x_g
        if (vel) vel[z0 + i] = v;
        if (q) q[z0 + i] += eps * v;
        kin += p[z0 + i] * v;
    }
    if (kinetic) {
        kin = block_sum<TREE_THREADS>(kin, sh);
        if (threadIdx.x == 0) *kinetic = 0.5 * kin;
    }
}

// The coupled coordinates' momentum given the rate block's: p_g = U^T p_z +
// chol(S) xi_g, xi_g = xi[0, nc).  One block.
__global__ void __launch_bounds__(TREE_THREADS)
    tree_mass_couple_momentum_kernel(int64_t m, int64_t z0, int nc, const double *__restrict__ cpl,
                                     const double *__restrict__ xi, double *__restrict__ p) {
    pdl_wait();
    __shared__ double sh[(TREE_THREADS / 32) * TMASS_MAX_COUPLED];
    double cv[TMASS_MAX_COUPLED];
#pragma unroll
    for (int j = 0; j < TMASS_MAX_COUPLED; ++j) cv[j] = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += TREE_THREADS) {
        const double pz = p[z0 + i];
#pragma unroll
        for (int j = 0; j < TMASS_MAX_COUPLED; ++j)
            if (j < nc) cv[j] = fma(cpl[(size_t)i * nc + j], pz, cv[j]);
    }
    const double c = block_sum_multi<TREE_THREADS, TMASS_MAX_COUPLED>(cv, sh);
    if (threadIdx.x < nc) {
        const int j = threadIdx.x;
        const double *Lc = cpl + (size_t)m * nc + (size_t)nc * nc;
        double v = c;
        for (int l = 0; l <= j; ++l) v = fma(Lc[j * nc + l], xi[l], v);
        p[j] = v;
    }
}

// Momentum p ~ N(0, M) from standard normals xi[k + 2m - 1]: outside the block
// p_i = xi_i / sqrt(minv_i); inside, p_z = sqrt(d) xi_z + (sigma^2 V)^-1 w with
// w ~ N(0, sigma^2 V) the Brownian motion down the tree driven by the node
// normals xi[k + v] (root: sqrt(sigma^2 root_var) xi; child: parent +
// sqrt(sigma^2 len) xi), so that Cov(p_z) = diag(d) + (sigma^2 V)^-1.  This
// kernel writes the first part and w; the prior kernel then applies
// (sigma^2 V)^-1 to w, and tree_mass_add_kernel adds it.
__global__ void __launch_bounds__(TREE_THREADS)
    tree_brownian_kernel(int64_t m_arg, const int *__restrict__ plan, const double *__restrict__ len,
                         double tau0, double sigma2, const double *__restrict__ dlik, int64_t k, int64_t z0,
                         const double *__restrict__ minv, const double *__restrict__ xi, double *__restrict__ p,
                         double *__restrict__ w) {
    pdl_wait();
    const TreePlan T = tree_plan_view(plan);
    const int m = T.m;
    const bool bad = (int64_t)m != m_arg || T.levels < 1 || T.levels > m - 1;
    for (int64_t i = threadIdx.x; i < k; i += TREE_THREADS) {
        if (bad) {
            p[i] = NAN;
        } else if (i >= z0 && i < z0 + m) {
            const double dv = dlik[i - z0];
            p[i] = sqrt(dv > 0.0 ? dv : 0.0) * xi[i];
        } else {
            p[i] = xi[i] * rsqrt(minv[i]);
        }
    }
    if (bad) {
        for (int64_t i = threadIdx.x; i < m_arg; i += TREE_THREADS) w[i] = NAN;
        return;
    }
    const double *xn = xi + k;
    const int root = T.order[m - 2];
    if (threadIdx.x == 0) w[root] = sqrt(sigma2 * tau0) * xn[root];
    __syncthreads();
    for (int L = T.levels - 1; L >= 0; --L) {
        for (int j = T.offs[L] + threadIdx.x; j < T.offs[L + 1]; j += TREE_THREADS) {
            const int v = T.order[j], a = T.ca[v], b = T.cb[v];
            const double wv = w[v];
            w[a] = fma(sqrt(sigma2 * len[a]), xn[a], wv);
            w[b] = fma(sqrt(sigma2 * len[b]), xn[b], wv);
        }
        __syncthreads();
    }
}

__global__ void tree_mass_add_kernel(int64_t m, int64_t z0, const double *__restrict__ pw, double *__restrict__ p) {
    pdl_wait();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) p[z0 + i] += pw[i];
}

cudaError_t launch_tree_mass_factor(int64_t m, const int *plan, const double *len, double tau0, double sigma2,
                                    const double *dlik, double *fac, double *scratch, cudaStream_t s) {
    launch_pdl(tree_mass_factor_kernel, 1, TREE_THREADS, 0, s, m, plan, len, tau0, sigma2, dlik, fac, scratch);
    return cudaGetLastError();
}

cudaError_t launch_tree_mass_velocity(int64_t m, const int *plan, const double *fac, int nc, const double *cpl,
                                      int64_t k, int64_t z0, const double *minv, const double *p, double *vel,
                                      double *q, double eps, double *kinetic, double *scratch, cudaStream_t s) {
    const int64_t nn = 2 * m - 1;
    double *H = scratch, *HA = H + nn;
    if (m <= TMASS_SMEM_MAX_TIPS) {
        static int attr_set[64] = {0};  // per-device opt-in, set on the first (eager) launch
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
        if (dev < 0 || dev >= 64 || !attr_set[dev]) {
            const cudaError_t e = cudaFuncSetAttribute(tree_mass_velocity_kernel<true>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)tmass_smem_bytes(TMASS_SMEM_MAX_TIPS));
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) attr_set[dev] = 1;
        }
        launch_pdl(tree_mass_velocity_kernel<true>, 1, TREE_THREADS, tmass_smem_bytes(m), s, m, plan, fac, nc, cpl, k,
                   z0, minv, p, vel, q, eps, kinetic, H, HA);
    } else {
        launch_pdl(tree_mass_velocity_kernel<false>, 1, TREE_THREADS, 0, s, m, plan, fac, nc, cpl, k, z0, minv, p, vel,
                   q, eps, kinetic, H, HA);
    }
    return cudaGetLastError();
}

cudaError_t launch_tree_mass_momentum(int64_t m, const int *plan, const double *len, double tau0, double sigma2,
                                      const double *dlik, int nc, const double *cpl, int64_t k, int64_t z0,
                                      const double *minv, const double *xi, double *p, double *scratch,
                                      cudaStream_t s) {
    const int64_t nn = 2 * m - 1;
    double *w = scratch, *pw = w + nn, *prior_scratch = pw + m;
    launch_pdl(tree_brownian_kernel, 1, TREE_THREADS, 0, s, m, plan, len, tau0, sigma2, dlik, k, z0, minv, xi, p, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_tree_prior(m, plan, len, tau0, sigma2, w, prior_scratch, nullptr, pw, nullptr, s);
    if (e != cudaSuccess) return e;
    launch_pdl(tree_mass_add_kernel, (unsigned)((m + 255) / 256), 256, 0, s, m, z0, (const double *)pw, p);
    if (nc > 0) {
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        launch_pdl(tree_mass_couple_momentum_kernel, 1, TREE_THREADS, 0, s, m, z0, nc, cpl, xi, p);
    }
    return cudaGetLastError();
}

}  // namespace hk

extern "C" {

size_t hawkes_tree_plan_size(int64_t m) {
    if (m < 2 || m > HAWKES_TREE_MAX_TIPS) return 0;
    return (size_t)(2 + 3 * (2 * m - 1) + (m - 1) + m) * sizeof(int);
}

size_t hawkes_tree_workspace_size(int64_t m) {
    if (m < 2 || m > HAWKES_TREE_MAX_TIPS) return 0;
    return (size_t)5 * (2 * m - 1) * sizeof(double);
}

int hawkes_tree_plan(int64_t m, const int64_t *parent, int *plan, size_t plan_bytes) {
    if (m < 2 || m > HAWKES_TREE_MAX_TIPS || !parent || !plan) return HAWKES_EINVAL;
    if (plan_bytes < hawkes_tree_plan_size(m)) return HAWKES_EWORKSPACE;
    const int nn = (int)(2 * m - 1), mi = (int)m;
    int *p = plan + 2;
    int *ca = p + nn, *cb = ca + nn, *order = cb + nn, *offs = order + (mi - 1);
    int roots = 0, root = -1;
    for (int v = 0; v < nn; ++v) ca[v] = cb[v] = -1;
    for (int v = 0; v < nn; ++v) {
        const int64_t pa = parent[v];
        if (pa < 0) {
            ++roots;
            root = v;
            p[v] = -1;
            continue;
        }
        if (pa < m || pa >= nn) return HAWKES_EINVAL;  // a parent must be an internal node
        p[v] = (int)pa;
        if (ca[pa] < 0) ca[pa] = v;
        else if (cb[pa] < 0) cb[pa] = v;
        else return HAWKES_EINVAL;  // more than two children
    }
    if (roots != 1 || root < mi) return HAWKES_EINVAL;
    for (int v = mi; v < nn; ++v)
        if (ca[v] < 0 || cb[v] < 0) return HAWKES_EINVAL;
    // breadth-first from the root: every node must be reached exactly once
    int *bfs = (int *)malloc(sizeof(int) * (size_t)nn);
    int *level = (int *)calloc((size_t)nn, sizeof(int));
    if (!bfs || !level) {
        free(bfs);
        free(level);
        return HAWKES_EINVAL;
    }
    int head = 0, tail = 0;
    bfs[tail++] = root;
    while (head < tail) {
        const int v = bfs[head++];
        if (v >= mi) {
            if (tail + 2 > nn) break;  // revisiting: not a tree
            bfs[tail++] = ca[v];
            bfs[tail++] = cb[v];
        }
    }
    if (tail != nn || head != nn) {
        free(bfs);
        free(level);
        return HAWKES_EINVAL;
    }
    // children follow their parent in breadth-first order: reverse sweep sets levels
    int maxl = 0;
    for (int k = nn - 1; k >= 0; --k) {
        const int v = bfs[k];
        if (v < mi) continue;
        const int l = 1 + (level[ca[v]] > level[cb[v]] ? level[ca[v]] : level[cb[v]]);
        level[v] = l;
        if (l > maxl) maxl = l;
    }
    free(bfs);
    if (maxl > mi - 1) {  // cannot happen for a binary tree on m tips
        free(level);
        return HAWKES_EINVAL;
    }
    // counting sort of the internal nodes by level: level l occupies order[offs[l-1], offs[l])
    for (int l = 0; l <= maxl; ++l) offs[l] = 0;
    for (int v = mi; v < nn; ++v) offs[level[v]]++;
    for (int l = 1; l <= maxl; ++l) offs[l] += offs[l - 1];
    int *fill = (int *)malloc(sizeof(int) * (size_t)(maxl + 1));
    if (!fill) {
        free(level);
        return HAWKES_EINVAL;
    }
    memcpy(fill, offs, sizeof(int) * (size_t)(maxl + 1));
    for (int v = mi; v < nn; ++v) order[fill[level[v] - 1]++] = v;
    free(fill);
    free(level);
    plan[0] = maxl;
    plan[1] = mi;
    return HAWKES_OK;
}

int hawkes_tree_prior(int64_t m, const int *plan, const double *length, double root_var, double sigma2,
                      const double *z, void *ws, size_t ws_bytes, double *logdens, double *pz, double *pdiag,
                      void *stream) {
    if (m < 2 || m > HAWKES_TREE_MAX_TIPS || !plan || !length || !z || !ws) return HAWKES_EINVAL;
    if (!(sigma2 > 0) || !(root_var >= 0) || !isfinite(sigma2) || !isfinite(root_var)) return HAWKES_EINVAL;
    if (ws_bytes < hawkes_tree_workspace_size(m)) return HAWKES_EWORKSPACE;
    return hk::launch_tree_prior(m, plan, length, root_var, sigma2, z, (double *)ws, logdens, pz, pdiag,
                                 (cudaStream_t)stream) == cudaSuccess
               ? HAWKES_OK
               : HAWKES_ECUDA;
}

size_t hawkes_tree_mass_workspace_size(int64_t m) {
    if (m < 2 || m > HAWKES_TREE_MAX_TIPS) return 0;
    // factor and velocity: 2 (2m - 1) doubles; momentum: w (2m - 1), (sigma^2 V)^-1 w (m), the prior's 5 (2m - 1)
    const size_t nn = (size_t)(2 * m - 1);
    return (nn + (size_t)m + 5 * nn) * sizeof(double);
}

static int tree_mass_args(int64_t m, const int *plan, int64_t nc, const double *cpl, int64_t k, int64_t z0,
                          const double *minv, void *ws, size_t ws_bytes) {
    if (m < 2 || m > HAWKES_TREE_MAX_TIPS || !plan || !minv || !ws) return HAWKES_EINVAL;
    if (z0 < 0 || k < m || z0 > k - m) return HAWKES_EINVAL;
    if (nc < 0 || nc > HAWKES_TREE_MASS_MAX_COUPLED || nc > z0 || (nc > 0 && !cpl)) return HAWKES_EINVAL;
    if (ws_bytes < hawkes_tree_mass_workspace_size(m)) return HAWKES_EWORKSPACE;
    return HAWKES_OK;
}

static bool tree_scalars_ok(double root_var, double sigma2) {
    return sigma2 > 0 && root_var >= 0 && isfinite(sigma2) && isfinite(root_var);
}

int hawkes_tree_mass_factor(int64_t m, const int *plan, const double *length, double root_var, double sigma2,
                            const double *dlik, double *fac, void *ws, size_t ws_bytes, void *stream) {
    if (m < 2 || m > HAWKES_TREE_MAX_TIPS || !plan || !length || !dlik || !fac || !ws) return HAWKES_EINVAL;
    if (!tree_scalars_ok(root_var, sigma2)) return HAWKES_EINVAL;
    if (ws_bytes < hawkes_tree_mass_workspace_size(m)) return HAWKES_EWORKSPACE;
    return hk::launch_tree_mass_factor(m, plan, length, root_var, sigma2, dlik, fac, (double *)ws,
                                       (cudaStream_t)stream) == cudaSuccess
               ? HAWKES_OK
               : HAWKES_ECUDA;
}

int hawkes_tree_mass_velocity(int64_t m, const int *plan, const double *fac, int64_t nc, const double *cpl,
                              int64_t k, int64_t z0, const double *minv, const double *p, double *vel, double *q,
                              double eps, double *kinetic, void *ws, size_t ws_bytes, void *stream) {
    const int rc = tree_mass_args(m, plan, nc, cpl, k, z0, minv, ws, ws_bytes);
    if (rc != HAWKES_OK) return rc;
    if (!fac || !p || (!vel && !q && !kinetic) || !isfinite(eps)) return HAWKES_EINVAL;
    return hk::launch_tree_mass_velocity(m, plan, fac, (int)nc, cpl, k, z0, minv, p, vel, q, eps, kinetic,
                                         (double *)ws, (cudaStream_t)stream) == cudaSuccess
               ? HAWKES_OK
               : HAWKES_ECUDA;
}

int hawkes_tree_mass_momentum(int64_t m, const int *plan, const double *length, double root_var, double sigma2,
                              const double *dlik, int64_t nc, const double *cpl, int64_t k, int64_t z0,
                              const double *minv, const double *xi, double *p, void *ws, size_t ws_bytes,
                              void *stream) {
    const int rc = tree_mass_args(m, plan, nc, cpl, k, z0, minv, ws, ws_bytes);
    if (rc != HAWKES_OK) return rc;
    if (!length || !dlik || !xi || !p || !tree_scalars_ok(root_var, sigma2)) return HAWKES_EINVAL;
    return hk::launch_tree_mass_momentum(m, plan, length, root_var, sigma2, dlik, (int)nc, cpl, k, z0, minv, xi, p,
                                         (double *)ws, (cudaStream_t)stream) == cudaSuccess
               ? HAWKES_OK
               : HAWKES_ECUDA;
}

}  // extern "C"
