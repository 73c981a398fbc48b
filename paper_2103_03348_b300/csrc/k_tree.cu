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

}  // extern "C"
