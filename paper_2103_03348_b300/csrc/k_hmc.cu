// Posterior assembly and leapfrog kernels for the adaptively preconditioned
// HMC of Section 2.3 (Eqs. 3-5).
//
// Sampler coordinates q = (log mu0, log tau_x, log tau_t, log theta0, log omega,
// log h, r_{s_1}, ..., r_{s_M}): the six globals on the log scale and the
// log-rates of the M sequenced events (theta_s = exp(r_s), Section 2.2).  The
// log posterior (up to a constant) is
//     log pi(q) = l(p, r) + sum_k [log prior_k(p_k) + q_k] - 1/2 r_S^T P r_S
// with p_k = exp(q_k) (the + q_k is the Jacobian of the log transform), priors
// Gamma(shape a, rate b) or inverse-Gamma(shape a, scale b) on each p_k, and
// the phylogenetic Brownian prior r_S ~ N(0, P^-1) (Eq. 2, P = (sigma^2 V)^-1).
// Its gradient and Hessian diagonal in q follow by the chain rule:
//     d/dq_k   = p_k (g_k + g'_k) + 1
//     d2/dq_k2 = p_k (g_k + g'_k) + p_k^2 (H_kk + g''_k)
//     d/dr_s   = dl/dr_s - (P r_S)_s,   d2/dr_s2 = d2l/dr_s2 - P_ss.
#include "hawkes_internal.cuh"

namespace hk {

constexpr int ASM_THREADS = 1024;
constexpr int MV_THREADS = 256;  // 8 warps, one matrix row per warp

// w = P r_S (row-major M x M, FP64): one warp per row, lanes stride the columns.
__global__ void __launch_bounds__(MV_THREADS) prec_matvec_kernel(int64_t m, const double *__restrict__ prec,
                                                                 const double *__restrict__ rs, double *__restrict__ w) {
    pdl_wait();
    const int warp = (blockIdx.x * MV_THREADS + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= m) return;
    const double *row = prec + (size_t)warp * m;
    double s = 0.0;
    for (int64_t j = lane; j < m; j += 32) s += row[j] * rs[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) w[warp] = s;
}

struct PostConsts {
    int kind[6];
    double a[6], b[6];
};

__global__ void __launch_bounds__(ASM_THREADS) posterior_assemble_kernel(
    int64_t m, PostConsts pc, const int *__restrict__ seq, const double *__restrict__ pdiag, int64_t pstride,
    const double *__restrict__ q, const double *__restrict__ w, const double *__restrict__ loglik,
    const double *__restrict__ grad, const double *__restrict__ hdiag, double *__restrict__ logpost,
    double *__restrict__ grad_q, double *__restrict__ hdiag_q) {
    pdl_wait();
    __shared__ double sh[ASM_THREADS];
    __shared__ double s_lp[6];
    __shared__ int s_ok[6];
    const double *rs = q + 6;  // the sequenced log-rates
    double quad = 0.0;
    for (int64_t j = threadIdx.x; j < m; j += ASM_THREADS) {
        const int i = seq[j];
        if (grad_q) grad_q[6 + j] = grad[6 + i] - w[j];
        if (hdiag_q) hdiag_q[6 + j] = hdiag[6 + i] - pdiag[(size_t)j * pstride];
        quad += rs[j] * w[j];
    }
    // one thread per global: its prior, the log-transform Jacobian and the chain rule
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        const double lq = q[k], p = exp(lq), ip = 1.0 / p, a = pc.a[k], b = pc.b[k];
        double lpr, d1, d2;
        if (pc.kind[k] == HAWKES_PRIOR_GAMMA) {
            lpr = (a - 1.0) * lq - b * p;
            d1 = (a - 1.0) * ip - b;
            d2 = -(a - 1.0) * ip * ip;
        } else {  // inverse gamma
            lpr = -(a + 1.0) * lq - b * ip;
            d1 = -(a + 1.0) * ip + b * ip * ip;
            d2 = (a + 1.0) * ip * ip - 2.0 * b * ip * ip * ip;
        }
        s_lp[k] = lpr + lq;  // log p_k = q_k
        s_ok[k] = isfinite(p) && p > 0.0;
        if (grad_q) {
            const double gk = grad[k] + d1;
            grad_q[k] = p * gk + 1.0;
            if (hdiag_q) hdiag_q[k] = p * gk + p * p * (hdiag[k] + d2);
        }
    }
    quad = block_sum<ASM_THREADS>(quad, sh);  // its barriers also publish s_lp, s_ok
    if (threadIdx.x == 0) {
        double lp = *loglik - 0.5 * quad;
        bool ok = true;
        for (int k = 0; k < 6; ++k) {
            lp += s_lp[k];
            ok = ok && s_ok[k];
        }
        *logpost = ok ? lp : -INFINITY;
    }
}

// r[seq[j]] = q[6 + j]: the sampler's log-rates into the likelihood's full vector.
__global__ void scatter_rates_kernel(int64_t m, const int *__restrict__ seq, const double *__restrict__ q,
                                     double *__restrict__ r) {
    pdl_wait();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        r[seq[j]] = q[6 + j];
}

// r[seq[j]] = z_j + sum_c F[j, c] beta_c with z = q[6..6+m), beta = q[6+m..6+m+k):
// the sequenced log-rates with the time trend of Section 2.2.
__global__ void scatter_rates_trend_kernel(int64_t m, int k, const int *__restrict__ seq,
                                           const double *__restrict__ F, const double *__restrict__ q,
                                           double *__restrict__ r) {
    pdl_wait();
    const double *beta = q + 6 + m;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        double v = q[6 + j];
        for (int c = 0; c < k; ++c) v += F[j * k + c] * beta[c];
        r[seq[j]] = v;
    }
}

// The trend coefficients' entries of the posterior, one block per coefficient c:
//   d log pi / d beta_c = sum_j F[j, c] dl/dr_{s_j} - beta_c / beta_var,
//   preconditioner      = sum_j F[j, c]^2 d2l/dr_{s_j}^2 - 1 / beta_var,
// and block 0 adds the N(0, beta_var I) log prior to log pi.
__global__ void __launch_bounds__(ASM_THREADS) trend_assemble_kernel(
    int64_t m, int k, const int *__restrict__ seq, const double *__restrict__ F, double beta_var,
    const double *__restrict__ q, const double *__restrict__ grad, const double *__restrict__ hdiag,
    double *__restrict__ logpost, double *__restrict__ grad_q, double *__restrict__ hdiag_q) {
    pdl_wait();
    __shared__ double sh[ASM_THREADS];
    const int c = blockIdx.x;
    const double *beta = q + 6 + m;
    double g = 0.0, h = 0.0;
    for (int64_t j = threadIdx.x; j < m; j += ASM_THREADS) {
        const double f = F[j * k + c];
        if (grad) g += f * grad[6 + seq[j]];
        if (hdiag) h += f * f * hdiag[6 + seq[j]];
    }
    g = block_sum<ASM_THREADS>(g, sh);
    if (hdiag) h = block_sum<ASM_THREADS>(h, sh);
    if (threadIdx.x == 0) {
        if (grad_q) grad_q[6 + m + c] = g - beta[c] / beta_var;
        if (hdiag_q) hdiag_q[6 + m + c] = h - 1.0 / beta_var;
        if (c == 0) {
            double quad = 0.0;
            for (int i = 0; i < k; ++i) quad += beta[i] * beta[i];
            *logpost -= 0.5 * quad / beta_var;
        }
    }
}

// p += a g
__global__ void momentum_kernel(int64_t k, double *__restrict__ p, const double *__restrict__ g, double a) {
    pdl_wait();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x)
        p[j] += a * g[j];
}

// q += eps minv p
__global__ void position_kernel(int64_t k, double *__restrict__ q, const double *__restrict__ p,
                                const double *__restrict__ minv, double eps) {
    pdl_wait();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x)
        q[j] += eps * minv[j] * p[j];
}

// One leapfrog step's state updates in one launch (diagonal mass): the
// momentum update p += a g that ends the previous step (or the first half
// step), the position update q += eps minv p, and the scatter of the new
// sequenced log-rates r[seq[j]] = q[6 + j] for the next evaluation.  Each
// entry is one thread's: the same expressions as momentum_kernel,
// position_kernel and scatter_rates_kernel in sequence, so the results are
// those of the three launches bit for bit.
__global__ void leapfrog_step_kernel(int64_t k, double *__restrict__ q, double *__restrict__ p,
                                     const double *__restrict__ g, double a, const double *__restrict__ minv,
                                     double eps, int64_t m, const int *__restrict__ seq, double *__restrict__ r) {
    pdl_wait();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
        if (g) p[j] += a * g[j];
        q[j] += eps * minv[j] * p[j];
        if (j >= 6 && j - 6 < m) r[seq[j - 6]] = q[j];
    }
}

// out = 1/2 sum_j minv_j p_j^2 (single block, fixed order)
__global__ void __launch_bounds__(ASM_THREADS) kinetic_kernel(int64_t k, const double *__restrict__ p,
                                                              const double *__restrict__ minv, double *__restrict__ out) {
    pdl_wait();
    __shared__ double sh[ASM_THREADS];
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < k; j += ASM_THREADS) s += minv[j] * p[j] * p[j];
    s = block_sum<ASM_THREADS>(s, sh);
    if (threadIdx.x == 0) *out = 0.5 * s;
}

// Dense mass matrix over k <= DENSE_MAX coordinates (a posterior over the six
// globals alone): minv is M^-1, k x k row-major.
//   position: q += eps M^-1 p        kinetic: out = 1/2 p^T M^-1 p
// One block; (M^-1 p)_j summed over i in order.
constexpr int DENSE_MAX = 64;

__global__ void __launch_bounds__(DENSE_MAX) position_dense_kernel(int k, double *__restrict__ q,
                                                                   const double *__restrict__ p,
                                                                   const double *__restrict__ minv, double eps) {
    pdl_wait();
    __shared__ double ps[DENSE_MAX];
    const int j = threadIdx.x;
    if (j < k) ps[j] = p[j];
    __syncthreads();
    if (j < k) {
        double v = 0.0;
        for (int i = 0; i < k; ++i) v += minv[j * k + i] * ps[i];
        q[j] += eps * v;
    }
}

__global__ void __launch_bounds__(DENSE_MAX) kinetic_dense_kernel(int k, const double *__restrict__ p,
                                                                  const double *__restrict__ minv,
                                                                  double *__restrict__ out) {
    pdl_wait();
    __shared__ double ps[DENSE_MAX], term[DENSE_MAX];
    const int j = threadIdx.x;
    if (j < k) ps[j] = p[j];
    __syncthreads();
    if (j < k) {
        double v = 0.0;
        for (int i = 0; i < k; ++i) v += minv[j * k + i] * ps[i];
        term[j] = ps[j] * v;
    }
    __syncthreads();
    if (j == 0) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += term[i];
        *out = 0.5 * s;
    }
}

// Metropolis accept/reject closing one trajectory (Section 2.3): with the energy
// H = -log pi(q) + K(p), the proposal is taken with probability
// a = min(1, exp(H0 - H1)), and with probability 0 when its log posterior or
// energy is not finite or its likelihood evaluation reported an error.  The
// uniform draw u decides (accepted iff u < a).  One block: thread 0 takes the
// decision, every thread copies its share of the state; the record slot gets
// the kept coordinates of the resulting state, its log posterior, a and the
// decision.
constexpr int ACCEPT_THREADS = 256;

__global__ void __launch_bounds__(ACCEPT_THREADS) accept_kernel(
    int64_t k, const double *__restrict__ u, const double *__restrict__ k0, const double *__restrict__ k1,
    const double *__restrict__ lp1, const double *__restrict__ grad1, const double *__restrict__ q1,
    const int *__restrict__ status, double *__restrict__ q, double *__restrict__ lp, double *__restrict__ grad,
    int64_t n_keep, const int64_t *__restrict__ keep, double *__restrict__ rec_q, double *__restrict__ rec) {
    pdl_wait();
    __shared__ int s_acc;
    __shared__ double s_lp;
    if (threadIdx.x == 0) {
        const double h0 = -lp[0] + k0[0];
        const double l1 = lp1[0], h1 = -l1 + k1[0];
        const bool ok = (status == nullptr || status[0] == 0) && isfinite(l1) && isfinite(h1);
        const double a = ok ? fmin(1.0, exp(fmin(0.0, h0 - h1))) : 0.0;
        const bool acc = u[0] < a;
        s_acc = acc ? 1 : 0;
        s_lp = acc ? l1 : lp[0];
        if (rec) { rec[0] = s_lp; rec[1] = a; rec[2] = acc ? 1.0 : 0.0; }
    }
    __syncthreads();
    const bool acc = s_acc != 0;
    // the record reads the proposal when accepted and the unchanged state when not,
    // so it never reads an entry that this launch writes
    if (rec_q) {
        for (int64_t i = threadIdx.x; i < n_keep; i += ACCEPT_THREADS) {
            const int64_t j = keep[i];
            rec_q[i] = (j >= 0 && j < k) ? (acc ? q1[j] : q[j]) : nan("");
        }
    }
    if (acc) {
        for (int64_t j = threadIdx.x; j < k; j += ACCEPT_THREADS) {
            q[j] = q1[j];
            grad[j] = grad1[j];
        }
        if (threadIdx.x == 0) lp[0] = s_lp;
    }
}

static int grid_for(int64_t k) {
    int64_t b = (k + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace hk

extern "C" {

size_t hawkes_posterior_workspace_size(int64_t m) { return m < 0 ? 0 : (size_t)(m > 0 ? m : 1) * sizeof(double); }

static int post_check(int64_t n, int64_t m, const hawkes_prior *prior, const double *q, const double *loglik,
                      const double *grad, const double *hdiag, const double *logpost, const double *grad_q,
                      const double *hdiag_q, hk::PostConsts *pc) {
    if (n < 2 || m < 0 || m > n || !prior || !q || !loglik || !logpost) return HAWKES_EINVAL;
    if ((grad == nullptr) != (grad_q == nullptr)) return HAWKES_EINVAL;
    if ((hdiag == nullptr) != (hdiag_q == nullptr)) return HAWKES_EINVAL;
    if (hdiag && !grad) return HAWKES_EINVAL;
    for (int k = 0; k < 6; ++k) {
        if (prior->kind[k] != HAWKES_PRIOR_GAMMA && prior->kind[k] != HAWKES_PRIOR_INVGAMMA) return HAWKES_EINVAL;
        if (!(prior->a[k] > 0) || !(prior->b[k] >= 0)) return HAWKES_EINVAL;
        pc->kind[k] = prior->kind[k];
        pc->a[k] = prior->a[k];
        pc->b[k] = prior->b[k];
    }
    return HAWKES_OK;
}

int hawkes_posterior(int64_t n, int64_t m, const int *seq_idx, const double *prec, const hawkes_prior *prior,
                     const double *q, const double *loglik, const double *grad, const double *hdiag, void *ws,
                     size_t ws_bytes, double *logpost, double *grad_q, double *hdiag_q, void *stream) {
    hk::PostConsts pc;
    const int rc = post_check(n, m, prior, q, loglik, grad, hdiag, logpost, grad_q, hdiag_q, &pc);
    if (rc != HAWKES_OK) return rc;
    if (!ws) return HAWKES_EINVAL;
    if (m > 0 && (!seq_idx || !prec)) return HAWKES_EINVAL;
    if (ws_bytes < hawkes_posterior_workspace_size(m)) return HAWKES_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    double *w = (double *)ws;
    const double *rs = q + 6;
    if (m > 0) {
        const int blocks = (int)((m * 32 + hk::MV_THREADS - 1) / hk::MV_THREADS);
        launch_pdl(hk::prec_matvec_kernel, blocks, hk::MV_THREADS, 0, s, m, prec, rs, w);
        if (cudaGetLastError() != cudaSuccess) return HAWKES_ECUDA;
    }
    launch_pdl(hk::posterior_assemble_kernel, 1, hk::ASM_THREADS, 0, s, m, pc, seq_idx, prec, m + 1, q, w, loglik, grad,
                                                                hdiag, logpost, grad_q, hdiag_q);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

size_t hawkes_posterior_tree_workspace_size(int64_t m) {
    if (m < 2 || m > HAWKES_TREE_MAX_TIPS) return 0;
    return (size_t)2 * m * sizeof(double) + hawkes_tree_workspace_size(m);
}

int hawkes_posterior_tree(int64_t n, int64_t m, const int *seq_idx, const int *plan, const double *length,
                          double root_var, double sigma2, const hawkes_prior *prior, const double *q,
                          const double *loglik, const double *grad, const double *hdiag, void *ws, size_t ws_bytes,
                          double *logpost, double *grad_q, double *hdiag_q, void *stream) {
    hk::PostConsts pc;
    const int rc = post_check(n, m, prior, q, loglik, grad, hdiag, logpost, grad_q, hdiag_q, &pc);
    if (rc != HAWKES_OK) return rc;
    if (!ws) return HAWKES_EINVAL;
    if (m < 2 || m > HAWKES_TREE_MAX_TIPS || !seq_idx || !plan || !length) return HAWKES_EINVAL;
    if (!(sigma2 > 0) || !(root_var >= 0) || !isfinite(sigma2) || !isfinite(root_var)) return HAWKES_EINVAL;
    if (ws_bytes < hawkes_posterior_tree_workspace_size(m)) return HAWKES_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    double *w = (double *)ws, *pd = w + m, *scratch = pd + m;
    if (hk::launch_tree_prior(m, plan, length, root_var, sigma2, q + 6, scratch, nullptr, w, hdiag ? pd : nullptr,
                              s) != cudaSuccess)
        return HAWKES_ECUDA;
    launch_pdl(hk::posterior_assemble_kernel, 1, hk::ASM_THREADS, 0, s, m, pc, seq_idx, pd, 1, q, w, loglik, grad, hdiag,
                                                                logpost, grad_q, hdiag_q);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_posterior_assemble(int64_t n, int64_t m, const int *seq_idx, const double *pz, const double *pdiag,
                               const hawkes_prior *prior, const double *q, const double *loglik, const double *grad,
                               const double *hdiag, double *logpost, double *grad_q, double *hdiag_q, void *stream) {
    hk::PostConsts pc;
    const int rc = post_check(n, m, prior, q, loglik, grad, hdiag, logpost, grad_q, hdiag_q, &pc);
    if (rc != HAWKES_OK) return rc;
    if (m > 0 && (!seq_idx || !pz || (hdiag && !pdiag))) return HAWKES_EINVAL;
    launch_pdl(hk::posterior_assemble_kernel, 1, hk::ASM_THREADS, 0, (cudaStream_t)stream,
        m, pc, seq_idx, pdiag, 1, q, pz, loglik, grad, hdiag, logpost, grad_q, hdiag_q);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_hmc_scatter_rates_trend(int64_t m, int k, const int *seq_idx, const double *F, const double *q, double *r,
                                   void *stream) {
    if (m < 0 || k < 0 || (m > 0 && (!seq_idx || !q || !r)) || (m > 0 && k > 0 && !F)) return HAWKES_EINVAL;
    if (m == 0) return HAWKES_OK;
    launch_pdl(hk::scatter_rates_trend_kernel, hk::grid_for(m), 256, 0, (cudaStream_t)stream, m, k, seq_idx, F, q, r);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_posterior_add_trend(int64_t m, int k, const int *seq_idx, const double *F, double beta_var,
                               const double *q, const double *grad, const double *hdiag, double *logpost,
                               double *grad_q, double *hdiag_q, void *stream) {
    if (m < 1 || k < 0 || !seq_idx || !q || !logpost || (k > 0 && !F)) return HAWKES_EINVAL;
    if (!(beta_var > 0) || !isfinite(beta_var)) return HAWKES_EINVAL;
    if ((grad == nullptr) != (grad_q == nullptr) || (hdiag == nullptr) != (hdiag_q == nullptr)) return HAWKES_EINVAL;
    if (hdiag && !grad) return HAWKES_EINVAL;
    if (k == 0) return HAWKES_OK;
    launch_pdl(hk::trend_assemble_kernel, k, hk::ASM_THREADS, 0, (cudaStream_t)stream, m, k, seq_idx, F, beta_var, q, grad,
                                                                               hdiag, logpost, grad_q, hdiag_q);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_hmc_scatter_rates(int64_t m, const int *seq_idx, const double *q, double *r, void *stream) {
    if (m < 0 || (m > 0 && (!seq_idx || !q || !r))) return HAWKES_EINVAL;
    if (m == 0) return HAWKES_OK;
    launch_pdl(hk::scatter_rates_kernel, hk::grid_for(m), 256, 0, (cudaStream_t)stream, m, seq_idx, q, r);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_hmc_momentum(int64_t k, double *p, const double *g, double a, void *stream) {
    if (k < 1 || !p || !g) return HAWKES_EINVAL;
    launch_pdl(hk::momentum_kernel, hk::grid_for(k), 256, 0, (cudaStream_t)stream, k, p, g, a);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_hmc_position(int64_t k, double *q, const double *p, const double *minv, double eps, void *stream) {
    if (k < 1 || !q || !p || !minv) return HAWKES_EINVAL;
    launch_pdl(hk::position_kernel, hk::grid_for(k), 256, 0, (cudaStream_t)stream, k, q, p, minv, eps);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_hmc_leapfrog_step(int64_t k, double *q, double *p, const double *g, double a, const double *minv,
                             double eps, int64_t m, const int *seq_idx, double *r, void *stream) {
    if (k < 1 || !q || !p || !minv || m < 0 || m > k - 6) return HAWKES_EINVAL;
    if (m > 0 && (!seq_idx || !r)) return HAWKES_EINVAL;
    launch_pdl(hk::leapfrog_step_kernel, hk::grid_for(k), 256, 0, (cudaStream_t)stream, k, q, p, g, a, minv, eps, m,
               seq_idx, r);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_hmc_kinetic(int64_t k, const double *p, const double *minv, double *out, void *stream) {
    if (k < 1 || !p || !minv || !out) return HAWKES_EINVAL;
    launch_pdl(hk::kinetic_kernel, 1, hk::ASM_THREADS, 0, (cudaStream_t)stream, k, p, minv, out);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_hmc_accept(int64_t k, const double *u, const double *k0, const double *k1, const double *lp1,
                      const double *grad1, const double *q1, const int *status, double *q, double *lp, double *grad,
                      int64_t n_keep, const int64_t *keep, double *rec_q, double *rec, void *stream) {
    if (k < 1 || !u || !k0 || !k1 || !lp1 || !grad1 || !q1 || !q || !lp || !grad) return HAWKES_EINVAL;
    if (n_keep < 0 || (n_keep > 0 && rec_q && !keep)) return HAWKES_EINVAL;
    if (q1 == q || grad1 == grad) return HAWKES_EINVAL;  // the proposal must not alias the state
    launch_pdl(hk::accept_kernel, 1, hk::ACCEPT_THREADS, 0, (cudaStream_t)stream, k, u, k0, k1, lp1, grad1, q1, status,
               q, lp, grad, rec_q ? n_keep : (int64_t)0, keep, rec_q, rec);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_hmc_position_dense(int64_t k, double *q, const double *p, const double *minv, double eps, void *stream) {
    if (k < 1 || k > hk::DENSE_MAX || !q || !p || !minv) return HAWKES_EINVAL;
    launch_pdl(hk::position_dense_kernel, 1, hk::DENSE_MAX, 0, (cudaStream_t)stream, (int)k, q, p, minv, eps);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_hmc_kinetic_dense(int64_t k, const double *p, const double *minv, double *out, void *stream) {
    if (k < 1 || k > hk::DENSE_MAX || !p || !minv || !out) return HAWKES_EINVAL;
    launch_pdl(hk::kinetic_dense_kernel, 1, hk::DENSE_MAX, 0, (cudaStream_t)stream, (int)k, p, minv, out);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

}  // extern "C"
