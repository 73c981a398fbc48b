/*
 * hawkes.h -- C ABI of libhawkes.so: the O(N^2) log-likelihood of the
 * spatiotemporal Hawkes process with per-event rates, its gradient and its
 * Hessian diagonal, on one B300 GPU (sm_103a).
 *
 * Model (Holbrook, Ji & Suchard, arXiv 2103.03348, Section 2.1, Eq. 1):
 *
 *   lambda_n = mu0 * sum_{n'} I[x_n != x_n'] (2 pi tau_x^2)^-1 exp(-|x_n-x_n'|^2 / (2 tau_x^2))
 *                                            (2 pi tau_t^2)^-1/2 exp(-(t_n-t_n')^2 / (2 tau_t^2))
 *            + theta0 omega (2 pi h^2)^-1 sum_{t_n' < t_n} exp(r_n') exp(-omega (t_n-t_n'))
 *                                            exp(-|x_n-x_n'|^2 / (2 h^2))
 *   Lambda   = mu0 sum_n' [Phi((t_N - t_n')/tau_t) - Phi(-t_n'/tau_t)]
 *            + theta0 sum_n' exp(r_n') (1 - exp(-omega (t_N - t_n')))        (Appendix A Claim)
 *   loglik   = sum_n log lambda_n - Lambda                                    (Eq. 1)
 *
 * r_n = log theta_n is the per-event log-rate (Section 2.2: theta_n =
 * exp(z_n + beta^T f(t_n)) for sequenced events, 1 otherwise; the caller forms
 * r_n and applies the chain rule to z and beta).  The paper's background has
 * no temporal factor; tau_t = +INFINITY selects exactly that model (the
 * temporal Gaussian is dropped and Lambda's background part is mu0 * N * t_N).
 * A finite tau_t gives the background a normalised temporal Gaussian too.
 * t_N is the last (largest) event time and integration starts at time 0.
 * Excitation is strict (t_n' < t_n): simultaneous events do not excite each
 * other.  The background indicator drops sources at exactly the target's
 * location (the event itself and exact duplicates, compared in FP64).
 *
 * Common arguments of the three evaluation calls
 *   x, y, t, r   DEVICE pointers to n doubles each (locations, times, log-rates),
 *                in time-ascending order (ties allowed).  Read only.
 *   n            number of events, 2 <= n <= HAWKES_MAX_EVENTS.
 *   params       HOST pointer to 6 doubles (mu0, tau_x, tau_t, theta0, omega, h),
 *                all finite and > 0, except tau_t which may be +INFINITY.
 *   precision    HAWKES_FP64: every pair in FP64 (libm-accurate exp).
 *                HAWKES_FP32C: pair terms in FP32 (ex2.approx), each row
 *                accumulated with compensated (two-level Kahan) FP32, rows
 *                finished, reduced and logged in FP64; rows whose FP32 sum is
 *                below 2^-60 are recomputed in FP64.
 *                HAWKES_FP32C_BAND: FP32C that also skips the tile pairs whose
 *                background terms all lie below 2^-130 because their time gap
 *                exceeds the background's temporal Gaussian (Section 2.1 with a
 *                finite tau_t).  Those terms are exactly 0 in FP32, so the results
 *                equal HAWKES_FP32C's bit for bit; only the work is smaller.
 *                HAWKES_FP32C_ST: FP32C on space-time tiles.  Inside each slab
 *                of 4096 time-consecutive events the events are regrouped by
 *                the Hilbert index of their location, so each group of 32
 *                events is compact in space and time; the pairs of groups
 *                whose terms all lie below 2^-126 (background: spatial and
 *                temporal gap; excitation and column pass: spatial gap,
 *                largest log-rate and time offset) are skipped, as their FP32
 *                terms are exactly 0.  The sums run in another order than
 *                HAWKES_FP32C's, so the results agree with it to rounding
 *                (the FP32C accuracy bars hold).  The workspace is larger and
 *                the shard entry points refuse this precision.
 *   ws, ws_bytes DEVICE workspace owned by the caller, at least
 *                hawkes_workspace_size(n, precision) bytes, 256-byte aligned.
 *                The library allocates nothing.  Calls that may overlap on the
 *                GPU need distinct workspaces.
 *   dev_status   DEVICE pointer to one int; receives a hawkes_status for the
 *                data-dependent checks (HAWKES_OK, HAWKES_EUNSORTED,
 *                HAWKES_ENONFINITE, HAWKES_EZERO_INTENSITY).
 *   stream       cudaStream_t (as void*), may be NULL for the legacy stream.
 *                Everything is enqueued on it; no call synchronises the host.
 *
 * Outputs are DEVICE pointers owned by the caller.  Gradient and Hessian
 * vectors hold 6 + n doubles: [0..5] w.r.t. (mu0, tau_x, tau_t, theta0,
 * omega, h) as given (not log-transformed), [6 + m] w.r.t. r_m in input order.
 * With tau_t = +INFINITY the tau_t entries are 0.
 *
 * Errors: the return value reports argument errors synchronously (no GPU work
 * is enqueued then) and launch failures (HAWKES_ECUDA).  Data-dependent
 * conditions are written to *dev_status by the GPU: for unsorted or
 * non-finite inputs every output is NaN; when some lambda_n == 0 even in FP64
 * the log-likelihood is -INFINITY and the gradient and Hessian are NaN.
 *
 * The library keeps no state between calls: every call is independent.
 */
#ifndef HAWKES_H
#define HAWKES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { HAWKES_FP64 = 0, HAWKES_FP32C = 1, HAWKES_FP32C_BAND = 2, HAWKES_FP32C_ST = 3 } hawkes_precision;

typedef enum {
    HAWKES_OK = 0,
    HAWKES_EINVAL = 1,          /* bad argument: n, null pointer, params, precision, alignment */
    HAWKES_EUNSORTED = 2,       /* t not ascending (device status) */
    HAWKES_ENONFINITE = 3,      /* NaN/Inf in x, y, t or r (device status) */
    HAWKES_EWORKSPACE = 4,      /* ws_bytes < hawkes_workspace_size(n, precision) */
    HAWKES_ECUDA = 5,           /* a CUDA launch or memset failed */
    HAWKES_EZERO_INTENSITY = 6, /* some lambda_n == 0 (device status) */
    HAWKES_ESCRATCH = 7         /* n above HAWKES_NOALLOC_MAX_EVENTS (hawkes_hess_diag_noalloc) */
} hawkes_status;

/* Largest supported n (indices are 32-bit inside the kernels). */
#define HAWKES_MAX_EVENTS (1 << 28)

/* Bytes of device workspace that any of the three calls needs for n events at
 * this precision (the same size serves all three).  0 for invalid n or
 * precision. */
size_t hawkes_workspace_size(int64_t n, int precision);

/* Eq. 1 only: writes *loglik (DEVICE, 1 double).  Row pass (Algorithm 2, step 1)
 * plus the integral term (Appendix A). */
int hawkes_loglik(const double *x, const double *y, const double *t, const double *r, int64_t n,
                  const double params[6], int precision, void *ws, size_t ws_bytes,
                  double *loglik, int *dev_status, void *stream);

/* Eq. 1 and its gradient: grad (DEVICE, 6 + n doubles, required); loglik may be
 * NULL.  The log-rate entries are Eq. 4 multiplied by theta_m (Algorithm 2,
 * step 2); the global entries differentiate Eq. 1 directly. */
int hawkes_grad(const double *x, const double *y, const double *t, const double *r, int64_t n,
                const double params[6], int precision, void *ws, size_t ws_bytes,
                double *loglik, double *grad, int *dev_status, void *stream);

/* Eq. 1, its gradient and the diagonal of its Hessian: hdiag (DEVICE, 6 + n
 * doubles, required); loglik and grad may be NULL.  The log-rate entries are
 * Eq. 5 in log-rate coordinates: d2l/dr_m^2 = dl/dr_m - sum_n (theta_m dlambda_n/dtheta_m / lambda_n)^2.
 * Every pair is visited once by the row pass and once more, within the
 * causal band, by the column pass. */
int hawkes_hess_diag(const double *x, const double *y, const double *t, const double *r, int64_t n,
                     const double params[6], int precision, void *ws, size_t ws_bytes,
                     double *loglik, double *grad, double *hdiag, int *dev_status, void *stream);

/* Mode of hawkes_eval_device_params.  The GLOBALS modes compute the loglik
 * and the six global entries of the gradient (and Hessian diagonal) only,
 * skipping the column pass: entries [6..6+n) of grad/hdiag are left as they
 * were.  They serve callers that keep the log-rates fixed. */
enum { HAWKES_MODE_LOGLIK = 0, HAWKES_MODE_GRAD = 1, HAWKES_MODE_HESS = 2,
       HAWKES_MODE_GRAD_GLOBALS = 3, HAWKES_MODE_HESS_GLOBALS = 4 };

/* Flag OR-ed into the mode of hawkes_eval_device_params: x, y, t, n and the
 * precision are those of an earlier call on this same workspace (whose
 * contents the caller has left alone), so their validation, tie groups,
 * location groups and tile bounds are reused instead of recomputed; only r
 * and the parameters may differ.  Results are identical to a call without
 * the flag.  A sampler over fixed events sets it after its first call. */
#define HAWKES_MODE_REUSE_EVENTS 16

/* The three evaluations with the parameter vector in DEVICE memory, so that a
 * caller whose parameters are produced on the GPU (a sampler's state) needs no
 * host round trip between evaluations.  params_dev: DEVICE double[6] in the
 * usual order; with log_params != 0 it holds their logarithms (the first six
 * sampler coordinates).  mode selects loglik / + grad / + hdiag exactly as
 * hawkes_loglik / hawkes_grad / hawkes_hess_diag (loglik is required for
 * mode 0, grad for modes 1 and 3, hdiag for modes 2 and 4).  Parameters that are not finite
 * and positive are found on the GPU: *dev_status = HAWKES_EINVAL and every
 * output is NaN. */
int hawkes_eval_device_params(const double *x, const double *y, const double *t, const double *r, int64_t n,
                              const double *params_dev, int log_params, int precision, int mode, void *ws,
                              size_t ws_bytes, double *loglik, double *grad, double *hdiag, int *dev_status,
                              void *stream);

/* hawkes_eval_device_params for modes HAWKES_MODE_GRAD / HAWKES_MODE_HESS (the
 * HAWKES_MODE_REUSE_EVENTS flag allowed) with the rate entries wanted only for
 * the sources rate_idx[0..k_rates) (DEVICE int, distinct, any order, each in
 * [0, n); sorted indices make the FP32C pass cheapest):
 * the column pass then costs O(n k) instead of O(n^2) in FP32C (FP64 covers
 * every source and writes the subset).  Entries 6 + rate_idx[j] of grad and
 * hdiag are written; the other rate entries are left as they were; loglik and
 * entries [0, 6) as usual.  An index outside [0, n) is skipped and gives
 * *dev_status = HAWKES_EINVAL (the outputs are then not valid).  Returns
 * HAWKES_EINVAL for k_rates < 0 or > n, a NULL rate_idx with k_rates > 0, or
 * another mode.  The paper's samplers move the rates of the M
 * sequenced events only (Section 2.3.2), which this serves. */
int hawkes_eval_rates_subset(const double *x, const double *y, const double *t, const double *r, int64_t n,
                             const double *params_dev, int log_params, int precision, int mode, const int *rate_idx,
                             int64_t k_rates, void *ws, size_t ws_bytes, double *loglik, double *grad, double *hdiag,
                             int *dev_status, void *stream);

/* hawkes_hess_diag with phase markers, for profiling.  phase_events holds four
 * cudaEvent_t handles (as void*, created by the caller; any may be NULL) that
 * are recorded on the stream: [0] before and [1] after the row pass (the
 * dominant O(N^2) kernel), [2] before and [3] after the column pass.  The
 * results are identical to hawkes_hess_diag. */
int hawkes_hess_diag_timed(const double *x, const double *y, const double *t, const double *r, int64_t n,
                           const double params[6], int precision, void *ws, size_t ws_bytes,
                           double *loglik, double *grad, double *hdiag, int *dev_status, void *stream,
                           void *const phase_events[4]);

/* ------------------------------------------------------------------------
 * Sharded evaluation: the double sum split over k shards (ranks), each with
 * its own workspace and a copy of the events.  Shard s owns the tiles of 128
 * events [s*T/k, (s+1)*T/k) (T = ceil(n/128)) as targets of the row pass
 * (Eq. 1 inner sums) and as sources of the column pass (Eqs. 4-5).  One
 * exchange sits between the two phases: each shard's row phase writes its
 * tiles' records (partial sums of the log-likelihood terms and the column
 * weights B / lambda_n) into its slice of the exchange buffer; the caller
 * all-gathers the slices so that every shard's buffer holds all records (an
 * NCCL all-gather across GPUs, or copies between buffers on one GPU); then each
 * shard's column phase reduces all records in a fixed order and runs its
 * columns.  Every shard's loglik and global entries [0..6) are identical, the
 * per-event entries [6+first, 6+end) are written by the shard that owns them,
 * and the union equals hawkes_hess_diag (or _grad / _loglik) bit for bit.
 * The paper evaluates on one device and has no counterpart.
 * ------------------------------------------------------------------------ */

/* Bytes of the exchange buffer (the same for every shard): T records of
 * (16 + 128) doubles. */
size_t hawkes_shard_exchange_size(int64_t n);

/* Events [*first_event, *end_event) owned by shard `shard` of n_shards, and
 * the byte slice [*xbuf_offset, *xbuf_offset + *xbuf_bytes) of the exchange
 * buffer that its row phase writes (any output may be NULL).  A shard may own
 * no events when n_shards exceeds T. */
int hawkes_shard_range(int64_t n, int shard, int n_shards, int64_t *first_event, int64_t *end_event,
                       size_t *xbuf_offset, size_t *xbuf_bytes);

/* Phase 1 of shard `shard`: validation and packing of all n events, the row
 * pass over the shard's target tiles, and its records into xbuf (DEVICE,
 * 16-byte aligned, hawkes_shard_exchange_size(n) bytes; only the shard's
 * slice is written).  Inputs, params, precision and ws as for
 * hawkes_hess_diag; mode is a HAWKES_MODE_* value (device-resident parameters
 * are not offered here).  The shard's workspace must be passed unchanged to
 * phase 2. */
int hawkes_shard_rows(const double *x, const double *y, const double *t, const double *r, int64_t n,
                      const double params[6], int precision, int mode, int shard, int n_shards, void *ws,
                      size_t ws_bytes, void *xbuf, size_t xbuf_bytes, int *dev_status, void *stream);

/* Phase 2 of shard `shard`, once xbuf holds every shard's records: loglik
 * and the global entries of grad / hdiag (all shards write the same values),
 * then the column pass for the shard's source events (entries 6 + [first,
 * end)).  Same arguments as phase 1 plus the outputs; *dev_status reports the
 * data-dependent conditions of all shards. */
int hawkes_shard_cols(const double *x, const double *y, const double *t, const double *r, int64_t n,
                      const double params[6], int precision, int mode, int shard, int n_shards, void *ws,
                      size_t ws_bytes, const void *xbuf, size_t xbuf_bytes, double *loglik, double *grad,
                      double *hdiag, int *dev_status, void *stream);

/* ------------------------------------------------------------------------
 * Adaptively preconditioned HMC (Section 2.3): posterior assembly and leapfrog
 * pieces.  Sampler coordinates q = (log mu0, log tau_x, log tau_t, log theta0,
 * log omega, log h, r_{s_1}, ..., r_{s_M}) with s_j the sequenced events.
 * ------------------------------------------------------------------------ */

/* Prior on each raw global parameter p_k (Section 3.2 uses gamma priors on mu0
 * and theta0 and inverse-gamma priors on the bandwidths and 1/omega; an
 * inverse-gamma prior on 1/omega is a gamma prior on omega). */
enum { HAWKES_PRIOR_GAMMA = 0,      /* density prop. to p^(a-1) exp(-b p): shape a, rate b */
       HAWKES_PRIOR_INVGAMMA = 1 }; /* density prop. to p^(-a-1) exp(-b / p): shape a, scale b */
typedef struct {
    int kind[6];
    double a[6], b[6];
} hawkes_prior;

/* Bytes of DEVICE workspace hawkes_posterior needs for M sequenced events. */
size_t hawkes_posterior_workspace_size(int64_t m);

/* Log posterior (Eq. 3, up to a constant) in sampler coordinates, its gradient
 * and optionally its Hessian diagonal, from a likelihood evaluation at the same
 * point:
 *   log pi(q) = loglik + sum_k [log prior_k(p_k) + log p_k] - 1/2 r_S^T P r_S,
 * where P = (sigma^2 V)^-1 is the precision of the phylogenetic Brownian prior
 * on the sequenced log-rates (Eq. 2).
 *   n, m        events and sequenced events (0 <= m <= n)
 *   seq_idx     DEVICE int[m]: event index of each sequenced event
 *   prec        DEVICE double[m*m], row-major P (read only)
 *   prior       HOST priors on the six globals
 *   q           DEVICE double[6+m]: the sampler state; p = exp(q[0..5])
 *   loglik, grad, hdiag   DEVICE outputs of the likelihood evaluation at
 *               (p, r with r[seq_idx[j]] = q[6+j]); hdiag may be NULL
 * A q whose p is not finite and positive gives log pi = -inf.
 *   ws          DEVICE workspace of hawkes_posterior_workspace_size(m) bytes
 *   logpost     DEVICE double[1]; grad_q, hdiag_q DEVICE double[6+m]
 *               (grad_q NULL exactly when grad is NULL: then only log pi is
 *               computed; hdiag_q NULL exactly when hdiag is NULL)
 * Enqueued on stream; returns HAWKES_EINVAL for bad arguments. */
int hawkes_posterior(int64_t n, int64_t m, const int *seq_idx, const double *prec,
                     const hawkes_prior *prior, const double *q, const double *loglik, const double *grad,
                     const double *hdiag, void *ws, size_t ws_bytes, double *logpost, double *grad_q,
                     double *hdiag_q, void *stream);

/* The assembly of hawkes_posterior_tree from a prior evaluated separately:
 * pz = (sigma^2 V)^-1 z and pdiag = its diagonal (DEVICE double[m], from
 * hawkes_tree_prior on z = q[6..6+m)), so that the prior can run on another
 * stream while the likelihood is evaluated.  pdiag may be NULL when hdiag is.
 * Other arguments and results as hawkes_posterior. */
int hawkes_posterior_assemble(int64_t n, int64_t m, const int *seq_idx, const double *pz, const double *pdiag,
                              const hawkes_prior *prior, const double *q, const double *loglik, const double *grad,
                              const double *hdiag, double *logpost, double *grad_q, double *hdiag_q, void *stream);

/* r[seq_idx[j]] = q[6 + j] for j < m (DEVICE vectors): the sampler's log-rates
 * into the likelihood's full log-rate vector. */
int hawkes_hmc_scatter_rates(int64_t m, const int *seq_idx, const double *q, double *r, void *stream);

/* The time trend of Section 2.2, theta_s = exp(z_s + beta^T f(t_s)): the
 * sampler state grows to q = (6 log globals, z[m], beta[k]) and the sequenced
 * log-rates are r[seq_idx[j]] = z_j + sum_c F[j*k + c] beta_c, with F the
 * DEVICE m x k matrix (row-major) of the fixed trend features f(t_s).
 * hawkes_hmc_scatter_rates_trend writes those r (k = 0 is the plain scatter). */
int hawkes_hmc_scatter_rates_trend(int64_t m, int k, const int *seq_idx, const double *F, const double *q,
                                   double *r, void *stream);

/* After hawkes_posterior or hawkes_posterior_tree on the same q (whose first
 * 6 + m entries they handle, with z as the phylogenetic variable), adds the
 * trend's part: log pi -= |beta|^2 / (2 beta_var) (prior beta ~ N(0, beta_var I)),
 * grad_q[6+m+c] = sum_j F[j, c] dl/dr_{s_j} - beta_c / beta_var, and
 * hdiag_q[6+m+c] = sum_j F[j, c]^2 d2l/dr_{s_j}^2 - 1 / beta_var.  The last is
 * a preconditioner entry, not the exact second derivative: the cross terms
 * d2l/dr_i dr_j (i != j) are not formed by the evaluation.  grad, hdiag are
 * the likelihood's DEVICE outputs at r (NULL exactly when grad_q / hdiag_q
 * are); logpost is updated in place.  Enqueued on stream; m >= 1, beta_var > 0. */
int hawkes_posterior_add_trend(int64_t m, int k, const int *seq_idx, const double *F, double beta_var,
                               const double *q, const double *grad, const double *hdiag, double *logpost,
                               double *grad_q, double *hdiag_q, void *stream);

/* Leapfrog pieces on DEVICE vectors of length k (Section 2.3.2, Hamilton's
 * equations with a diagonal mass matrix M, minv = 1/diag(M)):
 *   hawkes_hmc_momentum: p += a * g      (half or full momentum step, a = eps/2 or eps)
 *   hawkes_hmc_position: q += eps * minv * p
 *   hawkes_hmc_kinetic:  *out = 1/2 sum minv p^2 */
int hawkes_hmc_momentum(int64_t k, double *p, const double *g, double a, void *stream);
int hawkes_hmc_position(int64_t k, double *q, const double *p, const double *minv, double eps, void *stream);
int hawkes_hmc_kinetic(int64_t k, const double *p, const double *minv, double *out, void *stream);
/* One leapfrog step's state updates in one launch (Section 2.3.2's leapfrog
 * with a diagonal mass), on DEVICE vectors:
 *   p += a * g             (the previous step's momentum update, or the first
 *                           half step; skipped when g is NULL)
 *   q += eps * minv * p    (the position update)
 *   r[seq_idx[j]] = q[6 + j] for j < m  (the new sequenced log-rates, as
 *                           hawkes_hmc_scatter_rates writes them)
 * Equal bit for bit to hawkes_hmc_momentum, hawkes_hmc_position and
 * hawkes_hmc_scatter_rates in sequence.  HAWKES_EINVAL for k < 1, m < 0,
 * 6 + m > k, or NULL q, p, minv (or seq_idx, r when m > 0). */
int hawkes_hmc_leapfrog_step(int64_t k, double *q, double *p, const double *g, double a, const double *minv,
                             double eps, int64_t m, const int *seq_idx, double *r, void *stream);

/* The Metropolis accept/reject step that closes a trajectory (Section 2.3),
 * on the device, so that a sampler needs no host round trip per iteration.
 * With the energy H = -log pi(q) + K(p):
 *   H0 = -*lp + *k0 (the current state), H1 = -*lp1 + *k1 (the proposal),
 *   a = min(1, exp(H0 - H1)), or 0 when *lp1 or H1 is not finite or *status
 *   is non-zero (status may be NULL: no error);
 *   accepted iff *u < a (u: a uniform draw in [0, 1), a DEVICE double).
 * When accepted, q[k], *lp and grad[k] (DEVICE, in/out: the current state,
 * its log posterior and gradient) take the proposal's q1, *lp1 and grad1;
 * otherwise they are left unchanged.  Optional record slots (NULL: none):
 * rec_q[i] = the resulting state's q[keep[i]] for i < n_keep (keep: DEVICE
 * int64 indices; an index outside [0, k) records NaN) and rec[3] = (the
 * resulting log posterior, a, 1.0 if accepted else 0.0).  All pointers are
 * DEVICE; the proposal buffers must not alias the state's.  HAWKES_EINVAL for
 * k < 1, NULL required pointers, n_keep < 0 or aliasing. */
int hawkes_hmc_accept(int64_t k, const double *u, const double *k0, const double *k1, const double *lp1,
                      const double *grad1, const double *q1, const int *status, double *q, double *lp, double *grad,
                      int64_t n_keep, const int64_t *keep, double *rec_q, double *rec, void *stream);
/* The same pieces with a dense mass matrix (Section 2.3.2's preconditioned HMC,
 * with M dense) over k <= 64 coordinates (a posterior over the six globals
 * alone, whose correlations a diagonal mass cannot follow):
 * minv is M^-1 (DEVICE double[k*k], row-major).
 *   hawkes_hmc_position_dense: q += eps * M^-1 p
 *   hawkes_hmc_kinetic_dense:  *out = 1/2 p^T M^-1 p
 * HAWKES_EINVAL for k outside [1, 64] or NULL pointers. */
int hawkes_hmc_position_dense(int64_t k, double *q, const double *p, const double *minv, double eps, void *stream);
int hawkes_hmc_kinetic_dense(int64_t k, const double *p, const double *minv, double *out, void *stream);

/* ------------------------------------------------------------------------
 * The phylogenetic Brownian prior in O(M) (Section 2.2, Eq. 2; computed by
 * message passing on the tree as in Section 2.3.1) instead of through a dense
 * M x M precision.  z ~ N(0, sigma^2 V) with V_ij = root_var + (branch length
 * from the root to the most recent common ancestor of tips i and j).
 *
 * Tree encoding: nodes 0..m-1 are the tips, in the order of z (tip j carries
 * z_j, the log-rate of sequenced event j); nodes m..2m-2 are internal.  The
 * HOST array parent[2m-1] gives each node's parent (-1 at the root, which must
 * be an internal node); every internal node has exactly two children.
 * length[2m-1] (DEVICE) holds each node's branch length to its parent (the
 * root's entry is ignored).  Lengths must be non-negative and V positive
 * definite; a singular V gives non-finite outputs.
 * ------------------------------------------------------------------------ */
#define HAWKES_TREE_MAX_TIPS (1 << 24)

/* Bytes of the plan hawkes_tree_plan writes for m tips (0 if m is out of range). */
size_t hawkes_tree_plan_size(int64_t m);

/* Builds the traversal plan (children, and the internal nodes grouped by
 * height so that each level depends only on lower ones) on the HOST from
 * parent[].  plan is HOST memory of plan_bytes; copy it to the device for
 * hawkes_tree_prior.  Returns HAWKES_EINVAL if parent[] is not a rooted binary
 * tree on m tips (two roots, a cycle, a node with three children, a tip with
 * children), HAWKES_EWORKSPACE if plan_bytes is too small.  Runs on the host
 * only; O(m). */
int hawkes_tree_plan(int64_t m, const int64_t *parent, int *plan, size_t plan_bytes);

/* Bytes of DEVICE workspace hawkes_tree_prior needs for m tips. */
size_t hawkes_tree_workspace_size(int64_t m);

/* log N(z; 0, sigma^2 V) (Eq. 2) and its derivatives, in O(m) on one block:
 *   plan      DEVICE copy of the hawkes_tree_plan output
 *   length    DEVICE double[2m-1]; root_var >= 0 (the root's variance over sigma^2); sigma2 > 0
 *   z         DEVICE double[m]
 *   logdens   DEVICE double[1] or NULL: the log density, normalising constant included
 *   pz        DEVICE double[m] or NULL: (sigma^2 V)^-1 z (minus the density's gradient in z)
 *   pdiag     DEVICE double[m] or NULL: the diagonal of (sigma^2 V)^-1
 * Enqueued on stream; HAWKES_EINVAL for bad scalars or NULL inputs. */
int hawkes_tree_prior(int64_t m, const int *plan, const double *length, double root_var, double sigma2,
                      const double *z, void *ws, size_t ws_bytes, double *logdens, double *pz, double *pdiag,
                      void *stream);

/* Bytes of DEVICE workspace hawkes_posterior_tree needs for m sequenced events. */
size_t hawkes_posterior_tree_workspace_size(int64_t m);

/* hawkes_posterior with the phylogenetic prior taken from the tree
 * (P = (sigma^2 V)^-1 applied by hawkes_tree_prior) instead of a dense
 * precision; same arguments and results otherwise, m >= 2. */
int hawkes_posterior_tree(int64_t n, int64_t m, const int *seq_idx, const int *plan, const double *length,
                          double root_var, double sigma2, const hawkes_prior *prior, const double *q,
                          const double *loglik, const double *grad, const double *hdiag, void *ws,
                          size_t ws_bytes, double *logpost, double *grad_q, double *hdiag_q, void *stream);

/* ------------------------------------------------------------------------
 * Tree-structured HMC mass matrix (Section 2.3.2 preconditions the leapfrog
 * with a diagonal mass from the Hessian; this widens the rate block to the
 * phylogenetic prior's full precision, Section 2.2 Eq. 2, applied in O(m) on
 * the tree like Section 2.3.1's dynamic programme).  For a k-dimensional
 * sampler state whose coordinates [z0, z0 + m) are the sequenced log-rates
 * (tip j of the tree = coordinate z0 + j):
 *     M = diag(1 / minv)                       outside the block,
 *     M_z = diag(d) + (sigma^2 V)^-1           on the block,
 * with d[m] >= 0 the likelihood's curvature on the rates (entries below 0
 * or NaN count as 0).  V, plan, length, root_var and sigma2 are as for
 * hawkes_tree_prior; all arrays are DEVICE memory, enqueued on stream; one
 * block; no allocation.  Bad scalars, NULL inputs or z0 + m > k give
 * HAWKES_EINVAL, a short ws HAWKES_EWORKSPACE; a plan built for another m
 * makes every output NaN.
 *
 * Optionally the first nc coordinates (nc <= z0, nc <= 8: the globals) are
 * coupled to the rate block, M = [[A, B^T], [B, M_z]] with A nc x nc and
 * B m x nc.  The caller passes cpl (DEVICE doubles, m nc + 2 nc^2):
 *     U = M_z^-1 B          m x nc, row i = tip i      (from nc velocity calls)
 *     S^-1                  nc x nc, row-major, S = A - B^T U (positive definite)
 *     L                     nc x nc, row-major lower Cholesky factor of S
 * and then x_g = S^-1 (p_g - U^T p_z), x_z = M_z^-1 p_z - U x_g, and the
 * momentum's p_g = U^T p_z + L xi_g.  With nc = 0 (cpl may be NULL) the
 * first coordinates keep the diagonal minv.
 * ------------------------------------------------------------------------ */
#define HAWKES_TREE_MASS_MAX_COUPLED 8

/* Bytes of DEVICE workspace the three calls below need for m tips (scratch
 * only: nothing in it outlives a call). */
size_t hawkes_tree_mass_workspace_size(int64_t m);

/* The sweep coefficients of M_z for the curvature d (DEVICE double[m]):
 * fac (DEVICE double[2 (2m - 1)], caller-owned) receives, per tree node v,
 * r_v = 1 / (1 + s_v J_v) and s_v r_v, where s_v = sigma2 length_v (sigma2
 * root_var at the root) and J_v is the curvature gathered below v.  Call it
 * again whenever d changes; hawkes_tree_mass_velocity reads fac. */
int hawkes_tree_mass_factor(int64_t m, const int *plan, const double *length, double root_var, double sigma2,
                            const double *dlik, double *fac, void *ws, size_t ws_bytes, void *stream);

/* Velocity M^-1 p by one upward and one downward sweep of the tree, with
 * the coefficients fac from hawkes_tree_mass_factor:
 *   p        DEVICE double[k], the momentum
 *   vel      DEVICE double[k] or NULL: M^-1 p
 *   q        DEVICE double[k] or NULL: the leapfrog position step q += eps M^-1 p
 *   kinetic  DEVICE double[1] or NULL: p^T M^-1 p / 2
 * At least one of vel, q, kinetic must be given. */
int hawkes_tree_mass_velocity(int64_t m, const int *plan, const double *fac, int64_t nc, const double *cpl,
                              int64_t k, int64_t z0, const double *minv, const double *p, double *vel, double *q,
                              double eps, double *kinetic, void *ws, size_t ws_bytes, void *stream);

/* A momentum p ~ N(0, M) (DEVICE double[k]) from standard normals xi (DEVICE
 * double[k + 2m - 1]): p_i = xi_i / sqrt(minv_i) outside the block (and the
 * coupled set, whose p_g is U^T p_z + L xi[0, nc) when nc > 0) and
 * p_z = sqrt(d) xi_z + (sigma^2 V)^-1 w inside, where w is the Brownian motion
 * down the tree driven by the node normals xi[k + v] (v = 0..2m-2 in the
 * tree's node numbering): w_root = sqrt(sigma2 root_var) xi[k + root] and
 * w_v = w_parent + sqrt(sigma2 length_v) xi[k + v]. */
int hawkes_tree_mass_momentum(int64_t m, const int *plan, const double *length, double root_var, double sigma2,
                              const double *dlik, int64_t nc, const double *cpl, int64_t k, int64_t z0,
                              const double *minv, const double *xi, double *p, void *ws, size_t ws_bytes,
                              void *stream);

/* ------------------------------------------------------------------------
 * Posterior-predictive simulation (the forward simulation proposed in the
 * paper's Discussion: exact simulation of the Hawkes process with exponential
 * temporal trigger, run in parallel over posterior parameter settings with
 * counter-based random numbers).  For each of n_samples parameter settings,
 * the events of (T0, T0 + horizon], T0 = max t, are drawn exactly from the
 * intensity of Section 2.1 conditioned on the history, through the branching
 * representation: background events seeded by each past event's kernel, the
 * remaining children of past events (memorylessness of the exponential
 * trigger), then generation after generation of children of new events
 * (theta = 1 for new events).  Events are listed stage by stage, parent by
 * parent, child by child, so the output does not depend on the launch.
 * Random numbers: Philox4x32-10, key = seed, counter = (item, draw, stage,
 * sample_offset + s); the same draws give the same events on any GPU.
 * ------------------------------------------------------------------------ */
#define HAWKES_PREDICTIVE_MAX_CAPACITY (1 << 24)

/* Bytes of DEVICE workspace hawkes_predictive needs for n past events. */
size_t hawkes_predictive_workspace_size(int64_t n);

/*   x, y, t, r_base   DEVICE double[n]: the history (r_base the log-rates of
 *                     unsequenced events; any order of t)
 *   seq_idx           DEVICE int[m], distinct event indices of the sequenced events
 *   q                 DEVICE double[n_samples * q_stride]: row s holds a
 *                     parameter setting in sampler coordinates (log mu0,
 *                     log tau_x, log tau_t, log theta0, log omega, log h,
 *                     r of the m sequenced events); q_stride >= 6 + m
 *   horizon > 0, seed, sample_offset (added to s in the random counter)
 *   capacity          events kept per sample, 1..HAWKES_PREDICTIVE_MAX_CAPACITY
 *   out_x, out_y, out_t  DEVICE double[n_samples * capacity], row s at s * capacity
 *   out_src           DEVICE int64[n_samples * capacity]: -(n'+1) for background
 *                     seeded by past event n', n for a child of past event n,
 *                     n + e for a child of the sample's own event e
 *   out_count         DEVICE int64[n_samples]: events written
 *   out_status        DEVICE int[n_samples]: 0 complete; 1 the capacity was
 *                     reached (the first `capacity` events are written); 2 the
 *                     parameters are not finite and positive (tau_t may be +inf)
 * Enqueued on stream; HAWKES_EINVAL for bad arguments. */
int hawkes_predictive(const double *x, const double *y, const double *t, const double *r_base, int64_t n,
                      const int *seq_idx, int64_t m, const double *q, int64_t n_samples, int64_t q_stride,
                      double horizon, uint64_t seed, uint32_t sample_offset, int64_t capacity, void *ws,
                      size_t ws_bytes, double *out_x, double *out_y, double *out_t, int64_t *out_src,
                      int64_t *out_count, int *out_status, void *stream);

/* ------------------------------------------------------------------------
 * Learned gradient surrogate (the paper has none; the learned part of this
 * library): a 6 -> 128 -> 128 -> 6 tanh MLP with BF16 weights and FP32
 * accumulation, mapping standardised log-globals to the standardised gradient
 * of the log posterior, trained by these calls and used inside HMC leapfrog
 * trajectories while the exact likelihood keeps the accept step.
 * Weights: one vector of hawkes_mlp_param_count() values laid out as
 * W1[128x6], b1[128], W2[128x128], b2[128], W3[6x128], b3[6] (row-major, rows
 * are outputs).  BF16 arrays are uint16 bit patterns; all pointers DEVICE.
 * ------------------------------------------------------------------------ */
size_t hawkes_mlp_param_count(void);
/* DEVICE workspace bytes for hawkes_mlp_loss_grad with this batch size. */
size_t hawkes_mlp_workspace_size(int64_t batch);
/* y[batch x 6] = MLP(x[batch x 6]). */
int hawkes_mlp_forward(const void *w_bf16, const float *x, int64_t batch, float *y, void *stream);
/* Mean squared error over batch x 6 outputs and its gradient w.r.t. every
 * weight (FP32, summed over the batch's 8-sample blocks in a fixed order). */
int hawkes_mlp_loss_grad(const void *w_bf16, const float *x, const float *target, int64_t batch, void *ws,
                         size_t ws_bytes, float *grad, float *loss, void *stream);
/* One Adam step (bias-corrected, step >= 1) on the FP32 master weights and
 * moments m, v; refreshes the BF16 copy (round to nearest even). */
int hawkes_mlp_adam(float *w_master, void *w_bf16, float *m, float *v, const float *grad, float lr, float beta1,
                    float beta2, float eps, int step, void *stream);
/* Adam's bias corrections for steps 1..steps, as hawkes_mlp_adam forms them:
 * table[2 (s - 1)] = 1 - beta1^s, table[2 (s - 1) + 1] = 1 - beta2^s (HOST
 * float[2 steps]).  Host only. */
int hawkes_mlp_adam_table(float beta1, float beta2, int steps, float *table);
/* hawkes_mlp_adam with the step read from DEVICE memory, so that a captured
 * training step can be replayed: step s = *step + 1, the learning rate *lr
 * and the bias corrections table[2 (s - 1)], [+1] (DEVICE float[2 max_steps],
 * from hawkes_mlp_adam_table) are read on the device, and *step is advanced
 * by one after the update.  A step beyond max_steps leaves the weights alone.
 * Equal bit for bit to hawkes_mlp_adam at the same step and learning rate. */
int hawkes_mlp_adam_device(float *w_master, void *w_bf16, float *m, float *v, const float *grad, const float *lr,
                           const float *table, int max_steps, int *step, float beta1, float beta2, float eps,
                           void *stream);
/* Surrogate gradient at one sampler state q[0..5] and, when p is not NULL, the
 * leapfrog momentum update p[0..5] += a * g, with
 *   g = mean_g + A (q - mean_q) + sd_g * MLP((q - mean_q) / sd_q):
 * a linear model of the gradient plus the network's standardised residual.
 * norm = [mean_q(6), sd_q(6), mean_g(6), sd_g(6), A(6x6, row-major)] (DEVICE
 * doubles); g_out (DEVICE double[6]) receives g when not NULL. */
int hawkes_surrogate_momentum(const void *w_bf16, const double *q, double *p, double a, const double *norm,
                              double *g_out, void *stream);
/* A whole surrogate leapfrog trajectory over the six globals in one launch
 * (one block): p += eps/2 g(q), then n_steps times q += eps minv p and
 * p += eps g(q), the last momentum step halved, with g the surrogate gradient
 * of hawkes_surrogate_momentum.  Equal bit for bit to the sequence of
 * hawkes_surrogate_momentum and hawkes_hmc_position launches it replaces.
 * q, p: DEVICE double[6], updated in place; minv: DEVICE double[6], the
 * diagonal inverse mass; norm as for hawkes_surrogate_momentum; n_steps >= 0.
 * Returns HAWKES_EINVAL for NULL pointers, a negative n_steps or a NaN eps. */
int hawkes_surrogate_trajectory(const void *w_bf16, const double *norm, double *q, double *p, const double *minv,
                                double eps, int n_steps, void *stream);
/* The same trajectory with a dense inverse mass: minv is M^-1 (DEVICE
 * double[36], row-major) and each position step is q += eps M^-1 p, as in
 * hawkes_hmc_position_dense (equal bit for bit to those launches). */
int hawkes_surrogate_trajectory_dense(const void *w_bf16, const double *norm, double *q, double *p,
                                      const double *minv, double eps, int n_steps, void *stream);

/* Work count of the space-time passes (measurement for the roofline of
 * HAWKES_FP32C_ST; the paper has no counterpart).  ws must hold an
 * HAWKES_FP32C_ST hawkes_hess_diag evaluation of n events (its group records,
 * constants and column bounds); counts (DEVICE uint64[3], overwritten)
 * receives the ordered (target, source) pairs inside the group pairs whose
 * background [0] and excitation [1] terms the row pass evaluates, and the
 * (source, target) pairs inside the group pairs the column pass evaluates [2],
 * by the passes' own classification.  Enqueued on stream; the results of the
 * evaluation are not touched.  HAWKES_EINVAL for bad n, NULL or misaligned
 * pointers; HAWKES_EWORKSPACE when ws_bytes is too small. */
int hawkes_st_live_pairs(int64_t n, void *ws, size_t ws_bytes, unsigned long long *counts, void *stream);

/* Largest n accepted by hawkes_hess_diag_noalloc. */
#define HAWKES_NOALLOC_MAX_EVENTS 4096

/* hawkes_hess_diag for callers that cannot allocate device memory: the paper
 * has no counterpart; this is a deployment convenience.  Some callers cannot
 * call cudaMalloc when they evaluate -- a plugin inside a host program that
 * owns all device allocations, or a loop that cannot afford cudaMalloc's
 * implicit device synchronisation -- so this call takes no workspace and uses
 * a 16 MiB device array that the library owns (held on every GPU that loads
 * the library until exit).  Same inputs, outputs, results and errors as
 * hawkes_hess_diag with a workspace, for 2 <= n <= HAWKES_NOALLOC_MAX_EVENTS;
 * a larger n returns HAWKES_ESCRATCH without enqueuing anything.  The first
 * call on each device looks up the array's device address (make it before any
 * stream capture); that address dies with the device's context, so a process
 * that calls cudaDeviceReset must not call this entry point afterwards.  All calls on a device share the array, so calls that can
 * overlap on the GPU race on it: issue them in order on one stream.  Nothing
 * is allocated. */
int hawkes_hess_diag_noalloc(const double *x, const double *y, const double *t, const double *r, int64_t n,
                             const double params[6], int precision, double *loglik, double *grad, double *hdiag,
                             int *dev_status, void *stream);

/* ALU throughput microbenchmarks (the denominators of the roofline; the paper
 * has no counterpart): which = 0 packed FP32 FMA (f32x2), 1 MUFU exp2, 2 FP64
 * FMA.  hawkes_peak_launch enqueues blocks x 256 threads, each running
 * independent chains for iters steps, a multiple of 8 (sink: DEVICE float[1], written only to
 * keep the work live); the caller times it on its stream.  hawkes_peak_ops
 * gives the lane operations one launch performs (0 for bad arguments). */
int64_t hawkes_peak_ops(int which, int64_t blocks, int iters);
int hawkes_peak_launch(int which, int64_t blocks, int iters, float *sink, void *stream);

/* Static English description of a hawkes_status code. */
const char *hawkes_strerror(int status);

/* Library version string. */
const char *hawkes_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HAWKES_H */
