// Posterior-predictive simulation: the events of (T0, T0 + H] drawn exactly
// from the intensity of Section 2.1 conditioned on the history, for many
// parameter settings at once (one block per posterior draw), as the paper's
// Discussion proposes (exact simulation exploiting the exponential temporal
// trigger, parallel over parameter settings, counter-based random numbers).
//
// Branching representation, listed stage by stage, parent by parent:
//   stage 0  past event n' seeds Poisson(mu0 m_n') background events,
//            m_n' = Q((T0 - t_n')/tau_t) - Q((T1 - t_n')/tau_t) (H if tau_t is
//            infinite, Q the normal upper tail), at N(t_n', tau_t^2) truncated
//            to the window (uniform if tau_t is infinite), placed at
//            (x_n', y_n') + tau_x N(0, I);
//   stage 1  past event n has Poisson(theta0 theta_n e^{-omega (T0 - t_n)}
//            (1 - e^{-omega H})) children at T0 + Exp(omega) truncated to
//            (0, H] (memorylessness), placed at (x_n, y_n) + h N(0, I);
//   stage g  every event e of the previous generation (theta = 1) has
//            Poisson(theta0 (1 - e^{-omega (T1 - t_e)})) children at
//            t_e + Exp(omega) truncated to (0, T1 - t_e], at (x_e, y_e) + h N(0, I).
// Each chunk of 256 items draws its counts, takes a block-wide exclusive scan
// for the output offsets, and writes its children in order, so the output is
// independent of the launch shape.
//
// Random numbers: Philox4x32-10 (Salmon et al. 2011, written here from its
// definition), key = 64-bit seed, counter = (item, draw, stage, sample).
// Draw 0 decides an item's count; draws 2k+1 and 2k+2 give child k its time
// and place.  Uniforms (a 2^26 + b + 1/2) 2^-53, a = w0 >> 5, b = w1 >> 6.
// A Poisson mean above 500 is drawn as ceil(mean/500) equal parts (draws
// 2^31 + p); a mean above four times the capacity saturates the count, which
// makes the sample report an overflow with its first `capacity` events.
//
// Most past events have a tiny mean, and the count is 0 whenever
// u <= 1 - mean.  So stages 0 and 1 first bound the mean from above in FP32
// and integer arithmetic only: arguments rounded outward with directed-rounding
// intrinsics from per-event FP32 copies (T0 - t rounded down, r rounded up),
// and CUDA's documented error of expf and erfcf (a few ulp) covered 200 times
// over; 1 - u is bounded below from the random word in integers.  If the bound
// already gives K = 0 (bound < 2^-56, or 1 - u >= bound), the FP64 decision is
// the same and nothing in FP64 runs for that event.  The outputs are
// identical to the all-FP64 evaluation.
#include "hawkes_internal.cuh"

namespace hk {

constexpr int PRED_THREADS = 256;
constexpr double POISSON_PART = 500.0;
constexpr uint32_t PART_DRAW = 0x80000000u;

struct PhiloxOut {
    uint32_t w0, w1, w2, w3;
};

__device__ __forceinline__ PhiloxOut philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                   uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        if (i > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
        const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return {c0, c1, c2, c3};
}

__device__ __forceinline__ double u53(uint32_t w0, uint32_t w1) {
    return ((double)(w0 >> 5) * 67108864.0 + (double)(w1 >> 6) + 0.5) / 9007199254740992.0;
}

struct Rng {
    uint32_t k0, k1, sample;
    __device__ __forceinline__ void two(uint32_t item, uint32_t draw, uint32_t stage, double &a, double &b) const {
        const PhiloxOut w = philox4x32_10(item, draw, stage, sample, k0, k1);
        a = u53(w.w0, w.w1);
        b = u53(w.w2, w.w3);
    }
};

// The smallest k with u <= P(K <= k), K ~ Poisson(lam).
__device__ int64_t poisson_inv(double lam, double u) {
    if (!(lam > 0.0)) return 0;
    if (u <= 1.0 - lam) return 0;  // P(K = 0) = e^-lam > 1 - lam
    double p = exp(-lam), f = p;
    int64_t k = 0;
    while (u > f) {
        ++k;
        p *= lam / (double)k;
        f += p;
        if (p == 0.0 && (double)k > lam) break;
    }
    return k;
}

__device__ int64_t poisson_count(double lam, const Rng &rng, uint32_t item, uint32_t stage, int64_t cap) {
    if (!(lam > 0.0)) return 0;
    if (lam > 4.0 * (double)cap) return cap + 1;
    double u, unused;
    if (lam <= POISSON_PART) {
        rng.two(item, 0u, stage, u, unused);
        return poisson_inv(lam, u);
    }
    const int64_t parts = (int64_t)ceil(lam / POISSON_PART);
    const double sub = lam / (double)parts;
    int64_t k = 0;
    for (int64_t j = 0; j < parts; ++j) {
        rng.two(item, PART_DRAW + (uint32_t)j, stage, u, unused);
        k += poisson_inv(sub, u);
    }
    return k;
}

__device__ __forceinline__ double upper_tail(double z) { return 0.5 * erfc(z / 1.4142135623730951); }

// Relative slack for an FP32 exp / erfc value, and absolute slack covering
// FP32 underflow (the smallest subnormal).
constexpr float UB_REL = 1.0e-4f;
constexpr float UB_ABS = 1.5e-45f;
constexpr float NEGLIGIBLE = 1.3877787807814457e-17f;  // 2^-56: 1 - mean rounds to 1 in FP64

// Upper bound of 0.5 erfc(za / sqrt 2) for the FP64 path's za = fl((T0 - t) / tau_t),
// from d_lo <= fl(T0 - t) and inv_tt_lo <= 1 / tau_t.
__device__ __forceinline__ float tail_upper(float d_lo, float inv_tt_lo) {
    const float za_lo = fmaxf(__fsub_rd(__fmul_rd(d_lo, inv_tt_lo), 1.0e-6f), 0.0f);
    const float x_lo = __fmul_rd(za_lo, 0.70710677f);  // the FP32 constant is below 1/sqrt 2
    return __fadd_ru(__fmul_ru(__fmul_ru(0.5f, erfcf(x_lo)), 1.0f + UB_REL), UB_ABS);
}

// Upper bound of exp(arg) for the FP64 path's arg = fl(r - omega fl(T0 - t)),
// from r_up >= r, om_lo <= omega, d_lo <= fl(T0 - t); 1e-4 absorbs FP64 rounding.
__device__ __forceinline__ float exp_upper(float r_up, float om_lo, float d_lo) {
    const float arg = __fadd_ru(__fsub_ru(r_up, __fmul_rd(om_lo, d_lo)), 1.0e-4f);
    return __fadd_ru(__fmul_ru(expf(arg), 1.0f + UB_REL), UB_ABS);
}

// True when K = 0 is certain for every mean <= bound (so also for the FP64
// mean): the bound is negligible, or 1 - u >= bound with 1 - u bounded below
// from the random words in integers.  Decisions the bound cannot settle
// (false) go to FP64.
__device__ __forceinline__ bool surely_zero(float bound, const Rng &rng, uint32_t item, uint32_t stage) {
    if (!(bound <= (float)POISSON_PART)) return false;  // inf / NaN / large
    if (bound < NEGLIGIBLE) return true;
    const PhiloxOut w = philox4x32_10(item, 0u, stage, rng.sample, rng.k0, rng.k1);
    // u = (a 2^26 + b + 1/2) 2^-53 with a < 2^27, b < 2^26, so 1 - u >= (2^27 - 1 - a) 2^-27
    const float one_minus_u_lo = __uint2float_rd((1u << 27) - 1u - (w.w0 >> 5)) * 7.450580596923828e-09f;
    return one_minus_u_lo >= bound;
}

struct PredArgs {
    const double *x, *y, *t, *r_base;
    const int *seq_pos;  // [n]: position among the sequenced events, or -1
    const float *d_lo;   // [n]: T0 - t rounded down to FP32
    const float *rb_up;  // [n]: r_base rounded up to FP32
    const double *t0p;   // [1]: T0 = max t
    int64_t n, m;
    const double *q;
    int64_t q_stride;
    double horizon;
    uint32_t k0, k1, sample_offset;
    int64_t cap;
    double *ox, *oy, *ot;
    int64_t *osrc, *ocount;
    int *ostatus;
};

// inclusive-exclusive block scan of per-thread counts; returns the exclusive
// prefix and writes the block total into *total
__device__ int64_t block_scan(int64_t v, int64_t *sh, int64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t nb = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += nb;
    }
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < PRED_THREADS / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t nb = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += nb;
        }
        if (lane < PRED_THREADS / 32) sh[lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    const int64_t before = (warp > 0 ? sh[warp - 1] : 0) + incl - v;
    *total = sh[PRED_THREADS / 32 - 1];
    __syncthreads();
    return before;
}

// Upper bound of 1 - e^{-x} for the FP64 path's x = fl(omega fl(T1 - t)):
// min(x, 1 - expf(-x) + slack) at x rounded up (expf's few-ulp error on a
// value <= 1 and the subtraction's rounding stay below 4e-7).
__device__ __forceinline__ float one_minus_exp_upper(float x_up) {
    return fminf(x_up, __fadd_ru(__fsub_ru(1.0f, expf(-x_up)), 4.0e-7f));
}

// Shared state of one chunk of PRED_THREADS items.
struct Chunk {
    int64_t off[PRED_THREADS + 1];        // exclusive prefix of the counts; off[PRED_THREADS] = total
    int64_t k[PRED_THREADS];              // count of each item
    double pa[PRED_THREADS], pb[PRED_THREADS];  // stage 0: the tails Q(za), Q(zb); later: 1 - e^{-omega (T1 - t_e)}
    int queue[PRED_THREADS];              // items whose count the FP32 bound left undecided
    int n_queue;
    int64_t scan[PRED_THREADS / 32];
};

// Each chunk: (1) every thread bounds its item's mean in FP32 and settles
// K = 0 or queues the item; (2) all threads take the queued items in turn for
// the FP64 mean and the Poisson count; (3) a block scan gives the offsets;
// (4) all threads take the children in turn, each finding its parent by
// binary search over the offsets.  Lanes stay busy in the FP64 parts, and the
// output order (item by item, child by child) does not depend on the launch.
__global__ void __launch_bounds__(PRED_THREADS) predictive_kernel(PredArgs a) {
    __shared__ Chunk C;
    __shared__ int64_t s_count;
    __shared__ int s_status;
    const int64_t s = blockIdx.x;
    const double *qs = a.q + s * a.q_stride;
    const size_t row = (size_t)s * (size_t)a.cap;
    double *ox = a.ox + row, *oy = a.oy + row, *ot = a.ot + row;
    int64_t *osrc = a.osrc + row;
    const Rng rng{a.k0, a.k1, a.sample_offset + (uint32_t)s};
    const int tid = threadIdx.x;

    const double mu0 = exp(qs[0]), tx = exp(qs[1]), tt = exp(qs[2]), th0 = exp(qs[3]), om = exp(qs[4]),
                 h = exp(qs[5]);
    const bool ok = isfinite(mu0) && mu0 > 0 && isfinite(tx) && tx > 0 && tt > 0 && !isnan(tt) && isfinite(th0) &&
                    th0 > 0 && isfinite(om) && om > 0 && isfinite(h) && h > 0;
    if (!ok) {
        if (tid == 0) {
            a.ocount[s] = 0;
            a.ostatus[s] = 2;
        }
        return;  // uniform across the block
    }
    if (tid == 0) {
        s_count = 0;
        s_status = 0;
    }
    const double t0 = *a.t0p, t1 = t0 + a.horizon, H = a.horizon;
    const bool tt_inf = isinf(tt);
    const double one_m_h = -expm1(-om * H);
    // outward-rounded FP32 constants for the bounds
    const float mu0_up = __double2float_ru(mu0 * (1.0 + 1e-15)), th0_up = __double2float_ru(th0 * (1.0 + 1e-15));
    const float omh_up = __double2float_ru(one_m_h * (1.0 + 1e-15)), om_lo = __double2float_rd(om * (1.0 - 1e-15));
    const float om_up = __double2float_ru(om * (1.0 + 1e-15));
    const float inv_tt_lo = tt_inf ? 0.0f : __double2float_rd((1.0 / tt) * (1.0 - 1e-15));
    const float bg_inf_up = __fmul_ru(mu0_up, __double2float_ru(H));
    __syncthreads();

    int64_t gs = 0, ge = 0;
    for (uint32_t stage = 0; s_status == 0; ++stage) {
        int64_t lo = 0, hi = a.n;  // stages 0 and 1: the past events
        if (stage >= 2) {          // later stages: the previous generation of the sample's own events
            lo = gs;
            hi = ge;
            if (lo >= hi) break;
        }
        for (int64_t c0 = lo; c0 < hi; c0 += PRED_THREADS) {
            const int64_t item = c0 + tid;
            if (tid == 0) C.n_queue = 0;
            C.k[tid] = 0;
            __syncthreads();
            // (1) FP32 bound of the mean: K = 0 settled, or queued for FP64
            if (item < hi) {
                float bound;
                if (stage == 0) {
                    bound = tt_inf ? bg_inf_up : __fmul_ru(mu0_up, tail_upper(a.d_lo[item], inv_tt_lo));
                } else if (stage == 1) {
                    const int j = a.seq_pos[item];
                    const float r_up = j >= 0 ? __double2float_ru(qs[6 + j]) : a.rb_up[item];
                    bound = __fmul_ru(__fmul_ru(th0_up, exp_upper(r_up, om_lo, a.d_lo[item])), omh_up);
                } else {
                    const float x_up = __fmul_ru(om_up, __double2float_ru(t1 - ot[item]));
                    bound = __fmul_ru(th0_up, __fmul_ru(one_minus_exp_upper(x_up), 1.0f + UB_REL));
                }
                if (!surely_zero(bound, rng, (uint32_t)item, stage)) C.queue[atomicAdd(&C.n_queue, 1)] = tid;
            }
            __syncthreads();
            // (2) FP64 means and counts of the queued items
            for (int qi = tid; qi < C.n_queue; qi += PRED_THREADS) {
                const int slot = C.queue[qi];
                const int64_t it = c0 + slot;
                double lam = 0.0;
                if (stage == 0) {
                    double qa = 0.0, qb = 0.0;
                    if (tt_inf) {
                        lam = mu0 * H;
                    } else if ((t0 - a.t[it]) / tt <= 39.0) {  // beyond, both tails underflow to 0
                        qa = upper_tail((t0 - a.t[it]) / tt);
                        qb = upper_tail((t1 - a.t[it]) / tt);
                        lam = mu0 * (qa - qb);
                    }
                    C.pa[slot] = qa;
                    C.pb[slot] = qb;
                } else if (stage == 1) {
                    const int j = a.seq_pos[it];
                    const double ri = j >= 0 ? qs[6 + j] : a.r_base[it];
                    lam = th0 * exp(ri - om * (t0 - a.t[it])) * one_m_h;
                } else {
                    const double one_m = -expm1(-om * (t1 - ot[it]));
                    C.pa[slot] = one_m;
                    lam = th0 * one_m;
                }
                C.k[slot] = poisson_count(lam, rng, (uint32_t)it, stage, a.cap);
            }
            __syncthreads();
            // (3) offsets
            int64_t total;
            const int64_t off = block_scan(C.k[tid], C.scan, &total);
            C.off[tid] = off;
            if (tid == 0) C.off[PRED_THREADS] = total;
            __syncthreads();
            // (4) children, spread over all threads
            const int64_t base = s_count;
            const int64_t room = a.cap - base;
            const int64_t todo = total < room ? total : room;
            for (int64_t c = tid; c < todo; c += PRED_THREADS) {
                int lo_j = 0, hi_j = PRED_THREADS;  // the last j with off[j] <= c
                while (hi_j - lo_j > 1) {
                    const int mid = (lo_j + hi_j) >> 1;
                    if (C.off[mid] <= c) lo_j = mid;
                    else hi_j = mid;
                }
                const int j = lo_j;
                const int64_t it = c0 + j, kk = c - C.off[j], idx = base + c;
                double u1, u2, u3, unused;
                rng.two((uint32_t)it, (uint32_t)(2 * kk + 1), stage, u1, u2);
                rng.two((uint32_t)it, (uint32_t)(2 * kk + 2), stage, u3, unused);
                const double rad = sqrt(-2.0 * log(u2)), ang = 6.283185307179586 * u3;
                double px, py, tc, sd;
                int64_t src;
                if (stage == 0) {
                    px = a.x[it];
                    py = a.y[it];
                    sd = tx;
                    const double qa = C.pa[j], qb = C.pb[j];
                    tc = tt_inf ? t0 + u1 * H : a.t[it] + tt * (1.4142135623730951 * erfcinv(2.0 * (qa - u1 * (qa - qb))));
                    src = -(it + 1);
                } else if (stage == 1) {
                    px = a.x[it];
                    py = a.y[it];
                    sd = h;
                    tc = t0 - log1p(-u1 * one_m_h) / om;
                    src = it;
                } else {
                    px = ox[it];
                    py = oy[it];
                    sd = h;
                    tc = ot[it] - log1p(-u1 * C.pa[j]) / om;
                    src = a.n + it;
                }
                ox[idx] = px + sd * rad * cos(ang);
                oy[idx] = py + sd * rad * sin(ang);
                ot[idx] = tc;
                osrc[idx] = src;
            }
            __syncthreads();
            if (tid == 0) {
                s_count = base + todo;
                if (total > room) s_status = 1;
            }
            __syncthreads();
            if (s_status != 0) break;
        }
        if (stage == 1) {
            gs = 0;
            ge = s_count;
        } else if (stage >= 2) {
            gs = ge;
            ge = s_count;
        }
    }
    if (tid == 0) {
        a.ocount[s] = s_count;
        a.ostatus[s] = s_status;
    }
}

// seq_pos[n] = j for seq_idx[j] = n, else -1; t0 = max t (one block)
__global__ void __launch_bounds__(1024) predictive_prep_kernel(const double *__restrict__ t, int64_t n,
                                                              const int *__restrict__ seq_idx, int64_t m,
                                                              int *__restrict__ seq_pos, double *__restrict__ t0) {
    __shared__ double sh[32];
    double mx = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        seq_pos[i] = -1;
        mx = fmax(mx, t[i]);
    }
    __syncthreads();
    for (int64_t j = threadIdx.x; j < m; j += 1024) {
        const int i = seq_idx[j];
        if (i >= 0 && i < n) seq_pos[i] = (int)j;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        mx = sh[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (threadIdx.x == 0) *t0 = mx;
    }
}

// d_lo[i] = T0 - t_i rounded down, rb_up[i] = r_base[i] rounded up (FP32)
__global__ void predictive_pack_kernel(const double *__restrict__ t, const double *__restrict__ r_base, int64_t n,
                                       const double *__restrict__ t0, float *__restrict__ d_lo,
                                       float *__restrict__ rb_up) {
    const double T0 = *t0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        d_lo[i] = __double2float_rd(T0 - t[i]);
        rb_up[i] = __double2float_ru(r_base[i]);
    }
}

static size_t seg(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

}  // namespace hk

extern "C" {

size_t hawkes_predictive_workspace_size(int64_t n) {
    if (n < 1 || n > HAWKES_MAX_EVENTS) return 0;
    return hk::seg((size_t)n * sizeof(int)) + 2 * hk::seg((size_t)n * sizeof(float)) + 256;
}

int hawkes_predictive(const double *x, const double *y, const double *t, const double *r_base, int64_t n,
                      const int *seq_idx, int64_t m, const double *q, int64_t n_samples, int64_t q_stride,
                      double horizon, uint64_t seed, uint32_t sample_offset, int64_t capacity, void *ws,
                      size_t ws_bytes, double *out_x, double *out_y, double *out_t, int64_t *out_src,
                      int64_t *out_count, int *out_status, void *stream) {
    if (n < 1 || n > HAWKES_MAX_EVENTS || m < 0 || m > n || n_samples < 0 || n_samples > 0x7fffffff) return HAWKES_EINVAL;
    if (!x || !y || !t || !r_base || (m > 0 && !seq_idx) || !ws || !out_count || !out_status) return HAWKES_EINVAL;
    if (n_samples > 0 && (!q || !out_x || !out_y || !out_t || !out_src)) return HAWKES_EINVAL;
    if (q_stride < 6 + m || capacity < 1 || capacity > HAWKES_PREDICTIVE_MAX_CAPACITY) return HAWKES_EINVAL;
    if (!(horizon > 0) || !isfinite(horizon)) return HAWKES_EINVAL;
    if ((uint64_t)n_samples + sample_offset > 0x100000000ull) return HAWKES_EINVAL;  // sample counters stay distinct
    if (((uintptr_t)ws & 255) != 0) return HAWKES_EINVAL;
    if (ws_bytes < hawkes_predictive_workspace_size(n)) return HAWKES_EWORKSPACE;
    if (n_samples == 0) return HAWKES_OK;
    cudaStream_t s = (cudaStream_t)stream;
    char *base = (char *)ws;
    int *seq_pos = (int *)base;
    float *d_lo = (float *)(base + hk::seg((size_t)n * sizeof(int)));
    float *rb_up = (float *)((char *)d_lo + hk::seg((size_t)n * sizeof(float)));
    double *t0 = (double *)((char *)rb_up + hk::seg((size_t)n * sizeof(float)));
    hk::predictive_prep_kernel<<<1, 1024, 0, s>>>(t, n, seq_idx, m, seq_pos, t0);
    if (cudaGetLastError() != cudaSuccess) return HAWKES_ECUDA;
    const int pack_blocks = (int)((n + 255) / 256 < 1184 ? (n + 255) / 256 : 1184);
    hk::predictive_pack_kernel<<<pack_blocks, 256, 0, s>>>(t, r_base, n, t0, d_lo, rb_up);
    if (cudaGetLastError() != cudaSuccess) return HAWKES_ECUDA;
    hk::PredArgs a;
    a.x = x;
    a.y = y;
    a.t = t;
    a.r_base = r_base;
    a.seq_pos = seq_pos;
    a.d_lo = d_lo;
    a.rb_up = rb_up;
    a.t0p = t0;
    a.n = n;
    a.m = m;
    a.q = q;
    a.q_stride = q_stride;
    a.horizon = horizon;
    a.k0 = (uint32_t)(seed & 0xffffffffu);
    a.k1 = (uint32_t)(seed >> 32);
    a.sample_offset = sample_offset;
    a.cap = capacity;
    a.ox = out_x;
    a.oy = out_y;
    a.ot = out_t;
    a.osrc = out_src;
    a.ocount = out_count;
    a.ostatus = out_status;
    hk::predictive_kernel<<<(unsigned)n_samples, hk::PRED_THREADS, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

}  // extern "C"
