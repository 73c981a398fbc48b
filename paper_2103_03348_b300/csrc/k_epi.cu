// Row finish, integral term and deterministic reductions (steps a3, a4).
//
// combine   FP64 path: mom[k][i] = sum over chunks of the row partials (fixed
//           order); FP32C does this (and the fix-up of tiny rows) at the end
//           of the row kernel (rows_finish.cuh).
// epilogue  per event n, in FP64:
//             lambda_n = A sum G + B sum E                          (Eq. 1 inner sum)
//             q1_p = (d lambda_n / dp) / lambda_n,  q2_p = (d2 lambda_n / dp2) / lambda_n - q1_p^2
//           from the moments, and the event's share of the integral term
//             Lambda_n = mu0 [Phi((t_N - t_n)/tau_t) - Phi(-t_n/tau_t)] + theta0 theta_n (1 - e^{-omega (t_N - t_n)})
//           (Appendix A Claim, background integrated exactly) with its
//           derivatives; each block writes the 13 block sums of
//           (log lambda_n - Lambda_n, q1_p - dLambda_n/dp, q2_p - d2Lambda_n/dp2).
// finalize  one block sums the block partials in a fixed order -> loglik,
//           gradient[0..5], Hessian diagonal[0..5]; status -> dev_status.
// colfinish dl/dr_m = C1_m - dLambda/dr_m, d2l/dr_m^2 = C1_m - C2_m - dLambda/dr_m.
//
// Derivatives of lambda_n (moments M in raw units, see hawkes_internal.cuh):
//   mu0:    A S_G / mu0
//   tau_x:  A (MO_GD2/tx^3 - 2 S_G/tx),   second A (MO_GD4/tx^6 - 7 MO_GD2/tx^4 + 6 S_G/tx^2)
//   tau_t:  A (MO_GT2/tt^3 - S_G/tt),     second A (MO_GT4/tt^6 - 5 MO_GT2/tt^4 + 2 S_G/tt^2)
//   theta0: B S_E / theta0
//   omega:  B (S_E/omega - MO_ET),        second B (MO_ET2 - 2 MO_ET/omega)
//   h:      B (MO_ED2/h^3 - 2 S_E/h),     second B (MO_ED4/h^6 - 7 MO_ED2/h^4 + 6 S_E/h^2)
// (from f(s) = s^-k exp(-q/(2 s^2)): f'/f = q/s^3 - k/s, f''/f = (f'/f)^2 - 3q/s^4 + k/s^2).
#include "rows_finish.cuh"

namespace hk {

constexpr int CB_THREADS = 256;

__global__ void __launch_bounds__(CB_THREADS) combine_kernel(Consts c, Workspace ws) {
    pdl_wait();
    const int i = c.t0 * TILE + blockIdx.x * CB_THREADS + threadIdx.x;
    if (i >= c.g.n || i >= c.t1 * TILE) return;
    const int npad = c.g.npad;
    for (int k = 0; k < NMOM; ++k) {
        const bool used = c.mode == MODE_HESS ||
                          (c.mode == MODE_GRAD && (k == MO_G || k == MO_GD2 || k == MO_GT2 || k == MO_E || k == MO_ET || k == MO_ED2)) ||
                          (k == MO_G || k == MO_E);
        if (!used) continue;
        double s = 0.0;
        for (int ch = 0; ch < c.g.n_chunks; ++ch) s += ws.rowpart[((size_t)ch * NMOM + k) * npad + i];
        ws.mom[(size_t)k * npad + i] = s;
    }
}

cudaError_t launch_combine(const Consts &c, const Workspace &ws, cudaStream_t s) {
    launch_pdl(combine_kernel, ((c.t1 - c.t0) * TILE + CB_THREADS - 1) / CB_THREADS, CB_THREADS, 0, s, c, ws);
    return cudaGetLastError();
}


__global__ void __launch_bounds__(TILE) epilogue_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    const Derived &D = *c.d;
    __shared__ double sh[(TILE / 32) * NACC];
    __shared__ float shf[TILE];
    const int tile = c.t0 + blockIdx.x;
    const int i = tile * TILE + threadIdx.x;
    const int n = c.g.n, npad = c.g.npad;
    const bool valid = i < n;
    double acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
    float ghat = -INFINITY;

    if (valid) {
        double Mo[NMOM];
#pragma unroll
        for (int k = 0; k < NMOM; ++k) Mo[k] = ws.mom[(size_t)k * npad + i];
        epilogue_row<true>(c, D, in, ws, i, Mo, acc, ghat);
    }
    {
        const double v = block_sum_multi<TILE, NACC>(acc, sh);
        if (threadIdx.x < NACC) ws.blockpart[(size_t)tile * ACC_STRIDE + threadIdx.x] = v;
    }
    if (c.fp32c) {
        if (c.st) {  // per-group bound for the column pass's pruning
            const float wm = warp_maxf(ghat);
            if ((threadIdx.x & 31) == 0) ws.grp[i / GROUP].tr.w = wm;
        }
        const float gm = block_max<TILE>(ghat, shf);
        if (threadIdx.x == 0) ws.tstat32[tile].w = gm;
    }
}

// FP32C: one block per target tile finishes its rows (rows_finish.cuh).
__global__ void __launch_bounds__(TILE) finish_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    finish_tile_fp32c(c, in, ws, c.t0 + blockIdx.x);
}

// FP32C_ST with few tiles: one block of FG_WARPS warps per target group finishes its 32 rows (rows_finish.cuh).
__global__ void __launch_bounds__(FG_WARPS * 32) finish_st_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    finish_group_st(c, in, ws, c.t0 * (TILE / GROUP) + blockIdx.x);
}

cudaError_t launch_finish(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    if (c.fin_groups) launch_pdl(finish_st_kernel, (c.t1 - c.t0) * (TILE / GROUP), FG_WARPS * 32, 0, s, c, in, ws);
    else launch_pdl(finish_kernel, c.t1 - c.t0, TILE, 0, s, c, in, ws);
    return cudaGetLastError();
}

cudaError_t launch_epilogue(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    launch_pdl(epilogue_kernel, c.t1 - c.t0, TILE, 0, s, c, in, ws);
    return cudaGetLastError();
}

constexpr int FIN_THREADS = 256;

__global__ void __launch_bounds__(FIN_THREADS) finalize_kernel(Consts c, Workspace ws, Outputs out) {
    pdl_wait();
    const Derived &D = *c.d;
    __shared__ double tot[NACC];
    const int tiles = c.g.tiles;
    // the block partials: one per tile, or one per 32-row group (finish_group_st)
    const int nparts = c.fin_groups ? tiles * (TILE / GROUP) : tiles;
    {
        // Warp w sums components w and w + 8 over the partials: each lane a fixed
        // strided subset, then a fixed shuffle butterfly.  (FP64 instructions
        // are costly here, and this keeps them to a few per lane.)
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int k = warp; k < NACC; k += FIN_THREADS / 32) {
            double v = 0.0;
#pragma unroll 8
            for (int b = lane; b < nparts; b += 32) v += ws.blockpart[(size_t)b * ACC_STRIDE + k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) tot[k] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int bits = ws.hdr[0];
        int code = HAWKES_OK;
        if (bits & ST_BADPARAM) code = HAWKES_EINVAL;
        else if (bits & ST_NONFINITE) code = HAWKES_ENONFINITE;
        else if (bits & ST_UNSORTED) code = HAWKES_EUNSORTED;
        else if (bits & ST_ZERO) code = HAWKES_EZERO_INTENSITY;
        const double qnan = __longlong_as_double(0x7ff8000000000000LL);
        double ll = tot[0];
        if (code == HAWKES_ENONFINITE || code == HAWKES_EUNSORTED || code == HAWKES_EINVAL) ll = qnan;
        else if (code == HAWKES_EZERO_INTENSITY) ll = -INFINITY;
        if (out.loglik) *out.loglik = ll;
        for (int p = 0; p < 6; ++p) {
            double g = tot[1 + p], hd = tot[7 + p];
            if (p == 2 && D.tt_inf) { g = 0.0; hd = 0.0; }
            if (code != HAWKES_OK) { g = qnan; hd = qnan; }
            if (out.grad) out.grad[p] = g;
            if (out.hdiag) out.hdiag[p] = hd;
        }
        if (out.dev_status) *out.dev_status = code;
    }
    if (c.fp32c && c.mode >= MODE_GRAD) {
        // suffix max of the per-tile column weight bound, for the column sweep's stop test:
        // each thread owns a contiguous segment of tiles; segment maxima are scanned in shared memory
        // (max is exact, so the scan order does not matter)
        __shared__ float wmax[FIN_THREADS / 32];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int len = (tiles + FIN_THREADS - 1) / FIN_THREADS;
        const int b0 = threadIdx.x * len, b1 = min(tiles, b0 + len);
        // a tile's largest g^: the tile statistic, or after a per-group finish the largest of its groups'
        auto tile_gmax = [&](int b) -> float {
            if (!c.fin_groups) return ws.tstat32[b].w;
            const GroupStat *gs = ws.grp + (size_t)b * (TILE / GROUP);
            return fmaxf(fmaxf(gs[0].tr.w, gs[1].tr.w), fmaxf(gs[2].tr.w, gs[3].tr.w));
        };
        float m = -INFINITY;
        for (int b = b0; b < b1; ++b) m = fmaxf(m, tile_gmax(b));
        // inclusive suffix max within the warp, then over the later warps
        float v = m;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float u = __shfl_down_sync(0xffffffffu, v, o);
            if (lane + o < 32) v = fmaxf(v, u);
        }
        if (lane == 0) wmax[warp] = v;
        __syncthreads();
        float later = -INFINITY;
        for (int w = warp + 1; w < FIN_THREADS / 32; ++w) later = fmaxf(later, wmax[w]);
        float excl = __shfl_down_sync(0xffffffffu, v, 1);  // max over the later segments of this warp
        if (lane == 31) excl = -INFINITY;
        float run = fmaxf(excl, later);
        for (int b = b1 - 1; b >= b0; --b) {
            run = fmaxf(run, tile_gmax(b));
            ws.sufmax[b] = run;
        }
    }
}

cudaError_t launch_finalize(const Consts &c, const Workspace &ws, const Outputs &out, cudaStream_t s) {
    launch_pdl(finalize_kernel, 1, FIN_THREADS, 0, s, c, ws, out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(CB_THREADS) colfinish_kernel(Consts c, Workspace ws, Outputs out) {
    pdl_wait();
    const int m = c.t0 * TILE + blockIdx.x * CB_THREADS + threadIdx.x;
    if (m >= c.g.n || m >= c.t1 * TILE) return;
    const int npad = c.g.npad;
    double c1 = 0.0, c2 = 0.0;
#pragma unroll 8
    for (int ch = 0; ch < c.g.n_chunks; ++ch) {
        c1 += ws.colpart[((size_t)ch * 2 + 0) * npad + m];
        if (c.mode == MODE_HESS) c2 += ws.colpart[((size_t)ch * 2 + 1) * npad + m];
    }
    const double dl = ws.dLr[m];
    double g = c1 - dl, hd = c1 - c2 - dl;
    if (ws.hdr[0] != 0) {
        const double qnan = __longlong_as_double(0x7ff8000000000000LL);
        g = qnan;
        hd = qnan;
    }
    const int o = c.st ? ws.perm[m] : m;  // outputs in time order
    if (out.grad) out.grad[6 + o] = g;
    if (out.hdiag) out.hdiag[6 + o] = hd;
}

// The finish for a subset of sources: entry 6 + rate_idx[j] of grad / hdiag,
// with the partials at subset position j (FP32C subset pass) or at the event
// index (FP64, whose column pass covers every source).  An index outside
// [0, n) is reported here, after finalize (which has written the status).
__global__ void __launch_bounds__(CB_THREADS) colfinish_subset_kernel(Consts c, Workspace ws, Outputs out,
                                                                      const int *__restrict__ rate_idx, int k_rates,
                                                                      int by_position) {
    pdl_wait();
    const int j = blockIdx.x * CB_THREADS + threadIdx.x;
    const int bits = ws.hdr[0];
    if (j == 0 && (bits & ST_BADPARAM)) *out.dev_status = HAWKES_EINVAL;
    if (j >= k_rates) return;
    const int m = rate_idx[j];
    if (m < 0 || m >= c.g.n) {
        *out.dev_status = HAWKES_EINVAL;
        return;
    }
    const int npad = c.g.npad, at = by_position ? j : (c.st ? ws.inv[m] : m);
    double c1 = 0.0, c2 = 0.0;
#pragma unroll 8
    for (int ch = 0; ch < c.g.n_chunks; ++ch) {
        c1 += ws.colpart[((size_t)ch * 2 + 0) * npad + at];
        if (c.mode == MODE_HESS) c2 += ws.colpart[((size_t)ch * 2 + 1) * npad + at];
    }
    const double dl = ws.dLr[c.st ? ws.inv[m] : m];
    double g = c1 - dl, hd = c1 - c2 - dl;
    if (bits != 0) {
        const double qnan = __longlong_as_double(0x7ff8000000000000LL);
        g = qnan;
        hd = qnan;
    }
    if (out.grad) out.grad[6 + m] = g;
    if (out.hdiag) out.hdiag[6 + m] = hd;
}

cudaError_t launch_colfinish_subset(const Consts &c, const Workspace &ws, const Outputs &out, const int *rate_idx,
                                    int k_rates, int by_position, cudaStream_t s) {
    launch_pdl(colfinish_subset_kernel, (k_rates + CB_THREADS - 1) / CB_THREADS, CB_THREADS, 0, s, c, ws, out, rate_idx,
                                                                                           k_rates, by_position);
    return cudaGetLastError();
}

cudaError_t launch_colfinish(const Consts &c, const Workspace &ws, const Outputs &out, cudaStream_t s) {
    launch_pdl(colfinish_kernel, ((c.t1 - c.t0) * TILE + CB_THREADS - 1) / CB_THREADS, CB_THREADS, 0, s, c, ws, out);
    return cudaGetLastError();
}

}  // namespace hk
