// FP32-compensated column pass (Eqs. 4 and 5; Algorithm 2, step 2, redesigned).
//
// For every source m the gradient and Hessian diagonal w.r.t. r_m = log theta_m
// need, over the later targets n (t_n > t_m strictly),
//     v_nm = B theta_m E'_nm / lambda_n        (the share of lambda_n due to m; 0 <= v <= 1)
//     C1_m = sum_n v_nm,   C2_m = sum_n v_nm^2
// because dl/dr_m = C1_m - dLambda/dr_m and d2l/dr_m^2 = C1_m - C2_m - dLambda/dr_m.
// In the scaled base-2 coordinates of the row pass,
//     v_nm = 2^(g^_n + r^_m - hh d~^2) = 2^(g^_n + r^_m - d'^2),
//     g^_n = log2(B / lambda_n) - t~_n,  r^_m = r~_m + t~_m,  x' = x~ tau_x / h,
// where the row finish stored -g^_n in the fourth slot of each packed target
// (tgt32) and the targets' coordinates in the x' scale.
//
// One block of 128 threads owns 128 sources (one per thread) and sweeps a
// chunk of later target tiles staged in shared memory, two targets per packed
// f32x2 instruction.  A target tile is skipped when no target follows any
// source (tie-group index), or when 2^(max g^ + max r^) < 2^-128 so that every
// term underflows to exactly 0 in FP32; the sweep stops once the suffix max of
// g^ shows that all later tiles underflow too.  Precision as in the row pass.
#include <climits>

#include "col32_tile.cuh"

namespace hk {

template <int MODE>
__global__ void __launch_bounds__(TILE, 4) col32_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    const Derived &D = *c.d;
    const int tile = c.t0 + blockIdx.x, chunk = blockIdx.y;
    const int m = tile * TILE + threadIdx.x;
    const int n = c.g.n, npad = c.g.npad;
    __shared__ float4 sAB[2][TILE];
    __shared__ int sG[2][TILE];

    float2 xm, ym, nrm;
    {
        // the source in the targets' scaled coordinates x' = (x - xc) sxh, and -r^_m with
        // r^_m = r~_m + t~_m, from the FP64 inputs (as pack forms it)
        float x = 0.f, y = 0.f, r = -1.0e9f;
        if (m < n) {
            x = (float)((in.x[m] - ws.centre[0]) * D.sxh);
            y = (float)((in.y[m] - ws.centre[1]) * D.sxh);
            r = (float)(in.r[m] * LOG2E + (in.t[m] - ws.centre[2]) * D.st);
        }
        xm = splat(x);
        ym = splat(y);
        nrm = splat(-r);
    }
    const int4 tiM = ws.tinfo[tile];
    const float4 stM = ws.tstat32[tile];
    const int m_first = tile * TILE, m_last = m_first + tiM.w - 1;

    float2 run1 = make_float2(0.f, 0.f), run2 = make_float2(0.f, 0.f);
    float s1 = 0.f, k1 = 0.f, s2 = 0.f, k2 = 0.f;

    const int ub = tile + chunk * c.g.chunk_tiles;
    const int ue = min(c.g.tiles, ub + c.g.chunk_tiles);
    int buf = 0;
    for (int u = ub; u < ue; ++u) {
        // uniform decisions for the whole block
        if (ws.sufmax[u] + stM.z < EXP2_DEAD) break;  // this and every later tile underflow
        const int4 tiU = ws.tinfo[u];
        const float4 stU = ws.tstat32[u];
        if (tiU.y <= m_first) continue;                 // no target of u follows any source
        if (stU.w + stM.z < EXP2_DEAD) continue;        // every term underflows
        const int u0 = u * TILE;
        sAB[buf][threadIdx.x] = ws.tgt32[(size_t)u0 + threadIdx.x];
        sG[buf][threadIdx.x] = ws.gidx[(size_t)u0 + threadIdx.x];
        __syncthreads();
        const int npairs = (tiU.w + 1) >> 1;
        const bool all_causal = m_last < tiU.x;
        if (all_causal) col_tile<MODE, false>(sAB[buf], sG[buf], npairs, xm, ym, nrm, m, run1, run2);
        else col_tile<MODE, true>(sAB[buf], sG[buf], npairs, xm, ym, nrm, m, run1, run2);
        kahan(s1, k1, __fadd_rn(run1.x, run1.y));
        run1 = make_float2(0.f, 0.f);
        if (MODE == MODE_HESS) {
            kahan(s2, k2, __fadd_rn(run2.x, run2.y));
            run2 = make_float2(0.f, 0.f);
        }
        buf ^= 1;
    }
    ws.colpart[((size_t)chunk * 2 + 0) * npad + m] = (double)s1 - (double)k1;
    if (MODE == MODE_HESS) ws.colpart[((size_t)chunk * 2 + 1) * npad + m] = (double)s2 - (double)k2;
}

// The same pass for a subset of sources only (a sampler whose free log-rates are
// those of M sequenced events needs O(N M) work, not O(N^2)).  Block k owns
// sources rate_idx[128k .. 128k+128) (any order); its tile statistics (lowest
// and highest source index, largest r^) are reduced at the start, and the
// target sweep, chunking and skip rules are those of col32_kernel.  The
// partials go to colpart[chunk][.][j] for the subset position j.
template <int MODE>
__global__ void __launch_bounds__(TILE, 4) col32_subset_kernel(Consts c, Inputs in, Workspace ws,
                                                               const int *__restrict__ rate_idx, int k_rates) {
    pdl_wait();
    const Derived &D = *c.d;
    const int j = blockIdx.x * TILE + threadIdx.x, chunk = blockIdx.y;
    const int n = c.g.n, npad = c.g.npad;
    const int raw = j < k_rates ? rate_idx[j] : -1;
    const bool valid = raw >= 0 && raw < n;  // an index outside [0, n) is skipped and reported
    if (j < k_rates && !valid && chunk == 0) atomicOr(&ws.hdr[0], ST_BADPARAM);
    const int m = valid ? raw : 0;
    __shared__ float4 sAB[2][TILE];
    __shared__ int sG[2][TILE];
    __shared__ float shf[TILE];
    __shared__ int shi[TILE];

    float2 xm, ym, nrm;
    float r = -1.0e9f;
    {
        // as in col32_kernel; an invalid slot sits far away with r^ = -1e9 (exact zeros)
        float x = 1.0e9f, y = 1.0e9f;
        if (valid && m < n) {
            x = (float)((in.x[m] - ws.centre[0]) * D.sxh);
            y = (float)((in.y[m] - ws.centre[1]) * D.sxh);
            r = (float)(in.r[m] * LOG2E + (in.t[m] - ws.centre[2]) * D.st);
        }
        xm = splat(x);
        ym = splat(y);
        nrm = splat(-r);
    }
    // tile statistics of this block's sources (uniform for the block)
    const float rmax = block_max<TILE>(r, shf);
    shi[threadIdx.x] = valid ? m : INT_MAX;
    __syncthreads();
    for (int w = TILE / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) shi[threadIdx.x] = min(shi[threadIdx.x], shi[threadIdx.x + w]);
        __syncthreads();
    }
    const int m_first = shi[0];
    __syncthreads();
    shi[threadIdx.x] = valid ? m : -1;
    __syncthreads();
    for (int w = TILE / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) shi[threadIdx.x] = max(shi[threadIdx.x], shi[threadIdx.x + w]);
        __syncthreads();
    }
    const int m_last = shi[0];

    float2 run1 = make_float2(0.f, 0.f), run2 = make_float2(0.f, 0.f);
    float s1 = 0.f, k1 = 0.f, s2 = 0.f, k2 = 0.f;

    const int tile0 = m_first / TILE;
    const int ub = tile0 + chunk * c.g.chunk_tiles;
    const int ue = min(c.g.tiles, ub + c.g.chunk_tiles);
    int buf = 0;
    for (int u = ub; u < ue; ++u) {
        if (ws.sufmax[u] + rmax < EXP2_DEAD) break;  // this and every later tile underflow
        const int4 tiU = ws.tinfo[u];
        const float4 stU = ws.tstat32[u];
        if (tiU.y <= m_first) continue;               // no target of u follows any source
        if (stU.w + rmax < EXP2_DEAD) continue;       // every term underflows
        const int u0 = u * TILE;
        sAB[buf][threadIdx.x] = ws.tgt32[(size_t)u0 + threadIdx.x];
        sG[buf][threadIdx.x] = ws.gidx[(size_t)u0 + threadIdx.x];
        __syncthreads();
        const int npairs = (tiU.w + 1) >> 1;
        const bool all_causal = m_last < tiU.x;
        if (all_causal) col_tile<MODE, false>(sAB[buf], sG[buf], npairs, xm, ym, nrm, m, run1, run2);
        else col_tile<MODE, true>(sAB[buf], sG[buf], npairs, xm, ym, nrm, valid ? m : INT_MAX, run1, run2);
        kahan(s1, k1, __fadd_rn(run1.x, run1.y));
        run1 = make_float2(0.f, 0.f);
        if (MODE == MODE_HESS) {
            kahan(s2, k2, __fadd_rn(run2.x, run2.y));
            run2 = make_float2(0.f, 0.f);
        }
        buf ^= 1;
    }
    if (valid) {
        ws.colpart[((size_t)chunk * 2 + 0) * npad + j] = (double)s1 - (double)k1;
        if (MODE == MODE_HESS) ws.colpart[((size_t)chunk * 2 + 1) * npad + j] = (double)s2 - (double)k2;
    }
}

cudaError_t launch_col32_subset(const Consts &c, const Inputs &in, const Workspace &ws, const int *rate_idx,
                                int k_rates, cudaStream_t s) {
    if (c.st) return launch_col32_subset_st(c, in, ws, rate_idx, k_rates, s);
    const dim3 grid((k_rates + TILE - 1) / TILE, c.g.n_chunks);
    if (c.mode == MODE_HESS) launch_pdl(col32_subset_kernel<MODE_HESS>, grid, TILE, 0, s, c, in, ws, rate_idx, k_rates);
    else launch_pdl(col32_subset_kernel<MODE_GRAD>, grid, TILE, 0, s, c, in, ws, rate_idx, k_rates);
    return cudaGetLastError();
}

cudaError_t launch_col32(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    const dim3 grid(c.t1 - c.t0, c.g.n_chunks);
    if (c.st) return launch_col32_st(c, in, ws, s);
    if (c.mode == MODE_HESS) launch_pdl(col32_kernel<MODE_HESS>, grid, TILE, 0, s, c, in, ws);
    else launch_pdl(col32_kernel<MODE_GRAD>, grid, TILE, 0, s, c, in, ws);
    return cudaGetLastError();
}

}  // namespace hk
