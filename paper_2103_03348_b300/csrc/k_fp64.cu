// FP64 row and column passes.
//
// The FP64 path evaluates every pair with libm-accurate exp() and accumulates
// the same moments as the FP32C row pass, in FP64 and raw units:
//     G = exp(-d^2/(2 tau_x^2) - dt^2/(2 tau_t^2))  for sources at another location
//     E = exp(r_s - omega dt - d^2/(2 h^2))          for strictly earlier sources
// No cutoff: only source tiles in which no source precedes any target skip the
// excitation (those terms are zero by the indicator).  On B300 FP64 runs at
// 1/64 of the FP32 rate, which is why this path is the precision reference on
// the GPU and not the fast path.
#include "rows_finish.cuh"

namespace hk {

template <int MODE>
__global__ void __launch_bounds__(TILE) row64_kernel(Consts c, Workspace ws) {
    pdl_wait();
    const Derived &D = *c.d;
    const int tile = c.t0 + blockIdx.x, chunk = blockIdx.y;
    const int i = tile * TILE + threadIdx.x;
    const int npad = c.g.npad;
    __shared__ double4_32a sS[TILE];
    __shared__ int sLoc[TILE];
    const double4_32a me = ws.src64[i];
    const int locn = ws.loc[i], gn = ws.gidx[i];
    const int4 tiT = ws.tinfo[tile];
    double a[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) a[k] = 0.0;
    const int sb = chunk * c.g.chunk_tiles;
    const int se = min(c.g.tiles, sb + c.g.chunk_tiles);
    for (int s = sb; s < se; ++s) {
        __syncthreads();
        sS[threadIdx.x] = ws.src64[(size_t)s * TILE + threadIdx.x];
        sLoc[threadIdx.x] = ws.loc[(size_t)s * TILE + threadIdx.x];
        __syncthreads();
        const int4 tiS = ws.tinfo[s];
        const int s0 = s * TILE;
        const bool none_causal = s0 >= tiT.y;
        for (int j = 0; j < tiS.w; ++j) {
            const double4_32a src = sS[j];
            accumulate64<MODE>(a, src.x, src.y, src.z, src.w, sLoc[j] != locn, !none_causal && (s0 + j < gn),
                               me.x, me.y, me.z, D);
        }
    }
#pragma unroll
    for (int k = 0; k < NMOM; ++k)
        if (MODE == MODE_HESS || (MODE == MODE_GRAD && (k == MO_G || k == MO_GD2 || k == MO_GT2 || k == MO_E || k == MO_ET || k == MO_ED2)) ||
            (MODE == MODE_LL && (k == MO_G || k == MO_E)))
            ws.rowpart[((size_t)chunk * NMOM + k) * npad + i] = a[k];
}

cudaError_t launch_row64(const Consts &c, const Workspace &ws, cudaStream_t s) {
    const dim3 grid(c.t1 - c.t0, c.g.n_chunks);
    if (c.mode == MODE_HESS) launch_pdl(row64_kernel<MODE_HESS>, grid, TILE, 0, s, c, ws);
    else if (c.mode == MODE_GRAD) launch_pdl(row64_kernel<MODE_GRAD>, grid, TILE, 0, s, c, ws);
    else launch_pdl(row64_kernel<MODE_LL>, grid, TILE, 0, s, c, ws);
    return cudaGetLastError();
}

// Column pass in FP64: v_nm = exp(log(B / lambda_n) + r_m - omega (t_n - t_m) - d^2/(2h^2)),
// the weight kept in the log domain so that a tiny lambda_n cannot overflow it.
template <int MODE>
__global__ void __launch_bounds__(TILE) col64_kernel(Consts c, Workspace ws) {
    pdl_wait();
    const Derived &D = *c.d;
    const int tile = c.t0 + blockIdx.x, chunk = blockIdx.y;
    const int m = tile * TILE + threadIdx.x;
    const int npad = c.g.npad;
    __shared__ double4_32a sT[TILE];
    __shared__ double sW[TILE];
    __shared__ int sG[TILE];
    const double4_32a me = ws.src64[m];
    const int4 tiM = ws.tinfo[tile];
    const int m_first = tile * TILE;
    double c1 = 0.0, c2 = 0.0;
    const int ub = tile + chunk * c.g.chunk_tiles;
    const int ue = min(c.g.tiles, ub + c.g.chunk_tiles);
    for (int u = ub; u < ue; ++u) {
        const int4 tiU = ws.tinfo[u];
        if (tiU.y <= m_first) continue;  // uniform: no target of u follows any source
        __syncthreads();
        sT[threadIdx.x] = ws.src64[(size_t)u * TILE + threadIdx.x];
        sW[threadIdx.x] = ws.w64[(size_t)u * TILE + threadIdx.x];
        sG[threadIdx.x] = ws.gidx[(size_t)u * TILE + threadIdx.x];
        __syncthreads();
        for (int j = 0; j < tiU.w; ++j) {
            if (m < sG[j]) {
                const double4_32a t = sT[j];
                const double dx = t.x - me.x, dy = t.y - me.y, dt = t.z - me.z;
                const double v = exp(sW[j] + me.w - D.om * dt - D.ih * (dx * dx + dy * dy));
                c1 += v;
                if (MODE == MODE_HESS) c2 += v * v;
            }
        }
    }
    (void)tiM;
    ws.colpart[((size_t)chunk * 2 + 0) * npad + m] = c1;
    if (MODE == MODE_HESS) ws.colpart[((size_t)chunk * 2 + 1) * npad + m] = c2;
}

cudaError_t launch_col64(const Consts &c, const Workspace &ws, cudaStream_t s) {
    const dim3 grid(c.t1 - c.t0, c.g.n_chunks);
    if (c.mode == MODE_HESS) launch_pdl(col64_kernel<MODE_HESS>, grid, TILE, 0, s, c, ws);
    else launch_pdl(col64_kernel<MODE_GRAD>, grid, TILE, 0, s, c, ws);
    return cudaGetLastError();
}

}  // namespace hk
