// FP32C_ST column passes (space-time tiles); the pair arithmetic is that of
// the time-order column pass (col32_tile.cuh).
#include <climits>

#include "col32_tile.cuh"

namespace hk {

// ---------------------------------------------------------------------------
// FP32C_ST column passes.  Targets that follow a source can sit earlier in its
// slab (positions are permuted inside slabs), so the sweep starts at the first
// tile of the source's slab.  As in the row pass, each chunk's target tiles
// are classified in parallel against the union of the block's source groups
// and listed; each listed tile is staged in shared memory and each warp skips
// the target groups whose terms all underflow for its own 32 sources.  The
// causal mask compares the sources' time-order ranks with the targets'
// tie-group starts.
constexpr int CGPT = TILE / GROUP;

constexpr int CSTAGE = 4;  // listed target tiles staged per barrier (double-buffered)

struct ColShared {
    float4 ab[2][CSTAGE][TILE];
    int gi[2][CSTAGE][TILE];
    GroupStat gs[2][CSTAGE][CGPT];
    int list[TILE];
    int cnt[CGPT];
};

// One chunk [ub, ue) of target tiles for sources described by W (this warp)
// and U (the block); the compensated sums are carried in s1 / k1, s2 / k2.
template <int MODE>
__device__ __forceinline__ void col_sweep_st(const Workspace &ws, int ub, int ue, const GroupStat &W,
                                             const GroupStat &U, float2 xm, float2 ym, float2 rm, int rank,
                                             float2 nhh2, float hh, float &s1, float &k1, float &s2, float &k2,
                                             ColShared &sh) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool w_empty = group_empty(W);
    float2 run1 = make_float2(0.f, 0.f), run2 = make_float2(0.f, 0.f);
    int buf = 0;
    for (int base = ub; base < ue; base += TILE) {
        const int u = base + threadIdx.x;
        int live = 0;
        if (u < ue && !(ws.sufmax[u] + U.tr.z < EXP2_DEAD)) {
#pragma unroll
            for (int g = 0; g < CGPT; ++g) {
                const GroupStat G = ws.grp[(size_t)u * CGPT + g];
                if (!group_empty(G) && col_alive(U, G, hh)) live = 1;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, live != 0);
        if (lane == 0) sh.cnt[warp] = __popc(bal);
        __syncthreads();
        int off = 0, total = 0;
#pragma unroll
        for (int w = 0; w < CGPT; ++w) {
            if (w < warp) off += sh.cnt[w];
            total += sh.cnt[w];
        }
        if (live) sh.list[off + __popc(bal & ((1u << lane) - 1u))] = u;
        __syncthreads();
        for (int q0 = 0; q0 < total; q0 += CSTAGE) {
            const int nst = min(CSTAGE, total - q0);
#pragma unroll
            for (int kk = 0; kk < CSTAGE; ++kk) {
                if (kk < nst) {
                    const int uu = sh.list[q0 + kk];
                    const size_t u0 = (size_t)uu * TILE;
                    sh.ab[buf][kk][threadIdx.x] = ws.tgt32[u0 + threadIdx.x];
                    sh.gi[buf][kk][threadIdx.x] = ws.gidx[u0 + threadIdx.x];
                    if (threadIdx.x < CGPT) sh.gs[buf][kk][threadIdx.x] = ws.grp[(size_t)uu * CGPT + threadIdx.x];
                }
            }
            __syncthreads();
#pragma unroll 1
            for (int kk = 0; kk < nst; ++kk) {
                const int cnt = ws.tinfo[sh.list[q0 + kk]].w;
#pragma unroll 1
                for (int g = 0; g < CGPT; ++g) {
                    const int cntg = min(max(cnt - g * GROUP, 0), GROUP);
                    if (cntg == 0) continue;
                    const GroupStat G = sh.gs[buf][kk][g];
                    if (w_empty || !col_alive(W, G, hh)) continue;  // warp-uniform
                    const int np = (cntg + 1) >> 1;
                    const float4 *ab = sh.ab[buf][kk] + g * GROUP;
                    const int *gi = sh.gi[buf][kk] + g * GROUP;
                    if (W.ix.w < G.ix.x)  // every source precedes every target
                        col_tile<MODE, false>(ab, gi, np, xm, ym, rm, rank, nhh2, run1, run2);
                    else
                        col_tile<MODE, true>(ab, gi, np, xm, ym, rm, rank, nhh2, run1, run2);
                }
                kahan(s1, k1, __fadd_rn(run1.x, run1.y));
                run1 = make_float2(0.f, 0.f);
                if (MODE == MODE_HESS) {
                    kahan(s2, k2, __fadd_rn(run2.x, run2.y));
                    run2 = make_float2(0.f, 0.f);
                }
            }
            buf ^= 1;
        }
        __syncthreads();  // the list is read until here
    }
}

template <int MODE>
__global__ void __launch_bounds__(TILE, 4) col32_st_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    const Derived &D = *c.d;
    const int tile = c.t0 + blockIdx.x, chunk = blockIdx.y;
    const int m = tile * TILE + threadIdx.x;  // position
    const int n = c.g.n, npad = c.g.npad;
    const int warp = threadIdx.x >> 5;
    __shared__ ColShared sh;

    float2 xm, ym, rm;
    {
        const float *f = reinterpret_cast<const float *>(ws.src32);
        const int p = m >> 1, l = m & 1;
        xm = splat(-f[8 * p + 0 + l]);
        ym = splat(-f[8 * p + 2 + l]);
        float r = -1.0e9f;
        if (m < n) r = (float)(in.r[m] * LOG2E + (in.t[m] - ws.centre[2]) * D.st);
        rm = splat(r);
    }
    const int rank = ws.perm[m];
    const GroupStat W = ws.grp[tile * CGPT + warp];
    GroupStat U = ws.grp[tile * CGPT];
#pragma unroll
    for (int g = 1; g < CGPT; ++g) U = group_union(U, ws.grp[tile * CGPT + g]);
    const float hh = D.hh;
    const float2 nhh2 = splat(-hh);

    float s1 = 0.f, k1 = 0.f, s2 = 0.f, k2 = 0.f;
    const int start = (tile / SLAB_TILES) * SLAB_TILES;
    const int ub = start + chunk * c.g.chunk_tiles;
    const int ue = min(c.g.tiles, ub + c.g.chunk_tiles);
    col_sweep_st<MODE>(ws, ub, ue, W, U, xm, ym, rm, rank, nhh2, hh, s1, k1, s2, k2, sh);
    ws.colpart[((size_t)chunk * 2 + 0) * npad + m] = (double)s1 - (double)k1;
    if (MODE == MODE_HESS) ws.colpart[((size_t)chunk * 2 + 1) * npad + m] = (double)s2 - (double)k2;
}

// FP32C_ST subset: block k owns rate_idx[128k .. 128k+128) (time-order indices);
// their positions come from the inverse permutation, and the warp and block
// bounds are reduced from the sources themselves.
template <int MODE>
__global__ void __launch_bounds__(TILE, 4) col32_subset_st_kernel(Consts c, Inputs in, Workspace ws,
                                                                  const int *__restrict__ rate_idx, int k_rates) {
    pdl_wait();
    const Derived &D = *c.d;
    const int j = blockIdx.x * TILE + threadIdx.x, chunk = blockIdx.y;
    const int n = c.g.n, npad = c.g.npad;
    const int warp = threadIdx.x >> 5;
    const int raw = j < k_rates ? rate_idx[j] : -1;
    const bool valid = raw >= 0 && raw < n;  // an index outside [0, n) is skipped and reported
    if (j < k_rates && !valid && chunk == 0) atomicOr(&ws.hdr[0], ST_BADPARAM);
    const int m = valid ? ws.inv[raw] : 0;
    __shared__ ColShared sh;
    __shared__ GroupStat sW[CGPT];
    __shared__ int sStart[CGPT];

    float xw = 0.f, yw = 0.f, r = -1.0e9f;
    if (valid) {
        const float *f = reinterpret_cast<const float *>(ws.src32);
        const int p = m >> 1, l = m & 1;
        xw = -f[8 * p + 0 + l];
        yw = -f[8 * p + 2 + l];
        r = (float)(in.r[m] * LOG2E + (in.t[m] - ws.centre[2]) * D.st);
    }
    const float2 xm = splat(valid ? xw : 1.0e9f), ym = splat(valid ? yw : 1.0e9f), rm = splat(r);
    const int rank = valid ? raw : INT_MAX;  // an invalid slot is masked everywhere
    GroupStat W;
    W.box = make_float4(warp_minf(valid ? xw : INFINITY), warp_maxf(valid ? xw : -INFINITY),
                        warp_minf(valid ? yw : INFINITY), warp_maxf(valid ? yw : -INFINITY));
    W.tr = make_float4(0.f, 0.f, warp_maxf(r), 0.f);
    W.ix = make_int4(0, 0, warp_mini(valid ? raw : INT_MAX), warp_maxi(valid ? raw : INT_MIN));
    const int st0 = warp_mini(valid ? (m / SLAB_EVENTS) * SLAB_TILES : INT_MAX);
    if ((threadIdx.x & 31) == 0) {
        sW[warp] = W;
        sStart[warp] = st0;
    }
    __syncthreads();
    GroupStat U = sW[0];
    int start = sStart[0];
#pragma unroll
    for (int g = 1; g < CGPT; ++g) {
        U = group_union(U, sW[g]);
        start = min(start, sStart[g]);
    }
    const float hh = D.hh;
    const float2 nhh2 = splat(-hh);
    float s1 = 0.f, k1 = 0.f, s2 = 0.f, k2 = 0.f;
    if (start != INT_MAX) {  // block-uniform: some source is valid
        const int ub = start + chunk * c.g.chunk_tiles;
        const int ue = min(c.g.tiles, ub + c.g.chunk_tiles);
        col_sweep_st<MODE>(ws, ub, ue, W, U, xm, ym, rm, rank, nhh2, hh, s1, k1, s2, k2, sh);
    }
    if (valid) {
        ws.colpart[((size_t)chunk * 2 + 0) * npad + j] = (double)s1 - (double)k1;
        if (MODE == MODE_HESS) ws.colpart[((size_t)chunk * 2 + 1) * npad + j] = (double)s2 - (double)k2;
    }
}

cudaError_t launch_col32_st(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    const dim3 grid(c.t1 - c.t0, c.g.n_chunks);
    if (c.mode == MODE_HESS) launch_pdl(col32_st_kernel<MODE_HESS>, grid, TILE, 0, s, c, in, ws);
    else launch_pdl(col32_st_kernel<MODE_GRAD>, grid, TILE, 0, s, c, in, ws);
    return cudaGetLastError();
}

cudaError_t launch_col32_subset_st(const Consts &c, const Inputs &in, const Workspace &ws, const int *rate_idx,
                                   int k_rates, cudaStream_t s) {
    const dim3 grid((k_rates + TILE - 1) / TILE, c.g.n_chunks);
    if (c.mode == MODE_HESS) launch_pdl(col32_subset_st_kernel<MODE_HESS>, grid, TILE, 0, s, c, in, ws, rate_idx, k_rates);
    else launch_pdl(col32_subset_st_kernel<MODE_GRAD>, grid, TILE, 0, s, c, in, ws, rate_idx, k_rates);
    return cudaGetLastError();
}

}  // namespace hk
