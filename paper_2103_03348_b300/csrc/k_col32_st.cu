// FP32C_ST column passes (space-time tiles); the pair arithmetic is that of
// the time-order column pass (col32_tile.cuh).
#include <climits>

#include "col32_tile.cuh"

namespace hk {

// ---------------------------------------------------------------------------
// FP32C_ST column passes.  Targets that follow a source can sit earlier in its
// slab (positions are permuted inside slabs), so the sweep starts at the first
// tile of the source's slab.  As in the row pass, one block is one warp and
// owns 32 sources: it classifies each chunk's target tiles group by group
// against its sources' bounds, lists the tiles with a live group, and stages
// each live target group in a warp-private double buffer.  The causal mask
// compares the sources' time-order ranks with the targets' tie-group starts.
constexpr int CGPT = TILE / GROUP;

struct ColWarpShared {
    float4 ab[2][GROUP];
    int gi[2][GROUP];
    int item[GROUP * CGPT];  // live (tile, group) pairs, in order: tile * 4 + group, plus flags (below)
};

// One chunk [ub, ue) of target tiles for the warp's sources W; the
// compensated sums are carried in s1 / k1, s2 / k2.  The live target groups
// of up to 32 tiles are listed as items; each item's 32 targets are loaded
// into registers while the previous item is evaluated.
template <int MODE>
__device__ __forceinline__ void col_sweep_warp(const Workspace &ws, int ub, int ue, const GroupStat &W, float2 xm,
                                               float2 ym, float2 nrm, int rank, float hh, float &s1,
                                               float &k1, float &s2, float &k2, ColWarpShared &sh) {
    constexpr int ALLC = 1 << 30;  // item flag: every source precedes every target of the group
    const int lane = threadIdx.x & 31;
    float2 run1 = make_float2(0.f, 0.f), run2 = make_float2(0.f, 0.f);
    int buf = 0;
    for (int base = ub; base < ue; base += GROUP) {
        // classify target tile base + lane group by group; count its live groups
        const int u = base + lane;
        int live = 0, allc = 0, cnt = 0;
        if (u < ue && !(ws.sufmax[u] + W.tr.z < EXP2_DEAD)) {
            cnt = ws.tinfo[u].w;
#pragma unroll
            for (int g = 0; g < CGPT; ++g) {
                const GroupStat G = ws.grp[(size_t)u * CGPT + g];
                if (group_empty(G) || cnt <= g * GROUP || !col_alive(W, G, hh)) continue;
                live |= 1 << g;
                if (W.ix.w < G.ix.x) allc |= 1 << g;
            }
        }
        // exclusive prefix sum of the live counts over the warp: each lane's items go in order
        const int nl = __popc(live);
        int pre = nl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += v;
        }
        const int total = __shfl_sync(0xffffffffu, pre, 31);
        int pos = pre - nl;
#pragma unroll
        for (int g = 0; g < CGPT; ++g) {
            if ((live >> g) & 1) {
                const int cntg = min(cnt - g * GROUP, GROUP);
                sh.item[pos++] = (u * CGPT + g) | (((allc >> g) & 1) ? ALLC : 0) | ((cntg - 1) << 24);
            }
        }
        __syncwarp();
        float4 pab = make_float4(0.f, 0.f, 0.f, 0.f);
        int pg = 0;
        if (total > 0) {
            const int it = sh.item[0] & 0xffffff;
            pab = ws.tgt32[(size_t)it * GROUP + lane];
            pg = ws.gidx[(size_t)it * GROUP + lane];
        }
        for (int q = 0; q < total; ++q) {
            const int cur = sh.item[q];
            sh.ab[buf][lane] = pab;
            sh.gi[buf][lane] = pg;
            __syncwarp();
            int nt = -1;
            if (q + 1 < total) {  // the next group's loads are in flight during this one's arithmetic
                const int it = sh.item[q + 1] & 0xffffff;
                nt = it / CGPT;
                pab = ws.tgt32[(size_t)it * GROUP + lane];
                pg = ws.gidx[(size_t)it * GROUP + lane];
            }
            const int np = ((((cur >> 24) & 63) + 1) + 1) >> 1;
            if (cur & ALLC) col_tile<MODE, false>(sh.ab[buf], sh.gi[buf], np, xm, ym, nrm, rank, run1, run2);
            else col_tile<MODE, true>(sh.ab[buf], sh.gi[buf], np, xm, ym, nrm, rank, run1, run2);
            buf ^= 1;
            if (nt != (cur & 0xffffff) / CGPT) {  // tile boundary: merge the runs
                kahan(s1, k1, __fadd_rn(run1.x, run1.y));
                run1 = make_float2(0.f, 0.f);
                if (MODE == MODE_HESS) {
                    kahan(s2, k2, __fadd_rn(run2.x, run2.y));
                    run2 = make_float2(0.f, 0.f);
                }
            }
        }
        __syncwarp();  // the items are read until here
    }
}

template <int MODE>
__global__ void __launch_bounds__(GROUP, 24) col32_st_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    const Derived &D = *c.d;
    const int sg = c.t0 * CGPT + blockIdx.x;  // source group
    const int tile = sg / CGPT, chunk = blockIdx.y;
    const int m = sg * GROUP + threadIdx.x;  // position
    const int n = c.g.n, npad = c.g.npad;
    __shared__ ColWarpShared sh;

    float2 xm, ym, nrm;
    {
        // the source in the targets' scaled coordinates x' = (x - xc) sxh, and -r^_m
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
    const int rank = ws.perm[m];
    const GroupStat W = ws.grp[sg];
    const float hh = D.hh;

    float s1 = 0.f, k1 = 0.f, s2 = 0.f, k2 = 0.f;
    if (!group_empty(W)) {
        const int start = (tile / SLAB_TILES) * SLAB_TILES;
        const int ub = start + chunk * c.g.chunk_tiles;
        const int ue = min(c.g.tiles, ub + c.g.chunk_tiles);
        col_sweep_warp<MODE>(ws, ub, ue, W, xm, ym, nrm, rank, hh, s1, k1, s2, k2, sh);
    }
    ws.colpart[((size_t)chunk * 2 + 0) * npad + m] = (double)s1 - (double)k1;
    if (MODE == MODE_HESS) ws.colpart[((size_t)chunk * 2 + 1) * npad + m] = (double)s2 - (double)k2;
}

// FP32C_ST subset: block k (one warp) owns rate_idx[32k .. 32k+32) (time-order
// indices); their positions come from the inverse permutation and their
// bounds are reduced from the sources themselves.
template <int MODE>
__global__ void __launch_bounds__(GROUP, 24) col32_subset_st_kernel(Consts c, Inputs in, Workspace ws,
                                                                   const int *__restrict__ rate_idx, int k_rates) {
    pdl_wait();
    const Derived &D = *c.d;
    const int lane = threadIdx.x;
    const int j = blockIdx.x * GROUP + lane, chunk = blockIdx.y;
    const int n = c.g.n, npad = c.g.npad;
    const int raw = j < k_rates ? rate_idx[j] : -1;
    const bool valid = raw >= 0 && raw < n;  // an index outside [0, n) is skipped and reported
    if (j < k_rates && !valid && chunk == 0) atomicOr(&ws.hdr[0], ST_BADPARAM);
    const int m = valid ? ws.inv[raw] : 0;
    __shared__ ColWarpShared sh;

    float xw = 0.f, yw = 0.f, xh = 1.0e9f, yh = 1.0e9f, r = -1.0e9f;
    if (valid) {
        const float *f = reinterpret_cast<const float *>(ws.src32);
        const int p = m >> 1, l = m & 1;
        xw = -f[8 * p + 0 + l];  // the group bounds' scale (x~)
        yw = -f[8 * p + 2 + l];
        xh = (float)((in.x[m] - ws.centre[0]) * D.sxh);  // the targets' scale (x')
        yh = (float)((in.y[m] - ws.centre[1]) * D.sxh);
        r = (float)(in.r[m] * LOG2E + (in.t[m] - ws.centre[2]) * D.st);
    }
    const float2 xm = splat(xh), ym = splat(yh), nrm = splat(-r);
    const int rank = valid ? raw : INT_MAX;  // an invalid slot is masked everywhere
    GroupStat W;
    W.box = make_float4(warp_minf(valid ? xw : INFINITY), warp_maxf(valid ? xw : -INFINITY),
                        warp_minf(valid ? yw : INFINITY), warp_maxf(valid ? yw : -INFINITY));
    W.tr = make_float4(0.f, 0.f, warp_maxf(r), 0.f);
    W.ix = make_int4(0, 0, warp_mini(valid ? raw : INT_MAX), warp_maxi(valid ? raw : INT_MIN));
    const int start = warp_mini(valid ? (m / SLAB_EVENTS) * SLAB_TILES : INT_MAX);
    const float hh = D.hh;
    float s1 = 0.f, k1 = 0.f, s2 = 0.f, k2 = 0.f;
    if (start != INT_MAX) {  // warp-uniform: some source is valid
        const int ub = start + chunk * c.g.chunk_tiles;
        const int ue = min(c.g.tiles, ub + c.g.chunk_tiles);
        col_sweep_warp<MODE>(ws, ub, ue, W, xm, ym, nrm, rank, hh, s1, k1, s2, k2, sh);
    }
    if (valid) {
        ws.colpart[((size_t)chunk * 2 + 0) * npad + j] = (double)s1 - (double)k1;
        if (MODE == MODE_HESS) ws.colpart[((size_t)chunk * 2 + 1) * npad + j] = (double)s2 - (double)k2;
    }
}

cudaError_t launch_col32_st(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    const dim3 grid((c.t1 - c.t0) * CGPT, c.g.n_chunks);
    if (c.mode == MODE_HESS) launch_pdl(col32_st_kernel<MODE_HESS>, grid, GROUP, 0, s, c, in, ws);
    else launch_pdl(col32_st_kernel<MODE_GRAD>, grid, GROUP, 0, s, c, in, ws);
    return cudaGetLastError();
}

cudaError_t launch_col32_subset_st(const Consts &c, const Inputs &in, const Workspace &ws, const int *rate_idx,
                                   int k_rates, cudaStream_t s) {
    const dim3 grid((k_rates + GROUP - 1) / GROUP, c.g.n_chunks);
    if (c.mode == MODE_HESS) launch_pdl(col32_subset_st_kernel<MODE_HESS>, grid, GROUP, 0, s, c, in, ws, rate_idx, k_rates);
    else launch_pdl(col32_subset_st_kernel<MODE_GRAD>, grid, GROUP, 0, s, c, in, ws, rate_idx, k_rates);
    return cudaGetLastError();
}

}  // namespace hk
