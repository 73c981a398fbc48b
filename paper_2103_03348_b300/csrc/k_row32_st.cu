// FP32C_ST row pass (space-time tiles): see row32_st_kernel below; the pair
// arithmetic is that of the time-order row pass (row32_pair.cuh).
#include "row32_pair.cuh"
#include "rows_finish.cuh"

namespace hk {

// FP32C_ST row pass.  Positions hold events permuted inside slabs so that
// each group of 32 positions is compact in space and time.  One work unit is
// one target group (32 rows) against one chunk of source tiles, run by one
// warp, so no warp ever waits for another (the warps are persistent and take
// units in turn, row32_st_kernel below):
//   * classify: lane l tests source tile base + l group by group against the
//     warp's own target group (background live, excitation live, masks
//     needed), and the live groups of the 32 tiles are listed in order as
//     items (a warp prefix sum places each lane's items);
//   * sweep: each item's 32 sources are staged in the warp's shared buffer
//     (double-buffered, one __syncwarp) while the next item's load into
//     registers, and evaluated with the pair arithmetic, masks and
//     compensation of row32_kernel, the runs merged at each tile boundary;
//     the causal mask compares time-order ranks.
constexpr int GPT = TILE / GROUP;  // groups per tile

// One work unit: target group `bx` of the call's range against source chunk
// rotation `by` (the grid position of a one-warp block before the pass became
// persistent).
template <int MODE>
__device__ __forceinline__ void row32_st_unit(const Consts &c, const Inputs &in, const Workspace &ws, int bx,
                                              int by) {
    const Derived &D = *c.d;
    const int tg = c.t0 * GPT + bx;  // target group
    const int tile = tg / GPT, gw = tg % GPT;
    const int chunk = (tile / c.g.chunk_tiles - by + c.g.n_chunks) % c.g.n_chunks;
    const int lane = threadIdx.x;
    const int i = tg * GROUP + lane;
    const int npad = c.g.npad;
    // live (tile, group) items of up to 32 source tiles, in order: the source
    // group index (bits 0-23), plus bit 24 background, 25 excitation, 26
    // location mask, 27 causal mask
    __shared__ int sItem[GROUP * GPT];
    __shared__ int sItemCnt[GROUP * GPT];  // each item's source count
    __shared__ float4 sAB[2][GROUP];
    __shared__ int sLoc[2][GROUP];
    __shared__ int sRank[2][GROUP];

    RowTarget T;
    {
        const float *f = reinterpret_cast<const float *>(ws.src32);
        const int p = i >> 1, l = i & 1;
        const float x = -f[8 * p + 0 + l], y = -f[8 * p + 2 + l], t = -f[8 * p + 4 + l];
        T.xn = splat(x); T.yn = splat(y); T.tn = splat(t); T.ntn = splat(-t);
        T.locn = ws.loc[i];
        T.gn = ws.gidx[i];
    }
    const bool dupT = ws.tinfo[tile].z != 0;
    const GroupStat W = ws.grp[tg];
    const float cbt = D.cbt, hh = D.hh;
    const float2 cbt2 = splat(cbt), nhh2 = splat(-hh);

    float2 run[NMOM];
    float ks[NMOM], kc[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) { run[k] = make_float2(0.0f, 0.0f); ks[k] = 0.0f; kc[k] = 0.0f; }

    const int sb = chunk * c.g.chunk_tiles;
    const int se = min(c.g.tiles, sb + c.g.chunk_tiles);
    int buf = 0;
    if (!group_empty(W)) {
        for (int base = sb; base < se; base += GROUP) {
            // classify source tile base + lane group by group against this warp's targets
            const int s = base + lane;
            int live = 0, flags = 0, cnt = 0;  // flags: 4 bits per group (bg, exc, location mask, causal mask)
            if (s < se) {
                const int4 tiS = ws.tinfo[s];
                cnt = tiS.w;
                const bool dup = dupT && tiS.z;
#pragma unroll
                for (int g = 0; g < GPT; ++g) {
                    const GroupStat S = ws.grp[(size_t)s * GPT + g];
                    if (cnt <= g * GROUP || group_empty(S)) continue;
                    const bool bgw = bg_alive(W, S, cbt), exw = exc_alive(W, S, hh);
                    if (!bgw && !exw) continue;
                    live |= 1 << g;
                    int f = (bgw ? 1 : 0) | (exw ? 2 : 0);
                    if ((s == tile && g == gw) || dup) f |= 4;
                    if (exw && !(S.ix.w < W.ix.x)) f |= 8;
                    flags |= f << (4 * g);
                }
            }
            // exclusive prefix sum of the live counts: each lane's items go in order
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
            for (int g = 0; g < GPT; ++g) {
                if ((live >> g) & 1) {
                    const int cntg = min(cnt - g * GROUP, GROUP);
                    sItem[pos++] = (s * GPT + g) | (((flags >> (4 * g)) & 15) << 24);
                    sItemCnt[pos - 1] = cntg;
                }
            }
            __syncwarp();
            float4 pab = make_float4(0.f, 0.f, 0.f, 0.f);
            int pl = 0, pr = 0;
            if (total > 0) {
                const size_t src = (size_t)(sItem[0] & 0xffffff) * GROUP + lane;
                pab = ws.src32[src]; pl = ws.loc[src]; pr = ws.perm[src];
            }
            for (int q = 0; q < total; ++q) {
                const int cur = sItem[q], cntg = sItemCnt[q];
                sAB[buf][lane] = pab;
                sLoc[buf][lane] = pl;
                sRank[buf][lane] = pr;
                __syncwarp();
                int nt = -1;
                if (q + 1 < total) {  // the next group's loads are in flight during this one's arithmetic
                    const int ng = sItem[q + 1] & 0xffffff;
                    nt = ng / GPT;
                    const size_t src = (size_t)ng * GROUP + lane;
                    pab = ws.src32[src]; pl = ws.loc[src]; pr = ws.perm[src];
                }
                const int f = (cur >> 24) & 15;
                const int np = (cntg + 1) >> 1;
                const float4 *ab = sAB[buf];
                const int *lc = sLoc[buf], *rk = sRank[buf];
                if ((f & 3) == 3) {
                    if (f & 12) row_group<MODE, true, true, true>(ab, lc, rk, np, T, cbt2, nhh2, run);
                    else row_group<MODE, true, true, false>(ab, lc, rk, np, T, cbt2, nhh2, run);
                } else if (f & 1) {
                    if (f & 4) row_group<MODE, true, false, true>(ab, lc, rk, np, T, cbt2, nhh2, run);
                    else row_group<MODE, true, false, false>(ab, lc, rk, np, T, cbt2, nhh2, run);
                } else {
                    if (f & 8) row_group<MODE, false, true, true>(ab, lc, rk, np, T, cbt2, nhh2, run);
                    else row_group<MODE, false, true, false>(ab, lc, rk, np, T, cbt2, nhh2, run);
                }
                buf ^= 1;
                if (nt != (cur & 0xffffff) / GPT) {  // tile boundary: merge the runs
#pragma unroll
                    for (int k = 0; k < NMOM; ++k) {
                        if (mom_used(MODE, k)) {
                            kahan(ks[k], kc[k], __fadd_rn(run[k].x, run[k].y));
                            run[k] = make_float2(0.0f, 0.0f);
                        }
                    }
                }
            }
            __syncwarp();  // the items are read until here
        }
    }
#pragma unroll
    for (int k = 0; k < NMOM; ++k) {
        if (mom_used(MODE, k))
            // the Kahan pair (sum, -compensation), combined across chunks in float-float
            reinterpret_cast<float2 *>(ws.rowpart)[((size_t)chunk * NMOM + k) * npad + i] = make_float2(ks[k], -kc[k]);
    }
    // the unit of chunk rotation 0 also computes the group's integral-term shares (FP64)
    if (by == 0) integral_group(c, in, ws, tg);
}

// Persistent: a grid of as many one-warp blocks as fit on the GPU at once; each
// takes work units (target group, chunk rotation) from a counter in the call's
// header, in the order the launch grid dispatched them before (rotation-major:
// the heavy units first).  A unit's partials go to fixed places, so the result
// does not depend on which warp takes it (bit for bit the same as one block per
// unit), and taking a unit is one atomic add: no warp waits for another.
template <int MODE>
__global__ void __launch_bounds__(GROUP, 20) row32_st_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    const int nx = (c.t1 - c.t0) * GPT, total = nx * c.g.n_chunks;
    for (;;) {
        int u = 0;
        if (threadIdx.x == 0) u = atomicAdd(&ws.hdr[HDR_ST_ROW_UNITS], 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= total) break;
        row32_st_unit<MODE>(c, in, ws, u % nx, u / nx);
        __syncwarp();  // the unit's shared buffers are read until here
    }
}

template <int MODE>
static cudaError_t launch_row32_st_mode(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    const int units = (c.t1 - c.t0) * GPT * c.g.n_chunks;
    const int grid = min(units, resident_blocks(row32_st_kernel<MODE>, GROUP));
    if (grid < 1) return cudaErrorInvalidConfiguration;
    launch_pdl(row32_st_kernel<MODE>, grid, GROUP, 0, s, c, in, ws);
    return cudaGetLastError();
}

cudaError_t launch_row32_st(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    if (c.mode == MODE_HESS) return launch_row32_st_mode<MODE_HESS>(c, in, ws, s);
    if (c.mode == MODE_GRAD) return launch_row32_st_mode<MODE_GRAD>(c, in, ws, s);
    return launch_row32_st_mode<MODE_LL>(c, in, ws, s);
}

}  // namespace hk
