// FP32C_ST row pass (space-time tiles): see row32_st_kernel below; the pair
// arithmetic is that of the time-order row pass (row32_pair.cuh).
#include "row32_pair.cuh"
#include "rows_finish.cuh"

namespace hk {

// FP32C_ST row pass.  Positions hold events permuted inside slabs so that
// each group of 32 positions is compact in space and time.  One block is one
// warp and owns one target group (32 rows) for one chunk of source tiles, so
// no warp ever waits for another:
//   * classify: lane l tests source tile base + l group by group against the
//     warp's own target group (background live, excitation live, all sources
//     causal), and the tiles with a live group are listed in order;
//   * sweep: for each listed tile, each live source group (32 sources) is
//     staged in the warp's shared buffer (double-buffered, one __syncwarp)
//     and evaluated with the pair arithmetic, masks and compensation of
//     row32_kernel; the causal mask compares time-order ranks.
constexpr int GPT = TILE / GROUP;  // groups per tile

template <int MODE>
__global__ void __launch_bounds__(GROUP, 16) row32_st_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    const Derived &D = *c.d;
    const int tg = c.t0 * GPT + blockIdx.x;  // target group
    const int tile = tg / GPT, gw = tg % GPT;
    const int chunk = (tile / c.g.chunk_tiles - (int)blockIdx.y + c.g.n_chunks) % c.g.n_chunks;
    const int lane = threadIdx.x;
    const int i = tg * GROUP + lane;
    const int npad = c.g.npad;
    __shared__ int sList[GROUP];
    __shared__ int sInfo[GROUP];  // per listed tile: bits 0-3 background live, 4-7 excitation live,
                                  // 8-11 every source precedes every target, 12 duplicates, 13+ count
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
            // classify tiles base .. base + 31 against this warp's targets
            const int s = base + lane;
            int info = 0;
            if (s < se) {
                const int4 tiS = ws.tinfo[s];
#pragma unroll
                for (int g = 0; g < GPT; ++g) {
                    const GroupStat S = ws.grp[(size_t)s * GPT + g];
                    if (group_empty(S)) continue;
                    if (bg_alive(W, S, cbt)) info |= 1 << g;
                    if (exc_alive(W, S, hh)) info |= 16 << g;
                    if (S.ix.w < W.ix.x) info |= 256 << g;
                }
                if (info & 0xff) info |= (tiS.z ? 4096 : 0) | (tiS.w << 13);
                else info = 0;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, info != 0);
            if (info) sList[__popc(bal & ((1u << lane) - 1u))] = s;
            if (info) sInfo[__popc(bal & ((1u << lane) - 1u))] = info;
            __syncwarp();
            const int total = __popc(bal);
            for (int q = 0; q < total; ++q) {
                const int su = sList[q], inf = sInfo[q];
                const int cnt = inf >> 13;
                const bool dup = dupT && (inf & 4096);
#pragma unroll 1
                for (int g = 0; g < GPT; ++g) {
                    const bool bgw = (inf >> g) & 1, exw = (inf >> (4 + g)) & 1;
                    const int cntg = min(max(cnt - g * GROUP, 0), GROUP);
                    if ((!bgw && !exw) || cntg == 0) continue;
                    const size_t src = (size_t)su * TILE + g * GROUP + lane;
                    sAB[buf][lane] = ws.src32[src];
                    sLoc[buf][lane] = ws.loc[src];
                    sRank[buf][lane] = ws.perm[src];
                    __syncwarp();
                    const int np = (cntg + 1) >> 1;
                    const bool mask_bg = (su == tile && g == gw) || dup;
                    const bool mask_ex = exw && !((inf >> (8 + g)) & 1);
                    const float4 *ab = sAB[buf];
                    const int *lc = sLoc[buf], *rk = sRank[buf];
                    if (bgw && exw) {
                        if (mask_bg || mask_ex) row_group<MODE, true, true, true>(ab, lc, rk, np, T, cbt2, nhh2, run);
                        else row_group<MODE, true, true, false>(ab, lc, rk, np, T, cbt2, nhh2, run);
                    } else if (bgw) {
                        if (mask_bg) row_group<MODE, true, false, true>(ab, lc, rk, np, T, cbt2, nhh2, run);
                        else row_group<MODE, true, false, false>(ab, lc, rk, np, T, cbt2, nhh2, run);
                    } else {
                        if (mask_ex) row_group<MODE, false, true, true>(ab, lc, rk, np, T, cbt2, nhh2, run);
                        else row_group<MODE, false, true, false>(ab, lc, rk, np, T, cbt2, nhh2, run);
                    }
                    buf ^= 1;
                }
#pragma unroll
                for (int k = 0; k < NMOM; ++k) {
                    if (mom_used(MODE, k)) {
                        kahan(ks[k], kc[k], __fadd_rn(run[k].x, run[k].y));
                        run[k] = make_float2(0.0f, 0.0f);
                    }
                }
            }
            __syncwarp();  // the list is read until here
        }
    }
#pragma unroll
    for (int k = 0; k < NMOM; ++k) {
        if (mom_used(MODE, k))
            // the Kahan pair (sum, -compensation), combined across chunks in float-float
            reinterpret_cast<float2 *>(ws.rowpart)[((size_t)chunk * NMOM + k) * npad + i] = make_float2(ks[k], -kc[k]);
    }
    // one block per target group also computes the group's integral-term shares (FP64)
    if (blockIdx.y == 0) integral_group(c, in, ws, tg);
}

cudaError_t launch_row32_st(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    const dim3 grid((c.t1 - c.t0) * GPT, c.g.n_chunks);
    if (c.mode == MODE_HESS) launch_pdl(row32_st_kernel<MODE_HESS>, grid, GROUP, 0, s, c, in, ws);
    else if (c.mode == MODE_GRAD) launch_pdl(row32_st_kernel<MODE_GRAD>, grid, GROUP, 0, s, c, in, ws);
    else launch_pdl(row32_st_kernel<MODE_LL>, grid, GROUP, 0, s, c, in, ws);
    return cudaGetLastError();
}

}  // namespace hk
