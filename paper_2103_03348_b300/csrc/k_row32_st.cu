// FP32C_ST row pass (space-time tiles): see row32_st_kernel below; the pair
// arithmetic is that of the time-order row pass (row32_pair.cuh).
#include "row32_pair.cuh"
#include "rows_finish.cuh"

namespace hk {

// FP32C_ST row pass.  Positions hold events permuted inside slabs so that a
// tile (and each of its four warps' groups of 32) is compact in space and
// time.  Per source chunk, the block first classifies up to 128 source tiles
// at once (one per thread) against the union of its four target groups and
// lists, in order, those with a live background or excitation term; it then
// sweeps the listed tiles through shared memory, and each warp skips the
// source groups whose terms all underflow for its own 32 targets (bounds from
// the group statistics).  Pair arithmetic, masks and compensation are those
// of row32_kernel; the causal mask compares time-order ranks.
constexpr int GPT = TILE / GROUP;  // groups per tile
constexpr int STAGE = 4;           // listed source tiles staged per barrier

template <int MODE>
__global__ void __launch_bounds__(TILE, 4) row32_st_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    const Derived &D = *c.d;
    const int tile = c.t0 + blockIdx.x;
    const int chunk = (tile / c.g.chunk_tiles - (int)blockIdx.y + c.g.n_chunks) % c.g.n_chunks;
    const int i = tile * TILE + threadIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int npad = c.g.npad;
    // STAGE listed tiles per barrier (double-buffered), so that the warps' unequal
    // numbers of live groups even out over more work between barriers
    __shared__ float4 sAB[2][STAGE][TILE];
    __shared__ int sLoc[2][STAGE][TILE];
    __shared__ int sRank[2][STAGE][TILE];
    __shared__ GroupStat sGS[2][STAGE][GPT];
    __shared__ int sList[TILE];
    __shared__ int sFlag[TILE];
    __shared__ int sCnt[GPT];

    RowTarget T;
    {
        const float *f = reinterpret_cast<const float *>(ws.src32);
        const int p = i >> 1, l = i & 1;
        const float x = -f[8 * p + 0 + l], y = -f[8 * p + 2 + l], t = -f[8 * p + 4 + l];
        T.xn = splat(x); T.yn = splat(y); T.tn = splat(t); T.ntn = splat(-t);
        T.locn = ws.loc[i];
        T.gn = ws.gidx[i];
    }
    const int4 tiT = ws.tinfo[tile];
    const GroupStat W = ws.grp[tile * GPT + warp];
    GroupStat U = ws.grp[tile * GPT];
#pragma unroll
    for (int g = 1; g < GPT; ++g) U = group_union(U, ws.grp[tile * GPT + g]);
    const float cbt = D.cbt, hh = D.hh;
    const float2 cbt2 = splat(cbt), nhh2 = splat(-hh);

    float2 run[NMOM];
    float ks[NMOM], kc[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) { run[k] = make_float2(0.0f, 0.0f); ks[k] = 0.0f; kc[k] = 0.0f; }

    const int sb = chunk * c.g.chunk_tiles;
    const int se = min(c.g.tiles, sb + c.g.chunk_tiles);
    int buf = 0;
    for (int base = sb; base < se; base += TILE) {
        // classify tiles base .. base + 127 (bit 0: background live, bit 1: excitation live)
        const int s = base + threadIdx.x;
        int flag = 0;
        if (s < se) {
#pragma unroll
            for (int g = 0; g < GPT; ++g) {
                const GroupStat S = ws.grp[(size_t)s * GPT + g];
                if (group_empty(S)) continue;
                if (bg_alive(U, S, cbt)) flag |= 1;
                if (exc_alive(U, S, hh)) flag |= 2;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, flag != 0);
        if (lane == 0) sCnt[warp] = __popc(bal);
        __syncthreads();
        int off = 0, total = 0;
#pragma unroll
        for (int w = 0; w < GPT; ++w) {
            if (w < warp) off += sCnt[w];
            total += sCnt[w];
        }
        if (flag) {
            const int pos = off + __popc(bal & ((1u << lane) - 1u));
            sList[pos] = s;
            sFlag[pos] = flag;
        }
        __syncthreads();
        for (int q0 = 0; q0 < total; q0 += STAGE) {
            const int nst = min(STAGE, total - q0);
#pragma unroll
            for (int kk = 0; kk < STAGE; ++kk) {
                if (kk < nst) {
                    const int su = sList[q0 + kk];
                    const size_t s0 = (size_t)su * TILE;
                    sAB[buf][kk][threadIdx.x] = ws.src32[s0 + threadIdx.x];
                    sLoc[buf][kk][threadIdx.x] = ws.loc[s0 + threadIdx.x];
                    sRank[buf][kk][threadIdx.x] = ws.perm[s0 + threadIdx.x];
                    if (threadIdx.x < GPT) sGS[buf][kk][threadIdx.x] = ws.grp[(size_t)su * GPT + threadIdx.x];
                }
            }
            __syncthreads();
#pragma unroll 1
            for (int kk = 0; kk < nst; ++kk) {
            const int su = sList[q0 + kk], fl = sFlag[q0 + kk];
            const int4 tiS = ws.tinfo[su];
            const bool dup = tiT.z && tiS.z;
#pragma unroll 1
            for (int g = 0; g < GPT; ++g) {
                const int cntg = min(max(tiS.w - g * GROUP, 0), GROUP);
                if (cntg == 0) continue;
                const GroupStat S = sGS[buf][kk][g];
                // warp-uniform decisions for this warp's 32 targets
                const bool bgw = (fl & 1) && bg_alive(W, S, cbt);
                const bool exw = (fl & 2) && exc_alive(W, S, hh);
                if (!bgw && !exw) continue;
                const int np = (cntg + 1) >> 1;
                const float4 *ab = sAB[buf][kk] + g * GROUP;
                const int *lc = sLoc[buf][kk] + g * GROUP;
                const int *rk = sRank[buf][kk] + g * GROUP;
                const bool mask_bg = (su == tile && g == warp) || dup;
                const bool mask_ex = exw && !(S.ix.w < W.ix.x);
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
            }
#pragma unroll
            for (int k = 0; k < NMOM; ++k) {
                if (mom_used(MODE, k)) {
                    kahan(ks[k], kc[k], __fadd_rn(run[k].x, run[k].y));
                    run[k] = make_float2(0.0f, 0.0f);
                }
            }
            }
            buf ^= 1;
        }
        __syncthreads();  // the list is read until here
    }
#pragma unroll
    for (int k = 0; k < NMOM; ++k) {
        if (mom_used(MODE, k))
            // the Kahan pair (sum, -compensation), combined across chunks in float-float
            reinterpret_cast<float2 *>(ws.rowpart)[((size_t)chunk * NMOM + k) * npad + i] = make_float2(ks[k], -kc[k]);
    }
    // one block per tile also computes the tile's integral-term shares (FP64)
    if (blockIdx.y == 0) integral_tile(c, in, ws, tile);
}

cudaError_t launch_row32_st(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    const dim3 grid(c.t1 - c.t0, c.g.n_chunks);
    if (c.mode == MODE_HESS) launch_pdl(row32_st_kernel<MODE_HESS>, grid, TILE, 0, s, c, in, ws);
    else if (c.mode == MODE_GRAD) launch_pdl(row32_st_kernel<MODE_GRAD>, grid, TILE, 0, s, c, in, ws);
    else launch_pdl(row32_st_kernel<MODE_LL>, grid, TILE, 0, s, c, in, ws);
    return cudaGetLastError();
}

}  // namespace hk
