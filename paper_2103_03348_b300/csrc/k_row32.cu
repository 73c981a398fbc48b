// FP32-compensated row and column passes (Eq. 1's inner sum; Eqs. 4-5).
//
// Row pass (Algorithm 2, step 1, redesigned): one block of 128 threads owns a
// tile of 128 time-consecutive targets, one target per thread, and sweeps a
// chunk of source tiles.  Each source tile (128 events, 2 KB) is staged in
// shared memory and read back as broadcast float4 pairs, so one packed f32x2
// instruction evaluates a target against two sources.  With scaled, centred
// coordinates (x~ = (x - xc) sqrt(log2(e)/2)/tau_x, t~ = (t - tc) omega log2(e))
// the pair terms are
//     G = 2^-(d~^2 + cbt dt~^2)                      background (Section 2.1)
//     E = 2^(r^_s - t~_n - hh d~^2),  r^ = r~ + t~    excitation with theta_s = e^r
// and the row accumulates the moments listed in hawkes_internal.cuh.
// Precision: per-thread runs of 64 source pairs in plain FP32 (packed, two
// lanes), merged after every tile into a Kahan-compensated FP32 sum per
// moment; the chunk result is written in FP64 and chunks are combined in FP64.
//
// With band skipping (HAWKES_FP32C_BAND) a tile pair whose time gap g has
// cbt g^2 > 130 has every background term below 2^-130, exactly 0 in FP32, and
// its background work is skipped; results are unchanged bit for bit.
//
// Every source tile is classified for the whole block (no divergence):
//   * excitation skipped when no source precedes any target (exact, by the
//     tie-group index) or when 2^(max r^ - min t~) is below 2^-128, so every
//     excitation term would underflow to exactly 0 in FP32;
//   * masks (causal by tie-group index, background by exact-location group)
//     only where a tile pair can contain a masked pair: the diagonal tile,
//     tiles that straddle the causal boundary, and tiles that both hold events
//     with a duplicated location.
#include "hawkes_internal.cuh"

namespace hk {

__host__ __device__ constexpr bool mom_used(int mode, int k) {
    return mode == MODE_HESS ? true
         : mode == MODE_GRAD ? (k == MO_G || k == MO_GD2 || k == MO_GT2 || k == MO_E || k == MO_ET || k == MO_ED2)
                             : (k == MO_G || k == MO_E);
}

struct RowTarget {
    float2 xn, yn, tn, ntn;  // splatted target coordinates (ntn = -t~_n)
    int locn, gn;
};

// ra, rb: time-order indices of the two sources (their positions, except in FP32C_ST)
template <int MODE, bool BG, bool EXC, bool MASK>
__device__ __forceinline__ void row_pair(const float4 A, const float4 B, int la, int lb, int ra, int rb,
                                         const RowTarget &T, float2 cbt2, float2 nhh2, float2 (&run)[NMOM]) {
    // A = (-x0, -x1, -y0, -y1), B = (-t0, -t1, r^0, r^1)
    const float2 dx = add2(T.xn, make_float2(A.x, A.y));
    const float2 dy = add2(T.yn, make_float2(A.z, A.w));
    const float2 dt = add2(T.tn, make_float2(B.x, B.y));
    float2 d2 = mul2(dx, dx);
    d2 = fma2(dy, dy, d2);
    const float2 dt2 = mul2(dt, dt);
    float2 d4 = make_float2(0.0f, 0.0f);
    if (MODE == MODE_HESS) d4 = mul2(d2, d2);
    if (BG) {
        const float2 q = fma2(dt2, cbt2, d2);
        float2 gb = make_float2(ex2_ftz(-q.x), ex2_ftz(-q.y));
        if (MASK) {
            if (la == T.locn) gb.x = 0.0f;
            if (lb == T.locn) gb.y = 0.0f;
        }
        run[MO_G] = add2(run[MO_G], gb);
        if (MODE >= MODE_GRAD) {
            run[MO_GD2] = fma2(gb, d2, run[MO_GD2]);
            run[MO_GT2] = fma2(gb, dt2, run[MO_GT2]);
        }
        if (MODE == MODE_HESS) {
            const float2 dt4 = mul2(dt2, dt2);
            run[MO_GD4] = fma2(gb, d4, run[MO_GD4]);
            run[MO_GT4] = fma2(gb, dt4, run[MO_GT4]);
        }
    }
    if (EXC) {
        float2 ee = add2(make_float2(B.z, B.w), T.ntn);
        ee = fma2(d2, nhh2, ee);
        float2 e = make_float2(ex2_ftz(ee.x), ex2_ftz(ee.y));
        if (MASK) {
            if (!(ra < T.gn)) e.x = 0.0f;
            if (!(rb < T.gn)) e.y = 0.0f;
        }
        run[MO_E] = add2(run[MO_E], e);
        if (MODE >= MODE_GRAD) {
            run[MO_ET] = fma2(e, dt, run[MO_ET]);
            run[MO_ED2] = fma2(e, d2, run[MO_ED2]);
        }
        if (MODE == MODE_HESS) {
            run[MO_ET2] = fma2(e, dt2, run[MO_ET2]);
            run[MO_ED4] = fma2(e, d4, run[MO_ED4]);
        }
    }
}

template <int MODE, bool BG, bool EXC, bool MASK>
__device__ __forceinline__ void row_tile(const float4 *sAB, const int *sLoc, int s0, int npairs,
                                         const RowTarget &T, float2 cbt2, float2 nhh2, float2 (&run)[NMOM]) {
#pragma unroll 4
    for (int p = 0; p < npairs; ++p) {
        const float4 A = sAB[2 * p], B = sAB[2 * p + 1];
        int la = 0, lb = 0;
        if (MASK && BG) { la = sLoc[2 * p]; lb = sLoc[2 * p + 1]; }
        row_pair<MODE, BG, EXC, MASK>(A, B, la, lb, s0 + 2 * p, s0 + 2 * p + 1, T, cbt2, nhh2, run);
    }
}

// FP32C_ST: one group of up to 32 sources, with their time-order ranks for the causal mask.
template <int MODE, bool BG, bool EXC, bool MASK>
__device__ __forceinline__ void row_group(const float4 *sAB, const int *sLoc, const int *sRank, int npairs,
                                          const RowTarget &T, float2 cbt2, float2 nhh2, float2 (&run)[NMOM]) {
#pragma unroll 4
    for (int p = 0; p < npairs; ++p) {
        const float4 A = sAB[2 * p], B = sAB[2 * p + 1];
        int la = 0, lb = 0, ra = 0, rb = 0;
        if (MASK && BG) { la = sLoc[2 * p]; lb = sLoc[2 * p + 1]; }
        if (MASK && EXC) { ra = sRank[2 * p]; rb = sRank[2 * p + 1]; }
        row_pair<MODE, BG, EXC, MASK>(A, B, la, lb, ra, rb, T, cbt2, nhh2, run);
    }
}

template <int MODE, bool BAND>
__global__ void __launch_bounds__(TILE, 4) row32_kernel(Consts c, Workspace ws) {
    const Derived &D = *c.d;
    // Chunk order: blocks are dispatched y-major, so y = 0 takes the chunk that
    // holds the tile itself, y = 1 the chunk before it, and so on, wrapping to
    // the later (future, background-only) chunks last: the heavy blocks go
    // first and the light ones fill the tail.
    const int tile = c.t0 + blockIdx.x;
    const int chunk = (tile / c.g.chunk_tiles - (int)blockIdx.y + c.g.n_chunks) % c.g.n_chunks;
    const int i = tile * TILE + threadIdx.x;
    const int npad = c.g.npad;
    __shared__ float4 sAB[2][TILE];
    __shared__ int sLoc[2][TILE];

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
    const float4 stT = ws.tstat32[tile];
    const float2 cbt2 = splat(D.cbt), nhh2 = splat(-D.hh);

    float2 run[NMOM];
    float ks[NMOM], kc[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) { run[k] = make_float2(0.0f, 0.0f); ks[k] = 0.0f; kc[k] = 0.0f; }

    const int sb = chunk * c.g.chunk_tiles;
    const int se = min(c.g.tiles, sb + c.g.chunk_tiles);
    // register prefetch of the first source tile
    float4 pf = make_float4(0.f, 0.f, 0.f, 0.f);
    int pl = 0;
    if (sb < se) { pf = ws.src32[(size_t)sb * TILE + threadIdx.x]; pl = ws.loc[(size_t)sb * TILE + threadIdx.x]; }
    int buf = 0;
    for (int s = sb; s < se; ++s) {
        sAB[buf][threadIdx.x] = pf;
        sLoc[buf][threadIdx.x] = pl;
        __syncthreads();
        if (s + 1 < se) {
            pf = ws.src32[(size_t)(s + 1) * TILE + threadIdx.x];
            pl = ws.loc[(size_t)(s + 1) * TILE + threadIdx.x];
        }
        const int4 tiS = ws.tinfo[s];
        const float4 stS = ws.tstat32[s];
        const int s0 = s * TILE;
        const int npairs = (tiS.w + 1) >> 1;
        const bool none_causal = s0 >= tiT.y;                // no source precedes any target
        const bool all_causal = s0 + tiS.w - 1 < tiT.x;      // every source precedes every target
        const bool exc = !none_causal && (stS.z - stT.x >= EXP2_DEAD);
        bool bg = true;
        if (BAND) {
            // every background term of the tile pair is below 2^-130 when the time gap is wide enough
            const float gap = fmaxf(fmaxf(stS.x - stT.y, stT.x - stS.y), 0.0f);
            bg = !(D.cbt * gap * gap > BG_DEAD);
        }
        if (bg) {
            const bool mask = (s == tile) || (tiT.z && tiS.z) || (exc && !all_causal);
            if (exc) {
                if (mask) row_tile<MODE, true, true, true>(sAB[buf], sLoc[buf], s0, npairs, T, cbt2, nhh2, run);
                else row_tile<MODE, true, true, false>(sAB[buf], sLoc[buf], s0, npairs, T, cbt2, nhh2, run);
            } else {
                if (mask) row_tile<MODE, true, false, true>(sAB[buf], sLoc[buf], s0, npairs, T, cbt2, nhh2, run);
                else row_tile<MODE, true, false, false>(sAB[buf], sLoc[buf], s0, npairs, T, cbt2, nhh2, run);
            }
        } else if (exc) {
            if (!all_causal) row_tile<MODE, false, true, true>(sAB[buf], sLoc[buf], s0, npairs, T, cbt2, nhh2, run);
            else row_tile<MODE, false, true, false>(sAB[buf], sLoc[buf], s0, npairs, T, cbt2, nhh2, run);
        }
        // merge the tile's run into the compensated sums
#pragma unroll
        for (int k = 0; k < NMOM; ++k) {
            if (mom_used(MODE, k)) {
                kahan(ks[k], kc[k], __fadd_rn(run[k].x, run[k].y));
                run[k] = make_float2(0.0f, 0.0f);
            }
        }
        buf ^= 1;
    }
#pragma unroll
    for (int k = 0; k < NMOM; ++k) {
        if (mom_used(MODE, k))
            ws.rowpart[((size_t)chunk * NMOM + k) * npad + i] = (double)ks[k] - (double)kc[k];
    }
}

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

template <int MODE>
__global__ void __launch_bounds__(TILE, 4) row32_st_kernel(Consts c, Workspace ws) {
    const Derived &D = *c.d;
    const int tile = c.t0 + blockIdx.x;
    const int chunk = (tile / c.g.chunk_tiles - (int)blockIdx.y + c.g.n_chunks) % c.g.n_chunks;
    const int i = tile * TILE + threadIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int npad = c.g.npad;
    __shared__ float4 sAB[2][TILE];
    __shared__ int sLoc[2][TILE];
    __shared__ int sRank[2][TILE];
    __shared__ GroupStat sGS[2][GPT];
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
        for (int q = 0; q < total; ++q) {
            const int su = sList[q], fl = sFlag[q];
            const size_t s0 = (size_t)su * TILE;
            sAB[buf][threadIdx.x] = ws.src32[s0 + threadIdx.x];
            sLoc[buf][threadIdx.x] = ws.loc[s0 + threadIdx.x];
            sRank[buf][threadIdx.x] = ws.perm[s0 + threadIdx.x];
            if (threadIdx.x < GPT) sGS[buf][threadIdx.x] = ws.grp[(size_t)su * GPT + threadIdx.x];
            __syncthreads();
            const int4 tiS = ws.tinfo[su];
            const bool dup = tiT.z && tiS.z;
#pragma unroll 1
            for (int g = 0; g < GPT; ++g) {
                const int cntg = min(max(tiS.w - g * GROUP, 0), GROUP);
                if (cntg == 0) continue;
                const GroupStat S = sGS[buf][g];
                // warp-uniform decisions for this warp's 32 targets
                const bool bgw = (fl & 1) && bg_alive(W, S, cbt);
                const bool exw = (fl & 2) && exc_alive(W, S, hh);
                if (!bgw && !exw) continue;
                const int np = (cntg + 1) >> 1;
                const float4 *ab = sAB[buf] + g * GROUP;
                const int *lc = sLoc[buf] + g * GROUP;
                const int *rk = sRank[buf] + g * GROUP;
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
            buf ^= 1;
        }
        __syncthreads();  // the list is read until here
    }
#pragma unroll
    for (int k = 0; k < NMOM; ++k) {
        if (mom_used(MODE, k))
            ws.rowpart[((size_t)chunk * NMOM + k) * npad + i] = (double)ks[k] - (double)kc[k];
    }
}

cudaError_t launch_row32(const Consts &c, const Workspace &ws, cudaStream_t s) {
    const dim3 grid(c.t1 - c.t0, c.g.n_chunks);
    if (c.st) {
        if (c.mode == MODE_HESS) row32_st_kernel<MODE_HESS><<<grid, TILE, 0, s>>>(c, ws);
        else if (c.mode == MODE_GRAD) row32_st_kernel<MODE_GRAD><<<grid, TILE, 0, s>>>(c, ws);
        else row32_st_kernel<MODE_LL><<<grid, TILE, 0, s>>>(c, ws);
    } else if (c.band) {
        if (c.mode == MODE_HESS) row32_kernel<MODE_HESS, true><<<grid, TILE, 0, s>>>(c, ws);
        else if (c.mode == MODE_GRAD) row32_kernel<MODE_GRAD, true><<<grid, TILE, 0, s>>>(c, ws);
        else row32_kernel<MODE_LL, true><<<grid, TILE, 0, s>>>(c, ws);
    } else {
        if (c.mode == MODE_HESS) row32_kernel<MODE_HESS, false><<<grid, TILE, 0, s>>>(c, ws);
        else if (c.mode == MODE_GRAD) row32_kernel<MODE_GRAD, false><<<grid, TILE, 0, s>>>(c, ws);
        else row32_kernel<MODE_LL, false><<<grid, TILE, 0, s>>>(c, ws);
    }
    return cudaGetLastError();
}

}  // namespace hk
