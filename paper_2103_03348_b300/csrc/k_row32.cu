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
#include "row32_pair.cuh"
#include "rows_finish.cuh"

namespace hk {

template <int MODE, bool BAND>
__global__ void __launch_bounds__(TILE, 5) row32_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
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
            // the Kahan pair (sum, -compensation), combined across chunks in float-float
            reinterpret_cast<float2 *>(ws.rowpart)[((size_t)chunk * NMOM + k) * npad + i] = make_float2(ks[k], -kc[k]);
    }
    // one block per tile also computes the tile's integral-term shares (FP64), warp by warp
    if (blockIdx.y == 0) integral_group(c, in, ws, i / GROUP);
}

cudaError_t launch_row32(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    const dim3 grid(c.t1 - c.t0, c.g.n_chunks);
    if (c.st) return launch_row32_st(c, in, ws, s);
    if (c.band) {
        if (c.mode == MODE_HESS) launch_pdl(row32_kernel<MODE_HESS, true>, grid, TILE, 0, s, c, in, ws);
        else if (c.mode == MODE_GRAD) launch_pdl(row32_kernel<MODE_GRAD, true>, grid, TILE, 0, s, c, in, ws);
        else launch_pdl(row32_kernel<MODE_LL, true>, grid, TILE, 0, s, c, in, ws);
    } else {
        if (c.mode == MODE_HESS) launch_pdl(row32_kernel<MODE_HESS, false>, grid, TILE, 0, s, c, in, ws);
        else if (c.mode == MODE_GRAD) launch_pdl(row32_kernel<MODE_GRAD, false>, grid, TILE, 0, s, c, in, ws);
        else launch_pdl(row32_kernel<MODE_LL, false>, grid, TILE, 0, s, c, in, ws);
    }
    return cudaGetLastError();
}

}  // namespace hk
