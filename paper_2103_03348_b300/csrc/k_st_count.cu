// Work count of the FP32C_ST passes, for the roofline of the path the sampler
// runs: the ordered (target, source) pairs inside the group pairs that the
// space-time row pass evaluates (background live, excitation live) and the
// (source, target) pairs inside the group pairs that its column pass
// evaluates.  The classification is the passes' own (bg_alive, exc_alive,
// col_alive on the group records of the workspace), so the counts are exactly
// the pairs those kernels run their pair arithmetic on.  Measurement only: the
// evaluation's results do not depend on it.
#include <string.h>

#include "hawkes_internal.cuh"

namespace hk {

constexpr int CGROUPS = TILE / GROUP;  // groups per tile
constexpr int COUNT_THREADS = 256;

__device__ __forceinline__ int group_count(int tile_count, int g) {
    return max(0, min(tile_count - g * GROUP, GROUP));
}

// One warp per group W: as targets against every source tile (row pass), and
// as sources against every target tile from its slab's first tile on (column
// pass).  counts[0] background-live pairs, [1] excitation-live pairs, [2]
// column pairs.
__global__ void __launch_bounds__(COUNT_THREADS) st_live_pairs_kernel(Consts c, Workspace ws,
                                                                      unsigned long long *__restrict__ counts) {
    const Derived &D = *c.d;
    const int wg = (int)((blockIdx.x * (unsigned)COUNT_THREADS + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (wg >= c.g.tiles * CGROUPS) return;  // warp-uniform
    const int tile = wg / CGROUPS;
    const int cw = group_count(ws.tinfo[tile].w, wg % CGROUPS);
    const GroupStat W = ws.grp[wg];
    unsigned long long bg = 0, ex = 0, col = 0;
    if (cw > 0 && !group_empty(W)) {
        for (int s = lane; s < c.g.tiles; s += GROUP) {
            const int cnt = ws.tinfo[s].w;
            for (int g = 0; g < CGROUPS; ++g) {
                const GroupStat S = ws.grp[(size_t)s * CGROUPS + g];
                if (cnt <= g * GROUP || group_empty(S)) continue;
                const unsigned long long p = (unsigned long long)cw * group_count(cnt, g);
                if (bg_alive(W, S, D.cbt)) bg += p;
                if (exc_alive(W, S, D.hh)) ex += p;
            }
        }
        const int start = (tile / SLAB_TILES) * SLAB_TILES;
        for (int u = start + lane; u < c.g.tiles; u += GROUP) {
            if (ws.sufmax[u] + W.tr.z < EXP2_DEAD) continue;
            const int cnt = ws.tinfo[u].w;
            for (int g = 0; g < CGROUPS; ++g) {
                const GroupStat G = ws.grp[(size_t)u * CGROUPS + g];
                if (group_empty(G) || cnt <= g * GROUP || !col_alive(W, G, D.hh)) continue;
                col += (unsigned long long)cw * group_count(cnt, g);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bg += __shfl_down_sync(0xffffffffu, bg, o);
        ex += __shfl_down_sync(0xffffffffu, ex, o);
        col += __shfl_down_sync(0xffffffffu, col, o);
    }
    if (lane == 0) {
        atomicAdd(&counts[0], bg);
        atomicAdd(&counts[1], ex);
        atomicAdd(&counts[2], col);
    }
}

}  // namespace hk

extern "C" int hawkes_st_live_pairs(int64_t n, void *ws, size_t ws_bytes, unsigned long long *counts, void *stream) {
    if (n < 2 || n > HAWKES_MAX_EVENTS || !ws || !counts || ((uintptr_t)ws & 255) != 0) return HAWKES_EINVAL;
    const hk::Geometry g = hk::make_geometry(n);
    hk::Workspace w;
    if (ws_bytes < hk::carve(ws, g, HAWKES_FP32C_ST, &w)) return HAWKES_EWORKSPACE;
    hk::Consts c;
    memset(&c, 0, sizeof(c));
    c.g = g;
    c.fp32c = 1;
    c.st = true;
    c.t0 = 0;
    c.t1 = g.tiles;
    c.d = w.derived;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned long long), s) != cudaSuccess) return HAWKES_ECUDA;
    const int64_t threads = (int64_t)g.tiles * hk::CGROUPS * 32;
    const unsigned blocks = (unsigned)((threads + hk::COUNT_THREADS - 1) / hk::COUNT_THREADS);
    hk::st_live_pairs_kernel<<<blocks, hk::COUNT_THREADS, 0, s>>>(c, w, counts);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}
