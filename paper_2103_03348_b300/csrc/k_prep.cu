// Step a1 of the hot path: validation and packing of the time-sorted events.
//
// prep (one block per tile of 128 events):
//   * status bits for non-finite inputs and for t not ascending;
//   * gidx[i] = first index whose time equals t_i (binary search over [0, i]),
//     so that "t_s < t_n" (strict excitation, Section 2.1) becomes s < gidx[n];
//   * exact-location groups (background indicator I[x_n != x_n'], Section 2.1)
//     by open-addressing insertion of the FP64 (x, y) key: loc[i] is the group
//     representative and cnt[rep] the group size;
//   * per-tile x/y bounds; the last block to finish (atomic ticket, no waiting)
//     reduces them in fixed order to the centre used by the FP32 coordinates.
// pack (one block per tile):
//   * FP32C: scaled, centred FP32 sources stored as pairs for f32x2 arithmetic,
//     ((-x0,-x1,-y0,-y1),(-t0,-t1,r^0,r^1)) with r^ = r~ + t~, and per-tile
//     statistics;
//   * FP64: (x, y, t, r) as double4_32a;
//   * per-tile first/last tie-group start and duplicate-location flag.
#include "hawkes_internal.cuh"

namespace hk {

__device__ __forceinline__ uint64_t mix64(uint64_t k) {
    // splitmix64 finaliser
    k ^= k >> 30;
    k *= 0xbf58476d1ce4e5b9ULL;
    k ^= k >> 27;
    k *= 0x94d049bb133111ebULL;
    k ^= k >> 31;
    return k;
}

__global__ void __launch_bounds__(TILE) prep_kernel(Consts c, Inputs in, Workspace ws) {
    const int n = c.g.n;
    const int i = blockIdx.x * TILE + threadIdx.x;
    __shared__ double sh[TILE];
    __shared__ bool last;
    int bad = 0;
    double xi = 0.0, yi = 0.0;
    const bool valid = i < n;
    if (valid) {
        xi = in.x[i];
        yi = in.y[i];
        const double ti = in.t[i];
        if (!isfinite(xi) || !isfinite(yi) || !isfinite(ti)) bad |= ST_NONFINITE;  // r: checked by pack
        if (i > 0 && !(in.t[i - 1] <= ti)) bad |= ST_UNSORTED;
        // tie-group start: first index j <= i with t_j == t_i (lower bound on a sorted prefix)
        int lo = 0, hi = i;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (in.t[mid] < ti) lo = mid + 1; else hi = mid;
        }
        ws.gidx[i] = lo;
        // exact-location group: -0.0 and +0.0 are the same location
        const double kx = xi + 0.0, ky = yi + 0.0;
        const uint64_t hk = mix64((uint64_t)__double_as_longlong(kx) ^ mix64((uint64_t)__double_as_longlong(ky) + 0x9e3779b97f4a7c15ULL));
        const int mask = c.g.hash_size - 1;
        int slot = (int)(hk & (uint64_t)mask);
        int rep = i;
        for (int probe = 0; probe < c.g.hash_size; ++probe) {
            const int prev = atomicCAS(&ws.hash[slot], -1, i);
            if (prev == -1) { rep = i; break; }
            if (in.x[prev] + 0.0 == kx && in.y[prev] + 0.0 == ky) { rep = prev; break; }
            slot = (slot + 1) & mask;
        }
        ws.loc[i] = rep;
        atomicAdd(&ws.cnt[rep], 1);
    } else if (i < c.g.npad) {
        ws.gidx[i] = n;      // padding: never a causal source, never a target
        ws.loc[i] = -1 - i;  // padding: a location of its own
    }
    if (bad) {
        atomicOr(&ws.hdr[0], bad);
        atomicOr(&ws.hdr[3], bad);  // kept for calls that reuse these events
    }

    // per-tile bounds of x and y (valid events only)
    double4_32a box;
    {
        double v = valid ? xi : INFINITY;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int w = TILE / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + w]);
            __syncthreads();
        }
        box.x = sh[0];
        __syncthreads();
        v = valid ? xi : -INFINITY;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int w = TILE / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
            __syncthreads();
        }
        box.y = sh[0];
        __syncthreads();
        v = valid ? yi : INFINITY;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int w = TILE / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + w]);
            __syncthreads();
        }
        box.z = sh[0];
        __syncthreads();
        v = valid ? yi : -INFINITY;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int w = TILE / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
            __syncthreads();
        }
        box.w = sh[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ws.tbox[blockIdx.x] = box;
        __threadfence();
        const int k = atomicAdd(&ws.hdr[2], 1);
        last = (k == (int)gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        // the last block reduces the tile bounds (each thread a strided subset, then a tree)
        __threadfence();
        double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += TILE) {
            // written by other blocks: read through L2
            const double2 lo = __ldcg(reinterpret_cast<const double2 *>(&ws.tbox[b]));
            const double2 hi = __ldcg(reinterpret_cast<const double2 *>(&ws.tbox[b]) + 1);
            x0 = fmin(x0, lo.x); x1 = fmax(x1, lo.y); y0 = fmin(y0, hi.x); y1 = fmax(y1, hi.y);
        }
        __shared__ double4_32a shb[TILE];
        shb[threadIdx.x] = make_double4_32a(x0, x1, y0, y1);
        __syncthreads();
        for (int w = TILE / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) {
                const double4_32a a = shb[threadIdx.x], b = shb[threadIdx.x + w];
                shb[threadIdx.x] = make_double4_32a(fmin(a.x, b.x), fmax(a.y, b.y), fmin(a.z, b.z), fmax(a.w, b.w));
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double4_32a bb = shb[0];
            const double t0 = in.t[0], t1 = in.t[n - 1];
            ws.centre[0] = isfinite(bb.x + bb.y) ? 0.5 * (bb.x + bb.y) : 0.0;
            ws.centre[1] = isfinite(bb.z + bb.w) ? 0.5 * (bb.z + bb.w) : 0.0;
            ws.centre[2] = isfinite(t0 + t1) ? 0.5 * (t0 + t1) : 0.0;
            ws.centre[3] = t1;  // t_N: the last event time (sorted input)
            ws.hdr[2] = 0;      // ticket ready for the next call
        }
    }
}

__global__ void __launch_bounds__(TILE) pack_kernel(Consts c, Inputs in, Workspace ws) {
    const Derived &D = *c.d;
    const int n = c.g.n;
    const int i = blockIdx.x * TILE + threadIdx.x;
    const bool valid = i < n;
    __shared__ float shf[TILE];
    __shared__ int shi[TILE];

    const int dup = valid ? (ws.cnt[ws.loc[i]] >= 2) : 0;
    if (valid && !isfinite(in.r[i])) atomicOr(&ws.hdr[0], ST_NONFINITE);

    float tmin = INFINITY, tmax = -INFINITY, rtmax = -INFINITY;
    if (c.fp32c) {
        const double xc = ws.centre[0], yc = ws.centre[1], tc = ws.centre[2];
        float xs, ys, ts, rs;
        if (valid) {
            // stored negated so that target - source is one packed add; the
            // fourth slot holds r^ = r~ + t~ (log-rate and time folded, base 2)
            xs = -(float)((in.x[i] - xc) * D.sx);
            ys = -(float)((in.y[i] - yc) * D.sx);
            const double tsc = (in.t[i] - tc) * D.st;
            ts = -(float)tsc;
            rs = (float)(in.r[i] * LOG2E + tsc);
            tmin = (float)tsc;
            tmax = (float)tsc;
            rtmax = rs;
        } else {
            // padding source: far away in space and time, contributes exact zeros
            xs = -1.0e9f; ys = -1.0e9f; ts = -1.0e9f; rs = -1.0e9f;
        }
        float *f = reinterpret_cast<float *>(ws.src32);
        const int p = i >> 1, l = i & 1;
        f[8 * p + 0 + l] = xs;
        f[8 * p + 2 + l] = ys;
        f[8 * p + 4 + l] = ts;
        f[8 * p + 6 + l] = rs;
    } else {
        if (valid) ws.src64[i] = make_double4_32a(in.x[i], in.y[i], in.t[i], in.r[i]);
        else ws.src64[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);  // never read: loops stop at n
    }

    // per-tile statistics (FP32C scaled time bounds and max(r~ + t~))
    tmin = -block_max<TILE>(-tmin, shf);
    tmax = block_max<TILE>(tmax, shf);
    rtmax = block_max<TILE>(rtmax, shf);
    // duplicate flag: any event of the tile shares its location with another event
    shi[threadIdx.x] = dup;
    __syncthreads();
    for (int w = TILE / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) shi[threadIdx.x] |= shi[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int first = blockIdx.x * TILE;
        const int lastv = min(n, first + TILE) - 1;
        ws.tinfo[blockIdx.x] = make_int4(ws.gidx[first], ws.gidx[lastv], shi[0], lastv - first + 1);
        if (c.fp32c) ws.tstat32[blockIdx.x] = make_float4(tmin, tmax, rtmax, -INFINITY);
    }
}

cudaError_t launch_prep(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    prep_kernel<<<c.g.tiles, TILE, 0, s>>>(c, in, ws);
    return cudaGetLastError();
}

cudaError_t launch_pack(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    pack_kernel<<<c.g.tiles, TILE, 0, s>>>(c, in, ws);
    return cudaGetLastError();
}

}  // namespace hk
