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
// order (FP32C_ST only): the events of each slab of 4096 time-consecutive
// events are sorted by the Hilbert index of their cell on a 65536 x 65536 grid
// over the events' bounding square, so every tile of 128 positions covers a
// compact region of space inside the slab's time window; the permuted copies
// of x, y, t and of the tie-group and location indices are gathered.
// pack (one block per tile):
//   * FP32C: scaled, centred FP32 sources stored as pairs for f32x2 arithmetic,
//     ((-x0,-x1,-y0,-y1),(-t0,-t1,r^0,r^1)) with r^ = r~ + t~, and per-tile
//     statistics;
//   * FP64: (x, y, t, r) as double4_32a;
//   * per-tile lowest/highest tie-group start and duplicate-location flag;
//   * FP32C_ST: per-group (32 events) bounds for pruning, per-tile rank range.
#include <climits>

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
    pdl_wait();
    const int n = c.g.n;
    const int i = blockIdx.x * TILE + threadIdx.x;
    __shared__ bool last;
    int bad = 0;
    double xi = 0.0, yi = 0.0;
    const bool valid = i < n;
    if (valid) {
        xi = in.x[i];
        yi = in.y[i];
        const double ti = in.t[i];
        if (!isfinite(xi) || !isfinite(yi) || !isfinite(ti)) bad |= ST_NONFINITE;  // r: checked by pack
        const double tp = i > 0 ? in.t[i - 1] : -INFINITY;
        if (i > 0 && !(tp <= ti)) bad |= ST_UNSORTED;
        // tie-group start: first index j <= i with t_j == t_i (lower bound on a
        // sorted prefix); i itself when the previous time is smaller, the usual case
        int lo = i;
        if (i > 0 && !(tp < ti)) {
            lo = 0;
            int hi = i;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (in.t[mid] < ti) lo = mid + 1; else hi = mid;
            }
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
        atomicOr(ws.evbits, bad);  // kept for calls that reuse these events
    }

    // per-tile bounds of x and y (valid events only): warp shuffles, then the
    // four warps' bounds in shared memory (min and max are exact in any order)
    double4_32a box;
    {
        double bx0 = valid ? xi : INFINITY, bx1 = valid ? xi : -INFINITY;
        double by0 = valid ? yi : INFINITY, by1 = valid ? yi : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bx0 = fmin(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
            bx1 = fmax(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
            by0 = fmin(by0, __shfl_xor_sync(0xffffffffu, by0, o));
            by1 = fmax(by1, __shfl_xor_sync(0xffffffffu, by1, o));
        }
        __shared__ double4_32a wbox[TILE / 32];
        if ((threadIdx.x & 31) == 0) wbox[threadIdx.x >> 5] = make_double4_32a(bx0, bx1, by0, by1);
        __syncthreads();
        box = wbox[0];
#pragma unroll
        for (int w = 1; w < TILE / 32; ++w) {
            const double4_32a b = wbox[w];
            box = make_double4_32a(fmin(box.x, b.x), fmax(box.y, b.y), fmin(box.z, b.z), fmax(box.w, b.w));
        }
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
            ws.bbox[0] = bb.x; ws.bbox[1] = bb.y; ws.bbox[2] = bb.z; ws.bbox[3] = bb.w;
            const double t0 = in.t[0], t1 = in.t[n - 1];
            ws.centre[0] = isfinite(bb.x + bb.y) ? 0.5 * (bb.x + bb.y) : 0.0;
            ws.centre[1] = isfinite(bb.z + bb.w) ? 0.5 * (bb.z + bb.w) : 0.0;
            ws.centre[2] = isfinite(t0 + t1) ? 0.5 * (t0 + t1) : 0.0;
            ws.centre[3] = t1;  // t_N: the last event time (sorted input)
            ws.hdr[2] = 0;      // ticket ready for the next call
        }
    }
}

__global__ void __launch_bounds__(TILE) pack_kernel(Consts c, Inputs in, Workspace ws, const double *r_time_order) {
    pdl_wait();
    const Derived &D = *c.d;
    const int n = c.g.n;
    const int i = blockIdx.x * TILE + threadIdx.x;
    const bool valid = i < n;

    // FP32C_ST: position i holds event perm[i]; its log-rate is gathered here
    double ri = 0.0;
    if (valid) {
        ri = c.st ? r_time_order[ws.perm[i]] : in.r[i];
        if (c.st) ws.rp[i] = ri;
    }
    const int dup = valid ? (ws.cnt[ws.loc[i]] >= 2) : 0;
    if (valid && !isfinite(ri)) atomicOr(&ws.hdr[0], ST_NONFINITE);

    float tmin = INFINITY, tmax = -INFINITY, rtmax = -INFINITY;
    float xw = 0.0f, yw = 0.0f;  // scaled coordinates (FP32C_ST group bounds)
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
            rs = (float)(ri * LOG2E + tsc);
            tmin = (float)tsc;
            tmax = (float)tsc;
            rtmax = rs;
            xw = -xs;
            yw = -ys;
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
        if (valid) ws.src64[i] = make_double4_32a(in.x[i], in.y[i], in.t[i], ri);
        else ws.src64[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);  // never read: loops stop at n
    }

    if (c.st) {
        // group bounds (one warp = one group of 32 positions); empty groups get
        // empty bounds (min > max), which every pruning test treats as dead
        const int gi = valid ? ws.gidx[i] : INT_MAX, rk = valid ? ws.perm[i] : INT_MAX;
        GroupStat gs;
        gs.box = make_float4(warp_minf(valid ? xw : INFINITY), warp_maxf(valid ? xw : -INFINITY),
                             warp_minf(valid ? yw : INFINITY), warp_maxf(valid ? yw : -INFINITY));
        gs.tr = make_float4(warp_minf(tmin), warp_maxf(tmax), warp_maxf(rtmax), -INFINITY);
        gs.ix = make_int4(warp_mini(gi), warp_maxi(valid ? gi : INT_MIN), warp_mini(rk),
                          warp_maxi(valid ? rk : INT_MIN));
        if ((threadIdx.x & 31) == 0) ws.grp[i / GROUP] = gs;
    }

    // per-tile statistics: each warp reduces with shuffles, one barrier, then
    // thread 0 combines the four warps (FP32C scaled time bounds, max(r~ + t~),
    // duplicate flag; on space-time tiles the tie-group and rank ranges)
    __shared__ float wf[3][TILE / 32];
    __shared__ int wi[5][TILE / 32];
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const float a0 = warp_minf(tmin), a1 = warp_maxf(tmax), a2 = warp_maxf(rtmax);
        const int dupw = __any_sync(0xffffffffu, dup) ? 1 : 0;
        int b0 = 0, b1 = 0, b2 = 0, b3 = 0;
        if (c.st) {
            const int gi = valid ? ws.gidx[i] : INT_MAX, rk = valid ? ws.perm[i] : INT_MAX;
            b0 = warp_mini(gi);
            b1 = warp_maxi(valid ? gi : INT_MIN);
            b2 = warp_mini(rk);
            b3 = warp_maxi(valid ? rk : INT_MIN);
        }
        if (lane == 0) {
            wf[0][warp] = a0; wf[1][warp] = a1; wf[2][warp] = a2;
            wi[0][warp] = dupw; wi[1][warp] = b0; wi[2][warp] = b1; wi[3][warp] = b2; wi[4][warp] = b3;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t0 = wf[0][0], t1 = wf[1][0], rt = wf[2][0];
        int has_dup = wi[0][0], g_lo = wi[1][0], g_hi = wi[2][0], k_lo = wi[3][0], k_hi = wi[4][0];
        for (int w = 1; w < TILE / 32; ++w) {
            t0 = fminf(t0, wf[0][w]); t1 = fmaxf(t1, wf[1][w]); rt = fmaxf(rt, wf[2][w]);
            has_dup |= wi[0][w];
            g_lo = min(g_lo, wi[1][w]); g_hi = max(g_hi, wi[2][w]);
            k_lo = min(k_lo, wi[3][w]); k_hi = max(k_hi, wi[4][w]);
        }
        const int first = blockIdx.x * TILE;
        const int lastv = min(n, first + TILE) - 1;
        if (!c.st) {  // time order: gidx is non-decreasing
            g_lo = ws.gidx[first];
            g_hi = ws.gidx[lastv];
        }
        ws.tinfo[blockIdx.x] = make_int4(g_lo, g_hi, has_dup, lastv - first + 1);
        if (c.fp32c) ws.tstat32[blockIdx.x] = make_float4(t0, t1, rt, -INFINITY);
        if (c.st) ws.trank[blockIdx.x] = make_int2(k_lo, k_hi);
    }
}

// Position of cell (x, y) of a 65536 x 65536 grid along the Hilbert curve
// (the usual quadrant-by-quadrant construction: at each scale the quadrant
// index is added and the cell's coordinates are reflected and swapped into
// the quadrant's own orientation).  Runs of the curve are more compact than
// runs of a Morton (bit-interleaved) order, so groups of 32 consecutive
// positions have smaller boxes.
__device__ __forceinline__ unsigned hilbert16(unsigned x, unsigned y) {
    constexpr unsigned N = 65536u;
    unsigned d = 0;
    for (unsigned s = N >> 1; s > 0; s >>= 1) {
        const unsigned rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = N - 1 - x;
                y = N - 1 - y;
            }
            const unsigned t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

constexpr int ORDER_THREADS = 1024;

// The bitonic compare-exchanges of one merge size at strides first_stride,
// first_stride / 2, ..., 1 (all below 128) on a warp's run of 128 keys, key r
// of this lane at position base + 32 r + lane.  Position p of a pair (p, p +
// stride) keeps the smaller key when p's bit `size` is clear (an ascending
// run), the larger one otherwise.
__device__ __forceinline__ void sort_warp_run(unsigned (&k4)[4], int base, int lane, int size, int first_stride) {
#pragma unroll
    for (int stride = 64; stride > 0; stride >>= 1) {  // unrolled: the register indices are constants
        if (stride > first_stride) continue;
        if (stride >= 32) {  // a lane's own keys r and r + stride / 32
            const int d = stride >> 5;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r & d) continue;
                const bool up = ((base + 32 * r + lane) & size) == 0;
                const unsigned a = k4[r], b = k4[r + d];
                if ((a > b) == up) {
                    k4[r] = b;
                    k4[r + d] = a;
                }
            }
        } else {  // lanes l and l ^ stride, the lower one at position p
            const bool lo = (lane & stride) == 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const bool up = ((base + 32 * r + lane) & size) == 0;
                const unsigned o = __shfl_xor_sync(0xffffffffu, k4[r], stride);
                const unsigned mn = min(k4[r], o), mx = max(k4[r], o);
                k4[r] = (lo == up) ? mn : mx;
            }
        }
    }
}

// One block per slab: 32-bit keys (the top 20 bits of the Hilbert index, a
// 1024 x 1024 grid over the bounding square, then the 12-bit slot) sorted
// ascending in shared memory by a bitonic network; unique keys make the order
// deterministic, events of one cell keeping their time order.
__global__ void __launch_bounds__(ORDER_THREADS) order_sort_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    static_assert(SLAB_EVENTS == 4096, "12-bit slots");
    __shared__ unsigned keys[SLAB_EVENTS];
    const int n = c.g.n;
    const int e0 = blockIdx.x * SLAB_EVENTS;
    const int cnt = min(n - e0, SLAB_EVENTS);
    const double x0 = ws.bbox[0], x1 = ws.bbox[1], y0 = ws.bbox[2], y1 = ws.bbox[3];
    const double span = fmax(x1 - x0, y1 - y0);  // one scale for both axes: square cells
    const double sc = (isfinite(span) && span > 0.0) ? 65535.0 / span : 0.0;
    for (int k = threadIdx.x; k < SLAB_EVENTS; k += ORDER_THREADS) {
        unsigned key = ~0u;  // empty slots sort last (a full slab has none; below 4096 events slots stay < 4095)
        if (k < cnt) {
            // fmax / fmin map NaN to the bound, so non-finite inputs (reported by prep) stay in range
            const unsigned ix = (unsigned)fmin(fmax((in.x[e0 + k] - x0) * sc, 0.0), 65535.0);
            const unsigned iy = (unsigned)fmin(fmax((in.y[e0 + k] - y0) * sc, 0.0), 65535.0);
            key = ((hilbert16(ix, iy) >> 12) << 12) | (unsigned)k;
        }
        keys[k] = key;
    }
    __syncthreads();
    // Bitonic sort.  Compare-exchanges at strides of 128 and more go through
    // shared memory, one barrier each; the strides below 128 stay inside a
    // warp's run of 128 keys (key r of lane l at position 128 w + 32 r + l),
    // in registers: strides 64 and 32 pair a lane's own keys, the smaller
    // ones pair lanes by shuffles, with no barrier.
    static_assert(SLAB_EVENTS == ORDER_THREADS * 4, "four keys per thread");
    const int lane = threadIdx.x & 31, base = (threadIdx.x >> 5) * 128;
    unsigned k4[4];
    // sizes 2 to 128: whole in the warp
#pragma unroll
    for (int r = 0; r < 4; ++r) k4[r] = keys[base + 32 * r + lane];
    for (int size = 2; size <= 128; size <<= 1) sort_warp_run(k4, base, lane, size, size >> 1);
#pragma unroll
    for (int r = 0; r < 4; ++r) keys[base + 32 * r + lane] = k4[r];
    __syncthreads();
    for (int size = 256; size <= SLAB_EVENTS; size <<= 1) {
        for (int stride = size >> 1; stride >= 128; stride >>= 1) {
            for (int q = threadIdx.x; q < SLAB_EVENTS / 2; q += ORDER_THREADS) {
                const int lo = 2 * q - (q & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned a = keys[lo], b = keys[hi];
                if ((a > b) == up) {
                    keys[lo] = b;
                    keys[hi] = a;
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) k4[r] = keys[base + 32 * r + lane];
        sort_warp_run(k4, base, lane, size, 64);
#pragma unroll
        for (int r = 0; r < 4; ++r) keys[base + 32 * r + lane] = k4[r];
        __syncthreads();
    }
    for (int k = threadIdx.x; k < cnt; k += ORDER_THREADS) ws.perm[e0 + k] = e0 + (int)(keys[k] & 0xfffu);
}

// Position-order copies of the events and of prep's per-event indices.
__global__ void __launch_bounds__(TILE) order_gather_kernel(Consts c, Inputs in, Workspace ws) {
    pdl_wait();
    const int n = c.g.n;
    const int k = blockIdx.x * TILE + threadIdx.x;  // < npad
    if (k < n) {
        const int o = ws.perm[k];
        ws.inv[o] = k;
        ws.xp[k] = in.x[o];
        ws.yp[k] = in.y[o];
        ws.tp[k] = in.t[o];
        ws.gidx[k] = ws.gidx_o[o];
        ws.loc[k] = ws.loc_o[o];
    } else {
        ws.perm[k] = k;
        ws.inv[k] = k;
        ws.xp[k] = 0.0;
        ws.yp[k] = 0.0;
        ws.tp[k] = 0.0;
        ws.rp[k] = 0.0;
        ws.gidx[k] = n;      // padding: never a causal source, never a target
        ws.loc[k] = -1 - k;  // padding: a location of its own
    }
}

cudaError_t launch_prep(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    launch_pdl(prep_kernel, c.g.tiles, TILE, 0, s, c, in, ws);
    return cudaGetLastError();
}

cudaError_t launch_order(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s) {
    const int slabs = (c.g.n + SLAB_EVENTS - 1) / SLAB_EVENTS;
    launch_pdl(order_sort_kernel, slabs, ORDER_THREADS, 0, s, c, in, ws);
    if (cudaGetLastError() != cudaSuccess) return cudaErrorLaunchFailure;
    launch_pdl(order_gather_kernel, c.g.tiles, TILE, 0, s, c, in, ws);
    return cudaGetLastError();
}

cudaError_t launch_pack(const Consts &c, const Inputs &in, const Workspace &ws, const double *r_time_order,
                        cudaStream_t s) {
    launch_pdl(pack_kernel, c.g.tiles, TILE, 0, s, c, in, ws, r_time_order);
    return cudaGetLastError();
}

}  // namespace hk
