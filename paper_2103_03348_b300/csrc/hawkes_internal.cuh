// Internal declarations shared by the kernels of libhawkes.so.
//
// Data flow of one call (all enqueued on the caller's stream, no host sync):
//   prep     validate, per-event tie-group start, exact-location dedup, centre
//   order    FP32C_ST only: regroup each slab of time-consecutive events by a
//            Hilbert index of (x, y), so that tiles are compact in space and time
//   pack     FP32 scaled source pairs + per-tile statistics (FP32C), FP64 copy
//   row      per (target tile, source chunk): moment sums of the pair terms
//            (Eq. 1's inner sum and its parameter derivatives)
//   combine  sum the chunk partials of each row in FP64 (fixed order)
//   fixup    FP32C only: rows whose FP32 sum is below 2^-60 redone in FP64
//   epilogue per row: lambda_n, log lambda_n, derivative terms, the integral
//            term (Appendix A) per event, column-pass weights; block partials
//            (FP32C: combine, fixup and epilogue run as one kernel, finish)
//   finalize one block: deterministic sum of block partials -> outputs
//   col      per (source tile, target chunk): Eq. 4 / Eq. 5 column sums
//   colfin   per source: combine column partials, subtract dLambda/dr_m
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <utility>

#include "hawkes.h"

// Kernel launch with programmatic dependent launch allowed: in a stream (and
// in a graph captured from it) the next kernel is set up while this one
// drains, so a chain of short kernels loses less time between launches.
// Every kernel launched this way starts with hk::pdl_wait(), which holds it
// until everything before it on the stream has completed and is visible, so
// the ordering is that of a plain launch.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Blocks of a kernel (at `threads` threads per block, no dynamic shared
// memory) that are resident on the current device at once: SMs x blocks per
// SM, for a persistent grid.  A host-side query, cached per kernel, device and
// block size, so that launches after the first (and launches being captured
// into a graph) only read the cache.  0 on an error.
inline int resident_blocks_of(const void *kernel, int threads) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    struct Entry {
        const void *kernel;
        int dev, threads, blocks;
    };
    static std::mutex mu;
    static Entry cache[64];
    static int used = 0;
    std::lock_guard<std::mutex> lock(mu);
    for (int k = 0; k < used; ++k)
        if (cache[k].kernel == kernel && cache[k].dev == dev && cache[k].threads == threads) return cache[k].blocks;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) return 0;
    const int blocks = sms * per_sm;
    if (used < 64) cache[used++] = Entry{kernel, dev, threads, blocks};
    return blocks;
}

template <typename... KArgs>
inline int resident_blocks(void (*kernel)(KArgs...), int threads) {
    return resident_blocks_of(reinterpret_cast<const void *>(kernel), threads);
}

namespace hk {

constexpr int TILE = 128;   // events per tile: targets per row block, sources per shared-memory subtile
constexpr int GROUP = 32;   // events per group (one warp's targets or sources) in FP32C_ST
constexpr int SLAB_TILES = 32;                   // FP32C_ST: tiles per slab of time-consecutive events
constexpr int SLAB_EVENTS = SLAB_TILES * TILE;  // 4096: sorted by Hilbert index in shared memory
constexpr int NMOM = 10;    // row moments (hess mode)
constexpr int NACC = 13;    // per-row terms reduced across rows: loglik, 6 gradient, 6 Hessian
constexpr int ACC_STRIDE = 16;
constexpr int XREC_DOUBLES = 16 + TILE;  // one tile's record in the shard exchange buffer

constexpr int MODE_LL = 0, MODE_GRAD = 1, MODE_HESS = 2;

// device status bits (combined into a hawkes_status by finalize)
constexpr int ST_UNSORTED = 1, ST_NONFINITE = 2, ST_ZERO = 4, ST_BADPARAM = 8;

// log2(e) and the FP32C underflow threshold: an exponent (base 2) below this
// gives exactly 0 from ex2.approx.ftz, so tiles whose bound lies below it are
// skipped without changing the FP32 result (2 units of margin for rounding).
constexpr double LOG2E = 1.4426950408889634074;
constexpr float EXP2_DEAD = -128.0f;
// background band skipping: a tile pair whose time gap g has cbt g^2 above this
// has every background term below 2^-130, i.e. exactly 0 in FP32
constexpr float BG_DEAD = 130.0f;
// rows whose FP32 background and excitation sums are both below 2^-60 are
// recomputed in FP64 (terms below 2^-126 were flushed to zero in FP32)
constexpr float TINY_ROW = 8.673617379884035e-19f;  // 2^-60
// FP32C_ST: below this many tiles (about 1.35 per SM of a B300) the rows are
// finished per 32-row group (four blocks per tile, each a quarter of the chunk
// loads deep), so that a small problem spreads its finish over the SMs; from
// it on, per tile (more rows per block to hide the FP64 epilogue's latency).
// Measured: 183 tiles (23,422 events) 3.5 us faster per group; 274 tiles
// (35,000 events) 10 us faster per tile.
constexpr int FIN_GROUP_TILES = 200;
// Header slot of the persistent space-time row pass's work counter.
constexpr int HDR_ST_ROW_UNITS = 4;

// Moment index (row pass).  Background terms G, excitation terms E (with exp(r)):
//   0 sum G        1 sum G d^2     2 sum G dt^2    3 sum G d^4     4 sum G dt^4
//   5 sum E        6 sum E dt      7 sum E dt^2    8 sum E d^2     9 sum E d^4
enum { MO_G = 0, MO_GD2 = 1, MO_GT2 = 2, MO_GD4 = 3, MO_GT4 = 4, MO_E = 5, MO_ET = 6, MO_ET2 = 7, MO_ED2 = 8, MO_ED4 = 9 };

struct Geometry {
    int n, tiles, npad, chunk_tiles, n_chunks, hash_size;
};

Geometry make_geometry(int64_t n);

// Constants derived from the parameter vector.  setup_kernel computes them in
// FP64 on the device, from host values or from device memory, and every other
// kernel reads them from the workspace, so a call whose parameters live on the
// device needs no host round trip.
struct Derived {
    double mu0, tx, tt, th0, om, h;
    double A, B;          // lambda_n = A * sum G + B * sum E
    double sx, st;        // scaled coordinates x~ = (x - xc) sx, t~ = (t - tc) st of the row moments:
                          // FP32C sx = sqrt(log2(e)/2) / tau_x, st = omega log2(e); FP64 sx = sqrt(1/2) / tau_x,
                          // st = omega (moments in the kernels' own units stay far from FP64's subnormals)
    double sxe;           // the excitation moments' spatial scale: sx (FP32C), sqrt(1/2) / h (FP64)
    double sxh;           // FP32C column pass: x' = (x - xc) sxh, so that hh d~^2 = d'^2 (sxh = sx tau_x / h)
    double ibx, ibt, ih;  // FP64:  G = exp(-ibx d^2 - ibt dt^2), E = exp(r - om dt - ih d^2)
    float cbt, hh;        // FP32C: G = 2^-(d~^2 + cbt dt~^2), E = 2^(r^_s - t~_n - hh d~^2)
    int tt_inf, valid;
    double i_tt;          // 1/tau_t (0 when infinite), for the integral term
    double ln_b, log2_b;  // log B and log2 B: column weights in the log domain, log(B / lambda) = ln_b - log lambda
    // the row epilogue's coefficients on the moments (scaled units), so that
    // each row spends one multiply or fused multiply-add per term: lambda_n q1
    // and lambda_n s2 (the first and second parameter derivatives of lambda_n)
    // are sums of coefficient x moment
    double ep[21];
};

// Indices into Derived::ep.  dlam/dp:  mu0: G0 S_G;  tau_x: GD2 M_GD2 - G1 S_G;
// tau_t: GT2 M_GT2 - G2 S_G;  theta0: E3 S_E;  omega: E4 S_E - ET M_ET;
// h: ED2 M_ED2 - E5 S_E.  d2lam/dp2:  tau_x: GD4 M_GD4 - GD2B M_GD2 + G1B S_G;
// tau_t: GT4 M_GT4 - GT2B M_GT2 + G2B S_G;  omega: ET2 M_ET2 - ETB M_ET;
// h: ED4 M_ED4 - ED2B M_ED2 + E5B S_E  (mu0 and theta0 enter linearly).
enum {
    EP_G0, EP_GD2, EP_G1, EP_GT2, EP_G2, EP_E3, EP_E4, EP_ET, EP_ED2, EP_E5,
    EP_GD4, EP_GD2B, EP_G1B, EP_GT4, EP_GT2B, EP_G2B, EP_ET2, EP_ETB, EP_ED4, EP_ED2B, EP_E5B, EP_N
};

// Per-call constants known on the host (passed by value to every kernel).
struct Consts {
    Geometry g;
    int mode, fp32c, band;  // band: FP32C with exact background band skipping
    int st;            // FP32C_ST: space-time tiles (events permuted inside slabs), group pruning
    int fin_groups;    // FP32C_ST with few tiles: rows finished per 32-row group (finish_group_st)
    int t0, t1;        // the tiles this call owns as targets (row pass) and sources (column pass)
    const Derived *d;  // device: written by setup_kernel
};

// The parameter vector for setup_kernel: host values, or a device pointer
// (optionally holding the logarithms of the parameters).
struct ParamSource {
    double v[6];
    const double *dev;
    int log_scale;
};

// FP32C_ST statistics of a group of 32 consecutive events (in tile order), in
// the scaled FP32 units of the packed sources:
//   box = (x~ min, x~ max, y~ min, y~ max)
//   tr  = (t~ min, t~ max, max r^, max g^)   (g^ written by the epilogue)
//   ix  = (min gidx, max gidx, min rank, max rank), rank = time-order index
struct GroupStat {
    float4 box;
    float4 tr;
    int4 ix;
};

// Workspace carving.  Offsets are multiples of 256 bytes.
struct Workspace {
    int *hdr;            // [0] status bits, [2] prep's last-block ticket, [4] the space-time row pass's
                         // work counter (HDR_ST_ROW_UNITS); [1..7] cleared by every call's setup
    int *evbits;         // [1] prep's validation bits, kept for calls that reuse the events (follows hdr)
    Derived *derived;    // [1]  constants derived from the parameters
    double *centre;      // [4]: xc, yc, tc, tN
    int *hash;           // [hash_size]
    int *cnt;            // [npad]  members of each exact-location group (indexed by representative)
    int *loc;            // [npad]  representative index of the event's location
    int *gidx;           // [npad]  first index with the same time (tie-group start)
    int4 *tinfo;         // [tiles] min and max gidx of the tile's events, has_dup, valid count
    double4_32a *tbox;       // [tiles] xmin, xmax, ymin, ymax (prep)
    float4 *src32;       // [npad]  pairs: (-x0,-x1,-y0,-y1),(-t0,-t1,r^0,r^1), r^ = r~ + t~ (read-only
                         //         after pack: row blocks of other tiles read it while a tile finishes)
    float4 *tgt32;       // [npad]  the column pass's targets: (-x'0,-x'1,-y'0,-y'1),(-t0,-t1,-g^0,-g^1) in the
                         //         excitation's scaled coordinates x' = (x - xc) sxh, with the column
                         //         weight g^ = log2(B/lambda) - t~, written by the tile finish
    float4 *tstat32;     // [tiles] t~min, t~max, max r^, max g^
    double4_32a *src64;      // [npad]  (x, y, t, r) FP64 (FP64 path)
    double *rowpart;     // [n_chunks * NMOM * npad]: FP64 partials (FP64 path), FP32C Kahan pairs as float2
    double *mom;         // [NMOM * npad]
    double *w64;         // [npad]  FP64 column weight, in logs: log(B / lambda_n)
    double *dLr;         // [npad]  dLambda / dr_m
    double *blockpart;   // [tiles * ACC_STRIDE], or [groups * ACC_STRIDE] on space-time tiles (room for fin_groups)
    double *ipart;       // [tiles * 4 * ACC_STRIDE] FP32C: the integral-term sums of each 32-event group (row pass)
    float *sufmax;       // [tiles] suffix max of the column weight bound (FP32C)
    double *colpart;     // [n_chunks * 2 * npad]
    double *bbox;        // [4]: x min, x max, y min, y max of the events (prep)
    // FP32C_ST only (NULL otherwise).  Position k holds event perm[k] (time
    // order); gidx and loc above are then indexed by position.
    int *perm;           // [npad]  position -> time-order index (identity on padding)
    int *inv;            // [npad]  time-order index -> position
    int *gidx_o, *loc_o; // [npad]  prep's tie-group starts and location groups, time order
    double *xp, *yp, *tp, *rp;  // [npad] the events in position order
    GroupStat *grp;      // [npad / GROUP]
    int2 *trank;         // [tiles] min, max rank of the tile's events
};

size_t carve(void *base, const Geometry &g, int precision, Workspace *ws);  // returns total bytes; base may be NULL

struct Inputs {
    const double *x, *y, *t, *r;
};

struct Outputs {
    double *loglik, *grad, *hdiag;
    int *dev_status;
};

// launchers (return cudaGetLastError())
cudaError_t launch_setup(const Consts &c, const ParamSource &ps, const Workspace &ws, cudaStream_t s, int reuse);
cudaError_t launch_prep(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s);
cudaError_t launch_order(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s);
cudaError_t launch_pack(const Consts &c, const Inputs &in, const Workspace &ws, const double *r_time_order,
                        cudaStream_t s);
cudaError_t launch_row32(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s);
cudaError_t launch_finish(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s);
cudaError_t launch_row64(const Consts &c, const Workspace &ws, cudaStream_t s);
cudaError_t launch_combine(const Consts &c, const Workspace &ws, cudaStream_t s);
cudaError_t launch_epilogue(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s);
cudaError_t launch_finalize(const Consts &c, const Workspace &ws, const Outputs &out, cudaStream_t s);
cudaError_t launch_col32(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s);
cudaError_t launch_col64(const Consts &c, const Workspace &ws, cudaStream_t s);
cudaError_t launch_colfinish(const Consts &c, const Workspace &ws, const Outputs &out, cudaStream_t s);
cudaError_t launch_col32_subset(const Consts &c, const Inputs &in, const Workspace &ws, const int *rate_idx,
                                int k_rates, cudaStream_t s);
cudaError_t launch_row32_st(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s);
cudaError_t launch_col32_st(const Consts &c, const Inputs &in, const Workspace &ws, cudaStream_t s);
cudaError_t launch_col32_subset_st(const Consts &c, const Inputs &in, const Workspace &ws, const int *rate_idx,
                                   int k_rates, cudaStream_t s);
cudaError_t launch_colfinish_subset(const Consts &c, const Workspace &ws, const Outputs &out, const int *rate_idx,
                                    int k_rates, int by_position, cudaStream_t s);
cudaError_t launch_shard_export(const Consts &c, const Workspace &ws, double *xbuf, cudaStream_t s);
cudaError_t launch_shard_import(const Consts &c, const Inputs &in, const Workspace &ws, const double *xbuf,
                                cudaStream_t s);
cudaError_t launch_tree_prior(int64_t m, const int *plan, const double *len, double tau0, double sigma2,
                              const double *z, double *scratch, double *logdens, double *pz, double *pdiag,
                              cudaStream_t s);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

// Wait for the preceding kernel of the stream (programmatic dependent launch;
// a no-op for a plain launch).  The first statement of every kernel started
// with launch_pdl.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

// Kahan step: s + v with the running compensation c (true sum ~= s - c).
__device__ __forceinline__ void kahan(float &s, float &c, float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Deterministic block sum of one double per thread (fixed tree order).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
#pragma unroll
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Deterministic warp sums of K <= 16 doubles per lane by reduce-scatter: at
// each of the offsets 16, 8, 4, 2 a lane keeps half of its slots (the upper
// half where that bit of its lane index is set), sends the other half to the
// partner lane and adds what it receives; the last exchange (offset 1) adds
// the two halves of the warp.  Lane l returns the total of component l >> 1
// (meaningful for l >> 1 < K; lanes l and l ^ 1 return the same value).  16
// FP64 additions per lane instead of 5 K for a butterfly per component: FP64
// instructions are costly on this part.
template <int K>
__device__ __forceinline__ double warp_sum_scatter(const double (&v)[K]) {
    static_assert(K >= 1 && K <= 16, "at most 16 components");
    const int lane = threadIdx.x & 31;
    double a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = k < K ? v[k] : 0.0;
#pragma unroll
    for (int o = 16, m = 8; o >= 2; o >>= 1, m >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < m; ++j) {
            const double send = up ? a[j] : a[j + m];
            const double keep = up ? a[j + m] : a[j];
            a[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return a[0] + __shfl_xor_sync(0xffffffffu, a[0], 1);
}

// Deterministic block sums of K <= 16 doubles per thread: each warp's sums by
// warp_sum_scatter, then the warps' partials summed in warp order.  Thread
// k < K returns total k (other threads return 0).  sh holds (NT / 32) * K doubles.
template <int NT, int K>
__device__ __forceinline__ double block_sum_multi(const double (&v)[K], double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double w = warp_sum_scatter<K>(v);
    if ((lane & 1) == 0 && (lane >> 1) < K) sh[warp * K + (lane >> 1)] = w;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < K) {
#pragma unroll
        for (int q = 0; q < NT / 32; ++q) r += sh[q * K + threadIdx.x];
    }
    __syncthreads();
    return r;
}

template <int NT>
__device__ __forceinline__ float block_max(float v, float *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
#pragma unroll
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    const float r = sh[0];
    __syncthreads();
    return r;
}

// Warp-wide min / max (every lane gets the result).
__device__ __forceinline__ float warp_minf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_mini(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_maxi(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---- FP32C_ST pruning bounds between two groups (or unions of groups) ----
// Every bound is taken over the FP32 values the pair loops use, so a pruned
// group pair holds only terms that ex2.approx.ftz would flush to exactly 0.

__device__ __forceinline__ bool group_empty(const GroupStat &a) { return a.ix.z > a.ix.w; }

__device__ __forceinline__ GroupStat group_union(const GroupStat &a, const GroupStat &b) {
    GroupStat u;
    u.box = make_float4(fminf(a.box.x, b.box.x), fmaxf(a.box.y, b.box.y), fminf(a.box.z, b.box.z),
                        fmaxf(a.box.w, b.box.w));
    u.tr = make_float4(fminf(a.tr.x, b.tr.x), fmaxf(a.tr.y, b.tr.y), fmaxf(a.tr.z, b.tr.z), fmaxf(a.tr.w, b.tr.w));
    u.ix = make_int4(min(a.ix.x, b.ix.x), max(a.ix.y, b.ix.y), min(a.ix.z, b.ix.z), max(a.ix.w, b.ix.w));
    return u;
}

// smallest squared scaled distance between two boxes (0 when they overlap)
__device__ __forceinline__ float box_gap2(const float4 a, const float4 b) {
    const float gx = fmaxf(fmaxf(b.x - a.y, a.x - b.y), 0.0f);
    const float gy = fmaxf(fmaxf(b.z - a.w, a.z - b.w), 0.0f);
    return gx * gx + gy * gy;
}

// background terms between targets W and sources S: 2^-(d~^2 + cbt dt~^2)
__device__ __forceinline__ bool bg_alive(const GroupStat &W, const GroupStat &S, float cbt) {
    const float gt = fmaxf(fmaxf(S.tr.x - W.tr.y, W.tr.x - S.tr.y), 0.0f);
    const float q = box_gap2(W.box, S.box) + (cbt > 0.0f ? cbt * gt * gt : 0.0f);
    return !(q > BG_DEAD);
}

// a bound e on an exponent below which every term is 0, with a relative
// allowance for the rounding of the terms that make it up
__device__ __forceinline__ bool exp2_alive(float e, float scale) {
    return e >= EXP2_DEAD - 1.0e-5f * fminf(scale, 1.0e30f);  // e = -inf or NaN: dead
}

// excitation terms of the row pass: 2^(r^_s - t~_n - hh d~^2), s strictly earlier than n
__device__ __forceinline__ bool exc_alive(const GroupStat &W, const GroupStat &S, float hh) {
    if (S.ix.z >= W.ix.y) return false;  // no source precedes any target (rank vs tie-group start)
    const float d = hh * box_gap2(W.box, S.box);
    return exp2_alive(S.tr.z - W.tr.x - d, fabsf(S.tr.z) + fabsf(W.tr.x) + d);
}

// column terms: 2^(g^_n + r^_m - hh d~^2) for sources W and targets G
__device__ __forceinline__ bool col_alive(const GroupStat &W, const GroupStat &G, float hh) {
    if (G.ix.y <= W.ix.z) return false;  // no target follows any source
    const float d = hh * box_gap2(W.box, G.box);
    return exp2_alive(W.tr.z + G.tr.w - d, fabsf(W.tr.z) + fabsf(G.tr.w) + d);
}

// The column pass's packed target i (position order): (-x'_i, -y'_i) with
// x' = (x - xc) sxh from the FP64 inputs, so that the excitation's spatial
// exponent hh d~^2 is d'^2 with no multiply; -t~_i copied from the packed
// sources; and -g^_i (g^ = -inf for padding and rows without a weight, so
// that every term of that target is exactly 0).
__device__ __forceinline__ void pack_target(const Workspace &ws, const Inputs &in, const Derived &D, int i, int n,
                                            float ghat) {
    const float *f = reinterpret_cast<const float *>(ws.src32);
    float *o = reinterpret_cast<float *>(ws.tgt32);
    const int p = i >> 1, l = i & 1;
    float xs = 0.0f, ys = 0.0f;
    if (i < n) {
        xs = -(float)((in.x[i] - ws.centre[0]) * D.sxh);
        ys = -(float)((in.y[i] - ws.centre[1]) * D.sxh);
    }
    o[8 * p + 0 + l] = xs;
    o[8 * p + 2 + l] = ys;
    o[8 * p + 4 + l] = f[8 * p + 4 + l];
    o[8 * p + 6 + l] = -ghat;
}

#endif  // __CUDACC__

}  // namespace hk
