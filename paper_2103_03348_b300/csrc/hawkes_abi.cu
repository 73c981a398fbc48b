// extern "C" entry points of libhawkes.so (declared in include/hawkes.h).
//
// Argument checks, workspace carving and the launch sequence, plus the one-thread
// setup kernel that derives the per-call constants from the parameter vector
// (given on the host or in device memory).  No host synchronisation and no
// allocation: everything is enqueued on the caller's stream into the caller's
// workspace.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "hawkes_internal.cuh"

namespace hk {

static int ceil_div(int a, int b) { return (a + b - 1) / b; }

Geometry make_geometry(int64_t n) {
    Geometry g;
    g.n = (int)n;
    g.tiles = ceil_div(g.n, TILE);
    g.npad = g.tiles * TILE;
    // Enough (target tile, source chunk) blocks for several waves on 148 SMs
    // at 4 resident blocks each, without making chunks shorter than one tile.
    const int target_blocks = 148 * 32;
    int chunks = ceil_div(target_blocks, g.tiles);
    if (chunks < 1) chunks = 1;
    if (chunks > g.tiles) chunks = g.tiles;
    g.chunk_tiles = ceil_div(g.tiles, chunks);
    g.n_chunks = ceil_div(g.tiles, g.chunk_tiles);
    int hs = 1024;
    while (hs < 2 * g.n) hs <<= 1;
    g.hash_size = hs;
    return g;
}

size_t carve(void *base, const Geometry &g, int precision, Workspace *w) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return base ? (void *)((char *)base + o) : nullptr;
    };
    const size_t np = (size_t)g.npad, nt = (size_t)g.tiles;
    // the header and, after it, the validation bits kept for calls that reuse the events
    w->hdr = (int *)take((8 + 1) * sizeof(int));
    w->evbits = base ? w->hdr + 8 : nullptr;
    w->derived = (Derived *)take(sizeof(Derived));
    w->centre = (double *)take(4 * sizeof(double));
    w->hash = (int *)take((size_t)g.hash_size * sizeof(int));
    w->cnt = (int *)take(np * sizeof(int));
    w->loc = (int *)take(np * sizeof(int));
    w->gidx = (int *)take(np * sizeof(int));
    w->tinfo = (int4 *)take(nt * sizeof(int4));
    w->tbox = (double4_32a *)take(nt * sizeof(double4_32a));
    const bool f32 = precision == HAWKES_FP32C || precision == HAWKES_FP32C_BAND || precision == HAWKES_FP32C_ST;
    const bool st = precision == HAWKES_FP32C_ST;
    w->src32 = f32 ? (float4 *)take(np * sizeof(float4)) : nullptr;
    w->tgt32 = f32 ? (float4 *)take(np * sizeof(float4)) : nullptr;
    w->tstat32 = f32 ? (float4 *)take(nt * sizeof(float4)) : nullptr;
    w->sufmax = f32 ? (float *)take(nt * sizeof(float)) : nullptr;
    w->src64 = f32 ? nullptr : (double4_32a *)take(np * sizeof(double4_32a));
    w->w64 = f32 ? nullptr : (double *)take(np * sizeof(double));
    w->rowpart = (double *)take((size_t)g.n_chunks * NMOM * np * sizeof(double));
    w->mom = (double *)take((size_t)NMOM * np * sizeof(double));
    w->dLr = (double *)take(np * sizeof(double));
    // row-finish partials: one per tile, or one per 32-row group on space-time tiles
    w->blockpart = (double *)take((st ? np / GROUP : nt) * ACC_STRIDE * sizeof(double));
    w->ipart = f32 ? (double *)take(nt * (TILE / GROUP) * ACC_STRIDE * sizeof(double)) : nullptr;
    w->colpart = (double *)take((size_t)g.n_chunks * 2 * np * sizeof(double));
    w->bbox = (double *)take(4 * sizeof(double));
    w->perm = st ? (int *)take(np * sizeof(int)) : nullptr;
    w->inv = st ? (int *)take(np * sizeof(int)) : nullptr;
    w->gidx_o = st ? (int *)take(np * sizeof(int)) : nullptr;
    w->loc_o = st ? (int *)take(np * sizeof(int)) : nullptr;
    w->xp = st ? (double *)take(np * sizeof(double)) : nullptr;
    w->yp = st ? (double *)take(np * sizeof(double)) : nullptr;
    w->tp = st ? (double *)take(np * sizeof(double)) : nullptr;
    w->rp = st ? (double *)take(np * sizeof(double)) : nullptr;
    w->grp = st ? (GroupStat *)take(np / GROUP * sizeof(GroupStat)) : nullptr;
    w->trank = st ? (int2 *)take(nt * sizeof(int2)) : nullptr;
    return off;
}

static bool params_valid(const double *p) {
    for (int k = 0; k < 6; ++k) {
        if (k == 2 && isinf(p[k]) && p[k] > 0) continue;
        if (!isfinite(p[k]) || !(p[k] > 0)) return false;
    }
    return true;
}

// Every parameter-dependent constant, derived in FP64.  FP64 is slow on this
// part (one warp instruction holds an SM's FP64 pipe for about 19 cycles), so
// the constants are spread over SETUP_BLOCKS one-warp blocks, one group of
// constants per block and so per SM, each block first reading (and
// exponentiating) the six parameters on six lanes.  Parameters that are not
// finite and positive (tau_t may be +inf) set ST_BADPARAM, and finalize then
// reports HAWKES_EINVAL with NaN outputs.
constexpr int SETUP_BLOCKS = 13 + EP_N;

__global__ void setup_kernel(ParamSource ps, int fp32c, int reuse, Derived *out, int *hdr, const int *evbits) {
    pdl_wait();
    const int lane = threadIdx.x;
    double pv = 0.0;
    if (lane < 6) pv = ps.dev ? (ps.log_scale ? exp(ps.dev[lane]) : ps.dev[lane]) : ps.v[lane];
    double p[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = __shfl_sync(0xffffffffu, pv, k);
    const double mu0 = p[0], tx = p[1], tt = p[2], th0 = p[3], om = p[4], h = p[5];
    const int tt_inf = isinf(tt) ? 1 : 0;
    const double two_pi = 6.283185307179586476925286766559;
    const double B = th0 * om / (two_pi * h * h);
    const double sx = fp32c ? sqrt(LOG2E / 2.0) / tx : sqrt(0.5) / tx;
    const double st = fp32c ? om * LOG2E : om;
    const double sxe = fp32c ? sx : sqrt(0.5) / h;
    // the call's header: status bits (with the event checks of the call that
    // prepared these events, when they are reused), the rest cleared
    if (blockIdx.x == 0 && lane > 0 && lane < 8) hdr[lane] = 0;
    if (lane != 0) return;
    switch (blockIdx.x) {  // block-uniform: one group of constants per block
        case 0: {
            bool ok = true;
            for (int k = 0; k < 6; ++k) {
                if (k == 2 && isinf(p[k]) && p[k] > 0) continue;
                if (!isfinite(p[k]) || !(p[k] > 0)) ok = false;
            }
            out->mu0 = mu0; out->tx = tx; out->tt = tt; out->th0 = th0; out->om = om; out->h = h;
            out->tt_inf = tt_inf;
            out->valid = ok ? 1 : 0;
            hdr[0] = (reuse ? *evbits : 0) | (ok ? 0 : ST_BADPARAM);
            break;
        }
        case 1: out->A = tt_inf ? mu0 / (two_pi * tx * tx) : mu0 / (two_pi * sqrt(two_pi) * tx * tx * tt); break;
        case 2: out->B = B; break;
        case 3: out->ln_b = log(B); break;
        case 4: out->log2_b = log2(B); break;
        // FP64 pair constants (also used by the FP32C fix-up rows)
        case 5: out->ibx = 1.0 / (2.0 * tx * tx); break;
        case 6: out->ibt = tt_inf ? 0.0 : 1.0 / (2.0 * tt * tt); break;
        case 7: out->ih = 1.0 / (2.0 * h * h); break;
        // x~ = (x - xc) sqrt(log2(e)/2) / tau_x makes the background's spatial exponent -d~^2;
        // t~ = (t - tc) omega log2(e) makes the excitation's temporal exponent -dt~.
        case 8:
            out->sx = sx;
            out->sxh = fp32c ? sqrt(LOG2E / 2.0) / h : 1.0;
            out->sxe = sxe;
            break;
        case 9: out->st = st; break;
        case 10: out->cbt = (fp32c && !tt_inf) ? (float)(LOG2E / (2.0 * tt * tt) / (st * st)) : 0.0f; break;
        case 11: out->hh = fp32c ? (float)((tx / h) * (tx / h)) : 0.0f; break;
        case 12: out->i_tt = tt_inf ? 0.0 : 1.0 / tt; break;  // the integral term
        default: {
            // the row epilogue's coefficients (Derived::ep): A or B times the
            // moment's unit conversion (1/sx^2 per d~^2, 1/st per dt~) and the
            // parameter powers of the derivative
            const int j = blockIdx.x - 13;
            if (j < 0 || j >= EP_N) break;
            const double A = tt_inf ? mu0 / (two_pi * tx * tx) : mu0 / (two_pi * sqrt(two_pi) * tx * tx * tt);
            const double isx2 = 1.0 / (sx * sx), isxe2 = 1.0 / (sxe * sxe), ist = 1.0 / st, ist2 = ist * ist;
            const double ix = 1.0 / tx, it = tt_inf ? 0.0 : 1.0 / tt, ih = 1.0 / h;
            const double ix2 = ix * ix, it2 = it * it, ih2 = ih * ih;
            double v = 0.0;
            switch (j) {
                case EP_G0: v = A / mu0; break;
                case EP_GD2: v = A * isx2 * (ix2 * ix); break;
                case EP_G1: v = 2.0 * A * ix; break;
                case EP_GT2: v = A * ist2 * (it2 * it); break;
                case EP_G2: v = A * it; break;
                case EP_E3: v = B / th0; break;
                case EP_E4: v = B / om; break;
                case EP_ET: v = B * ist; break;
                case EP_ED2: v = B * isxe2 * (ih2 * ih); break;
                case EP_E5: v = 2.0 * B * ih; break;
                case EP_GD4: v = A * (isx2 * isx2) * (ix2 * ix2 * ix2); break;
                case EP_GD2B: v = 7.0 * A * isx2 * (ix2 * ix2); break;
                case EP_G1B: v = 6.0 * A * ix2; break;
                case EP_GT4: v = A * (ist2 * ist2) * (it2 * it2 * it2); break;
                case EP_GT2B: v = 5.0 * A * ist2 * (it2 * it2); break;
                case EP_G2B: v = 2.0 * A * it2; break;
                case EP_ET2: v = B * ist2; break;
                case EP_ETB: v = 2.0 * B * ist / om; break;
                case EP_ED4: v = B * (isxe2 * isxe2) * (ih2 * ih2 * ih2); break;
                case EP_ED2B: v = 7.0 * B * isxe2 * (ih2 * ih2); break;
                case EP_E5B: v = 6.0 * B * ih2; break;
                default: break;
            }
            out->ep[j] = v;
            break;
        }
    }
}

cudaError_t launch_setup(const Consts &c, const ParamSource &ps, const Workspace &ws, cudaStream_t s, int reuse) {
    launch_pdl(setup_kernel, SETUP_BLOCKS, 32, 0, s, ps, c.fp32c, reuse, ws.derived, ws.hdr, ws.evbits);
    return cudaGetLastError();
}

// One evaluation's constants, carved workspace and outputs.
struct Call {
    Consts c;
    Workspace ws;
    Inputs in;   // as given (time order)
    Inputs inw;  // what the kernels after prep read: the FP32C_ST position-order copies, else in
    Outputs out;
    ParamSource ps;
    cudaStream_t s;
    bool rates;   // the column pass runs
    bool reuse;   // x, y, t and the workspace are those of an earlier call: skip their preparation
    bool subset = false;            // rate entries only for rate_idx[0..k_rates)
    const int *rate_idx = nullptr;
    int k_rates = 0;
};

static int prepare(const double *x, const double *y, const double *t, const double *r, int64_t n,
                   const double *params, const double *params_dev, int log_params, int precision, void *wsp,
                   size_t ws_bytes, int mode, double *loglik, double *grad, double *hdiag, int *dev_status,
                   void *stream, Call *k) {
    if (n < 2 || n > HAWKES_MAX_EVENTS) return HAWKES_EINVAL;
    if (precision != HAWKES_FP64 && precision != HAWKES_FP32C && precision != HAWKES_FP32C_BAND &&
        precision != HAWKES_FP32C_ST)
        return HAWKES_EINVAL;
    k->reuse = (mode & HAWKES_MODE_REUSE_EVENTS) != 0;
    mode &= ~HAWKES_MODE_REUSE_EVENTS;
    // modes 3 and 4: gradient / Hessian diagonal of the six globals only (no column pass)
    if (mode < 0 || mode > 4) return HAWKES_EINVAL;
    k->rates = mode == MODE_GRAD || mode == MODE_HESS;
    if (mode == 3) mode = MODE_GRAD;
    if (mode == 4) mode = MODE_HESS;
    if (!x || !y || !t || !r || !(params || params_dev) || !wsp || !dev_status) return HAWKES_EINVAL;
    if (mode == MODE_LL && !loglik) return HAWKES_EINVAL;
    if (mode == MODE_GRAD && !grad) return HAWKES_EINVAL;
    if (mode == MODE_HESS && !hdiag) return HAWKES_EINVAL;
    if (((uintptr_t)wsp & 255) != 0) return HAWKES_EINVAL;
    if (params && !params_valid(params)) return HAWKES_EINVAL;
    const Geometry g = make_geometry(n);
    const size_t need = carve(wsp, g, precision, &k->ws);
    if (ws_bytes < need) return HAWKES_EWORKSPACE;

    Consts &c = k->c;
    memset(&c, 0, sizeof(c));
    c.g = g;
    c.mode = mode;
    c.fp32c = precision == HAWKES_FP32C || precision == HAWKES_FP32C_BAND || precision == HAWKES_FP32C_ST;
    c.band = precision == HAWKES_FP32C_BAND;
    c.st = precision == HAWKES_FP32C_ST;
    c.fin_groups = c.st && g.tiles < FIN_GROUP_TILES;
    c.t0 = 0;
    c.t1 = g.tiles;
    c.d = k->ws.derived;
    memset(&k->ps, 0, sizeof(k->ps));
    if (params) {
        for (int j = 0; j < 6; ++j) k->ps.v[j] = params[j];
    } else {
        k->ps.dev = params_dev;
        k->ps.log_scale = log_params ? 1 : 0;
    }
    k->in = {x, y, t, r};
    k->inw = c.st ? Inputs{k->ws.xp, k->ws.yp, k->ws.tp, k->ws.rp} : k->in;
    k->out = {loglik, mode >= MODE_GRAD ? grad : nullptr, mode == MODE_HESS ? hdiag : nullptr, dev_status};
    k->s = (cudaStream_t)stream;
    return HAWKES_OK;
}

static bool mark(void *const *events, int j, cudaStream_t s) {
    return !(events && events[j]) || cudaEventRecord((cudaEvent_t)events[j], s) == cudaSuccess;
}

// Validation, packing (all events), then the row pass, row combine, FP64
// fix-up and row epilogue for the target tiles [t0, t1).
static int phase_rows(const Call &k, void *const *events) {
    const Consts &c = k.c;
    const Workspace &ws = k.ws;
    cudaStream_t s = k.s;
    const size_t hdr_ints = 8;  // the header; evbits follows
    if (k.reuse) {  // setup clears the header; evbits keeps the event checks of the call that prepared the events
        if (launch_setup(c, k.ps, ws, s, 1) != cudaSuccess) return HAWKES_ECUDA;
    } else {
        if (cudaMemsetAsync(ws.hdr, 0, (hdr_ints + 1) * sizeof(int), s) != cudaSuccess) return HAWKES_ECUDA;
        if (cudaMemsetAsync(ws.hash, 0xFF, (size_t)c.g.hash_size * sizeof(int), s) != cudaSuccess) return HAWKES_ECUDA;
        if (cudaMemsetAsync(ws.cnt, 0, (size_t)c.g.npad * sizeof(int), s) != cudaSuccess) return HAWKES_ECUDA;
        if (launch_setup(c, k.ps, ws, s, 0) != cudaSuccess) return HAWKES_ECUDA;
        if (c.st) {  // prep's per-event indices in time order, then regrouped by position
            Workspace wt = ws;
            wt.gidx = ws.gidx_o;
            wt.loc = ws.loc_o;
            if (launch_prep(c, k.in, wt, s) != cudaSuccess) return HAWKES_ECUDA;
            if (launch_order(c, k.in, ws, s) != cudaSuccess) return HAWKES_ECUDA;
        } else {
            if (launch_prep(c, k.in, ws, s) != cudaSuccess) return HAWKES_ECUDA;
        }
    }
    if (launch_pack(c, k.inw, ws, k.in.r, s) != cudaSuccess) return HAWKES_ECUDA;
    if (!mark(events, 0, s)) return HAWKES_ECUDA;
    if (c.t1 > c.t0) {
        if ((c.fp32c ? launch_row32(c, k.inw, ws, s) : launch_row64(c, ws, s)) != cudaSuccess) return HAWKES_ECUDA;
    }
    if (!mark(events, 1, s)) return HAWKES_ECUDA;
    if (c.t1 > c.t0) {
        if (c.fp32c) {  // combine, FP64 fix-up of tiny rows and epilogue, one block per tile
            if (launch_finish(c, k.inw, ws, s) != cudaSuccess) return HAWKES_ECUDA;
        } else {
            if (launch_combine(c, ws, s) != cudaSuccess) return HAWKES_ECUDA;
            if (launch_epilogue(c, k.inw, ws, s) != cudaSuccess) return HAWKES_ECUDA;
        }
    }
    return HAWKES_OK;
}

// The fixed-order reduction over every tile's partials (loglik, global
// gradient and Hessian diagonal), then the column pass and its finish for the
// source tiles [t0, t1).
static int phase_cols(const Call &k, void *const *events) {
    const Consts &c = k.c;
    cudaStream_t s = k.s;
    if (launch_finalize(c, k.ws, k.out, s) != cudaSuccess) return HAWKES_ECUDA;
    if (c.mode >= MODE_GRAD && k.rates) {
        if (!mark(events, 2, s)) return HAWKES_ECUDA;
        if (k.subset) {  // a subset of the sources (FP64 covers all of them and writes the subset)
            if (k.k_rates > 0) {
                if ((c.fp32c ? launch_col32_subset(c, k.inw, k.ws, k.rate_idx, k.k_rates, s)
                             : launch_col64(c, k.ws, s)) != cudaSuccess)
                    return HAWKES_ECUDA;
            }
            if (!mark(events, 3, s)) return HAWKES_ECUDA;
            if (k.k_rates > 0 &&
                launch_colfinish_subset(c, k.ws, k.out, k.rate_idx, k.k_rates, c.fp32c, s) != cudaSuccess)
                return HAWKES_ECUDA;
            return HAWKES_OK;
        }
        if (c.t1 > c.t0) {
            if ((c.fp32c ? launch_col32(c, k.inw, k.ws, s) : launch_col64(c, k.ws, s)) != cudaSuccess)
                return HAWKES_ECUDA;
        }
        if (!mark(events, 3, s)) return HAWKES_ECUDA;
        if (c.t1 > c.t0 && launch_colfinish(c, k.ws, k.out, s) != cudaSuccess) return HAWKES_ECUDA;
    }
    return HAWKES_OK;
}

static int run(const double *x, const double *y, const double *t, const double *r, int64_t n,
               const double *params, const double *params_dev, int log_params, int precision, void *wsp,
               size_t ws_bytes, int mode, double *loglik, double *grad, double *hdiag, int *dev_status, void *stream,
               void *const *events = nullptr) {
    Call k;
    int rc = prepare(x, y, t, r, n, params, params_dev, log_params, precision, wsp, ws_bytes, mode, loglik, grad,
                     hdiag, dev_status, stream, &k);
    if (rc != HAWKES_OK) return rc;
    rc = phase_rows(k, events);
    if (rc != HAWKES_OK) return rc;
    return phase_cols(k, events);
}

// Shard s of k owns tiles [s * tiles / k, (s + 1) * tiles / k).
static void shard_range(int tiles, int shard, int n_shards, int *t0, int *t1) {
    *t0 = (int)((int64_t)shard * tiles / n_shards);
    *t1 = (int)((int64_t)(shard + 1) * tiles / n_shards);
}

static int shard_phase(const double *x, const double *y, const double *t, const double *r, int64_t n,
                       const double params[6], int precision, int mode, int shard, int n_shards, void *wsp,
                       size_t ws_bytes, void *xbuf, size_t xbuf_bytes, double *loglik, double *grad, double *hdiag,
                       int *dev_status, void *stream, bool second) {
    if (n_shards < 1 || shard < 0 || shard >= n_shards || !params || !xbuf) return HAWKES_EINVAL;
    if (precision == HAWKES_FP32C_ST) return HAWKES_EINVAL;  // shards own tiles of the time order
    if (((uintptr_t)xbuf & 15) != 0) return HAWKES_EINVAL;
    if (n < 2 || n > HAWKES_MAX_EVENTS) return HAWKES_EINVAL;
    const Geometry g = make_geometry(n);
    if (xbuf_bytes < (size_t)g.tiles * XREC_DOUBLES * sizeof(double)) return HAWKES_EWORKSPACE;
    // the output pointers are checked (and used) only in the second phase
    double dummy_out = 0.0;
    Call k;
    int rc = prepare(x, y, t, r, n, params, nullptr, 0, precision, wsp, ws_bytes, mode,
                     second ? loglik : &dummy_out, second ? grad : &dummy_out, second ? hdiag : &dummy_out,
                     dev_status, stream, &k);
    if (rc != HAWKES_OK) return rc;
    shard_range(g.tiles, shard, n_shards, &k.c.t0, &k.c.t1);
    if (!second) {
        rc = phase_rows(k, nullptr);
        if (rc != HAWKES_OK) return rc;
        return launch_shard_export(k.c, k.ws, (double *)xbuf, k.s) == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
    }
    if (launch_shard_import(k.c, k.inw, k.ws, (const double *)xbuf, k.s) != cudaSuccess) return HAWKES_ECUDA;
    return phase_cols(k, nullptr);
}

}  // namespace hk

extern "C" {

size_t hawkes_workspace_size(int64_t n, int precision) {
    if (n < 2 || n > HAWKES_MAX_EVENTS) return 0;
    if (precision != HAWKES_FP64 && precision != HAWKES_FP32C && precision != HAWKES_FP32C_BAND &&
        precision != HAWKES_FP32C_ST)
        return 0;
    hk::Workspace w;
    return hk::carve(nullptr, hk::make_geometry(n), precision, &w);
}

int hawkes_loglik(const double *x, const double *y, const double *t, const double *r, int64_t n,
                  const double params[6], int precision, void *ws, size_t ws_bytes,
                  double *loglik, int *dev_status, void *stream) {
    return hk::run(x, y, t, r, n, params, nullptr, 0, precision, ws, ws_bytes, hk::MODE_LL, loglik, nullptr, nullptr,
                   dev_status, stream);
}

int hawkes_grad(const double *x, const double *y, const double *t, const double *r, int64_t n,
                const double params[6], int precision, void *ws, size_t ws_bytes,
                double *loglik, double *grad, int *dev_status, void *stream) {
    return hk::run(x, y, t, r, n, params, nullptr, 0, precision, ws, ws_bytes, hk::MODE_GRAD, loglik, grad, nullptr,
                   dev_status, stream);
}

int hawkes_hess_diag(const double *x, const double *y, const double *t, const double *r, int64_t n,
                     const double params[6], int precision, void *ws, size_t ws_bytes,
                     double *loglik, double *grad, double *hdiag, int *dev_status, void *stream) {
    return hk::run(x, y, t, r, n, params, nullptr, 0, precision, ws, ws_bytes, hk::MODE_HESS, loglik, grad, hdiag,
                   dev_status, stream);
}

int hawkes_hess_diag_timed(const double *x, const double *y, const double *t, const double *r, int64_t n,
                           const double params[6], int precision, void *ws, size_t ws_bytes,
                           double *loglik, double *grad, double *hdiag, int *dev_status, void *stream,
                           void *const phase_events[4]) {
    return hk::run(x, y, t, r, n, params, nullptr, 0, precision, ws, ws_bytes, hk::MODE_HESS, loglik, grad, hdiag,
                   dev_status, stream, phase_events);
}

int hawkes_eval_device_params(const double *x, const double *y, const double *t, const double *r, int64_t n,
                              const double *params_dev, int log_params, int precision, int mode, void *ws,
                              size_t ws_bytes, double *loglik, double *grad, double *hdiag, int *dev_status,
                              void *stream) {
    if (!params_dev) return HAWKES_EINVAL;
    return hk::run(x, y, t, r, n, nullptr, params_dev, log_params, precision, ws, ws_bytes, mode, loglik, grad,
                   hdiag, dev_status, stream);
}

size_t hawkes_shard_exchange_size(int64_t n) {
    if (n < 2 || n > HAWKES_MAX_EVENTS) return 0;
    return (size_t)hk::make_geometry(n).tiles * hk::XREC_DOUBLES * sizeof(double);
}

int hawkes_shard_range(int64_t n, int shard, int n_shards, int64_t *first_event, int64_t *end_event,
                       size_t *xbuf_offset, size_t *xbuf_bytes) {
    if (n < 2 || n > HAWKES_MAX_EVENTS || n_shards < 1 || shard < 0 || shard >= n_shards) return HAWKES_EINVAL;
    const hk::Geometry g = hk::make_geometry(n);
    int t0, t1;
    hk::shard_range(g.tiles, shard, n_shards, &t0, &t1);
    const size_t rec = hk::XREC_DOUBLES * sizeof(double);
    if (first_event) *first_event = (int64_t)t0 * hk::TILE < n ? (int64_t)t0 * hk::TILE : n;
    if (end_event) *end_event = (int64_t)t1 * hk::TILE < n ? (int64_t)t1 * hk::TILE : n;
    if (xbuf_offset) *xbuf_offset = (size_t)t0 * rec;
    if (xbuf_bytes) *xbuf_bytes = (size_t)(t1 - t0) * rec;
    return HAWKES_OK;
}

int hawkes_shard_rows(const double *x, const double *y, const double *t, const double *r, int64_t n,
                      const double params[6], int precision, int mode, int shard, int n_shards, void *ws,
                      size_t ws_bytes, void *xbuf, size_t xbuf_bytes, int *dev_status, void *stream) {
    return hk::shard_phase(x, y, t, r, n, params, precision, mode, shard, n_shards, ws, ws_bytes, xbuf, xbuf_bytes,
                           nullptr, nullptr, nullptr, dev_status, stream, false);
}

int hawkes_shard_cols(const double *x, const double *y, const double *t, const double *r, int64_t n,
                      const double params[6], int precision, int mode, int shard, int n_shards, void *ws,
                      size_t ws_bytes, const void *xbuf, size_t xbuf_bytes, double *loglik, double *grad,
                      double *hdiag, int *dev_status, void *stream) {
    return hk::shard_phase(x, y, t, r, n, params, precision, mode, shard, n_shards, ws, ws_bytes, (void *)xbuf,
                           xbuf_bytes, loglik, grad, hdiag, dev_status, stream, true);
}

int hawkes_eval_rates_subset(const double *x, const double *y, const double *t, const double *r, int64_t n,
                             const double *params_dev, int log_params, int precision, int mode, const int *rate_idx,
                             int64_t k_rates, void *ws, size_t ws_bytes, double *loglik, double *grad, double *hdiag,
                             int *dev_status, void *stream) {
    if (!params_dev || k_rates < 0 || k_rates > n || (k_rates > 0 && !rate_idx)) return HAWKES_EINVAL;
    const int base = mode & ~HAWKES_MODE_REUSE_EVENTS;
    if (base != HAWKES_MODE_GRAD && base != HAWKES_MODE_HESS) return HAWKES_EINVAL;
    hk::Call k;
    int rc = hk::prepare(x, y, t, r, n, nullptr, params_dev, log_params, precision, ws, ws_bytes, mode, loglik, grad,
                         hdiag, dev_status, stream, &k);
    if (rc != HAWKES_OK) return rc;
    k.subset = true;
    k.rate_idx = rate_idx;
    k.k_rates = (int)k_rates;
    rc = hk::phase_rows(k, nullptr);
    if (rc != HAWKES_OK) return rc;
    return hk::phase_cols(k, nullptr);
}

const char *hawkes_strerror(int status) {
    switch (status) {
        case HAWKES_OK: return "success";
        case HAWKES_EINVAL: return "invalid argument (n, null pointer, parameters, precision or workspace alignment)";
        case HAWKES_EUNSORTED: return "event times are not in ascending order";
        case HAWKES_ENONFINITE: return "an event coordinate, time or log-rate is not finite";
        case HAWKES_EWORKSPACE: return "workspace smaller than hawkes_workspace_size(n, precision)";
        case HAWKES_ECUDA: return "a CUDA launch or memset failed";
        case HAWKES_EZERO_INTENSITY: return "some event has zero intensity: the log-likelihood is -inf";
        case HAWKES_ESCRATCH: return "n exceeds HAWKES_NOALLOC_MAX_EVENTS, the capacity of the allocation-free call";
        default: return "unknown status";
    }
}

const char *hawkes_version(void) { return "hawkes-b300 0.1 (sm_103a)"; }

}  // extern "C"
