// Row finishing shared by the FP64 path (k_fp64.cu, k_epi.cu) and the FP32C
// finish kernel (k_epi.cu): the FP64 pair terms (also used to redo tiny FP32C
// rows), the per-row epilogue, and the FP32C tile finish.
#pragma once

#include "hawkes_internal.cuh"

namespace hk {

// The moments are taken in the scaled units of Derived (d~^2 = d^2 sx^2 for the
// background, d^2 sxe^2 for the excitation, dt~ = dt st): with raw units a
// small bandwidth would push moments such as G d^4 of a tiny-intensity row
// into FP64's subnormal range (at tau_x = 6e-4 and an intensity of 1e-302,
// G d^4 is about 1e-315, with 27 significant bits left), and the Hessian
// entry, a difference of such moments, would lose them.
template <int MODE>
__device__ __forceinline__ void accumulate64(double (&a)[NMOM], double xs, double ys, double ts, double rs,
                                             bool bg_on, bool ex_on, double xn, double yn, double tn,
                                             const Derived &D) {
    const double dx = xn - xs, dy = yn - ys, dt = tn - ts;
    const double d2 = dx * dx + dy * dy, dt2 = dt * dt;
    const double ut = dt * D.st, ut2 = ut * ut;
    if (bg_on) {
        const double g = exp(-D.ibx * d2 - D.ibt * dt2);
        const double u2 = d2 * (D.sx * D.sx);
        a[MO_G] += g;
        if (MODE >= MODE_GRAD) { a[MO_GD2] += g * u2; a[MO_GT2] += g * ut2; }
        if (MODE == MODE_HESS) { a[MO_GD4] += g * u2 * u2; a[MO_GT4] += g * ut2 * ut2; }
    }
    if (ex_on) {
        const double e = exp(rs - D.om * dt - D.ih * d2);
        const double v2 = d2 * (D.sxe * D.sxe);
        a[MO_E] += e;
        if (MODE >= MODE_GRAD) { a[MO_ET] += e * ut; a[MO_ED2] += e * v2; }
        if (MODE == MODE_HESS) { a[MO_ET2] += e * ut2; a[MO_ED4] += e * v2 * v2; }
    }
}

__device__ __forceinline__ double std_pdf(double z) { return 0.3989422804014327 * exp(-0.5 * z * z); }
__device__ __forceinline__ double std_cdf(double z) { return 0.5 * erfc(-z * 0.7071067811865476); }

// This event's share of the integral term (Appendix A Claim, the background
// integrated exactly over [0, t_N]) and its derivatives, subtracted from
// acc[0], acc[1..6] and acc[7..12]; dLambda/dr_i goes to dLr[i].  It depends
// on the parameters and the event alone, not on the row sums.
__device__ __forceinline__ void integral_row(const Derived &D, const Inputs &in, const Workspace &ws, int i,
                                             double (&acc)[NACC]) {
    const double tN = ws.centre[3];
    const double ti = in.t[i], a_ = tN - ti, b_ = -ti;
    const double th = exp(in.r[i]);
    const double dec = exp(-D.om * a_);
    const double one_m = -expm1(-D.om * a_);
    double L = 0.0, dL[6] = {0, 0, 0, 0, 0, 0}, d2L[6] = {0, 0, 0, 0, 0, 0};
    if (D.tt_inf) {
        dL[0] = tN;
    } else {
        const double it = D.i_tt, za = a_ * it, zb = b_ * it;
        const double pa = std_pdf(za), pb = std_pdf(zb);
        dL[0] = std_cdf(za) - std_cdf(zb);
        const double it2 = it * it, it3 = it2 * it, it5 = it3 * it2;
        dL[2] = D.mu0 * (-(a_ * it2) * pa + (b_ * it2) * pb);
        d2L[2] = D.mu0 * (pa * (2.0 * a_ * it3 - a_ * a_ * a_ * it5) - pb * (2.0 * b_ * it3 - b_ * b_ * b_ * it5));
    }
    L = D.mu0 * dL[0] + D.th0 * th * one_m;
    dL[3] = th * one_m;
    dL[4] = D.th0 * th * a_ * dec;
    d2L[4] = -D.th0 * th * a_ * a_ * dec;
    ws.dLr[i] = D.th0 * th * one_m;
    acc[0] -= L;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        acc[1 + p] -= dL[p];
        acc[7 + p] -= d2L[p];
    }
}

// The row epilogue of event i (one thread): lambda_n and its derivative terms
// from the moments Mo (Eq. 1 and its parameter derivatives) into acc (the
// 13 per-row terms: log lambda_n, the six q1 and the six q2), the FP32C column
// weight g^ (returned in ghat) or the FP64 weight, and with INTEGRAL the
// event's share of the integral term subtracted (integral_row).
template <bool INTEGRAL>
__device__ __forceinline__ void epilogue_row(const Consts &c, const Derived &D, const Inputs &in, const Workspace &ws,
                                             int i, const double (&Mo)[NMOM], double (&acc)[NACC], float &ghat) {
    const int mode = c.mode;
    const double SG = Mo[MO_G], SE = Mo[MO_E];
    const double lam = D.A * SG + D.B * SE;
    double q1[6] = {0, 0, 0, 0, 0, 0}, q2[6] = {0, 0, 0, 0, 0, 0};
    double ll = 0.0;
    if (lam > 0.0) {
        ll = log(lam);
        if (mode >= MODE_GRAD) {
            // lambda_n q1 and lambda_n s2 as coefficient x moment sums (Derived::ep),
            // then divided by lambda_n.  Each numerator is (A or B) x moments of
            // the size of lambda_n's terms; below 1e-300, where 1 / lambda_n could
            // overflow, numerators and lambda_n are first scaled by 2^600 (exact).
            const bool tiny = !(lam > 1e-300);
            const double il = 1.0 / (tiny ? lam * 0x1p600 : lam);  // before the numerators: fewer live values
            const double *e = D.ep;
            double n1[6], n2[6] = {0, 0, 0, 0, 0, 0};
            n1[0] = e[EP_G0] * SG;
            n1[1] = e[EP_GD2] * Mo[MO_GD2] - e[EP_G1] * SG;
            n1[2] = e[EP_GT2] * Mo[MO_GT2] - e[EP_G2] * SG;
            n1[3] = e[EP_E3] * SE;
            n1[4] = e[EP_E4] * SE - e[EP_ET] * Mo[MO_ET];
            n1[5] = e[EP_ED2] * Mo[MO_ED2] - e[EP_E5] * SE;
            if (mode == MODE_HESS) {
                n2[1] = e[EP_GD4] * Mo[MO_GD4] - e[EP_GD2B] * Mo[MO_GD2] + e[EP_G1B] * SG;
                n2[2] = e[EP_GT4] * Mo[MO_GT4] - e[EP_GT2B] * Mo[MO_GT2] + e[EP_G2B] * SG;
                n2[4] = e[EP_ET2] * Mo[MO_ET2] - e[EP_ETB] * Mo[MO_ET];
                n2[5] = e[EP_ED4] * Mo[MO_ED4] - e[EP_ED2B] * Mo[MO_ED2] + e[EP_E5B] * SE;
            }
            if (tiny) {
#pragma unroll
                for (int p = 0; p < 6; ++p) { n1[p] *= 0x1p600; n2[p] *= 0x1p600; }
            }
#pragma unroll
            for (int p = 0; p < 6; ++p) { q1[p] = n1[p] * il; n2[p] *= il; }
            if (D.tt_inf) q1[2] = 0.0;
            if (mode == MODE_HESS) {
#pragma unroll
                for (int p = 0; p < 6; ++p) q2[p] = n2[p] - q1[p] * q1[p];
                if (D.tt_inf) q2[2] = 0.0;
            }
        }
        if (c.fp32c) {
            // column weight g^ = log2(B / lambda_n) - t~_n (t~_n as packed), formed in logs
            const float *f = reinterpret_cast<const float *>(ws.src32);
            const float tt_n = -f[8 * (i >> 1) + 4 + (i & 1)];
            ghat = (float)((D.log2_b - ll * LOG2E) - (double)tt_n);
        } else {
            ws.w64[i] = D.ln_b - ll;  // log(B / lambda_n)
        }
    } else {
        atomicOr(&ws.hdr[0], ST_ZERO);
        if (!c.fp32c) ws.w64[i] = -INFINITY;  // weight 0
    }

    acc[0] = ll;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        acc[1 + p] = q1[p];
        acc[7 + p] = q2[p];
    }
    if (INTEGRAL) integral_row(D, in, ws, i, acc);
    if (lam <= 0.0) acc[0] = 0.0;  // the status carries the -inf
}

__host__ __device__ constexpr bool row_mom_used(int mode, int k) {
    return mode == MODE_HESS ? true
         : mode == MODE_GRAD ? (k == MO_G || k == MO_GD2 || k == MO_GT2 || k == MO_E || k == MO_ET || k == MO_ED2)
                             : (k == MO_G || k == MO_E);
}

// The FP64 fix-up of a row whose FP32 background and excitation sums are both
// below 2^-60 (terms under 2^-126 were flushed to zero in FP32): the calling
// warp recomputes row `row` over all sources in FP64; every lane returns the
// warp's sums in a (a fixed butterfly), in the FP32C scaled units as
// accumulate64 forms them.  A term more than 2^80 below the row's largest term
// of its kind cannot change the FP64 sum, so an FP32 pass over the packed
// sources first finds the largest background and excitation exponents (base
// 2, as the row pass forms them); the FP64 pass then evaluates only the terms
// within 2^80 of them.  (FP32 exponents are off by far less than 80 units, and
// FP64 coordinates keep the kept terms exact where FP32 ones would cost a far
// pair its relative accuracy.)
__device__ __forceinline__ void fixup_row64(const Consts &c, const Inputs &in, const Workspace &ws, int row,
                                            double (&a)[NMOM]) {
    const Derived &D = *c.d;
    const int n = c.g.n;
    const int lane = threadIdx.x & 31;
    const float *f = reinterpret_cast<const float *>(ws.src32);
    const float cbt = D.cbt, hh = D.hh;
    constexpr float KEEP = 80.0f;
    const int pr = row >> 1, lr = row & 1;
    const float xn = -f[8 * pr + lr], yn = -f[8 * pr + 2 + lr], tn = -f[8 * pr + 4 + lr];
    const int locn = ws.loc[row], gn = ws.gidx[row];
    float mg = -INFINITY, me = -INFINITY;
    for (int j = lane; j < n; j += 32) {
        const int p = j >> 1, l = j & 1;
        const float dx = xn + f[8 * p + l], dy = yn + f[8 * p + 2 + l], dt = tn + f[8 * p + 4 + l];
        const float d2 = dx * dx + dy * dy;
        if (ws.loc[j] != locn) mg = fmaxf(mg, -(d2 + cbt * dt * dt));
        // FP32C_ST: the causal test compares time-order ranks
        if ((c.st ? ws.perm[j] : j) < gn) me = fmaxf(me, f[8 * p + 6 + l] - tn - hh * d2);
    }
    mg = warp_maxf(mg);
    me = warp_maxf(me);
    const double xn64 = in.x[row], yn64 = in.y[row], tn64 = in.t[row];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) a[k] = 0.0;
    for (int j = lane; j < n; j += 32) {
        const int p = j >> 1, l = j & 1;
        const float dx = xn + f[8 * p + l], dy = yn + f[8 * p + 2 + l], dt = tn + f[8 * p + 4 + l];
        const float d2 = dx * dx + dy * dy;
        const bool bg_on = ws.loc[j] != locn && -(d2 + cbt * dt * dt) > mg - KEEP;
        const bool ex_on = (c.st ? ws.perm[j] : j) < gn && f[8 * p + 6 + l] - tn - hh * d2 > me - KEEP;
        if (bg_on || ex_on)
            accumulate64<MODE_HESS>(a, in.x[j], in.y[j], in.t[j], in.r[j], bg_on, ex_on, xn64, yn64, tn64, D);
    }
#pragma unroll
    for (int k = 0; k < NMOM; ++k) {
        double v = a[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        a[k] = v;
    }
}

// FP32C: the rows of target tile `tile`, finished by one block of TILE
// threads (one row each) after the row pass:
//   * the chunk partials summed in FP64 in chunk order;
//   * rows whose FP32 background and excitation sums are both below 2^-60
//     (terms under 2^-126 were flushed to zero in FP32) redone in FP64 over
//     all sources, the block cooperating on one row at a time;
//   * the row epilogue, the tile's 13 block sums, and the tile (and, on
//     space-time tiles, group) maxima of the column weight g^.  (Problems of
//     fewer than FIN_GROUP_TILES space-time tiles use finish_group_st.)
__device__ __forceinline__ void finish_tile_fp32c(const Consts &c, const Inputs &in, const Workspace &ws, int tile) {
    const Derived &D = *c.d;
    __shared__ double fsh[TILE];
    __shared__ float fshf[TILE];
    __shared__ int ftiny[TILE];
    __shared__ int fcnt[TILE / 32];
    const int i = tile * TILE + threadIdx.x;
    const int n = c.g.n, npad = c.g.npad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool valid = i < n;
    // The chunk partials are FP32 Kahan pairs (sum, -compensation); they are
    // summed in chunk order in float-float arithmetic (Knuth's two-sum for the
    // leading part, the low parts and rounding errors carried in a second
    // float), about 2^-44 relative, and only the total is made FP64: FP64
    // additions cost an SM's FP64 pipe about 19 cycles per warp instruction.
    // Chunks outer, moments inner: each chunk's loads of all moments are in
    // flight together (the order of each moment's sum is unchanged).
    const float2 *part = reinterpret_cast<const float2 *>(ws.rowpart);
    float hi[NMOM], lo[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) { hi[k] = 0.0f; lo[k] = 0.0f; }
    if (valid) {
#pragma unroll 2
        for (int ch = 0; ch < c.g.n_chunks; ++ch) {
            float2 v[NMOM];
#pragma unroll
            for (int k = 0; k < NMOM; ++k)
                if (row_mom_used(c.mode, k)) v[k] = part[((size_t)ch * NMOM + k) * npad + i];
#pragma unroll
            for (int k = 0; k < NMOM; ++k) {
                if (!row_mom_used(c.mode, k)) continue;
                const float s = __fadd_rn(hi[k], v[k].x);
                const float bb = __fsub_rn(s, hi[k]);
                const float err = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(s, bb)), __fsub_rn(v[k].x, bb));
                hi[k] = s;
                lo[k] = __fadd_rn(lo[k], __fadd_rn(err, v[k].y));
            }
        }
    }
    double Mo[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) Mo[k] = (double)hi[k] + (double)lo[k];
    // rows to redo in FP64, listed in thread order
    const bool tiny = valid && Mo[MO_G] < (double)TINY_ROW && Mo[MO_E] < (double)TINY_ROW;
    const unsigned bal = __ballot_sync(0xffffffffu, tiny);
    if (lane == 0) fcnt[warp] = __popc(bal);
    __syncthreads();
    int off = 0, ntiny = 0;
#pragma unroll
    for (int w = 0; w < TILE / 32; ++w) {
        if (w < warp) off += fcnt[w];
        ntiny += fcnt[w];
    }
    if (tiny) ftiny[off + __popc(bal & ((1u << lane) - 1u))] = threadIdx.x;
    __syncthreads();
    if (ntiny > 0) {
        // One warp per listed row (fixup_row64).
        __shared__ double fmom[TILE][NMOM];  // in the FP32C scaled units, as accumulate64 forms them
        for (int q = warp; q < ntiny; q += TILE / 32) {
            const int owner = ftiny[q];
            double a[NMOM];
            fixup_row64(c, in, ws, tile * TILE + owner, a);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < NMOM; ++k) fmom[owner][k] = a[k];
            }
        }
        __syncthreads();
        if (tiny) {
#pragma unroll
            for (int k = 0; k < NMOM; ++k) Mo[k] = fmom[threadIdx.x][k];
        }
    }
    double acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
    float ghat = -INFINITY;
    if (valid) epilogue_row<false>(c, D, in, ws, i, Mo, acc, ghat);  // the integral term came with the row pass
    pack_target(ws, in, D, i, c.g.n, ghat);  // the column pass's packed target
    {
        const double v = block_sum_multi<TILE, NACC>(acc, fsh);
        if (threadIdx.x < NACC)
            ws.blockpart[(size_t)tile * ACC_STRIDE + threadIdx.x] =
                v + (((ws.ipart[((size_t)tile * 4 + 0) * ACC_STRIDE + threadIdx.x] +
                       ws.ipart[((size_t)tile * 4 + 1) * ACC_STRIDE + threadIdx.x]) +
                      ws.ipart[((size_t)tile * 4 + 2) * ACC_STRIDE + threadIdx.x]) +
                     ws.ipart[((size_t)tile * 4 + 3) * ACC_STRIDE + threadIdx.x]);
    }
    if (c.st) {  // per-group bound for the column pass's pruning
        const float wm = warp_maxf(ghat);
        if (lane == 0) ws.grp[i / GROUP].tr.w = wm;
    }
    const float gm = block_max<TILE>(ghat, fshf);
    if (threadIdx.x == 0) ws.tstat32[tile].w = gm;
}

// FP32C_ST with fewer than FIN_GROUP_TILES tiles: the rows of target group `g`
// (32 rows), finished by one block of
// FG_WARPS warps after the row pass (four times the blocks of a per-tile
// finish, each a quarter of the chunk loads deep):
//   * warp s sums, for all 32 rows, the chunk partials of the contiguous chunk
//     range [s C / 4, (s + 1) C / 4) in chunk order in float-float, and warp 0
//     adds the four ranges in order (two-sum of the leading parts, the low
//     parts and rounding errors carried in the second float, as above);
//   * rows whose FP32 background and excitation sums are both below 2^-60
//     redone in FP64, one warp per row (fixup_row64);
//   * warp 0: the row epilogue, the packed column targets, the group's 13 sums
//     (a fixed butterfly) plus its integral shares into blockpart[g], and the
//     group maximum of g^ for the column pass's pruning.  The finalize sums
//     blockpart over the groups in order.
constexpr int FG_WARPS = 4;

__device__ __forceinline__ void finish_group_st(const Consts &c, const Inputs &in, const Workspace &ws, int g) {
    const Derived &D = *c.d;
    __shared__ float fhi[FG_WARPS][NMOM][GROUP], flo[FG_WARPS][NMOM][GROUP];
    __shared__ double fmom[GROUP][NMOM];
    __shared__ int ftiny[GROUP];
    __shared__ int fntiny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = g * GROUP + lane;
    const int n = c.g.n, npad = c.g.npad;
    const bool valid = i < n;
    {
        const int nc = c.g.n_chunks;
        const int c0 = warp * nc / FG_WARPS, c1 = (warp + 1) * nc / FG_WARPS;
        const float2 *part = reinterpret_cast<const float2 *>(ws.rowpart);
        float hi[NMOM], lo[NMOM];
#pragma unroll
        for (int k = 0; k < NMOM; ++k) { hi[k] = 0.0f; lo[k] = 0.0f; }
        if (valid) {
#pragma unroll 2
            for (int ch = c0; ch < c1; ++ch) {
                float2 v[NMOM];
#pragma unroll
                for (int k = 0; k < NMOM; ++k)
                    if (row_mom_used(c.mode, k)) v[k] = part[((size_t)ch * NMOM + k) * npad + i];
#pragma unroll
                for (int k = 0; k < NMOM; ++k) {
                    if (!row_mom_used(c.mode, k)) continue;
                    const float s = __fadd_rn(hi[k], v[k].x);
                    const float bb = __fsub_rn(s, hi[k]);
                    const float err = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(s, bb)), __fsub_rn(v[k].x, bb));
                    hi[k] = s;
                    lo[k] = __fadd_rn(lo[k], __fadd_rn(err, v[k].y));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NMOM; ++k) {
            fhi[warp][k][lane] = hi[k];
            flo[warp][k][lane] = lo[k];
        }
    }
    __syncthreads();
    double Mo[NMOM];
    bool tiny = false;
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NMOM; ++k) {
            float h = fhi[0][k][lane], l = flo[0][k][lane];
#pragma unroll
            for (int q = 1; q < FG_WARPS; ++q) {
                const float b = fhi[q][k][lane];
                const float s = __fadd_rn(h, b);
                const float bb = __fsub_rn(s, h);
                const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(b, bb));
                h = s;
                l = __fadd_rn(l, __fadd_rn(err, flo[q][k][lane]));
            }
            Mo[k] = (double)h + (double)l;
        }
        tiny = valid && Mo[MO_G] < (double)TINY_ROW && Mo[MO_E] < (double)TINY_ROW;
        const unsigned bal = __ballot_sync(0xffffffffu, tiny);
        if (tiny) ftiny[__popc(bal & ((1u << lane) - 1u))] = lane;
        if (lane == 0) fntiny = __popc(bal);
    }
    __syncthreads();
    const int ntiny = fntiny;
    if (ntiny > 0) {
        for (int q = warp; q < ntiny; q += FG_WARPS) {
            const int owner = ftiny[q];
            double a[NMOM];
            fixup_row64(c, in, ws, g * GROUP + owner, a);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < NMOM; ++k) fmom[owner][k] = a[k];
            }
        }
        __syncthreads();
        if (warp == 0 && tiny) {
#pragma unroll
            for (int k = 0; k < NMOM; ++k) Mo[k] = fmom[lane][k];
        }
    }
    if (warp != 0) return;  // no block barrier below
    double acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
    float ghat = -INFINITY;
    if (valid) epilogue_row<false>(c, D, in, ws, i, Mo, acc, ghat);  // the integral term came with the row pass
    pack_target(ws, in, D, i, n, ghat);
    const double w = warp_sum_scatter<NACC>(acc);  // lane 2k holds the group's sum k
    if ((lane & 1) == 0 && (lane >> 1) < NACC) {
        const int k = lane >> 1;
        ws.blockpart[(size_t)g * ACC_STRIDE + k] = w + ws.ipart[(size_t)g * ACC_STRIDE + k];
    }
    const float wm = warp_maxf(ghat);
    if (lane == 0) ws.grp[g].tr.w = wm;
}

// FP32C: the integral-term shares of one group of 32 events (FP64), summed
// over the group by the calling warp into ipart[group], with dLambda/dr per
// event.  Called by the row blocks of one source chunk after their pair loops,
// so this FP64 work runs beside other blocks' FP32 pair arithmetic instead of
// in the finish kernel.  Every lane of the warp calls it.
static __device__ __noinline__ void integral_group(const Consts &c, const Inputs &in, const Workspace &ws, int group) {
    const Derived &D = *c.d;
    const int i = group * GROUP + (threadIdx.x & 31);
    double a[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) a[k] = 0.0;
    if (i < c.g.n) integral_row(D, in, ws, i, a);
    const double v = warp_sum_scatter<NACC>(a);
    const int lane = threadIdx.x & 31;
    if ((lane & 1) == 0 && (lane >> 1) < NACC) ws.ipart[(size_t)group * ACC_STRIDE + (lane >> 1)] = v;
}

}  // namespace hk
