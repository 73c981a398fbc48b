// FP32C row-pass pair arithmetic shared by the time-order and space-time row
// kernels (k_row32.cu, k_row32_st.cu): the pair terms of Eq. 1's inner sum
// and their moments, two sources per packed f32x2 instruction.
#pragma once

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

}  // namespace hk
