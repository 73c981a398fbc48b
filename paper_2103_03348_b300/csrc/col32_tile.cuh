// FP32C column-pass pair arithmetic shared by the time-order and space-time
// column kernels (k_col32.cu, k_col32_st.cu): the terms of Eqs. 4 and 5 for
// one source against two targets per packed f32x2 instruction.
#pragma once

#include "hawkes_internal.cuh"

namespace hk {

// Coordinates are the excitation's scaled ones, x' = (x - xc) sxh, so that the
// term is v = 2^(g^_n + r^_m - d'^2): per target pair three packed adds and
// two packed FMAs form -log2 v = d'^2 - g^_n - r^_m (the targets carry -g^_n,
// the source -r^_m), and the exp2 takes its negation.
template <int MODE, bool MASK>
__device__ __forceinline__ void col_tile(const float4 *sAB, const int *sG, int npairs, float2 xm, float2 ym,
                                         float2 nrm, int m, float2 &c1, float2 &c2) {
#pragma unroll 8
    for (int p = 0; p < npairs; ++p) {
        const float4 A = sAB[2 * p], B = sAB[2 * p + 1];  // (-x', -y') and (-t~, -g^) of targets 2p, 2p+1
        const float2 dx = add2(xm, make_float2(A.x, A.y));
        const float2 dy = add2(ym, make_float2(A.z, A.w));
        float2 nl = add2(make_float2(B.z, B.w), nrm);
        nl = fma2(dy, dy, nl);
        nl = fma2(dx, dx, nl);
        float2 v = make_float2(ex2_ftz(-nl.x), ex2_ftz(-nl.y));
        if (MASK) {
            // target n is excited by m iff m < gidx[n] (strictly earlier time)
            if (!(m < sG[2 * p])) v.x = 0.0f;
            if (!(m < sG[2 * p + 1])) v.y = 0.0f;
        }
        c1 = add2(c1, v);
        if (MODE == MODE_HESS) c2 = fma2(v, v, c2);
    }
}

}  // namespace hk
