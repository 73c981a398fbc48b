// Learned gradient surrogate: a 6 -> 128 -> 128 -> 6 tanh MLP with BF16 weights
// and FP32 accumulation, trained and evaluated by these kernels.
//
// It maps standardised sampler coordinates of the six globals to the
// standardised gradient of the log posterior there; the HMC driver uses it for
// surrogate leapfrog trajectories and keeps the exact likelihood for the
// Metropolis accept step.  The paper has no counterpart: this is the learned
// part asked of the build.
//
// Parameter layout (element offsets, one vector of PARAM_COUNT values; FP32
// master copy for Adam, BF16 working copy for the forward/backward passes):
//   W1 [128 x 6] @ 0, b1 [128] @ 768, W2 [128 x 128] @ 896, b2 [128] @ 17280,
//   W3 [6 x 128] @ 17408, b3 [6] @ 18176; 18182 values in all.
// Loss: mean over the batch and the six outputs of (y - target)^2.
#include <cuda_bf16.h>

#include "hawkes_internal.cuh"

namespace hk {

constexpr int MI = 6, MH = 128, MO = 6;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MH * MI, OFF_W2 = OFF_B1 + MH, OFF_B2 = OFF_W2 + MH * MH;
constexpr int OFF_W3 = OFF_B2 + MH, OFF_B3 = OFF_W3 + MO * MH, PARAM_COUNT = OFF_B3 + MO;
constexpr int SB = 8;           // samples per block: 32 blocks for a minibatch of 256
constexpr int W2_STRIDE = MH + 1;  // padded rows: row and column walks are bank-conflict free

constexpr size_t mlp_smem_bytes() {
    return sizeof(float) * ((size_t)MH * W2_STRIDE + SB * MI + 3 * SB * MH + SB * MO + MH);
}

__device__ __forceinline__ float bf(const __nv_bfloat16 *w, int i) { return __bfloat162float(w[i]); }

// One block: forward pass of SB samples; with BACKWARD, also the loss and the
// block's share of the gradient (written to part[blockIdx.x][PARAM_COUNT]).
template <bool BACKWARD>
__global__ void __launch_bounds__(MH) mlp_block_kernel(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ x,
                                                       const float *__restrict__ target, int64_t batch,
                                                       float *__restrict__ y_out, float *__restrict__ part,
                                                       float *__restrict__ loss_part) {
    extern __shared__ float sm[];
    float *W2s = sm;                       // [MH][W2_STRIDE]
    float *X = W2s + MH * W2_STRIDE;       // [SB][MI]
    float *H1 = X + SB * MI;               // [SB][MH]
    float *H2 = H1 + SB * MH;              // [SB][MH]
    float *G = H2 + SB * MH;               // [SB][MH] (dZ2, then dZ1)
    float *DY = G + SB * MH;               // [SB][MO]
    float *LS = DY + SB * MO;              // [MH] per-thread loss partials
    const int j = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * SB;
    const int ns = (int)min((int64_t)SB, batch - s0);

    for (int i = j; i < MH * MH; i += MH) W2s[(i / MH) * W2_STRIDE + (i % MH)] = bf(w, OFF_W2 + i);
    for (int i = j; i < SB * MI; i += MH) X[i] = (i / MI < ns) ? x[s0 * MI + i] : 0.0f;
    __syncthreads();

    // layer 1: thread j is hidden unit j
    {
        float w1[MI];
#pragma unroll
        for (int k = 0; k < MI; ++k) w1[k] = bf(w, OFF_W1 + j * MI + k);
        const float b1 = bf(w, OFF_B1 + j);
        for (int s = 0; s < SB; ++s) {
            float a = b1;
#pragma unroll
            for (int k = 0; k < MI; ++k) a = fmaf(w1[k], X[s * MI + k], a);
            H1[s * MH + j] = tanhf(a);
        }
    }
    __syncthreads();
    // layer 2
    {
        float acc[SB];
        const float b2 = bf(w, OFF_B2 + j);
#pragma unroll
        for (int s = 0; s < SB; ++s) acc[s] = b2;
        for (int k = 0; k < MH; ++k) {
            const float wk = W2s[j * W2_STRIDE + k];
#pragma unroll
            for (int s = 0; s < SB; ++s) acc[s] = fmaf(wk, H1[s * MH + k], acc[s]);
        }
#pragma unroll
        for (int s = 0; s < SB; ++s) H2[s * MH + j] = tanhf(acc[s]);
    }
    __syncthreads();
    // layer 3 (+ loss gradient)
    float lsum = 0.0f;
    for (int idx = j; idx < SB * MO; idx += MH) {
        const int s = idx / MO, o = idx % MO;
        float a = bf(w, OFF_B3 + o);
        for (int k = 0; k < MH; ++k) a = fmaf(bf(w, OFF_W3 + o * MH + k), H2[s * MH + k], a);
        if (s < ns) {
            if (!BACKWARD) y_out[(s0 + s) * MO + o] = a;
            if (BACKWARD) {
                const float d = a - target[(s0 + s) * MO + o];
                lsum = fmaf(d, d, lsum);
                DY[idx] = 2.0f * d / (float)(batch * MO);
            }
        } else if (BACKWARD) {
            DY[idx] = 0.0f;
        }
    }
    if (!BACKWARD) return;
    LS[j] = lsum;
    __syncthreads();
    if (j == 0) {
        float t = 0.0f;
        for (int i = 0; i < MH; ++i) t += LS[i];
        loss_part[blockIdx.x] = t;
    }
    float *P = part + (size_t)blockIdx.x * PARAM_COUNT;
    // dZ2 = (W3^T dY) * (1 - H2^2); dW3, db3
    {
        float w3[MO];
#pragma unroll
        for (int o = 0; o < MO; ++o) w3[o] = bf(w, OFF_W3 + o * MH + j);
        float gw3[MO] = {0, 0, 0, 0, 0, 0};
        for (int s = 0; s < SB; ++s) {
            float g = 0.0f;
            const float h2 = H2[s * MH + j];
#pragma unroll
            for (int o = 0; o < MO; ++o) {
                const float dy = DY[s * MO + o];
                g = fmaf(dy, w3[o], g);
                gw3[o] = fmaf(dy, h2, gw3[o]);
            }
            G[s * MH + j] = g * (1.0f - h2 * h2);
        }
#pragma unroll
        for (int o = 0; o < MO; ++o) P[OFF_W3 + o * MH + j] = gw3[o];
        if (j < MO) {
            float b = 0.0f;
            for (int s = 0; s < SB; ++s) b += DY[s * MO + j];
            P[OFF_B3 + j] = b;
        }
    }
    __syncthreads();
    // dW2[r][j] = sum_s dZ2[s][r] H1[s][j] (thread j owns column j: coalesced writes); db2
    {
        float h1c[SB];
#pragma unroll
        for (int s = 0; s < SB; ++s) h1c[s] = H1[s * MH + j];
        for (int r = 0; r < MH; ++r) {
            float a = 0.0f;
#pragma unroll
            for (int s = 0; s < SB; ++s) a = fmaf(G[s * MH + r], h1c[s], a);
            P[OFF_W2 + r * MH + j] = a;
        }
        float b = 0.0f;
        for (int s = 0; s < SB; ++s) b += G[s * MH + j];
        P[OFF_B2 + j] = b;
    }
    // dZ1[s][j] = (sum_r dZ2[s][r] W2[r][j]) (1 - H1[s][j]^2), into H2's buffer
    {
        float acc[SB];
#pragma unroll
        for (int s = 0; s < SB; ++s) acc[s] = 0.0f;
        for (int r = 0; r < MH; ++r) {
            const float wr = W2s[r * W2_STRIDE + j];
#pragma unroll
            for (int s = 0; s < SB; ++s) acc[s] = fmaf(G[s * MH + r], wr, acc[s]);
        }
        __syncthreads();  // every thread is done reading H2 (layer 3) and G as dZ2
#pragma unroll
        for (int s = 0; s < SB; ++s) {
            const float h1 = H1[s * MH + j];
            H2[s * MH + j] = acc[s] * (1.0f - h1 * h1);
        }
    }
    __syncthreads();
    // dW1, db1 (thread j owns hidden unit j)
    {
        float gw1[MI] = {0, 0, 0, 0, 0, 0};
        float b = 0.0f;
        for (int s = 0; s < SB; ++s) {
            const float dz = H2[s * MH + j];
            b += dz;
#pragma unroll
            for (int k = 0; k < MI; ++k) gw1[k] = fmaf(dz, X[s * MI + k], gw1[k]);
        }
#pragma unroll
        for (int k = 0; k < MI; ++k) P[OFF_W1 + j * MI + k] = gw1[k];
        P[OFF_B1 + j] = b;
    }
}

// grad[i] = sum over blocks of part[b][i] (fixed order); loss = sum of loss parts / (batch * MO)
__global__ void mlp_reduce_kernel(int nblocks, int64_t batch, const float *__restrict__ part,
                                  const float *__restrict__ loss_part, float *__restrict__ grad, float *__restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < PARAM_COUNT) {
        float a = 0.0f;
        for (int b = 0; b < nblocks; ++b) a += part[(size_t)b * PARAM_COUNT + i];
        grad[i] = a;
    }
    if (i == 0 && loss) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += loss_part[b];
        *loss = (float)(t / (double)(batch * MO));
    }
}

// Adam's bias corrections for step s (1-based), as hawkes_mlp_adam forms them.
static inline void adam_bias_corrections(float b1, float b2, int step, float *bc1, float *bc2) {
    *bc1 = 1.0f - powf(b1, (float)step);
    *bc2 = 1.0f - powf(b2, (float)step);
}

// Adam on the FP32 master weights; the BF16 working copy is rounded to nearest even.
__global__ void mlp_adam_kernel(int64_t count, float *__restrict__ wm, __nv_bfloat16 *__restrict__ wb,
                                float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g, float lr,
                                float b1, float b2, float eps, float bc1, float bc2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float w = wm[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        wm[i] = w;
        wb[i] = __float2bfloat16_rn(w);
    }
}

// The same Adam step with its step number, learning rate and bias corrections
// read from device memory (step = *step_dev + 1; table[2 (step - 1)], [+1]),
// so that a captured training graph replays with a fresh step each time.  A
// step beyond the table leaves the weights alone.
__global__ void mlp_adam_dev_kernel(int64_t count, float *__restrict__ wm, __nv_bfloat16 *__restrict__ wb,
                                    float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g,
                                    const float *__restrict__ lr_dev, const float *__restrict__ table, int max_steps,
                                    const int *__restrict__ step_dev, float b1, float b2, float eps) {
    const int s = *step_dev;
    if (s < 0 || s >= max_steps) return;
    const float lr = *lr_dev, bc1 = table[2 * s], bc2 = table[2 * s + 1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float w = wm[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        wm[i] = w;
        wb[i] = __float2bfloat16_rn(w);
    }
}

__global__ void step_advance_kernel(int *step) { *step += 1; }

// Surrogate gradient at one state, fused with the leapfrog momentum update:
//   z = (q - mu_q) / sd_q,  g = mu_g + A (q - mu_q) + sd_g * MLP(z),  p += a * g
// norm = [mu_q(6), sd_q(6), mu_g(6), sd_g(6), A(6x6 row-major)]: a linear
// model of the gradient plus the MLP's standardised residual.  Optionally
// writes g.
__global__ void __launch_bounds__(MH) surrogate_momentum_kernel(const __nv_bfloat16 *__restrict__ w,
                                                                const double *__restrict__ q, double *__restrict__ p,
                                                                double a, const double *__restrict__ norm,
                                                                double *__restrict__ g_out) {
    __shared__ float z[MI], h1[MH], h2[MH];
    const int j = threadIdx.x;
    if (j < MI) z[j] = (float)((q[j] - norm[j]) / norm[6 + j]);
    __syncthreads();
    float acc = bf(w, OFF_B1 + j);
#pragma unroll
    for (int k = 0; k < MI; ++k) acc = fmaf(bf(w, OFF_W1 + j * MI + k), z[k], acc);
    h1[j] = tanhf(acc);
    __syncthreads();
    acc = bf(w, OFF_B2 + j);
    for (int k = 0; k < MH; ++k) acc = fmaf(bf(w, OFF_W2 + j * MH + k), h1[k], acc);
    h2[j] = tanhf(acc);
    __syncthreads();
    if (j < MO) {
        float y = bf(w, OFF_B3 + j);
        for (int k = 0; k < MH; ++k) y = fmaf(bf(w, OFF_W3 + j * MH + k), h2[k], y);
        double g = norm[12 + j] + norm[18 + j] * (double)y;
#pragma unroll
        for (int k = 0; k < MI; ++k) g += norm[24 + j * MI + k] * (q[k] - norm[k]);
        if (g_out) g_out[j] = g;
        if (p) p[j] += a * g;
    }
}

// A whole surrogate leapfrog trajectory over the six globals in one block:
//   p += eps/2 g(q);  n_steps times { q += eps minv p;  p += eps g(q) },
// the last momentum step halved.  g is the surrogate gradient of
// surrogate_momentum_kernel, computed with the same operations in the same
// order, so the trajectory equals the sequence of surrogate_momentum and
// position launches bit for bit.  Each thread keeps its row of W2 in
// registers across the n_steps + 1 evaluations; W3 is staged in shared memory.
// DENSE: minv is a dense 6 x 6 inverse mass (row-major) and the position step
// is q += eps M^-1 p, summed as in the dense position kernel.
template <bool DENSE>
__global__ void __launch_bounds__(MH) surrogate_trajectory_kernel(const __nv_bfloat16 *__restrict__ w,
                                                                  const double *__restrict__ norm,
                                                                  double *__restrict__ q, double *__restrict__ p,
                                                                  const double *__restrict__ minv, double eps,
                                                                  int n_steps) {
    __shared__ float z[MI], h1[MH], h2[MH], w3s[MO * MH];
    __shared__ double qs[MI], ps[MI];
    const int j = threadIdx.x;
    float w2r[MH], w1r[MI];
#pragma unroll
    for (int k = 0; k < MH; ++k) w2r[k] = bf(w, OFF_W2 + j * MH + k);
#pragma unroll
    for (int k = 0; k < MI; ++k) w1r[k] = bf(w, OFF_W1 + j * MI + k);
    const float b1 = bf(w, OFF_B1 + j), b2 = bf(w, OFF_B2 + j);
    for (int i = j; i < MO * MH; i += MH) w3s[i] = bf(w, OFF_W3 + i);
    float b3 = 0.0f;
    double mi[DENSE ? MI : 1];
    if (j < MI) {
        qs[j] = q[j];
        ps[j] = p[j];
        b3 = bf(w, OFF_B3 + j);
        if (DENSE) {
#pragma unroll
            for (int i = 0; i < MI; ++i) mi[i] = minv[j * MI + i];
        } else {
            mi[0] = minv[j];
        }
    }
    __syncthreads();
    for (int step = 0; step <= n_steps; ++step) {
        if (j < MI) z[j] = (float)((qs[j] - norm[j]) / norm[6 + j]);
        __syncthreads();
        float acc = b1;
#pragma unroll
        for (int k = 0; k < MI; ++k) acc = fmaf(w1r[k], z[k], acc);
        h1[j] = tanhf(acc);
        __syncthreads();
        acc = b2;
#pragma unroll
        for (int k = 0; k < MH; ++k) acc = fmaf(w2r[k], h1[k], acc);
        h2[j] = tanhf(acc);
        __syncthreads();
        if (j < MO) {  // threads 0..5: one warp, so __syncwarp orders their shared-memory updates
            float y = b3;
            for (int k = 0; k < MH; ++k) y = fmaf(w3s[j * MH + k], h2[k], y);
            double g = norm[12 + j] + norm[18 + j] * (double)y;
#pragma unroll
            for (int k = 0; k < MI; ++k) g += norm[24 + j * MI + k] * (qs[k] - norm[k]);
            const double a = (step == 0 || step == n_steps) ? 0.5 * eps : eps;
            __syncwarp(0x3fu);  // every g is formed from the old q before any q moves
            ps[j] += a * g;
            if (step < n_steps) {
                if (DENSE) {
                    __syncwarp(0x3fu);  // every p is updated before M^-1 p is formed
                    double v = 0.0;
#pragma unroll
                    for (int i = 0; i < MI; ++i) v += mi[i] * ps[i];
                    qs[j] += eps * v;
                } else {
                    qs[j] += eps * mi[0] * ps[j];
                }
            }
        }
        __syncthreads();
    }
    if (j < MI) {
        q[j] = qs[j];
        p[j] = ps[j];
    }
}

}  // namespace hk

extern "C" {

size_t hawkes_mlp_param_count(void) { return (size_t)hk::PARAM_COUNT; }

size_t hawkes_mlp_workspace_size(int64_t batch) {
    if (batch < 1) return 0;
    const int64_t nb = (batch + hk::SB - 1) / hk::SB;
    return (size_t)nb * (hk::PARAM_COUNT + 1) * sizeof(float) + 256;
}

static int mlp_launch(bool backward, const void *w, const float *x, const float *target, int64_t batch, float *y,
                      void *ws, size_t ws_bytes, float *grad, float *loss, void *stream) {
    if (batch < 1 || batch > ((int64_t)1 << 30) || !w || !x) return HAWKES_EINVAL;
    const int64_t nb = (batch + hk::SB - 1) / hk::SB;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = hk::mlp_smem_bytes();
    const __nv_bfloat16 *wb = (const __nv_bfloat16 *)w;
    if (!backward) {
        if (!y) return HAWKES_EINVAL;
        if (cudaFuncSetAttribute(hk::mlp_block_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return HAWKES_ECUDA;
        hk::mlp_block_kernel<false><<<(unsigned)nb, hk::MH, smem, s>>>(wb, x, nullptr, batch, y, nullptr, nullptr);
        return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
    }
    if (!target || !ws || !grad) return HAWKES_EINVAL;
    if (ws_bytes < hawkes_mlp_workspace_size(batch) || ((uintptr_t)ws & 255)) return HAWKES_EWORKSPACE;
    float *part = (float *)ws;
    float *loss_part = part + (size_t)nb * hk::PARAM_COUNT;
    if (cudaFuncSetAttribute(hk::mlp_block_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return HAWKES_ECUDA;
    hk::mlp_block_kernel<true><<<(unsigned)nb, hk::MH, smem, s>>>(wb, x, target, batch, nullptr, part, loss_part);
    if (cudaGetLastError() != cudaSuccess) return HAWKES_ECUDA;
    hk::mlp_reduce_kernel<<<(hk::PARAM_COUNT + 255) / 256, 256, 0, s>>>((int)nb, batch, part, loss_part, grad, loss);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_mlp_forward(const void *w_bf16, const float *x, int64_t batch, float *y, void *stream) {
    return mlp_launch(false, w_bf16, x, nullptr, batch, y, nullptr, 0, nullptr, nullptr, stream);
}

int hawkes_mlp_loss_grad(const void *w_bf16, const float *x, const float *target, int64_t batch, void *ws,
                         size_t ws_bytes, float *grad, float *loss, void *stream) {
    return mlp_launch(true, w_bf16, x, target, batch, nullptr, ws, ws_bytes, grad, loss, stream);
}

int hawkes_mlp_adam(float *w_master, void *w_bf16, float *m, float *v, const float *grad, float lr, float beta1,
                    float beta2, float eps, int step, void *stream) {
    if (!w_master || !w_bf16 || !m || !v || !grad || step < 1 || !(lr > 0)) return HAWKES_EINVAL;
    float bc1, bc2;
    hk::adam_bias_corrections(beta1, beta2, step, &bc1, &bc2);
    hk::mlp_adam_kernel<<<(hk::PARAM_COUNT + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        hk::PARAM_COUNT, w_master, (__nv_bfloat16 *)w_bf16, m, v, grad, lr, beta1, beta2, eps, bc1, bc2);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_mlp_adam_table(float beta1, float beta2, int steps, float *table) {
    if (steps < 1 || !table || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f))
        return HAWKES_EINVAL;
    for (int s = 1; s <= steps; ++s) hk::adam_bias_corrections(beta1, beta2, s, &table[2 * (s - 1)], &table[2 * s - 1]);
    return HAWKES_OK;
}

int hawkes_mlp_adam_device(float *w_master, void *w_bf16, float *m, float *v, const float *grad, const float *lr,
                           const float *table, int max_steps, int *step, float beta1, float beta2, float eps,
                           void *stream) {
    if (!w_master || !w_bf16 || !m || !v || !grad || !lr || !table || !step || max_steps < 1) return HAWKES_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    hk::mlp_adam_dev_kernel<<<(hk::PARAM_COUNT + 255) / 256, 256, 0, s>>>(
        hk::PARAM_COUNT, w_master, (__nv_bfloat16 *)w_bf16, m, v, grad, lr, table, max_steps, step, beta1, beta2, eps);
    if (cudaGetLastError() != cudaSuccess) return HAWKES_ECUDA;
    hk::step_advance_kernel<<<1, 1, 0, s>>>(step);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_surrogate_momentum(const void *w_bf16, const double *q, double *p, double a, const double *norm,
                              double *g_out, void *stream) {
    if (!w_bf16 || !q || !norm || (!p && !g_out)) return HAWKES_EINVAL;
    hk::surrogate_momentum_kernel<<<1, hk::MH, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)w_bf16, q, p, a,
                                                                          norm, g_out);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_surrogate_trajectory(const void *w_bf16, const double *norm, double *q, double *p, const double *minv,
                                double eps, int n_steps, void *stream) {
    if (!w_bf16 || !norm || !q || !p || !minv || n_steps < 0 || !(eps == eps)) return HAWKES_EINVAL;
    hk::surrogate_trajectory_kernel<false><<<1, hk::MH, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)w_bf16,
                                                                                   norm, q, p, minv, eps, n_steps);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

int hawkes_surrogate_trajectory_dense(const void *w_bf16, const double *norm, double *q, double *p,
                                      const double *minv, double eps, int n_steps, void *stream) {
    if (!w_bf16 || !norm || !q || !p || !minv || n_steps < 0 || !(eps == eps)) return HAWKES_EINVAL;
    hk::surrogate_trajectory_kernel<true><<<1, hk::MH, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)w_bf16,
                                                                                  norm, q, p, minv, eps, n_steps);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ECUDA;
}

}  // extern "C"
