// The exchange step of the sharded evaluation.
//
// The double sum splits by target rows for the intensities (Eq. 1 inner sum)
// and by source columns for the rate gradient (Eq. 4) and Hessian (Eq. 5); the
// column pass of a source needs the column weight B / lambda_n of every later
// target, and the log-likelihood and global derivatives need every row's
// partial sums.  So after its rows, a shard publishes one record per target
// tile it owns:
//   [0, NACC)      the tile's 13 partial sums (log-likelihood, gradient and
//                  Hessian diagonal of the six globals, in the epilogue's order)
//   [NACC]         the shard's status bits (bit pattern of an int)
//   [NACC + 1]     FP32C: the tile's largest column weight exponent g^ (float bits)
//   [16, 16 + TILE) the tile's column weights: FP32C g^_n = log2(B / lambda_n) - t~_n
//                  (float bits), FP64 log(B / lambda_n)
// An all-gather of the records gives every shard what the unsharded call
// holds after its row epilogue, so every per-tile kernel that follows sees
// identical inputs and the outputs match the unsharded call bit for bit.
#include "hawkes_internal.cuh"

namespace hk {

static_assert(16 + TILE == XREC_DOUBLES, "exchange record layout");
static_assert(NACC + 2 <= 16, "exchange record header");

__device__ __forceinline__ double float_bits(float v) { return __longlong_as_double((long long)__float_as_uint(v)); }
__device__ __forceinline__ float bits_float(double v) { return __uint_as_float((unsigned)__double_as_longlong(v)); }

// one block per owned tile
__global__ void __launch_bounds__(TILE) shard_export_kernel(Consts c, Workspace ws, double *__restrict__ xbuf) {
    pdl_wait();
    const int tile = c.t0 + blockIdx.x;
    double *rec = xbuf + (size_t)tile * XREC_DOUBLES;
    const int i = tile * TILE + threadIdx.x;
    if (threadIdx.x < NACC) rec[threadIdx.x] = ws.blockpart[(size_t)tile * ACC_STRIDE + threadIdx.x];
    if (threadIdx.x == NACC) rec[NACC] = __longlong_as_double((long long)ws.hdr[0]);
    if (threadIdx.x == NACC + 1) rec[NACC + 1] = c.fp32c ? float_bits(ws.tstat32[tile].w) : 0.0;
    if (c.fp32c) {
        const float *f = reinterpret_cast<const float *>(ws.tgt32);
        rec[16 + threadIdx.x] = float_bits(f[8 * (i >> 1) + 6 + (i & 1)]);  // -g^, as packed
    } else {
        rec[16 + threadIdx.x] = ws.w64[i];
    }
}

// one block per tile of the whole problem
__global__ void __launch_bounds__(TILE) shard_import_kernel(Consts c, Inputs in, Workspace ws,
                                                            const double *__restrict__ xbuf) {
    pdl_wait();
    const int tile = blockIdx.x;
    const double *rec = xbuf + (size_t)tile * XREC_DOUBLES;
    const int i = tile * TILE + threadIdx.x;
    if (threadIdx.x < NACC) ws.blockpart[(size_t)tile * ACC_STRIDE + threadIdx.x] = rec[threadIdx.x];
    if (threadIdx.x == NACC) {
        const int bits = (int)__double_as_longlong(rec[NACC]);
        if (bits) atomicOr(&ws.hdr[0], bits);
    }
    if (threadIdx.x == NACC + 1 && c.fp32c) ws.tstat32[tile].w = bits_float(rec[NACC + 1]);
    if (c.fp32c) {
        // the column pass's packed targets, as the tile finish writes them
        pack_target(ws, in, *c.d, i, c.g.n, -bits_float(rec[16 + threadIdx.x]));
    } else {
        ws.w64[i] = rec[16 + threadIdx.x];
    }
}

cudaError_t launch_shard_export(const Consts &c, const Workspace &ws, double *xbuf, cudaStream_t s) {
    if (c.t1 <= c.t0) return cudaSuccess;
    launch_pdl(shard_export_kernel, c.t1 - c.t0, TILE, 0, s, c, ws, xbuf);
    return cudaGetLastError();
}

cudaError_t launch_shard_import(const Consts &c, const Inputs &in, const Workspace &ws, const double *xbuf,
                                cudaStream_t s) {
    launch_pdl(shard_import_kernel, c.g.tiles, TILE, 0, s, c, in, ws, xbuf);
    return cudaGetLastError();
}

}  // namespace hk
