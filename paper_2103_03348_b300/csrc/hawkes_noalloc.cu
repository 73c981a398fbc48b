// hawkes_hess_diag_noalloc: the fused log-likelihood + gradient + Hessian
// diagonal with its scratch memory in a fixed, library-owned device array
// instead of a caller-provided workspace.
//
// Who needs it: a caller that cannot call cudaMalloc at evaluation time, for
// example a sampler plugin loaded into a host application that owns every
// device allocation (it gets device pointers for its data but no allocator),
// or a latency-sensitive loop where cudaMalloc's implicit synchronisation of
// the device is not acceptable.  Such a caller still owns and passes the
// inputs (x, y, t, r) and the outputs (loglik, grad, hdiag, dev_status).
//
// How: the scratch is the file-scope array below, sized for up to
// HAWKES_NOALLOC_MAX_EVENTS events at any precision (the largest workspace
// for n <= 4096 is 12.7 MiB).  Every GPU that loads the library holds these
// 16 MiB until the process exits.  Host code cannot use the array's name as a
// device address, so the first call on each device (with that device current)
// looks the address up with cudaGetSymbolAddress, checks it, and caches it;
// that first call should therefore come before any stream capture.  The
// cached address belongs to the device's context of that moment: a host
// program that calls cudaDeviceReset (which unloads this module's device copy
// of the array) must not call this entry point again in the same process.  The
// evaluation itself is hawkes_hess_diag with this array as its workspace; its
// first steps clear what has to start at zero (status words, the location hash
// table, the group counters) and every other byte is rewritten before it is
// read, so leftovers from the previous call do no harm.  All calls on a device
// share the one array: calls that can overlap on the GPU (different streams,
// or different host threads without ordering) race on it and must not be
// issued.  Nothing here allocates: no cudaMalloc, cudaFree or allocating
// library routine.
#include <mutex>

#include "hawkes_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];  // device address of g_scratch on each device, looked up once

}  // namespace

extern "C" int hawkes_hess_diag_noalloc(const double *x, const double *y, const double *t, const double *r,
                                        int64_t n, const double params[6], int precision, double *loglik,
                                        double *grad, double *hdiag, int *dev_status, void *stream) {
    if (n < 2) return HAWKES_EINVAL;
    if (n > HAWKES_NOALLOC_MAX_EVENTS) return HAWKES_ESCRATCH;
    const size_t need = hawkes_workspace_size(n, precision);
    if (need == 0) return HAWKES_EINVAL;
    if (need > kScratchBytes) return HAWKES_ESCRATCH;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HAWKES_ECUDA;
    void *addr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (g_scratch_addr[dev] == nullptr) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return HAWKES_ECUDA;
            g_scratch_addr[dev] = p;
        }
        addr = g_scratch_addr[dev];
    }
    return hawkes_hess_diag(x, y, t, r, n, params, precision, addr, kScratchBytes, loglik, grad, hdiag,
                            dev_status, stream);
}
