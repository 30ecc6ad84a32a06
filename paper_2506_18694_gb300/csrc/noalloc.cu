// hh_multidot_noalloc: the FP64 multi-vector inner product x^H y of the outer Krylov
// iteration, for callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc at the point of use - a serving
// loop that has already handed all free device memory to its own pool, a caller that
// runs under a fixed memory budget it reserved up front, or a caller that has no
// hh_problem (whose creation allocates the Krylov basis) and only wants the reduction.
// The regular path keeps its block partial sums in memory owned by an hh_problem; this
// entry point keeps them in a fixed array compiled into the library instead.
#include <mutex>

#include "hh.h"
#include "internal.h"

namespace {

constexpr int kNoAllocMaxVectors = 64;
constexpr int kMaxDevices = 64;

// Block partial sums: kNoAllocMaxVectors x kRedBlocks complex doubles (304 KiB).  Every
// GPU that loads the library holds this array until the process exits.  Each call
// overwrites every entry it reads (the partial kernel writes all nvec x kRedBlocks
// slots before the final kernel reads them), so nothing has to be cleared between calls.
static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocMaxVectors * hh::kRedBlocks];

std::mutex g_mu;
double2* g_ptr[kMaxDevices] = {};

// Device address of g_noalloc_partials on the current device (looked up once per device).
cudaError_t partials_on_current_device(double2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = static_cast<double2*>(p);
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" hh_status hh_multidot_noalloc(const void* V, long long ld, int nvec, const void* w, long long n,
                                         void* out, void* cuda_stream) {
    if (!V || !w || !out) {
        hh::set_last_error("hh_multidot_noalloc: null pointer");
        return HH_ERR_INVALID;
    }
    if (nvec < 1 || nvec > kNoAllocMaxVectors) {
        hh::set_last_error("hh_multidot_noalloc: nvec must be in 1..64 (the static scratch holds 64 vectors)");
        return HH_ERR_INVALID;
    }
    if (n < 0 || ld < n) {
        hh::set_last_error("hh_multidot_noalloc: need n >= 0 and ld >= n");
        return HH_ERR_INVALID;
    }
    double2* partials = nullptr;
    cudaError_t e = partials_on_current_device(&partials);
    if (e == cudaSuccess)
        e = hh::launch_multidot(static_cast<const double2*>(V), ld, nvec, static_cast<const double2*>(w), n,
                                partials, static_cast<double2*>(out), hh::KBatch{1, 0, 0, 0, nullptr},
                                (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        hh::set_last_error(cudaGetErrorString(e));
        return HH_ERR_CUDA;
    }
    return HH_OK;
}
