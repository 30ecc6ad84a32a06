// Launchers shared between the translation units of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace hh {

// Kernels launched by this thread through the launchers below (graph captures included).
extern thread_local long long g_kernel_launches;

enum StencilMode {
    MODE_APPLY = 0,   // y = op x
    MODE_AXPBY = 1,   // y = alpha (op x) + beta z          (x == nullptr: op x = 0)
    MODE_JACOBI = 2   // y = x + omega D^{-1} (z - op x)    (x == nullptr: x = 0)
};

template <typename T>
cudaError_t launch_stencil(int mode, const GridDesc& g, const OpCoef<T>& op, const vec2<T>* x,
                           const vec2<T>* z, vec2<T>* y, Cx<T> alpha, Cx<T> beta, T omega,
                           cudaStream_t s);

// rc = P^T rf (rf on the fine grid of gc)
template <typename T>
cudaError_t launch_restrict(const GridDesc& gc, const vec2<T>* rf, vec2<T>* rc, cudaStream_t s);

// rc = P^T (b - A x); scratch holds the fine residual (fine-grid length)
template <typename T>
cudaError_t launch_residual_restrict(const GridDesc& gf, const GridDesc& gc, const OpCoef<T>& op,
                                     const vec2<T>* b, const vec2<T>* x, vec2<T>* rc,
                                     vec2<T>* scratch, cudaStream_t s);

// x += P ec (ec on the coarse grid of gf)
template <typename T>
cudaError_t launch_prolong(const GridDesc& gf, const vec2<T>* ec, vec2<T>* x, cudaStream_t s);

// x += e elementwise
template <typename T>
cudaError_t launch_add(vec2<T>* x, const vec2<T>* e, long long N, cudaStream_t s);

cudaError_t launch_cast_d2f(const double2* a, float2* b, long long N, cudaStream_t s);
cudaError_t launch_cast_f2d(const float2* a, double2* b, long long N, cudaStream_t s);
// dst = src with exact zeros at the Dirichlet nodes of g
cudaError_t launch_mask_copy(const GridDesc& g, const double2* src, double2* dst, cudaStream_t s);

// ---- FP64 Krylov kernels (blas.cu) ----
// Fixed reduction grid: results do not depend on timing or launch history.
constexpr int kRedBlocks = 304;
constexpr int kRedThreads = 256;

// out[i] = sum_p conj(V_i[p]) w[p] for i < nvec (V_i = V + i*ld); partials holds nvec*kRedBlocks
cudaError_t launch_multidot(const double2* V, long long ld, int nvec, const double2* w,
                            long long N, double2* partials, double2* out, cudaStream_t s);
// w[p] -= sum_i coef[i] V_i[p]    (sign = -1)   or   w[p] += sum_i coef[i] V_i[p] (sign = +1)
cudaError_t launch_multi_axpy(double2* w, const double2* V, long long ld, int nvec,
                              const double2* coef, double sign, long long N, cudaStream_t s);
// x *= 1 / sqrt(nrm2->x) (nrm2 on the device, skipped when zero)
cudaError_t launch_scale_by_rnorm(double2* x, const double2* nrm2, long long N, cudaStream_t s);
// x *= s
cudaError_t launch_scale(double2* x, double s, long long N, cudaStream_t st);

}  // namespace hh
