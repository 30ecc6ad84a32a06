// Launchers shared between the translation units of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace hh {

// Message returned by hh_last_error() for the calling thread.
void set_last_error(const char* msg);

// Kernels launched by this thread through the launchers below (graph captures included).
extern thread_local long long g_kernel_launches;
// 1: launch with programmatic stream serialization (overlaps a kernel's launch with the
// tail of its predecessor; every kernel starts with pdl_entry()).
extern thread_local int g_use_pdl;

#define HH_KRET(call)                        \
    do {                                     \
        cudaError_t e_ = (call);             \
        if (e_ != cudaSuccess) return e_;    \
    } while (0)

// Launch `kernel` on stream s (optionally as clusters of `cluster` CTAs along x).
template <typename... KArgs, typename... Args>
inline cudaError_t klaunch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                           int cluster, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    int na = 0;
    if (g_use_pdl) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    if (cluster > 1) {
        at[na].id = cudaLaunchAttributeClusterDimension;
        at[na].val.clusterDim.x = cluster;
        at[na].val.clusterDim.y = 1;
        at[na].val.clusterDim.z = 1;
        ++na;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    ++g_kernel_launches;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// rc = P^T rf (rf on the fine grid of gc)
template <typename T>
cudaError_t launch_restrict(const GridDesc& gc, const vec2<T>* rf, vec2<T>* rc, cudaStream_t s);

// x += P ec (ec on the coarse grid of gf)
template <typename T>
cudaError_t launch_prolong(const GridDesc& gf, const vec2<T>* ec, vec2<T>* x, cudaStream_t s);

// x += e elementwise
template <typename T>
cudaError_t launch_add(vec2<T>* x, const vec2<T>* e, long long N, cudaStream_t s);

// ---- coarsest level inside one thread-block cluster, in distributed shared memory (coarse.cu) ----
constexpr int kCoarseThreads = 512;
constexpr int kCoarseNodesPerThread = 2;
constexpr size_t kCoarseSmemMax = 200 * 1024;

// CTAs per cluster (16 or 8 when the device can co-schedule them, else 1)
int coarse_cluster_size();
// whether a grid's slabs fit the shared memory of the cluster's CTAs
template <typename T>
bool coarse_fits(const GridDesc& g);
// one-time set-up (shared-memory limit, cluster query); call before any stream capture
template <typename T>
cudaError_t prepare_coarse();
// nsweeps scaled-Jacobi sweeps on A x = b from x = 0
template <typename T>
cudaError_t launch_coarse_solve(const GridDesc& g, const OpCoef<T>& op, const vec2<T>* b, vec2<T>* x, int nsweeps,
                                T omega, cudaStream_t s);

// ---- fused 2D marching kernels (march2.cu) ----
enum MarchMode {
    M_APPLY = 0,          // y = op x
    M_AXPBY = 1,          // y = alpha (op x) + beta z
    M_JACOBI = 2,         // y = x + omega D^{-1} (z - op x),          D = diag(op)
    M_HSS_FIRST = 3,      // y = alpha (op x) + beta z;  y2 = omega diag(opd)^{-1} y
    M_JACOBI2_ZERO = 4,   // two sweeps from x = 0 reading only z:  x1 = omega D^{-1} z,
                          // y = x1 + omega D^{-1} (z - op x1)
    M_PROLONG_JACOBI = 5, // x~ = x + P ec;  y = x~ + omega D^{-1} (z - op x~)
    M_RESID_RESTRICT = 6  // y (coarse) = P^T (z - op x)
};

template <typename T> struct MArgs {
    GridDesc g;          // grid of the level the stencil runs on
    OpCoef<T> op;        // stencil operator
    OpCoef<T> opd;       // operator whose diagonal scales the HSS-first Jacobi step (A_L)
    const vec2<T>* x;    // stencil input (ignored for M_JACOBI2_ZERO; nullptr = 0 when xzero)
    const vec2<T>* z;    // right side / second vector
    const vec2<T>* ec;   // coarse correction (M_PROLONG_JACOBI)
    vec2<T>* y;          // output
    vec2<T>* y2;         // second output (M_HSS_FIRST)
    Cx<T> alpha, beta;
    T omega;
    int xzero;           // 1: x is identically zero
    int tile_rows;       // 0: automatic; else 2, 4 or 8 rows (2D) / planes (3D) per tile
    // filled by the launcher
    T h, ih;
    int rows;
    // interior stencil weights of op by neighbour class (how many coordinates differ from
    // the centre: 0 centre, 1 edge/face, 2 diagonal/edge, 3 corner in 3D)
    Cx<T> iw[4];
    Cx<T> wdinv;         // omega / (interior diagonal of opd)
};

// ---- fused 3D tile kernels (march3.cu): modes as above except M_RESID_RESTRICT ----
template <typename T>
cudaError_t launch_march3(int mode, const MArgs<T>& a, cudaStream_t s);
// interior weights (iw, wdinv) of a.op / a.opd on grid a.g (filled by the launchers)
template <typename T>
void interior_weights(MArgs<T>& a);

template <typename T>
cudaError_t launch_march2(int mode, const MArgs<T>& a, cudaStream_t s);

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
