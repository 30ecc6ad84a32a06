// Persistent 2D shifted-HSS loop: every step of the preconditioner of Def. 4.1 (the HSS right
// side c1 A_R u + c2 r and one V(2,2) cycle on A_L) in ONE cooperative launch.
//
// At the sizes where the fused 2D passes are used (the whole hierarchy L2-resident) a V-cycle
// is a chain of small dependent passes and its time goes to launching them, not to memory
// traffic.  Here the resident CTAs walk the same warp tiles as the separate kernels (the same
// device functions, so every node is computed bit for bit as there), pass by pass, and meet
// at a grid-wide barrier between passes instead of ending the kernel.  Per HSS step:
//   level 0   HSS right side + two sweeps + restricted residual     (rr_tile, HSS mode)
//   level l   two sweeps from 0 + restricted residual, 1 <= l < L-1  (rr_tile)
//   coarsest  nu_coarse sweeps from 0: each CTA takes a band of rows, stages the band and a
//             halo of nu_coarse - 1 rows on each side in shared memory and runs all sweeps
//             there with block barriers only (the halo rows are recomputed, so no exchange
//             between CTAs is needed)
//   level l   prolongation + two sweeps, l = L-2 .. 0                (tilef_*, PROLONG mode)
// Every wait at a grid barrier is bounded: after spin_limit polls the CTA records
// HH_ERR_TIMEOUT in the status word and returns, and every other CTA returns at its next
// barrier when it sees a non-zero status.  A non-zero status on entry (an earlier launch
// failed and the host has not cleared it) makes the kernel return at once.
#include <mutex>

#include "hh.h"
#include "internal.h"
#include "march2_common.cuh"

namespace hh {

namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier number `epoch` (1, 2, ...) of the whole grid.  Thread 0 of each CTA publishes the
// CTA's writes (fence, then one arrival on the counter) and polls the counter with acquire
// loads; the block barrier after it orders the CTA's later reads after what the others wrote.
__device__ __forceinline__ bool grid_barrier(unsigned* count, int* status, unsigned epoch,
                                             unsigned long long spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = epoch * gridDim.x;
        __threadfence();
        atomicAdd(count, 1u);
        int ok = 1;
        unsigned long long polls = 0;
        while (ld_acquire_u32(count) < target) {
            if (ld_relaxed_s32(status) != 0) {
                ok = 0;
                break;
            }
            if (polls >= spin_limit) {
                atomicCAS(status, 0, (int)HH_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            ++polls;
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ bool loop_skipped(const MArgs<T>& a, int b, int it) {
    if (a.active && !a.active[b]) return true;
    return it >= a.nhss[b];
}

// rr_tile over every tile of a pass (CR = 1), warp-strided over the grid
template <typename T, int MODE, bool BATCH>
__device__ __forceinline__ void rr_pass(const MArgs<T>& a, int strips, int chunks, int it, int gw, int nw) {
    const int per = strips * chunks;
    const int tiles = per * a.nb;
    for (int t = gw; t < tiles; t += nw) {
        const int b = BATCH ? t / per : 0;
        if (BATCH && loop_skipped(a, b, it)) continue;
        const int r = t - b * per;
        rr_tile<T, MODE, 1, BATCH>(a, b, r % strips, r / strips);
    }
}

// prolongation + two sweeps (2-row tiles) over every tile of a pass
template <typename T, bool BATCH>
__device__ __forceinline__ void f_pass(const MArgs<T>& a, int strips, int chunks, int it, int gw, int nw) {
    const int per = strips * chunks;
    const int tiles = per * a.nb;
    for (int t = gw; t < tiles; t += nw) {
        const int b = BATCH ? t / per : 0;
        if (BATCH && loop_skipped(a, b, it)) continue;
        const int r = t - b * per;
        const PCoef<T>& c = BATCH ? a.pc[b] : a.c0;
        const PCoef<T>& cl = BATCH ? a.pc2[b] : a.c02;
        const VPtrs<T> v = problem_ptrs(a, b, false);
        TileF<T, 2> tl;
        tilef_load<T, M_PROLONG_JACOBI2, 2>(a, v, r % strips, r / strips, tl);
        tilef_compute<T, M_PROLONG_JACOBI2, 2>(a, c, cl, v, r % strips, r / strips, tl);
    }
}

// nsw scaled-Jacobi sweeps from 0 on the coarsest level, one band of R rows per CTA job
template <typename T, bool BATCH>
__device__ __forceinline__ void coarse_pass(const MArgs<T>& a, int nsw, int R, int it, unsigned char* smem) {
    const int nn = a.g.nn;
    const int bands = (nn + R - 1) / R;
    const int jobs = bands * a.nb;
    for (int job = blockIdx.x; job < jobs; job += gridDim.x) {
        const int b = BATCH ? job / bands : 0;
        if (BATCH && loop_skipped(a, b, it)) continue;  // uniform over the CTA
        const int r0 = (job - b * bands) * R;
        coarse_band2<T>(a, BATCH ? a.pc[b] : a.c0, b, r0, min(r0 + R, nn), nsw, smem);
        __syncthreads();  // before the next job overwrites the buffers
    }
}

}  // namespace

template <typename T, bool BATCH>
__global__ void __launch_bounds__(128) k_hss2p(const __grid_constant__ HssLoop2<T> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (ld_relaxed_s32(P.status) != 0) return;
    const int gw = blockIdx.x * 4 + (threadIdx.x >> 5), nw = gridDim.x * 4;
    const int L = P.levels;
    unsigned epoch = 0;
    for (int it = 0; it < P.nsteps; ++it) {
        rr_pass<T, M_HSS_FIRST2_RR, BATCH>(it == 0 ? P.first : P.pre[0], P.pre_strips[0], P.pre_chunks[0], it, gw,
                                           nw);
        if (!grid_barrier(P.count, P.status, ++epoch, P.spin_limit)) return;
        for (int l = 1; l < L - 1; ++l) {
            rr_pass<T, M_JACOBI2_ZERO_RR, BATCH>(P.pre[l], P.pre_strips[l], P.pre_chunks[l], it, gw, nw);
            if (!grid_barrier(P.count, P.status, ++epoch, P.spin_limit)) return;
        }
        coarse_pass<T, BATCH>(P.coarse, P.nu_coarse, P.coarse_rows, it, smem_raw);
        if (!grid_barrier(P.count, P.status, ++epoch, P.spin_limit)) return;
        for (int l = L - 2; l >= 0; --l) {
            f_pass<T, BATCH>(P.post[l], P.post_strips[l], P.post_chunks[l], it, gw, nw);
            if (it + 1 == P.nsteps && l == 0) break;  // the kernel's end orders the last pass
            if (!grid_barrier(P.count, P.status, ++epoch, P.spin_limit)) return;
        }
    }
}

template <typename T>
size_t hss_loop2_smem(const GridDesc& gc, int nu_coarse, int rows) {
    return band2_smem<T>(gc.nn, nu_coarse, rows);
}

template <typename T>
static auto hss2p_kernel(bool batch) {
    return batch ? k_hss2p<T, true> : k_hss2p<T, false>;
}

// The kernels' dynamic shared memory limit is raised once per process to kLoopSmemMax (the
// attribute belongs to the kernel, not to a launch: problems of different sizes on several
// threads must not lower it under each other).
template <typename T>
static bool raise_smem_limit() {
    static std::once_flag once;
    static bool ok = false;
    std::call_once(once, [] {
        ok = cudaFuncSetAttribute(k_hss2p<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kLoopSmemMax) == cudaSuccess &&
             cudaFuncSetAttribute(k_hss2p<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kLoopSmemMax) == cudaSuccess;
        if (!ok) cudaGetLastError();
    });
    return ok;
}

template <typename T>
int hss_loop2_ctas(bool batch, size_t smem) {
    auto kern = hss2p_kernel<T>(batch);
    if (smem > kLoopSmemMax || !raise_smem_limit<T>()) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    per_sm = per_sm > 4 ? 4 : per_sm;
    return per_sm * num_sms();
}

template <typename T>
cudaError_t launch_hss_loop2(const HssLoop2<T>& P, int ctas, size_t smem, cudaStream_t s) {
    if (ctas < 1 || P.levels < 2 || P.levels > kPMaxLevels) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(P.count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident at once, or the launch fails
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ++g_kernel_launches;
    return cudaLaunchKernelEx(&cfg, hss2p_kernel<T>(P.nb > 1 || P.first.pc != nullptr), P);
}

template size_t hss_loop2_smem<float>(const GridDesc&, int, int);
template size_t hss_loop2_smem<double>(const GridDesc&, int, int);
template int hss_loop2_ctas<float>(bool, size_t);
template int hss_loop2_ctas<double>(bool, size_t);
template cudaError_t launch_hss_loop2<float>(const HssLoop2<float>&, int, size_t, cudaStream_t);
template cudaError_t launch_hss_loop2<double>(const HssLoop2<double>&, int, size_t, cudaStream_t);

}  // namespace hh
