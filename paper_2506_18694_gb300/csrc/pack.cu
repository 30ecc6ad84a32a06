// Packed passes: one launch runs one pass of the V-cycle (Def. 4.1's inner A_L solve) for
// several independent 2D problems of DIFFERENT grids at once.  Problem m's arguments of every
// pass are its persistent-loop plan (HssLoop2, in device memory: the same buffers and
// coefficients its own kernels would use); its tiles of the pass occupy the tile numbers
// starts[m] .. starts[m + 1] - 1 of the launch, so a warp (or, for the coarsest level, a
// CTA) finds its problem by a binary search in the prefix table.  Each tile is computed by the
// device functions the single-problem kernels use, so every node of every problem gets the
// same bits as in a launch of its own.  A problem takes part in a launch when live[m] is set
// and the HSS step `it` is one of its steps.
#include "internal.h"
#include "march2_common.cuh"

namespace hh {

namespace {

// the last m with starts[m] <= t (starts nondecreasing, starts[0] = 0)
__device__ __forceinline__ int find_member(const int* starts, int nm, int t) {
    int lo = 0, hi = nm - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace

// pre-smoothing + restriction passes: level 0 (the HSS right side, MODE M_HSS_FIRST2_RR) or
// level `level` >= 1 (two sweeps from 0, MODE M_JACOBI2_ZERO_RR); 4 warp tiles per CTA
template <typename T, int MODE>
__global__ void __launch_bounds__(128) k_pack_rr(const HssLoop2<T>* __restrict__ plans, const int* __restrict__ starts,
                                                 int nm, int level, int it, const int* __restrict__ live) {
    pdl_entry();
    const int t = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (t >= starts[nm]) return;
    const int m = find_member(starts, nm, t);
    const HssLoop2<T>& P = plans[m];
    if (!live[m] || it >= P.nsteps) return;
    const MArgs<T>& a = MODE == M_HSS_FIRST2_RR ? (it == 0 ? P.first : P.pre[0]) : P.pre[level];
    const int strips = P.pre_strips[level];
    const int r = t - starts[m];
    rr_tile<T, MODE, 1, false>(a, 0, r % strips, r / strips);
}

// prolongation + two sweeps on level `level`; 4 warp tiles per CTA
template <typename T>
__global__ void __launch_bounds__(128) k_pack_f(const HssLoop2<T>* __restrict__ plans, const int* __restrict__ starts,
                                                int nm, int level, int it, const int* __restrict__ live) {
    pdl_entry();
    const int t = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (t >= starts[nm]) return;
    const int m = find_member(starts, nm, t);
    const HssLoop2<T>& P = plans[m];
    if (!live[m] || it >= P.nsteps) return;
    const MArgs<T>& a = P.post[level];
    const int strips = P.post_strips[level];
    const int r = t - starts[m];
    const VPtrs<T> v = problem_ptrs(a, 0, false);
    TileF<T, 2> tl;
    tilef_load<T, M_PROLONG_JACOBI2, 2>(a, v, r % strips, r / strips, tl);
    tilef_compute<T, M_PROLONG_JACOBI2, 2>(a, a.c0, a.c02, v, r % strips, r / strips, tl);
}

// the coarsest level: one CTA per band of coarse_rows rows of one problem
template <typename T>
__global__ void __launch_bounds__(kCoarseThreads) k_pack_coarse(const HssLoop2<T>* __restrict__ plans,
                                                                const int* __restrict__ starts, int nm, int it,
                                                                const int* __restrict__ live) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = blockIdx.x;
    if (t >= starts[nm]) return;
    const int m = find_member(starts, nm, t);
    const HssLoop2<T>& P = plans[m];
    if (!live[m] || it >= P.nsteps) return;
    const MArgs<T>& a = P.coarse;
    const int R = P.coarse_rows;
    const int r0 = (t - starts[m]) * R;
    coarse_band2<T>(a, a.c0, 0, r0, min(r0 + R, a.g.nn), P.nu_coarse, smem_raw);
}

template <typename T>
cudaError_t prepare_pack() {
    return cudaFuncSetAttribute(k_pack_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLoopSmemMax);
}

template <typename T>
cudaError_t launch_pack_pass(int kind, const HssLoop2<T>* plans, const int* starts, int nm, int total, int level,
                             int it, const int* live, size_t smem, cudaStream_t s) {
    if (total <= 0) return cudaSuccess;
    const dim3 warps((unsigned)((total + 3) / 4));
    switch (kind) {
        case 0: return klaunch(k_pack_rr<T, M_HSS_FIRST2_RR>, warps, dim3(128), 0, s, 1, plans, starts, nm, 0, it, live);
        case 1:
            return klaunch(k_pack_rr<T, M_JACOBI2_ZERO_RR>, warps, dim3(128), 0, s, 1, plans, starts, nm, level, it, live);
        case 2:
            return klaunch(k_pack_coarse<T>, dim3((unsigned)total), dim3(kCoarseThreads), smem, s, 1, plans, starts, nm, it,
                           live);
        case 3: return klaunch(k_pack_f<T>, warps, dim3(128), 0, s, 1, plans, starts, nm, level, it, live);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t prepare_pack<float>();
template cudaError_t prepare_pack<double>();
template cudaError_t launch_pack_pass<float>(int, const HssLoop2<float>*, const int*, int, int, int, int, const int*,
                                             size_t, cudaStream_t);
template cudaError_t launch_pack_pass<double>(int, const HssLoop2<double>*, const int*, int, int, int, int,
                                              const int*, size_t, cudaStream_t);

}  // namespace hh
