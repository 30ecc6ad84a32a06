// 2D pre-smoothing fused with the residual restriction: the two pre-sweeps of a level (from
// x = 0, or the HSS right side and its two sweeps on the finest level) and r_c = P^T (b - A x)
// in one pass.  One warp owns a strip of fine columns and CR coarse rows; it forms each stage
// on a halo one row and one lane wider than the next needs, keeps everything in registers,
// writes the smoothed x (and the HSS right side) on its own fine rows and columns, and the
// restricted residual on its own coarse nodes.  Every node's arithmetic is that of the
// one-stage kernels (march2.cu), so the result equals the separate passes bit for bit.
#include "internal.h"
#include "march2_common.cuh"

namespace hh {

// grid (strips, ceil(chunks / 4), problems); chunk = CR coarse rows
template <typename T, int MODE, int CR, bool BATCH>
__global__ void __launch_bounds__(128) k_march2rr(const __grid_constant__ MArgs<T> a, int chunks) {
    pdl_entry();
    const int b = BATCH ? (int)blockIdx.z : 0;
    const int cy = blockIdx.y * 4 + (threadIdx.x >> 5);
    if (cy >= chunks) return;
    if (BATCH && problem_skipped(a, b)) return;
    rr_tile<T, MODE, CR, BATCH>(a, b, blockIdx.x, cy);
}

template <typename T, int MODE>
static cudaError_t gorr(MArgs<T> a, cudaStream_t s) {
    using G1 = RRGeo<MODE, 1>;
    if (a.pc && !a.pc2) return cudaErrorInvalidValue;
    const int nnc = a.g.n / 2 + 1;
    const int strips = (a.g.nn + G1::S - 1) / G1::S;
    // two coarse rows per tile (fewer halo rows recomputed per output) once there are enough tiles
    // to fill the SMs: 24 warps per SM, 16 for the HSS pass, whose first stage is the widest
    // (measured on the 513^2 V-cycle: 43.27 us with two rows, 43.52 with one)
    const long long want = (MODE == M_HSS_FIRST2_RR ? 16LL : 24LL) * num_sms();
    int cr = ((long long)strips * ((nnc + 1) / 2) * a.nb >= want) ? 2 : 1;
    if (a.tile_rows == 1 || a.tile_rows == 2) cr = a.tile_rows;
    const int chunks = (nnc + cr - 1) / cr;
    const dim3 grd((unsigned)strips, (unsigned)((chunks + 3) / 4), (unsigned)a.nb);
    if (a.pc) {
        if (cr == 2) return klaunch(k_march2rr<T, MODE, 2, true>, grd, dim3(128), 0, s, 1, a, chunks);
        return klaunch(k_march2rr<T, MODE, 1, true>, grd, dim3(128), 0, s, 1, a, chunks);
    }
    if (a.nb != 1) return cudaErrorInvalidValue;
    if (cr == 2) return klaunch(k_march2rr<T, MODE, 2, false>, grd, dim3(128), 0, s, 1, a, chunks);
    return klaunch(k_march2rr<T, MODE, 1, false>, grd, dim3(128), 0, s, 1, a, chunks);
}

template <typename T>
cudaError_t launch_march2rr(int mode, const MArgs<T>& a, cudaStream_t s) {
    if (a.g.dim != 2 || a.g.n < 2 || (a.g.n & 1)) return cudaErrorInvalidValue;
    MArgs<T> b = a;
    b.h = T(a.g.h);
    b.ih = T(1.0 / a.g.h);
    switch (mode) {
        case M_JACOBI2_ZERO_RR: return gorr<T, M_JACOBI2_ZERO_RR>(b, s);
        case M_HSS_FIRST2_RR: return gorr<T, M_HSS_FIRST2_RR>(b, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_march2rr<float>(int, const MArgs<float>&, cudaStream_t);
template cudaError_t launch_march2rr<double>(int, const MArgs<double>&, cudaStream_t);

}  // namespace hh
