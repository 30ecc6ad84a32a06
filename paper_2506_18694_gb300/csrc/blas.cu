// FP64 complex vector kernels of the outer flexible GMRES (Sec. 5.1): block-partial
// inner products with a fixed reduction tree (bitwise reproducible), fused
// multi-vector updates for classical Gram-Schmidt, scaling by a device-held norm.
#include "internal.h"

namespace hh {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Block reduction of a double2 (warp shuffles, then one warp over the warp sums).
__device__ __forceinline__ double2 block_sum(double2 v) {
    __shared__ double2 warp_sums[32];
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(full, v.x, o);
        v.y += __shfl_down_sync(full, v.y, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_sums[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? warp_sums[lane] : make_double2(0.0, 0.0);
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_down_sync(full, v.x, o);
            v.y += __shfl_down_sync(full, v.y, o);
        }
    }
    return v;  // valid in thread 0
}

// partials[(b * nvec + i) * gridDim.x + blockIdx.x] = sum over this block's slice of conj(V_i) w
// for problem b = blockIdx.z.  grid = (kRedBlocks, nvec, problems); block slices are fixed so
// the sum order never changes.
__global__ void __launch_bounds__(kRedThreads) k_multidot_partial(const double2* __restrict__ V, long long ld,
                                                                  const double2* __restrict__ w, long long N,
                                                                  double2* __restrict__ partials, KBatch kb) {
    pdl_entry();
    const int vi = blockIdx.y, b = blockIdx.z;
    if (kb.active && !kb.active[b]) return;
    const double2* __restrict__ v = V + (long long)b * kb.bs_v + (long long)vi * ld;
    w += (long long)b * kb.bs_w;
    double2 acc = make_double2(0.0, 0.0);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += stride) {
        const double2 a = v[p], c = w[p];
        acc.x = fma(a.x, c.x, fma(a.y, c.y, acc.x));
        acc.y = fma(a.x, c.y, fma(-a.y, c.x, acc.y));
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[((long long)b * gridDim.y + vi) * gridDim.x + blockIdx.x] = acc;
}

// out[b * bs_out + i] = sum of the partials of (b, i); grid = (nvec, problems)
__global__ void __launch_bounds__(kRedThreads) k_multidot_final(const double2* __restrict__ partials, int nblk,
                                                                double2* __restrict__ out, KBatch kb) {
    pdl_entry();
    const int vi = blockIdx.x, b = blockIdx.y;
    if (kb.active && !kb.active[b]) return;
    const double2* pp = partials + ((long long)b * gridDim.x + vi) * nblk;
    double2 acc = make_double2(0.0, 0.0);
    for (int t = threadIdx.x; t < nblk; t += blockDim.x) acc = cadd(acc, pp[t]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[(long long)b * kb.bs_out + vi] = acc;
}

cudaError_t launch_multidot(const double2* V, long long ld, int nvec, const double2* w, long long N, double2* partials,
                            double2* out, const KBatch& kb, cudaStream_t s) {
    if (nvec <= 0) return cudaSuccess;
    HH_KRET(klaunch(k_multidot_partial, dim3(kRedBlocks, nvec, kb.nb), dim3(kRedThreads), 0, s, 1, V, ld, w, N,
                    partials, kb));
    HH_KRET(klaunch(k_multidot_final, dim3(nvec, kb.nb), dim3(kRedThreads), 0, s, 1, (const double2*)partials,
                    kRedBlocks, out, kb));
    return cudaSuccess;
}

// w_b += sign * sum_i coef[b * bs_out + i] V_{b,i}   (coefficients read from device memory)
__global__ void __launch_bounds__(256) k_multi_axpy(double2* __restrict__ w, const double2* __restrict__ V,
                                                    long long ld, int nvec, const double2* __restrict__ coef,
                                                    double sign, long long N, KBatch kb) {
    pdl_entry();
    const int b = blockIdx.y;
    if (kb.active && !kb.active[b]) return;
    __shared__ double2 c[64];
    for (int t = threadIdx.x; t < nvec && t < 64; t += blockDim.x) {
        double2 v = coef[(long long)b * kb.bs_out + t];
        c[t] = make_double2(sign * v.x, sign * v.y);
    }
    __syncthreads();
    w += (long long)b * kb.bs_w;
    V += (long long)b * kb.bs_v;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += stride) {
        double2 acc = w[p];
        for (int i = 0; i < nvec; ++i) {
            const double2 a = V[(long long)i * ld + p];
            const double2 k = c[i];
            acc.x = fma(k.x, a.x, fma(-k.y, a.y, acc.x));
            acc.y = fma(k.x, a.y, fma(k.y, a.x, acc.y));
        }
        w[p] = acc;
    }
}

static inline unsigned ew_blocks(long long N) {
    long long b = (N + 255) / 256;
    const long long cap = 8LL * num_sms();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

cudaError_t launch_multi_axpy(double2* w, const double2* V, long long ld, int nvec, const double2* coef, double sign,
                              long long N, const KBatch& kb, cudaStream_t s) {
    if (nvec <= 0) return cudaSuccess;
    if (nvec > 64) return cudaErrorInvalidValue;
    return klaunch(k_multi_axpy, dim3(ew_blocks(N), kb.nb), dim3(256), 0, s, 1, w, V, ld, nvec, coef, sign, N, kb);
}

// x_b *= 1 / sqrt(nrm2[b * bs_out].x) (skipped when zero); x_b at offset b * bs_w
__global__ void k_scale_by_rnorm(double2* __restrict__ x, const double2* __restrict__ nrm2, long long N, KBatch kb) {
    pdl_entry();
    const int b = blockIdx.y;
    if (kb.active && !kb.active[b]) return;
    const double n2 = nrm2[(long long)b * kb.bs_out].x;
    if (!(n2 > 0.0)) return;
    const double sc = 1.0 / sqrt(n2);
    x += (long long)b * kb.bs_w;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += stride) {
        double2 v = x[p];
        x[p] = make_double2(v.x * sc, v.y * sc);
    }
}

cudaError_t launch_scale_by_rnorm(double2* x, const double2* nrm2, long long N, const KBatch& kb, cudaStream_t s) {
    return klaunch(k_scale_by_rnorm, dim3(ew_blocks(N), kb.nb), dim3(256), 0, s, 1, x, nrm2, N, kb);
}

}  // namespace hh
