// Vector kernels of the GMRES smoother (Sec. 5.3: GMRES with a Jacobi preconditioner on
// every level).  One smoothing step of s iterations on A x = b from x runs, with
// M = omega D^{-1} A applied by the stencil kernels' M_DAXPBY mode:
//   z0 = omega D^{-1} (b - A x), beta = ||z0||, v_0 = z0 / beta;
//   for j < s: w = M v_j; two passes of classical Gram-Schmidt against v_0..v_j (the
//   coefficients of both passes added into column j of H); h_{j+1,j} = ||w||, v_{j+1} = w / h;
//   y = argmin ||beta e1 - H y|| by Givens rotations; x += V y.
// Inner products and norms are summed in FP64: each block writes its share, and the kernel
// that uses a sum adds the shares in block order (every block of that kernel the same way),
// so the result is the same whatever ran before and however the problems are batched.
#include "internal.h"

namespace hh {

namespace {

__device__ __forceinline__ bool gs_skip(const Batch& bt, int b) {
    if (bt.active && !bt.active[b]) return true;
    return bt.hss_it >= 0 && bt.hss_it >= bt.nhss[b];
}

__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// sum of every thread's acc[i] (i < nv) into out[i] (valid in thread 0's block, read after the
// barrier); sh holds kGsThreads / 32 * kGsMaxVec entries
__device__ void block_sums(double2 (&acc)[kGsMaxVec], int nv, double2* sh, double2* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kGsMaxVec; ++i) {
        if (i >= nv) break;
        double2 v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        }
        if (lane == 0) sh[wid * kGsMaxVec + i] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nv) {
        double2 t = make_double2(0.0, 0.0);
        for (int w = 0; w < kGsThreads / 32; ++w) t = dadd(t, sh[w * kGsMaxVec + threadIdx.x]);
        out[threadIdx.x] = t;
    }
}

// grid (nblk, nb)
template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs_dot(const vec2<T>* __restrict__ V, long long ldv, int nv,
                                                       const vec2<T>* __restrict__ w, long long N,
                                                       double2* __restrict__ part, Batch bt) {
    pdl_entry();
    const int b = blockIdx.y;
    if (gs_skip(bt, b)) return;
    __shared__ double2 sh[kGsThreads / 32 * kGsMaxVec];
    const vec2<T>* Vb = V + (long long)b * N;
    const vec2<T>* wb = w + (long long)b * N;
    double2 acc[kGsMaxVec];
#pragma unroll
    for (int i = 0; i < kGsMaxVec; ++i) acc[i] = make_double2(0.0, 0.0);
    const long long stride = (long long)gridDim.x * kGsThreads;
    for (long long p = (long long)blockIdx.x * kGsThreads + threadIdx.x; p < N; p += stride) {
        const Cx<T> x = ld<T>(wb, p);
        const double xr = x.re, xi = x.im;
#pragma unroll
        for (int i = 0; i < kGsMaxVec; ++i) {
            if (i >= nv) break;
            const Cx<T> v = ld<T>(Vb + i * ldv, p);
            const double vr = v.re, vi = v.im;
            // conj(v) * x
            acc[i].x = fma(vr, xr, fma(vi, xi, acc[i].x));
            acc[i].y = fma(vr, xi, fma(-vi, xr, acc[i].y));
        }
    }
    block_sums(acc, nv, sh, part + ((long long)b * gridDim.x + blockIdx.x) * kGsMaxVec);
}

// grid (nblk, nb)
template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs_orth(vec2<T>* __restrict__ w, const vec2<T>* __restrict__ V,
                                                        long long ldv, int nv, long long N,
                                                        const double2* __restrict__ part, double2* H, int col,
                                                        int accumulate, double2* __restrict__ part2, Batch bt) {
    pdl_entry();
    const int b = blockIdx.y;
    if (gs_skip(bt, b)) return;
    __shared__ double2 c[kGsMaxVec];
    __shared__ double2 sh[kGsThreads / 32 * kGsMaxVec];
    const int nblk = gridDim.x;
    if ((int)threadIdx.x < nv) {
        double2 t = make_double2(0.0, 0.0);
        const double2* pb = part + (long long)b * nblk * kGsMaxVec + threadIdx.x;
        for (int k = 0; k < nblk; ++k) t = dadd(t, pb[(long long)k * kGsMaxVec]);
        c[threadIdx.x] = t;
        if (blockIdx.x == 0) {
            double2& h = H[((long long)b * kGsMaxVec + threadIdx.x) * kGsMaxIts + col];
            h = accumulate ? dadd(h, t) : t;
        }
    }
    __syncthreads();
    Cx<T> cc[kGsMaxVec];
#pragma unroll
    for (int i = 0; i < kGsMaxVec; ++i) cc[i] = i < nv ? cx<T>(T(-c[i].x), T(-c[i].y)) : cx<T>(0, 0);
    vec2<T>* wb = w + (long long)b * N;
    const vec2<T>* Vb = V + (long long)b * N;
    double2 acc[kGsMaxVec];
    acc[0] = make_double2(0.0, 0.0);
    const long long stride = (long long)nblk * kGsThreads;
    for (long long p = (long long)blockIdx.x * kGsThreads + threadIdx.x; p < N; p += stride) {
        Cx<T> x = ld<T>(wb, p);
#pragma unroll
        for (int i = 0; i < kGsMaxVec; ++i) {
            if (i >= nv) break;
            x = fma_c(cc[i], ld<T>(Vb + i * ldv, p), x);
        }
        st<T>(wb, p, x);
        const double xr = x.re, xi = x.im;
        acc[0].x = fma(xr, xr, fma(xi, xi, acc[0].x));
    }
    if (part2) block_sums(acc, 1, sh, part2 + ((long long)b * nblk + blockIdx.x) * kGsMaxVec);
}

// grid (nblk, nb)
template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs_scale(vec2<T>* __restrict__ out, const vec2<T>* __restrict__ w,
                                                         long long N, const double2* __restrict__ part2, int nsum,
                                                         double2* H, int row, int col, double* beta, Batch bt) {
    pdl_entry();
    const int b = blockIdx.y;
    if (gs_skip(bt, b)) return;
    __shared__ T inv;
    if (threadIdx.x == 0) {
        double t = 0.0;
        const double2* pb = part2 + (long long)b * nsum * kGsMaxVec;
        for (int k = 0; k < nsum; ++k) t += pb[(long long)k * kGsMaxVec].x;
        const double h = sqrt(t);
        inv = h > 0.0 ? T(1.0 / h) : T(0);
        if (blockIdx.x == 0) {
            if (row < 0) {
                beta[b] = h;
            } else {
                H[((long long)b * kGsMaxVec + row) * kGsMaxIts + col] = make_double2(h, 0.0);
            }
        }
    }
    __syncthreads();
    const T s = inv;
    const vec2<T>* wb = w + (long long)b * N;
    vec2<T>* ob = out + (long long)b * N;
    const long long stride = (long long)gridDim.x * kGsThreads;
    for (long long p = (long long)blockIdx.x * kGsThreads + threadIdx.x; p < N; p += stride) {
        const Cx<T> x = ld<T>(wb, p);
        st<T>(ob, p, cx<T>(x.re * s, x.im * s));
    }
}

// grid (nblk, nb)
template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs_update(vec2<T>* __restrict__ x, const vec2<T>* __restrict__ V,
                                                          long long ldv, int m, long long N, const double2* H,
                                                          const double* beta, int overwrite, Batch bt) {
    pdl_entry();
    const int b = blockIdx.y;
    if (gs_skip(bt, b)) return;
    __shared__ double2 ys[kGsMaxIts];
    if (threadIdx.x == 0) {
        // least squares min ||beta e1 - H y|| by Givens rotations (H is (m+1) x m, Hessenberg)
        double2 R[kGsMaxVec][kGsMaxIts];
        double2 g[kGsMaxVec];
        const double2* Hb = H + (long long)b * kGsMaxVec * kGsMaxIts;
        for (int i = 0; i <= m; ++i) {
            g[i] = make_double2(i == 0 ? beta[b] : 0.0, 0.0);
            for (int j = 0; j < m; ++j) R[i][j] = Hb[i * kGsMaxIts + j];
        }
        for (int j = 0; j < m; ++j) {
            // rotation zeroing R[j+1][j] against R[j][j]: [c s; -conj(s) c] with c real
            const double2 a = R[j][j], e = R[j + 1][j];
            const double na = hypot(a.x, a.y), ne = hypot(e.x, e.y);
            const double den = hypot(na, ne);
            if (den == 0.0) continue;
            double cs;
            double2 sn;
            if (na == 0.0) {
                cs = 0.0;
                sn = make_double2(1.0, 0.0);
            } else {
                cs = na / den;
                // sn = (a / |a|) conj(e) / den
                const double2 u = make_double2(a.x / na, a.y / na);
                sn = make_double2((u.x * e.x + u.y * e.y) / den, (u.y * e.x - u.x * e.y) / den);
            }
            for (int k = j; k < m; ++k) {
                const double2 p = R[j][k], q = R[j + 1][k];
                // p' = cs p + sn q ; q' = -conj(sn) p + cs q
                R[j][k] = make_double2(cs * p.x + (sn.x * q.x - sn.y * q.y), cs * p.y + (sn.x * q.y + sn.y * q.x));
                R[j + 1][k] = make_double2(-(sn.x * p.x + sn.y * p.y) + cs * q.x, -(sn.x * p.y - sn.y * p.x) + cs * q.y);
            }
            const double2 p = g[j], q = g[j + 1];
            g[j] = make_double2(cs * p.x + (sn.x * q.x - sn.y * q.y), cs * p.y + (sn.x * q.y + sn.y * q.x));
            g[j + 1] = make_double2(-(sn.x * p.x + sn.y * p.y) + cs * q.x, -(sn.x * p.y - sn.y * p.x) + cs * q.y);
        }
        // back substitution; a zero pivot (breakdown: the space was already invariant) gives y_j = 0
        for (int j = m - 1; j >= 0; --j) {
            double2 t = g[j];
            for (int k = j + 1; k < m; ++k) {
                const double2 r = R[j][k], yk = ys[k];
                t = make_double2(t.x - (r.x * yk.x - r.y * yk.y), t.y - (r.x * yk.y + r.y * yk.x));
            }
            const double2 d = R[j][j];
            const double dd = d.x * d.x + d.y * d.y;
            ys[j] = dd > 0.0 ? make_double2((t.x * d.x + t.y * d.y) / dd, (t.y * d.x - t.x * d.y) / dd)
                             : make_double2(0.0, 0.0);
        }
    }
    __syncthreads();
    Cx<T> yc[kGsMaxIts];
#pragma unroll
    for (int i = 0; i < kGsMaxIts; ++i) yc[i] = i < m ? cx<T>(T(ys[i].x), T(ys[i].y)) : cx<T>(0, 0);
    vec2<T>* xb = x + (long long)b * N;
    const vec2<T>* Vb = V + (long long)b * N;
    const long long stride = (long long)gridDim.x * kGsThreads;
    for (long long p = (long long)blockIdx.x * kGsThreads + threadIdx.x; p < N; p += stride) {
        Cx<T> acc = overwrite ? cx<T>(0, 0) : ld<T>(xb, p);
#pragma unroll
        for (int i = 0; i < kGsMaxIts; ++i) {
            if (i >= m) break;
            acc = fma_c(yc[i], ld<T>(Vb + i * ldv, p), acc);
        }
        st<T>(xb, p, acc);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_gs_dot(const vec2<T>* V, long long ldv, int nv, const vec2<T>* w, long long N, double2* part,
                          const Batch& bt, cudaStream_t s) {
    if (nv < 1 || nv > kGsMaxVec) return cudaErrorInvalidValue;
    const dim3 grd((unsigned)gs_blocks(N), (unsigned)bt.nb);
    return klaunch(k_gs_dot<T>, grd, dim3(kGsThreads), 0, s, 1, V, ldv, nv, w, N, part, bt);
}

template <typename T>
cudaError_t launch_gs_orth(vec2<T>* w, const vec2<T>* V, long long ldv, int nv, long long N, const double2* part,
                           double2* H, int col, int accumulate, double2* part2, const Batch& bt, cudaStream_t s) {
    if (nv < 1 || nv > kGsMaxVec || col < 0 || col >= kGsMaxIts) return cudaErrorInvalidValue;
    const dim3 grd((unsigned)gs_blocks(N), (unsigned)bt.nb);
    return klaunch(k_gs_orth<T>, grd, dim3(kGsThreads), 0, s, 1, w, V, ldv, nv, N, part, H, col, accumulate, part2,
                   bt);
}

template <typename T>
cudaError_t launch_gs_scale(vec2<T>* out, const vec2<T>* w, long long N, const double2* part2, double2* H, int row,
                            int col, double* beta, const Batch& bt, cudaStream_t s) {
    if (row >= kGsMaxVec || col >= kGsMaxIts) return cudaErrorInvalidValue;
    const int nblk = gs_blocks(N);
    const dim3 grd((unsigned)nblk, (unsigned)bt.nb);
    return klaunch(k_gs_scale<T>, grd, dim3(kGsThreads), 0, s, 1, out, w, N, part2, nblk, H, row, col, beta, bt);
}

template <typename T>
cudaError_t launch_gs_update(vec2<T>* x, const vec2<T>* V, long long ldv, int m, long long N, const double2* H,
                             const double* beta, int overwrite, const Batch& bt, cudaStream_t s) {
    if (m < 1 || m > kGsMaxIts) return cudaErrorInvalidValue;
    const dim3 grd((unsigned)gs_blocks(N), (unsigned)bt.nb);
    return klaunch(k_gs_update<T>, grd, dim3(kGsThreads), 0, s, 1, x, V, ldv, m, N, H, beta, overwrite, bt);
}

#define HH_GS_INST(T)                                                                                                 \
    template cudaError_t launch_gs_dot<T>(const vec2<T>*, long long, int, const vec2<T>*, long long, double2*,        \
                                          const Batch&, cudaStream_t);                                                \
    template cudaError_t launch_gs_orth<T>(vec2<T>*, const vec2<T>*, long long, int, long long, const double2*,       \
                                           double2*, int, int, double2*, const Batch&, cudaStream_t);                 \
    template cudaError_t launch_gs_scale<T>(vec2<T>*, const vec2<T>*, long long, const double2*, double2*, int, int, \
                                            double*, const Batch&, cudaStream_t);                                     \
    template cudaError_t launch_gs_update<T>(vec2<T>*, const vec2<T>*, long long, int, long long, const double2*,     \
                                             const double*, int, const Batch&, cudaStream_t);
HH_GS_INST(float)
HH_GS_INST(double)
#undef HH_GS_INST

}  // namespace hh
