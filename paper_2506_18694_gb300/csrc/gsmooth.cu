// Vector kernels of the GMRES smoother (Sec. 5.3: GMRES with a Jacobi preconditioner on
// every level).  One smoothing step of s iterations on A x = b from x runs, with
// M = omega D^{-1} A applied by the stencil kernels' M_DAXPBY mode:
//   z0 = omega D^{-1} (b - A x), beta = ||z0||, v_0 = z0 / beta;
//   for j < s: w = M v_j; two passes of classical Gram-Schmidt against v_0..v_j (the
//   coefficients of both passes added into column j of H); h_{j+1,j} = ||w||, v_{j+1} = w / h,
//   and column j reduced by Givens rotations (as in GMRES, one new rotation per step);
//   y = R^{-1} g minimises ||beta e1 - H y||; x += V y.
// Inner products and norms are summed in the level precision within a block (FP64 arithmetic
// is slow on this part and the complex64 smoother does not need it) and the block shares are
// combined in FP64: each block writes its share, and the kernel that uses a sum adds the
// shares in a fixed order (every block of that kernel the same way), so the result is the
// same whatever ran before and however the problems are batched.
#include "internal.h"
#include "march2_common.cuh"

namespace hh {

namespace {

__device__ __forceinline__ bool gs_skip(const Batch& bt, int b) {
    if (bt.active && !bt.active[b]) return true;
    return bt.hss_it >= 0 && bt.hss_it >= bt.nhss[b];
}

__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// fused multiply-add in the level precision (FP64 arithmetic, conversions included, runs on
// this part's narrow FP64 pipe: kept out of the per-element loops of the complex64 smoother)
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// sum of every thread's acc[i] (i < nv) over the block into out[i] (as FP64), by warp
// butterflies and then the warps in order; sh holds kGsThreads / 32 * kGsMaxVec entries
template <typename T>
__device__ void block_sums(Cx<T> (&acc)[kGsMaxVec], int nv, Cx<T>* sh, double2* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kGsMaxVec; ++i) {
        if (i >= nv) break;
        Cx<T> v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
            v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
        }
        if (lane == 0) sh[wid * kGsMaxVec + i] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nv) {
        Cx<T> t = cx<T>(0, 0);
        for (int w = 0; w < kGsThreads / 32; ++w) t = t + sh[w * kGsMaxVec + threadIdx.x];
        out[threadIdx.x] = make_double2(t.re, t.im);
    }
}

// sum of n block shares p[0], p[stride], ... by one warp: lane t adds shares t, t + 32, ...
// in order, then the lanes are combined by a fixed butterfly (the same order on every call)
__device__ __forceinline__ double2 warp_sum_shares(const double2* p, int n, int stride) {
    const int lane = threadIdx.x & 31;
    double2 t = make_double2(0.0, 0.0);
    for (int k = lane; k < n; k += 32) t = dadd(t, p[(long long)k * stride]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
        t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
    }
    return t;
}

// grid (nblk, nb)
template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs_dot(const vec2<T>* __restrict__ V, long long ldv, int nv,
                                                       const vec2<T>* __restrict__ w, long long N,
                                                       double2* __restrict__ part, Batch bt) {
    pdl_entry();
    const int b = blockIdx.y;
    if (gs_skip(bt, b)) return;
    __shared__ Cx<T> sh[kGsThreads / 32 * kGsMaxVec];
    const vec2<T>* Vb = V + (long long)b * N;
    const vec2<T>* wb = w + (long long)b * N;
    Cx<T> acc[kGsMaxVec];
#pragma unroll
    for (int i = 0; i < kGsMaxVec; ++i) acc[i] = cx<T>(0, 0);
    const long long stride = (long long)gridDim.x * kGsThreads;
    for (long long p = (long long)blockIdx.x * kGsThreads + threadIdx.x; p < N; p += stride) {
        const Cx<T> x = ld<T>(wb, p);
#pragma unroll
        for (int i = 0; i < kGsMaxVec; ++i) {
            if (i >= nv) break;
            const Cx<T> v = ld<T>(Vb + i * ldv, p);
            // conj(v) * x
            acc[i].re = fmaT(v.re, x.re, fmaT(v.im, x.im, acc[i].re));
            acc[i].im = fmaT(v.re, x.im, fmaT(-v.im, x.re, acc[i].im));
        }
    }
    block_sums(acc, nv, sh, part + ((long long)b * gridDim.x + blockIdx.x) * kGsMaxVec);
}

// grid (nblk, nb)
template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs_orth(vec2<T>* __restrict__ w, const vec2<T>* __restrict__ V,
                                                        long long ldv, int nv, long long N,
                                                        const double2* __restrict__ part, double2* ls, int col,
                                                        int accumulate, double2* __restrict__ part2, Batch bt) {
    pdl_entry();
    const int b = blockIdx.y;
    if (gs_skip(bt, b)) return;
    __shared__ Cx<T> cneg[kGsMaxVec];  // -c_i in the level precision
    __shared__ Cx<T> sh[kGsThreads / 32 * kGsMaxVec];
    const int nblk = gridDim.x;
    // coefficient i summed by warp i % 8
    for (int i = threadIdx.x >> 5; i < nv; i += kGsThreads / 32) {
        const double2 t = warp_sum_shares(part + (long long)b * nblk * kGsMaxVec + i, nblk, kGsMaxVec);
        if ((threadIdx.x & 31) == 0) {
            cneg[i] = cx<T>(T(-t.x), T(-t.y));
            if (blockIdx.x == 0) {
                double2& h = ls[(long long)b * kGsState + i * kGsMaxIts + col];
                h = accumulate ? dadd(h, t) : t;
            }
        }
    }
    __syncthreads();
    Cx<T> cc[kGsMaxVec];
#pragma unroll
    for (int i = 0; i < kGsMaxVec; ++i) cc[i] = i < nv ? cneg[i] : cx<T>(0, 0);
    vec2<T>* wb = w + (long long)b * N;
    const vec2<T>* Vb = V + (long long)b * N;
    Cx<T> acc[kGsMaxVec];
    acc[0] = cx<T>(0, 0);
    const long long stride = (long long)nblk * kGsThreads;
    for (long long p = (long long)blockIdx.x * kGsThreads + threadIdx.x; p < N; p += stride) {
        Cx<T> x = ld<T>(wb, p);
#pragma unroll
        for (int i = 0; i < kGsMaxVec; ++i) {
            if (i >= nv) break;
            x = fma_c(cc[i], ld<T>(Vb + i * ldv, p), x);
        }
        st<T>(wb, p, x);
        acc[0].re = fmaT(x.re, x.re, fmaT(x.im, x.im, acc[0].re));
    }
    if (part2) block_sums(acc, 1, sh, part2 + ((long long)b * nblk + blockIdx.x) * kGsMaxVec);
}

// complex helpers in the level precision for the small least-squares problem
template <typename T>
__device__ __forceinline__ Cx<T> cget(const double2& d) {
    return cx<T>(T(d.x), T(d.y));
}
template <typename T>
__device__ __forceinline__ double2 cput(Cx<T> v) {
    return make_double2(v.re, v.im);
}
// (p, q) <- (c p + s q, -conj(s) p + c q), c real
template <typename T>
__device__ __forceinline__ void rotate(T c, Cx<T> s, Cx<T>& p, Cx<T>& q) {
    const Cx<T> p0 = p, q0 = q;
    p = cx<T>(c * p0.re + (s.re * q0.re - s.im * q0.im), c * p0.im + (s.re * q0.im + s.im * q0.re));
    q = cx<T>(-(s.re * p0.re + s.im * p0.im) + c * q0.re, -(s.re * p0.im - s.im * p0.re) + c * q0.im);
}

// grid (nblk, nb)
template <typename T>
__global__ void __launch_bounds__(kGsThreads) k_gs_scale(vec2<T>* __restrict__ out, const vec2<T>* __restrict__ w,
                                                         long long N, const double2* __restrict__ part2, int nsum,
                                                         double2* ls, int col, Batch bt) {
    pdl_entry();
    const int b = blockIdx.y;
    if (gs_skip(bt, b)) return;
    __shared__ T inv;
    if (threadIdx.x < 32) {
        const T h = sqrt(T(warp_sum_shares(part2 + (long long)b * nsum * kGsMaxVec, nsum, kGsMaxVec).x));
        if (threadIdx.x == 0) {
            inv = h > T(0) ? T(1) / h : T(0);
            if (blockIdx.x == 0) {
                double2* S = ls + (long long)b * kGsState;
                if (col < 0) {
                    S[kGsRhs] = make_double2(h, 0.0);
                    for (int i = 1; i < kGsMaxVec; ++i) S[kGsRhs + i] = make_double2(0.0, 0.0);
                } else {
                    // column col: previous rotations, then the one that zeroes h = H[col + 1][col]
                    for (int i = 0; i < col; ++i) {
                        Cx<T> p = cget<T>(S[i * kGsMaxIts + col]), q = cget<T>(S[(i + 1) * kGsMaxIts + col]);
                        rotate<T>(T(S[kGsCos + i].x), cget<T>(S[kGsSin + i]), p, q);
                        S[i * kGsMaxIts + col] = cput(p);
                        S[(i + 1) * kGsMaxIts + col] = cput(q);
                    }
                    const Cx<T> a = cget<T>(S[col * kGsMaxIts + col]);
                    const T na = sqrt(a.re * a.re + a.im * a.im);
                    const T den = sqrt(na * na + h * h);
                    T cs = T(1);
                    Cx<T> sn = cx<T>(0, 0);
                    if (den > T(0)) {
                        if (na == T(0)) {
                            cs = T(0);
                            sn = cx<T>(1, 0);
                        } else {
                            // s = (a / |a|) conj(h) / den, h real
                            cs = na / den;
                            sn = cx<T>(a.re / na * h / den, a.im / na * h / den);
                        }
                    }
                    Cx<T> p = a, q = cx<T>(h, 0);
                    rotate<T>(cs, sn, p, q);
                    S[col * kGsMaxIts + col] = cput(p);
                    S[(col + 1) * kGsMaxIts + col] = make_double2(0.0, 0.0);
                    S[kGsCos + col] = make_double2(cs, 0.0);
                    S[kGsSin + col] = cput(sn);
                    Cx<T> g0 = cget<T>(S[kGsRhs + col]), g1 = cget<T>(S[kGsRhs + col + 1]);
                    rotate<T>(cs, sn, g0, g1);
                    S[kGsRhs + col] = cput(g0);
                    S[kGsRhs + col + 1] = cput(g1);
                }
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
                                                          long long ldv, int m, long long N, const double2* ls,
                                                          int overwrite, Batch bt) {
    pdl_entry();
    const int b = blockIdx.y;
    if (gs_skip(bt, b)) return;
    __shared__ Cx<T> ys[kGsMaxIts];
    if (threadIdx.x == 0) {
        // back substitution R y = g; a zero pivot (breakdown: the space was already
        // invariant) gives y_j = 0
        const double2* S = ls + (long long)b * kGsState;
        for (int j = m - 1; j >= 0; --j) {
            Cx<T> t = cget<T>(S[kGsRhs + j]);
            for (int k = j + 1; k < m; ++k) {
                const Cx<T> r = cget<T>(S[j * kGsMaxIts + k]), yk = ys[k];
                t = cx<T>(t.re - (r.re * yk.re - r.im * yk.im), t.im - (r.re * yk.im + r.im * yk.re));
            }
            const Cx<T> d = cget<T>(S[j * kGsMaxIts + j]);
            const T dd = d.re * d.re + d.im * d.im;
            ys[j] = dd > T(0) ? cx<T>((t.re * d.re + t.im * d.im) / dd, (t.im * d.re - t.re * d.im) / dd)
                              : cx<T>(0, 0);
        }
    }
    __syncthreads();
    Cx<T> yc[kGsMaxIts];
#pragma unroll
    for (int i = 0; i < kGsMaxIts; ++i) yc[i] = i < m ? ys[i] : cx<T>(0, 0);
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

// ---- the whole smoothing step in one CTA per problem (small 2D levels) ----
constexpr int kGsCtaThreads = 1024;

// sum over the block of every thread's acc[i] (i < nv) into out[i] (shared), fixed order
template <typename T>
__device__ void cta_sums(Cx<T> (&acc)[kGsMaxVec], int nv, Cx<T> (*red)[kGsMaxVec], Cx<T>* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kGsMaxVec; ++i) {
        if (i >= nv) break;
        Cx<T> v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
            v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
        }
        if (lane == 0) red[wid][i] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nv) {
        Cx<T> t = cx<T>(0, 0);
        for (int w = 0; w < kGsCtaThreads / 32; ++w) t = t + red[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// grid (nb): problem blockIdx.x.  x (in/out), b, and the basis V_0..V_its (+ work vector
// V_{its+1}) at Vb + i * ldv, all with problem offsets b * N.
template <typename T>
__global__ void __launch_bounds__(kGsCtaThreads) k_gs_cta(const __grid_constant__ MArgs<T> a,
                                                          const vec2<T>* __restrict__ bvec, vec2<T>* x, int xzero,
                                                          int its, vec2<T>* Vb, long long ldv) {
    pdl_entry();
    const int pb = blockIdx.x;
    if (a.pc && problem_skipped(a, pb)) return;  // the whole CTA
    const PCoef<T>& c = a.pc ? a.pc[pb] : a.c0;
    const int n = a.g.n, nn = a.g.nn;
    const long long N = a.g.N;
    const long long off = (long long)pb * N;
    const vec2<T>* bb = bvec + off;
    vec2<T>* xb = x + off;
    auto V = [&](int i) { return Vb + (long long)i * ldv + off; };
    vec2<T>* W = V(its + 1);
    __shared__ Cx<T> red[kGsCtaThreads / 32][kGsMaxVec];
    __shared__ Cx<T> hc[kGsMaxVec];
    __shared__ Cx<T> R[kGsMaxVec][kGsMaxIts];
    __shared__ Cx<T> g[kGsMaxVec], sn[kGsMaxIts], ys[kGsMaxIts];
    __shared__ T csv[kGsMaxIts];
    __shared__ T scal;
    auto dirn = [&](int i, int j) {
        return (i == 0 && a.g.dir[0]) || (i == n && a.g.dir[1]) || (j == 0 && a.g.dir[2]) || (j == n && a.g.dir[3]);
    };
    auto val = [&](const vec2<T>* v, int i, int j) {
        return (i < 0 || i > n || j < 0 || j > n || dirn(i, j)) ? cx<T>(0, 0) : ld<T>(v, (long long)j * nn + i);
    };
    // omega D^{-1} (alpha (A v) + beta z) at node (i, j); v == nullptr: v = 0
    auto dapply = [&](const vec2<T>* v, const vec2<T>* z, Cx<T> alpha, Cx<T> beta, int i, int j) {
        if (dirn(i, j)) return cx<T>(0, 0);
        Cx<T> ax = cx<T>(0, 0), dinv_w;
        const bool fast = i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1;
        const int tx = i == 0 ? 0 : (i == n ? 2 : 1), ty = j == 0 ? 0 : (j == n ? 2 : 1);
        if (v) {
            stencil_node2<T>(c, val(v, i, j - 1), val(v, i, j), val(v, i, j + 1), val(v, i - 1, j - 1),
                             val(v, i - 1, j), val(v, i - 1, j + 1), val(v, i + 1, j - 1), val(v, i + 1, j),
                             val(v, i + 1, j + 1), fast, tx, ty, ax, dinv_w);
        } else {
            dinv_w = fast ? c.wdinv : c.bdinv[bclass2(tx, ty)];
        }
        const Cx<T> zv = z ? ld<T>(z, (long long)j * nn + i) : cx<T>(0, 0);
        return cmul(dinv_w, fma_c(alpha, ax, cmul(beta, zv)));
    };
    const Cx<T> one = cx<T>(1, 0), mone = cx<T>(-1, 0), zero = cx<T>(0, 0);
    Cx<T> acc[kGsMaxVec];
    // z0 = omega D^{-1} (b - A x), beta = ||z0||, v_0 = z0 / beta
    acc[0] = zero;
    for (long long p = threadIdx.x; p < N; p += kGsCtaThreads) {
        const int i = (int)(p % nn), j = (int)(p / nn);
        const Cx<T> w = dapply(xzero ? nullptr : xb, bb, mone, one, i, j);
        st<T>(W, p, w);
        acc[0].re += w.re * w.re + w.im * w.im;
    }
    cta_sums<T>(acc, 1, red, hc);
    if (threadIdx.x == 0) {
        const T beta = sqrt(hc[0].re);
        scal = beta > T(0) ? T(1) / beta : T(0);
        g[0] = cx<T>(beta, 0);
        for (int i = 1; i < kGsMaxVec; ++i) g[i] = zero;
    }
    __syncthreads();
    for (long long p = threadIdx.x; p < N; p += kGsCtaThreads) {
        const Cx<T> w = ld<T>(W, p);
        st<T>(V(0), p, cx<T>(w.re * scal, w.im * scal));
    }
    __syncthreads();
    for (int j = 0; j < its; ++j) {
        const vec2<T>* vj = V(j);
        for (long long p = threadIdx.x; p < N; p += kGsCtaThreads) {
            const int i = (int)(p % nn), jj = (int)(p / nn);
            st<T>(W, p, dapply(vj, nullptr, one, zero, i, jj));
        }
        __syncthreads();
        // classical Gram-Schmidt, twice
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = 0; i <= j; ++i) acc[i] = zero;
            for (long long p = threadIdx.x; p < N; p += kGsCtaThreads) {
                const Cx<T> w = ld<T>(W, p);
                for (int i = 0; i <= j; ++i) {
                    const Cx<T> v = ld<T>(V(i), p);
                    acc[i].re += v.re * w.re + v.im * w.im;
                    acc[i].im += v.re * w.im - v.im * w.re;
                }
            }
            cta_sums<T>(acc, j + 1, red, hc);
            if ((int)threadIdx.x <= j) R[threadIdx.x][j] = pass ? R[threadIdx.x][j] + hc[threadIdx.x] : hc[threadIdx.x];
            acc[0] = zero;
            for (long long p = threadIdx.x; p < N; p += kGsCtaThreads) {
                Cx<T> w = ld<T>(W, p);
                for (int i = 0; i <= j; ++i) w = fma_c(cx<T>(-hc[i].re, -hc[i].im), ld<T>(V(i), p), w);
                st<T>(W, p, w);
                acc[0].re += w.re * w.re + w.im * w.im;
            }
            __syncthreads();
        }
        cta_sums<T>(acc, 1, red, hc);  // ||w||^2 after the second pass
        if (threadIdx.x == 0) {
            const T h = sqrt(hc[0].re);
            scal = h > T(0) ? T(1) / h : T(0);
            // previous rotations on column j, then the one that zeroes h
            for (int i = 0; i < j; ++i) {
                const Cx<T> p0 = R[i][j], q0 = R[i + 1][j];
                const T cc = csv[i];
                const Cx<T> s0 = sn[i];
                R[i][j] = cx<T>(cc * p0.re + (s0.re * q0.re - s0.im * q0.im), cc * p0.im + (s0.re * q0.im + s0.im * q0.re));
                R[i + 1][j] = cx<T>(-(s0.re * p0.re + s0.im * p0.im) + cc * q0.re, -(s0.re * p0.im - s0.im * p0.re) + cc * q0.im);
            }
            const Cx<T> av = R[j][j];
            const T na = sqrt(av.re * av.re + av.im * av.im), den = sqrt(na * na + h * h);
            T cc = T(1);
            Cx<T> s0 = zero;
            if (den > T(0)) {
                if (na == T(0)) {
                    cc = T(0);
                    s0 = one;
                } else {
                    cc = na / den;
                    s0 = cx<T>(av.re / na * h / den, av.im / na * h / den);
                }
            }
            csv[j] = cc;
            sn[j] = s0;
            R[j][j] = cx<T>(cc * av.re + s0.re * h, cc * av.im + s0.im * h);
            const Cx<T> g0 = g[j];
            g[j] = cx<T>(cc * g0.re, cc * g0.im);
            g[j + 1] = cx<T>(-(s0.re * g0.re + s0.im * g0.im), -(s0.re * g0.im - s0.im * g0.re));
        }
        __syncthreads();
        vec2<T>* vn = V(j + 1);
        for (long long p = threadIdx.x; p < N; p += kGsCtaThreads) {
            const Cx<T> w = ld<T>(W, p);
            st<T>(vn, p, cx<T>(w.re * scal, w.im * scal));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int j = its - 1; j >= 0; --j) {
            Cx<T> t = g[j];
            for (int k = j + 1; k < its; ++k) t = t - cmul(R[j][k], ys[k]);
            const Cx<T> d = R[j][j];
            const T dd = d.re * d.re + d.im * d.im;
            ys[j] = dd > T(0) ? cx<T>((t.re * d.re + t.im * d.im) / dd, (t.im * d.re - t.re * d.im) / dd) : zero;
        }
    }
    __syncthreads();
    for (long long p = threadIdx.x; p < N; p += kGsCtaThreads) {
        Cx<T> u = xzero ? zero : ld<T>(xb, p);
        for (int i = 0; i < its; ++i) u = fma_c(ys[i], ld<T>(V(i), p), u);
        st<T>(xb, p, u);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_gs_cta(const MArgs<T>& a, const vec2<T>* b, vec2<T>* x, int xzero, int its, vec2<T>* V,
                          long long ldv, cudaStream_t s) {
    if (a.g.dim != 2 || its < 1 || its > kGsMaxIts || a.g.N > kGsCtaNodes) return cudaErrorInvalidValue;
    if (!a.pc && a.nb != 1) return cudaErrorInvalidValue;
    return klaunch(k_gs_cta<T>, dim3((unsigned)a.nb), dim3(kGsCtaThreads), 0, s, 1, a, b, x, xzero, its, V, ldv);
}

template <typename T>
cudaError_t launch_gs_dot(const vec2<T>* V, long long ldv, int nv, const vec2<T>* w, long long N, double2* part,
                          const Batch& bt, cudaStream_t s) {
    if (nv < 1 || nv > kGsMaxVec) return cudaErrorInvalidValue;
    const dim3 grd((unsigned)gs_blocks(N), (unsigned)bt.nb);
    return klaunch(k_gs_dot<T>, grd, dim3(kGsThreads), 0, s, 1, V, ldv, nv, w, N, part, bt);
}

template <typename T>
cudaError_t launch_gs_orth(vec2<T>* w, const vec2<T>* V, long long ld, int nv, long long N, const double2* part,
                           double2* ls, int col, int accumulate, double2* part2, const Batch& bt, cudaStream_t s) {
    if (nv < 1 || nv > kGsMaxVec || col < 0 || col >= kGsMaxIts) return cudaErrorInvalidValue;
    const dim3 grd((unsigned)gs_blocks(N), (unsigned)bt.nb);
    return klaunch(k_gs_orth<T>, grd, dim3(kGsThreads), 0, s, 1, w, V, ld, nv, N, part, ls, col, accumulate, part2,
                   bt);
}

template <typename T>
cudaError_t launch_gs_scale(vec2<T>* out, const vec2<T>* w, long long N, const double2* part2, double2* ls, int col,
                            const Batch& bt, cudaStream_t s) {
    if (col >= kGsMaxIts) return cudaErrorInvalidValue;
    const int nblk = gs_blocks(N);
    const dim3 grd((unsigned)nblk, (unsigned)bt.nb);
    return klaunch(k_gs_scale<T>, grd, dim3(kGsThreads), 0, s, 1, out, w, N, part2, nblk, ls, col, bt);
}

template <typename T>
cudaError_t launch_gs_update(vec2<T>* x, const vec2<T>* V, long long ld, int m, long long N, const double2* ls,
                             int overwrite, const Batch& bt, cudaStream_t s) {
    if (m < 1 || m > kGsMaxIts) return cudaErrorInvalidValue;
    const dim3 grd((unsigned)gs_blocks(N), (unsigned)bt.nb);
    return klaunch(k_gs_update<T>, grd, dim3(kGsThreads), 0, s, 1, x, V, ld, m, N, ls, overwrite, bt);
}

#define HH_GS_INST(T)                                                                                                 \
    template cudaError_t launch_gs_dot<T>(const vec2<T>*, long long, int, const vec2<T>*, long long, double2*,        \
                                          const Batch&, cudaStream_t);                                                \
    template cudaError_t launch_gs_orth<T>(vec2<T>*, const vec2<T>*, long long, int, long long, const double2*,       \
                                           double2*, int, int, double2*, const Batch&, cudaStream_t);                 \
    template cudaError_t launch_gs_scale<T>(vec2<T>*, const vec2<T>*, long long, const double2*, double2*, int,       \
                                            const Batch&, cudaStream_t);                                              \
    template cudaError_t launch_gs_update<T>(vec2<T>*, const vec2<T>*, long long, int, long long, const double2*,     \
                                             int, const Batch&, cudaStream_t);
template cudaError_t launch_gs_cta<float>(const MArgs<float>&, const vec2<float>*, vec2<float>*, int, int,
                                          vec2<float>*, long long, cudaStream_t);
template cudaError_t launch_gs_cta<double>(const MArgs<double>&, const vec2<double>*, vec2<double>*, int, int,
                                           vec2<double>*, long long, cudaStream_t);
HH_GS_INST(float)
HH_GS_INST(double)
#undef HH_GS_INST

}  // namespace hh
