// Grid-transfer and elementwise kernels: full-weighting restriction (3D and the
// building-block API), bi/trilinear prolongation, precision casts, masked copies.
#include "internal.h"

namespace hh {

thread_local long long g_kernel_launches = 0;
thread_local int g_use_pdl = 1;

// ---------------------------------------------------------------- restriction
// Full weighting R = P^T: coarse node I gathers fine nodes 2I + a, a in {-1,0,1}^dim,
// with weight prod (a == 0 ? 1 : 1/2) (the transpose of bi/trilinear interpolation).
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(GridDesc gc, const vec2<T>* __restrict__ rf,
                                                  vec2<T>* __restrict__ rc) {
    pdl_entry();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int L = blockIdx.z;
    if (I > gc.n || J > gc.n) return;
    const int nf = 2 * gc.n, nnf = nf + 1;
    const bool d3 = gc.dim == 3;
    const long long p = d3 ? ((long long)L * gc.nn + J) * gc.nn + I : (long long)J * gc.nn + I;
    bool masked = (I == 0 && gc.dir[0]) || (I == gc.n && gc.dir[1]) || (J == 0 && gc.dir[2]) ||
                  (J == gc.n && gc.dir[3]);
    if (d3) masked = masked || (L == 0 && gc.dir[4]) || (L == gc.n && gc.dir[5]);
    if (masked) {
        st<T>(rc, p, cx<T>(0, 0));
        return;
    }
    Cx<T> acc = cx<T>(0, 0);
    const int cmin = d3 ? -1 : 0, cmax = d3 ? 1 : 0;
    for (int c = cmin; c <= cmax; ++c) {
        const int fl = 2 * L + c;
        if (fl < 0 || fl > nf) continue;
        const T wc = c == 0 ? T(1) : T(0.5);
#pragma unroll
        for (int b = -1; b <= 1; ++b) {
            const int fj = 2 * J + b;
            if (fj < 0 || fj > nf) continue;
            const T wb = b == 0 ? wc : T(0.5) * wc;
#pragma unroll
            for (int a = -1; a <= 1; ++a) {
                const int fi = 2 * I + a;
                if (fi < 0 || fi > nf) continue;
                const T w = a == 0 ? wb : T(0.5) * wb;
                const long long q = ((long long)(d3 ? fl : 0) * nnf + fj) * nnf + fi;
                acc = fma_r(w, ld<T>(rf, q), acc);
            }
        }
    }
    st<T>(rc, p, acc);
}

template <typename T>
cudaError_t launch_restrict(const GridDesc& gc, const vec2<T>* rf, vec2<T>* rc, cudaStream_t s) {
    dim3 blk(32, 8, 1);
    dim3 grd((gc.nn + 31) / 32, (gc.nn + 7) / 8, gc.dim == 3 ? gc.nn : 1);
    HH_KRET(klaunch(k_restrict<T>, dim3(grd), dim3(blk), 0, s, 1, gc, rf, rc));
    return cudaSuccess;
}

// ---------------------------------------------------------------- prolongation
// x_f += P e_c: fine node i takes coarse node i/2 (even i) or the mean of (i-1)/2 and
// (i+1)/2 (odd i) along each axis (bi/trilinear interpolation of the coarse Q1 field).
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(GridDesc gf, const vec2<T>* __restrict__ ec,
                                                 vec2<T>* __restrict__ x) {
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int l = blockIdx.z;
    if (i > gf.n || j > gf.n) return;
    const bool d3 = gf.dim == 3;
    const long long p = d3 ? ((long long)l * gf.nn + j) * gf.nn + i : (long long)j * gf.nn + i;
    bool masked = (i == 0 && gf.dir[0]) || (i == gf.n && gf.dir[1]) || (j == 0 && gf.dir[2]) ||
                  (j == gf.n && gf.dir[3]);
    if (d3) masked = masked || (l == 0 && gf.dir[4]) || (l == gf.n && gf.dir[5]);
    if (masked) {
        st<T>(x, p, cx<T>(0, 0));
        return;
    }
    const int nc = gf.n / 2, nnc = nc + 1;
    const int I0 = i >> 1, J0 = j >> 1, L0 = l >> 1;
    const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nl = (d3 && (l & 1)) ? 2 : 1;
    const T wi = (i & 1) ? T(0.5) : T(1), wj = (j & 1) ? T(0.5) : T(1),
            wl = (d3 && (l & 1)) ? T(0.5) : T(1);
    // coarse Dirichlet nodes carry no basis function: their entries are never read
    auto coarse_dir = [&](int I, int lo, int hi) { return (I == 0 && lo) || (I == nc && hi); };
    Cx<T> e = cx<T>(0, 0);
    for (int c = 0; c < nl; ++c) {
        if (d3 && coarse_dir(L0 + c, gf.dir[4], gf.dir[5])) continue;
        for (int b = 0; b < nj; ++b) {
            if (coarse_dir(J0 + b, gf.dir[2], gf.dir[3])) continue;
            for (int a = 0; a < ni; ++a) {
                if (coarse_dir(I0 + a, gf.dir[0], gf.dir[1])) continue;
                const long long q = ((long long)(d3 ? L0 + c : 0) * nnc + (J0 + b)) * nnc + (I0 + a);
                e = fma_r(wi * wj * wl, ld<T>(ec, q), e);
            }
        }
    }
    st<T>(x, p, ld<T>(x, p) + e);
}

template <typename T>
cudaError_t launch_prolong(const GridDesc& gf, const vec2<T>* ec, vec2<T>* x, cudaStream_t s) {
    dim3 blk(32, 8, 1);
    dim3 grd((gf.nn + 31) / 32, (gf.nn + 7) / 8, gf.dim == 3 ? gf.nn : 1);
    HH_KRET(klaunch(k_prolong<T>, dim3(grd), dim3(blk), 0, s, 1, gf, ec, x));
    return cudaSuccess;
}

// ---------------------------------------------------------------- elementwise
template <typename T>
__global__ void k_add(vec2<T>* __restrict__ x, const vec2<T>* __restrict__ e, long long N) {
    pdl_entry();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x)
        st<T>(x, p, ld<T>(x, p) + ld<T>(e, p));
}

static inline unsigned ew_blocks(long long N) {
    long long b = (N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <typename T>
cudaError_t launch_add(vec2<T>* x, const vec2<T>* e, long long N, cudaStream_t s) {
    HH_KRET(klaunch(k_add<T>, dim3(ew_blocks(N)), dim3(256), 0, s, 1, x, e, N));
    return cudaSuccess;
}

__global__ void k_cast_d2f(const double2* __restrict__ a, float2* __restrict__ b, long long N) {
    pdl_entry();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        double2 v = a[p];
        b[p] = make_float2((float)v.x, (float)v.y);
    }
}
__global__ void k_cast_f2d(const float2* __restrict__ a, double2* __restrict__ b, long long N) {
    pdl_entry();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        float2 v = a[p];
        b[p] = make_double2((double)v.x, (double)v.y);
    }
}

cudaError_t launch_cast_d2f(const double2* a, float2* b, long long N, cudaStream_t s) {
    HH_KRET(klaunch(k_cast_d2f, dim3(ew_blocks(N)), dim3(256), 0, s, 1, a, b, N));
    return cudaSuccess;
}
cudaError_t launch_cast_f2d(const float2* a, double2* b, long long N, cudaStream_t s) {
    HH_KRET(klaunch(k_cast_f2d, dim3(ew_blocks(N)), dim3(256), 0, s, 1, a, b, N));
    return cudaSuccess;
}

__global__ void k_mask_copy(GridDesc g, const double2* __restrict__ src, double2* __restrict__ dst) {
    pdl_entry();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.N;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.nn);
        const int j = (int)((p / g.nn) % g.nn);
        const int l = g.dim == 3 ? (int)(p / ((long long)g.nn * g.nn)) : 0;
        bool masked = (i == 0 && g.dir[0]) || (i == g.n && g.dir[1]) || (j == 0 && g.dir[2]) ||
                      (j == g.n && g.dir[3]);
        if (g.dim == 3) masked = masked || (l == 0 && g.dir[4]) || (l == g.n && g.dir[5]);
        dst[p] = masked ? make_double2(0.0, 0.0) : src[p];
    }
}

cudaError_t launch_mask_copy(const GridDesc& g, const double2* src, double2* dst, cudaStream_t s) {
    HH_KRET(klaunch(k_mask_copy, dim3(ew_blocks(g.N)), dim3(256), 0, s, 1, g, src, dst));
    return cudaSuccess;
}

#define HH_INSTANTIATE(T)                                                                          \
    template cudaError_t launch_restrict<T>(const GridDesc&, const vec2<T>*, vec2<T>*,             \
                                            cudaStream_t);                                         \
    template cudaError_t launch_prolong<T>(const GridDesc&, const vec2<T>*, vec2<T>*,              \
                                           cudaStream_t);                                          \
    template cudaError_t launch_add<T>(vec2<T>*, const vec2<T>*, long long, cudaStream_t);


HH_INSTANTIATE(float)
HH_INSTANTIATE(double)

}  // namespace hh
