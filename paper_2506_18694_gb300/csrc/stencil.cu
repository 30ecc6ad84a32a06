// Matrix-free Q1 operator kernels: operator apply, scaled Jacobi, residual,
// full-weighting restriction, bi/trilinear prolongation, precision casts.
//
// Every operator is c_K K + c_M M + c_G M_Gamma (primal weak form b_delta, Sec. 2;
// A_L / A_R of Def. 4.1).  On a uniform grid the Q1 stiffness and mass matrices are
// sums of tensor products of the 1D matrices (1/h)[-1 2 -1] and (h/6)[1 4 1], so the
// row of a node is built from three 1D weight triples (one per axis) that encode the
// domain ends and Dirichlet elimination; a Sommerfeld side adds the (dim-1)-
// dimensional mass of that side.  No matrix is stored: one output node reads the
// 3^dim neighbourhood of x once.
#include "internal.h"

namespace hh {

thread_local long long g_kernel_launches = 0;

template <typename T> struct NodeResult {
    Cx<T> ax;  // (op x) at the node
    Cx<T> d;   // diagonal entry of op at the node
};

// (op x) and diag(op) at node (i,j) of a 2D grid; rows rx, ry precomputed.
template <typename T, bool NEED_AX>
__device__ __forceinline__ NodeResult<T> node2(const vec2<T>* __restrict__ x, int nn, int i, int j,
                                               const Row1<T>& rx, const Row1<T>& ry,
                                               const OpCoef<T>& op) {
    NodeResult<T> r;
    const T fxw = rx.face ? ry.mc : T(0);
    const T fyw = ry.face ? rx.mc : T(0);
    const T dr = op.cK * (rx.kc * ry.mc + rx.mc * ry.kc);
    const T dm = rx.mc * ry.mc;
    const T dg = fxw + fyw;
    r.d = cx<T>(dr + op.cM.re * dm + op.cG.re * dg, op.cM.im * dm + op.cG.im * dg);
    if (!NEED_AX) {
        r.ax = cx<T>(0, 0);
        return r;
    }
    const int ia[3] = {rx.lo, i, rx.hi};
    const int jb[3] = {ry.lo, j, ry.hi};
    const T myw[3] = {ry.ml, ry.mc, ry.mr};
    const T kyw[3] = {ry.kl, ry.kc, ry.kr};
    Cx<T> Mx = cx<T>(0, 0), Kx = cx<T>(0, 0), Fx = cx<T>(0, 0), mxc = cx<T>(0, 0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const long long row = (long long)jb[b] * nn;
        const Cx<T> v0 = ld<T>(x, row + ia[0]);
        const Cx<T> v1 = ld<T>(x, row + ia[1]);
        const Cx<T> v2 = ld<T>(x, row + ia[2]);
        Cx<T> mx = fma_r(rx.mr, v2, fma_r(rx.mc, v1, rx.ml * v0));
        Cx<T> kx = fma_r(rx.kr, v2, fma_r(rx.kc, v1, rx.kl * v0));
        Mx = fma_r(myw[b], mx, Mx);
        Kx = fma_r(myw[b], kx, fma_r(kyw[b], mx, Kx));
        Fx = fma_r(myw[b], v1, Fx);
        if (b == 1) mxc = mx;
    }
    Cx<T> F = rx.face ? Fx : cx<T>(0, 0);
    if (ry.face) F = F + mxc;
    Cx<T> ax = op.cK * Kx;
    ax = fma_c(op.cM, Mx, ax);
    ax = fma_c(op.cG, F, ax);
    r.ax = ax;
    return r;
}

// (op x) and diag(op) at node (i,j,l) of a 3D grid.
template <typename T, bool NEED_AX>
__device__ __forceinline__ NodeResult<T> node3(const vec2<T>* __restrict__ x, int nn, int i, int j,
                                               int l, const Row1<T>& rx, const Row1<T>& ry,
                                               const Row1<T>& rz, const OpCoef<T>& op) {
    NodeResult<T> r;
    const T dr = op.cK * (rx.kc * ry.mc * rz.mc + rx.mc * ry.kc * rz.mc + rx.mc * ry.mc * rz.kc);
    const T dm = rx.mc * ry.mc * rz.mc;
    const T dg = (rx.face ? ry.mc * rz.mc : T(0)) + (ry.face ? rx.mc * rz.mc : T(0)) +
                 (rz.face ? rx.mc * ry.mc : T(0));
    r.d = cx<T>(dr + op.cM.re * dm + op.cG.re * dg, op.cM.im * dm + op.cG.im * dg);
    if (!NEED_AX) {
        r.ax = cx<T>(0, 0);
        return r;
    }
    const int ia[3] = {rx.lo, i, rx.hi};
    const int jb[3] = {ry.lo, j, ry.hi};
    const int lc[3] = {rz.lo, l, rz.hi};
    const T myw[3] = {ry.ml, ry.mc, ry.mr};
    const T kyw[3] = {ry.kl, ry.kc, ry.kr};
    const T mzw[3] = {rz.ml, rz.mc, rz.mr};
    const T kzw[3] = {rz.kl, rz.kc, rz.kr};
    Cx<T> Mx = cx<T>(0, 0), Kx = cx<T>(0, 0);
    Cx<T> Fxf = cx<T>(0, 0), Fyf = cx<T>(0, 0), Fzf = cx<T>(0, 0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Cx<T> PM = cx<T>(0, 0), PK = cx<T>(0, 0), Pf = cx<T>(0, 0), mxc = cx<T>(0, 0);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const long long row = ((long long)lc[c] * nn + jb[b]) * nn;
            const Cx<T> v0 = ld<T>(x, row + ia[0]);
            const Cx<T> v1 = ld<T>(x, row + ia[1]);
            const Cx<T> v2 = ld<T>(x, row + ia[2]);
            Cx<T> mx = fma_r(rx.mr, v2, fma_r(rx.mc, v1, rx.ml * v0));
            Cx<T> kx = fma_r(rx.kr, v2, fma_r(rx.kc, v1, rx.kl * v0));
            PM = fma_r(myw[b], mx, PM);
            PK = fma_r(myw[b], kx, fma_r(kyw[b], mx, PK));
            Pf = fma_r(myw[b], v1, Pf);
            if (b == 1) mxc = mx;
        }
        Mx = fma_r(mzw[c], PM, Mx);
        Kx = fma_r(mzw[c], PK, fma_r(kzw[c], PM, Kx));
        Fxf = fma_r(mzw[c], Pf, Fxf);   // x-side face: (M_y x M_z) on the centre column
        Fyf = fma_r(mzw[c], mxc, Fyf);  // y-side face: (M_x x M_z) on the centre row
        if (c == 1) Fzf = PM;           // z-side face: (M_x x M_y) on the centre plane
    }
    Cx<T> F = cx<T>(0, 0);
    if (rx.face) F = F + Fxf;
    if (ry.face) F = F + Fyf;
    if (rz.face) F = F + Fzf;
    Cx<T> ax = op.cK * Kx;
    ax = fma_c(op.cM, Mx, ax);
    ax = fma_c(op.cG, F, ax);
    r.ax = ax;
    return r;
}

template <typename T, int MODE, bool XZERO>
__device__ __forceinline__ Cx<T> epilogue(const NodeResult<T>& nr, const vec2<T>* __restrict__ x,
                                          const vec2<T>* __restrict__ z, long long p, Cx<T> alpha,
                                          Cx<T> beta, T omega) {
    if (MODE == MODE_APPLY) return nr.ax;
    if (MODE == MODE_AXPBY) {
        Cx<T> out = cmul(beta, ld<T>(z, p));
        if (!XZERO) out = fma_c(alpha, nr.ax, out);
        return out;
    }
    // MODE_JACOBI: x + omega D^{-1} (z - op x)
    const Cx<T> dinv = cinv(nr.d);
    Cx<T> res = ld<T>(z, p);
    if (!XZERO) res = res - nr.ax;
    Cx<T> upd = omega * cmul(dinv, res);
    if (!XZERO) upd = upd + ld<T>(x, p);
    return upd;
}

template <typename T, int MODE, bool XZERO>
__global__ void __launch_bounds__(256) k_stencil2(GridDesc g, OpCoef<T> op, T h, T ih,
                                                  const vec2<T>* __restrict__ x,
                                                  const vec2<T>* __restrict__ z,
                                                  vec2<T>* __restrict__ y, Cx<T> alpha,
                                                  Cx<T> beta, T omega) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.n || j > g.n) return;
    const long long p = (long long)j * g.nn + i;
    const Row1<T> rx = row1<T>(i, g.n, g.dir[0], g.dir[1], h, ih);
    const Row1<T> ry = row1<T>(j, g.n, g.dir[2], g.dir[3], h, ih);
    if (rx.masked || ry.masked) {
        st<T>(y, p, cx<T>(0, 0));
        return;
    }
    constexpr bool NEED = !XZERO;
    const NodeResult<T> nr = node2<T, NEED>(x, g.nn, i, j, rx, ry, op);
    st<T>(y, p, epilogue<T, MODE, XZERO>(nr, x, z, p, alpha, beta, omega));
}

template <typename T, int MODE, bool XZERO>
__global__ void __launch_bounds__(256) k_stencil3(GridDesc g, OpCoef<T> op, T h, T ih,
                                                  const vec2<T>* __restrict__ x,
                                                  const vec2<T>* __restrict__ z,
                                                  vec2<T>* __restrict__ y, Cx<T> alpha,
                                                  Cx<T> beta, T omega) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int l = blockIdx.z;
    if (i > g.n || j > g.n) return;
    const long long p = ((long long)l * g.nn + j) * g.nn + i;
    const Row1<T> rx = row1<T>(i, g.n, g.dir[0], g.dir[1], h, ih);
    const Row1<T> ry = row1<T>(j, g.n, g.dir[2], g.dir[3], h, ih);
    const Row1<T> rz = row1<T>(l, g.n, g.dir[4], g.dir[5], h, ih);
    if (rx.masked || ry.masked || rz.masked) {
        st<T>(y, p, cx<T>(0, 0));
        return;
    }
    constexpr bool NEED = !XZERO;
    const NodeResult<T> nr = node3<T, NEED>(x, g.nn, i, j, l, rx, ry, rz, op);
    st<T>(y, p, epilogue<T, MODE, XZERO>(nr, x, z, p, alpha, beta, omega));
}

template <typename T, int MODE, bool XZERO>
static void launch_mode(const GridDesc& g, const OpCoef<T>& op, const vec2<T>* x, const vec2<T>* z,
                        vec2<T>* y, Cx<T> alpha, Cx<T> beta, T omega, cudaStream_t s) {
    const T h = T(g.h), ih = T(1.0 / g.h);
    ++g_kernel_launches;
    dim3 blk(32, 8, 1);
    if (g.dim == 2) {
        dim3 grd((g.nn + 31) / 32, (g.nn + 7) / 8, 1);
        k_stencil2<T, MODE, XZERO><<<grd, blk, 0, s>>>(g, op, h, ih, x, z, y, alpha, beta, omega);
    } else {
        dim3 grd((g.nn + 31) / 32, (g.nn + 7) / 8, g.nn);
        k_stencil3<T, MODE, XZERO><<<grd, blk, 0, s>>>(g, op, h, ih, x, z, y, alpha, beta, omega);
    }
}

template <typename T>
cudaError_t launch_stencil(int mode, const GridDesc& g, const OpCoef<T>& op, const vec2<T>* x,
                           const vec2<T>* z, vec2<T>* y, Cx<T> alpha, Cx<T> beta, T omega,
                           cudaStream_t s) {
    const bool xz = (x == nullptr);
    if (mode == MODE_APPLY) {
        if (xz) return cudaErrorInvalidValue;
        launch_mode<T, MODE_APPLY, false>(g, op, x, z, y, alpha, beta, omega, s);
    } else if (mode == MODE_AXPBY) {
        if (xz) launch_mode<T, MODE_AXPBY, true>(g, op, x, z, y, alpha, beta, omega, s);
        else launch_mode<T, MODE_AXPBY, false>(g, op, x, z, y, alpha, beta, omega, s);
    } else {
        if (xz) launch_mode<T, MODE_JACOBI, true>(g, op, x, z, y, alpha, beta, omega, s);
        else launch_mode<T, MODE_JACOBI, false>(g, op, x, z, y, alpha, beta, omega, s);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- restriction
// Full weighting R = P^T: coarse node I gathers fine nodes 2I + a, a in {-1,0,1}^dim,
// with weight prod (a == 0 ? 1 : 1/2) (the transpose of bi/trilinear interpolation).
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(GridDesc gc, const vec2<T>* __restrict__ rf,
                                                  vec2<T>* __restrict__ rc) {
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
    ++g_kernel_launches;
    k_restrict<T><<<grd, blk, 0, s>>>(gc, rf, rc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_restrict(const GridDesc& gf, const GridDesc& gc, const OpCoef<T>& op,
                                     const vec2<T>* b, const vec2<T>* x, vec2<T>* rc,
                                     vec2<T>* scratch, cudaStream_t s) {
    cudaError_t e = launch_stencil<T>(MODE_AXPBY, gf, op, x, b, scratch, cx<T>(-1, 0), cx<T>(1, 0),
                                      T(0), s);
    if (e != cudaSuccess) return e;
    return launch_restrict<T>(gc, scratch, rc, s);
}

// ---------------------------------------------------------------- prolongation
// x_f += P e_c: fine node i takes coarse node i/2 (even i) or the mean of (i-1)/2 and
// (i+1)/2 (odd i) along each axis (bi/trilinear interpolation of the coarse Q1 field).
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(GridDesc gf, const vec2<T>* __restrict__ ec,
                                                 vec2<T>* __restrict__ x) {
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
    ++g_kernel_launches;
    k_prolong<T><<<grd, blk, 0, s>>>(gf, ec, x);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- elementwise
template <typename T>
__global__ void k_add(vec2<T>* __restrict__ x, const vec2<T>* __restrict__ e, long long N) {
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
    ++g_kernel_launches;
    k_add<T><<<ew_blocks(N), 256, 0, s>>>(x, e, N);
    return cudaGetLastError();
}

__global__ void k_cast_d2f(const double2* __restrict__ a, float2* __restrict__ b, long long N) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        double2 v = a[p];
        b[p] = make_float2((float)v.x, (float)v.y);
    }
}
__global__ void k_cast_f2d(const float2* __restrict__ a, double2* __restrict__ b, long long N) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        float2 v = a[p];
        b[p] = make_double2((double)v.x, (double)v.y);
    }
}

cudaError_t launch_cast_d2f(const double2* a, float2* b, long long N, cudaStream_t s) {
    ++g_kernel_launches;
    k_cast_d2f<<<ew_blocks(N), 256, 0, s>>>(a, b, N);
    return cudaGetLastError();
}
cudaError_t launch_cast_f2d(const float2* a, double2* b, long long N, cudaStream_t s) {
    ++g_kernel_launches;
    k_cast_f2d<<<ew_blocks(N), 256, 0, s>>>(a, b, N);
    return cudaGetLastError();
}

__global__ void k_mask_copy(GridDesc g, const double2* __restrict__ src, double2* __restrict__ dst) {
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
    ++g_kernel_launches;
    k_mask_copy<<<ew_blocks(g.N), 256, 0, s>>>(g, src, dst);
    return cudaGetLastError();
}

#define HH_INSTANTIATE(T)                                                                          \
    template cudaError_t launch_stencil<T>(int, const GridDesc&, const OpCoef<T>&, const vec2<T>*, \
                                           const vec2<T>*, vec2<T>*, Cx<T>, Cx<T>, T, cudaStream_t); \
    template cudaError_t launch_restrict<T>(const GridDesc&, const vec2<T>*, vec2<T>*,             \
                                            cudaStream_t);                                         \
    template cudaError_t launch_residual_restrict<T>(const GridDesc&, const GridDesc&,             \
                                                     const OpCoef<T>&, const vec2<T>*,             \
                                                     const vec2<T>*, vec2<T>*, vec2<T>*,           \
                                                     cudaStream_t);                                \
    template cudaError_t launch_prolong<T>(const GridDesc&, const vec2<T>*, vec2<T>*,              \
                                           cudaStream_t);                                          \
    template cudaError_t launch_add<T>(vec2<T>*, const vec2<T>*, long long, cudaStream_t);

HH_INSTANTIATE(float)
HH_INSTANTIATE(double)

}  // namespace hh
