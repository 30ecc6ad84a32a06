// 3D fused V-cycle kernels.  A CTA of 8 warps owns a tile of 30 x-nodes, 8 consecutive
// y-rows (the first and last are halo rows) and R + 2 consecutive z-planes (the first and
// last are halo planes); it writes the 30 x 6 x R interior outputs.  Warp w loads its row
// of every plane with one coalesced access per plane (all loads in flight before any
// arithmetic), forms the x-neighbour sum by warp shuffles, and publishes the value and the
// x-sum of each plane in shared memory; after one barrier the six output warps read rows
// j-1 and j+1 from shared memory and keep their own row in registers.  Interior nodes use
// the four neighbour-class weights of the 27-point Q1 operator (centre, face, edge,
// corner); nodes near the boundary rebuild their row from the 1D weight triples, as in the
// 2D kernels.
#include "internal.h"

namespace hh {

namespace {

__device__ __forceinline__ int clampi3(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename T>
__device__ __forceinline__ Cx<T> shfl_up3(Cx<T> v) {
    return Cx<T>{__shfl_up_sync(0xffffffffu, v.re, 1), __shfl_up_sync(0xffffffffu, v.im, 1)};
}
template <typename T>
__device__ __forceinline__ Cx<T> shfl_dn3(Cx<T> v) {
    return Cx<T>{__shfl_down_sync(0xffffffffu, v.re, 1), __shfl_down_sync(0xffffffffu, v.im, 1)};
}

template <typename T>
__device__ __forceinline__ Cx<T> diag3(const Row1<T>& rx, const Row1<T>& ry, const Row1<T>& rz, const OpCoef<T>& op) {
    const T dr = op.cK * (rx.kc * ry.mc * rz.mc + rx.mc * ry.kc * rz.mc + rx.mc * ry.mc * rz.kc);
    const T dm = rx.mc * ry.mc * rz.mc;
    const T dg = (rx.face ? ry.mc * rz.mc : T(0)) + (ry.face ? rx.mc * rz.mc : T(0)) + (rz.face ? rx.mc * ry.mc : T(0));
    return cx<T>(dr + op.cM.re * dm + op.cG.re * dg, op.cM.im * dm + op.cG.im * dg);
}

__device__ __forceinline__ bool coarse_dir(int I, int nc, int lo, int hi) { return (I == 0 && lo) || (I == nc && hi); }

// Value of the stencil field at node (i, j, l) (all clamped into the grid).
template <typename T, int MODE>
__device__ __forceinline__ Cx<T> field3(const MArgs<T>& a, const PCoef<T>& c, const VPtrs<T>& v, int i, int j, int l,
                                        const Row1<T>& rx, const Row1<T>& ry, T h, T ih) {
    const int n = a.g.n, nn = a.g.nn;
    const long long p = ((long long)l * nn + j) * nn + i;
    if (MODE == M_JACOBI2_ZERO) {
        // first sweep from x = 0: x1 = omega D^{-1} b (zero at Dirichlet nodes)
        const Cx<T> b = ld<T>(v.z, p);
        if (i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1 && l >= 1 && l <= n - 1) return cmul(c.wdinv, b);
        const Row1<T> rz = row1<T>(l, n, a.g.dir[4], a.g.dir[5], h, ih);
        if (rx.masked || ry.masked || rz.masked) return cx<T>(0, 0);
        return a.omega * cmul(cinv(diag3(rx, ry, rz, c.op)), b);
    } else if (MODE == M_PROLONG_JACOBI) {
        // x + P e_c: trilinear interpolation of the coarse correction
        if (rx.masked || ry.masked) return cx<T>(0, 0);
        const Row1<T> rz = row1<T>(l, n, a.g.dir[4], a.g.dir[5], h, ih);
        if (rz.masked) return cx<T>(0, 0);
        const int nc = n >> 1, nnc = nc + 1;
        const int I0 = i >> 1, J0 = j >> 1, L0 = l >> 1;
        const bool oi = i & 1, oj = j & 1, ol = l & 1;
        Cx<T> e = cx<T>(0, 0);
#pragma unroll
        for (int cl = 0; cl < 2; ++cl) {
            if (cl == 1 && !ol) break;
            const int L = L0 + cl;
            if (coarse_dir(L, nc, a.g.dir[4], a.g.dir[5])) continue;
            const T wl = ol ? T(0.5) : T(1);
#pragma unroll
            for (int bj = 0; bj < 2; ++bj) {
                if (bj == 1 && !oj) break;
                const int J = J0 + bj;
                if (coarse_dir(J, nc, a.g.dir[2], a.g.dir[3])) continue;
                const T wj = oj ? T(0.5) * wl : wl;
#pragma unroll
                for (int ai = 0; ai < 2; ++ai) {
                    if (ai == 1 && !oi) break;
                    const int I = I0 + ai;
                    if (coarse_dir(I, nc, a.g.dir[0], a.g.dir[1])) continue;
                    const T w = oi ? T(0.5) * wj : wj;
                    e = fma_r(w, ld<T>(v.ec, ((long long)L * nnc + J) * nnc + I), e);
                }
            }
        }
        return ld<T>(v.x, p) + e;
    } else {
        return a.xzero ? cx<T>(0, 0) : ld<T>(v.x, p);
    }
}

constexpr int kWarps3 = 8;  // y-rows per tile, including the two halo rows

}  // namespace

// BATCH = false: a batch of one, coefficients from the kernel parameters, no activity flags.
template <typename T, int MODE, int R, bool BATCH>
__global__ void __launch_bounds__(32 * kWarps3) k_march3(const __grid_constant__ MArgs<T> a, int zt) {
    pdl_entry();
    const int b = BATCH ? (int)blockIdx.z / zt : 0;  // problem; blockIdx.z % zt: z-tile
    if (BATCH && problem_skipped(a, b)) return;
    const PCoef<T>& cf = BATCH ? a.pc[b] : a.c0;
    const VPtrs<T> v = problem_ptrs(a, b, false);
    constexpr int NP = R + 2;  // planes loaded
    constexpr bool NEEDZ = MODE != M_APPLY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [warp][plane][lane]: field value and x-neighbour sum
    vec2<T>* sv = reinterpret_cast<vec2<T>*>(smem_raw);
    vec2<T>* ss = sv + kWarps3 * NP * 32;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int n = a.g.n, nn = a.g.nn;
    const T h = a.h, ih = a.ih;
    const int i = blockIdx.x * 30 + lane - 1;
    const int j = blockIdx.y * (kWarps3 - 2) + w - 1;
    const int l0 = (blockIdx.z - b * zt) * R;
    const int ic = clampi3(i, 0, n), jc = clampi3(j, 0, n);
    const Row1<T> rx = row1<T>(ic, n, a.g.dir[0], a.g.dir[1], h, ih);
    const Row1<T> ry = row1<T>(jc, n, a.g.dir[2], a.g.dir[3], h, ih);

    Cx<T> fv[NP], xs[NP];
#pragma unroll
    for (int t = 0; t < NP; ++t) fv[t] = field3<T, MODE>(a, cf, v, ic, jc, clampi3(l0 - 1 + t, 0, n), rx, ry, h, ih);
    Cx<T> zv[R];
    const bool out_row = w >= 1 && w <= kWarps3 - 2;
#pragma unroll
    for (int t = 0; t < R; ++t)
        zv[t] = (NEEDZ && out_row) ? ld<T>(v.z, ((long long)clampi3(l0 + t, 0, n) * nn + jc) * nn + ic) : cx<T>(0, 0);
#pragma unroll
    for (int t = 0; t < NP; ++t) {
        xs[t] = shfl_up3(fv[t]) + shfl_dn3(fv[t]);
        st<T>(sv, (w * NP + t) * 32 + lane, fv[t]);
        st<T>(ss, (w * NP + t) * 32 + lane, xs[t]);
    }
    __syncthreads();
    if (!out_row || !(lane >= 1 && lane <= 30) || i > n || j > n) return;
    const bool colrow_fast = i >= 2 && i <= n - 2 && j >= 2 && j <= n - 2;
    const int wm = w - 1, wp = w + 1;
    // rows j-1 + j+1 summed (value and x-sum) per plane, in a rolling window of 3 planes
    auto ysum = [&](const vec2<T>* arr, int tpl) {
        return ld<T>(arr, (wm * NP + tpl) * 32 + lane) + ld<T>(arr, (wp * NP + tpl) * 32 + lane);
    };
    Cx<T> vy0 = ysum(sv, 0), vy1 = ysum(sv, 1), sy0 = ysum(ss, 0), sy1 = ysum(ss, 1);
#pragma unroll
    for (int t = 0; t < R; ++t) {
        const int l = l0 + t;
        if (l > n) break;
        const int tp = t + 1;  // local plane of the output
        const Cx<T> vy2 = ysum(sv, tp + 1), sy2 = ysum(ss, tp + 1);
        const long long p = ((long long)l * nn + j) * nn + i;
        Cx<T> ax, dinv_w;
        bool masked = false;
        if (colrow_fast && l >= 2 && l <= n - 2) {
            const Cx<T> face = xs[tp] + vy1 + (fv[tp - 1] + fv[tp + 1]);
            const Cx<T> edge = sy1 + (xs[tp - 1] + xs[tp + 1]) + (vy0 + vy2);
            const Cx<T> corner = sy0 + sy2;
            ax = fma_c(cf.iw[3], corner, fma_c(cf.iw[2], edge, fma_c(cf.iw[1], face, cmul(cf.iw[0], fv[tp]))));
            dinv_w = cf.wdinv;
        } else {
            const Row1<T> rz = row1<T>(l, n, a.g.dir[4], a.g.dir[5], h, ih);
            masked = rx.masked || ry.masked || rz.masked;
            const T myw[3] = {ry.ml, ry.mc, ry.mr};
            const T kyw[3] = {ry.kl, ry.kc, ry.kr};
            const T mzw[3] = {rz.ml, rz.mc, rz.mr};
            const T kzw[3] = {rz.kl, rz.kc, rz.kr};
            Cx<T> Mx = cx<T>(0, 0), Kx = cx<T>(0, 0), Fxf = cx<T>(0, 0), Fyf = cx<T>(0, 0), Fzf = cx<T>(0, 0);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Cx<T> PM = cx<T>(0, 0), PK = cx<T>(0, 0), Pf = cx<T>(0, 0), mxc = cx<T>(0, 0);
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int base = ((w - 1 + b) * NP + tp - 1 + c) * 32 + lane;
                    const Cx<T> v0 = ld<T>(sv, base - 1), v1 = ld<T>(sv, base), v2 = ld<T>(sv, base + 1);
                    const Cx<T> mx = fma_r(rx.mr, v2, fma_r(rx.mc, v1, rx.ml * v0));
                    const Cx<T> kx = fma_r(rx.kr, v2, fma_r(rx.kc, v1, rx.kl * v0));
                    PM = fma_r(myw[b], mx, PM);
                    PK = fma_r(myw[b], kx, fma_r(kyw[b], mx, PK));
                    Pf = fma_r(myw[b], v1, Pf);
                    if (b == 1) mxc = mx;
                }
                Mx = fma_r(mzw[c], PM, Mx);
                Kx = fma_r(mzw[c], PK, fma_r(kzw[c], PM, Kx));
                Fxf = fma_r(mzw[c], Pf, Fxf);
                Fyf = fma_r(mzw[c], mxc, Fyf);
                if (c == 1) Fzf = PM;
            }
            Cx<T> F = cx<T>(0, 0);
            if (rx.face) F = F + Fxf;
            if (ry.face) F = F + Fyf;
            if (rz.face) F = F + Fzf;
            ax = cf.op.cK * Kx;
            ax = fma_c(cf.op.cM, Mx, ax);
            ax = fma_c(cf.op.cG, F, ax);
            dinv_w = (MODE == M_APPLY || MODE == M_AXPBY) ? cx<T>(0, 0) : a.omega * cinv(diag3(rx, ry, rz, cf.opd));
        }
        const Cx<T> alpha = a.use_pc_ab ? cf.alpha : a.alpha, beta = a.use_pc_ab ? cf.beta : a.beta;
        if (masked) {
            st<T>(v.y, p, cx<T>(0, 0));
            if (MODE == M_HSS_FIRST) st<T>(v.y2, p, cx<T>(0, 0));
        } else if (MODE == M_APPLY) {
            st<T>(v.y, p, ax);
        } else if (MODE == M_AXPBY) {
            st<T>(v.y, p, fma_c(alpha, ax, cmul(beta, zv[t])));
        } else if (MODE == M_HSS_FIRST) {
            const Cx<T> rhs = fma_c(alpha, ax, cmul(beta, zv[t]));
            st<T>(v.y, p, rhs);
            st<T>(v.y2, p, cmul(dinv_w, rhs));
        } else {
            st<T>(v.y, p, fma_c(dinv_w, zv[t] - ax, fv[tp]));
        }
        vy0 = vy1;
        vy1 = vy2;
        sy0 = sy1;
        sy1 = sy2;
    }
}

template <typename T, int MODE, int R>
static cudaError_t go3(MArgs<T> a, cudaStream_t s) {
    // at most 40 KiB: within the default dynamic shared-memory limit, no opt-in needed
    const size_t smem = 2 * (size_t)kWarps3 * (R + 2) * 32 * sizeof(vec2<T>);
    static_assert(2 * kWarps3 * (R + 2) * 32 * sizeof(vec2<T>) <= 48 * 1024, "tile too large");
    const int zt = (a.g.nn + R - 1) / R;
    dim3 grd((unsigned)((a.g.nn + 29) / 30), (unsigned)((a.g.nn + kWarps3 - 3) / (kWarps3 - 2)),
             (unsigned)(zt * a.nb));
    if (a.pc) return klaunch(k_march3<T, MODE, R, true>, grd, dim3(32 * kWarps3), smem, s, 1, a, zt);
    if (a.nb != 1) return cudaErrorInvalidValue;
    return klaunch(k_march3<T, MODE, R, false>, grd, dim3(32 * kWarps3), smem, s, 1, a, zt);
}

template <typename T, int MODE>
static cudaError_t pick3(MArgs<T> a, cudaStream_t s) {
    a.h = T(a.g.h);
    a.ih = T(1.0 / a.g.h);
    // more planes per tile on large grids (fewer halo planes), fewer on small ones (more CTAs)
    const long long ctas4 = (long long)((a.g.nn + 29) / 30) * ((a.g.nn + 5) / 6) * ((a.g.nn + 3) / 4) * a.nb;
    if constexpr (sizeof(T) == 4) {
        if (a.tile_rows == 2) return go3<T, MODE, 2>(a, s);
        if (a.tile_rows == 4) return go3<T, MODE, 4>(a, s);
        if (a.tile_rows == 8 || ctas4 >= 152LL * 16) return go3<T, MODE, 8>(a, s);
        return go3<T, MODE, 4>(a, s);
    } else {
        return go3<T, MODE, 2>(a, s);
    }
}

template <typename T>
cudaError_t launch_march3(int mode, const MArgs<T>& a, cudaStream_t s) {
    if (a.g.dim != 3) return cudaErrorInvalidValue;
    switch (mode) {
        case M_APPLY: return pick3<T, M_APPLY>(a, s);
        case M_AXPBY: return pick3<T, M_AXPBY>(a, s);
        case M_JACOBI: return pick3<T, M_JACOBI>(a, s);
        case M_HSS_FIRST: return pick3<T, M_HSS_FIRST>(a, s);
        case M_JACOBI2_ZERO: return pick3<T, M_JACOBI2_ZERO>(a, s);
        case M_PROLONG_JACOBI: return pick3<T, M_PROLONG_JACOBI>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_march3<float>(int, const MArgs<float>&, cudaStream_t);
template cudaError_t launch_march3<double>(int, const MArgs<double>&, cudaStream_t);

}  // namespace hh
