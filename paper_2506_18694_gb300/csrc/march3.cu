// 3D fused V-cycle kernels.  A CTA of 8 warps owns a tile of 30 x-nodes, 8 consecutive
// y-rows (the first and last are halo rows) and R + 2 consecutive z-planes (the first and
// last are halo planes); it writes the 30 x 6 x R interior outputs.  Warp w loads its row
// of every plane with one coalesced access per plane (all loads in flight before any
// arithmetic), forms the x-neighbour sum by warp shuffles, and publishes the value and the
// x-sum of each plane in shared memory; after one barrier the six output warps read rows
// j-1 and j+1 from shared memory and keep their own row in registers.  Interior nodes use
// the four neighbour-class weights of the 27-point Q1 operator (centre, face, edge,
// corner).  The field is loaded as zero outside the cube and at Dirichlet nodes, so a node
// on a face, edge or corner sums its existing neighbours by group (centre; x, y, z faces;
// xy, xz, yz edges; corners) with the eight weights of its boundary class.
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

__device__ __forceinline__ bool coarse_dir(int I, int nc, int lo, int hi) { return (I == 0 && lo) || (I == nc && hi); }

// Whether coordinate v of an axis with Dirichlet flags lo, hi holds no unknown.
__device__ __forceinline__ bool void1(int v, int n, int lo, int hi) {
    return v < 0 || v > n || (v == 0 && lo) || (v == n && hi);
}

__device__ __forceinline__ int type1(int v, int n) { return v <= 0 ? 0 : (v >= n ? 2 : 1); }

// Boundary-class index of a node with axis types tx, ty, tz (not all inner).
__device__ __forceinline__ int bclass3(int tx, int ty, int tz) {
    const int c = (tz * 3 + ty) * 3 + tx;
    return c - (c > 13);
}

// Value of the stencil field at node (i, j, l) of the grid (offset p), which holds an unknown
// there (INNER: the node is known to lie inside the cube, off every face).
template <typename T, int MODE, bool INNER>
__device__ __forceinline__ Cx<T> field3(const MArgs<T>& a, const PCoef<T>& c, const Cx<T>* bw, const VPtrs<T>& v,
                                        int i, int j, int l, long long p) {
    const int n = a.g.n;
    if (MODE == M_JACOBI2_ZERO) {
        // first sweep from x = 0: x1 = omega D^{-1} b
        const Cx<T> b = ld<T>(v.z, p);
        if (INNER || (i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1 && l >= 1 && l <= n - 1)) return cmul(c.wdinv, b);
        const int q = bclass3(type1(i, n), type1(j, n), type1(l, n));
        return cmul(bw[q * kClass3Len + 8], b);
    } else if (MODE == M_PROLONG_JACOBI) {
        // x + P e_c: trilinear interpolation of the coarse correction
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

// Window of a node: the field value (f*) and x-neighbour sum (x*) of its column on planes
// l-1, l, l+1, and the sums over rows j-1 and j+1 of the value (vy*) and of the x-sum (sy*).
template <typename T> struct Win3 {
    Cx<T> fm, f0, fp, xm, x0, xp, vy0, vy1, vy2, sy0, sy1, sy2;
};

// The output of one node (offset p) from its window: the 27-point product A x assembled by
// neighbour group, then the mode's update.  FAST: an interior node (the four weights of the
// interior stencil); else the eight group weights of the node's boundary class (tx, ty, l).
template <typename T, int MODE, bool FAST>
__device__ __forceinline__ void out3(const MArgs<T>& a, const PCoef<T>& cf, const Cx<T>* bw, const VPtrs<T>& v,
                                     const Win3<T>& q, Cx<T> zq, int tx, int ty, int l, bool cvoid, long long p) {
    const int n = a.g.n;
    Cx<T> ax, dinv_w;
    bool masked = false;
    if (FAST) {
        const Cx<T> face = q.x0 + q.vy1 + (q.fm + q.fp);
        const Cx<T> edge = q.sy1 + (q.xm + q.xp) + (q.vy0 + q.vy2);
        const Cx<T> corner = q.sy0 + q.sy2;
        ax = fma_c(cf.iw[3], corner, fma_c(cf.iw[2], edge, fma_c(cf.iw[1], face, cmul(cf.iw[0], q.f0))));
        dinv_w = cf.wdinv;
    } else {
        // neighbour groups: centre; x, y, z faces; xy, xz, yz edges; corners
        masked = cvoid || void1(l, n, a.g.dir[4], a.g.dir[5]);
        const Cx<T>* wq = bw + bclass3(tx, ty, type1(l, n)) * kClass3Len;
        ax = cmul(wq[0], q.f0);
        ax = fma_c(wq[1], q.x0, ax);
        ax = fma_c(wq[2], q.vy1, ax);
        ax = fma_c(wq[3], q.fm + q.fp, ax);
        ax = fma_c(wq[4], q.sy1, ax);
        ax = fma_c(wq[5], q.xm + q.xp, ax);
        ax = fma_c(wq[6], q.vy0 + q.vy2, ax);
        ax = fma_c(wq[7], q.sy0 + q.sy2, ax);
        dinv_w = wq[8];
    }
    const Cx<T> alpha = a.use_pc_ab ? cf.alpha : a.alpha, beta = a.use_pc_ab ? cf.beta : a.beta;
    if (masked) {
        st<T>(v.y, p, cx<T>(0, 0));
        if (MODE == M_HSS_FIRST) st<T>(v.y2, p, cx<T>(0, 0));
    } else if (MODE == M_APPLY) {
        st<T>(v.y, p, ax);
    } else if (MODE == M_AXPBY) {
        st<T>(v.y, p, fma_c(alpha, ax, cmul(beta, zq)));
    } else if (MODE == M_DAXPBY) {
        st<T>(v.y, p, cmul(dinv_w, fma_c(alpha, ax, cmul(beta, zq))));
    } else if (MODE == M_HSS_FIRST) {
        const Cx<T> rhs = fma_c(alpha, ax, cmul(beta, zq));
        st<T>(v.y, p, rhs);
        st<T>(v.y2, p, cmul(dinv_w, rhs));
    } else {
        st<T>(v.y, p, fma_c(dinv_w, zq - ax, q.f0));
    }
}

}  // namespace

// One tile.  INNER: every node the tile loads (halos included) lies inside the cube, off every
// face, so no node is void or on the boundary and no check or boundary-class code is needed;
// the node arithmetic is the same as on the general path.
template <typename T, int MODE, int R, bool BATCH, bool INNER>
__device__ __forceinline__ void march3_tile(const MArgs<T>& a, int b, int bx, int by, int l0,
                                            unsigned char* smem_raw) {
    const PCoef<T>& cf = BATCH ? a.pc[b] : a.c0;
    const Cx<T>* bw = a.bw3 + (long long)b * kClass3 * kClass3Len;
    const VPtrs<T> v = problem_ptrs(a, b, false);
    constexpr int NP = R + 2;  // planes loaded
    constexpr bool NEEDZ = MODE != M_APPLY;
    // [warp][plane][lane]: field value and x-neighbour sum
    vec2<T>* sv = reinterpret_cast<vec2<T>*>(smem_raw);
    vec2<T>* ss = sv + kWarps3 * NP * 32;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int n = a.g.n, nn = a.g.nn;
    const int i = bx * 30 + lane - 1;
    const int j = by * (kWarps3 - 2) + w - 1;
    const int ic = INNER ? i : clampi3(i, 0, n), jc = INNER ? j : clampi3(j, 0, n);
    const bool cvoid = !INNER && (void1(i, n, a.g.dir[0], a.g.dir[1]) || void1(j, n, a.g.dir[2], a.g.dir[3]));
    const long long ps = (long long)nn * nn;
    const long long colc = (long long)jc * nn + ic;

    Cx<T> fv[NP], xs[NP];
#pragma unroll
    for (int t = 0; t < NP; ++t) {
        const int l = l0 - 1 + t;
        // (a node of a plane that is not void lies inside the cube: no clamp needed)
        fv[t] = (!INNER && (cvoid || void1(l, n, a.g.dir[4], a.g.dir[5])))
                    ? cx<T>(0, 0)
                    : field3<T, MODE, INNER>(a, cf, bw, v, ic, jc, l, colc + l * ps);
    }
    Cx<T> zv[R];
    const bool out_row = w >= 1 && w <= kWarps3 - 2;
#pragma unroll
    for (int t = 0; t < R; ++t)
        zv[t] = (NEEDZ && out_row) ? ld<T>(v.z, colc + (INNER ? l0 + t : clampi3(l0 + t, 0, n)) * ps) : cx<T>(0, 0);
#pragma unroll
    for (int t = 0; t < NP; ++t) {
        xs[t] = shfl_up3(fv[t]) + shfl_dn3(fv[t]);
        st<T>(sv, (w * NP + t) * 32 + lane, fv[t]);
        st<T>(ss, (w * NP + t) * 32 + lane, xs[t]);
    }
    __syncthreads();
    if (!out_row || !(lane >= 1 && lane <= 30) || (!INNER && (i > n || j > n))) return;
    const bool colrow_inner = INNER || (i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1);
    const int tx = type1(i, n), ty = type1(j, n);
    const int wm = w - 1, wp = w + 1;
    // rows j-1 + j+1 summed (value and x-sum) per plane, in a rolling window of 3 planes
    auto ysum = [&](const vec2<T>* arr, int tpl) {
        return ld<T>(arr, (wm * NP + tpl) * 32 + lane) + ld<T>(arr, (wp * NP + tpl) * 32 + lane);
    };
    Win3<T> q;
    q.vy0 = ysum(sv, 0);
    q.vy1 = ysum(sv, 1);
    q.sy0 = ysum(ss, 0);
    q.sy1 = ysum(ss, 1);
#pragma unroll
    for (int t = 0; t < R; ++t) {
        const int l = l0 + t;
        if (!INNER && l > n) break;
        const int tp = t + 1;  // local plane of the output
        q.vy2 = ysum(sv, tp + 1);
        q.sy2 = ysum(ss, tp + 1);
        q.fm = fv[tp - 1];
        q.f0 = fv[tp];
        q.fp = fv[tp + 1];
        q.xm = xs[tp - 1];
        q.x0 = xs[tp];
        q.xp = xs[tp + 1];
        const long long p = colc + l * ps;
        if (INNER || (colrow_inner && l >= 1 && l <= n - 1))
            out3<T, MODE, true>(a, cf, bw, v, q, zv[t], tx, ty, l, cvoid, p);
        else
            out3<T, MODE, false>(a, cf, bw, v, q, zv[t], tx, ty, l, cvoid, p);
        q.vy0 = q.vy1;
        q.vy1 = q.vy2;
        q.sy0 = q.sy1;
        q.sy1 = q.sy2;
    }
}

// Whether tile (bx, by, z from l0) with its halos lies inside the cube, off every face.
__device__ __forceinline__ bool tile_inner3(int n, int bx, int by, int l0, int R) {
    const int i0 = bx * 30 - 1, j0 = by * (kWarps3 - 2) - 1, z0 = l0 - 1;
    return i0 >= 1 && i0 + 31 <= n - 1 && j0 >= 1 && j0 + kWarps3 - 1 <= n - 1 && z0 >= 1 && z0 + R + 1 <= n - 1;
}

// BATCH = false: a batch of one, coefficients from the kernel parameters, no activity flags.
// Each CTA takes the check-free path when its whole tile (halos included) lies inside the cube.
template <typename T, int MODE, int R, bool BATCH>
__global__ void __launch_bounds__(32 * kWarps3) k_march3(const __grid_constant__ MArgs<T> a, int zt) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = BATCH ? (int)blockIdx.z / zt : 0;  // problem; blockIdx.z % zt: z-tile
    if (BATCH && problem_skipped(a, b)) return;
    const int l0 = (blockIdx.z - b * zt) * R;
    if (tile_inner3(a.g.n, blockIdx.x, blockIdx.y, l0, R))
        march3_tile<T, MODE, R, BATCH, true>(a, b, blockIdx.x, blockIdx.y, l0, smem_raw);
    else
        march3_tile<T, MODE, R, BATCH, false>(a, b, blockIdx.x, blockIdx.y, l0, smem_raw);
}

// Weights of the 3D boundary classes.  1D rows (Q1): stiffness (1/h)(-1, cnt, -1), mass
// (h/6)(1, 2 cnt, 1), cnt = 2 inside and 1 at the ends of the axis.  Group S (the axes along
// which the neighbour is offset) has stiffness weight sum_a K_a prod_{b != a} M_b and mass
// weight prod_b M_b, with K_a, M_b the side weights (-1/h, h/6) on offset axes and the
// centre weights otherwise; a node on the side of axis a also carries the 2D boundary mass
// of that face, prod_{b != a} M_b, for the groups not offset along a.
template <typename T>
void boundary_weights3(Cx<T>* out, const PCoef<T>& c, const GridDesc& g, double omega) {
    const double h = g.h, ks = -1.0 / h, ms = h / 6.0;
    // groups: centre; x, y, z faces; xy, xz, yz edges; corners (bit a set: offset along axis a)
    const int groups[8] = {0, 1, 2, 4, 3, 5, 6, 7};
    for (int tz = 0; tz < 3; ++tz)
        for (int ty = 0; ty < 3; ++ty)
            for (int tx = 0; tx < 3; ++tx) {
                const int cl = (tz * 3 + ty) * 3 + tx;
                if (cl == 13) continue;
                const int q = cl - (cl > 13);
                const int typ[3] = {tx, ty, tz};
                double kc[3], mc[3];
                for (int a = 0; a < 3; ++a) {
                    const double cnt = typ[a] == 1 ? 2.0 : 1.0;
                    kc[a] = cnt / h;
                    mc[a] = cnt * h / 3.0;
                }
                double A[8], M[8], F[8];
                for (int u = 0; u < 8; ++u) {
                    const int S = groups[u];
                    double kk[3], mm[3];
                    for (int a = 0; a < 3; ++a) {
                        const bool off = (S >> a) & 1;
                        kk[a] = off ? ks : kc[a];
                        mm[a] = off ? ms : mc[a];
                    }
                    A[u] = kk[0] * mm[1] * mm[2] + mm[0] * kk[1] * mm[2] + mm[0] * mm[1] * kk[2];
                    M[u] = mm[0] * mm[1] * mm[2];
                    F[u] = 0.0;
                    for (int a = 0; a < 3; ++a)
                        if (typ[a] != 1 && !((S >> a) & 1)) F[u] += mm[(a + 1) % 3] * mm[(a + 2) % 3];
                }
                Cx<T>* o = out + (size_t)q * kClass3Len;
                for (int u = 0; u < 8; ++u)
                    o[u] = cx<T>(T(double(c.op.cK) * A[u] + double(c.op.cM.re) * M[u] + double(c.op.cG.re) * F[u]),
                                 T(double(c.op.cM.im) * M[u] + double(c.op.cG.im) * F[u]));
                const double dr = double(c.opd.cK) * A[0] + double(c.opd.cM.re) * M[0] + double(c.opd.cG.re) * F[0];
                const double di = double(c.opd.cM.im) * M[0] + double(c.opd.cG.im) * F[0];
                const double d2 = dr * dr + di * di;
                o[8] = d2 > 0 ? cx<T>(T(omega * dr / d2), T(-omega * di / d2)) : cx<T>(T(0), T(0));
            }
}

template void boundary_weights3<float>(Cx<float>*, const PCoef<float>&, const GridDesc&, double);
template void boundary_weights3<double>(Cx<double>*, const PCoef<double>&, const GridDesc&, double);

template <typename T, int MODE, int R>
static cudaError_t go3(MArgs<T> a, cudaStream_t s) {
    // at most 40 KiB: within the default dynamic shared-memory limit, no opt-in needed
    const size_t smem = 2 * (size_t)kWarps3 * (R + 2) * 32 * sizeof(vec2<T>);
    static_assert(2 * kWarps3 * (R + 2) * 32 * sizeof(vec2<T>) <= 48 * 1024, "tile too large");
    const int zt = (a.g.nn + R - 1) / R;
    const int tx = (a.g.nn + 29) / 30, ty = (a.g.nn + kWarps3 - 3) / (kWarps3 - 2);
    dim3 grd((unsigned)tx, (unsigned)ty, (unsigned)(zt * a.nb));
    if (a.pc) return klaunch(k_march3<T, MODE, R, true>, grd, dim3(32 * kWarps3), smem, s, 1, a, zt);
    if (a.nb != 1) return cudaErrorInvalidValue;
    return klaunch(k_march3<T, MODE, R, false>, grd, dim3(32 * kWarps3), smem, s, 1, a, zt);
}

template <typename T, int MODE>
static cudaError_t pick3(MArgs<T> a, cudaStream_t s) {
    a.h = T(a.g.h);
    a.ih = T(1.0 / a.g.h);
    // 4 planes per tile unless tuned otherwise (measured best on 257^3: 8 planes halve the
    // resident CTAs, 2 planes double the halo planes)
    if constexpr (sizeof(T) == 4) {
        if (a.tile_rows == 2) return go3<T, MODE, 2>(a, s);
        if (a.tile_rows == 8) return go3<T, MODE, 8>(a, s);
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
        case M_DAXPBY: return pick3<T, M_DAXPBY>(a, s);
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
