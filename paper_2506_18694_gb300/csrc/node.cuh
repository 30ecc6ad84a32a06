// Per-node evaluation of a Q1 operator row from the 3^dim neighbourhood (generic
// one-thread-per-node form, used by the 3D kernels and the small-grid solvers).
#pragma once

#include "common.cuh"

namespace hh {

template <typename T> struct NodeResult {
    Cx<T> ax;  // (op x) at the node
    Cx<T> d;   // diagonal entry of op at the node
};

// (op x) and diag(op) at node (i,j) of a 2D grid; rows rx, ry precomputed.
// x is indexed by global node number minus `off` (a slab window of the grid).
template <typename T, bool NEED_AX>
__device__ __forceinline__ NodeResult<T> node2(const vec2<T>* __restrict__ x, int nn, int i, int j,
                                               const Row1<T>& rx, const Row1<T>& ry,
                                               const OpCoef<T>& op, long long off = 0) {
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
        const long long row = (long long)jb[b] * nn - off;
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
                                               const Row1<T>& rz, const OpCoef<T>& op, long long off = 0) {
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
            const long long row = ((long long)lc[c] * nn + jb[b]) * nn - off;
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

}  // namespace hh
