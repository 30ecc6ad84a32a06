// Device helpers shared by the 2D stencil kernels (march2.cu, march2rr.cu): warp shuffles
// of complex values, the zero-padding predicates, boundary classes and the per-node stencil.
#pragma once

#include "internal.h"

namespace hh {

template <typename T>
__device__ __forceinline__ Cx<T> shfl_up(Cx<T> v) {
    return Cx<T>{__shfl_up_sync(0xffffffffu, v.re, 1), __shfl_up_sync(0xffffffffu, v.im, 1)};
}
template <typename T>
__device__ __forceinline__ Cx<T> shfl_dn(Cx<T> v) {
    return Cx<T>{__shfl_down_sync(0xffffffffu, v.re, 1), __shfl_down_sync(0xffffffffu, v.im, 1)};
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Boundary-class index of a node with axis types tx, ty (0 first node, 1 inner, 2 last);
// not called for the inner class.
__device__ __forceinline__ int bclass2(int tx, int ty) {
    const int c = ty * 3 + tx;
    return c - (c > 4);
}

// Whether node (i, r) of the tile holds no unknown: outside the grid or on a Dirichlet side.
template <typename T>
__device__ __forceinline__ bool col_void(const MArgs<T>& a, int i) {
    return i < 0 || i > a.g.n || (i == 0 && a.g.dir[0]) || (i == a.g.n && a.g.dir[1]);
}
template <typename T>
__device__ __forceinline__ bool row_void(const MArgs<T>& a, int r) {
    return r < 0 || r > a.g.n || (r == 0 && a.g.dir[2]) || (r == a.g.n && a.g.dir[3]);
}

// op f at row t of a tile column (interior weights or the node's boundary class), with
// omega D^{-1} of the record's opd.
template <typename T>
__device__ __forceinline__ void stencil_node2(const PCoef<T>& c, Cx<T> fm, Cx<T> f0, Cx<T> fp, Cx<T> lm, Cx<T> l0,
                                              Cx<T> lp, Cx<T> rm, Cx<T> r0, Cx<T> rp, bool fast, int tx, int ty,
                                              Cx<T>& ax, Cx<T>& dinv_w) {
    if (fast) {
        const Cx<T> edge = (l0 + r0) + (fm + fp);
        const Cx<T> diag = (lm + rm) + (lp + rp);
        ax = fma_c(c.iw[2], diag, fma_c(c.iw[1], edge, cmul(c.iw[0], f0)));
        dinv_w = c.wdinv;
    } else {
        const int q = bclass2(tx, ty);
        const Cx<T> hx = l0 + r0;
        const Cx<T> vy = fm + fp;
        const Cx<T> dg = (lm + rm) + (lp + rp);
        ax = fma_c(c.bw[q][3], dg, fma_c(c.bw[q][2], vy, fma_c(c.bw[q][1], hx, cmul(c.bw[q][0], f0))));
        dinv_w = c.bdinv[q];
    }
}

}  // namespace hh
