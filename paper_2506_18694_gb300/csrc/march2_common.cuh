// Device helpers shared by the 2D stencil kernels (march2.cu, march2rr.cu, coarse.cu and the
// persistent HSS loop, hssp.cu): warp shuffles of complex values, the zero-padding predicates,
// boundary classes, the per-node stencil, and the warp tiles of the fused passes (prolongation
// with two sweeps; two pre-sweeps with the residual restriction), so that every kernel that
// runs a pass computes each node with the same arithmetic.
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


// x + P e_c on the NR fine rows rfirst, rfirst + 1, ... of this lane's column ic (P = parity
// of rfirst), zero where no unknown lives.  Each coarse row the tile touches is read once
// per lane: the lane at an even fine column takes its coarse value, a lane at an odd column
// the mean of its own and its right neighbour's (by shuffle; lane 31 reads its second value
// itself); odd fine rows then average two interpolated coarse rows.  Coarse nodes on a
// Dirichlet side carry no basis function and count as zero.
template <typename T, int NR, int P>
__device__ __forceinline__ void prolong_rows(const MArgs<T>& a, const VPtrs<T>& v, int ic, int rfirst, bool cvoid,
                                             Cx<T>* out) {
    const int n = a.g.n, nc = n >> 1, nnc = nc + 1;
    const int lane = threadIdx.x & 31;
    const int I = ic >> 1;
    const int I1 = I + 1 <= nc ? I + 1 : nc;
    const bool odd = ic & 1;
    const bool v0 = (I == 0 && a.g.dir[0]) || (I == nc && a.g.dir[1]);
    const bool v1 = (I1 == 0 && a.g.dir[0]) || (I1 == nc && a.g.dir[1]);
    constexpr int NCR = ((P + NR) >> 1) + 1;
    const int J0 = rfirst >> 1;  // floor(rfirst / 2)
    Cx<T> ex[NCR];
#pragma unroll
    for (int q = 0; q < NCR; ++q) {
        const int J = J0 + q;
        const bool jv = J < 0 || J > nc || (J == 0 && a.g.dir[2]) || (J == nc && a.g.dir[3]);
        const long long row = (long long)clampi(J, 0, nc) * nnc;
        const Cx<T> c0 = (jv || v0) ? cx<T>(0, 0) : ld<T>(v.ec, row + I);
        Cx<T> c1 = shfl_dn(c0);
        if (lane == 31) c1 = (jv || v1) ? cx<T>(0, 0) : ld<T>(v.ec, row + I1);
        ex[q] = odd ? half_rn(c0 + c1) : c0;
    }
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        const int r = rfirst + t;
        const long long p = (long long)clampi(r, 0, n) * a.g.nn + ic;
        const int lq = (P + t) >> 1;
        const Cx<T> e = ((P + t) & 1) == 0 ? ex[lq] : half_rn(ex[lq] + ex[lq + 1]);
        out[t] = (cvoid || row_void(a, r)) ? cx<T>(0, 0) : ld<T>(v.x, p) + e;
    }
}

// ---- two sweeps in one pass ----
// Tile of the fused modes: 28 output columns (lanes 2..29) and ROWS output rows.  The field
// is loaded on ROWS + 4 rows; the first stage (a sweep, or the HSS right side and its
// pointwise first sweep) is formed on the ROWS + 2 rows and lanes 1..30 around the outputs,
// the second sweep on the outputs.  Every node's arithmetic is that of the one-sweep modes,
// so the result equals the two separate passes bit for bit.
template <typename T, int ROWS> struct TileF {
    static constexpr int NR = ROWS + 4;
    Cx<T> fv[NR];      // field: x + P ec (PROLONG_JACOBI2) or u (HSS_FIRST2)
    Cx<T> zv[NR - 2];  // b (PROLONG_JACOBI2) or r (HSS_FIRST2) on rows 1..NR-2
};

template <typename T, int MODE, int ROWS>
__device__ __forceinline__ void tilef_load(const MArgs<T>& a, const VPtrs<T>& v, int strip, int cy,
                                           TileF<T, ROWS>& tl) {
    constexpr int NR = TileF<T, ROWS>::NR;
    const int lane = threadIdx.x & 31;
    const int n = a.g.n;
    const int i = strip * 28 + lane - 2;
    const int rfirst = cy * ROWS - 2;
    const int ic = clampi(i, 0, n);
    const bool cvoid = col_void(a, i);
    if (MODE == M_PROLONG_JACOBI2) {
        prolong_rows<T, NR, 0>(a, v, ic, rfirst, cvoid, tl.fv);  // (first row cy * ROWS - 2 is even)
    } else {
#pragma unroll
        for (int t = 0; t < NR; ++t) {
            const int r = rfirst + t;
            const long long p = (long long)clampi(r, 0, n) * a.g.nn + ic;
            tl.fv[t] = (a.xzero || cvoid || row_void(a, r)) ? cx<T>(0, 0) : ld<T>(v.x, p);
        }
    }
#pragma unroll
    for (int t = 0; t < NR - 2; ++t) tl.zv[t] = ld<T>(v.z, (long long)clampi(rfirst + 1 + t, 0, n) * a.g.nn + ic);
}

template <typename T, int MODE, int ROWS>
__device__ __forceinline__ void tilef_compute(const MArgs<T>& a, const PCoef<T>& c, const PCoef<T>& cl,
                                              const VPtrs<T>& v, int strip, int cy, TileF<T, ROWS>& tl) {
    constexpr int NR = TileF<T, ROWS>::NR;
    const int lane = threadIdx.x & 31;
    const int n = a.g.n;
    const int i = strip * 28 + lane - 2;
    const int rfirst = cy * ROWS - 2;
    const int ic = clampi(i, 0, n);
    const bool col_in = (i >= 0 && i <= n);
    const bool col_inner = (i >= 1 && i <= n - 1);
    const bool cvoid = col_void(a, i);
    const int tx = ic == 0 ? 0 : (ic == n ? 2 : 1);
    const Cx<T>* fv = tl.fv;
    Cx<T> lf[NR], rg[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        lf[t] = shfl_up(fv[t]);
        rg[t] = shfl_dn(fv[t]);
    }
    // first stage on rows 1..NR-2: x1, and the right side of the second sweep
    Cx<T> x1[NR], b2[NR];
    x1[0] = x1[NR - 1] = b2[0] = b2[NR - 1] = cx<T>(0, 0);
    const Cx<T> alpha = a.use_pc_ab ? c.alpha : a.alpha, beta = a.use_pc_ab ? c.beta : a.beta;
#pragma unroll
    for (int t = 1; t < NR - 1; ++t) {
        const int j = rfirst + t;
        const int jc = clampi(j, 0, n);
        const bool fast = col_inner && j >= 1 && j <= n - 1;
        const int ty = jc == 0 ? 0 : (jc == n ? 2 : 1);
        Cx<T> ax, dinv_w;
        stencil_node2(c, fv[t - 1], fv[t], fv[t + 1], lf[t - 1], lf[t], lf[t + 1], rg[t - 1], rg[t], rg[t + 1], fast,
                      tx, ty, ax, dinv_w);
        const bool vd = cvoid || row_void(a, j);
        if (MODE == M_PROLONG_JACOBI2) {
            b2[t] = tl.zv[t - 1];
            x1[t] = vd ? cx<T>(0, 0) : fma_c(dinv_w, tl.zv[t - 1] - ax, fv[t]);
        } else {
            const Cx<T> rhs = fma_c(alpha, ax, cmul(beta, tl.zv[t - 1]));
            b2[t] = vd ? cx<T>(0, 0) : rhs;
            x1[t] = vd ? cx<T>(0, 0) : cmul(dinv_w, rhs);
        }
    }
    // second sweep (operator cl) on the output rows 2..NR-3
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        lf[t] = shfl_up(x1[t]);
        rg[t] = shfl_dn(x1[t]);
    }
#pragma unroll
    for (int t = 2; t < NR - 2; ++t) {
        const int j = rfirst + t;
        const bool row_in = (j >= 0 && j <= n);
        const int jc = clampi(j, 0, n);
        const bool fast = col_inner && j >= 1 && j <= n - 1;
        const int ty = jc == 0 ? 0 : (jc == n ? 2 : 1);
        Cx<T> ax, dinv_w;
        stencil_node2(cl, x1[t - 1], x1[t], x1[t + 1], lf[t - 1], lf[t], lf[t + 1], rg[t - 1], rg[t], rg[t + 1], fast,
                      tx, ty, ax, dinv_w);
        if (!(lane >= 2 && lane <= 29 && col_in && row_in)) continue;
        const long long p = (long long)jc * a.g.nn + ic;
        const bool masked = !fast && (cvoid || row_void(a, j));
        if (masked) {
            st<T>(v.y, p, cx<T>(0, 0));
            if (MODE == M_HSS_FIRST2) st<T>(v.y2, p, cx<T>(0, 0));
            continue;
        }
        const Cx<T> x2 = fma_c(dinv_w, b2[t] - ax, x1[t]);
        if (MODE == M_PROLONG_JACOBI2) {
            st<T>(v.y, p, x2);
        } else {
            st<T>(v.y, p, b2[t]);
            st<T>(v.y2, p, x2);
        }
    }
}

// Geometry of a mode: lane of the first output column (fine column strip * S + lane - OFF),
// fine columns per strip, stencil rows loaded.
template <int MODE, int CR> struct RRGeo {
    static constexpr bool HSS = MODE == M_HSS_FIRST2_RR;
    static constexpr int OFF = HSS ? 4 : 3;
    static constexpr int S = HSS ? 24 : 26;
    static constexpr int NF = 2 * CR + (HSS ? 7 : 5);  // loaded rows
    static constexpr int RES0 = HSS ? 3 : 2;           // first residual row of the tile
};

// One warp's tile of the pre-smoothing + residual-restriction pass: fine-column strip
// `strip`, coarse rows cy * CR .. cy * CR + CR - 1 of problem b.
template <typename T, int MODE, int CR, bool BATCH>
__device__ __forceinline__ void rr_tile(const MArgs<T>& a, int b, int strip, int cy) {
    using G = RRGeo<MODE, CR>;
    constexpr int NF = G::NF;
    const PCoef<T>& c = BATCH ? a.pc[b] : a.c0;    // first stage (A_R for the HSS step, else A_L)
    const PCoef<T>& cl = BATCH ? a.pc2[b] : a.c02;  // A_L
    const VPtrs<T> v = problem_ptrs(a, b, false);
    vec2<T>* __restrict__ yc = a.yc + (long long)b * a.bsc;
    const int lane = threadIdx.x & 31;
    const int n = a.g.n, nn = a.g.nn, nc = n >> 1;
    const int i = strip * G::S + lane - G::OFF;
    const int J0 = cy * CR;
    const int rfirst = 2 * J0 - 1 - G::RES0;  // fine row of tile row 0
    const int ic = clampi(i, 0, n);
    const bool col_in = i >= 0 && i <= n;
    const bool col_inner = i >= 1 && i <= n - 1;
    const bool cvoid = col_void(a, i);
    const int tx = ic == 0 ? 0 : (ic == n ? 2 : 1);
    auto row_of = [&](int t) { return rfirst + t; };
    auto ptr = [&](int t) { return (long long)clampi(row_of(t), 0, n) * nn + ic; };

    // ---- loads: the field source on every tile row, the right side where it is used
    Cx<T> f[NF], z[NF];
#pragma unroll
    for (int t = 0; t < NF; ++t) {
        if (G::HSS) {
            f[t] = (a.xzero || cvoid || row_void(a, row_of(t))) ? cx<T>(0, 0) : ld<T>(v.x, ptr(t));
            z[t] = (t >= 1 && t <= NF - 2) ? ld<T>(v.z, ptr(t)) : cx<T>(0, 0);
        } else {
            z[t] = ld<T>(v.z, ptr(t));  // b, also the source of the first sweep
            f[t] = cx<T>(0, 0);
        }
    }
    // ---- stage 1: the right side b of the sweeps and the first sweep x1
    Cx<T> bb[NF], x1[NF];
    if (G::HSS) {
        Cx<T> lf[NF], rg[NF];
#pragma unroll
        for (int t = 0; t < NF; ++t) {
            lf[t] = shfl_up(f[t]);
            rg[t] = shfl_dn(f[t]);
        }
        const Cx<T> alpha = a.use_pc_ab ? c.alpha : a.alpha, beta = a.use_pc_ab ? c.beta : a.beta;
        bb[0] = bb[NF - 1] = x1[0] = x1[NF - 1] = cx<T>(0, 0);
#pragma unroll
        for (int t = 1; t < NF - 1; ++t) {
            const int j = row_of(t), jc = clampi(j, 0, n);
            const bool fast = col_inner && j >= 1 && j <= n - 1;
            const int ty = jc == 0 ? 0 : (jc == n ? 2 : 1);
            Cx<T> ax, dinv_w;
            stencil_node2(c, f[t - 1], f[t], f[t + 1], lf[t - 1], lf[t], lf[t + 1], rg[t - 1], rg[t], rg[t + 1], fast,
                          tx, ty, ax, dinv_w);
            const bool vd = cvoid || row_void(a, j);
            const Cx<T> rhs = fma_c(alpha, ax, cmul(beta, z[t]));
            bb[t] = vd ? cx<T>(0, 0) : rhs;
            x1[t] = vd ? cx<T>(0, 0) : cmul(dinv_w, rhs);
        }
    } else {
        // first sweep from x = 0: x1 = omega D^{-1} b, zero where no unknown lives
#pragma unroll
        for (int t = 0; t < NF; ++t) {
            const int r = row_of(t);
            bb[t] = z[t];
            if (cvoid || row_void(a, r)) {
                x1[t] = cx<T>(0, 0);
            } else if (col_inner && r >= 1 && r <= n - 1) {
                x1[t] = cmul(cl.wdinv, z[t]);
            } else {
                const int ty = r == 0 ? 0 : (r == n ? 2 : 1);
                x1[t] = cmul(cl.bdinv[bclass2(tx, ty)], z[t]);
            }
        }
    }
    // ---- stage 2: the second sweep x2 on rows s2 .. NF - 1 - s2
    constexpr int s2 = G::HSS ? 2 : 1;
    Cx<T> x2[NF];
    {
        Cx<T> lf[NF], rg[NF];
#pragma unroll
        for (int t = 0; t < NF; ++t) {
            lf[t] = shfl_up(x1[t]);
            rg[t] = shfl_dn(x1[t]);
            x2[t] = cx<T>(0, 0);
        }
#pragma unroll
        for (int t = s2; t < NF - s2; ++t) {
            const int j = row_of(t), jc = clampi(j, 0, n);
            const bool fast = col_inner && j >= 1 && j <= n - 1;
            const int ty = jc == 0 ? 0 : (jc == n ? 2 : 1);
            Cx<T> ax, dinv_w;
            stencil_node2(cl, x1[t - 1], x1[t], x1[t + 1], lf[t - 1], lf[t], lf[t + 1], rg[t - 1], rg[t], rg[t + 1],
                          fast, tx, ty, ax, dinv_w);
            const bool vd = cvoid || row_void(a, j);
            x2[t] = vd ? cx<T>(0, 0) : fma_c(dinv_w, bb[t] - ax, x1[t]);
        }
    }
    // ---- the tile's own fine nodes: x2 (and the HSS right side)
    const bool own_col = lane >= G::OFF && lane < G::OFF + G::S && col_in;
#pragma unroll
    for (int t = G::RES0 + 1; t < G::RES0 + 1 + 2 * CR; ++t) {
        const int j = row_of(t);
        if (!own_col || j < 0 || j > n) continue;
        const long long p = (long long)j * nn + ic;
        if (G::HSS) {
            st<T>(v.y, p, bb[t]);
            st<T>(v.y2, p, x2[t]);
        } else {
            st<T>(v.y, p, x2[t]);
        }
    }
    // ---- residual b - A_L x2 on rows RES0 .. RES0 + 2 CR and its full-weighting restriction
    Cx<T> lf[NF], rg[NF];
#pragma unroll
    for (int t = 0; t < NF; ++t) {
        lf[t] = shfl_up(x2[t]);
        rg[t] = shfl_dn(x2[t]);
    }
    Cx<T> acc = cx<T>(0, 0);  // restriction accumulator of the coarse row in progress
#pragma unroll
    for (int t = G::RES0; t <= G::RES0 + 2 * CR; ++t) {
        const int j = row_of(t);
        const bool row_in = j >= 0 && j <= n;
        const int jc = clampi(j, 0, n);
        const bool fast = col_inner && j >= 1 && j <= n - 1;
        const int ty = jc == 0 ? 0 : (jc == n ? 2 : 1);
        Cx<T> ax, dinv_w;
        stencil_node2(cl, x2[t - 1], x2[t], x2[t + 1], lf[t - 1], lf[t], lf[t + 1], rg[t - 1], rg[t], rg[t + 1], fast,
                      tx, ty, ax, dinv_w);
        const bool masked = !fast && (cvoid || row_void(a, j));
        const Cx<T> res = (row_in && col_in && !masked) ? bb[t] - ax : cx<T>(0, 0);
        // full weighting along x: r(i) + (r(i-1) + r(i+1)) / 2
        const Cx<T> rr = fma_r(T(0.5), shfl_up(res) + shfl_dn(res), res);
        const int tl = t - G::RES0;  // 0 .. 2 CR; even: the first row of a coarse row, 2J - 1
        if (tl & 1) {
            acc = acc + rr;  // centre row 2J
        } else {
            if (tl >= 2) {  // row 2J + 1 closes coarse row J
                acc = fma_r(T(0.5), rr, acc);
                const int J = J0 + tl / 2 - 1;
                const int I = strip * (G::S / 2) + ((lane - G::OFF) >> 1);
                if (lane >= G::OFF && lane < G::OFF + G::S && !((lane - G::OFF) & 1) && I <= nc && J <= nc) {
                    const bool cm = (I == 0 && a.g.dir[0]) || (I == nc && a.g.dir[1]) || (J == 0 && a.g.dir[2]) ||
                                    (J == nc && a.g.dir[3]);
                    st<T>(yc, (long long)J * (nc + 1) + I, cm ? cx<T>(0, 0) : acc);
                }
            }
            acc = half_rn(rr);
        }
    }
}

// One scaled-Jacobi update of node pi of a padded 2D slab (row width W), with the weights of its
// kind (8 inner, else its boundary class): the arithmetic of stencil_node2.
template <typename T>
__device__ __forceinline__ Cx<T> coarse_update2(const PCoef<T>& c, const vec2<T>* __restrict__ xc, int pi, int W,
                                               int kind, Cx<T> bq) {
    const bool inner = kind == 8;
    const Cx<T> dinv = inner ? c.wdinv : c.bdinv[kind];
    const Cx<T> f0 = ld<T>(xc, pi), fm = ld<T>(xc, pi - W), fp = ld<T>(xc, pi + W);
    const Cx<T> l0 = ld<T>(xc, pi - 1), r0v = ld<T>(xc, pi + 1);
    const Cx<T> lm = ld<T>(xc, pi - W - 1), rm = ld<T>(xc, pi - W + 1);
    const Cx<T> lp = ld<T>(xc, pi + W - 1), rp = ld<T>(xc, pi + W + 1);
    Cx<T> ax;
    if (inner) {
        const Cx<T> edge = (l0 + r0v) + (fm + fp);
        const Cx<T> diag = (lm + rm) + (lp + rp);
        ax = fma_c(c.iw[2], diag, fma_c(c.iw[1], edge, cmul(c.iw[0], f0)));
    } else {
        const Cx<T> hx = l0 + r0v;
        const Cx<T> vy = fm + fp;
        const Cx<T> dg = (lm + rm) + (lp + rp);
        ax = fma_c(c.bw[kind][3], dg, fma_c(c.bw[kind][2], vy, fma_c(c.bw[kind][1], hx, cmul(c.bw[kind][0], f0))));
    }
    return fma_c(dinv, bq - ax, f0);
}


// The coarsest-level solve on one band of rows r0 .. r1 - 1 of problem b: nsw scaled-Jacobi sweeps
// from x = 0 with coefficients c, the result written to a.y.  The band and a halo of nsw - 1 rows
// on each side are staged in shared memory (smem: hss_band2_smem bytes) and every sweep runs
// there, the halo rows recomputed instead of exchanged, so that one CTA needs nothing from any
// other; each node's arithmetic is that of coarse_update2 (the one-sweep kernels' arithmetic).
template <typename T>
__host__ __device__ __forceinline__ size_t band2_smem(int nn, int nsw, int R) {
    const int H = nsw > 1 ? nsw - 1 : 0;
    return (size_t)3 * (R + 2 * H + 2) * (nn + 2) * sizeof(vec2<T>);
}

template <typename T>
__device__ __forceinline__ void coarse_band2(const MArgs<T>& a, const PCoef<T>& c, int b, int r0, int r1, int nsw,
                                             unsigned char* smem) {
    const int nn = a.g.nn, n = a.g.n, Wd = nn + 2;
    const int H = nsw > 1 ? nsw - 1 : 0;
    const int buf = (r1 - r0 + 2 * H + 2) * Wd;
    vec2<T>* xs[2] = {reinterpret_cast<vec2<T>*>(smem), reinterpret_cast<vec2<T>*>(smem) + buf};
    vec2<T>* bs = reinterpret_cast<vec2<T>*>(smem) + 2 * buf;
    const int top = r0 - H - 1;  // grid row of buffer row 0
    const vec2<T>* bz = a.z + (long long)b * a.bs;
    vec2<T>* y = a.y + (long long)b * a.bs;
    // iterates start at 0 (and stay 0 outside the grid and at Dirichlet nodes); the right side
    // of the band and its halo rows is staged once
    for (int q = threadIdx.x; q < 3 * buf; q += blockDim.x) st<T>(xs[0], q, cx<T>(0, 0));
    __syncthreads();
    {
        const int ja = max(r0 - H, 0), jb = min(r1 + H, nn);
        for (int q = threadIdx.x; q < (jb - ja) * nn; q += blockDim.x) {
            const int j = ja + q / nn, i = q - (q / nn) * nn;
            st<T>(bs, (j - top) * Wd + i + 1, ld<T>(bz, (long long)j * nn + i));
        }
    }
    __syncthreads();
    int cur = 0;
    for (int s = 1; s <= nsw; ++s) {
        const int ext = nsw - s;  // rows beyond the band that later sweeps still read
        const int ja = max(r0 - ext, 0), jb = min(r1 + ext, nn);
        const vec2<T>* xin = xs[cur];
        vec2<T>* xout = xs[cur ^ 1];
        for (int q = threadIdx.x; q < (jb - ja) * nn; q += blockDim.x) {
            const int j = ja + q / nn, i = q - (q / nn) * nn;
            const bool vd = (i == 0 && a.g.dir[0]) || (i == n && a.g.dir[1]) || (j == 0 && a.g.dir[2]) ||
                            (j == n && a.g.dir[3]);
            if (vd) continue;
            const int tx = i == 0 ? 0 : (i == n ? 2 : 1), ty = j == 0 ? 0 : (j == n ? 2 : 1);
            const int cls = ty * 3 + tx;
            const int kind = cls == 4 ? 8 : cls - (cls > 4);
            const int pi = (j - top) * Wd + i + 1;
            const Cx<T> bq = ld<T>(bs, pi);
            const Cx<T> xv = s == 1 ? cmul(kind == 8 ? c.wdinv : c.bdinv[kind], bq)
                                    : coarse_update2(c, xin, pi, Wd, kind, bq);
            st<T>(xout, pi, xv);
        }
        __syncthreads();
        cur ^= 1;
    }
    for (int q = threadIdx.x; q < (r1 - r0) * nn; q += blockDim.x) {
        const int j = r0 + q / nn, i = q - (q / nn) * nn;
        st<T>(y, (long long)j * nn + i, ld<T>(xs[cur], (j - top) * Wd + i + 1));
    }
}

}  // namespace hh
