// 2D pre-smoothing fused with the residual restriction: the two pre-sweeps of a level (from
// x = 0, or the HSS right side and its two sweeps on the finest level) and r_c = P^T (b - A x)
// in one pass.  One warp owns a strip of fine columns and CR coarse rows; it forms each stage
// on a halo one row and one lane wider than the next needs, keeps everything in registers,
// writes the smoothed x (and the HSS right side) on its own fine rows and columns, and the
// restricted residual on its own coarse nodes.  Every node's arithmetic is that of the
// one-stage kernels (march2.cu), so the result equals the separate passes bit for bit.
#include "internal.h"
#include "march2_common.cuh"

namespace hh {

namespace {

// Geometry of a mode: lane of the first output column (fine column strip * S + lane - OFF),
// fine columns per strip, stencil rows loaded.
template <int MODE, int CR> struct RRGeo {
    static constexpr bool HSS = MODE == M_HSS_FIRST2_RR;
    static constexpr int OFF = HSS ? 4 : 3;
    static constexpr int S = HSS ? 24 : 26;
    static constexpr int NF = 2 * CR + (HSS ? 7 : 5);  // loaded rows
    static constexpr int RES0 = HSS ? 3 : 2;           // first residual row of the tile
};

}  // namespace

// grid (strips, ceil(chunks / 4), problems); chunk = CR coarse rows
template <typename T, int MODE, int CR, bool BATCH>
__global__ void __launch_bounds__(128) k_march2rr(const __grid_constant__ MArgs<T> a, int chunks) {
    using G = RRGeo<MODE, CR>;
    constexpr int NF = G::NF;
    pdl_entry();
    const int b = BATCH ? (int)blockIdx.z : 0;
    const int cy = blockIdx.y * 4 + (threadIdx.x >> 5);
    if (cy >= chunks) return;
    if (BATCH && problem_skipped(a, b)) return;
    const PCoef<T>& c = BATCH ? a.pc[b] : a.c0;    // first stage (A_R for the HSS step, else A_L)
    const PCoef<T>& cl = BATCH ? a.pc2[b] : a.c02;  // A_L
    const VPtrs<T> v = problem_ptrs(a, b, false);
    vec2<T>* __restrict__ yc = a.yc + (long long)b * a.bsc;
    const int lane = threadIdx.x & 31;
    const int n = a.g.n, nn = a.g.nn, nc = n >> 1;
    const int strip = blockIdx.x;
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
            acc = T(0.5) * rr;
        }
    }
}

template <typename T, int MODE>
static cudaError_t gorr(MArgs<T> a, cudaStream_t s) {
    using G1 = RRGeo<MODE, 1>;
    if (a.pc && !a.pc2) return cudaErrorInvalidValue;
    const int nnc = a.g.n / 2 + 1;
    const int strips = (a.g.nn + G1::S - 1) / G1::S;
    int cr = ((long long)strips * ((nnc + 1) / 2) * a.nb >= 24LL * num_sms()) ? 2 : 1;
    if (a.tile_rows == 1 || a.tile_rows == 2) cr = a.tile_rows;
    const int chunks = (nnc + cr - 1) / cr;
    const dim3 grd((unsigned)strips, (unsigned)((chunks + 3) / 4), (unsigned)a.nb);
    if (a.pc) {
        if (cr == 2) return klaunch(k_march2rr<T, MODE, 2, true>, grd, dim3(128), 0, s, 1, a, chunks);
        return klaunch(k_march2rr<T, MODE, 1, true>, grd, dim3(128), 0, s, 1, a, chunks);
    }
    if (a.nb != 1) return cudaErrorInvalidValue;
    if (cr == 2) return klaunch(k_march2rr<T, MODE, 2, false>, grd, dim3(128), 0, s, 1, a, chunks);
    return klaunch(k_march2rr<T, MODE, 1, false>, grd, dim3(128), 0, s, 1, a, chunks);
}

template <typename T>
cudaError_t launch_march2rr(int mode, const MArgs<T>& a, cudaStream_t s) {
    if (a.g.dim != 2 || a.g.n < 2 || (a.g.n & 1)) return cudaErrorInvalidValue;
    MArgs<T> b = a;
    b.h = T(a.g.h);
    b.ih = T(1.0 / a.g.h);
    switch (mode) {
        case M_JACOBI2_ZERO_RR: return gorr<T, M_JACOBI2_ZERO_RR>(b, s);
        case M_HSS_FIRST2_RR: return gorr<T, M_HSS_FIRST2_RR>(b, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_march2rr<float>(int, const MArgs<float>&, cudaStream_t);
template cudaError_t launch_march2rr<double>(int, const MArgs<double>&, cudaStream_t);

}  // namespace hh
