// 2D fused V-cycle kernels: one warp owns a strip of 32 consecutive x-nodes (30 outputs,
// one halo lane on each side) and marches along y.  Each step loads one row of the
// stencil field with a single coalesced 256-byte access per warp, takes the x-neighbours
// from the adjacent lanes with warp shuffles, forms the x-direction mass and stiffness
// passes once per row and keeps them for the three output rows that use them.  The Q1
// row weights (1D stiffness/mass triples per axis, Dirichlet elimination, Sommerfeld
// side mass) are the same as in stencil.cu; the modes below fuse the V-cycle's vector
// updates into the stencil pass so that each fine-level sweep reads and writes each
// vector once.
#include <algorithm>

#include "internal.h"
#include "march2_common.cuh"

namespace hh {

// One warp tile: a strip of 30 output columns (lanes 1..30; lanes 0 and 31 are the halo)
// and ROWS consecutive output rows (RESID_RESTRICT: ROWS coarse rows, 2 ROWS + 1 residual
// rows, 28 fine columns per strip).  tile_load issues every load of the tile (all in
// flight at once); tile_compute does the arithmetic and the stores.  The stencil field is
// loaded as zero outside the grid and at Dirichlet nodes (their unknowns are eliminated),
// so every node sums its existing neighbours by group: inner nodes with the interior
// weights (centre, edge, diagonal), nodes on a side with the weights of their boundary
// class (centre, x-neighbours, y-neighbours, diagonals).
template <typename T, int MODE, int ROWS> struct Tile2 {
    static constexpr bool RR = MODE == M_RESID_RESTRICT;
    static constexpr int NR = RR ? 2 * ROWS + 3 : ROWS + 2;  // stencil rows
    static constexpr int NZ = NR - 2;                         // rows whose right side is read
    static constexpr bool NEEDZ = MODE != M_APPLY && MODE != M_JACOBI2_ZERO;
    Cx<T> fv[NR];  // stencil field (M_JACOBI2_ZERO: filled from bv in tile_compute)
    Cx<T> bv[NR];  // right side on every stencil row (M_JACOBI2_ZERO only)
    Cx<T> zv[NZ];  // right side / second vector on the output rows
};

template <typename T, int MODE, int ROWS>
__device__ __forceinline__ void tile_load(const MArgs<T>& a, const VPtrs<T>& v, int strip, int cy,
                                          Tile2<T, MODE, ROWS>& tl) {
    using TL = Tile2<T, MODE, ROWS>;
    const int lane = threadIdx.x & 31;
    const int n = a.g.n;
    const int i = strip * (TL::RR ? 28 : 30) + lane - (TL::RR ? 2 : 1);
    const int base = cy * ROWS;
    const int rfirst = TL::RR ? 2 * base - 2 : base - 1;
    const int ic = clampi(i, 0, n);
    const bool cvoid = col_void(a, i);
    // (ROWS is even, so the first stencil row base - 1 is odd)
    if (MODE == M_PROLONG_JACOBI) prolong_rows<T, TL::NR, 1>(a, v, ic, rfirst, cvoid, tl.fv);
#pragma unroll
    for (int t = 0; t < TL::NR; ++t) {
        const int r = rfirst + t;
        const int rc = clampi(r, 0, n);
        const long long p = (long long)rc * a.g.nn + ic;
        const bool vd = cvoid || row_void(a, r);
        if (MODE == M_JACOBI2_ZERO) {
            tl.bv[t] = ld<T>(v.z, p);
        } else if (MODE != M_PROLONG_JACOBI) {
            tl.fv[t] = (a.xzero || vd) ? cx<T>(0, 0) : ld<T>(v.x, p);
        }
    }
#pragma unroll
    for (int t = 0; t < TL::NZ; ++t)
        tl.zv[t] = TL::NEEDZ ? ld<T>(v.z, (long long)clampi(rfirst + 1 + t, 0, n) * a.g.nn + ic) : cx<T>(0, 0);
}

template <typename T, int MODE, int ROWS>
__device__ __forceinline__ void tile_compute(const MArgs<T>& a, const PCoef<T>& c, const VPtrs<T>& v, int strip,
                                             int cy, Tile2<T, MODE, ROWS>& tl) {
    using TL = Tile2<T, MODE, ROWS>;
    constexpr bool RR = TL::RR;
    constexpr int NR = TL::NR;
    const int lane = threadIdx.x & 31;
    const int n = a.g.n;
    const int nc = n >> 1;
    const int i = strip * (RR ? 28 : 30) + lane - (RR ? 2 : 1);
    const int base = cy * ROWS;
    const int rfirst = RR ? 2 * base - 2 : base - 1;
    const int ic = clampi(i, 0, n);
    const bool col_in = (i >= 0 && i <= n);
    const bool col_inner = (i >= 1 && i <= n - 1);
    const bool cvoid = col_void(a, i);
    const int tx = ic == 0 ? 0 : (ic == n ? 2 : 1);

    if (MODE == M_JACOBI2_ZERO) {
        // first sweep from x = 0: x1 = omega D^{-1} b, zero where no unknown lives
#pragma unroll
        for (int t = 0; t < NR; ++t) {
            const int r = rfirst + t;
            if (cvoid || row_void(a, r)) {
                tl.fv[t] = cx<T>(0, 0);
            } else if (col_inner && r >= 1 && r <= n - 1) {
                tl.fv[t] = cmul(c.wdinv, tl.bv[t]);
            } else {
                const int ty = r == 0 ? 0 : (r == n ? 2 : 1);
                tl.fv[t] = cmul(c.bdinv[bclass2(tx, ty)], tl.bv[t]);
            }
        }
    }
    const Cx<T>* fv = tl.fv;
    Cx<T> lf[NR], rg[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        lf[t] = shfl_up(fv[t]);
        rg[t] = shfl_dn(fv[t]);
    }

    Cx<T> acc = cx<T>(0, 0);  // restriction accumulator of the coarse row in progress
#pragma unroll
    for (int t = 1; t < NR - 1; ++t) {
        const int j = rfirst + t;
        const bool row_in = (j >= 0 && j <= n);
        const bool fast = col_inner && j >= 1 && j <= n - 1;
        const int jc = clampi(j, 0, n);
        const long long p = (long long)jc * a.g.nn + ic;
        Cx<T> ax;
        Cx<T> dinv_w;  // omega D^{-1} of opd at the node
        bool masked = false;
        if (fast) {
            const Cx<T> edge = (lf[t] + rg[t]) + (fv[t - 1] + fv[t + 1]);
            const Cx<T> diag = (lf[t - 1] + rg[t - 1]) + (lf[t + 1] + rg[t + 1]);
            ax = fma_c(c.iw[2], diag, fma_c(c.iw[1], edge, cmul(c.iw[0], fv[t])));
            dinv_w = c.wdinv;
        } else {
            const int ty = jc == 0 ? 0 : (jc == n ? 2 : 1);
            const int q = bclass2(tx, ty);
            const Cx<T> hx = lf[t] + rg[t];
            const Cx<T> vy = fv[t - 1] + fv[t + 1];
            const Cx<T> dg = (lf[t - 1] + rg[t - 1]) + (lf[t + 1] + rg[t + 1]);
            ax = fma_c(c.bw[q][3], dg, fma_c(c.bw[q][2], vy, fma_c(c.bw[q][1], hx, cmul(c.bw[q][0], fv[t]))));
            dinv_w = c.bdinv[q];
            masked = cvoid || row_void(a, j);
        }
        if (RR) {
            const Cx<T> res = (row_in && col_in && !masked) ? tl.zv[t - 1] - ax : cx<T>(0, 0);
            // full weighting along x: r(i) + (r(i-1) + r(i+1)) / 2
            const Cx<T> rr = fma_r(T(0.5), shfl_up(res) + shfl_dn(res), res);
            if ((t & 1) == 0) {  // j = 2 base - 1 + t - 1 is even: centre row of coarse row j/2
                acc = acc + rr;
            } else {
                if (t >= 3) {  // odd row closes coarse row (j - 1)/2
                    acc = fma_r(T(0.5), rr, acc);
                    const int J = (j - 1) >> 1;
                    const int I = strip * 14 + ((lane - 2) >> 1);
                    if (lane >= 2 && lane <= 28 && !(lane & 1) && I <= nc && J <= nc) {
                        const bool cm = (I == 0 && a.g.dir[0]) || (I == nc && a.g.dir[1]) ||
                                        (J == 0 && a.g.dir[2]) || (J == nc && a.g.dir[3]);
                        st<T>(v.y, (long long)J * (nc + 1) + I, cm ? cx<T>(0, 0) : acc);
                    }
                }
                acc = half_rn(rr);
            }
            continue;
        }
        if (!(lane >= 1 && lane <= 30 && col_in && row_in)) continue;
        if (masked) {
            st<T>(v.y, p, cx<T>(0, 0));
            if (MODE == M_HSS_FIRST) st<T>(v.y2, p, cx<T>(0, 0));
            continue;
        }
        const Cx<T> alpha = a.use_pc_ab ? c.alpha : a.alpha, beta = a.use_pc_ab ? c.beta : a.beta;
        if (MODE == M_APPLY) {
            st<T>(v.y, p, ax);
        } else if (MODE == M_AXPBY) {
            st<T>(v.y, p, fma_c(alpha, ax, cmul(beta, tl.zv[t - 1])));
        } else if (MODE == M_DAXPBY) {
            st<T>(v.y, p, cmul(dinv_w, fma_c(alpha, ax, cmul(beta, tl.zv[t - 1]))));
        } else if (MODE == M_HSS_FIRST) {
            const Cx<T> rhs = fma_c(alpha, ax, cmul(beta, tl.zv[t - 1]));
            st<T>(v.y, p, rhs);
            st<T>(v.y2, p, cmul(dinv_w, rhs));
        } else {
            // Jacobi update of the field: field + omega D^{-1} (b - op field)
            const Cx<T> b = (MODE == M_JACOBI2_ZERO) ? tl.bv[t] : tl.zv[t - 1];
            st<T>(v.y, p, fma_c(dinv_w, b - ax, fv[t]));
        }
    }
}

// grid (strips of 28 columns, ceil(chunks / 4), problems)
template <typename T, int MODE, int ROWS, bool BATCH>
__global__ void __launch_bounds__(128) k_march2f(const __grid_constant__ MArgs<T> a, int chunks) {
    pdl_entry();
    const int b = BATCH ? (int)blockIdx.z : 0;
    const int cy = blockIdx.y * 4 + (threadIdx.x >> 5);
    if (cy >= chunks) return;
    if (BATCH && problem_skipped(a, b)) return;
    const PCoef<T>& c = BATCH ? a.pc[b] : a.c0;
    const PCoef<T>& cl = BATCH ? a.pc2[b] : a.c02;
    const VPtrs<T> v = problem_ptrs(a, b, false);
    TileF<T, ROWS> tl;
    tilef_load<T, MODE, ROWS>(a, v, blockIdx.x, cy, tl);
    tilef_compute<T, MODE, ROWS>(a, c, cl, v, blockIdx.x, cy, tl);
}

template <typename T, int MODE>
static cudaError_t gof(MArgs<T> a, cudaStream_t s) {
    a.h = T(a.g.h);
    a.ih = T(1.0 / a.g.h);
    if (a.pc && !a.pc2) return cudaErrorInvalidValue;
    const int strips = (a.g.nn + 27) / 28;
    int rows = ((long long)strips * ((a.g.nn + 3) / 4) * a.nb >= 24LL * num_sms()) ? 4 : 2;
    if (a.tile_rows == 2 || a.tile_rows == 4) rows = a.tile_rows;
    const int chunks = (a.g.nn + rows - 1) / rows;
    const dim3 grd((unsigned)strips, (unsigned)((chunks + 3) / 4), (unsigned)a.nb);
    if (a.pc) {
        if (rows == 4) return klaunch(k_march2f<T, MODE, 4, true>, grd, dim3(128), 0, s, 1, a, chunks);
        return klaunch(k_march2f<T, MODE, 2, true>, grd, dim3(128), 0, s, 1, a, chunks);
    }
    if (a.nb != 1) return cudaErrorInvalidValue;
    if (rows == 4) return klaunch(k_march2f<T, MODE, 4, false>, grd, dim3(128), 0, s, 1, a, chunks);
    return klaunch(k_march2f<T, MODE, 2, false>, grd, dim3(128), 0, s, 1, a, chunks);
}

// One tile per warp; grid (strips, ceil(chunks / 4), problems).  BATCH = false: a batch of
// one, coefficients from the kernel parameters and no activity flags.
template <typename T, int MODE, int ROWS, bool BATCH>
__global__ void __launch_bounds__(128) k_march2(const __grid_constant__ MArgs<T> a, int chunks) {
    pdl_entry();
    const int b = BATCH ? (int)blockIdx.z : 0;
    const int cy = blockIdx.y * 4 + (threadIdx.x >> 5);
    if (cy >= chunks) return;
    if (BATCH && problem_skipped(a, b)) return;
    const PCoef<T>& c = BATCH ? a.pc[b] : a.c0;
    const VPtrs<T> v = problem_ptrs(a, b, MODE == M_RESID_RESTRICT);
    Tile2<T, MODE, ROWS> tl;
    tile_load<T, MODE, ROWS>(a, v, blockIdx.x, cy, tl);
    tile_compute<T, MODE, ROWS>(a, c, v, blockIdx.x, cy, tl);
}

// Persistent form for grids with many more tiles than resident warps: each warp walks the
// tiles t, t + W, t + 2W, ... (strip fastest; in a batch, the problems' tiles one after
// another) and issues the loads of its next tile before computing the current one, so that
// its loads stay in flight while it computes.
template <typename T, int MODE, int ROWS, bool BATCH>
__global__ void __launch_bounds__(128) k_march2p(const __grid_constant__ MArgs<T> a, int strips, int per_problem,
                                                 int tiles) {
    pdl_entry();
    const int W = gridDim.x * 4;
    int t = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (t >= tiles) return;
    if constexpr (!BATCH) {
        const PCoef<T>& c = a.c0;
        const VPtrs<T> v = problem_ptrs(a, 0, MODE == M_RESID_RESTRICT);
        Tile2<T, MODE, ROWS> cur;
        tile_load<T, MODE, ROWS>(a, v, t % strips, t / strips, cur);
        for (; t < tiles; t += W) {
            Tile2<T, MODE, ROWS> nxt;
            const int tn = t + W;
            if (tn < tiles) tile_load<T, MODE, ROWS>(a, v, tn % strips, tn / strips, nxt);
            tile_compute<T, MODE, ROWS>(a, c, v, t % strips, t / strips, cur);
            cur = nxt;
        }
    } else {
        auto split = [&](int tt, int* b, int* strip, int* cy) {
            *b = tt / per_problem;
            const int r = tt - *b * per_problem;
            *strip = r % strips;
            *cy = r / strips;
        };
        int b, strip, cy;
        split(t, &b, &strip, &cy);
        Tile2<T, MODE, ROWS> cur;
        bool have = !problem_skipped(a, b);
        if (have) tile_load<T, MODE, ROWS>(a, problem_ptrs(a, b, MODE == M_RESID_RESTRICT), strip, cy, cur);
        for (; t < tiles; t += W) {
            Tile2<T, MODE, ROWS> nxt;
            const int tn = t + W;
            int bn = 0, sn = 0, cn = 0;
            bool next = false;
            if (tn < tiles) {
                split(tn, &bn, &sn, &cn);
                next = !problem_skipped(a, bn);
                if (next) tile_load<T, MODE, ROWS>(a, problem_ptrs(a, bn, MODE == M_RESID_RESTRICT), sn, cn, nxt);
            }
            if (have) tile_compute<T, MODE, ROWS>(a, a.pc[b], problem_ptrs(a, b, MODE == M_RESID_RESTRICT), strip, cy, cur);
            cur = nxt;
            have = next;
            b = bn;
            strip = sn;
            cy = cn;
        }
    }
}

// Interior stencil weights of op by neighbour class and omega / (interior diagonal of opd),
// in double precision.  Q1 on a uniform grid: 2D stiffness 8/3, -1/3, -1/3 and mass
// h^2 (16, 4, 1)/36 for the centre, edge and diagonal neighbours; 3D stiffness
// h (8/3, 0, -1/6, -1/12) and mass h^3 (8/27, 2/27, 1/54, 1/216) for the centre, face,
// edge and corner neighbours.
template <typename T>
void interior_weights(PCoef<T>& c, const GridDesc& g, double omega) {
    const double h = g.h;
    double kw[4], mw[4];
    if (g.dim == 2) {
        const double k2[4] = {8.0 / 3.0, -1.0 / 3.0, -1.0 / 3.0, 0.0};
        const double m2[4] = {16.0 / 36.0, 4.0 / 36.0, 1.0 / 36.0, 0.0};
        for (int q = 0; q < 4; ++q) {
            kw[q] = k2[q];
            mw[q] = m2[q] * h * h;
        }
    } else {
        const double k3[4] = {8.0 / 3.0, 0.0, -1.0 / 6.0, -1.0 / 12.0};
        const double m3[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
        for (int q = 0; q < 4; ++q) {
            kw[q] = k3[q] * h;
            mw[q] = m3[q] * h * h * h;
        }
    }
    auto weight = [](const OpCoef<T>& o, double A, double M, double F) {
        return cx<T>(T(double(o.cK) * A + double(o.cM.re) * M + double(o.cG.re) * F),
                     T(double(o.cM.im) * M + double(o.cG.im) * F));
    };
    auto winv = [&](const OpCoef<T>& o, double A, double M, double F) {
        const double dr = double(o.cK) * A + double(o.cM.re) * M + double(o.cG.re) * F;
        const double di = double(o.cM.im) * M + double(o.cG.im) * F;
        const double d2 = dr * dr + di * di;
        return d2 > 0 ? cx<T>(T(omega * dr / d2), T(-omega * di / d2)) : cx<T>(T(0), T(0));
    };
    for (int q = 0; q < 4; ++q) c.iw[q] = weight(c.op, kw[q], mw[q], 0.0);
    c.wdinv = winv(c.opd, kw[0], mw[0], 0.0);
    for (int q = 0; q < 8; ++q) {
        for (int u = 0; u < 4; ++u) c.bw[q][u] = cx<T>(T(0), T(0));
        c.bdinv[q] = cx<T>(T(0), T(0));
    }
    if (g.dim != 2) return;
    // 2D side nodes.  1D rows (Q1): stiffness (1/h)(-1, cnt, -1), mass (h/6)(1, 2 cnt, 1) with
    // cnt = 2 inside, 1 at the ends; a node on a side also carries the 1D boundary mass of
    // that side (centre: the along-side mass row's centre, neighbours along the side h/6).
    const double ks = -1.0 / h, ms = h / 6.0;
    for (int ty = 0; ty < 3; ++ty)
        for (int tx = 0; tx < 3; ++tx) {
            if (tx == 1 && ty == 1) continue;
            const int cl = ty * 3 + tx, q = cl - (cl > 4);
            const double cnx = tx == 1 ? 2.0 : 1.0, cny = ty == 1 ? 2.0 : 1.0;
            const double kcx = cnx / h, kcy = cny / h, mcx = cnx * h / 3.0, mcy = cny * h / 3.0;
            const bool fx = tx != 1, fy = ty != 1;  // on an x-side / a y-side
            const double A[4] = {kcx * mcy + mcx * kcy, ks * mcy + ms * kcy, kcx * ms + mcx * ks, 2.0 * ks * ms};
            const double M[4] = {mcx * mcy, ms * mcy, mcx * ms, ms * ms};
            const double F[4] = {(fx ? mcy : 0.0) + (fy ? mcx : 0.0), fy ? ms : 0.0, fx ? ms : 0.0, 0.0};
            for (int u = 0; u < 4; ++u) c.bw[q][u] = weight(c.op, A[u], M[u], F[u]);
            c.bdinv[q] = winv(c.opd, A[0], M[0], F[0]);
        }
}

template void interior_weights<float>(PCoef<float>&, const GridDesc&, double);
template void interior_weights<double>(PCoef<double>&, const GridDesc&, double);

template <typename T, int MODE, int ROWS, bool BATCH>
static cudaError_t run2b(const MArgs<T>& a, int strips, int chunks, cudaStream_t s) {
    const long long tiles = (long long)strips * chunks * a.nb;
    // prolongation tiles run one tile per warp; residual-restriction tiles (more rows) only
    // when tuned to the persistent form
    if constexpr (MODE != M_PROLONG_JACOBI) {
        static int per_sm = 0;
        if (!per_sm) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_march2p<T, MODE, ROWS, BATCH>, 128, 0) !=
                    cudaSuccess ||
                per_sm < 1) {
                cudaGetLastError();
                per_sm = 1;
            }
        }
        const long long resident_blocks = (long long)num_sms() * per_sm;
        // automatic: persistent once there are several tiles per resident warp
        const bool persist =
            a.tile_form == 2 || (a.tile_form == 0 && MODE != M_RESID_RESTRICT && tiles >= 16 * resident_blocks);
        if (persist && tiles < (1LL << 31)) {
            const long long blocks = std::min(resident_blocks, (tiles + 3) / 4);
            return klaunch(k_march2p<T, MODE, ROWS, BATCH>, dim3((unsigned)blocks), dim3(128), 0, s, 1, a, strips,
                           strips * chunks, (int)tiles);
        }
    }
    dim3 grd((unsigned)strips, (unsigned)((chunks + 3) / 4), (unsigned)a.nb);
    return klaunch(k_march2<T, MODE, ROWS, BATCH>, grd, dim3(128), 0, s, 1, a, chunks);
}

template <typename T, int MODE, int ROWS>
static cudaError_t run2(const MArgs<T>& a, int strips, int chunks, cudaStream_t s) {
    if (a.pc) return run2b<T, MODE, ROWS, true>(a, strips, chunks, s);
    if (a.nb != 1) return cudaErrorInvalidValue;
    return run2b<T, MODE, ROWS, false>(a, strips, chunks, s);
}

// Rows per warp tile: the largest that still leaves about 24 warps per SM (loads in flight),
// 8-row persistent tiles on large grids.
template <typename T, int MODE>
static cudaError_t go2(MArgs<T> a, cudaStream_t s) {
    a.h = T(a.g.h);
    a.ih = T(1.0 / a.g.h);
    const long long want = 24LL * num_sms();
    if constexpr (MODE == M_RESID_RESTRICT) {
        const int nnc = a.g.n / 2 + 1;
        const int strips = (nnc + 13) / 14;
        int rows = ((long long)strips * ((nnc + 3) / 4) * a.nb >= want) ? 4 : 2;
        if (a.tile_rows == 2 || a.tile_rows == 4) rows = a.tile_rows;
        if (rows == 4) return run2<T, MODE, 4>(a, strips, (nnc + 3) / 4, s);
        return run2<T, MODE, 2>(a, strips, (nnc + 1) / 2, s);
    } else {
        const int strips = (a.g.nn + 29) / 30;
        int rows = 2;
        if ((long long)strips * ((a.g.nn + 3) / 4) * a.nb >= want) rows = 4;
        // large grids run persistent 8-row tiles (measured best on 4097^2)
        if (sizeof(T) == 4 && MODE != M_PROLONG_JACOBI && (long long)strips * ((a.g.nn + 7) / 8) * a.nb >= 16 * want)
            rows = 8;
        if (a.tile_rows == 2 || a.tile_rows == 4 || (a.tile_rows == 8 && sizeof(T) == 4)) rows = a.tile_rows;
        if constexpr (sizeof(T) == 4) {
            if (rows == 8) return run2<T, MODE, 8>(a, strips, (a.g.nn + 7) / 8, s);
        }
        if (rows == 4) return run2<T, MODE, 4>(a, strips, (a.g.nn + 3) / 4, s);
        return run2<T, MODE, 2>(a, strips, (a.g.nn + 1) / 2, s);
    }
}

template <typename T>
cudaError_t launch_march2(int mode, const MArgs<T>& a, cudaStream_t s) {
    if (a.g.dim != 2) return cudaErrorInvalidValue;
    switch (mode) {
        case M_APPLY: return go2<T, M_APPLY>(a, s);
        case M_AXPBY: return go2<T, M_AXPBY>(a, s);
        case M_DAXPBY: return go2<T, M_DAXPBY>(a, s);
        case M_JACOBI: return go2<T, M_JACOBI>(a, s);
        case M_HSS_FIRST: return go2<T, M_HSS_FIRST>(a, s);
        case M_JACOBI2_ZERO: return go2<T, M_JACOBI2_ZERO>(a, s);
        case M_PROLONG_JACOBI: return go2<T, M_PROLONG_JACOBI>(a, s);
        case M_RESID_RESTRICT: return go2<T, M_RESID_RESTRICT>(a, s);
        case M_PROLONG_JACOBI2: return gof<T, M_PROLONG_JACOBI2>(a, s);
        case M_HSS_FIRST2: return gof<T, M_HSS_FIRST2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_march2<float>(int, const MArgs<float>&, cudaStream_t);
template cudaError_t launch_march2<double>(int, const MArgs<double>&, cudaStream_t);

}  // namespace hh
