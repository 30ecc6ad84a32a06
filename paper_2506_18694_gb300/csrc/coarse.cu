// Coarsest multigrid level in one launch: all nu_coarse Jacobi sweeps from x = 0 run
// inside one thread-block cluster with the level held in distributed shared memory.
//
// The grid is cut into slabs along its slowest axis (rows in 2D, z-planes in 3D); CTA r
// of the cluster owns a contiguous run of slabs and keeps them, plus one halo slab on
// each side, in two shared-memory buffers (ping-pong) next to its slabs of b.  A sweep
// reads only the CTA's own shared memory; the CTA writes its first and last new slab
// straight into the halo slots of its two neighbours (remote shared-memory stores), and
// one cluster barrier (release/acquire at cluster scope) then makes every write of the
// sweep visible.  A launch per sweep would cost far more than a sweep of a few thousand
// nodes.
#include <cooperative_groups.h>

#include <algorithm>

#include "internal.h"
#include "march2_common.cuh"
#include "node.cuh"

namespace cg = cooperative_groups;

namespace hh {

struct SlabPlan {
    int per;        // slabs owned by each CTA (the last CTAs may own fewer or none)
    long long S;    // nodes per slab
    size_t smem;    // dynamic shared memory per CTA
    int depth;      // 2D: sweeps between two exchanges of halo rows
};

// Nodes one CTA can own: the 2D kernel keeps 4 per thread, the 3D kernel 2.
static long long cta_capacity(const GridDesc& g) {
    return (long long)(g.dim == 2 ? kCoarseNodesPerThread2 : kCoarseNodesPerThread) * kCoarseThreads;
}

// 2D: sweeps per exchange, at most kCoarseDepth2.  A CTA computes the first sweep of a group of
// d on its rows and d - 1 rows of each neighbour, the next on d - 2, ..., the last on its own
// rows, so it stages d halo rows per side, all from the adjacent CTA (per >= d).
constexpr int kCoarseDepth2 = 4;

template <typename T>
static SlabPlan slab_plan(const GridDesc& g, int cs) {
    SlabPlan sp;
    sp.per = (g.nn + cs - 1) / cs;
    sp.S = g.dim == 3 ? (long long)g.nn * g.nn : g.nn;
    sp.depth = 1;
    if (g.dim == 3) {
        // two iterate buffers with a halo slab on each side
        sp.smem = (size_t)(2 * (sp.per + 2)) * sp.S * sizeof(vec2<T>);
    } else {
        // three padded buffers (rows padded by a zero column on both sides) with `depth` halo
        // rows on each side; the deepest groups the slab's entries and shared memory allow
        auto smem2 = [&](int d) { return (size_t)(3 * (sp.per + 2 * d)) * (sp.S + 2) * sizeof(vec2<T>); };
        int d = std::min(kCoarseDepth2, sp.per);
        while (d > 1 && ((sp.per + 2LL * (d - 1)) * sp.S > cta_capacity(g) || smem2(d) > kCoarseSmemMax)) --d;
        sp.depth = std::max(d, 1);
        sp.smem = smem2(sp.depth);
    }
    return sp;
}

// One cluster per problem of the batch: problem = blockIdx.x / cluster size.  Coefficients
// from the table entry of A_L on this level (interior weights and omega D^{-1} included).
template <typename T>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse_dsmem(const __grid_constant__ MArgs<T> a, int nsweeps,
                                                                 int per) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int prob = blockIdx.x / (int)cl.num_blocks();
    if (problem_skipped(a, prob)) return;  // uniform over the cluster: no barrier is left waiting
    const GridDesc& g = a.g;
    const PCoef<T>& pcf = coef_of(a, prob);
    const OpCoef<T> op = pcf.op;
    const vec2<T>* __restrict__ b = a.z + (long long)prob * a.bs;
    vec2<T>* __restrict__ xout = a.y + (long long)prob * a.bs;
    const T omega = a.omega;
    const int nn = g.nn, n = g.n;
    const bool d3 = g.dim == 3;
    const long long S = d3 ? (long long)nn * nn : nn;
    const int r0 = min(rank * per, nn);
    const int r1 = min(r0 + per, nn);
    const int own = (r1 - r0) * (int)S;               // owned nodes (at most kCoarseNodesPerThread per thread)
    const long long buf = (long long)(per + 2) * S;   // one iterate buffer, halos included
    vec2<T>* xs[2] = {reinterpret_cast<vec2<T>*>(smem_raw), reinterpret_cast<vec2<T>*>(smem_raw) + buf};
    const T h = T(g.h), ih = T(1.0 / g.h);
    const long long off = (long long)(r0 - 1) * S;    // global node number of local index 0

    // per owned node, once: coordinates, class, b and omega D^{-1}
    constexpr int K = kCoarseNodesPerThread;
    int ii[K], jj[K], ll[K];
    unsigned char cls[K];  // 0 masked, 1 interior (fast), 2 boundary (general)
    Cx<T> bq[K], dw[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int q = threadIdx.x + k * blockDim.x;
        cls[k] = 0;
        ii[k] = jj[k] = ll[k] = 0;
        bq[k] = dw[k] = cx<T>(0, 0);
        if (q >= own) continue;
        const unsigned pu = (unsigned)((long long)r0 * S + q), nnu = (unsigned)nn, qq = pu / nnu;
        ii[k] = (int)(pu - qq * nnu);
        jj[k] = (int)(qq % nnu);
        ll[k] = d3 ? (int)(qq / nnu) : 0;
        const Row1<T> rx = row1<T>(ii[k], n, g.dir[0], g.dir[1], h, ih);
        const Row1<T> ry = row1<T>(jj[k], n, g.dir[2], g.dir[3], h, ih);
        Row1<T> rz = rx;
        bool masked = rx.masked || ry.masked;
        if (d3) {
            rz = row1<T>(ll[k], n, g.dir[4], g.dir[5], h, ih);
            masked = masked || rz.masked;
        }
        if (masked) continue;
        const bool fast = ii[k] >= 2 && ii[k] <= n - 2 && jj[k] >= 2 && jj[k] <= n - 2 &&
                          (!d3 || (ll[k] >= 2 && ll[k] <= n - 2));
        cls[k] = fast ? 1 : 2;
        bq[k] = ld<T>(b, (long long)r0 * S + q);
        if (fast) {
            dw[k] = pcf.wdinv;
        } else {
            const NodeResult<T> r = d3 ? node3<T, false>(xs[0], nn, ii[k], jj[k], ll[k], rx, ry, rz, op, off)
                                       : node2<T, false>(xs[0], nn, ii[k], jj[k], rx, ry, op, off);
            dw[k] = omega * cinv(r.d);
        }
    }
    int cur = 0;
    for (int s = 0; s < nsweeps; ++s) {
        const vec2<T>* __restrict__ xc = xs[cur];
        vec2<T>* xn = xs[cur ^ 1];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int q = threadIdx.x + k * blockDim.x;
            if (q >= own) continue;
            const long long lq = q + S;  // local index of the node
            Cx<T> xv = cx<T>(0, 0);
            if (cls[k] != 0) {
                if (s == 0) {
                    xv = cmul(dw[k], bq[k]);
                } else {
                    Cx<T> ax;
                    if (cls[k] == 1) {
                        if (!d3) {
                            const Cx<T> e = (ld<T>(xc, lq - 1) + ld<T>(xc, lq + 1)) +
                                            (ld<T>(xc, lq - nn) + ld<T>(xc, lq + nn));
                            const Cx<T> dg = (ld<T>(xc, lq - nn - 1) + ld<T>(xc, lq - nn + 1)) +
                                             (ld<T>(xc, lq + nn - 1) + ld<T>(xc, lq + nn + 1));
                            ax = fma_c(pcf.iw[2], dg, fma_c(pcf.iw[1], e, cmul(pcf.iw[0], ld<T>(xc, lq))));
                        } else {
                            // neighbours grouped by how many coordinates differ: 6 faces, 12 edges, 8 corners
                            Cx<T> fa = cx<T>(0, 0), ed = cx<T>(0, 0), co = cx<T>(0, 0);
#pragma unroll
                            for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
                                for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                                    for (int dx = -1; dx <= 1; ++dx) {
                                        const int m = (dx != 0) + (dy != 0) + (dz != 0);
                                        if (m == 0) continue;
                                        const Cx<T> v = ld<T>(xc, lq + ((long long)dz * nn + dy) * nn + dx);
                                        if (m == 1) fa = fa + v;
                                        else if (m == 2) ed = ed + v;
                                        else co = co + v;
                                    }
                            ax = fma_c(pcf.iw[3], co, fma_c(pcf.iw[2], ed, fma_c(pcf.iw[1], fa, cmul(pcf.iw[0], ld<T>(xc, lq)))));
                        }
                    } else {
                        const Row1<T> rx = row1<T>(ii[k], n, g.dir[0], g.dir[1], h, ih);
                        const Row1<T> ry = row1<T>(jj[k], n, g.dir[2], g.dir[3], h, ih);
                        if (d3) {
                            const Row1<T> rz = row1<T>(ll[k], n, g.dir[4], g.dir[5], h, ih);
                            ax = node3<T, true>(xc, nn, ii[k], jj[k], ll[k], rx, ry, rz, op, off).ax;
                        } else {
                            ax = node2<T, true>(xc, nn, ii[k], jj[k], rx, ry, op, off).ax;
                        }
                    }
                    xv = fma_c(dw[k], bq[k] - ax, ld<T>(xc, lq));
                }
            }
            st<T>(xn, lq, xv);
            // boundary slabs also go to the neighbours' halo slots of the same buffer
            if (q < S && rank > 0) st<T>(cl.map_shared_rank(xn, rank - 1), (long long)(per + 1) * S + q, xv);
            if (q >= own - S && r1 < nn) st<T>(cl.map_shared_rank(xn, rank + 1), q - (own - S), xv);
        }
        cl.sync();
        cur ^= 1;
    }
    for (int q = threadIdx.x; q < own; q += blockDim.x) xout[(long long)r0 * S + q] = xs[cur][q + S];
}

// ---- 2D: padded slabs, boundary classes, `depth` sweeps per cluster barrier ----
// The 2D form keeps each slab row with a zero column on both sides and `depth` halo rows above
// and below, so that every node reads its 8 neighbours unconditionally (Dirichlet nodes and
// nodes outside the grid stay 0).  Sweeps run in groups of up to `depth`: a CTA computes the
// first sweep of a group on its own rows and on depth - 1 rows of each neighbour (recomputed,
// so no exchange is needed in between), each further sweep on one row less per side, the last
// on its own rows, and only then writes its top and bottom `depth` rows into the neighbours'
// halo rows: one cluster barrier per group.  The first sweep (from x = 0) is pointwise.
// Inner nodes use the interior weights and side nodes the weights of their boundary class,
// exactly as the 2D stencil kernels do, so the result equals nsweeps separate sweeps bit for
// bit.  Slabs of one row (tiny grids) exchange after every sweep (depth 1).
template <typename T>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse_dsmem2(const __grid_constant__ MArgs<T> a, int nsweeps,
                                                                  int per, int depth) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int prob = blockIdx.x / (int)cl.num_blocks();
    if (problem_skipped(a, prob)) return;  // uniform over the cluster: no barrier is left waiting
    // the coefficients in shared memory: read there at every update, they need neither the
    // parameter space's nor global memory's latency, nor a reload after each remote store
    __shared__ PCoef<T> cs;
    {
        const PCoef<T>& src = coef_of(a, prob);
        const unsigned* w = reinterpret_cast<const unsigned*>(&src);
        unsigned* d = reinterpret_cast<unsigned*>(&cs);
        for (int q = threadIdx.x; q < (int)(sizeof(PCoef<T>) / sizeof(unsigned)); q += blockDim.x) d[q] = w[q];
    }
    const PCoef<T>& c = cs;
    const vec2<T>* __restrict__ b = a.z + (long long)prob * a.bs;
    vec2<T>* __restrict__ xout = a.y + (long long)prob * a.bs;
    const int nn = a.g.nn, n = a.g.n, W = nn + 2;
    const int r0 = min(rank * per, nn);
    const int r1 = min(r0 + per, nn);
    const int rows = r1 - r0;
    const int H = depth - 1;                // neighbour rows recomputed on each side
    const int buf = (per + 2 * depth) * W;  // one padded buffer: rows -depth .. per + depth - 1
    vec2<T>* const xs0 = reinterpret_cast<vec2<T>*>(smem_raw);
    auto xs = [&](int q) { return xs0 + q * buf; };  // buffer q of 3
    for (int q = threadIdx.x; q < 3 * buf; q += blockDim.x) st<T>(xs0, q, cx<T>(0, 0));

    // entries: the slab's rows and H rows of each neighbour (rl = -H .. rows + H - 1).  Per
    // entry: padded index, kind (-1 none, 8 inner, 0..7 boundary class), b, its distance from
    // the slab (0: an own node), and where its value goes in the neighbours' halo rows.
    constexpr int K = kCoarseNodesPerThread2;
    int pidx[K], kind[K], dist[K], hm[K], hp[K];
    Cx<T> bq[K];
    const int ents = (rows + 2 * H) * nn;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = threadIdx.x + k * blockDim.x;
        pidx[k] = 0;
        kind[k] = hm[k] = hp[k] = -1;
        dist[k] = depth;
        bq[k] = cx<T>(0, 0);
        if (e >= ents || rows <= 0) continue;
        const int rl = -H + e / nn, i = e % nn, j = r0 + rl;
        if (j < 0 || j >= nn) continue;
        const bool vd = (i == 0 && a.g.dir[0]) || (i == n && a.g.dir[1]) || (j == 0 && a.g.dir[2]) ||
                        (j == n && a.g.dir[3]);
        if (vd) continue;
        pidx[k] = (rl + depth) * W + (i + 1);
        const int tx = i == 0 ? 0 : (i == n ? 2 : 1), ty = j == 0 ? 0 : (j == n ? 2 : 1);
        const int cls = ty * 3 + tx;
        kind[k] = cls == 4 ? 8 : cls - (cls > 4);
        bq[k] = ld<T>(b, (long long)j * nn + i);
        dist[k] = rl < 0 ? -rl : (rl >= rows ? rl - rows + 1 : 0);
        if (dist[k] > 0) continue;
        // upper neighbour (per rows): our row rl < depth is its row per + rl
        if (rank > 0 && rl < depth) hm[k] = (per + rl + depth) * W + (i + 1);
        // lower neighbour: our row rl >= rows - depth is its row rl - rows
        if (r1 < nn && rl >= rows - depth) hp[k] = (rl - rows + depth) * W + (i + 1);
    }
    cl.sync();  // every CTA's buffers are zero before any halo row arrives
    int in = 0;  // buffer holding the current iterate (own rows and valid halo rows)
    int s = 0;
    while (s < nsweeps) {
        const int g = min(depth, nsweeps - s);  // sweeps in this group
        const int tmp = (in + 1) % 3, out = (in + 2) % 3;
        // sweep t reads src and writes dst on the entries within g - 1 - t rows of the slab:
        // in -> tmp -> in -> ... -> out, so the buffer the neighbours write into (out) holds
        // only the last sweep's own rows until their halo rows arrive
        int src = in;
        for (int t = 0; t < g; ++t) {
            const int dst = t == g - 1 ? out : ((t & 1) ? in : tmp);
            const int ext = g - 1 - t;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (kind[k] < 0 || dist[k] > ext) continue;
                const Cx<T> xv = s + t == 0 ? cmul(kind[k] == 8 ? c.wdinv : c.bdinv[kind[k]], bq[k])
                                            : coarse_update2(c, xs(src), pidx[k], W, kind[k], bq[k]);
                st<T>(xs(dst), pidx[k], xv);
            }
            src = dst;
            if (t + 1 < g) __syncthreads();
        }
        __syncthreads();
        // own boundary rows of the new iterate into the neighbours' halo rows
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (kind[k] < 0 || dist[k] > 0 || (hm[k] < 0 && hp[k] < 0)) continue;
            const Cx<T> xv = ld<T>(xs(out), pidx[k]);
            if (hm[k] >= 0) st<T>(cl.map_shared_rank(xs(out), rank - 1), hm[k], xv);
            if (hp[k] >= 0) st<T>(cl.map_shared_rank(xs(out), rank + 1), hp[k], xv);
        }
        cl.sync();
        in = out;
        s += g;
    }
    for (int q = threadIdx.x; q < rows * nn; q += blockDim.x) {
        const int rl = q / nn, i = q - rl * nn;
        xout[(long long)(r0 + rl) * nn + i] = xs(in)[(rl + depth) * W + (i + 1)];
    }
}

// ---- 2D: one CTA per band of rows, no communication between CTAs (coarse_band2) ----
// grid (bands, problems); R rows per band
template <typename T, bool BATCH>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse_band2(const __grid_constant__ MArgs<T> a, int nsweeps,
                                                                 int R) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = BATCH ? (int)blockIdx.y : 0;
    if (BATCH && problem_skipped(a, b)) return;
    const int r0 = blockIdx.x * R;
    if (r0 >= a.g.nn) return;
    coarse_band2<T>(a, coef_of(a, b), b, r0, min(r0 + R, a.g.nn), nsweeps, smem_raw);
}

// rows per band: enough bands to spread the level over many SMs, within the shared memory
template <typename T>
static int band_rows(const GridDesc& g, int nsweeps, int want) {
    int R = want > 0 ? want : std::max(1, (g.nn + 63) / 64);
    while (R > 1 && band2_smem<T>(g.nn, nsweeps, R) > kCoarseSmemMax) --R;
    return band2_smem<T>(g.nn, nsweeps, R) <= kCoarseSmemMax ? R : 0;
}

static int g_cluster_size = 0;

int coarse_cluster_size() {
    if (g_cluster_size) return g_cluster_size;
    cudaFuncSetAttribute(k_coarse_dsmem<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_coarse_dsmem<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_coarse_dsmem2<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_coarse_dsmem2<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(kCoarseThreads, 1, 1);
    cfg.dynamicSmemBytes = kCoarseSmemMax;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_dsmem<float>, &cfg) == cudaSuccess && nclusters >= 1) {
        g_cluster_size = cs;
        return cs;
    }
    cudaGetLastError();
    }
    g_cluster_size = 1;
    return 1;
}

template <typename T>
bool coarse_cluster_ok(const GridDesc& g, int cs) {
    if (cs < 1 || cs > coarse_cluster_size()) return false;
    const SlabPlan sp = slab_plan<T>(g, cs);
    // 2D CTAs also hold depth - 1 rows of each neighbour
    const long long rows = g.dim == 2 ? sp.per + 2LL * (sp.depth - 1) : sp.per;
    return sp.smem <= kCoarseSmemMax && rows * sp.S <= cta_capacity(g);
}

template <typename T>
bool coarse_fits(const GridDesc& g) {
    return coarse_cluster_ok<T>(g, coarse_cluster_size());
}

template <typename T>
cudaError_t prepare_coarse() {
    cudaError_t e = cudaFuncSetAttribute(k_coarse_dsmem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kCoarseSmemMax);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_coarse_dsmem2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmemMax);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_coarse_band2<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kCoarseSmemMax);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_coarse_band2<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kCoarseSmemMax);
    if (e != cudaSuccess) return e;
    coarse_cluster_size();
    return cudaSuccess;
}

// Cluster size for nb problems: the largest (fastest for one problem) unless the batch's
// clusters would not all be resident at once; then halve it while the slabs still fit.
// Every size gives the same sweeps bit for bit (the slab cut only moves work between CTAs).
template <typename T>
static int batch_cluster_size(const GridDesc& g, int nb) {
    int cs = coarse_cluster_size();
    while (cs > 1 && (long long)nb * cs > 2LL * num_sms() && coarse_cluster_ok<T>(g, cs / 2)) cs /= 2;
    return cs;
}

template <typename T>
cudaError_t launch_coarse_solve(const MArgs<T>& a, int nsweeps, cudaStream_t s) {
    if (nsweeps < 1) return cudaErrorInvalidValue;
    // 2D bands of rows, one CTA each (tile_form 3, tile_rows rows per band or 0 for the default);
    // otherwise the cluster (a cluster size in tile_rows, 0 for the default).  Measured on the
    // 513^2, k = 80 workload: a V-cycle takes 41.5 us with the cluster and 45.4 us with bands.
    if (a.g.dim == 2 && a.tile_form == 3) {
        const int R = band_rows<T>(a.g, nsweeps, a.tile_form == 3 ? a.tile_rows : 0);
        if (R > 0) {
            const dim3 grd((unsigned)((a.g.nn + R - 1) / R), (unsigned)a.nb);
            const size_t smem = band2_smem<T>(a.g.nn, nsweeps, R);
            if (a.pc) return klaunch(k_coarse_band2<T, true>, grd, dim3(kCoarseThreads), smem, s, 1, a, nsweeps, R);
            if (a.nb != 1) return cudaErrorInvalidValue;
            return klaunch(k_coarse_band2<T, false>, grd, dim3(kCoarseThreads), smem, s, 1, a, nsweeps, R);
        }
    }
    // a tuned cluster size arrives in tile_rows
    const int cs = coarse_cluster_ok<T>(a.g, a.tile_rows) ? a.tile_rows : batch_cluster_size<T>(a.g, a.nb);
    if (!coarse_cluster_ok<T>(a.g, cs)) return cudaErrorInvalidValue;
    const SlabPlan sp = slab_plan<T>(a.g, cs);
    if (a.g.dim == 2)
        return klaunch(k_coarse_dsmem2<T>, dim3(cs * a.nb), dim3(kCoarseThreads), sp.smem, s, cs, a, nsweeps, sp.per,
                       sp.depth);
    return klaunch(k_coarse_dsmem<T>, dim3(cs * a.nb), dim3(kCoarseThreads), sp.smem, s, cs, a, nsweeps, sp.per);
}

template bool coarse_fits<float>(const GridDesc&);
template bool coarse_fits<double>(const GridDesc&);
template bool coarse_cluster_ok<float>(const GridDesc&, int);
template bool coarse_cluster_ok<double>(const GridDesc&, int);
template cudaError_t prepare_coarse<float>();
template cudaError_t prepare_coarse<double>();
template cudaError_t launch_coarse_solve<float>(const MArgs<float>&, int, cudaStream_t);
template cudaError_t launch_coarse_solve<double>(const MArgs<double>&, int, cudaStream_t);

}  // namespace hh
