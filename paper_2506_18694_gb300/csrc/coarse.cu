// Bottom of the V-cycle in one launch: the coarsest levels (a few thousand to a few
// tens of thousands of nodes) run inside a single thread-block cluster.  Every phase
// (a Jacobi sweep, a residual, a restriction, a prolongation) is spread over all the
// cluster's CTAs and closed by a cluster barrier, whose release/acquire semantics make
// the phase's global (L2-resident) writes visible to every CTA of the cluster.  This
// replaces one grid-wide launch per phase, which on grids this small costs more than
// the phase itself.
#include <cooperative_groups.h>

#include "internal.h"
#include "node.cuh"

namespace cg = cooperative_groups;

namespace hh {

template <typename T>
struct NodeCtx {
    int i, j, l;
    Row1<T> rx, ry, rz;
    bool masked;
};

template <typename T>
__device__ __forceinline__ NodeCtx<T> node_ctx(const GridDesc& g, long long pl) {
    NodeCtx<T> c;
    const T h = T(g.h), ih = T(1.0 / g.h);
    // levels handled here hold far fewer than 2^31 nodes: 32-bit index arithmetic
    const unsigned p = (unsigned)pl, nn = (unsigned)g.nn;
    const unsigned q = p / nn;
    c.i = (int)(p - q * nn);
    c.j = (int)(q % nn);
    c.l = g.dim == 3 ? (int)(q / nn) : 0;
    c.rx = row1<T>(c.i, g.n, g.dir[0], g.dir[1], h, ih);
    c.ry = row1<T>(c.j, g.n, g.dir[2], g.dir[3], h, ih);
    c.masked = c.rx.masked || c.ry.masked;
    if (g.dim == 3) {
        c.rz = row1<T>(c.l, g.n, g.dir[4], g.dir[5], h, ih);
        c.masked = c.masked || c.rz.masked;
    } else {
        c.rz = c.rx;
    }
    return c;
}

template <typename T, bool NEED>
__device__ __forceinline__ NodeResult<T> eval(const GridDesc& g, const NodeCtx<T>& c, const vec2<T>* x,
                                              const OpCoef<T>& op) {
    return g.dim == 3 ? node3<T, NEED>(x, g.nn, c.i, c.j, c.l, c.rx, c.ry, c.rz, op)
                      : node2<T, NEED>(x, g.nn, c.i, c.j, c.rx, c.ry, op);
}

// xout = xin + omega D^{-1} (b - A xin)   (xin == nullptr: xin = 0)
template <typename T>
__device__ void ph_sweep(const GridDesc& g, const OpCoef<T>& op, T omega, const vec2<T>* b, const vec2<T>* xin,
                         vec2<T>* xout, long long tid, long long nthr) {
    for (long long p = tid; p < g.N; p += nthr) {
        const NodeCtx<T> c = node_ctx<T>(g, p);
        if (c.masked) {
            st<T>(xout, p, cx<T>(0, 0));
            continue;
        }
        if (xin) {
            const NodeResult<T> r = eval<T, true>(g, c, xin, op);
            st<T>(xout, p, fma_c(cinv(r.d), omega * (ld<T>(b, p) - r.ax), ld<T>(xin, p)));
        } else {
            const NodeResult<T> r = eval<T, false>(g, c, nullptr, op);
            st<T>(xout, p, omega * cmul(cinv(r.d), ld<T>(b, p)));
        }
    }
}

template <typename T>
__device__ void ph_residual(const GridDesc& g, const OpCoef<T>& op, const vec2<T>* b, const vec2<T>* x,
                            vec2<T>* r, long long tid, long long nthr) {
    for (long long p = tid; p < g.N; p += nthr) {
        const NodeCtx<T> c = node_ctx<T>(g, p);
        if (c.masked) {
            st<T>(r, p, cx<T>(0, 0));
            continue;
        }
        st<T>(r, p, ld<T>(b, p) - eval<T, true>(g, c, x, op).ax);
    }
}

// bc = P^T r (full weighting) on the coarse grid gc
template <typename T>
__device__ void ph_restrict(const GridDesc& gc, const vec2<T>* r, vec2<T>* bc, long long tid, long long nthr) {
    const int nf = 2 * gc.n, nnf = nf + 1;
    const bool d3 = gc.dim == 3;
    for (long long p = tid; p < gc.N; p += nthr) {
        const NodeCtx<T> c = node_ctx<T>(gc, p);
        if (c.masked) {
            st<T>(bc, p, cx<T>(0, 0));
            continue;
        }
        Cx<T> acc = cx<T>(0, 0);
        for (int dz = d3 ? -1 : 0; dz <= (d3 ? 1 : 0); ++dz) {
            const int fl = 2 * c.l + dz;
            if (fl < 0 || fl > nf) continue;
            const T wz = dz == 0 ? T(1) : T(0.5);
            for (int dy = -1; dy <= 1; ++dy) {
                const int fj = 2 * c.j + dy;
                if (fj < 0 || fj > nf) continue;
                const T wy = dy == 0 ? wz : T(0.5) * wz;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int fi = 2 * c.i + dx;
                    if (fi < 0 || fi > nf) continue;
                    const T w = dx == 0 ? wy : T(0.5) * wy;
                    acc = fma_r(w, ld<T>(r, ((long long)(d3 ? fl : 0) * nnf + fj) * nnf + fi), acc);
                }
            }
        }
        st<T>(bc, p, acc);
    }
}

// x += P e (e on the coarse grid of gf)
template <typename T>
__device__ void ph_prolong(const GridDesc& gf, const vec2<T>* e, vec2<T>* x, long long tid, long long nthr) {
    const int nc = gf.n / 2, nnc = nc + 1;
    const bool d3 = gf.dim == 3;
    for (long long p = tid; p < gf.N; p += nthr) {
        const NodeCtx<T> c = node_ctx<T>(gf, p);
        if (c.masked) {
            st<T>(x, p, cx<T>(0, 0));
            continue;
        }
        const int I0 = c.i >> 1, J0 = c.j >> 1, L0 = c.l >> 1;
        const int ni = (c.i & 1) ? 2 : 1, nj = (c.j & 1) ? 2 : 1, nl = (d3 && (c.l & 1)) ? 2 : 1;
        const T w = ((c.i & 1) ? T(0.5) : T(1)) * ((c.j & 1) ? T(0.5) : T(1)) *
                    ((d3 && (c.l & 1)) ? T(0.5) : T(1));
        Cx<T> acc = cx<T>(0, 0);
        for (int dz = 0; dz < nl; ++dz) {
            const int L = L0 + dz;
            if (d3 && ((L == 0 && gf.dir[4]) || (L == nc && gf.dir[5]))) continue;
            for (int dy = 0; dy < nj; ++dy) {
                const int J = J0 + dy;
                if ((J == 0 && gf.dir[2]) || (J == nc && gf.dir[3])) continue;
                for (int dx = 0; dx < ni; ++dx) {
                    const int I = I0 + dx;
                    if ((I == 0 && gf.dir[0]) || (I == nc && gf.dir[1])) continue;
                    acc = fma_r(w, ld<T>(e, ((long long)(d3 ? L : 0) * nnc + J) * nnc + I), acc);
                }
            }
        }
        st<T>(x, p, ld<T>(x, p) + acc);
    }
}

template <typename T>
__global__ void __launch_bounds__(kClusterThreads) k_coarse_cluster(CoarseArgs<T> a) {
    pdl_entry();
    cg::cluster_group cl = cg::this_cluster();
    const long long nthr = (long long)blockDim.x * gridDim.x;  // the grid is one cluster
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    vec2<T>* cur[kMaxClusterLevels];
    // down: pre-smoothing, residual, restriction; the last level is smoothed from zero
    for (int lv = 0; lv < a.nlev; ++lv) {
        const GridDesc& g = a.g[lv];
        const bool coarsest = lv == a.nlev - 1;
        const int nsw = coarsest ? a.nu_coarse : a.nu_pre;
        vec2<T>* x = a.xa[lv];
        vec2<T>* o = a.xb[lv];
        if (nsw == 0) {
            for (long long p = tid; p < g.N; p += nthr) st<T>(x, p, cx<T>(0, 0));
            cl.sync();
        }
        for (int s = 0; s < nsw; ++s) {
            if (s == 0) {
                ph_sweep<T>(g, a.op, a.omega, a.b[lv], nullptr, x, tid, nthr);
            } else {
                ph_sweep<T>(g, a.op, a.omega, a.b[lv], x, o, tid, nthr);
                vec2<T>* t = x;
                x = o;
                o = t;
            }
            cl.sync();
        }
        cur[lv] = x;
        if (!coarsest) {
            ph_residual<T>(g, a.op, a.b[lv], x, a.t[lv], tid, nthr);
            cl.sync();
            ph_restrict<T>(a.g[lv + 1], a.t[lv], a.b[lv + 1], tid, nthr);
            cl.sync();
        }
    }
    // up: prolongation of the correction, post-smoothing
    for (int lv = a.nlev - 2; lv >= 0; --lv) {
        const GridDesc& g = a.g[lv];
        vec2<T>* x = cur[lv];
        vec2<T>* o = (x == a.xa[lv]) ? a.xb[lv] : a.xa[lv];
        ph_prolong<T>(g, cur[lv + 1], x, tid, nthr);
        cl.sync();
        for (int s = 0; s < a.nu_post; ++s) {
            ph_sweep<T>(g, a.op, a.omega, a.b[lv], x, o, tid, nthr);
            vec2<T>* t = x;
            x = o;
            o = t;
            cl.sync();
        }
        cur[lv] = x;
    }
    // the result of the top level always ends in xa[0]
    if (cur[0] != a.xa[0])
        for (long long p = tid; p < a.g[0].N; p += nthr) a.xa[0][p] = cur[0][p];
}

template <typename T>
int cluster_size_for() {
    static int cached = 0;
    if (cached) return cached;
    cudaFuncSetAttribute(k_coarse_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    for (int cs : {16, 8, 4, 2, 1}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs, 1, 1);
        cfg.blockDim = dim3(kClusterThreads, 1, 1);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_cluster<T>, &cfg) == cudaSuccess && nclusters > 0) {
            cached = cs;
            return cs;
        }
        cudaGetLastError();
    }
    cached = 1;
    return 1;
}

template <typename T>
cudaError_t launch_coarse_cluster(const CoarseArgs<T>& a, cudaStream_t s) {
    if (a.nlev < 1 || a.nlev > kMaxClusterLevels) return cudaErrorInvalidValue;
    const int cs = cluster_size_for<T>();
    return klaunch(k_coarse_cluster<T>, dim3(cs), dim3(kClusterThreads), 0, s, cs, a);
}

template int cluster_size_for<float>();
template int cluster_size_for<double>();
template cudaError_t launch_coarse_cluster<float>(const CoarseArgs<float>&, cudaStream_t);
template cudaError_t launch_coarse_cluster<double>(const CoarseArgs<double>&, cudaStream_t);

}  // namespace hh
