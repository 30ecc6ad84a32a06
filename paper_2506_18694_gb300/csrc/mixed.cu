// Kernels of the mixed formulation (Sec. 2) and of its shifted-HSS preconditioner after the
// elimination of sigma (Def. 4.2).  sigma lives in the broken space V_h whose component a is,
// on each cell, multilinear in the coordinates other than a and constant along a; its basis
// on a cell is the tensor products of the 1D hat functions of the other axes, so that
//   M_sigma (cell block, component a)[s][t] = h prod_{b != a} m(s_b, t_b),
//   G[(cell, a, s)][node A of the cell]   = sign(A_a) prod_{b != a} m(s_b, A_b),
// with the 1D hat mass m(p, q) = h/3 (p = q) or h/6, sign(A_a) = +1 on the cell's far side of
// axis a and -1 on its near side, and D u (the gradient of u in V_h, G = M_sigma D) taking the
// differences (u_far - u_near) / h along a.  M_sigma^{-1} is the tensor product of the 1D
// inverses (4/h, -2/h) over the other axes, divided by h.  sigma DoFs are numbered
// ((cell * dim + a) * 2^(dim-1) + s), cells x fastest, s the bits of the other axes in order.
#include "internal.h"

namespace hh {

namespace {

template <typename T>
__device__ __forceinline__ T m1(int p, int q, T h) {
    return p == q ? h / T(3) : h / T(6);
}
template <typename T>
__device__ __forceinline__ T m1inv(int p, int q, T ih) {
    return p == q ? T(4) * ih : T(-2) * ih;
}

__device__ __forceinline__ bool dir_node(const GridDesc& g, int i, int j, int l) {
    const int n = g.n;
    if ((i == 0 && g.dir[0]) || (i == n && g.dir[1]) || (j == 0 && g.dir[2]) || (j == n && g.dir[3])) return true;
    return g.dim == 3 && ((l == 0 && g.dir[4]) || (l == n && g.dir[5]));
}

// u at a node, zero at Dirichlet nodes (their unknowns are eliminated)
template <typename T>
__device__ __forceinline__ Cx<T> u_at(const GridDesc& g, const vec2<T>* u, int i, int j, int l) {
    if (!u || dir_node(g, i, j, l)) return cx<T>(0, 0);
    return ld<T>(u, ((long long)l * g.nn + j) * g.nn + i);
}

// one thread per (cell, component) (grid-stride)
template <typename T, int DIM>
__global__ void k_mix_sigma(MixArgs<T> a) {
    pdl_entry();
    constexpr int NS = 1 << (DIM - 1);
    const GridDesc& g = a.g;
    const int n = g.n;
    const long long ncells = (long long)n * n * (DIM == 3 ? n : 1);
    const long long total = ncells * DIM;
    const T h = T(g.h), ih = T(1) / T(g.h);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long c = q / DIM;
        const int ax = (int)(q - c * DIM);
        const int ci = (int)(c % n), cj = (int)((c / n) % n), ck = DIM == 3 ? (int)(c / ((long long)n * n)) : 0;
        int oth[2] = {0, 0};
        {
            int k = 0;
            for (int b = 0; b < DIM; ++b)
                if (b != ax) oth[k++] = b;
        }
        const long long base = q * NS;
        Cx<T> v[NS], z[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            // vertex of the other axes' bits s, near (0) and far (1) along ax
            int vn[3] = {ci, cj, ck};
            for (int k = 0; k < DIM - 1; ++k) vn[oth[k]] += (s >> k) & 1;
            Cx<T> du = cx<T>(0, 0);
            if (a.u) {
                int vf[3] = {vn[0], vn[1], vn[2]};
                vf[ax] += 1;
                const Cx<T> uf = u_at<T>(g, a.u, vf[0], vf[1], vf[2]);
                const Cx<T> un = u_at<T>(g, a.u, vn[0], vn[1], vn[2]);
                du = cx<T>((uf.re - un.re) * ih, (uf.im - un.im) * ih);
            }
            const Cx<T> sg = a.sig ? ld<T>(a.sig, base + s) : cx<T>(0, 0);
            v[s] = fma_c(a.cs, sg, cmul(a.cd, du));
            z[s] = a.z ? ld<T>(a.z, base + s) : cx<T>(0, 0);
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            Cx<T> acc = cx<T>(0, 0);
            Cx<T> zz = cx<T>(0, 0);
#pragma unroll
            for (int t = 0; t < NS; ++t) {
                T w = T(1), wi = T(1);
                for (int k = 0; k < DIM - 1; ++k) {
                    const int sb = (s >> k) & 1, tb = (t >> k) & 1;
                    w *= m1<T>(sb, tb, h);
                    wi *= m1inv<T>(sb, tb, ih);
                }
                if (a.mass_out) {
                    acc = fma_r(h * w, v[t], acc);
                } else {
                    zz = fma_r(ih * wi, z[t], zz);
                }
            }
            const Cx<T> out = a.mass_out ? fma_c(a.cz, z[s], acc) : fma_c(a.cz, zz, v[s]);
            st<T>(a.y, base + s, out);
        }
    }
}

// one thread per node: y += G^T (d1 sig1 + d2 sig2) on the free nodes
template <typename T, int DIM>
__global__ void k_mix_div(MixArgs<T> a) {
    pdl_entry();
    constexpr int NS = 1 << (DIM - 1);
    const GridDesc& g = a.g;
    const int n = g.n, nn = g.nn;
    const long long N = (long long)nn * nn * (DIM == 3 ? nn : 1);
    const T h = T(g.h);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % nn), j = (int)((p / nn) % nn), l = DIM == 3 ? (int)(p / ((long long)nn * nn)) : 0;
        if (dir_node(g, i, j, l)) continue;
        Cx<T> acc = cx<T>(0, 0);
        for (int A = 0; A < (1 << DIM); ++A) {
            const int Ab[3] = {A & 1, (A >> 1) & 1, (A >> 2) & 1};
            const int cx_ = i - Ab[0], cy_ = j - Ab[1], cz_ = DIM == 3 ? l - Ab[2] : 0;
            if (cx_ < 0 || cx_ >= n || cy_ < 0 || cy_ >= n || (DIM == 3 && (cz_ < 0 || cz_ >= n))) continue;
            const long long c = ((long long)cz_ * n + cy_) * n + cx_;
            for (int ax = 0; ax < DIM; ++ax) {
                int oth[2] = {0, 0};
                int k = 0;
                for (int b = 0; b < DIM; ++b)
                    if (b != ax) oth[k++] = b;
                const long long base = (c * DIM + ax) * NS;
                const T sgn = Ab[ax] ? T(1) : T(-1);
                for (int s = 0; s < NS; ++s) {
                    T w = sgn;
                    for (int kk = 0; kk < DIM - 1; ++kk) w *= m1<T>((s >> kk) & 1, Ab[oth[kk]], h);
                    Cx<T> sv = cmul(a.cs, ld<T>(a.sig, base + s));
                    if (a.sig2) sv = fma_c(a.cd, ld<T>(a.sig2, base + s), sv);
                    acc = fma_r(w, sv, acc);
                }
            }
        }
        st<T>(a.y, p, ld<T>(a.y, p) + acc);
    }
}

int mix_blocks(long long work) {
    const long long b = (work + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

}  // namespace

template <typename T>
cudaError_t launch_mix_sigma(const MixArgs<T>& a, cudaStream_t s) {
    const int dim = a.g.dim;
    const long long work = (long long)a.g.n * a.g.n * (dim == 3 ? a.g.n : 1) * dim;
    if (!a.y || (dim != 2 && dim != 3)) return cudaErrorInvalidValue;
    if (dim == 2) return klaunch(k_mix_sigma<T, 2>, dim3(mix_blocks(work)), dim3(256), 0, s, 1, a);
    return klaunch(k_mix_sigma<T, 3>, dim3(mix_blocks(work)), dim3(256), 0, s, 1, a);
}

template <typename T>
cudaError_t launch_mix_div(const MixArgs<T>& a, cudaStream_t s) {
    const int dim = a.g.dim;
    if (!a.y || !a.sig || (dim != 2 && dim != 3)) return cudaErrorInvalidValue;
    const long long work = a.g.N;
    if (dim == 2) return klaunch(k_mix_div<T, 2>, dim3(mix_blocks(work)), dim3(256), 0, s, 1, a);
    return klaunch(k_mix_div<T, 3>, dim3(mix_blocks(work)), dim3(256), 0, s, 1, a);
}

template cudaError_t launch_mix_sigma<float>(const MixArgs<float>&, cudaStream_t);
template cudaError_t launch_mix_sigma<double>(const MixArgs<double>&, cudaStream_t);
template cudaError_t launch_mix_div<float>(const MixArgs<float>&, cudaStream_t);
template cudaError_t launch_mix_div<double>(const MixArgs<double>&, cudaStream_t);

}  // namespace hh
