// Grid-transfer and elementwise kernels over a batch of problems: full-weighting
// restriction (3D and the building-block API), bi/trilinear prolongation, vector add and
// copy, precision casts, masked copies.  Problem b of a batch works at offset b * bs (its
// level vector) or b * bsc (its coarse vector); blockIdx.z (or y) selects the problem.
#include <atomic>

#include "internal.h"

namespace hh {

thread_local long long g_kernel_launches = 0;
thread_local int g_use_pdl = 1;

int num_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 1;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
        cudaGetLastError();
        v = 1;
    }
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

__device__ __forceinline__ bool batch_skipped(const Batch& bt, int b) {
    if (bt.active && !bt.active[b]) return true;
    return bt.hss_it >= 0 && bt.hss_it >= bt.nhss[b];
}

__device__ __forceinline__ bool node_masked(const GridDesc& g, int i, int j, int l) {
    bool m = (i == 0 && g.dir[0]) || (i == g.n && g.dir[1]) || (j == 0 && g.dir[2]) || (j == g.n && g.dir[3]);
    if (g.dim == 3) m = m || (l == 0 && g.dir[4]) || (l == g.n && g.dir[5]);
    return m;
}

// ---------------------------------------------------------------- restriction
// Full weighting R = P^T: coarse node I gathers fine nodes 2I + a, a in {-1,0,1}^dim,
// with weight prod (a == 0 ? 1 : 1/2) (the transpose of bi/trilinear interpolation).
// grid.z = planes x problems (3D) or problems (2D).
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(GridDesc gc, const vec2<T>* __restrict__ rf,
                                                  vec2<T>* __restrict__ rc, Batch bt) {
    pdl_entry();
    const bool d3 = gc.dim == 3;
    const int planes = d3 ? gc.nn : 1;
    const int b = blockIdx.z / planes;
    const int L = blockIdx.z - b * planes;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I > gc.n || J > gc.n || batch_skipped(bt, b)) return;
    const int nf = 2 * gc.n, nnf = nf + 1;
    rf += (long long)b * bt.bs;
    rc += (long long)b * bt.bsc;
    const long long p = d3 ? ((long long)L * gc.nn + J) * gc.nn + I : (long long)J * gc.nn + I;
    if (node_masked(gc, I, J, L)) {
        st<T>(rc, p, cx<T>(0, 0));
        return;
    }
    Cx<T> acc = cx<T>(0, 0);
    const int cmin = d3 ? -1 : 0, cmax = d3 ? 1 : 0;
    for (int c = cmin; c <= cmax; ++c) {
        const int fl = 2 * L + c;
        if (fl < 0 || fl > nf) continue;
        const T wc = c == 0 ? T(1) : T(0.5);
#pragma unroll
        for (int bb = -1; bb <= 1; ++bb) {
            const int fj = 2 * J + bb;
            if (fj < 0 || fj > nf) continue;
            const T wb = bb == 0 ? wc : T(0.5) * wc;
#pragma unroll
            for (int a = -1; a <= 1; ++a) {
                const int fi = 2 * I + a;
                if (fi < 0 || fi > nf) continue;
                const T w = a == 0 ? wb : T(0.5) * wb;
                const long long q = ((long long)(d3 ? fl : 0) * nnf + fj) * nnf + fi;
                acc = fma_r(w, ld<T>(rf, q), acc);
            }
        }
    }
    st<T>(rc, p, acc);
}

template <typename T>
cudaError_t launch_restrict(const GridDesc& gc, const vec2<T>* rf, vec2<T>* rc, const Batch& bt, cudaStream_t s) {
    dim3 blk(32, 8, 1);
    dim3 grd((gc.nn + 31) / 32, (gc.nn + 7) / 8, (gc.dim == 3 ? gc.nn : 1) * bt.nb);
    return klaunch(k_restrict<T>, grd, blk, 0, s, 1, gc, rf, rc, bt);
}

// ---------------------------------------------------------------- prolongation
// x_f += P e_c: fine node i takes coarse node i/2 (even i) or the mean of (i-1)/2 and
// (i+1)/2 (odd i) along each axis (bi/trilinear interpolation of the coarse Q1 field).
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(GridDesc gf, const vec2<T>* __restrict__ ec,
                                                 vec2<T>* __restrict__ x, Batch bt) {
    pdl_entry();
    const bool d3 = gf.dim == 3;
    const int planes = d3 ? gf.nn : 1;
    const int b = blockIdx.z / planes;
    const int l = blockIdx.z - b * planes;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > gf.n || j > gf.n || batch_skipped(bt, b)) return;
    x += (long long)b * bt.bs;
    ec += (long long)b * bt.bsc;
    const long long p = d3 ? ((long long)l * gf.nn + j) * gf.nn + i : (long long)j * gf.nn + i;
    if (node_masked(gf, i, j, l)) {
        st<T>(x, p, cx<T>(0, 0));
        return;
    }
    const int nc = gf.n / 2, nnc = nc + 1;
    const int I0 = i >> 1, J0 = j >> 1, L0 = l >> 1;
    const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nl = (d3 && (l & 1)) ? 2 : 1;
    const T wi = (i & 1) ? T(0.5) : T(1), wj = (j & 1) ? T(0.5) : T(1),
            wl = (d3 && (l & 1)) ? T(0.5) : T(1);
    // coarse Dirichlet nodes carry no basis function: their entries are never read
    auto coarse_dir = [&](int I, int lo, int hi) { return (I == 0 && lo) || (I == nc && hi); };
    Cx<T> e = cx<T>(0, 0);
    for (int c = 0; c < nl; ++c) {
        if (d3 && coarse_dir(L0 + c, gf.dir[4], gf.dir[5])) continue;
        for (int bb = 0; bb < nj; ++bb) {
            if (coarse_dir(J0 + bb, gf.dir[2], gf.dir[3])) continue;
            for (int a = 0; a < ni; ++a) {
                if (coarse_dir(I0 + a, gf.dir[0], gf.dir[1])) continue;
                const long long q = ((long long)(d3 ? L0 + c : 0) * nnc + (J0 + bb)) * nnc + (I0 + a);
                e = fma_r(wi * wj * wl, ld<T>(ec, q), e);
            }
        }
    }
    st<T>(x, p, ld<T>(x, p) + e);
}

template <typename T>
cudaError_t launch_prolong(const GridDesc& gf, const vec2<T>* ec, vec2<T>* x, const Batch& bt, cudaStream_t s) {
    dim3 blk(32, 8, 1);
    dim3 grd((gf.nn + 31) / 32, (gf.nn + 7) / 8, (gf.dim == 3 ? gf.nn : 1) * bt.nb);
    return klaunch(k_prolong<T>, grd, blk, 0, s, 1, gf, ec, x, bt);
}

// ---------------------------------------------------------------- elementwise
static inline unsigned ew_blocks(long long N) {
    long long b = (N + 255) / 256;
    const long long cap = 16LL * num_sms();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// x_b += e_b (MODE 0), x_b = e_b (MODE 1) or x_b = 0 (MODE 2) over the first N entries of
// each problem's vector
template <typename T, int MODE>
__global__ void k_axpy1(vec2<T>* __restrict__ x, const vec2<T>* __restrict__ e, long long N, Batch bt) {
    pdl_entry();
    const int b = blockIdx.y;
    if (batch_skipped(bt, b)) return;
    x += (long long)b * bt.bs;
    e += (long long)b * bt.bs;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x)
        st<T>(x, p, MODE == 0 ? ld<T>(x, p) + ld<T>(e, p) : MODE == 1 ? ld<T>(e, p) : cx<T>(0, 0));
}

template <typename T>
cudaError_t launch_add(vec2<T>* x, const vec2<T>* e, long long N, const Batch& bt, cudaStream_t s) {
    return klaunch(k_axpy1<T, 0>, dim3(ew_blocks(N), bt.nb), dim3(256), 0, s, 1, x, e, N, bt);
}

template <typename T>
cudaError_t launch_copy(vec2<T>* x, const vec2<T>* e, long long N, const Batch& bt, cudaStream_t s) {
    return klaunch(k_axpy1<T, 1>, dim3(ew_blocks(N), bt.nb), dim3(256), 0, s, 1, x, e, N, bt);
}

// unlike a memset, leaves the vectors of skipped problems alone
template <typename T>
cudaError_t launch_zero(vec2<T>* x, long long N, const Batch& bt, cudaStream_t s) {
    return klaunch(k_axpy1<T, 2>, dim3(ew_blocks(N), bt.nb), dim3(256), 0, s, 1, x, (const vec2<T>*)x, N, bt);
}

__global__ void k_cast_d2f(const double2* __restrict__ a, float2* __restrict__ b, long long N) {
    pdl_entry();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        double2 v = a[p];
        b[p] = make_float2((float)v.x, (float)v.y);
    }
}

cudaError_t launch_cast_d2f(const double2* a, float2* b, long long N, cudaStream_t s) {
    return klaunch(k_cast_d2f, dim3(ew_blocks(N)), dim3(256), 0, s, 1, a, b, N);
}

// dst_b (complex128) = the vector that src[b] points to (problem b may end its HSS loop in a
// different buffer than its neighbours), for the active b < nb; N entries each.
template <typename T>
__global__ void k_gather_c128(const vec2<T>* const* __restrict__ src, double2* __restrict__ dst, long long N,
                              const int* __restrict__ active) {
    pdl_entry();
    const int b = blockIdx.y;
    if (active && !active[b]) return;
    const vec2<T>* s = src[b];
    dst += (long long)b * N;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const vec2<T> v = s[p];
        dst[p] = make_double2((double)v.x, (double)v.y);
    }
}

template <typename T>
cudaError_t launch_gather_c128(const vec2<T>* const* src, double2* dst, long long N, int nb, const int* active,
                               cudaStream_t s) {
    return klaunch(k_gather_c128<T>, dim3(ew_blocks(N), nb), dim3(256), 0, s, 1, src, dst, N, active);
}

// dst = src with exact zeros at the Dirichlet nodes; nb consecutive problems of g.N nodes
__global__ void k_mask_copy(GridDesc g, const double2* __restrict__ src, double2* __restrict__ dst, long long total) {
    pdl_entry();
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long p = q % g.N;
        const int i = (int)(p % g.nn);
        const int j = (int)((p / g.nn) % g.nn);
        const int l = g.dim == 3 ? (int)(p / ((long long)g.nn * g.nn)) : 0;
        dst[q] = node_masked(g, i, j, l) ? make_double2(0.0, 0.0) : src[q];
    }
}

cudaError_t launch_mask_copy(const GridDesc& g, const double2* src, double2* dst, int nb, cudaStream_t s) {
    const long long total = g.N * nb;
    return klaunch(k_mask_copy, dim3(ew_blocks(total)), dim3(256), 0, s, 1, g, src, dst, total);
}

#define HH_INSTANTIATE(T)                                                                                         \
    template cudaError_t launch_restrict<T>(const GridDesc&, const vec2<T>*, vec2<T>*, const Batch&, cudaStream_t); \
    template cudaError_t launch_prolong<T>(const GridDesc&, const vec2<T>*, vec2<T>*, const Batch&, cudaStream_t);  \
    template cudaError_t launch_add<T>(vec2<T>*, const vec2<T>*, long long, const Batch&, cudaStream_t);           \
    template cudaError_t launch_copy<T>(vec2<T>*, const vec2<T>*, long long, const Batch&, cudaStream_t);          \
    template cudaError_t launch_zero<T>(vec2<T>*, long long, const Batch&, cudaStream_t);                          \
    template cudaError_t launch_gather_c128<T>(const vec2<T>* const*, double2*, long long, int, const int*, cudaStream_t);

HH_INSTANTIATE(float)
HH_INSTANTIATE(double)

}  // namespace hh
