// Launchers shared between the translation units of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace hh {

// Message returned by hh_last_error() for the calling thread.
void set_last_error(const char* msg);

// Streaming multiprocessors of the current device (queried once per device; the launch
// heuristics size persistent grids and occupancy targets by it).
int num_sms();

// Kernels launched by this thread through the launchers below (graph captures included).
extern thread_local long long g_kernel_launches;
// 1: launch with programmatic stream serialization (overlaps a kernel's launch with the
// tail of its predecessor; every kernel starts with pdl_entry()).
extern thread_local int g_use_pdl;

#define HH_KRET(call)                        \
    do {                                     \
        cudaError_t e_ = (call);             \
        if (e_ != cudaSuccess) return e_;    \
    } while (0)

// Launch `kernel` on stream s (optionally as clusters of `cluster` CTAs along x).
template <typename... KArgs, typename... Args>
inline cudaError_t klaunch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                           int cluster, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    int na = 0;
    if (g_use_pdl) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    if (cluster > 1) {
        at[na].id = cudaLaunchAttributeClusterDimension;
        at[na].val.clusterDim.x = cluster;
        at[na].val.clusterDim.y = 1;
        at[na].val.clusterDim.z = 1;
        ++na;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    ++g_kernel_launches;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Batch selection for the transfer and elementwise kernels: nb problems, problem b at offset
// b * bs in its level vector and b * bsc in its coarse vector; skipped like MArgs.
struct Batch {
    int nb;
    long long bs, bsc;
    int hss_it;
    const int* nhss;
    const int* active;
};

// rc = P^T rf (rf on the fine grid of gc), every problem of the batch
template <typename T>
cudaError_t launch_restrict(const GridDesc& gc, const vec2<T>* rf, vec2<T>* rc, const Batch& bt, cudaStream_t s);

// x += P ec (ec on the coarse grid of gf)
template <typename T>
cudaError_t launch_prolong(const GridDesc& gf, const vec2<T>* ec, vec2<T>* x, const Batch& bt, cudaStream_t s);

// x += e, x = e (first N entries of each problem's vector)
template <typename T>
cudaError_t launch_add(vec2<T>* x, const vec2<T>* e, long long N, const Batch& bt, cudaStream_t s);
template <typename T>
cudaError_t launch_copy(vec2<T>* x, const vec2<T>* e, long long N, const Batch& bt, cudaStream_t s);
template <typename T>
cudaError_t launch_zero(vec2<T>* x, long long N, const Batch& bt, cudaStream_t s);

cudaError_t launch_cast_d2f(const double2* a, float2* b, long long N, cudaStream_t s);
// dst (nb consecutive complex128 vectors of N) = *src[b] (device array of nb pointers)
template <typename T>
cudaError_t launch_gather_c128(const vec2<T>* const* src, double2* dst, long long N, int nb, const int* active,
                               cudaStream_t s);
// dst = src with exact zeros at the Dirichlet nodes of g (nb consecutive vectors)
cudaError_t launch_mask_copy(const GridDesc& g, const double2* src, double2* dst, int nb, cudaStream_t s);

// ---- fused 2D marching kernels (march2.cu) ----
enum MarchMode {
    M_APPLY = 0,          // y = op x
    M_AXPBY = 1,          // y = alpha (op x) + beta z
    M_JACOBI = 2,         // y = x + omega D^{-1} (z - op x),          D = diag(op)
    M_HSS_FIRST = 3,      // y = alpha (op x) + beta z;  y2 = omega diag(opd)^{-1} y
    M_JACOBI2_ZERO = 4,   // two sweeps from x = 0 reading only z:  x1 = omega D^{-1} z,
                          // y = x1 + omega D^{-1} (z - op x1)
    M_PROLONG_JACOBI = 5, // x~ = x + P ec;  y = x~ + omega D^{-1} (z - op x~)
    M_RESID_RESTRICT = 6, // y (coarse) = P^T (z - op x)
    // two sweeps in one pass (2D): the second sweep's operator is pc2 / c02 (A_L)
    M_PROLONG_JACOBI2 = 7,  // x~ = x + P ec;  x1 = x~ + omega D^{-1} (z - op x~);  y = x1 + omega D^{-1} (z - op x1)
    M_HSS_FIRST2 = 8,       // rhs = alpha (op x) + beta z;  x1 = omega D^{-1} rhs;  y = rhs,
                            // y2 = x1 + omega D^{-1} (rhs - A_L x1)
    // two pre-sweeps and the residual restriction in one pass (2D, march2rr.cu)
    M_JACOBI2_ZERO_RR = 9,  // y = two sweeps on A_L x = z from 0;  yc (coarse) = P^T (z - A_L y)
    M_HSS_FIRST2_RR = 10,   // as M_HSS_FIRST2 (y = rhs, y2 = x2), and yc = P^T (rhs - A_L x2)
    // (11 is the coarse solve's slot in the tuning table)
    M_DAXPBY = 12           // y = omega D^{-1} (alpha (op x) + beta z): the Jacobi-preconditioned
                            // residual and operator of the GMRES smoother (march2.cu, march3.cu)
};

// Coefficients of one operator on one level for one problem of a batch (a device table
// indexed by problem): the stencil operator, the operator whose diagonal scales the Jacobi
// update (A_L), the interior weights of op by neighbour class (how many coordinates differ
// from the centre: 0 centre, 1 edge/face, 2 diagonal/edge, 3 corner in 3D), omega / interior
// diag(opd), and two per-problem scalars (the HSS weights (k-1)/(k+1), 2k/(k+1)).
template <typename T> struct PCoef {
    OpCoef<T> op;
    OpCoef<T> opd;
    Cx<T> iw[4];
    Cx<T> wdinv;
    Cx<T> alpha, beta;
    // 2D nodes on a side of the square, by class (y type * 3 + x type, the interior class
    // 4 left out; type 0: first node of the axis, 1: inner, 2: last): weights of the centre,
    // the x-neighbours, the y-neighbours and the diagonal neighbours, and omega / diag(opd)
    Cx<T> bw[8][4];
    Cx<T> bdinv[8];
};

// Host: fill the interior and boundary-class weights of c for grid g and damping omega.
template <typename T>
void interior_weights(PCoef<T>& c, const GridDesc& g, double omega);

// 3D nodes on a face, edge or corner of the cube: 26 classes ((z type * 3 + y type) * 3 +
// x type, the inner class 13 left out), each with the weights of its 8 neighbour groups
// (centre; x, y, z faces; xy, xz, yz edges; corners) and omega / diag(opd) last.
constexpr int kClass3 = 26;
constexpr int kClass3Len = 9;
// Host: fill out[kClass3][kClass3Len] for the operators of c on grid g.
template <typename T>
void boundary_weights3(Cx<T>* out, const PCoef<T>& c, const GridDesc& g, double omega);

// Arguments of the stencil kernels.  Problem b of a batch of nb reads x, z, y, y2 at
// offset b * bs, ec (and writes the coarse output of RESID_RESTRICT) at offset b * bsc,
// and its coefficients at pc[b].
template <typename T> struct MArgs {
    GridDesc g;          // grid of the level the stencil runs on
    const PCoef<T>* pc;  // device coefficient table of this operator and level (nullptr: c0)
    PCoef<T> c0;         // the coefficients of a batch of one, passed by value
    const Cx<T>* bw3;    // 3D: device boundary-class weights, problem b at b * kClass3 * kClass3Len
    const PCoef<T>* pc2; // second operator of the fused two-sweep modes (nullptr: c02)
    PCoef<T> c02;
    vec2<T>* yc;         // coarse output of the *_RR modes (problem b at b * bsc)
    const vec2<T>* x;    // stencil input (ignored for M_JACOBI2_ZERO; nullptr = 0 when xzero)
    const vec2<T>* z;    // right side / second vector
    const vec2<T>* ec;   // coarse correction (M_PROLONG_JACOBI)
    vec2<T>* y;          // output
    vec2<T>* y2;         // second output (M_HSS_FIRST)
    long long bs, bsc;
    int nb;
    Cx<T> alpha, beta;   // AXPBY / HSS_FIRST scalars when use_pc_ab == 0
    int use_pc_ab;       // 1: alpha, beta of problem b from pc[b]
    T omega;
    int xzero;           // 1: x is identically zero
    int tile_rows;       // 0: automatic; else 2, 4 or 8 rows (2D) / planes (3D) per tile
    int tile_form;       // 2D: 0 automatic, 1 one tile per warp, 2 persistent warps walking the tiles
    int hss_it;          // >= 0: problem b is skipped when hss_it >= nhss[b]
    const int* nhss;     // device: HSS iterations of each problem
    const int* active;   // device: 0 = problem skipped (nullptr: all active)
    // filled by the launcher
    T h, ih;
    int rows;
};

// Vector pointers of problem b.
template <typename T> struct VPtrs {
    const vec2<T>* x;
    const vec2<T>* z;
    const vec2<T>* ec;
    vec2<T>* y;
    vec2<T>* y2;
};

template <typename T>
__device__ __forceinline__ VPtrs<T> problem_ptrs(const MArgs<T>& a, int b, bool coarse_out) {
    const long long o = (long long)b * a.bs, oc = (long long)b * a.bsc;
    VPtrs<T> v;
    v.x = a.x ? a.x + o : nullptr;
    v.z = a.z ? a.z + o : nullptr;
    v.ec = a.ec ? a.ec + oc : nullptr;
    v.y = a.y ? a.y + (coarse_out ? oc : o) : nullptr;
    v.y2 = a.y2 ? a.y2 + o : nullptr;
    return v;
}

// Coefficients of problem b (a reference into the table or into the kernel parameters:
// kernels taking it declare their MArgs __grid_constant__).
template <typename T>
__device__ __forceinline__ const PCoef<T>& coef_of(const MArgs<T>& a, int b) {
    return a.pc ? a.pc[b] : a.c0;
}

// Whether problem b takes part in a launch.
template <typename T>
__device__ __forceinline__ bool problem_skipped(const MArgs<T>& a, int b) {
    if (a.active && !a.active[b]) return true;
    return a.hss_it >= 0 && a.hss_it >= a.nhss[b];
}

template <typename T>
cudaError_t launch_march2(int mode, const MArgs<T>& a, cudaStream_t s);
// the pre-smoothing + residual-restriction passes (M_JACOBI2_ZERO_RR, M_HSS_FIRST2_RR)
template <typename T>
cudaError_t launch_march2rr(int mode, const MArgs<T>& a, cudaStream_t s);

// ---- fused 3D tile kernels (march3.cu): modes as above except M_RESID_RESTRICT ----
template <typename T>
cudaError_t launch_march3(int mode, const MArgs<T>& a, cudaStream_t s);

// ---- coarsest level inside one thread-block cluster per problem, in distributed shared
//      memory (coarse.cu) ----
constexpr int kCoarseThreads = 512;
constexpr int kCoarseNodesPerThread = 2;   // 3D kernel
constexpr int kCoarseNodesPerThread2 = 4;  // 2D kernel
constexpr size_t kCoarseSmemMax = 200 * 1024;

// CTAs per cluster (16 or 8 when the device can co-schedule them, else 1)
int coarse_cluster_size();
// whether a grid's slabs fit the shared memory of the cluster's CTAs
template <typename T>
bool coarse_fits(const GridDesc& g);
// whether clusters of cs CTAs can hold the grid (cs up to the device's cluster size)
template <typename T>
bool coarse_cluster_ok(const GridDesc& g, int cs);
// one-time set-up (shared-memory limit, cluster query); call before any stream capture
template <typename T>
cudaError_t prepare_coarse();
// a.nb problems: nsweeps scaled-Jacobi sweeps on op x = z from x = 0 into y (coefficients
// from a.pc), one cluster per problem; a.tile_rows, if a valid cluster size, picks it
template <typename T>
cudaError_t launch_coarse_solve(const MArgs<T>& a, int nsweeps, cudaStream_t s);


// ---- the whole 2D HSS loop in one cooperative launch (hssp.cu) ----
// Passes of one HSS step with one V(2,2) cycle on L levels (2 <= L <= kPMaxLevels): pre[0]
// the HSS right side, two sweeps and the restricted residual on level 0 (`first` is the same
// for the first step, with u = 0); pre[l], 1 <= l < L - 1, two sweeps from 0 and the
// restricted residual; `coarse` nu_coarse sweeps from 0 on level L - 1 (z: right side, y:
// result), `coarse_rows` rows per CTA band; post[l], l < L - 1, the prolongation of the coarse
// result and two sweeps.  Strips and chunks give each pass's warp tiles (as the separate
// kernels would launch them).  count: the grid barrier's arrival counter (zeroed by the
// launcher); status: 0, or an hh_status a CTA recorded (HH_ERR_TIMEOUT when a barrier wait
// ran past spin_limit polls); the host reads and clears it.
constexpr int kPMaxLevels = 5;
template <typename T> struct HssLoop2 {
    MArgs<T> first;
    MArgs<T> pre[kPMaxLevels];
    MArgs<T> post[kPMaxLevels];
    MArgs<T> coarse;
    int pre_strips[kPMaxLevels], pre_chunks[kPMaxLevels];
    int post_strips[kPMaxLevels], post_chunks[kPMaxLevels];
    int levels, nsteps, nb, nu_coarse, coarse_rows;
    unsigned* count;
    int* status;
    unsigned long long spin_limit;
};
// dynamic shared memory of the coarsest-level pass for coarse grid gc and bands of `rows` rows
// (at most kLoopSmemMax; the solver takes narrower bands until it fits, else one kernel per pass)
constexpr size_t kLoopSmemMax = 96 * 1024;
template <typename T>
size_t hss_loop2_smem(const GridDesc& gc, int nu_coarse, int rows);
// CTAs of the cooperative grid (resident at once; at most 4 per SM), 0 if none fit
template <typename T>
int hss_loop2_ctas(bool batch, size_t smem);
template <typename T>
cudaError_t launch_hss_loop2(const HssLoop2<T>& P, int ctas, size_t smem, cudaStream_t s);

// ---- packed passes over problems of different grids (pack.cu) ----
// One launch of pass `kind` for nm problems: 0 level-0 HSS right side + two sweeps + restriction,
// 1 two sweeps from 0 + restriction on `level`, 2 the coarsest level (bands; smem bytes of shared
// memory), 3 prolongation + two sweeps on `level`.  plans[m]: problem m's loop plan (nb = 1);
// starts: prefix of the problems' tiles (warp tiles; bands for kind 2), total = starts[nm].
template <typename T>
cudaError_t prepare_pack();
template <typename T>
cudaError_t launch_pack_pass(int kind, const HssLoop2<T>* plans, const int* starts, int nm, int total, int level,
                             int it, const int* live, size_t smem, cudaStream_t s);

// ---- GMRES smoother with a Jacobi preconditioner (gsmooth.cu) ----
// Level vectors of nb problems (problem b at offset b * N); the Krylov basis holds vector i
// of problem b at V + i * ld + b * N.  Sums in FP64 over a fixed block grid (gs_blocks(N)), so
// the results do not depend on launch history.  Problems skipped as in Batch.
constexpr int kGsMaxIts = 8;                // iterations per smoothing step at most
constexpr int kGsMaxVec = kGsMaxIts + 1;    // basis vectors
constexpr int kGsThreads = 256;
inline int gs_blocks(long long N) {
    const long long b = (N + 4 * kGsThreads - 1) / (4 * kGsThreads);
    return (int)(b < 1 ? 1 : (b > 304 ? 304 : b));
}
// part[(b * nblk + blk) * kGsMaxVec + i] = block blk's share of V_i^H w (i < nv)
template <typename T>
cudaError_t launch_gs_dot(const vec2<T>* V, long long ld, int nv, const vec2<T>* w, long long N, double2* part,
                          const Batch& bt, cudaStream_t s);
// A whole smoothing step of `its` iterations in one CTA per problem, for 2D levels of at most
// kGsCtaNodes nodes: x (in/out; xzero: from 0) on b, basis and work vector at V + i * ldv
// (i <= its + 1), the operator and batch from a (margs of R_AL).
constexpr long long kGsCtaNodes = 4225;
template <typename T>
cudaError_t launch_gs_cta(const MArgs<T>& a, const vec2<T>* b, vec2<T>* x, int xzero, int its, vec2<T>* V,
                          long long ldv, cudaStream_t s);
// Per-problem least-squares state (double2 entries, kGsState per problem): the Hessenberg
// matrix H[i][j] at i * kGsMaxIts + j (rotated in place into R as columns complete), the
// Givens rotations (c_j real at kGsCos + j, s_j at kGsSin + j) and the rotated right side g.
constexpr int kGsCos = kGsMaxVec * kGsMaxIts;
constexpr int kGsSin = kGsCos + kGsMaxIts;
constexpr int kGsRhs = kGsSin + kGsMaxIts;
constexpr int kGsState = kGsRhs + kGsMaxVec;
// c_i = sum over blocks of part (i < nv); w -= sum_i c_i V_i; H[i][col] = c_i (accumulate:
// += c_i); part2 != nullptr: block shares of ||w||^2 into part2[(b * nblk + blk) * kGsMaxVec]
template <typename T>
cudaError_t launch_gs_orth(vec2<T>* w, const vec2<T>* V, long long ld, int nv, long long N, const double2* part,
                           double2* st, int col, int accumulate, double2* part2, const Batch& bt, cudaStream_t s);
// h = sqrt(sum over blocks of part2); out = w / h (0 when h = 0).  col < 0: h is the initial
// residual norm (g = h e1); else h = H[col + 1][col], and column col is rotated by the
// previous rotations and a new one that zeroes h (applied to g too)
template <typename T>
cudaError_t launch_gs_scale(vec2<T>* out, const vec2<T>* w, long long N, const double2* part2, double2* st, int col,
                            const Batch& bt, cudaStream_t s);
// y = R^{-1} g over the first m columns (back substitution); x += V y (overwrite: x = V y)
template <typename T>
cudaError_t launch_gs_update(vec2<T>* x, const vec2<T>* V, long long ld, int m, long long N, const double2* st,
                             int overwrite, const Batch& bt, cudaStream_t s);

// ---- mixed formulation (mixed.cu): sigma-space kernels, one problem ----
// sigma vectors hold n^dim cells x dim components x 2^(dim-1) entries; u vectors the nodes.
template <typename T> struct MixArgs {
    GridDesc g;
    const vec2<T>* sig;   // sigma input (launch_mix_sigma: null = 0)
    const vec2<T>* sig2;  // launch_mix_div: second sigma input (null = 0)
    const vec2<T>* u;     // launch_mix_sigma: u input (null = 0)
    const vec2<T>* z;     // launch_mix_sigma: sigma-space input (null = 0)
    vec2<T>* y;           // output
    Cx<T> cs, cd, cz;
    int mass_out;
};
// mass_out = 1: y = M_sigma (cs sig + cd D u) + cz z;  mass_out = 0: y = cs sig + cd D u + cz M_sigma^{-1} z
// (D u: the gradient of u in V_h, so that M_sigma D = G)
template <typename T>
cudaError_t launch_mix_sigma(const MixArgs<T>& a, cudaStream_t s);
// y += G^T (cs sig + cd sig2) on the free nodes (y a u vector)
template <typename T>
cudaError_t launch_mix_div(const MixArgs<T>& a, cudaStream_t s);

// ---- FP64 Krylov kernels (blas.cu) ----
// Fixed reduction grid: results do not depend on timing or launch history.
constexpr int kRedBlocks = 304;
constexpr int kRedThreads = 256;

// Batch of nb problems for the Krylov kernels: problem b's V (or x) at offset b * bs_v, its w
// at b * bs_w, its results / coefficients / norms at b * bs_out; active[b] == 0 skips it.
struct KBatch {
    int nb;
    long long bs_v, bs_w, bs_out;
    const int* active;
};

// out[b*bs_out + i] = sum_p conj(V_{b,i}[p]) w_b[p], i < nvec (V_{b,i} = V + b*bs_v + i*ld);
// partials holds nb * nvec * kRedBlocks
cudaError_t launch_multidot(const double2* V, long long ld, int nvec, const double2* w, long long N, double2* partials,
                            double2* out, const KBatch& kb, cudaStream_t s);
// w_b += sign * sum_i coef[b*bs_out + i] V_{b,i}
cudaError_t launch_multi_axpy(double2* w, const double2* V, long long ld, int nvec, const double2* coef, double sign,
                              long long N, const KBatch& kb, cudaStream_t s);
// x_b *= 1 / sqrt(nrm2[b*bs_out].x) (x_b = x + b*bs_w; skipped when zero)
cudaError_t launch_scale_by_rnorm(double2* x, const double2* nrm2, long long N, const KBatch& kb, cudaStream_t s);

}  // namespace hh
