// Problems and batches of problems, the multigrid V-cycle, the shifted-HSS preconditioner
// (Def. 4.1) and the FP64 flexible GMRES outer iteration (Sec. 5.1), behind the C ABI of
// include/hh.h.
//
// A problem object holds nb >= 1 independent Helmholtz problems on the same grid (each with
// its own k, delta, delta_hat, HSS length and Krylov basis).  Every kernel launch covers all
// of them; a problem whose HSS loop has ended, or whose outer iteration has converged, is
// skipped on the device.  hh_create_problem is the batch of one.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <tuple>
#include <chrono>
#include <cmath>
#include <atomic>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hh.h"
#include "internal.h"

using hh::Cx;
using hh::GridDesc;
using hh::OpCoef;
using hh::PCoef;
using zc = std::complex<double>;

namespace {

thread_local std::string g_last_error;

hh_status fail(hh_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

#define HH_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? HH_ERR_OOM : HH_ERR_CUDA,       \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

#define HH_TRY(call)                  \
    do {                                \
        hh_status s_ = (call);          \
        if (s_ != HH_OK) return s_;     \
    } while (0)

#define HH_LAUNCH(call)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(HH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct Triple {
    double cK;
    zc cM, cG;
};

// Coefficient triples (c_K, c_M, c_Gamma) of the operators (Sec. 2, Def. 4.1).
Triple triple_B(double k, double delta) {
    const zc s(-delta, k);
    return {1.0, s * s, -s};
}
Triple triple_AL(double k, double dh) { return {1.0, zc(dh * dh - k * k, -2.0 * dh * k * k), zc(dh, -k * k)}; }
Triple triple_AR(double k, double dh) { return {-1.0, zc(k * k - dh * dh, -2.0 * dh * k * k), zc(-dh, -k * k)}; }
// the u-operator of the mixed shifted-HSS step after eliminating sigma (Def. 4.2):
// K + k^2 (dh - i)^2 M + k^2 (dh - i) M_Gamma
Triple triple_AMIX(double k, double dh) {
    const zc s(dh, -1.0);
    return {1.0, k * k * s * s, k * k * s};
}

template <typename T>
OpCoef<T> to_coef(const Triple& t) {
    OpCoef<T> o;
    o.cK = T(t.cK);
    o.cM = Cx<T>{T(t.cM.real()), T(t.cM.imag())};
    o.cG = Cx<T>{T(t.cG.real()), T(t.cG.imag())};
    return o;
}

int n_hss(double k, double theta) {
    const double v = std::pow(k, theta);
    const double r = std::round(v);
    if (std::fabs(v - r) <= 1e-9 * std::max(1.0, v)) return (int)r;
    return (int)std::ceil(v);
}

constexpr int kModes = 12;      // hh::MarchMode values 0..10 and the coarsest-level solve
constexpr int kCoarseMode = 11;

// Operators with a coefficient table (per problem and level).
// R_AL is the operator the cycles solve (A_mix for a mixed problem); R_MIXU the u-rows of the
// mixed system, (delta - i k) M + M_Gamma; R_MIXH those of the mixed HSS step's right side,
// k (dh + i) M + k M_Gamma.
enum Role { R_K = 0, R_M, R_MG, R_AL, R_AR, R_B, R_BHAT, R_MIXU, R_MIXH, R_COUNT };

// Device buffers of the multigrid hierarchy in one precision (nb problems per vector).
struct Hier {
    bool ready = false;
    size_t elem = 0;                  // bytes per complex entry
    std::vector<void*> xa, xb, b, t;  // per level: ping-pong iterates, right side, residual scratch
    std::vector<void*> wk, wr;        // W-cycles (levels >= 1): kept correction, its residual
    std::vector<void*> gv, gsm;       // GMRES smoother, per level: basis and work vector; sums,
                                      // Hessenberg matrices and norms (FP64)
    void* sig = nullptr;              // mixed: sigma iterate of the HSS loop and M_sigma^{-1} g_s
    void* ws = nullptr;
    void** ssrc = nullptr;            // mixed: device pointer to sig (for the gather kernel)
    void* r_lo = nullptr;             // level-0 copy of the preconditioner input
    void* rhs = nullptr;              // level-0 HSS right side
    void* ca = nullptr;               // extra level-0 buffers for cycles_per_hss > 1
    void* cb = nullptr;
    void* cres = nullptr;
    void* pc = nullptr;               // coefficient tables: [role][level][problem] PCoef<T>
    void* bw3 = nullptr;              // 3D boundary-class weights: [role][level][problem][26][9] Cx<T>
    std::vector<unsigned char> pc_host;  // host copy of the tables
    void** usrc = nullptr;            // device: per problem, the buffer holding u after the HSS loop
    cudaGraphExec_t graph = nullptr;  // one preconditioner application (the HSS loop)
    long long graph_kernels = 0;      // kernel nodes in the graph
    // the persistent form of the HSS loop (hh::HssLoop2<T> of this precision), built with the
    // graph's buffers and coefficients and dropped when they change
    std::vector<unsigned char> loop;
    int loop_ctas = 0;
    size_t loop_smem = 0;
    bool loop_unfit = false;  // its grid does not fit the device: separate kernels instead
};

}  // namespace

namespace hh {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace hh

struct hh_problem {
    int device = 0;
    hh_grid grid{};
    int nb = 1;
    std::vector<double> k, delta, dh;
    std::vector<int> nhss;
    int max_nhss = 0;
    int bc[6] = {0, 0, 0, 0, 0, 0};
    hh_options o{};
    std::vector<GridDesc> lv;
    cudaStream_t user = nullptr;
    cudaStream_t s = nullptr;  // the problem's own stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int* d_nhss = nullptr;     // device: HSS iterations per problem
    int* d_active = nullptr;   // device: 1 = problem takes part in the launches
    int* h_active = nullptr;   // pinned mirror
    unsigned* d_sync = nullptr;  // device: grid-barrier counter [0] and status word [1] of the
                                 // persistent HSS loop
    int* h_sync = nullptr;       // pinned copy of the status word
    Hier hier[2];
    // FP64 Krylov storage (level 0), laid out [vector][problem][node]
    long long N = 0;            // entries per problem of the Krylov vectors (+ ns when mixed)
    bool mixed = false;         // mixed formulation (one problem)
    long long ns = 0;           // its sigma entries
    double2* V = nullptr;       // (restart+1) x nb x N
    double2* Z = nullptr;       // restart x nb x N
    double2* x = nullptr;       // nb x N
    double2* bvec = nullptr;    // nb x N masked right side
    double2* r = nullptr;       // nb x N residual / scratch
    double2* partials = nullptr;
    double2* hbuf = nullptr;    // nb x [hA (restart+1) | hB (restart+1) | nrm2]
    double2* ybuf = nullptr;    // nb x restart back-substitution results
    double2* h_host = nullptr;  // pinned mirror of hbuf (and of ybuf)
    size_t bytes = 0;
    std::vector<void*> allocs;
    // tile shapes of the stencil kernels per precision, level and mode: {rows, form}, 0 = automatic
    std::vector<std::array<std::array<int, 2>, kModes>> tune[2];
};

namespace {

// process-wide cap on the device bytes one problem may hold (0: none), for failure injection
// and for callers that share the device
std::atomic<size_t> g_alloc_limit{0};

hh_status dmalloc(hh_problem* p, void** ptr, size_t bytes) {
    const size_t cap = g_alloc_limit.load();
    if (cap && p->bytes + bytes > cap) {
        *ptr = nullptr;
        return fail(HH_ERR_OOM, "allocation of " + std::to_string(bytes) + " bytes exceeds the limit of " +
                                    std::to_string(cap) + " bytes per problem");
    }
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(HH_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    p->allocs.push_back(*ptr);
    p->bytes += bytes;
    return HH_OK;
}

GridDesc level_desc(const hh_grid& grid, const int* bc, int l) {
    GridDesc g;
    g.dim = grid.dim;
    g.n = grid.n >> l;
    g.nn = g.n + 1;
    g.N = 1;
    for (int d = 0; d < g.dim; ++d) g.N *= g.nn;
    g.h = 1.0 / g.n;
    for (int s = 0; s < 6; ++s) g.dir[s] = (s < 2 * g.dim) ? (bc[s] == HH_BC_DIRICHLET) : 0;
    return g;
}

// Device bytes of the Krylov storage and batch bookkeeping for nb problems (matches create).
long long sigma_dofs(const hh_grid* grid) {
    const long long n = grid->n;
    return grid->dim == 3 ? n * n * n * 3 * 4 : n * n * 2 * 2;
}

size_t krylov_bytes(const hh_grid* grid, int restart, int nb, long long extra) {
    long long nn = grid->n + 1;
    long long N = nn * nn * (grid->dim == 3 ? nn : 1) + extra;
    const size_t m = (size_t)restart, B = (size_t)nb;
    size_t tot = 2 * sizeof(int) * B + 16;                 // nhss, active, barrier words
    tot += (2 * m + 1 + 3) * B * (size_t)N * 16;           // V, Z, x, bvec, r
    tot += B * (m + 1) * hh::kRedBlocks * 16;              // partials
    tot += B * (2 * (m + 1) + 1) * 16 + B * m * 16;        // hbuf, ybuf
    return tot;
}

// Coefficient table entry of operator `role` on grid g for problem b.
template <typename T>
PCoef<T> make_pcoef(const hh_problem* p, int role, const GridDesc& g, int b) {
    const double k = p->k[b], dh = p->dh[b], delta = p->delta[b];
    Triple op, opd = p->mixed ? triple_AMIX(k, dh) : triple_AL(k, dh);
    double al = 0.0, be = 0.0;
    switch (role) {
        case R_K: op = {1.0, 0.0, 0.0}; break;
        case R_M: op = {0.0, 1.0, 0.0}; break;
        case R_MG: op = {0.0, 0.0, 1.0}; break;
        case R_AL: op = opd; break;
        case R_AR:
            op = triple_AR(k, dh);
            al = (k - 1.0) / (k + 1.0);
            be = 2.0 * k / (k + 1.0);
            break;
        case R_B: op = triple_B(k, delta); break;
        case R_MIXU: op = {0.0, zc(delta, -k), 1.0}; break;
        case R_MIXH: op = {0.0, zc(k * dh, k), k}; break;
        default: op = triple_B(k, dh); break;
    }
    if (role != R_AR && role != R_AL) opd = op;
    PCoef<T> c{};
    c.op = to_coef<T>(op);
    c.opd = to_coef<T>(opd);
    c.alpha = Cx<T>{T(al), T(0)};
    c.beta = Cx<T>{T(be), T(0)};
    hh::interior_weights<T>(c, g, p->o.omega);
    return c;
}

template <typename T>
hh_status build_tables(hh_problem* p, Hier& H) {
    const int L = p->o.levels, nb = p->nb;
    std::vector<PCoef<T>> tab((size_t)R_COUNT * L * nb);
    for (int role = 0; role < R_COUNT; ++role)
        for (int l = 0; l < L; ++l)
            for (int b = 0; b < nb; ++b) tab[((size_t)role * L + l) * nb + b] = make_pcoef<T>(p, role, p->lv[l], b);
    const size_t bytes = tab.size() * sizeof(PCoef<T>);
    H.pc_host.assign((const unsigned char*)tab.data(), (const unsigned char*)tab.data() + bytes);
    if (!H.pc) HH_TRY(dmalloc(p, &H.pc, bytes));  // kept when the parameters change
    HH_CUDA(cudaMemcpyAsync(H.pc, tab.data(), bytes, cudaMemcpyHostToDevice, p->s));
    if (p->grid.dim == 3) {
        const size_t per = (size_t)hh::kClass3 * hh::kClass3Len;
        std::vector<Cx<T>> w3(tab.size() * per);
        for (int role = 0; role < R_COUNT; ++role)
            for (int l = 0; l < L; ++l)
                for (int b = 0; b < nb; ++b) {
                    const size_t e = ((size_t)role * L + l) * nb + b;
                    hh::boundary_weights3<T>(w3.data() + e * per, tab[e], p->lv[l], p->o.omega);
                }
        if (!H.bw3) HH_TRY(dmalloc(p, &H.bw3, w3.size() * sizeof(Cx<T>)));
        HH_CUDA(cudaMemcpyAsync(H.bw3, w3.data(), w3.size() * sizeof(Cx<T>), cudaMemcpyHostToDevice, p->s));
    }
    HH_CUDA(cudaStreamSynchronize(p->s));
    return HH_OK;
}

// GMRES smoother: iterations of the longest smoothing step (0 with the Jacobi smoother)
int gs_its(const hh_options* o) {
    return o->smoother == HH_SMOOTH_GMRES ? std::max(o->nu_pre, std::max(o->nu_post, o->nu_coarse)) : 0;
}
// its FP64 scratch of one level: block sums (two sets), Hessenberg matrices, norms
size_t gs_small_bytes(long long N, int nb) {
    return (size_t)nb * (2 * (size_t)hh::gs_blocks(N) * hh::kGsMaxVec + hh::kGsState) * sizeof(double2);
}

// Device bytes of one precision's multigrid buffers for nb problems plus the coefficient
// tables (matches ensure_hier and ensure_tables).
size_t hier_bytes(const hh_grid* grid, const hh_options* o, int prec, int nb) {
    const int levels = o->levels, gamma = o->cycle_gamma, gs = gs_its(o);
    const size_t elem = prec == HH_C64 ? 8 : 16, B = (size_t)nb;
    size_t tot = 0;
    for (int l = 0; l < levels; ++l) {
        long long nn = (grid->n >> l) + 1;
        long long N = nn * nn * (grid->dim == 3 ? nn : 1);
        tot += 4 * (size_t)N * elem * B;  // xa, xb, b, t
        if (gamma > 1 && l >= 1) tot += 2 * (size_t)N * elem * B;  // W-cycle correction and residual
        if (l == 0) tot += 5 * (size_t)N * elem * B;  // r_lo, rhs, ca, cb, cres
        if (gs > 0) tot += (size_t)(gs + 2) * N * elem * B + gs_small_bytes(N, nb);  // basis, w, sums
    }
    if (o->formulation == HH_FORM_MIXED)  // r_lo's sigma part, sig, ws, the pointer table
        tot += 3 * (size_t)sigma_dofs(grid) * elem * B + sizeof(void*) * B;
    tot += sizeof(void*) * B;  // usrc
    // coefficient tables of both precisions (and the 3D boundary-class tables)
    tot += (size_t)R_COUNT * levels * B * (sizeof(PCoef<float>) + sizeof(PCoef<double>));
    if (grid->dim == 3)
        tot += (size_t)R_COUNT * levels * B * hh::kClass3 * hh::kClass3Len * (sizeof(Cx<float>) + sizeof(Cx<double>));
    return tot;
}

// Coefficient tables of both precisions (small; built at creation, so that the FP64 outer
// operator never needs the FP64 multigrid buffers).
hh_status ensure_tables(hh_problem* p) {
    if (!p->hier[HH_C64].pc) HH_TRY(build_tables<float>(p, p->hier[HH_C64]));
    if (!p->hier[HH_C128].pc) HH_TRY(build_tables<double>(p, p->hier[HH_C128]));
    return HH_OK;
}

// Multigrid buffers of one precision (allocated on first use).
hh_status ensure_hier(hh_problem* p, int prec) {
    Hier& H = p->hier[prec];
    if (H.ready) return HH_OK;
    HH_TRY(ensure_tables(p));
    H.elem = prec == HH_C64 ? 8 : 16;
    const int L = p->o.levels;
    H.xa.assign(L, nullptr);
    H.xb.assign(L, nullptr);
    H.b.assign(L, nullptr);
    H.t.assign(L, nullptr);
    H.wk.assign(L, nullptr);
    H.wr.assign(L, nullptr);
    H.gv.assign(L, nullptr);
    H.gsm.assign(L, nullptr);
    const int gs = gs_its(&p->o);
    for (int l = 0; l < L; ++l) {
        const size_t nbytes = (size_t)p->lv[l].N * p->nb * H.elem;
        if (gs > 0) {
            const size_t sb = gs_small_bytes(p->lv[l].N, p->nb);
            HH_TRY(dmalloc(p, &H.gv[l], (size_t)(gs + 2) * nbytes));
            HH_TRY(dmalloc(p, &H.gsm[l], sb));
            HH_CUDA(cudaMemsetAsync(H.gv[l], 0, (size_t)(gs + 2) * nbytes, p->s));
            HH_CUDA(cudaMemsetAsync(H.gsm[l], 0, sb, p->s));
        }
        if (p->o.cycle_gamma > 1 && l >= 1) {
            HH_TRY(dmalloc(p, &H.wk[l], nbytes));
            HH_TRY(dmalloc(p, &H.wr[l], nbytes));
        }
        HH_TRY(dmalloc(p, &H.xa[l], nbytes));
        HH_TRY(dmalloc(p, &H.xb[l], nbytes));
        HH_TRY(dmalloc(p, &H.b[l], nbytes));
        HH_TRY(dmalloc(p, &H.t[l], nbytes));
        HH_CUDA(cudaMemsetAsync(H.xa[l], 0, nbytes, p->s));
        HH_CUDA(cudaMemsetAsync(H.xb[l], 0, nbytes, p->s));
        HH_CUDA(cudaMemsetAsync(H.b[l], 0, nbytes, p->s));
        HH_CUDA(cudaMemsetAsync(H.t[l], 0, nbytes, p->s));
    }
    const size_t n0 = (size_t)p->lv[0].N * p->nb * H.elem;
    const size_t nsb = (size_t)p->ns * p->nb * H.elem;
    HH_TRY(dmalloc(p, &H.r_lo, n0 + nsb));
    if (p->mixed) {
        HH_TRY(dmalloc(p, &H.sig, nsb));
        HH_TRY(dmalloc(p, &H.ws, nsb));
        HH_TRY(dmalloc(p, (void**)&H.ssrc, sizeof(void*)));
        HH_CUDA(cudaMemcpyAsync(H.ssrc, &H.sig, sizeof(void*), cudaMemcpyHostToDevice, p->s));
        HH_CUDA(cudaStreamSynchronize(p->s));
    }
    HH_TRY(dmalloc(p, &H.rhs, n0));
    HH_TRY(dmalloc(p, &H.ca, n0));
    HH_TRY(dmalloc(p, &H.cb, n0));
    HH_TRY(dmalloc(p, &H.cres, n0));
    HH_TRY(dmalloc(p, (void**)&H.usrc, sizeof(void*) * p->nb));
    // one-time kernel configuration now: nothing may call into the runtime's
    // configuration API later, while the stream is being captured
    HH_CUDA(prec == HH_C64 ? hh::prepare_coarse<float>() : hh::prepare_coarse<double>());
    H.ready = true;
    return HH_OK;
}

// Order work on the problem stream after the caller's stream, and back.
hh_status join_in(hh_problem* p) {
    hh::g_use_pdl = p->o.use_pdl ? 1 : 0;
    HH_CUDA(cudaEventRecord(p->ev_in, p->user));
    HH_CUDA(cudaStreamWaitEvent(p->s, p->ev_in, 0));
    return HH_OK;
}
hh_status join_out(hh_problem* p) {
    HH_CUDA(cudaEventRecord(p->ev_out, p->s));
    HH_CUDA(cudaStreamWaitEvent(p->user, p->ev_out, 0));
    return HH_OK;
}

// Set the device activity flags of the batch (all problems when flags == nullptr).
hh_status set_active(hh_problem* p, const std::vector<char>* flags) {
    for (int b = 0; b < p->nb; ++b) p->h_active[b] = flags ? (*flags)[b] : 1;
    HH_CUDA(cudaMemcpyAsync(p->d_active, p->h_active, sizeof(int) * p->nb, cudaMemcpyHostToDevice, p->s));
    // the pinned mirror may be rewritten right after: wait for the copy
    HH_CUDA(cudaStreamSynchronize(p->s));
    return HH_OK;
}

// Device activity flags for the kernels.  A batch of one is never launched while inactive
// (its outer loop ends first) and its HSS loop is the whole loop: no flags to read.
const int* active_flags(const hh_problem* p) { return p->nb == 1 ? nullptr : p->d_active; }

// ------------------------------------------------------------------ V-cycle
template <typename T>
struct MG {
    using V2 = hh::vec2<T>;
    hh_problem* p;
    Hier* H;
    cudaStream_t s;
    T omega;
    int hss_it = -1;  // HSS iteration being recorded (problems whose loop has ended are skipped)

    bool d2() const { return p->grid.dim == 2; }
    long long Nl(int l) const { return p->lv[l].N; }

    const PCoef<T>* table(int role, int l) const {
        return (const PCoef<T>*)H->pc + ((size_t)role * p->o.levels + l) * p->nb;
    }

    hh::MArgs<T> margs(int l, int role) const {
        hh::MArgs<T> a{};
        a.g = p->lv[l];
        if (p->nb == 1) {
            // a batch of one: coefficients in the kernel parameters, no device flags to read
            a.pc = nullptr;
            std::memcpy(&a.c0, H->pc_host.data() + ((size_t)role * p->o.levels + l) * sizeof(PCoef<T>),
                        sizeof(PCoef<T>));
        } else {
            a.pc = table(role, l);
        }
        if (H->bw3)
            a.bw3 = (const Cx<T>*)H->bw3 + ((size_t)role * p->o.levels + l) * p->nb * hh::kClass3 * hh::kClass3Len;
        a.nb = p->nb;
        a.bs = Nl(l);
        a.bsc = l + 1 < p->o.levels ? Nl(l + 1) : 0;
        a.omega = omega;
        a.tile_rows = p->o.tile_rows;
        a.tile_form = p->o.tile_form;
        a.hss_it = p->nb == 1 ? -1 : hss_it;
        a.nhss = p->d_nhss;
        a.active = active_flags(p);
        return a;
    }

    // arguments of the fused two-sweep modes: role for the first stage, A_L for the second
    hh::MArgs<T> margs2(int l, int role) const {
        hh::MArgs<T> a = margs(l, role);
        if (p->nb == 1) {
            std::memcpy(&a.c02, H->pc_host.data() + ((size_t)R_AL * p->o.levels + l) * sizeof(PCoef<T>),
                        sizeof(PCoef<T>));
        } else {
            a.pc2 = table(R_AL, l);
        }
        return a;
    }

    // two consecutive sweeps of level l run as one pass (2D): it removes a launch and a trip
    // through memory but computes the first sweep on a wider halo, which pays while the
    // level is latency-bound (measured: faster up to 513^2 nodes, slower from 1025^2)
    bool fused2(int l) const { return d2() && p->o.fuse_sweeps && Nl(l) * p->nb <= 600000; }

    hh::Batch batch(int l) const {
        return hh::Batch{p->nb, Nl(l), l + 1 < p->o.levels ? Nl(l + 1) : 0, p->nb == 1 ? -1 : hss_it, p->d_nhss,
                         active_flags(p)};
    }

    // the tuned tile shape of (level of a.g, mode), if any
    cudaError_t march(int mode, const hh::MArgs<T>& a) const {
        hh::MArgs<T> t = a;
        const int prec = sizeof(T) == 4 ? HH_C64 : HH_C128;
        const auto& tab = p->tune[prec];
        int l = 0;
        while ((p->grid.n >> l) != a.g.n) ++l;
        if (mode < kModes && l < (int)tab.size() && tab[l][mode][0] != 0) {
            t.tile_rows = tab[l][mode][0];
            t.tile_form = tab[l][mode][1];
        }
        if (mode == hh::M_JACOBI2_ZERO_RR || mode == hh::M_HSS_FIRST2_RR) return hh::launch_march2rr<T>(mode, t, s);
        return d2() ? hh::launch_march2<T>(mode, t, s) : hh::launch_march3<T>(mode, t, s);
    }

    // ---- level kernels ----
    // x_out = x_in + omega D^{-1} (b - A_L x_in); x_in == nullptr means 0
    hh_status jacobi(int l, const V2* b, const V2* xin, V2* xout) {
        hh::MArgs<T> a = margs(l, R_AL);
        a.x = xin;
        a.xzero = xin == nullptr;
        a.z = b;
        a.y = xout;
        HH_LAUNCH(march(hh::M_JACOBI, a));
        return HH_OK;
    }
    // two sweeps from x = 0
    hh_status jacobi2_zero(int l, const V2* b, V2* xout) {
        hh::MArgs<T> a = margs(l, R_AL);
        a.z = b;
        a.y = xout;
        HH_LAUNCH(march(hh::M_JACOBI2_ZERO, a));
        return HH_OK;
    }
    // rc = P^T (b - A_L x)
    hh_status resid_restrict(int l, const V2* b, const V2* x, V2* rc) {
        hh::MArgs<T> a = margs(l, R_AL);
        a.x = x;
        a.z = b;
        if (d2()) {
            a.y = rc;
            HH_LAUNCH(march(hh::M_RESID_RESTRICT, a));
        } else {
            a.y = (V2*)H->t[l];
            a.alpha = Cx<T>{-1, 0};
            a.beta = Cx<T>{1, 0};
            HH_LAUNCH(hh::launch_march3<T>(hh::M_AXPBY, a, s));
            HH_LAUNCH(hh::launch_restrict<T>(p->lv[l + 1], (const V2*)H->t[l], rc, batch(l), s));
        }
        return HH_OK;
    }
    // xout = x~ + omega D^{-1} (b - A_L x~), x~ = x + P ec
    hh_status prolong_jacobi(int l, V2* x, const V2* ec, const V2* b, V2* xout) {
        hh::MArgs<T> a = margs(l, R_AL);
        a.x = x;
        a.ec = ec;
        a.z = b;
        a.y = xout;
        HH_LAUNCH(march(hh::M_PROLONG_JACOBI, a));
        return HH_OK;
    }
    // xout = two sweeps from x~ = x + P ec, in one pass
    hh_status prolong_jacobi2(int l, V2* x, const V2* ec, const V2* b, V2* xout) {
        hh::MArgs<T> a = margs2(l, R_AL);
        a.x = x;
        a.ec = ec;
        a.z = b;
        a.y = xout;
        HH_LAUNCH(march(hh::M_PROLONG_JACOBI2, a));
        return HH_OK;
    }
    // pre-smoothing passes that also restrict the residual (2D levels where fused2 holds)
    bool fused_rr(int l) const { return fused2(l) && p->o.nu_pre == 2 && l + 1 < p->o.levels; }
    // xout = two sweeps from 0 on A_L x = b, rc = P^T (b - A_L xout), in one pass
    hh_status jacobi2_zero_rr(int l, const V2* b, V2* xout, V2* rc) {
        hh::MArgs<T> a = margs2(l, R_AL);
        a.z = b;
        a.y = xout;
        a.yc = rc;
        HH_LAUNCH(march(hh::M_JACOBI2_ZERO_RR, a));
        return HH_OK;
    }
    // the HSS right side, two sweeps and the restricted residual, in one pass
    hh_status hss_first2_rr(const V2* u, const V2* r, V2* rhs, V2* x2, V2* rc) {
        hh::MArgs<T> a = margs2(0, R_AR);
        a.x = u;
        a.xzero = u == nullptr;
        a.z = r;
        a.y = rhs;
        a.y2 = x2;
        a.yc = rc;
        a.use_pc_ab = 1;
        HH_LAUNCH(march(hh::M_HSS_FIRST2_RR, a));
        return HH_OK;
    }
    // rhs = c1 A_R u + c2 r and two Jacobi sweeps from 0 on A_L x = rhs, in one pass
    hh_status hss_first2(const V2* u, const V2* r, V2* rhs, V2* x2) {
        hh::MArgs<T> a = margs2(0, R_AR);
        a.x = u;
        a.xzero = u == nullptr;
        a.z = r;
        a.y = rhs;
        a.y2 = x2;
        a.use_pc_ab = 1;
        HH_LAUNCH(march(hh::M_HSS_FIRST2, a));
        return HH_OK;
    }
    // rhs = c1 A_R u + c2 r and the first Jacobi sweep x1 = omega D^{-1} rhs (u == nullptr: u = 0)
    hh_status hss_first(const V2* u, const V2* r, V2* rhs, V2* x1) {
        hh::MArgs<T> a = margs(0, R_AR);
        a.x = u;
        a.xzero = u == nullptr;
        a.z = r;
        a.y = rhs;
        a.y2 = x1;
        a.use_pc_ab = 1;
        HH_LAUNCH(march(hh::M_HSS_FIRST, a));
        return HH_OK;
    }
    hh_status hss_rhs(const V2* u, const V2* r, V2* rhs) {
        hh::MArgs<T> a = margs(0, R_AR);
        a.x = u;
        a.xzero = u == nullptr;
        a.z = r;
        a.y = rhs;
        a.use_pc_ab = 1;
        HH_LAUNCH(march(hh::M_AXPBY, a));
        return HH_OK;
    }

    V2* other(int l, V2* x) { return x == (V2*)H->xa[l] ? (V2*)H->xb[l] : (V2*)H->xa[l]; }

    // nsweeps more sweeps starting from the iterate in *x (ping-pong within level l)
    hh_status smooth(int l, const V2* b, int nsweeps, V2** x) {
        V2* cur = *x;
        for (int k = 0; k < nsweeps; ++k) {
            V2* oth = other(l, cur);
            HH_TRY(jacobi(l, b, cur, oth));
            cur = oth;
        }
        *x = cur;
        return HH_OK;
    }

    // nsweeps sweeps from x = 0 into the level-l buffers
    hh_status smooth_from_zero(int l, const V2* b, int nsweeps, V2** out) {
        V2* cur = (V2*)H->xa[l];
        if (nsweeps == 0) {
            HH_LAUNCH(hh::launch_zero<T>(cur, Nl(l), batch(l), s));
        } else if (nsweeps == 1) {
            HH_TRY(jacobi(l, b, nullptr, cur));
        } else {
            HH_TRY(jacobi2_zero(l, b, cur));
            HH_TRY(smooth(l, b, nsweeps - 2, &cur));
        }
        *out = cur;
        return HH_OK;
    }

    bool gm() const { return p->o.smoother == HH_SMOOTH_GMRES; }

    // GMRES smoother on level l: `its` iterations of GMRES on omega D^{-1} A_L x = omega D^{-1} b
    // from x (xzero: from 0), the result written over x.  omega scales the preconditioned system
    // and its residual alike, so the iterates are those of the plain Jacobi preconditioner.
    hh_status gsmooth(int l, const V2* b, V2* x, bool xzero, int its) {
        const long long N = Nl(l);
        const hh::Batch bt = batch(l);
        if (its == 0) {
            if (xzero) HH_LAUNCH(hh::launch_zero<T>(x, N, bt, s));
            return HH_OK;
        }
        const long long ld = N * p->nb;  // basis vector stride
        V2* Vb = (V2*)H->gv[l];
        if (d2() && N <= hh::kGsCtaNodes) {
            // small 2D level: the whole step in one CTA per problem (one launch instead of 6 its + 4)
            hh::MArgs<T> a = margs(l, R_AL);
            HH_LAUNCH(hh::launch_gs_cta<T>(a, b, x, xzero ? 1 : 0, its, Vb, ld, s));
            return HH_OK;
        }
        V2* W = Vb + (long long)(its + 1) * ld;  // after the basis
        const int nblk = hh::gs_blocks(N);
        double2* part = (double2*)H->gsm[l];
        double2* part2 = part + (size_t)p->nb * nblk * hh::kGsMaxVec;
        double2* st = part2 + (size_t)p->nb * nblk * hh::kGsMaxVec;  // least-squares state
        // z0 = omega D^{-1} (b - A_L x), beta = ||z0||, v_0 = z0 / beta
        hh::MArgs<T> a = margs(l, R_AL);
        a.x = xzero ? nullptr : x;
        a.xzero = xzero;
        a.z = b;
        a.y = W;
        a.alpha = Cx<T>{-1, 0};
        a.beta = Cx<T>{1, 0};
        HH_LAUNCH(march(hh::M_DAXPBY, a));
        HH_LAUNCH(hh::launch_gs_dot<T>(W, ld, 1, W, N, part, bt, s));
        HH_LAUNCH(hh::launch_gs_scale<T>(Vb, W, N, part, st, -1, bt, s));
        for (int j = 0; j < its; ++j) {
            V2* vj = Vb + (long long)j * ld;
            hh::MArgs<T> m = margs(l, R_AL);
            m.x = vj;
            m.z = vj;  // beta = 0: read, not used
            m.y = W;
            m.alpha = Cx<T>{1, 0};
            m.beta = Cx<T>{0, 0};
            HH_LAUNCH(march(hh::M_DAXPBY, m));
            // classical Gram-Schmidt, twice
            HH_LAUNCH(hh::launch_gs_dot<T>(Vb, ld, j + 1, W, N, part, bt, s));
            HH_LAUNCH(hh::launch_gs_orth<T>(W, Vb, ld, j + 1, N, part, st, j, 0, nullptr, bt, s));
            HH_LAUNCH(hh::launch_gs_dot<T>(Vb, ld, j + 1, W, N, part, bt, s));
            HH_LAUNCH(hh::launch_gs_orth<T>(W, Vb, ld, j + 1, N, part, st, j, 1, part2, bt, s));
            HH_LAUNCH(hh::launch_gs_scale<T>(Vb + (long long)(j + 1) * ld, W, N, part2, st, j, bt, s));
        }
        HH_LAUNCH(hh::launch_gs_update<T>(x, Vb, ld, its, N, st, xzero ? 1 : 0, bt, s));
        return HH_OK;
    }

    // the coarse correction of level l (one cycle on level l + 1 for the right side in
    // H->b[l + 1], and gamma - 1 more on what it leaves for a W-cycle); result buffer in *ec
    hh_status coarse_correction(int l, V2** ec_out) {
        V2* ec;
        HH_TRY(vcycle(l + 1, (const V2*)H->b[l + 1], nullptr, &ec));
        if (p->o.cycle_gamma > 1) {
            // W-cycle: further cycles on the coarse problem, each on the residual that the
            // correction so far leaves, kept outside the coarse ping-pong buffers
            const int c = l + 1;
            V2* keep = (V2*)H->wk[c];
            HH_LAUNCH(hh::launch_copy<T>(keep, ec, Nl(c), batch(c), s));
            for (int g = 1; g < p->o.cycle_gamma; ++g) {
                hh::MArgs<T> a = margs(c, R_AL);
                a.x = keep;
                a.z = (const V2*)H->b[c];
                a.y = (V2*)H->wr[c];
                a.alpha = Cx<T>{-1, 0};
                a.beta = Cx<T>{1, 0};
                HH_LAUNCH(march(hh::M_AXPBY, a));
                V2* corr;
                HH_TRY(vcycle(c, (const V2*)H->wr[c], nullptr, &corr));
                HH_LAUNCH(hh::launch_add<T>(keep, corr, Nl(c), batch(c), s));
            }
            ec = keep;
        }
        *ec_out = ec;
        return HH_OK;
    }

    // One cycle with the GMRES smoother: every step in place in the level's first buffer
    hh_status gcycle(int l, const V2* b, V2** out) {
        V2* x = (V2*)H->xa[l];
        if (l == p->o.levels - 1) {
            HH_TRY(gsmooth(l, b, x, true, p->o.nu_coarse));
        } else {
            HH_TRY(gsmooth(l, b, x, true, p->o.nu_pre));
            HH_TRY(resid_restrict(l, b, x, (V2*)H->b[l + 1]));
            V2* ec;
            HH_TRY(coarse_correction(l, &ec));
            HH_LAUNCH(hh::launch_prolong<T>(p->lv[l], ec, x, batch(l), s));
            HH_TRY(gsmooth(l, b, x, false, p->o.nu_post));
        }
        *out = x;
        return HH_OK;
    }

    // One V-cycle on level l for right side b from x = 0; result buffer in *out.
    // xstart: the first `done` pre-smoothing sweeps were already done and sit in xstart;
    // restricted: all pre-sweeps are done and the coarse residual already sits in H->b[l + 1].
    hh_status vcycle(int l, const V2* b, V2* xstart, V2** out, int done = 1, bool restricted = false) {
        const int L = p->o.levels;
        if (gm()) return gcycle(l, b, out);  // never entered with a started iterate
        if (l == L - 1) {
            V2* x = (V2*)H->xa[l];
            if (xstart) {
                x = xstart;
                HH_TRY(smooth(l, b, p->o.nu_coarse - done, &x));
            } else if (p->o.nu_coarse >= 1 && Nl(l) <= p->o.coarse_cluster_nodes && hh::coarse_fits<T>(p->lv[l])) {
                hh::MArgs<T> a = margs(l, R_AL);
                a.z = b;
                a.y = x;
                const auto& tab = p->tune[sizeof(T) == 4 ? HH_C64 : HH_C128];
                a.tile_rows = l < (int)tab.size() ? tab[l][kCoarseMode][0] : 0;
                a.tile_form = l < (int)tab.size() ? tab[l][kCoarseMode][1] : 0;
                if (a.tile_rows == 0 && p->o.coarse_kernel == 1) a.tile_rows = hh::coarse_cluster_size();
                if (a.tile_rows == 0 && p->o.coarse_kernel == 2) a.tile_form = 3;
                HH_LAUNCH(hh::launch_coarse_solve<T>(a, p->o.nu_coarse, s));
            } else {
                HH_TRY(smooth_from_zero(l, b, p->o.nu_coarse, &x));
            }
            *out = x;
            return HH_OK;
        }
        V2* x;
        if (restricted) {
            x = xstart;
        } else if (xstart) {
            x = xstart;
            HH_TRY(smooth(l, b, p->o.nu_pre - done, &x));
        } else if (fused_rr(l)) {
            x = (V2*)H->xa[l];
            HH_TRY(jacobi2_zero_rr(l, b, x, (V2*)H->b[l + 1]));
            restricted = true;
        } else {
            HH_TRY(smooth_from_zero(l, b, p->o.nu_pre, &x));
        }
        if (!restricted) HH_TRY(resid_restrict(l, b, x, (V2*)H->b[l + 1]));
        V2* ec;
        HH_TRY(coarse_correction(l, &ec));
        if (p->o.nu_post == 0) {
            HH_LAUNCH(hh::launch_prolong<T>(p->lv[l], ec, x, batch(l), s));
        } else if (p->o.nu_post >= 2 && fused2(l)) {
            V2* oth = other(l, x);
            HH_TRY(prolong_jacobi2(l, x, ec, b, oth));
            x = oth;
            HH_TRY(smooth(l, b, p->o.nu_post - 2, &x));
        } else {
            V2* oth = other(l, x);
            HH_TRY(prolong_jacobi(l, x, ec, b, oth));
            x = oth;
            HH_TRY(smooth(l, b, p->o.nu_post - 1, &x));
        }
        *out = x;
        return HH_OK;
    }

    // cycles_per_hss V-cycles for A_L x = b; the first may start from xstart (`done` sweeps,
    // `restricted` as in vcycle).
    hh_status mg_solve(const V2* b, V2* xstart, V2** out, int done = 1, bool restricted = false) {
        V2* x;
        HH_TRY(vcycle(0, b, xstart, &x, done, restricted));
        const long long N = Nl(0);
        for (int c = 1; c < p->o.cycles_per_hss; ++c) {
            // keep x outside the level-0 ping-pong buffers the next cycle overwrites
            V2* keep = (V2*)((x == (V2*)H->ca) ? H->cb : H->ca);
            HH_LAUNCH(hh::launch_copy<T>(keep, x, N, batch(0), s));
            hh::MArgs<T> a = margs(0, R_AL);
            a.x = keep;
            a.z = b;
            a.y = (V2*)H->cres;
            a.alpha = Cx<T>{-1, 0};
            a.beta = Cx<T>{1, 0};
            HH_LAUNCH(march(hh::M_AXPBY, a));
            V2* corr;
            HH_TRY(vcycle(0, (const V2*)H->cres, nullptr, &corr));
            HH_LAUNCH(hh::launch_add<T>(keep, corr, N, batch(0), s));
            x = keep;
        }
        *out = x;
        return HH_OK;
    }

    // The shifted-HSS preconditioner of Def. 4.2 for a mixed problem on r_lo = (R_s, R_u),
    // through the elimination of sigma.  Each step, from (sigma, u):
    //   w_s    = M_s^{-1} g_s = c1 k (dh + i) sigma + c1 D u + c2 M_s^{-1} R_s
    //   rhs_u  = k (dh - i) [c1 (k (dh + i) M + k M_Gamma) u + c2 R_u] - G^T (k (dh - i) c1 sigma + w_s)
    //   u'     = cycles on A_mix u' = rhs_u
    //   sigma' = (w_s + D u') / (k (dh - i))
    // (g_s, g_u: the right sides of Def. 4.2's tau- and v-rows; G = M_s D).  *u_out receives the
    // buffer holding u; sigma ends in H->sig.
    hh_status mixed_hss_loop(V2** u_out) {
        const double k = p->k[0], dh = p->dh[0];
        const double c1 = (k - 1.0) / (k + 1.0), c2 = 2.0 * k / (k + 1.0);
        const std::complex<double> kp(k * dh, k), km(k * dh, -k);  // k (dh + i), k (dh - i)
        auto C = [](std::complex<double> z) { return Cx<T>{T(z.real()), T(z.imag())}; };
        const V2* Rs = (const V2*)H->r_lo;
        const V2* Ru = Rs + p->ns;
        V2* sig = (V2*)H->sig;
        V2* ws = (V2*)H->ws;
        V2* rhs = (V2*)H->rhs;
        HH_LAUNCH(hh::launch_zero<T>(sig, p->ns, batch(0), s));
        V2* u = nullptr;
        for (int it = 0; it < p->max_nhss; ++it) {
            hh::MixArgs<T> a{};
            a.g = p->lv[0];
            a.sig = sig;
            a.u = u;
            a.z = Rs;
            a.y = ws;
            a.cs = C(c1 * kp);
            a.cd = C(std::complex<double>(c1, 0.0));
            a.cz = C(std::complex<double>(c2, 0.0));
            a.mass_out = 0;
            HH_LAUNCH(hh::launch_mix_sigma<T>(a, s));
            hh::MArgs<T> m = margs(0, R_MIXH);
            m.x = u;
            m.xzero = u == nullptr;
            m.z = Ru;
            m.y = rhs;
            m.alpha = C(c1 * km);
            m.beta = C(c2 * km);
            HH_LAUNCH(march(hh::M_AXPBY, m));
            hh::MixArgs<T> d{};
            d.g = p->lv[0];
            d.sig = sig;
            d.sig2 = ws;
            d.y = rhs;
            d.cs = C(-c1 * km);
            d.cd = C(std::complex<double>(-1.0, 0.0));
            HH_LAUNCH(hh::launch_mix_div<T>(d, s));
            HH_TRY(mg_solve(rhs, nullptr, &u));
            hh::MixArgs<T> r{};
            r.g = p->lv[0];
            r.sig = ws;
            r.u = u;
            r.y = sig;
            r.cs = C(1.0 / km);
            r.cd = C(1.0 / km);
            r.mass_out = 0;
            HH_LAUNCH(hh::launch_mix_sigma<T>(r, s));
        }
        if (!u) {  // no HSS step: u = 0
            u = (V2*)H->cres;
            HH_LAUNCH(hh::launch_zero<T>(u, Nl(0), batch(0), s));
        }
        *u_out = u;
        return HH_OK;
    }

    // The passes of the persistent HSS loop (hssp.cu) with the buffers hss_loop uses for the same
    // cycle: level 0 x1 in xa[0] and u in xb[0], level l's pre-smoothed x in xa[l] and its
    // post-smoothed x in xb[l], right sides in b[l], the coarsest result in xa[L - 1].
    void loop_plan(hh::HssLoop2<T>* P) {
        const int L = p->o.levels;
        std::memset((void*)P, 0, sizeof(*P));
        P->levels = L;
        P->nsteps = p->max_nhss;
        P->nb = p->nb;
        P->nu_coarse = p->o.nu_coarse;
        auto geo = [&](hh::MArgs<T>& a, int l) {
            a.h = T(p->lv[l].h);
            a.ih = T(1.0 / p->lv[l].h);
            a.hss_it = -1;
        };
        auto X = [&](std::vector<void*>& v, int l) { return (V2*)v[l]; };
        hh::MArgs<T> a = margs2(0, R_AR);
        geo(a, 0);
        a.x = X(H->xb, 0);
        a.z = (const V2*)H->r_lo;
        a.y = (V2*)H->rhs;
        a.y2 = X(H->xa, 0);
        a.yc = X(H->b, 1);
        a.use_pc_ab = 1;
        P->pre[0] = a;
        a.x = nullptr;
        a.xzero = 1;
        P->first = a;
        const int nn0 = p->lv[0].n + 1;
        P->pre_strips[0] = (nn0 + 23) / 24;
        P->pre_chunks[0] = p->lv[0].n / 2 + 1;
        for (int l = 1; l < L - 1; ++l) {
            hh::MArgs<T> q = margs2(l, R_AL);
            geo(q, l);
            q.z = X(H->b, l);
            q.y = X(H->xa, l);
            q.yc = X(H->b, l + 1);
            P->pre[l] = q;
            P->pre_strips[l] = (p->lv[l].nn + 25) / 26;
            P->pre_chunks[l] = p->lv[l].n / 2 + 1;
        }
        hh::MArgs<T> c = margs(L - 1, R_AL);
        geo(c, L - 1);
        c.z = X(H->b, L - 1);
        c.y = X(H->xa, L - 1);
        P->coarse = c;
        P->coarse_rows = std::max(1, (p->lv[L - 1].nn + 31) / 32);
        while (P->coarse_rows > 1 &&
               hh::hss_loop2_smem<T>(p->lv[L - 1], p->o.nu_coarse, P->coarse_rows) > hh::kLoopSmemMax)
            --P->coarse_rows;
        for (int l = L - 2; l >= 0; --l) {
            hh::MArgs<T> q = margs2(l, R_AL);
            geo(q, l);
            q.x = X(H->xa, l);
            q.ec = l == L - 2 ? X(H->xa, L - 1) : X(H->xb, l + 1);
            q.z = l == 0 ? (const V2*)H->rhs : X(H->b, l);
            q.y = X(H->xb, l);
            P->post[l] = q;
            P->post_strips[l] = (p->lv[l].nn + 27) / 28;
            P->post_chunks[l] = (p->lv[l].nn + 1) / 2;
        }
        P->count = p->d_sync;
        P->status = (int*)(p->d_sync + 1);
        P->spin_limit = p->o.sync_spin_limit > 0 ? (unsigned long long)p->o.sync_spin_limit : 4194304ULL;
    }

    // The HSS loop of Def. 4.1 on r_lo (already in this precision).  src[b] receives the
    // buffer that holds problem b's result (its loop may end before the others').
    hh_status hss_loop(std::vector<V2*>* src) {
        // the GMRES smoother's first step needs the right side whole: no fused first sweep
        const bool fuse = !gm() && p->o.nu_pre >= 1 && !(p->o.levels == 1 && p->o.nu_coarse == 0);
        const bool two = fuse && fused2(0) && (p->o.levels > 1 ? p->o.nu_pre : p->o.nu_coarse) >= 2;
        std::vector<V2*> after(p->max_nhss, nullptr);
        V2* u = nullptr;
        for (int it = 0; it < p->max_nhss; ++it) {
            hss_it = it;
            if (fuse) {
                // the first pre-smoothing sweep of the fine level is fused with the right side
                V2* x1 = (u == (V2*)H->xa[0]) ? (V2*)H->xb[0] : (V2*)H->xa[0];
                if (two && fused_rr(0)) {
                    HH_TRY(hss_first2_rr(u, (const V2*)H->r_lo, (V2*)H->rhs, x1, (V2*)H->b[1]));
                    HH_TRY(mg_solve((const V2*)H->rhs, x1, &u, 2, true));
                } else if (two) {
                    HH_TRY(hss_first2(u, (const V2*)H->r_lo, (V2*)H->rhs, x1));
                    HH_TRY(mg_solve((const V2*)H->rhs, x1, &u, 2));
                } else {
                    HH_TRY(hss_first(u, (const V2*)H->r_lo, (V2*)H->rhs, x1));
                    HH_TRY(mg_solve((const V2*)H->rhs, x1, &u));
                }
            } else {
                HH_TRY(hss_rhs(u, (const V2*)H->r_lo, (V2*)H->rhs));
                HH_TRY(mg_solve((const V2*)H->rhs, nullptr, &u));
            }
            after[it] = u;
        }
        hss_it = -1;
        // problems with no HSS iteration (theta such that ceil(k^theta) = 0) get u = 0
        V2* zero = (V2*)H->cres;
        bool need_zero = false;
        src->assign(p->nb, nullptr);
        for (int b = 0; b < p->nb; ++b) {
            if (p->nhss[b] > 0) {
                (*src)[b] = after[p->nhss[b] - 1] + (long long)b * Nl(0);
            } else {
                (*src)[b] = zero + (long long)b * Nl(0);
                need_zero = true;
            }
        }
        if (need_zero) HH_CUDA(cudaMemsetAsync(zero, 0, (size_t)Nl(0) * p->nb * sizeof(V2), s));
        return HH_OK;
    }
};

template <typename T>
MG<T> make_mg(hh_problem* p, int prec, cudaStream_t s) {
    MG<T> m;
    m.p = p;
    m.H = &p->hier[prec];
    m.s = s;
    m.omega = T(p->o.omega);
    return m;
}

template <typename T>
hh_status run_hss(MG<T>& m, std::vector<hh::vec2<T>*>* src) {
    if (!m.p->mixed) return m.hss_loop(src);
    hh::vec2<T>* u;
    HH_TRY(m.mixed_hss_loop(&u));
    src->assign(1, u);
    return HH_OK;
}

template <typename T>
hh_status record_hss(hh_problem* p, int prec) {
    MG<T> m = make_mg<T>(p, prec, p->s);
    std::vector<hh::vec2<T>*> src;
    HH_TRY(run_hss<T>(m, &src));
    Hier& H = p->hier[prec];
    // the pointer table is read by the gather kernel after the loop (constant per problem)
    static_assert(sizeof(void*) == sizeof(hh::vec2<T>*), "pointer size");
    HH_CUDA(cudaMemcpyAsync(H.usrc, src.data(), sizeof(void*) * p->nb, cudaMemcpyHostToDevice, p->s));
    return HH_OK;
}

// Whether the whole HSS loop runs as one cooperative kernel (hssp.cu): 2D primal problems with
// V(2,2) scaled-Jacobi cycles, one per HSS step, on 2..kPMaxLevels levels; automatically only
// while the fused two-sweep passes are used (levels of at most 600000 nodes).
bool persistent_loop(const hh_problem* p) {
    const hh_options& o = p->o;
    if (o.persistent == 0 || p->grid.dim != 2 || p->mixed) return false;
    if (o.smoother != HH_SMOOTH_JACOBI || o.cycle_gamma != 1 || o.cycles_per_hss != 1) return false;
    if (o.nu_pre != 2 || o.nu_post != 2 || o.levels < 2 || o.levels > hh::kPMaxLevels) return false;
    return o.persistent == 2 || p->lv[0].N * p->nb <= 600000;
}

// Launch the persistent HSS loop; *used = false (and nothing launched) when its grid does not
// fit the device, so that the caller runs the passes as separate kernels instead.
template <typename T>
hh_status launch_loop(hh_problem* p, int prec, bool* used) {
    Hier& H = p->hier[prec];
    *used = false;
    if (H.loop_unfit) return HH_OK;
    if (H.loop.empty()) {
        MG<T> m = make_mg<T>(p, prec, p->s);
        H.loop.resize(sizeof(hh::HssLoop2<T>));
        m.loop_plan(reinterpret_cast<hh::HssLoop2<T>*>(H.loop.data()));
        const auto* P = reinterpret_cast<const hh::HssLoop2<T>*>(H.loop.data());
        H.loop_smem = hh::hss_loop2_smem<T>(p->lv[p->o.levels - 1], p->o.nu_coarse, P->coarse_rows);
        H.loop_ctas = hh::hss_loop2_ctas<T>(p->nb > 1, H.loop_smem);
        if (H.loop_ctas < 1) {
            H.loop.clear();
            H.loop_unfit = true;
            return HH_OK;
        }
        // the result pointer table of the gather (u in xb[0]; problems without HSS steps: 0)
        std::vector<hh::vec2<T>*> src(p->nb);
        const long long N0 = p->lv[0].N;
        bool need_zero = false;
        for (int b = 0; b < p->nb; ++b) {
            src[b] = (p->nhss[b] > 0 ? (hh::vec2<T>*)H.xb[0] : (hh::vec2<T>*)H.cres) + (long long)b * N0;
            need_zero = need_zero || p->nhss[b] == 0;
        }
        if (need_zero) HH_CUDA(cudaMemsetAsync(H.cres, 0, (size_t)N0 * p->nb * sizeof(hh::vec2<T>), p->s));
        HH_CUDA(cudaMemcpyAsync(H.usrc, src.data(), sizeof(void*) * p->nb, cudaMemcpyHostToDevice, p->s));
        HH_CUDA(cudaStreamSynchronize(p->s));
    }
    HH_CUDA(hh::launch_hss_loop2<T>(*reinterpret_cast<const hh::HssLoop2<T>*>(H.loop.data()), H.loop_ctas,
                                     H.loop_smem, p->s));
    *used = true;
    return HH_OK;
}

// z (c128, nb x N) = shifted-HSS preconditioner of r (c128), on the problem stream, for the
// active problems.
hh_status precondition_async(hh_problem* p, const double2* r, double2* z) {
    const int prec = p->o.precision;
    HH_TRY(ensure_hier(p, prec));
    Hier& H = p->hier[prec];
    const long long N = p->lv[0].N;
    const long long NT = p->N * p->nb;  // (sigma and) nodes
    if (prec == HH_C64) {
        HH_LAUNCH(hh::launch_cast_d2f(r, (float2*)H.r_lo, NT, p->s));
    } else {
        HH_CUDA(cudaMemcpyAsync(H.r_lo, r, (size_t)NT * 16, cudaMemcpyDeviceToDevice, p->s));
    }
    bool looped = false;
    if (persistent_loop(p))
        HH_TRY(prec == HH_C64 ? launch_loop<float>(p, prec, &looped) : launch_loop<double>(p, prec, &looped));
    if (looped) {
    } else if (p->o.use_graphs) {
        if (!H.graph) {
            // the pointer table of the results is written once, outside the graph
            cudaGraph_t g;
            const long long k0 = hh::g_kernel_launches;
            HH_CUDA(cudaStreamBeginCapture(p->s, cudaStreamCaptureModeThreadLocal));
            MG<float> mf = make_mg<float>(p, prec, p->s);
            MG<double> md = make_mg<double>(p, prec, p->s);
            std::vector<float2*> sf;
            std::vector<double2*> sd;
            hh_status st = prec == HH_C64 ? run_hss<float>(mf, &sf) : run_hss<double>(md, &sd);
            cudaError_t ec = cudaStreamEndCapture(p->s, &g);
            if (st != HH_OK) {
                if (ec == cudaSuccess) cudaGraphDestroy(g);
                return st;
            }
            HH_CUDA(ec);
            cudaError_t ei = cudaGraphInstantiate(&H.graph, g, 0);
            cudaGraphDestroy(g);
            HH_CUDA(ei);
            H.graph_kernels = hh::g_kernel_launches - k0;
            hh::g_kernel_launches = k0;
            const void* srcp = prec == HH_C64 ? (const void*)sf.data() : (const void*)sd.data();
            HH_CUDA(cudaMemcpyAsync(H.usrc, srcp, sizeof(void*) * p->nb, cudaMemcpyHostToDevice, p->s));
            HH_CUDA(cudaStreamSynchronize(p->s));
        }
        HH_CUDA(cudaGraphLaunch(H.graph, p->s));
        hh::g_kernel_launches += H.graph_kernels;
    } else {
        if (prec == HH_C64) {
            HH_TRY(record_hss<float>(p, prec));
        } else {
            HH_TRY(record_hss<double>(p, prec));
        }
    }
    double2* zu = z + p->ns;  // mixed (one problem): sigma, then the nodes
    if (prec == HH_C64) {
        if (p->mixed)
            HH_LAUNCH(hh::launch_gather_c128<float>((const float2* const*)H.ssrc, z, p->ns, 1, nullptr, p->s));
        HH_LAUNCH(hh::launch_gather_c128<float>((const float2* const*)H.usrc, zu, N, p->nb, active_flags(p), p->s));
    } else {
        if (p->mixed)
            HH_LAUNCH(hh::launch_gather_c128<double>((const double2* const*)H.ssrc, z, p->ns, 1, nullptr, p->s));
        HH_LAUNCH(hh::launch_gather_c128<double>((const double2* const*)H.usrc, zu, N, p->nb, active_flags(p), p->s));
    }
    return HH_OK;
}

// ------------------------------------------------------------------ FP64 helpers
// y = alpha (op x) + beta z  (z == nullptr: y = op x) on level l for every active problem
template <typename T>
hh_status op_axpby(hh_problem* p, int l, int role, const hh::vec2<T>* x, const hh::vec2<T>* z, hh::vec2<T>* y,
                   Cx<T> alpha, Cx<T> beta, cudaStream_t st) {
    const int prec = sizeof(T) == 4 ? HH_C64 : HH_C128;
    HH_TRY(ensure_tables(p));
    MG<T> m = make_mg<T>(p, prec, st);
    hh::MArgs<T> a = m.margs(l, role);
    a.x = x;
    a.z = z;
    a.y = y;
    a.alpha = alpha;
    a.beta = beta;
    HH_LAUNCH(m.march(z ? hh::M_AXPBY : hh::M_APPLY, a));
    return HH_OK;
}

// Mixed system (Sec. 2): y = sgn A_delta x + b, x = (sigma, u), b = (b_s, b_u) or none:
//   sigma-rows: M_s (sgn (delta - i k) sigma - sgn D u) + b_s;
//   u-rows:     sgn ((delta - i k) M + M_Gamma) u + b_u + sgn G^T sigma.
hh_status mixed_system(hh_problem* p, const double2* x, const double2* b, double sgn, double2* y) {
    const zc z(p->delta[0], -p->k[0]);
    hh::MixArgs<double> a{};
    a.g = p->lv[0];
    a.sig = x;
    a.u = x + p->ns;
    a.z = b;
    a.y = y;
    a.cs = Cx<double>{sgn * z.real(), sgn * z.imag()};
    a.cd = Cx<double>{-sgn, 0};
    a.cz = Cx<double>{b ? 1.0 : 0.0, 0};
    a.mass_out = 1;
    HH_LAUNCH(hh::launch_mix_sigma<double>(a, p->s));
    HH_TRY(op_axpby<double>(p, 0, R_MIXU, x + p->ns, b ? b + p->ns : nullptr, y + p->ns, Cx<double>{sgn, 0},
                            Cx<double>{b ? 1.0 : 0.0, 0}, p->s));
    hh::MixArgs<double> d{};
    d.g = p->lv[0];
    d.sig = x;
    d.y = y + p->ns;
    d.cs = Cx<double>{sgn, 0};
    HH_LAUNCH(hh::launch_mix_div<double>(d, p->s));
    return HH_OK;
}

hh_status apply_B(hh_problem* p, const double2* x, double2* y) {
    if (p->mixed) return mixed_system(p, x, nullptr, 1.0, y);
    return op_axpby<double>(p, 0, R_B, x, nullptr, y, Cx<double>{1, 0}, Cx<double>{0, 0}, p->s);
}

// r = bvec - B x
hh_status residual_B(hh_problem* p, const double2* x, double2* r) {
    if (p->mixed) return mixed_system(p, x, p->bvec, -1.0, r);
    return op_axpby<double>(p, 0, R_B, x, p->bvec, r, Cx<double>{-1, 0}, Cx<double>{1, 0}, p->s);
}

// ------------------------------------------------------------------ autotuner
// Every tile shape gives the same result bit for bit (each node's arithmetic does not depend
// on the tiling); only the time differs.  Measured choices are kept per process, keyed by
// (device, dim, level grid n, batch size, precision, mode), so that problems of the same shape
// reuse them.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, std::array<int, 2>> g_tune_cache;

// Candidate {rows, form} of a stencil kernel (form: 1 one tile per warp, 2 persistent); for
// the coarsest-level solve, {cluster size, 0}.
std::vector<std::array<int, 2>> tile_candidates(const GridDesc& g, int prec, int mode) {
    const int dim = g.dim;
    std::vector<std::array<int, 2>> c;
    if (mode == kCoarseMode) {
        for (int cs : {16, 8, 4, 2, 1}) {
            const bool ok = prec == HH_C64 ? hh::coarse_cluster_ok<float>(g, cs) : hh::coarse_cluster_ok<double>(g, cs);
            if (ok) c.push_back({cs, 0});
        }
        return c;
    }
    if (mode == hh::M_PROLONG_JACOBI2 || mode == hh::M_HSS_FIRST2) {
        if (dim == 2) c = {{2, 1}, {4, 1}};
        return c;
    }
    if (mode == hh::M_JACOBI2_ZERO_RR || mode == hh::M_HSS_FIRST2_RR) {
        if (dim == 2) c = {{1, 1}, {2, 1}};  // coarse rows per tile
        return c;
    }
    if (dim == 2) {
        std::vector<int> rows = {2, 4};
        if (prec == HH_C64 && mode != hh::M_RESID_RESTRICT) rows.push_back(8);
        const bool persist_ok = mode != hh::M_PROLONG_JACOBI;
        for (int r : rows) {
            c.push_back({r, 1});
            if (persist_ok) c.push_back({r, 2});
        }
    } else if (prec == HH_C64) {
        c = {{2, 0}, {4, 0}, {8, 0}};
    }
    return c;
}

// Average device time of one launch of `mode` on level l with tile shape cand (scratch buffers).
template <typename T>
hh_status time_shape(hh_problem* p, int l, int mode, const std::array<int, 2>& cand, float* ms) {
    using V2 = hh::vec2<T>;
    const int prec = sizeof(T) == 4 ? HH_C64 : HH_C128;
    MG<T> m = make_mg<T>(p, prec, p->s);
    const bool fgm = prec == HH_C128 && l == 0 && (mode == hh::M_APPLY || mode == hh::M_AXPBY) &&
                     !p->hier[HH_C128].ready;
    const bool hssm = mode == hh::M_HSS_FIRST || mode == hh::M_HSS_FIRST2 || mode == hh::M_HSS_FIRST2_RR;
    const int role = hssm ? R_AR : (mode == hh::M_APPLY ? R_B : R_AL);
    const bool two = mode == hh::M_PROLONG_JACOBI2 || mode == hh::M_HSS_FIRST2 || mode == hh::M_JACOBI2_ZERO_RR ||
                     mode == hh::M_HSS_FIRST2_RR;
    hh::MArgs<T> a = two ? m.margs2(l, role) : m.margs(l, role);
    if (fgm) {
        // the FP64 outer operator: Krylov buffers stand in for the hierarchy
        a.x = (const V2*)p->V;
        a.z = (const V2*)p->r;
        a.y = (V2*)(p->V + (long long)p->nb * p->N);
    } else {
        Hier& H = p->hier[prec];
        a.x = (const V2*)H.xa[l];
        a.z = (const V2*)H.b[l];
        a.y = (V2*)H.xb[l];
        a.y2 = (V2*)H.t[l];
        if (l + 1 < p->o.levels) a.ec = (const V2*)H.xa[l + 1];
        if (mode == hh::M_RESID_RESTRICT) a.y = (V2*)H.t[l + 1];
        if (mode == hh::M_JACOBI2_ZERO_RR || mode == hh::M_HSS_FIRST2_RR) a.yc = (V2*)H.t[l + 1];
    }
    a.use_pc_ab = hssm;
    a.alpha = Cx<T>{-1, 0};
    a.beta = Cx<T>{1, 0};
    a.tile_rows = cand[0];
    a.tile_form = cand[1];
    if (mode == kCoarseMode) a.y = (V2*)p->hier[prec].xa[l];
    auto launch = [&]() {
        if (mode == kCoarseMode) return hh::launch_coarse_solve<T>(a, p->o.nu_coarse, p->s);
        if (mode == hh::M_JACOBI2_ZERO_RR || mode == hh::M_HSS_FIRST2_RR) return hh::launch_march2rr<T>(mode, a, p->s);
        return m.d2() ? hh::launch_march2<T>(mode, a, p->s) : hh::launch_march3<T>(mode, a, p->s);
    };
    cudaEvent_t e0, e1;
    HH_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(HH_ERR_CUDA, "event creation failed");
    }
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < 2 && err == cudaSuccess; ++i) err = launch();
    const int reps = 5;
    if (err == cudaSuccess) err = cudaEventRecord(e0, p->s);
    for (int i = 0; i < reps && err == cudaSuccess; ++i) err = launch();
    if (err == cudaSuccess) err = cudaEventRecord(e1, p->s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    HH_CUDA(err);
    *ms = t / reps;
    return HH_OK;
}

// Pick the fastest tile shape of every (level, mode) the solver runs in precision prec, and of
// the FP64 outer operator on level 0.
hh_status autotune(hh_problem* p, int prec) {
    HH_TRY(ensure_hier(p, prec));
    const int L = p->o.levels;
    for (int q = 0; q < 2; ++q)
        if (p->tune[q].empty()) p->tune[q].assign(L, {});
    std::vector<std::tuple<int, int, int>> work;  // (precision, level, mode)
    for (int l = 0; l < L; ++l)
        for (int mode = 0; mode < kModes; ++mode) {
            const bool coarse_cluster = p->o.nu_coarse >= 1 && p->lv[l].N <= p->o.coarse_cluster_nodes &&
                                        (prec == HH_C64 ? hh::coarse_fits<float>(p->lv[l])
                                                        : hh::coarse_fits<double>(p->lv[l]));
            if (mode == kCoarseMode && (l != L - 1 || !coarse_cluster)) continue;
            const bool needs_coarser = mode == hh::M_PROLONG_JACOBI || mode == hh::M_RESID_RESTRICT ||
                                       mode == hh::M_PROLONG_JACOBI2 || mode == hh::M_JACOBI2_ZERO_RR ||
                                       mode == hh::M_HSS_FIRST2_RR;
            if (needs_coarser && l == L - 1) continue;
            if ((mode == hh::M_RESID_RESTRICT || mode == hh::M_PROLONG_JACOBI2 || mode == hh::M_HSS_FIRST2 ||
                 mode == hh::M_JACOBI2_ZERO_RR || mode == hh::M_HSS_FIRST2_RR) &&
                p->grid.dim == 3)
                continue;
            if ((mode == hh::M_HSS_FIRST || mode == hh::M_HSS_FIRST2 || mode == hh::M_HSS_FIRST2_RR) && l != 0) continue;
            work.emplace_back(prec, l, mode);
        }
    if (prec == HH_C64) {
        work.emplace_back(HH_C128, 0, (int)hh::M_APPLY);
        work.emplace_back(HH_C128, 0, (int)hh::M_AXPBY);
    }
    const int nb = p->nb;
    for (auto& [q, l, mode] : work) {
        const auto key = std::make_tuple(p->device, p->grid.dim, p->lv[l].n, nb, q, mode);
        std::array<int, 2> best{0, 0};
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) best = it->second;
        }
        if (best[0] == 0) {
            const auto cands = tile_candidates(p->lv[l], q, mode);
            if (cands.size() < 2) continue;
            float tbest = 0.f;
            for (const auto& c : cands) {
                float ms = 0.f;
                HH_TRY(q == HH_C64 ? time_shape<float>(p, l, mode, c, &ms) : time_shape<double>(p, l, mode, c, &ms));
                if (best[0] == 0 || ms < tbest) {
                    best = c;
                    tbest = ms;
                }
            }
            std::lock_guard<std::mutex> g(g_tune_mu);
            g_tune_cache[key] = best;
        }
        p->tune[q][l][mode] = best;
    }
    // captured preconditioner graphs hold the old shapes
    for (int q = 0; q < 2; ++q)
        if (p->hier[q].graph) {
            cudaGraphExecDestroy(p->hier[q].graph);
            p->hier[q].graph = nullptr;
        }
    return HH_OK;
}

int hstride(const hh_problem* p) { return 2 * (p->o.restart + 1) + 1; }

// ||v_b||^2 into hbuf[b][slot] (device) for every active problem (v_b = v + b N)
hh_status norm2_dev(hh_problem* p, const double2* v, int slot) {
    const hh::KBatch kb{p->nb, p->N, p->N, hstride(p), active_flags(p)};
    HH_CUDA(hh::launch_multidot(v, 0, 1, v, p->N, p->partials, p->hbuf + slot, kb, p->s));
    return HH_OK;
}

// The status word of the persistent HSS loop (copied with every fetch): a non-zero value is
// an error a CTA recorded; it is cleared here and returned.
hh_status check_sync(hh_problem* p) {
    const int st = *p->h_sync;
    if (st == 0) return HH_OK;
    *p->h_sync = 0;
    HH_CUDA(cudaMemsetAsync(p->d_sync + 1, 0, sizeof(int), p->s));
    HH_CUDA(cudaStreamSynchronize(p->s));
    return fail((hh_status)st, st == HH_ERR_TIMEOUT ? "a grid-wide barrier wait of the persistent HSS loop ran out"
                                                    : "the persistent HSS loop reported an error");
}

hh_status fetch(hh_problem* p) {
    HH_CUDA(cudaMemcpyAsync(p->h_host, p->hbuf, (size_t)p->nb * hstride(p) * sizeof(double2), cudaMemcpyDeviceToHost,
                            p->s));
    HH_CUDA(cudaMemcpyAsync(p->h_sync, p->d_sync + 1, sizeof(int), cudaMemcpyDeviceToHost, p->s));
    HH_CUDA(cudaStreamSynchronize(p->s));
    return check_sync(p);
}

bool finite(double v) { return std::isfinite(v); }

// Column j of the Hessenberg matrix (H[i] for i <= j + 1, stored with stride 1): apply the j
// earlier Givens rotations, compute rotation j that zeroes H[j + 1] and apply it to H and to the
// rotated right side g.  Shared by every FGMRES driver, so that their arithmetic is one code.
void givens_column(zc* H, double* cs, zc* sn, zc* g, int j) {
    for (int i = 0; i < j; ++i) {
        const zc t = cs[i] * H[i] + sn[i] * H[i + 1];
        H[i + 1] = -std::conj(sn[i]) * H[i] + cs[i] * H[i + 1];
        H[i] = t;
    }
    const zc h1 = H[j], h2 = H[j + 1];
    const double den = std::hypot(std::abs(h1), std::abs(h2));
    if (std::abs(h1) == 0.0) {
        cs[j] = 0.0;
        sn[j] = 1.0;
    } else {
        cs[j] = std::abs(h1) / den;
        sn[j] = (h1 / std::abs(h1)) * std::conj(h2) / den;
    }
    H[j] = cs[j] * h1 + sn[j] * h2;
    H[j + 1] = 0.0;
    g[j + 1] = -std::conj(sn[j]) * g[j];
    g[j] = cs[j] * g[j];
}

// y (m entries) = R^{-1} g over the first jend columns (R: the rotated Hessenberg matrix, column j
// at Hm + j * (m + 1)), zero beyond; false if a value is not finite.
bool back_substitute(const zc* Hm, int m, const zc* g, int jend, zc* y) {
    std::fill(y, y + m, zc(0));
    for (int i = jend - 1; i >= 0; --i) {
        zc acc = g[i];
        for (int c = i + 1; c < jend; ++c) acc -= Hm[(size_t)c * (m + 1) + i] * y[c];
        y[i] = acc / Hm[(size_t)i * (m + 1) + i];
        if (!finite(y[i].real()) || !finite(y[i].imag())) return false;
    }
    return true;
}

// Flexible GMRES(m) with classical Gram-Schmidt applied twice (CGS2) and Givens rotations,
// the nb problems in lockstep: a problem that converges leaves the launches at once.
hh_status fgmres(hh_problem* p, double tol, hh_info* info) {
    const int m = p->o.restart, nb = p->nb, hs = hstride(p);
    const long long N = p->N;
    const int nrm = 2 * (m + 1);
    auto H = [&](int b, int i) -> double2& { return p->h_host[(size_t)b * hs + i]; };
    std::vector<char> solving(nb, 1), in_cycle(nb, 0), ran(nb, 0);
    HH_TRY(set_active(p, nullptr));
    HH_TRY(norm2_dev(p, p->bvec, nrm));
    HH_TRY(fetch(p));
    std::vector<double> bnorm(nb), beta(nb), rel(nb);
    for (int b = 0; b < nb; ++b) {
        bnorm[b] = std::sqrt(H(b, nrm).x);
        if (!finite(bnorm[b])) return fail(HH_ERR_NONFINITE, "right-hand side " + std::to_string(b) + " is not finite");
    }
    HH_TRY(residual_B(p, p->x, p->r));
    HH_TRY(norm2_dev(p, p->r, nrm));
    HH_TRY(fetch(p));
    for (int b = 0; b < nb; ++b) {
        beta[b] = std::sqrt(H(b, nrm).x);
        if (!finite(beta[b])) return fail(HH_ERR_NONFINITE, "initial residual is not finite");
        rel[b] = bnorm[b] > 0 ? beta[b] / bnorm[b] : 0.0;
        info[b].outer_its = 0;
        if (bnorm[b] == 0.0 || rel[b] <= tol || p->o.max_outer == 0) solving[b] = 0;
    }
    // zero right sides: u = 0 exactly
    for (int b = 0; b < nb; ++b)
        if (bnorm[b] == 0.0) HH_CUDA(cudaMemsetAsync(p->x + (long long)b * N, 0, (size_t)N * 16, p->s));
    std::vector<zc> Hm((size_t)nb * (m + 1) * m), g((size_t)nb * (m + 1)), sn((size_t)nb * m), y((size_t)nb * m);
    std::vector<double> cs((size_t)nb * m);
    // true residual at the end of every restart cycle, per problem (stall detection)
    std::vector<std::vector<double>> cycle_rel(nb);
    for (int b = 0; b < nb; ++b) cycle_rel[b].push_back(rel[b]);
    std::vector<int> jend(nb, 0);
    auto Hc = [&](int b, int i, int j) -> zc& { return Hm[((size_t)b * m + j) * (m + 1) + i]; };
    // Krylov layout [vector][problem][node]: basis vector j of the whole batch is one block
    const long long blk = (long long)nb * N;
    while (std::any_of(solving.begin(), solving.end(), [](char c) { return c != 0; })) {
        in_cycle = solving;
        std::fill(jend.begin(), jend.end(), 0);
        HH_TRY(set_active(p, &in_cycle));
        // V_0 = r / beta (the residual norms are still in hbuf)
        HH_CUDA(cudaMemcpyAsync(p->V, p->r, (size_t)blk * 16, cudaMemcpyDeviceToDevice, p->s));
        HH_CUDA(hh::launch_scale_by_rnorm(p->V, p->hbuf + nrm, N, hh::KBatch{nb, N, N, hs, active_flags(p)}, p->s));
        for (int b = 0; b < nb; ++b) {
            std::fill(g.begin() + (size_t)b * (m + 1), g.begin() + (size_t)(b + 1) * (m + 1), zc(0));
            g[(size_t)b * (m + 1)] = beta[b];
        }
        for (int j = 0; j < m; ++j) {
            double2* vj = p->V + (long long)j * blk;
            double2* zj = p->Z + (long long)j * blk;
            double2* w = p->V + (long long)(j + 1) * blk;
            HH_TRY(precondition_async(p, vj, zj));
            for (int b = 0; b < nb; ++b)
                if (in_cycle[b]) {
                    info[b].hss_its += p->nhss[b];
                    info[b].vcycles += (long long)p->nhss[b] * p->o.cycles_per_hss;
                }
            HH_TRY(apply_B(p, zj, w));
            // CGS2: two passes of h = V^H w, w -= V h
            const hh::KBatch kb{nb, N, N, hs, active_flags(p)};
            double2* hA = p->hbuf;
            double2* hB = p->hbuf + (m + 1);
            HH_CUDA(hh::launch_multidot(p->V, blk, j + 1, w, N, p->partials, hA, kb, p->s));
            HH_CUDA(hh::launch_multi_axpy(w, p->V, blk, j + 1, hA, -1.0, N, kb, p->s));
            HH_CUDA(hh::launch_multidot(p->V, blk, j + 1, w, N, p->partials, hB, kb, p->s));
            HH_CUDA(hh::launch_multi_axpy(w, p->V, blk, j + 1, hB, -1.0, N, kb, p->s));
            HH_CUDA(hh::launch_multidot(w, 0, 1, w, N, p->partials, p->hbuf + nrm, kb, p->s));
            HH_CUDA(hh::launch_scale_by_rnorm(w, p->hbuf + nrm, N, kb, p->s));
            HH_TRY(fetch(p));
            bool changed = false;
            for (int b = 0; b < nb; ++b) {
                if (!in_cycle[b]) continue;
                for (int i = 0; i <= j; ++i)
                    Hc(b, i, j) = zc(H(b, i).x + H(b, m + 1 + i).x, H(b, i).y + H(b, m + 1 + i).y);
                const double hn = std::sqrt(H(b, nrm).x);
                if (!finite(hn)) return fail(HH_ERR_NONFINITE, "Arnoldi produced a non-finite value");
                Hc(b, j + 1, j) = hn;
                zc* gb = &g[(size_t)b * (m + 1)];
                givens_column(&Hc(b, 0, j), &cs[(size_t)b * m], &sn[(size_t)b * m], gb, j);
                info[b].outer_its += 1;
                jend[b] = j + 1;
                if (std::abs(gb[j + 1]) / bnorm[b] <= tol || info[b].outer_its >= p->o.max_outer || hn == 0.0) {
                    in_cycle[b] = 0;
                    changed = true;
                }
            }
            if (!std::any_of(in_cycle.begin(), in_cycle.end(), [](char c) { return c != 0; })) break;
            if (changed) HH_TRY(set_active(p, &in_cycle));
        }
        // x += Z y for every problem that ran this cycle
        int jmax = 0;
        for (int b = 0; b < nb; ++b) {
            ran[b] = jend[b] > 0;
            jmax = std::max(jmax, jend[b]);
            zc* yb = &y[(size_t)b * m];
            if (!back_substitute(&Hc(b, 0, 0), m, &g[(size_t)b * (m + 1)], jend[b], yb))
                return fail(HH_ERR_NONFINITE, "least-squares update is not finite");
            for (int i = 0; i < m; ++i) p->h_host[(size_t)b * m + i] = make_double2(yb[i].real(), yb[i].imag());
        }
        HH_CUDA(cudaMemcpyAsync(p->ybuf, p->h_host, (size_t)nb * m * 16, cudaMemcpyHostToDevice, p->s));
        HH_TRY(set_active(p, &ran));  // also waits for the copy above
        HH_CUDA(hh::launch_multi_axpy(p->x, p->Z, blk, jmax, p->ybuf, 1.0, N, hh::KBatch{nb, N, N, m, active_flags(p)},
                                      p->s));
        HH_TRY(residual_B(p, p->x, p->r));
        HH_TRY(norm2_dev(p, p->r, nrm));
        HH_TRY(fetch(p));
        for (int b = 0; b < nb; ++b) {
            if (!ran[b]) continue;
            beta[b] = std::sqrt(H(b, nrm).x);
            if (!finite(beta[b])) return fail(HH_ERR_NONFINITE, "residual is not finite");
            rel[b] = beta[b] / bnorm[b];
            if (rel[b] <= tol || info[b].outer_its >= p->o.max_outer) solving[b] = 0;
            // stalled: stall_cycles restart cycles did not halve the true residual
            cycle_rel[b].push_back(rel[b]);
            const int sc = p->o.stall_cycles, nc = (int)cycle_rel[b].size() - 1;
            if (sc > 0 && nc >= sc && rel[b] > 0.5 * cycle_rel[b][nc - sc]) solving[b] = 0;
        }
    }
    HH_TRY(set_active(p, nullptr));
    bool all = true;
    for (int b = 0; b < nb; ++b) {
        info[b].rel_residual = rel[b];
        all = all && rel[b] <= tol;
    }
    return all ? HH_OK : HH_NOT_CONVERGED;
}

// Preconditioned Richardson (the stationary iteration after Def. 4.1): u += P (b - B u)
// with the FP64 residual recomputed every step, the nb problems in lockstep; a problem
// leaves the launches when it converges or reaches max_outer.
hh_status richardson(hh_problem* p, double tol, hh_info* info) {
    const int nb = p->nb, hs = hstride(p), nrm = 2 * (p->o.restart + 1);
    const long long N = p->N;
    std::vector<char> solving(nb, 1);
    std::vector<double> bnorm(nb), rel(nb);
    HH_TRY(set_active(p, nullptr));
    HH_TRY(norm2_dev(p, p->bvec, nrm));
    HH_TRY(fetch(p));
    for (int b = 0; b < nb; ++b) {
        bnorm[b] = std::sqrt(p->h_host[(size_t)b * hs + nrm].x);
        if (!finite(bnorm[b])) return fail(HH_ERR_NONFINITE, "right-hand side " + std::to_string(b) + " is not finite");
    }
    HH_TRY(residual_B(p, p->x, p->r));
    HH_TRY(norm2_dev(p, p->r, nrm));
    HH_TRY(fetch(p));
    for (int b = 0; b < nb; ++b) {
        const double beta = std::sqrt(p->h_host[(size_t)b * hs + nrm].x);
        if (!finite(beta)) return fail(HH_ERR_NONFINITE, "initial residual is not finite");
        rel[b] = bnorm[b] > 0 ? beta / bnorm[b] : 0.0;
        info[b].outer_its = 0;
        if (bnorm[b] == 0.0 || rel[b] <= tol || p->o.max_outer == 0) solving[b] = 0;
    }
    for (int b = 0; b < nb; ++b)
        if (bnorm[b] == 0.0) HH_CUDA(cudaMemsetAsync(p->x + (long long)b * N, 0, (size_t)N * 16, p->s));
    const hh::Batch all{nb, N, 0, -1, nullptr, active_flags(p)};
    while (std::any_of(solving.begin(), solving.end(), [](char c) { return c != 0; })) {
        HH_TRY(set_active(p, &solving));
        HH_TRY(precondition_async(p, p->r, p->Z));
        HH_LAUNCH(hh::launch_add<double>(p->x, p->Z, N, all, p->s));
        HH_TRY(residual_B(p, p->x, p->r));
        HH_TRY(norm2_dev(p, p->r, nrm));
        HH_TRY(fetch(p));
        for (int b = 0; b < nb; ++b) {
            if (!solving[b]) continue;
            info[b].outer_its += 1;
            info[b].hss_its += p->nhss[b];
            info[b].vcycles += (long long)p->nhss[b] * p->o.cycles_per_hss;
            const double beta = std::sqrt(p->h_host[(size_t)b * hs + nrm].x);
            if (!finite(beta)) return fail(HH_ERR_NONFINITE, "Richardson residual is not finite");
            rel[b] = beta / bnorm[b];
            if (rel[b] <= tol || info[b].outer_its >= p->o.max_outer) solving[b] = 0;
        }
    }
    HH_TRY(set_active(p, nullptr));
    bool ok = true;
    for (int b = 0; b < nb; ++b) {
        info[b].rel_residual = rel[b];
        ok = ok && rel[b] <= tol;
    }
    return ok ? HH_OK : HH_NOT_CONVERGED;
}

}  // namespace

namespace {

hh_status validate_level(const hh_problem* p, int level, int need_coarser) {
    if (!p) return fail(HH_ERR_INVALID, "null problem");
    if (level < 0 || level >= p->o.levels - need_coarser) return fail(HH_ERR_INVALID, "level out of range");
    return HH_OK;
}

hh_status validate_prec(int prec) {
    if (prec != HH_C64 && prec != HH_C128) return fail(HH_ERR_INVALID, "precision must be HH_C128 or HH_C64");
    return HH_OK;
}

hh_status check_args(const hh_grid* grid, int nb, const double* k, const double* delta, const double* dh,
                     const int* bc, const hh_options* o) {
    if (!grid || !o) return fail(HH_ERR_INVALID, "null grid or options");
    if (grid->dim != 2 && grid->dim != 3) return fail(HH_ERR_INVALID, "dim must be 2 or 3");
    // problems index grid.z (2D) or share it with the planes of a 3D level
    if (nb < 1 || nb > 65535) return fail(HH_ERR_INVALID, "batch size must be in 1..65535");
    if (grid->dim == 3 && (long long)(grid->n + 1) * nb > 65535)
        return fail(HH_ERR_INVALID, "3D batch: (n + 1) * nb must not exceed 65535");
    if (!k || !delta || !dh) return fail(HH_ERR_INVALID, "null k, delta or delta_hat");
    for (int b = 0; b < nb; ++b)
        if (!(k[b] > 0) || !(delta[b] >= 0) || !(dh[b] > 0) || !std::isfinite(k[b]) || !std::isfinite(delta[b]) ||
            !std::isfinite(dh[b]))
            return fail(HH_ERR_INVALID, "need k > 0, delta >= 0, delta_hat > 0 (finite)");
    if (o->levels < 1 || o->levels > 16) return fail(HH_ERR_INVALID, "levels must be in 1..16");
    if (grid->n < 2 || grid->n > (1 << 20)) return fail(HH_ERR_INVALID, "n out of range");
    if (grid->n % (1 << (o->levels - 1)) != 0 || (grid->n >> (o->levels - 1)) < 1)
        return fail(HH_ERR_INVALID, "n must be divisible by 2^(levels-1)");
    if (o->nu_pre < 0 || o->nu_post < 0 || o->nu_coarse < 0 || o->cycles_per_hss < 1)
        return fail(HH_ERR_INVALID, "negative sweep count or cycles_per_hss < 1");
    if (o->restart < 1 || o->restart > 63) return fail(HH_ERR_INVALID, "restart must be in 1..63");
    if (o->max_outer < 0) return fail(HH_ERR_INVALID, "max_outer < 0");
    if (!(o->theta >= 0) || !(o->omega >= 0) || !(o->omega < 2))
        return fail(HH_ERR_INVALID, "theta >= 0 and 0 <= omega < 2 required");
    if (o->precision != HH_C64 && o->precision != HH_C128) return fail(HH_ERR_INVALID, "bad precision");
    if (o->coarse_cluster_nodes < 0) return fail(HH_ERR_INVALID, "coarse_cluster_nodes < 0");
    if (o->tile_rows != 0 && o->tile_rows != 2 && o->tile_rows != 4 && o->tile_rows != 8)
        return fail(HH_ERR_INVALID, "tile_rows must be 0, 2, 4 or 8");
    if (o->tile_form < 0 || o->tile_form > 2) return fail(HH_ERR_INVALID, "tile_form must be 0, 1 or 2");
    if (o->formulation != HH_FORM_PRIMAL && o->formulation != HH_FORM_MIXED)
        return fail(HH_ERR_INVALID, "formulation must be HH_FORM_PRIMAL or HH_FORM_MIXED");
    if (o->formulation == HH_FORM_MIXED && nb != 1) return fail(HH_ERR_INVALID, "mixed problems are not batched");
    if (o->smoother != HH_SMOOTH_JACOBI && o->smoother != HH_SMOOTH_GMRES)
        return fail(HH_ERR_INVALID, "smoother must be HH_SMOOTH_JACOBI or HH_SMOOTH_GMRES");
    if (o->smoother == HH_SMOOTH_GMRES &&
        (o->nu_pre > hh::kGsMaxIts || o->nu_post > hh::kGsMaxIts || o->nu_coarse > hh::kGsMaxIts))
        return fail(HH_ERR_INVALID, "the GMRES smoother takes at most 8 iterations per smoothing step");
    if (o->autotune != 0 && o->autotune != 1) return fail(HH_ERR_INVALID, "autotune must be 0 or 1");
    if (o->fuse_sweeps != 0 && o->fuse_sweeps != 1) return fail(HH_ERR_INVALID, "fuse_sweeps must be 0 or 1");
    if (o->cycle_gamma < 1 || o->cycle_gamma > 4) return fail(HH_ERR_INVALID, "cycle_gamma must be in 1..4");
    if (o->outer != HH_OUTER_FGMRES && o->outer != HH_OUTER_RICHARDSON)
        return fail(HH_ERR_INVALID, "outer must be HH_OUTER_FGMRES or HH_OUTER_RICHARDSON");
    if (o->persistent < 0 || o->persistent > 2) return fail(HH_ERR_INVALID, "persistent must be 0, 1 or 2");
    if (o->sync_spin_limit < 0) return fail(HH_ERR_INVALID, "sync_spin_limit < 0");
    if (o->stall_cycles < 0) return fail(HH_ERR_INVALID, "stall_cycles < 0");
    if (o->coarse_kernel < 0 || o->coarse_kernel > 2) return fail(HH_ERR_INVALID, "coarse_kernel must be 0, 1 or 2");
    if (!bc) return fail(HH_ERR_INVALID, "null bc");
    for (int s = 0; s < 2 * grid->dim; ++s)
        if (bc[s] != HH_BC_SOMMERFELD && bc[s] != HH_BC_DIRICHLET) return fail(HH_ERR_INVALID, "bad boundary tag");
    return HH_OK;
}

hh_status solve_core(hh_problem* p, double tol, hh_info* info) {
    const long long k0 = hh::g_kernel_launches;
    hh_status st = p->o.outer == HH_OUTER_RICHARDSON ? richardson(p, tol, info) : fgmres(p, tol, info);
    for (int b = 0; b < p->nb; ++b) info[b].device_bytes = p->bytes;
    info[0].kernel_launches += hh::g_kernel_launches - k0;
    return st;
}

void op_role(int op, bool* ok, int* role) {
    *ok = true;
    switch (op) {
        case HH_OP_K: *role = R_K; break;
        case HH_OP_M: *role = R_M; break;
        case HH_OP_MGAMMA: *role = R_MG; break;
        case HH_OP_AL: *role = R_AL; break;
        case HH_OP_AR: *role = R_AR; break;
        case HH_OP_B: *role = R_B; break;
        case HH_OP_BHAT: *role = R_BHAT; break;
        default: *ok = false; *role = 0;
    }
}

}  // namespace

// ====================================================================== packs
// A pack runs the FGMRES solves of several problems of DIFFERENT grids side by side: every
// outer iteration of every member is the same sequence of operations as in its own solve
// (fgmres above, one problem), on the member's own stream, except that the preconditioner
// applications of all members that need one in the same round run as one sequence of packed
// launches (pack.cu): one launch per pass of the V-cycle covers the tiles of every member, so
// small problems fill the GPU together instead of one after the other.  Members join and leave
// between rounds (continuous batching); each result equals the member's own solve bit for bit.
namespace {

enum PackState {
    PK_FREE = 0,     // empty slot
    PK_BNORM,        // waiting for ||b||
    PK_RES0,         // waiting for the initial residual norm
    PK_NEED_ITER,    // ready for iteration j (needs a preconditioner application)
    PK_ITER,         // waiting for iteration j's Arnoldi sums
    PK_CYCLE_END,    // waiting for the true residual after the update of x
    PK_DONE          // finished: result written, waiting to be taken
};

struct PackMember {
    hh_problem* p = nullptr;
    int state = PK_FREE;
    int io = 0;  // 0: device load vector in / device u out; 1: host load vector; 2: host nodal source
    void* u = nullptr;
    double tol = 0.0;
    int j = 0, jend = 0;
    double bnorm = 0.0, beta = 0.0, rel = 0.0;
    std::vector<zc> Hm, g, sn, y;
    std::vector<double> cs, cycle_rel;
    hh_info info{};
    hh_status st = HH_OK;
    std::string err;
    std::chrono::steady_clock::time_point t0;
};

// a problem the packed passes can run: 2D primal, one problem, V(2,2) scaled-Jacobi cycles with
// one cycle per HSS step, complex64 cycles, FGMRES
bool packable(const hh_problem* p, int levels, std::string* why) {
    const hh_options& o = p->o;
    if (p->grid.dim != 2 || p->nb != 1 || p->mixed) return *why = "packs hold 2D primal problems of one member each", false;
    if (o.smoother != HH_SMOOTH_JACOBI || o.cycle_gamma != 1 || o.cycles_per_hss != 1 || o.nu_pre != 2 ||
        o.nu_post != 2)
        return *why = "packs run V(2,2) scaled-Jacobi cycles, one per HSS step", false;
    if (o.precision != HH_C64 || o.outer != HH_OUTER_FGMRES) return *why = "packs run complex64 cycles inside FGMRES", false;
    if (o.levels < 2 || o.levels > hh::kPMaxLevels) return *why = "packs need 2..5 levels", false;
    if (levels && o.levels != levels) return *why = "every member of a pack has the same number of levels", false;
    return true;
}

int pack_passes(int L) { return 2 * L - 1; }
// kind and level of pass q (see launch_pack_pass)
void pass_kind(int L, int q, int* kind, int* level) {
    if (q == 0) *kind = 0, *level = 0;
    else if (q < L - 1) *kind = 1, *level = q;
    else if (q == L - 1) *kind = 2, *level = L - 1;
    else *kind = 3, *level = 2 * L - 2 - q;
}
int pass_tiles(const hh::HssLoop2<float>& P, const hh_problem* p, int kind, int level) {
    switch (kind) {
        case 0:
        case 1: return P.pre_strips[level] * P.pre_chunks[level];
        case 2: return (p->lv[level].nn + P.coarse_rows - 1) / P.coarse_rows;
        default: return P.post_strips[level] * P.post_chunks[level];
    }
}

hh_status enqueue_fetch(hh_problem* p) {
    HH_CUDA(cudaMemcpyAsync(p->h_host, p->hbuf, (size_t)hstride(p) * sizeof(double2), cudaMemcpyDeviceToHost, p->s));
    return HH_OK;
}

}  // namespace

struct hh_pack {
    int device = 0;
    int capacity = 0;
    int levels = 0;
    cudaStream_t s = nullptr;     // the packed preconditioner launches
    cudaEvent_t ev_prec = nullptr;
    std::vector<cudaEvent_t> ev_m;
    std::vector<PackMember> m;
    hh::HssLoop2<float>* d_plans = nullptr;
    std::vector<unsigned char> h_plans;
    int* d_starts = nullptr;      // pass q: capacity + 1 prefix entries at q * (capacity + 1)
    int* d_live = nullptr;
    int* h_live = nullptr;        // pinned
    std::vector<int> totals;
    size_t coarse_smem = 0;
    int maxsteps = 0;
    cudaGraphExec_t graph = nullptr;
    long long graph_kernels = 0;
    bool dirty = true;            // membership changed: tables and graph to rebuild
};

namespace {

hh_status pack_fail(PackMember& x, hh_status st) {
    x.st = st;
    x.err = hh_last_error();
    x.info.rel_residual = NAN;
    x.state = PK_DONE;
    return HH_OK;
}

// the member's result: u and info, then PK_DONE
hh_status pack_finish(PackMember& x) {
    hh_problem* p = x.p;
    const size_t bytes = (size_t)p->N * 16;
    if (x.io == 0) HH_CUDA(cudaMemcpyAsync(x.u, p->x, bytes, cudaMemcpyDeviceToDevice, p->s));
    else HH_CUDA(cudaMemcpyAsync(x.u, p->x, bytes, cudaMemcpyDeviceToHost, p->s));
    HH_CUDA(cudaStreamSynchronize(p->s));
    x.info.rel_residual = x.rel;
    x.info.device_bytes = p->bytes;
    x.info.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - x.t0).count();
    x.st = x.rel <= x.tol ? HH_OK : HH_NOT_CONVERGED;
    x.state = PK_DONE;
    return HH_OK;
}

// start a restart cycle: V_0 = r / beta (the residual norm is still in hbuf)
hh_status pack_cycle(PackMember& x) {
    hh_problem* p = x.p;
    const int m = p->o.restart, nrm = 2 * (m + 1);
    HH_CUDA(cudaMemcpyAsync(p->V, p->r, (size_t)p->N * 16, cudaMemcpyDeviceToDevice, p->s));
    HH_CUDA(hh::launch_scale_by_rnorm(p->V, p->hbuf + nrm, p->N, hh::KBatch{1, p->N, p->N, hstride(p), nullptr}, p->s));
    std::fill(x.g.begin(), x.g.end(), zc(0));
    x.g[0] = x.beta;
    x.j = 0;
    x.jend = 0;
    x.state = PK_NEED_ITER;
    return HH_OK;
}

// x += Z y, then the true residual and its norm
hh_status pack_cycle_end(PackMember& x) {
    hh_problem* p = x.p;
    const int m = p->o.restart, nrm = 2 * (m + 1);
    if (!back_substitute(x.Hm.data(), m, x.g.data(), x.jend, x.y.data()))
        return pack_fail(x, fail(HH_ERR_NONFINITE, "least-squares update is not finite"));
    for (int i = 0; i < m; ++i) p->h_host[i] = make_double2(x.y[i].real(), x.y[i].imag());
    HH_CUDA(cudaMemcpyAsync(p->ybuf, p->h_host, (size_t)m * 16, cudaMemcpyHostToDevice, p->s));
    if (x.jend > 0)
        HH_CUDA(hh::launch_multi_axpy(p->x, p->Z, p->N, x.jend, p->ybuf, 1.0, p->N, hh::KBatch{1, p->N, p->N, m, nullptr},
                                      p->s));
    HH_TRY(residual_B(p, p->x, p->r));
    HH_TRY(norm2_dev(p, p->r, nrm));
    HH_TRY(enqueue_fetch(p));
    x.state = PK_CYCLE_END;
    return HH_OK;
}

// what a member does after the round's synchronisation
hh_status pack_after_sync(PackMember& x) {
    hh_problem* p = x.p;
    const int m = p->o.restart, nrm = 2 * (m + 1);
    auto H = [&](int i) -> double2& { return p->h_host[i]; };
    auto Hc = [&](int i, int j) -> zc& { return x.Hm[(size_t)j * (m + 1) + i]; };
    switch (x.state) {
        case PK_BNORM:
            x.bnorm = std::sqrt(H(nrm).x);
            if (!finite(x.bnorm)) return pack_fail(x, fail(HH_ERR_NONFINITE, "right-hand side is not finite"));
            HH_TRY(residual_B(p, p->x, p->r));
            HH_TRY(norm2_dev(p, p->r, nrm));
            HH_TRY(enqueue_fetch(p));
            x.state = PK_RES0;
            return HH_OK;
        case PK_RES0:
            x.beta = std::sqrt(H(nrm).x);
            if (!finite(x.beta)) return pack_fail(x, fail(HH_ERR_NONFINITE, "initial residual is not finite"));
            x.rel = x.bnorm > 0 ? x.beta / x.bnorm : 0.0;
            x.cycle_rel.assign(1, x.rel);
            if (x.bnorm == 0.0) HH_CUDA(cudaMemsetAsync(p->x, 0, (size_t)p->N * 16, p->s));
            if (x.bnorm == 0.0 || x.rel <= x.tol || p->o.max_outer == 0) return pack_finish(x);
            return pack_cycle(x);
        case PK_ITER: {
            const int j = x.j;
            for (int i = 0; i <= j; ++i) Hc(i, j) = zc(H(i).x + H(m + 1 + i).x, H(i).y + H(m + 1 + i).y);
            const double hn = std::sqrt(H(nrm).x);
            if (!finite(hn)) return pack_fail(x, fail(HH_ERR_NONFINITE, "Arnoldi produced a non-finite value"));
            Hc(j + 1, j) = hn;
            givens_column(&Hc(0, j), x.cs.data(), x.sn.data(), x.g.data(), j);
            x.info.outer_its += 1;
            x.jend = j + 1;
            const bool leave = std::abs(x.g[j + 1]) / x.bnorm <= x.tol || x.info.outer_its >= p->o.max_outer || hn == 0.0;
            if (leave || j + 1 == m) return pack_cycle_end(x);
            x.j = j + 1;
            x.state = PK_NEED_ITER;
            return HH_OK;
        }
        case PK_CYCLE_END: {
            x.beta = std::sqrt(H(nrm).x);
            if (!finite(x.beta)) return pack_fail(x, fail(HH_ERR_NONFINITE, "residual is not finite"));
            x.rel = x.beta / x.bnorm;
            bool stop = x.rel <= x.tol || x.info.outer_its >= p->o.max_outer;
            x.cycle_rel.push_back(x.rel);
            const int sc = p->o.stall_cycles, nc = (int)x.cycle_rel.size() - 1;
            if (sc > 0 && nc >= sc && x.rel > 0.5 * x.cycle_rel[nc - sc]) stop = true;
            if (stop) return pack_finish(x);
            return pack_cycle(x);
        }
        default: return HH_OK;
    }
}

// member tables, tile prefixes and the graph of one packed preconditioner application
hh_status pack_rebuild(hh_pack* k) {
    const int cap = k->capacity, L = k->levels, Q = pack_passes(L);
    k->h_plans.assign((size_t)cap * sizeof(hh::HssLoop2<float>), 0);
    auto* plans = reinterpret_cast<hh::HssLoop2<float>*>(k->h_plans.data());
    std::vector<int> starts((size_t)Q * (cap + 1), 0);
    k->totals.assign(Q, 0);
    k->coarse_smem = 0;
    k->maxsteps = 0;
    for (int i = 0; i < cap; ++i) {
        PackMember& x = k->m[i];
        const bool in = x.state != PK_FREE && x.state != PK_DONE;
        if (in) {
            MG<float> mg = make_mg<float>(x.p, HH_C64, x.p->s);
            mg.loop_plan(&plans[i]);
            k->maxsteps = std::max(k->maxsteps, plans[i].nsteps);
            k->coarse_smem = std::max(k->coarse_smem, hh::hss_loop2_smem<float>(x.p->lv[L - 1], x.p->o.nu_coarse,
                                                                               plans[i].coarse_rows));
        }
        for (int q = 0; q < Q; ++q) {
            int kind, level;
            pass_kind(L, q, &kind, &level);
            const int t = in ? pass_tiles(plans[i], x.p, kind, level) : 0;
            starts[(size_t)q * (cap + 1) + i + 1] = starts[(size_t)q * (cap + 1) + i] + t;
        }
    }
    for (int q = 0; q < Q; ++q) k->totals[q] = starts[(size_t)q * (cap + 1) + cap];
    if (k->coarse_smem > hh::kLoopSmemMax) return fail(HH_ERR_INVALID, "a member's coarsest level is too wide to pack");
    HH_CUDA(cudaMemcpyAsync(k->d_plans, k->h_plans.data(), k->h_plans.size(), cudaMemcpyHostToDevice, k->s));
    HH_CUDA(cudaMemcpyAsync(k->d_starts, starts.data(), starts.size() * sizeof(int), cudaMemcpyHostToDevice, k->s));
    HH_CUDA(cudaStreamSynchronize(k->s));
    if (k->graph) {
        cudaGraphExecDestroy(k->graph);
        k->graph = nullptr;
    }
    if (k->maxsteps > 0) {
        cudaGraph_t g;
        const long long k0 = hh::g_kernel_launches;
        HH_CUDA(cudaStreamBeginCapture(k->s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int it = 0; it < k->maxsteps && e == cudaSuccess; ++it)
            for (int q = 0; q < Q && e == cudaSuccess; ++q) {
                int kind, level;
                pass_kind(L, q, &kind, &level);
                e = hh::launch_pack_pass<float>(kind, k->d_plans, k->d_starts + (size_t)q * (cap + 1), cap, k->totals[q],
                                                level, it, k->d_live, k->coarse_smem, k->s);
            }
        cudaError_t ec = cudaStreamEndCapture(k->s, &g);
        if (e != cudaSuccess) {
            if (ec == cudaSuccess) cudaGraphDestroy(g);
            return fail(HH_ERR_CUDA, std::string("packed launch: ") + cudaGetErrorString(e));
        }
        HH_CUDA(ec);
        cudaError_t ei = cudaGraphInstantiate(&k->graph, g, 0);
        cudaGraphDestroy(g);
        HH_CUDA(ei);
        k->graph_kernels = hh::g_kernel_launches - k0;
        hh::g_kernel_launches = k0;
    }
    k->dirty = false;
    return HH_OK;
}

// one round: every member advances to its next synchronisation point
hh_status pack_round(hh_pack* k) {
    hh::g_use_pdl = 1;
    if (k->dirty) HH_TRY(pack_rebuild(k));
    const int cap = k->capacity;
    bool any = false;
    for (int i = 0; i < cap; ++i) {
        PackMember& x = k->m[i];
        k->h_live[i] = 0;
        if (x.state != PK_NEED_ITER) continue;
        hh_problem* p = x.p;
        Hier& H = p->hier[HH_C64];
        HH_LAUNCH(hh::launch_cast_d2f(p->V + (long long)x.j * p->N, (float2*)H.r_lo, p->N, p->s));
        HH_CUDA(cudaEventRecord(k->ev_m[i], p->s));
        HH_CUDA(cudaStreamWaitEvent(k->s, k->ev_m[i], 0));
        k->h_live[i] = 1;
        any = true;
    }
    if (any) {
        HH_CUDA(cudaMemcpyAsync(k->d_live, k->h_live, sizeof(int) * cap, cudaMemcpyHostToDevice, k->s));
        if (k->graph) HH_CUDA(cudaGraphLaunch(k->graph, k->s));
        HH_CUDA(cudaEventRecord(k->ev_prec, k->s));
    }
    for (int i = 0; i < cap; ++i) {
        PackMember& x = k->m[i];
        if (x.state != PK_NEED_ITER) continue;
        hh_problem* p = x.p;
        Hier& H = p->hier[HH_C64];
        const int m = p->o.restart, nrm = 2 * (m + 1);
        HH_CUDA(cudaStreamWaitEvent(p->s, k->ev_prec, 0));
        double2* zj = p->Z + (long long)x.j * p->N;
        double2* w = p->V + (long long)(x.j + 1) * p->N;
        HH_LAUNCH(hh::launch_gather_c128<float>((const float2* const*)H.usrc, zj, p->lv[0].N, 1, nullptr, p->s));
        x.info.hss_its += p->nhss[0];
        x.info.vcycles += p->nhss[0];
        HH_TRY(apply_B(p, zj, w));
        const hh::KBatch kb{1, p->N, p->N, hstride(p), nullptr};
        double2* hA = p->hbuf;
        double2* hB = p->hbuf + (m + 1);
        HH_CUDA(hh::launch_multidot(p->V, p->N, x.j + 1, w, p->N, p->partials, hA, kb, p->s));
        HH_CUDA(hh::launch_multi_axpy(w, p->V, p->N, x.j + 1, hA, -1.0, p->N, kb, p->s));
        HH_CUDA(hh::launch_multidot(p->V, p->N, x.j + 1, w, p->N, p->partials, hB, kb, p->s));
        HH_CUDA(hh::launch_multi_axpy(w, p->V, p->N, x.j + 1, hB, -1.0, p->N, kb, p->s));
        HH_CUDA(hh::launch_multidot(w, 0, 1, w, p->N, p->partials, p->hbuf + nrm, kb, p->s));
        HH_CUDA(hh::launch_scale_by_rnorm(w, p->hbuf + nrm, p->N, kb, p->s));
        HH_TRY(enqueue_fetch(p));
        x.state = PK_ITER;
    }
    if (any) HH_CUDA(cudaStreamSynchronize(k->s));
    for (int i = 0; i < cap; ++i) {
        PackMember& x = k->m[i];
        if (x.state == PK_FREE || x.state == PK_DONE) continue;
        cudaError_t e = cudaStreamSynchronize(x.p->s);
        if (e != cudaSuccess) {
            pack_fail(x, fail(HH_ERR_CUDA, cudaGetErrorString(e)));
            k->dirty = true;
            continue;
        }
        const hh_status st = pack_after_sync(x);
        if (st != HH_OK) pack_fail(x, st);
        if (x.state == PK_DONE) k->dirty = true;
    }
    return HH_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void hh_options_default(hh_options* o) {
    if (!o) return;
    o->theta = 1.0;
    o->levels = 4;
    o->nu_pre = 2;
    o->nu_post = 2;
    o->nu_coarse = 8;
    o->cycles_per_hss = 1;
    o->omega = 0.0;  // automatic: 0.6 in 2D, 0.5 in 3D
    o->restart = 30;
    o->max_outer = 1000;
    o->precision = HH_C64;
    o->use_graphs = 1;
    o->use_pdl = 1;
    o->coarse_cluster_nodes = 100000;
    o->tile_rows = 0;
    o->autotune = 0;
    o->fuse_sweeps = 1;
    o->outer = HH_OUTER_FGMRES;
    o->cycle_gamma = 1;
    o->tile_form = 0;
    o->smoother = HH_SMOOTH_JACOBI;
    o->formulation = HH_FORM_PRIMAL;
    o->persistent = 0;
    o->sync_spin_limit = 0;
    o->stall_cycles = 0;
    o->coarse_kernel = 0;
}

size_t hh_footprint_batch_bytes(const hh_grid* grid, const hh_options* o, int nb) {
    if (!grid || !o || nb < 1) return 0;
    const int bc0[6] = {0, 0, 0, 0, 0, 0};
    std::vector<double> one(nb, 1.0), zero(nb, 0.0);
    if (check_args(grid, nb, one.data(), zero.data(), one.data(), bc0, o) != HH_OK) return 0;
    return hier_bytes(grid, o, o->precision, nb) +
           krylov_bytes(grid, o->restart, nb, o->formulation == HH_FORM_MIXED ? sigma_dofs(grid) : 0);
}

size_t hh_footprint_bytes(const hh_grid* grid, const hh_options* o) { return hh_footprint_batch_bytes(grid, o, 1); }

void hh_destroy(hh_problem* p) {
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    if (p->s) cudaStreamSynchronize(p->s);
    for (int i = 0; i < 2; ++i)
        if (p->hier[i].graph) cudaGraphExecDestroy(p->hier[i].graph);
    for (void* a : p->allocs) cudaFree(a);
    if (p->h_host) cudaFreeHost(p->h_host);
    if (p->h_active) cudaFreeHost(p->h_active);
    if (p->h_sync) cudaFreeHost(p->h_sync);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->s) cudaStreamDestroy(p->s);
    cudaSetDevice(cur);
    delete p;
}

hh_status hh_create_batch(const hh_grid* grid, int nb, const double* k, const double* delta, const double* delta_hat,
                          const int* bc, const hh_options* opts, void* cuda_stream, hh_problem** out) {
    if (!out) return fail(HH_ERR_INVALID, "null out");
    *out = nullptr;
    HH_TRY(check_args(grid, nb, k, delta, delta_hat, bc, opts));
    hh_problem* p = new hh_problem();
    cudaGetDevice(&p->device);
    p->grid = *grid;
    p->nb = nb;
    p->k.assign(k, k + nb);
    p->delta.assign(delta, delta + nb);
    p->dh.assign(delta_hat, delta_hat + nb);
    for (int s = 0; s < 6; ++s) p->bc[s] = s < 2 * grid->dim ? bc[s] : 0;
    p->o = *opts;
    // automatic damping: on levels where the shifted mass term dominates, D^{-1} A_L has
    // spectrum close to D^{-1} M, which reaches 9/4 in 2D and 27/8 in 3D; omega must stay
    // below 2 / 27 * 8 = 0.59 in 3D for the sweeps not to amplify smooth modes
    if (p->o.omega == 0.0) p->o.omega = grid->dim == 3 ? 0.5 : 0.6;
    for (int b = 0; b < nb; ++b) {
        p->nhss.push_back(n_hss(k[b], p->o.theta));
        p->max_nhss = std::max(p->max_nhss, p->nhss.back());
    }
    for (int l = 0; l < opts->levels; ++l) p->lv.push_back(level_desc(*grid, p->bc, l));
    p->mixed = opts->formulation == HH_FORM_MIXED;
    p->ns = p->mixed ? sigma_dofs(grid) : 0;
    p->N = p->lv[0].N + p->ns;
    p->user = (cudaStream_t)cuda_stream;
    hh_status st = HH_OK;
    auto bail = [&](hh_status s) {
        hh_destroy(p);
        return s;
    };
    if (cudaStreamCreateWithFlags(&p->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(HH_ERR_CUDA, "stream/event creation failed"));
    const int m = opts->restart;
    const long long N = p->N;
    const size_t hs = (size_t)(2 * (m + 1) + 1);
    if ((st = dmalloc(p, (void**)&p->d_nhss, sizeof(int) * nb)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->d_active, sizeof(int) * nb)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->d_sync, 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->V, (size_t)(m + 1) * nb * N * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->Z, (size_t)m * nb * N * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->x, (size_t)nb * N * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->bvec, (size_t)nb * N * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->r, (size_t)nb * N * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->partials, (size_t)nb * (m + 1) * hh::kRedBlocks * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->hbuf, (size_t)nb * hs * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->ybuf, (size_t)nb * m * 16)) != HH_OK) return bail(st);
    if (cudaMallocHost((void**)&p->h_host, (size_t)nb * hs * 16) != cudaSuccess ||
        cudaMallocHost((void**)&p->h_active, sizeof(int) * nb) != cudaSuccess ||
        cudaMallocHost((void**)&p->h_sync, sizeof(int)) != cudaSuccess)
        return bail(fail(HH_ERR_OOM, "pinned host allocation failed"));
    *p->h_sync = 0;
    if (cudaMemcpyAsync(p->d_nhss, p->nhss.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, p->s) != cudaSuccess ||
        cudaMemsetAsync(p->d_sync, 0, 16, p->s) != cudaSuccess)
        return bail(fail(HH_ERR_CUDA, "initialisation failed"));
    if ((st = set_active(p, nullptr)) != HH_OK) return bail(st);
    if ((st = ensure_hier(p, opts->precision)) != HH_OK) return bail(st);
    if (cudaMemsetAsync(p->V, 0, (size_t)(m + 1) * nb * N * 16, p->s) != cudaSuccess ||
        cudaMemsetAsync(p->Z, 0, (size_t)m * nb * N * 16, p->s) != cudaSuccess ||
        cudaMemsetAsync(p->r, 0, (size_t)nb * N * 16, p->s) != cudaSuccess ||
        cudaStreamSynchronize(p->s) != cudaSuccess)
        return bail(fail(HH_ERR_CUDA, "initialisation failed"));
    if (opts->autotune && (st = autotune(p, opts->precision)) != HH_OK) return bail(st);
    *out = p;
    return HH_OK;
}

hh_status hh_set_params(hh_problem* p, const double* k, const double* delta, const double* delta_hat) {
    if (!p) return fail(HH_ERR_INVALID, "null problem");
    HH_TRY(check_args(&p->grid, p->nb, k, delta, delta_hat, p->bc, &p->o));
    HH_CUDA(cudaStreamSynchronize(p->s));
    p->k.assign(k, k + p->nb);
    p->delta.assign(delta, delta + p->nb);
    p->dh.assign(delta_hat, delta_hat + p->nb);
    p->max_nhss = 0;
    for (int b = 0; b < p->nb; ++b) {
        p->nhss[b] = n_hss(k[b], p->o.theta);
        p->max_nhss = std::max(p->max_nhss, p->nhss[b]);
    }
    HH_CUDA(cudaMemcpyAsync(p->d_nhss, p->nhss.data(), sizeof(int) * p->nb, cudaMemcpyHostToDevice, p->s));
    HH_TRY(build_tables<float>(p, p->hier[HH_C64]));
    HH_TRY(build_tables<double>(p, p->hier[HH_C128]));
    // the preconditioner graphs and loop plans hold the old coefficients and HSS lengths
    for (int q = 0; q < 2; ++q) {
        if (p->hier[q].graph) {
            cudaGraphExecDestroy(p->hier[q].graph);
            p->hier[q].graph = nullptr;
        }
        p->hier[q].loop.clear();
    }
    return HH_OK;
}

hh_status hh_prepare(hh_problem* p) {
    if (!p) return fail(HH_ERR_INVALID, "null problem");
    HH_TRY(join_in(p));
    HH_CUDA(cudaMemsetAsync(p->r, 0, (size_t)p->nb * p->N * 16, p->s));
    HH_TRY(precondition_async(p, p->r, p->Z));
    HH_CUDA(cudaMemcpyAsync(p->h_sync, p->d_sync + 1, sizeof(int), cudaMemcpyDeviceToHost, p->s));
    HH_TRY(join_out(p));
    HH_CUDA(cudaStreamSynchronize(p->s));
    return check_sync(p);
}

hh_status hh_create_problem(const hh_grid* grid, double k, double delta, double delta_hat, const int* bc,
                            const hh_options* opts, void* cuda_stream, hh_problem** out) {
    return hh_create_batch(grid, 1, &k, &delta, &delta_hat, bc, opts, cuda_stream, out);
}

int hh_batch_size(const hh_problem* p) { return p ? p->nb : 0; }

hh_status hh_autotune(hh_problem* p, int precision, int* shapes) {
    if (!p) return fail(HH_ERR_INVALID, "null problem");
    HH_TRY(validate_prec(precision));
    HH_TRY(join_in(p));
    HH_TRY(autotune(p, precision));
    HH_TRY(join_out(p));
    if (shapes) {
        for (int l = 0; l < p->o.levels; ++l)
            for (int mode = 0; mode < kModes; ++mode)
                for (int c = 0; c < 2; ++c) shapes[((size_t)l * kModes + mode) * 2 + c] = p->tune[precision][l][mode][c];
    }
    return HH_OK;
}

long long hh_level_nodes(const hh_problem* p, int level) {
    if (!p || level < 0 || level >= p->o.levels) return 0;
    return p->lv[level].N;
}

// dst = src with exact zeros at the Dirichlet nodes (a mixed problem's sigma part copied as is)
hh_status masked_copy(hh_problem* p, const double2* src, double2* dst) {
    if (p->mixed) {
        HH_CUDA(cudaMemcpyAsync(dst, src, (size_t)p->ns * 16, cudaMemcpyDeviceToDevice, p->s));
        HH_LAUNCH(hh::launch_mask_copy(p->lv[0], src + p->ns, dst + p->ns, 1, p->s));
    } else {
        HH_LAUNCH(hh::launch_mask_copy(p->lv[0], src, dst, p->nb, p->s));
    }
    return HH_OK;
}

hh_status hh_solve(hh_problem* p, const void* rhs, double tol, void* u, const void* x0, hh_info* info) {
    if (!p || !rhs || !u) return fail(HH_ERR_INVALID, "null argument");
    if (!(tol > 0)) return fail(HH_ERR_INVALID, "tol must be > 0");
    std::vector<hh_info> local(p->nb);
    hh_info* inf = info ? info : local.data();
    for (int b = 0; b < p->nb; ++b) {
        inf[b] = hh_info{};
        inf[b].rel_residual = NAN;
    }
    auto t0 = std::chrono::steady_clock::now();
    HH_TRY(join_in(p));
    HH_TRY(masked_copy(p, (const double2*)rhs, p->bvec));
    if (x0) {
        HH_TRY(masked_copy(p, (const double2*)x0, p->x));
    } else {
        HH_CUDA(cudaMemsetAsync(p->x, 0, (size_t)p->nb * p->N * 16, p->s));
    }
    hh_status st = solve_core(p, tol, inf);
    if (st == HH_OK || st == HH_NOT_CONVERGED) {
        HH_CUDA(cudaMemcpyAsync(u, p->x, (size_t)p->nb * p->N * 16, cudaMemcpyDeviceToDevice, p->s));
    } else {
        for (int b = 0; b < p->nb; ++b) inf[b].rel_residual = NAN;
        set_active(p, nullptr);
    }
    HH_TRY(join_out(p));
    HH_CUDA(cudaStreamSynchronize(p->s));
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int b = 0; b < p->nb; ++b) inf[b].seconds = sec;
    return st;
}

static hh_status solve_host_impl(hh_problem* p, const void* rhs_host, bool nodal, double tol, void* u_host,
                                 hh_info* info) {
    if (!p || !rhs_host || !u_host) return fail(HH_ERR_INVALID, "null argument");
    if (!(tol > 0)) return fail(HH_ERR_INVALID, "tol must be > 0");
    std::vector<hh_info> local(p->nb);
    hh_info* inf = info ? info : local.data();
    for (int b = 0; b < p->nb; ++b) {
        inf[b] = hh_info{};
        inf[b].rel_residual = NAN;
    }
    const size_t bytes = (size_t)p->nb * p->N * 16;
    auto t0 = std::chrono::steady_clock::now();
    HH_TRY(join_in(p));
    // stage the right side through r, then mask into bvec (nodal source: bvec = M f)
    HH_CUDA(cudaMemcpyAsync(p->r, rhs_host, bytes, cudaMemcpyHostToDevice, p->s));
    if (nodal) {
        HH_TRY(op_axpby<double>(p, 0, R_M, p->r, nullptr, p->bvec, Cx<double>{1, 0}, Cx<double>{0, 0}, p->s));
    } else {
        HH_TRY(masked_copy(p, p->r, p->bvec));
    }
    HH_CUDA(cudaMemsetAsync(p->x, 0, bytes, p->s));
    hh_status st = solve_core(p, tol, inf);
    if (st == HH_OK || st == HH_NOT_CONVERGED) {
        HH_CUDA(cudaMemcpyAsync(u_host, p->x, bytes, cudaMemcpyDeviceToHost, p->s));
    } else {
        for (int b = 0; b < p->nb; ++b) inf[b].rel_residual = NAN;
        set_active(p, nullptr);
    }
    HH_TRY(join_out(p));
    HH_CUDA(cudaStreamSynchronize(p->s));
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int b = 0; b < p->nb; ++b) inf[b].seconds = sec;
    return st;
}

hh_status hh_solve_host(hh_problem* p, const void* rhs_host, double tol, void* u_host, hh_info* info) {
    return solve_host_impl(p, rhs_host, false, tol, u_host, info);
}

hh_status hh_solve_host_nodal(hh_problem* p, const void* f_host, double tol, void* u_host, hh_info* info) {
    if (p && p->mixed) return fail(HH_ERR_INVALID, "nodal sources are for primal problems");
    return solve_host_impl(p, f_host, true, tol, u_host, info);
}

long long hh_sigma_dofs(const hh_grid* grid) {
    if (!grid || (grid->dim != 2 && grid->dim != 3) || grid->n < 1) return 0;
    return sigma_dofs(grid);
}

long long hh_vector_length(const hh_problem* p) { return p ? p->N : 0; }

void hh_set_allocation_limit(size_t bytes) { g_alloc_limit.store(bytes); }

hh_status hh_apply_system(hh_problem* p, const void* x, void* y) {
    if (!p || !x || !y) return fail(HH_ERR_INVALID, "null argument");
    if (p->mixed && x == y) return fail(HH_ERR_INVALID, "x and y must differ");
    HH_TRY(join_in(p));
    HH_TRY(apply_B(p, (const double2*)x, (double2*)y));
    return join_out(p);
}

// ---------------------------------------------------------------- building blocks
hh_status hh_apply(hh_problem* p, int level, int op, int precision, const void* x, void* y) {
    HH_TRY(validate_level(p, level, 0));
    HH_TRY(validate_prec(precision));
    if (!x || !y) return fail(HH_ERR_INVALID, "null vector");
    bool ok;
    int role;
    op_role(op, &ok, &role);
    if (!ok) return fail(HH_ERR_INVALID, "unknown operator");
    HH_TRY(join_in(p));
    if (precision == HH_C64) {
        HH_TRY(op_axpby<float>(p, level, role, (const float2*)x, nullptr, (float2*)y, Cx<float>{1, 0},
                               Cx<float>{0, 0}, p->s));
    } else {
        HH_TRY(op_axpby<double>(p, level, role, (const double2*)x, nullptr, (double2*)y, Cx<double>{1, 0},
                                Cx<double>{0, 0}, p->s));
    }
    return join_out(p);
}

hh_status hh_jacobi(hh_problem* p, int level, int precision, const void* b, const void* x_in, void* x_out) {
    HH_TRY(validate_level(p, level, 0));
    HH_TRY(validate_prec(precision));
    if (!b || !x_out || x_out == x_in || x_out == b) return fail(HH_ERR_INVALID, "bad vectors");
    HH_TRY(ensure_tables(p));
    HH_TRY(join_in(p));
    if (precision == HH_C64) {
        MG<float> m = make_mg<float>(p, precision, p->s);
        HH_TRY(m.jacobi(level, (const float2*)b, (const float2*)x_in, (float2*)x_out));
    } else {
        MG<double> m = make_mg<double>(p, precision, p->s);
        HH_TRY(m.jacobi(level, (const double2*)b, (const double2*)x_in, (double2*)x_out));
    }
    return join_out(p);
}

hh_status hh_residual_restrict(hh_problem* p, int level, int precision, const void* b, const void* x, void* rc) {
    HH_TRY(validate_level(p, level, 1));
    HH_TRY(validate_prec(precision));
    if (!b || !x || !rc) return fail(HH_ERR_INVALID, "null vector");
    HH_TRY(ensure_hier(p, precision));
    HH_TRY(join_in(p));
    if (precision == HH_C64) {
        MG<float> m = make_mg<float>(p, precision, p->s);
        HH_TRY(m.resid_restrict(level, (const float2*)b, (const float2*)x, (float2*)rc));
    } else {
        MG<double> m = make_mg<double>(p, precision, p->s);
        HH_TRY(m.resid_restrict(level, (const double2*)b, (const double2*)x, (double2*)rc));
    }
    return join_out(p);
}

hh_status hh_prolong_correct(hh_problem* p, int level, int precision, const void* ec, void* x) {
    HH_TRY(validate_level(p, level, 1));
    HH_TRY(validate_prec(precision));
    if (!ec || !x) return fail(HH_ERR_INVALID, "null vector");
    HH_TRY(join_in(p));
    const hh::Batch bt{p->nb, p->lv[level].N, p->lv[level + 1].N, -1, nullptr, nullptr};
    if (precision == HH_C64) {
        HH_LAUNCH(hh::launch_prolong<float>(p->lv[level], (const float2*)ec, (float2*)x, bt, p->s));
    } else {
        HH_LAUNCH(hh::launch_prolong<double>(p->lv[level], (const double2*)ec, (double2*)x, bt, p->s));
    }
    return join_out(p);
}

hh_status hh_vcycle(hh_problem* p, int precision, const void* b, void* x) {
    HH_TRY(validate_level(p, 0, 0));
    HH_TRY(validate_prec(precision));
    if (!b || !x) return fail(HH_ERR_INVALID, "null vector");
    HH_TRY(ensure_hier(p, precision));
    HH_TRY(join_in(p));
    const size_t nbytes = (size_t)p->nb * p->N * (precision == HH_C64 ? 8 : 16);
    if (precision == HH_C64) {
        MG<float> m = make_mg<float>(p, precision, p->s);
        float2* out;
        HH_TRY(m.vcycle(0, (const float2*)b, nullptr, &out));
        HH_CUDA(cudaMemcpyAsync(x, out, nbytes, cudaMemcpyDeviceToDevice, p->s));
    } else {
        MG<double> m = make_mg<double>(p, precision, p->s);
        double2* out;
        HH_TRY(m.vcycle(0, (const double2*)b, nullptr, &out));
        HH_CUDA(cudaMemcpyAsync(x, out, nbytes, cudaMemcpyDeviceToDevice, p->s));
    }
    return join_out(p);
}

hh_status hh_hss_rhs(hh_problem* p, int precision, const void* u, const void* r, void* rhs) {
    HH_TRY(validate_level(p, 0, 0));
    HH_TRY(validate_prec(precision));
    if (!r || !rhs) return fail(HH_ERR_INVALID, "null vector");
    HH_TRY(ensure_tables(p));
    HH_TRY(join_in(p));
    if (precision == HH_C64) {
        MG<float> m = make_mg<float>(p, precision, p->s);
        HH_TRY(m.hss_rhs((const float2*)u, (const float2*)r, (float2*)rhs));
    } else {
        MG<double> m = make_mg<double>(p, precision, p->s);
        HH_TRY(m.hss_rhs((const double2*)u, (const double2*)r, (double2*)rhs));
    }
    return join_out(p);
}

hh_status hh_precondition(hh_problem* p, const void* r, void* z) {
    if (!p || !r || !z) return fail(HH_ERR_INVALID, "null argument");
    HH_TRY(join_in(p));
    HH_TRY(precondition_async(p, (const double2*)r, (double2*)z));
    HH_CUDA(cudaMemcpyAsync(p->h_sync, p->d_sync + 1, sizeof(int), cudaMemcpyDeviceToHost, p->s));
    HH_TRY(join_out(p));
    HH_CUDA(cudaStreamSynchronize(p->s));
    return check_sync(p);
}

hh_status hh_load_vector(hh_problem* p, const void* f, void* b) {
    if (!p || !f || !b) return fail(HH_ERR_INVALID, "null argument");
    HH_TRY(join_in(p));
    HH_TRY(op_axpby<double>(p, 0, R_M, (const double2*)f, nullptr, (double2*)b, Cx<double>{1, 0}, Cx<double>{0, 0},
                            p->s));
    return join_out(p);
}

hh_status hh_dot(hh_problem* p, const void* x, const void* y, double* out) {
    if (!p || !x || !y || !out) return fail(HH_ERR_INVALID, "null argument");
    HH_TRY(join_in(p));
    const int hs = hstride(p);
    HH_CUDA(hh::launch_multidot((const double2*)x, 0, 1, (const double2*)y, p->N, p->partials, p->hbuf,
                                hh::KBatch{p->nb, p->N, p->N, hs, nullptr}, p->s));
    HH_TRY(fetch(p));
    for (int b = 0; b < p->nb; ++b) {
        out[2 * b] = p->h_host[(size_t)b * hs].x;
        out[2 * b + 1] = p->h_host[(size_t)b * hs].y;
    }
    return HH_OK;
}

const char* hh_status_string(hh_status s) {
    switch (s) {
        case HH_OK: return "ok";
        case HH_NOT_CONVERGED: return "not converged";
        case HH_ERR_INVALID: return "invalid argument";
        case HH_ERR_OOM: return "out of device memory";
        case HH_ERR_CUDA: return "CUDA error";
        case HH_ERR_NONFINITE: return "non-finite value";
        case HH_ERR_TIMEOUT: return "timeout";
    }
    return "unknown status";
}

const char* hh_last_error(void) { return g_last_error.c_str(); }

hh_status hh_pack_create(int capacity, hh_pack** out) {
    if (!out) return fail(HH_ERR_INVALID, "null out");
    *out = nullptr;
    if (capacity < 1 || capacity > 256) return fail(HH_ERR_INVALID, "capacity must be in 1..256");
    hh_pack* k = new hh_pack();
    cudaGetDevice(&k->device);
    k->capacity = capacity;
    k->m.resize(capacity);
    k->ev_m.assign(capacity, nullptr);
    auto bail = [&](hh_status s) {
        hh_pack_destroy(k);
        return s;
    };
    if (cudaStreamCreateWithFlags(&k->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&k->ev_prec, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(HH_ERR_CUDA, "stream/event creation failed"));
    for (int i = 0; i < capacity; ++i)
        if (cudaEventCreateWithFlags(&k->ev_m[i], cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(HH_ERR_CUDA, "event creation failed"));
    const size_t Q = 2 * hh::kPMaxLevels - 1;
    if (cudaMalloc((void**)&k->d_plans, (size_t)capacity * sizeof(hh::HssLoop2<float>)) != cudaSuccess ||
        cudaMalloc((void**)&k->d_starts, Q * (capacity + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&k->d_live, capacity * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&k->h_live, capacity * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(HH_ERR_OOM, "pack allocation failed"));
    }
    if (hh::prepare_pack<float>() != cudaSuccess) return bail(fail(HH_ERR_CUDA, "pack kernel set-up failed"));
    *out = k;
    return HH_OK;
}

void hh_pack_destroy(hh_pack* k) {
    if (!k) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(k->device);
    if (k->s) cudaStreamSynchronize(k->s);
    for (auto& x : k->m)
        if (x.p) cudaStreamSynchronize(x.p->s);
    if (k->graph) cudaGraphExecDestroy(k->graph);
    for (auto e : k->ev_m)
        if (e) cudaEventDestroy(e);
    if (k->ev_prec) cudaEventDestroy(k->ev_prec);
    if (k->d_plans) cudaFree(k->d_plans);
    if (k->d_starts) cudaFree(k->d_starts);
    if (k->d_live) cudaFree(k->d_live);
    if (k->h_live) cudaFreeHost(k->h_live);
    if (k->s) cudaStreamDestroy(k->s);
    cudaSetDevice(cur);
    delete k;
}

int hh_pack_members(const hh_pack* k) {
    if (!k) return 0;
    int n = 0;
    for (const auto& x : k->m) n += x.state != PK_FREE;
    return n;
}

hh_status hh_pack_add(hh_pack* k, hh_problem* p, const void* rhs, int io, double tol, void* u, int* slot) {
    if (!k || !p || !rhs || !u || !slot) return fail(HH_ERR_INVALID, "null argument");
    if (!(tol > 0)) return fail(HH_ERR_INVALID, "tol must be > 0");
    if (io < 0 || io > 2) return fail(HH_ERR_INVALID, "io must be 0 (device), 1 (host load vector) or 2 (host nodal source)");
    std::string why;
    if (!packable(p, hh_pack_members(k) ? k->levels : 0, &why)) return fail(HH_ERR_INVALID, why);
    int i = 0;
    while (i < k->capacity && k->m[i].state != PK_FREE) ++i;
    if (i == k->capacity) return fail(HH_ERR_INVALID, "the pack is full");
    for (const auto& x : k->m)
        if (x.p == p && x.state != PK_FREE) return fail(HH_ERR_INVALID, "the problem is already in the pack");
    HH_TRY(ensure_hier(p, HH_C64));
    Hier& H = p->hier[HH_C64];
    // the packed passes leave u in xb[0]; a later solve of its own captures its graph anew
    if (H.graph) {
        cudaGraphExecDestroy(H.graph);
        H.graph = nullptr;
    }
    H.loop.clear();
    const long long N0 = p->lv[0].N;
    void* src = p->nhss[0] > 0 ? H.xb[0] : H.cres;
    if (p->nhss[0] == 0) HH_CUDA(cudaMemsetAsync(H.cres, 0, (size_t)N0 * sizeof(float2), p->s));
    HH_CUDA(cudaMemcpyAsync(H.usrc, &src, sizeof(void*), cudaMemcpyHostToDevice, p->s));
    const size_t bytes = (size_t)p->N * 16;
    if (io == 0) {
        HH_TRY(masked_copy(p, (const double2*)rhs, p->bvec));
    } else {
        HH_CUDA(cudaMemcpyAsync(p->r, rhs, bytes, cudaMemcpyHostToDevice, p->s));
        if (io == 2)
            HH_TRY(op_axpby<double>(p, 0, R_M, p->r, nullptr, p->bvec, Cx<double>{1, 0}, Cx<double>{0, 0}, p->s));
        else
            HH_TRY(masked_copy(p, p->r, p->bvec));
    }
    HH_CUDA(cudaMemsetAsync(p->x, 0, bytes, p->s));
    const int m = p->o.restart;
    HH_TRY(norm2_dev(p, p->bvec, 2 * (m + 1)));
    HH_TRY(enqueue_fetch(p));
    HH_CUDA(cudaStreamSynchronize(p->s));  // the source (the address of src, host data) is read
    PackMember& x = k->m[i];
    x = PackMember{};
    x.p = p;
    x.io = io;
    x.u = u;
    x.tol = tol;
    x.Hm.assign((size_t)(m + 1) * m, zc(0));
    x.g.assign(m + 1, zc(0));
    x.sn.assign(m, zc(0));
    x.y.assign(m, zc(0));
    x.cs.assign(m, 0.0);
    x.t0 = std::chrono::steady_clock::now();
    x.state = PK_BNORM;
    if (hh_pack_members(k) == 1) k->levels = p->o.levels;
    k->dirty = true;
    *slot = i;
    return HH_OK;
}

hh_status hh_pack_run(hh_pack* k, int max_rounds, int* done, int* ndone) {
    if (!k || !done || !ndone) return fail(HH_ERR_INVALID, "null argument");
    *ndone = 0;
    for (int round = 0;; ++round) {
        bool active = false;
        *ndone = 0;
        for (int i = 0; i < k->capacity; ++i) {
            const PackMember& x = k->m[i];
            if (x.state == PK_DONE) done[(*ndone)++] = i;
            active = active || (x.state != PK_FREE && x.state != PK_DONE);
        }
        if (*ndone > 0 || !active || (max_rounds > 0 && round >= max_rounds)) return HH_OK;
        HH_TRY(pack_round(k));
    }
}

hh_status hh_pack_take(hh_pack* k, int slot, hh_info* info) {
    if (!k || slot < 0 || slot >= k->capacity) return fail(HH_ERR_INVALID, "bad slot");
    PackMember& x = k->m[slot];
    if (x.state != PK_DONE) return fail(HH_ERR_INVALID, "the slot holds no finished solve");
    if (info) *info = x.info;
    const hh_status st = x.st;
    if (st != HH_OK && st != HH_NOT_CONVERGED) g_last_error = x.err;
    x = PackMember{};
    return st;
}

}  // extern "C"
