// Problem set-up, multigrid V-cycle, shifted-HSS preconditioner (Def. 4.1) and the
// FP64 flexible GMRES outer iteration (Sec. 5.1), behind the C ABI of include/hh.h.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
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

// Device buffers of the multigrid hierarchy in one precision.
struct Hier {
    bool ready = false;
    size_t elem = 0;                  // bytes per complex entry
    std::vector<void*> xa, xb, b, t;  // per level: ping-pong iterates, right side, residual scratch
    void* r_lo = nullptr;             // level-0 copy of the preconditioner input
    void* rhs = nullptr;              // level-0 HSS right side
    void* ca = nullptr;               // extra level-0 buffers for cycles_per_hss > 1
    void* cb = nullptr;
    void* cres = nullptr;
    cudaGraphExec_t graph = nullptr;  // one preconditioner application (the HSS loop)
    void* graph_out = nullptr;        // buffer that holds u after the graph
    long long graph_kernels = 0;      // kernel nodes in the graph
};

}  // namespace

namespace hh {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace hh

struct hh_problem {
    int device = 0;
    hh_grid grid{};
    double k = 0, delta = 0, dh = 0;
    int bc[6] = {0, 0, 0, 0, 0, 0};
    hh_options o{};
    std::vector<GridDesc> lv;
    Triple AL, AR, B, Bhat;
    cudaStream_t user = nullptr;
    cudaStream_t s = nullptr;  // the problem's own stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    Hier hier[2];
    // FP64 Krylov storage (level 0)
    long long N = 0;
    double2* V = nullptr;     // (restart+1) * N
    double2* Z = nullptr;     // restart * N
    double2* x = nullptr;     // iterate
    double2* bvec = nullptr;  // masked right side
    double2* r = nullptr;     // residual / scratch
    double2* partials = nullptr;
    double2* hbuf = nullptr;  // [hA (restart+1) | hB (restart+1) | nrm2]
    double2* ybuf = nullptr;  // back-substitution result
    double2* h_host = nullptr;  // pinned mirror of hbuf
    size_t bytes = 0;
    std::vector<void*> allocs;
};

namespace {

hh_status dmalloc(hh_problem* p, void** ptr, size_t bytes) {
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

GridDesc level_desc(const hh_problem* p, int l) {
    GridDesc g;
    g.dim = p->grid.dim;
    g.n = p->grid.n >> l;
    g.nn = g.n + 1;
    g.N = 1;
    for (int d = 0; d < g.dim; ++d) g.N *= g.nn;
    g.h = 1.0 / g.n;
    for (int s = 0; s < 6; ++s) g.dir[s] = (s < 2 * g.dim) ? (p->bc[s] == HH_BC_DIRICHLET) : 0;
    return g;
}

size_t hier_bytes(const hh_grid* grid, int levels, size_t elem) {
    size_t tot = 0;
    for (int l = 0; l < levels; ++l) {
        long long nn = (grid->n >> l) + 1;
        long long N = nn * nn * (grid->dim == 3 ? nn : 1);
        tot += 4 * (size_t)N * elem;  // xa, xb, b, t
        if (l == 0) tot += 5 * (size_t)N * elem;
    }
    return tot;
}

size_t krylov_bytes(const hh_grid* grid, int restart) {
    long long nn = grid->n + 1;
    long long N = nn * nn * (grid->dim == 3 ? nn : 1);
    size_t tot = (size_t)(2 * restart + 1) * N * 16 + 3 * (size_t)N * 16;
    tot += (size_t)(restart + 1) * hh::kRedBlocks * 16 + (2 * (restart + 1) + 1) * 16 + (restart + 1) * 16;
    return tot;
}

hh_status ensure_hier(hh_problem* p, int prec) {
    Hier& H = p->hier[prec];
    if (H.ready) return HH_OK;
    H.elem = prec == HH_C64 ? 8 : 16;
    const int L = p->o.levels;
    H.xa.assign(L, nullptr);
    H.xb.assign(L, nullptr);
    H.b.assign(L, nullptr);
    H.t.assign(L, nullptr);
    for (int l = 0; l < L; ++l) {
        const size_t nb = (size_t)p->lv[l].N * H.elem;
        HH_TRY(dmalloc(p, &H.xa[l], nb));
        HH_TRY(dmalloc(p, &H.xb[l], nb));
        HH_TRY(dmalloc(p, &H.b[l], nb));
        HH_TRY(dmalloc(p, &H.t[l], nb));
        HH_CUDA(cudaMemsetAsync(H.xa[l], 0, nb, p->s));
        HH_CUDA(cudaMemsetAsync(H.xb[l], 0, nb, p->s));
        HH_CUDA(cudaMemsetAsync(H.b[l], 0, nb, p->s));
        HH_CUDA(cudaMemsetAsync(H.t[l], 0, nb, p->s));
    }
    const size_t n0 = (size_t)p->lv[0].N * H.elem;
    HH_TRY(dmalloc(p, &H.r_lo, n0));
    HH_TRY(dmalloc(p, &H.rhs, n0));
    HH_TRY(dmalloc(p, &H.ca, n0));
    HH_TRY(dmalloc(p, &H.cb, n0));
    HH_TRY(dmalloc(p, &H.cres, n0));
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

// ------------------------------------------------------------------ V-cycle
#define HH_LAUNCH(call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return fail(HH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
struct MG {
    using V2 = hh::vec2<T>;
    hh_problem* p;
    Hier* H;
    cudaStream_t s;
    OpCoef<T> al;
    T omega;

    bool d2() const { return p->grid.dim == 2; }

    cudaError_t march(int mode, const hh::MArgs<T>& a) const {
        return d2() ? hh::launch_march2<T>(mode, a, s) : hh::launch_march3<T>(mode, a, s);
    }

    hh::MArgs<T> margs(int l, const OpCoef<T>& op) const {
        hh::MArgs<T> a{};
        a.g = p->lv[l];
        a.op = op;
        a.opd = al;
        a.omega = omega;
        a.tile_rows = p->o.tile_rows;
        return a;
    }

    // ---- level kernels: fused 2D marching kernels, composed generic kernels in 3D ----
    // x_out = x_in + omega D^{-1} (b - A_L x_in); x_in == nullptr means 0
    hh_status jacobi(int l, const V2* b, const V2* xin, V2* xout) {
        hh::MArgs<T> a = margs(l, al);
        a.x = xin;
        a.xzero = xin == nullptr;
        a.z = b;
        a.y = xout;
        HH_LAUNCH(march(hh::M_JACOBI, a));
        return HH_OK;
    }
    // two sweeps from x = 0
    hh_status jacobi2_zero(int l, const V2* b, V2* xout) {
        hh::MArgs<T> a = margs(l, al);
        a.z = b;
        a.y = xout;
        HH_LAUNCH(march(hh::M_JACOBI2_ZERO, a));
        return HH_OK;
    }
    // rc = P^T (b - A_L x)
    hh_status resid_restrict(int l, const V2* b, const V2* x, V2* rc) {
        if (d2()) {
            hh::MArgs<T> a = margs(l, al);
            a.x = x;
            a.z = b;
            a.y = rc;
            HH_LAUNCH(hh::launch_march2<T>(hh::M_RESID_RESTRICT, a, s));
        } else {
            hh::MArgs<T> a = margs(l, al);
            a.x = x;
            a.z = b;
            a.y = (V2*)H->t[l];
            a.alpha = Cx<T>{-1, 0};
            a.beta = Cx<T>{1, 0};
            HH_LAUNCH(hh::launch_march3<T>(hh::M_AXPBY, a, s));
            HH_LAUNCH(hh::launch_restrict<T>(p->lv[l + 1], (const V2*)H->t[l], rc, s));
        }
        return HH_OK;
    }
    // xout = x~ + omega D^{-1} (b - A_L x~), x~ = x + P ec
    hh_status prolong_jacobi(int l, V2* x, const V2* ec, const V2* b, V2* xout) {
        hh::MArgs<T> a = margs(l, al);
        a.x = x;
        a.ec = ec;
        a.z = b;
        a.y = xout;
        HH_LAUNCH(march(hh::M_PROLONG_JACOBI, a));
        return HH_OK;
    }
    // rhs = c1 A_R u + c2 r and the first Jacobi sweep x1 = omega D^{-1} rhs (u == nullptr: u = 0)
    hh_status hss_first(const V2* u, const V2* r, V2* rhs, V2* x1, T c1, T c2) {
        const OpCoef<T> ar = to_coef<T>(p->AR);
        hh::MArgs<T> a = margs(0, ar);
        a.x = u;
        a.xzero = u == nullptr;
        a.z = r;
        a.y = rhs;
        a.y2 = x1;
        a.alpha = Cx<T>{c1, 0};
        a.beta = Cx<T>{c2, 0};
        HH_LAUNCH(march(hh::M_HSS_FIRST, a));
        return HH_OK;
    }
    hh_status hss_rhs(const V2* u, const V2* r, V2* rhs, T c1, T c2) {
        const OpCoef<T> ar = to_coef<T>(p->AR);
        hh::MArgs<T> a = margs(0, ar);
        a.x = u;
        a.xzero = u == nullptr;
        a.z = r;
        a.y = rhs;
        a.alpha = Cx<T>{c1, 0};
        a.beta = Cx<T>{c2, 0};
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
            HH_CUDA(cudaMemsetAsync(cur, 0, (size_t)p->lv[l].N * sizeof(V2), s));
        } else if (nsweeps == 1) {
            HH_TRY(jacobi(l, b, nullptr, cur));
        } else {
            HH_TRY(jacobi2_zero(l, b, cur));
            HH_TRY(smooth(l, b, nsweeps - 2, &cur));
        }
        *out = cur;
        return HH_OK;
    }

    // One V-cycle on level l for right side b from x = 0; result buffer in *out.
    // xstart: the first pre-smoothing sweep was already done and sits in xstart.
    hh_status vcycle(int l, const V2* b, V2* xstart, V2** out) {
        const int L = p->o.levels;
        if (l == L - 1) {
            V2* x = (V2*)H->xa[l];
            if (xstart) {
                x = xstart;
                HH_TRY(smooth(l, b, p->o.nu_coarse - 1, &x));
            } else if (p->o.nu_coarse >= 1 && p->lv[l].N <= p->o.coarse_cluster_nodes && hh::coarse_fits<T>(p->lv[l])) {
                HH_LAUNCH(hh::launch_coarse_solve<T>(p->lv[l], al, b, x, p->o.nu_coarse, omega, s));
            } else {
                HH_TRY(smooth_from_zero(l, b, p->o.nu_coarse, &x));
            }
            *out = x;
            return HH_OK;
        }
        V2* x;
        if (xstart) {
            x = xstart;
            HH_TRY(smooth(l, b, p->o.nu_pre - 1, &x));
        } else {
            HH_TRY(smooth_from_zero(l, b, p->o.nu_pre, &x));
        }
        HH_TRY(resid_restrict(l, b, x, (V2*)H->b[l + 1]));
        V2* ec;
        HH_TRY(vcycle(l + 1, (const V2*)H->b[l + 1], nullptr, &ec));
        if (p->o.nu_post == 0) {
            HH_LAUNCH(hh::launch_prolong<T>(p->lv[l], ec, x, s));
        } else {
            V2* oth = other(l, x);
            HH_TRY(prolong_jacobi(l, x, ec, b, oth));
            x = oth;
            HH_TRY(smooth(l, b, p->o.nu_post - 1, &x));
        }
        *out = x;
        return HH_OK;
    }

    // cycles_per_hss V-cycles for A_L x = b; the first may start from xstart.
    hh_status mg_solve(const V2* b, V2* xstart, V2** out) {
        V2* x;
        HH_TRY(vcycle(0, b, xstart, &x));
        const long long N = p->lv[0].N;
        for (int c = 1; c < p->o.cycles_per_hss; ++c) {
            // keep x outside the level-0 ping-pong buffers the next cycle overwrites
            V2* keep = (V2*)((x == (V2*)H->ca) ? H->cb : H->ca);
            HH_CUDA(cudaMemcpyAsync(keep, x, (size_t)N * sizeof(V2), cudaMemcpyDeviceToDevice, s));
            hh::MArgs<T> a = margs(0, al);
            a.x = keep;
            a.z = b;
            a.y = (V2*)H->cres;
            a.alpha = Cx<T>{-1, 0};
            a.beta = Cx<T>{1, 0};
            HH_LAUNCH(march(hh::M_AXPBY, a));
            V2* corr;
            HH_TRY(vcycle(0, (const V2*)H->cres, nullptr, &corr));
            HH_LAUNCH(hh::launch_add<T>(keep, corr, N, s));
            x = keep;
        }
        *out = x;
        return HH_OK;
    }

    // The HSS loop of Def. 4.1 on r_lo (already in this precision); result buffer in *out.
    hh_status hss_loop(V2** out) {
        const double k = p->k;
        const T c1 = T((k - 1.0) / (k + 1.0)), c2 = T(2.0 * k / (k + 1.0));
        const int nh = n_hss(k, p->o.theta);
        const bool fuse = p->o.nu_pre >= 1 && p->o.levels >= 1 &&
                          !(p->o.levels == 1 && p->o.nu_coarse == 0);
        V2* u = nullptr;
        for (int it = 0; it < nh; ++it) {
            if (fuse) {
                // the first pre-smoothing sweep of the fine level is fused with the right side
                V2* x1 = (u == (V2*)H->xa[0]) ? (V2*)H->xb[0] : (V2*)H->xa[0];
                HH_TRY(hss_first(u, (const V2*)H->r_lo, (V2*)H->rhs, x1, c1, c2));
                HH_TRY(mg_solve((const V2*)H->rhs, x1, &u));
            } else {
                HH_TRY(hss_rhs(u, (const V2*)H->r_lo, (V2*)H->rhs, c1, c2));
                HH_TRY(mg_solve((const V2*)H->rhs, nullptr, &u));
            }
        }
        if (!u) {  // theta such that no iteration runs: u = 0
            u = (V2*)H->xa[0];
            HH_CUDA(cudaMemsetAsync(u, 0, (size_t)p->lv[0].N * sizeof(V2), s));
        }
        *out = u;
        return HH_OK;
    }
};

template <typename T>
MG<T> make_mg(hh_problem* p, int prec, cudaStream_t s) {
    MG<T> m;
    m.p = p;
    m.H = &p->hier[prec];
    m.s = s;
    m.al = to_coef<T>(p->AL);
    m.omega = T(p->o.omega);
    return m;
}

// z (c128) = shifted-HSS preconditioner of r (c128), on the problem stream.
hh_status precondition_async(hh_problem* p, const double2* r, double2* z) {
    const int prec = p->o.precision;
    HH_TRY(ensure_hier(p, prec));
    Hier& H = p->hier[prec];
    const long long N = p->lv[0].N;
    if (prec == HH_C64) {
        HH_CUDA(hh::launch_cast_d2f(r, (float2*)H.r_lo, N, p->s));
    } else {
        HH_CUDA(cudaMemcpyAsync(H.r_lo, r, (size_t)N * 16, cudaMemcpyDeviceToDevice, p->s));
    }
    void* u = nullptr;
    if (p->o.use_graphs) {
        if (!H.graph) {
            cudaGraph_t g;
            const long long k0 = hh::g_kernel_launches;
            HH_CUDA(cudaStreamBeginCapture(p->s, cudaStreamCaptureModeThreadLocal));
            hh_status st;
            if (prec == HH_C64) {
                MG<float> m = make_mg<float>(p, prec, p->s);
                float2* uo;
                st = m.hss_loop(&uo);
                u = uo;
            } else {
                MG<double> m = make_mg<double>(p, prec, p->s);
                double2* uo;
                st = m.hss_loop(&uo);
                u = uo;
            }
            cudaError_t ec = cudaStreamEndCapture(p->s, &g);
            if (st != HH_OK) {
                if (ec == cudaSuccess) cudaGraphDestroy(g);
                return st;
            }
            HH_CUDA(ec);
            cudaError_t ei = cudaGraphInstantiate(&H.graph, g, 0);
            cudaGraphDestroy(g);
            HH_CUDA(ei);
            H.graph_out = u;
            H.graph_kernels = hh::g_kernel_launches - k0;
            hh::g_kernel_launches = k0;
        }
        HH_CUDA(cudaGraphLaunch(H.graph, p->s));
        hh::g_kernel_launches += H.graph_kernels;
        u = H.graph_out;
    } else {
        if (prec == HH_C64) {
            MG<float> m = make_mg<float>(p, prec, p->s);
            float2* uo;
            HH_TRY(m.hss_loop(&uo));
            u = uo;
        } else {
            MG<double> m = make_mg<double>(p, prec, p->s);
            double2* uo;
            HH_TRY(m.hss_loop(&uo));
            u = uo;
        }
    }
    if (prec == HH_C64) {
        HH_CUDA(hh::launch_cast_f2d((const float2*)u, z, N, p->s));
    } else {
        HH_CUDA(cudaMemcpyAsync(z, u, (size_t)N * 16, cudaMemcpyDeviceToDevice, p->s));
    }
    return HH_OK;
}

// ------------------------------------------------------------------ FP64 helpers
// y = alpha (op x) + beta z  (z == nullptr: y = op x) on level l, stream st
template <typename T>
hh_status op_axpby(hh_problem* p, int l, const Triple& t, const hh::vec2<T>* x, const hh::vec2<T>* z,
                   hh::vec2<T>* y, Cx<T> alpha, Cx<T> beta, cudaStream_t st) {
    const OpCoef<T> op = to_coef<T>(t);
    hh::MArgs<T> a{};
    a.g = p->lv[l];
    a.op = op;
    a.opd = op;
    a.x = x;
    a.z = z;
    a.y = y;
    a.alpha = alpha;
    a.beta = beta;
    a.tile_rows = p->o.tile_rows;
    const int mode = z ? hh::M_AXPBY : hh::M_APPLY;
    HH_LAUNCH(p->grid.dim == 2 ? hh::launch_march2<T>(mode, a, st) : hh::launch_march3<T>(mode, a, st));
    return HH_OK;
}

hh_status apply_B(hh_problem* p, const double2* x, double2* y) {
    return op_axpby<double>(p, 0, p->B, x, nullptr, y, Cx<double>{1, 0}, Cx<double>{0, 0}, p->s);
}

// r = bvec - B x
hh_status residual_B(hh_problem* p, const double2* x, double2* r) {
    return op_axpby<double>(p, 0, p->B, x, p->bvec, r, Cx<double>{-1, 0}, Cx<double>{1, 0}, p->s);
}

// ||v||^2 into hbuf[slot] (device), and optionally fetched to the host.
hh_status norm2_dev(hh_problem* p, const double2* v, int slot) {
    HH_CUDA(hh::launch_multidot(v, 0, 1, v, p->N, p->partials, p->hbuf + slot, p->s));
    return HH_OK;
}

hh_status fetch(hh_problem* p, int count) {
    HH_CUDA(cudaMemcpyAsync(p->h_host, p->hbuf, (size_t)count * sizeof(double2), cudaMemcpyDeviceToHost, p->s));
    HH_CUDA(cudaStreamSynchronize(p->s));
    return HH_OK;
}

bool finite(double v) { return std::isfinite(v); }

// Flexible GMRES(m) with classical Gram-Schmidt applied twice (CGS2) and Givens rotations.
hh_status fgmres(hh_problem* p, double tol, hh_info* info) {
    const int m = p->o.restart;
    const long long N = p->N;
    const int nrm_slot = 2 * (m + 1);
    HH_TRY(norm2_dev(p, p->bvec, nrm_slot));
    HH_TRY(fetch(p, nrm_slot + 1));
    const double bnorm = std::sqrt(p->h_host[nrm_slot].x);
    if (!finite(bnorm)) return fail(HH_ERR_NONFINITE, "right-hand side is not finite");
    if (bnorm == 0.0) {
        HH_CUDA(cudaMemsetAsync(p->x, 0, (size_t)N * 16, p->s));
        info->rel_residual = 0.0;
        return HH_OK;
    }
    HH_TRY(residual_B(p, p->x, p->r));
    HH_TRY(norm2_dev(p, p->r, nrm_slot));
    HH_TRY(fetch(p, nrm_slot + 1));
    double beta = std::sqrt(p->h_host[nrm_slot].x);
    if (!finite(beta)) return fail(HH_ERR_NONFINITE, "initial residual is not finite");
    int its = 0;
    std::vector<zc> Hm((size_t)(m + 1) * m), g(m + 1), sn(m), y(m);
    std::vector<double> cs(m);
    auto Hc = [&](int i, int j) -> zc& { return Hm[(size_t)j * (m + 1) + i]; };
    double rel = beta / bnorm;
    while (rel > tol && its < p->o.max_outer) {
        // V_0 = r / beta
        HH_CUDA(cudaMemcpyAsync(p->V, p->r, (size_t)N * 16, cudaMemcpyDeviceToDevice, p->s));
        HH_CUDA(hh::launch_scale(p->V, 1.0 / beta, N, p->s));
        std::fill(g.begin(), g.end(), zc(0));
        g[0] = beta;
        int jend = 0;
        for (int j = 0; j < m; ++j) {
            double2* vj = p->V + (long long)j * N;
            double2* zj = p->Z + (long long)j * N;
            double2* w = p->V + (long long)(j + 1) * N;
            HH_TRY(precondition_async(p, vj, zj));
            info->hss_its += n_hss(p->k, p->o.theta);
            info->vcycles += (long long)n_hss(p->k, p->o.theta) * p->o.cycles_per_hss;
            HH_TRY(apply_B(p, zj, w));
            // CGS2: two passes of h = V^H w, w -= V h
            double2* hA = p->hbuf;
            double2* hB = p->hbuf + (m + 1);
            HH_CUDA(hh::launch_multidot(p->V, N, j + 1, w, N, p->partials, hA, p->s));
            HH_CUDA(hh::launch_multi_axpy(w, p->V, N, j + 1, hA, -1.0, N, p->s));
            HH_CUDA(hh::launch_multidot(p->V, N, j + 1, w, N, p->partials, hB, p->s));
            HH_CUDA(hh::launch_multi_axpy(w, p->V, N, j + 1, hB, -1.0, N, p->s));
            HH_TRY(norm2_dev(p, w, nrm_slot));
            HH_CUDA(hh::launch_scale_by_rnorm(w, p->hbuf + nrm_slot, N, p->s));
            HH_TRY(fetch(p, nrm_slot + 1));
            for (int i = 0; i <= j; ++i)
                Hc(i, j) = zc(p->h_host[i].x + p->h_host[m + 1 + i].x, p->h_host[i].y + p->h_host[m + 1 + i].y);
            const double hn = std::sqrt(p->h_host[nrm_slot].x);
            if (!finite(hn)) return fail(HH_ERR_NONFINITE, "Arnoldi produced a non-finite value");
            Hc(j + 1, j) = hn;
            for (int i = 0; i < j; ++i) {
                const zc t = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
                Hc(i + 1, j) = -std::conj(sn[i]) * Hc(i, j) + cs[i] * Hc(i + 1, j);
                Hc(i, j) = t;
            }
            const zc h1 = Hc(j, j), h2 = Hc(j + 1, j);
            const double den = std::hypot(std::abs(h1), std::abs(h2));
            if (std::abs(h1) == 0.0) {
                cs[j] = 0.0;
                sn[j] = 1.0;
            } else {
                cs[j] = std::abs(h1) / den;
                sn[j] = (h1 / std::abs(h1)) * std::conj(h2) / den;
            }
            Hc(j, j) = cs[j] * h1 + sn[j] * h2;
            Hc(j + 1, j) = 0.0;
            g[j + 1] = -std::conj(sn[j]) * g[j];
            g[j] = cs[j] * g[j];
            ++its;
            jend = j + 1;
            if (std::abs(g[j + 1]) / bnorm <= tol || its >= p->o.max_outer || hn == 0.0) break;
        }
        for (int i = jend - 1; i >= 0; --i) {
            zc acc = g[i];
            for (int c = i + 1; c < jend; ++c) acc -= Hc(i, c) * y[c];
            y[i] = acc / Hc(i, i);
            if (!finite(y[i].real()) || !finite(y[i].imag()))
                return fail(HH_ERR_NONFINITE, "least-squares update is not finite");
        }
        for (int i = 0; i < jend; ++i) p->h_host[i] = make_double2(y[i].real(), y[i].imag());
        HH_CUDA(cudaMemcpyAsync(p->ybuf, p->h_host, (size_t)jend * 16, cudaMemcpyHostToDevice, p->s));
        HH_CUDA(hh::launch_multi_axpy(p->x, p->Z, N, jend, p->ybuf, 1.0, N, p->s));
        HH_TRY(residual_B(p, p->x, p->r));
        HH_TRY(norm2_dev(p, p->r, nrm_slot));
        HH_TRY(fetch(p, nrm_slot + 1));
        beta = std::sqrt(p->h_host[nrm_slot].x);
        if (!finite(beta)) return fail(HH_ERR_NONFINITE, "residual is not finite");
        rel = beta / bnorm;
    }
    info->outer_its = its;
    info->rel_residual = rel;
    return rel <= tol ? HH_OK : HH_NOT_CONVERGED;
}

hh_status validate_level(const hh_problem* p, int level, int need_coarser) {
    if (!p) return fail(HH_ERR_INVALID, "null problem");
    if (level < 0 || level >= p->o.levels - need_coarser) return fail(HH_ERR_INVALID, "level out of range");
    return HH_OK;
}

hh_status validate_prec(int prec) {
    if (prec != HH_C64 && prec != HH_C128) return fail(HH_ERR_INVALID, "precision must be HH_C128 or HH_C64");
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
}

static hh_status check_args(const hh_grid* grid, double k, double delta, double dh, const int* bc,
                            const hh_options* o) {
    if (!grid || !o) return fail(HH_ERR_INVALID, "null grid or options");
    if (grid->dim != 2 && grid->dim != 3) return fail(HH_ERR_INVALID, "dim must be 2 or 3");
    if (!(k > 0) || !(delta >= 0) || !(dh > 0) || !std::isfinite(k) || !std::isfinite(delta) ||
        !std::isfinite(dh))
        return fail(HH_ERR_INVALID, "need k > 0, delta >= 0, delta_hat > 0 (finite)");
    if (o->levels < 1 || o->levels > 16) return fail(HH_ERR_INVALID, "levels must be in 1..16");
    if (grid->n < 2 || grid->n > (1 << 20)) return fail(HH_ERR_INVALID, "n out of range");
    if (grid->n % (1 << (o->levels - 1)) != 0 || (grid->n >> (o->levels - 1)) < 1)
        return fail(HH_ERR_INVALID, "n must be divisible by 2^(levels-1)");
    if (o->nu_pre < 0 || o->nu_post < 0 || o->nu_coarse < 0 || o->cycles_per_hss < 1)
        return fail(HH_ERR_INVALID, "negative sweep count or cycles_per_hss < 1");
    if (o->restart < 1 || o->restart > 63) return fail(HH_ERR_INVALID, "restart must be in 1..63");
    if (o->max_outer < 0) return fail(HH_ERR_INVALID, "max_outer < 0");
    if (!(o->theta >= 0) || !(o->omega >= 0) || !(o->omega < 2)) return fail(HH_ERR_INVALID, "theta >= 0 and 0 <= omega < 2 required");
    if (o->precision != HH_C64 && o->precision != HH_C128) return fail(HH_ERR_INVALID, "bad precision");
    if (o->coarse_cluster_nodes < 0) return fail(HH_ERR_INVALID, "coarse_cluster_nodes < 0");
    if (o->tile_rows != 0 && o->tile_rows != 2 && o->tile_rows != 4 && o->tile_rows != 8)
        return fail(HH_ERR_INVALID, "tile_rows must be 0, 2, 4 or 8");
    if (!bc) return fail(HH_ERR_INVALID, "null bc");
    for (int s = 0; s < 2 * grid->dim; ++s)
        if (bc[s] != HH_BC_SOMMERFELD && bc[s] != HH_BC_DIRICHLET) return fail(HH_ERR_INVALID, "bad boundary tag");
    return HH_OK;
}

size_t hh_footprint_bytes(const hh_grid* grid, const hh_options* o) {
    if (!grid || !o) return 0;
    const int bc0[6] = {0, 0, 0, 0, 0, 0};
    if (check_args(grid, 1.0, 0.0, 1.0, bc0, o) != HH_OK) return 0;
    return hier_bytes(grid, o->levels, o->precision == HH_C64 ? 8 : 16) + krylov_bytes(grid, o->restart);
}

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
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->s) cudaStreamDestroy(p->s);
    cudaSetDevice(cur);
    delete p;
}

hh_status hh_create_problem(const hh_grid* grid, double k, double delta, double delta_hat, const int* bc,
                            const hh_options* opts, void* cuda_stream, hh_problem** out) {
    if (!out) return fail(HH_ERR_INVALID, "null out");
    *out = nullptr;
    HH_TRY(check_args(grid, k, delta, delta_hat, bc, opts));
    hh_problem* p = new hh_problem();
    cudaGetDevice(&p->device);
    p->grid = *grid;
    p->k = k;
    p->delta = delta;
    p->dh = delta_hat;
    for (int s = 0; s < 6; ++s) p->bc[s] = s < 2 * grid->dim ? bc[s] : 0;
    p->o = *opts;
    // automatic damping: on levels where the shifted mass term dominates, D^{-1} A_L has
    // spectrum close to D^{-1} M, which reaches 9/4 in 2D and 27/8 in 3D; omega must stay
    // below 2 / 27 * 8 = 0.59 in 3D for the sweeps not to amplify smooth modes
    if (p->o.omega == 0.0) p->o.omega = grid->dim == 3 ? 0.5 : 0.6;
    p->AL = triple_AL(k, delta_hat);
    p->AR = triple_AR(k, delta_hat);
    p->B = triple_B(k, delta);
    p->Bhat = triple_B(k, delta_hat);
    for (int l = 0; l < opts->levels; ++l) p->lv.push_back(level_desc(p, l));
    p->N = p->lv[0].N;
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
    if ((st = ensure_hier(p, opts->precision)) != HH_OK) return bail(st);
    const int m = opts->restart;
    const long long N = p->N;
    if ((st = dmalloc(p, (void**)&p->V, (size_t)(m + 1) * N * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->Z, (size_t)m * N * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->x, (size_t)N * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->bvec, (size_t)N * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->r, (size_t)N * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->partials, (size_t)(m + 1) * hh::kRedBlocks * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->hbuf, (size_t)(2 * (m + 1) + 1) * 16)) != HH_OK) return bail(st);
    if ((st = dmalloc(p, (void**)&p->ybuf, (size_t)(m + 1) * 16)) != HH_OK) return bail(st);
    if (cudaMallocHost((void**)&p->h_host, (size_t)(2 * (m + 1) + 1) * 16) != cudaSuccess) {
        p->h_host = nullptr;
        return bail(fail(HH_ERR_OOM, "pinned host allocation failed"));
    }
    if (cudaMemsetAsync(p->V, 0, (size_t)(m + 1) * N * 16, p->s) != cudaSuccess ||
        cudaMemsetAsync(p->Z, 0, (size_t)m * N * 16, p->s) != cudaSuccess ||
        cudaStreamSynchronize(p->s) != cudaSuccess)
        return bail(fail(HH_ERR_CUDA, "initialisation failed"));
    *out = p;
    return HH_OK;
}

long long hh_level_nodes(const hh_problem* p, int level) {
    if (!p || level < 0 || level >= p->o.levels) return 0;
    return p->lv[level].N;
}

static hh_status solve_core(hh_problem* p, double tol, hh_info* info) {
    const long long k0 = hh::g_kernel_launches;
    hh_status st = fgmres(p, tol, info);
    info->device_bytes = p->bytes;
    info->kernel_launches += hh::g_kernel_launches - k0;
    return st;
}

hh_status hh_solve(hh_problem* p, const void* rhs, double tol, void* u, const void* x0, hh_info* info) {
    if (!p || !rhs || !u) return fail(HH_ERR_INVALID, "null argument");
    if (!(tol > 0)) return fail(HH_ERR_INVALID, "tol must be > 0");
    hh_info local{};
    hh_info* inf = info ? info : &local;
    *inf = hh_info{};
    inf->rel_residual = NAN;
    auto t0 = std::chrono::steady_clock::now();
    HH_TRY(join_in(p));
    HH_CUDA(hh::launch_mask_copy(p->lv[0], (const double2*)rhs, p->bvec, p->s));
    if (x0) {
        HH_CUDA(hh::launch_mask_copy(p->lv[0], (const double2*)x0, p->x, p->s));
    } else {
        HH_CUDA(cudaMemsetAsync(p->x, 0, (size_t)p->N * 16, p->s));
    }
    hh_status st = solve_core(p, tol, inf);
    if (st == HH_OK || st == HH_NOT_CONVERGED) {
        HH_CUDA(cudaMemcpyAsync(u, p->x, (size_t)p->N * 16, cudaMemcpyDeviceToDevice, p->s));
    } else {
        inf->rel_residual = NAN;
    }
    HH_TRY(join_out(p));
    HH_CUDA(cudaStreamSynchronize(p->s));
    inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

hh_status hh_solve_host(hh_problem* p, const void* rhs_host, double tol, void* u_host, hh_info* info) {
    if (!p || !rhs_host || !u_host) return fail(HH_ERR_INVALID, "null argument");
    if (!(tol > 0)) return fail(HH_ERR_INVALID, "tol must be > 0");
    hh_info local{};
    hh_info* inf = info ? info : &local;
    *inf = hh_info{};
    inf->rel_residual = NAN;
    auto t0 = std::chrono::steady_clock::now();
    HH_TRY(join_in(p));
    // stage the right side through r, then mask into bvec
    HH_CUDA(cudaMemcpyAsync(p->r, rhs_host, (size_t)p->N * 16, cudaMemcpyHostToDevice, p->s));
    HH_CUDA(hh::launch_mask_copy(p->lv[0], p->r, p->bvec, p->s));
    HH_CUDA(cudaMemsetAsync(p->x, 0, (size_t)p->N * 16, p->s));
    hh_status st = solve_core(p, tol, inf);
    if (st == HH_OK || st == HH_NOT_CONVERGED) {
        HH_CUDA(cudaMemcpyAsync(u_host, p->x, (size_t)p->N * 16, cudaMemcpyDeviceToHost, p->s));
    } else {
        inf->rel_residual = NAN;
    }
    HH_TRY(join_out(p));
    HH_CUDA(cudaStreamSynchronize(p->s));
    inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

// ---------------------------------------------------------------- building blocks
static Triple op_triple(const hh_problem* p, int op, bool* ok) {
    *ok = true;
    switch (op) {
        case HH_OP_K: return {1.0, 0.0, 0.0};
        case HH_OP_M: return {0.0, 1.0, 0.0};
        case HH_OP_MGAMMA: return {0.0, 0.0, 1.0};
        case HH_OP_AL: return p->AL;
        case HH_OP_AR: return p->AR;
        case HH_OP_B: return p->B;
        case HH_OP_BHAT: return p->Bhat;
        default: *ok = false; return {0.0, 0.0, 0.0};
    }
}

hh_status hh_apply(hh_problem* p, int level, int op, int precision, const void* x, void* y) {
    HH_TRY(validate_level(p, level, 0));
    HH_TRY(validate_prec(precision));
    if (!x || !y) return fail(HH_ERR_INVALID, "null vector");
    bool ok;
    Triple t = op_triple(p, op, &ok);
    if (!ok) return fail(HH_ERR_INVALID, "unknown operator");
    HH_TRY(join_in(p));
    if (precision == HH_C64) {
        HH_TRY(op_axpby<float>(p, level, t, (const float2*)x, nullptr, (float2*)y, Cx<float>{1, 0}, Cx<float>{0, 0},
                               p->s));
    } else {
        HH_TRY(op_axpby<double>(p, level, t, (const double2*)x, nullptr, (double2*)y, Cx<double>{1, 0},
                                Cx<double>{0, 0}, p->s));
    }
    return join_out(p);
}

hh_status hh_jacobi(hh_problem* p, int level, int precision, const void* b, const void* x_in, void* x_out) {
    HH_TRY(validate_level(p, level, 0));
    HH_TRY(validate_prec(precision));
    if (!b || !x_out || x_out == x_in || x_out == b) return fail(HH_ERR_INVALID, "bad vectors");
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
    if (precision == HH_C64) {
        HH_CUDA(hh::launch_prolong<float>(p->lv[level], (const float2*)ec, (float2*)x, p->s));
    } else {
        HH_CUDA(hh::launch_prolong<double>(p->lv[level], (const double2*)ec, (double2*)x, p->s));
    }
    return join_out(p);
}

hh_status hh_vcycle(hh_problem* p, int precision, const void* b, void* x) {
    HH_TRY(validate_level(p, 0, 0));
    HH_TRY(validate_prec(precision));
    if (!b || !x) return fail(HH_ERR_INVALID, "null vector");
    HH_TRY(ensure_hier(p, precision));
    HH_TRY(join_in(p));
    const size_t nb = (size_t)p->N * (precision == HH_C64 ? 8 : 16);
    if (precision == HH_C64) {
        MG<float> m = make_mg<float>(p, precision, p->s);
        float2* out;
        HH_TRY(m.vcycle(0, (const float2*)b, nullptr, &out));
        HH_CUDA(cudaMemcpyAsync(x, out, nb, cudaMemcpyDeviceToDevice, p->s));
    } else {
        MG<double> m = make_mg<double>(p, precision, p->s);
        double2* out;
        HH_TRY(m.vcycle(0, (const double2*)b, nullptr, &out));
        HH_CUDA(cudaMemcpyAsync(x, out, nb, cudaMemcpyDeviceToDevice, p->s));
    }
    return join_out(p);
}

hh_status hh_hss_rhs(hh_problem* p, int precision, const void* u, const void* r, void* rhs) {
    HH_TRY(validate_level(p, 0, 0));
    HH_TRY(validate_prec(precision));
    if (!r || !rhs) return fail(HH_ERR_INVALID, "null vector");
    const double k = p->k, c1 = (k - 1.0) / (k + 1.0), c2 = 2.0 * k / (k + 1.0);
    HH_TRY(join_in(p));
    if (precision == HH_C64) {
        MG<float> m = make_mg<float>(p, precision, p->s);
        HH_TRY(m.hss_rhs((const float2*)u, (const float2*)r, (float2*)rhs, float(c1), float(c2)));
    } else {
        MG<double> m = make_mg<double>(p, precision, p->s);
        HH_TRY(m.hss_rhs((const double2*)u, (const double2*)r, (double2*)rhs, c1, c2));
    }
    return join_out(p);
}

hh_status hh_precondition(hh_problem* p, const void* r, void* z) {
    if (!p || !r || !z) return fail(HH_ERR_INVALID, "null argument");
    HH_TRY(join_in(p));
    HH_TRY(precondition_async(p, (const double2*)r, (double2*)z));
    HH_TRY(join_out(p));
    HH_CUDA(cudaStreamSynchronize(p->s));
    return HH_OK;
}

hh_status hh_load_vector(hh_problem* p, const void* f, void* b) {
    if (!p || !f || !b) return fail(HH_ERR_INVALID, "null argument");
    HH_TRY(join_in(p));
    HH_TRY(op_axpby<double>(p, 0, Triple{0.0, 1.0, 0.0}, (const double2*)f, nullptr, (double2*)b, Cx<double>{1, 0},
                            Cx<double>{0, 0}, p->s));
    return join_out(p);
}

hh_status hh_dot(hh_problem* p, const void* x, const void* y, double* out) {
    if (!p || !x || !y || !out) return fail(HH_ERR_INVALID, "null argument");
    HH_TRY(join_in(p));
    HH_CUDA(hh::launch_multidot((const double2*)x, 0, 1, (const double2*)y, p->N, p->partials, p->hbuf, p->s));
    HH_TRY(fetch(p, 1));
    out[0] = p->h_host[0].x;
    out[1] = p->h_host[0].y;
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

}  // extern "C"
