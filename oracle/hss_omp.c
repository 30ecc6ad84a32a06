/*
 * hss_omp.c - FP64 CPU oracle of the shifted-HSS solver, in plain C with OpenMP over the
 * rows of CSR matrices.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__ (build) and the CPU legs of
 * bench.py use it; the product (the CUDA library) never links, loads or calls it, and it
 * shares no code with the CUDA library.
 *
 * It restates, step for step, the multigrid cycle, the shifted-HSS preconditioner and the
 * flexible GMRES of oracle/hh_oracle.py for grids where the Python oracle is too slow
 * (millions of nodes): the matrices themselves are assembled, element by element, by the
 * Python oracle and handed over in CSR form, so this file holds no discretisation at all.
 * What it computes (Cotter, Hope-Collins & Knook, arXiv 2506.18694):
 *   - scaled Jacobi on A_L:  x <- x + omega D^{-1} (b - A_L x),  D = diag(A_L);
 *   - one V-cycle on level l from x = 0: nu_pre sweeps, r_c = P^T (b - A_L x), the cycle
 *     on level l + 1 (nu_coarse sweeps from 0 on the coarsest level), x += P e_c,
 *     nu_post sweeps (Sec. 5.3's cycle shape with a Jacobi smoother);
 *   - cycles_per_hss cycles per inexact A_L solve, each on the residual left so far;
 *   - the shifted-HSS preconditioner of Def. 4.1: u_0 = 0, then nhss times
 *     u <- (A_L solve)( (k-1)/(k+1) A_R u + 2k/(k+1) r );
 *   - flexible GMRES(m) with right preconditioning, modified Gram-Schmidt and Givens
 *     rotations (Sec. 5.1's outer method), the true residual recomputed at the end of each
 *     restart cycle.
 * All arithmetic is complex double.  Vectors hold every node of the level; entries at
 * Dirichlet nodes stay exactly zero (their rows and columns are empty and D^{-1} is 0).
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define HSS_MAX_LEVELS 12

/* CSR matrix: nrows rows; row i's entries at rowptr[i] .. rowptr[i+1]-1, column col[],
 * value val[] (complex) or rval[] (real, used for the prolongation). */
typedef struct {
    long long nrows;
    const long long* rowptr;
    const int* col;
    const cplx* val;
    const double* rval;
} hss_csr;

typedef struct {
    int levels;
    long long N[HSS_MAX_LEVELS];         /* nodes of level l                                */
    hss_csr AL[HSS_MAX_LEVELS];          /* A_L of level l                                  */
    const cplx* dinv[HSS_MAX_LEVELS];    /* 1 / diag(A_L) at free nodes, 0 at Dirichlet ones */
    hss_csr P[HSS_MAX_LEVELS];           /* prolongation level l+1 -> l  (N_l x N_{l+1})     */
    hss_csr PT[HSS_MAX_LEVELS];          /* its transpose (restriction)                      */
    hss_csr AR;                          /* A_R on level 0                                   */
    hss_csr B;                           /* B_delta on level 0 (the outer operator)          */
    double k, omega;
    int nu_pre, nu_post, nu_coarse, cycles_per_hss, nhss;
} hss_problem;

void hss_set_threads(int t) {
    if (t > 0) omp_set_num_threads(t);
}

int hss_max_threads(void) { return omp_get_max_threads(); }

/* y = A x */
static void matvec(const hss_csr* A, const cplx* x, cplx* y) {
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < A->nrows; ++i) {
        cplx s = 0.0;
        for (long long e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e)
            s += (A->val ? A->val[e] : (cplx)A->rval[e]) * x[A->col[e]];
        y[i] = s;
    }
}

/* one sweep x_out = x_in + omega D^{-1} (b - A x_in) */
static void jacobi(const hss_problem* p, int l, const cplx* b, const cplx* xin, cplx* xout) {
    const hss_csr* A = &p->AL[l];
    const cplx* dinv = p->dinv[l];
    const double w = p->omega;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < A->nrows; ++i) {
        cplx s = 0.0;
        for (long long e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) s += A->val[e] * xin[A->col[e]];
        xout[i] = xin[i] + w * dinv[i] * (b[i] - s);
    }
}

/* work vectors of every level: x, another iterate, the residual, the coarse right side */
typedef struct {
    cplx* x[HSS_MAX_LEVELS];
    cplx* y[HSS_MAX_LEVELS];
    cplx* r[HSS_MAX_LEVELS];
    cplx* bc[HSS_MAX_LEVELS];
    cplx* ec[HSS_MAX_LEVELS];
} work;

static int work_alloc(const hss_problem* p, work* w) {
    memset(w, 0, sizeof(*w));
    for (int l = 0; l < p->levels; ++l) {
        const size_t bytes = (size_t)p->N[l] * sizeof(cplx);
        w->x[l] = malloc(bytes);
        w->y[l] = malloc(bytes);
        w->r[l] = malloc(bytes);
        w->bc[l] = malloc(bytes);
        w->ec[l] = malloc(bytes);
        if (!w->x[l] || !w->y[l] || !w->r[l] || !w->bc[l] || !w->ec[l]) return -1;
    }
    return 0;
}

static void work_free(const hss_problem* p, work* w) {
    for (int l = 0; l < p->levels; ++l) {
        free(w->x[l]);
        free(w->y[l]);
        free(w->r[l]);
        free(w->bc[l]);
        free(w->ec[l]);
    }
}

static void zero(cplx* v, long long n) {
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) v[i] = 0.0;
}

/* nu sweeps from the iterate in x (x overwritten; y is scratch) */
static void sweeps(const hss_problem* p, int l, const cplx* b, int nu, cplx* x, cplx* y) {
    for (int s = 0; s < nu; ++s) {
        jacobi(p, l, b, x, y);
        memcpy(x, y, (size_t)p->N[l] * sizeof(cplx));
    }
}

/* out = one V-cycle on A_L of level l from x = 0 for the right side b */
static void vcycle(const hss_problem* p, int l, const cplx* b, cplx* out, work* w) {
    const long long n = p->N[l];
    cplx* x = w->x[l];
    zero(x, n);
    if (l == p->levels - 1) {
        sweeps(p, l, b, p->nu_coarse, x, w->y[l]);
        memcpy(out, x, (size_t)n * sizeof(cplx));
        return;
    }
    sweeps(p, l, b, p->nu_pre, x, w->y[l]);
    /* r = b - A_L x, restricted: b_c = P^T r */
    matvec(&p->AL[l], x, w->r[l]);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) w->r[l][i] = b[i] - w->r[l][i];
    matvec(&p->PT[l], w->r[l], w->bc[l + 1]);
    cplx* ec = w->ec[l + 1];
    vcycle(p, l + 1, w->bc[l + 1], ec, w);
    matvec(&p->P[l], ec, w->y[l]);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) x[i] += w->y[l][i];
    sweeps(p, l, b, p->nu_post, x, w->y[l]);
    memcpy(out, x, (size_t)n * sizeof(cplx));
}

/* x = cycles_per_hss cycles for A_L x = b from 0, each on the residual left so far;
 * t, c are level-0 scratch */
static void mg_solve(const hss_problem* p, const cplx* b, cplx* x, cplx* t, cplx* c, work* w) {
    const long long n = p->N[0];
    vcycle(p, 0, b, x, w);
    for (int q = 1; q < p->cycles_per_hss; ++q) {
        matvec(&p->AL[0], x, t);
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < n; ++i) t[i] = b[i] - t[i];
        vcycle(p, 0, t, c, w);
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < n; ++i) x[i] += c[i];
    }
}

/* hss work: u, rhs, A_R u, and the two mg_solve scratch vectors */
typedef struct {
    cplx *u, *rhs, *aru, *t, *c;
} hwork;

static int hwork_alloc(long long n, hwork* h) {
    memset(h, 0, sizeof(*h));
    const size_t bytes = (size_t)n * sizeof(cplx);
    h->u = malloc(bytes);
    h->rhs = malloc(bytes);
    h->aru = malloc(bytes);
    h->t = malloc(bytes);
    h->c = malloc(bytes);
    return (h->u && h->rhs && h->aru && h->t && h->c) ? 0 : -1;
}

static void hwork_free(hwork* h) {
    free(h->u);
    free(h->rhs);
    free(h->aru);
    free(h->t);
    free(h->c);
}

/* one HSS step of Def. 4.1: u <- (A_L solve)(c1 A_R u + c2 r) */
static void hss_step(const hss_problem* p, const cplx* r, hwork* h, work* w) {
    const long long n = p->N[0];
    const double c1 = (p->k - 1.0) / (p->k + 1.0), c2 = 2.0 * p->k / (p->k + 1.0);
    matvec(&p->AR, h->u, h->aru);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) h->rhs[i] = c1 * h->aru[i] + c2 * r[i];
    mg_solve(p, h->rhs, h->u, h->t, h->c, w);
}

static void prec(const hss_problem* p, const cplx* r, cplx* z, hwork* h, work* w) {
    zero(h->u, p->N[0]);
    for (int it = 0; it < p->nhss; ++it) hss_step(p, r, h, w);
    memcpy(z, h->u, (size_t)p->N[0] * sizeof(cplx));
}

/* ---- entry points ---- */

int hss_vcycle(const hss_problem* p, int l, const cplx* b, cplx* x) {
    work w = {0};
    int st = -1;
    if (l >= 0 && l < p->levels && !work_alloc(p, &w)) {
        vcycle(p, l, b, x, &w);
        st = 0;
    }
    work_free(p, &w);
    return st;
}

int hss_mg_solve(const hss_problem* p, const cplx* b, cplx* x) {
    work w = {0};
    hwork h = {0};
    int st = -1;
    if (!work_alloc(p, &w) && !hwork_alloc(p->N[0], &h)) {
        mg_solve(p, b, x, h.t, h.c, &w);
        st = 0;
    }
    work_free(p, &w);
    hwork_free(&h);
    return st;
}

int hss_prec(const hss_problem* p, const cplx* r, cplx* z) {
    work w = {0};
    hwork h = {0};
    int st = -1;
    if (!work_alloc(p, &w) && !hwork_alloc(p->N[0], &h)) {
        prec(p, r, z, &h, &w);
        st = 0;
    }
    work_free(p, &w);
    hwork_free(&h);
    return st;
}

/* HSS steps u <- (A_L solve)(c1 A_R u + c2 r) from u = 0 until `seconds` have passed or
 * max_steps were taken; returns the steps taken and their wall time in *elapsed. */
long long hss_time_steps(const hss_problem* p, const cplx* r, double seconds, long long max_steps,
                         double* elapsed) {
    work w = {0};
    hwork h = {0};
    long long steps = -1;
    if (!work_alloc(p, &w) && !hwork_alloc(p->N[0], &h)) {
        zero(h.u, p->N[0]);
        const double t0 = omp_get_wtime();
        steps = 0;
        do {
            hss_step(p, r, &h, &w);
            ++steps;
        } while (steps < max_steps && omp_get_wtime() - t0 < seconds);
        *elapsed = omp_get_wtime() - t0;
    }
    work_free(p, &w);
    hwork_free(&h);
    return steps;
}

static double nrm2(const cplx* v, long long n) {
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (long long i = 0; i < n; ++i) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
    return sqrt(s);
}

/* a^H b */
static cplx vdot(const cplx* a, const cplx* b, long long n) {
    double re = 0.0, im = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : re, im)
    for (long long i = 0; i < n; ++i) {
        const cplx t = conj(a[i]) * b[i];
        re += creal(t);
        im += cimag(t);
    }
    return re + I * im;
}

/* Flexible GMRES(restart) on B x = b, right-preconditioned by the shifted-HSS operator,
 * from x (the initial guess on entry, the result on exit).  Stops when the Givens
 * estimate of the relative residual reaches tol or max_it iterations were taken; the true
 * residual ||b - B x|| / ||b|| is recomputed after every restart cycle and returned in
 * *relres (the loop goes on while it is above tol).  Returns the iterations taken, or -1
 * when memory ran out. */
int hss_fgmres(const hss_problem* p, const cplx* b, double tol, int restart, int max_it, cplx* x,
               double* relres) {
    const long long n = p->N[0];
    const int m = restart;
    const size_t vb = (size_t)n * sizeof(cplx);
    cplx* V = malloc(vb * (size_t)(m + 1));
    cplx* Z = malloc(vb * (size_t)m);
    cplx* r = malloc(vb);
    cplx* wv = malloc(vb);
    cplx* H = calloc((size_t)(m + 1) * m, sizeof(cplx));
    double* cs = calloc((size_t)m, sizeof(double));
    cplx* sn = calloc((size_t)m, sizeof(cplx));
    cplx* g = calloc((size_t)m + 1, sizeof(cplx));
    cplx* y = calloc((size_t)m, sizeof(cplx));
    work w = {0};
    hwork h = {0};
    int its = -1;
    if (!V || !Z || !r || !wv || !H || !cs || !sn || !g || !y || work_alloc(p, &w) || hwork_alloc(n, &h))
        goto out;
    its = 0;
#define HH(i, j) H[(size_t)(i) * m + (j)]
    const double bnorm = nrm2(b, n);
    if (bnorm == 0.0) {
        zero(x, n);
        *relres = 0.0;
        goto out;
    }
    matvec(&p->B, x, r);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) r[i] = b[i] - r[i];
    for (;;) {
        const double beta = nrm2(r, n);
        *relres = beta / bnorm;
        if (beta / bnorm <= tol || its >= max_it) break;
        memset(H, 0, (size_t)(m + 1) * m * sizeof(cplx));
        memset(g, 0, ((size_t)m + 1) * sizeof(cplx));
        g[0] = beta;
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < n; ++i) V[i] = r[i] / beta;
        int jend = 0;
        for (int j = 0; j < m; ++j) {
            cplx* vj = V + (size_t)j * n;
            cplx* zj = Z + (size_t)j * n;
            prec(p, vj, zj, &h, &w);
            matvec(&p->B, zj, wv);
            for (int i = 0; i <= j; ++i) { /* modified Gram-Schmidt */
                const cplx* vi = V + (size_t)i * n;
                const cplx hij = vdot(vi, wv, n);
                HH(i, j) = hij;
#pragma omp parallel for schedule(static)
                for (long long q = 0; q < n; ++q) wv[q] -= hij * vi[q];
            }
            const double hn = nrm2(wv, n);
            HH(j + 1, j) = hn;
            if (hn != 0.0) {
                cplx* vn = V + (size_t)(j + 1) * n;
#pragma omp parallel for schedule(static)
                for (long long q = 0; q < n; ++q) vn[q] = wv[q] / hn;
            }
            for (int i = 0; i < j; ++i) { /* previous rotations */
                const cplx t = cs[i] * HH(i, j) + sn[i] * HH(i + 1, j);
                HH(i + 1, j) = -conj(sn[i]) * HH(i, j) + cs[i] * HH(i + 1, j);
                HH(i, j) = t;
            }
            const cplx h1 = HH(j, j), h2 = HH(j + 1, j);
            const double den = hypot(cabs(h1), cabs(h2));
            if (cabs(h1) == 0.0) {
                cs[j] = 0.0;
                sn[j] = 1.0;
            } else {
                cs[j] = cabs(h1) / den;
                sn[j] = (h1 / cabs(h1)) * conj(h2) / den;
            }
            HH(j, j) = cs[j] * h1 + sn[j] * h2;
            HH(j + 1, j) = 0.0;
            g[j + 1] = -conj(sn[j]) * g[j];
            g[j] = cs[j] * g[j];
            ++its;
            jend = j + 1;
            if (cabs(g[j + 1]) / bnorm <= tol || its >= max_it) break;
        }
        for (int i = jend - 1; i >= 0; --i) { /* back substitution */
            cplx s = g[i];
            for (int q = i + 1; q < jend; ++q) s -= HH(i, q) * y[q];
            y[i] = s / HH(i, i);
        }
        for (int i = 0; i < jend; ++i) {
            const cplx* zi = Z + (size_t)i * n;
            const cplx yi = y[i];
#pragma omp parallel for schedule(static)
            for (long long q = 0; q < n; ++q) x[q] += yi * zi[q];
        }
        matvec(&p->B, x, r);
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < n; ++i) r[i] = b[i] - r[i];
    }
#undef HH
out:
    work_free(p, &w);
    hwork_free(&h);
    free(V);
    free(Z);
    free(r);
    free(wv);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
    return its;
}
