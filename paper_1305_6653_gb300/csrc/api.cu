// C ABI of libfde (declared in include/fde.h): problem lifecycle, BVM coefficient
// derivation, and the host driver of the flexible GMRES iteration.  All numerical
// work of the path runs in the kernels of the other translation units.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fde_internal.h"

namespace fde {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return FDE_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// launch counter and per-stage profiler
// ---------------------------------------------------------------------------
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static cudaEvent_t next_event(Problem& P) {
    if (P.ev_used == P.ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        P.ev_pool.push_back(e);
    }
    return P.ev_pool[P.ev_used++];
}

StageTimer::StageTimer(Problem& P, int stage, cudaStream_t on)
    : P_(&P), stage_(stage), st_(on ? on : P.stream) {
    if (P.prof) {
        e0_ = next_event(P);
        if (e0_) cudaEventRecord(e0_, st_);
        return;
    }
    if (!(P.prof_mask & (1u << stage))) return;
    if (P.capturing_events) {
        // inside a stream capture: an event-record node of the graph (a plain record
        // would only mark a capture dependency); the graph owns the event
        if (cudaEventCreate(&e0_) != cudaSuccess) { e0_ = nullptr; return; }
        graph_ = true;
        cudaEventRecordWithFlags(e0_, st_, cudaEventRecordExternal);
    } else {
        e0_ = next_event(P);
        if (e0_) cudaEventRecord(e0_, st_);
    }
}

StageTimer::~StageTimer() {
    if (!e0_) return;
    if (graph_) {
        cudaEvent_t e1 = nullptr;
        if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0_); return; }
        cudaEventRecordWithFlags(e1, st_, cudaEventRecordExternal);
        P_->capturing_events->push_back({stage_, e0_, e1});
        return;
    }
    cudaEvent_t e1 = next_event(*P_);
    if (!e1) return;
    cudaEventRecord(e1, st_);
    P_->prof_rec[stage_].push_back({e0_, e1});
}

// Sum the stage times recorded by the last replay of iteration graph gi (its stream
// has been synchronised).
static void harvest_graph_events(Problem& P, int gi) {
    if (gi >= (int)P.iter_graph_events.size()) return;
    for (const Problem::GraphEvent& g : P.iter_graph_events[gi]) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g.e0, g.e1) == cudaSuccess) {
            P.prof_acc_ms[g.stage] += ms;
            P.prof_acc_n[g.stage] += 1;
        }
    }
}

// ---------------------------------------------------------------------------
// exact rational arithmetic for the BVM coefficients (Sec. 2.2)
// ---------------------------------------------------------------------------
struct Rat {
    __int128 p = 0, q = 1;
};
static __int128 gcd128(__int128 a, __int128 b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b != 0) {
        __int128 t = a % b;
        a = b;
        b = t;
    }
    return a;
}
static Rat norm(Rat r) {
    if (r.q < 0) { r.p = -r.p; r.q = -r.q; }
    __int128 g = gcd128(r.p, r.q);
    if (g > 1) { r.p /= g; r.q /= g; }
    if (r.p == 0) r.q = 1;
    return r;
}
static Rat R(long v) { Rat r; r.p = v; r.q = 1; return r; }
static Rat add(Rat a, Rat b) { Rat r; r.p = a.p * b.q + b.p * a.q; r.q = a.q * b.q; return norm(r); }
static Rat sub(Rat a, Rat b) { b.p = -b.p; return add(a, b); }
static Rat mul(Rat a, Rat b) { Rat r; r.p = a.p * b.p; r.q = a.q * b.q; return norm(r); }
static Rat dvd(Rat a, Rat b) { Rat r; r.p = a.p * b.q; r.q = a.q * b.p; return norm(r); }
static double to_d(Rat a) { return (double)a.p / (double)a.q; }
static Rat ipow(long base, int e) {
    Rat r = R(1);
    for (int i = 0; i < e; ++i) r = mul(r, R(base));
    return r;
}

// Solve the (n x n) system a x = b exactly (Gauss-Jordan with a nonzero pivot).
static bool solve_exact(std::vector<std::vector<Rat>> a, std::vector<Rat> b, std::vector<Rat>& x) {
    const int n = (int)b.size();
    for (int c = 0; c < n; ++c) {
        int piv = -1;
        for (int r = c; r < n; ++r)
            if (a[r][c].p != 0) { piv = r; break; }
        if (piv < 0) return false;
        std::swap(a[c], a[piv]);
        std::swap(b[c], b[piv]);
        for (int r = 0; r < n; ++r) {
            if (r == c || a[r][c].p == 0) continue;
            Rat f = dvd(a[r][c], a[c][c]);
            for (int k = c; k < n; ++k) a[r][k] = sub(a[r][k], mul(f, a[c][k]));
            b[r] = sub(b[r], mul(f, b[c]));
        }
    }
    x.resize(n);
    for (int i = 0; i < n; ++i) x[i] = dvd(b[i], a[i][i]);
    return true;
}

static int nu_for(int family, int mu) {
    if (family == FDE_GBDF) return (mu % 2) ? (mu + 1) / 2 : mu / 2 + 1;
    if (family == FDE_GAM) return (mu % 2) ? (mu + 1) / 2 : mu / 2;
    if (family == FDE_ETR) return (mu % 2) ? (mu + 1) / 2 : -1;
    return -1;
}

// Coefficients of the mu-step formula on points 0..mu approximating u' at point ell.
// Order conditions sum_i a_i i^q = q sum_i b_i i^(q-1):
//   GBDF: b = e_ell, q = 0..mu;  GAM/ETR: a = e_ell - e_{ell-1}, q = 1..mu+1.
static bool formula(int family, int mu, int ell, double* a, double* b) {
    std::vector<Rat> av(mu + 1, R(0)), bv(mu + 1, R(0));
    const int n = mu + 1;
    std::vector<std::vector<Rat>> mat(n, std::vector<Rat>(n));
    std::vector<Rat> rhs(n), sol;
    if (family == FDE_GBDF) {
        bv[ell] = R(1);
        for (int q = 0; q <= mu; ++q) {
            for (int i = 0; i <= mu; ++i) mat[q][i] = ipow(i, q);
            rhs[q] = q == 0 ? R(0) : mul(R(q), ipow(ell, q - 1));
        }
        if (!solve_exact(mat, rhs, sol)) return false;
        av = sol;
    } else {
        av[ell] = R(1);
        av[ell - 1] = R(-1);
        for (int q = 1; q <= mu + 1; ++q) {
            for (int i = 0; i <= mu; ++i) mat[q - 1][i] = mul(R(q), ipow(i, q - 1));
            rhs[q - 1] = sub(ipow(ell, q), ipow(ell - 1, q));
        }
        if (!solve_exact(mat, rhs, sol)) return false;
        bv = sol;
    }
    for (int i = 0; i <= mu; ++i) {
        a[i] = to_d(av[i]);
        b[i] = to_d(bv[i]);
    }
    return true;
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
template <typename T>
static int dalloc(T** p, size_t count) {
    void* q = nullptr;
    const int rc = dev_alloc(&q, count * sizeof(T));
    *p = static_cast<T*>(q);
    return rc;
}

// The caller makes sure that no queued GPU work still uses p.
static void dfree(void* p) { dev_free(p); }

static void free_workspace(Problem& P) {
    dfree(P.d_V); dfree(P.d_Z); dfree(P.d_H); dfree(P.d_cs); dfree(P.d_sn); dfree(P.d_gv); dfree(P.d_y);
    P.d_V = P.d_Z = P.d_H = P.d_cs = P.d_sn = P.d_gv = P.d_y = nullptr;
    P.restart_cap = 0;
}

int ensure_workspace(Problem& P, int restart) {
    if (P.restart_cap >= restart) return FDE_OK;
    ++P.graph_gen;
    if (P.d_V) FDE_CUDA_TRY(cudaStreamSynchronize(P.stream));
    free_workspace(P);
    int rc;
    if ((rc = dalloc(&P.d_V, (size_t)(restart + 1) * P.n))) return rc;
    if ((rc = dalloc(&P.d_Z, (size_t)restart * P.n))) return rc;
    if ((rc = dalloc(&P.d_H, (size_t)(restart + 1) * restart))) return rc;
    if ((rc = dalloc(&P.d_cs, (size_t)restart))) return rc;
    if ((rc = dalloc(&P.d_sn, (size_t)restart))) return rc;
    if ((rc = dalloc(&P.d_gv, (size_t)restart + 1))) return rc;
    if ((rc = dalloc(&P.d_y, (size_t)restart))) return rc;
    P.restart_cap = restart;
    return FDE_OK;
}

int ensure_solution_buffer(Problem& P) {
    if (P.d_xsol) return FDE_OK;
    return dalloc(&P.d_xsol, (size_t)P.n);
}

// Factor planes, 1/U_ii and the frequency-domain vector in the precision's storage
// type (FP64 for FDE_FP64, FP32 otherwise); reallocated when the size changes.
int ensure_factor_buffers(Problem& P, int precision) {
    const size_t esz = precision == FDE_FP64 ? sizeof(double) : sizeof(float);
    const size_t fac_bytes = (size_t)P.nblk * 2 * P.mp * P.mp * esz;
    int rc;
    if (P.d_fac && P.fac_bytes != fac_bytes) {
        ++P.graph_gen;
        FDE_CUDA_TRY(cudaStreamSynchronize(P.stream));
        dfree(P.d_fac); dfree(P.d_dinv); dfree(P.d_rhat);
        P.d_fac = P.d_dinv = P.d_rhat = nullptr;
        P.fac_bytes = 0;
    }
    if (!P.d_fac) {
        unsigned char* f = nullptr;
        if ((rc = dalloc(&f, fac_bytes))) return rc;
        P.d_fac = f;
        P.fac_bytes = fac_bytes;
        unsigned char* dv = nullptr;
        if ((rc = dalloc(&dv, (size_t)P.nblk * P.mp * 2 * esz))) return rc;
        P.d_dinv = dv;
        unsigned char* rh = nullptr;
        if ((rc = dalloc(&rh, (size_t)P.nblk * P.mp * 2 * esz))) return rc;
        P.d_rhat = rh;
    }
    return FDE_OK;
}

static int apply_precond(Problem& P, const double* r, double* z) {
    int rc;
    if (P.precond == FDE_PRECOND_NONE) {  // plain GMRES: z = r
        StageTimer t(P, FDE_STAGE_TRSV);
        FDE_CUDA_TRY(cudaMemcpyAsync(z, r, (size_t)P.n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
        return FDE_OK;
    }
    if (P.precond != FDE_PRECOND_STRANG) {  // S^(2) / S~^(2): time FFT, circulant solves, inverse
        {
            StageTimer t(P, FDE_STAGE_TFFT_FWD);
            if ((rc = launch_time_fft_fwd(P, r, P.d_rhat_b, P.bccb_precision, P.stream))) return rc;
        }
        {
            StageTimer t(P, FDE_STAGE_TRSV);
            if ((rc = launch_bccb_solve(P, P.d_rhat_b, P.bccb_precision, P.stream))) return rc;
        }
        StageTimer t(P, FDE_STAGE_TFFT_INV);
        return launch_time_fft_inv(P, P.d_rhat_b, z, P.bccb_precision, P.stream);
    }
    {
        StageTimer t(P, FDE_STAGE_TFFT_FWD);
        if ((rc = launch_time_fft_fwd(P, r, P.d_rhat, P.precision, P.stream))) return rc;
    }
    {
        StageTimer t(P, FDE_STAGE_TRSV);
        if ((rc = launch_block_trsv(P, P.d_rhat, P.stream))) return rc;
    }
    StageTimer t(P, FDE_STAGE_TFFT_INV);
    return launch_time_fft_inv(P, P.d_rhat, z, P.precision, P.stream);
}

static int matvec(Problem& P, const double* z, double* y, bool fp32 = false) {
    StageTimer t(P, FDE_STAGE_MATVEC);
    return fp32 ? launch_matvec32(P, z, y, P.stream) : launch_matvec64(P, z, y, P.stream);
}

// ||v||^2 on the device into d_scal[slot]; optionally returned to the host (synchronises).
static int norm2(Problem& P, const double* v, int slot, double* host_out, double* pinned) {
    int rc = launch_norm(v, P.n, P.d_scal + slot, P.d_partial, P.d_counter, P.stream);
    if (rc) return rc;
    if (host_out) {
        FDE_CUDA_TRY(cudaMemcpyAsync(pinned, P.d_scal + slot, sizeof(double), cudaMemcpyDeviceToHost, P.stream));
        FDE_CUDA_TRY(cudaStreamSynchronize(P.stream));
        *host_out = *pinned;
    }
    return FDE_OK;
}

static void drop_iter_graphs(Problem& P) {
    for (cudaGraphExec_t g : P.iter_graph)
        if (g) cudaGraphExecDestroy(g);
    P.iter_graph.clear();
    P.iter_graph_launches.clear();
    for (auto& v : P.iter_graph_events)
        for (const Problem::GraphEvent& g : v) {
            cudaEventDestroy(g.e0);
            cudaEventDestroy(g.e1);
        }
    P.iter_graph_events.clear();
}

// One inner iteration j of pgmres_solve as a stream of launches: z_j = P^{-1} v_j,
// w = M z_j (Toeplitz part in FP32 when fp32), CGS2 against v_0..v_j, Hessenberg
// column / Givens rotation, w /= |w|.
static int iteration_launches(Problem& P, int j, int ldh, int reorth, bool fp32) {
    const long n = P.n;
    cudaStream_t st = P.stream;
    double* V = P.d_V;
    double* sc = P.d_scal;
    double* vj = V + (size_t)j * n;
    double* w = V + (size_t)(j + 1) * n;
    double* zj = P.d_Z + (size_t)j * n;
    int rc;
    if ((rc = apply_precond(P, vj, zj))) return rc;
    if ((rc = matvec(P, zj, w, fp32))) return rc;
    StageTimer kt(P, FDE_STAGE_KRYLOV);
    // CGS2 in three passes over V: h1 = V^T w; w -= V h1 and h2 = V^T w;
    // w -= V h2 and |w|^2 (one pass fewer without re-orthogonalisation)
    if ((rc = launch_cgs_pass(0, V, j + 1, nullptr, w, n, sc, P.d_partial, P.d_counter, st))) return rc;
    if (reorth) {
        if ((rc = launch_cgs_pass(1, V, j + 1, sc, w, n, sc + 64, P.d_partial, P.d_counter, st))) return rc;
    }
    if ((rc = launch_cgs_pass(2, V, j + 1, reorth ? sc + 64 : sc, w, n, sc + 128, P.d_partial, P.d_counter, st)))
        return rc;
    if ((rc = launch_arnoldi_finish(P.d_H, ldh, j, sc, reorth ? sc + 64 : nullptr, sc + 128, P.d_cs, P.d_sn,
                                    P.d_gv, sc + 129, st)))
        return rc;
    return launch_scale(w, sc + 128, w, n, st);
}

// Run iteration j: replay its CUDA graph or launch the kernels directly.  Graphs are
// captured only for a problem that is solved again (from its second pgmres_solve on),
// so a one-shot solve pays no capture; the stage profiler always launches directly.
static int run_iteration(Problem& P, int j, int ldh, int reorth, int restart, bool fp32, bool* replayed) {
    *replayed = false;
    if (P.prof || P.solves < 1) return iteration_launches(P, j, ldh, reorth, fp32);
    const int gi = j + (fp32 ? restart : 0);  // graph of iteration j with the FP64 / FP32 product
    const long long key = (((((long long)P.graph_gen * 8 + P.precond) * 8 + (P.precision + 1)) * 8 +
                            (P.bccb_precision + 1)) * 128 * 2 + (long long)ldh * 2 + (reorth ? 1 : 0)) *
                              (1LL << FDE_NUM_STAGES) + (long long)P.prof_mask;
    if (key != P.graph_key) {
        drop_iter_graphs(P);
        P.graph_key = key;
    }
    if ((int)P.iter_graph.size() < 2 * restart) {
        P.iter_graph.resize(2 * restart, nullptr);
        P.iter_graph_launches.resize(2 * restart, 0);
        P.iter_graph_events.resize(2 * restart);
    }
    if (!P.iter_graph[gi]) {
        if (!P.cap_stream) FDE_CUDA_TRY(cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking));
        // the capture stream follows the work already queued on P.stream
        cudaEvent_t fork;
        FDE_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        cudaEventRecord(fork, P.stream);
        cudaStreamWaitEvent(P.cap_stream, fork, 0);
        cudaEventDestroy(fork);
        cudaStream_t user = P.stream;
        P.stream = P.cap_stream;
        const long long l0 = fde_launch_count();
        std::vector<Problem::GraphEvent> events;
        cudaError_t e = cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeRelaxed);
        P.capturing_events = &events;
        int rc = e == cudaSuccess ? iteration_launches(P, j, ldh, reorth, fp32) : FDE_OK;
        P.capturing_events = nullptr;
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(P.cap_stream, &graph);
        P.stream = user;
        for (const Problem::GraphEvent& g : P.iter_graph_events[gi]) {
            cudaEventDestroy(g.e0);
            cudaEventDestroy(g.e1);
        }
        P.iter_graph_events[gi] = events;  // owned by graph gi from here on
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamBeginCapture");
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e2 != cudaSuccess) return cuda_error(e2, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
        P.iter_graph[gi] = exec;
        P.iter_graph_launches[gi] = fde_launch_count() - l0;
        // the launches were counted once while capturing; each replay adds them below
        note_launches(-P.iter_graph_launches[gi]);
    }
    FDE_CUDA_TRY(cudaGraphLaunch(P.iter_graph[gi], P.stream));
    note_launches(P.iter_graph_launches[gi]);
    *replayed = true;
    return FDE_OK;
}

}  // namespace fde

using namespace fde;

struct fde_problem {
    Problem P;
    double* pinned = nullptr;  // small pinned host buffer for device -> host scalars
};

namespace fde {
Problem* problem_of(fde_problem* h) { return h ? &h->P : nullptr; }
}  // namespace fde

extern "C" {

const char* fde_last_error(void) { return g_last_error.c_str(); }

int fde_problem_create(const fde_problem_desc* d, void* stream, fde_problem** out) {
    g_last_error.clear();
    if (!d || !out) return set_error(FDE_ERR_ARG, "desc and out must not be NULL");
    *out = nullptr;
    if (d->m < 1 || d->m > FDE_MAX_M) return set_error(FDE_ERR_ARG, "m out of range [1, FDE_MAX_M]");
    if (d->s < 2 || d->s > FDE_MAX_S || (d->s & (d->s - 1)))
        return set_error(FDE_ERR_ARG, "s must be a power of two in [2, FDE_MAX_S]");
    if (!(d->alpha > 1.0 && d->alpha < 2.0)) return set_error(FDE_ERR_ARG, "alpha must lie in (1, 2)");
    if (!(d->xR > d->xL) || !std::isfinite(d->xL) || !std::isfinite(d->xR))
        return set_error(FDE_ERR_ARG, "need finite xL < xR");
    if (!(d->T > d->t0) || !std::isfinite(d->t0) || !std::isfinite(d->T))
        return set_error(FDE_ERR_ARG, "need finite t0 < T");
    if (d->mu < 1 || d->mu > FDE_MAX_MU) return set_error(FDE_ERR_ARG, "mu out of range [1, FDE_MAX_MU]");
    const int nu = nu_for(d->family, d->mu);
    if (nu < 0) return set_error(FDE_ERR_ARG, "unknown BVM family or ETR with even mu");
    if (d->s < 2 * d->mu) return set_error(FDE_ERR_ARG, "need s >= 2*mu");
    if (!d->u0 || !d->f) return set_error(FDE_ERR_ARG, "u0 and f must not be NULL");

    fde_problem* h = new (std::nothrow) fde_problem();
    if (!h) return set_error(FDE_ERR_ALLOC, "host allocation failed");
    Problem& P = h->P;
    P.m = d->m;
    P.s = d->s;
    P.mu = d->mu;
    P.nu = nu;
    P.family = d->family;
    P.alpha = d->alpha;
    P.xL = d->xL; P.xR = d->xR; P.t0 = d->t0; P.T = d->T;
    P.dx = (d->xR - d->xL) / (d->m + 1);
    P.h = (d->T - d->t0) / d->s;
    P.dxa = std::pow(P.dx, -d->alpha);
    P.L = 1;
    while (P.L < 2 * P.m) P.L <<= 1;
    if (P.L < 2) P.L = 2;
    P.logL = ilog2(P.L);
    P.logs = ilog2(P.s);
    P.nblk = P.s / 2 + 1;
    P.mp = round_up(P.m, 64);
    P.n = (long)P.m * P.s;
    P.stream = (cudaStream_t)stream;
    P.device_ptrs = d->device_ptrs != 0;

    // BVM band rows t = 1..s (eqs. (1.7)-(1.9)); row 0 is the initial condition.
    std::vector<double> ha((size_t)(P.s + 1) * (P.mu + 1), 0.0), hb((size_t)(P.s + 1) * (P.mu + 1), 0.0);
    std::vector<int> hst(P.s + 1, 0);
    ha[0] = 1.0;
    for (int t = 1; t <= P.s; ++t) {
        int st;
        if (t < nu) st = 0;
        else if (t <= P.s - P.mu + nu) st = t - nu;
        else st = P.s - P.mu;
        hst[t] = st;
        if (!formula(P.family, P.mu, t - st, &ha[(size_t)t * (P.mu + 1)], &hb[(size_t)t * (P.mu + 1)])) {
            delete h;
            return set_error(FDE_ERR_ARG, "BVM order conditions are singular");
        }
    }
    if (!formula(P.family, P.mu, nu, P.h_a_main, P.h_b_main)) {
        delete h;
        return set_error(FDE_ERR_ARG, "BVM order conditions are singular");
    }
    for (int t = 0; t <= P.s; ++t) P.h_start[t] = hst[t];

    // validate coefficient arrays on the host when they are host pointers
    const size_t m = P.m;
    std::vector<double> dp(m), dm(m);
    auto fetch = [&](const double* src, double cval, std::vector<double>& dst) -> int {
        if (!src) {
            for (size_t i = 0; i < m; ++i) dst[i] = cval;
            return FDE_OK;
        }
        if (d->device_ptrs) {
            cudaError_t e = cudaMemcpy(dst.data(), src, m * sizeof(double), cudaMemcpyDefault);
            if (e != cudaSuccess) return cuda_error(e, "copy of d+/d-");
        } else {
            std::memcpy(dst.data(), src, m * sizeof(double));
        }
        return FDE_OK;
    };
    int rc;
    if ((d->dplus_t == nullptr) != (d->dminus_t == nullptr)) {
        delete h;
        return set_error(FDE_ERR_ARG, "give both dplus_t and dminus_t or neither");
    }
    P.timevar = d->dplus_t != nullptr;
    std::vector<double> dpt, dmt;  // time-dependent coefficients, (s+1) x m
    if (P.timevar) {
        const size_t cnt = (size_t)(P.s + 1) * m;
        dpt.resize(cnt);
        dmt.resize(cnt);
        for (int w = 0; w < 2; ++w) {
            const double* src = w == 0 ? d->dplus_t : d->dminus_t;
            double* dst = w == 0 ? dpt.data() : dmt.data();
            if (d->device_ptrs) {
                cudaError_t e = cudaMemcpy(dst, src, cnt * sizeof(double), cudaMemcpyDefault);
                if (e != cudaSuccess) {
                    delete h;
                    return cuda_error(e, "copy of dplus_t/dminus_t");
                }
            } else {
                std::memcpy(dst, src, cnt * sizeof(double));
            }
        }
        for (size_t k = 0; k < cnt; ++k) {
            if (!(dpt[k] >= 0.0) || !(dmt[k] >= 0.0) || !(dpt[k] + dmt[k] > 0.0) || !std::isfinite(dpt[k]) ||
                !std::isfinite(dmt[k])) {
                delete h;
                return set_error(FDE_ERR_ARG,
                                 "need d+ >= 0, d- >= 0, d+ + d- != 0 and finite at every point and time level");
            }
        }
        // the preconditioners use the means over the unknown time levels n = 1..s
        for (size_t i = 0; i < m; ++i) {
            double sp = 0.0, sm = 0.0;
            for (int n = 1; n <= P.s; ++n) {
                sp += dpt[(size_t)n * m + i];
                sm += dmt[(size_t)n * m + i];
            }
            dp[i] = sp / P.s;
            dm[i] = sm / P.s;
        }
    } else if ((rc = fetch(d->dplus, d->dplus_c, dp)) || (rc = fetch(d->dminus, d->dminus_c, dm))) {
        delete h;
        return rc;
    }
    for (size_t i = 0; i < m; ++i) {
        if (!(dp[i] >= 0.0) || !(dm[i] >= 0.0) || !(dp[i] + dm[i] > 0.0) || !std::isfinite(dp[i]) ||
            !std::isfinite(dm[i])) {
            delete h;
            return set_error(FDE_ERR_ARG, "need d+ >= 0, d- >= 0, d+ + d- != 0 and finite at every point");
        }
    }
    if (!d->device_ptrs) {
        for (size_t i = 0; i < m; ++i)
            if (!std::isfinite(d->u0[i])) { delete h; return set_error(FDE_ERR_ARG, "u0 is not finite"); }
        for (size_t i = 0; i < (size_t)(P.s + 1) * m; ++i)
            if (!std::isfinite(d->f[i])) { delete h; return set_error(FDE_ERR_ARG, "f is not finite"); }
    }

#define TRY(x)            \
    do {                  \
        rc = (x);         \
        if (rc) {         \
            fde_problem_destroy(h); \
            return rc;    \
        }                 \
    } while (0)
    TRY(dalloc(&P.d_start, P.s + 1));
    TRY(dalloc(&P.d_a, ha.size()));
    TRY(dalloc(&P.d_b, hb.size()));
    TRY(dalloc(&P.d_dplus, m));
    TRY(dalloc(&P.d_dminus, m));
    TRY(dalloc(&P.d_u0, m));
    TRY(dalloc(&P.d_f, (size_t)(P.s + 1) * m));
    TRY(dalloc(&P.d_g, m + 2));
    TRY(dalloc(&P.d_twL, (size_t)P.L + 1));
    TRY(dalloc(&P.d_twL32, (size_t)P.L + 1));
    TRY(dalloc(&P.d_sym, (size_t)P.L));
    TRY(dalloc(&P.d_sym32, (size_t)P.L));
    TRY(dalloc(&P.d_tws, (size_t)P.s / 2 + 1));
    TRY(dalloc(&P.d_tws32, (size_t)P.s / 2 + 1));
    TRY(dalloc(&P.d_phi, (size_t)P.nblk));
    TRY(dalloc(&P.d_psi, (size_t)P.nblk));
    TRY(dalloc(&P.d_b_rhs, (size_t)P.n));
    TRY(dalloc(&P.d_work, (size_t)P.n));
    TRY(dalloc(&P.d_scal, 256));
    TRY(dalloc(&P.d_partial, (size_t)304 * 64));
    TRY(dalloc(&P.d_counter, 4));
    TRY(dalloc(&P.d_info, (size_t)P.nblk));
    TRY(dalloc(&P.d_err, 1));
    if (P.timevar) {
        TRY(dalloc(&P.d_dplus_t, (size_t)(P.s + 1) * m));
        TRY(dalloc(&P.d_dminus_t, (size_t)(P.s + 1) * m));
        TRY(dalloc(&P.d_jz, (size_t)P.n));
    }
    if (cudaMallocHost((void**)&h->pinned, 64 * sizeof(double)) != cudaSuccess) {
        h->pinned = nullptr;
        fde_problem_destroy(h);
        return set_error(FDE_ERR_ALLOC, "cudaMallocHost failed");
    }
    cudaStream_t st = P.stream;
    const cudaMemcpyKind kind = cudaMemcpyDefault;
#define CUTRY(x)                                  \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) {                  \
            rc = cuda_error(e_, #x);              \
            fde_problem_destroy(h);               \
            return rc;                            \
        }                                         \
    } while (0)
    CUTRY(cudaMemcpyAsync(P.d_start, hst.data(), (P.s + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    CUTRY(cudaMemcpyAsync(P.d_a, ha.data(), ha.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CUTRY(cudaMemcpyAsync(P.d_b, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CUTRY(cudaMemcpyAsync(P.d_dplus, dp.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
    CUTRY(cudaMemcpyAsync(P.d_dminus, dm.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
    CUTRY(cudaMemcpyAsync(P.d_u0, d->u0, m * sizeof(double), kind, st));
    CUTRY(cudaMemcpyAsync(P.d_f, d->f, (size_t)(P.s + 1) * m * sizeof(double), kind, st));
    if (P.timevar) {
        CUTRY(cudaMemcpyAsync(P.d_dplus_t, dpt.data(), dpt.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        CUTRY(cudaMemcpyAsync(P.d_dminus_t, dmt.data(), dmt.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    CUTRY(cudaMemsetAsync(P.d_counter, 0, 4 * sizeof(unsigned int), st));
    CUTRY(cudaMemsetAsync(P.d_scal, 0, 256 * sizeof(double), st));
    // host vectors go out of scope: wait for the copies
    CUTRY(cudaStreamSynchronize(st));
#undef CUTRY
#undef TRY
    *out = h;
    return FDE_OK;
}

void fde_problem_destroy(fde_problem* h) {
    if (!h) return;
    Problem& P = h->P;
    if (P.stream) cudaStreamSynchronize(P.stream);
    else cudaDeviceSynchronize();
    if (P.lu_hi) cudaStreamSynchronize(P.lu_hi);
    if (P.lu_lo) cudaStreamSynchronize(P.lu_lo);
    if (P.lu_x) cudaStreamSynchronize(P.lu_x);
    free_workspace(P);
    void* bufs[] = {P.d_start, P.d_a, P.d_b, P.d_dplus, P.d_dminus, P.d_u0, P.d_f, P.d_g, P.d_twL, P.d_twL32,
                    P.d_sym, P.d_sym32, P.d_tws, P.d_tws32, P.d_phi, P.d_psi, P.d_b_rhs, P.d_work, P.d_rhat,
                    P.d_fac, P.d_dinv, P.d_info, P.d_err, P.d_pack, P.d_tinv, P.d_dtile, P.d_strips, P.d_scal, P.d_partial,
                    P.d_counter, P.d_bccb_K64, P.d_bccb_K32, P.d_rhat_b, P.d_dplus_t, P.d_dminus_t,
                    P.d_jz, P.d_xsol};
    for (void* b : bufs) dfree(b);
    if (h->pinned) cudaFreeHost(h->pinned);
    for (cudaEvent_t e : P.ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : P.lu_ev)
        if (e) cudaEventDestroy(e);
    if (P.lu_hi) cudaStreamDestroy(P.lu_hi);
    if (P.lu_lo) cudaStreamDestroy(P.lu_lo);
    if (P.lu_x) cudaStreamDestroy(P.lu_x);
    drop_iter_graphs(P);
    if (P.cap_stream) cudaStreamDestroy(P.cap_stream);
    delete h;
}

long long fde_launch_count(void) { return g_launches.load(); }

int fde_release_cached_memory(void) { return dev_release_cached(); }

static void profile_reset(Problem& P) {
    if (P.stream) cudaStreamSynchronize(P.stream);
    else cudaDeviceSynchronize();
    for (auto& r : P.prof_rec) r.clear();
    P.ev_used = 0;
    for (int k = 0; k < FDE_NUM_STAGES; ++k) {
        P.prof_acc_ms[k] = 0.0;
        P.prof_acc_n[k] = 0;
    }
}

int fde_profile_enable(fde_problem* h, int on) {
    if (!h) return set_error(FDE_ERR_ARG, "NULL problem");
    Problem& P = h->P;
    profile_reset(P);
    P.prof = on != 0;
    P.prof_mask = 0;
    return FDE_OK;
}

int fde_profile_select(fde_problem* h, unsigned stage_mask) {
    if (!h) return set_error(FDE_ERR_ARG, "NULL problem");
    if (stage_mask >> FDE_NUM_STAGES) return set_error(FDE_ERR_ARG, "stage mask has bits beyond FDE_NUM_STAGES");
    Problem& P = h->P;
    profile_reset(P);
    P.prof = false;
    P.prof_mask = stage_mask;
    return FDE_OK;
}

int fde_profile_read(fde_problem* h, int stage, double* total_ms, int* launches) {
    if (!h || stage < 0 || stage >= FDE_NUM_STAGES) return set_error(FDE_ERR_ARG, "bad problem or stage");
    Problem& P = h->P;
    FDE_CUDA_TRY(cudaStreamSynchronize(P.stream));
    double tot = P.prof_acc_ms[stage];
    for (auto& pr : P.prof_rec[stage]) {
        float ms = 0.f;
        FDE_CUDA_TRY(cudaEventElapsedTime(&ms, pr.first, pr.second));
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = (int)P.prof_rec[stage].size() + P.prof_acc_n[stage];
    return FDE_OK;
}

int fde_problem_sizes(const fde_problem* h, int* m, int* s, int* nblocks) {
    if (!h) return set_error(FDE_ERR_ARG, "NULL problem");
    if (m) *m = h->P.m;
    if (s) *s = h->P.s;
    if (nblocks) *nblocks = h->P.nblk;
    return FDE_OK;
}

int bvm_assemble(fde_problem* h) {
    g_last_error.clear();
    if (!h) return set_error(FDE_ERR_ARG, "NULL problem");
    Problem& P = h->P;
    int rc;
    double* d_main = nullptr;
    StageTimer timer(P, FDE_STAGE_ASSEMBLE);
    if ((rc = launch_grunwald(P.alpha, P.m + 2, P.d_g, P.stream))) return rc;
    if ((rc = launch_twiddles(P.L, P.L, P.d_twL, P.d_twL32, P.stream))) return rc;      // L + 1 allocated
    if ((rc = launch_twiddles(P.s, P.s / 2, P.d_tws, P.d_tws32, P.stream))) return rc;  // s/2 + 1 allocated
    if ((rc = launch_toeplitz_symbol(P.d_g, P.m, P.L, P.dxa, P.d_twL, P.d_sym, P.d_sym32, nullptr, P.stream)))
        return rc;
    // main-formula coefficients for the Strang symbols
    if ((rc = dalloc(&d_main, 2 * (FDE_MAX_MU + 1)))) return rc;
    double hm[2 * (FDE_MAX_MU + 1)];
    for (int i = 0; i <= P.mu; ++i) {
        hm[i] = P.h_a_main[i];
        hm[FDE_MAX_MU + 1 + i] = P.h_b_main[i];
    }
    cudaError_t e = cudaMemcpyAsync(d_main, hm, sizeof(hm), cudaMemcpyHostToDevice, P.stream);
    if (e == cudaSuccess)
        rc = launch_strang_symbols(d_main, d_main + FDE_MAX_MU + 1, P.mu, P.nu, P.s, P.d_phi, P.d_psi, P.stream);
    else
        rc = cuda_error(e, "copy of BVM coefficients");
    if (!rc) {
        e = cudaStreamSynchronize(P.stream);  // hm is a stack buffer; d_main is freed below
        if (e != cudaSuccess) rc = cuda_error(e, "bvm_assemble");
    }
    cudaFree(d_main);
    if (rc) return rc;
    // J u0 (one Toeplitz-like apply), then b
    // J u_0 (with time-dependent coefficients: J_0, the coefficients of time level 0)
    if (P.timevar)
        rc = launch_japply64_d(P, P.d_u0, P.d_work, 1, P.d_dplus_t, P.d_dminus_t, 0, P.stream);
    else
        rc = launch_japply64(P, P.d_u0, P.d_work, 1, P.stream);
    if (rc) return rc;
    if ((rc = launch_rhs(P, P.d_work, P.stream))) return rc;
    FDE_CUDA_TRY(cudaGetLastError());
    P.assembled = true;
    // first problem of this shape: time the launch shapes of the space-time product
    return autotune_matvec(P);
}

int fde_factor_storage(fde_problem* h, int storage) {
    g_last_error.clear();
    if (!h) return set_error(FDE_ERR_ARG, "NULL problem");
    if (storage != FDE_STORAGE_FP32 && storage != FDE_STORAGE_BF16)
        return set_error(FDE_ERR_ARG, "storage must be FDE_STORAGE_FP32 or FDE_STORAGE_BF16");
    h->P.strip_storage = storage;
    return FDE_OK;
}

int strang_precond_factor(fde_problem* h, int precision) {
    g_last_error.clear();
    if (!h) return set_error(FDE_ERR_ARG, "NULL problem");
    Problem& P = h->P;
    if (!P.assembled) return set_error(FDE_ERR_STATE, "bvm_assemble must run before strang_precond_factor");
    if (precision != FDE_FP64 && precision != FDE_FP32 && precision != FDE_TF32 && precision != FDE_BF16 &&
        precision != FDE_TF32X3)
        return set_error(FDE_ERR_ARG, "precision must be FDE_FP64, FDE_FP32, FDE_TF32, FDE_BF16 or FDE_TF32X3");
    int rc = ensure_factor_buffers(P, precision);
    if (rc) return rc;
    P.factored = false;
    P.precision = precision;
    FDE_CUDA_TRY(cudaMemsetAsync(P.d_info, 0, P.nblk * sizeof(int), P.stream));
    FDE_CUDA_TRY(cudaMemsetAsync(P.d_err, 0, sizeof(int), P.stream));
    if ((rc = launch_block_lu(P, precision, P.stream))) return rc;
    std::vector<int> info(P.nblk);
    int derr = 0;
    FDE_CUDA_TRY(cudaMemcpyAsync(info.data(), P.d_info, P.nblk * sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    FDE_CUDA_TRY(cudaMemcpyAsync(&derr, P.d_err, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    FDE_CUDA_TRY(cudaStreamSynchronize(P.stream));
    if (derr) return set_error(FDE_ERR_TIMEOUT, "a bounded wait in the tensor-core LU update ran out");
    for (int k = 0; k < P.nblk; ++k)
        if (info[k]) {
            char buf[128];
            std::snprintf(buf, sizeof buf, "zero or non-finite pivot in Strang block %d at row %d", k, info[k] - 1);
            return set_error(FDE_ERR_SINGULAR, buf);
        }
    P.factored = true;
    P.precond = FDE_PRECOND_STRANG;
    // first factors of this shape: time the launch shapes of the block solves
    return autotune_trsv(P);
}

int bccb_precond_setup(fde_problem* h, int modified, int precision) {
    g_last_error.clear();
    if (!h) return set_error(FDE_ERR_ARG, "NULL problem");
    Problem& P = h->P;
    if (!P.assembled) return set_error(FDE_ERR_STATE, "bvm_assemble must run before bccb_precond_setup");
    if (precision != FDE_FP64 && precision != FDE_FP32)
        return set_error(FDE_ERR_ARG, "the BCCB apply runs in FDE_FP64 or FDE_FP32");
    if (P.L < 2 * P.m) return set_error(FDE_ERR_ARG, "the BCCB apply needs the FFT length L >= 2m");
    const int nk = P.nblk, m = P.m;
    int rc;
    P.factored = false;
    if (!P.d_bccb_K64) {
        if ((rc = dalloc(&P.d_bccb_K64, (size_t)nk * P.L))) return rc;
        if ((rc = dalloc(&P.d_bccb_K32, (size_t)nk * P.L))) return rc;
    }
    if (P.d_rhat_b && P.rhat_b_prec != precision) {
        ++P.graph_gen;
        FDE_CUDA_TRY(cudaStreamSynchronize(P.stream));
        dfree(P.d_rhat_b);
        P.d_rhat_b = nullptr;
    }
    if (!P.d_rhat_b) {
        unsigned char* rb = nullptr;
        const size_t esz = precision == FDE_FP64 ? sizeof(double) : sizeof(float);
        if ((rc = dalloc(&rb, (size_t)nk * P.mp * 2 * esz))) return rc;
        FDE_CUDA_TRY(cudaMemsetAsync(rb, 0, (size_t)nk * P.mp * 2 * esz, P.stream));
        P.d_rhat_b = rb;
        P.rhat_b_prec = precision;
    }
    // Re(phi_{s-1}) = Re(phi_1) = sum_r alpha_{r+nu} cos(2 pi r / s) (Sec. 3.1)
    double phi0_mod = 0.0;
    for (int r = -P.nu; r <= P.mu - P.nu; ++r) phi0_mod += P.h_a_main[r + P.nu] * std::cos(2.0 * M_PI * r / P.s);
    double* c = nullptr;
    double2 *tw = nullptr, *mu = nullptr, *cinv = nullptr;
    if ((rc = dalloc(&c, m)) || (rc = dalloc(&tw, m)) || (rc = dalloc(&mu, m)) ||
        (rc = dalloc(&cinv, (size_t)nk * m))) {
        dfree(c); dfree(tw); dfree(mu); dfree(cinv);
        return rc;
    }
    FDE_CUDA_TRY(cudaMemsetAsync(P.d_err, 0, sizeof(int), P.stream));
    rc = launch_bccb_setup(P, modified ? 1 : 0, phi0_mod, c, tw, mu, cinv, P.d_bccb_K64, P.d_bccb_K32, P.d_err,
                           P.stream);
    int singular = 0;
    cudaError_t e = cudaMemcpyAsync(&singular, P.d_err, sizeof(int), cudaMemcpyDeviceToHost, P.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P.stream);
    dfree(c); dfree(tw); dfree(mu); dfree(cinv);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_error(e, "bccb_precond_setup");
    if (singular) return set_error(FDE_ERR_SINGULAR, "the BCCB preconditioner has a zero eigenvalue");
    P.bccb_precision = precision;
    P.precond = modified ? FDE_PRECOND_BCCB_MODIFIED : FDE_PRECOND_BCCB;
    P.factored = true;
    return FDE_OK;
}

int fde_precond_none(fde_problem* h) {
    g_last_error.clear();
    if (!h) return set_error(FDE_ERR_ARG, "NULL problem");
    Problem& P = h->P;
    if (!P.assembled) return set_error(FDE_ERR_STATE, "bvm_assemble must run before fde_precond_none");
    P.precond = FDE_PRECOND_NONE;
    P.factored = true;
    return FDE_OK;
}

int fde_matvec(fde_problem* h, const double* z, double* y) {
    g_last_error.clear();
    if (!h || !z || !y) return set_error(FDE_ERR_ARG, "NULL argument");
    if (!h->P.assembled) return set_error(FDE_ERR_STATE, "bvm_assemble must run first");
    return matvec(h->P, z, y);
}

int fde_matvec_fp32(fde_problem* h, const double* z, double* y) {
    g_last_error.clear();
    if (!h || !z || !y) return set_error(FDE_ERR_ARG, "NULL argument");
    if (!h->P.assembled) return set_error(FDE_ERR_STATE, "bvm_assemble must run first");
    return matvec(h->P, z, y, true);
}

int fde_precond_apply(fde_problem* h, const double* r, double* z) {
    g_last_error.clear();
    if (!h || !r || !z) return set_error(FDE_ERR_ARG, "NULL argument");
    if (!h->P.factored) return set_error(FDE_ERR_STATE, "strang_precond_factor must run first");
    return apply_precond(h->P, r, z);
}

int fde_get_rhs(fde_problem* h, double* b) {
    g_last_error.clear();
    if (!h || !b) return set_error(FDE_ERR_ARG, "NULL argument");
    if (!h->P.assembled) return set_error(FDE_ERR_STATE, "bvm_assemble must run first");
    FDE_CUDA_TRY(cudaMemcpyAsync(b, h->P.d_b_rhs, h->P.n * sizeof(double), cudaMemcpyDeviceToDevice, h->P.stream));
    return FDE_OK;
}

int fde_get_grunwald(fde_problem* h, double* g) {
    g_last_error.clear();
    if (!h || !g) return set_error(FDE_ERR_ARG, "NULL argument");
    if (!h->P.assembled) return set_error(FDE_ERR_STATE, "bvm_assemble must run first");
    FDE_CUDA_TRY(cudaMemcpyAsync(g, h->P.d_g, (h->P.m + 2) * sizeof(double), cudaMemcpyDeviceToHost, h->P.stream));
    FDE_CUDA_TRY(cudaStreamSynchronize(h->P.stream));
    return FDE_OK;
}

int fde_get_factor_block(fde_problem* h, int k, double* re, double* im) {
    g_last_error.clear();
    if (!h || !re || !im) return set_error(FDE_ERR_ARG, "NULL argument");
    Problem& P = h->P;
    if (!P.factored || P.precond != FDE_PRECOND_STRANG)
        return set_error(FDE_ERR_STATE, "strang_precond_factor must run first");
    if (k < 0 || k >= P.nblk) return set_error(FDE_ERR_ARG, "block index out of range");
    const size_t mp2 = (size_t)P.mp * P.mp;
    const bool f64 = P.precision == FDE_FP64;
    const size_t esz = f64 ? 8 : 4;
    std::vector<unsigned char> buf(2 * mp2 * esz);
    const unsigned char* src = (const unsigned char*)P.d_fac + (size_t)k * 2 * mp2 * esz;
    FDE_CUDA_TRY(cudaMemcpyAsync(buf.data(), src, buf.size(), cudaMemcpyDeviceToHost, P.stream));
    FDE_CUDA_TRY(cudaStreamSynchronize(P.stream));
    for (int i = 0; i < P.m; ++i)
        for (int j = 0; j < P.m; ++j) {
            const size_t e = (size_t)i * P.mp + j;
            if (f64) {
                re[(size_t)i * P.m + j] = ((const double*)buf.data())[e];
                im[(size_t)i * P.m + j] = ((const double*)buf.data())[mp2 + e];
            } else {
                re[(size_t)i * P.m + j] = ((const float*)buf.data())[e];
                im[(size_t)i * P.m + j] = ((const float*)buf.data())[mp2 + e];
            }
        }
    return FDE_OK;
}

int pgmres_solve(fde_problem* h, const fde_pgmres_opts* opts, const double* x0_arg, double* x_arg,
                 fde_stats* stats) {
    g_last_error.clear();
    if (!h || !x_arg) return set_error(FDE_ERR_ARG, "NULL argument");
    Problem& P = h->P;
    if (!P.factored) return set_error(FDE_ERR_STATE, "strang_precond_factor must run before pgmres_solve");
    fde_pgmres_opts o{1e-10, 20, 1000, 1, FDE_FP64, 0.0};
    if (opts) o = *opts;
    if (!(o.tol > 0.0) || o.restart < 1 || o.restart > 63 || o.maxit < 1)
        return set_error(FDE_ERR_ARG, "need tol > 0, 1 <= restart <= 63, maxit >= 1");
    if ((o.matvec_precision != FDE_FP64 && o.matvec_precision != FDE_FP32) || !(o.relax >= 0.0))
        return set_error(FDE_ERR_ARG, "matvec_precision must be FDE_FP64 or FDE_FP32, relax >= 0");
    int rc = ensure_workspace(P, o.restart);
    if (rc) return rc;
    cudaStream_t st = P.stream;
    const long n = P.n;
    double* pin = h->pinned;
    // Host solve vectors (desc->device_ptrs == 0): the iteration runs on the device copy
    // d_xsol; x0 is copied in first and the solution copied out at the end, on the stream.
    const bool host_x = !P.device_ptrs;
    double* x = x_arg;
    const double* x0 = x0_arg;
    if (host_x) {
        if ((rc = ensure_solution_buffer(P))) return rc;
        x = P.d_xsol;
        if (x0_arg) {
            FDE_CUDA_TRY(cudaMemcpyAsync(P.d_xsol, x0_arg, n * sizeof(double), cudaMemcpyHostToDevice, st));
            x0 = P.d_xsol;
        }
    }
    FDE_CUDA_TRY(cudaMemsetAsync(P.d_err, 0, sizeof(int), st));  // bounded-wait flag of the block solves
    cudaEvent_t ev0, ev1;
    FDE_CUDA_TRY(cudaEventCreate(&ev0));
    FDE_CUDA_TRY(cudaEventCreate(&ev1));
    FDE_CUDA_TRY(cudaEventRecord(ev0, st));

    fde_stats S;
    std::memset(&S, 0, sizeof S);
    S.precision = P.precision;
    double* V = P.d_V;
    double* Z = P.d_Z;
    double* sc = P.d_scal;
    const int ldh = o.restart + 1;
    int status = FDE_OK;
    double bnorm2 = 0, beta2 = 0;

    auto finish = [&](int code) -> int {
        int derr = 0;  // a bounded wait of the block solves ran out
        if (cudaMemcpyAsync(&derr, P.d_err, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess && derr && code == FDE_OK)
            code = set_error(FDE_ERR_TIMEOUT, "a bounded wait in the block solves ran out");
        if (host_x) {  // the solution (or last iterate) back to the caller's host array
            cudaError_t e = cudaMemcpyAsync(x_arg, x, n * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess && code == FDE_OK) code = cuda_error(e, "copy of the solution to the host");
        }
        cudaEventRecord(ev1, st);
        cudaEventSynchronize(ev1);
        float ms = 0;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        S.ms_solve = ms;
        S.status = code;
        if (stats) *stats = S;
        return code;
    };

    if (x0 && x0 != x) {
        cudaError_t e = cudaMemcpyAsync(x, x0, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return finish(cuda_error(e, "copy of x0"));
    } else if (!x0) {
        cudaError_t e = cudaMemsetAsync(x, 0, n * sizeof(double), st);
        if (e != cudaSuccess) return finish(cuda_error(e, "zero x"));
    }
    if ((rc = norm2(P, P.d_b_rhs, 131, &bnorm2, pin))) return finish(rc);
    const double bnorm = std::sqrt(bnorm2);
    if (!std::isfinite(bnorm)) return finish(set_error(FDE_ERR_NAN, "right-hand side is not finite"));
    if (bnorm == 0.0) {
        cudaMemsetAsync(x, 0, n * sizeof(double), st);
        S.rel_residual = 0.0;
        return finish(FDE_OK);
    }
    // r = b - M x -> V_0
    if (x0) {
        if ((rc = matvec(P, x, P.d_work))) return finish(rc);
        if ((rc = launch_sub(P.d_b_rhs, P.d_work, V, n, st))) return finish(rc);
    } else {
        cudaError_t e = cudaMemcpyAsync(V, P.d_b_rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return finish(cuda_error(e, "copy of b"));
    }
    if ((rc = norm2(P, V, 132, &beta2, pin))) return finish(rc);
    if (x0 && !(beta2 <= bnorm2)) {
        // the initial guess is worse than zero (or not finite): start from x = 0
        FDE_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), st));
        FDE_CUDA_TRY(cudaMemcpyAsync(V, P.d_b_rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if ((rc = norm2(P, V, 132, &beta2, pin))) return finish(rc);
        S.x0_rejected = 1;
    }
    int its = 0;
    std::vector<double> g0(o.restart + 1, 0.0);
    double est = 0.0;
    for (;;) {
        const double beta = std::sqrt(beta2);
        S.rel_residual = beta / bnorm;
        if (!std::isfinite(beta)) { status = set_error(FDE_ERR_NAN, "residual is not finite"); break; }
        if (beta <= o.tol * bnorm) { status = FDE_OK; break; }
        if (its >= o.maxit) {
            status = set_error(FDE_ERR_NOT_CONVERGED, "maxit reached before the tolerance");
            break;
        }
        if ((rc = launch_scale(V, sc + 132, V, n, st))) return finish(rc);
        g0[0] = beta;
        std::fill(g0.begin() + 1, g0.end(), 0.0);
        FDE_CUDA_TRY(cudaMemcpyAsync(P.d_gv, g0.data(), g0.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        int j = 0;
        double est_rel = beta / bnorm;  // residual estimate before iteration j
        for (; j < o.restart; ++j) {
            bool replayed = false;
            const bool fp32 = o.matvec_precision == FDE_FP32 && !P.timevar && (o.relax <= 0.0 || est_rel > o.relax);
            if ((rc = run_iteration(P, j, ldh, o.reorth, o.restart, fp32, &replayed))) return finish(rc);
            ++its;
            if (fp32) ++S.matvecs_fp32;
            FDE_CUDA_TRY(cudaMemcpyAsync(pin, sc + 128, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
            FDE_CUDA_TRY(cudaStreamSynchronize(st));
            if (replayed && P.prof_mask) harvest_graph_events(P, j + (fp32 ? o.restart : 0));
            est = pin[1];
            est_rel = est / bnorm;
            const double hnext = std::fabs(pin[2]);
            if (!std::isfinite(est) || !std::isfinite(pin[0])) {
                status = set_error(FDE_ERR_NAN, "non-finite Hessenberg entry");
                break;
            }
            if (est <= o.tol * bnorm || its >= o.maxit || hnext <= 1e-300) {
                ++j;
                break;
            }
        }
        if (status == FDE_ERR_NAN) break;
        const int k = j < o.restart ? j : o.restart;
        if ((rc = launch_lsq_solve(P.d_H, ldh, k, P.d_gv, P.d_y, st))) return finish(rc);
        if ((rc = launch_update(Z, k, P.d_y, 1.0, x, n, st))) return finish(rc);
        ++S.restarts;
        S.rel_residual_estimate = est / bnorm;
        if ((rc = matvec(P, x, P.d_work))) return finish(rc);
        if ((rc = launch_sub(P.d_b_rhs, P.d_work, V, n, st))) return finish(rc);
        if ((rc = norm2(P, V, 132, &beta2, pin))) return finish(rc);
    }
    S.iterations = its;
    ++P.solves;
    return finish(status);
}

}  // extern "C"
