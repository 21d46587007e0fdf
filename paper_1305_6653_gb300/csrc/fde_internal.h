// Internal declarations shared by the CUDA translation units of libfde.
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/fde.h"

namespace fde {

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);

#define FDE_CUDA_TRY(call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return ::fde::cuda_error(e_, #call); \
    } while (0)

void note_launch();
void note_launches(long long k);  // k kernels launched at once (a graph replay; negative: uncount)

#define FDE_LAUNCH_CHECK(what)                               \
    do {                                                     \
        ::fde::note_launch();                                \
        cudaError_t e_ = cudaGetLastError();                 \
        if (e_ != cudaSuccess) return ::fde::cuda_error(e_, what); \
    } while (0)

inline int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}
inline int round_up(int v, int q) { return (v + q - 1) / q * q; }

constexpr int LU_NB = 32;  // panel width of the blocked Strang-block LU

// ---------------------------------------------------------------------------
// Device descriptors of a batch of independent problems (batch.cu).  One InstDev
// per instance (sizes, coefficient / symbol pointers, factor and Krylov buffers),
// one BlkDev per Strang block of every instance.
// ---------------------------------------------------------------------------
struct InstDev {
    int m, s, mp, L, logL, logs, mu, nblk;
    long n;
    double h, dxa;
    const int* start;
    const double* A;
    const double* B;
    const double* dplus;
    const double* dminus;
    const double2* sym;
    const double2* twL;
    const float2* tws32;
    const double2* tws;
    void* rhat;
    void* fac;
    void* dinv;
    void* tinv;            // inverted 32 x 32 diagonal tiles of the factors, or NULL
    const void* strips;    // bfloat16 strip-major copy of the factors (with tinv), or NULL
    double* b;
    double* x;
    double* V;
    double* Z;
    double* work;
    double* H;
    double* cs;
    double* sn;
    double* gv;
    double* y;
    double* scal;          // [0..63] h1, [64..127] h2, [128] |w|^2, [129] est, [130] H(j+1,j), [132] beta^2
    double* partial;       // RED_CTAS x 64
    unsigned int* counter;
    // per-instance control words of a batched solve: [0] live (the batched GMRES
    // kernels skip an instance whose flag is 0), [1] Arnoldi steps taken in the
    // current restart cycle, [2] total steps, [3] 1 = a non-finite value was met
    int* ctl;
};

struct BlkDev {
    int inst, k, m, mp, ntile_max;  // ntile_max: bytes of the block's A' tiles (tensor-core paths)
    double h, dxa;
    const double2* phi;  // &phi_k, &psi_k of the instance
    const double2* psi;
    const double* g;
    const double* dplus;
    const double* dminus;
    void* fac;    // this block's planes (Re then Im, mp x mp each)
    void* dinv;   // this block's 1/U_ii (mp complex)
    unsigned char* apack;  // this block's packed operand tiles (tensor-core paths)
    unsigned char* bpack;
    unsigned char* ipack;  // L11^{-1} (A') and U11^{-1} (B') tiles of the current panel
    int* info;
    unsigned short* strips;  // this block's bfloat16 strip-major copy (Re then Im), or NULL
};

// ---------------------------------------------------------------------------
// kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
struct Problem;

// setup.cu
int launch_grunwald(double alpha, int count, double* g, cudaStream_t st);
// tw[k] = exp(-2 pi i k / L) for k < count (count = the table's length)
int launch_twiddles(int L, int count, double2* tw64, float2* tw32, cudaStream_t st);
int launch_toeplitz_symbol(const double* g, int m, int L, double scale, const double2* tw, double2* sym64,
                           float2* sym32, double2* work, cudaStream_t st);
int launch_strang_symbols(const double* a_main, const double* b_main, int mu, int nu, int s, double2* phi,
                          double2* psi, cudaStream_t st);
int launch_rhs(const Problem& P, const double* Ju0, cudaStream_t st);

// matvec.cu: y = M z (mode 0) or y = J z for ncols columns (mode 1)
int launch_matvec64(const Problem& P, const double* z, double* y, cudaStream_t st);
// y = M z with the Toeplitz apply in FP32 (the band, its A part and y in FP64)
int launch_matvec32(const Problem& P, const double* z, double* y, cudaStream_t st);
int launch_japply64(const Problem& P, const double* z, double* y, int ncols, cudaStream_t st);
// J_n z for ncols columns with per-column coefficients dplus + c*dstride (dstride 0: shared)
int launch_japply64_d(const Problem& P, const double* z, double* y, int ncols, const double* dplus,
                      const double* dminus, int dstride, cudaStream_t st);

// timefft.cu
int launch_time_fft_fwd(const Problem& P, const double* r, void* rhat, int prec, cudaStream_t st);
int launch_time_fft_inv(const Problem& P, const void* xhat, double* z, int prec, cudaStream_t st);

// lu.cu
int launch_block_lu(Problem& P, int prec, cudaStream_t st);
// The FP32 inverses of the 32 x 32 diagonal tiles of P's factors (P.d_tinv).
int launch_tile_inverse_fp32(Problem& P, cudaStream_t st);
int launch_block_trsv(const Problem& P, void* rhat, cudaStream_t st);

// krylov.cu
int launch_dots(const double* V, int k, const double* w, long n, double* out, double* partial,
                unsigned int* counter, cudaStream_t st);
int launch_update(const double* V, int k, const double* coef, double sign, double* w, long n, cudaStream_t st);
int launch_norm(const double* w, long n, double* out, double* partial, unsigned int* counter, cudaStream_t st);
// Fused classical Gram-Schmidt pass over V_0..V_{k-1} (V row-major [k][n], w length n):
// mode 0: out = V^T w;  1: w -= V c, then out = V^T w;  2: w -= V c, then out[0] = |w|^2
int launch_cgs_pass(int mode, const double* V, int k, const double* c, double* w, long n, double* out,
                    double* partial, unsigned int* counter, cudaStream_t st);
int launch_scale(const double* src, const double* nrm_sq, double* dst, long n, cudaStream_t st);
int launch_arnoldi_finish(double* H, int ldh, int j, const double* h1, const double* h2, const double* nrm_sq,
                          double* cs, double* sn, double* g, double* est, cudaStream_t st);
int launch_lsq_solve(const double* H, int ldh, int k, const double* g, double* y, cudaStream_t st);
int launch_axpy(double a, const double* x, double* y, long n, cudaStream_t st);
int launch_sub(const double* b, const double* ax, double* r, long n, cudaStream_t st);

// ---------------------------------------------------------------------------
// The problem object.
// ---------------------------------------------------------------------------
struct Problem {
    // description
    int m = 0, s = 0, mu = 0, nu = 0, family = 0;
    double alpha = 0, xL = 0, xR = 0, t0 = 0, T = 0, dx = 0, h = 0, dxa = 0;  // dxa = dx^-alpha
    int L = 0, logL = 0;        // Toeplitz circulant embedding length (power of two >= 2m)
    int logs = 0;               // log2(s)
    int nblk = 0;               // s/2 + 1 Strang blocks
    int mp = 0;                 // m rounded up to the LU tile (64)
    long n = 0;                 // s*m unknowns
    cudaStream_t stream = nullptr;
    bool device_ptrs = false;   // desc->device_ptrs: solve vectors (x0, x_out) are device pointers
    double* d_xsol = nullptr;   // n: device copy of the solution when x0 / x_out are host pointers

    // host copies of the BVM band (rows 0..s of A and B)
    int h_start[FDE_MAX_S + 1];
    double h_a_main[FDE_MAX_MU + 1], h_b_main[FDE_MAX_MU + 1];

    // device buffers
    int* d_start = nullptr;
    double* d_a = nullptr;      // (s+1)*(mu+1)
    double* d_b = nullptr;
    double* d_dplus = nullptr;  // m (time-dependent coefficients: their means over n = 1..s)
    double* d_dminus = nullptr; // m
    bool timevar = false;        // d+-(x, t) given
    double* d_dplus_t = nullptr;  // (s+1)*m, [n][i], when timevar
    double* d_dminus_t = nullptr;
    double* d_jz = nullptr;       // n: J_n z_n of the time-dependent matvec
    double* d_u0 = nullptr;     // m
    double* d_f = nullptr;      // (s+1)*m
    double* d_g = nullptr;      // m+2 Grunwald weights
    double2* d_twL = nullptr;   // L twiddles exp(-2 pi i k / L), FP64
    float2* d_twL32 = nullptr;  // same, FP32
    double2* d_sym = nullptr;   // L: (lambda + i conj(lambda)) / L, lambda = FFT of the circulant embedding of G
    float2* d_sym32 = nullptr;
    double2* d_tws = nullptr;   // s/2 twiddles exp(-2 pi i k / s)
    float2* d_tws32 = nullptr;
    double2* d_phi = nullptr;   // s/2+1
    double2* d_psi = nullptr;
    double* d_b_rhs = nullptr;  // n
    double* d_work = nullptr;   // n scratch (J u0, residuals)
    void* d_rhat = nullptr;     // nblk * mp complex (FP64 or FP32 by precision)
    void* d_fac = nullptr;      // nblk * 2 * mp * mp (planar re/im), FP64 or FP32
    void* d_dinv = nullptr;     // nblk * mp complex: 1 / U_ii
    int* d_info = nullptr;      // nblk: first singular pivot (+1) or 0
    int* d_err = nullptr;       // device error flag of bounded waits (0 = none)
    size_t fac_bytes = 0;
    void* d_tinv = nullptr;     // inverted 32 x 32 diagonal tiles of L and U (block solves)
    size_t tinv_bytes = 0;
    void* d_pack = nullptr;     // packed tensor-core operand tiles of the LU panels
    size_t pack_bytes = 0;
    // inverted 128 x 128 diagonal blocks of L and U, packed as TF32 A' operand tiles,
    // one pair per 128-row strip of every Strang block (the tensor-core block solves of
    // a shared-operator batch); written by the TF32 tensor-core LU when save_dtile is set
    void* d_dtile = nullptr;
    size_t dtile_bytes = 0;
    bool save_dtile = false;
    // the FP32 factor in strip-major layout (32-column strips, rows contiguous), written
    // by the tensor-core LU beside the row-major planes for the block solves
    void* d_strips = nullptr;
    size_t strips_bytes = 0;
    bool strips_ok = false;
    bool strips_bf16 = false;  // the copy holds bfloat16 values (fde_factor_storage)
    int strip_storage = FDE_STORAGE_FP32;
    bool want_strips = true;   // off for a shared-operator batch, whose solves read the planes
    // Strang-type BCCB preconditioner (bccb_precond_setup): the spectra K_k of the
    // circulant inverses, k = 0..s/2, length L each, and its frequency-side vectors
    int precond = 0;            // FDE_PRECOND_STRANG or FDE_PRECOND_BCCB / FDE_PRECOND_BCCB_MODIFIED
    int bccb_precision = -1;    // FDE_FP64 or FDE_FP32 arithmetic of the apply
    double2* d_bccb_K64 = nullptr;
    float2* d_bccb_K32 = nullptr;
    void* d_rhat_b = nullptr;   // nblk * mp complex (FP64 or FP32 by bccb_precision)
    int rhat_b_prec = -1;
    // CUDA graphs of the GMRES inner iteration j (preconditioner apply, matvec, Gram-
    // Schmidt passes, Givens update, normalisation), captured on first use and replayed;
    // graph_key names the set-up they were captured for (stale graphs are destroyed)
    cudaStream_t cap_stream = nullptr;
    std::vector<cudaGraphExec_t> iter_graph;
    std::vector<long long> iter_graph_launches;  // kernels per replay (launch counter)
    long long graph_key = -1;
    int graph_gen = 0;                           // bumped whenever a buffer the graphs use changes
    int solves = 0;                              // completed pgmres_solve calls
    // tensor-core LU look-ahead: panel chain on lu_hi, interior updates on lu_lo, the
    // cross tiles other than the next diagonal block on lu_x
    cudaStream_t lu_hi = nullptr, lu_lo = nullptr, lu_x = nullptr;
    // fork / panel products done / interior done / next diagonal block updated / cross tiles done
    cudaEvent_t lu_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

    // Krylov workspace
    int restart_cap = 0;
    double* d_V = nullptr;      // (restart+1) * n
    double* d_Z = nullptr;      // restart * n
    double* d_H = nullptr;      // (restart+1) * restart, column-major ldh = restart+1
    double* d_cs = nullptr;
    double* d_sn = nullptr;
    double* d_gv = nullptr;     // restart+1
    double* d_y = nullptr;      // restart
    double* d_scal = nullptr;   // scalars: [0..63] dots h1, [64..127] dots h2, [128] norm^2, [129] est, ...
    double* d_partial = nullptr;
    unsigned int* d_counter = nullptr;

    bool assembled = false;
    bool factored = false;
    int precision = -1;

    // per-stage CUDA-event profiler (fde_profile_enable: every stage, direct launches)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_rec[FDE_NUM_STAGES];
    // selected-stage timer (fde_profile_select): event pairs around the stages in the
    // mask; inside a captured iteration graph they become event-record nodes owned by
    // that graph, read after each replay and summed into prof_acc
    unsigned prof_mask = 0;
    struct GraphEvent {
        int stage;
        cudaEvent_t e0, e1;
    };
    std::vector<GraphEvent>* capturing_events = nullptr;   // graph being captured
    std::vector<std::vector<GraphEvent>> iter_graph_events;  // per iteration graph
    double prof_acc_ms[FDE_NUM_STAGES] = {};
    int prof_acc_n[FDE_NUM_STAGES] = {};
};

// preconditioner in use by pgmres_solve / fde_precond_apply
constexpr int FDE_PRECOND_STRANG = 0;         // block-circulant S (eq. 1.11), block LU
constexpr int FDE_PRECOND_BCCB = 1;           // S^(2) (eq. x1)
constexpr int FDE_PRECOND_BCCB_MODIFIED = 2;  // S~^(2) (eq. xc)
constexpr int FDE_PRECOND_NONE = 3;           // plain GMRES (column I of Tables 1-2)

// bccb.cu: set-up of the BCCB spectra (scratch: c, tw, mu of length m, cinv of nblk * m;
// *singular set to 1 on a zero or non-finite eigenvalue of the preconditioner)
// and the per-frequency circulant solves in place on rhat ([nblk][mp] complex)
int launch_bccb_setup(const Problem& P, int modified, double phi0_mod, double* c, double2* tw, double2* mu,
                      double2* cinv, double2* K64, float2* K32, int* singular, cudaStream_t st);
int launch_bccb_solve(const Problem& P, void* rhat, int prec, cudaStream_t st);

// devmem.cu: device buffers through a cache of freed blocks (exact size, per device).
// dev_free: no queued GPU work may still use the block.
int dev_alloc(void** p, size_t bytes);
void dev_free(void* p);
// Frees every cached block (blocks in use are not affected).
int dev_release_cached();

// tune.cu: launch-shape autotuner.  tune_lookup returns the variant to launch for a
// shape (forced, tabulated, or 0 = the built-in default, with *need_tuning set when
// the shape has not been measured yet); tune_measure times every variant of fn and
// returns the fastest; tune_store records it (memory and the cache file).
int tune_variants(int kernel);
int tune_lookup(int kernel, int mp, int nb, int prec, bool* need_tuning);
void tune_store(int kernel, int mp, int nb, int prec, int variant, const float* ms);  // ms: per variant, or NULL
// ms_out: the median time of every variant, or NULL; nv > 0: only variants 0 .. nv-1
int tune_measure(int kernel, cudaStream_t st, int (*fn)(void*, int, cudaStream_t), void* ctx, int* best,
                 float* ms_out, int default_variant, int nv = 0);
int tune_default_variant(int kernel, int prec);
constexpr int TUNE_MAX_VARIANTS = 8;
// the tuned kernels' variant launchers (matvec.cu, lu.cu) and the tuning passes
int launch_matvec64_variant(const Problem& P, const double* z, double* y, int variant, cudaStream_t st);
int launch_block_trsv_variant(const Problem& P, void* rhat, int variant, cudaStream_t st);
int autotune_matvec(Problem& P);
int autotune_trsv(Problem& P);

// The problem behind a C-ABI handle (defined in api.cu).
Problem* problem_of(fde_problem* h);
int ensure_factor_buffers(Problem& P, int precision);
int ensure_workspace(Problem& P, int restart);
int ensure_solution_buffer(Problem& P);  // d_xsol for problems whose solve vectors are host memory

// batched launchers (lu.cu, timefft.cu, matvec.cu, krylov.cu)
int launch_lu_batched(const BlkDev* d_blk, const std::vector<int>& mp_sorted, int precision, int* err,
                      cudaStream_t st);
size_t tc_pack_bytes_per_block(int precision, int mp);    // packed tensor-core operands of one block
size_t tc_pack_a_bytes_per_block(int precision, int mp);  // the A' part (B' follows)
size_t tc_pack_b_bytes_per_block(int precision, int mp);  // the B' part (inverse tiles follow)
int launch_trsv_batched(const InstDev* I, const int* act, int nact, int max_nblk, int max_mp, cudaStream_t st);
// Block solves of instances that share one operator's factors (FP32 with inverted
// diagonal tiles): groups of 8 right-hand sides per CTA, each factor plane streamed once
// per group
int launch_trsv_multi(const InstDev* I, const int* act, int nact, int nblk, int mp, cudaStream_t st);
// trsm.cu: tensor-core block solves of a shared-operator batch (groups of 16 right-hand
// sides; TF32 factors with the inverted 128 x 128 diagonal blocks kept by the LU)
bool trsm_tc_supported(int mp);
// FP32 factor planes of nblk blocks as one 2-D tensor map (rows of m_p floats, block k's
// Re plane from row 2 k m_p, Im plane from (2 k + 1) m_p), boxes of 128 rows x 32
// columns, 128-byte swizzle
int factor_tensor_map_sw128(const void* fac, int mp, int nblk, CUtensorMap* map);
// The strip-major copy (rows of 32 floats: element (r, c) of block k's plane at row
// ((2 k + plane) m_p / 32 + c / 32) m_p + r), same boxes and swizzle
int strip_tensor_map_sw128(const void* strips, int mp, int nblk, CUtensorMap* map);
int launch_trsm_tc(const InstDev* I, const int* act, int nact, const void* fac, const void* dtile, int mp, int nblk,
                   int* err, cudaStream_t st);
int launch_time_fft_batched(const InstDev* I, const int* act, int nact, int max_mp, int max_s, int j,
                            cudaStream_t st);
int launch_time_ifft_batched(const InstDev* I, const int* act, int nact, int max_mp, int max_s, int j,
                             cudaStream_t st);
int launch_matvec_batched(const InstDev* I, const int* act, int nact, int max_s, int max_L, int max_m, int which,
                          int j, cudaStream_t st);
int launch_dots_batched(const InstDev* I, const int* act, int nact, int mode, int j, cudaStream_t st);
int launch_update_batched(const InstDev* I, const int* act, int nact, int mode, int j, const int* kvec, long max_n,
                          cudaStream_t st);
int launch_scale_batched(const InstDev* I, const int* act, int nact, int mode, int j, int restart, long max_n,
                         cudaStream_t st);
int launch_residual_batched(const InstDev* I, const int* act, int nact, long max_n, cudaStream_t st);
// finish_batched also decides, on the device, whether the instance leaves the cycle
// (estimate <= tol |b|, maxit total steps, breakdown or a non-finite value)
int launch_finish_batched(const InstDev* I, const int* act, int nact, int j, int ldh, int reorth, double tol,
                          int maxit, cudaStream_t st);
// ctl[0] = live for the listed instances; reset: also zero ctl[1] (and ctl[2], ctl[3] when reset > 1)
int launch_ctl_set_batched(const InstDev* I, const int* act, int nact, int live, int reset, cudaStream_t st);
int launch_lsq_batched(const InstDev* I, const int* act, int nact, const int* kvec, int ldh, cudaStream_t st);
int launch_gather_scalars(const InstDev* I, int ninst, double* out, cudaStream_t st);

// Records a CUDA event pair around the launches made in its scope when the
// problem's profiler is on.
class StageTimer {
  public:
    StageTimer(Problem& P, int stage, cudaStream_t on = nullptr);  // on: default P.stream
    ~StageTimer();

  private:
    Problem* P_;
    int stage_;
    cudaStream_t st_;
    cudaEvent_t e0_ = nullptr;
    bool graph_ = false;  // recorded into the iteration graph being captured
};

}  // namespace fde
