// Space-time matvec y = M z, M = A_1 (x) I - h B_1 (x) J (eq. (1.10) with u_0
// eliminated), and the plain Toeplitz-like apply y = J z (eq. (1.4)).
//
// One CTA per time row t.  By linearity
//     y_t = sum_q A[t][c_q] z_{c_q}  -  h J ( sum_q B[t][c_q] z_{c_q} ),
// so each CTA forms both band combinations of the mu+1 neighbouring time columns
// (read straight from HBM; the neighbours are shared through L2), then applies J
// once: J v = dx^-alpha (D+ G v + D- G^T v) through the length-L circulant
// embedding of G (Sec. 2.1: Toeplitz matvec by FFT), with one forward FFT of v
// (real input: a half-length complex FFT and a split) and one inverse FFT whose
// real / imaginary parts are G v and G^T v, both as radix-4 passes in FP64.
#include "fde_internal.h"
#include "fft_device.cuh"

namespace fde {

template <typename T, int MODE>
__device__ __forceinline__ void matvec_body(int m, int logL, int mu, double h, const int* __restrict__ start,
                                            const double* __restrict__ A, const double* __restrict__ B,
                                            const double* __restrict__ dplus, const double* __restrict__ dminus,
                                            const cplx_t<T>* __restrict__ sym, const cplx_t<T>* __restrict__ tw,
                                            const double* __restrict__ z, double* __restrict__ y, int row,
                                            int dstride = 0) {
    // T = double: the FP64 product.  T = float: the band sums, the A-band part and the
    // output stay FP64; only the Toeplitz apply J w (both FFTs and the symbol product)
    // runs in FP32 (the inexact inner product of the flexible GMRES).
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = 1 << logL, N = L >> 1, logN = logL - 1;
    C* buf = reinterpret_cast<C*>(smem_raw);
    double* ubuf = reinterpret_cast<double*>(buf + L);  // row = reduced time row: unknown u_{row+1}

    double ca[FDE_MAX_MU + 1], cb[FDE_MAX_MU + 1];
    int st = 0;
    if (MODE == 0) {
        const int t = row + 1;
        st = start[t];
#pragma unroll
        for (int q = 0; q <= FDE_MAX_MU; ++q) {
            ca[q] = q <= mu ? A[(size_t)t * (mu + 1) + q] : 0.0;
            cb[q] = q <= mu ? B[(size_t)t * (mu + 1) + q] : 0.0;
        }
    }
    // The input v of the Toeplitz apply is real: its length-L FFT comes from the
    // length-N = L/2 FFT of zc[n] = v[2n] + i v[2n+1] (bit-reversed for the DIT).
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        double v2[2] = {0.0, 0.0};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int i = 2 * n + e;
            if (i < m) {
                if (MODE == 0) {
                    double u = 0.0, w = 0.0;
#pragma unroll
                    for (int q = 0; q <= FDE_MAX_MU; ++q) {
                        const int col = st + q;  // full-system time index; column 0 (u_0) is eliminated
                        if (q <= mu && col >= 1) {
                            const double zz = z[(size_t)(col - 1) * m + i];
                            u += ca[q] * zz;
                            w += cb[q] * zz;
                        }
                    }
                    ubuf[i] = u;
                    v2[e] = w;
                } else {
                    v2[e] = z[(size_t)row * m + i];
                }
            }
        }
        buf[bitrev(n, logN)] = mk((T)v2[0], (T)v2[1]);
    }
    __syncthreads();
    fft_dit4<false>(buf, logN, tw, 2);  // tw holds W_L^k; stride 2 gives W_N^k
    // Split Zc into V (length L) and multiply by the symbol, in place: the thread of
    // pair (k, N-k) reads Zc[k], Zc[N-k] and writes V[k], V[k+N], V[N-k], V[2N-k] with
    //   E = (Zc[k] + conj Zc[N-k]) / 2,  O = (Zc[k] - conj Zc[N-k]) / 2i,
    //   V[k] = E + W_L^k O,  V[k+N] = E - W_L^k O.
    for (int k = threadIdx.x; k <= N / 2; k += blockDim.x) {
        const int kk = (N - k) & (N - 1);
        const C zk = buf[k], zn = buf[kk];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (e == 1 && kk == k) break;
            const int idx = e == 0 ? k : kk;
            const C za = e == 0 ? zk : zn, zb = e == 0 ? zn : zk;
            const T half = T(0.5);
            const C E = mk(half * (za.x + zb.x), half * (za.y - zb.y));
            const C O = mk(half * (za.y + zb.y), -half * (za.x - zb.x));
            const C wo = cmul(tw[idx], O);
            buf[idx] = cmul(cadd(E, wo), sym[idx]);
            buf[idx + N] = cmul(csub(E, wo), sym[idx + N]);
        }
    }
    __syncthreads();
    fft_dif4<true>(buf, logL, tw, 1);
    const double* dp = dplus + (size_t)row * dstride;  // MODE 1 with per-column coefficients
    const double* dm = dminus + (size_t)row * dstride;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const C wv = buf[bitrev(i, logL)];
        const double jz = dp[i] * (double)wv.x + dm[i] * (double)wv.y;
        if (MODE == 0)
            y[(size_t)row * m + i] = ubuf[i] - h * jz;
        else
            y[(size_t)row * m + i] = jz;
    }
}

// NT: the most threads a launch uses (the launch takes min(NT, L/2), at least 64);
// every loop is strided by blockDim.x, so all thread counts compute the same result
// (each butterfly and each output is the same arithmetic on the same operands).
// Register use is capped so that 1024 / NT CTAs fit an SM when shared memory allows.
template <typename T, int MODE, int NT = 1024>
__global__ void __launch_bounds__(NT, 1024 / NT)
st_matvec_kernel(int m, int logL, int mu, double h, const int* __restrict__ start, const double* __restrict__ A,
                 const double* __restrict__ B, const double* __restrict__ dplus, const double* __restrict__ dminus,
                 const cplx_t<T>* __restrict__ sym, const cplx_t<T>* __restrict__ tw, const double* __restrict__ z,
                 double* __restrict__ y, int dstride) {
    matvec_body<T, MODE>(m, logL, mu, h, start, A, B, dplus, dminus, sym, tw, z, y, blockIdx.x, dstride);
}

// Time-dependent coefficients: y_n = sum_q a_{n,q} z_q - h sum_q b_{n,q} (J_q z_q) over the
// BVM band of row n (u_0 eliminated), with jz = [J_1 z_1; ..; J_s z_s] from the Toeplitz
// apply; one CTA per time row, threads along x.
__global__ void __launch_bounds__(256)
st_band_kernel(int m, int mu, double h, const int* __restrict__ start, const double* __restrict__ A,
               const double* __restrict__ B, const double* __restrict__ z, const double* __restrict__ jz,
               double* __restrict__ y) {
    const int row = blockIdx.x, t = row + 1;
    const int st = start[t];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double u = 0.0, w = 0.0;
        for (int q = 0; q <= mu; ++q) {
            const int col = st + q;  // full-system time index; column 0 (u_0) is eliminated
            if (col >= 1) {
                u += A[(size_t)t * (mu + 1) + q] * z[(size_t)(col - 1) * m + i];
                w += B[(size_t)t * (mu + 1) + q] * jz[(size_t)(col - 1) * m + i];
            }
        }
        y[(size_t)row * m + i] = u - h * w;
    }
}

// Batched M z over the active instances: grid (max s, active count).
// which = 0: z = Z_j, y = V_{j+1} (Arnoldi step); which = 1: z = x, y = work (residual).
__global__ void __launch_bounds__(1024)
st_matvec_batched(const InstDev* __restrict__ I, const int* __restrict__ act, int which, int j) {
    const InstDev& d = I[act[blockIdx.y]];
    if ((int)blockIdx.x >= d.s || !d.ctl[0]) return;
    const double* z = which == 0 ? d.Z + (size_t)j * d.n : d.x;
    double* y = which == 0 ? d.V + (size_t)(j + 1) * d.n : d.work;
    matvec_body<double, 0>(d.m, d.logL, d.mu, d.h, d.start, d.A, d.B, d.dplus, d.dminus, d.sym, d.twL, z, y,
                           blockIdx.x);
}

int launch_matvec_batched(const InstDev* I, const int* act, int nact, int max_s, int max_L, int max_m, int which,
                          int j, cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    const size_t smem = (size_t)max_L * sizeof(double2) + (size_t)max_m * sizeof(double);
    int threads = max_L / 2;
    if (threads > 1024) threads = 1024;
    if (threads < 64) threads = 64;
    FDE_CUDA_TRY(cudaFuncSetAttribute(st_matvec_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    st_matvec_batched<<<dim3(max_s, nact), threads, smem, st>>>(I, act, which, j);
    FDE_LAUNCH_CHECK("st_matvec_batched");
    return FDE_OK;
}

template <int MODE, typename T = double, int NT = 1024>
static int launch_st(const Problem& P, const double* z, double* y, int ncols, cudaStream_t st,
                     const double* dplus = nullptr, const double* dminus = nullptr, int dstride = 0) {
    const int L = P.L;
    size_t smem = (size_t)L * sizeof(cplx_t<T>) + (MODE == 0 ? (size_t)P.m * sizeof(double) : 0);
    int threads = L / 2;
    if (threads > NT) threads = NT;
    if (threads < 64) threads = 64;
    auto kern = st_matvec_kernel<T, MODE, NT>;
    FDE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    const cplx_t<T>* sym;
    const cplx_t<T>* tw;
    if constexpr (sizeof(T) == 8) {
        sym = P.d_sym;
        tw = P.d_twL;
    } else {
        sym = P.d_sym32;
        tw = P.d_twL32;
    }
    kern<<<ncols, threads, smem, st>>>(P.m, P.logL, P.mu, P.h, P.d_start, P.d_a, P.d_b,
                                       dplus ? dplus : P.d_dplus, dminus ? dminus : P.d_dminus, sym, tw, z, y,
                                       dstride);
    FDE_LAUNCH_CHECK("st_matvec_kernel");
    return FDE_OK;
}

int launch_matvec32(const Problem& P, const double* z, double* y, cudaStream_t st) {
    if (P.timevar) return launch_matvec64(P, z, y, st);  // the time-level products stay FP64
    return launch_st<0, float>(P, z, y, P.s, st);
}

// The tuned variants of the FP64 space-time product: at most 1024, 512 or 256
// threads per time row (FDE_TUNE_MATVEC).
int launch_matvec64_variant(const Problem& P, const double* z, double* y, int variant, cudaStream_t st) {
    if (variant == 1) return launch_st<0, double, 512>(P, z, y, P.s, st);
    if (variant == 2) return launch_st<0, double, 256>(P, z, y, P.s, st);
    return launch_st<0, double, 1024>(P, z, y, P.s, st);
}

namespace {
struct MatvecTuneCtx {
    const Problem* P;
    const double* z;
    double* y;
};
int matvec_trial(void* ctx, int v, cudaStream_t st) {
    const MatvecTuneCtx& c = *static_cast<const MatvecTuneCtx*>(ctx);
    return launch_matvec64_variant(*c.P, c.z, c.y, v, st);
}
}  // namespace

// Measure the variants for this shape (z = b, y = the work vector) unless the table
// already has it or a variant is forced.
int autotune_matvec(Problem& P) {
    if (P.timevar) return FDE_OK;
    bool need = false;
    tune_lookup(FDE_TUNE_MATVEC, P.mp, P.s, FDE_FP64, &need);
    if (!need) return FDE_OK;
    MatvecTuneCtx ctx{&P, P.d_b_rhs, P.d_work};
    int best = 0;
    float ms[TUNE_MAX_VARIANTS] = {};
    const int rc = tune_measure(FDE_TUNE_MATVEC, P.stream, matvec_trial, &ctx, &best, ms,
                                tune_default_variant(FDE_TUNE_MATVEC, FDE_FP64));
    if (rc) return rc;
    tune_store(FDE_TUNE_MATVEC, P.mp, P.s, FDE_FP64, best, ms);
    return FDE_OK;
}

int launch_matvec64(const Problem& P, const double* z, double* y, cudaStream_t st) {
    if (!P.timevar)
        return launch_matvec64_variant(P, z, y, tune_lookup(FDE_TUNE_MATVEC, P.mp, P.s, FDE_FP64, nullptr), st);
    // J_q z_q for q = 1..s with the coefficients of time level q, then the BVM band
    int rc = launch_st<1>(P, z, P.d_jz, P.s, st, P.d_dplus_t + P.m, P.d_dminus_t + P.m, P.m);
    if (rc) return rc;
    st_band_kernel<<<P.s, 256, 0, st>>>(P.m, P.mu, P.h, P.d_start, P.d_a, P.d_b, z, P.d_jz, y);
    FDE_LAUNCH_CHECK("st_band_kernel");
    return FDE_OK;
}

int launch_japply64(const Problem& P, const double* z, double* y, int ncols, cudaStream_t st) {
    return launch_st<1>(P, z, y, ncols, st);
}

int launch_japply64_d(const Problem& P, const double* z, double* y, int ncols, const double* dplus,
                      const double* dminus, int dstride, cudaStream_t st) {
    return launch_st<1>(P, z, y, ncols, st, dplus, dminus, dstride);
}

}  // namespace fde
