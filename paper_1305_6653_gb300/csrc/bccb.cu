// Strang-type BCCB preconditioners S^(2) = s(A) (x) I - h s(B) (x) s(J)  (eq. x1)
// and S~^(2) with s~(A) (eq. xc), Sec. 3.1; applied by the two-dimensional
// Fourier diagonalisation of Sec. 3.3.
//
// s(J) = dx^-alpha (mean(d+) s(G) + mean(d-) s(G)^T) is an N x N circulant
// (N = m), s(G) with first column [g_1 .. g_K, 0 .. 0, g_0], K = floor((m+1)/2).
// After the FFT along time (shared with the block-circulant preconditioner),
// frequency k needs x_k = C_k^{-1} r_k with the circulant C_k = phi_k I - h psi_k s(J).
// C_k^{-1} is a circulant too; with its first column c'_k, x_k is the cyclic
// convolution c'_k * r_k, computed as a linear convolution of length L >= 2m
// (power of two) by FFT and folded: x_i = z_i + z_{i+m}.
//
// Set-up (once): c = first column of s(J); its eigenvalues mu_j (length-m DFT,
// direct sum: m need not be a power of two); c'_k[i] = (1/m) sum_j
// exp(2 pi i ij/m) / (phi_k - h psi_k mu_j); K_k = FFT_L(c'_k) / L.  Apply (per
// GMRES iteration): one CTA per frequency, FFT_L, product with K_k, inverse FFT_L,
// fold.  The set-up is FP64; the apply runs in FP64 or FP32.
#include "fde_internal.h"
#include "fft_device.cuh"

namespace fde {

// First column of s(J) (length m) from the Grunwald weights and the means of d+-.
// One CTA; FP64 block reduction of the coefficient sums.
__global__ void __launch_bounds__(1024)
bccb_column_kernel(int m, double dxa, const double* __restrict__ g, const double* __restrict__ dplus,
                   const double* __restrict__ dminus, double* __restrict__ c) {
    __shared__ double red[2][32];
    double sp = 0.0, sm = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        sp += dplus[i];
        sm += dminus[i];
    }
    for (int off = 16; off; off >>= 1) {
        sp += __shfl_xor_sync(0xffffffffu, sp, off);
        sm += __shfl_xor_sync(0xffffffffu, sm, off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = sp;
        red[1][warp] = sm;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        sp = lane < nw ? red[0][lane] : 0.0;
        sm = lane < nw ? red[1][lane] : 0.0;
        for (int off = 16; off; off >>= 1) {
            sp += __shfl_xor_sync(0xffffffffu, sp, off);
            sm += __shfl_xor_sync(0xffffffffu, sm, off);
        }
        if (lane == 0) {
            red[0][0] = sp;
            red[1][0] = sm;
        }
    }
    __syncthreads();
    const double dp = red[0][0] / m, dm = red[1][0] / m;
    const int K = (m + 1) / 2;
    auto cg = [&](int i) {  // first column of s(G)
        double v = i < K ? g[i + 1] : 0.0;
        if (i == m - 1) v += g[0];
        return v;
    };
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        // s(G)^T has first column cg((m - i) mod m)
        const int it = i == 0 ? 0 : m - i;
        c[i] = dxa * (dp * cg(i) + dm * cg(it));
    }
}

// tw[t] = exp(-2 pi i t / m), t < m (any m)
__global__ void bccb_twiddle_kernel(int m, double2* __restrict__ tw) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    double sn, cs;
    sincospi(-2.0 * (double)t / (double)m, &sn, &cs);
    tw[t] = make_double2(cs, sn);
}

// mu_j = sum_i c_i exp(-2 pi i ij / m): the eigenvalues of s(J) in the order that
// pairs with the DFT of a vector (direct sum, the phase index (i j) mod m stepped).
__global__ void bccb_eig_kernel(int m, const double* __restrict__ c, const double2* __restrict__ tw,
                                double2* __restrict__ mu) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double re = 0.0, im = 0.0;
    int idx = 0;
    for (int i = 0; i < m; ++i) {
        const double2 w = tw[idx];
        re += c[i] * w.x;
        im += c[i] * w.y;
        idx += j;
        if (idx >= m) idx -= m;
    }
    mu[j] = make_double2(re, im);
}

// c'_k[i] = (1/m) sum_j exp(+2 pi i ij/m) / (phi_k - h psi_k mu_j), k = blockIdx.y:
// the first column of C_k^{-1}.  The reciprocal eigenvalues of a chunk of j are
// staged in shared memory; phi_0 is replaced by phi0_mod when modified (eq. xc).
constexpr int BCCB_JCH = 1024;
__global__ void __launch_bounds__(256)
bccb_invcol_kernel(int m, double h, const double2* __restrict__ phi, const double2* __restrict__ psi,
                   const double2* __restrict__ mu, const double2* __restrict__ tw, int modified, double phi0_mod,
                   double2* __restrict__ cinv, int* __restrict__ singular) {
    __shared__ double2 w[BCCB_JCH];
    const int k = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double2 ph = phi[k];
    if (k == 0 && modified) ph = make_double2(phi0_mod, 0.0);
    const double2 ps = psi[k];
    double re = 0.0, im = 0.0;
    int idx = 0;  // (i j) mod m for the current j
    const int istep = i < m ? i : 0;
    for (int j0 = 0; j0 < m; j0 += BCCB_JCH) {
        const int nj = min(BCCB_JCH, m - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < nj; e += blockDim.x) {
            const double2 u = mu[j0 + e];
            // lambda = phi_k - h psi_k mu_j
            const double lr = ph.x - h * (ps.x * u.x - ps.y * u.y);
            const double li = ph.y - h * (ps.x * u.y + ps.y * u.x);
            const double den = lr * lr + li * li;
            if (!(den > 0.0) || !isfinite(den)) atomicCAS(singular, 0, 1);
            w[e] = make_double2(lr / den, -li / den);
        }
        __syncthreads();
        for (int e = 0; e < nj; ++e) {
            const double2 t = tw[idx];  // exp(-2 pi i ij/m); its conjugate is wanted
            const double2 v = w[e];
            re += v.x * t.x + v.y * t.y;
            im += v.y * t.x - v.x * t.y;
            idx += istep;
            if (idx >= m) idx -= m;
        }
    }
    if (i < m) cinv[(size_t)k * m + i] = make_double2(re / m, im / m);
}

// K_k = FFT_L(c'_k zero-padded) / L in FP64 and FP32 (one CTA per frequency).
__global__ void __launch_bounds__(512)
bccb_spectrum_kernel(int m, int logL, const double2* __restrict__ cinv, const double2* __restrict__ tw,
                     double2* __restrict__ K64, float2* __restrict__ K32) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    const int L = 1 << logL, k = blockIdx.x;
    for (int i = threadIdx.x; i < L; i += blockDim.x)
        buf[bitrev(i, logL)] = i < m ? cinv[(size_t)k * m + i] : make_double2(0.0, 0.0);
    __syncthreads();
    fft_dit4<false>(buf, logL, tw, 1);
    const double sc = 1.0 / L;
    for (int f = threadIdx.x; f < L; f += blockDim.x) {
        const double2 v = make_double2(buf[f].x * sc, buf[f].y * sc);
        K64[(size_t)k * L + f] = v;
        K32[(size_t)k * L + f] = make_float2((float)v.x, (float)v.y);
    }
}

// x_k = C_k^{-1} r_k in place on rhat[k][0..m) (row pitch mp), one CTA per k.
template <typename T>
__global__ void __launch_bounds__(512)
bccb_solve_kernel(int m, int mp, int logL, cplx_t<T>* __restrict__ rhat, const cplx_t<T>* __restrict__ K,
                  const cplx_t<T>* __restrict__ tw) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int L = 1 << logL, k = blockIdx.x;
    C* row = rhat + (size_t)k * mp;
    const C* Kk = K + (size_t)k * L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) buf[bitrev(i, logL)] = i < m ? row[i] : mk(T(0), T(0));
    __syncthreads();
    if constexpr (sizeof(T) == 8)
        fft_dit4<false>(buf, logL, tw, 1);
    else
        fft_dit<C, false>(buf, logL, 1, L, tw);
    for (int f = threadIdx.x; f < L; f += blockDim.x) buf[f] = cmul(buf[f], Kk[f]);
    __syncthreads();
    if constexpr (sizeof(T) == 8)
        fft_dif4<true>(buf, logL, tw, 1);
    else
        fft_dif<C, true>(buf, logL, 1, L, tw);
    // the inverse transform leaves z in bit-reversed order; cyclic fold x_i = z_i + z_{i+m}
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        row[i] = cadd(buf[bitrev(i, logL)], buf[bitrev(i + m, logL)]);
}

int launch_bccb_setup(const Problem& P, int modified, double phi0_mod, double* c, double2* tw, double2* mu,
                      double2* cinv, double2* K64, float2* K32, int* singular, cudaStream_t st) {
    const int m = P.m, nk = P.nblk, L = P.L;
    if (L < 2 * m) return set_error(FDE_ERR_ARG, "the BCCB apply needs the FFT length L >= 2m");
    bccb_column_kernel<<<1, 1024, 0, st>>>(m, P.dxa, P.d_g, P.d_dplus, P.d_dminus, c);
    FDE_LAUNCH_CHECK("bccb_column_kernel");
    bccb_twiddle_kernel<<<(m + 255) / 256, 256, 0, st>>>(m, tw);
    FDE_LAUNCH_CHECK("bccb_twiddle_kernel");
    bccb_eig_kernel<<<(m + 127) / 128, 128, 0, st>>>(m, c, tw, mu);
    FDE_LAUNCH_CHECK("bccb_eig_kernel");
    bccb_invcol_kernel<<<dim3((m + 255) / 256, nk), 256, 0, st>>>(m, P.h, P.d_phi, P.d_psi, mu, tw, modified, phi0_mod,
                                                                cinv, singular);
    FDE_LAUNCH_CHECK("bccb_invcol_kernel");
    const size_t smem = (size_t)L * sizeof(double2);
    FDE_CUDA_TRY(cudaFuncSetAttribute(bccb_spectrum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    bccb_spectrum_kernel<<<nk, 512, smem, st>>>(m, P.logL, cinv, P.d_twL, K64, K32);
    FDE_LAUNCH_CHECK("bccb_spectrum_kernel");
    return FDE_OK;
}

int launch_bccb_solve(const Problem& P, void* rhat, int prec, cudaStream_t st) {
    if (prec == FDE_FP64) {
        const size_t smem = (size_t)P.L * sizeof(double2);
        FDE_CUDA_TRY(cudaFuncSetAttribute(bccb_solve_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        bccb_solve_kernel<double><<<P.nblk, 512, smem, st>>>(P.m, P.mp, P.logL, (double2*)rhat, P.d_bccb_K64,
                                                              P.d_twL);
    } else {
        const size_t smem = (size_t)P.L * sizeof(float2);
        FDE_CUDA_TRY(cudaFuncSetAttribute(bccb_solve_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        bccb_solve_kernel<float><<<P.nblk, 512, smem, st>>>(P.m, P.mp, P.logL, (float2*)rhat, P.d_bccb_K32,
                                                             P.d_twL32);
    }
    FDE_LAUNCH_CHECK("bccb_solve_kernel");
    return FDE_OK;
}

}  // namespace fde
