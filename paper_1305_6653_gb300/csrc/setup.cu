// Set-up kernels: Grunwald weights (eq. (1.2)), FFT twiddles, the FFT symbol of the
// circulant embedding of the shifted-Grunwald Toeplitz matrix G (eq. (1.5)), the
// Strang symbols phi_k / psi_k (Sec. 3.1) and the right-hand side of eq. (1.10).
#include "fde_internal.h"
#include "fft_device.cuh"

namespace fde {

// g_0 = 1, g_{k+1} = (1 - (alpha+1)/(k+1)) g_k (eq. (1.2)).  One warp: lane l runs
// the recurrence over its own contiguous chunk of factors starting from 1, the
// chunk products are scanned across lanes (multiplicative prefix), and each lane
// rescales its chunk.  The result is the same product of the same factors as the
// sequential recurrence, associated differently (a few ulps apart).
__global__ void grunwald_kernel(double alpha, int count, double* __restrict__ g) {
    const int lane = threadIdx.x;
    const int chunk = (count + 31) / 32;
    const int k0 = lane * chunk;  // this lane produces g[k0+1 .. k0+chunk]
    double prod = 1.0;
    for (int k = k0; k < k0 + chunk && k + 1 < count; ++k) {
        prod *= (1.0 - (alpha + 1.0) / (double)(k + 1));
        g[k + 1] = prod;  // partial product, rescaled below
    }
    double pre = prod;  // inclusive scan of chunk products
    for (int off = 1; off < 32; off <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, pre, off);
        if (lane >= off) pre *= v;
    }
    double excl = __shfl_up_sync(0xffffffffu, pre, 1);
    if (lane == 0) excl = 1.0;
    __syncwarp();
    for (int k = k0; k < k0 + chunk && k + 1 < count; ++k) g[k + 1] *= excl;
    if (lane == 0) g[0] = 1.0;
}

// tw[k] = exp(-2 pi i k / L) for k < count (the caller's table length: L/2 for
// radix-2 stages, L for the radix-4 passes, which read up to 3L/4).
__global__ void twiddle_kernel(int L, int count, double2* __restrict__ tw64, float2* __restrict__ tw32) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)L, &sn, &cs);
    if (tw64) tw64[k] = make_double2(cs, sn);
    if (tw32) tw32[k] = make_float2((float)cs, (float)sn);
}

// First column of the L-periodic circulant C that embeds G (G[i][j] = g_{i-j+1}
// for j <= i+1): c[k] = g_{k+1} for 0 <= k < m, c[L-1] = g_0, zero elsewhere.
// lambda = FFT_L(c); the symbol stored is scale * (lambda + i conj(lambda)) / L so
// that one inverse FFT of sym * FFT(z) returns (G z) + i (G^T z) for real z
// (C^T has eigenvalues conj(lambda) in the same Fourier basis).
__global__ void toeplitz_symbol_kernel(const double* __restrict__ g, int m, int logL, double scale,
                                       const double2* __restrict__ tw, double2* __restrict__ sym64,
                                       float2* __restrict__ sym32) {
    extern __shared__ double2 sbuf[];
    const int L = 1 << logL;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        double v = 0.0;
        if (k < m) v = g[k + 1];
        else if (k == L - 1) v = g[0];
        sbuf[bitrev(k, logL)] = make_double2(v, 0.0);
    }
    __syncthreads();
    fft_dit<double2, false>(sbuf, logL, 1, L, tw);
    const double inv = scale / (double)L;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        double2 l = sbuf[k];
        // lambda + i conj(lambda) = (lr + i li) + (li + i lr) = (lr + li) (1 + i)
        const double kap = (l.x + l.y) * inv;
        double2 v = make_double2(kap, kap);
        if (sym64) sym64[k] = v;
        if (sym32) sym32[k] = make_float2((float)v.x, (float)v.y);
    }
}

// phi_k = sum_{r=-nu}^{mu-nu} a_{r+nu} exp(2 pi i r k / s), psi_k likewise with b, k = 0..s/2
__global__ void strang_symbol_kernel(const double* __restrict__ a, const double* __restrict__ b, int mu, int nu,
                                     int s, double2* __restrict__ phi, double2* __restrict__ psi) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > s / 2) return;
    double pr = 0, pi = 0, qr = 0, qi = 0;
    for (int r = -nu; r <= mu - nu; ++r) {
        long rk = ((long)r * k) % s;
        double sn, cs;
        sincospi(2.0 * (double)rk / (double)s, &sn, &cs);
        pr += a[r + nu] * cs;
        pi += a[r + nu] * sn;
        qr += b[r + nu] * cs;
        qi += b[r + nu] * sn;
    }
    phi[k] = make_double2(pr, pi);
    psi[k] = make_double2(qr, qi);
}

// b_t = h sum_q B[t][start+q] f_{start+q} - A[t][0] u0 + h B[t][0] J u0, t = 1..s
// (eq. (1.10) with the known block u_0 moved to the right-hand side).
__global__ void rhs_kernel(int m, int s, int mu, double h, const int* __restrict__ start,
                           const double* __restrict__ A, const double* __restrict__ B,
                           const double* __restrict__ f, const double* __restrict__ u0,
                           const double* __restrict__ Ju0, double* __restrict__ b) {
    const int t = blockIdx.y + 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int st = start[t];
    const double* a = A + (size_t)t * (mu + 1);
    const double* bb = B + (size_t)t * (mu + 1);
    double acc = 0.0;
    for (int q = 0; q <= mu; ++q) acc += bb[q] * f[(size_t)(st + q) * m + i];
    acc *= h;
    if (st == 0) acc += -a[0] * u0[i] + h * bb[0] * Ju0[i];
    b[(size_t)(t - 1) * m + i] = acc;
}

int launch_grunwald(double alpha, int count, double* g, cudaStream_t st) {
    grunwald_kernel<<<1, 32, 0, st>>>(alpha, count, g);
    FDE_LAUNCH_CHECK("grunwald_kernel");
    return FDE_OK;
}

int launch_twiddles(int L, int count, double2* tw64, float2* tw32, cudaStream_t st) {
    if (count <= 0) return FDE_OK;
    twiddle_kernel<<<(count + 255) / 256, 256, 0, st>>>(L, count, tw64, tw32);
    FDE_LAUNCH_CHECK("twiddle_kernel");
    return FDE_OK;
}

int launch_toeplitz_symbol(const double* g, int m, int L, double scale, const double2* tw, double2* sym64,
                           float2* sym32, double2* /*work*/, cudaStream_t st) {
    size_t smem = (size_t)L * sizeof(double2);
    static bool attr = false;
    if (!attr) {
        FDE_CUDA_TRY(cudaFuncSetAttribute(toeplitz_symbol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          227 * 1024));
        attr = true;
    }
    toeplitz_symbol_kernel<<<1, 1024, smem, st>>>(g, m, ilog2(L), scale, tw, sym64, sym32);
    FDE_LAUNCH_CHECK("toeplitz_symbol_kernel");
    return FDE_OK;
}

int launch_strang_symbols(const double* a_main, const double* b_main, int mu, int nu, int s, double2* phi,
                          double2* psi, cudaStream_t st) {
    int n = s / 2 + 1;
    strang_symbol_kernel<<<(n + 127) / 128, 128, 0, st>>>(a_main, b_main, mu, nu, s, phi, psi);
    FDE_LAUNCH_CHECK("strang_symbol_kernel");
    return FDE_OK;
}

int launch_rhs(const Problem& P, const double* Ju0, cudaStream_t st) {
    dim3 grid((P.m + 255) / 256, P.s);
    rhs_kernel<<<grid, 256, 0, st>>>(P.m, P.s, P.mu, P.h, P.d_start, P.d_a, P.d_b, P.d_f, P.d_u0, Ju0, P.d_b_rhs);
    FDE_LAUNCH_CHECK("rhs_kernel");
    return FDE_OK;
}

}  // namespace fde
