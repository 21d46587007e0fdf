// FFT along time for every spatial index (Sec. 3.2: S^{-1} = (F^* (x) I)
// (Lambda_A (x) I - h Lambda_B (x) J)^{-1} (F (x) I)).
//
// Vectors are time-major [t][x] (x contiguous), so a CTA takes a tile of XW = 16
// consecutive x and all s time levels: each time row of the tile is one coalesced
// 128-byte read.  Two real columns are packed into one complex FFT
// (z = r_a + i r_b) and separated with the Hermitian split, so 8 complex length-s
// FFTs per tile.  Output / input of the frequency side: [k][mp] complex for
// k = 0..s/2 (the distinct frequencies of a real signal), padded to mp with zeros.
#include "fde_internal.h"
#include "fft_device.cuh"

namespace fde {

constexpr int XW = 16;      // spatial indices per CTA
constexpr int NCOL = XW / 2; // packed complex columns per CTA

template <typename T>
__device__ __forceinline__ void fwd_body(int m, int mp, int logs, const double* __restrict__ r,
                                         const cplx_t<T>* __restrict__ tw, cplx_t<T>* __restrict__ rhat, int bx) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);  // NCOL columns of length s
    const int s = 1 << logs;
    const int x0 = bx * XW;
    for (int e = threadIdx.x; e < s * XW; e += blockDim.x) {
        const int t = e / XW;
        const int xx = e - t * XW;
        const int x = x0 + xx;
        const T v = x < m ? (T)r[(size_t)t * m + x] : T(0);
        T* dst = reinterpret_cast<T*>(&buf[(xx >> 1) * s + bitrev(t, logs)]);
        dst[xx & 1] = v;
    }
    __syncthreads();
    fft_dit<C, false>(buf, logs, NCOL, s, tw);
    const int nk = s / 2 + 1;
    for (int e = threadIdx.x; e < nk * NCOL; e += blockDim.x) {
        const int k = e / NCOL;
        const int c = e - k * NCOL;
        const C Z = buf[c * s + k];
        const C Zc = cconj(buf[c * s + ((s - k) & (s - 1))]);
        const T half = T(0.5);
        // Ra = (Z + conj Z_{s-k}) / 2,  Rb = (Z - conj Z_{s-k}) / (2i)
        C Ra = mk((Z.x + Zc.x) * half, (Z.y + Zc.y) * half);
        C Rb = mk((Z.y - Zc.y) * half, -(Z.x - Zc.x) * half);
        const int xa = x0 + 2 * c;
        if (xa < mp) rhat[(size_t)k * mp + xa] = Ra;
        if (xa + 1 < mp) rhat[(size_t)k * mp + xa + 1] = Rb;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
time_fft_fwd_kernel(int m, int mp, int logs, const double* __restrict__ r, const cplx_t<T>* __restrict__ tw,
                    cplx_t<T>* __restrict__ rhat) {
    fwd_body<T>(m, mp, logs, r, tw, rhat, blockIdx.x);
}

template <typename T>
__device__ __forceinline__ void inv_body(int m, int mp, int logs, const cplx_t<T>* __restrict__ xhat,
                                         const cplx_t<T>* __restrict__ tw, double* __restrict__ z, int bx) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int s = 1 << logs;
    const int x0 = bx * XW;
    const int nk = s / 2 + 1;
    for (int e = threadIdx.x; e < nk * NCOL; e += blockDim.x) {
        const int k = e / NCOL;
        const int c = e - k * NCOL;
        const int xa = x0 + 2 * c;
        C Xa = xa < mp ? xhat[(size_t)k * mp + xa] : mk(T(0), T(0));
        C Xb = xa + 1 < mp ? xhat[(size_t)k * mp + xa + 1] : mk(T(0), T(0));
        if (k == 0 || k == s / 2) {  // real signal: DC and Nyquist terms are real
            Xa.y = T(0);
            Xb.y = T(0);
        }
        // Z_k = Xa_k + i Xb_k; for the mirrored frequency Z_{s-k} = conj(Xa_k) + i conj(Xb_k)
        buf[c * s + bitrev(k, logs)] = mk(Xa.x - Xb.y, Xa.y + Xb.x);
        if (k > 0 && k < s / 2) buf[c * s + bitrev(s - k, logs)] = mk(Xa.x + Xb.y, Xb.x - Xa.y);
    }
    __syncthreads();
    fft_dit<C, true>(buf, logs, NCOL, s, tw);
    const double inv = 1.0 / (double)s;
    for (int e = threadIdx.x; e < s * XW; e += blockDim.x) {
        const int t = e / XW;
        const int xx = e - t * XW;
        const int x = x0 + xx;
        if (x < m) {
            const T* src = reinterpret_cast<const T*>(&buf[(xx >> 1) * s + t]);
            z[(size_t)t * m + x] = (double)src[xx & 1] * inv;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
time_fft_inv_kernel(int m, int mp, int logs, const cplx_t<T>* __restrict__ xhat, const cplx_t<T>* __restrict__ tw,
                    double* __restrict__ z) {
    inv_body<T>(m, mp, logs, xhat, tw, z, blockIdx.x);
}

// Batched over the active instances act[]: grid (max x-tiles, active count), FP32
// transforms (the batched path uses FP32/TF32/BF16 preconditioners).  The forward
// transform reads the Krylov vector V_j, the inverse one writes Z_j.
__global__ void __launch_bounds__(256)
time_fft_fwd_batched(const InstDev* __restrict__ I, const int* __restrict__ act, int j) {
    const InstDev& d = I[act[blockIdx.y]];
    if ((int)blockIdx.x * XW >= d.mp || !d.ctl[0]) return;
    fwd_body<float>(d.m, d.mp, d.logs, d.V + (size_t)j * d.n, d.tws32, (float2*)d.rhat, blockIdx.x);
}

__global__ void __launch_bounds__(256)
time_fft_inv_batched(const InstDev* __restrict__ I, const int* __restrict__ act, int j) {
    const InstDev& d = I[act[blockIdx.y]];
    if ((int)blockIdx.x * XW >= d.mp || !d.ctl[0]) return;
    inv_body<float>(d.m, d.mp, d.logs, (const float2*)d.rhat, d.tws32, d.Z + (size_t)j * d.n, blockIdx.x);
}

int launch_time_fft_batched(const InstDev* I, const int* act, int nact, int max_mp, int max_s, int j,
                            cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    const dim3 grid((max_mp + XW - 1) / XW, nact);
    const size_t smem = (size_t)NCOL * max_s * sizeof(float2);
    FDE_CUDA_TRY(cudaFuncSetAttribute(time_fft_fwd_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    time_fft_fwd_batched<<<grid, 256, smem, st>>>(I, act, j);
    FDE_LAUNCH_CHECK("time_fft_fwd_batched");
    return FDE_OK;
}

int launch_time_ifft_batched(const InstDev* I, const int* act, int nact, int max_mp, int max_s, int j,
                             cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    const dim3 grid((max_mp + XW - 1) / XW, nact);
    const size_t smem = (size_t)NCOL * max_s * sizeof(float2);
    FDE_CUDA_TRY(cudaFuncSetAttribute(time_fft_inv_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    time_fft_inv_batched<<<grid, 256, smem, st>>>(I, act, j);
    FDE_LAUNCH_CHECK("time_fft_inv_batched");
    return FDE_OK;
}

int launch_time_fft_fwd(const Problem& P, const double* r, void* rhat, int prec, cudaStream_t st) {
    const int grid = (P.mp + XW - 1) / XW;
    if (prec == FDE_FP64) {
        size_t smem = (size_t)NCOL * P.s * sizeof(double2);
        FDE_CUDA_TRY(cudaFuncSetAttribute(time_fft_fwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          227 * 1024));
        time_fft_fwd_kernel<double><<<grid, 256, smem, st>>>(P.m, P.mp, P.logs, r, P.d_tws, (double2*)rhat);
    } else {
        size_t smem = (size_t)NCOL * P.s * sizeof(float2);
        FDE_CUDA_TRY(cudaFuncSetAttribute(time_fft_fwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          227 * 1024));
        time_fft_fwd_kernel<float><<<grid, 256, smem, st>>>(P.m, P.mp, P.logs, r, P.d_tws32, (float2*)rhat);
    }
    FDE_LAUNCH_CHECK("time_fft_fwd_kernel");
    return FDE_OK;
}

int launch_time_fft_inv(const Problem& P, const void* xhat, double* z, int prec, cudaStream_t st) {
    const int grid = (P.mp + XW - 1) / XW;
    if (prec == FDE_FP64) {
        size_t smem = (size_t)NCOL * P.s * sizeof(double2);
        FDE_CUDA_TRY(cudaFuncSetAttribute(time_fft_inv_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          227 * 1024));
        time_fft_inv_kernel<double><<<grid, 256, smem, st>>>(P.m, P.mp, P.logs, (const double2*)xhat, P.d_tws, z);
    } else {
        size_t smem = (size_t)NCOL * P.s * sizeof(float2);
        FDE_CUDA_TRY(cudaFuncSetAttribute(time_fft_inv_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          227 * 1024));
        time_fft_inv_kernel<float><<<grid, 256, smem, st>>>(P.m, P.mp, P.logs, (const float2*)xhat, P.d_tws32, z);
    }
    FDE_LAUNCH_CHECK("time_fft_inv_kernel");
    return FDE_OK;
}

}  // namespace fde
