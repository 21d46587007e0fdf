// Device helpers: complex arithmetic on double2 / float2 and an in-shared-memory
// radix-2 FFT used by the Toeplitz matvec (length L along x) and by the time
// transforms (length s along t).
#pragma once

#include <cuda_runtime.h>

namespace fde {

template <typename T> struct cvec;
template <> struct cvec<double> { using type = double2; };
template <> struct cvec<float> { using type = float2; };
template <typename T> using cplx_t = typename cvec<T>::type;

__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

__device__ __forceinline__ int bitrev(int v, int logn) { return logn ? (int)(__brev((unsigned)v) >> (32 - logn)) : 0; }

// Decimation-in-time radix-2 FFT of `ncol` independent columns held in shared
// memory (column c occupies buf[c*stride .. c*stride + N)), input in bit-reversed
// order, output in natural order.  Twiddles tw[k] = exp(-2 pi i k / N), k < N/2;
// INVERSE uses their conjugates (unnormalised).  All threads of the block call it.
template <typename C, bool INVERSE>
__device__ void fft_dit(C* buf, int logn, int ncol, int stride, const C* __restrict__ tw) {
    const int N = 1 << logn;
    const int half_total = N >> 1;
    const int work = half_total * ncol;
    for (int st = 1; st <= logn; ++st) {
        const int half = 1 << (st - 1);
        const int tws = N >> st;
        for (int b = threadIdx.x; b < work; b += blockDim.x) {
            const int col = b / half_total;
            const int bb = b - col * half_total;
            const int grp = bb >> (st - 1);
            const int pos = bb & (half - 1);
            const int i0 = col * stride + (grp << st) + pos;
            const int i1 = i0 + half;
            C w = tw[pos * tws];
            if (INVERSE) w.y = -w.y;
            C a = buf[i0];
            C t = cmul(w, buf[i1]);
            buf[i0] = cadd(a, t);
            buf[i1] = csub(a, t);
        }
        __syncthreads();
    }
}

// Decimation-in-frequency radix-2 FFT: natural-order input, bit-reversed output.
template <typename C, bool INVERSE>
__device__ void fft_dif(C* buf, int logn, int ncol, int stride, const C* __restrict__ tw) {
    const int N = 1 << logn;
    const int half_total = N >> 1;
    const int work = half_total * ncol;
    for (int st = logn; st >= 1; --st) {
        const int half = 1 << (st - 1);
        const int tws = N >> st;
        for (int b = threadIdx.x; b < work; b += blockDim.x) {
            const int col = b / half_total;
            const int bb = b - col * half_total;
            const int grp = bb >> (st - 1);
            const int pos = bb & (half - 1);
            const int i0 = col * stride + (grp << st) + pos;
            const int i1 = i0 + half;
            C w = tw[pos * tws];
            if (INVERSE) w.y = -w.y;
            C a = buf[i0];
            C c = buf[i1];
            buf[i0] = cadd(a, c);
            buf[i1] = cmul(csub(a, c), w);
        }
        __syncthreads();
    }
}

}  // namespace fde
