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

// Radix-4 passes over one column of N = 2^logn points (FP64 double2 or FP32 float2): each pass is the exact
// regrouping of two consecutive radix-2 stages of fft_dit / fft_dif (same data order
// in and out), with three twiddle products per four points instead of four and half
// the passes through shared memory.  tw[k * ts] = exp(-2 pi i k / N) for k < N (ts:
// stride into the table of a longer transform).
//
// DIT, stages s and s+1 (half = 2^(s-1)), w2 = W_{2^(s+1)}^pos, w1 = w2^2, w3 = w2^3:
//   a = x0, b = w1 x1, c = w2 x2, d = w3 x3;
//   y0 = a+b+c+d, y1 = a-b-i(c-d), y2 = a+b-c-d, y3 = a-b+i(c-d)   (i -> -i inverse).
template <bool INVERSE, typename C>
__device__ void fft_dit4(C* buf, int logn, const C* __restrict__ tw, int ts) {
    const int N = 1 << logn;
    int st = 1;
    if (logn & 1) {  // a first radix-2 stage (twiddle 1)
        for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const C a = buf[2 * b], c = buf[2 * b + 1];
            buf[2 * b] = cadd(a, c);
            buf[2 * b + 1] = csub(a, c);
        }
        __syncthreads();
        st = 2;
    }
    for (; st < logn; st += 2) {
        const int half = 1 << (st - 1);
        const int tws = (N >> (st + 1)) * ts;
        for (int g = threadIdx.x; g < N / 4; g += blockDim.x) {
            const int pos = g & (half - 1);
            const int i0 = ((g >> (st - 1)) << (st + 1)) + pos;
            C w2 = tw[pos * tws], w1 = tw[2 * pos * tws], w3 = tw[3 * pos * tws];
            if (INVERSE) {
                w1.y = -w1.y;
                w2.y = -w2.y;
                w3.y = -w3.y;
            }
            const C a = buf[i0];
            const C b = cmul(w1, buf[i0 + half]);
            const C c = cmul(w2, buf[i0 + 2 * half]);
            const C d = cmul(w3, buf[i0 + 3 * half]);
            const C apb = cadd(a, b), amb = csub(a, b), cpd = cadd(c, d), cmd = csub(c, d);
            // -i (c - d) forward, +i (c - d) inverse
            const C rot = INVERSE ? mk(-cmd.y, cmd.x) : mk(cmd.y, -cmd.x);
            buf[i0] = cadd(apb, cpd);
            buf[i0 + half] = cadd(amb, rot);
            buf[i0 + 2 * half] = csub(apb, cpd);
            buf[i0 + 3 * half] = csub(amb, rot);
        }
        __syncthreads();
    }
}

// DIF, stages S and S-1 (h = 2^(S-2)), u = W_{2^S}^pos:
//   y0 = (x0+x2) + (x1+x3), y1 = ((x0+x2) - (x1+x3)) u^2,
//   y2 = u ((x0-x2) - i(x1-x3)), y3 = u^3 ((x0-x2) + i(x1-x3))   (conjugates inverse).
template <bool INVERSE, typename C>
__device__ void fft_dif4(C* buf, int logn, const C* __restrict__ tw, int ts) {
    const int N = 1 << logn;
    int S = logn;
    for (; S >= 2; S -= 2) {
        const int h = 1 << (S - 2);
        const int tws = (N >> S) * ts;
        for (int g = threadIdx.x; g < N / 4; g += blockDim.x) {
            const int pos = g & (h - 1);
            const int i0 = ((g >> (S - 2)) << S) + pos;
            C u1 = tw[pos * tws], u2 = tw[2 * pos * tws], u3 = tw[3 * pos * tws];
            if (INVERSE) {
                u1.y = -u1.y;
                u2.y = -u2.y;
                u3.y = -u3.y;
            }
            const C x0 = buf[i0], x1 = buf[i0 + h], x2 = buf[i0 + 2 * h], x3 = buf[i0 + 3 * h];
            const C s02 = cadd(x0, x2), d02 = csub(x0, x2), s13 = cadd(x1, x3), d13 = csub(x1, x3);
            // -i (x1 - x3) forward, +i (x1 - x3) inverse
            const C rot = INVERSE ? mk(-d13.y, d13.x) : mk(d13.y, -d13.x);
            buf[i0] = cadd(s02, s13);
            buf[i0 + h] = cmul(csub(s02, s13), u2);
            buf[i0 + 2 * h] = cmul(cadd(d02, rot), u1);
            buf[i0 + 3 * h] = cmul(csub(d02, rot), u3);
        }
        __syncthreads();
    }
    if (S == 1) {  // a last radix-2 stage (twiddle 1)
        for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const C a = buf[2 * b], c = buf[2 * b + 1];
            buf[2 * b] = cadd(a, c);
            buf[2 * b + 1] = csub(a, c);
        }
        __syncthreads();
    }
}

}  // namespace fde
