// Strang blocks B_k = phi_k I - h psi_k J (Sec. 3.2), k = 0..s/2, formed on the
// device from (g, d+, d-) and factored B_k = L_k U_k by right-looking blocked LU
// without pivoting (every B_k is strictly row diagonally dominant: J is, by
// Proposition 2.2, and Re(phi_k / psi_k) >= 0 for the A_{nu,mu-nu}-stable
// schemes), then solved once per GMRES iteration by blocked forward / backward
// substitution.
//
// Storage: planar complex, one m_p x m_p row-major plane for Re and one for Im per
// block (m_p = m rounded up to 64; the padding is the identity), packed L\U in
// place, plus 1/U_ii per row.  Precision T = double (plain method) or float.
//
// Per panel step p (columns [p NB, (p+1) NB)):
//   1. lu_diag:   factor the NB x NB diagonal block in shared memory (one CTA per block)
//   2. lu_panel:  L21 = A21 U11^{-1} and U12 = L11^{-1} A12 (row / column chunks)
//   3. lu_update: A22 -= L21 U12 (complex GEMM on CUDA cores; the tensor-core
//                 variant lives in lu_tc.cu)
#include "fde_internal.h"
#include "fft_device.cuh"
#include "lu_tc.cuh"

namespace fde {

constexpr int NB = LU_NB;

template <typename T>
__device__ __forceinline__ T* plane_re(T* fac, int k, int mp) { return fac + (size_t)k * 2 * mp * mp; }
template <typename T>
__device__ __forceinline__ T* plane_im(T* fac, int k, int mp) { return fac + (size_t)k * 2 * mp * mp + (size_t)mp * mp; }

// J[i][j] = dx^-alpha (d+_i G[i][j] + d-_i G[j][i]),  G[i][j] = g_{i-j+1} (i-j+1 >= 0), eq. (1.4)/(1.5)
__device__ __forceinline__ double j_entry(int i, int j, double dxa, const double* __restrict__ g,
                                          const double* __restrict__ dp, const double* __restrict__ dm) {
    const int a = i - j + 1;
    const int b = j - i + 1;
    double v = 0.0;
    if (a >= 0) v += dp[i] * g[a];
    if (b >= 0) v += dm[i] * g[b];
    return dxa * v;
}

// One CTA row-loop per matrix row, threads along the columns (no index division).
// FP64 blocks are formed in FP64; FP32 blocks in FP32 from FP32 copies of the
// per-row coefficients dx^-alpha d+_i, dx^-alpha d-_i and of h psi_k.
template <typename T>
__device__ __forceinline__ void form_body(int m, int mp, double h, double dxa, const double* __restrict__ g,
                                          const double* __restrict__ dp, const double* __restrict__ dm, double2 ph,
                                          double2 ps, T* __restrict__ re, int row0, int rowstride) {
    const T hpr = (T)(h * ps.x), hpi = (T)(h * ps.y);
    T* im = re + (size_t)mp * mp;
    for (int i = row0; i < mp; i += rowstride) {
        T* rr = re + (size_t)i * mp;
        T* ri = im + (size_t)i * mp;
        if (i >= m) {
            for (int j = threadIdx.x; j < mp; j += blockDim.x) {
                rr[j] = (i == j) ? T(1) : T(0);
                ri[j] = T(0);
            }
            continue;
        }
        const T rp = (T)(dxa * dp[i]), rm = (T)(dxa * dm[i]);
        for (int j = threadIdx.x; j < mp; j += blockDim.x) {
            T vr = T(0), vi = T(0);
            if (j < m) {
                const int a = i - j + 1, b = j - i + 1;
                T jv = T(0);
                if (a >= 0) jv += rp * (T)g[a];
                if (b >= 0) jv += rm * (T)g[b];
                vr = -hpr * jv;
                vi = -hpi * jv;
                if (i == j) {
                    vr += (T)ph.x;
                    vi += (T)ph.y;
                }
            }
            rr[j] = vr;
            ri[j] = vi;
        }
    }
}

template <typename T>
__global__ void form_blocks_kernel(int m, int mp, double h, double dxa, const double* __restrict__ g,
                                   const double* __restrict__ dp, const double* __restrict__ dm,
                                   const double2* __restrict__ phi, const double2* __restrict__ psi, T* __restrict__ fac) {
    const int k = blockIdx.y;
    form_body<T>(m, mp, h, dxa, g, dp, dm, phi[k], psi[k], plane_re(fac, k, mp), blockIdx.x, gridDim.x);
}

// Batched: grid.y runs over the block table of every instance.
template <typename T>
__global__ void form_blocks_batched(const BlkDev* __restrict__ B) {
    const BlkDev& d = B[blockIdx.y];
    form_body<T>(d.m, d.mp, d.h, d.dxa, d.g, d.dplus, d.dminus, *d.phi, *d.psi, (T*)d.fac, blockIdx.x, gridDim.x);
}

// Unblocked LU (no pivoting) of the NB x NB diagonal block of every matrix.
template <typename T>
__device__ __forceinline__ void diag_body(int mp, int p, T* __restrict__ re, cplx_t<T>* __restrict__ dinv,
                                          int* __restrict__ info) {
    using C = cplx_t<T>;
    __shared__ C D[NB][NB + 1];
    T* im = re + (size_t)mp * mp;
    const int o = p * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        const size_t idx = (size_t)(o + r) * mp + o + c;
        D[r][c] = mk(re[idx], im[idx]);
    }
    __syncthreads();
    for (int c = 0; c < NB; ++c) {
        const C piv = D[c][c];
        const T den = piv.x * piv.x + piv.y * piv.y;
        const bool bad = !(den > T(0)) || !isfinite((double)den);
        if (bad && threadIdx.x == 0) atomicCAS(info, 0, o + c + 1);
        C inv = mk(piv.x / den, -piv.y / den);
        if (bad) inv = mk(T(0), T(0));
        __syncthreads();
        // scale the column below the pivot: l_rc = a_rc / u_cc
        for (int r = c + 1 + threadIdx.x; r < NB; r += blockDim.x) D[r][c] = cmul(D[r][c], inv);
        __syncthreads();
        const int w = NB - c - 1;
        for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
            const int r = c + 1 + e / w, cc = c + 1 + e % w;
            D[r][cc] = csub(D[r][cc], cmul(D[r][c], D[c][cc]));
        }
        if (threadIdx.x == 0) dinv[o + c] = inv;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        const size_t idx = (size_t)(o + r) * mp + o + c;
        re[idx] = D[r][c].x;
        im[idx] = D[r][c].y;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
lu_diag_kernel(int mp, int p, T* __restrict__ fac, cplx_t<T>* __restrict__ dinv, int* __restrict__ info) {
    const int k = blockIdx.x;
    diag_body<T>(mp, p, plane_re(fac, k, mp), dinv + (size_t)k * mp, info + k);
}

template <typename T>
__global__ void __launch_bounds__(256) lu_diag_batched(const BlkDev* __restrict__ B, int p) {
    const BlkDev& d = B[blockIdx.x];
    if (p * NB >= d.mp) return;
    diag_body<T>(d.mp, p, (T*)d.fac, (cplx_t<T>*)d.dinv, d.info);
}

// Panel solves.  blockIdx.x < nrow: a chunk of RC rows of A21 -> L21 = A21 U11^{-1};
// otherwise a chunk of RC columns of A12 -> U12 = L11^{-1} A12.  One thread per
// row (column): the NB values live in registers and the triangular solve against
// the factored diagonal block (shared memory, broadcast reads) needs no barrier.
// Loads and stores go through shared memory so that global accesses stay coalesced.
// PACK < 0: plain; PACK = 0 / 1: also write the panels as packed TF32 / BF16
// tensor-core operand tiles (A' from L21 rows, B' from U12 columns; see lu_tc.cuh).
constexpr int RC = 128;
template <typename T, int PACK>
__device__ __forceinline__ void panel_body(int mp, int p, int nrow, T* __restrict__ re, unsigned char* __restrict__ apack,
                                           unsigned char* __restrict__ bpack, int bx) {
    using C = cplx_t<T>;
    __shared__ C D[NB][NB + 1];
    __shared__ C dinv_s[NB];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C (*X)[NB + 1] = reinterpret_cast<C (*)[NB + 1]>(smem_raw);  // [RC][NB+1]
    T* im = re + (size_t)mp * mp;
    const int o = p * NB;
    const int rest = o + NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        const size_t idx = (size_t)(o + r) * mp + o + c;
        D[r][c] = mk(re[idx], im[idx]);
    }
    const bool rows = bx < nrow;
    const int chunk = rows ? bx : bx - nrow;
    const int b0 = rest + chunk * RC;
    // X[q][c]: rows mode -> A21[b0+q][o+c]; columns mode -> A12[o+c][b0+q] (stored transposed)
    for (int e = threadIdx.x; e < RC * NB; e += blockDim.x) {
        int q, c;
        size_t idx;
        if (rows) {
            q = e / NB; c = e % NB;
            idx = (size_t)(b0 + q) * mp + o + c;
        } else {
            c = e / RC; q = e % RC;
            idx = (size_t)(o + c) * mp + b0 + q;
        }
        X[q][c] = (b0 + q < mp) ? mk(re[idx], im[idx]) : mk(T(0), T(0));
    }
    __syncthreads();
    if (rows && threadIdx.x < NB) {
        const C piv = D[threadIdx.x][threadIdx.x];
        const T den = piv.x * piv.x + piv.y * piv.y;
        dinv_s[threadIdx.x] = den > T(0) ? mk(piv.x / den, -piv.y / den) : mk(T(0), T(0));
    }
    __syncthreads();
    const int q = threadIdx.x;
    C x[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) x[c] = X[q][c];
    if (rows) {
        // x U11 = a: x_c = (a_c - sum_{c'<c} x_c' U[c'][c]) / U[c][c]
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            x[c] = cmul(x[c], dinv_s[c]);
#pragma unroll
            for (int cc = c + 1; cc < NB; ++cc) x[cc] = csub(x[cc], cmul(x[c], D[c][cc]));
        }
    } else {
        // L11 u = a (unit lower): u_rr -= L[rr][c] u_c, rr > c
#pragma unroll
        for (int c = 0; c < NB; ++c) {
#pragma unroll
            for (int rr = c + 1; rr < NB; ++rr) x[rr] = csub(x[rr], cmul(D[rr][c], x[c]));
        }
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) X[q][c] = x[c];
    __syncthreads();
    for (int e = threadIdx.x; e < RC * NB; e += blockDim.x) {
        int qq, c;
        size_t idx;
        if (rows) {
            qq = e / NB; c = e % NB;
            idx = (size_t)(b0 + qq) * mp + o + c;
        } else {
            c = e / RC; qq = e % RC;
            idx = (size_t)(o + c) * mp + b0 + qq;
        }
        if (b0 + qq < mp) {
            re[idx] = X[qq][c].x;
            im[idx] = X[qq][c].y;
        }
        if constexpr (PACK >= 0) {
            const int tile = (chunk * RC + qq) / TC_BM;
            const int rt = (chunk * RC + qq) % TC_BM;  // row of the operand tile (A': output row, B': output column)
            const float vr = (float)X[qq][c].x, vi = (float)X[qq][c].y;
            if (rows) {
                unsigned char* t = apack + (size_t)tile * TcCfg<PACK>::A_BYTES;
                pack_store<PACK>(t, rt, c, vr);
                pack_store<PACK>(t, rt, NB + c, vi);
            } else {
                unsigned char* t = bpack + (size_t)tile * TcCfg<PACK>::B_BYTES;
                pack_store<PACK>(t, rt, c, vr);            // Re part of the product: Re L Re U - Im L Im U
                pack_store<PACK>(t, rt, NB + c, -vi);
                pack_store<PACK>(t, TC_BN + rt, c, vi);    // Im part: Re L Im U + Im L Re U
                pack_store<PACK>(t, TC_BN + rt, NB + c, vr);
            }
        }
    }
}

template <int PACK>
__device__ __forceinline__ size_t pack_stride(bool a_side, int ntile_max) {
    if constexpr (PACK >= 0) return (size_t)ntile_max * (a_side ? TcCfg<PACK>::A_BYTES : TcCfg<PACK>::B_BYTES);
    return 0;
}

template <typename T, int PACK>
__global__ void __launch_bounds__(RC)
lu_panel_kernel(int mp, int p, int nrow, T* __restrict__ fac, unsigned char* __restrict__ apack,
                unsigned char* __restrict__ bpack, int ntile_max) {
    const int k = blockIdx.y;
    panel_body<T, PACK>(mp, p, nrow, plane_re(fac, k, mp), apack ? apack + k * pack_stride<PACK>(true, ntile_max) : nullptr,
                        bpack ? bpack + k * pack_stride<PACK>(false, ntile_max) : nullptr, blockIdx.x);
}

template <typename T, int PACK>
__global__ void __launch_bounds__(RC) lu_panel_batched(const BlkDev* __restrict__ B, int p) {
    const BlkDev& d = B[blockIdx.y];
    const int rem = d.mp - (p + 1) * NB;
    if (rem <= 0) return;
    const int nrow = (rem + RC - 1) / RC;
    if ((int)blockIdx.x >= 2 * nrow) return;
    panel_body<T, PACK>(d.mp, p, nrow, (T*)d.fac, d.apack, d.bpack, blockIdx.x);
}

// Trailing update A22 -= L21 U12 on CUDA cores: 64 x 64 output tile per CTA,
// 4 x 4 complex outputs per thread, K = NB.
template <typename T>
__device__ __forceinline__ void update_body(int mp, int p, T* __restrict__ re, int ti, int tj) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C (*Ls)[NB + 1] = reinterpret_cast<C (*)[NB + 1]>(smem_raw);                        // [64][NB+1]
    C (*Us)[64 + 1] = reinterpret_cast<C (*)[64 + 1]>(smem_raw + 64 * (NB + 1) * sizeof(C));  // [NB][65]
    T* im = re + (size_t)mp * mp;
    const int o = p * NB;
    const int rest = o + NB;
    const int r0 = rest + ti * 64, c0 = rest + tj * 64;
    for (int e = threadIdx.x; e < 64 * NB; e += blockDim.x) {
        const int q = e / NB, c = e % NB;
        const int r = r0 + q;
        Ls[q][c] = r < mp ? mk(re[(size_t)r * mp + o + c], im[(size_t)r * mp + o + c]) : mk(T(0), T(0));
        const int c2 = e / 64, q2 = e % 64;
        const int cc = c0 + q2;
        Us[c2][q2] = cc < mp ? mk(re[(size_t)(o + c2) * mp + cc], im[(size_t)(o + c2) * mp + cc]) : mk(T(0), T(0));
    }
    __syncthreads();
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mk(T(0), T(0));
#pragma unroll 4
    for (int kk = 0; kk < NB; ++kk) {
        C av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = Ls[tr + 16 * a][kk];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Us[kk][tc + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                acc[a][b].x += av[a].x * bv[b].x - av[a].y * bv[b].y;
                acc[a][b].y += av[a].x * bv[b].y + av[a].y * bv[b].x;
            }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = r0 + tr + 16 * a;
        if (r >= mp) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = c0 + tc + 16 * b;
            if (c >= mp) continue;
            const size_t idx = (size_t)r * mp + c;
            re[idx] -= acc[a][b].x;
            im[idx] -= acc[a][b].y;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
lu_update_kernel(int mp, int p, int ntile, T* __restrict__ fac) {
    const int k = blockIdx.y;
    update_body<T>(mp, p, plane_re(fac, k, mp), blockIdx.x / ntile, blockIdx.x % ntile);
}

// Batched: grid.x covers the tiles of the largest trailing matrix (ntile_grid^2).
template <typename T>
__global__ void __launch_bounds__(256) lu_update_batched(const BlkDev* __restrict__ B, int p, int ntile_grid) {
    const BlkDev& d = B[blockIdx.y];
    const int rem = d.mp - (p + 1) * NB;
    if (rem <= 0) return;
    const int nt = (rem + 63) / 64;
    const int ti = blockIdx.x / ntile_grid, tj = blockIdx.x % ntile_grid;
    if (ti >= nt || tj >= nt) return;
    update_body<T>(d.mp, p, (T*)d.fac, ti, tj);
}

// Forward (unit lower L) then backward (U) substitution for one block per CTA,
// in place on rhat[k] (length mp), column-oriented ("right-looking"): for each
// 32-row diagonal tile, warp 0 resolves the tile from shared memory, then all
// warps subtract the tile's 32-column strip of L (or U) times the new 32 values
// from the remaining right-hand side.  In the strip update eight threads share a
// row (one contiguous 32-value segment per plane), every load is independent of
// the others, and the next diagonal tile is prefetched into shared memory, so
// the factor planes stream at full memory-level parallelism.
struct dvec4 {
    double x, y, z, w;
};
template <typename T> struct vec4;
template <> struct vec4<float> { using type = float4; };
template <> struct vec4<double> { using type = dvec4; };

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ dvec4 ld4(const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    return dvec4{a.x, a.y, b.x, b.y};
}

constexpr int TRSV_THREADS = 512;
constexpr int TRSV_TPR = 8;                              // threads per row in the strip update
constexpr int TRSV_RPP = TRSV_THREADS / TRSV_TPR;        // rows per pass

template <typename T>
__device__ __forceinline__ void load_diag_tile(cplx_t<T> (*D)[33], const T* re, const T* im, int mp, int r0) {
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int q = e >> 5, c = e & 31;
        const size_t idx = (size_t)(r0 + q) * mp + r0 + c;
        D[q][c] = mk(re[idx], im[idx]);
    }
}

// y[rows] -= strip[rows][c0 .. c0+32) * xs[0..32), rows in [rbeg, rend)
template <typename T>
__device__ __forceinline__ void strip_update(cplx_t<T>* y, const cplx_t<T>* xs, const T* re, const T* im, int mp,
                                             int c0, int rbeg, int rend) {
    using C = cplx_t<T>;
    const int sub = threadIdx.x & (TRSV_TPR - 1);
    const int c = c0 + sub * 4;
    const C x0 = xs[sub * 4], x1 = xs[sub * 4 + 1], x2 = xs[sub * 4 + 2], x3 = xs[sub * 4 + 3];
    for (int rb = rbeg + (int)(threadIdx.x / TRSV_TPR); rb < rend; rb += 4 * TRSV_RPP) {
        typename vec4<T>::type ar[4], ai[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = rb + u * TRSV_RPP;
            if (r < rend) {
                ar[u] = ld4(re + (size_t)r * mp + c);
                ai[u] = ld4(im + (size_t)r * mp + c);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = rb + u * TRSV_RPP;
            T sx = ar[u].x * x0.x - ai[u].x * x0.y + ar[u].y * x1.x - ai[u].y * x1.y + ar[u].z * x2.x -
                   ai[u].z * x2.y + ar[u].w * x3.x - ai[u].w * x3.y;
            T sy = ar[u].x * x0.y + ai[u].x * x0.x + ar[u].y * x1.y + ai[u].y * x1.x + ar[u].z * x2.y +
                   ai[u].z * x2.x + ar[u].w * x3.y + ai[u].w * x3.x;
#pragma unroll
            for (int off = 1; off < TRSV_TPR; off <<= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, off);
                sy += __shfl_xor_sync(0xffffffffu, sy, off);
            }
            if (sub == 0 && r < rend) {
                C v = y[r];
                v.x -= sx;
                v.y -= sy;
                y[r] = v;
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ void trsv_body(int mp, const T* __restrict__ re, const cplx_t<T>* __restrict__ dv,
                                          cplx_t<T>* __restrict__ x) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* y = reinterpret_cast<C*>(smem_raw);                        // mp
    C (*D)[32][33] = reinterpret_cast<C (*)[32][33]>(y + mp);     // 2 diagonal tiles (double buffer)
    __shared__ C xs[32];
    const T* im = re + (size_t)mp * mp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = mp / 32;
    for (int i = threadIdx.x; i < mp; i += blockDim.x) y[i] = x[i];
    load_diag_tile<T>(D[0], re, im, mp, 0);
    __syncthreads();
    // forward: y <- L^{-1} y
    for (int t = 0; t < nt; ++t) {
        const int r0 = t * 32;
        if (warp == 0) {
            C a = y[r0 + lane];
            for (int c = 0; c < 32; ++c) {
                const T yx = __shfl_sync(0xffffffffu, a.x, c);
                const T yy = __shfl_sync(0xffffffffu, a.y, c);
                if (lane > c) {
                    const C l = D[t & 1][lane][c];
                    a.x -= l.x * yx - l.y * yy;
                    a.y -= l.x * yy + l.y * yx;
                }
            }
            y[r0 + lane] = a;
            xs[lane] = a;
        }
        __syncthreads();
        if (t + 1 < nt) {
            load_diag_tile<T>(D[(t + 1) & 1], re, im, mp, r0 + 32);
            strip_update<T>(y, xs, re, im, mp, r0, r0 + 32, mp);
        }
        __syncthreads();
    }
    // backward: y <- U^{-1} y
    load_diag_tile<T>(D[(nt - 1) & 1], re, im, mp, (nt - 1) * 32);
    __syncthreads();
    for (int t = nt - 1; t >= 0; --t) {
        const int r0 = t * 32;
        if (warp == 0) {
            C a = y[r0 + lane];
            const C di = dv[r0 + lane];
            for (int c = 31; c >= 0; --c) {
                if (lane == c) a = cmul(a, di);
                const T yx = __shfl_sync(0xffffffffu, a.x, c);
                const T yy = __shfl_sync(0xffffffffu, a.y, c);
                if (lane < c) {
                    const C u = D[t & 1][lane][c];
                    a.x -= u.x * yx - u.y * yy;
                    a.y -= u.x * yy + u.y * yx;
                }
            }
            y[r0 + lane] = a;
            xs[lane] = a;
        }
        __syncthreads();
        if (t > 0) {
            load_diag_tile<T>(D[(t - 1) & 1], re, im, mp, r0 - 32);
            strip_update<T>(y, xs, re, im, mp, r0, 0, r0);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < mp; i += blockDim.x) x[i] = y[i];
}

template <typename T>
__global__ void __launch_bounds__(TRSV_THREADS)
block_trsv_kernel(int mp, const T* __restrict__ fac, const cplx_t<T>* __restrict__ dinv, cplx_t<T>* __restrict__ rhat) {
    const int k = blockIdx.x;
    trsv_body<T>(mp, fac + (size_t)k * 2 * mp * mp, dinv + (size_t)k * mp, rhat + (size_t)k * mp);
}

// Batched over the active instances act[0..gridDim.y): block k = blockIdx.x of instance act[blockIdx.y].
template <typename T>
__global__ void __launch_bounds__(TRSV_THREADS)
block_trsv_batched(const InstDev* __restrict__ I, const int* __restrict__ act) {
    const InstDev& d = I[act[blockIdx.y]];
    const int k = blockIdx.x;
    if (k >= d.nblk) return;
    const size_t mp = d.mp;
    trsv_body<T>(d.mp, (const T*)d.fac + (size_t)k * 2 * mp * mp, (const cplx_t<T>*)d.dinv + (size_t)k * mp,
                 (cplx_t<T>*)d.rhat + (size_t)k * mp);
}

template <typename T>
static int run_lu(Problem& P, cudaStream_t st) {
    using C = cplx_t<T>;
    T* fac = reinterpret_cast<T*>(P.d_fac);
    C* dinv = reinterpret_cast<C*>(P.d_dinv);
    const int mp = P.mp, nb = P.nblk;
    {
        dim3 grid(mp < 64 ? mp : 64, nb);
        StageTimer t(P, FDE_STAGE_FORM);
        form_blocks_kernel<T><<<grid, 256, 0, st>>>(P.m, mp, P.h, P.dxa, P.d_g, P.d_dplus, P.d_dminus, P.d_phi,
                                                   P.d_psi, fac);
        FDE_LAUNCH_CHECK("form_blocks_kernel");
    }
    const size_t panel_smem = (size_t)RC * (NB + 1) * sizeof(C);
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_panel_kernel<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)panel_smem));
    const size_t upd_smem = (64 * (NB + 1) + NB * 65) * sizeof(C);
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd_smem));
    const int steps = mp / NB;
    for (int p = 0; p < steps; ++p) {
        {
            StageTimer t(P, FDE_STAGE_LU_DIAG);
            lu_diag_kernel<T><<<nb, 256, 0, st>>>(mp, p, fac, dinv, P.d_info);
            FDE_LAUNCH_CHECK("lu_diag_kernel");
        }
        const int rem = mp - (p + 1) * NB;
        if (rem <= 0) break;
        const int nch = (rem + RC - 1) / RC;
        {
            StageTimer t(P, FDE_STAGE_LU_PANEL);
            lu_panel_kernel<T, -1><<<dim3(2 * nch, nb), RC, panel_smem, st>>>(mp, p, nch, fac, nullptr, nullptr, 0);
            FDE_LAUNCH_CHECK("lu_panel_kernel");
        }
        const int nt = (rem + 63) / 64;
        StageTimer t(P, FDE_STAGE_LU_UPDATE);
        lu_update_kernel<T><<<dim3(nt * nt, nb), 256, upd_smem, st>>>(mp, p, nt, fac);
        FDE_LAUNCH_CHECK("lu_update_kernel");
    }
    return FDE_OK;
}

// FP32 factors whose trailing updates run on the tcgen05 tensor cores.
template <int KIND>
static int run_lu_tc(Problem& P, cudaStream_t st) {
    using Cfg = TcCfg<KIND>;
    static_assert(TC_KP == 2 * NB, "packed K' must be 2 NB");
    float* fac = reinterpret_cast<float*>(P.d_fac);
    float2* dinv = reinterpret_cast<float2*>(P.d_dinv);
    const int mp = P.mp, nb = P.nblk;
    const int ntile_max = (mp - NB + TC_BM - 1) / TC_BM;
    const size_t abytes = (size_t)nb * ntile_max * Cfg::A_BYTES;
    const size_t bbytes = (size_t)nb * ntile_max * Cfg::B_BYTES;
    if (P.pack_bytes < abytes + bbytes) {
        if (P.d_pack) cudaFree(P.d_pack);
        P.d_pack = nullptr;
        P.pack_bytes = 0;
        FDE_CUDA_TRY(cudaMalloc(&P.d_pack, abytes + bbytes));
        P.pack_bytes = abytes + bbytes;
        FDE_CUDA_TRY(cudaMemsetAsync(P.d_pack, 0, abytes + bbytes, st));
    }
    unsigned char* apack = reinterpret_cast<unsigned char*>(P.d_pack);
    unsigned char* bpack = apack + abytes;
    {
        dim3 grid(mp < 64 ? mp : 64, nb);
        StageTimer t(P, FDE_STAGE_FORM);
        form_blocks_kernel<float><<<grid, 256, 0, st>>>(P.m, mp, P.h, P.dxa, P.d_g, P.d_dplus, P.d_dminus,
                                                        P.d_phi, P.d_psi, fac);
        FDE_LAUNCH_CHECK("form_blocks_kernel");
    }
    // at most 2 CTAs per SM: each holds 256 of the SM's 512 TMEM columns
    const int smem = (Cfg::A_BYTES + Cfg::B_BYTES) > 100 * 1024 ? (Cfg::A_BYTES + Cfg::B_BYTES) : 100 * 1024;
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_tc_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const size_t panel_smem = (size_t)RC * (NB + 1) * sizeof(float2);
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_panel_kernel<float, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)panel_smem));
    const int steps = mp / NB;
    for (int p = 0; p < steps; ++p) {
        {
            StageTimer t(P, FDE_STAGE_LU_DIAG);
            lu_diag_kernel<float><<<nb, 256, 0, st>>>(mp, p, fac, dinv, P.d_info);
            FDE_LAUNCH_CHECK("lu_diag_kernel");
        }
        const int rest = (p + 1) * NB;
        const int rem = mp - rest;
        if (rem <= 0) break;
        const int nch = (rem + RC - 1) / RC;
        {
            StageTimer t(P, FDE_STAGE_LU_PANEL);
            lu_panel_kernel<float, KIND><<<dim3(2 * nch, nb), RC, panel_smem, st>>>(mp, p, nch, fac, apack, bpack,
                                                                                ntile_max);
            FDE_LAUNCH_CHECK("lu_panel_kernel");
        }
        const int nt = (rem + TC_BM - 1) / TC_BM;
        StageTimer t(P, FDE_STAGE_LU_UPDATE);
        lu_update_tc_kernel<KIND><<<dim3(nt * nt, nb), 128, smem, st>>>(mp, rest, nt, ntile_max, fac, apack, bpack,
                                                                        P.d_err);
        FDE_LAUNCH_CHECK("lu_update_tc_kernel");
    }
    return FDE_OK;
}

// Batched LU over a block table sorted by m_p (descending): at step p the blocks
// still being factored form a prefix of the table.  FP32 storage; trailing
// updates on CUDA cores (FDE_FP32) or tcgen05 (FDE_TF32 / FDE_BF16).
template <int KIND>
static int run_lu_batched(const BlkDev* d_blk, const std::vector<int>& mps, int* err, cudaStream_t st) {
    const int nbt = (int)mps.size();
    const int max_mp = mps[0];
    {
        form_blocks_batched<float><<<dim3(64, nbt), 256, 0, st>>>(d_blk);
        FDE_LAUNCH_CHECK("form_blocks_batched");
    }
    const size_t panel_smem = (size_t)RC * (NB + 1) * sizeof(float2);
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_panel_batched<float, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)panel_smem));
    const size_t upd_smem = (64 * (NB + 1) + NB * 65) * sizeof(float2);
    int tc_smem = 0;
    if constexpr (KIND >= 0) {
        using Cfg = TcCfg<KIND>;
        tc_smem = (Cfg::A_BYTES + Cfg::B_BYTES) > 100 * 1024 ? (Cfg::A_BYTES + Cfg::B_BYTES) : 100 * 1024;
        FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_tc_batched<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tc_smem));
    } else {
        FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)upd_smem));
    }
    for (int p = 0; p * NB < max_mp; ++p) {
        int nd = 0, nu = 0;
        while (nd < nbt && mps[nd] > p * NB) ++nd;
        while (nu < nbt && mps[nu] > (p + 1) * NB) ++nu;
        lu_diag_batched<float><<<nd, 256, 0, st>>>(d_blk, p);
        FDE_LAUNCH_CHECK("lu_diag_batched");
        if (nu == 0) break;
        const int rem = max_mp - (p + 1) * NB;
        const int nch = (rem + RC - 1) / RC;
        lu_panel_batched<float, KIND><<<dim3(2 * nch, nu), RC, panel_smem, st>>>(d_blk, p);
        FDE_LAUNCH_CHECK("lu_panel_batched");
        if constexpr (KIND >= 0) {
            const int ntg = (rem + TC_BM - 1) / TC_BM;
            lu_update_tc_batched<KIND><<<dim3(ntg * ntg, nu), 128, tc_smem, st>>>(d_blk, p, NB, ntg, err);
            FDE_LAUNCH_CHECK("lu_update_tc_batched");
        } else {
            const int ntg = (rem + 63) / 64;
            lu_update_batched<float><<<dim3(ntg * ntg, nu), 256, upd_smem, st>>>(d_blk, p, ntg);
            FDE_LAUNCH_CHECK("lu_update_batched");
        }
    }
    return FDE_OK;
}

int launch_lu_batched(const BlkDev* d_blk, const std::vector<int>& mp_sorted, int precision, int* err,
                      cudaStream_t st) {
    if (mp_sorted.empty()) return FDE_OK;
    if (precision == FDE_TF32) return run_lu_batched<0>(d_blk, mp_sorted, err, st);
    if (precision == FDE_BF16) return run_lu_batched<1>(d_blk, mp_sorted, err, st);
    return run_lu_batched<-1>(d_blk, mp_sorted, err, st);
}

int launch_trsv_batched(const InstDev* I, const int* act, int nact, int max_nblk, int max_mp, cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    const size_t smem = ((size_t)max_mp + 2 * 32 * 33) * sizeof(float2);
    FDE_CUDA_TRY(cudaFuncSetAttribute(block_trsv_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    block_trsv_batched<float><<<dim3(max_nblk, nact), TRSV_THREADS, smem, st>>>(I, act);
    FDE_LAUNCH_CHECK("block_trsv_batched");
    return FDE_OK;
}

int launch_block_lu(Problem& P, int prec, cudaStream_t st) {
    if (prec == FDE_FP64) return run_lu<double>(P, st);
    if (prec == FDE_TF32) return run_lu_tc<0>(P, st);
    if (prec == FDE_BF16) return run_lu_tc<1>(P, st);
    return run_lu<float>(P, st);
}

int launch_block_trsv(const Problem& P, void* rhat, cudaStream_t st) {
    if (P.precision == FDE_FP64) {
        size_t smem = ((size_t)P.mp + 2 * 32 * 33) * sizeof(double2);
        FDE_CUDA_TRY(cudaFuncSetAttribute(block_trsv_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        block_trsv_kernel<double><<<P.nblk, TRSV_THREADS, smem, st>>>(P.mp, (const double*)P.d_fac,
                                                                       (const double2*)P.d_dinv, (double2*)rhat);
    } else {
        size_t smem = ((size_t)P.mp + 2 * 32 * 33) * sizeof(float2);
        FDE_CUDA_TRY(cudaFuncSetAttribute(block_trsv_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        block_trsv_kernel<float><<<P.nblk, TRSV_THREADS, smem, st>>>(P.mp, (const float*)P.d_fac,
                                                                      (const float2*)P.d_dinv, (float2*)rhat);
    }
    FDE_LAUNCH_CHECK("block_trsv_kernel");
    return FDE_OK;
}

}  // namespace fde
