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
//   3. lu_update: A22 -= L21 U12 (complex GEMM on CUDA cores; the two-level
//                 tensor-core variant is run_lu_tc below, its tile kernels in
//                 lu_tc2.cuh and lu_tc2w.cuh)
#include <algorithm>

#include <cuda.h>  // CUtensorMap (the encoder is fetched from the driver at run time)

#include "fde_internal.h"
#include "fft_device.cuh"
#include "lu_tc2.cuh"
#include "lu_tc2w.cuh"
#include "lu_tc2s.cuh"

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
// per-row coefficients dx^-alpha d+_i, dx^-alpha d-_i and of h psi_k.  The CTA
// stages g_0..g_{m+1} in shared memory in the block's precision (dynamic shared
// memory of (m + 2) elements), so no element converts FP64 values.
template <typename T>
__device__ __forceinline__ void form_body(int m, int mp, double h, double dxa, const double* __restrict__ g,
                                          const double* __restrict__ dp, const double* __restrict__ dm, double2 ph,
                                          double2 ps, T* __restrict__ re, int row0, int rowstride) {
    extern __shared__ __align__(16) unsigned char form_smem[];
    T* gs = reinterpret_cast<T*>(form_smem);
    for (int q = threadIdx.x; q < m + 2; q += blockDim.x) gs[q] = (T)g[q];
    __syncthreads();
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
                if (a >= 0) jv += rp * gs[a];
                if (b >= 0) jv += rm * gs[b];
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
// tensor-core operand tiles (A' from L21 rows, B' from U12 columns; see lu_tc2.cuh).
constexpr int RC = 128;
// Ranges: rows mode over rows [rb, rend) against the diagonal block at (od, od);
// columns mode over columns [cb, cend).  Tensor-core packing (PACK >= 0): rows r >= R0
// of L21 go to A' tiles at K' offset kq (Re) and TB + kq (Im), columns >= R0 of U12 to
// B' tiles at K offset kq (rows j: Re, TB + j: Im) -- the layout of lu_tc2.cuh.
template <typename T, int PACK>
__device__ __forceinline__ void panel_body(int mp, int od, int rb, int rend, int cb, int cend, int nrow,
                                           T* __restrict__ re, unsigned char* __restrict__ apack,
                                           unsigned char* __restrict__ bpack, int R0, int kq, int bx) {
    using C = cplx_t<T>;
    __shared__ C D[NB][NB + 1];
    __shared__ C dinv_s[NB];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C (*X)[NB + 1] = reinterpret_cast<C (*)[NB + 1]>(smem_raw);  // [RC][NB+1]
    T* im = re + (size_t)mp * mp;
    const int o = od;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        const size_t idx = (size_t)(o + r) * mp + o + c;
        D[r][c] = mk(re[idx], im[idx]);
    }
    const bool rows = bx < nrow;
    const int chunk = rows ? bx : bx - nrow;
    const int b0 = (rows ? rb : cb) + chunk * RC;
    const int bend = rows ? rend : cend;
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
        X[q][c] = (b0 + q < bend) ? mk(re[idx], im[idx]) : mk(T(0), T(0));
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
        if (b0 + qq < bend) {
            re[idx] = X[qq][c].x;
            im[idx] = X[qq][c].y;
            if constexpr (PACK >= 0) {
                using Cfg = Tc2<PACK>;
                const int g = b0 + qq - R0;  // position in the outer trailing matrix
                if (g >= 0) {
                    const int tile = g / T2_BM, rt = g % T2_BM;
                    const float vr = (float)X[qq][c].x, vi = (float)X[qq][c].y;
                    if (rows) {
                        unsigned char* t = apack + (size_t)tile * Cfg::A_TILE;
                        pack2_store<PACK>(t, T2_BM, rt, kq + c, vr, false);
                        pack2_store<PACK>(t, T2_BM, rt, TB + kq + c, vi, false);
                    } else {
                        unsigned char* t = bpack + (size_t)tile * Cfg::B_TILE;
                        pack2_store<PACK>(t, 2 * T2_BN, rt, kq + c, vr, true);  // Re part
                        pack2_store<PACK>(t, 2 * T2_BN, T2_BN + rt, kq + c, vi, true);  // Im part
                    }
                }
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(RC)
lu_panel_kernel(int mp, int p, int nrow, T* __restrict__ fac) {
    const int k = blockIdx.y;
    const int rest = (p + 1) * NB;
    panel_body<T, -1>(mp, p * NB, rest, mp, rest, mp, nrow, plane_re(fac, k, mp), nullptr, nullptr, 0, 0, blockIdx.x);
}

// General ranges (two-level LU): grid (nrow + ncol, nblk).
template <typename T, int PACK>
__global__ void __launch_bounds__(RC)
lu_panel_range_kernel(int mp, int od, int rb, int rend, int cb, int cend, int nrow, T* __restrict__ fac,
                      unsigned char* __restrict__ apack, unsigned char* __restrict__ bpack, size_t pack_a_stride,
                      size_t pack_b_stride, int R0, int kq) {
    const int k = blockIdx.y;
    panel_body<T, PACK>(mp, od, rb, rend, cb, cend, nrow, plane_re(fac, k, mp),
                        apack ? apack + k * pack_a_stride : nullptr, bpack ? bpack + k * pack_b_stride : nullptr, R0,
                        kq, blockIdx.x);
}

template <typename T, int PACK>
__global__ void __launch_bounds__(RC) lu_panel_batched(const BlkDev* __restrict__ B, int p) {
    const BlkDev& d = B[blockIdx.y];
    const int rest = (p + 1) * NB;
    const int rem = d.mp - rest;
    if (rem <= 0) return;
    const int nrow = (rem + RC - 1) / RC;
    if ((int)blockIdx.x >= 2 * nrow) return;
    panel_body<T, PACK>(d.mp, p * NB, rest, d.mp, rest, d.mp, nrow, (T*)d.fac, d.apack, d.bpack, 0, 0, blockIdx.x);
}

// Batched general ranges; the ranges are relative to the outer step offset o and
// clipped to each block's m_p.
template <typename T, int PACK>
__global__ void __launch_bounds__(RC)
lu_panel_range_batched(const BlkDev* __restrict__ B, int od, int rows_from, int cols_from, int cols_to, int R0,
                       int kq) {
    const BlkDev& d = B[blockIdx.y];
    if (od + NB > d.mp) return;
    const int rend = d.mp, cend = cols_to < d.mp ? cols_to : d.mp;
    const int nrow = rows_from < rend ? (rend - rows_from + RC - 1) / RC : 0;
    const int ncol = cols_from < cend ? (cend - cols_from + RC - 1) / RC : 0;
    if ((int)blockIdx.x >= nrow + ncol) return;
    panel_body<T, PACK>(d.mp, od, rows_from, rend, cols_from, cend, nrow, (T*)d.fac, d.apack, d.bpack, R0, kq,
                        blockIdx.x);
}

// Trailing update A22 -= L21 U12 on CUDA cores: 64 x 64 output tile per CTA,
// 4 x 4 complex outputs per thread, K = NB.
// C[r][c] -= sum_{k<NB} L[r][kb+k] U[kb+k][c] over the 64 x 64 tile at (r0, c0),
// rows < rend, columns < cend.
template <typename T>
__device__ __forceinline__ void update_body(int mp, int kb, int r0, int c0, int rend, int cend, T* __restrict__ re) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C (*Ls)[NB + 1] = reinterpret_cast<C (*)[NB + 1]>(smem_raw);                        // [64][NB+1]
    C (*Us)[64 + 1] = reinterpret_cast<C (*)[64 + 1]>(smem_raw + 64 * (NB + 1) * sizeof(C));  // [NB][65]
    T* im = re + (size_t)mp * mp;
    const int o = kb;
    for (int e = threadIdx.x; e < 64 * NB; e += blockDim.x) {
        const int q = e / NB, c = e % NB;
        const int r = r0 + q;
        Ls[q][c] = r < rend ? mk(re[(size_t)r * mp + o + c], im[(size_t)r * mp + o + c]) : mk(T(0), T(0));
        const int c2 = e / 64, q2 = e % 64;
        const int cc = c0 + q2;
        Us[c2][q2] = cc < cend ? mk(re[(size_t)(o + c2) * mp + cc], im[(size_t)(o + c2) * mp + cc]) : mk(T(0), T(0));
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
        if (r >= rend) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = c0 + tc + 16 * b;
            if (c >= cend) continue;
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
    const int rest = (p + 1) * NB;
    update_body<T>(mp, p * NB, rest + (blockIdx.x / ntile) * 64, rest + (blockIdx.x % ntile) * 64, mp, mp,
                   plane_re(fac, k, mp));
}

// General ranges: rows [rb, rend) x columns [cb, cend), K block [kb, kb+NB); grid (ntr * ntc, nblk).
template <typename T>
__global__ void __launch_bounds__(256)
lu_update_range_kernel(int mp, int kb, int rb, int rend, int cb, int cend, int ntc, T* __restrict__ fac) {
    const int k = blockIdx.y;
    update_body<T>(mp, kb, rb + (blockIdx.x / ntc) * 64, cb + (blockIdx.x % ntc) * 64, rend, cend,
                   plane_re(fac, k, mp));
}

template <typename T>
__global__ void __launch_bounds__(256)
lu_update_range_batched(const BlkDev* __restrict__ B, int kb, int rb, int rend_max, int cb, int cend_max, int ntc) {
    const BlkDev& d = B[blockIdx.y];
    const int rend = rend_max < d.mp ? rend_max : d.mp;
    const int cend = cend_max < d.mp ? cend_max : d.mp;
    const int r0 = rb + (blockIdx.x / ntc) * 64, c0 = cb + (blockIdx.x % ntc) * 64;
    if (kb + NB > d.mp || r0 >= rend || c0 >= cend) return;
    update_body<T>(d.mp, kb, r0, c0, rend, cend, (T*)d.fac);
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
    update_body<T>(d.mp, p * NB, (p + 1) * NB + ti * 64, (p + 1) * NB + tj * 64, d.mp, d.mp, (T*)d.fac);
}

// Forward (unit lower L) then backward (U) substitution for one block per CTA, in
// place on rhat[k] (length mp), column-oriented over 32-row tiles.  Step d of a
// sweep resolves tile T(d) (T(d) = d forward, nt-1-d backward) and subtracts the
// 32-column strip of L (U) below (above) it, times the 32 new values, from the
// remaining right-hand side.
//
// The dependency chain (tile d needs the strips of every earlier tile) is kept off
// the warps that stream the factor planes:
//   * warp 0, the solver, resolves the diagonal tiles.  Before solving tile d it
//     applies strip d-1 to tile d's own rows itself (look-ahead), so it only needs
//     the streaming warps to have finished tile d's rows of strips <= d-2.  Its
//     diagonal and look-ahead tiles arrive by cp.async two steps ahead.
//   * warps 1..15 stream strip d over the rows of tiles d+2, d+3, ... (tile d+2
//     first), eight threads per row, each factor element read once with 16-byte
//     streaming loads.  The loads of a strip's first batch are issued before the
//     wait for its 32 values, so the memory pipe does not drain between strips.
// The two sides hand over through named barriers (producer arrives, consumer
// syncs): X[d&1] -- x_d is in shared memory; B[d&1] -- strip d has reached every
// row of tile d+2.  A barrier id is reused only every other step, after its
// previous phase has completed (the solver passes B of step d before it arrives on
// X of step d+2; the streaming warps pass X of step d+2 before they arrive on B of
// step d+2), so phases never mix.  All waits are hardware barriers of this CTA.
struct dvec4 {
    double x, y, z, w;
};
template <typename T> struct vec4;
template <> struct vec4<float> { using type = float4; };
template <> struct vec4<double> { using type = dvec4; };

// Streaming loads (the factor planes are read once per solve).
__device__ __forceinline__ float4 ld4(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ dvec4 ld4(const double* p) {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    return dvec4{a.x, a.y, b.x, b.y};
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void named_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

constexpr int TRSV_THREADS = 512;                           // the default launch shape
constexpr int TRSV_TPR = 8;                                  // threads per row in the strip update
constexpr int TRSV_BAR_X = 1, TRSV_BAR_B = 3;                // named barrier ids (+ d & 1)
// Rows per group whose loads are in flight together: 8 x 2 x 16 B per thread for
// FP32 factors; FP64 rows are twice as wide per element, 4 keep it spill-free.
template <typename T> struct trsv_unroll { static constexpr int value = sizeof(T) == 4 ? 8 : 4; };
// Launch shapes of the block solves (FDE_TUNE_TRSV): NT threads (warp 0 the solver,
// NT/32 - 1 streaming warps of (NT - 32) / TRSV_TPR row groups) and H rows per
// register buffer.  The arithmetic of every row does not depend on the shape: each
// row's strip product is the same 32-term sum, reduced by the same TRSV_TPR lanes in
// the same order, so all shapes give bit-identical results.
template <typename T, int V> struct trsv_shape;
template <typename T> struct trsv_shape<T, 0> { static constexpr int NT = 512, H = trsv_unroll<T>::value / 2; };
template <typename T> struct trsv_shape<T, 1> { static constexpr int NT = 384, H = trsv_unroll<T>::value; };
template <typename T> struct trsv_shape<T, 2> { static constexpr int NT = 640, H = trsv_unroll<T>::value / 4; };
// Solver tiles in shared memory: planar, rows padded by 16 bytes (16-byte aligned
// cp.async destinations); [buffer 2][D, L][Re, Im][32][LD].
template <typename T> struct trsv_tile { static constexpr int LD = 32 + 16 / (int)sizeof(T); };

__host__ __device__ static size_t trsv_smem_bytes(int mp, size_t elem) {
    const size_t ld = 32 + 16 / elem;
    return (size_t)mp * 2 * elem + 8 * 32 * ld * elem;
}

// 32 x 32 tile with row pitch `pitch` (elements) -> shared tile with pitch LD.
template <typename T>
__device__ __forceinline__ void tile_async(T* dst, const T* src, size_t pitch, int lane) {
    constexpr int EPC = 16 / (int)sizeof(T), CPR = 32 / EPC, LD = trsv_tile<T>::LD;
    for (int e = lane; e < 32 * CPR; e += 32) {
        const int r = e / CPR, ch = e % CPR;
        cp_async16(dst + r * LD + ch * EPC, src + (size_t)r * pitch + ch * EPC);
    }
}
template <typename T>
__device__ __forceinline__ void tile_async(T* dst, const T* plane, int mp, int r0, int c0, int lane) {
    tile_async<T>(dst, plane + (size_t)r0 * mp + c0, (size_t)mp, lane);
}

// Factor planes as the block solves read them (LAY): 0 row-major in the compute type
// (element (r, c) at r m_p + c); 1 strip-major in the compute type (32-column strips
// one after the other, each strip's rows contiguous: (c / 32) 32 m_p + 32 r + c mod 32),
// so every strip of a sweep is one sequential stream; 2 strip-major in bfloat16 (FP32
// compute).  The tensor-core LU writes the final factor row-major and, where it can,
// in one of the strip-major forms as well.
constexpr int LAY_PLANES = 0, LAY_STRIPS = 1, LAY_STRIPS_BF16 = 2;
template <int LAY>
__device__ __forceinline__ size_t fac_at(int mp, int r, int c) {
    return LAY != LAY_PLANES ? (size_t)(c >> 5) * 32 * mp + (size_t)r * 32 + (c & 31) : (size_t)r * mp + c;
}
template <typename T, int LAY>
__device__ __forceinline__ void tile_async_l(T* dst, const T* plane, int mp, int r0, int c0, int lane) {
    tile_async<T>(dst, plane + fac_at<LAY>(mp, r0, c0), LAY != LAY_PLANES ? (size_t)32 : (size_t)mp, lane);
}
// Element type of the factor as stored for layout LAY, and its streaming loads: four
// consecutive entries of one row, widened to the compute type (a bfloat16 is the top
// half of the float it came from, so the widening is exact).
template <typename T, int LAY> struct fac_store {
    using elem = T;
    using raw = typename vec4<T>::type;
    static __device__ __forceinline__ raw load(const elem* p) { return ld4(p); }
    static __device__ __forceinline__ raw widen(const raw& v) { return v; }
};
template <> struct fac_store<float, LAY_STRIPS_BF16> {
    using elem = unsigned short;
    using raw = uint2;
    static __device__ __forceinline__ raw load(const elem* p) { return __ldcs(reinterpret_cast<const uint2*>(p)); }
    static __device__ __forceinline__ float4 widen(const raw& v) {
        return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                           __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
    }
};
// 32 x 32 bfloat16 tile of a strip (rows of 64 bytes, contiguous) -> shared rows of
// TRSV_LDH elements (80 bytes: 16-byte aligned cp.async destinations).
constexpr int TRSV_LDH = 40;
__device__ __forceinline__ void tile_async_bf16(unsigned short* dst, const unsigned short* src, int lane) {
    for (int e = lane; e < 32 * 4; e += 32) {
        const int r = e >> 2, ch = e & 3;
        cp_async16(dst + r * TRSV_LDH + ch * 8, src + r * 32 + ch * 8);
    }
}

// Solver side of one sweep (warp 0).  INV: the inverted diagonal tiles are given
// (tinv: per tile [L^-1 re, L^-1 im, U^-1 re, U^-1 im][32][32]) and a tile solve is
// the product x = D^-1 a; otherwise the tile is solved by substitution.
template <typename T, bool FWD, bool INV, int NT, int LAY = LAY_PLANES>
__device__ __forceinline__ void trsv_solver(int mp, int nt, const typename fac_store<T, LAY>::elem* re,
                                            const typename fac_store<T, LAY>::elem* im, const cplx_t<T>* dv,
                                            const T* tinv, cplx_t<T>* y, cplx_t<T> (*xs)[32], T* tiles,
                                            cplx_t<T>* av, int lane) {
    using C = cplx_t<T>;
    static_assert(INV || LAY != LAY_STRIPS_BF16, "substitution reads the diagonal tiles in the compute type");
    constexpr int LD = trsv_tile<T>::LD, TS = 32 * LD;
    auto tile_of = [&](int d) { return FWD ? d : nt - 1 - d; };
    auto issue = [&](int d) {
        T* b = tiles + (d & 1) * 4 * TS;  // [D re, D im, L re, L im]
        const int j = tile_of(d);
        if (INV) {
            const T* ti = tinv + (size_t)j * 4096 + (FWD ? 0 : 2048);
            tile_async<T>(b, ti, 32, lane);
            tile_async<T>(b + TS, ti + 1024, 32, lane);
        } else if constexpr (LAY != LAY_STRIPS_BF16) {
            tile_async_l<T, LAY>(b, re, mp, 32 * j, 32 * j, lane);
            tile_async_l<T, LAY>(b + TS, im, mp, 32 * j, 32 * j, lane);
        }
        if (d >= 1) {
            if constexpr (LAY == LAY_STRIPS_BF16) {  // bfloat16 rows in the L slots
                const size_t o = fac_at<LAY>(mp, 32 * j, 32 * tile_of(d - 1));
                tile_async_bf16(reinterpret_cast<unsigned short*>(b + 2 * TS), re + o, lane);
                tile_async_bf16(reinterpret_cast<unsigned short*>(b + 3 * TS), im + o, lane);
            } else {
                tile_async_l<T, LAY>(b + 2 * TS, re, mp, 32 * j, 32 * tile_of(d - 1), lane);
                tile_async_l<T, LAY>(b + 3 * TS, im, mp, 32 * j, 32 * tile_of(d - 1), lane);
            }
        }
    };
    issue(0);
    cp_async_commit();
    if (nt > 1) issue(1);
    cp_async_commit();
    for (int d = 0; d < nt; ++d) {
        const int r0 = 32 * tile_of(d);
        const T* Dre = tiles + (d & 1) * 4 * TS;
        const T* Dim = Dre + TS;
        const T* Lre = Dre + 2 * TS;
        const T* Lim = Dre + 3 * TS;
        cp_async_wait1();
        __syncwarp();
        if (d >= 2) named_sync(TRSV_BAR_B + (d & 1), NT);  // strip d-2 has reached tile d
        C a = y[r0 + lane];
        // Every product below is written as explicit fused multiply-adds, so that the
        // rounding is fixed by the source and not by how the compiler contracts a
        // particular instantiation (the launch shapes must give bit-identical results).
        if (d >= 1) {  // look-ahead: strip d-1 on tile d's rows
            const C* xp = xs[(d - 1) & 1];
            T sx0 = 0, sy0 = 0, sx1 = 0, sy1 = 0;
#pragma unroll
            for (int c = 0; c < 32; c += 2) {
                const C x0 = xp[c], x1 = xp[c + 1];
                T l0r, l0i, l1r, l1i;
                if constexpr (LAY == LAY_STRIPS_BF16) {  // a pair of bfloat16 per 32-bit word
                    const uint32_t wr = reinterpret_cast<const uint32_t*>(Lre)[lane * (TRSV_LDH / 2) + c / 2];
                    const uint32_t wi = reinterpret_cast<const uint32_t*>(Lim)[lane * (TRSV_LDH / 2) + c / 2];
                    l0r = __uint_as_float(wr << 16);
                    l1r = __uint_as_float(wr & 0xffff0000u);
                    l0i = __uint_as_float(wi << 16);
                    l1i = __uint_as_float(wi & 0xffff0000u);
                } else {
                    l0r = Lre[lane * LD + c];
                    l0i = Lim[lane * LD + c];
                    l1r = Lre[lane * LD + c + 1];
                    l1i = Lim[lane * LD + c + 1];
                }
                sx0 = fma(-l0i, x0.y, fma(l0r, x0.x, sx0));
                sy0 = fma(l0i, x0.x, fma(l0r, x0.y, sy0));
                sx1 = fma(-l1i, x1.y, fma(l1r, x1.x, sx1));
                sy1 = fma(l1i, x1.x, fma(l1r, x1.y, sy1));
            }
            a.x -= sx0 + sx1;
            a.y -= sy0 + sy1;
        }
        if (INV) {  // x = D^-1 a (D^-1 stored with its zeros and unit / inverted diagonal)
            av[lane] = a;
            __syncwarp();
            T sx0 = 0, sy0 = 0, sx1 = 0, sy1 = 0;
#pragma unroll
            for (int c = 0; c < 32; c += 2) {
                const C a0 = av[c], a1 = av[c + 1];
                const T d0r = Dre[lane * LD + c], d0i = Dim[lane * LD + c];
                const T d1r = Dre[lane * LD + c + 1], d1i = Dim[lane * LD + c + 1];
                sx0 = fma(-d0i, a0.y, fma(d0r, a0.x, sx0));
                sy0 = fma(d0i, a0.x, fma(d0r, a0.y, sy0));
                sx1 = fma(-d1i, a1.y, fma(d1r, a1.x, sx1));
                sy1 = fma(d1i, a1.x, fma(d1r, a1.y, sy1));
            }
            a.x = sx0 + sx1;
            a.y = sy0 + sy1;
        } else if (FWD) {
#pragma unroll 8
            for (int c = 0; c < 32; ++c) {
                const T yx = __shfl_sync(0xffffffffu, a.x, c);
                const T yy = __shfl_sync(0xffffffffu, a.y, c);
                if (lane > c) {
                    const T lr = Dre[lane * LD + c], li = Dim[lane * LD + c];
                    a.x = fma(li, yy, fma(-lr, yx, a.x));
                    a.y = fma(-li, yx, fma(-lr, yy, a.y));
                }
            }
        } else {
            const C di = dv[r0 + lane];
#pragma unroll 8
            for (int c = 31; c >= 0; --c) {
                if (lane == c) a = cmul(a, di);
                const T yx = __shfl_sync(0xffffffffu, a.x, c);
                const T yy = __shfl_sync(0xffffffffu, a.y, c);
                if (lane < c) {
                    const T ur = Dre[lane * LD + c], ui = Dim[lane * LD + c];
                    a.x = fma(ui, yy, fma(-ur, yx, a.x));
                    a.y = fma(-ui, yx, fma(-ur, yy, a.y));
                }
            }
        }
        y[r0 + lane] = a;
        xs[d & 1][lane] = a;
        __syncwarp();
        if (d <= nt - 3) named_arrive(TRSV_BAR_X + (d & 1), NT);
        if (d + 2 < nt) issue(d + 2);  // buffer d & 1 is free again
        cp_async_commit();
    }
}

// Streaming side of one sweep (warps 1..15): strip d over rows of tiles >= d+2.
// Row index q in [0, len) maps to row lo + q forward and hi - 1 - q backward, so
// tile d+2's rows are q < 32 in both directions.  The four groups of a warp hold
// q values of one aligned quartet and len is a multiple of 32, so loop exits and
// the shuffles stay warp-uniform.  Two register buffers of H rows alternate: the
// loads of one are in flight while the other is applied, so the load pipe does
// not drain between batches.
template <typename T, bool FWD, int NT, int H, int LAY = LAY_PLANES>
__device__ __forceinline__ void trsv_stream(int mp, int nt, const typename fac_store<T, LAY>::elem* re,
                                            const typename fac_store<T, LAY>::elem* im, cplx_t<T>* y,
                                            const cplx_t<T> (*xs)[32], int bt) {
    using C = cplx_t<T>;
    using V = typename vec4<T>::type;
    using FS = fac_store<T, LAY>;
    constexpr int TRSV_GROUPS = (NT - 32) / TRSV_TPR;  // a multiple of 4 (NT is a multiple of 32)
    constexpr int HG = H * TRSV_GROUPS;
    static_assert(HG >= 32, "the first batch must cover tile d+2");
    const int g = bt / TRSV_TPR, sub = bt % TRSV_TPR;
    for (int d = 0; d + 2 < nt; ++d) {
        const int col = 32 * (FWD ? d : nt - 1 - d) + sub * 4;
        const int lo = FWD ? 32 * (d + 2) : 0;
        const int hi = FWD ? mp : 32 * (nt - 2 - d);
        const int len = hi - lo;
        typename FS::raw ar[2][H], ai[2][H];
        auto load = [&](int b, int q0) {
#pragma unroll
            for (int u = 0; u < H; ++u) {
                const int q = q0 + u * TRSV_GROUPS;
                if (q < len) {
                    const int r = FWD ? lo + q : hi - 1 - q;
                    ar[b][u] = FS::load(re + fac_at<LAY>(mp, r, col));
                    ai[b][u] = FS::load(im + fac_at<LAY>(mp, r, col));
                }
            }
        };
        C x0, x1, x2, x3;
        auto apply = [&](int b, int q0) {
#pragma unroll
            for (int u = 0; u < H; ++u) {
                const int q = q0 + u * TRSV_GROUPS;
                const V vr = FS::widen(ar[b][u]);
                const V vi = FS::widen(ai[b][u]);
                // explicit fused multiply-adds: the same rounding in every launch shape
                T sx = vr.x * x0.x;
                sx = fma(-vi.x, x0.y, sx);
                sx = fma(vr.y, x1.x, sx);
                sx = fma(-vi.y, x1.y, sx);
                sx = fma(vr.z, x2.x, sx);
                sx = fma(-vi.z, x2.y, sx);
                sx = fma(vr.w, x3.x, sx);
                sx = fma(-vi.w, x3.y, sx);
                T sy = vr.x * x0.y;
                sy = fma(vi.x, x0.x, sy);
                sy = fma(vr.y, x1.y, sy);
                sy = fma(vi.y, x1.x, sy);
                sy = fma(vr.z, x2.y, sy);
                sy = fma(vi.z, x2.x, sy);
                sy = fma(vr.w, x3.y, sy);
                sy = fma(vi.w, x3.x, sy);
#pragma unroll
                for (int off = 1; off < TRSV_TPR; off <<= 1) {
                    sx += __shfl_xor_sync(0xffffffffu, sx, off);
                    sy += __shfl_xor_sync(0xffffffffu, sy, off);
                }
                if (sub == 0 && q < len) {
                    const int r = FWD ? lo + q : hi - 1 - q;
                    C v = y[r];
                    v.x -= sx;
                    v.y -= sy;
                    y[r] = v;
                }
            }
        };
        load(0, g);  // independent of x_d: in flight across the wait
        load(1, g + HG);
        named_sync(TRSV_BAR_X + (d & 1), NT);
        x0 = xs[d & 1][sub * 4];
        x1 = xs[d & 1][sub * 4 + 1];
        x2 = xs[d & 1][sub * 4 + 2];
        x3 = xs[d & 1][sub * 4 + 3];
        apply(0, g);  // covers q < 32 (tile d+2): groups 0..31, u = 0
        named_arrive(TRSV_BAR_B + (d & 1), NT);
        for (int q0 = g + HG; q0 < len; q0 += 2 * HG) {
            load(0, q0 + HG);
            apply(1, q0);
            if (q0 + HG >= len) break;
            load(1, q0 + 2 * HG);
            apply(0, q0 + HG);
        }
    }
}

// Streaming side for the bfloat16 strip copy: a row's 32 entries of a strip are 64
// bytes, so four lanes take a row, eight entries (one 16-byte load per plane) each, and
// a warp's load covers eight consecutive rows (512 contiguous bytes).  Row groups of a
// warp hold q values of one aligned octet (GROUPS is a multiple of 8), so the loop exits
// and shuffles stay warp-uniform.  Otherwise as trsv_stream; every launch shape sums a
// row's products in the same order, so the shapes agree bit for bit.
constexpr int TRSV_TPR_H = 4;  // threads per row of the bfloat16 stream
__device__ __forceinline__ void widen8(const uint4& v, float* f) {
    f[0] = __uint_as_float(v.x << 16); f[1] = __uint_as_float(v.x & 0xffff0000u);
    f[2] = __uint_as_float(v.y << 16); f[3] = __uint_as_float(v.y & 0xffff0000u);
    f[4] = __uint_as_float(v.z << 16); f[5] = __uint_as_float(v.z & 0xffff0000u);
    f[6] = __uint_as_float(v.w << 16); f[7] = __uint_as_float(v.w & 0xffff0000u);
}
template <bool FWD, int NT, int H>
__device__ __forceinline__ void trsv_stream_bf16(int mp, int nt, const unsigned short* re, const unsigned short* im,
                                                 float2* y, const float2 (*xs)[32], int bt) {
    constexpr int GROUPS = (NT - 32) / TRSV_TPR_H;
    constexpr int HG = H * GROUPS;
    static_assert(GROUPS % 8 == 0, "a warp's row groups must form aligned octets");
    static_assert(HG >= 32, "the first batch must cover tile d+2");
    const int g = bt / TRSV_TPR_H, sub = bt % TRSV_TPR_H;
    for (int d = 0; d + 2 < nt; ++d) {
        const int col = 32 * (FWD ? d : nt - 1 - d) + sub * 8;
        const int lo = FWD ? 32 * (d + 2) : 0;
        const int hi = FWD ? mp : 32 * (nt - 2 - d);
        const int len = hi - lo;
        uint4 ar[2][H], ai[2][H];
        auto load = [&](int b, int q0) {
#pragma unroll
            for (int u = 0; u < H; ++u) {
                const int q = q0 + u * GROUPS;
                if (q < len) {
                    const int r = FWD ? lo + q : hi - 1 - q;
                    const size_t o = fac_at<LAY_STRIPS_BF16>(mp, r, col);
                    ar[b][u] = __ldcs(reinterpret_cast<const uint4*>(re + o));
                    ai[b][u] = __ldcs(reinterpret_cast<const uint4*>(im + o));
                }
            }
        };
        float2 x[8];
        auto apply = [&](int b, int q0) {
#pragma unroll
            for (int u = 0; u < H; ++u) {
                const int q = q0 + u * GROUPS;
                float vr[8], vi[8];
                widen8(ar[b][u], vr);
                widen8(ai[b][u], vi);
                float sx = vr[0] * x[0].x;
                sx = fmaf(-vi[0], x[0].y, sx);
                float sy = vr[0] * x[0].y;
                sy = fmaf(vi[0], x[0].x, sy);
#pragma unroll
                for (int c = 1; c < 8; ++c) {
                    sx = fmaf(vr[c], x[c].x, sx);
                    sx = fmaf(-vi[c], x[c].y, sx);
                    sy = fmaf(vr[c], x[c].y, sy);
                    sy = fmaf(vi[c], x[c].x, sy);
                }
#pragma unroll
                for (int off = 1; off < TRSV_TPR_H; off <<= 1) {
                    sx += __shfl_xor_sync(0xffffffffu, sx, off);
                    sy += __shfl_xor_sync(0xffffffffu, sy, off);
                }
                if (sub == 0 && q < len) {
                    const int r = FWD ? lo + q : hi - 1 - q;
                    float2 v = y[r];
                    v.x -= sx;
                    v.y -= sy;
                    y[r] = v;
                }
            }
        };
        load(0, g);  // independent of x_d: in flight across the wait
        load(1, g + HG);
        named_sync(TRSV_BAR_X + (d & 1), NT);
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = xs[d & 1][sub * 8 + c];
        apply(0, g);  // covers q < 32 (tile d+2)
        named_arrive(TRSV_BAR_B + (d & 1), NT);
        for (int q0 = g + HG; q0 < len; q0 += 2 * HG) {
            load(0, q0 + HG);
            apply(1, q0);
            if (q0 + HG >= len) break;
            load(1, q0 + 2 * HG);
            apply(0, q0 + HG);
        }
    }
}

// ---------------------------------------------------------------------------
// Block solves with the strips streamed by the copy engine.  Same roles and
// hand-over as trsv_body, but warp 1 is a producer that loads every strip (32
// columns of the Re and Im planes, R rows per stage, in sweep order) into a ring of
// shared-memory stages with tensor-map copies (cp.async.bulk.tensor, completion
// counted on a full[] mbarrier), running ahead of the consumers through both sweeps
// (the factors do not depend on the solution); warps 2.. consume one stage row per
// group of TRSV_TPR lanes with the same fused multiply-adds and the same shuffle
// reduction as trsv_stream, so the result is bit-identical.  A stage holds
// RING_R = (NT - 64) / TRSV_TPR rows (>= 32: the first stage of a strip covers tile
// d+2).  The producer takes no part in the named barriers; every mbarrier wait is
// bounded (on timeout the kernel records an error and carries on, so no thread is
// left waiting at a barrier).
// ---------------------------------------------------------------------------
constexpr int TRSV_BAR_SWEEP = 5;  // solver + consumers between the two sweeps

template <typename T> struct ring_cfg {
    static constexpr int NT = 512;
    static constexpr int R = (NT - 64) / TRSV_TPR;        // 56 rows per stage
    static constexpr int ROWB = 2 * 32 * (int)sizeof(T);  // bytes per stage row (Re | Im)
    static constexpr int S = sizeof(T) == 4 ? 10 : 4;     // stages
    static constexpr int CW = (NT - 64) / 32;             // consumer warps
};

static size_t trsv_ring_smem_bytes(int mp, size_t elem) {
    const size_t s = elem == 4 ? ring_cfg<float>::S : ring_cfg<double>::S;
    const size_t rowb = 2 * 32 * elem;
    return trsv_smem_bytes(mp, elem) + 128 + s * ((size_t)(512 - 64) / TRSV_TPR) * rowb;  // + alignment slack
}

template <typename T>
__device__ __forceinline__ void ring_wait(uint64_t* bar, uint32_t parity, int* err) {
    if (!tc::mbar_wait(bar, parity)) atomicCAS(err, 0, 3);  // recorded; carry on (no hang)
}

// Producer (lane 0 of warp 1): every stage of both sweeps, in the order the consumers
// take them.  A stage is two tensor-map (TMA) boxes of R rows x 32 columns, one per
// plane, landing as [Re rows][Im rows]; forward sweeps load rows lo+q0 .. upward,
// backward sweeps the R rows that end at hi-q0 (the last boxes of a sweep may start
// below row 0 or end past m_p: those rows are filled with zeros and never read).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(tc::smem_u32(bar))
        : "memory");
}

template <typename T>
__device__ __forceinline__ void trsv_ring_producer(int mp, int nt, int k, const CUtensorMap* map, unsigned char* ring,
                                                   uint64_t* full, uint64_t* empty, int* err) {
    using Cf = ring_cfg<T>;
    long g = 0;
    for (int sweep = 0; sweep < 2; ++sweep) {
        const bool fwd = sweep == 0;
        for (int d = 0; d + 2 < nt; ++d) {
            const int col = 32 * (fwd ? d : nt - 1 - d);
            const int lo = fwd ? 32 * (d + 2) : 0;
            const int hi = fwd ? mp : 32 * (nt - 2 - d);
            const int len = hi - lo;
            for (int q0 = 0; q0 < len; q0 += Cf::R, ++g) {
                const int s = (int)(g % Cf::S);
                if (g >= Cf::S) ring_wait<T>(&empty[s], (uint32_t)((g / Cf::S - 1) & 1), err);
                unsigned char* st = ring + (size_t)s * Cf::R * Cf::ROWB;
                const int y0 = fwd ? lo + q0 : hi - q0 - Cf::R;
                tc::mbar_arrive_expect_tx(&full[s], (uint32_t)(Cf::R * Cf::ROWB));
                tma_load_3d(st, map, col, y0, 2 * k, &full[s]);
                tma_load_3d(st + Cf::R * Cf::ROWB / 2, map, col, y0, 2 * k + 1, &full[s]);
            }
        }
    }
}

// Consumers (warps 2..): strip d of one sweep from the ring, stage by stage; g is the
// running stage count shared with the producer's enumeration.
template <typename T, bool FWD>
__device__ __forceinline__ void trsv_ring_stream(int mp, int nt, cplx_t<T>* y, const cplx_t<T> (*xs)[32],
                                                 const unsigned char* ring, uint64_t* full, uint64_t* empty,
                                                 int* err, int bt, long& g) {
    using C = cplx_t<T>;
    using V = typename vec4<T>::type;
    using Cf = ring_cfg<T>;
    const int grp = bt / TRSV_TPR, sub = bt % TRSV_TPR, lane = bt & 31;
    for (int d = 0; d + 2 < nt; ++d) {
        const int lo = FWD ? 32 * (d + 2) : 0;
        const int hi = FWD ? mp : 32 * (nt - 2 - d);
        const int len = hi - lo;
        named_sync(TRSV_BAR_X + (d & 1), Cf::NT - 32);
        const C x0 = xs[d & 1][sub * 4], x1 = xs[d & 1][sub * 4 + 1];
        const C x2 = xs[d & 1][sub * 4 + 2], x3 = xs[d & 1][sub * 4 + 3];
        for (int q0 = 0; q0 < len; q0 += Cf::R, ++g) {
            const int s = (int)(g % Cf::S);
            ring_wait<T>(&full[s], (uint32_t)((g / Cf::S) & 1), err);
            const int q = q0 + grp;
            if (q < len) {  // uniform across a warp: an aligned quartet of groups, len a multiple of 32
                const int br = FWD ? grp : Cf::R - 1 - grp;  // row within the stage's boxes
                const T* pre = reinterpret_cast<const T*>(ring + (size_t)s * Cf::R * Cf::ROWB) + br * 32;
                const T* pim = pre + Cf::R * 32;
                const V vr = *reinterpret_cast<const V*>(pre + sub * 4);
                const V vi = *reinterpret_cast<const V*>(pim + sub * 4);
                T sx = vr.x * x0.x;
                sx = fma(-vi.x, x0.y, sx);
                sx = fma(vr.y, x1.x, sx);
                sx = fma(-vi.y, x1.y, sx);
                sx = fma(vr.z, x2.x, sx);
                sx = fma(-vi.z, x2.y, sx);
                sx = fma(vr.w, x3.x, sx);
                sx = fma(-vi.w, x3.y, sx);
                T sy = vr.x * x0.y;
                sy = fma(vi.x, x0.x, sy);
                sy = fma(vr.y, x1.y, sy);
                sy = fma(vi.y, x1.x, sy);
                sy = fma(vr.z, x2.y, sy);
                sy = fma(vi.z, x2.x, sy);
                sy = fma(vr.w, x3.y, sy);
                sy = fma(vi.w, x3.x, sy);
#pragma unroll
                for (int off = 1; off < TRSV_TPR; off <<= 1) {
                    sx += __shfl_xor_sync(0xffffffffu, sx, off);
                    sy += __shfl_xor_sync(0xffffffffu, sy, off);
                }
                if (sub == 0) {
                    const int r = FWD ? lo + q : hi - 1 - q;
                    C v = y[r];
                    v.x -= sx;
                    v.y -= sy;
                    y[r] = v;
                }
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&empty[s]))
                                        : "memory");
            if (q0 == 0) named_arrive(TRSV_BAR_B + (d & 1), Cf::NT - 32);  // stage 0 covers tile d+2
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(512)
block_trsv_ring_kernel(int mp, const T* __restrict__ fac, const cplx_t<T>* __restrict__ dinv,
                       const T* __restrict__ tinv, cplx_t<T>* __restrict__ rhat, int* __restrict__ err,
                       const __grid_constant__ CUtensorMap fmap) {
    using C = cplx_t<T>;
    using Cf = ring_cfg<T>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int k = blockIdx.x;
    const T* re = fac + (size_t)k * 2 * mp * mp;
    const T* im = re + (size_t)mp * mp;
    const C* dv = dinv + (size_t)k * mp;
    const T* ti = tinv + (size_t)k * (mp / 32) * 4096;
    C* x = rhat + (size_t)k * mp;
    C* y = reinterpret_cast<C*>(smem_raw);       // mp
    T* tiles = reinterpret_cast<T*>(y + mp);     // solver tiles
    // the ring starts at the next 128-byte boundary of the shared window (TMA destinations)
    const uint32_t base = tc::smem_u32(smem_raw) + (uint32_t)trsv_smem_bytes(mp, sizeof(T));
    unsigned char* ring = smem_raw + ((base + 127u) & ~127u) - tc::smem_u32(smem_raw);
    __shared__ C xs[2][32];
    __shared__ C av[32];
    __shared__ __align__(8) uint64_t full[Cf::S], empty[Cf::S];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = mp / 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < Cf::S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], Cf::CW);
        }
        tc::fence_barrier_init();
    }
    for (int i = threadIdx.x; i < mp; i += blockDim.x) y[i] = x[i];
    __syncthreads();
    if (warp == 1) {
        if (lane == 0) trsv_ring_producer<T>(mp, nt, k, &fmap, ring, full, empty, err);
    } else if (warp == 0) {
        trsv_solver<T, true, true, Cf::NT - 32>(mp, nt, re, im, dv, ti, y, xs, tiles, av, lane);
        named_sync(TRSV_BAR_SWEEP, Cf::NT - 32);
        trsv_solver<T, false, true, Cf::NT - 32>(mp, nt, re, im, dv, ti, y, xs, tiles, av, lane);
    } else {
        long g = 0;
        trsv_ring_stream<T, true>(mp, nt, y, xs, ring, full, empty, err, threadIdx.x - 64, g);
        named_sync(TRSV_BAR_SWEEP, Cf::NT - 32);
        trsv_ring_stream<T, false>(mp, nt, y, xs, ring, full, empty, err, threadIdx.x - 64, g);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < mp; i += blockDim.x) x[i] = y[i];
}

template <typename T, bool INV, int NT = TRSV_THREADS, int H = trsv_unroll<T>::value / 2, int LAY = LAY_PLANES>
__device__ __forceinline__ void trsv_body(int mp, const typename fac_store<T, LAY>::elem* __restrict__ re,
                                          const cplx_t<T>* __restrict__ dv,
                                          const T* __restrict__ tinv, cplx_t<T>* __restrict__ x) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* y = reinterpret_cast<C*>(smem_raw);        // mp
    T* tiles = reinterpret_cast<T*>(y + mp);      // solver tiles
    __shared__ C xs[2][32];
    __shared__ C av[32];
    const auto* im = re + (size_t)mp * mp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = mp / 32;
    for (int i = threadIdx.x; i < mp; i += blockDim.x) y[i] = x[i];
    __syncthreads();
    if constexpr (LAY == LAY_STRIPS_BF16) {
        if (warp == 0) trsv_solver<T, true, INV, NT, LAY>(mp, nt, re, im, dv, tinv, y, xs, tiles, av, lane);
        else trsv_stream_bf16<true, NT, H>(mp, nt, re, im, y, xs, threadIdx.x - 32);
        __syncthreads();
        if (warp == 0) trsv_solver<T, false, INV, NT, LAY>(mp, nt, re, im, dv, tinv, y, xs, tiles, av, lane);
        else trsv_stream_bf16<false, NT, H>(mp, nt, re, im, y, xs, threadIdx.x - 32);
    } else {
        if (warp == 0) trsv_solver<T, true, INV, NT, LAY>(mp, nt, re, im, dv, tinv, y, xs, tiles, av, lane);
        else trsv_stream<T, true, NT, H, LAY>(mp, nt, re, im, y, xs, threadIdx.x - 32);
        __syncthreads();
        if (warp == 0) trsv_solver<T, false, INV, NT, LAY>(mp, nt, re, im, dv, tinv, y, xs, tiles, av, lane);
        else trsv_stream<T, false, NT, H, LAY>(mp, nt, re, im, y, xs, threadIdx.x - 32);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < mp; i += blockDim.x) x[i] = y[i];
}

// (The bfloat16 stream loads 16 bytes per lane and plane like the FP32 one, so it keeps
// the shape's rows per register buffer, at most 7: its eight x values per lane take the
// registers of an eighth row; the 640-thread shape takes 3, which its registers allow.)
template <typename T, int V = 0, int LAY = LAY_PLANES>
__global__ void __launch_bounds__(trsv_shape<T, V>::NT)
block_trsv_kernel(int mp, const typename fac_store<T, LAY>::elem* __restrict__ fac,
                  const cplx_t<T>* __restrict__ dinv, const T* __restrict__ tinv, cplx_t<T>* __restrict__ rhat) {
    const int k = blockIdx.x;
    constexpr int HS = trsv_shape<T, V>::H;
    constexpr int H = LAY != LAY_STRIPS_BF16 ? HS : HS > 7 ? 7 : HS == 2 ? 3 : HS;
    trsv_body<T, true, trsv_shape<T, V>::NT, H, LAY>(mp, fac + (size_t)k * 2 * mp * mp,
                                                                  dinv + (size_t)k * mp,
                                                                  tinv + (size_t)k * (mp / 32) * 4096,
                                                                  rhat + (size_t)k * mp);
}

// Batched over the active instances act[0..gridDim.x): block k = blockIdx.y of instance act[blockIdx.x].
// The instance index runs fastest, so the CTAs of one block index are scheduled together:
// when the instances share their factors (many right-hand sides of one operator) they
// stream the same factor planes at the same time and HBM serves them once, through L2.
template <typename T>
__global__ void __launch_bounds__(TRSV_THREADS)
block_trsv_batched(const InstDev* __restrict__ I, const int* __restrict__ act) {
    const InstDev& d = I[act[blockIdx.x]];
    const int k = blockIdx.y;
    if (k >= d.nblk || !d.ctl[0]) return;
    const size_t mp = d.mp;
    const T* fac = (const T*)d.fac + (size_t)k * 2 * mp * mp;
    const cplx_t<T>* dinv = (const cplx_t<T>*)d.dinv + (size_t)k * mp;
    cplx_t<T>* rhat = (cplx_t<T>*)d.rhat + (size_t)k * mp;
    if constexpr (sizeof(T) == 4) {
        if (d.strips) {  // the bfloat16 strip copy, diagonal tiles through their FP32 inverses
            trsv_body<T, true, TRSV_THREADS, trsv_unroll<T>::value / 2, LAY_STRIPS_BF16>(
                d.mp, (const unsigned short*)d.strips + (size_t)k * 2 * mp * mp, dinv,
                (const T*)d.tinv + (size_t)k * (mp / 32) * 4096, rhat);
            return;
        }
    }
    if (d.tinv)  // diagonal tiles solved as products with their inverses
        trsv_body<T, true>(d.mp, fac, dinv, (const T*)d.tinv + (size_t)k * (mp / 32) * 4096, rhat);
    else
        trsv_body<T, false>(d.mp, fac, dinv, nullptr, rhat);
}

// ---------------------------------------------------------------------------
// Block solves for many right-hand sides of one operator (the instances of a batch
// that share their factors): one CTA per Strang block and group of up to TRSV_R
// right-hand sides, so each factor plane is streamed from HBM once per group instead
// of once per right-hand side.  Same roles and hand-over as trsv_body: warp 0 solves
// the 32 x 32 diagonal tiles (inverted tiles, look-ahead of the previous strip) for
// all TRSV_R columns; warps 1.. stream the strips, TRSV_TPR lanes per row, each lane
// four factor columns times TRSV_R right-hand sides, and a reduce-scatter over the
// row's lanes leaves lane `sub` with column sub's sum.  The y vectors live in shared
// memory as [row][column].  Columns without an instance (a short last group) or whose
// instance has left the restart cycle are computed on zeros and not written back.
// ---------------------------------------------------------------------------
constexpr int TRSV_R = 8;           // right-hand sides per CTA (= TRSV_TPR: one column per lane)
constexpr int TRSVM_THREADS = 384;  // warp 0 + 11 streaming warps (44 row groups)
static_assert(TRSV_R == TRSV_TPR, "the reduce-scatter leaves one column per lane of a row group");

__host__ __device__ static size_t trsv_multi_smem_bytes(int mp) {
    return (size_t)mp * TRSV_R * sizeof(float2) + 8 * 32 * trsv_tile<float>::LD * sizeof(float);
}

// One row's strip product for TRSV_R columns: lane `sub` holds factor columns
// 4 sub .. 4 sub + 3 (re v, im w) and, in registers, the strip's solution values
// xr[c][j] of those columns; returns column `sub`'s sum, reduced
// over the TRSV_TPR lanes of the row by a reduce-scatter (each step keeps half of
// the columns and adds the partner's half).
__device__ __forceinline__ float2 multi_row_product(const float4& v, const float4& w, const float2 (&xr)[4][TRSV_R],
                                                    int sub) {
    float pr[TRSV_R], pi[TRSV_R];
#pragma unroll
    for (int j = 0; j < TRSV_R; ++j) {
        const float2 x0 = xr[0][j], x1 = xr[1][j], x2 = xr[2][j], x3 = xr[3][j];
        float a = v.x * x0.x;
        a = fmaf(-w.x, x0.y, a);
        a = fmaf(v.y, x1.x, a);
        a = fmaf(-w.y, x1.y, a);
        a = fmaf(v.z, x2.x, a);
        a = fmaf(-w.z, x2.y, a);
        a = fmaf(v.w, x3.x, a);
        a = fmaf(-w.w, x3.y, a);
        float b = v.x * x0.y;
        b = fmaf(w.x, x0.x, b);
        b = fmaf(v.y, x1.y, b);
        b = fmaf(w.y, x1.x, b);
        b = fmaf(v.z, x2.y, b);
        b = fmaf(w.z, x2.x, b);
        b = fmaf(v.w, x3.y, b);
        b = fmaf(w.w, x3.x, b);
        pr[j] = a;
        pi[j] = b;
    }
    // reduce-scatter over lanes sub = 0..7 (xor 4, 2, 1): after the step with offset h
    // a lane keeps the half of its columns selected by (sub & h)
#pragma unroll
    for (int h = 4, n = TRSV_R; h >= 1; h >>= 1, n >>= 1) {
        const bool upper = (sub & h) != 0;
#pragma unroll
        for (int j = 0; j < n / 2; ++j) {
            const float sr = upper ? pr[j] : pr[j + n / 2], si = upper ? pi[j] : pi[j + n / 2];
            const float rr = __shfl_xor_sync(0xffffffffu, sr, h), ri = __shfl_xor_sync(0xffffffffu, si, h);
            const float kr = upper ? pr[j + n / 2] : pr[j], ki = upper ? pi[j + n / 2] : pi[j];
            pr[j] = kr + rr;
            pi[j] = ki + ri;
        }
    }
    return make_float2(pr[0], pi[0]);
}

template <bool FWD>
__device__ __forceinline__ void trsv_multi_stream(int mp, int nt, const float* re, const float* im,
                                                  float2 (*y)[TRSV_R], const float2 (*xs)[32][TRSV_R], int bt) {
    constexpr int GROUPS = (TRSVM_THREADS - 32) / TRSV_TPR;  // 44, a multiple of 4
    constexpr int H = 2;                                      // rows per register buffer
    constexpr int HG = H * GROUPS;
    static_assert(HG >= 32, "the first batch must cover tile d+2");
    const int g = bt / TRSV_TPR, sub = bt % TRSV_TPR;
    for (int d = 0; d + 2 < nt; ++d) {
        const int col = 32 * (FWD ? d : nt - 1 - d) + sub * 4;
        const int lo = FWD ? 32 * (d + 2) : 0;
        const int hi = FWD ? mp : 32 * (nt - 2 - d);
        const int len = hi - lo;
        float4 ar[2][H], ai[2][H];
        float2 xr[4][TRSV_R];
        auto load = [&](int b, int q0) {
#pragma unroll
            for (int u = 0; u < H; ++u) {
                const int q = q0 + u * GROUPS;
                if (q < len) {
                    const int r = FWD ? lo + q : hi - 1 - q;
                    ar[b][u] = ld4(re + (size_t)r * mp + col);
                    ai[b][u] = ld4(im + (size_t)r * mp + col);
                }
            }
        };
        auto apply = [&](int b, int q0) {
#pragma unroll
            for (int u = 0; u < H; ++u) {
                const int q = q0 + u * GROUPS;
                if (q < len) {  // uniform across a warp (aligned quartets of groups, len a multiple of 32)
                    const float2 s2 = multi_row_product(ar[b][u], ai[b][u], xr, sub);
                    const int r = FWD ? lo + q : hi - 1 - q;
                    float2 v = y[r][sub];
                    v.x -= s2.x;
                    v.y -= s2.y;
                    y[r][sub] = v;
                }
            }
        };
        load(0, g);
        load(1, g + HG);
        named_sync(TRSV_BAR_X + (d & 1), TRSVM_THREADS);
#pragma unroll
        for (int c = 0; c < 4; ++c)  // this lane's four columns of x_d, all right-hand sides
#pragma unroll
            for (int j = 0; j < TRSV_R; ++j) xr[c][j] = xs[d & 1][sub * 4 + c][j];
        apply(0, g);  // covers q < 32 (tile d+2)
        named_arrive(TRSV_BAR_B + (d & 1), TRSVM_THREADS);
        for (int q0 = g + HG; q0 < len; q0 += 2 * HG) {
            load(0, q0 + HG);
            apply(1, q0);
            if (q0 + HG >= len) break;
            load(1, q0 + 2 * HG);
            apply(0, q0 + HG);
        }
    }
}

// Solver warp for TRSV_R columns: lane = row of the diagonal tile; the inverted tiles
// D^-1 (tinv) and the look-ahead tile L(d, d-1) arrive by cp.async two steps ahead.
template <bool FWD>
__device__ __forceinline__ void trsv_multi_solver(int mp, int nt, const float* re, const float* im,
                                                  const float* tinv, float2 (*y)[TRSV_R], float2 (*xs)[32][TRSV_R],
                                                  float* tiles, float2 (*av)[TRSV_R], int lane) {
    constexpr int LD = trsv_tile<float>::LD, TS = 32 * LD;
    auto tile_of = [&](int d) { return FWD ? d : nt - 1 - d; };
    auto issue = [&](int d) {
        float* b = tiles + (d & 1) * 4 * TS;
        const int j = tile_of(d);
        const float* ti = tinv + (size_t)j * 4096 + (FWD ? 0 : 2048);
        tile_async<float>(b, ti, 32, lane);
        tile_async<float>(b + TS, ti + 1024, 32, lane);
        if (d >= 1) {
            tile_async<float>(b + 2 * TS, re, mp, 32 * j, 32 * tile_of(d - 1), lane);
            tile_async<float>(b + 3 * TS, im, mp, 32 * j, 32 * tile_of(d - 1), lane);
        }
    };
    issue(0);
    cp_async_commit();
    if (nt > 1) issue(1);
    cp_async_commit();
    for (int d = 0; d < nt; ++d) {
        const int r0 = 32 * tile_of(d);
        const float* Dre = tiles + (d & 1) * 4 * TS;
        const float* Dim = Dre + TS;
        const float* Lre = Dre + 2 * TS;
        const float* Lim = Dre + 3 * TS;
        cp_async_wait1();
        __syncwarp();
        if (d >= 2) named_sync(TRSV_BAR_B + (d & 1), TRSVM_THREADS);
        float2 a[TRSV_R];
#pragma unroll
        for (int j = 0; j < TRSV_R; ++j) a[j] = y[r0 + lane][j];
        if (d >= 1) {  // look-ahead: strip d-1 on tile d's rows
            const float2(*xp)[TRSV_R] = xs[(d - 1) & 1];
            for (int c = 0; c < 32; ++c) {
                const float lr = Lre[lane * LD + c], li = Lim[lane * LD + c];
#pragma unroll
                for (int j = 0; j < TRSV_R; ++j) {
                    const float2 x = xp[c][j];
                    a[j].x = fmaf(li, x.y, fmaf(-lr, x.x, a[j].x));
                    a[j].y = fmaf(-li, x.x, fmaf(-lr, x.y, a[j].y));
                }
            }
        }
#pragma unroll
        for (int j = 0; j < TRSV_R; ++j) av[lane][j] = a[j];
        __syncwarp();
        float2 x[TRSV_R];
#pragma unroll
        for (int j = 0; j < TRSV_R; ++j) x[j] = make_float2(0.f, 0.f);
        for (int c = 0; c < 32; ++c) {  // x = D^-1 a
            const float dr = Dre[lane * LD + c], di = Dim[lane * LD + c];
#pragma unroll
            for (int j = 0; j < TRSV_R; ++j) {
                const float2 v = av[c][j];
                x[j].x = fmaf(-di, v.y, fmaf(dr, v.x, x[j].x));
                x[j].y = fmaf(di, v.x, fmaf(dr, v.y, x[j].y));
            }
        }
#pragma unroll
        for (int j = 0; j < TRSV_R; ++j) {
            y[r0 + lane][j] = x[j];
            xs[d & 1][lane][j] = x[j];
        }
        __syncwarp();
        if (d <= nt - 3) named_arrive(TRSV_BAR_X + (d & 1), TRSVM_THREADS);
        if (d + 2 < nt) issue(d + 2);
        cp_async_commit();
    }
}

// grid (ceil(nact / TRSV_R), max_nblk): CTA (x, k) solves block k for the instances
// act[TRSV_R x ..], which all use the factors of instance act[0]'s descriptor.
__global__ void __launch_bounds__(TRSVM_THREADS)
block_trsv_multi_kernel(const InstDev* __restrict__ I, const int* __restrict__ act, int nact) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float2 xs[2][32][TRSV_R];
    __shared__ float2 av[32][TRSV_R];
    const InstDev& d0 = I[act[0]];
    const int k = blockIdx.y;
    if (k >= d0.nblk) return;
    const int mp = d0.mp, nt = mp / 32;
    const float* re = (const float*)d0.fac + (size_t)k * 2 * mp * mp;
    const float* im = re + (size_t)mp * mp;
    const float* tinv = (const float*)d0.tinv + (size_t)k * (mp / 32) * 4096;
    float2(*y)[TRSV_R] = reinterpret_cast<float2(*)[TRSV_R]>(smem_raw);
    float* tiles = reinterpret_cast<float*>(smem_raw + (size_t)mp * TRSV_R * sizeof(float2));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the group's right-hand sides: column j <- instance act[TRSV_R blockIdx.x + j] (if live)
    for (int e = threadIdx.x; e < mp * TRSV_R; e += blockDim.x) {
        const int r = e / TRSV_R, j = e % TRSV_R, a = TRSV_R * blockIdx.x + j;
        float2 v = make_float2(0.f, 0.f);
        if (a < nact) {
            const InstDev& d = I[act[a]];
            if (d.ctl[0]) v = ((const float2*)d.rhat)[(size_t)k * mp + r];
        }
        y[r][j] = v;
    }
    __syncthreads();
    if (warp == 0) trsv_multi_solver<true>(mp, nt, re, im, tinv, y, xs, tiles, av, lane);
    else trsv_multi_stream<true>(mp, nt, re, im, y, xs, threadIdx.x - 32);
    __syncthreads();
    if (warp == 0) trsv_multi_solver<false>(mp, nt, re, im, tinv, y, xs, tiles, av, lane);
    else trsv_multi_stream<false>(mp, nt, re, im, y, xs, threadIdx.x - 32);
    __syncthreads();
    for (int e = threadIdx.x; e < mp * TRSV_R; e += blockDim.x) {
        const int r = e / TRSV_R, j = e % TRSV_R, a = TRSV_R * blockIdx.x + j;
        if (a < nact) {
            const InstDev& d = I[act[a]];
            if (d.ctl[0]) ((float2*)d.rhat)[(size_t)k * mp + r] = y[r][j];
        }
    }
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
        const size_t gsm = (size_t)(P.m + 2) * sizeof(T);
        form_blocks_kernel<T><<<grid, 256, gsm, st>>>(P.m, mp, P.h, P.dxa, P.d_g, P.d_dplus, P.d_dminus, P.d_phi,
                                                      P.d_psi, fac);
        FDE_LAUNCH_CHECK("form_blocks_kernel");
    }
    const size_t panel_smem = (size_t)RC * (NB + 1) * sizeof(C);
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
            lu_panel_kernel<T><<<dim3(2 * nch, nb), RC, panel_smem, st>>>(mp, p, nch, fac);
            FDE_LAUNCH_CHECK("lu_panel_kernel");
        }
        const int nt = (rem + 63) / 64;
        StageTimer t(P, FDE_STAGE_LU_UPDATE);
        lu_update_kernel<T><<<dim3(nt * nt, nb), 256, upd_smem, st>>>(mp, p, nt, fac);
        FDE_LAUNCH_CHECK("lu_update_kernel");
    }
    return FDE_OK;
}

// ---------------------------------------------------------------------------
// Two-level LU for the tensor-core precisions (see lu_tc2.cuh)
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(128)
lu_update_tc2_kernel(int mp, int R0, int nt, int part, float* __restrict__ fac,
                     const unsigned char* __restrict__ apack, const unsigned char* __restrict__ bpack, size_t pa,
                     size_t pb, int* __restrict__ err, unsigned char* __restrict__ bpack_next = nullptr,
                     const unsigned char* __restrict__ apack_old = nullptr,
                     const unsigned char* __restrict__ bpack_old = nullptr) {
    // part 0: all nt^2 tiles; 1: the cross ti = 0 or tj = 0 (2 nt - 1 tiles: the next
    // panel's rows and columns); 2: the interior ti, tj >= 1 ((nt - 1)^2 tiles); 3: the
    // row ti = 0 only (nt tiles; the column below it goes to the row-pair kernel); 4: the
    // row ti = 0 without its first tile (tj >= 1, nt - 1 tiles)
    const int k = blockIdx.y, x = blockIdx.x;
    int ti, tj;
    if (part == 0) {
        ti = x / nt;
        tj = x % nt;
    } else if (part == 3 || part == 4) {
        ti = 0;
        tj = part == 3 ? x : 1 + x;
    } else if (part == 1) {
        ti = x < nt ? 0 : x - nt + 1;
        tj = x < nt ? x : 0;
    } else {
        ti = 1 + x / (nt - 1);
        tj = 1 + x % (nt - 1);
    }
    // the next panel's row block (ti = 0, tj >= 1) is also packed as the next step's B' tile tj - 1
    unsigned char* pkn = bpack_next && ti == 0 && tj >= 1
                             ? bpack_next + (size_t)k * pb + (size_t)(tj - 1) * Tc2<KIND>::B_TILE
                             : nullptr;
    tc2_update_body<KIND>(mp, R0, fac + (size_t)k * 2 * mp * mp, apack + k * pa, bpack + k * pb, err, ti, tj, pkn,
                          apack_old ? apack_old + k * pa : nullptr, bpack_old ? bpack_old + k * pb : nullptr);
}

// Rows ti >= 1 of the trailing update in row pairs, over the columns tj0 .. tj0 + ncol - 1:
// CTA x takes tiles (1 + 2p, tj) and (2 + 2p, tj), p = x / ncol, tj = tj0 + x % ncol.
// The interior is tj0 = 1, ncol = nt - 1; the next panel's column below its diagonal
// block is tj0 = 0, ncol = 1.
template <int KIND>
__global__ void __launch_bounds__(128)
lu_update_tc2p_kernel(int mp, int R0, int nt, int tj0, int ncol, float* __restrict__ fac,
                      const unsigned char* __restrict__ apack, const unsigned char* __restrict__ bpack, size_t pa,
                      size_t pb, int* __restrict__ err, unsigned char* __restrict__ apack_next = nullptr,
                      const unsigned char* __restrict__ apack_old = nullptr,
                      const unsigned char* __restrict__ bpack_old = nullptr) {
    using Cfg = Tc2<KIND>;
    const int k = blockIdx.y, x = blockIdx.x;
    const int p = x / ncol, tj = tj0 + x % ncol;
    const int ti0 = 1 + 2 * p;
    const bool two = ti0 + 1 < nt;
    const unsigned char* ab = apack + (size_t)k * pa;
    // the next panel's column block (tj = 0) is also packed as the next step's A' tiles ti - 1
    unsigned char* an = apack_next && tj == 0 ? apack_next + (size_t)k * pa : nullptr;
    // the previous step's operands (merged update): tile indices one larger
    const unsigned char* abo = apack_old ? apack_old + (size_t)k * pa : nullptr;
    tc2_pair_body<KIND>(mp, R0 + ti0 * T2_BM, R0 + tj * T2_BN, two, fac + (size_t)k * 2 * mp * mp,
                        ab + (size_t)ti0 * Cfg::A_TILE, ab + (size_t)(two ? ti0 + 1 : ti0) * Cfg::A_TILE,
                        bpack + (size_t)k * pb + (size_t)tj * Cfg::B_TILE, err,
                        an ? an + (size_t)(ti0 - 1) * Cfg::A_TILE : nullptr,
                        an && two ? an + (size_t)ti0 * Cfg::A_TILE : nullptr,
                        abo ? abo + (size_t)(ti0 + 1) * Cfg::A_TILE : nullptr,
                        abo ? abo + (size_t)((two ? ti0 + 1 : ti0) + 1) * Cfg::A_TILE : nullptr,
                        bpack_old ? bpack_old + (size_t)k * pb + (size_t)(tj + 1) * Cfg::B_TILE : nullptr);
}

// Interior of the trailing update (ti, tj >= 1), warp-specialized: CTA x takes tiles
// x WQ .. x WQ + WQ - 1 of the (nt - 1)^2 interior tiles of block blockIdx.y.
template <int KIND>
__global__ void __launch_bounds__(W_THREADS)
lu_update_tc2w_kernel(int mp, int R0, int nt, float* __restrict__ fac, const unsigned char* __restrict__ apack,
                      const unsigned char* __restrict__ bpack, size_t pa, size_t pb, int* __restrict__ err) {
    const int k = blockIdx.y, ni = nt - 1;
    const int x0 = blockIdx.x * WQ, nq = min(WQ, ni * ni - x0);
    if (nq <= 0) return;
    tc2w_body<KIND>(mp, R0, ni, x0, nq, fac + (size_t)k * 2 * mp * mp, apack + (size_t)k * pa,
                    bpack + (size_t)k * pb, err);
}

// Trailing-update tiles with the C tiles streamed by tensor-map copies (m_p a multiple
// of 128): front = 0 -> the square ti, tj >= f ((nt - f)^2 tiles); front = 1 -> row 1 and
// column 1 (2 nt - 3 tiles).  CTA x takes tiles x S_WQ .. x S_WQ + S_WQ - 1 of block
// blockIdx.y.  apack_old / bpack_old: the previous step's operands (or NULL).
static __host__ __device__ int tc2s_tiles(int nt, int f, int front) {
    return front ? 2 * nt - 3 : (nt - f) * (nt - f);
}

template <int KIND>
__global__ void __launch_bounds__(S_THREADS, 1)
lu_update_tc2s_kernel(int mp, int R0, int nt, int f, int front, const unsigned char* __restrict__ apack,
                      const unsigned char* __restrict__ bpack, const unsigned char* __restrict__ apack_old,
                      const unsigned char* __restrict__ bpack_old, size_t pa, size_t pb, int* __restrict__ err,
                      const __grid_constant__ CUtensorMap cmap) {
    const int k = blockIdx.y;
    const int x0 = blockIdx.x * S_WQ, nq = min(S_WQ, tc2s_tiles(nt, f, front) - x0);
    if (nq <= 0) return;
    tc2s_body<KIND>(mp, R0, nt, f, front, x0, nq, k, apack + (size_t)k * pa, bpack + (size_t)k * pb,
                    apack_old ? apack_old + (size_t)k * pa : nullptr, bpack_old ? bpack_old + (size_t)k * pb : nullptr,
                    err, &cmap);
}

// Batched, in row pairs over every tile of each active block: grid.x = ceil(ntg / 2) * ntg
// covers the largest block (ntg tiles per dimension); CTA x takes tiles (2p, tj) and
// (2p + 1, tj), p = x / ntg, tj = x % ntg.
template <int KIND>
__global__ void __launch_bounds__(128)
lu_update_tc2p_batched(const BlkDev* __restrict__ B, int R0, int ntg, int* __restrict__ err) {
    using Cfg = Tc2<KIND>;
    const BlkDev& d = B[blockIdx.y];
    if (R0 >= d.mp) return;
    const int nt = (d.mp - R0 + T2_BM - 1) / T2_BM;
    const int p = blockIdx.x / ntg, tj = blockIdx.x % ntg;
    const int ti0 = 2 * p;
    if (ti0 >= nt || tj >= nt) return;
    const bool two = ti0 + 1 < nt;
    tc2_pair_body<KIND>(d.mp, R0 + ti0 * T2_BM, R0 + tj * T2_BN, two, (float*)d.fac,
                        d.apack + (size_t)ti0 * Cfg::A_TILE, d.apack + (size_t)(two ? ti0 + 1 : ti0) * Cfg::A_TILE,
                        d.bpack + (size_t)tj * Cfg::B_TILE, err);
}

static inline int cdiv(int a, int b) { return a > 0 ? (a + b - 1) / b : 0; }

template <int KIND>
static int set_tc_attrs() {
    const size_t panel_smem = (size_t)RC * (NB + 1) * sizeof(float2);
    const size_t upd_smem = (64 * (NB + 1) + NB * 65) * sizeof(float2);
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_panel_range_kernel<float, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)panel_smem));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_panel_range_batched<float, KIND>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_range_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)upd_smem));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_range_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)upd_smem));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_tc2_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Tc2<KIND>::SMEM));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_tc2p_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Tc2p<KIND>::SMEM));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_tc2p_batched<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Tc2p<KIND>::SMEM));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_tc2w_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Tc2w<KIND>::SMEM));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_tc2s_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Tc2s<KIND>::SMEM));
    return FDE_OK;
}

// Packed operand bytes per block (A' tiles then B' tiles) for a block of size mp.
template <int KIND>
static void tc2_pack_sizes(int mp, size_t* pa, size_t* pb) {
    const int ntile = mp > TB ? (mp - TB + T2_BM - 1) / T2_BM : 0;
    *pa = (size_t)ntile * Tc2<KIND>::A_TILE;
    *pb = (size_t)ntile * Tc2<KIND>::B_TILE;
}

// ---------------------------------------------------------------------------
// Tensor-core panel level of the two-level LU (FDE_TF32 / FDE_BF16 / FDE_TF32X3).
// Per outer step o (panel width W = 128, trailing matrix from R0 = o + W):
//   lu_diag128_kernel    L11 U11 = A11 in shared memory; L11^{-1}, U11^{-1} packed
//   lu_pack_panel_kernel A21 -> A' tiles, A12 -> B' tiles
//   lu_panel_tc2_kernel  L21 = A21 U11^{-1}, U12 = L11^{-1} A12 (tcgen05, store mode)
//   lu_pack_panel_kernel L21 -> A' tiles, U12 -> B' tiles
//   lu_update_tc2_kernel A22 -= L21 U12 (tcgen05)
// The triangular panel solves become products with the inverted diagonal
// triangles, so every O(m^2 W) term of the step runs on the tensor cores.
// ---------------------------------------------------------------------------
constexpr int D128_LD = TB + 1;  // shared row pitch in floats (column reads conflict-free)
constexpr int D128_THREADS = 512;
constexpr int DB = 32;           // leaf block of the blocked LU and inversion

// planes [128][129] x 2 | T [2 sides][3 targets][32][33] x 2 | per-warp vectors [8][32] complex | 1/U_cc of a leaf [32]
constexpr int D128_NT = 3;  // inversion targets per side in one round (distance 1: three blocks)
static size_t diag128_smem() {
    return (size_t)(2 * TB * D128_LD + 4 * D128_NT * DB * (DB + 1)) * sizeof(float) +
           (size_t)(8 * DB + DB) * sizeof(float2);
}

// Panel solves of the 128 x 128 diagonal block with the 32 values of one row
// (x U_pp = a, U_pp the leaf's unit-free upper factor, 1/U_cc given) or one column
// (L_pp x = a, L_pp unit lower) in registers; the leaf's factors are read from shared
// memory (broadcast; row pitch D128_LD keeps a warp's rows / columns in distinct banks).
__device__ __noinline__ void panel_row_solve(float* Ar, float* Ai, int row, int P0, const float2* pinv) {
    constexpr int LD = D128_LD;
    float xr[DB], xi[DB];
    const int ri = row * LD + P0;
#pragma unroll
    for (int c = 0; c < DB; ++c) {
        xr[c] = Ar[ri + c];
        xi[c] = Ai[ri + c];
    }
#pragma unroll
    for (int c = 0; c < DB; ++c) {
        const float2 pv = pinv[c];
        const float a = xr[c] * pv.x - xi[c] * pv.y, b = xr[c] * pv.y + xi[c] * pv.x;
        xr[c] = a;
        xi[c] = b;
        const int ci = (P0 + c) * LD + P0;
#pragma unroll
        for (int cc = c + 1; cc < DB; ++cc) {
            const float ur = Ar[ci + cc], ui = Ai[ci + cc];
            xr[cc] -= a * ur - b * ui;
            xi[cc] -= a * ui + b * ur;
        }
    }
#pragma unroll
    for (int c = 0; c < DB; ++c) {
        Ar[ri + c] = xr[c];
        Ai[ri + c] = xi[c];
    }
}

__device__ __noinline__ void panel_col_solve(float* Ar, float* Ai, int col, int P0) {
    constexpr int LD = D128_LD;
    float xr[DB], xi[DB];
#pragma unroll
    for (int c = 0; c < DB; ++c) {
        xr[c] = Ar[(P0 + c) * LD + col];
        xi[c] = Ai[(P0 + c) * LD + col];
    }
#pragma unroll
    for (int c = 0; c < DB; ++c) {
#pragma unroll
        for (int rr = c + 1; rr < DB; ++rr) {
            const float lr = Ar[(P0 + rr) * LD + P0 + c], li = Ai[(P0 + rr) * LD + P0 + c];
            xr[rr] -= lr * xr[c] - li * xi[c];
            xi[rr] -= lr * xi[c] + li * xr[c];
        }
    }
#pragma unroll
    for (int c = 0; c < DB; ++c) {
        Ar[(P0 + c) * LD + col] = xr[c];
        Ai[(P0 + c) * LD + col] = xi[c];
    }
}

// One CTA per Strang block: LU (no pivoting) of the W x W block at (o, o), W = 128
// (or 64 for a last panel), blocked over 32 x 32 leaves in shared memory:
//   leaf LU by four warps; panel solves X U_pp = A (rows) and L_pp X = A (columns)
//   with one thread per row / column and the 32 values in registers; rank-32
//   trailing update with 4 x 4 complex register tiles.
// L\U and 1/U_ii are written back.  With invert (a trailing matrix follows, W = 128)
// both triangles are then inverted in place:
//   phase 0: the eight diagonal 32 x 32 triangles, one warp each, column by column;
//   phase d = 1..3: the blocks at distance d from the diagonal,
//     X_ij = -X_ii sum_{j<=k<i} L_ik X_kj   (L^{-1}, i = j + d),
//     Y_ij = -Y_ii sum_{i<k<=j} U_ik Y_kj   (U^{-1}, j = i + d),
//   with the original L_ik, U_ik read back from the factor just written (L2).
// L^{-1} (unit diagonal, zeros above) is packed as the A' tile and U^{-1} (zeros
// below) as the B' tile of the panel products (layout of lu_tc2.cuh).  With psave
// set, L^{-1} and U^{-1} are also packed as two A' tiles (row i, K' = [Re | Im] of
// row i of the inverse) at psave, for the tensor-core block solves.
template <int KIND>
__device__ __forceinline__ void diag128_body(int mp, int o, float* __restrict__ re, float2* __restrict__ dk,
                                             int* __restrict__ info, unsigned char* __restrict__ pA, bool invert,
                                             unsigned char* __restrict__ psave = nullptr,
                                             void* __restrict__ strips = nullptr, bool strips_bf16 = false) {
    using Cfg = Tc2<KIND>;
    constexpr int LD = D128_LD;
    extern __shared__ __align__(16) float dsm[];
    float* Ar = dsm;
    float* Ai = dsm + TB * LD;
    float* Tr = dsm + 2 * TB * LD;                     // [2][3][32][33]
    float* Ti = Tr + 2 * D128_NT * DB * (DB + 1);      // [2][3][32][33]
    float2* vec = reinterpret_cast<float2*>(Ti + 2 * D128_NT * DB * (DB + 1));  // [8][32]
    float2* pinv = vec + 8 * DB;                                   // [32]
    float* im = re + (size_t)mp * mp;
    const int W = mp - o < TB ? mp - o : TB;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int sh4 = W == TB ? 5 : 4;  // log2(W / 4): float4 columns per row
    {
        // 4-byte asynchronous copies straight into the padded planes, all in flight
        // at once (the row pitch of 129 floats rules out 16-byte copies)
        const int shw = sh4 + 2;
        for (int e = t; e < W * W; e += blockDim.x) {
            const int r = e >> shw, c = e & (W - 1);
            const size_t g = (size_t)(o + r) * mp + o + c;
            cp_async4(Ar + r * LD + c, re + g);
            cp_async4(Ai + r * LD + c, im + g);
        }
        cp_async_commit();
        cp_async_wait_all();
    }
    __syncthreads();
    for (int P0 = 0; P0 < W; P0 += DB) {
        if (warp < 4) {  // leaf LU: lane = row; warp 0 scales column c, warp w updates columns c+1+w, c+5+w, ..
            const int ri = (P0 + lane) * LD + P0;
            for (int c = 0; c < DB; ++c) {
                const int ci = (P0 + c) * LD + P0;
                if (warp == 0) {
                    const float pr = Ar[ci + c], pim = Ai[ci + c];
                    const float den = pr * pr + pim * pim;
                    const bool bad = !(den > 0.f) || !isfinite(den);
                    const float ir = bad ? 0.f : pr / den, ii = bad ? 0.f : -pim / den;
                    if (lane == c) {
                        if (bad) atomicCAS(info, 0, o + P0 + c + 1);
                        pinv[c] = make_float2(ir, ii);
                        dk[o + P0 + c] = make_float2(ir, ii);
                    }
                    if (lane > c) {
                        const float ar = Ar[ri + c], ai = Ai[ri + c];
                        Ar[ri + c] = ar * ir - ai * ii;
                        Ai[ri + c] = ar * ii + ai * ir;
                    }
                }
                named_sync(1, 128);  // multipliers of column c
                if (lane > c) {
                    const float lr = Ar[ri + c], li = Ai[ri + c];
                    for (int cc = c + 1 + warp; cc < DB; cc += 4) {
                        const float ur = Ar[ci + cc], ui = Ai[ci + cc];
                        Ar[ri + cc] -= lr * ur - li * ui;
                        Ai[ri + cc] -= lr * ui + li * ur;
                    }
                }
                named_sync(1, 128);  // step c complete before the next pivot
            }
        }
        __syncthreads();
        const int Q0 = P0 + DB, nrest = W - Q0;
        if (nrest <= 0) break;
        // panel solves with the 32 values of one row (x U_pp = a) or one column
        // (L_pp x = a) in registers (separate functions: their register arrays stay
        // out of the kernel's own allocation)
        if (t < nrest) panel_row_solve(Ar, Ai, Q0 + t, P0, pinv);                     // column panel
        else if (t >= 256 && t - 256 < nrest) panel_col_solve(Ar, Ai, Q0 + t - 256, P0);  // row panel
        __syncthreads();
        // rank-32 trailing update; a task owns rows Q0 + tr + q n4 and columns Q0 + tc + w n4
        const int n4 = nrest / 4;
        for (int task = t; task < n4 * n4; task += blockDim.x) {
            const int tr = task / n4, tc = task % n4;
            float accr[4][4], acci[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int w = 0; w < 4; ++w) accr[q][w] = acci[q][w] = 0.f;
#pragma unroll 4
            for (int k = 0; k < DB; ++k) {
                float ar[4], ai[4], br[4], bi[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ar[q] = Ar[(Q0 + tr + q * n4) * LD + P0 + k];
                    ai[q] = Ai[(Q0 + tr + q * n4) * LD + P0 + k];
                    br[q] = Ar[(P0 + k) * LD + Q0 + tc + q * n4];
                    bi[q] = Ai[(P0 + k) * LD + Q0 + tc + q * n4];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        accr[q][w] += ar[q] * br[w] - ai[q] * bi[w];
                        acci[q][w] += ar[q] * bi[w] + ai[q] * br[w];
                    }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int idx = (Q0 + tr + q * n4) * LD + Q0 + tc + w * n4;
                    Ar[idx] -= accr[q][w];
                    Ai[idx] -= acci[q][w];
                }
        }
        __syncthreads();
    }
#pragma unroll 4
    for (int e = t; e < W * W / 4; e += blockDim.x) {
        const int r = e >> sh4, c = (e & ((1 << sh4) - 1)) * 4;
        const size_t g = (size_t)(o + r) * mp + o + c;
        const float* pr = Ar + r * LD + c;
        const float* pi = Ai + r * LD + c;
        *reinterpret_cast<float4*>(re + g) = make_float4(pr[0], pr[1], pr[2], pr[3]);
        *reinterpret_cast<float4*>(im + g) = make_float4(pi[0], pi[1], pi[2], pi[3]);
        if (strips) {  // the strip-major copy of the final factor
            const size_t gs = fac_at<LAY_STRIPS>(mp, o + r, o + c);
            if (strips_bf16) {
                unsigned short* sb = static_cast<unsigned short*>(strips);
                *reinterpret_cast<uint2*>(sb + gs) = make_uint2(bf16x2_bits(pr[0], pr[1]), bf16x2_bits(pr[2], pr[3]));
                *reinterpret_cast<uint2*>(sb + (size_t)mp * mp + gs) =
                    make_uint2(bf16x2_bits(pi[0], pi[1]), bf16x2_bits(pi[2], pi[3]));
            } else {
                float* sf = static_cast<float*>(strips);
                *reinterpret_cast<float4*>(sf + gs) = make_float4(pr[0], pr[1], pr[2], pr[3]);
                *reinterpret_cast<float4*>(sf + (size_t)mp * mp + gs) = make_float4(pi[0], pi[1], pi[2], pi[3]);
            }
        }
    }
    if (!invert || W != TB) return;
    __syncthreads();  // the factor in HBM is read back below by other threads of this CTA
    // phase 0: diagonal triangles, warps 0-3 invert L_pp (lane = row), 4-7 U_pp (lane = column)
    if (warp < 8) {
        const int P0 = (warp & 3) * DB;
        float2* v = vec + warp * DB;
        if (warp < 4) {
            const int ri = (P0 + lane) * LD + P0;
            for (int j = DB - 1; j >= 0; --j) {
                v[lane] = lane > j ? make_float2(Ar[ri + j], Ai[ri + j]) : make_float2(0.f, 0.f);
                __syncwarp();
                float sr = 0.f, si = 0.f;
                if (lane > j) {
                    sr = v[lane].x;
                    si = v[lane].y;
                    for (int k = j + 1; k < lane; ++k) {
                        const float xr = Ar[ri + k], xi = Ai[ri + k];
                        const float2 x = v[k];
                        sr += xr * x.x - xi * x.y;
                        si += xr * x.y + xi * x.x;
                    }
                }
                __syncwarp();
                if (lane > j) {
                    Ar[ri + j] = -sr;
                    Ai[ri + j] = -si;
                }
                __syncwarp();
            }
        } else {
            for (int j = DB - 1; j >= 0; --j) {
                const int ji = (P0 + j) * LD + P0;
                v[lane] = lane > j ? make_float2(Ar[ji + lane], Ai[ji + lane]) : make_float2(0.f, 0.f);
                const float pr = Ar[ji + j], pim = Ai[ji + j];
                __syncwarp();
                const float den = pr * pr + pim * pim;
                const float dr = den > 0.f ? pr / den : 0.f, di = den > 0.f ? -pim / den : 0.f;
                float nr = dr, ni = di;
                if (lane > j) {
                    float sr = 0.f, si = 0.f;
                    for (int k = j + 1; k <= lane; ++k) {
                        const float2 y = v[k];
                        const float ur = Ar[(P0 + k) * LD + P0 + lane], ui = Ai[(P0 + k) * LD + P0 + lane];
                        sr += y.x * ur - y.y * ui;
                        si += y.x * ui + y.y * ur;
                    }
                    nr = -(dr * sr - di * si);
                    ni = -(dr * si + di * sr);
                }
                __syncwarp();
                if (lane >= j) {
                    Ar[ji + lane] = nr;
                    Ai[ji + lane] = ni;
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    // phases d = 1..3: every target at distance d in one round -- the L-side targets
    // (q + d, q) on threads 0..255, the U-side targets (q, q + d) on threads 256..511,
    // q = 0 .. 3 - d; a thread owns row r and the four columns c + 8u of each target
    {
        constexpr int TS = DB * (DB + 1);
        const bool lower = t < 256;
        const int lt = t & 255, r = lt >> 3, c = lt & 7;
        float* Th_r = Tr + (lower ? 0 : D128_NT * TS);
        float* Th_i = Ti + (lower ? 0 : D128_NT * TS);
        for (int d = 1; d < TB / DB; ++d) {
            const int nq = TB / DB - d;
            float tr[D128_NT][4], tim[D128_NT][4];
#pragma unroll
            for (int q = 0; q < D128_NT; ++q)
#pragma unroll
                for (int u = 0; u < 4; ++u) tr[q][u] = tim[q][u] = 0.f;
            // off-diagonal source blocks (L side kb in (j, i), U side kb in (i, j)): their
            // originals were overwritten by earlier rounds, so each is staged from the
            // factor in L2 into the target's T buffer (free until T is stored)
            for (int kq = 0; kq < d - 1; ++kq) {
#pragma unroll
                for (int q = 0; q < D128_NT; ++q) {
                    if (q >= nq) break;
                    const int i = lower ? d + q : q, j = lower ? q : q + d;
                    const int kb = lower ? j + 1 + kq : i + 1 + kq;
                    for (int e = lt; e < DB * DB; e += 256) {
                        const int rr = e >> 5, cc = e & 31;
                        const size_t g = (size_t)(o + DB * i + rr) * mp + o + DB * kb + cc;
                        Th_r[q * TS + rr * (DB + 1) + cc] = __ldcg(re + g);
                        Th_i[q * TS + rr * (DB + 1) + cc] = __ldcg(im + g);
                    }
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < D128_NT; ++q) {
                    if (q >= nq) break;
                    const int j = lower ? q : q + d;
                    const int kb = lower ? j + 1 + kq : q + 1 + kq;
#pragma unroll 4
                    for (int kk = 0; kk < DB; ++kk) {
                        const float sr = Th_r[q * TS + r * (DB + 1) + kk], si = Th_i[q * TS + r * (DB + 1) + kk];
                        const int zi = (DB * kb + kk) * LD + DB * j + c;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float zr = Ar[zi + 8 * u], zm = Ai[zi + 8 * u];
                            tr[q][u] += sr * zr - si * zm;
                            tim[q][u] += sr * zm + si * zr;
                        }
                    }
                }
                __syncthreads();
            }
            // the diagonal term: the target's own original block (still in place) times
            // the inverted diagonal block of column block j, unit lower (L) / upper (U)
#pragma unroll
            for (int q = 0; q < D128_NT; ++q) {
                if (q >= nq) break;
                const int i = lower ? d + q : q, j = lower ? q : q + d;
                const int srow = (DB * i + r) * LD + DB * j;
#pragma unroll 4
                for (int kk = 0; kk < DB; ++kk) {
                    const float sr = Ar[srow + kk], si = Ai[srow + kk];
                    const int zi = (DB * j + kk) * LD + DB * j + c;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int col = c + 8 * u;
                        float zr = Ar[zi + 8 * u], zm = Ai[zi + 8 * u];
                        if (lower) {
                            if (kk < col) zr = zm = 0.f;
                            else if (kk == col) zr = 1.f, zm = 0.f;
                        } else if (kk > col) {
                            zr = zm = 0.f;
                        }
                        tr[q][u] += sr * zr - si * zm;
                        tim[q][u] += sr * zm + si * zr;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    Th_r[q * TS + r * (DB + 1) + c + 8 * u] = tr[q][u];
                    Th_i[q * TS + r * (DB + 1) + c + 8 * u] = tim[q][u];
                }
            }
            __syncthreads();
            // Z_ij = -Z_ii T: L side unit lower (kk < r, plus T[r]), U side upper (kk >= r)
#pragma unroll
            for (int q = 0; q < D128_NT; ++q) {
                if (q >= nq) break;
                const int i = lower ? d + q : q, j = lower ? q : q + d;
                float orr[4], oii[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    orr[u] = lower ? Th_r[q * TS + r * (DB + 1) + c + 8 * u] : 0.f;
                    oii[u] = lower ? Th_i[q * TS + r * (DB + 1) + c + 8 * u] : 0.f;
                }
                const int zrow = (DB * i + r) * LD + DB * i;
                const int k0 = lower ? 0 : r, k1 = lower ? r : DB;
                for (int kk = k0; kk < k1; ++kk) {
                    const float zr = Ar[zrow + kk], zm = Ai[zrow + kk];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float ar = Th_r[q * TS + kk * (DB + 1) + c + 8 * u];
                        const float ai = Th_i[q * TS + kk * (DB + 1) + c + 8 * u];
                        orr[u] += zr * ar - zm * ai;
                        oii[u] += zr * ai + zm * ar;
                    }
                }
                const int oi = (DB * i + r) * LD + DB * j + c;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    Ar[oi + 8 * u] = -orr[u];
                    Ai[oi + 8 * u] = -oii[u];
                }
            }
            __syncthreads();
        }
    }
    // pack: L^{-1} as A' (row i, K' = [Re | Im] of L^{-1}[i][:]), U^{-1} as B'.
    // Consecutive threads take consecutive rows of one segment column: eight threads
    // fill one 128-byte core-matrix group, and a warp's shared reads hit 32 banks.
    constexpr int EPS = Cfg::PER_CORE;
    constexpr int SEGS = 2 * TB / EPS;  // segments per packed row
    unsigned char* pB = pA + Cfg::A_TILE;
    for (int e = t; e < TB * SEGS; e += blockDim.x) {
        const int i = e % TB, kp0 = (e / TB) * EPS;
        const bool imag = kp0 >= TB;
        float v[EPS];
#pragma unroll
        for (int u = 0; u < EPS; ++u) {
            const int kk = (kp0 + u) & (TB - 1);
            v[u] = kk < i ? (imag ? Ai[i * LD + kk] : Ar[i * LD + kk]) : (kk == i && !imag ? 1.f : 0.f);
        }
        pack2_seg<KIND>(pA, T2_BM, i, kp0, v, false);
    }
    for (int e = t; e < TB * SEGS; e += blockDim.x) {
        const int brow = e % (2 * TB), kp0 = (e / (2 * TB)) * EPS;
        const int j = brow & (TB - 1);
        const bool im_part = brow >= TB;
        // B' row j: Re U^{-1}[k][j]; row TB + j: Im U^{-1}[k][j] (k = K index)
        float v[EPS];
#pragma unroll
        for (int u = 0; u < EPS; ++u) {
            const int kk = kp0 + u;
            v[u] = kk <= j ? (im_part ? Ai[kk * LD + j] : Ar[kk * LD + j]) : 0.f;
        }
        pack2_seg<KIND>(pB, 2 * T2_BN, brow, kp0, v, true);
    }
    if (psave) {
        for (int e = t; e < TB * SEGS; e += blockDim.x) {
            const int i = e % TB, kp0 = (e / TB) * EPS;
            const bool imag = kp0 >= TB;
            float vl[EPS], vu[EPS];
#pragma unroll
            for (int u = 0; u < EPS; ++u) {
                const int kk = (kp0 + u) & (TB - 1);
                const float x = imag ? Ai[i * LD + kk] : Ar[i * LD + kk];
                vl[u] = kk < i ? x : (kk == i && !imag ? 1.f : 0.f);
                vu[u] = kk >= i ? x : 0.f;
            }
            pack2_seg<KIND>(psave, T2_BM, i, kp0, vl, false);
            pack2_seg<KIND>(psave + Cfg::A_TILE, T2_BM, i, kp0, vu, false);
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(D128_THREADS)
lu_diag128_kernel(int mp, int o, float* __restrict__ fac, float2* __restrict__ dinv, int* __restrict__ info,
                  unsigned char* __restrict__ ipack, size_t ipack_stride, int invert,
                  unsigned char* __restrict__ dsave = nullptr, size_t dsave_stride = 0,
                  void* __restrict__ strips = nullptr, int strips_bf16 = 0) {
    const int k = blockIdx.x;
    const size_t soff = (size_t)k * 2 * mp * mp * (strips_bf16 ? 2 : 4);
    diag128_body<KIND>(mp, o, fac + (size_t)k * 2 * mp * mp, dinv + (size_t)k * mp, info + k,
                       ipack ? ipack + (size_t)k * ipack_stride : nullptr, invert != 0,
                       dsave ? dsave + (size_t)k * dsave_stride : nullptr,
                       strips ? static_cast<unsigned char*>(strips) + soff : nullptr, strips_bf16 != 0);
}

// Batched: blocks with m_p > o (a prefix of the table sorted by m_p).
template <int KIND>
__global__ void __launch_bounds__(D128_THREADS) lu_diag128_batched(const BlkDev* __restrict__ B, int o) {
    const BlkDev& d = B[blockIdx.x];
    diag128_body<KIND>(d.mp, o, (float*)d.fac, (float2*)d.dinv, d.info, d.ipack, o + TB < d.mp, nullptr, d.strips,
                       true);
}

// Operand tiles of the current panels: rows R0.. of columns o..o+128 (A21 or L21)
// as A' tiles, rows o..o+128 of columns R0.. (A12 or U12) as B' tiles.  One thread
// per 16-byte segment; A' segments read one contiguous row piece, B' segments one
// column piece (consecutive threads take consecutive columns: coalesced).
template <int KIND>
__device__ __forceinline__ void pack_panel_body(int mp, int o, int R0, const float* __restrict__ re,
                                                unsigned char* __restrict__ apack, unsigned char* __restrict__ bpack) {
    using Cfg = Tc2<KIND>;
    constexpr int EPS = Cfg::PER_CORE;
    constexpr int GPR = TB / EPS;  // segments per plane row of a panel
    const float* im = re + (size_t)mp * mp;
    const int nr = mp - R0;
    const long items = (long)nr * GPR;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * items; e += (long)gridDim.x * blockDim.x) {
        float vr[EPS], vi[EPS];
        if (e < items) {
            const int rl = (int)(e / GPR), g = (int)(e % GPR);
            const size_t off = (size_t)(R0 + rl) * mp + o + g * EPS;
#pragma unroll
            for (int u = 0; u < EPS; u += 4) {
                const float4 a = *reinterpret_cast<const float4*>(re + off + u);
                const float4 b = *reinterpret_cast<const float4*>(im + off + u);
                vr[u] = a.x; vr[u + 1] = a.y; vr[u + 2] = a.z; vr[u + 3] = a.w;
                vi[u] = b.x; vi[u + 1] = b.y; vi[u + 2] = b.z; vi[u + 3] = b.w;
            }
            unsigned char* tile = apack + (size_t)(rl / T2_BM) * Cfg::A_TILE;
            pack2_seg<KIND>(tile, T2_BM, rl % T2_BM, g * EPS, vr, false);
            pack2_seg<KIND>(tile, T2_BM, rl % T2_BM, TB + g * EPS, vi, false);
        } else {
            const long e2 = e - items;
            const int g = (int)(e2 / nr), jl = (int)(e2 % nr);
#pragma unroll
            for (int u = 0; u < EPS; ++u) {
                const size_t off = (size_t)(o + g * EPS + u) * mp + R0 + jl;
                vr[u] = re[off];
                vi[u] = im[off];
            }
            unsigned char* tile = bpack + (size_t)(jl / T2_BN) * Cfg::B_TILE;
            const int jr = jl % T2_BN;
            pack2_seg<KIND>(tile, 2 * T2_BN, jr, g * EPS, vr, true);
            pack2_seg<KIND>(tile, 2 * T2_BN, T2_BN + jr, g * EPS, vi, true);
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(256)
lu_pack_panel_kernel(int mp, int o, int R0, const float* __restrict__ fac, unsigned char* __restrict__ apack,
                     unsigned char* __restrict__ bpack, size_t pa, size_t pb) {
    const int k = blockIdx.y;
    pack_panel_body<KIND>(mp, o, R0, fac + (size_t)k * 2 * mp * mp, apack + (size_t)k * pa, bpack + (size_t)k * pb);
}

template <int KIND>
__global__ void __launch_bounds__(256) lu_pack_panel_batched(const BlkDev* __restrict__ B, int o, int R0) {
    const BlkDev& d = B[blockIdx.y];
    if (R0 >= d.mp) return;
    pack_panel_body<KIND>(d.mp, o, R0, (const float*)d.fac, d.apack, d.bpack);
}

// Panel products in store mode: blockIdx.x < ntr -> L21 tile (rows R0 + 128 x,
// columns o..o+128) = A21 tile x U11^{-1}; otherwise U12 tile (rows o..o+128,
// columns R0 + 128 (x - ntr)) = L11^{-1} A12 tile.
template <int KIND>
__global__ void __launch_bounds__(128)
lu_panel_tc2_kernel(int mp, int o, int R0, int ntr, float* __restrict__ fac, const unsigned char* __restrict__ apack,
                    const unsigned char* __restrict__ bpack, const unsigned char* __restrict__ ipack, size_t pa,
                    size_t pb, size_t pi, int* __restrict__ err, int strips, unsigned short* __restrict__ sbf,
                    const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap smap) {
    using Cfg = Tc2<KIND>;
    const int k = blockIdx.y, x = blockIdx.x;
    float* re = fac + (size_t)k * 2 * mp * mp;
    // strips: 1 FP32 copy through smap, 2 bfloat16 copy at sbf (block k at 2 k m_p^2)
    const CUtensorMap* fm = strips ? &fmap : nullptr;
    const CUtensorMap* sm = strips == 1 ? &smap : nullptr;
    unsigned short* sb = strips == 2 ? sbf + (size_t)k * 2 * mp * mp : nullptr;
    const unsigned char* ip = ipack + (size_t)k * pi;
    // D is packed over the operand tile it was computed from (A21 -> L21, A12 -> U12)
    if (x < ntr) {
        unsigned char* at = const_cast<unsigned char*>(apack) + (size_t)k * pa + (size_t)x * Cfg::A_TILE;
        tc2_tile_body<KIND, true>(mp, R0 + x * T2_BM, o, re, at, ip + Cfg::A_TILE, err, at, 0, nullptr, nullptr, fm,
                                  sm, k, sb);
    } else {
        unsigned char* bt = const_cast<unsigned char*>(bpack) + (size_t)k * pb + (size_t)(x - ntr) * Cfg::B_TILE;
        tc2_tile_body<KIND, true>(mp, o, R0 + (x - ntr) * T2_BN, re, ip, bt, err, bt, 1, nullptr, nullptr, fm, sm, k,
                                  sb);
    }
}

// Batched: grid.x = 2 ntg covers the largest active block (ntg tiles per panel).
template <int KIND>
__global__ void __launch_bounds__(128)
lu_panel_tc2_batched(const BlkDev* __restrict__ B, int o, int R0, int ntg, int* __restrict__ err) {
    using Cfg = Tc2<KIND>;
    const BlkDev& d = B[blockIdx.y];
    if (R0 >= d.mp) return;
    const int nt = (d.mp - R0 + T2_BM - 1) / T2_BM;
    const int x = blockIdx.x;
    float* re = (float*)d.fac;
    if (x < ntg) {
        if (x >= nt) return;
        unsigned char* at = d.apack + (size_t)x * Cfg::A_TILE;
        tc2_tile_body<KIND, true>(d.mp, R0 + x * T2_BM, o, re, at, d.ipack + Cfg::A_TILE, err, at, 0, nullptr, nullptr,
                                  nullptr, nullptr, 0, d.strips);
    } else {
        if (x - ntg >= nt) return;
        unsigned char* bt = d.bpack + (size_t)(x - ntg) * Cfg::B_TILE;
        tc2_tile_body<KIND, true>(d.mp, o, R0 + (x - ntg) * T2_BN, re, d.ipack, bt, err, bt, 1, nullptr, nullptr,
                                  nullptr, nullptr, 0, d.strips);
    }
}

static int ensure_lu_streams(Problem& P) {
    if (P.lu_hi) return FDE_OK;
    int least = 0, greatest = 0;
    FDE_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    FDE_CUDA_TRY(cudaStreamCreateWithPriority(&P.lu_hi, cudaStreamNonBlocking, greatest));
    FDE_CUDA_TRY(cudaStreamCreateWithPriority(&P.lu_lo, cudaStreamNonBlocking, least));
    // the cross tiles one level below the panel chain (the next diagonal kernel gets the SMs
    // first), above the interior updates
    const int mid = greatest < least ? greatest + 1 : greatest;
    FDE_CUDA_TRY(cudaStreamCreateWithPriority(&P.lu_x, cudaStreamNonBlocking, mid));
    for (cudaEvent_t& e : P.lu_ev) FDE_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return FDE_OK;
}

// Two-level tensor-core LU with look-ahead.  The panel chain (diagonal block,
// packing, panel products) and the part of each trailing update that the next
// panel needs (its rows and columns: the cross tiles) run on a high-priority
// stream; the interior of the trailing update runs on a low-priority stream
// alongside the cross tiles and the next panel's chain.  The packed L21 / U12
// operands alternate between two buffers by step parity, so the interior update of
// step o keeps reading its operands while step o + 1 packs its own.  Dependencies:
// the interior of step o waits for the panel products of step o (and, in stream
// order, the interior of step o - 1); the cross tiles of step o wait for the
// interior of step o - 1 (they update tiles it wrote, and pack over the buffer it reads).
template <int KIND>
static int run_lu_tc(Problem& P, cudaStream_t st) {
    using Cfg = Tc2<KIND>;
    float* fac = reinterpret_cast<float*>(P.d_fac);
    float2* dinv = reinterpret_cast<float2*>(P.d_dinv);
    const int mp = P.mp, nb = P.nblk;
    size_t pa, pb;
    tc2_pack_sizes<KIND>(mp, &pa, &pb);
    const size_t pi = (size_t)Cfg::A_TILE + Cfg::B_TILE;  // L11^{-1} (A') and U11^{-1} (B') per block
    // interior update kernel (FDE_TUNE_LU: 0 row pairs, 1 warp-specialized, 2 C streamed by
    // tensor-map copies with the updates of consecutive steps merged (m_p a multiple of 128))
    int interior = tune_lookup(FDE_TUNE_LU, mp, nb, P.precision, nullptr);
    if (interior == 2 && mp % TB != 0) interior = 0;
    const bool merge = interior == 2;
    // operand buffer sets, by step: two alternate; merged updates read two steps' sets
    // while the next two steps pack theirs, so four rotate
    const int nsets = merge ? 4 : 2;
    const size_t need = mp > TB ? (size_t)nb * (nsets * (pa + pb) + pi) : 0;
    if (need > 0 && P.pack_bytes < need) {
        if (P.d_pack) {
            FDE_CUDA_TRY(cudaStreamSynchronize(st));
            dev_free(P.d_pack);
        }
        P.d_pack = nullptr;
        P.pack_bytes = 0;
        int arc = dev_alloc(&P.d_pack, need);
        if (arc) return arc;
        P.pack_bytes = need;
        FDE_CUDA_TRY(cudaMemsetAsync(P.d_pack, 0, need, st));
    }
    unsigned char* base = reinterpret_cast<unsigned char*>(P.d_pack);
    auto apk = [&](int o) { return base ? base + (size_t)((o / TB) % nsets) * nb * (pa + pb) : nullptr; };
    auto bpk = [&](int o) { return base ? apk(o) + (size_t)nb * pa : nullptr; };
    unsigned char* ipack = base ? base + (size_t)nsets * nb * (pa + pb) : nullptr;
    int rc = set_tc_attrs<KIND>();
    if (rc) return rc;
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_diag128_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)diag128_smem()));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_panel_tc2_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Cfg::SMEM_STORE_EPI));
    if ((rc = ensure_lu_streams(P))) return rc;
    cudaStream_t sh = P.lu_hi, sl = P.lu_lo, sx = P.lu_x;
    // inverted diagonal blocks kept for the tensor-core block solves (TF32, whole 128-row strips)
    const int nst = mp / TB;
    const size_t dtile_stride = (size_t)nst * 2 * Cfg::A_TILE;
    unsigned char* dsave = nullptr;
    if (KIND == 0 && P.save_dtile && mp % TB == 0 && mp > TB) {
        const size_t dneed = (size_t)nb * dtile_stride;
        if (P.dtile_bytes < dneed) {
            if (P.d_dtile) {
                FDE_CUDA_TRY(cudaStreamSynchronize(st));
                dev_free(P.d_dtile);
            }
            P.d_dtile = nullptr;
            P.dtile_bytes = 0;
            int arc = dev_alloc(&P.d_dtile, dneed);
            if (arc) return arc;
            P.dtile_bytes = dneed;
        }
        dsave = reinterpret_cast<unsigned char*>(P.d_dtile);
    }
    // the strip-major copy of the factor for the block solves (whole 128-wide panels); without
    // the memory for it the block solves read the row-major planes
    void* strips = nullptr;
    const bool sbf16 = P.strip_storage == FDE_STORAGE_BF16;
    if (mp % TB == 0 && P.want_strips) {
        const size_t sneed = (size_t)nb * 2 * mp * mp * (sbf16 ? 2 : 4);
        if (P.strips_bytes < sneed) {
            ++P.graph_gen;  // captured block solves may hold the old copy's address
            if (P.d_strips) {
                FDE_CUDA_TRY(cudaStreamSynchronize(st));
                dev_free(P.d_strips);
            }
            P.d_strips = nullptr;
            P.strips_bytes = 0;
            if (dev_alloc(&P.d_strips, sneed) == FDE_OK) P.strips_bytes = sneed;
            else set_error(FDE_OK, "");  // not an error: the block solves read the planes
        }
        strips = P.d_strips;
    }
    CUtensorMap cmap{}, smap{};
    if ((merge || strips) && (rc = factor_tensor_map_sw128(fac, mp, nb, &cmap))) return rc;
    if (strips && !sbf16 && (rc = strip_tensor_map_sw128(strips, mp, nb, &smap))) return rc;
    const int smode = strips ? (sbf16 ? 2 : 1) : 0;
    FDE_CUDA_TRY(cudaEventRecord(P.lu_ev[0], st));  // fork after the work already queued on st
    FDE_CUDA_TRY(cudaStreamWaitEvent(sh, P.lu_ev[0], 0));
    FDE_CUDA_TRY(cudaStreamWaitEvent(sl, P.lu_ev[0], 0));
    FDE_CUDA_TRY(cudaStreamWaitEvent(sx, P.lu_ev[0], 0));

    // diagonal block, then (if a trailing matrix follows) packing and panel products
    // after_cross: the panel products wait for the cross tiles of the previous step (on
    // sx), the diagonal block only for its own tile (queued on sh before)
    auto panel = [&](int o, bool after_cross) -> int {
        const int R0 = o + (mp - o < TB ? mp - o : TB);
        const bool more = R0 < mp;
        {
            StageTimer t(P, FDE_STAGE_LU_DIAG, sh);
            lu_diag128_kernel<KIND><<<nb, D128_THREADS, diag128_smem(), sh>>>(
                mp, o, fac, dinv, P.d_info, ipack, pi, (more || dsave) ? 1 : 0,
                dsave ? dsave + (size_t)(o / TB) * 2 * Cfg::A_TILE : nullptr, dtile_stride, strips, sbf16 ? 1 : 0);
            FDE_LAUNCH_CHECK("lu_diag128_kernel");
        }
        if (after_cross) FDE_CUDA_TRY(cudaStreamWaitEvent(sh, P.lu_ev[4], 0));
        if (!more) return FDE_OK;
        const int nt = cdiv(mp - R0, T2_BM);
        const long items = 2L * (mp - R0) * (TB / Cfg::PER_CORE);
        const int pgrid = (int)std::min<long>((items + 255) / 256, 1024);
        if (o == 0) {  // later panels were packed by the previous step's update of their rows and columns
            StageTimer t(P, FDE_STAGE_LU_PACK, sh);
            lu_pack_panel_kernel<KIND><<<dim3(pgrid, nb), 256, 0, sh>>>(mp, o, R0, fac, apk(o), bpk(o), pa, pb);
            FDE_LAUNCH_CHECK("lu_pack_panel_kernel");
        }
        {  // the products also pack L21 / U12 as the update's operand tiles
            StageTimer t(P, FDE_STAGE_LU_PANEL_TC, sh);
            lu_panel_tc2_kernel<KIND><<<dim3(2 * nt, nb), 128, Cfg::SMEM_STORE_EPI, sh>>>(
                mp, o, R0, nt, fac, apk(o), bpk(o), ipack, pa, pb, pi, P.d_err, smode,
                static_cast<unsigned short*>(strips), cmap, smap);
            FDE_LAUNCH_CHECK("lu_panel_tc2_kernel");
        }
        return FDE_OK;
    };
    auto body = [&]() -> int {
        {
            dim3 grid(mp < 64 ? mp : 64, nb);
            StageTimer t(P, FDE_STAGE_FORM, sh);
            const size_t gsm = (size_t)(P.m + 2) * sizeof(float);
            form_blocks_kernel<float><<<grid, 256, gsm, sh>>>(P.m, mp, P.h, P.dxa, P.d_g, P.d_dplus, P.d_dminus,
                                                              P.d_phi, P.d_psi, fac);
            FDE_LAUNCH_CHECK("form_blocks_kernel");
        }
        int r = panel(0, false);
        if (r) return r;
        const int nsteps = mp > TB ? cdiv(mp - TB, TB) : 0;  // outer steps with a trailing matrix
        for (int p = 0; p < nsteps; ++p) {
            const int o = p * TB, R0 = o + TB;
            const int nt = cdiv(mp - R0, T2_BM);
            // merged updates (C streamed): an even step with a successor leaves its interior to the
            // next step, which applies both steps' products (K = 256) in one pass over C; that odd
            // step also brings row and column 1 of its trailing matrix (the panel after next) up to
            // date, so the even step after it needs nothing from the interior update
            const bool a_step = merge && p % 2 == 0 && p + 1 < nsteps;
            const bool b_step = merge && p % 2 == 1;
            const unsigned char* ao = b_step ? apk(o - TB) : nullptr;  // the previous step's operands
            const unsigned char* bo = b_step ? bpk(o - TB) : nullptr;
            // the interior update of step p needs this step's packed L21 / U12 (the panel
            // products just queued on sh), not the cross tiles below: it touches other tiles
            // and reads other operand buffers, so it runs beside them
            FDE_CUDA_TRY(cudaEventRecord(P.lu_ev[1], sh));
            // the cross tiles update tiles the last interior update wrote and pack over a buffer
            // it may read (an even step of a merged pair touches neither)
            if (p > 0 && !a_step) FDE_CUDA_TRY(cudaStreamWaitEvent(sh, P.lu_ev[2], 0));
            const bool next = R0 + TB < mp;
            {  // the next diagonal block (tile 0, 0): all the next diagonal kernel waits for
                StageTimer t(P, FDE_STAGE_LU_TC, sh);
                lu_update_tc2_kernel<KIND><<<dim3(1, nb), 128, Cfg::SMEM, sh>>>(mp, R0, nt, 3, fac, apk(o), bpk(o), pa,
                                                                              pb, P.d_err, nullptr, ao, bo);
                FDE_LAUNCH_CHECK("lu_update_tc2_kernel");
            }
            FDE_CUDA_TRY(cudaEventRecord(P.lu_ev[3], sh));
            FDE_CUDA_TRY(cudaStreamWaitEvent(sx, P.lu_ev[3], 0));
            {  // the rest of the next panel's rows (single tiles) and the column below them (row
               // pairs) beside the next diagonal block; when that panel has a trailing matrix, they
               // are packed as its operand tiles as well
                StageTimer t(P, FDE_STAGE_LU_TC, sx);
                if (nt > 1) {
                    lu_update_tc2_kernel<KIND><<<dim3(nt - 1, nb), 128, Cfg::SMEM, sx>>>(
                        mp, R0, nt, 4, fac, apk(o), bpk(o), pa, pb, P.d_err, next ? bpk(R0) : nullptr, ao, bo);
                    FDE_LAUNCH_CHECK("lu_update_tc2_kernel");
                    lu_update_tc2p_kernel<KIND><<<dim3((nt - 1 + 1) / 2, nb), 128, Tc2p<KIND>::SMEM, sx>>>(
                        mp, R0, nt, 0, 1, fac, apk(o), bpk(o), pa, pb, P.d_err, next ? apk(R0) : nullptr, ao, bo);
                    FDE_LAUNCH_CHECK("lu_update_tc2p_kernel");
                }
                if (b_step && nt > 1) {  // row and column 1, both steps' products
                    lu_update_tc2s_kernel<KIND>
                        <<<dim3(cdiv(tc2s_tiles(nt, 1, 1), S_WQ), nb), S_THREADS, Tc2s<KIND>::SMEM, sx>>>(
                            mp, R0, nt, 1, 1, apk(o), bpk(o), ao, bo, pa, pb, P.d_err, cmap);
                    FDE_LAUNCH_CHECK("lu_update_tc2s_kernel");
                }
            }
            FDE_CUDA_TRY(cudaEventRecord(P.lu_ev[4], sx));
            const int f = b_step ? 2 : 1;  // first row / column of the interior update
            if (!a_step && nt > f) {
                FDE_CUDA_TRY(cudaStreamWaitEvent(sl, P.lu_ev[1], 0));
                StageTimer t(P, FDE_STAGE_LU_TC, sl);
                if (interior == 2) {  // warp-specialized, C through a ring of tensor-map copies
                    lu_update_tc2s_kernel<KIND>
                        <<<dim3(cdiv(tc2s_tiles(nt, f, 0), S_WQ), nb), S_THREADS, Tc2s<KIND>::SMEM, sl>>>(
                            mp, R0, nt, f, 0, apk(o), bpk(o), ao, bo, pa, pb, P.d_err, cmap);
                    FDE_LAUNCH_CHECK("lu_update_tc2s_kernel");
                } else if (interior == 1) {  // warp-specialized, two accumulators, WQ tiles per CTA
                    const int tiles = (nt - 1) * (nt - 1);
                    lu_update_tc2w_kernel<KIND><<<dim3((tiles + WQ - 1) / WQ, nb), W_THREADS, Tc2w<KIND>::SMEM, sl>>>(
                        mp, R0, nt, fac, apk(o), bpk(o), pa, pb, P.d_err);
                    FDE_LAUNCH_CHECK("lu_update_tc2w_kernel");
                } else {  // row pairs
                    lu_update_tc2p_kernel<KIND><<<dim3(((nt - 1 + 1) / 2) * (nt - 1), nb), 128, Tc2p<KIND>::SMEM,
                                                  sl>>>(mp, R0, nt, 1, nt - 1, fac, apk(o), bpk(o), pa, pb, P.d_err);
                    FDE_LAUNCH_CHECK("lu_update_tc2p_kernel");
                }
                FDE_CUDA_TRY(cudaEventRecord(P.lu_ev[2], sl));
            }
            if ((r = panel(R0, true))) return r;
        }
        return FDE_OK;
    };
    rc = body();
    P.strips_ok = rc == FDE_OK && strips != nullptr;
    P.strips_bf16 = sbf16;
    // join: st continues after all three streams
    cudaEventRecord(P.lu_ev[1], sl);
    cudaStreamWaitEvent(st, P.lu_ev[1], 0);
    cudaEventRecord(P.lu_ev[1], sx);
    cudaStreamWaitEvent(st, P.lu_ev[1], 0);
    cudaEventRecord(P.lu_ev[1], sh);
    cudaStreamWaitEvent(st, P.lu_ev[1], 0);
    return rc;
}

// Batched LU over a block table sorted by m_p (descending): blocks still being
// factored form a prefix of the table.  FP32 storage; trailing updates on CUDA
// cores (FDE_FP32, NB = 32 steps) or two-level with tcgen05 (FDE_TF32 / FDE_BF16).
static int run_lu_batched_simt(const BlkDev* d_blk, const std::vector<int>& mps, cudaStream_t st) {
    const int nbt = (int)mps.size();
    const int max_mp = mps[0];
    form_blocks_batched<float><<<dim3(64, nbt), 256, (size_t)(max_mp + 2) * sizeof(float), st>>>(d_blk);
    FDE_LAUNCH_CHECK("form_blocks_batched");
    const size_t panel_smem = (size_t)RC * (NB + 1) * sizeof(float2);
    const size_t upd_smem = (64 * (NB + 1) + NB * 65) * sizeof(float2);
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_panel_batched<float, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)panel_smem));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_update_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)upd_smem));
    for (int p = 0; p * NB < max_mp; ++p) {
        int nd = 0, nu = 0;
        while (nd < nbt && mps[nd] > p * NB) ++nd;
        while (nu < nbt && mps[nu] > (p + 1) * NB) ++nu;
        lu_diag_batched<float><<<nd, 256, 0, st>>>(d_blk, p);
        FDE_LAUNCH_CHECK("lu_diag_batched");
        if (nu == 0) break;
        const int rem = max_mp - (p + 1) * NB;
        const int nch = (rem + RC - 1) / RC;
        lu_panel_batched<float, -1><<<dim3(2 * nch, nu), RC, panel_smem, st>>>(d_blk, p);
        FDE_LAUNCH_CHECK("lu_panel_batched");
        const int ntg = (rem + 63) / 64;
        lu_update_batched<float><<<dim3(ntg * ntg, nu), 256, upd_smem, st>>>(d_blk, p, ntg);
        FDE_LAUNCH_CHECK("lu_update_batched");
    }
    return FDE_OK;
}

template <int KIND>
static int run_lu_batched_tc(const BlkDev* d_blk, const std::vector<int>& mps, int* err, cudaStream_t st) {
    using Cfg = Tc2<KIND>;
    const int nbt = (int)mps.size();
    const int max_mp = mps[0];
    form_blocks_batched<float><<<dim3(64, nbt), 256, (size_t)(max_mp + 2) * sizeof(float), st>>>(d_blk);
    FDE_LAUNCH_CHECK("form_blocks_batched");
    int rc = set_tc_attrs<KIND>();
    if (rc) return rc;
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_diag128_batched<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)diag128_smem()));
    FDE_CUDA_TRY(cudaFuncSetAttribute(lu_panel_tc2_batched<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Cfg::SMEM_STORE_EPI));
    auto active = [&](int lim) {  // blocks with m_p > lim (a prefix of the sorted table)
        int n = 0;
        while (n < nbt && mps[n] > lim) ++n;
        return n;
    };
    for (int o = 0; o < max_mp; o += TB) {
        const int nd = active(o);
        if (nd == 0) break;
        lu_diag128_batched<KIND><<<nd, D128_THREADS, diag128_smem(), st>>>(d_blk, o);
        FDE_LAUNCH_CHECK("lu_diag128_batched");
        const int R0 = o + TB;
        const int nact = active(R0);
        if (nact == 0) continue;
        const int top = mps[0];  // the largest active block bounds the grids
        const int ntg = cdiv(top - R0, T2_BM);
        const long items = 2L * (top - R0) * (TB / Cfg::PER_CORE);
        const int pgrid = (int)std::min<long>((items + 255) / 256, 1024);
        lu_pack_panel_batched<KIND><<<dim3(pgrid, nact), 256, 0, st>>>(d_blk, o, R0);
        FDE_LAUNCH_CHECK("lu_pack_panel_batched");
        lu_panel_tc2_batched<KIND><<<dim3(2 * ntg, nact), 128, Cfg::SMEM_STORE_EPI, st>>>(d_blk, o, R0, ntg, err);
        FDE_LAUNCH_CHECK("lu_panel_tc2_batched");  // also packs L21 / U12
        lu_update_tc2p_batched<KIND><<<dim3(((ntg + 1) / 2) * ntg, nact), 128, Tc2p<KIND>::SMEM, st>>>(d_blk, R0,
                                                                                                     ntg, err);
        FDE_LAUNCH_CHECK("lu_update_tc2p_batched");
    }
    return FDE_OK;
}

int launch_lu_batched(const BlkDev* d_blk, const std::vector<int>& mp_sorted, int precision, int* err,
                      cudaStream_t st) {
    if (mp_sorted.empty()) return FDE_OK;
    if (precision == FDE_TF32) return run_lu_batched_tc<0>(d_blk, mp_sorted, err, st);
    if (precision == FDE_BF16) return run_lu_batched_tc<1>(d_blk, mp_sorted, err, st);
    if (precision == FDE_TF32X3) return run_lu_batched_tc<2>(d_blk, mp_sorted, err, st);
    return run_lu_batched_simt(d_blk, mp_sorted, st);
}

// A' tiles, B' tiles, then the L11^{-1} / U11^{-1} tiles of the panel products.
size_t tc_pack_bytes_per_block(int precision, int mp) {
    size_t pa = 0, pb = 0, pi = 0;
    if (precision == FDE_TF32) tc2_pack_sizes<0>(mp, &pa, &pb), pi = Tc2<0>::A_TILE + Tc2<0>::B_TILE;
    else if (precision == FDE_BF16) tc2_pack_sizes<1>(mp, &pa, &pb), pi = Tc2<1>::A_TILE + Tc2<1>::B_TILE;
    else if (precision == FDE_TF32X3) tc2_pack_sizes<2>(mp, &pa, &pb), pi = Tc2<2>::A_TILE + Tc2<2>::B_TILE;
    return mp > TB ? pa + pb + pi : 0;
}

size_t tc_pack_b_bytes_per_block(int precision, int mp) {
    size_t pa = 0, pb = 0;
    if (precision == FDE_TF32) tc2_pack_sizes<0>(mp, &pa, &pb);
    else if (precision == FDE_BF16) tc2_pack_sizes<1>(mp, &pa, &pb);
    else if (precision == FDE_TF32X3) tc2_pack_sizes<2>(mp, &pa, &pb);
    return pb;
}

size_t tc_pack_a_bytes_per_block(int precision, int mp) {
    size_t pa = 0, pb = 0;
    if (precision == FDE_TF32) tc2_pack_sizes<0>(mp, &pa, &pb);
    else if (precision == FDE_BF16) tc2_pack_sizes<1>(mp, &pa, &pb);
    else if (precision == FDE_TF32X3) tc2_pack_sizes<2>(mp, &pa, &pb);
    return pa;
}

int launch_trsv_multi(const InstDev* I, const int* act, int nact, int nblk, int mp, cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    const size_t smem = trsv_multi_smem_bytes(mp);
    if (smem > 227 * 1024) return launch_trsv_batched(I, act, nact, nblk, mp, st);  // m_p > 2560: one per CTA
    FDE_CUDA_TRY(cudaFuncSetAttribute(block_trsv_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    block_trsv_multi_kernel<<<dim3((nact + TRSV_R - 1) / TRSV_R, nblk), TRSVM_THREADS, smem, st>>>(I, act, nact);
    FDE_LAUNCH_CHECK("block_trsv_multi_kernel");
    return FDE_OK;
}

int launch_trsv_batched(const InstDev* I, const int* act, int nact, int max_nblk, int max_mp, cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    const size_t smem = trsv_smem_bytes(max_mp, sizeof(float));
    FDE_CUDA_TRY(cudaFuncSetAttribute(block_trsv_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    block_trsv_batched<float><<<dim3(nact, max_nblk), TRSV_THREADS, smem, st>>>(I, act);
    FDE_LAUNCH_CHECK("block_trsv_batched");
    return FDE_OK;
}

// Inverses of the 32 x 32 diagonal tiles of every block's factors, for the block
// solves: warp 0 inverts the unit lower tile of L, warp 1 the upper tile of U (its
// diagonal included), both in place column by column / row by row from the last,
//   L^-1[i][j] = -(L[i][j] + sum_{j<k<i} L^-1[i][k] L[k][j])          (i > j)
//   U^-1[j][c] = -(1/U[j][j]) sum_{j<k<=c} U[j][k] U^-1[k][c]         (c > j).
// Output per block and tile: [L^-1 re, L^-1 im, U^-1 re, U^-1 im][32][32], with the
// zeros and the unit (L) / inverted (U) diagonal written out.
template <typename T>
__global__ void __launch_bounds__(64) tile_inverse_kernel(int mp, const T* __restrict__ fac, T* __restrict__ tinv) {
    using C = cplx_t<T>;
    __shared__ C tl[2][32][33];
    __shared__ C vb[2][32];
    const int k = blockIdx.y, t = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T* re = fac + (size_t)k * 2 * mp * mp;
    const T* im = re + (size_t)mp * mp;
    const int r0 = 32 * t;
    C (*A)[33] = tl[warp];
    C* v = vb[warp];
    for (int r = 0; r < 32; ++r) {
        const size_t g = (size_t)(r0 + r) * mp + r0 + lane;
        A[r][lane] = mk(re[g], im[g]);
    }
    __syncwarp();
    if (warp == 0) {  // lane = row
        for (int j = 31; j >= 0; --j) {
            v[lane] = lane > j ? A[lane][j] : mk(T(0), T(0));
            __syncwarp();
            C sum = mk(T(0), T(0));
            if (lane > j) {
                sum = v[lane];
                for (int q = j + 1; q < lane; ++q) sum = cadd(sum, cmul(A[lane][q], v[q]));
            }
            __syncwarp();
            if (lane > j) A[lane][j] = mk(-sum.x, -sum.y);
            __syncwarp();
        }
    } else {  // lane = column
        for (int j = 31; j >= 0; --j) {
            v[lane] = lane > j ? A[j][lane] : mk(T(0), T(0));
            const C piv = A[j][j];
            __syncwarp();
            const T den = piv.x * piv.x + piv.y * piv.y;
            const C dj = den > T(0) ? mk(piv.x / den, -piv.y / den) : mk(T(0), T(0));
            C nv = dj;
            if (lane > j) {
                C sum = mk(T(0), T(0));
                for (int q = j + 1; q <= lane; ++q) sum = cadd(sum, cmul(v[q], A[q][lane]));
                nv = cmul(dj, sum);
                nv = mk(-nv.x, -nv.y);
            }
            __syncwarp();
            if (lane >= j) A[j][lane] = nv;
            __syncwarp();
        }
    }
    T* out = tinv + ((size_t)k * (mp / 32) + t) * 4096 + warp * 2048;
    for (int r = 0; r < 32; ++r) {
        C e = A[r][lane];
        if (warp == 0) {
            if (lane > r) e = mk(T(0), T(0));
            else if (lane == r) e = mk(T(1), T(0));
        } else if (lane < r) {
            e = mk(T(0), T(0));
        }
        out[r * 32 + lane] = e.x;
        out[1024 + r * 32 + lane] = e.y;
    }
}

static int launch_tile_inverse(Problem& P, int prec, cudaStream_t st) {
    const size_t esz = prec == FDE_FP64 ? sizeof(double) : sizeof(float);
    const size_t bytes = (size_t)P.nblk * (P.mp / 32) * 4096 * esz;
    if (P.tinv_bytes < bytes) {
        if (P.d_tinv) {
            FDE_CUDA_TRY(cudaStreamSynchronize(st));
            dev_free(P.d_tinv);
        }
        P.d_tinv = nullptr;
        P.tinv_bytes = 0;
        int arc = dev_alloc(&P.d_tinv, bytes);
        if (arc) return arc;
        P.tinv_bytes = bytes;
    }
    StageTimer t(P, FDE_STAGE_LU_DIAG);
    const dim3 grid(P.mp / 32, P.nblk);
    if (prec == FDE_FP64)
        tile_inverse_kernel<double><<<grid, 64, 0, st>>>(P.mp, (const double*)P.d_fac, (double*)P.d_tinv);
    else
        tile_inverse_kernel<float><<<grid, 64, 0, st>>>(P.mp, (const float*)P.d_fac, (float*)P.d_tinv);
    FDE_LAUNCH_CHECK("tile_inverse_kernel");
    return FDE_OK;
}

int launch_tile_inverse_fp32(Problem& P, cudaStream_t st) { return launch_tile_inverse(P, FDE_FP32, st); }

int launch_block_lu(Problem& P, int prec, cudaStream_t st) {
    int rc;
    const bool was_ok = P.strips_ok, was_bf16 = P.strips_bf16;
    P.strips_ok = false;  // set by the tensor-core LU once it has written the strip-major copy
    if (prec == FDE_FP64) rc = run_lu<double>(P, st);
    else if (prec == FDE_TF32) rc = run_lu_tc<0>(P, st);
    else if (prec == FDE_BF16) rc = run_lu_tc<1>(P, st);
    else if (prec == FDE_TF32X3) rc = run_lu_tc<2>(P, st);
    else rc = run_lu<float>(P, st);
    // the captured block solves name the layout they read: a change of it retires them
    // (a factorisation that keeps the layout keeps the graphs)
    if (P.strips_ok != was_ok || (P.strips_ok && P.strips_bf16 != was_bf16)) ++P.graph_gen;
    if (rc) return rc;
    return launch_tile_inverse(P, prec, st);
}

template <typename T, int V>
static int launch_trsv_shape(const Problem& P, void* rhat, cudaStream_t st) {
    const size_t smem = trsv_smem_bytes(P.mp, sizeof(T));
    // the strip-major copy of the factor (FP32 or bfloat16), where the tensor-core LU wrote one
    const bool strips = sizeof(T) == 4 && P.strips_ok && P.d_strips;
    if constexpr (sizeof(T) == 4) {
        if (strips && P.strips_bf16) {
            auto kern = block_trsv_kernel<T, V, LAY_STRIPS_BF16>;
            FDE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<P.nblk, trsv_shape<T, V>::NT, smem, st>>>(P.mp, (const unsigned short*)P.d_strips,
                                                              (const cplx_t<T>*)P.d_dinv, (const T*)P.d_tinv,
                                                              (cplx_t<T>*)rhat);
            FDE_LAUNCH_CHECK("block_trsv_kernel");
            return FDE_OK;
        }
    }
    {
        constexpr int LS = sizeof(T) == 4 ? LAY_STRIPS : LAY_PLANES;  // FP64 factors have no copy
        auto kern = strips ? block_trsv_kernel<T, V, LS> : block_trsv_kernel<T, V, LAY_PLANES>;
        FDE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<P.nblk, trsv_shape<T, V>::NT, smem, st>>>(P.mp, (const T*)(strips ? P.d_strips : P.d_fac),
                                                          (const cplx_t<T>*)P.d_dinv, (const T*)P.d_tinv,
                                                          (cplx_t<T>*)rhat);
    }
    FDE_LAUNCH_CHECK("block_trsv_kernel");
    return FDE_OK;
}

constexpr size_t TRSV_SMEM_MAX = 227 * 1024;  // dynamic shared memory of one CTA

// Tensor map of the factor planes as a 3-D array [2 nblk planes][m_p rows][m_p columns],
// boxes of R rows x 32 columns of one plane (made once per factor buffer).
template <typename T>
static int trsv_tensor_map(const Problem& P, CUtensorMap* map) {
    using Fn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                            const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                            CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Fn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        FDE_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) return set_error(FDE_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        encode = reinterpret_cast<Fn>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)P.mp, (cuuint64_t)P.mp, (cuuint64_t)2 * P.nblk};
    const cuuint64_t strides[2] = {(cuuint64_t)P.mp * sizeof(T), (cuuint64_t)P.mp * P.mp * sizeof(T)};
    const cuuint32_t box[3] = {32, (cuuint32_t)ring_cfg<T>::R, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                              3, P.d_fac, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FDE_ERR_CUDA, "cuTensorMapEncodeTiled failed for the factor planes");
    return FDE_OK;
}

template <typename T>
static int launch_trsv_ring(const Problem& P, void* rhat, cudaStream_t st) {
    const size_t smem = trsv_ring_smem_bytes(P.mp, sizeof(T));
    if (smem > TRSV_SMEM_MAX) return launch_trsv_shape<T, 0>(P, rhat, st);  // the ring does not fit: default
    CUtensorMap map;
    int rc = trsv_tensor_map<T>(P, &map);
    if (rc) return rc;
    auto kern = block_trsv_ring_kernel<T>;
    FDE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<P.nblk, ring_cfg<T>::NT, smem, st>>>(P.mp, (const T*)P.d_fac, (const cplx_t<T>*)P.d_dinv,
                                                 (const T*)P.d_tinv, (cplx_t<T>*)rhat, P.d_err, map);
    FDE_LAUNCH_CHECK("block_trsv_ring_kernel");
    return FDE_OK;
}

// The tuning key of the block solves: the storage of the factors they read (FP64,
// FP32, or FDE_BF16 for the bfloat16 strip copy).
static int trsv_key(const Problem& P) {
    if (P.precision == FDE_FP64) return FDE_FP64;
    return P.strips_ok && P.d_strips && P.strips_bf16 ? FDE_BF16 : FDE_FP32;
}

int launch_block_trsv_variant(const Problem& P, void* rhat, int variant, cudaStream_t st) {
    // the ring has no form for the bfloat16 copy: there the register shape 0 stands in for it
    if (variant == 3 && trsv_key(P) == FDE_BF16) variant = 0;
    if (variant == 3) {  // strips streamed through a shared-memory ring by bulk copies
        if (P.precision == FDE_FP64) return launch_trsv_ring<double>(P, rhat, st);
        return launch_trsv_ring<float>(P, rhat, st);
    }
    if (P.precision == FDE_FP64) {
        if (variant == 1) return launch_trsv_shape<double, 1>(P, rhat, st);
        if (variant == 2) return launch_trsv_shape<double, 2>(P, rhat, st);
        return launch_trsv_shape<double, 0>(P, rhat, st);
    }
    if (variant == 1) return launch_trsv_shape<float, 1>(P, rhat, st);
    if (variant == 2) return launch_trsv_shape<float, 2>(P, rhat, st);
    return launch_trsv_shape<float, 0>(P, rhat, st);
}

int launch_block_trsv(const Problem& P, void* rhat, cudaStream_t st) {
    return launch_block_trsv_variant(P, rhat, tune_lookup(FDE_TUNE_TRSV, P.mp, P.nblk, trsv_key(P), nullptr), st);
}

namespace {
struct TrsvTuneCtx {
    const Problem* P;
    void* rhat;
};
int trsv_trial(void* ctx, int v, cudaStream_t st) {
    const TrsvTuneCtx& c = *static_cast<const TrsvTuneCtx*>(ctx);
    return launch_block_trsv_variant(*c.P, c.rhat, v, st);
}
}  // namespace

// Measure the block-solve shapes for this problem's factors, on its frequency-side
// vector (zeroed first: the solves run in place and their timing does not depend on
// the data), unless the table already has the shape or a variant is forced.
int autotune_trsv(Problem& P) {
    const int prec = trsv_key(P);
    bool need = false;
    tune_lookup(FDE_TUNE_TRSV, P.mp, P.nblk, prec, &need);
    if (!need) return FDE_OK;
    const size_t esz = P.precision == FDE_FP64 ? sizeof(double) : sizeof(float);
    FDE_CUDA_TRY(cudaMemsetAsync(P.d_rhat, 0, (size_t)P.nblk * P.mp * 2 * esz, P.stream));
    TrsvTuneCtx ctx{&P, P.d_rhat};
    int best = 0;
    float ms[TUNE_MAX_VARIANTS] = {};
    // on the bfloat16 copy the three register shapes (the ring reads the FP32 planes)
    const int rc = tune_measure(FDE_TUNE_TRSV, P.stream, trsv_trial, &ctx, &best, ms,
                                tune_default_variant(FDE_TUNE_TRSV, prec), prec == FDE_BF16 ? 3 : 0);
    if (rc) return rc;
    tune_store(FDE_TUNE_TRSV, P.mp, P.nblk, prec, best, ms);
    return FDE_OK;
}

}  // namespace fde
