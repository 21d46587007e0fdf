// Trailing update A22 -= L21 U12 of the blocked Strang-block LU on the tcgen05
// tensor cores (TF32 or BF16 inputs, FP32 accumulation in TMEM).
//
// Complex product as one real GEMM with K' = 2 NB and N' = 2 x 128:
//   A' = [Re L21 | Im L21]                     (128 rows x K')
//   B' = [[Re U12 ; -Im U12] | [Im U12 ; Re U12]]  (K' x 256: Re outputs | Im outputs)
//   D  = A' B'  ->  D[:, 0:128] = Re(L21 U12),  D[:, 128:256] = Im(L21 U12).
// The panel kernel writes A' and B' already packed in the canonical no-swizzle
// K-major core-matrix layout (8 rows x 16 bytes per core matrix, LBO = 128 bytes
// along K, SBO = (K' bytes / 16) x 128 bytes between 8-row groups), so each
// operand tile arrives in shared memory with one bulk copy.
#pragma once

#include <cuda_bf16.h>

#include "tc_ptx.cuh"

namespace fde {

constexpr int TC_BM = 128;          // output rows per CTA (MMA M)
constexpr int TC_BN = 128;          // complex output columns per CTA (MMA N = 256 real)
constexpr int TC_KP = 64;           // K' = 2 NB real columns of the packed operands
constexpr int TC_TMEM_COLS = 256;

template <int KIND>  // 0: TF32, 1: BF16
struct TcCfg {
    static constexpr int ESZ = KIND == 0 ? 4 : 2;
    static constexpr int PER_CORE = 16 / ESZ;               // elements of one core-matrix row
    static constexpr int KCORES = TC_KP / PER_CORE;          // core matrices along K'
    static constexpr int SBO = KCORES * 128;                 // bytes between 8-row groups
    static constexpr int A_BYTES = (TC_BM / 8) * SBO;        // 128 rows
    static constexpr int B_BYTES = (2 * TC_BN / 8) * SBO;    // 256 rows
    static constexpr int KSTEP = KIND == 0 ? 8 : 16;         // K per MMA instruction
    static constexpr int NSTEP = TC_KP / KSTEP;
    static constexpr uint32_t IDESC = tc::instr_desc(KIND == 0 ? 2u : 1u, TC_BM, 2 * TC_BN);
};

// Byte offset of element (row, kp) inside a packed operand tile.
template <int KIND>
__device__ __forceinline__ uint32_t pack_off(int row, int kp) {
    using C = TcCfg<KIND>;
    return (uint32_t)((row >> 3) * C::SBO + (kp / C::PER_CORE) * 128 + (row & 7) * 16 + (kp % C::PER_CORE) * C::ESZ);
}

template <int KIND>
__device__ __forceinline__ void pack_store(unsigned char* tile, int row, int kp, float v) {
    unsigned char* p = tile + pack_off<KIND>(row, kp);
    if (KIND == 0) {
        *reinterpret_cast<float*>(p) = tc::to_tf32(v);
    } else {
        *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
    }
}

// One 128 x 128 complex output tile (ti, tj) of one block; 128 threads.
// re: the block's Re plane (Im follows); apack / bpack: the block's packed
// operand tiles.  err: first failure code of a bounded wait.
template <int KIND>
__device__ __forceinline__ void tc_update_body(int mp, int rest, float* __restrict__ re_plane,
                                               const unsigned char* __restrict__ apack,
                                               const unsigned char* __restrict__ bpack, int* __restrict__ err, int ti,
                                               int tj) {
    using Cfg = TcCfg<KIND>;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + Cfg::A_BYTES;
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int ok_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tc::tmem_alloc(&tmem_base, TC_TMEM_COLS);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar_load, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::fence_barrier_init();
        ok_flag = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;

    if (threadIdx.x == 0) {
        const unsigned char* ga = apack + (size_t)ti * Cfg::A_BYTES;
        const unsigned char* gb = bpack + (size_t)tj * Cfg::B_BYTES;
        tc::mbar_arrive_expect_tx(&bar_load, Cfg::A_BYTES + Cfg::B_BYTES);
        tc::bulk_g2s(sA, ga, Cfg::A_BYTES, &bar_load);
        tc::bulk_g2s(sB, gb, Cfg::B_BYTES, &bar_load);
        if (tc::mbar_wait(&bar_load, 0)) {
            const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
            for (int s = 0; s < Cfg::NSTEP; ++s) {
                // each MMA consumes K = KSTEP elements = 2 core matrices along K'
                const uint64_t ad = tc::smem_desc(a0 + s * 256, 128, Cfg::SBO);
                const uint64_t bd = tc::smem_desc(b0 + s * 256, 128, Cfg::SBO);
                if (KIND == 0)
                    tc::mma_tf32(tbase, ad, bd, Cfg::IDESC, s > 0);
                else
                    tc::mma_f16(tbase, ad, bd, Cfg::IDESC, s > 0);
            }
            tc::mma_commit(&bar_mma);
        } else {
            ok_flag = 0;
            atomicCAS(err, 0, 1);
            tc::mbar_wait(&bar_load, 0);  // let the copies in flight land before the CTA exits
        }
    }
    __syncthreads();
    const bool ok = ok_flag != 0;
    bool mma_done = false;
    if (ok) {
        mma_done = tc::mbar_wait(&bar_mma, 0);
        if (!mma_done && lane == 0) atomicCAS(err, 0, 2);
    }
    tc::fence_after_sync();
    if (ok && mma_done) {
        const int r = rest + ti * TC_BM + warp * 32 + lane;
        const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
        float* re = re_plane;
        float* im = re + (size_t)mp * mp;
#pragma unroll 1
        for (int ch = 0; ch < TC_BN / 16; ++ch) {
            float dr[16], di[16];
            tc::tmem_ld16(lane_addr + ch * 16, dr);
            tc::tmem_ld16(lane_addr + TC_BN + ch * 16, di);
            tc::tmem_ld_wait();
            const int c0 = rest + tj * TC_BN + ch * 16;
            if (r < mp && c0 < mp) {
                float4* pr = reinterpret_cast<float4*>(re + (size_t)r * mp + c0);
                float4* pi = reinterpret_cast<float4*>(im + (size_t)r * mp + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 a = pr[q], b = pi[q];
                    a.x -= dr[4 * q]; a.y -= dr[4 * q + 1]; a.z -= dr[4 * q + 2]; a.w -= dr[4 * q + 3];
                    b.x -= di[4 * q]; b.y -= di[4 * q + 1]; b.z -= di[4 * q + 2]; b.w -= di[4 * q + 3];
                    pr[q] = a;
                    pi[q] = b;
                }
            }
        }
    } else if (ok && !mma_done) {
        tc::mbar_wait(&bar_mma, 0);  // bounded: give in-flight MMAs a chance to retire before dealloc
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, TC_TMEM_COLS);
}

// grid: (ntile * ntile, nblk)
template <int KIND>
__global__ void __launch_bounds__(128)
lu_update_tc_kernel(int mp, int rest, int ntile, int ntile_max, float* __restrict__ fac,
                    const unsigned char* __restrict__ apack, const unsigned char* __restrict__ bpack,
                    int* __restrict__ err) {
    using Cfg = TcCfg<KIND>;
    const int k = blockIdx.y;
    tc_update_body<KIND>(mp, rest, fac + (size_t)k * 2 * mp * mp, apack + (size_t)k * ntile_max * Cfg::A_BYTES,
                         bpack + (size_t)k * ntile_max * Cfg::B_BYTES, err, blockIdx.x / ntile, blockIdx.x % ntile);
}

// Batched over the block table: grid (ntile_grid^2, blocks); tiles outside a
// smaller block's trailing matrix exit at once.
template <int KIND>
__global__ void __launch_bounds__(128)
lu_update_tc_batched(const BlkDev* __restrict__ B, int p, int nb, int ntile_grid, int* __restrict__ err) {
    const BlkDev& d = B[blockIdx.y];
    const int rest = (p + 1) * nb;
    const int rem = d.mp - rest;
    if (rem <= 0) return;
    const int nt = (rem + TC_BM - 1) / TC_BM;
    const int ti = blockIdx.x / ntile_grid, tj = blockIdx.x % ntile_grid;
    if (ti >= nt || tj >= nt) return;
    tc_update_body<KIND>(d.mp, rest, (float*)d.fac, d.apack, d.bpack, err, ti, tj);
}

}  // namespace fde
