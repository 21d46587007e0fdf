// Tensor-core tiles of the two-level blocked LU of the Strang blocks (FDE_TF32,
// FDE_BF16, FDE_TF32X3).  Outer panels of TB = 128 columns; per panel the
// diagonal block is factored and its triangles inverted on CUDA cores, and the
// panel products L21 = A21 U11^{-1}, U12 = L11^{-1} A12 and the rank-128 trailing
// update A22 -= L21 U12 run here, each as complex GEMMs with K' = 2 x 128.
//
// Complex product D = L U of 128 x 128 complex tiles (Re and Im outputs side by
// side in N' = 2 x 128 accumulator columns), operands packed as
//   A' = [Re L | Im L]                         128 rows x K' = 256
//   B' = [Re U | Im U]^T                       256 rows x K = 128
// (B' row j holds Re U[:, j], row 128 + j holds Im U[:, j]).  Per K step the
// product is three MMAs:
//   D[:, 0:256]   += Re L . [Re U | Im U]        (N = 256)
//   D[:, 0:128]   -= Im L . Im U                 (N = 128, A negated by the instruction)
//   D[:, 128:256] += Im L . Re U                 (N = 128)
// so a tile streams 256 KB of operands (A' 128 KB, B' 128 KB) instead of the 384 KB
// of one real GEMM with the B' operand doubled to [[Re U ; -Im U] | [Im U ; Re U]].
// Operands are pre-packed as K-chunks of 64 bytes per row, each chunk in the
// canonical no-swizzle K-major core-matrix layout (8 rows x 16 B core matrices,
// LBO = 128 B along K, SBO = 512 B between 8-row groups), so one bulk copy lands
// a chunk of a tile in shared memory.
//
// The tile kernel (one 128 x 128 complex output tile per CTA, 128 threads):
//   * streams the K steps (A' real and imaginary chunk, B' chunk) through a full /
//     empty mbarrier ring, one thread issuing the MMAs (accumulator in 256 TMEM columns);
//   * update mode (C -= D): prefetches its C rows into L2 at the start, runs a
//     6-stage ring (192 KB in flight), then copies C from L2 into the freed ring,
//     subtracts D (tcgen05.ld) and writes the tile back with bulk copies;
//   * store mode (C = D): a 3-stage ring (two CTAs per SM) and D goes from TMEM
//     straight to HBM; C is never read.
// Every mbarrier wait is bounded; on timeout the CTA records an error, waits
// (bounded) for its own copies and MMAs, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "tc_ptx.cuh"

namespace fde {

constexpr int TB = 128;             // outer panel width (complex K of the tensor-core update)
constexpr int T2_BM = 128;          // output rows per CTA
constexpr int T2_BN = 128;          // complex output columns per CTA (N' = 256)
constexpr int T2_KP = 2 * TB;       // K' = 256 real (one product)
constexpr int T2_STAGES = 3;       // store mode
constexpr int T2_STAGES_UPD = 6;   // update mode
constexpr int T2_STAGES_MAX = 6;
constexpr int T2_CROW = 528;        // bytes per C-tile row in shared memory (512 + 16 pad, 16-B aligned)
constexpr int T2_C_BYTES = T2_BM * T2_CROW;  // one plane

// KIND 0: TF32; 1: BF16; 2: split TF32 -- every operand as hi + lo (both TF32) and
// the product as A_hi B_hi + A_lo B_hi + A_hi B_lo (three K' = 256 segments), which
// restores FP32-level accuracy at three times the tensor work.
template <int KIND>
struct Tc2 {
    static constexpr int ESZ = KIND == 1 ? 2 : 4;
    static constexpr int KP = KIND == 2 ? 3 * T2_KP : T2_KP;  // K' of the packed operands
    static constexpr int PER_CORE = 16 / ESZ;   // elements per core-matrix row
    static constexpr int KCH = 64 / ESZ;        // elements per 64-byte K-chunk
    static constexpr int NCH = KP / KCH;        // chunks per tile
    static constexpr int A_CHUNK = T2_BM * 64;  // bytes
    static constexpr int B_CHUNK = 2 * T2_BN * 64;
    static constexpr int CPS = T2_KP / KCH;   // A' chunks per K' = 256 product segment
    static constexpr int HALF = CPS / 2;      // chunks of its real (or imaginary) K half
    static constexpr int NIT = NCH / 2;       // main-loop steps: A' re + im chunk, B' chunk
    static constexpr int A_TILE = NCH * A_CHUNK;
    static constexpr int B_TILE = NIT * B_CHUNK;  // B' keeps K = 128 per product segment
    static constexpr int STAGE = 2 * A_CHUNK + B_CHUNK;
    static constexpr int SMEM = T2_STAGES_UPD * STAGE;  // the C tile reuses the ring after the main loop
    static_assert(SMEM >= 2 * T2_C_BYTES, "C tile must fit the freed operand ring");
    // Store mode (no C tile): the operand ring only; at most two CTAs (2 x 256 TMEM
    // columns) share an SM.
    static constexpr int SMEM_STORE = T2_STAGES * STAGE;
    static_assert(3 * SMEM_STORE > 227 * 1024, "store mode: at most two CTAs per SM");
    // store mode with whole tiles: two staged 32-column strips of both planes in FP32
    // (64 KB) and, for a bfloat16 strip copy, in bfloat16 (32 KB), at a 1024-byte boundary
    static constexpr int SMEM_STORE_EPI = SMEM_STORE + 1024;
    static_assert(SMEM_STORE_EPI >= 2 * 32768 + 2 * 16384 + 1024, "store mode: the staged strips fit the ring");
    static constexpr int KSTEP = KIND == 1 ? 16 : 8;          // K per MMA = 32 bytes = 2 core matrices
    static constexpr int MMAS = KCH / KSTEP;                  // MMAs per chunk (2)
    static constexpr uint32_t IDESC = tc::instr_desc(KIND == 1 ? 1u : 2u, T2_BM, 2 * T2_BN);
    static constexpr uint32_t IDESC_H = tc::instr_desc(KIND == 1 ? 1u : 2u, T2_BM, T2_BN);
    static constexpr uint32_t IDESC_HN = IDESC_H | tc::IDESC_NEGATE_A;
    // A' chunk holding the real K part of main-loop step it (its imaginary part is HALF
    // chunks further; the step's B' chunk is chunk it)
    __host__ __device__ static constexpr int re_chunk(int it) { return (it / HALF) * CPS + it % HALF; }
};

// The MMAs of one main-loop step into the accumulator at tacc (256 columns): a_re /
// a_im the shared addresses of the A' chunks of the real and imaginary K part, b the
// B' chunk (rows 0..127 Re U, rows 128..255 Im U).  first: the step that starts D.
template <int KIND>
__device__ __forceinline__ void cplx_mma_step(uint32_t tacc, uint32_t a_re, uint32_t a_im, uint32_t b, bool first) {
    using Cfg = Tc2<KIND>;
    constexpr uint32_t B_IM = (T2_BN / 8) * 512;  // row 128 of the B' chunk
#pragma unroll
    for (int j = 0; j < Cfg::MMAS; ++j) {
        const uint64_t ar = tc::smem_desc(a_re + j * 256, 128, 512);
        const uint64_t ai = tc::smem_desc(a_im + j * 256, 128, 512);
        const uint64_t bb = tc::smem_desc(b + j * 256, 128, 512);
        const uint64_t bi = tc::smem_desc(b + B_IM + j * 256, 128, 512);
        const uint32_t acc = (!first || j > 0) ? 1u : 0u;
        if (KIND == 1) {
            tc::mma_f16(tacc, ar, bb, Cfg::IDESC, acc);
            tc::mma_f16(tacc, ai, bi, Cfg::IDESC_HN, 1u);
            tc::mma_f16(tacc + T2_BN, ai, bb, Cfg::IDESC_H, 1u);
        } else {
            tc::mma_tf32(tacc, ar, bb, Cfg::IDESC, acc);
            tc::mma_tf32(tacc, ai, bi, Cfg::IDESC_HN, 1u);
            tc::mma_tf32(tacc + T2_BN, ai, bb, Cfg::IDESC_H, 1u);
        }
    }
}

// Byte offset of element (row, kp) of a packed tile whose chunks hold `rows` rows.
template <int KIND>
__device__ __forceinline__ uint32_t pack2_off(int rows, int row, int kp) {
    using C = Tc2<KIND>;
    return (uint32_t)((kp / C::KCH) * rows * 64 + (row >> 3) * 512 + ((kp % C::KCH) / C::PER_CORE) * 128 +
                      (row & 7) * 16 + (kp % C::PER_CORE) * C::ESZ);
}

template <int KIND>
__device__ __forceinline__ void pack2_raw(unsigned char* tile, int rows, int row, int kp, float v) {
    unsigned char* p = tile + pack2_off<KIND>(rows, row, kp);
    if (KIND == 1)
        *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
    else
        *reinterpret_cast<float*>(p) = tc::to_tf32(v);
}

// Store value v at K' position kp of an A' tile (b_side = false, kp < 256) or a B'
// tile (kp < 128).  Split TF32 repeats each value per product segment (256 K' for A',
// 128 for B').
template <int KIND>
__device__ __forceinline__ void pack2_store(unsigned char* tile, int rows, int row, int kp, float v, bool b_side) {
    if constexpr (KIND == 2) {
        const float hi = tc::to_tf32(v);
        const float lo = tc::to_tf32(v - hi);
        const int seg = b_side ? TB : T2_KP;
        pack2_raw<KIND>(tile, rows, row, kp, hi);
        pack2_raw<KIND>(tile, rows, row, seg + kp, b_side ? hi : lo);
        pack2_raw<KIND>(tile, rows, row, 2 * seg + kp, b_side ? lo : hi);
    } else {
        pack2_raw<KIND>(tile, rows, row, kp, v);
    }
}

// Store the PER_CORE values v[0..PER_CORE) at K' positions kp0 .. kp0 + PER_CORE - 1
// (kp0 a multiple of PER_CORE, < 256 for A', < 128 for B') of one row: one 16-byte
// core-matrix row segment per product segment.
template <int KIND>
__device__ __forceinline__ void pack2_seg(unsigned char* tile, int rows, int row, int kp0, const float* v,
                                          bool b_side) {
    if constexpr (KIND == 1) {
        __align__(16) __nv_bfloat16 hv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) hv[t] = __float2bfloat16_rn(v[t]);
        *reinterpret_cast<uint4*>(tile + pack2_off<KIND>(rows, row, kp0)) = *reinterpret_cast<const uint4*>(hv);
    } else {
        float4 hi = make_float4(tc::to_tf32(v[0]), tc::to_tf32(v[1]), tc::to_tf32(v[2]), tc::to_tf32(v[3]));
        *reinterpret_cast<float4*>(tile + pack2_off<KIND>(rows, row, kp0)) = hi;
        if constexpr (KIND == 2) {
            const float4 lo = make_float4(tc::to_tf32(v[0] - hi.x), tc::to_tf32(v[1] - hi.y),
                                          tc::to_tf32(v[2] - hi.z), tc::to_tf32(v[3] - hi.w));
            const int seg = b_side ? TB : T2_KP;
            *reinterpret_cast<float4*>(tile + pack2_off<KIND>(rows, row, seg + kp0)) = b_side ? hi : lo;
            *reinterpret_cast<float4*>(tile + pack2_off<KIND>(rows, row, 2 * seg + kp0)) = b_side ? lo : hi;
        }
    }
}

// Two floats rounded to bfloat16 (to nearest even), the first in the low half.
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

__device__ __forceinline__ void bulk_s2g(void* dst_gmem, const void* src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(tc::smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_prefetch_l2(const void* gmem, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until the committed bulk stores have read their shared-memory source (all a
// CTA needs before it exits or reuses the buffer; the global writes complete on their own).
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// ... until at most one committed group is still reading its source
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }

// 2-D tensor copies (tensor maps with 128-byte swizzle: row r's 16-byte chunk u of a
// 128-byte box row sits at r * 128 + ((u ^ (r mod 8)) << 4) of a 1024-byte aligned buffer)
__device__ __forceinline__ void tma2d_load(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(tc::smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma2d_store(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(tc::smem_u32(src))
                 : "memory");
}


// Operand tiles of the next outer step packed from an updated C tile staged in shared
// memory (row pitch T2_CROW), one thread per row (A') or column (B'):
//   A' -- tile row r -> A' row r, K' = [Re | Im] of the tile's 128 columns (the next L21 source);
//   B' -- tile column j -> B' rows j (Re part) and T2_BN + j (Im part), K = the tile
//         row (the next U12 source).
template <int KIND>
__device__ __forceinline__ void pack_staged_a(unsigned char* __restrict__ pk, const unsigned char* sCr,
                                              const unsigned char* sCi, int nrows) {
    constexpr int EPS = Tc2<KIND>::PER_CORE;
    const int r = threadIdx.x;
    if (r >= nrows) return;
    const float* cr = reinterpret_cast<const float*>(sCr + r * T2_CROW);
    const float* ci = reinterpret_cast<const float*>(sCi + r * T2_CROW);
#pragma unroll 4
    for (int kp0 = 0; kp0 < TB; kp0 += EPS) {
        float vr[EPS], vi[EPS];
#pragma unroll
        for (int u = 0; u < EPS; ++u) {
            vr[u] = cr[kp0 + u];
            vi[u] = ci[kp0 + u];
        }
        pack2_seg<KIND>(pk, T2_BM, r, kp0, vr, false);
        pack2_seg<KIND>(pk, T2_BM, r, TB + kp0, vi, false);
    }
}

template <int KIND>
__device__ __forceinline__ void pack_staged_b(unsigned char* __restrict__ pk, const unsigned char* sCr,
                                              const unsigned char* sCi, int ncols) {
    constexpr int EPS = Tc2<KIND>::PER_CORE;
    const int j = threadIdx.x;
    if (j >= ncols) return;
#pragma unroll 2
    for (int kp0 = 0; kp0 < TB; kp0 += EPS) {
        float vr[EPS], vi[EPS];
#pragma unroll
        for (int u = 0; u < EPS; ++u) {
            vr[u] = reinterpret_cast<const float*>(sCr + (kp0 + u) * T2_CROW)[j];
            vi[u] = reinterpret_cast<const float*>(sCi + (kp0 + u) * T2_CROW)[j];
        }
        pack2_seg<KIND>(pk, 2 * T2_BN, j, kp0, vr, true);
        pack2_seg<KIND>(pk, 2 * T2_BN, T2_BN + j, kp0, vi, true);
    }
}

// One 128 x 128 complex output tile at (r0, c0) of one block, D = A' B'^T from the
// packed tiles ga (A') and gb (B'):
//   STORE = false: C[r0.., c0..] -= D (C prefetched into L2 at the start, staged
//                  in the freed operand ring after the last MMA);
//   STORE = true:  C[r0.., c0..]  = D (no read of C; D goes from TMEM to HBM).
// Store mode also packs D as an operand tile of the trailing update when pk is set:
// pk_side 0 -- an A' tile (tile rows, K' = [Re | Im] of the 128 columns: L21);
// pk_side 1 -- a B' tile (K' = the tile rows, output rows = its columns: U12).
// The operand tile that D replaces is no longer read once the MMAs are complete.
// Update mode with pk set packs the updated tile as a B' tile of the next outer step
// (a tile of the next panel's row block).
//
// With ga_old / gb_old set (update mode), D is the sum of two rank-128 products: the
// K steps of (ga_old, gb_old) first, then those of (ga, gb) -- the trailing updates of
// two consecutive outer steps applied in one pass over C.
template <int KIND, bool STORE>
__device__ __forceinline__ void tc2_tile_body(int mp, int r0, int c0, float* __restrict__ re_plane,
                                              const unsigned char* __restrict__ ga,
                                              const unsigned char* __restrict__ gb, int* __restrict__ err,
                                              unsigned char* __restrict__ pk = nullptr, int pk_side = 0,
                                              const unsigned char* __restrict__ ga_old = nullptr,
                                              const unsigned char* __restrict__ gb_old = nullptr,
                                              const CUtensorMap* fmap = nullptr, const CUtensorMap* smap = nullptr,
                                              int kblk = 0, unsigned short* __restrict__ sbf = nullptr) {
    using Cfg = Tc2<KIND>;
    const int nsteps = (ga_old ? 2 : 1) * Cfg::NIT;
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int NS = STORE ? T2_STAGES : T2_STAGES_UPD;
    unsigned char* sStage = smem;
    unsigned char* sCr = smem;  // update mode: the C tile, after the last MMA
    unsigned char* sCi = smem + T2_C_BYTES;
    __shared__ __align__(8) uint64_t bar_c, bar_mma, bar_full[T2_STAGES_MAX], bar_empty[T2_STAGES_MAX];
    __shared__ uint32_t tmem_base;
    __shared__ int ok_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nrows = min(T2_BM, mp - r0);
    const int ncols = min(T2_BN, mp - c0);  // multiple of 64 (mp and R0 are)
    const uint32_t row_bytes = (uint32_t)ncols * 4;
    float* gre = re_plane;
    float* gim = re_plane + (size_t)mp * mp;

    if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar_c, 1);
        tc::mbar_init(&bar_mma, 1);
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&bar_full[s], 1);
            tc::mbar_init(&bar_empty[s], 1);
        }
        tc::fence_barrier_init();
        ok_flag = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    if (!STORE) {  // C rows towards L2 while the operands stream
        const int r = threadIdx.x;
        if (r < nrows) {
            bulk_prefetch_l2(gre + (size_t)(r0 + r) * mp + c0, row_bytes);
            bulk_prefetch_l2(gim + (size_t)(r0 + r) * mp + c0, row_bytes);
        }
    }
    if (threadIdx.x == 0) {
        auto load_chunk = [&](int c) {  // main-loop step c: A' re, A' im, B' chunks
            const int s = c % NS;
            const bool old = ga_old && c < Cfg::NIT;
            const unsigned char* a = old ? ga_old : ga;
            const unsigned char* b = old ? gb_old : gb;
            const int cl = old || !ga_old ? c : c - Cfg::NIT;
            const int kc = Cfg::re_chunk(cl);
            unsigned char* sa = sStage + s * Cfg::STAGE;
            tc::mbar_arrive_expect_tx(&bar_full[s], Cfg::STAGE);
            tc::bulk_g2s(sa, a + (size_t)kc * Cfg::A_CHUNK, Cfg::A_CHUNK, &bar_full[s]);
            tc::bulk_g2s(sa + Cfg::A_CHUNK, a + (size_t)(kc + Cfg::HALF) * Cfg::A_CHUNK, Cfg::A_CHUNK, &bar_full[s]);
            tc::bulk_g2s(sa + 2 * Cfg::A_CHUNK, b + (size_t)cl * Cfg::B_CHUNK, Cfg::B_CHUNK, &bar_full[s]);
        };
        for (int c = 0; c < NS - 1 && c < nsteps; ++c) load_chunk(c);
        bool ok = true;
        for (int c = 0; c < nsteps && ok; ++c) {
            const int s = c % NS;
            if (!tc::mbar_wait(&bar_full[s], (c / NS) & 1)) {
                ok = false;
                break;
            }
            const uint32_t a0 = tc::smem_u32(sStage + s * Cfg::STAGE);
            cplx_mma_step<KIND>(tbase, a0, a0 + Cfg::A_CHUNK, a0 + 2 * Cfg::A_CHUNK, c == 0);
            tc::mma_commit(&bar_empty[s]);
            // refill the stage freed by step c-1 with step c + STAGES - 1
            const int nxt = c + NS - 1;
            if (nxt < nsteps) {
                if (c >= 1) {
                    const int sp = (c - 1) % NS;
                    if (!tc::mbar_wait(&bar_empty[sp], ((c - 1) / NS) & 1)) {
                        ok = false;
                        break;
                    }
                }
                load_chunk(nxt);
            }
        }
        // bar_mma tracks every MMA this thread issued, also after a failed wait
        tc::mma_commit(&bar_mma);
        if (!ok) {
            ok_flag = 0;
            atomicCAS(err, 0, 1);
        }
    }
    __syncthreads();
    const bool ok = ok_flag != 0;
    bool mine = false;
    if (ok) {
        mine = tc::mbar_wait(&bar_mma, 0);
        if (!mine && lane == 0) atomicCAS(err, 0, 2);
    }
    bool done = __syncthreads_and(mine) != 0;  // uniform across the CTA
    tc::fence_after_sync();
    bool staged = false;  // update mode: C copies in flight into the ring
    if (!STORE && ok && done) {
        // every MMA has completed, so the operand ring is free for the C tile
        if (threadIdx.x == 0) tc::mbar_arrive_expect_tx(&bar_c, 2u * (uint32_t)nrows * row_bytes);
        __syncthreads();
        const int r = threadIdx.x;
        if (r < nrows) {
            tc::bulk_g2s(sCr + r * T2_CROW, gre + (size_t)(r0 + r) * mp + c0, row_bytes, &bar_c);
            tc::bulk_g2s(sCi + r * T2_CROW, gim + (size_t)(r0 + r) * mp + c0, row_bytes, &bar_c);
        }
        staged = true;
        const bool cok = tc::mbar_wait(&bar_c, 0);
        if (!cok && lane == 0) atomicCAS(err, 0, 2);
        done = __syncthreads_and(cok) != 0;
    }
    if (STORE && ok && done && (smap || sbf)) {
        // D through shared memory: per 32-column strip, both planes staged with the 128-byte
        // swizzle in one of two buffers of the freed ring, then stored by tensor copies to the
        // row-major planes (fmap) and to the strip-major copy (smap), where the strip's 128
        // rows are one contiguous 16 KB range; or, for a bfloat16 copy (sbf: this block's), the
        // strip also staged as bfloat16 rows of 64 bytes and stored by one bulk copy of 8 KB
        // per plane (without fmap -- the blocks of a batch have no common tensor map -- the
        // planes are then written from registers).  Whole tiles only (m_p a multiple of 128).
        const int r = warp * 32 + lane;  // TMEM lane = tile row
        const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
        unsigned char* sbuf = smem + ((1024u - (tc::smem_u32(smem) & 1023u)) & 1023u);
        const int yf = kblk * 2 * mp;                 // block kblk's Re plane in fmap
        const int ys = kblk * 2 * (mp / 32) * mp;     // its first Re strip in smap
#pragma unroll 1
        for (int sx = 0; sx < T2_BN / 32; ++sx) {
            unsigned char* bre = sbuf + (sx & 1) * 32768;
            unsigned char* bim = bre + 16384;
            unsigned char* hre = sbuf + 65536 + (sx & 1) * 16384;  // bfloat16 rows of 64 bytes
            unsigned char* him = hre + 8192;
            if (sx >= 2) {  // the stores of strip sx - 2 have read this buffer
                if (threadIdx.x == 0) bulk_wait_read_1();
                __syncthreads();
            }
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const int ch = 2 * sx + h;
                float dr[16], di[16];
                tc::tmem_ld16(lane_addr + ch * 16, dr);
                tc::tmem_ld16(lane_addr + T2_BN + ch * 16, di);
                tc::tmem_ld_wait();
                if (fmap) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int off = r * 128 + (((4 * h + q) ^ (r & 7)) << 4);
                        *reinterpret_cast<float4*>(bre + off) =
                            make_float4(dr[4 * q], dr[4 * q + 1], dr[4 * q + 2], dr[4 * q + 3]);
                        *reinterpret_cast<float4*>(bim + off) =
                            make_float4(di[4 * q], di[4 * q + 1], di[4 * q + 2], di[4 * q + 3]);
                    }
                } else {
                    float* pr = gre + (size_t)(r0 + r) * mp + c0 + ch * 16;
                    float* pi = gim + (size_t)(r0 + r) * mp + c0 + ch * 16;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        reinterpret_cast<float4*>(pr)[q] =
                            make_float4(dr[4 * q], dr[4 * q + 1], dr[4 * q + 2], dr[4 * q + 3]);
                        reinterpret_cast<float4*>(pi)[q] =
                            make_float4(di[4 * q], di[4 * q + 1], di[4 * q + 2], di[4 * q + 3]);
                    }
                }
                if (sbf) {  // columns 16 h .. 16 h + 15 of row r: 32 bytes per plane
                    uint32_t wr[8], wi[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        wr[e] = bf16x2_bits(dr[2 * e], dr[2 * e + 1]);
                        wi[e] = bf16x2_bits(di[2 * e], di[2 * e + 1]);
                    }
                    uint4* hr = reinterpret_cast<uint4*>(hre + r * 64 + h * 32);
                    uint4* hi = reinterpret_cast<uint4*>(him + r * 64 + h * 32);
                    hr[0] = make_uint4(wr[0], wr[1], wr[2], wr[3]);
                    hr[1] = make_uint4(wr[4], wr[5], wr[6], wr[7]);
                    hi[0] = make_uint4(wi[0], wi[1], wi[2], wi[3]);
                    hi[1] = make_uint4(wi[4], wi[5], wi[6], wi[7]);
                }
                if (pk && pk_side == 0) {  // L21 row r: K' = column (Re), TB + column (Im)
                    constexpr int EPS = Cfg::PER_CORE;
#pragma unroll
                    for (int u = 0; u < 16 / EPS; ++u) {
                        pack2_seg<KIND>(pk, T2_BM, r, ch * 16 + u * EPS, dr + u * EPS, false);
                        pack2_seg<KIND>(pk, T2_BM, r, TB + ch * 16 + u * EPS, di + u * EPS, false);
                    }
                } else if (pk) {  // U12 row r = K index: B' rows j (Re) and T2_BN + j (Im)
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int j = ch * 16 + e;
                        pack2_store<KIND>(pk, 2 * T2_BN, j, r, dr[e], true);
                        pack2_store<KIND>(pk, 2 * T2_BN, T2_BN + j, r, di[e], true);
                    }
                }
            }
            fence_async_shared();
            __syncthreads();
            if (threadIdx.x == 0) {
                const int col = c0 + 32 * sx;
                if (fmap) {
                    tma2d_store(fmap, col, yf + r0, bre);
                    tma2d_store(fmap, col, yf + mp + r0, bim);
                }
                if (sbf) {  // 128 rows of strip col / 32 from row r0: 8 KB contiguous per plane
                    unsigned short* g = sbf + (size_t)(col >> 5) * 32 * mp + (size_t)r0 * 32;
                    bulk_s2g(g, hre, 8192);
                    bulk_s2g(g + (size_t)mp * mp, him, 8192);
                } else {
                    tma2d_store(smap, 0, ys + (col >> 5) * mp + r0, bre);
                    tma2d_store(smap, 0, ys + (mp / 32 + (col >> 5)) * mp + r0, bim);
                }
                bulk_commit();
            }
        }
        if (threadIdx.x == 0) bulk_wait_read_all();  // the buffers stay valid until read
    } else if (STORE && ok && done) {
        const int r = warp * 32 + lane;  // TMEM lane = tile row
        const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
        float* pr = gre + (size_t)(r0 + r) * mp + c0;
        float* pi = gim + (size_t)(r0 + r) * mp + c0;
#pragma unroll 1
        for (int ch = 0; ch < T2_BN / 16; ++ch) {
            float dr[16], di[16];
            tc::tmem_ld16(lane_addr + ch * 16, dr);
            tc::tmem_ld16(lane_addr + T2_BN + ch * 16, di);
            tc::tmem_ld_wait();
            if (r < nrows && ch * 16 < ncols) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    reinterpret_cast<float4*>(pr + ch * 16)[q] =
                        make_float4(dr[4 * q], dr[4 * q + 1], dr[4 * q + 2], dr[4 * q + 3]);
                    reinterpret_cast<float4*>(pi + ch * 16)[q] =
                        make_float4(di[4 * q], di[4 * q + 1], di[4 * q + 2], di[4 * q + 3]);
                }
                if (pk && pk_side == 0) {  // L21 row r: K' = column (Re), TB + column (Im)
                    constexpr int EPS = Cfg::PER_CORE;
#pragma unroll
                    for (int u = 0; u < 16 / EPS; ++u) {
                        pack2_seg<KIND>(pk, T2_BM, r, ch * 16 + u * EPS, dr + u * EPS, false);
                        pack2_seg<KIND>(pk, T2_BM, r, TB + ch * 16 + u * EPS, di + u * EPS, false);
                    }
                } else if (pk) {  // U12 row r = K index: B' rows j (Re) and T2_BN + j (Im)
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int j = ch * 16 + e;
                        if (j < ncols) {
                            pack2_store<KIND>(pk, 2 * T2_BN, j, r, dr[e], true);
                            pack2_store<KIND>(pk, 2 * T2_BN, T2_BN + j, r, di[e], true);
                        }
                    }
                }
            }
        }
    } else if (!STORE && ok && done) {
        const int r = warp * 32 + lane;  // TMEM lane = tile row
        const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
        float4* cr = reinterpret_cast<float4*>(sCr + r * T2_CROW);
        float4* ci = reinterpret_cast<float4*>(sCi + r * T2_CROW);
#pragma unroll 1
        for (int ch = 0; ch < T2_BN / 16; ++ch) {
            float dr[16], di[16];
            tc::tmem_ld16(lane_addr + ch * 16, dr);
            tc::tmem_ld16(lane_addr + T2_BN + ch * 16, di);
            tc::tmem_ld_wait();
            if (ch * 16 < ncols) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 a = cr[ch * 4 + q], b = ci[ch * 4 + q];
                    a.x -= dr[4 * q]; a.y -= dr[4 * q + 1]; a.z -= dr[4 * q + 2]; a.w -= dr[4 * q + 3];
                    b.x -= di[4 * q]; b.y -= di[4 * q + 1]; b.z -= di[4 * q + 2]; b.w -= di[4 * q + 3];
                    cr[ch * 4 + q] = a;
                    ci[ch * 4 + q] = b;
                }
            }
        }
        fence_async_shared();
        __syncthreads();
        if (r < nrows) {
            bulk_s2g(gre + (size_t)(r0 + r) * mp + c0, sCr + r * T2_CROW, row_bytes);
            bulk_s2g(gim + (size_t)(r0 + r) * mp + c0, sCi + r * T2_CROW, row_bytes);
            bulk_commit();
        }
        if (pk) pack_staged_b<KIND>(pk, sCr, sCi, ncols);  // reads the tile beside the bulk stores
        if (r < nrows) bulk_wait_read_all();
    } else if (!(ok && done)) {
        // bounded: let in-flight copies and MMAs land before TMEM is released
        if (staged) tc::mbar_wait(&bar_c, 0);
        tc::mbar_wait(&bar_mma, 0);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

// ---------------------------------------------------------------------------
// Row-pair tile for the interior of the trailing update: two vertically adjacent
// 128 x 128 complex tiles (rows r0 .. r0 + 256, columns c0 .. c0 + 128) share each
// B' chunk, so a CTA brings the A' chunks of both tiles and one B' chunk per K step
// into shared memory (192 KB of operands per 128 x 128 tile instead of 256 KB; the
// operand stream through L2 is what bounds the single-tile kernel).  The MMAs of a
// K step go into two accumulators of 256 TMEM columns.  The
// epilogue runs half by half: C rows staged in the freed operand ring with bulk
// copies, D subtracted, rows written back with bulk copies; the second half reuses
// the ring once the first half's stores have read it.  A missing second half (odd
// tile count) is neither loaded nor computed.  Every wait is bounded.
// ---------------------------------------------------------------------------
constexpr int T2P_STAGES = 4;

template <int KIND>
struct Tc2p {
    static constexpr int STAGE = 4 * Tc2<KIND>::A_CHUNK + Tc2<KIND>::B_CHUNK;  // A0 re, im | A1 re, im | B'
    static_assert(T2P_STAGES * STAGE <= 227 * 1024, "ring must fit one CTA");
    static constexpr int SMEM = T2P_STAGES * STAGE;
    static_assert(SMEM >= 2 * T2_C_BYTES, "a half tile of C must fit the freed operand ring");
};

// pk0 / pk1 (nullable): A' tiles of the next outer step to pack the updated halves into
// (tiles of the next panel's column block).
template <int KIND>
__device__ __forceinline__ void tc2_pair_body(int mp, int r0, int c0, bool two, float* __restrict__ re_plane,
                                              const unsigned char* __restrict__ ga0,
                                              const unsigned char* __restrict__ ga1,
                                              const unsigned char* __restrict__ gb, int* __restrict__ err,
                                              unsigned char* __restrict__ pk0 = nullptr,
                                              unsigned char* __restrict__ pk1 = nullptr,
                                              const unsigned char* __restrict__ ga0_old = nullptr,
                                              const unsigned char* __restrict__ ga1_old = nullptr,
                                              const unsigned char* __restrict__ gb_old = nullptr) {
    using Cfg = Tc2<KIND>;
    using Pc = Tc2p<KIND>;
    const int nsteps = (ga0_old ? 2 : 1) * Cfg::NIT;
    constexpr int NS = T2P_STAGES;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sCr = smem;
    unsigned char* sCi = smem + T2_C_BYTES;
    __shared__ __align__(8) uint64_t bar_c, bar_mma, bar_full[NS], bar_empty[NS];
    __shared__ uint32_t tmem_base;
    __shared__ int ok_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncols = min(T2_BN, mp - c0);  // multiple of 64
    const uint32_t row_bytes = (uint32_t)ncols * 4;
    const int nrow0 = min(T2_BM, mp - r0);
    const int nrow1 = two ? min(T2_BM, mp - r0 - T2_BM) : 0;
    float* gre = re_plane;
    float* gim = re_plane + (size_t)mp * mp;
    const uint32_t stage_tx = (uint32_t)((two ? 4 : 2) * Cfg::A_CHUNK + Cfg::B_CHUNK);

    if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar_c, 1);
        tc::mbar_init(&bar_mma, 1);
        for (int st = 0; st < NS; ++st) {
            tc::mbar_init(&bar_full[st], 1);
            tc::mbar_init(&bar_empty[st], 1);
        }
        tc::fence_barrier_init();
        ok_flag = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    {  // C rows of both halves towards L2 while the operands stream
        const int r = threadIdx.x;
        if (r < nrow0) {
            bulk_prefetch_l2(gre + (size_t)(r0 + r) * mp + c0, row_bytes);
            bulk_prefetch_l2(gim + (size_t)(r0 + r) * mp + c0, row_bytes);
        }
        if (r < nrow1) {
            bulk_prefetch_l2(gre + (size_t)(r0 + T2_BM + r) * mp + c0, row_bytes);
            bulk_prefetch_l2(gim + (size_t)(r0 + T2_BM + r) * mp + c0, row_bytes);
        }
    }
    if (threadIdx.x == 0) {
        auto load_chunk = [&](int c) {  // main-loop step c (the older operand set first, if any)
            const int st = c % NS;
            const bool old = ga0_old && c < Cfg::NIT;
            const unsigned char* a0 = old ? ga0_old : ga0;
            const unsigned char* a1 = old ? ga1_old : ga1;
            const unsigned char* b = old ? gb_old : gb;
            const int cl = old || !ga0_old ? c : c - Cfg::NIT;
            const int kc = Cfg::re_chunk(cl);
            const size_t ka = (size_t)kc * Cfg::A_CHUNK, kai = (size_t)(kc + Cfg::HALF) * Cfg::A_CHUNK;
            unsigned char* sa = smem + st * Pc::STAGE;
            tc::mbar_arrive_expect_tx(&bar_full[st], stage_tx);
            tc::bulk_g2s(sa, a0 + ka, Cfg::A_CHUNK, &bar_full[st]);
            tc::bulk_g2s(sa + Cfg::A_CHUNK, a0 + kai, Cfg::A_CHUNK, &bar_full[st]);
            if (two) {
                tc::bulk_g2s(sa + 2 * Cfg::A_CHUNK, a1 + ka, Cfg::A_CHUNK, &bar_full[st]);
                tc::bulk_g2s(sa + 3 * Cfg::A_CHUNK, a1 + kai, Cfg::A_CHUNK, &bar_full[st]);
            }
            tc::bulk_g2s(sa + 4 * Cfg::A_CHUNK, b + (size_t)cl * Cfg::B_CHUNK, Cfg::B_CHUNK, &bar_full[st]);
        };
        for (int c = 0; c < NS - 1 && c < nsteps; ++c) load_chunk(c);
        bool ok = true;
        for (int c = 0; c < nsteps && ok; ++c) {
            const int st = c % NS;
            if (!tc::mbar_wait(&bar_full[st], (c / NS) & 1)) {
                ok = false;
                break;
            }
            const uint32_t a0 = tc::smem_u32(smem + st * Pc::STAGE);
            const uint32_t b0 = a0 + 4 * Cfg::A_CHUNK;
            cplx_mma_step<KIND>(tbase, a0, a0 + Cfg::A_CHUNK, b0, c == 0);
            if (two) cplx_mma_step<KIND>(tbase + 2u * T2_BN, a0 + 2 * Cfg::A_CHUNK, a0 + 3 * Cfg::A_CHUNK, b0, c == 0);
            tc::mma_commit(&bar_empty[st]);
            const int nxt = c + NS - 1;
            if (nxt < nsteps) {
                if (c >= 1) {
                    const int sp = (c - 1) % NS;
                    if (!tc::mbar_wait(&bar_empty[sp], ((c - 1) / NS) & 1)) {
                        ok = false;
                        break;
                    }
                }
                load_chunk(nxt);
            }
        }
        tc::mma_commit(&bar_mma);  // tracks every MMA issued, also after a failed wait
        if (!ok) {
            ok_flag = 0;
            atomicCAS(err, 0, 1);
        }
    }
    __syncthreads();
    const bool ok = ok_flag != 0;
    bool mine = false;
    if (ok) {
        mine = tc::mbar_wait(&bar_mma, 0);
        if (!mine && lane == 0) atomicCAS(err, 0, 2);
    }
    bool done = __syncthreads_and(mine) != 0;
    tc::fence_after_sync();
    bool staged = false;   // C copies of the current half in flight
    uint32_t cphase = 0;   // bar_c phase of the current half
    for (int h = 0; h < 2 && ok && done; ++h) {
        const int nrows = h == 0 ? nrow0 : nrow1;
        if (nrows <= 0) break;
        const int rh = r0 + h * T2_BM;
        if (threadIdx.x == 0) tc::mbar_arrive_expect_tx(&bar_c, 2u * (uint32_t)nrows * row_bytes);
        __syncthreads();
        const int r = threadIdx.x;
        if (r < nrows) {
            tc::bulk_g2s(sCr + r * T2_CROW, gre + (size_t)(rh + r) * mp + c0, row_bytes, &bar_c);
            tc::bulk_g2s(sCi + r * T2_CROW, gim + (size_t)(rh + r) * mp + c0, row_bytes, &bar_c);
        }
        staged = true;
        const bool cok = tc::mbar_wait(&bar_c, cphase);
        if (!cok && lane == 0) atomicCAS(err, 0, 2);
        done = __syncthreads_and(cok) != 0;
        if (!done) break;
        staged = false;
        cphase ^= 1u;
        const uint32_t lane_addr = tbase + (uint32_t)h * 2u * T2_BN + ((uint32_t)(warp * 32) << 16);
        float4* cr = reinterpret_cast<float4*>(sCr + r * T2_CROW);
        float4* ci = reinterpret_cast<float4*>(sCi + r * T2_CROW);
#pragma unroll 1
        for (int ch = 0; ch < T2_BN / 16; ++ch) {
            float dr[16], di[16];
            tc::tmem_ld16(lane_addr + ch * 16, dr);
            tc::tmem_ld16(lane_addr + T2_BN + ch * 16, di);
            tc::tmem_ld_wait();
            if (ch * 16 < ncols) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 a = cr[ch * 4 + q], b = ci[ch * 4 + q];
                    a.x -= dr[4 * q]; a.y -= dr[4 * q + 1]; a.z -= dr[4 * q + 2]; a.w -= dr[4 * q + 3];
                    b.x -= di[4 * q]; b.y -= di[4 * q + 1]; b.z -= di[4 * q + 2]; b.w -= di[4 * q + 3];
                    cr[ch * 4 + q] = a;
                    ci[ch * 4 + q] = b;
                }
            }
        }
        fence_async_shared();
        __syncthreads();
        if (r < nrows) {
            bulk_s2g(gre + (size_t)(rh + r) * mp + c0, sCr + r * T2_CROW, row_bytes);
            bulk_s2g(gim + (size_t)(rh + r) * mp + c0, sCi + r * T2_CROW, row_bytes);
            bulk_commit();
        }
        unsigned char* pkh = h == 0 ? pk0 : pk1;
        if (pkh) pack_staged_a<KIND>(pkh, sCr, sCi, nrows);  // reads the half beside the bulk stores
        if (r < nrows) bulk_wait_read_all();  // the next half reuses the buffer
        __syncthreads();
    }
    if (!(ok && done)) {
        // bounded: let in-flight copies and MMAs land before TMEM is released
        if (staged) tc::mbar_wait(&bar_c, cphase);
        tc::mbar_wait(&bar_mma, 0);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

// Outer trailing update of tile (ti, tj): C[R0 + 128 ti.., R0 + 128 tj..] -= D.
// apack_old / bpack_old (optional): the previous outer step's packed operands, whose
// tiles are one index further (their trailing matrix starts 128 rows and columns earlier).
template <int KIND>
__device__ __forceinline__ void tc2_update_body(int mp, int R0, float* __restrict__ re_plane,
                                                const unsigned char* __restrict__ apack,
                                                const unsigned char* __restrict__ bpack, int* __restrict__ err, int ti,
                                                int tj, unsigned char* __restrict__ pk_next = nullptr,
                                                const unsigned char* __restrict__ apack_old = nullptr,
                                                const unsigned char* __restrict__ bpack_old = nullptr) {
    using Cfg = Tc2<KIND>;
    tc2_tile_body<KIND, false>(mp, R0 + ti * T2_BM, R0 + tj * T2_BN, re_plane, apack + (size_t)ti * Cfg::A_TILE,
                               bpack + (size_t)tj * Cfg::B_TILE, err, pk_next, 1,
                               apack_old ? apack_old + (size_t)(ti + 1) * Cfg::A_TILE : nullptr,
                               bpack_old ? bpack_old + (size_t)(tj + 1) * Cfg::B_TILE : nullptr);
}

}  // namespace fde
