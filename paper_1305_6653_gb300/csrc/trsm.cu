// Tensor-core block solves for many right-hand sides of one Strang-preconditioned
// operator (Sec. 3.2: the factors of the s/2+1 blocks depend only on the operator, so
// every right-hand side of a shared-operator batch reuses them).
//
// One CTA solves L U x = r for one Strang block and a group of TRSM_R = 16
// right-hand sides, in strips of 128 rows, right-looking:
//   forward  y_d = L_dd^{-1} (r_d - acc_d),  then acc_e += L_ed y_d  for e > d;
//   backward x_d = U_dd^{-1} (y_d - acc_d),  then acc_e += U_ed x_d  for e < d.
// Every product is a tcgen05 MMA (kind::tf32, M = 128, N = 2 x 16: Re and Im of the
// 16 right-hand sides side by side), the complex product split as in lu_tc2.cuh:
//   acc[:, 0:32] += Re A . [Re X | Im X],  acc[:, 0:16] -= Im A . Im X,
//   acc[:, 16:32] += Im A . Re X.
// The accumulators of all strips stay in TMEM (32 columns each, 512 for m_p = 2048),
// so the factor is read once per group: the off-diagonal 128 x 128 blocks of L and U
// come straight from the FP32 factor planes by tensor-map copies (128-byte swizzle,
// boxes of 128 rows x 32 columns), and the diagonal blocks' inverses L_dd^{-1},
// U_dd^{-1} are the ones the tensor-core LU computed for its panel products (kept as
// packed TF32 operand tiles).  The solved strip, rounded to TF32, is the B operand of
// its column's products.
//
// Roles (192 threads): warp 0 lane 0 streams operands through a ring of 32 KB stages
// (full / empty mbarriers); warp 1 lane 0 issues the MMAs; warps 2..5 (one TMEM lane
// quadrant each, thread = strip row) read the accumulators, form the right-hand side
// of the diagonal product, and write the solved strip to global memory and to the B
// buffer.  The strip after d only waits for the first block of column d (its own
// accumulator), so the diagonal work of one strip overlaps the column stream of the
// previous one.  Every wait is bounded: on a timeout the CTA records an error, stops,
// lets its copies and MMAs land, frees its TMEM and returns.
#include <cuda.h>

#include "fde_internal.h"
#include "lu_tc2.cuh"

namespace fde {

namespace {

constexpr int TRSM_R = 16;             // right-hand sides per CTA
constexpr int TRSM_ST = 128;           // strip rows
constexpr int TRSM_STAGES = 5;
constexpr int TRSM_STAGE = 32 * 1024;  // a 128 x 32 column chunk of both planes, or 32 K of a diagonal inverse
constexpr int TRSM_XBUF = TRSM_ST * 2 * TRSM_R * 4;  // B operand: 128 K x 32 TF32 = 16 KB
constexpr int TRSM_THREADS = 192;
constexpr int TRSM_SMEM = TRSM_STAGES * TRSM_STAGE + 3 * TRSM_XBUF + 1024;  // + alignment slack

// Byte offset of B-operand element (n, k): K-major core matrices of 8 n x 4 k, one
// 1 KB block per MMA K step of 8 (LBO = 128 B along K, SBO = 256 B between n groups).
__device__ __forceinline__ uint32_t xoff(int n, int k) {
    return (uint32_t)((k >> 3) * 1024 + (n >> 3) * 256 + ((k & 7) >> 2) * 128 + (n & 7) * 16 + (k & 3) * 4);
}

// Shared-memory descriptor of a K-major tile written by a 128-byte-swizzled tensor-map
// copy (rows of 128 B, 8-row groups 1024 B apart; the start may be advanced by the
// K offset inside the 128-byte row).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading offset: unused for swizzled K-major
    d |= (uint64_t)(1024 >> 4) << 32;    // stride between 8-row groups
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(tc::smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// AND of v over the 128 epilogue threads (named barrier 1).
__device__ __forceinline__ bool epi_and(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.and.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

constexpr uint32_t ID32 = tc::instr_desc(2u, 128, 2 * TRSM_R);
constexpr uint32_t ID16 = tc::instr_desc(2u, 128, TRSM_R);
constexpr uint32_t ID16N = ID16 | tc::IDESC_NEGATE_A;

// One K step of 8: A real / imaginary parts (descriptors), B = the X buffer block of
// this K step (1 KB: n groups 0, 1 Re, 2, 3 Im).
__device__ __forceinline__ void trsm_mma(uint32_t tacc, uint64_t are, uint64_t aim, uint32_t xb, bool first) {
    const uint64_t bfull = tc::smem_desc(xb, 128, 256);
    const uint64_t bim = tc::smem_desc(xb + 512, 128, 256);
    tc::mma_tf32(tacc, are, bfull, ID32, first ? 0u : 1u);
    tc::mma_tf32(tacc, aim, bim, ID16N, 1u);
    tc::mma_tf32(tacc + TRSM_R, aim, bfull, ID16, 1u);
}

}  // namespace

// grid (ceil(nact / 16), nblk).  fmap: the factor planes as a 2-D array of
// nblk * 2 * m_p rows of m_p floats (block k's Re plane at row 2 k m_p, Im plane at
// row (2 k + 1) m_p); dtile: per block and strip, the packed L_dd^{-1} and U_dd^{-1}.
__global__ void __launch_bounds__(TRSM_THREADS, 1)
block_trsm_tc_kernel(const InstDev* __restrict__ I, const int* __restrict__ act, int nact, int mp, int nblk,
                     const unsigned char* __restrict__ dtile, int* __restrict__ err,
                     const __grid_constant__ CUtensorMap fmap) {
    using Cfg = Tc2<0>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[TRSM_STAGES], empty[TRSM_STAGES], a_full, y_full, diag_full, acc_full,
        xfree[2], mma_done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ long n_issued, n_taken;
    __shared__ float2* rh[TRSM_R];  // the group's frequency-side vectors (NULL: no live instance)

    const int k = blockIdx.y;
    if (k >= nblk) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nst = mp / TRSM_ST;
    const uint32_t ncols = nst <= 1 ? 32u : nst <= 2 ? 64u : nst <= 4 ? 128u : nst <= 8 ? 256u : 512u;
    const uint32_t sbase = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char* smem = smem_raw + (sbase - tc::smem_u32(smem_raw));
    unsigned char* ring = smem;
    unsigned char* abuf = smem + TRSM_STAGES * TRSM_STAGE;
    unsigned char* xbuf = abuf + TRSM_XBUF;  // [2][16 KB]
    const unsigned char* dblk = dtile + (size_t)k * nst * 2 * Cfg::A_TILE;
    auto fail = [&](int code) {
        abort_flag = 1;
        atomicCAS(err, 0, code);
    };
    // strip g = 0 .. 2 nst - 1: forward strips 0 .. nst-1, then backward nst-1 .. 0
    auto strip = [&](int g) { return g < nst ? g : 2 * nst - 1 - g; };
    auto ncol = [&](int g) { return g < nst ? nst - 1 - g : 2 * nst - 1 - g; };  // off-diagonal blocks of column g
    auto col_e = [&](int g, int i) { return g < nst ? g + 1 + i : 2 * nst - 2 - g - i; };

    if (warp == 1) tc::tmem_alloc(&tmem_base, ncols);
    if (threadIdx.x == 0) {
        for (int s = 0; s < TRSM_STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&a_full, 1);
        tc::mbar_init(&y_full, 1);
        tc::mbar_init(&diag_full, 1);
        tc::mbar_init(&acc_full, 1);
        tc::mbar_init(&xfree[0], 1);
        tc::mbar_init(&xfree[1], 1);
        tc::mbar_init(&mma_done, 1);
        tc::fence_barrier_init();
        abort_flag = 0;
        n_issued = n_taken = 0;
    }
    if (threadIdx.x < TRSM_R) {
        const int a = TRSM_R * blockIdx.x + threadIdx.x;
        float2* p = nullptr;
        if (a < nact) {
            const InstDev& d = I[act[a]];
            if (d.ctl[0]) p = (float2*)d.rhat + (size_t)k * mp;
        }
        rh[threadIdx.x] = p;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;

    if (warp == 0) {
        if (lane == 0) {  // producer: every stage of both sweeps, in the order the MMA issuer takes them
            long u = 0;
            auto stage = [&](uint32_t& slot) -> bool {
                slot = (uint32_t)(u % TRSM_STAGES);
                if (u >= TRSM_STAGES && !tc::mbar_wait(&empty[slot], (uint32_t)((u / TRSM_STAGES - 1) & 1))) {
                    fail(1);
                    return false;
                }
                tc::mbar_arrive_expect_tx(&full[slot], TRSM_STAGE);
                return true;
            };
            for (int g = 0; g < 2 * nst && !abort_flag; ++g) {
                const int d = strip(g);
                const unsigned char* inv = dblk + ((size_t)d * 2 + (g < nst ? 0 : 1)) * Cfg::A_TILE;
                bool ok = true;
                for (int s = 0; s < 4 && ok; ++s) {  // diagonal inverse: A' chunks 2s, 2s+1 (Re K) and 2s+8, 2s+9 (Im K)
                    uint32_t slot;
                    if (!(ok = stage(slot))) break;
                    unsigned char* dst = ring + slot * TRSM_STAGE;
                    tc::bulk_g2s(dst, inv + (size_t)(2 * s) * Cfg::A_CHUNK, 2 * Cfg::A_CHUNK, &full[slot]);
                    tc::bulk_g2s(dst + 2 * Cfg::A_CHUNK, inv + (size_t)(2 * s + Cfg::HALF) * Cfg::A_CHUNK,
                                 2 * Cfg::A_CHUNK, &full[slot]);
                    n_issued = ++u;
                }
                for (int i = 0; i < ncol(g) && ok; ++i) {
                    const int e = col_e(g, i);
                    const int y = k * 2 * mp + TRSM_ST * e;
                    for (int c = 0; c < 4 && ok; ++c) {
                        uint32_t slot;
                        if (!(ok = stage(slot))) break;
                        unsigned char* dst = ring + slot * TRSM_STAGE;
                        tma_load_2d(dst, &fmap, TRSM_ST * d + 32 * c, y, &full[slot]);
                        tma_load_2d(dst + TRSM_STAGE / 2, &fmap, TRSM_ST * d + 32 * c, y + mp, &full[slot]);
                        n_issued = ++u;
                    }
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            long u = 0;
            auto take = [&](uint32_t& slot) -> bool {
                slot = (uint32_t)(u % TRSM_STAGES);
                if (abort_flag || !tc::mbar_wait(&full[slot], (uint32_t)((u / TRSM_STAGES) & 1))) {
                    fail(1);
                    return false;
                }
                n_taken = ++u;
                tc::fence_after_sync();
                return true;
            };
            for (int g = 0; g < 2 * nst && !abort_flag; ++g) {
                const int d = strip(g);
                const uint32_t tacc_d = tbase + (uint32_t)(32 * d);
                if (!tc::mbar_wait(&a_full, (uint32_t)(g & 1))) {
                    fail(2);
                    break;
                }
                tc::fence_after_sync();
                bool ok = true;
                const uint32_t ab = tc::smem_u32(abuf);
                for (int s = 0; s < 4; ++s) {  // X_d = inverse . A  (32 K per stage)
                    uint32_t slot;
                    if (!(ok = take(slot))) break;
                    const uint32_t st = tc::smem_u32(ring + slot * TRSM_STAGE);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t ao = (uint32_t)((ks >> 1) * Cfg::A_CHUNK + (ks & 1) * 256);
                        trsm_mma(tacc_d, tc::smem_desc(st + ao, 128, 512),
                                 tc::smem_desc(st + 2 * Cfg::A_CHUNK + ao, 128, 512), ab + (uint32_t)(4 * s + ks) * 1024u,
                                 s == 0 && ks == 0);
                    }
                    tc::mma_commit(&empty[slot]);
                }
                if (!ok) break;
                tc::mma_commit(&diag_full);
                if (!tc::mbar_wait(&y_full, (uint32_t)(g & 1))) {
                    fail(2);
                    break;
                }
                tc::fence_after_sync();
                const uint32_t xb = tc::smem_u32(xbuf + (g & 1) * TRSM_XBUF);
                const bool first_col = g == 0 || g == nst;
                for (int i = 0; i < ncol(g) && ok; ++i) {
                    const uint32_t tacc_e = tbase + (uint32_t)(32 * col_e(g, i));
                    for (int c = 0; c < 4; ++c) {  // acc_e += A_ed X_d, columns 32c .. 32c + 31 of the block
                        uint32_t slot;
                        if (!(ok = take(slot))) break;
                        const uint32_t st = tc::smem_u32(ring + slot * TRSM_STAGE);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks)
                            trsm_mma(tacc_e, sw128_desc(st + 32u * ks), sw128_desc(st + TRSM_STAGE / 2 + 32u * ks),
                                     xb + (uint32_t)(4 * c + ks) * 1024u, first_col && c == 0 && ks == 0);
                        tc::mma_commit(&empty[slot]);
                    }
                    if (ok && i == 0) tc::mma_commit(&acc_full);  // the next strip's accumulator is complete
                }
                if (!ok) break;
                tc::mma_commit(&xfree[g & 1]);
            }
            tc::mma_commit(&mma_done);  // tracks every MMA issued
        }
    } else {  // epilogue: thread = strip row (TMEM lane quadrant warp % 4)
        const int q = warp & 3, r = 32 * q + lane;
        const uint32_t tl = tbase + ((uint32_t)(32 * q) << 16);
        float2* rp[TRSM_R];
#pragma unroll
        for (int j = 0; j < TRSM_R; ++j) rp[j] = rh[j];
        long acc_n = 0;
        // right-hand side of the strip (r_d forward, y_d backward), loaded one strip ahead
        float2 bv[TRSM_R];
#pragma unroll
        for (int j = 0; j < TRSM_R; ++j) bv[j] = rp[j] ? rp[j][r] : make_float2(0.f, 0.f);
        for (int g = 0; g < 2 * nst; ++g) {
            const int d = strip(g);
            const size_t row = (size_t)TRSM_ST * d + r;
            float acc[2 * TRSM_R];
            if (g != 0 && g != nst) {  // the strip's accumulator (complete after the previous column's first block)
                const bool ok = epi_and(!abort_flag && tc::mbar_wait(&acc_full, (uint32_t)(acc_n & 1)));
                ++acc_n;
                if (!ok) {
                    fail(3);
                    break;
                }
                tc::fence_after_sync();
                tc::tmem_ld16(tl + 32u * d, acc);
                tc::tmem_ld16(tl + 32u * d + 16u, acc + 16);
                tc::tmem_ld_wait();
            } else {
#pragma unroll
                for (int j = 0; j < 2 * TRSM_R; ++j) acc[j] = 0.f;
            }
            // A = (r or y) - acc as the B operand of the diagonal product
#pragma unroll
            for (int j = 0; j < TRSM_R; ++j) {
                *reinterpret_cast<float*>(abuf + xoff(j, r)) = tc::to_tf32(bv[j].x - acc[j]);
                *reinterpret_cast<float*>(abuf + xoff(TRSM_R + j, r)) = tc::to_tf32(bv[j].y - acc[TRSM_R + j]);
            }
            fence_async_shared();
            tc::fence_before_sync();
            epi_bar();
            if (r == 0) arrive(&a_full);
            // the solved strip
            bool ok = epi_and(!abort_flag && tc::mbar_wait(&diag_full, (uint32_t)(g & 1)));
            if (!ok) {
                fail(3);
                break;
            }
            tc::fence_after_sync();
            float x[2 * TRSM_R];
            tc::tmem_ld16(tl + 32u * d, x);
            tc::tmem_ld16(tl + 32u * d + 16u, x + 16);
            tc::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < TRSM_R; ++j)
                if (rp[j]) rp[j][row] = make_float2(x[j], x[TRSM_R + j]);
            if (g + 1 < 2 * nst) {  // the next strip's right-hand side (a forward strip's y was stored above)
                const size_t nrow = (size_t)TRSM_ST * strip(g + 1) + r;
#pragma unroll
                for (int j = 0; j < TRSM_R; ++j) bv[j] = rp[j] ? rp[j][nrow] : make_float2(0.f, 0.f);
            }
            if (g >= 2) {  // the X buffer of strip g - 2 is free once its column's MMAs completed
                ok = epi_and(!abort_flag && tc::mbar_wait(&xfree[g & 1], (uint32_t)(((g - 2) >> 1) & 1)));
                if (!ok) {
                    fail(3);
                    break;
                }
            }
            unsigned char* xb = xbuf + (g & 1) * TRSM_XBUF;
#pragma unroll
            for (int j = 0; j < TRSM_R; ++j) {
                *reinterpret_cast<float*>(xb + xoff(j, r)) = tc::to_tf32(x[j]);
                *reinterpret_cast<float*>(xb + xoff(TRSM_R + j, r)) = tc::to_tf32(x[TRSM_R + j]);
            }
            fence_async_shared();
            tc::fence_before_sync();
            epi_bar();
            if (r == 0) arrive(&y_full);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) {
        // bounded: let the copies that were issued land before the CTA goes away
        for (long u = n_taken; u < n_issued; ++u)
            tc::mbar_wait(&full[u % TRSM_STAGES], (uint32_t)((u / TRSM_STAGES) & 1));
    }
    if (threadIdx.x == 32) tc::mbar_wait(&mma_done, 0);  // every MMA has completed
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, ncols);
    }
}

// A 2-D FP32 array (rows of `width` floats, `rows` rows) as a tensor map with boxes of
// 128 rows x 32 columns and 128-byte swizzle (the K-major layout the MMAs read).
static int tensor_map_sw128(const void* base, uint64_t width, uint64_t rows, CUtensorMap* map, const char* what) {
    using Fn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                            const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                            CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Fn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult qr;
        FDE_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr));
        if (qr != cudaDriverEntryPointSuccess || !fn)
            return set_error(FDE_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        encode = reinterpret_cast<Fn>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)width * sizeof(float)};
    const cuuint32_t box[2] = {32, (cuuint32_t)TRSM_ST};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult res = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (res != CUDA_SUCCESS) return set_error(FDE_ERR_CUDA, std::string("cuTensorMapEncodeTiled failed for ") + what);
    return FDE_OK;
}

// Factor planes of nblk blocks: rows of m_p floats, row y = (2 k + plane) m_p + r.
int factor_tensor_map_sw128(const void* fac, int mp, int nblk, CUtensorMap* map) {
    return tensor_map_sw128(fac, (uint64_t)mp, (uint64_t)nblk * 2 * mp, map, "the factor planes");
}

// Strip-major copy of the factor planes: rows of 32 floats, row y = ((2 k + plane) m_p / 32
// + c / 32) m_p + r for element (r, c), so a box is 128 consecutive rows of one strip.
int strip_tensor_map_sw128(const void* strips, int mp, int nblk, CUtensorMap* map) {
    return tensor_map_sw128(strips, 32, (uint64_t)nblk * 2 * (mp / 32) * mp, map, "the factor strips");
}

bool trsm_tc_supported(int mp) { return mp % TRSM_ST == 0 && mp >= 2 * TRSM_ST && mp <= 16 * TRSM_ST; }

int launch_trsm_tc(const InstDev* I, const int* act, int nact, const void* fac, const void* dtile, int mp, int nblk,
                   int* err, cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    if (!trsm_tc_supported(mp) || !dtile) return set_error(FDE_ERR_ARG, "tensor-core block solves need 256 <= m_p <= 2048, m_p % 128 == 0 and saved diagonal inverses");
    CUtensorMap map;
    int rc = factor_tensor_map_sw128(fac, mp, nblk, &map);
    if (rc) return rc;
    FDE_CUDA_TRY(cudaFuncSetAttribute(block_trsm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TRSM_SMEM));
    block_trsm_tc_kernel<<<dim3((nact + TRSM_R - 1) / TRSM_R, nblk), TRSM_THREADS, TRSM_SMEM, st>>>(
        I, act, nact, mp, nblk, (const unsigned char*)dtile, err, map);
    FDE_LAUNCH_CHECK("block_trsm_tc_kernel");
    return FDE_OK;
}

}  // namespace fde
