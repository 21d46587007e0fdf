// Interior trailing update of the tensor-core LU (A22 -= L21 U12 over the tiles
// ti, tj >= 1 of an outer step) with the C tiles streamed by tensor-map copies.
//
// One CTA takes up to S_WQ consecutive 128 x 128 complex tiles of one Strang block
// (same packed operands and the same MMAs in the same K order as the row-pair and
// single-tile kernels of lu_tc2.cuh, so the factors are bit-identical) with 256 threads:
//   warp 0 (lane 0)  operand producer: the A' (real and imaginary K part) and B' chunks
//                    of each K step into a ring of S_OPS stages (bulk copies);
//   warp 1 (lane 0)  MMA issuer: one of two 256-column TMEM accumulators per tile,
//                    alternating, so the MMAs of tile q + 1 run during the epilogue of q;
//   warp 2 (lane 0)  C producer: the C tile in four chunks of 32 columns (Re and Im
//                    planes, 128 rows each) by 128-byte-swizzled tensor-map loads into a
//                    ring of S_C chunks;
//   warps 4..7       epilogue, one TMEM lane quadrant each (thread = tile row): per chunk
//                    D is read with tcgen05.ld and subtracted from the staged C, and the
//                    chunk goes back to global memory by a tensor-map store.
// A C chunk is two 16 KB copies each way instead of 128-row bulk copies, and the ring
// keeps up to three chunks of C reads in flight beside the operand stream.  Every wait
// is bounded: on a timeout the CTA records an error, stops issuing, lets its copies and
// MMAs land, frees its TMEM and returns; the epilogue warps decide together (a barrier
// reduction), so none is left at a named barrier.
#pragma once

#include <cuda.h>

#include "lu_tc2w.cuh"

namespace fde {

constexpr int S_OPS = 4;            // operand stages (one K step of A' re, A' im and B' each)
constexpr int S_C = 3;              // C chunks in flight
constexpr int S_CHUNK = 32 * 1024;  // Re and Im of 128 rows x 32 columns
constexpr int S_WQ = 8;             // tiles per CTA
constexpr int S_THREADS = 256;

template <int KIND>
struct Tc2s {
    static constexpr int SMEM = S_OPS * Tc2<KIND>::STAGE + S_C * S_CHUNK + 1024;  // + alignment slack
    static_assert(Tc2<KIND>::STAGE % 1024 == 0, "stages keep the 1024-byte alignment of the swizzled chunks");
    static_assert(SMEM <= 227 * 1024, "rings must fit one CTA");
};

// Tiles x0 .. x0 + nq - 1 of one block's trailing matrix (tiles of 128 from R0, nt per
// dimension): front = 0 -> the square of tiles ti, tj >= f, x -> (f + x / (nt - f),
// f + x % (nt - f)); front = 1 -> row 1 and column 1, x -> (1, 1 + x) for x < nt - 1,
// else (2 + x - (nt - 1), 1).  apack / bpack: this block's packed operand tiles of the
// step; apack_old / bpack_old (optional): the previous step's, applied first in the same
// accumulator (their tile indices are one larger).  cmap: the factor planes of all blocks
// as rows of m_p floats (block k's Re plane from row 2 k m_p, Im plane from row
// (2 k + 1) m_p), boxes of 128 rows x 32 columns, 128-byte swizzle.
template <int KIND>
__device__ __forceinline__ void tc2s_body(int mp, int R0, int nt, int f, int front, int x0, int nq, int k,
                                          const unsigned char* __restrict__ apack,
                                          const unsigned char* __restrict__ bpack,
                                          const unsigned char* __restrict__ apack_old,
                                          const unsigned char* __restrict__ bpack_old, int* __restrict__ err,
                                          const CUtensorMap* cmap) {
    using Cfg = Tc2<KIND>;
    const int nsteps = (apack_old ? 2 : 1) * Cfg::NIT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t ofull[S_OPS], oempty[S_OPS], cfull[S_C], cempty[S_C], acc_full[2],
        acc_empty[2], mma_done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ int n_oi, n_ot, n_ci, n_ct;  // operand stages / C chunks issued and taken

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char* ring = smem_raw + (sbase - tc::smem_u32(smem_raw));
    unsigned char* cring = ring + S_OPS * Cfg::STAGE;
    const int yre0 = k * 2 * mp;  // tensor-map row of block k's Re plane
    auto tile_rc = [&](int q, int& r0, int& c0, int& ti, int& tj) {
        const int x = x0 + q;
        if (front) {
            ti = x < nt - 1 ? 1 : 2 + x - (nt - 1);
            tj = x < nt - 1 ? 1 + x : 1;
        } else {
            ti = f + x / (nt - f);
            tj = f + x % (nt - f);
        }
        r0 = R0 + ti * T2_BM;
        c0 = R0 + tj * T2_BN;
    };
    auto fail = [&](int code) {
        abort_flag = 1;
        atomicCAS(err, 0, code);
    };

    if (warp == 1) tc::tmem_alloc(&tmem_base, 512);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S_OPS; ++s) {
            tc::mbar_init(&ofull[s], 1);
            tc::mbar_init(&oempty[s], 1);
        }
        for (int s = 0; s < S_C; ++s) {
            tc::mbar_init(&cfull[s], 1);
            tc::mbar_init(&cempty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&acc_full[a], 1);
            tc::mbar_init(&acc_empty[a], 1);
        }
        tc::mbar_init(&mma_done, 1);
        tc::fence_barrier_init();
        abort_flag = 0;
        n_oi = n_ot = n_ci = n_ct = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;

    if (warp == 0) {
        if (lane == 0) {  // operand producer
            int u = 0;
            for (int q = 0; q < nq && !abort_flag; ++q) {
                int r0, c0, ti, tj;
                tile_rc(q, r0, c0, ti, tj);
                const unsigned char* ga = apack + (size_t)ti * Cfg::A_TILE;
                const unsigned char* gb = bpack + (size_t)tj * Cfg::B_TILE;
                const unsigned char* gao = apack_old ? apack_old + (size_t)(ti + 1) * Cfg::A_TILE : nullptr;
                const unsigned char* gbo = bpack_old ? bpack_old + (size_t)(tj + 1) * Cfg::B_TILE : nullptr;
                bool ok = true;
                for (int c = 0; c < nsteps; ++c) {
                    const int s = u % S_OPS;
                    if (u >= S_OPS && !tc::mbar_wait(&oempty[s], (uint32_t)((u / S_OPS - 1) & 1))) {
                        fail(1);
                        ok = false;
                        break;
                    }
                    const bool old = gao && c < Cfg::NIT;
                    const unsigned char* a = old ? gao : ga;
                    const unsigned char* b = old ? gbo : gb;
                    const int cl = old || !gao ? c : c - Cfg::NIT;
                    const int kc = Cfg::re_chunk(cl);
                    unsigned char* dst = ring + s * Cfg::STAGE;
                    tc::mbar_arrive_expect_tx(&ofull[s], Cfg::STAGE);
                    tc::bulk_g2s(dst, a + (size_t)kc * Cfg::A_CHUNK, Cfg::A_CHUNK, &ofull[s]);
                    tc::bulk_g2s(dst + Cfg::A_CHUNK, a + (size_t)(kc + Cfg::HALF) * Cfg::A_CHUNK, Cfg::A_CHUNK,
                                 &ofull[s]);
                    tc::bulk_g2s(dst + 2 * Cfg::A_CHUNK, b + (size_t)cl * Cfg::B_CHUNK, Cfg::B_CHUNK, &ofull[s]);
                    n_oi = ++u;
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int u = 0;
            for (int q = 0; q < nq && !abort_flag; ++q) {
                const int a = q & 1;
                if (q >= 2 && !tc::mbar_wait(&acc_empty[a], (uint32_t)(((q >> 1) - 1) & 1))) {
                    fail(2);
                    break;
                }
                tc::fence_after_sync();
                const uint32_t tacc = tbase + (uint32_t)a * 2u * T2_BN;
                bool ok = true;
                for (int c = 0; c < nsteps; ++c) {
                    const int s = u % S_OPS;
                    if (abort_flag || !tc::mbar_wait(&ofull[s], (uint32_t)((u / S_OPS) & 1))) {
                        fail(1);
                        ok = false;
                        break;
                    }
                    n_ot = ++u;
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_u32(ring + s * Cfg::STAGE);
                    cplx_mma_step<KIND>(tacc, a0, a0 + Cfg::A_CHUNK, a0 + 2 * Cfg::A_CHUNK, c == 0);
                    tc::mma_commit(&oempty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&acc_full[a]);
            }
            tc::mma_commit(&mma_done);  // tracks every MMA issued
        }
    } else if (warp == 2) {
        if (lane == 0) {  // C producer
            int v = 0;
            for (int q = 0; q < nq && !abort_flag; ++q) {
                int r0, c0, ti, tj;
                tile_rc(q, r0, c0, ti, tj);
                bool ok = true;
                for (int ch = 0; ch < 4; ++ch) {
                    const int s = v % S_C;
                    if (v >= S_C && !tc::mbar_wait(&cempty[s], (uint32_t)((v / S_C - 1) & 1))) {
                        fail(3);
                        ok = false;
                        break;
                    }
                    unsigned char* dst = cring + s * S_CHUNK;
                    tc::mbar_arrive_expect_tx(&cfull[s], S_CHUNK);
                    tma2d_load(dst, cmap, c0 + 32 * ch, yre0 + r0, &cfull[s]);
                    tma2d_load(dst + S_CHUNK / 2, cmap, c0 + 32 * ch, yre0 + mp + r0, &cfull[s]);
                    n_ci = ++v;
                }
                if (!ok) break;
            }
        }
    } else if (warp >= 4) {  // epilogue: thread r = tile row, TMEM lane quadrant warp - 4
        const int r = (warp - 4) * 32 + lane;
        const uint32_t tl = tbase + ((uint32_t)((warp - 4) * 32) << 16);
        int v = 0;
        for (int q = 0; q < nq; ++q) {
            int r0, c0, ti, tj;
            tile_rc(q, r0, c0, ti, tj);
            const int a = q & 1;
            bool ok = named_and(2, 128, !abort_flag && tc::mbar_wait(&acc_full[a], (uint32_t)((q >> 1) & 1)));
            if (!ok) {
                fail(2);
                break;
            }
            tc::fence_after_sync();
            for (int ch = 0; ch < 4; ++ch) {
                const int s = v % S_C;
                ok = named_and(2, 128, !abort_flag && tc::mbar_wait(&cfull[s], (uint32_t)((v / S_C) & 1)));
                if (!ok) {
                    fail(3);
                    break;
                }
                float dr[32], di[32];
                const uint32_t ta = tl + (uint32_t)a * 2u * T2_BN + 32u * ch;
                tc::tmem_ld16(ta, dr);
                tc::tmem_ld16(ta + 16u, dr + 16);
                tc::tmem_ld16(ta + T2_BN, di);
                tc::tmem_ld16(ta + T2_BN + 16u, di + 16);
                tc::tmem_ld_wait();
                unsigned char* cr = cring + s * S_CHUNK;
                unsigned char* ci = cr + S_CHUNK / 2;
#pragma unroll
                for (int u = 0; u < 8; ++u) {  // 16-byte unit u of row r sits at unit u ^ (r mod 8)
                    const uint32_t off = (uint32_t)(r * 128 + ((u ^ (r & 7)) << 4));
                    float4 x = *reinterpret_cast<float4*>(cr + off);
                    float4 y = *reinterpret_cast<float4*>(ci + off);
                    x.x -= dr[4 * u]; x.y -= dr[4 * u + 1]; x.z -= dr[4 * u + 2]; x.w -= dr[4 * u + 3];
                    y.x -= di[4 * u]; y.y -= di[4 * u + 1]; y.z -= di[4 * u + 2]; y.w -= di[4 * u + 3];
                    *reinterpret_cast<float4*>(cr + off) = x;
                    *reinterpret_cast<float4*>(ci + off) = y;
                }
                fence_async_shared();
                tc::fence_before_sync();
                epi_sync();  // the chunk is complete (and this tile's TMEM reads, after the last chunk)
                if (r == 0) {
                    tma2d_store(cmap, c0 + 32 * ch, yre0 + r0, cr);
                    tma2d_store(cmap, c0 + 32 * ch, yre0 + mp + r0, ci);
                    bulk_commit();
                    bulk_wait_read_all();  // the stores have read the chunk: the slot is free
                    mbar_arrive_local(&cempty[s]);
                    n_ct = v + 1;
                }
                ++v;
            }
            if (!ok) break;
            if (r == 0) mbar_arrive_local(&acc_empty[a]);  // the accumulator has been read
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) {
        // bounded: let what was issued land before the CTA (and its TMEM) goes away
        for (int u = n_ot; u < n_oi; ++u) tc::mbar_wait(&ofull[u % S_OPS], (uint32_t)((u / S_OPS) & 1));
        for (int v = n_ct; v < n_ci; ++v) tc::mbar_wait(&cfull[v % S_C], (uint32_t)((v / S_C) & 1));
    }
    if (threadIdx.x == 32) tc::mbar_wait(&mma_done, 0);  // every MMA has completed
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, 512);
    }
}

}  // namespace fde
