// Interior trailing update of the tensor-core LU (A22 -= L21 U12 over the tiles
// ti, tj >= 1 of an outer step), warp-specialized so that one tile's epilogue runs
// while the next tile's operands stream and its MMAs issue.
//
// One CTA takes up to WQ consecutive 128 x 128 complex tiles of one Strang block
// (same layout and packed operands as tc2_tile_body in lu_tc2.cuh) with 256 threads:
//   warp 0 (lane 0)  producer: the A' (real and imaginary K part) and B' chunks of
//                    each K step into a ring of W_STAGES stages (bulk copies, full /
//                    empty mbarriers);
//   warp 1 (lane 0)  MMA issuer: the complex K step of lu_tc2.cuh into one of two
//                    TMEM accumulators (512 columns), alternating by tile, so that the
//                    MMAs of tile q + 1 do not wait for the epilogue of tile q;
//   warps 4..7       epilogue, one TMEM lane quadrant each (thread = tile row): the C
//                    tile is staged and written back in two 64-column halves with bulk
//                    copies (C prefetched into L2 one tile ahead), D read with
//                    tcgen05.ld and subtracted; the accumulator is then released to the
//                    MMA issuer.
// The MMAs, their K order and the subtraction are those of the single-tile and
// row-pair kernels, so the result is bit-identical to theirs.  Every wait is bounded.
// On a timeout the CTA records an error, stops issuing, waits (bounded) for the copies
// and MMAs it already issued, frees its TMEM and returns; the epilogue leaves its loop
// only together (a barrier reduction), so no thread is left at a named barrier.
#pragma once

#include "lu_tc2.cuh"

namespace fde {

constexpr int W_STAGES = 4;
constexpr int WQ = 4;                    // tiles per CTA
constexpr int W_CROW = 64 * 4 + 16;      // bytes per staged half-row (64 floats + pad)
constexpr int W_CHALF = T2_BM * W_CROW;  // one plane of a staged half tile
constexpr int W_THREADS = 256;

template <int KIND>
struct Tc2w {
    static constexpr int STAGE = Tc2<KIND>::STAGE;  // A' re, A' im, B' chunk of one main-loop step
    static constexpr int RING = W_STAGES * STAGE;
    static constexpr int SMEM = RING + 2 * W_CHALF;
    static_assert(SMEM <= 227 * 1024, "ring + staged C half must fit one CTA");
};

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, 128;" ::: "memory"); }  // warps 4..7

__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// AND of v over the n threads of named barrier id (all of them must call it).
__device__ __forceinline__ bool named_and(int id, int n, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// Tiles x0 .. x0 + nq - 1 of the interior of one block: x -> (ti, tj) = (1 + x / ni, 1 + x % ni),
// ni = nt - 1 interior tiles per dimension; A' tile ti and B' tile tj of the step's
// packed operands (tile 0 of each belongs to the next panel's column / row).
template <int KIND>
__device__ __forceinline__ void tc2w_body(int mp, int R0, int ni, int x0, int nq, float* __restrict__ re_plane,
                                          const unsigned char* __restrict__ apack,
                                          const unsigned char* __restrict__ bpack, int* __restrict__ err) {
    using Cfg = Tc2<KIND>;
    using Wc = Tc2w<KIND>;
    constexpr int NS = W_STAGES;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* ring = smem;
    unsigned char* sCr = smem + Wc::RING;
    unsigned char* sCi = sCr + W_CHALF;
    __shared__ __align__(8) uint64_t full[NS], empty[NS], acc_full[2], acc_empty[2], c_full, mma_done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ long n_issued, n_taken;  // chunks the producer issued / the MMA issuer took
    __shared__ int c_pending;           // 1: C copies of the epilogue issued and not waited for
    __shared__ uint32_t c_phase_left;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* gre = re_plane;
    float* gim = re_plane + (size_t)mp * mp;
    auto tile_rc = [&](int q, int& r0, int& c0, int& ti, int& tj) {
        const int x = x0 + q;
        ti = 1 + x / ni;
        tj = 1 + x % ni;
        r0 = R0 + ti * T2_BM;
        c0 = R0 + tj * T2_BN;
    };
    auto fail = [&](int code) {
        abort_flag = 1;
        atomicCAS(err, 0, code);
    };

    if (warp == 1) tc::tmem_alloc(&tmem_base, 512);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&acc_full[a], 1);
            tc::mbar_init(&acc_empty[a], 4);  // one arrival per epilogue warp
        }
        tc::mbar_init(&c_full, 1);
        tc::mbar_init(&mma_done, 1);
        tc::fence_barrier_init();
        abort_flag = 0;
        n_issued = n_taken = 0;
        c_pending = 0;
        c_phase_left = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;

    if (warp == 0) {
        if (lane == 0) {  // producer
            long g = 0;
            for (int q = 0; q < nq && !abort_flag; ++q) {
                int r0, c0, ti, tj;
                tile_rc(q, r0, c0, ti, tj);
                const unsigned char* ga = apack + (size_t)ti * Cfg::A_TILE;
                const unsigned char* gb = bpack + (size_t)tj * Cfg::B_TILE;
                for (int c = 0; c < Cfg::NIT && !abort_flag; ++c) {
                    const int s = (int)(g % NS);
                    if (g >= NS && !tc::mbar_wait(&empty[s], (uint32_t)((g / NS - 1) & 1))) {
                        fail(1);
                        break;
                    }
                    const int kc = Cfg::re_chunk(c);
                    unsigned char* sa = ring + s * Wc::STAGE;
                    tc::mbar_arrive_expect_tx(&full[s], Wc::STAGE);
                    tc::bulk_g2s(sa, ga + (size_t)kc * Cfg::A_CHUNK, Cfg::A_CHUNK, &full[s]);
                    tc::bulk_g2s(sa + Cfg::A_CHUNK, ga + (size_t)(kc + Cfg::HALF) * Cfg::A_CHUNK, Cfg::A_CHUNK,
                                 &full[s]);
                    tc::bulk_g2s(sa + 2 * Cfg::A_CHUNK, gb + (size_t)c * Cfg::B_CHUNK, Cfg::B_CHUNK, &full[s]);
                    n_issued = ++g;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            long g = 0;
            for (int q = 0; q < nq && !abort_flag; ++q) {
                const int a = q & 1;
                if (q >= 2 && !tc::mbar_wait(&acc_empty[a], (uint32_t)(((q - 2) >> 1) & 1))) {
                    fail(2);
                    break;
                }
                tc::fence_after_sync();
                const uint32_t tacc = tbase + (uint32_t)a * 2u * T2_BN;
                for (int c = 0; c < Cfg::NIT; ++c) {
                    const int s = (int)(g % NS);
                    if (abort_flag || !tc::mbar_wait(&full[s], (uint32_t)((g / NS) & 1))) {
                        fail(1);
                        break;
                    }
                    n_taken = ++g;
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_u32(ring + s * Wc::STAGE);
                    cplx_mma_step<KIND>(tacc, a0, a0 + Cfg::A_CHUNK, a0 + 2 * Cfg::A_CHUNK, c == 0);
                    tc::mma_commit(&empty[s]);
                }
                if (abort_flag) break;
                tc::mma_commit(&acc_full[a]);
            }
            tc::mma_commit(&mma_done);  // tracks every MMA this thread issued
        }
    } else if (warp >= 4) {  // epilogue: thread r = tile row, TMEM lane quadrant warp - 4
        const int r = (warp - 4) * 32 + lane;
        const uint32_t lane_addr = (uint32_t)((warp - 4) * 32) << 16;
        uint32_t cphase = 0;
        bool stored = false;  // this thread's bulk stores may still be reading the staging rows
        bool ok = true;
        {  // the first tile's C rows towards L2
            int r0, c0, ti, tj;
            tile_rc(0, r0, c0, ti, tj);
            if (r < min(T2_BM, mp - r0)) {
                const uint32_t rb = (uint32_t)min(T2_BN, mp - c0) * 4;
                bulk_prefetch_l2(gre + (size_t)(r0 + r) * mp + c0, rb);
                bulk_prefetch_l2(gim + (size_t)(r0 + r) * mp + c0, rb);
            }
        }
        for (int q = 0; q < nq && ok; ++q) {
            int r0, c0, ti, tj;
            tile_rc(q, r0, c0, ti, tj);
            const int nrows = min(T2_BM, mp - r0), ncols = min(T2_BN, mp - c0);  // multiples of 64
            if (q + 1 < nq) {  // the next tile's C rows towards L2 while this one finishes
                int r1, c1, t1, u1;
                tile_rc(q + 1, r1, c1, t1, u1);
                if (r < min(T2_BM, mp - r1)) {
                    const uint32_t rb = (uint32_t)min(T2_BN, mp - c1) * 4;
                    bulk_prefetch_l2(gre + (size_t)(r1 + r) * mp + c1, rb);
                    bulk_prefetch_l2(gim + (size_t)(r1 + r) * mp + c1, rb);
                }
            }
            const int a = q & 1;
            bool mine = !abort_flag && tc::mbar_wait(&acc_full[a], (uint32_t)((q >> 1) & 1));
            ok = named_and(2, 128, mine);  // together or not at all
            if (!ok) {
                fail(2);
                break;
            }
            tc::fence_after_sync();
            for (int h = 0; h < 2 && h * 64 < ncols; ++h) {
                if (stored) bulk_wait_read_all();  // the staging rows are free again
                stored = false;
                epi_sync();  // every epilogue thread is done with the staging buffer
                if (warp == 4 && lane == 0) {
                    tc::mbar_arrive_expect_tx(&c_full, 2u * (uint32_t)nrows * 256u);
                    c_pending = 1;
                    c_phase_left = cphase;
                }
                epi_sync();
                if (r < nrows) {
                    tc::bulk_g2s(sCr + r * W_CROW, gre + (size_t)(r0 + r) * mp + c0 + h * 64, 256, &c_full);
                    tc::bulk_g2s(sCi + r * W_CROW, gim + (size_t)(r0 + r) * mp + c0 + h * 64, 256, &c_full);
                }
                mine = tc::mbar_wait(&c_full, cphase);
                ok = named_and(2, 128, mine);
                if (!ok) {
                    fail(2);
                    break;
                }
                if (warp == 4 && lane == 0) c_pending = 0;
                cphase ^= 1u;
                float4* cr = reinterpret_cast<float4*>(sCr + r * W_CROW);
                float4* ci = reinterpret_cast<float4*>(sCi + r * W_CROW);
                const uint32_t tre = tbase + lane_addr + (uint32_t)a * 2u * T2_BN + (uint32_t)h * 64u;
#pragma unroll 1
                for (int ch = 0; ch < 4; ++ch) {
                    float dr[16], di[16];
                    tc::tmem_ld16(tre + ch * 16, dr);
                    tc::tmem_ld16(tre + T2_BN + ch * 16, di);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float4 x = cr[ch * 4 + u], y = ci[ch * 4 + u];
                        x.x -= dr[4 * u]; x.y -= dr[4 * u + 1]; x.z -= dr[4 * u + 2]; x.w -= dr[4 * u + 3];
                        y.x -= di[4 * u]; y.y -= di[4 * u + 1]; y.z -= di[4 * u + 2]; y.w -= di[4 * u + 3];
                        cr[ch * 4 + u] = x;
                        ci[ch * 4 + u] = y;
                    }
                }
                fence_async_shared();
                if (r < nrows) {
                    bulk_s2g(gre + (size_t)(r0 + r) * mp + c0 + h * 64, sCr + r * W_CROW, 256);
                    bulk_s2g(gim + (size_t)(r0 + r) * mp + c0 + h * 64, sCi + r * W_CROW, 256);
                    bulk_commit();
                    stored = true;
                }
            }
            if (!ok) break;
            // the accumulator has been read: release it to the MMA issuer
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive_local(&acc_empty[a]);
        }
        if (stored) bulk_wait_read_all();
    }
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) {
        // bounded: let what was issued land before the CTA (and its TMEM) goes away
        for (long g = n_taken; g < n_issued; ++g) tc::mbar_wait(&full[g % NS], (uint32_t)((g / NS) & 1));
        if (c_pending) tc::mbar_wait(&c_full, c_phase_left);
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
