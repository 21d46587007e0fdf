// Batched solve of many independent problems (uneven m, s, alpha, d and BVM
// scheme) with one set of kernel launches per step for the whole batch.
//
// Each instance keeps its own buffers (it is an ordinary fde_problem); the batch
// adds device descriptor tables (InstDev per instance, BlkDev per Strang block)
// that the batched kernels index by blockIdx.y:
//   * LU: the block table of every instance, sorted by m_p, so the blocks still
//     being factored at step p are a prefix of the table (one launch per kernel
//     and step for the whole batch);
//   * GMRES: flexible GMRES(restart) in lock-stepped restart rounds.  Within a
//     round all active instances take iteration j together; an instance whose
//     residual estimate meets the tolerance drops out of the active list (its
//     kernels are no longer launched) until the round ends; then every instance
//     of the round forms x += Z y and its true FP64 residual, and the unconverged
//     ones start the next round.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "fde_internal.h"

using namespace fde;

#include <cstdio>

struct fde_batch {
    std::vector<fde_problem*> probs;
    cudaStream_t stream = nullptr;
    int precision = -1;
    bool assembled = false, factored = false;
    BlkDev* d_blk = nullptr;
    std::vector<int> blk_mp;
    InstDev* d_inst = nullptr;
    int* d_act = nullptr;
    int* d_kvec = nullptr;
    int* d_err = nullptr;
    double* d_gather = nullptr;
    double* h_gather = nullptr;  // pinned
    int* h_act = nullptr;        // pinned
    int* h_kvec = nullptr;       // pinned
    unsigned char* d_pack = nullptr;
    size_t pack_bytes = 0;
    int max_mp = 0, max_s = 0, max_L = 0, max_m = 0, max_nblk = 0;
    long max_n = 0;
    // many right-hand sides of one operator (fde_batch_share_operator): instance 0
    // holds the only factors; every instance solves against them with its own
    // frequency-side vectors
    bool shared = false;
    void* d_rhat_shared = nullptr;  // count * nblk * mp complex FP32
    int block_solver = FDE_BLOCK_SOLVE_AUTO;  // fde_batch_block_solver
    bool trsm_tc = false;                     // the factorisation kept what the tensor-core block solves need
    // batched GMRES: per-instance control words (InstDev::ctl, 4 ints each) and their
    // host copy; restart cycles captured as CUDA graphs, keyed by the cycle's shape
    int* d_ctl = nullptr;
    int* h_ctl = nullptr;  // pinned
    cudaStream_t cap_stream = nullptr;
    std::map<std::string, std::pair<cudaGraphExec_t, long long>> cycle_graphs;  // key -> (graph, kernels)
};

namespace {

int upload_list(fde_batch* b, const std::vector<int>& v, int* host, int* dev) {
    if (v.empty()) return FDE_OK;
    std::memcpy(host, v.data(), v.size() * sizeof(int));
    FDE_CUDA_TRY(cudaMemcpyAsync(dev, host, v.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    return FDE_OK;
}

int gather(fde_batch* b) {
    const int n = (int)b->probs.size();
    int rc = launch_gather_scalars(b->d_inst, n, b->d_gather, b->stream);
    if (rc) return rc;
    FDE_CUDA_TRY(cudaMemcpyAsync(b->h_gather, b->d_gather, 4 * n * sizeof(double), cudaMemcpyDeviceToHost,
                                 b->stream));
    FDE_CUDA_TRY(cudaStreamSynchronize(b->stream));
    return FDE_OK;
}

// One restart cycle of the batched flexible GMRES for the nr instances of the current
// round list (b->d_act): iterations j = 0..restart-1, each a fixed sequence of launches
// over the whole round.  An instance that meets its tolerance (or maxit, a breakdown,
// a non-finite value) has its live flag cleared by finish_batched on the device, and
// every later kernel of the cycle skips it; nothing returns to the host until the
// cycle is over.
int cycle_launches(fde_batch* b, int nr, const fde_pgmres_opts& o, cudaStream_t st) {
    const int ldh = o.restart + 1;
    int rc;
    for (int j = 0; j < o.restart; ++j) {
        if ((rc = launch_time_fft_batched(b->d_inst, b->d_act, nr, b->max_mp, b->max_s, j, st))) return rc;
        // shared operator: groups of right-hand sides per CTA, each factor plane streamed once per group
        if (b->shared && b->trsm_tc) {
            const Problem& P0 = *problem_of(b->probs[0]);
            rc = launch_trsm_tc(b->d_inst, b->d_act, nr, P0.d_fac, P0.d_dtile, P0.mp, P0.nblk, b->d_err, st);
        } else if (b->shared) {
            rc = launch_trsv_multi(b->d_inst, b->d_act, nr, b->max_nblk, b->max_mp, st);
        } else {
            rc = launch_trsv_batched(b->d_inst, b->d_act, nr, b->max_nblk, b->max_mp, st);
        }
        if (rc) return rc;
        if ((rc = launch_time_ifft_batched(b->d_inst, b->d_act, nr, b->max_mp, b->max_s, j, st))) return rc;
        if ((rc = launch_matvec_batched(b->d_inst, b->d_act, nr, b->max_s, b->max_L, b->max_m, 0, j, st))) return rc;
        if ((rc = launch_dots_batched(b->d_inst, b->d_act, nr, 0, j, st))) return rc;
        if ((rc = launch_update_batched(b->d_inst, b->d_act, nr, 0, j, b->d_kvec, b->max_n, st))) return rc;
        if (o.reorth) {
            if ((rc = launch_dots_batched(b->d_inst, b->d_act, nr, 1, j, st))) return rc;
            if ((rc = launch_update_batched(b->d_inst, b->d_act, nr, 1, j, b->d_kvec, b->max_n, st))) return rc;
        }
        if ((rc = launch_dots_batched(b->d_inst, b->d_act, nr, 2, j, st))) return rc;
        if ((rc = launch_finish_batched(b->d_inst, b->d_act, nr, j, ldh, o.reorth, o.tol, o.maxit, st))) return rc;
        if ((rc = launch_scale_batched(b->d_inst, b->d_act, nr, 0, j, o.restart, b->max_n, st))) return rc;
    }
    return FDE_OK;
}

// Run the cycle: replay its CUDA graph (captured on first use for this shape: round
// size, restart, re-orthogonalisation, tolerance and maxit, which enter as kernel
// arguments; the round list itself is read from device memory when the graph runs).
int run_cycle(fde_batch* b, int nr, const fde_pgmres_opts& o, cudaStream_t st) {
    char key[128];
    std::snprintf(key, sizeof key, "%d/%d/%d/%a/%d", nr, o.restart, o.reorth, o.tol, o.maxit);
    auto it = b->cycle_graphs.find(key);
    if (it == b->cycle_graphs.end()) {
        if (!b->cap_stream) FDE_CUDA_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        const long long l0 = fde_launch_count();
        cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamBeginCapture");
        int rc = cycle_launches(b, nr, o, b->cap_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
        const long long k = fde_launch_count() - l0;
        note_launches(-k);  // counted once while capturing; each replay adds them below
        it = b->cycle_graphs.emplace(key, std::make_pair(exec, k)).first;
    }
    FDE_CUDA_TRY(cudaGraphLaunch(it->second.first, st));
    note_launches(it->second.second);
    return FDE_OK;
}

}  // namespace

extern "C" {

void fde_batch_destroy(fde_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    for (fde_problem* p : b->probs) fde_problem_destroy(p);
    void* dev[] = {b->d_blk, b->d_inst, b->d_act, b->d_kvec, b->d_err, b->d_gather, b->d_pack,
                   b->d_rhat_shared};
    for (void* d : dev)
        if (d) cudaFree(d);
    if (b->h_gather) cudaFreeHost(b->h_gather);
    if (b->h_act) cudaFreeHost(b->h_act);
    if (b->h_kvec) cudaFreeHost(b->h_kvec);
    if (b->d_ctl) cudaFree(b->d_ctl);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    for (auto& kv : b->cycle_graphs) cudaGraphExecDestroy(kv.second.first);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

int fde_batch_create(const fde_problem_desc* descs, int count, void* stream, fde_batch** out) {
    if (!descs || !out || count < 1) return set_error(FDE_ERR_ARG, "need descs, out and count >= 1");
    *out = nullptr;
    fde_batch* b = new (std::nothrow) fde_batch();
    if (!b) return set_error(FDE_ERR_ALLOC, "host allocation failed");
    b->stream = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i) {
        if (descs[i].dplus_t || descs[i].dminus_t) {
            fde_batch_destroy(b);
            return set_error(FDE_ERR_ARG, std::string("instance ") + std::to_string(i) +
                                              ": time-dependent coefficients are not batched");
        }
        fde_problem* p = nullptr;
        int rc = fde_problem_create(&descs[i], stream, &p);
        if (rc) {
            std::string msg = std::string("instance ") + std::to_string(i) + ": " + fde_last_error();
            fde_batch_destroy(b);
            return set_error(rc, msg);
        }
        b->probs.push_back(p);
        const Problem& P = *problem_of(p);
        b->max_mp = std::max(b->max_mp, P.mp);
        b->max_s = std::max(b->max_s, P.s);
        b->max_L = std::max(b->max_L, P.L);
        b->max_m = std::max(b->max_m, P.m);
        b->max_nblk = std::max(b->max_nblk, P.nblk);
        b->max_n = std::max(b->max_n, P.n);
    }
    bool ok = cudaMalloc(&b->d_act, count * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&b->d_kvec, count * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&b->d_err, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&b->d_gather, 4 * count * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&b->d_inst, count * sizeof(InstDev)) == cudaSuccess &&
              cudaMallocHost(&b->h_gather, 4 * count * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&b->h_act, count * sizeof(int)) == cudaSuccess &&
              cudaMallocHost(&b->h_kvec, count * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&b->d_ctl, 4 * count * sizeof(int)) == cudaSuccess &&
              cudaMallocHost(&b->h_ctl, 4 * count * sizeof(int)) == cudaSuccess;
    if (!ok) {
        fde_batch_destroy(b);
        return set_error(FDE_ERR_ALLOC, "batch allocation failed");
    }
    *out = b;
    return FDE_OK;
}

int fde_batch_share_operator(fde_batch* b) {
    if (!b) return set_error(FDE_ERR_ARG, "NULL batch");
    if (b->factored) return set_error(FDE_ERR_STATE, "fde_batch_share_operator must run before fde_batch_factor");
    const Problem& P0 = *problem_of(b->probs[0]);
    std::vector<double> d0(2 * (size_t)P0.m), di(2 * (size_t)P0.m);
    FDE_CUDA_TRY(cudaMemcpy(d0.data(), P0.d_dplus, P0.m * sizeof(double), cudaMemcpyDeviceToHost));
    FDE_CUDA_TRY(cudaMemcpy(d0.data() + P0.m, P0.d_dminus, P0.m * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t i = 1; i < b->probs.size(); ++i) {
        const Problem& P = *problem_of(b->probs[i]);
        const bool same = P.m == P0.m && P.s == P0.s && P.mu == P0.mu && P.family == P0.family &&
                          P.alpha == P0.alpha && P.xL == P0.xL && P.xR == P0.xR && P.t0 == P0.t0 && P.T == P0.T;
        if (!same)
            return set_error(FDE_ERR_ARG, "instance " + std::to_string(i) + " has another operator (m, s, alpha, "
                                          "interval or BVM scheme)");
        FDE_CUDA_TRY(cudaMemcpy(di.data(), P.d_dplus, P.m * sizeof(double), cudaMemcpyDeviceToHost));
        FDE_CUDA_TRY(cudaMemcpy(di.data() + P.m, P.d_dminus, P.m * sizeof(double), cudaMemcpyDeviceToHost));
        if (di != d0)
            return set_error(FDE_ERR_ARG, "instance " + std::to_string(i) + " has other coefficients d+, d-");
    }
    b->shared = true;
    return FDE_OK;
}

int fde_batch_block_solver(fde_batch* b, int solver) {
    if (!b) return set_error(FDE_ERR_ARG, "NULL batch");
    if (solver != FDE_BLOCK_SOLVE_AUTO && solver != FDE_BLOCK_SOLVE_CUDA_CORES &&
        solver != FDE_BLOCK_SOLVE_TENSOR_CORES)
        return set_error(FDE_ERR_ARG, "unknown block solver");
    if (b->factored) return set_error(FDE_ERR_STATE, "fde_batch_block_solver must run before fde_batch_factor");
    b->block_solver = solver;
    return FDE_OK;
}

int fde_batch_size(const fde_batch* b) { return b ? (int)b->probs.size() : 0; }

fde_problem* fde_batch_problem(fde_batch* b, int i) {
    if (!b || i < 0 || i >= (int)b->probs.size()) return nullptr;
    return b->probs[i];
}

int fde_batch_assemble(fde_batch* b) {
    if (!b) return set_error(FDE_ERR_ARG, "NULL batch");
    for (size_t i = 0; i < b->probs.size(); ++i) {
        int rc = bvm_assemble(b->probs[i]);
        if (rc) return rc;
    }
    b->assembled = true;
    return FDE_OK;
}

int fde_batch_factor(fde_batch* b, int precision) {
    if (!b) return set_error(FDE_ERR_ARG, "NULL batch");
    if (!b->assembled) return set_error(FDE_ERR_STATE, "fde_batch_assemble must run first");
    if (precision != FDE_FP32 && precision != FDE_TF32 && precision != FDE_BF16 && precision != FDE_TF32X3)
        return set_error(FDE_ERR_ARG, "batched factorisation supports FDE_FP32, FDE_TF32, FDE_BF16 and FDE_TF32X3");
    // the captured cycles hold the block-solve kernel and factor layout of the last
    // factorisation (an executable graph still in flight is freed when it completes)
    for (auto& kv : b->cycle_graphs) cudaGraphExecDestroy(kv.second.first);
    b->cycle_graphs.clear();
    if (b->shared) {
        // one factorisation (the single-problem path: look-ahead tensor-core LU), used by all;
        // for the tensor-core block solves it also keeps the inverted diagonal blocks
        Problem& P0w = *problem_of(b->probs[0]);
        const bool tc = b->shared && b->block_solver != FDE_BLOCK_SOLVE_CUDA_CORES && precision == FDE_TF32 &&
                        trsm_tc_supported(P0w.mp);
        if (b->block_solver == FDE_BLOCK_SOLVE_TENSOR_CORES && !tc)
            return set_error(FDE_ERR_ARG, "tensor-core block solves need FDE_TF32 factors and 256 <= m_p <= 2048");
        P0w.save_dtile = tc;
        P0w.want_strips = false;  // the shared-operator block solves read the factor planes
        b->trsm_tc = false;
        int rc = strang_precond_factor(b->probs[0], precision);
        P0w.save_dtile = false;
        P0w.want_strips = true;
        if (rc) return rc;
        b->trsm_tc = tc && P0w.d_dtile != nullptr;
        const Problem& P0 = P0w;
        const size_t per = (size_t)P0.nblk * P0.mp * 2 * sizeof(float);
        if (!b->d_rhat_shared) FDE_CUDA_TRY(cudaMalloc(&b->d_rhat_shared, per * b->probs.size()));
        FDE_CUDA_TRY(cudaMemsetAsync(b->d_rhat_shared, 0, per * b->probs.size(), b->stream));
        for (fde_problem* p : b->probs) {
            problem_of(p)->factored = true;
            problem_of(p)->precision = precision;
        }
        b->precision = precision;
        b->factored = true;
        return FDE_OK;
    }
    const int kind = precision == FDE_FP32 ? -1 : 0;  // >= 0: tensor-core path with packed operands
    // buffers and the block table
    std::vector<BlkDev> blks;
    size_t pack_total = 0;
    for (size_t i = 0; i < b->probs.size(); ++i) {
        Problem& P = *problem_of(b->probs[i]);
        int rc = ensure_factor_buffers(P, precision);
        if (rc) return rc;
        P.factored = false;
        P.precision = precision;
        // an instance set to FDE_STORAGE_BF16 (tensor-core LU, m_p a multiple of 128) gets the
        // bfloat16 strip-major copy of its factors for the block solves; without the memory
        // for it, its solves read the planes
        P.strips_ok = false;
        unsigned short* strips = nullptr;
        if (kind >= 0 && P.strip_storage == FDE_STORAGE_BF16 && P.mp % 128 == 0) {
            const size_t sneed = (size_t)P.nblk * 2 * P.mp * P.mp * sizeof(unsigned short);
            if (P.strips_bytes < sneed) {
                if (P.d_strips) {
                    FDE_CUDA_TRY(cudaStreamSynchronize(b->stream));
                    dev_free(P.d_strips);
                }
                P.d_strips = nullptr;
                P.strips_bytes = 0;
                if (dev_alloc(&P.d_strips, sneed) == FDE_OK) P.strips_bytes = sneed;
                else set_error(FDE_OK, "");
            }
            strips = static_cast<unsigned short*>(P.d_strips);
        }
        P.strips_bf16 = strips != nullptr;
        const size_t pack_a = tc_pack_a_bytes_per_block(precision, P.mp);
        const size_t pack_all = tc_pack_bytes_per_block(precision, P.mp);
        for (int k = 0; k < P.nblk; ++k) {
            BlkDev d{};
            d.inst = (int)i;
            d.k = k;
            d.m = P.m;
            d.mp = P.mp;
            d.ntile_max = (int)pack_a;  // bytes of this block's A' tiles (B' tiles follow)
            d.h = P.h;
            d.dxa = P.dxa;
            d.phi = P.d_phi + k;
            d.psi = P.d_psi + k;
            d.g = P.d_g;
            d.dplus = P.d_dplus;
            d.dminus = P.d_dminus;
            d.fac = (float*)P.d_fac + (size_t)k * 2 * P.mp * P.mp;
            d.dinv = (float2*)P.d_dinv + (size_t)k * P.mp;
            d.info = P.d_info + k;
            d.strips = strips ? strips + (size_t)k * 2 * P.mp * P.mp : nullptr;
            if (kind >= 0) {
                d.apack = (unsigned char*)pack_total;  // offset, rebased below
                pack_total += pack_all;
            }
            blks.push_back(d);
        }
        FDE_CUDA_TRY(cudaMemsetAsync(P.d_info, 0, P.nblk * sizeof(int), b->stream));
    }
    if (kind >= 0 && b->pack_bytes < pack_total) {
        if (b->d_pack) cudaFree(b->d_pack);
        b->d_pack = nullptr;
        b->pack_bytes = 0;
        FDE_CUDA_TRY(cudaMalloc(&b->d_pack, pack_total));
        b->pack_bytes = pack_total;
        FDE_CUDA_TRY(cudaMemsetAsync(b->d_pack, 0, pack_total, b->stream));
    }
    if (kind >= 0) {
        for (BlkDev& d : blks) {
            const size_t off = (size_t)d.apack;
            d.apack = b->d_pack + off;
            d.bpack = d.apack + (size_t)d.ntile_max;
            d.ipack = d.bpack + tc_pack_b_bytes_per_block(precision, d.mp);
        }
    }
    std::stable_sort(blks.begin(), blks.end(), [](const BlkDev& a, const BlkDev& c) { return a.mp > c.mp; });
    b->blk_mp.resize(blks.size());
    for (size_t i = 0; i < blks.size(); ++i) b->blk_mp[i] = blks[i].mp;
    if (b->d_blk) cudaFree(b->d_blk);
    b->d_blk = nullptr;
    FDE_CUDA_TRY(cudaMalloc(&b->d_blk, blks.size() * sizeof(BlkDev)));
    FDE_CUDA_TRY(cudaMemcpyAsync(b->d_blk, blks.data(), blks.size() * sizeof(BlkDev), cudaMemcpyHostToDevice,
                                 b->stream));
    FDE_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
    int rc = launch_lu_batched(b->d_blk, b->blk_mp, precision, b->d_err, b->stream);
    if (rc) return rc;
    // pivots and bounded waits
    int derr = 0;
    FDE_CUDA_TRY(cudaMemcpyAsync(&derr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    std::vector<std::vector<int>> infos(b->probs.size());
    for (size_t i = 0; i < b->probs.size(); ++i) {
        Problem& P = *problem_of(b->probs[i]);
        infos[i].resize(P.nblk);
        FDE_CUDA_TRY(cudaMemcpyAsync(infos[i].data(), P.d_info, P.nblk * sizeof(int), cudaMemcpyDeviceToHost,
                                     b->stream));
    }
    FDE_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (derr) return set_error(FDE_ERR_TIMEOUT, "a bounded wait in the tensor-core LU update ran out");
    for (size_t i = 0; i < b->probs.size(); ++i)
        for (int k = 0; k < (int)infos[i].size(); ++k)
            if (infos[i][k])
                return set_error(FDE_ERR_SINGULAR, "zero or non-finite pivot in instance " + std::to_string(i) +
                                                       ", block " + std::to_string(k));
    // the FP32 inverses of the diagonal tiles, through which the solves from a bfloat16 copy
    // apply the diagonal tiles
    for (fde_problem* p : b->probs) {
        Problem& P = *problem_of(p);
        if (!P.strips_bf16) continue;
        if ((rc = launch_tile_inverse_fp32(P, b->stream))) return rc;
        P.strips_ok = true;
    }
    for (fde_problem* p : b->probs) problem_of(p)->factored = true;
    b->precision = precision;
    b->factored = true;
    return FDE_OK;
}

int fde_batch_solve(fde_batch* b, const fde_pgmres_opts* opts, double* const* x_out, fde_stats* stats) {
    if (!b || !x_out) return set_error(FDE_ERR_ARG, "NULL argument");
    if (!b->factored) return set_error(FDE_ERR_STATE, "fde_batch_factor must run first");
    fde_pgmres_opts o{1e-10, 20, 1000, 1};
    if (opts) o = *opts;
    if (!(o.tol > 0.0) || o.restart < 1 || o.restart > 63 || o.maxit < 1)
        return set_error(FDE_ERR_ARG, "need tol > 0, 1 <= restart <= 63, maxit >= 1");
    const int n = (int)b->probs.size();
    cudaStream_t st = b->stream;
    cudaEvent_t ev0, ev1;
    FDE_CUDA_TRY(cudaEventCreate(&ev0));
    FDE_CUDA_TRY(cudaEventCreate(&ev1));
    FDE_CUDA_TRY(cudaEventRecord(ev0, st));
    std::vector<InstDev> inst(n);
    for (int i = 0; i < n; ++i) {
        if (!x_out[i]) return set_error(FDE_ERR_ARG, "x_out has a NULL entry");
        Problem& P = *problem_of(b->probs[i]);
        int rc = ensure_workspace(P, o.restart);
        if (rc) return rc;
        InstDev d{};
        d.m = P.m; d.s = P.s; d.mp = P.mp; d.L = P.L; d.logL = P.logL; d.logs = P.logs; d.mu = P.mu;
        d.nblk = P.nblk; d.n = P.n; d.h = P.h; d.dxa = P.dxa;
        d.start = P.d_start; d.A = P.d_a; d.B = P.d_b; d.dplus = P.d_dplus; d.dminus = P.d_dminus;
        d.sym = P.d_sym; d.twL = P.d_twL; d.tws32 = P.d_tws32; d.tws = P.d_tws;
        if (b->shared) {  // the factors of instance 0, frequency vectors of its own
            const Problem& P0 = *problem_of(b->probs[0]);
            d.fac = P0.d_fac;
            d.dinv = P0.d_dinv;
            d.tinv = P0.d_tinv;
            d.rhat = (unsigned char*)b->d_rhat_shared + (size_t)i * P0.nblk * P0.mp * 2 * sizeof(float);
        } else {
            d.rhat = P.d_rhat; d.fac = P.d_fac; d.dinv = P.d_dinv; d.tinv = nullptr;
            if (P.strips_ok && P.strips_bf16 && P.d_strips) {  // the bfloat16 copy and the tile inverses
                d.strips = P.d_strips;
                d.tinv = P.d_tinv;
            }
        }
        // host solution arrays (the instance's desc->device_ptrs == 0): solve into the
        // instance's device copy, copied out when the batch is done
        double* xd = x_out[i];
        if (!P.device_ptrs) {
            if ((rc = ensure_solution_buffer(P))) return rc;
            xd = P.d_xsol;
        }
        d.b = P.d_b_rhs; d.x = xd; d.V = P.d_V; d.Z = P.d_Z; d.work = P.d_work; d.H = P.d_H;
        d.cs = P.d_cs; d.sn = P.d_sn; d.gv = P.d_gv; d.y = P.d_y; d.scal = P.d_scal;
        d.partial = P.d_partial; d.counter = P.d_counter;
        d.ctl = b->d_ctl + 4 * i;
        inst[i] = d;
        FDE_CUDA_TRY(cudaMemsetAsync(xd, 0, P.n * sizeof(double), st));
    }
    FDE_CUDA_TRY(cudaMemcpyAsync(b->d_inst, inst.data(), n * sizeof(InstDev), cudaMemcpyHostToDevice, st));
    FDE_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), st));  // bounded waits of the block solves
    const int ldh = o.restart + 1;
    std::vector<int> all(n);
    std::iota(all.begin(), all.end(), 0);
    int rc;
    auto fail = [&](int code) {
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        return code;
    };
    // r_0 = b - M x_0 (x_0 = 0) into V_0, |b|^2 and |r_0|^2
    if ((rc = upload_list(b, all, b->h_act, b->d_act))) return fail(rc);
    if ((rc = launch_ctl_set_batched(b->d_inst, b->d_act, n, 1, 2, st))) return fail(rc);
    if ((rc = launch_matvec_batched(b->d_inst, b->d_act, n, b->max_s, b->max_L, b->max_m, 1, 0, st))) return fail(rc);
    if ((rc = launch_residual_batched(b->d_inst, b->d_act, n, b->max_n, st))) return fail(rc);
    if ((rc = launch_dots_batched(b->d_inst, b->d_act, n, 4, 0, st))) return fail(rc);
    if ((rc = launch_dots_batched(b->d_inst, b->d_act, n, 3, 0, st))) return fail(rc);
    std::vector<double> bnorm(n), beta(n), est(n, 0.0);
    // |b|^2 sits in scal[131]; gather it through a one-off copy per instance
    for (int i = 0; i < n; ++i) {
        Problem& P = *problem_of(b->probs[i]);
        FDE_CUDA_TRY(cudaMemcpyAsync(b->h_gather + 4 * i, P.d_scal + 131, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    FDE_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) bnorm[i] = std::sqrt(b->h_gather[4 * i]);
    if ((rc = gather(b))) return fail(rc);
    for (int i = 0; i < n; ++i) beta[i] = std::sqrt(b->h_gather[4 * i + 3]);
    std::vector<int> its(n, 0), restarts(n, 0), status(n, FDE_OK), kk(n, 0);
    std::vector<char> done(n, 0);
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(beta[i]) || !std::isfinite(bnorm[i])) { status[i] = FDE_ERR_NAN; done[i] = 1; }
        else if (bnorm[i] == 0.0 || beta[i] <= o.tol * bnorm[i]) done[i] = 1;
    }
    for (;;) {
        // a restart round: every unconverged instance runs one cycle of up to `restart`
        // Arnoldi steps, leaving it on the device as soon as its estimate meets the tolerance
        std::vector<int> round;
        for (int i = 0; i < n; ++i)
            if (!done[i]) round.push_back(i);
        if (round.empty()) break;
        const int nr = (int)round.size();
        if ((rc = upload_list(b, round, b->h_act, b->d_act))) return fail(rc);
        if ((rc = launch_ctl_set_batched(b->d_inst, b->d_act, nr, 1, 1, st))) return fail(rc);
        if ((rc = launch_scale_batched(b->d_inst, b->d_act, nr, 1, 0, o.restart, b->max_n, st))) return fail(rc);
        if ((rc = run_cycle(b, nr, o, st))) return fail(rc);
        FDE_CUDA_TRY(cudaMemcpyAsync(b->h_ctl, b->d_ctl, 4 * n * sizeof(int), cudaMemcpyDeviceToHost, st));
        if ((rc = gather(b))) return fail(rc);  // synchronises
        for (int i : round) {
            const int* c = b->h_ctl + 4 * i;
            kk[i] = c[1];
            its[i] = c[2];
            est[i] = b->h_gather[4 * i + 1];
            if (c[3]) status[i] = FDE_ERR_NAN;
        }
        // end of the round: x += Z y, true residual
        std::vector<int> upd;
        for (int i : round)
            if (status[i] == FDE_OK && kk[i] > 0) upd.push_back(i);
        for (int i : round)
            if (status[i] != FDE_OK) done[i] = 1;
        if (upd.empty()) continue;
        const int nu = (int)upd.size();
        for (int i = 0; i < n; ++i) b->h_kvec[i] = kk[i];
        FDE_CUDA_TRY(cudaMemcpyAsync(b->d_kvec, b->h_kvec, n * sizeof(int), cudaMemcpyHostToDevice, st));
        if ((rc = upload_list(b, upd, b->h_act, b->d_act))) return fail(rc);
        if ((rc = launch_ctl_set_batched(b->d_inst, b->d_act, nu, 1, 0, st))) return fail(rc);
        if ((rc = launch_lsq_batched(b->d_inst, b->d_act, nu, b->d_kvec, ldh, st))) return fail(rc);
        if ((rc = launch_update_batched(b->d_inst, b->d_act, nu, 2, 0, b->d_kvec, b->max_n, st))) return fail(rc);
        if ((rc = launch_matvec_batched(b->d_inst, b->d_act, nu, b->max_s, b->max_L, b->max_m, 1, 0, st)))
            return fail(rc);
        if ((rc = launch_residual_batched(b->d_inst, b->d_act, nu, b->max_n, st))) return fail(rc);
        if ((rc = launch_dots_batched(b->d_inst, b->d_act, nu, 3, 0, st))) return fail(rc);
        if ((rc = gather(b))) return fail(rc);
        for (int i : upd) {
            ++restarts[i];
            beta[i] = std::sqrt(b->h_gather[4 * i + 3]);
            if (!std::isfinite(beta[i])) {
                status[i] = FDE_ERR_NAN;
                done[i] = 1;
            } else if (beta[i] <= o.tol * bnorm[i]) {
                done[i] = 1;
            } else if (its[i] >= o.maxit) {
                status[i] = FDE_ERR_NOT_CONVERGED;
                done[i] = 1;
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        const Problem& P = *problem_of(b->probs[i]);
        if (!P.device_ptrs)
            FDE_CUDA_TRY(cudaMemcpyAsync(x_out[i], P.d_xsol, P.n * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    int derr = 0;
    FDE_CUDA_TRY(cudaMemcpyAsync(&derr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    FDE_CUDA_TRY(cudaEventRecord(ev1, st));
    FDE_CUDA_TRY(cudaEventSynchronize(ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (derr) return set_error(FDE_ERR_TIMEOUT, "a bounded wait of the block solves timed out");
    int worst = FDE_OK;
    for (int i = 0; i < n; ++i) {
        if (stats) {
            fde_stats& S = stats[i];
            std::memset(&S, 0, sizeof S);
            S.status = status[i];
            S.iterations = its[i];
            S.restarts = restarts[i];
            S.precision = b->precision;
            S.rel_residual = bnorm[i] > 0 ? beta[i] / bnorm[i] : 0.0;
            S.rel_residual_estimate = bnorm[i] > 0 ? est[i] / bnorm[i] : 0.0;
            S.ms_solve = ms;
        }
        if (status[i] != FDE_OK && worst == FDE_OK) worst = status[i];
    }
    if (worst == FDE_ERR_NOT_CONVERGED) return set_error(worst, "some instances reached maxit");
    if (worst == FDE_ERR_NAN) return set_error(worst, "non-finite residual in some instance");
    return FDE_OK;
}

}  // extern "C"
