// Autotuner of launch shapes: for a kernel family and a problem shape it keeps the
// fastest of a few variants that compute bit-identical results (they differ only in
// how the work is spread over threads), measured with CUDA events on the GPU at
// first use and kept in a process-wide table that is also written to a text file
// (one line per shape) and read back by later processes.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>

#include <sys/stat.h>

#include "fde_internal.h"

namespace fde {

namespace {

struct TuneState {
    std::mutex mu;
    bool loaded = false;
    bool path_set = false;
    std::string path;                       // empty: no file
    int mode[FDE_TUNE_KERNELS] = {-1, -1, -1};  // -1 autotune, >= 0 forced variant
    std::map<std::tuple<int, int, int, int>, int> table;
};

TuneState& state() {
    static TuneState s;
    return s;
}

std::string default_path() {
    const char* env = std::getenv("FDE_TUNE_CACHE");
    if (env) return env;  // "" disables the file
    const char* home = std::getenv("HOME");
    return home ? std::string(home) + "/.cache/libfde_tune.txt" : std::string();
}

void load_locked(TuneState& s) {
    if (s.loaded) return;
    s.loaded = true;
    if (!s.path_set) s.path = default_path();
    if (s.path.empty()) return;
    FILE* f = std::fopen(s.path.c_str(), "r");
    if (!f) return;
    char line[512], name[32];
    int k, mp, nb, prec, v;
    while (std::fgets(line, sizeof line, f))  // "name kernel mp nb precision variant [# measured ms ...]"
        if (std::sscanf(line, "%31s %d %d %d %d %d", name, &k, &mp, &nb, &prec, &v) == 6 && k >= 0 &&
            k < FDE_TUNE_KERNELS && v >= 0 && v < tune_variants(k))
            s.table[{k, mp, nb, prec}] = v;
    std::fclose(f);
}

}  // namespace

int tune_variants(int kernel) {
    return kernel == FDE_TUNE_MATVEC ? 3 : kernel == FDE_TUNE_TRSV ? 4 : kernel == FDE_TUNE_LU ? 3 : 0;
}

// The variant used before a shape is measured (or when tuning is impossible): the
// 384 x 8 block-solve shape for FP32 factors (never slower than 512 x 4 where both were
// timed), the first variant otherwise.
// Built-in defaults: block solves with FP32 factors 384 x 8; the LU interior update with
// C streamed by tensor-map copies (its kernel falls back to row pairs where m_p is not a
// multiple of 128); everything else variant 0.
static int tune_default(int kernel, int prec) {
    if (kernel == FDE_TUNE_TRSV) return prec == FDE_FP32 ? 1 : 0;
    if (kernel == FDE_TUNE_LU) return 2;
    return 0;
}

int tune_lookup(int kernel, int mp, int nb, int prec, bool* need_tuning) {
    TuneState& s = state();
    std::lock_guard<std::mutex> lock(s.mu);
    load_locked(s);
    if (need_tuning) *need_tuning = false;
    if (s.mode[kernel] >= 0) return s.mode[kernel];
    auto it = s.table.find({kernel, mp, nb, prec});
    if (it != s.table.end()) return it->second;
    if (need_tuning) *need_tuning = true;
    return tune_default(kernel, prec);
}

int tune_default_variant(int kernel, int prec) { return tune_default(kernel, prec); }

void tune_store(int kernel, int mp, int nb, int prec, int variant, const float* ms) {
    TuneState& s = state();
    std::lock_guard<std::mutex> lock(s.mu);
    load_locked(s);
    s.table[{kernel, mp, nb, prec}] = variant;
    if (s.path.empty()) return;
    FILE* f = std::fopen(s.path.c_str(), "a");
    if (!f) {  // the cache directory may not exist yet: create its last level and retry
        const size_t slash = s.path.rfind('/');
        if (slash != std::string::npos && slash > 0) mkdir(s.path.substr(0, slash).c_str(), 0755);
        f = std::fopen(s.path.c_str(), "a");
        if (!f) return;  // the table stays in memory only
    }
    std::fprintf(f, "%s %d %d %d %d %d #", kernel == FDE_TUNE_MATVEC ? "matvec" : kernel == FDE_TUNE_TRSV ? "trsv" : "lu",
                 kernel, mp, nb, prec,
                 variant);
    for (int i = 0; ms && i < tune_variants(kernel); ++i) std::fprintf(f, " %.4f", ms[i]);
    std::fprintf(f, " ms\n");
    std::fclose(f);
}

// Time fn(variant) for every variant on stream st and return the fastest: one untimed
// launch of each, then five rounds that launch every variant once in turn (so that a
// drift of clocks or memory state during the measurement falls on all of them), the
// median of each variant's five times.  The fastest variant is taken if it beats the
// default by more than 2 % (launch-to-launch noise), else the default is kept.  fn launches one kernel and returns
// an FDE status.
int tune_measure(int kernel, cudaStream_t st, int (*fn)(void*, int, cudaStream_t), void* ctx, int* best,
                 float* ms_out, int default_variant, int nv_limit) {
    constexpr int ROUNDS = 5;
    const int nv = nv_limit > 0 && nv_limit < tune_variants(kernel) ? nv_limit : tune_variants(kernel);
    cudaEvent_t ev[2 * ROUNDS * TUNE_MAX_VARIANTS];
    int created = 0, rc = FDE_OK;
    for (; created < 2 * ROUNDS * nv; ++created)
        if (cudaEventCreate(&ev[created]) != cudaSuccess) {
            rc = cuda_error(cudaGetLastError(), "autotune events");
            break;
        }
    for (int v = 0; v < nv && !rc; ++v) rc = fn(ctx, v, st);
    for (int r = 0; r < ROUNDS && !rc; ++r)
        for (int v = 0; v < nv && !rc; ++v) {
            cudaEventRecord(ev[2 * (r * nv + v)], st);
            rc = fn(ctx, v, st);
            cudaEventRecord(ev[2 * (r * nv + v) + 1], st);
        }
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = cuda_error(cudaGetLastError(), "autotune");
    *best = default_variant;
    if (!rc) {
        float med[TUNE_MAX_VARIANTS];
        for (int v = 0; v < nv; ++v) {
            float t[ROUNDS];
            for (int r = 0; r < ROUNDS; ++r) {
                t[r] = 0.f;
                cudaEventElapsedTime(&t[r], ev[2 * (r * nv + v)], ev[2 * (r * nv + v) + 1]);
            }
            for (int a = 1; a < ROUNDS; ++a)  // insertion sort of five
                for (int b = a; b > 0 && t[b] < t[b - 1]; --b) std::swap(t[b], t[b - 1]);
            med[v] = t[ROUNDS / 2];
            if (ms_out) ms_out[v] = med[v];
        }
        int fastest = default_variant;
        for (int v = 0; v < nv; ++v)
            if (med[v] < med[fastest]) fastest = v;
        if (med[fastest] < 0.98f * med[default_variant]) *best = fastest;
    }
    for (int i = 0; i < created; ++i) cudaEventDestroy(ev[i]);
    return rc;
}

}  // namespace fde

using namespace fde;

extern "C" int fde_tune_set(int kernel, int variant) {
    if (kernel < 0 || kernel >= FDE_TUNE_KERNELS) return set_error(FDE_ERR_ARG, "unknown kernel family");
    if (variant < -1 || variant >= tune_variants(kernel)) return set_error(FDE_ERR_ARG, "variant out of range");
    TuneState& s = state();
    std::lock_guard<std::mutex> lock(s.mu);
    s.mode[kernel] = variant;
    return FDE_OK;
}

extern "C" int fde_tune_cache(const char* path) {
    TuneState& s = state();
    std::lock_guard<std::mutex> lock(s.mu);
    s.path_set = true;
    s.path = path ? path : "";
    s.table.clear();
    s.loaded = false;
    load_locked(s);
    return FDE_OK;
}

extern "C" int fde_tune_query(int kernel, int mp, int nb, int precision, int* variant) {
    if (kernel < 0 || kernel >= FDE_TUNE_KERNELS || !variant) return set_error(FDE_ERR_ARG, "bad argument");
    TuneState& s = state();
    std::lock_guard<std::mutex> lock(s.mu);
    load_locked(s);
    if (s.mode[kernel] >= 0) {
        *variant = s.mode[kernel];
        return FDE_OK;
    }
    auto it = s.table.find({kernel, mp, nb, precision});
    *variant = it == s.table.end() ? -1 : it->second;
    return FDE_OK;
}
