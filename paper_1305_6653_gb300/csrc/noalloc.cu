// fde_precond_apply_noalloc: the preconditioner apply z = S^{-1} r for callers
// that cannot allocate device memory when they call it.
//
// Its frequency-domain scratch (the s/2+1 transformed right-hand sides, solved
// in place) lives in a file-scope static device array instead of a buffer the
// library allocates.  The array is part of the library image: every GPU that
// loads the library holds it until the process exits.
#include <mutex>

#include "fde_internal.h"

namespace fde {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(8) << 20;  // 8 MiB

static __device__ __align__(256) unsigned char g_freq_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_freq_scratch on the current device.  In host code the
// array's name only stands for a host-side shadow, so the address is looked up
// once per device (with that device current) and cached.
static int scratch_address(void** out) {
    static std::mutex mu;
    static void* addr[256] = {};
    int dev = 0;
    FDE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return set_error(FDE_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_freq_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_freq_scratch)");
        addr[dev] = p;
    }
    *out = addr[dev];
    return FDE_OK;
}

}  // namespace fde

using namespace fde;

extern "C" int fde_precond_apply_noalloc(fde_problem* h, const double* r, double* z) {
    set_error(FDE_OK, "");
    if (!h || !r || !z) return set_error(FDE_ERR_ARG, "NULL argument");
    Problem& P = *problem_of(h);
    // The state comes first: the scratch size depends on the precision of the factors.
    if (!P.factored || P.precond != FDE_PRECOND_STRANG)
        return set_error(FDE_ERR_STATE, "strang_precond_factor must run first");
    const size_t esz = P.precision == FDE_FP64 ? sizeof(double) : sizeof(float);
    const size_t need = (size_t)P.nblk * P.mp * 2 * esz;
    if (need > NOALLOC_SCRATCH_BYTES)
        return set_error(FDE_ERR_ARG, "fde_precond_apply_noalloc: (s/2+1) * mp complex values exceed the 8 MiB "
                                      "static scratch; use fde_precond_apply");
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    // The forward transform writes every entry that the block solves and the
    // inverse transform read, so nothing needs clearing between calls.
    if ((rc = launch_time_fft_fwd(P, r, scratch, P.precision, P.stream))) return rc;
    if ((rc = launch_block_trsv(P, scratch, P.stream))) return rc;
    return launch_time_fft_inv(P, scratch, z, P.precision, P.stream);
}
