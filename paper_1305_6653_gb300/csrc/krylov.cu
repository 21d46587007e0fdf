// FP64 Krylov kernels of the flexible GMRES(restart) iteration (Sec. 3.2 cites
// Saad's GMRES; Sec. 4 runs GMRES(20)): classical Gram-Schmidt with one
// re-orthogonalisation (CGS2) as multi-dot / multi-axpy passes over the basis V,
// the Givens least-squares update, and small vector kernels.
//
// Reductions are deterministic: every CTA writes its partial sums, and the last
// CTA to finish (atomic ticket after a fence; nothing waits) adds them in a fixed
// order (one warp per vector, lanes over the partials, then a shuffle tree) and
// resets the ticket.
#include <algorithm>

#include "fde_internal.h"

namespace fde {

constexpr int RED_CTAS = 304;  // 2 per SM on 152 SMs
constexpr int RED_THREADS = 256;
constexpr int KMAX = 64;       // max Krylov vectors per multi-dot

// Per-thread partial sums acc[0..k) -> out[0..k): each CTA stores its partials,
// and the last CTA to finish adds them in a fixed order.
template <int KC>
__device__ __forceinline__ void reduce_partials(const double (&acc)[KC], int k, double* __restrict__ out,
                                                double* __restrict__ partial, unsigned int* __restrict__ counter,
                                                int bx, int nblocks) {
    __shared__ double red[RED_THREADS / 32][KC];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < KC; ++i) {
        double v = acc[i];
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double v = 0.0;
        for (int q = 0; q < RED_THREADS / 32; ++q) v += red[q][i];
        partial[(size_t)bx * KMAX + i] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == (unsigned)nblocks - 1);
    __syncthreads();
    if (last) {
        __threadfence();
        // warp q adds vectors i = q, q + 8, ..: its lanes split the CTA partials (fixed
        // order, independent L2 loads), then a fixed shuffle tree
        for (int i = warp; i < k; i += RED_THREADS / 32) {
            double v = 0.0;
            for (int c = lane; c < nblocks; c += 32) v += __ldcg(partial + (size_t)c * KMAX + i);
            for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) out[i] = v;
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

template <int KC>
__device__ __forceinline__ void dots_body(const double* __restrict__ V, int k, const double* __restrict__ w, long n,
                                          double* __restrict__ out, double* __restrict__ partial,
                                          unsigned int* __restrict__ counter, int bx, int nblocks) {
    double acc[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) acc[i] = 0.0;
    const long stride = (long)nblocks * blockDim.x;
    for (long x = (long)bx * blockDim.x + threadIdx.x; x < n; x += stride) {
        const double wx = w[x];
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if (i < k) acc[i] += V[(size_t)i * n + x] * wx;
    }
    reduce_partials<KC>(acc, k, out, partial, counter, bx, nblocks);
}

// One pass of classical Gram-Schmidt over the basis V_0..V_{k-1} (x: element):
//   MODE 0: out[i] = sum_x V_i[x] w[x]
//   MODE 1: w[x] -= sum_i c[i] V_i[x], then out[i] = sum_x V_i[x] w[x] of the new w
//   MODE 2: w[x] -= sum_i c[i] V_i[x], then out[0] = sum_x w[x]^2
// The V_i[x] of an element are loaded once and serve both the update and the
// sums, so CGS2 (dots, update + dots, update + norm) reads V three times.
// PAIR: two neighbouring elements per thread with 16-byte loads (n even, so every
// V_i starts on a 16-byte boundary).
template <int KC, int MODE, bool PAIR>
__global__ void __launch_bounds__(RED_THREADS)
cgs_pass_kernel(const double* __restrict__ V, int k, const double* __restrict__ c, double* __restrict__ w, long n,
                double* __restrict__ out, double* __restrict__ partial, unsigned int* __restrict__ counter) {
    constexpr int NA = MODE == 2 ? 1 : KC;
    constexpr int E = PAIR ? 2 : 1;
    __shared__ double cs[KC];
    if (MODE > 0) {
        for (int i = threadIdx.x; i < KC; i += blockDim.x) cs[i] = i < k ? c[i] : 0.0;
        __syncthreads();
    }
    double acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[i] = 0.0;
    const long ne = n / E;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < ne; q += stride) {
        const long x = q * E;
        double wx[E], v[KC][E];
        if (PAIR) {
            const double2 t = *reinterpret_cast<const double2*>(w + x);
            wx[0] = t.x;
            wx[E - 1] = t.y;
        } else {
            wx[0] = w[x];
        }
#pragma unroll
        for (int i = 0; i < KC; ++i) {
            if (i < k) {
                if (PAIR) {
                    const double2 t = *reinterpret_cast<const double2*>(V + (size_t)i * n + x);
                    v[i][0] = t.x;
                    v[i][E - 1] = t.y;
                } else {
                    v[i][0] = V[(size_t)i * n + x];
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) v[i][e] = 0.0;
            }
        }
        if (MODE > 0) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                double a = wx[e];
#pragma unroll
                for (int i = 0; i < KC; ++i)
                    if (i < k) a -= cs[i] * v[i][e];
                wx[e] = a;
            }
            if (PAIR)
                *reinterpret_cast<double2*>(w + x) = make_double2(wx[0], wx[E - 1]);
            else
                w[x] = wx[0];
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (MODE == 2) {
                acc[0] += wx[e] * wx[e];
            } else {
#pragma unroll
                for (int i = 0; i < NA; ++i)
                    if (i < k) acc[i] += v[i][e] * wx[e];
            }
        }
    }
    reduce_partials<NA>(acc, MODE == 2 ? 1 : k, out, partial, counter, blockIdx.x, gridDim.x);
}

template <int KC>
__global__ void __launch_bounds__(RED_THREADS)
dots_kernel(const double* __restrict__ V, int k, const double* __restrict__ w, long n, double* __restrict__ out,
            double* __restrict__ partial, unsigned int* __restrict__ counter) {
    dots_body<KC>(V, k, w, n, out, partial, counter, blockIdx.x, gridDim.x);
}

// w += sign * sum_i coef[i] V_i
__global__ void update_kernel(const double* __restrict__ V, int k, const double* __restrict__ coef, double sign,
                              double* __restrict__ w, long n) {
    __shared__ double c[KMAX];
    for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = sign * coef[i];
    __syncthreads();
    const long stride = (long)gridDim.x * blockDim.x;
    for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        double acc = w[x];
        for (int i = 0; i < k; ++i) acc += c[i] * V[(size_t)i * n + x];
        w[x] = acc;
    }
}

__global__ void scale_kernel(const double* __restrict__ src, const double* __restrict__ nrm_sq,
                             double* __restrict__ dst, long n) {
    const double nr = sqrt(*nrm_sq);
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) dst[x] = src[x] * inv;
}

__global__ void axpy_kernel(double a, const double* __restrict__ x, double* __restrict__ y, long n) {
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] += a * x[i];
}

__global__ void sub_kernel(const double* __restrict__ b, const double* __restrict__ ax, double* __restrict__ r,
                           long n) {
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) r[i] = b[i] - ax[i];
}

// Column j of the Hessenberg matrix from the Gram-Schmidt coefficients, the
// previous Givens rotations applied to it, a new rotation that annihilates
// H[j+1][j], and the rotated right-hand side g; est = |g_{j+1}| is the residual
// norm of the current cycle.  H is column-major with leading dimension ldh.
__global__ void arnoldi_finish_kernel(double* __restrict__ H, int ldh, int j, const double* __restrict__ h1,
                                      const double* __restrict__ h2, const double* __restrict__ nrm_sq,
                                      double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                                      double* __restrict__ est) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double* col = H + (size_t)j * ldh;
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + (h2 ? h2[i] : 0.0);
    col[j + 1] = sqrt(*nrm_sq);
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double a = col[j], b = col[j + 1];
    const double r = hypot(a, b);
    const double c = r > 0.0 ? a / r : 1.0;
    const double s = r > 0.0 ? b / r : 0.0;
    cs[j] = c;
    sn[j] = s;
    col[j] = r;
    col[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    est[0] = fabs(g[j + 1]);
    est[1] = b;  // H[j+1][j] before rotation (breakdown test)
}

// y = R^{-1} g with R the k x k upper-triangular part of the rotated H.
__global__ void lsq_solve_kernel(const double* __restrict__ H, int ldh, int k, const double* __restrict__ g,
                                 double* __restrict__ y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double v = g[i];
        for (int c = i + 1; c < k; ++c) v -= H[(size_t)c * ldh + i] * y[c];
        y[i] = v / H[(size_t)i * ldh + i];
    }
}

// ---------------------------------------------------------------------------
// Batched variants over the active instances act[0..gridDim.y) of a batch.
// Each instance owns its vectors, scalars, partial sums and reduction ticket.
// ---------------------------------------------------------------------------
constexpr int RED_CTAS_B = 32;  // reduction CTAs per instance in a batch

// mode 0 / 1: h1 / h2 = V_{0..j}^T V_{j+1};  mode 2: |V_{j+1}|^2 -> scal[128];
// mode 3: |V_0|^2 -> scal[132];  mode 4: |b|^2 -> scal[131]
template <int KC>
__global__ void __launch_bounds__(RED_THREADS)
dots_batched(const InstDev* __restrict__ I, const int* __restrict__ act, int mode, int j) {
    const InstDev& d = I[act[blockIdx.y]];
    if (!d.ctl[0]) return;  // the instance has left the cycle: no CTA of it takes part
    const double* w;
    const double* V;
    int k;
    double* out;
    if (mode <= 1) {
        V = d.V; k = j + 1; w = d.V + (size_t)(j + 1) * d.n; out = d.scal + (mode == 0 ? 0 : 64);
    } else if (mode == 2) {
        V = w = d.V + (size_t)(j + 1) * d.n; k = 1; out = d.scal + 128;
    } else if (mode == 3) {
        V = w = d.V; k = 1; out = d.scal + 132;
    } else {
        V = w = d.b; k = 1; out = d.scal + 131;
    }
    dots_body<KC>(V, k, w, d.n, out, d.partial, d.counter, blockIdx.x, gridDim.x);
}

// mode 0 / 1: V_{j+1} -= V_{0..j} h1 / h2;  mode 2: x += Z_{0..k-1} y with k = kvec[instance]
__global__ void update_batched(const InstDev* __restrict__ I, const int* __restrict__ act, int mode, int j,
                               const int* __restrict__ kvec) {
    __shared__ double c[KMAX];
    const int inst = act[blockIdx.y];
    const InstDev& d = I[inst];
    if (!d.ctl[0]) return;
    const double* V;
    double* w;
    const double* coef;
    int k;
    double sign;
    if (mode <= 1) {
        V = d.V; w = d.V + (size_t)(j + 1) * d.n; coef = d.scal + (mode == 0 ? 0 : 64); k = j + 1; sign = -1.0;
    } else {
        V = d.Z; w = d.x; coef = d.y; k = kvec[inst]; sign = 1.0;
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = sign * coef[i];
    __syncthreads();
    const long stride = (long)gridDim.x * blockDim.x;
    for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < d.n; x += stride) {
        double acc = w[x];
        for (int i = 0; i < k; ++i) acc += c[i] * V[(size_t)i * d.n + x];
        w[x] = acc;
    }
}

// mode 0: V_{j+1} /= sqrt(scal[128]);  mode 1: V_0 /= sqrt(scal[132]) and g = (sqrt(scal[132]), 0, ...)
__global__ void scale_batched(const InstDev* __restrict__ I, const int* __restrict__ act, int mode, int j,
                              int restart) {
    const InstDev& d = I[act[blockIdx.y]];
    if (!d.ctl[0]) return;
    double* v = mode == 0 ? d.V + (size_t)(j + 1) * d.n : d.V;
    const double nr = sqrt(d.scal[mode == 0 ? 128 : 132]);
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < d.n; x += stride) v[x] *= inv;
    if (mode == 1 && blockIdx.x == 0)
        for (int i = threadIdx.x; i <= restart; i += blockDim.x) d.gv[i] = i == 0 ? nr : 0.0;
}

// V_0 = b - work (work = M x)
__global__ void residual_batched(const InstDev* __restrict__ I, const int* __restrict__ act) {
    const InstDev& d = I[act[blockIdx.y]];
    if (!d.ctl[0]) return;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < d.n; x += stride) d.V[x] = d.b[x] - d.work[x];
}

// one thread per active instance
__global__ void finish_batched(const InstDev* __restrict__ I, const int* __restrict__ act, int nact, int j, int ldh,
                               int reorth, double tol, int maxit) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nact) return;
    const InstDev& d = I[act[a]];
    if (!d.ctl[0]) return;
    double* col = d.H + (size_t)j * ldh;
    const double* h1 = d.scal;
    const double* h2 = d.scal + 64;
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + (reorth ? h2[i] : 0.0);
    col[j + 1] = sqrt(d.scal[128]);
    for (int i = 0; i < j; ++i) {
        const double t = d.cs[i] * col[i] + d.sn[i] * col[i + 1];
        col[i + 1] = -d.sn[i] * col[i] + d.cs[i] * col[i + 1];
        col[i] = t;
    }
    const double aa = col[j], bb = col[j + 1];
    const double r = hypot(aa, bb);
    const double c = r > 0.0 ? aa / r : 1.0;
    const double sn = r > 0.0 ? bb / r : 0.0;
    d.cs[j] = c;
    d.sn[j] = sn;
    col[j] = r;
    col[j + 1] = 0.0;
    d.gv[j + 1] = -sn * d.gv[j];
    d.gv[j] = c * d.gv[j];
    const double est = fabs(d.gv[j + 1]);
    d.scal[129] = est;
    d.scal[130] = bb;
    // leave the cycle: tolerance met (Givens estimate), maxit, breakdown, or non-finite
    const int its = d.ctl[2] + 1;
    d.ctl[2] = its;
    d.ctl[1] = j + 1;
    if (!isfinite(est) || !isfinite(d.scal[128])) {
        d.ctl[3] = 1;
        d.ctl[0] = 0;
    } else if (est <= tol * sqrt(d.scal[131]) || its >= maxit || fabs(bb) <= 1e-300) {
        d.ctl[0] = 0;
    }
}

__global__ void ctl_set_batched(const InstDev* __restrict__ I, const int* __restrict__ act, int nact, int live,
                                int reset) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nact) return;
    int* c = I[act[a]].ctl;
    c[0] = live;
    if (reset) c[1] = 0;
    if (reset > 1) {
        c[2] = 0;
        c[3] = 0;
    }
}

__global__ void lsq_batched(const InstDev* __restrict__ I, const int* __restrict__ act, int nact,
                            const int* __restrict__ kvec, int ldh) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nact) return;
    const int inst = act[a];
    const InstDev& d = I[inst];
    if (!d.ctl[0]) return;
    const int k = kvec[inst];
    for (int i = k - 1; i >= 0; --i) {
        double v = d.gv[i];
        for (int c = i + 1; c < k; ++c) v -= d.H[(size_t)c * ldh + i] * d.y[c];
        d.y[i] = v / d.H[(size_t)i * ldh + i];
    }
}

// out[4*i + q] = scal[128 + q] of instance i (q = 0..3), and out[4*i+3] = scal[132]
__global__ void gather_scalars(const InstDev* __restrict__ I, int ninst, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    const double* sc = I[i].scal;
    out[4 * i + 0] = sc[128];
    out[4 * i + 1] = sc[129];
    out[4 * i + 2] = sc[130];
    out[4 * i + 3] = sc[132];
}

static int grid_for(long n);

int launch_dots_batched(const InstDev* I, const int* act, int nact, int mode, int j, cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    const int k = mode <= 1 ? j + 1 : 1;
    const dim3 grid(RED_CTAS_B, nact);
    if (k <= 8) dots_batched<8><<<grid, RED_THREADS, 0, st>>>(I, act, mode, j);
    else if (k <= 16) dots_batched<16><<<grid, RED_THREADS, 0, st>>>(I, act, mode, j);
    else if (k <= 32) dots_batched<32><<<grid, RED_THREADS, 0, st>>>(I, act, mode, j);
    else dots_batched<64><<<grid, RED_THREADS, 0, st>>>(I, act, mode, j);
    FDE_LAUNCH_CHECK("dots_batched");
    return FDE_OK;
}

int launch_update_batched(const InstDev* I, const int* act, int nact, int mode, int j, const int* kvec, long max_n,
                          cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    int g = (int)((max_n + 255) / 256);
    if (g > 64) g = 64;
    update_batched<<<dim3(g, nact), 256, 0, st>>>(I, act, mode, j, kvec);
    FDE_LAUNCH_CHECK("update_batched");
    return FDE_OK;
}

int launch_scale_batched(const InstDev* I, const int* act, int nact, int mode, int j, int restart, long max_n,
                         cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    int g = (int)((max_n + 255) / 256);
    if (g > 64) g = 64;
    scale_batched<<<dim3(g, nact), 256, 0, st>>>(I, act, mode, j, restart);
    FDE_LAUNCH_CHECK("scale_batched");
    return FDE_OK;
}

int launch_residual_batched(const InstDev* I, const int* act, int nact, long max_n, cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    int g = (int)((max_n + 255) / 256);
    if (g > 64) g = 64;
    residual_batched<<<dim3(g, nact), 256, 0, st>>>(I, act);
    FDE_LAUNCH_CHECK("residual_batched");
    return FDE_OK;
}

int launch_finish_batched(const InstDev* I, const int* act, int nact, int j, int ldh, int reorth, double tol,
                          int maxit, cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    finish_batched<<<(nact + 63) / 64, 64, 0, st>>>(I, act, nact, j, ldh, reorth, tol, maxit);
    FDE_LAUNCH_CHECK("finish_batched");
    return FDE_OK;
}

int launch_ctl_set_batched(const InstDev* I, const int* act, int nact, int live, int reset, cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    ctl_set_batched<<<(nact + 63) / 64, 64, 0, st>>>(I, act, nact, live, reset);
    FDE_LAUNCH_CHECK("ctl_set_batched");
    return FDE_OK;
}

int launch_lsq_batched(const InstDev* I, const int* act, int nact, const int* kvec, int ldh, cudaStream_t st) {
    if (nact <= 0) return FDE_OK;
    lsq_batched<<<(nact + 63) / 64, 64, 0, st>>>(I, act, nact, kvec, ldh);
    FDE_LAUNCH_CHECK("lsq_batched");
    return FDE_OK;
}

int launch_gather_scalars(const InstDev* I, int ninst, double* out, cudaStream_t st) {
    gather_scalars<<<(ninst + 63) / 64, 64, 0, st>>>(I, ninst, out);
    FDE_LAUNCH_CHECK("gather_scalars");
    return FDE_OK;
}

static int grid_for(long n) {
    long g = (n + 255) / 256;
    if (g > 4 * 152) g = 4 * 152;
    if (g < 1) g = 1;
    return (int)g;
}

int launch_dots(const double* V, int k, const double* w, long n, double* out, double* partial, unsigned int* counter,
                cudaStream_t st) {
    if (k <= 0) return FDE_OK;
    if (k > KMAX) return set_error(FDE_ERR_ARG, "too many Krylov vectors for one multi-dot");
    if (k <= 8)
        dots_kernel<8><<<RED_CTAS, RED_THREADS, 0, st>>>(V, k, w, n, out, partial, counter);
    else if (k <= 16)
        dots_kernel<16><<<RED_CTAS, RED_THREADS, 0, st>>>(V, k, w, n, out, partial, counter);
    else if (k <= 32)
        dots_kernel<32><<<RED_CTAS, RED_THREADS, 0, st>>>(V, k, w, n, out, partial, counter);
    else
        dots_kernel<64><<<RED_CTAS, RED_THREADS, 0, st>>>(V, k, w, n, out, partial, counter);
    FDE_LAUNCH_CHECK("dots_kernel");
    return FDE_OK;
}

// One wave: as many CTAs as fit on the device at once (the wide variants hold
// their basis values in registers and fit one CTA per SM), at most RED_CTAS.
template <int KC, int MODE, bool PAIR>
static int one_wave_grid() {
    static int grid = 0;  // per kernel instantiation
    if (grid == 0) {
        auto kernel = cgs_pass_kernel<KC, MODE, PAIR>;
        int dev = 0, sms = 0, occ = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, RED_THREADS, 0) != cudaSuccess || occ < 1)
            return RED_CTAS;
        grid = std::min(RED_CTAS, sms * occ);
    }
    return grid;
}

template <int KC, int MODE>
static void cgs_pass_launch(const double* V, int k, const double* c, double* w, long n, double* out, double* partial,
                            unsigned int* counter, cudaStream_t st) {
    if constexpr (KC <= 24) {  // wider paired variants would spill
        if ((n & 1) == 0) {
            auto kern = cgs_pass_kernel<KC, MODE, true>;
            kern<<<one_wave_grid<KC, MODE, true>(), RED_THREADS, 0, st>>>(V, k, c, w, n, out, partial, counter);
            return;
        }
    }
    auto kern = cgs_pass_kernel<KC, MODE, false>;
    kern<<<one_wave_grid<KC, MODE, false>(), RED_THREADS, 0, st>>>(V, k, c, w, n, out, partial, counter);
}

template <int MODE>
static void cgs_pass_dispatch(const double* V, int k, const double* c, double* w, long n, double* out,
                              double* partial, unsigned int* counter, cudaStream_t st) {
    if (k <= 8)
        cgs_pass_launch<8, MODE>(V, k, c, w, n, out, partial, counter, st);
    else if (k <= 16)
        cgs_pass_launch<16, MODE>(V, k, c, w, n, out, partial, counter, st);
    else if (k <= 24)
        cgs_pass_launch<24, MODE>(V, k, c, w, n, out, partial, counter, st);
    else if (k <= 32)
        cgs_pass_launch<32, MODE>(V, k, c, w, n, out, partial, counter, st);
    else
        cgs_pass_launch<64, MODE>(V, k, c, w, n, out, partial, counter, st);
}

int launch_cgs_pass(int mode, const double* V, int k, const double* c, double* w, long n, double* out,
                    double* partial, unsigned int* counter, cudaStream_t st) {
    if (k <= 0 || n <= 0) return set_error(FDE_ERR_ARG, "empty Gram-Schmidt pass");
    if (k > KMAX) return set_error(FDE_ERR_ARG, "too many Krylov vectors for one Gram-Schmidt pass");
    if (mode == 0)
        cgs_pass_dispatch<0>(V, k, c, w, n, out, partial, counter, st);
    else if (mode == 1)
        cgs_pass_dispatch<1>(V, k, c, w, n, out, partial, counter, st);
    else if (mode == 2)
        cgs_pass_dispatch<2>(V, k, c, w, n, out, partial, counter, st);
    else
        return set_error(FDE_ERR_ARG, "unknown Gram-Schmidt pass mode");
    FDE_LAUNCH_CHECK("cgs_pass_kernel");
    return FDE_OK;
}

int launch_update(const double* V, int k, const double* coef, double sign, double* w, long n, cudaStream_t st) {
    if (k <= 0) return FDE_OK;
    update_kernel<<<grid_for(n), 256, 0, st>>>(V, k, coef, sign, w, n);
    FDE_LAUNCH_CHECK("update_kernel");
    return FDE_OK;
}

int launch_norm(const double* w, long n, double* out, double* partial, unsigned int* counter, cudaStream_t st) {
    dots_kernel<8><<<RED_CTAS, RED_THREADS, 0, st>>>(w, 1, w, n, out, partial, counter);
    FDE_LAUNCH_CHECK("dots_kernel(norm)");
    return FDE_OK;
}

int launch_scale(const double* src, const double* nrm_sq, double* dst, long n, cudaStream_t st) {
    scale_kernel<<<grid_for(n), 256, 0, st>>>(src, nrm_sq, dst, n);
    FDE_LAUNCH_CHECK("scale_kernel");
    return FDE_OK;
}

int launch_arnoldi_finish(double* H, int ldh, int j, const double* h1, const double* h2, const double* nrm_sq,
                          double* cs, double* sn, double* g, double* est, cudaStream_t st) {
    arnoldi_finish_kernel<<<1, 32, 0, st>>>(H, ldh, j, h1, h2, nrm_sq, cs, sn, g, est);
    FDE_LAUNCH_CHECK("arnoldi_finish_kernel");
    return FDE_OK;
}

int launch_lsq_solve(const double* H, int ldh, int k, const double* g, double* y, cudaStream_t st) {
    lsq_solve_kernel<<<1, 32, 0, st>>>(H, ldh, k, g, y);
    FDE_LAUNCH_CHECK("lsq_solve_kernel");
    return FDE_OK;
}

int launch_axpy(double a, const double* x, double* y, long n, cudaStream_t st) {
    axpy_kernel<<<grid_for(n), 256, 0, st>>>(a, x, y, n);
    FDE_LAUNCH_CHECK("axpy_kernel");
    return FDE_OK;
}

int launch_sub(const double* b, const double* ax, double* r, long n, cudaStream_t st) {
    sub_kernel<<<grid_for(n), 256, 0, st>>>(b, ax, r, n);
    FDE_LAUNCH_CHECK("sub_kernel");
    return FDE_OK;
}

}  // namespace fde
