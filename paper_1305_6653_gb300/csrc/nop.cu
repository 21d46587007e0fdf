// Learned warm start: a small 1-D convolutional neural operator that maps the data
// of eq. (1.1) -- u0, f(., t_n) for n = 0..s, alpha, d+, d- -- to a space-time
// initial guess u_1..u_s of the GMRES solve.  It works with sine-series
// coefficients c_j (v(x_i) = sum_j c_j sin(j pi x_i), j = 1..K): the convolution runs
// along the mode index (length K) over channels [c_j(u0), c_j(f(., t_n)) for
// n = 0..s, (alpha-1.5)/0.4, (mean d+ - 1.25)/0.75, (mean d- - 1.25)/0.75, j/K], and
// its s output channels are the coefficients of u_1..u_s, synthesised back to the
// grid.  The paper has no learned component; the solve is still judged by
// its true FP64 residual, and pgmres_solve falls back to the zero guess when the
// predicted guess is worse than zero.
//
// Network: L convolution layers (kernel K, zero padding, same length), ReLU after
// all but the last; parameters flat per layer: W (C_out, C_in, K) then b (C_out).
// Kernels: tiled forward convolution (FP32, or FP16 storage with FP32 accumulation
// for inference), backward-data as the forward kernel on the flipped / transposed
// weights with the ReLU mask fused, backward-weight reduction split over the
// batch, MSE loss gradient and Adam.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fde_internal.h"

namespace fde {

constexpr int CV_TCO = 16;   // output channels per CTA
constexpr int CV_TX = 128;   // positions per CTA
constexpr int CV_CI = 16;    // input channels per shared-memory chunk
constexpr int CV_KMAX = 7;

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
__device__ __forceinline__ void stf(__half* p, float v) { *p = __float2half_rn(v); }

// y[b][p][x] = bias[p] + sum_q sum_k Wacc(p,q,k) x[b][q][x + k - K/2]
//   TRANS = false: Wacc(p,q,k) = W[p][q][k]            (W: P x Q x K)
//   TRANS = true : Wacc(p,q,k) = W[q][p][K-1-k]        (W: Q x P x K; gradient w.r.t. the input)
// relu: apply max(., 0); mask: multiply by (mask[b][p][x] > 0) (backward through a ReLU).
template <typename TI, typename TW, typename TO, bool TRANS>
__global__ void __launch_bounds__(256)
conv_kernel(const TI* __restrict__ x, int Q, const TW* __restrict__ W, const float* __restrict__ bias, int P, int K,
            int m, int relu, const float* __restrict__ mask, TO* __restrict__ y) {
    __shared__ float s_in[CV_CI][CV_TX + CV_KMAX - 1];
    __shared__ float s_w[CV_TCO][CV_CI][CV_KMAX];
    const int b = blockIdx.z;
    const int p0 = blockIdx.y * CV_TCO;
    const int x0 = blockIdx.x * CV_TX;
    const int h = K / 2;
    const int pl = threadIdx.x / 16, xg = threadIdx.x % 16;
    float acc[CV_TX / 16];
#pragma unroll
    for (int j = 0; j < CV_TX / 16; ++j) acc[j] = 0.f;
    const TI* xb = x + (size_t)b * Q * m;
    for (int q0 = 0; q0 < Q; q0 += CV_CI) {
        for (int e = threadIdx.x; e < CV_CI * (CV_TX + K - 1); e += blockDim.x) {
            const int c = e / (CV_TX + K - 1), t = e % (CV_TX + K - 1);
            const int xx = x0 - h + t;
            s_in[c][t] = (q0 + c < Q && xx >= 0 && xx < m) ? ldf(xb + (size_t)(q0 + c) * m + xx) : 0.f;
        }
        for (int e = threadIdx.x; e < CV_TCO * CV_CI * K; e += blockDim.x) {
            const int o = e / (CV_CI * K), r = e % (CV_CI * K), c = r / K, k = r % K;
            float v = 0.f;
            if (p0 + o < P && q0 + c < Q) {
                v = TRANS ? ldf(W + ((size_t)(q0 + c) * P + (p0 + o)) * K + (K - 1 - k))
                          : ldf(W + ((size_t)(p0 + o) * Q + (q0 + c)) * K + k);
            }
            s_w[o][c][k] = v;
        }
        __syncthreads();
        for (int c = 0; c < CV_CI; ++c)
            for (int k = 0; k < K; ++k) {
                const float w = s_w[pl][c][k];
#pragma unroll
                for (int j = 0; j < CV_TX / 16; ++j) acc[j] += w * s_in[c][xg + 16 * j + k];
            }
        __syncthreads();
    }
    const int p = p0 + pl;
    if (p >= P) return;
    const float bb = bias ? bias[p] : 0.f;
#pragma unroll
    for (int j = 0; j < CV_TX / 16; ++j) {
        const int xx = x0 + xg + 16 * j;
        if (xx >= m) continue;
        float v = acc[j] + bb;
        if (relu) v = fmaxf(v, 0.f);
        const size_t idx = ((size_t)b * P + p) * m + xx;
        if (mask && !(mask[idx] > 0.f)) v = 0.f;
        stf(y + idx, v);
    }
}

// dW[o][c][k] += sum_{b in group} sum_x g[b][o][x] a[b][c][x + k - K/2]; one thread per (o, c)
// of a 16 x 16 tile, the batch split over gridDim.z groups (atomic accumulation).
__global__ void __launch_bounds__(256)
conv_wgrad_kernel(const float* __restrict__ g, int O, const float* __restrict__ a, int C, int K, int m, int B,
                  float* __restrict__ dW) {
    __shared__ float s_g[16][64];
    __shared__ float s_a[16][64 + CV_KMAX - 1];
    const int o0 = blockIdx.y * 16, c0 = blockIdx.x * 16;
    const int ol = threadIdx.x / 16, cl = threadIdx.x % 16;
    const int h = K / 2;
    float acc[CV_KMAX];
#pragma unroll
    for (int k = 0; k < CV_KMAX; ++k) acc[k] = 0.f;
    const int groups = gridDim.z;
    for (int b = blockIdx.z; b < B; b += groups) {
        for (int x0 = 0; x0 < m; x0 += 64) {
            for (int e = threadIdx.x; e < 16 * 64; e += blockDim.x) {
                const int r = e / 64, t = e % 64;
                const int xx = x0 + t;
                s_g[r][t] = (o0 + r < O && xx < m) ? g[((size_t)b * O + o0 + r) * m + xx] : 0.f;
            }
            for (int e = threadIdx.x; e < 16 * (64 + K - 1); e += blockDim.x) {
                const int r = e / (64 + K - 1), t = e % (64 + K - 1);
                const int xx = x0 - h + t;
                s_a[r][t] = (c0 + r < C && xx >= 0 && xx < m) ? a[((size_t)b * C + c0 + r) * m + xx] : 0.f;
            }
            __syncthreads();
            for (int t = 0; t < 64; ++t) {
                const float gv = s_g[ol][t];
#pragma unroll
                for (int k = 0; k < CV_KMAX; ++k)
                    if (k < K) acc[k] += gv * s_a[cl][t + k];
            }
            __syncthreads();
        }
    }
    if (o0 + ol < O && c0 + cl < C)
        for (int k = 0; k < K; ++k) atomicAdd(dW + ((size_t)(o0 + ol) * C + c0 + cl) * K + k, acc[k]);
}

// db[o] = sum_{b,x} g[b][o][x]
__global__ void bias_grad_kernel(const float* __restrict__ g, int O, int m, int B, float* __restrict__ db) {
    const int o = blockIdx.x;
    float s = 0.f;
    for (int b = 0; b < B; ++b)
        for (int x = threadIdx.x; x < m; x += blockDim.x) s += g[((size_t)b * O + o) * m + x];
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[o] = red[0];
}

// g = 2 (y - t) / N, loss += sum (y - t)^2 / N
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, long n, float* __restrict__ g,
                           double* __restrict__ loss) {
    double s = 0.0;
    const double inv = 1.0 / (double)n;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        g[i] = (float)(2.0 * d * inv);
        s += (double)d * d;
    }
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

// splitmix64 (Steele, Lea & Flood 2014) on (seed, index) -> uniform in [-1, 1)
__device__ __forceinline__ float splitmix_uniform(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
}

__global__ void init_kernel(float* __restrict__ p, long off, long n, float scale, unsigned long long seed) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        p[off + i] = scale * splitmix_uniform(seed, (unsigned long long)(off + i));
}

__global__ void to_half_kernel(const float* __restrict__ a, __half* __restrict__ b, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        b[i] = __float2half_rn(a[i]);
}

// Sine-series coefficients c[r][j] = 2/(m+1) sum_i v_r[i] sin(j pi (i+1)/(m+1)) of
// `rows` grid vectors v_r (stride m), so that v_r[i] = sum_j c[r][j] sin(j pi (i+1)/(m+1))
// on the first modes: one warp per (row, mode).
__global__ void sine_analysis_kernel(const double* __restrict__ v, int rows, int m, int K, float* __restrict__ out,
                                     int out_stride, int out_off) {
    const int lane = threadIdx.x & 31;
    const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (long)rows * K) return;
    const int r = (int)(w / K), j = (int)(w % K);
    const double* vr = v + (size_t)r * m;
    double c = 0.0;
    for (int i = lane; i < m; i += 32) c += vr[i] * sinpi((double)(j + 1) * (i + 1) / (double)(m + 1));
    for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if (lane == 0) out[(size_t)(out_off + r) * out_stride + j] = (float)(c * (2.0 / (double)(m + 1)));
}

// Scalar channels of the spectral input: (alpha-1.5)/0.4, mean d+, mean d- (normalised), j/K.
__global__ void scalar_channels_kernel(int m, int K, int c0, double alpha, const double* __restrict__ dp,
                                       const double* __restrict__ dm, float* __restrict__ in) {
    __shared__ double sp[256], sm[256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        a += dp[i];
        b += dm[i];
    }
    sp[threadIdx.x] = a;
    sm[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sp[threadIdx.x] += sp[threadIdx.x + w];
            sm[threadIdx.x] += sm[threadIdx.x + w];
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        in[(size_t)(c0 + 0) * K + j] = (float)((alpha - 1.5) / 0.4);
        in[(size_t)(c0 + 1) * K + j] = (float)((sp[0] / m - 1.25) / 0.75);
        in[(size_t)(c0 + 2) * K + j] = (float)((sm[0] / m - 1.25) / 0.75);
        in[(size_t)(c0 + 3) * K + j] = (float)(j + 1) / (float)K;
    }
}

// x0[t][i] = sum_j c[t][j] sin(j pi (i+1)/(m+1)): one CTA per time level.
__global__ void sine_synthesis_kernel(const float* __restrict__ c, int m, int K, double* __restrict__ x0) {
    extern __shared__ double coef[];
    const int t = blockIdx.x;
    for (int j = threadIdx.x; j < K; j += blockDim.x) coef[j] = (double)c[(size_t)t * K + j];
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double v = 0.0;
        for (int j = 0; j < K; ++j) v += coef[j] * sinpi((double)(j + 1) * (i + 1) / (double)(m + 1));
        x0[(size_t)t * m + i] = v;
    }
}

static int grid1(long n) {
    long g = (n + 255) / 256;
    return (int)(g > 1216 ? 1216 : (g < 1 ? 1 : g));
}

}  // namespace fde

using namespace fde;

struct fde_nop {
    int m = 0, s = 0, cin = 0, cout = 0, width = 0, layers = 0, K = 0;
    int modes = 0;                   // length of the convolution axis (sine modes)
    cudaStream_t stream = nullptr;
    std::vector<int> din, dout;      // per layer
    std::vector<long> woff, boff;    // offsets in the flat parameter vector
    long nparam = 0;
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    __half* p16 = nullptr;
    bool p16_valid = false;
    int t = 0;
    int bcap = 0;
    std::vector<float*> act;         // act[1..L], float, bcap x C_l x m
    float *ga = nullptr, *gb = nullptr;  // gradient ping-pong, bcap x max C x m
    __half *h_a = nullptr, *h_b = nullptr;  // FP16 inference activations (batch 1)
    float* feat = nullptr;           // features of one problem (cin x m)
    float* out1 = nullptr;           // output of one inference (s x m)
    double* d_loss = nullptr;
    double* h_loss = nullptr;        // pinned
};

namespace {

template <typename TI, typename TW, typename TO, bool TRANS>
int conv(const TI* x, int Q, const TW* W, const float* bias, int P, int K, int m, int B, int relu, const float* mask,
         TO* y, cudaStream_t st) {
    dim3 grid((m + CV_TX - 1) / CV_TX, (P + CV_TCO - 1) / CV_TCO, B);
    conv_kernel<TI, TW, TO, TRANS><<<grid, 256, 0, st>>>(x, Q, W, bias, P, K, m, relu, mask, y);
    FDE_LAUNCH_CHECK("conv_kernel");
    return FDE_OK;
}

int ensure_batch(fde_nop* n, int B) {
    if (B <= n->bcap) return FDE_OK;
    for (size_t l = 1; l < n->act.size(); ++l)
        if (n->act[l]) cudaFree(n->act[l]);
    if (n->ga) cudaFree(n->ga);
    if (n->gb) cudaFree(n->gb);
    n->act.assign(n->layers + 1, nullptr);
    int cmax = n->cin;
    for (int l = 0; l < n->layers; ++l) {
        FDE_CUDA_TRY(cudaMalloc(&n->act[l + 1], (size_t)B * n->dout[l] * n->modes * sizeof(float)));
        cmax = std::max(cmax, n->dout[l]);
    }
    FDE_CUDA_TRY(cudaMalloc(&n->ga, (size_t)B * cmax * n->modes * sizeof(float)));
    FDE_CUDA_TRY(cudaMalloc(&n->gb, (size_t)B * cmax * n->modes * sizeof(float)));
    n->bcap = B;
    return FDE_OK;
}

int forward32(fde_nop* n, const float* in, int B) {
    int rc = ensure_batch(n, B);
    if (rc) return rc;
    const float* x = in;
    for (int l = 0; l < n->layers; ++l) {
        rc = conv<float, float, float, false>(x, n->din[l], n->p + n->woff[l], n->p + n->boff[l], n->dout[l], n->K,
                                              n->modes, B, l < n->layers - 1, nullptr, n->act[l + 1], n->stream);
        if (rc) return rc;
        x = n->act[l + 1];
    }
    return FDE_OK;
}

}  // namespace

extern "C" {

void fde_nop_destroy(fde_nop* n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    for (size_t l = 1; l < n->act.size(); ++l)
        if (n->act[l]) cudaFree(n->act[l]);
    void* bufs[] = {n->p, n->g, n->m1, n->m2, n->p16, n->ga, n->gb, n->h_a, n->h_b, n->feat, n->out1, n->d_loss};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (n->h_loss) cudaFreeHost(n->h_loss);
    delete n;
}

int fde_nop_create(int m, int s, int modes, int width, int layers, int ksize, unsigned long long seed, void* stream,
                   fde_nop** out) {
    if (!out || m < 1 || s < 1 || modes < 1 || modes > m || width < 1 || layers < 1 || ksize < 1 ||
        ksize > CV_KMAX || ksize % 2 == 0)
        return set_error(FDE_ERR_ARG, "need m, s, width, layers >= 1, 1 <= modes <= m, odd kernel size <= 7");
    *out = nullptr;
    fde_nop* n = new (std::nothrow) fde_nop();
    if (!n) return set_error(FDE_ERR_ALLOC, "host allocation failed");
    n->m = m; n->s = s; n->modes = modes; n->cin = s + 6; n->cout = s; n->width = width; n->layers = layers;
    n->K = ksize;
    n->stream = (cudaStream_t)stream;
    for (int l = 0; l < layers; ++l) {
        n->din.push_back(l == 0 ? n->cin : width);
        n->dout.push_back(l == layers - 1 ? n->cout : width);
        n->woff.push_back(n->nparam);
        n->nparam += (long)n->dout[l] * n->din[l] * ksize;
        n->boff.push_back(n->nparam);
        n->nparam += n->dout[l];
    }
    const size_t pb = (size_t)n->nparam * sizeof(float);
    bool ok = cudaMalloc(&n->p, pb) == cudaSuccess && cudaMalloc(&n->g, pb) == cudaSuccess &&
              cudaMalloc(&n->m1, pb) == cudaSuccess && cudaMalloc(&n->m2, pb) == cudaSuccess &&
              cudaMalloc(&n->p16, (size_t)n->nparam * sizeof(__half)) == cudaSuccess &&
              cudaMalloc(&n->h_a, (size_t)std::max(n->cin, width) * modes * sizeof(__half)) == cudaSuccess &&
              cudaMalloc(&n->h_b, (size_t)std::max(n->cin, width) * modes * sizeof(__half)) == cudaSuccess &&
              cudaMalloc(&n->feat, (size_t)n->cin * modes * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&n->out1, (size_t)s * modes * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&n->d_loss, sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&n->h_loss, sizeof(double)) == cudaSuccess;
    if (!ok) {
        fde_nop_destroy(n);
        return set_error(FDE_ERR_ALLOC, "device allocation failed");
    }
    // He-uniform weights (last layer scaled down), zero biases, zero Adam moments
    cudaMemsetAsync(n->p, 0, pb, n->stream);
    cudaMemsetAsync(n->m1, 0, pb, n->stream);
    cudaMemsetAsync(n->m2, 0, pb, n->stream);
    for (int l = 0; l < layers; ++l) {
        const long nw = (long)n->dout[l] * n->din[l] * ksize;
        float a = std::sqrt(6.0f / (float)(n->din[l] * ksize));
        if (l == layers - 1) a *= 0.1f;
        init_kernel<<<grid1(nw), 256, 0, n->stream>>>(n->p, n->woff[l], nw, a, seed);
        note_launch();
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fde_nop_destroy(n);
        return cuda_error(e, "fde_nop_create");
    }
    *out = n;
    return FDE_OK;
}

long long fde_nop_num_params(const fde_nop* n) { return n ? n->nparam : 0; }
int fde_nop_in_channels(const fde_nop* n) { return n ? n->cin : 0; }

int fde_nop_set_params(fde_nop* n, const float* params) {
    if (!n || !params) return set_error(FDE_ERR_ARG, "NULL argument");
    FDE_CUDA_TRY(cudaMemcpyAsync(n->p, params, n->nparam * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    FDE_CUDA_TRY(cudaStreamSynchronize(n->stream));
    n->p16_valid = false;
    return FDE_OK;
}

int fde_nop_get_params(fde_nop* n, float* params) {
    if (!n || !params) return set_error(FDE_ERR_ARG, "NULL argument");
    FDE_CUDA_TRY(cudaMemcpyAsync(params, n->p, n->nparam * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    FDE_CUDA_TRY(cudaStreamSynchronize(n->stream));
    return FDE_OK;
}

int fde_nop_forward(fde_nop* n, const float* in, float* out, int batch) {
    if (!n || !in || !out || batch < 1) return set_error(FDE_ERR_ARG, "bad argument");
    int rc = forward32(n, in, batch);
    if (rc) return rc;
    FDE_CUDA_TRY(cudaMemcpyAsync(out, n->act[n->layers], (size_t)batch * n->cout * n->modes * sizeof(float),
                                 cudaMemcpyDeviceToDevice, n->stream));
    return FDE_OK;
}

int fde_nop_loss_grad(fde_nop* n, const float* in, const float* target, int batch, double* loss, float* grad_host) {
    if (!n || !in || !target || batch < 1) return set_error(FDE_ERR_ARG, "bad argument");
    int rc = forward32(n, in, batch);
    if (rc) return rc;
    const int L = n->layers, m = n->modes, B = batch;
    const long ny = (long)B * n->cout * m;
    FDE_CUDA_TRY(cudaMemsetAsync(n->d_loss, 0, sizeof(double), n->stream));
    FDE_CUDA_TRY(cudaMemsetAsync(n->g, 0, n->nparam * sizeof(float), n->stream));
    mse_kernel<<<grid1(ny), 256, 0, n->stream>>>(n->act[L], target, ny, n->ga, n->d_loss);
    FDE_LAUNCH_CHECK("mse_kernel");
    float* g = n->ga;      // gradient w.r.t. the output of layer l (after its ReLU mask)
    float* gnext = n->gb;
    for (int l = L - 1; l >= 0; --l) {
        const float* a = l == 0 ? in : n->act[l];
        const int O = n->dout[l], C = n->din[l];
        dim3 wg((C + 15) / 16, (O + 15) / 16, std::min(B, 16));
        conv_wgrad_kernel<<<wg, 256, 0, n->stream>>>(g, O, a, C, n->K, m, B, n->g + n->woff[l]);
        FDE_LAUNCH_CHECK("conv_wgrad_kernel");
        bias_grad_kernel<<<O, 256, 0, n->stream>>>(g, O, m, B, n->g + n->boff[l]);
        FDE_LAUNCH_CHECK("bias_grad_kernel");
        if (l > 0) {
            // gradient w.r.t. the layer input, through the ReLU of layer l-1 (mask = its output)
            rc = conv<float, float, float, true>(g, O, n->p + n->woff[l], nullptr, C, n->K, m, B, 0, n->act[l], gnext,
                                                 n->stream);
            if (rc) return rc;
            std::swap(g, gnext);
        }
    }
    FDE_CUDA_TRY(cudaMemcpyAsync(n->h_loss, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    if (grad_host)
        FDE_CUDA_TRY(cudaMemcpyAsync(grad_host, n->g, n->nparam * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    FDE_CUDA_TRY(cudaStreamSynchronize(n->stream));
    if (loss) *loss = *n->h_loss;
    return FDE_OK;
}

int fde_nop_adam_step(fde_nop* n, float lr) {
    if (!n) return set_error(FDE_ERR_ARG, "NULL network");
    ++n->t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->t), c2 = 1.f - std::pow(b2, (float)n->t);
    adam_kernel<<<grid1(n->nparam), 256, 0, n->stream>>>(n->p, n->g, n->m1, n->m2, n->nparam, lr, b1, b2, 1e-8f, c1,
                                                         c2);
    FDE_LAUNCH_CHECK("adam_kernel");
    n->p16_valid = false;
    return FDE_OK;
}

int fde_nop_features(fde_nop* n, fde_problem* h, float* in) {
    if (!n || !h || !in) return set_error(FDE_ERR_ARG, "NULL argument");
    Problem& P = *problem_of(h);
    if (P.m != n->m || P.s != n->s) return set_error(FDE_ERR_ARG, "problem size differs from the network's");
    const int K = n->modes;
    const long w0 = (long)1 * K * 32, w1 = (long)(P.s + 1) * K * 32;
    sine_analysis_kernel<<<(int)((w0 + 255) / 256), 256, 0, n->stream>>>(P.d_u0, 1, P.m, K, in, K, 0);
    FDE_LAUNCH_CHECK("sine_analysis_kernel(u0)");
    sine_analysis_kernel<<<(int)((w1 + 255) / 256), 256, 0, n->stream>>>(P.d_f, P.s + 1, P.m, K, in, K, 1);
    FDE_LAUNCH_CHECK("sine_analysis_kernel(f)");
    scalar_channels_kernel<<<1, 256, 0, n->stream>>>(P.m, K, P.s + 2, P.alpha, P.d_dplus, P.d_dminus, in);
    FDE_LAUNCH_CHECK("scalar_channels_kernel");
    return FDE_OK;
}

int fde_nop_coefficients(fde_nop* n, const double* x, float* coef) {
    if (!n || !x || !coef) return set_error(FDE_ERR_ARG, "NULL argument");
    const long w = (long)n->s * n->modes * 32;
    sine_analysis_kernel<<<(int)((w + 255) / 256), 256, 0, n->stream>>>(x, n->s, n->m, n->modes, coef, n->modes, 0);
    FDE_LAUNCH_CHECK("sine_analysis_kernel(x)");
    return FDE_OK;
}

int fde_nop_warm_start(fde_nop* n, fde_problem* h, double* x0) {
    if (!n || !h || !x0) return set_error(FDE_ERR_ARG, "NULL argument");
    int rc = fde_nop_features(n, h, n->feat);
    if (rc) return rc;
    if (!n->p16_valid) {
        to_half_kernel<<<grid1(n->nparam), 256, 0, n->stream>>>(n->p, n->p16, n->nparam);
        FDE_LAUNCH_CHECK("to_half_kernel");
        n->p16_valid = true;
    }
    // FP16 storage of weights and activations, FP32 accumulation and biases
    const int L = n->layers, m = n->modes;
    const __half* xh = nullptr;
    for (int l = 0; l < L; ++l) {
        __half* dst = (l % 2 == 0) ? n->h_a : n->h_b;
        const float* bias = n->p + n->boff[l];
        if (l == L - 1) {
            if (l == 0)
                rc = conv<float, __half, float, false>(n->feat, n->din[l], n->p16 + n->woff[l], bias, n->dout[l], n->K,
                                                       m, 1, 0, nullptr, n->out1, n->stream);
            else
                rc = conv<__half, __half, float, false>(xh, n->din[l], n->p16 + n->woff[l], bias, n->dout[l], n->K, m,
                                                        1, 0, nullptr, n->out1, n->stream);
        } else if (l == 0) {
            rc = conv<float, __half, __half, false>(n->feat, n->din[l], n->p16 + n->woff[l], bias, n->dout[l], n->K,
                                                    m, 1, 1, nullptr, dst, n->stream);
        } else {
            rc = conv<__half, __half, __half, false>(xh, n->din[l], n->p16 + n->woff[l], bias, n->dout[l], n->K, m, 1,
                                                     1, nullptr, dst, n->stream);
        }
        if (rc) return rc;
        xh = dst;
    }
    sine_synthesis_kernel<<<n->s, 256, n->modes * sizeof(double), n->stream>>>(n->out1, n->m, n->modes, x0);
    FDE_LAUNCH_CHECK("sine_synthesis_kernel");
    return FDE_OK;
}

int fde_nop_synthesize(fde_nop* n, const float* coef, double* x) {
    if (!n || !coef || !x) return set_error(FDE_ERR_ARG, "NULL argument");
    sine_synthesis_kernel<<<n->s, 256, n->modes * sizeof(double), n->stream>>>(coef, n->m, n->modes, x);
    FDE_LAUNCH_CHECK("sine_synthesis_kernel");
    return FDE_OK;
}

}  // extern "C"
