// mlp.cu -- the learned sketch-size predictor: a multilayer perceptron
// 9 -> 128 -> 128 -> 128 -> 1 (GELU after each hidden layer) that maps features of
// a network and a sketch size to log10 of the estimator's relative error, trained
// on the GPU by these kernels (mean squared error, Adam) and evaluated in FP32 or
// with BF16 operands (FP32 accumulation). tnsk_choose_params uses it to pick the
// smallest m whose predicted error meets a target, with the paper's variance bound
// (Theorem "general" / "acyclic" bounds, m R >= 3^t / (eps^2 delta) resp.
// 32 t / (eps^2 delta)) when no predictor is given.
//
// Parameters: for each layer W [n_out][n_in] row-major then b [n_out], layers in
// order, one flat FP32 vector; inputs are standardised per feature, z = (x - mu) /
// sigma, with mu and sigma taken from the training set.
//
// The products are at most [batch x 128] x [128 x 128]: launch-bound, not
// throughput-bound, so they run as one small tiled SIMT kernel (32 x 32 output
// tile, 256 threads, 2 x 2 outputs per thread) rather than on the tensor cores.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "kernels.cuh"
#include "plan.cuh"

namespace tnsk {
namespace {

constexpr int kFeatures = TNSK_MLP_FEATURES;
constexpr int kHidden = 128;
constexpr int kLayers = 4;
constexpr int kDims[kLayers + 1] = {kFeatures, kHidden, kHidden, kHidden, 1};
constexpr int kTile = 32;

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}
__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

}  // namespace

// C[M][N] (+)= sum_k A(m, k) B(k, n), then an epilogue. A(m, k) = A[m * lda + k], or
// A[k * lda + m] when TA; B(k, n) = B[k * ldb + n], or B[n * ldb + k] when TB.
// Epilogue: + bias[n] (if bias), pre = value (if pre), C = gelu(value) (if gelu).
// BF16: A and B are rounded to bfloat16 as they are loaded (FP32 accumulation).
template <bool TA, bool TB, bool BF16>
__global__ void __launch_bounds__(256) mlp_gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                       const float* __restrict__ B, int ldb, float* __restrict__ C,
                                                       int ldc, const float* __restrict__ bias, float* __restrict__ pre,
                                                       int gelu) {
    __shared__ float As[kTile][kTile + 1];  // [m][k]
    __shared__ float Bs[kTile][kTile + 1];  // [k][n]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k0 = 0; k0 < K; k0 += kTile) {
        for (int q = threadIdx.x; q < kTile * kTile; q += blockDim.x) {
            const int r = q / kTile, c = q % kTile;
            {  // As[r = m][c = k]
                const int mm = m0 + r, kk = k0 + c;
                float v = 0.f;
                if (mm < M && kk < K) v = TA ? A[(size_t)kk * lda + mm] : A[(size_t)mm * lda + kk];
                As[r][c] = BF16 ? round_bf16(v) : v;
            }
            {  // Bs[r = k][c = n]
                const int kk = k0 + r, nn = n0 + c;
                float v = 0.f;
                if (kk < K && nn < N) v = TB ? B[(size_t)nn * ldb + kk] : B[(size_t)kk * ldb + nn];
                Bs[r][c] = BF16 ? round_bf16(v) : v;
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kTile; ++k) {
            const float a0 = As[ty][k], a1 = As[ty + 16][k];
            const float b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
            acc[0][0] += a0 * b0;
            acc[0][1] += a0 * b1;
            acc[1][0] += a1 * b0;
            acc[1][1] += a1 * b1;
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int mm = m0 + ty + 16 * i, nn = n0 + tx + 16 * j;
            if (mm >= M || nn >= N) continue;
            float v = acc[i][j] + (bias ? bias[nn] : 0.f);
            if (pre) pre[(size_t)mm * ldc + nn] = v;
            C[(size_t)mm * ldc + nn] = gelu ? gelu_f(v) : v;
        }
}

// z = (x - mu) / sigma per feature; rows picked by idx when idx != nullptr.
__global__ void mlp_standardize_kernel(const float* __restrict__ X, const int64_t* __restrict__ idx, int64_t n,
                                       const float* __restrict__ mu, const float* __restrict__ sigma,
                                       float* __restrict__ Z) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * kFeatures;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = q / kFeatures;
        const int f = (int)(q - row * kFeatures);
        const int64_t src = idx ? idx[row] : row;
        Z[q] = (X[src * kFeatures + f] - mu[f]) / sigma[f];
    }
}

// dout = 2 (out - y) / B for the picked rows; loss += sum (out - y)^2 / B.
__global__ void mlp_mse_kernel(const float* __restrict__ out, const float* __restrict__ y,
                               const int64_t* __restrict__ idx, int B, float* __restrict__ dout,
                               double* __restrict__ loss) {
    double part = 0.0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const float d = out[b] - y[idx ? idx[b] : b];
        dout[b] = 2.f * d / (float)B;
        part += (double)d * d / B;
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) part += __shfl_xor_sync(0xffffffffu, part, s);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, part);
}

__global__ void mlp_gelu_bwd_kernel(float* __restrict__ d, const float* __restrict__ pre, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        d[q] *= gelu_grad_f(pre[q]);
}

// db[n] = sum_b d[b][n]
__global__ void mlp_bias_grad_kernel(const float* __restrict__ d, int B, int N, float* __restrict__ db) {
    const int nn = blockIdx.x * blockDim.x + threadIdx.x;
    if (nn >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += d[(size_t)b * N + nn];
    db[nn] = s;
}

// Adam (Kingma & Ba), bias-corrected.
__global__ void mlp_adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                                float c2) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        theta[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    }
}

// Sums of squares of many tensors in FP64 (features: Frobenius norms), one launch:
// each tensor is cut into chunks of kSqChunk entries numbered from jobs[j].chunk0; a
// block takes chunks round-robin, finds a chunk's tensor by binary search over chunk0
// and adds its chunk's sum into out[j].
struct SqJob {
    const void* data;
    int64_t n;
    int64_t chunk0;
    int32_t dtype;
    int32_t pad_;
};
constexpr int kSqChunk = 8192;

__global__ void __launch_bounds__(256) sumsq_batch_kernel(const SqJob* __restrict__ jobs, int nj, int64_t nchunks,
                                                          double* __restrict__ out) {
    __shared__ double red[8];
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        int lo = 0, hi = nj - 1;  // the last job whose first chunk is <= c
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].chunk0 <= c) lo = mid;
            else hi = mid - 1;
        }
        const SqJob J = jobs[lo];
        const int64_t i0 = (c - J.chunk0) * kSqChunk;
        const int64_t i1 = J.n < i0 + kSqChunk ? J.n : i0 + kSqChunk;
        double s = 0.0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const double x = load_as<double>(J.data, J.dtype, i);
            s += x * x;
        }
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) s += __shfl_xor_sync(0xffffffffu, s, sh);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            atomicAdd(out + lo, t);
        }
        __syncthreads();
    }
}

}  // namespace tnsk

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
#include "ctx.cuh"

using namespace tnsk;

struct tnsk_mlp {
    int device = 0;
    int64_t n = 0;  // parameters
    float* theta = nullptr;
    float* grad = nullptr;
    float* m1 = nullptr;  // Adam moments
    float* m2 = nullptr;
    float* norm = nullptr;  // device [2F]: mu, sigma
    float h_norm[2 * kFeatures];
    int64_t step = 0;
    // activation buffers for `cap` rows
    int64_t cap = 0;
    float* Z = nullptr;
    float* pre[kLayers] = {};
    float* out[kLayers] = {};
    float* d0 = nullptr;
    float* d1 = nullptr;
    double* loss = nullptr;
};

namespace {

int64_t param_count() {
    int64_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += (int64_t)kDims[l + 1] * kDims[l] + kDims[l + 1];
    return n;
}
int64_t w_off(int l) {
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += (int64_t)kDims[i + 1] * kDims[i] + kDims[i + 1];
    return o;
}
int64_t b_off(int l) { return w_off(l) + (int64_t)kDims[l + 1] * kDims[l]; }

void free_acts(tnsk_mlp* p) {
    cudaFree(p->Z);
    for (int l = 0; l < kLayers; ++l) {
        cudaFree(p->pre[l]);
        cudaFree(p->out[l]);
        p->pre[l] = p->out[l] = nullptr;
    }
    cudaFree(p->d0);
    cudaFree(p->d1);
    p->Z = p->d0 = p->d1 = nullptr;
    p->cap = 0;
}

bool ensure_acts(tnsk_mlp* p, int64_t rows) {
    if (rows <= p->cap) return true;
    free_acts(p);
    bool ok = cudaMalloc((void**)&p->Z, rows * kFeatures * sizeof(float)) == cudaSuccess;
    for (int l = 0; l < kLayers; ++l) {
        ok = ok && cudaMalloc((void**)&p->pre[l], rows * kDims[l + 1] * sizeof(float)) == cudaSuccess;
        ok = ok && cudaMalloc((void**)&p->out[l], rows * kDims[l + 1] * sizeof(float)) == cudaSuccess;
    }
    ok = ok && cudaMalloc((void**)&p->d0, rows * kHidden * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&p->d1, rows * kHidden * sizeof(float)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_acts(p);
        return false;
    }
    p->cap = rows;
    return true;
}

template <bool TA, bool TB, bool BF16>
void gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc, const float* bias,
          float* pre, bool gelu, cudaStream_t s) {
    dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
    mlp_gemm_kernel<TA, TB, BF16><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, pre, gelu ? 1 : 0);
}

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8); }

// standardise rows (picked by idx) of X into p->Z and run the layers; the output
// column is p->out[kLayers - 1]
void forward(tnsk_mlp* p, const float* X, const int64_t* idx, int64_t B, bool bf16, cudaStream_t s) {
    mlp_standardize_kernel<<<grid_for(B * kFeatures), 256, 0, s>>>(X, idx, B, p->norm, p->norm + kFeatures, p->Z);
    const float* h = p->Z;
    for (int l = 0; l < kLayers; ++l) {
        const bool act = l < kLayers - 1;
        if (bf16)
            gemm<false, true, true>((int)B, kDims[l + 1], kDims[l], h, kDims[l], p->theta + w_off(l), kDims[l],
                                    p->out[l], kDims[l + 1], p->theta + b_off(l), p->pre[l], act, s);
        else
            gemm<false, true, false>((int)B, kDims[l + 1], kDims[l], h, kDims[l], p->theta + w_off(l), kDims[l],
                                     p->out[l], kDims[l + 1], p->theta + b_off(l), p->pre[l], act, s);
        h = p->out[l];
    }
}

// mean squared error of the last forward against y (rows idx) and its gradient
// into p->grad; adds the loss to p->loss
void backward(tnsk_mlp* p, const float* y, const int64_t* idx, int64_t B, cudaStream_t s) {
    float* d = p->d0;
    float* dn = p->d1;
    mlp_mse_kernel<<<grid_for(B), 256, 0, s>>>(p->out[kLayers - 1], y, idx, (int)B, d, p->loss);
    for (int l = kLayers - 1; l >= 0; --l) {
        const int no = kDims[l + 1], ni = kDims[l];
        const float* in = l > 0 ? p->out[l - 1] : p->Z;
        // gW[o][i] = sum_b d[b][o] in[b][i]
        gemm<true, false, false>(no, ni, (int)B, d, no, in, ni, p->grad + w_off(l), ni, nullptr, nullptr, false, s);
        mlp_bias_grad_kernel<<<(no + 127) / 128, 128, 0, s>>>(d, (int)B, no, p->grad + b_off(l));
        if (l > 0) {
            // d_prev[b][i] = sum_o d[b][o] W[o][i], times gelu'(pre_prev)
            gemm<false, false, false>((int)B, ni, no, d, no, p->theta + w_off(l), ni, dn, ni, nullptr, nullptr, false,
                                      s);
            mlp_gelu_bwd_kernel<<<grid_for(B * ni), 256, 0, s>>>(dn, p->pre[l - 1], B * ni);
            std::swap(d, dn);
        }
    }
}

}  // namespace

extern "C" {

tnsk_status tnsk_mlp_num_params(int64_t* n) {
    if (!n) return TNSK_ERR_INVALID;
    *n = param_count();
    return TNSK_OK;
}

tnsk_status tnsk_mlp_create(tnsk_ctx* ctx, uint64_t seed, tnsk_mlp** out) {
    if (!out) return TNSK_ERR_INVALID;
    *out = nullptr;
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    tnsk_mlp* p = new tnsk_mlp();
    p->device = ctx->device;
    p->n = param_count();
    const size_t bytes = (size_t)p->n * sizeof(float);
    bool ok = cudaMalloc((void**)&p->theta, bytes) == cudaSuccess && cudaMalloc((void**)&p->grad, bytes) == cudaSuccess &&
              cudaMalloc((void**)&p->m1, bytes) == cudaSuccess && cudaMalloc((void**)&p->m2, bytes) == cudaSuccess &&
              cudaMalloc((void**)&p->norm, 2 * kFeatures * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&p->loss, sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        tnsk_mlp_destroy(p);
        return ctx_fail(ctx, TNSK_ERR_OOM, "predictor allocation failed");
    }
    // W ~ U(-a, a), a = sqrt(6 / n_in), b = 0; identity standardisation
    std::mt19937_64 rng(seed);
    std::vector<float> h((size_t)p->n, 0.f);
    for (int l = 0; l < kLayers; ++l) {
        std::uniform_real_distribution<double> u(-std::sqrt(6.0 / kDims[l]), std::sqrt(6.0 / kDims[l]));
        for (int64_t q = 0; q < (int64_t)kDims[l + 1] * kDims[l]; ++q) h[(size_t)(w_off(l) + q)] = (float)u(rng);
    }
    for (int f = 0; f < kFeatures; ++f) {
        p->h_norm[f] = 0.f;
        p->h_norm[kFeatures + f] = 1.f;
    }
    cudaMemcpy(p->theta, h.data(), bytes, cudaMemcpyHostToDevice);
    cudaMemcpy(p->norm, p->h_norm, sizeof(p->h_norm), cudaMemcpyHostToDevice);
    cudaMemset(p->m1, 0, bytes);
    cudaMemset(p->m2, 0, bytes);
    if (cudaGetLastError() != cudaSuccess) {
        tnsk_mlp_destroy(p);
        return ctx_fail(ctx, TNSK_ERR_CUDA, "predictor initialisation failed");
    }
    *out = p;
    return TNSK_OK;
}

tnsk_status tnsk_mlp_destroy(tnsk_mlp* p) {
    if (!p) return TNSK_ERR_INVALID;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    free_acts(p);
    cudaFree(p->theta);
    cudaFree(p->grad);
    cudaFree(p->m1);
    cudaFree(p->m2);
    cudaFree(p->norm);
    cudaFree(p->loss);
    delete p;
    return TNSK_OK;
}

tnsk_status tnsk_mlp_get(tnsk_mlp* p, float* theta, float* norm) {
    if (!p || !theta || !norm) return TNSK_ERR_INVALID;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    if (cudaMemcpy(theta, p->theta, (size_t)p->n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return TNSK_ERR_CUDA;
    }
    std::memcpy(norm, p->h_norm, sizeof(p->h_norm));
    return TNSK_OK;
}

tnsk_status tnsk_mlp_set(tnsk_ctx* ctx, tnsk_mlp* p, const float* theta, const float* norm) {
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    if (!p || !theta || !norm) return ctx_fail(ctx, TNSK_ERR_INVALID, "mlp_set: NULL argument");
    for (int f = 0; f < kFeatures; ++f)
        if (!(norm[kFeatures + f] > 0.f)) return ctx_fail(ctx, TNSK_ERR_INVALID, "mlp_set: sigma must be > 0");
    std::memcpy(p->h_norm, norm, sizeof(p->h_norm));
    cudaStreamSynchronize(ctx->stream);
    if (cudaMemcpy(p->theta, theta, (size_t)p->n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->norm, p->h_norm, sizeof(p->h_norm), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, TNSK_ERR_CUDA, "mlp_set: copy failed");
    }
    p->step = 0;
    cudaMemset(p->m1, 0, (size_t)p->n * sizeof(float));
    cudaMemset(p->m2, 0, (size_t)p->n * sizeof(float));
    return TNSK_OK;
}

}  // extern "C"

extern "C" {

tnsk_status tnsk_mlp_loss_grad(tnsk_ctx* ctx, tnsk_mlp* p, const float* X, const float* y, int64_t n, float* grad,
                               double* loss) {
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    if (!p || !X || !y || n < 1 || n > (1 << 24)) return ctx_fail(ctx, TNSK_ERR_INVALID, "mlp_loss_grad: arguments");
    if (!ensure_acts(p, n)) return ctx_fail(ctx, TNSK_ERR_OOM, "mlp_loss_grad: activations");
    cudaStream_t s = ctx->stream;
    cudaMemsetAsync(p->loss, 0, sizeof(double), s);
    forward(p, X, nullptr, n, false, s);
    backward(p, y, nullptr, n, s);
    if (grad) cudaMemcpyAsync(grad, p->grad, (size_t)p->n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    double h = 0;
    cudaMemcpyAsync(&h, p->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "mlp_loss_grad");
    if (loss) *loss = h;
    return TNSK_OK;
}

tnsk_status tnsk_mlp_train(tnsk_ctx* ctx, tnsk_mlp* p, const float* X, const float* y, int64_t n, int32_t epochs,
                           int32_t batch, float lr, uint64_t seed, double* final_loss) {
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    if (!p || !X || !y || n < 2 || n > (1 << 24) || epochs < 0 || batch < 1 || !(lr > 0.f))
        return ctx_fail(ctx, TNSK_ERR_INVALID, "mlp_train: arguments");
    cudaStream_t s = ctx->stream;
    // standardisation from the training set (host, FP64)
    std::vector<float> hx((size_t)n * kFeatures);
    if (cudaMemcpy(hx.data(), X, hx.size() * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, TNSK_ERR_CUDA, "mlp_train: reading X");
    }
    for (int f = 0; f < kFeatures; ++f) {
        double m = 0, v = 0;
        for (int64_t i = 0; i < n; ++i) m += hx[(size_t)(i * kFeatures + f)];
        m /= (double)n;
        for (int64_t i = 0; i < n; ++i) {
            const double d = hx[(size_t)(i * kFeatures + f)] - m;
            v += d * d;
        }
        const double sd = std::sqrt(v / (double)n);
        p->h_norm[f] = (float)m;
        p->h_norm[kFeatures + f] = sd > 1e-6 ? (float)sd : 1.f;
    }
    cudaMemcpy(p->norm, p->h_norm, sizeof(p->h_norm), cudaMemcpyHostToDevice);
    const int64_t B = std::min<int64_t>(batch, n);
    if (!ensure_acts(p, std::max<int64_t>(B, 1))) return ctx_fail(ctx, TNSK_ERR_OOM, "mlp_train: activations");
    int64_t* d_idx = nullptr;
    if (cudaMalloc((void**)&d_idx, (size_t)n * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, TNSK_ERR_OOM, "mlp_train: index buffer");
    }
    std::mt19937_64 rng(seed);
    std::vector<int64_t> perm((size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = i;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = n - 1; i > 0; --i)  // Fisher-Yates, the same order on every platform
            std::swap(perm[(size_t)i], perm[(size_t)(rng() % (uint64_t)(i + 1))]);
        // the host vector is reused next epoch: copy synchronously with the stream
        cudaMemcpyAsync(d_idx, perm.data(), (size_t)n * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        for (int64_t b0 = 0; b0 < n; b0 += B) {
            const int64_t nb = std::min<int64_t>(B, n - b0);
            forward(p, X, d_idx + b0, nb, false, s);
            backward(p, y, d_idx + b0, nb, s);
            ++p->step;
            const float c1 = 1.f - std::pow(b1, (float)p->step), c2 = 1.f - std::pow(b2, (float)p->step);
            mlp_adam_kernel<<<grid_for(p->n), 256, 0, s>>>(p->theta, p->grad, p->m1, p->m2, p->n, lr, b1, b2, eps, c1,
                                                           c2);
        }
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(d_idx);
            return ctx_cuda_fail(ctx, e, "mlp_train");
        }
    }
    cudaFree(d_idx);
    if (final_loss) {  // mean squared error over the whole training set, in chunks
        double tot = 0.0;
        for (int64_t b0 = 0; b0 < n; b0 += B) {
            const int64_t nb = std::min<int64_t>(B, n - b0);
            cudaMemsetAsync(p->loss, 0, sizeof(double), s);
            forward(p, X + b0 * kFeatures, nullptr, nb, false, s);
            mlp_mse_kernel<<<grid_for(nb), 256, 0, s>>>(p->out[kLayers - 1], y + b0, nullptr, (int)nb, p->d0, p->loss);
            double h = 0;
            cudaMemcpyAsync(&h, p->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "mlp_train: loss");
            tot += h * (double)nb;
        }
        *final_loss = tot / (double)n;
    }
    return TNSK_OK;
}

tnsk_status tnsk_mlp_predict(tnsk_ctx* ctx, tnsk_mlp* p, const float* X, int64_t n, float* y, int32_t bf16) {
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    if (!p || (n > 0 && (!X || !y)) || n < 0) return ctx_fail(ctx, TNSK_ERR_INVALID, "mlp_predict: arguments");
    const int64_t chunk = 65536;
    if (!ensure_acts(p, std::min<int64_t>(std::max<int64_t>(n, 1), chunk)))
        return ctx_fail(ctx, TNSK_ERR_OOM, "mlp_predict: activations");
    cudaStream_t s = ctx->stream;
    for (int64_t b0 = 0; b0 < n; b0 += chunk) {
        const int64_t nb = std::min<int64_t>(chunk, n - b0);
        forward(p, X + b0 * kFeatures, nullptr, nb, bf16 != 0, s);
        cudaMemcpyAsync(y + b0, p->out[kLayers - 1], (size_t)nb * sizeof(float), cudaMemcpyDeviceToDevice, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "mlp_predict");
    return TNSK_OK;
}

// file: "TNSKMLP1", int32 features, int32 hidden, int64 parameters, float mu[F],
// float sigma[F], float theta[parameters] (little-endian, as written by this library)
tnsk_status tnsk_mlp_save(tnsk_mlp* p, const char* path) {
    if (!p || !path) return TNSK_ERR_INVALID;
    std::vector<float> th((size_t)p->n);
    float nm[2 * kFeatures];
    tnsk_status st = tnsk_mlp_get(p, th.data(), nm);
    if (st != TNSK_OK) return st;
    FILE* f = std::fopen(path, "wb");
    if (!f) return TNSK_ERR_INVALID;
    const int32_t hdr[2] = {kFeatures, kHidden};
    const int64_t n = p->n;
    bool ok = std::fwrite("TNSKMLP1", 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              std::fwrite(&n, sizeof(n), 1, f) == 1 && std::fwrite(nm, sizeof(nm), 1, f) == 1 &&
              std::fwrite(th.data(), sizeof(float), th.size(), f) == th.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? TNSK_OK : TNSK_ERR_INVALID;
}

tnsk_status tnsk_mlp_load(tnsk_ctx* ctx, tnsk_mlp* p, const char* path) {
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    if (!p || !path) return ctx_fail(ctx, TNSK_ERR_INVALID, "mlp_load: NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return ctx_fail(ctx, TNSK_ERR_INVALID, std::string("mlp_load: cannot open ") + path);
    char magic[8];
    int32_t hdr[2];
    int64_t n = 0;
    float nm[2 * kFeatures];
    std::vector<float> th((size_t)p->n);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "TNSKMLP1", 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == kFeatures && hdr[1] == kHidden &&
              std::fread(&n, sizeof(n), 1, f) == 1 && n == p->n && std::fread(nm, sizeof(nm), 1, f) == 1 &&
              std::fread(th.data(), sizeof(float), th.size(), f) == th.size();
    std::fclose(f);
    if (!ok) return ctx_fail(ctx, TNSK_ERR_INVALID, std::string("mlp_load: not a predictor file of this shape: ") + path);
    return tnsk_mlp_set(ctx, p, th.data(), nm);
}

}  // extern "C"

namespace {

// Features of a network at sketch size m and R reps (the predictor's inputs):
// p, t, cycle rank t - p + components, log2 of the largest and mean log2 of the
// contraction dims, mean and standard deviation of ln ||X_k||_F, log2 m, log2 R.
// net_structure fills all but the two norm features (5, 6) and validates the network.
tnsk_status net_structure(tnsk_ctx* ctx, const tnsk_network& net, const tnsk_params& prm, NetInfo& I, float* feat) {
    std::string why;
    tnsk_params q = prm;
    q.m = 1;  // the features take log2 m from prm; validation needs any valid m
    tnsk_status st = validate(net, q, I, why);
    if (st != TNSK_OK) return ctx_fail(ctx, st, why);
    for (int k = 0; k < I.p; ++k)
        if (I.rung[k]) return ctx_fail(ctx, TNSK_ERR_UNSUPPORTED, "features: grouped (rung) tensors have no stored entries");
    // connected components of the tensors joined by contractions
    std::vector<int> parent(I.p);
    for (int k = 0; k < I.p; ++k) parent[k] = k;
    auto find = [&](int x) {
        while (parent[x] != x) x = parent[x] = parent[parent[x]];
        return x;
    };
    double lmax = 0.0, lsum = 0.0;
    for (int e = 0; e < I.t; ++e) {
        const int u = net.edges[2 * e], v = net.edges[2 * e + 1];
        parent[find(I.tensor_of[u])] = find(I.tensor_of[v]);
        const double l = std::log2((double)std::max<int64_t>(I.dims[u], 1));
        lmax = std::max(lmax, l);
        lsum += l;
    }
    int comps = 0;
    for (int k = 0; k < I.p; ++k) comps += find(k) == k;
    feat[0] = (float)I.p;
    feat[1] = (float)I.t;
    feat[2] = (float)(I.t - I.p + comps);
    feat[3] = (float)lmax;
    feat[4] = I.t > 0 ? (float)(lsum / I.t) : 0.f;
    feat[5] = feat[6] = 0.f;
    feat[7] = (float)std::log2((double)std::max<int64_t>(prm.m, 1));
    feat[8] = (float)std::log2((double)std::max(prm.reps, 1));
    return TNSK_OK;
}

// Features 5 and 6 from the sums of squares ss[k] of the network's p tensors.
void norm_features(int p, const double* ss, float* feat) {
    double mean = 0.0, var = 0.0;
    std::vector<double> ln(p);
    for (int k = 0; k < p; ++k) {
        ln[k] = 0.5 * std::log(std::max(ss[k], 1e-300));
        mean += ln[k];
    }
    mean /= std::max(p, 1);
    for (int k = 0; k < p; ++k) var += (ln[k] - mean) * (ln[k] - mean);
    var /= std::max(p, 1);
    feat[5] = (float)mean;
    feat[6] = (float)std::sqrt(var);
}

// One sum of squares per job (FP64), in one launch and one synchronisation.
tnsk_status batch_sumsq(tnsk_ctx* ctx, std::vector<SqJob>& jobs, std::vector<double>& ss) {
    ss.assign(jobs.size(), 0.0);
    if (jobs.empty()) return TNSK_OK;
    int64_t nchunks = 0;
    for (auto& j : jobs) {
        j.chunk0 = nchunks;
        nchunks += (j.n + kSqChunk - 1) / kSqChunk;
    }
    const size_t jb = (jobs.size() * sizeof(SqJob) + 15) / 16 * 16;
    tnsk_status st = ctx_ensure_work(ctx, jb + jobs.size() * sizeof(double));
    if (st != TNSK_OK) return st;
    unsigned char* d = ctx->work;
    double* dout = (double*)(d + jb);
    cudaMemcpyAsync(d, jobs.data(), jobs.size() * sizeof(SqJob), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemsetAsync(dout, 0, jobs.size() * sizeof(double), ctx->stream);
    if (nchunks > 0) {
        const int grid = (int)std::min<int64_t>(nchunks, 4096);
        sumsq_batch_kernel<<<grid, 256, 0, ctx->stream>>>((const SqJob*)d, (int)jobs.size(), nchunks, dout);
    }
    cudaMemcpyAsync(ss.data(), dout, jobs.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    const cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "features");
    return TNSK_OK;
}

void push_jobs(const tnsk_network& net, const NetInfo& I, std::vector<SqJob>& jobs) {
    for (int k = 0; k < I.p; ++k) jobs.push_back(SqJob{net.X[k].data, I.numel[k], 0, net.X[k].dtype, 0});
}

tnsk_status network_features(tnsk_ctx* ctx, const tnsk_network& net, const tnsk_params& prm, NetInfo& I,
                             float* feat) {
    tnsk_status st = net_structure(ctx, net, prm, I, feat);
    if (st != TNSK_OK) return st;
    std::vector<SqJob> jobs;
    push_jobs(net, I, jobs);
    std::vector<double> ss;
    st = batch_sumsq(ctx, jobs, ss);
    if (st != TNSK_OK) return st;
    norm_features(I.p, ss.data(), feat);
    return TNSK_OK;
}

}  // namespace

extern "C" {

tnsk_status tnsk_features(tnsk_ctx* ctx, const tnsk_network* net, const tnsk_params* params, float* features) {
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    if (!net || !params || !features) return ctx_fail(ctx, TNSK_ERR_INVALID, "features: NULL argument");
    NetInfo I;
    return network_features(ctx, *net, *params, I, features);
}

tnsk_status tnsk_choose_params(tnsk_ctx* ctx, const tnsk_network* net, double target_err, tnsk_mlp* mlp,
                               tnsk_params* inout, double* predicted_err) {
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    if (!net || !inout || !(target_err > 0.0)) return ctx_fail(ctx, TNSK_ERR_INVALID, "choose_params: arguments");
    constexpr int kLo = 6, kHi = 16;  // candidate m = 2^6 .. 2^16
    const double R = std::max(inout->reps, 1);
    if (inout->method == TNSK_CROSSCORR)
        return ctx_fail(ctx, TNSK_ERR_UNSUPPORTED,
                        "choose_params: the cross-correlation estimator has no variance bound (biased on cycles)");
    if (!mlp || inout->method != TNSK_GENERAL) {
        // the variance bound with delta = 0.1: m R >= 3^t / (eps^2 delta) (general), 32 t / (eps^2 delta) (acyclic)
        NetInfo I;
        std::string why;
        tnsk_params q = *inout;
        q.m = 1;
        st = validate(*net, q, I, why);
        if (st != TNSK_OK) return ctx_fail(ctx, st, why);
        const double delta = 0.1;
        const double num = inout->method == TNSK_GENERAL ? std::pow(3.0, I.t) : 32.0 * I.t;
        for (int l = kLo; l <= kHi; ++l) {
            const double m = std::ldexp(1.0, l);
            const double eps = std::sqrt(num / (m * R * delta));
            if (eps <= target_err || l == kHi) {
                if (predicted_err) *predicted_err = eps;
                if (eps > target_err) return ctx_fail(ctx, TNSK_ERR_UNREACHABLE, "choose_params: bound not met at m = 2^16");
                inout->m = (int64_t)1 << l;
                return TNSK_OK;
            }
        }
    }
    float base[kFeatures];
    NetInfo I;
    st = network_features(ctx, *net, *inout, I, base);
    if (st != TNSK_OK) return st;
    const int nc = kHi - kLo + 1;
    std::vector<float> hx((size_t)nc * kFeatures), hy(nc);
    for (int c = 0; c < nc; ++c) {
        std::memcpy(&hx[(size_t)c * kFeatures], base, sizeof(base));
        hx[(size_t)c * kFeatures + 7] = (float)(kLo + c);
    }
    st = ctx_ensure_work(ctx, (hx.size() + hy.size()) * sizeof(float));
    if (st != TNSK_OK) return st;
    float* d = (float*)ctx->work;
    cudaMemcpyAsync(d, hx.data(), hx.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    st = tnsk_mlp_predict(ctx, mlp, d, nc, d + hx.size(), 1);
    if (st == TNSK_OK) {
        cudaMemcpyAsync(hy.data(), d + hx.size(), hy.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = ctx_cuda_fail(ctx, e, "choose_params");
    }
    if (st != TNSK_OK) return st;
    // The predictor gives the expected log10 of one estimate's relative error. With
    // the estimate's error ~ sigma Z (a mean of reps; Z standard normal),
    // E log10 |Z| = -(gamma + ln 2) / (2 ln 10) = -0.2757 and P(|Z| <= 1.6449) = 0.9,
    // so the error's 90% quantile is 10^(pred + 0.2757 + log10 1.6449) = 10^pred / 0.3224;
    // that quantile must meet the target. The smallest such m wins.
    constexpr double kQuantile90 = 1.0 / 0.3224;
    double best = 1e300;
    for (int c = 0; c < nc; ++c) {
        const double err = std::pow(10.0, (double)hy[c]) * kQuantile90;
        best = std::min(best, err);
        if (err <= target_err) {
            inout->m = (int64_t)1 << (kLo + c);
            if (predicted_err) *predicted_err = err;
            return TNSK_OK;
        }
    }
    if (predicted_err) *predicted_err = best;
    return ctx_fail(ctx, TNSK_ERR_UNREACHABLE, "choose_params: no m <= 2^16 meets the target");
}

}  // extern "C"

namespace {

// The sizing policies of a batch (tnsk_choose_params_batch, tnsk_choose_params_rate).
// Both see every candidate (m, R), m = 2^6 .. 2^16 and R in {16, 32, 64}, through the
// same normal model of one estimate's relative error, sigma |Z|: from the learned
// predictor (log10 sigma = prediction + 0.2757, since E log10 |Z| = -0.2757), or from a
// pilot (sigma = s / |mean|, s^2 the pilot's per-rep variance taken one standard error
// up and scaled by 2^12 / (m R)). Its 90% quantile is 1.6449 sigma. The cost of a
// candidate is R (sum_k q_k N_k + p m log2 m).
// quantile policy (rate = false): the cheapest candidate whose 90% quantile meets the
//   target; predictor first, the pilot for the networks it leaves, else flagged;
// rate policy (rate = true): the candidates that maximise the batch's expected number
//   of estimates within the target per unit of cost, sum_b P_b / sum_b cost_b with
//   P = erf(target / (sigma sqrt 2)) (Dinkelbach's iteration); the pilot only for
//   networks without a prediction; flagged where the chosen chance is below 1/2.
tnsk_status choose_batch(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, double target_err, tnsk_mlp* mlp,
                         int32_t pilot_reps, tnsk_params* inout, double* predicted_err, int32_t* how, bool rate) {
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    const char* who = rate ? "choose_params_rate" : "choose_params_batch";
    if (B < 0 || (B > 0 && (!nets || !inout || !predicted_err || !how)) || !(target_err > 0.0) || pilot_reps < 0 ||
        pilot_reps == 1 || pilot_reps > 4096)
        return ctx_fail(ctx, TNSK_ERR_INVALID, std::string(who) + ": arguments");
    constexpr int kLo = 6, kHi = 16, kPilotLog2m = 12;
    // R from 16 up: the normal quantile of the mean is not trusted below (heavy tails)
    static const int kReps[] = {16, 32, 64};
    constexpr int nR = 3, nL = kHi - kLo + 1, nO = nL * nR;
    constexpr double kZ90 = 1.6449;         // P(|Z| <= 1.6449) = 0.9
    constexpr double kGeoZ = 0.2757;        // -E log10 |Z|
    std::vector<double> work(B, 0.0);  // sum_k q_k N_k
    std::vector<int> pterms(B, 0);
    // sigma of every candidate (o = (l - kLo) nR + j), +inf where nothing predicts it
    std::vector<double> sig((size_t)B * nO, HUGE_VAL);
    std::vector<char> predicted(B, 0);
    // ---- the learned predictor (method 1 networks)
    std::vector<float> hx;
    std::vector<int> rows_of;  // network of each block of nL * nR rows
    std::vector<float> bases;  // features of those networks (norm features filled below)
    std::vector<SqJob> jobs;   // their tensors, for one batched norm pass
    for (int b = 0; b < B; ++b) {
        if (inout[b].method == TNSK_CROSSCORR)
            return ctx_fail(ctx, TNSK_ERR_UNSUPPORTED, std::string(who) + ": the cross-correlation estimator");
        NetInfo I;
        float base[kFeatures];
        tnsk_params q = inout[b];
        q.reps = 16;
        if (mlp && inout[b].method == TNSK_GENERAL) {
            st = net_structure(ctx, nets[b], q, I, base);
            if (st != TNSK_OK) return st;
            rows_of.push_back(b);
            bases.insert(bases.end(), base, base + kFeatures);
            push_jobs(nets[b], I, jobs);
        } else {
            std::string why;
            q.m = 1;
            st = validate(nets[b], q, I, why);
            if (st != TNSK_OK) return ctx_fail(ctx, st, "network " + std::to_string(b) + ": " + why);
        }
        for (int k = 0; k < I.p; ++k)
            work[b] += (double)(I.mode_off[k + 1] - I.mode_off[k]) * (double)I.numel[k];
        pterms[b] = I.p;
    }
    if (!rows_of.empty()) {
        std::vector<double> ss;
        st = batch_sumsq(ctx, jobs, ss);
        if (st != TNSK_OK) return st;
        size_t at_ss = 0;
        for (size_t i = 0; i < rows_of.size(); ++i) {
            float* base = &bases[i * kFeatures];
            norm_features(pterms[rows_of[i]], ss.data() + at_ss, base);
            at_ss += pterms[rows_of[i]];
            for (int l = kLo; l <= kHi; ++l)
                for (int j = 0; j < nR; ++j) {
                    const size_t at = hx.size();
                    hx.insert(hx.end(), base, base + kFeatures);
                    hx[at + 7] = (float)l;
                    hx[at + 8] = (float)std::log2((double)kReps[j]);
                }
        }
        const size_t n = hx.size() / kFeatures;
        st = ctx_ensure_work(ctx, (hx.size() + n) * sizeof(float));
        if (st != TNSK_OK) return st;
        float* d = (float*)ctx->work;
        std::vector<float> hy(n);
        cudaMemcpyAsync(d, hx.data(), hx.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
        st = tnsk_mlp_predict(ctx, mlp, d, (int64_t)n, d + hx.size(), 1);
        if (st == TNSK_OK) {
            cudaMemcpyAsync(hy.data(), d + hx.size(), n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
            const cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) st = ctx_cuda_fail(ctx, e, who);
        }
        if (st != TNSK_OK) return st;
        for (size_t i = 0; i < rows_of.size(); ++i) {
            const int b = rows_of[i];
            predicted[b] = 1;
            for (int o = 0; o < nO; ++o) sig[(size_t)b * nO + o] = std::pow(10.0, (double)hy[i * nO + o] + kGeoZ);
        }
    }
    auto cost = [&](int b, int o) {
        const int l = kLo + o / nR, R = kReps[o % nR];
        return (double)R * (work[b] + (double)pterms[b] * std::ldexp(1.0, l) * (double)l);
    };
    // the cheapest candidate whose 90% quantile meets the target, -1 if none
    auto cheapest_meeting = [&](int b) {
        int best = -1;
        for (int o = 0; o < nO; ++o)
            if (kZ90 * sig[(size_t)b * nO + o] <= target_err && (best < 0 || cost(b, o) < cost(b, best))) best = o;
        return best;
    };
    for (int b = 0; b < B; ++b) how[b] = 2;
    // ---- the pilot: pilot_reps repetitions at m = 2^12 of the networks the predictor
    // leaves (no prediction; for the quantile policy also no candidate meeting the
    // target), in one batch; the per-rep variance scales as 1/m (both variance
    // lemmas), the mean of R reps as 1/R
    std::vector<int> pil;
    for (int b = 0; b < B; ++b)
        if (pilot_reps > 0 && (!predicted[b] || (!rate && cheapest_meeting(b) < 0))) pil.push_back(b);
    std::vector<char> piloted(B, 0);
    if (!pil.empty()) {
        const int P = (int)pil.size();
        const size_t nd = (size_t)P * (pilot_reps + 1);
        st = ctx_ensure_work(ctx, nd * sizeof(double));
        if (st != TNSK_OK) return st;
        double* d = (double*)ctx->work;
        std::vector<tnsk_network> pn(P);
        std::vector<tnsk_params> pp(P);
        std::vector<double*> po(P), pr(P);
        for (int i = 0; i < P; ++i) {
            pn[i] = nets[pil[i]];
            pp[i] = inout[pil[i]];
            pp[i].m = (int64_t)1 << kPilotLog2m;
            pp[i].reps = pilot_reps;
            pp[i].groups = 1;
            pp[i].rep0 = 1 << 20;  // repetitions apart from those of the estimate itself
            po[i] = d + (size_t)i * (pilot_reps + 1);
            pr[i] = po[i] + 1;
        }
        st = tnsk_estimate_batch(ctx, P, pn.data(), pp.data(), po.data(), pr.data());
        std::vector<double> h(nd);
        if (st == TNSK_OK) {
            cudaMemcpyAsync(h.data(), d, nd * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
            const cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) st = ctx_cuda_fail(ctx, e, who);
        }
        if (st != TNSK_OK) return st;
        for (int i = 0; i < P; ++i) {
            const int b = pil[i];
            const double* y = h.data() + (size_t)i * (pilot_reps + 1) + 1;
            double mean = 0.0, var = 0.0;
            for (int r = 0; r < pilot_reps; ++r) mean += y[r];
            mean /= pilot_reps;
            for (int r = 0; r < pilot_reps; ++r) var += (y[r] - mean) * (y[r] - mean);
            var /= (pilot_reps - 1);
            // one standard error up (a normal sample variance has relative error sqrt(2/(n-1))),
            // so a pilot that happens to see a small spread does not undersize
            var *= 1.0 + std::sqrt(2.0 / (pilot_reps - 1));
            piloted[b] = 1;
            for (int o = 0; o < nO; ++o) {
                const int l = kLo + o / nR;
                const double sd = std::sqrt(var * std::ldexp(1.0, kPilotLog2m - l) / kReps[o % nR]);
                sig[(size_t)b * nO + o] = mean != 0.0 ? sd / std::fabs(mean) : HUGE_VAL;
            }
        }
    }
    std::vector<int> pick(B, 0);  // candidate per network (0: the cheapest, m = 2^6, R = 16)
    if (!rate) {
        for (int b = 0; b < B; ++b) {
            const int o = cheapest_meeting(b);
            if (o >= 0) {
                pick[b] = o;
                how[b] = piloted[b] ? 1 : 0;
            }
        }
    } else {
        // Dinkelbach's iteration for max sum P / sum cost: with lambda the current ratio,
        // each network takes the candidate maximising P - lambda cost; the new ratio is at
        // least the old one, and a repeat of it ends the iteration
        std::vector<double> chance((size_t)B * nO);
        for (size_t i = 0; i < chance.size(); ++i)
            chance[i] = std::isfinite(sig[i]) ? std::erf(target_err / (sig[i] * std::sqrt(2.0))) : 0.0;
        double lambda = 0.0;
        for (int it = 0; it < 64; ++it) {
            double num = 0.0, den = 0.0;
            for (int b = 0; b < B; ++b) {
                int best = 0;
                double bv = -HUGE_VAL;
                for (int o = 0; o < nO; ++o) {
                    const double v = chance[(size_t)b * nO + o] - lambda * cost(b, o);
                    if (v > bv || (v == bv && cost(b, o) < cost(b, best))) bv = v, best = o;
                }
                pick[b] = best;
                num += chance[(size_t)b * nO + best];
                den += cost(b, best);
            }
            const double next = den > 0.0 ? num / den : 0.0;
            if (!(next > lambda * (1.0 + 1e-12))) break;
            lambda = next;
        }
        for (int b = 0; b < B; ++b)
            if (chance[(size_t)b * nO + pick[b]] >= 0.5) how[b] = piloted[b] ? 1 : 0;
    }
    for (int b = 0; b < B; ++b) {
        const int o = how[b] == 2 && !rate ? 0 : pick[b];
        inout[b].m = (int64_t)1 << (kLo + o / nR);
        inout[b].reps = kReps[o % nR];
        inout[b].groups = 1;
        if (how[b] != 2 || rate) {
            const double e = kZ90 * sig[(size_t)b * nO + o];
            predicted_err[b] = std::isfinite(e) ? e : 1e300;
        } else {  // flagged: the best candidate's 90% quantile
            double best = HUGE_VAL;
            for (int q = 0; q < nO; ++q) best = std::min(best, kZ90 * sig[(size_t)b * nO + q]);
            predicted_err[b] = std::isfinite(best) ? best : 1e300;
        }
    }
    return TNSK_OK;
}

}  // namespace

extern "C" {

tnsk_status tnsk_choose_params_batch(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, double target_err,
                                     tnsk_mlp* mlp, int32_t pilot_reps, tnsk_params* inout, double* predicted_err,
                                     int32_t* how) {
    return choose_batch(ctx, B, nets, target_err, mlp, pilot_reps, inout, predicted_err, how, false);
}

tnsk_status tnsk_choose_params_rate(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, double target_err,
                                    tnsk_mlp* mlp, int32_t pilot_reps, tnsk_params* inout, double* predicted_err,
                                    int32_t* how) {
    return choose_batch(ctx, B, nets, target_err, mlp, pilot_reps, inout, predicted_err, how, true);
}

}  // extern "C"
