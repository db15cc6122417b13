// streams.cu -- turnstile updates of stored method-1 sketches (Sec. 4.2: the sketches
// x_k are kept, so the general turnstile model is served by applying each update to
// every repetition's sketch in O(q_k)); the sparse input path and the join-size
// application feed all-zero tensors through the same kernel, and the diagonal copy
// tensors of WLOG 1 are sketched the same way from their n nonzeros.
#include <algorithm>

#include "kernels.cuh"
#include "plan.cuh"

namespace tnsk {

// ---------------------------------------------------------------------------
// Turnstile updates (Sec. 4.2: the sketches x_k are stored, so an update X_k(i) += delta
// changes every rep's sketch by sigma(i) delta at bin b(i), in O(q_k)): one thread per
// (update, rep), the reps of one update in neighbouring threads (same entry, same table
// offsets). Updates with a tensor or entry index out of range set the bounds flag and
// change nothing.
// ---------------------------------------------------------------------------
template <typename AccT>
__global__ void __launch_bounds__(256) m1_update_kernel(const M1Tensor* __restrict__ tens,
                                                        const M1Net* __restrict__ nets,
                                                        const uint32_t* __restrict__ tabs, AccT* __restrict__ xs,
                                                        int64_t n, const int32_t* __restrict__ tk,
                                                        const int64_t* __restrict__ ti,
                                                        const double* __restrict__ dv, int* __restrict__ err) {
    const M1Net& N = nets[0];
    const int R = N.R;
    const uint32_t mask = (uint32_t)(N.m - 1);
    const int64_t total = n * R;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = g / R;
        const int r = (int)(g - u * R);
        const int k = tk[u];
        const int64_t i = ti[u];
        if (k < 0 || k >= N.p) {
            atomicExch(err, DEVERR_BOUNDS);
            continue;
        }
        const M1Tensor& T = tens[N.t0 + k];
        if (i < 0 || i >= T.numel) {
            atomicExch(err, DEVERR_BOUNDS);
            continue;
        }
        const uint32_t* tabr = tabs + N.tab_off + (int64_t)r * N.L;
        uint32_t h = 0;
        int64_t o = 0, rem = i;
        for (int d = T.order - 1; d >= 0; --d) {
            const int64_t q = rem / T.dims[d];
            const int dig = (int)(rem - q * T.dims[d]);
            rem = q;
            if (T.tab[d] >= 0) {
                uint32_t w = tabr[T.tab[d] + dig];
                if (T.comp[d]) w = ((((uint32_t)N.m) - (w & mask)) & mask) | (w & TNSK_SIGN_BIT);
                h += w;
            } else {
                o += (int64_t)dig * T.ostride[d];
            }
        }
        const AccT v = (AccT)dv[u];
        atomicAdd(&xs[N.x_off + (int64_t)r * N.X + T.xoff + o * N.m + (h & mask)], (h & TNSK_SIGN_BIT) ? -v : v);
    }
}

cudaError_t launch_m1_updates(const BatchPlan& plan, unsigned char* base, int64_t n, const int32_t* tensor,
                              const int64_t* index, const double* delta, bool fp64, int* err, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const M1Tensor* tens = (const M1Tensor*)(base + plan.m1.tens_off);
    const M1Net* nets = (const M1Net*)(base + plan.m1.nets_off);
    const uint32_t* tabs = (const uint32_t*)(base + plan.tabs_off);
    const int64_t total = n * (int64_t)plan.m1_reps;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
    if (fp64)
        m1_update_kernel<double><<<blocks, 256, 0, s>>>(tens, nets, tabs, (double*)(base + plan.m1.xs_off), n, tensor,
                                                        index, delta, err);
    else
        m1_update_kernel<float><<<blocks, 256, 0, s>>>(tens, nets, tabs, (float*)(base + plan.m1.xs_off), n, tensor,
                                                       index, delta, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagonal copy tensors of WLOG 1 (Sec. 4.1): delta(i, ..., i) = 1 for i < n, never
// stored. Each of its n nonzeros adds sigma_r(i) at bin b_r(i) of every rep's sketch,
// like an update of value 1 (all modes contracted, all at index i): one thread per
// (entry, rep), blockIdx.y the copy tensor.
// ---------------------------------------------------------------------------
template <typename AccT>
__global__ void __launch_bounds__(256) m1_diag_kernel(const M1Tensor* __restrict__ tens,
                                                      const M1Net* __restrict__ nets,
                                                      const uint32_t* __restrict__ tabs, AccT* __restrict__ xs,
                                                      const M1Diag* __restrict__ items) {
    const M1Diag it = items[blockIdx.y];
    const M1Tensor& T = tens[it.tensor];
    const M1Net& N = nets[it.net];
    const int R = N.R;
    const uint32_t mask = (uint32_t)(N.m - 1);
    const int64_t total = it.n * R;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = g / R;
        const int r = (int)(g - i * R);
        const uint32_t* tabr = tabs + N.tab_off + (int64_t)r * N.L;
        uint32_t h = 0;  // bins add below bit 24 (at most 12 modes of < 2^16), sign bits by parity
        for (int d = 0; d < T.order; ++d) {
            uint32_t w = tabr[T.tab[d] + i];
            if (T.comp[d]) w = ((((uint32_t)N.m) - (w & mask)) & mask) | (w & TNSK_SIGN_BIT);
            h += w;
        }
        atomicAdd(&xs[N.x_off + (int64_t)r * N.X + T.xoff + (h & mask)], (h & TNSK_SIGN_BIT) ? (AccT)-1 : (AccT)1);
    }
}

cudaError_t launch_m1_diag(const BatchPlan& plan, unsigned char* base, void* xs, bool fp64, cudaStream_t s) {
    if (plan.m1.n_diag <= 0) return cudaSuccess;
    const M1Tensor* tens = (const M1Tensor*)(base + plan.m1.tens_off);
    const M1Net* nets = (const M1Net*)(base + plan.m1.nets_off);
    const uint32_t* tabs = (const uint32_t*)(base + plan.tabs_off);
    const M1Diag* items = (const M1Diag*)(base + plan.m1.diag_off);
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((plan.m1.diag_most + 255) / 256, 2048));
    for (int first = 0; first < plan.m1.n_diag; first += 65535) {
        const unsigned gy = (unsigned)std::min(65535, plan.m1.n_diag - first);
        if (fp64)
            m1_diag_kernel<double><<<dim3(gx, gy), 256, 0, s>>>(tens, nets, tabs, (double*)xs, items + first);
        else
            m1_diag_kernel<float><<<dim3(gx, gy), 256, 0, s>>>(tens, nets, tabs, (float*)xs, items + first);
    }
    return cudaGetLastError();
}

}  // namespace tnsk
