// method1.cu -- method 1 of the paper (Sec. 4.2, Eq. 1, Alg. 1): complement count
// sketches on every contraction, one tensor sketch per tensor, composition in
// the Fourier domain.
//
//   a2  m1_scatter_kernel   x_k[r] = T_k vec(X_k): signed scatter-add by the hash
//                           form of the tensor sketch (Alg. 3), shared-memory
//                           privatised bins for a batch of repetitions
//   a3  m1_spectrum_kernel  F x_k by a shared-memory real FFT
//   a4                      y_r = (1/m) sum_j prod_k (F x_k)(j) (Alg. 1 last line;
//                           open output entries per Corollary "full-to-partial-tc")
//   a9  combine_kernel      median of group means in FP64 (Theorem 1)
#include "fft.cuh"
#include "kernels.cuh"

namespace tnsk {

// ---------------------------------------------------------------------------
// a2: scatter
// ---------------------------------------------------------------------------
// Shared memory: [nrep][TT] packed table words (complement applied), then the
// privatised bins [nrep][O][m] when w.priv. TT = sum of the contracted dims.
template <typename AccT, typename IdxT>
__global__ void __launch_bounds__(256) m1_scatter_kernel(const M1Tensor* __restrict__ tens,
                                                         const M1Net* __restrict__ nets,
                                                         const M1Work* __restrict__ work,
                                                         const uint32_t* __restrict__ tabs, AccT* __restrict__ xs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ M1Tensor sT;
    __shared__ int32_t sbase[TNSK_MAX_ORDER];
    __shared__ int32_t sTT;
    const M1Work w = work[blockIdx.x];
    if (threadIdx.x == 0) {
        sT = tens[w.tensor];
        int acc = 0;
        for (int d = 0; d < TNSK_MAX_ORDER; ++d) {
            sbase[d] = acc;
            if (d < sT.order && sT.tab[d] >= 0) acc += sT.dims[d];
        }
        sTT = acc;
    }
    __syncthreads();
    const M1Net& N = nets[sT.net];
    const int64_t m = N.m;
    const uint32_t mask = (uint32_t)(m - 1);
    const int TT = sTT;
    const int nrep = w.nrep;
    const int order = sT.order;
    uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem_raw);
    AccT* s_bin = reinterpret_cast<AccT*>(smem_raw + (((size_t)nrep * TT * 4 + 15) & ~(size_t)15));

    // tables of this tensor's contracted modes for the batch of reps
    const int64_t tab_words = (int64_t)nrep * TT;
    for (int64_t q = threadIdx.x; q < tab_words; q += blockDim.x) {
        int r = (int)(q / TT);
        int loc = (int)(q - (int64_t)r * TT);
        int d = 0;
        for (int dd = 0; dd < order; ++dd)
            if (sT.tab[dd] >= 0 && loc >= sbase[dd] && loc < sbase[dd] + sT.dims[dd]) d = dd;
        int i = loc - sbase[d];
        uint32_t word = tabs[N.tab_off + (int64_t)(w.rep0 + r) * N.L + sT.tab[d] + i];
        if (sT.comp[d]) word = (((uint32_t)m - (word & mask)) & mask) | (word & TNSK_SIGN_BIT);
        s_tab[q] = word;
    }
    const int64_t O = sT.O;
    const int64_t nbins = (int64_t)nrep * O * m;
    if (w.priv)
        for (int64_t q = threadIdx.x; q < nbins; q += blockDim.x) s_bin[q] = AccT(0);
    __syncthreads();

    AccT* gx = xs + N.x_off + sT.xoff;  // + (rep0 + r) * N.X + o * m + b
    for (int64_t f = w.begin + threadIdx.x; f < w.end; f += blockDim.x) {
        const AccT v = load_as<AccT>(sT.data, sT.dtype, f);
        int32_t midx[TNSK_MAX_ORDER];
        int64_t o = 0;
        IdxT rem = (IdxT)f;
#pragma unroll
        for (int d = TNSK_MAX_ORDER - 1; d >= 0; --d) {
            if (d < order) {
                IdxT n = (IdxT)sT.dims[d];
                IdxT qt = rem / n;
                int i = (int)(rem - qt * n);
                rem = qt;
                midx[d] = sbase[d] + i;
                o += (int64_t)i * sT.ostride[d];
            }
        }
        for (int r = 0; r < nrep; ++r) {
            uint32_t h = 0;
            const uint32_t* tr = s_tab + r * TT;
#pragma unroll
            for (int d = 0; d < TNSK_MAX_ORDER; ++d)
                if (d < order && sT.tab[d] >= 0) h += tr[midx[d]];
            const AccT sv = (h & TNSK_SIGN_BIT) ? -v : v;
            const uint32_t b = h & mask;
            if (w.priv)
                atomicAdd(&s_bin[((int64_t)r * O + o) * m + b], sv);
            else
                atomicAdd(&gx[(int64_t)(w.rep0 + r) * N.X + o * m + b], sv);
        }
    }
    if (!w.priv) return;
    __syncthreads();
    for (int64_t q = threadIdx.x; q < nbins; q += blockDim.x) {
        AccT val = s_bin[q];
        if (val != AccT(0)) {
            int64_t r = q / (O * m);
            int64_t ob = q - r * (O * m);
            atomicAdd(&gx[(int64_t)(w.rep0 + r) * N.X + ob], val);
        }
    }
}

// ---------------------------------------------------------------------------
// a3 + a4: spectra, Hadamard product, bin sum
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T block_max(T v, T* red) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, s));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : T(0);
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, s));
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    T r = red[0];
    __syncthreads();
    return r;
}

// Loads sketch x (length m) as packed complex z[n] = x[2n] + i x[2n+1] (m >= 2) or
// z[0] = x[0] (m = 1), FFTs it, and leaves its power-of-two exponent e (so that
// 2^-e F x has entries of magnitude < 1) in *s_e. All threads must call.
template <typename T>
__device__ void load_fft_scale(const T* __restrict__ x, int64_t m, int log2m, Cplx<T>* z,
                               const Cplx<T>* __restrict__ tw, T* red, int* s_e) {
    const int log2M = log2m > 0 ? log2m - 1 : 0;
    const int M = 1 << log2M;
    if (m == 1) {
        if (threadIdx.x == 0) z[0] = {x[0], T(0)};
    } else {
        for (int n = threadIdx.x; n < M; n += blockDim.x) z[n] = {x[2 * n], x[2 * n + 1]};
    }
    __syncthreads();
    if (m > 1) block_fft_dif(z, 1, log2M, tw);
    const int K = m == 1 ? 1 : M + 1;
    T mx = T(0);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        Cplx<T> X = m == 1 ? z[0] : unpack_bin(z, k, log2M, tw);
        mx = fmax(mx, fmax(fabs(X.x), fabs(X.y)));
    }
    mx = block_max(mx, red);
    if (threadIdx.x == 0) {
        int e = 0;
        if (mx > T(0)) frexp(mx, &e);
        *s_e = e;
    }
    __syncthreads();
}

// One CTA per (network, rep). Shared memory: z [M] and P [M+1] complex (T).
template <typename T>
__global__ void __launch_bounds__(256) m1_spectrum_kernel(const M1Tensor* __restrict__ tens,
                                                          const M1Net* __restrict__ nets,
                                                          const OpenMode* __restrict__ opens,
                                                          const int2* __restrict__ items, const T* __restrict__ xs,
                                                          const Cplx<T>* const* __restrict__ tws,
                                                          Cplx<T>* __restrict__ spec, int* __restrict__ sexp,
                                                          double* __restrict__ yrep) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[32];
    __shared__ int s_e;
    __shared__ double dred[32];
    const int2 it = items[blockIdx.x];
    const M1Net& N = nets[it.x];
    const int r = it.y;
    const int64_t m = N.m;
    const int log2m = N.log2m;
    const int log2M = log2m > 0 ? log2m - 1 : 0;
    const int M = 1 << log2M;
    const int K = m == 1 ? 1 : M + 1;
    const Cplx<T>* tw = tws[log2m];
    Cplx<T>* z = reinterpret_cast<Cplx<T>*>(smem_raw);
    Cplx<T>* P = z + M;
    const int64_t O = N.O;
    if (O == 0) return;
    for (int k = threadIdx.x; k < K; k += blockDim.x) P[k] = {T(1), T(0)};
    int E = 0;  // P holds 2^-E prod_k F x_k
    const T* xr = xs + N.x_off + (int64_t)r * N.X;
    for (int k = 0; k < N.p; ++k) {
        const M1Tensor& Tk = tens[N.t0 + k];
        const bool folded = Tk.soff < 0;
        const int64_t nsk = folded ? 1 : Tk.O;
        for (int64_t o = 0; o < nsk; ++o) {
            load_fft_scale(xr + Tk.xoff + o * m, m, log2m, z, tw, red, &s_e);
            const int e = s_e;
            const T sc = (T)ldexp(1.0, -e);
            if (folded) {
                for (int kk = threadIdx.x; kk < K; kk += blockDim.x) {
                    Cplx<T> X = m == 1 ? z[0] : unpack_bin(z, kk, log2M, tw);
                    X.x *= sc;
                    X.y *= sc;
                    P[kk] = cmul(P[kk], X);
                }
                E += e;
            } else {
                Cplx<T>* S = spec + N.spec_off + (int64_t)r * N.spec_per_rep + Tk.soff + o * K;
                for (int kk = threadIdx.x; kk < K; kk += blockDim.x) {
                    Cplx<T> X = m == 1 ? z[0] : unpack_bin(z, kk, log2M, tw);
                    X.x *= sc;
                    X.y *= sc;
                    S[kk] = X;
                }
                if (threadIdx.x == 0) sexp[N.exp_off + (int64_t)r * N.exp_per_rep + Tk.eoff + o] = e;
            }
            __syncthreads();
        }
    }
    // y_r(o) = (1/m) sum_j prod_k (F x_k[o_k])(j); the full spectrum is Hermitian,
    // so sum_j = P[0] + P[M] + 2 Re sum_{0<k<M} P[k] (m >= 2).
    double* yr = yrep + N.y_off + (int64_t)r * O;
    if (N.n_ot == 0) {
        double acc = 0;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            double wgt = (m == 1 || k == 0 || k == M) ? 1.0 : 2.0;
            acc += wgt * (double)P[k].x;
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) dred[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += dred[q];
            yr[0] = ldexp(t, E) / (double)m;
        }
        return;
    }
    // open outputs: one warp per output entry
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const Cplx<T>* Sb = spec + N.spec_off + (int64_t)r * N.spec_per_rep;
    const int* Eb = sexp + N.exp_off + (int64_t)r * N.exp_per_rep;
    for (int64_t o = warp; o < O; o += nw) {
        int64_t oo[TNSK_MAX_OPEN_TENSORS] = {0, 0, 0, 0};
        for (int j = 0; j < N.n_open; ++j) {
            const OpenMode om = opens[N.open0 + j];
            int64_t digit = (o / om.ostride) % om.dim;
#pragma unroll
            for (int s = 0; s < TNSK_MAX_OPEN_TENSORS; ++s)
                if (s == om.slot) oo[s] += digit * om.tstride;
        }
        const Cplx<T>* sp[TNSK_MAX_OPEN_TENSORS];
        int Eo = E;
#pragma unroll
        for (int s = 0; s < TNSK_MAX_OPEN_TENSORS; ++s) {
            if (s < N.n_ot) {
                const M1Tensor& Tt = tens[N.ot[s]];
                sp[s] = Sb + Tt.soff + oo[s] * K;
                Eo += Eb[Tt.eoff + oo[s]];
            } else {
                sp[s] = nullptr;
            }
        }
        double acc = 0;
        for (int k = lane; k < K; k += 32) {
            Cplx<T> v = P[k];
#pragma unroll
            for (int s = 0; s < TNSK_MAX_OPEN_TENSORS; ++s)
                if (s < N.n_ot) v = cmul(v, sp[s][k]);
            double wgt = (m == 1 || k == 0 || k == M) ? 1.0 : 2.0;
            acc += wgt * (double)v.x;
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
        if (lane == 0) yr[o] = ldexp(acc, Eo) / (double)m;
    }
}

// ---------------------------------------------------------------------------
// a9: median of group means (Theorem 1), FP64
// ---------------------------------------------------------------------------
__global__ void combine_kernel(const CombineItem* __restrict__ items, int n_items, const double* __restrict__ yrep) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_items; i += gridDim.x * blockDim.x) {
        const CombineItem c = items[i];
        const double* y = yrep + c.y_off;
        const int gs = c.R / c.groups;
        double med[64];
        for (int g = 0; g < c.groups; ++g) {
            double s = 0;
            for (int r = g * gs; r < (g + 1) * gs; ++r) s += y[(int64_t)r * c.O + c.o];
            double mean = s / gs;
            int q = g;  // insertion sort
            while (q > 0 && med[q - 1] > mean) {
                med[q] = med[q - 1];
                --q;
            }
            med[q] = mean;
        }
        const int g = c.groups;
        c.out[c.o] = (g & 1) ? med[g / 2] : 0.5 * (med[g / 2 - 1] + med[g / 2]);
        if (c.per_rep)
            for (int r = 0; r < c.R; ++r) c.per_rep[(int64_t)r * c.O + c.o] = y[(int64_t)r * c.O + c.o];
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename AccT>
cudaError_t launch_m1_scatter_t(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                                const uint32_t* d_tabs, AccT* d_xs, size_t smem, bool idx32, cudaStream_t s) {
    if (n_work <= 0) return cudaSuccess;
    if (idx32) {
        auto k = m1_scatter_kernel<AccT, uint32_t>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<n_work, 256, smem, s>>>(d_tens, d_nets, d_work, d_tabs, d_xs);
    } else {
        auto k = m1_scatter_kernel<AccT, uint64_t>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<n_work, 256, smem, s>>>(d_tens, d_nets, d_work, d_tabs, d_xs);
    }
    return cudaGetLastError();
}

cudaError_t launch_m1_scatter(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                              const uint32_t* d_tabs, void* d_xs, bool fp64, size_t smem, bool idx32,
                              cudaStream_t s) {
    if (fp64)
        return launch_m1_scatter_t<double>(d_tens, d_nets, d_work, n_work, d_tabs, (double*)d_xs, smem, idx32, s);
    return launch_m1_scatter_t<float>(d_tens, d_nets, d_work, n_work, d_tabs, (float*)d_xs, smem, idx32, s);
}

cudaError_t launch_m1_spectrum(const M1Tensor* d_tens, const M1Net* d_nets, const OpenMode* d_opens,
                               const int2* d_items, int n_items, const void* d_xs, const void* const* d_tws,
                               void* d_spec, int* d_sexp, double* d_yrep, bool fp64, int max_log2m,
                               cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const int M = max_log2m > 0 ? 1 << (max_log2m - 1) : 1;
    if (fp64) {
        size_t smem = (size_t)(2 * M + 1) * sizeof(Cplx<double>);
        auto k = m1_spectrum_kernel<double>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<n_items, 256, smem, s>>>(d_tens, d_nets, d_opens, d_items, (const double*)d_xs,
                                     (const Cplx<double>* const*)d_tws, (Cplx<double>*)d_spec, d_sexp, d_yrep);
    } else {
        size_t smem = (size_t)(2 * M + 1) * sizeof(Cplx<float>);
        auto k = m1_spectrum_kernel<float>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<n_items, 256, smem, s>>>(d_tens, d_nets, d_opens, d_items, (const float*)d_xs,
                                     (const Cplx<float>* const*)d_tws, (Cplx<float>*)d_spec, d_sexp, d_yrep);
    }
    return cudaGetLastError();
}

cudaError_t launch_combine(const CombineItem* d_items, int n_items, const double* d_yrep, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    int blocks = (n_items + 127) / 128;
    if (blocks > 152 * 16) blocks = 152 * 16;
    combine_kernel<<<blocks, 128, 0, s>>>(d_items, n_items, d_yrep);
    return cudaGetLastError();
}

}  // namespace tnsk
