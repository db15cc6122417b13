// method2.cu -- method 2 of the paper (Sec. 4.4): recursive sketches on the
// rooted tree, evaluated leaves to root (Alg. 2), with the sign and row of a
// recursive-sketch column from Alg. 4 and the fused sketch / matrix-vector
// product of Alg. 5 batched over repetitions.
//
//   a5  m2_leaf_kernel     x_l = C_{k,l} vec(X_l) for the leaves
//   a6  m2_compose_kernel  r_k = Q_k((x) x_l): per level l = qt..2 and pair j,
//                          T_{l,j}(u (x) v) = F^{-1}(F C_a u o F C_b v) (Def.
//                          "Tensor sketch" of order 2) by shared-memory FFTs
//   a7  m2_vbuild_kernel   V(col, r) = sigma_r(col) r_k[r][b_r(col)] (Alg. 4)
//       m2_gemm_kernel     x_k[r] += C_{par,k} (mat(X_k) V)[:, r]  (Alg. 5 for all
//                          reps at once: each entry of X_k is read once per
//                          batch of 64 reps); FP64 path. The FP32 path uses the
//                          tensor-core kernel of m2_gemm_tc.cu.
//   a8  m2_root_kernel     y_r = sum_i X_o(i) sigma_r(i) r_o[r][b_r(i)] = x_o^T r_o
#include "fft.cuh"
#include "kernels.cuh"
#include "method2.cuh"
#include "plan.cuh"

namespace tnsk {

// Sign and row of the recursive sketch R_k for one column (Alg. 4). b[j] holds
// the bin of slot j (child count sketch C_{k,l} at the child-mode index, or the
// padding slot's word at index 0); levels l = qt..2 combine pairs by
// TensorSketchHash (Alg. 3) with T_{l,j}. QTMAX bounds qt at compile time.
template <int QTMAX>
__device__ __forceinline__ void rsh_reduce(uint32_t (&b)[QTMAX], uint32_t& neg, int qt,
                                           const uint32_t* __restrict__ ttab, int64_t m, uint32_t mask) {
#pragma unroll
    for (int lv = QTMAX; lv >= 2; lv >>= 1) {
        if (lv <= qt) {
            const int64_t before = qt - lv;  // pairs stored before level lv
#pragma unroll
            for (int j = 0; j < lv / 2; ++j) {
                const uint32_t* ta = ttab + ((before + j) * 2 + 0) * m;
                const uint32_t* tb = ttab + ((before + j) * 2 + 1) * m;
                uint32_t wa = ta[b[2 * j]];
                uint32_t wb = tb[b[2 * j + 1]];
                neg ^= wa ^ wb;
                b[j] = (wa + wb) & mask;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// a5: leaves
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) m2_leaf_kernel(const M2Node* __restrict__ nodes, const M2Net* __restrict__ nets,
                                                      const M2Item* __restrict__ items,
                                                      const uint32_t* __restrict__ tabs, T* __restrict__ ws) {
    const M2Item it = items[blockIdx.x];  // entries [begin, end), reps [a, a + b)
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const uint32_t mask = (uint32_t)(N.m - 1);
    for (int64_t i = it.begin + threadIdx.x; i < it.end; i += blockDim.x) {
        const T v = load_as<T>(nd.data, nd.dtype, i);
        for (int r = it.a; r < it.a + it.b; ++r) {
            const uint32_t w = tabs[N.tab_off + (int64_t)r * N.Lrep + nd.ptab + i];
            atomicAdd(&ws[nd.x_off + (int64_t)r * N.m + (w & mask)], (w & TNSK_SIGN_BIT) ? -v : v);
        }
    }
}

// ---------------------------------------------------------------------------
// a6: Q_k composition
// ---------------------------------------------------------------------------
// One CTA per (node, rep). Shared memory: cu [M], cv [M], Y [M+1] complex.
template <typename T>
__global__ void __launch_bounds__(256) m2_compose_kernel(const M2Node* __restrict__ nodes,
                                                         const M2Net* __restrict__ nets,
                                                         const M2Item* __restrict__ items,
                                                         const uint32_t* __restrict__ tabs, T* __restrict__ ws,
                                                         const Cplx<T>* const* __restrict__ tws) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const M2Item it = items[blockIdx.x];
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const int r = it.a;
    const int64_t m = N.m;
    const uint32_t mask = (uint32_t)(m - 1);
    const int log2m = N.log2m;
    const int log2M = log2m > 0 ? log2m - 1 : 0;
    const int M = 1 << log2M;
    const Cplx<T>* tw = tws[log2m];
    const uint32_t* tabr = tabs + N.tab_off + (int64_t)r * N.Lrep;
    const int qt = nd.qt;
    Cplx<T>* cu = reinterpret_cast<Cplx<T>*>(smem_raw);
    Cplx<T>* cv = cu + M;
    Cplx<T>* Y = cv + M;
    T* ru = reinterpret_cast<T*>(cu);  // real views (length 2M = m, or 1 when m = 1)
    T* rv = reinterpret_cast<T*>(cv);
    T* rbuf = ws + nd.r_off + (int64_t)r * (qt - 1) * m;
    for (int lv = qt; lv >= 2; lv >>= 1) {
        for (int j = 0; j < lv / 2; ++j) {
            const uint32_t* ta = tabr + nd.t_tab + ((int64_t)(qt - lv + j) * 2 + 0) * m;
            const uint32_t* tb = tabr + nd.t_tab + ((int64_t)(qt - lv + j) * 2 + 1) * m;
            for (int64_t i = threadIdx.x; i < 2 * (int64_t)M; i += blockDim.x) {
                ru[i] = T(0);
                rv[i] = T(0);
            }
            __syncthreads();
            // count-sketch both inputs by the sides of T_{lv,j}
            for (int side = 0; side < 2; ++side) {
                const int s = 2 * j + side;
                const uint32_t* th = side ? tb : ta;
                T* dst = side ? rv : ru;
                if (lv == qt && s >= nd.c) {
                    // padding slot: C_pad e_1 is a signed one-hot vector
                    if (threadIdx.x == 0) {
                        uint32_t pw = tabr[nd.pad_tab + s];
                        uint32_t w = th[pw & mask];
                        T val = ((pw ^ w) & TNSK_SIGN_BIT) ? T(-1) : T(1);
                        atomicAdd(&dst[w & mask], val);
                    }
                } else {
                    const T* src = lv == qt ? ws + nd.child_x[s] + (int64_t)r * m
                                            : rbuf + (int64_t)(qt - 2 * lv + s) * m;
                    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
                        T v = src[i];
                        if (v != T(0)) {
                            uint32_t w = th[i];
                            atomicAdd(&dst[w & mask], (w & TNSK_SIGN_BIT) ? -v : v);
                        }
                    }
                }
            }
            __syncthreads();
            T* out = rbuf + (int64_t)(qt - lv + j) * m;
            if (m == 1) {
                if (threadIdx.x == 0) out[0] = ru[0] * rv[0];
                __syncthreads();
                continue;
            }
            block_fft_dif(cu, 2, log2M, tw);  // cu and cv are adjacent
            for (int k = threadIdx.x; k <= M; k += blockDim.x)
                Y[k] = cmul(unpack_bin(cu, k, log2M, tw), unpack_bin(cv, k, log2M, tw));
            __syncthreads();
            // inverse real transform: Z[k] = E[k] + i O[k] with E = (Y[k] + conj Y[M-k]) / 2,
            // O = (Y[k] - conj Y[M-k]) conj(W^k) / 2; z = F_M^{-1} Z = conj(F_M conj Z) / M
            for (int k = threadIdx.x; k < M; k += blockDim.x) {
                Cplx<T> a = Y[k], c = cconj(Y[M - k]);
                Cplx<T> e = {(a.x + c.x) * T(0.5), (a.y + c.y) * T(0.5)};
                Cplx<T> o = cmul(csub(a, c), cconj(tw[k]));
                o.x *= T(0.5);
                o.y *= T(0.5);
                Cplx<T> z = {e.x - o.y, e.y + o.x};  // E + i O
                cu[k] = cconj(z);
            }
            __syncthreads();
            block_fft_dif(cu, 1, log2M, tw);
            const T invM = T(1) / T(M);
            for (int n = threadIdx.x; n < M; n += blockDim.x) {
                Cplx<T> z = cconj(cu[bitrev(n, log2M)]);
                out[2 * n] = z.x * invM;
                out[2 * n + 1] = z.y * invM;
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// a7: V = sigma_r(col) r_k[r][b_r(col)], and the batched sketched matvec
// ---------------------------------------------------------------------------
// Items: columns [begin, end) x reps [a, a + b). Plain form (pad_ == 0): every table
// word and child-sketch entry read from global memory (L2). Staged form (pad_ == 1):
// the reps' T tables and child sketches copied to shared memory first, so the
// data-dependent lookups are shared-memory reads; the plan takes this form where they
// fit (the launch's dynamic shared memory).
template <typename T, typename IdxT, int QTMAX, int MAXD>
__global__ void __launch_bounds__(256) m2_vbuild_kernel(const M2Node* __restrict__ nodes,
                                                        const M2Net* __restrict__ nets,
                                                        const M2Item* __restrict__ items,
                                                        const uint32_t* __restrict__ tabs, T* __restrict__ ws) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const M2Item it = items[blockIdx.x];
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const int R = N.R;
    const int64_t m = N.m;
    const uint32_t mask = (uint32_t)(m - 1);
    const int order = nd.order, pmode = nd.pmode, c = nd.c, qt = nd.qt;
    // the node's offsets in registers (one read of the descriptor per block)
    const int64_t tab_off = N.tab_off, Lrep = N.Lrep, pad_tab = nd.pad_tab, t_tab = nd.t_tab;
    const int64_t src_off = nd.src_off, src_stride = nd.src_stride, v_off = nd.v_off, cols = nd.cols;
    const bool split = sizeof(T) == 4 && !nd.is_root;
    // block-uniform per-mode data: dim and child-table offset of each mode
    IdxT dim[MAXD];
    int64_t ctab[MAXD];
#pragma unroll
    for (int d = 0; d < MAXD; ++d) {
        const bool child = d < order && d != pmode;
        dim[d] = child ? (IdxT)nd.dims[d] : (IdxT)1;
        const int slot = (pmode >= 0 && d > pmode) ? d - 1 : d;
        ctab[d] = child ? nd.ctab[slot < TNSK_MAX_ORDER ? slot : 0] : 0;
    }
    // sign word and bin of V(col, r): the child count-sketch words of col's indices, the
    // padding words, then the T-table levels (ttab: rep r's T tables)
    // one child mode (the common case of a chain or a binary tree's matrices): its index
    // is the column itself, no mixed-radix decode
    int n_child_modes = 0, child_mode = 0;
#pragma unroll
    for (int d = 0; d < MAXD; ++d)
        if (d < order && d != pmode) ++n_child_modes, child_mode = d;
    const bool one_child = n_child_modes == 1;
    const int one_slot = (pmode >= 0 && child_mode > pmode) ? child_mode - 1 : child_mode;
    const int64_t one_ctab = nd.ctab[one_slot < TNSK_MAX_ORDER ? one_slot : 0];
    auto lookup = [&](const uint32_t* __restrict__ tabr, const uint32_t* ttab, int64_t col, uint32_t& neg) {
        uint32_t b[QTMAX];
        neg = 0;
        if (one_child) {
            const uint32_t w = tabr[one_ctab + col];
            neg = w;
#pragma unroll
            for (int j = 0; j < QTMAX; ++j)
                if (j == one_slot) b[j] = w & mask;
#pragma unroll
            for (int j = 0; j < QTMAX; ++j)
                if (j >= c && j < qt) {
                    uint32_t wp = tabr[pad_tab + j];
                    neg ^= wp;
                    b[j] = wp & mask;
                }
            rsh_reduce<QTMAX>(b, neg, qt, ttab, m, mask);
            return b[0];
        }
        IdxT rem = (IdxT)col;
        // children are the non-parent modes in mode order: slot = d, or d - 1 after the parent
#pragma unroll
        for (int d = MAXD - 1; d >= 0; --d) {
            if (d < order && d != pmode) {
                const IdxT qd = rem / dim[d];
                const IdxT i = rem - qd * dim[d];
                rem = qd;
                const uint32_t w = tabr[ctab[d] + (int64_t)i];
                neg ^= w;
                if (pmode >= 0 && d > pmode) {
                    if (d - 1 < QTMAX) b[d > 0 ? d - 1 : 0] = w & mask;
                } else {
                    if (d < QTMAX) b[d] = w & mask;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < QTMAX; ++j)
            if (j >= c && j < qt) {
                uint32_t w = tabr[pad_tab + j];
                neg ^= w;
                b[j] = w & mask;
            }
        rsh_reduce<QTMAX>(b, neg, qt, ttab, m, mask);
        return b[0];
    };
    const bool vbf16 = sizeof(T) == 4 && nd.vbf16;
    auto store = [&](int r, int64_t col, T v) {
        const int64_t dst = v_off + (int64_t)r * cols + col;
        if (vbf16) {
            // operand of the BF16 product: three BF16 parts, each the rounding of what the
            // previous ones leave (the differences are exact in FP32)
            __nv_bfloat16* vb = reinterpret_cast<__nv_bfloat16*>(ws + v_off) + (int64_t)r * cols + col;
            const float x = (float)v;
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            const float x1 = x - __bfloat162float(h);
            const __nv_bfloat16 mm = __float2bfloat16_rn(x1);
            const __nv_bfloat16 l = __float2bfloat16_rn(x1 - __bfloat162float(mm));
            const int64_t part = (int64_t)R * cols;
            vb[0] = h;
            vb[part] = mm;
            vb[2 * part] = l;
        } else if (split) {
            // operand of the tensor-core product: TF32 hi part, then its lo part R*cols later
            uint32_t hi, lo;
            tf32_split((float)v, hi, lo);
            ws[dst] = (T)__uint_as_float(hi);
            ws[dst + (int64_t)R * cols] = (T)__uint_as_float(lo);
        } else {
            ws[dst] = v;
        }
    };
    // Each (rep, column) is a chain of dependent loads (child table word, T-table words,
    // the child sketch entry): a thread takes kU of them at once, all loads before any
    // store, so kU chains are in flight per thread.
    constexpr int kU = 4;
    if (it.pad_ == 1 && one_child && qt <= 1 && it.b <= 2 && it.end - it.begin <= 4 * (int64_t)blockDim.x &&
        (int64_t)it.b * m <= 8 * (int64_t)blockDim.x) {
        // One child mode, no padding words or T tables (chains): every global load of the
        // item, the column words of all its reps and their child sketches, is issued at
        // once, then one barrier, the gathers from shared memory and the stores
        const int G = it.b, r0 = it.a;
        const int bd = (int)blockDim.x;
        T* s_src = reinterpret_cast<T*>(smem_raw);
        uint32_t wv[2][4];
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const uint32_t* tabr = tabs + tab_off + (int64_t)(r0 + (g < G ? g : 0)) * Lrep + one_ctab;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t col = it.begin + threadIdx.x + (int64_t)u * bd;
                wv[g][u] = (g < G && col < it.end) ? __ldg(tabr + col) : 0u;
            }
        }
        const int64_t nsrc = (int64_t)G * m;
        T cv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t q = threadIdx.x + (int64_t)i * bd;
            const int64_t g = q >> N.log2m;
            cv[i] = q < nsrc ? ws[src_off + (r0 + g) * src_stride + (q - (g << N.log2m))] : (T)0;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t q = threadIdx.x + (int64_t)i * bd;
            if (q < nsrc) s_src[q] = cv[i];
        }
        __syncthreads();
#pragma unroll
        for (int g = 0; g < 2; ++g)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t col = it.begin + threadIdx.x + (int64_t)u * bd;
                if (g < G && col < it.end) {
                    const T z = s_src[g * m + (wv[g][u] & mask)];
                    store(r0 + g, col, (wv[g][u] & TNSK_SIGN_BIT) ? -z : z);
                }
            }
        return;
    }
    if (it.pad_ == 1) {
        const int G = it.b, r0 = it.a;
        const int64_t tw = qt >= 2 ? 2 * (int64_t)(qt - 1) * m : 0;  // T-table words of one rep
        uint32_t* s_t = reinterpret_cast<uint32_t*>(smem_raw);
        T* s_src = reinterpret_cast<T*>(smem_raw + (((size_t)G * tw * 4 + 15) & ~(size_t)15));
        // the copies, kU loads in flight per thread
        for (int64_t q0 = threadIdx.x; q0 < (int64_t)G * tw; q0 += kU * blockDim.x) {
            uint32_t v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int64_t q = q0 + (int64_t)u * blockDim.x;
                const int64_t g = q / tw;
                v[u] = q < (int64_t)G * tw ? tabs[tab_off + (r0 + g) * Lrep + t_tab + (q - g * tw)] : 0u;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (q0 + (int64_t)u * blockDim.x < (int64_t)G * tw) s_t[q0 + (int64_t)u * blockDim.x] = v[u];
        }
        for (int64_t q0 = threadIdx.x; q0 < (int64_t)G * m; q0 += kU * blockDim.x) {
            T v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int64_t q = q0 + (int64_t)u * blockDim.x;
                const int64_t g = q >> N.log2m;
                v[u] = q < (int64_t)G * m ? ws[src_off + (r0 + g) * src_stride + (q - g * m)] : (T)0;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (q0 + (int64_t)u * blockDim.x < (int64_t)G * m) s_src[q0 + (int64_t)u * blockDim.x] = v[u];
        }
        __syncthreads();
        for (int g = 0; g < G; ++g) {
            const int r = r0 + g;
            const uint32_t* tabr = tabs + tab_off + (int64_t)r * Lrep;
            for (int64_t c0 = it.begin + threadIdx.x; c0 < it.end; c0 += kU * blockDim.x) {
                T val[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int64_t col = c0 + (int64_t)u * blockDim.x;
                    val[u] = (T)0;
                    if (col >= it.end) continue;
                    uint32_t neg;
                    const uint32_t b0 = lookup(tabr, s_t + g * tw, col, neg);
                    const T z = s_src[g * m + b0];
                    val[u] = (neg & TNSK_SIGN_BIT) ? -z : z;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int64_t col = c0 + (int64_t)u * blockDim.x;
                    if (col < it.end) store(r, col, val[u]);
                }
            }
        }
        return;
    }
    const uint32_t len = (uint32_t)(it.end - it.begin);  // <= 128
    const uint32_t cnt = len * (uint32_t)it.b;
    for (uint32_t q0 = threadIdx.x; q0 < cnt; q0 += kU * blockDim.x) {
        T val[kU];
        int rr[kU];
        int64_t cc[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t q = q0 + (uint32_t)u * blockDim.x;
            rr[u] = -1;
            val[u] = (T)0;
            cc[u] = 0;
            if (q >= cnt) continue;
            const int rl = (int)(len == 128 ? q >> 7 : q / len);
            const int r = it.a + rl;
            const int64_t col = it.begin + (q - (uint32_t)rl * len);
            const uint32_t* tabr = tabs + tab_off + (int64_t)r * Lrep;
            uint32_t neg;
            const uint32_t b0 = lookup(tabr, tabr + t_tab, col, neg);
            const T z = ws[src_off + (int64_t)r * src_stride + b0];
            val[u] = (neg & TNSK_SIGN_BIT) ? -z : z;
            rr[u] = r;
            cc[u] = col;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (rr[u] >= 0) store(rr[u], cc[u], val[u]);
    }
}

template <typename T, typename IdxT, int QTMAX>
static void launch_vbuild_q(int n, const M2Node* nodes, const M2Net* nets, const M2Item* its, const uint32_t* tabs,
                            T* ws, int max_order, size_t smem, cudaStream_t s) {
    if (max_order <= 4)
        m2_vbuild_kernel<T, IdxT, QTMAX, 4><<<n, 256, smem, s>>>(nodes, nets, its, tabs, ws);
    else
        m2_vbuild_kernel<T, IdxT, QTMAX, TNSK_MAX_ORDER><<<n, 256, smem, s>>>(nodes, nets, its, tabs, ws);
}

template <typename T, typename IdxT>
static void launch_vbuild(int n, const M2Node* nodes, const M2Net* nets, const M2Item* its, const uint32_t* tabs,
                          T* ws, int max_qt, int max_order, size_t smem, cudaStream_t s) {
    if (max_qt <= 1)
        launch_vbuild_q<T, IdxT, 1>(n, nodes, nets, its, tabs, ws, max_order, smem, s);
    else if (max_qt <= 4)
        launch_vbuild_q<T, IdxT, 4>(n, nodes, nets, its, tabs, ws, max_order, smem, s);
    else
        launch_vbuild_q<T, IdxT, TNSK_MAX_SLOTS>(n, nodes, nets, its, tabs, ws, max_order, smem, s);
}

// W = mat(X_k)[rows, :] V[:, reps] for a 64 x 64 tile, then x_k[r][h(i)] += s(i) W[i][r]
// with (h, s) the count sketch C_{par,k} of the parent edge (Alg. 5 scatter).
template <typename T>
__global__ void __launch_bounds__(256) m2_gemm_kernel(const M2Node* __restrict__ nodes, const M2Net* __restrict__ nets,
                                                      const M2Item* __restrict__ items,
                                                      const uint32_t* __restrict__ tabs, T* __restrict__ ws) {
    __shared__ __align__(16) T Xs[32][64 + 4];
    __shared__ __align__(16) T Vs[32][64 + 1];
    const M2Item it = items[blockIdx.x];
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const int R = N.R;
    const int64_t m = N.m;
    const uint32_t mask = (uint32_t)(m - 1);
    const int64_t row0 = (int64_t)it.a * 64;
    const int rep0 = it.b * 64;
    const int64_t npar = nd.npar, cols = nd.cols, Bc = nd.Bc;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    const T* V = ws + nd.v_off;
    for (int64_t k0 = 0; k0 < cols; k0 += 32) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = threadIdx.x + 256 * q;
            const int row = e >> 5, kk = e & 31;
            const int64_t gr = row0 + row, gc = k0 + kk;
            T v = T(0);
            if (gr < npar && gc < cols) {
                int64_t flat;
                if (nd.A == 1) {
                    flat = gr * Bc + gc;
                } else {
                    const uint32_t a = (uint32_t)gc / (uint32_t)Bc;  // cols < 2^32 (checked by the planner)
                    flat = ((int64_t)a * npar + gr) * Bc + (gc - (int64_t)a * Bc);
                }
                v = load_as<T>(nd.data, nd.dtype, flat);
            }
            Xs[kk][row] = v;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = threadIdx.x + 256 * q;
            const int kk = e & 31, rr = e >> 5;
            const int64_t gc = k0 + kk;
            Vs[kk][rr] = (gc < cols && rep0 + rr < R) ? V[(int64_t)(rep0 + rr) * cols + gc] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            T a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Xs[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Vs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t row = row0 + ty * 4 + i;
        if (row >= npar) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int rep = rep0 + tx * 4 + j;
            if (rep >= R) continue;
            const uint32_t w = tabs[N.tab_off + (int64_t)rep * N.Lrep + nd.ptab + row];
            const T val = acc[i][j];
            atomicAdd(&ws[nd.x_off + (int64_t)rep * m + (w & mask)], (w & TNSK_SIGN_BIT) ? -val : val);
        }
    }
}

// ---------------------------------------------------------------------------
// a7 (tensor-core path): x_k[r][h_r(i)] += s_r(i) W^T[r][i], the count sketch of the
// parent edge applied to the rows of W = mat(X_k) V. One CTA per (node, block of
// reps), shared-memory bins, plain stores (x_k has no other producer).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) m2_wscatter_kernel(const M2Node* __restrict__ nodes,
                                                          const M2Net* __restrict__ nets,
                                                          const M2Item* __restrict__ items,
                                                          const uint32_t* __restrict__ tabs, float* __restrict__ ws) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* bins = reinterpret_cast<float*>(smem_raw);
    const M2Item it = items[blockIdx.x];
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const int64_t m = N.m;
    const uint32_t mask = (uint32_t)(m - 1);
    const int r0 = it.a, nr = it.b;
    const int64_t npar = nd.npar;
    const uint32_t* __restrict__ tw0 = tabs + N.tab_off + nd.ptab;  // + r * Lrep + i
    const float* __restrict__ w0 = ws + nd.w_off;                   // + r * npar + i
    float* __restrict__ x0 = ws + nd.x_off + (int64_t)r0 * m;
    const int64_t Lrep = N.Lrep;
    for (int64_t q = threadIdx.x; q < (int64_t)nr * m; q += blockDim.x) bins[q] = 0.f;
    __syncthreads();
    // (rep, row) pairs flat, kU per thread at once: all table words and W values are
    // loaded before the shared-memory adds, so the loads of kU pairs overlap
    // per rep, rows strided over the threads, kU rows per thread at once: all table
    // words and W values are loaded before the shared-memory adds, so the loads overlap
    constexpr int kU = 4;
    for (int j = 0; j < nr; ++j) {
        const uint32_t* __restrict__ twr = tw0 + (int64_t)(r0 + j) * Lrep;
        const float* __restrict__ wr = w0 + (int64_t)(r0 + j) * npar;
        float* bj = bins + (int64_t)j * m;
        for (int64_t i0 = threadIdx.x; i0 < npar; i0 += kU * blockDim.x) {
            uint32_t t[kU];
            float v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int64_t i = i0 + (int64_t)u * blockDim.x;
                t[u] = i < npar ? twr[i] : 0u;
                v[u] = i < npar ? wr[i] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (i0 + (int64_t)u * blockDim.x < npar)
                    atomicAdd(&bj[t[u] & mask], (t[u] & TNSK_SIGN_BIT) ? -v[u] : v[u]);
        }
    }
    __syncthreads();
    for (int64_t q = threadIdx.x; q < (int64_t)nr * m; q += blockDim.x) x0[q] = bins[q];
}

// ---------------------------------------------------------------------------
// a8: root, y_r = sum_col X_o[col] V[r][col]
// ---------------------------------------------------------------------------
// One warp per rep at a time, lanes over the chunk's columns (coalesced X and V).
template <typename T>
__global__ void __launch_bounds__(256) m2_root_kernel(const M2Node* __restrict__ nodes, const M2Net* __restrict__ nets,
                                                      const M2Item* __restrict__ items, const T* __restrict__ ws,
                                                      double* __restrict__ yrep) {
    const M2Item it = items[blockIdx.x];  // columns [begin, end), reps [a, a + b)
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const T* V = nd.v_off >= 0 ? ws + nd.v_off : nullptr;
    for (int r = it.a + warp; r < it.a + it.b; r += nw) {
        double acc = 0;
        for (int64_t col = it.begin + lane; col < it.end; col += 32) {
            const T x = load_as<T>(nd.data, nd.dtype, col);
            acc += (double)(V ? x * V[(int64_t)r * nd.cols + col] : x);
        }
#pragma unroll
        for (int sft = 16; sft > 0; sft >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, sft);
        if (lane == 0) atomicAdd(&yrep[N.y_off + r], acc);
    }
}

// ---------------------------------------------------------------------------
// host driver: heights 0..H, kinds in order leaf, compose, vbuild, gemm, root
// ---------------------------------------------------------------------------
template <typename T>
static cudaError_t run_m2_t(const BatchPlan& P, unsigned char* base, const void* const* d_tws, cudaStream_t s,
                            Profiler& prof, int* d_err, int inject) {
    static const int kKind[M2_NKINDS] = {TNSK_K_M2_LEAF, TNSK_K_M2_COMPOSE, TNSK_K_M2_VBUILD, TNSK_K_M2_GEMM,
                                         TNSK_K_M2_GEMM, TNSK_K_M2_GEMM,    TNSK_K_M2_GEMM,   TNSK_K_M2_GEMM,
                                         TNSK_K_M2_GEMM, TNSK_K_M2_SCATTER, TNSK_K_M2_ROOT,   TNSK_K_M2_PREP};
    const M2Node* nodes = (const M2Node*)(base + P.m2.nodes_off);
    const M2Net* nets = (const M2Net*)(base + P.m2.nets_off);
    const M2Item* items = (const M2Item*)(base + P.m2.items_off);
    const uint32_t* tabs = (const uint32_t*)(base + P.tabs_off);
    T* ws = (T*)(base + P.m2.ws_off);
    double* yrep = (double*)(base + P.yrep_off);
    const int M = P.m2.max_log2m > 0 ? 1 << (P.m2.max_log2m - 1) : 1;
    const size_t csmem = (size_t)(3 * M + 1) * sizeof(Cplx<T>);
    cudaFuncSetAttribute(m2_compose_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem);
    for (int h = 0; h <= P.m2.max_height; ++h) {
        for (int kind = 0; kind < M2_NKINDS; ++kind) {
            const int n = P.m2.count[h * M2_NKINDS + kind];
            if (n == 0) continue;
            const M2Item* its = items + P.m2.first[h * M2_NKINDS + kind];
            prof.begin(kKind[kind], s);
            switch (kind) {
                case M2_LEAF: m2_leaf_kernel<T><<<n, 256, 0, s>>>(nodes, nets, its, tabs, ws); break;
                case M2_COMPOSE:
                    m2_compose_kernel<T><<<n, 256, csmem, s>>>(nodes, nets, its, tabs, ws,
                                                                (const Cplx<T>* const*)d_tws);
                    break;
                case M2_VBUILD:
                    if (P.m2.idx32)
                        launch_vbuild<T, uint32_t>(n, nodes, nets, its, tabs, ws, P.m2.max_qt, P.m2.max_order, P.m2.vbuild_smem,
                                                   s);
                    else
                        launch_vbuild<T, uint64_t>(n, nodes, nets, its, tabs, ws, P.m2.max_qt, P.m2.max_order, P.m2.vbuild_smem,
                                                   s);
                    break;
                case M2_GEMM:
                case M2_GEMM_STREAM:
                    if (sizeof(T) == 4)  // FP32: tensor cores (3-pass TF32 split)
                        launch_m2_gemm_tc(n, nodes, nets, its, tabs, (float*)ws, base + P.m2.tmaps_off, d_err,
                                          kind == M2_GEMM_STREAM, inject, s);
                    else
                        m2_gemm_kernel<T><<<n, 256, 0, s>>>(nodes, nets, its, tabs, ws);
                    break;
                case M2_GEMM_RUNG:  // FP32 plans only (the plan rejects grouped tensors in FP64)
                    if (sizeof(T) == 4)
                        launch_m2_gemm_tc_rung(n, nodes, nets, its, (float*)ws, base + P.m2.tmaps_off, d_err,
                                               P.m2.rung_smem, s);
                    break;
                case M2_GEMM_BF16:  // BF16 nodes of FP32-accumulating plans
                    if (sizeof(T) == 4)
                        launch_m2_gemm_bf16(n, nodes, nets, its, (float*)ws, base + P.m2.tmaps_off, d_err, inject,
                                            s);
                    break;
                case M2_GEMM_RUNGF:  // FP32 plans only
                    if (sizeof(T) == 4) {
                        const cudaError_t e = launch_m2_rung_fact(n, nodes, nets, its, (float*)ws, P.m2.rungf_smem, s);
                        if (e != cudaSuccess) return e;
                    }
                    break;
                case M2_GEMM_RUNGT:  // FP32 plans only
                    if (sizeof(T) == 4) {
                        const cudaError_t e = launch_m2_rung_tc(n, nodes, its, (float*)ws,
                                                                base + P.m2.tmaps_off, d_err, inject, s);
                        if (e != cudaSuccess) return e;
                    }
                    break;
                case M2_RUNG_PREP:  // FP32 plans only
                    if (sizeof(T) == 4) {
                        const cudaError_t e = launch_m2_rung_prep(n, nodes, its, (float*)ws, s);
                        if (e != cudaSuccess) return e;
                    }
                    break;
                case M2_WSCATTER: {
                    const size_t smem = P.m2.scatter_smem;
                    cudaFuncSetAttribute(m2_wscatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    m2_wscatter_kernel<<<n, 256, smem, s>>>(nodes, nets, its, tabs, (float*)ws);
                    break;
                }
                case M2_ROOT: m2_root_kernel<T><<<n, 256, 0, s>>>(nodes, nets, its, ws, yrep); break;
            }
            prof.end(s);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

tnsk_status run_method2(const BatchPlan& plan, unsigned char* base, bool fp64, const void* const* d_tws,
                        cudaStream_t s, Profiler& prof, int* d_err, std::string& err, int inject) {
    cudaError_t e = fp64 ? run_m2_t<double>(plan, base, d_tws, s, prof, d_err, inject)
                         : run_m2_t<float>(plan, base, d_tws, s, prof, d_err, inject);
    if (e != cudaSuccess) {
        err = std::string("method 2 launch: ") + cudaGetErrorString(e);
        return TNSK_ERR_CUDA;
    }
    return TNSK_OK;
}

}  // namespace tnsk
