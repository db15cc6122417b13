/*
 * tnsk_oracle.h -- FP64 CPU oracle for the two sketching estimators of
 * "Approximating Tensor Network Contraction with Sketches" (arXiv 2603.07387).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the slow, plain reference that the
 * GPU path is checked against. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table or
 * constant generator with the CUDA library: the hash contract below is
 * implemented here a second time, from its written definition.
 *
 * All arithmetic is IEEE binary64. Indices are 0-based (the paper is 1-based).
 * Tensors are row-major (the paper's vec(): last mode fastest, Sec. 2).
 *
 * Hash contract (the paper leaves the construction of its k-wise independent
 * families open, Sec. 2.1 Def. "k-wise independence" / "Count sketch"):
 *   sm(x)   = SplitMix64 output for state x (Steele, Lea, Flood 2014):
 *             z = x + 0x9E3779B97F4A7C15; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
 *             z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31.
 *   K       = sm(sm(sm(seed) ^ rep) ^ tid)
 *   c(rho,j)= red61(sm(K ^ (8*rho + j)))     rho=0 bin, rho=1 sign, j=0..3
 *   P       = 2^61 - 1, red61 folds a 64-bit word into [0, P).
 *   h(i)    = ((c(0,1)*i + c(0,0)) mod P) mod m          (2-wise, m = 2^k)
 *   g(i)    = c(1,3) i^3 + c(1,2) i^2 + c(1,1) i + c(1,0)  mod P  (4-wise)
 *   s(i)    = +1 if g(i) even, -1 if odd.
 *   complement (Def. "Complement count sketch"): h'(i) = (m - h(i)) mod m, same s.
 * Table ids (tid):
 *   method 1, edge e (index into E):                 (1<<56) | e
 *   method 2, edge e (count sketch C_{k,l}):         (2<<56) | e
 *   method 2, padding slot j of tensor k:            (3<<56) | (k<<24) | j
 *   method 2, tensor sketch T_{l,j} of tensor k,
 *             l = 2^lam, side s in {0,1}:            (4<<56) | (k<<24) | (lam<<16) | (j<<1) | s
 */
#ifndef TNSK_ORACLE_H
#define TNSK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t p;                  /* number of tensors X_1..X_p */
    const int32_t* order;       /* [p] order q_k of each tensor (0 = scalar) */
    const int64_t* dims;        /* [sum q_k] dims, tensor k's modes consecutive */
    const double* const* data;  /* [p] row-major FP64 entries */
    int32_t t;                  /* number of contractions |E| */
    const int32_t* edges;       /* [2t] global 0-based mode ids, pair (u,v) */
    int32_t n_open;             /* |K'| */
    const int32_t* open;        /* [n_open] permutation of K' = output mode order */
} orc_net;

/* status codes */
#define ORC_OK 0
#define ORC_INVALID (-1)
#define ORC_CYCLIC (-2)
#define ORC_UNSUPPORTED (-3)

uint64_t orc_splitmix64(uint64_t state);
uint64_t orc_tid(int32_t kind, int64_t a, int64_t b, int64_t c, int64_t d);
void orc_count_sketch(uint64_t seed, uint64_t rep, uint64_t tid, int64_t n, int64_t m,
                      int64_t* bins, int8_t* signs);

/* DFT (F_{jk} = exp(-2 pi i jk/m), unnormalised) by definition, O(m^2). */
void orc_dft(int64_t m, const double* re, const double* im, double* ore, double* oim);
/* Same transform by recursive radix-2 Cooley-Tukey (m a power of two). */
void orc_fft(int64_t m, const double* re, const double* im, double* ore, double* oim);

/* Method 1 tables: for rep r and edge e, bins[r*L + eoff_e + i], signs likewise,
 * L = sum_e n_e, eoff_e = sum_{e'<e} n_e'. The edge's first mode u uses (h, s),
 * its second mode v the complement. */
int orc_m1_tables(const orc_net* net, uint64_t seed, int32_t R, int64_t m,
                  int64_t* bins, int8_t* signs);
/* Per-tensor sketches x_k = T_k vec(X_k) (Eq. 1 via the hash form, Alg. 3).
 * x_out[r][xoff_k + o_k*m + b], O_k = product of tensor k's open dims. */
int orc_m1_sketch(const orc_net* net, int64_t m, int32_t R, const int64_t* bins,
                  const int8_t* signs, int32_t abs_mode, double* x_out);
/* Per-rep estimates y[r][o] (Alg. 1; open legs per Corollary "full-to-partial")
 * and the cancellation-aware scale s[r][o] = max((1/m) sum_j prod_k |F x_k(j)|,
 * root-sum-square of the terms of y expanded over index combinations). */
int orc_m1_estimate(const orc_net* net, int64_t m, int32_t R, const int64_t* bins,
                    const int8_t* signs, double* y_out, double* s_out);

/* Method 2 (Alg. 2 with Alg. 4 and Alg. 5) for an acyclic full network rooted at
 * `root`. Edge count sketches may be overridden ([R][L], same layout as method 1).
 * s_out = max(||x_o|| ||r_o||, the root-sum-square of the terms of y expanded
 * over all index combinations (the same recursion on X_k^2 with every sign +1)),
 * the scale of rounding tolerances. */
int orc_m2_estimate(const orc_net* net, int32_t root, int64_t m, int32_t R, uint64_t seed,
                    const int64_t* edge_bins, const int8_t* edge_signs,
                    double* y_out, double* s_out);

/* Median of `groups` contiguous group means over reps (Theorem 1 median trick). */
int orc_combine(int32_t R, int64_t O, const double* per_rep, int32_t groups, double* out);

#ifdef __cplusplus
}
#endif
#endif
