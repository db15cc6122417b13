/*
 * tnsk_oracle.c -- FP64 CPU oracle for the sketching estimators of
 * "Approximating Tensor Network Contraction with Sketches" (arXiv 2603.07387).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path. Plain loops in the
 * order the paper states them; no blocking, fusion or reordering. The hash
 * contract is documented in tnsk_oracle.h.
 *
 * Parity status of each function (what pins it) is listed in the tests:
 *   hash       -- SplitMix64 reference sequence, uniformity / independence stats
 *   dft/fft    -- closed forms, each other, numpy.fft
 *   method 1   -- exactness special case, count-sketch inner product (t = 1),
 *                 time-domain convolution and the brute expansion of the proof
 *                 of Lemma "general-expectation-variance", unbiasedness, variance
 *   method 2   -- exactness special case, Eq. 2 with materialised R_k,
 *                 unbiasedness, variance bound of Lemma "acyclic-expectation-variance"
 *   combine    -- brute-force median / mean
 */
#include "tnsk_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* Hash contract                                                              */
/* ------------------------------------------------------------------------- */

#define P61 ((uint64_t)0x1FFFFFFFFFFFFFFFull)

uint64_t orc_splitmix64(uint64_t state) {
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t red61(uint64_t x) {
    uint64_t r = (x & P61) + (x >> 61);
    if (r >= P61) r -= P61;
    return r;
}

/* (a * b) mod P for a, b < P, through a 128-bit product. */
static uint64_t mulmod61(uint64_t a, uint64_t b) {
    unsigned __int128 prod = (unsigned __int128)a * b;
    uint64_t lo = (uint64_t)(prod & P61);
    uint64_t hi = (uint64_t)(prod >> 61);
    return red61(lo + hi);
}

static uint64_t addmod61(uint64_t a, uint64_t b) { return red61(a + b); }

uint64_t orc_tid(int32_t kind, int64_t a, int64_t b, int64_t c, int64_t d) {
    uint64_t k = (uint64_t)kind << 56;
    switch (kind) {
        case 1: /* method 1 edge a */
        case 2: /* method 2 edge a */
            return k | (uint64_t)a;
        case 3: /* padding slot b of tensor a */
            return k | ((uint64_t)a << 24) | (uint64_t)b;
        case 4: /* T_{2^b, c} side d of tensor a */
            return k | ((uint64_t)a << 24) | ((uint64_t)b << 16) | ((uint64_t)c << 1) | (uint64_t)d;
        default:
            return 0;
    }
}

typedef struct {
    uint64_t a0, a1;         /* bin polynomial */
    uint64_t c0, c1, c2, c3; /* sign polynomial */
} hashfn;

static hashfn make_hash(uint64_t seed, uint64_t rep, uint64_t tid) {
    uint64_t key = orc_splitmix64(orc_splitmix64(orc_splitmix64(seed) ^ rep) ^ tid);
    hashfn f;
    f.a0 = red61(orc_splitmix64(key ^ 0));
    f.a1 = red61(orc_splitmix64(key ^ 1));
    f.c0 = red61(orc_splitmix64(key ^ 8));
    f.c1 = red61(orc_splitmix64(key ^ 9));
    f.c2 = red61(orc_splitmix64(key ^ 10));
    f.c3 = red61(orc_splitmix64(key ^ 11));
    return f;
}

static int64_t hash_bin(const hashfn* f, uint64_t i, int64_t m) {
    uint64_t x = red61(i);
    uint64_t v = addmod61(mulmod61(f->a1, x), f->a0);
    return (int64_t)(v % (uint64_t)m);
}

static int8_t hash_sign(const hashfn* f, uint64_t i) {
    uint64_t x = red61(i);
    uint64_t g = f->c3;
    g = addmod61(mulmod61(g, x), f->c2);
    g = addmod61(mulmod61(g, x), f->c1);
    g = addmod61(mulmod61(g, x), f->c0);
    return (g & 1) ? (int8_t)-1 : (int8_t)1;
}

void orc_count_sketch(uint64_t seed, uint64_t rep, uint64_t tid, int64_t n, int64_t m,
                      int64_t* bins, int8_t* signs) {
    hashfn f = make_hash(seed, rep, tid);
    for (int64_t i = 0; i < n; ++i) {
        if (bins) bins[i] = hash_bin(&f, (uint64_t)i, m);
        if (signs) signs[i] = hash_sign(&f, (uint64_t)i);
    }
}

/* ------------------------------------------------------------------------- */
/* Discrete Fourier transform (Sec. 2, F unnormalised with exp(-2 pi i jk/m)) */
/* ------------------------------------------------------------------------- */

void orc_dft(int64_t m, const double* re, const double* im, double* ore, double* oim) {
    for (int64_t k = 0; k < m; ++k) {
        cplx acc = 0;
        for (int64_t j = 0; j < m; ++j) {
            double ang = -2.0 * M_PI * (double)((k * j) % m) / (double)m;
            cplx x = re[j] + (im ? im[j] : 0.0) * I;
            acc += x * cexp(ang * I);
        }
        ore[k] = creal(acc);
        oim[k] = cimag(acc);
    }
}

/* Radix-2 decimation in time: F_n x = [E + w O, E - w O], w_k = exp(-2 pi i k/n). */
static void fft_rec(cplx* x, int64_t n, int64_t stride, cplx* out) {
    if (n == 1) {
        out[0] = x[0];
        return;
    }
    int64_t h = n / 2;
    fft_rec(x, h, 2 * stride, out);
    fft_rec(x + stride, h, 2 * stride, out + h);
    for (int64_t k = 0; k < h; ++k) {
        cplx w = cexp(-2.0 * M_PI * I * (double)k / (double)n);
        cplx e = out[k], o = w * out[k + h];
        out[k] = e + o;
        out[k + h] = e - o;
    }
}

static void fft_c(cplx* x, int64_t m, cplx* out) { fft_rec(x, m, 1, out); }

void orc_fft(int64_t m, const double* re, const double* im, double* ore, double* oim) {
    cplx* x = (cplx*)malloc(sizeof(cplx) * (size_t)m);
    cplx* y = (cplx*)malloc(sizeof(cplx) * (size_t)m);
    for (int64_t j = 0; j < m; ++j) x[j] = re[j] + (im ? im[j] : 0.0) * I;
    fft_c(x, m, y);
    for (int64_t j = 0; j < m; ++j) {
        ore[j] = creal(y[j]);
        oim[j] = cimag(y[j]);
    }
    free(x);
    free(y);
}

/* ------------------------------------------------------------------------- */
/* Network bookkeeping (Def. "Tensor contraction", "Tensor product", "TNC")   */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t q;            /* total number of modes */
    int32_t* mode_off;    /* [p+1] first global mode of tensor k */
    int32_t* tensor_of;   /* [q] tensor owning global mode g */
    int32_t* edge_of;     /* [q] edge index or -1 (open) */
    int32_t* side_of;     /* [q] 0 = first mode of its edge (C), 1 = second (C') */
    int32_t* open_pos;    /* [q] position in the open list or -1 */
    int64_t* eoff;        /* [t+1] table offsets, n_e = dim of the edge */
    int64_t* numel;       /* [p] */
    int64_t* n_opentot;   /* [p] O_k = product of tensor k's open dims */
    int64_t O;            /* product of all open dims */
} netinfo;

static void free_info(netinfo* in) {
    free(in->mode_off);
    free(in->tensor_of);
    free(in->edge_of);
    free(in->side_of);
    free(in->open_pos);
    free(in->eoff);
    free(in->numel);
    free(in->n_opentot);
}

static int64_t dim_of(const orc_net* net, const netinfo* in, int32_t g) {
    (void)in;
    return net->dims[g];
}

/* Validates the statement of Def. "Tensor contraction": u != v, n_u = n_v, every
 * mode in at most one contraction (hyperedges are WLOG 1, not accepted), open
 * list a permutation of K'. */
static int build_info(const orc_net* net, netinfo* in) {
    memset(in, 0, sizeof(*in));
    if (net->p <= 0) return ORC_INVALID;
    in->mode_off = (int32_t*)calloc((size_t)net->p + 1, sizeof(int32_t));
    for (int32_t k = 0; k < net->p; ++k) {
        if (net->order[k] < 0) return ORC_INVALID;
        in->mode_off[k + 1] = in->mode_off[k] + net->order[k];
    }
    in->q = in->mode_off[net->p];
    int32_t q = in->q;
    in->tensor_of = (int32_t*)calloc((size_t)q + 1, sizeof(int32_t));
    in->edge_of = (int32_t*)malloc(sizeof(int32_t) * ((size_t)q + 1));
    in->side_of = (int32_t*)calloc((size_t)q + 1, sizeof(int32_t));
    in->open_pos = (int32_t*)malloc(sizeof(int32_t) * ((size_t)q + 1));
    in->eoff = (int64_t*)calloc((size_t)net->t + 1, sizeof(int64_t));
    in->numel = (int64_t*)calloc((size_t)net->p, sizeof(int64_t));
    in->n_opentot = (int64_t*)calloc((size_t)net->p, sizeof(int64_t));
    for (int32_t k = 0; k < net->p; ++k)
        for (int32_t g = in->mode_off[k]; g < in->mode_off[k + 1]; ++g) in->tensor_of[g] = k;
    for (int32_t g = 0; g < q; ++g) {
        in->edge_of[g] = -1;
        in->open_pos[g] = -1;
        if (net->dims[g] < 0) return ORC_INVALID;
    }
    for (int32_t e = 0; e < net->t; ++e) {
        int32_t u = net->edges[2 * e], v = net->edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= q || v >= q || u == v) return ORC_INVALID;
        if (net->dims[u] != net->dims[v]) return ORC_INVALID;
        if (in->edge_of[u] >= 0 || in->edge_of[v] >= 0) return ORC_UNSUPPORTED;
        in->edge_of[u] = e;
        in->side_of[u] = 0;
        in->edge_of[v] = e;
        in->side_of[v] = 1;
        in->eoff[e + 1] = in->eoff[e] + net->dims[u];
    }
    int32_t n_free = 0;
    for (int32_t g = 0; g < q; ++g)
        if (in->edge_of[g] < 0) ++n_free;
    if (n_free != net->n_open) return ORC_INVALID;
    for (int32_t j = 0; j < net->n_open; ++j) {
        int32_t g = net->open[j];
        if (g < 0 || g >= q || in->edge_of[g] >= 0 || in->open_pos[g] >= 0) return ORC_INVALID;
        in->open_pos[g] = j;
    }
    in->O = 1;
    for (int32_t j = 0; j < net->n_open; ++j) in->O *= net->dims[net->open[j]];
    for (int32_t k = 0; k < net->p; ++k) {
        int64_t n = 1, o = 1;
        for (int32_t g = in->mode_off[k]; g < in->mode_off[k + 1]; ++g) {
            n *= net->dims[g];
            if (in->edge_of[g] < 0) o *= net->dims[g];
        }
        in->numel[k] = n;
        in->n_opentot[k] = o;
    }
    (void)dim_of;
    return ORC_OK;
}

/* Row-major multi-index of flat index f of tensor k (vec() order, Sec. 2). */
static void unravel(const orc_net* net, const netinfo* in, int32_t k, int64_t f, int64_t* idx) {
    int32_t lo = in->mode_off[k], hi = in->mode_off[k + 1];
    for (int32_t g = hi - 1; g >= lo; --g) {
        int64_t n = net->dims[g];
        idx[g - lo] = f % n;
        f /= n;
    }
}

/* ------------------------------------------------------------------------- */
/* Method 1: complement count sketches, Eq. 1 and Alg. 1                      */
/* ------------------------------------------------------------------------- */

int orc_m1_tables(const orc_net* net, uint64_t seed, int32_t R, int64_t m, int64_t* bins,
                  int8_t* signs) {
    netinfo in;
    int st = build_info(net, &in);
    if (st == ORC_OK) {
        int64_t L = in.eoff[net->t];
        for (int32_t r = 0; r < R; ++r)
            for (int32_t e = 0; e < net->t; ++e) {
                int64_t n = in.eoff[e + 1] - in.eoff[e];
                orc_count_sketch(seed, (uint64_t)r, orc_tid(1, e, 0, 0, 0), n, m,
                                 bins + (int64_t)r * L + in.eoff[e], signs + (int64_t)r * L + in.eoff[e]);
            }
    }
    free_info(&in);
    return st;
}

static int64_t m1_x_per_rep(const orc_net* net, const netinfo* in, int64_t m, int64_t* xoff) {
    int64_t acc = 0;
    for (int32_t k = 0; k < net->p; ++k) {
        if (xoff) xoff[k] = acc;
        acc += in->n_opentot[k] * m;
    }
    return acc;
}

/* x_k = T_k vec(X_k) with T_k the tensor sketch of the count sketches of the
 * modes of X_k (Eq. 1, Alg. 1 "x_k <- T_k vec(X_k)"), evaluated per component by
 * TensorSketchHash (Alg. 3): sigma = prod_u s_u(i_u), b = sum_u h_u(i_u) mod m,
 * where the second mode of every contraction uses the complement (Def.
 * "Complement count sketch"). Open modes are not hashed: they index separate
 * sketches, one per open multi-index of the tensor (Corollary
 * "full-to-partial-tc": the estimator applied to each subtensor). */
static void m1_sketch_one(const orc_net* net, const netinfo* in, int64_t m, const int64_t* bins,
                          const int8_t* signs, int abs_mode, int32_t k, double* xk) {
    int32_t qk = net->order[k];
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * ((size_t)qk + 1));
    memset(xk, 0, sizeof(double) * (size_t)(in->n_opentot[k] * m));
    for (int64_t f = 0; f < in->numel[k]; ++f) {
        unravel(net, in, k, f, idx);
        int64_t sigma = 1, b = 0, o = 0;
        for (int32_t d = 0; d < qk; ++d) {
            int32_t g = in->mode_off[k] + d;
            int32_t e = in->edge_of[g];
            if (e < 0) {
                o = o * net->dims[g] + idx[d];
                continue;
            }
            int64_t h = bins[in->eoff[e] + idx[d]];
            if (in->side_of[g] == 1) h = (m - h) % m; /* complement: -h mod m */
            b += h;
            if (!abs_mode) sigma *= signs[in->eoff[e] + idx[d]];
        }
        b %= m;
        double v = net->data[k][f];
        if (abs_mode == 1) v = fabs(v);
        if (abs_mode == 2) v = v * v;
        xk[o * m + b] += (double)sigma * v;
    }
    free(idx);
}

int orc_m1_sketch(const orc_net* net, int64_t m, int32_t R, const int64_t* bins, const int8_t* signs,
                  int32_t abs_mode, double* x_out) {
    netinfo in;
    int st = build_info(net, &in);
    if (st != ORC_OK || m < 1) {
        free_info(&in);
        return st != ORC_OK ? st : ORC_INVALID;
    }
    int64_t L = in.eoff[net->t];
    int64_t* xoff = (int64_t*)malloc(sizeof(int64_t) * (size_t)net->p);
    int64_t X = m1_x_per_rep(net, &in, m, xoff);
    for (int32_t r = 0; r < R; ++r)
        for (int32_t k = 0; k < net->p; ++k)
            m1_sketch_one(net, &in, m, bins + (int64_t)r * L, signs + (int64_t)r * L, abs_mode, k,
                          x_out + (int64_t)r * X + xoff[k]);
    free(xoff);
    free_info(&in);
    return ORC_OK;
}

/* Alg. 1: z = prod_k F x_k (Hadamard), y = (1/m) sum_j z_j. For an open output
 * entry o, each tensor contributes the spectrum of its sketch at its own part
 * of o. The scale s_out is the larger of (1/m) sum_j prod_k |F x_k(j)| and the
 * root-sum-square of the terms of the expansion of y in the proof of Lemma
 * "general-expectation-variance" (the same estimator on X_k^2 with unit signs). */
int orc_m1_estimate(const orc_net* net, int64_t m, int32_t R, const int64_t* bins, const int8_t* signs,
                    double* y_out, double* s_out) {
    netinfo in;
    int st = build_info(net, &in);
    if (st != ORC_OK || m < 1) {
        free_info(&in);
        return st != ORC_OK ? st : ORC_INVALID;
    }
    int64_t L = in.eoff[net->t];
    int64_t* xoff = (int64_t*)malloc(sizeof(int64_t) * (size_t)net->p);
    int64_t X = m1_x_per_rep(net, &in, m, xoff);
    double* x = (double*)malloc(sizeof(double) * (size_t)(X > 0 ? X : 1));
    cplx* xf = (cplx*)malloc(sizeof(cplx) * (size_t)(X > 0 ? X : 1));
    cplx* xf2 = (cplx*)malloc(sizeof(cplx) * (size_t)(X > 0 ? X : 1)); /* squared terms */
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)m);
    int64_t* oidx = (int64_t*)malloc(sizeof(int64_t) * ((size_t)net->n_open + 1));
    int64_t* ok = (int64_t*)malloc(sizeof(int64_t) * (size_t)net->p);
    for (int32_t r = 0; r < R; ++r) {
        for (int32_t k = 0; k < net->p; ++k) {
            m1_sketch_one(net, &in, m, bins + (int64_t)r * L, signs + (int64_t)r * L, 0, k, x + xoff[k]);
            for (int64_t o = 0; o < in.n_opentot[k]; ++o) {
                for (int64_t j = 0; j < m; ++j) tmp[j] = x[xoff[k] + o * m + j];
                fft_c(tmp, m, xf + xoff[k] + o * m); /* F x_k */
            }
            if (s_out) {
                m1_sketch_one(net, &in, m, bins + (int64_t)r * L, signs + (int64_t)r * L, 2, k, x + xoff[k]);
                for (int64_t o = 0; o < in.n_opentot[k]; ++o) {
                    for (int64_t j = 0; j < m; ++j) tmp[j] = x[xoff[k] + o * m + j];
                    fft_c(tmp, m, xf2 + xoff[k] + o * m);
                }
            }
        }
        for (int64_t o = 0; o < in.O; ++o) {
            /* output multi-index over the open list, row-major */
            int64_t rem = o;
            for (int32_t j = net->n_open - 1; j >= 0; --j) {
                int64_t n = net->dims[net->open[j]];
                oidx[j] = rem % n;
                rem /= n;
            }
            for (int32_t k = 0; k < net->p; ++k) {
                int64_t a = 0;
                for (int32_t g = in.mode_off[k]; g < in.mode_off[k + 1]; ++g)
                    if (in.edge_of[g] < 0) a = a * net->dims[g] + oidx[in.open_pos[g]];
                ok[k] = a;
            }
            cplx acc = 0, acc2 = 0;
            double sacc = 0;
            for (int64_t j = 0; j < m; ++j) {
                cplx z = 1, z2 = 1;
                double za = 1;
                for (int32_t k = 0; k < net->p; ++k) {
                    cplx v = xf[xoff[k] + ok[k] * m + j];
                    z *= v;
                    za *= cabs(v);
                    if (s_out) z2 *= xf2[xoff[k] + ok[k] * m + j];
                }
                acc += z;
                acc2 += z2;
                sacc += za;
            }
            y_out[(int64_t)r * in.O + o] = creal(acc) / (double)m;
            if (s_out) {
                double rss = sqrt(fmax(creal(acc2) / (double)m, 0.0));
                s_out[(int64_t)r * in.O + o] = fmax(sacc / (double)m, rss);
            }
        }
    }
    free(x);
    free(xf);
    free(xf2);
    free(tmp);
    free(oidx);
    free(ok);
    free(xoff);
    free_info(&in);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Method 2: recursive sketches on the rooted tree (Eq. 2, Alg. 2, 4, 5)       */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t parent;       /* parent tensor or -1 for the root */
    int32_t parent_mode;  /* local mode contracting with the parent, -1 for root */
    int32_t parent_edge;  /* edge to the parent */
    int32_t c;            /* number of children |Gamma(k)| */
    int32_t qt;           /* slots: next power of two >= c (0 for a leaf) */
    int32_t* child;       /* [c] child tensors, in the order of k's modes */
    int32_t* child_mode;  /* [c] local mode of k for each child */
    int32_t* child_edge;  /* [c] edge of each child */
} tnode;

typedef struct {
    const orc_net* net;
    netinfo in;
    tnode* node;
    int64_t m;
    int sq_mode; /* 1: entries squared and every sign +1 (root-sum-square pass) */
    /* tables of the current rep */
    const int64_t* ebins;   /* [L] edge count sketches C_{k,l} */
    const int8_t* esigns;
    int64_t** pad_bin;      /* [p][qt] (only slots >= c used) */
    int8_t** pad_sign;
    int64_t** t_bin;        /* [p][(qt-1)*2*m]: T_{l,j} sides, level-major */
    int8_t** t_sign;
} m2ctx;

static int32_t next_pow2(int32_t c) {
    int32_t q = 1;
    while (q < c) q <<= 1;
    return q;
}

static int32_t ilog2(int32_t x) {
    int32_t l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

/* Offset of T_{l,j} side s inside tensor k's T table block: levels are stored
 * from l = qt down to 2; level l holds l/2 pairs. */
static int64_t t_off(int32_t qt, int32_t l, int32_t j, int32_t s, int64_t m) {
    int64_t pairs_before = 0;
    for (int32_t ll = qt; ll > l; ll >>= 1) pairs_before += ll / 2;
    return ((pairs_before + j) * 2 + s) * m;
}

/* RecursiveSketchHash (Alg. 4): base count sketches on every slot, then the
 * binary reduction l = qt, qt/2, ..., 2 by TensorSketchHash (Alg. 3) of the
 * pair (b_{2j}, b_{2j+1}) with T_{l,j}. slot_idx holds the index value of each
 * real child slot; padding slots use index 0 (the e_1 embedding of the footnote
 * to Def. "Recursive sketch"). */
static void rsh(const m2ctx* cx, int32_t k, const int64_t* slot_idx, int64_t* b, int64_t* sigma_out,
                int64_t* bin_out) {
    const tnode* nd = &cx->node[k];
    int64_t m = cx->m;
    int64_t sigma = 1;
    if (nd->qt == 0) {
        *sigma_out = 1;
        *bin_out = 0;
        return;
    }
    for (int32_t j = 0; j < nd->qt; ++j) {
        if (j < nd->c) {
            int32_t e = nd->child_edge[j];
            int64_t pos = cx->in.eoff[e] + slot_idx[j];
            b[j] = cx->ebins[pos];
            if (!cx->sq_mode) sigma *= cx->esigns[pos];
        } else {
            b[j] = cx->pad_bin[k][j];
            if (!cx->sq_mode) sigma *= cx->pad_sign[k][j];
        }
    }
    for (int32_t l = nd->qt; l >= 2; l >>= 1) {
        for (int32_t j = 0; j < l / 2; ++j) {
            const int64_t* ha = cx->t_bin[k] + t_off(nd->qt, l, j, 0, m);
            const int64_t* hb = cx->t_bin[k] + t_off(nd->qt, l, j, 1, m);
            const int8_t* sa = cx->t_sign[k] + t_off(nd->qt, l, j, 0, m);
            const int8_t* sb = cx->t_sign[k] + t_off(nd->qt, l, j, 1, m);
            if (!cx->sq_mode) sigma *= sa[b[2 * j]] * sb[b[2 * j + 1]];
            b[j] = (ha[b[2 * j]] + hb[b[2 * j + 1]]) % m;
        }
    }
    *sigma_out = sigma;
    *bin_out = b[0];
}

/* Child-slot index values of a component of tensor k. */
static void slot_values(const m2ctx* cx, int32_t k, const int64_t* idx, int64_t* slot_idx) {
    const tnode* nd = &cx->node[k];
    for (int32_t j = 0; j < nd->c; ++j) slot_idx[j] = idx[nd->child_mode[j]];
}

static double* neighbors_sketch(const m2ctx* cx, int32_t k);

/* SketchedMatrixVectorProduct (Alg. 5): y = C mat(X_l) R_l^T z, with C the count
 * sketch of the edge to the parent applied to the parent mode, and (sigma, b)
 * of R_l from Alg. 4 on the remaining (child) modes. */
static double* sketched_matvec(const m2ctx* cx, int32_t l, const double* z) {
    const orc_net* net = cx->net;
    const tnode* nd = &cx->node[l];
    int64_t m = cx->m;
    int32_t ql = net->order[l];
    double* y = (double*)calloc((size_t)m, sizeof(double));
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * ((size_t)ql + 1));
    int64_t* sidx = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nd->qt + 1));
    int64_t* b = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nd->qt + 1));
    for (int64_t f = 0; f < cx->in.numel[l]; ++f) {
        unravel(net, &cx->in, l, f, idx);
        int64_t ipar = idx[nd->parent_mode];
        int64_t pos = cx->in.eoff[nd->parent_edge] + ipar;
        int64_t j = cx->ebins[pos];
        int64_t s = cx->sq_mode ? 1 : cx->esigns[pos];
        slot_values(cx, l, idx, sidx);
        int64_t sigma, bb;
        rsh(cx, l, sidx, b, &sigma, &bb);
        double v = net->data[l][f];
        if (cx->sq_mode) v = v * v;
        y[j] += v * z[bb] * (double)sigma * (double)s;
    }
    free(idx);
    free(sidx);
    free(b);
    return y;
}

/* T(u (x) v) for a tensor sketch T of order 2 made of count sketches (ha, sa)
 * and (hb, sb) on [m]: component form of Def. "Tensor sketch" (Alg. 3). */
static double* tensor_sketch_pair(const m2ctx* cx, const int64_t* ha, const int8_t* sa, const int64_t* hb,
                                  const int8_t* sb, const double* u, const double* v) {
    int64_t m = cx->m;
    double* out = (double*)calloc((size_t)m, sizeof(double));
    for (int64_t a = 0; a < m; ++a) {
        if (u[a] == 0.0) continue;
        for (int64_t c = 0; c < m; ++c) {
            double sg = cx->sq_mode ? 1.0 : (double)(sa[a] * sb[c]);
            out[(ha[a] + hb[c]) % m] += sg * u[a] * v[c];
        }
    }
    return out;
}

/* NeighborsSketch (Alg. 2): r_k = Q_k( (x) over slots of x_l ), where every real
 * child l gives x_l = C_{k,l} mat(X_l) R_l^T r_l and every padding slot the count
 * sketch of e_1. A leaf returns the scalar 1. */
static double* neighbors_sketch(const m2ctx* cx, int32_t k) {
    const tnode* nd = &cx->node[k];
    int64_t m = cx->m;
    if (nd->c == 0) {
        double* one = (double*)malloc(sizeof(double));
        one[0] = 1.0;
        return one;
    }
    double** x = (double**)malloc(sizeof(double*) * (size_t)nd->qt);
    for (int32_t j = 0; j < nd->qt; ++j) {
        if (j < nd->c) {
            int32_t l = nd->child[j];
            double* rl = neighbors_sketch(cx, l);
            x[j] = sketched_matvec(cx, l, rl);
            free(rl);
        } else {
            x[j] = (double*)calloc((size_t)m, sizeof(double));
            x[j][cx->pad_bin[k][j]] = cx->sq_mode ? 1.0 : (double)cx->pad_sign[k][j];
        }
    }
    /* Q_k = Q_2 Q_4 ... Q_qt: apply level qt first, then qt/2, ..., 2 */
    for (int32_t l = nd->qt; l >= 2; l >>= 1) {
        for (int32_t j = 0; j < l / 2; ++j) {
            int64_t o0 = t_off(nd->qt, l, j, 0, m), o1 = t_off(nd->qt, l, j, 1, m);
            double* y = tensor_sketch_pair(cx, cx->t_bin[k] + o0, cx->t_sign[k] + o0, cx->t_bin[k] + o1,
                                           cx->t_sign[k] + o1, x[2 * j], x[2 * j + 1]);
            free(x[2 * j]);
            free(x[2 * j + 1]);
            x[2 * j] = NULL;
            x[2 * j + 1] = NULL;
            x[j] = y;
        }
    }
    double* r = x[0];
    free(x);
    return r;
}

int orc_m2_estimate(const orc_net* net, int32_t root, int64_t m, int32_t R, uint64_t seed,
                    const int64_t* edge_bins, const int8_t* edge_signs, double* y_out, double* s_out) {
    m2ctx cx;
    memset(&cx, 0, sizeof(cx));
    cx.net = net;
    cx.m = m;
    int st = build_info(net, &cx.in);
    if (st != ORC_OK || m < 1 || root < 0 || root >= net->p) {
        free_info(&cx.in);
        return st != ORC_OK ? st : ORC_INVALID;
    }
    int32_t p = net->p;
    if (net->n_open != 0) {
        free_info(&cx.in);
        return ORC_UNSUPPORTED;
    }
    /* acyclic and connected: a tree has t = p - 1 edges, no self contraction
     * and every tensor reachable from the root */
    for (int32_t e = 0; e < net->t; ++e)
        if (cx.in.tensor_of[net->edges[2 * e]] == cx.in.tensor_of[net->edges[2 * e + 1]]) {
            free_info(&cx.in);
            return ORC_CYCLIC;
        }
    if (net->t != p - 1) {
        free_info(&cx.in);
        return net->t > p - 1 ? ORC_CYCLIC : ORC_UNSUPPORTED;
    }
    cx.node = (tnode*)calloc((size_t)p, sizeof(tnode));
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)p);
    int32_t* seen = (int32_t*)calloc((size_t)p, sizeof(int32_t));
    for (int32_t k = 0; k < p; ++k) {
        cx.node[k].parent = -1;
        cx.node[k].parent_mode = -1;
        cx.node[k].parent_edge = -1;
        cx.node[k].child = (int32_t*)malloc(sizeof(int32_t) * ((size_t)net->order[k] + 1));
        cx.node[k].child_mode = (int32_t*)malloc(sizeof(int32_t) * ((size_t)net->order[k] + 1));
        cx.node[k].child_edge = (int32_t*)malloc(sizeof(int32_t) * ((size_t)net->order[k] + 1));
    }
    int32_t head = 0, tail = 0, nseen = 1;
    queue[tail++] = root;
    seen[root] = 1;
    while (head < tail) {
        int32_t k = queue[head++];
        /* children of k in the order of k's modes (footnote to Gamma(k)) */
        for (int32_t g = cx.in.mode_off[k]; g < cx.in.mode_off[k + 1]; ++g) {
            int32_t e = cx.in.edge_of[g];
            int32_t other = net->edges[2 * e] == g ? net->edges[2 * e + 1] : net->edges[2 * e];
            int32_t l = cx.in.tensor_of[other];
            if (l == cx.node[k].parent && e == cx.node[k].parent_edge) continue;
            if (seen[l]) {
                st = ORC_CYCLIC;
                break;
            }
            seen[l] = 1;
            ++nseen;
            tnode* nk = &cx.node[k];
            nk->child[nk->c] = l;
            nk->child_mode[nk->c] = g - cx.in.mode_off[k];
            nk->child_edge[nk->c] = e;
            nk->c++;
            cx.node[l].parent = k;
            cx.node[l].parent_edge = e;
            cx.node[l].parent_mode = other - cx.in.mode_off[l];
            queue[tail++] = l;
        }
        if (st != ORC_OK) break;
    }
    if (st == ORC_OK && nseen != p) st = ORC_UNSUPPORTED; /* disconnected */
    int64_t L = cx.in.eoff[net->t];
    int64_t* eb = NULL;
    int8_t* es = NULL;
    if (st == ORC_OK) {
        for (int32_t k = 0; k < p; ++k) {
            cx.node[k].qt = cx.node[k].c == 0 ? 0 : next_pow2(cx.node[k].c);
        }
        cx.pad_bin = (int64_t**)calloc((size_t)p, sizeof(int64_t*));
        cx.pad_sign = (int8_t**)calloc((size_t)p, sizeof(int8_t*));
        cx.t_bin = (int64_t**)calloc((size_t)p, sizeof(int64_t*));
        cx.t_sign = (int8_t**)calloc((size_t)p, sizeof(int8_t*));
        for (int32_t k = 0; k < p; ++k) {
            int32_t qt = cx.node[k].qt;
            cx.pad_bin[k] = (int64_t*)calloc((size_t)qt + 1, sizeof(int64_t));
            cx.pad_sign[k] = (int8_t*)calloc((size_t)qt + 1, sizeof(int8_t));
            int64_t nt = qt > 1 ? (int64_t)(qt - 1) * 2 * m : 1;
            cx.t_bin[k] = (int64_t*)calloc((size_t)nt, sizeof(int64_t));
            cx.t_sign[k] = (int8_t*)calloc((size_t)nt, sizeof(int8_t));
        }
        eb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(L > 0 ? L : 1));
        es = (int8_t*)malloc(sizeof(int8_t) * (size_t)(L > 0 ? L : 1));
    }
    for (int32_t r = 0; st == ORC_OK && r < R; ++r) {
        /* draw the rep's independent sketches (Alg. 2: R_o and every R_k) */
        if (edge_bins) {
            memcpy(eb, edge_bins + (int64_t)r * L, sizeof(int64_t) * (size_t)L);
            memcpy(es, edge_signs + (int64_t)r * L, sizeof(int8_t) * (size_t)L);
        } else {
            for (int32_t e = 0; e < net->t; ++e)
                orc_count_sketch(seed, (uint64_t)r, orc_tid(2, e, 0, 0, 0), cx.in.eoff[e + 1] - cx.in.eoff[e], m,
                                 eb + cx.in.eoff[e], es + cx.in.eoff[e]);
        }
        cx.ebins = eb;
        cx.esigns = es;
        for (int32_t k = 0; k < p; ++k) {
            int32_t qt = cx.node[k].qt;
            for (int32_t j = cx.node[k].c; j < qt; ++j) {
                int64_t hb;
                int8_t sg;
                orc_count_sketch(seed, (uint64_t)r, orc_tid(3, k, j, 0, 0), 1, m, &hb, &sg);
                cx.pad_bin[k][j] = hb;
                cx.pad_sign[k][j] = sg;
            }
            for (int32_t l = qt; l >= 2; l >>= 1)
                for (int32_t j = 0; j < l / 2; ++j)
                    for (int32_t s = 0; s < 2; ++s) {
                        int64_t o = t_off(qt, l, j, s, m);
                        orc_count_sketch(seed, (uint64_t)r, orc_tid(4, k, ilog2(l), j, s), m, m, cx.t_bin[k] + o,
                                         cx.t_sign[k] + o);
                    }
        }
        for (int pass = 0; pass < (s_out ? 2 : 1); ++pass) {
            cx.sq_mode = pass;
            /* x_o = R_o vec(X_o): scatter every component of the root by Alg. 4 */
            const tnode* nd = &cx.node[root];
            int32_t qo = net->order[root];
            double* xo = (double*)calloc((size_t)m, sizeof(double));
            int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * ((size_t)qo + 1));
            int64_t* sidx = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nd->qt + 1));
            int64_t* b = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nd->qt + 1));
            for (int64_t f = 0; f < cx.in.numel[root]; ++f) {
                unravel(net, &cx.in, root, f, idx);
                slot_values(&cx, root, idx, sidx);
                int64_t sigma, bb;
                rsh(&cx, root, sidx, b, &sigma, &bb);
                double v = net->data[root][f];
                if (cx.sq_mode) v = v * v;
                xo[bb] += (double)sigma * v;
            }
            /* r_o = NeighborsSketch(o); y = x_o^T r_o */
            double* ro = neighbors_sketch(&cx, root);
            int64_t len = nd->c == 0 ? 1 : m;
            double y = 0, nx = 0, nr = 0;
            for (int64_t j = 0; j < len; ++j) {
                y += xo[j] * ro[j];
                nx += xo[j] * xo[j];
                nr += ro[j] * ro[j];
            }
            if (pass == 0) {
                y_out[r] = y;
                /* |y| <= ||x_o|| ||r_o|| (Cauchy-Schwarz) */
                if (s_out) s_out[r] = sqrt(nx) * sqrt(nr);
            } else { /* root-sum-square of the terms of the expansion of Eq. 2 */
                s_out[r] = fmax(s_out[r], sqrt(fmax(y, 0.0)));
            }
            free(ro);
            free(xo);
            free(idx);
            free(sidx);
            free(b);
        }
    }
    if (cx.node) {
        for (int32_t k = 0; k < p; ++k) {
            free(cx.node[k].child);
            free(cx.node[k].child_mode);
            free(cx.node[k].child_edge);
            if (cx.pad_bin) {
                free(cx.pad_bin[k]);
                free(cx.pad_sign[k]);
                free(cx.t_bin[k]);
                free(cx.t_sign[k]);
            }
        }
    }
    free(cx.pad_bin);
    free(cx.pad_sign);
    free(cx.t_bin);
    free(cx.t_sign);
    free(cx.node);
    free(queue);
    free(seen);
    free(eb);
    free(es);
    free_info(&cx.in);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Combination of repetitions (Theorem 1, median trick)                       */
/* ------------------------------------------------------------------------- */

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

int orc_combine(int32_t R, int64_t O, const double* per_rep, int32_t groups, double* out) {
    if (R < 1 || groups < 1 || R % groups != 0) return ORC_INVALID;
    int32_t gs = R / groups;
    double* means = (double*)malloc(sizeof(double) * (size_t)groups);
    for (int64_t o = 0; o < O; ++o) {
        for (int32_t g = 0; g < groups; ++g) {
            double s = 0;
            for (int32_t r = g * gs; r < (g + 1) * gs; ++r) s += per_rep[(int64_t)r * O + o];
            means[g] = s / (double)gs;
        }
        qsort(means, (size_t)groups, sizeof(double), cmp_double);
        out[o] = (groups % 2) ? means[groups / 2] : 0.5 * (means[groups / 2 - 1] + means[groups / 2]);
    }
    free(means);
    return ORC_OK;
}
