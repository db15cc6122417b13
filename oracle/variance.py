"""Exact variance of one repetition of the prior (cross-correlation) estimator on the
all-ones chain of Lemma "exponential-dependence" (Sec. 4.3), in FP64 (test
infrastructure only: the tests and the benchmark's CPU-side legs are the callers).

The chain: X_1 = 1_n, X_2 .. X_q = 1_{n x n}, X_{q+1} = 1_n, contraction k between
X_k and X_{k+1} with its own count sketch C_k (bins h_k: 2-wise independent, signs
s_k: 4-wise independent, independent across k). The proof of the lemma reduces one
repetition to y = ||s||^2 with s = T(1_n^{(x) q}) the tensor sketch of the all-ones
order-q tensor: s[b] = sum_{i in [n]^q} prod_k s_k(i_k) [sum_k h_k(i_k) = b mod m].

So y = sum_{i, j} sigma(i) sigma(j) [h(i) = h(j)] and E[y] = n^q = tc. For E[y^2]
= sum over (i, j, i', j') of E[sigma(i) sigma(j) sigma(i') sigma(j')] P(h(i) = h(j),
h(i') = h(j')): per mode k the sign factor is 1 exactly when the four indices pair up,
and otherwise 0. Per mode the pairings are
  - all four equal, or i_k = j_k != i'_k = j'_k: n^2 index tuples, no bin difference;
  - i_k = i'_k = a != b = j_k = j'_k ("B"): n(n - 1) tuples; the difference
    d_k = h_k(a) - h_k(b), uniform on Z_m, enters both bin conditions;
  - i_k = j'_k = a != b = j_k = i'_k ("C"): n(n - 1) tuples; d_k enters the first
    condition and -d_k the second.
With S_B, S_C the sums of the d_k of the B and C modes, the conditions are
S_B + S_C = 0 and S_B - S_C = 0 (mod m): probability 1 with no B or C mode, 1/m with
only one of the kinds present, and P(S_B = S_C, 2 S_C = 0) = (1/m)(g/m) with both
(g = 2 for even m, 1 for odd m). Summing the multinomial counts,
  Var[y] = n^{2q} [ (2/m) ((1 + u)^q - 1) + (g/m^2) ((1 + 2u)^q - 2 (1 + u)^q + 1) ],
u = 1 - 1/n, and n^{2q} = prod_k ||X_k||_F^2 (the normalisation of the lemma).
The formula assumes exactly uniform bin differences and exactly 4-wise independent
signs (an ideal family; the library's polynomial hashes mod 2^61 - 1 reduced mod m
are within ~m / 2^61 of it).

parity: pinned by tests/test_oracle_variance.py against the exact mean and variance
over all hash functions of tiny domains (brute-force enumeration).
"""
from __future__ import annotations


def chain_allones_variance(n: int, q: int, m: int) -> float:
    """Var[y] / prod_k ||X_k||_F^2 for one repetition on the all-ones chain (q
    contractions, bond n, sketch size m); see the module docstring."""
    u = 1.0 - 1.0 / n
    g = 2.0 if m % 2 == 0 else 1.0
    a = (1.0 + u) ** q
    return (2.0 / m) * (a - 1.0) + (g / (m * m)) * ((1.0 + 2.0 * u) ** q - 2.0 * a + 1.0)


def lemma_lower_bound(q: int, m: int) -> float:
    """The lemma's stated lower bound (3^q / (2 m^2) - 1), as a fraction of
    prod_k ||X_k||_F^2."""
    return 3.0 ** q / (2.0 * m * m) - 1.0
