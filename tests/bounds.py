"""Error bars of the mixed-precision parity tests, derived from a rounding model.

Mixed modes compute X_i = L_i^{-1} P B_i^T in FP32 (panel updates on the
tensor cores in split bf16) and F_i = X_i^T X_i on the tensor cores with FP32
accumulation.  For the SYRK, with X the FP32 operand and K = n_i the longest
reduction:

  * TF32: X is rounded to TF32 (10 explicit mantissa bits, to nearest), so
    each operand carries a relative error of at most u_t = 2^-11; products of
    two TF32 values are exact in FP32.
  * split bf16: x = hi + lo + e with hi = bf16(x), lo = bf16(x - hi), so
    |e| <= 2^-16 |x|; the product is summed as hi*hi' + hi*lo' + lo*hi', which
    drops lo*lo' (<= 2^-16 |x y|) and the terms with e or e': at most
    3 * 2^-16 |x y| per product.
  * FP32 accumulation of K terms (the tensor cores may truncate rather than
    round, so u_acc = 2^-23): gamma_K = K u_acc / (1 - K u_acc).

Entrywise |F^ - X^T X| <= c (|X|^T |X|) with c = 2 u_t + u_t^2 + gamma_K
(TF32) or 3 * 2^-16 + gamma_K (split), and by Cauchy-Schwarz
(|X|^T |X|)_ab <= ||X_a|| ||X_b|| = sqrt(F_aa F_bb), so
||F^ - X^T X||_F <= c tr(F).  Both mixed modes run the same TRSM, so
F_tf32 - F_split isolates the two SYRK roundings:
||F_tf32 - F_split||_F <= (c_tf32 + c_split) tr(F).  The split-bf16 path is
held to the FP32-level bar SPLIT_BAR against the FP64 oracle (it covers the
FP32 TRSM as well), and the TF32 bar against the oracle follows by the
triangle inequality.
"""
from __future__ import annotations

import numpy as np

U_TF32 = 2.0 ** -11
U_ACC = 2.0 ** -23
SPLIT_OPERAND = 3 * 2.0 ** -16
SPLIT_BAR = 1e-4      # relative Frobenius error of split-bf16 F_i against the FP64 oracle
FP64_BAR = 1e-12      # the plain FP64 path: relative Frobenius error of F_i


def gamma(k: int, u: float = U_ACC) -> float:
    return k * u / (1.0 - k * u)


def syrk_coeff(prec: str, K: int) -> float:
    """c of |F^ - X^T X| <= c |X|^T |X| for the tensor-core SYRK in `prec`."""
    if prec == "tf32":
        return 2 * U_TF32 + U_TF32 ** 2 + gamma(K)
    if prec == "split_bf16":
        return SPLIT_OPERAND + gamma(K)
    raise ValueError(prec)


def tf32_vs_split_bar(F: np.ndarray, n: int) -> float:
    """Absolute Frobenius bound on F_tf32 - F_split for one subdomain."""
    return (syrk_coeff("tf32", n) + syrk_coeff("split_bf16", n)) * float(np.trace(F))


def F_bar(prec: str, F: np.ndarray, n: int) -> float:
    """Relative Frobenius bar of the GPU F_i against the oracle's F (n = DOFs of the subdomain)."""
    if prec == "fp64":
        return FP64_BAR
    if prec == "split_bf16":
        return SPLIT_BAR
    if prec == "tf32":
        return tf32_vs_split_bar(F, n) / np.linalg.norm(F) + SPLIT_BAR
    raise ValueError(prec)


def apply_scale(subs, Fs, p: np.ndarray, n_lambda: int) -> np.ndarray:
    """Componentwise scale of q = F p: s_j = sum over the subdomains i owning
    multiplier j of sqrt(F_i[j, j]) * sum_k sqrt(F_i[k, k]) |p_k|.  An error
    |dF_ab| <= c sqrt(F_aa F_bb) in F_i (the Cauchy-Schwarz form above, and the
    natural form of a columnwise-relative error in X_i) changes q_j by at most
    c s_j."""
    s = np.zeros(n_lambda)
    for sub, F in zip(subs, Fs):
        lam = np.asarray(sub.B_lambda, dtype=np.int64)
        d = np.sqrt(np.maximum(np.diag(F), 0.0))
        np.add.at(s, lam, d * float(d @ np.abs(p[lam])))
    return s
