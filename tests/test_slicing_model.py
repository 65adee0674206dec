"""Host model of the exact bf16 slicing that the tensor-core Cholesky uses for
the rank-k updates of its large fronts (`chol_tc_kernel`): every FP64 entry
of a row scaled by 2^(e_i - 6) (e_i the row's largest exponent) and its 63
leading fixed-point bits cut into 9 signed 7-bit integers; products of slices
p, q with p + q <= 8 summed per d = p + q in FP32, the d = 8 products into the
d = 7 accumulator with a factor 2^-7 (exact for d <= 6: every partial sum an
integer below 2^24 for K = 128); recombined as
2^(e_i + e_j - 40) (sum_{d<=4} acc_d 2^(7(4-d)) + small), the first sum in
64-bit integers, `small` the FP32 Horner sum of the d >= 5 accumulators.

The model repeats the kernel's arithmetic on the host (integer matrix products
for the slice products, float32 for the small accumulators and their Horner
sum, float64 for the last step) and checks it against the exact dot products
(Python integers): the integer bounds behind the exactness claims (every
accumulator with d <= 6 an integer below 2^24), and the error bound
K 2^-52 sigma_i sigma_j (sigma = 2^(e + 1) above every entry of the row: FP64's
own normwise bound for a K-term dot product is larger), on rows whose entries
spread over 2^-12 .. 1 of their largest."""
import math

import numpy as np
import pytest

K = 128
S = 9


def _slices(A):
    """Row exponents and the 9 slices (int64 arrays, sign included) of A (n x K, float64)."""
    n = A.shape[0]
    ex = np.zeros(n, dtype=np.int64)
    sl = np.zeros((S, n, A.shape[1]), dtype=np.int64)
    for i in range(n):
        nz = A[i][A[i] != 0]
        e = max(math.frexp(float(x))[1] - 1 for x in nz) if nz.size else -1074
        ex[i] = e
        for k, x in enumerate(A[i]):
            if x == 0:
                continue
            m, be = math.frexp(abs(float(x)))      # |x| = m 2^be, m in [0.5, 1)
            mant = int(m * (1 << 53))              # 53-bit integer mantissa
            shift = (be - 53) + 62 - e             # |x| = mant 2^(be - 53); F = |x| 2^(62 - e)
            F = mant << shift if shift >= 0 else mant >> -shift
            assert F < (1 << 63)
            for p in range(S):
                v = (F >> (56 - 7 * p)) & 127
                sl[p, i, k] = -v if x < 0 else v
    return ex, sl


def _model(A):
    ex, sl = _slices(A)
    n = A.shape[0]
    acc = [np.zeros((n, n), dtype=np.int64) for _ in range(S)]
    for p in range(S):
        for q in range(S - p):
            acc[p + q] += sl[p] @ sl[q].T
    bound = [int(np.abs(a).max()) for a in acc]
    I = sum(acc[d] << (7 * (4 - d)) for d in range(5))
    # the kernel's eight accumulators: d = 8 folded into d = 7 (B slices scaled by 2^-7), summed in FP32
    acc7 = (acc[7].astype(np.float64) + acc[8].astype(np.float64) / 128.0).astype(np.float32)
    small = np.zeros((n, n), dtype=np.float32)
    for a in (acc7, acc[6].astype(np.float32), acc[5].astype(np.float32)):
        small = ((small + a) * np.float32(2.0 ** -7)).astype(np.float32)
    t = I.astype(np.float64) + small.astype(np.float64)
    scale = np.ldexp(1.0, (ex[:, None] + ex[None, :] - 40).astype(np.int64))
    return t * scale, ex, bound


def _exact_dot(a, b):
    """sum_k a_k b_k exactly (Python integers over a common power of two), returned as (num, exp2)."""
    terms = []
    for x, y in zip(a, b):
        if x == 0 or y == 0:
            continue
        mx, ex_ = math.frexp(float(x))
        my, ey = math.frexp(float(y))
        terms.append((int(mx * (1 << 53)) * int(my * (1 << 53)), ex_ + ey - 106))
    if not terms:
        return 0, 0
    e0 = min(e for _, e in terms)
    return sum(v << (e - e0) for v, e in terms), e0


@pytest.mark.parametrize("seed", [0, 1])
def test_slicing_exact_bound_and_error(seed):
    rng = np.random.default_rng([seed, 41])
    n = 24
    # entries spread over 2^-12 .. 1 of a per-row scale, random signs, some exact zeros
    scale = 2.0 ** rng.integers(-30, 30, size=n)
    A = rng.choice([-1.0, 1.0], size=(n, K)) * 2.0 ** rng.uniform(-12, 0, size=(n, K)) * scale[:, None]
    A[rng.random((n, K)) < 0.05] = 0.0
    C, ex, bound = _model(A)
    # exactness of the FP32 accumulators for d <= 6: (d + 1) K 127^2 < 2^24
    for d in range(7):
        assert bound[d] <= (d + 1) * K * 127 * 127 < 2 ** 24, (d, bound[d])
    worst = 0.0
    for i in range(n):
        for j in range(n):
            num, e0 = _exact_dot(A[i], A[j])
            exact = math.ldexp(num, e0) if num else 0.0  # correctly rounded to FP64 is enough for the bound
            err = abs(C[i, j] - exact)
            tol = K * math.ldexp(1.0, int(ex[i] + ex[j] - 50))  # K 2^-52 sigma_i sigma_j
            assert err <= tol, (i, j, err, tol)
            worst = max(worst, err / tol)
    print(f"slicing model: worst error {worst:.3f} of the bound")


def test_slicing_reconstructs_entries():
    """The 9 slices give every entry to 2^(e_i - 62): exact for entries within 2^9 of the row's largest."""
    rng = np.random.default_rng([7, 41])
    A = rng.standard_normal((8, K)) * 2.0 ** rng.integers(-20, 20, size=(8, 1))
    ex, sl = _slices(A)
    for i in range(8):
        for k in range(K):
            rec = sum(int(sl[p, i, k]) * 2.0 ** (56 - 7 * p) for p in range(S)) * 2.0 ** (int(ex[i]) - 62)
            x = A[i, k]
            assert abs(rec - x) <= 2.0 ** (int(ex[i]) - 62) + 2.0 ** -53 * abs(x)
            if abs(x) >= 2.0 ** (int(ex[i]) - 9):
                assert rec == x
