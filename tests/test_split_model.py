"""The per-product rounding model behind the mixed-precision parity bars
(tests/bounds.py), checked by emulating the operand splits bit for bit on the
host: bf16 and TF32 rounding to nearest even from FP32 bit patterns, the
split x = hi + lo with hi = bf16(x), lo = bf16(x - hi) as the kernels form it,
and the three-product sum hi*hi' + hi*lo' + lo*hi' the tensor cores add up
(each product of two bf16 values and the exact FP32 product x*y are
representable in FP64).  The bars may only rely on bounds that hold here."""
import numpy as np

from bounds import SPLIT_OPERAND, U_TF32


def _round_bits(x32, drop):
    """Round FP32 values to nearest even, keeping 23 - drop explicit mantissa bits."""
    b = x32.view(np.uint32).astype(np.uint64)
    lsb = (b >> drop) & 1
    b = (b + (1 << (drop - 1)) - 1 + lsb) & ~np.uint64((1 << drop) - 1)
    return b.astype(np.uint32).view(np.float32)


def bf16(x32):
    return _round_bits(x32, 16)


def tf32(x32):
    return _round_bits(x32, 13)


def _operands(n, seed):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    return (mant * 2.0 ** rng.integers(-30, 30, n)).astype(np.float32)


def test_bf16_and_tf32_rounding_emulation():
    # exact cases: halfway values round to even, representable values stay
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7], dtype=np.float32)
    assert bf16(x).tolist() == [1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7]
    y = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11], dtype=np.float32)
    assert tf32(y).tolist() == [1.0, 1.0 + 2.0 ** -9]


def test_split_product_bound():
    x, y = _operands(200000, 1), _operands(200000, 2)
    hx, hy = bf16(x), bf16(y)
    lx, ly = bf16((x - hx).astype(np.float32)), bf16((y - hy).astype(np.float32))
    # the FP32 differences x - hi are exact (hi is x rounded at bit 16)
    assert np.all((x.astype(np.float64) - hx) == (x - hx).astype(np.float64))
    exact = x.astype(np.float64) * y.astype(np.float64)
    hxd, hyd, lxd, lyd = (a.astype(np.float64) for a in (hx, hy, lx, ly))
    approx = hxd * hyd + hxd * lyd + lxd * hyd
    rel = np.abs(exact - approx) / np.abs(exact)
    assert rel.max() <= SPLIT_OPERAND, rel.max()
    # the operand split itself: |x - hi - lo| <= 2^-16 |x|
    ex = np.abs(x.astype(np.float64) - hxd - lxd) / np.abs(x.astype(np.float64))
    assert ex.max() <= 2.0 ** -16
    # and the model is not vacuous: the dropped terms do reach the 2^-18 scale
    assert rel.max() >= 2.0 ** -19


def test_tf32_operand_bound():
    x = _operands(200000, 3)
    rel = np.abs(x.astype(np.float64) - tf32(x)) / np.abs(x.astype(np.float64))
    assert rel.max() <= U_TF32
    assert rel.max() >= U_TF32 / 2
