"""Bit-level claims behind the FP16 split path, checked on the CPU with NumPy
restatements of the integer conversions (FP64 -> FP32 truncated and rounded
heads, FP32 -> FP64 widening with an exponent rebase, the FP16 scale exponent
from FP32 bits).  Each is compared with NumPy's own IEEE operations, and the
field pass's pass-1 bound is checked to cover the values pass 2 forms."""
import numpy as np
import pytest

U64, U32 = np.uint64, np.uint32


def _split_words(x):
    b = np.asarray(x, np.float64).view(U64)
    return (b >> U64(32)) & U64(0xFFFFFFFF), b & U64(0xFFFFFFFF)


def _finish(hw, E, m):
    m = np.where(E < 897, U64(0), np.where(E > 1150, U64(0x7F800000), m & U64(0xFFFFFFFF)))
    return ((hw & U64(0x80000000)) | m).astype(U32).view(np.float32)


def trunc_head(x):
    """FP64 -> FP32 keeping the top 24 significant bits (normal range only)."""
    hw, lw = _split_words(x)
    E = (hw >> U64(20)) & U64(0x7FF)
    m = ((E - U64(896)) << U64(23)) | (((hw << U64(3)) | (lw >> U64(29))) & U64(0x7FFFFF))
    return _finish(hw, E, m)


def round_head(x):
    """FP64 -> FP32 rounded to nearest, ties away (normal range only)."""
    hw, lw = _split_words(x)
    E = (hw >> U64(20)) & U64(0x7FF)
    m = (((E - U64(896)) << U64(23)) | (((hw << U64(3)) | (lw >> U64(29))) & U64(0x7FFFFF))) + ((lw >> U64(28)) & U64(1))
    return _finish(hw, E, m)


def widen_pow2(f, d):
    """FP32 f -> FP64 f * 2^d by rebasing the exponent while widening."""
    u = np.asarray(f, np.float32).view(U32).astype(U64)
    mag, sign = u & U64(0x7FFFFFFF), u & U64(0x80000000)
    c20 = U64((896 + d) << 20)
    hi = np.where(mag < 0x00800000, sign, (((mag >> U64(3)) + c20) & U64(0xFFFFFFFF)) | sign)
    lo = (u << U64(29)) & U64(0xFFFFFFFF)
    return ((hi << U64(32)) | lo).view(np.float64)


def fp16_exp_from_bits(m):
    """frexp's exponent of an FP32 m > 0 from its bits."""
    u = np.asarray(m, np.float32).view(U32).astype(np.int64)
    be = u >> 23
    mant = u & 0x7FFFFF
    clz = np.array([32 - int(v).bit_length() for v in mant])
    return np.where(be > 0, be - 126, -117 - clz)


def _doubles(rng, n, lo=-30, hi=30):
    return rng.standard_normal(n) * 10.0 ** rng.uniform(lo, hi, n)


def test_round_head_is_ieee_round_to_nearest():
    x = _doubles(np.random.default_rng(1), 200000)
    got = round_head(x).astype(np.float64)
    ref = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(got, ref)  # ties are measure-zero in random doubles
    assert np.all(np.abs(got - x) <= 2.0 ** -24 * np.abs(x))


def test_trunc_head_truncates():
    x = _doubles(np.random.default_rng(2), 200000)
    t = trunc_head(x).astype(np.float64)
    assert np.all(np.abs(t) <= np.abs(x))
    assert np.all(np.abs(x - t) < 2.0 ** -23 * np.abs(x))
    assert np.all(np.sign(t) == np.sign(x))


def test_out_of_range_flushes():
    x = np.array([1e-39, -1e-40, 0.0, -0.0, 1e39, -1e300])
    for f in (trunc_head, round_head):
        r = f(x).astype(np.float64)
        assert np.all(r[:4] == 0.0)
        assert np.all(np.isinf(r[4:])) and r[5] < 0


@pytest.mark.parametrize("kind", ["random", "cancel", "same_sign"])
def test_pass1_bound_covers_pass2_sums(kind):
    """|t0 +- t1| + 2^-22 (|t0| + |t1|), times (1 + 2^-16), bounds the rounded
    TwoSum head fl(h0 +- h1) that pass 2 scales, for every cell."""
    rng = np.random.default_rng(3)
    x0 = _doubles(rng, 100000, -5, 5)
    if kind == "random":
        x1 = _doubles(rng, 100000, -5, 5)
    elif kind == "cancel":  # rho_Yang within a few ulp of rho_Yin: sigma- cancels
        x1 = x0 * (1.0 + rng.integers(-8, 9, 100000) * 2.0 ** -52)
    else:
        x1 = np.abs(x0) * rng.uniform(0.5, 2.0, 100000) * np.sign(x0)
    t0, t1 = trunc_head(x0), trunc_head(x1)
    h0, h1 = round_head(x0), round_head(x1)
    slack = np.float32(2.0 ** -22) * (np.abs(t0) + np.abs(t1))
    for sgn in (1, -1):
        bound = (np.abs(t0 + np.float32(sgn) * t1) + slack).astype(np.float64) * (1.0 + 2.0 ** -16)
        s = (h0 + np.float32(sgn) * h1).astype(np.float64)  # fl(h0 +- h1) in FP32
        assert np.all(np.abs(s) <= bound)


def test_widening_matches_ieee_and_scales_exactly():
    rng = np.random.default_rng(4)
    f = (rng.standard_normal(100000) * 10.0 ** rng.uniform(-30, 30, 100000)).astype(np.float32)
    for d in (0, -37, 25):
        got = widen_pow2(f, d)
        assert np.array_equal(got, f.astype(np.float64) * 2.0 ** d)
    z = widen_pow2(np.array([0.0, -0.0], np.float32), -20)
    assert np.all(z == 0.0) and np.signbit(z[1])


def test_fp16_exponent_from_bits_is_frexp():
    rng = np.random.default_rng(5)
    m = np.abs(rng.standard_normal(50000) * 10.0 ** rng.uniform(-44, 38, 50000)).astype(np.float32)
    m = m[(m > 0) & np.isfinite(m)]
    _, ref = np.frexp(m.astype(np.float64))
    assert np.array_equal(fp16_exp_from_bits(m), ref)
