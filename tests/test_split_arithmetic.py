"""Bit-level claims behind the FP16 split path, checked on the CPU with NumPy
restatements of the integer conversions (FP64 -> FP32 truncated and rounded
heads, FP32 -> FP64 widening with an exponent rebase, the FP16 scale exponent
from FP32 bits).  Each is compared with NumPy's own IEEE operations; the
field pass's per-group scaling is checked to fit FP16 and keep 22 bits, and
scaled flushes to sum like unscaled ones."""
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


def group_exp(m):
    """The field pass's exponent of a group whose largest |head| is m (FP32):
    m 2^e in [2^14, 2^15), kept within [-126, 126]."""
    return np.clip(15 - fp16_exp_from_bits(np.atleast_1d(np.float32(m)))[0], -126, 126)


def fp16_slices(hi, lo, e):
    """Two FP16 slices of (hi + lo) 2^e as the field pass forms them."""
    f = np.float32(2.0 ** e)
    a, b = (hi * f).astype(np.float32), (lo * f).astype(np.float32)
    s0 = a.astype(np.float16)
    s1 = ((a - s0.astype(np.float32)) + b).astype(np.float16)
    return s0, s1


@pytest.mark.parametrize("kind", ["random", "cancel", "wide"])
def test_group_exponent_fits_fp16_and_keeps_22_bits(kind):
    """Per 128-cell group: sigma+- from the FP32-rounded values by TwoSum,
    scaled by 2^e from the group's largest head, split into two FP16 slices:
    no slice overflows and the slices hold sigma to 2^-22 of the group max."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        x0 = _doubles(rng, 128, -3, 3)
        if kind == "random":
            x1 = _doubles(rng, 128, -3, 3)
        elif kind == "cancel":  # rho_Yang within a few ulp of rho_Yin: sigma- cancels
            x1 = x0 * (1.0 + rng.integers(-8, 9, 128) * 2.0 ** -52)
        else:  # one group spanning many decades
            x1 = _doubles(rng, 128, -20, 20)
        h0, h1 = round_head(x0), round_head(x1)
        for sgn in (1.0, -1.0):
            hi = (h0 + np.float32(sgn) * h1).astype(np.float32)  # TwoSum head
            lo = ((h0.astype(np.float64) + sgn * h1.astype(np.float64)) - hi.astype(np.float64)).astype(np.float32)
            m = np.max(np.abs(hi))
            if m == 0:
                continue
            e = int(group_exp(np.float32(m)))
            assert 2.0 ** 14 <= m * 2.0 ** e < 2.0 ** 15
            s0, s1 = fp16_slices(hi, lo, e)
            assert np.all(np.isfinite(s0)) and np.all(np.abs(s0.astype(np.float64)) <= 2.0 ** 15)
            back = (s0.astype(np.float64) + s1.astype(np.float64)) * 2.0 ** -e
            sig = h0.astype(np.float64) + sgn * h1.astype(np.float64)
            assert np.max(np.abs(back - sig)) <= 2.0 ** -22 * m * 1.01


def test_scaled_flushes_sum_like_unscaled():
    """A float-float running sum of accumulator flushes, each in its own
    group's units 2^e and brought back by the exact factor 2^-e before
    FastTwoSum, carries the same error as flushes that were never scaled."""
    rng = np.random.default_rng(7)
    f32 = np.float32

    def ff_sum(vals, scales):
        H = np.zeros(vals.shape[1], np.float32)
        L = np.zeros_like(H)
        for v, sc in zip(vals, scales):
            b = (v * f32(sc)).astype(np.float32)  # exact: a power of two
            s = (H + b).astype(np.float32)
            e = (b - (s - H)).astype(np.float32)
            H, L = s, (L + e).astype(np.float32)
        return H.astype(np.float64) + L.astype(np.float64)

    # same-sign flushes of one order of magnitude: FastTwoSum is exact once
    # the running sum dominates, and within one rounding of a flush before
    true = rng.uniform(0.5, 2.0, (60, 4096)).astype(np.float32).astype(np.float64)
    exps = rng.integers(-40, 40, 60)
    scaled = (true * 2.0 ** exps[:, None]).astype(np.float32)  # exact scaling of FP32 values
    got = ff_sum(scaled, 2.0 ** -exps.astype(np.float64))
    ref = ff_sum(true.astype(np.float32), np.ones(60))
    assert np.array_equal(got, ref)
    exact = true.sum(axis=0)
    assert np.all(np.abs(got - exact) <= 2.0 ** -23 * true.max(axis=0))
    assert np.median(np.abs(got - exact) / exact) < 2.0 ** -40


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
