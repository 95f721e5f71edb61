"""Numerical building blocks of the kernels, on the GPU."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def quotient():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_1111_2142_gb300 import lwacm as lw
    lib = lw.load()

    def run(a, b, packed):
        ad = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
        bd = torch.from_numpy(np.ascontiguousarray(b, dtype=np.float32)).cuda()
        out = torch.empty_like(ad)
        st = torch.cuda.current_stream()
        assert lib.lwacm_selftest_quotient(ctypes.c_void_p(ad.data_ptr()), ctypes.c_void_p(bd.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), a.size, int(packed),
                                           ctypes.c_void_p(st.cuda_stream)) == lw.OK
        return out.cpu().numpy()
    return run


def _f32_range(lo, hi):
    """Every FP32 value in [lo, hi) (lo, hi positive powers of two)."""
    b0 = int(np.float32(lo).view(np.uint32))
    b1 = int(np.float32(hi).view(np.uint32))
    return np.arange(b0, b1, dtype=np.uint32).view(np.float32)


def _mismatches(got, a, b):
    """Elements where the kernel's quotient differs, bit for bit, from the host's
    IEEE round-to-nearest FP32 division. A zero numerator gives +0 where IEEE
    division gives a zero with the quotient's sign: the residual a - b q of a zero
    quotient is +0 in round-to-nearest, so the correction returns +0; the two zeros
    compare equal, and a velocity's sign of zero changes no later value."""
    ref = np.divide(a.astype(np.float32), b.astype(np.float32), dtype=np.float32)
    differ = got.view(np.uint32) != ref.view(np.uint32)
    return np.flatnonzero(differ & ~((got == 0) & (ref == 0)))


def test_reciprocal_every_divisor_in_half_to_two(quotient):
    """The quotient divides with RN(1/b), the correctly rounded reciprocal (Markstein's
    correction needs it): for every FP32 b in [1/2, 2) (2^24 values, among them the
    all-ones significands 1 - 2^-24 and 2 - 2^-23 that the Newton step rounds low)
    and for powers of two times them up to 2^+-60, the kernel's reciprocal equals the
    host's IEEE 1/b bit for bit."""
    b = _f32_range(0.5, 2.0)
    for scale in (1.0, 2.0 ** 60, 2.0 ** -60):
        bs = (b * np.float32(scale)).astype(np.float32)
        got = quotient(np.ones_like(bs), bs, 2)
        ref = np.divide(np.float32(1.0), bs, dtype=np.float32)
        bad = np.flatnonzero(got.view(np.uint32) != ref.view(np.uint32))
        assert bad.size == 0, (scale, bs[bad[:5]], got[bad[:5]], ref[bad[:5]])


@pytest.mark.parametrize("packed", [1, 0])
def test_quotient_every_divisor_in_half_to_two(quotient, packed):
    """The kernels form u = j / rho (step a5). For every FP32 divisor in [1/2, 2)
    (all 2^24 of them; the density of the method stays in this range) and numerators
    of either sign drawn log-uniformly over [1e-6, 1] (twice, two draws per divisor),
    the quotient equals the IEEE round-to-nearest FP32 quotient bit for bit. Scaling
    a divisor by a power of two scales the reciprocal exactly, so the binade [1/2, 2)
    covers the relative behaviour of every normal divisor."""
    b = _f32_range(0.5, 2.0)
    rng = np.random.default_rng(11)
    for rep in range(2):
        a = (np.exp(rng.uniform(np.log(1e-6), 0.0, b.size)) * rng.choice([-1.0, 1.0], b.size)).astype(np.float32)
        bad = _mismatches(quotient(a, b, packed), a, b)
        assert bad.size == 0, (rep, a[bad[:5]], b[bad[:5]])


@pytest.mark.parametrize("packed", [1, 0])
def test_quotient_hard_divisors_every_numerator(quotient, packed):
    """Divisors whose significand is all ones (1 - 2^-24, 2 - 2^-23) or all zeros (1),
    or one ulp from 1, where the reciprocal sits next to a rounding boundary, each
    against every FP32 numerator in [1, 2) (2^23 values) and every power of two
    from 2^-40 to 2^10."""
    num = np.concatenate([_f32_range(1.0, 2.0), np.float32(2.0) ** np.arange(-40, 11, dtype=np.float32)])
    for bv in (1 - 2.0 ** -24, 2 - 2.0 ** -23, 1.0, 1 + 2.0 ** -23, 0.5 + 2.0 ** -24, 1.5, 0.75):
        b = np.full(num.size, bv, dtype=np.float32)
        bad = _mismatches(quotient(num, b, packed), num, b)
        assert bad.size == 0, (bv, num[bad[:5]])


def test_quotient_wide_range(quotient):
    """Random numerators log-uniform over [1e-25, 1e25] and divisors over
    [1e-12, 1e12], both signs (every quotient normal, every numerator above
    2^-100); zero numerators give zero."""
    rng = np.random.default_rng(12)
    n = 1 << 22
    a = (np.exp(rng.uniform(np.log(1e-25), np.log(1e25), n)) * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    b = (np.exp(rng.uniform(np.log(1e-12), np.log(1e12), n)) * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    a[:4] = [0.0, -0.0, 0.0, -0.0]
    b[:4] = [1.0, 1.0, -2.0, 3.0]
    for packed in (1, 0):
        bad = _mismatches(quotient(a, b, packed), a, b)
        assert bad.size == 0, (packed, a[bad[:5]], b[bad[:5]])


# ---- stochastic rounding of BF16 / FP16 stores ---------------------------------

def _neighbours(x, storage):
    """The storage values lo (x rounded toward zero) and hi (the next one away from
    zero) around each FP32 value x, as FP64."""
    x = np.asarray(x, dtype=np.float32)
    if storage == 1:  # bfloat16: the upper 16 bits of an FP32
        b = x.view(np.uint32)
        lo = (b & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
        hi = ((b & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32).astype(np.float64)
        return lo, hi
    h = x.astype(np.float16)  # to nearest, then step toward zero where it overshot
    over = np.abs(h.astype(np.float64)) > np.abs(x.astype(np.float64))
    h = np.where(over, np.nextafter(h, np.float16(0)), h)
    away = np.where(np.signbit(x), np.float16(-np.inf), np.float16(np.inf))
    return h.astype(np.float64), np.nextafter(h, away).astype(np.float64)


@pytest.fixture(scope="module")
def rounding():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_1111_2142_gb300 import lwacm as lw
    lib = lw.load()

    def run(x, storage, step):
        xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
        out = torch.empty_like(xd)
        st = torch.cuda.current_stream()
        assert lib.lwacm_selftest_round(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(out.data_ptr()), x.size,
                                        int(storage), int(step), ctypes.c_void_p(st.cuda_stream)) == lw.OK
        return out.cpu().numpy().astype(np.float64)
    return run


@pytest.mark.parametrize("storage", [1, 2])
def test_stochastic_rounding_is_unbiased(rounding, storage):
    """Each stored value is one of the two storage values around x, never another;
    exact values stay; over S step keys the fraction rounded away from zero matches
    (x - lo) / (hi - lo) for every x (binomial bound, 6 sigma plus the 2^-16
    resolution of the random bits), and the mean of the rounding error over all
    values and keys is zero within its standard error (round to nearest would be
    biased by the full per-value distance to the nearer neighbour)."""
    rng = np.random.default_rng(31)
    n, S = 6000, 256
    mag = 10.0 ** rng.uniform(-7 if storage == 2 else -20, 0, n)
    x = (mag * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    x[:64] = np.float32(0.0)
    lo, hi = _neighbours(x, storage)
    x[64:128] = lo[64:128].astype(np.float32)  # exactly representable values
    lo, hi = _neighbours(x, storage)
    xd = x.astype(np.float64)
    up = np.zeros(n)
    err = np.zeros(n)
    for s in range(S):
        got = rounding(x, storage, s)
        is_lo, is_hi = got == lo, got == hi
        assert np.all(is_lo | is_hi), np.flatnonzero(~(is_lo | is_hi))[:5]
        up += is_hi & ~is_lo
        err += got - xd
    frac = np.where(hi != lo, (xd - lo) / (hi - lo), 0.0)
    obs = up / S
    sig = np.sqrt(frac * (1 - frac) / S)
    assert np.all(obs[64:128] == 0) and np.all(obs[:64] == 0)
    assert np.all(np.abs(obs - frac) <= 6 * sig + 2.0 ** -16 + 1e-12), float(np.max(np.abs(obs - frac) - 6 * sig))
    # mean rounding error in units of each value's spacing: zero within 5 standard errors
    spacing = np.where(hi != lo, np.abs(hi - lo), 1.0)
    e = (err / S) / spacing
    se = np.sqrt(np.sum(frac * (1 - frac) / S)) / n
    assert abs(float(np.mean(e))) <= 5 * se + 2.0 ** -16, (float(np.mean(e)), se)
