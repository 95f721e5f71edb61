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
