"""omega_p (Section 2.2, item 3): the pressure (density) update relaxed with
omega_p, the momentum with omega. Pins of the oracle's nu_p path: the exact
linear (acoustic) amplification matrix derived from Eq. ACM2.0 by hand, exact
conservation, the nu_p = nu identity, and the effect the paper states (larger nu_p
improves the divergence-free condition)."""
import numpy as np
import pytest

import oracle
from paper_1111_2142_gb300 import inputs


def test_nu_p_equal_nu_is_the_plain_scheme():
    f = inputs.smooth_random((11, 13), seed=2, u_amp=0.05, d_amp=0.01)
    a = oracle.step(9, *f, nu=0.03, nsteps=7)
    b = oracle.step_nu_p(9, *f, nu=0.03, nu_p=0.03, nsteps=7)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("Q,shape", [(9, (12, 17)), (19, (5, 6, 7))])
def test_nu_p_conserves_mass_and_momentum(Q, shape):
    f = inputs.smooth_random(shape, seed=3, u_amp=0.05, d_amp=0.02)
    out = oracle.step_nu_p(Q, *f, nu=0.01, nu_p=0.15, nsteps=5)
    r0, r1 = 1.0 + f[0], 1.0 + out[0]
    assert abs(out[0].sum() - f[0].sum()) < 1e-13 * f[0].size
    for u0, u1 in zip(f[1:], out[1:]):
        assert abs((r1 * u1).sum() - (r0 * u0).sum()) < 1e-13 * f[0].size


def test_linear_acoustic_mode_matches_closed_form():
    """A small density wave rho = 1 + eps cos(k x) at rest on D2Q9, linearised:
    (rho^, j^)+ = M (rho^, j^) with
      M = [[2/3 + cos(k)/3, -i (1 - a_p) sin k], [-(i/3) sin k, (1 - a) cos k + a]],
    a = 1 - 6 nu, a_p = 1 - 6 nu_p (sums of w_i c_i^n exp(-i k c_ix) over D2Q9).
    The nonlinear oracle agrees to O(eps^2)."""
    nx, eps, nu, nu_p, n = 16, 1e-7, 0.03, 0.12, 6
    k = 2 * np.pi / nx
    a, ap = 1 - 6 * nu, 1 - 6 * nu_p
    M = np.array([[2 / 3 + np.cos(k) / 3, -1j * (1 - ap) * np.sin(k)],
                  [-1j / 3 * np.sin(k), (1 - a) * np.cos(k) + a]])
    v = np.linalg.matrix_power(M, n) @ np.array([eps, 0.0])
    x = np.arange(nx)
    d0 = (eps * np.cos(k * x))[None, :].repeat(3, 0)
    z = np.zeros_like(d0)
    d, ux, uy = oracle.step_nu_p(9, d0, z, z, nu=nu, nu_p=nu_p, nsteps=n)
    pred_d = np.real(v[0] * np.exp(1j * k * x))
    pred_j = np.real(v[1] * np.exp(1j * k * x))
    assert np.max(np.abs(d[0] - pred_d)) < 1e-6 * eps
    assert np.max(np.abs((1 + d[0]) * ux[0] - pred_j)) < 1e-6 * eps
    assert np.max(np.abs(uy)) < 1e-9 * eps  # zero up to FP64 rounding of the sums
    # the same with a_p = a would differ: the pin sees which a enters which sum
    v_same = np.linalg.matrix_power(np.array([[M[0, 0], -1j * (1 - a) * np.sin(k)], [M[1, 0], M[1, 1]]]), n) @ \
        np.array([eps, 0.0])
    assert np.max(np.abs(np.real(v_same[0] * np.exp(1j * k * x)) - pred_d)) > 1e-3 * eps


def test_larger_nu_p_reduces_the_divergence_error():
    """Section 2.2 item 3 / Section 3.2 (Minion & Brown): nu_p > nu weakens the
    pseudo-compressibility term (proportional to eps^2 / nu_p), so the velocity
    field of the forced Taylor-Green vortex is closer to divergence-free."""
    n = 32
    eps = 2 * np.pi / n
    divs = []
    for nu_p in (0.1, 0.13, 1 / 6):
        d, ux, uy = inputs.gtg_state(n, 0.0)
        for s in range(inputs.gtg_steps(n) // 4):
            g = inputs.gtg_force(n, s * eps ** 2)
            d, ux, uy = oracle.step_nu_p(9, d, ux, uy, nu=inputs.GTG_NU, nu_p=nu_p, g=g)
        div = (np.roll(ux, -1, 1) - np.roll(ux, 1, 1) + np.roll(uy, -1, 0) - np.roll(uy, 1, 0)) / (2 * eps ** 2)
        divs.append(float(np.mean(np.abs(div))))
    assert divs[0] > divs[1] > divs[2], divs

