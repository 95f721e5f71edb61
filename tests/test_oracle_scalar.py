"""The passive scalar of Eq. ACM2.0t (thermal LW-ACM): pins of the oracle's
lwo_step_scalar against closed forms derived from the equation by hand.

With a uniform velocity u the flow is a fixed point and the scalar update is a
linear shift-invariant stencil: for T = exp(i k.x),
    T+ = lambda(k) T,  lambda(k) = a_t + sum_i w_i (1 - a_t + 3 c_i.u) exp(-i k.c_i),
a_t = 2(omega_t - 1)/omega_t = 1 - 6 alpha (the quadratic terms of g^(e) sum to
zero). At u = 0 this is pure diffusion, lambda = 1 - alpha |k|^2 + O(|k|^4)
(Eq. diffusivity2)."""
import numpy as np
import pytest

import oracle
from paper_1111_2142_gb300 import inputs


def lattice(Q):
    c, w, _ = oracle.lattice(Q)
    return np.asarray(c, dtype=float), np.asarray(w, dtype=float)


def amplification(Q, k, u, alpha):
    c, w = lattice(Q)
    at = 1.0 - 6.0 * alpha
    e = c @ np.asarray(u, dtype=float)
    return at + np.sum(w * (1.0 - at + 3.0 * e) * np.exp(-1j * (c @ np.asarray(k, dtype=float))))


@pytest.mark.parametrize("Q", [9, 19])
def test_uniform_flow_mode_matches_closed_form(Q):
    if Q == 9:
        shape, kk, u = (12, 16), (2 * np.pi * 3 / 16, 2 * np.pi * 1 / 12, 0.0), (0.07, -0.04, 0.0)
    else:
        shape, kk, u = (6, 8, 10), (2 * np.pi * 2 / 10, 2 * np.pi / 8, 2 * np.pi / 6), (0.05, 0.03, -0.06)
    alpha, n, amp = 0.02, 9, 0.1
    grids = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")  # (z,) y, x
    pos = grids[::-1]  # x, y[, z]
    phase = sum(kk[a] * pos[a] for a in range(len(pos)))
    T0 = 1.0 + amp * np.cos(phase)
    d = np.zeros(shape)
    ufields = [np.full(shape, u[a]) for a in range(2 if Q == 9 else 3)]
    out = oracle.step_scalar(Q, d, *ufields, T=T0, nu=0.03, alpha=alpha, nsteps=n)
    lam = amplification(Q, kk[: len(pos)] + (0.0,) * (3 - len(pos)), u, alpha)
    pred = 1.0 + amp * np.real(lam ** n * np.exp(1j * phase))
    assert np.max(np.abs(out[-1] - pred)) < 1e-13
    # the flow itself did not move (uniform flow is a fixed point)
    assert np.max(np.abs(out[1] - u[0])) < 1e-15


def test_pure_diffusion_is_second_order_in_k():
    """u = 0: lambda(k) against exp(-alpha |k|^2): the gap falls as |k|^4."""
    alpha = 0.05
    gaps = []
    for kx in (0.2, 0.1, 0.05):
        lam = amplification(9, (kx, 0.0, 0.0), (0, 0, 0), alpha)
        assert abs(lam.imag) < 1e-15
        gaps.append(abs(lam.real - np.exp(-alpha * kx * kx)))
    assert 14 < gaps[0] / gaps[1] < 18 and 14 < gaps[1] / gaps[2] < 18


@pytest.mark.parametrize("Q,shape", [(9, (20, 24)), (19, (6, 7, 8))])
def test_scalar_is_conserved_in_a_moving_flow(Q, shape):
    f = inputs.smooth_random(shape, seed=9, u_amp=0.05, d_amp=0.01)
    T0 = 1.0 + 0.2 * inputs.smooth_random(shape, seed=10, u_amp=0.0, d_amp=1.0)[0]
    out = oracle.step_scalar(Q, *f, T=T0, nu=0.02, alpha=0.03, nsteps=12)
    assert abs(out[-1].sum() - T0.sum()) < 1e-12 * T0.size
    # the flow part is the plain scheme
    ref = oracle.step(Q, *f, nu=0.02, nsteps=12)
    for a, b in zip(out[:-1], ref):
        assert np.array_equal(a, b)
