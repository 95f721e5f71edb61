"""Pins of the bulk-viscosity variant (Appendix "Computing derivatives locally",
Eq. quasi-equilibrium2) in the FP64 oracle, D2Q9, periodic.

Reading (also in the oracle's header): the equilibrium is
f^(e*) = f^(e) + f^(qe)(Tr*) - f^(qe)(Tr^(e)), Tr* = Tr^(e) + gamma (Tr^(+) - Tr^(e)),
with f^(qe) the product-form quasi-equilibrium (Eqs. d2q9_equilibrium_gen,
quasi-equilibrium), Tr^(e) = 2/3 + |u|^2 and Tr^(+) the trace of sum_i c_i c_i f_i of
the node's last update over its density, carried from step to step.

What pins it:
  * gamma = 0 is the standard scheme, to rounding;
  * Eq. second-quasi-equilibrium2 (exact): the second moment of f^(e*) is
    Pi^(e) + rho gamma/2 (Tr^(+) - Tr^(e)) I, mass and momentum unchanged;
  * Eq. trAA3: one update from equilibrium changes the unnormalised trace by
    -8 nu div(rho u) while the density changes by -6 nu div(rho u), so the stored
    Tr^(+) (over the updated density) moves by -4 nu div(rho u);
  * hence Tr^(+) - Tr^(e) follows dTr <- gamma dTr - 4 nu div(rho u) and the
    modified stress is -2 nu gamma/(1 - gamma) div u I: a linear longitudinal wave
    of wave number k is damped by an extra nu gamma k^2 / (1 - gamma) per step
    (bulk viscosity raised by 2 rho0 nu gamma/(1 - gamma); the paper's leading-order
    count, which takes the -8 nu of the unnormalised trace and no feedback, gives
    4 rho0 nu gamma), and a shear wave, whose divergence is zero, is unchanged."""
import numpy as np
import pytest

import oracle
from paper_1111_2142_gb300 import inputs


def test_gamma_zero_is_the_standard_step():
    f = inputs.smooth_random((24, 20), seed=3)
    a = oracle.step(9, *f, nu=0.02, nsteps=20)
    b = oracle.step_bulk(*f, nu=0.02, gamma=0.0, nsteps=20)
    assert max(float(np.max(np.abs(x - y))) for x, y in zip(a, b[:3])) < 1e-14
    c = oracle.step_bulk(*f, nu=0.02, gamma=0.4, nsteps=20)
    assert max(float(np.max(np.abs(x - y))) for x, y in zip(a, c[:3])) > 1e-5  # gamma acts


def test_with_omega_p_reduces_to_each_variant():
    """Both improvements of Section 3.2 together (omega_p for the density, the
    modified equilibrium everywhere): gamma = 0 is the omega_p step and nu_p = nu
    the bulk-viscosity step, to rounding; with both on, the result differs from each."""
    f = inputs.smooth_random((24, 20), seed=3)
    a = oracle.step_nu_p(9, *f, nu=0.02, nu_p=0.1, nsteps=20)
    b = oracle.step_bulk(*f, nu=0.02, nu_p=0.1, gamma=0.0, nsteps=20)
    assert max(float(np.max(np.abs(x - y))) for x, y in zip(a, b[:3])) < 1e-14
    c = oracle.step_bulk(*f, nu=0.02, gamma=0.4, nsteps=20)
    e = oracle.step_bulk(*f, nu=0.02, nu_p=0.02, gamma=0.4, nsteps=20)
    assert max(float(np.max(np.abs(x - y))) for x, y in zip(c, e)) < 1e-14
    g = oracle.step_bulk(*f, nu=0.02, nu_p=0.1, gamma=0.4, nsteps=20)
    assert max(float(np.max(np.abs(x - y))) for x, y in zip(c[:3], g[:3])) > 1e-4
    assert max(float(np.max(np.abs(x - y))) for x, y in zip(a, g[:3])) > 1e-5


def test_second_moment_of_the_modified_equilibrium():
    c = oracle.lattice(9)[0][:, :2].astype(float)
    rng = np.random.default_rng(0)
    for _ in range(100):
        rho = 1.0 + 0.05 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(2)
        trp = 2.0 / 3.0 + 0.02 * rng.standard_normal()
        g = rng.uniform(-0.9, 0.9)
        f = oracle.feq_star(rho, u, trp, g)
        tre = 2.0 / 3.0 + u @ u
        pi = np.einsum("i,ia,ib->ab", f, c, c)
        expect = rho * (np.outer(u, u) + np.eye(2) / 3.0) + rho * 0.5 * g * (trp - tre) * np.eye(2)
        assert np.max(np.abs(pi - expect)) < 1e-15
        assert abs(f.sum() - rho) < 1e-15 and np.max(np.abs(f @ c - rho * u)) < 1e-15
        # at Tr^(+) = Tr^(e) it is f^(e) itself
        fe, _ = oracle.equilibria(9, rho, [u[0], u[1], 0.0])
        assert np.max(np.abs(oracle.feq_star(rho, u, tre, g) - fe)) < 1e-15


def test_quasi_equilibrium_at_tr_e_is_feq_to_third_order():
    """Appendix "Equilibrium distribution functions": the product form at
    Pxx = 1/3 + u^2, Pyy = 1/3 + v^2 (Eq. quasi-equilibrium at Tr = Tr^(e)) is f^(e)
    when third-order terms are neglected: its moments up to the second equal f^(e)'s
    exactly, and the difference shrinks as |u|^3."""
    c = oracle.lattice(9)[0][:, :2].astype(float)
    rng = np.random.default_rng(5)
    direction = rng.standard_normal(2)
    diffs = []
    for amp in (0.04, 0.02, 0.01):
        u = amp * direction
        rho = 1.02
        f = oracle.fqe(rho, u, 2.0 / 3.0 + u @ u)
        fe, _ = oracle.equilibria(9, rho, [u[0], u[1], 0.0])
        assert abs(f.sum() - rho) < 1e-15
        assert np.max(np.abs(f @ c - rho * u)) < 1e-15
        pi = np.einsum("i,ia,ib->ab", f, c, c)
        assert np.max(np.abs(pi - rho * (np.outer(u, u) + np.eye(2) / 3.0))) < 1e-15
        diffs.append(float(np.max(np.abs(f - fe))))
    assert diffs[0] > 1e-8  # not f^(e) itself
    for a, b in zip(diffs, diffs[1:]):
        assert a / b == pytest.approx(8.0, rel=0.05)


def _smooth_divergent(n, amp, k):
    x = np.arange(n)
    X, Y = np.meshgrid(x, x)
    ux = amp * np.sin(k * X) * np.cos(2 * k * Y)
    uy = 0.5 * amp * np.cos(k * X) * np.sin(k * Y)
    d = 0.3 * amp * np.cos(k * X + k * Y)
    return d, ux, uy


@pytest.mark.parametrize("nu", [0.02, 0.05])
def test_trace_after_one_update(nu):
    """Eq. trAA3 on the unnormalised trace, and the stored (normalised) trace."""
    n = 128
    k = 2 * np.pi / n
    d, ux, uy = _smooth_divergent(n, 1e-4, k)
    out = oracle.step_bulk(d, ux, uy, None, nu=nu, gamma=0.7, nsteps=1)
    rho = 1.0 + d
    jx, jy = rho * ux, rho * uy
    div = 0.5 * (np.roll(jx, -1, 1) - np.roll(jx, 1, 1) + np.roll(jy, -1, 0) - np.roll(jy, 1, 0))
    scale = np.max(np.abs(div)) * nu
    unnorm = out[3] * (1.0 + out[0]) - rho * (2.0 / 3.0 + ux ** 2 + uy ** 2)
    assert np.max(np.abs(unnorm + 8 * nu * div)) < 0.05 * 8 * scale
    assert np.max(np.abs(out[0] - d + 6 * nu * div)) < 0.05 * 6 * scale
    assert np.max(np.abs(out[3] - (2.0 / 3.0 + ux ** 2 + uy ** 2) + 4 * nu * div)) < 0.05 * 4 * scale


def _mode_matrix(n, nu, gamma, delta=1e-7):
    """One-step linear map of the Fourier mode k = 2 pi / n of (d, ux, Tr) about rest."""
    x = np.arange(n)
    k = 2 * np.pi / n
    e = np.exp(-1j * k * x)
    M = np.zeros((3, 3), complex)
    for j in range(3):
        fields = [np.zeros((1, n)), np.zeros((1, n)), np.full((1, n), 2.0 / 3.0)]
        fields[j][0] += delta * np.cos(k * x)
        out = oracle.step_bulk(fields[0], fields[1], np.zeros((1, n)), fields[2], nu=nu, gamma=gamma, nsteps=1)
        resp = [out[0][0], out[1][0], out[3][0] - 2.0 / 3.0]
        M[:, j] = [2.0 * np.mean(r * e) / delta for r in resp]
    return M, k


def _acoustic_damping(M):
    lam = [l for l in np.linalg.eigvals(M) if abs(l.imag) > 1e-9]
    return -np.log(abs(lam[0]))


@pytest.mark.parametrize("nu", [0.01, 0.05])
def test_longitudinal_damping_closed_form(nu):
    n = 256
    M0, k = _mode_matrix(n, nu, 0.0)
    r0 = _acoustic_damping(M0)
    for g in (0.2, 0.4, 0.6):
        M, _ = _mode_matrix(n, nu, g)
        excess = _acoustic_damping(M) - r0
        assert excess == pytest.approx(nu * g * k * k / (1.0 - g), rel=2e-3)


def test_shear_wave_unchanged():
    n = 64
    x = np.arange(n)
    k = 2 * np.pi / n
    v0 = 1e-7 * np.sin(k * x)[None, :]
    rates = []
    for g in (0.0, 0.4):
        out = oracle.step_bulk(np.zeros((1, n)), np.zeros((1, n)), v0, None, nu=0.02, gamma=g, nsteps=50)
        rates.append(-np.log(np.sum(out[2][0] * np.sin(k * x)) / np.sum(v0[0] * np.sin(k * x))) / 50)
    assert rates[1] == pytest.approx(rates[0], rel=1e-7)
    assert rates[0] == pytest.approx(0.02 * k * k, rel=2e-3)  # nu k^2 of the shear wave


def test_increment_regrouped_per_link_pair():
    """The increment f^(e*) - f^(e) of the oracle, split per link pair (c, -c) into
    its even and odd parts, has closed forms (the 2D-tile kernel builds them this
    way), with h = gamma (Tr^(+) - Tr^(e)) / 2 and P = Pxx + Pyy = 2/3 + |u|^2:
      axis:     even rho h (1 - P - h) / 2,  odd -rho h (c.u) / 2
      diagonal: even rho h (h + P) / 4,      odd  rho h (c.u) / 4
      rest:     rho h (h - 2 + P)
    (the product form of Eq. d2q9_equilibrium_gen moved from Pxx, Pyy to Pxx + h,
    Pyy + h, Eq. quasi-equilibrium). A slip in the kernel's regrouping is a slip in
    one of these lines."""
    c = oracle.lattice(9)[0][:, :2].astype(int)
    opp = [int(np.flatnonzero((c == -ci).all(axis=1))[0]) for ci in c]
    rng = np.random.default_rng(8)
    for _ in range(200):
        rho = 1.0 + 0.05 * rng.standard_normal()
        u = 0.08 * rng.standard_normal(2)
        tre = 2.0 / 3.0 + u @ u
        trp = tre + 0.05 * rng.standard_normal()
        g = rng.uniform(-0.9, 0.9)
        fe, _ = oracle.equilibria(9, rho, [u[0], u[1], 0.0])
        df = oracle.feq_star(rho, u, trp, g) - fe
        h = 0.5 * g * (trp - tre)
        P = 2.0 / 3.0 + u @ u
        for i, ci in enumerate(c):
            n2 = int(ci @ ci)
            if n2 == 0:
                assert abs(df[i] - rho * h * (h - 2.0 + P)) < 1e-15
                continue
            even, odd = 0.5 * (df[i] + df[opp[i]]), 0.5 * (df[i] - df[opp[i]])
            e = float(ci @ u)
            if n2 == 1:
                assert abs(even - 0.5 * rho * h * (1.0 - P - h)) < 1e-15
                assert abs(odd + 0.5 * rho * h * e) < 1e-15
            else:
                assert abs(even - 0.25 * rho * h * (h + P)) < 1e-15
                assert abs(odd - 0.25 * rho * h * e) < 1e-15
