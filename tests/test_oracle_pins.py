"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a printed formula,
an exact identity stated in the paper, a closed-form solution, a lattice
property from the textbook definition, or a brute-force derivative.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1111_2142_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def maxdiff(a, b):
    return max(float(np.max(np.abs(np.asarray(x) - np.asarray(y)))) for x, y in zip(a, b))


# --- lattice tables -----------------------------------------------------------

@pytest.mark.parametrize("Q", [9, 19])
def test_lattice_isotropy(Q):
    """Weights and velocities satisfy the moment conditions that make the
    second-order equilibrium recover Euler/Navier-Stokes (Section 2.1: sum f^e = rho,
    sum c f^e = rho u, sum cc f^e = rho uu + p I with p = rho/3): sum w = 1,
    sum w c = 0, sum w c_a c_b = delta/3, 4th moment = (dd + dd + dd)/9."""
    c, w, bb = oracle.lattice(Q)
    D = 2 if Q == 9 else 3
    assert len({tuple(v) for v in c}) == Q
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-15)
    m2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(m2[:D, :D], np.eye(D) / 3, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)[:D, :D, :D, :D]
    I = np.eye(D)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.allclose(m4, iso, atol=1e-15)
    # odd moments vanish
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-15)
    # bounce-back: c_BB(i) = -c_i, an involution
    assert np.array_equal(c[bb], -c)
    assert np.array_equal(bb[bb], np.arange(Q))
    if Q == 19:
        # Appendix: 1 rest, 6 axis links (w 1/18), 12 face diagonals (w 1/36)
        n2 = (c * c).sum(1)
        assert sorted(n2.tolist()) == [0] + [1] * 6 + [2] * 12
        assert np.allclose(w[n2 == 1], 1 / 18) and np.allclose(w[n2 == 2], 1 / 36)


def _golden_d2q9():
    rows = []
    with open(os.path.join(GOLDEN, "d2q9_equilibria.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(Fraction(t)) for t in line.split()])
    return np.array(rows)


def test_d2q9_equilibria_match_printed_rows():
    """Eq. d2q9_equilibrium printed row by row (index order and coefficients)."""
    coef = _golden_d2q9()
    rng = np.random.default_rng(0)
    for _ in range(20):
        rho = rng.uniform(0.8, 1.2)
        u, v = rng.uniform(-0.2, 0.2, 2)
        mono = np.array([rho, rho * u, rho * v, rho * u * u, rho * v * v, rho * u * v])
        fe, fo = oracle.equilibria(9, rho, (u, v))
        assert np.allclose(fe, coef @ mono, atol=1e-15, rtol=0)
        # Eq. feqo: odd part = the terms odd in u -> the linear columns only
        assert np.allclose(fo, coef[:, 1:3] @ mono[1:3], atol=1e-15, rtol=0)


@pytest.mark.parametrize("Q", [9, 19])
def test_equilibrium_moments(Q):
    """sum f^e = rho, sum c f^e = rho u, sum cc f^e = rho uu + (rho/3) I (Section 2.1,
    p = rho/3 from the Appendix); sum f^eo = 0, sum c f^eo = rho u."""
    c, w, _ = oracle.lattice(Q)
    D = 2 if Q == 9 else 3
    rng = np.random.default_rng(1)
    for _ in range(10):
        rho = rng.uniform(0.8, 1.2)
        u = np.zeros(3)
        u[:D] = rng.uniform(-0.2, 0.2, D)
        fe, fo = oracle.equilibria(Q, rho, u)
        assert np.isclose(fe.sum(), rho, atol=1e-15)
        assert np.allclose(fe @ c, rho * u, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", fe, c, c)[:D, :D]
        assert np.allclose(P, rho * np.outer(u[:D], u[:D]) + rho / 3 * np.eye(D), atol=1e-15)
        assert np.isclose(fo.sum(), 0.0, atol=1e-15)
        assert np.allclose(fo @ c, rho * u, atol=1e-15)


# --- exact identities of the update -------------------------------------------

def test_fd_formulas_equal_linkwise_update():
    """Appendix C: Eqs. FDjx, FDjy, FDpressure equal Eq. ACM2.0 to machine precision."""
    for seed, (ny, nx), nu in [(3, (12, 14), 0.02), (4, (9, 16), 0.1), (5, (16, 16), 0.004)]:
        d, u, v = inputs.smooth_random((ny, nx), seed=seed, u_amp=0.08, d_amp=0.05)
        a = oracle.step(9, d, u, v, nu=nu, nsteps=6)
        b = oracle.fd_step_d2q9(d, u, v, nu=nu, nsteps=6)
        assert maxdiff(a, b) < 1e-14


@pytest.mark.parametrize("bc,lid", [(oracle.PERIODIC, None), (oracle.CAVITY, (0.1, 0.0, 0.0)),
                                    (oracle.CHANNEL, (0.05, 0.0, 0.0))])
def test_omega_one_is_bgk_lbm_d2q9(bc, lid):
    """omega = 1 reduces the update to equilibrium-streaming LBM (Section 2.2); with walls
    the rule becomes half-way bounce-back plus the moving-wall term of
    Eq. ACM2.0movebb (a = 0 in Eq. ACM2.0cccbb2, factor 1 in Eq. ACM2.0ccccbb)."""
    d, u, v = inputs.smooth_random((11, 13), seed=7, u_amp=0.05)
    a = oracle.step(9, d, u, v, nu=1 / 6, bc=bc, lid=lid, nsteps=12)
    b = oracle.bgk_run(9, d, u, v, omega=1.0, bc=bc, lid=lid, nsteps=12)
    assert maxdiff(a, b) < 1e-14


@pytest.mark.parametrize("bc,lid", [(oracle.PERIODIC, None),
                                    (oracle.CAVITY, (0.05, 0.03, 0.0))])
def test_omega_one_is_bgk_lbm_d3q19(bc, lid):
    d, u, v, w = inputs.smooth_random((5, 6, 7), seed=8, u_amp=0.05)
    a = oracle.step(19, d, u, v, w, nu=1 / 6, bc=bc, lid=lid, nsteps=6)
    b = oracle.bgk_run(19, d, u, v, w, omega=1.0, bc=bc, lid=lid, nsteps=6)
    assert maxdiff(a, b) < 1e-14


def test_omega_not_one_differs_from_bgk():
    """Guard: the identity above is specific to omega = 1."""
    d, u, v = inputs.smooth_random((11, 13), seed=7, u_amp=0.05)
    a = oracle.step(9, d, u, v, nu=0.05, nsteps=5)
    b = oracle.bgk_run(9, d, u, v, omega=oracle.omega_of_nu(0.05), nsteps=5)
    assert maxdiff(a, b) > 1e-6


@pytest.mark.parametrize("Q,shape", [(9, (24, 20)), (19, (6, 7, 8))])
def test_conservation_periodic(Q, shape):
    """sum rho and sum rho u are invariant on periodic grids: sum_i f^e = rho,
    sum_i c f^e = rho u and the odd-part correction telescopes (Section 2.1)."""
    f = inputs.smooth_random(shape, seed=11, u_amp=0.05, d_amp=0.02)
    d0 = oracle.diagnostics(*f)
    out = oracle.step(Q, *f, nu=0.01, nsteps=200)
    d1 = oracle.diagnostics(*out)
    N = np.prod(shape)
    assert abs(d1["mass"] - d0["mass"]) / N < 1e-13
    for k in ("jx", "jy", "jz"):
        assert abs(d1[k] - d0[k]) / N < 1e-15


@pytest.mark.parametrize("lid", [(0.0, 0.0, 0.0), (0.1, 0.0, 0.0)])
def test_cavity_conserves_mass(lid):
    """Half-way bounce-back returns every outgoing f* into the domain, so mass is
    exact with stationary walls; with the lid, the moving-wall terms of the two
    diagonal links at each lid node (including the lid corners, where the lid
    velocity is imposed, Section 2.6.1) cancel pairwise."""
    d, u, v = inputs.smooth_random((10, 12), seed=12, u_amp=0.05, d_amp=0.02)
    m0 = np.sum(1 + d)
    out = oracle.step(9, d, u, v, nu=0.02, bc=oracle.CAVITY, lid=lid, nsteps=100)
    assert abs(np.sum(1 + out[0]) - m0) < 1e-11


def test_cavity_3d_conserves_mass():
    f = inputs.smooth_random((6, 5, 7), seed=13, u_amp=0.05, d_amp=0.02)
    m0 = np.sum(1 + f[0])
    lid = (np.sqrt(2) / 20, np.sqrt(2) / 20, 0.0)
    out = oracle.step(19, *f, nu=0.03, bc=oracle.CAVITY, lid=lid, nsteps=40)
    assert abs(np.sum(1 + out[0]) - m0) < 1e-11


@pytest.mark.parametrize("Q,shape", [(9, (9, 11)), (19, (5, 6, 7))])
def test_uniform_flow_fixed_point(Q, shape):
    D = 2 if Q == 9 else 3
    U = [0.03, -0.02, 0.01][:D]
    f = [np.zeros(shape)] + [np.full(shape, ui) for ui in U]
    out = oracle.step(Q, *f, nu=0.013, nsteps=10)
    assert maxdiff(out, f) < 1e-14  # fixed point up to FP64 rounding


def test_rest_state_fixed_point_with_walls():
    f = [np.zeros((8, 9))] * 3
    out = oracle.step(9, *f, nu=0.02, bc=oracle.CAVITY, lid=(0, 0, 0), nsteps=10)
    assert maxdiff(out, f) < 1e-15  # fixed point up to FP64 rounding of d = rho - 1


# --- lattice symmetries -------------------------------------------------------

def test_equivariance_d2q9():
    """Rotating the fields by 90 degrees (and the velocity with them) commutes with
    the update, as does the reflection x -> -x; catches sign/index slips."""
    n = 12
    d, u, v = inputs.smooth_random((n, n), seed=21, u_amp=0.06)
    out = oracle.step(9, d, u, v, nu=0.02, nsteps=4)

    def rot(dd, uu, vv):  # (x,y) -> (-y, x) on a periodic square: u' = -v, v' = u
        R = lambda a: np.rot90(a, k=1, axes=(1, 0))
        return R(dd), -R(vv), R(uu)

    a = oracle.step(9, *rot(d, u, v), nu=0.02, nsteps=4)
    assert maxdiff(a, rot(*out)) < 1e-15

    def refl(dd, uu, vv):
        F = lambda a: np.roll(a[:, ::-1], 1, axis=1)  # x -> -x mod n
        return F(dd), -F(uu), F(vv)

    b = oracle.step(9, *refl(d, u, v), nu=0.02, nsteps=4)
    assert maxdiff(b, refl(*out)) < 1e-15


def test_equivariance_d3q19():
    n = 6
    f = inputs.smooth_random((n, n, n), seed=22, u_amp=0.06)
    out = oracle.step(19, *f, nu=0.02, nsteps=3)

    def cyc(d, ux, uy, uz):  # axes (z,y,x) arrays; map x->y, y->z, z->x
        T = lambda a: np.transpose(a, (1, 2, 0))
        return T(d), T(uz), T(ux), T(uy)

    a = oracle.step(19, *cyc(*f), nu=0.02, nsteps=3)
    assert maxdiff(a, cyc(*out)) < 1e-15

    def refl(d, ux, uy, uz):
        F = lambda a: np.roll(a[:, ::-1, :], 1, axis=1)  # y -> -y
        return F(d), F(ux), -F(uy), F(uz)

    b = oracle.step(19, *refl(*f), nu=0.02, nsteps=3)
    assert maxdiff(b, refl(*out)) < 1e-15


def test_cavity_mirror_symmetry():
    """Reflecting x with the lid velocity reversed is an exact symmetry of the
    cavity rules (including the lid-corner rule)."""
    d, u, v = inputs.smooth_random((9, 10), seed=23, u_amp=0.05)
    out = oracle.step(9, d, u, v, nu=0.02, bc=oracle.CAVITY, lid=(0.1, 0, 0), nsteps=6)
    F = lambda a: a[:, ::-1]
    a = oracle.step(9, F(d), -F(u), F(v), nu=0.02, bc=oracle.CAVITY, lid=(-0.1, 0, 0), nsteps=6)
    assert maxdiff(a, (F(out[0]), -F(out[1]), F(out[2]))) < 1e-15


def test_cavity_3d_diagonal_lid_symmetries():
    """Section 3.3.2's cubic cavity with the diagonal lid (a, a, 0) on the top z
    face: swapping x and y (with u and v) and reflecting x with the lid's x
    component reversed are exact symmetries of the 3D wall and lid rules, so a
    wrong index or sign in one axis's wall treatment breaks one of them."""
    n, a = 7, 0.05
    f = inputs.smooth_random((n, n, n), seed=24, u_amp=0.04, d_amp=0.005)
    out = oracle.step(19, *f, nu=0.03, bc=oracle.CAVITY, lid=(a, a, 0.0), nsteps=5)

    def swap(d, ux, uy, uz):  # arrays (z, y, x): x <-> y
        T = lambda q: np.transpose(q, (0, 2, 1))
        return T(d), T(uy), T(ux), T(uz)

    b = oracle.step(19, *swap(*f), nu=0.03, bc=oracle.CAVITY, lid=(a, a, 0.0), nsteps=5)
    assert maxdiff(b, swap(*out)) < 1e-15

    def refl(d, ux, uy, uz):  # x -> -x about the box centre
        F = lambda q: q[:, :, ::-1]
        return F(d), -F(ux), F(uy), F(uz)

    c = oracle.step(19, *refl(*f), nu=0.03, bc=oracle.CAVITY, lid=(-a, a, 0.0), nsteps=5)
    assert maxdiff(c, refl(*out)) < 1e-15
    # the lid drives the flow: without it the state differs
    r = oracle.step(19, *f, nu=0.03, bc=oracle.CAVITY, lid=(0.0, 0.0, 0.0), nsteps=5)
    assert maxdiff(r, out) > 1e-4


def test_d3q19_z_uniform_equals_d2q9():
    """D3Q19 weights project onto D2Q9 (1/3 + 2/18 = 4/9, 1/18 + 2/36 = 1/9, 1/36):
    on z-uniform data with u_z = 0 the two lattices give the same update."""
    d, u, v = inputs.smooth_random((10, 12), seed=5, u_amp=0.06)
    a = oracle.step(9, d, u, v, nu=0.03, nsteps=7)
    R = lambda x: np.repeat(x[None], 4, 0)
    b = oracle.step(19, R(d), R(u), R(v), np.zeros((4, 10, 12)), nu=0.03, nsteps=7)
    assert maxdiff([R(x) for x in a], b[:3]) < 1e-15
    assert np.max(np.abs(b[3])) == 0.0
    # walls too: 2D cavity == 3D slab periodic in z? (walls on z would differ) ->
    # check the channel, which is walled in y only
    c = oracle.step(9, d, u, v, nu=0.03, bc=oracle.CHANNEL, nsteps=5)
    e = oracle.step(19, R(d), R(u), R(v), np.zeros((4, 10, 12)), nu=0.03, bc=oracle.CHANNEL,
                    nsteps=5)
    assert maxdiff([R(x) for x in c], e[:3]) < 1e-15


# --- closed-form solutions ----------------------------------------------------

def _tgv_amp(N, u0, nu, T):
    d, u, v = inputs.tgv2d(N, u0=u0)
    out = oracle.step(9, d, u, v, nu=nu, nsteps=T)
    return np.sum(out[1] * u) / np.sum(u * u)


def test_tgv2d_decay_and_second_order():
    """2D Taylor-Green: velocity amplitude decays as exp(-2 nu k^2 t); under diffusive
    scaling (u0 ~ 1/N, T ~ N^2, nu fixed) the error falls at second order
    (Section 2.3 and Table gtg)."""
    nu = 0.01
    errs = []
    for N in (16, 32, 64):
        u0 = 0.01 * 64 / N
        T = int(1000 * (N / 64) ** 2)
        k = 2 * np.pi / N
        errs.append(abs(_tgv_amp(N, u0, nu, T) / np.exp(-2 * nu * k * k * T) - 1))
    assert errs[-1] < 1e-3
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # pre-asymptotic at N = 16; the finest pair must be close to 2
    assert orders[0] > 1.4 and orders[1] > 1.8, (errs, orders)


def test_tgv3d_stokes_decay():
    """Tiny-amplitude 3D Taylor-Green: |k|^2 = 3 k^2, energy decays as exp(-6 nu k^2 t);
    the decay-rate error of the lattice operator falls at second order in k."""
    nu = 0.02
    errs = []
    for n, T in ((12, 113), (24, 450)):
        f = inputs.tgv3d(n, u0=1e-5)
        ke0 = oracle.diagnostics(*f)["ke"]
        out = oracle.step(19, *f, nu=nu, nsteps=T)
        ke = oracle.diagnostics(*out)["ke"]
        k = 2 * np.pi / n
        errs.append(abs(-np.log(ke / ke0) / (6 * nu * k * k * T) - 1))
    assert errs[1] < 0.02 and np.log2(errs[0] / errs[1]) > 1.9, errs


def test_poiseuille_second_order():
    """Body-forced channel (Eq. force, half-way walls at y = -1/2 and ny - 1/2):
    steady profile -> g/(2 nu) (y + 1/2)(ny - 1/2 - y) at second order (Couette Test 1
    with u_L = 0)."""
    nu, g = 0.1, 1e-6
    errs = []
    for ny in (8, 16):
        z = np.zeros((ny, 3))
        out = oracle.step(9, z, z, z, nu=nu, bc=oracle.CHANNEL, force=(g, 0, 0),
                          nsteps=int(10 * ny * ny / nu))
        y = np.arange(ny)
        ex = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
        errs.append(np.max(np.abs(out[1][:, 0] - ex)) / ex.max())
        assert np.max(np.abs(out[2])) < 1e-14 * g / g
    assert errs[0] < 0.02
    assert np.log2(errs[0] / errs[1]) > 1.9


def test_couette_moving_wall():
    """Top wall moving at U (moving-wall term, Eq. ACM2.0ccccbb): linear steady profile
    U (y + 1/2)/ny, exact up to the decay of the transient."""
    ny, U, nu = 12, 1e-3, 0.1
    z = np.zeros((ny, 3))
    out = oracle.step(9, z, z, z, nu=nu, bc=oracle.CHANNEL, lid=(U, 0, 0),
                      nsteps=int(12 * ny * ny / nu))
    y = np.arange(ny)
    assert np.max(np.abs(out[1][:, 0] - U * (y + 0.5) / ny)) / U < 1e-9


# --- the adjoint, by brute force ----------------------------------------------

def _loss(Q, state, target, nu, T, **kw):
    out = oracle.step(Q, *state, nu=nu, nsteps=T, **kw)
    return 0.5 * sum(np.sum((o - t) ** 2) for o, t in zip(out[1:], target))


@pytest.mark.parametrize("Q,shape,kw", [
    (9, (7, 9), dict()),
    (9, (6, 7), dict(bc=oracle.CAVITY, lid=(0.08, 0, 0))),
    (9, (6, 5), dict(bc=oracle.CHANNEL, force=(1e-3, 0, 0))),
    (19, (4, 5, 3), dict()),
    (19, (4, 4, 4), dict(bc=oracle.CAVITY, lid=(0.05, 0.05, 0))),
])
def test_adjoint_matches_central_differences(Q, shape, kw):
    """Reverse-mode gradient of 0.5|u(T) - u_t|^2 vs FP64 central differences of the
    forward oracle, in random directions and in nu."""
    T, nu = 4, 0.03
    st = inputs.smooth_random(shape, seed=31, u_amp=0.05, d_amp=0.02)
    tgt = inputs.smooth_random(shape, seed=32, u_amp=0.05)[1:]
    loss, g, gnu = oracle.grad(Q, st, tgt, nu=nu, T=T, **kw)
    assert np.isclose(loss, _loss(Q, st, tgt, nu, T, **kw), rtol=1e-14)
    rng = np.random.default_rng(33)
    h = 1e-6
    for _ in range(3):
        dirs = [rng.standard_normal(shape) for _ in st]
        lp = _loss(Q, [s + h * e for s, e in zip(st, dirs)], tgt, nu, T, **kw)
        lm = _loss(Q, [s - h * e for s, e in zip(st, dirs)], tgt, nu, T, **kw)
        fd = (lp - lm) / (2 * h)
        an = sum(np.sum(gi * e) for gi, e in zip(g, dirs))
        assert abs(fd - an) <= 1e-7 * max(abs(fd), 1e-3 * loss), (fd, an)
    hn = 1e-6
    fdn = (_loss(Q, st, tgt, nu + hn, T, **kw) - _loss(Q, st, tgt, nu - hn, T, **kw)) / (2 * hn)
    assert abs(fdn - gnu) <= 1e-6 * max(abs(fdn), 1e-6), (fdn, gnu)
