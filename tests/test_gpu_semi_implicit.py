"""The semi-implicit pressure update (Section 2.2 item 2, Eq. FDcompact_si) on the
GPU against the FP64 oracle's, element by element: the explicit step's velocity,
then the density summed again from the old density and the new velocity.

Bounds as for the explicit update (FP32 arithmetic and storage, a few hundred
steps): max|du| / U <= 1e-5 and max|dd| / max(max|d_ref|, 3 U^2) <= 1e-4."""
import numpy as np
import pytest

import oracle
from paper_1111_2142_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_2142_gb300 import lwacm
    return lwacm


def errs(got, ref, u_scale):
    eu = max(float(np.max(np.abs(g - r))) for g, r in zip(got[1:], ref[1:])) / u_scale
    dmax = max(float(np.max(np.abs(ref[0]))), 3.0 * u_scale ** 2)
    return eu, float(np.max(np.abs(got[0] - ref[0]))) / dmax


# D2Q9 on the 2D-tile kernel (automatic) and the generic kernel; D3Q19 on the
# half-row kernel (automatic for 128-wide rows) and the generic kernel
@pytest.mark.parametrize("Q,shape,kernel", [(9, (23, 37), 0), (9, (23, 37), 1), (9, (64, 64), 0),
                                            (19, (9, 11, 13), 0), (19, (6, 16, 128), 0), (19, (6, 16, 128), 1)])
def test_semi_implicit_matches_oracle(lw, Q, shape, kernel):
    f = inputs.smooth_random(shape, seed=51, u_amp=0.05, d_amp=0.01)
    ny, nx = shape[-2], shape[-1]
    nz = 1 if Q == 9 else shape[0]
    sim = lw.Lwacm(Q, nx, ny, nz, 0.02, kernel=kernel, semi_implicit=True)
    sim.set_fields(*f)
    sim.step(200)
    got = sim.get_fields()
    name = sim.kernel_name
    sim.close()
    ref = oracle.step_semi_implicit(Q, *f, nu=0.02, nsteps=200)
    exp = oracle.step(Q, *f, nu=0.02, nsteps=200)
    eu, ed = errs(got, ref, 0.05)
    sep = errs(exp, ref, 0.05)
    print(f"[{name}] semi-implicit Q{Q} {shape} x200: du/U={eu:.2e} dd/d={ed:.2e} "
          f"(explicit vs semi-implicit oracle: {sep[0]:.1e}, {sep[1]:.1e})")
    assert eu < 1e-5 and ed < 1e-4
    assert max(sep) > 50 * max(eu, ed)  # the two updates differ far beyond the GPU's deviation


def test_semi_implicit_forced_tgv(lw):
    """The generalized Taylor-Green vortex of Table gtg (time-dependent force field,
    Eq. force) at N = 32 for 400 steps, with the semi-implicit update. The flow is
    driven and does not decay, so the FP32 rounding of each step is carried forward
    linearly: bound 2e-8 eps (|v0| + 1) per step, as for the explicit forced vortex."""
    n = 32
    eps = 2 * np.pi / n
    f = inputs.gtg_state(n, 0.0)
    sim = lw.Lwacm(lw.D2Q9, n, n, 1, inputs.GTG_NU, force_field=True, semi_implicit=True)
    sim.set_fields(*f)
    ref = tuple(np.array(a, dtype=np.float64) for a in f)
    for k in range(400):
        g = inputs.gtg_force(n, k * eps ** 2)
        sim.set_force_field(*g)
        sim.step(1)
        ref = oracle.step_semi_implicit(9, *ref, nu=inputs.GTG_NU, g=g)
    got = sim.get_fields()
    sim.close()
    U = 0.6 * eps
    eu, ed = errs(got, ref, U)
    print(f"semi-implicit forced TGV 32^2 x400: du/U={eu:.2e} dd/d={ed:.2e}")
    assert eu * U < 400 * 2e-8 * eps * (0.6 + 1.0) and ed < 1e-4


def test_semi_implicit_with_nu_p(lw):
    """With omega_p as well the density pass uses nu_p (the oracle's density of
    Eq. FDcompact c relaxed with omega_p, from the old density and the new velocity):
    checked against a step-by-step composition of the oracle's two functions."""
    f = inputs.smooth_random((20, 24), seed=52, u_amp=0.04, d_amp=0.01)
    sim = lw.Lwacm(lw.D2Q9, 24, 20, 1, 0.01, semi_implicit=True)
    sim.set_option(lw.OPT_NU_P, 0.05)
    sim.set_fields(*f)
    sim.step(50)
    got = sim.get_fields()
    sim.close()
    ref = tuple(np.array(a, dtype=np.float64) for a in f)
    for _ in range(50):
        u_new = oracle.step_nu_p(9, *ref, nu=0.01, nu_p=0.05)[1:]
        d_new = oracle.step_nu_p(9, ref[0], *u_new, nu=0.01, nu_p=0.05)[0]
        ref = (d_new,) + tuple(u_new)
    eu, ed = errs(got, ref, 0.04)
    print(f"semi-implicit + nu_p: du/U={eu:.2e} dd/d={ed:.2e}")
    assert eu < 1e-5 and ed < 1e-4
