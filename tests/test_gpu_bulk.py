"""The D2Q9 bulk-viscosity variant (LWACM_OPT_BULK_GAMMA, Appendix "Computing
derivatives locally") on the GPU against the FP64 oracle (oracle.step_bulk): the
flow fields and the carried trace Tr^(+), on a smooth random field and on a
longitudinal wave, whose extra damping the oracle pins to nu gamma k^2/(1-gamma)
per step. Tolerances as for the plain scheme (FP32 rounding once per stored value
per step, random-walking): velocity 1e-5 of its scale, density 1e-4 of its scale,
and the trace deviation Tr^(+) - Tr^(e) (stored in place of Tr^(+), which sits
near 2/3) within 1e-3 of its scale (its largest oracle value)."""
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


def _run(lw, fields, nu, gamma, steps, nu_p=None, kernel=0, tile=0):
    """kernel 0: the automatic choice, the 2D-tile kernel; 1: the generic kernel;
    tile: the 2D-tile shape (0: 30 x 14)."""
    ny, nx = fields[0].shape
    sim = lw.Lwacm(9, nx, ny, 1, nu, bulk_gamma=gamma)
    if nu_p:
        sim.set_option(lw.OPT_NU_P, nu_p)
    if tile:
        sim.set_option(lw.OPT_BATCH_TILE, tile)
    if kernel:
        sim.set_option(lw.OPT_KERNEL, kernel)
    assert sim.kernel_name.startswith("generic" if kernel == 1 else "tiles2d"), sim.kernel_name
    sim.set_fields(*fields)
    tr0 = sim.get_trace()
    sim.step(steps)
    got = [a.reshape(ny, nx) for a in sim.get_fields()]
    tr = sim.get_trace().reshape(ny, nx)
    sim.close()
    return got, tr, tr0.reshape(ny, nx)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("gamma", [0.4, -0.3])
@pytest.mark.parametrize("shape", [(40, 48), (17, 33)])
def test_bulk_matches_oracle(lw, gamma, shape, kernel):
    f = inputs.smooth_random(shape, seed=31, u_amp=0.05, d_amp=0.01)
    got, tr, tr0 = _run(lw, f, 0.02, gamma, 200, kernel=kernel)
    assert np.all(tr0 == 0.0)  # starts at Tr^(e)
    ref = oracle.step_bulk(*f, nu=0.02, gamma=gamma, nsteps=200)
    u_scale = 0.05
    eu = max(float(np.max(np.abs(g - r))) for g, r in zip(got[1:], ref[1:3])) / u_scale
    ed = float(np.max(np.abs(got[0] - ref[0]))) / max(float(np.max(np.abs(ref[0]))), 3 * u_scale ** 2)
    dev = ref[3] - (2.0 / 3.0 + ref[1] ** 2 + ref[2] ** 2)
    et = float(np.max(np.abs(tr - dev))) / float(np.max(np.abs(dev)))
    print(f"bulk gamma={gamma} {shape}: du/U={eu:.2e} dd/d={ed:.2e} dTr/Tr_scale={et:.2e}")
    assert eu < 1e-5 and ed < 1e-4 and et < 1e-3
    # gamma acts: the plain scheme differs by far more than the tolerance
    plain = oracle.step(9, *f, nu=0.02, nsteps=200)
    assert max(float(np.max(np.abs(a - b))) for a, b in zip(plain[1:], ref[1:3])) / u_scale > 1e-3


@pytest.mark.parametrize("kernel", [0, 1])
def test_bulk_with_omega_p_matches_oracle(lw, kernel):
    """Both improvements of Section 3.2 (omega_p and gamma) on one context."""
    f = inputs.smooth_random((40, 48), seed=33, u_amp=0.05, d_amp=0.01)
    got, tr, _ = _run(lw, f, 0.02, 0.4, 200, nu_p=0.1, kernel=kernel)
    ref = oracle.step_bulk(*f, nu=0.02, nu_p=0.1, gamma=0.4, nsteps=200)
    eu = max(float(np.max(np.abs(g - r))) for g, r in zip(got[1:], ref[1:3])) / 0.05
    ed = float(np.max(np.abs(got[0] - ref[0]))) / max(float(np.max(np.abs(ref[0]))), 3 * 0.05 ** 2)
    dev = ref[3] - (2.0 / 3.0 + ref[1] ** 2 + ref[2] ** 2)
    et = float(np.max(np.abs(tr - dev))) / float(np.max(np.abs(dev)))
    print(f"bulk + nu_p: du/U={eu:.2e} dd/d={ed:.2e} dTr/Tr_scale={et:.2e}")
    assert eu < 1e-5 and ed < 1e-4 and et < 1e-3


def test_longitudinal_wave_matches_oracle(lw):
    n = 256
    k = 2 * np.pi / n
    x = np.arange(n)
    ux = np.tile(1e-3 * np.sin(k * x), (4, 1))
    f = (np.zeros_like(ux), ux, np.zeros_like(ux))
    got, tr, _ = _run(lw, f, 0.05, 0.4, 400)
    ref = oracle.step_bulk(*f, nu=0.05, gamma=0.4, nsteps=400)
    dev = ref[3] - (2.0 / 3.0 + ref[1] ** 2 + ref[2] ** 2)
    eu = float(np.max(np.abs(got[1] - ref[1]))) / 1e-3
    et = float(np.max(np.abs(tr - dev))) / float(np.max(np.abs(dev)))
    print(f"longitudinal wave: du/U={eu:.2e} dTr/Tr_scale={et:.2e}")
    assert eu < 1e-5 and et < 1e-3


@pytest.mark.parametrize("tile", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("nu_p", [None, 0.1])
def test_bulk_tile_shapes(lw, tile, nu_p):
    """Every 2D-tile shape on domains narrower and wider than the tiles (ragged
    edges, wrap across one tile), 60 steps at gamma = 0.4, alone and with omega_p,
    against the oracle."""
    for shape in ((23, 37), (33, 130), (5, 7)):
        f = inputs.smooth_random(shape, seed=35, u_amp=0.05, d_amp=0.01)
        got, tr, _ = _run(lw, f, 0.02, 0.4, 60, tile=tile, nu_p=nu_p)
        ref = oracle.step_bulk(*f, nu=0.02, gamma=0.4, nu_p=nu_p, nsteps=60)
        eu = max(float(np.max(np.abs(g - r))) for g, r in zip(got[1:], ref[1:3])) / 0.05
        ed = float(np.max(np.abs(got[0] - ref[0]))) / max(float(np.max(np.abs(ref[0]))), 3 * 0.05 ** 2)
        dev = ref[3] - (2.0 / 3.0 + ref[1] ** 2 + ref[2] ** 2)
        et = float(np.max(np.abs(tr - dev))) / float(np.max(np.abs(dev)))
        assert eu < 1e-5 and ed < 1e-4 and et < 1e-3, (tile, shape, eu, ed, et)
