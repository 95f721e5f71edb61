"""Forcing with a space- and time-dependent acceleration (Eq. force) on the GPU:
the generalized Taylor-Green vortex of Section 3.2 against the FP64 oracle and
against the paper's Table gtg, and one-step parity of the force-field path.

The L1 readings are the ones stated in tests/test_oracle_forced_tgv.py."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1111_2142_gb300 import inputs

sys.path.insert(0, os.path.dirname(__file__))
from test_oracle_forced_tgv import gtg_l1, paper_table  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_2142_gb300 import lwacm
    return lwacm


def run_gpu_gtg(lw, n):
    """Every step: g(x, t) evaluated on the device in FP64 at the state's time
    level, copied in with lwacm_set_force_field, then one step."""
    import torch
    eps = 2.0 * np.pi / n
    sim = lw.Lwacm(lw.D2Q9, n, n, 1, inputs.GTG_NU, force_field=True)
    sim.set_fields(*inputs.gtg_state(n, 0.0))
    x = torch.arange(n, dtype=torch.float64, device="cuda") * eps
    Y, X = torch.meshgrid(x, x, indexing="ij")
    steps = inputs.gtg_steps(n)
    with torch.cuda.stream(sim.stream):
        for k in range(steps):
            t = k * eps ** 2
            a, b = X - inputs.GTG_U0 * t, Y - inputs.GTG_V0 * t
            amp = eps ** 3 * (2.0 * inputs.GTG_NU * np.cos(t) - np.sin(t))
            sim.set_force_field(torch.sin(a) * torch.cos(b) * amp, -torch.cos(a) * torch.sin(b) * amp)
            sim.step(1)
    name = sim.kernel_name
    got = sim.get_fields()
    sim.close()
    return got, steps * eps ** 2, name


def test_generalized_tgv(lw):
    """N = 32 and 64: every node against the FP64 oracle after 1556 / 6225 steps.
    The FP32 run drifts from the FP64 one about linearly in the step count (the
    forcing is re-rounded to FP32 every step and the flow never decays). One step
    rounds each stored value once, at most 2^-24 = 6e-8 of it, so the linear worst
    case is 6e-8 of the velocity scale eps (|v0| + 1) per step; bound 2e-8 per step.
    Measured: the generic kernel ~2.5e-9 per step, the 2D-tile kernel (the automatic
    choice, whose link values and sums round in another order) ~8e-9. N = 32, 64, 128: L1 errors against Table gtg. The table's
    eps = pi/64 values fall off second order (ratio 3.1 against 3.9 one level
    up), the oracle's do not, so at N = 128 the band is wider."""
    paper = paper_table()
    for n in (32, 64, 128):
        got, t_end, name = run_gpu_gtg(lw, n)
        assert name.startswith("tiles2d")  # the 2D-tile kernel carries the force field
        l1 = gtg_l1(n, *got, t_end)
        for k, nm in enumerate("uvp"):
            r = l1[k] / paper[n][k]
            print(f"[{name}] GTG N={n}: L1[{nm}] {l1[k]:.5e} paper {paper[n][k]:.5e} ratio {r:.3f}")
            lo = 0.8 if n < 128 else 0.65
            assert lo < r < 1.05, (n, nm, r)
        if n <= 64:
            eps = 2.0 * np.pi / n
            d, ux, uy = inputs.gtg_state(n, 0.0)
            for k in range(inputs.gtg_steps(n)):
                d, ux, uy = oracle.step_force_field(9, d, ux, uy, nu=inputs.GTG_NU,
                                                    g=inputs.gtg_force(n, k * eps ** 2))
            uscale = eps * (1.0 + abs(inputs.GTG_V0))
            eu = max(float(np.max(np.abs(g - r))) for g, r in zip(got[1:], (ux, uy))) / uscale
            ed = float(np.max(np.abs(got[0] - d))) / float(np.max(np.abs(d)))
            steps = inputs.gtg_steps(n)
            print(f"GTG N={n}: GPU vs oracle du/U = {eu:.2e}, dd/max|d| = {ed:.2e} after {steps} steps")
            assert eu < 2e-8 * steps and ed < 2e-8 * steps


@pytest.mark.parametrize("kernel", [1, 0])
@pytest.mark.parametrize("Q,shape,bc", [(9, (19, 23), 0), (9, (16, 21), 2), (9, (17, 15), 1),
                                        (19, (6, 8, 128), 0), (19, (5, 7, 9), 1)])
def test_force_field_one_step(lw, Q, shape, bc, kernel):
    """One step with a random force field (plus a constant force) from a random
    state: GPU == oracle to FP32 rounding, periodic, channel and cavity, on the
    generic kernel and on the automatic choice (the 2D-tile kernel for D2Q9, which
    adds the forcing itself; the generic kernel for D3Q19)."""
    rng = np.random.default_rng(11)
    f = inputs.smooth_random(shape, seed=21, u_amp=0.04, d_amp=0.01)
    D = 2 if Q == 9 else 3
    g = tuple(rng.normal(size=shape) * 2e-4 for _ in range(D))
    g0 = (1e-4, -5e-5, 2e-5) if D == 3 else (1e-4, -5e-5)
    dims = (shape[1], shape[0], 1) if Q == 9 else (shape[2], shape[1], shape[0])
    lid = (0.05, 0.0) if (bc == 1 and Q == 9) else ((0.05, 0.0, 0.0) if bc == 1 else None)
    sim = lw.Lwacm(Q, *dims, 0.02, bc, force_field=True, force=g0, lid=lid, kernel=kernel)
    sim.set_fields(*f)
    sim.set_force_field(*g)
    assert sim.kernel_name.startswith("tiles2d" if (Q == 9 and kernel == 0) else "generic")
    sim.step(2)
    got = sim.get_fields()
    ref = f
    gsum = tuple(gi + g0[a] for a, gi in enumerate(g))
    for _ in range(2):
        ref = oracle.step_force_field(Q, *ref, nu=0.02, g=gsum, bc=bc,
                                      lid=(0.05, 0.0, 0.0) if bc == 1 else None)
    eu = max(float(np.max(np.abs(a - b))) for a, b in zip(got[1:], ref[1:])) / 0.04
    ed = float(np.max(np.abs(got[0] - ref[0]))) / max(float(np.max(np.abs(ref[0]))), 3 * 0.04 ** 2)
    print(f"force field Q{Q} {shape} bc={bc}: du/U={eu:.2e} dd/d={ed:.2e}")
    assert eu < 1e-6 and ed < 1e-5
    # switching the field off again returns to the fastest kernel for the shape
    sim.set_force_field(None, None, None)
    sim.close()


@pytest.mark.parametrize("shape,storage", [((3, 8, 256), 0), ((11, 24, 128), 0), ((6, 16, 256), 2),
                                           ((4, 16, 384), 0), ((3, 8, 512), 2)])
def test_constant_force_on_the_half_kernel(lw, shape, storage):
    """A constant acceleration (Eq. force) on the half-row D3Q19 kernel (256- and
    128-node rows and rows of 128-node segments, FP32 and FP16 storage), 60 steps
    against the oracle; with a force
    field instead, the generic kernel runs."""
    f = inputs.smooth_random(shape, seed=31, u_amp=0.03, d_amp=0.01)
    nz, ny, nx = shape
    g = (1e-4, 2e-5, -1e-4)
    sim = lw.Lwacm(lw.D3Q19, nx, ny, nz, 0.02, force=g, storage=storage)
    assert sim.kernel_name.startswith("half")
    sim.set_fields(*f)
    sim.step(60)
    got = sim.get_fields()
    sim.close()
    ref = oracle.step(19, *f, nu=0.02, force=g, nsteps=60)
    eu = max(float(np.max(np.abs(a - b))) for a, b in zip(got[1:], ref[1:])) / 0.03
    ed = float(np.max(np.abs(got[0] - ref[0]))) / max(float(np.max(np.abs(ref[0]))), 3 * 0.03 ** 2)
    print(f"forced half kernel {shape} storage {storage} x60: du/U = {eu:.2e}, dd/d = {ed:.2e}")
    if storage == 0:
        assert eu < 1e-5 and ed < 1e-4
    else:  # FP16 storage: 60 roundings to 11 significant bits of O(0.03) velocities
        assert eu < 60 * 2.0 ** -11 and ed < 60 * 2.0 ** -11
    ff = lw.Lwacm(lw.D3Q19, nx, ny, nz, 0.02, force_field=True)
    ff.set_fields(*f)
    ff.set_force_field(*[np.full(shape, c) for c in g])
    assert ff.kernel_name.startswith("generic")
    ff.close()
