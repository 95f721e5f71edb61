"""The benchmarked kernel against the FP64 oracle over the workload's full 1000 steps.

The 3D Taylor-Green vortex with the benchmark's parameters (u0 = 0.02, nu = 0.005,
k = 2 pi / N; Section 2.1's update of Eq. ACM2.0 with u = rho u / rho) is advanced
1000 steps on the GPU by the half-row kernel (the automatic choice for nx = 128 and
256, the kernel the benchmark times) and by the FP64 oracle from the same
initial fields, rounded once to FP32. Every node of every field is compared after
the 1000 steps, and the kinetic energy every 10 steps.

Bounds (FP32 arithmetic and storage): max|du| / u0 <= 1e-5 and
max|dd| / max(max|d_oracle|, 3 u0^2) <= 1e-4 (each stored value rounds once per
step, 2^-24 relative, after O(Q) single-precision sums; the diffusive update does
not amplify these errors, which random-walk). The kinetic energy
0.5 sum rho |u|^2 then agrees to 2 max|du| mean|u| / mean|u|^2 <= 4e-5 relative
(mean|u| / mean|u|^2 = 1.72 / u0 for this field), the bound checked on the curve.
"""
import numpy as np
import pytest

import oracle
from paper_1111_2142_gb300 import inputs

pytestmark = pytest.mark.gpu

U0, NU, T, EVERY = 0.02, 0.005, 1000, 10


@pytest.fixture(scope="module")
def lw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_2142_gb300 import lwacm
    return lwacm


def _rel_l2(g, r):
    return float(np.linalg.norm((g - r).ravel()) / max(np.linalg.norm(r.ravel()), 1e-300))


@pytest.mark.parametrize("n", [128, 256])
def test_benchmark_kernel_thousand_steps_vs_oracle(lw, n):
    f = inputs.tgv3d(n, u0=U0)
    f32 = [a.astype(np.float32).astype(np.float64) for a in f]  # the GPU's rounded initial state
    sim = lw.Lwacm(lw.D3Q19, n, n, n, NU)
    sim.set_fields(*f32)
    ke_gpu = [sim.diagnostics()["ke"]]
    for _ in range(T // EVERY):
        sim.step(EVERY)
        ke_gpu.append(sim.diagnostics()["ke"])
    got = [a.reshape(n, n, n) for a in sim.get_fields()]
    name = sim.kernel_name
    sim.close()

    state = tuple(f32)
    ke_ref = [oracle.diagnostics(*state)["ke"]]
    for _ in range(T // EVERY):
        state = oracle.step(19, *state, nu=NU, nsteps=EVERY)
        ke_ref.append(oracle.diagnostics(*state)["ke"])

    eu = max(float(np.max(np.abs(g - r))) for g, r in zip(got[1:], state[1:])) / U0
    dscale = max(float(np.max(np.abs(state[0]))), 3 * U0 ** 2)
    ed = float(np.max(np.abs(got[0] - state[0]))) / dscale
    l2 = [_rel_l2(g, r) for g, r in zip(got, state)]
    ke_gpu, ke_ref = np.array(ke_gpu), np.array(ke_ref)
    eke = float(np.max(np.abs(ke_gpu - ke_ref) / ke_ref))
    print(f"[{name}] D3Q19 TGV {n}^3 x {T}: max|du|/u0 = {eu:.2e}, max|dd|/d = {ed:.2e}, "
          f"rel L2 (d, ux, uy, uz) = {', '.join(f'{x:.1e}' for x in l2)}, "
          f"KE curve max rel = {eke:.1e}, KE(T)/KE(0) = {ke_ref[-1] / ke_ref[0]:.6f}")
    assert name.startswith("half")
    assert eu <= 1e-5 and ed <= 1e-4
    assert eke <= 4e-5
    assert np.all(np.diff(ke_ref) < 0) and np.all(np.diff(ke_gpu) < 0)
