"""The passive scalar (Eq. ACM2.0t) on the GPU against the FP64 oracle."""
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


# D2Q9 and odd D3Q19 shapes run on the generic kernel (flow and scalar in one
# pass); D3Q19 boxes with 128- or 256-node rows and ny % 8 == 0 run the flow on the
# half-row kernel and the scalar on its own row-tiled kernel (several columns,
# ragged z-chunks, one plane, y wrapping inside a column, equal runs that cross
# columns: 7 and 9 columns, none a divisor of the grid)
@pytest.mark.parametrize("Q,shape,T,kern", [(9, (48, 64), 150, "generic"), (9, (17, 23), 60, "generic"),
                                            (19, (10, 12, 14), 40, "generic"),
                                            (19, (6, 16, 128), 40, "half_d3q19_tma+scalar_rows"),
                                            (19, (5, 8, 256), 40, "half_d3q19_tma+scalar_rows"),
                                            (19, (37, 24, 128), 30, "half_d3q19_tma+scalar_rows"),
                                            (19, (1, 8, 256), 20, "half_d3q19_tma+scalar_rows"),
                                            (19, (90, 56, 128), 20, "half_d3q19_tma+scalar_rows"),
                                            (19, (70, 72, 256), 20, "half_d3q19_tma+scalar_rows")])
def test_scalar_matches_oracle(lw, Q, shape, T, kern):
    """Flow and scalar together, every node against the oracle; the scalar's total
    is conserved to FP32 rounding."""
    f = inputs.smooth_random(shape, seed=31, u_amp=0.05, d_amp=0.01)
    T0 = 1.0 + 0.2 * inputs.smooth_random(shape, seed=32, u_amp=0.0, d_amp=1.0)[0]
    nz = 1 if Q == 9 else shape[0]
    ny, nx = shape[-2], shape[-1]
    sim = lw.Lwacm(Q, nx, ny, nz, 0.02, scalar_alpha=0.03)
    assert sim.kernel_name.startswith(kern)
    sim.set_fields(*f)
    sim.set_scalar(T0)
    sim.step(T)
    got = sim.get_fields()
    gT = sim.get_scalar()
    sim.close()
    ref = oracle.step_scalar(Q, *f, T=T0, nu=0.02, alpha=0.03, nsteps=T)
    eu = max(float(np.max(np.abs(g - r))) for g, r in zip(got[1:], ref[1:-1])) / 0.05
    eT = float(np.max(np.abs(gT - ref[-1])))
    drift = abs(float(gT.sum()) - float(T0.sum())) / T0.size
    print(f"scalar Q{Q} {shape} x{T}: du/U={eu:.2e} max|dT|={eT:.2e} mean drift of T={drift:.2e}")
    assert eu < 1e-5
    assert eT < 2e-6  # T ~ 1: FP32 rounding, a few ulp per step, diffusion damps it
    assert drift < 1e-6
