"""GPU adjoint (lwacm_forward_record / lwacm_backward and the autograd wrapper)
against the FP64 oracle's reverse-mode gradient and against central finite
differences of the GPU forward run.

Loss: J = 0.5 sum |u(T) - u_target|^2; gradients with respect to the initial
(d, u) and nu. Tolerances: the adjoint runs in FP32 through T steps, like the
forward, so its element errors against the FP64 gradient are bounded like the
forward's (1e-5 of the gradient scale per few hundred steps); dJ/dnu is a sum
over all nodes and steps accumulated in FP64 from FP32 terms (relative 1e-4).
"""
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


def gpu_grad(lw, Q, f, target, nu, T, stride=0, force=None, bc=0, lid=None):
    import torch
    shape = f[0].shape
    nz = 1 if Q == 9 else shape[0]
    sim = lw.Lwacm(Q, shape[-1], shape[-2], nz, nu, bc, force=force, lid=lid)
    sim.set_fields(*f)
    sim.forward_record(T, stride)
    out = sim.get_fields()
    lam = [torch.zeros(shape, dtype=torch.float64, device="cuda")]
    loss = 0.0
    for o, t in zip(out[1:], target):
        lam.append(torch.tensor(o - t, device="cuda"))
        loss += 0.5 * float(np.sum((o - t) ** 2))
    g, gnu = sim.backward(lam)
    sim.close()
    return loss, [x.cpu().numpy() for x in g], gnu


# (8, 16, 128), (5, 8, 256), (9, 24, 128) and (4, 8, 128) with a force run the
# row-tiled gather (128- and 256-node rows: several columns, ragged z-runs, one
# plane's rows wrapping in y); the other shapes the tiled gather
@pytest.mark.parametrize("Q,shape,force", [(19, (8, 10, 12), None), (9, (16, 20), None),
                                           (19, (6, 8, 10), (2e-4, -1e-4, 5e-5)),
                                           (9, (12, 16), (1e-4, 2e-4)),
                                           (19, (8, 16, 128), None), (19, (5, 8, 256), None),
                                           (19, (9, 24, 128), None), (19, (4, 8, 128), (2e-4, -1e-4, 5e-5))])
def test_adjoint_matches_fp64_oracle(lw, Q, shape, force):
    T, nu = 6, 0.03
    st = inputs.smooth_random(shape, seed=51, u_amp=0.05, d_amp=0.01)
    tgt = inputs.smooth_random(shape, seed=52, u_amp=0.05)[1:]
    f3 = None if force is None else tuple(force) + (0.0,) * (3 - len(force))
    loss, g, gnu = gpu_grad(lw, Q, st, tgt, nu, T, force=force)
    rl, rg, rnu = oracle.grad(Q, st, tgt, nu=nu, T=T, force=f3)
    assert abs(loss - rl) <= 1e-5 * rl
    scale = max(float(np.max(np.abs(x))) for x in rg)
    err = max(float(np.max(np.abs(a - b))) for a, b in zip(g, rg)) / scale
    print(f"adjoint Q{Q} {shape} force={force}: max|dg|/max|g| = {err:.2e}, dnu rel = "
          f"{abs(gnu - rnu) / abs(rnu):.2e}")
    assert err < 1e-5
    assert abs(gnu - rnu) <= 1e-4 * abs(rnu)


@pytest.mark.parametrize("Q,shape,bc,lid", [(9, (16, 20), 1, (0.05, 0.0)), (9, (12, 14), 2, (0.03, 0.0)),
                                           (19, (6, 8, 10), 1, (0.04, 0.02, 0.0)), (9, (11, 13), 1, None)])
def test_adjoint_with_walls_matches_fp64_oracle(lw, Q, shape, bc, lid):
    """The adjoint through the link-wise wall rule (bounce-back of Eq. ACM2.0cccbb2
    and the moving-wall term of Eq. ACM2.0ccccbb, whose nu-dependence enters dL/dnu):
    cavity with a lid, channel with a moving wall, a resting cavity."""
    T, nu = 6, 0.03
    st = inputs.smooth_random(shape, seed=53, u_amp=0.05, d_amp=0.01)
    tgt = inputs.smooth_random(shape, seed=54, u_amp=0.05)[1:]
    lid3 = None if lid is None else tuple(lid) + (0.0,) * (3 - len(lid))
    loss, g, gnu = gpu_grad(lw, Q, st, tgt, nu, T, bc=bc, lid=lid)
    rl, rg, rnu = oracle.grad(Q, st, tgt, nu=nu, T=T, bc=bc, lid=lid3)
    assert abs(loss - rl) <= 1e-5 * rl
    scale = max(float(np.max(np.abs(x))) for x in rg)
    err = max(float(np.max(np.abs(a - b))) for a, b in zip(g, rg)) / scale
    print(f"adjoint walls Q{Q} {shape} bc={bc} lid={lid}: max|dg|/max|g| = {err:.2e}, dnu rel = "
          f"{abs(gnu - rnu) / abs(rnu):.2e}")
    assert err < 1e-5
    assert abs(gnu - rnu) <= 1e-4 * abs(rnu)


def test_adjoint_checkpoint_stride_invariance(lw):
    """The recomputation from checkpoints reproduces the recorded states exactly,
    so the gradient does not depend on the checkpoint stride."""
    shape = (6, 8, 9)
    st = inputs.smooth_random(shape, seed=53, u_amp=0.05)
    tgt = inputs.smooth_random(shape, seed=54, u_amp=0.05)[1:]
    res = [gpu_grad(lw, 19, st, tgt, 0.02, 11, stride=s) for s in (1, 3, 0, 11)]
    for r in res[1:]:
        for a, b in zip(r[1], res[0][1]):
            assert np.array_equal(a, b)
        assert r[2] == res[0][2]


def test_adjoint_fp64_oracle_32cubed(lw):
    """The FP64 CPU adjoint at 32^3 (random divergence-free initial field,
    wave numbers 1-8, rms 0.03; target from a second seed; nu = 0.01)."""
    n, T, nu = 32, 20, 0.01
    st = inputs.random_divfree_3d(n, n, n, rms=0.03, kmax=8, seed=2)
    tgt = inputs.random_divfree_3d(n, n, n, rms=0.03, kmax=8, seed=3)[1:]
    loss, g, gnu = gpu_grad(lw, 19, st, tgt, nu, T)
    rl, rg, rnu = oracle.grad(19, st, tgt, nu=nu, T=T)
    scale = max(float(np.max(np.abs(x))) for x in rg)
    err = max(float(np.max(np.abs(a - b))) for a, b in zip(g, rg)) / scale
    print(f"adjoint 32^3 T={T}: max|dg|/max|g| = {err:.2e}, dnu {gnu:.6e} vs {rnu:.6e}")
    assert abs(loss - rl) <= 1e-5 * rl
    assert err < 1e-5 and abs(gnu - rnu) <= 1e-4 * abs(rnu)


def test_autograd_function(lw):
    import torch
    shape = (8, 8, 16)
    st = inputs.smooth_random(shape, seed=55, u_amp=0.05)
    tgt = [torch.tensor(a, device="cuda") for a in inputs.smooth_random(shape, seed=56, u_amp=0.05)[1:]]
    sim = lw.Lwacm(19, 16, 8, 8, 0.02)
    x = [torch.tensor(a, dtype=torch.float32, device="cuda", requires_grad=True) for a in st]
    nu = torch.tensor(0.02, dtype=torch.float64, requires_grad=True)
    out = lw.run(sim, 9, nu, *x)
    loss = sum(0.5 * ((o.double() - t) ** 2).sum() for o, t in zip(out[1:], tgt))
    loss.backward()
    rl, rg, rnu = oracle.grad(19, st, [t.cpu().numpy() for t in tgt], nu=0.02, T=9)
    scale = max(float(np.max(np.abs(r))) for r in rg)
    err = max(float(np.max(np.abs(xi.grad.cpu().numpy() - r))) for xi, r in zip(x, rg)) / scale
    assert err < 1e-5
    assert abs(nu.grad.item() - rnu) <= 1e-4 * abs(rnu)
    sim.close()


def test_adjoint_central_differences_128(lw):
    """The adjoint workload: D3Q19 128^3 periodic, initial velocity divergence-free
    (wave numbers 1-8, rms 0.03, seed 2), target from seed 3, nu = 0.01, T = 500.
    * Directional derivatives along 32 random unit-rms directions (seed 4) from the
      adjoint vs FP32 central differences of the GPU loss (accumulated in FP64),
      step h = 3e-2 * rms(u0). Error measure: |fd - an| / |an| over the vector of
      the 32 directional derivatives (a single direction nearly orthogonal to the
      gradient has a tiny |an|, and its ratio measures the FP32 noise, not the
      adjoint): bound 1e-4.
    * dJ/dnu vs a central difference of the FP64 oracle's loss in nu (h = 1e-5):
      a change of nu changes every rounding of an FP32 run, so an FP32 difference
      in nu is too noisy to check against; the FP64 one is exact to ~1e-8. The GPU
      value carries the FP32 forward's and adjoint's rounding: bound 5e-4 relative.
    """
    import torch
    n, T, nu = 128, 500, 0.01
    st = inputs.random_divfree_3d(n, n, n, rms=0.03, kmax=8, seed=2)
    tgt_np = inputs.random_divfree_3d(n, n, n, rms=0.03, kmax=8, seed=3)[1:]
    tgt = [torch.tensor(a, device="cuda") for a in tgt_np]
    sim = lw.Lwacm(19, n, n, n, nu)
    f32 = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in st]

    def loss_of(fields, sim_):
        sim_.set_fields(*fields)
        sim_.step(T)
        outs = [torch.empty((n, n, n), dtype=torch.float32, device="cuda") for _ in range(4)]
        sim_.get_fields_into(outs)
        return sum(0.5 * ((o.double() - t) ** 2).sum().item() for o, t in zip(outs[1:], tgt))

    sim.set_fields(*f32)
    sim.forward_record(T)
    outs = [torch.empty((n, n, n), dtype=torch.float32, device="cuda") for _ in range(4)]
    sim.get_fields_into(outs)
    lam = [torch.zeros_like(outs[0])] + [(o.double() - t).float() for o, t in zip(outs[1:], tgt)]
    g, gnu = sim.backward(lam)
    gen = torch.Generator(device="cuda").manual_seed(4)
    h = 3e-2 * 0.03
    ans, fds = [], []
    for _ in range(32):
        dirs = [torch.randn((n, n, n), generator=gen, device="cuda") for _ in range(3)]
        ans.append(sum((gi.double() * di.double()).sum().item() for gi, di in zip(g[1:], dirs)))
        lp = loss_of([f32[0]] + [a + h * di for a, di in zip(f32[1:], dirs)], sim)
        lm = loss_of([f32[0]] + [a - h * di for a, di in zip(f32[1:], dirs)], sim)
        fds.append((lp - lm) / (2 * h))
    sim.close()
    ans, fds = np.array(ans), np.array(fds)
    agg = float(np.linalg.norm(fds - ans) / np.linalg.norm(ans))

    def oracle_loss(nu_):
        out = oracle.step(19, *st, nu=nu_, nsteps=T)
        return 0.5 * sum(float(np.sum((o - t) ** 2)) for o, t in zip(out[1:], tgt_np))
    hn = 1e-5
    fdn = (oracle_loss(nu + hn) - oracle_loss(nu - hn)) / (2 * hn)
    print(f"adjoint 128^3 T=500: 32 directions, |fd - an|/|an| = {agg:.1e} (per direction: "
          f"median {np.median(np.abs(fds - ans) / np.abs(ans)):.1e}); "
          f"dJ/dnu {gnu:.6e} vs FP64 difference {fdn:.6e} (rel {abs(gnu - fdn) / abs(fdn):.1e})")
    assert agg < 1e-4
    assert abs(gnu - fdn) <= 5e-4 * abs(fdn)
