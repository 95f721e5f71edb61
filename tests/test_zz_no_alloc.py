"""The allocation-free diagnostics entry point against the workspace-based one.

lwacm_diagnostics_noalloc serves callers that cannot allocate device memory: it
keeps its partial sums in a fixed device array inside the library instead of a
caller-bound workspace. It must give the same FP64 global quantities as
lwacm_diagnostics, on repeated calls (the shared array keeps the previous call's
contents), called through the C ABI. This file sorts last so that a run that
stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from paper_1111_2142_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("mass", "jx", "jy", "jz", "ke", "umax", "mpar", "mperp")


@pytest.fixture(scope="module")
def lw():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_2142_gb300 import lwacm
    lib = lwacm.load()
    lib.lwacm_diagnostics_noalloc.argtypes = [ctypes.c_void_p] * 4 + [
        ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.lwacm_diagnostics_noalloc.restype = ctypes.c_int
    return lwacm


def _noalloc(lw, sim, out):
    lib = lw.load()
    vp = [ctypes.c_void_p() for _ in range(4)]
    dt, pitch = ctypes.c_int(), ctypes.c_longlong()
    assert lib.lwacm_fields(sim._h, *[ctypes.byref(v) for v in vp], ctypes.byref(dt),
                            ctypes.byref(pitch)) == lw.OK
    n = sim.nx * sim.ny * sim.nz
    st = lib.lwacm_diagnostics_noalloc(vp[0], vp[1], vp[2], vp[3], n, dt.value,
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(sim.stream.cuda_stream))
    assert st == lw.OK
    sim.sync()
    return out.cpu().numpy().copy()


# One partial-sum block covers 32768 nodes: the small shapes use one block, 64^3 eight
# (the final pass then sums several partials) and 256^3, the benchmark's lattice,
# 512; FP32, BF16 and FP16 storage.
@pytest.mark.parametrize("Q,shape,storage", [(19, (12, 16, 20), 0), (9, (48, 40), 0),
                                             (19, (9, 10, 11), 1), (19, (13, 9, 7), 2),
                                             (19, (64, 64, 64), 0), (9, (300, 333), 2),
                                             (19, (256, 256, 256), 0)])
def test_noalloc_matches_workspace_diagnostics(lw, Q, shape, storage):
    import torch
    f = inputs.smooth_random(shape, seed=40, u_amp=0.05, d_amp=0.01)
    ny, nx = shape[-2], shape[-1]
    nz = shape[0] if Q == 19 else 1
    sim = lw.Lwacm(Q, nx, ny, nz, 0.02, storage=storage)
    sim.set_fields(*f)
    out = torch.full((9,), float("nan"), dtype=torch.float64, device="cuda")
    n = nx * ny * nz
    for call in range(2):  # two calls in a row, the state changing in between
        sim.step(5)
        ref = sim.diagnostics()
        st = sim.get_fields()
        dm = float(np.max(np.abs(st[0])))
        um = float(np.sqrt(np.max(sum(c.astype(np.float64) ** 2 for c in st[1:]))))
        scale = {"mass": dm, "jx": (1 + dm) * um, "jy": (1 + dm) * um, "jz": (1 + dm) * um,
                 "ke": (1 + dm) * um * um, "umax": 0.0, "mpar": 2 * um * um, "mperp": 2 * um * um}
        got = _noalloc(lw, sim, out)
        for k, key in enumerate(KEYS):
            # the two reductions add the same FP64 terms in different orders; each
            # order is off by at most a few hundred roundings (2^-53) of the sum of
            # the terms' magnitudes, bounded by n times the largest term
            assert abs(got[k] - ref[key]) <= 1e-13 * max(1.0, abs(ref[key]), n * scale[key]), \
                (call, key, got[k], ref[key])
        assert got[8] == 0.0
    sim.close()


def test_noalloc_counts_non_finite_nodes(lw):
    """Planted NaN / infinity values over several partial-sum blocks (64^3 nodes, eight
    blocks): out_dev[8] is the number of nodes with a non-finite field value (a node
    with several counts once); two calls in a row, the second with more planted."""
    import torch
    lib = lw.load()
    n = 64 ** 3
    rng = np.random.default_rng(41)
    fields = [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(4)]
    out = torch.full((9,), -1.0, dtype=torch.float64, device="cuda")
    planted = set()
    for call, count in enumerate((7, 23)):
        idx = rng.choice(n, size=count, replace=False)
        for k, i in enumerate(idx):
            f = fields[k % 4]
            f[int(i)] = float("nan") if k % 3 else float("inf")
            planted.add(int(i))
        nodes = set(planted)
        # one node with two non-finite fields still counts once
        j = int(idx[0])
        fields[(0 + 1) % 4][j] = float("-inf")
        st = lib.lwacm_diagnostics_noalloc(*[ctypes.c_void_p(f.data_ptr()) for f in fields], n, lw.F32,
                                           ctypes.c_void_p(out.data_ptr()), None)
        assert st == lw.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[8] == float(len(nodes)), (call, got[8], len(nodes))


def test_noalloc_rejects_oversize_and_bad_args(lw):
    import torch
    lib = lw.load()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(9, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    o = ctypes.c_void_p(out.data_ptr())
    big = 33554432 + 1  # one node more than the static scratch covers
    assert lib.lwacm_diagnostics_noalloc(p, p, p, None, big, lw.F32, o, None) == lw.E_RANGE
    assert lib.lwacm_diagnostics_noalloc(p, p, p, None, 0, lw.F32, o, None) == lw.E_ARG
    assert lib.lwacm_diagnostics_noalloc(None, p, p, None, 4, lw.F32, o, None) == lw.E_ARG
    assert lib.lwacm_diagnostics_noalloc(p, p, p, None, 4, 7, o, None) == lw.E_ARG
    # a valid small call still works after the rejected ones
    assert lib.lwacm_diagnostics_noalloc(p, p, p, None, 16, lw.F32, o, None) == lw.OK
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy()[:8], 0.0)
