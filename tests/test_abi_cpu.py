"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/*.h declares, and validates arguments without device
work (lwacm_create / lwacm_set_option / lwacm_workspace_bytes are host-only)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_2142_gb300 import lwacm as lw
    return lw.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(lwacm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "lwacm_create" in names and "lwacm_step" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def _create(lib, *args):
    h = ctypes.c_void_p()
    st = lib.lwacm_create(*args, ctypes.byref(h))
    return st, h


def test_create_validation(lib):
    from paper_1111_2142_gb300 import lwacm as lw
    st, h = _create(lib, lw.D3Q19, 16, 16, 16, 0.01, lw.PERIODIC)
    assert st == lw.OK and h.value
    lib.lwacm_destroy(h)
    # nu range: 0 < nu <= 1/6  (1 <= omega < 2)
    for nu in (0.0, -0.1, 0.2, float("nan")):
        assert _create(lib, lw.D3Q19, 8, 8, 8, nu, lw.PERIODIC)[0] == lw.E_RANGE
    st, h = _create(lib, lw.D2Q9, 8, 8, 1, 1.0 / 6.0, lw.PERIODIC)
    assert st == lw.OK
    lib.lwacm_destroy(h)
    bad = [(7, 8, 8, 1), (9, 8, 8, 2), (9, 0, 8, 1), (19, 8, -1, 8), (9, 1, 8, 1)]
    for Q, nx, ny, nz in bad[:4]:
        assert _create(lib, Q, nx, ny, nz, 0.01, lw.PERIODIC)[0] == lw.E_ARG
    # walled axes need two nodes
    assert _create(lib, lw.D2Q9, 1, 8, 1, 0.01, lw.CAVITY)[0] == lw.E_ARG
    assert _create(lib, lw.D2Q9, 8, 1, 1, 0.01, lw.CHANNEL)[0] == lw.E_ARG
    assert _create(lib, lw.D2Q9, 8, 8, 1, 0.01, 7)[0] == lw.E_ARG


def test_workspace_and_options(lib):
    from paper_1111_2142_gb300 import lwacm as lw
    st, h = _create(lib, lw.D3Q19, 32, 16, 8, 0.01, lw.PERIODIC)
    assert st == lw.OK
    nb = ctypes.c_size_t()
    assert lib.lwacm_workspace_bytes(h, ctypes.byref(nb)) == lw.OK
    N = 32 * 16 * 8
    # two ping-pong buffers of 4 FP32 fields + FP64 staging + reduction scratch
    assert nb.value >= 2 * 4 * N * 4 + N * 8
    assert lib.lwacm_set_option(h, lw.OPT_STORAGE, float(lw.BF16)) == lw.OK
    nb2 = ctypes.c_size_t()
    lib.lwacm_workspace_bytes(h, ctypes.byref(nb2))
    assert nb2.value < nb.value
    assert lib.lwacm_set_option(h, lw.OPT_STORAGE, 9.0) == lw.E_ARG
    assert lib.lwacm_set_option(h, lw.OPT_GRAPH_CHUNK, 3.0) == lw.E_ARG
    assert lib.lwacm_set_option(h, 99, 1.0) == lw.E_ARG
    assert lib.lwacm_set_option(h, lw.OPT_RHO0, -1.0) == lw.E_ARG
    assert lib.lwacm_set_option(h, lw.OPT_LID_X, float("inf")) == lw.E_ARG
    assert b"non-finite" in lib.lwacm_last_error(h)
    # calls that need a bound workspace report a state error, not a crash
    assert lib.lwacm_step(h, 1) == lw.E_STATE
    assert lib.lwacm_sync(h) == lw.E_STATE
    out = (ctypes.c_double * 8)()
    assert lib.lwacm_diagnostics(h, out) == lw.E_STATE
    # a misaligned or short workspace is refused before any device work
    assert lib.lwacm_bind(h, ctypes.c_void_p(4096 + 8), nb2.value, None) == lw.E_ARG
    assert lib.lwacm_bind(h, ctypes.c_void_p(4096 * 256), 16, None) == lw.E_NOMEM
    lib.lwacm_destroy(h)
    lib.lwacm_destroy(None)


def test_null_arguments(lib):
    from paper_1111_2142_gb300 import lwacm as lw
    assert lib.lwacm_create(9, 8, 8, 1, 0.01, 0, None) == lw.E_ARG
    assert lib.lwacm_workspace_bytes(None, None) == lw.E_ARG
    assert lib.lwacm_step(None, 1) == lw.E_ARG


def test_measure_fp32_peak_validation(lib):
    """The FMA-throughput probe rejects bad arguments before touching the device."""
    from paper_1111_2142_gb300 import lwacm as lw
    tf, ms = ctypes.c_double(), ctypes.c_double()
    assert lib.lwacm_measure_fp32_peak(0, None, ctypes.byref(tf), ctypes.byref(ms)) == lw.E_ARG
    assert lib.lwacm_measure_fp32_peak((1 << 20) + 1, None, ctypes.byref(tf), ctypes.byref(ms)) == lw.E_ARG
    assert lib.lwacm_measure_fp32_peak(16, None, None, ctypes.byref(ms)) == lw.E_ARG
    assert lib.lwacm_measure_fp32_peak(16, None, ctypes.byref(tf), None) == lw.E_ARG


def test_selftest_quotient_validation(lib):
    from paper_1111_2142_gb300 import lwacm as lw
    p = ctypes.c_void_p(16)
    assert lib.lwacm_selftest_quotient(None, p, p, 4, 1, None) == lw.E_ARG
    assert lib.lwacm_selftest_quotient(p, None, p, 4, 1, None) == lw.E_ARG
    assert lib.lwacm_selftest_quotient(p, p, None, 4, 0, None) == lw.E_ARG
    assert lib.lwacm_selftest_quotient(p, p, p, 0, 1, None) == lw.E_ARG
    assert lib.lwacm_selftest_quotient(p, p, p, 1 << 31, 1, None) == lw.E_ARG
    assert lib.lwacm_selftest_quotient(p, p, p, 4, 3, None) == lw.E_ARG
    assert lib.lwacm_selftest_quotient(p, p, p, 4, -1, None) == lw.E_ARG


def test_force_field_option(lib):
    """The force-field room is reserved before bind and grows the workspace by D
    FP32 fields; batched contexts refuse it; setting a field needs a bound context."""
    from paper_1111_2142_gb300 import lwacm as lw
    st, h = _create(lib, 19, 16, 8, 4, 0.02, 0)
    assert st == lw.OK
    n0 = ctypes.c_size_t()
    assert lib.lwacm_workspace_bytes(h, ctypes.byref(n0)) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_FORCE_FIELD, 2.0) == lw.E_ARG
    assert lib.lwacm_set_option(h, lw.OPT_FORCE_FIELD, 1.0) == lw.OK
    n1 = ctypes.c_size_t()
    assert lib.lwacm_workspace_bytes(h, ctypes.byref(n1)) == lw.OK
    assert n1.value - n0.value >= 3 * 16 * 8 * 4 * 4
    assert lib.lwacm_set_force_field(h, None, None, None, lw.F32, lw.DEVICE) == lw.E_STATE
    assert lib.lwacm_set_option(h, lw.OPT_FORCE_FIELD, 0.0) == lw.OK
    n2 = ctypes.c_size_t()
    assert lib.lwacm_workspace_bytes(h, ctypes.byref(n2)) == lw.OK and n2.value == n0.value
    lib.lwacm_destroy(h)
    hb = ctypes.c_void_p()
    nx = (ctypes.c_int * 2)(8, 9)
    ny = (ctypes.c_int * 2)(8, 7)
    nu = (ctypes.c_double * 2)(0.01, 0.02)
    assert lib.lwacm_batch_create(9, 2, nx, ny, None, nu, 0, ctypes.byref(hb)) == lw.OK
    assert lib.lwacm_set_option(hb, lw.OPT_FORCE_FIELD, 1.0) == lw.E_UNSUPPORTED
    lib.lwacm_destroy(hb)


def test_batch_tile_option(lib):
    """2D tile shapes: D2Q9 ensembles only; unknown shapes refused."""
    from paper_1111_2142_gb300 import lwacm as lw
    nx = (ctypes.c_int * 2)(40, 9)
    ny = (ctypes.c_int * 2)(17, 70)
    nz = (ctypes.c_int * 2)(3, 2)
    nu = (ctypes.c_double * 2)(0.01, 0.02)
    h = ctypes.c_void_p()
    assert lib.lwacm_batch_create(9, 2, nx, ny, None, nu, 0, ctypes.byref(h)) == lw.OK
    for k in range(7):
        assert lib.lwacm_set_option(h, lw.OPT_BATCH_TILE, float(k)) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_BATCH_TILE, 7.0) == lw.E_ARG
    assert lib.lwacm_set_option(h, lw.OPT_BATCH_TILE, 1.5) == lw.E_ARG
    assert lib.lwacm_kernel_name(h).decode() == "batch_tiles126x6_step"
    lib.lwacm_destroy(h)
    h3 = ctypes.c_void_p()
    assert lib.lwacm_batch_create(19, 2, nx, ny, nz, nu, 0, ctypes.byref(h3)) == lw.OK
    assert lib.lwacm_set_option(h3, lw.OPT_BATCH_TILE, 1.0) == lw.E_UNSUPPORTED
    assert lib.lwacm_set_option(h3, lw.OPT_BATCH_TILE, 0.0) == lw.OK
    lib.lwacm_destroy(h3)
    hs = ctypes.c_void_p()
    assert lib.lwacm_create(9, 8, 8, 1, 0.01, 0, ctypes.byref(hs)) == lw.OK
    assert lib.lwacm_set_option(hs, lw.OPT_BATCH_TILE, 1.0) == lw.OK  # shape of kernel 6
    assert lib.lwacm_set_option(hs, lw.OPT_KERNEL, 6.0) == lw.OK
    assert lib.lwacm_kernel_name(hs).decode() == "tiles2d_d2q9_30x6"
    lib.lwacm_destroy(hs)
    h19 = ctypes.c_void_p()
    assert lib.lwacm_create(19, 8, 8, 8, 0.01, 0, ctypes.byref(h19)) == lw.OK
    assert lib.lwacm_set_option(h19, lw.OPT_BATCH_TILE, 1.0) == lw.E_UNSUPPORTED
    assert lib.lwacm_set_option(h19, lw.OPT_KERNEL, 6.0) == lw.E_UNSUPPORTED
    lib.lwacm_destroy(h19)


def test_autotune_needs_a_bound_fresh_context(lib):
    from paper_1111_2142_gb300 import lwacm as lw
    assert lib.lwacm_autotune(None, None, 0, None, 0) == lw.E_ARG
    st, h = _create(lib, 9, 16, 16, 1, 0.02, 0)
    assert st == lw.OK
    assert lib.lwacm_autotune(h, None, 0, None, 0) == lw.E_STATE  # not bound
    lib.lwacm_destroy(h)


def test_nu_p_option(lib):
    from paper_1111_2142_gb300 import lwacm as lw
    st, h = _create(lib, 19, 16, 8, 4, 0.02, 0)
    assert lib.lwacm_set_option(h, lw.OPT_NU_P, 0.1) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_NU_P, 0.2) == lw.E_RANGE
    assert lib.lwacm_set_option(h, lw.OPT_NU_P, -0.1) == lw.E_RANGE
    assert lib.lwacm_set_option(h, lw.OPT_NU_P, 0.0) == lw.OK
    lib.lwacm_destroy(h)
    st, hc = _create(lib, 9, 16, 16, 1, 0.02, 1)
    assert lib.lwacm_set_option(hc, lw.OPT_NU_P, 0.1) == lw.E_UNSUPPORTED
    lib.lwacm_destroy(hc)


def test_scalar_option(lib):
    from paper_1111_2142_gb300 import lwacm as lw
    st, h = _create(lib, 9, 16, 12, 1, 0.02, 0)
    n0 = ctypes.c_size_t()
    assert lib.lwacm_workspace_bytes(h, ctypes.byref(n0)) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_SCALAR_ALPHA, 0.3) == lw.E_RANGE
    assert lib.lwacm_set_option(h, lw.OPT_SCALAR_ALPHA, 0.05) == lw.OK
    n1 = ctypes.c_size_t()
    assert lib.lwacm_workspace_bytes(h, ctypes.byref(n1)) == lw.OK
    assert n1.value >= n0.value + 2 * 16 * 12 * 4  # one more field in each buffer
    assert lib.lwacm_set_scalar(h, ctypes.c_void_p(16), lw.F32, lw.DEVICE) == lw.E_STATE  # not bound
    lib.lwacm_destroy(h)
    st, hc = _create(lib, 9, 16, 16, 1, 0.02, 1)
    assert lib.lwacm_set_option(hc, lw.OPT_SCALAR_ALPHA, 0.05) == lw.E_UNSUPPORTED
    lib.lwacm_destroy(hc)


def test_bulk_gamma_option(lib):
    """LWACM_OPT_BULK_GAMMA: range, one more field, periodic D2Q9 only, exclusive
    with the scalar (not with omega_p), before bind; lwacm_get_trace needs it."""
    from paper_1111_2142_gb300 import lwacm as lw
    st, h = _create(lib, 9, 16, 12, 1, 0.02, 0)
    n0 = ctypes.c_size_t()
    assert lib.lwacm_workspace_bytes(h, ctypes.byref(n0)) == lw.OK
    assert lib.lwacm_get_trace(h, ctypes.c_void_p(16), lw.F32, lw.DEVICE) == lw.E_STATE  # not bound
    for bad in (1.0, -1.0, 2.5):
        assert lib.lwacm_set_option(h, lw.OPT_BULK_GAMMA, bad) == lw.E_RANGE
    assert lib.lwacm_set_option(h, lw.OPT_BULK_GAMMA, 0.4) == lw.OK
    n1 = ctypes.c_size_t()
    assert lib.lwacm_workspace_bytes(h, ctypes.byref(n1)) == lw.OK
    assert n1.value >= n0.value + 2 * 16 * 12 * 4  # the trace field in each buffer
    assert lib.lwacm_set_option(h, lw.OPT_SCALAR_ALPHA, 0.05) == lw.E_UNSUPPORTED
    assert lib.lwacm_set_option(h, lw.OPT_NU_P, 0.1) == lw.OK  # both improvements of Section 3.2
    assert lib.lwacm_set_option(h, lw.OPT_NU_P, 0.0) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_BULK_GAMMA, 0.0) == lw.OK  # off again
    n2 = ctypes.c_size_t()
    assert lib.lwacm_workspace_bytes(h, ctypes.byref(n2)) == lw.OK and n2.value == n0.value
    assert lib.lwacm_set_option(h, lw.OPT_SCALAR_ALPHA, 0.05) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_BULK_GAMMA, 0.4) == lw.E_UNSUPPORTED
    lib.lwacm_destroy(h)
    for args in ((19, 8, 8, 8, 0.02, 0), (9, 16, 16, 1, 0.02, 1)):  # D3Q19; a cavity
        st, hb = _create(lib, *args)
        assert st == lw.OK
        assert lib.lwacm_set_option(hb, lw.OPT_BULK_GAMMA, 0.4) == lw.E_UNSUPPORTED
        lib.lwacm_destroy(hb)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library the binding raises."""
    from paper_1111_2142_gb300 import lwacm as lw
    monkeypatch.setattr(lw, "_lib", None)
    monkeypatch.setattr(lw, "LIB_PATH", str(tmp_path / "liblwacm.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lw.load()


def test_d2q9_variant_kernel_choice(lib):
    """The automatic choice for a periodic D2Q9 domain (decided without a device):
    the 2D-tile kernel for the plain scheme, omega_p, the bulk-viscosity variant
    and both together; the generic kernel for the passive scalar and for omega_p
    on D3Q19."""
    from paper_1111_2142_gb300 import lwacm as lw
    st, h = _create(lib, 9, 40, 24, 1, 0.02, 0)
    assert st == lw.OK
    name = lambda: lib.lwacm_kernel_name(h).decode()
    assert name() == "tiles2d_d2q9_30x14"
    assert lib.lwacm_set_option(h, lw.OPT_NU_P, 0.1) == lw.OK
    assert name() == "tiles2d_d2q9_30x14"
    assert lib.lwacm_set_option(h, lw.OPT_BULK_GAMMA, 0.4) == lw.OK
    assert name() == "tiles2d_d2q9_30x14"  # both improvements of Section 3.2
    assert lib.lwacm_set_option(h, lw.OPT_NU_P, 0.0) == lw.OK
    assert name() == "tiles2d_d2q9_30x14"
    assert lib.lwacm_set_option(h, lw.OPT_BULK_GAMMA, 0.0) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_SCALAR_ALPHA, 0.05) == lw.OK
    assert name() == "generic_d2q9"
    lib.lwacm_destroy(h)
    st, h3 = _create(lib, 19, 16, 8, 4, 0.02, 0)
    assert lib.lwacm_set_option(h3, lw.OPT_NU_P, 0.1) == lw.OK
    assert lib.lwacm_kernel_name(h3).decode() == "generic_d3q19"
    lib.lwacm_destroy(h3)


def test_semi_implicit_option(lib):
    """The semi-implicit pressure update (Eq. FDcompact_si) is a 0/1 option for single
    periodic domains, exclusive with the passive scalar and the bulk-viscosity
    variant; checked without a device."""
    from paper_1111_2142_gb300 import lwacm as lw
    st, h = _create(lib, 9, 40, 24, 1, 0.02, lw.PERIODIC)
    assert st == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_SEMI_IMPLICIT, 2.0) == lw.E_ARG
    assert lib.lwacm_set_option(h, lw.OPT_SEMI_IMPLICIT, 1.0) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_SCALAR_ALPHA, 0.01) == lw.E_UNSUPPORTED
    assert lib.lwacm_set_option(h, lw.OPT_BULK_GAMMA, 0.4) == lw.E_UNSUPPORTED
    assert lib.lwacm_set_option(h, lw.OPT_NU_P, 0.05) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_SEMI_IMPLICIT, 0.0) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_SCALAR_ALPHA, 0.01) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_SEMI_IMPLICIT, 1.0) == lw.E_UNSUPPORTED
    lib.lwacm_destroy(h)
    for bc in (lw.CAVITY, lw.CHANNEL):
        st, h = _create(lib, 19, 8, 8, 8, 0.02, bc)
        assert st == lw.OK
        assert lib.lwacm_set_option(h, lw.OPT_SEMI_IMPLICIT, 1.0) == lw.E_UNSUPPORTED
        lib.lwacm_destroy(h)


def test_stochastic_rounding_option(lib):
    """Stochastic rounding of BF16 / FP16 stores is a 0/1 option for single periodic
    D3Q19 domains with half-width storage and the plain scheme; checked without a
    device (the kernel choice itself is made at bind)."""
    from paper_1111_2142_gb300 import lwacm as lw
    st, h = _create(lib, 19, 256, 16, 8, 0.02, lw.PERIODIC)
    assert st == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_STOCHASTIC_ROUNDING, 2.0) == lw.E_ARG
    assert lib.lwacm_set_option(h, lw.OPT_STOCHASTIC_ROUNDING, 1.0) == lw.E_UNSUPPORTED  # FP32 storage
    assert lib.lwacm_set_option(h, lw.OPT_STORAGE, float(lw.F16)) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_STOCHASTIC_ROUNDING, 1.0) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_STORAGE, float(lw.F32)) == lw.E_UNSUPPORTED
    assert lib.lwacm_set_option(h, lw.OPT_STORAGE, float(lw.BF16)) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_STOCHASTIC_ROUNDING, 0.0) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_SEMI_IMPLICIT, 1.0) == lw.OK
    assert lib.lwacm_set_option(h, lw.OPT_STOCHASTIC_ROUNDING, 1.0) == lw.E_UNSUPPORTED
    lib.lwacm_destroy(h)
    for lat, bc in ((9, lw.PERIODIC), (19, lw.CAVITY), (19, lw.CHANNEL)):
        st, h = _create(lib, lat, 256, 16, 8 if lat == 19 else 1, 0.02, bc)
        assert st == lw.OK
        assert lib.lwacm_set_option(h, lw.OPT_STORAGE, float(lw.BF16)) == lw.OK
        assert lib.lwacm_set_option(h, lw.OPT_STOCHASTIC_ROUNDING, 1.0) == lw.E_UNSUPPORTED
        lib.lwacm_destroy(h)


def test_selftest_round_validation(lib):
    from paper_1111_2142_gb300 import lwacm as lw
    p = ctypes.c_void_p(16)
    assert lib.lwacm_selftest_round(None, p, 4, lw.BF16, 0, None) == lw.E_ARG
    assert lib.lwacm_selftest_round(p, None, 4, lw.BF16, 0, None) == lw.E_ARG
    assert lib.lwacm_selftest_round(p, p, 0, lw.F16, 0, None) == lw.E_ARG
    assert lib.lwacm_selftest_round(p, p, 1 << 31, lw.F16, 0, None) == lw.E_ARG
    assert lib.lwacm_selftest_round(p, p, 4, lw.F32, 0, None) == lw.E_ARG


def test_prepare_validation(lib):
    """lwacm_prepare needs a bound context with fields and a step count >= 0."""
    from paper_1111_2142_gb300 import lwacm as lw
    st, h = _create(lib, 19, 16, 8, 4, 0.02, 0)
    assert st == lw.OK
    assert lib.lwacm_prepare(h, 64) == lw.E_STATE
    assert lib.lwacm_prepare(None, 64) == lw.E_ARG
    lib.lwacm_destroy(h)
