"""FP64 CPU oracle for the LW-ACM update (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It is the plain, slow reference the CUDA
library is checked against and shares no code with it. The arithmetic lives in
``lwacm_oracle.c`` (populations form of Eq. ACM2.0, walls of Eqs. ACM2.0cccbb2 /
ACM2.0ccccbb, forcing of Eq. force, omega_p, the semi-implicit pressure update of
Eq. FDcompact_si, the passive scalar, the
bulk-viscosity quasi-equilibrium, the BGK comparator, the Appendix-C
finite-difference formulas and the reverse-mode adjoint); this module only
marshals numpy arrays and adds FP64 diagnostics sums (Eq. global.quantities,
Eq. 3Dmomenta).

Fields are numpy float64 arrays shaped (ny, nx) for D2Q9 or (nz, ny, nx) for
D3Q19, x fastest; d = rho - 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lwacm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblwacm_oracle.so")

PERIODIC, CAVITY, CHANNEL = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O3, OpenMP, no host-specific flags)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    import fcntl
    with open(_LIB_PATH + ".lock", "w") as lk:  # one builder at a time (multi-rank)
        fcntl.flock(lk, fcntl.LOCK_EX)
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        _compile()
    return _LIB_PATH


def _compile():
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-Wno-unused-parameter", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(ctypes.c_double)
        IP = ctypes.POINTER(ctypes.c_int)
        i, d, l = ctypes.c_int, ctypes.c_double, ctypes.c_long
        lib.lwo_step.argtypes = [i, i, i, i, d, i, d, P, P, l, P, P, P, P, i]
        lib.lwo_step_force_field.argtypes = [i, i, i, i, d, i, d, P, P, P, P, l, P, P, P, P, i]
        lib.lwo_step_scalar.argtypes = [i, i, i, i, d, d, l, P, P, P, P, P, i]
        lib.lwo_step_nu_p.argtypes = [i, i, i, i, d, d, P, P, P, P, l, P, P, P, P, i]
        lib.lwo_step_semi_implicit.argtypes = [i, i, i, i, d, P, P, P, l, P, P, P, P, i]
        lib.lwo_step_bulk.argtypes = [i, i, d, d, d, l, P, P, P, P, i]
        lib.lwo_feq_star.argtypes = [d, P, d, d, P]
        lib.lwo_fqe.argtypes = [d, P, d, P]
        lib.lwo_lattice_tables.argtypes = [i, IP, P, IP]
        lib.lwo_equilibria.argtypes = [i, d, P, P, P]
        lib.lwo_bgk_init.argtypes = [i, i, i, i, P, P, P, P, P]
        lib.lwo_bgk_step.argtypes = [i, i, i, i, d, i, d, P, l, P, i]
        lib.lwo_bgk_moments.argtypes = [i, i, i, i, P, P, P, P, P]
        lib.lwo_fd_step_d2q9.argtypes = [i, i, d, l, P, P, P]
        lib.lwo_grad.argtypes = [i, i, i, i, d, i, d, P, P, l, P, P, P, P, P, P, P,
                                 P, P, P, P, P, P]
        lib.lwo_max_threads.argtypes = []
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec3(v):
    if v is None:
        return None
    a = np.zeros(3, dtype=np.float64)
    a[:len(v)] = v
    return a


def _dims(Q, d):
    if Q == 9:
        ny, nx = d.shape
        return nx, ny, 1
    nz, ny, nx = d.shape
    return nx, ny, nz


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64).copy()


def max_threads() -> int:
    return int(_load().lwo_max_threads())


def omega_of_nu(nu: float) -> float:
    """Eq. viscosity2 solved for omega."""
    return 2.0 / (6.0 * nu + 1.0)


def lattice(Q: int):
    """Return (c [Q,3] int, w [Q], bb [Q]) of the oracle's lattice."""
    lib = _load()
    c = np.zeros(Q * 3, dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    bb = np.zeros(Q, dtype=np.int32)
    rc = lib.lwo_lattice_tables(Q, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(w),
                                bb.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    assert rc == 0
    return c.reshape(Q, 3), w, bb


def equilibria(Q: int, rho: float, u):
    """f^(e)_i and f^(e,o)_i at one state (Eq. d2q9_equilibrium_compact, Eq. feqo)."""
    lib = _load()
    fe = np.zeros(Q)
    fo = np.zeros(Q)
    rc = lib.lwo_equilibria(Q, float(rho), _p(_vec3(u)), _p(fe), _p(fo))
    assert rc == 0
    return fe, fo


def step(Q, d, ux, uy, uz=None, *, nu, bc=PERIODIC, nsteps=1, rho0=1.0, lid=None, force=None,
         nthreads=0):
    """Advance the state by nsteps updates of Eq. ACM2.0; returns new arrays."""
    lib = _load()
    d, ux, uy, uz = _f64(d), _f64(ux), _f64(uy), _f64(uz)
    nx, ny, nz = _dims(Q, d)
    rc = lib.lwo_step(Q, nx, ny, nz, float(nu), int(bc), float(rho0), _p(_vec3(lid)),
                      _p(_vec3(force)), int(nsteps), _p(d), _p(ux), _p(uy), _p(uz), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle step failed: {rc}")
    return (d, ux, uy) if Q == 9 else (d, ux, uy, uz)


def step_nu_p(Q, d, ux, uy, uz=None, *, nu, nu_p, force=None, g=None, nsteps=1, nthreads=0):
    """As step() on a periodic domain, with the pressure (density) update relaxed
    with nu_p (omega_p of Section 2.2, item 3) and the momentum with nu; force: a
    constant acceleration, g: a per-node field (gx, gy[, gz])."""
    lib = _load()
    d, ux, uy, uz = _f64(d), _f64(ux), _f64(uy), _f64(uz)
    nx, ny, nz = _dims(Q, d)
    gx = gy = gz = None
    if g is not None:
        gx, gy = _f64(g[0]), _f64(g[1])
        gz = _f64(g[2]) if len(g) > 2 and g[2] is not None else None
    rc = lib.lwo_step_nu_p(Q, nx, ny, nz, float(nu), float(nu_p), _p(_vec3(force)), _p(gx), _p(gy), _p(gz),
                           int(nsteps), _p(d), _p(ux), _p(uy), _p(uz), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle step failed: {rc}")
    return (d, ux, uy) if Q == 9 else (d, ux, uy, uz)


def step_semi_implicit(Q, d, ux, uy, uz=None, *, nu, g=None, nsteps=1, nthreads=0):
    """As step() on a periodic domain, with the semi-implicit pressure update of
    Eq. FDcompact_si (Section 2.2, item 2): the density is summed again from the
    old density and the velocity of the explicit step. g: a per-node acceleration
    field (gx, gy[, gz]) held fixed over the nsteps (Eq. force), or None."""
    lib = _load()
    d, ux, uy, uz = _f64(d), _f64(ux), _f64(uy), _f64(uz)
    nx, ny, nz = _dims(Q, d)
    gs = [None, None, None] if g is None else [_f64(c) for c in g] + [None] * (3 - len(g))
    rc = lib.lwo_step_semi_implicit(Q, nx, ny, nz, float(nu), _p(gs[0]), _p(gs[1]), _p(gs[2]), int(nsteps),
                                    _p(d), _p(ux), _p(uy), _p(uz), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle semi-implicit step failed: {rc}")
    return (d, ux, uy) if Q == 9 else (d, ux, uy, uz)


def step_scalar(Q, d, ux, uy, uz=None, *, T, nu, alpha, nsteps=1, nthreads=0):
    """Advance the flow (Eq. ACM2.0) and a passive scalar T (Eq. ACM2.0t, thermal
    diffusivity alpha, advected by the flow velocity at each step's time level) on a
    periodic domain; returns (d, ux, uy[, uz], T)."""
    lib = _load()
    d, ux, uy, uz, T = _f64(d), _f64(ux), _f64(uy), _f64(uz), _f64(T)
    nx, ny, nz = _dims(Q, d)
    rc = lib.lwo_step_scalar(Q, nx, ny, nz, float(nu), float(alpha), int(nsteps), _p(d), _p(ux), _p(uy), _p(uz),
                             _p(T), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle scalar step failed: {rc}")
    return (d, ux, uy, T) if Q == 9 else (d, ux, uy, uz, T)


def step_bulk(d, ux, uy, tr=None, *, nu, gamma, nu_p=None, nsteps=1, nthreads=0):
    """D2Q9, periodic: Eq. ACM2.0 with the modified equilibrium f^(e*) of Eq.
    quasi-equilibrium2 (the reading is in lwacm_oracle.c; it raises the bulk
    viscosity by 2 rho0 nu gamma / (1 - gamma)); tr is the normalised trace Tr^(+)
    of the last update (default Tr^(e) = 2/3 + |u|^2); nu_p: with omega_p as well
    (the density relaxed with nu_p). Returns (d, ux, uy, tr)."""
    lib = _load()
    d, ux, uy = _f64(d), _f64(ux), _f64(uy)
    tr = 2.0 / 3.0 + ux * ux + uy * uy if tr is None else _f64(tr)
    ny, nx = d.shape[-2], d.shape[-1]
    rc = lib.lwo_step_bulk(nx, ny, float(nu), float(nu_p or 0.0), float(gamma), int(nsteps), _p(d), _p(ux), _p(uy), _p(tr),
                           int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle bulk step failed: {rc}")
    return d, ux, uy, tr


def feq_star(rho, u, tr_plus, gamma):
    """The nine values f^(e*)_i (oracle link order) at one node."""
    lib = _load()
    f = np.zeros(9)
    uu = np.array([u[0], u[1]], dtype=np.float64)
    rc = lib.lwo_feq_star(float(rho), _p(uu), float(tr_plus), float(gamma), _p(f))
    if rc != 0:
        raise ValueError(f"oracle feq_star failed: {rc}")
    return f


def fqe(rho, u, tr):
    """The nine values of the quasi-equilibrium f^(qe)(rho, u, Tr) (Eq.
    quasi-equilibrium, oracle link order) at one node."""
    lib = _load()
    f = np.zeros(9)
    uu = np.array([u[0], u[1]], dtype=np.float64)
    rc = lib.lwo_fqe(float(rho), _p(uu), float(tr), _p(f))
    if rc != 0:
        raise ValueError(f"oracle fqe failed: {rc}")
    return f


def step_force_field(Q, d, ux, uy, uz=None, *, nu, g, bc=PERIODIC, nsteps=1, rho0=1.0, lid=None,
                     nthreads=0):
    """As step(), with a per-node acceleration field g = (gx, gy[, gz]) of the
    fields' shape (Eq. force with a space-dependent g), fixed over the nsteps."""
    lib = _load()
    d, ux, uy, uz = _f64(d), _f64(ux), _f64(uy), _f64(uz)
    nx, ny, nz = _dims(Q, d)
    gx, gy = _f64(g[0]), _f64(g[1])
    gz = _f64(g[2]) if len(g) > 2 and g[2] is not None else None
    rc = lib.lwo_step_force_field(Q, nx, ny, nz, float(nu), int(bc), float(rho0), _p(_vec3(lid)),
                                  _p(gx), _p(gy), _p(gz), int(nsteps), _p(d), _p(ux), _p(uy), _p(uz),
                                  int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle step failed: {rc}")
    return (d, ux, uy) if Q == 9 else (d, ux, uy, uz)


def bgk_run(Q, d, ux, uy, uz=None, *, omega, bc=PERIODIC, nsteps=1, rho0=1.0, lid=None,
            nthreads=0):
    """Equilibrium-initialised BGK-LBM comparator; returns the moments after nsteps."""
    lib = _load()
    d, ux, uy, uz = _f64(d), _f64(ux), _f64(uy), _f64(uz)
    nx, ny, nz = _dims(Q, d)
    N = nx * ny * nz
    f = np.zeros(Q * N)
    assert lib.lwo_bgk_init(Q, nx, ny, nz, _p(d), _p(ux), _p(uy), _p(uz), _p(f)) == 0
    rc = lib.lwo_bgk_step(Q, nx, ny, nz, float(omega), int(bc), float(rho0), _p(_vec3(lid)),
                          int(nsteps), _p(f), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle bgk failed: {rc}")
    assert lib.lwo_bgk_moments(Q, nx, ny, nz, _p(f), _p(d), _p(ux), _p(uy), _p(uz)) == 0
    return (d, ux, uy) if Q == 9 else (d, ux, uy, uz)


def fd_step_d2q9(d, ux, uy, *, nu, nsteps=1):
    """Appendix-C finite-difference formulas (periodic D2Q9)."""
    lib = _load()
    d, ux, uy = _f64(d), _f64(ux), _f64(uy)
    ny, nx = d.shape
    rc = lib.lwo_fd_step_d2q9(nx, ny, float(nu), int(nsteps), _p(d), _p(ux), _p(uy))
    assert rc == 0
    return d, ux, uy


def grad(Q, state, target, *, nu, T, bc=PERIODIC, rho0=1.0, lid=None, force=None):
    """Loss 0.5 sum|u(T)-u_target|^2 and its gradient w.r.t. (d0, u0) and nu.

    state: (d0, ux0, uy0[, uz0]); target: tuple of target velocity components.
    Returns (loss, (g_d, g_ux, g_uy[, g_uz]), g_nu).
    """
    lib = _load()
    d0, ux0, uy0 = _f64(state[0]), _f64(state[1]), _f64(state[2])
    uz0 = _f64(state[3]) if Q == 19 else None
    tx, ty = _f64(target[0]), _f64(target[1])
    tz = _f64(target[2]) if Q == 19 else None
    nx, ny, nz = _dims(Q, d0)
    gd, gx, gy = np.zeros_like(d0), np.zeros_like(d0), np.zeros_like(d0)
    gz = np.zeros_like(d0) if Q == 19 else None
    loss = ctypes.c_double(0.0)
    gnu = ctypes.c_double(0.0)
    rc = lib.lwo_grad(Q, nx, ny, nz, float(nu), int(bc), float(rho0), _p(_vec3(lid)),
                      _p(_vec3(force)), int(T), _p(d0), _p(ux0), _p(uy0), _p(uz0), _p(tx), _p(ty),
                      _p(tz), ctypes.byref(loss), _p(gd), _p(gx), _p(gy), _p(gz),
                      ctypes.byref(gnu))
    if rc != 0:
        raise ValueError(f"oracle grad failed: {rc}")
    gs = (gd, gx, gy) if Q == 9 else (gd, gx, gy, gz)
    return loss.value, gs, gnu.value


def diagnostics(d, ux, uy, uz=None):
    """FP64 global quantities: mass sum(d), momentum sum(rho u), kinetic energy
    0.5 sum(rho |u|^2), max |u| (cf. Eq. global.quantities)."""
    rho = 1.0 + np.asarray(d, dtype=np.float64)
    comps = [np.asarray(c, dtype=np.float64) for c in (ux, uy, uz) if c is not None]
    uu = sum(c * c for c in comps)
    mom = [float(np.sum(rho * c)) for c in comps] + [0.0] * (3 - len(comps))
    return {
        "mass": float(np.sum(d, dtype=np.float64)),
        "jx": mom[0], "jy": mom[1], "jz": mom[2],
        "ke": float(0.5 * np.sum(rho * uu)),
        "umax": float(np.sqrt(np.max(uu))),
    }
