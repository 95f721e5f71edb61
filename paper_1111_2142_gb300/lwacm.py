"""Thin ctypes binding of the C ABI in include/lwacm.h.

Argument marshalling only: every step of the LW-ACM path runs in the CUDA
library. PyTorch provides device memory (the workspace) and the stream. There
is no CPU fallback: loading fails loudly if liblwacm.so is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblwacm.so")

# constants mirrored from include/lwacm.h
OK, E_ARG, E_RANGE, E_STATE, E_NOMEM, E_CUDA, E_NONFINITE, E_TIMEOUT, E_UNSUPPORTED = range(9)
D2Q9, D3Q19 = 9, 19
PERIODIC, CAVITY, CHANNEL = 0, 1, 2
F32, BF16, F16, F64 = 0, 1, 2, 3
DEVICE, HOST = 0, 1
OPT_LID_X, OPT_LID_Y, OPT_LID_Z, OPT_FORCE_X, OPT_FORCE_Y, OPT_FORCE_Z = range(6)
OPT_RHO0, OPT_STORAGE, OPT_GRAPH_CHUNK, OPT_KERNEL = 6, 7, 8, 9
OPT_BATCH_MODE, OPT_TEST_WITHHOLD, OPT_FORCE_FIELD, OPT_BATCH_TILE, OPT_NU_P = 10, 11, 12, 13, 14
OPT_SCALAR_ALPHA, OPT_BULK_GAMMA, OPT_SEMI_IMPLICIT = 15, 16, 17
OPT_STOCHASTIC_ROUNDING = 18
# 2D tile shapes of the D2Q9 batched kernel (LWACM_OPT_BATCH_TILE 1..6); 0 = 1D runs
BATCH_TILE_SHAPES = {0: None, 1: (30, 6), 2: (30, 14), 3: (62, 6), 4: (30, 30), 5: (62, 14), 6: (126, 6)}

STATUS_NAMES = {OK: "OK", E_ARG: "E_ARG", E_RANGE: "E_RANGE", E_STATE: "E_STATE",
                E_NOMEM: "E_NOMEM", E_CUDA: "E_CUDA", E_NONFINITE: "E_NONFINITE",
                E_TIMEOUT: "E_TIMEOUT", E_UNSUPPORTED: "E_UNSUPPORTED"}

_lib = None


class LwacmError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load():
    """Load liblwacm.so (built by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    P = ctypes.POINTER
    sig = {
        "lwacm_create": [i, i, i, i, d, i, P(vp)],
        "lwacm_set_option": [vp, i, d],
        "lwacm_workspace_bytes": [vp, P(ctypes.c_size_t)],
        "lwacm_bind": [vp, vp, ctypes.c_size_t, vp],
        "lwacm_set_fields": [vp, vp, vp, vp, vp, i, i],
        "lwacm_step": [vp, ll],
        "lwacm_prepare": [vp, ll],
        "lwacm_fields": [vp, P(vp), P(vp), P(vp), P(vp), P(i), P(ll)],
        "lwacm_get_fields": [vp, vp, vp, vp, vp, i, i],
        "lwacm_get_fields_async": [vp, vp, vp, vp, vp, i, i],
        "lwacm_diagnostics": [vp, P(d)],
        "lwacm_step_count": [vp, P(ll)],
        "lwacm_sync": [vp],
        "lwacm_adjoint_workspace_bytes": [vp, ll, i, P(ctypes.c_size_t)],
        "lwacm_forward_record": [vp, ll, i, vp, ctypes.c_size_t],
        "lwacm_backward": [vp, vp, vp, vp, vp, i, vp, vp, vp, vp, P(d)],
        "lwacm_diagnostics_noalloc": [vp, vp, vp, vp, ll, i, vp, vp],
        "lwacm_batch_create": [i, i, P(i), P(i), P(i), P(d), i, P(vp)],
        "lwacm_batch_offsets": [vp, P(ll)],
        "lwacm_measure_fp32_peak": [ll, vp, P(d), P(d)],
        "lwacm_selftest_quotient": [vp, vp, vp, ll, i, vp],
        "lwacm_selftest_round": [vp, vp, ll, i, ctypes.c_uint, vp],
        "lwacm_selftest_schedule": [i, i, i, vp, vp, vp, vp, ll, vp],
        "lwacm_set_force_field": [vp, vp, vp, vp, i, i],
        "lwacm_autotune": [vp, ctypes.c_char_p, i, ctypes.c_char_p, ctypes.c_size_t],
        "lwacm_set_scalar": [vp, vp, i, i],
        "lwacm_get_scalar": [vp, vp, i, i],
        "lwacm_get_trace": [vp, vp, i, i],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.lwacm_last_error.argtypes = [vp]
    lib.lwacm_last_error.restype = ctypes.c_char_p
    lib.lwacm_kernel_name.argtypes = [vp]
    lib.lwacm_kernel_name.restype = ctypes.c_char_p
    lib.lwacm_destroy.argtypes = [vp]
    lib.lwacm_destroy.restype = None
    _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Lwacm:
    """One LW-ACM domain on the current CUDA device.

    Wraps lwacm_create / lwacm_set_option / lwacm_bind; the workspace is a torch
    uint8 tensor owned by this object and the stream is torch's current stream
    (or the one given).
    """

    def __init__(self, lattice, nx, ny, nz=1, nu=0.01, bc=PERIODIC, *, storage=F32, lid=None,
                 force=None, rho0=None, kernel=0, graph_chunk=None, device=None, stream=None,
                 force_field=False, scalar_alpha=None, bulk_gamma=None, semi_implicit=False,
                 stochastic_rounding=False):
        lib = load()
        self.lattice, self.nx, self.ny, self.nz = int(lattice), int(nx), int(ny), int(nz)
        self.nu, self.bc = float(nu), int(bc)
        self.n_nodes = self.nx * self.ny * self.nz
        h = ctypes.c_void_p()
        st = lib.lwacm_create(self.lattice, self.nx, self.ny, self.nz, self.nu, self.bc,
                              ctypes.byref(h))
        if st != OK:
            raise LwacmError(st, "lwacm_create")
        extra = {}
        if force_field:
            extra[OPT_FORCE_FIELD] = 1
        if scalar_alpha:
            extra[OPT_SCALAR_ALPHA] = scalar_alpha
        if bulk_gamma:
            extra[OPT_BULK_GAMMA] = bulk_gamma
        if semi_implicit:
            extra[OPT_SEMI_IMPLICIT] = 1
        if stochastic_rounding:
            extra[OPT_STOCHASTIC_ROUNDING] = 1
        self._setup(lib, h, storage, lid, force, rho0, kernel, graph_chunk, device, stream, extra)

    def _setup(self, lib, h, storage, lid, force, rho0, kernel, graph_chunk, device, stream,
               extra):
        torch = _torch()
        self._lib = lib
        self._h = h
        try:
            if storage != F32:
                self._check(lib.lwacm_set_option(h, OPT_STORAGE, float(storage)))
            for k, vec in ((OPT_LID_X, lid), (OPT_FORCE_X, force)):
                if vec is not None:
                    for a, v in enumerate(vec):
                        self._check(lib.lwacm_set_option(h, k + a, float(v)))
            if rho0 is not None:
                self._check(lib.lwacm_set_option(h, OPT_RHO0, float(rho0)))
            if graph_chunk is not None:
                self._check(lib.lwacm_set_option(h, OPT_GRAPH_CHUNK, float(graph_chunk)))
            for key, val in extra.items():
                self._check(lib.lwacm_set_option(h, key, float(val)))
            nbytes = ctypes.c_size_t()
            self._check(lib.lwacm_workspace_bytes(h, ctypes.byref(nbytes)))
            self.device = torch.device(device if device is not None else "cuda")
            self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._check(lib.lwacm_bind(h, self.workspace.data_ptr(), nbytes.value,
                                       ctypes.c_void_p(self.stream.cuda_stream)))
            if kernel:  # explicit kernels are checked against the bound device
                self._check(lib.lwacm_set_option(h, OPT_KERNEL, float(kernel)))
        except Exception:
            lib.lwacm_destroy(h)
            self._h = None
            raise
        self.storage = storage
        self.nf = 3 if self.lattice == D2Q9 else 4

    # -- helpers --
    def _check(self, st):
        if st != OK:
            msg = self._lib.lwacm_last_error(self._h).decode() if self._h else ""
            raise LwacmError(st, msg)
        return st

    @property
    def shape(self):
        return (self.ny, self.nx) if self.lattice == D2Q9 else (self.nz, self.ny, self.nx)

    def set_option(self, key, value):
        self._check(self._lib.lwacm_set_option(self._h, int(key), float(value)))

    @property
    def kernel_name(self):
        return self._lib.lwacm_kernel_name(self._h).decode()

    def close(self):
        if getattr(self, "_h", None):
            # work still enqueued on the stream may read the workspace or write the
            # destinations of enqueue-only read-backs: let it finish first
            try:
                self.stream.synchronize()
            except Exception:
                pass
            self._lib.lwacm_destroy(self._h)
            self._h = None
            self._pending = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C-ABI calls --
    def set_fields(self, d, ux, uy, uz=None):
        """Initial state from numpy arrays (host, any float -> FP64) or torch tensors
        (CUDA or host, float32/float64)."""
        arrs = [d, ux, uy] + ([uz] if self.lattice == D3Q19 else [])
        torch = _torch()
        if all(isinstance(a, np.ndarray) for a in arrs):
            keep = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in arrs]
            dtype, where = F64, HOST
        else:
            keep = [a.contiguous().reshape(-1) for a in arrs]
            dt = keep[0].dtype
            dtype = {torch.float32: F32, torch.float64: F64}[dt]
            where = DEVICE if keep[0].is_cuda else HOST
        for a in keep:
            assert (a.size if isinstance(a, np.ndarray) else a.numel()) == self.n_nodes
        ptrs = [_ptr(a) for a in keep] + [None] * (4 - len(keep))
        self._check(self._lib.lwacm_set_fields(self._h, *ptrs, dtype, where))
        if where == HOST:
            self._hold = keep  # host memory must outlive the asynchronous copy
            self.sync()
            self._hold = None

    def set_force_field(self, gx, gy, gz=None):
        """Per-node acceleration g(x) of Eq. force for the following steps (needs
        force_field=True at construction): torch tensors (CUDA or host, float32 /
        float64) or numpy arrays; set_force_field(None, None) switches it off."""
        if gx is None and gy is None and gz is None:
            self._check(self._lib.lwacm_set_force_field(self._h, None, None, None, F32, DEVICE))
            return
        arrs = [gx, gy] + ([gz] if self.lattice == D3Q19 else [])
        if all(isinstance(a, np.ndarray) for a in arrs):
            keep = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in arrs]
            dtype, where = F64, HOST
        else:
            torch = _torch()
            keep = [a.contiguous().reshape(-1) for a in arrs]
            dtype = {torch.float32: F32, torch.float64: F64}[keep[0].dtype]
            where = DEVICE if keep[0].is_cuda else HOST
        for a in keep:
            assert (a.size if isinstance(a, np.ndarray) else a.numel()) == self.n_nodes
        ptrs = [_ptr(a) for a in keep] + [None] * (3 - len(keep))
        self._check(self._lib.lwacm_set_force_field(self._h, *ptrs, dtype, where))
        if where == HOST:
            self._hold = keep  # host memory must outlive the asynchronous copy
            self.sync()
            self._hold = None
        else:
            for a in keep:  # the copy runs on the library's stream
                a.record_stream(self.stream)

    def set_scalar(self, T):
        """The passive scalar (needs scalar_alpha at construction; after set_fields):
        a numpy array (host, FP64) or a torch tensor (CUDA or host, FP32/FP64)."""
        torch = _torch()
        if isinstance(T, np.ndarray):
            keep = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
            dtype, where = F64, HOST
        else:
            keep = T.contiguous().reshape(-1)
            dtype = {torch.float32: F32, torch.float64: F64}[keep.dtype]
            where = DEVICE if keep.is_cuda else HOST
        assert (keep.size if isinstance(keep, np.ndarray) else keep.numel()) == self.n_nodes
        self._check(self._lib.lwacm_set_scalar(self._h, _ptr(keep), dtype, where))
        if where == HOST:
            self._hold = keep
            self.sync()
            self._hold = None
        else:
            keep.record_stream(self.stream)

    def get_scalar(self):
        """The passive scalar as an FP64 numpy array of the domain's shape."""
        out = np.empty(self.n_nodes, dtype=np.float64)
        self._check(self._lib.lwacm_get_scalar(self._h, out.ctypes.data, F64, HOST))
        return out.reshape(self.shape)

    def get_trace(self):
        """Tr^(+) - Tr^(e) of the bulk-viscosity variant (needs bulk_gamma at
        construction) as an FP64 numpy array of the domain's shape."""
        out = np.empty(self.n_nodes, dtype=np.float64)
        self._check(self._lib.lwacm_get_trace(self._h, out.ctypes.data, F64, HOST))
        return out.reshape(self.shape)

    def autotune(self, cache=None, steps=0):
        """lwacm_autotune: time the candidate kernel configurations and keep the
        fastest (call before set_fields). cache: path of the JSON cache or None.
        Returns the report as a dict."""
        import json
        buf = ctypes.create_string_buffer(16384)
        path = None if cache is None else str(cache).encode()
        self._check(self._lib.lwacm_autotune(self._h, path, int(steps), buf, len(buf)))
        return json.loads(buf.value.decode())

    def step(self, n=1):
        self._check(self._lib.lwacm_step(self._h, int(n)))

    def prepare(self, n):
        """Build the CUDA graph that step(n) would replay, without stepping."""
        self._check(self._lib.lwacm_prepare(self._h, int(n)))

    def sync(self):
        self._check(self._lib.lwacm_sync(self._h))
        self._pending = []  # the enqueued read-backs have landed

    def step_count(self):
        v = ctypes.c_longlong()
        self._check(self._lib.lwacm_step_count(self._h, ctypes.byref(v)))
        return v.value

    def get_fields(self, dtype=np.float64):
        """Current state copied to host numpy arrays (converted on the device)."""
        code = F64 if np.dtype(dtype) == np.float64 else F32
        outs = [np.empty(self.shape, dtype=np.float64 if code == F64 else np.float32)
                for _ in range(self.nf)]
        ptrs = [o.ctypes.data for o in outs] + [None] * (4 - self.nf)
        self._check(self._lib.lwacm_get_fields(self._h, *ptrs, code, HOST))
        return tuple(outs)

    def get_fields_into(self, outs, where=DEVICE):
        """Copy the current state into caller tensors/arrays (float32 or float64)."""
        torch = _torch()
        first = outs[0]
        if isinstance(first, np.ndarray):
            code = F64 if first.dtype == np.float64 else F32
        else:
            code = F64 if first.dtype == torch.float64 else F32
        ptrs = [_ptr(o) for o in outs] + [None] * (4 - len(outs))
        self._check(self._lib.lwacm_get_fields(self._h, *ptrs, code, where))

    def get_fields_async(self, outs, where=HOST):
        """As get_fields_into, only enqueued on this context's stream
        (lwacm_get_fields_async): host arrays (page-locked for overlap) hold the
        state once the stream has reached the copies (sync())."""
        torch = _torch()
        first = outs[0]
        if isinstance(first, np.ndarray):
            code = F64 if first.dtype == np.float64 else F32
        else:
            code = F64 if first.dtype == torch.float64 else F32
        ptrs = [_ptr(o) for o in outs] + [None] * (4 - len(outs))
        self._check(self._lib.lwacm_get_fields_async(self._h, *ptrs, code, where))
        # the destinations must outlive the copies: held until sync() or close()
        self._pending = getattr(self, "_pending", []) + [list(outs)]

    def fields(self):
        """Zero-copy torch views of the current state (storage dtype)."""
        torch = _torch()
        vp = [ctypes.c_void_p() for _ in range(4)]
        dt = ctypes.c_int()
        pitch = ctypes.c_longlong()
        self._check(self._lib.lwacm_fields(self._h, *[ctypes.byref(v) for v in vp],
                                           ctypes.byref(dt), ctypes.byref(pitch)))
        tdt = {F32: torch.float32, BF16: torch.bfloat16, F16: torch.float16}[dt.value]
        esz = 4 if dt.value == F32 else 2
        base = self.workspace.data_ptr()
        n = self.n_nodes
        views = []
        for k in range(self.nf):
            off = vp[k].value - base
            views.append(self.workspace[off:off + n * esz].view(tdt).view(self.shape))
        return tuple(views)

    # -- adjoint --
    def forward_record(self, T, stride=0):
        """Advance T steps keeping sqrt(T) checkpoints (lwacm_forward_record); the
        adjoint workspace is a torch tensor owned by this object."""
        torch = _torch()
        nb = ctypes.c_size_t()
        self._check(self._lib.lwacm_adjoint_workspace_bytes(self._h, int(T), int(stride),
                                                             ctypes.byref(nb)))
        if getattr(self, "adj_workspace", None) is None or self.adj_workspace.numel() < nb.value:
            self.adj_workspace = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        self._check(self._lib.lwacm_forward_record(self._h, int(T), int(stride),
                                                   self.adj_workspace.data_ptr(), nb.value))

    def backward(self, lam):
        """lam: dL/d(d, ux, uy[, uz]) at the end of the recorded run (CUDA tensors,
        float32 or float64). Returns (grads at the start, dL/dnu)."""
        torch = _torch()
        lam = [t.contiguous() for t in lam]
        code = F64 if lam[0].dtype == torch.float64 else F32
        outs = [torch.empty_like(t) for t in lam]
        ptrs_in = [t.data_ptr() for t in lam] + [None] * (4 - len(lam))
        ptrs_out = [t.data_ptr() for t in outs] + [None] * (4 - len(outs))
        g_nu = ctypes.c_double()
        self._check(self._lib.lwacm_backward(self._h, *ptrs_in, code, *ptrs_out, ctypes.byref(g_nu)))
        return tuple(outs), g_nu.value

    def diagnostics(self):
        out = (ctypes.c_double * 8)()
        st = self._lib.lwacm_diagnostics(self._h, out)
        res = {"mass": out[0], "jx": out[1], "jy": out[2], "jz": out[3], "ke": out[4],
               "umax": out[5], "mpar": out[6], "mperp": out[7], "finite": st != E_NONFINITE}
        if st not in (OK, E_NONFINITE):
            self._check(st)
        return res


class LwacmBatch(Lwacm):
    """Many independent periodic domains advanced together (lwacm_batch_create).

    dims: list of (nx, ny) for D2Q9 or (nx, ny, nz) for D3Q19; nus: viscosities.
    Fields are packed domain after domain; set_domains / get_domains pack and
    unpack per-domain numpy arrays. mode 0: one launch per step (graphs); mode 1:
    one persistent cooperative launch per step() call. tile: LWACM_OPT_BATCH_TILE
    (0 = runs of 256 nodes; 1..6 = the 2D shapes of BATCH_TILE_SHAPES, D2Q9).
    """

    def __init__(self, lattice, dims, nus, *, storage=F32, mode=0, tile=0, graph_chunk=None,
                 device=None, stream=None):
        lib = load()
        n = len(dims)
        self.lattice = int(lattice)
        self.dims = [tuple(int(v) for v in d) for d in dims]
        nx = (ctypes.c_int * n)(*[d[0] for d in self.dims])
        ny = (ctypes.c_int * n)(*[d[1] for d in self.dims])
        nz = (ctypes.c_int * n)(*[(d[2] if len(d) > 2 else 1) for d in self.dims])
        nu = (ctypes.c_double * n)(*[float(v) for v in nus])
        h = ctypes.c_void_p()
        st = lib.lwacm_batch_create(self.lattice, n, nx, ny, nz, nu, PERIODIC, ctypes.byref(h))
        if st != OK:
            raise LwacmError(st, "lwacm_batch_create")
        offs = (ctypes.c_longlong * (n + 1))()
        lib.lwacm_batch_offsets(h, offs)
        self.offsets = list(offs)
        self.n_nodes = self.offsets[-1]
        self.nx, self.ny, self.nz = self.n_nodes, 1, 1
        self.nu, self.bc = float(nus[0]), PERIODIC
        extra = {}
        if mode:
            extra[OPT_BATCH_MODE] = mode
        if tile:
            extra[OPT_BATCH_TILE] = tile
        self._setup(lib, h, storage, None, None, None, 0, graph_chunk, device, stream, extra)

    @property
    def shape(self):
        return (self.n_nodes,)

    def domain_shape(self, b):
        d = self.dims[b]
        return (d[1], d[0]) if self.lattice == D2Q9 else (d[2], d[1], d[0])

    def set_domains(self, fields):
        """fields: per domain a tuple (d, ux, uy[, uz]) of numpy arrays."""
        nf = 3 if self.lattice == D2Q9 else 4
        packed = [np.concatenate([np.asarray(f[k], dtype=np.float64).reshape(-1) for f in fields])
                  for k in range(nf)]
        self.set_fields(*packed)

    def get_domains(self):
        packed = self.get_fields()
        out = []
        for b in range(len(self.dims)):
            lo, hi = self.offsets[b], self.offsets[b + 1]
            out.append(tuple(p[lo:hi].reshape(self.domain_shape(b)) for p in packed))
        return out


def measure_fp32_peak(iters=4096, stream=None):
    """Measured FP32 FMA throughput of the current device: (TFLOP/s, ms of the
    timed launch). Runs the library's register-only FMA-chain kernel on `stream`
    (a torch.cuda.Stream, or the current stream) and waits for it."""
    torch = _torch()
    lib = load()
    st = stream if stream is not None else torch.cuda.current_stream()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib.lwacm_measure_fp32_peak(int(iters), ctypes.c_void_p(st.cuda_stream), ctypes.byref(tf),
                                     ctypes.byref(ms))
    if rc != OK:
        raise LwacmError(rc, "lwacm_measure_fp32_peak failed")
    return tf.value, ms.value


def _make_function():
    torch = _torch()

    class LwacmRun(torch.autograd.Function):
        """T LW-ACM steps as a differentiable function of the initial fields and nu.

        forward(sim, T, stride, nu, d0, ux0, uy0[, uz0]) -> (d, ux, uy[, uz]) after T
        steps (CUDA float32 tensors); backward uses the hand-written adjoint kernels
        with sqrt(T) checkpointing (lwacm_forward_record / lwacm_backward). `nu` is a
        0-d tensor equal to the simulation's viscosity; its gradient is dL/dnu.
        """

        @staticmethod
        def forward(ctx, sim, T, stride, nu, *fields):
            sim.set_fields(*[f.detach().to(torch.float32) for f in fields])
            sim.forward_record(int(T), int(stride))
            outs = [torch.empty(sim.shape, dtype=torch.float32, device=sim.device)
                    for _ in range(sim.nf)]
            sim.get_fields_into(outs, DEVICE)
            ctx.sim = sim
            ctx.nu_dtype = nu.dtype if torch.is_tensor(nu) else torch.float64
            return tuple(outs)

        @staticmethod
        def backward(ctx, *grads):
            sim = ctx.sim
            lam = [g if g is not None else torch.zeros(sim.shape, device=sim.device)
                   for g in grads]
            lam = [g.to(torch.float32).contiguous() for g in lam]
            gfields, g_nu = sim.backward(lam)
            return (None, None, None, torch.tensor(g_nu, dtype=ctx.nu_dtype), *gfields)

    return LwacmRun


_LwacmRun = None


def run(sim, T, nu, *fields, stride=0):
    """Differentiable T-step run: returns the fields after T steps; gradients flow
    to `fields` and to the 0-d tensor `nu` (which must equal the sim's viscosity)."""
    global _LwacmRun
    if _LwacmRun is None:
        _LwacmRun = _make_function()
    return _LwacmRun.apply(sim, T, stride, nu, *fields)
