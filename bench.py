"""Benchmark: LW-ACM D3Q19 update on a 256^3 periodic 3D Taylor-Green vortex, FP32.

One bench "step" is one LW-ACM time step over the whole 256^3 lattice
(16.8 M node updates). Prints one JSON line (rank 0):

  value      GLUPS (10^9 node updates / s), inputs resident in HBM, CUDA events on
             the library's stream around exactly K steps, max over ranks;
  e2e        the same metric through the C ABI with host buffers: each step
             copies the fields of one 256^3 problem in from pinned host memory
             (lwacm_set_fields), advances it one step and copies the fields back
             (lwacm_get_fields_async); consecutive steps rotate over three
             contexts on three streams (three independent problems), so that one
             problem's copy back overlaps the next ones' copies in;
  roofline   the dominant kernel (the interior update) against the measured HBM
             copy bandwidth: 32 algorithmic bytes per node (4 FP32 fields read
             once, written once);
  cpu_baseline  the FP64 oracle timed on the host cores on a bounded sample (1000
             steps of the workload's vortex on 128^3);
  accuracy   the same 1000 steps through the benchmarked kernel against the
             oracle: per-field errors and the kinetic-energy curve.

--impl reference times the FP64 oracle (the plain CPU restatement of the
method) on the same workload, metric and unit.
Multi-GPU: one independent 256^3 domain per rank (replicas; no data-path
collective), value = all ranks' node updates / max time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_SIDE = 256
U0, NU = 0.02, 0.005
BYTES_PER_NODE = 32  # FP32 (d, ux, uy, uz): read once, written once
FLOPS_PER_NODE = 146  # FP32 operations of the moment form per D3Q19 node update (FMA = 2)
WORKLOAD = "D3Q19 3D Taylor-Green 256^3 periodic, u0=0.02, nu=0.005, FP32 fields (d=rho-1, ux, uy, uz)"
METRIC = "GLUPS, D3Q19 256^3 FP32 LW-ACM update"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to a scratch file; the JSON line carries their summary
        self.path = os.path.join(os.environ.get("LWACM_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"lwacm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    try:
                        rows.append((float(p[1]), float(p[2]), p[5:9]))
                    except ValueError:
                        pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags)
                          if f.lower() == "active"})
        sm = [r[0] for r in rows]
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


ACC_SIDE, ACC_EVERY = 128, 10  # the accuracy sample: the workload's parameters on 128^3


def cpu_baseline(steps=1000, n=ACC_SIDE, every=ACC_EVERY):
    """The FP64 oracle as it stands on the host cores, timed on a bounded sample:
    `steps` updates of the Taylor-Green workload (same u0, nu) on n^3, in runs of
    `every` steps (only the updates are timed). The same run on the GPU, through
    the benchmarked kernel from the same FP32-rounded fields, is compared with it:
    the per-field errors after `steps` steps and the kinetic energy every `every`
    steps (the metric's stated error), and the same for FP16 storage rounded
    stochastically. Returns (cpu_baseline, accuracy)."""
    import numpy as np
    import oracle
    from paper_1111_2142_gb300 import inputs
    from paper_1111_2142_gb300 import lwacm as lw
    f32 = [a.astype(np.float32).astype(np.float64) for a in inputs.tgv3d(n, u0=U0)]

    def gpu(**kw):
        sim = lw.Lwacm(lw.D3Q19, n, n, n, NU, **kw)
        sim.set_fields(*f32)
        ke = [sim.diagnostics()["ke"]]
        for _ in range(steps // every):
            sim.step(every)
            ke.append(sim.diagnostics()["ke"])
        out = [a.reshape(n, n, n) for a in sim.get_fields()]
        name = sim.kernel_name
        sim.close()
        return out, np.array(ke), name

    got, ke_gpu, kname = gpu()
    got16, ke16, _ = gpu(storage=lw.F16, stochastic_rounding=True)
    oracle.step(19, *[a[:8] for a in f32], nu=NU, nsteps=1)  # load/build outside the timing
    state = tuple(f32)
    ke_ref = [oracle.diagnostics(*state)["ke"]]
    dt = 0.0
    for _ in range(steps // every):
        t0 = time.perf_counter()
        state = oracle.step(19, *state, nu=NU, nsteps=every)
        dt += time.perf_counter() - t0
        ke_ref.append(oracle.diagnostics(*state)["ke"])
    ke_ref = np.array(ke_ref)
    done = (steps // every) * every
    base = {"value": done * n ** 3 / dt / 1e9, "unit": "GLUPS", "cores": oracle.max_threads(),
            "kind": "oracle", "sample": f"{done} FP64 oracle steps of the workload's Taylor-Green vortex "
            f"on {n}^3 ({dt:.1f} s)"}

    def errs(g, ke):
        dscale = max(float(np.max(np.abs(state[0]))), 3 * U0 ** 2)
        return {"max_abs_du_over_u0": max(float(np.max(np.abs(a - b))) for a, b in zip(g[1:], state[1:])) / U0,
                "max_abs_dd_over_dscale": float(np.max(np.abs(g[0] - state[0]))) / dscale,
                "ke_curve_max_rel": float(np.max(np.abs(ke - ke_ref) / ke_ref))}
    acc = {"workload": f"D3Q19 3D Taylor-Green {n}^3, u0={U0}, nu={NU}, {done} steps, KE every {every}",
           "kernel": kname, "fp32": errs(got, ke_gpu), "fp16_stochastic_rounding": errs(got16, ke16),
           "ke_ratio_oracle": float(ke_ref[-1] / ke_ref[0]), "reference": "FP64 oracle"}
    return base, acc


REF_SIDE = 128  # the reference arm's bounded sample: the same workload on 128^3


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_1111_2142_gb300 import inputs
    n = REF_SIDE
    f = inputs.tgv3d(n, u0=U0)
    oracle.step(19, *[a[:8] for a in f], nu=NU, nsteps=1)
    # each reference "step" is one FP64 oracle update of a 128^3 Taylor-Green lattice
    # with the benchmark's parameters (a bounded sample of the 256^3 workload; the
    # oracle's per-node cost does not depend on the lattice size)
    state = oracle.step(19, *f, nu=NU, nsteps=args.warmup)
    t0 = time.perf_counter()
    oracle.step(19, *state, nu=NU, nsteps=args.steps)  # one call: K updates
    dt = time.perf_counter() - t0
    v = args.steps * n ** 3 / dt / 1e9
    cores = oracle.max_threads()
    # the oracle runs on the host cores of rank 0; n_gpus echoes the launch
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (FP64 oracle)"},
            "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed FP64 oracle steps of the workload "
                                       f"on a {n}^3 lattice (same u0, nu)"},
            "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _events_ms(stream, fn):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


KERNEL_SOURCES = {
    "half_d3q19_tma": ("kernels_half.cu", "tile_common.cuh", "lwacm_core.cuh"),
}


def _kernel_source_hash(kname):
    """SHA-256 over the CUDA sources of an interior kernel: stored ncu traffic is
    used only while it matches the kernel as built."""
    import hashlib
    files = KERNEL_SOURCES.get(kname)
    if not files:
        return None
    h = hashlib.sha256()
    for fn in files:
        with open(os.path.join(ROOT, "paper_1111_2142_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def variants(hbm):
    """The other configurations and forms, each timed with CUDA events on its own
    stream after a warm-up: storage modes and kernels for the 256^3 workload, the
    batched ensemble (persistent launch / per-step graphs / per-domain launches),
    the adjoint at 128^3, the 1024^2 cavity and the 64^2 2D Taylor-Green vortex."""
    import torch
    from paper_1111_2142_gb300 import inputs
    from paper_1111_2142_gb300 import lwacm as lw
    out = {}

    def glups(nodes, steps, ms):
        return nodes * steps / (ms * 1e-3) / 1e9

    n = N_SIDE
    f = inputs.tgv3d(n, u0=U0)
    for name, kw, bpn in (("d3q19_256_bf16_storage", dict(storage=lw.BF16), 16),
                          ("d3q19_256_fp16_storage", dict(storage=lw.F16), 16),
                          ("d3q19_256_fp16_stochastic_rounding", dict(storage=lw.F16, stochastic_rounding=True), 16),
                          ("d3q19_256_bf16_stochastic_rounding", dict(storage=lw.BF16, stochastic_rounding=True), 16),
                          ("d3q19_256_generic_kernel", dict(kernel=1), 32)):
        sim = lw.Lwacm(lw.D3Q19, n, n, n, NU, **kw)
        sim.set_fields(*f)
        sim.step(20)
        steps = 400
        sim.prepare(steps)
        ms = _events_ms(sim.stream, lambda: sim.step(steps))
        g = glups(n ** 3, steps, ms)
        out[name] = {"value": g, "unit": "GLUPS", "kernel": sim.kernel_name,
                     "hbm_frac": bpn * g / hbm, "bytes_per_node": bpn}
        sim.close()
        torch.cuda.empty_cache()
    # rows longer than 256: the half-row kernel on 128-node segments, and the generic kernel
    sx, sy, sz = 384, 256, 256
    fs = inputs.tgv3d(sx, u0=U0, ny=sy, nz=sz)
    seg = {"shape": [sx, sy, sz], "unit": "GLUPS", "bytes_per_node": 32}
    for label, kw in (("segments", {}), ("generic_kernel", dict(kernel=1))):
        sim = lw.Lwacm(lw.D3Q19, sx, sy, sz, NU, **kw)
        sim.set_fields(*fs)
        sim.step(20)
        sim.prepare(300)
        ms = _events_ms(sim.stream, lambda: sim.step(300))
        seg[label] = glups(sx * sy * sz, 300, ms)
        seg[label + "_kernel"] = sim.kernel_name
        sim.close()
        torch.cuda.empty_cache()
    seg["hbm_frac"] = 32 * seg["segments"] / hbm
    out["d3q19_384x256x256"] = seg

    # batched ensemble: 256 D2Q9 domains (seed 1), 2000 steps
    doms = inputs.ensemble_2d(256, seed=1)
    dims = [(d["nx"], d["ny"]) for d in doms]
    nus = [d["nu"] for d in doms]
    fields = [(d["d"], d["ux"], d["uy"]) for d in doms]
    nodes = sum(a * b for a, b in dims)
    T = 2000
    ens = {"domains": 256, "nodes": nodes, "steps": T}
    for mode, label in ((1, "persistent_launch"), (0, "per_step_graphs")):
        sim = lw.LwacmBatch(lw.D2Q9, dims, nus, mode=mode)
        sim.set_domains(fields)
        sim.step(10)
        sim.prepare(T)
        ms = _events_ms(sim.stream, lambda: sim.step(T))
        ens[label] = glups(nodes, T, ms)
        sim.close()
    # the autotuner's choice among the tile layouts and launch forms
    sim = lw.LwacmBatch(lw.D2Q9, dims, nus)
    rep = sim.autotune(steps=256)
    sim.set_domains(fields)
    sim.step(10)
    sim.prepare(T)
    ms = _events_ms(sim.stream, lambda: sim.step(T))
    ens["autotuned"] = {"value": glups(nodes, T, ms), "kernel": sim.kernel_name,
                        "candidates": {c["name"]: round(nodes / c["us_per_step"] / 1e3, 2)
                                       for c in rep["candidates"]}}
    sim.close()
    # per-domain launches: one context per domain, each stepped on its own
    sims = []
    for (nx, ny), nu_b, fb in zip(dims, nus, fields):
        s_ = lw.Lwacm(lw.D2Q9, nx, ny, 1, nu_b)
        s_.set_fields(*fb)
        sims.append(s_)
    Tpd = 200
    for s_ in sims:
        s_.step(2)
    ms = _events_ms(sims[0].stream, lambda: [s_.step(Tpd) for s_ in sims])
    ens["per_domain_launches"] = glups(nodes, Tpd, ms)
    ens["per_domain_steps"] = Tpd
    ens["unit"] = "GLUPS"
    for s_ in sims:
        s_.close()
    out["ensemble_256_d2q9"] = ens

    # adjoint: D3Q19 128^3, T = 500, sqrt(T) checkpoints
    n3, T3 = 128, 500
    fa = inputs.random_divfree_3d(n3, n3, n3, rms=0.03, kmax=8, seed=2)
    sim = lw.Lwacm(lw.D3Q19, n3, n3, n3, 0.01)
    sim.set_fields(*fa)
    sim.step(10)
    sim.prepare(T3)
    ms_fwd = _events_ms(sim.stream, lambda: sim.step(T3))
    sim.set_fields(*fa)
    ms_rec = _events_ms(sim.stream, lambda: sim.forward_record(T3))
    lam = [torch.zeros((n3, n3, n3), device="cuda")] + [
        torch.tensor(a, dtype=torch.float32, device="cuda") for a in fa[1:]]
    ms_bwd = _events_ms(sim.stream, lambda: sim.backward(lam))
    # with every state of the run kept (stride = T: 502 states of 33.5 MB, 16.8 GB),
    # the backward sweep recomputes nothing
    sim.set_fields(*fa)
    ms_rec_all = _events_ms(sim.stream, lambda: sim.forward_record(T3, stride=T3))
    ms_bwd_all = _events_ms(sim.stream, lambda: sim.backward(lam))
    out["adjoint_d3q19_128_T500"] = {
        "forward_glups": glups(n3 ** 3, T3, ms_fwd),
        "recorded_forward_glups": glups(n3 ** 3, T3, ms_rec),
        "backward_glups_equiv": glups(n3 ** 3, T3, ms_bwd),
        "backward_over_forward_time": ms_bwd / ms_fwd, "checkpoints": "sqrt(T)",
        "all_states_kept": {"recorded_forward_glups": glups(n3 ** 3, T3, ms_rec_all),
                            "backward_glups_equiv": glups(n3 ** 3, T3, ms_bwd_all),
                            "backward_over_forward_time": ms_bwd_all / ms_fwd},
        "unit": "GLUPS", "kernel_forward": sim.kernel_name}
    sim.close()
    torch.cuda.empty_cache()

    out["cavity_d2q9_1024"] = cavity_1024(glups)

    # 2D Taylor-Green 64^2
    sim = lw.Lwacm(lw.D2Q9, 64, 64, 1, 0.01)
    sim.set_fields(*inputs.tgv2d(64, u0=0.01))
    sim.step(64)
    ms = _events_ms(sim.stream, lambda: sim.step(6400))
    out["tgv_d2q9_64"] = {"value": glups(64 ** 2, 6400, ms), "unit": "GLUPS",
                          "kernel": sim.kernel_name, "l2_resident": True}
    sim.close()
    out["next_rows"] = next_rows(hbm, glups)
    return out


def cavity_1024(glups, steps=200000, chunk=1000):
    """The 2D lid-driven cavity as configured (Section 2.6.1 wall rules): 1024^2,
    lid speed U = 0.1, Re = U N / nu = 1000 (nu = 0.1024), from rest for 200,000
    steps (about 20 lid travel times) in CUDA-graph chunks of 1000 steps, timed as
    one run. Reports the centreline profiles u(x = N/2, y) and v(x, y = N/2) (the
    mean of the two node columns / rows either side of the centre, every 32nd
    node, in units of U) and how much the field still changed over the last
    1000 steps."""
    import numpy as np
    import torch
    from paper_1111_2142_gb300 import lwacm as lw
    n, U = 1024, 0.1
    nu = U * n / 1000.0
    z = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    sim = lw.Lwacm(lw.D2Q9, n, n, 1, nu, lw.CAVITY, lid=(U, 0.0), graph_chunk=chunk)
    sim.set_fields(z, z, z)
    sim.step(2 * chunk)  # warm-up: builds the graphs
    sim.set_fields(z, z, z)
    ms = _events_ms(sim.stream, lambda: sim.step(steps - chunk))
    prev = [a.reshape(n, n) for a in sim.get_fields()]
    ms += _events_ms(sim.stream, lambda: sim.step(chunk))
    d, u, v = [a.reshape(n, n) for a in sim.get_fields()]
    kname = sim.kernel_name
    sim.close()
    h = n // 2
    ucl = 0.5 * (u[:, h - 1] + u[:, h]) / U  # u along y at the vertical centreline
    vcl = 0.5 * (v[h - 1, :] + v[h, :]) / U  # v along x at the horizontal centreline
    idx = list(range(0, n, 32)) + [n - 1]
    return {"value": glups(n * n, steps, ms), "unit": "GLUPS", "steps": steps, "gpu_seconds": ms * 1e-3,
            "kernel": kname + ("+wall_pass" if kname.startswith("generic") else ""), "l2_resident": True,
            "re": 1000, "lid": U, "nu": nu,
            "last_1000_steps_max_change_over_U": float(max(np.max(np.abs(u - prev[1])),
                                                             np.max(np.abs(v - prev[2]))) / U),
            "centreline_nodes": idx,
            "u_over_U_at_x_centre": [round(float(ucl[i]), 5) for i in idx],
            "v_over_U_at_y_centre": [round(float(vcl[i]), 5) for i in idx],
            "u_min_over_U": float(ucl.min()), "v_max_over_U": float(vcl.max()), "v_min_over_U": float(vcl.min())}


def next_rows(hbm, glups):
    """The variants beyond the plain scheme, each on a workload larger than L2 (HBM
    fractions against the bytes each node moves per step), plus the Section 3.2
    shear layer at its own 128^2 size: the 3D diagonally driven cavity (walls), the
    forced Taylor-Green vortex (a per-node force field), omega_p, the bulk-viscosity
    variant, the semi-implicit pressure update and the passive scalar."""
    import torch
    from paper_1111_2142_gb300 import inputs
    from paper_1111_2142_gb300 import lwacm as lw
    out = {}

    def timed(name, sim, fields, steps, nodes, bpn, extra=None):
        sim.set_fields(*fields)
        if extra:
            extra(sim)
        sim.step(8)
        sim.prepare(steps)
        ms = _events_ms(sim.stream, lambda: sim.step(steps))
        g = glups(nodes, steps, ms)
        out[name] = {"value": g, "unit": "GLUPS", "kernel": sim.kernel_name, "hbm_frac": bpn * g / hbm,
                     "bytes_per_node": bpn}
        sim.close()
        torch.cuda.empty_cache()

    n3 = 256
    z3 = torch.zeros((n3, n3, n3), dtype=torch.float32, device="cuda")
    lid = (2 ** 0.5 / 20, 2 ** 0.5 / 20, 0.0)
    timed("cavity3d_d3q19_256", lw.Lwacm(lw.D3Q19, n3, n3, n3, 0.01, lw.CAVITY, lid=lid), (z3, z3, z3, z3),
          100, n3 ** 3, 32)
    timed("cavity3d_d3q19_256_bf16", lw.Lwacm(lw.D3Q19, n3, n3, n3, 0.01, lw.CAVITY, lid=lid, storage=lw.BF16),
          (z3, z3, z3, z3), 100, n3 ** 3, 16)
    f3 = inputs.tgv3d(n3, u0=U0)
    t3 = torch.cos(2 * torch.pi * torch.arange(n3, device="cuda") / n3).expand(n3, n3, n3).contiguous()
    timed("scalar_d3q19_256", lw.Lwacm(lw.D3Q19, n3, n3, n3, NU, scalar_alpha=0.01), f3, 100, n3 ** 3, 40,
          extra=lambda s: s.set_scalar(t3))
    # a constant acceleration (Eq. force) on the 256^3 Taylor-Green workload (half-row kernel)
    timed("forced_d3q19_256", lw.Lwacm(lw.D3Q19, n3, n3, n3, NU, force=(1e-6, 0.0, 0.0)), f3, 200, n3 ** 3, 32)
    # omega_p on the 256^3 Taylor-Green workload: the density-term pass (reads the state,
    # writes one FP32 field) and the half-row kernel (reads that field too): 52 B/node
    sim = lw.Lwacm(lw.D3Q19, n3, n3, n3, NU)
    sim.set_option(lw.OPT_NU_P, 0.05)
    timed("nu_p_d3q19_256", sim, f3, 200, n3 ** 3, 52)
    del z3, t3
    n2 = 4096
    f2 = inputs.gtg_state(n2, 0.0)
    gx, gy = inputs.gtg_force(n2, 0.0)
    timed("forced_tgv_d2q9_4096", lw.Lwacm(lw.D2Q9, n2, n2, 1, inputs.GTG_NU, force_field=True), f2, 200,
          n2 ** 2, 32, extra=lambda s: s.set_force_field(gx, gy))
    sim = lw.Lwacm(lw.D2Q9, n2, n2, 1, 0.01)
    sim.set_option(lw.OPT_NU_P, 0.1)
    timed("nu_p_d2q9_4096", sim, f2, 200, n2 ** 2, 24)
    timed("bulk_d2q9_4096", lw.Lwacm(lw.D2Q9, n2, n2, 1, 0.01, bulk_gamma=0.4), f2, 200, n2 ** 2, 32)
    # semi-implicit pressure update: the explicit step (24 B/node) plus the density pass
    # (old density and new velocity read, new density written: 16 B/node)
    timed("semi_implicit_d2q9_4096", lw.Lwacm(lw.D2Q9, n2, n2, 1, 0.01, semi_implicit=True), f2, 200, n2 ** 2,
          40)
    # Section 3.2 shear layer, 128^2 to t = 1 (3200 steps): plain and nu_p = 170 nu (L2-resident)
    nu, steps = inputs.minion_brown_lattice(128)
    fm = inputs.minion_brown(128)
    for name, nu_p, gamma in (("shear_layer_d2q9_128", None, None), ("shear_layer_nu_p_d2q9_128", 170 * nu, None),
                              ("shear_layer_nu_p_bulk_d2q9_128", 170 * nu, 0.4)):
        sim = lw.Lwacm(lw.D2Q9, 128, 128, 1, nu, bulk_gamma=gamma)
        if nu_p:
            sim.set_option(lw.OPT_NU_P, nu_p)
        sim.set_fields(*fm)
        sim.prepare(steps)  # graph capture outside the time to t = 1
        ms = _events_ms(sim.stream, lambda: sim.step(steps))
        out[name] = {"value": glups(128 ** 2, steps, ms), "unit": "GLUPS", "kernel": sim.kernel_name,
                     "ms_to_t1": ms, "l2_resident": True}
        sim.close()
    return out


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1111_2142_gb300 import inputs
    from paper_1111_2142_gb300 import lwacm as lw

    n = N_SIDE
    f = inputs.tgv3d(n, u0=U0)
    sim = lw.Lwacm(lw.D3Q19, n, n, n, NU, graph_chunk=args.graph_chunk, kernel=args.kernel)
    sim.set_fields(*f)
    stream = sim.stream
    N = n ** 3

    # warm-up (also builds the CUDA graph)
    sim.step(args.warmup)
    sim.prepare(args.steps)  # the CUDA graph the timed steps replay, captured outside the timing
    torch.cuda.synchronize()

    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()

    from paper_1111_2142_gb300.shard import aggregate_throughput
    units, t_max_s = aggregate_throughput(args.steps * N, ms * 1e-3, device="cuda")
    t_max = t_max_s * 1e3
    glups = units / t_max_s / 1e9
    ms_step = t_max / args.steps
    diag = sim.diagnostics()

    # roofline of the interior kernel: one launch per step for a periodic domain
    hbm, src = _peaks()
    achieved = BYTES_PER_NODE * N / (ms_step * 1e-3) / 1e9
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic_d3q19_256.json")
    if os.path.exists(tf):
        try:
            with open(tf) as fh:
                tj = json.load(fh)
            if tj.get("kernel") == sim.kernel_name and tj.get("source_sha256") == _kernel_source_hash(
                    sim.kernel_name):
                traffic = tj.get("bytes_per_launch")
        except Exception:
            traffic = None

    # the FP32 compute roof, measured on this GPU (register-only FMA chains)
    try:
        fp32_tflops, fp32_ms = lw.measure_fp32_peak(4096, sim.stream)
    except Exception:
        fp32_tflops, fp32_ms = None, None
    fp32_achieved = FLOPS_PER_NODE * N / (ms_step * 1e-3) / 1e12

    # end-to-end through the C ABI with pinned host buffers: three independent
    # problems on three contexts (three streams), one step each in turn
    e2e_steps = max(3, min(args.e2e_steps, args.steps))
    extra = [lw.Lwacm(lw.D3Q19, n, n, n, NU, graph_chunk=args.graph_chunk, kernel=args.kernel,
                      stream=torch.cuda.Stream()) for _ in range(2)]
    e2e_sims = [sim] + extra
    ns = len(e2e_sims)
    host_in = [[torch.from_numpy(a.astype(np.float32)).pin_memory() for a in f] for _ in e2e_sims]
    host_out = [[torch.empty_like(h).pin_memory() for h in hi] for hi in host_in]
    ptr_in = [[h.data_ptr() for h in hi] for hi in host_in]
    lib = lw.load()

    def e2e_step(k):
        s = e2e_sims[k % ns]
        s._check(lib.lwacm_set_fields(s._h, *ptr_in[k % ns], lw.F32, lw.HOST))
        s._check(lib.lwacm_step(s._h, 1))
        s.get_fields_async(host_out[k % ns], lw.HOST)

    for k in range(ns):
        e2e_step(k)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier()
    e2e_units, e2e_s = aggregate_throughput(e2e_steps * N, time.perf_counter() - t0, device="cuda")
    e2e_glups = e2e_units / e2e_s / 1e9
    for s in extra:
        s.close()
    field_bytes = 4 * N * 4

    line = {
        "metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nodes_per_gpu": N, "parallelism": f"replicas x{ws}",
                   "kernel": sim.kernel_name,
                   "l2": "inputs larger than L2 (2 ping-pong buffers of 268 MB)",
                   "graph_chunk": args.graph_chunk},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "peak_source": f"{src} hbm_gbs (copy test)",
                     "bytes_per_node": BYTES_PER_NODE,
                     "fp32": {"flops_per_node": FLOPS_PER_NODE, "achieved": fp32_achieved,
                              "peak": fp32_tflops, "unit": "TFLOP/s",
                              "frac": fp32_achieved / fp32_tflops if fp32_tflops else None,
                              "peak_source": "measured: FMA-chain kernel (lwacm_measure_fp32_peak)"}},
        "e2e": {"value": e2e_glups, "unit": "GLUPS", "h2d_bytes_per_step": field_bytes,
                "d2h_bytes_per_step": field_bytes, "steps": e2e_steps,
                "pipeline": "3 independent problems on 3 contexts/streams, one step each in turn"},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "check": {"mass": diag["mass"], "ke": diag["ke"], "finite": diag["finite"]},
    }
    if rank == 0 and not args.no_variants and ws == 1:
        line["variants"] = variants(hbm)
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        try:
            line["cpu_baseline"], line["accuracy"] = cpu_baseline(args.cpu_steps)
        except Exception as exc:  # the oracle is a reported baseline, not a requirement
            line["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_case(name, steps):
    """One variant workload, stepped without timing (a target for profilers)."""
    import torch
    from paper_1111_2142_gb300 import inputs
    from paper_1111_2142_gb300 import lwacm as lw
    if name == "adjoint":  # D3Q19 128^3: recorded forward + backward over `steps` steps
        n3 = 128
        fa = inputs.random_divfree_3d(n3, n3, n3, rms=0.03, kmax=8, seed=2)
        sim = lw.Lwacm(lw.D3Q19, n3, n3, n3, 0.01)
        sim.set_fields(*fa)
        sim.forward_record(steps)
        lam = [torch.zeros((n3, n3, n3), device="cuda")] + [
            torch.tensor(a, dtype=torch.float32, device="cuda") for a in fa[1:]]
        sim.backward(lam)
    elif name == "ensemble":  # 256 D2Q9 domains (seed 1), 2D tiles 30x14
        doms = inputs.ensemble_2d(256, seed=1)
        sim = lw.LwacmBatch(lw.D2Q9, [(d["nx"], d["ny"]) for d in doms], [d["nu"] for d in doms], tile=2)
        sim.set_domains([(d["d"], d["ux"], d["uy"]) for d in doms])
        sim.step(steps)
    elif name == "cavity":  # D2Q9 1024^2 lid-driven cavity, Re 1000, from rest
        z = torch.zeros((1024, 1024), dtype=torch.float32, device="cuda")
        sim = lw.Lwacm(lw.D2Q9, 1024, 1024, 1, 0.1024, lw.CAVITY, lid=(0.1, 0.0))
        sim.set_fields(z, z, z)
        sim.step(steps)
    elif name == "cavity3d":  # D3Q19 256^3 diagonally driven cavity from rest (half-row kernel + walls)
        z = torch.zeros((256, 256, 256), dtype=torch.float32, device="cuda")
        sim = lw.Lwacm(lw.D3Q19, 256, 256, 256, 0.01, lw.CAVITY, lid=(2 ** 0.5 / 20, 2 ** 0.5 / 20, 0.0))
        sim.set_fields(z, z, z, z)
        sim.step(steps)
    elif name == "scalar":  # D3Q19 256^3 Taylor-Green with a passive scalar (half-row + scalar row kernels)
        n3 = 256
        sim = lw.Lwacm(lw.D3Q19, n3, n3, n3, NU, scalar_alpha=0.01)
        sim.set_fields(*inputs.tgv3d(n3, u0=U0))
        sim.set_scalar(torch.cos(2 * torch.pi * torch.arange(n3, device="cuda") / n3).expand(n3, n3, n3).contiguous())
        sim.step(steps)
    elif name == "nu_p3d":  # D3Q19 256^3 Taylor-Green with omega_p (density pass + half-row kernel)
        sim = lw.Lwacm(lw.D3Q19, 256, 256, 256, NU)
        sim.set_option(lw.OPT_NU_P, 0.05)
        sim.set_fields(*inputs.tgv3d(256, u0=U0))
        sim.step(steps)
    elif name == "segments":  # D3Q19 384 x 256 x 128 Taylor-Green (half-row kernel on 128-node segments)
        sim = lw.Lwacm(lw.D3Q19, 384, 256, 128, NU)
        sim.set_fields(*inputs.tgv3d(384, u0=U0, ny=256, nz=128))
        sim.step(steps)
    elif name == "bulk2d":  # D2Q9 4096^2 bulk-viscosity variant, gamma 0.4 (2D tiles 30x14)
        sim = lw.Lwacm(lw.D2Q9, 4096, 4096, 1, 0.01, bulk_gamma=0.4)
        sim.set_fields(*inputs.gtg_state(4096, 0.0))
        sim.step(steps)
    else:
        raise SystemExit(f"unknown case {name}")
    sim.sync()
    sim.close()
    print(json.dumps({"case": name, "steps": steps, "done": True}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--graph-chunk", type=int, default=64)
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=90)
    ap.add_argument("--cpu-steps", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--profile-case", choices=["adjoint", "ensemble", "cavity", "cavity3d", "bulk2d", "scalar",
                                               "segments", "nu_p3d"],
                    help="run one variant workload for --steps steps without timing (for profilers)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__
    __graft_entry__.build()
    if args.profile_case:
        return run_case(args.profile_case, args.steps)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
