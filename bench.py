"""Benchmark: DOF-stage updates/s of the tree-based dGSEM hot path on one GB300.

A step is one SSP-RK3 step (three fused RHS+stage launches plus the mortar launches) on the 3D
octree warm-bubble workload (16^3 roots, N = 7, two extra levels where |theta'| > 0.05 K,
dt = 0.005 s), with the regrid (indicator, host tree, conservative transfer) every 20 steps
inside the timed region.  DOF-stage updates = nodes per variable x 3 stages per step.

The main line is the FP32-perturbation path; the FP64 path is measured in the same run and
reported under "fp64".  With --impl reference the oracle (plain NumPy FP64) is timed on the
host cores on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "DOF-stage updates/s"
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, gpu_index, log_dir=None):
        import tempfile
        self.proc = None
        d = log_dir if log_dir else tempfile.gettempdir()
        self.path = os.path.join(d, "clocks_rank%d_%d.csv" % (gpu_index, os.getpid()))
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + CLOCK_QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # the timed region starts only once nvidia-smi has produced its first sample
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier_max(t, world, device="cuda"):
    """Maximum over ranks of a time (the slowest rank defines the job time)."""
    if world == 1:
        return t
    import torch
    import torch.distributed as dist
    x = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


STAGE_KERNEL = None   # None: library default; 0 column layout; 1 node-per-thread layout


def build_mesh(pkg, cfg, precision):
    m = pkg.Mesh(cfg["dim"], cfg["N"], cfg["base"], cfg["length"], max_level=cfg["max_level"],
                 precision=precision)
    if STAGE_KERNEL is not None:
        m.set_stage_kernel(STAGE_KERNEL)
    pkg.adapt_initial(m, cfg["bubble"], cfg["threshold"], cfg["buffer"])
    return m


def measured_traffic(D, N, precision, layout):
    """DRAM bytes per node of each stage launch from the committed ncu record, if that record
    was taken on the current kernel sources and configuration; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "stage_traffic_bubble3d_N7.json")
    try:
        rec = json.load(open(path))
    except OSError:
        return None
    if (D, N, precision, layout) != (3, 7, "fp32", rec.get("layout", 2)):
        return None
    h = hashlib.sha1()
    for f in rec["sources"]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != rec["sources_sha1"]:
        return None
    b = rec["bytes_per_node"]
    return [b["stage1"], b["stage2"], b["stage3"]]


def stage_bytes(E, NP, NV, b, n1, D):
    """Algorithmic HBM bytes of the three stage launches of one RK3 step: stage 1 reads q^n and
    writes q^1; stages 2 and 3 read q^s and q^n and write the next state; every launch reads
    the per-element tables (FP64 background column, level/coordinates, face connectivity)."""
    nodes = E * NP
    per_elem = n1 * 4 * 8 + 16 + 2 * D * 5 * 4
    return nodes * NV * b * (2 + 3 + 3) + 3 * E * per_elem


def stage_flops(E, NP, NV, n1, D):
    """Algorithmic flops of the three stage launches of one RK3 step: the sum-factorised
    derivative (2 NV D (N+1) per node), the D flux evaluations (D (D + 6) per node) and the
    stage combination (4 NV per node); transcendental functions and face terms not counted."""
    per_node = 2 * NV * D * n1 + D * (D + 6) + 4 * NV
    return 3 * E * NP * per_node


def paired_meshes(pkg, cfg):
    """An FP64 and an FP32-perturbation mesh of the workload with identical trees: the initial
    adaptation is driven by the FP64 mesh's theta' indicator and applied to both as flags."""
    import numpy as np
    ms = [pkg.Mesh(cfg["dim"], cfg["N"], cfg["base"], cfg["length"], max_level=cfg["max_level"],
                   precision=p) for p in ("fp64", "fp32")]
    if STAGE_KERNEL is not None:
        for m in ms:
            m.set_stage_kernel(STAGE_KERNEL)
    for _ in range(cfg["max_level"]):
        ms[0].set_bubble(**cfg["bubble"])
        flags = (ms[0].indicator() > cfg["threshold"]).astype(np.uint8)
        for m in ms:
            m.adapt(flags=flags, buffer=cfg["buffer"])
    for m in ms:
        m.set_bubble(**cfg["bubble"])
    return ms


def fp32_accuracy(pkg, cfg, steps):
    """FP32-perturbation path against the FP64 path after `steps` SSP-RK3 steps of the workload,
    regridding both every `regrid_every` steps with the FP64 mesh's flags so that the trees stay
    identical.  Returns max |theta' error| (K), max |w error| (m/s), the relative differences of
    total mass and energy, and each path's relative mass change over the run."""
    import numpy as np
    import torch
    m64, m32 = paired_meshes(pkg, cfg)
    I0 = [m.integrals() for m in (m64, m32)]
    every = cfg.get("regrid_every") or steps
    done = 0
    while done < steps:
        k = min(every, steps - done)
        for m in (m64, m32):
            m.step(cfg["dt"], k)
        done += k
        if cfg.get("regrid_every") and done < steps:
            flags = (m64.indicator() > cfg["threshold"]).astype(np.uint8)
            for m in (m64, m32):
                m.adapt(flags=flags, buffer=cfg["buffer"])
    assert np.array_equal(m64.leaves(), m32.leaves())
    p64, p32 = m64.primitives(), m32.primitives()
    D = cfg["dim"]
    I1 = [m.integrals() for m in (m64, m32)]
    out = {"steps": steps, "elements": m64.num_elements,
           "theta_max_abs_err_K": float((p32[D] - p64[D]).abs().max()),
           "theta_max_abs_K": float(p64[D].abs().max()),
           "w_max_abs_err": float((p32[D - 1] - p64[D - 1]).abs().max()),
           "w_max_abs": float(p64[D - 1].abs().max()),
           "mass_rel_err": abs(I1[1][0] - I1[0][0]) / I1[0][0],
           "energy_rel_err": abs(I1[1][1] - I1[0][1]) / abs(I1[0][1]),
           "mass_drift_fp64": abs(I1[0][0] - I0[0][0]) / I0[0][0],
           "mass_drift_fp32": abs(I1[1][0] - I0[1][0]) / I0[1][0],
           "reference": "FP64 path on the same trees (matches the oracle to 1e-12 per RHS)"}
    for m in (m64, m32):
        m.close()
    torch.cuda.synchronize()
    return out


def _timed_steps(m, cfg, steps, regrid_every, NP, NV, b, n1, D, per_node=None, face_kernel=False):
    """Runs `steps` SSP-RK3 steps (regrid every `regrid_every` inside) between two CUDA events on
    the mesh stream; returns the elapsed ms and the work counters of the region."""
    import torch
    dt = cfg["dt"]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    c = dict(dof_stage=0, alg_bytes=0, alg_flops=0, launches=0, traffic=0.0, regrid_s=[])
    ev0.record()
    for i in range(steps):
        E = m.num_elements
        m.step(dt, 1)
        c["dof_stage"] += 3 * E * NP
        c["alg_bytes"] += stage_bytes(E, NP, NV, b, n1, D)
        c["alg_flops"] += stage_flops(E, NP, NV, n1, D)
        if per_node:
            c["traffic"] += E * NP * sum(per_node)
        # stage (+ mortar, + face kernel in layout 5) launches per step
        c["launches"] += 3 * (1 + (m.num_mortars > 0) + face_kernel)
        if regrid_every and (i + 1) % regrid_every == 0:
            torch.cuda.synchronize()     # dg_adapt starts with this wait anyway
            tr = time.perf_counter()
            rep = m.adapt(threshold=cfg["threshold"], buffer=cfg["buffer"])
            c["regrid_s"].append(time.perf_counter() - tr)
            # indicator; transfer and background only when the pass changes the mesh
            c["launches"] += 1 + (2 if rep["refined"] or rep["coarsened"] else 0)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), c


def run_path(pkg, cfg, precision, steps, warmup, regrid_every, sampler=None, world=1, repeats=5):
    """The production path timed `repeats` times over `steps` steps each (the stage kernels run
    as in any dg_step call: after their mortar kernels as programmatic dependent launches); the
    median repeat is the result.  A further region of `steps` steps with per-stage CUDA events
    (dg_enable_timing, which needs an event between the mortar and the stage launch and so runs
    them without the dependent launch) gives the stage kernel's own time per launch."""
    import torch
    m = build_mesh(pkg, cfg, precision)
    dt = cfg["dt"]
    D, N = cfg["dim"], cfg["N"]
    n1, NP, NV = N + 1, (N + 1) ** D, D + 2
    b = 8 if precision == "fp64" else 4
    for i in range(warmup):
        m.step(dt, 1)
    torch.cuda.synchronize()
    m.integrals()
    default_layout = 4 if (precision == "fp32" and D == 3) else (5 if precision == "fp64" else 2)
    layout = default_layout if STAGE_KERNEL is None else STAGE_KERNEL
    per_node = measured_traffic(D, N, precision, layout)
    _barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    reps = []
    for r in range(repeats):
        _barrier(world)
        torch.cuda.synchronize()
        ms, c = _timed_steps(m, cfg, steps, regrid_every, NP, NV, b, n1, D, face_kernel=layout == 5)
        ms = _barrier_max(ms, world)
        reps.append((c["dof_stage"] / (ms / 1e3), ms, c))
    clocks = sampler.stop() if sampler else None
    rates = sorted(x[0] for x in reps)
    med = rates[len(rates) // 2]
    rate, ms, c = next(x for x in reps if x[0] == med)
    # stage-kernel time per launch, from a region with per-stage events
    m.enable_timing(True)
    m.stage_timing(reset=True)
    _barrier(world)
    torch.cuda.synchronize()
    ms_t, ct = _timed_steps(m, cfg, steps, regrid_every, NP, NV, b, n1, D, per_node, face_kernel=layout == 5)
    stage_ms, stage_launches = m.stage_timing(reset=True)
    m.enable_timing(False)
    integ = m.integrals()
    regrid_s = [t for x in reps for t in x[2]["regrid_s"]]
    out = dict(ms=ms, rate=rate, rates=[x[0] for x in reps], dof_stage=c["dof_stage"],
               launches=c["launches"], clocks=clocks,
               stage_ms=stage_ms, stage_launches=stage_launches, ms_timed_region=ms_t,
               alg_bytes=ct["alg_bytes"], alg_flops=ct["alg_flops"],
               elements=m.num_elements, nodes=m.num_nodes, integrals=integ.tolist(),
               state_bytes=NV * m.num_nodes * b, mortars=m.num_mortars,
               traffic_per_launch=(ct["traffic"] / (3 * steps)) if per_node else None,
               regrid_ms=(1e3 * sum(regrid_s) / len(regrid_s)) if regrid_s else None,
               regrids=len(regrid_s))
    return m, out


def run_e2e(pkg, m, cfg, steps, regrid_every, world=1):
    """Same metric through the public API with host buffers: each step copies the state in from
    pinned host memory, advances one step, and copies the state and the integrals back, with one
    host wait per step: the state's copy back runs on a copy stream while the integrals are
    computed on the mesh stream (dg_*_async)."""
    import torch
    dt = cfg["dt"]
    dtype = torch.float64 if m.precision == "fp64" else torch.float32
    host = torch.empty(m.state_shape, dtype=dtype).pin_memory()
    integ = torch.empty(6, dtype=torch.float64).pin_memory()
    copy = torch.cuda.Stream()
    m.get_state(host)
    torch.cuda.synchronize()
    h2d = d2h = 0
    dof = 0
    _barrier(world)
    t0 = time.perf_counter()
    for i in range(steps):
        if tuple(host.shape) != m.state_shape:
            host = torch.empty(m.state_shape, dtype=dtype).pin_memory()
            m.get_state(host)
            d2h += host.numel() * host.element_size()
        m.set_state_async(host)
        h2d += host.numel() * host.element_size()
        m.step(dt, 1)
        dof += 3 * m.num_nodes
        m.get_state_async(host, stream=copy)
        m.integrals_async(integ)
        torch.cuda.synchronize()
        d2h += host.numel() * host.element_size() + integ.numel() * 8
        if regrid_every and (i + 1) % regrid_every == 0:
            m.adapt(threshold=cfg["threshold"], buffer=cfg["buffer"])
    torch.cuda.synchronize()
    sec = _barrier_max(time.perf_counter() - t0, world)      # the slowest rank sets the job time
    return dict(value=world * dof / sec, unit=METRIC, h2d_bytes_per_step=h2d // steps,
                d2h_bytes_per_step=d2h // steps,
                pipeline="state in (pinned, mesh stream), step, state out (copy stream) alongside the "
                         "integrals (mesh stream), one host wait per step")


def run_adjoint(pkg):
    """Adjoint/forward time ratio on the 3D adjoint workload (12^3 elements, N = 5, FP64, bubble
    plus Gaussian random theta', 200 steps, checkpoints every 20): time of J(theta') alone
    against the time of J and dJ/dtheta' through the hand-written adjoint."""
    import torch
    from paper_2404_16648_gb300 import adjoint as ladj
    cfg = workloads.ADJOINT_3D
    m = pkg.Mesh(3, cfg["N"], cfg["base"], cfg["length"])
    r = cfg["rff"]
    theta = m.bubble_theta(**cfg["bubble"], rff=workloads.rff_draws(3, r["sigma"], r["length"], r["features"]))
    dt, nsteps = cfg["dt"], cfg["steps"]
    ladj.ke_gradient(m, theta, dt, 4, every=2)          # warm-up of both paths
    torch.cuda.synchronize()
    fwd, grad = [], []
    for _ in range(3):
        t0 = time.perf_counter()
        ladj.final_ke(m, theta, dt, nsteps)
        torch.cuda.synchronize()
        fwd.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        ladj.ke_gradient(m, theta, dt, nsteps, every=20)
        torch.cuda.synchronize()
        grad.append(time.perf_counter() - t0)
    f, g = min(fwd), min(grad)
    nodes = m.num_nodes
    m.close()
    return {"workload": cfg["name"], "steps": nsteps, "checkpoint_every": 20, "forward_ms": 1e3 * f,
            "gradient_ms": 1e3 * g, "adjoint_over_forward": g / f,
            "forward_dof_stage_per_s": 3 * nsteps * nodes / f}


def run_cold2d(pkg, steps=200):
    """The 2D tree-AMR cold bubble with viscosity (32 x 8 roots on 25.6 x 6.4 km, N = 5, up to 3
    levels, nu = 75 m^2/s by BR1, FP64, regrid every 10 steps inside the timed region)."""
    import torch
    cfg = workloads.COLD_2D
    m = pkg.Mesh(2, cfg["N"], cfg["base"], cfg["length"], max_level=cfg["max_level"], nu=cfg["nu"])
    pkg.adapt_initial(m, cfg["bubble"], cfg["threshold"], cfg["buffer"])
    m.step(cfg["dt"], 10)
    m.adapt(threshold=cfg["threshold"], buffer=cfg["buffer"])
    torch.cuda.synchronize()
    M0 = m.integrals()
    NP = (cfg["N"] + 1) ** 2
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    dof = 0
    ev0.record()
    for i in range(steps):
        dof += 3 * m.num_elements * NP
        m.step(cfg["dt"], 1)
        if (i + 1) % cfg["regrid_every"] == 0:
            m.adapt(threshold=cfg["threshold"], buffer=cfg["buffer"])
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    M1 = m.integrals()
    out = {"workload": cfg["name"], "precision": "fp64", "nu": cfg["nu"], "steps": steps,
           "regrid_every": cfg["regrid_every"], "elements": m.num_elements, "mortar_groups": m.num_mortars,
           "value": dof / (ms / 1e3), "unit": METRIC, "ms_per_step": ms / steps,
           "mass_rel_change": abs(M1[0] - M0[0]) / M0[0]}
    m.close()
    return out


def run_leveque(pkg):
    """Swirling deformational flow (Sec. 4.2): tracer bell on [0, 1]^2, 16 x 16 roots, N = 4,
    one level where |C| > 0.05, buffer 2, T = 5 in 2000 steps with 80 regrids, mortar and
    point-interpolation hanging faces, and uniform 16 x 16 and 32 x 32 grids; the paper times
    these runs (11 s, 18 s and 51 s on its hardware)."""
    import torch
    cfg = workloads.LEVEQUE_2D
    NP = (cfg["N"] + 1) ** 2
    out = {"workload": cfg["name"], "steps": cfg["steps"], "period": cfg["period"]}
    for name, mode, base, L in (("amr_mortar", "mortar", cfg["base"], 1), ("amr_interp", "interp", cfg["base"], 1),
                                ("uniform16", "mortar", cfg["base"], 0), ("uniform32", "mortar", (32, 32), 0)):
        m = pkg.Mesh(2, cfg["N"], base, cfg["length"], max_level=L, equations="tracer", face_mode=mode,
                     wind_period=cfg["period"])
        if L:
            pkg.adapt_initial(m, cfg["bubble"], cfg["threshold"], cfg["buffer"])
        else:
            m.set_bubble(**cfg["bubble"])
        m0 = m.integrals()[0]
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        dof = 0
        regrids = 0
        ev0.record()
        for _ in range(cfg["steps"] // cfg["regrid_every"]):
            dof += 3 * cfg["regrid_every"] * m.num_elements * NP
            m.step(cfg["dt"], cfg["regrid_every"])
            if L:
                m.adapt(threshold=cfg["threshold"], buffer=cfg["buffer"])
                regrids += 1
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        C = m.get_state()
        m.set_bubble(**cfg["bubble"])
        C0 = m.get_state()
        m.set_state(C)
        drift = abs(m.integrals()[0] - m0) / m0
        m.set_state((C - C0) ** 2)
        e2 = m.integrals()[0]
        m.set_state(C0 ** 2)
        n2 = m.integrals()[0]
        out[name] = {"seconds": ms / 1e3, "value": dof / (ms / 1e3), "unit": METRIC, "regrids": regrids,
                     "elements_at_T": m.num_elements, "tracer_rel_change": drift,
                     "l2_rel_error_at_T": float(np.sqrt(e2 / n2))}
        m.close()
    return out


def run_vortex(pkg, t_end=3.0, dt=0.0025, regrid_every=40, thr=1e-3):
    """Isentropic vortex (Sec. 4.1) on the periodic [0, 12]^2 box, 32 x 32 roots, N = 3, FP64:
    one refinement level where max |rho'| > thr (flags from the state), SSP-RK3 to t = 3 s, and
    the uniform 32 x 32 grid; the error in the paper's norm (1/N_dof) sqrt(sum |q - q_exact|^2)
    against the exact translated vortex (paper: about 8.75e-4 after 3 s)."""
    import torch
    out = {"workload": "isentropic_vortex_32x32_N3_L1", "t_end": t_end, "dt": dt}
    NP = 16
    for name, L in (("amr", 1), ("uniform32", 0)):
        m = pkg.Mesh(2, 3, (32, 32), (12.0, 12.0), max_level=L, theta0=1.0, p0=1.0, g=0.0, R=1.0,
                     cp=3.5, periodic=(True, True))

        def flags():
            return (np.abs(m.get_state()[0]).reshape(-1, NP).max(axis=1) > thr).astype(np.uint8)
        if L:
            m.set_vortex((6.0, 6.0), 5.0, (1.0, 1.0), 0.0)
            m.adapt(flags=flags(), buffer=1)
        m.set_vortex((6.0, 6.0), 5.0, (1.0, 1.0), 0.0)
        m0 = m.integrals()[0]
        nsteps = int(round(t_end / dt))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dof = 0
        done = 0
        while done < nsteps:
            k = min(regrid_every, nsteps - done)
            dof += 3 * k * m.num_elements * NP
            m.step(dt, k)
            done += k
            if L and done < nsteps:
                m.adapt(flags=flags(), buffer=1)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        q = m.get_state()
        drift = abs(m.integrals()[0] - m0) / m0
        m.set_vortex((6.0, 6.0), 5.0, (1.0, 1.0), t_end)
        e = q - m.get_state()
        out[name] = {"seconds": sec, "value": dof / sec, "unit": METRIC, "elements": m.num_elements,
                     "l2_paper_norm": float(np.sqrt(np.sum(e * e)) / e.size), "mass_rel_change": drift}
        m.close()
    out["paper_l2_at_t3"] = 8.75e-4
    return out


def _batch_member_work(m):
    """Algorithmic HBM bytes and flops of one SSP-RK3 step of a batch member."""
    D, N = m.dim, m.N
    b = 8 if m.precision == "fp64" else 4
    E, NP = m.num_elements, (N + 1) ** D
    return stage_bytes(E, NP, D + 2, b, N + 1, D), stage_flops(E, NP, D + 2, N + 1, D)


def run_batch(pkg, steps=500, compare_steps=50, check_steps=5, peaks=None):
    """Batched workload: 256 seeded 2D bubble instances (mesh 10x10 ... 64x32, N 3..7, FP32/FP64
    50/50, per-instance dt), autotuned shapes, `steps` graph-replayed SSP-RK3 steps (one
    persistent launch per stage); the same instances advanced one mesh launch at a time for
    `compare_steps` steps; bit-identity of the two after `check_steps` steps from the initial
    state; and per (precision, N) group the time of a batch of that group's members alone,
    against the group's roofline (its algorithmic bytes at the measured HBM copy rate or its
    counted flops at the measured FMA rate of its precision, whichever takes longer)."""
    import torch
    cfg = workloads.BATCH_2D
    inst = workloads.batch_instances(cfg["count"])

    def make():
        ms = []
        for d in inst:
            m = pkg.Mesh(2, d["N"], d["base"], cfg["length"], precision=d["precision"])
            m.set_bubble(**d["bubble"])
            ms.append(m)
        return ms

    meshes = make()
    dts = [d["dt"] for d in inst]
    nodes = sum(m.num_nodes for m in meshes)
    batch = pkg.Batch(meshes, dts)
    layouts = batch.autotune(reps=3)
    shape = batch.shape()
    batch.run(2, graph=True)                      # warm-up (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.run(steps, graph=True, sync=False)
    batch.sync()
    t_batch = time.perf_counter() - t0
    batch.close()
    # one mesh launch at a time, and the bit-identity check from the initial state
    singles = make()
    for m, lay in zip(singles, layouts):
        m.set_stage_kernel(int(lay))
    fresh = make()
    for m, lay in zip(fresh, layouts):
        m.set_stage_kernel(int(lay))
    fb = pkg.Batch(fresh, dts)
    fb.run(check_steps, graph=True)
    for m, dt in zip(singles, dts):
        m.step(dt, check_steps)
    torch.cuda.synchronize()
    identical = all(np.array_equal(a.get_state(), b.get_state()) for a, b in zip(fresh, singles))
    fb.close()
    t0 = time.perf_counter()
    for _ in range(compare_steps):
        for m, dt in zip(singles, dts):
            m.step(dt, 1)
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    # per (precision, N) group: a batch of its members alone
    groups = {}
    for k, d in enumerate(inst):
        groups.setdefault((d["precision"], d["N"]), []).append(k)
    peaks = peaks or {}
    hbm = peaks.get("hbm_gbs", 6800.0) * 1e9
    pipe = {"fp64": peaks.get("fp64_flops"), "fp32": peaks.get("fp32_flops")}
    per_group, bound_s = [], 0.0
    for (prec, N), ks in sorted(groups.items()):
        sub = pkg.Batch([meshes[k] for k in ks], [dts[k] for k in ks])
        sub.autotune(reps=2)
        sub.run(2, graph=True)
        torch.cuda.synchronize()
        gs = 20
        t0 = time.perf_counter()
        sub.run(gs, graph=True, sync=False)
        sub.sync()
        ms = 1e3 * (time.perf_counter() - t0) / gs
        sub.close()
        byt = sum(_batch_member_work(meshes[k])[0] for k in ks)
        flo = sum(_batch_member_work(meshes[k])[1] for k in ks)
        tb = max(byt / hbm, flo / pipe[prec] if pipe[prec] else 0.0)
        bound_s += tb
        per_group.append({"precision": prec, "N": N, "members": len(ks),
                          "nodes_per_variable": sum(meshes[k].num_nodes for k in ks),
                          "ms_per_step_alone": ms, "roofline_ms": 1e3 * tb,
                          "bound": "hbm" if byt / hbm >= (flo / pipe[prec] if pipe[prec] else 0.0) else "alu"})
    for m in meshes + singles + fresh:
        m.close()
    rate_b = 3 * steps * nodes / t_batch
    rate_s = 3 * compare_steps * nodes / t_single
    ms_step = 1e3 * t_batch / steps
    return {"workload": cfg["name"], "instances": len(inst), "nodes_per_variable": nodes,
            "steps": steps, "value": rate_b, "unit": METRIC, "ms_per_step": ms_step,
            "launch": "one persistent launch per stage over all members (mortar and element-tile "
                      "work items, graph-replayed)",
            "shape": shape,
            "one_at_a_time_value": rate_s, "speedup_vs_one_at_a_time": rate_b / rate_s,
            "bit_identical_to_one_at_a_time": bool(identical), "identity_steps": check_steps,
            "layouts": {"node": int(np.sum(layouts == 1)), "column_async": int(np.sum(layouts == 2)),
                        "column_async_face_items": int(np.sum(layouts == 5))},
            "roofline": {"bound": "mixed", "roofline_ms_per_step": 1e3 * bound_s,
                         "frac": 1e3 * bound_s / ms_step,
                         "note": "sum over (precision, N) groups of max(algorithmic bytes / measured "
                                 "HBM copy rate, counted flops / measured FMA rate of the precision), "
                                 "against the batch's measured step time"},
            "groups": per_group}


_ORACLE = {}


def _oracle_setup(cfg):
    """The oracle mesh of a workload and its initial state (built once per process)."""
    from oracle import dg as odg, forest as ofo
    cfg_name = cfg["name"]
    if cfg_name not in _ORACLE:
        b = cfg["bubble"]
        om = odg.adapt_initial(ofo.Forest(cfg["base"], cfg["max_level"]), cfg["N"], cfg["length"],
                               lambda mm: odg.bubble_theta(mm, b["center"], b["radius"], b["amp"]),
                               cfg["threshold"], cfg["buffer"])
        q = odg.state_from_theta(om, odg.bubble_theta(om, b["center"], b["radius"], b["amp"]))
        _ORACLE[cfg_name] = (om, q)
    return _ORACLE[cfg_name]


def _oracle_block_step(args):
    """One SSP-RK3 step of the oracle (mortars included) for a block of consecutive elements;
    its stages are evaluated on the block's two- and one-hop neighbourhoods as the step needs."""
    cfg, start, n = args
    from oracle import dg as odg
    om, q = _oracle_setup(cfg)
    elems = np.arange(start, min(om.E, start + n))
    t0 = time.perf_counter()
    odg.step_on(om, q, cfg["dt"], elems)
    sec = time.perf_counter() - t0
    # node-stage updates the oracle performed: stage 1 on the two-hop neighbourhood, stage 2 on
    # the one-hop neighbourhood, stage 3 on the block
    hop1 = set(elems.tolist())
    for e in elems:
        hop1 |= set(om.forest.face_neighbors(int(e)))
    hop2 = set(hop1)
    for e in list(hop1):
        hop2 |= set(om.forest.face_neighbors(int(e)))
    return len(hop2) + len(hop1) + len(elems), sec


def host_description():
    """CPU model and core count of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


class OraclePool:
    """The oracle stepped on blocks of consecutive elements by a pool of host processes (spawned,
    so the pool is safe to start after the GPU is in use).  A timed map is one SSP-RK3 step of
    `procs` blocks of `block` elements taken from the middle of the leaf order."""

    def __init__(self, cfg, procs, block):
        import multiprocessing as mp
        self.cfg, self.procs, self.block = cfg, procs, block
        self.pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_setup, initargs=(cfg,))
        om, _ = _oracle_setup(cfg)   # for the sizes (and the single-core leg)
        self.E, self.NP = om.E, om.np_
        first = max(0, om.E // 2 - procs * block // 2)
        self.tasks = [(cfg, first + k * block, block) for k in range(procs)]
        self.pool.map(_oracle_block_step, self.tasks, chunksize=1)   # warm-up: every worker ready

    def step(self):
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_block_step, self.tasks, chunksize=1)
        sec = time.perf_counter() - t0
        return sum(r[0] for r in res) * self.NP, sec

    def single(self):
        n, sec = _oracle_block_step(self.tasks[0])
        return n * self.NP, sec

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(cfg, procs=None, block=96, maps=2):
    """The oracle timed on the host cores on a bounded sample of the workload: one SSP-RK3 step
    (three RHS evaluations with mortars, Shu-Osher combination) on blocks of consecutive
    elements, single-threaded and on all cores."""
    procs = procs or os.cpu_count() or 1
    pool = OraclePool(cfg, procs, block)
    units = sec = 0.0
    for _ in range(maps):
        u, t = pool.step()
        units += u
        sec += t
    u1, t1 = pool.single()
    pool.close()
    host = host_description()
    return {"value": units / sec, "unit": METRIC, "cores": procs, "kind": "oracle",
            "sample": "one SSP-RK3 step (mortars included) of %d blocks of %d consecutive elements "
                      "of %d, %d times (%.1f s); single core: one block (%.1f s).  Counted: every "
                      "node-stage update performed (stage 1 on a block's two-hop face "
                      "neighbourhood, stage 2 on its one-hop neighbourhood, stage 3 on the block)"
                      % (procs, block, pool.E, maps, sec, t1),
            "single_core": {"value": u1 / t1, "cores": 1},
            "cpu_model": host["cpu_model"], "nproc": host["nproc"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--base-div", type=int, default=1,
                    help="divide the workload's root grid by this factor (a smaller copy of the same "
                         "workload, for profiler captures; the default is the full workload)")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed repeats of --steps steps each; the median is reported (at least 5)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=workloads.BUBBLE_3D["name"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-cold2d", action="store_true",
                    help="skip the 2D viscous cold-bubble leg")
    ap.add_argument("--no-leveque", action="store_true",
                    help="skip the tracer swirling-flow leg")
    ap.add_argument("--no-vortex", action="store_true",
                    help="skip the isentropic-vortex leg")
    ap.add_argument("--clock-log", default=None,
                    help="directory for the raw nvidia-smi clock samples (default: a temporary one)")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the FP32-vs-FP64 field comparison over the workload's full step count")
    ap.add_argument("--stage-kernel", type=int, default=None, choices=[0, 1, 2, 3, 4, 5],
                    help="stage kernel layout: 0 column, 1 node-per-thread, 2 column with "
                         "asynchronous staging, 3 as 2 with two threads per column, 4 line, "
                         "5 as 2 with the face fluxes once per face (default: the library's)")
    args = ap.parse_args()
    global STAGE_KERNEL
    STAGE_KERNEL = args.stage_kernel
    cfg = workloads.CONFIGS[args.config]
    if args.base_div > 1:
        cfg = workloads.scaled(cfg, base_div=args.base_div)
    world, rank, local = _dist()
    regrid_every = cfg.get("regrid_every")
    config = {"workload": cfg["name"], "dim": cfg["dim"], "N": cfg["N"], "base": list(cfg["base"]),
              "max_level": cfg["max_level"], "dt": cfg["dt"], "regrid_every": regrid_every,
              "buffer": cfg["buffer"], "l2": "inputs larger than L2 (state > 129 MB)",
              "parallelism": "replicas" if world > 1 else "single"}

    if args.impl == "reference":
        if rank != 0:
            return
        procs = os.cpu_count() or 1
        pool = OraclePool(cfg, procs, block=48)
        for _ in range(args.warmup):
            pool.step()
        units = sec = 0.0
        for _ in range(max(1, args.steps)):
            u, t = pool.step()
            units += u
            sec += t
        pool.close()
        rate = units / sec
        host = host_description()
        line = {"metric": METRIC, "value": rate, "unit": METRIC, "impl": "reference",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * sec / max(1, args.steps), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config,
                "cpu_baseline": {"value": rate, "unit": METRIC, "cores": procs, "kind": "oracle",
                                 "sample": "per step: one SSP-RK3 step (mortars included) of %d blocks of "
                                           "48 consecutive elements of %d; every node-stage update "
                                           "performed is counted (stages 1 and 2 on the blocks' two- "
                                           "and one-hop face neighbourhoods)" % (procs, pool.E),
                                 "cpu_model": host["cpu_model"], "nproc": host["nproc"]},
                "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import paper_2404_16648_gb300 as pkg
    pkg.load_library()
    peaks, peak_kind = _peaks()
    sampler = ClockSampler(local, args.clock_log)
    R = max(5, args.repeats)
    m32, r32 = run_path(pkg, cfg, "fp32", args.steps, args.warmup, regrid_every, sampler, world, R)
    e2e = run_e2e(pkg, m32, cfg, max(4, min(args.steps, 20)), regrid_every, world)
    m32.close()
    r64 = None
    if not args.no_fp64:
        m64, r64 = run_path(pkg, cfg, "fp64", args.steps, args.warmup, regrid_every, None, world, R)
        m64.close()
    value = world * r32["rate"]
    achieved = r32["alg_bytes"] / (r32["stage_ms"] / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r32["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config,
            "timing": {"repeats": R, "statistic": "median repeat of %d steps each" % args.steps,
                       "repeat_values": [world * v for v in r32["rates"]],
                       "path": "production dg_step (stage kernels as programmatic dependent launches "
                               "after their mortar kernels)"},
            "precision_path": "FP32 state/flux arithmetic; FP64 background and integrals; P' to FP64 accuracy before its FP32 rounding",
            "stage_kernel": {None: "default", 0: "column", 1: "node", 2: "column-async", 3: "half-column-async", 4: "line",
                             5: "column-async with face kernel"}[STAGE_KERNEL],
            "elements": r32["elements"], "nodes_per_variable": r32["nodes"],
            "gpu_launches": r32["launches"], "mortar_groups": r32["mortars"],
            "roofline": {"bound": "hbm", "kernel": "stage_kernel", "achieved": achieved,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "peak_kind": peak_kind,
                         "traffic": r32["traffic_per_launch"],
                         "traffic_note": "ncu dram read+write per node of each stage launch "
                                         "(profiles/stage_traffic_bubble3d_N7.json) scaled to this run's "
                                         "nodes; null when the kernel sources changed",
                         "algorithmic_bytes_per_launch": r32["alg_bytes"] / (3 * args.steps),
                         "stage_ms_per_launch": r32["stage_ms"] / max(1, r32["stage_launches"]),
                         "stage_timing": "CUDA events around each stage launch over a further "
                                         "%d-step region (%.3f ms per step there)"
                                         % (args.steps, r32["ms_timed_region"] / args.steps)},
            "clocks": r32["clocks"], "e2e": e2e,
            "regrid": {"count": r32["regrids"], "ms_avg_host_wall": r32["regrid_ms"],
                       "note": "dg_adapt inside the timed region: indicator, host tree work, "
                               "topology tables, conservative transfer"}}
    if r64 is not None:
        v64 = world * r64["rate"]
        fp64_peak = pkg.probe_fma_rate("fp64") / 1e12
        ach64 = r64["alg_flops"] / (r64["stage_ms"] / 1e3) / 1e12
        line["fp64"] = {"value": v64, "ms_per_step": r64["ms"] / args.steps, "dtype": "f64",
                        "repeat_values": [world * v for v in r64["rates"]],
                        "roofline": {"bound": "alu", "kernel": "stage_kernel (+ face_kernel in layout 5)",
                                     "achieved": ach64,
                                     "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach64 / fp64_peak,
                                     "peak_kind": "measured: dg_probe_fma_rate (independent FP64 "
                                                  "multiply-adds on every SM, CUDA events)",
                                     "stage_ms_per_launch": r64["stage_ms"] / max(1, r64["stage_launches"]),
                                     "stage_timing": "CUDA events around each stage's face kernel "
                                                     "(layout 5) and stage kernel"},
                        "integrals": r64["integrals"]}
        line["fp32_over_fp64"] = value / v64
    if not args.no_accuracy and cfg.get("threshold") is not None:
        line["fp32_accuracy"] = fp32_accuracy(pkg, cfg, cfg["steps"])
    if not args.no_adjoint:
        line["adjoint"] = run_adjoint(pkg)
    if not args.no_batch:
        bpeaks = dict(peaks)
        bpeaks["fp64_flops"] = pkg.probe_fma_rate("fp64")
        bpeaks["fp32_flops"] = pkg.probe_fma_rate("fp32")
        line["batch"] = run_batch(pkg, peaks=bpeaks)
    if not args.no_cold2d:
        line["cold2d"] = run_cold2d(pkg)
    if not args.no_leveque:
        line["leveque"] = run_leveque(pkg)
    if not args.no_vortex:
        line["vortex"] = run_vortex(pkg)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(cfg)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
