"""Benchmark: the batched-shot gradient step on one GB300.

Default workload: the 16-shot layered mesh (96x96x48 interior elements + 10-element PML,
6.35 M nodes, three layers and a stiff inclusion, 16 vertical surface sources on a 4x4
grid, 48x48 surface receivers). One step = one gradient evaluation of all 16 shots
advanced together (B shots per launch of every stage kernel, B picked by the library's
autotuner, at most 16), each sweep replayed as a recorded CUDA graph: forward RK4 sweep
with source injection and receiver sampling, misfit (7), reversed-time adjoint sweep,
FP64 gradient time integrals (C.1f)/(C.1g), with inputs resident in HBM. A step covers a
window of --window time steps (default 50) of the configuration's 3000: the per-step work
of the stage kernels does not depend on the step count, and 3000 steps of 16 shots take
minutes per evaluation. value is element-stage updates per second (elements x 4 RK4
stages x time steps x shots, forward and adjoint sweeps); a projection to full-length
evaluations is reported beside it. The e2e figure repeats the step through the C ABI with
host buffers (material and observed traces uploaded, gradients downloaded every step).

--workload grf_64x64x32: the single-shot mesh (64x64x32 + 10 PML, 2000 steps); one step
is one full-length single-shot gradient evaluation (value in shot-gradient evals/s).

Multi-GPU: each rank evaluates its own group of shots of the workload, and the misfits and
FP64 gradients are summed over the ranks once per step (rank-order all-gather on NCCL),
inside the timed region; the value is the sum over ranks (weak scaling).

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload (the
reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import fwi_inputs as fi  # noqa: E402

METRIC = "shot-gradient evals/s (element-stage updates/s), HBM roofline %, misfit drop/sec"
UNIT = "shot-gradient evals/s"
UNIT_ES = "element-stage updates/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_peak():
    """Dense BF16 tensor throughput (TFLOP/s) for a kernel timed alone: the measured burst
    figure, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    except Exception:
        return 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# the sources of the four stage kernels (interior, shell, PML face, PML) and of the host
# code that builds their node lists and launch shapes
STAGE_SOURCES = ("fwi_api.cu", "fwi_interior.cu", "fwi_internal.h", "fwi_pml.cu", "fwi_stage.cu")


def kernel_sources_sha256():
    """Digest of the stage kernels' sources: a committed ncu traffic figure is reported
    only while the kernels it was measured on are unchanged."""
    import hashlib

    d = os.path.join(ROOT, "paper_1504_08340_gb300", "csrc")
    h = hashlib.sha256()
    for name in STAGE_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def measured_traffic(workload_name, batch=1, nmat=0):
    """DRAM bytes (read + write) of one stage launch set from the committed ncu summary, or
    None. A summary taken on one shot is scaled to a launch set of `batch` shots: the state
    traffic grows with the shots, lambda and mu (8 bytes a material node) are read once."""
    path = os.path.join(ROOT, "profiles", f"stage_traffic_{workload_name}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("csrc_sha256") != kernel_sources_sha256():
        return None
    one = rec.get("dram_bytes_per_stage")
    shots = rec.get("shots_per_launch", 1)
    if one is None or batch == shots:
        return one
    mat = 8.0 * nmat
    return (one - mat) / shots * batch + mat


TRAFFIC_COMMAND = ('ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum --clock-control none '
                   '-k regex:"interior_kernel|shell_kernel|pml_kernel|pml_face_kernel" -s 16 -c 16 --csv '
                   '--log-file traffic_layered.csv python bench.py --profile-forward 3 --max-batch 1')


def traffic_summary(csv_path, workload_name):
    """The per-stage DRAM traffic summary of the stage kernels from an ncu CSV log of
    TRAFFIC_COMMAND (16 launches: the four kernels of each of the four stages of one
    forward step of one shot), keyed to the current stage-kernel sources."""
    import csv

    per = {}
    launches = set()
    with open(csv_path) as f:
        rows = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(rows):
        name = r["Kernel Name"]
        if name.endswith(")"):  # drop the argument list (template arguments may hold parentheses)
            depth, i = 0, len(name) - 1
            while i >= 0:
                depth += {")": 1, "(": -1}.get(name[i], 0)
                if depth == 0:
                    break
                i -= 1
            name = name[:i]
        if name.startswith("void "):
            name = name[5:]
        launches.add(r["ID"])
        per.setdefault(name, {})
        per[name][r["Metric Name"]] = per[name].get(r["Metric Name"], 0.0) + float(r["Metric Value"].replace(",", ""))
    stages = len(launches) / 4
    rd = sum(k.get("dram__bytes_read.sum", 0.0) for k in per.values()) / stages
    wr = sum(k.get("dram__bytes_write.sum", 0.0) for k in per.values()) / stages
    for k in per.values():  # durations in seconds
        if "gpu__time_duration.sum" in k:
            k["gpu__time_duration.sum"] *= 1e-9
    return {"workload": workload_name, "shots_per_launch": 1, "csrc_sha256": kernel_sources_sha256(),
            "stages_captured": stages, "kernel_launches_captured": len(launches),
            "dram_bytes_per_stage": rd + wr, "dram_read_bytes_per_stage": rd, "dram_write_bytes_per_stage": wr,
            "per_kernel": per, "command": TRAFFIC_COMMAND}


WORKLOADS = {"layered_96x96x48": fi.layered_96x96x48, "grf_64x64x32": fi.grf_64x64x32}


def workload(name="grf_64x64x32"):
    return WORKLOADS[name]()


def stage_bytes_per_step_17(ctx):
    """The same stage traffic in a streaming model of 17 state accesses per
    variable per step (an RK4 accumulator read and written at every stage)."""
    p = ctx.npml_nodes
    n = ctx.nnode
    return 17 * 4 * (27 * p + 6 * (n - p))


def stage_bytes_per_step(ctx, nmat):
    """Algorithmic HBM bytes of the four stage kernels of one RK4 step: each stage reads
    its input state and writes its output once (13 floats per state variable per step:
    2 + 3 + 3 + 5), 27 variables on PML nodes, 6 elsewhere, plus lambda and mu per stage."""
    p = ctx.npml_nodes
    n = ctx.nnode
    return 13 * 4 * (27 * p + 6 * (n - p)) + 4 * 8 * nmat


def setup(w, torch, dev):
    from paper_1504_08340_gb300 import Context

    ctx = Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho)
    lt, mt = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "true"))
    l0, m0 = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "trial"))
    ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
    ctx.set_receivers(w.receivers())
    ctx.set_material(lt, mt)
    obs = torch.zeros(ctx.trace_shape(1), dtype=torch.float32, device=dev)
    ctx.forward(out=obs)  # observed data: the true medium's response (outside the timed region)
    ctx.set_material(torch.tensor(l0, device=dev), torch.tensor(m0, device=dev))
    return ctx, obs, (l0, m0)


_ORACLE_MESH = {}


def cpu_baseline_es(w, steps_sample=1):
    """The oracle, as it stands, on a bounded sample of the batched workload: `steps_sample`
    forward and adjoint RK4 steps of one shot on the full-size mesh, as element-stage
    updates per second (elements x 4 stages x steps x 2 sweeps / wall time of the sweeps;
    the mesh set-up is built once and not timed)."""
    import oracle

    if w.name not in _ORACLE_MESH:
        o = oracle.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
        l0, m0 = fi.medium(w, "trial")
        o.set_material(l0, m0)
        _ORACLE_MESH[w.name] = o
    o = _ORACLE_MESH[w.name]
    src = [o.node_id(*w.sources()[0])]
    rec = [o.node_id(*r) for r in w.receivers()]
    t0 = time.perf_counter()
    tr, hist = o.forward(w.dt, steps_sample, src, w.source_dirs()[:1], "ricker", (w.f0, 0.0, w.amp), rec,
                         keep_history=True)
    o.adjoint_gradient(w.dt, steps_sample, rec, tr, hist)
    t = time.perf_counter() - t0
    nelem = o.N[0] * o.N[1] * o.N[2]
    return {"value": nelem * 4 * steps_sample * 2 / t, "unit": UNIT_ES, "cores": o.threads, "kind": "oracle",
            "sample": f"{steps_sample} forward + {steps_sample} adjoint RK4 step(s) of one shot on the {w.name} mesh, "
                      f"FP64 C oracle, {o.threads} threads", "sample_seconds": t}


def cpu_baseline(w, steps_sample=2, repeats=1):
    """The oracle, as it stands, on a bounded sample: `steps_sample` forward and adjoint RK4
    steps of the full-size mesh, scaled to one full gradient evaluation."""
    import oracle

    o = oracle.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
    l0, m0 = fi.medium(w, "trial")
    o.set_material(l0, m0)
    src = [o.node_id(*s) for s in w.sources()]
    rec = [o.node_id(*r) for r in w.receivers()]
    best = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        tr, hist = o.forward(w.dt, steps_sample, src, w.source_dirs(), "ricker", (w.f0, 0.0, w.amp), rec,
                             keep_history=True)
        o.adjoint_gradient(w.dt, steps_sample, rec, tr, hist)
        t = time.perf_counter() - t0
        best = t if best is None else min(best, t)
    per_eval = best * (w.nsteps / steps_sample)
    return {"value": 1.0 / per_eval, "unit": UNIT, "cores": o.threads, "kind": "oracle",
            "sample": f"{steps_sample} forward + {steps_sample} adjoint RK4 steps of the {w.name} mesh "
                      f"(of {w.nsteps} each), FP64 C oracle, {o.threads} threads, scaled x{w.nsteps / steps_sample:g}",
            "sample_seconds": best}


def run_reference_batched(args, w):
    """The reference arm on the batched workload: each step times the oracle on one forward
    and one adjoint step of one shot of the full-size mesh (element-stage updates/s)."""
    for _ in range(args.warmup):
        cpu_baseline_es(w)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline_es(w)["value"])
    total = time.perf_counter() - t0
    v = float(np.mean(vals))
    per_step_work = w.elements * 4 * 2  # one shot, one forward and one adjoint RK4 step
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT_ES, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_step_work / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "mesh": f"{w.nx}x{w.ny}x{w.nz}+{w.npml} PML", "shots": w.nshots,
                       "nsteps_of_configuration": w.nsteps, "receivers": w.nrec_side ** 2},
            "cpu_baseline": {"value": v, "unit": UNIT_ES, "kind": "oracle", "cores": os.cpu_count(),
                             "sample": f"each step: 1 forward + 1 adjoint RK4 step of one shot on the {w.name} mesh; "
                                       f"wall {total:.1f} s for {args.steps} steps"},
            "e2e": {"value": v, "unit": UNIT_ES, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if w.nshots > 1:
        return run_reference_batched(args, w)
    for _ in range(args.warmup):
        cpu_baseline(w, steps_sample=1)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, steps_sample=1)["value"])
    total = time.perf_counter() - t0
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "mesh": f"{w.nx}x{w.ny}x{w.nz}+{w.npml} PML", "nsteps": w.nsteps,
                       "receivers": w.nrec_side ** 2, "shots_per_step": 1},
            "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": os.cpu_count(),
                             "sample": f"each step: 1 forward + 1 adjoint RK4 step of {w.name} "
                                       f"(of {w.nsteps}), scaled x{w.nsteps}; wall {total:.1f} s for {args.steps} steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def profile_forward(w, nsteps, repeats, batch=1):
    """Short forward sweeps on the benchmark mesh (no history) for ncu captures; with the
    batched workload, `batch` shots per launch."""
    import torch

    w.nsteps = nsteps
    dev = torch.device("cuda", 0)
    ctx, obs, _ = setup(w, torch, dev)
    nb = min(batch, w.nshots)
    if nb > 1:
        ctx.set_shot_batch(nb)
        obs = torch.zeros(ctx.trace_shape(nb), dtype=torch.float32, device=dev)
    for _ in range(repeats):
        ctx.forward(0, nb, out=obs)
    torch.cuda.synchronize()
    print(json.dumps({"profile_forward": w.name, "nsteps": nsteps, "repeats": repeats}))
    ctx.close()
    return 0


def run_batch_sweep(args):
    """Multi-shot gradient evaluations on the 96x96x48-element layered mesh (16 shots on a 4x4
    surface grid, 48x48 receivers) with B shots advanced by each launch of the stage kernels,
    one JSON line per B. nsteps is cut to --sweep-nsteps (of the configuration's 3000) so that
    a sweep over B takes minutes; the per-step work, and so the throughput, does not depend
    on the step count."""
    import torch

    w = fi.layered_96x96x48()
    full_steps = w.nsteps
    w.nsteps = args.sweep_nsteps
    dev = torch.device("cuda", 0)
    from paper_1504_08340_gb300 import Context

    ctx = Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho)
    l0, m0 = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "trial"))
    ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
    ctx.set_receivers(w.receivers())
    ctx.set_shot_batch(max(args.shot_batches))
    # observed data: within the cut step count no wave has reached the layers below the
    # top one, where the true and the starting media differ, so their responses agree and
    # the residual would vanish; seeded smooth synthetic traces keep it (and the gradient)
    # nonzero. The work per step does not depend on the values.
    obs = torch.tensor(np.stack([fi.synthetic_traces(w.nsteps, w.nrec_side ** 2, 100 + s)
                                 for s in range(w.nshots)]), dtype=torch.float32, device=dev)
    ctx.set_material(torch.tensor(l0, device=dev), torch.tensor(m0, device=dev))
    gl = torch.empty(ctx.mat_shape(), dtype=torch.float64, device=dev)
    gm = torch.empty_like(gl)
    hbm, peak_kind = _peaks()
    state_bytes = stage_bytes_per_step(ctx, 0) / 4.0  # one shot's state traffic per stage
    mat_bytes = 8.0 * ctx.nmat  # lambda, mu once per stage launch
    ref = None
    for B in args.shot_batches:
        ctx.set_shot_batch(B)
        for _ in range(args.warmup):
            J, _, _ = ctx.adjoint_gradient(obs, 0, w.nshots, g_lambda=gl, g_mu=gm)
        ctx.reset_timing()
        ctx.set_timing(True)
        sampler = ClockSampler(0)
        sampler.start()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            J, _, _ = ctx.adjoint_gradient(obs, 0, w.nshots, g_lambda=gl, g_mu=gm)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ctx.set_timing(False)
        ms = e0.elapsed_time(e1) / args.steps
        stage_ms, stage_launches = ctx.timing(0)
        _, all_launches = ctx.timing(3)
        if ref is None:
            ref = (J, gl.clone(), gm.clone())
        drift = float(max(torch.linalg.vector_norm(gl - ref[1]) / torch.linalg.vector_norm(ref[1]),
                          torch.linalg.vector_norm(gm - ref[2]) / torch.linalg.vector_norm(ref[2])))
        per_launch = B * state_bytes + mat_bytes
        achieved = per_launch * stage_launches / (stage_ms / 1e3) / 1e9 if stage_ms > 0 else None
        print(json.dumps({
            "metric": "multi-shot gradient: shot-gradient evals/s", "value": w.nshots / (ms / 1e3),
            "unit": "shot-gradient evals/s (at the reduced step count)", "shot_batch": B, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "mesh": f"{w.nx}x{w.ny}x{w.nz}+{w.npml} PML, h={w.h} m",
                       "nodes": ctx.nnode, "elements": ctx.nelem, "shots": w.nshots,
                       "nsteps": w.nsteps, "nsteps_of_configuration": full_steps,
                       "receivers": w.nrec_side ** 2, "forward_history": "stored every step",
                       "observed": "seeded synthetic traces", "l2": "inputs larger than L2"},
            "element_stage_updates_per_s": w.nshots * ctx.nelem * 8 * w.nsteps / (ms / 1e3),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm if achieved else None, "peak_kind": peak_kind,
                         "kernel": "RK4 stage launch set advancing B shots", "bytes_per_launch": per_launch,
                         "avg_launch_ms": stage_ms / max(stage_launches, 1)},
            "gpu_launches": int(all_launches), "misfit": J, "J_equal_to_B1": J == ref[0],
            "gradient_rel_l2_vs_B1": drift, "clocks": clocks}), flush=True)
    # the library's own choice: fwi_tune_shot_batch times 10 forward steps per candidate
    t0 = time.perf_counter()
    chosen = ctx.tune_shot_batch(0, w.nshots, max_batch=max(args.shot_batches), steps=10)
    print(json.dumps({"autotune": {"chosen_shot_batch": chosen, "max_batch": max(args.shot_batches),
                                   "steps_per_candidate": 10, "seconds": time.perf_counter() - t0}}), flush=True)
    ctx.close()
    return 0


def profile_gradient(w, nsteps, repeats, batch=1):
    """Short gradient evaluations on the benchmark mesh (nsteps + 1 history levels) for ncu
    captures of the adjoint and gradient kernels; with the batched workload, `batch` shots
    per launch."""
    import torch

    w.nsteps = nsteps
    dev = torch.device("cuda", 0)
    ctx, obs, _ = setup(w, torch, dev)
    nb = min(batch, w.nshots)
    if nb > 1:
        ctx.set_shot_batch(nb)
    obs = torch.tensor(np.stack([fi.synthetic_traces(nsteps, w.nrec_side ** 2, 7 + s) for s in range(nb)]),
                       dtype=torch.float32, device=dev).contiguous()
    for _ in range(repeats):
        J, _, _ = ctx.adjoint_gradient(obs, 0, nb)
    torch.cuda.synchronize()
    print(json.dumps({"profile_gradient": w.name, "nsteps": nsteps, "repeats": repeats, "misfit": J}))
    ctx.close()
    return 0


# FP32 CUDA-core peak of a GB300 at its 2070 MHz maximum clock: 152 SMs x 128 FP32 lanes x
# 2 flops per fused multiply-add (the bound of the direct convolutions, which do not use
# tensor cores)
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def run_precond_bench(args):
    """The learned preconditioner's 3x3x3 convolution kernels on the interior material grid of
    the 64x64x32 mesh (65 x 129 x 129 voxels), 32 -> 32 channels, BF16 activations and
    weights with FP32 accumulation (inputs larger than L2), and one training step of a
    4 -> 16 -> 16 -> 2 network on the same grid. One JSON line per kernel."""
    import ctypes

    import torch

    from paper_1504_08340_gb300.fwi import load_library
    from paper_1504_08340_gb300.precond import ConvNet

    lib = load_library()
    dev = torch.device("cuda", 0)
    D, H, W = fi.grf_64x64x32().mat_shape
    nv = D * H * W
    c = 32
    g = torch.Generator(device=dev).manual_seed(0)
    x32 = torch.randn((c, D, H, W), generator=g, device=dev)
    net = ConvNet((4, 16, 16, 2), (D, H, W), seed=0, device=dev)
    x = net.to_bf16(x32)
    w = net.to_bf16(torch.randn((c, c, 27), generator=g, device=dev) / (27 * c) ** 0.5)
    b = torch.zeros(c, device=dev)
    y = torch.empty((c, D, H, W), dtype=torch.bfloat16, device=dev)
    dy = torch.randn((c, D, H, W), generator=g, device=dev)
    dx = torch.empty_like(dy)
    dw = torch.empty((c, c, 27), device=dev)
    db = torch.empty(c, device=dev)
    work = torch.empty(lib.fwi_nn_conv3d_backward_weight_work(c, c, D, H, W), device=dev)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    kernels = {
        "conv3d_forward (ReLU)": lambda: lib.fwi_nn_conv3d_forward(P(x), P(w), P(b), c, c, D, H, W, 1, P(y), st),
        "conv3d_backward_data": lambda: lib.fwi_nn_conv3d_backward_data(P(dy), P(w), c, c, D, H, W, P(dx), st),
        "conv3d_backward_weight": lambda: lib.fwi_nn_conv3d_backward_weight(P(dy), P(x), c, c, D, H, W, P(dw), P(db),
                                                                            P(work), st),
    }
    flops = 2.0 * c * c * 27 * nv
    bf16_peak, bf16_kind = _bf16_peak()
    # the tensor-core kernels against the BF16 tensor peak (the backward ones take the FP32
    # gradient as three BF16 parts, so their MMAs execute 3x the algorithmic products)
    tensor = {"conv3d_forward (ReLU)": 1.0, "conv3d_backward_data": 3.0, "conv3d_backward_weight": 3.0}
    for name, fn in kernels.items():
        for _ in range(max(args.warmup, 3)):
            assert fn() == 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            assert fn() == 0
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        tf = flops / (ms * 1e-3) / 1e12
        if name in tensor:
            roof = {"bound": "tensor", "achieved": tf, "peak": bf16_peak, "unit": "TFLOP/s", "frac": tf / bf16_peak,
                    "peak_kind": bf16_kind, "mma_TFLOP/s": tf * tensor[name]}
        else:
            roof = {"bound": "alu", "achieved": tf, "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s",
                    "frac": tf / FP32_ALU_TFLOPS, "peak_kind": "derived (FP32 lanes x clock)"}
        print(json.dumps({"metric": "learned preconditioner kernel", "kernel": name, "ms_per_launch": ms,
                          "TFLOP/s": tf, "dtype": "bf16 storage, f32 accumulate", "data": "synthetic",
                          "config": {"grid": [D, H, W], "channels": [c, c], "l2": "inputs larger than L2"},
                          "roofline": roof}), flush=True)
    inp = torch.randn((4, D, H, W), generator=g, device=dev)
    target = torch.randn((2, D, H, W), generator=g, device=dev)
    xb = net.to_bf16(inp)
    for _ in range(2):
        net.train_step(xb, target)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = [net.train_step(xb, target) for _ in range(args.steps)]
    sec = (time.perf_counter() - t0) / args.steps
    print(json.dumps({"metric": "learned preconditioner training step", "network": "4-16-16-2, 3x3x3 convolutions",
                      "grid": [D, H, W], "seconds_per_step": sec, "loss_first": losses[0], "loss_last": losses[-1]}),
          flush=True)
    return 0


def misfit_drop_small(torch, dev, iterations=2):
    """Misfit drop per second of the inversion (fwi_step: gradient, L-BFGS direction, Armijo
    line search, update) on the grf_16x16x8 box, from the homogeneous trial medium toward the
    Gaussian-random-field medium whose full 2000-step response is the observed data, with the
    model error before and after (relative L2 of lambda and mu against the true medium)."""
    from paper_1504_08340_gb300 import Context

    w = fi.grf_16x16x8()
    lt, mt = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "true"))
    l0, m0 = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "trial"))
    with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho) as ctx:
        ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
        ctx.set_receivers(w.receivers())
        ctx.set_graphs(True)
        ctx.set_material(lt, mt)
        obs = torch.zeros(ctx.trace_shape(1), dtype=torch.float32, device=dev)
        ctx.forward(out=obs)
        ctx.set_material(l0, m0)
        ctx.step_reset()

        def model_err():
            lam, mu = ctx.get_material()
            return float(np.sqrt(((lam - lt) ** 2).sum() / ((l0 - lt) ** 2).sum())), \
                float(np.sqrt(((mu - mt) ** 2).sum() / ((m0 - mt) ** 2).sum()))

        err0 = model_err()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = [ctx.step(obs, first_step=0.05) for _ in range(iterations)]
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        err1 = model_err()
    J_start, J_end = infos[0].J_old, infos[-1].J_new
    return {"workload": w.name, "iterations": iterations, "J_start": J_start, "J_end": J_end, "seconds": sec,
            "misfit_drop_per_s": (J_start - J_end) / sec,
            "log10_misfit_reduction_per_s": float(np.log10(J_start / J_end)) / sec if J_end > 0 else None,
            "model_error_start": {"lambda": err0[0], "mu": err0[1]},
            "model_error_end": {"lambda": err1[0], "mu": err1[1]},
            "line_search_trials": [i.trials for i in infos]}


def run_batched(args, w):
    """The default benchmark: gradient evaluations of the 16-shot layered workload, all shots
    in shot batches of the tuned width, each sweep a replayed CUDA graph (see the module
    docstring)."""
    import torch

    from paper_1504_08340_gb300 import Context
    from paper_1504_08340_gb300.distributed import max_over_ranks, reduce_gradient

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    full_steps = w.nsteps
    w.nsteps = args.window
    ctx = Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho)
    l0, m0 = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "trial"))
    ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
    ctx.set_receivers(w.receivers())
    ctx.set_material(torch.tensor(l0, device=dev), torch.tensor(m0, device=dev))
    nrec = w.nrec_side ** 2
    # observed data: within a window of tens of steps the waves stay in the top layer, where
    # the true and the starting media agree, so their responses would agree and the residual
    # vanish; seeded smooth synthetic traces (one set per shot, per rank) keep the residual
    # and the gradient nonzero. The work of a step does not depend on the values.
    obs = torch.tensor(np.stack([fi.synthetic_traces(w.nsteps, nrec, 1000 * rank + 100 + s)
                                 for s in range(w.nshots)]), dtype=torch.float32, device=dev).contiguous()
    t_tune = time.perf_counter()
    B = ctx.tune_shot_batch(0, w.nshots, max_batch=min(args.max_batch, w.nshots), steps=min(5, w.nsteps - 1))
    t_tune = time.perf_counter() - t_tune
    ctx.set_shot_batch(B)
    t_tiles = time.perf_counter()
    tiles = ctx.tune_tiles(0, w.nshots, steps=min(3, w.nsteps - 1))
    t_tune += time.perf_counter() - t_tiles
    ctx.set_graphs(not args.no_graphs)
    gl = torch.empty(ctx.mat_shape(), dtype=torch.float64, device=dev)
    gm = torch.empty_like(gl)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def step():
        J, a, b = ctx.adjoint_gradient(obs, 0, w.nshots, g_lambda=gl, g_mu=gm)
        return reduce_gradient(J, a, b) if dist else (J, a, b)

    for _ in range(args.warmup):
        J, _, _ = step()
    ctx.reset_timing()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        J, _, _ = step()
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    _, all_launches = ctx.timing(3)
    ms_max = max_over_ranks(ms, device=dev)
    work = ctx.nelem * 4 * w.nsteps * 2 * w.nshots  # element-stage updates per step and rank
    value = world * work / (ms_max / 1e3)

    # kernel split in a separate pass (timing brackets every stage launch set with events,
    # so it stays out of the timed region)
    ctx.reset_timing()
    ctx.set_timing(True)
    ctx.adjoint_gradient(obs, 0, w.nshots, g_lambda=gl, g_mu=gm)
    ctx.set_timing(False)
    stage_ms, stage_launches = ctx.timing(0)
    grad_ms, _ = ctx.timing(1)
    torch.cuda.synchronize()
    hbm, peak_kind = _peaks()
    per_launch = B * stage_bytes_per_step(ctx, 0) / 4.0 + 8.0 * ctx.nmat  # B shots' state, lambda and mu once
    per_launch_17 = B * stage_bytes_per_step_17(ctx) / 4.0 + 8.0 * ctx.nmat
    avg = stage_ms / max(stage_launches, 1)
    achieved = per_launch / (avg / 1e3) / 1e9 if avg > 0 else None
    achieved_17 = per_launch_17 / (avg / 1e3) / 1e9 if avg > 0 else None

    e2e = None
    if not args.no_e2e:
        obs_h = torch.empty(obs.shape, dtype=torch.float32, pin_memory=True)
        obs_h.copy_(obs.cpu())
        lam_h = torch.tensor(l0).pin_memory()
        mu_h = torch.tensor(m0).pin_memory()
        gl_h = torch.empty(ctx.mat_shape(), dtype=torch.float64, pin_memory=True)
        gm_h = torch.empty_like(gl_h).pin_memory()
        on, ln, mn, gln, gmn = obs_h.numpy(), lam_h.numpy(), mu_h.numpy(), gl_h.numpy(), gm_h.numpy()
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx.set_material(ln, mn)
            Je, _, _ = ctx.adjoint_gradient(on, 0, w.nshots, g_lambda=gln, g_mu=gmn)
        barrier()
        te = (time.perf_counter() - t0) / e2e_steps
        e2e = {"value": world * work / max_over_ranks(te, device=dev), "unit": UNIT_ES, "steps": e2e_steps,
               "h2d_bytes_per_step": int(on.nbytes + ln.nbytes + mn.nbytes),
               "d2h_bytes_per_step": int(gln.nbytes + gmn.nbytes + 8)}
        if not dist:
            assert abs(Je - J) <= 1e-12 * abs(J)

    misfit_drop = None
    if args.inversion_steps > 0:
        misfit_drop = misfit_drop_small(torch, dev, args.inversion_steps)

    if rank == 0:
        # a full-length evaluation (3000 steps) keeps the forward wavefield by sqrt(N)
        # checkpointing, i.e. one more forward sweep: 3 sweeps of stage work instead of 2
        evals_full = value / (ctx.nelem * 4 * full_steps * 3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT_ES, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "mesh": f"{w.nx}x{w.ny}x{w.nz}+{w.npml} PML, h={w.h} m",
                       "nodes": ctx.nnode, "elements": ctx.nelem, "shots": w.nshots, "shot_batch": B,
                       "tiles": {"interior_planes_per_block": tiles[0], "pml_pairs_per_segment": tiles[1]},
                       "autotuning_s": t_tune, "nsteps_per_step": w.nsteps,
                       "nsteps_of_configuration": full_steps, "dt": w.dt, "receivers": nrec,
                       "graphs": not args.no_graphs, "forward_history": "stored every step of the window",
                       "observed": "seeded synthetic traces", "parallelism": f"shot groups x{world}",
                       "l2": f"inputs larger than L2 ({4 * B * 27 * ctx.stride * 4 / 1e9:.0f} GB of RK4 state)"},
            "shot_gradient_evals_per_s_projected": {
                "value": evals_full, "nsteps": full_steps, "sweeps": 3,
                "basis": "the measured element-stage rate, with sqrt(N) checkpointing (one extra forward sweep)"},
            "misfit": J,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": (achieved / hbm) if achieved else None,
                         "traffic": measured_traffic(w.name, B, ctx.nmat),
                         "kernel": "RK4 stage launch set advancing B shots (interior_kernel, shell_kernel, "
                                   "pml_face_kernel, pml_kernel)", "peak_kind": peak_kind,
                         "bytes_per_launch": per_launch, "bytes_model": "13 state accesses per variable per step",
                         "frac_17_access_model": (achieved_17 / hbm) if achieved_17 else None,
                         "avg_launch_ms": avg, "stage_share_of_step": stage_ms / ms if ms > 0 else None},
            "gradient_kernel_ms_per_step": grad_ms,
            "gpu_launches": int(all_launches),
            "clocks": clocks,
            "e2e": e2e,
            "misfit_drop": misfit_drop,
        }
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline_es(w)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_precond_study(args):
    """The learned preconditioner end to end, on the 16x16x8 + 10 PML box (one shot, 600
    steps): training pairs (gradient, model) -> remaining model error from the plain
    inversion (the library's L-BFGS, fwi_step) on --study-train seeded random media,
    the U-Net trained on them, and --study-test held-out media inverted for
    --study-iters iterations by plain L-BFGS and by the network's updates with a
    backtracking line search. One JSON line with the per-iteration means of the misfit
    and of the lambda / mu model errors, and the wall seconds."""
    import torch

    from paper_1504_08340_gb300 import Context, FWIError
    from paper_1504_08340_gb300.precond import UNet, learned_update, precond_inputs, precond_targets

    dev = torch.device("cuda", 0)
    w0 = fi.media_16x16x8(0)
    lam_bg, mu_bg = (float(a.flat[0]) for a in fi.medium(w0, "trial"))
    ctx = Context(w0.nx, w0.ny, w0.nz, w0.npml, w0.h, w0.dt, w0.nsteps, rho=w0.rho)
    ctx.set_sources(w0.sources(), w0.source_dirs(), "ricker", w0.ricker())
    ctx.set_receivers(w0.receivers())
    ctx.set_graphs(True)
    l0, m0 = (torch.tensor(a, dtype=torch.float32, device=dev) for a in fi.medium(w0, "trial"))
    obs = torch.zeros(ctx.trace_shape(1), dtype=torch.float32, device=dev)

    def truth(seed):
        lt, mt = (torch.tensor(a, dtype=torch.float32, device=dev) for a in fi.medium(fi.media_16x16x8(seed), "true"))
        ctx.set_material(lt, mt)
        ctx.forward(out=obs)
        return lt, mt

    def errors(lt, mt):
        lam, mu = (torch.tensor(a, device=dev) for a in ctx.get_material())
        return (float(torch.linalg.vector_norm(lam - lt) / torch.linalg.vector_norm(l0 - lt)),
                float(torch.linalg.vector_norm(mu - mt) / torch.linalg.vector_norm(m0 - mt)))

    # ---- training pairs along the plain inversion
    t0 = time.perf_counter()
    xs, ts = [], []
    for k in range(args.study_train):
        lt, mt = truth(1000 + k)
        ctx.set_material(l0, m0)
        ctx.step_reset()
        for it in range(args.study_pair_iters + 1):
            _, gl, gm = ctx.adjoint_gradient(obs)
            lam, mu = (torch.tensor(a, device=dev) for a in ctx.get_material())
            xs.append(precond_inputs(gl, gm, lam, mu, lam_bg, mu_bg))
            ts.append(precond_targets(lt, mt, lam, mu, lam_bg, mu_bg))
            if it < args.study_pair_iters:
                ctx.step(obs, first_step=0.05)
    t_pairs = time.perf_counter() - t0
    # ---- training
    net = UNet(4, 2, tuple(args.study_widths), ctx.mat_shape(), seed=0, lr=args.study_lr)
    xb = [net.to_bf16(x) for x in xs]
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    losses = []
    for step in range(args.study_train_steps):
        i = int(rng.integers(len(xb)))
        losses.append(net.train_step(xb[i], ts[i]))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # ---- evaluation on held-out media
    # plain L-BFGS, L-BFGS with the lambda-direction biasing (25) (W = 1 at the first
    # iteration, lowered linearly to 0 by the 50th, as Sec. 3.3.3 schedules it), and the
    # network's updates with a backtracking line search
    hist = {"plain": [], "biased": [], "learned": []}
    for k in range(args.study_test):
        lt, mt = truth(5000 + k)
        for method in ("plain", "biased", "learned"):
            ctx.set_material(l0, m0)
            ctx.step_reset()
            J = ctx.misfit(obs)
            rec = [(0.0, J, *errors(lt, mt))]
            torch.cuda.synchronize()
            t = time.perf_counter()
            for it in range(args.study_iters):
                if method == "plain":
                    J = ctx.step(obs, first_step=0.05).J_new
                elif method == "biased":
                    J = ctx.step(obs, first_step=0.05, bias_w=max(0.0, 1.0 - it / 50.0)).J_new
                else:
                    J, gl, gm = ctx.adjoint_gradient(obs)
                    lam, mu = (torch.tensor(a, device=dev) for a in ctx.get_material())
                    dl, dm = learned_update(net, gl, gm, lam, mu, lam_bg, mu_bg)
                    gtd = float((gl * dl).sum() + (gm * dm).sum())
                    if not gtd < 0:  # not a descent direction: steepest descent, 5 % of the model
                        s_ = 0.05 * float(torch.maximum(lam.abs().max(), mu.abs().max())) / float(
                            torch.maximum(gl.abs().max(), gm.abs().max()))
                        dl, dm = -s_ * gl, -s_ * gm
                        gtd = float((gl * dl).sum() + (gm * dm).sum())
                    alpha, Jn = 1.0, None
                    for _ in range(8):  # Armijo backtracking (Algorithm 1), c1 = 1e-4
                        tl, tm = (lam + alpha * dl).clamp_min(1.0), (mu + alpha * dm).clamp_min(1.0)
                        try:  # a trial beyond the time-step limit counts as a rejected trial
                            ctx.set_material(tl.to(torch.float32).contiguous(), tm.to(torch.float32).contiguous())
                            Jn = ctx.misfit(obs)
                        except FWIError:
                            Jn = float("inf")
                        if Jn <= J + 1e-4 * alpha * gtd:
                            break
                        alpha *= 0.5
                    else:
                        ctx.set_material(lam.to(torch.float32).contiguous(), mu.to(torch.float32).contiguous())
                        Jn = J
                    J = Jn
                torch.cuda.synchronize()
                rec.append((time.perf_counter() - t, J, *errors(lt, mt)))
            hist[method].append(rec)
    win = max(1, min(50, len(losses) // 10))  # mean loss over the first and the last tenth (at most 50 steps)
    out = {"metric": "learned preconditioner study", "workload": "media_16x16x8 (16x16x8 + 10 PML, 600 steps, 1 shot)",
           "network": {"widths": list(args.study_widths), "params": net.num_params(), "steps": args.study_train_steps,
                       "loss_window": win, "loss_first": float(np.mean(losses[:win])),
                       "loss_last": float(np.mean(losses[-win:]))},
           "pairs": len(xs), "train_media": args.study_train, "test_media": args.study_test,
           "seconds": {"pairs": t_pairs, "training": t_train}}
    for method, recs in hist.items():
        a = np.array(recs)  # [media][iteration][t, J, err_lambda, err_mu]
        J0 = a[:, :1, 1]
        out[method] = {"seconds": a[:, :, 0].mean(0).round(3).tolist(),
                       "misfit_rel": (a[:, :, 1] / J0).mean(0).round(5).tolist(),
                       "err_lambda": a[:, :, 2].mean(0).round(5).tolist(),
                       "err_mu": a[:, :, 3].mean(0).round(5).tolist()}
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


def _bytes_in_use(torch, dev):
    free, total = torch.cuda.mem_get_info(dev)
    return total - free


def run_full_evaluation(args):
    """One-off measurement: the whole 16-shot gradient evaluation of the layered workload at
    its full 3000 steps, observed traces computed from the true medium, the adjoint fed by
    sqrt(T) compact snapshots with recompute, shots in groups of --full-batch, each sweep a
    replayed CUDA graph. --steps evaluations are timed after --warmup (default 0 here: one
    evaluation is minutes of GPU work; its one-time graph recording and allocations are
    under a second of it). One JSON line."""
    import math

    import torch

    from paper_1504_08340_gb300 import Context

    w = fi.layered_96x96x48()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = _bytes_in_use(torch, dev)
    ctx = Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho)
    ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
    ctx.set_receivers(w.receivers())
    ctx.set_shot_batch(args.full_batch)
    ctx.set_graphs(True)
    lt, mt = (torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev) for a in fi.medium(w, "true"))
    l0, m0 = (torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev) for a in fi.medium(w, "trial"))
    obs = torch.empty(ctx.trace_shape(w.nshots), dtype=torch.float32, device=dev)
    t = time.perf_counter()
    ctx.set_material(lt, mt)
    ctx.forward(0, w.nshots, out=obs)
    torch.cuda.synchronize()
    t_obs = time.perf_counter() - t
    ctx.set_material(l0, m0)
    ctx.set_checkpointing(-1)
    gl = torch.empty(ctx.mat_shape(), dtype=torch.float64, device=dev)
    gm = torch.empty_like(gl)
    for _ in range(args.warmup):
        ctx.adjoint_gradient(obs, 0, w.nshots, g_lambda=gl, g_mu=gm)
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        J, _, _ = ctx.adjoint_gradient(obs, 0, w.nshots, g_lambda=gl, g_mu=gm)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    every = math.ceil(math.sqrt(w.nsteps))
    work = ctx.nelem * 4 * w.nsteps * 2 * w.nshots  # forward and adjoint sweeps; the recompute is not counted
    print(json.dumps({
        "metric": "full-length 16-shot gradient evaluations/s", "value": 1e3 / ms, "unit": "evaluations/s",
        "workload": "layered_96x96x48", "nsteps": w.nsteps, "shots": w.nshots, "shot_batch": args.full_batch,
        "checkpoint": {"interval": every, "snapshots_per_shot": math.ceil(w.nsteps / every), "kind": "compact"},
        "observed": "forward traces of the true medium", "warmup": args.warmup, "steps": args.steps,
        "seconds_per_evaluation": ms / 1e3, "shot_gradient_evals_per_s": w.nshots * 1e3 / ms,
        "element_stage_updates_per_s": work / (ms / 1e3), "J": J, "observed_forward_s": t_obs,
        "device_bytes": _bytes_in_use(torch, dev) - base, "clocks": clocks}))


def run_large_iteration(args):
    """One-off measurement: one torch.autograd-driven inversion iteration on the large
    workload (160x160x80 + 12 PML, 64 shots, 4000 steps, 80x80 receivers) over its first
    --large-shots shots. Observed traces come from the true medium; J and g_mis come from
    MisfitFunction (forward, misfit, adjoint with sqrt(T) compact snapshots); the direction
    is -M~^-1 g_mis scaled to max |d| = 5 % of max |m|; Armijo backtracking (Algorithm 1,
    c1 = 1e-4, halving) evaluates misfit-only trials. One JSON line with the seconds of
    each part and the device memory the context holds."""
    import math

    import torch

    from paper_1504_08340_gb300 import Context, FWIError
    from paper_1504_08340_gb300.autograd import misfit

    w = fi.large_160x160x80()
    S = args.large_shots
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = _bytes_in_use(torch, dev)
    ctx = Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho)
    ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
    ctx.set_receivers(w.receivers())
    ctx.set_shot_batch(min(S, args.full_batch))
    ctx.set_graphs(True)
    lt, mt = (torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev) for a in fi.medium(w, "true"))
    l0, m0 = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "trial"))
    obs = torch.empty(ctx.trace_shape(S), dtype=torch.float32, device=dev)
    t = time.perf_counter()
    ctx.set_material(lt, mt)
    ctx.forward(0, S, out=obs)
    torch.cuda.synchronize()
    t_obs = time.perf_counter() - t
    del lt, mt
    ctx.set_checkpointing(-1)
    lam = torch.tensor(l0, device=dev, requires_grad=True)
    mu = torch.tensor(m0, device=dev, requires_grad=True)
    t = time.perf_counter()
    J = misfit(ctx, lam, mu, obs, 0, S)
    J.backward()
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t
    held = _bytes_in_use(torch, dev) - base
    J0 = float(J.detach())
    mt_inv = 1.0 / torch.tensor(ctx.mass_tilde(), device=dev)
    gl, gm = lam.grad.double(), mu.grad.double()
    ml, mm = lam.detach().double(), mu.detach().double()
    dl, dm = -mt_inv * gl, -mt_inv * gm
    scale = 0.05 * float(torch.maximum(ml.abs().max(), mm.abs().max())) / float(torch.maximum(dl.abs().max(), dm.abs().max()))
    dl, dm = scale * dl, scale * dm
    gtd = float((gl * dl).sum() + (gm * dm).sum())
    t = time.perf_counter()
    alpha, trials, J1 = 1.0, 0, J0
    for _ in range(args.large_backtracks):
        trials += 1
        try:
            ctx.set_material((ml + alpha * dl).float().contiguous(), (mm + alpha * dm).float().contiguous())
            Jt = ctx.misfit(obs, 0, S)
        except FWIError:  # beyond the time-step limit: a rejected trial
            Jt = float("inf")
        if Jt <= J0 + 1e-4 * alpha * gtd:
            J1 = Jt
            break
        alpha *= 0.5
    else:
        alpha = 0.0
    torch.cuda.synchronize()
    t_ls = time.perf_counter() - t
    every = math.ceil(math.sqrt(w.nsteps))
    work = ctx.nelem * 4 * w.nsteps * 2 * S  # forward and adjoint sweeps of the gradient
    print(json.dumps({
        "metric": "large autograd inversion iteration", "workload": "large_160x160x80",
        "mesh": f"{w.nx}x{w.ny}x{w.nz}+{w.npml} PML", "elements": ctx.nelem, "nodes": ctx.nnode, "nsteps": w.nsteps,
        "shots": S, "shots_of_configuration": w.nshots, "shot_batch": min(S, args.full_batch),
        "checkpoint": {"interval": every, "snapshots_per_shot": math.ceil(w.nsteps / every), "kind": "compact"},
        "device_bytes_held": held, "J_start": J0, "J_end": J1, "alpha": alpha, "line_search_trials": trials,
        "directional_derivative": gtd,
        "seconds": {"observed_forward": t_obs, "misfit_and_gradient": t_grad, "line_search": t_ls},
        "element_stage_updates_per_s": work / t_grad,
        "gradient_seconds_per_shot": t_grad / S,
        "full_iteration_projected_s": (t_grad + t_ls) * w.nshots / S}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--inversion-steps", type=int, default=2,
                    help="iterations of Algorithm 2 (fwi_step) timed after the gradient benchmark (0: skip)")
    ap.add_argument("--checkpoint", type=int, default=0, metavar="K",
                    help="forward history of the adjoint: 0 stored every step, K > 0 snapshots every K "
                         "steps with recompute, K < 0 every ceil(sqrt(nsteps)) steps")
    ap.add_argument("--profile-forward", type=int, default=0, metavar="NSTEPS",
                    help="profiling aid: run only short forward sweeps (NSTEPS RK4 steps) on the same mesh")
    ap.add_argument("--shot-batch-sweep", type=str, default="", metavar="B1,B2,...",
                    help="instead of the headline benchmark: the 16-shot layered 96x96x48 mesh with B shots "
                         "per stage launch, one line per B")
    ap.add_argument("--sweep-nsteps", type=int, default=100,
                    help="RK4 steps of the shot-batch sweep (the configuration has 3000)")
    ap.add_argument("--profile-gradient", type=int, default=0, metavar="NSTEPS",
                    help="profiling aid: run only short gradient evaluations (NSTEPS RK4 steps) on the same mesh")
    ap.add_argument("--precond-bench", action="store_true",
                    help="instead of the headline benchmark: the learned preconditioner's kernels")
    ap.add_argument("--workload", default="layered_96x96x48", choices=sorted(WORKLOADS),
                    help="layered_96x96x48: the batched 16-shot step (default); grf_64x64x32: full-length "
                         "single-shot evaluations")
    ap.add_argument("--window", type=int, default=50,
                    help="time steps per step of the batched workload (of its 3000)")
    ap.add_argument("--max-batch", type=int, default=16, help="largest shot batch the autotuner may pick")
    ap.add_argument("--no-graphs", action="store_true", help="direct launches instead of replayed CUDA graphs")
    ap.add_argument("--e2e-steps", type=int, default=5, help="steps of the end-to-end measurement (at most --steps)")
    ap.add_argument("--precond-study", action="store_true",
                    help="instead of the headline benchmark: train and evaluate the learned preconditioner")
    ap.add_argument("--study-train", type=int, default=200)
    ap.add_argument("--study-test", type=int, default=20)
    ap.add_argument("--study-iters", type=int, default=20)
    ap.add_argument("--study-pair-iters", type=int, default=2)
    ap.add_argument("--study-train-steps", type=int, default=3000)
    ap.add_argument("--study-lr", type=float, default=3e-4)
    ap.add_argument("--study-widths", type=int, nargs=3, default=[28, 56, 112])
    ap.add_argument("--full-evaluation", action="store_true",
                    help="instead of the headline benchmark: whole 3000-step 16-shot gradient evaluations of "
                         "the layered workload (minutes each; --warmup defaults to 0 here)")
    ap.add_argument("--full-batch", type=int, default=4, help="shot batch of --full-evaluation / --large-iteration")
    ap.add_argument("--large-iteration", action="store_true",
                    help="instead of the headline benchmark: one autograd inversion iteration on the "
                         "160x160x80 + 12 PML workload (4000 steps) over --large-shots shots")
    ap.add_argument("--large-shots", type=int, default=1)
    ap.add_argument("--large-backtracks", type=int, default=6)
    ap.add_argument("--traffic-json", metavar="CSV",
                    help="write profiles/stage_traffic_layered_96x96x48.json from an ncu CSV log of the "
                         "stage-traffic capture (see TRAFFIC_COMMAND) and exit")
    args = ap.parse_args()
    if args.traffic_json:
        rec = traffic_summary(args.traffic_json, "layered_96x96x48")
        with open(os.path.join(ROOT, "profiles", "stage_traffic_layered_96x96x48.json"), "w") as f:
            json.dump(rec, f, indent=1)
        print(json.dumps({k: v for k, v in rec.items() if k != "per_kernel"}))
        return
    if args.full_evaluation:
        if "--warmup" not in sys.argv:
            args.warmup = 0
        if "--steps" not in sys.argv:
            args.steps = 1
        return run_full_evaluation(args)
    if args.large_iteration:
        return run_large_iteration(args)
    if args.precond_study:
        return run_precond_study(args)
    if args.precond_bench:
        return run_precond_bench(args)
    if args.shot_batch_sweep:
        args.shot_batches = [int(b) for b in args.shot_batch_sweep.split(",")]
        return run_batch_sweep(args)
    w = workload(args.workload)
    if args.profile_forward:
        return profile_forward(w, args.profile_forward, max(args.steps, 1), args.max_batch)
    if args.profile_gradient:
        return profile_gradient(w, args.profile_gradient, max(args.steps, 1), args.max_batch)
    if args.impl == "reference":
        return run_reference(args, w)
    if w.nshots > 1:
        return run_batched(args, w)
    return run_single(args, w)


def run_single(args, w):
    """Full-length single-shot gradient evaluations (--workload grf_64x64x32)."""
    import torch

    from paper_1504_08340_gb300.distributed import max_over_ranks

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx, obs, (l0, m0) = setup(w, torch, dev)
    ctx.set_checkpointing(args.checkpoint)
    gl = torch.empty(ctx.mat_shape(), dtype=torch.float64, device=dev)
    gm = torch.empty_like(gl)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        J, _, _ = ctx.adjoint_gradient(obs, g_lambda=gl, g_mu=gm)
    ctx.reset_timing()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        J, _, _ = ctx.adjoint_gradient(obs, g_lambda=gl, g_mu=gm)
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    _, all_launches = ctx.timing(3)
    ms_max = max_over_ranks(ms, device=dev)
    # kernel split in a separate pass (timing brackets every stage launch set with events,
    # so it stays out of the timed region)
    ctx.reset_timing()
    ctx.set_timing(True)
    ctx.adjoint_gradient(obs, g_lambda=gl, g_mu=gm)
    ctx.set_timing(False)
    stage_ms, stage_launches = ctx.timing(0)
    grad_ms, grad_launches = ctx.timing(1)
    value = world / (ms_max / 1e3)

    hbm, peak_kind = _peaks()
    bytes_step = stage_bytes_per_step(ctx, ctx.nmat)
    total_stage_bytes = bytes_step / 4.0 * stage_launches
    achieved = total_stage_bytes / (stage_ms / 1e3) / 1e9 if stage_ms > 0 else None
    elem_stage = ctx.nelem * 4 * w.nsteps * 2  # forward + adjoint sweeps

    e2e = None
    if not args.no_e2e:
        obs_h = torch.empty(ctx.trace_shape(1), dtype=torch.float32, pin_memory=True)
        obs_h.copy_(obs.cpu())
        lam_h = torch.tensor(l0).pin_memory()
        mu_h = torch.tensor(m0).pin_memory()
        gl_h = torch.empty(ctx.mat_shape(), dtype=torch.float64, pin_memory=True)
        gm_h = torch.empty_like(gl_h).pin_memory()
        on, mn, gln, gmn = obs_h.numpy(), lam_h.numpy(), gl_h.numpy(), gm_h.numpy()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_material(mn, mu_h.numpy())
            Je, _, _ = ctx.adjoint_gradient(on, g_lambda=gln, g_mu=gmn)
        barrier()
        te = (time.perf_counter() - t0) / args.steps
        e2e = {"value": world / max_over_ranks(te, device=dev), "unit": UNIT,
               "h2d_bytes_per_step": int(on.nbytes + mn.nbytes + mu_h.numpy().nbytes),
               "d2h_bytes_per_step": int(gln.nbytes + gmn.nbytes + 8)}
        assert abs(Je - J) <= 1e-12 * abs(J)

    misfit_drop = None
    if args.inversion_steps > 0:
        # misfit drop per second of the full inversion iteration (gradient, L-BFGS direction,
        # Armijo line search, update), from the trial model
        ctx.set_material(torch.tensor(l0, device=dev), torch.tensor(m0, device=dev))
        ctx.step_reset()
        barrier()
        t0 = time.perf_counter()
        infos = [ctx.step(obs, first_step=0.05) for _ in range(args.inversion_steps)]
        barrier()
        sec = time.perf_counter() - t0
        J_start, J_end = infos[0].J_old, infos[-1].J_new
        misfit_drop = {"iterations": args.inversion_steps, "J_start": J_start, "J_end": J_end, "seconds": sec,
                       "misfit_drop_per_s": (J_start - J_end) / sec,
                       "log10_misfit_reduction_per_s": float(np.log10(J_start / J_end)) / sec if J_end > 0 else None,
                       "line_search_trials": [i.trials for i in infos]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "mesh": f"{w.nx}x{w.ny}x{w.nz}+{w.npml} PML, h={w.h} m",
                       "nodes": ctx.nnode, "elements": ctx.nelem, "nsteps": w.nsteps, "dt": w.dt,
                       "receivers": w.nrec_side ** 2, "shots_per_step_per_gpu": 1,
                       "parallelism": f"shot replicas x{world}",
                       "forward_history": ("stored every step" if args.checkpoint == 0 else
                                           f"checkpoint every {args.checkpoint if args.checkpoint > 0 else 'ceil(sqrt(N))'}"
                                           " steps, recomputed"),
                       "l2": "inputs larger than L2 (1 GB state, 26 GB history per step)"},
            "element_stage_updates_per_s": value * elem_stage,
            "misfit": J,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": (achieved / hbm) if achieved else None, "traffic": measured_traffic(w.name),
                         "kernel": "RK4 stage launch set (interior_kernel, shell_kernel, pml_face_kernel, pml_kernel)",
                         "peak_kind": peak_kind, "frac_17_access_model": (
                             stage_bytes_per_step_17(ctx) / 4.0 / (stage_ms / max(stage_launches, 1) / 1e3) / 1e9 / hbm
                             if stage_ms > 0 else None),
                         "bytes_per_launch": bytes_step / 4.0,
                         "avg_launch_ms": stage_ms / max(stage_launches, 1),
                         "stage_share_of_step": stage_ms / ms if ms > 0 else None},
            "gradient_kernel_ms_per_step": grad_ms,
            "gpu_launches": int(all_launches),
            "clocks": clocks,
            "e2e": e2e,
            "misfit_drop": misfit_drop,
        }
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
