"""Benchmark: grid-point RK-stage updates per second of the residual path.

Default workload (N = 1): the 3D Taylor-Green vortex, compressible
Navier-Stokes at Re 1600, Ma 0.1, Pr 0.71, on one periodic 384^3 block with a
0.02 L sinusoidal warp (56.6 M nodes) -- the largest precision-form
configuration.  The line's ``value`` is the FP64 form; ``mixed`` carries the
same workload in the mixed FP32/FP64 form and the ratio.  A "step" is one
full RK3 step (three stages) over the block; value = nodes * 3 * steps /
device time (Mpts/s).

--impl reference times the FP64 CPU oracle (as it stands) on this host's
cores on the same workload instead, each timed step a bounded sample of it.
Under torchrun (N > 1) each rank runs an independent replica on its own GPU
(the path keeps every block on one GPU).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point RK-stage updates/s (Mpts/s) mixed vs FP64 on 1 GB300; HBM GB/s fraction"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}

# Algorithmic work of one flux-sweep launch per interior node (one direction):
# modified AFWENO inviscid part and, for Navier-Stokes, the projection of the
# node stress tensor on the direction's metric and its central derivative
# (counts derived operation by operation, a multiply and an add counted
# apart; the stress tensor itself is formed once per node by the gradient
# kernel).
FLUX_FLOPS_INV = 1060
FLUX_FLOPS_VISC = 50
# The FP64 form reads the sweeps' unit normals, formed once from the static
# metrics: per node and direction the sixth-order midpoint face metric
# (3 x 9), its norm, square root and normalisation (10) and the node
# normal's norm and normalisation (9) are not part of a stage.
FLUX_FLOPS_STATIC_FP64 = 46
RK_FLOPS = 30   # R = -J A and the three-term combination, five components


def stage_bytes_per_node(precision):
    """Compulsory HBM bytes of one RK stage per interior node (the
    algorithmic bytes of the hot-path scope): the FP64 metrics and J
    (10 words), Q^n, the stage input Q^(k) (the same array as Q^n in stage
    1) and the output Q^(k+1), all FP64; the mixed form also reads and
    writes the FP32 copy of the state (5 + 5 words of 4 B).  Gradients,
    stresses, face states and accumulators are intermediates.  Mean over the
    three stages: FP64 (160 + 200 + 200) / 3, mixed (200 + 240 + 240) / 3."""
    per_stage = [(10 + 5 + 5) * 8, (10 + 5 + 5 + 5) * 8, (10 + 5 + 5 + 5) * 8]
    if precision == "mixed":
        per_stage = [b + 10 * 4 for b in per_stage]
    return sum(per_stage) / 3.0


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per interior node
# of one launch of each stage kernel, from one ncu capture of the kernels
# whose sources hash to TRAFFIC_SOURCES_SHA: the 192^3 Taylor-Green block
# (7,077,888 nodes) with the fixed tiles, the mean over the three RK
# stages' launches of the second warm-up step:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       --clock-control none -k regex:'k_flux|k_grad|k_prep|k_rk_stage'
#       -s 22 -c 18 (mixed; FP64: -s 15 -c 15) --csv
#       python bench.py --workload tgv192 --steps 1 --warmup 3 --no-cpu-baseline
#       --no-autotune --forms mixed (or fp64)
# Scaled to the benchmark's workload by its node count; null when the
# kernel sources differ from the captured ones.
TRAFFIC_SOURCES_SHA = "c3135e334f6465f9"
TRAFFIC_PER_NODE = {
    ("mixed", "prep"): 21.1, ("mixed", "stress"): 100.9, ("mixed", "flux_xi"): 97.7,
    ("mixed", "flux_eta"): 115.6, ("mixed", "flux_zeta"): 144.7, ("mixed", "rk_stage"): 185.2,
    ("fp64", "prep"): 196.8, ("fp64", "stress"): 211.8, ("fp64", "flux_xi"): 352.0,
    ("fp64", "flux_eta"): 404.9, ("fp64", "flux_zeta_rk"): 444.0,
}

# Algorithmic work per node and RK stage besides the three sweeps: the
# stress tensor (12 gradients by the sixth-order difference and the chain
# rule, the stress and heat flux; about 200 flops), the primitives (10) and
# the RK combination (30).
STAGE_FLOPS_OTHER = 240


def kernel_sources_sha():
    """sha256 (first 16 hex digits) of the library's CUDA sources and headers,
    in name order: the key of the traffic table."""
    import hashlib
    import glob
    h = hashlib.sha256()
    for path in sorted(glob.glob(os.path.join(ROOT, "paper_2006_07964_gb300", "csrc", "*"))):
        with open(path, "rb") as fh:
            h.update(os.path.basename(path).encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


WORKLOADS = {
    "tgv128": ("Taylor-Green vortex, NS Re1600 Ma0.1 Pr0.71, warped periodic 128^3 block", lambda W: W.tgv(128)),
    "tgv256": ("Taylor-Green vortex, NS Re1600 Ma0.1 Pr0.71, warped periodic 256^3 block", lambda W: W.tgv(256)),
    "tgv384": ("Taylor-Green vortex, NS Re1600 Ma0.1 Pr0.71, warped periodic 384^3 block", lambda W: W.tgv(384)),
    "tgv192": ("Taylor-Green vortex, NS Re1600 Ma0.1 Pr0.71, warped periodic 192^3 block", lambda W: W.tgv(192)),
    "vortex32": ("isentropic vortex, Euler, warped periodic 32^3 block", lambda W: W.vortex(32)),
    "ogrid": ("cylinder O-grid, NS Ma0.2 Re3900, 8 blocks, 3,538,944 nodes", lambda W: W.ogrid()),
    "batch64": ("64 isentropic-vortex instances, edges from {24..96}, seeded", lambda W: W.batch(64)),
    "shock512": ("two Sod shock tubes in a warped periodic 512x64x64 box, Euler",
                 lambda W: W.shocktube((512, 64, 64), amp=0.02)),
    "shockvortex512": ("Mach 1.2 shock into an isentropic vortex, warped periodic 512x256x16 box, Euler",
                       lambda W: W.shock_vortex((512, 256, 16), amp=0.02)),
}


# The oracle's timed samples of workloads too large to step on the host within
# minutes: the same flow on a coarser grid (the per-node work is the same).
ORACLE_SAMPLE = {"tgv256": "tgv128", "tgv384": "tgv128"}


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


class Ranks:
    """Replica bookkeeping for torchrun launches: every rank runs the whole
    workload on its own GPU (the path keeps every block on one GPU, so there
    is no data exchange); a barrier brackets the timed region and the job's
    time is the maximum over ranks."""

    def __init__(self, world):
        self.world = world

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, x):
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def throughput(self, npts, steps, seconds):
        """Whole-job Mpts/s: all replicas' node RK-stage updates over the
        slowest rank's time."""
        return self.world * npts * 3 * steps / seconds / 1e6


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return {"hbm_gbs": float(p["hbm_gbs"]), "src": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": PEAKS_FALLBACK["hbm_gbs"], "src": "fallback"}


def alu_peaks(hx):
    """FP64 and FP32 FMA throughput of this GPU measured in this run by the
    probe of include/hx_probe.h (TFLOP/s, 2 flops per FMA)."""
    f64, f32 = hx.probe_fma_peaks()
    return {"fp64_tflops": f64, "fp32_tflops": f32, "alu_src": "measured in this run (FMA-chain probe, hx_probe.h)"}


def page_locked(torch, arrays):
    """Page-locks host numpy arrays for the copy engines (cudaHostRegister;
    release with page_unlocked).  Measured on a GB300 host: 2.26 GB each way
    in 13 ms, steadily, against 20-160 ms, varying from run to run, for the
    same copies from buffers of torch's pin_memory()."""
    cudart = torch.cuda.cudart()
    done = []
    for a in arrays:
        rc = int(cudart.cudaHostRegister(a.ctypes.data, a.nbytes, 0))
        if rc != 0:
            page_unlocked(torch, done)
            raise RuntimeError("cudaHostRegister failed (error %d)" % rc)
        done.append(a)


def page_unlocked(torch, arrays):
    cudart = torch.cuda.cudart()
    for a in arrays:
        cudart.cudaHostUnregister(a.ctypes.data)


def run_form(torch, hx, w, precision, steps, warmup, stream, dt, autotune=1):
    """Times `steps` graph-replayed RK3 steps with CUDA events on the
    context's stream; returns (seconds, ctx)."""
    ctx = hx.from_workload(w, precision=precision, stream=stream.cuda_stream, autotune=autotune)
    ctx.step(warmup, dt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.step(steps, dt)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3, ctx


def sweep_flops_per_node(name, precision, viscous):
    """Algorithmic flops of one sweep launch per node (FP64: less the static
    normals; the fused FP64 zeta sweep adds the RK combination)."""
    f = FLUX_FLOPS_INV + (FLUX_FLOPS_VISC if viscous else 0)
    if precision == "fp64":
        f -= FLUX_FLOPS_STATIC_FP64
    if name == "flux_zeta_rk":
        f += RK_FLOPS
    return f


def roofline_for(ctx, w, precision, steps, dt, peaks, ms_per_step):
    """Per-kernel CUDA-event durations of `steps` launch-by-launch steps of
    the same workload on the same stream, and the roofline of the dominant
    kernel.  A flux sweep is bound by its arithmetic (FP64 pipe; FP32 issue
    in the mixed form): achieved = its algorithmic flops per launch / launch
    time against the FMA peak measured in this run; a point kernel by HBM.
    hbm_view: the stage's algorithmic bytes (stage_bytes_per_node x nodes)
    over this launch's time; traffic_view: the kernel's measured DRAM bytes
    over its time; stage_view: the stage's bytes and flops over the mean
    graph-replayed stage time."""
    stats = ctx.profile_step(steps, dt)
    name, (launches, tot) = max(stats.items(), key=lambda kv: kv[1][1])
    per_launch_s = tot / launches / 1e3
    npts = w.npts
    out = {"kernel": name, "launch_ms": tot / launches, "share": tot / sum(v[1] for v in stats.values())}
    alu_peak = peaks["fp64_tflops"] if precision == "fp64" else peaks["fp32_tflops"]
    alu_src = "%s FMA, %s" % ("FP64" if precision == "fp64" else "FP32", peaks["alu_src"])
    bytes_ = stage_bytes_per_node(precision) * npts
    hbm = {"achieved": bytes_ / per_launch_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": bytes_ / per_launch_s / 1e9 / peaks["hbm_gbs"], "peak_src": peaks["src"],
           "note": "the whole stage's algorithmic bytes over this launch"}
    if name.startswith("flux_"):
        tfl = sweep_flops_per_node(name, precision, w.viscous) * npts / per_launch_s / 1e12
        out.update({"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s", "frac": tfl / alu_peak,
                    "peak_src": alu_src, "hbm_view": hbm})
    else:
        out.update({"bound": "hbm", "achieved": hbm["achieved"], "peak": hbm["peak"], "unit": "GB/s",
                    "frac": hbm["frac"], "peak_src": peaks["src"]})
    stage_s = ms_per_step / 3.0 / 1e3
    stage_flops = (3 * sweep_flops_per_node("flux_xi", precision, w.viscous) + STAGE_FLOPS_OTHER) * npts
    out["stage_view"] = {"stage_ms": stage_s * 1e3, "bytes_per_node": stage_bytes_per_node(precision),
                         "hbm_achieved": bytes_ / stage_s / 1e9, "hbm_frac": bytes_ / stage_s / 1e9 / peaks["hbm_gbs"],
                         "flops_per_node": stage_flops / npts, "alu_achieved": stage_flops / stage_s / 1e12,
                         "alu_frac": stage_flops / stage_s / 1e12 / alu_peak}
    sha = kernel_sources_sha()
    per_node = TRAFFIC_PER_NODE.get((precision, name)) if sha == TRAFFIC_SOURCES_SHA else None
    out["traffic"] = per_node * npts if per_node is not None else None
    if per_node is not None:
        out["traffic_src"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, %.1f B per node on "
                              "192^3 scaled by the nodes (profiles/traffic_tgv192.md)" % per_node)
        out["traffic_view"] = {"achieved": per_node * npts / per_launch_s / 1e9, "unit": "GB/s",
                               "frac": per_node * npts / per_launch_s / 1e9 / peaks["hbm_gbs"]}
    else:
        out["traffic_src"] = "null: no ncu capture of kernel sources %s" % sha
    out["per_kernel_ms"] = {k: v[1] / v[0] for k, v in stats.items()}
    out["autotune"] = ctx.tuning()
    return out


def cpu_baseline(w, steps=2, single_thread_w=None):
    """The FP64 oracle as it stands on this host's cores: `steps` whole RK3
    steps of the workload on all cores; then, on one thread, `steps` whole
    steps of `single_thread_w` (a bounded sample of the same flow; the
    workload itself when None)."""
    import oracle
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    P = oracle.from_workload(w)
    dt, _ = P.dt(0.5)
    t0 = time.perf_counter()
    P.step(steps, dt)
    el = time.perf_counter() - t0
    out = {"value": w.npts * 3 * steps / el / 1e6, "unit": "Mpts/s", "cores": oracle.max_threads(),
           "kind": "oracle", "sample": "%d full RK3 steps of the %d-node workload, %.1f s" % (steps, w.npts, el)}
    del P
    s = single_thread_w if single_thread_w is not None else w
    oracle.set_threads(1)
    P1 = oracle.from_workload(s)
    dt1, _ = P1.dt(0.5)
    t0 = time.perf_counter()
    P1.step(steps, dt1)
    el1 = time.perf_counter() - t0
    oracle.set_threads(threads)
    out["single_thread"] = {"value": s.npts * 3 * steps / el1 / 1e6, "unit": "Mpts/s", "cores": 1,
                            "sample": "%d full RK3 steps of %s (%d nodes), %.1f s"
                                      % (steps, "the same workload" if s is w else s.name, s.npts, el1)}
    return out


def _rel_errors(a, b):
    """Relative L2 and L-infinity of rho, rho u (vector) and E between two
    states [5][...] (b is the reference)."""
    out_l2, out_inf = {}, {}
    for name, idx in (("rho", [0]), ("rho_u", [1, 2, 3]), ("E", [4])):
        da, db = a[idx], b[idx]
        out_l2[name] = float(np.sqrt(((da - db) ** 2).sum() / (db ** 2).sum()))
        out_inf[name] = float(np.abs(da - db).max() / np.abs(db).max())
    return out_l2, out_inf


def precision_report(torch, hx, w, steps, warmup, stream):
    """Mixed form against the FP64 form on the same workload, same dt, same
    number of steps: throughput of each and the relative L2 / L-infinity
    error of rho, rho u, E after the steps (the FP64 GPU path, checked
    against the oracle at full size elsewhere, is the reference)."""
    probe = hx.from_workload(w, precision="fp64", stream=stream.cuda_stream)
    dt, _ = probe.compute_dt(0.5)
    probe.close()
    res = {}
    states = {}
    for form in ("fp64", "mixed"):
        ctx = hx.from_workload(w, precision=form, stream=stream.cuda_stream)
        ctx.step(warmup, dt)          # warm-up, autotune, graph capture
        for b, blk in enumerate(w.blocks):
            ctx.set_state(b, blk.q0)  # restart from the initial state
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(steps, dt)
        e1.record(stream)
        e1.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        res[form] = {"mpts": w.npts * 3 * steps / secs / 1e6, "ms_per_step": secs / steps * 1e3}
        states[form] = [ctx.get_state(b) for b in range(len(w.blocks))]
        ctx.close()
    a = np.concatenate([s.reshape(5, -1) for s in states["mixed"]], axis=1)
    b = np.concatenate([s.reshape(5, -1) for s in states["fp64"]], axis=1)
    l2, linf = _rel_errors(a, b)
    return {"report": "precision", "workload": w.name, "points": w.npts, "steps": steps, "dt": dt,
            "time": dt * steps, "fp64": res["fp64"], "mixed": res["mixed"],
            "ratio_mixed_vs_fp64": res["mixed"]["mpts"] / res["fp64"]["mpts"],
            "rel_l2_mixed_vs_fp64": l2, "rel_linf_mixed_vs_fp64": linf}


def batch_report(torch, hx, w, steps, warmup, stream):
    """Many uneven instances: all blocks in one context (one launch per
    kernel family over the block / line-group work lists, the RK step in one
    CUDA graph, per-instance dt) against one context per instance stepped one
    after another, in both forms."""
    from paper_2006_07964_gb300 import workloads as W
    out = {"report": "batch", "workload": w.name, "instances": len(w.blocks), "points": w.npts, "steps": steps}
    probe = hx.from_workload(w, precision="fp64", stream=stream.cuda_stream)
    _, dts = probe.compute_dt(0.5)
    probe.close()
    for form in ("fp64", "mixed"):
        ctx = hx.from_workload(w, precision=form, stream=stream.cuda_stream)
        ctx.step(warmup, dts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(steps, dts)
        e1.record(stream)
        e1.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        out["batched_" + form] = {"mpts": w.npts * 3 * steps / secs / 1e6, "launches_per_step": ctx.launches_per_step}
        ctx.close()
        singles = []
        for b, blk in enumerate(w.blocks):
            one = W.Workload(w.name + "_%d" % b, [W.Block(blk.xyz, [W.Face(f.kind, 0, f.nbr_face, f.translate)
                                                                     for f in blk.faces], blk.q0)],
                             gamma=w.gamma, mach=w.mach, reynolds=w.reynolds, prandtl=w.prandtl,
                             viscous=w.viscous, mu_law=w.mu_law)
            c = hx.from_workload(one, precision=form, stream=stream.cuda_stream)
            c.step(warmup, dts[b])
            singles.append(c)
        torch.cuda.synchronize()
        e0.record(stream)
        for b, c in enumerate(singles):
            c.step(steps, dts[b])
        e1.record(stream)
        e1.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        out["per_instance_" + form] = {"mpts": w.npts * 3 * steps / secs / 1e6,
                                       "launches_per_step": sum(c.launches_per_step for c in singles)}
        for c in singles:
            c.close()
    out["batched_mixed_vs_per_instance_fp64"] = out["batched_mixed"]["mpts"] / out["per_instance_fp64"]["mpts"]
    return out


def scheme_report(torch, hx, w, steps, warmup, stream):
    """The paper's modified AFWENO (characteristic space at the node,
    indicators shared) against its original AFWENO (characteristic space at
    the face, two WENOs per face): throughput of both on the workload in
    both forms, and accuracy on the 32^3 warped isentropic vortex after 10
    steps against the exact translated vortex."""
    from paper_2006_07964_gb300 import workloads as W
    out = {"report": "scheme", "workload": w.name, "points": w.npts, "steps": steps}
    probe = hx.from_workload(w, precision="fp64", stream=stream.cuda_stream)
    dt, _ = probe.compute_dt(0.5)
    probe.close()
    for scheme, name in ((0, "modified"), (1, "original")):
        for form in ("fp64", "mixed"):
            ctx = hx.from_workload(w, precision=form, stream=stream.cuda_stream, scheme=scheme)
            ctx.step(warmup, dt)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.step(steps, dt)
            e1.record(stream)
            e1.synchronize()
            secs = e0.elapsed_time(e1) / 1e3
            out["%s_%s_mpts" % (name, form)] = w.npts * 3 * steps / secs / 1e6
            ctx.close()
        v = W.vortex(32)
        ctx = hx.from_workload(v, precision="fp64", stream=stream.cuda_stream, scheme=scheme)
        vdt, _ = ctx.compute_dt(0.5)
        ctx.step(10, vdt)
        xyz = v.blocks[0].xyz
        ex = W.conservative(v.gamma, *W.isentropic_vortex(v.gamma, xyz[0], xyz[1], t=10 * vdt))
        q = ctx.get_state(0)
        out["%s_vortex32_rms_error" % name] = float(np.sqrt(((q - ex) ** 2).mean()))
        out["%s_vortex32_max_error" % name] = float(np.abs(q - ex).max())
        ctx.close()
    for form in ("fp64", "mixed"):
        out["speedup_modified_vs_original_" + form] = out["modified_%s_mpts" % form] / out["original_%s_mpts" % form]
    return out


ORACLE_REPORT_WORKLOADS = ["vortex32", "tgv128", "shock512", "shockvortex512", "ogrid", "batch64"]


def oracle_report(W, steps=2):
    """The FP64 oracle as it stands, per workload: whole RK3 steps on all of
    this host's cores and on one thread (CPU only; no GPU is used)."""
    import oracle
    threads = os.cpu_count() or 1
    out = {"report": "oracle", "steps": steps, "host_threads": threads, "workloads": {}}
    for name in ORACLE_REPORT_WORKLOADS:
        desc, make = WORKLOADS[name]
        w = make(W)
        oracle.set_threads(threads)
        P = oracle.from_workload(w)
        dt, _ = P.dt(0.5)
        row = {"nodes": w.npts}
        for label, nt in (("all_cores", threads), ("one_thread", 1)):
            oracle.set_threads(nt)
            t0 = time.perf_counter()
            P.step(steps, dt)
            el = time.perf_counter() - t0
            row[label] = {"mpts": w.npts * 3 * steps / el / 1e6, "threads": oracle.max_threads(), "seconds": el}
        out["workloads"][name] = row
    oracle.set_threads(threads)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv384", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed 128-thread tiles instead of timing the candidates (reproducible profiles)")
    ap.add_argument("--forms", default="fp64,mixed", help="comma list of fp64, mixed")
    ap.add_argument("--report", choices=["precision", "batch", "scheme", "oracle"], default=None,
                    help="print a precision (mixed vs FP64 errors), batch (batched vs per-instance), scheme "
                         "(modified vs original AFWENO) or oracle (CPU oracle per workload, all cores and one "
                         "thread) report instead of the benchmark line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    forms = [f for f in args.forms.split(",") if f]
    if args.no_mixed and "mixed" in forms:
        forms.remove("mixed")
    if not forms or any(f not in ("fp64", "mixed") for f in forms):
        ap.error("--forms takes fp64 and/or mixed")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2006_07964_gb300 import workloads as W
    desc, make = WORKLOADS[args.workload]

    if args.report == "oracle":
        if rank == 0:
            print(json.dumps(oracle_report(W, max(2, args.steps))))
        return

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        full = make(W)
        # each timed step: one whole RK3 step of the workload, or of its
        # bounded sample (the same flow on a coarser grid) when the workload
        # is too large for the host to step within minutes
        sname = ORACLE_SAMPLE.get(args.workload)
        w = WORKLOADS[sname][1](W) if sname else full
        threads = os.cpu_count() or 1
        oracle.set_threads(threads)
        P = oracle.from_workload(w)
        dt, _ = P.dt(0.5)
        P.step(min(args.warmup, 1), dt)
        t0 = time.perf_counter()
        P.step(args.steps, dt)
        el = time.perf_counter() - t0
        v = w.npts * 3 * args.steps / el / 1e6
        sample = "%d full RK3 steps of %s" % (args.steps, "the whole workload" if not sname else
                                              "%s (%d nodes), the same flow on a coarser grid: a bounded sample "
                                              "of the %d-node workload" % (sname, w.npts, full.npts))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpts/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": args.workload + ": " + desc, "points": full.npts},
                "cpu_baseline": {"value": v, "unit": "Mpts/s", "cores": oracle.max_threads(), "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": v, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_2006_07964_gb300 import build, hx
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    w = make(W)
    stream = torch.cuda.Stream()
    peaks = load_peaks()
    if args.report == "precision":
        print(json.dumps(precision_report(torch, hx, w, args.steps, args.warmup, stream)))
        return
    if args.report == "batch":
        print(json.dumps(batch_report(torch, hx, w, args.steps, args.warmup, stream)))
        return
    if args.report == "scheme":
        print(json.dumps(scheme_report(torch, hx, w, args.steps, args.warmup, stream)))
        return

    ranks = Ranks(world)
    barrier = ranks.barrier
    max_over_ranks = ranks.max

    # time step from the FP64 state (held fixed, as the oracle does)
    probe = hx.from_workload(w, precision="fp64", stream=stream.cuda_stream)
    dt, _ = probe.compute_dt(0.5)
    probe.close()

    # headline form first (fp64 unless only mixed is asked for), clocks sampled
    # during its timed region
    head = forms[0]
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    tune = 0 if args.no_autotune else 1
    secs, ctx = run_form(torch, hx, w, head, args.steps, args.warmup, stream, dt, tune)
    ck = clocks.stop()
    barrier()
    secs = max_over_ranks(secs)
    launches = ctx.launches_per_step * args.steps
    value = ranks.throughput(w.npts, args.steps, secs)
    peaks.update(alu_peaks(hx))
    roof = roofline_for(ctx, w, head, 2, dt, peaks, secs / args.steps * 1e3)
    ctx.close()

    mixed = None
    if head == "fp64" and "mixed" in forms:
        msecs, mctx = run_form(torch, hx, w, "mixed", args.steps, args.warmup, stream, dt, tune)
        msecs = max_over_ranks(msecs)
        mval = ranks.throughput(w.npts, args.steps, msecs)
        mixed = {"value": mval, "ms_per_step": msecs / args.steps * 1e3, "ratio_vs_fp64": mval / value,
                 "dtype": "f32 state/fluxes/WENO, f64 metrics/RK", "gpu_launches": mctx.launches_per_step * args.steps,
                 "roofline": roofline_for(mctx, w, "mixed", 2, dt, peaks, msecs / args.steps * 1e3)}
        mctx.close()

    # end to end through the C ABI with page-locked host buffers: per step
    # the state goes host -> device, one RK3 step runs, the state comes back
    ectx = hx.from_workload(w, precision=head, stream=stream.cuda_stream, autotune=tune)
    hq = [np.array(b.q0, dtype=np.float64, order="C") for b in w.blocks]
    hout = [np.zeros_like(q) for q in hq]
    page_locked(torch, hq + hout)
    h2d = sum(b.q0.nbytes for b in w.blocks)
    e_steps = max(3, min(args.steps, 10))
    for b in range(len(w.blocks)):
        ectx.set_state(b, hq[b])
    ectx.step(1, dt)
    torch.cuda.synchronize()
    eclocks = Clocks(local)
    eclocks.start()
    phases = []   # per step: copy in, RK3 step, copy out (host clock)
    t0 = time.perf_counter()
    for _ in range(e_steps):
        ta = time.perf_counter()
        for b in range(len(w.blocks)):
            ectx.set_state(b, hq[b])
        tb = time.perf_counter()
        ectx.step(1, dt)
        tc = time.perf_counter()
        for b in range(len(w.blocks)):
            ectx.get_state(b, hout[b])
        phases.append((tb - ta, tc - tb, time.perf_counter() - tc))
    e_secs = time.perf_counter() - t0
    eck = eclocks.stop()
    e_secs = max_over_ranks(e_secs)
    ectx.close()
    page_unlocked(torch, hq + hout)
    e2e = {"value": ranks.throughput(w.npts, e_steps, e_secs), "unit": "Mpts/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": h2d, "steps": e_steps, "clocks": eck,
           "median_ms": {k: statistics.median(ph[i] for ph in phases) * 1e3
                         for i, k in enumerate(("copy_in", "step", "copy_out"))},
           "max_ms": {k: max(ph[i] for ph in phases) * 1e3 for i, k in enumerate(("copy_in", "step", "copy_out"))}}

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        sname = ORACLE_SAMPLE.get(args.workload)
        cpu = cpu_baseline(w, 2, WORKLOADS[sname][1](W) if sname else None)
    line = {
        "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else "f32 state/fluxes/WENO, f64 metrics/RK", "data": "synthetic",
        "config": {"workload": args.workload + ": " + desc, "points": w.npts, "blocks": len(w.blocks),
                   "dt": dt, "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (resident state and metrics %.0f MB per replica)"
                         % (w.npts * (10 + 15) * 8 / 1e6),
                   "alu_peaks_tflops": {"fp64": peaks["fp64_tflops"], "fp32": peaks["fp32_tflops"]}},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": ck,
        "mixed": mixed,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
