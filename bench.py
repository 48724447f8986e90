#!/usr/bin/env python3
"""Benchmark of the TT-rBKI hot path on GB300.

One step = one whole TT-rBKI decomposition (every mode: Omega draw, sketch,
Krylov powers, orthonormalisation, Rayleigh-Ritz, projection) of the
40^5 precision-form workload: a tensor of TT ranks 20 with 0.8^j slice
scales plus 5% Gaussian noise, stored once in BF16 (204.8 MB, larger than
the 129 MB L2), target ranks 20, p = 10, q = 4.  The same tensor is also
decomposed in the plain FP32 form for the BF16-vs-FP32 comparison at
matched TT error.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank decomposes its own copy (independent
replicas, weak scaling); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
# more hardware work queues for the batched form's concurrent worker streams
# (a per-process setting read when the CUDA context is created)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
sys.path.insert(0, ROOT)

from paper_2308_01480_gb300 import workloads as W  # noqa: E402

METRIC = "rBKI-TT time and HBM-roofline fraction, BF16 vs FP32 at matched TT error"
CONFIG_ID = 3
# kernel families that are library calls (cuBLAS and the like), not this
# library's kernels: none on the decomposition path
LIBRARY_FAMILIES = ()

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum per launch,
# averaged over the launches of one decomposition of this workload) by
# kernel family; an entry is removed when its kernel changes after the
# capture.
NCU_TRAFFIC = {
    "proj_tc": 128750677.0,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form measurement")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the lines for the other single-GPU workloads")
    ap.add_argument("--config", type=int, default=CONFIG_ID, choices=sorted(W.CONFIGS),
                    help="workload (default: the 40^5 BF16 workload the metric is quoted on)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def rel_error_dev(A64, cores):
    """||A - A_hat||_F / ||A||_F on the device in float64 (A64 is the float64
    tensor on the GPU); A_hat is contracted core by core."""
    import torch
    dims = A64.shape
    M = cores[-1].double().reshape(cores[-1].shape[0], -1)
    for G in reversed(cores[1:-1]):
        ra, I, rb = G.shape
        M = (G.double().reshape(ra * I, rb) @ M).reshape(ra, -1)
    F = cores[0].double().reshape(dims[0], -1)
    Am = A64.reshape(dims[0], -1)
    num = 0.0
    for s in range(0, dims[0], 8):
        num += float(torch.sum((Am[s:s + 8] - F[s:s + 8] @ M) ** 2))
    return float(np.sqrt(num) / float(torch.linalg.norm(Am)))


def workload_config(w, world):
    nbytes = w.numel * 2
    return {
        "workload": f"{w.name}: {w.notes}; BF16 storage and remainders, "
                    f"ranks {w.ranks[0]}, p={w.oversample}, q={w.q}",
        "dims": list(w.dims), "ranks": list(w.ranks), "oversample": w.oversample, "q": w.q,
        "omega": "Philox4x32-10 + Box-Muller, seed %d" % w.omega_seed,
        "l2": (f"input ({nbytes / 1e6:.1f} MB BF16) larger than L2 (129 MB); no flush" if nbytes > 129e6
               else f"input ({nbytes / 1e6:.1f} MB BF16) fits L2; no flush"),
        "parallelism": f"replicas{world}" if world > 1 else "single GPU",
    }


def plan_summary(tt, w, opts):
    """The route the planner takes at each mode of the timed decomposition
    (host-only query), e.g. "800x64000 gram_power tc"."""
    return [f"{e['m']}x{e['n']} {e['route']}" + (" tc" if e["tensor_cores"] else "")
            for e in tt.plan_modes(w.dims, w.ranks, w.oversample, w.q, opts)]


def algorithmic_bytes(tt, w, opts, elem):
    """Bytes the method must move for one decomposition: per mode, (q_eff + 2)
    reads of the unfolding C (sketch, q_eff Krylov steps, projection), one
    read of Omega and one write of the remainder, q_eff = min(q, ceil(D / b) - 1)
    (the Krylov dimension cap), elem bytes per entry."""
    total = 0
    for e in tt.plan_modes(w.dims, w.ranks, w.oversample, w.q, opts):
        m, n, b, r = e["m"], e["n"], e["b"], e["r_out"]
        d = min(m, n)
        q_eff = min(w.q, -(-d // b) - 1)
        total += ((q_eff + 2) * m * n + n * b + r * n) * elem
    return total


def config_line(tt, torch, dev, cfg_id, forms, steps, sync_all, peaks):
    """Time one decomposition of workload cfg_id in each storage form
    ("bf16" and/or "fp32", graph-launched), with its TT error against the
    float64 tensor and its whole-step HBM roofline fraction."""
    w = W.CONFIGS[cfg_id]
    A = W.make_tensor(w)
    A32 = torch.from_numpy(A.astype(np.float32)).to(dev)
    A64 = torch.from_numpy(A).to(dev)
    out = {"workload": f"{w.name}: {w.notes}", "dims": list(w.dims), "ranks": list(w.ranks),
           "oversample": w.oversample, "q": w.q}
    for form in forms:
        code = tt.TT_BF16 if form == "bf16" else tt.TT_F32
        x = tt.permute_convert(A32, dst_dtype=torch.bfloat16) if form == "bf16" else A32
        opts = tt.options(storage=code, remainder=code)
        prob = tt.Problem(x, w.ranks, w.oversample, w.q, w.omega_seed)
        g = tt.BatchGraph([prob], opts)
        ms = time_steps(g.launch, steps, 3, sync_all)
        if g.device_status() != [0]:
            raise RuntimeError(f"device status not OK on config {cfg_id} ({form})")
        g.close()
        nbytes = algorithmic_bytes(tt, w, opts, 2 if form == "bf16" else 4)
        per = ms / steps
        out[form] = {"ms_per_step": per, "decompositions_per_s": 1e3 / per,
                     "tt_error": rel_error_dev(A64, prob.cores),
                     "algorithmic_bytes": nbytes,
                     "step_roofline": {"achieved": nbytes / (per * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                                       "unit": "GB/s", "frac": nbytes / (per * 1e-3) / 1e9 / peaks["hbm_gbs"]},
                     "plan": plan_summary(tt, w, opts)}
        del x
    if "bf16" in out and "fp32" in out:
        out["speedup_bf16_over_fp32"] = out["fp32"]["ms_per_step"] / out["bf16"]["ms_per_step"]
        out["bf16_meets_error_criterion"] = out["bf16"]["tt_error"] <= 1.05 * out["fp32"]["tt_error"] + 1e-4
    del A64, A32
    return out


def max_over_ranks(x, dist, device=None):
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(fn, steps, warmup, sync_all):
    """Runs fn() warmup times, then times `steps` calls with CUDA events on
    the current stream; returns milliseconds for the timed steps."""
    import torch
    for _ in range(warmup):
        fn()
    sync_all()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        fn()
    e1.record(st)
    e1.synchronize()
    sync_all()
    return e0.elapsed_time(e1)


def run_ours(args):
    import torch
    import paper_2308_01480_gb300 as tt

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl", device_id=dev)

    def barrier_sync():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = W.CONFIGS[args.config]
    t0 = time.time()
    A = W.make_tensor(w)                     # float64 host tensor, seeded
    gen_s = time.time() - t0
    A32 = torch.from_numpy(A.astype(np.float32)).to(dev)
    # canonical BF16 copy made by the library's own convert kernel
    Abf = tt.permute_convert(A32, dst_dtype=torch.bfloat16)
    torch.cuda.synchronize()

    ranks, p, q, seed = w.ranks, w.oversample, w.q, w.omega_seed
    opts_bf = tt.options(storage=tt.TT_BF16, remainder=tt.TT_BF16)
    opts_32 = tt.options(storage=tt.TT_F32, remainder=tt.TT_F32)
    rr, _ = tt.core_sizes(w.dims, ranks)
    cores_bf = [torch.empty((rr[k], w.dims[k], rr[k + 1]), dtype=torch.float32, device=dev)
                for k in range(len(w.dims))]
    cores_32 = [torch.empty_like(c) for c in cores_bf]
    ws_bf = torch.empty(tt.workspace_size(w.dims, ranks, p, q, opts_bf), dtype=torch.uint8, device=dev)
    ws_32 = torch.empty(tt.workspace_size(w.dims, ranks, p, q, opts_32), dtype=torch.uint8, device=dev)

    def step_bf():
        tt.decompose(Abf, ranks, p, q, omega_seed=seed, opts=opts_bf, workspace=ws_bf, cores=cores_bf)

    # The timed steps replay each form as one CUDA graph through the
    # library's graph API (the same kernels as an eager call, bit-identical
    # cores; checked below).
    prob_bf = tt.Problem(Abf, ranks, p, q, seed, cores=cores_bf)
    graph_bf = tt.BatchGraph([prob_bf], opts_bf)
    prob_32 = tt.Problem(A32, ranks, p, q, seed, cores=cores_32)
    graph_32 = tt.BatchGraph([prob_32], opts_32)

    # ---- timed region: BF16 precision form (the headline)
    for _ in range(args.warmup):
        graph_bf.launch()
    barrier_sync()
    clocks = ClockSampler(local)
    clocks.start()
    ms = time_steps(graph_bf.launch, args.steps, 0, barrier_sync)
    clk = clocks.stop()
    if graph_bf.device_status() != [0]:
        raise RuntimeError("device status not OK after the BF16 runs")
    ms_max = max_over_ranks(ms, dist, dev)
    graph_cores = [c.clone() for c in cores_bf]

    # ---- second timed pass of the same K steps, launched eagerly with a
    # CUDA event pair around every kernel: per-kernel durations for the
    # roofline (kept out of the headline, whose events would add to it)
    step_bf()
    barrier_sync()
    tt.profile_begin(event_timing=True)
    ms_prof = time_steps(step_bf, args.steps, 0, barrier_sync)
    stats = tt.profile_end()
    if tt.device_status(ws_bf) != 0:
        raise RuntimeError("device status not OK after the profiled BF16 runs")
    if not all(torch.equal(a, b) for a, b in zip(graph_cores, cores_bf)):
        raise RuntimeError("graph replay and eager launch disagree")

    # ---- FP32 form on the same tensor (comparison point)
    fp32_steps = max(1, min(args.steps, 10))
    ms32 = time_steps(graph_32.launch, fp32_steps, 2, barrier_sync)

    # ---- the paper's comparison methods on the same BF16 tensor (Alg. 4
    # TT-rSI with the same q, and TT-rSVD = q = 0), graph-launched like the
    # headline
    methods = {}
    cores_m = {}
    # the paper's Alg. 3 taken literally (right-side Krylov matrix, first-r
    # truncation): the study form beside the Rayleigh-Ritz reading
    for name, method, qm, lit in (("tt_rsi", tt.TT_METHOD_RSI, q, False), ("tt_rsvd", tt.TT_METHOD_RBKI, 0, False),
                                  ("tt_rbki_literal", tt.TT_METHOD_RBKI, q, True)):
        pm = tt.Problem(Abf, ranks, p, qm, seed)
        gm = tt.BatchGraph([pm], tt.options(storage=tt.TT_BF16, remainder=tt.TT_BF16, method=method,
                                            paper_literal=lit))
        msm = time_steps(gm.launch, fp32_steps, 2, barrier_sync)
        if gm.device_status() != [0]:
            raise RuntimeError(f"device status not OK after {name}")
        gm.close()
        methods[name] = {"ms_per_step": msm / fp32_steps, "q": qm}
        cores_m[name] = pm.cores

    # ---- TT-SVD (Alg. 1), the deterministic baseline, at the same ranks
    # (eps = 0 with the target ranks as caps); host-synchronous per mode
    svd_ws = {}

    def step_svd():
        c, _ = tt.tt_svd(Abf, eps=0.0, max_ranks=ranks, workspace=svd_ws.get("ws"))
        cores_m["tt_svd"] = c

    step_svd()
    svd_steps = 3
    mss = time_steps(step_svd, svd_steps, 1, barrier_sync)
    methods["tt_svd"] = {"ms_per_step": mss / svd_steps, "q": None,
                         "note": "FP64 Gram DGEMM + cuSOLVER Dsyevd per mode, ranks capped at the targets"}

    # ---- accuracy against the float64 tensor
    A64 = torch.from_numpy(A).to(dev)
    eps_bf = rel_error_dev(A64, cores_bf)
    eps_32 = rel_error_dev(A64, cores_32)
    for name in methods:
        methods[name]["tt_error"] = rel_error_dev(A64, cores_m[name])
    methods["tt_rbki"] = {"ms_per_step": ms_max / args.steps, "q": q, "tt_error": eps_bf}
    del A64

    # ---- end to end through the public API with host buffers: every step
    # copies its input from pinned host memory into a device input buffer,
    # runs the decomposition graph on it and reads the cores back to pinned
    # host memory.  Two slots, each with its own input buffer, graph and
    # cores, let the input copy of step i + 1 (copy stream) and the read-back
    # of step i - 1 (read-back stream) overlap the decomposition of step i,
    # as a serving loop would.  The cores of a slot are views of one flat
    # buffer, so the read-back is one copy.  Every copy lies inside the timed
    # region: the first waits for its start, the last read-back ends it.
    host_bf = torch.empty(Abf.shape, dtype=torch.bfloat16, pin_memory=True)
    host_bf.copy_(Abf.cpu())
    A_in = [Abf, torch.empty_like(Abf)]
    offs, flat_n = [], 0
    for c in cores_bf:
        offs.append(flat_n)
        flat_n += -(-c.numel() // 64) * 64        # 256-byte aligned core offsets
    flat_dev = [torch.empty(flat_n, dtype=torch.float32, device=dev) for _ in range(2)]
    flat_host = [torch.empty(flat_n, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    cores_in = [[flat_dev[s][o:o + c.numel()].view(c.shape) for o, c in zip(offs, cores_bf)] for s in range(2)]
    graphs_in = [tt.BatchGraph([tt.Problem(A_in[s], ranks, p, q, seed, cores=cores_in[s])], opts_bf)
                 for s in range(2)]
    copy_stream = torch.cuda.Stream()
    read_stream = torch.cuda.Stream()

    def run_e2e(steps):
        cur = torch.cuda.current_stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        read = [torch.cuda.Event(), torch.cuda.Event()]
        used = [False, False]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier_sync()
        e0.record(cur)
        copy_stream.wait_event(e0)
        with torch.cuda.stream(copy_stream):
            A_in[0].copy_(host_bf, non_blocking=True)
        copied[0].record(copy_stream)
        for i in range(steps):
            j = i % 2
            if i + 1 < steps:
                nj = 1 - j
                if used[nj]:
                    copy_stream.wait_event(done[nj])     # its previous decomposition has read it
                with torch.cuda.stream(copy_stream):
                    A_in[nj].copy_(host_bf, non_blocking=True)
                copied[nj].record(copy_stream)
            cur.wait_event(copied[j])
            if used[j]:
                cur.wait_event(read[j])                  # this slot's previous cores are on the host
            graphs_in[j].launch()
            done[j].record(cur)
            read_stream.wait_event(done[j])
            with torch.cuda.stream(read_stream):
                flat_host[j].copy_(flat_dev[j], non_blocking=True)
            read[j].record(read_stream)
            used[j] = True
        for j in range(2):
            if used[j]:
                cur.wait_event(read[j])
        e1.record(cur)
        e1.synchronize()
        barrier_sync()
        return e0.elapsed_time(e1)

    e2e_steps = args.steps                       # the first input copy (~1 ms) fills the pipeline once
    run_e2e(3)                                   # warm-up
    ms_e2e = max_over_ranks(run_e2e(e2e_steps), dist, dev)     # whole job: all ranks' steps
    if any(g.device_status() != [0] for g in graphs_in):
        raise RuntimeError("device status not OK after the end-to-end steps")
    # the cores read back equal the headline graph's (same input, same kernels)
    for s in range(2):
        for o, c in zip(offs, graph_cores):
            if not torch.equal(flat_host[s][o:o + c.numel()].view(c.shape), c.cpu()):
                raise RuntimeError("end-to-end cores differ from the headline decomposition")
    h2d = host_bf.numel() * host_bf.element_size()
    d2h = flat_host[0].numel() * flat_host[0].element_size()
    for g in graphs_in:
        g.close()
    graph_bf.close()
    graph_32.close()

    # ---- roofline of the dominant streaming kernel (HBM-bound family)
    peaks, peak_src = measured_peaks()
    hbm_fams = {"proj_tc", "cs_tc", "gram_tc", "gram_apply_tc"}
    pass_stats = {k: v for k, v in stats.items() if k in hbm_fams and v["bytes"] > 0 and v["ms"] > 0}
    dom_name, dom = max(pass_stats.items(), key=lambda kv: kv[1]["ms"])
    launches_dom = max(1, dom["launches"])
    per_launch_ms = dom["ms"] / launches_dom
    per_launch_bytes = dom["bytes"] / launches_dom
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    traffic = NCU_TRAFFIC.get(dom_name)
    library = {k: v["launches"] for k, v in stats.items() if k in LIBRARY_FAMILIES}
    total_launches = sum(v["launches"] for k, v in stats.items() if k not in LIBRARY_FAMILIES)
    # where the time goes: the family with the largest share of the timed
    # kernel time, and the whole step against the HBM roofline
    kern_ms = sum(v["ms"] for v in stats.values())
    top_name, top = max(stats.items(), key=lambda kv: kv[1]["ms"])
    step_bytes = algorithmic_bytes(tt, w, opts_bf, 2)
    step_ms = ms_max / args.steps
    dominant = {"kernel": top_name, "share": top["ms"] / kern_ms if kern_ms else None,
                "ms_per_step": top["ms"] / args.steps,
                "bound": "hbm" if top_name in hbm_fams else
                         ("tensor" if top_name == "gram_tc_tiled" else "latency (small dense algebra on one SM or cluster)")}
    step_roof = {"achieved": step_bytes / (step_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": step_bytes / (step_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "algorithmic_bytes": step_bytes,
                 "ideal_ms": step_bytes / (peaks["hbm_gbs"] * 1e9) * 1e3}
    gram_roof = None
    if "gram_tc_tiled" in stats and stats["gram_tc_tiled"]["ms"] > 0:
        gstat = stats["gram_tc_tiled"]
        tflops = gstat["flops"] / (gstat["ms"] * 1e-3) / 1e12
        gram_roof = {"bound": "tensor", "kernel": "gram_tc_tiled", "achieved": tflops,
                     "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "frac": tflops / peaks["bf16_tflops"],
                     "flops_note": "algorithmic 2 m^2 n per Gram (both triangles), averaged over the launches "
                                   "(the 800 x 64000 and 800 x 1600 unfoldings)",
                     "launches": gstat["launches"], "ms_per_launch": gstat["ms"] / gstat["launches"]}

    result = {
        "metric": METRIC,
        "value": world * args.steps / (ms_max * 1e-3),
        "unit": "decompositions/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16",
        "data": "synthetic (seeded; paper's datasets unavailable)",
        "config": workload_config(w, world),
        "plan": plan_summary(tt, w, opts_bf),
        "tt_error": {"bf16": eps_bf, "fp32": eps_32},
        "methods_bf16": methods,
        "fp32_form": {"ms_per_step": ms32 / fp32_steps, "decompositions_per_s": fp32_steps / (ms32 * 1e-3),
                      "tt_error": eps_32, "speedup_bf16_over_fp32": (ms32 / fp32_steps) / (ms_max / args.steps)},
        "e2e": {"value": world * e2e_steps / (ms_e2e * 1e-3), "unit": "decompositions/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "overlap": "input copy of step i+1 (pinned host -> device, copy stream) and read-back of "
                           "step i-1's cores (one device -> pinned host copy, read-back stream) overlap the "
                           "decomposition of step i; two slots, every copy inside the timed region"},
        "gpu_launches": total_launches,
        "library_gemm_launches": library,
        "launch": "one CUDA graph per decomposition (library graph API); kernel timings from a second "
                  "timed pass of the same steps launched eagerly with per-kernel CUDA events",
        "profiled_ms_per_step": ms_prof / args.steps,
        "step_roofline": step_roof,
        "dominant_kernel": dominant,
        "gram_roofline": gram_roof,
        "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "peak_source": peak_src, "traffic": traffic,
                     "bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_ms,
                     "launches": dom["launches"]},
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                        "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 and v["bytes"] > 0 else None}
                    for k, v in stats.items()},
        "clocks": clk,
        "input_gen_s": gen_s,
    }

    if not args.no_extra_configs:
        # the other single-GPU workloads: 256 x 256 x 64 x 32 in both forms
        # (the largest), 32^5 in the plain FP32 form
        result["other_configs"] = {
            "config4": config_line(tt, torch, dev, 4, ("bf16", "fp32"), 10, barrier_sync, peaks),
            "config2": config_line(tt, torch, dev, 2, ("fp32",), 10, barrier_sync, peaks),
        }
    if not args.no_batched:
        result["batched"] = batched_measure(tt, torch, dev, barrier_sync)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(A, w)
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


def batched_measure(tt, torch, dev, sync_all, launches=5):
    """The batched form: 256 independent problems (orders 3-6, modes 8-64,
    ranks 2-16, 5% noise, BF16, p = 5, q = 2) decomposed by one CUDA graph
    launch; reports problems/s and the input bytes streamed per second."""
    ws_list = W.batch_workloads()
    probs = []
    for wl in ws_list:
        t = torch.from_numpy(W.make_tensor(wl).astype(np.float32)).to(dev)
        probs.append(tt.Problem(tt.permute_convert(t, dst_dtype=torch.bfloat16), wl.ranks, wl.oversample, wl.q,
                                wl.omega_seed))
        del t
    g = tt.BatchGraph(probs, tt.options(storage=tt.TT_BF16, remainder=tt.TT_BF16, batch_streams=32))
    ms = time_steps(g.launch, launches, 2, sync_all)
    ok = g.device_status() == [0] * len(probs)
    g.close()
    nbytes = sum(wl.numel for wl in ws_list) * 2
    return {"workload": f"{len(probs)} problems, orders 3-6, modes 8-64, TT ranks 2-16, 5% noise, BF16, p=5, q=2",
            "input_bytes": nbytes, "ms_per_batch": ms / launches,
            "problems_per_s": len(probs) * launches / (ms * 1e-3),
            "input_GBps": nbytes * launches / (ms * 1e-3) / 1e9, "statuses_ok": ok,
            "launch": "one CUDA graph per batch, 32 worker streams, CUDA_DEVICE_MAX_CONNECTIONS=" +
                      os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "default")}


def oracle_step(A, w):
    """One TT-rBKI decomposition by the FP64 oracle on the host cores."""
    import oracle
    oracle.tt_rbki(A, w.ranks, w.oversample, w.q, seed=w.omega_seed)


def cpu_baseline(A, w, reps=2):
    t0 = time.time()
    for _ in range(reps):
        oracle_step(A, w)
    dt = time.time() - t0
    return {"value": reps / dt, "unit": "decompositions/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{reps} full decompositions of the same workload (same tensor, ranks, p, q, seed) "
                      "by the float64 numpy oracle (BLAS/LAPACK threads = all host cores)", "seconds": dt}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    w = W.CONFIGS[args.config]
    A = W.make_tensor(w)
    for _ in range(args.warmup):
        oracle_step(A, w)
    t0 = time.time()
    for _ in range(args.steps):
        oracle_step(A, w)
    dt = time.time() - t0
    v = args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "decompositions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; paper's datasets unavailable)", "config": workload_config(w, world),
        "cpu_baseline": {"value": v, "unit": "decompositions/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "one full decomposition per step by the float64 numpy oracle"},
        "e2e": {"value": v, "unit": "decompositions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
