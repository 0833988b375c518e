"""Throughput of the sketched column-ID hot path on GB300.

One step = one pass of the whole hot path over one window: Gaussian sketch
(Omega regenerated on the fly), batched pivoted QR + rank decision +
coefficients, and the fused reconstruction / relative Frobenius error, plus
the compression factor.  Default workload: the 3D TGV + Fourier field on a
64^3 grid split into 64 boxes of 16^3 x 5 QoIs (m = 20480), n = 512
snapshots, k = 20, p = 10, FP32 data, TF32 tensor-core sketch.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(the only reference this method has) on a bounded sample of the same
workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "snapshot GB/s compressed at rel. err <=1e-3: mixed-prec batched vs plain FP32"
WORKLOAD = ("TGV+Fourier 64^3 grid, 64 subdomains of 16^3 x 5 QoIs (m=20480), n=512 snapshots, "
            "k=20, p=10, FP32 window")


# DRAM bytes (read + write) of one launch of each hot kernel on the default
# workload, from `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum`
# (profiles/dram_traffic_tf32_tgv3d_64sub.md).  A figure is reported only while
# the kernel's sources hash to the value they had when it was measured.
MEASURED_TRAFFIC = {
    "sketch": {"bytes": 2693764352 + 7260672,
               "sources": ('sketch_tc.cu', 'sketch_pack.cuh', 'tcgen05_ptx.cuh', 'spid_internal.cuh'),
               "sha256_16": "cbd243bb97a2ae45"},
    "error": {"bytes": 2684926720 + 221696, "sources": ('error.cu', 'error_fold.cuh', 'spid_internal.cuh'),
              "sha256_16": "22989af0ca8d0f0d"},
}
# the tile shapes the counters were taken with (the library defaults)
MEASURED_TUNING = {"sketch_pack_slices": 8, "sketch_stages": 0, "error_path": 0,
                   "error_rows": 512, "error_cols": 256}


def measured_traffic(kernel: str):
    import hashlib
    rec = MEASURED_TRAFFIC.get(kernel)
    if rec is None:
        return None
    m = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, "paper_2103_01380_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    return rec["bytes"] if m.hexdigest()[:16] == rec["sha256_16"] else None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            os.unlink(self.path)
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() in ("active", "1"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons),
                       samples=len(sm))
        return out


def bind_to_gpu_numa_node(device: int):
    """Pin this process to the CPUs local to the GPU, so that pinned host
    buffers are first-touched on the memory node attached to the GPU (on a
    Grace-based GB300 the other socket's memory is reached through the CPU-CPU
    link and halves host->device bandwidth).  Returns what was done."""
    import torch
    try:
        p = torch.cuda.get_device_properties(device)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        base = f"/sys/bus/pci/devices/{bus}"
        node = int(open(f"{base}/numa_node").read().strip())
        cpus = set()
        for part in open(f"{base}/local_cpulist").read().strip().split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if cpus:
            os.sched_setaffinity(0, cpus)
        return {"pci": bus, "numa_node": node, "cpus": len(cpus)}
    except Exception as exc:  # sysfs layout differs: leave affinity alone
        return {"error": type(exc).__name__}


def make_window(rank: int = 0, boxes=None):
    from paper_2103_01380_gb300 import inputs
    return inputs.tgv3d_window(grid=64, box=16, n=512, seed=2 + rank, boxes=boxes)


def cpu_baseline(win, sample_subs: int, precision: str = "tf32"):
    """The FP64 oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    idx = np.linspace(0, win.num_sub - 1, sample_subs).round().astype(int)
    blocks = [win.block(int(s)) for s in idx]
    from paper_2103_01380_gb300 import inputs
    sub = inputs.pack_blocks(blocks, dtype=np.float64)
    u = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "tf32": 2.0 ** -11}[precision]
    t0 = time.perf_counter()
    oracle.spid_batch(sub.data, sub.m, sub.n, sub.off, sub.ld, 30, 20, 0.0, u, 0x5EED0001)
    dt = time.perf_counter() - t0
    nbytes = 4.0 * float((sub.m * sub.n).sum())
    return {"value": nbytes / dt / 1e9, "unit": "GB/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{sample_subs} of {win.num_sub} subdomains (m=20480, n=512), FP64 oracle "
                      f"sketch+QR+coefficients+error, {dt:.2f} s wall"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    win = make_window(0, boxes=max(args.ref_subs, 1))
    ts = []
    nb = None
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(win, args.ref_subs)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            ts.append(dt)
            nb = cb
    value = float(np.median([nb["value"]]))
    sample_bytes = 4.0 * 20480 * 512 * args.ref_subs
    ms = 1e3 * float(np.mean(ts))
    line = {"impl": "reference", "metric": METRIC, "value": sample_bytes / (ms / 1e3) / 1e9,
            "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_subdomains": args.ref_subs},
            "cpu_baseline": {"kind": "oracle", "cores": nb["cores"], "sample": nb["sample"],
                             "value": sample_bytes / (ms / 1e3) / 1e9, "unit": "GB/s"},
            "e2e": {"value": sample_bytes / (ms / 1e3) / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
# Other workloads of the paper-derived configuration list (one GPU each)
# ----------------------------------------------------------------------------
def _stage_times(torch, plan, window, steps, warmup, err, tot, sketch_calls):
    """Mean sketch / finalize / error times (ms) over `steps` CUDA-event-timed
    steps on the current stream; sketch_calls = list of (col0, ncols)."""
    stream = torch.cuda.current_stream()

    def step():
        for c0, nc in sketch_calls:
            plan.sketch(window, c0, nc)
        plan.finalize()
        plan.error(window, err, tot)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(stream)
        for c0, nc in sketch_calls:
            plan.sketch(window, c0, nc)
        ev[i][1].record(stream)
        plan.finalize()
        ev[i][2].record(stream)
        plan.error(window, err, tot)
        ev[i][3].record(stream)
    torch.cuda.synchronize()
    sk = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    fi = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    er = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)
    return sk, fi, er


def _graph_ms(torch, plan, window, err, tot, steps, warmup=2):
    """Mean time (ms) of one whole step (sketch, finalize, error) replayed as a
    CUDA graph of the plan, CUDA events on the current stream."""
    g = plan.graph(window, err=err, total=tot)
    for _ in range(warmup):
        g.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        g.launch()
    e1.record()
    torch.cuda.synchronize()
    g.close()
    return e0.elapsed_time(e1) / steps


def _summary(plan, tot):
    t = tot.detach().cpu().numpy()
    k, _, _ = plan.factors()
    return {"rel_err": float(np.sqrt(t[0] / t[1])), "compression_factor": float(t[2] / t[3]),
            "k_mean": float(np.mean(k)), "k_max": int(np.max(k))}


def run_workload(args):
    import torch
    from paper_2103_01380_gb300 import build, inputs, spid
    torch.cuda.set_device(0)
    build.build()
    spid.load_library()
    peak, peak_kind = load_peaks()
    if args.workload == "spectrum256":
        line = _run_spectrum(args, torch, inputs, spid)
    elif args.workload == "uneven4096":
        line = _run_uneven(args, torch, inputs, spid)
    elif args.workload == "coarse_tgv3d64":
        line = _run_coarse(args, torch, inputs, spid)
    elif args.workload == "points_tgv2d":
        line = _run_points(args, torch, inputs, spid)
    elif args.workload == "two_stage_tgv3d64":
        line = _run_two_stage(args, torch, inputs, spid)
    else:
        line = _run_insitu(args, torch, inputs, spid)
    line.update({"metric": METRIC, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
                 "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                 "vs_baseline": None, "data": "synthetic", "gpu_launches": None})
    sk = line.pop("_sketch_gbs", None)
    if sk is not None:
        line["roofline"] = {"bound": "hbm", "kernel": "sketch", "achieved": sk, "peak": peak,
                            "unit": "GB/s", "frac": sk / peak, "peak_kind": peak_kind,
                            "traffic": None}
    print(json.dumps(line))
    return 0


def _coarse_stage_times(torch, plan, window, steps, warmup, err, tot, form):
    """Mean sample / finalize / error times (ms) of the coarse-grid ID."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.sample(window)
        plan.finalize()
        plan.error(window, form, err, tot)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(stream)
        plan.sample(window)
        ev[i][1].record(stream)
        plan.finalize()
        ev[i][2].record(stream)
        plan.error(window, form, err, tot)
        ev[i][3].record(stream)
    torch.cuda.synchronize()
    return tuple(statistics.mean(e[a].elapsed_time(e[a + 1]) for e in ev) for a in range(3))


def _run_coarse(args, torch, inputs, spid):
    """Coarse-grid column ID (Section 2 SubID / SPID, Algorithms 2-3; Section
    5.2): the bench window (64 boxes of 16^3 x 5 QoIs, n = 512) at coarse
    intervals 3 and 5, adaptive tol 1e-3 on B, and the paper's E3 case (64^3
    TGV u1, 100 snapshots, interval 3)."""
    win = make_window(0, None)
    w = torch.from_numpy(win.data).cuda()
    nbytes = float(win.nbytes_payload())
    boxes = np.tile(np.array([5, 16, 16, 16], dtype=np.int32), (win.num_sub, 1))
    err = torch.zeros(2 * win.num_sub, dtype=torch.float64, device="cuda")
    tot = torch.zeros(4, dtype=torch.float64, device="cuda")
    study = {}
    for stride in (3, 5):
        plan = spid.SubPlan(boxes, win.n, win.off, win.ld, (stride,) * 3, k_max=20, tol=1e-3)
        res = {"coarse_rows": int(plan.mc[0]), "fine_rows": int(win.m[0])}
        for form, tag in ((spid.FORM_SPID, "spid"), (spid.FORM_SUBID, "subid")):
            sa, fi, er = _coarse_stage_times(torch, plan, w, args.steps, args.warmup, err, tot,
                                             form)
            t = tot.cpu().numpy()
            res[tag] = {"value": nbytes / ((sa + fi + er) / 1e3) / 1e9,
                        "single_pass_gbs": nbytes / ((sa + fi) / 1e3) / 1e9,
                        "stages_ms": {"sample": sa, "finalize": fi, "error": er},
                        "error_gbs": nbytes / (er / 1e3) / 1e9,
                        "rel_err": float(np.sqrt(t[0] / t[1])),
                        "compression_factor": float(t[2] / t[3])}
        k, _, _, _ = plan.factors()
        res["k_mean"], res["k_max"] = float(np.mean(k)), int(np.max(k))
        study[f"interval{stride}"] = res
        plan.close()
    # E3 (Section 5.2): 64^3 TGV u1, n = 100, interval 3, rank decided at tol 1e-3
    t = np.linspace(0.0, 10.0, 100)
    u1 = inputs.tgv3d_u1(64, t)
    e3 = inputs.pack_blocks([u1])
    we = torch.from_numpy(e3.data).cuda()
    plan = spid.SubPlan([[1, 64, 64, 64]], e3.n, e3.off, e3.ld, (3, 3, 3), k_max=4, tol=1e-3)
    err1 = torch.zeros(2, dtype=torch.float64, device="cuda")
    sa, fi, er = _coarse_stage_times(torch, plan, we, args.steps, args.warmup, err1, tot,
                                     spid.FORM_SPID)
    tt = tot.cpu().numpy()
    k, _, _, _ = plan.factors()
    e3b = float(e3.nbytes_payload())
    study["e3_tgv64_u1_interval3"] = {
        "k": int(k[0]), "rel_err": float(np.sqrt(tt[0] / tt[1])),
        "compression_factor": float(tt[2] / tt[3]),
        "paper": "interval 3: ~2% error, compression ~2400",
        "stages_ms": {"sample": sa, "finalize": fi, "error": er},
        "single_pass_gbs": e3b / ((sa + fi) / 1e3) / 1e9}
    plan.close()
    main = study["interval3"]["spid"]
    line = {"value": main["value"], "ms_per_step": nbytes / main["value"] / 1e6,
            "dtype": "f32", "config": {
                "workload": "coarse-grid SPID (trilinear M) of the TGV+Fourier 64^3 window: "
                            "64 boxes of 16^3 x 5 QoIs, n=512, coarse interval 3 "
                            "(m_c = 6^3 x 5 = 1080), adaptive tol 1e-3 on B, k_max=20",
                "l2": "inputs (2.68 GB) larger than L2; no flush"},
            "study": study}
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        for s in (0, win.num_sub - 1):
            oracle.subid(win.block(s).astype(np.float64), (5, 16, 16, 16), (3, 3, 3), 20, 1e-3,
                         2.0 ** -24)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 2 * 4.0 * int(win.m[0]) * int(win.n[0]) / dt / 1e9,
                                "unit": "GB/s", "cores": 1, "kind": "oracle",
                                "sample": "subdomains 0 and 63, interval 3 (FP64 oracle)"}
    return line


def _run_points(args, torch, inputs, spid):
    """Coarse-grid ID on an unstructured point set (Section 2: rows in any order;
    Section 5.1: random points): the 2D TGV (u1, u2) plus 4 smooth modes at 2^20
    uniformly random points of [0, 2 pi)^2 in 16 x 16 spatial blocks (about
    4096 points x 2 QoIs per block, rows in random order), n = 256 snapshots;
    per block a random coarse subset of 1/8 of its points with barycentric
    Delaunay stencils (t = 3); adaptive tol 1e-3 on B, k_max = 16."""
    rng = np.random.default_rng(5)
    npts, n = 1 << 20, 256
    pts = rng.uniform(0.0, 2.0 * np.pi, size=(npts, 2))
    parts = inputs.point_partitions(pts, 16, 16)
    win, m, nn, off, ld = inputs.tgv2d_points_window_device(pts, parts, n, seed=5)
    crows, idxs, ws = [], [], []
    for b, part in enumerate(parts):
        cr, ix, w = inputs.coarse_stencil(pts[part], max(4, len(part) // 8), 3, seed=500 + b,
                                          nq=2)
        crows.append(cr)
        idxs.append(ix)
        ws.append(w)
    S = len(parts)
    nbytes = 4.0 * float((m * nn).sum())
    plan = spid.SubPlan.from_points(m, nn, off, ld, crows, idxs, ws, k_max=16, tol=1e-3)
    err = torch.zeros(2 * S, dtype=torch.float64, device="cuda")
    tot = torch.zeros(4, dtype=torch.float64, device="cuda")
    res = {}
    for form, tag in ((spid.FORM_SPID, "spid"), (spid.FORM_SUBID, "subid")):
        sa, fi, er = _coarse_stage_times(torch, plan, win, args.steps, args.warmup, err, tot, form)
        t = tot.cpu().numpy()
        res[tag] = {"value": nbytes / ((sa + fi + er) / 1e3) / 1e9,
                    "single_pass_gbs": nbytes / ((sa + fi) / 1e3) / 1e9,
                    "stages_ms": {"sample": sa, "finalize": fi, "error": er},
                    "error_gbs": nbytes / (er / 1e3) / 1e9,
                    "rel_err": float(np.sqrt(t[0] / t[1])),
                    "compression_factor": float(t[2] / t[3])}
    k, _, _, _ = plan.factors()
    status = plan.device_status()
    plan.close()
    main = res["spid"]
    return {"value": main["value"], "ms_per_step": sum(main["stages_ms"].values()),
            "dtype": "f32",
            "config": {"workload": "coarse-grid SPID on an unstructured point set: 2D TGV "
                                   "(u1, u2) + 4 smooth modes at 2^20 random points in 16 x 16 "
                                   "blocks (~4096 points x 2 QoIs each, random row order), "
                                   "n=256, coarse subsets of 1/8 of the points, Delaunay "
                                   "barycentric stencils (t=3), adaptive tol 1e-3, k_max=16",
                       "l2": f"inputs ({nbytes / 1e9:.2f} GB) larger than L2; no flush"},
            "forms": res, "k_mean": float(np.mean(k)), "k_max": int(np.max(k)),
            "status": status, "_sketch_gbs": main["single_pass_gbs"]}


def _run_two_stage(args, torch, inputs, spid):
    """Modified two-stage SPID (Section 3.3.2, Algorithm 6) on the bench window:
    64 boxes of 16^3 x 5 QoIs, n = 512 cut into N time blocks with a target-rank
    k sketched ID each (TF32), then the tolerance-1e-3 ID of the skeletons."""
    win = make_window(0, None)
    w = torch.from_numpy(win.data).cuda()
    nbytes = float(win.nbytes_payload())
    S = win.num_sub
    err = torch.zeros(2 * S, dtype=torch.float64, device="cuda")
    tot = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    study = {}
    for N, k in ((4, 20), (8, 10), (16, 6)):
        plan = spid.TsPlan.for_window(win, blocks=N, k=k, k2_max=min(32, N * k), tol2=1e-3,
                                      p=10, precision="tf32", seed=0x5EED0001)

        def step():
            for b in range(N):
                plan.block(w, b)
            plan.finalize(w)
            plan.error(w, err, tot)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        for i in range(args.steps):
            ev[i][0].record(stream)
            for b in range(N):
                plan.block(w, b)
            ev[i][1].record(stream)
            plan.finalize(w)
            ev[i][2].record(stream)
            plan.error(w, err, tot)
            ev[i][3].record(stream)
        torch.cuda.synchronize()
        s1, s2, er = (statistics.mean(e[a].elapsed_time(e[a + 1]) for e in ev) for a in range(3))
        t = tot.cpu().numpy()
        k2, _, _ = plan.factors()
        kb = plan.block_factors(0)[0]
        study[f"N{N}_k{k}"] = {
            "value": nbytes / ((s1 + s2 + er) / 1e3) / 1e9,
            "stages_ms": {"stage1_all_blocks": s1, "stage2_and_compose": s2, "error": er},
            "stage1_gbs": nbytes / (s1 / 1e3) / 1e9,
            "rel_err": float(np.sqrt(t[0] / t[1])), "compression_factor": float(t[2] / t[3]),
            "k2_mean": float(np.mean(k2)), "k_block0_mean": float(np.mean(kb)),
            "status": plan.device_status()}
        plan.close()
    main = study["N4_k20"]
    return {"value": main["value"], "ms_per_step": nbytes / main["value"] / 1e6,
            "dtype": "f32 (tf32 sketch)",
            "config": {"workload": "modified two-stage SPID of the TGV+Fourier 64^3 window: 64 "
                                   "boxes of 16^3 x 5 QoIs, n=512 in N=4 time blocks, stage-1 "
                                   "rank k=20, stage-2 tol 1e-3 (k2 <= 32), p=10",
                       "l2": "inputs (2.68 GB) larger than L2; no flush"},
            "study": study}


def _run_spectrum(args, torch, inputs, spid):
    """256 subdomains, A = U diag(sigma) V^T with sigma_i = 10^{-i/4}, m = 16384,
    n = 256, adaptive rank to 1e-3 (k_max 32, p 10), every sketch precision."""
    S, m, n, r = 256, 16384, 256, 32
    sig = torch.tensor(10.0 ** (-np.arange(1, r + 1) / 4.0), device="cuda", dtype=torch.float32)
    window = torch.empty(S * m * n, device="cuda", dtype=torch.float32)
    g = torch.Generator(device="cuda")
    for s in range(S):
        g.manual_seed(3 + s)
        U, _ = torch.linalg.qr(torch.randn(m, r, device="cuda", generator=g))
        V, _ = torch.linalg.qr(torch.randn(n, r, device="cuda", generator=g))
        window[s * m * n:(s + 1) * m * n].view(n, m).copy_(((U * sig) @ V.T).T)
    nbytes = 4.0 * S * m * n
    err = torch.zeros(2 * S, dtype=torch.float64, device="cuda")
    tot = torch.zeros(4, dtype=torch.float64, device="cuda")
    study = {}
    # "tf32_tensor_core_error": the same TF32 plan with the rank-k product of the
    # error pass on the tensor cores
    for label, prec, flags in (("tf32", "tf32", 0), ("bf16x3", "bf16x3", 0), ("bf16", "bf16", 0),
                               ("fp32", "fp32", 0),
                               ("tf32_tensor_core_error", "tf32", spid.FLAG_TC_ERROR)):
        plan = spid.Plan([m] * S, [n] * S, np.arange(S) * m * n, [m] * S, k_max=32, p=10,
                         tol=1e-3, precision=prec, seed=0x5EED0003, flags=flags)
        sk, fi, er = _stage_times(torch, plan, window, args.steps, args.warmup, err, tot,
                                  [(0, n)])
        study[label] = dict(value=nbytes / ((sk + fi + er) / 1e3) / 1e9,
                           sketch_gbs=nbytes / (sk / 1e3) / 1e9, finalize_ms=fi,
                           error_gbs=nbytes / (er / 1e3) / 1e9, **_summary(plan, tot))
        plan.close()
    line = {"value": study["tf32"]["value"], "ms_per_step": nbytes / study["tf32"]["value"] / 1e6,
            "dtype": "f32 (tf32 sketch)",
            "config": {"workload": "spectrum: 256 subdomains, A = U diag(10^{-i/4}) V^T "
                                   "(Haar U, V; components beyond 32 sit below FP32 rounding), "
                                   "m=16384, n=256, adaptive tol 1e-3, k_max=32, p=10",
                       "l2": "inputs (4.29 GB) larger than L2; no flush"},
            "precision_study": study, "_sketch_gbs": study["tf32"]["sketch_gbs"]}
    if not args.no_cpu_baseline:
        # the oracle on two sampled subdomains: its own error at the same tolerance
        import oracle
        host = window.view(S, n, m)[[0, S - 1]].cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        errs = []
        for blk in host:
            o = oracle.spid(blk.T, 42, 32, 1e-3, 2.0 ** -53, 0x5EED0003)
            errs.append(float(np.sqrt(o["e2"] / o["a2"])))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 2 * 4.0 * m * n / dt / 1e9, "unit": "GB/s",
                                "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": "subdomains 0 and 255 (FP64 oracle, adaptive 1e-3)",
                                "oracle_rel_err": errs}
    return line


def _run_uneven(args, torch, inputs, spid):
    """4096 cubic boxes, edges {8,12,16,24,32} x 5 QoIs, windows 64..1024 snapshots,
    of the TGV+Fourier field on a 256^3 grid; adaptive 1e-3 (k_max 32, p 10);
    processed in waves that fit HBM, one plan per wave."""
    boxes = inputs.uneven_boxes(4096, seed=4)
    modes = inputs.fourier_modes(seed=2)
    waves, cur, cur_b = [], [], 0.0
    for b in boxes:
        nb = 4.0 * 5 * b[1] ** 3 * b[2]
        if cur and cur_b + nb > args.wave_gb * 1e9:
            waves.append(cur)
            cur, cur_b = [], 0.0
        cur.append(b)
        cur_b += nb
    waves.append(cur)
    tot_bytes, tot_ms, sk_ms_all, ks, e2, a2, mn, kd = 0.0, 0.0, 0.0, [], 0.0, 0.0, 0.0, 0.0
    stage_ms = 0.0
    tuning = None
    for wv in waves:
        m = np.array([5 * e ** 3 for _, e, _ in wv], dtype=np.int64)
        n = np.array([nn for _, _, nn in wv], dtype=np.int64)
        off = np.concatenate([[0], np.cumsum(m * n)[:-1]])
        window = torch.empty(int((m * n).sum()), device="cuda", dtype=torch.float32)
        for s, (org, e, nn) in enumerate(wv):
            f = inputs.DeviceField([org], e, 256, modes)
            t = 10.0 * np.arange(nn) / max(nn - 1, 1)
            blk = f.snapshots(t).reshape(5 * e ** 3, nn)                  # [m, n]
            window[int(off[s]):int(off[s] + m[s] * nn)].view(nn, int(m[s])).copy_(blk.T)
        S = len(wv)
        err = torch.zeros(2 * S, dtype=torch.float64, device="cuda")
        tot = torch.zeros(4, dtype=torch.float64, device="cuda")
        plan = spid.Plan(m, n, off, m, k_max=32, p=10, tol=1e-3, precision="tf32",
                         seed=0x5EED0004)
        # the waves share one size distribution: tune on the first, reuse after
        if not args.no_autotune:
            if tuning is None:
                tuning = plan.autotune(window)
            else:
                plan.set_tuning(tuning)
        sk, fi, er = _stage_times(torch, plan, window, max(1, args.steps // 4), 1, err, tot,
                                  [(0, int(n.max()))])
        # the step as the batched form runs it: one graph launch per wave
        step_ms = _graph_ms(torch, plan, window, err, tot, max(1, args.steps // 4))
        t = tot.detach().cpu().numpy()
        e2, a2, mn, kd = e2 + t[0], a2 + t[1], mn + t[2], kd + t[3]
        ks.extend(plan.factors()[0].tolist())
        tot_bytes += 4.0 * float((m * n).sum())
        tot_ms += step_ms
        stage_ms += sk + fi + er
        sk_ms_all += sk
        plan.close()
        del window
        torch.cuda.empty_cache()
    return {"value": tot_bytes / (tot_ms / 1e3) / 1e9, "ms_per_step": tot_ms,
            "dtype": "f32 (tf32 sketch)",
            "config": {"workload": f"uneven: 4096 cubic boxes (edges 8..32) x 5 QoIs of a 256^3 "
                                   f"TGV+Fourier field, n in 64..1024, adaptive 1e-3, "
                                   f"{len(waves)} waves of <= {args.wave_gb:g} GB",
                       "total_gb": tot_bytes / 1e9, "l2": "inputs larger than L2",
                       "launch": "one CUDA graph per wave step", "tuning": tuning},
            "eager_stage_sum_gbs": tot_bytes / (stage_ms / 1e3) / 1e9,
            "rel_err": float(np.sqrt(e2 / a2)), "compression_factor": float(mn / kd),
            "k_mean": float(np.mean(ks)), "k_max": int(np.max(ks)),
            "_sketch_gbs": tot_bytes / (sk_ms_all / 1e3) / 1e9}


def _insitu_solver(torch, spid, plan, window, field, t_all, calls, S, m, n, err, tot,
                   substeps=4, dt=0.003, nu=0.01):
    """Compression next to a running solver on the same GPU: the producer (an
    advection-diffusion stand-in for the paper's flow solver, spid_producer_step)
    advances the TGV+Fourier state `substeps` steps per snapshot and writes each
    snapshot into the window; the sketch consumes each micro-batch of snapshots
    on a second stream as soon as it lands, then finalize + error close the
    window.  Times: solver alone, compression alone, and both overlapped."""
    # subdomain-major window: snapshot j of box b starts at b n m + j m
    scratch = [torch.empty(S * m, device="cuda"), torch.empty(S * m, device="cuda")]

    def produce(j):
        src, src_stride = window[(j - 1) * m:], n * m
        for i in range(substeps):
            last = i == substeps - 1
            dst, dst_stride = (window[j * m:], n * m) if last else (scratch[i % 2], m)
            spid.producer_step(src, dst, 256, 32, 5, dt, nu, in_box_stride=src_stride,
                               out_box_stride=dst_stride)
            src, src_stride = dst, dst_stride

    def initial():
        field.fill_subdomain_major(window, t_all[:1], 0, n)

    ev = lambda: torch.cuda.Event(enable_timing=True)
    cons = torch.cuda.current_stream()
    prod = torch.cuda.Stream()
    initial()
    torch.cuda.synchronize()
    a0, a1 = ev(), ev()
    a0.record(cons)
    for j in range(1, n):
        produce(j)
    a1.record(cons)
    torch.cuda.synchronize()
    solver_ms = a0.elapsed_time(a1)
    # compression alone on the solver's window
    b0, b1, b2 = ev(), ev(), ev()
    b0.record(cons)
    for j0, nc in calls:
        plan.sketch(window, j0, nc)
    b1.record(cons)
    plan.finalize()
    plan.error(window, err, tot)
    b2.record(cons)
    torch.cuda.synchronize()
    sketch_ms, close_ms = b0.elapsed_time(b1), b1.elapsed_time(b2)
    t = tot.cpu().numpy()
    k, _, _ = plan.factors()
    # both: the producer stream writes the window while the sketch consumes it
    initial()
    torch.cuda.synchronize()
    ready = {}
    c0, c1, c2 = ev(), ev(), ev()
    c0.record(cons)
    prod.wait_event(c0)
    with torch.cuda.stream(prod):
        for j0, nc in calls:
            for j in range(max(j0, 1), j0 + nc):
                produce(j)
            ready[j0] = torch.cuda.Event()
            ready[j0].record(prod)
    for j0, nc in calls:
        cons.wait_event(ready[j0])
        plan.sketch(window, j0, nc)
    c1.record(cons)
    plan.finalize()
    plan.error(window, err, tot)
    c2.record(cons)
    torch.cuda.synchronize()
    both_ms = c0.elapsed_time(c2)
    overlap_sketch_ms = c0.elapsed_time(c1)
    return {"producer": "advection-diffusion stand-in (upwind + 7-point Laplacian), "
                        f"{substeps} steps of dt={dt} per snapshot, nu={nu}",
            "solver_ms": solver_ms, "sketch_ms": sketch_ms, "finalize_error_ms": close_ms,
            "overlapped_ms": both_ms,
            "sketch_hidden_fraction": max(0.0, (solver_ms + sketch_ms - overlap_sketch_ms) /
                                          sketch_ms),
            "overhead_vs_solver": both_ms / solver_ms - 1.0,
            "rel_err": float(np.sqrt(t[0] / t[1])), "compression_factor": float(t[2] / t[3]),
            "k_mean": float(np.mean(k)), "k_max": int(np.max(k))}


def _run_insitu(args, torch, inputs, spid):
    """512 boxes of 32^3 x 5 QoIs of a 256^3 field, n = 256, retained in a
    subdomain-major window (86 GB, [box][snapshot][rows]: each arriving snapshot
    lands as 512 contiguous 655 KB pieces); the sketch runs per micro-batch of
    snapshots as they arrive; k 30, p 10 (TF32).  Also: a producer stream writes
    each batch while the sketch consumes the previous one.  (A snapshot-major
    window, where the 64 columns of a sketch tile are 335 MB apart, held the
    sketch at 4.7 TB/s against 7.0 TB/s for this layout: address translation,
    not DRAM, limits the 335 MB column stride.)"""
    S, edge, grid, n, b = 512, 32, 256, 256, args.microbatch
    origins = [(bx * edge, by * edge, bz * edge) for bz in range(8) for by in range(8)
               for bx in range(8)]
    field = inputs.DeviceField(origins, edge, grid, inputs.fourier_modes(seed=2))
    m = 5 * edge ** 3
    window = torch.empty(n * S * m, device="cuda", dtype=torch.float32)
    t_all = 10.0 * np.arange(n) / (n - 1)
    calls = [(j0, min(b, n - j0)) for j0 in range(0, n, b)]
    for j0, nc in calls:
        field.fill_subdomain_major(window, t_all[j0:j0 + nc], j0, n)
    torch.cuda.synchronize()
    nbytes = 4.0 * S * m * n
    err = torch.zeros(2 * S, dtype=torch.float64, device="cuda")
    tot = torch.zeros(4, dtype=torch.float64, device="cuda")
    plan = spid.Plan([m] * S, [n] * S, np.arange(S) * n * m, [m] * S, k_max=30, p=10,
                     precision="tf32", seed=0x5EED0005)
    tuning = None if args.no_autotune else plan.autotune(window)
    sk, fi, er = _stage_times(torch, plan, window, args.steps, args.warmup, err, tot, calls)
    summ = _summary(plan, tot)
    # in-situ overlap: producer writes batch i+1 while the sketch consumes batch i
    prod = torch.cuda.Stream()
    cons = torch.cuda.current_stream()
    ready = [torch.cuda.Event() for _ in calls]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(cons)
    prod.wait_event(e0)
    with torch.cuda.stream(prod):
        for i, (j0, nc) in enumerate(calls):
            field.fill_subdomain_major(window, t_all[j0:j0 + nc], j0, n)
            ready[i].record(prod)
    for i, (j0, nc) in enumerate(calls):
        cons.wait_event(ready[i])
        plan.sketch(window, j0, nc)
    plan.finalize()
    plan.error(window, err, tot)
    e1.record(cons)
    torch.cuda.synchronize()
    overlapped = e0.elapsed_time(e1)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(cons)
    for j0, nc in calls:
        field.fill_subdomain_major(window, t_all[j0:j0 + nc], j0, n)
    p1.record(cons)
    torch.cuda.synchronize()
    produce = p0.elapsed_time(p1)
    solver = _insitu_solver(torch, spid, plan, window, field, t_all, calls, S, m, n, err, tot)
    plan.close()
    step = sk + fi + er
    return {"value": nbytes / (step / 1e3) / 1e9, "ms_per_step": step,
            "dtype": "f32 (tf32 sketch)",
            "config": {"workload": f"in-situ: 512 boxes of 32^3 x 5 QoIs of a 256^3 TGV+Fourier "
                                   f"field, n=256, subdomain-major window (85.9 GB), sketch per "
                                   f"micro-batch of {b} snapshots, k=30, p=10",
                       "l2": "inputs larger than L2", "tuning": tuning},
            "stages_ms": {"sketch": sk, "finalize": fi, "error": er},
            "sketch_gbs": nbytes / (sk / 1e3) / 1e9, "error_gbs": nbytes / (er / 1e3) / 1e9,
            **summ,
            "insitu_overlap": {"producer_ms": produce, "compress_ms": step,
                               "overlapped_ms": overlapped,
                               "hidden_fraction": max(0.0, (produce + step - overlapped) / step)},
            "insitu_solver": solver,
            "_sketch_gbs": nbytes / (sk / 1e3) / 1e9}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="tf32", choices=["tf32", "bf16x3", "bf16", "fp32"])
    ap.add_argument("--ref-subs", type=int, default=16)
    ap.add_argument("--cpu-sample", type=int, default=64)
    ap.add_argument("--boxes", type=int, default=None,
                    help="first N boxes only (small profiling case; not the bench workload)")
    ap.add_argument("--tc-error", action="store_true",
                    help="error pass with the rank-k product on the tensor cores")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default tile shapes (no measurement)")
    ap.add_argument("--workload", default="tgv3d64",
                    choices=["tgv3d64", "spectrum256", "uneven4096", "insitu256",
                             "coarse_tgv3d64", "two_stage_tgv3d64", "points_tgv2d"],
                    help="tgv3d64 is the bench workload; the others print their own line")
    ap.add_argument("--microbatch", type=int, default=64, help="insitu256: columns per call")
    ap.add_argument("--wave-gb", type=float, default=48.0, help="uneven4096: GB per wave")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "tgv3d64":
        return run_workload(args)

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    numa = bind_to_gpu_numa_node(local)
    from paper_2103_01380_gb300 import build, spid
    build.build()
    spid.load_library()

    win = make_window(rank, boxes=args.boxes)
    nbytes = float(win.nbytes_payload())
    host = torch.from_numpy(win.data).pin_memory()
    dev = host.cuda()
    stream = torch.cuda.current_stream()
    err = torch.zeros(2 * win.num_sub, dtype=torch.float64, device="cuda")
    tot = torch.zeros(4, dtype=torch.float64, device="cuda")

    def make_plan(precision, flags=0):
        return spid.Plan.for_window(win, k_max=20, p=10, tol=0.0, precision=precision,
                                    seed=0x5EED0001, flags=flags)

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(plan, steps, warmup, per_stage=True):
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        for _ in range(warmup):
            plan.sketch(dev); plan.finalize(); plan.error(dev, err, tot)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(steps):
            ev[i][0].record(stream)
            plan.sketch(dev)
            ev[i][1].record(stream)
            plan.finalize()
            ev[i][2].record(stream)
            plan.error(dev, err, tot)
            ev[i][3].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier()
        total_ms = t_start.elapsed_time(t_end)
        sk = [e[0].elapsed_time(e[1]) for e in ev]
        fi = [e[1].elapsed_time(e[2]) for e in ev]
        er = [e[2].elapsed_time(e[3]) for e in ev]
        return total_ms, sk, fi, er

    plan = make_plan(args.precision, flags=spid.FLAG_TC_ERROR if args.tc_error else 0)
    # tile shapes and schedules: measured on this window by the library's autotuner
    if args.no_autotune:
        tuning = dict(plan.tuning(), cached=None)
    else:
        tuning = plan.autotune(dev)
    # one step = one CUDA-graph launch (sketch, finalize, error kernels)
    graph = plan.graph(dev, err=err, total=tot)

    def timed_graph(steps, warmup):
        for _ in range(warmup):
            graph.launch()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(steps):
            graph.launch()
        g1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return g0.elapsed_time(g1)

    with ClockSampler(local) as clk:
        # per-stage durations (eager launches, events between the stages), then
        # the headline: the same steps replayed as one graph launch each
        _, sk, fi, er = timed(plan, args.steps, args.warmup)
        total_ms = timed_graph(args.steps, args.warmup)
    clocks = clk.summary()
    t = torch.tensor([total_ms], dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * nbytes * args.steps / (total_ms / 1e3) / 1e9

    # global error / CF across ranks: one host-side sum of four doubles
    from paper_2103_01380_gb300 import shard
    rel_err, cf, _ = shard.combine_totals(tot.detach().cpu().numpy())
    k, J, C = plan.factors()

    # end to end through the public API (spid_graph_launch_host): every step
    # copies the pinned host window to a device window, runs the step's graph
    # and copies the four error sums back to pinned host memory.  Two device
    # windows with a graph each alternate, so one step's copy (on its own
    # stream) overlaps the other's compute; the copies run back to back on the
    # host link, which bounds the rate.
    extent = int(np.max(win.off + win.ld * (win.n.astype(np.int64) - 1) + win.m))
    h2d_bytes = 4 * extent
    dev2 = torch.empty_like(dev)
    graph2 = plan.graph(dev2, err=err, total=tot)
    pair = (graph, graph2)
    copy_stream = torch.cuda.Stream()
    host_tot = [torch.zeros(4, dtype=torch.float64).pin_memory() for _ in range(2)]
    for i in range(2 * max(args.warmup, 1)):
        pair[i % 2].launch_host(host, host_tot[i % 2], copy_stream=copy_stream, stream=stream)
    torch.cuda.synchronize()
    # the host link alone, for reference
    h0 = torch.cuda.Event(enable_timing=True)
    h1 = torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(3):
        dev2.copy_(host, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize()
    h2d_ms = h0.elapsed_time(h1) / 3
    barrier()
    e2e_steps = max(3, args.steps // 4)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy_stream.wait_event(e0)   # no copy starts before the timed region
    for i in range(e2e_steps):
        pair[i % 2].launch_host(host, host_tot[i % 2], copy_stream=copy_stream, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    if not np.array_equal(host_tot[(e2e_steps - 1) % 2].numpy(), tot.cpu().numpy()):
        raise RuntimeError("end-to-end step returned other error sums than the device step")
    te = torch.tensor([e2e_ms], dtype=torch.float64)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = world * nbytes / (float(te.item()) / 1e3) / 1e9
    graph.close()
    graph2.close()
    del dev2

    # comparator: plain FP32 (SIMT sketch, one launch per subdomain per stage, no graph)
    comparator = None
    if not args.no_comparator:
        pl = make_plan("fp32", flags=spid.FLAG_PER_SUBDOMAIN)
        c_ms, c_sk, c_fi, c_er = timed(pl, max(3, args.steps // 4), args.warmup)
        torch.cuda.synchronize()
        c_tot = tot.detach().cpu().numpy()
        comparator = {"form": "plain FP32 (SIMT sketch, per-subdomain launches)",
                      "value": nbytes * max(3, args.steps // 4) / (c_ms / 1e3) / 1e9,
                      "sketch_gbs": nbytes / (statistics.mean(c_sk) / 1e3) / 1e9,
                      "rel_err": float(np.sqrt(c_tot[0] / c_tot[1]))}
        pl.close()
        pb = make_plan("fp32")
        b_ms, b_sk, b_fi, b_er = timed(pb, max(3, args.steps // 4), args.warmup)
        comparator["batched_fp32_value"] = nbytes * max(3, args.steps // 4) / (b_ms / 1e3) / 1e9
        comparator["batched_fp32_sketch_gbs"] = nbytes / (statistics.mean(b_sk) / 1e3) / 1e9
        pb.close()

    peak, peak_kind = load_peaks()
    sk_ms, er_ms, fi_ms = statistics.mean(sk), statistics.mean(er), statistics.mean(fi)
    dominant = "sketch" if sk_ms >= er_ms else "error"
    dom_ms = max(sk_ms, er_ms)
    # algorithmic bytes: sketch reads A once (4 B / element); the error pass reads
    # A once plus the k skeleton columns of every subdomain
    alg_bytes = nbytes if dominant == "sketch" else nbytes + 4.0 * float((k * win.m).sum())
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
            "traffic": measured_traffic(dominant) if (
                args.boxes is None and args.precision == "tf32" and
                all(tuning.get(k) == v for k, v in MEASURED_TUNING.items())) else None,
            "alg_bytes": alg_bytes}

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else f"f32 ({args.precision} sketch)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.boxes is None else
                       f"first {args.boxes} boxes of: " + WORKLOAD, "precision": args.precision,
                       "subdomains_per_gpu": win.num_sub, "bytes_per_step_per_gpu": nbytes,
                       "error_pass": "tensor-core (3xTF32)" if (args.tc_error and
                                                                args.precision != "fp32")
                       else "cuda-core",
                       "l2": "inputs (2.68 GB) larger than L2; no flush",
                       "launch": "one CUDA graph per step (sketch, finalize, error kernels)",
                       "tuning": tuning},
            "stages_ms": {"sketch": sk_ms, "finalize": fi_ms, "error": er_ms},
            "sketch_gbs": nbytes / (sk_ms / 1e3) / 1e9,
            "error_gbs": nbytes / (er_ms / 1e3) / 1e9,
            "rel_err": rel_err, "compression_factor": cf,
            "k_mean": float(np.mean(k)), "k_max": int(np.max(k)),
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": h2d_bytes,
                    "d2h_bytes_per_step": 32, "ms_per_step": e2e_ms,
                    "api": "spid_graph_launch_host, two device windows alternating",
                    "h2d_ms_per_step": h2d_ms, "h2d_gbs": h2d_bytes / (h2d_ms / 1e3) / 1e9,
                    "host_binding": numa},
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
            "comparator": comparator}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(win, min(args.cpu_sample, win.num_sub))
    plan.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
