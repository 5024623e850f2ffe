#!/usr/bin/env python
"""ADMM throughput and time-to-solution for face-staggered SAC on GB300.

A step is one ADMM iteration (b-step, z-step, dual update and residual norms;
Sec. 4.2) over the whole volume.  Default workload: the 256 x 256 x 80 3D
phantom (5 263 360 faces), mixed precision (FP32 lines and DCTs, FP64
reductions and near-bound line re-solves).  Inputs are synthetic and seeded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the machine's host cores on the same workload.  With N > 1 each rank runs an
independent replica (the single-volume solve does not shard): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADMM voxel-iters/s (faces x ADMM iterations / s), 5.26M-face 3D SAC"
UNIT = "voxel-iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d_256x256x80")
    ap.add_argument("--no-tts", action="store_true", help="skip the time-to-solution runs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--tts-cap", type=int, default=2000)
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-pair batch run")
    ap.add_argument("--cpu-full", action="store_true",
                    help="CPU oracle baseline in full: also the 128^2 and 128x128x64 configurations to convergence")
    ap.add_argument("--serve-seconds", type=float, default=3.0,
                    help="arrival window of the serving run (Poisson, 20 requests/s); 0 skips it")
    ap.add_argument("--profile-direct", type=int, default=0, metavar="K",
                    help="only run K mixed ADMM iterations through sac_admm_solve (no CUDA graphs, no "
                         "timing line): the launch sequence for kernel profilers")
    ap.add_argument("--only-mixed", action="store_true",
                    help="only the warm-up and the timed mixed-precision iterations (profiling runs)")
    return ap.parse_args()


def load_workload(name):
    """The seeded phantom pair (cached in the temporary directory)."""
    from paper_1607_00531_gb300 import phantoms as ph
    return ph.load_pair(name, np.float32)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.marks = []

    def __enter__(self):
        # started ahead of the timed region so that it samples during it
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.5)
        except OSError:
            self.p = None
        return self

    def mark(self):
        """Call at the start and at the end of the timed region."""
        self.marks.append(time.time())

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if len(self.marks) >= 2:
            import datetime
            t0, t1 = self.marks[0], self.marks[-1]
            sel = []
            for r in rows:
                try:
                    ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    continue
                if t0 - 0.02 <= ts <= t1 + 0.02:
                    sel.append(r)
            rows = sel
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def max_over_ranks(t_ms, dist_mod, device):
    """The slowest rank's time: every rank takes part (any backend); one rank
    or no process group returns its own."""
    if not dist_mod:
        return t_ms
    import torch
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist_mod.all_reduce(tt, op=dist_mod.ReduceOp.MAX)
    return float(tt.item())


def job_value(world, units_per_rank, steps, t_ms):
    """Whole-job throughput: the units of every rank (replicas of the same
    volume) over the slowest rank's time."""
    return world * units_per_rank * steps / (t_ms / 1e3)


def roofline(prof, w, g, nf, sac):
    """Per phase: algorithmic HBM bytes and algorithmic flops per launch over
    the measured average launch time; the binding roof (larger fraction) of
    the dominant phase is reported."""
    hbm, smmax, src = peaks()
    bf16 = 1955.6
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            bf16 = json.load(fh).get("bf16_tflops", bf16)
    tf32_peak = bf16 * (1.1 / 2.25)          # measured BF16 x nominal TF32/BF16 ratio (dense)
    fp16_peak = bf16                         # FP16 products run at the BF16 rate (dense)
    fp32_peak = 152 * 128 * 2 * smmax * 1e6 / 1e12
    cells = int(np.prod(w.m))
    F = sac.face_shape(g)
    axes = [a for a in range(3) if a != w.pe]
    L1 = F[axes[0]] if axes[0] < len(F) else 1
    L2 = F[axes[1]] if axes[1] < len(F) else 1
    # FP32 arrays read + written per face: pass 0 b, u -> t1; passes 1-3
    # one array in, one out; the update reads b, u, t2, z and writes u, z
    # On the chip (one launch per iteration, fused stopping test): b, u and
    # z^k read, z and u written; the four contractions' products
    per_face_bytes = {"zpass0": 12, "zpass1": 8, "zpass2": 8, "zpass3": 8, "admm_update": 24, "zslab": 20}
    flops = {"zpass0": 2 * L1 * nf, "zpass3": 2 * L1 * nf, "zpass1": 2 * L2 * nf, "zpass2": 2 * L2 * nf,
             "zslab": 2 * (2 * L1 + 2 * L2) * nf}
    mode = sac.zstep_fused(g, sac.params(alpha=w.alpha, rho=w.rho, prec="mixed"))
    fused = mode == 1
    if fused:
        # passes 1 and 2 in one launch (phase 1): one array in, one out, both products
        flops["zpass1"] = 4 * L2 * nf
    nphase = {k: v for k, v in prof.items() if v[1] > 0 and not (fused and k == "zpass2")}
    tot_ms = sum(v[0] for v in nphase.values())
    kernels = {}
    for k, (ms, n) in nphase.items():
        avg = ms / n / 1e3
        if k == "admm_update":
            byts = per_face_bytes[k] * nf
            ach_b = byts / avg / 1e9
            ent = {"ms_total": ms, "launches": n, "share": ms / tot_ms, "bytes": byts, "achieved_gbs": ach_b,
                   "frac_hbm": ach_b / hbm, "bound": "hbm"}
        elif k in ("bstep", "bstep_refine"):
            byts = 2 * 4 * cells + 4 * 4 * nf if k == "bstep" else None
            ent = {"ms_total": ms, "launches": n, "share": ms / tot_ms}
            if byts:
                ent.update(bound="hbm", bytes=byts, achieved_gbs=byts / avg / 1e9, frac_hbm=byts / avg / 1e9 / hbm)
        else:
            byts = per_face_bytes[k] * nf
            ach_b = byts / avg / 1e9
            ach_f = flops[k] / avg / 1e12
            tpk = fp16_peak if k == "zslab" else tf32_peak
            ent = {"ms_total": ms, "launches": n, "share": ms / tot_ms, "bytes": byts, "flops": flops[k],
                   "achieved_gbs": ach_b, "frac_hbm": ach_b / hbm, "achieved_tflops": ach_f,
                   "tensor_peak": tpk, "frac_tensor": ach_f / tpk}
            ent["bound"] = "hbm" if ent["frac_hbm"] >= ent["frac_tensor"] else "tensor"
        kernels[k] = ent
    # kernels behind each phase: axes of at most 128 faces run the lines-in-N
    # tensor-core kernel, longer ones the lines-in-M kernel; the element-wise
    # ADMM update also runs the stopping test (in each volume's last block)
    def zk(L, q):
        return (f"k_axis_tcn<{q}>" if L <= 128 else f"k_axis_tc<{q}>")
    # b-step: strided PE lines of at most 272 faces take the segment kernel
    # (9 faces per segment up to 144 faces, else 17), others one warp per line
    nfl = w.m[w.pe] + 1
    kpl = next(k for k in (3, 5, 9, 15) if (nfl + 31) // 32 <= k)
    if w.pe < len(w.m) - 1 and nfl <= 272:
        bname = f"k_bstep_seg<{9 if nfl <= 144 else 17}>"
    else:
        bname = f"k_bstep<float,float,{kpl}>"
    names = {"bstep": bname, "bstep_refine": f"k_bstep_list<double,float,{kpl}>",
             "zpass0": zk(L1, 0), "zpass1": "k_axis_tc<4>" if fused else zk(L2, 1), "zpass2": zk(L2, 2),
             "zpass3": zk(L1, 3), "admm_update": "k_admm_update", "zslab": "k_zslab<1>"}
    for k in kernels:
        kernels[k]["kernel"] = names.get(k, k)
    dom = max(nphase, key=lambda k: nphase[k][0])
    e = kernels[dom]
    traffic = ncu_traffic().get(names[dom].split(" ")[0])
    if e.get("bound") == "tensor":
        psrc = (f"{src}: bf16 {bf16:.1f} TFLOP/s (FP16 at the BF16 rate; split FP16 runs 3 MMAs per product)"
                if dom == "zslab" else
                f"{src}: bf16 {bf16:.1f} TFLOP/s x nominal TF32/BF16 1.1/2.25 (split TF32 runs 3 MMAs per product)")
        roof = {"kernel": names[dom], "bound": "tensor", "achieved": e["achieved_tflops"],
                "peak": e["tensor_peak"], "unit": "TFLOP/s", "frac": e["frac_tensor"], "traffic": traffic,
                "algorithmic_flops_per_launch": e["flops"], "peak_source": psrc}
    else:
        roof = {"kernel": names[dom], "bound": "hbm", "achieved": e["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                "frac": e["frac_hbm"], "traffic": traffic, "algorithmic_bytes_per_launch": e["bytes"],
                "peak_source": f"{src} HBM copy bandwidth (MEASURED_PEAKS.json)"}
    roof["fp32_simt_peak_tflops"] = fp32_peak
    return roof, kernels


def ncu_traffic():
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    of kernels from one ncu capture each, as recorded in
    profiles/ncu_traffic.json (absent: null traffic)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        d = json.load(fh)
    return {k: v.get("bytes_per_launch") for k, v in d.get("kernels", {}).items()}


def serve_run(args, sac, dev):
    """Requests drawn uniformly from the five serving kinds (2D 128^2 and 256^2,
    3D 96x96x60, 128x128x64 and 256x256x80), arriving as a Poisson process of
    20 requests per second for args.serve_seconds, each with its own seeded
    phantom and field (generated before the arrival window).  The server
    admits requests while its 40 GB pool has room, iterates all admitted ones
    together and retires them at relative residual 1e-4 (at most 2000
    iterations).  Beside it: one request of each kind solved alone in plain
    FP64 (sac_admm_solve, same stop), measured."""
    import torch
    from paper_1607_00531_gb300 import phantoms as ph
    rng = np.random.default_rng(5)
    arrivals = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / 20.0)
        if t > args.serve_seconds:
            break
        arrivals.append((t, int(rng.integers(len(ph.SERVING_KINDS)))))
    t0 = time.perf_counter()
    pairs = []
    for i, (_, kind) in enumerate(arrivals):
        wk = ph.serving_workload(kind, 1000 + i)
        dk = ph.make_pair(wk, dtype=np.float32, device=dev)
        pairs.append((sac.grid(wk.m, wk.h, wk.pe), dk["I1"], dk["I2"], kind))
    gen_s = time.perf_counter() - t0
    p = sac.params(alpha=50.0, rho=1e2, prec="mixed", max_iter=2000, eps_abs=0.0, eps_rel=1e-4, near_bound=1e-3)
    srv = sac.Server(p, pool_bytes=40 << 30, max_jobs=64)
    kinds = {}
    open_t = {}
    done = {}
    t0 = time.perf_counter()
    i = 0
    while i < len(arrivals) or open_t:
        now = time.perf_counter() - t0
        while i < len(arrivals) and arrivals[i][0] <= now:
            g, A, B, _ = pairs[i]
            tk = srv.submit(g, A, B)
            open_t[tk] = i
            i += 1
        if open_t:
            srv.step(20, chunk=10)
            for tk in list(open_t):
                info = srv.poll(tk)
                if info["state"] == 2:
                    done[tk] = (open_t.pop(tk), info)
        elif i < len(arrivals):
            time.sleep(max(0.0, arrivals[i][0] - (time.perf_counter() - t0)))
    torch.cuda.synchronize()
    lat = np.array([inf["t_done"] - inf["t_submit"] for _, inf in done.values()])
    first = min(inf["t_submit"] for _, inf in done.values())
    last = max(inf["t_done"] for _, inf in done.values())
    work = 0
    for i_req, inf in done.values():
        g, kind = pairs[i_req][0], pairs[i_req][3]
        work += int(np.prod(sac.face_shape(g))) * inf["iters"]
        kinds.setdefault(str(tuple(ph.SERVING_KINDS[kind][0])), []).append(inf["iters"])
    srv.close()
    # plain FP64 alone: the first request of each kind, same stopping test
    alone = {}
    for i_req, (g, A, B, kind) in enumerate(pairs):
        key = str(tuple(ph.SERVING_KINDS[kind][0]))
        if key in alone:
            continue
        pf = sac.params(alpha=50.0, rho=1e2, prec="f64", max_iter=2000, eps_abs=0.0, eps_rel=1e-4, check_every=10)
        A1 = torch.as_tensor(A, device=dev).double()
        A2 = torch.as_tensor(B, device=dev).double()
        bk = torch.zeros(sac.face_shape(g), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = sac.admm_solve(g, pf, A1, A2, bk)
        torch.cuda.synchronize()
        alone[key] = {"request": i_req, "seconds": time.perf_counter() - t0, "iterations": r["iters"],
                      "converged": r["converged"]}
    # every request's latency alone in FP64 = its kind's measured time, back to back
    f64_lat = np.array([alone[str(tuple(ph.SERVING_KINDS[pairs[i_req][3]][0]))]["seconds"]
                        for i_req, _ in done.values()])
    return {"requests": len(done), "arrival_rate_per_s": 20.0, "window_s": args.serve_seconds,
            "budget_bytes": 40 << 30, "stop": "relative residual 1e-4, at most 2000 iterations",
            "phantoms": "one seeded phantom and field per request", "phantoms_s": gen_s,
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
            "converged": int(sum(1 for _, inf in done.values() if inf["converged"])),
            "makespan_s": last - first, "value": work / (last - first), "unit": UNIT,
            "iterations_by_kind": {k: {"n": len(v), "mean": float(np.mean(v))} for k, v in kinds.items()},
            "f64_alone": {"by_kind": alone,
                          "solve_s": {"p50": float(np.percentile(f64_lat, 50)),
                                      "p99": float(np.percentile(f64_lat, 99))},
                          "sum_s": float(f64_lat.sum()),
                          "note": "one request per kind solved alone in plain FP64 (measured); every request "
                                  "assigned its kind's time; sum_s: all requests back to back"}}


def workload_config(w, nf, world):
    """The workload both arms run (the same dict in both JSON lines)."""
    return {"workload": w.name, "faces": nf, "grid": list(w.m), "pe_axis": w.pe, "alpha": w.alpha, "rho": w.rho,
            "parallelism": f"replicas{world}",
            "l2": "working set > 129 MB L2 (images, b, z, u, two scratch arrays)"}


def batch64_run(args, sac, dev):
    """The DTI-like batch: 64 pairs of 96 x 96 x 60 (independent seeded
    fields of 2-6 px, SNR 10-40) in one engine, one launch per phase over all
    lines and slabs of all pairs, CUDA-graph replay, autotuned line tiles,
    mixed precision.  Throughput over K timed iterations, then the time to
    solution (relative residual 1e-4, device-side stopping per pair), against
    pairs solved alone in plain FP64 (a sample of 4, extrapolated to 64)."""
    import torch
    from paper_1607_00531_gb300 import phantoms as ph
    ws = ph.batch_workloads(64)
    t0 = time.perf_counter()
    pairs = [ph.make_pair(wk, dtype=np.float32, device=dev) for wk in ws]
    gen_s = time.perf_counter() - t0
    grids = [sac.grid(wk.m, wk.h, wk.pe) for wk in ws]
    nf = sum(int(np.prod(sac.face_shape(gk))) for gk in grids)
    I1s = [torch.as_tensor(pk["I1"], device=dev) for pk in pairs]
    I2s = [torch.as_tensor(pk["I2"], device=dev) for pk in pairs]
    K = 20

    def engine(max_iter, eps_rel, autotune):
        p = sac.params(alpha=ws[0].alpha, rho=ws[0].rho, prec="mixed", max_iter=max_iter, eps_abs=0.0,
                       eps_rel=eps_rel, near_bound=1e-3, autotune=autotune)
        bs = [torch.zeros(sac.face_shape(gk), dtype=torch.float64, device=dev) for gk in grids]
        return sac.Batch(grids, p, I1s, I2s, bs), bs

    bt, _ = engine(1 << 30, 0.0, 1)
    bt.run(5, chunk=5)
    bt.run(K, chunk=K)
    ms = bt.last_run_ms()
    bt.close()
    cap = args.tts_cap
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt, _ = engine(cap, 1e-4, 0)
    bt.run(cap, chunk=10)
    st = bt.stats()
    bt.finish()
    torch.cuda.synchronize()
    tts_s = time.perf_counter() - t0
    bt.close()
    its = st["iters"]
    # plain FP64, one pair at a time (sac_admm_solve), on a sample of pairs
    sample = [0, 21, 42, 63]
    alone = []
    for k in sample:
        gk = grids[k]
        pf = sac.params(alpha=ws[k].alpha, rho=ws[k].rho, prec="f64", max_iter=cap, eps_abs=0.0, eps_rel=1e-4,
                        check_every=10)
        bk = torch.zeros(sac.face_shape(gk), dtype=torch.float64, device=dev)
        A1, A2 = I1s[k].double(), I2s[k].double()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = sac.admm_solve(gk, pf, A1, A2, bk)
        torch.cuda.synchronize()
        alone.append({"pair": k, "seconds": time.perf_counter() - t0, "iterations": r["iters"],
                      "converged": r["converged"]})
    mean_alone = float(np.mean([a["seconds"] for a in alone]))
    return {"pairs": 64, "grid": [96, 96, 60], "faces": nf, "prec": "mixed",
            "phantoms_s": gen_s,
            "throughput": {"value": nf * K / (ms / 1e3), "unit": UNIT, "iterations": K, "ms_per_iteration": ms / K,
                           "timed": "sac_batch_run: CUDA-graph replay, device time"},
            "time_to_solution": {"seconds": tts_s, "stop": "relative residual 1e-4 per pair, at most %d" % cap,
                                 "converged": int(np.sum(st["converged"])),
                                 "iterations": {"min": int(its.min()), "median": float(np.median(its)),
                                                "max": int(its.max())}},
            "f64_alone": {"sample": alone, "mean_seconds_per_pair": mean_alone,
                          "extrapolated_64_pairs_s": 64 * mean_alone,
                          "note": "4 pairs solved one at a time in plain FP64 (sac_admm_solve), extrapolated"},
            "speedup_vs_f64_alone": 64 * mean_alone / tts_s}


def cpu_baseline_run(args, d, w):
    """The FP64 oracle as it stands on the host cores: K = 5 ADMM iterations
    of the bench volume on all cores (the reported value) and one on a single
    thread; the 128^2 slice to the benchmark's stopping test (relative
    residual 1e-4, at most 2000 iterations) on all cores; with --cpu-full
    also 5 single-thread iterations and the 128 x 128 x 64 volume to that
    test."""
    import oracle
    nfc, ts, cores = oracle_cpu_baseline(d, w, iters=5)
    out = {"value": nfc * len(ts) / sum(ts), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"5 full FP64 ADMM iterations of {w.name} ({nfc} faces) on {cores} threads, "
                     f"{sum(ts):.2f} s"}
    n1 = 5 if args.cpu_full else 1
    _, ts1, _ = oracle_cpu_baseline(d, w, iters=n1, nthreads=1)
    out["one_thread"] = {"value": nfc * n1 / sum(ts1), "unit": UNIT, "iterations": n1, "seconds": sum(ts1)}
    out["nproc"] = os.cpu_count()
    tts = {}
    for name in (("2d_128", "3d_128x128x64") if args.cpu_full else ("2d_128",)):
        wc, dc = load_workload(name)
        og = oracle.Grid(wc.m, wc.h, wc.pe)
        prm = oracle.Params(alpha=wc.alpha, rho=wc.rho, max_iter=args.tts_cap, eps_abs=0.0, eps_rel=1e-4)
        t0 = time.perf_counter()
        r = oracle.admm(og, prm, dc["I1"].astype(np.float64), dc["I2"].astype(np.float64), np.zeros(og.face_shape))
        tts[name] = {"seconds": time.perf_counter() - t0, "iterations": r["iters"], "converged": r["converged"],
                     "cores": cores}
    out["time_to_solution"] = tts
    return out


def oracle_cpu_baseline(d, w, iters=1, nthreads=0):
    """The FP64 oracle as it stands, on the host cores: `iters` ADMM
    iterations over the full volume."""
    import oracle
    og = oracle.Grid(w.m, w.h, w.pe)
    prm = oracle.Params(alpha=w.alpha, rho=w.rho, max_iter=1, eps_abs=0.0, eps_rel=0.0, nthreads=nthreads)
    I1 = d["I1"].astype(np.float64)
    I2 = d["I2"].astype(np.float64)
    b = np.zeros(og.face_shape)
    z = b.copy()
    u = b.copy()
    ts = []
    for _ in range(iters):
        t0 = time.perf_counter()
        r = oracle.admm(og, prm, I1, I2, b, z, u)
        ts.append(time.perf_counter() - t0)
        b, z, u = r["b"], r["z"], r["u"]
    nf = int(np.prod(og.face_shape))
    return nf, ts, oracle.max_threads()


def run_reference(args, w, d, rank):
    """--impl reference: the CPU oracle timed on the same workload."""
    if rank != 0:
        return
    nf, ts, cores = oracle_cpu_baseline(d, w, iters=args.warmup + args.steps)
    t = sum(ts[args.warmup:])
    val = nf * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, nf, args.gpus),
            "timed": "the FP64 CPU oracle (sac_oracle.c) as it stands: K full ADMM iterations on the host cores",
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full ADMM iterations of {w.name} after {args.warmup} warm-up"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w, d = load_workload(args.workload)
    if args.impl == "reference":
        run_reference(args, w, d, rank)
        return

    import torch
    from paper_1607_00531_gb300 import build as sac_build
    from paper_1607_00531_gb300 import sac

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(sac.LIB_PATH):
        sac_build.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", local)
    g = sac.grid(w.m, w.h, w.pe)
    nf = int(np.prod(sac.face_shape(g)))
    I1 = torch.as_tensor(d["I1"], dtype=torch.float32, device=dev)
    I2 = torch.as_tensor(d["I2"], dtype=torch.float32, device=dev)
    I1d, I2d = I1.double(), I2.double()

    def params(prec, iters, eps_rel=0.0, every=None):
        return sac.params(alpha=w.alpha, rho=w.rho, prec=prec, max_iter=iters, eps_abs=0.0, eps_rel=eps_rel,
                          check_every=every or max(iters, 1), near_bound=1e-3)

    def batch(prec, I1x, I2x, max_iter, eps_rel=0.0, autotune=1, **kw):
        p = sac.params(alpha=w.alpha, rho=w.rho, prec=prec, max_iter=max_iter, eps_abs=0.0, eps_rel=eps_rel,
                       near_bound=1e-3, autotune=autotune)
        for k, v in kw.items():
            setattr(p, k, v)
        bb = torch.zeros(sac.face_shape(g), dtype=torch.float64, device=dev)
        return sac.Batch([g], p, [I1x], [I2x], [bb]), bb

    stream = torch.cuda.current_stream()

    if args.profile_direct > 0:
        pm = sac.params(alpha=w.alpha, rho=w.rho, prec="mixed", max_iter=args.profile_direct, eps_abs=0.0,
                        eps_rel=0.0, check_every=args.profile_direct, near_bound=1e-3)
        b0 = torch.zeros(sac.face_shape(g), dtype=torch.float64, device=dev)
        r = sac.admm_solve(g, pm, I1, I2, b0)
        torch.cuda.synchronize()
        print(json.dumps({"profile_direct": args.profile_direct, "workload": args.workload, "iters": r["iters"],
                          "r_pri": r["r_pri"]}))
        return

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # headline: the batched engine on this volume (tables built once, CUDA-graph
    # replay, device-side stopping); warm-up W iterations (autotuning the
    # b-step tile width on live iterations), then exactly K timed iterations
    big = 1 << 30
    bt, bmix = batch("mixed", I1, I2, big)
    bt.run(args.warmup, chunk=args.warmup)
    barrier()
    n0 = sac.launch_count()
    with Clocks(local) as clk:
        clk.mark()
        bt.run(args.steps, chunk=args.steps)
        barrier()
        clk.mark()
    launches = sac.launch_count() - n0
    t_ms = bt.last_run_ms()
    # the per-phase device times (CUDA events recorded between the kernels
    # of the graph) from a second run of the same K iterations: the event
    # nodes are kept out of the timed run above
    sac.profile_enable(True)
    sac.profile_read(reset=True)
    bt.run(args.steps, chunk=args.steps)
    barrier()
    prof = sac.profile_read(reset=True)
    sac.profile_enable(False)
    t_prof_ms = bt.last_run_ms()
    assert int(bt.stats()["iters"][0]) == args.warmup + 2 * args.steps
    bt.finish()
    bt.close()
    t_ms = max_over_ranks(t_ms, dist, dev)
    value = job_value(world, nf, args.steps, t_ms)
    clocks = clk.summary()
    if args.only_mixed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "steps": args.steps,
                              "ms_per_step": t_ms / args.steps, "gpu_launches": launches,
                              "profiled_run_ms_per_step": t_prof_ms / args.steps,
                              "kernels": {k: v for k, v in prof.items()}}), flush=True)
        return

    # plain FP64 GPU path, same engine (FP64 is slow on GB300: fewer iterations)
    kf = max(3, min(args.steps, 10))
    btf, _ = batch("f64", I1d, I2d, big, autotune=0)
    btf.run(2, chunk=2)
    btf.run(kf, chunk=kf)
    f64_ms = btf.last_run_ms()
    # the FP64 path's z-step passes (SIMT FP64 DCT contractions) against the
    # GPU's FP64 rate, measured here as a cuBLAS DGEMM (4096^3, best of 3)
    sac.profile_enable(True)
    sac.profile_read(reset=True)
    btf.run(kf, chunk=kf)
    prof64 = sac.profile_read(reset=True)
    sac.profile_enable(False)
    btf.close()
    f64_val = nf * kf / (f64_ms / 1e3)
    f64_detail = {}
    try:
        import torch
        A = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
        B = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
        torch.matmul(A, B)
        best = 1e30
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(A, B)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        dgemm = 2 * 4096 ** 3 / (best / 1e3) / 1e12
        del A, B
        Fs = sac.face_shape(g)
        ax = [a for a in range(3) if a != w.pe]
        Ls = [Fs[ax[0]], Fs[ax[1]], Fs[ax[1]], Fs[ax[0]]]
        passes = {}
        for q in range(4):
            ms_q, n_q = prof64.get(f"zpass{q}", (0.0, 0))
            if n_q:
                tf = 2 * Ls[q] * nf / (ms_q / n_q / 1e3) / 1e12
                passes[f"zpass{q}"] = {"us": ms_q / n_q * 1e3, "tflops": tf, "frac_of_dgemm": tf / dgemm}
        f64_detail = {"fp64_dgemm_tflops": dgemm, "zstep_passes": passes,
                      "note": "SIMT FP64 DCT contractions (2 L flop per face per pass) against a measured cuBLAS DGEMM"}
    except Exception as ex:   # reported, not fatal
        f64_detail = {"error": str(ex)[:200]}

    # end to end through the single-volume public call (sac_admm_solve) with
    # host buffers: H2D inputs, K iterations (set-up of the DCT tables
    # included), D2H result
    pm = sac.params(alpha=w.alpha, rho=w.rho, prec="mixed", max_iter=args.steps, eps_abs=0.0, eps_rel=0.0,
                    check_every=args.steps, near_bound=1e-3)
    ws = sac.workspace(g, pm, device=dev)
    hI1 = torch.empty(I1.shape, dtype=torch.float32, pin_memory=True).copy_(I1.cpu())
    hI2 = torch.empty(I2.shape, dtype=torch.float32, pin_memory=True).copy_(I2.cpu())
    hb = torch.zeros(sac.face_shape(g), dtype=torch.float64, pin_memory=True)
    hout = torch.empty(sac.face_shape(g), dtype=torch.float64, pin_memory=True)
    dI1, dI2, db = torch.empty_like(I1), torch.empty_like(I2), torch.zeros(sac.face_shape(g), dtype=torch.float64, device=dev)
    sac.admm_solve(g, sac.params(alpha=w.alpha, rho=w.rho, prec="mixed", max_iter=2, eps_abs=0.0, eps_rel=0.0),
                   I1, I2, torch.zeros_like(db), ws=ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    dI1.copy_(hI1, non_blocking=True)
    dI2.copy_(hI2, non_blocking=True)
    db.copy_(hb, non_blocking=True)
    sac.admm_solve(g, pm, dI1, dI2, db, ws=ws)
    hout.copy_(db, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    del ws
    h2d = hI1.numel() * 4 + hI2.numel() * 4 + hb.numel() * 8
    d2h = hout.numel() * 8
    e2e = {"value": world * nf * args.steps / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "per_solve": {"call": "sac_admm_solve", "iterations": args.steps, "h2d_bytes": h2d, "d2h_bytes": d2h,
                         "stopping_test_every": args.steps,
                         "note": "one stopping test per solve (the headline engine run tests every iteration)"}}

    # time to solution at relative residual 1e-4 (Eq. admmStop with eps_abs = 0,
    # eps_rel = 1e-4), device-side stopping, mixed and plain FP64
    tts = None
    if not args.no_tts:
        tts = {}
        b_by = {}
        for prec, A1, A2 in (("mixed", I1, I2), ("f64", I1d, I2d)):
            cap = args.tts_cap
            barrier()
            t0 = time.perf_counter()
            btt, bres = batch(prec, A1, A2, cap, eps_rel=1e-4, autotune=0)
            btt.run(cap, chunk=10)
            st = btt.stats()
            btt.finish()
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            btt.close()
            b_by[prec] = (int(st["iters"][0]), bres.clone())
            tts[prec] = {"seconds": sec, "device_ms": None, "iterations": int(st["iters"][0]),
                         "converged": bool(st["converged"][0]), "r_pri": float(st["r_pri"][0]),
                         "r_dual": float(st["r_dual"][0]), "cap": cap}
        # the two converged results: field difference and relative objective
        # (FP64 objective on the GPU, parity-tested against the oracle)
        po = sac.params(alpha=w.alpha, prec="f64", beta=0.0)
        Jm = sac.objective(g, po, I1d, I2d, b_by["mixed"][1])["J"]
        Jf = sac.objective(g, po, I1d, I2d, b_by["f64"][1])["J"]
        tts["converged_mixed_vs_f64"] = {
            "max_abs_db_voxels": float((b_by["mixed"][1] - b_by["f64"][1]).abs().max().item() / w.h[w.pe]),
            "relative_objective": abs(Jm - Jf) / abs(Jf), "J_mixed": Jm, "J_f64": Jf,
            "speedup_time_to_solution": tts["f64"]["seconds"] / tts["mixed"]["seconds"]}
        # accuracy of the mixed path against the plain FP64 path after the same
        # number of iterations
        kk = min(b_by["mixed"][0], b_by["f64"][0])
        btm, bm = batch("mixed", I1, I2, kk, autotune=0)
        btm.run(kk, chunk=10); btm.finish(); btm.close()
        bt6, b6 = batch("f64", I1d, I2d, kk, autotune=0)
        bt6.run(kk, chunk=10); bt6.finish(); bt6.close()
        tts["mixed_vs_f64_same_iterations"] = {
            "iterations": kk, "max_abs_db_voxels": float((bm - b6).abs().max().item() / w.h[w.pe])}
        # the paper's augmentation schedule (Sec. 6): adaptive rho from 1e6,
        # bounded below by 1e2 (the fixed value above), one level and three
        # levels (coarse-to-fine, Sec. 4.4), mixed precision
        cap = args.tts_cap
        barrier()
        t0 = time.perf_counter()
        bta, bra = batch("mixed", I1, I2, cap, eps_rel=1e-4, autotune=0, rho=1e6, adapt_rho=2, rho_min=w.rho)
        bta.run(cap, chunk=10)
        st = bta.stats()
        bta.finish()
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        bta.close()
        tts["mixed_adaptive_rho"] = {"seconds": sec, "iterations": int(st["iters"][0]),
                                     "converged": bool(st["converged"][0]), "r_pri": float(st["r_pri"][0]),
                                     "r_dual": float(st["r_dual"][0]), "cap": cap,
                                     "rho": {"start": 1e6, "min": w.rho, "tau": 1.3, "mu": 10.0}}
        levels = 3
        if all(x % (1 << (levels - 1)) == 0 for x in w.m):
            pml = sac.params(alpha=w.alpha, rho=1e6, prec="mixed", max_iter=cap, eps_abs=0.0, eps_rel=1e-4,
                             near_bound=1e-3, adapt_rho=2, rho_min=w.rho)
            bml = torch.zeros(sac.face_shape(g), dtype=torch.float64, device=dev)
            barrier()
            t0 = time.perf_counter()
            rml = sac.multilevel_solve(g, levels, pml, I1, I2, bml)
            torch.cuda.synchronize()
            tts["mixed_multilevel"] = {"seconds": time.perf_counter() - t0, "levels": levels,
                                       "iterations_per_level": rml["iters"], "converged": rml["status"] == 0,
                                       "rho_final": rml["rho"], "cap_per_level": cap}

    # GN-PCG preconditioners (Sec. 4.1, Sec. 6): Jacobi against block-Jacobi
    # on the 2D 128 x 128 slice (the paper compares them in 2D), FP64
    pcg = None
    if not args.no_tts and rank == 0:
        wp, dp_ = load_workload("2d_128")
        gp = sac.grid(wp.m, wp.h, wp.pe)
        A1 = torch.as_tensor(dp_["I1"], dtype=torch.float64, device=dev)
        A2 = torch.as_tensor(dp_["I2"], dtype=torch.float64, device=dev)
        pcg = {"workload": wp.name, "faces": int(np.prod(sac.face_shape(gp))), "prec": "f64",
               "alpha": wp.alpha, "beta": 10.0, "max_gn": 10, "eta": 0.1, "max_pcg": 500}
        for name, pc in (("none", 0), ("jacobi", 1), ("block_jacobi", 2)):
            pp = sac.params(alpha=wp.alpha, beta=10.0, prec="f64", max_gn=10, eta=0.1, precond=pc, max_pcg=500)
            bp = torch.zeros(sac.face_shape(gp), dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rp = sac.gnpcg_solve(gp, pp, A1, A2, bp, want_hist=True)
            torch.cuda.synchronize()
            pcg[name] = {"seconds": time.perf_counter() - t0, "gn_iterations": rp["iters"],
                         "pcg_iterations": int(rp["hist"][:, 2].sum()),
                         "pcg_per_gn": [int(x) for x in rp["hist"][:, 2]], "J": rp["J"]}

    # serving (continuous batching, Poisson arrivals of mixed-size requests,
    # 40 GB device budget, stop at relative residual 1e-4): per-request latency
    # and throughput
    serving = None
    if args.serve_seconds > 0 and rank == 0 and world == 1:
        serving = serve_run(args, sac, dev)
    batch64 = None
    if not args.no_batch and rank == 0 and world == 1:
        batch64 = batch64_run(args, sac, dev)

    # roofline of the dominant kernel (largest summed device time in the timed region)
    roof, kernels = roofline(prof, w, g, nf, sac)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_run(args, d, w)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": workload_config(w, nf, world),
                "prec": "mixed",
                "timed": "sac_batch_run (one volume): CUDA-graph replay of K iterations, device time",
                "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "profiled_run_ms_per_step": t_prof_ms / args.steps,
                "f64_path": {"value": f64_val, "unit": UNIT, "iterations": kf,
                             "mixed_over_f64": value / world / f64_val, **f64_detail},
                "time_to_solution": tts,
                "gnpcg_preconditioners": pcg,
                "serving": serving,
                "batch64": batch64,
                "context": "paper: < 50 s for > 5M dof, three-level ADMM, MATLAB on a laptop CPU"}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
