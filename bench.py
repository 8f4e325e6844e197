"""Benchmark: fill + factor + solve throughput of the H-matrix CBIE solver on one GB300.

One step = the whole hot path on one batch of synthetic input: node geometry,
cluster/block trees and near pairs, near-field CBIE quadrature, dense leaves, ACA +
recompression, H-LU, H-solve for the workload's plane waves, far field / RCS.
The default workload is the PEC sphere of 8 wavelengths diameter (96 patches x
10 x 10 nodes, 19,200 unknowns, leaf 128, eta 2, ACA tolerance 1e-7, 4 seeded
plane waves).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Under torchrun (N > 1) every rank solves its own replica of the workload (the
H-LU does not shard; replicas only) and value = unknowns solved by all ranks / the
slowest rank's time.
"""
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

METRIC = "fill+factor+solve unknowns/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 on GB300: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz (nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64 flops per near-field kernel evaluation: geometry map (2 tan, sqrt, rcp, ~60 fma),
# distance (sqrt), sincos, g(R) (~12), two cross products (12), four dots (12), Chebyshev
# recurrence of one axis (2 Nc) and the moment accumulation (4 components x 2 x Nc) --
# counted as 100 + 18 Nc flops with transcendental calls counted as one flop each.
NEAR_FLOPS_PER_POINT = lambda nc: 100 + 18 * nc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def load_workload(name):
    from paper_2408_17116_gb300 import workloads
    return workloads.workload(name)


def cpu_baseline(wl, budget_s=20.0):
    """The oracle as it stands, on a bounded sample of the workload, scaled to unknowns/s.

    Sample: dense MFIE fill of R rows of the full matrix, and the oracle's dense LU +
    solve of an n_s x n_s leading block of the same matrix's rows/columns.  Full-size
    time = fill_time * N / R + lu_time * (N / n_s)^3 + solve_time * (N / n_s)^2.
    """
    import oracle
    t0 = time.perf_counter()
    o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], wl["k"])
    N = o.N
    rng = np.random.default_rng(0)
    R = 32
    rows = np.sort(rng.choice(N, R, replace=False))
    t = time.perf_counter()
    A = o.matrix_rows(rows)
    t_rows = time.perf_counter() - t
    ns = min(N, 2048)
    idx = np.sort(rng.choice(N, ns, replace=False))
    Bm = o.matrix_rows(idx)[:, idx]  # a principal submatrix of the same operator
    t = time.perf_counter()
    LU, piv, info = oracle.zgetrf(Bm)
    t_lu = time.perf_counter() - t
    b = np.ones(ns, dtype=complex)
    t = time.perf_counter()
    oracle.zgetrs(LU, piv, b)
    t_sol = time.perf_counter() - t
    nrhs = wl["kdirs"].shape[0]
    est = t_rows * N / R + t_lu * (N / ns) ** 3 + t_sol * nrhs * (N / ns) ** 2
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": N / est, "unit": "unknowns/s", "cores": cores, "kind": "oracle",
            "sample": "dense fill of %d of %d rows (%.2f s) + dense LU of a %d x %d principal submatrix "
                      "(%.2f s) + %d solves, extrapolated by N/R, (N/n)^3, (N/n)^2; est. full dense "
                      "fill+LU+solve %.0f s" % (R, N, t_rows, ns, ns, t_lu, nrhs, est),
            "wall_s": time.perf_counter() - t0, "est_full_s": est}


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = load_workload(args.workload)
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(wl)
        if i >= args.warmup:
            vals.append(cb)
    v = statistics.median([c["value"] for c in vals])
    cb = dict(vals[-1])
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "unknowns/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wl_N(wl) / v,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload}, "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def wl_N(wl):
    return 2 * 6 * int(np.sum(np.asarray(wl["ms"]) ** 2)) * wl["nc"] ** 2


PRECISION = {"fp32r": 1, "fp64": 0}


def one_step(s, wl, dirs, host=False, precision="fp32r"):
    s.hm_build_geometry(wl["bodies"], wl["ms"], wl["nc"], wl["k"], wl["leaf"], wl["eta"], wl["aca_tol"],
                        precision=PRECISION[precision])
    s.hm_fill()
    s.hm_factor()
    if host:
        x = s.hm_solve_host(wl["kdirs"], wl["pols"])
        import torch
        xd = torch.from_numpy(x).cuda()
        _, rcs = s.hm_farfield(xd, dirs, want_efar=False)
        return x, rcs
    x = s.hm_solve(wl["kdirs"], wl["pols"])
    efar, rcs = s.hm_farfield(x, dirs)
    return x, rcs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="sphere_d8_m4_nc10")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp32r", choices=sorted(PRECISION),
                    help="fp32r: FP32 H-LU + FP64 refinement (default); fp64: the plain FP64 H-LU")
    ap.add_argument("--no-compare", action="store_true", help="skip the one-step run of the other precision")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        return

    import torch
    from paper_2408_17116_gb300 import build, hm, workloads
    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = load_workload(args.workload)
    _, dirs = workloads.rcs_cuts()
    s = hm.Solver()
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    prec = args.precision
    for _ in range(args.warmup):
        one_step(s, wl, dirs, precision=prec)
    barrier()
    L0 = s.hm_query("LAUNCHES")
    clk = ClockSampler(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    phases = {k: 0.0 for k in ("T_GEOMETRY", "T_NEAR", "T_ACA", "T_RECOMPRESS", "T_DENSE", "T_FACTOR", "T_SOLVE")}
    near_pts = 0.0
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        x, rcs = one_step(s, wl, dirs, precision=prec)
        for k in phases:
            phases[k] += s.hm_query(k)
        near_pts += s.hm_query("NEAR_QPOINTS")
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = int(s.hm_query("LAUNCHES") - L0)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    N = s.N
    value = N * world / (ms / 1000.0)
    stats = {k.lower(): s.hm_query(k) for k in ("CR", "MAX_RANK", "MEAN_RANK", "LR_BLOCKS", "DENSE_BLOCKS",
                                                 "NEAR_PAIRS", "ACA_NONCONV", "FLOPS_FACTOR", "REFINE_ITERS",
                                                 "REFINE_RES", "STORAGE", "STORAGE32")}
    # e2e: host buffers in and out, wall clock around the public API calls
    barrier()
    t = time.perf_counter()
    xh, rcs_h = one_step(s, wl, dirs, host=True, precision=prec)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t
    nrhs = wl["kdirs"].shape[0]
    h2d = 152 * len(wl["ms"]) + 64 + 48 * nrhs + 24 * dirs.shape[0]  # bodies, params, waves, directions
    d2h = 16 * N * nrhs + 8 * nrhs * dirs.shape[0]
    # roofline of the near-field quadrature kernel (FP64 ALU bound), per launch
    per = {k: v / args.steps for k, v in phases.items()}
    near_flops = (near_pts / args.steps) * NEAR_FLOPS_PER_POINT(wl["nc"])
    near_tflops = near_flops / per["T_NEAR"] / 1e12 if per["T_NEAR"] > 0 else 0.0
    roof = {"kernel": "k_near (self/near CBIE quadrature)", "bound": "alu", "achieved": near_tflops,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": near_tflops / FP64_PEAK_TFLOPS, "traffic": None,
            "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz"}
    out = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64 fill; c64 H-LU + f64 refinement" if prec == "fp32r" else "f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "unknowns": N, "rhs": nrhs, "leaf": wl["leaf"], "eta": wl["eta"],
                      "aca_tol": wl["aca_tol"], "precision": prec,
                      "parallelism": "replicas" if world > 1 else "single",
                      "l2": "working set (H-matrix, near store) > L2 between steps"},
           "phases_s": per, "stats": stats, "gpu_launches": launches, "clocks": clocks,
           "e2e": {"value": N / e2e_s, "unit": "unknowns/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "wall_s": e2e_s},
           "roofline": roof}
    if not args.no_compare:
        # the other precision on the same GPU: one untimed warm-up step, one step timed
        other = "fp64" if prec == "fp32r" else "fp32r"
        one_step(s, wl, dirs, precision=other)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step(s, wl, dirs, precision=other)
        e1.record(stream)
        barrier()
        cms = e0.elapsed_time(e1)
        out["compare"] = {"precision": other, "value": N / (cms / 1000.0), "ms_per_step": cms, "steps": 1,
                          "phases_s": {k: s.hm_query(k) for k in phases},
                          "refine_iters": s.hm_query("REFINE_ITERS")}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
