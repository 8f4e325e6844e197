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
# DRAM bytes (read + write) of one k_near launch per near patch pair, from the ncu capture of
# the 4,800-unknown sphere (0.630 MB read + 62.312 MB written for 192 pairs; part of the
# written near store was still in L2 when that kernel ended, so this is a lower bound)
NEAR_DRAM_BYTES_PER_PAIR = (0.630272e6 + 62.311936e6) / 192


def tensor_peak():
    """Sustained dense BF16 tensor rate (TFLOP/s) of this GPU and where it comes from."""
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "of measured (MEASURED_PEAKS.json bf16_tflops_sustained)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "of fallback (1.7 PFLOP/s sustained BF16)"
# ALU peaks derived from unit counts and the maximum SM clock (2.07 GHz): FP64 on GB300,
# 152 SMs x 2 FP64 FMA/clk x 2 flops (nominal 1.25 TFLOP/s); FP32 CUDA cores,
# 152 SMs x 128 FP32 FMA/clk x 2 flops.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
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


_LU_SAMPLE = {}


def cpu_baseline(wl, workload_name):
    """The oracle as it stands, timed on a bounded sample of the workload (host cores).

    Sample of one step: the dense fill of R = 32 evenly spaced rows of the full N x N
    matrix, and the oracle's right-looking LU with partial pivoting plus the solves of an
    n_s x n_s principal submatrix of the same operator (n_s = 3,072: 151 MB, larger than
    the host's caches, so the LU streams memory as the full-size one does).  The
    submatrix's rows are filled once per process, outside the timed step.
    Estimate of the full dense fill + LU + solve (not a measurement; the fill is linear in
    the rows, the LU's work and memory traffic cubic and the solves quadratic in the size):
        t_full = t_rows N / R + t_lu (N / n_s)^3 + t_solve (N / n_s)^2.
    Returns the estimate as unknowns/s, with the sample's own wall time.
    """
    import oracle
    if wl.get("formulation") == "MULLER":
        return None  # the row sampler of the oracle covers the MFIE system
    if wl.get("independent"):
        return None  # a batch of uncoupled bodies: the oracle holds one coupled system
    t0 = time.perf_counter()
    o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], wl["k"])
    N = o.N
    R = 32
    rows = np.linspace(0, N - 1, R).astype(np.int64)
    ns = min(N, 3072)
    key = (workload_name, ns)
    if key not in _LU_SAMPLE:
        idx = np.sort(np.random.default_rng(0).choice(N, ns, replace=False))
        _LU_SAMPLE[key] = o.matrix_rows(idx)[:, idx]  # a principal submatrix of the same operator
    t_setup = time.perf_counter() - t0
    t1 = time.perf_counter()
    t = time.perf_counter()
    o.matrix_rows(rows)
    t_rows = time.perf_counter() - t
    t = time.perf_counter()
    LU, piv, info = oracle.zgetrf(_LU_SAMPLE[key])
    t_lu = time.perf_counter() - t
    nrhs = wl["kdirs"].shape[0]
    b = np.ones((ns, nrhs), dtype=complex)
    t = time.perf_counter()
    oracle.zgetrs(LU, piv, b)
    t_sol = time.perf_counter() - t
    step_s = time.perf_counter() - t1
    est = t_rows * N / R + t_lu * (N / ns) ** 3 + t_sol * (N / ns) ** 2
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": N / est, "unit": "unknowns/s", "cores": cores, "kind": "oracle",
            "sample": "ESTIMATE from a bounded sample: dense fill of %d of %d rows (%.2f s) + oracle LU of a "
                      "%d x %d principal submatrix (%.2f s, out of cache) + %d solves (%.3f s); scaled by N/R, "
                      "(N/n)^3, (N/n)^2 to an estimated full dense fill+LU+solve of %.0f s"
                      % (R, N, t_rows, ns, ns, t_lu, nrhs, t_sol, est),
            "step_s": step_s, "setup_s": t_setup, "est_full_s": est}


def full_oracle(wl):
    """The oracle's full dense fill, LU and solve of the workload, each timed (a measurement,
    minutes at 19,200 unknowns; run on its own with --impl reference --full-oracle)."""
    import oracle
    o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], wl["k"])
    b = o.rhs(wl["kdirs"], wl["pols"])
    t = time.perf_counter()
    A = o.dense()
    t_fill = time.perf_counter() - t
    t = time.perf_counter()
    LU, piv, info = oracle.zgetrf(A)
    t_lu = time.perf_counter() - t
    del A
    t = time.perf_counter()
    oracle.zgetrs(LU, piv, b.T)
    t_sol = time.perf_counter() - t
    tot = t_fill + t_lu + t_sol
    return {"unknowns": o.N, "fill_s": t_fill, "lu_s": t_lu, "solve_s": t_sol, "total_s": tot,
            "value": o.N / tot, "unit": "unknowns/s", "nproc": os.cpu_count(),
            "omp_num_threads": os.environ.get("OMP_NUM_THREADS")}


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = load_workload(args.workload)
    if args.full_oracle:
        print(json.dumps(dict(full_oracle(wl), workload=args.workload, impl="reference", kind="oracle-full")),
              flush=True)
        return
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(wl, args.workload)
        if i >= args.warmup:
            vals.append(cb)
    v = statistics.median([c["value"] for c in vals])
    step_ms = 1000.0 * statistics.median([c["step_s"] for c in vals])
    cb = dict(vals[-1])
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "unknowns/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
           "ms_per_step_is": "wall time of one bounded sample step; value is the full-size estimate",
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(args, wl), "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def bench_config(args, wl):
    """The workload description both arms print (identical keys and values)."""
    return {"workload": args.workload, "formulation": wl.get("formulation", "MFIE"), "unknowns": wl_N(wl),
            "bodies": len(wl["ms"]), "independent_bodies": bool(wl.get("independent", False)),
            "rhs": int(wl["kdirs"].shape[0]),
            "leaf": wl["leaf"], "eta": wl["eta"], "aca_tol": wl["aca_tol"],
            "l2": "working set (H-matrix, near store) > L2 between steps"}


def wl_N(wl):
    dof = 4 if wl.get("formulation") == "MULLER" else 2
    return dof * 6 * int(np.sum(np.asarray(wl["ms"]) ** 2)) * wl["nc"] ** 2


def formulation_args(wl):
    """hm_build_geometry keywords of the workload's integral equation."""
    from paper_2408_17116_gb300 import hm
    if wl.get("formulation") == "MULLER":
        return dict(formulation=hm.HM_DIEL_MULLER, eps_r=wl["eps_r"])
    if wl.get("independent"):
        return dict(independent=True)
    return {}


PRECISION = {"fp32r": 1, "fp64": 0}


def solution_error(name, x):
    """max over right-hand sides of |x - x_o| / |x_o| against the dense oracle's solution
    stored in tests/golden (written by tests/golden/make_dense_solution.py), or None."""
    path = os.path.join(ROOT, "tests", "golden", name + "_x.npy")
    if not os.path.exists(path):
        return None
    xo = np.load(path)
    xs = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    if xs.shape != xo.shape:
        return None
    return float(max(np.linalg.norm(xs[r] - xo[r]) / np.linalg.norm(xo[r]) for r in range(xo.shape[0])))


def aggregate(ms_local, unknowns_local, dist=None, device="cpu"):
    """Whole-job throughput of replicas: the slowest rank's time per step (max over ranks)
    and the unknowns all ranks solved per second.  Returns (ms_max, unknowns_per_s)."""
    import torch
    world = dist.get_world_size() if dist is not None else 1
    t = torch.tensor([float(ms_local), float(unknowns_local)], dtype=torch.float64, device=device)
    if dist is not None:
        tm = t[:1].clone()
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        tn = t[1:].clone()
        dist.all_reduce(tn, op=dist.ReduceOp.SUM)
        t = torch.cat([tm, tn])
    ms = float(t[0].item())
    return ms, float(t[1].item()) / (ms / 1000.0) if world else 0.0


def one_step(s, wl, dirs, host=False, precision="fp32r", factor_leaf=0):
    s.hm_build_geometry(wl["bodies"], wl["ms"], wl["nc"], wl["k"], wl["leaf"], wl["eta"], wl["aca_tol"],
                        precision=PRECISION[precision], factor_leaf=factor_leaf, **formulation_args(wl))
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


def train_rank_model(s):
    """Train the learned ACA-rank predictor on the ranks plain ACA reaches on four bodies
    other than the bench workload (spheres and ellipsoids of 3.5-5 wavelengths, 4,800
    unknowns each) and install it on the solver s (its fills then skip the attempts it
    predicts to fail and size ACA buffers by its prediction; plain adaptive ACA re-runs any
    under-predicted block)."""
    import torch
    from paper_2408_17116_gb300 import hm, workloads
    t0 = time.perf_counter()
    base = dict(load_workload("sphere_d8_m4_nc10"), ms=[2], nc=10)
    bodies = [workloads.body(semi=(1.75,) * 3), workloads.body(semi=(2.5, 2.0, 1.5)),
              workloads.body(semi=(2.25,) * 3), workloads.body(semi=(2.4, 1.6, 2.0))]
    feats, targs = [], []
    for bd in bodies:
        t = hm.Solver()
        t.hm_build_geometry(bd[None], base["ms"], base["nc"], base["k"], base["leaf"], base["eta"], base["aca_tol"])
        t.hm_fill()
        f, y = t.rank_samples()
        feats.append(f)
        targs.append(y)
        t.close()
    X, y = np.concatenate(feats), np.concatenate(targs)
    m = hm.MLP(hm.RANK_NFEAT, 32)
    m.set_params(workloads.mlp_init(hm.RANK_NFEAT, 32))
    loss = m.train(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"), 2000, 3e-3)
    s.set_rank_model(m)
    return {"trained_on": "4 bodies of 4,800 unknowns (spheres D = 3.5 and 4.5, ellipsoids)", "samples": int(len(y)),
            "loss": loss, "r2": float(1.0 - loss / np.var(y)), "setup_s": time.perf_counter() - t0}


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
    ap.add_argument("--no-compare", action="store_true", help="skip the one-step runs of both precisions")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the host-buffer end-to-end step (for kernel launch lists under a profiler)")
    ap.add_argument("--full-oracle", action="store_true",
                    help="with --impl reference: time the oracle's full dense fill, LU and solve once")
    ap.add_argument("--no-rank-model", action="store_true",
                    help="plain adaptive ACA: do not train and use the learned ACA-rank predictor (by default "
                         "it is trained before the warm-up on four other bodies of 4,800 unknowns, not the "
                         "bench workload, and every fill of the run uses it)")
    ap.add_argument("--compare-workload", default=None,
                    help="workload of the FP32-refined vs plain-FP64 comparison, one step each "
                         "(default: the bench workload)")
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

    def progress(msg):
        if rank == 0:
            print("[bench] %s" % msg, file=sys.stderr, flush=True)

    rank_info = None
    if not args.no_rank_model:
        rank_info = train_rank_model(s)
        progress("rank model: %s" % json.dumps(rank_info))
    for i in range(args.warmup):
        t = time.perf_counter()
        one_step(s, wl, dirs, precision=prec)
        progress("warm-up %d: %.1f s (factor %.1f s, solve %.1f s, %d refinement steps)" % (
            i, time.perf_counter() - t, s.hm_query("T_FACTOR"), s.hm_query("T_SOLVE"), s.hm_query("REFINE_ITERS")))
    barrier()
    L0 = s.hm_query("LAUNCHES")
    clk = ClockSampler(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    phases = {k: 0.0 for k in ("T_GEOMETRY", "T_NEAR", "T_ACA", "T_RECOMPRESS", "T_DENSE", "T_FACTOR", "T_SOLVE")}
    near_pts = 0.0
    kern = {k: 0.0 for k in ("KQR_SECONDS", "KQR_FLOPS", "KQR_LAUNCHES", "KCORE_SECONDS", "KCORE_FLOPS",
                             "KCORE_LAUNCHES", "KGEMM_SECONDS", "KGEMM_FLOPS", "KGEMM_LAUNCHES", "KTC_SECONDS",
                             "KTC_FLOPS", "KTC_LAUNCHES")}
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        x, rcs = one_step(s, wl, dirs, precision=prec)
        for k in phases:
            phases[k] += s.hm_query(k)
        near_pts += s.hm_query("NEAR_QPOINTS")
        for k in kern:  # counters of the last reset: hm_factor's recompressions
            kern[k] += s.hm_query(k)
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    progress("timed: %.1f ms per step" % ms)
    launches = int(s.hm_query("LAUNCHES") - L0)
    N = s.N
    sol_err = solution_error(args.workload, x)
    ms, value = aggregate(ms, N, dist, device="cuda")
    stats = {k.lower(): s.hm_query(k) for k in ("CR", "MAX_RANK", "MEAN_RANK", "LR_BLOCKS", "DENSE_BLOCKS",
                                                 "NEAR_PAIRS", "ACA_NONCONV", "FLOPS_FACTOR", "REFINE_ITERS",
                                                 "REFINE_RES", "STORAGE", "STORAGE32", "DENSE_LEVEL",
                                                 "TRUNC_BATCHES", "TRUNC_JOBS", "TRUNC_MAXK", "T_LU_PANEL",
                                                 "T_LU_U12", "T_TILE_BUILD", "T_SOLVE_SWEEP", "T_SOLVE_MATVEC")}
    # e2e: host buffers in and out, wall clock around the public API calls
    e2e_s = None
    if not args.no_e2e:
        barrier()
        t = time.perf_counter()
        xh, rcs_h = one_step(s, wl, dirs, host=True, precision=prec)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t
        progress("e2e: %.1f s" % e2e_s)
    nrhs = wl["kdirs"].shape[0]
    h2d = 152 * len(wl["ms"]) + 64 + 48 * nrhs + 24 * dirs.shape[0]  # bodies, params, waves, directions
    d2h = 16 * N * nrhs + 8 * nrhs * dirs.shape[0]
    # rooflines of the kernels timed live with CUDA events (per launch: algorithmic flops of
    # one launch / its average device time); the one with the most device time per step is
    # reported as "roofline", the others under "kernels"
    per = {k: v / args.steps for k, v in phases.items()}
    near_flops = (near_pts / args.steps) * NEAR_FLOPS_PER_POINT(wl["nc"])
    cands = []
    if per["T_NEAR"] > 0:
        a = near_flops / per["T_NEAR"] / 1e12
        npairs = s.hm_query("NEAR_PAIRS")
        cands.append({"kernel": "k_near (self/near CBIE quadrature, FP64)", "bound": "alu", "achieved": a,
                      "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": a / FP64_PEAK_TFLOPS,
                      "traffic": NEAR_DRAM_BYTES_PER_PAIR * npairs if wl.get("formulation") != "MULLER" else None,
                      "traffic_source": "ncu capture of the 4,800-unknown sphere (192 near pairs), scaled by near pairs",
                      "launches_per_step": 1, "seconds_per_step": per["T_NEAR"],
                      "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz"})
    fp32 = prec == "fp32r"
    pk = FP32_PEAK_TFLOPS if fp32 else FP64_PEAK_TFLOPS
    src = ("derived: 152 SMs x 128 FP32 FMA/clk x 2 flops x 2.07 GHz" if fp32
           else "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz")
    if kern["KQR_SECONDS"] > 0:
        a = kern["KQR_FLOPS"] / kern["KQR_SECONDS"] / 1e12
        cands.append({"kernel": "k_qr<%s> (Householder QR of low-rank factors in the H-LU recompression)"
                      % ("float2" if fp32 else "double2"), "bound": "alu", "achieved": a, "peak": pk,
                      "unit": "TFLOP/s", "frac": a / pk, "traffic": None,
                      "launches_per_step": kern["KQR_LAUNCHES"] / args.steps,
                      "seconds_per_step": kern["KQR_SECONDS"] / args.steps, "peak_source": src})
    if kern["KCORE_SECONDS"] > 0 and kern["KCORE_FLOPS"] > 0:
        a = kern["KCORE_FLOPS"] / kern["KCORE_SECONDS"] / 1e12
        cands.append({"kernel": "k_qrcp<float2> (pivoted QR of the recompression core)", "bound": "alu",
                      "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk, "traffic": None,
                      "launches_per_step": kern["KCORE_LAUNCHES"] / args.steps,
                      "seconds_per_step": kern["KCORE_SECONDS"] / args.steps, "peak_source": src})
    if kern["KGEMM_SECONDS"] > 0:
        a = kern["KGEMM_FLOPS"] / kern["KGEMM_SECONDS"] / 1e12
        cands.append({"kernel": "k_zgemm<%s> (dense Schur-complement products of the H-LU, >= 1e9 flops each)"
                      % ("float2" if fp32 else "double2"), "bound": "alu", "achieved": a, "peak": pk,
                      "unit": "TFLOP/s", "frac": a / pk, "traffic": None,
                      "launches_per_step": kern["KGEMM_LAUNCHES"] / args.steps,
                      "seconds_per_step": kern["KGEMM_SECONDS"] / args.steps, "peak_source": src})
    if kern["KTC_SECONDS"] > 0:
        # BF16 tensor flops of the split products (3 x 8 m n k per complex64 product) against
        # the measured sustained BF16 rate (the kernel runs inside a seconds-long step)
        tpk, tsrc = tensor_peak()
        a = kern["KTC_FLOPS"] / kern["KTC_SECONDS"] / 1e12
        cands.append({"kernel": "k_tc_gemm (tcgen05 + TMA complex64 products of the H-LU, split-BF16, "
                                ">= 1e9 tensor flops each)", "bound": "tensor", "achieved": a, "peak": tpk,
                      "unit": "TFLOP/s", "frac": a / tpk, "traffic": None,
                      "launches_per_step": kern["KTC_LAUNCHES"] / args.steps,
                      "seconds_per_step": kern["KTC_SECONDS"] / args.steps, "peak_source": tsrc})
    cands.sort(key=lambda c: -c["seconds_per_step"])
    roof = dict(cands[0]) if cands else None
    out = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64 fill; c64 H-LU + f64 refinement" if prec == "fp32r" else "f64",
           "data": "synthetic",
           "config": bench_config(args, wl), "precision": prec,
           "parallelism": "replicas" if world > 1 else "single",
           "solution_error_vs_oracle": sol_err,
           "phases_s": per, "stats": stats, "gpu_launches": launches, "clocks": clocks,
           "e2e": ({"value": N / e2e_s, "unit": "unknowns/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "wall_s": e2e_s} if e2e_s else None),
           "roofline": roof, "kernels": cands[1:]}
    if rank_info is not None:
        out["rank_model"] = dict(rank_info, aca_skipped=s.hm_query("ACA_SKIPPED"), aca_reruns=s.hm_query("ACA_RERUNS"))
    # the tensor-core variant autotuner: per packed depth 64 << c the chosen kernel (2 / 4 =
    # 2- / 4-stage ring, 1 = persistent) and the timed milliseconds of the three variants
    st, tms = hm.tc_tuning()
    out["tc_tuning"] = {str(64 << c): {"variant": int(st[c]), "ms_2stage_4stage_persistent": [round(float(x), 4)
                                                                                                for x in tms[c]]}
                        for c in range(8) if st[c]}
    if not args.no_compare:
        # FP32 H-LU + FP64 refinement against the plain FP64 H-LU on the same GPU, one timed
        # step each, with each solution's error against the stored dense-oracle solution
        cname = args.compare_workload or args.workload
        cwl = load_workload(cname)
        cmp = {"workload": cname}
        for p in ("fp32r", "fp64"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            e0.record(stream)
            cx, _ = one_step(s, cwl, dirs, precision=p)
            e1.record(stream)
            barrier()
            cms = e0.elapsed_time(e1)
            cmp[p] = {"value": s.N / (cms / 1000.0), "unit": "unknowns/s", "ms_per_step": cms, "unknowns": s.N,
                      "phases_s": {k: s.hm_query(k) for k in phases}, "refine_iters": s.hm_query("REFINE_ITERS"),
                      "refine_res": s.hm_query("REFINE_RES"), "dense_level": s.hm_query("DENSE_LEVEL"),
                      "solution_error_vs_oracle": solution_error(cname, cx)}
        cmp["fp32r_speedup"] = cmp["fp64"]["ms_per_step"] / cmp["fp32r"]["ms_per_step"]
        # the same FP32 path with the formatted H-LU above dense blocks of at most 2,400
        # unknowns (low-rank blocks, recompressions) instead of the adaptive dense level
        try:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            e0.record(stream)
            cx, _ = one_step(s, cwl, dirs, precision="fp32r", factor_leaf=2400)
            e1.record(stream)
            barrier()
            cms = e0.elapsed_time(e1)
            cmp["fp32r_hlu_2400"] = {"value": s.N / (cms / 1000.0), "unit": "unknowns/s", "ms_per_step": cms,
                                     "phases_s": {k: s.hm_query(k) for k in phases},
                                     "dense_level": s.hm_query("DENSE_LEVEL"), "lr_blocks": s.hm_query("LR_BLOCKS"),
                                     "solution_error_vs_oracle": solution_error(cname, cx)}
        except Exception as exc:  # reported, not fatal: the headline line stays valid
            cmp["fp32r_hlu_2400"] = {"error": repr(exc)[:200]}
        out["compare"] = cmp
        progress("compare: %s" % json.dumps(cmp))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, args.workload)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
