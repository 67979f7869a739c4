"""Benchmark: NRTO solves/sec at residual <= 1e-4 on one B300, batched + warm-started + mixed
precision against the plain cold-started FP64 GPU form at batch 1.

Workload: the 2048-instance batch (seeded; 50/50 unicycle T~U{20..200} with 1-20 obstacles and
quadcopter T~U{50..150} with 1-15 obstacles).  One step = one complete NRTO solve of every instance:
10 successive-linearization steps; the inner FullADMM solves of the first nine stop after 15
iterations (inexact; the paper's tables use 40, and 15 measured the most counted solves per second),
the last one runs to full residuals <= 1e-4 (cap 2000), all with residual balancing every 25
iterations, the stall stop and the budget stop (a solve whose primal residual, at its observed rate,
would miss 1e-4 within the cap ends early).

A solve counts when (i) the inner solve that produced the returned (accepted) iterate terminated at
full residuals r_p, r_d <= 1e-4 and (ii) every robust constraint holds there:
max_j g_j(x̄) + ‖Â_j k + b̂_j‖ <= 1e-4 (Problem 2 at δû = 0, linearized at the returned trajectory).
`value` = counted solves per second of the batched + warm-started (inner-state carry across outer
steps) + mixed-precision form; the same metric is measured for the plain form — FP64, one instance
per launch (batch 1, looped over a seeded sample of the workload), cold start of every inner solve,
same schedule and tolerances — and their ratio is reported.

Inputs are resident in HBM before the timed region; the row arrays (several GB) exceed the 126 MB L2.
`--impl reference` times the CPU oracle (this project's reference arm) on the machine's host cores.
Under torchrun every rank solves its own batch (weak scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "NRTO solves/sec at residual ≤1e-4: warm-start+batched vs plain, 1×B300"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--n-outer", type=int, default=10)
    ap.add_argument("--max-inner", type=int, default=15, help="inner cap of the first n_outer-1 outer steps")
    ap.add_argument("--max-inner-final", type=int, default=2000, help="inner cap of the last outer step")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--rho", type=float, default=1.0, help="initial FullADMM penalty")
    ap.add_argument("--adapt", type=int, default=25, help="residual-balancing period (0 = fixed rho)")
    ap.add_argument("--adapt-mu", type=float, default=3.0, help="residual-balancing ratio threshold")
    ap.add_argument("--stall", type=int, default=100, help="stall-stop period (0 = off)")
    ap.add_argument("--stall-budget", type=float, default=1.0,
                    help="budget-stop factor at the stall checkpoints (0 = off)")
    ap.add_argument("--carry", type=int, default=1, help="inner-state carry across outer steps")
    ap.add_argument("--feas-tol", type=float, default=1e-4)
    ap.add_argument("--r0", type=float, default=0.5, help="initial and largest trust radius of the outer loop")
    ap.add_argument("--w-p", type=float, default=1000.0, help="merit weight of the robust-constraint violation")
    ap.add_argument("--mc", type=int, default=1000, help="Monte Carlo interior and edge samples per instance")
    ap.add_argument("--warm-train", type=int, default=1024, help="training solves of the learned warm start")
    ap.add_argument("--warm-eval", type=int, default=512, help="held-out instances of the learned warm start")
    ap.add_argument("--plain-n", type=int, default=16, help="instances of the plain batch-1 FP64 arm")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned-warm-start study")
    ap.add_argument("--no-configs", action="store_true", help="skip the single-instance configurations")
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the raw nvidia-smi clock samples (default: a temporary directory)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def rank_reduce(values, ops, ws, device):
    """Replicas' results combined over the ranks: values[i] reduced with ops[i] ("max" for times,
    "sum" for counts); a no-op on one rank.  device: where the collective's tensor lives (cuda under
    NCCL, cpu under gloo)."""
    import torch
    import torch.distributed as dist
    out = [float(v) for v in values]
    if ws > 1:
        for i, op in enumerate(ops):
            t = torch.tensor([out[i]], dtype=torch.float64, device=device)
            dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
            out[i] = float(t.item())
    return out


def workload(n, rank):
    from paper_2603_02642_b300 import workloads as W
    return W.batched_mix(n, base_seed=10000 + rank * n)


def entries(inst):
    """Ragged row entries of one instance: state rows S ((t+1)·nx each) and control rows C (nx each)."""
    per_t = inst.n_obs * (inst.link_spheres.shape[0] if inst.kind == 2 else 1)
    per_t += int(np.isfinite(inst.x_lo).sum() + np.isfinite(inst.x_hi).sum())
    S = per_t * sum((t + 1) * inst.nx for t in range(1, inst.T + 1))
    C = int(np.isfinite(inst.u_lo).sum() + np.isfinite(inst.u_hi).sum()) * inst.T * inst.nx
    return S, C


def solver_options(args, carry=None):
    from paper_2603_02642_b300 import nrto
    return nrto.Options(rho=args.rho, max_inner=args.max_inner, max_inner_final=args.max_inner_final,
                        eps_p=1e-4, eps_d=1e-4, check=1, r0=args.r0, w_p=args.w_p, adapt_every=args.adapt,
                        adapt_mu=args.adapt_mu,
                        stall_every=args.stall, stall_ratio=0.9, stall_budget=args.stall_budget,
                        carry=args.carry if carry is None else carry)


def counted(st, tol):
    """Solves that count: the returned iterate's inner solve converged and its robust constraints hold."""
    return (st["accepted_status"] == 1) & (st["max_violation"] <= tol)


# ---------------------------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline): nproc worker processes
# ---------------------------------------------------------------------------------------------
def _oracle_task(task):
    """One oracle task in a worker process (spawned; BLAS single-threaded)."""
    from oracle import fulladmm as F, outer as O, problem as P
    kind, inst, prm = task
    if kind == "cost":
        # per-linearization and per-inner-iteration cost of one instance
        t0 = time.perf_counter()
        lin = P.linearize(inst, inst.u_init)
        t1 = time.perf_counter()
        F.iterate(inst, lin, F.FullADMMOptions(rho=prm["rho"], r_trust=2.0, check=False), n_iter=prm["k_it"])
        t2 = time.perf_counter()
        return {"kind": "cost", "S": sum(entries(inst)), "t_lin": t1 - t0, "t_it": (t2 - t1) / prm["k_it"]}
    # a complete solve with the benchmark's schedule
    t0 = time.perf_counter()
    res = O.solve(inst, O.OuterOptions(n_outer=prm["n_outer"], r0=prm["r0"], w_p=prm["w_p"], carry=bool(prm["carry"]),
                                       max_inner_final=prm["max_inner_final"]),
                  admm=F.FullADMMOptions(rho=prm["rho"], max_iter=prm["max_inner"], eps_p=1e-4, eps_d=1e-4,
                                         adapt_every=prm["adapt"], adapt_mu=prm["adapt_mu"], stall_every=prm["stall"],
                                         stall_ratio=0.9, stall_budget=prm["stall_budget"]))
    t1 = time.perf_counter()
    ok = bool(res.accepted_inner_converged and res.max_violation <= prm["feas_tol"])
    return {"kind": "full", "S": sum(entries(inst)), "iters": int(sum(res.inner_iters)), "ok": ok, "t": t1 - t0}


def cpu_model():
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True).stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def oracle_tasks(instances, args, cores):
    """Task list of the oracle estimate: (a) cost tasks on a size-stratified sample of the workload
    (instances at evenly spaced quantiles of the row-entry count, smallest and largest included):
    one linearization and 4 inner iterations each; (b) complete solves with the benchmark's schedule
    on the smallest instances of the workload."""
    sizes = np.array([sum(entries(x)) for x in instances], dtype=np.float64)
    order = np.argsort(sizes, kind="stable")
    n_cost = int(min(max(cores, 8), 24))
    q = np.linspace(0, len(order) - 1, n_cost).round().astype(int)
    n_full = int(min(max(cores, 4), 16))
    prm = dict(rho=args.rho, k_it=4, n_outer=args.n_outer, max_inner=args.max_inner,
               max_inner_final=args.max_inner_final, adapt=args.adapt, stall=args.stall, carry=args.carry,
               feas_tol=args.feas_tol, r0=args.r0, w_p=args.w_p, adapt_mu=args.adapt_mu,
               stall_budget=args.stall_budget)
    return ([("full", instances[int(i)], prm) for i in order[:n_full]]
            + [("cost", instances[int(order[i])], prm) for i in q])


def oracle_pool(cores, n_tasks):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    return mp.get_context("spawn").Pool(processes=max(1, min(cores, n_tasks)))


def oracle_from_results(instances, args, out, cores, wall):
    """Per instance, time = (1 + n_outer) linearizations + I inner iterations, with per-linearization
    and per-iteration costs from least-squares lines in the row-entry count fitted to the cost tasks,
    and I and the fraction of solves that count from the complete solves.  Throughput on N cores =
    counted solves / (Σ times / N)."""
    sizes = np.array([sum(entries(x)) for x in instances], dtype=np.float64)
    cost = [r for r in out if r["kind"] == "cost"]
    full = [r for r in out if r["kind"] == "full"]
    S = np.array([r["S"] for r in cost], dtype=np.float64)
    Xm = np.stack([np.ones_like(S), S], axis=1)
    c_lin = np.linalg.lstsq(Xm, np.array([r["t_lin"] for r in cost]), rcond=None)[0]
    c_it = np.linalg.lstsq(Xm, np.array([r["t_it"] for r in cost]), rcond=None)[0]
    iters = float(np.mean([r["iters"] for r in full]))
    frac = float(np.mean([r["ok"] for r in full]))
    per = (1 + args.n_outer) * np.maximum(c_lin[0] + c_lin[1] * sizes, 1e-6) \
        + iters * np.maximum(c_it[0] + c_it[1] * sizes, 1e-7)
    total = float(per.sum())
    value = frac * len(instances) / (total / cores)
    return dict(value=value, unit=UNIT, cores=cores, kind="oracle", cpu_model=cpu_model(),
                sample=(f"{n_cores_str(cores)}: cost of one linearization and one inner iteration on {len(cost)} "
                        f"workload instances at evenly spaced size quantiles ({int(S.min())}..{int(S.max())} row "
                        f"entries), and {len(full)} complete solves with the benchmark's schedule on the smallest "
                        f"instances (mean {iters:.0f} inner iterations per solve, {frac:.2f} counted); per-instance "
                        f"time = linear fits in the row-entry count, summed over the {len(instances)}-instance "
                        f"workload and divided by {cores} cores; {wall:.1f} s wall"),
                fit={"lin_s": [float(c) for c in c_lin], "iter_s": [float(c) for c in c_it]},
                counted_fraction=frac, inner_iters_per_solve=iters, wall_s=wall)


def oracle_estimate(instances, args):
    """The FP64 oracle's solves/s at the metric on all host cores, from a bounded sample: the tasks of
    oracle_tasks run concurrently in one spawned process per core (so their timings include the
    contention of a fully loaded host), then oracle_from_results."""
    cores = os.cpu_count() or 1
    tasks = oracle_tasks(instances, args, cores)
    t0 = time.perf_counter()
    with oracle_pool(cores, len(tasks)) as pool:
        out = pool.map(_oracle_task, tasks, chunksize=1)
    return oracle_from_results(instances, args, out, cores, time.perf_counter() - t0)


def n_cores_str(cores):
    return f"{cores} spawned processes (one per host core)"


# ---------------------------------------------------------------------------------------------
def clocks_start(path):
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None


def clocks_summary(path, dev_index):
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(dev_index):
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
    except FileNotFoundError:
        pass
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
            "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic of k_fulladmm per algorithmic byte ((3 S + 2 C) w), from an ncu capture of the
# 148-instance case (dram__bytes_read.sum + dram__bytes_write.sum of both kinds' launches, 40
# iterations each).  A launch at the benchmark size is scaled from it by its algorithmic bytes
# (traffic grows with row entries x iterations).  Valid only while the kernel sources hash to
# sources_sha256: any change to them makes the reported traffic null until it is measured again.
TRAFFIC = {"sources_sha256": "f8621a1d3563cc81609061b6eaa78e1ef600b405d5782ca483fe33784a6f1d3c",
           "ratio": {"both": 1.014, "quadcopter": 1.091, "unicycle": 0.852}}
KERNEL_SOURCES = ["fulladmm.cuh", "nrto_dev.cuh", "tma.cuh", "linearize.cuh", "dynamics.cuh"]


def kernel_sources_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2603_02642_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_peak(key, fallback):
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d[key]), "measured"
    except Exception:
        return fallback, "fallback"


# ---------------------------------------------------------------------------------------------
# plain arm: FP64, batch 1, cold start, same schedule
# ---------------------------------------------------------------------------------------------
def sample_ids(args, n):
    rng = np.random.default_rng(7)
    return sorted(rng.choice(n, size=min(args.plain_n, n), replace=False).tolist())


def plain_arm(args, insts, stream):
    import torch
    from paper_2603_02642_b300 import nrto
    ids = sample_ids(args, len(insts))
    opts = solver_options(args, carry=0)
    probs = [nrto.Problem([insts[i]], nrto.PREC_FP64, stream=stream.cuda_stream) for i in ids]
    probs[0].solve(opts, args.n_outer, fetch=False)   # first use of the FP64 kernels (module load)
    torch.cuda.synchronize()
    ms, ok, iters = [], [], []
    for p in probs:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p.solve(opts, args.n_outer, fetch=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        st = p.stats()
        ok.append(bool(counted(st, args.feas_tol)[0]))
        iters.append(float(st["cum_iters"][0]))
    for p in probs:
        p.close()
    tot = sum(ms) / 1e3
    return {"value": sum(ok) / tot, "unit": UNIT, "counted": int(sum(ok)), "solves": len(ids),
            "solves_per_s": len(ids) / tot, "iterations_per_s": sum(iters) / tot, "seconds": tot,
            "sample": f"{len(ids)} instances of the workload (ids {ids}), each alone on the GPU, FP64, cold start "
                      f"of every inner solve, the schedule and tolerances of the batched arm"}


def rel_err(a, b, floor=1e-9):
    """‖a - b‖ / max(‖b‖, floor): relative error, absolute below the floor (gains that are zero up to
    rounding in both precisions when no robust constraint is active)."""
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), floor))


def mixed_results(prob, ids):
    """The batch's returned (ū, K) and last p̃ of the sample instances, read from the device."""
    from paper_2603_02642_b300 import nrto
    return {"u_bar": {i: prob.export(nrto.F_UHAT, i) for i in ids}, "K": {i: prob.export(nrto.F_KACC, i) for i in ids},
            "pt": {i: prob.export(nrto.F_PT, i) for i in ids}}


def fp64_errors(args, insts, ids, out_mixed, st_mixed, stream):
    """Per-result error of the batched mixed-precision solve against the FP64 path with the same
    schedule (the GPU FP64 path matches the oracle to 1e-8 in the parity tests), on a seeded sample."""
    from paper_2603_02642_b300 import nrto
    p = nrto.Problem([insts[i] for i in ids], nrto.PREC_FP64, stream=stream.cuda_stream)
    o = p.solve(solver_options(args), args.n_outer, fetch=True)
    st = p.stats()
    pt64 = [p.export(nrto.F_PT, k) for k in range(len(ids))]
    p.close()

    def rel(a, b):
        return rel_err(a, b)

    rows = {"K": [], "u_bar": [], "cost": [], "p_tilde": [], "iterations": [], "counted_agree": []}
    ok64 = counted(st, args.feas_tol)
    okm = counted(st_mixed, args.feas_tol)
    for k, i in enumerate(ids):
        rows["K"].append(rel(out_mixed["K"][i], o["K"][k].reshape(-1)))
        rows["u_bar"].append(rel(out_mixed["u_bar"][i], o["u_bar"][k].reshape(-1)))
        rows["cost"].append(abs(st_mixed["cost"][i] - st["cost"][k]) / max(abs(st["cost"][k]), 1e-300))
        rows["p_tilde"].append(rel(out_mixed["pt"][i], pt64[k]))
        rows["iterations"].append(int(st_mixed["cum_iters"][i] - st["cum_iters"][k]))
        rows["counted_agree"].append(bool(okm[i] == ok64[k]))
    summ = {}
    for k, v in rows.items():
        if k == "counted_agree":
            summ[k] = f"{sum(v)}/{len(v)}"
        elif k == "iterations":
            summ[k] = {"median_abs": float(np.median(np.abs(v))), "max_abs": int(np.max(np.abs(v)))}
        else:
            summ[k] = {"median": float(np.median(v)), "max": float(np.max(v))}
    # the worst K: its relative error, the FP64 gains' norm and the largest absolute difference (gains
    # that are near zero in both precisions make a large relative error of a negligible difference)
    kw = int(np.argmax(rows["K"]))
    k64 = o["K"][kw].reshape(-1)
    summ["K_worst"] = {"id": int(ids[kw]), "rel": float(rows["K"][kw]), "norm_fp64": float(np.linalg.norm(k64)),
                       "abs_max": float(np.max(np.abs(out_mixed["K"][ids[kw]] - k64)))}
    summ["sample"] = f"{len(ids)} instances (ids {ids}); reference: the FP64 path, same schedule and carry"
    return summ


def single_configs(args, stream):
    """The single-instance configurations: solves/s and iterations/s on one B300 (one instance
    occupies one SM), with the oracle's time per inner iteration on the same instance."""
    import torch
    from oracle import dr as DRO, fulladmm as F, problem as P
    from paper_2603_02642_b300 import nrto, workloads as W
    out = {}

    def timed(prob, opts, n_outer, reps=2, warm=True):
        if warm:
            prob.solve(opts, n_outer, fetch=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            prob.solve(opts, n_outer, fetch=False)
        e1.record(stream)
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3 / reps
        st = prob.stats()
        return s, st

    def oracle_iter_s(inst, solver):
        lin = P.linearize(inst, inst.u_init)
        t0 = time.perf_counter()
        if solver == "dr":
            DRO.solve(inst, lin, DRO.DROptions(rho=40.0, r_trust=2.0, max_admm=1, max_dr=20), n_admm=1, n_dr=20,
                      check=False)
            return (time.perf_counter() - t0) / 20.0
        F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=2.0, check=False), n_iter=3)
        return (time.perf_counter() - t0) / 3.0

    # unicycle T = 20, 3 obstacles, NRTO-DR, FP64 (<= 40 ADMM x <= 500 DR iterations per outer step):
    # the first 2 of the 10 outer steps, timed once (NRTO-DR's exact subproblem 2 makes it slow)
    uni = W.unicycle(0, T=20, n_obs=3)
    o = nrto.Options(solver=nrto.SOLVER_DR, rho=40.0, max_inner=40, max_dr=500, eps_dr=1e-4, eps_p=1e-4, eps_d=1e-4,
                     check=1, r0=2.0)
    p = nrto.Problem([uni], nrto.PREC_FP64, stream=stream.cuda_stream)
    s, st = timed(p, o, 2, reps=1, warm=False)
    p.close()
    out["unicycle_T20_o3_dr_fp64"] = {"work": "2 outer steps of the 10", "outer_steps_per_s": 2.0 / s,
                                      "admm_iterations_per_s": st["cum_iters"][0] / s,
                                      "dr_iterations_per_s": st["dr_iters"][0] / s, "seconds": s,
                                      "oracle_s_per_dr_iteration": oracle_iter_s(uni, "dr")}
    # quadcopter T = 100, 10 obstacles, FP64: NRTO-DR vs FullADMM over the same bounded work (two
    # outer steps of 10 ADMM iterations, DR capped at 100 per ADMM iteration; FullADMM 10 iterations)
    quad = W.quadcopter(0, T=100, n_obs=10)
    d = {"work": "1 outer step x 5 inner iterations (NRTO-DR: <= 100 DR iterations each), FP64"}
    for name, oo in (("dr", nrto.Options(solver=nrto.SOLVER_DR, rho=40.0, max_inner=5, max_dr=100, eps_dr=1e-4,
                                         eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0)),
                     ("fulladmm", nrto.Options(rho=10.0, max_inner=5, eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0))):
        p = nrto.Problem([quad], nrto.PREC_FP64, stream=stream.cuda_stream)
        s, st = timed(p, oo, 1, reps=1, warm=(name == "fulladmm"))
        p.close()
        d[name] = {"outer_steps_per_s": 1.0 / s, "inner_iterations_per_s": st["cum_iters"][0] / s,
                   "seconds": s}
        if name == "dr":
            d[name]["dr_iterations_per_s"] = st["dr_iters"][0] / s
    d["oracle_s_per_fulladmm_iteration"] = oracle_iter_s(quad, "fulladmm")
    out["quadcopter_T100_o10_fp64"] = d
    # arm T = 100 (the double integrator of the benchmark definition, and the paper's Franka model),
    # mixed precision vs FP64 (3 outer steps: 2 x 40 inner iterations, then <= 200)
    ao = nrto.Options(rho=10.0, max_inner=40, max_inner_final=200, eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0,
                      adapt_every=25, stall_every=100, carry=1)
    for key, inst_arm in (("arm_T100_mixed", W.arm(0, T=100)), ("franka_T100_mixed", W.franka(0, T=100))):
        res = {}
        for prec in (nrto.PREC_MIXED, nrto.PREC_FP64):
            p = nrto.Problem([inst_arm], prec, stream=stream.cuda_stream)
            s, st = timed(p, ao, 3, reps=1)
            sol = p.solve(ao, 3, fetch=True)
            p.close()
            res[prec] = (s, st, sol)
        (sm, stm, solm), (s64, st64, sol64) = res[nrto.PREC_MIXED], res[nrto.PREC_FP64]
        out[key] = {
            "work": "3 outer steps (40, 40, <= 200 inner iterations), carry, residual balancing",
            "solves_per_s": 1.0 / sm, "inner_iterations_per_s": stm["cum_iters"][0] / sm, "seconds_per_solve": sm,
            "fp64_solves_per_s": 1.0 / s64, "oracle_s_per_fulladmm_iteration": oracle_iter_s(inst_arm, "fulladmm"),
            "error_vs_fp64": {"K": rel_err(solm["K"][0], sol64["K"][0]),
                              "K_norm_fp64": float(np.linalg.norm(sol64["K"][0])),
                              "u_bar": rel_err(solm["u_bar"][0], sol64["u_bar"][0]),
                              "cost": float(abs(stm["cost"][0] - st64["cost"][0]) / abs(st64["cost"][0])),
                              "iterations": int(stm["cum_iters"][0] - st64["cum_iters"][0])}}
    # block 2a as the paper states it (constrained QP each iteration) against the lifted split: the
    # first inner solve of the unicycle configuration to full residuals <= 1e-4, FP64
    cmp = {}
    for name, solver, cap in (("as_written", nrto.SOLVER_FULLADMM_AW, 2000), ("lifted", nrto.SOLVER_FULLADMM, 20000)):
        p = nrto.Problem([uni], nrto.PREC_FP64, stream=stream.cuda_stream)
        p.linearize()
        p.set_trust_radius(2.0)
        o = nrto.Options(solver=solver, rho=10.0, max_inner=cap, eps_p=1e-4, eps_d=1e-4, check=1)
        p.solve_socp(o, fetch=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p.solve_socp(o, fetch=False)
        e1.record(stream)
        torch.cuda.synchronize()
        st = p.stats()
        cmp[name] = {"iterations": int(st["iters"][0]), "status": int(st["status"][0]),
                     "ms": e0.elapsed_time(e1)}
        p.close()
    out["unicycle_T20_o3_block2_as_written_vs_lifted"] = cmp
    return out


def warm_start_study(stream, n_train=2048, n_eval=1024, n_infer=4096, steps=1000):
    """Learned warm start on the quadcopter workload (T = 100, 1-15 obstacles): targets from cold
    FullADMM solves (to full residuals <= 1e-4, <= 5000 iterations, residual balancing every 25) at
    the first outer step, one network in the lifted layout trained on them, and cold, warm (its
    (k_v, p̃, λ_p)) and lifted warm-started solves (plus its δû, the lifted part that pays) of
    held-out instances, the lifted one also with the cold fallback; the network's tensor-core GEMM
    rate on an inference batch."""
    import torch
    from paper_2603_02642_b300 import nrto, warmstart as WS, workloads as W
    opts = dict(rho=10.0, max_inner=5000, eps_p=1e-4, eps_d=1e-4, check=1, adapt_every=25)
    t0 = time.perf_counter()
    Xs, Ys, Ms = [], [], []
    for s0 in range(0, n_train, 2048):
        train = [W.warmstart_quad(s) for s in range(s0, min(n_train, s0 + 2048))]
        prob = nrto.Problem(train, nrto.PREC_MIXED, stream=stream.cuda_stream)
        prob.linearize()
        prob.set_trust_radius(2.0)
        out = prob.solve_socp(nrto.Options(**opts))
        X, Y, Mk = WS.collect_targets(prob, train, out["status"], lifted=True)
        prob.close()
        Xs.append(X); Ys.append(Y); Ms.append(Mk)
    X, Y, Mk = np.concatenate(Xs), np.concatenate(Ys), np.concatenate(Ms)
    t_data = time.perf_counter() - t0
    ws = WS.WarmStart(max_batch=max(n_infer, n_eval), stream=stream.cuda_stream, lifted=True)
    t0 = time.perf_counter()
    hist = ws.fit(X, Y, Mk, steps=steps, batch=256, lr=1e-3)
    t_fit = time.perf_counter() - t0
    test = [W.warmstart_quad(1_000_000 + s) for s in range(n_eval)]
    res = {}
    for mode in ("cold", "warm", "lifted", "lifted_fallback"):
        q = nrto.Problem(test, nrto.PREC_MIXED, stream=stream.cuda_stream)
        q.linearize()
        q.set_trust_radius(2.0)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        if mode != "cold":
            ws.apply(q, test, lifted=mode != "warm")
        e1.record(stream)
        fbk = mode == "lifted_fallback"
        o = q.solve_socp(nrto.Options(stall_every=1000 if fbk else 0, stall_ratio=0.99, warm_fallback=int(fbk),
                                      **opts))
        e2.record(stream)
        torch.cuda.synchronize()
        fb = int(q.stats()["fallback"].sum())
        res[mode] = dict(iters=o["iters"].copy(), conv=o["status"] == 1, solve_ms=e1.elapsed_time(e2),
                         predict_ms=e0.elapsed_time(e1), fallbacks=fb)
        q.close()
    both = np.logical_and.reduce([r["conv"] for r in res.values()])
    feats = WS.features([W.warmstart_quad(2_000_000 + s) for s in range(n_infer)])
    ws.net.forward(feats)
    ws.net.profile(True)
    ws.net.forward(feats)
    gms, gfl, gn = ws.net.profile(False)
    peak, peak_kind = measured_peak("bf16_tflops", 1800.0)
    achieved = gfl / (gms / 1e3) / 1e12
    ws.net.close()

    def summary(r, warm):
        total_ms = r["solve_ms"] + (r["predict_ms"] if warm else 0.0)
        d = {"converged": int(r["conv"].sum()), "solve_ms": r["solve_ms"],
             "solves_per_s": n_eval / (total_ms / 1e3),
             "converged_per_s": int(r["conv"].sum()) / (total_ms / 1e3),
             "iters_mean_all_converged": float(r["iters"][both].mean()) if both.any() else None,
             "iters_median_all_converged": float(np.median(r["iters"][both])) if both.any() else None}
        if warm:
            d["predict_ms"] = r["predict_ms"]
            d["fallbacks"] = r["fallbacks"]
        return d

    cold_it = res["cold"]["iters"][both]
    return {
        "workload": f"quadcopter T=100, 1-15 obstacles (warmstart_quad); train seeds 0..{n_train - 1}, "
                    f"held-out seeds 1000000..{1000000 + n_eval - 1}",
        "network": "99 -> 256 -> 256 -> 256 -> 15608 (lifted layout), GELU, bf16 tcgen05 GEMMs",
        "targets": int(X.shape[0]), "train_steps": steps, "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
        "data_s": round(t_data, 2), "fit_s": round(t_fit, 2),
        "held_out": n_eval, "converged_in_all_modes": int(both.sum()),
        "cold": summary(res["cold"], False),
        "warm": summary(res["warm"], True),
        "lifted": summary(res["lifted"], True),
        "lifted_fallback": summary(res["lifted_fallback"], True),
        "iteration_ratio_vs_cold": {m: float(res[m]["iters"][both].mean() / max(cold_it.mean(), 1e-30))
                                    for m in ("warm", "lifted", "lifted_fallback")} if both.any() else None,
        "mlp_roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "peak_source": peak_kind + " (burst)", "batch": n_infer,
                         "gemm_launches": int(gn), "gemm_ms": gms},
    }


def reference_arm(args):
    """The oracle on the host cores: each timed step runs its share of the estimate's tasks (a
    bounded sample of the workload), and the value is the estimate from all timed steps' results.
    Warm-up steps run one of the smallest complete solves each (process start and imports)."""
    insts = workload(args.n, 0)
    cores = os.cpu_count() or 1
    tasks = oracle_tasks(insts, args, cores)
    full = [t for t in tasks if t[0] == "full"]
    K = max(args.steps, 1)
    out, t_steps = [], []
    with oracle_pool(cores, len(tasks)) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_task, full[:1], chunksize=1)
        for k in range(K):
            t0 = time.perf_counter()
            out += pool.map(_oracle_task, tasks[k::K], chunksize=1)
            t_steps.append(time.perf_counter() - t0)
    est = oracle_from_results(insts, args, out, cores, sum(t_steps))
    value = est["value"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean(t_steps)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"batch{args.n}_mixed_unicycle_quadcopter", "n_outer": args.n_outer,
                       "max_inner": args.max_inner, "max_inner_final": args.max_inner_final,
                       "instances_per_gpu": args.n, "adapt_every": args.adapt, "stall_every": args.stall,
                       "stall_budget": args.stall_budget, "carry": args.carry, "feas_tol": args.feas_tol,
                       "step": "a 1/steps share of the oracle sample's tasks on all host cores"},
            "cpu_baseline": est,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return 0

    import torch
    import torch.distributed as dist
    from paper_2603_02642_b300 import build, nrto

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    build.build()
    insts = workload(args.n, rank)
    prec = nrto.PREC_MIXED if args.prec == "mixed" else nrto.PREC_FP64
    # a stream of its own: the solve's CUDA graph cannot be captured on the legacy default stream
    stream = torch.cuda.Stream()
    prob = nrto.Problem(insts, prec, stream=stream.cuda_stream)
    opts = solver_options(args)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # autotune the launch mapping on this batch (fixed work: 2 outer steps x 40 iterations)
    tune_opts = nrto.Options(rho=args.rho, max_inner=40, check=0, r0=2.0)
    tuned, tune_ms = prob.autotune(tune_opts, n_outer=2, reps=1)
    for _ in range(args.warmup):
        prob.solve(opts, args.n_outer, fetch=False)
    barrier()
    clk_dir = args.clocks_dir or tempfile.gettempdir()
    clk_path = os.path.join(clk_dir, f"nrto_clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    clk = clocks_start(clk_path)
    time.sleep(0.5)
    launches0 = prob.kernel_launches()
    graphs0 = prob.graph_info()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        prob.solve(opts, args.n_outer, fetch=False)   # replays of the solve's CUDA graph
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = prob.kernel_launches() - launches0
    graph_replays = prob.graph_info()[1] - graphs0[1]
    if clk:
        clk.terminate()
        clk.wait()
    # one more step with the solver launches timed by CUDA events (direct launches, no graph) for
    # the dominant kernel's rate, and the per-phase cycle counters
    prob.profile(True)
    prob.solve(opts, args.n_outer, fetch=False)
    solver_ms, solver_launches = prob.profile(False)
    phases = prob.phase_cycles()
    tot = max(sum(v for k, v in phases.items() if k != "rows_copy_wait"), 1)
    phase_share = {k: round(v / tot, 4) for k, v in phases.items()}
    ms_max = rank_reduce([ms], ["max"], ws, "cuda")[0]
    step_s = ms_max / 1000.0 / args.steps

    # every step is the same computation: the last step's per-instance outcome holds for all
    st = prob.stats()
    ok = counted(st, args.feas_tol)
    n_ok = int(ok.sum())
    value = rank_reduce([n_ok], ["sum"], ws, "cuda")[0] / step_s
    iters = st["cum_iters"]
    w = 4 if prec == nrto.PREC_MIXED else 8
    bytes_step = bytes_design = 0.0
    for i, x in enumerate(insts):
        S, C = entries(x)
        bytes_step += (3 * S + 2 * C) * w * iters[i]
        bytes_design += ((3 + x.nu / x.nx) * S + 2 * C) * w * iters[i]
    launches_per_step = solver_launches
    solver_s_step = solver_ms / 1000.0
    achieved = bytes_step / solver_s_step / 1e9
    peak, peak_kind = measured_peak("hbm_gbs", 6400.0)
    # per-launch DRAM traffic scaled from the capture by the algorithmic bytes (units processed)
    traffic = None
    if kernel_sources_sha() == TRAFFIC["sources_sha256"]:
        traffic = TRAFFIC["ratio"]["both"] * bytes_step / max(launches_per_step, 1e-30)
    # the batch's mixed-precision results of the sample, for the per-result comparison with FP64
    ids = sample_ids(args, len(insts))
    sol_mixed = mixed_results(prob, ids) if rank == 0 and not args.no_plain else None

    # end to end through the C ABI with host buffers: upload the step's problem data, solve, read
    # back the solution and the per-instance outcome
    e2e = None
    if not args.no_e2e:
        h2d = 0
        for x in insts:
            h2d += 8 * (x.u_init.size + x.Sigma.size + x.x0.size + x.x_goal.size + x.obs_center.size
                        + x.obs_radius.size + x.dyn_params.size + 4 * x.nx + 6 * x.nu)
        d2h = 8 * sum(x.T * x.nu * (1 + x.nx) + 1 for x in insts) + 8 * nrto.NSTAT * len(insts)
        n_e2e = min(args.steps, 2)
        barrier()
        t0 = time.perf_counter()
        n_ok_e2e = 0
        for _ in range(n_e2e):
            prob.update(insts)
            prob.solve(opts, args.n_outer, fetch=True)
            n_ok_e2e = int(counted(prob.stats(), args.feas_tol).sum())
        barrier()
        t1 = time.perf_counter()
        e2e_s, e2e_ok = rank_reduce([t1 - t0, n_ok_e2e], ["max", "sum"], ws, "cuda")
        e2e = {"value": e2e_ok * n_e2e / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": n_e2e}

    # Monte Carlo robust-constraint satisfaction of the returned iterates (Sec. V, Methodology),
    # outside the timed region: interior and edge disturbances per instance, rollouts through the
    # nonlinear dynamics, a rollout counting when every constraint holds to the solve's tolerance
    mc = None
    if args.mc > 0:
        st_mc = prob.stats()
        ok_mc = counted(st_mc, args.feas_tol)
        t0 = time.perf_counter()
        sat = prob.monte_carlo(args.mc, args.mc, seed=2603, tol=args.feas_tol)
        mc_s = time.perf_counter() - t0
        ns = 2 * args.mc
        mc = {"samples_per_instance": ns, "interior": args.mc, "edge": args.mc, "tol": args.feas_tol,
              "satisfied_frac_counted": float(sat[ok_mc].sum() / (ns * max(1, int(ok_mc.sum())))),
              "counted_all_satisfied": int((sat[ok_mc] == ns).sum()), "counted": int(ok_mc.sum()),
              "satisfied_frac_all": float(sat.sum() / (ns * len(insts))),
              "seconds": mc_s, "precision": "f64", "iterate": "the returned iterate of the end-to-end run"}

    plain = errs = cfgs = warm = cpu = None
    if rank == 0:
        if not args.no_plain:
            plain = plain_arm(args, insts, stream)
            errs = fp64_errors(args, insts, ids, sol_mixed, st, stream)
        if not args.no_configs:
            cfgs = single_configs(args, stream)
    # the dominant kernel's steady rate, beside the schedule's: fixed work (2 outer steps x 40
    # iterations, no termination checks), so that every instance runs to the end of its launch and
    # the launches have no tail of a few long solves on otherwise idle SMs
    fixed = None
    if rank == 0:
        prob.profile(True)
        prob.solve(tune_opts, 2, fetch=False)
        fw_ms, fw_launches = prob.profile(False)
        fw_iters = prob.stats()["cum_iters"]
        fw_bytes = sum((3 * S + 2 * C) * w * fw_iters[i] for i, (S, C) in enumerate(entries(x) for x in insts))
        fw_gbs = fw_bytes / (fw_ms / 1000.0) / 1e9
        fixed = {"work": "2 outer steps x 40 FullADMM iterations, no termination checks", "achieved": fw_gbs,
                 "frac": fw_gbs / peak, "solver_ms": fw_ms, "launches": int(fw_launches)}
    prob.close()
    if rank == 0 and not args.no_warm:
        warm = warm_start_study(stream, n_train=args.warm_train, n_eval=args.warm_eval)
    if rank == 0 and not args.no_cpu:
        cpu = oracle_estimate(insts, args)
    clocks = clocks_summary(clk_path, local)
    if rank == 0:
        kinds = np.array([x.kind for x in insts])
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == nrto.PREC_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": f"batch{args.n}_mixed_unicycle_quadcopter", "instances_per_gpu": args.n,
                       "n_outer": args.n_outer, "max_inner": args.max_inner, "max_inner_final": args.max_inner_final,
                       "precision": args.prec, "rho0": args.rho, "adapt_every": args.adapt,
                       "stall_every": args.stall, "stall_budget": args.stall_budget, "carry": args.carry,
                       "feas_tol": args.feas_tol, "r0": args.r0, "w_p": args.w_p, "adapt_mu": args.adapt_mu,
                       "l2": "inputs larger than L2 (row arrays of several GB)",
                       "counted": n_ok, "counted_frac": n_ok / prob.n,
                       "counted_by_kind": {"unicycle": int(ok[kinds == 0].sum()), "quadcopter": int(ok[kinds == 1].sum())},
                       "solves_per_s_all": ws * args.n / step_s,
                       "final_inner_converged_frac": float(np.mean(st["status"] == 1)),
                       "final_inner_stalled_frac": float(np.mean(st["status"] == 5)),
                       "inner_iters_per_solve_mean": float(np.mean(iters)),
                       "iterations_per_s": ws * float(np.sum(iters)) / step_s},
            "plain_fp64_gpu": plain,
            "ratio_vs_plain": (value / plain["value"]) if plain and plain["value"] > 0 else None,
            "error_vs_fp64": errs,
            "monte_carlo": mc,
            "gpu_launches": int(launches),
            "graph_replays": int(graph_replays),
            "autotune": {"chosen_mapping": int(tuned), "ms_per_mapping": [float(x) for x in tune_ms],
                         "mappings": ["kinds in sequence", "kinds concurrent", "concurrent, SMs split by row entries",
                                      "concurrent, SMs split by row entries x horizon"],
                         "work": "2 outer steps x 40 FullADMM iterations per candidate"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": "k_fulladmm",
                         "peak_source": peak_kind, "solver_ms_per_step": solver_ms,
                         "avg_launch_ms": solver_ms / max(solver_launches / max(len(set(int(x.kind) for x in insts)), 1), 1),
                         "launches": int(solver_launches),
                         "timing": "one step with CUDA events around each inner solve's persistent launches (the "
                                   "dynamics kinds' launches run concurrently; avg_launch_ms is per concurrent pair)",
                         "algorithmic_bytes_per_launch": bytes_step / max(launches_per_step, 1e-30),
                         "bytes_per_iteration": "(3 S + 2 C) w: read b-hat and the adjoint rows, read and write "
                                                "lambda_nu (state rows), read and write lambda_nu (control rows)",
                         "design_bytes_per_launch": bytes_design / max(launches_per_step, 1e-30),
                         "fixed_work": fixed},
            "phase_share": phase_share,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "configs": cfgs,
            "warm_start": warm,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
