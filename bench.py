"""Benchmark: NRTO solves/sec of the batched, mixed-precision FullADMM path on one B300.

One step = one full NRTO solve (10 successive-linearization outer steps, each with a FullADMM
inner solve that stops at full residuals <= 1e-4 or after --max-inner iterations; the default 40
iterations and rho = 10 are the paper's FullADMM settings, Supplementary Tables VI-VIII) of every
instance of the batched workload (2048 seeded instances, 50/50 unicycle T~U{20..200} with 1-20
obstacles and quadcopter T~U{50..150} with 1-15 obstacles).  Inputs are resident in HBM before the
timed region; the row arrays (several GB) exceed the 126 MB L2, so no flush is needed.

`--impl reference` times the CPU oracle (the reference arm of this project) on a bounded sample of
the same workload.  Under torchrun, every rank solves its own batch (weak scaling); there is no
collective on the data path, only a barrier and a max-reduction of the timings.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "NRTO solves/sec at residual <=1e-4 (batched mixed-precision FullADMM, 10 outer steps)"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--n-outer", type=int, default=10)
    ap.add_argument("--max-inner", type=int, default=40)
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--rho", type=float, default=10.0)
    ap.add_argument("--adapt", type=int, default=0, help="residual-balancing period (0 = fixed rho)")
    ap.add_argument("--stall", type=int, default=0, help="stall-stop period (0 = off)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned-warm-start study")
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the raw nvidia-smi clock samples (default: a temporary directory)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def workload(n, rank):
    from paper_2603_02642_b300 import workloads as W
    return W.batched_mix(n, base_seed=10000 + rank * n)


def row_entries(inst):
    """Ragged row entries of one instance (state rows: (t+1)·nx, control bounds: nx)."""
    per_t = inst.n_obs * (inst.link_spheres.shape[0] if inst.kind == 2 else 1)
    per_t += int(np.isfinite(inst.x_lo).sum() + np.isfinite(inst.x_hi).sum())
    nst = sum((t + 1) * inst.nx for t in range(1, inst.T + 1))
    nc = int(np.isfinite(inst.u_lo).sum() + np.isfinite(inst.u_hi).sum())
    return per_t * nst + nc * inst.T * inst.nx


# ---------------------------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------------------------
def oracle_estimate(instances, n_outer, max_inner, budget_s=20.0, seed=0):
    """Time the FP64 NumPy oracle on a bounded sample of the workload and scale to solves/s.

    Sample: instances drawn with a fixed seed among those whose rows hold <= 60k entries; for each,
    one linearization and one complete FullADMM inner solve (tolerance 1e-4, cap max_inner), until
    `budget_s` of CPU time is used.  Scaling: oracle seconds per (row entry × inner iteration) and
    per (row entry × linearization) from the sample, times the workload's row entries, the sample's
    mean inner iterations per outer step, n_outer outer steps and two linearizations per outer step."""
    from oracle import fulladmm as F, problem as P

    rng = np.random.default_rng(seed)
    cand = [i for i in rng.permutation(len(instances)) if row_entries(instances[i]) <= 60000]
    t_in = t_lin = s_it = s_ent = 0.0
    iters, used = [], []
    t_start = time.perf_counter()
    for i in cand:
        if time.perf_counter() - t_start > budget_s and used:
            break
        inst = instances[i]
        t0 = time.perf_counter()
        lin = P.linearize(inst, inst.u_init)
        t1 = time.perf_counter()
        s = F.iterate(inst, lin, F.FullADMMOptions(rho=10.0, r_trust=2.0, max_iter=max_inner))
        t2 = time.perf_counter()
        e = row_entries(inst)
        t_lin += t1 - t0
        t_in += t2 - t1
        s_it += s.iters * e
        s_ent += e
        iters.append(s.iters)
        used.append(int(i))
    c_it = t_in / s_it
    c_lin = t_lin / s_ent
    m_it = float(np.mean(iters))
    total_entries = float(sum(row_entries(x) for x in instances))
    per_step_s = n_outer * (m_it * c_it * total_entries + 2 * c_lin * total_entries)
    return dict(value=len(instances) / per_step_s, unit=UNIT, cores=1, kind="oracle",
                sample=(f"{len(used)} workload instances (ids {used}) with <=60k row entries: one linearization "
                        f"+ one FullADMM inner solve each (mean {m_it:.0f} iterations), {t_in + t_lin:.1f} s of "
                        f"single-thread CPU; scaled per row entry to the {len(instances)}-instance workload "
                        f"x {n_outer} outer steps"))


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


# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) over algorithmic bytes of one
# k_fulladmm launch per dynamics kind (0 unicycle, 1 quadcopter), from a full capture of 148 mixed
# instances x 40 iterations.  The launch at the benchmark size is scaled from it by its algorithmic
# bytes (traffic grows with row entries x iterations).  Valid only for the kernel sources it was
# measured on: any change to them makes the reported traffic null until it is measured again.
TRAFFIC = {"sources_sha256": "eff2433af36d414ff3515553259a35ce1cff0034a51ebd97c1c7c299926fa02c",
           "ratio": {0: 0.6565, 1: 0.9781}}
KERNEL_SOURCES = ["fulladmm.cuh", "nrto_dev.cuh", "tma.cuh", "linearize.cuh", "dynamics.cuh"]


def kernel_sources_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2603_02642_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_peak_bf16():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["bf16_tflops"]), "measured (burst)"
    except Exception:
        return 1800.0, "fallback"


def warm_start_study(stream, n_train=512, n_eval=256, n_infer=4096, steps=1000):
    """Learned warm start on the quadcopter workload (T = 100, 1-15 obstacles): targets from cold
    FullADMM solves of the first outer step, training by the library's kernels, then cold vs
    warm-started solves (to full residuals <= 1e-4, <= 5000 iterations, residual balancing every 25)
    of held-out instances, and the network's tensor-core GEMM rate on an inference batch."""
    import torch
    from paper_2603_02642_b300 import nrto, warmstart as WS, workloads as W
    opts = dict(rho=10.0, max_inner=5000, eps_p=1e-4, eps_d=1e-4, check=1, adapt_every=25)
    t0 = time.perf_counter()
    train = [W.warmstart_quad(s) for s in range(n_train)]
    prob = nrto.Problem(train, nrto.PREC_MIXED, stream=stream.cuda_stream)
    prob.linearize()
    prob.set_trust_radius(2.0)
    out = prob.solve_socp(nrto.Options(**opts))
    X, Y, Mk = WS.collect_targets(prob, train, out["status"])
    prob.close()
    t_data = time.perf_counter() - t0
    ws = WS.WarmStart(max_batch=n_infer, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    hist = ws.fit(X, Y, Mk, steps=steps, batch=256, lr=1e-3)
    t_fit = time.perf_counter() - t0
    test = [W.warmstart_quad(1_000_000 + s) for s in range(n_eval)]
    res = {}
    # cold start; warm start; warm start with the cold fallback on a residual plateau (r_p above its
    # tolerance and down by less than 1% over 1000 iterations)
    for mode in ("cold", "warm", "warm_fallback"):
        q = nrto.Problem(test, nrto.PREC_MIXED, stream=stream.cuda_stream)
        q.linearize()
        q.set_trust_radius(2.0)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        if mode != "cold":
            ws.apply(q, test)
        e1.record(stream)
        fbk = mode == "warm_fallback"
        o = q.solve_socp(nrto.Options(stall_every=1000 if fbk else 0, stall_ratio=0.99, warm_fallback=int(fbk),
                                      **opts))
        e2.record(stream)
        torch.cuda.synchronize()
        fb = sum(int(q.export(nrto.F_STATS, i)[6]) for i in range(n_eval))
        res[mode] = dict(iters=o["iters"].copy(), conv=o["status"] == 1, solve_ms=e1.elapsed_time(e2),
                         predict_ms=e0.elapsed_time(e1), fallbacks=fb)
        q.close()
    both = res["cold"]["conv"] & res["warm"]["conv"] & res["warm_fallback"]["conv"]
    # tensor-core rate of the network's GEMMs on an inference batch
    feats = WS.features([W.warmstart_quad(2_000_000 + s) for s in range(n_infer)])
    ws.net.forward(feats)
    ws.net.profile(True)
    ws.net.forward(feats)
    gms, gfl, gn = ws.net.profile(False)
    peak, peak_kind = measured_peak_bf16()
    achieved = gfl / (gms / 1e3) / 1e12
    ws.net.close()
    def summary(r, warm):
        total_ms = r["solve_ms"] + (r["predict_ms"] if warm else 0.0)
        d = {"converged": int(r["conv"].sum()), "solve_ms": r["solve_ms"],
             "solves_per_s": n_eval / (total_ms / 1e3),
             "converged_per_s": int(r["conv"].sum()) / (total_ms / 1e3),
             "iters_mean_all_converged": float(r["iters"][both].mean()) if both.any() else None}
        if warm:
            d["predict_ms"] = r["predict_ms"]
            d["fallbacks"] = r["fallbacks"]
        return d

    return {
        "workload": f"quadcopter T=100, 1-15 obstacles (warmstart_quad); train seeds 0..{n_train - 1}, "
                    f"held-out seeds 1000000..{1000000 + n_eval - 1}",
        "targets": int(X.shape[0]), "train_steps": steps, "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
        "data_s": round(t_data, 2), "fit_s": round(t_fit, 2),
        "held_out": n_eval, "converged_in_all_three": int(both.sum()),
        "cold": summary(res["cold"], False),
        "warm": summary(res["warm"], True),
        "warm_fallback": summary(res["warm_fallback"], True),
        "mlp_roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "peak_source": peak_kind, "batch": n_infer,
                         "gemm_launches": int(gn), "gemm_ms": gms},
    }


def measured_peak_gbs():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def reference_arm(args):
    insts = workload(args.n, 0)
    vals = []
    for k in range(args.warmup + args.steps):
        est = oracle_estimate(insts, args.n_outer, args.max_inner, budget_s=15.0, seed=k)
        if k >= args.warmup:
            vals.append(est)
    value = float(np.mean([v["value"] for v in vals]))
    est = dict(vals[-1])
    est["value"] = value
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * args.n / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"batch{args.n}_mixed_unicycle_quadcopter", "n_outer": args.n_outer,
                       "max_inner": args.max_inner, "instances_per_gpu": args.n},
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
    stream = torch.cuda.current_stream()
    prob = nrto.Problem(insts, prec, stream=stream.cuda_stream)
    opts = nrto.Options(rho=args.rho, max_inner=args.max_inner, eps_p=1e-4, eps_d=1e-4, check=1, r0=2.0,
                        adapt_every=args.adapt, stall_every=args.stall)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        prob.solve(opts, args.n_outer, fetch=False)
    barrier()
    clk_dir = args.clocks_dir or tempfile.gettempdir()
    clk_path = os.path.join(clk_dir, f"nrto_clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    clk = clocks_start(clk_path)
    time.sleep(0.5)
    launches0 = prob.kernel_launches()
    prob.profile(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        prob.solve(opts, args.n_outer, fetch=False)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    solver_ms, solver_launches = prob.profile(False)
    phases = prob.phase_cycles()
    tot = max(sum(v for k, v in phases.items() if k != "rows_copy_wait"), 1)
    phase_share = {k: round(v / tot, 4) for k, v in phases.items()}
    launches = prob.kernel_launches() - launches0
    if clk:
        clk.terminate()
        clk.wait()
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = ws * args.n * args.steps / (ms_max / 1000.0)

    # per-instance iteration counts of the last step (every step is the same computation)
    stats = np.array([prob.export(nrto.F_STATS, i) for i in range(prob.n)])
    iters = stats[:, 0]
    w = 4 if prec == nrto.PREC_MIXED else 8
    bytes_step = 0.0
    bytes_kind = {}
    for i, inf in enumerate(prob.info):
        s_state = inf.n_entries_state
        per_it = (3 + inf.nu / inf.nx) * s_state * w + 2 * w * (inf.n_entries - s_state)
        bytes_step += per_it * iters[i]
        bytes_kind[insts[i].kind] = bytes_kind.get(insts[i].kind, 0.0) + per_it * iters[i]
    launches_per_step = solver_launches / max(args.steps, 1)
    avg_launch_s = solver_ms / 1000.0 / max(solver_launches, 1)
    achieved = bytes_step / launches_per_step / avg_launch_s / 1e9
    peak, peak_kind = measured_peak_gbs()
    traffic = None
    if (prec == nrto.PREC_MIXED and kernel_sources_sha() == TRAFFIC["sources_sha256"]
            and all(k in TRAFFIC["ratio"] for k in bytes_kind)):
        traffic = sum(TRAFFIC["ratio"][k] * b for k, b in bytes_kind.items()) / max(launches_per_step, 1e-30)
    conv = int(np.sum(stats[:, 2] == 1))
    stalled = int(np.sum(stats[:, 2] == 5))

    # end to end through the C ABI with host buffers: upload the step's problem data, solve, read back
    e2e = None
    if not args.no_e2e:
        h2d = 0
        for x in insts:
            h2d += 8 * (x.u_init.size + x.Sigma.size + x.x0.size + x.x_goal.size + x.obs_center.size
                        + x.obs_radius.size + x.dyn_params.size + 4 * x.nx + 6 * x.nu)
        d2h = 8 * sum(x.T * x.nu * (1 + x.nx) + 1 for x in insts)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            prob.update(insts)
            prob.solve(opts, args.n_outer, fetch=True)
        barrier()
        t1 = time.perf_counter()
        tt = torch.tensor([t1 - t0], dtype=torch.float64, device="cuda")
        if ws > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e = {"value": ws * args.n * args.steps / float(tt.item()), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    warm = None
    if rank == 0 and not args.no_warm:
        prob.close()
        warm = warm_start_study(stream)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_estimate(insts, args.n_outer, args.max_inner)
    clocks = clocks_summary(clk_path, local)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == nrto.PREC_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": f"batch{args.n}_mixed_unicycle_quadcopter", "instances_per_gpu": args.n,
                       "n_outer": args.n_outer, "max_inner": args.max_inner, "precision": args.prec, "rho0": args.rho,
                       "adapt_every": args.adapt, "stall_every": args.stall,
                       "l2": "inputs larger than L2 (row arrays of several GB)",
                       "inner_iters_per_solve_mean": float(np.mean(iters)),
                       "final_inner_converged_frac": conv / prob.n,
                       "final_inner_stalled_frac": stalled / prob.n,
                       "iterations_per_s": ws * float(np.sum(iters)) * args.steps / (ms_max / 1000.0)},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": "k_fulladmm",
                         "peak_source": peak_kind, "avg_launch_ms": avg_launch_s * 1000.0,
                         "launches": int(solver_launches),
                         "algorithmic_bytes_per_launch": bytes_step / max(launches_per_step, 1e-30)},
            "phase_share": phase_share,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "warm_start": warm,
        }
        print(json.dumps(line))
    prob.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
