#!/usr/bin/env python
"""Benchmark of the two-site A2DMRG hot path on one GB300.

Workload (default): random chemistry-like Hamiltonian, L = 16 spatial orbitals
(n = 4), integrals seed 2505, exact operator-string MPO, TT bond cap D = 256,
P = 4 groups of bonds [4, 4, 4, 3], seeded initial TT (SplitMix64 seed 23429,
initial bond 4).  A step is one A2DMRG global iteration (Alg. 2): LQ sweep,
environments, the P groups of local two-site Lanczos solves (tensor-core BF16
matvecs, FP32 refinement), truncated SVDs, coarse problem, compression.

Timing: W untimed warm-up iterations from the seeded TT, then K timed
iterations bracketed by a barrier and device synchronisation, CUDA events on
the library's stream.  The working set (environments, intermediates of several
GB) is far larger than the 129 MB L2, so no explicit flush is done.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the oracle is the reference of this build).
"""
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
sys.path.insert(0, ROOT)

METRIC = ("additive-sweep time to |dE|<1e-6 vs FP64 oracle; "
          "H_eff matvec TFLOP/s vs plain")
# classes reported by time share only (latency-bound FP64 factorisations)
LATENCY_BOUND = ("svd", "lq")
# DRAM traffic / algorithmic bytes of a kernel class, from its ncu capture at D = 128;
# the bench scales it to its own launches
DRAM_TRAFFIC_RATIO = {"emu_s2": 0.963, "emu_s3": 0.961}
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
FP64_PEAK_TFLOPS = 1.2   # FP64 (SIMT) rate measured on this part with a DGEMM loop


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default="bf16",
                   choices=["bf16", "f32emu", "fp32", "fp64", "f64emu"])
    p.add_argument("--solver", default="lanczos", choices=["lanczos", "davidson"])
    p.add_argument("--converge", type=int, default=45,
                   help="after the timed steps, keep iterating (up to this many iterations in "
                        "total) until |dE|/|E| < 1e-6, to report the time from the seeded TT")
    p.add_argument("--groups", default="sequential", choices=["sequential", "concurrent"],
                   help="run the P groups one after another (default: each local matvec "
                        "already fills the GPU, and per-kernel timings stay unshared) or "
                        "concurrently on one stream per group")
    p.add_argument("--sequential", action="store_true", help="same as --groups sequential")
    p.add_argument("--coarse-eps", type=float, default=None,
                   help="S_hat eigenvalue cut (default 1e-10; 1e-5 for plain fp32)")
    p.add_argument("--no-refine", action="store_true",
                   help="bf16 / f32emu: skip the FP64 refinement of the local Ritz pairs")
    p.add_argument("--no-fold", action="store_true",
                   help="keep every MPO core fully sparse (no identity-block fold)")
    p.add_argument("--config", default="chem_L16_D256")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-mv", action="store_true",
                   help="skip the H_eff matvec comparison (e.g. under a profiler)")
    p.add_argument("--profile-matvec", action="store_true",
                   help="small case for ncu: H_eff applications at the middle bond only")
    p.add_argument("--D", type=int, default=128, help="bond dimension of --profile-matvec")
    p.add_argument("--bond", type=int, default=None,
                   help="bond of --profile-matvec (default: the one left of the middle)")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--one-site", action="store_true",
                   help="the one-site case of Alg. 2 (P groups of the L cores)")
    p.add_argument("--n-eig", type=int, default=1,
                   help="Extension One: eigenvectors kept per group's last local problem")
    p.add_argument("--low-memory", action="store_true",
                   help="memory-limited environment mode (environments rebuilt on demand)")
    p.add_argument("--graphs", action="store_true",
                   help="replay every local operator's H_eff applications from a CUDA graph")
    p.add_argument("--f64emu", action="store_true",
                   help="--profile-matvec also applies the FP64-emulated chain")
    return p.parse_args()


def workload(name):
    from synthetic import (chemistry_integrals, chemistry_mpo, get_config, heisenberg_mpo,
                           random_tt_cores)
    cfg = get_config(name)
    if cfg["kind"] == "chemistry":
        h, eri = chemistry_integrals(cfg["L"], cfg["seed_int"])
        mpo = chemistry_mpo(h, eri)
    elif cfg["kind"] == "heisenberg":
        mpo = heisenberg_mpo(cfg["L"], cfg["J"])
    else:
        raise SystemExit(f"config {name} not supported by this bench")
    raw = random_tt_cores([cfg["n"]] * cfg["L"], cfg["r0"], cfg["seed_tt"])
    return cfg, mpo, raw


def sweep_kwargs(cfg, prec, solver="lanczos", coarse_eps=None, refine=1):
    if coarse_eps is None:
        # A_hat and S_hat are FP64-class in every precision but plain FP32
        coarse_eps = 1e-5 if prec == "fp32" else 1e-10
    return dict(partition=cfg["partition"], D_max=cfg["D"], svd_tol=1e-6, eig_tol=1e-6,
                coarse_eps=coarse_eps, max_krylov=40, max_restarts=50, prec=prec,
                solver=solver, refine=refine)


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"],
                    src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""
    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9
                          for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(mx) if mx else None, reasons=reasons, samples=len(rows))


def oracle_sample(cfg, mpo):
    """One oracle H_eff application at the middle bond with D = D_max (bounded CPU sample)."""
    from oracle.env import heff_apply
    L, D, n = cfg["L"], cfg["D"], cfg["n"]
    k = L // 2 - 1
    rng = np.random.default_rng(0)
    W1, W2 = mpo[k], mpo[k + 1]
    HL = rng.standard_normal((D, W1.shape[0], D))
    HR = rng.standard_normal((D, W2.shape[3], D))
    x = rng.standard_normal((D, n, n, D))
    t = time.perf_counter()
    heff_apply(HL, W1, W2, HR, x)
    dt = time.perf_counter() - t
    nnz1, nnz2 = np.count_nonzero(W1), np.count_nonzero(W2)
    flops = (2.0 * n * n * D * D * (W1.shape[0] * D + W2.shape[3] * D)
             + 2.0 * n * D * D * (nnz1 + nnz2))
    return dt, flops, k


def reference_arm(args):
    cfg, mpo, _ = workload(args.config)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    samples = []
    for _ in range(args.warmup + args.steps):
        samples.append(oracle_sample(cfg, mpo))
    timed = samples[args.warmup:]
    dt = sum(s[0] for s in timed) / len(timed)
    rate = timed[0][1] / dt
    # scale to one global iteration with the algorithmic flops of a full-rank iteration
    flops_iter = est_iteration_flops(cfg, mpo)
    value = rate / flops_iter
    cores = os.cpu_count()
    line = dict(impl="reference", metric=METRIC, value=value, unit="additive sweeps/s",
                n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 / value, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=args.config, L=cfg["L"], n=cfg["n"], D=cfg["D"], P=cfg["P"]),
                cpu_baseline=dict(value=value, unit="additive sweeps/s", cores=cores,
                                  kind="oracle",
                                  sample=(f"one FP64 oracle H_eff application at bond {timed[0][2]} "
                                          f"(D={cfg['D']}) per step, {dt:.2f} s, "
                                          f"{rate / 1e9:.1f} GFLOP/s algorithmic, scaled by "
                                          f"{flops_iter:.3e} algorithmic flops per global iteration")),
                e2e=dict(value=value, unit="additive sweeps/s", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0))
    print(json.dumps(line))


def est_iteration_flops(cfg, mpo, matvecs_per_bond=30):
    """Algorithmic flops of one full-rank global iteration (matvec + env dominated)."""
    L, D, n = cfg["L"], cfg["D"], cfg["n"]
    dims = [1] + [min(D, n ** min(k, L - k)) for k in range(1, L)] + [1]
    tot = 0.0
    for k in range(L - 1):
        Dl, Dr = dims[k], dims[k + 2]
        W1, W2 = mpo[k], mpo[k + 1]
        fmv = (2.0 * n * n * Dl * Dr * (W1.shape[0] * Dl + W2.shape[3] * Dr)
               + 2.0 * n * Dl * Dr * (np.count_nonzero(W1) + np.count_nonzero(W2)))
        tot += matvecs_per_bond * fmv
    for j in range(L):
        Dl, Dr = dims[j], dims[j + 1]
        W = mpo[j]
        fenv = (2.0 * n * Dl * Dr * (W.shape[0] * Dl + W.shape[3] * Dr)
                + 2.0 * Dl * Dr * np.count_nonzero(W))
        tot += (2 + cfg["P"]) * fenv
    return tot


def profile_matvec(args):
    """H_eff at one bond of the L=16 chemistry MPO with random environments of bond
    dimension --D: BF16, FP32-accurate and (with --f64emu) FP64-emulated tensor-core chains
    (operator handles, the environments converted once), --reps applications each."""
    import torch
    import paper_2505_23429_gb300 as a2
    cfg, cores, _ = workload(args.config)
    ctx = a2.Context(0)
    mpo = a2.MPO(ctx, cores)
    k = cfg["L"] // 2 - 1 if args.bond is None else args.bond
    D, n = args.D, cfg["n"]
    g = torch.Generator(device="cuda").manual_seed(0)
    HL = torch.randn(D, cores[k].shape[0], D, device="cuda", dtype=torch.float64, generator=g)
    HR = torch.randn(D, cores[k + 1].shape[3], D, device="cuda", dtype=torch.float64, generator=g)
    x = torch.randn(D, n, n, D, device="cuda", dtype=torch.float64, generator=g)
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    classes = {}
    for prec in ("bf16", "f32emu") + (("f64emu",) if args.f64emu else ()):
        op = a2.HeffOp(ctx, mpo, k, HL, HR, prec=prec)
        op.apply(x, y)                       # first application: autotuner, scratch growth
        ctx.synchronize()
        a2.profile(ctx, "reset")
        a2.profile(ctx, "on")
        for _ in range(args.reps):
            op.apply(x, y)
        ctx.synchronize()
        a2.profile(ctx, "off")
        op.close()
        for i, name in enumerate(a2.a2dmrg.PROFILE_KINDS):   # per-application class times
            r = a2.profile(ctx, "read", i)
            if r["launches"]:
                classes[f"{prec}:{name}"] = round(r["ms"] / max(args.reps, 1), 3)
    print(json.dumps(dict(profile_matvec=True, D=D, bond=k, reps=args.reps,
                          ms_per_application=classes, error_flag=a2.device_error(ctx))))


def class_roofline(name, d, peaks, prec):
    """(bound, unit, peak, achieved) of one kernel class from its CUDA-event totals and
    the algorithmic flops / bytes the library counts for it."""
    rate_f = d["flops"] / (d["ms"] * 1e-3) / 1e12
    rate_b = d["bytes"] / (d["ms"] * 1e-3) / 1e9
    if name in ("tc_s1", "tc_s4", "emu_s1", "emu_s4"):
        return "tensor", "TFLOP/s", peaks["bf16_sus"], rate_f
    if name in ("sparse_s2", "sparse_s3", "emu_s2", "emu_s3", "lanczos", "f64e_split"):
        return "hbm", "GB/s", peaks["hbm"], rate_b
    if name in ("f64e_s1", "f64e_s4"):   # 36 BF16 products per FP64-equivalent flop
        return "tensor", "TFLOP/s", peaks["bf16_sus"], 36.0 * rate_f
    if name == "f64e_sparse":
        return "alu", "TFLOP/s", FP32_SIMT_PEAK_TFLOPS, rate_f
    if name == "env" and prec in ("bf16", "f32emu"):
        return "tensor", "TFLOP/s", peaks["bf16_sus"], rate_f
    if name in ("heff_simt", "env") and prec != "fp64":
        return "alu", "TFLOP/s", FP32_SIMT_PEAK_TFLOPS, rate_f
    return "alu", "TFLOP/s", FP64_PEAK_TFLOPS, rate_f        # FP64 factorisations / SIMT


def nvtx(torch, name):
    """Push (name) or pop (None) an NVTX range on this thread, if NVTX is available."""
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def max_over_ranks(ms, world, device):
    """Slowest rank's timed-region length (the job ends when the last replica ends)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps, ms, world):
    """Whole-job global iterations per second: every rank runs `steps` independent
    replica iterations in `ms` (max over ranks)."""
    return steps * world / (ms * 1e-3)


def main():
    args = parse()
    if args.profile_matvec:
        profile_matvec(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.cuda.current_device()
    import paper_2505_23429_gb300 as a2

    cfg, mpo_cores, raw = workload(args.config)
    stream = torch.cuda.Stream()
    ctx = a2.Context(dev, stream.cuda_stream)
    mpo = a2.MPO(ctx, mpo_cores)
    if args.no_fold:
        mpo.set_fold(False)
    kw = sweep_kwargs(cfg, args.prec, args.solver, args.coarse_eps, 0 if args.no_refine else 1)
    kw["sequential"] = args.sequential or args.groups == "sequential"
    P = cfg["P"]
    if args.one_site:   # the one-site case of Alg. 2: P groups of the L cores
        L = cfg["L"]
        kw["partition"] = [L // P + (1 if g < L % P else 0) for g in range(P)]
        kw["one_site"] = True
    if args.n_eig > 1:
        kw["n_eig"] = args.n_eig
    if args.low_memory:
        kw["low_memory"] = True
    if args.graphs:
        kw["graphs"] = True
    t = a2.TT.from_cores(ctx, raw)
    t.left_orthogonalize()

    history = []   # (seconds, energy_in) of every iteration from the seeded TT
    for _ in range(args.warmup):
        rep = a2.additive_sweep(ctx, t, mpo, P, **kw)
        history.append((rep["seconds"], rep["energy_in"]))

    start_cores = t.cores()          # the end-to-end run repeats the timed iterations
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    a2.profile(ctx, "reset")
    a2.profile(ctx, "on")
    launches0 = a2.profile(ctx, "launches")
    clocks = Clocks()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    w0 = time.perf_counter()
    reps = []
    nvtx(torch, "timed_steps")     # lets a profiler select the timed region
    for _ in range(args.steps):
        rep = a2.additive_sweep(ctx, t, mpo, P, **kw)
        reps.append(rep)
        history.append((rep["seconds"], rep["energy_in"]))
        print(json.dumps(dict(iteration=len(history), seconds=rep["seconds"],
                              energy_in=rep["energy_in"], lambda_coarse=rep["lambda_coarse"],
                              coarse_rank=rep["coarse_rank"], krylov=rep["krylov"],
                              max_discarded=rep["max_discarded"])), file=sys.stderr)
    ev1.record(stream)
    torch.cuda.synchronize()
    nvtx(torch, None)
    wall = time.perf_counter() - w0
    clk = clocks.stop()
    a2.profile(ctx, "off")
    launches = a2.profile(ctx, "launches") - launches0
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, "cuda")
    prof = {k: a2.profile(ctx, "read", i) for i, k in enumerate(a2.a2dmrg.PROFILE_KINDS)}

    def converged(hist):
        e = [x[1] for x in hist]
        return any(abs(e[i] - e[i - 1]) < 1e-6 * abs(e[i]) for i in range(2, len(e)))
    while args.converge and len(history) < args.converge and not converged(history):
        rep = a2.additive_sweep(ctx, t, mpo, P, **kw)
        history.append((rep["seconds"], rep["energy_in"]))
        print(json.dumps(dict(iteration=len(history), seconds=rep["seconds"],
                              energy_in=rep["energy_in"], lambda_coarse=rep["lambda_coarse"],
                              krylov=sum(rep["krylov"]))), file=sys.stderr)
    E_final, _ = a2.energy(ctx, t, mpo, "fp64")

    # time to |dE| < 1e-6 (relative, between successive global iterations, as in the
    # stopping rule of the experiments), from the seeded TT, if reached in W+K iterations
    # energies[i] = energy after i+1 iterations; the stopping rule compares successive ones
    energies = [e for _, e in history[1:]] + [E_final]
    t_conv, it_conv, cum = None, None, history[0][0]
    for i in range(1, len(energies)):
        cum += history[i][0]
        if abs(energies[i] - energies[i - 1]) < 1e-6 * abs(energies[i]):
            t_conv, it_conv = cum, i + 1
            break

    # dominant kernel class and its roofline (and the same figures for every class)
    peaks = read_peaks()
    # the FP64 factorisations (truncated-SVD eigensolve, LQ) are latency-bound library
    # calls: they get a time share, the roofline goes to the dominant contraction class
    dom = max((k for k in prof if k not in LATENCY_BOUND), key=lambda k: prof[k]["ms"])
    d = prof[dom]
    total_ms = sum(v["ms"] for v in prof.values())
    shares = {k: round(v["ms"] / total_ms, 4) for k, v in prof.items() if v["ms"] > 0}
    ratio = DRAM_TRAFFIC_RATIO.get(dom)
    traffic = ratio * d["bytes"] / max(d["launches"], 1) if ratio else None
    bound, unit, peak, achieved = class_roofline(dom, d, peaks, args.prec)
    per_launch = d["ms"] / max(d["launches"], 1)
    rooflines = {}
    for k, v in prof.items():
        if v["launches"] and v["ms"] > 0:
            b_, u_, p_, a_ = class_roofline(k, v, peaks, args.prec)
            rooflines[k] = dict(bound=b_, achieved=round(a_, 2), peak=p_, unit=u_,
                                frac=round(a_ / p_, 4))

    # H_eff matvec TFLOP/s: tensor-core chain vs a plain torch.einsum chain (dense MPO, BF16)
    mv = None if args.no_mv else matvec_compare(a2, ctx, mpo, mpo_cores, cfg, torch, stream)

    value = job_throughput(args.steps, ms, world)
    line = dict(metric=METRIC, value=value, unit="additive sweeps/s", n_gpus=world,
                steps=args.steps, warmup=args.warmup, ms_per_step=ms / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="bf16+f32 (f64 vectors/SVD/coarse)" if args.prec == "bf16" else args.prec,
                data="synthetic",
                config=dict(workload=args.config, L=cfg["L"], n=cfg["n"], D=cfg["D"], P=P,
                            partition=kw["partition"], eig_tol=1e-6, svd_tol=1e-6,
                            variant=("one-site" if args.one_site else "two-site")
                            + (f", n_eig={args.n_eig}" if args.n_eig > 1 else "")
                            + (", memory-limited environments" if args.low_memory else "")
                            + (", CUDA-graph matvecs" if args.graphs else ""),
                            coarse_eps=kw["coarse_eps"],
                            precision=args.prec, solver=args.solver,
                            groups="sequential" if kw["sequential"] else "concurrent streams",
                            identity_fold=not args.no_fold,
                            parallelism="replicas" if world > 1 else "1gpu",
                            l2="working set >> 129 MB L2 (no flush)"),
                energy_final=E_final, time_to_dE_1e6_s=t_conv, iterations_to_dE_1e6=it_conv,
                iterations_run=len(history),
                roofline=dict(kernel=dom, bound=bound, achieved=achieved, peak=peak, unit=unit,
                              frac=achieved / peak, traffic=traffic,
                              traffic_source=(None if ratio is None else
                                              "ncu DRAM bytes / algorithmic bytes of the same "
                                              "kernel at D=128 (profiles/), scaled to this "
                                              "launch's algorithmic bytes"),
                              per_launch_ms=per_launch, launches=d["launches"],
                              peak_source=peaks["src"]),
                time_shares=shares,
                roofline_classes=rooflines,
                kernel_classes={k: dict(ms=round(v["ms"], 3), launches=v["launches"],
                                        tflops=round(v["flops"] / (v["ms"] * 1e9), 2)
                                        if v["ms"] > 0 else None,
                                        gbs=round(v["bytes"] / (v["ms"] * 1e6), 1)
                                        if v["ms"] > 0 else None)
                                for k, v in prof.items()},
                heff_matvec=mv, clocks=clk, wall_s=wall,
                gpu_launches=int(launches))
    if not args.no_e2e:
        line["e2e"] = e2e_run(a2, ctx, mpo, cfg, kw, start_cores, args.steps, torch, stream,
                              world)
    if rank == 0 and world == 1 and not args.no_cpu:
        dt, fl, k = oracle_sample(cfg, mpo_cores)
        rate = fl / dt
        flops_iter = sum(r["alg_flops"] for r in reps) / len(reps)
        line["cpu_baseline"] = dict(value=rate / flops_iter, unit="additive sweeps/s",
                                    cores=os.cpu_count(), kind="oracle",
                                    sample=(f"one FP64 oracle H_eff application at bond {k} "
                                            f"(D={cfg['D']}), {dt:.2f} s, scaled by the measured "
                                            f"algorithmic flops per global iteration "
                                            f"({flops_iter:.3e})"))
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def matvec_compare(a2, ctx, mpo, cores, cfg, torch, stream):
    """H_eff applications at full bond dimension: the tensor-core chains (BF16,
    FP32-accurate split products, FP64 emulation), the FP64 SIMT chain, and a plain torch.tensordot
    chain of the same contraction in BF16 with the dense MPO cores (cuBLAS), at the
    hand-over bond of the operator automaton and at a typical middle bond."""
    L, D, n = cfg["L"], cfg["D"], cfg["n"]
    out = []
    for k in (L // 2 - 1, L // 2 - 3):
        W1, W2 = cores[k], cores[k + 1]
        g = torch.Generator(device="cuda").manual_seed(0)
        with torch.cuda.stream(stream):
            HL = torch.randn(D, W1.shape[0], D, device="cuda", dtype=torch.float64, generator=g)
            HR = torch.randn(D, W2.shape[3], D, device="cuda", dtype=torch.float64, generator=g)
            x = torch.randn(D, n, n, D, device="cuda", dtype=torch.float64, generator=g)
            y = torch.empty_like(x)
        torch.cuda.synchronize()
        nnz = np.count_nonzero(W1) + np.count_nonzero(W2)
        flops = (2.0 * n * n * D * D * (W1.shape[0] * D + W2.shape[3] * D)
                 + 2.0 * n * D * D * nnz)

        def timeit(fn, reps=10):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        res = dict(bond=k, D=D, R=[int(W1.shape[0]), int(W1.shape[3]), int(W2.shape[3])],
                   nnz=[int(np.count_nonzero(W1)), int(np.count_nonzero(W2))], alg_flops=flops)
        ys = {}
        for prec, reps in (("bf16", 10), ("f32emu", 10), ("f64emu", 3), ("fp64", 1)):
            op = a2.HeffOp(ctx, mpo, k, HL, HR, prec=prec)
            ms = timeit(lambda: op.apply(x, y), reps)
            op.close()
            ys[prec] = y.clone()
            res[f"{prec}_ms"] = ms
            res[f"{prec}_tflops"] = flops / (ms * 1e-3) / 1e12
        ref = ys["fp64"]
        for prec in ("bf16", "f32emu", "f64emu"):   # accuracy against the FP64 SIMT chain
            res[f"{prec}_rel_err"] = float((ys[prec] - ref).norm() / ref.norm())
        with torch.cuda.stream(stream):
            Lb, Rb, xb = HL.bfloat16(), HR.bfloat16(), x.bfloat16()
            W1b = torch.from_numpy(W1).cuda().bfloat16()
            W2b = torch.from_numpy(W2).cuda().bfloat16()

        def plain():
            with torch.cuda.stream(stream):
                T = torch.tensordot(Lb, xb, dims=([2], [0]))                  # a w t1 t2 b'
                T = torch.tensordot(T, W1b, dims=([1, 2], [0, 2]))            # a t2 b' s1 w1
                T = torch.tensordot(T, W2b, dims=([1, 4], [2, 0]))            # a b' s1 s2 w2
                return torch.tensordot(T, Rb, dims=([1, 4], [2, 1]))          # a s1 s2 b
        pl = timeit(plain)
        res["plain_bf16_ms"] = pl
        res["plain_bf16_tflops"] = flops / (pl * 1e-3) / 1e12
        out.append(res)
    return dict(bonds=out, note="timed through a2_heff_apply_op (environments converted once, "
                "as inside a local solve; FP64 x in, FP64 y out); plain = torch.tensordot chain "
                "in BF16 with the dense MPO cores (cuBLAS) on BF16 environments converted "
                "beforehand; TFLOP/s use the algorithmic count with MPO nonzeros")


def e2e_run(a2, ctx, mpo, cfg, kw, cores, steps, torch, stream, world):
    """The timed global iterations again, from the same starting iterate, through the
    host-buffer API: every step uploads the iterate's cores from pinned host memory,
    runs the sweep and reads the cores and the energy back."""
    pinned = [torch.from_numpy(c).pin_memory().numpy() for c in cores]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = d2h = 0
    for _ in range(steps):
        tt = a2.TT.from_cores(ctx, pinned)
        h2d += sum(c.nbytes for c in pinned)
        rep = a2.additive_sweep(ctx, tt, mpo, len(kw["partition"]), **kw)
        out = tt.cores()
        d2h += sum(c.nbytes for c in out) + 8
        pinned = [torch.from_numpy(c).pin_memory().numpy() for c in out]
        tt.close()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return dict(value=steps / dt * world, unit="additive sweeps/s",
                h2d_bytes_per_step=h2d // steps, d2h_bytes_per_step=d2h // steps)


if __name__ == "__main__":
    main()
