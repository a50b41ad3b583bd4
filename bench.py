"""Benchmark of the GB300 excited-state path (one JSON line on rank 0).

A step is one whole excited-state solve (Davidson to convergence: P build,
G build, back-transform, float64 subspace, oscillator strengths) of the
seeded large TDHF workload -- 400 C/N/O + 600 H atoms, 2200 AOs, 10 roots --
with the ground state already resident on the GPU.  value = roots / second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl xs|reference]
                  [--workload large|medium] [--precision mixed|fp64]

Under torchrun (N > 1) every rank solves its own seeded copy of the workload
(independent molecules, no collective) and rank 0 reports the aggregate.
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

import molgen  # noqa: E402

WORKLOADS = {
    "large": dict(gen=molgen.config_large, method="TDHF", nroots=10, tol=1e-5,
                  desc="TDHF, seeded chain of 400 C/N/O + 600 H atoms, 2200 AOs, 10 roots"),
    "medium": dict(gen=molgen.config_medium, method="TDHF", nroots=10, tol=1e-5,
                   desc="TDHF, seeded chain of 100 C/N/O + 200 H atoms, 600 AOs, 10 roots"),
    "batch": dict(method="CIS", nroots=6, tol=1e-5, n_mol=256,
                  desc="CIS, 256 seeded molecules of 20-200 atoms (40% heavy), 6 roots each, batched"),
    "learned": dict(method="TDHF", nroots=8, tol=1e-5, n_train=256, n_test=512,
                    desc="TDHF, 8 roots; MLP guess (the committed network, trained on seeded molecules of "
                         "20-120 atoms) evaluated on 512 held-out molecules of 20-300 atoms, batched"),
}
METRIC = "TDHF roots/s @1e-5 eV"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return dict(hbm_gbs=p.get("hbm_gbs", 6800.0), bf16_tflops=p.get("bf16_tflops", 1900.0),
                    bf16_sustained=p.get("bf16_tflops_sustained", 1700.0), source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_sustained=1700.0, source="fallback")


# float64 and float32 SIMT FMA throughput of this GB300 measured by the
# project's own probe kernel (paper_2505_24807_gb300/probe_peaks.cu): 1.195
# and 72.99 TFLOP/s.
FP64_SIMT_TFLOPS = 1.195
FP32_SIMT_TFLOPS = 72.99


def kernel_roofline(name, t, pk):
    """Achieved rate of one profiled kernel family against its bound: digit
    products, digit splits and the G build stream HBM (algorithmic bytes);
    tensor-core GEMMs against the TF32 peak; SIMT kernels against the float64
    or float32 pipe."""
    per_launch_s = t["ms"] / 1e3 / t["launches"]
    if name.startswith(("oz_", "gbuild")) and t["bytes"] > 0:
        ach = t["bytes"] / t["launches"] / per_launch_s / 1e9
        return dict(kernel=name, bound="hbm", achieved=ach, peak=pk["hbm_gbs"], unit="GB/s",
                    frac=ach / pk["hbm_gbs"], traffic=None, peak_source=pk["source"] + " hbm_gbs",
                    bytes_per_launch=t["bytes"] / t["launches"], ms_per_launch=per_launch_s * 1e3)
    ach = t["flops"] / t["launches"] / per_launch_s / 1e12
    if name.startswith("tc_"):
        peak, src, bound = pk["bf16_sustained"] / 2.0, pk["source"] + " bf16 sustained x 1/2 (tf32)", "tensor"
    elif "f64" in name:
        peak, src, bound = FP64_SIMT_TFLOPS, "measured fp64 FMA probe", "alu"
    else:
        peak, src, bound = FP32_SIMT_TFLOPS, "measured fp32 FMA probe", "alu"
    return dict(kernel=name, bound=bound, achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak, traffic=None,
                peak_source=src, flops_per_launch=t["flops"] / t["launches"], ms_per_launch=per_launch_s * 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_molecule_seed(rank):
    """Seed of the molecule rank r solves: ranks take independent problems
    (weak scaling, no data-path collective)."""
    return rank


def max_over_ranks(x, device):
    """Largest x over all ranks (every rank receives it); x itself without a
    process group.  Used for the timed region: the job is as slow as its
    slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(world, roots_per_solve, steps, seconds):
    """Whole-job roots/s: every rank's roots over the slowest rank's time."""
    return world * roots_per_solve * steps / seconds


def cpu_sample(wl, seconds_budget=20.0):
    """Oracle (A+B)X and (A-B)X products on the same molecule, seeded orbitals."""
    from oracle import excited, nddo
    params = molgen.make_params(0)
    Z, xyz = wl["gen"](0)
    mol = nddo.Molecule(Z, xyz, params)
    t0 = time.perf_counter()
    ints = nddo.Integrals(mol)
    t_ints = time.perf_counter() - t0
    Cm = molgen.orthonormal_matrix(11, mol.nao)
    eps = np.sort(np.random.default_rng(3).uniform(-40.0, 10.0, mol.nao))
    X = molgen.trial_vectors(5, 1, mol.nocc, mol.nvir)
    n = 0
    t0 = time.perf_counter()
    while True:
        excited.apply_kind(mol, ints, Cm, eps, mol.nocc, X, "ApB")
        excited.apply_kind(mol, ints, Cm, eps, mol.nocc, X, "AmB")
        n += 1
        if time.perf_counter() - t0 > seconds_budget or n >= 64:
            break
    per_vector = (time.perf_counter() - t0) / n
    return per_vector, n, t_ints


def oracle_products(workload, method):
    """Trial-vector count of the oracle's own Davidson run stored in
    tests/golden (written by the oracle only): this workload's if stored, else
    the medium molecule's."""
    for name in (workload, "medium"):
        path = os.path.join(ROOT, "tests", "golden", f"{name}.json")
        if os.path.exists(path):
            with open(path) as f:
                g = json.load(f)
            if method in g.get("roots", {}):
                return int(g["roots"][method]["products"]), f"oracle Davidson product count, {name} molecule"
    return 200, "no stored oracle run: 200 products"


def run_reference(args, wl):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    # each step: the oracle's products for the number of trial vectors the
    # oracle's own Davidson needs on this workload (its stored run of the same
    # molecule and method, else of the medium molecule), timed on a sample
    per_vector, n, _ = cpu_sample(wl, seconds_budget=max(5.0, 20.0 / max(args.steps, 1)))
    products_per_solve, source = oracle_products(args.workload, "RPA" if wl["method"] == "TDHF" else "CIS")
    step_s = per_vector * products_per_solve
    value = wl["nroots"] / step_s
    line = dict(impl="reference", metric=METRIC, value=value, unit="roots/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=step_s * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload, desc=wl["desc"]),
                cpu_baseline=dict(kind="oracle", value=value, unit="roots/s", cores=os.cpu_count(),
                                  sample=f"{n} oracle (A+B)X,(A-B)X products on the {args.workload} molecule "
                                         f"(seeded orbitals), {per_vector:.3f} s each, x{products_per_solve} "
                                         f"products per solve ({source})"),
                e2e=dict(value=value, unit="roots/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def timed(torch, stream, fn):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / 1e3


def run_many(args, wl):
    """Batched workloads: one step = one batched solve of every molecule."""
    import torch
    from paper_2505_24807_gb300 import xs
    torch.cuda.set_device(0)
    params = molgen.make_params(0)
    stream = torch.cuda.Stream(device=0)
    ctx = xs.xs_create(0, stream.cuda_stream)
    xs.xs_set_params(ctx, molgen.params_table(params))
    method = xs.XS_TDHF if wl["method"] == "TDHF" else xs.XS_CIS
    K = wl["nroots"]
    extra = {}
    t0 = time.perf_counter()
    if args.workload == "batch":
        mols = [molgen.config_batch(s) for s in range(wl["n_mol"])]
        guess = xs.XS_GUESS_PLAIN
    elif os.path.exists(os.path.join(ROOT, "paper_2505_24807_gb300", "guess_weights.f32")):
        # the committed network (paper_2505_24807_gb300/train_guess.py), seeds disjoint from the test set
        base = os.path.join(ROOT, "paper_2505_24807_gb300", "guess_weights")
        xs.xs_mlp_set_weights(ctx, np.fromfile(base + ".f32", dtype=np.float32))
        if os.path.exists(base + ".json"):
            with open(base + ".json") as f:
                extra["training"] = json.load(f)
        mols = [molgen.config_sized(9000 + s, 20 + (s * 4099) % 281) for s in range(wl["n_test"])]
        guess = xs.XS_GUESS_LEARNED
    else:
        train = [molgen.config_sized(1000 + s, 20 + (s * 7919) % 101) for s in range(wl["n_train"])]
        mols = [molgen.config_sized(9000 + s, 20 + (s * 4099) % 281) for s in range(wl["n_test"])]
        xs.xs_ground_state(ctx, train)
        xs.xs_excited(ctx, method=method, nroots=K, tol=1e-6, batched=1, n_mol=len(train))
        feats, targs = [], []
        for i in range(len(train)):
            F, pairs = xs.xs_mlp_features(ctx, i, 2048)
            feats.append(F)
            targs.append(xs.xs_mlp_targets(ctx, i, pairs))
        F = np.concatenate(feats)
        T = np.concatenate(targs)
        perm = np.random.default_rng(0).permutation(len(F))
        xs.xs_mlp_init(ctx, seed=1)
        tt = time.perf_counter()
        loss = xs.xs_mlp_train(ctx, F[perm], T[perm], epochs=60, batch=4096, lr=2e-3)
        extra["training"] = dict(molecules=len(train), samples=int(len(F)), epochs=60,
                                 loss_first=float(loss[0]), loss_last=float(loss[-1]),
                                 seconds=round(time.perf_counter() - tt, 3))
        guess = xs.XS_GUESS_LEARNED
    gs = xs.xs_ground_state(ctx, mols)
    setup_s = time.perf_counter() - t0
    nm = len(mols)

    def solve(g=guess, batched=1, prec=xs.XS_MIXED):
        return xs.xs_excited(ctx, method=method, nroots=K, tol=wl["tol"], precision=prec, guess=g, batched=batched,
                             n_mol=nm)

    for _ in range(args.warmup):
        solve()
    clocks = ClockSampler(0)
    clocks.start()
    res, sec = None, 0.0
    for _ in range(args.steps):
        res, dt = timed(torch, stream, solve)
        sec += dt
    clk = clocks.stop()
    value = nm * K * args.steps / sec
    seq, seq_s = timed(torch, stream, lambda: solve(batched=0))
    extra["one_at_a_time"] = dict(value=nm * K / seq_s, unit="roots/s", seconds=seq_s)
    if args.workload == "learned":
        plain, plain_s = timed(torch, stream, lambda: solve(g=xs.XS_GUESS_PLAIN))
        extra["plain_guess"] = dict(value=nm * K / plain_s, unit="roots/s", seconds=plain_s,
                                    mean_iterations=float(np.mean(plain["iters"])),
                                    max_abs_domega_vs_learned_eV=float(np.abs(plain["omega"] - res["omega"]).max()))
        extra["learned_guess"] = dict(mean_iterations=float(np.mean(res["iters"])), fallback=res["info"]["fallback"])
    if not args.no_fp64_baseline:
        r64, s64 = timed(torch, stream, lambda: solve(g=xs.XS_GUESS_PLAIN, prec=xs.XS_FP64))
        extra["fp64_gpu"] = dict(value=nm * K / s64, unit="roots/s", seconds=s64,
                                 max_abs_domega_vs_chosen_eV=float(np.abs(r64["omega"] - res["omega"]).max()),
                                 speedup_of_chosen_form=value / (nm * K / s64))
    line = dict(metric=METRIC.replace("TDHF", wl["method"]), value=value, unit="roots/s", n_gpus=1,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * sec / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32+f64", data="synthetic",
                config=dict(workload=args.workload, desc=wl["desc"], molecules=nm, precision="mixed",
                            setup_seconds=round(setup_s, 2), scf_iterations_max=gs["max_scf_iter_used"]),
                iterations_mean=float(np.mean(res["iters"])), converged=int(res["info"]["converged"]),
                clocks=clk, **extra)
    print(json.dumps(line), flush=True)
    xs.xs_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="xs", choices=["xs", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--guess", default="auto", choices=["auto", "plain", "learned"],
                    help="learned: the network in paper_2505_24807_gb300/guess_weights.f32 (auto: if present)")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.workload in ("batch", "learned"):
        return run_many(args, wl)

    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    from paper_2505_24807_gb300 import xs

    params = molgen.make_params(0)
    Z, xyz = wl["gen"](rank_molecule_seed(rank))   # rank r solves its own seeded molecule
    stream = torch.cuda.Stream(device=local)   # the library launches on this stream
    ctx = xs.xs_create(local, stream.cuda_stream)
    xs.xs_set_params(ctx, molgen.params_table(params))
    t0 = time.perf_counter()
    gs = xs.xs_ground_state(ctx, [(Z, xyz)])
    setup_s = time.perf_counter() - t0
    nao, nocc, _ = xs.xs_get_sizes(ctx, 0)
    method = xs.XS_TDHF if wl["method"] == "TDHF" else xs.XS_CIS
    prec = xs.XS_MIXED if args.precision == "mixed" else xs.XS_FP64
    K = wl["nroots"]
    wpath = os.path.join(ROOT, "paper_2505_24807_gb300", "guess_weights.f32")
    guess = xs.XS_GUESS_PLAIN
    if args.guess == "learned" or (args.guess == "auto" and os.path.exists(wpath)):
        xs.xs_mlp_set_weights(ctx, np.fromfile(wpath, dtype=np.float32))
        guess = xs.XS_GUESS_LEARNED

    def solve(p=prec, g=None):
        return xs.xs_excited(ctx, method=method, nroots=K, tol=wl["tol"], precision=p,
                             guess=guess if g is None else g)

    for _ in range(args.warmup):
        solve()
    # timed region: K solves bracketed by barrier + synchronize, CUDA events on the stream
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    xs.xs_profile(ctx, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(solve())
    e1.record(stream)
    torch.cuda.synchronize()
    prof = xs.xs_profile_read(ctx)
    xs.xs_profile(ctx, False)
    clk = clocks.stop()
    dev_ms = max_over_ranks(e0.elapsed_time(e1), "cuda")
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = dev_ms / args.steps
    value = throughput(world, K, args.steps, dev_ms / 1e3)
    last = results[-1]

    # end to end through the public API with host buffers: upload C and eps from
    # pinned host memory, solve, read the roots back
    Cm, eps = xs.xs_get_orbitals(ctx, 0)
    Cp = torch.from_numpy(Cm).pin_memory().numpy()
    Ep = torch.from_numpy(eps).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xs.xs_set_orbitals(ctx, 0, Cp, Ep)
        solve()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, "cuda")
    e2e = dict(value=throughput(world, K, 1, e2e_s), unit="roots/s", h2d_bytes_per_step=8 * (nao * nao + nao),
               d2h_bytes_per_step=8 * 3 * K + 4)

    # plain float64 GPU Davidson on the same molecule (the metric's denominator)
    fp64 = None
    if not args.no_fp64_baseline and prec == xs.XS_MIXED:
        # a short untimed float64 solve first: the float64 path's GEMM shape
        # classes are autotuned on first use, as the mixed path's were in warm-up
        xs.xs_excited(ctx, method=method, nroots=K, tol=wl["tol"], precision=xs.XS_FP64,
                      guess=xs.XS_GUESS_PLAIN, max_iter=25, allow=(xs.XS_ENOCONV,))
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        r64 = solve(xs.XS_FP64, xs.XS_GUESS_PLAIN)
        f1.record(stream)
        torch.cuda.synchronize()
        s64 = f0.elapsed_time(f1) / 1e3
        err = float(np.abs(last["omega"][0] - r64["omega"][0]).max())
        fp64 = dict(value=K / s64, unit="roots/s", seconds=s64, iterations=int(r64["info"]["iterations"]),
                    products=int(r64["info"]["products"]), max_abs_domega_vs_mixed_eV=err,
                    speedup_of_chosen_form=(K / (ms_per_step / 1e3)) / (K / s64))

    # parity against the oracle's stored roots for this workload, when present
    oracle_err = None
    gpath = os.path.join(ROOT, "tests", "golden", f"{args.workload}.json")
    if os.path.exists(gpath) and rank == 0:
        with open(gpath) as f:
            g = json.load(f)
        key = "RPA" if wl["method"] == "TDHF" else "CIS"
        if key in g["roots"]:
            ref = np.array(g["roots"][key]["omega"])
            oracle_err = float(np.abs(last["omega"][0][: len(ref)] - ref).max())

    # roofline of the dominant kernel, from the library's CUDA-event profile
    pk = peaks()
    kernels = {k: v for k, v in prof.items()
               if k != "all_launches" and not k.startswith("host:") and v["launches"] > 0}
    # host wall time of the solver's phases (setup, iteration loop, time spent
    # waiting for the device at the per-iteration read-back), per step
    host_phases = {k[5:]: round(v["ms"] / args.steps, 2) for k, v in prof.items() if k.startswith("host:")}
    top_name = max(kernels, key=lambda k: kernels[k]["ms"]) if kernels else None
    roof = kernel_roofline(top_name, kernels[top_name], pk) if top_name else None
    # the A.X product itself: its transforms (tensor cores) and G build (HBM)
    ax = {k: kernel_roofline(k, kernels[k], pk) for k in kernels if k.startswith(("tc_gemm", "gbuild"))}
    def _rate(v):
        sec = v["ms"] / 1e3
        out = {}
        if v["bytes"] > 0:
            out["GBps"] = round(v["bytes"] / sec / 1e9, 1)
        if v["flops"] > 0:
            out["TFLOPps"] = round(v["flops"] / sec / 1e12, 2)
        return out

    kernel_table = {k: dict(launches=v["launches"], ms=round(v["ms"], 3),
                            share=round(v["ms"] / max(sum(x["ms"] for x in kernels.values()), 1e-9), 4), **_rate(v))
                    for k, v in sorted(kernels.items(), key=lambda kv: -kv[1]["ms"])}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        per_vector, n, _ = cpu_sample(wl, seconds_budget=20.0)
        prods = int(last["info"]["products"])
        cpu_value = K / (per_vector * max(prods, 1))
        cpu = dict(value=cpu_value, unit="roots/s", cores=os.cpu_count(), kind="oracle",
                   sample=f"{n} oracle (A+B)X,(A-B)X product pairs on the {args.workload} molecule with seeded "
                          f"orbitals ({per_vector:.3f} s each) x {prods} products of the GPU solve")

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit="roots/s", n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=ms_per_step, higher_is_better=True, scaling="weak",
                    vs_baseline=None,
                    dtype="f32+f64" if prec == xs.XS_MIXED else "f64",
                    data="synthetic",
                    config=dict(workload=args.workload, desc=wl["desc"], precision=args.precision,
                                guess="learned" if guess == xs.XS_GUESS_LEARNED else "plain",
                                nao=nao, nocc=nocc, tol_eV=wl["tol"], l2="working set > L2 (V, (A+B)V, (A-B)V)",
                                setup_seconds=round(setup_s, 3), scf_iterations=gs["max_scf_iter_used"]),
                    iterations=int(last["info"]["iterations"]), products=int(last["info"]["products"]),
                    converged=int(last["info"]["converged"]),
                    max_abs_err_vs_oracle_eV=oracle_err,
                    roofline=roof, ax_product=ax, kernels=kernel_table, host_ms_per_step=host_phases,
                    cpu_baseline=cpu, e2e=e2e,
                    gpu_launches=int(prof.get("all_launches", {}).get("launches", 0)),
                    clocks=clk, fp64_gpu=fp64)
        print(json.dumps(line), flush=True)
    xs.xs_destroy(ctx)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
