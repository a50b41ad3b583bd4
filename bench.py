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


# SIMT peaks from unit counts and the maximum clock: 152 SMs x 128 float32
# lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s; float64: NVIDIA's 1.25 TFLOP/s
# for the part (a warp-wide DFMA holds a sub-partition's float64 unit for 64
# cycles: 152 x 4 x 32 / 64 x 2 x 2.07 GHz = 1.26 TFLOP/s).
FP64_SIMT_TFLOPS = 1.25
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# DRAM traffic per launch of the dominant kernels (dram__bytes_read.sum +
# dram__bytes_write.sum, mean over the captured launches of one solve of the
# workload), from the ncu summaries named in "source"; a kernel absent here
# (or changed since its capture) reports traffic null.
TRAFFIC = {
    ("tc_gemm_tf32x3", "large"): dict(bytes_per_launch=7.228e8, source="profiles/tc_gemm_tf32x3_large.md"),
    ("gbuild_assemble_f32", "large"): dict(bytes_per_launch=1.2246e9, source="profiles/tc_gemm_tf32x3_large.md"),
}


def traffic_of(name, workload):
    t = TRAFFIC.get((name, workload))
    return (t["bytes_per_launch"], t["source"]) if t else (None, None)


def kernel_roofline(name, t, pk, workload=None):
    """Achieved rate of one profiled kernel family against its bound: digit
    products, digit splits and the G build stream HBM (algorithmic bytes);
    tensor-core GEMMs against the TF32 peak; SIMT kernels against the float64
    or float32 pipe."""
    per_launch_s = t["ms"] / 1e3 / t["launches"]
    if name.startswith(("oz_", "gbuild")) and t["bytes"] > 0:
        ach = t["bytes"] / t["launches"] / per_launch_s / 1e9
        traffic, tsrc = traffic_of(name, workload)
        return dict(kernel=name, bound="hbm", achieved=ach, peak=pk["hbm_gbs"], unit="GB/s",
                    frac=ach / pk["hbm_gbs"], traffic=traffic, traffic_source=tsrc,
                    peak_source=pk["source"] + " hbm_gbs",
                    bytes_per_launch=t["bytes"] / t["launches"], ms_per_launch=per_launch_s * 1e3)
    ach = t["flops"] / t["launches"] / per_launch_s / 1e12
    if name.startswith("tc_"):
        peak, src, bound = pk["bf16_sustained"] / 2.0, pk["source"] + " bf16 sustained x 1/2 (tf32)", "tensor"
    elif "f64" in name:
        peak, src, bound = FP64_SIMT_TFLOPS, "float64 SIMT, nominal 1.25 TFLOP/s", "alu"
    else:
        peak, src, bound = FP32_SIMT_TFLOPS, "float32 SIMT, 152 SMs x 128 lanes x 2 x 2.07 GHz", "alu"
    traffic, tsrc = traffic_of(name, workload)
    return dict(kernel=name, bound=bound, achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak, traffic=traffic,
                traffic_source=tsrc,
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


def blas_threads():
    """Threads of the BLAS that numpy uses (the oracle's products run there)."""
    try:
        from threadpoolctl import threadpool_info
        n = [d["num_threads"] for d in threadpool_info() if d.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except ImportError:
        pass
    import ctypes
    import glob
    libdir = os.path.join(os.path.dirname(np.__file__), "..", "numpy.libs")
    for path in glob.glob(os.path.join(libdir, "*openblas*")):
        lib = ctypes.CDLL(path)
        for fn in ("scipy_openblas_get_num_threads64_", "openblas_get_num_threads64_", "openblas_get_num_threads"):
            if hasattr(lib, fn):
                return int(getattr(lib, fn)())
    return None


class OracleSample:
    """The oracle's (A+B)X and (A-B)X products of one trial vector on the
    workload's molecule with seeded orthonormal orbitals: the unit of work of
    an oracle Davidson solve (its stored run counts these vectors)."""

    def __init__(self, wl):
        from oracle import excited, nddo
        self.excited = excited
        params = molgen.make_params(0)
        Z, xyz = wl["gen"](0)
        self.mol = nddo.Molecule(Z, xyz, params)
        self.ints = nddo.Integrals(self.mol)
        self.C = molgen.orthonormal_matrix(11, self.mol.nao)
        self.eps = np.sort(np.random.default_rng(3).uniform(-40.0, 10.0, self.mol.nao))
        self.X = molgen.trial_vectors(5, 1, self.mol.nocc, self.mol.nvir)

    def product(self):
        m = self.mol
        t0 = time.perf_counter()
        self.excited.apply_kind(m, self.ints, self.C, self.eps, m.nocc, self.X, "ApB")
        self.excited.apply_kind(m, self.ints, self.C, self.eps, m.nocc, self.X, "AmB")
        return time.perf_counter() - t0


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


def cpu_baseline_leg(wl, workload, seconds_budget=20.0):
    """Oracle roots/s on the host cores, extrapolated from a bounded sample:
    products timed for ~seconds_budget, times the oracle's own product count
    per solve (its stored Davidson run of this molecule)."""
    smp = OracleSample(wl)
    times = []
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds_budget and len(times) < 64:
        times.append(smp.product())
    per_vector = float(np.mean(times))
    prods, source = oracle_products(workload, "RPA" if wl["method"] == "TDHF" else "CIS")
    value = wl["nroots"] / (per_vector * prods)
    return dict(value=value, unit="roots/s", cores=os.cpu_count(), blas_threads=blas_threads(), kind="oracle",
                extrapolated=True, sampled_products=len(times), products_per_solve=prods,
                sample=f"{len(times)} oracle (A+B)X,(A-B)X trial-vector products on the {workload} molecule "
                       f"(seeded orbitals), {per_vector:.3f} s each, x {prods} products per solve ({source})")


def run_reference(args, wl):
    """The oracle as the reference arm: every step is one bounded sample of the
    workload -- the oracle's (A+B)X and (A-B)X products of one trial vector --
    timed on the host cores; roots/s extrapolates to a whole solve with the
    oracle's own Davidson product count."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    smp = OracleSample(wl)
    for _ in range(args.warmup):
        smp.product()
    step_s = [smp.product() for _ in range(max(args.steps, 1))]
    per_vector = float(np.mean(step_s))
    prods, source = oracle_products(args.workload, "RPA" if wl["method"] == "TDHF" else "CIS")
    value = wl["nroots"] / (per_vector * prods)
    sample = (f"each step: one trial vector's oracle (A+B)X and (A-B)X products on the {args.workload} molecule "
              f"(seeded orbitals), {per_vector:.3f} s; roots/s = {wl['nroots']} roots / ({prods} products per "
              f"solve ({source}) x the mean step)")
    line = dict(impl="reference", metric=METRIC, value=value, unit="roots/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=per_vector * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", extrapolated=True,
                config=dict(workload=args.workload, desc=wl["desc"], step="one oracle product pair"),
                cpu_baseline=dict(kind="oracle", value=value, unit="roots/s", cores=os.cpu_count(),
                                  blas_threads=blas_threads(), extrapolated=True, products_per_solve=prods,
                                  sample=sample),
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
    xs.xs_profile(ctx, 2)   # launch counts only
    res, sec = None, 0.0
    for _ in range(args.steps):
        res, dt = timed(torch, stream, solve)
        sec += dt
    counts = xs.xs_profile_read(ctx)
    xs.xs_profile(ctx, 0)
    clk = clocks.stop()
    value = nm * K * args.steps / sec
    extra["graph_launches_per_step"] = int(res["info"]["graph_launches"])
    extra["iterations_max"] = int(res["info"]["iterations"])
    extra["gpu_launches"] = int(counts.get("all_launches", {}).get("launches", 0))
    extra["host_ms_per_step"] = {k[5:]: round(v["ms"] / args.steps, 2) for k, v in counts.items()
                                 if k.startswith("host:")}
    conc, conc_s = timed(torch, stream, lambda: solve(batched=2))
    extra["concurrent_streams"] = dict(value=nm * K / conc_s, unit="roots/s", seconds=conc_s,
                                       max_abs_domega_vs_chosen_eV=float(np.abs(conc["omega"] - res["omega"]).max()))
    seq, seq_s = timed(torch, stream, lambda: solve(batched=0))
    extra["one_at_a_time"] = dict(value=nm * K / seq_s, unit="roots/s", seconds=seq_s)
    if args.workload == "learned":
        plain, plain_s = timed(torch, stream, lambda: solve(g=xs.XS_GUESS_PLAIN))
        extra["plain_guess"] = dict(value=nm * K / plain_s, unit="roots/s", seconds=plain_s,
                                    mean_iterations=float(np.mean(plain["iters"])),
                                    max_abs_domega_vs_learned_eV=float(np.abs(plain["omega"] - res["omega"]).max()))
        extra["learned_guess"] = dict(mean_iterations=float(np.mean(res["iters"])), fallback=res["info"]["fallback"])
    if not args.no_fp64_baseline:
        # plain float64 Davidson, one molecule after another (the per-molecule
        # float64 path), plain guess, at the residual threshold the chosen form applied
        tol_same = float(res["info"]["tol_used"])

        def solve64(batched):
            return xs.xs_excited(ctx, method=method, nroots=K, tol=tol_same, precision=xs.XS_FP64,
                                 guess=xs.XS_GUESS_PLAIN, batched=batched, n_mol=nm)

        r64, s64 = timed(torch, stream, lambda: solve64(0))
        extra["fp64_gpu"] = dict(value=nm * K / s64, unit="roots/s", seconds=s64,
                                 stopping_rule=f"residual <= {tol_same:g} eV (the chosen form's)",
                                 max_abs_domega_vs_chosen_eV=float(np.abs(r64["omega"] - res["omega"]).max()),
                                 speedup_of_chosen_form=value / (nm * K / s64))
        b64, bs64 = timed(torch, stream, lambda: solve64(1))
        extra["fp64_lockstep"] = dict(value=nm * K / bs64, unit="roots/s", seconds=bs64,
                                      max_abs_domega_vs_fp64_gpu_eV=float(np.abs(b64["omega"] - r64["omega"]).max()))
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
    # timed region: K solves bracketed by barrier + synchronize, CUDA events on
    # the stream; the library only counts its launches here (no per-kernel events)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    xs.xs_profile(ctx, 2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(solve())
    e1.record(stream)
    torch.cuda.synchronize()
    counts = xs.xs_profile_read(ctx)
    xs.xs_profile(ctx, 0)
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

    # one more solve with per-kernel CUDA events (outside the timed region):
    # the kernel table and the rooflines
    xs.xs_profile(ctx, 1)
    solve()
    prof = xs.xs_profile_read(ctx)
    xs.xs_profile(ctx, 0)

    def timed_solve(p, g, tol):
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        f0.record(stream)
        r = xs.xs_excited(ctx, method=method, nroots=K, tol=tol, precision=p, guess=g)
        f1.record(stream)
        torch.cuda.synchronize()
        return r, f0.elapsed_time(f1) / 1e3

    def record(r, sec):
        return dict(value=K / sec, unit="roots/s", seconds=sec, iterations=int(r["info"]["iterations"]),
                    products=int(r["info"]["products"]), tol_used_eV=r["info"]["tol_used"],
                    converged=int(r["info"]["converged"]))

    # the same mixed solve with the plain guess: the learned guess's own gain
    plain_mixed = None
    if prec == xs.XS_MIXED and guess == xs.XS_GUESS_LEARNED and not args.no_fp64_baseline:
        rp, sp = timed_solve(prec, xs.XS_GUESS_PLAIN, wl["tol"])
        plain_mixed = record(rp, sp)
        plain_mixed["roots"] = rp

    # plain float64 GPU Davidson on the same molecule (the metric's
    # denominator), plain guess, stopping at the residual threshold the mixed
    # solve applied (same stopping rule), and at the requested tolerance
    fp64 = None
    if not args.no_fp64_baseline and prec == xs.XS_MIXED:
        # a short untimed float64 solve first: the float64 path's GEMM shape
        # classes are autotuned on first use, as the mixed path's were in warm-up
        xs.xs_excited(ctx, method=method, nroots=K, tol=wl["tol"], precision=xs.XS_FP64,
                      guess=xs.XS_GUESS_PLAIN, max_iter=25, allow=(xs.XS_ENOCONV,))
        tol_same = float(last["info"]["tol_used"])
        r64, s64 = timed_solve(xs.XS_FP64, xs.XS_GUESS_PLAIN, tol_same)
        fp64 = record(r64, s64)
        fp64["roots"] = r64
        fp64["stopping_rule"] = f"residual <= {tol_same:g} eV (the mixed solve's)"
        fp64["speedup_of_chosen_form"] = (K / (ms_per_step / 1e3)) / fp64["value"]
        r64t, s64t = timed_solve(xs.XS_FP64, xs.XS_GUESS_PLAIN, wl["tol"])
        fp64["at_requested_tol"] = record(r64t, s64t)
        fp64["at_requested_tol"]["roots"] = r64t

    # per-root errors against the oracle's stored roots for this workload
    golden = None
    gpath = os.path.join(ROOT, "tests", "golden", f"{args.workload}.json")
    if os.path.exists(gpath) and rank == 0:
        with open(gpath) as f:
            g = json.load(f)
        key = "RPA" if wl["method"] == "TDHF" else "CIS"
        if key in g["roots"]:
            golden = (np.array(g["roots"][key]["omega"]), np.array(g["roots"][key]["f"]))

    def per_root(r):
        if golden is None or r is None:
            return None
        w, f = golden
        n = min(len(w), K)
        dw = np.abs(r["omega"][0][:n] - w[:n])
        df = np.abs(r["osc"][0][:n] - f[:n])
        return dict(abs_domega_eV=[float(x) for x in dw], abs_df=[float(x) for x in df],
                    max_abs_domega_eV=float(dw.max()), max_abs_df=float(df.max()))

    errors = dict(chosen=per_root(last))
    for name, rec in (("mixed_plain_guess", plain_mixed), ("fp64_gpu", fp64),
                      ("fp64_gpu_requested_tol", fp64["at_requested_tol"] if fp64 else None)):
        if rec is not None:
            errors[name] = per_root(rec.pop("roots"))
    oracle_err = errors["chosen"]["max_abs_domega_eV"] if errors["chosen"] else None

    # roofline of the dominant kernel, from the profiled solve
    pk = peaks()
    kernels = {k: v for k, v in prof.items()
               if k != "all_launches" and not k.startswith("host:") and v["launches"] > 0}
    # host wall time of the solver's phases in the timed region (setup, iteration
    # loop, time spent waiting for the device at the per-iteration read-back), per step
    host_phases = {k[5:]: round(v["ms"] / args.steps, 2) for k, v in counts.items() if k.startswith("host:")}
    top_name = max(kernels, key=lambda k: kernels[k]["ms"]) if kernels else None
    roof = kernel_roofline(top_name, kernels[top_name], pk, args.workload) if top_name else None
    # the A.X product itself: its transforms (tensor cores) and G build (HBM)
    ax = {k: kernel_roofline(k, kernels[k], pk, args.workload) for k in kernels
          if k.startswith(("tc_gemm", "gbuild", "coulomb"))}

    def _rate(v):
        sec = v["ms"] / 1e3
        out = {}
        if v["bytes"] > 0:
            out["GBps"] = round(v["bytes"] / sec / 1e9, 1)
        if v["flops"] > 0:
            out["TFLOPps"] = round(v["flops"] / sec / 1e12, 2)
        return out

    total_ms = max(sum(x["ms"] for x in kernels.values()), 1e-9)
    kernel_table = {k: dict(launches=v["launches"], ms=round(v["ms"], 3), share=round(v["ms"] / total_ms, 4),
                            **_rate(v))
                    for k, v in sorted(kernels.items(), key=lambda kv: -kv[1]["ms"])}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(wl, args.workload, seconds_budget=20.0)

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit="roots/s", n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=ms_per_step, higher_is_better=True, scaling="weak",
                    vs_baseline=None,
                    dtype="f32+f64" if prec == xs.XS_MIXED else "f64",
                    data="synthetic",
                    config=dict(workload=args.workload, desc=wl["desc"], precision=args.precision,
                                guess="learned" if guess == xs.XS_GUESS_LEARNED else "plain",
                                nao=nao, nocc=nocc, tol_eV=wl["tol"], tol_used_eV=last["info"]["tol_used"],
                                l2="inputs larger than L2 (V, (A+B)V, (A-B)V and their digit operands: ~21 GB working set)",
                                setup_seconds=round(setup_s, 3), scf_iterations=gs["max_scf_iter_used"]),
                    iterations=int(last["info"]["iterations"]), products=int(last["info"]["products"]),
                    converged=int(last["info"]["converged"]),
                    max_abs_err_vs_oracle_eV=oracle_err, errors_vs_oracle=errors,
                    roofline=roof, ax_product=ax, kernels=kernel_table,
                    kernels_note="per-kernel CUDA events from one extra untimed solve",
                    host_ms_per_step=host_phases,
                    cpu_baseline=cpu, e2e=e2e,
                    gpu_launches=int(counts.get("all_launches", {}).get("launches", 0)),
                    clocks=clk, mixed_plain_guess=plain_mixed, fp64_gpu=fp64)
        print(json.dumps(line), flush=True)
    xs.xs_destroy(ctx)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
