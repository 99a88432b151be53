#!/usr/bin/env python3
"""Throughput of the GB300 PSD-cone projection (projections/s).

Default workload (the ADMM-like process-matrix step at d = 5): a sequence of
200 projections of 625 x 625 FP64 symmetric matrices X_{k+1} = X_k +
1e-3 Sym(G_k) from X_0 = Q diag(lam) Q^T with a spectrum clustered at zero,
svec in and out (195,625 doubles each); one step = the 200 projections as
200 dependent calls of the library's C-ABI on one stream.  Other workloads:
--config single81 | precision4096 | uneven | vjp1296 | herm625.
--method poly runs the factorization-free approximate projection (the
composite matrix polynomial of the paper's outlook) on the same workload,
for the speed/accuracy comparison against the eigensolver path.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the launching stream (L2 flushed before every step by writing a 256 MB
buffer, outside the timed interval), barrier + synchronize on both sides,
max over ranks.  `e2e` repeats the step through the same C-ABI with the
inputs in pinned host memory and the host<->device copies inside the timed
region.  The dominant phase's roofline uses per-phase CUDA events recorded
by the library on the same stream during the timed steps.

The default run also measures the metric's other legs, keyed under "legs"
in the same JSON line: n = 4096 x 4 forward and n = 1296 x 8 forward + VJP,
each in FP64 and in the split precision (3 warm-up and 3 timed steps each,
with their own comparator, roofline, error against the construction and
clock record); --no-legs skips them.

--impl reference times the FP64 CPU oracle (the plain cyclic-Jacobi
implementation the tests pin) on the host cores, on a bounded sample of the
same workload.  For N > 1 (torchrun) every rank runs an independent replica
of the workload (the projection does not shard: there is no exchange step)
and `value` is the total over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_20519_gb300 import workloads as W  # noqa: E402

METRIC = "PSD projections/s (fwd, fwd+VJP) at n=625/4096 vs plain FP64 GPU path at stated error"
# FP64 ALU peak from unit counts and clock: 152 SMs x 2 FP64 FMA per clock per SM
# x 2 flops x 2.07 GHz (the nominal 1.25 TFLOP/s of the part)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
FP64_PEAK_NOTE = "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="admm625",
                   choices=["admm625", "single81", "precision4096", "uneven", "vjp1296", "herm625", "mixing",
                            "scs625", "scs625kron"])
    p.add_argument("--band", type=int, default=0)
    p.add_argument("--method", default="eig", choices=["eig", "poly"],
                   help="eig: projection by eigendecomposition; poly: factorization-free composite polynomial")
    p.add_argument("--poly-lo", type=float, default=1e-9,
                   help="poly: relative eigenvalue resolution lo (eigenvalues above lo * ||X||_F are thresholded)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "split"],
                   help="fp64: FP64 throughout; split: split-TF32 tensor-core contractions")
    p.add_argument("--no-comparator", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true",
                   help="skip the library's autotuner (launch shapes by default heuristics)")
    p.add_argument("--no-legs", action="store_true",
                   help="default run: skip the metric's other legs (n = 4096 forward, n = 1296 forward + VJP)")
    p.add_argument("--calls", type=int, default=0,
                   help="use only the first N calls of the workload per step (profiling runs)")
    return p.parse_args()


# ---------------------------------------------------------------- workloads
class Workload:
    """Host arrays: xs (list of svec inputs, one per call), sides per call,
    units per step (projections), algorithmic counts."""

    def __init__(self, name: str, calls: int = 0):
        self.name = name
        self.vjp = False
        self.herm = False
        self.mixing = False
        self.scs = None
        if name == "admm625":
            seq, Q, lam = W.admm_sequence()
            self.calls = [(x, [625]) for x in seq]
            self.desc = "ADMM-like sequence of 200 projections, n=625 (d=5), 200 dependent calls"
            self.exact0 = (Q, lam)
        elif name == "single81":
            x, Q, lam = W.single_projection()
            self.calls = [(x, [81])] * 100
            self.desc = "single projection n=81 (d=3), 100 calls per step"
            self.exact0 = (Q, lam)
        elif name == "precision4096":
            b = W.precision_batch()
            self.calls = [(b.x, list(b.sides))]
            self.desc = "4 matrices n=4096 (d=8), precision stress spectrum, one batched call"
            self.exact0 = (b.extra["Q"][0], b.extra["lam"][0])
        elif name == "uneven":
            b = W.uneven_batch()
            self.calls = [(b.x, list(b.sides))]
            self.desc = "960 uneven cones (64 restarts x {2 x sides 4..64 + one 625/1296}) in one call"
            self.exact0 = None
        elif name == "mixing":
            # App. C / D positivity post-processing on the uneven batch: the two
            # outcome blocks of each instrument side d^2 form a group with
            # nu = 1/(2 d) (n_a = 2, d_Ao = d); each process block is a group of
            # its own with nu = gamma = 1/n; eps = 1e-16 as in the paper
            b = W.uneven_batch()
            self.calls = [(b.x, list(b.sides))]
            groups, nu, i = [0], [], 0
            sides = [int(v) for v in b.sides]
            while i < len(sides):
                if i + 1 < len(sides) and sides[i + 1] == sides[i] and sides[i] <= 64:
                    groups.append(i + 2)
                    nu.append(1.0 / (2.0 * round(sides[i] ** 0.5)))
                    i += 2
                else:
                    groups.append(i + 1)
                    nu.append(1.0 / sides[i])
                    i += 1
            self.groups, self.nu, self.eps = groups, nu, 1e-16
            self.mixing = True
            self.desc = ("positivity post-processing (lambda_min + mixing with nu * identity) of 960 uneven cones "
                         "(64 restarts x {2 outcome blocks of sides 4..64 + one 625/1296 process block}), one call")
            self.exact0 = None
        elif name == "scs625":
            # App. D.1 SCS iterations around the projection: one PSD cone of side
            # 625 (m = 195,625), k = 1000 parameters (orthonormal A), 10 iterations
            # per step from SCS's initial iterates
            At, b, c, u0, v0 = W.scs_problem()
            self.calls = [(u0, [625])]
            self.scs = ("dense", At, b, c, u0, v0)
            self.iters = 10
            self.desc = ("10 SCS iterations (closed-form affine step with A^T A = I, PSD projection of the "
                         "n = 625 cone, dual update), m = 195,625, k = 1000")
            self.exact0 = None
        elif name == "scs625kron":
            # the same iterations at the process-matrix step's real size: A applied
            # as contractions over four local bases of side 5 (App. D.2), the
            # 14,805 coefficients of the real process subspace (App. B)
            bases, index, b, c, u0, v0 = W.scs_kron_problem()
            self.calls = [(u0, [625])]
            self.scs = ("kron", bases, index, b, c, u0, v0)
            self.iters = 10
            self.desc = ("10 SCS iterations, process-matrix step at d = 5 (n = 625, m = 195,625): A applied as "
                         "contractions over four real Gell-Mann-type local bases, k = 14,805 (real process subspace)")
            self.exact0 = None
        elif name == "herm625":
            seq, U, lam = W.herm_admm_sequence()
            self.calls = [(x, [625]) for x in seq]
            self.herm = True
            self.desc = "ADMM-like sequence of 50 complex Hermitian projections, n=625 (d=5), 50 dependent calls"
            self.exact0 = (U, lam)
        elif name == "vjp1296":
            b = W.vjp_batch()
            self.calls = [(b.x, list(b.sides))]
            self.g = b.extra["g"]
            self.vjp = True
            self.desc = "forward + Daleckii-Krein VJP, 8 matrices n=1296 (d=6), +-1e-9 clusters"
            self.exact0 = (b.extra["Q"][0], b.extra["lam"][0])
        self.svec_len = (lambda n: n * n) if self.herm else (lambda n: n * (n + 1) // 2)
        if calls:
            self.calls = self.calls[:calls]
            self.desc += f" (first {calls} call(s) only)"
        self.units = sum(len(s) for _, s in self.calls) if self.scs is None else self.iters
        self.bytes_in = sum(x.nbytes for x, _ in self.calls) + (self.g.nbytes if self.vjp else 0)
        self.bytes_out = sum(x.nbytes for x, _ in self.calls) * (2 if self.vjp else 1)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def phase_kernels(phase: str, n: int, band: int) -> str:
    """The kernel(s) a traced phase consists of, for the path a side-n cone takes."""
    one_stage = band == 1 or (band == 0 and n <= 6144)  # the library's automatic route
    return {
        "unpack": "unpack_kernel",
        "dense_to_band": "sytrd1_kernel" if one_stage else "panel_kernel + grouped GEMMs",
        "band_to_tridiag": "tridiag_extract_kernel" if one_stage else "bulge_kernel",
        "tridiag_dc": "divide-and-conquer kernels + grouped GEMMs",
        "backtransform_2": "backtr2_kernel",
        "backtransform_1": ("larft1_kernel + bt1_kernel" if one_stage else "grouped GEMMs"),
        "reconstruct": "recon_kernel",
        "derivative": "grouped GEMMs + loewner_scale_kernel",
    }.get(phase, phase)


def algorithmic_flops(phase: str, n: int, k: int, b: int, kbt: int | None = None) -> float:
    """Algorithmic FP64 flops of one cone for a phase: k = eigenpairs of the
    route's side (min(k+, k-)), kbt = columns back-transformed (k for the
    projection, n when the derivative needs all pairs), b = band width."""
    kbt = k if kbt is None else kbt
    if phase == "dense_to_band":
        return 4.0 / 3.0 * n ** 3
    if phase == "band_to_tridiag":
        return 6.0 * b * n * n
    if phase == "tridiag_dc":
        return 4.0 / 3.0 * n ** 3
    if phase in ("backtransform_2", "backtransform_1"):
        return 2.0 * n * n * kbt
    if phase == "reconstruct":
        return 1.0 * n * n * k
    if phase == "derivative":
        return 8.0 * k * n * n
    return 0.0


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_value(wl: Workload, budget_s: float = 12.0, poly_lo: float | None = None):
    """Oracle projections/s on a bounded sample of the workload (host cores);
    with poly_lo, the oracle of the factorization-free composite instead."""
    import oracle
    from oracle import poly as oracle_poly
    oracle.build()
    done, t0 = 0, time.perf_counter()
    sample = []
    for x, sides in wl.calls:
        offs = np.zeros(len(sides) + 1, dtype=np.int64)
        np.cumsum([wl.svec_len(s) for s in sides], out=offs[1:])
        if wl.scs is not None:
            from oracle import scs as oracle_scs
            kind, *prob = wl.scs
            uu, vv = prob[-2], prob[-1]
            while time.perf_counter() - t0 <= budget_s and done < wl.iters:
                if kind == "dense":
                    At, b, c = prob[:3]
                    uu, vv = oracle_scs.iterate(At.T, b, c, [0, len(b)], uu, vv, 1)
                else:
                    bases, index, b, c = prob[:4]
                    uu, vv = oracle_scs.iterate_kron(bases, index, b, c, [0, len(b)], uu, vv, 1)
                done += 1
                sample.append(625)
            break
        if wl.mixing:
            from oracle import mixing as oracle_mixing
            for i in range(len(sides)):
                oracle_mixing.lambda_min(x[offs[i]:offs[i + 1]])
                done += 1
                sample.append(sides[i])
                if time.perf_counter() - t0 > budget_s:
                    break
            break
        for i in range(len(sides)):
            xi = x[offs[i]:offs[i + 1]]
            if poly_lo is not None:
                oracle_poly.proj_poly(xi, poly_lo)
            elif wl.herm:
                oracle.herm_proj(xi)
            elif wl.vjp:
                oracle.proj(xi)
                oracle.jvp(xi, wl.g[offs[i]:offs[i + 1]])
            else:
                oracle.proj(xi)
            done += 1
            sample.append(sides[i])
            if time.perf_counter() - t0 > budget_s:
                break
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt, oracle.max_threads(), sample


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = Workload(args.config, args.calls)
    import oracle
    oracle.build()
    times = []
    info = None
    for it in range(args.warmup + args.steps):
        v, done, dt, cores, sample = oracle_value(wl, budget_s=4.0)
        if it >= args.warmup:
            times.append((done, dt))
        info = (cores, done)
    units = sum(d for d, _ in times)
    secs = sum(t for _, t in times)
    value = units / secs
    unit = ("cones/s (lambda_min + mixing)" if wl.mixing else
            "SCS iterations/s" if wl.scs is not None else "projections/s")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded PCG64), shaped like the paper's SCS iterates",
        "config": {"workload": wl.desc, "sample": "bounded: about 4 s of oracle work per step"},
        "cpu_baseline": {"value": value, "unit": unit, "cores": info[0], "kind": "oracle",
                         "sample": f"{info[1]} projections per step of the same workload"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- our arm
# The metric's other legs (forward at n = 4096, forward + VJP at n = 1296, each
# in FP64 and in the split precision), measured in the default single-GPU run
# beside the headline n = 625 workload.
LEGS = (("precision4096", "fp64"), ("precision4096", "split"), ("vjp1296", "fp64"), ("vjp1296", "split"))
LEG_STEPS, LEG_WARMUP = 3, 3


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2606_20519_gb300 import _lib as lib, build
    build.build()
    lib.load()
    env = (lib, dev, local, world, rank)
    line = measure(args, env, args.config, args.precision, args.steps, args.warmup, full=True)
    default_run = (args.config == "admm625" and args.method == "eig" and args.precision == "fp64"
                   and not args.calls and not args.band)
    if world == 1 and default_run and not args.no_legs:
        line["legs"] = {f"{cfg}_{prec}": measure(args, env, cfg, prec, min(args.steps, LEG_STEPS),
                                                 max(args.warmup, LEG_WARMUP), full=False)
                        for cfg, prec in LEGS}
    if rank == 0:
        print(json.dumps(line))
    return 0


def measure(args, env, config, precision, steps, warmup, full):
    """Time `steps` steps of one workload after `warmup` untimed ones and
    return its JSON record (None on ranks other than 0).  full=False (a leg
    of the default run): no autotuning, no e2e pass, no CPU baseline, the
    comparator on one call."""
    import torch
    lib, dev, local, world, rank = env
    prec = lib.SPLIT_TF32 if precision == "split" else lib.FP64
    opts = lib.make_opts(band=args.band, precision=prec) if (args.band or prec != lib.FP64) else None
    b_used = args.band or 16
    poly = args.method == "poly" and full
    if poly and (config in ("herm625", "vjp1296")):
        raise SystemExit("--method poly covers the real projection workloads (no Hermitian or derivative path)")

    wl = Workload(config, args.calls if full else 0)
    xs = [torch.from_numpy(x).to(dev) for x, _ in wl.calls]
    ys = [torch.empty_like(x) for x in xs]
    gs = [torch.from_numpy(wl.g).to(dev)] if wl.vjp else None
    shapes = [(lib.hshapes(s) if wl.herm else lib.shapes(s)) for _, s in wl.calls]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(x_list, y_list):
        for i in range(len(x_list)):
            offs, sides = shapes[i]
            if wl.scs is not None:
                scs_u.copy_(x_list[i])
                scs_v.copy_(scs_v0)
                scs_run(sides, offs)
                y_list[i].copy_(scs_u)
            elif poly:
                lib.proj_poly(x_list[i], sides, args.poly_lo, out=y_list[i], opts=opts, offsets=offs)
            elif wl.mixing:
                lib.mix_identity(x_list[i], sides, wl.groups, wl.nu, wl.eps, out=y_list[i], opts=opts, offsets=offs)
            elif wl.vjp:
                lib.proj_vjp(x_list[i], gs[0], sides, xbar=y_list[i], y=yb, opts=opts, offsets=offs)
            elif wl.herm:
                lib.proj_hermitian(x_list[i], sides, out=y_list[i], opts=opts, offsets=offs)
            else:
                lib.proj_batched(x_list[i], sides, out=y_list[i], opts=opts, offsets=offs)

    yb = torch.empty_like(xs[0]) if wl.vjp else None
    if wl.scs is not None:
        kind, *prob = wl.scs
        b_h, c_h, u0, v0 = prob[-4:]
        if kind == "dense":
            scs_A = torch.from_numpy(prob[0]).to(dev).t()   # m x k, column-major
        else:
            kron_bases = [torch.from_numpy(B).to(dev) for B in prob[0]]
            kron_index = torch.from_numpy(prob[1]).to(dev)
        scs_b, scs_c = torch.from_numpy(b_h).to(dev), torch.from_numpy(c_h).to(dev)
        scs_v0 = torch.from_numpy(v0).to(dev)
        scs_u, scs_v = torch.empty_like(scs_v0), torch.empty_like(scs_v0)

        def scs_run(sides, offs):
            if kind == "dense":
                lib.scs_iterate(scs_A, scs_b, scs_c, sides, scs_u, scs_v, wl.iters, opts=opts, offsets=offs)
            else:
                lib.scs_iterate_kron(kron_bases, kron_index, scs_b, scs_c, scs_u, scs_v, wl.iters, opts=opts)

    # launch shapes: the library's autotuner on the first call's input (setup, untimed)
    tuning = None
    if full and not args.no_autotune and not args.band and not wl.herm and not poly and not wl.mixing and wl.scs is None:
        tuning = lib.autotune(xs[0], shapes[0][1], opts=opts, offsets=shapes[0][0])
        if tuning["band"] >= 2:
            b_used = tuning["band"]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # correctness guard on the first call (status, error vs the construction)
    step(xs, ys)
    st = lib.status(local)
    err0 = None
    if wl.exact0 is not None:
        Q, lam = wl.exact0
        n0 = Q.shape[0]
        Pm = (Q * np.maximum(lam, 0)) @ Q.conj().T
        P = W.to_hsvec(Pm) if wl.herm else W.to_svec(Pm)
        y0 = (yb if wl.vjp else ys[0])[: wl.svec_len(n0)].cpu().numpy()
        err0 = rel(y0, P)
    # the error statement the library returns with each result (opts.stats):
    # the FP64 complementarity residual <Y, Y - X> / (||Y|| ||X||) of every cone
    # of the first call, untimed
    stats0 = None
    if not poly and not wl.herm and not wl.mixing and wl.scs is None:
        offs0, sides0 = shapes[0]
        sopts = lib.make_opts(band=args.band, precision=prec, stats=True)
        ytmp = torch.empty_like(xs[0])
        if wl.vjp:
            lib.proj_vjp(xs[0], gs[0], sides0, xbar=torch.empty_like(xs[0]), y=ytmp, opts=sopts, offsets=offs0)
        else:
            lib.proj_batched(xs[0], sides0, out=ytmp, opts=sopts, offsets=offs0)
        recs = lib.last_stats(len(sides0), local)
        comp = [abs(r["complementarity"]) for r in recs]
        stats0 = {"cones": len(recs), "max_abs_complementarity": max(comp),
                  "k_pos_first": recs[0]["k_pos"], "k_neg_first": recs[0]["k_neg"],
                  "status": max(r["status"] for r in recs)}

    for _ in range(warmup):
        step(xs, ys)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()

    def timed_steps():
        ms, launches = 0.0, 0
        for _ in range(steps):
            flush.fill_(1.0)
            barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(xs, ys)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            ms += e0.elapsed_time(e1)
            launches = lib.last_launch_count(local) * len(xs)
        return ms, launches

    # value: the steps as a user runs them (recorded launch sequences replayed)
    total_ms, launches_per_step = timed_steps()
    # roofline: the same K steps again with the library's per-phase CUDA events
    # on the launching stream (phase tracing launches kernel by kernel)
    lib.trace(True, local)
    traced_ms, _ = timed_steps()
    phases = lib.trace_read(local)
    lib.trace(False, local)
    clk = clocks.stop()
    status = lib.status(local)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / steps
    value = world * wl.units / (ms_per_step * 1e-3)

    # ---- e2e: host buffers, copies inside the timed region
    if not full:
        return None if rank != 0 else leg_record(args, wl, config, precision, steps, warmup, ms_per_step, value,
                                                  phases, tuning, b_used, clk, status, err0, launches_per_step,
                                                  traced_ms, xs, dev, stream, ys, yb, stats0)
    hx = [torch.from_numpy(x).pin_memory() for x, _ in wl.calls]
    hy = [torch.empty_like(h).pin_memory() for h in hx]
    hg = torch.from_numpy(wl.g).pin_memory() if wl.vjp else None
    dx = [torch.empty_like(x) for x in xs]
    dy = [torch.empty_like(x) for x in xs]

    def e2e_step():
        if wl.vjp:
            gs[0].copy_(hg, non_blocking=True)
        for i in range(len(hx)):
            dx[i].copy_(hx[i], non_blocking=True)
            offs, sides = shapes[i]
            if wl.scs is not None:
                scs_u.copy_(dx[i])
                scs_v.copy_(scs_v0)
                scs_run(sides, offs)
                dy[i].copy_(scs_u)
            elif poly:
                lib.proj_poly(dx[i], sides, args.poly_lo, out=dy[i], opts=opts, offsets=offs)
            elif wl.mixing:
                lib.mix_identity(dx[i], sides, wl.groups, wl.nu, wl.eps, out=dy[i], opts=opts, offsets=offs)
            elif wl.vjp:
                lib.proj_vjp(dx[i], gs[0], sides, xbar=dy[i], y=yb, opts=opts, offsets=offs)
            elif wl.herm:
                lib.proj_hermitian(dx[i], sides, out=dy[i], opts=opts, offsets=offs)
            else:
                lib.proj_batched(dx[i], sides, out=dy[i], opts=opts, offsets=offs)
            hy[i].copy_(dy[i], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms += e0.elapsed_time(e1)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = world * wl.units / (e2e_ms / steps * 1e-3)

    if rank != 0:
        return None

    unit = ("cones/s (lambda_min + mixing)" if wl.mixing else
            "SCS iterations/s" if wl.scs is not None else "projections/s")
    if poly:
        roofline, poly_info = poly_roofline(lib, args, wl, ms_per_step, prec)
    else:
        roofline = eig_roofline(args, wl, phases, tuning, b_used, steps)

    line = {
        "metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if precision == "fp64" else
        ("f64 io, tf32x8 split products" if poly else "f64 io, tf32x6 split products"),
        "data": "synthetic (seeded PCG64), shaped like the paper's SCS iterates; no dataset",
        "config": {"workload": wl.desc, "config": config, "method": poly_info if poly else "eigendecomposition",
                   "cones_per_step": wl.units, "band": None if poly else b_used,
                   "precision": precision, "tuning": tuning,
                   "parallelism": f"replicas x{world}", "l2": "flushed before every timed step (256 MB write)"},
        "e2e": {"value": e2e_value, "unit": unit, "h2d_bytes_per_step": wl.bytes_in,
                "d2h_bytes_per_step": wl.bytes_out},
        "gpu_launches": int(launches_per_step * steps),
        "timing": {"value": "K untraced steps (graph replay)",
                   "roofline": "phase CUDA events of a second, traced pass over the same K steps",
                   "traced_ms_per_step": traced_ms / steps},
        "roofline": roofline,
        "phases_ms_per_step": {k2: v[0] / steps for k2, v in phases.items() if v[1]},
        "clocks": clk,
        "status": int(status) if status == st else int(status),
        "max_rel_err_first_cone_vs_construction": err0,
        "stats_first_call": stats0,
    }
    if not args.no_comparator:
        line["comparator"] = comparator(wl, xs, dev, stream)
    if not args.no_cpu_baseline:
        v, done, dt, cores, sample = oracle_value(wl, budget_s=12.0, poly_lo=args.poly_lo if poly else None)
        line["cpu_baseline"] = {"value": v, "unit": unit, "cores": cores, "kind": "oracle",
                                "sample": f"{done} {'iterations' if wl.scs is not None else 'projections'} "
                                          f"(sides {sorted(set(sample))}) in {dt:.1f} s"}
    if wl.vjp:
        line["max_rel_err_vjp_first_cone_vs_construction"] = vjp_construction_error(wl, ys[0])
    return line


def leg_record(args, wl, config, precision, steps, warmup, ms_per_step, value, phases, tuning, b_used, clk,
               status, err0, launches_per_step, traced_ms, xs, dev, stream, ys, yb, stats0):
    """The record of one leg of the default run: value, comparator, roofline,
    error against the construction, clocks."""
    unit = "projections/s" if not wl.vjp else "(projection + VJP)/s"
    rec = {
        "value": value, "unit": unit, "workload": wl.desc, "precision": precision, "steps": steps,
        "warmup": warmup, "ms_per_step": ms_per_step, "cones_per_step": wl.units,
        "dtype": "f64" if precision == "fp64" else "f64 io, split-tf32 products",
        "roofline": eig_roofline(args, wl, phases, tuning, b_used, steps),
        "phases_ms_per_step": {k2: v[0] / steps for k2, v in phases.items() if v[1]},
        "timing": {"value": "K untraced steps (graph replay)", "traced_ms_per_step": traced_ms / steps},
        "gpu_launches": int(launches_per_step * steps),
        "clocks": clk, "status": int(status),
        "max_rel_err_first_cone_vs_construction": err0,
        "stats_first_call": stats0,
        "l2": "flushed before every timed step (256 MB write)",
    }
    if wl.vjp:
        rec["max_rel_err_vjp_first_cone_vs_construction"] = vjp_construction_error(wl, ys[0])
    if not args.no_comparator:
        rec["comparator"] = comparator(wl, xs, dev, stream, max_calls=1)
    return rec


def vjp_construction_error(wl, xbar_dev):
    """Relative error of the first cone's VJP against the derivative formed
    from the construction X = Q diag(lam) Q^T: Q (L o (Q^T G Q)) Q^T with the
    Loewner matrix of max(., 0) (App. E's derivative through the
    eigendecomposition; at eigenvalues +-1e-9 of opposite sign the computed
    cross block is fixed only to about eps ||X|| / 2e-9 by any
    backward-stable eigensolver)."""
    Q, lam = wl.exact0
    n = Q.shape[0]
    ln = n * (n + 1) // 2
    G = W_smat_host(wl.g[:ln], n)
    lp = np.maximum(lam, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        L = (lp[:, None] - lp[None, :]) / (lam[:, None] - lam[None, :])
    pos = lam > 0
    L = np.where(pos[:, None] & pos[None, :], 1.0, L)
    L = np.where(~pos[:, None] & ~pos[None, :], 0.0, L)
    J = Q @ (L * (Q.T @ G @ Q)) @ Q.T
    ref = W.to_svec(J)
    got = xbar_dev[:ln].cpu().numpy()
    return rel(got, ref)


def eig_roofline(args, wl, phases, tuning, b_used, steps):
    """Roofline of the dominant traced phase of the eigendecomposition path
    (per-phase CUDA events on the launching stream)."""
    dom = max(phases.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_count) = dom
    n0 = wl.calls[0][1][0]
    if wl.exact0 is not None:
        lam_sample = wl.exact0[1]          # spectrum of the construction
    else:
        lam_sample = np.linalg.eigvalsh(W_smat_host(wl.calls[0][0][: n0 * (n0 + 1) // 2], n0))
    kp, kn = int((lam_sample > 0).sum()), int((lam_sample < 0).sum())
    k = min(kp, kn)
    kbt = n0 if wl.vjp else k
    cones_per_call = len(wl.calls[0][1])
    # Hermitian cones: the native complex route (sides up to 1100, automatic route) does
    # four real flops' work per complex operation in every phase but the real divide and
    # conquer; the real embedding of side 2n (every eigenvalue twice) otherwise
    native = wl.herm and args.band == 0 and max(int(s) for s in wl.calls[0][1]) <= 1100
    emb = 2 if (wl.herm and not native) else 1
    cplx = 4.0 if (native and dom_name != "tridiag_dc") else 1.0
    flops_launch = sum(cplx * algorithmic_flops(dom_name, emb * int(s), emb * k, b_used, emb * kbt)
                       for s in wl.calls[0][1])
    # per call: a phase may be traced as several segments within one call
    per_call = wl.iters if wl.scs is not None else 1  # projections per call (SCS: one per iteration)
    avg_ms = dom_ms / max(1, steps * len(wl.calls) * per_call)
    achieved = flops_launch / (avg_ms * 1e-3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "peak_source": FP64_PEAK_NOTE,
                "unit": "GFLOP/s FP64",
                "frac": achieved / FP64_PEAK_GFLOPS, "traffic": _traffic(wl.name, dom_name),
                "phase": dom_name, "kernel": phase_kernels(dom_name, n0, tuning["band"] if tuning else args.band),
                "ms_per_launch": avg_ms, "flops_per_launch": flops_launch,
                "share": dom_ms / max(1e-9, sum(v[0] for v in phases.values()))}


def poly_roofline(lib, args, wl, ms_per_step, prec):
    """Roofline of the factorization-free path from the whole step: its work
    is the composite's products, K (2 n^3) + n^3 flops per cone (every product
    forms a lower triangle).  Split-TF32 products of this path issue eight
    TF32 products per FP64 product (tc2_gemm_kernel); their peak is the
    measured bf16 peak x the nominal TF32/BF16 ratio 1.1/2.25."""
    a, b, lk = lib.poly_schedule(args.poly_lo)
    K = len(a)
    flops = sum(K * 2.0 * float(n) ** 3 + float(n) ** 3 for _, sides in wl.calls for n in sides)
    achieved = flops / (ms_per_step * 1e-3)
    info = {"name": "factorization-free composite polynomial (scaled Newton-Schulz sign)", "lo": args.poly_lo,
            "steps": K, "one_minus_l_final": 1.0 - lk}
    if prec == lib.FP64:
        return {"bound": "alu", "achieved": achieved / 1e9, "peak": FP64_PEAK_GFLOPS, "peak_source": FP64_PEAK_NOTE,
                "unit": "GFLOP/s FP64", "frac": achieved / 1e9 / FP64_PEAK_GFLOPS, "traffic": None,
                "phase": "polynomial products", "kernel": "gemm_f64_kernel (grouped)",
                "flops_per_step": flops}, info
    peak = _tf32_peak()
    ach = 8.0 * achieved / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": peak[0], "peak_source": peak[1], "unit": "TFLOP/s TF32",
            "frac": ach / peak[0], "traffic": None, "phase": "polynomial products",
            "kernel": "tc2_gemm_kernel (split-TF32, operands sliced once)", "flops_per_step_fp64_equivalent": flops}, info


def _tf32_peak():
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return mp["bf16_tflops"] * 1.1 / 2.25, "measured bf16 burst x nominal TF32/BF16 ratio 1.1/2.25"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "fallback bf16 1.9 PFLOP/s x nominal TF32/BF16 ratio 1.1/2.25"


def W_smat_host(s, n):
    """Host unpacking of an svec, only to count the kept eigenpairs for the flop count."""
    r, c = np.triu_indices(n)
    A = np.zeros((n, n))
    v = s * np.where(r == c, 1.0, 1.0 / np.sqrt(2.0))
    A[r, c] = v
    A[c, r] = v
    return A


def _smat_torch(s, n):
    """Plain torch unpacking of an svec (comparator and flop counting only)."""
    import torch
    r, c = np.triu_indices(n)
    A = torch.zeros((n, n), dtype=torch.float64, device=s.device)
    rr = torch.from_numpy(r).to(s.device)
    cc = torch.from_numpy(c).to(s.device)
    scale = torch.where(rr == cc, 1.0, 1.0 / np.sqrt(2.0)).to(torch.float64)
    A[rr, cc] = s * scale
    A[cc, rr] = s * scale
    return A


def comparator(wl, xs, dev, stream, max_calls: int = 20):
    """The plain FP64 GPU path: torch.linalg.eigh (vendor solver) + clamp +
    reconstruct, on the same inputs (at most max_calls calls); for the mixing
    workload torch.linalg.eigvalsh + the same weight rule."""
    import torch
    r_idx = {}

    def proj_one(s, n):
        if wl.herm:
            return proj_one_herm(s, n)
        A = _smat_torch(s, n)
        w, V = torch.linalg.eigh(A)
        P = (V * w.clamp(min=0)) @ V.T
        if n not in r_idx:
            r, c = np.triu_indices(n)
            r_idx[n] = (torch.from_numpy(r).to(dev), torch.from_numpy(c).to(dev))
        r, c = r_idx[n]
        return P[r, c] * torch.where(r == c, 1.0, np.sqrt(2.0)).to(torch.float64)

    h_idx = {}

    def proj_one_herm(s, n):
        # Hermitian svec: per column the diagonal, then sqrt(2) Re, sqrt(2) Im of every row below
        if n not in h_idx:
            d_pos, rows, cols, re_pos = [], [], [], []
            k = 0
            for j in range(n):
                d_pos.append(k)
                k += 1
                for i in range(j + 1, n):
                    rows.append(i); cols.append(j); re_pos.append(k)
                    k += 2
            t = lambda a: torch.tensor(a, dtype=torch.long, device=dev)
            h_idx[n] = (t(d_pos), t(rows), t(cols), t(re_pos))
        d_pos, rows, cols, re_pos = h_idx[n]
        ar = torch.arange(n, device=dev)
        A = torch.zeros((n, n), dtype=torch.complex128, device=dev)
        A[ar, ar] = s[d_pos].to(torch.complex128)
        off = torch.complex(s[re_pos], s[re_pos + 1]) / np.sqrt(2.0)
        A[rows, cols] = off
        A[cols, rows] = off.conj()
        w, V = torch.linalg.eigh(A)
        P = (V * w.clamp(min=0)) @ V.conj().T
        out = torch.empty(n * n, dtype=torch.float64, device=dev)
        out[d_pos] = P[ar, ar].real
        po = P[rows, cols] * np.sqrt(2.0)
        out[re_pos] = po.real
        out[re_pos + 1] = po.imag
        return out

    calls = list(range(min(max_calls, len(xs))))
    offs_all = [wl.calls[i][1] for i in calls]

    def run_mixing():
        # torch.linalg.eigvalsh per block, the weight rule per group, the mixed svec
        out = 0
        for i in calls:
            sides = offs_all[i]
            offs = np.concatenate([[0], np.cumsum([wl.svec_len(n) for n in sides])])
            lam = [torch.linalg.eigvalsh(_smat_torch(xs[i][offs[a]:offs[a + 1]], n))[0]
                   for a, n in enumerate(sides)]
            for g in range(len(wl.groups) - 1):
                a0, a1 = wl.groups[g], wl.groups[g + 1]
                lg = torch.stack(lam[a0:a1])
                nu = wl.nu[g]
                cand = torch.where(lg < wl.eps, (nu - wl.eps) / (nu - lg), torch.ones_like(lg))
                p = torch.where(lg.min() >= 0, torch.ones((), dtype=lg.dtype, device=lg.device), cand.min())
                for a in range(a0, a1):
                    n = sides[a]
                    r, c = np.triu_indices(n)
                    dia = torch.from_numpy((r == c).astype(np.float64)).to(xs[i].device)
                    _ = p * xs[i][offs[a]:offs[a + 1]] + (1 - p) * nu * dia
                    out += 1
        return out

    def run_scs():
        # the same iterations with torch ops: matmuls (dense A) or einsum
        # contractions (structured A) for the affine step, eigh for the projection
        kind, *prob = wl.scs
        b_h, c_h, u0, v0 = prob[-4:]
        bt, ct = torch.from_numpy(b_h).to(dev), torch.from_numpy(c_h).to(dev)
        m = b_h.size
        k = c_h.size
        r, cc = np.triu_indices(625)
        rr, ccd = torch.from_numpy(r).to(dev), torch.from_numpy(cc).to(dev)
        scale = torch.from_numpy(np.where(r == cc, 1.0, np.sqrt(2.0))).to(dev)
        if kind == "dense":
            A = torch.from_numpy(prob[0]).to(dev).t()
            op_n = lambda x: A @ x  # noqa: E731
            op_t = lambda y: A.t() @ y  # noqa: E731
        else:
            Bs = [torch.from_numpy(B).to(dev) for B in prob[0]]
            idx = torch.from_numpy(prob[1]).to(dev)
            shape = [B.shape[0] for B in Bs]
            N = 625

            def op_n(x):
                T = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device=dev)
                T[idx] = x
                Wm = torch.einsum("abcd,aim,bjn,cko,dlp->ijklmnop", T.reshape(shape), *Bs).reshape(N, N)
                return Wm[ccd, rr] * scale

            def op_t(y):
                Y = _smat_torch(y, N).reshape(5, 5, 5, 5, 5, 5, 5, 5)
                T = torch.einsum("ijklmnop,aim,bjn,cko,dlp->abcd", Y, *Bs)
                return T.reshape(-1)[idx]
        u, v = torch.from_numpy(u0).to(dev), torch.from_numpy(v0).to(dev)
        px = 0.5 * (ct - op_t(bt))
        py = bt + op_n(px)
        hp = ct @ px + bt @ py
        for _ in range(wl.iters):
            w = u + v
            zx = 0.5 * (w[:k] - op_t(w[k:k + m]))
            zy = w[k:k + m] + op_n(zx)
            tau = (w[-1] + ct @ zx + bt @ zy) / (1 + hp)
            ut = torch.cat([zx - tau * px, zy - tau * py, tau.reshape(1)])
            t = ut - v
            Y = _smat_torch(t[k:k + m], 625)
            ev, V = torch.linalg.eigh(Y)
            P = (V * ev.clamp(min=0)) @ V.T
            un = torch.cat([t[:k], P[torch.from_numpy(cc).to(dev), torch.from_numpy(r).to(dev)] * scale,
                            t[-1:].clamp(min=0)])
            v = v - ut + un
            u = un
        return wl.iters

    def run():
        if wl.scs is not None:
            return run_scs()
        if wl.mixing:
            return run_mixing()
        out = 0
        for i in calls:
            sides = offs_all[i]
            o = 0
            for n in sides:
                ln = wl.svec_len(n)
                proj_one(xs[i][o:o + ln], n)
                o += ln
                out += 1
        return out

    run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    units = run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if wl.scs is not None:
        return {"impl": "the same iterations in torch: " + ("matmuls" if wl.scs[0] == "dense" else "einsum contractions")
                + " + torch.linalg.eigh float64 projection",
                "value": units / (ms * 1e-3), "unit": "SCS iterations/s", "sample": f"{units} iterations"}
    if wl.mixing:
        return {"impl": "torch.linalg.eigvalsh float64 per block + the same weight rule + mixed svec",
                "value": units / (ms * 1e-3), "unit": "cones/s", "sample": f"{units} cones"}
    return {"impl": ("torch.linalg.eigh complex128" if wl.herm else "torch.linalg.eigh float64") + " + clamp + reconstruct",
            "value": units / (ms * 1e-3),
            "unit": "projections/s", "sample": f"{units} projections"}


def _traffic(config, phase):
    """DRAM bytes per call of the phase's kernel from the committed ncu summary
    (a table row "| config | phase | bytes | ..." in profiles/traffic.md), if any."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    try:
        for line in open(path):
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 3 and cells[0] == config and cells[1] == phase:
                return float(cells[2])
    except (OSError, ValueError):
        return None
    return None


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
