#!/usr/bin/env python
"""Benchmark: space-time unknowns/s of the mixed-precision refined FDM solve against the FP64 FDM.

Workload (default, `--config c3`): 384x384 squares P1 in space (146,689 interior nodes, half
bandwidth 384), P2 time on 512 uniform elements (n_t = 1024), T = 2: 150,209,536 unknowns;
psi0 = four seeded Gaussian wave packets, f = 0; mixed precision refined to a relative FP64
residual of 1e-10.  The factors of all 1024 spatial systems (463 GB) do not fit in HBM: the
leading systems' factors are kept, the others are refactorised at every FP32 application.

`--config c2`: 256x256 squares P1 (65,025 nodes), P1 time on 512 uniform elements, T = 1
(33,292,800 unknowns); manufactured psi = sin(pi x1) sin(pi x2) (1+t) e^{-it}, the interpolated
load (M_t,full (x) M_x) f built on the device (st_load_nodal), psi0 = psi(., 0), refined to 1e-11.

One step = one H2D copy of the step's inputs (F, psi0) from pinned host memory, one full
st_fdm_solve (lifting, forward transform, banded LDL^T factor and solve of the spatial systems,
back transform, FP64 residual, refinement until the target), one D2H copy of psi.  CUDA events
split every step: `value` counts the solve alone (its inputs resident in HBM), `e2e` the whole
step.  The inputs (2.4 GB / 533 MB of c128) exceed the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config c3|c2|c5]

Multi-GPU: the single-problem workload does not shard without an exchange step; N ranks
run N independent replicas (weak scaling), timed with a barrier and the max over ranks.
`--impl reference` times the CPU oracle (the FP64 fast diagonalisation of the paper on
the host cores) on a bounded sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "space-time unknowns/s at <=1e-9 rel. error, mixed vs FP64 FDM; % roofline"
UNIT = "unknowns/s"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="c3")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp32"])
    ap.add_argument("--spatial", default="multifrontal", choices=["banded", "multifrontal"],
                    help="spatial solver of step 3: the sparse-direct multifrontal LDL^T (default) or banded LDL^T")
    ap.add_argument("--no-compare-banded", dest="compare_banded", action="store_false",
                    help="skip the banded solver's comparison measurement")
    ap.add_argument("--no-fp64-check", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-step", action="store_true",
                    help="set up, then run exactly one solve and exit (for ncu launch lists)")
    ap.add_argument("--profile-xform", action="store_true",
                    help="set up, then run one tensor-core forward time transform and exit (small device footprint)")
    ap.add_argument("--profile-mf", action="store_true",
                    help="set up, then run one multifrontal FP32 factorisation of all systems and one substitution "
                         "pass with the kept factors, and exit (for ncu captures of those kernels)")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ distributed helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of a float over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sms, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sms.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sms)}


# ------------------------------------------------------------------ roofline helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return None


def kernel_source_sha(kind: str = "band"):
    """Hash of the source of the kernels whose DRAM traffic was recorded: for "band" the FP32 banded
    spatial solve (the blocked-panel factor kernel's section of k_band.cu, the substitution kernels,
    the asynchronous-copy helpers, and the complex helpers and launch arguments of the device header);
    for "mf" the multifrontal kernels (k_mf.cu, the complex helpers and the front/launch-argument
    structs of the device header).  The recorded traffic is used only while this is unchanged."""
    csrc = os.path.join(ROOT, "paper_2504_07269_gb300", "csrc")
    with open(os.path.join(csrc, "device.cuh")) as fh:
        dev = fh.read()
    helpers = dev[dev.index("// ------------------------------------------------------------------ complex helpers"):
                  dev.index("// ------------------------------------------------------------------ handle")]
    if kind == "mf":
        with open(os.path.join(csrc, "k_mf.cu")) as fh:
            h = hashlib.sha256(fh.read().encode())
        a = dev.index("struct MfFrontDev {")
        b = dev.index("\n};", dev.index("struct MfArgs {")) + 3
        h.update((helpers + dev[a:b]).encode())
        return h.hexdigest()[:16]
    with open(os.path.join(csrc, "k_band.cu")) as fh:
        text = fh.read()
    start = text.index("// ------------------------------------------------------------------ complex64, blocked panel")
    end = text.index("// ------------------------------------------------------------------ backward substitution by one CTA")
    h = hashlib.sha256(text[start:end].encode())
    for name in ("k_subst.cu", "async.cuh"):
        with open(os.path.join(csrc, name)) as fh:
            h.update(fh.read().encode())
    c = dev.index("struct BandArgs {")
    h.update((helpers + dev[c:dev.index("\n};", c) + 3]).encode())
    return h.hexdigest()[:16]


def profiled_traffic(key: str, kind: str = "band"):
    """DRAM bytes per launch of the kernels named by key (e.g. band_factor_fp32_c3: one FP32 banded
    spatial solve, the factorisation with the fused forward substitution, then the backward
    substitution) from the committed ncu summary, or None if the kernels' source changed since the
    capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(key)
    if not e or e.get("src_sha", e.get("k_band_sha")) != kernel_source_sha(kind):
        return None
    return e.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ inputs
def make_inputs(pr, h, device):
    """The step's load F (c128, (n_t, n_x)) and psi0 on the device.  384^2/P2-1024 (c3): f = 0 and psi0
    = four seeded packets; otherwise the manufactured psi of the 16^2/256^2 workloads: F is the
    interpolated load (M_t,full (x) M_x) f of f's nodal values at every DOF time (st_load_nodal),
    psi0 = psi(., 0)."""
    import torch

    from paper_2504_07269_gb300 import stfdm

    x1, x2 = synth.interior_coords(pr.n, pr.Lx, pr.Ly)
    if pr.name == "c3":
        psi0 = synth.packet_values(synth.packet_params(pr.seed), x1, x2)
        F = torch.zeros((pr.n_t, pr.n_x), dtype=torch.complex128, device=device)
        return F, torch.from_numpy(psi0).to(device)
    tf = synth.dof_times(pr.p_t, pr.t_nodes)                 # t_0 included
    f = torch.from_numpy(synth.f_c1(x1[None, :], x2[None, :], tf[:, None])).to(device)
    F = stfdm.st_load_nodal(h, f)
    del f
    return F, torch.from_numpy(synth.psi0_c1(x1, x2)).to(device)


# ------------------------------------------------------------------ CPU baseline (oracle)
def cpu_oracle_sample(pr, n_solves=None, workers=None):
    """Times the CPU oracle's FP64 FDM on a bounded sample of the workload: both dense time
    transforms in full and `n_solves` of the n_t sparse-direct spatial solves (process pool,
    one BLAS thread per worker); the solve time is extrapolated to all n_t systems."""
    from oracle import cpu_fdm, fe_space, fe_time, timedec

    workers = workers or os.cpu_count()
    n_solves = n_solves or max(workers, 8)
    M_t, B_t, m_t, _ = fe_time.assemble_time(pr.p_t, pr.t_nodes)
    X, s, Y, _ = timedec.fdm_decomposition(M_t, B_t)
    F = synth.cn01((pr.n_t, pr.n_x), seed=pr.seed)
    t0 = time.perf_counter()
    G = Y @ F
    _ = X @ G
    t_xf = time.perf_counter() - t0
    idx = np.linspace(0, pr.n_t - 1, n_solves).astype(int)
    t0 = time.perf_counter()
    cpu_fdm.spatial_solves(pr.n, s[idx], G[idx], pr.Lx, pr.Ly, workers=workers)
    t_sol = time.perf_counter() - t0
    est = t_xf + t_sol * pr.n_t / len(idx)
    return {"value": pr.unknowns / est, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": (f"CPU FP64 FDM (numpy eig, SuperLU per eigen-index): both transforms in full, "
                       f"{len(idx)} of {pr.n_t} spatial solves on a {workers}-process pool, extrapolated; "
                       f"measured {t_xf + t_sol:.1f} s, estimated full solve {est:.1f} s")}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    pr = synth.config_problem(args.config)
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_sample(pr)
        if i >= args.warmup:
            vals.append(r["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * pr.unknowns / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(pr, args),
            "cpu_baseline": dict(r, value=v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# Relative residual target of the single-problem mixed solve per workload.  384^2/P2-1024: the
# configuration's 1e-10.  256^2/512: on that workload the error against the FP64 FDM is about 6x the
# final residual, so 1e-11 keeps it two orders below the metric's 1e-9 bar (the line prints it);
# 1e-12 sits at the FP64 residual floor (the GMRES estimate reaches 5e-13 while the true residual is
# 1.2e-12) and costs a second restart cycle.
SINGLE_TOL = {"c3": 1e-10, "c2": 1e-11}
# Error target of the single-problem mixed solve (the library's error estimate ||FDM32(R)|| / ||psi_hat||,
# checked each time the residual target is met).  At 384^2/P2-1024 a residual of 2e-11 still leaves an
# error of 1e-8 against the FP64 references (the error/residual ratio approaches cond(K)), so the residual
# target alone does not give the metric's 1e-9; the estimate keeps the iteration going until it does.
SINGLE_ERR_TOL = {"c3": 2e-10}


def single_tol(pr):
    return SINGLE_TOL.get(pr.name, 1e-11)


def single_err_tol(pr):
    return SINGLE_ERR_TOL.get(pr.name, 0.0)


def _config(pr, args):
    inputs = ("psi0 = 4 seeded Gaussian packets, f = 0" if pr.name == "c3"
              else "manufactured psi = sin(pi x1) sin(pi x2)(1+t)e^{-it}, interpolated load")
    gb = pr.unknowns * 16 / 1e9
    return {"workload": f"{pr.n}x{pr.n} squares P1 space ({pr.n_x} nodes), P{pr.p_t} time {len(pr.t_nodes) - 1} "
                        f"uniform elements (n_t={pr.n_t}), T={pr.t_nodes[-1]:g}; {pr.unknowns} unknowns; {inputs}",
            "name": pr.name, "precision": args.precision, "spatial_solver": getattr(args, "spatial", "banded"),
            "tol": single_tol(pr), "err_tol": single_err_tol(pr), "n_x": pr.n_x, "n_t": pr.n_t,
            "unknowns": pr.unknowns, "l2_flush": f"inputs ({gb:.2f} GB c128 load) larger than the 129 MB L2",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


# ------------------------------------------------------------------ our solver
def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2504_07269_gb300 import stfdm

    pr = synth.config_problem(args.config)
    tol = single_tol(pr)
    etol = single_err_tol(pr)
    t0 = time.perf_counter()
    h = stfdm.setup_problem(pr.n, pr.p_t, pr.t_nodes, Lx=pr.Lx, Ly=pr.Ly, device=local, spatial_solver=args.spatial)
    setup_s = time.perf_counter() - t0
    kappa = h.kappa
    F, p0 = make_inputs(pr, h, dev)
    dt = torch.complex64 if args.precision == "fp32" else torch.complex128
    F = F.to(dt)
    p0 = p0.to(dt)
    psi = torch.empty_like(F)
    info = {}
    if args.profile_xform:
        G32 = stfdm.st_time_transform(h, "Y", "mixed", F.to(torch.complex64))
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_xform": args.config, "norm": float(torch.linalg.vector_norm(G32))}))
        return 0
    if args.profile_mf:
        G = F.to(torch.complex64) + torch.from_numpy(synth.cn01((pr.n_t, pr.n_x), seed=11)).to(dev).to(torch.complex64)
        stfdm.st_spatial_factor(h, "fp32")
        W = stfdm.st_spatial_substitute(h, "fp32", G)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_mf": args.config, "norm": float(torch.linalg.vector_norm(W))}))
        return 0
    if args.profile_step:
        _, info = stfdm.st_fdm_solve(h, F, p0, psi=psi, precision=args.precision, tol=tol, err_tol=etol)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_step": args.config, "precision": args.precision, "info": info}))
        return 0

    # One step: H2D of the inputs from pinned host memory, the solve (inputs resident), D2H of psi.
    # Four events per step on the launching stream split it into copy-in, solve and copy-out.
    Fh = F.cpu().pin_memory()
    p0h = p0.cpu().pin_memory()
    psih = torch.empty(F.shape, dtype=dt).pin_memory()
    h2d = Fh.numel() * Fh.element_size() + p0h.numel() * p0h.element_size()
    d2h = psih.numel() * psih.element_size()
    Fd = F
    p0d = p0

    def step(ev):
        nonlocal info
        ev[0].record()
        Fd.copy_(Fh, non_blocking=True)
        p0d.copy_(p0h, non_blocking=True)
        ev[1].record()
        _, info = stfdm.st_fdm_solve(h, Fd, p0d, psi=psi, precision=args.precision, tol=tol, err_tol=etol)
        ev[2].record()
        psih.copy_(psi, non_blocking=True)
        ev[3].record()

    def events():
        return [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    for _ in range(args.warmup):
        step(events())
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    barrier(world)
    torch.cuda.synchronize()
    evs = [events() for _ in range(args.steps)]
    for i in range(args.steps):
        step(evs[i])
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    solve_ms = [e[1].elapsed_time(e[2]) for e in evs]
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    h2d_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    d2h_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    t_ms = reduce_max(statistics.mean(solve_ms), world, dev)
    e2e_ms = reduce_max(statistics.mean(step_ms), world, dev)
    value = world * pr.unknowns / (t_ms * 1e-3)
    print(f"timed: solve {t_ms:.1f} ms, step {e2e_ms:.1f} ms, {value:.4e} unknowns/s, info {info}", file=sys.stderr,
          flush=True)
    sweeps = int(info.get("sweeps", 1)) if info else 1
    # our kernels per step: the library counts the launches each solve issues (an ncu launch list of
    # one step agrees with it); the copies are not kernels
    launches_per_step = int(info.get("kernel_launches", 0)) if info else 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # ---- error against the FP64 FDM on the same inputs, and against a tightly refined solution
    err = err_tight = fp64_res = tight_res = None
    fp64_value = None
    fp32_value = fp32_err = None
    if not args.no_fp64_check and args.precision != "fp64":
        mine = psi.to(torch.complex128)
        # the plain complex-FP32 FDM on the same inputs (3xTF32 tensor-core transforms, FP32 solves)
        F32, p032 = F.to(torch.complex64), p0.to(torch.complex64)
        psi32 = torch.empty_like(F32)
        stfdm.st_fdm_solve(h, F32, p032, psi=psi32, precision="fp32", want_info=False)
        torch.cuda.synchronize()
        e0.record()
        stfdm.st_fdm_solve(h, F32, p032, psi=psi32, precision="fp32", want_info=False)
        e1.record()
        torch.cuda.synchronize()
        fp32_value = pr.unknowns / (e0.elapsed_time(e1) * 1e-3)
        del F32, p032
        # the FP64 FDM (one solve: at the 384^2/P2-1024 workload it takes minutes)
        ref = torch.empty(F.shape, dtype=torch.complex128, device=dev)
        F64, p064 = F.to(torch.complex128), p0.to(torch.complex128)
        torch.cuda.synchronize()
        e0.record()
        stfdm.st_fdm_solve(h, F64, p064, psi=ref, precision="fp64", want_info=False)
        e1.record()
        torch.cuda.synchronize()
        fp64_value = pr.unknowns / (e0.elapsed_time(e1) * 1e-3)
        nref = torch.linalg.vector_norm(ref)
        err = float(torch.linalg.vector_norm(mine - ref) / nref)
        fp32_err = float(torch.linalg.vector_norm(psi32.to(torch.complex128) - ref) / nref)
        del psi32
        fp64_res = float(stfdm.st_residual(h, F64, p064, ref)[0])
        # the FP64 FDM carries the rounding of X_t (about kappa_2(X_t) eps in the residual): a solution
        # refined to 1e-13 says which of the two is off
        try:
            stfdm.st_fdm_solve(h, F64, p064, psi=ref, precision="mixed", tol=1e-12, err_tol=1e-12, max_sweeps=60,
                               want_info=False)
        except Exception as ex:   # at the FP64 floor: the iterate is still the tightest reference at hand
            print(f"tight reference: {ex}", file=sys.stderr)
        err_tight = float(torch.linalg.vector_norm(mine - ref) / torch.linalg.vector_norm(ref))
        tight_res = float(stfdm.st_residual(h, F64, p064, ref)[0])
        del ref, mine, F64, p064
        torch.cuda.empty_cache()

    # ---- rooflines: the multifrontal substitution pass (the kernels of every later FP32 application,
    # HBM) and its factorisation (ALU), or the banded factor-and-solve (ALU)
    kprec = "fp64" if args.precision == "fp64" else "fp32"
    if args.spatial == "multifrontal":
        roof, roof_factor = multifrontal_rooflines(stfdm, h, pr, kprec, dev, clocks, args.config)
    else:
        roof, roof_factor = banded_roofline(stfdm, h, pr, kprec, dev, clocks, args.config), None

    # ---- the banded solver (the fixed spatial design) on the same workload, for comparison
    banded = None
    if args.spatial == "multifrontal" and args.compare_banded and args.precision == "mixed":
        h.close()      # release the multifrontal handle's factors and workspace before the banded solver's
        torch.cuda.empty_cache()
        banded = banded_comparison(stfdm, pr, F, p0, psi, tol, etol, kprec, dev, clocks, args.config, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_oracle_sample(pr)
        except Exception as ex:  # the baseline is reported, not required
            cpu = {"error": str(ex)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"mixed": "c64+f64", "fp64": "f64", "fp32": "f32"}[args.precision],
                "data": ("synthetic (seeded Gaussian packets, f = 0)" if pr.name == "c3"
                         else "synthetic (manufactured solution, interpolated load)"),
                "config": _config(pr, args),
                "err_vs_fp64": err, "fp64_fdm_rel_residual": fp64_res, "err_vs_tight": err_tight,
                "tight_rel_residual": tight_res,
                "err_estimate": info.get("rel_error_estimate") if info else None,
                "fp64_fdm_unknowns_per_s": fp64_value,
                "fp32_fdm_unknowns_per_s": fp32_value, "fp32_fdm_err_vs_fp64": fp32_err, "sweeps": sweeps,
                "restart": info.get("restart") if info else None,
                "kept_systems": info.get("kept_systems") if info else None,
                "final_rel_residual": info.get("rel_residual") if info else None,
                "setup_s": setup_s, "kappa_x": kappa,
                "e2e": {"value": world * pr.unknowns / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "h2d_ms": h2d_ms, "d2h_ms": d2h_ms,
                        "h2d_gbs": h2d / (h2d_ms * 1e6), "d2h_gbs": d2h / (d2h_ms * 1e6),
                        "timing": "same steps as value: events around H2D + solve + D2H (e2e) and the solve (value)"},
                "gpu_launches": launches_per_step * args.steps,
                "roofline": roof, "roofline_factor": roof_factor, "banded": banded,
                "cpu_baseline": cpu, "clocks": clocks}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def _peak_alu(dev, clocks, kprec):
    import torch

    props = torch.cuda.get_device_properties(dev)
    max_mhz = (clocks or {}).get("sm_max_mhz") or (measured_peaks() or {}).get("sm_max_mhz", 2070.0)
    lanes = 128 if kprec == "fp32" else 2             # FP32 / FP64 FMA lanes per SM per clock
    basis = (f"{props.multi_processor_count} SMs x {lanes} {kprec.upper()} FMA lanes x 2 x {max_mhz:.0f} MHz "
             "(derived, max SM clock)")
    return props.multi_processor_count * lanes * 2 * max_mhz * 1e6 / 1e12, basis


def _time3(fn):
    """Median of three CUDA-event timings of fn() on the current stream, seconds."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    return statistics.median(times)


def banded_roofline(stfdm, h, pr, kprec, dev, clocks, config):
    """The banded LDL^T factor-and-solve of all n_t systems (factor kernel with the fused forward
    substitution, then the backward substitution), against the FP32 (or FP64) ALU peak."""
    import torch

    kdt = torch.complex128 if kprec == "fp64" else torch.complex64
    G0 = torch.from_numpy(synth.cn01((pr.n_t, pr.n_x), seed=11)).to(dev).to(kdt)
    Gw = torch.empty_like(G0)

    def run():
        Gw.copy_(G0)
        stfdm.st_spatial_solve(h, kprec, Gw, Gw)

    tk = _time3(run)            # the copy is 0.1% of the launch
    b = pr.n
    # complex MAC = 8 real flops; per system n_x b^2/2 for the factorisation and n_x b for each of the
    # two substitutions (the forward one fused into the factor kernel)
    flops = 8.0 * pr.n_t * pr.n_x * (b * b / 2.0 + 2.0 * b)
    peak, basis = _peak_alu(dev, clocks, kprec)
    achieved = flops / tk / 1e12
    kname = ("k_band_factor_v4 (complex64, fused forward substitution) + k_subst_bwd<float>" if kprec == "fp32"
             else "k_band_factor_solve<double,32> + k_subst_bwd<double>")
    return {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": profiled_traffic(f"band_factor_fp32_{config}"), "launch_ms": tk * 1e3,
            "peak_basis": basis}


def multifrontal_rooflines(stfdm, h, pr, kprec, dev, clocks, config):
    """(1) The substitution pass with kept factors, forward and backward over every level (what each
    later FP32 application runs): algorithmic bytes = the factor blocks read twice plus the right-hand
    sides read and written, against the measured HBM bandwidth.  (2) The factorisation of all n_t
    systems: the plan's flops (8 per complex multiply-add of every front's eliminations) against the
    ALU peak."""
    import torch

    kdt = torch.complex128 if kprec == "fp64" else torch.complex64
    esz = 16 if kprec == "fp64" else 8
    plan = stfdm.st_space_mf_plan(h.space, 0)
    tf = _time3(lambda: stfdm.st_spatial_factor(h, kprec))
    G0 = torch.from_numpy(synth.cn01((pr.n_t, pr.n_x), seed=11)).to(dev).to(kdt)
    Gw = torch.empty_like(G0)
    ts = _time3(lambda: stfdm.st_spatial_substitute(h, kprec, G0, Gw))
    # the substitute call first copies G into W (one read and one write of n_t n_x entries)
    nbytes = pr.n_t * (2.0 * plan["factor_entries"] * esz + 6.0 * pr.n_x * esz)
    peaks = measured_peaks() or {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    sub = {"bound": "hbm", "kernel": "k_mf_solve_small<32|64|96|128> + k_mf_fwd + k_mf_bwd (every level, both directions)",
           "achieved": nbytes / ts / 1e9, "peak": hbm, "unit": "GB/s", "frac": nbytes / ts / 1e9 / hbm,
           "traffic": profiled_traffic(f"mf_subst_{kprec}_{config}", "mf"), "launch_ms": ts * 1e3,
           "algorithmic_bytes": nbytes,
           "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks
           else "fallback 6.8 TB/s"}
    flops = pr.n_t * plan["flops"]
    peak, basis = _peak_alu(dev, clocks, kprec)
    fac = {"bound": "alu", "kernel": "k_mf_factor_small<32|64> + k_mf_factor (every level)",
           "achieved": flops / tf / 1e12, "peak": peak, "unit": "TFLOP/s", "frac": flops / tf / 1e12 / peak,
           "traffic": profiled_traffic(f"mf_factor_{kprec}_{config}", "mf"), "launch_ms": tf * 1e3,
           "peak_basis": basis,
           "plan": {"fronts": plan["fronts"], "levels": plan["levels"], "max_front": plan["max_front"],
                    "factor_entries_per_system": plan["factor_entries"], "flops_per_system": plan["flops"]}}
    return sub, fac


def banded_comparison(stfdm, pr, F, p0, psi, tol, etol, kprec, dev, clocks, config, local):
    """The same mixed solve with the banded spatial solver: one warm-up and one timed step (at the
    384^2/P2-1024 workload a banded solve takes tens of seconds), its factor roofline, and its error
    against the multifrontal solution just timed (both refined to the same targets)."""
    import torch

    t0 = time.perf_counter()
    hb = stfdm.setup_problem(pr.n, pr.p_t, pr.t_nodes, Lx=pr.Lx, Ly=pr.Ly, device=local, spatial_solver="banded")
    setup_s = time.perf_counter() - t0
    out = torch.empty_like(psi)
    stfdm.st_fdm_solve(hb, F, p0, psi=out, precision="mixed", tol=tol, err_tol=etol)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    _, info = stfdm.st_fdm_solve(hb, F, p0, psi=out, precision="mixed", tol=tol, err_tol=etol)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    diff = float(torch.linalg.vector_norm(out - psi) / torch.linalg.vector_norm(psi))
    roof = banded_roofline(stfdm, hb, pr, kprec, dev, clocks, config)
    hb.close()
    torch.cuda.empty_cache()
    return {"value": pr.unknowns / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": 1, "warmup": 1,
            "sweeps": info["sweeps"], "restart": info["restart"], "kept_systems": info["kept_systems"],
            "final_rel_residual": info["rel_residual"], "rel_diff_vs_multifrontal": diff, "setup_s": setup_s,
            "roofline": roof}


# ------------------------------------------------------------------ batched workload
def run_batch(args):
    """64 independent problems of uneven size (n in {32,...,192}, P1/P2 time, N_t in [32, 512],
    T in [0.5, 2], packet psi0, half of them forced) solved together by one batched plan,
    refined to 1e-12 relative residual (the configuration's 1e-10 leaves errors near 1e-8: a
    GMRES error/residual ratio approaches cond(K)); one step = one st_batch_solve of the batch."""
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2504_07269_gb300 import stfdm

    tol = 1e-12
    probs = synth.batch_problems(64, 5)
    t0 = time.perf_counter()
    hs = stfdm.setup_problems([(pr.n, pr.p_t, pr.t_nodes, pr.Lx, pr.Ly) for pr in probs], device=local)
    setup_s = time.perf_counter() - t0
    Fs, P0 = [], []
    for h, pr in zip(hs, probs):
        psi0, a, bx = synth.batch_inputs(pr)
        P0.append(torch.from_numpy(psi0).to(dev))
        if a is None:
            Fs.append(torch.zeros((pr.n_t, pr.n_x), dtype=torch.complex128, device=dev))
        else:
            f = torch.outer(torch.from_numpy(a).to(dev), torch.from_numpy(bx).to(dev))
            Fs.append(stfdm.st_load_nodal(h, f))
            del f
    psis = [torch.empty_like(F) for F in Fs]
    unknowns = sum(pr.unknowns for pr in probs)
    t0 = time.perf_counter()
    b = stfdm.st_batch_create(hs, tol=tol)
    plan_s = time.perf_counter() - t0
    if args.profile_step:
        _, infos = stfdm.st_batch_solve(b, Fs, P0, psis)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_step": "c5", "stats": stfdm.st_batch_stats_get(b),
                              "sweeps": [i["sweeps"] for i in infos]}))
        return 0
    infos = None

    def step():
        nonlocal infos
        _, infos = stfdm.st_batch_solve(b, Fs, P0, psis)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    t_ms = reduce_max(e0.elapsed_time(e1) / args.steps, world, dev)
    value = world * unknowns / (t_ms * 1e-3)
    stats = stfdm.st_batch_stats_get(b)
    # our kernels per step: the captured cycle's kernel nodes (all but the pending-counter and the
    # m work-counter memsets) per cycle, plus A_x psi0 and psi0 added back per problem and the init
    launches = stats["cycles"] * (stats["graph_nodes"] - 1 - stats["restart"]) + 2 * len(probs) + 1
    # end to end: inputs from pinned host memory, results back, every step
    Fh = [F.cpu().pin_memory() for F in Fs]
    P0h = [p.cpu().pin_memory() for p in P0]
    Ph = [torch.empty(F.shape, dtype=F.dtype).pin_memory() for F in Fs]

    def e2e_step():
        for F, Fhh, p, ph in zip(Fs, Fh, P0, P0h):
            F.copy_(Fhh, non_blocking=True)
            p.copy_(ph, non_blocking=True)
        stfdm.st_batch_solve(b, Fs, P0, psis, want_info=False)
        for o, oh in zip(psis, Ph):
            oh.copy_(o, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        e2e_step()
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1) / args.steps, world, dev)
    h2d = sum(x.numel() * x.element_size() for x in Fh + P0h)
    d2h = sum(x.numel() * x.element_size() for x in Ph)
    # residual of every problem (FP64, separate kernel)
    stfdm.st_batch_solve(b, Fs, P0, psis, want_info=False)
    worst_res = max(stfdm.st_residual(h, F, p, o)[0] for h, F, p, o in zip(hs, Fs, P0, psis))
    # dominant kernel: the persistent factor-and-solve over all 26,570 systems
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        e0.record()
        stfdm.st_batch_spatial_solve(b)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    tk = statistics.median(times)
    # factorisation n_x b^2/2 plus both substitutions 2 n_x b complex MAC per system; b = n per problem
    flops = sum(8.0 * pr.n_t * pr.n_x * (pr.n * pr.n / 2.0 + 2.0 * pr.n) for pr in probs)
    # the plan's workspace (kept factors included) is released before the FP64 reference solves
    stfdm.st_destroy_batch(b)
    torch.cuda.synchronize()
    # the error of three problems against the FP64 FDM, beside that reference's own residual and the
    # error against a tightly refined single solve (FP64 GMRES to 1e-13): at kappa_2(X_t) ~ 1e4 the
    # plain FP64 FDM carries about 1e-9 error itself, so the tight reference says which one is off
    errs, errs_tight, ref_res = {}, {}, {}
    fp64_s = 0.0
    if not args.no_fp64_check:
        sizes = [pr.unknowns for pr in probs]
        for i in sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2])}):
            torch.cuda.synchronize()
            ta = time.perf_counter()
            ref, _ = stfdm.st_fdm_solve(hs[i], Fs[i], P0[i], precision="fp64")
            torch.cuda.synchronize()
            fp64_s += time.perf_counter() - ta
            nref = torch.linalg.vector_norm(ref)
            errs[i] = float(torch.linalg.vector_norm(psis[i] - ref) / nref)
            ref_res[i] = float(stfdm.st_residual(hs[i], Fs[i], P0[i], ref)[0])
            del ref
            tight, _ = stfdm.st_fdm_solve(hs[i], Fs[i], P0[i], precision="mixed", tol=1e-13, max_sweeps=80)
            errs_tight[i] = float(torch.linalg.vector_norm(psis[i] - tight) / torch.linalg.vector_norm(tight))
            del tight
    props = torch.cuda.get_device_properties(dev)
    max_mhz = (clocks or {}).get("sm_max_mhz") or (measured_peaks() or {}).get("sm_max_mhz", 2070.0)
    peak = props.multi_processor_count * 128 * 2 * max_mhz * 1e6 / 1e12
    roof = {"bound": "alu", "kernel": "k_band_batch_v4 (complex64, factor + both substitutions)",
            "achieved": flops / tk / 1e12, "peak": peak, "unit": "TFLOP/s", "frac": flops / tk / 1e12 / peak,
            "traffic": None, "launch_ms": tk * 1e3,
            "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 FMA lanes x 2 x {max_mhz:.0f} MHz (derived)"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic (seeded packets and forcing)",
                "config": {"workload": f"64 uneven problems (n in 32..192, P1/P2, N_t in 32..512, T in 0.5..2), "
                                       f"{unknowns} unknowns, refined to {tol:g}",
                           "name": "c5", "tol": tol, "unknowns": unknowns,
                           "l2_flush": "inputs (5.9 GB c128) larger than the 129 MB L2",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "max_rel_residual": worst_res, "err_vs_fp64": errs, "fp64_fdm_rel_residual": ref_res,
                "err_vs_refined_1e-13": errs_tight, "fp64_fdm_s_for_checked": fp64_s,
                "sweeps": [i["sweeps"] for i in infos], "setup_s": setup_s, "plan_s": plan_s, "batch": stats,
                "e2e": {"value": world * unknowns / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches * args.steps, "roofline": roof, "cpu_baseline": None, "clocks": clocks}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "c5":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
