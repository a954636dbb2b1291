"""Benchmark: converged RPM-FFT solves per second on the 128^3 near-void cell.

One step = one RPM-FFT solve (Algorithm 2 on the map of Eq. 3.9) to the
fixed-point increment tolerance 1e-6 of the 128^3 soft-inclusion cell (RSA
spheres of radius 6-12 voxels, 20 % volume fraction, seed 0, inclusion
E = 1e-3, matrix E = 1, nu = 0.3, C0 = matrix moduli, macroscopic strain
e1 (x) e1, p_max = 20, n_max = 10), through the C ABI on the library's CUDA
kernels.  By default the solve is warm-started: the Accelerated scheme
(Algorithm 3, alpha = beta = 2, C0 at the geometric mean of the phase
moduli) runs until its own increment is 1e-4, then RPM on Eq. 3.9 iterates
from that strain to 1e-6; only the second stage's test decides convergence.
The cold-start form (eps0 = E) is timed in the same run and reported in
config.cold_start (`--form cold` makes it the headline).

The inclusion modulus is 1e-3 rather than the near-void 1e-6: with
E = 1e-6 the fixed-point increment of the basic scheme wrapped by RPM stalls
near 1e-4 (a dense band of interface modes with eigenvalues close to 1; the
FP64 oracle reproduces the stall), so no converged solve exists to time.
E = 1e-3 is the softest inclusion for which RPM with p_max = 20 reaches 1e-6
(the basic scheme alone does not within 5000 steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own seeded cell (weak scaling, no
collective on the data path); rank 0 prints one JSON line.  `--impl
reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
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

import microstructure as ms  # noqa: E402

METRIC = "converged RPM-FFT solves/s at 128^3, tol 1e-6"
UNIT = "solves/s"
N = 128
TOL = 1e-6
P_MAX = 20
E_INCL = 1e-3                       # inclusion modulus (matrix E = 1); see the docstring
WARM_TOL = 1e-4                     # increment at which the warm-start stage hands over
BYTES_PER_VOXEL_GAMMA = 49          # read eps 24 B + phase 1 B, write xi 24 B
L2_FLUSH_BYTES = 256 << 20
PROFILE_EVERY = 16                  # launch groups per CUDA-event sample (opt.profile)


def workload_config(extra: dict | None = None) -> dict:
    cfg = {"workload": "softincl128: RPM-FFT solve, 128^3 cell, RSA spheres r 6-12 vox (seed 0), "
                       "E_incl 1e-3 (near-void 1e-6 stalls above tol), vf 0.20, C0 = matrix, "
                       "E = e1(x)e1, tol 1e-6, p_max 20, n_max 10",
           "e_incl": E_INCL,
           "grid": [N, N, N], "tol": TOL, "p_max": P_MAX, "n_max": 10, "c0_scale": 1.0,
           "load": "e11", "precision": "fp32 fields, fp64 reductions/QR/Newton",
           "l2": "flushed before every timed step (256 MiB write)"}
    if extra:
        cfg.update(extra)
    return cfg


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


def recorded_traffic(key: str):
    """DRAM bytes per launch recorded from an ncu capture (profiles/), or None
    when the kernel sources changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(key)
    if not rec:
        return None
    h = hashlib.sha256()
    for f in ("gamma_kernels.cu", "fft_smem.cuh"):
        with open(os.path.join(ROOT, "paper_2003_07720_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec["dram_bytes_per_launch"] if h.hexdigest()[:16] == rec["source_sha256_16"] else None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"rpm_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_seed(rank: int) -> int:
    """Seed of the cell a rank solves: every rank gets its own microstructure
    (weak scaling over independent cells, no collective on the data path)."""
    return rank


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous share of n_items for one rank (sizes differ by at most 1)."""
    q, r = divmod(n_items, world)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over the default process group (the timing
    rule: the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# RPM iterations of the bounded oracle sample behind cpu_baseline (one basis
# growth included; on the order of 10 s of single-core FP64 work at 128^3)
CPU_SAMPLE_ITERS = 16


def oracle_sample(cell, iters_sample: int = 2) -> dict:
    """Time the FP64 oracle on a bounded sample of the workload: the first
    `iters_sample` RPM iterations (plus the initial F) of the same solve."""
    from oracle import rpm_oracle as o
    prob = o.Problem.from_cell(cell)
    E = ms.unit_strain(0)
    o.apply_F(prob, o.uniform(E, prob.shape), E)       # builds the Green cache, not timed
    t0 = time.perf_counter()
    r = o.rpm_solve(prob, E, o.Options(tol=TOL, p_max=P_MAX, max_iters=iters_sample))
    dt = time.perf_counter() - t0
    return {"seconds": dt, "f_applies": r.f_applies, "sec_per_f": dt / max(r.f_applies, 1)}


def _oracle_sample_worker(args):
    """One process of the all-core oracle sample: builds the benchmark cell
    itself (seeded, so every process solves the same cell) and times the
    bounded oracle sample on it."""
    n, seed, e_incl, iters = args
    cell = ms.cell_nearvoid(n, seed, c0_scale=1.0, e_incl=e_incl)
    return oracle_sample(cell, iters)


def oracle_sample_all_cores(iters: int, workers: int) -> dict:
    """The bounded oracle sample run by `workers` processes at once (one
    independent copy of the same solve per host core; processes started with
    spawn, after CUDA was initialised in this process): F applications per
    second of the whole host."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_sample_worker, [(N, 0, E_INCL, iters)] * workers)
    wall = time.perf_counter() - t0
    f_total = sum(r["f_applies"] for r in res)
    busy = max(r["seconds"] for r in res)
    return {"workers": workers, "f_applies": f_total, "seconds_max_worker": busy,
            "wall_s_incl_startup": wall, "f_per_s": f_total / busy,
            "sec_per_f_per_worker": statistics.median(r["sec_per_f"] for r in res)}


def oracle_reference_iters(form: str = "warm") -> int | None:
    """F applications of the oracle's own converged solve of the workload, in
    the headline form (stored by tests/golden/make_golden.py, oracle only)."""
    name = ("softincl128_warm_oracle_solve.json" if form == "warm"
            else "nearvoid128_oracle_solve.json")
    p = os.path.join(ROOT, "tests", "golden", name)
    if os.path.exists(p):
        with open(p) as f:
            return int(json.load(f)["f_applies"])
    return None


def oracle_error(form: str, mean_stress) -> dict | None:
    """Relative error of the GPU's mean stress against the FP64 oracle's
    converged solve of the cell (stored under tests/golden): its solve of the
    same form where one is stored, else the warm-form solve, which converges
    to the same fixed point of F."""
    name = ("softincl128_warm_oracle_solve.json" if form == "warm"
            else "nearvoid128_oracle_solve.json")
    p = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(p):
        name = "softincl128_warm_oracle_solve.json"
        p = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        ref = np.array(json.load(f)["mean_stress"], float)
    got = np.array(mean_stress, float)
    return {"mean_stress_max_rel": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
            "reference": f"tests/golden/{name}"}


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return
    cell = ms.cell_nearvoid(N, 0, c0_scale=1.0, e_incl=E_INCL)
    nF = oracle_reference_iters(args.form)
    times = []
    for i in range(args.warmup + args.steps):
        s = oracle_sample(cell, 1)
        if i >= args.warmup:
            times.append(s["sec_per_f"])
    sec_per_f = statistics.median(times)
    f_per_solve = nF if nF else None
    value = 1.0 / (sec_per_f * f_per_solve) if f_per_solve else None
    sample = (f"each step: oracle RPM solve of the 128^3 cell bounded to 1 iteration "
              f"(2 F applications); solves/s = 1 / (median s per F x {f_per_solve} F per "
              f"converged oracle solve of the same form ({args.form}), stored under tests/golden)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_per_f * 1e3 * 2,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_solves(ctx, E, steps, warmup, stream, flush, eps_out, raise_ok=True):
    """Warm-up solves, then `steps` timed solves (L2 flushed before each),
    CUDA events on the library's stream.  Returns (device ms, infos)."""
    import torch
    for _ in range(warmup):
        ctx.solve(E, eps_out=eps_out, raise_on_failure=raise_ok)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    infos = []
    torch.cuda.synchronize()
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        st, info = ctx.solve(E, eps_out=eps_out, raise_on_failure=raise_ok)
        ev[k][1].record(stream)
        infos.append(info)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev), infos


def kernel_classes(infos, n_vox: int, pk: dict) -> dict:
    """Rooflines of the two kernel classes of a set of solves, from the CUDA
    events the library records around every k-th launch group of each class
    (opt.profile = k; the sampled time scaled to all groups): the
    Gamma0 application (algorithmic 49 B/voxel per application) and the
    projections (the bytes the library counts for each dots/combine launch)."""
    gamma_ms = sum(i["gamma_ms"] for i in infos)
    n_gamma = sum(i["gamma_applies"] for i in infos)
    proj_ms = sum(i["proj_ms"] for i in infos)
    proj_bytes = sum(i["proj_bytes"] for i in infos)
    t_gamma = gamma_ms / max(n_gamma, 1) / 1e3
    alg_gamma = BYTES_PER_VOXEL_GAMMA * n_vox
    ach_gamma = alg_gamma / t_gamma / 1e9 if t_gamma > 0 else 0.0
    ach_proj = proj_bytes / (proj_ms / 1e3) / 1e9 if proj_ms > 0 else 0.0
    gamma_line = {"bound": "hbm",
                  "kernel": "gamma_apply (pass A+B+C: one F application; in the warm-start stage "
                            "with Algorithm 3's post-step)",
                  "achieved": round(ach_gamma, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                  "frac": round(ach_gamma / pk["hbm_gbs"], 4),
                  "algorithmic_bytes_per_launch": alg_gamma,
                  "avg_launch_ms": round(t_gamma * 1e3, 4), "launches": n_gamma,
                  "total_ms": round(gamma_ms, 3)}
    proj_line = {"bound": "hbm", "kernel": "projections (k_dots + k_reduce + k_combine)",
                 "achieved": round(ach_proj, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": round(ach_proj / pk["hbm_gbs"], 4), "traffic": None,
                 "algorithmic_bytes_per_solve": proj_bytes / max(len(infos), 1),
                 "total_ms": round(proj_ms, 3)}
    return {"gamma_apply": gamma_line, "projections": proj_line}


NEARVOID_C0 = (0.25, 0.5, 1.0, 2.0)
NEARVOID_BUDGET = 1000      # RPM steps (and warm-start steps) per solve of the sweep


def nearvoid_sweep(rpm, stream) -> dict:
    """The near-void cell itself (inclusion E = 1e-6) with C0 at 0.25, 0.5, 1
    and 2 x the matrix moduli, cold and warm-started, each solve capped at a
    fixed step budget: status, steps, increment reached."""
    E = ms.unit_strain(0)
    rows = []
    for scale in NEARVOID_C0:
        cell = ms.cell_nearvoid(N, 0, c0_scale=scale, e_incl=1e-6)
        for form in ("cold", "warm"):
            kw = dict(tol=TOL, p_max=P_MAX, n_max=10, max_iters=NEARVOID_BUDGET)
            if form == "warm":
                kw.update(warm_tol=WARM_TOL, warm_max_iters=NEARVOID_BUDGET)
            with rpm.Context(cell, rpm.rpm_default_options(**kw), stream=stream) as ctx:
                st, info = ctx.solve(E, raise_on_failure=False)
            rows.append({"c0_scale": scale, "form": form, "status": rpm.status_name(st),
                         "iters": info["iters"], "warm_iters": info["warm_iters"],
                         "basis": info["basis_size"], "residual0": info["residual0"],
                         "residual": info["residual"], "F": info["gamma_applies"],
                         "ms": round(info["ms"], 2)})
    return {"cell": "128^3 RSA spheres r 6-12 vox (seed 0), vf 0.20, E_incl 1e-6, matrix E 1",
            "budget_steps": NEARVOID_BUDGET, "tol": TOL, "load": "e11", "rows": rows}


def run_ours(args):
    import torch
    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__ as entry
    entry.build()
    from paper_2003_07720_gb300 import rpm

    cell = ms.cell_nearvoid(N, rank_seed(rank), c0_scale=1.0, e_incl=E_INCL)
    E = ms.unit_strain(0)
    # kernel-class times from CUDA events around every PROFILE_EVERY-th launch
    # group of each class (bracketing every group costs 5 % of the solve)
    opts = rpm.rpm_default_options(tol=TOL, p_max=P_MAX, n_max=10, profile=PROFILE_EVERY)
    if args.max_iters:
        opts.max_iters = args.max_iters          # profiling captures only (not converged)
    if args.scheme == "polarization":
        # Algorithm 3 wrapped by RPM; C0 at the geometric mean of the phase moduli
        cell = ms.Cell(phase=cell.phase, lam=cell.lam, mu=cell.mu,
                       lam0=float(np.sqrt(cell.lam[0] * cell.lam[1])),
                       mu0=float(np.sqrt(cell.mu[0] * cell.mu[1])))
        opts.scheme = rpm.RPM_SCHEME_POLARIZATION
    cold_opts = rpm.rpm_default_options(**{f: getattr(opts, f) for f, _ in opts._fields_})
    if args.form == "warm":
        opts.warm_tol = WARM_TOL
        opts.warm_c0_scale = 1.0
    stream = torch.cuda.current_stream()
    ctx = rpm.Context(cell, opts, stream=stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    eps_out = torch.empty((6, N, N, N), dtype=torch.float32, device="cuda")
    raise_ok = not args.max_iters

    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    if world > 1:
        torch.distributed.barrier()
    wall0 = time.perf_counter()
    dev_ms, infos = time_solves(ctx, E, args.steps, args.warmup, stream, flush, eps_out, raise_ok)
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop() if rank == 0 else None
    dev_ms_max = max_over_ranks(dev_ms, "cuda")
    value = world * args.steps / (dev_ms_max / 1e3)

    # The same solves without the library's event records (opt.profile, which
    # the kernel-class rooflines below come from): what the sampled records
    # cost inside the timed region.
    unprofiled = None
    if world == 1:
        opts_np = rpm.rpm_default_options(**{f: getattr(opts, f) for f, _ in opts._fields_})
        opts_np.profile = 0
        rpm.rpm_set_options(ctx.handle, opts_np)
        np_ms, _ = time_solves(ctx, E, args.steps, 1, stream, flush, eps_out, raise_ok)
        rpm.rpm_set_options(ctx.handle, opts)
        unprofiled = {"value": round(args.steps / (np_ms / 1e3), 4), "unit": UNIT,
                      "ms_per_step": round(np_ms / args.steps, 3),
                      "note": "same timed solves with opt.profile = 0 (no event records); "
                              "the headline brackets every %d-th launch group of each class "
                              "with CUDA events for the rooflines" % PROFILE_EVERY}

    # Kernel classes and their rooflines, from CUDA events the library records
    # on this stream around a sample of launch groups during the timed steps.
    launches = sum(i["launches"] for i in infos)
    pk = peaks()
    classes = kernel_classes(infos, N ** 3, pk)
    gamma_line, proj_line = classes["gamma_apply"], classes["projections"]
    # DRAM bytes per application from the ncu record of the map the timed form
    # applies most: Algorithm 3's map in the warm form, Eq. 3.9 in the cold form
    tr_key = f"polarization_map_{N}" if args.form == "warm" else f"gamma_apply_{N}"
    tr = recorded_traffic(tr_key)
    gamma_line["traffic"] = tr
    gamma_line["traffic_record"] = tr_key
    gamma_line["dram_gbs_from_traffic"] = (round(tr / (gamma_line["avg_launch_ms"] / 1e3) / 1e9, 1)
                                           if tr else None)
    dominant = proj_line if proj_line["total_ms"] >= gamma_line["total_ms"] else gamma_line
    roofline = dict(dominant)
    roofline.update({"peak_src": pk["src"],
                     "time_share": {"gamma_ms": gamma_line["total_ms"],
                                    "projection_ms": proj_line["total_ms"],
                                    "solve_ms": round(dev_ms, 3)},
                     "classes": classes})

    # the cold-start form on the same cell, same timing (comparison inside the line)
    cold = None
    if args.form == "warm" and not args.no_cold:
        ctx_c = rpm.Context(cell, cold_opts, stream=stream)
        c_steps = max(1, min(args.steps, 5))
        c_ms, c_inf = time_solves(ctx_c, E, c_steps, 1, stream, flush, eps_out, raise_ok)
        ctx_c.close()
        cold = {"value": round(c_steps / (c_ms / 1e3), 4), "unit": UNIT, "steps": c_steps,
                "ms_per_step": round(c_ms / c_steps, 3), "iters": c_inf[0]["iters"],
                "basis_size": c_inf[0]["basis_size"],
                "mean_stress_11": c_inf[0]["mean_stress"][0],
                "oracle_rel_err": oracle_error("cold", c_inf[0]["mean_stress"]),
                "launches_per_solve": c_inf[0]["launches"],
                "roofline_classes": kernel_classes(c_inf, N ** 3, pk)}
        cold["roofline_classes"]["gamma_apply"]["traffic"] = recorded_traffic(f"gamma_apply_{N}")

    # the same form with the RPM stage's reference medium at 2x the matrix
    c0x2 = None
    if args.form == "warm" and not args.no_cold and world == 1:
        cell2 = ms.cell_nearvoid(N, rank_seed(rank), c0_scale=2.0, e_incl=E_INCL)
        ctx_2 = rpm.Context(cell2, opts, stream=stream)
        c2_steps = max(1, min(args.steps, 5))
        c2_ms, c2_inf = time_solves(ctx_2, E, c2_steps, 1, stream, flush, eps_out, raise_ok)
        ctx_2.close()
        c0x2 = {"value": round(c2_steps / (c2_ms / 1e3), 4), "unit": UNIT, "steps": c2_steps,
                "iters": c2_inf[0]["iters"], "warm_iters": c2_inf[0]["warm_iters"],
                "gamma_applies": c2_inf[0]["gamma_applies"],
                "mean_stress_11": c2_inf[0]["mean_stress"][0]}

    # BASELINE config 2 itself: the near-void cell at the four reference media
    nearvoid = None
    if args.form == "warm" and not args.no_cold and world == 1:
        nearvoid = nearvoid_sweep(rpm, stream)

    # end to end through the C ABI with host buffers: phase map in, strain field out
    phase_host = np.ascontiguousarray(cell.phase)
    out_host = torch.empty((6, N, N, N), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    e2e_t = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rpm.rpm_set_phase(ctx.handle, phase_host)
        st, info = ctx.solve(E, eps_out=out_host, out_on_host=True, raise_on_failure=raise_ok)
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = world * args.steps / max_over_ranks(sum(e2e_t), "cuda")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nF_gpu = statistics.median(i["gamma_applies"] for i in infos)
        s1 = oracle_sample(cell, CPU_SAMPLE_ITERS)
        ncores = os.cpu_count() or 1
        sa = oracle_sample_all_cores(CPU_SAMPLE_ITERS, ncores)
        cpu = {"value": sa["f_per_s"] / nF_gpu, "unit": UNIT, "cores": ncores, "kind": "oracle",
               "sample": f"{ncores} host processes (one per core, os.cpu_count() = {ncores}), each "
                         f"the oracle RPM solve of this cell bounded to {CPU_SAMPLE_ITERS} "
                         f"iterations ({sa['f_applies']} F applications in all, slowest process "
                         f"{sa['seconds_max_worker']:.1f} s); F applications per second of the "
                         f"whole host divided by the {nF_gpu:g} F applications of the GPU solve",
               "one_core": {"value": 1.0 / (s1["sec_per_f"] * nF_gpu), "unit": UNIT, "cores": 1,
                            "sample": f"the same bounded solve in this process alone "
                                      f"({s1['f_applies']} F applications, {s1['seconds']:.1f} s)"}}
    ctx.close()
    if rank == 0:
        form = ("warm-started: Algorithm 3 (Accelerated, alpha = beta = 2, C0 at the geometric "
                f"mean of the phases) to its increment {WARM_TOL:g}, then RPM on Eq. 3.9 to "
                f"tol {TOL:g}" if args.form == "warm" else "cold start (eps0 = E)")
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(dev_ms_max / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded RSA soft-inclusion cell per rank)",
                "config": workload_config({
                    "form": form, "scheme": args.scheme,
                    "iters": [i["iters"] for i in infos][:3],
                    "warm_iters": [i["warm_iters"] for i in infos][:3],
                    "basis_size": [i["basis_size"] for i in infos][:3],
                    "gamma_applies": [i["gamma_applies"] for i in infos][:3],
                    "residual": [i["residual"] for i in infos][:3],
                    "mean_stress_11": infos[0]["mean_stress"][0],
                    "cold_start": cold,
                    "without_event_records": unprofiled,
                    "c0_2x_matrix": c0x2,
                    "nearvoid_1e-6_c0_sweep": nearvoid,
                    "oracle_rel_err": oracle_error(args.form, infos[0]["mean_stress"]),
                    "parallelism": f"replicas x{world}"}),
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": round(e2e_value, 3), "unit": UNIT,
                        "h2d_bytes_per_step": int(phase_host.nbytes) + 48,
                        "d2h_bytes_per_step": int(out_host.numel() * 4)},
                "gpu_launches": int(launches), "clocks": clocks, "wall_s": round(wall, 3)}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_gamma_only(args):
    """Time the fused Gamma0 application alone (pass A + B + C) on the bench
    cell: `--kernel gamma`.  Prints one JSON line with its HBM roofline."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as entry
    entry.build()
    from paper_2003_07720_gb300 import rpm
    n = args.grid
    cell = (ms.cell_nearvoid(N, 0, c0_scale=1.0, e_incl=E_INCL) if n == N
            else ms.cell_laminate(n, 8, 1e3))
    E = ms.unit_strain(0)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((6, n, n, n), device="cuda", generator=g)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    ctx = rpm.Context(cell, rpm.rpm_default_options(), stream=stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        ctx.apply_gamma(x, E, y)
    ts = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.apply_gamma(x, E, y)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ctx.close()
    t = statistics.median(ts) / 1e3
    pk = peaks()
    ach = BYTES_PER_VOXEL_GAMMA * n ** 3 / t / 1e9
    print(json.dumps({"kernel": "gamma_apply", "grid": [n, n, n], "median_ms": round(t * 1e3, 4),
                      "all_ms": [round(v, 4) for v in ts],
                      "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"],
                                   "unit": "GB/s", "frac": round(ach / pk["hbm_gbs"], 4),
                                   "traffic": recorded_traffic(f"gamma_apply_{n}"),
                                   "algorithmic_bytes_per_launch": BYTES_PER_VOXEL_GAMMA * n ** 3}}),
          flush=True)


def run_study_fibre2d(args):
    """2D fibre-in-matrix study (nz = 1, plane strain), Section 5.1 setting:
    256^2 cell, fibre fraction 0.3 %, nu = 0.25, shear E12 = 0.5 %, contrast
    K = 10 ... 1e5.  Iterations and device time to the increment tolerance for
    the classical scheme, RPM, the Accelerated scheme, RPM around it, and the
    warm-started form.  Prints one JSON line."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as entry
    entry.build()
    from paper_2003_07720_gb300 import rpm
    E = np.zeros(6)
    E[5] = 0.005
    rows = []
    for K in (10.0, 1e2, 1e3, 1e4, 1e5):
        runs = {
            "classical": ("mean", dict(p_max=0)),
            "rpm": ("mean", dict(p_max=20)),
            "accelerated": ("geometric", dict(p_max=0, scheme=rpm.RPM_SCHEME_POLARIZATION)),
            "rpm_accelerated": ("geometric", dict(p_max=20, scheme=rpm.RPM_SCHEME_POLARIZATION)),
            "warm_started": ("mean", dict(p_max=20, warm_tol=1e-4)),
        }
        for name, (c0, kw) in runs.items():
            cell = ms.cell_fibre2d(256, K, c0=c0)
            opts = rpm.rpm_default_options(tol=args.study_tol, max_iters=20000, **kw)
            with rpm.Context(cell, opts) as ctx:
                st, info = ctx.solve(E, raise_on_failure=False)
            rows.append({"K": K, "method": name, "status": int(st), "iters": info["iters"],
                         "warm_iters": info["warm_iters"], "basis": info["basis_size"],
                         "ms": round(info["ms"], 2), "sigma12": info["mean_stress"][5],
                         "residual": info["residual"]})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"study": "fibre2d", "grid": [256, 256, 1], "load": "E12 = 0.005",
                      "tol": args.study_tol, "rows": rows}), flush=True)


NMAX_SWEEP = (1, 2, 5, 10, 20, 50)


def run_study_nmax(args):
    """Section 5.2 setting: RPM on the 2D fibre cell (256^2, C0 = mean,
    p_max 20) with the growth interval n_max in {1, 2, 5, 10, 20, 50} at
    contrast K = 50 and 1e3: steps, final basis size and device time to the
    increment tolerance.  Prints one JSON line."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as entry
    entry.build()
    from paper_2003_07720_gb300 import rpm
    E = np.zeros(6)
    E[5] = 0.005
    rows = []
    for K in (50.0, 1e3):
        cell = ms.cell_fibre2d(256, K, c0="mean")
        for nmax in NMAX_SWEEP:
            opts = rpm.rpm_default_options(tol=args.study_tol, max_iters=20000, p_max=20,
                                           n_max=nmax)
            with rpm.Context(cell, opts) as ctx:
                ctx.solve(E, raise_on_failure=False)          # warm-up (kernel attributes)
                st, info = ctx.solve(E, raise_on_failure=False)
            rows.append({"K": K, "n_max": nmax, "status": rpm.status_name(st),
                         "iters": info["iters"], "basis": info["basis_size"],
                         "F": info["gamma_applies"], "ms": round(info["ms"], 2),
                         "sigma12": info["mean_stress"][5], "residual": info["residual"]})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"study": "nmax", "grid": [256, 256, 1], "load": "E12 = 0.005",
                      "tol": args.study_tol, "p_max": 20, "rows": rows}), flush=True)


def run_study_batch(args):
    """NEXT-1 measurement: C_eff of a set of batched-sweep cells (grids 32^3,
    48^3, 64^3, 96^3; inclusion contrast within [1e-2, 1e2] so that every
    solve converges at tol 1e-6), 6 unit loads each.  Times the cell-by-cell
    form (one context per cell, rpm_effective_stiffness) against the batch
    driver with 1 and with several worker streams, cold and warm-started.
    Prints one JSON line with solves/s per form."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as entry
    entry.build()
    from paper_2003_07720_gb300 import rpm
    cells = []
    s = 0
    while len(cells) < args.batch_cells:
        c = ms.cell_batch_member(s)
        k = c.mu[1] / c.mu[0]
        if 1e-2 <= k <= 1e2:
            cells.append(c)
        s += 1
    n_solves = 6 * len(cells)
    cold = rpm.rpm_default_options(tol=TOL, p_max=P_MAX)
    warm = rpm.rpm_default_options(tol=TOL, p_max=P_MAX, warm_tol=WARM_TOL)
    out = {"study": "batch", "cells": [[int(x) for x in c.shape] + [float(c.mu[1] / c.mu[0])]
                                       for c in cells], "n_solves": n_solves}
    # warm-up (library load, kernel attributes)
    rpm.rpm_effective_stiffness_batch(cells[:1], cold, n_workers=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    C_seq = []
    for c in cells:
        with rpm.Context(c, cold) as ctx:
            C, _, _ = ctx.effective_stiffness()
        C_seq.append(C)
    t_seq = time.perf_counter() - t0
    out["cell_by_cell_cold"] = {"seconds": round(t_seq, 3), "solves_per_s": round(n_solves / t_seq, 2)}
    warm_tuned = rpm.rpm_default_options(tol=TOL, p_max=P_MAX, warm_tol=WARM_TOL, autotune=1)
    for name, opts, workers in (("batch_cold_1", cold, 1), ("batch_cold_w", cold, args.batch_workers),
                                ("batch_warm_w", warm, args.batch_workers),
                                ("batch_warm_w_autotuned", warm_tuned, args.batch_workers)):
        t0 = time.perf_counter()
        Cb, infos, stat, st = rpm.rpm_effective_stiffness_batch(cells, opts, n_workers=workers,
                                                                raise_on_failure=False)
        dt = time.perf_counter() - t0
        err = max(float(np.max(np.abs(Cb[i] - C_seq[i])) / np.max(np.abs(C_seq[i])))
                  for i in range(len(cells)))
        out[name] = {"workers": workers, "seconds": round(dt, 3),
                     "solves_per_s": round(n_solves / dt, 2), "status": int(st),
                     "max_rel_diff_vs_cell_by_cell": err}
    print(json.dumps(out), flush=True)


def run_study_c4(args):
    """The batched effective-stiffness sweep as specified: 96 seeded cells
    (grids 32^3, 48^3, 64^3, 96^3 by seed mod 4; spheres to a volume fraction
    U(0.1, 0.35); inclusion contrast 10^U(-6, 3); C0 = mean) x 6 unit loads
    through rpm_effective_stiffness_batch (worker streams), each solve capped
    at a step budget.  Reports solves/s and, per cell, the status of every
    load, the steps and the 6 x 6 C_eff.  Prints one JSON line."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as entry
    entry.build()
    from paper_2003_07720_gb300 import rpm
    cells = [ms.cell_batch_member(s) for s in range(args.c4_cells)]
    budget = args.c4_budget
    forms = {"cold": rpm.rpm_default_options(tol=TOL, p_max=P_MAX, max_iters=budget),
             "warm": rpm.rpm_default_options(tol=TOL, p_max=P_MAX, max_iters=budget,
                                             warm_tol=WARM_TOL, warm_max_iters=budget)}
    rpm.rpm_effective_stiffness_batch(cells[:1], forms["cold"], n_workers=1,
                                      raise_on_failure=False)      # warm-up
    torch.cuda.synchronize()
    out = {"study": "c4", "cells": len(cells), "loads": 6, "budget_steps": budget, "tol": TOL,
           "workers": args.batch_workers}
    for name, opts in forms.items():
        t0 = time.perf_counter()
        C, infos, stat, st = rpm.rpm_effective_stiffness_batch(cells, opts,
                                                               n_workers=args.batch_workers,
                                                               raise_on_failure=False)
        dt = time.perf_counter() - t0
        rows = []
        for i, c in enumerate(cells):
            inf = infos[i]
            rows.append({"seed": i, "grid": int(c.shape[0]),
                         "contrast": float(c.mu[1] / c.mu[0]),
                         "volume_fraction": round(float(c.phase.mean()), 4),
                         "status": rpm.status_name(stat[i]),
                         "converged_loads": int(sum(1 for j in inf if j["converged"])),
                         "steps": [int(j["iters"]) for j in inf],
                         "basis_reused": [int(j["basis_reused"]) for j in inf],
                         "C_eff": [[float("%.7g" % v) for v in row] for row in C[i]]})
        conv = [r for r in rows if r["converged_loads"] == 6]
        out[name] = {"seconds": round(dt, 3), "solves_per_s": round(6 * len(cells) / dt, 2),
                     "steps": int(sum(sum(r["steps"]) for r in rows)),
                     "cells_all_loads_converged": len(conv),
                     "solves_converged": int(sum(r["converged_loads"] for r in rows)),
                     "rows": rows}
        print(json.dumps({k: v for k, v in out[name].items() if k != "rows"}), file=sys.stderr,
              flush=True)
    print(json.dumps(out), flush=True)


def fno_flops_per_sample(n: int, m: int, layers: int, width: int = 16) -> dict:
    """Algorithmic FLOPs of one sample through the spectral neural operator
    (truncated DFT stages as sums over N points per kept frequency; a real x
    complex term is 4 flops, a complex multiply-add 8): forward, and forward
    plus backward (the backward repeats the forward transform of dz, the
    spectral mixing twice (dV and the R gradient), the inverse transforms and
    the pointwise maps twice)."""
    W = width
    per_ch = 4 * m * n ** 3 + 16 * m * m * n * n + 32 * m ** 3 * n      # x, y, z forward
    inv_ch = 32 * m ** 3 * n + 16 * m * m * n * n + 4 * m * n ** 3      # z, y, x inverse
    mix = 32 * m ** 3 * W * W
    pw = 2 * n ** 3 * W * W
    fwd_layer = W * (per_ch + inv_ch) + mix + pw
    bwd_layer = W * (per_ch + inv_ch) + 2 * mix + 2 * pw + 2 * n ** 3 * W * W   # + gA tiles
    head = 2 * n ** 3 * (36 * W + 36)
    return {"forward": layers * fwd_layer + head,
            "train": layers * (fwd_layer + bwd_layer) + 3 * head}


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def run_fno_kernel(args):
    """Time one loss-and-gradient pass of the spectral neural operator (64^3,
    12 modes, 4 layers, width 16, batch 8) on random inputs: `--kernel fno`.
    Prints one JSON line with its FP32-ALU roofline."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as entry
    entry.build()
    from paper_2003_07720_gb300 import fno
    n, m, L, B = args.fno_n, 12, 4, args.fno_batch
    g = torch.Generator(device="cuda").manual_seed(0)
    feat = torch.randn((B, 2, n, n, n), device="cuda", generator=g)
    tgt = torch.randn((B, 6, n, n, n), device="cuda", generator=g)
    E = np.stack([ms.strain_direction(i) for i in range(B)])
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    with fno.Fno(n, m, L, max_batch=B, stream=stream, precision=args.fno_precision) as net:
        net.set_params(ms.fno_params(m, L, seed=0))
        for _ in range(args.warmup):
            net.loss_grad(feat, E, tgt)
        ts = []
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            net.loss_grad(feat, E, tgt)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
    t = statistics.median(ts) / 1e3
    fl = fno_flops_per_sample(n, m, L)
    ach = fl["train"] * B / t / 1e12
    print(json.dumps({"kernel": "fno_loss_grad", "precision": args.fno_precision,
                      "grid": [n, n, n], "batch": B, "modes": m,
                      "layers": L, "median_ms": round(t * 1e3, 4),
                      "all_ms": [round(v, 4) for v in ts],
                      "roofline": {"bound": "alu", "achieved": round(ach, 2),
                                   "peak": round(FP32_PEAK_TFLOPS, 1), "unit": "TFLOP/s",
                                   "frac": round(ach / FP32_PEAK_TFLOPS, 4),
                                   "flops_per_launch_group": fl["train"] * B}}), flush=True)


def run_study_fno(args):
    """NEXT-2 measurement: train the spectral neural operator on solver
    solutions of cell_fno_member cells (64^3), then compare, on held-out
    cells at 64^3 and 128^3, the solve from eps0 = E, from the Algorithm 3
    warm-start stage, from the learned guess and from the learned guess
    followed by the stage.  Prints one JSON line."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as entry
    entry.build()
    from paper_2003_07720_gb300 import fno, fno_train
    n, m, L, B = args.fno_n, 12, 4, args.fno_batch
    out = {"study": "fno", "grid": n, "modes": m, "layers": L, "width": 16, "batch": B}
    seeds = list(range(1000, 1000 + args.fno_train))
    data = fno_train.make_dataset(n, seeds)
    out["dataset"] = {"cells": len(seeds), "solve_seconds": round(data.solve_s, 2),
                      "converged": int(data.converged.sum()), "train_samples": len(data.seeds)}
    net = fno.Fno(n, m, L, max_batch=B, precision=args.fno_precision)
    net.set_params(ms.fno_params(m, L, seed=0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = fno_train.train(net, data, args.fno_epochs, B, lr=args.fno_lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out["training"] = {"epochs": args.fno_epochs, "seconds": round(t_train, 2), "lr": args.fno_lr,
                       "samples_per_s": round(args.fno_epochs * (len(data.seeds) // B) * B
                                              / t_train, 1),
                       "loss_per_epoch": [float("%.5g" % v) for v in hist],
                       "target_mean_square": float((data.target ** 2).mean().item())}
    del data
    torch.cuda.empty_cache()
    params = net.get_params()
    net.close()
    test = list(range(5000, 5000 + args.fno_test))
    res = {}
    for nn in (n, 2 * n):
        with fno.Fno(nn, m, L, max_batch=1, precision=args.fno_precision) as net2:
            net2.set_params(params)
            rows = fno_train.evaluate(net2, nn, test)
        summ = {}
        both = [r for r in rows if all(r[f]["converged"] for f in ("cold", "learned"))]
        for form in ("cold", "alg3_stage", "learned", "learned_alg3_stage"):
            ok = [r[form] for r in rows if r[form]["converged"]]
            summ[form] = {"converged": len(ok),
                          "median_F": float(np.median([r["F"] for r in ok])) if ok else None,
                          "median_ms": float(np.median([r["ms"] + r["guess_ms"] for r in ok]))
                          if ok else None,
                          "F_on_cells_cold_and_learned_both_converge":
                              int(sum(r[form]["F"] for r in both))}
        res[str(nn)] = {"summary": summ, "rows": rows}
    out["evaluation"] = res
    if args.fno_save:
        np.save(args.fno_save, params)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="warm", choices=["warm", "cold"],
                    help="warm: Algorithm 3 warm start then RPM (default); cold: eps0 = E")
    ap.add_argument("--no-cold", action="store_true", help="skip the cold-start comparison")
    ap.add_argument("--scheme", default="basic", choices=["basic", "polarization"],
                    help="fixed-point map wrapped by RPM (polarization: Algorithm 3, C0 at the "
                         "geometric mean)")
    ap.add_argument("--max-iters", type=int, default=0,
                    help="cap the solve (profiling captures only; the result is not converged)")
    ap.add_argument("--fno-n", type=int, default=64)
    ap.add_argument("--fno-train", type=int, default=2000)
    ap.add_argument("--fno-test", type=int, default=20)
    ap.add_argument("--fno-epochs", type=int, default=60)
    ap.add_argument("--fno-batch", type=int, default=8)
    ap.add_argument("--fno-lr", type=float, default=2e-3)
    ap.add_argument("--fno-save", default="", help="write the trained parameters (.npy)")
    ap.add_argument("--fno-precision", default="bf16", choices=["bf16", "fp32"],
                    help="network transforms: BF16 tensor cores (default) or float32")
    ap.add_argument("--study", default=None,
                    choices=[None, "fibre2d", "nmax", "batch", "c4", "fno"],
                    help="run a study instead of the benchmark")
    ap.add_argument("--study-tol", type=float, default=1e-6)
    ap.add_argument("--grid", type=int, default=N, help="cube size for --kernel gamma "
                    "(the benchmark cell at 128, a laminate otherwise)")
    ap.add_argument("--batch-cells", type=int, default=16)
    ap.add_argument("--batch-workers", type=int, default=8)
    ap.add_argument("--c4-cells", type=int, default=96)
    ap.add_argument("--c4-budget", type=int, default=2000, help="step budget per solve")
    ap.add_argument("--kernel", default=None, choices=[None, "gamma", "fno"],
                    help="time one kernel group alone instead of the solve")
    args = ap.parse_args()
    if args.study == "fibre2d":
        run_study_fibre2d(args)
    elif args.study == "nmax":
        run_study_nmax(args)
    elif args.study == "batch":
        run_study_batch(args)
    elif args.study == "c4":
        run_study_c4(args)
    elif args.study == "fno":
        run_study_fno(args)
    elif args.kernel == "fno":
        run_fno_kernel(args)
    elif args.kernel == "gamma":
        run_gamma_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
