"""Training and evaluation of the learned warm start (include/rpm_fno.h).

Data: cells of microstructure.cell_fno_member on an n^3 grid, each with its
own strain direction (microstructure.strain_direction); the target is the
fluctuation eps - E of the strain field the solver (rpm_solve) returns for
that cell and direction (rpm_fno_warm_start projects the network output onto
the compatible fields of mean E, so a fluctuation is all it needs).
Inputs are the voxel features (rpm_fno_features) and the direction.

Everything numerical runs in the CUDA library: the solves, the features, the
network's forward and backward passes and Adam.  This module sequences the
calls and keeps the data resident on the device.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

import microstructure as ms

from . import fno, rpm


@dataclasses.dataclass
class Dataset:
    n: int
    seeds: list
    feat: object          # torch [S, 2, n, n, n] float32 (device)
    E: np.ndarray         # [S, 6] unit directions
    target: object        # torch [S, 6, n, n, n] float32 (device)
    converged: np.ndarray
    solve_s: float


def _phase_list(cell):
    return list(zip(np.asarray(cell.lam, float), np.asarray(cell.mu, float)))


def make_dataset(n: int, seeds, options=None, stream=None) -> Dataset:
    """Solve each training cell once; targets stay on the device."""
    import torch
    S = len(seeds)
    feat = torch.empty((S, 2, n, n, n), device="cuda")
    target = torch.empty((S, 6, n, n, n), device="cuda")
    E = np.stack([ms.strain_direction(s) for s in seeds])
    conv = np.zeros(S, bool)
    opts = options or rpm.rpm_default_options(warm_tol=1e-4, max_iters=1000)
    first = ms.cell_fno_member(seeds[0], n)
    t0 = time.perf_counter()
    with rpm.Context(first, opts, stream=stream) as ctx:
        for i, s in enumerate(seeds):
            cell = first if i == 0 else ms.cell_fno_member(s, n)
            if i:
                rpm.rpm_set_phase(ctx.handle, cell.phase)
                rpm.rpm_set_materials(ctx.handle, _phase_list(cell), (cell.lam0, cell.mu0))
            st, info = ctx.solve(E[i], eps_out=target[i], raise_on_failure=False)
            conv[i] = info["converged"]
            target[i] -= torch.tensor(E[i], dtype=torch.float32, device="cuda").view(6, 1, 1, 1)
            ph = torch.from_numpy(np.ascontiguousarray(cell.phase, np.uint8)).cuda()
            fno.features(ph, _phase_list(cell), feat[i], stream=stream)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # train only on solutions that met the stopping test (compacted in place
    # by device copies, front to back)
    keep = np.flatnonzero(conv)
    if len(keep) < S:
        for j, i in enumerate(keep):
            if i != j:
                feat[j].copy_(feat[i])
                target[j].copy_(target[i])
        feat, target = feat[:len(keep)], target[:len(keep)]
        E = E[keep]
    return Dataset(n, [seeds[i] for i in keep], feat, E, target, conv, dt)


def train(net: "fno.Fno", data: Dataset, epochs: int, batch: int, lr: float = 2e-3,
          lr_final: float = 1e-4, seed: int = 0, log=None):
    """Adam with a cosine learning-rate decay; one pass over the (shuffled)
    training cells per epoch.  Returns the mean loss of each epoch."""
    import torch
    S = len(data.seeds)
    rng = np.random.Generator(np.random.PCG64(seed))
    steps = epochs * (S // batch)
    hist = []
    k = 0
    net.epoch_s = []
    fb = torch.empty((batch,) + tuple(data.feat.shape[1:]), device="cuda")
    tb = torch.empty((batch,) + tuple(data.target.shape[1:]), device="cuda")
    for ep in range(epochs):
        te = time.perf_counter()
        order = rng.permutation(S)
        tot = 0.0
        nb = 0
        for j in range(0, S - batch + 1, batch):
            for q, i in enumerate(order[j:j + batch]):    # gather by device copies
                fb[q].copy_(data.feat[int(i)])
                tb[q].copy_(data.target[int(i)])
            e = data.E[order[j:j + batch]]
            a = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * k / max(steps - 1, 1)))
            tot += net.train_step(fb, e, tb, lr=float(a))
            nb += 1
            k += 1
        hist.append(tot / max(nb, 1))
        net.epoch_s.append(time.perf_counter() - te)
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def evaluate(net: "fno.Fno", n: int, seeds, options=None):
    """Per held-out cell: F applications and device time of the solve from
    (a) eps0 = E, (b) the Algorithm 3 warm-start stage, (c) the learned guess,
    (d) the learned guess followed by the Algorithm 3 stage.  All four end at
    the same stopping test."""
    import torch
    base = options or rpm.rpm_default_options()
    forms = {
        "cold": dict(warm_tol=0.0),
        "alg3_stage": dict(warm_tol=1e-4),
        "learned": dict(warm_tol=0.0),
        "learned_alg3_stage": dict(warm_tol=1e-4, warm_from_eps0=1),
    }
    rows = []
    eps0 = torch.empty((6, n, n, n), device="cuda")
    for s in seeds:
        cell = ms.cell_fno_member(s, n)
        E = 0.01 * ms.strain_direction(s)
        row = {"seed": s}
        with rpm.Context(cell, base) as ctx:
            for name, kw in forms.items():
                o = rpm.rpm_default_options(**{f: getattr(base, f) for f, _ in base._fields_})
                for key, v in kw.items():
                    setattr(o, key, v)
                rpm.rpm_set_options(ctx.handle, o)
                t0 = time.perf_counter()
                start = None
                if name.startswith("learned"):
                    net.warm_start(ctx, E, eps0)
                    start = eps0
                t_net = time.perf_counter() - t0
                st, info = ctx.solve(E, eps0=start, raise_on_failure=False)
                row[name] = {"converged": info["converged"], "F": info["gamma_applies"],
                             "iters": info["iters"], "warm_iters": info["warm_iters"],
                             "ms": info["ms"], "guess_ms": round(t_net * 1e3, 3),
                             "residual": info["residual"],
                             "mean_stress": list(info["mean_stress"])}
        rows.append(row)
    return rows
