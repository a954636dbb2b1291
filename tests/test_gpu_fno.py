"""Parity of the learned warm start (include/rpm_fno.h) with the FP64
reference oracle/fno_oracle.py, through the C ABI: network forward, loss and
every parameter gradient, Adam, voxel features, the compatible projection of
rpm_apply_gamma and the warm-started solve.

Tolerances: the CUDA path computes in float32 with sums of at most N terms
per transform stage (relative rounding ~1e-6 per stage, four stages per
layer, up to four layers): outputs agree to 2e-4 of their largest magnitude,
gradients to 1e-3 in relative L2 per parameter group."""
import numpy as np
import pytest

import microstructure as ms
from oracle import fno_oracle as fo
from oracle import rpm_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT_TOL = 2e-4
GRAD_TOL = 1e-3
# BF16 tensor-core transforms (precision "bf16"): every truncated DFT stage
# rounds its operands to bfloat16 (unit roundoff 2^-9 ~ 2e-3) and accumulates
# in float32; a layer chains two such stages forward (and the backward two
# more), so outputs are held to 2e-2 of their largest magnitude and gradient
# groups to 5e-2 in relative L2.
BF16_OUT_TOL = 2e-2
BF16_GRAD_TOL = 5e-2


@pytest.fixture(scope="module")
def fno():
    from paper_2003_07720_gb300 import fno as f
    return f


def _inputs(N, B, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    ph = (rng.random((B, N, N, N)) < 0.3).astype(np.int64)
    feat = np.stack([np.where(ph == 1, rng.uniform(-2, 2, size=(B, 1, 1, 1)), 0.0),
                     np.where(ph == 1, 0.25, 0.3)], axis=1)          # [B, 2, N, N, N]
    E = np.stack([ms.strain_direction(seed * 10 + b) for b in range(B)])
    return feat, E


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _params(m, L, seed, scale_r=8.0):
    p = ms.fno_params(m, L, seed=seed)
    for l in range(L):
        p[f"R{l}"] *= scale_r          # make the spectral branch carry weight
        p[f"a{l}"] = 0.05 * np.random.Generator(np.random.PCG64(seed + l)).standard_normal(16)
    p["p"] = 0.1 * np.ones(16)
    p["q"] = 0.01 * np.arange(36)
    return p


def _round32(p):
    return {k: (v.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(v)
                else np.asarray(v, np.float32).astype(np.float64)) for k, v in p.items()}


@pytest.mark.parametrize("N,m,L,B", [(32, 12, 4, 2), (48, 8, 2, 1), (40, 5, 1, 3), (24, 12, 2, 1)])
def test_forward_matches_oracle(fno, N, m, L, B):
    p = _round32(_params(m, L, 100 + N))
    feat, E = _inputs(N, B, N)
    ref = fo.forward(p, feat, E.astype(np.float32).astype(np.float64), m, L)
    out = torch.empty((B, 6, N, N, N), device="cuda")
    with fno.Fno(N, m, L, max_batch=B, precision="fp32") as net:
        net.set_params(p)
        net.forward(_dev(feat), E, out)
        torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < OUT_TOL, err


def test_loss_and_every_gradient_match_oracle(fno):
    N, m, L, B = 32, 6, 3, 2
    p = _round32(_params(m, L, 7))
    feat, E = _inputs(N, B, 3)
    rng = np.random.Generator(np.random.PCG64(4))
    target = rng.standard_normal((B, 6, N, N, N)).astype(np.float32).astype(np.float64)
    E = E.astype(np.float32).astype(np.float64)
    loss_ref, g_ref = fo.backward(p, feat, E, target, m, L)
    with fno.Fno(N, m, L, max_batch=B, precision="fp32") as net:
        net.set_params(p)
        loss = net.loss_grad(_dev(feat), E, _dev(target))
        g1 = net.get_grads()
        net.loss_grad(_dev(feat), E, _dev(target))
        g2 = net.get_grads()
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    assert np.array_equal(g1, g2), "gradients must be deterministic"
    g = fno.unpack_params(g1, m, L)
    for k in g_ref:
        a, b = g[k], g_ref[k]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel < GRAD_TOL, (k, rel)


def test_adam_step_matches_definition(fno):
    N, m, L, B = 24, 3, 1, 1
    p = _params(m, L, 11)
    feat, E = _inputs(N, B, 5)
    target = np.zeros((B, 6, N, N, N))
    opt = dict(lr=1e-2, beta1=0.8, beta2=0.95, eps=1e-6, weight_decay=0.1)
    with fno.Fno(N, m, L, max_batch=B, precision="fp32") as net:
        net.set_params(p)
        p0 = net.get_params().astype(np.float64)
        m1 = np.zeros_like(p0)
        m2 = np.zeros_like(p0)
        cur = p0
        for t in (1, 2):
            net.loss_grad(_dev(feat), E, _dev(target))
            g = net.get_grads().astype(np.float64)
            net.adam_step(**opt)
            cur, m1, m2 = fo.adam_step(cur, g, m1, m2, t, opt["lr"], opt["beta1"], opt["beta2"],
                                       opt["eps"], opt["weight_decay"])
            got = net.get_params().astype(np.float64)
            assert np.max(np.abs(got - cur)) < 1e-5 * max(1.0, np.max(np.abs(cur)))


def test_features_match_oracle(fno):
    N = 16
    rng = np.random.Generator(np.random.PCG64(8))
    ph = rng.integers(0, 3, size=(N, N, N)).astype(np.uint8)
    lam = [ms.lame(1.0, 0.3)[0], ms.lame(1e-3, 0.2)[0], ms.lame(50.0, 0.35)[0]]
    mu = [ms.lame(1.0, 0.3)[1], ms.lame(1e-3, 0.2)[1], ms.lame(50.0, 0.35)[1]]
    out = torch.empty((2, N, N, N), device="cuda")
    fno.features(torch.from_numpy(ph).cuda(), list(zip(lam, mu)), out)
    torch.cuda.synchronize()
    ref = fo.features(ph, lam, mu)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-6


def test_projection_matches_oracle():
    from paper_2003_07720_gb300 import rpm
    cell = ms.cell_fno_member(1000, 32)
    prob = o.Problem.from_cell(cell)
    E = ms.strain_direction(0)
    rng = np.random.Generator(np.random.PCG64(9))
    x = rng.standard_normal((6,) + cell.shape)
    out = torch.empty((6,) + cell.shape, device="cuda")
    with rpm.Context(cell, rpm.rpm_default_options()) as ctx:
        ctx.apply_gamma(_dev(x), E, out, rpm.RPM_GAMMA_PROJECT)
        torch.cuda.synchronize()
    ref = o.project_compatible(prob, x, E)
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) < 1e-5 * np.max(np.abs(ref))


def test_warm_started_solve_matches_cold(fno):
    """An untrained network still gives a valid start: the guess has mean E,
    and the solve from it converges to the cold solve's answer."""
    from paper_2003_07720_gb300 import rpm
    N, m, L = 32, 6, 2
    cell = ms.cell_fno_member(1001, N)
    E = 0.01 * ms.strain_direction(1)
    opts = rpm.rpm_default_options(tol=1e-6, p_max=20)
    eps0 = torch.empty((6, N, N, N), device="cuda")
    with fno.Fno(N, m, L, precision="fp32") as net, rpm.Context(cell, opts) as ctx:
        net.set_params(_params(m, L, 12))
        net.warm_start(ctx, E, eps0)
        mean = eps0.double().mean(dim=(1, 2, 3)).cpu().numpy()
        assert np.allclose(mean, E, atol=1e-6 * np.max(np.abs(E)) + 1e-9)
        st1, cold = ctx.solve(E)
        st2, warm = ctx.solve(E, eps0=eps0)
    assert cold["converged"] and warm["converged"]
    a, b = np.array(cold["mean_stress"]), np.array(warm["mean_stress"])
    assert np.max(np.abs(a - b)) < 1e-4 * np.max(np.abs(a))


def test_training_lowers_the_loss(fno):
    """A few Adam steps on one sample: the loss falls (optimizer and
    gradients in the same direction as the loss)."""
    N, m, L, B = 32, 4, 2, 2
    feat, E = _inputs(N, B, 13)
    # a target linear in E with a pointwise localisation: eps_o = E_o (1 + tanh f0)
    target = E[:, :, None, None, None] * (1.0 + np.tanh(feat[:, :1]))
    with fno.Fno(N, m, L, max_batch=B, precision="fp32") as net:
        net.set_params(ms.fno_params(m, L, seed=14))
        f, t = _dev(feat), _dev(target)
        l0 = net.train_step(f, E, t, lr=3e-3)
        for _ in range(60):
            l1 = net.train_step(f, E, t, lr=3e-3)
    assert l1 < 0.5 * l0, (l0, l1)


def test_bad_arguments(fno):
    from paper_2003_07720_gb300 import rpm
    with fno.Fno(32, 4, 1, max_batch=1, precision="fp32") as net:
        feat = torch.zeros((2, 2, 32, 32, 32), device="cuda")
        out = torch.empty((2, 6, 32, 32, 32), device="cuda")
        with pytest.raises(fno.FnoError):
            net.forward(feat, np.zeros((2, 6)), out)          # batch above max_batch
        cell = ms.cell_fno_member(1002, 48)
        with rpm.Context(cell, rpm.rpm_default_options()) as ctx:
            eps0 = torch.empty((6, 48, 48, 48), device="cuda")
            with pytest.raises(fno.FnoError):
                net.warm_start(ctx, ms.strain_direction(0), eps0)   # grid mismatch
        cell = ms.cell_fno_member(1003, 32)
        with rpm.Context(cell, rpm.rpm_default_options()) as ctx:
            eps0 = torch.empty((6, 32, 32, 32), device="cuda")
            with pytest.raises(fno.FnoError):
                net.warm_start(ctx, np.zeros(6), eps0)             # E = 0


def test_warm_stage_from_uniform_eps0_equals_default_warm_form():
    """warm_from_eps0 = 1 with eps0 = E everywhere follows exactly the
    trajectory of the default warm form (which starts from E)."""
    from paper_2003_07720_gb300 import rpm
    N = 32
    cell = ms.cell_fno_member(1004, N)
    E = 0.01 * ms.strain_direction(4)
    eps0 = torch.from_numpy(np.broadcast_to(E[:, None, None, None], (6, N, N, N))
                            .astype(np.float32).copy()).cuda()
    with rpm.Context(cell, rpm.rpm_default_options(warm_tol=1e-4)) as ctx:
        _, a = ctx.solve(E)
        rpm.rpm_set_options(ctx.handle, rpm.rpm_default_options(warm_tol=1e-4, warm_from_eps0=1))
        _, b = ctx.solve(E, eps0=eps0)
    assert a["converged"] and b["converged"]
    assert (a["warm_iters"], a["iters"], a["gamma_applies"]) == (b["warm_iters"], b["iters"],
                                                                 b["gamma_applies"])
    assert a["mean_stress"] == b["mean_stress"]


def test_trained_network_gain_is_measured(fno):
    """Train the network (BF16 tensor-core transforms, as the 64^3 study) on
    solver solutions (48 cells at 32^3, as the 64^3 study does at a smaller
    size), then solve held-out cells from the
    cold start and from the learned guess.  Where both converge they reach
    the same answer; the gain (cold minus learned F applications) and the
    learned starts that fail are reported, not asserted: the 64^3 study finds
    the gain near zero or negative, and on soft-inclusion cells Algorithm 2 on
    Eq. 3.9 can diverge from a perturbed start where the start from E
    converges (cell_fno_member(5004) at 32^3 diverges after 182 steps in the
    FP64 oracle as on the GPU)."""
    from paper_2003_07720_gb300 import fno_train
    N, m, L, B = 32, 12, 4, 8
    data = fno_train.make_dataset(N, list(range(1000, 1048)))
    assert len(data.seeds) >= 24
    with fno.Fno(N, m, L, max_batch=B, precision="bf16") as net:
        net.set_params(ms.fno_params(m, L, seed=0))
        hist = fno_train.train(net, data, epochs=30, batch=B, lr=4e-3)
        assert hist[-1] < 0.9 * hist[0], hist
        rows = fno_train.evaluate(net, N, list(range(5000, 5006)))
        gains, failed = [], []
        for r in rows:
            if not r["cold"]["converged"]:
                continue
            if not r["learned"]["converged"]:
                failed.append(r["seed"])
                # rpm_fno_solve falls back to the cold start and reaches its answer
                from paper_2003_07720_gb300 import rpm
                cell = ms.cell_fno_member(r["seed"], N)
                with rpm.Context(cell, rpm.rpm_default_options()) as ctx:
                    st, info, used = net.solve(ctx, 0.01 * ms.strain_direction(r["seed"]))
                assert st == rpm.RPM_OK and info["converged"] and not used, info
                a = np.array(r["cold"]["mean_stress"])
                assert np.max(np.abs(np.array(info["mean_stress"]) - a)) < 1e-4 * np.max(np.abs(a))
                continue
            a, b = np.array(r["cold"]["mean_stress"]), np.array(r["learned"]["mean_stress"])
            assert np.max(np.abs(a - b)) < 1e-4 * np.max(np.abs(a)), r
            gains.append(r["cold"]["F"] - r["learned"]["F"])
    assert gains, rows
    print("F saved by the learned start per held-out cell:", gains,
          "; learned starts that did not converge (cold did):", failed)


@pytest.mark.parametrize("N,m,L,B", [(32, 12, 4, 2), (48, 8, 2, 1), (64, 12, 4, 2), (32, 5, 1, 3)])
def test_forward_bf16_tensor_cores_matches_oracle(fno, N, m, L, B):
    """The BF16 tensor-core transforms against the FP64 reference network."""
    p = _round32(_params(m, L, 300 + N))
    feat, E = _inputs(N, B, N + 1)
    ref = fo.forward(p, feat, E.astype(np.float32).astype(np.float64), m, L)
    out = torch.empty((B, 6, N, N, N), device="cuda")
    with fno.Fno(N, m, L, max_batch=B, precision="bf16") as net:
        net.set_params(p)
        net.forward(_dev(feat), E, out)
        torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert np.all(np.isfinite(got))
    print(f"bf16 forward N={N} m={m} L={L}: max rel err {err:.2e}")
    assert err < BF16_OUT_TOL, err


def test_bf16_loss_and_gradients_match_oracle(fno):
    N, m, L, B = 32, 6, 3, 2
    p = _round32(_params(m, L, 7))
    feat, E = _inputs(N, B, 3)
    rng = np.random.Generator(np.random.PCG64(4))
    target = rng.standard_normal((B, 6, N, N, N)).astype(np.float32).astype(np.float64)
    E = E.astype(np.float32).astype(np.float64)
    loss_ref, g_ref = fo.backward(p, feat, E, target, m, L)
    with fno.Fno(N, m, L, max_batch=B, precision="bf16") as net:
        net.set_params(p)
        loss = net.loss_grad(_dev(feat), E, _dev(target))
        g1 = net.get_grads()
        net.loss_grad(_dev(feat), E, _dev(target))
        g2 = net.get_grads()
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    assert np.array_equal(g1, g2), "gradients must be deterministic"
    g = fno.unpack_params(g1, m, L)
    for k in g_ref:
        a, b = g[k], g_ref[k]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        print(f"bf16 gradient {k}: rel L2 err {rel:.2e}")
        assert rel < BF16_GRAD_TOL, (k, rel)
