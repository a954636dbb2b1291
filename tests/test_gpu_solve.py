"""Parity of the CUDA solvers (Algorithm 1 and Algorithm 2) with the FP64
oracle, through the C ABI, plus the error paths."""
import numpy as np
import pytest

import microstructure as ms
from oracle import rpm_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CEFF_TOL = 1e-5     # effective stiffness, relative to max |C_eff|
FIELD_TOL = 1e-4    # strain field, relative L2


@pytest.fixture(scope="module")
def rpm():
    from paper_2003_07720_gb300 import rpm as r
    return r


@pytest.fixture(scope="module")
def sphere32():
    cell = ms.cell_sphere32(32)
    prob = o.Problem.from_cell(cell)
    ref = o.rpm_solve(prob, ms.unit_strain(0), o.Options(tol=1e-11, p_max=20))
    return cell, prob, ref


@pytest.mark.parametrize("p_max", [0, 10])
def test_sphere32_solve_matches_oracle(rpm, sphere32, p_max):
    cell, prob, ref = sphere32
    E = ms.unit_strain(0)
    eps = torch.empty((6,) + cell.shape, device="cuda")
    sig = torch.empty_like(eps)
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=p_max)) as ctx:
        st, info = ctx.solve(E, eps_out=eps, sig_out=sig)
    assert info["converged"] and info["residual"] <= 1e-6
    if p_max == 0:
        assert info["basis_size"] == 0
    else:
        assert info["basis_size"] > 0
    e = eps.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(e - ref.eps) / np.linalg.norm(ref.eps)
    assert err < FIELD_TOL, err
    s = sig.cpu().numpy().astype(np.float64)
    sref = o.stress(prob, ref.eps)
    assert np.linalg.norm(s - sref) / np.linalg.norm(sref) < FIELD_TOL
    ms_ = np.array(info["mean_stress"])
    assert np.max(np.abs(ms_ - ref.mean_stress)) < CEFF_TOL * np.max(np.abs(ref.mean_stress))


def test_rpm_iteration_count_tracks_oracle(rpm, sphere32):
    """Same algorithm at the same tolerance: iteration counts agree closely."""
    cell, prob, _ = sphere32
    E = ms.unit_strain(0)
    r = o.rpm_solve(prob, E, o.Options(tol=1e-6, p_max=10))
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=10)) as ctx:
        st, info = ctx.solve(E)
    assert abs(info["iters"] - r.iters) <= max(3, r.iters // 5), (info, r.iters)


@pytest.mark.parametrize("s", [1, 3])
def test_batch_member_solve_matches_oracle(rpm, s):
    """Batched-sweep cells of 48^3 and 96^3 (radix-3 grids): one RPM solve
    each, mean stress against the FP64 oracle at a tight tolerance."""
    cell = ms.cell_batch_member(s)
    l1, m1 = ms.lame(5.0, 0.3)        # moderate contrast so the oracle finishes quickly
    cell = ms.Cell(phase=cell.phase, lam=np.array([cell.lam[0], l1]), mu=np.array([cell.mu[0], m1]),
                   lam0=0.5 * (cell.lam[0] + l1), mu0=0.5 * (cell.mu[0] + m1))
    prob = o.Problem.from_cell(cell)
    E = ms.unit_strain(5)
    ref = o.rpm_solve(prob, E, o.Options(tol=1e-10, p_max=10))
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=10)) as ctx:
        st, info = ctx.solve(E)
    assert info["converged"]
    d = np.max(np.abs(np.array(info["mean_stress"]) - ref.mean_stress))
    assert d < CEFF_TOL * np.max(np.abs(ref.mean_stress)), d


def test_effective_stiffness_sphere16(rpm):
    cell = ms.cell_sphere32(16)
    prob = o.Problem.from_cell(cell)
    C_ref, _ = o.effective_stiffness(prob, o.rpm_solve, o.Options(tol=1e-10, p_max=10))
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=10)) as ctx:
        C, infos, st = ctx.effective_stiffness()
    assert all(i["converged"] for i in infos)
    assert np.max(np.abs(C - C_ref)) < CEFF_TOL * np.max(np.abs(C_ref))


def test_laminate_closed_form_on_gpu(rpm):
    """Unequal layers normal to e3, contrast 1e3: exact closed form."""
    n = 32
    z = np.arange(n)
    lay = ((z % 8) < 3).astype(np.uint8)
    phase = np.broadcast_to(lay[:, None, None], (n, n, n)).copy()
    l0, m0 = ms.lame(1.0, 0.3)
    l1, m1 = ms.lame(1e3, 0.3)
    cell = ms.Cell(phase=phase, lam=np.array([l0, l1]), mu=np.array([m0, m1]),
                   lam0=0.5 * (l0 + l1), mu0=0.5 * (m0 + m1))
    ref = o.laminate_ceff([5 / 8, 3 / 8], cell.lam, cell.mu)
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=20)) as ctx:
        C, infos, st = ctx.effective_stiffness()
    assert np.max(np.abs(C - ref)) < CEFF_TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("n,frac", [(256, 0.5), (256, 3 / 8)])
def test_laminate_256_closed_form(rpm, n, frac):
    """256^3 laminate (8 layer pairs along z, contrast 1e3, C0 at the mean):
    the five-pass Gamma0 path at full size against the exact C_eff columns of
    the two hardest loads (normal 33 and shear 13)."""
    z = np.arange(n)
    period = n // 8
    lay = ((z % period) < round(frac * period)).astype(np.uint8)
    phase = np.broadcast_to(lay[:, None, None], (n, n, n)).copy()
    l0, m0 = ms.lame(1.0, 0.3)
    l1, m1 = ms.lame(1e3, 0.3)
    cell = ms.Cell(phase=phase, lam=np.array([l0, l1]), mu=np.array([m0, m1]),
                   lam0=0.5 * (l0 + l1), mu0=0.5 * (m0 + m1))
    f1 = float(lay.mean())
    ref = o.laminate_ceff([1 - f1, f1], cell.lam, cell.mu)
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=20)) as ctx:
        for j in (2, 4):
            st, info = ctx.solve(ms.unit_strain(j))
            assert info["converged"]
            col = np.array(info["mean_stress"])
            assert np.max(np.abs(col - ref[:, j])) < CEFF_TOL * np.max(np.abs(ref)), (j, col, ref[:, j])


def test_softincl_128_solution_is_fixed_point(rpm):
    """128^3 RSA cell of the benchmark (inclusion E = 1e-3): the GPU solution
    is a fixed point of the oracle's F to the solver tolerance (FP64 check)."""
    cell = ms.cell_nearvoid(128, 0, e_incl=1e-3)
    prob = o.Problem.from_cell(cell)
    E = ms.unit_strain(0)
    eps = torch.empty((6,) + cell.shape, device="cuda")
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=20)) as ctx:
        st, info = ctx.solve(E, eps_out=eps)
    assert info["converged"] and info["basis_size"] > 0
    e = eps.cpu().numpy().astype(np.float64)
    r = o.residual(prob, o.apply_F(prob, e, E), e, E)
    assert r < 2e-6, r
    assert np.max(np.abs(e.reshape(6, -1).mean(1) - E)) < 1e-5
    s = o.stress(prob, e).reshape(6, -1).mean(1)
    assert np.max(np.abs(s - np.array(info["mean_stress"]))) < 1e-6


def test_nearvoid_trajectory_matches_oracle(rpm):
    """Near-void cell (E_incl = 1e-6) at 32^3: Algorithm 2 stalls far above
    1e-6 on both sides, and the GPU residual history follows the FP64
    oracle's step by step (same basis growth, same residuals)."""
    cell = ms.cell_nearvoid(32, 0)
    prob = o.Problem.from_cell(cell)
    E = ms.unit_strain(0)
    steps = 150
    r = o.rpm_solve(prob, E, o.Options(tol=1e-6, p_max=20, max_iters=steps))
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=20, max_iters=steps)) as ctx:
        res, ps = ctx.trace(steps + 1)
        st, info = ctx.solve(E, raise_on_failure=False)
    assert st == rpm.RPM_ERR_NOT_CONVERGED and r.status == "not_converged"
    assert info["basis_size"] == r.basis
    got = res[:steps + 1]
    ref = np.array(r.residuals[:steps + 1])
    seen = np.isfinite(got)          # with an empty basis only every few steps are tested
    assert seen.sum() > 0.8 * steps
    assert np.max(np.abs(got[seen] - ref[seen]) / ref[seen]) < 2e-2
    assert got[-1] > 1e-4


def test_failure_paths(rpm):
    cell = ms.cell_sphere32(16)
    E = ms.unit_strain(0)
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-9, p_max=0, max_iters=2)) as ctx:
        st, info = ctx.solve(E, raise_on_failure=False)
        assert st == rpm.RPM_ERR_NOT_CONVERGED and info["iters"] == 2
    # reference medium far below the phases: the basic scheme diverges
    bad = ms.Cell(phase=cell.phase, lam=cell.lam, mu=cell.mu, lam0=0.05 * cell.lam0,
                  mu0=0.05 * cell.mu0)
    with rpm.Context(bad, rpm.rpm_default_options(tol=1e-9, p_max=0, diverge_factor=1e3)) as ctx:
        st, info = ctx.solve(E, raise_on_failure=False)
        assert st == rpm.RPM_ERR_DIVERGED
    # NaN planted in the initial field
    with rpm.Context(cell) as ctx:
        eps0 = torch.zeros((6,) + cell.shape, device="cuda")
        eps0[0, 3, 3, 3] = float("nan")
        st, info = ctx.solve(E, eps0=eps0, raise_on_failure=False)
        assert st == rpm.RPM_ERR_DIVERGED
    # allocation cap injected on the host
    with pytest.raises(rpm.RpmError) as ei:
        rpm.Context(cell, rpm.rpm_default_options(max_device_gb=1e-6))
    assert ei.value.status == rpm.RPM_ERR_OOM


def _three_phase_cell(shape, seed):
    """Voxel-wise random three-phase cell with different Poisson ratios, so
    that every per-phase modulus of Algorithm 3's tables differs."""
    ph = ms.random_two_phase(shape, seed, 0.3) + ms.random_two_phase(shape, seed + 1, 0.2)
    lm = [ms.lame(E, nu) for E, nu in ((1.0, 0.3), (10.0, 0.2), (0.3, 0.4))]
    l0, m0 = ms.lame(2.0, 0.3)
    return ms.Cell(phase=ph.astype(np.uint8), lam=np.array([a for a, _ in lm]),
                   mu=np.array([b for _, b in lm]), lam0=l0, mu0=m0)


# 32^3 runs the separate post-step; the square planes of 48, 64 and 128
# run it inside the last pass (clusters of three blocks), nz = 32 included
POL_CELLS = {
    "sphere32": lambda: ms.cell_sphere32(32),
    "three_phase_48": lambda: _three_phase_cell((48, 48, 48), 21),
    "three_phase_32x64x64": lambda: _three_phase_cell((32, 64, 64), 23),
    "three_phase_48x96x96": lambda: _three_phase_cell((48, 96, 96), 25),
    "sphere128": lambda: ms.cell_sphere32(128),
}


@pytest.mark.parametrize("alpha,beta", [(2.0, 2.0), (1.5, 1.0)])
@pytest.mark.parametrize("which", list(POL_CELLS))
def test_polarization_map_matches_oracle(rpm, alpha, beta, which):
    """One application of Algorithm 3 on the GPU (warm start x, one step)
    against the oracle's map, element by element."""
    cell = POL_CELLS[which]()
    prob = o.Problem.from_cell(cell)
    E = ms.unit_strain(0)
    rng = np.random.Generator(np.random.PCG64(4))
    x = (E.reshape(6, 1, 1, 1) + 0.2 * rng.standard_normal((6,) + cell.shape)).astype(np.float32)
    out = torch.empty((6,) + cell.shape, device="cuda")
    opts = rpm.rpm_default_options(scheme=rpm.RPM_SCHEME_POLARIZATION, alpha=alpha, beta=beta,
                                   max_iters=1, tol=0.0, p_max=0)
    with rpm.Context(cell, opts) as ctx:
        st, info = ctx.solve(E, eps0=torch.from_numpy(x).cuda(), eps_out=out, raise_on_failure=False)
    assert st == rpm.RPM_ERR_NOT_CONVERGED and info["iters"] == 1
    ref = o.apply_F_polarization(prob, x.astype(np.float64), E, alpha, beta)
    got = out.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_rpm_accelerated_solve_matches_oracle(rpm):
    """RPM wrapped around the Accelerated scheme (Section 5.5) on the 32^3
    sphere cell with C0 at the geometric mean of the phase moduli."""
    cell = ms.cell_sphere32(32)
    g = np.sqrt(10.0)
    l0, m0 = ms.lame(g, 0.3)
    cell = ms.Cell(phase=cell.phase, lam=cell.lam, mu=cell.mu, lam0=l0, mu0=m0)
    prob = o.Problem.from_cell(cell)
    E = ms.unit_strain(3)
    ref = o.rpm_solve(prob, E, o.Options(tol=1e-11, p_max=10, scheme="polarization"))
    r6 = o.rpm_solve(prob, E, o.Options(tol=1e-6, p_max=10, scheme="polarization"))
    eps = torch.empty((6,) + cell.shape, device="cuda")
    opts = rpm.rpm_default_options(scheme=rpm.RPM_SCHEME_POLARIZATION, tol=1e-6, p_max=10)
    with rpm.Context(cell, opts) as ctx:
        st, info = ctx.solve(E, eps_out=eps)
    assert info["converged"]
    assert abs(info["iters"] - r6.iters) <= max(3, r6.iters // 5)
    d = np.max(np.abs(np.array(info["mean_stress"]) - ref.mean_stress))
    assert d < CEFF_TOL * np.max(np.abs(ref.mean_stress))
    e = eps.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(e - ref.eps) / np.linalg.norm(ref.eps) < FIELD_TOL


def test_softincl128_warm_solve_matches_oracle_golden(rpm):
    """The benchmark's headline form at full size: warm start by Algorithm 3,
    then RPM on Eq. 3.9, against the oracle's own solve of the same form
    (tests/golden/softincl128_warm_oracle_solve.json, written by
    tests/golden/make_golden.py from the oracle only)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "softincl128_warm_oracle_solve.json")
    ref = json.load(open(path))
    cell = ms.cell_nearvoid(128, 0, e_incl=1e-3)
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=20, warm_tol=1e-4)) as ctx:
        st, info = ctx.solve(ms.unit_strain(0))
    assert info["converged"]
    sig = np.array(info["mean_stress"])
    sref = np.array(ref["mean_stress"])
    assert np.max(np.abs(sig - sref)) < CEFF_TOL * np.max(np.abs(sref)), (sig, sref)
    assert abs(info["warm_iters"] - ref["warm_iters"]) <= 8
    assert abs(info["gamma_applies"] - ref["f_applies"]) <= 12


def test_softincl128_cold_solve_matches_oracle_fixed_point(rpm):
    """The cold form of the benchmark (RPM on Eq. 3.9 from eps = E, C0 =
    matrix, 1575 steps and a 20-vector basis on the GPU) at full size against
    the oracle's converged solve of the same cell and load
    (tests/golden/softincl128_warm_oracle_solve.json, written by
    tests/golden/make_golden.py from the oracle only): both forms converge to
    the one fixed point of F, so the mean stresses agree to the tolerance."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "softincl128_warm_oracle_solve.json")
    ref = json.load(open(path))
    cell = ms.cell_nearvoid(128, 0, c0_scale=1.0, e_incl=1e-3)
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=20)) as ctx:
        st, info = ctx.solve(ms.unit_strain(0))
    assert info["converged"] and info["basis_size"] > 0 and info["warm_iters"] == 0
    sig = np.array(info["mean_stress"])
    sref = np.array(ref["mean_stress"])
    assert np.max(np.abs(sig - sref)) < CEFF_TOL * np.max(np.abs(sref)), (sig, sref)


def test_warm_started_solve_matches_cold(rpm, sphere32):
    """Warm start by the Accelerated scheme (Algorithm 3) followed by RPM on
    Eq. 3.9: same converged result as the cold start, within tolerance."""
    cell, prob, ref = sphere32
    E = ms.unit_strain(0)
    eps = torch.empty((6,) + cell.shape, device="cuda")
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=10, warm_tol=1e-4)) as ctx:
        st, info = ctx.solve(E, eps_out=eps)
    assert info["converged"] and info["warm_iters"] > 0 and info["warm_residual"] <= 1e-4
    e = eps.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(e - ref.eps) / np.linalg.norm(ref.eps) < FIELD_TOL
    d = np.max(np.abs(np.array(info["mean_stress"]) - ref.mean_stress))
    assert d < CEFF_TOL * np.max(np.abs(ref.mean_stress))


def test_effective_stiffness_batch_matches_single_contexts(rpm):
    """NEXT-1 batch driver: cells of different grids solved concurrently on
    worker streams give the same C_eff as one context per cell, and the
    materials of a reused context are replaced correctly."""
    cells = [ms.cell_sphere32(16), ms.cell_batch_member(1), ms.cell_sphere32(16)]
    l1, m1 = ms.lame(4.0, 0.3)
    cells[1] = ms.Cell(phase=cells[1].phase, lam=np.array([cells[1].lam[0], l1]),
                       mu=np.array([cells[1].mu[0], m1]), lam0=0.5 * (cells[1].lam[0] + l1),
                       mu0=0.5 * (cells[1].mu[0] + m1))
    l2, m2 = ms.lame(25.0, 0.3)      # same grid as cell 0, other materials (context reuse)
    cells[2] = ms.Cell(phase=cells[2].phase, lam=np.array([cells[2].lam[0], l2]),
                       mu=np.array([cells[2].mu[0], m2]), lam0=0.5 * (cells[2].lam[0] + l2),
                       mu0=0.5 * (cells[2].mu[0] + m2))
    opts = rpm.rpm_default_options(tol=1e-6, p_max=10)
    Cb, infos, stat, st = rpm.rpm_effective_stiffness_batch(cells, opts, n_workers=4)
    assert st == rpm.RPM_OK and stat == [0, 0, 0]
    for i, cell in enumerate(cells):
        with rpm.Context(cell, opts) as ctx:
            C, _, _ = ctx.effective_stiffness()
        assert np.max(np.abs(Cb[i] - C)) <= 1e-12 * np.max(np.abs(C)), i
    assert np.max(np.abs(Cb[0] - Cb[2])) > 1e-3      # different materials, different C_eff


def test_degenerate_cases(rpm):
    """E = 0 gives the zero field at once; a homogeneous cell (one phase, any
    C0) gives eps = E after at most one step; the 2D limit nz = 1 runs."""
    cell = ms.cell_sphere32(16)
    eps = torch.full((6,) + cell.shape, 7.0, device="cuda")
    with rpm.Context(cell) as ctx:
        st, info = ctx.solve(np.zeros(6), eps_out=eps)
    assert info["converged"] and info["iters"] == 0
    assert float(eps.abs().max()) == 0.0
    l, m = ms.lame(3.0, 0.3)
    hom = ms.Cell(phase=np.zeros((8, 8, 8), np.uint8), lam=np.array([l]), mu=np.array([m]),
                  lam0=2 * l, mu0=2 * m)
    E = np.array([0.1, -0.2, 0.3, 0.05, 0.01, -0.04])
    eps = torch.empty((6, 8, 8, 8), device="cuda")
    with rpm.Context(hom) as ctx:
        st, info = ctx.solve(E, eps_out=eps)
    assert info["converged"] and info["iters"] <= 1
    assert np.max(np.abs(eps.cpu().numpy() - E.reshape(6, 1, 1, 1))) < 1e-6
    f2 = ms.cell_fibre2d(64, 10.0, radius=0.2)
    prob = o.Problem.from_cell(f2)
    E2 = np.zeros(6)
    E2[5] = 0.5
    ref = o.rpm_solve(prob, E2, o.Options(tol=1e-10, p_max=10))
    with rpm.Context(f2, rpm.rpm_default_options(tol=1e-7, p_max=10)) as ctx:
        st, info = ctx.solve(E2)
    assert info["converged"]
    assert np.max(np.abs(np.array(info["mean_stress"]) - ref.mean_stress)) < 1e-5 * np.max(np.abs(ref.mean_stress))


@pytest.mark.parametrize("seed", [5012, 5013])
def test_stiff_cell_converges_and_matches_oracle_golden(rpm, seed):
    """Stiff inclusions (contrast 373 and 182, C0 = mean): in float32 the plain
    RPM iteration stalled above 1e-6 (5012) or diverged after a late basis
    growth from a non-trivial start (5013).  With the growth noise guard and
    re-centring after a stall it converges, within twice the oracle's steps,
    to the FP64 oracle's answer (solved to 1e-8 in tests/golden) within the
    effective-stiffness tolerance.  The oracle's own answer at tol 1e-6 lies
    within 2e-6 of its 1e-8 answer on these cells (stored beside it), so the
    method's tolerance is not what separates the two: the float32 fixed point
    itself sits 8e-6 (5012) and 3e-6 (5013) from the FP64 one, at tol 1e-6 as
    at 1e-8."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "stiff64_oracle_solve.json")))[str(seed)]
    cell = ms.cell_fno_member(seed, 64)
    E = np.array(g["E"])
    with rpm.Context(cell, rpm.rpm_default_options(tol=1e-6, p_max=20, max_iters=1000)) as ctx:
        st, info = ctx.solve(E)
    assert info["converged"], info
    assert info["iters"] <= 2 * g["iters_to_1e-6"], (info["iters"], g["iters_to_1e-6"])
    ref = np.array(g["mean_stress"])
    spread = (np.max(np.abs(np.array(g["tol_1e-6"]["mean_stress"]) - ref)) / np.max(np.abs(ref)))
    assert spread < 1e-5, spread
    err = np.max(np.abs(np.array(info["mean_stress"]) - ref)) / np.max(np.abs(ref))
    assert err < CEFF_TOL, err


def test_ellipsoids_256_warm_form_converges_within_bounds(rpm):
    """256^3 cell of random ellipsoids at 30 % volume fraction, contrast 1e4
    (the high-contrast full-size case): the warm-started form reaches tol 1e-6
    (the cold start does not within 3000 steps), and the mean stress of the
    e11 load, column 1 of C_eff, lies between the Reuss and Voigt bounds."""
    cell = ms.cell_ellipsoids(256, 0, contrast=1e4)
    f1 = float(cell.phase.mean())
    opts = rpm.rpm_default_options(warm_tol=1e-4, max_iters=3000, warm_max_iters=3000)
    with rpm.Context(cell, opts) as ctx:
        st, info = ctx.solve(ms.unit_strain(0))
    assert info["converged"] and info["residual"] <= 1e-6, info
    V = o.voigt_bound([1 - f1, f1], cell.lam, cell.mu)
    R = o.reuss_bound([1 - f1, f1], cell.lam, cell.mu)
    s = np.array(info["mean_stress"])
    assert R[0, 0] < s[0] < V[0, 0], (R[0, 0], s[0], V[0, 0])


@pytest.mark.parametrize("n", [48, 128])
def test_autotuned_variants_give_the_same_solve(rpm, n):
    """The autotuner times every available pair of plane-pass kernels (fused,
    whole-plane, five-pass) and z-pass variants (fused, half, default, twice
    the pencils per block) and keeps the fastest; every pair computes the
    same map up to float32 rounding, so the solve matches the default one
    to rounding and converges in the same number of steps (within one)."""
    cell = ms.cell_nearvoid(n, 0, e_incl=1e-1) if n == 128 else ms.cell_batch_member(1)
    E = ms.unit_strain(0)
    with rpm.Context(cell, rpm.rpm_default_options()) as a:
        assert rpm.rpm_plane_variant(a.handle) == 0
        _, ia = a.solve(E)
    with rpm.Context(cell, rpm.rpm_default_options(autotune=1)) as b:
        v = rpm.rpm_plane_variant(b.handle)
        t = rpm.rpm_pencil_tile(b.handle)
        _, ib = b.solve(E)
    assert v in (0, 1, 2) and t >= 1
    assert ia["converged"] and ib["converged"]
    assert abs(ia["iters"] - ib["iters"]) <= 1
    sa, sb = np.array(ia["mean_stress"]), np.array(ib["mean_stress"])
    assert np.max(np.abs(sa - sb)) <= 1e-6 * np.max(np.abs(sa))


_VARIANT_CASES = {}


def _variant_case(n):
    """Cell, input field, load and the oracle's map of it (computed once per n)."""
    if n not in _VARIANT_CASES:
        cell = ms.cell_nearvoid(n, 0, e_incl=1e-1)
        E = ms.unit_strain(0)
        rng = np.random.Generator(np.random.PCG64(5))
        x = (E.reshape(6, 1, 1, 1)
             + 0.3 * rng.standard_normal((6,) + cell.shape)).astype(np.float32)
        ref = o.apply_F(o.Problem.from_cell(cell), x.astype(np.float64), E)
        _VARIANT_CASES[n] = (cell, x, E, ref)
    return _VARIANT_CASES[n]


@pytest.mark.parametrize("plane,pencil", [(0, 0), (1, 0), (2, 0), (0, 1), (0, 2), (0, 3),
                                          (1, 3), (2, 2)])
@pytest.mark.parametrize("n", [64, 128])
def test_forced_variants_match_oracle(rpm, n, plane, pencil):
    """Every plane-pass / z-pass variant a context can be given (and the
    autotuner can choose) applies the map of Eq. 3.9 on the fused sizes:
    one application against the FP64 oracle, element by element."""
    cell, x, E, ref = _variant_case(n)
    out = torch.empty((6,) + cell.shape, device="cuda")
    opts = rpm.rpm_default_options(plane_variant=plane, pencil_variant=pencil)
    with rpm.Context(cell, opts) as ctx:
        assert rpm.rpm_plane_variant(ctx.handle) == plane
        ctx.apply_gamma(torch.from_numpy(x).cuda(), E, out)
    got = out.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_batched_sweep_32_members_ceff_match_oracle(rpm):
    """The 32^3 members of the batched effective-stiffness sweep (contrast
    1e-2 ... 6e2) through the batch driver, every entry of C_eff against the
    FP64 oracle's (tests/golden, solved to 1e-8) at the effective-stiffness
    tolerance 1e-5 -- or, for stiff inclusions, at the float32 bound
    4e-8 x contrast: the float32 map's fixed point lies about 2.3e-8 x
    contrast from the FP64 one whatever the tolerance (measured: 8.1e-6 at
    contrast 373, 1.4e-5 at contrast 603), so above contrast 250 the
    fields' precision, not the solver, sets the error."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "c4_32_oracle_ceff.json")))
    seeds = sorted(int(k) for k in g)
    cells = [ms.cell_batch_member(s) for s in seeds]
    opts = rpm.rpm_default_options(tol=1e-7, p_max=20, max_iters=3000)
    C, infos, stat, st = rpm.rpm_effective_stiffness_batch(cells, opts, n_workers=4,
                                                           raise_on_failure=False)
    for i, s in enumerate(seeds):
        assert stat[i] == rpm.RPM_OK, (s, stat[i])
        ref = np.array(g[str(s)]["C_eff"])
        err = np.max(np.abs(C[i] - ref)) / np.max(np.abs(ref))
        bound = max(CEFF_TOL, 4e-8 * g[str(s)]["contrast"])
        assert err < bound, (s, g[str(s)]["contrast"], err)


def test_sampled_event_profile_scales_to_all_groups(rpm):
    """opt.profile = k brackets every k-th launch group of each class with
    CUDA events and scales the sampled time to all groups: the estimate of
    the Gamma0 time agrees with the all-groups figure and stays inside the
    solve's own time."""
    cell = ms.cell_sphere32(64)
    E = ms.unit_strain(0)
    out = {}
    for k in (1, 4):
        with rpm.Context(cell, rpm.rpm_default_options(profile=k, p_max=4)) as ctx:
            ctx.solve(E)   # warm-up
            _, info = ctx.solve(E)
        out[k] = info
        assert 0 < info["gamma_ms"] <= info["ms"]
    assert out[1]["gamma_applies"] == out[4]["gamma_applies"]
    assert 0.5 < out[4]["gamma_ms"] / out[1]["gamma_ms"] < 2.0


def test_bounded_wait_gives_up_and_the_stream_stays_usable(rpm):
    """The bulk-copy passes wait on an mbarrier with a bound (about one
    second on the global timer) and report RPM_ERR_TIMEOUT instead of
    hanging.  A barrier that no copy completes (a flag that nothing sets)
    must make the wait give up by itself, and the next launches on the same
    stream must run normally."""
    gave_up, ms_waited = rpm.rpm_bounded_wait_check(torch.cuda.current_stream())
    assert gave_up
    assert 500.0 < ms_waited < 10000.0, ms_waited
    cell = ms.cell_sphere32(48)
    with rpm.Context(cell) as ctx:
        st, info = ctx.solve(ms.unit_strain(0))
    assert st == rpm.RPM_OK and info["converged"]


def _soft_sphere_cell(n):
    """Centred sphere R = L/4 of E = 1e-2 in a matrix E = 1, C0 = matrix:
    RPM needs a basis here (the basic scheme's slow modes sit near 1)."""
    return ms._two_phase(ms.centred_sphere(n, 0.25), 1.0, 1e-2, c0_scale=1.0, name="softsphere")


_SHARED_REF = {}


@pytest.mark.parametrize("share", [0, 1])
def test_effective_stiffness_shared_basis_matches_oracle(rpm, share):
    """Block RPM (options.share_basis): F_u does not depend on the load, so
    the six loads of C_eff can start from the unstable basis the previous
    load left; the fixed point is the same, so C_eff matches the FP64 oracle
    either way, and with sharing loads 2-6 report the vectors they took
    over.  (Sharing is not faster: each unit load excites its own part of
    the slow eigenspace, which a basis filled by the earlier loads leaves no
    room for.)"""
    cell = _soft_sphere_cell(24)
    if "C" not in _SHARED_REF:
        prob = o.Problem.from_cell(cell)
        _SHARED_REF["C"], _ = o.effective_stiffness(prob, o.rpm_solve,
                                                    o.Options(tol=1e-10, p_max=20))
    C_ref = _SHARED_REF["C"]
    opts = rpm.rpm_default_options(tol=1e-6, p_max=20, share_basis=share)
    with rpm.Context(cell, opts) as ctx:
        C, infos, st = ctx.effective_stiffness()
    assert st == rpm.RPM_OK and all(i["converged"] for i in infos)
    assert np.max(np.abs(C - C_ref)) < CEFF_TOL * np.max(np.abs(C_ref))
    assert infos[0]["basis_reused"] == 0
    if share:
        assert all(i["basis_reused"] > 0 for i in infos[1:])
    else:
        assert all(i["basis_reused"] == 0 for i in infos)


def test_shared_basis_is_dropped_when_the_map_changes(rpm):
    """A stored basis belongs to one map F_u: changing C0 (or the phases or
    materials) drops it, and the next solve starts from an empty basis."""
    cell = _soft_sphere_cell(24)
    E = ms.unit_strain(0)
    opts = rpm.rpm_default_options(tol=1e-6, p_max=20, share_basis=1)
    with rpm.Context(cell, opts) as ctx:
        _, a = ctx.solve(E)
        _, b = ctx.solve(E)
        assert a["basis_size"] > 0 and b["basis_reused"] == a["basis_size"] and b["converged"]
        rpm.rpm_set_materials(ctx.handle, list(zip(cell.lam, cell.mu)),
                              (0.9 * cell.lam0, 0.9 * cell.mu0))
        _, c = ctx.solve(E)
        assert c["basis_reused"] == 0 and c["converged"]


def test_host_phase_map_with_an_unknown_id_is_refused(rpm):
    """A host phase map is checked before upload: an id at or above the
    number of phases (here in the last voxel) is RPM_ERR_INVALID_ARG and the
    context keeps its previous map."""
    cell = ms.cell_sphere32(16)
    E = ms.unit_strain(0)
    with rpm.Context(cell) as ctx:
        _, ref = ctx.solve(E)
        bad = cell.phase.copy()
        bad.reshape(-1)[-1] = 2
        with pytest.raises(rpm.RpmError) as ei:
            rpm.rpm_set_phase(ctx.handle, bad)
        assert ei.value.status == rpm.RPM_ERR_INVALID_ARG
        _, again = ctx.solve(E)
        assert again["mean_stress"] == ref["mean_stress"]
