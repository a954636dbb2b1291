"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test names what fixes the expected value: a textbook closed form, an
identity of the Lippmann-Schwinger operator, a brute-force solve, or a
library routine.  They are chosen so that a dropped term, a wrong sign, a
transposed index or a wrong Nyquist rule in the oracle fails one of them.
"""
import math

import numpy as np
import pytest

import microstructure as ms
from oracle import rpm_oracle as o


def _rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def _prob(shape, seed=1, c_ratio=(1.0, 10.0), nu=0.3, c0=None, vf=0.4):
    phase = ms.random_two_phase(shape, seed, vf)
    lams, mus = zip(*[ms.lame(E, nu) for E in c_ratio])
    if c0 is None:
        c0 = ms.lame(0.5 * sum(c_ratio), nu)
    return o.Problem(phase=phase, lam=np.array(lams), mu=np.array(mus),
                     lam0=c0[0], mu0=c0[1])


def _compatible_field(shape, seed=3, amp=1.0):
    """A real, zero-mean compatible strain field sym(grad v) built from a
    random periodic displacement v given on the grid (finite displacement
    field -> exact trigonometric-interpolation strain)."""
    rng = _rng(seed)
    nz, ny, nx = shape
    v = rng.standard_normal((3, nz, ny, nx)) * amp
    vh = np.fft.rfftn(v, axes=(1, 2, 3))
    p = o.Problem(phase=np.zeros(shape, np.uint8), lam=np.ones(1), mu=np.ones(1),
                  lam0=1.0, mu0=1.0)
    xi, m, nyq = o.frequencies(p)
    keep = o.green_mask(p)
    vh = vh * keep
    # eps_ij = (i/2)(xi_i v_j + xi_j v_i)
    grad = 1j * np.einsum("i...,j...->ij...", xi, vh)
    eh = 0.5 * (grad + np.swapaxes(grad, 0, 1))
    return o.ifft_fields(o.from_full(eh), shape)


# ----------------------------------------------------------------------------
# Fourier transform (library routine) vs brute-force DFT
# ----------------------------------------------------------------------------
def test_fft_matches_bruteforce_dft():
    shape = (4, 6, 8)
    f = _rng(0).standard_normal((6,) + shape)
    got = o.fft_fields(f)
    nz, ny, nx = shape
    kz = np.arange(nz)[:, None, None, None, None, None]
    ky = np.arange(ny)[None, :, None, None, None, None]
    kx = np.arange(nx // 2 + 1)[None, None, :, None, None, None]
    z = np.arange(nz)[None, None, None, :, None, None]
    y = np.arange(ny)[None, None, None, None, :, None]
    x = np.arange(nx)[None, None, None, None, None, :]
    W = np.exp(-2j * np.pi * (kz * z / nz + ky * y / ny + kx * x / nx))
    ref = np.einsum("abcxyz,nxyz->nabc", W, f)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    back = o.ifft_fields(got, shape)
    assert np.max(np.abs(back - f)) < 1e-13


# ----------------------------------------------------------------------------
# Green operator
# ----------------------------------------------------------------------------
def test_acoustic_inverse_matches_isotropic_closed_form():
    """N0 = (1/(mu0 |xi|^2)) [I - (lam0+mu0)/(lam0+2mu0) xi xi^T/|xi|^2]."""
    rng = _rng(5)
    xi = rng.standard_normal((3, 50)) * 7.0
    lam0, mu0 = 1.7, 0.9
    N0 = o.acoustic_tensor_inverse(xi, lam0, mu0)
    for m in range(xi.shape[1]):
        x = xi[:, m]
        r2 = x @ x
        ref = (np.eye(3) - (lam0 + mu0) / (lam0 + 2 * mu0) * np.outer(x, x) / r2) / (mu0 * r2)
        assert np.max(np.abs(N0[m] - ref)) < 1e-13 * np.max(np.abs(ref))


def _gamma_moulinec_suquet(x, lam0, mu0):
    """Textbook 4th-order Green operator of an isotropic medium (Moulinec &
    Suquet 1998):
    G_khij = [d_ki x_h x_j + d_hi x_k x_j + d_kj x_h x_i + d_hj x_k x_i]/(4 mu0 |x|^2)
             - (lam0 + mu0)/(mu0 (lam0 + 2 mu0)) x_i x_j x_k x_h / |x|^4."""
    d = np.eye(3)
    r2 = x @ x
    G = (np.einsum("ki,h,j->khij", d, x, x) + np.einsum("hi,k,j->khij", d, x, x)
         + np.einsum("kj,h,i->khij", d, x, x) + np.einsum("hj,k,i->khij", d, x, x)) / (4 * mu0 * r2)
    G -= (lam0 + mu0) / (mu0 * (lam0 + 2 * mu0)) * np.einsum("i,j,k,h->khij", x, x, x, x) / r2 ** 2
    return G


def test_gamma_matches_textbook_fourth_order_tensor():
    shape = (4, 6, 8)
    p = _prob(shape)
    th = _rng(2).standard_normal((6, 4, 6, 5)) + 1j * _rng(3).standard_normal((6, 4, 6, 5))
    got = o.gamma_hat_apply(p, th)
    xi, _, _ = o.frequencies(p)
    keep = o.green_mask(p)
    T = o.to_full(th)
    for iz in range(4):
        for iy in range(6):
            for ix in range(5):
                if not keep[iz, iy, ix]:
                    assert np.all(got[:, iz, iy, ix] == 0)
                    continue
                G = _gamma_moulinec_suquet(xi[:, iz, iy, ix], p.lam0, p.mu0)
                ref = o.from_full(np.einsum("khij,ij->kh", G, T[:, :, iz, iy, ix]))
                assert np.max(np.abs(got[:, iz, iy, ix] - ref)) < 1e-12 * (1 + np.max(np.abs(ref)))


def test_green_mask_nyquist_rule():
    """k = 0 and mixed Nyquist frequencies are masked, pure-axis Nyquist kept."""
    p = _prob((4, 4, 4))
    keep = o.green_mask(p)
    assert not keep[0, 0, 0]
    assert keep[0, 0, 2] and keep[0, 2, 0] and keep[2, 0, 0]      # pure-axis Nyquist
    assert not keep[0, 1, 2] and not keep[2, 1, 0] and not keep[2, 2, 2]
    assert keep[1, 1, 1] and keep[3, 1, 1]


def test_projector_identity_gamma_c0_gamma():
    """Gamma0 : C0 : Gamma0 = Gamma0, i.e. G(C0 : G(tau)) = -G(tau) for
    G(tau) = -Gamma0 * tau."""
    shape = (6, 8, 8)
    p = _prob(shape)
    tau = _rng(4).standard_normal((6,) + shape)
    g = o.apply_gamma_raw(p, tau)
    c0 = o.Problem(phase=np.zeros(shape, np.uint8), lam=np.array([p.lam0]), mu=np.array([p.mu0]),
                   lam0=0.0, mu0=0.0)
    c0g = o.stress(c0, g)
    gg = o.apply_gamma_raw(p, c0g)
    assert np.max(np.abs(gg + g)) < 1e-12 * np.max(np.abs(g))


def test_gamma_inverts_c0_on_compatible_fields():
    """For compatible zero-mean e: -Gamma0 * (C0 : e) = -e."""
    shape = (8, 8, 6)
    p = _prob(shape)
    e = _compatible_field(shape)
    c0 = o.Problem(phase=np.zeros(shape, np.uint8), lam=np.array([p.lam0]), mu=np.array([p.mu0]),
                   lam0=0.0, mu0=0.0)
    g = o.apply_gamma_raw(p, o.stress(c0, e))
    assert np.max(np.abs(g + e)) < 1e-12 * np.max(np.abs(e))


def _incompatibility(eh, xi):
    """eta_ij = e_ikl e_jmn xi_k xi_m eps_ln (Saint-Venant in Fourier space)."""
    lc = np.zeros((3, 3, 3))
    lc[0, 1, 2] = lc[1, 2, 0] = lc[2, 0, 1] = 1
    lc[0, 2, 1] = lc[2, 1, 0] = lc[1, 0, 2] = -1
    T = o.to_full(eh)
    return np.einsum("ikl,jmn,k...,m...,ln...->ij...", lc, lc, xi, xi, T)


def test_gamma_output_is_compatible_and_zero_mean():
    shape = (6, 8, 8)
    p = _prob(shape)
    g = o.apply_gamma_raw(p, _rng(6).standard_normal((6,) + shape))
    assert np.max(np.abs(g.reshape(6, -1).mean(axis=1))) < 1e-13
    xi, _, _ = o.frequencies(p)
    eta = _incompatibility(o.fft_fields(g), xi)
    assert np.max(np.abs(eta)) < 1e-9 * np.max(np.abs(o.fft_fields(g))) * np.max(np.abs(xi)) ** 2


def test_gamma_commutes_with_reflection_and_axis_swap():
    """Gamma0_hat is even in xi and isotropic: G commutes with x -> -x and,
    on a cubic grid, with the x<->y swap (components permuted accordingly)."""
    shape = (8, 8, 8)
    p = _prob(shape)
    tau = _rng(7).standard_normal((6,) + shape)

    def reflect(f):
        return np.roll(f[:, ::-1, ::-1, ::-1], 1, axis=(1, 2, 3))

    g = o.apply_gamma_raw(p, tau)
    g2 = o.apply_gamma_raw(p, reflect(tau))
    assert np.max(np.abs(g2 - reflect(g))) < 1e-12

    perm = [1, 0, 2, 4, 3, 5]          # 11<->22, 23<->13 under x<->y

    def swap(f):
        return np.swapaxes(f[perm], 2, 3)

    g3 = o.apply_gamma_raw(p, swap(tau))
    assert np.max(np.abs(g3 - swap(g))) < 1e-12


# ----------------------------------------------------------------------------
# fixed-point map
# ----------------------------------------------------------------------------
def test_homogeneous_medium_is_fixed_point():
    """C(x) = C0 everywhere: tau = 0, so F(eps) = E for any eps."""
    shape = (4, 6, 8)
    p = _prob(shape, c_ratio=(2.0, 2.0), c0=ms.lame(2.0, 0.3))
    E = _rng(1).standard_normal(6)
    eps = _rng(2).standard_normal((6,) + shape)
    assert np.max(np.abs(o.apply_F(p, eps, E) - E.reshape(6, 1, 1, 1))) < 1e-13


def test_uniform_medium_closed_form():
    """C = c C0 (same nu) uniform: on eps = E + e, e compatible zero-mean,
    F(eps) = E - (c - 1) e; the basic scheme is exact after one step from E."""
    shape = (8, 6, 6)
    c = 3.5
    l0, m0 = ms.lame(2.0, 0.3)
    p = o.Problem(phase=np.zeros(shape, np.uint8), lam=np.array([c * l0]), mu=np.array([c * m0]),
                  lam0=l0, mu0=m0)
    E = _rng(3).standard_normal(6)
    e = _compatible_field(shape, seed=9)
    F = o.apply_F(p, E.reshape(6, 1, 1, 1) + e, E)
    assert np.max(np.abs(F - (E.reshape(6, 1, 1, 1) - (c - 1) * e))) < 1e-12
    res = o.basic_solve(p, E, o.Options(tol=1e-12))
    assert res.iters == 0 and res.converged


def test_polarization_form_equals_classical_form_on_compatible_fields():
    """Eq. (3.9) as printed and the polarization form agree on E + compatible."""
    shape = (6, 8, 8)
    p = _prob(shape)
    E = _rng(4).standard_normal(6)
    eps = E.reshape(6, 1, 1, 1) + _compatible_field(shape, seed=11, amp=0.3)
    a = o.apply_F(p, eps, E)
    b = o.apply_F_classical(p, eps, E)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


# ----------------------------------------------------------------------------
# brute force on tiny grids
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny():
    shape = (4, 4, 4)
    p = _prob(shape, seed=21, c_ratio=(1.0, 20.0))
    L = o.dense_linear_operator(p)
    return p, L


def test_dense_operator_spectrum_within_phase_bounds(tiny):
    """Equal-nu phases C_r = (c_r/c0) C0: eigenvalues of F_u lie in
    [1 - c_max/c0, 1 - c_min/c0] (or are 0, off the compatible range)."""
    p, L = tiny
    ev = np.linalg.eigvals(L)
    c = p.mu / p.mu0
    lo, hi = 1 - c.max(), 1 - c.min()
    assert np.max(np.abs(ev.imag)) < 1e-8
    r = ev.real
    ok = (np.abs(r) < 1e-9) | ((r > lo - 1e-9) & (r < hi + 1e-9))
    assert ok.all()


def test_direct_solution_satisfies_cell_problem(tiny):
    """The dense solve of eps = E + F_u eps is the discrete cell-problem
    solution: mean E, compatible, and in equilibrium (zero k . sigma_hat at
    every frequency where Gamma0 acts) - checked without the Green operator."""
    p, L = tiny
    E = np.array([0.3, -0.1, 0.2, 0.05, -0.07, 0.11])
    rhs = o.uniform(E, p.shape).ravel()
    eps = np.linalg.solve(np.eye(L.shape[0]) - L, rhs).reshape((6,) + p.shape)
    assert np.max(np.abs(eps.reshape(6, -1).mean(1) - E)) < 1e-12
    xi, _, _ = o.frequencies(p)
    eh = o.fft_fields(eps)
    assert np.max(np.abs(_incompatibility(eh, xi))) < 1e-9
    assert o.equilibrium_error(p, o.stress(p, eps)) < 1e-12
    # frequencies where Gamma0 is zeroed carry no strain
    keep = o.green_mask(p)
    keep[0, 0, 0] = True
    assert np.max(np.abs(eh[:, ~keep])) < 1e-10


def test_basic_and_rpm_match_direct_solve(tiny):
    p, L = tiny
    E = ms.unit_strain(3)
    eps_ref = np.linalg.solve(np.eye(L.shape[0]) - L, o.uniform(E, p.shape).ravel())
    rb = o.basic_solve(p, E, o.Options(tol=1e-12, max_iters=20000))
    rr = o.rpm_solve(p, E, o.Options(tol=1e-12, p_max=10))
    assert rb.converged and rr.converged
    assert rr.iters < rb.iters
    for r in (rb, rr):
        err = np.linalg.norm(r.eps.ravel() - eps_ref) / np.linalg.norm(eps_ref)
        assert err < 1e-9


def test_rpm_basis_orthonormal_and_H_matches_dense(tiny):
    p, L = tiny
    E = ms.unit_strain(0)
    st_holder = {}
    orig = o._grow_basis

    def spy(prob, st, hist, opts):
        n = orig(prob, st, hist, opts)
        st_holder["st"] = st
        return n
    o._grow_basis = spy
    try:
        o.rpm_solve(p, E, o.Options(tol=1e-12, p_max=8, n_max=3))
    finally:
        o._grow_basis = orig
    st = st_holder["st"]
    Z = np.stack([z.ravel() for z in st.Z], axis=1)
    W = np.diag(np.repeat(o.WEIGHTS, p.n))
    G = Z.T @ W @ Z
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-12
    Hd = Z.T @ W @ L @ Z
    assert np.max(np.abs(Hd - st.H)) < 1e-12


def test_rpm_without_basis_is_basic_scheme():
    """p_max = 0: RPM reduces to Algorithm 1 iterate for iterate."""
    p = _prob((6, 6, 6), seed=4, c_ratio=(1.0, 8.0))
    E = ms.unit_strain(1)
    a = o.basic_solve(p, E, o.Options(tol=1e-9))
    b = o.rpm_solve(p, E, o.Options(tol=1e-9, p_max=0))
    assert a.iters == b.iters
    assert np.allclose(a.residuals, b.residuals, rtol=1e-12, atol=0)
    assert np.max(np.abs(a.eps - b.eps)) < 1e-14


def test_rpm_converges_where_basic_diverges():
    """C0 = 1.3 x the soft phase with a 3x stiffer phase puts dozens of
    eigenvalues of F_u outside the unit disk: the fixed point diverges, and
    RPM's Newton step on the identified subspace restores convergence to the
    direct solution (Section 3)."""
    shape = (6, 6, 6)
    l1, m1 = ms.lame(1.0, 0.3)
    p = _prob(shape, seed=8, c_ratio=(1.0, 3.0), c0=(1.3 * l1, 1.3 * m1))
    L = o.dense_linear_operator(p)
    assert np.sum(np.abs(np.linalg.eigvals(L)) > 1.0) > 10
    E = ms.unit_strain(0)
    rb = o.basic_solve(p, E, o.Options(tol=1e-9, max_iters=300))
    rr = o.rpm_solve(p, E, o.Options(tol=1e-9, p_max=40, n_max=5, max_iters=3000))
    assert rb.status == "diverged"
    assert rr.converged
    ref = np.linalg.solve(np.eye(L.shape[0]) - L, o.uniform(E, shape).ravel())
    assert np.linalg.norm(rr.eps.ravel() - ref) / np.linalg.norm(ref) < 1e-6


# ----------------------------------------------------------------------------
# effective stiffness: closed forms, bounds, symmetry, C0 independence
# ----------------------------------------------------------------------------
def test_laminate_matches_closed_form():
    """Layers normal to e3 with unequal thicknesses and C0 off the mean."""
    n = 16
    z = np.arange(n)
    lay = ((z % 8) < 3).astype(np.uint8)          # phase 1 fraction 3/8
    phase = np.broadcast_to(lay[:, None, None], (n, 4, 4)).copy()
    l0, m0 = ms.lame(1.0, 0.3)
    l1, m1 = ms.lame(1e3, 0.3)
    p = o.Problem(phase=phase, lam=np.array([l0, l1]), mu=np.array([m0, m1]),
                  lam0=300 * l0, mu0=300 * m0)
    C, res = o.effective_stiffness(p, o.rpm_solve, o.Options(tol=1e-11, p_max=20, max_iters=5000))
    f1 = 3.0 / 8.0
    ref = o.laminate_ceff([1 - f1, f1], p.lam, p.mu)
    assert all(r.converged for r in res)
    assert np.max(np.abs(C - ref)) < 1e-8 * np.max(np.abs(ref))


def test_laminate_closed_form_is_between_bounds_and_symmetric():
    f = [0.3, 0.7]
    lam = [ms.lame(1, 0.3)[0], ms.lame(50, 0.2)[0]]
    mu = [ms.lame(1, 0.3)[1], ms.lame(50, 0.2)[1]]
    C = o.laminate_ceff(f, lam, mu)
    V = o.voigt_bound(f, lam, mu)
    R = o.reuss_bound(f, lam, mu)
    assert np.max(np.abs(C - C.T)) < 1e-12 * np.max(np.abs(C))
    assert np.linalg.eigvalsh(V - C).min() > -1e-10
    assert np.linalg.eigvalsh(C - R).min() > -1e-10
    # in-plane shear is the Voigt average, out-of-plane shear the Reuss one
    assert math.isclose(C[5, 5], f[0] * mu[0] + f[1] * mu[1], rel_tol=1e-13)
    assert math.isclose(C[3, 3], 1 / (f[0] / mu[0] + f[1] / mu[1]), rel_tol=1e-13)


@pytest.fixture(scope="module")
def sphere16():
    cell = ms.cell_sphere32(16)
    p = o.Problem.from_cell(cell)
    C, res = o.effective_stiffness(p, o.rpm_solve, o.Options(tol=1e-10, p_max=10))
    return cell, p, C, res


def test_sphere_ceff_bounds_symmetry_cubic(sphere16):
    cell, p, C, res = sphere16
    assert all(r.converged for r in res)
    f1 = cell.volume_fraction(1)
    fr = [1 - f1, f1]
    V = o.voigt_bound(fr, p.lam, p.mu)
    R = o.reuss_bound(fr, p.lam, p.mu)
    assert np.max(np.abs(C - C.T)) < 1e-8 * np.max(np.abs(C))
    assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0
    assert np.linalg.eigvalsh(V - 0.5 * (C + C.T)).min() > 0
    assert np.linalg.eigvalsh(0.5 * (C + C.T) - R).min() > 0
    # cubic symmetry of the centred sphere
    s = np.max(np.abs(C))
    assert abs(C[0, 0] - C[1, 1]) < 1e-8 * s and abs(C[1, 1] - C[2, 2]) < 1e-8 * s
    assert abs(C[0, 1] - C[0, 2]) < 1e-8 * s and abs(C[0, 1] - C[1, 2]) < 1e-8 * s
    assert abs(C[3, 3] - C[4, 4]) < 1e-8 * s and abs(C[3, 3] - C[5, 5]) < 1e-8 * s
    off = C.copy()
    off[:3, :3] = 0
    np.fill_diagonal(off, 0)
    assert np.max(np.abs(off)) < 1e-8 * s


def test_equilibrium_error_small_at_convergence(sphere16):
    cell, p, C, res = sphere16
    e = o.equilibrium_error(p, o.stress(p, res[0].eps))
    assert e < 1e-5


def test_c0_independence(sphere16):
    """The converged result does not depend on the reference medium
    (Section 5.5); RPM converges for every choice."""
    cell, p, C, res = sphere16
    E = ms.unit_strain(0)
    for scale, n_max in ((0.6, 3), (1.0, 10), (3.0, 10)):
        q = o.Problem.from_cell(cell)
        q.lam0 = scale * p.lam0
        q.mu0 = scale * p.mu0
        r = o.rpm_solve(q, E, o.Options(tol=1e-10, p_max=40, n_max=n_max, max_iters=4000,
                                        diverge_factor=1e30))
        assert r.converged
        assert np.max(np.abs(r.mean_stress - C[:, 0])) < 1e-7 * np.max(np.abs(C))


def test_hashin_shtrikman_random_spheres():
    """Random non-overlapping spheres, contrast 10: isotropic projections of
    C_eff fall inside the HS bounds (1 % slack for finite-cell anisotropy)."""
    n = 16
    mask, _ = ms.rsa_spheres(n, 3, 2.0, 3.0, 0.15)
    l0, m0 = ms.lame(1.0, 0.3)
    l1, m1 = ms.lame(10.0, 0.3)
    p = o.Problem(phase=mask, lam=np.array([l0, l1]), mu=np.array([m0, m1]),
                  lam0=0.5 * (l0 + l1), mu0=0.5 * (m0 + m1))
    C, res = o.effective_stiffness(p, o.rpm_solve, o.Options(tol=1e-8, p_max=10))
    K, G = o.isotropic_projection(C)
    f1 = float(mask.mean())
    K0, G0 = l0 + 2 * m0 / 3, m0
    K1, G1 = l1 + 2 * m1 / 3, m1
    Kl, Ku, Gl, Gu = o.hashin_shtrikman(1 - f1, K0, G0, K1, G1)
    assert Kl * 0.99 <= K <= Ku * 1.01
    assert Gl * 0.99 <= G <= Gu * 1.01
    assert K > Kl and G > Gl


# ----------------------------------------------------------------------------
# Algorithm 3 (polarization / Accelerated scheme)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("alpha,beta", [(2.0, 2.0), (1.0, 1.0), (1.5, 0.7)])
def test_polarization_homogeneous_closed_form(alpha, beta):
    """C = c C0 uniform (same nu), eps = E + e with e compatible, zero mean:
    F(eps) = E + ((1 - alpha) c + 1) / (c + 1) e  (for alpha = 2 the
    Eyre-Milton contraction (1 - c)/(1 + c), derived independently from the
    Cayley transform of C0^-1 C and the reflection 2 Gamma0 C0 - I)."""
    shape = (6, 8, 8)
    c = 4.0
    l0, m0 = ms.lame(1.5, 0.3)
    p = o.Problem(phase=np.zeros(shape, np.uint8), lam=np.array([c * l0]), mu=np.array([c * m0]),
                  lam0=l0, mu0=m0)
    E = _rng(8).standard_normal(6)
    e = _compatible_field(shape, seed=13, amp=0.2)
    got = o.apply_F_polarization(p, E.reshape(6, 1, 1, 1) + e, E, alpha, beta)
    fac = ((1 - alpha) * c + 1) / (c + 1)
    assert np.max(np.abs(got - (E.reshape(6, 1, 1, 1) + fac * e))) < 1e-12


@pytest.mark.parametrize("alpha,beta", [(2.0, 2.0), (1.0, 1.0), (1.5, 1.5)])
def test_polarization_solution_is_fixed_point_and_solvers_converge(tiny, alpha, beta):
    """The cell-problem solution (dense solve of the basic map) is a fixed
    point of Algorithm 3, and Algorithm 3 alone and wrapped by RPM converge to
    it."""
    p, L = tiny
    E = ms.unit_strain(1)
    ref = np.linalg.solve(np.eye(L.shape[0]) - L, o.uniform(E, p.shape).ravel()).reshape((6,) + p.shape)
    assert np.max(np.abs(o.apply_F_polarization(p, ref, E, alpha, beta) - ref)) < 1e-12
    kw = dict(scheme="polarization", alpha=alpha, beta=beta, tol=1e-11, max_iters=4000)
    for r in (o.basic_solve(p, E, o.Options(**kw)), o.rpm_solve(p, E, o.Options(p_max=20, **kw))):
        assert r.converged
        assert np.max(np.abs(r.eps - ref)) < 1e-8


def test_compatible_projection_fixes_compatible_fields_and_is_idempotent():
    """project_compatible(E + e) = E + e for compatible zero-mean e; applied
    to any field it gives mean E, a compatible fluctuation, and is idempotent."""
    shape = (8, 8, 6)
    p = _prob(shape)
    E = np.array([0.01, -0.02, 0.005, 0.003, -0.004, 0.002])
    e = _compatible_field(shape)
    f = E.reshape(6, 1, 1, 1) + e
    assert np.max(np.abs(o.project_compatible(p, f, E) - f)) < 1e-12 * np.max(np.abs(f))
    g = _rng(21).standard_normal((6,) + shape)
    pg = o.project_compatible(p, g, E)
    assert np.allclose(pg.reshape(6, -1).mean(axis=1), E, atol=1e-13)
    assert np.max(np.abs(o.project_compatible(p, pg, E) - pg)) < 1e-12 * np.max(np.abs(pg))
    xi, _, _ = o.frequencies(p)
    eta = _incompatibility(o.fft_fields(pg - E.reshape(6, 1, 1, 1)), xi)
    assert np.max(np.abs(eta)) < 1e-9 * np.max(np.abs(o.fft_fields(pg))) * np.max(np.abs(xi)) ** 2
    # the projection does not depend on the phases, only on C0
    p2 = o.Problem(phase=np.zeros(shape, np.uint8), lam=np.array([1.0]), mu=np.array([1.0]),
                   lam0=p.lam0, mu0=p.mu0)
    assert np.allclose(o.project_compatible(p2, g, E), pg, atol=1e-14)


@pytest.mark.parametrize("ratio,n_added", [(0.05, 1), (0.3, 2)])
def test_growth_rule_adds_one_or_two_columns_by_the_qr_ratio(ratio, n_added):
    """Eq. 3.8 on hand-built increments: with d1 = xi^nu - xi^(nu-1) = a and
    d2 = xi^(nu-1) - xi^(nu-2) = b orthogonal to a, the QR factors are
    T11 = |a|, T12 = 0, T22 = |b|; the rule keeps q1 = a/|a| alone when
    |T22| <= kappa |T11| and both q1 and q2 = b/|b| otherwise, and H is
    Z^T F_u Z for the vectors kept."""
    prob = _prob((4, 4, 4), seed=2)
    rng = _rng(11)
    a = rng.standard_normal((6, 4, 4, 4))
    b = rng.standard_normal((6, 4, 4, 4))
    b -= o.inner(a, b) / o.inner(a, a) * a
    b *= ratio * o.norm(a) / o.norm(b)
    x0 = rng.standard_normal((6, 4, 4, 4))
    hist = [x0, x0 + b, x0 + b + a]
    st = o.RPMState([], [], np.zeros((0, 0)))
    opts = o.Options(kappa=0.1, p_max=20)
    assert o._grow_basis(prob, st, hist, opts) == n_added
    assert len(st.Z) == n_added
    assert np.allclose(st.Z[0], a / o.norm(a), atol=1e-12)
    if n_added == 2:
        assert np.allclose(st.Z[1], b / o.norm(b), atol=1e-12)
    for i in range(n_added):
        fu = o.apply_F_linear(prob, st.Z[i])
        for j in range(n_added):
            assert math.isclose(st.H[j, i], o.inner(st.Z[j], fu), rel_tol=1e-12, abs_tol=1e-12)


def test_growth_projects_out_the_existing_basis_and_respects_p_max():
    """With a basis Z already present, the increments are first projected
    onto its orthogonal complement (the Q of Eq. 3.8), so an increment
    inside span Z adds nothing; and no column is added beyond p_max."""
    prob = _prob((4, 4, 4), seed=2)
    rng = _rng(12)
    e = rng.standard_normal((6, 4, 4, 4))
    e /= o.norm(e)
    st = o.RPMState([e], [o.apply_F_linear(prob, e)], np.zeros((1, 1)))
    x0 = rng.standard_normal((6, 4, 4, 4))
    hist = [x0, x0 + 2.0 * e, x0 + 5.0 * e]          # both increments inside span Z
    assert o._grow_basis(prob, st, hist, o.Options()) == 0 and len(st.Z) == 1
    a = rng.standard_normal((6, 4, 4, 4))
    b = rng.standard_normal((6, 4, 4, 4))
    hist = [x0, x0 + b + 3.0 * e, x0 + b + a - e]
    assert o._grow_basis(prob, st, hist, o.Options(p_max=2)) == 1    # capped at p_max
    Z = np.array([z.ravel() for z in st.Z])
    w = np.tile(np.repeat([1.0, 1.0, 1.0, 2.0, 2.0, 2.0], 64), 1)
    G = (Z * w) @ Z.T
    assert np.allclose(G, np.eye(2), atol=1e-12)
    # the new column is the normalised part of a - 4e orthogonal to e
    d1 = a - 4.0 * e
    d1 -= o.inner(e, d1) * e
    assert np.allclose(st.Z[1], d1 / o.norm(d1), atol=1e-12)


@pytest.mark.parametrize("m", [(1, 2, 0), (0, 0, 3), (2, 1, 1)])
def test_equilibrium_error_of_a_single_mode_closed_form(m):
    """Algorithm 1's error for sigma(x) = sigma0 + S cos(2 pi m . x) on a unit
    cell (x along the last axis): the only non-zero frequencies are +-m with
    sigma_hat = S/2 each (after the 1/n normalisation), so the error is
    sqrt(2 |S (2 pi m) / 2|^2) / |sigma0| = |S xi_m| / (sqrt(2) |sigma0|),
    whichever half of the spectrum stores +-m."""
    n = 8
    prob = _prob((n, n, n), seed=1)
    rng = _rng(21)
    s0 = rng.standard_normal(6)
    S6 = rng.standard_normal(6)
    c = np.arange(n) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    phase = 2 * math.pi * (m[0] * x + m[1] * y + m[2] * z)
    sig = s0[:, None, None, None] + S6[:, None, None, None] * np.cos(phase)[None]
    S = o.to_full(S6)
    xi = 2 * math.pi * np.array(m, float)
    s0_norm = math.sqrt(float(np.sum(np.array([1, 1, 1, 2, 2, 2]) * s0 * s0)))
    expect = np.linalg.norm(S @ xi) / (math.sqrt(2.0) * s0_norm)
    assert math.isclose(o.equilibrium_error(prob, sig), expect, rel_tol=1e-12)


def test_bound_helpers_against_independent_results():
    """The bound helpers used by the C_eff pins: the isotropic projection of an
    isotropic stiffness returns its own K = lambda + 2 mu / 3 and G = mu; the
    Hashin-Shtrikman bounds collapse to a phase at f = 0 and 1, are ordered
    between the Reuss and Voigt averages, and for equal shear moduli both
    bulk bounds equal Hill's exact result
    1 / (K* + 4G/3) = f1 / (K1 + 4G/3) + f2 / (K2 + 4G/3)."""
    for lam, mu in [(0.6, 0.4), (3.0, 1.2), (1e-3, 2e-3)]:
        K, G = o.isotropic_projection(o.voigt_matrix(lam, mu))
        assert math.isclose(K, lam + 2 * mu / 3, rel_tol=1e-13)
        assert math.isclose(G, mu, rel_tol=1e-13)
    K1, G1, K2, G2 = 1.0, 0.5, 20.0, 7.0
    assert np.allclose(o.hashin_shtrikman(1.0, K1, G1, K2, G2), (K1, K1, G1, G1), rtol=1e-13)
    assert np.allclose(o.hashin_shtrikman(0.0, K1, G1, K2, G2), (K2, K2, G2, G2), rtol=1e-13)
    for f1 in (0.1, 0.4, 0.8):
        Kl, Ku, Gl, Gu = o.hashin_shtrikman(f1, K1, G1, K2, G2)
        f2 = 1 - f1
        assert 1 / (f1 / K1 + f2 / K2) <= Kl <= Ku <= f1 * K1 + f2 * K2
        assert 1 / (f1 / G1 + f2 / G2) <= Gl <= Gu <= f1 * G1 + f2 * G2
        G = 0.9                          # (the shear terms need G2 != G1)
        Kl, Ku, _, _ = o.hashin_shtrikman(f1, K1, G, K2, G * (1 + 1e-12))
        hill = 1 / (f1 / (K1 + 4 * G / 3) + f2 / (K2 + 4 * G / 3)) - 4 * G / 3
        assert math.isclose(Kl, hill, rel_tol=1e-9) and math.isclose(Ku, hill, rel_tol=1e-9)
    # the Reuss and Voigt averages of one phase are its stiffness
    C = o.voigt_matrix(1.3, 0.7)
    assert np.allclose(o.reuss_bound([1.0], [1.3], [0.7]), C, rtol=1e-13)
    assert np.allclose(o.voigt_bound([0.3, 0.7], [1.3, 1.3], [0.7, 0.7]), C, rtol=1e-13)


def test_laminate_closed_form_matches_backus_averages():
    """Layers normal to e3 give a transversely isotropic C_eff whose entries
    are Backus's averages of the layer moduli (M = lambda + 2 mu):
    C33 = <1/M>^-1, C13 = <lambda/M> <1/M>^-1, C66 = <mu>, C44 = <1/mu>^-1,
    C11 = <4 mu (lambda + mu) / M> + <lambda/M>^2 <1/M>^-1, C12 = C11 - 2 C66."""
    f = np.array([0.25, 0.45, 0.30])
    lam = np.array([ms.lame(1, 0.3)[0], ms.lame(40, 0.25)[0], ms.lame(1e-3, 0.3)[0]])
    mu = np.array([ms.lame(1, 0.3)[1], ms.lame(40, 0.25)[1], ms.lame(1e-3, 0.3)[1]])
    C = o.laminate_ceff(f, lam, mu)
    M = lam + 2 * mu
    avg = lambda v: float(np.sum(f * v))          # noqa: E731
    c33 = 1 / avg(1 / M)
    c13 = avg(lam / M) * c33
    c66 = avg(mu)
    c44 = 1 / avg(1 / mu)
    c11 = avg(4 * mu * (lam + mu) / M) + avg(lam / M) ** 2 * c33
    c12 = c11 - 2 * c66
    ref = np.array([[c11, c12, c13, 0, 0, 0], [c12, c11, c13, 0, 0, 0], [c13, c13, c33, 0, 0, 0],
                    [0, 0, 0, c44, 0, 0], [0, 0, 0, 0, c44, 0], [0, 0, 0, 0, 0, c66]])
    assert np.allclose(C, ref, rtol=1e-12, atol=1e-14 * np.max(np.abs(ref)))


def test_tensor_helpers_stress_and_polarization_by_independent_routes():
    """The stored-component helpers against full 3x3 tensors: inner() is the
    Frobenius contraction of the full tensors; stress() equals the full
    fourth-order contraction C_ijkl eps_kl of each phase and the Voigt matrix
    applied to engineering strains; polarization() is stress() with C - C0."""
    prob = _prob((2, 3, 4), seed=5, c_ratio=(1.0, 7.0), vf=0.5)
    rng = _rng(31)
    a = rng.standard_normal((6, 2, 3, 4))
    b = rng.standard_normal((6, 2, 3, 4))
    assert math.isclose(o.inner(a, b), float(np.sum(o.to_full(a) * o.to_full(b))), rel_tol=1e-13)
    assert np.allclose(o.from_full(o.to_full(a)), a)
    sig = o.stress(prob, a)
    full = o.to_full(a)
    for r in range(2):
        sel = prob.phase == r
        C4 = o.isotropic_stiffness(prob.lam[r], prob.mu[r])
        ref = np.einsum("ijkl,kl...->ij...", C4, full[:, :, sel])
        assert np.allclose(o.to_full(sig)[:, :, sel], ref, rtol=1e-13, atol=1e-13)
        eng = a[:, sel] * np.array([1, 1, 1, 2, 2, 2])[:, None]
        assert np.allclose(sig[:, sel], o.voigt_matrix(prob.lam[r], prob.mu[r]) @ eng,
                           rtol=1e-13, atol=1e-13)
    tau = o.polarization(prob, a)
    p0 = o.Problem(phase=prob.phase, lam=prob.lam - prob.lam0, mu=prob.mu - prob.mu0,
                   lam0=prob.lam0, mu0=prob.mu0)
    assert np.allclose(tau, o.stress(p0, a), rtol=1e-13, atol=1e-13)


def test_recentring_reading_preserves_the_map():
    """The float32 re-centring of the GPU solver (eps = base + y, iterate
    y -> r + F_u y with r = F(base) - base) is the same affine map written in
    shifted coordinates: F(base + y) - base = r + F_u y for any base and y, so
    Z, H and the fixed point are unchanged."""
    prob = _prob((4, 4, 4), seed=4, c_ratio=(1.0, 30.0))
    rng = _rng(41)
    E = np.array([0.2, -0.1, 0.05, 0.03, 0.0, -0.02])
    base = rng.standard_normal((6, 4, 4, 4))
    y = rng.standard_normal((6, 4, 4, 4))
    lhs = o.apply_F(prob, base + y, E) - base
    r = o.apply_F(prob, base, E) - base
    rhs = r + o.apply_F_linear(prob, y)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.max(np.abs(lhs)))


# ----------------------------------------------------------------------------
# The stopping test (fixed-point increment) on a homogeneous cell
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("E_comp,E_val,U_comp,expected_over_a", [
    (0, 1.0, 5, 1.0),              # E = e1 (x) e1, |E| = 1; u12 = a: |U| = a sqrt 2
    (3, 0.5, 0, 1.0),              # E = eps23 = 1/2 (gamma23 = 1), |E| = 1/sqrt 2; u11 = a
    (3, 0.5, 4, math.sqrt(2.0)),   # same E; u13 = a: |U| = a sqrt 2
    (2, 2.0, 1, 0.25 * math.sqrt(2.0)),   # E = 2 e3 (x) e3, |E| = 2; u22 = a: a / (2 sqrt 2)
])
def test_residual_is_frobenius_rms_of_the_increment_over_the_norm_of_E(E_comp, E_val, U_comp,
                                                                      expected_over_a):
    """On a homogeneous cell (C = C0) the polarization vanishes, so F(eps) = E
    for every eps (Section 2, Eq. 2.5).  With eps = E + U cos(2 pi m . x) the
    increment F(eps) - eps is -U cos(.), and the stopping test of reading 6
    is its root-mean-square Frobenius norm over the voxels divided by the
    Frobenius norm of E: sqrt(<cos^2>) |U|_F / |E|_F = |U|_F / (sqrt 2 |E|_F),
    the mean of cos^2 over the grid being 1/2 for a mode whose double is not
    a multiple of the grid in every direction.  The expected values are
    worked out by hand from the full 3x3 tensors (a shear entry appears
    twice), so a dropped sqrt(n), a missing shear weight or a wrong norm of E
    changes them."""
    shape = (4, 6, 8)
    lam, mu = ms.lame(1.0, 0.3)
    prob = o.Problem(phase=np.zeros(shape, np.uint8), lam=np.array([lam]), mu=np.array([mu]),
                     lam0=lam, mu0=mu)
    E = np.zeros(6)
    E[E_comp] = E_val
    nz, ny, nx = shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny,
                          (np.arange(nx) + 0.5) / nx, indexing="ij")
    wave = np.cos(2 * np.pi * (1 * x + 2 * y + 1 * z))
    a = 0.37
    eps = o.uniform(E, shape)
    eps[U_comp] += a * wave
    xi = o.apply_F(prob, eps, E)
    assert np.allclose(xi, o.uniform(E, shape), atol=1e-13)
    got = o.residual(prob, xi, eps, E)
    assert abs(got - a * expected_over_a) < 1e-12 * a
