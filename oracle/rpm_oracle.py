"""FP64 CPU oracle for the RPM-FFT method (test infrastructure only).

This module is the plain, slow reference that the CUDA path is checked
against.  Only the test-suite, the package smoke check and the CPU-baseline
leg of the benchmark may import it; the library itself never calls it.

It follows the paper (Peng, Nepal & Dayal, "Effective response of
heterogeneous materials using the recursive projection method", CMAME 2020):

* Section 2, Eqs. (2.1)-(2.5): periodic cell problem, polarization with a
  homogeneous reference medium C0, Lippmann-Schwinger equation in Fourier
  space with the Green operator Gamma0 of C0.
* Algorithm 1: the classical (basic) fixed-point scheme and its
  equilibrium error.
* Section 3, Eqs. (3.1)-(3.13) and Algorithm 2: the recursive projection
  method wrapped around the fixed-point map F of Eq. (3.9).
* Section 5.5, Algorithm 3: the polarization-based (Accelerated for
  alpha = beta = 2) fixed-point map, alone or wrapped by RPM.

A library FFT (numpy.fft) serves as the Fourier transform step; everything
else is written out in plain numpy, in float64, with no blocking or fusion.

Readings where the paper is silent (each one is listed with its reason in the
repository's design notes):

* frequencies xi_j = 2 pi m_j / L_j with m_j in numpy ``fftfreq`` order and
  L_j = 1 unless given;
* the Green operator, which the paper does not print, is obtained from
  div(C0 : eps(v) + tau) = 0 with d/dx_j -> i xi_j:
  Gamma0_hat : tau_hat = sym(xi (x) N0 (tau_hat xi)), N0 = K0^-1,
  K0_ik = C0_ijkl xi_j xi_l; this module inverts K0 numerically;
* Nyquist frequencies (index N/2 of an even axis) that coexist with another
  non-zero frequency component get Gamma0_hat := 0 ("zero mixed"), pure-axis
  Nyquist frequencies are kept;
* F is evaluated in polarization form F(eps) = E - Gamma0 * ((C - C0) : eps),
  which equals the classical form of Eq. (3.9) on compatible fields;
* inner products are the tensor Frobenius product summed over voxels
  (weights 1,1,1,2,2,2 on the stored components);
* the stopping test is the fixed-point increment
  ||F(eps) - eps|| / (||E|| sqrt(n)); the equilibrium error of Algorithm 1
  is reported as a diagnostic;
* "T11 >> T22" of Eq. (3.8) is read as |T22| <= kappa |T11| with
  kappa = 0.1; the basis is capped at p_max vectors; the iteration counter
  nu counts fixed-point steps since the last basis growth;
* Algorithm 3's s_b is read as alpha sigma - beta C0 : eps (the printed plus
  sign does not keep the solution a fixed point).

Parity: every function here is pinned by tests under tests/ against closed
forms, brute-force solves, invariants or library routines.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# stored order of symmetric tensor components: 11, 22, 33, 23, 13, 12
PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
WEIGHTS = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])

NYQ_ZERO_MIXED = 0
NYQ_SIGNED = 1      # plain fftfreq signs everywhere (not used by the tests: the
                    # result is then not real; see green_mask)


# ----------------------------------------------------------------------------
# tensor helpers
# ----------------------------------------------------------------------------
def to_full(f6):
    """[6, ...] stored components -> [3, 3, ...] symmetric tensor."""
    f6 = np.asarray(f6)
    out = np.empty((3, 3) + f6.shape[1:], dtype=f6.dtype)
    for c, (i, j) in enumerate(PAIRS):
        out[i, j] = f6[c]
        out[j, i] = f6[c]
    return out


def from_full(t):
    """[3, 3, ...] tensor -> [6, ...] stored components (symmetric part)."""
    t = np.asarray(t)
    return np.stack([0.5 * (t[i, j] + t[j, i]) for (i, j) in PAIRS])


def inner(a, b) -> float:
    """Tensor Frobenius inner product summed over voxels."""
    a = np.asarray(a).reshape(6, -1)
    b = np.asarray(b).reshape(6, -1)
    return float(np.sum(WEIGHTS[:, None] * a * b))


def norm(a) -> float:
    return math.sqrt(max(inner(a, a), 0.0))


def isotropic_stiffness(lam: float, mu: float) -> np.ndarray:
    """C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk) as a [3,3,3,3] array."""
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def voigt_matrix(lam: float, mu: float) -> np.ndarray:
    """6x6 Voigt matrix (engineering shear strains) of an isotropic C."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[0, 0] = C[1, 1] = C[2, 2] = lam + 2 * mu
    C[3, 3] = C[4, 4] = C[5, 5] = mu
    return C


# ----------------------------------------------------------------------------
# problem definition (Section 2)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    """Periodic cell: phase map, per-phase isotropic moduli, reference medium."""
    phase: np.ndarray          # [nz, ny, nx] integer phase ids
    lam: np.ndarray            # per phase
    mu: np.ndarray
    lam0: float
    mu0: float
    lengths: tuple = (1.0, 1.0, 1.0)   # (Lz, Ly, Lx)
    nyquist: int = NYQ_ZERO_MIXED

    @property
    def shape(self):
        return tuple(self.phase.shape)

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    @classmethod
    def from_cell(cls, cell, **kw):
        return cls(phase=np.asarray(cell.phase), lam=np.asarray(cell.lam, float),
                   mu=np.asarray(cell.mu, float), lam0=float(cell.lam0),
                   mu0=float(cell.mu0), **kw)


def stress(prob: Problem, eps: np.ndarray) -> np.ndarray:
    """sigma = C(x) : eps for isotropic phases, Eq. (2.2)."""
    lam = prob.lam[prob.phase]
    mu = prob.mu[prob.phase]
    tr = eps[0] + eps[1] + eps[2]
    sig = 2.0 * mu[None] * eps
    sig[:3] += (lam * tr)[None]
    return sig


def polarization(prob: Problem, eps: np.ndarray) -> np.ndarray:
    """tau = (C(x) - C0) : eps, the polarization defined before Eq. (2.3)."""
    dlam = prob.lam[prob.phase] - prob.lam0
    dmu = prob.mu[prob.phase] - prob.mu0
    tr = eps[0] + eps[1] + eps[2]
    tau = 2.0 * dmu[None] * eps
    tau[:3] += (dlam * tr)[None]
    return tau


def _freq_index(n: int) -> np.ndarray:
    """Integer frequencies m in fftfreq order (index n/2 -> -n/2)."""
    return np.fft.fftfreq(n) * n


def frequencies(prob: Problem):
    """Half-spectrum wave vectors xi_j = 2 pi m_j / L_j (x along the rfft axis).

    Returns (xi, m, nyq): xi [3, nz, ny, nxh] in (x, y, z) order, the integer
    frequencies m likewise, and a boolean [nz, ny, nxh] Nyquist flag per axis.
    """
    nz, ny, nx = prob.shape
    Lz, Ly, Lx = prob.lengths
    mz = _freq_index(nz)
    my = _freq_index(ny)
    mx = np.arange(nx // 2 + 1).astype(float)
    if nx % 2 == 0:
        mx[-1] = -(nx // 2)          # the Nyquist index keeps the fftfreq sign
    MZ, MY, MX = np.meshgrid(mz, my, mx, indexing="ij")
    m = np.stack([MX, MY, MZ])
    xi = np.stack([2 * np.pi * MX / Lx, 2 * np.pi * MY / Ly, 2 * np.pi * MZ / Lz])
    nyq = np.stack([
        (nx % 2 == 0) & (np.abs(MX) == nx // 2),
        (ny % 2 == 0) & (np.abs(MY) == ny // 2) & (ny > 1),
        (nz % 2 == 0) & (np.abs(MZ) == nz // 2) & (nz > 1),
    ])
    # a length-1 or length-2 axis: index n/2 of n = 2 is a Nyquist index too
    if nx == 1:
        nyq[0] = False
    return xi, m, nyq


def green_mask(prob: Problem) -> np.ndarray:
    """Frequencies where Gamma0_hat is applied (False: k = 0, and mixed Nyquist
    frequencies under the "zero mixed" reading)."""
    xi, m, nyq = frequencies(prob)
    nonzero = (m != 0)
    keep = nonzero.any(axis=0)
    if prob.nyquist == NYQ_ZERO_MIXED:
        mixed = nyq.any(axis=0) & (nonzero.sum(axis=0) >= 2)
        keep &= ~mixed
    return keep


def acoustic_tensor_inverse(xi: np.ndarray, lam0: float, mu0: float) -> np.ndarray:
    """N0 = K0^-1 with K0_ik = C0_ijkl xi_j xi_l, inverted numerically.

    xi: [3, M] wave vectors (non-zero).  Returns [M, 3, 3]."""
    C0 = isotropic_stiffness(lam0, mu0)
    K0 = np.einsum("ijkl,jm,lm->mik", C0, xi, xi)
    return np.linalg.inv(K0)


def gamma_hat_apply(prob: Problem, tau_hat: np.ndarray) -> np.ndarray:
    """Gamma0_hat(xi) : tau_hat per frequency (Eq. 2.5), zero where masked.

    tau_hat: [6, nz, ny, nxh] complex.  Returns the same shape."""
    xi, _, _ = frequencies(prob)
    keep = green_mask(prob)
    out = np.zeros_like(tau_hat)
    idx = np.nonzero(keep)
    if idx[0].size == 0:
        return out
    x = xi[:, idx[0], idx[1], idx[2]]                       # [3, M]
    key = (prob.shape, prob.lengths, prob.nyquist, prob.lam0, prob.mu0)
    cache = getattr(prob, "_n0_cache", None)
    if cache is None or cache[0] != key:
        cache = (key, acoustic_tensor_inverse(x, prob.lam0, prob.mu0))
        prob._n0_cache = cache
    N0 = cache[1]                                            # [M, 3, 3]
    t = to_full(tau_hat[:, idx[0], idx[1], idx[2]])          # [3, 3, M]
    v = np.einsum("ijm,jm->im", t, x)                        # tau_hat . xi
    w = np.einsum("mik,km->im", N0, v)                       # N0 (tau_hat xi)
    g = 0.5 * (np.einsum("km,lm->klm", x, w) + np.einsum("lm,km->klm", x, w))
    res = from_full(g)
    out[:, idx[0], idx[1], idx[2]] = res
    return out


def fft_fields(f: np.ndarray) -> np.ndarray:
    """Real [6, nz, ny, nx] -> half spectrum [6, nz, ny, nx//2+1] (unnormalised)."""
    return np.fft.rfftn(f, axes=(1, 2, 3))


def ifft_fields(fh: np.ndarray, shape) -> np.ndarray:
    return np.fft.irfftn(fh, s=shape, axes=(1, 2, 3))


def apply_gamma_raw(prob: Problem, tau: np.ndarray) -> np.ndarray:
    """-Gamma0 * tau with zero mean (Eq. 2.4)."""
    th = fft_fields(tau)
    eh = -gamma_hat_apply(prob, th)
    return ifft_fields(eh, prob.shape)


def apply_F(prob: Problem, eps: np.ndarray, E) -> np.ndarray:
    """Fixed-point map F (Eq. 3.9) in polarization form:
    F(eps) = E - Gamma0 * ((C - C0) : eps), mean E (Eqs. 2.3-2.5)."""
    E = np.asarray(E, float)
    xi = apply_gamma_raw(prob, polarization(prob, eps))
    return xi + E.reshape(6, 1, 1, 1)


def project_compatible(prob: Problem, eps: np.ndarray, E) -> np.ndarray:
    """E + Gamma0 * (C0 : eps): the field of mean E whose fluctuation is the
    compatible part of eps's fluctuation (Section 2: Gamma0 C0 acts as the
    identity on compatible fluctuations and Gamma0 annihilates equilibrated
    stress fluctuations).  Used to clean a warm-start guess."""
    E = np.asarray(E, float)
    tr = eps[0] + eps[1] + eps[2]
    tau0 = 2.0 * prob.mu0 * eps
    tau0[:3] += prob.lam0 * tr[None]
    return E.reshape(6, 1, 1, 1) - apply_gamma_raw(prob, tau0)


def apply_F_classical(prob: Problem, eps: np.ndarray, E) -> np.ndarray:
    """Eq. (3.9) as printed: F^-1[F[eps] - Gamma0_hat : F[C : eps]], with the
    zero frequency set to E (Algorithm 1)."""
    E = np.asarray(E, float)
    eh = fft_fields(eps)
    sh = fft_fields(stress(prob, eps))
    out = eh - gamma_hat_apply(prob, sh)
    out[:, 0, 0, 0] = E * prob.n
    return ifft_fields(out, prob.shape)


def apply_F_polarization(prob: Problem, eps: np.ndarray, E, alpha: float = 2.0,
                         beta: float = 2.0) -> np.ndarray:
    """Algorithm 3 (polarization-based scheme; alpha = beta = 2 is the
    Accelerated scheme), Section 5.5, with s_b read as alpha sigma - beta C0 eps.

    Steps in the algorithm's order:
      sigma = C : eps;  s_a = sigma + (1 - beta) C0 : eps;
      s_b = alpha sigma - beta C0 : eps;
      eps_b_hat = -Gamma0_hat : s_b_hat (k != 0),  eps_b_hat(0) = beta E;
      eps_next = (C + C0)^-1 : (s_a + C0 : eps_b).
    (The listing prints s_b = alpha sigma + beta C0 eps; with that sign the
    cell-problem solution is not a fixed point, so the minus sign is taken.)"""
    E = np.asarray(E, float)
    c0 = Problem(phase=np.zeros(prob.shape, np.uint8), lam=np.array([prob.lam0]),
                 mu=np.array([prob.mu0]), lam0=0.0, mu0=0.0, lengths=prob.lengths,
                 nyquist=prob.nyquist)
    sig = stress(prob, eps)
    c0eps = stress(c0, eps)
    s_a = sig + (1.0 - beta) * c0eps
    s_b = alpha * sig - beta * c0eps
    sh = fft_fields(s_b)
    eh = -gamma_hat_apply(prob, sh)
    eh[:, 0, 0, 0] = beta * E * prob.n
    eps_b = ifft_fields(eh, prob.shape)
    t = s_a + stress(c0, eps_b)
    # (C + C0)^-1 of an isotropic stiffness (lam_s, mu_s):
    #   X = (t - lam_s / (3 lam_s + 2 mu_s) tr(t) I) / (2 mu_s)
    lam_s = prob.lam[prob.phase] + prob.lam0
    mu_s = prob.mu[prob.phase] + prob.mu0
    tr = t[0] + t[1] + t[2]
    out = t.copy()
    out[:3] -= (lam_s / (3.0 * lam_s + 2.0 * mu_s) * tr)[None]
    return out / (2.0 * mu_s)[None]


def fixed_point_map(prob: Problem, opts):
    """The map F of Algorithm 1/2 for opts.scheme: 'basic' (Eq. 3.9) or
    'polarization' (Algorithm 3 with opts.alpha, opts.beta)."""
    if getattr(opts, "scheme", "basic") == "polarization":
        a, b = opts.alpha, opts.beta
        return lambda eps, E: apply_F_polarization(prob, eps, E, a, b)
    return lambda eps, E: apply_F(prob, eps, E)


def uniform(E, shape) -> np.ndarray:
    return np.broadcast_to(np.asarray(E, float).reshape(6, 1, 1, 1), (6,) + tuple(shape)).copy()


def residual(prob: Problem, xi: np.ndarray, eps: np.ndarray, E) -> float:
    """Fixed-point increment ||F(eps) - eps|| / (||E|| sqrt(n))."""
    En = math.sqrt(float(np.sum(WEIGHTS * np.asarray(E, float) ** 2)))
    return norm(xi - eps) / (En * math.sqrt(prob.n))


def equilibrium_error(prob: Problem, sig: np.ndarray) -> float:
    """Algorithm 1's error: <|k . sigma_hat(k)|^2>^(1/2) / |sigma_hat(0)|,
    with sigma_hat normalised by 1/n (mean at k = 0), summed over frequencies
    where Gamma0_hat is applied."""
    sh = fft_fields(sig) / prob.n
    xi, _, _ = frequencies(prob)
    keep = green_mask(prob)
    S = to_full(sh)
    div = np.einsum("ij...,j...->i...", S, xi)                  # [3, nz, ny, nxh]
    nx = prob.shape[2]
    # half spectrum: interior kx columns stand for two frequencies
    wgt = np.full(sh.shape[-1], 2.0)
    wgt[0] = 1.0
    if nx % 2 == 0:
        wgt[-1] = 1.0
    p = np.sum(np.abs(div) ** 2, axis=0) * wgt[None, None, :] * keep
    mean = sh[:, 0, 0, 0].real
    return math.sqrt(float(np.sum(p))) / math.sqrt(float(np.sum(WEIGHTS * mean ** 2)))


# ----------------------------------------------------------------------------
# solvers
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Options:
    tol: float = 1e-6
    max_iters: int = 5000
    n_max: int = 10
    p_max: int = 20
    kappa: float = 0.1          # |T22| <= kappa |T11|  ->  add one vector
    diverge_factor: float = 1e10
    scheme: str = "basic"       # or "polarization" (Algorithm 3)
    alpha: float = 2.0
    beta: float = 2.0


@dataclasses.dataclass
class Result:
    eps: np.ndarray
    converged: bool
    status: str
    iters: int = 0
    f_applies: int = 0
    basis: int = 0
    residual: float = float("nan")
    residuals: list = dataclasses.field(default_factory=list)
    mean_stress: np.ndarray | None = None
    growth_iters: list = dataclasses.field(default_factory=list)


def _finish(prob, res: Result) -> Result:
    res.mean_stress = stress(prob, res.eps).reshape(6, -1).mean(axis=1)
    return res


def basic_solve(prob: Problem, E, opts: Options | None = None, eps0=None) -> Result:
    """Algorithm 1: eps^0 = E, eps^{i+1} = F(eps^i) until the increment
    residual is below tol."""
    opts = opts or Options()
    F = fixed_point_map(prob, opts)
    eps = uniform(E, prob.shape) if eps0 is None else np.array(eps0, float)
    xi = F(eps, E)
    nF = 1
    r = residual(prob, xi, eps, E)
    r0 = r
    hist = [r]
    it = 0
    while r > opts.tol:
        if it >= opts.max_iters:
            return _finish(prob, Result(eps, False, "not_converged", it, nF, 0, r, hist))
        eps = xi
        xi = F(eps, E)
        nF += 1
        it += 1
        r = residual(prob, xi, eps, E)
        hist.append(r)
        if not math.isfinite(r) or r > opts.diverge_factor * max(r0, 1e-300):
            return _finish(prob, Result(eps, False, "diverged", it, nF, 0, r, hist))
    return _finish(prob, Result(eps, True, "ok", it, nF, 0, r, hist))


def apply_F_linear(prob: Problem, u: np.ndarray, opts=None) -> np.ndarray:
    """Jacobian F_u applied to u: F(u) with E = 0 (F is affine)."""
    if opts is not None and getattr(opts, "scheme", "basic") == "polarization":
        return apply_F_polarization(prob, u, np.zeros(6), opts.alpha, opts.beta)
    return apply_gamma_raw(prob, polarization(prob, u))


@dataclasses.dataclass
class RPMState:
    Z: list
    FZ: list
    H: np.ndarray


def _grow_basis(prob, st: RPMState, hist, opts: Options) -> int:
    """In(q, Z) of Algorithm 2 with Eq. (3.8): QR of the Q-projected latest
    increments D = [dq^nu, dq^(nu-1)] (newest first), add one or two
    orthonormal columns, then extend H = Z^T F_u Z."""
    def Qproj(v):
        for zj in st.Z:
            v = v - inner(zj, v) * zj
        return v
    d1 = Qproj(hist[-1] - hist[-2])
    d2 = Qproj(hist[-2] - hist[-3])
    T11 = norm(d1)
    scale = max(norm(hist[-1]), 1e-300)
    if not (T11 > 1e-14 * scale):
        return 0
    u1 = d1 / T11
    T12 = inner(u1, d2)
    r2 = d2 - T12 * u1
    T22 = norm(r2)
    cands = [u1]
    if abs(T22) > opts.kappa * abs(T11):
        cands.append(r2 / T22)
    added = 0
    for u in cands:
        if len(st.Z) >= opts.p_max:
            break
        for _ in range(2):                  # classical Gram-Schmidt, twice
            u = Qproj(u)
        nu_ = norm(u)
        if not (nu_ > 1e-10):
            continue
        u = u / nu_
        st.Z.append(u)
        st.FZ.append(apply_F_linear(prob, u, opts))
        added += 1
    p = len(st.Z)
    st.H = np.array([[inner(st.Z[i], st.FZ[j]) for j in range(p)] for i in range(p)])
    return added


def rpm_solve(prob: Problem, E, opts: Options | None = None, eps0=None) -> Result:
    """Algorithm 2 (RPM-FFT), with the reduced-coordinate form Eqs. (3.10)-(3.13).

    eps^0 = E (or a given compatible start), xi^0 = F(eps^0); each step:
    z = Z^T eps, zeta = Z^T xi, z+ = z + (I - H)^-1 (zeta - z),
    eps <- Z z+ + (xi - Z zeta), xi <- F(eps); after more than n_max
    fixed-point steps since the last growth the basis grows.
    """
    opts = opts or Options()
    F = fixed_point_map(prob, opts)
    E = np.asarray(E, float)
    eps = uniform(E, prob.shape) if eps0 is None else np.array(eps0, float)
    xi = F(eps, E)
    nF = 1
    st = RPMState([], [], np.zeros((0, 0)))
    hist = [xi]
    r = residual(prob, xi, eps, E)
    r0 = r
    rs = [r]
    nu = 0
    it = 0
    growth = []
    while r > opts.tol:
        if it >= opts.max_iters:
            return _finish(prob, Result(eps, False, "not_converged", it, nF, len(st.Z), r, rs, growth_iters=growth))
        p = len(st.Z)
        if p:
            z = np.array([inner(zj, eps) for zj in st.Z])
            zeta = np.array([inner(zj, xi) for zj in st.Z])
            zp = z + np.linalg.solve(np.eye(p) - st.H, zeta - z)
            eps = xi.copy()
            for j in range(p):
                eps += (zp[j] - zeta[j]) * st.Z[j]
        else:
            eps = xi
        xi = F(eps, E)
        nF += 1
        it += 1
        nu += 1
        hist = (hist + [xi])[-3:]
        r = residual(prob, xi, eps, E)
        rs.append(r)
        if not math.isfinite(r) or r > opts.diverge_factor * max(r0, 1e-300):
            return _finish(prob, Result(eps, False, "diverged", it, nF, len(st.Z), r, rs, growth_iters=growth))
        if r <= opts.tol:
            break
        if nu > opts.n_max:
            if len(st.Z) < opts.p_max and len(hist) == 3:
                added = _grow_basis(prob, st, hist, opts)
                nF += added
                if added:
                    growth.append(it)
            nu = 0
    return _finish(prob, Result(eps, True, "ok", it, nF, len(st.Z), r, rs, growth_iters=growth))


def effective_stiffness(prob: Problem, solver=rpm_solve, opts: Options | None = None):
    """C_eff (6x6 Voigt, engineering shear) from six unit macroscopic strains;
    column j is the mean stress of load j in Voigt order."""
    C = np.zeros((6, 6))
    results = []
    for j in range(6):
        E = np.zeros(6)
        E[j] = 1.0 if j < 3 else 0.5
        res = solver(prob, E, opts)
        C[:, j] = res.mean_stress
        results.append(res)
    return C, results


# ----------------------------------------------------------------------------
# closed forms and bounds used to pin the solvers
# ----------------------------------------------------------------------------
def laminate_ceff(fracs, lams, mus) -> np.ndarray:
    """Exact C_eff of a laminate with layers normal to e3 (Voigt, engineering
    shear): in-plane strains are uniform, sigma_33, sigma_13, sigma_23 are
    uniform across layers."""
    f = np.asarray(fracs, float)
    lam = np.asarray(lams, float)
    mu = np.asarray(mus, float)
    M = lam + 2 * mu
    C = np.zeros((6, 6))
    for j in range(6):
        E = np.zeros(6)
        E[j] = 1.0 if j < 3 else 0.5
        E11, E22, E33, E23, E13, E12 = E
        S = (E33 + (E11 + E22) * np.sum(f * lam / M)) / np.sum(f / M)
        e33 = (S - lam * (E11 + E22)) / M                  # per layer
        s23 = E23 / np.sum(f / (2 * mu))
        s13 = E13 / np.sum(f / (2 * mu))
        tr = E11 + E22 + e33
        s11 = lam * tr + 2 * mu * E11
        s22 = lam * tr + 2 * mu * E22
        s12 = 2 * mu * E12
        C[:, j] = [np.sum(f * s11), np.sum(f * s22), S, s23, s13, np.sum(f * s12)]
    return C


def voigt_bound(fracs, lams, mus) -> np.ndarray:
    return sum(f * voigt_matrix(l, m) for f, l, m in zip(fracs, lams, mus))


def reuss_bound(fracs, lams, mus) -> np.ndarray:
    S = sum(f * np.linalg.inv(voigt_matrix(l, m)) for f, l, m in zip(fracs, lams, mus))
    return np.linalg.inv(S)


def isotropic_projection(C: np.ndarray) -> tuple[float, float]:
    """Bulk and shear moduli of the isotropic (Voigt-average) projection."""
    K = (C[0, 0] + C[1, 1] + C[2, 2] + 2 * (C[0, 1] + C[0, 2] + C[1, 2])) / 9.0
    G = ((C[0, 0] + C[1, 1] + C[2, 2]) - (C[0, 1] + C[0, 2] + C[1, 2])
         + 3 * (C[3, 3] + C[4, 4] + C[5, 5])) / 15.0
    return K, G


def hashin_shtrikman(f1, K1, G1, K2, G2):
    """HS bounds (lower, upper) on bulk and shear modulus for two well-ordered
    isotropic phases (phase 1 the softer): returns (Kl, Ku, Gl, Gu)."""
    f2 = 1.0 - f1
    Kl = K1 + f2 / (1.0 / (K2 - K1) + 3 * f1 / (3 * K1 + 4 * G1))
    Ku = K2 + f1 / (1.0 / (K1 - K2) + 3 * f2 / (3 * K2 + 4 * G2))
    Gl = G1 + f2 / (1.0 / (G2 - G1) + 6 * f1 * (K1 + 2 * G1) / (5 * G1 * (3 * K1 + 4 * G1)))
    Gu = G2 + f1 / (1.0 / (G1 - G2) + 6 * f2 * (K2 + 2 * G2) / (5 * G2 * (3 * K2 + 4 * G2)))
    return Kl, Ku, Gl, Gu


def dense_linear_operator(prob: Problem, opts=None) -> np.ndarray:
    """Dense matrix of F_u on R^(6n) (stored components), built column by
    column by applying F with E = 0 to unit vectors (tiny grids only)."""
    N = 6 * prob.n
    L = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        L[:, k] = apply_F_linear(prob, e.reshape((6,) + prob.shape), opts).ravel()
    return L
