"""Seeded synthetic periodic microstructures and load cases.

This module only *generates inputs*: voxel phase maps, per-phase isotropic
elastic moduli, the reference medium and macroscopic strains.  It contains no
step of the solution method (no polarization, Fourier transform, Green
operator or iteration), so both the FP64 oracle and the CUDA path may use it.

Conventions shared by every generator
-------------------------------------
* A grid is ``(nz, ny, nx)``; arrays are indexed ``[z, y, x]`` with x fastest.
* Voxel centres sit at ``((i + 1/2) / n)`` in a unit periodic cell.
* Inclusion membership is the strict test ``distance < radius`` with
  periodic (minimum-image) distances.
* Phase 0 is the matrix.  Every phase is isotropic with Poisson ratio 0.3
  unless stated, so all phases share nu with the reference medium.
* Symmetric 2-tensors are stored as 6 components in the order
  (11, 22, 33, 23, 13, 12) - tensor components, not engineering shears.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Cell", "lame", "unit_strain", "centred_sphere", "rsa_spheres", "ellipsoids",
    "laminate", "random_two_phase", "cell_sphere32", "cell_nearvoid",
    "cell_ellipsoids", "cell_laminate", "cell_batch_member", "cell_fibre2d", "BATCH_SIZES",
    "cell_fno_member", "fno_params", "strain_direction",
]

BATCH_SIZES = (32, 48, 64, 96)


def lame(E: float, nu: float) -> tuple[float, float]:
    """Young's modulus and Poisson ratio -> Lame constants (lambda, mu)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def unit_strain(j: int) -> np.ndarray:
    """Macroscopic strain of the j-th Voigt unit load (tensor components).

    j = 0, 1, 2: eps_jj = 1.  j = 3, 4, 5: engineering shear gamma = 1, i.e.
    the tensor component eps_ij = eps_ji = 1/2.
    """
    E = np.zeros(6)
    E[j] = 1.0 if j < 3 else 0.5
    return E


@dataclasses.dataclass
class Cell:
    """A periodic two- (or multi-) phase cell with isotropic phases."""
    phase: np.ndarray            # uint8 [nz, ny, nx]
    lam: np.ndarray              # float64 [n_phases]
    mu: np.ndarray               # float64 [n_phases]
    lam0: float                  # reference medium
    mu0: float
    name: str = ""

    @property
    def shape(self):
        return self.phase.shape

    @property
    def n_vox(self) -> int:
        return int(self.phase.size)

    def volume_fraction(self, r: int = 1) -> float:
        return float(np.mean(self.phase == r))


def _centres(n: int) -> np.ndarray:
    return (np.arange(n) + 0.5) / n


def _wrap(d: np.ndarray) -> np.ndarray:
    return d - np.round(d)


def centred_sphere(n: int, radius: float = 0.25) -> np.ndarray:
    """One sphere of the given radius (fraction of L) at the cell centre."""
    c = _centres(n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    d2 = _wrap(x - 0.5) ** 2 + _wrap(y - 0.5) ** 2 + _wrap(z - 0.5) ** 2
    return (d2 < radius * radius).astype(np.uint8)


def _stamp_sphere(mask: np.ndarray, centre_vox, r_vox: float) -> None:
    """Set voxels whose centre lies strictly within r_vox of centre_vox
    (coordinates in voxel units, periodic)."""
    nz, ny, nx = mask.shape
    cz, cy, cx = centre_vox
    rr = int(math.ceil(r_vox)) + 1
    iz = np.arange(int(math.floor(cz)) - rr, int(math.floor(cz)) + rr + 1)
    iy = np.arange(int(math.floor(cy)) - rr, int(math.floor(cy)) + rr + 1)
    ix = np.arange(int(math.floor(cx)) - rr, int(math.floor(cx)) + rr + 1)
    dz = (iz + 0.5 - cz)[:, None, None]
    dy = (iy + 0.5 - cy)[None, :, None]
    dx = (ix + 0.5 - cx)[None, None, :]
    inside = dz * dz + dy * dy + dx * dx < r_vox * r_vox
    sel = np.nonzero(inside)
    mask[iz[sel[0]] % nz, iy[sel[1]] % ny, ix[sel[2]] % nx] = 1


def rsa_spheres(n: int, seed: int, r_min: float, r_max: float, target_vf: float,
                max_tries: int = 200000) -> tuple[np.ndarray, list]:
    """Random sequential addition of non-overlapping spheres.

    Radii U[r_min, r_max] voxels, centres uniform in the cell; a candidate is
    rejected if its periodic centre distance to any accepted sphere is below
    r1 + r2.  Stops once the voxel volume fraction reaches target_vf.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    mask = np.zeros((n, n, n), np.uint8)
    spheres: list = []
    tries = 0
    while mask.mean() < target_vf:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("RSA did not reach the target volume fraction")
        r = rng.uniform(r_min, r_max)
        c = rng.uniform(0.0, n, size=3)
        ok = True
        for (c2, r2) in spheres:
            d = c - c2
            d -= n * np.round(d / n)
            if float(d @ d) < (r + r2) ** 2:
                ok = False
                break
        if not ok:
            continue
        spheres.append((c, r))
        _stamp_sphere(mask, c, r)
    return mask, spheres


def ellipsoids(n: int, seed: int, a_min: float, a_max: float, target_vf: float) -> np.ndarray:
    """Randomly oriented ellipsoids (overlap allowed) up to a volume fraction.

    Semi-axes U[a_min, a_max] voxels; orientation from a normalised Gaussian
    quaternion (uniform on SO(3)); centres uniform.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    mask = np.zeros((n, n, n), np.uint8)
    while mask.mean() < target_vf:
        a = rng.uniform(a_min, a_max, size=3)
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        R = np.array([
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ])
        c = rng.uniform(0.0, n, size=3)          # (x, y, z) in voxel units
        rr = int(math.ceil(a.max())) + 1
        off = np.arange(-rr, rr + 1)
        base = np.floor(c).astype(int)
        X = (base[0] + off)[None, None, :]
        Y = (base[1] + off)[None, :, None]
        Zc = (base[2] + off)[:, None, None]
        dx = X + 0.5 - c[0]
        dy = Y + 0.5 - c[1]
        dz = Zc + 0.5 - c[2]
        # body-frame coordinates u = R^T d
        u0 = R[0, 0] * dx + R[1, 0] * dy + R[2, 0] * dz
        u1 = R[0, 1] * dx + R[1, 1] * dy + R[2, 1] * dz
        u2 = R[0, 2] * dx + R[1, 2] * dy + R[2, 2] * dz
        inside = (u0 / a[0]) ** 2 + (u1 / a[1]) ** 2 + (u2 / a[2]) ** 2 < 1.0
        sel = np.nonzero(inside)
        mask[(Zc.ravel()[sel[0]]) % n, (Y.ravel()[sel[1]]) % n, (X.ravel()[sel[2]]) % n] = 1
    return mask


def laminate(n: int, layers: int = 8, axis: int = 0) -> np.ndarray:
    """Voxel-aligned layers normal to `axis` (0 = z); odd layers are phase 1."""
    idx = np.arange(n) * layers // n
    lay = (idx % 2).astype(np.uint8)
    shape = [1, 1, 1]
    shape[axis] = n
    return np.broadcast_to(lay.reshape(shape), (n, n, n)).copy()


def random_two_phase(shape, seed: int, vf: float = 0.5) -> np.ndarray:
    """Voxel-wise i.i.d. two-phase map (for tiny brute-force test cells)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.random(shape) < vf).astype(np.uint8)


def _two_phase(phase: np.ndarray, E_m: float, E_i: float, nu: float = 0.3,
               c0_scale: float | None = None, name: str = "") -> Cell:
    lm, mm = lame(E_m, nu)
    li, mi = lame(E_i, nu)
    if c0_scale is None:
        # reference medium at the arithmetic mean of the phase moduli
        # (the classical-scheme rule of Section 5)
        l0, m0 = lame(0.5 * (E_m + E_i), nu)
    else:
        l0, m0 = c0_scale * lm, c0_scale * mm
    return Cell(phase=phase, lam=np.array([lm, li]), mu=np.array([mm, mi]),
                lam0=l0, mu0=m0, name=name)


def cell_sphere32(n: int = 32) -> Cell:
    """Centred sphere R = L/4, matrix E = 1, inclusion E = 10, nu = 0.3,
    C0 at the mean of the phase moduli."""
    return _two_phase(centred_sphere(n, 0.25), 1.0, 10.0, name=f"sphere{n}")


def cell_nearvoid(n: int = 128, seed: int = 0, c0_scale: float = 1.0,
                  r_min: float | None = None, r_max: float | None = None,
                  target_vf: float = 0.20, e_incl: float = 1e-6) -> Cell:
    """Near-void cell: RSA spheres (radius 6-12 voxels at n = 128, scaled with
    n otherwise) of E = e_incl (1e-6 by default) in a matrix E = 1;
    C0 = c0_scale x matrix."""
    if r_min is None:
        r_min = 6.0 * n / 128.0
    if r_max is None:
        r_max = 12.0 * n / 128.0
    mask, _ = rsa_spheres(n, seed, r_min, r_max, target_vf)
    return _two_phase(mask, 1.0, e_incl, c0_scale=c0_scale,
                      name=f"nearvoid{n}_s{seed}_c0x{c0_scale:g}_e{e_incl:g}")


def cell_ellipsoids(n: int = 256, seed: int = 0, contrast: float = 1e4,
                    target_vf: float = 0.30) -> Cell:
    """Random ellipsoids (semi-axes 4-20 voxels at n = 256, scaled otherwise),
    stiffness contrast `contrast` against E = 1, C0 at the mean modulus."""
    s = n / 256.0
    mask = ellipsoids(n, seed, max(1.0, 4.0 * s), max(1.5, 20.0 * s), target_vf)
    return _two_phase(mask, 1.0, contrast, name=f"ellipsoids{n}_s{seed}")


def cell_laminate(n: int = 256, layers: int = 8, contrast: float = 1e3) -> Cell:
    """Laminate of `layers` voxel-aligned layers along z, E = 1 / E = contrast."""
    return _two_phase(laminate(n, layers, 0), 1.0, contrast, name=f"laminate{n}")


def cell_batch_member(s: int) -> Cell:
    """Member s of the batched sweep: grid [32, 48, 64, 96][s mod 4], spheres
    (overlap allowed) of radius U[0.05, 0.10] N voxels (min 2) to a volume
    fraction U(0.1, 0.35), contrast 10^U(-6, 3), C0 at the mean modulus."""
    rng = np.random.Generator(np.random.PCG64(10_000 + s))
    n = BATCH_SIZES[s % 4]
    vf = rng.uniform(0.1, 0.35)
    contrast = 10.0 ** rng.uniform(-6.0, 3.0)
    mask = np.zeros((n, n, n), np.uint8)
    while mask.mean() < vf:
        r = max(2.0, rng.uniform(0.05, 0.10) * n)
        _stamp_sphere(mask, rng.uniform(0.0, n, size=3), r)
    return _two_phase(mask, 1.0, contrast, name=f"batch_s{s}_n{n}")


def cell_fibre2d(n: int = 256, contrast: float = 10.0, radius: float = 1.0 / 32.0,
                 nu: float = 0.25, c0: str = "mean") -> Cell:
    """2D circular fibre (stiffness `contrast`, matrix E = 1, common Poisson
    ratio nu) at the centre of a square cell, one voxel thick (nz = 1: plane
    strain).  radius as a fraction of the cell side; 1/32 gives the 0.3 %
    fibre fraction quoted with the Section 5 geometry.  c0: "mean" (the
    classical rule of Section 5) or "geometric" (the Accelerated-scheme rule
    of Section 5.5)."""
    c = _centres(n)
    y, x = np.meshgrid(c, c, indexing="ij")
    d2 = _wrap(x - 0.5) ** 2 + _wrap(y - 0.5) ** 2
    phase = (d2 < radius * radius).astype(np.uint8)[None]
    lm, mm = lame(1.0, nu)
    lf, mf = lame(contrast, nu)
    if c0 == "geometric":
        l0, m0 = lame(math.sqrt(contrast), nu)
    else:
        l0, m0 = lame(0.5 * (1.0 + contrast), nu)
    return Cell(phase=phase, lam=np.array([lm, lf]), mu=np.array([mm, mf]), lam0=l0, mu0=m0,
                name=f"fibre2d_{n}_K{contrast:g}")


def cell_fno_member(s: int, n: int = 64) -> Cell:
    """Training / test cell s of the learned warm start: the batched-sweep
    recipe (spheres of radius U[0.05, 0.10] n voxels, min 2, to a volume
    fraction U(0.1, 0.35), contrast 10^U(-6, 3), C0 at the mean modulus) on a
    fixed n^3 grid.  Seeds 1000-2999 train, 5000-5019 test."""
    rng = np.random.Generator(np.random.PCG64(20_000 + s))
    vf = rng.uniform(0.1, 0.35)
    contrast = 10.0 ** rng.uniform(-6.0, 3.0)
    mask = np.zeros((n, n, n), np.uint8)
    while mask.mean() < vf:
        r = max(2.0, rng.uniform(0.05, 0.10) * n)
        _stamp_sphere(mask, rng.uniform(0.0, n, size=3), r)
    return _two_phase(mask, 1.0, contrast, name=f"fno_s{s}_n{n}")


def strain_direction(s: int) -> np.ndarray:
    """Macroscopic strain direction s: a Gaussian 6-vector scaled to unit
    Frobenius norm of the tensor (shear components counted twice)."""
    rng = np.random.Generator(np.random.PCG64(30_000 + s))
    e = rng.standard_normal(6)
    w = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])
    return e / math.sqrt(float(np.sum(w * e * e)))


def fno_params(modes: int, layers: int, seed: int = 0, width: int = 16, cin: int = 2,
               cout: int = 36) -> dict:
    """Random parameters of the spectral neural operator: dense maps
    N(0, 1 / fan_in), biases zero, spectral weights with real and imaginary
    parts uniform in [0, 1 / width^2); R{l} is complex [in][out][4 modes^3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M = 4 * modes ** 3
    p = {"P": rng.standard_normal((width, cin)) / math.sqrt(cin), "p": np.zeros(width),
         "Q": rng.standard_normal((cout, width)) / math.sqrt(width), "q": np.zeros(cout)}
    for l in range(layers):
        p[f"A{l}"] = rng.standard_normal((width, width)) / math.sqrt(width)
        p[f"a{l}"] = np.zeros(width)
        p[f"R{l}"] = (rng.random((width, width, M)) + 1j * rng.random((width, width, M))) / (
            width * width)
    return p
