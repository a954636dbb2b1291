"""The seeded input generators (microstructure/) follow the recipes they state:
membership by strict periodic distance, non-overlapping random sequential
addition, volume-fraction stopping rules, load-case conventions and the
reference-medium rules.  CPU only; no step of the solution method is involved."""
import itertools
import math

import numpy as np

import microstructure as ms


def test_lame_round_trip():
    for E, nu in [(1.0, 0.3), (1e-6, 0.3), (1e3, 0.25), (7.5, 0.1)]:
        lam, mu = ms.lame(E, nu)
        assert math.isclose(mu * (3 * lam + 2 * mu) / (lam + mu), E, rel_tol=1e-13)
        assert math.isclose(lam / (2 * (lam + mu)), nu, rel_tol=1e-13)


def test_unit_strains_use_engineering_shear():
    """Unit load j: eps_jj = 1 for j < 3; gamma = 1 (eps_ij = eps_ji = 1/2)
    for the shears, so the six loads have Frobenius norms 1 and 1/sqrt(2)."""
    w = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])
    for j in range(6):
        E = ms.unit_strain(j)
        assert np.count_nonzero(E) == 1 and E[j] == (1.0 if j < 3 else 0.5)
        assert math.isclose(float(np.sum(w * E * E)), 1.0 if j < 3 else 0.5)


def test_strain_direction_is_unit_frobenius():
    w = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])
    for s in range(20):
        e = ms.strain_direction(s)
        assert math.isclose(float(np.sum(w * e * e)), 1.0, rel_tol=1e-12)
    assert not np.allclose(ms.strain_direction(0), ms.strain_direction(1))


def test_centred_sphere_has_the_cube_symmetry_and_no_boundary_voxel():
    n = 32
    m = ms.centred_sphere(n, 0.25)
    for perm in itertools.permutations(range(3)):
        assert np.array_equal(np.transpose(m, perm), m)
    for ax in range(3):
        assert np.array_equal(np.flip(m, ax), m)
    c = (np.arange(n) + 0.5) / n - 0.5
    d2 = c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2
    assert np.min(np.abs(d2 - 0.0625)) > 1e-6          # strict "< R" is unambiguous
    assert abs(m.mean() - 4 / 3 * math.pi * 0.25 ** 3) < 0.01


def _brute_union(n, spheres):
    """Voxels whose centre lies strictly within r of a sphere centre given as
    (x, y, z) in voxel units (minimum-image distances), over the whole grid,
    as a map indexed [z, y, x]."""
    c = np.arange(n) + 0.5
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    mask = np.zeros((n, n, n), bool)
    for (cen, r) in spheres:
        dx = x - cen[0]
        dy = y - cen[1]
        dz = z - cen[2]
        dx -= n * np.round(dx / n)
        dy -= n * np.round(dy / n)
        dz -= n * np.round(dz / n)
        mask |= dx * dx + dy * dy + dz * dz < r * r
    return mask


def test_rsa_spheres_are_disjoint_and_stamped_exactly():
    n, r_min, r_max, vf = 32, 2.0, 4.0, 0.2
    mask, spheres = ms.rsa_spheres(n, 3, r_min, r_max, vf)
    assert all(r_min <= r <= r_max for _, r in spheres)
    for (c1, r1), (c2, r2) in itertools.combinations(spheres, 2):
        d = c1 - c2
        d -= n * np.round(d / n)
        assert math.sqrt(float(d @ d)) >= r1 + r2
    # the map is the union of the listed spheres (centres stored as (z, y, x)
    # in voxel units)
    union = _brute_union(n, [((c[2], c[1], c[0]), r) for c, r in spheres])
    assert np.array_equal(mask.astype(bool), union)
    # stops at the first sphere that reaches the target
    assert vf <= mask.mean() < vf + 4 / 3 * math.pi * r_max ** 3 / n ** 3
    m2, _ = ms.rsa_spheres(n, 3, r_min, r_max, vf)
    m3, _ = ms.rsa_spheres(n, 4, r_min, r_max, vf)
    assert np.array_equal(mask, m2) and not np.array_equal(mask, m3)


def test_nearvoid_cell_recipe():
    cell = ms.cell_nearvoid(32, 0, c0_scale=0.5, e_incl=1e-3)
    assert cell.shape == (32, 32, 32)
    assert 0.20 <= cell.volume_fraction(1) < 0.25
    lm, mm = ms.lame(1.0, 0.3)
    li, mi = ms.lame(1e-3, 0.3)
    assert np.allclose(cell.lam, [lm, li]) and np.allclose(cell.mu, [mm, mi])
    assert math.isclose(cell.lam0, 0.5 * lm) and math.isclose(cell.mu0, 0.5 * mm)


def test_ellipsoids_reach_the_volume_fraction_deterministically():
    a = ms.ellipsoids(32, 1, 1.5, 4.0, 0.3)
    assert 0.3 <= a.mean() < 0.3 + 4 / 3 * math.pi * 4.0 ** 3 / 32 ** 3
    assert np.array_equal(a, ms.ellipsoids(32, 1, 1.5, 4.0, 0.3))


def test_ellipsoid_with_equal_axes_is_a_sphere():
    """With a_min = a_max every ellipsoid is a sphere whatever its rotation:
    the stamped map equals the strict-distance union of those spheres."""
    n, r = 24, 3.0
    m = ms.ellipsoids(n, 5, r, r, 0.02)
    rng = np.random.Generator(np.random.PCG64(5))
    spheres = []
    while len(spheres) == 0 or _brute_union(n, spheres).mean() < 0.02:
        rng.uniform(r, r, size=3)          # semi-axes
        rng.standard_normal(4)             # orientation
        c = rng.uniform(0.0, n, size=3)    # (x, y, z)
        spheres.append(((c[0], c[1], c[2]), r))
    union = _brute_union(n, spheres)       # (x, y, z) centres, [z, y, x] map
    assert np.array_equal(m.astype(bool), union)


def test_laminate_layers():
    lam = ms.laminate(32, 8, 0)
    assert np.all(lam == lam[:, :1, :1])            # constant in each z-slab
    prof = lam[:, 0, 0]
    assert np.array_equal(prof, np.repeat(np.arange(8) % 2, 4).astype(np.uint8))
    assert lam.mean() == 0.5


def test_batch_members_cycle_grid_sizes_and_ranges():
    for s in range(8):
        c = ms.cell_batch_member(s)
        n = ms.BATCH_SIZES[s % 4]
        assert c.shape == (n, n, n)
        contrast = (c.mu[1] / c.mu[0])
        assert 1e-6 <= contrast <= 1e3
        assert 0.1 <= c.volume_fraction(1) < 0.35 + 4 / 3 * math.pi * 0.1 ** 3 + 1e-9
        # C0 at the arithmetic mean of the phase moduli (common nu)
        assert math.isclose(c.mu0, 0.5 * (c.mu[0] + c.mu[1]), rel_tol=1e-12)
        assert math.isclose(c.lam0, 0.5 * (c.lam[0] + c.lam[1]), rel_tol=1e-12)


def test_fibre2d_fraction_and_reference_media():
    c = ms.cell_fibre2d(256, contrast=100.0)
    assert c.shape == (1, 256, 256)
    assert abs(c.volume_fraction(1) - math.pi / 32 ** 2) < 2e-4     # ~0.3 %
    g = ms.cell_fibre2d(64, contrast=100.0, c0="geometric")
    assert math.isclose(g.mu0, ms.lame(10.0, 0.25)[1], rel_tol=1e-12)
    assert math.isclose(c.mu0, ms.lame(50.5, 0.25)[1], rel_tol=1e-12)
