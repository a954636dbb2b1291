"""Parity of the CUDA Gamma0 application (pass A/B/C kernels) with the FP64
oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import microstructure as ms
from oracle import rpm_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5      # single Gamma0-apply, relative L2 (float32 fields)


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


def _cell(shape, seed, contrast=10.0):
    phase = ms.random_two_phase(shape, seed, 0.35)
    l0, m0 = ms.lame(1.0, 0.3)
    l1, m1 = ms.lame(contrast, 0.3)
    l_0, m_0 = ms.lame(0.5 * (1 + contrast), 0.3)
    return ms.Cell(phase=phase, lam=np.array([l0, l1]), mu=np.array([m0, m1]), lam0=l_0, mu0=m_0)


def _run(cell, mode, nyq=0, seed=1, E=None):
    from paper_2003_07720_gb300 import rpm
    E = np.array([0.3, -0.2, 0.1, 0.05, -0.04, 0.07]) if E is None else E
    x = _rng(seed).standard_normal((6,) + cell.shape).astype(np.float32)
    prob = o.Problem.from_cell(cell, nyquist=nyq)
    xd = torch.from_numpy(x).cuda()
    out = torch.full_like(xd, float("nan"))
    with rpm.Context(cell, rpm.rpm_default_options(nyquist=nyq)) as ctx:
        ctx.apply_gamma(xd, E, out, mode)
        torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    xx = x.astype(np.float64)
    if mode == 0:
        ref = o.apply_F(prob, xx, E)
    elif mode == 1:
        ref = o.apply_F_linear(prob, xx)
    else:
        ref = o.apply_gamma_raw(prob, xx)
    return got, ref


@pytest.mark.parametrize("shape", [(4, 4, 4), (8, 8, 8), (16, 16, 16), (32, 32, 32),
                                   (16, 8, 8), (2, 16, 16), (1, 32, 32), (64, 16, 16),
                                   (8, 64, 64), (4, 128, 128), (256, 8, 8),
                                   # five-pass path: 256^2 planes and nx != ny
                                   (4, 256, 256), (2, 256, 16), (16, 32, 64), (8, 16, 128),
                                   (1, 8, 256), (32, 64, 32),
                                   # radix-3 lengths (2^a 3^b)
                                   (48, 48, 48), (96, 96, 96), (12, 24, 24), (6, 12, 12),
                                   (3, 48, 48), (24, 6, 6), (16, 96, 48), (8, 96, 256),
                                   # fused plane and pencil kernels (square planes 48-128,
                                   # nz 32, 48, 96, 128), alone and with the original ones
                                   (128, 64, 64), (64, 96, 96), (32, 128, 128), (48, 64, 64),
                                   (128, 48, 48), (96, 32, 64), (64, 128, 128), (6, 96, 96),
                                   (256, 48, 48), (256, 16, 32)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_apply_gamma_matches_oracle(shape, mode):
    got, ref = _run(_cell(shape, 3), mode)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert np.all(np.isfinite(got))
    assert err < TOL, err


def test_apply_gamma_full_size_128():
    """The 128^3 near-void cell of the benchmark, full map, all elements."""
    cell = ms.cell_nearvoid(128, 0)
    E = ms.unit_strain(0)
    got, ref = _run(cell, 0, seed=2, E=E)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < TOL, err


def test_gamma_projector_identity_on_gpu():
    """Gamma0 C0 Gamma0 = Gamma0 evaluated entirely by the CUDA path."""
    from paper_2003_07720_gb300 import rpm
    cell = _cell((16, 16, 16), 7)
    tau = torch.from_numpy(_rng(3).standard_normal((6, 16, 16, 16)).astype(np.float32)).cuda()
    g1 = torch.empty_like(tau)
    g2 = torch.empty_like(tau)
    with rpm.Context(cell) as ctx:
        ctx.apply_gamma(tau, None, g1, rpm.RPM_GAMMA_RAW_TAU)
        # C0 : g1 on the device with torch elementwise ops (test-side only)
        l0, m0 = cell.lam0, cell.mu0
        tr = g1[0] + g1[1] + g1[2]
        c0g = 2 * m0 * g1
        c0g[:3] += l0 * tr
        ctx.apply_gamma(c0g.contiguous(), None, g2, rpm.RPM_GAMMA_RAW_TAU)
        torch.cuda.synchronize()
    err = (torch.linalg.vector_norm(g2 + g1) / torch.linalg.vector_norm(g1)).item()
    assert err < 1e-5


def test_apply_gamma_full_size_256_ellipsoids():
    """The 256^3 high-contrast cell (random ellipsoids, 30 % volume fraction,
    contrast 1e4, C0 = arithmetic mean): one full map F on a random field,
    every element against the FP64 oracle's map, in the launch configuration
    the solver uses at this size."""
    from paper_2003_07720_gb300 import rpm
    cell = ms.cell_ellipsoids(256, 0, contrast=1e4)
    E = np.array([0.3, -0.2, 0.1, 0.05, -0.04, 0.07])
    x = _rng(11).standard_normal((6,) + cell.shape).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    out = torch.full_like(xd, float("nan"))
    with rpm.Context(cell, rpm.rpm_default_options(p_max=0)) as ctx:
        ctx.apply_gamma(xd, E, out, rpm.RPM_GAMMA_FULL_MAP)
        torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    del xd, out
    ref = o.apply_F(o.Problem.from_cell(cell), x.astype(np.float64), E)
    assert np.all(np.isfinite(got))
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < TOL, err
    # element by element: no voxel off by more than 1e-5 of the field's scale
    assert np.max(np.abs(got - ref)) < TOL * np.max(np.abs(ref)), np.max(np.abs(got - ref))
