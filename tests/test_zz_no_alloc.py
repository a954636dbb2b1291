"""rpm_apply_gamma_noalloc: the allocation-free Gamma0 application.

Some callers cannot allocate device memory (their host application owns the
device memory, or they may not pay cudaMalloc's synchronisation); this entry
point serves them from fixed file-scope scratch.  The test calls it through
the C ABI twice in a row and compares each result with rpm_apply_gamma, the
context-based entry point, and with the FP64 oracle's map, within the
Gamma0-apply tolerance of the other tests.  The file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest

import microstructure as ms
from oracle import rpm_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_noalloc_matches_context_entry_point():
    import __graft_entry__ as entry
    entry.build()
    from paper_2003_07720_gb300 import rpm
    L = rpm.lib()
    L.rpm_apply_gamma_noalloc.argtypes = [
        ctypes.POINTER(rpm.rpm_grid), ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(rpm.rpm_iso),
        rpm.rpm_iso, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
        ctypes.c_int, ctypes.c_void_p]
    L.rpm_apply_gamma_noalloc.restype = ctypes.c_int

    torch.cuda.set_device(0)
    shapes = [(32, 32, 32), (16, 64, 64)]
    (l1, m1), (l2, m2), (l0, m0) = ms.lame(1, 0.3), ms.lame(20, 0.3), ms.lame(10.5, 0.3)
    cells = [ms.cell_nearvoid(32, 3, e_incl=1e-2),
             ms.Cell(phase=ms.random_two_phase(shapes[1], 4, 0.3), lam=np.array([l1, l2]),
                     mu=np.array([m1, m2]), lam0=l0, mu0=m0)]
    for k, (shape, cell) in enumerate(zip(shapes, cells)):
        nz, ny, nx = shape
        E = np.array([0.2, -0.1, 0.3, 0.05, 0.0, -0.02])
        Ec = (ctypes.c_double * 6)(*E)
        phases = list(zip(cell.lam, cell.mu))
        iso = (rpm.rpm_iso * len(phases))(*[rpm.rpm_iso(float(l), float(m)) for l, m in phases])
        c0 = rpm.rpm_iso(float(cell.lam0), float(cell.mu0))
        grid = rpm.rpm_grid(nx, ny, nz, 1.0, 1.0, 1.0)
        phase_d = torch.from_numpy(np.ascontiguousarray(cell.phase)).cuda()
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):                      # two calls in a row share the scratch
            g = torch.Generator(device="cuda").manual_seed(10 * k + call)
            x = torch.randn((6,) + shape, device="cuda", generator=g)
            for flags in (rpm.RPM_GAMMA_FULL_MAP, rpm.RPM_GAMMA_LINEAR):
                got = torch.full_like(x, float("nan"))
                st = L.rpm_apply_gamma_noalloc(ctypes.byref(grid), phase_d.data_ptr(), len(phases),
                                               iso, c0, x.data_ptr(), Ec, got.data_ptr(), flags,
                                               stream)
                assert st == rpm.RPM_OK
                ref = torch.empty_like(x)
                with rpm.Context(cell) as ctx:
                    ctx.apply_gamma(x, E, ref, flags)
                torch.cuda.synchronize()
                err = (torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref)).item()
                assert err < TOL, (shape, call, flags, err)
                prob = o.Problem.from_cell(cell)
                xh = x.cpu().numpy().astype(np.float64)
                want = (o.apply_F(prob, xh, E) if flags == rpm.RPM_GAMMA_FULL_MAP
                        else o.apply_F(prob, xh, np.zeros(6)))
                gh = got.cpu().numpy().astype(np.float64)
                err_o = np.linalg.norm(gh - want) / np.linalg.norm(want)
                assert err_o < TOL, (shape, call, flags, err_o)
    # sizes beyond the fixed scratch are refused
    big = rpm.rpm_grid(128, 128, 128, 1.0, 1.0, 1.0)
    st = L.rpm_apply_gamma_noalloc(ctypes.byref(big), phase_d.data_ptr(), len(phases), iso, c0,
                                   x.data_ptr(), Ec, got.data_ptr(), 0, None)
    assert st == rpm.RPM_ERR_UNSUPPORTED_GRID
    # planes that are not square are refused (the fixed scratch serves the
    # three-pass kernels only)
    rect = rpm.rpm_grid(64, 32, 32, 1.0, 1.0, 1.0)
    st = L.rpm_apply_gamma_noalloc(ctypes.byref(rect), phase_d.data_ptr(), len(phases), iso, c0,
                                   x.data_ptr(), Ec, got.data_ptr(), 0, None)
    assert st == rpm.RPM_ERR_UNSUPPORTED_GRID
    # a stream under graph capture is refused before any CUDA work is issued
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        x.add_(0.0)
        st_cap = L.rpm_apply_gamma_noalloc(ctypes.byref(grid), phase_d.data_ptr(), len(phases),
                                           iso, c0, x.data_ptr(), Ec, got.data_ptr(), 0,
                                           torch.cuda.current_stream().cuda_stream)
    assert st_cap == rpm.RPM_ERR_INVALID_ARG
