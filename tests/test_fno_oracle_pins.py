"""Pins of the FP64 spectral-neural-operator reference (oracle/fno_oracle.py)
against library transforms, closed forms and finite differences."""
import numpy as np
import pytest

from microstructure import fno_params, lame
from oracle import fno_oracle as fo

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


def test_trunc_dft_is_fftn_restricted():
    # the truncated transform equals numpy's full 3D FFT at the kept modes
    N, m = 12, 3
    v = _rng(1).standard_normal((2, N, N, N))
    V = fo.trunc_dft(v, m)
    full = np.fft.fftn(v, axes=(1, 2, 3))
    kx, kyz = fo.kept_freqs(N, m)
    ref = full[:, kyz][:, :, kyz][:, :, :, kx]
    assert np.allclose(V, ref, atol=1e-10)


def test_inverse_is_irfftn_of_padded_half_spectrum():
    N, m = 12, 3
    U = _rng(2).standard_normal((2, 2 * m, 2 * m, m)) + 1j * _rng(3).standard_normal(
        (2, 2 * m, 2 * m, m))
    half = np.zeros((2, N, N, N // 2 + 1), complex)
    kx, kyz = fo.kept_freqs(N, m)
    for a, kz in enumerate(kyz):
        for b, ky in enumerate(kyz):
            half[:, kz, ky, :m] = U[:, a, b, :]
    ref = np.fft.irfftn(half, s=(N, N, N), axes=(1, 2, 3))
    assert np.allclose(fo.inv_trunc(U, N, m), ref, atol=1e-12)


def test_identity_mixing_reproduces_kept_modes_and_filters_the_rest():
    # with R = identity per mode, the spectral branch returns a band-limited
    # cosine whose +-k pair is kept, and removes a mode with kx >= m
    N, m, W = 16, 4, 2
    z, y, x = np.meshgrid(*(np.arange(N),) * 3, indexing="ij")
    kept = np.cos(2 * np.pi * (2 * x + 1 * y - 3 * z) / N)
    cut = np.cos(2 * np.pi * (5 * x) / N)
    v = np.stack([kept, kept + cut])[None]
    V = fo.trunc_dft(v, m).reshape(1, W, -1)
    R = np.zeros((W, W, V.shape[-1]), complex)
    R[0, 0] = R[1, 1] = 1.0
    U = np.einsum("bim,iom->bom", V, R).reshape(1, W, 2 * m, 2 * m, m)
    u = fo.inv_trunc(U, N, m)
    assert np.allclose(u[0, 0], kept, atol=1e-12)
    assert np.allclose(u[0, 1], kept, atol=1e-12)


def test_zero_spectral_weights_reduce_to_pointwise_network():
    N, m, L = 8, 2, 2
    p = fno_params(m, L, seed=4, width=5)
    for l in range(L):
        p[f"R{l}"][:] = 0
    x = _rng(5).standard_normal((1, 2, N, N, N))
    E = _rng(15).standard_normal((1, 6))
    out = fo.forward(p, x, E, m, L)
    h = np.einsum("oc,c...->o...", p["P"], x[0]) + p["p"][:, None, None, None]
    h = np.einsum("oc,c...->o...", p["A0"], h) + p["a0"][:, None, None, None]
    h = 0.5 * h * (1 + np.tanh(np.sqrt(2 / np.pi) * (h + 0.044715 * h ** 3)))
    h = np.einsum("oc,c...->o...", p["A1"], h) + p["a1"][:, None, None, None]
    H = np.einsum("oc,c...->o...", p["Q"], h) + p["q"][:, None, None, None]
    ref = sum(E[0, j] * H[j::6] for j in range(6))       # H channel 6 o + j, out_o = H_oj E_j
    assert np.allclose(out[0], ref, atol=1e-12)


def test_output_is_linear_in_the_macroscopic_strain():
    N, m, L = 8, 2, 2
    p = fno_params(m, L, seed=16, width=4)
    f = _rng(17).standard_normal((1, 2, N, N, N))
    E1, E2 = _rng(18).standard_normal((1, 6)), _rng(19).standard_normal((1, 6))
    a = fo.forward(p, f, 2.0 * E1 - 3.0 * E2, m, L)
    b = 2.0 * fo.forward(p, f, E1, m, L) - 3.0 * fo.forward(p, f, E2, m, L)
    assert np.allclose(a, b, atol=1e-12)


def test_gelu_derivative_matches_difference_quotient():
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (fo.gelu(x + h) - fo.gelu(x - h)) / (2 * h)
    assert np.allclose(fo.gelu_grad(x), fd, atol=1e-8)
    # closed values: gelu(0) = 0, gelu'(0) = 1/2, gelu(x) -> x for large x
    assert fo.gelu(0.0) == 0.0 and fo.gelu_grad(0.0) == 0.5
    assert abs(fo.gelu(10.0) - 10.0) < 1e-12


@pytest.mark.parametrize("name", ["P", "p", "Q", "q", "A0", "a0", "A1", "a1", "R0", "R1"])
def test_gradient_matches_central_differences(name):
    N, m, L, B = 8, 2, 2, 2
    p = fno_params(m, L, seed=6, width=3)
    for l in range(L):   # larger spectral weights so the branch matters
        p[f"R{l}"] *= 20.0
        p[f"a{l}"] = 0.1 * _rng(7 + l).standard_normal(3)
    x = _rng(9).standard_normal((B, 2, N, N, N))
    E = _rng(20).standard_normal((B, 6))
    t = _rng(10).standard_normal((B, 6, N, N, N))
    _, g = fo.backward(p, x, E, t, m, L)
    a = p[name]
    rng = _rng(11)
    idx = [tuple(rng.integers(0, s) for s in a.shape) for _ in range(4)]
    h = 1e-5
    for ix in idx:
        parts = [1.0, 1j] if np.iscomplexobj(a) else [1.0]
        for unit in parts:
            old = a[ix]
            a[ix] = old + h * unit
            lp = fo.loss(p, x, E, t, m, L)
            a[ix] = old - h * unit
            lm = fo.loss(p, x, E, t, m, L)
            a[ix] = old
            fd = (lp - lm) / (2 * h)
            got = g[name][ix].real if unit == 1.0 else g[name][ix].imag
            assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, ix, unit, got, fd)


def test_input_gradient_matches_central_differences():
    # backward's dL/dv chain checked end to end through the loss w.r.t. a
    # voxel input (the first-layer input gradient is g["P"]'s factor)
    N, m, L = 8, 2, 2
    p = fno_params(m, L, seed=12, width=3)
    x = _rng(13).standard_normal((1, 2, N, N, N))
    E = _rng(21).standard_normal((1, 6))
    t = _rng(14).standard_normal((1, 6, N, N, N))
    _, g = fo.backward(p, x, E, t, m, L)
    # gP[o][c] = sum_vox dv0[o] x[c]: perturbing x scaled by (1 + s) along
    # channel c changes the loss by s * sum_o P[o][c] gP-contributions; use
    # the exact identity d/ds L(P with column c scaled) = sum_o gP[o][c] P[o][c]
    c = 1
    h = 1e-6
    pp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    pp["P"][:, c] *= 1 + h
    lp = fo.loss(pp, x, E, t, m, L)
    pp["P"][:, c] = p["P"][:, c] * (1 - h)
    lm = fo.loss(pp, x, E, t, m, L)
    fd = (lp - lm) / (2 * h)
    assert abs(fd - np.sum(g["P"][:, c] * p["P"][:, c])) < 1e-7 * max(1, abs(fd))


def test_adam_first_step_is_sign_step():
    # at t = 1 bias correction makes m/sqrt(v) = g/|g|: a step of lr * sign(g)
    g = np.array([0.3, -2.0, 1e-3])
    p, _, _ = fo.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1, eps=0.0)
    assert np.allclose(p, -0.1 * np.sign(g))


def test_features_closed_form():
    lm, mm = lame(1.0, 0.3)
    li, mi = lame(100.0, 0.25)
    f = fo.features(np.array([[[0, 1]]]), [lm, li], [mm, mi])
    assert np.allclose(f[0].ravel(), [0.0, 2.0]) and np.allclose(f[1].ravel(), [0.3, 0.25])


def test_adam_constant_gradient_steps_by_lr_every_step():
    """With a constant gradient the bias-corrected moments are exactly g and
    g^2 at every step t (m_t = (1 - b1^t) g, v_t = (1 - b2^t) g^2), so each
    step moves by lr * sign(g)."""
    g = np.array([0.7, -3.0, 2e-4])
    p, m1, m2 = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 6):
        p, m1, m2 = fo.adam_step(p, g, m1, m2, t, lr=0.01, eps=0.0)
        assert np.allclose(p, -0.01 * t * np.sign(g), rtol=1e-12, atol=0)
        assert np.allclose(m1, (1 - 0.9 ** t) * g, rtol=1e-12)
        assert np.allclose(m2, (1 - 0.999 ** t) * g * g, rtol=1e-12)


def test_adam_weight_decay_is_decoupled():
    """With zero gradient the moments stay zero and decoupled weight decay
    alone shrinks the parameters geometrically: p_t = (1 - lr wd)^t p_0."""
    p0 = np.array([1.5, -0.2, 4.0])
    p, m1, m2 = p0.copy(), np.zeros(3), np.zeros(3)
    for t in range(1, 4):
        p, m1, m2 = fo.adam_step(p, np.zeros(3), m1, m2, t, lr=0.05, wd=0.1)
    assert np.allclose(p, (1 - 0.05 * 0.1) ** 3 * p0, rtol=1e-13)
