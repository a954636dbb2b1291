"""FP64 reference of the spectral neural operator used as a learned warm start
(test infrastructure only: imported by the tests, never by the library).

Network (width W, L Fourier layers, m modes per axis), on a periodic N^3 grid:

  v0       = P f + p                               (lift, per voxel; f: 2 voxel features)
  v_{l+1}  = act_l( A_l v_l + a_l + K_l v_l )       l = 0 .. L-1, act = GELU except the last
  H        = Q v_L + q                             (36 channels per voxel: a 6 x 6 map)
  out[o]   = sum_j H[o, j] E_j                     (strain for the macroscopic strain E)

The output is linear in E, as the solution of the linear cell problem is:
the network maps the microstructure to a localisation field H(x) and the
strain for any E follows by one contraction.

K_l is the truncated spectral convolution: forward transform of each channel
restricted to the kept modes (kx in [0, m), ky, kz in {0..m-1} U {N-m..N-1}),
per-mode complex channel mixing by R_l [W, W, modes], and the inverse
transform of those modes only:

  V[k]  = sum_x v[x] exp(-i theta_k(x)),   theta_k(x) = 2 pi (kx x + ky y + kz z) / N
  U[k]  = sum_i V_i[k] R[i, o, k]
  u[x]  = (1 / N^3) sum_k c_kx Re(U[k] exp(+i theta_k(x))),   c_0 = 1, c_kx = 2 (kx >= 1)

(the real inverse of a half spectrum that is zero outside the kept modes).
GELU is the tanh form 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
The loss is the mean squared error over all output elements.

Gradients are written out by hand (no autograd) and pinned in the tests by
central finite differences.
"""
from __future__ import annotations

import numpy as np

GELU_C = np.sqrt(2.0 / np.pi)


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(GELU_C * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_C * (1.0 + 3 * 0.044715 * x * x)


def kept_freqs(N: int, m: int):
    """Kept integer frequencies: x in [0, m); y and z in {0..m-1} U {N-m..N-1}."""
    kx = np.arange(m)
    kyz = np.concatenate([np.arange(m), np.arange(N - m, N)])
    return kx, kyz


def dft_mats(N: int, m: int):
    """Forward DFT matrices restricted to the kept modes: Fx [m, N], Fyz [2m, N]."""
    kx, kyz = kept_freqs(N, m)
    n = np.arange(N)
    Fx = np.exp(-2j * np.pi * np.outer(kx, n) / N)
    Fyz = np.exp(-2j * np.pi * np.outer(kyz, n) / N)
    return Fx, Fyz


def trunc_dft(v, m):
    """v [..., N, N, N] (z, y, x) real -> V [..., 2m, 2m, m] complex (kz, ky, kx)."""
    N = v.shape[-1]
    Fx, Fyz = dft_mats(N, m)
    a = np.einsum("...zyx,kx->...zyk", v, Fx)
    a = np.einsum("...zyk,jy->...zjk", a, Fyz)
    return np.einsum("...zjk,iz->...ijk", a, Fyz)


def inv_trunc(U, N, m, weighted=True):
    """U [..., 2m, 2m, m] -> real [..., N, N, N]:
    weighted: (1/N^3) sum_k c_kx Re(U e^{+i theta});  unweighted: sum_k Re(U e^{+i theta})."""
    Fx, Fyz = dft_mats(N, m)
    a = np.einsum("...ijk,iz->...zjk", U, np.conj(Fyz))
    a = np.einsum("...zjk,jy->...zyk", a, np.conj(Fyz))
    if weighted:
        c = np.full(m, 2.0)
        c[0] = 1.0
        a = a * (c / N ** 3)
    return np.einsum("...zyk,kx->...zyx", a, np.conj(Fx)).real


def forward(params, f, E, modes: int, layers: int, keep=False):
    """f [B, 2, N, N, N] voxel features, E [B, 6] -> out [B, 6, N, N, N]
    (and the saved activations)."""
    N = f.shape[-1]
    M2 = 2 * modes
    v = np.einsum("oc,bc...->bo...", params["P"], f) + params["p"][None, :, None, None, None]
    saved = {"x": f, "v": [v], "z": [], "V": []}
    for l in range(layers):
        V = trunc_dft(v, modes).reshape(v.shape[0], v.shape[1], -1)          # [B, W, M]
        U = np.einsum("bim,iom->bom", V, params[f"R{l}"]).reshape(v.shape[0], -1, M2, M2, modes)
        u = inv_trunc(U, N, modes)
        z = (np.einsum("oc,bc...->bo...", params[f"A{l}"], v)
             + params[f"a{l}"][None, :, None, None, None] + u)
        v = gelu(z) if l < layers - 1 else z
        saved["z"].append(z)
        saved["V"].append(V)
        saved["v"].append(v)
    H = np.einsum("oc,bc...->bo...", params["Q"], v) + params["q"][None, :, None, None, None]
    H = H.reshape((H.shape[0], 6, 6) + H.shape[2:])
    out = np.einsum("boj...,bj->bo...", H, np.asarray(E, float))
    return (out, saved) if keep else out


def loss(params, f, E, target, modes, layers):
    out = forward(params, f, E, modes, layers)
    return float(np.mean((out - target) ** 2))


def _outer_sum(a, b):
    """sum over samples and voxels of a[o] b[c]: [B, O, ...] x [B, C, ...] -> [O, C]."""
    B = a.shape[0]
    return np.einsum("bon,bcn->oc", a.reshape(B, a.shape[1], -1), b.reshape(B, b.shape[1], -1))


def backward(params, f, E, target, modes: int, layers: int):
    """Loss and gradients of every parameter (complex R: dL/dRe + i dL/dIm)."""
    out, s = forward(params, f, E, modes, layers, keep=True)
    N = f.shape[-1]
    B = f.shape[0]
    M2 = 2 * modes
    nel = out.size
    g = {}
    d_out = 2.0 * (out - target) / nel
    vL = s["v"][-1]
    dH = np.einsum("bo...,bj->boj...", d_out, np.asarray(E, float))
    dH = dH.reshape((B, 36) + dH.shape[3:])
    g["Q"] = _outer_sum(dH, vL)
    g["q"] = dH.sum(axis=(0, 2, 3, 4))
    dv = np.einsum("oc,bo...->bc...", params["Q"], dH)
    for l in reversed(range(layers)):
        z = s["z"][l]
        v = s["v"][l]
        dz = dv * gelu_grad(z) if l < layers - 1 else dv
        g[f"A{l}"] = _outer_sum(dz, v)
        g[f"a{l}"] = dz.sum(axis=(0, 2, 3, 4))
        dv_prev = np.einsum("oc,bo...->bc...", params[f"A{l}"], dz)
        # spectral branch: u = inv_trunc(U) (weighted) -> dU = (c_kx / N^3) trunc_dft(dz)
        c = np.full(modes, 2.0)
        c[0] = 1.0
        dU = (trunc_dft(dz, modes) * (c / N ** 3)).reshape(B, -1, M2 * M2 * modes)
        V = s["V"][l]
        g[f"R{l}"] = np.einsum("bom,bim->iom", dU, np.conj(V))
        dV = np.einsum("bom,iom->bim", dU, np.conj(params[f"R{l}"]))
        dv_prev = dv_prev + inv_trunc(dV.reshape(B, -1, M2, M2, modes), N, modes, weighted=False)
        dv = dv_prev
    g["P"] = _outer_sum(dv, f)
    g["p"] = dv.sum(axis=(0, 2, 3, 4))
    return float(np.mean((out - target) ** 2)), g


def adam_step(p, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One step of Adam (Kingma & Ba, 2015) with decoupled weight decay
    (Loshchilov & Hutter, 2019), on flat arrays; t is the 1-based step."""
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** t)
    vh = m2 / (1 - b2 ** t)
    return p - lr * (mh / (np.sqrt(vh) + eps) + wd * p), m1, m2


def features(phase, lam, mu):
    """Voxel inputs of the network: log10(Young / Young of phase 0) and the
    Poisson ratio, from isotropic Lame moduli per phase."""
    lam = np.asarray(lam, float)
    mu = np.asarray(mu, float)
    young = mu * (3 * lam + 2 * mu) / (lam + mu)
    nu = lam / (2 * (lam + mu))
    return np.stack([np.log10(young / young[0])[phase], nu[phase]])
