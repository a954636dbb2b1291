"""ctypes binding of include/rpm_fno.h, the learned warm start (argument
marshalling and parameter-layout conversion only; every step of the network
runs in the CUDA library).

Parameters travel as one float32 vector in the library's layout.  The
dictionary form used here (`P`, `p`, `Q`, `q`, `A{l}`, `a{l}`, `R{l}`) keeps
R_l as a complex array [in][out][kz_i][ky_i][kx] (kz_i, ky_i in [0, 2m), kx in
[0, m)); pack_params / unpack_params convert between the two.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import rpm

WIDTH = 16
CIN = 2          # voxel features
COUT = 36        # localisation channels H[o][j] (channel 6 o + j)
HEADER = 768


RPM_FNO_FP32 = 0
RPM_FNO_BF16 = 1
PRECISIONS = {"fp32": RPM_FNO_FP32, "bf16": RPM_FNO_BF16}


class rpm_fno_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("modes", ctypes.c_int), ("layers", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("precision", ctypes.c_int)]


class rpm_fno_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("weight_decay", ctypes.c_float)]


EXPORTS = ("rpm_fno_param_count", "rpm_fno_create", "rpm_fno_set_params", "rpm_fno_get_params",
           "rpm_fno_get_grads", "rpm_fno_forward", "rpm_fno_loss_grad", "rpm_fno_adam_step",
           "rpm_fno_train_step", "rpm_fno_features", "rpm_fno_warm_start", "rpm_fno_solve",
           "rpm_fno_device_bytes", "rpm_fno_last_error", "rpm_fno_destroy")

_done = False


def lib():
    global _done
    L = rpm.lib()
    if _done:
        return L
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    i = ctypes.c_int
    L.rpm_fno_param_count.argtypes = [i, i]
    L.rpm_fno_param_count.restype = ctypes.c_size_t
    L.rpm_fno_create.argtypes = [P(rpm_fno_config), vp, P(vp)]
    L.rpm_fno_create.restype = i
    for n in ("rpm_fno_set_params", "rpm_fno_get_params", "rpm_fno_get_grads"):
        getattr(L, n).argtypes = [vp, vp]
        getattr(L, n).restype = i
    L.rpm_fno_forward.argtypes = [vp, i, vp, vp, vp]
    L.rpm_fno_forward.restype = i
    L.rpm_fno_loss_grad.argtypes = [vp, i, vp, vp, vp, P(ctypes.c_double)]
    L.rpm_fno_loss_grad.restype = i
    L.rpm_fno_adam_step.argtypes = [vp, P(rpm_fno_adam)]
    L.rpm_fno_adam_step.restype = i
    L.rpm_fno_train_step.argtypes = [vp, i, vp, vp, vp, P(rpm_fno_adam), P(ctypes.c_double)]
    L.rpm_fno_train_step.restype = i
    L.rpm_fno_features.argtypes = [vp, ctypes.c_longlong, i, P(rpm.rpm_iso), vp, vp]
    L.rpm_fno_features.restype = i
    L.rpm_fno_warm_start.argtypes = [vp, vp, P(ctypes.c_double), vp]
    L.rpm_fno_warm_start.restype = i
    L.rpm_fno_solve.argtypes = [vp, vp, P(ctypes.c_double), vp, vp, i, P(rpm.rpm_solve_info),
                                P(ctypes.c_int)]
    L.rpm_fno_solve.restype = i
    L.rpm_fno_device_bytes.argtypes = [vp]
    L.rpm_fno_device_bytes.restype = ctypes.c_size_t
    L.rpm_fno_last_error.argtypes = [vp]
    L.rpm_fno_last_error.restype = ctypes.c_char_p
    L.rpm_fno_destroy.argtypes = [vp]
    L.rpm_fno_destroy.restype = None
    _done = True
    return L


def param_count(modes: int, layers: int) -> int:
    return int(lib().rpm_fno_param_count(modes, layers))


def _layer_off(modes: int, l: int) -> int:
    r = 2 * (2 * modes * modes) * (2 * modes) * WIDTH * WIDTH
    return HEADER + l * (WIDTH * WIDTH + WIDTH + r)


def pack_params(p: dict, modes: int, layers: int) -> np.ndarray:
    """Dictionary form -> the library's float32 vector."""
    m, W = modes, WIDTH
    out = np.zeros(param_count(m, layers), np.float32)
    out[0:W * CIN] = np.asarray(p["P"]).ravel()
    out[W * CIN:W * CIN + W] = p["p"]
    o = W * CIN + W
    out[o:o + COUT * W] = np.asarray(p["Q"]).ravel()
    out[o + COUT * W:o + COUT * W + COUT] = p["q"]
    for l in range(layers):
        b = _layer_off(m, l)
        out[b:b + W * W] = np.asarray(p[f"A{l}"]).ravel()
        out[b + W * W:b + W * W + W] = p[f"a{l}"]
        R = np.asarray(p[f"R{l}"]).reshape(W, W, 2 * m, 2 * m, m)      # i, o, kz, ky, kx
        R = np.transpose(R, (3, 4, 2, 0, 1))                            # ky, kx, kz, i, o
        rr = np.stack([R.real, R.imag], axis=-1).astype(np.float32).ravel()
        out[b + W * W + W:b + W * W + W + rr.size] = rr
    return out


def unpack_params(v: np.ndarray, modes: int, layers: int) -> dict:
    """The library's vector -> dictionary form (R complex [i][o][kz*ky*kx])."""
    m, W = modes, WIDTH
    v = np.asarray(v, np.float64)
    o = W * CIN + W
    p = {"P": v[0:W * CIN].reshape(W, CIN), "p": v[W * CIN:o].copy(),
         "Q": v[o:o + COUT * W].reshape(COUT, W), "q": v[o + COUT * W:o + COUT * W + COUT].copy()}
    nr = 2 * (2 * m * m) * (2 * m) * W * W
    for l in range(layers):
        b = _layer_off(m, l)
        p[f"A{l}"] = v[b:b + W * W].reshape(W, W)
        p[f"a{l}"] = v[b + W * W:b + W * W + W].copy()
        rr = v[b + W * W + W:b + W * W + W + nr].reshape(2 * m, m, 2 * m, W, W, 2)
        R = rr[..., 0] + 1j * rr[..., 1]                                 # ky, kx, kz, i, o
        p[f"R{l}"] = np.transpose(R, (3, 4, 2, 0, 1)).reshape(W, W, -1)
    return p


class FnoError(RuntimeError):
    pass


def _ck(h, st):
    if st != rpm.RPM_OK:
        msg = lib().rpm_fno_last_error(h).decode() if h else ""
        raise FnoError(f"{lib().rpm_status_string(st).decode()}: {msg}")


class Fno:
    """Owning wrapper of an rpm_fno handle on grid N^3."""

    def __init__(self, n: int, modes: int = 12, layers: int = 4, max_batch: int = 1,
                 stream=None, precision: str = "bf16"):
        """precision "bf16": the truncated DFT stages as BF16 tensor-core products
        with float32 accumulation (grids with n % 16 == 0); "fp32": float32
        throughout."""
        self.n, self.modes, self.layers, self.max_batch = n, modes, layers, max_batch
        self.precision = precision
        h = ctypes.c_void_p()
        cfg = rpm_fno_config(n, modes, layers, max_batch, PRECISIONS[precision])
        st = lib().rpm_fno_create(ctypes.byref(cfg), rpm._stream_ptr(stream), ctypes.byref(h))
        if st != rpm.RPM_OK:
            raise FnoError(f"rpm_fno_create: {lib().rpm_status_string(st).decode()}")
        self.h = h.value
        self.nparam = param_count(modes, layers)

    # parameters -----------------------------------------------------------
    def set_params(self, p):
        v = p if isinstance(p, np.ndarray) else pack_params(p, self.modes, self.layers)
        v = np.ascontiguousarray(v, np.float32)
        assert v.size == self.nparam
        _ck(self.h, lib().rpm_fno_set_params(self.h, v.ctypes.data))

    def get_params(self) -> np.ndarray:
        v = np.empty(self.nparam, np.float32)
        _ck(self.h, lib().rpm_fno_get_params(self.h, v.ctypes.data))
        return v

    def get_grads(self) -> np.ndarray:
        v = np.empty(self.nparam, np.float32)
        _ck(self.h, lib().rpm_fno_get_grads(self.h, v.ctypes.data))
        return v

    # compute --------------------------------------------------------------
    @staticmethod
    def _e(E, B):
        e = np.ascontiguousarray(np.asarray(E, np.float32).reshape(B, 6))
        return e

    def forward(self, feat, E_dir, out):
        B = feat.shape[0]
        e = self._e(E_dir, B)
        _ck(self.h, lib().rpm_fno_forward(self.h, B, rpm._ptr(feat), e.ctypes.data,
                                          rpm._ptr(out)))

    def loss_grad(self, feat, E_dir, target) -> float:
        B = feat.shape[0]
        e = self._e(E_dir, B)
        loss = ctypes.c_double()
        _ck(self.h, lib().rpm_fno_loss_grad(self.h, B, rpm._ptr(feat), e.ctypes.data,
                                            rpm._ptr(target), ctypes.byref(loss)))
        return loss.value

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        o = rpm_fno_adam(lr, beta1, beta2, eps, weight_decay)
        _ck(self.h, lib().rpm_fno_adam_step(self.h, ctypes.byref(o)))

    def train_step(self, feat, E_dir, target, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   weight_decay=0.0, want_loss=True):
        B = feat.shape[0]
        e = self._e(E_dir, B)
        o = rpm_fno_adam(lr, beta1, beta2, eps, weight_decay)
        loss = ctypes.c_double()
        _ck(self.h, lib().rpm_fno_train_step(self.h, B, rpm._ptr(feat), e.ctypes.data,
                                             rpm._ptr(target), ctypes.byref(o),
                                             ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def warm_start(self, ctx, E, eps0):
        """eps0 <- projected network guess for the context's cell and strain E."""
        handle = ctx.handle if hasattr(ctx, "handle") else ctx
        _ck(self.h, lib().rpm_fno_warm_start(self.h, handle, rpm._E(E), rpm._ptr(eps0)))

    def solve(self, ctx, E, eps_out=None, sig_out=None, out_on_host=False):
        """rpm_solve from the learned guess, falling back to the cold start;
        returns (status, info dict, used_guess)."""
        handle = ctx.handle if hasattr(ctx, "handle") else ctx
        info = rpm.rpm_solve_info()
        used = ctypes.c_int()
        st = lib().rpm_fno_solve(self.h, handle, rpm._E(E), rpm._ptr(eps_out), rpm._ptr(sig_out),
                                 int(out_on_host), ctypes.byref(info), ctypes.byref(used))
        if st in (rpm.RPM_ERR_INVALID_ARG, rpm.RPM_ERR_CUDA):
            _ck(self.h, st)
        return st, info.as_dict(), bool(used.value)

    def device_bytes(self) -> int:
        return int(lib().rpm_fno_device_bytes(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().rpm_fno_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def features(phase, phases, out, stream=None):
    """out [2][n] (device float32) <- voxel features of a device uint8 phase map."""
    arr = (rpm.rpm_iso * len(phases))(*[rpm.rpm_iso(float(l), float(m)) for (l, m) in phases])
    st = lib().rpm_fno_features(rpm._ptr(phase), int(phase.numel()), len(phases), arr,
                                rpm._ptr(out), rpm._stream_ptr(stream))
    _ck(None, st)
