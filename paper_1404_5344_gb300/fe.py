"""Python binding of libfe (C ABI in include/fe.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; this module only
converts arguments (NumPy arrays -> host pointers, torch CUDA tensors -> device
pointers, torch streams -> cudaStream_t) and checks status codes.  Importing it
loads ``_build/libfe.so`` and raises ImportError if the library is missing;
there is no fallback path.

Names follow the C ABI: ``fe_init_batch`` -> :class:`Solver`, ``fe_step`` ->
:meth:`Solver.step`, ``fe_solve`` -> :meth:`Solver.solve`, ``fe_energy`` ->
:meth:`Solver.energy`, ``fe_gradient`` -> :meth:`Solver.gradient`, etc.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libfe.so")

FE_OK, FE_EINVAL, FE_ENOMEM, FE_ECUDA, FE_ENONFINITE = 0, 1, 2, 3, 4
FE_EBACKTRACK, FE_ETIMEOUT, FE_ENOTCONVERGED, FE_EUNSUPPORTED = 5, 6, 7, 8
FE_FP32, FE_TF32, FE_BF16, FE_BF16R = 0, 1, 2, 3
FE_TILE_CLUSTER4 = 0x100
PRECISIONS = {"fp32": FE_FP32, "tf32": FE_TF32, "bf16": FE_BF16, "bf16r": FE_BF16R}

#: every symbol include/fe.h declares
EXPORTS = (
    "fe_default_params", "fe_init_batch", "fe_init", "fe_reset", "fe_destroy", "fe_step",
    "fe_solve", "fe_get_info", "fe_get_u", "fe_energy", "fe_gradient", "fe_get_state",
    "fe_set_state", "fe_num_images", "fe_image_size", "fe_launch_count", "fe_set_loop_mode", "fe_tile_size",
    "fe_ssim", "fe_psnr", "fe_tc_wait_selftest", "fe_persist_wait_selftest", "fe_tile_cluster",
    "fe_last_error", "fe_status_string", "fe_abi_version", "fe_gradient_noalloc",
    "fe_tc_gemm_selftest", "fe_cnn_create", "fe_cnn_destroy", "fe_cnn_num_params",
    "fe_cnn_last_error", "fe_cnn_set_params", "fe_cnn_get_params", "fe_cnn_forward",
    "fe_cnn_loss_grad", "fe_cnn_train_step", "fe_peak", "fe_device_sms", "fe_solve_to_energy",
)


class FeParams(C.Structure):
    _fields_ = [("nf", C.c_int), ("ksize", C.c_int), ("filters", C.POINTER(C.c_float)),
                ("theta", C.POINTER(C.c_float)), ("lambda_", C.c_double), ("beta", C.c_double),
                ("L0", C.c_double), ("eta", C.c_double), ("c2", C.c_double),
                ("max_backtrack", C.c_int), ("prec", C.c_int), ("tile", C.c_int), ("model", C.c_int),
                ("lambda1", C.c_double)]


MODELS = {"variant": 0, "combined": 1}


class FeInfo(C.Structure):
    _fields_ = [("n", C.c_longlong), ("trials", C.c_longlong), ("backtracks", C.c_longlong),
                ("L", C.c_double), ("alpha", C.c_double), ("F", C.c_double), ("G", C.c_double),
                ("H", C.c_double), ("H_prev", C.c_double), ("rel_change", C.c_double),
                ("last_gd", C.c_double), ("last_dd", C.c_double), ("last_dp", C.c_double),
                ("status", C.c_int), ("converged", C.c_int), ("G_floor", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError("libfe.so not built at %s (run __graft_entry__.build())" % path)
    L = C.CDLL(path)
    P, I, D, VP = C.POINTER, C.c_int, C.c_double, C.c_void_p
    L.fe_default_params.argtypes = [P(FeParams)]
    L.fe_default_params.restype = None
    L.fe_init_batch.argtypes = [P(VP), P(FeParams), I, P(I), P(I), P(VP), P(VP), VP]
    L.fe_init.argtypes = [P(VP), P(FeParams), I, I, VP, VP, VP]
    L.fe_reset.argtypes = [VP, P(VP), P(VP)]
    L.fe_destroy.argtypes = [VP]
    L.fe_destroy.restype = None
    L.fe_step.argtypes = [VP, I, P(I)]
    L.fe_solve.argtypes = [VP, I, D]
    L.fe_solve_to_energy.argtypes = [VP, I, D, VP]
    L.fe_get_info.argtypes = [VP, I, P(FeInfo)]
    L.fe_get_u.argtypes = [VP, I, VP]
    L.fe_energy.argtypes = [VP, I, VP, P(D), P(D), P(D)]
    L.fe_gradient.argtypes = [VP, I, VP, VP, P(D)]
    L.fe_get_state.argtypes = [VP, I, VP, VP, VP, P(FeInfo)]
    L.fe_set_state.argtypes = [VP, I, VP, VP, VP, P(FeInfo)]
    L.fe_num_images.argtypes = [VP]
    L.fe_image_size.argtypes = [VP, I, P(I), P(I)]
    L.fe_tile_size.argtypes = [VP, P(I), P(I)]
    L.fe_tile_cluster.argtypes = [VP]
    L.fe_ssim.argtypes = [VP, VP, I, I, D, P(D), VP]
    L.fe_tc_wait_selftest.argtypes = [C.c_uint, P(I)]
    L.fe_persist_wait_selftest.argtypes = [D, P(I), P(D)]
    L.fe_psnr.argtypes = [VP, VP, C.c_longlong, D, P(D), VP]
    L.fe_launch_count.argtypes = [VP]
    L.fe_launch_count.restype = C.c_longlong
    L.fe_set_loop_mode.argtypes = [VP, I]
    L.fe_last_error.argtypes = [VP]
    L.fe_last_error.restype = C.c_char_p
    L.fe_status_string.argtypes = [I]
    L.fe_status_string.restype = C.c_char_p
    L.fe_abi_version.argtypes = []
    L.fe_gradient_noalloc.argtypes = [VP, VP, VP, I, I, VP, VP, I, VP]
    L.fe_tc_gemm_selftest.argtypes = [I, I, I, VP, VP, VP]
    L.fe_cnn_create.argtypes = [P(VP), C.c_ulonglong, VP]
    L.fe_cnn_destroy.argtypes = [VP]
    L.fe_cnn_destroy.restype = None
    L.fe_cnn_num_params.argtypes = [VP]
    L.fe_cnn_last_error.argtypes = [VP]
    L.fe_cnn_last_error.restype = C.c_char_p
    L.fe_cnn_set_params.argtypes = [VP, VP]
    L.fe_cnn_get_params.argtypes = [VP, VP]
    L.fe_cnn_forward.argtypes = [VP, VP, I, I, I, VP, VP]
    L.fe_cnn_loss_grad.argtypes = [VP, VP, VP, I, I, I, P(D), VP]
    L.fe_cnn_train_step.argtypes = [VP, VP, VP, I, I, I, C.c_float, P(D)]
    L.fe_peak.argtypes = [I, D, I, P(D), P(D), P(I)]
    L.fe_device_sms.argtypes = [P(I)]
    for name in ("fe_cnn_create", "fe_cnn_num_params", "fe_cnn_set_params", "fe_cnn_get_params",
                 "fe_cnn_forward", "fe_cnn_loss_grad", "fe_cnn_train_step"):
        getattr(L, name).restype = C.c_int
    for name in ("fe_tc_gemm_selftest", "fe_gradient_noalloc", "fe_init_batch","fe_init", "fe_reset", "fe_step", "fe_solve", "fe_get_info",
                 "fe_get_u", "fe_energy", "fe_gradient", "fe_get_state", "fe_set_state",
                 "fe_image_size", "fe_set_loop_mode", "fe_num_images", "fe_abi_version", "fe_tile_size",
                 "fe_ssim", "fe_psnr", "fe_tc_wait_selftest", "fe_persist_wait_selftest", "fe_tile_cluster", "fe_peak",
                 "fe_device_sms", "fe_solve_to_energy"):
        getattr(L, name).restype = C.c_int
    return L


lib = _load()


class FeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (lib.fe_status_string(status).decode(), status, msg))
        self.status = status


def _ptr(a):
    """Host or device address of an array-like (NumPy array or torch tensor)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor
        if a.dtype.__repr__() != "torch.float32" or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float32")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise TypeError("arrays must be C-contiguous float32")
        return a.ctypes.data
    if isinstance(a, int):
        return a
    raise TypeError("unsupported buffer type %r" % type(a))


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def default_params() -> FeParams:
    p = FeParams()
    lib.fe_default_params(C.byref(p))
    return p


class Solver:
    """A libfe context over one or more images (``fe_init_batch``).

    f: list of H x W float32 arrays (NumPy = host, torch CUDA = device).
    filters: (nf, 7, 7) float32, theta: (nf,) float32.
    model: "variant" (Eq. variant, iterate u, weight lam) or "combined"
    (Eq. newmodel, iterate w = log u, weights lam1 for the log-domain term
    and lam for the variant term; lam = 0 is Eq. original).
    """

    def __init__(self, f, filters, theta, lam=5.0, beta=0.8, L0=1.0, eta=2.0, c2=1e-6,
                 max_backtrack=30, prec="fp32", tile=0, u0=None, stream=None, loop_mode=None,
                 model="variant", lam1=0.0):
        if not isinstance(f, (list, tuple)):
            f = [f]
        self._keep = list(f) + (list(u0) if isinstance(u0, (list, tuple)) else [u0])
        self.shapes = [tuple(int(s) for s in x.shape) for x in f]
        self._filters = np.ascontiguousarray(filters, dtype=np.float32).reshape(-1, 49)
        self._theta = np.ascontiguousarray(theta, dtype=np.float32).reshape(-1)
        p = default_params()
        p.nf = self._filters.shape[0]
        p.ksize = 7
        p.filters = self._filters.ctypes.data_as(C.POINTER(C.c_float))
        p.theta = self._theta.ctypes.data_as(C.POINTER(C.c_float))
        p.lambda_, p.beta, p.L0, p.eta, p.c2 = float(lam), float(beta), float(L0), float(eta), float(c2)
        p.max_backtrack = int(max_backtrack)
        p.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        p.tile = int(tile)
        p.model = MODELS[model] if isinstance(model, str) else int(model)
        p.lambda1 = float(lam1)
        self.params = p
        n = len(f)
        Hs = (C.c_int * n)(*[s[0] for s in self.shapes])
        Ws = (C.c_int * n)(*[s[1] for s in self.shapes])
        fp = (C.c_void_p * n)(*[_ptr(x) for x in f])
        up = None
        if u0 is not None:
            u0l = u0 if isinstance(u0, (list, tuple)) else [u0]
            up = (C.c_void_p * n)(*[_ptr(x) for x in u0l])
        self.ctx = C.c_void_p()
        st = lib.fe_init_batch(C.byref(self.ctx), C.byref(p), n, Hs, Ws, fp, up, _stream_handle(stream))
        if st != FE_OK:
            raise FeError(st, lib.fe_last_error(None).decode())
        if loop_mode is not None:
            self._check(lib.fe_set_loop_mode(self.ctx, int(loop_mode)))

    # -- plumbing ------------------------------------------------------
    def _check(self, st):
        if st != FE_OK:
            raise FeError(st, lib.fe_last_error(self.ctx).decode())
        return st

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            lib.fe_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def nimg(self):
        return lib.fe_num_images(self.ctx)

    @property
    def tile(self):
        """(rows, columns) of the trial kernel's output tile."""
        ty, tx = C.c_int(), C.c_int()
        self._check(lib.fe_tile_size(self.ctx, C.byref(ty), C.byref(tx)))
        return ty.value, tx.value

    @property
    def cluster(self) -> int:
        """CTAs working on one tile (4: a thread-block cluster per tile)."""
        return int(lib.fe_tile_cluster(self.ctx))

    # -- ABI calls -----------------------------------------------------
    def reset(self, f, u0=None):
        f = f if isinstance(f, (list, tuple)) else [f]
        n = len(f)
        fp = (C.c_void_p * n)(*[_ptr(x) for x in f])
        up = None
        if u0 is not None:
            u0l = u0 if isinstance(u0, (list, tuple)) else [u0]
            up = (C.c_void_p * n)(*[_ptr(x) for x in u0l])
        self._check(lib.fe_reset(self.ctx, fp, up))

    def step(self, n: int = 1, sync: bool = True) -> int:
        """fe_step: n accepted iterations per image; returns the worst status."""
        if sync:
            w = C.c_int(0)
            self._check(lib.fe_step(self.ctx, int(n), C.byref(w)))
            return w.value
        self._check(lib.fe_step(self.ctx, int(n), None))
        return FE_OK

    def solve(self, max_iter: int, rel_tol: float) -> int:
        st = lib.fe_solve(self.ctx, int(max_iter), float(rel_tol))
        if st not in (FE_OK, FE_ENOTCONVERGED):
            self._check(st)
        return st

    def solve_to_energy(self, max_iter: int, H_target, rel_tol: float = 0.0) -> int:
        """fe_solve_to_energy: also stop image j once an accepted H <= H_target[j]."""
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(H_target, np.float64), (self.nimg,)))
        st = lib.fe_solve_to_energy(self.ctx, int(max_iter), float(rel_tol), t.ctypes.data)
        if st not in (FE_OK, FE_ENOTCONVERGED):
            self._check(st)
        return st

    def info(self, img: int = 0) -> dict:
        i = FeInfo()
        self._check(lib.fe_get_info(self.ctx, int(img), C.byref(i)))
        return i.as_dict()

    def get_u(self, img: int = 0, out=None):
        if out is None:
            out = np.empty(self.shapes[img], np.float32)
        self._check(lib.fe_get_u(self.ctx, int(img), _ptr(out)))
        return out

    def get_state(self, img: int = 0):
        H, W = self.shapes[img]
        u, up, g = (np.empty((H, W), np.float32) for _ in range(3))
        i = FeInfo()
        self._check(lib.fe_get_state(self.ctx, int(img), _ptr(u), _ptr(up), _ptr(g), C.byref(i)))
        return u, up, g, i.as_dict()

    def set_state(self, img, u, u_prev, g, info: dict):
        i = FeInfo()
        for k, v in info.items():
            setattr(i, k, v)
        self._check(lib.fe_set_state(self.ctx, int(img), _ptr(u), _ptr(u_prev), _ptr(g), C.byref(i)))

    def energy(self, img, u):
        E, F, G = C.c_double(), C.c_double(), C.c_double()
        self._check(lib.fe_energy(self.ctx, int(img), _ptr(u), C.byref(E), C.byref(F), C.byref(G)))
        return E.value, F.value, G.value

    def gradient(self, img, u, out=None):
        if out is None:
            out = np.empty(self.shapes[img], np.float32)
        F = C.c_double()
        self._check(lib.fe_gradient(self.ctx, int(img), _ptr(u), _ptr(out), C.byref(F)))
        return out, F.value

    def launch_count(self) -> int:
        return int(lib.fe_launch_count(self.ctx))

    def set_loop_mode(self, mode: int):
        self._check(lib.fe_set_loop_mode(self.ctx, int(mode)))


def ssim(x, y, peak: float = 255.0, stream=None) -> float:
    """fe_ssim: mean SSIM index of x against y (contiguous float32 CUDA
    tensors of the same H x W shape)."""
    H, W = (int(v) for v in x.shape)
    if tuple(y.shape) != (H, W):
        raise ValueError("x and y must have the same shape")
    out = C.c_double()
    st = lib.fe_ssim(_ptr(x), _ptr(y), H, W, float(peak), C.byref(out), _stream_handle(stream))
    if st != FE_OK:
        raise FeError(st, lib.fe_last_error(None).decode())
    return out.value


def psnr(x, y, peak: float = 255.0, stream=None) -> float:
    """fe_psnr: 10 log10(peak^2 / MSE) of x against y (float32 CUDA tensors)."""
    n = int(np.prod(x.shape))
    if int(np.prod(y.shape)) != n:
        raise ValueError("x and y must have the same size")
    out = C.c_double()
    st = lib.fe_psnr(_ptr(x), _ptr(y), n, float(peak), C.byref(out), _stream_handle(stream))
    if st != FE_OK:
        raise FeError(st, lib.fe_last_error(None).decode())
    return out.value


PEAK_KINDS = {"ffma": 0, "ffma2": 1, "dfma": 2, "mufu_rcp": 3, "mufu_lg2": 4, "tc_bf16": 5, "tc_tf32": 6}


def peak(kind: str, target_ms: float = 20.0, reps: int = 5) -> dict:
    """fe_peak: measured rate of one unit of the current device (flop/s for
    the FMA and tensor kinds, instructions/s for the MUFU kinds)."""
    rate, ms, sms = C.c_double(), C.c_double(), C.c_int()
    st = lib.fe_peak(PEAK_KINDS[kind], float(target_ms), int(reps), C.byref(rate), C.byref(ms), C.byref(sms))
    if st != FE_OK:
        raise FeError(st, lib.fe_last_error(None).decode())
    return {"rate": rate.value, "ms": ms.value, "sms": sms.value}


def device_sms() -> int:
    """fe_device_sms: multiprocessor count of the current device."""
    n = C.c_int()
    st = lib.fe_device_sms(C.byref(n))
    if st != FE_OK:
        raise FeError(st, lib.fe_last_error(None).decode())
    return n.value


class CNN:
    """The warm-start network of the C ABI (``fe_cnn_*``): 5 x (3x3 conv), 32
    channels, BF16 weights, FP32 activations; predicts u0 = f exp(d)."""

    def __init__(self, seed: int = 0, stream=None):
        self.ptr = C.c_void_p()
        st = lib.fe_cnn_create(C.byref(self.ptr), int(seed), _stream_handle(stream))
        if st != FE_OK:
            raise FeError(st, "fe_cnn_create")
        self.num_params = lib.fe_cnn_num_params(self.ptr)

    def _check(self, st):
        if st != FE_OK:
            raise FeError(st, lib.fe_cnn_last_error(self.ptr).decode())

    def close(self):
        if getattr(self, "ptr", None) and self.ptr.value:
            lib.fe_cnn_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _bhw(x):
        s = tuple(int(v) for v in x.shape)
        return (1,) + s if len(s) == 2 else s

    def get_params(self):
        p = np.empty(self.num_params, np.float32)
        self._check(lib.fe_cnn_get_params(self.ptr, _ptr(p)))
        return p

    def set_params(self, p):
        p = p if hasattr(p, "data_ptr") else np.ascontiguousarray(p, np.float32)
        self._check(lib.fe_cnn_set_params(self.ptr, _ptr(p)))

    def forward(self, f, u0=None, d=None):
        """u0 = f exp(d) into u0 (and d into d); f is [H, W] or [B, H, W]."""
        B, H, W = self._bhw(f)
        if u0 is None and d is None:
            u0 = np.empty(f.shape, np.float32)
        self._check(lib.fe_cnn_forward(self.ptr, _ptr(f), B, H, W, _ptr(u0), _ptr(d)))
        return u0 if u0 is not None else d

    def loss_grad(self, f, u_target):
        B, H, W = self._bhw(f)
        loss = C.c_double()
        g = np.empty(self.num_params, np.float32)
        self._check(lib.fe_cnn_loss_grad(self.ptr, _ptr(f), _ptr(u_target), B, H, W, C.byref(loss), _ptr(g)))
        return loss.value, g

    def train_step(self, f, u_target, lr: float) -> float:
        B, H, W = self._bhw(f)
        loss = C.c_double()
        self._check(lib.fe_cnn_train_step(self.ptr, _ptr(f), _ptr(u_target), B, H, W, float(lr), C.byref(loss)))
        return loss.value
