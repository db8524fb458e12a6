"""Thin Python binding of the C ABI in include/lat.h (argument marshalling only).

Every step of the lattice method runs in the CUDA library ``liblat.so``; this module only
passes pointers, sizes and the current CUDA stream.  PyTorch provides device memory and
streams.  There is no CPU fallback: importing this module fails if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_longlong, c_void_p

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblat.so")

LAT_OK, LAT_EINVAL, LAT_ECFL, LAT_ENOMEM, LAT_ECUDA = 0, 1, 2, 3, 4
LAT_ENUMERIC, LAT_ETIMEOUT, LAT_EOVERFLOW, LAT_ENOISE = 5, 6, 7, 8
LAT_F64, LAT_F32, LAT_F16, LAT_BF16 = 0, 1, 2, 3
FLOW_NONE, FLOW_FIELD, FLOW_MODES = 0, 1, 2
LEARN_NPARAM = 5378
SCHEME_UPWIND, SCHEME_KOREN = 0, 1

_DTYPES = {torch.float64: LAT_F64, torch.float32: LAT_F32, torch.float16: LAT_F16,
           torch.bfloat16: LAT_BF16}


class LatGrid(ctypes.Structure):
    _fields_ = [("d", c_int), ("nx", c_int), ("ny", c_int), ("nv", c_int), ("dtype", c_int),
                ("L", c_double), ("tau_p", c_double), ("kappa", c_double), ("dt", c_double)]


class LatInstance(ctypes.Structure):
    _fields_ = [("nx", c_int), ("L", c_double), ("tau_p", c_double), ("kappa", c_double),
                ("dt", c_double)]


class LatFlow(ctypes.Structure):
    _fields_ = [("kind", c_int), ("field", c_void_p), ("nmodes", c_int), ("k", POINTER(c_int)),
                ("amp0", POINTER(c_double)), ("phase0", POINTER(c_double)),
                ("tau_f", c_double), ("sigma", c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "lat_init": (c_int, [POINTER(P), POINTER(LatGrid), P, P, P]),
        "lat_ensemble_init": (c_int, [POINTER(P), c_int, POINTER(LatInstance), c_int, c_int,
                                      P, P, P]),
        "lat_set_flow": (c_int, [P, POINTER(LatFlow)]),
        "lat_set_noise": (c_int, [P, POINTER(c_double), c_longlong]),
        "lat_step": (c_int, [P, c_int]),
        "lat_prepare": (c_int, [P, c_int]),
        "lat_moments": (c_int, [P, P, P, P, POINTER(c_double)]),
        "lat_step_moments": (c_int, [P, c_int, P, P, P, POINTER(c_double)]),
        "lat_step_moments_async": (c_int, [P, c_int, P]),
        "lat_status": (c_int, [P]),
        "lat_current": (c_int, [P]),
        "lat_steps_done": (c_longlong, [P]),
        "lat_set_launch": (c_int, [P, c_int, c_int, c_int, c_int]),
        "lat_set_scheme": (c_int, [P, c_int, c_double]),
        "lat_coarse_moment": (c_int, [P, c_int, P, P]),
        "lat_s1": (c_int, [P, c_int, P, P, P]),
        "lat_autotune": (c_int, [P, c_int, POINTER(c_double)]),
        "lat_strerror": (ctypes.c_char_p, [c_int]),
        "lat_free": (None, [P]),
        "lat_moments1d_noalloc": (c_int, [P, c_int, c_int, c_double, c_double, P, P]),
        "lat_encode": (c_int, [P, P]),
        "lat_learn": (c_int, [P, POINTER(ctypes.c_float), c_int]),
        "lat_restrict": (c_int, [P, c_int, c_int, c_int, P, P]),
        "lat_learn_corrections": (c_int, [P, P, c_int]),
        "lat_learn_grad": (c_int, [P, c_int, P, c_double, POINTER(c_double),
                                   POINTER(ctypes.c_float)]),
        "lat_decode": (c_int, [P, P, P]),
        "lat_get_density": (c_int, [P, POINTER(c_double)]),
        "lat_set_density": (c_int, [P, POINTER(c_double)]),
        "lat_state_bytes": (c_int, [P, POINTER(c_longlong)]),
        "lat_get_state": (c_int, [P, P, c_longlong]),
        "lat_set_state": (c_int, [P, P, c_longlong]),
        "lat_debug_stall": (c_int, [P, c_int]),
        "lat_adam": (c_int, [P, P, P, P, c_int, c_int, c_double, c_double, c_double, c_double,
                             c_double, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


class LatError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {_lib.lat_strerror(code).decode()} (code {code})")


def _check(code: int, what: str):
    if code != LAT_OK:
        raise LatError(code, what)


def _ptr(t: torch.Tensor | None):
    return None if t is None else c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


class _Ctx:
    """Common part of single-lattice and ensemble contexts."""

    def __init__(self):
        self._h = c_void_p()
        self._keep = []

    @property
    def handle(self):
        return self._h

    def _set_flow(self, kind, field=None, k=None, amp0=None, phase0=None, tau_f=0.0, sigma=0.0):
        fl = LatFlow()
        fl.kind = kind
        fl.field = None if field is None else field.data_ptr()
        if k is not None:
            k = np.ascontiguousarray(k, dtype=np.int32)
            fl.k = k.ctypes.data_as(POINTER(c_int))
            fl.nmodes = k.shape[0]
        if amp0 is not None:
            amp0 = np.ascontiguousarray(amp0, dtype=np.float64)
            fl.amp0 = _dptr(amp0)
        if phase0 is not None:
            phase0 = np.ascontiguousarray(phase0, dtype=np.float64)
            fl.phase0 = _dptr(phase0)
        fl.tau_f = float(tau_f)
        fl.sigma = float(sigma)
        self._field = field
        _check(_lib.lat_set_flow(self._h, byref(fl)), "lat_set_flow")

    def set_flow_none(self):
        self._set_flow(FLOW_NONE)

    def set_flow_field(self, u: torch.Tensor):
        self._set_flow(FLOW_FIELD, field=u)

    def set_noise(self, noise: np.ndarray):
        noise = np.ascontiguousarray(noise, dtype=np.float64)
        self._keep = [noise]
        _check(_lib.lat_set_noise(self._h, _dptr(noise), noise.shape[0] if noise.size else 0),
               "lat_set_noise")

    def set_noise_pinned(self, noise: torch.Tensor):
        """noise: pinned host float64 tensor (asynchronous copy)."""
        self._keep = [noise]
        _check(_lib.lat_set_noise(self._h, ctypes.cast(noise.data_ptr(), POINTER(c_double)),
                                  noise.shape[0]), "lat_set_noise")

    def step(self, n: int = 1):
        _check(_lib.lat_step(self._h, int(n)), "lat_step")

    def prepare(self, n: int):
        _check(_lib.lat_prepare(self._h, int(n)), "lat_prepare")

    def status(self) -> int:
        return _lib.lat_status(self._h)

    @property
    def current_index(self) -> int:
        return _lib.lat_current(self._h)

    @property
    def steps_done(self) -> int:
        return _lib.lat_steps_done(self._h)

    def step_moments_async(self, n: int, globals_out: torch.Tensor):
        """n steps and the globals of the final state into globals_out (a pinned host float64
        tensor, per instance [M, P_1..P_d, E]) without synchronising: the values are there once
        the stream has passed this point.  The tensor is kept referenced until then."""
        if globals_out.is_cuda or globals_out.dtype != torch.float64 or not globals_out.is_pinned():
            raise ValueError("globals_out must be a pinned host float64 tensor")
        self._keep_async = getattr(self, "_keep_async", [])[-63:] + [globals_out]
        _check(_lib.lat_step_moments_async(self._h, int(n), c_void_p(globals_out.data_ptr())),
               "lat_step_moments_async")

    def set_launch(self, kernel=0, block=0, blocks_per_sm=0, mode=-1):
        _check(_lib.lat_set_launch(self._h, kernel, block, blocks_per_sm, mode), "lat_set_launch")

    def set_scheme(self, scheme: int, mu: float = 2.0 / 3.0):
        """Drag sub-step scheme: SCHEME_UPWIND or SCHEME_KOREN (limiter bound mu)."""
        _check(_lib.lat_set_scheme(self._h, scheme, mu), "lat_set_scheme")

    def coarse_moment(self, widths):
        """<rho_r^2> for window widths in cells: array [instances, len(widths)]."""
        w = np.ascontiguousarray(widths, dtype=np.int32)
        out = np.zeros((self._n_out(), len(w)))
        _check(_lib.lat_coarse_moment(self._h, len(w), w.ctypes.data_as(POINTER(c_int)),
                                       _dptr(out)),
               "lat_coarse_moment")
        return out

    def s1(self, seps):
        """Eulerian S1 terms for separations in cells: (num, den), each [instances, len(seps)];
        S1 = num / den."""
        s = np.ascontiguousarray(seps, dtype=np.int32)
        num = np.zeros((self._n_out(), len(s)))
        den = np.zeros_like(num)
        _check(_lib.lat_s1(self._h, len(s), s.ctypes.data_as(POINTER(c_int)), _dptr(num),
                           _dptr(den)), "lat_s1")
        return num, den

    def _n_out(self):
        return 1

    def autotune(self, reps: int = 5):
        best = np.zeros(4)
        _check(_lib.lat_autotune(self._h, reps, _dptr(best)), "lat_autotune")
        return {"kernel": int(best[0]), "block": int(best[1]), "blocks_per_sm": int(best[2]),
                "us_per_step": float(best[3])}

    def _values(self) -> int:
        return self.f[0].numel()

    def get_density(self) -> np.ndarray:
        """The current state as FP64 host values, flat in the layout of f."""
        out = np.empty(self._values(), dtype=np.float64)
        _check(_lib.lat_get_density(self._h, _dptr(out)), "lat_get_density")
        return out

    def set_density(self, f: np.ndarray):
        """Replace the current state by the FP64 host values f (layout of f)."""
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        if f.size != self._values():
            raise ValueError(f"expected {self._values()} values")
        _check(_lib.lat_set_density(self._h, _dptr(f)), "lat_set_density")

    def get_state(self) -> np.ndarray:
        """Checkpoint image of the context (host bytes)."""
        n = c_longlong()
        _check(_lib.lat_state_bytes(self._h, byref(n)), "lat_state_bytes")
        img = np.empty(n.value, dtype=np.uint8)
        _check(_lib.lat_get_state(self._h, c_void_p(img.ctypes.data), n.value), "lat_get_state")
        return img

    def set_state(self, img: np.ndarray):
        """Restore a checkpoint image made by get_state."""
        img = np.ascontiguousarray(img, dtype=np.uint8)
        _check(_lib.lat_set_state(self._h, c_void_p(img.ctypes.data), img.size), "lat_set_state")

    def debug_stall(self, on: bool):
        """Timeout-path test hook: the pipeline kernels' producers issue no copies while on."""
        _check(_lib.lat_debug_stall(self._h, int(bool(on))), "lat_debug_stall")

    def close(self):
        if self._h:
            _lib.lat_free(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice(_Ctx):
    """One 1D or 2D lattice.  f0 (device tensor) holds the initial state in the layout of
    include/lat.h; a second buffer of the same shape is allocated here (torch)."""

    def __init__(self, f0: torch.Tensor, *, d: int, nx: int, ny: int = 1, nv: int, L: float,
                 tau_p: float, kappa: float, dt: float, stream=None):
        super().__init__()
        if f0.dtype not in _DTYPES or not f0.is_cuda or not f0.is_contiguous():
            raise ValueError("f0 must be a contiguous CUDA tensor of float64/32/16 or bfloat16")
        self.d, self.nx, self.ny, self.nv = d, nx, ny, nv
        self.L, self.dt = L, dt
        self.dx = L / nx
        self.dv = self.dx / dt
        self.f = [f0, torch.empty_like(f0)]
        g = LatGrid(d, nx, ny, nv, _DTYPES[f0.dtype], L, tau_p, kappa, dt)
        _check(_lib.lat_init(byref(self._h), byref(g), _ptr(self.f[0]), _ptr(self.f[1]),
                             _stream(stream)), "lat_init")

    @property
    def state(self) -> torch.Tensor:
        return self.f[self.current_index]

    def set_flow_modes_1d(self, k, amp0, tau_f: float, sigma: float):
        self._set_flow(FLOW_MODES, k=k, amp0=np.asarray(amp0).reshape(-1), tau_f=tau_f,
                       sigma=sigma)

    def set_flow_modes_2d(self, kvec, a, phi0, tau_f: float):
        self._set_flow(FLOW_MODES, k=np.asarray(kvec, dtype=np.int32).reshape(-1, 2), amp0=a,
                       phase0=phi0, tau_f=tau_f)

    def encode(self, src: torch.Tensor):
        """16-bit storage: replace the state by the encoding of the FP32 tensor src."""
        if src.dtype != torch.float32 or not src.is_cuda or not src.is_contiguous():
            raise ValueError("src must be a contiguous CUDA float32 tensor")
        if src.numel() != self.f[0].numel():
            raise ValueError("src must have the state's size")
        _check(_lib.lat_encode(self._h, _ptr(src)), "lat_encode")

    def learn(self, params, mode: int = 1):
        """Learned flux closure (2D FP32): params = the LAT_LEARN_NPARAM parameters (numpy);
        mode 0 off, 1 FP32 network, 2 BF16 tensor-core network."""
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
        if p.size != LEARN_NPARAM:
            raise ValueError(f"expected {LEARN_NPARAM} parameters")
        _check(_lib.lat_learn(self._h, p.ctypes.data_as(POINTER(ctypes.c_float)), mode),
               "lat_learn")

    def learn_corrections(self, out: torch.Tensor | None = None, reuse_inputs: bool = False):
        """Correction fluxes of the current state (enqueued; copied into out when given);
        reuse_inputs runs the network alone on the previous call's flow and density."""
        _check(_lib.lat_learn_corrections(self._h, _ptr(out), int(reuse_inputs)),
               "lat_learn_corrections")
        return out

    def learn_grad(self, nsteps: int, target: torch.Tensor, rho_weight: float = 0.0):
        """Loss of an nsteps rollout against target (device FP32) and its gradient (numpy)."""
        if target.dtype != torch.float32 or not target.is_cuda or not target.is_contiguous():
            raise ValueError("target must be a contiguous CUDA float32 tensor")
        loss = np.zeros(1)
        grad = np.zeros(LEARN_NPARAM, dtype=np.float32)
        _check(_lib.lat_learn_grad(self._h, nsteps, _ptr(target), float(rho_weight), _dptr(loss),
                                   grad.ctypes.data_as(POINTER(ctypes.c_float))), "lat_learn_grad")
        return float(loss[0]), grad

    def decode(self):
        """16-bit storage: the current state as FP32 and its line scales [N_v^2 N_y]."""
        dst = torch.empty(self.f[0].shape, dtype=torch.float32, device=self.f[0].device)
        sc = torch.empty(self.nv * self.nv * self.ny, dtype=torch.float32,
                         device=self.f[0].device)
        _check(_lib.lat_decode(self._h, _ptr(dst), _ptr(sc)), "lat_decode")
        return dst, sc

    def moments(self, per_cell: bool = True):
        ncell = self.nx * self.ny
        dev = self.f[0].device
        rho = torch.empty(ncell, dtype=torch.float64, device=dev) if per_cell else None
        mv = torch.empty(self.d * ncell, dtype=torch.float64, device=dev) if per_cell else None
        mv2 = torch.empty(ncell, dtype=torch.float64, device=dev) if per_cell else None
        glob = np.zeros(self.d + 2)
        code = _lib.lat_moments(self._h, _ptr(rho), _ptr(mv), _ptr(mv2), _dptr(glob))
        return code, rho, mv, mv2, glob

    def step_moments(self, n: int = 1, per_cell: bool = True,
                     globals_out: np.ndarray | None = None):
        """n steps, then the moments of the new state (fused into the last step where the
        launch allows it); the outputs of moments()."""
        ncell = self.nx * self.ny
        dev = self.f[0].device
        rho = torch.empty(ncell, dtype=torch.float64, device=dev) if per_cell else None
        mv = torch.empty(self.d * ncell, dtype=torch.float64, device=dev) if per_cell else None
        mv2 = torch.empty(ncell, dtype=torch.float64, device=dev) if per_cell else None
        glob = globals_out if globals_out is not None else np.zeros(self.d + 2)
        code = _lib.lat_step_moments(self._h, int(n), _ptr(rho), _ptr(mv), _ptr(mv2),
                                     _dptr(glob))
        return code, rho, mv, mv2, glob


class Ensemble(_Ctx):
    """Independent 1D lattices advanced together (one persistent launch per step)."""

    def __init__(self, f0: torch.Tensor, *, nv: int, nx, L, tau_p, kappa, dt, stream=None):
        super().__init__()
        n = len(nx)
        if f0.dtype not in (torch.float32, torch.float64) or not f0.is_cuda:
            raise ValueError("f0 must be a CUDA float32/float64 tensor")
        self.n, self.nv = n, nv
        self.nx = np.asarray(nx, dtype=np.int64)
        self.offsets = np.concatenate([[0], np.cumsum(self.nx * nv)])
        self.xoff = np.concatenate([[0], np.cumsum(self.nx)])
        self.f = [f0, torch.empty_like(f0)]
        arr = (LatInstance * n)()
        for i in range(n):
            arr[i] = LatInstance(int(nx[i]), float(L[i]), float(tau_p[i]), float(kappa[i]),
                                 float(dt[i]))
        _check(_lib.lat_ensemble_init(byref(self._h), n, arr, nv, _DTYPES[f0.dtype],
                                      _ptr(self.f[0]), _ptr(self.f[1]), _stream(stream)),
               "lat_ensemble_init")

    def _n_out(self):
        return self.n

    @property
    def state(self) -> torch.Tensor:
        return self.f[self.current_index]

    def instance_view(self, i: int, t: torch.Tensor | None = None) -> torch.Tensor:
        t = self.state if t is None else t
        return t[int(self.offsets[i]):int(self.offsets[i + 1])].view(self.nv, int(self.nx[i]))

    def set_flow_modes(self, k, amp0, tau_f: float, sigma: float):
        self._set_flow(FLOW_MODES, k=k, amp0=np.asarray(amp0).reshape(-1), tau_f=tau_f,
                       sigma=sigma)

    def moments(self, per_cell: bool = False, globals_out: np.ndarray | None = None):
        ncell = int(self.xoff[-1])
        dev = self.f[0].device
        rho = torch.empty(ncell, dtype=torch.float64, device=dev) if per_cell else None
        mv = torch.empty(ncell, dtype=torch.float64, device=dev) if per_cell else None
        mv2 = torch.empty(ncell, dtype=torch.float64, device=dev) if per_cell else None
        glob = globals_out if globals_out is not None else np.zeros((self.n, 3))
        code = _lib.lat_moments(self._h, _ptr(rho), _ptr(mv), _ptr(mv2), _dptr(glob))
        return code, rho, mv, mv2, glob

    def step_moments(self, n: int = 1, per_cell: bool = False,
                     globals_out: np.ndarray | None = None):
        """n steps, then the moments of the new state (fused into the last step when the
        producer/consumer kernel runs)."""
        ncell = int(self.xoff[-1])
        dev = self.f[0].device
        rho = torch.empty(ncell, dtype=torch.float64, device=dev) if per_cell else None
        mv = torch.empty(ncell, dtype=torch.float64, device=dev) if per_cell else None
        mv2 = torch.empty(ncell, dtype=torch.float64, device=dev) if per_cell else None
        glob = globals_out if globals_out is not None else np.zeros((self.n, 3))
        code = _lib.lat_step_moments(self._h, int(n), _ptr(rho), _ptr(mv), _ptr(mv2),
                                     _dptr(glob))
        return code, rho, mv, mv2, glob


def exported_symbols():
    return [n for n in dir(_lib) if n.startswith("lat_")]


def adam(params: torch.Tensor, m: torch.Tensor, v: torch.Tensor, grad: torch.Tensor, t: int,
         lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
         grad_scale: float = 1.0, stream=None):
    """One Adam step on device float32 tensors of the same size (in place: params, m, v)."""
    for x in (params, m, v, grad):
        if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("adam takes contiguous CUDA float32 tensors")
    _check(_lib.lat_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), params.numel(), int(t),
                         lr, beta1, beta2, eps, grad_scale, _stream(stream)), "lat_adam")


def restrict(fine: torch.Tensor, nx: int, ny: int, stream=None) -> torch.Tensor:
    """Fine 2D FP32 state (N_v = 4 m + 1) -> coarse state (N_v = m + 1), on the device."""
    nvf = fine.shape[0]
    nvc = (nvf - 1) // 4 + 1
    out = torch.empty((nvc, nvc, ny, nx), dtype=torch.float32, device=fine.device)
    _check(_lib.lat_restrict(_ptr(fine), nvf, nx, ny, _ptr(out), _stream(stream)), "lat_restrict")
    return out
