"""Python binding of libkry_gb300.so (C ABI in include/kry.h).

Argument marshalling only: every step of the Krylov path runs in the library's CUDA
kernels.  PyTorch provides device memory and the current stream.  There is no fallback:
if the library is missing or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libkry_gb300.so")

KRY_OK, KRY_EINVAL, KRY_ENOMEM, KRY_ETOL, KRY_ETIMEOUT, KRY_ECUDA = range(6)
KRY_OBC, KRY_PBC = 0, 1
KRY_C128, KRY_C64, KRY_C128E = 0, 1, 2
# dtype names: complex128 (FP64 arithmetic), complex64 (mixed precision), and complex128 in
# and out with float-float vectors and arithmetic on the FP32 pipe inside
_CODES = {"c128": KRY_C128, "complex128": KRY_C128, "c64": KRY_C64, "complex64": KRY_C64,
          "c128e": KRY_C128E}
MMAX = 32

# Every symbol the header declares, with (restype, argtypes).
_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)


class Stats(ctypes.Structure):
    """kry_stats: counters of one evolution."""
    _fields_ = [("n_hv", ctypes.c_int64), ("n_krylov_steps", ctypes.c_int64),
                ("n_second_pass", ctypes.c_int64), ("n_breakdowns", ctypes.c_int64),
                ("err_estimate", ctypes.c_double), ("max_orth_loss", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("algo_bytes", ctypes.c_double),
                ("n_launches", ctypes.c_int64), ("n_second_dots", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


SIGNATURES = {
    "kry_basis_create": (_i, [_i, _i, ctypes.POINTER(_vp)]),
    "kry_basis_create_list": (_i, [_i, _i, ctypes.POINTER(_vp)]),
    "kry_basis_destroy": (_i, [_vp]),
    "kry_basis_dim": (_i64, [_vp]),
    "kry_basis_rank": (_i, [_vp, _vp, _vp, _i64, _vp]),
    "kry_basis_unrank": (_i, [_vp, _vp, _vp, _i64, _vp]),
    "kry_hamiltonian_set": (_i, [_vp, _d, _d, _dp, _i, _i, ctypes.POINTER(_vp)]),
    "kry_hamiltonian_destroy": (_i, [_vp]),
    "kry_apply": (_i, [_vp, _i, _vp, _vp, _vp]),
    "kry_evolve": (_i, [_vp, _i, _vp, _dp, _i, _i, _d, _vp, _dp, ctypes.POINTER(Stats), _vp]),
    "kry_return_probability": (_i, [_vp, _i, ctypes.c_uint64, _dp, _i, _i, _d, _dp,
                                    ctypes.POINTER(Stats), _vp]),
    "kry_autocorrelation": (_i, [_vp, _i, ctypes.c_uint64, _dp, _i, _i, _d, _dp, _dp,
                                 ctypes.POINTER(Stats), _vp]),
    "kry_return_probability_states": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_uint64), _dp, _i, _i, _d, _dp,
                                           _dp, ctypes.POINTER(Stats), _vp]),
    "kry_decay_exponent": (_i, [_dp, _dp, _i, _d, _d, _dp, _dp]),
    "kry_grad": (_i, [_vp, ctypes.c_uint64, _d, _i, _d, _i, _dp, _dp, _dp, ctypes.POINTER(Stats), _vp]),
    "kry_tridiag_expv": (_i, [_dp, _dp, _i, _d, _d, _dp, _dp, _vp]),
    "kry_tridiag_expv_noalloc": (_i, [_dp, _dp, _i, _d, _d, _dp, _dp, _vp]),
    "kry_workspace_size": (_i64, [_vp, _i, _i]),
    "kry_workspace_bytes": (_i64, [_vp, _i, _i, _i]),
    "kry_set_workspace": (_i, [_vp, _vp, _i64]),
    "kry_autotune": (_i, [_vp, _i, _i, ctypes.c_uint64, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_i),
                          _dp, _i, ctypes.POINTER(_i), _vp]),
    "kry_set_grid": (_i, [_vp, _i, _i]),
    "kry_set_shape": (_i, [_vp, _i, ctypes.POINTER(_i)]),
    "kry_get_shape": (_i, [_vp, _i, ctypes.POINTER(_i)]),
    "kry_set_orth_check": (_i, [_vp, _i]),
    "kry_set_second_pass_node": (_i, [_vp, _i]),
    "kry_profile_enable": (_i, [_vp, _i]),
    "kry_profile_read": (_i, [_vp, _dp, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "kry_measure_peaks": (_i, [_dp, _dp, _vp]),
    "kry_last_error": (ctypes.c_char_p, []),
}

_lib = None


class KryError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"kry error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_1704_02770_gb300.build.build() first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc):
    if rc != KRY_OK:
        raise KryError(rc, load().kry_last_error().decode())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _code(dtype: str) -> int:
    if dtype not in _CODES:
        raise ValueError(f"unknown dtype {dtype!r}: use one of {sorted(_CODES)}")
    return _CODES[dtype]


def _dtype_code(t, emulated: bool = False):
    import torch
    if t.dtype == torch.complex128:
        return KRY_C128E if emulated else KRY_C128
    if t.dtype == torch.complex64:
        return KRY_C64
    raise TypeError(f"unsupported dtype {t.dtype}: use complex128 or complex64")


def _dev_ptr(t, n=None, dtype=None):
    """The device address of a tensor that the library reads or writes as n elements of
    `dtype`: anything else (another element type or size, host memory, a strided view, a
    tensor of another device) is refused here, before a kernel could touch memory outside it."""
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected a {dtype} tensor, got {t.dtype}")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    import torch
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"tensor on {t.device}, but the current device is cuda:{torch.cuda.current_device()}")
    return ctypes.c_void_p(t.data_ptr())


def _host_doubles(x):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a, a.ctypes.data_as(_dp)


class Basis:
    """Sector of L sites with n_up particles (Sec. 2): split rank tables for L <= 32, the
    sorted list of Alg. 2 with combinadic ranks for L > 32 or when `list` is set."""

    def __init__(self, L: int, n_up: int, list: bool = False):
        lib = load()
        h = _vp()
        create = lib.kry_basis_create_list if list else lib.kry_basis_create
        _check(create(L, n_up, ctypes.byref(h)))
        self.list = bool(list) or L > 32
        self._h, self.L, self.n_up = h, L, n_up
        self.dim = int(lib.kry_basis_dim(h))

    def rank(self, states, stream=None):
        """Ranks (int32) of the basis states in an int64 CUDA tensor (kry_basis_rank)."""
        import torch
        ptr = _dev_ptr(states, dtype=torch.int64)
        out = torch.empty(states.numel(), dtype=torch.int32, device=states.device)
        _check(load().kry_basis_rank(self._h, ptr, _dev_ptr(out), states.numel(), _stream(stream)))
        return out

    def unrank(self, ranks, stream=None):
        """Basis states (int64) of the ranks in an int32 CUDA tensor (kry_basis_unrank)."""
        import torch
        ptr = _dev_ptr(ranks, dtype=torch.int32)
        out = torch.empty(ranks.numel(), dtype=torch.int64, device=ranks.device)
        _check(load().kry_basis_unrank(self._h, ptr, _dev_ptr(out), ranks.numel(), _stream(stream)))
        return out

    def close(self):
        if self._h:
            load().kry_basis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hamiltonian:
    """Eq. 1 (XXZ form) bound to a basis; fields h has shape [K][L] or [L]."""

    def __init__(self, basis: Basis, J: float, Delta: float, h, pbc: bool = True):
        import numpy as np
        hh = np.atleast_2d(np.asarray(h, dtype=np.float64))
        if hh.shape[1] != basis.L:
            raise ValueError("h must have L columns")
        self.K = hh.shape[0]
        arr, ptr = _host_doubles(hh.ravel())
        hnd = _vp()
        _check(load().kry_hamiltonian_set(basis._h, float(J), float(Delta), ptr, self.K,
                                          KRY_PBC if pbc else KRY_OBC, ctypes.byref(hnd)))
        self._h, self.basis, self.J, self.Delta, self.h, self.pbc = hnd, basis, J, Delta, hh, pbc
        self._ws = None   # a caller-owned workspace tensor (set_workspace)

    def apply(self, x, out=None, stream=None):
        import torch
        code = _dtype_code(x)
        n = self.basis.dim * self.K
        px = _dev_ptr(x, n)
        y = torch.empty_like(x) if out is None else out
        _check(load().kry_apply(self._h, code, px, _dev_ptr(y, n, x.dtype), _stream(stream)))
        return y

    def evolve(self, psi0, times, m: int = 30, tol: float = 1e-10, psi_out=None, emulated: bool = False,
               stream=None):
        """kry_evolve; a complex128 psi0 runs in FP64, or with `emulated` in float-float on the
        FP32 pipe (KRY_C128E)."""
        import numpy as np
        t, tp = _host_doubles(times)
        P = np.zeros(t.size * self.K)
        st = Stats()
        n = self.basis.dim * self.K
        code = _dtype_code(psi0, emulated)
        p0 = _dev_ptr(psi0, n)
        pout = _dev_ptr(psi_out, n, psi0.dtype) if psi_out is not None else None
        _check(load().kry_evolve(self._h, code, p0, tp, t.size, m, tol, pout,
                                 P.ctypes.data_as(_dp), ctypes.byref(st), _stream(stream)))
        return P.reshape(t.size, self.K) if self.K > 1 else P, st.as_dict()

    def return_probability(self, state: int, times, m: int = 30, tol: float = 1e-10,
                           dtype: str = "c128", stream=None):
        import numpy as np
        t, tp = _host_doubles(times)
        P = np.zeros(t.size * self.K)
        st = Stats()
        code = _code(dtype)
        _check(load().kry_return_probability(self._h, code, ctypes.c_uint64(state), tp, t.size, m, tol,
                                             P.ctypes.data_as(_dp), ctypes.byref(st), _stream(stream)))
        return P.reshape(t.size, self.K) if self.K > 1 else P, st.as_dict()

    def autocorrelation(self, state: int, times, m: int = 30, tol: float = 1e-10,
                        dtype: str = "c128", stream=None):
        """C(t) = (1/t) int_0^t P (Sec. 4) and P(t) at `times` from one evolution; arrays of
        shape [n_times] for K = 1, else [n_times][K]."""
        import numpy as np
        t, tp = _host_doubles(times)
        C = np.zeros(t.size * self.K)
        P = np.zeros(t.size * self.K)
        st = Stats()
        code = _code(dtype)
        _check(load().kry_autocorrelation(self._h, code, ctypes.c_uint64(state), tp, t.size, m, tol,
                                          C.ctypes.data_as(_dp), P.ctypes.data_as(_dp), ctypes.byref(st),
                                          _stream(stream)))
        if self.K > 1:
            C, P = C.reshape(t.size, self.K), P.reshape(t.size, self.K)
        return C, P, st.as_dict()

    def return_probability_states(self, states, times, m: int = 30, tol: float = 1e-10,
                                  dtype: str = "c128", autocorrelation: bool = False, stream=None):
        """P (and C when `autocorrelation`) with realisation k started from basis state
        states[k]: arrays [n_times][K] (kry_return_probability_states)."""
        import numpy as np
        s = np.ascontiguousarray(np.asarray(states, dtype=np.uint64).ravel())
        if s.size != self.K:
            raise ValueError(f"need one initial state per realisation ({self.K}), got {s.size}")
        t, tp = _host_doubles(times)
        P = np.zeros(t.size * self.K)
        C = np.zeros(t.size * self.K) if autocorrelation else None
        st = Stats()
        code = _code(dtype)
        _check(load().kry_return_probability_states(
            self._h, code, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), tp, t.size, m, tol,
            P.ctypes.data_as(_dp), C.ctypes.data_as(_dp) if C is not None else None, ctypes.byref(st),
            _stream(stream)))
        P = P.reshape(t.size, self.K)
        return (P, C.reshape(t.size, self.K), st.as_dict()) if C is not None else (P, st.as_dict())

    def autotune(self, state: int, t_probe: float, dtype: str = "c128", m: int = 30, reps: int = 2,
                 cache: str | None = None, stream=None):
        """Pick the launch shape of the vector kernels by timing probe evolutions (kry_autotune).

        Returns {"shape": [grid, hv form, dots form, update rows, batched chunk], "candidates": [[shape, ms],
        ...]}.  With `cache` (a JSON file path), a result stored for the same sector, K, dtype, m
        and GPU is reused instead of measuring, and new results are added to the file."""
        import json
        import torch
        code = _code(dtype)
        key = (f"{torch.cuda.get_device_name()}|L{self.basis.L}|N{self.basis.n_up}|K{self.K}|"
               f"{dtype}|m{m}")
        db = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                db = json.load(f)
            if key in db and "shape" in db[key]:
                self.set_shape(db[key]["shape"], dtype)
                return db[key]
        nmax = 16
        shp = (ctypes.c_int * 5)()
        cand = (ctypes.c_int * (5 * nmax))()
        ms = (ctypes.c_double * nmax)()
        n = ctypes.c_int(0)
        _check(load().kry_autotune(self._h, code, m, ctypes.c_uint64(state), float(t_probe), reps,
                                   shp, cand, ms, nmax, ctypes.byref(n), _stream(stream)))
        res = {"shape": list(shp), "candidates": [[list(cand[5 * i:5 * i + 5]), float(ms[i])]
                                                  for i in range(n.value)]}
        if cache:
            db[key] = res
            with open(cache, "w") as f:
                json.dump(db, f, indent=1)
        return res

    def set_shape(self, shape, dtype: str = "c128"):
        """Launch shape [grid, hv form, dots form, update rows, batched chunk] (kry_set_shape)."""
        arr = (ctypes.c_int * 5)(*[int(x) for x in shape])
        _check(load().kry_set_shape(self._h, _code(dtype), arr))

    def get_shape(self, dtype: str = "c128"):
        arr = (ctypes.c_int * 5)()
        _check(load().kry_get_shape(self._h, _code(dtype), arr))
        return list(arr)

    def orth_check(self, on=True):
        """Measure (and subtract when needed) <v_i, w> after every Lanczos update; on = 2
        subtracts them after every update (kry_set_orth_check)."""
        _check(load().kry_set_orth_check(self._h, int(on)))

    def second_pass_node(self, on=True):
        """Launch the second Gram-Schmidt pass through a conditional graph node (True) or as
        kernels that return at once unless needed (False, the default)
        (kry_set_second_pass_node)."""
        _check(load().kry_set_second_pass_node(self._h, int(on)))

    def set_grid(self, grid: int, dtype: str = "c128"):
        _check(load().kry_set_grid(self._h, _code(dtype), grid))

    def grad(self, state: int, t: float, m: int = 30, tol: float = 1e-10, ckpt_every: int = 8,
             stream=None):
        """P(t) and its gradient: returns (P, dP/dh [L], dP/dDelta, stats)."""
        import numpy as np
        P = np.zeros(1)
        gh = np.zeros(self.basis.L)
        gd = np.zeros(1)
        st = Stats()
        _check(load().kry_grad(self._h, ctypes.c_uint64(state), float(t), m, tol, ckpt_every,
                               P.ctypes.data_as(_dp), gh.ctypes.data_as(_dp), gd.ctypes.data_as(_dp),
                               ctypes.byref(st), _stream(stream)))
        return float(P[0]), gh, float(gd[0]), st.as_dict()

    def profile(self, on=True):
        """Turn per-kernel CUDA-event profiling of later evolutions on or off (resets it); on = 2
        builds the step graph without conditional nodes, for external profilers
        (kry_profile_enable)."""
        _check(load().kry_profile_enable(self._h, int(on)))

    # pass A's dots, pass B's update, pass C, the small exponential, the combine, pass A's H.v
    KINDS = ("dots", "update", "passC", "smallexp", "combine", "hv")

    def profile_read(self):
        import numpy as np
        ms, by = np.zeros(6), np.zeros(6)
        n = (ctypes.c_int64 * 6)()
        _check(load().kry_profile_read(self._h, ms.ctypes.data_as(_dp), by.ctypes.data_as(_dp), n))
        return {k: dict(ms=float(ms[i]), bytes=float(by[i]), launches=int(n[i]))
                for i, k in enumerate(self.KINDS)}

    def workspace_size(self, dtype: str = "c128", m: int = 30, n_times: int = 1) -> int:
        return int(load().kry_workspace_bytes(self._h, _code(dtype), m, n_times))

    def set_workspace(self, buf=None):
        """Use a caller-owned device buffer (a CUDA tensor, kept referenced here) as the evolution
        workspace, or None to return to library-managed memory (kry_set_workspace)."""
        if buf is None:
            _check(load().kry_set_workspace(self._h, None, 0))
            self._ws = None
            return
        ptr = _dev_ptr(buf)
        nbytes = buf.numel() * buf.element_size()
        _check(load().kry_set_workspace(self._h, ptr, nbytes))
        self._ws = buf

    def close(self):
        if self._h:
            load().kry_hamiltonian_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tridiag_expv(alpha, beta, h: float, tau: float, stream=None):
    """Device small exponential: returns (y = exp(-i tau T) e_1, err estimate)."""
    import numpy as np
    a, ap = _host_doubles(alpha)
    b, bp = _host_doubles(beta if len(beta) else [0.0])
    y = np.zeros(2 * a.size)
    err = np.zeros(1)
    _check(load().kry_tridiag_expv(ap, bp, a.size, float(h), float(tau), y.ctypes.data_as(_dp),
                                   err.ctypes.data_as(_dp), _stream(stream)))
    return y[0::2] + 1j * y[1::2], float(err[0])


def measure_peaks(stream=None):
    """(FP64, FP32) fused multiply-add throughput of the current GPU in TFLOP/s (kry_measure_peaks)."""
    f64, f32 = ctypes.c_double(), ctypes.c_double()
    _check(load().kry_measure_peaks(ctypes.byref(f64), ctypes.byref(f32), _stream(stream)))
    return f64.value, f32.value


def decay_exponent(times, C, t_min: float, t_max: float):
    """(gamma, log a) of the fit C(t) ~ a t^-gamma over t_min <= t <= t_max (kry_decay_exponent)."""
    t, tp = _host_doubles(times)
    c, cp = _host_doubles(C)
    if c.size != t.size:
        raise ValueError("times and C differ in length")
    g, la = ctypes.c_double(), ctypes.c_double()
    _check(load().kry_decay_exponent(tp, cp, t.size, float(t_min), float(t_max), ctypes.byref(g), ctypes.byref(la)))
    return g.value, la.value


def _return_probability_fn():
    import torch

    class ReturnProbability(torch.autograd.Function):
        """P(t) = |<psi0| exp(-iHt) |psi0>|^2 as a differentiable function of the on-site
        fields h [L] and of Delta (float64 tensors on any device; the values are read on the
        host).  When a gradient is wanted, forward runs kry_grad on the GPU (P and the adjoint
        (costate) evolution) and backward returns grad_output * dP/dh and grad_output *
        dP/dDelta on the inputs' devices; otherwise forward runs only the evolution of P."""

        @staticmethod
        def forward(ctx, h, Delta, basis, J, state, t, pbc, m, tol, ckpt_every, want_grad):
            H = Hamiltonian(basis, float(J), float(Delta.item()), h.detach().cpu().numpy(), pbc=pbc)
            try:
                if want_grad:
                    P, gh, gd, _ = H.grad(state, t, m=m, tol=tol, ckpt_every=ckpt_every)
                    ctx.save_for_backward(torch.from_numpy(gh).to(h.device),
                                          torch.tensor(gd, dtype=torch.float64, device=Delta.device))
                else:
                    Pv, _ = H.return_probability(state, [t], m=m, tol=tol)
                    P = float(Pv[0])
            finally:
                H.close()
            return torch.tensor(P, dtype=torch.float64, device=h.device)

        @staticmethod
        def backward(ctx, g):
            gh, gd = ctx.saved_tensors
            return g.to(gh.device) * gh, g.to(gd.device) * gd, None, None, None, None, None, None, None, None, None

    return ReturnProbability


def return_probability(h, Delta, basis, J, state, t, pbc=True, m=30, tol=1e-10, ckpt_every=8):
    """Differentiable P(t): h a float64 tensor [L], Delta a float64 scalar tensor.  The adjoint
    runs only when grad mode is on and h or Delta requires a gradient."""
    import torch
    want = torch.is_grad_enabled() and (h.requires_grad or Delta.requires_grad)
    return _return_probability_fn().apply(h, Delta, basis, J, state, t, pbc, m, tol, ckpt_every, want)
