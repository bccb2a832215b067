"""Thin Python binding of libewald.so (argument marshalling only).

Every numerical step runs in the library's CUDA kernels; this module only passes device
pointers (``torch.Tensor.data_ptr()``), sizes and the current CUDA stream across the C ABI
declared in ``include/ewald.h``, and turns status codes into exceptions.  The library is
loaded from the package directory; if it is missing, every call raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libewald.so")

FP64, MIXED, MIXED_BF16, FP32 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "mixed": MIXED, "mixed_bf16": MIXED_BF16, "fp32": FP32}
PART_REAL, PART_RECIP, PART_SELF, PART_ALL = 1, 2, 4, 7
MD_RECORD = 6      # E_real, E_recip, E_self, E_pot, E_kin, E_total per ewald_md record

OK, PENDING = 0, 1
E_INVAL, E_NONNEUTRAL, E_CUTOFF, E_NOMEM, E_CUDA = -1, -2, -3, -4, -5
E_TIMEOUT, E_BUSY, E_NOTFOUND, E_NONFINITE, E_UNSUPPORTED = -6, -7, -8, -9, -10

_lock = threading.Lock()
_lib = None

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_d = ctypes.c_double
_i = ctypes.c_int


class EwaldError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


class _Request(ctypes.Structure):
    _fields_ = [("L", _d), ("beta", _d), ("r_c", _d), ("k_max", _i), ("precision", _i),
                ("n", _i64), ("pos", _p), ("q", _p), ("forces", _p), ("stream", _p)]


class _Result(ctypes.Structure):
    _fields_ = [("status", _i), ("energy", _d * 4), ("t_submit", _d), ("t_admit", _d),
                ("t_done", _d), ("footprint_bytes", _i64)]


def lib() -> ctypes.CDLL:
    """Load libewald.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_1708_01135_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            sig = {
                "ewald_create": (_i, [_d, _d, _d, _i, _i, ctypes.POINTER(_p)]),
                "ewald_destroy": (None, [_p]),
                "ewald_compute": (_i, [_p, _i64, _p, _p, _p, _p, _p]),
                "ewald_compute_async": (_i, [_p, _i64, _p, _p, _p, _p, _i, _p]),
                "ewald_compute_phi_async": (_i, [_p, _i64, _p, _p, _p, _p, _p, _i, _p]),
                "ewald_compute_virial_async": (_i, [_p, _i64, _p, _p, _p, _p, _p, _i, _p]),
                "ewald_set_lj": (_i, [_p, _i, _p, _p, _p]),
                "ewald_set_spme": (_i, [_p, _i, _i]),
                "ewald_set_near_pairs": (_i, [_p, _i]),
                "ewald_probe_timeout": (_i, [_p, _p]),
                "ewald_status_sync": (_i, [_p]),
                "ewald_compute_host": (_i, [_p, _i64, _p, _p, _p, _p, _p]),
                "ewald_plan_info": (_i, [_p, _p]),
                "ewald_profile": (_i, [_p, _i, _p, ctypes.POINTER(_i)]),
                "ewald_kset": (_i, [_p, _p, _i64, ctypes.POINTER(_i64)]),
                "ewald_structure_factor": (_i, [_p, _p, _p]),
                "ewald_cell_sort": (_i, [_p, _p, _p, _p]),
                "ewald_tune": (_i, [_i64, _d, _d, ctypes.POINTER(_d), ctypes.POINTER(_d),
                                    ctypes.POINTER(_i)]),
                "ewald_strerror": (ctypes.c_char_p, [_i]),
                "ewald_server_create": (_i, [_i, ctypes.c_size_t, ctypes.POINTER(_p)]),
                "ewald_submit": (_i, [_p, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)]),
                "ewald_poll": (_i, [_p, ctypes.c_uint64, ctypes.POINTER(_Result)]),
                "ewald_wait": (_i, [_p, ctypes.c_uint64, _d, ctypes.POINTER(_Result)]),
                "ewald_server_stats": (_i, [_p, _p]),
                "ewald_server_destroy": (_i, [_p]),
                "ewald_server_simulate": (_i, [_i, _i64, _i, _p, _p, _p, _p, _p,
                                               ctypes.POINTER(_i64)]),
                "ewald_real_noalloc": (_i, [_d, _d, _d, _i64, _p, _p, _p, _p, _p]),
                "ewald_md": (_i, [_p, _i64, _p, _p, _p, _p, _d, _i, _p, _p, _p]),
                "ewald_fma_peak": (_i, [_i, ctypes.POINTER(_d)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def simulate_admission(max_slots: int, budget: int, footprint, t_arrive, duration):
    """Replay of the server's admission policy on the host (ewald_server_simulate): returns
    (admission order, admission times, peak held bytes)."""
    fp = np.ascontiguousarray(footprint, dtype=np.int64)
    ta = np.ascontiguousarray(t_arrive, dtype=np.float64)
    du = np.ascontiguousarray(duration, dtype=np.float64)
    n = len(fp)
    order = np.zeros(n, dtype=np.int64)
    tad = np.zeros(n, dtype=np.float64)
    peak = _i64(0)
    _check(lib().ewald_server_simulate(int(max_slots), int(budget), n, fp.ctypes.data,
                                       ta.ctypes.data, du.ctypes.data, order.ctypes.data,
                                       tad.ctypes.data, ctypes.byref(peak)),
           "ewald_server_simulate")
    return order, tad, peak.value


def strerror(status: int) -> str:
    return lib().ewald_strerror(int(status)).decode()


def _check(status: int, what: str) -> int:
    if status != OK:
        raise EwaldError(status, what)
    return status


def _stream_handle(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def _dev_f64(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {tuple(shape)}")
    return t.data_ptr()


def tune(n: int, L: float, tol: float = 1e-6, r_c: float | None = None):
    """(r_c, beta, k_max) for a target relative RMS force error (ewald_tune)."""
    rc = _d(r_c if r_c else 0.0)
    beta = _d(0.0)
    km = _i(0)
    _check(lib().ewald_tune(int(n), float(L), float(tol), ctypes.byref(rc), ctypes.byref(beta),
                            ctypes.byref(km)), "ewald_tune")
    return rc.value, beta.value, km.value


NOALLOC_MAX_N = 16384
PROFILE_TIMES = 11          # entries of ewald_profile's times (EWALD_PROFILE_TIMES)


def fma_peak(precision: str = "fp32") -> float:
    """Measured CUDA-core FMA rate of the current device in TFLOP/s (ewald_fma_peak):
    precision 'fp32' or 'fp64'."""
    code = {"fp32": FP32, "fp64": FP64}[precision]
    out = _d(0.0)
    _check(lib().ewald_fma_peak(code, ctypes.byref(out)), "ewald_fma_peak")
    return out.value


def real_noalloc(L, beta, r_c, pos, q, forces, energy, stream=None):
    """Real-space part without any device allocation (ewald_real_noalloc): for callers that
    cannot allocate (stream capture, foreign allocators, allocation-free loops).  pos [n,3],
    q [n], forces [n,3], energy [4] are CUDA float64 tensors; n <= NOALLOC_MAX_N."""
    n = int(q.shape[0])
    _check(lib().ewald_real_noalloc(float(L), float(beta), float(r_c), n, _dev_f64(pos, (n, 3), "pos"),
                                    _dev_f64(q, (n,), "q"), _dev_f64(forces, (n, 3), "forces"),
                                    _dev_f64(energy, (4,), "energy"), _stream_handle(stream)),
           "ewald_real_noalloc")


class Ewald:
    """A plan: box side L, splitting parameter beta (the paper's alpha is beta^2), cutoff r_c,
    integer reciprocal cutoff k_max and a precision mode (fp64, mixed, mixed_bf16, fp32)."""

    def __init__(self, L: float, beta: float, r_c: float, k_max: int, precision="fp64"):
        self.L, self.beta, self.r_c, self.k_max = float(L), float(beta), float(r_c), int(k_max)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = _p()
        _check(lib().ewald_create(self.L, self.beta, self.r_c, self.k_max, self.precision,
                                  ctypes.byref(h)), "ewald_create")
        self._h = h

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            lib().ewald_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- evaluation --
    def compute(self, pos, q, forces=None, stream=None):
        """Synchronous evaluation on device tensors: returns (forces [n,3], energy float64[4]:
        real, reciprocal, self, total)."""
        import torch
        n = int(q.shape[0])
        if forces is None:
            forces = torch.empty((n, 3), dtype=torch.float64, device=q.device)
        e = (ctypes.c_double * 4)()
        _check(lib().ewald_compute(self._h, n, _dev_f64(pos, (n, 3), "pos"), _dev_f64(q, (n,), "q"),
                                   _dev_f64(forces, (n, 3), "forces"), e, _stream_handle(stream)),
               "ewald_compute")
        return forces, np.array(list(e))

    def compute_async(self, pos, q, forces, energy, parts=PART_ALL, stream=None):
        """Asynchronous evaluation into device tensors forces [n,3] and energy [4]."""
        n = int(q.shape[0])
        _check(lib().ewald_compute_async(self._h, n, _dev_f64(pos, (n, 3), "pos"),
                                         _dev_f64(q, (n,), "q"), _dev_f64(forces, (n, 3), "forces"),
                                         _dev_f64(energy, (4,), "energy"), int(parts),
                                         _stream_handle(stream)), "ewald_compute_async")

    def md(self, pos, vel, q, forces, dt: float, steps: int, mass=None, log=None, stream=None):
        """Velocity-Verlet MD (ewald_md), asynchronous on the stream: pos and vel [n,3] are
        advanced in place, forces [n,3] ends with the forces at the final positions, and log
        (None or [steps + 1, 6]: E_real, E_recip, E_self, E_pot, E_kin, E_total per step,
        record 0 the initial state) is filled on the device.  mass: None (unit masses) or [n].
        Call status() for the device-side validation of the run."""
        n = int(q.shape[0])
        _check(lib().ewald_md(self._h, n, _dev_f64(pos, (n, 3), "pos"), _dev_f64(vel, (n, 3), "vel"),
                              _dev_f64(q, (n,), "q"),
                              None if mass is None else _dev_f64(mass, (n,), "mass"),
                              float(dt), int(steps), _dev_f64(forces, (n, 3), "forces"),
                              None if log is None else _dev_f64(log, (int(steps) + 1, MD_RECORD), "log"),
                              _stream_handle(stream)), "ewald_md")

    def compute_phi_async(self, pos, q, forces, phi, energy, parts=PART_ALL, stream=None):
        """Asynchronous evaluation into device tensors forces [n,3], phi [n] (the potential at
        every particle, so that E = 1/2 sum q_i phi_i) and energy [4]."""
        n = int(q.shape[0])
        _check(lib().ewald_compute_phi_async(self._h, n, _dev_f64(pos, (n, 3), "pos"),
                                             _dev_f64(q, (n,), "q"), _dev_f64(forces, (n, 3), "forces"),
                                             _dev_f64(phi, (n,), "phi"), _dev_f64(energy, (4,), "energy"),
                                             int(parts), _stream_handle(stream)), "ewald_compute_phi_async")

    def compute_virial_async(self, pos, q, forces, virial, energy, parts=PART_ALL, stream=None):
        """Asynchronous evaluation into device tensors forces [n,3], virial [4,3,3] (the real,
        reciprocal and self virial tensors W_ab = -dE/d(eps_ab) and their sum) and energy [4]."""
        n = int(q.shape[0])
        _check(lib().ewald_compute_virial_async(self._h, n, _dev_f64(pos, (n, 3), "pos"),
                                                _dev_f64(q, (n,), "q"), _dev_f64(forces, (n, 3), "forces"),
                                                _dev_f64(virial, (4, 3, 3), "virial"),
                                                _dev_f64(energy, (4,), "energy"), int(parts),
                                                _stream_handle(stream)), "ewald_compute_virial_async")

    def set_lj(self, epsilon=None, sigma=None, types=None):
        """Fuse truncated and shifted Lennard-Jones pairs into the real-space kernel
        (ewald_set_lj): epsilon and sigma symmetric [T, T] host arrays, types a CUDA int32
        tensor [n] in particle order that must stay alive while the plan uses it.  No
        arguments: switch the pairs off."""
        import torch
        if epsilon is None:
            _check(lib().ewald_set_lj(self._h, 0, None, None, None), "ewald_set_lj")
            self._lj_types = None
            return
        eps = np.ascontiguousarray(epsilon, dtype=np.float64)
        sig = np.ascontiguousarray(sigma, dtype=np.float64)
        if eps.ndim != 2 or eps.shape[0] != eps.shape[1] or sig.shape != eps.shape:
            raise ValueError("epsilon and sigma must be square tables of one shape")
        if not isinstance(types, torch.Tensor) or not types.is_cuda or types.dtype != torch.int32 \
                or not types.is_contiguous():
            raise TypeError("types must be a contiguous CUDA int32 tensor")
        _check(lib().ewald_set_lj(self._h, int(eps.shape[0]), eps.ctypes.data, sig.ctypes.data,
                                  types.data_ptr()), "ewald_set_lj")
        self._lj_types = types      # keep the caller's tensor alive with the plan

    def set_spme(self, K: int = 0, order: int = 6):
        """Reciprocal part by smooth particle-mesh Ewald on a K^3 mesh with B-splines of the
        given even order (ewald_set_spme); K = 0 returns to the classical k-space sum."""
        _check(lib().ewald_set_spme(self._h, int(K), int(order)), "ewald_set_spme")

    def set_near_pairs(self, double_float: bool):
        """Near real-space Coulomb pairs (within a few mean spacings) in double-float
        arithmetic (True) or FP32 with the exact r^2 (False, the default)
        (ewald_set_near_pairs)."""
        _check(lib().ewald_set_near_pairs(self._h, 1 if double_float else 0),
               "ewald_set_near_pairs")

    def probe_timeout(self, stream=None):
        """One device wait that cannot complete (ewald_probe_timeout): the next status() is
        the timeout status, about one second later."""
        _check(lib().ewald_probe_timeout(self._h, _stream_handle(stream)), "ewald_probe_timeout")

    def status(self) -> int:
        """Synchronise and return the device-side status of the last evaluation."""
        return int(lib().ewald_status_sync(self._h))

    def compute_host(self, pos: np.ndarray, q: np.ndarray, forces: np.ndarray | None = None,
                     stream=None):
        """End-to-end evaluation from host arrays (copies inside the call)."""
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        n = len(q)
        if forces is None:
            forces = np.empty((n, 3), dtype=np.float64)
        e = (ctypes.c_double * 4)()
        _check(lib().ewald_compute_host(self._h, n, pos.ctypes.data, q.ctypes.data,
                                        forces.ctypes.data, e, _stream_handle(stream)),
               "ewald_compute_host")
        return forces, np.array(list(e))

    # -- profiling --
    def profile(self, enable: int = -1):
        """Stage times (ms) of the last recorded evaluation and its kernel launch count.
        enable: 1 start recording, 0 stop, -1 leave as is."""
        t = np.zeros(PROFILE_TIMES)
        nl = _i(0)
        _check(lib().ewald_profile(self._h, int(enable), t.ctypes.data, ctypes.byref(nl)),
               "ewald_profile")
        names = ["binning", "to_real_end", "recip_forward", "recip_coef", "recip_back",
                 "real_end_to_end", "total", "recip_branch", "real_kernel", "backscatter_kernel",
                 "finalize_kernels"]
        return dict(zip(names, t.tolist())), nl.value

    # -- introspection --
    def info(self) -> dict:
        a = np.zeros(6, dtype=np.int64)
        _check(lib().ewald_plan_info(self._h, a.ctypes.data), "ewald_plan_info")
        return dict(cells_per_side=int(a[0]), stencil=int(a[1]), nk=int(a[2]), rows=int(a[3]),
                    k_max=int(a[4]), precision=int(a[5]))

    def kset(self) -> np.ndarray:
        cnt = _i64(0)
        _check(lib().ewald_kset(self._h, None, 0, ctypes.byref(cnt)), "ewald_kset")
        m = np.zeros((cnt.value, 3), dtype=np.int32)
        _check(lib().ewald_kset(self._h, m.ctypes.data, cnt.value, ctypes.byref(cnt)), "ewald_kset")
        return m

    def structure_factor(self, stream=None):
        """S(k) of the last evaluation (complex128 numpy, kset() order)."""
        import torch
        nk = self.info()["nk"]
        S = torch.empty((nk, 2), dtype=torch.float64, device="cuda")
        _check(lib().ewald_structure_factor(self._h, S.data_ptr(), _stream_handle(stream)),
               "ewald_structure_factor")
        torch.cuda.synchronize()
        s = S.cpu().numpy()
        return s[:, 0] + 1j * s[:, 1]

    def cell_sort(self, n: int, stream=None):
        """(key [n], perm [n]) int32 numpy views of the last binning."""
        import torch
        key = torch.empty(n, dtype=torch.int32, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        _check(lib().ewald_cell_sort(self._h, key.data_ptr(), perm.data_ptr(), _stream_handle(stream)),
               "ewald_cell_sort")
        torch.cuda.synchronize()
        return key.cpu().numpy(), perm.cpu().numpy()


class Server:
    """Continuous-batching server (ewald_server_*): submit independent systems, poll results."""

    def __init__(self, max_slots: int = 8, hbm_budget_bytes: int = 0):
        h = _p()
        _check(lib().ewald_server_create(int(max_slots), int(hbm_budget_bytes), ctypes.byref(h)),
               "ewald_server_create")
        self._h = h
        self._keep = {}

    def submit(self, pos, q, forces, L, beta, r_c, k_max, precision="mixed", stream=None) -> int:
        n = int(q.shape[0])
        req = _Request(float(L), float(beta), float(r_c), int(k_max),
                       PRECISIONS[precision] if isinstance(precision, str) else int(precision), n,
                       _dev_f64(pos, (n, 3), "pos"), _dev_f64(q, (n,), "q"),
                       _dev_f64(forces, (n, 3), "forces"), _stream_handle(stream))
        t = ctypes.c_uint64(0)
        _check(lib().ewald_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "ewald_submit")
        self._keep[t.value] = (pos, q, forces)
        return t.value

    def _result(self, r: _Result):
        return dict(status=r.status, energy=np.array(list(r.energy)), t_submit=r.t_submit,
                    t_admit=r.t_admit, t_done=r.t_done, footprint_bytes=r.footprint_bytes)

    def poll(self, ticket: int):
        r = _Result()
        s = lib().ewald_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(r))
        if s == PENDING:
            return None
        _check(s, "ewald_poll")
        self._keep.pop(ticket, None)
        return self._result(r)

    def wait(self, ticket: int, timeout_s: float = 60.0):
        r = _Result()
        _check(lib().ewald_wait(self._h, ctypes.c_uint64(ticket), float(timeout_s), ctypes.byref(r)),
               "ewald_wait")
        self._keep.pop(ticket, None)
        return self._result(r)

    def stats(self) -> dict:
        a = np.zeros(5, dtype=np.int64)
        _check(lib().ewald_server_stats(self._h, a.ctypes.data), "ewald_server_stats")
        return dict(submitted=int(a[0]), completed=int(a[1]), admitted_bytes=int(a[2]),
                    peak_admitted_bytes=int(a[3]), peak_concurrent=int(a[4]))

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().ewald_server_destroy(self._h), "ewald_server_destroy")
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
