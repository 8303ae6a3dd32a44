"""Thin ctypes binding of libqcd (include/qcd.h), argument marshalling only.

Every operation runs in the CUDA library; this module only converts Python
arguments (numpy arrays, torch tensors, enums, streams) into the C ABI's
plain pointers and sizes, and raises ``QcdError`` on a non-zero status.
The library must be built first (``__graft_entry__.build()``): importing
the binding on a machine where ``libqcd.so`` is missing raises at the first
call, there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqcd.so")

PREC = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3, "df64": 4}
PARITY = {"even": 0, "odd": 1, "full": 2}
STATUS = {0: "QCD_OK", 1: "QCD_ERR_INVALID_ARG", 2: "QCD_ERR_OOM", 3: "QCD_ERR_CUDA",
          4: "QCD_ERR_NOT_CONVERGED", 5: "QCD_ERR_BREAKDOWN", 6: "QCD_ERR_TIMEOUT",
          7: "QCD_ERR_CANCELLED"}

_p = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


class SolverParams(ctypes.Structure):
    _fields_ = [("kappa", _d), ("mu", _d), ("tol", _d), ("maxiter", _i), ("eo", _i), ("normal", _i),
                ("inner_prec", _i), ("inner_recon", _i), ("reliable_delta", _d)]


class SolverStats(ctypes.Structure):
    _fields_ = [("iterations", _i), ("reliable_updates", _i), ("true_rel_residual", _d),
                ("full_rel_residual", _d), ("seconds", _d)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", _d), ("bytes", _d), ("flops", _d), ("sites", _d)]


class Profile(ctypes.Structure):
    _fields_ = [("prec", ProfileEntry * 5)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", _i), ("memory_budget", ctypes.c_size_t), ("batch_small_sites", _i)]


class Request(ctypes.Structure):
    _fields_ = [("gauge_id", _i), ("kappa", _d), ("mu", _d), ("tol", _d), ("maxiter", _i), ("inner_prec", _i),
                ("inner_recon", _i), ("reliable_delta", _d), ("b_host", _p), ("x_host", _p)]


class RequestResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", _i), ("slot", _i), ("stats", SolverStats),
                ("t_submit", _d), ("t_start", _d), ("t_end", _d)]


# name -> (restype, argtypes); mirrors include/qcd.h
_SIGS = {
    "qcd_status_string": (ctypes.c_char_p, [_i]),
    "qcd_last_error": (ctypes.c_char_p, []),
    "qcd_version": (ctypes.c_char_p, []),
    "qcd_stream_sync": (_i, [_p]),
    "qcd_lattice_create": (_i, [ctypes.POINTER(_i), _i, ctypes.POINTER(_p)]),
    "qcd_lattice_destroy": (None, [_p]),
    "qcd_gauge_create": (_i, [_p, _i, _i, ctypes.POINTER(_p)]),
    "qcd_gauge_upload": (_i, [_p, _p, _p]),
    "qcd_gauge_prepare": (_i, [_p, _i, _i, _p]),
    "qcd_gauge_destroy": (None, [_p]),
    "qcd_spinor_create": (_i, [_p, _i, _i, ctypes.POINTER(_p)]),
    "qcd_spinor_create_ks": (_i, [_p, _i, _i, ctypes.POINTER(_p)]),
    "qcd_apply_dslash_ks": (_i, [_p, _p, _p, _p]),
    "qcd_spinor_bytes": (_i, [_p, _i, _i, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "qcd_spinor_wrap_device": (_i, [_p, _i, _i, _p, _p, ctypes.POINTER(_p)]),
    "qcd_spinor_upload": (_i, [_p, _p, _p]),
    "qcd_spinor_download": (_i, [_p, _p, _p]),
    "qcd_spinor_zero": (_i, [_p, _p]),
    "qcd_spinor_convert": (_i, [_p, _p, _p]),
    "qcd_spinor_norm2": (_i, [_p, _p, _p]),
    "qcd_spinor_destroy": (None, [_p]),
    "qcd_apply_dslash": (_i, [_p, _p, _p, _i, _p]),
    "qcd_apply_M": (_i, [_p, _p, _p, _d, _d, _i, _i, _p]),
    "qcd_solve_cg": (_i, [_p, _p, _p, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats), _p]),
    "qcd_profile_begin": (_i, []),
    "qcd_profile_end": (_i, [ctypes.POINTER(Profile)]),
    "qcd_kernel_launches": (ctypes.c_ulonglong, []),
    "qcd_debug_inject": (_i, [_i, _i]),
    "qcd_set_hop_threads": (_i, [_i]),
    "qcd_norm2_noalloc": (_i, [_p, ctypes.c_size_t, _p, _p]),
    "qcd_server_create": (_i, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_p)]),
    "qcd_server_add_gauge": (_i, [_p, _p, ctypes.POINTER(_i)]),
    "qcd_server_submit": (_i, [_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_longlong)]),
    "qcd_server_wait": (_i, [_p, ctypes.c_longlong, ctypes.POINTER(RequestResult)]),
    "qcd_server_info": (_i, [_p, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "qcd_server_destroy": (None, [_p]),
    "qcd_apply_dslash_multi": (_i, [_p, ctypes.POINTER(_p), ctypes.POINTER(_p), _i, _i, _p]),
    "qcd_solve_cg_multi": (_i, [_p, ctypes.POINTER(_p), ctypes.POINTER(_p), _i, ctypes.POINTER(SolverParams),
                                ctypes.POINTER(SolverStats), _p]),
    "qcd_face_pack": (_i, [_p, _p, _i, _i, ctypes.c_double, _p, _p]),
    "qcd_face_unpack": (_i, [_p, _i, _p, _p]),
    "qcd_solve_cg_many": (_i, [_i, ctypes.POINTER(_p), ctypes.POINTER(_p), ctypes.POINTER(_p),
                               ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats), ctypes.c_longlong, _i,
                               _p]),
    "qcd_solve_cg_batch": (_i, [_p, ctypes.POINTER(_p), ctypes.POINTER(_p), _i, ctypes.POINTER(SolverParams),
                                ctypes.POINTER(SolverStats), _p]),
}

_lib = None


class QcdError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")
        self.status = status


def lib():
    """Load libqcd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        l = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise QcdError(status, where, lib().qcd_last_error().decode())


def _stream(stream):
    """cudaStream_t handle: an int, a torch stream, or torch's current stream."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return _p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return _p(0)
    if isinstance(stream, int):
        return _p(stream)
    return _p(stream.cuda_stream)


def _host_ptr(a, dtype=np.complex128):
    """Pointer of a host buffer: numpy array or (pinned) CPU torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host array must be C-contiguous complex128")
        return _p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("host tensor must be a contiguous CPU tensor")
        return _p(a.data_ptr())
    raise TypeError("expected a numpy array or a CPU torch tensor")


def stream_sync(stream=None):
    _check(lib().qcd_stream_sync(_stream(stream)), "qcd_stream_sync")


class Lattice:
    """qcd_lattice: extents (Lx, Ly, Lz, Lt), time boundary t_bc = +1 or -1."""

    def __init__(self, dims, t_bc: int = -1):
        self.dims = tuple(int(d) for d in dims)
        self.t_bc = int(t_bc)
        h = _p()
        _check(lib().qcd_lattice_create((_i * 4)(*self.dims), self.t_bc, ctypes.byref(h)), "qcd_lattice_create")
        self._h = h
        self.volume = int(np.prod(self.dims))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().qcd_lattice_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


class Gauge:
    """qcd_gauge in precision `prec` with `recon` reals per link."""

    def __init__(self, lat: Lattice, prec: str = "f64", recon: int = 18):
        self.lat, self.prec, self.recon = lat, prec, int(recon)
        h = _p()
        _check(lib().qcd_gauge_create(lat.handle, PREC[prec], self.recon, ctypes.byref(h)), "qcd_gauge_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def upload(self, U, stream=None):
        """U: host field [t,z,y,x,mu,3,3] complex128."""
        if hasattr(U, "shape") and tuple(U.shape[:4]) != self.lat.dims[::-1]:
            raise ValueError("gauge field shape does not match the lattice")
        _check(lib().qcd_gauge_upload(self._h, _host_ptr(U), _stream(stream)), "qcd_gauge_upload")

    def prepare(self, prec: str, recon: int, stream=None):
        _check(lib().qcd_gauge_prepare(self._h, PREC[prec], int(recon), _stream(stream)), "qcd_gauge_prepare")

    def close(self):
        if getattr(self, "_h", None):
            lib().qcd_gauge_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


class Spinor:
    """qcd_spinor on parity 'even', 'odd' or 'full' in precision `prec`.

    With ``torch_alloc=True`` the device memory is a torch tensor wrapped
    through qcd_spinor_wrap_device (torch's allocator owns it)."""

    def __init__(self, lat: Lattice, parity: str = "full", prec: str = "f64", torch_alloc: bool = False,
                 ks: bool = False):
        self.lat, self.parity, self.prec, self.ks = lat, parity, prec, bool(ks)
        h = _p()
        self._buffers = None
        if ks:
            _check(lib().qcd_spinor_create_ks(lat.handle, PARITY[parity], PREC[prec], ctypes.byref(h)),
                   "qcd_spinor_create_ks")
        elif torch_alloc:
            import torch
            nd, nn = ctypes.c_size_t(), ctypes.c_size_t()
            _check(lib().qcd_spinor_bytes(lat.handle, PARITY[parity], PREC[prec], ctypes.byref(nd),
                                          ctypes.byref(nn)), "qcd_spinor_bytes")
            data = torch.zeros(nd.value, dtype=torch.uint8, device="cuda")
            norm = torch.zeros(max(nn.value, 1), dtype=torch.uint8, device="cuda")
            self._buffers = (data, norm)
            _check(lib().qcd_spinor_wrap_device(lat.handle, PARITY[parity], PREC[prec], _p(data.data_ptr()),
                                                _p(norm.data_ptr()), ctypes.byref(h)), "qcd_spinor_wrap_device")
        else:
            _check(lib().qcd_spinor_create(lat.handle, PARITY[parity], PREC[prec], ctypes.byref(h)),
                   "qcd_spinor_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def host_shape(self):
        lx, ly, lz, lt = self.lat.dims
        inner = (3,) if self.ks else (4, 3)
        if self.parity == "full":
            return (lt, lz, ly, lx) + inner
        return (self.lat.volume // 2,) + inner

    def upload(self, psi, stream=None):
        if tuple(psi.shape) != self.host_shape:
            raise ValueError(f"host spinor shape {tuple(psi.shape)} != {self.host_shape}")
        _check(lib().qcd_spinor_upload(self._h, _host_ptr(psi), _stream(stream)), "qcd_spinor_upload")

    def download(self, out=None, stream=None, sync=True):
        if out is None:
            out = np.empty(self.host_shape, dtype=np.complex128)
        _check(lib().qcd_spinor_download(self._h, _host_ptr(out), _stream(stream)), "qcd_spinor_download")
        if sync:
            stream_sync(stream)
        return out

    def zero(self, stream=None):
        _check(lib().qcd_spinor_zero(self._h, _stream(stream)), "qcd_spinor_zero")

    def convert_from(self, src: "Spinor", stream=None):
        _check(lib().qcd_spinor_convert(self._h, src.handle, _stream(stream)), "qcd_spinor_convert")

    def norm2(self, stream=None) -> float:
        import torch
        res = torch.zeros(1, dtype=torch.float64, device="cuda")
        _check(lib().qcd_spinor_norm2(self._h, _p(res.data_ptr()), _stream(stream)), "qcd_spinor_norm2")
        stream_sync(stream)
        return float(res.cpu()[0])

    def close(self):
        if getattr(self, "_h", None):
            lib().qcd_spinor_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def apply_dslash(gauge: Gauge, out: Spinor, inp: Spinor, dagger: bool = False, stream=None):
    """out = D_hop inp (parity block or full lattice); see qcd_apply_dslash."""
    _check(lib().qcd_apply_dslash(gauge.handle, out.handle, inp.handle, int(bool(dagger)), _stream(stream)),
           "qcd_apply_dslash")


def apply_dslash_ks(gauge: Gauge, out: Spinor, inp: Spinor, stream=None):
    """out = D_KS inp, the staggered derivative (qcd_apply_dslash_ks)."""
    _check(lib().qcd_apply_dslash_ks(gauge.handle, out.handle, inp.handle, _stream(stream)), "qcd_apply_dslash_ks")


def apply_M(gauge: Gauge, out: Spinor, inp: Spinor, kappa: float, mu: float = 0.0, eo: bool = False,
            dagger: bool = False, stream=None):
    """out = M inp (full) or Mhat inp (even-odd); see qcd_apply_M."""
    _check(lib().qcd_apply_M(gauge.handle, out.handle, inp.handle, float(kappa), float(mu), int(bool(eo)),
                             int(bool(dagger)), _stream(stream)), "qcd_apply_M")


def _handles(fields):
    return (_p * len(fields))(*[f.handle.value for f in fields])


def apply_dslash_multi(gauge: Gauge, outs, ins, dagger: bool = False, stream=None):
    """outs[k] = D_hop ins[k] for all k in one batched launch (qcd_apply_dslash_multi)."""
    if len(outs) != len(ins):
        raise ValueError("outs and ins differ in length")
    _check(lib().qcd_apply_dslash_multi(gauge.handle, _handles(outs), _handles(ins), len(ins), int(bool(dagger)),
                                        _stream(stream)), "qcd_apply_dslash_multi")


def solve_cg_multi(gauge: Gauge, xs, bs, kappa: float, mu: float = 0.0, tol: float = 1e-10, maxiter: int = 20000,
                   eo: bool = True, normal: bool = False, inner_prec: str = "f64", inner_recon: int = 12,
                   reliable_delta: float = 0.0, stream=None, raise_on_error: bool = True):
    """Batched CG over len(bs) systems (qcd_solve_cg_multi); returns (status, [stats dict])."""
    if len(xs) != len(bs):
        raise ValueError("xs and bs differ in length")
    n = len(bs)
    prm = SolverParams(float(kappa), float(mu), float(tol), int(maxiter), int(bool(eo)), int(bool(normal)),
                       PREC[inner_prec], int(inner_recon), float(reliable_delta))
    st = (SolverStats * n)()
    status = lib().qcd_solve_cg_multi(gauge.handle, _handles(xs), _handles(bs), n, ctypes.byref(prm), st,
                                      _stream(stream))
    if raise_on_error and status != 0:
        _check(status, "qcd_solve_cg_multi")
    return status, [{k: getattr(st[i], k) for k, _ in SolverStats._fields_} for i in range(n)]


def solve_cg_batch(gauge: Gauge, xs, bs, kappas, mus=None, tols=None, maxiter: int = 20000, eo: bool = True,
                   normal: bool = False, inner_prec: str = "f64", inner_recon: int = 12, reliable_delta: float = 0.0,
                   stream=None, raise_on_error: bool = True):
    """Batched CG over systems with their own kappa, mu and tol (qcd_solve_cg_batch);
    returns (status, [stats dict])."""
    n = len(bs)
    if len(xs) != n or len(kappas) != n:
        raise ValueError("xs, bs and kappas differ in length")
    mus = [0.0] * n if mus is None else list(mus)
    tols = [1e-10] * n if tols is None else list(tols)
    if len(mus) != n or len(tols) != n:
        raise ValueError("mus / tols differ in length from bs")
    prm = (SolverParams * n)(*[SolverParams(float(kappas[k]), float(mus[k]), float(tols[k]), int(maxiter),
                                            int(bool(eo)), int(bool(normal)), PREC[inner_prec], int(inner_recon),
                                            float(reliable_delta)) for k in range(n)])
    st = (SolverStats * n)()
    status = lib().qcd_solve_cg_batch(gauge.handle, _handles(xs), _handles(bs), n, prm, st, _stream(stream))
    if raise_on_error and status != 0:
        _check(status, "qcd_solve_cg_batch")
    return status, [{k: getattr(st[i], k) for k, _ in SolverStats._fields_} for i in range(n)]


FACE_TO_PREV, FACE_TO_NEXT, FACE_FROM_PREV, FACE_FROM_NEXT = 0, 1, 2, 3


def face_pack(gauge: Gauge, inp: Spinor, face: int, face_ptr: int, dagger: bool = False, sign: float = 1.0,
              stream=None):
    """qcd_face_pack into the device buffer at face_ptr (6 x sites-per-slice double2)."""
    _check(lib().qcd_face_pack(gauge.handle, inp.handle, int(face), int(bool(dagger)), float(sign), _p(face_ptr),
                               _stream(stream)), "qcd_face_pack")


def face_unpack(out: Spinor, face: int, face_ptr: int, stream=None):
    """qcd_face_unpack of the device buffer at face_ptr into a halo slice of `out`."""
    _check(lib().qcd_face_unpack(out.handle, int(face), _p(face_ptr), _stream(stream)), "qcd_face_unpack")


def solve_cg_many(gauges, xs, bs, kappas, mus=None, tols=None, maxiter: int = 20000, wait_cycles: int = 0,
                  max_blocks: int = 0,
                  stream=None, raise_on_error: bool = True):
    """FP64 even-odd CG of several systems, each on its own gauge field and
    lattice, in one persistent launch (qcd_solve_cg_many); returns (status,
    [stats dict])."""
    n = len(bs)
    if len(xs) != n or len(kappas) != n or len(gauges) != n:
        raise ValueError("gauges, xs, bs and kappas differ in length")
    mus = [0.0] * n if mus is None else list(mus)
    tols = [1e-10] * n if tols is None else list(tols)
    prm = (SolverParams * n)(*[SolverParams(float(kappas[k]), float(mus[k]), float(tols[k]), int(maxiter), 1, 0,
                                            PREC["f64"], 18, 0.1) for k in range(n)])
    st = (SolverStats * n)()
    status = lib().qcd_solve_cg_many(n, _handles(gauges), _handles(xs), _handles(bs), prm, st, int(wait_cycles),
                                     int(max_blocks), _stream(stream))
    if raise_on_error and status != 0:
        _check(status, "qcd_solve_cg_many")
    return status, [{k: getattr(st[i], k) for k, _ in SolverStats._fields_} for i in range(n)]


def solve_cg(gauge: Gauge, x: Spinor, b: Spinor, kappa: float, mu: float = 0.0, tol: float = 1e-10,
             maxiter: int = 20000, eo: bool = True, normal: bool = False, inner_prec: str = "f64",
             inner_recon: int = 12, reliable_delta: float = 0.0, stream=None, raise_on_error: bool = True):
    """CG solve (see qcd_solve_cg); returns (status, stats dict)."""
    prm = SolverParams(float(kappa), float(mu), float(tol), int(maxiter), int(bool(eo)), int(bool(normal)),
                       PREC[inner_prec], int(inner_recon), float(reliable_delta))
    st = SolverStats()
    status = lib().qcd_solve_cg(gauge.handle, x.handle, b.handle, ctypes.byref(prm), ctypes.byref(st),
                                _stream(stream))
    if raise_on_error and status not in (0,):
        _check(status, "qcd_solve_cg")
    stats = {k: getattr(st, k) for k, _ in SolverStats._fields_}
    return status, stats


def profile_begin():
    """Start recording every hopping-kernel launch (qcd_profile_begin)."""
    _check(lib().qcd_profile_begin(), "qcd_profile_begin")


def profile_end():
    """Stop recording; returns {prec: {launches, ms, bytes, flops, sites}}."""
    pr = Profile()
    _check(lib().qcd_profile_end(ctypes.byref(pr)), "qcd_profile_end")
    inv = {v: k for k, v in PREC.items()}
    return {inv[i]: {k: getattr(pr.prec[i], k) for k, _ in ProfileEntry._fields_} for i in range(5)}


def kernel_launches() -> int:
    """Kernels libqcd has launched since it was loaded."""
    return int(lib().qcd_kernel_launches())


NORM2_NOALLOC_MAX = 16_777_216


INJECT_SPINOR_CREATE = 1


def set_hop_threads(threads_per_site: int):
    """qcd_set_hop_threads: 0 autotuned, 1 or 8 threads per site forced for the
    FP64 reconstruct-18 hopping kernel."""
    _check(lib().qcd_set_hop_threads(int(threads_per_site)), "qcd_set_hop_threads")


def debug_inject(what: int, count: int):
    """qcd_debug_inject: the next `count` calls of kind `what` fail with
    QCD_ERR_OOM on the host (tests of error paths)."""
    _check(lib().qcd_debug_inject(int(what), int(count)), "qcd_debug_inject")


def norm2_noalloc(x_ptr: int, n: int, result_ptr: int, stream=None):
    """qcd_norm2_noalloc on raw device pointers (no allocation in the library)."""
    _check(lib().qcd_norm2_noalloc(_p(x_ptr), ctypes.c_size_t(n), _p(result_ptr), _stream(stream)),
           "qcd_norm2_noalloc")


class Server:
    """qcd_server: concurrent even-odd solves admitted by slot and memory budget."""

    def __init__(self, slots: int = 4, memory_budget: int = 32 << 30, batch_small_sites: int = 0):
        h = _p()
        cfg = ServerConfig(int(slots), int(memory_budget), int(batch_small_sites))
        _check(lib().qcd_server_create(ctypes.byref(cfg), ctypes.byref(h)), "qcd_server_create")
        self._h = h
        self._keep = {}

    def add_gauge(self, gauge: Gauge) -> int:
        gid = _i()
        _check(lib().qcd_server_add_gauge(self._h, gauge.handle, ctypes.byref(gid)), "qcd_server_add_gauge")
        self._keep[("g", gid.value)] = gauge
        return gid.value

    def submit(self, gauge_id: int, b_host, x_host, kappa: float, mu: float = 0.0, tol: float = 1e-10,
               maxiter: int = 20000, inner_prec: str = "f16", inner_recon: int = 12,
               reliable_delta: float = 0.0) -> int:
        req = Request(int(gauge_id), float(kappa), float(mu), float(tol), int(maxiter), PREC[inner_prec],
                      int(inner_recon), float(reliable_delta), _host_ptr(b_host), _host_ptr(x_host))
        rid = ctypes.c_longlong()
        _check(lib().qcd_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid)), "qcd_server_submit")
        self._keep[rid.value] = (b_host, x_host)
        return rid.value

    def wait(self, request_id: int) -> dict:
        res = RequestResult()
        _check(lib().qcd_server_wait(self._h, int(request_id), ctypes.byref(res)), "qcd_server_wait")
        self._keep.pop(request_id, None)
        out = {k: getattr(res, k) for k, _ in RequestResult._fields_ if k != "stats"}
        out["stats"] = {k: getattr(res.stats, k) for k, _ in SolverStats._fields_}
        return out

    def info(self):
        used, q, r = ctypes.c_size_t(), _i(), _i()
        _check(lib().qcd_server_info(self._h, ctypes.byref(used), ctypes.byref(q), ctypes.byref(r)), "qcd_server_info")
        return {"used_bytes": used.value, "queued": q.value, "running": r.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().qcd_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()
