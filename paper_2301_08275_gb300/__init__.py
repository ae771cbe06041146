"""GB300 TSSP Gross-Pitaevskii library: thin Python binding of libgpe.so.

Argument marshalling only.  Every computation runs in the CUDA library
(include/gpe.h); this module converts torch tensors and numpy arrays to
pointers and status codes to exceptions.  There is no CPU fallback: if the
shared library is missing or a call fails, an exception is raised.

Entry points keep the C names (``gpe_plan_create``, ``gpe_step_real``, ...);
``Plan`` wraps them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpe.so")
_lock = threading.Lock()
_lib = None

GPE_C64, GPE_C128 = 0, 1
GPE_SPEC_INC, GPE_SPEC_COMP, GPE_SPEC_QP, GPE_SPEC_NUM = 1, 2, 4, 8
STATUS = {0: "GPE_OK", 1: "GPE_EINVAL", 2: "GPE_EUNSUPPORTED", 3: "GPE_ENOMEM", 4: "GPE_ECUDA",
          5: "GPE_ENUMERIC", 6: "GPE_ETIMEOUT", 7: "GPE_EBUSY", 8: "GPE_ENOTREADY"}

EXPORTS = ["gpe_plan_create", "gpe_plan_destroy", "gpe_step_real", "gpe_step_real_host", "gpe_step_real_trap",
           "gpe_step_imag",
           "gpe_norm_energy", "gpe_rms_size", "gpe_spectrum_nshells", "gpe_spectrum", "gpe_last_error",
           "gpe_trace_enable", "gpe_trace_count", "gpe_trace_read", "gpe_norm_energy_noalloc",
           "gpe_batch_create", "gpe_batch_destroy", "gpe_batch_step_real", "gpe_batch_norm_energy",
           "gpe_batch_groups", "gpe_server_create", "gpe_server_destroy", "gpe_serve_submit", "gpe_serve_poll",
           "gpe_server_stats", "gpe_plan_set_option", "gpe_plan_get_option",
           "gpe_plan_autotune", "gpe_measure_fp64_peak"]


class GpeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), msg))
        self.status = status


class gpe_plan_desc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int64 * 3),
        ("lo", ctypes.c_double * 3),
        ("len", ctypes.c_double * 3),
        ("g", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma", ctypes.c_double * 3),
        ("prec", ctypes.c_int),
        ("batch", ctypes.c_int),
        ("g_each", ctypes.POINTER(ctypes.c_double)),
        ("gamma_each", ctypes.POINTER(ctypes.c_double)),
        ("V_host", ctypes.POINTER(ctypes.c_double)),
    ]


class gpe_request(ctypes.Structure):
    _fields_ = [
        ("desc", gpe_plan_desc),
        ("imag", ctypes.c_int),
        ("nsteps", ctypes.c_int64),
        ("etol", ctypes.c_double),
        ("check_every", ctypes.c_int),
        ("target_norm", ctypes.c_double),
        ("psi0_host", ctypes.c_void_p),
    ]


class gpe_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("steps_done", ctypes.c_int64),
        ("norm", ctypes.c_double),
        ("energy", ctypes.c_double),
        ("t_submit", ctypes.c_double),
        ("t_admit", ctypes.c_double),
        ("t_done", ctypes.c_double),
    ]


def build(force=False, verbose=False):
    """Compile libgpe.so in-tree (nvcc, sm_103a)."""
    from . import buildlib as _b
    return _b.build(force=force, verbose=verbose)


def lib():
    """Load libgpe.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgpe.so is not built; call paper_2301_08275_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        L.gpe_plan_create.argtypes = [ctypes.POINTER(gpe_plan_desc), vp, ctypes.POINTER(vp)]
        L.gpe_plan_destroy.argtypes = [vp]
        L.gpe_step_real.argtypes = [vp, vp, i64]
        L.gpe_step_real_trap.argtypes = [vp, vp, i64, dp]
        L.gpe_step_real_host.argtypes = [vp, vp, i64]
        L.gpe_step_imag.argtypes = [vp, vp, i64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(i64), dp]
        L.gpe_norm_energy.argtypes = [vp, vp, dp]
        L.gpe_rms_size.argtypes = [vp, vp, dp]
        L.gpe_spectrum_nshells.argtypes = [vp]
        L.gpe_spectrum_nshells.restype = i64
        L.gpe_spectrum.argtypes = [vp, vp, ctypes.c_uint, dp, i64]
        L.gpe_last_error.restype = ctypes.c_char_p
        L.gpe_norm_energy_noalloc.argtypes = [ctypes.POINTER(gpe_plan_desc), vp, vp, dp]
        L.gpe_batch_create.argtypes = [ctypes.POINTER(gpe_plan_desc), ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.gpe_batch_destroy.argtypes = [vp]
        L.gpe_batch_step_real.argtypes = [vp, ctypes.POINTER(vp), i64, ctypes.c_int]
        L.gpe_batch_norm_energy.argtypes = [vp, ctypes.POINTER(vp), dp]
        L.gpe_batch_groups.argtypes = [vp]
        L.gpe_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
        L.gpe_server_destroy.argtypes = [vp]
        L.gpe_serve_submit.argtypes = [vp, ctypes.POINTER(gpe_request), ctypes.POINTER(ctypes.c_uint64)]
        L.gpe_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(gpe_result), vp]
        L.gpe_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_size_t)]
        L.gpe_trace_enable.argtypes = [vp, ctypes.c_int]
        L.gpe_plan_set_option.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
        L.gpe_plan_get_option.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
        L.gpe_plan_autotune.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
        L.gpe_trace_count.argtypes = [vp]
        L.gpe_measure_fp64_peak.argtypes = [vp, dp]
        L.gpe_trace_read.argtypes = [vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t,
                                     ctypes.POINTER(i64), dp]
        for name in EXPORTS:
            if name != "gpe_last_error" and name != "gpe_spectrum_nshells":
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(rc):
    if rc != 0:
        raise GpeError(rc, lib().gpe_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------- C-named calls
def gpe_last_error():
    return lib().gpe_last_error().decode()


def gpe_plan_create(desc, stream=None):
    h = ctypes.c_void_p()
    _check(lib().gpe_plan_create(ctypes.byref(desc), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def gpe_plan_destroy(plan):
    _check(lib().gpe_plan_destroy(plan))


def gpe_step_real(plan, psi_ptr, nsteps):
    _check(lib().gpe_step_real(plan, ctypes.c_void_p(psi_ptr), int(nsteps)))


def gpe_step_real_trap(plan, psi_ptr, gamma_t):
    """gamma_t: array (nsteps + 1, ndim) of trap frequencies at the time levels."""
    g = np.ascontiguousarray(gamma_t, dtype=np.float64)
    if g.ndim != 2 or g.shape[0] < 1 or g.shape[1] < 1 or g.shape[1] > 3:
        raise ValueError("gamma_t must have shape (nsteps + 1, ndim)")
    g3 = np.zeros((g.shape[0], 3))
    g3[:, :g.shape[1]] = g
    _check(lib().gpe_step_real_trap(plan, ctypes.c_void_p(psi_ptr), int(g.shape[0] - 1),
                                    g3.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def gpe_step_real_host(plan, psi_host_ptr, nsteps):
    _check(lib().gpe_step_real_host(plan, ctypes.c_void_p(psi_host_ptr), int(nsteps)))


def gpe_step_imag(plan, psi_ptr, max_steps, target_norm, etol, check_every, batch):
    sd = ctypes.c_int64(0)
    ef = np.zeros(batch)
    _check(lib().gpe_step_imag(plan, ctypes.c_void_p(psi_ptr), int(max_steps), float(target_norm),
                               float(etol), int(check_every), ctypes.byref(sd), _dptr(ef)))
    return sd.value, ef


def gpe_norm_energy(plan, psi_ptr, batch):
    out = np.zeros(6 * batch)
    _check(lib().gpe_norm_energy(plan, ctypes.c_void_p(psi_ptr), _dptr(out)))
    return out.reshape(batch, 6)


def gpe_rms_size(plan, psi_ptr, batch):
    out = np.zeros(4 * batch)
    _check(lib().gpe_rms_size(plan, ctypes.c_void_p(psi_ptr), _dptr(out)))
    return out.reshape(batch, 4)


def gpe_spectrum_nshells(plan):
    return int(lib().gpe_spectrum_nshells(plan))


def gpe_spectrum(plan, psi_ptr, kinds, batch):
    ns = gpe_spectrum_nshells(plan)
    nk = bin(int(kinds) & 15).count("1")
    out = np.zeros(nk * batch * ns)
    _check(lib().gpe_spectrum(plan, ctypes.c_void_p(psi_ptr), int(kinds), _dptr(out), ns))
    return out.reshape(nk, batch, ns)


def gpe_norm_energy_noalloc(desc, psi_ptr, stream=None):
    """Norm/energy of one instance without any allocation by the library
    (see include/gpe.h); returns [norm, E_kin, E_pot, E_int, E, mu]."""
    out = np.zeros(6)
    _check(lib().gpe_norm_energy_noalloc(ctypes.byref(desc), ctypes.c_void_p(psi_ptr),
                                         ctypes.c_void_p(stream or 0), _dptr(out)))
    return out


GPE_OPT_TMA_STAGING, GPE_OPT_TILE_X, GPE_OPT_TILE_Y, GPE_OPT_TILE_Z, GPE_OPT_TMA_Y, GPE_OPT_TMA_Z = 1, 2, 3, 4, 5, 6
GPE_OPT_GENERIC_PASSES = 7
GPE_OPT_NO_DITHER = 8
GPE_OPT_LINE_CLUSTER = 9
GPE_OPT_TEST_STALL_COPIES = 99
GPE_TUNE_NO_TMA = 1


def gpe_plan_set_option(plan, option, value):
    _check(lib().gpe_plan_set_option(plan, int(option), int(value)))


def gpe_plan_get_option(plan, option):
    v = ctypes.c_int64(0)
    _check(lib().gpe_plan_get_option(plan, int(option), ctypes.byref(v)))
    return v.value


def gpe_plan_autotune(plan, psi_ptr, reps=3, flags=0):
    """psi_ptr: device address of a state to time on (read only), or 0 for zeros."""
    _check(lib().gpe_plan_autotune(plan, ctypes.c_void_p(psi_ptr or None), int(reps), int(flags)))


def gpe_measure_fp64_peak(stream=0):
    """Measured FP64 FMA throughput of the current device in FLOP/s."""
    out = ctypes.c_double(0.0)
    _check(lib().gpe_measure_fp64_peak(ctypes.c_void_p(stream or None), ctypes.byref(out)))
    return out.value


def gpe_trace_enable(plan, enable=True):
    _check(lib().gpe_trace_enable(plan, 1 if enable else 0))


def gpe_trace_count(plan):
    n = lib().gpe_trace_count(plan)
    if n < 0:
        raise GpeError(4, gpe_last_error())
    return n


def gpe_trace_read(plan, i):
    buf = ctypes.create_string_buffer(128)
    cnt = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    _check(lib().gpe_trace_read(plan, int(i), buf, 128, ctypes.byref(cnt), ctypes.byref(ms)))
    return buf.value.decode(), cnt.value, ms.value


# ------------------------------------------------------------- torch-facing plan
def make_desc(n, lo, length, g=0.0, dt=1e-3, gamma=None, prec=GPE_C64, batch=1, g_each=None,
              gamma_each=None, V=None):
    d = gpe_plan_desc()
    nd = len(n)
    d.ndim = nd
    for a in range(3):
        d.n[a] = int(n[a]) if a < nd else 1
        d.lo[a] = float(lo[a]) if a < nd else 0.0
        d.len[a] = float(length[a]) if a < nd else 1.0
        d.gamma[a] = float(gamma[a]) if (gamma is not None and a < nd) else 0.0
    d.g = float(g)
    d.dt = float(dt)
    d.prec = int(prec)
    d.batch = int(batch)
    keep = []
    if g_each is not None:
        ge = np.ascontiguousarray(g_each, dtype=np.float64)
        keep.append(ge)
        d.g_each = _dptr(ge)
    if gamma_each is not None:
        gm = np.ascontiguousarray(gamma_each, dtype=np.float64).reshape(-1)
        keep.append(gm)
        d.gamma_each = _dptr(gm)
    if V is not None:
        vv = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        keep.append(vv)
        d.V_host = _dptr(vv)
    return d, keep


class Plan:
    """A plan bound to a CUDA stream; psi arguments are torch tensors on that device.

    prec: GPE_C64 (torch.complex64) or GPE_C128 (torch.complex128).  psi holds
    batch instances back to back, x fastest (e.g. shape (batch, nz, ny, nx)).
    """

    def __init__(self, n, lo, length, g=0.0, dt=1e-3, gamma=None, prec=GPE_C64, batch=1, g_each=None,
                 gamma_each=None, stream=None, V=None):
        import torch
        self.n = tuple(int(v) for v in n)
        self.batch = int(batch)
        self.prec = int(prec)
        self.dtype = torch.complex64 if prec == GPE_C64 else torch.complex128
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        desc, keep = make_desc(n, lo, length, g, dt, gamma, prec, batch, g_each, gamma_each, V)
        self._h = gpe_plan_create(desc, stream.cuda_stream)
        del keep

    def close(self):
        if getattr(self, "_h", None):
            gpe_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptr(self, psi):
        import torch
        if not isinstance(psi, torch.Tensor) or not psi.is_cuda:
            raise TypeError("psi must be a CUDA tensor")
        if psi.dtype != self.dtype or not psi.is_contiguous():
            raise TypeError("psi must be a contiguous %s tensor" % self.dtype)
        if psi.numel() != self.batch * int(np.prod(self.n)):
            raise ValueError("psi has %d points, plan expects %d" % (psi.numel(), self.batch * int(np.prod(self.n))))
        return psi.data_ptr()

    def step_real(self, psi, nsteps):
        gpe_step_real(self._h, self._ptr(psi), nsteps)
        return psi

    def step_real_trap(self, psi, gamma_t):
        gpe_step_real_trap(self._h, self._ptr(psi), gamma_t)
        return psi

    def step_imag(self, psi, max_steps, target_norm=1.0, etol=0.0, check_every=1):
        return gpe_step_imag(self._h, self._ptr(psi), max_steps, target_norm, etol, check_every, self.batch)

    def norm_energy(self, psi):
        return gpe_norm_energy(self._h, self._ptr(psi), self.batch)

    def rms_size(self, psi):
        return gpe_rms_size(self._h, self._ptr(psi), self.batch)

    def nshells(self):
        return gpe_spectrum_nshells(self._h)

    def spectrum(self, psi, kinds=GPE_SPEC_INC | GPE_SPEC_COMP):
        return gpe_spectrum(self._h, self._ptr(psi), kinds, self.batch)

    def set_option(self, option, value):
        gpe_plan_set_option(self._h, option, value)

    def get_option(self, option):
        return gpe_plan_get_option(self._h, option)

    def autotune(self, psi=None, reps=6, flags=0):
        """Time the tile shapes / staging modes on a scratch copy of psi (a CUDA
        tensor, only read) and keep the fastest; returns the chosen options."""
        gpe_plan_autotune(self._h, self._ptr(psi) if psi is not None else 0, reps, flags)
        return {name: self.get_option(opt) for name, opt in
                (("tile_x", GPE_OPT_TILE_X), ("tile_y", GPE_OPT_TILE_Y), ("tile_z", GPE_OPT_TILE_Z),
                 ("tma_y", GPE_OPT_TMA_Y), ("tma_z", GPE_OPT_TMA_Z))}

    def trace(self, enable=True):
        gpe_trace_enable(self._h, enable)

    def trace_read(self):
        """{kind: (launches, total_ms)} recorded since tracing was enabled."""
        return {k: (c, t) for k, c, t in (gpe_trace_read(self._h, i) for i in range(gpe_trace_count(self._h)))}

    def step_real_host(self, psi_np, nsteps):
        """psi_np: C-contiguous numpy complex64/complex128 array (modified in place)."""
        want = np.complex64 if self.prec == GPE_C64 else np.complex128
        if psi_np.dtype != want or not psi_np.flags["C_CONTIGUOUS"]:
            raise TypeError("psi must be a C-contiguous %s array" % np.dtype(want).name)
        gpe_step_real_host(self._h, psi_np.ctypes.data, nsteps)
        return psi_np


# ------------------------------------------------------------- batches and serving
def gpe_batch_create(descs, stream=None):
    arr = (gpe_plan_desc * len(descs))(*descs)
    h = ctypes.c_void_p()
    _check(lib().gpe_batch_create(arr, len(descs), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def gpe_batch_destroy(batch):
    _check(lib().gpe_batch_destroy(batch))


def _ptr_array(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*[ctypes.c_void_p(int(p)) for p in ptrs])


def gpe_batch_step_real(batch, ptrs, nsteps, use_graph=True):
    _check(lib().gpe_batch_step_real(batch, _ptr_array(ptrs), int(nsteps), 1 if use_graph else 0))


def gpe_batch_norm_energy(batch, ptrs):
    out = np.zeros(6 * len(ptrs))
    _check(lib().gpe_batch_norm_energy(batch, _ptr_array(ptrs), _dptr(out)))
    return out.reshape(len(ptrs), 6)


def gpe_batch_groups(batch):
    return int(lib().gpe_batch_groups(batch))


def gpe_server_create(hbm_budget_bytes, max_active, chunk_steps=64):
    h = ctypes.c_void_p()
    _check(lib().gpe_server_create(ctypes.c_size_t(int(hbm_budget_bytes)), int(max_active), int(chunk_steps),
                                   ctypes.byref(h)))
    return h


def gpe_server_destroy(server):
    _check(lib().gpe_server_destroy(server))


def gpe_serve_submit(server, desc, psi0, imag=False, nsteps=1, etol=0.0, check_every=1, target_norm=1.0):
    """psi0: C-contiguous numpy array (copied by the call)."""
    r = gpe_request()
    r.desc = desc
    r.imag = 1 if imag else 0
    r.nsteps = int(nsteps)
    r.etol = float(etol)
    r.check_every = int(check_every)
    r.target_norm = float(target_norm)
    r.psi0_host = psi0.ctypes.data
    t = ctypes.c_uint64(0)
    _check(lib().gpe_serve_submit(server, ctypes.byref(r), ctypes.byref(t)))
    return t.value


def gpe_serve_poll(server, ticket, timeout_ms=-1, psi_out=None):
    """Returns a gpe_result, or None if the request has not finished."""
    res = gpe_result()
    rc = lib().gpe_serve_poll(server, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(res),
                              ctypes.c_void_p(psi_out.ctypes.data if psi_out is not None else 0))
    if rc == 8:
        return None
    _check(rc)
    return res


def gpe_server_stats(server):
    q, a, u = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_size_t(0)
    _check(lib().gpe_server_stats(server, ctypes.byref(q), ctypes.byref(a), ctypes.byref(u)))
    return q.value, a.value, u.value
