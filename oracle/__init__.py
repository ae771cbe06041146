"""FP64 CPU oracle for the TSSP Gross-Pitaevskii step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this package.  The product library never does, and this package
never imports the product library: the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, double precision, own radix-2
FFT); this module compiles it on demand with gcc and marshals numpy arrays.

Array convention: a wave function on an ``n = (nx, ny, nz)`` grid is a
complex128 array of ``nx*ny*nz`` elements in C order with x fastest
(numpy shape ``(nz, ny, nx)``, ``(ny, nx)`` or ``(nx,)``).

Parity status of each function (what pins it in ``tests/test_oracle.py``):
  fft / dft_brute ...... brute-force DFT, numpy.fft, inverse round trip
  step_real ............ plane wave (exact), norm conservation, time reversal,
                         bright soliton, Bogoliubov frequency, g=0 breathing
                         Gaussian (closed form sigma(t))
  step_real_trap ....... a constant schedule equals step_real; g=0 quench of
                         the trap (closed form sigma(t)); g=0 modulated trap
                         against the moment equations integrated by RK4, with
                         second-order convergence in dt
  step_imag / ground ... g=0 harmonic ground state (closed form), 2D rows of
                         the paper's Table 1 (soft pin)
  norm_energy .......... closed-form Gaussian energies, plane-wave energy
  rms .................. closed-form Gaussian widths
  spectrum ............. Parseval, irrotational (E_inc=0) and solenoidal
                         (E_comp=0) fields
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None


class _Grid(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_long * 3),
        ("lo", ctypes.c_double * 3),
        ("len", ctypes.c_double * 3),
        ("g", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma", ctypes.c_double * 3),
        ("V", ctypes.POINTER(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (gcc, -O2, OpenMP). Returns the path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        cd = ctypes.c_void_p
        G = P(_Grid)
        lib.orc_fft.argtypes = [cd, ctypes.c_int, P(ctypes.c_long), ctypes.c_int]
        lib.orc_dft_brute.argtypes = [cd, cd, ctypes.c_int, P(ctypes.c_long), ctypes.c_int]
        lib.orc_step_real.argtypes = [cd, G, ctypes.c_long]
        lib.orc_step_real_trap.argtypes = [cd, G, ctypes.c_long, cd]
        lib.orc_step_imag.argtypes = [cd, G, ctypes.c_long, ctypes.c_double]
        lib.orc_norm_energy.argtypes = [cd, G, P(ctypes.c_double)]
        lib.orc_rms.argtypes = [cd, G, P(ctypes.c_double)]
        lib.orc_ground.argtypes = [cd, G, ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_long, P(ctypes.c_long), P(ctypes.c_double)]
        lib.orc_spectrum_nshells.argtypes = [G]
        lib.orc_spectrum_nshells.restype = ctypes.c_long
        lib.orc_spectrum.argtypes = [cd, G, cd, cd, ctypes.c_long]
        lib.orc_spectrum_qp_num.argtypes = [cd, G, cd, cd, ctypes.c_long]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def set_threads(nt: int = 0) -> int:
    """Set the OpenMP thread count (0 keeps the current one); returns it."""
    return _load().orc_set_threads(int(nt))


def _grid(n, lo=None, length=None, g=0.0, dt=0.0, gamma=None) -> _Grid:
    n = tuple(int(v) for v in n)
    d = len(n)
    if d < 1 or d > 3:
        raise ValueError("1 to 3 axes")
    gr = _Grid()
    gr.ndim = d
    for a in range(3):
        gr.n[a] = n[a] if a < d else 1
        gr.lo[a] = float(lo[a]) if (lo is not None and a < d) else 0.0
        gr.len[a] = float(length[a]) if (length is not None and a < d) else 1.0
        gr.gamma[a] = float(gamma[a]) if (gamma is not None and a < d) else 0.0
    gr.g = float(g)
    gr.dt = float(dt)
    return gr


def _as_c128(psi, N):
    a = np.ascontiguousarray(psi, dtype=np.complex128)
    if a.size != N:
        raise ValueError("array has %d points, grid has %d" % (a.size, N))
    return a


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def fft(x, n, sign=-1):
    """Unnormalised DFT over all axes (sign -1 forward, +1 inverse); returns a copy."""
    n = tuple(int(v) for v in n)
    y = _as_c128(x, int(np.prod(n))).copy()
    arr = (ctypes.c_long * 3)(*(list(n) + [1] * (3 - len(n))))
    _check(_load().orc_fft(_ptr(y), len(n), arr, int(sign)), "fft")
    return y


def dft_brute(x, n, sign=-1):
    """Direct O(N^2) DFT from the definition (tiny grids)."""
    n = tuple(int(v) for v in n)
    xa = _as_c128(x, int(np.prod(n)))
    y = np.empty_like(xa)
    arr = (ctypes.c_long * 3)(*(list(n) + [1] * (3 - len(n))))
    _check(_load().orc_dft_brute(_ptr(xa), _ptr(y), len(n), arr, int(sign)), "dft_brute")
    return y


class Problem:
    """Grid + physical parameters of one GPE instance.

    n: points per axis (x first); lo, length: box corner and size per axis;
    g: interaction; dt: time step; gamma: trap frequencies, V = 1/2 sum g_a^2 x_a^2;
    V: optional potential sampled on the grid (array of the grid's shape, x
    fastest), used instead of the harmonic one.
    """

    def __init__(self, n, lo, length, g=0.0, dt=1e-3, gamma=None, V=None):
        self.n = tuple(int(v) for v in n)
        self.lo = tuple(float(v) for v in lo)
        self.length = tuple(float(v) for v in length)
        self.g = float(g)
        self.dt = float(dt)
        self.gamma = tuple(float(v) for v in (gamma if gamma is not None else [0.0] * len(self.n)))
        self._g = _grid(self.n, self.lo, self.length, self.g, self.dt, self.gamma)
        self.N = int(np.prod(self.n))
        self.V = None
        if V is not None:
            self.V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1).copy()
            if self.V.size != self.N:
                raise ValueError("V has %d values, grid has %d" % (self.V.size, self.N))
            self._g.V = self.V.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def replace(self, **kw):
        args = dict(n=self.n, lo=self.lo, length=self.length, g=self.g, dt=self.dt,
                    gamma=self.gamma, V=self.V)
        args.update(kw)
        return Problem(**args)

    def step_real(self, psi, nsteps=1):
        """Advance nsteps real-time TSSP steps; returns a new array."""
        y = _as_c128(psi, self.N).copy()
        _check(_load().orc_step_real(_ptr(y), ctypes.byref(self._g), int(nsteps)), "step_real")
        return y.reshape(np.shape(psi))

    def step_real_trap(self, psi, gamma_t):
        """Real-time steps in a trap with time-dependent frequencies: gamma_t is
        an array of shape (nsteps + 1, ndim), the trap at the time levels of the
        call; step n uses row n for its first nonlinear half-step and row n + 1
        for its second.  Returns a new array."""
        g = np.ascontiguousarray(gamma_t, dtype=np.float64)
        if g.ndim != 2 or g.shape[1] != len(self.n) or g.shape[0] < 1:
            raise ValueError("gamma_t must have shape (nsteps + 1, ndim)")
        g3 = np.zeros((g.shape[0], 3))
        g3[:, :len(self.n)] = g
        y = _as_c128(psi, self.N).copy()
        _check(_load().orc_step_real_trap(_ptr(y), ctypes.byref(self._g), int(g.shape[0] - 1), _ptr(g3)),
               "step_real_trap")
        return y.reshape(np.shape(psi))

    def step_imag(self, psi, nsteps=1, target_norm=1.0):
        """Advance nsteps imaginary-time steps, renormalising after each."""
        y = _as_c128(psi, self.N).copy()
        _check(_load().orc_step_imag(_ptr(y), ctypes.byref(self._g), int(nsteps),
                                     float(target_norm)), "step_imag")
        return y.reshape(np.shape(psi))

    def ground(self, psi, max_steps, target_norm=1.0, etol=1e-10, check_every=1):
        """Imaginary time until |dE| < etol between checks. Returns (psi, steps, E)."""
        y = _as_c128(psi, self.N).copy()
        sd = ctypes.c_long(0)
        ef = ctypes.c_double(0.0)
        _check(_load().orc_ground(_ptr(y), ctypes.byref(self._g), int(max_steps),
                                  float(target_norm), float(etol), int(check_every),
                                  ctypes.byref(sd), ctypes.byref(ef)), "ground")
        return y.reshape(np.shape(psi)), sd.value, ef.value

    def norm_energy(self, psi):
        """Returns [norm, E_kin, E_pot, E_int, E, mu]."""
        x = _as_c128(psi, self.N)
        out = (ctypes.c_double * 6)()
        _check(_load().orc_norm_energy(_ptr(x), ctypes.byref(self._g), out), "norm_energy")
        return np.array(out[:])

    def rms(self, psi):
        """Returns [sigma_x, sigma_y, sigma_z, r_rms]."""
        x = _as_c128(psi, self.N)
        out = (ctypes.c_double * 4)()
        _check(_load().orc_rms(_ptr(x), ctypes.byref(self._g), out), "rms")
        return np.array(out[:])

    def nshells(self):
        return int(_load().orc_spectrum_nshells(ctypes.byref(self._g)))

    def spectrum(self, psi):
        """Returns (E_inc[nshells], E_comp[nshells])."""
        x = _as_c128(psi, self.N)
        ns = self.nshells()
        ei = np.zeros(ns)
        ec = np.zeros(ns)
        _check(_load().orc_spectrum(_ptr(x), ctypes.byref(self._g), _ptr(ei), _ptr(ec), ns),
               "spectrum")
        return ei, ec

    def spectrum_qp_num(self, psi):
        """Returns (E_qp[nshells], N[nshells]): quantum-pressure and particle-number spectra."""
        x = _as_c128(psi, self.N)
        ns = self.nshells()
        eq = np.zeros(ns)
        nn = np.zeros(ns)
        _check(_load().orc_spectrum_qp_num(_ptr(x), ctypes.byref(self._g), _ptr(eq), _ptr(nn), ns),
               "spectrum_qp_num")
        return eq, nn
