"""Seeded synthetic inputs for the TSSP Gross-Pitaevskii workloads.

This module is shared by the tests, the benchmark, the oracle side and the
GPU side.  It builds initial wave functions and problem descriptions only; it
holds none of the solver's arithmetic (no FFT, no splitting step, no
diagnostics).  Every generator is deterministic in its seed
(``numpy.random.default_rng``, PCG64) and returns complex128 arrays in C order
with x fastest (numpy shape ``(nz, ny, nx)`` / ``(ny, nx)`` / ``(nx,)``).

Workload recipes (readings of the paper where it is silent):
  * 1D: n=256 on [-16,16), V=x^2/2, g=10, dt=1e-3; psi0 = pi^-1/4 exp(-(x-0.5)^2/2)
    with i.i.d. U(-0.01,0.01) phase noise, renormalised discretely to unit norm.
  * 2D quantum turbulence: 1024^2 box of side 2*pi*32, V=0, g=1, rho0=1;
    512 point vortices of alternating charge at >= 4 healing lengths (periodic
    distance), phase from a product of Jacobi theta functions (periodic in x
    and y after a linear correction), amplitude prod tanh(r_j/xi).
  * 3D Taylor-Green: 512^3 box of side 2*pi*16, phase
    arg(cos kx + i cos ky) + arg(cos kx + i cos kz), k = 4*2*pi/L, density
    rho0 (1 + 0.01 eta), eta i.i.d. U(-1,1).
  * 3D trap: 256^3 on [-8,8)^3, gamma=(1,2,4), g=200, start from the g=0
    ground-state Gaussian.
  * batched 2D instances and a Poisson request stream (see ``batched_specs`` and
    ``request_stream``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Spec", "axes", "gaussian_1d", "harmonic_gaussian", "bao_gaussian", "plane_wave",
    "vortex_positions", "vortex_field_2d", "taylor_green_3d", "random_field",
    "batched_specs", "request_stream", "CONFIG_1D", "CONFIG_2D", "CONFIG_3D_TG",
    "CONFIG_3D_TRAP",
]


@dataclass
class Spec:
    """One GPE instance: grid, box and physical parameters."""
    n: tuple
    lo: tuple
    length: tuple
    g: float = 0.0
    dt: float = 1e-3
    gamma: tuple = (0.0, 0.0, 0.0)
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self):
        return len(self.n)

    @property
    def N(self):
        return int(np.prod(self.n))

    @property
    def shape(self):
        """numpy shape, slowest axis first."""
        return tuple(reversed(self.n))

    def cell_volume(self):
        return float(np.prod([L / n for L, n in zip(self.length, self.n)]))

    def kwargs(self):
        return dict(n=self.n, lo=self.lo, length=self.length, g=self.g, dt=self.dt,
                    gamma=tuple(self.gamma[: self.ndim]))


def axes(spec: Spec):
    """Per-axis coordinate vectors x_j = lo + j*L/n (x first)."""
    return [spec.lo[a] + np.arange(spec.n[a]) * (spec.length[a] / spec.n[a])
            for a in range(spec.ndim)]


def _mesh(spec: Spec):
    """Coordinate arrays broadcast to the numpy shape (slowest axis first)."""
    xs = axes(spec)
    grids = np.meshgrid(*reversed(xs), indexing="ij")
    return list(reversed(grids))          # x, y, z order


def _discrete_normalise(psi, spec: Spec, target=1.0):
    nrm = float(np.sum(np.abs(psi) ** 2) * spec.cell_volume())
    return psi * math.sqrt(target / nrm)


# ---------------------------------------------------------------- configs
CONFIG_1D = Spec(n=(256,), lo=(-16.0,), length=(32.0,), g=10.0, dt=1e-3, gamma=(1.0,))
CONFIG_2D = Spec(n=(1024, 1024), lo=(0.0, 0.0), length=(2 * math.pi * 32,) * 2,
                 g=1.0, dt=5e-4, gamma=(0.0, 0.0))
CONFIG_3D_TG = Spec(n=(512, 512, 512), lo=(0.0,) * 3, length=(2 * math.pi * 16,) * 3,
                    g=1.0, dt=1e-3, gamma=(0.0, 0.0, 0.0))
CONFIG_3D_TRAP = Spec(n=(256, 256, 256), lo=(-8.0,) * 3, length=(16.0,) * 3,
                      g=200.0, dt=1e-3, gamma=(1.0, 2.0, 4.0))


def gaussian_1d(spec: Spec = CONFIG_1D, seed: int = 0, x0: float = 0.5, noise: float = 0.01):
    """pi^-1/4 exp(-(x-x0)^2/2) times exp(i*phi), phi ~ U(-noise, noise) per point,
    renormalised to sum |psi|^2 dx = 1."""
    rng = np.random.default_rng(seed)
    x = axes(spec)[0]
    amp = math.pi ** -0.25 * np.exp(-(x - x0) ** 2 / 2)
    phi = rng.uniform(-noise, noise, size=spec.n[0])
    return _discrete_normalise(amp * np.exp(1j * phi), spec)


def harmonic_gaussian(spec: Spec, seed: int | None = None, noise: float = 0.0):
    """g=0 ground state of V = 1/2 sum gamma_a^2 x_a^2:
    prod_a (gamma_a/pi)^(1/4) exp(-gamma_a x_a^2 / 2), optional phase noise."""
    X = _mesh(spec)
    psi = np.ones(spec.shape, dtype=np.complex128)
    for a in range(spec.ndim):
        ga = spec.gamma[a]
        psi = psi * (ga / math.pi) ** 0.25 * np.exp(-ga * X[a] ** 2 / 2)
    if noise:
        rng = np.random.default_rng(seed)
        psi = psi * np.exp(1j * rng.uniform(-noise, noise, size=spec.shape))
    return psi


def bao_gaussian(spec: Spec, gamma_y=2.0, gamma_z=4.0, eps1=0.25):
    """Initial state of the paper's dynamics validation (3D):
    (gy gz)^(1/4) / (pi eps1)^(3/4) exp(-(x^2 + gy y^2 + gz z^2)/(2 eps1)),
    the normalised reading of the printed prefactor."""
    X = _mesh(spec)
    w = [1.0, gamma_y, gamma_z][: spec.ndim]
    pref = (np.prod(w) ** 0.25) / (math.pi * eps1) ** (spec.ndim / 4.0)
    expo = sum(w[a] * X[a] ** 2 for a in range(spec.ndim)) / (2 * eps1)
    return (pref * np.exp(-expo)).astype(np.complex128)


def plane_wave(spec: Spec, modes, amp=1.0):
    """amp * exp(i k.x) with k_a = 2 pi m_a / L_a."""
    X = _mesh(spec)
    ph = sum(2 * math.pi * modes[a] / spec.length[a] * X[a] for a in range(spec.ndim))
    return amp * np.exp(1j * ph)


def random_field(spec: Spec, seed=0, smooth=0.0):
    """Complex Gaussian noise (optionally damped at high |k| by exp(-smooth k^2)),
    normalised to unit norm.  Used as a generic parity input."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(spec.shape) + 1j * rng.standard_normal(spec.shape)
    if smooth > 0:
        ks = [2 * math.pi * np.fft.fftfreq(spec.n[a], d=spec.length[a] / spec.n[a])
              for a in range(spec.ndim)]
        K = np.meshgrid(*reversed(ks), indexing="ij")
        k2 = sum(k ** 2 for k in K)
        z = np.fft.ifftn(np.fft.fftn(z) * np.exp(-smooth * k2))
    return _discrete_normalise(z, spec)


# ---------------------------------------------------------------- vortices
def _theta1_grid(ax, ay, nterms=8):
    """theta_1 on the grid u = ax[None,:] + i*ay[:,None] (ax, ay real vectors),
    via sin(a+ib) = sin a cosh b + i cos a sinh b summed over the series."""
    q = math.exp(-math.pi)
    re = np.zeros((ay.size, ax.size))
    im = np.zeros((ay.size, ax.size))
    for n in range(nterms):
        c = 2.0 * (-1) ** n * q ** ((n + 0.5) ** 2)
        m = 2 * n + 1
        re += c * np.outer(np.cosh(m * ay), np.sin(m * ax))
        im += c * np.outer(np.sinh(m * ay), np.cos(m * ax))
    return re, im


def vortex_positions(nv, L, min_sep, seed):
    """nv positions in [0,L)^2 by rejection sampling with periodic (minimum
    image) separation >= min_sep; charges alternate +1,-1 in insertion order."""
    rng = np.random.default_rng(seed)
    pos = np.zeros((nv, 2))
    k = 0
    tries = 0
    while k < nv:
        tries += 1
        if tries > 200000 * max(nv, 1):
            raise RuntimeError("could not place vortices")
        p = rng.uniform(0.0, L, size=2)
        if k:
            d = pos[:k] - p
            d -= L * np.round(d / L)
            if np.min(np.hypot(d[:, 0], d[:, 1])) < min_sep:
                continue
        pos[k] = p
        k += 1
    charges = np.array([1 if i % 2 == 0 else -1 for i in range(nv)])
    return pos, charges


def vortex_field_2d(spec: Spec = CONFIG_2D, nv=512, seed=0, rho0=1.0, min_sep_xi=4.0):
    """Periodic 2D field with nv point vortices (see module docstring).
    Returns (psi, positions, charges).  Requires a square box."""
    assert spec.ndim == 2 and spec.length[0] == spec.length[1] and spec.n[0] == spec.n[1]
    L = spec.length[0]
    g = spec.g if spec.g > 0 else 1.0
    xi = 1.0 / math.sqrt(g * rho0)
    pos, q = vortex_positions(nv, L, min_sep_xi * xi, seed)
    x, y = axes(spec)
    # x, y measured from the box corner: the construction is translation invariant
    xr = x - spec.lo[0]
    yr = y - spec.lo[1]
    theta = np.zeros((spec.n[1], spec.n[0]))
    amp = np.ones((spec.n[1], spec.n[0]))
    for j in range(nv):
        ax = math.pi * (xr - pos[j, 0]) / L
        dy = yr - pos[j, 1]
        ay = math.pi * dy / L
        re, im = _theta1_grid(ax, ay)
        theta += q[j] * np.arctan2(im, re)
        dxm = (xr - pos[j, 0]) - L * np.round((xr - pos[j, 0]) / L)
        dym = dy - L * np.round(dy / L)
        r = np.sqrt(dxm[None, :] ** 2 + dym[:, None] ** 2)
        amp *= np.tanh(r / xi)
    X = float(np.sum(q * pos[:, 0]))
    theta -= 2 * math.pi * X * yr[:, None] / L ** 2
    psi = math.sqrt(rho0) * amp * np.exp(1j * theta)
    return psi, pos, q


def taylor_green_3d(spec: Spec = CONFIG_3D_TG, seed=0, rho0=1.0, noise=0.01, kmode=4):
    """sqrt(rho0 (1 + noise*eta)) exp(i theta_TG), eta ~ U(-1,1) per point,
    theta_TG = arg(cos kx + i cos ky) + arg(cos kx + i cos kz), k = kmode*2*pi/L.
    Returns complex64 when the grid is large (to bound host memory), else complex128."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = spec.n
    x, y, z = axes(spec)
    kx = kmode * 2 * math.pi / spec.length[0]
    ky = kmode * 2 * math.pi / spec.length[1]
    kz = kmode * 2 * math.pi / spec.length[2]
    cx = np.cos(kx * x)[None, None, :]
    cy = np.cos(ky * y)[None, :, None]
    cz = np.cos(kz * z)[:, None, None]
    dtype = np.complex64 if spec.N > (1 << 24) else np.complex128
    out = np.empty(spec.shape, dtype=dtype)
    for iz in range(nz):                       # plane by plane: bounded temporaries
        th = np.arctan2(cy[0], cx[0]) + np.arctan2(cz[iz], cx[0])
        eta = rng.uniform(-1.0, 1.0, size=(ny, nx))
        out[iz] = np.sqrt(rho0 * (1.0 + noise * eta)) * np.exp(1j * th)
    return out


# ---------------------------------------------------------------- batched / serving
def optical_lattice(spec: Spec, v0=5.0, periods=4, gamma=None):
    """V = v0 sum_a sin^2(pi periods (x_a - lo_a) / L_a) (periodic on the box), plus an
    optional harmonic confinement 1/2 sum gamma_a^2 x_a^2; grid-shaped float64 array."""
    mesh = _mesh(spec)
    v = np.zeros(spec.shape)
    for a in range(spec.ndim):
        v = v + v0 * np.sin(np.pi * periods * (mesh[a] - spec.lo[a]) / spec.length[a]) ** 2
        if gamma is not None:
            v = v + 0.5 * gamma[a] ** 2 * mesh[a] ** 2
    return np.ascontiguousarray(v)


def anharmonic(spec: Spec, gamma=(1.0, 1.0, 1.0), lam=0.05):
    """V = 1/2 sum gamma_a^2 x_a^2 + lam (sum x_a^2)^2; grid-shaped float64 array."""
    mesh = _mesh(spec)
    r2 = sum(mesh[a] ** 2 for a in range(spec.ndim))
    v = sum(0.5 * gamma[a] ** 2 * mesh[a] ** 2 for a in range(spec.ndim)) + lam * r2 ** 2
    return np.ascontiguousarray(v)


def batched_specs(count=512, seed=0, sizes=(64, 128, 256, 512), g_range=(0.0, 1000.0),
                  gamma_range=(1.0, 4.0), half_width=12.0, dt=1e-3, noise=0.01):
    """Uneven 2D instances: n uniform over `sizes` (square), box [-12,12)^2,
    g ~ U(g_range), gamma_x, gamma_y ~ U(gamma_range).  Returns a list of
    (Spec, psi0) with psi0 the anisotropic Gaussian times phase noise."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(sizes[rng.integers(0, len(sizes))])
        g = float(rng.uniform(*g_range))
        gx, gy = (float(v) for v in rng.uniform(*gamma_range, size=2))
        sp = Spec(n=(n, n), lo=(-half_width,) * 2, length=(2 * half_width,) * 2, g=g, dt=dt,
                  gamma=(gx, gy))
        psi = harmonic_gaussian(sp)
        psi = psi * np.exp(1j * rng.uniform(-noise, noise, size=sp.shape))
        out.append((sp, psi))
    return out


def request_stream(count=2000, rate=200.0, seed=0, budget_scale=1.0, max3d=256, max2d=2048):
    """Poisson arrivals (mean `rate` per second) of mixed GPE solves.  Each item is
    a dict with arrival time, Spec, mode ('real' or 'imag'), steps, etol and a
    seed for its initial state.  A third each of 1D 4096, 2D n in
    {256..max2d}^2 and 3D n in {64..max3d}^3; 25% imaginary time."""
    rng = np.random.default_rng(seed)
    t = 0.0
    items = []
    sizes2 = [s for s in (256, 512, 1024, 2048) if s <= max2d]
    sizes3 = [s for s in (64, 128, 256) if s <= max3d]
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        kind = int(rng.integers(0, 3))
        g = float(rng.uniform(0.0, 500.0))
        if kind == 0:
            n = (4096,)
        elif kind == 1:
            s = int(sizes2[rng.integers(0, len(sizes2))])
            n = (s, s)
        else:
            s = int(sizes3[rng.integers(0, len(sizes3))])
            n = (s, s, s)
        d = len(n)
        gam = tuple(float(v) for v in rng.uniform(1.0, 4.0, size=d))
        sp = Spec(n=n, lo=(-12.0,) * d, length=(24.0,) * d, g=g, dt=1e-3, gamma=gam)
        imag = bool(rng.uniform() < 0.25)
        steps = int(rng.integers(100, 2001))
        items.append(dict(t=t, spec=sp, mode="imag" if imag else "real", steps=steps,
                          etol=1e-9, seed=int(rng.integers(0, 2 ** 31))))
    return items
