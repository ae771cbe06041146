"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a brute-force
definition, numpy's FFT, a closed-form solution of the GPE, an exact invariance
of the splitting, or numbers printed in the paper (tests/golden/).  Together
they fail on a dropped factor, a wrong sign, a transposed axis or a wrong
normalisation anywhere in the oracle.
"""
import json
import math
import os

import numpy as np
import pytest

import gpe_inputs as gi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# --------------------------------------------------------------------- FFT
@pytest.mark.parametrize("n", [(1,), (2,), (4,), (8,), (16,), (32,), (64,),
                               (8, 4), (2, 16), (16, 16), (4, 2, 8), (8, 8, 4), (2, 2, 2)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_bruteforce_dft(orc, n, sign):
    rng = np.random.default_rng(sum(n) + sign)
    N = int(np.prod(n))
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    assert rel(orc.fft(x, n, sign), orc.dft_brute(x, n, sign)) < 1e-13


@pytest.mark.parametrize("n", [(256,), (4096,), (128, 64), (32, 16, 8)])
def test_fft_matches_numpy(orc, n):
    rng = np.random.default_rng(7)
    shape = tuple(reversed(n))
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    assert rel(orc.fft(x, n, -1), np.fft.fftn(x)) < 1e-13
    assert rel(orc.fft(x, n, +1), np.fft.ifftn(x) * x.size) < 1e-13


def test_fft_round_trip_and_axis_order(orc):
    # a field varying along x only must transform into the ky=kz=0 plane
    n = (16, 8, 4)
    sp = gi.Spec(n=n, lo=(0, 0, 0), length=(1, 1, 1))
    x = gi.axes(sp)[0]
    f = np.broadcast_to(np.exp(2j * math.pi * 3 * x), (4, 8, 16)).copy()
    F = orc.fft(f, n, -1).reshape(4, 8, 16)
    assert abs(F[0, 0, 3] - 16 * 8 * 4) < 1e-10
    F[0, 0, 3] = 0
    assert np.max(np.abs(F)) < 1e-10
    back = orc.fft(orc.fft(f, n, -1), n, +1) / f.size
    assert rel(back, f) < 1e-14


def test_fft_rejects_non_power_of_two(orc):
    with pytest.raises(RuntimeError):
        orc.fft(np.zeros(12, complex), (12,), -1)


# ------------------------------------------------------- real-time dynamics
@pytest.mark.parametrize("n,modes", [((64,), (3,)), ((32, 16), (2, -1)), ((8, 16, 8), (1, 2, -3))])
def test_plane_wave_is_propagated_exactly(orc, n, modes):
    """V=0: psi = A e^{ik.x} solves the GPE with psi(t) = A e^{i(k.x - (k^2/2 + g A^2) t)},
    and every TSSP substep is exact for it."""
    d = len(n)
    L = [2 * math.pi * 2, 2 * math.pi, 2 * math.pi * 3][:d]
    A, g, dt, steps = 0.7, 2.5, 1e-3, 50
    sp = gi.Spec(n=n, lo=(-1.0,) * d, length=tuple(L), g=g, dt=dt, gamma=(0.0,) * d)
    P = orc.Problem(**sp.kwargs())
    psi0 = gi.plane_wave(sp, modes, A)
    k2 = sum((2 * math.pi * modes[a] / L[a]) ** 2 for a in range(d))
    t = steps * dt
    exact = psi0 * np.exp(-1j * (k2 / 2 + g * A * A) * t)
    assert rel(P.step_real(psi0, steps), exact) < 1e-12


def test_norm_conserved_in_real_time(orc):
    sp = gi.CONFIG_1D
    P = orc.Problem(**sp.kwargs())
    psi0 = gi.gaussian_1d(sp, seed=0)
    n0 = P.norm_energy(psi0)[0]
    psi = P.step_real(psi0, 1000)
    assert abs(P.norm_energy(psi)[0] - n0) < 1e-13


@pytest.mark.parametrize("spec", [
    gi.CONFIG_1D,
    gi.Spec(n=(32, 64), lo=(-6, -8), length=(12, 16), g=50.0, dt=1e-3, gamma=(1.0, 2.0)),
    gi.Spec(n=(16, 8, 32), lo=(-5, -4, -6), length=(10, 8, 12), g=20.0, dt=2e-3,
            gamma=(1.0, 1.5, 3.0)),
])
def test_time_reversal(orc, spec):
    """Each substep is inverted by the same substep with -dt (the nonlinear
    phase does not change |psi|), so S(-dt) S(dt) = identity."""
    P = orc.Problem(**spec.kwargs())
    Pm = P.replace(dt=-spec.dt)
    psi0 = gi.random_field(spec, seed=3, smooth=0.5)
    psi = Pm.step_real(P.step_real(psi0, 20), 20)
    assert rel(psi, psi0) < 1e-12


def test_bright_soliton(orc):
    """g<0, V=0: psi = b/sqrt(-g) sech(bx) e^{i b^2 t/2} is an exact solution."""
    g, b = -2.0, 1.5
    A = b / math.sqrt(-g)
    sp = gi.Spec(n=(512,), lo=(-20.0,), length=(40.0,), g=g, dt=1e-3, gamma=(0.0,))
    x = gi.axes(sp)[0]
    psi0 = (A / np.cosh(b * x)).astype(complex)
    out = orc.Problem(**sp.kwargs()).step_real(psi0, 1000)
    assert rel(out, psi0 * np.exp(1j * b * b * 1.0 / 2)) < 5e-6


def test_bogoliubov_frequency(orc):
    """Small density wave on a uniform condensate oscillates at
    omega = sqrt(k^2/2 (k^2/2 + 2 g rho0)) (linearised GPE)."""
    g, rho0, m, delta = 1.0, 1.0, 3, 1e-5
    L = 2 * math.pi * 4
    sp = gi.Spec(n=(64,), lo=(0.0,), length=(L,), g=g, dt=1e-3, gamma=(0.0,))
    x = gi.axes(sp)[0]
    k = 2 * math.pi * m / L
    w = math.sqrt(k * k / 2 * (k * k / 2 + 2 * g * rho0))
    psi = math.sqrt(rho0) * (1 + delta * np.cos(k * x)) + 0j
    P = orc.Problem(**sp.kwargs())
    t, amps = 0.0, []
    for _ in range(8):
        psi = P.step_real(psi, 400)
        t += 0.4
        rho_hat = np.fft.fft(np.abs(psi) ** 2) / sp.n[0]
        amps.append((t, 2 * rho_hat[m].real))
    for t, a in amps:
        assert abs(a - 2 * delta * math.cos(w * t)) < 2e-3 * 2 * delta


@pytest.mark.parametrize("dt,tol", [(2e-3, 3e-5), (1e-3, 8e-6)])
def test_breathing_gaussian_rms_g0(orc, dt, tol):
    """Dynamics validation setup of the paper at g=0: each axis is a harmonic
    oscillator, so sigma_a^2(t) = eps/(2 gamma_a) cos^2(gamma_a t)
    + 1/(2 gamma_a eps) sin^2(gamma_a t) (Heisenberg evolution of a real
    Gaussian); TSSP error is O(dt^2)."""
    eps = 0.25
    sp = gi.Spec(n=(64, 64, 64), lo=(-8, -6, -4.5), length=(16, 12, 9), g=0.0, dt=dt,
                 gamma=(1, 2, 4))
    P = orc.Problem(**sp.kwargs())
    psi = gi.bao_gaussian(sp)
    T = 0.4
    psi = P.step_real(psi, int(round(T / dt)))
    r = P.rms(psi)
    for a, ga in enumerate((1.0, 2.0, 4.0)):
        ex = math.sqrt(eps / (2 * ga) * math.cos(ga * T) ** 2
                       + 1 / (2 * ga * eps) * math.sin(ga * T) ** 2)
        assert abs(r[a] - ex) / ex < tol
    assert abs(r[3] - math.sqrt(sum(v * v for v in r[:3]))) < 1e-14


# ---------------------------------------------------------- time-dependent trap
def test_constant_trap_schedule_is_the_static_trap(orc):
    """A schedule that keeps the trap fixed runs exactly the static step."""
    sp = gi.Spec(n=(32, 16), lo=(-6, -4), length=(12, 8), g=20.0, dt=1e-3, gamma=(1.0, 1.7))
    psi = gi.random_field(sp, seed=2, smooth=0.1)
    P = orc.Problem(**sp.kwargs())
    gt = np.tile(np.array([1.0, 1.7]), (8, 1))
    assert np.array_equal(P.step_real_trap(psi, gt), P.step_real(psi, 7))


@pytest.mark.parametrize("dt,tol", [(2e-3, 2e-5), (1e-3, 5e-6)])
def test_trap_quench_g0_closed_form(orc, dt, tol):
    """g = 0, the oscillator ground state of gamma0 in a trap switched to
    gamma1 at t = 0: <x^2>(t) = 1/(2 gamma0) cos^2(gamma1 t)
    + gamma0/(2 gamma1^2) sin^2(gamma1 t) per axis (Heisenberg evolution of
    x and p); the schedule holds gamma1 at every time level."""
    g0, g1 = (1.0, 2.0), (2.0, 1.5)
    sp = gi.Spec(n=(64, 64), lo=(-8, -8), length=(16, 16), g=0.0, dt=dt, gamma=g0)
    P = orc.Problem(**sp.kwargs())
    psi = gi.harmonic_gaussian(sp)
    T = 0.6
    ns = int(round(T / dt))
    psi = P.step_real_trap(psi, np.tile(np.array(g1), (ns + 1, 1)))
    r = P.rms(psi)
    for a in range(2):
        ex = math.sqrt(math.cos(g1[a] * T) ** 2 / (2 * g0[a]) + g0[a] / (2 * g1[a] ** 2) * math.sin(g1[a] * T) ** 2)
        assert abs(r[a] - ex) / ex < tol


def _moments_rk4(w2, x2, xp, p2, T, nsub):
    """<x^2>, <xp+px>, <p^2> of H = p^2/2 + w(t)^2 x^2/2 (exact moment
    equations, Heisenberg picture), integrated by classical RK4."""
    h = T / nsub

    def f(t, y):
        a, b, c = y
        return np.array([b, 2 * c - 2 * w2(t) * a, -w2(t) * b])

    y, t = np.array([x2, xp, p2]), 0.0
    for _ in range(nsub):
        k1 = f(t, y)
        k2 = f(t + h / 2, y + h / 2 * k1)
        k3 = f(t + h / 2, y + h / 2 * k2)
        k4 = f(t + h, y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += h
    return y[0]


def test_modulated_trap_g0_matches_moment_equations_at_second_order(orc):
    """g = 0 in a trap whose frequency is modulated, gamma(t) = 1 + 0.5 sin(3 t):
    the width follows the exact moment equations (integrated to 1e-12 by RK4).
    The TSSP error must shrink four-fold when dt halves: evaluating V at the
    wrong time levels would leave a first-order error."""
    w = lambda t: 1.0 + 0.5 * math.sin(3.0 * t)
    T = 0.8
    ref = _moments_rk4(lambda t: w(t) ** 2, 0.5, 0.0, 0.5, T, 20000)
    errs = []
    for dt in (4e-3, 2e-3, 1e-3):
        sp = gi.Spec(n=(256,), lo=(-12,), length=(24,), g=0.0, dt=dt, gamma=(1.0,))
        P = orc.Problem(**sp.kwargs())
        ns = int(round(T / dt))
        gt = np.array([[w(k * dt)] for k in range(ns + 1)])
        psi = P.step_real_trap(gi.harmonic_gaussian(sp), gt)
        errs.append(abs(P.rms(psi)[0] ** 2 - ref))
    assert errs[2] < 2e-6
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


# ---------------------------------------------------------- imaginary time
@pytest.mark.parametrize("spec", [
    gi.Spec(n=(128,), lo=(-10,), length=(20,), g=0.0, dt=1e-3, gamma=(1.0,)),
    gi.Spec(n=(64, 64), lo=(-8, -6), length=(16, 12), g=0.0, dt=1e-3, gamma=(1.0, 2.0)),
    gi.Spec(n=(32, 32, 32), lo=(-6, -4, -3), length=(12, 8, 6), g=0.0, dt=1e-3,
            gamma=(1.0, 2.0, 4.0)),
])
def test_ground_state_g0_is_the_oscillator_gaussian(orc, spec):
    """g=0 ground state: E = mu = sum gamma_a/2, sigma_a^2 = 1/(2 gamma_a)."""
    P = orc.Problem(**spec.kwargs())
    wide = gi.Spec(n=spec.n, lo=spec.lo, length=spec.length,
                   gamma=tuple(0.6 * g_ for g_ in spec.gamma))
    psi0 = gi.harmonic_gaussian(wide)
    psi, steps, E = P.ground(psi0, max_steps=20000, etol=1e-13, check_every=50)
    o = P.norm_energy(psi)
    r = P.rms(psi)
    E0 = sum(spec.gamma) / 2
    assert abs(o[0] - 1.0) < 1e-12
    assert abs(o[4] - E0) / E0 < 1e-6
    assert abs(o[5] - E0) / E0 < 1e-6
    for a in range(spec.ndim):
        s = math.sqrt(1 / (2 * spec.gamma[a]))
        assert abs(r[a] - s) / s < 2e-6


def test_convergence_test_stops_by_its_rule(orc):
    """Convergence test (imaginary time): after every check_every steps (the
    last chunk cut at max_steps) the energy is compared with the previous
    check, the input's energy serving as the first; the run stops at the first
    change below etol and reports that check's energy.  Checked against the
    rule stepped by hand with the oracle's own step and energy: a loose etol
    stops at the first check, etol = 0 runs max_steps (with a partial last
    chunk), and a mid-range etol stops where the hand-run first meets it."""
    sp = gi.Spec(n=(64, 32), lo=(-8, -6), length=(16, 12), g=20.0, dt=2e-3, gamma=(1.0, 1.5))
    P = orc.Problem(**sp.kwargs())
    psi0 = gi.harmonic_gaussian(gi.Spec(n=sp.n, lo=sp.lo, length=sp.length, gamma=(0.5, 0.5)))

    def by_hand(max_steps, etol, every):
        y = psi0.astype(np.complex128)
        eprev = P.norm_energy(y)[4]
        done = 0
        while done < max_steps:
            chunk = min(every, max_steps - done)
            y = P.step_imag(y, chunk)
            done += chunk
            e = P.norm_energy(y)[4]
            if abs(e - eprev) < etol:
                return y, done, e
            eprev = e
        return y, done, eprev

    # loose tolerance: the first check already meets it
    psi, steps, E = P.ground(psi0, max_steps=1000, etol=1e3, check_every=7)
    assert steps == 7
    # etol = 0 never stops early; 23 = 3 * 7 + 2 leaves a 2-step last chunk
    psi, steps, E = P.ground(psi0, max_steps=23, etol=0.0, check_every=7)
    ref, rsteps, rE = by_hand(23, 0.0, 7)
    assert steps == 23 == rsteps and E == rE and np.array_equal(psi, ref)
    assert E == P.norm_energy(psi)[4]
    # a tolerance met part-way: the same stopping check as the hand-run, and
    # the energy change there is below etol while the one before is not
    psi, steps, E = P.ground(psi0, max_steps=5000, etol=1e-6, check_every=10)
    ref, rsteps, rE = by_hand(5000, 1e-6, 10)
    assert 10 < steps < 5000 and steps == rsteps and E == rE and np.array_equal(psi, ref)
    e_before = P.norm_energy(P.step_imag(psi0.astype(np.complex128), steps - 10))[4]
    assert abs(E - e_before) < 1e-6
    e_two_before = P.norm_energy(P.step_imag(psi0.astype(np.complex128), steps - 20))[4]
    assert abs(e_before - e_two_before) >= 1e-6


def test_table1_2d_ground_states(orc):
    """2D rows of the paper's Table 1 (r_rms and mu of the ground state in
    V=(x^2+y^2)/2 from psi0 = pi^-1/2 e^{-r^2/2}).  128^2 on [-10,10)^2 at
    dt=1e-3 reproduces every printed row to better than 1e-5 relative."""
    rows = json.load(open(os.path.join(GOLDEN, "table1_2d.json")))["rows"]
    for g, r_ref, mu_ref in rows:
        sp = gi.Spec(n=(128, 128), lo=(-10, -10), length=(20, 20), g=g, dt=1e-3,
                     gamma=(1.0, 1.0))
        P = orc.Problem(**sp.kwargs())
        psi, steps, E = P.ground(gi.harmonic_gaussian(sp), max_steps=40000, etol=1e-12,
                                 check_every=50)
        r = P.rms(psi)[3]
        mu = P.norm_energy(psi)[5]
        assert abs(r - r_ref) / r_ref < 2e-5, (g, r, r_ref)
        assert abs(mu - mu_ref) / mu_ref < 2e-5, (g, mu, mu_ref)


def test_imag_step_renormalises(orc):
    sp = gi.Spec(n=(32, 32), lo=(-6, -6), length=(12, 12), g=30.0, dt=1e-3, gamma=(1, 1))
    P = orc.Problem(**sp.kwargs())
    psi = P.step_imag(gi.random_field(sp, seed=1, smooth=0.3) * 3.0, 5, target_norm=2.5)
    assert abs(P.norm_energy(psi)[0] - 2.5) < 1e-12


# -------------------------------------------------------------- diagnostics
def test_energy_of_plane_wave(orc):
    n = (32, 16)
    L = (2 * math.pi * 2, 2 * math.pi)
    A, g = 0.8, 3.0
    sp = gi.Spec(n=n, lo=(0, 0), length=L, g=g, gamma=(0.0, 0.0))
    psi = gi.plane_wave(sp, (3, -2), A)
    o = orc.Problem(**sp.kwargs()).norm_energy(psi)
    vol = L[0] * L[1]
    k2 = (2 * math.pi * 3 / L[0]) ** 2 + (2 * math.pi * 2 / L[1]) ** 2
    assert abs(o[0] - A * A * vol) < 1e-12 * vol
    assert abs(o[1] - 0.5 * k2 * A * A * vol) < 1e-11 * vol
    assert abs(o[2]) < 1e-15
    assert abs(o[3] - 0.5 * g * A ** 4 * vol) < 1e-12 * vol
    assert abs(o[5] - (0.5 * k2 + g * A * A)) < 1e-12


def test_energy_of_oscillator_gaussian(orc):
    sp = gi.Spec(n=(64, 32, 32), lo=(-8, -5, -4), length=(16, 10, 8), g=0.0,
                 gamma=(1.0, 2.0, 3.0))
    psi = gi.harmonic_gaussian(sp)
    o = orc.Problem(**sp.kwargs()).norm_energy(psi)
    assert abs(o[0] - 1) < 1e-12
    # kinetic and potential each carry half of gamma/2 per axis
    assert abs(o[1] - 1.5) < 1e-10 and abs(o[2] - 1.5) < 1e-10
    assert abs(o[4] - 3.0) < 1e-10


# ------------------------------------------------------------------ spectra
def _velocity(psi, sp):
    """u_a = Im(conj psi d_a psi)/|psi| with numpy spectral derivatives."""
    ks = [2 * math.pi * np.fft.fftfreq(sp.n[a], d=sp.length[a] / sp.n[a]) for a in range(sp.ndim)]
    for a in range(sp.ndim):
        if sp.n[a] % 2 == 0:
            ks[a][sp.n[a] // 2] = 0.0
    K = list(reversed(np.meshgrid(*reversed(ks), indexing="ij")))
    ph = np.fft.fftn(psi)
    rho = np.abs(psi) ** 2
    us = []
    for a in range(sp.ndim):
        d = np.fft.ifftn(1j * K[a] * ph)
        us.append(np.where(rho >= 1e-30, np.imag(np.conj(psi) * d) / np.sqrt(np.maximum(rho, 1e-300)), 0.0))
    return us


@pytest.mark.parametrize("sp", [
    gi.Spec(n=(64, 64), lo=(0, 0), length=(2 * math.pi * 4,) * 2, g=1.0),
    gi.Spec(n=(32, 16, 16), lo=(0, 0, 0), length=(2 * math.pi * 2, 2 * math.pi, 2 * math.pi),
            g=1.0),
])
def test_spectrum_parseval(orc, sp):
    psi, _, _ = gi.vortex_field_2d(sp, nv=8, seed=2) if sp.ndim == 2 else (
        gi.random_field(sp, seed=4, smooth=0.05), None, None)
    ei, ec = orc.Problem(**sp.kwargs()).spectrum(psi)
    us = _velocity(psi, sp)
    half_u2 = 0.5 * sum(np.sum(u * u) for u in us) * sp.cell_volume()
    assert abs((ei.sum() + ec.sum()) - half_u2) < 1e-12 * half_u2


def test_spectrum_irrotational_has_no_incompressible_part(orc):
    sp = gi.Spec(n=(64, 32), lo=(0, 0), length=(2 * math.pi, 2 * math.pi), g=1.0)
    x, y = gi.axes(sp)
    th = 0.3 * np.sin(2 * x)[None, :] + 0.2 * np.cos(3 * y)[:, None]
    ei, ec = orc.Problem(**sp.kwargs()).spectrum(np.exp(1j * th))
    assert ec.sum() > 1e-2
    assert ei.sum() < 1e-13 * ec.sum()


def test_spectrum_solenoidal_has_no_compressible_part(orc):
    sp = gi.Spec(n=(32, 64), lo=(0, 0), length=(2 * math.pi, 2 * math.pi), g=1.0)
    x, y = gi.axes(sp)
    rho = 1.0 + 0.5 * np.cos(y)[:, None] + 0 * x[None, :]
    psi = np.sqrt(rho) * np.exp(1j * 2 * x)[None, :]
    ei, ec = orc.Problem(**sp.kwargs()).spectrum(psi)
    assert ei.sum() > 1e-2
    assert ec.sum() < 1e-13 * ei.sum()


def test_spectrum_shell_count(orc):
    sp = gi.Spec(n=(1024, 1024), lo=(0, 0), length=(2 * math.pi * 32,) * 2, g=1.0)
    assert orc.Problem(**sp.kwargs()).nshells() == 725      # round(sqrt(2)*512) + 1


# ------------------------------------------------------- input generators
def test_vortex_field_is_periodic_and_winds_once_per_vortex():
    sp = gi.Spec(n=(128, 128), lo=(0, 0), length=(2 * math.pi * 8,) * 2, g=1.0)
    psi, pos, q = gi.vortex_field_2d(sp, nv=16, seed=1)
    th = np.angle(psi)
    h = sp.length[0] / sp.n[0]
    # edge continuity: the wrapped phase jump across each periodic edge is no
    # larger than the largest jump between interior neighbours
    wrap = lambda d: (d + math.pi) % (2 * math.pi) - math.pi
    inner = max(np.max(np.abs(wrap(np.diff(th, axis=0)))), np.max(np.abs(wrap(np.diff(th, axis=1)))))
    assert np.max(np.abs(wrap(th[:, 0] - th[:, -1]))) <= inner + 1e-9
    assert np.max(np.abs(wrap(th[0, :] - th[-1, :]))) <= inner + 1e-9
    # winding number around each vortex on a small square loop
    x, y = gi.axes(sp)
    for (px, py), qj in zip(pos, q):
        r = 1.2
        pts = [(px + r * math.cos(t), py + r * math.sin(t)) for t in np.linspace(0, 2 * math.pi, 65)]
        ang = []
        for xx, yy in pts:
            i = int(round((xx % sp.length[0]) / h)) % sp.n[0]
            j = int(round((yy % sp.length[1]) / h)) % sp.n[1]
            ang.append(th[j, i])
        wind = sum(wrap(ang[i + 1] - ang[i]) for i in range(len(ang) - 1)) / (2 * math.pi)
        assert round(wind) == qj


# -------------------------------------------------------------- sampled potential
# The model equation allows any potential V(r) (Eq. ndGPE); the oracle takes V
# sampled at the grid points.  Pins: a constant potential only adds the global
# phase exp(-i V0 t) in real time (every substep commutes with it), is removed
# by the renormalisation in imaginary time, and shifts E and mu by V0 (norm 1).
def _sp_v():
    return gi.Spec(n=(32, 16, 8), lo=(-6.0, -5.0, -4.0), length=(12.0, 10.0, 8.0), g=40.0, dt=2e-3,
                   gamma=(0.0, 0.0, 0.0))


def test_constant_potential_is_a_global_phase(orc):
    sp = _sp_v()
    psi0 = gi.random_field(sp, seed=4, smooth=0.1)
    v0, steps = 3.7, 25
    ref = orc.Problem(**sp.kwargs()).step_real(psi0, steps)
    out = orc.Problem(**sp.kwargs(), V=np.full(sp.shape, v0)).step_real(psi0, steps)
    expect = ref * np.exp(-1j * v0 * steps * sp.dt)
    assert np.max(np.abs(out - expect)) < 1e-12 * np.max(np.abs(ref))


def test_constant_potential_drops_out_of_imaginary_time(orc):
    """At g = 0 the factor exp(-V0 tau) commutes with every substep and the
    renormalisation removes it.  (At g != 0 it would not: the second nonlinear
    half-step sees |psi|^2 already scaled by the first.)"""
    sp = gi.Spec(n=_sp_v().n, lo=_sp_v().lo, length=_sp_v().length, g=0.0, dt=2e-3, gamma=(0.0, 0.0, 0.0))
    psi0 = gi.random_field(sp, seed=5, smooth=0.1)
    v0 = 2.5
    a = orc.Problem(**sp.kwargs()).step_imag(psi0, 12)
    b = orc.Problem(**sp.kwargs(), V=np.full(sp.shape, v0)).step_imag(psi0, 12)
    assert np.max(np.abs(a - b)) < 1e-12


def test_constant_potential_shifts_energy_and_mu(orc):
    sp = _sp_v()
    psi = gi.random_field(sp, seed=5, smooth=0.1)
    v0 = 2.5
    e0 = orc.Problem(**sp.kwargs()).norm_energy(psi)
    e1 = orc.Problem(**sp.kwargs(), V=np.full(sp.shape, v0)).norm_energy(psi)
    assert abs(e1[2] - (e0[2] + v0 * e0[0])) < 1e-11 * e0[0]
    assert abs(e1[4] - (e0[4] + v0 * e0[0])) < 1e-11 * e0[0]
    assert abs(e1[5] - (e0[5] + v0)) < 1e-11


def test_sampled_potential_follows_the_grid_points(orc):
    """V sampled at x_j = lo + j*L/n equals the built-in harmonic trap there, and
    E_pot is the grid sum of V |psi|^2 dV."""
    sp = gi.Spec(n=(16, 32, 8), lo=(-4.0, -6.0, -3.0), length=(8.0, 12.0, 6.0), g=10.0, dt=1e-3,
                 gamma=(1.0, 1.5, 2.0))
    psi0 = gi.random_field(sp, seed=6, smooth=0.1)
    mesh = gi._mesh(sp)
    V = sum(0.5 * sp.gamma[a] ** 2 * mesh[a] ** 2 for a in range(3))
    a = orc.Problem(**sp.kwargs()).step_real(psi0, 9)
    b = orc.Problem(**dict(sp.kwargs(), gamma=(0.0, 0.0, 0.0)), V=V).step_real(psi0, 9)
    assert np.max(np.abs(a - b)) < 1e-12
    lat = gi.optical_lattice(sp, v0=4.0, periods=2)
    e = orc.Problem(**dict(sp.kwargs(), gamma=(0.0, 0.0, 0.0)), V=lat).norm_energy(psi0)
    dv = np.prod([sp.length[i] / sp.n[i] for i in range(3)])
    assert abs(e[2] - np.sum(lat * np.abs(psi0) ** 2) * dv) < 1e-12 * abs(e[2])


# ------------------------------------------------ quantum-pressure / number spectra
def _band_limited(sp, seed, kmax_frac=0.25):
    """Smooth complex field whose Fourier modes all lie below kmax_frac * n/2 on
    every axis, with |psi| bounded away from 0 (no Nyquist content, no zeros)."""
    rng = np.random.default_rng(seed)
    ph = np.zeros(sp.shape, complex)
    sl = tuple(slice(0, max(1, int(kmax_frac * n / 2))) for n in reversed(sp.n))
    ph[sl] = rng.normal(size=ph[sl].shape) + 1j * rng.normal(size=ph[sl].shape)
    f = np.fft.ifftn(ph)
    f = f / np.max(np.abs(f))
    return 2.0 + f + 0.3j * np.conj(f) * f


@pytest.mark.parametrize("sp", [
    gi.Spec(n=(32, 16), lo=(0, 0), length=(8.0, 4.0), g=1.0, gamma=(0.0, 0.0)),
    gi.Spec(n=(16, 8, 32), lo=(0, 0, 0), length=(4.0, 2.0, 8.0), g=1.0, gamma=(0.0, 0.0, 0.0)),
])
def test_spectra_add_up_to_the_kinetic_energy_and_the_norm(orc, sp):
    """|grad psi|^2 = |grad |psi||^2 + |psi|^2 |grad theta|^2 point by point, so the
    incompressible, compressible and quantum-pressure spectra sum to E_kin (for a
    field without Nyquist content); the particle-number spectrum sums to the norm."""
    P = orc.Problem(**sp.kwargs())
    psi = _band_limited(sp, seed=7)
    ei, ec = P.spectrum(psi)
    eq, nn = P.spectrum_qp_num(psi)
    e = P.norm_energy(psi)
    assert abs(ei.sum() + ec.sum() + eq.sum() - e[1]) < 1e-11 * e[1]
    assert abs(nn.sum() - e[0]) < 1e-12 * e[0]


def test_real_positive_field_is_all_quantum_pressure(orc):
    sp = gi.Spec(n=(32, 32), lo=(-4, -4), length=(8.0, 8.0), g=1.0, gamma=(0.0, 0.0))
    psi = np.abs(_band_limited(sp, seed=3)).astype(complex)
    psi = np.real(np.fft.ifftn(np.where(np.abs(np.fft.fftfreq(32))[None, :] < 0.2, 1, 0)
                               * np.where(np.abs(np.fft.fftfreq(32))[:, None] < 0.2, 1, 0)
                               * np.fft.fftn(psi))).astype(complex) + 0.5
    P = orc.Problem(**sp.kwargs())
    ei, ec = P.spectrum(psi)
    eq, nn = P.spectrum_qp_num(psi)
    e = P.norm_energy(psi)
    assert ei.sum() < 1e-25 and ec.sum() < 1e-25
    assert abs(eq.sum() - e[1]) < 1e-11 * e[1]


def test_uniform_density_plane_wave_has_no_quantum_pressure(orc):
    sp = gi.Spec(n=(32, 16), lo=(0, 0), length=(2 * math.pi * 2, 2 * math.pi), g=1.0, gamma=(0.0, 0.0))
    psi = gi.plane_wave(sp, (3, -2), 0.8)
    P = orc.Problem(**sp.kwargs())
    eq, nn = P.spectrum_qp_num(psi)
    assert eq.sum() < 1e-25
    # all particles sit in the plane wave's shell: n = round(|m| dk_ratio) for m = (3, -2)
    k = math.sqrt(3 ** 2 + (2 * 2) ** 2)          # mode numbers in units of 2 pi / max L
    assert abs(nn[int(round(k))] - P.norm_energy(psi)[0]) < 1e-12 * nn.sum()
