"""Time-dependent harmonic trap (gpe_step_real_trap) against the oracle.

A schedule of trap frequencies per time level replaces the plan's static trap.
The library merges the nonlinear half-steps next to each time level; the oracle
applies them unmerged, so the two agree to rounding: complex128 relative L2
<= 1e-12, complex64 <= 2e-5 over these short runs.  The quench case is also
checked against its closed form (g = 0).
"""
import math

import numpy as np
import pytest

import gpe_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpe():
    import torch
    import paper_2301_08275_gb300 as g
    g.build()
    g.lib()
    assert torch.cuda.is_available()
    return g


def rel(a, b):
    a = np.ravel(np.asarray(a, dtype=np.complex128))
    b = np.ravel(np.asarray(b, dtype=np.complex128))
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def schedule(ndim, steps, dt, seed):
    """trap frequencies modulated in time, with a quench halfway"""
    rng = np.random.default_rng(seed)
    base = rng.uniform(1.0, 2.5, size=ndim)
    amp = rng.uniform(0.1, 0.4, size=ndim)
    t = np.arange(steps + 1)[:, None] * dt
    g = base * (1.0 + amp * np.sin(7.0 * t + np.arange(ndim)))
    g[steps // 2 + 1:] *= 1.5
    return g


CASES = [(128,), (64, 32), (16, 32, 64)]


@pytest.mark.parametrize("n", CASES, ids=lambda n: "x".join(map(str, n)))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_trap_schedule_matches_oracle(gpe, orc, n, prec):
    import torch
    d = len(n)
    L = [12.0, 10.0, 8.0][:d]
    sp = gi.Spec(n=n, lo=tuple(-x / 2 for x in L), length=tuple(L), g=25.0, dt=1e-3, gamma=(1.0, 1.0, 1.0)[:d])
    psi0 = gi.random_field(sp, seed=sum(n), smooth=0.05)
    steps = 40
    gt = schedule(d, steps, sp.dt, seed=d)
    ref = orc.Problem(**sp.kwargs()).step_real_trap(psi0, gt)
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    dt = np.complex128 if prec == "c128" else np.complex64
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=pv)
    x = torch.from_numpy(psi0.astype(dt)).cuda()
    p.step_real_trap(x, gt)
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    p.close()
    assert rel(out, ref) < (1e-12 if prec == "c128" else 2e-5)


def test_trap_schedule_on_an_untrapped_plan_and_in_pieces(gpe, orc):
    """The schedule traps axes the plan leaves free, and two calls over the two
    halves of a schedule give the run of one call (to rounding)."""
    import torch
    sp = gi.Spec(n=(64, 64), lo=(-8.0, -8.0), length=(16.0, 16.0), g=10.0, dt=1e-3)
    psi0 = gi.random_field(sp, seed=5, smooth=0.05)
    gt = schedule(2, 30, sp.dt, seed=9)
    ref = orc.Problem(**sp.kwargs()).step_real_trap(psi0, gt)
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, prec=gpe.GPE_C128)
    x = torch.from_numpy(psi0.copy()).cuda()
    p.step_real_trap(x, gt[:16])
    p.step_real_trap(x, gt[15:])
    torch.cuda.synchronize()
    assert rel(x.cpu().numpy(), ref) < 1e-12
    with pytest.raises(gpe.GpeError):
        p.step_real_trap(x, np.full((3, 2), np.nan))
    p.close()


def test_trap_quench_closed_form_on_gpu(gpe):
    """g = 0 oscillator ground state of gamma0, trap switched to gamma1:
    sigma_a^2(t) = cos^2(g1 t)/(2 g0) + g0 sin^2(g1 t)/(2 g1^2), 3D complex64."""
    import torch
    g0, g1 = (1.0, 2.0, 1.5), (2.0, 1.0, 3.0)
    sp = gi.Spec(n=(64, 64, 64), lo=(-8.0,) * 3, length=(16.0,) * 3, g=0.0, dt=1e-3, gamma=g0)
    T = 0.5
    ns = int(round(T / sp.dt))
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=0.0, dt=sp.dt, gamma=g0, prec=gpe.GPE_C64)
    x = torch.from_numpy(gi.harmonic_gaussian(sp).astype(np.complex64)).cuda()
    p.step_real_trap(x, np.tile(np.array(g1), (ns + 1, 1)))
    r = p.rms_size(x)[0]
    p.close()
    for a in range(3):
        ex = math.sqrt(math.cos(g1[a] * T) ** 2 / (2 * g0[a]) + g0[a] / (2 * g1[a] ** 2) * math.sin(g1[a] * T) ** 2)
        assert abs(r[a] - ex) / ex < 2e-5
