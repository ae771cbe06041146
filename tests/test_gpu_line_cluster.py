"""The cluster kernel of complex128 1D real-time steps (one line of 64, 128 or
256 points spread over 4, 8 or 16 CTAs) against the FP64 oracle and against
the one-CTA-per-line kernel (GPE_OPT_LINE_CLUSTER = 0).

Both kernels compute the split-step scheme in FP64 with different
factorisations of the transform, so they agree to rounding: relative L2
<= 1e-12 against the oracle (the library-wide complex128 tolerance), <= 1e-13
between the two kernels over 50 steps.
"""
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


def spec(n, g=30.0, trap=True, dt=1e-3):
    return gi.Spec(n=(n,), lo=(-8.0,), length=(16.0,), g=g, dt=dt, gamma=(1.3 if trap else 0.0,))


def run(gpe, sp, psi0, steps, cluster, batch=1, g_each=None):
    import torch
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C128, batch=batch,
                 g_each=g_each)
    p.set_option(gpe.GPE_OPT_LINE_CLUSTER, 1 if cluster else 0)
    x = torch.from_numpy(np.ascontiguousarray(psi0, dtype=np.complex128)).cuda()
    p.step_real(x, steps)
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    p.close()
    return out


@pytest.mark.parametrize("n", [64, 128, 256])
@pytest.mark.parametrize("trap", [True, False], ids=["trap", "free"])
def test_cluster_line_matches_oracle_and_one_cta_kernel(gpe, orc, n, trap):
    sp = spec(n, trap=trap)
    psi0 = gi.random_field(sp, seed=n + trap, smooth=0.05)
    steps = 50
    ref = orc.Problem(**sp.kwargs()).step_real(psi0, steps)
    out = run(gpe, sp, psi0, steps, cluster=True)
    one = run(gpe, sp, psi0, steps, cluster=False)
    assert rel(out, ref) < 1e-12
    assert rel(out, one) < 1e-13


@pytest.mark.parametrize("n,batch", [(64, 3), (256, 5), (128, 32), (128, 33)])
def test_cluster_batches_match_oracle_per_instance(gpe, orc, n, batch):
    """Instances with their own g, one cluster per line; 33 lines are above the
    cluster kernel's batch limit and take the one-CTA kernel (same results to
    rounding)."""
    sp = spec(n)
    g_each = [5.0 + 7.0 * b for b in range(batch)]
    psi0 = np.stack([gi.random_field(sp, seed=100 + b, smooth=0.05) for b in range(batch)])
    steps = 9
    out = run(gpe, sp, psi0, steps, cluster=True, batch=batch, g_each=g_each)
    for b in sorted({0, batch // 2, batch - 1}):
        sb = gi.Spec(n=sp.n, lo=sp.lo, length=sp.length, g=g_each[b], dt=sp.dt, gamma=sp.gamma)
        ref = orc.Problem(**sb.kwargs()).step_real(psi0[b], steps)
        assert rel(out[b], ref) < 1e-12, b


def test_cluster_line_large_nonlinear_angles(gpe, orc):
    """A dense cloud at g = 2000: angles above 1/16 (library sincos, up to 1.1)
    at the centre, below it (series) in the tails."""
    sp = gi.Spec(n=(256,), lo=(-6.0,), length=(12.0,), g=2000.0, dt=1e-3, gamma=(1.0,))
    psi0 = gi.harmonic_gaussian(sp, seed=3, noise=0.01)
    th = sp.g * sp.dt * np.abs(psi0) ** 2
    assert th.max() > 0.5 and np.any(th < 0.0625)
    steps = 5
    ref = orc.Problem(**sp.kwargs()).step_real(psi0, steps)
    assert rel(run(gpe, sp, psi0, steps, cluster=True), ref) < 1e-12


def test_cluster_line_1000_steps_single_step_calls_and_norm(gpe, orc):
    """The 1D workload (256 points, V = x^2/2, g = 10) over 1000 steps in one
    call: the oracle's state to 1e-12 and the norm to 1e-13; and one step per
    call (each call opens and closes with a nonlinear half-step) against the
    oracle's single steps."""
    import torch
    sp = gi.CONFIG_1D
    psi0 = gi.gaussian_1d(sp, seed=0)
    pr = orc.Problem(**sp.kwargs())
    ref = pr.step_real(psi0, 1000)
    out = run(gpe, sp, psi0, 1000, cluster=True)
    assert rel(out, ref) < 1e-12
    assert abs(pr.norm_energy(out)[0] / pr.norm_energy(psi0)[0] - 1) < 1e-13
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C128)
    x = torch.from_numpy(psi0.copy()).cuda()
    for _ in range(5):
        p.step_real(x, 1)
    torch.cuda.synchronize()
    p.close()
    assert rel(x.cpu().numpy(), pr.step_real(psi0, 5)) < 1e-12


def test_cluster_line_with_trap_schedule(gpe, orc):
    """Time-dependent trap, one launch per step with the tables of both time
    levels (the last half-step takes its own table)."""
    import torch
    sp = gi.Spec(n=(128,), lo=(-6.0,), length=(12.0,), g=25.0, dt=1e-3, gamma=(1.0,))
    psi0 = gi.random_field(sp, seed=11, smooth=0.05)
    t = np.arange(31)[:, None] * sp.dt
    gt = 1.5 * (1.0 + 0.3 * np.sin(9.0 * t))
    ref = orc.Problem(**sp.kwargs()).step_real_trap(psi0, gt)
    outs = []
    for cluster in (1, 0):
        p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C128)
        p.set_option(gpe.GPE_OPT_LINE_CLUSTER, cluster)
        x = torch.from_numpy(psi0.copy()).cuda()
        p.step_real_trap(x, gt)
        torch.cuda.synchronize()
        p.close()
        outs.append(x.cpu().numpy())
    assert rel(outs[0], ref) < 1e-12
    assert rel(outs[0], outs[1]) < 1e-13


def test_cluster_option_round_trip(gpe):
    sp = spec(64)
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C128)
    assert p.get_option(gpe.GPE_OPT_LINE_CLUSTER) == 1
    p.set_option(gpe.GPE_OPT_LINE_CLUSTER, 0)
    assert p.get_option(gpe.GPE_OPT_LINE_CLUSTER) == 0
    p.close()
