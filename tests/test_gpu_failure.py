"""Failure handling on the GPU without a fault: a copy wait that runs out of
its time limit is reported as GPE_ETIMEOUT by the next synchronising call and
leaves the context usable (no trap, no hang, no bad address)."""
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


def test_copy_wait_that_runs_out_is_reported_and_the_context_survives(gpe):
    import torch
    sp = gi.Spec(n=(64, 64), lo=(-6.0, -6.0), length=(12.0, 12.0), g=10.0, dt=1e-3, gamma=(1.0, 1.0))
    psi0 = gi.harmonic_gaussian(sp).astype(np.complex64)
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C64)
    p.set_option(gpe.GPE_OPT_TMA_STAGING, 1)
    p.set_option(gpe.GPE_OPT_TEST_STALL_COPIES, 1)       # every y-tile wait expects 16 bytes too many
    x = torch.from_numpy(psi0.copy()).cuda()
    p.step_real(x, 1)                                     # asynchronous: no error yet
    with pytest.raises(gpe.GpeError) as ei:
        p.norm_energy(x)                                  # synchronises, reads the error word
    assert ei.value.status == 6                           # GPE_ETIMEOUT
    # the context still works: the same plan with the hook off agrees with a fresh plan
    p.set_option(gpe.GPE_OPT_TEST_STALL_COPIES, 0)
    q = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C64)
    y = torch.from_numpy(psi0.copy()).cuda()
    z = torch.from_numpy(psi0.copy()).cuda()
    p.step_real(y, 5)
    q.step_real(z, 5)
    e = p.norm_energy(y)
    torch.cuda.synchronize()
    assert torch.equal(y, z)
    assert abs(e[0][0] - 1.0) < 1e-5
    p.close()
    q.close()


def test_cluster_exchange_wait_that_runs_out_is_reported(gpe):
    """The 1D cluster kernel's exchange waits are bounded the same way: with
    the hook every wait expects 16 bytes more than arrive, each CTA gives up
    after its limit, all leave together, and GPE_ETIMEOUT is reported; the
    context then computes correct results."""
    import torch
    sp = gi.CONFIG_1D
    psi0 = gi.gaussian_1d(sp, seed=0)
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C128)
    assert p.get_option(gpe.GPE_OPT_LINE_CLUSTER) == 1
    p.set_option(gpe.GPE_OPT_TEST_STALL_COPIES, 1)
    x = torch.from_numpy(psi0.copy()).cuda()
    p.step_real(x, 3)
    with pytest.raises(gpe.GpeError) as ei:
        p.norm_energy(x)
    assert ei.value.status == 6                           # GPE_ETIMEOUT
    p.set_option(gpe.GPE_OPT_TEST_STALL_COPIES, 0)
    q = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C128)
    y = torch.from_numpy(psi0.copy()).cuda()
    z = torch.from_numpy(psi0.copy()).cuda()
    p.step_real(y, 5)
    q.step_real(z, 5)
    torch.cuda.synchronize()
    assert torch.equal(y, z)
    p.close()
    q.close()
