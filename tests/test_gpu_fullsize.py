"""Parity at the full workload sizes, in the launch configuration bench.py times.

The oracle runs whole steps of the same grids on the host cores (a few seconds
per 512^3 step); longer runs are checked through properties that hold at any
size: norm conservation and exact time reversal of the splitting.
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


def plan_for(gpe, sp, prec):
    return gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=prec)


@pytest.fixture(scope="module")
def tg512():
    return gi.taylor_green_3d(gi.CONFIG_3D_TG, seed=0)          # complex64, 1 GiB


def test_tg512_one_step_matches_oracle(gpe, orc, tg512):
    import torch
    sp = gi.CONFIG_3D_TG
    x = torch.from_numpy(tg512).cuda()
    p = plan_for(gpe, sp, gpe.GPE_C64)
    p.step_real(x, 1)
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    del x
    p.close()
    ref = orc.Problem(**sp.kwargs()).step_real(tg512.astype(np.complex128), 1)
    assert rel(out, ref) < 2e-6


def test_tg512_norm_and_time_reversal_over_100_steps(gpe, tg512):
    import torch
    sp = gi.CONFIG_3D_TG
    fwd = plan_for(gpe, sp, gpe.GPE_C64)
    back = plan_for(gpe, gi.Spec(n=sp.n, lo=sp.lo, length=sp.length, g=sp.g, dt=-sp.dt), gpe.GPE_C64)
    x = torch.from_numpy(tg512).cuda()
    n0 = fwd.norm_energy(x)[0]
    fwd.step_real(x, 100)
    n1 = fwd.norm_energy(x)[0]
    back.step_real(x, 100)
    torch.cuda.synchronize()
    assert abs(n1[0] / n0[0] - 1) < 1e-6
    x0 = torch.from_numpy(tg512).cuda()
    err = float(torch.linalg.vector_norm((x - x0).to(torch.complex128)) /
                torch.linalg.vector_norm(x0.to(torch.complex128)))
    assert err < 1e-5


@pytest.fixture(scope="module")
def turb1024():
    psi, _, _ = gi.vortex_field_2d(gi.CONFIG_2D, nv=512, seed=0)
    return psi


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 2e-5)], ids=["c128", "c64"])
def test_turbulence_1024_twenty_steps_match_oracle(gpe, orc, turb1024, prec, tol):
    import torch
    sp = gi.CONFIG_2D
    dt = np.complex128 if prec == 1 else np.complex64
    x = torch.from_numpy(turb1024.astype(dt)).cuda()
    p = plan_for(gpe, sp, prec)
    p.step_real(x, 20)
    torch.cuda.synchronize()
    ref = orc.Problem(**sp.kwargs()).step_real(turb1024.astype(dt).astype(np.complex128), 20)
    assert rel(x.cpu().numpy(), ref) < tol
    p.close()


def test_turbulence_1024_spectrum_matches_oracle(gpe, orc, turb1024):
    import torch
    sp = gi.CONFIG_2D
    ei, ec = orc.Problem(**sp.kwargs()).spectrum(turb1024)
    p = plan_for(gpe, sp, gpe.GPE_C128)
    out = p.spectrum(torch.from_numpy(turb1024).cuda())
    assert out.shape == (2, 1, 725)
    scale = max(ei.max(), ec.max())
    assert np.max(np.abs(out[0, 0] - ei)) < 1e-10 * scale
    assert np.max(np.abs(out[1, 0] - ec)) < 1e-10 * scale
    p.close()


def test_trap256_imaginary_steps_match_oracle(gpe, orc):
    import torch
    sp = gi.CONFIG_3D_TRAP
    psi0 = gi.harmonic_gaussian(sp)
    steps = 4
    ref = orc.Problem(**sp.kwargs()).step_imag(psi0, steps)
    p = plan_for(gpe, sp, gpe.GPE_C64)
    x = torch.from_numpy(psi0.astype(np.complex64)).cuda()
    done, _ = p.step_imag(x, steps, etol=0.0, check_every=steps)
    torch.cuda.synchronize()
    assert done == steps
    assert rel(x.cpu().numpy(), ref) < 2e-5
    e = p.norm_energy(x)[0]
    assert abs(e[0] - 1.0) < 1e-6
    p.close()
