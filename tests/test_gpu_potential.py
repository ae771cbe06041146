"""Sampled potentials (desc.V_host) against the oracle: real and imaginary
time, diagnostics, 1D/2D/3D, both precisions."""
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


def _case(n, kind):
    d = len(n)
    L = [12.0, 10.0, 8.0][:d]
    sp = gi.Spec(n=n, lo=tuple(-x / 2 for x in L), length=tuple(L), g=30.0, dt=1e-3, gamma=(0.0,) * d)
    if kind == "lattice":
        V = gi.optical_lattice(sp, v0=8.0, periods=3, gamma=(1.0, 1.5, 2.0)[:d])
    else:
        V = gi.anharmonic(sp, gamma=(1.0, 1.3, 1.7)[:d], lam=0.2)
    return sp, V


SHAPES = [(256,), (64, 32), (32, 16, 8), (16, 64, 32)]


@pytest.mark.parametrize("kind", ["lattice", "anharmonic"])
@pytest.mark.parametrize("n", SHAPES, ids=lambda n: "x".join(map(str, n)))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_sampled_potential_real_time_and_energy(gpe, orc, n, kind, prec):
    import torch
    sp, V = _case(n, kind)
    psi0 = gi.random_field(sp, seed=sum(n), smooth=0.05)
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    dt = np.complex128 if prec == "c128" else np.complex64
    P = orc.Problem(**sp.kwargs(), V=V)
    ref = P.step_real(psi0, 9)
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, prec=pv, V=V)
    x = torch.from_numpy(psi0.astype(dt)).cuda()
    p.step_real(x, 9)
    e = p.norm_energy(x)[0]
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    assert rel(out, ref) < (1e-12 if prec == "c128" else 2e-5)
    e_ref = P.norm_energy(out.astype(np.complex128))
    tol = 1e-11 if prec == "c128" else 1e-5
    assert np.allclose(e, e_ref, rtol=tol, atol=tol * abs(e_ref[4]))
    p.close()


@pytest.mark.parametrize("n", SHAPES, ids=lambda n: "x".join(map(str, n)))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_sampled_potential_imaginary_time(gpe, orc, n, prec):
    import torch
    sp, V = _case(n, "lattice")
    psi0 = gi.random_field(sp, seed=3 + sum(n), smooth=0.1)
    psi0 = psi0 / np.sqrt(np.sum(np.abs(psi0) ** 2) * np.prod([sp.length[a] / sp.n[a] for a in range(len(n))]))
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    dt = np.complex128 if prec == "c128" else np.complex64
    ref = orc.Problem(**sp.kwargs(), V=V).step_imag(psi0, 6)
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, prec=pv, V=V)
    x = torch.from_numpy(psi0.astype(dt)).cuda()
    done, _ = p.step_imag(x, 6, etol=0.0, check_every=6)
    torch.cuda.synchronize()
    assert done == 6
    assert rel(x.cpu().numpy(), ref) < (1e-12 if prec == "c128" else 2e-5)
    p.close()


def test_sampled_harmonic_potential_matches_the_built_in_trap(gpe):
    """The harmonic trap sampled on the grid and the separable trap tables agree
    to rounding (complex128)."""
    import torch
    sp = gi.Spec(n=(32, 16, 8), lo=(-6.0, -5.0, -4.0), length=(12.0, 10.0, 8.0), g=30.0, dt=1e-3,
                 gamma=(1.0, 1.7, 2.5))
    mesh = gi._mesh(sp)
    V = sum(0.5 * sp.gamma[a] ** 2 * mesh[a] ** 2 for a in range(3))
    psi0 = gi.random_field(sp, seed=2, smooth=0.05)
    outs = []
    for kw in (dict(gamma=sp.gamma), dict(V=V)):
        p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, prec=gpe.GPE_C128, **kw)
        x = torch.from_numpy(psi0.copy()).cuda()
        p.step_real(x, 20)
        outs.append((x.cpu().numpy(), np.asarray(p.norm_energy(x)[0])))
        p.close()
    assert rel(outs[1][0], outs[0][0]) < 1e-12
    assert np.allclose(outs[1][1], outs[0][1], rtol=1e-11)


def test_sampled_potential_argument_checks(gpe):
    sp, V = _case((16, 16), "lattice")
    with pytest.raises(gpe.GpeError):
        gpe.Plan(sp.n, sp.lo, sp.length, g=1.0, dt=1e-3, gamma=(1.0, 1.0), V=V)   # both traps
    bad = V.copy()
    bad[3, 4] = np.nan
    with pytest.raises(gpe.GpeError):
        gpe.Plan(sp.n, sp.lo, sp.length, g=1.0, dt=1e-3, V=bad)
    d = gpe.make_desc(sp.n, sp.lo, sp.length, g=1.0, dt=1e-3, V=V)
    with pytest.raises(gpe.GpeError) as ei:
        gpe.gpe_batch_create([d[0]], 0)
    assert ei.value.status == 2
