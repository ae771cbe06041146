"""Batches of independent instances and the request server (include/gpe_serve.h)."""
import time

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


def mixed_specs(count, seed):
    """Uneven instances: several shapes, g and trap drawn per instance."""
    rng = np.random.default_rng(seed)
    shapes = [(64, 64), (128, 32), (32, 64), (256,), (16, 16, 16)]
    out = []
    for i in range(count):
        n = shapes[i % len(shapes)]
        d = len(n)
        gam = tuple(float(v) for v in rng.uniform(1.0, 3.0, size=d))
        out.append(gi.Spec(n=n, lo=(-6.0,) * d, length=(12.0,) * d, g=float(rng.uniform(0, 200)), dt=1e-3,
                           gamma=gam))
    return out


def desc_of(gpe, sp, prec):
    return gpe.make_desc(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=prec)[0]


@pytest.mark.parametrize("prec", [1, 0], ids=["c128", "c64"])
@pytest.mark.parametrize("use_graph", [True, False], ids=["graph", "direct"])
def test_batch_equals_individual_plans_and_oracle(gpe, orc, prec, use_graph):
    import torch
    dt = np.complex128 if prec == 1 else np.complex64
    specs = mixed_specs(11, seed=3)
    psis = [gi.random_field(sp, seed=40 + i, smooth=0.05).astype(dt) for i, sp in enumerate(specs)]
    xs = [torch.from_numpy(p.copy()).cuda() for p in psis]
    ys = [torch.from_numpy(p.copy()).cuda() for p in psis]
    stream = torch.cuda.current_stream()
    b = gpe.gpe_batch_create([desc_of(gpe, sp, prec) for sp in specs], stream.cuda_stream)
    assert gpe.gpe_batch_groups(b) == 5
    steps = 6
    gpe.gpe_batch_step_real(b, [x.data_ptr() for x in xs], steps, use_graph)
    gpe.gpe_batch_step_real(b, [x.data_ptr() for x in xs], steps, use_graph)   # replay
    torch.cuda.synchronize()
    e_batch = gpe.gpe_batch_norm_energy(b, [x.data_ptr() for x in xs])
    for i, sp in enumerate(specs):
        p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=prec)
        p.step_real(ys[i], steps)
        p.step_real(ys[i], steps)
        torch.cuda.synchronize()
        assert torch.equal(xs[i], ys[i]), i
        e = p.norm_energy(ys[i])[0]
        assert np.allclose(e, e_batch[i], rtol=1e-12, atol=0), i
        p.close()
    for i in (0, 3, 4):
        ref = orc.Problem(**specs[i].kwargs()).step_real(psis[i].astype(np.complex128), 2 * steps)
        assert rel(xs[i].cpu().numpy(), ref) < (1e-12 if prec == 1 else 2e-5)
    gpe.gpe_batch_destroy(b)


def test_resident_batch_groups_equal_individual_plans(gpe):
    """64^2 and 128^2 complex64 groups are stepped in shared memory for the
    whole call (one launch per group); they give the bits of per-instance
    plans, including instances with g up to 1000 whose nonlinear angles exceed
    1/16 in the core (the long series there)."""
    import torch
    items = [(sp, psi) for sp, psi in gi.batched_specs(count=24, seed=7, sizes=(64, 128))]
    xs = [torch.from_numpy(psi.astype(np.complex64)).cuda() for _, psi in items]
    ys = [x.clone() for x in xs]
    stream = torch.cuda.current_stream()
    b = gpe.gpe_batch_create([desc_of(gpe, sp, gpe.GPE_C64) for sp, _ in items], stream.cuda_stream)
    steps = 40
    gpe.gpe_batch_step_real(b, [x.data_ptr() for x in xs], steps, True)
    torch.cuda.synchronize()
    assert max(sp.g for sp, _ in items) > 500
    for (sp, _), x, y in zip(items, xs, ys):
        p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C64)
        p.step_real(y, steps)
        torch.cuda.synchronize()
        assert torch.equal(x, y)
        p.close()
    gpe.gpe_batch_destroy(b)


def _standalone(gpe, sp, psi0, prec, imag, nsteps, etol=0.0, check_every=1):
    import torch
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=prec)
    x = torch.from_numpy(psi0.copy()).cuda()
    if imag:
        done, _ = p.step_imag(x, nsteps, target_norm=1.0, etol=etol, check_every=check_every)
    else:
        p.step_real(x, nsteps)
        done = nsteps
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    p.close()
    return out, done


def test_server_results_match_standalone_runs_alone_and_in_the_mix(gpe):
    prec = 1
    specs = mixed_specs(10, seed=9)
    psis = [gi.random_field(sp, seed=70 + i, smooth=0.1) for i, sp in enumerate(specs)]
    modes = [(i % 3 == 2) for i in range(len(specs))]
    nsteps = [37 + 11 * i for i in range(len(specs))]
    # alone: request 1 on an otherwise idle server
    srv = gpe.gpe_server_create(8 << 30, max_active=4, chunk_steps=16)
    t = gpe.gpe_serve_submit(srv, desc_of(gpe, specs[1], prec), psis[1], imag=modes[1], nsteps=nsteps[1])
    alone = np.empty_like(psis[1])
    r = gpe.gpe_serve_poll(srv, t, timeout_ms=-1, psi_out=alone)
    assert r.status == 0 and r.steps_done == nsteps[1]
    # in the mix: all requests at once, more than fit at a time
    tickets = []
    for i, sp in enumerate(specs):
        tickets.append(gpe.gpe_serve_submit(srv, desc_of(gpe, sp, prec), psis[i], imag=modes[i], nsteps=nsteps[i],
                                            etol=1e-9 if modes[i] else 0.0, check_every=8))
    outs, results = [], []
    for i, t in enumerate(tickets):
        o = np.empty_like(psis[i])
        res = gpe.gpe_serve_poll(srv, t, timeout_ms=-1, psi_out=o)
        assert res.status == 0, (i, res.status)
        assert res.t_submit <= res.t_admit <= res.t_done
        outs.append(o)
        results.append(res)
    assert rel(outs[1], alone) < 1e-12
    for i, sp in enumerate(specs):
        ref, done = _standalone(gpe, sp, psis[i], prec, modes[i], nsteps[i], etol=1e-9 if modes[i] else 0.0,
                                check_every=8)
        assert results[i].steps_done == done, i
        assert rel(outs[i], ref) < 1e-11, (i, rel(outs[i], ref))
    gpe.gpe_server_destroy(srv)


def test_server_admission_respects_budget_and_slots(gpe):
    prec = 0
    sp = gi.Spec(n=(128, 128), lo=(-6.0, -6.0), length=(12.0, 12.0), g=10.0, dt=1e-3, gamma=(1.0, 1.0))
    psi = gi.harmonic_gaussian(sp).astype(np.complex64)
    srv = gpe.gpe_server_create(64 << 20, max_active=2, chunk_steps=8)
    tickets = [gpe.gpe_serve_submit(srv, desc_of(gpe, sp, prec), psi, nsteps=400) for _ in range(6)]
    seen = 0
    deadline = time.time() + 60
    while time.time() < deadline:
        q, a, used = gpe.gpe_server_stats(srv)
        assert a <= 2 and used <= (64 << 20)
        seen = max(seen, a)
        if q == 0 and a == 0:
            break
        time.sleep(0.005)
    assert seen >= 1
    for t in tickets:
        assert gpe.gpe_serve_poll(srv, t, timeout_ms=-1).status == 0
    # a request larger than the whole budget is refused, not hung
    big = gi.Spec(n=(4096, 4096), lo=(-6.0, -6.0), length=(12.0, 12.0), g=1.0, dt=1e-3)    # 128 MiB
    zb = np.zeros(big.shape, np.complex64)
    t = gpe.gpe_serve_submit(srv, desc_of(gpe, big, prec), zb, nsteps=1)
    assert gpe.gpe_serve_poll(srv, t, timeout_ms=-1).status == 7
    gpe.gpe_server_destroy(srv)
