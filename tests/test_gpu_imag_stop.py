"""The device-side stopping rule of gpe_step_imag (|E - E_prev| < etol for every
instance at a check every check_every steps, tested on the device; the host
queues chunks a window at a time) against the oracle's host loop: the same
step counts, energies and states in the edge cases of the windowing."""
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


SP = gi.Spec(n=(32, 32), lo=(-6.0, -6.0), length=(12.0, 12.0), g=20.0, dt=1e-3, gamma=(1.0, 1.5))


def run(gpe, sp, psi0, max_steps, etol, check_every, batch=1, g_each=None):
    import torch
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=gpe.GPE_C128, batch=batch,
                 g_each=g_each)
    x = torch.from_numpy(np.ascontiguousarray(psi0)).cuda()
    done, E = p.step_imag(x, max_steps, target_norm=1.0, etol=etol, check_every=check_every)
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    p.close()
    return done, E, out


@pytest.mark.parametrize("max_steps,check_every", [(37, 5), (100, 1), (3, 50), (0, 4)])
def test_runs_to_max_steps_without_a_stop(gpe, orc, max_steps, check_every):
    """etol = 0 never stops: exactly max_steps steps, also when max_steps is
    not a multiple of check_every, with a check after every step (many
    windows), with one short chunk, and with none."""
    psi0 = gi.random_field(SP, seed=4, smooth=0.1)
    pr = orc.Problem(**SP.kwargs())
    done, E, out = run(gpe, SP, psi0, max_steps, 0.0, check_every)
    assert done == max_steps
    if max_steps == 0:
        assert np.array_equal(out, psi0)
        assert abs(E[0] - pr.norm_energy(psi0)[4]) < 1e-12 * abs(E[0])
        return
    ref = pr.step_imag(psi0, max_steps, target_norm=1.0)
    assert rel(out, ref) < 1e-11
    assert abs(E[0] - pr.norm_energy(ref)[4]) < 1e-11 * abs(E[0])


def test_stops_at_the_first_check(gpe, orc):
    psi0 = gi.random_field(SP, seed=5, smooth=0.1)
    ref, steps_ref, e_ref = orc.Problem(**SP.kwargs()).ground(psi0, 1000, etol=1e9, check_every=7)
    assert steps_ref == 7
    done, E, out = run(gpe, SP, psi0, 1000, 1e9, 7)
    assert done == 7
    assert abs(E[0] - e_ref) < 1e-11 * abs(e_ref)
    assert rel(out, ref) < 1e-11


@pytest.mark.parametrize("check_every", [1, 16])
def test_long_stop_matches_the_oracle_rule(gpe, orc, check_every):
    """A ground state that needs many windows (2, 4, 8, then 16 chunks): the
    stopping step, energy and state of the oracle's host loop."""
    psi0 = gi.harmonic_gaussian(SP)
    ref, steps_ref, e_ref = orc.Problem(**SP.kwargs()).ground(psi0, 20000, etol=1e-9, check_every=check_every)
    assert steps_ref > 40 * check_every or check_every == 1
    done, E, out = run(gpe, SP, psi0, 20000, 1e-9, check_every)
    assert done == steps_ref
    assert abs(E[0] - e_ref) < 1e-11 * abs(e_ref)
    assert rel(out, ref) < 1e-10


def test_batch_stops_when_every_instance_has_converged(gpe, orc):
    """Instances with their own g converge at different checks; the batch stops
    at the first check where all have, i.e. the latest of their own stops
    (|dE| only decreases here), and every instance has taken that many steps."""
    gs = [5.0, 20.0, 60.0]
    psi0 = np.stack([gi.harmonic_gaussian(SP) for _ in gs])
    own = []
    for g in gs:
        sb = gi.Spec(n=SP.n, lo=SP.lo, length=SP.length, g=g, dt=SP.dt, gamma=SP.gamma)
        own.append(orc.Problem(**sb.kwargs()).ground(psi0[0], 20000, etol=1e-8, check_every=10)[1])
    assert len(set(own)) > 1
    done, E, out = run(gpe, SP, psi0, 20000, 1e-8, 10, batch=len(gs), g_each=gs)
    assert done == max(own)
    for b, g in enumerate(gs):
        sb = gi.Spec(n=SP.n, lo=SP.lo, length=SP.length, g=g, dt=SP.dt, gamma=SP.gamma)
        pr = orc.Problem(**sb.kwargs())
        ref = pr.step_imag(psi0[b], done, target_norm=1.0)
        assert rel(out[b], ref) < 1e-10, b
        assert abs(E[b] - pr.norm_energy(ref)[4]) < 1e-10 * abs(E[b]), b


def test_zero_state_is_reported(gpe):
    import torch
    p = gpe.Plan(SP.n, SP.lo, SP.length, g=SP.g, dt=SP.dt, gamma=SP.gamma, prec=gpe.GPE_C128)
    x = torch.zeros(SP.n, dtype=torch.complex128, device="cuda")
    with pytest.raises(gpe.GpeError) as ei:
        p.step_imag(x, 50, target_norm=1.0, etol=1e-9, check_every=5)
    assert ei.value.status == 5                      # GPE_ENUMERIC
    # the plan still works afterwards
    y = torch.from_numpy(gi.harmonic_gaussian(SP)).cuda()
    done, _ = p.step_imag(y, 10, target_norm=1.0, etol=0.0, check_every=5)
    assert done == 10
    p.close()
