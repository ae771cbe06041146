"""gpe_step_real_host on large states in pinned host memory: the state moves in
slabs of planes while the sweeps that stay inside a slab run on the slabs
already moved.  Every line is computed as on the device path, so the results
are bit-identical to gpe_step_real on a device copy."""
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


def pinned_copy(a):
    import torch
    t = torch.empty(a.shape, dtype=torch.complex64 if a.dtype == np.complex64 else torch.complex128, pin_memory=True)
    h = t.numpy()
    h[...] = a
    return t, h


CASES = [
    ("3d_c64_trap", (256, 256, 256), np.complex64, True),
    ("3d_c64_free", (128, 256, 512), np.complex64, False),
    ("3d_c128", (128, 128, 512), np.complex128, True),
    ("2d_c64", (2048, 4096), np.complex64, True),
]


@pytest.mark.parametrize("name,n,dt,trap", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("steps", [0, 1, 3])
def test_pinned_host_steps_equal_device_steps(gpe, name, n, dt, trap, steps):
    import torch
    d = len(n)
    L = [12.0, 10.0, 8.0][:d]
    sp = gi.Spec(n=n, lo=tuple(-x / 2 for x in L), length=tuple(L), g=20.0, dt=1e-3,
                 gamma=tuple([1.0, 1.5, 2.0][:d]) if trap else (0.0,) * d)
    rng = np.random.default_rng(sum(n) + steps)
    psi0 = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(dt) * np.asarray(0.01, dtype=dt)
    prec = gpe.GPE_C64 if dt == np.complex64 else gpe.GPE_C128
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=prec)
    keep, h = pinned_copy(psi0)
    p.step_real_host(h, steps)
    x = torch.from_numpy(psi0).cuda()
    p.step_real(x, steps)
    torch.cuda.synchronize()
    assert np.array_equal(h, x.cpu().numpy())
    # a second call on the same plan (events and copy stream reused)
    p.step_real_host(h, 1)
    p.step_real(x, 1)
    torch.cuda.synchronize()
    assert np.array_equal(h, x.cpu().numpy())
    p.close()
    del keep
