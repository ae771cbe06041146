"""gpe_norm_energy_noalloc: the norm/energy diagnostics for callers that
cannot allocate device memory (their framework owns all device memory, or
cudaMalloc's implicit synchronisation is not acceptable in their loop).

The entry point must give the same values as the plan-based gpe_norm_energy,
within the diagnostics tolerance of the other GPU tests, on consecutive calls
that share its static scratch array, and reject grids beyond its limit.
This file is collected last so that a failure here does not hide others.
"""
import numpy as np
import pytest

import gpe_inputs as gi

pytestmark = pytest.mark.gpu

CASES = [
    gi.Spec(n=(256, 128), lo=(-8.0, -6.0), length=(16.0, 12.0), g=40.0, gamma=(1.0, 1.7)),
    gi.Spec(n=(32, 16, 64), lo=(-4.0, -3.0, -5.0), length=(8.0, 6.0, 10.0), g=15.0, gamma=(1.0, 2.0, 0.5)),
    gi.Spec(n=(4096,), lo=(-30.0,), length=(60.0,), g=5.0, gamma=(1.0,)),
]


@pytest.fixture(scope="module")
def gpe():
    import torch
    import paper_2301_08275_gb300 as g
    g.build()
    g.lib()
    assert torch.cuda.is_available()
    return g


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-5)], ids=["c128", "c64"])
@pytest.mark.parametrize("sp", CASES, ids=["2d", "3d", "1d"])
def test_noalloc_matches_plan_on_two_calls(gpe, prec, tol, sp):
    import torch
    dt = np.complex64 if prec == gpe.GPE_C64 else np.complex128
    stream = torch.cuda.current_stream()
    plan = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=prec)
    desc, keep = gpe.make_desc(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=prec)
    for seed in (1, 2):
        psi = torch.from_numpy(gi.random_field(sp, seed=seed, smooth=0.05).astype(dt)).to("cuda")
        ref = plan.norm_energy(psi)[0]
        out = gpe.gpe_norm_energy_noalloc(desc, psi.data_ptr(), stream.cuda_stream)
        for i in range(6):
            assert abs(out[i] - ref[i]) <= tol * max(abs(ref[i]), abs(ref[4])), (seed, i, out[i], ref[i])
    plan.close()


def test_noalloc_second_call_takes_no_device_memory(gpe):
    import torch
    sp = CASES[0]
    psi = torch.from_numpy(gi.random_field(sp, seed=3).astype(np.complex64)).to("cuda")
    desc, keep = gpe.make_desc(sp.n, sp.lo, sp.length, g=sp.g, gamma=sp.gamma[:2], prec=gpe.GPE_C64)
    s = torch.cuda.current_stream().cuda_stream
    first = gpe.gpe_norm_energy_noalloc(desc, psi.data_ptr(), s)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    second = gpe.gpe_norm_energy_noalloc(desc, psi.data_ptr(), s)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(first, second)


def test_noalloc_rejects_grids_beyond_its_limit(gpe):
    import torch
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    desc, keep = gpe.make_desc((256, 256, 256), (0.0,) * 3, (1.0,) * 3, prec=gpe.GPE_C64)
    with pytest.raises(gpe.GpeError) as ei:
        gpe.gpe_norm_energy_noalloc(desc, x.data_ptr())
    assert ei.value.status == 2
    assert "GPE_NOALLOC_MAX_LINES" in str(ei.value)
    desc2, keep2 = gpe.make_desc((64, 64), (0.0,) * 2, (1.0,) * 2, prec=gpe.GPE_C64, batch=2)
    with pytest.raises(gpe.GpeError):
        gpe.gpe_norm_energy_noalloc(desc2, x.data_ptr())
