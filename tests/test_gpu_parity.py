"""Parity of the CUDA library (through its C ABI) with the FP64 oracle.

Tolerances:
  complex128: relative L2 of psi <= 1e-12 (after up to 1000 steps),
  complex64 : relative L2 <= 2e-4, norm drift <= 1e-6, energy rel. error <= 1e-5,
  diagnostics: 1e-12 (complex128) / 1e-5 (complex64) relative.
"""
import math

import numpy as np
import pytest

import gpe_inputs as gi

pytestmark = pytest.mark.gpu

TOL128 = 1e-12
TOL64 = 2e-4


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


def to_dev(psi, prec, gpe):
    import torch
    dt = np.complex64 if prec == gpe.GPE_C64 else np.complex128
    return torch.from_numpy(np.ascontiguousarray(psi, dtype=dt)).to("cuda")


def plan_for(gpe, sp, prec, batch=1, g_each=None, gamma_each=None):
    return gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=prec,
                    batch=batch, g_each=g_each, gamma_each=gamma_each)


def gpu_real(gpe, sp, psi0, steps, prec):
    import torch
    p = plan_for(gpe, sp, prec)
    x = to_dev(psi0, prec, gpe)
    p.step_real(x, steps)
    torch.cuda.synchronize()
    out = x.cpu().numpy().astype(np.complex128)
    p.close()
    return out


def P(orc, sp):
    return orc.Problem(**sp.kwargs())


# ------------------------------------------------------------------ real time
def test_config_1d_complex128_1000_steps(gpe, orc):
    sp = gi.CONFIG_1D
    psi0 = gi.gaussian_1d(sp, seed=0)
    ref = P(orc, sp).step_real(psi0, 1000)
    out = gpu_real(gpe, sp, psi0, 1000, gpe.GPE_C128)
    assert rel(out, ref) < TOL128


def test_config_1d_complex64_1000_steps(gpe, orc):
    sp = gi.CONFIG_1D
    psi0 = gi.gaussian_1d(sp, seed=1)
    pr = P(orc, sp)
    ref = pr.step_real(psi0, 1000)
    out = gpu_real(gpe, sp, psi0, 1000, gpe.GPE_C64)
    assert rel(out, ref) < TOL64
    e0, e1 = pr.norm_energy(ref), pr.norm_energy(out)
    assert abs(e1[0] - pr.norm_energy(psi0)[0]) < 1e-6
    assert abs(e1[4] - e0[4]) / abs(e0[4]) < 1e-5


def test_complex64_norm_drift_3d(gpe, orc):
    """complex64 bulk over 1000 steps of a 64^3 Taylor-Green field: norm drift
    <= 1e-6 and energy within 1e-5 of the complex128 oracle run."""
    sp = gi.Spec(n=(64, 64, 64), lo=(0.0,) * 3, length=(2 * math.pi * 4,) * 3, g=1.0, dt=1e-3)
    psi0 = gi.taylor_green_3d(sp, seed=0).astype(np.complex128)
    pr = P(orc, sp)
    n0 = pr.norm_energy(psi0)
    out = gpu_real(gpe, sp, psi0, 1000, gpe.GPE_C64)
    e1 = pr.norm_energy(out)
    assert abs(e1[0] / n0[0] - 1) < 1e-6
    ref = pr.step_real(psi0, 1000)
    assert rel(out, ref) < TOL64
    e_ref = pr.norm_energy(ref)
    assert abs(e1[4] - e_ref[4]) / abs(e_ref[4]) < 1e-5


SHAPES = [(2,), (64,), (4096,), (8, 4), (64, 32), (16, 256), (128, 128), (2, 1024), (2, 2, 2),
          (32, 16, 8), (8, 64, 16), (4, 4, 512), (64, 64, 64)]


def _spec(n, g=30.0, dt=1e-3, trap=True):
    d = len(n)
    L = [12.0, 10.0, 8.0][:d]
    gam = [1.0, 1.7, 2.5][:d] if trap else [0.0] * d
    return gi.Spec(n=n, lo=tuple(-x / 2 for x in L), length=tuple(L), g=g, dt=dt, gamma=tuple(gam))


@pytest.mark.parametrize("n", SHAPES, ids=lambda n: "x".join(map(str, n)))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_real_steps_match_oracle(gpe, orc, n, prec):
    sp = _spec(n)
    psi0 = gi.random_field(sp, seed=sum(n), smooth=0.05)
    steps = 7
    ref = P(orc, sp).step_real(psi0, steps)
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    out = gpu_real(gpe, sp, psi0, steps, pv)
    assert rel(out, ref) < (TOL128 if prec == "c128" else 2e-5)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_single_step_and_zero_steps(gpe, orc, prec):
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    sp = _spec((32, 16, 8))
    psi0 = gi.random_field(sp, seed=5, smooth=0.05)
    ref1 = P(orc, sp).step_real(psi0, 1)
    assert rel(gpu_real(gpe, sp, psi0, 1, pv), ref1) < (TOL128 if prec == "c128" else 2e-5)
    out0 = gpu_real(gpe, sp, psi0, 0, pv)
    assert rel(out0, psi0) < (1e-15 if prec == "c128" else 1e-7)


@pytest.mark.parametrize("n,batch", [((64,), 5), ((32, 4), 3), ((16, 8, 4), 3), ((64, 64), 2)])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_batched_instances_match_oracle(gpe, orc, n, batch, prec):
    """Instances with their own g and trap, stored back to back; odd batch
    sizes leave a ragged last tile."""
    import torch
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    rng = np.random.default_rng(11)
    g_each = rng.uniform(0, 80, size=batch)
    gam_each = rng.uniform(0.5, 3.0, size=(batch, 3))
    sp0 = _spec(n)
    psis = [gi.random_field(sp0, seed=100 + b, smooth=0.05) for b in range(batch)]
    steps = 5
    p = plan_for(gpe, sp0, pv, batch=batch, g_each=g_each, gamma_each=gam_each)
    x = to_dev(np.stack(psis), pv, gpe)
    p.step_real(x, steps)
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    for b in range(batch):
        spb = gi.Spec(n=sp0.n, lo=sp0.lo, length=sp0.length, g=float(g_each[b]), dt=sp0.dt,
                      gamma=tuple(gam_each[b][: sp0.ndim]))
        ref = P(orc, spb).step_real(psis[b], steps)
        assert rel(out[b], ref) < (TOL128 if prec == "c128" else 2e-5), b
    p.close()


def test_time_reversal_on_gpu(gpe):
    import torch
    sp = _spec((64, 32, 16))
    psi0 = gi.random_field(sp, seed=9, smooth=0.05)
    fwd = plan_for(gpe, sp, gpe.GPE_C128)
    back = plan_for(gpe, gi.Spec(n=sp.n, lo=sp.lo, length=sp.length, g=sp.g, dt=-sp.dt, gamma=sp.gamma),
                    gpe.GPE_C128)
    x = to_dev(psi0, gpe.GPE_C128, gpe)
    fwd.step_real(x, 50)
    back.step_real(x, 50)
    torch.cuda.synchronize()
    assert rel(x.cpu().numpy(), psi0) < 1e-12


def test_host_buffer_entry_point_matches_device_path(gpe):
    import torch
    sp = _spec((64, 64))
    psi0 = gi.random_field(sp, seed=3, smooth=0.05).astype(np.complex64)
    p = plan_for(gpe, sp, gpe.GPE_C64)
    h = psi0.copy()
    p.step_real_host(h, 10)
    x = to_dev(psi0, gpe.GPE_C64, gpe)
    p.step_real(x, 10)
    torch.cuda.synchronize()
    assert np.array_equal(h, x.cpu().numpy())
    p.close()


# ------------------------------------------------------------------ diagnostics
@pytest.mark.parametrize("n", [(256,), (64, 32), (16, 32, 8)], ids=lambda n: "x".join(map(str, n)))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_norm_energy_rms_match_oracle(gpe, orc, n, prec):
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    sp = _spec(n)
    psi = gi.random_field(sp, seed=21, smooth=0.05)
    if prec == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    pr = P(orc, sp)
    e_ref, r_ref = pr.norm_energy(psi), pr.rms(psi)
    p = plan_for(gpe, sp, pv)
    x = to_dev(psi, pv, gpe)
    e, r = p.norm_energy(x)[0], p.rms_size(x)[0]
    tol = 1e-12 if prec == "c128" else 1e-5
    for i in range(6):
        assert abs(e[i] - e_ref[i]) <= tol * max(abs(e_ref[i]), 1e-300 + abs(e_ref[4])), (i, e[i], e_ref[i])
    for i in range(4):
        assert abs(r[i] - r_ref[i]) <= tol * max(r_ref[3], 1e-300), (i, r[i], r_ref[i])
    p.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_spectrum_matches_oracle(gpe, orc, prec):
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    sp = gi.Spec(n=(128, 128), lo=(0, 0), length=(2 * math.pi * 8,) * 2, g=1.0)
    psi, _, _ = gi.vortex_field_2d(sp, nv=16, seed=4)
    if prec == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    ei, ec = P(orc, sp).spectrum(psi)
    p = plan_for(gpe, sp, pv)
    assert p.nshells() == len(ei)
    out = p.spectrum(to_dev(psi, pv, gpe))
    tol = 1e-10 if prec == "c128" else 1e-4
    scale = max(ei.max(), ec.max())
    assert np.max(np.abs(out[0, 0] - ei)) < tol * scale
    assert np.max(np.abs(out[1, 0] - ec)) < tol * scale
    assert abs(out[0, 0].sum() - ei.sum()) < tol * ei.sum()
    p.close()


def test_spectrum_3d_and_single_kind(gpe, orc):
    sp = gi.Spec(n=(16, 32, 8), lo=(0, 0, 0), length=(2 * math.pi, 4 * math.pi, 2 * math.pi), g=1.0)
    psi = gi.random_field(sp, seed=8, smooth=0.02)
    ei, ec = P(orc, sp).spectrum(psi)
    p = plan_for(gpe, sp, gpe.GPE_C128)
    out = p.spectrum(to_dev(psi, gpe.GPE_C128, gpe), kinds=gpe.GPE_SPEC_COMP)
    assert out.shape == (1, 1, len(ec))
    assert np.max(np.abs(out[0, 0] - ec)) < 1e-10 * ec.max()
    p.close()


# ------------------------------------------------------------------ imaginary time
@pytest.mark.parametrize("n", [(128,), (64, 32), (16, 16, 32)], ids=lambda n: "x".join(map(str, n)))
def test_imag_steps_match_oracle(gpe, orc, n):
    import torch
    sp = _spec(n, g=40.0)
    psi0 = gi.random_field(sp, seed=31, smooth=0.1)
    steps = 60
    ref = P(orc, sp).step_imag(psi0, steps, target_norm=1.0)
    p = plan_for(gpe, sp, gpe.GPE_C128)
    x = to_dev(psi0, gpe.GPE_C128, gpe)
    done, E = p.step_imag(x, steps, target_norm=1.0, etol=0.0, check_every=25)
    torch.cuda.synchronize()
    assert done == steps
    assert rel(x.cpu().numpy(), ref) < 1e-11
    p.close()


def test_ground_state_stopping_rule_matches_oracle(gpe, orc):
    import torch
    sp = gi.Spec(n=(64, 64), lo=(-8, -8), length=(16, 16), g=12.5484, dt=1e-3, gamma=(1.0, 1.0))
    psi0 = gi.harmonic_gaussian(sp)
    ref, steps_ref, e_ref = P(orc, sp).ground(psi0, max_steps=20000, etol=1e-9, check_every=50)
    p = plan_for(gpe, sp, gpe.GPE_C128)
    x = to_dev(psi0, gpe.GPE_C128, gpe)
    done, E = p.step_imag(x, 20000, target_norm=1.0, etol=1e-9, check_every=50)
    torch.cuda.synchronize()
    assert done == steps_ref
    assert abs(E[0] - e_ref) < 1e-11 * abs(e_ref)
    assert rel(x.cpu().numpy(), ref) < 1e-10
    p.close()


def test_table1_row_on_gpu(gpe):
    """2D row g=62.742 of the paper's Table 1 (r_rms 1.78722, mu 4.61136)."""
    import torch
    sp = gi.Spec(n=(128, 128), lo=(-10, -10), length=(20, 20), g=62.742, dt=1e-3, gamma=(1.0, 1.0))
    p = plan_for(gpe, sp, gpe.GPE_C128)
    x = to_dev(gi.harmonic_gaussian(sp), gpe.GPE_C128, gpe)
    p.step_imag(x, 40000, etol=1e-12, check_every=50)
    torch.cuda.synchronize()
    r = p.rms_size(x)[0][3]
    mu = p.norm_energy(x)[0][5]
    assert abs(r - 1.78722) / 1.78722 < 2e-5
    assert abs(mu - 4.61136) / 4.61136 < 2e-5
    p.close()


# ------------------------------------------------------------------ errors
def test_invalid_arguments_are_reported(gpe):
    import torch
    with pytest.raises(gpe.GpeError) as ei:
        gpe.Plan((12,), (0.0,), (1.0,))
    assert ei.value.status == 2
    with pytest.raises(gpe.GpeError):
        gpe.Plan((8192,), (0.0,), (1.0,))
    with pytest.raises(gpe.GpeError) as ei:
        gpe.Plan((16, 16), (0.0, 0.0), (1.0, -1.0))
    assert ei.value.status == 1
    p = gpe.Plan((16, 16), (0.0, 0.0), (1.0, 1.0))
    with pytest.raises(gpe.GpeError):
        gpe.gpe_step_real(p._h, 0, 1)
    x = torch.zeros(16 * 16 + 1, dtype=torch.complex64, device="cuda")
    with pytest.raises(gpe.GpeError):
        gpe.gpe_step_real(p._h, x.data_ptr() + 8, 1)      # misaligned
    with pytest.raises(gpe.GpeError):
        gpe.gpe_step_real(p._h, x.data_ptr(), -1)
    p.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_nonlinear_phase_over_all_angle_ranges(gpe, orc, prec):
    """A narrow dense cloud at large g: nonlinear angles above 1/2 at the centre
    (library sincos), between 1/16 and 1/2 on the flanks (long series) and
    below 1/16 in the tails (short series), all in one grid."""
    sp = gi.Spec(n=(64, 64), lo=(-6.0, -6.0), length=(12.0, 12.0), g=2000.0, dt=1e-3, gamma=(1.0, 1.0))
    psi0 = gi.harmonic_gaussian(sp, seed=3, noise=0.01)
    th = sp.g * sp.dt * np.abs(psi0) ** 2
    assert th.max() > 0.5 and np.any((th > 0.0625) & (th < 0.5)) and np.any(th < 0.0625)
    steps = 5
    ref = P(orc, sp).step_real(psi0, steps)
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    out = gpu_real(gpe, sp, psi0, steps, pv)
    assert rel(out, ref) < (TOL128 if prec == "c128" else 2e-5)


@pytest.mark.parametrize("n,batch", [((64, 32, 16), 1), ((32, 16, 8), 3), ((512, 8, 256), 1), ((64, 256), 2),
                                     ((2048, 4), 1), ((8, 64, 16), 1), ((16, 512), 1)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_copy_engine_staging_is_bit_identical(gpe, n, batch, prec):
    """Tiles fetched by the tensor-memory accelerator and by per-thread copies
    feed the same arithmetic: steps, imaginary-time steps and diagnostics agree
    bit for bit (grids include ones where n0 is too small for the copy engine)."""
    import torch
    sp = _spec(n)
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    dt = np.complex128 if prec == "c128" else np.complex64
    psi0 = np.stack([gi.random_field(sp, seed=11 + b, smooth=0.05) for b in range(batch)]).astype(dt)
    outs = []
    for tma in (1, 0):
        p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=pv, batch=batch)
        p.set_option(gpe.GPE_OPT_TMA_STAGING, tma)
        x = torch.from_numpy(psi0.copy()).cuda()
        p.step_real(x, 3)
        e = p.norm_energy(x)
        y = torch.from_numpy(psi0.copy()).cuda()
        p.step_imag(y, 2, etol=0.0, check_every=2)
        torch.cuda.synchronize()
        outs.append((x.cpu().numpy(), y.cpu().numpy(), np.asarray(e)))
        p.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [(64, 32, 16), (512, 8, 64), (16, 512), (1024, 64), (8, 64, 16)],
                         ids=lambda n: "x".join(map(str, n)))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_tile_shapes_and_autotuner_keep_results_bit_identical(gpe, n, prec):
    """Every tile shape / staging combination gives the same bits; the autotuner
    only reads the state it times on and picks one of the combinations."""
    import torch
    sp = _spec(n)
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    dt = np.complex128 if prec == "c128" else np.complex64
    psi0 = gi.random_field(sp, seed=21, smooth=0.05).astype(dt)
    combos = [{}, {gpe.GPE_OPT_TILE_X: 1}, {gpe.GPE_OPT_TILE_Y: 1, gpe.GPE_OPT_TILE_Z: 1},
              {gpe.GPE_OPT_TILE_Y: 1, gpe.GPE_OPT_TILE_Z: 1, gpe.GPE_OPT_TMA_STAGING: 0},
              {gpe.GPE_OPT_TILE_X: 1, gpe.GPE_OPT_TILE_Y: 1, gpe.GPE_OPT_TILE_Z: 1, gpe.GPE_OPT_TMA_Y: 0}]
    outs = []
    for opts in combos + ["tuned"]:
        p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=pv)
        x = torch.from_numpy(psi0.copy()).cuda()
        if opts == "tuned":
            chosen = p.autotune(x, reps=2)
            assert set(chosen.values()) <= {0, 1}
            assert np.array_equal(x.cpu().numpy(), psi0)       # the tuner only read x
        else:
            for k, v in opts.items():
                p.set_option(k, v)
                assert p.get_option(k) == v
        p.step_real(x, 3)
        e = p.norm_energy(x)
        torch.cuda.synchronize()
        outs.append((x.cpu().numpy(), np.asarray(e)))
        p.close()
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


@pytest.mark.parametrize("n", [(512, 256, 16), (256, 1024), (1024, 16, 256)], ids=lambda n: "x".join(map(str, n)))
def test_fixed_program_kernels_match_the_generic_kernel(gpe, n):
    """Sweeps with their program compiled in (complex64 lines of 256 to 1024
    points) against the generic kernel that reads the program from its
    arguments, in both tile shapes, with a trap: real-time steps give the same
    bits; imaginary-time steps agree to a few units in the last place (the
    decay sweeps' compiled instances may round differently)."""
    import torch
    sp = _spec(n)
    psi0 = gi.random_field(sp, seed=31, smooth=0.05).astype(np.complex64)
    outs = []
    for generic in (0, 1):
        for shape in (0, 1):
            p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=gpe.GPE_C64)
            p.set_option(gpe.GPE_OPT_GENERIC_PASSES, generic)
            assert p.get_option(gpe.GPE_OPT_GENERIC_PASSES) == generic
            for opt in (gpe.GPE_OPT_TILE_X, gpe.GPE_OPT_TILE_Y, gpe.GPE_OPT_TILE_Z):
                p.set_option(opt, shape)
            x = torch.from_numpy(psi0.copy()).cuda()
            p.step_real(x, 4)
            y = torch.from_numpy(psi0.copy()).cuda()
            p.step_imag(y, 3, etol=0.0, check_every=3)
            torch.cuda.synchronize()
            outs.append((x.cpu().numpy(), y.cpu().numpy()))
            p.close()
    assert np.isfinite(outs[0][0]).all() and np.abs(outs[0][0]).max() > 0
    scale = np.abs(outs[0][1]).max()
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0])
        assert np.abs(o[1] - outs[0][1]).max() <= 1e-6 * scale


def test_plan_options_reject_bad_values(gpe):
    sp = _spec((32, 16))
    p = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma[: sp.ndim], prec=gpe.GPE_C64)
    for opt, val in ((gpe.GPE_OPT_TILE_X, 2), (gpe.GPE_OPT_TMA_STAGING, -1), (98, 0)):
        with pytest.raises(gpe.GpeError) as ei:
            p.set_option(opt, val)
        assert ei.value.status == 1
    with pytest.raises(gpe.GpeError):
        gpe.gpe_plan_autotune(p._h, 0, 0, 0)
    p.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_1d_small_and_full_tiles_give_the_same_bits(gpe, prec):
    """A plan of many 1D instances (tiles of several lines per CTA) and single-
    instance plans (one line per CTA) compute every line with the same
    arithmetic: real and imaginary steps agree bit for bit.  (Single complex128
    lines take the cluster kernel by default, which factors the transform
    differently; it is turned off here and checked in test_gpu_line_cluster.)"""
    import torch
    sp = gi.Spec(n=(64,), lo=(-6.0,), length=(12.0,), g=30.0, dt=1e-3, gamma=(1.0,))
    B = 200
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    dt = np.complex128 if prec == "c128" else np.complex64
    psi0 = np.stack([gi.random_field(sp, seed=b, smooth=0.05) for b in range(B)]).astype(dt)
    for imag in (False, True):
        pb = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=pv, batch=B)
        x = torch.from_numpy(psi0.copy()).cuda()
        if imag:
            pb.step_imag(x, 7, etol=0.0, check_every=7)
        else:
            pb.step_real(x, 7)
        torch.cuda.synchronize()
        allb = x.cpu().numpy()
        pb.close()
        p1 = gpe.Plan(sp.n, sp.lo, sp.length, g=sp.g, dt=sp.dt, gamma=sp.gamma, prec=pv)
        p1.set_option(gpe.GPE_OPT_LINE_CLUSTER, 0)
        for b in (0, 37, 199):
            y = torch.from_numpy(psi0[b].copy()).cuda()
            if imag:
                p1.step_imag(y, 7, etol=0.0, check_every=7)
            else:
                p1.step_real(y, 7)
            torch.cuda.synchronize()
            assert np.array_equal(y.cpu().numpy(), allb[b]), (imag, b)
        p1.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_quantum_pressure_and_number_spectra_match_oracle(gpe, orc, prec):
    """All four spectra in one call, in kind order, against the oracle (2D
    vortex field), and INC + COMP + QP summed against E_kin of the same state."""
    pv = gpe.GPE_C128 if prec == "c128" else gpe.GPE_C64
    sp = gi.Spec(n=(128, 128), lo=(0, 0), length=(2 * math.pi * 8,) * 2, g=1.0)
    psi, _, _ = gi.vortex_field_2d(sp, nv=16, seed=4)
    if prec == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    pr = P(orc, sp)
    ei, ec = pr.spectrum(psi)
    eq, nn = pr.spectrum_qp_num(psi)
    p = plan_for(gpe, sp, pv)
    x = to_dev(psi, pv, gpe)
    k = gpe.GPE_SPEC_INC | gpe.GPE_SPEC_COMP | gpe.GPE_SPEC_QP | gpe.GPE_SPEC_NUM
    out = p.spectrum(x, kinds=k)
    assert out.shape == (4, 1, len(ei))
    tol = 1e-10 if prec == "c128" else 1e-4
    for got, ref in zip(out[:, 0], (ei, ec, eq, nn)):
        assert np.max(np.abs(got - ref)) < tol * ref.max()
    e = p.norm_energy(x)[0]
    assert abs(out[3, 0].sum() - e[0]) < (1e-12 if prec == "c128" else 1e-6) * e[0]
    # |grad psi|^2 = |grad|psi||^2 + |psi|^2 |grad theta|^2: the three parts sum to E_kin
    # (to 7e-11 in the oracle for this field: its Nyquist content is that small)
    assert abs(out[0, 0].sum() + out[1, 0].sum() + out[2, 0].sum() - e[1]) < (1e-9 if prec == "c128" else 1e-5) * e[1]
    only = p.spectrum(x, kinds=gpe.GPE_SPEC_QP)
    # shells are summed in fixed point: repeated calls give the same bits
    assert only.shape == (1, 1, len(eq)) and np.array_equal(only[0, 0], out[2, 0])
    again = p.spectrum(x, kinds=k)
    assert np.array_equal(again, out)
    p.close()


def test_quantum_pressure_spectrum_3d_matches_oracle(gpe, orc):
    sp = gi.Spec(n=(16, 32, 8), lo=(0, 0, 0), length=(2 * math.pi, 4 * math.pi, 2 * math.pi), g=1.0)
    psi = gi.random_field(sp, seed=8, smooth=0.02) + 2.0
    eq, nn = P(orc, sp).spectrum_qp_num(psi)
    p = plan_for(gpe, sp, gpe.GPE_C128)
    out = p.spectrum(to_dev(psi, gpe.GPE_C128, gpe), kinds=gpe.GPE_SPEC_QP | gpe.GPE_SPEC_NUM)
    assert np.max(np.abs(out[0, 0] - eq)) < 1e-10 * eq.max()
    assert np.max(np.abs(out[1, 0] - nn)) < 1e-10 * nn.max()
    p.close()
