"""Parity of the CUDA path (libak through its C-ABI) against the FP64 CPU oracle.

Tolerances: FP64 form, max state-normalised difference <= 1e-12 after one step and
<= 1e-9 after 100 steps (the oracle and the GPU are driven with the same dt sequence).
Mixed form: FP32-class agreement with the oracle on O(1) flows, and a linear-wave L1
error within 1% of the FP64 one.  Sizes span several 16x16 column tiles with ragged
edges, several MeshBlocks, and the full 256^3 / 64^3-block workload the benchmark
times.
"""
import math

import numpy as np
import pytest

import oracle
import pgen
from _helpers import l1_wave_error, max_norm_diff

pytestmark = pytest.mark.gpu

G53 = 5.0 / 3.0


@pytest.fixture(scope="module")
def ak():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2409_16053_gb300 import build
    build.build()
    from paper_2409_16053_gb300 import ak as mod
    oracle.build()
    return mod


def _mesh(ak, root, block, **kw):
    return ak.Mesh(root, block, **kw)


# ---------------------------------------------------------------------------------
# ghost fill and CFL
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("root,block,ng", [((24, 16, 12), (12, 8, 6), 2),
                                          ((18, 12, 9), (6, 4, 3), 3),
                                          ((8, 8, 8), (8, 8, 8), 2)])
def test_fill_ghosts_is_periodic_wrap(ak, root, block, ng):
    recon = ak.AK_PLM if ng == 2 else ak.AK_PPM4
    m = _mesh(ak, root, block, recon=recon, rk=2 if ng == 2 else 3)
    U = np.random.default_rng(5).normal(size=(5, root[2], root[1], root[0]))
    m.upload(U)
    m.fill_ghosts(0)
    R = m.register_view(0).cpu().numpy()
    P = np.pad(U, ((0, 0), (ng, ng), (ng, ng), (ng, ng)), mode="wrap")
    for b, row in enumerate(m.table):
        _, lx, ly, lz, n1, n2, n3 = row
        ref = P[:, lz:lz + n3 + 2 * ng, ly:ly + n2 + 2 * ng, lx:lx + n1 + 2 * ng]
        assert np.array_equal(R[b], ref), b
    m.close()


def test_new_dt_matches_oracle(ak):
    n = (32, 24, 16)
    U = pgen.turbulence(n, seed=3, kmin=1, kmax=6, mach=1.2)
    g = oracle.Grid(n, length=(1.0, 0.75, 0.5))
    m = _mesh(ak, n, (16, 12, 8), xmax=(1.0, 0.75, 0.5))
    m.upload(U)
    dt = m.new_dt(0)
    assert math.isclose(dt, oracle.new_dt(U, g, 0.3), rel_tol=1e-14)
    m.close()


# ---------------------------------------------------------------------------------
# FP64 form
# ---------------------------------------------------------------------------------
CASES = [
    # root, block, problem
    ((32, 32, 32), (16, 16, 16), "turb"),
    ((40, 36, 24), (20, 18, 12), "turb"),      # ragged 16x16 tiles, 2x2x2 blocks
    ((32, 32, 32), (32, 32, 32), "sound"),     # one block, x3 split in segments
    ((12, 40, 10), (6, 20, 10), "tube_x2"),    # discontinuities across block faces
    ((33, 18, 21), (11, 9, 7), "turb"),        # odd sizes, 27 blocks
    ((8, 8, 8), (2, 2, 2), "turb"),            # blocks as thin as the ghost zone
]


def _problem(kind, n):
    if kind == "turb":
        return pgen.turbulence(n, seed=17, kmin=1, kmax=5, mach=1.0), G53
    if kind == "sound":
        return pgen.linear_wave(n)[0], G53
    if kind == "tube_x2":
        return pgen.shock_tube(n, direction=1, gamma=1.4), 1.4
    raise ValueError(kind)


@pytest.mark.parametrize("root,block,kind", CASES)
def test_fp64_one_step_parity(ak, root, block, kind):
    U0, gamma = _problem(kind, root)
    g = oracle.Grid(root, gamma=gamma)
    dt = oracle.new_dt(U0, g, 0.3)
    ref, nf = oracle.rk_step(U0, g, dt, 2)
    m = _mesh(ak, root, block, gamma=gamma)
    m.upload(U0)
    dt_next = m.step(dt)
    out = m.download()
    err = max_norm_diff(out, ref, gamma)
    assert err <= 1e-12, err
    assert math.isclose(dt_next, oracle.new_dt(ref, g, 0.3), rel_tol=1e-12)
    assert m.counters()[:2] == [0, 0]
    m.close()


def test_stage_calls_equal_graph_step(ak):
    root, block = (32, 32, 16), (16, 16, 16)
    U0 = pgen.turbulence(root, seed=2, kmin=1, kmax=4, mach=0.7)
    a = _mesh(ak, root, block)
    a.upload(U0)
    dt = a.new_dt()
    a.step(dt)
    a.step(dt)          # second call replays the captured graph
    b = _mesh(ak, root, block)
    b.upload(U0)
    for _ in range(2):
        b.fill_ghosts(0)
        b.stage(1, dt)
        b.fill_ghosts(1)
        b.stage(2, dt)
    assert np.array_equal(a.download(), b.download())
    a.close()
    b.close()


def test_fp64_100_steps_parity(ak):
    root, block = (32, 32, 32), (16, 16, 16)
    U = pgen.turbulence(root, seed=23, kmin=2, kmax=8, mach=0.5)
    g = oracle.Grid(root)
    m = _mesh(ak, root, block)
    m.upload(U)
    for _ in range(100):
        dt = oracle.new_dt(U, g, 0.3)
        U, nf = oracle.rk_step(U, g, dt, 2)
        m.step(dt, want_dt_next=False)
    out = m.download()
    err = max_norm_diff(out, U, G53)
    assert err <= 1e-9, err
    m.close()


def test_device_resident_dt_loop(ak):
    # ak_step(dt <= 0) uses the device-resident CFL dt: same trajectory as host dt
    root, block = (32, 16, 16), (16, 16, 16)
    U0 = pgen.turbulence(root, seed=5, kmin=1, kmax=4, mach=0.9)
    g = oracle.Grid(root)
    m = _mesh(ak, root, block)
    m.upload(U0)
    m.new_dt()
    for _ in range(5):
        m.step(0.0, want_dt_next=False)
    out = m.download()
    U = U0
    for _ in range(5):
        U, _ = oracle.rk_step(U, g, oracle.new_dt(U, g, 0.3), 2)
    assert max_norm_diff(out, U, G53) <= 1e-12
    m.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_uniform_state_bitwise(ak, precision):
    root = (32, 16, 16)
    U0 = pgen.uniform(root, rho=1.2, p=0.9, v=(0.3, -0.4, 0.2))
    m = _mesh(ak, root, (16, 16, 16), precision=precision, ref_rho=1.0, ref_p=1.0)
    m.upload(U0)
    for _ in range(3):
        m.step(0.01, want_dt_next=False)
    assert np.array_equal(m.download(), U0)
    m.close()


def test_fp64_conservation(ak):
    root = (32, 32, 32)
    U0 = pgen.turbulence(root, seed=9, kmin=1, kmax=6, mach=2.0)
    m = _mesh(ak, root, (16, 16, 16))
    m.upload(U0)
    dt = m.new_dt()
    for _ in range(10):
        dt = m.step(dt)
    U = m.download()
    for k in range(5):
        tol = 200 * 2.2e-16 * np.abs(U0[k]).sum()
        assert abs(U[k].sum() - U0[k].sum()) <= tol, (k, U[k].sum() - U0[k].sum(), tol)
    m.close()


# ---------------------------------------------------------------------------------
# PPM4 + RK3 (the production setup named in Section 3.1)
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("root,block,kind", [((36, 24, 18), (18, 12, 9), "turb"),
                                            ((24, 30, 12), (12, 15, 12), "tube_x2")])
def test_ppm4_rk3_parity(ak, root, block, kind):
    U0, gamma = _problem(kind, root)
    g = oracle.Grid(root, gamma=gamma, recon=oracle.PPM4)
    m = _mesh(ak, root, block, gamma=gamma, recon=ak.AK_PPM4, rk=3)
    m.upload(U0)
    U = U0
    for s in range(10):
        dt = oracle.new_dt(U, g, 0.3)
        U, _ = oracle.rk_step(U, g, dt, 3)
        m.step(dt, want_dt_next=False)
        if s == 0:
            assert max_norm_diff(m.download(), U, gamma) <= 1e-12
    assert max_norm_diff(m.download(), U, gamma) <= 1e-10
    m.close()


# ---------------------------------------------------------------------------------
# mixed form
# ---------------------------------------------------------------------------------
def _run_wave(ak, n, precision, recon=0, rk=2):
    U0, T = pgen.linear_wave((n, n, n))
    m = _mesh(ak, (n, n, n), (n, n, n), precision=precision, recon=recon, rk=rk,
              ref_rho=1.0, ref_p=1.0 / G53)
    m.upload(U0)
    t = 0.0
    dt = m.new_dt()
    while t < T:
        dt = min(dt, T - t)
        dt_next = m.step(dt)
        t += dt
        dt = dt_next
    out = m.download()
    m.close()
    return l1_wave_error(out, U0), out


def test_mixed_linear_wave_l1_within_one_percent(ak):
    e64, _ = _run_wave(ak, 32, 0)
    e32, _ = _run_wave(ak, 32, 1)
    # and the FP64 GPU error is the oracle's
    g = oracle.Grid((32, 2, 2))
    U0, T = pgen.linear_wave((32, 2, 2))
    Uo, _, _, _ = oracle.run(U0, g, 0.3, t_end=T)
    eo = l1_wave_error(Uo, U0)
    assert math.isclose(e64, eo, rel_tol=1e-6), (e64, eo)
    assert abs(e32 - e64) <= 0.01 * e64, (e32, e64)


def _run_wave_bg(ak, n, rho_b, p_b):
    U0, T = pgen.linear_wave((n, n, n))
    m = _mesh(ak, (n, n, n), (n, n, n), precision=1, ref_rho=rho_b, ref_p=p_b)
    m.upload(U0)
    t, dt = 0.0, m.new_dt()
    while t < T:
        dt = min(dt, T - t)
        dt_next = m.step(dt)
        t += dt
        dt = dt_next
    out = m.download()
    m.close()
    return l1_wave_error(out, U0)


@pytest.mark.parametrize("factor,bound", [(1.01, 1.01), (1.1, 1.03), (10.0, None)])
def test_mixed_wave_error_against_background_choice(ak, factor, bound):
    """The mixed form's error as the background (ref_rho, ref_p) moves off the flow's
    state (rho = 1, p = 3/5) by a factor: on the 1e-6 sound wave a background within 1%
    keeps the L1 error within 1% of the FP64 one, within 10% within 3%; a background 10x
    off leaves O(1) deviations in the FP32 arithmetic, whose rounding (~1e-7 of them) is
    then not small against the 1e-6 wave: the error grows several-fold (measured 14x)."""
    e64, _ = _run_wave(ak, 32, 0)
    ratio = _run_wave_bg(ak, 32, factor, factor * 0.6) / e64
    if bound is not None:
        assert ratio <= bound, ratio
    else:
        assert ratio > 5.0, ratio


def test_mixed_turbulence_error_against_background_choice(ak):
    """Mach-0.5 turbulence (O(1) fluctuations) after one step: a background 10x off
    the mean state stays within 5e-7 of the oracle (4.6e-8 at the mean state), 100x off
    within 1e-5 -- the FP32 rounding of deviations that carry the background mismatch."""
    root = (32, 32, 32)
    U0 = pgen.turbulence(root, seed=31, kmin=2, kmax=8, mach=0.5)
    g = oracle.Grid(root)
    dt = oracle.new_dt(U0, g, 0.3)
    ref, _ = oracle.rk_step(U0, g, dt, 2)
    errs = {}
    for f in (1.0, 10.0, 100.0):
        m = _mesh(ak, root, (16, 16, 16), precision=1, ref_rho=f, ref_p=f)
        m.upload(U0)
        m.step(dt)
        errs[f] = max_norm_diff(m.download(), ref, G53)
        m.close()
    assert errs[1.0] <= 2e-7 and errs[10.0] <= 5e-7 and errs[100.0] <= 1e-5, errs
    assert errs[100.0] > 10 * errs[1.0], errs


def test_mixed_turbulence_close_to_oracle(ak):
    root = (32, 32, 32)
    U0 = pgen.turbulence(root, seed=31, kmin=2, kmax=8, mach=0.5)
    g = oracle.Grid(root)
    dt = oracle.new_dt(U0, g, 0.3)
    ref, _ = oracle.rk_step(U0, g, dt, 2)
    m = _mesh(ak, root, (16, 16, 16), precision=1, ref_rho=1.0, ref_p=1.0)
    m.upload(U0)
    m.step(dt)
    out = m.download()
    err = max_norm_diff(out, ref, G53)
    assert err <= 2e-6, err
    m.close()


def test_mixed_conservation(ak):
    root = (32, 32, 32)
    U0 = pgen.turbulence(root, seed=9, kmin=1, kmax=6, mach=2.0)
    m = _mesh(ak, root, (16, 16, 16), precision=1, ref_rho=1.0, ref_p=1.0)
    m.upload(U0)
    dt = m.new_dt()
    for _ in range(10):
        dt = m.step(dt)
    U = m.download()
    for k in range(5):
        # FP32 flux differences: conservation to FP32 rounding of the updates
        tol = 1e-6 * np.abs(U[k] - U0[k]).sum() + 200 * 2.2e-16 * np.abs(U0[k]).sum()
        assert abs(U[k].sum() - U0[k].sum()) <= tol, (k, U[k].sum() - U0[k].sum(), tol)
    m.close()


# ---------------------------------------------------------------------------------
# status reporting
# ---------------------------------------------------------------------------------
def test_negative_internal_energy_reported(ak):
    root = (16, 16, 16)
    U0 = pgen.uniform(root, rho=1.0, p=0.6)
    U0[4, 3, 4, 5] = 0.5 * U0[0, 3, 4, 5] * 0.0 - 1.0  # E < kinetic energy: u_g < 0
    m = _mesh(ak, root, (16, 16, 16))
    m.upload(U0)
    dt, st = ak.ak_new_dt(m.handle, 0)
    assert st == ak.AK_OK  # the CFL pass alone applies floors silently
    _, st = ak.ak_step(m.handle, 1e-4, True)
    assert st == ak.AK_ENEGATIVE
    c = m.counters()
    assert c[0] > 0 and c[1] == 0
    _, st = ak.ak_step(m.handle, 1e-4, True)  # still negative: reported again
    m.close()


def test_invalid_calls_on_live_mesh(ak):
    m = _mesh(ak, (16, 16, 16), (16, 16, 16))
    with pytest.raises(ak.AkError):
        ak.ak_stage(m.handle, 3, 0.1)          # RK2 has 2 stages
    with pytest.raises(ak.AkError):
        ak.ak_stage(m.handle, 0, 0.1)
    with pytest.raises(ak.AkError):
        ak.ak_fill_ghosts(m.handle, 2)
    with pytest.raises(ak.AkError):
        ak.ak_mesh_bind(m.handle, 0, m.regs[0].data_ptr() + 8)  # misaligned
    m.close()


# ---------------------------------------------------------------------------------
# full benchmark workload: 256^3 in 64 blocks of 64^3, the launch configuration the
# benchmark times (graph-replayed ak_step)
# ---------------------------------------------------------------------------------
@pytest.mark.slow
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-6)])
def test_full_size_one_step(ak, precision, tol):
    root = (256, 256, 256)
    U0 = pgen.turbulence(root, seed=1, kmin=2, kmax=8, mach=0.5)
    g = oracle.Grid(root)
    dt = oracle.new_dt(U0, g, 0.3)
    m = _mesh(ak, root, (64, 64, 64), precision=precision, ref_rho=1.0, ref_p=1.0)
    m.upload(U0)
    m.step(dt)
    out = m.download()
    m.close()
    ref, nf = oracle.rk_step(U0, g, dt, 2)
    assert nf == 0
    err = max_norm_diff(out, ref, G53)
    assert err <= tol, err


@pytest.mark.slow
def test_full_size_100_steps_properties(ak):
    root = (256, 256, 256)
    U0 = pgen.turbulence(root, seed=1, kmin=2, kmax=8, mach=0.5)
    m = _mesh(ak, root, (64, 64, 64))
    m.upload(U0)
    dts = [m.new_dt()]
    for _ in range(100):
        dts.append(m.step(0.0))
    U = m.download()
    assert m.counters()[:2] == [0, 0]
    assert all(d > 0 for d in dts)
    assert max(dts) / min(dts) < 1.5
    for k in range(5):
        tol = 1000 * 2.2e-16 * np.abs(U0[k]).sum()
        assert abs(U[k].sum() - U0[k].sum()) <= tol
    m.close()


# ---------------------------------------------------------------------------------
# stage schedule autotuner: any tile shape / x3 split / CTA order gives the same bits
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_keeps_results_bitwise(ak, precision):
    root, block = (64, 64, 64), (32, 32, 32)
    U0 = pgen.turbulence(root, seed=4, kmin=1, kmax=6, mach=0.8)
    a = _mesh(ak, root, block, precision=precision, ref_rho=1.0, ref_p=1.0)
    a.upload(U0)
    tile, seg, order, us, fused = a.autotune()
    assert tile in (0, 1, 2) and seg >= 1 and order in (0, 1) and us > 0
    b = _mesh(ak, root, block, precision=precision, ref_rho=1.0, ref_p=1.0)
    b.upload(U0)
    dt = a.new_dt()
    assert dt == b.new_dt()
    for _ in range(3):
        a.step(dt, want_dt_next=False)
        b.step(dt, want_dt_next=False)
    assert np.array_equal(a.download(), b.download())
    a.close()
    b.close()


@pytest.mark.parametrize("root,block", [((64, 64, 64), (32, 32, 32)),
                                        ((40, 24, 16), (20, 12, 8))])
def test_mixed_kernel_variants_bitwise(ak, root, block):
    """The paired 16x16 kernel, the 32x8 and the unpaired 16x16 column kernels, with x3
    segments and either CTA order, give the same bits (ragged tiles in the second case);
    the 2-step result stays within the mixed form's tolerance of the FP64 oracle."""
    U0 = pgen.turbulence(root, seed=9, kmin=1, kmax=5, mach=0.7)
    ref = None
    for tile, seg, order in [(2, 1, 0), (0, 1, 0), (0, 4, 1), (1, 2, 0), (2, 8, 1)]:
        m = _mesh(ak, root, block, precision=ak.AK_MIXED, ref_rho=1.0, ref_p=1.0)
        m.schedule(tile, seg, order)
        m.upload(U0)
        dt = m.new_dt()
        for _ in range(2):
            m.step(dt, want_dt_next=False)
        U = m.download()
        assert m.counters()[:2] == [0, 0]
        m.close()
        if ref is None:
            ref = U
        else:
            assert np.array_equal(U, ref), (tile, seg, order)
    grid = oracle.Grid(root)
    O = U0
    for _ in range(2):
        O, _ = oracle.rk_step(O, grid, dt, 2)
    err = max_norm_diff(ref, O, G53)
    assert err <= 5e-6, err


def test_schedule_rejects_bad_arguments(ak):
    m = _mesh(ak, (32, 32, 32), (16, 16, 16))
    for args in [(1, 1, 0), (3, 1, 0), (0, 0, 0), (0, 65, 0), (0, 1, 2)]:
        with pytest.raises(ak.AkError):
            m.schedule(*args)
    m.schedule(0, 2, 1)
    m.close()


@pytest.mark.parametrize("recon,block", [(0, (16, 1, 1)), (1, (2, 2, 2)), (2, (4, 2, 4))])
def test_blocks_thinner_than_the_ghost_zone_are_refused(ak, recon, block):
    with pytest.raises(ak.AkError, match="nghost"):
        _mesh(ak, (16, 8, 8), block, recon=recon, rk=3 if recon else 2)


def test_upload_download_pinned_and_pageable_paths(ak):
    """Mapped page-locked buffers go through the (un)pack kernels directly, pageable ones
    through the staging buffer: every combination returns the uploaded bits."""
    import torch
    root, block = (24, 20, 16), (12, 10, 8)
    m = _mesh(ak, root, block)
    P = m.pack(pgen.turbulence(root, seed=5, kmin=1, kmax=4, mach=1.0))
    pinned = torch.from_numpy(P.copy()).pin_memory()
    pageable = np.ascontiguousarray(P.copy())
    for src in (pinned.data_ptr(), pageable.ctypes.data):
        ak.ak_upload(m.handle, 1, src)
        m.stream.synchronize()
        out_pinned = torch.empty_like(pinned).pin_memory()
        out_pageable = np.empty_like(pageable)
        ak.ak_download(m.handle, 1, out_pinned.data_ptr())
        ak.ak_download(m.handle, 1, out_pageable.ctypes.data)
        assert np.array_equal(out_pinned.numpy(), P)
        assert np.array_equal(out_pageable, P)
    m.close()
