"""The HLLE and LLF Riemann solvers on the GPU against the oracle: FP64 parity after one
step (PLM + RK2 and PPM4 + RK3, uniform and refined meshes), the mixed form within its
tolerance, the sound-wave L1 of the mixed form within 1% of the FP64 one, and the
paired and unpaired mixed kernels giving the same bits."""
import math

import numpy as np
import pytest

import oracle
import pgen
from _helpers import l1_wave_error, max_norm_diff

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0
SOLVERS = [("hlle", 1, oracle.HLLE), ("llf", 2, oracle.LLF)]


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


@pytest.mark.parametrize("name,rs,ors", SOLVERS)
@pytest.mark.parametrize("recon,rk", [(0, 2), (1, 3)])
def test_fp64_one_step_parity(ak, name, rs, ors, recon, rk):
    root, block = (36, 24, 18), (18, 12, 9)
    U0 = pgen.turbulence(root, seed=21, kmin=1, kmax=5, mach=1.0)
    g = oracle.Grid(root, recon=recon, riemann=ors)
    dt = oracle.new_dt(U0, g, 0.3)
    ref, nf = oracle.rk_step(U0, g, dt, rk)
    assert nf == 0
    m = ak.Mesh(root, block, recon=recon, rk=rk, riemann=rs)
    m.upload(U0)
    dt_next = m.step(dt)
    out = m.download()
    err = max_norm_diff(out, ref, G53)
    assert err <= 1e-12, (name, err)
    assert math.isclose(dt_next, oracle.new_dt(ref, g, 0.3), rel_tol=1e-12)
    assert m.counters()[:2] == [0, 0]
    m.close()


@pytest.mark.parametrize("name,rs,ors", SOLVERS)
def test_fp64_shock_tube_ten_steps(ak, name, rs, ors):
    root, block = (64, 8, 8), (16, 8, 8)
    U0 = pgen.shock_tube(root, direction=0, gamma=1.4)
    g = oracle.Grid(root, gamma=1.4, riemann=ors)
    m = ak.Mesh(root, block, gamma=1.4, riemann=rs)
    m.upload(U0)
    U = U0
    for _ in range(10):
        dt = oracle.new_dt(U, g, 0.3)
        U, _ = oracle.rk_step(U, g, dt, 2)
        m.step(dt, want_dt_next=False)
    err = max_norm_diff(m.download(), U, 1.4)
    assert err <= 1e-11, (name, err)
    m.close()


@pytest.mark.parametrize("name,rs,ors", SOLVERS)
def test_mixed_close_to_oracle_and_variants_bitwise(ak, name, rs, ors):
    root, block = (32, 32, 32), (16, 16, 16)
    U0 = pgen.turbulence(root, seed=31, kmin=2, kmax=8, mach=0.5)
    g = oracle.Grid(root, riemann=ors)
    dt = oracle.new_dt(U0, g, 0.3)
    ref, _ = oracle.rk_step(U0, g, dt, 2)
    outs = []
    for tile in (0, 1, 2):
        m = ak.Mesh(root, block, precision=1, riemann=rs, ref_rho=1.0, ref_p=1.0)
        m.schedule(tile, 1, 0)
        m.upload(U0)
        m.step(dt)
        outs.append(m.download())
        m.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    err = max_norm_diff(outs[0], ref, G53)
    assert err <= 2e-6, (name, err)


@pytest.mark.parametrize("name,rs,ors", SOLVERS)
def test_mixed_sound_wave_l1_within_one_percent(ak, name, rs, ors):
    n = (32, 32, 32)
    U0, T = pgen.linear_wave(n)
    errs = []
    for prec in (0, 1):
        m = ak.Mesh(n, n, precision=prec, riemann=rs, ref_rho=1.0, ref_p=0.6)
        m.upload(U0)
        t, dt = 0.0, m.new_dt()
        while t < T:
            dt = min(dt, T - t)
            dn = m.step(dt)
            t += dt
            dt = dn
        errs.append(l1_wave_error(m.download(), U0))
        m.close()
    e64, e32 = errs
    assert abs(e32 - e64) <= 0.01 * e64, (name, e32, e64)


@pytest.mark.parametrize("name,rs,ors", SOLVERS)
def test_refined_mesh_parity_and_conservation(ak, name, rs, ors):
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)

    def fn(x, y, z):
        tp = 2 * np.pi
        return (1.0 + 0.3 * np.sin(tp * x) * np.cos(tp * y), 0.5 * np.sin(tp * y + 0.3),
                0.4 * np.cos(tp * z), 0.3 * np.sin(tp * x + tp * z),
                1.0 + 0.2 * np.cos(tp * (x + y + z)))
    P = pgen.field_blocks(t, 32, fn)
    om = oracle.SmrMesh(t, (32, 32, 32), riemann=ors)
    U = om.from_packed(P)
    tot0 = om.totals(U)
    dt = om.new_dt(U, 0.3)
    m = ak.Mesh((32,) * 3, table=t, riemann=rs)
    m.upload_packed(P)
    for _ in range(3):
        U = om.rk_step(U, dt)
        m.step(dt, want_dt_next=False)
    out = m.download_packed()
    ref = om.to_packed(U)
    err = np.abs(out - ref).max() / np.abs(ref).max()
    assert err <= 1e-12, (name, err)
    # composite conservation (cell volumes by level)
    tot = np.zeros(5)
    o = 0
    for r in t:
        nc = int(np.prod(r[4:7]))
        blk = out[o:o + 5 * nc].reshape(5, nc)
        tot += blk.sum(axis=1) * (1.0 / (32 << int(r[0]))) ** 3
        o += 5 * nc
    assert np.abs(tot - tot0).max() <= 1e-13 * (np.abs(tot0).max() + 1), (tot - tot0)
    m.close()
