"""The large configurations at full size, in the launch configuration the benchmark's
--case c3 / c5 runs time: 512^3 in 64 MeshBlocks of 128^3 with PPM4 + HLLC + RK3 (FP64
and mixed), and 768^3 in 512 MeshBlocks of 96^3, mixed, Mach-2 solenoidal turbulence.

The oracle cannot step these grids, so one step is checked on sampled outputs: 64^3
sub-boxes of the initial state are stepped by the (periodic) oracle with the GPU's dt.
Only the cells within the step's stencil reach of a sub-box edge see the wrong (wrapped)
neighbours -- 3 stages x 3 cells for PPM4 + RK3, 2 x 2 for PLM + RK2 -- so the interior
must match the GPU to the parity tolerance.  Longer runs are checked by properties that
hold at any size: conservation, no floors, a steady dt."""
import numpy as np
import pytest

import oracle
import pgen
from _helpers import max_norm_diff

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


def _totals(m, reg=0):
    """Sum of the interior of a uniform mesh's register, per variable (on the device)."""
    g = m.ng
    R = m.register_view(reg)
    m.stream.synchronize()
    return R[:, :, g:-g, g:-g, g:-g].sum(dim=(0, 2, 3, 4)).cpu().numpy()


@pytest.mark.slow
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-6)])
def test_c3_512_ppm_rk3_one_step_subbox_replay(ak, precision, tol):
    import torch
    root = 512
    U0 = pgen.turbulence_device((root,) * 3, seed=3, kmin=2, kmax=8, mach=0.5)
    m = ak.Mesh((root,) * 3, (128,) * 3, recon=ak.AK_PPM4, rk=3, precision=precision,
                ref_rho=1.0, ref_p=1.0)
    m.upload_device(U0)
    dt = m.new_dt()
    boxes = [(100, 100, 100), (440, 16, 250)]
    subs = {lo: U0[:, lo[2]:lo[2] + 64, lo[1]:lo[1] + 64, lo[0]:lo[0] + 64].clone()
            for lo in boxes}
    tot0 = _totals(m)
    del U0
    torch.cuda.empty_cache()
    m.step(dt, want_dt_next=False)
    assert m.counters()[:2] == [0, 0]
    for lo, sub in subs.items():
        sub_np = sub.cpu().numpy()
        grid = oracle.Grid((64,) * 3, length=(64 / root,) * 3, recon=oracle.PPM4)
        ref, nf = oracle.rk_step(sub_np, grid, dt, 3)
        assert nf == 0
        got = m.download_box(lo, (64,) * 3)
        c = slice(9, 55)
        err = max_norm_diff(got[:, c, c, c], ref[:, c, c, c], G53)
        assert err <= tol, (lo, err)
    tot1 = _totals(m)
    for k in range(5):
        assert abs(tot1[k] - tot0[k]) <= 1e-12 * (abs(tot0[k]) + root ** 3), (k, tot1 - tot0)
    m.close()


@pytest.mark.slow
def test_c5_768_mixed_mach2_replay_and_50_steps(ak):
    import torch
    root = 768
    U0 = pgen.turbulence_device((root,) * 3, seed=5, kmin=2, kmax=16, mach=2.0,
                                solenoidal=True)
    m = ak.Mesh((root,) * 3, (96,) * 3, precision=ak.AK_MIXED, ref_rho=1.0, ref_p=1.0)
    m.upload_device(U0)
    dt = m.new_dt()
    lo = (90, 300, 700)
    sub = U0[:, lo[2]:lo[2] + 64, lo[1]:lo[1] + 64, lo[0]:lo[0] + 64].cpu().numpy()
    del U0
    torch.cuda.empty_cache()
    tot0 = _totals(m)
    m.step(dt, want_dt_next=False)
    grid = oracle.Grid((64,) * 3, length=(64 / root,) * 3)
    ref, nf = oracle.rk_step(sub, grid, dt, 2)
    assert nf == 0
    got = m.download_box(lo, (64,) * 3)
    c = slice(4, 60)
    err = max_norm_diff(got[:, c, c, c], ref[:, c, c, c], G53)
    assert err <= 2e-6, err
    dts = [dt]
    for _ in range(49):
        dts.append(m.step(0.0))
    assert m.counters()[:2] == [0, 0]
    assert all(d > 0 for d in dts) and max(dts) / min(dts) < 2.0, (min(dts), max(dts))
    tot1 = _totals(m)
    for k in range(5):
        assert abs(tot1[k] - tot0[k]) <= 1e-11 * (abs(tot0[k]) + root ** 3), (k, tot1 - tot0)
    m.close()
