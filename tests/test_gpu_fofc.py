"""First-order flux correction (FOFC) on the GPU against the oracle: Mach-5 turbulence,
where the plain scheme needs floors, on a mesh of 8 MeshBlocks (corrections cross block
boundaries), FP64 parity step by step with the oracle's dt sequence and the same number
of corrected cells, PPM4 + RK3, the mixed form, and a two-level refined mesh whose
flagged cells sit on both levels and next to the level boundaries."""
import numpy as np
import pytest

import oracle
import pgen
from _helpers import max_norm_diff

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0
N = (24, 24, 24)


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


def _run(ak, precision, recon, rk, steps, tol, seed=3):
    U = pgen.turbulence(N, seed=seed, kmin=1, kmax=6, mach=5.0)
    g = oracle.Grid(N, recon=recon, fofc=True)
    m = ak.Mesh(N, (12, 12, 12), recon=recon, rk=rk, precision=precision, fofc=True,
                ref_rho=1.0, ref_p=1.0)
    m.upload(U)
    tot0 = U.reshape(5, -1).sum(axis=1)
    flagged = 0
    errs = []
    for _ in range(steps):
        dt = oracle.new_dt(U, g, 0.3)
        U, nf, nfl = oracle.rk_step_fofc(U, g, dt, rk)
        assert nf == 0
        flagged += nfl
        m.step(dt, want_dt_next=False)
        errs.append(max_norm_diff(m.download(), U, G53))
    out = m.download()
    c = m.counters()
    m.close()
    assert max(errs) <= tol, errs
    assert c[0] == 0 and c[1] == 0, c       # no floors, no non-finite cells
    # FP64: conservation to round-off; mixed: to the FP32 rounding of the divergence
    tot = out.reshape(5, -1).sum(axis=1)
    scale = np.abs(out).reshape(5, -1).sum(axis=1)
    ctol = 1e-12 if precision == 0 else 1e-8
    assert np.all(np.abs(tot - tot0) <= ctol * scale), (tot - tot0)
    return c[3], flagged


def test_fp64_plm_rk2_mach5_step_parity(ak):
    gpu_cells, oracle_cells = _run(ak, 0, 0, 2, 15, 1e-10)
    assert oracle_cells > 0
    assert gpu_cells == oracle_cells, (gpu_cells, oracle_cells)


# PPM4, WENO-Z, PPMX.  WENO-Z and PPMX can overshoot to a face state with rho p < 0:
# its sound speed is NaN, and the solvers' wave-speed tests then take the branch the
# definition takes (an upwind flux, or a NaN flux whose cells FOFC flags and redoes).
@pytest.mark.parametrize("recon,seed,steps", [(1, 3, 8), (2, 3, 8), (2, 1, 8), (3, 3, 8)])
def test_fp64_3ghost_rk3_mach5_step_parity(ak, recon, seed, steps):
    gpu_cells, oracle_cells = _run(ak, 0, recon, 3, steps, 1e-10, seed)
    assert oracle_cells > 0
    assert gpu_cells == oracle_cells, (gpu_cells, oracle_cells)


def test_mixed_mach5_positive_and_close(ak):
    gpu_cells, oracle_cells = _run(ak, 1, 0, 2, 15, 5e-3)
    assert gpu_cells > 0 and oracle_cells > 0


def test_plain_scheme_needs_floors_on_the_gpu(ak):
    U = pgen.turbulence(N, seed=3, kmin=1, kmax=6, mach=5.0)
    g = oracle.Grid(N)
    m = ak.Mesh(N, (12, 12, 12))
    m.upload(U)
    for _ in range(15):
        dt = oracle.new_dt(U, g, 0.3)
        U, _ = oracle.rk_step(U, g, dt, 2)
        m.step(dt, want_dt_next=False)
    assert m.counters()[0] > 0 and m.counters()[3] == 0
    m.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 5e-3)])
def test_refined_mesh_cold_shear_parity(ak, precision, tol):
    t = pgen.nested_refinement_blocks(16, 4, 8, 1)
    # p = 1e-3: flagged cells on both levels, coarse and fine ones next to the level
    # boundary among them
    P = pgen.cold_shear_blocks(t, 16, 0.001)
    om = oracle.SmrMesh(t, (16, 16, 16), fofc=True)
    U = om.from_packed(P)
    m = ak.Mesh((16,) * 3, table=t, fofc=True, precision=precision, xmin=(-0.5,) * 3,
                xmax=(0.5,) * 3, ref_rho=1.0, ref_p=0.001)
    m.upload_packed(P)
    tot0 = om.totals(U)
    flagged, errs = 0, []
    for _ in range(4):
        dt = om.new_dt(U, 0.3)
        U, nfl = om.rk_step_fofc(U, dt, 2)
        flagged += nfl
        m.step(dt, want_dt_next=False)
        ref = om.to_packed(U)
        errs.append(np.abs(m.download_packed() - ref).max() / np.abs(ref).max())
    out = om.from_packed(m.download_packed())
    c = m.counters()
    m.close()
    assert flagged > 0
    assert max(errs) <= tol, errs
    # no non-finite value; floors do occur, in prolongated ghost cells of this cold flow
    # (the conserved-variable interpolation can leave u_g below its floor there), and
    # both sides apply them
    assert c[1] == 0, c
    tot = om.totals(out)
    ctol = 1e-13 if precision == 0 else 1e-8
    assert np.all(np.abs(tot - tot0) <= ctol * (np.abs(tot0) + 1.0)), tot - tot0
    if precision == 0:
        assert c[3] == flagged, (c[3], flagged)
    else:
        assert c[3] > 0


def test_fused_launch_bitwise_with_fofc(ak):
    # a uniform FOFC mesh needs a ghost fill: the fused stage launch gives the same bits
    outs = []
    for fused in (False, True):
        U = pgen.turbulence(N, seed=3, kmin=1, kmax=6, mach=5.0)
        g = oracle.Grid(N)
        m = ak.Mesh(N, (12, 12, 12), fofc=True)
        m.fuse(fused)
        m.upload(U)
        for _ in range(12):
            dt = oracle.new_dt(U, g, 0.3)
            U, _ = oracle.rk_step(U, g, dt, 2)
            m.step(dt, want_dt_next=False)
        outs.append((m.download(), m.counters()))
        m.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1] and outs[0][1][3] > 0


def test_list_overflow_is_reported(ak):
    # A uniform state with negative internal energy flags every cell of a 64^3 mesh, four
    # times the list's 65536 entries (max(65536, cells / 64)).  The listed cells are
    # corrected, the others keep their stage output; with uniform fluxes both leave the
    # state as it was.  Each step reports AK_EOVERFLOW (the drop count starts again after
    # a report), and every stage counts a full list of corrected cells.
    n = (64, 64, 64)
    U = np.zeros((5,) + n)
    U[0] = 1.0
    U[4] = -0.1
    m = ak.Mesh(n, (32, 32, 32), fofc=True)
    m.upload(U)
    for s in (1, 2):
        with pytest.raises(ak.AkError) as e:
            m.step(1e-4)
        assert e.value.status == ak.AK_EOVERFLOW, str(e.value)
        assert "not corrected" in str(e.value)
        c = m.counters()
        assert c[3] == 2 * s * 65536 and c[0] > 0 and c[1] == 0 and c[2] == 0, c
    out = m.download()
    m.close()
    assert np.allclose(out, U, rtol=0.0, atol=1e-12)
