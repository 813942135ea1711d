"""Static refinement on the GPU: leaf MeshBlocks of several levels advance with one dt
(ghost fill by copy / restriction / prolongation, flux correction at level boundaries),
through the C-ABI, against the SMR oracle.  Cases: the small nested mesh (root 32^3 in 8^3
blocks, two levels of 8^3 blocks, 176 leaves) with a smooth flow and with a Sedov blast,
and the full benchmark mesh (root 128^3 in 32^3 blocks, 16^3 blocks on two levels, 1016
leaves)."""
import math

import numpy as np
import pytest

import oracle
import pgen

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


def _smooth(t, root):
    def fn(x, y, z):
        tp = 2 * np.pi
        return (1.0 + 0.3 * np.sin(tp * x) * np.cos(tp * y), 0.5 * np.sin(tp * y + 0.3),
                0.4 * np.cos(tp * z), 0.3 * np.sin(tp * x + tp * z),
                1.0 + 0.2 * np.cos(tp * (x + y + z)))
    return pgen.field_blocks(t, root, fn)


def _norm_diff(a, b):
    """max over components of max |a-b| / max|b| (packed arrays, 5 vars per block)."""
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _per_var_diff(mesh_table, a, b):
    """max over components of max |a-b| / S_k with S_rho = max|rho|, S_E = max|E| and
    S_M = sqrt(max|rho| max|E|) for the momenta (a momentum scale from rho and E)."""
    diff, scale = np.zeros(5), np.zeros(5)
    o = 0
    for r in mesh_table:
        n = int(np.prod(r[4:7]))
        A, B = a[o:o + 5 * n].reshape(5, n), b[o:o + 5 * n].reshape(5, n)
        diff = np.maximum(diff, np.abs(A - B).max(axis=1))
        scale = np.maximum(scale, np.abs(B).max(axis=1))
        o += 5 * n
    s = np.array([scale[0], 0, 0, 0, scale[4]])
    s[1:4] = np.sqrt(scale[0] * scale[4])
    return float(np.max(diff / s))


def _gpu_mesh(ak, t, root, **kw):
    return ak.Mesh((root,) * 3, table=t, xmin=(-0.5,) * 3, xmax=(0.5,) * 3, **kw)


@pytest.mark.parametrize("precision", [0, 1])
def test_smr_uniform_state_bitwise(ak, precision):
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = pgen.field_blocks(t, 32, lambda x, y, z: (1.3, 0.4, -0.2, 0.3, 0.7))
    m = _gpu_mesh(ak, t, 32, precision=precision, ref_rho=1.0, ref_p=0.7)
    m.upload_packed(P)
    for _ in range(3):
        m.step(1e-3, want_dt_next=False)
    assert np.array_equal(m.download_packed(), P)
    m.close()


def test_smr_fp64_parity_smooth(ak):
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = _smooth(t, 32)
    om = oracle.SmrMesh(t, (32, 32, 32))
    U = om.from_packed(P)
    m = _gpu_mesh(ak, t, 32)
    m.upload_packed(P)
    dt0 = om.new_dt(U, 0.3)
    assert math.isclose(m.new_dt(), dt0, rel_tol=1e-14)
    for s in range(10):
        dt = om.new_dt(U, 0.3)
        U = om.rk_step(U, dt)
        dn = m.step(dt)
        if s == 0:
            assert _per_var_diff(t, m.download_packed(), om.to_packed(U)) <= 1e-12
            assert math.isclose(dn, om.new_dt(U, 0.3), rel_tol=1e-12)
    assert _per_var_diff(t, m.download_packed(), om.to_packed(U)) <= 1e-11
    assert m.counters()[:2] == [0, 0]
    m.close()


def test_smr_fp64_conservation(ak):
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = _smooth(t, 32)
    om = oracle.SmrMesh(t, (32, 32, 32))
    tot0 = om.totals(om.from_packed(P))
    m = _gpu_mesh(ak, t, 32)
    m.upload_packed(P)
    dt = m.new_dt()
    for _ in range(10):
        dt = m.step(dt)
    tot = om.totals(om.from_packed(m.download_packed()))
    assert np.all(np.abs(tot - tot0) / (np.abs(tot0) + 1.0) < 1e-13), tot - tot0
    m.close()


def test_smr_sedov_fp64_parity(ak):
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = pgen.sedov_blocks(t, 32)
    om = oracle.SmrMesh(t, (32, 32, 32))
    U = om.from_packed(P)
    m = _gpu_mesh(ak, t, 32, ref_rho=1.0, ref_p=1e-5)
    m.upload_packed(P)
    for _ in range(20):
        dt = om.new_dt(U, 0.3)
        U = om.rk_step(U, dt)
        m.step(dt, want_dt_next=False)
    a, b = m.download_packed(), om.to_packed(U)
    assert _norm_diff(a, b) <= 1e-11, _norm_diff(a, b)
    assert m.counters()[:2] == [0, 0]
    m.close()


def test_smr_mixed_close_to_oracle(ak):
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = _smooth(t, 32)
    om = oracle.SmrMesh(t, (32, 32, 32))
    U = om.from_packed(P)
    dt = om.new_dt(U, 0.3)
    U = om.rk_step(U, dt)
    m = _gpu_mesh(ak, t, 32, precision=1, ref_rho=1.0, ref_p=1.0)
    m.upload_packed(P)
    m.step(dt)
    assert _per_var_diff(t, m.download_packed(), om.to_packed(U)) <= 2e-6
    m.close()


@pytest.mark.slow
def test_smr_full_mesh_one_step_parity(ak):
    t = pgen.nested_refinement_blocks()  # 1016 leaves, 5,767,168 cells
    P = pgen.sedov_blocks(t, 128)
    om = oracle.SmrMesh(t, (128, 128, 128))
    U = om.from_packed(P)
    dt = om.new_dt(U, 0.3)
    U = om.rk_step(U, dt)
    m = _gpu_mesh(ak, t, 128, ref_rho=1.0, ref_p=1e-5)
    m.upload_packed(P)
    m.step(dt)
    a, b = m.download_packed(), om.to_packed(U)
    assert _norm_diff(a, b) <= 1e-12, _norm_diff(a, b)
    m.close()


def test_smr_autotune_keeps_results_bitwise(ak):
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = _smooth(t, 32)
    a = _gpu_mesh(ak, t, 32)
    a.upload_packed(P)
    a.autotune()
    b = _gpu_mesh(ak, t, 32)
    b.upload_packed(P)
    dt = a.new_dt()
    for _ in range(3):
        a.step(dt, want_dt_next=False)
        b.step(dt, want_dt_next=False)
    assert np.array_equal(a.download_packed(), b.download_packed())
    a.close()
    b.close()


def test_smr_mixed_kernel_variants_bitwise(ak):
    """Every mixed-form kernel variant gives the same bits on a refined mesh (16^3 and
    8^3 leaves: tiles larger than the blocks)."""
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = _smooth(t, 32)
    ref = None
    for tile, seg, order in [(2, 1, 0), (0, 1, 0), (0, 2, 1), (1, 1, 1)]:
        m = _gpu_mesh(ak, t, 32, precision=1, ref_rho=1.0, ref_p=1.0)
        m.schedule(tile, seg, order)
        m.upload_packed(P)
        dt = m.new_dt()
        for _ in range(3):
            m.step(dt, want_dt_next=False)
        out = m.download_packed()
        m.close()
        if ref is None:
            ref = out
        else:
            assert np.array_equal(out, ref), (tile, seg, order)


@pytest.mark.parametrize("precision,recon", [(0, 0), (1, 0), (0, 1), (1, 3)])
def test_smr_fused_launch_bitwise(ak, precision, recon):
    """The persistent fused stage (fill, flux correction and stage in one cooperative
    launch) gives the bits of the separate launches."""
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = _smooth(t, 32)
    outs = []
    for fused in (False, True):
        m = _gpu_mesh(ak, t, 32, precision=precision, recon=recon, rk=3 if recon else 2,
                      ref_rho=1.0, ref_p=1.0)
        m.fuse(fused)
        m.upload_packed(P)
        dt = m.new_dt()
        for _ in range(3):
            m.step(dt, want_dt_next=False)
        outs.append(m.download_packed())
        assert m.counters()[:3] == [0, 0, 0]   # no floors, non-finite cells or timeouts
        m.close()
    assert np.array_equal(outs[0], outs[1])


def test_fuse_refused_without_ghost_fill(ak):
    m = ak.Mesh((32, 32, 32), (16, 16, 16))
    with pytest.raises(ak.AkError):
        m.fuse(True)
    m.close()


def _padded_blocks(m, reg=0):
    """Every block's padded array (5, p3, p2, p1) of a GPU register, ghosts included
    (ak_mesh_layout's rule: rows padded to a multiple of 4 elements)."""
    R = m.regs[reg].cpu().numpy()
    out = []
    for b, r in enumerate(m.table):
        p1, p2, p3 = (int(r[4 + d]) + 2 * m.ng for d in range(3))
        s1 = (p1 + 3) // 4 * 4
        if b == 0:
            assert tuple(m.strides) == (s1 * p2 * p3, s1 * p2, s1, 1)
        o = int(m.offsets[b])
        a = R[o:o + 5 * s1 * p2 * p3].reshape(5, p3, p2, s1)[..., :p1]
        out.append(a)
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_fill_ghosts_refined_matches_oracle(ak, precision):
    """ak_fill_ghosts fills every ghost cell of a refined mesh -- copies, restrictions,
    prolongations, edges and corners -- as the SMR oracle does, also on meshes whose
    stages read same-level halos directly (and so fill only level boundaries)."""
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = _smooth(t, 32)
    om = oracle.SmrMesh(t, (32, 32, 32))
    U = om.from_packed(P)
    om.fill_ghosts(U)
    m = _gpu_mesh(ak, t, 32, precision=precision, ref_rho=1.0, ref_p=1.0)
    m.upload_packed(P)
    m.fill_ghosts(0)
    m.stream.synchronize()
    got = _padded_blocks(m)
    for b in range(len(t)):
        want = om.block(U, b)
        assert np.allclose(got[b], want, rtol=1e-14, atol=1e-14), b
    m.close()


@pytest.mark.parametrize("precision,recon", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_direct_halo_reads_match_full_fill_bitwise(ak, precision, recon):
    """Without FOFC the stage kernels read same-level halo cells from the neighbour
    blocks and the fill before a stage keeps only the level-boundary entries; with FOFC
    (here on a smooth flow that flags no cell) every ghost cell is filled and read from
    the block's own ghost zone.  Both give the same bits."""
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = _smooth(t, 32)
    outs = []
    for fofc in (False, True):
        m = _gpu_mesh(ak, t, 32, precision=precision, recon=recon, rk=3 if recon else 2,
                      fofc=fofc, ref_rho=1.0, ref_p=1.0)
        m.upload_packed(P)
        dt = m.new_dt()
        for _ in range(3):
            m.step(dt, want_dt_next=False)
        outs.append(m.download_packed())
        assert m.counters()[:3] == [0, 0, 0]
        m.close()
    assert np.array_equal(outs[0], outs[1])
