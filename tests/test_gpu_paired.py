"""The paired mixed-form stage kernel (x1/x2 edges and faces in the two lanes of packed
FP32x2 arithmetic) for the three-ghost-cell reconstructions (PPM4, WENO-Z, PPMX), against
the kernel with one thread per column: the same bits on uniform meshes with ragged tiles,
with x3 segments and either CTA order, with HLLC (the kernel's fast path) and HLLE, with
FOFC and on a refined mesh; and within the mixed form's tolerance of the FP64 oracle.
Meshes whose blocks have an odd number of cells in x1 do not offer the paired kernel."""
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


def _steps(m, U0, steps):
    m.upload(U0)
    dt = m.new_dt()
    for _ in range(steps):
        m.step(dt, want_dt_next=False)
    return m.download(), dt


@pytest.mark.parametrize("recon", [1, 2, 3])
@pytest.mark.parametrize("riemann,fofc", [(0, False), (1, False), (0, True)])
def test_paired_3ghost_kernel_bitwise_and_close(ak, recon, riemann, fofc):
    root, block = (40, 24, 32), (20, 12, 16)   # ragged 16x16 tiles, 2x2x2 blocks
    U0 = pgen.turbulence(root, seed=13, kmin=1, kmax=5, mach=0.8)
    outs, dt = [], None
    for tile, seg, order in [(2, 1, 0), (0, 1, 0), (0, 2, 1)]:
        m = ak.Mesh(root, block, recon=recon, rk=3, precision=ak.AK_MIXED, riemann=riemann,
                    fofc=fofc, ref_rho=1.0, ref_p=1.0)
        m.schedule(tile, seg, order)
        out, dt = _steps(m, U0, 2)
        assert m.counters()[:2] == [0, 0]
        m.close()
        outs.append(out)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    g = oracle.Grid(root, recon=recon, riemann=riemann)
    O = U0
    for _ in range(2):
        O, _ = oracle.rk_step(O, g, dt, 3)
    err = max_norm_diff(outs[0], O, G53)
    assert err <= 5e-6, err


def test_paired_ppm4_refined_mesh_bitwise(ak):
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    P = pgen.field_blocks(t, 32, lambda x, y, z: (1.0 + 0.2 * np.sin(2 * np.pi * x), 0.3, -0.2,
                                                  0.1 * np.cos(2 * np.pi * y), 1.0))
    outs = []
    for tile in (2, 0):
        m = ak.Mesh((32, 32, 32), table=t, recon=1, rk=3, precision=1, xmin=(-0.5,) * 3,
                    xmax=(0.5,) * 3, ref_rho=1.0, ref_p=1.0)
        m.schedule(tile, 1, 0)
        m.upload_packed(P)
        dt = m.new_dt()
        for _ in range(3):
            m.step(dt, want_dt_next=False)
        outs.append(m.download_packed())
        assert m.counters()[:2] == [0, 0]
        m.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("recon", [0, 1])
def test_odd_x1_blocks_take_the_column_kernel(ak, recon):
    root, block = (33, 18, 21), (11, 9, 7)
    m = ak.Mesh(root, block, recon=recon, rk=3 if recon else 2, precision=ak.AK_MIXED,
                ref_rho=1.0, ref_p=1.0)
    with pytest.raises(ak.AkError):
        m.schedule(0, 1, 0)
    U0 = pgen.turbulence(root, seed=17, kmin=1, kmax=5, mach=1.0)
    out, dt = _steps(m, U0, 1)
    m.close()
    g = oracle.Grid(root, recon=recon)
    ref, _ = oracle.rk_step(U0, g, dt, 3 if recon else 2)
    assert max_norm_diff(out, ref, G53) <= 2e-6
