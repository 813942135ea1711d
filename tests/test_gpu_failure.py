"""Failure detection without a GPU fault: the bounded wait of the grid barrier that the
fused stage uses runs out when a CTA never arrives (a flag that nothing sets).  The host
sees AK_ETIMEOUT and the timeout count, and the mesh keeps stepping with the right bits."""
import numpy as np
import pytest

import pgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ak():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2409_16053_gb300 import build
    build.build()
    from paper_2409_16053_gb300 import ak as mod
    return mod


def _mesh(ak):
    t = pgen.nested_refinement_blocks(16, 4, 8, 1)
    m = ak.Mesh((16,) * 3, table=t, xmin=(-0.5,) * 3, xmax=(0.5,) * 3)
    m.fuse(True)
    P = pgen.field_blocks(t, 16, lambda x, y, z: (1.0 + 0.2 * np.sin(2 * np.pi * x), 0.3, -0.2,
                                                  0.1 * np.cos(2 * np.pi * y), 1.0))
    m.upload_packed(P)
    return m


def test_barrier_met(ak):
    m = _mesh(ak)
    ak.ak_selftest_barrier(m.handle, False)
    assert m.counters()[2] == 0
    m.close()


def test_barrier_wait_runs_out_and_mesh_stays_usable(ak):
    a, b = _mesh(ak), _mesh(ak)
    with pytest.raises(ak.AkError) as e:
        ak.ak_selftest_barrier(a.handle, True)
    assert e.value.status == ak.AK_ETIMEOUT
    assert a.counters()[2] == 1
    # the status was reported once; the barrier state is clean for the fused stage
    dt = a.new_dt()
    assert dt == b.new_dt()
    for _ in range(2):
        a.step(dt, want_dt_next=False)
        b.step(dt, want_dt_next=False)
    assert np.array_equal(a.download_packed(), b.download_packed())
    assert a.counters()[2] == 1 and b.counters()[2] == 0
    a.close()
    b.close()
