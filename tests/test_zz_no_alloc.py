"""ak_cfl_dt_noalloc: the CFL time step computed with no device allocation.

Callers that cannot call cudaMalloc (their host code's pool owns all device memory,
or the device is out of memory when they need a time step) use this entry point; its
scratch is a static device array.  It must give the same dt as ak_new_dt, call after
call, for meshes of different sizes sharing that one array.  This file is collected
last so that a failure here stops a -x run only after every other test ran.
"""
import math

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


def _noalloc_dt(ak, m, reg=0):
    dx = [1.0 / m.root_nx[d] for d in range(3)]
    return ak.ak_cfl_dt_noalloc(m.regs[reg].data_ptr(), m.nblocks, m.block_nx, m.ng, dx,
                                5.0 / 3.0, 0.3, m.stream.cuda_stream)


@pytest.mark.parametrize("root,block,recon", [((64, 48, 32), (16, 16, 16), 0),
                                             ((36, 24, 18), (12, 12, 9), 1)])
def test_noalloc_dt_matches_ak_new_dt_twice(ak, root, block, recon):
    U = pgen.turbulence(root, seed=41, kmin=1, kmax=6, mach=1.5)
    m = ak.Mesh(root, block, recon=recon, rk=2 if recon == 0 else 3)
    m.upload(U)
    ref = m.new_dt(0)
    for _ in range(2):  # two calls in a row share the static scratch
        dt = _noalloc_dt(ak, m)
        assert math.isclose(dt, ref, rel_tol=1e-14), (dt, ref)
    m.close()


def test_noalloc_dt_after_a_larger_call_and_after_steps(ak):
    big = ak.Mesh((64, 64, 64), (16, 16, 16))
    big.upload(pgen.turbulence((64, 64, 64), seed=42, kmin=1, kmax=6, mach=2.0))
    small = ak.Mesh((16, 16, 16), (16, 16, 16))
    small.upload(pgen.uniform((16, 16, 16), rho=2.0, p=0.5, v=(0.1, 0.0, 0.0)))
    assert math.isclose(_noalloc_dt(ak, big), big.new_dt(0), rel_tol=1e-14)
    # one block now: stale partial minima of the 64-block call must not leak in
    assert math.isclose(_noalloc_dt(ak, small), small.new_dt(0), rel_tol=1e-14)
    big.step(0.0)
    assert math.isclose(_noalloc_dt(ak, big), big.new_dt(0), rel_tol=1e-14)
    big.close()
    small.close()


def test_noalloc_calls_allocate_nothing(ak):
    """After one warm-up call (which may load the library's device code on the device),
    further calls leave the device's free memory and torch's allocator unchanged."""
    import torch
    root, block = (32, 32, 32), (16, 16, 16)
    m = ak.Mesh(root, block)
    m.upload(pgen.turbulence(root, seed=43, kmin=1, kmax=6, mach=1.0))
    ref = m.new_dt(0)
    _noalloc_dt(ak, m)                                   # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for _ in range(5):
        assert math.isclose(_noalloc_dt(ak, m), ref, rel_tol=1e-14)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0, (free0, free1)
    for key in ("allocated_bytes.all.current", "reserved_bytes.all.current",
                "allocation.all.allocated"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
    m.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(ak):
    m = ak.Mesh((16, 16, 16), (16, 16, 16))
    with pytest.raises(ak.AkError) as e:
        ak.ak_cfl_dt_noalloc(m.regs[0].data_ptr(), 65537, (16, 16, 16), 2, (1, 1, 1),
                             5.0 / 3.0, 0.3, m.stream.cuda_stream)
    assert e.value.status == ak.AK_EINVAL and "65536" in str(e.value)
    m.close()
