"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
entry point include/ak.h declares, and rejects invalid mesh descriptions before any
device work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ak():
    from paper_2409_16053_gb300 import build
    build.build()
    from paper_2409_16053_gb300 import ak as mod
    return mod


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:ak_status|void|const char\*)\s+(ak_\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(ak):
    lib = ctypes.CDLL(ak._build.LIB)
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(ak.EXPORTED) <= set(names)


def _desc(ak, **kw):
    table = ak.uniform_block_table((32, 32, 32), (16, 16, 16))
    d = ak.ak_mesh_desc()
    d.nblocks = table.shape[0]
    d.nghost = 2
    d.blocks = table.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    for a in range(3):
        d.xmin[a], d.xmax[a], d.root_nx[a] = 0.0, 1.0, 32
    d.recon, d.rk, d.precision = ak.AK_PLM, 2, ak.AK_FP64
    d.gamma, d.cfl, d.ref_rho, d.ref_p = 5 / 3, 0.3, 1.0, 1.0
    for k, v in kw.items():
        setattr(d, k, v)
    return d, table


@pytest.mark.parametrize("field,value", [
    ("nghost", 3), ("rk", 4), ("recon", 7), ("precision", 5), ("gamma", 1.0),
    ("cfl", 0.0), ("cfl", 1.5), ("nblocks", 0), ("nblocks", 7)])
def test_invalid_descriptions_rejected(ak, field, value):
    d, table = _desc(ak, **{field: value})
    out = ctypes.c_void_p()
    st = ak._lib.ak_mesh_create(ctypes.byref(d), None, ctypes.byref(out))
    assert st == ak.AK_EINVAL, (field, value, st)
    assert out.value is None
    assert ak.ak_last_error()


def test_mixed_needs_background_and_tiling_checked(ak):
    d, table = _desc(ak, precision=1, ref_rho=0.0)
    out = ctypes.c_void_p()
    assert ak._lib.ak_mesh_create(ctypes.byref(d), None, ctypes.byref(out)) == ak.AK_EINVAL
    d, table = _desc(ak)
    table[3, 1] = table[2, 1]  # duplicate a block origin -> overlap
    table[3, 2] = table[2, 2]
    d.blocks = table.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    assert ak._lib.ak_mesh_create(ctypes.byref(d), None, ctypes.byref(out)) == ak.AK_EINVAL
    assert "overlap" in ak.ak_last_error()


def test_null_arguments_rejected(ak):
    assert ak._lib.ak_mesh_create(None, None, None) == ak.AK_EINVAL
    assert ak._lib.ak_fill_ghosts(None, 0) == ak.AK_EINVAL
    assert ak._lib.ak_stage(None, 1, 0.1) == ak.AK_EINVAL
    assert ak._lib.ak_step(None, 0.1, None) == ak.AK_EINVAL
    ak.ak_mesh_destroy(None)


def test_pack_unpack_round_trip_host(ak):
    # the binding's global <-> block-order conversion (host only, no device)
    class M(ak.Mesh):
        def __init__(self):
            self.root_nx, self.block_nx = (12, 8, 6), (4, 4, 3)
            self.nb = (3, 2, 2)
    m = M()
    U = np.random.default_rng(0).normal(size=(5, 6, 8, 12))
    P = m.pack(U)
    # block (bx=1, by=1, bz=1) is block index (1*2+1)*3+1 = 10; its var 4 cell (2,3,1)
    blk = P.reshape(12, 5, 3, 4, 4)[10]
    assert blk[4, 2, 3, 1] == U[4, 3 + 2, 4 + 3, 4 + 1]
    assert np.array_equal(m.unpack(P), U)


def _desc_table(ak, table, root, recon=0):
    d = ak.ak_mesh_desc()
    d.nblocks = table.shape[0]
    d.nghost = 2 if recon == 0 else 3
    d.blocks = table.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    for a in range(3):
        d.xmin[a], d.xmax[a], d.root_nx[a] = -0.5, 0.5, root
    d.recon, d.rk, d.precision = recon, 2, ak.AK_FP64
    d.gamma, d.cfl, d.ref_rho, d.ref_p = 5 / 3, 0.3, 1.0, 1.0
    return d


def test_refined_mesh_validation(ak):
    import pgen
    out = ctypes.c_void_p()
    # valid nested refinement: passes validation (fails later only without a GPU)
    t = pgen.nested_refinement_blocks(32, 8, 8, 2)
    d = _desc_table(ak, t, 32)
    st = ak._lib.ak_mesh_create(ctypes.byref(d), None, ctypes.byref(out))
    assert st != ak.AK_EINVAL, ak.ak_last_error()
    if st == ak.AK_OK:
        ak.ak_mesh_destroy(out)
    # a level-1 block removed: the leaves no longer tile the box
    t2 = t[1:].copy()
    d = _desc_table(ak, t2, 32)
    assert ak._lib.ak_mesh_create(ctypes.byref(d), None, ctypes.byref(out)) == ak.AK_EINVAL
    # level 2 next to level 0 (two-level jump): no level-1 buffer around level 2
    t3 = pgen.nested_refinement_blocks(32, 8, 8, 2)
    lv1 = np.where(t3[:, 0] == 1)[0]
    # replace level-1 leaves by their level-0 parents where possible is complex; instead
    # move one level-2 block far away so that it overlaps a level-0 leaf
    bad = t3.copy()
    bad[np.where(bad[:, 0] == 2)[0][0], 1:4] = 0
    d = _desc_table(ak, bad, 32)
    assert ak._lib.ak_mesh_create(ctypes.byref(d), None, ctypes.byref(out)) == ak.AK_EINVAL
    assert len(lv1) == 56


def test_binding_constants_match_the_header(ak):
    # every enum value and integer #define of include/ak.h that the binding names has the
    # header's value, and every status code of the header has a name in the binding
    src = open(os.path.join(ROOT, "include", "ak.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {n: int(v) for n, v in re.findall(r"\b(AK_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    consts.update({n: int(v) for n, v in re.findall(r"#define\s+(AK_[A-Z0-9_]+)\s+(-?\d+)\s*$",
                                                    src, re.M)})
    assert {"AK_OK", "AK_EOVERFLOW", "AK_PPMX", "AK_LLF", "AK_MIXED"} <= set(consts)
    named = [n for n in consts if hasattr(ak, n)]
    assert len(named) >= 16, named
    for n in named:
        assert getattr(ak, n) == consts[n], n
    status = re.search(r"typedef enum \{(.*?)\} ak_status;", src, re.S).group(1)
    for n in re.findall(r"\b(AK_[A-Z0-9_]+)\s*=", status):
        assert ak._STATUS_NAMES[consts[n]] == n


def _uniform_rows(n, b, level=0, skip=()):
    return [(level, i, j, k, b, b, b) for k in range(0, n, b) for j in range(0, n, b)
            for i in range(0, n, b) if (i, j, k) not in skip]


def _invalid_table(case):
    """(table, root, recon, message fragment) of a mesh that breaks one rule."""
    import pgen
    base = pgen.nested_refinement_blocks(16, 4, 8, 1)
    if case == "level":
        t = base.copy()
        t[0, 0] = 16
        return t, 16, 0, "level out of range"
    if case == "small_block":
        return np.array(_uniform_rows(4, 1), np.int32), 4, 0, "block sizes must be >= nghost"
    if case == "mixed_sizes":
        t = base.copy()
        t[0, 4] = 2
        return t, 16, 0, "same size"
    if case == "off_lattice":
        t = base.copy()
        t[1, 1] += 1
        return t, 16, 0, "block lattice"
    if case == "not_tiling_level":
        # 16^3 in 4^3 blocks on a root of 18: the blocks do not divide the level
        return np.array(_uniform_rows(16, 4), np.int32), 18, 0, "tile each level"
    if case == "single_block_refined":
        t = np.array([(0, 0, 0, 0, 8, 8, 8), (1, 0, 0, 0, 4, 4, 4)], np.int32)
        return t, 8, 0, "more than one block per level"
    if case == "odd_refined":
        t = np.array(_uniform_rows(20, 5) + [(1, 0, 0, 0, 10, 10, 10)], np.int32)
        return t, 20, 0, "even block sizes"
    if case == "over_coarser":
        # a level-0 block put back where level 1 already covers the box
        t = np.concatenate([base, np.array([(0, 4, 4, 4, 4, 4, 4)], np.int32)])
        return t, 16, 0, "overlaps a coarser block"
    if case == "gap":
        return base[1:].copy(), 16, 0, "do not tile the domain"
    if case == "level_jump":
        # root 16 in 4^3 blocks; the corner block refined to level 1, and that block's
        # own corner block refined to level 2, which then touches level 0 (periodic)
        rows = _uniform_rows(16, 4, 0, skip={(0, 0, 0)})
        rows += _uniform_rows(8, 4, 1, skip={(0, 0, 0)})
        rows += _uniform_rows(8, 4, 2)
        return np.array(rows, np.int32), 16, 0, "more than one level"
    raise KeyError(case)


@pytest.mark.parametrize("case", [
    "level", "small_block", "mixed_sizes", "off_lattice", "not_tiling_level",
    "single_block_refined", "odd_refined", "over_coarser", "gap", "level_jump"])
def test_each_mesh_rule_is_enforced(ak, case):
    # every refusal of ak_mesh_create's mesh validation, one broken rule at a time; the
    # checks run on the host before any device call
    t, root, recon, msg = _invalid_table(case)
    d = _desc_table(ak, t, root, recon)
    out = ctypes.c_void_p()
    st = ak._lib.ak_mesh_create(ctypes.byref(d), None, ctypes.byref(out))
    assert st == ak.AK_EINVAL, (case, st, ak.ak_last_error())
    assert msg in ak.ak_last_error(), (case, ak.ak_last_error())
    assert out.value is None


def test_valid_tables_pass_the_host_checks(ak):
    # the refined tables of the tests and the bench pass validation (a machine without a
    # GPU then stops at the first device call, with AK_ECUDA)
    import pgen
    tables = [(pgen.nested_refinement_blocks(16, 4, 8, 1), 16),
              (pgen.nested_refinement_blocks(32, 8, 8, 2), 32),
              (pgen.nested_refinement_blocks(), 128)]
    rows = _uniform_rows(16, 4, 0, skip={(0, 0, 0)}) + _uniform_rows(8, 4, 1)
    tables.append((np.array(rows, np.int32), 16))
    for t, root in tables:
        d = _desc_table(ak, t, root)
        out = ctypes.c_void_p()
        st = ak._lib.ak_mesh_create(ctypes.byref(d), None, ctypes.byref(out))
        assert st in (ak.AK_OK, ak.AK_ECUDA, ak.AK_ENOMEM), (st, ak.ak_last_error())
        if st == ak.AK_OK:
            ak.ak_mesh_destroy(out)
