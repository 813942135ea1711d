"""Pins of the static-refinement (SMR) oracle: prolongation and restriction against their
definitions, a uniform state across levels, composite conservation with flux correction
(and its failure without, as a negative control), equality with the uniform-grid oracle
when every block is on one level, the Sedov-Taylor blast radius across levels, second-
order convergence of a sound wave through two level boundaries, and the locality of FOFC
on two levels."""
import math

import numpy as np
import pytest

import oracle
import pgen

G53 = 5.0 / 3.0


def small_table():
    # root 32^3 in 8^3 blocks, level 1 over the central half, level 2 over the central
    # quarter, 8^3 blocks: 56 + 56 + 64 leaves, 90,112 cells
    return pgen.nested_refinement_blocks(32, 8, 8, 2)


def test_small_mesh_geometry():
    t = small_table()
    assert [int((t[:, 0] == l).sum()) for l in range(3)] == [56, 56, 64]
    # the leaves tile the box: volumes add up to 1
    vol = sum(np.prod(r[4:7]) * (1.0 / (32 << int(r[0]))) ** 3 for r in t)
    assert math.isclose(vol, 1.0, rel_tol=1e-15)
    big = pgen.nested_refinement_blocks()
    assert [int((big[:, 0] == l).sum()) for l in range(3)] == [56, 448, 512]


def test_prolongation_exact_on_linear_data():
    rng = np.random.default_rng(0)
    for _ in range(100):
        uc, a = rng.normal(size=1)[0], rng.normal(size=3)
        um, up = uc - a, uc + a
        for hi in [(0, 0, 0), (1, 0, 1), (1, 1, 1), (0, 1, 0)]:
            expect = uc + sum((0.25 if h else -0.25) * a[d] for d, h in enumerate(hi))
            assert math.isclose(oracle.prolong(uc, um, up, hi), expect, rel_tol=1e-14,
                                abs_tol=1e-14)


def test_restriction_of_prolongation_is_identity():
    rng = np.random.default_rng(1)
    for _ in range(200):
        uc = rng.normal()
        um, up = uc + rng.normal(size=3), uc + rng.normal(size=3)
        fine = [oracle.prolong(uc, um, up, (i, j, k)) for k in (0, 1) for j in (0, 1)
                for i in (0, 1)]
        assert math.isclose(oracle.restrict(fine), uc, rel_tol=1e-14, abs_tol=1e-15)


def test_prolongation_is_limited_at_extrema():
    # a coarse extremum has zero minmod slope: all fine values equal the coarse value
    assert oracle.prolong(2.0, [1.0, 1.0, 1.0], [1.5, 0.5, 1.0], (1, 0, 1)) == 2.0


def test_uniform_state_bitwise_across_levels():
    t = small_table()
    m = oracle.SmrMesh(t, (32, 32, 32))
    P = pgen.field_blocks(t, 32, lambda x, y, z: (1.3, 0.4, -0.2, 0.3, 0.7))
    U = m.from_packed(P)
    U1 = m.rk_step(U, 1e-3)
    assert np.array_equal(m.to_packed(U1), P)


def _smooth_blocks(t, root_nx):
    def fn(x, y, z):
        tp = 2 * np.pi
        rho = 1.0 + 0.3 * np.sin(tp * x) * np.cos(tp * y)
        v1 = 0.5 * np.sin(tp * y + 0.3)
        v2 = 0.4 * np.cos(tp * z)
        v3 = 0.3 * np.sin(tp * x + tp * z)
        p = 1.0 + 0.2 * np.cos(tp * (x + y + z))
        return rho, v1, v2, v3, p
    return pgen.field_blocks(t, root_nx, fn)


def test_composite_conservation_and_negative_control():
    t = small_table()
    P = _smooth_blocks(t, 32)
    res = {}
    for fc in (True, False):
        m = oracle.SmrMesh(t, (32, 32, 32), flux_correction=fc)
        U = m.from_packed(P)
        tot0 = m.totals(U)
        dt = m.new_dt(U, 0.3)
        for _ in range(3):
            U = m.rk_step(U, dt)
        res[fc] = np.abs(m.totals(U) - tot0) / (np.abs(tot0) + 1.0)
    assert res[True].max() < 1e-13, res[True]
    # without the correction the level interfaces leak, far above round-off
    assert res[False].max() > 1e-7, res[False]


@pytest.mark.parametrize("riemann,recon", [
    (oracle.HLLC, oracle.PLM), (oracle.HLLE, oracle.PLM), (oracle.LLF, oracle.PLM),
    (oracle.HLLC, oracle.PPMX), (oracle.HLLC, oracle.WENOZ)])
def test_single_level_equals_uniform_oracle(riemann, recon):
    # every block on level 0: the SMR oracle must reproduce the uniform-grid oracle
    t = pgen.nested_refinement_blocks(16, 8, 8, 0)
    P = _smooth_blocks(t, 16)
    m = oracle.SmrMesh(t, (16, 16, 16), riemann=riemann, recon=recon)
    U = m.from_packed(P)
    # global array from the blocks
    G = np.zeros((5, 16, 16, 16))
    g, o = m.ng, 0
    for b, r in enumerate(t):
        G[:, r[3]:r[3] + 8, r[2]:r[2] + 8, r[1]:r[1] + 8] = P[o:o + 5 * 512].reshape(5, 8, 8, 8)
        o += 5 * 512
    grid = oracle.Grid((16, 16, 16), riemann=riemann, recon=recon)
    dt = oracle.new_dt(G, grid, 0.3)
    assert dt == m.new_dt(U, 0.3)
    Gn, _ = oracle.rk_step(G, grid, dt, 2)
    Un = m.to_packed(m.rk_step(U, dt))
    o = 0
    for r in t:
        blk = Un[o:o + 5 * 512].reshape(5, 8, 8, 8)
        assert np.array_equal(blk, Gn[:, r[3]:r[3] + 8, r[2]:r[2] + 8, r[1]:r[1] + 8])
        o += 5 * 512


def _shock_radius(m, U, t):
    """Radius of the density maximum of the shell-averaged radial density profile, from
    the leaf blocks' cell centres."""
    cents = pgen.block_cell_centres(t, 32)
    g = m.ng
    pts, vals = [], []
    for b, (x, y, z) in enumerate(cents):
        rho = m.block(U, b)[0, g:-g, g:-g, g:-g]
        X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
        pts.append(np.stack([X.T.ravel(), Y.T.ravel(), Z.T.ravel()], axis=1))
        vals.append(rho.ravel())
    pts = np.concatenate(pts)
    vals = np.concatenate(vals)
    r = np.sqrt((pts ** 2).sum(axis=1))
    # radial profile in thin shells; the shock sits at the density peak
    edges = np.linspace(0.0, 0.12, 49)
    idx = np.digitize(r, edges)
    prof = np.array([vals[idx == i].mean() if np.any(idx == i) else 0 for i in range(1, 49)])
    k = int(np.argmax(prof))
    return 0.5 * (edges[k] + edges[k + 1])


def test_sedov_taylor_radius_across_levels():
    t = small_table()
    m = oracle.SmrMesh(t, (32, 32, 32))
    U = m.from_packed(pgen.sedov_blocks(t, 32))
    t_end, time = 1.2e-3, 0.0
    while time < t_end:
        dt = min(m.new_dt(U, 0.3), t_end - time)
        U = m.rk_step(U, dt)
        time += dt
    R = _shock_radius(m, U, t)
    R_st = 1.15 * (1.0 * t_end ** 2 / 1.0) ** 0.2  # Sedov-Taylor, gamma = 5/3
    dx2 = 1.0 / 128
    assert abs(R - R_st) < 1.0 * dx2, (R, R_st)


def test_overlapping_leaves_refused():
    # root blocks of 8 cells cannot leave out the central half of a 16-cell root grid:
    # the refined blocks would overlap root leaves
    t = pgen.nested_refinement_blocks(16, 8, 8, 1)
    m = oracle.SmrMesh(t, (16, 16, 16))
    with pytest.raises(ValueError):
        m.fill_ghosts(np.ones(m.size))


# ---------------------------------------------------------------------------------
# FOFC on refined meshes (Section 3: before the level flux correction)
# ---------------------------------------------------------------------------------
def _bad_cells(m, t, U):
    """Leaf cells with rho <= 0 or u_g <= 0."""
    P, o, bad = m.to_packed(U), 0, 0
    for r in t:
        n = int(r[4] * r[5] * r[6])
        u = P[o:o + 5 * n].reshape(5, n)
        o += 5 * n
        ug = u[4] - 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / u[0]
        bad += int(np.sum((u[0] <= 0) | (ug <= 0)))
    return bad


def test_smr_fofc_is_identity_without_flags():
    t = pgen.nested_refinement_blocks(16, 4, 8, 1)
    P = pgen.cold_shear_blocks(t, 16, 1.0)
    a = oracle.SmrMesh(t, (16, 16, 16))
    b = oracle.SmrMesh(t, (16, 16, 16), fofc=True)
    U = a.from_packed(P)
    dt = a.new_dt(U, 0.3)
    Ub, nflag = b.rk_step_fofc(U, dt, 2)
    assert nflag == 0 and np.array_equal(a.rk_step(U, dt), Ub)


def test_smr_fofc_single_level_equals_uniform_oracle():
    # every block on level 0: the SMR FOFC step must reproduce the uniform-grid FOFC step
    n = (24, 24, 24)
    G = pgen.turbulence(n, seed=3, kmin=1, kmax=6, mach=5.0)
    t = pgen.nested_refinement_blocks(24, 8, 8, 0)
    m = oracle.SmrMesh(t, n, fofc=True)
    U = m.from_packed(np.concatenate(
        [G[:, r[3]:r[3] + 8, r[2]:r[2] + 8, r[1]:r[1] + 8].reshape(-1) for r in t]))
    grid = oracle.Grid(n, fofc=True)
    total = 0
    for _ in range(15):
        dt = oracle.new_dt(G, grid, 0.3)
        G, _, nfl = oracle.rk_step_fofc(G, grid, dt, 2)
        U, nfl2 = m.rk_step_fofc(U, dt, 2)
        assert nfl == nfl2
        total += nfl
        P, o = m.to_packed(U), 0
        for r in t:
            blk = P[o:o + 5 * 512].reshape(5, 8, 8, 8)
            assert np.array_equal(blk, G[:, r[3]:r[3] + 8, r[2]:r[2] + 8, r[1]:r[1] + 8])
            o += 5 * 512
    assert total > 0


def test_smr_fofc_two_levels_positive_and_conservative():
    t = pgen.nested_refinement_blocks(16, 4, 8, 1)
    P = pgen.cold_shear_blocks(t, 16, 0.003)
    res = {}
    for fofc in (False, True):
        m = oracle.SmrMesh(t, (16, 16, 16), fofc=fofc)
        U = m.from_packed(P)
        tot0 = m.totals(U)
        flagged = 0
        for _ in range(6):
            U, nfl = m.rk_step_fofc(U, m.new_dt(U, 0.3), 2)
            flagged += nfl
        res[fofc] = (flagged, _bad_cells(m, t, U), np.abs(m.totals(U) - tot0))
    # the plain scheme leaves cells with negative internal energy; FOFC flags and
    # corrects them, conserving the totals to round-off
    assert res[False][0] == 0 and res[False][1] > 0
    assert res[True][0] > 0 and res[True][1] == 0
    assert res[True][2].max() < 1e-14, res[True][2]


def test_blocks_from_fine_keeps_totals():
    t = pgen.nested_refinement_blocks(16, 4, 8, 1)
    Uf = pgen.turbulence((32, 32, 32), seed=53, kmin=1, kmax=6, mach=1.0)
    m = oracle.SmrMesh(t, (16, 16, 16))
    tot = m.totals(m.from_packed(pgen.blocks_from_fine(t, Uf)))
    ref = Uf.reshape(5, -1).sum(axis=1) / 32 ** 3
    assert np.allclose(tot, ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("where", ["coarse", "fine"])
def test_smr_flagged_cell_next_to_the_level_boundary_is_local(where):
    # Section 3 (FOFC) on two levels.  A flagged coarse cell next to the refined region:
    # its level-boundary face is the mean of four fine faces, and those turn first order
    # too (the fine blocks see the flag in their ghost cells), so L changes in the cell,
    # its five same-level neighbours and the four fine cells across that face.  A flagged
    # fine cell on the level boundary: L changes in the cell, its five fine neighbours and,
    # through the flux correction of the face it shares, the coarse cell across it.
    # Nothing else changes in either case.
    t = pgen.nested_refinement_blocks(16, 4, 8, 1)
    P = _smooth_blocks(t, 16)
    m = oracle.SmrMesh(t, (16, 16, 16))
    U = m.from_packed(P)
    m.fill_ghosts(U)
    sizes = [int(r[4] * r[5] * r[6]) for r in t]
    offs = np.concatenate([[0], np.cumsum(sizes)])

    def packed_index(level, q):
        for b, r in enumerate(t):
            lo = r[1:4]
            if r[0] == level and all(lo[d] <= q[d] < lo[d] + r[4 + d] for d in range(3)):
                i, j, k = (q[d] - lo[d] for d in range(3))
                return int(offs[b] + (k * r[5] + j) * r[4] + i)
        raise AssertionError(q)

    def around(c):
        return [c] + [tuple(c[e] + (s if e == d else 0) for e in range(3))
                      for d in range(3) for s in (-1, 1)]

    flag = np.zeros(offs[-1], np.uint8)
    # the refined region covers [4, 12)^3 of level 0, [8, 24)^3 of level 1
    if where == "coarse":
        c = (3, 6, 6)
        flag[packed_index(0, c)] = 1
        expect = {packed_index(0, q) for q in around(c)
                  if not all(4 <= q[d] < 12 for d in range(3))}
        expect |= {packed_index(1, (8, 12 + dy, 12 + dz)) for dy in (0, 1) for dz in (0, 1)}
    else:
        c = (8, 12, 12)
        flag[packed_index(1, c)] = 1
        expect = {packed_index(1, q) for q in around(c) if q[0] >= 8}
        expect.add(packed_index(0, (3, 6, 6)))
    Lf = m.rhs_flagged(U, flag)
    # the flux correction keeps the composite sum of L dV at zero with the flag too
    scale = m.totals(np.abs(Lf)) + 1.0
    assert np.all(np.abs(m.totals(Lf)) <= 1e-13 * scale), m.totals(Lf)
    L0 = m.to_packed(m.rhs(U))
    L1 = m.to_packed(Lf)
    # the packed layout is [block][var][k][j][i]: reduce over the variables per block
    d = np.abs(L1 - L0)
    per_cell = np.concatenate([d[5 * offs[b]:5 * offs[b + 1]].reshape(5, -1).max(axis=0)
                               for b in range(len(t))])
    changed = {int(p) for p in np.nonzero(per_cell > 0)[0]}
    assert len(expect) == (10 if where == "coarse" else 7)
    assert changed == expect, (sorted(changed), sorted(expect))


def _slab_table(n1, n23=8, b=4):
    # root (n1, n23, n23) in b^3 blocks; level 1 (2b)^3 blocks over the slab of root
    # cells n1/4 <= x1 < 3 n1/4, across the whole x2-x3 extent: the level boundaries are
    # two x1 faces
    rows = [(0, i, j, k, b, b, b) for k in range(0, n23, b) for j in range(0, n23, b)
            for i in range(0, n1, b) if not n1 // 4 <= i < 3 * n1 // 4]
    rows += [(1, i, j, k, 2 * b, 2 * b, 2 * b) for k in range(0, 2 * n23, 2 * b)
             for j in range(0, 2 * n23, 2 * b) for i in range(n1 // 2, 3 * n1 // 2, 2 * b)]
    return np.array(rows, dtype=np.int32)


def _sound_wave_l1(n1, refined):
    # sound eigenmode along x1 (rho = 1, p = 1/gamma, c_s = 1, amplitude 1e-6), one
    # period, PLM + HLLC + RK2, CFL 0.3; L1 error (volume weighted) against the start
    n23 = 8
    if refined:
        t = _slab_table(n1, n23)
    else:
        t = np.array([(0, i, j, k, 4, 4, 4) for k in range(0, n23, 4)
                      for j in range(0, n23, 4) for i in range(0, n1, 4)], dtype=np.int32)
    root = (n1, n23, n23)

    def fn(x, y, z):
        s = 1e-6 * np.sin(2 * np.pi * (x + 0.5))
        return 1.0 + s, s, 0.0 * x, 0.0 * x, 1.0 / G53 + s
    P = pgen.field_blocks(t, root, fn)
    m = oracle.SmrMesh(t, root)
    U, time = m.from_packed(P), 0.0
    while time < 1.0:
        dt = min(m.new_dt(U, 0.3), 1.0 - time)
        U = m.rk_step(U, dt, 2)
        time += dt
    Q = m.to_packed(U)
    err, off = np.zeros(5), 0
    for r in t:
        n = int(r[4] * r[5] * r[6])
        dv = 1.0 / ((n1 << int(r[0])) * (n23 << int(r[0])) ** 2)
        err += np.abs(Q[5 * off:5 * (off + n)] - P[5 * off:5 * (off + n)]).reshape(5, -1).sum(axis=1) * dv
        off += n
    return math.sqrt(float((err ** 2).sum()))


def test_sound_wave_through_two_level_boundaries_converges():
    # Section 3.1 (PLM is second order) with the refinement of Section 2: the wave
    # crosses both level boundaries each period.  The two-level error converges like the
    # uniform one, and lies between the uniform errors at the root and at the fine
    # resolution (the slab holds half the box).
    e = {(n, r): _sound_wave_l1(n, r) for n in (16, 32) for r in (True, False)}
    e[(64, False)] = _sound_wave_l1(64, False)
    assert e[(16, True)] / e[(32, True)] > 2.5, e
    for n in (16, 32):
        assert e[(2 * n, False)] < e[(n, True)] < e[(n, False)], (n, e)
