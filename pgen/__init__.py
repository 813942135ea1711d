"""Seeded synthetic initial conditions ("problem generators") for the hydro stage.

This module is the one piece shared by the oracle side and the CUDA side: it only
builds input arrays and holds none of the finite-volume method's arithmetic.  Every
generator returns conserved variables U = (rho, M1, M2, M3, E) as a float64 numpy
array of shape (5, n3, n2, n1) (x1 fastest) with point values at cell centres, on a
box of unit side (or [-1/2, 1/2]^3 where stated).

Recipes (workloads of the paper's Section 3.1 tests and Section 5 benchmarks):
  linear_wave   3D-embedded 1D sound or entropy eigenmode along x1 (Section 3.1 and
                the Section 5.1 linear-wave benchmark), amplitude 1e-6, one
                wavelength per box.
  turbulence    Gaussian random-phase velocity field with shell spectrum E(k) ~ k^-2
                (per-mode variance ~ |k|^-4) on integer modes kmin <= |k| <= kmax,
                optional solenoidal projection, mean removed, scaled to a given rms
                Mach number; uniform rho and p.
  shock_tube    Sod-type Riemann problem along x1, x2 or x3 (two interfaces on the
                periodic box so that the tube is periodic).
  sedov         thermal energy deposited uniformly in r < r0 of a cold uniform medium.
  uniform       a uniform state, optionally moving.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20240924


def _cons(rho, v1, v2, v3, p, gamma):
    """Conserved variables of the initial state (Section 3.1 Eq. (4) definitions)."""
    e = p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2 + v3 * v3)
    return np.ascontiguousarray(np.stack([rho, rho * v1, rho * v2, rho * v3, e]),
                                dtype=np.float64)


def cell_centres(n, lo=0.0, length=1.0):
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def uniform(n, rho=1.0, p=0.6, v=(0.0, 0.0, 0.0), gamma=5.0 / 3.0):
    n1, n2, n3 = n
    shp = (n3, n2, n1)
    ones = np.ones(shp)
    return _cons(rho * ones, v[0] * ones, v[1] * ones, v[2] * ones, p * ones, gamma)


def linear_wave(n, wave="sound", amp=1.0e-6, gamma=5.0 / 3.0, vflow=1.0):
    """Exact eigenmode on a uniform background, along x1, one wavelength per box.

    sound:   rho=1, p=1/gamma (c_s=1), v=0; right eigenvector of the eigenvalue u+c in
             conserved variables, R = (1, c, 0, 0, H) with H = c^2/(gamma-1).
             Period T = 1.
    entropy: rho=1, p=1/gamma, v=(vflow,0,0); R = (1, u, 0, 0, u^2/2).  T = 1/vflow.
    Returns (U, period).
    """
    n1, n2, n3 = n
    x = cell_centres(n1)
    s = np.sin(2.0 * np.pi * x)[None, None, :] * np.ones((n3, n2, 1))
    rho0, p0 = 1.0, 1.0 / gamma
    if wave == "sound":
        c = np.sqrt(gamma * p0 / rho0)
        u0 = 0.0
        r = (1.0, u0 + c, 0.0, 0.0, c * c / (gamma - 1.0) + 0.5 * u0 * u0 + u0 * c)
        period = 1.0 / c
    elif wave == "entropy":
        u0 = float(vflow)
        r = (1.0, u0, 0.0, 0.0, 0.5 * u0 * u0)
        period = 1.0 / abs(u0)
    else:
        raise ValueError(wave)
    base = uniform(n, rho=rho0, p=p0, v=(u0, 0.0, 0.0), gamma=gamma)
    for m in range(5):
        base[m] += amp * r[m] * s
    return np.ascontiguousarray(base), period


def turbulence(n, seed, kmin=2, kmax=8, mach=0.5, solenoidal=False, rho=1.0, p=1.0,
               gamma=5.0 / 3.0):
    """Random-phase Gaussian velocity field, E(k) ~ k^-2, rms Mach `mach`."""
    n1, n2, n3 = n
    rng = np.random.default_rng(SEED_BASE + int(seed))
    k3 = np.fft.fftfreq(n3, d=1.0 / n3)[:, None, None]
    k2 = np.fft.fftfreq(n2, d=1.0 / n2)[None, :, None]
    k1 = np.fft.rfftfreq(n1, d=1.0 / n1)[None, None, :]
    kk = np.sqrt(k1 * k1 + k2 * k2 + k3 * k3)
    band = (kk >= kmin) & (kk <= kmax)
    amp = np.zeros_like(kk)
    amp[band] = kk[band] ** -2.0  # per-mode rms ~ k^-2  <=>  shell E(k) ~ k^-2
    shp = amp.shape
    vh = []
    for _ in range(3):
        re = rng.standard_normal(shp)
        im = rng.standard_normal(shp)
        vh.append(amp * (re + 1j * im))
    if solenoidal:
        kd = kk.copy()
        kd[kd == 0] = 1.0
        kdotv = (k1 * vh[0] + k2 * vh[1] + k3 * vh[2]) / (kd * kd)
        vh = [vh[0] - k1 * kdotv, vh[1] - k2 * kdotv, vh[2] - k3 * kdotv]
    v = [np.fft.irfftn(c, s=(n3, n2, n1), axes=(0, 1, 2)) for c in vh]
    v = [c - c.mean() for c in v]
    vrms = np.sqrt(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
    cs = np.sqrt(gamma * p / rho)
    scale = mach * cs / vrms
    v = [c * scale for c in v]
    ones = np.ones((n3, n2, n1))
    return _cons(rho * ones, v[0], v[1], v[2], p * ones, gamma)


def turbulence_device(n, seed, kmin=2, kmax=8, mach=0.5, solenoidal=False, rho=1.0, p=1.0,
                      gamma=5.0 / 3.0, device="cuda"):
    """The recipe of `turbulence` generated with torch on a GPU, for grids whose FFT is too
    large for the host (512^3, 768^3): random-phase Gaussian modes with per-mode rms
    k^-2 on kmin <= |k| <= kmax, optional solenoidal projection, mean removed, scaled to
    rms Mach `mach`.  Its random stream (torch's, seeded with SEED_BASE + seed) differs
    from the numpy one.  Returns a float64 torch tensor (5, n3, n2, n1) on `device`."""
    import torch
    n1, n2, n3 = n
    f64 = torch.float64
    gen = torch.Generator(device=device)
    gen.manual_seed(SEED_BASE + int(seed))
    k3 = torch.fft.fftfreq(n3, d=1.0 / n3, dtype=f64, device=device).view(-1, 1, 1)
    k2 = torch.fft.fftfreq(n2, d=1.0 / n2, dtype=f64, device=device).view(1, -1, 1)
    k1 = torch.fft.rfftfreq(n1, d=1.0 / n1, dtype=f64, device=device).view(1, 1, -1)
    kk = torch.sqrt(k1 * k1 + k2 * k2 + k3 * k3)
    band = (kk >= kmin) & (kk <= kmax)
    amp = torch.where(band, kk.clamp(min=1.0) ** -2.0, torch.zeros_like(kk))
    shp = amp.shape
    vh = []
    for _ in range(3):
        re = torch.randn(shp, generator=gen, dtype=f64, device=device)
        im = torch.randn(shp, generator=gen, dtype=f64, device=device)
        vh.append(amp * torch.complex(re, im))
        del re, im
    if solenoidal:
        kd = torch.where(kk == 0, torch.ones_like(kk), kk)
        kdotv = (k1 * vh[0] + k2 * vh[1] + k3 * vh[2]) / (kd * kd)
        vh = [vh[0] - k1 * kdotv, vh[1] - k2 * kdotv, vh[2] - k3 * kdotv]
        del kdotv
    U = torch.empty((5, n3, n2, n1), dtype=f64, device=device)
    for c in range(3):
        v = torch.fft.irfftn(vh[c], s=(n3, n2, n1), dim=(0, 1, 2))
        vh[c] = None
        U[1 + c] = v - v.mean()
        del v
    vrms = torch.sqrt((U[1] ** 2 + U[2] ** 2 + U[3] ** 2).mean())
    cs = (gamma * p / rho) ** 0.5
    scale = mach * cs / vrms
    U[0].fill_(rho)
    for c in range(3):
        U[1 + c] *= scale
    # conserved: M = rho v, E = p / (gamma - 1) + rho |v|^2 / 2
    U[4] = 0.5 * rho * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) + p / (gamma - 1.0)
    for c in range(3):
        U[1 + c] *= rho
    return U


def shock_tube(n, direction=0, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1),
               gamma=1.4, x0=0.25, x1=0.75):
    """Riemann problem along `direction`: state `left` (rho, u, p) for x0 <= x < x1,
    `right` elsewhere (periodic box, so there are two interfaces).  The normal
    velocity is along `direction`."""
    nd = n[direction]
    x = cell_centres(nd)
    inside = (x >= x0) & (x < x1)
    shp = (n[2], n[1], n[0])
    axis = 2 - direction
    line = inside.astype(np.float64)
    shape = [1, 1, 1]
    shape[axis] = nd
    line = line.reshape(shape)
    m = np.broadcast_to(line, shp)
    rho = right[0] + (left[0] - right[0]) * m
    un = right[1] + (left[1] - right[1]) * m
    p = right[2] + (left[2] - right[2]) * m
    zero = np.zeros(shp)
    v = [zero, zero, zero]
    v[direction] = un
    return _cons(rho, v[0], v[1], v[2], p, gamma)


def sedov(n, e_blast=1.0, r0=0.02, rho=1.0, p_amb=1.0e-5, gamma=5.0 / 3.0, lo=-0.5,
          length=1.0):
    """Thermal energy e_blast spread uniformly (by volume) over cells with centres at
    r < r0 in a uniform medium on [lo, lo+length]^3.  Returns (U, ncells_in_blast)."""
    n1, n2, n3 = n
    x = cell_centres(n1, lo, length)[None, None, :]
    y = cell_centres(n2, lo, length)[None, :, None]
    z = cell_centres(n3, lo, length)[:, None, None]
    r = np.sqrt(x * x + y * y + z * z)
    inside = r < r0
    dv = (length / n1) * (length / n2) * (length / n3)
    ncell = int(inside.sum())
    if ncell == 0:
        raise ValueError("blast radius smaller than a cell")
    shp = (n3, n2, n1)
    p = np.full(shp, p_amb)
    p[inside] += (gamma - 1.0) * e_blast / (ncell * dv)
    zero = np.zeros(shp)
    return _cons(np.full(shp, rho), zero, zero, zero, p, gamma), ncell


def nested_refinement_blocks(root_nx=128, root_block=32, fine_block=16, levels=2):
    """Leaf MeshBlocks of a static nested refinement on the periodic box [-1/2, 1/2]^3:
    a root grid of root_nx^3 cells in root_block^3 blocks, and `levels` refined levels,
    level l covering the central cube of side 2^-l in fine_block^3 blocks (cell size
    halves per level).  Blocks covered by a finer level are not leaves and are omitted.

    Returns an int32 array of rows (level, lx1, lx2, lx3, nx1, nx2, nx3), where
    (lx1, lx2, lx3) is the block's first cell in the cell index space of its level
    (root_nx * 2^level cells per direction)."""
    rows = []

    def region(level):  # index range [lo, hi) of the refined cube at `level`
        n = root_nx << level
        side = n >> level  # the cube's side, 2^-level of the box, in level cells
        return (n - side) // 2, (n + side) // 2

    for level in range(levels + 1):
        bs = root_block if level == 0 else fine_block
        n = root_nx << level
        lo, hi = (0, n) if level == 0 else region(level)
        nxt = region(level + 1) if level < levels else None
        for bz in range(lo, hi, bs):
            for by in range(lo, hi, bs):
                for bx in range(lo, hi, bs):
                    if nxt is not None:
                        # covered if the block lies inside the next level's cube
                        c_lo, c_hi = nxt[0] // 2, nxt[1] // 2
                        if all(c_lo <= b and b + bs <= c_hi for b in (bx, by, bz)):
                            continue
                    rows.append([level, bx, by, bz, bs, bs, bs])
    return np.ascontiguousarray(np.array(rows, dtype=np.int32))


def block_cell_centres(table, root_nx, lo=-0.5, length=1.0):
    """Per leaf block, the cell-centre coordinates (x1, x2, x3) as 1-D arrays.  root_nx:
    root cells per direction, one int (a cube) or three."""
    rn = (int(root_nx),) * 3 if np.isscalar(root_nx) else tuple(int(n) for n in root_nx)
    out = []
    for r in np.asarray(table):
        lev = int(r[0])
        out.append(tuple(lo + (r[1 + d] + np.arange(r[4 + d]) + 0.5) * (length / (rn[d] << lev))
                         for d in range(3)))
    return out


def sedov_blocks(table, root_nx, e_blast=1.0, r0=0.02, rho=1.0, p_amb=1.0e-5,
                 gamma=5.0 / 3.0, lo=-0.5, length=1.0):
    """Sedov deposit on leaf blocks of several levels: thermal energy e_blast spread
    uniformly by volume over the cells whose centres lie at r < r0.  Returns the
    interior data packed block after block as [block][var][k][j][i]."""
    tab = np.asarray(table)
    cents = block_cell_centres(tab, root_nx, lo, length)
    vol_in = 0.0
    masks = []
    for r, (x, y, z) in zip(tab, cents):
        rr = np.sqrt(x[None, None, :] ** 2 + y[None, :, None] ** 2 + z[:, None, None] ** 2)
        m = rr < r0
        masks.append(m)
        vol_in += m.sum() * (length / (root_nx << int(r[0]))) ** 3
    if vol_in == 0.0:
        raise ValueError("blast radius smaller than a cell")
    parts = []
    for r, m in zip(tab, masks):
        p = np.where(m, p_amb + (gamma - 1.0) * e_blast / vol_in, p_amb)
        z = np.zeros_like(p)
        parts.append(_cons(np.full_like(p, rho), z, z, z, p, gamma).reshape(-1))
    return np.concatenate(parts)


def field_blocks(table, root_nx, fn, gamma=5.0 / 3.0, lo=-0.5, length=1.0):
    """Conserved variables from a primitive-state function fn(x, y, z) -> (rho, v1, v2,
    v3, p) evaluated at the cell centres of every leaf; packed block after block.
    root_nx: root cells per direction, one int (a cube) or three."""
    parts = []
    for r, (x, y, z) in zip(np.asarray(table), block_cell_centres(table, root_nx, lo, length)):
        shape = (len(z), len(y), len(x))
        Xg = np.broadcast_to(x[None, None, :], shape)
        Yg = np.broadcast_to(y[None, :, None], shape)
        Zg = np.broadcast_to(z[:, None, None], shape)
        rho, v1, v2, v3, p = fn(Xg, Yg, Zg)
        parts.append(_cons(rho * np.ones(shape), v1 * np.ones(shape), v2 * np.ones(shape),
                           v3 * np.ones(shape), p * np.ones(shape), gamma).reshape(-1))
    return np.concatenate(parts)


def cold_shear_blocks(table, root_nx, p, gamma=5.0 / 3.0):
    """A cold (pressure p) diverging and shearing flow of unit-order speed on leaf blocks
    of several levels, with its divergence centred on a level boundary of the nested
    refinement; at p ~ 1e-3 the plain scheme drives cells to negative internal energy.
    Packed block after block as [block][var][k][j][i]."""
    def fn(x, y, z):
        tp = 2 * np.pi
        return (1.0 + 0.5 * np.cos(tp * (x + y)),
                np.sin(tp * (x - 0.25)) * (1 + 0.3 * np.cos(tp * y)),
                0.5 * np.sin(tp * (y + 0.1)) * np.cos(tp * z), 0.3 * np.cos(tp * x), p)
    return field_blocks(table, root_nx, fn, gamma)


def blocks_from_fine(table, Uf):
    """Leaf-block data of a nested mesh from a uniform field Uf (5, n3, n2, n1) given at
    the resolution of the finest level: each leaf of level l takes the means of the
    2^(L-l)-cubes of fine cells it covers (L the finest level), so the totals are those
    of Uf.  Packed block after block as [block][var][k][j][i]."""
    tab = np.asarray(table)
    top = int(tab[:, 0].max())
    parts = []
    for r in tab:
        f = 1 << (top - int(r[0]))
        lx, ly, lz, nx, ny, nz = (int(v) for v in r[1:7])
        sub = Uf[:, f * lz:f * (lz + nz), f * ly:f * (ly + ny), f * lx:f * (lx + nx)]
        parts.append(sub.reshape(5, nz, f, ny, f, nx, f).mean(axis=(2, 4, 6)).reshape(-1))
    return np.concatenate(parts)
