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
