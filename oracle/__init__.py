"""FP64 CPU oracle for the AthenaK hydro stage (arXiv 2409.16053, Section 3 and 3.1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_2409_16053_gb300``), and neither imports the other.

The arithmetic lives in ``ak_oracle.c`` (plain C, FP64, ``-ffp-contract=off``); this
module compiles it with gcc into ``oracle/_build/`` and wraps it with ctypes.  Arrays
are numpy float64 of shape (5, n3, n2, n1), x1 fastest: U = (rho, M1, M2, M3, E).

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  cons_to_prim / prim_to_cons   round trip; Section 3.1 Eq. (4) closed forms
  plm_slope                     linear data, extrema, translation invariance
  ppm4_edges                    parabola reproduction, monotonicity
  ppmx_edges                    cubic / smooth-extremum reproduction, spike and step
                                cases by hand, mirror symmetry, 1D wave convergence
  wenoz_edges                   exact for quadratic cell averages, 5th order on
                                smooth data, mirror symmetry, step; RK3 wave rate
  hllc                          supersonic upwinding, stationary contact, symmetry,
                                consistency, entropy-wave/sound-wave convergence;
                                no mass or energy flux through symmetric colliding
                                streams up to Mach 50 (the Davis bound)
  pvrs_pressure / shock_factor  p_pv within O(eps^2) of the exact star pressure for
  / hllc_speeds                 jumps of size eps; u_K -+ c_K q_K(p*) equals the
                                Rankine-Hugoniot shock speed for the exact p*; the
                                speeds bracket the exact fan of weak shocks
  roe_average / hlle_speeds     u~ -+ c~ equals the shock speed across any single
                                shock (Roe's property)
  hlle / llf                    consistency, reflection symmetry, upwinding, LLF's
                                closed form on a contact, Sod errors ordered
                                HLLC < HLLE < LLF; HLLE gives the exact Godunov
                                flux of an isolated shock in any frame
  rhs / rk_step                 2nd-order sound and entropy wave convergence,
                                uniform state bitwise, periodic conservation,
                                x1/x2/x3 bitwise permutation, Sod vs exact solver
  rhs_flagged / rk_step_fofc    identity without flags, Rusanov scheme with every
                                cell flagged, one flagged cell local and
                                conservative, Mach-5 turbulence kept positive
  new_dt                        closed form on uniform states
  exact_star / exact_sample     Rankine-Hugoniot and isentrope/Riemann-invariant
                                relations across each wave; Toro's star states
  prolong / restrict            linear data exact, restriction of prolongation is
                                the identity, limited at extrema
  SmrMesh (ak_oracle_smr.c)     uniform state bitwise across levels, composite
                                conservation (and its failure without the flux
                                correction), single-level equality with rk_step /
                                rk_step_fofc, Sedov-Taylor radius, 2nd-order sound
                                wave through two level boundaries, FOFC locality
                                across a level boundary
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ak_oracle.c")
_SRC_SMR = os.path.join(_HERE, "ak_oracle_smr.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libak_oracle.so")
_lock = threading.Lock()
_lib = None

PLM = 0
PPM4 = 1
WENOZ = 2
PPMX = 3
HLLC = 0
HLLE = 1
LLF = 2


def build(force: bool = False) -> str:
    """Compile ak_oracle.c into a shared library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(_SRC_SMR))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, _SRC_SMR, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64 * 3), ("dx", ctypes.c_double * 3),
                ("gamma", ctypes.c_double), ("recon", ctypes.c_int32),
                ("riemann", ctypes.c_int32), ("fofc", ctypes.c_int32), ("pad", ctypes.c_int32)]


class _Smr(ctypes.Structure):
    _fields_ = [("nblocks", ctypes.c_int32), ("ng", ctypes.c_int32),
                ("recon", ctypes.c_int32), ("flux_correction", ctypes.c_int32),
                ("blocks", ctypes.POINTER(ctypes.c_int32)),
                ("root_nx", ctypes.c_int32 * 3), ("length", ctypes.c_double * 3),
                ("gamma", ctypes.c_double), ("riemann", ctypes.c_int32),
                ("fofc", ctypes.c_int32)]


_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            G = ctypes.POINTER(_Grid)
            lib.orc_cons_to_prim.argtypes = [_dp, _dp, _i64p]
            lib.orc_prim_to_cons.argtypes = [_dp, _dp]
            lib.orc_plm_slope.argtypes = [ctypes.c_double] * 3
            lib.orc_plm_slope.restype = ctypes.c_double
            lib.orc_ppm4_edges.argtypes = [_dp, _dp, _dp]
            lib.orc_wenoz_edges.argtypes = [_dp, _dp, _dp]
            lib.orc_ppmx_edges.argtypes = [_dp, _dp, _dp]
            lib.orc_hllc.argtypes = [_dp, _dp, ctypes.c_double, _dp]
            lib.orc_hlle.argtypes = [_dp, _dp, ctypes.c_double, _dp]
            lib.orc_llf.argtypes = [_dp, _dp, ctypes.c_double, _dp]
            lib.orc_pvrs_pressure.argtypes = [_dp, _dp, ctypes.c_double]
            lib.orc_pvrs_pressure.restype = ctypes.c_double
            lib.orc_shock_factor.argtypes = [ctypes.c_double] * 3
            lib.orc_shock_factor.restype = ctypes.c_double
            _d = ctypes.POINTER(ctypes.c_double)
            lib.orc_hllc_speeds.argtypes = [_dp, _dp, ctypes.c_double, _d, _d]
            lib.orc_hlle_speeds.argtypes = [_dp, _dp, ctypes.c_double, _d, _d]
            lib.orc_roe_average.argtypes = [_dp, _dp, ctypes.c_double, _d, _d]
            lib.orc_rhs.argtypes = [G, _dp, _dp]
            lib.orc_rhs.restype = ctypes.c_int64
            lib.orc_rhs_flagged.argtypes = [G, _dp, _dp, ctypes.POINTER(ctypes.c_uint8)]
            lib.orc_rhs_flagged.restype = ctypes.c_int64
            lib.orc_rk_step.argtypes = [G, _dp, ctypes.c_double, ctypes.c_int]
            lib.orc_rk_step.restype = ctypes.c_int64
            lib.orc_rk_step_fofc.argtypes = [G, _dp, ctypes.c_double, ctypes.c_int, _i64p]
            lib.orc_rk_step_fofc.restype = ctypes.c_int64
            lib.orc_new_dt.argtypes = [G, _dp, ctypes.c_double]
            lib.orc_new_dt.restype = ctypes.c_double
            lib.orc_exact_star.argtypes = [_dp, _dp, ctypes.c_double, _dp, _dp]
            lib.orc_exact_star.restype = ctypes.c_int
            lib.orc_exact_sample.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_double, _dp]
            lib.orc_exact_sample.restype = ctypes.c_int
            lib.orc_num_threads.restype = ctypes.c_int
            S = ctypes.POINTER(_Smr)
            lib.orc_smr_storage.argtypes = [S]
            lib.orc_smr_storage.restype = ctypes.c_int64
            lib.orc_smr_fill_ghosts.argtypes = [S, _dp]
            lib.orc_smr_fill_ghosts.restype = ctypes.c_int
            lib.orc_smr_rhs.argtypes = [S, _dp, _dp]
            lib.orc_smr_rhs.restype = ctypes.c_int64
            lib.orc_smr_rk_step.argtypes = [S, _dp, ctypes.c_double, ctypes.c_int]
            lib.orc_smr_rk_step.restype = ctypes.c_int64
            lib.orc_smr_rk_step_fofc.argtypes = [S, _dp, ctypes.c_double, ctypes.c_int, _i64p]
            lib.orc_smr_rhs_flagged.argtypes = [S, _dp, _dp, ctypes.POINTER(ctypes.c_uint8)]
            lib.orc_smr_rhs_flagged.restype = ctypes.c_int64
            lib.orc_smr_rk_step_fofc.restype = ctypes.c_int64
            lib.orc_smr_new_dt.argtypes = [S, _dp, ctypes.c_double]
            lib.orc_smr_new_dt.restype = ctypes.c_double
            lib.orc_prolong.argtypes = [ctypes.c_double, _dp, _dp, ctypes.POINTER(ctypes.c_int)]
            lib.orc_prolong.restype = ctypes.c_double
            lib.orc_restrict.argtypes = [_dp]
            lib.orc_restrict.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class Grid:
    """Periodic uniform grid: n = (n1, n2, n3) cells on a box of side lengths `length`."""

    def __init__(self, n, length=(1.0, 1.0, 1.0), gamma=5.0 / 3.0, recon=PLM, riemann=HLLC,
                 fofc=False):
        self.riemann = int(riemann)
        self.fofc = bool(fofc)
        self.n = tuple(int(v) for v in n)
        self.length = tuple(float(v) for v in length)
        self.dx = tuple(self.length[d] / self.n[d] for d in range(3))
        self.gamma = float(gamma)
        self.recon = int(recon)

    def _c(self):
        g = _Grid()
        for d in range(3):
            g.n[d] = self.n[d]
            g.dx[d] = self.dx[d]
        g.gamma = self.gamma
        g.recon = self.recon
        g.riemann = self.riemann
        g.fofc = 1 if self.fofc else 0
        return ctypes.byref(g)

    @property
    def shape(self):
        return (5, self.n[2], self.n[1], self.n[0])


def num_threads() -> int:
    return int(_load().orc_num_threads())


def cons_to_prim(u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.empty(5)
    nf = ctypes.c_int64(0)
    _load().orc_cons_to_prim(_ptr(u), _ptr(w), ctypes.byref(nf))
    return w, int(nf.value)


def prim_to_cons(w):
    w = np.ascontiguousarray(w, dtype=np.float64)
    u = np.empty(5)
    _load().orc_prim_to_cons(_ptr(w), _ptr(u))
    return u


def plm_slope(qm, q0, qp) -> float:
    return float(_load().orc_plm_slope(float(qm), float(q0), float(qp)))


def ppm4_edges(q5):
    q = np.ascontiguousarray(q5, dtype=np.float64)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _load().orc_ppm4_edges(_ptr(q), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def ppmx_edges(q5):
    """PPMX (extremum-preserving PPM) edge values of the middle cell of q5."""
    q = np.ascontiguousarray(q5, dtype=np.float64)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _load().orc_ppmx_edges(_ptr(q), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def wenoz_edges(q5):
    """WENO-Z values at x_{i-1/2} and x_{i+1/2} of the middle cell of q5."""
    q = np.ascontiguousarray(q5, dtype=np.float64)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _load().orc_wenoz_edges(_ptr(q), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def _flux(name, wl, wr, gamma):
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.empty(5)
    getattr(_load(), name)(_ptr(wl), _ptr(wr), float(gamma), _ptr(f))
    return f


def hllc(wl, wr, gamma):
    """HLLC flux; w = (rho, u_normal, v_t1, v_t2, u_g)."""
    return _flux("orc_hllc", wl, wr, gamma)


def hlle(wl, wr, gamma):
    """HLLE flux (HLL with Einfeldt's Roe-average speeds)."""
    return _flux("orc_hlle", wl, wr, gamma)


def llf(wl, wr, gamma):
    """LLF (Rusanov) flux."""
    return _flux("orc_llf", wl, wr, gamma)


def pvrs_pressure(wl, wr, gamma) -> float:
    """PVRS star-pressure estimate p_pv of the HLLC wave speeds; w as for hllc()."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    return float(_load().orc_pvrs_pressure(_ptr(wl), _ptr(wr), float(gamma)))


def shock_factor(pstar, pk, gamma) -> float:
    """Shock factor q_K of the HLLC wave speeds for star pressure pstar over p_K."""
    return float(_load().orc_shock_factor(float(pstar), float(pk), float(gamma)))


def _pair(name, wl, wr, gamma):
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    a, b = ctypes.c_double(), ctypes.c_double()
    getattr(_load(), name)(_ptr(wl), _ptr(wr), float(gamma), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def hllc_speeds(wl, wr, gamma):
    """(S_L, S_R) of the HLLC solver: PVRS speeds bounded outward by the Davis speeds."""
    return _pair("orc_hllc_speeds", wl, wr, gamma)


def hlle_speeds(wl, wr, gamma):
    """(S_L, S_R) of the HLLE solver: Einfeldt's speeds from the Roe averages."""
    return _pair("orc_hlle_speeds", wl, wr, gamma)


def roe_average(wl, wr, gamma):
    """(u~, c~): Roe-averaged normal velocity and sound speed of two states."""
    return _pair("orc_roe_average", wl, wr, gamma)


def rhs(U, grid: Grid):
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == grid.shape, (U.shape, grid.shape)
    L = np.empty_like(U)
    nf = _load().orc_rhs(grid._c(), _ptr(U), _ptr(L))
    if nf < 0:
        raise MemoryError("oracle rhs allocation failed")
    return L, int(nf)


def rhs_flagged(U, grid: Grid, flag):
    """L(U) with first-order LLF fluxes on the faces of the cells where flag (shape
    (n3, n2, n1)) is nonzero: the FOFC right-hand side of one stage."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    f = np.ascontiguousarray(flag, dtype=np.uint8)
    L = np.zeros_like(U)
    nf = _load().orc_rhs_flagged(grid._c(), _ptr(U), _ptr(L),
                                f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return L, int(nf)


def rk_step(U, grid: Grid, dt: float, rk: int = 2):
    """One full SSP-RK step; returns (U_new, floors)."""
    Un = np.array(U, dtype=np.float64, order="C", copy=True)
    assert Un.shape == grid.shape
    nf = _load().orc_rk_step(grid._c(), _ptr(Un), float(dt), int(rk))
    if nf < 0:
        raise MemoryError("oracle rk_step allocation failed")
    return Un, int(nf)


def rk_step_fofc(U, grid: Grid, dt: float, rk: int = 2):
    """One full SSP-RK step; returns (U_new, floors, cells flagged by FOFC over its
    stages)."""
    Un = np.array(U, dtype=np.float64, order="C", copy=True)
    assert Un.shape == grid.shape
    nfl = ctypes.c_int64(0)
    nf = _load().orc_rk_step_fofc(grid._c(), _ptr(Un), float(dt), int(rk), ctypes.byref(nfl))
    if nf < 0:
        raise MemoryError("oracle rk_step allocation failed")
    return Un, int(nf), int(nfl.value)


def new_dt(U, grid: Grid, cfl: float) -> float:
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == grid.shape
    return float(_load().orc_new_dt(grid._c(), _ptr(U), float(cfl)))


def run(U, grid: Grid, cfl: float, t_end: float | None = None, nsteps: int | None = None,
        rk: int = 2):
    """Advance with dt from the CFL rule before every step; the last step is clipped to
    land on t_end exactly.  Returns (U, t, steps, floors)."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    t, steps, floors = 0.0, 0, 0
    while True:
        if nsteps is not None and steps >= nsteps:
            break
        if t_end is not None and t >= t_end:
            break
        dt = new_dt(U, grid, cfl)
        if t_end is not None and t + dt > t_end:
            dt = t_end - t
        U, nf = rk_step(U, grid, dt, rk)
        floors += nf
        t += dt
        steps += 1
    return U, t, steps, floors


def exact_star(wl, wr, gamma):
    """Star-region (p*, u*) of the exact Riemann problem; w = (rho, u, p)."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    ps, us = ctypes.c_double(), ctypes.c_double()
    rc = _load().orc_exact_star(_ptr(wl), _ptr(wr), float(gamma), ctypes.byref(ps),
                                ctypes.byref(us))
    if rc != 0:
        raise ValueError("vacuum generated")
    return ps.value, us.value


def exact_sample(wl, wr, gamma, xi):
    """Exact solution (rho, u, p) at each xi = x/t; returns array (3, len(xi))."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.empty((3, xi.size))
    o = np.empty(3)
    lib = _load()
    for m, x in enumerate(xi):
        if lib.orc_exact_sample(_ptr(wl), _ptr(wr), float(gamma), float(x), _ptr(o)) != 0:
            raise ValueError("vacuum generated")
        out[:, m] = o
    return out


# ---- static refinement (ak_oracle_smr.c) -----------------------------------------------
def prolong(uc, um, up, hi):
    """Fine value from coarse centre uc, coarse neighbours um[d]/up[d], upper half hi[d]."""
    um = np.ascontiguousarray(um, dtype=np.float64)
    up = np.ascontiguousarray(up, dtype=np.float64)
    h = (ctypes.c_int * 3)(*[int(v) for v in hi])
    return float(_load().orc_prolong(float(uc), _ptr(um), _ptr(up), h))


def restrict(f8):
    f = np.ascontiguousarray(f8, dtype=np.float64)
    return float(_load().orc_restrict(_ptr(f)))


class SmrMesh:
    """Leaf MeshBlocks on several levels (rows: level, lx1, lx2, lx3, nx1, nx2, nx3) of a
    periodic box; storage = padded arrays block after block (see ak_oracle_smr.c)."""

    def __init__(self, table, root_nx, length=(1.0, 1.0, 1.0), gamma=5.0 / 3.0,
                 recon=PLM, flux_correction=True, riemann=HLLC, fofc=False):
        self.table = np.ascontiguousarray(np.asarray(table, dtype=np.int32))
        self.root_nx = tuple(int(v) for v in root_nx)
        self.length = tuple(float(v) for v in length)
        self.gamma = float(gamma)
        self.ng = 2 if recon == PLM else 3
        self.recon = int(recon)
        c = _Smr()
        c.nblocks = self.table.shape[0]
        c.ng = self.ng
        c.recon = self.recon
        c.flux_correction = 1 if flux_correction else 0
        c.blocks = self.table.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        for d in range(3):
            c.root_nx[d] = self.root_nx[d]
            c.length[d] = self.length[d]
        c.gamma = self.gamma
        c.riemann = int(riemann)
        c.fofc = 1 if fofc else 0
        self._c = c
        g = self.ng
        self.shapes = [(5, r[6] + 2 * g, r[5] + 2 * g, r[4] + 2 * g) for r in self.table]
        sizes = [int(np.prod(s)) for s in self.shapes]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.size = int(self.offsets[-1])

    def _ref(self):
        return ctypes.byref(self._c)

    def block(self, U, b):
        """Padded view (5, p3, p2, p1) of block b inside the storage array U."""
        return U[self.offsets[b]:self.offsets[b + 1]].reshape(self.shapes[b])

    def from_packed(self, P):
        """Storage array (ghosts zero) from interior data packed block after block as
        [block][var][k][j][i]."""
        U = np.zeros(self.size)
        g, o = self.ng, 0
        for b, r in enumerate(self.table):
            n = 5 * int(r[4]) * int(r[5]) * int(r[6])
            self.block(U, b)[:, g:-g, g:-g, g:-g] = P[o:o + n].reshape(5, r[6], r[5], r[4])
            o += n
        return U

    def to_packed(self, U):
        g = self.ng
        return np.concatenate([self.block(U, b)[:, g:-g, g:-g, g:-g].reshape(-1)
                               for b in range(len(self.table))])

    def fill_ghosts(self, U):
        if _load().orc_smr_fill_ghosts(self._ref(), _ptr(U)) != 0:
            raise ValueError("inconsistent SMR mesh")

    def rhs(self, U):
        L = np.zeros_like(U)
        if _load().orc_smr_rhs(self._ref(), _ptr(U), _ptr(L)) != 0:
            raise ValueError("inconsistent SMR mesh")
        return L

    def rk_step(self, U, dt, rk=2):
        Un = np.array(U, dtype=np.float64, copy=True)
        if _load().orc_smr_rk_step(self._ref(), _ptr(Un), float(dt), int(rk)) != 0:
            raise ValueError("inconsistent SMR mesh")
        return Un

    def rhs_flagged(self, U, flag_packed):
        """L(U) (ghosts of U filled) with FOFC flags given per interior cell, packed block
        after block as [block][k][j][i]."""
        L = np.zeros_like(U)
        f = np.ascontiguousarray(flag_packed, dtype=np.uint8)
        if _load().orc_smr_rhs_flagged(self._ref(), _ptr(U), _ptr(L),
                                       f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))) != 0:
            raise ValueError("inconsistent SMR mesh")
        return L

    def rk_step_fofc(self, U, dt, rk=2):
        """One RK step with FOFC (the mesh must be built with fofc=True); returns the new
        state and the number of flagged cells summed over the stages."""
        Un = np.array(U, dtype=np.float64, copy=True)
        n = ctypes.c_int64(0)
        if _load().orc_smr_rk_step_fofc(self._ref(), _ptr(Un), float(dt), int(rk),
                                        ctypes.byref(n)) != 0:
            raise ValueError("inconsistent SMR mesh")
        return Un, int(n.value)

    def new_dt(self, U, cfl):
        return float(_load().orc_smr_new_dt(self._ref(), _ptr(U), float(cfl)))

    def totals(self, U):
        """Sum of U dV over every leaf's interior, per conserved variable."""
        g = self.ng
        tot = np.zeros(5)
        for b, r in enumerate(self.table):
            dv = np.prod([self.length[d] / (self.root_nx[d] << int(r[0])) for d in range(3)])
            tot += self.block(U, b)[:, g:-g, g:-g, g:-g].sum(axis=(1, 2, 3)) * dv
        return tot
