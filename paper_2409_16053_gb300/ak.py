"""Thin ctypes binding of libak (include/ak.h), with the C-ABI's names.

Argument marshalling only: every step of the hydro stage runs in the CUDA kernels of
libak.so.  There is no CPU fallback: if the library cannot be loaded, importing this
module raises.  PyTorch is used only to own device memory (the registers) and the
CUDA stream.

Low level (same names and arguments as the C functions):
    ak_mesh_create, ak_mesh_destroy, ak_mesh_layout, ak_mesh_bind, ak_fill_ghosts,
    ak_stage, ak_new_dt, ak_step, ak_upload, ak_download, ak_status_counters,
    ak_mesh_autotune, ak_mesh_schedule, ak_mesh_fuse, ak_selftest_barrier, ak_cfl_dt_noalloc,
    ak_probe_fp64_rate, ak_last_error
High level: ``Mesh`` builds a uniform mesh of equal MeshBlocks, allocates and binds
its registers as torch tensors, and converts between a global (5, n3, n2, n1) array
and the library's block layout.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

AK_OK, AK_EINVAL, AK_ENOMEM, AK_ECUDA, AK_ENEGATIVE, AK_ETIMEOUT, AK_ESTATE, AK_EOVERFLOW = \
    0, -1, -2, -3, -4, -5, -6, -7
AK_PLM, AK_PPM4, AK_WENOZ, AK_PPMX = 0, 1, 2, 3
AK_FP64, AK_MIXED = 0, 1
AK_HLLC, AK_HLLE, AK_LLF = 0, 1, 2
AK_BLOCK_INTS = 7

_STATUS_NAMES = {0: "AK_OK", -1: "AK_EINVAL", -2: "AK_ENOMEM", -3: "AK_ECUDA",
                 -4: "AK_ENEGATIVE", -5: "AK_ETIMEOUT", -6: "AK_ESTATE", -7: "AK_EOVERFLOW"}


class AkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ak_mesh_desc(ctypes.Structure):
    _fields_ = [
        ("nblocks", ctypes.c_int32), ("nghost", ctypes.c_int32),
        ("blocks", ctypes.POINTER(ctypes.c_int32)),
        ("xmin", ctypes.c_double * 3), ("xmax", ctypes.c_double * 3),
        ("root_nx", ctypes.c_int32 * 3),
        ("recon", ctypes.c_int32), ("rk", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("riemann", ctypes.c_int32), ("fofc", ctypes.c_int32),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("ref_rho", ctypes.c_double), ("ref_p", ctypes.c_double),
    ]


def _load_lib():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libak.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    i32 = ctypes.c_int32
    lib.ak_mesh_create.argtypes = [ctypes.POINTER(ak_mesh_desc), vp, ctypes.POINTER(vp)]
    lib.ak_mesh_destroy.argtypes = [vp]
    lib.ak_mesh_destroy.restype = None
    lib.ak_mesh_layout.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_size_t),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.ak_mesh_bind.argtypes = [vp, i32, vp]
    lib.ak_fill_ghosts.argtypes = [vp, i32]
    lib.ak_stage.argtypes = [vp, i32, ctypes.c_double]
    lib.ak_new_dt.argtypes = [vp, i32, dp]
    lib.ak_step.argtypes = [vp, ctypes.c_double, dp]
    lib.ak_upload.argtypes = [vp, i32, vp]
    lib.ak_download.argtypes = [vp, i32, vp]
    lib.ak_status_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.ak_mesh_autotune.argtypes = [vp, ctypes.POINTER(i32)]
    lib.ak_mesh_autotune.restype = ctypes.c_int
    lib.ak_mesh_schedule.argtypes = [vp, i32, i32, i32]
    lib.ak_mesh_schedule.restype = ctypes.c_int
    lib.ak_mesh_fuse.argtypes = [vp, i32]
    lib.ak_mesh_fuse.restype = ctypes.c_int
    lib.ak_selftest_barrier.argtypes = [vp, i32]
    lib.ak_selftest_barrier.restype = ctypes.c_int
    lib.ak_cfl_dt_noalloc.argtypes = [vp, i32, ctypes.POINTER(i32), i32, dp, ctypes.c_double,
                                      ctypes.c_double, vp, dp]
    lib.ak_cfl_dt_noalloc.restype = ctypes.c_int
    lib.ak_probe_fp64_rate.argtypes = [vp, dp]
    lib.ak_probe_fp64_rate.restype = ctypes.c_int
    lib.ak_last_error.restype = ctypes.c_char_p
    for name in ("ak_mesh_create", "ak_mesh_layout", "ak_mesh_bind", "ak_fill_ghosts",
                 "ak_stage", "ak_new_dt", "ak_step", "ak_upload", "ak_download",
                 "ak_status_counters"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


_lib = _load_lib()
EXPORTED = ("ak_mesh_create", "ak_mesh_destroy", "ak_mesh_layout", "ak_mesh_bind",
            "ak_fill_ghosts", "ak_stage", "ak_new_dt", "ak_step", "ak_upload",
            "ak_download", "ak_status_counters", "ak_mesh_autotune", "ak_mesh_schedule", "ak_mesh_fuse",
            "ak_selftest_barrier",
            "ak_cfl_dt_noalloc", "ak_probe_fp64_rate", "ak_last_error")


def ak_last_error() -> str:
    return _lib.ak_last_error().decode()


def _check(st, allow=()):
    if st != AK_OK and st not in allow:
        raise AkError(st, ak_last_error())
    return st


# ---- C-ABI, one wrapper per entry point ---------------------------------------------
def ak_mesh_create(desc: ak_mesh_desc, cuda_stream: int):
    out = ctypes.c_void_p()
    _check(_lib.ak_mesh_create(ctypes.byref(desc), ctypes.c_void_p(cuda_stream),
                               ctypes.byref(out)))
    return out


def ak_mesh_destroy(mesh) -> None:
    _lib.ak_mesh_destroy(mesh)


def ak_mesh_layout(mesh, nblocks: int):
    """Returns (nregisters, register_bytes, block_offsets, strides(var, k, j, i))."""
    nreg, nbytes = ctypes.c_int32(), ctypes.c_size_t()
    offs = (ctypes.c_int64 * nblocks)()
    strides = (ctypes.c_int64 * 4)()
    _check(_lib.ak_mesh_layout(mesh, ctypes.byref(nreg), ctypes.byref(nbytes), offs, strides))
    return (int(nreg.value), int(nbytes.value), np.array(offs[:], dtype=np.int64),
            tuple(int(v) for v in strides))


def ak_mesh_bind(mesh, reg: int, dev_ptr: int) -> None:
    _check(_lib.ak_mesh_bind(mesh, reg, ctypes.c_void_p(dev_ptr)))


def ak_fill_ghosts(mesh, reg: int) -> None:
    _check(_lib.ak_fill_ghosts(mesh, reg))


def ak_stage(mesh, stage: int, dt: float) -> None:
    _check(_lib.ak_stage(mesh, stage, float(dt)))


def ak_new_dt(mesh, reg: int):
    """Returns (dt, status); status AK_ENEGATIVE (floors were hit) is not raised."""
    dt = ctypes.c_double()
    st = _check(_lib.ak_new_dt(mesh, reg, ctypes.byref(dt)), allow=(AK_ENEGATIVE,))
    return dt.value, st


def ak_step(mesh, dt: float, want_dt_next: bool = True):
    """Returns (dt_next or None, status); AK_ENEGATIVE is returned, not raised (any other
    error, e.g. AK_ETIMEOUT or AK_EOVERFLOW, raises AkError)."""
    if want_dt_next:
        dn = ctypes.c_double()
        st = _check(_lib.ak_step(mesh, float(dt), ctypes.byref(dn)), allow=(AK_ENEGATIVE,))
        return dn.value, st
    st = _check(_lib.ak_step(mesh, float(dt), None), allow=(AK_ENEGATIVE,))
    return None, st


def ak_upload(mesh, reg: int, host_ptr: int) -> None:
    _check(_lib.ak_upload(mesh, reg, ctypes.c_void_p(host_ptr)))


def ak_download(mesh, reg: int, host_ptr: int) -> None:
    _check(_lib.ak_download(mesh, reg, ctypes.c_void_p(host_ptr)))


def ak_status_counters(mesh):
    out = (ctypes.c_int64 * 4)()
    _check(_lib.ak_status_counters(mesh, out))
    return list(out)


def ak_mesh_autotune(mesh):
    """Times stage-kernel schedules on this mesh and keeps the fastest (and, on meshes
    with a ghost fill, the separate or the fused stage launch).  Returns (tile, segments,
    order, microseconds per stage, fused)."""
    out = (ctypes.c_int32 * 5)()
    _check(_lib.ak_mesh_autotune(mesh, out))
    return tuple(int(v) for v in out)


def ak_mesh_schedule(mesh, tile: int, nseg: int, order: int):
    """Sets the stage kernel's schedule (tile variant, x3 segments, CTA order)."""
    _check(_lib.ak_mesh_schedule(mesh, tile, nseg, order))


def ak_mesh_fuse(mesh, fused: bool):
    """Fill, flux correction and stage in one persistent cooperative launch per stage."""
    _check(_lib.ak_mesh_fuse(mesh, 1 if fused else 0))


def ak_selftest_barrier(mesh, absent: bool):
    """Bounded-wait self-test: raises AkError(AK_ETIMEOUT) when the barrier's wait ran
    out (absent=True makes it run out)."""
    _check(_lib.ak_selftest_barrier(mesh, 1 if absent else 0))


def ak_cfl_dt_noalloc(reg_ptr: int, nblocks: int, nx, nghost: int, dx, gamma: float,
                      cfl: float, cuda_stream: int) -> float:
    """CFL dt of a register without any device allocation (static device scratch)."""
    nx_c = (ctypes.c_int32 * 3)(*[int(v) for v in nx])
    dx_c = (ctypes.c_double * 3)(*[float(v) for v in dx])
    out = ctypes.c_double()
    _check(_lib.ak_cfl_dt_noalloc(ctypes.c_void_p(reg_ptr), int(nblocks), nx_c, int(nghost),
                                  dx_c, float(gamma), float(cfl),
                                  ctypes.c_void_p(cuda_stream), ctypes.byref(out)))
    return out.value


def ak_probe_fp64_rate(cuda_stream: int = 0) -> float:
    """Measured FP64 fused multiply-adds per second of the current device."""
    out = ctypes.c_double()
    _check(_lib.ak_probe_fp64_rate(ctypes.c_void_p(cuda_stream), ctypes.byref(out)))
    return out.value


# ---- convenience layer ---------------------------------------------------------------
def uniform_block_table(root_nx, block_nx):
    """Block table of a uniform level-0 mesh, blocks in x1-fastest order."""
    nb = [root_nx[d] // block_nx[d] for d in range(3)]
    rows = []
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                rows.append([0, bx * block_nx[0], by * block_nx[1], bz * block_nx[2],
                             block_nx[0], block_nx[1], block_nx[2]])
    return np.ascontiguousarray(np.array(rows, dtype=np.int32))


class Mesh:
    """A periodic mesh of MeshBlocks with torch-owned registers: a uniform mesh of equal
    blocks (block_nx), or any leaf table (rows level, lx1, lx2, lx3, nx1, nx2, nx3) of a
    statically refined mesh (table)."""

    def __init__(self, root_nx, block_nx=None, *, table=None, recon=AK_PLM, rk=2,
                 precision=AK_FP64, riemann=0, fofc=False, gamma=5.0 / 3.0, cfl=0.3,
                 xmin=(0.0, 0.0, 0.0),
                 xmax=(1.0, 1.0, 1.0), ref_rho=1.0, ref_p=1.0, device="cuda", stream=None):
        import torch
        self.torch = torch
        self.root_nx = tuple(int(v) for v in root_nx)
        self.ng = 2 if recon == AK_PLM else 3
        if table is None:
            self.block_nx = tuple(int(v) for v in block_nx)
            self.nb = tuple(self.root_nx[d] // self.block_nx[d] for d in range(3))
            self.table = uniform_block_table(self.root_nx, self.block_nx)
            self.uniform = True
        else:
            self.table = np.ascontiguousarray(np.asarray(table, dtype=np.int32))
            self.block_nx = tuple(int(v) for v in self.table[0, 4:7])
            self.uniform = bool((self.table[:, 0] == 0).all() and
                                (self.table[:, 4:7] == self.table[0, 4:7]).all())
            self.nb = tuple(self.root_nx[d] // self.block_nx[d] for d in range(3))
        self.nblocks = int(self.table.shape[0])
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        d = ak_mesh_desc()
        d.nblocks = self.nblocks
        d.nghost = self.ng
        d.blocks = self.table.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        for a in range(3):
            d.xmin[a] = float(xmin[a])
            d.xmax[a] = float(xmax[a])
            d.root_nx[a] = self.root_nx[a]
        d.recon, d.rk, d.precision = int(recon), int(rk), int(precision)
        d.riemann = int(riemann)
        d.fofc = 1 if fofc else 0
        d.gamma, d.cfl = float(gamma), float(cfl)
        d.ref_rho, d.ref_p = float(ref_rho), float(ref_p)
        self.desc = d
        self.handle = ak_mesh_create(d, self.stream.cuda_stream)
        self.nreg, self.reg_bytes, self.offsets, self.strides = ak_mesh_layout(self.handle,
                                                                               self.nblocks)
        self.regs = [torch.empty(self.reg_bytes // 8, dtype=torch.float64, device=self.device)
                     for _ in range(self.nreg)]
        for r, t in enumerate(self.regs):
            ak_mesh_bind(self.handle, r, t.data_ptr())
        self.interior_count = 5 * int(np.prod(self.table[:, 4:7].astype(np.int64), axis=1).sum())
        # uniform meshes without FOFC: every halo cell lies in a same-level block, which
        # the stage kernels read directly, so a stage needs no ghost fill before it
        self.direct = bool((self.table[:, 0] == 0).all()) and not fofc

    def close(self):
        if getattr(self, "handle", None):
            self.stream.synchronize()
            ak_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # global (5, n3, n2, n1) <-> packed interior [block][var][k][j][i]
    def pack(self, U):
        n1, n2, n3 = self.block_nx
        b1, b2, b3 = self.nb
        U = np.asarray(U, dtype=np.float64)
        assert U.shape == (5, self.root_nx[2], self.root_nx[1], self.root_nx[0]), U.shape
        P = U.reshape(5, b3, n3, b2, n2, b1, n1).transpose(1, 3, 5, 0, 2, 4, 6)
        return np.ascontiguousarray(P).reshape(-1)

    def unpack(self, P):
        n1, n2, n3 = self.block_nx
        b1, b2, b3 = self.nb
        P = np.asarray(P).reshape(b3, b2, b1, 5, n3, n2, n1).transpose(3, 0, 4, 1, 5, 2, 6)
        return np.ascontiguousarray(P).reshape(5, self.root_nx[2], self.root_nx[1],
                                               self.root_nx[0])

    def upload_packed(self, P, reg=0):
        """Interior data packed block after block as [block][var][k][j][i]."""
        P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1)
        assert P.size == self.interior_count, (P.size, self.interior_count)
        host = self.torch.from_numpy(P).pin_memory()
        ak_upload(self.handle, reg, host.data_ptr())
        self.stream.synchronize()  # the pinned buffer may be freed after return

    def download_packed(self, reg=0):
        host = self.torch.empty(self.interior_count, dtype=self.torch.float64).pin_memory()
        ak_download(self.handle, reg, host.data_ptr())
        return host.numpy().copy()

    def upload(self, U, reg=0):
        """Global (5, n3, n2, n1) array of a uniform mesh."""
        self.upload_packed(self.pack(U), reg)

    def download(self, reg=0):
        return self.unpack(self.download_packed(reg))

    def upload_device(self, U, reg=0):
        """Global (5, n3, n2, n1) float64 torch tensor on the mesh's device (uniform
        mesh): each block's interior is copied device to device."""
        torch = self.torch
        assert self.uniform and tuple(U.shape) == (5, self.root_nx[2], self.root_nx[1],
                                                   self.root_nx[0])
        g = self.ng
        n1, n2, n3 = self.block_nx
        R = self.register_view(reg)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(self.stream):
            for b, row in enumerate(self.table):
                lx, ly, lz = int(row[1]), int(row[2]), int(row[3])
                R[b, :, g:g + n3, g:g + n2, g:g + n1].copy_(U[:, lz:lz + n3, ly:ly + n2,
                                                            lx:lx + n1])
        self.stream.synchronize()

    def download_box(self, lo, size, reg=0):
        """Interior cells lo <= (i, j, k) < lo + size of the global grid of a uniform mesh
        (no periodic wrap), as a numpy (5, s3, s2, s1) array."""
        torch = self.torch
        g = self.ng
        lo = [int(v) for v in lo]
        size = [int(v) for v in size]
        assert all(lo[d] >= 0 and lo[d] + size[d] <= self.root_nx[d] for d in range(3))
        out = torch.empty((5, size[2], size[1], size[0]), dtype=torch.float64,
                          device=self.device)
        R = self.register_view(reg)
        self.stream.synchronize()
        for b, row in enumerate(self.table):
            org = [int(row[1]), int(row[2]), int(row[3])]
            n = [int(row[4]), int(row[5]), int(row[6])]
            a = [max(lo[d], org[d]) for d in range(3)]
            e = [min(lo[d] + size[d], org[d] + n[d]) for d in range(3)]
            if any(a[d] >= e[d] for d in range(3)):
                continue
            src = R[b, :, g + a[2] - org[2]:g + e[2] - org[2], g + a[1] - org[1]:g + e[1] - org[1],
                    g + a[0] - org[0]:g + e[0] - org[0]]
            out[:, a[2] - lo[2]:e[2] - lo[2], a[1] - lo[1]:e[1] - lo[1],
                a[0] - lo[0]:e[0] - lo[0]].copy_(src)
        return out.cpu().numpy()

    def fill_ghosts(self, reg=0):
        ak_fill_ghosts(self.handle, reg)

    def stage(self, s, dt):
        ak_stage(self.handle, s, dt)

    def new_dt(self, reg=0):
        return ak_new_dt(self.handle, reg)[0]

    def step(self, dt=0.0, want_dt_next=True):
        return ak_step(self.handle, dt, want_dt_next)[0]

    def counters(self):
        return ak_status_counters(self.handle)

    def autotune(self):
        return ak_mesh_autotune(self.handle)

    def schedule(self, tile, nseg=1, order=0):
        ak_mesh_schedule(self.handle, tile, nseg, order)

    def fuse(self, fused=True):
        ak_mesh_fuse(self.handle, fused)

    def register_view(self, reg=0):
        """Torch view (nblocks, 5, p3, p2, p1) of a register, ghosts included."""
        p = [n + 2 * self.ng for n in self.block_nx]
        bstride = int(self.offsets[1] - self.offsets[0]) if self.nblocks > 1 else 0
        sv, sk, sj, si = self.strides
        t = self.regs[reg]
        return t.as_strided((self.nblocks, 5, p[2], p[1], p[0]), (bstride, sv, sk, sj, si),
                            int(self.offsets[0]))
