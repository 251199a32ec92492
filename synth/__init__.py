"""Seeded synthetic inputs for batched pose evaluation.

Ligands are random trees of heavy atoms with marked rotatable bonds; pockets
are noisy ellipsoidal cavities given as probe points on voxel centres (the
paper docks into PASS probe-sphere centres, Sec. 3.1 and 4.1; its 113K-ligand
library and PDB pockets are not available, so these stand in for them with
the same ranges of atom and rotamer counts).

This module draws inputs only. It holds none of the docking arithmetic (no
field, score, rotation, clash test or sweep), so both the CUDA path and the
CPU oracle can take its arrays. The generator itself is C (``synth.c``),
compiled on first use into ``_libsynth.so`` beside this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_libsynth.so")
_SRC = os.path.join(_HERE, "synth.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into _libsynth.so (plain C, no FP contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            i32p, f64p = P(ctypes.c_int), P(ctypes.c_double)
            lib.synth_batch_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, f64p, i32p, i32p]
            lib.synth_batch_sizes.restype = None
            lib.synth_batch.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, i32p, i32p, i32p, i32p, i32p,
                                        f64p, i32p, i32p]
            lib.synth_batch.restype = ctypes.c_int
            lib.synth_pocket.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, i32p,
                                         ctypes.c_int, i32p, f64p, f64p]
            lib.synth_pocket.restype = ctypes.c_int
            lib.synth_semi_axes.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_double, f64p]
            lib.synth_semi_axes.restype = None
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


class LigandBatch:
    """CSR batch of ligands.

    atom_off, bond_off, rot_off: int32 [n+1]; xyz: float32 [atoms, 3] (Å);
    bonds: int32 [bonds, 2] (ligand-local atom indices); rot: int32 [rot]
    (ligand-local bond indices, ascending per ligand); id_base: id of ligand 0.
    """

    def __init__(self, atom_off, bond_off, rot_off, xyz, bonds, rot, id_base=0):
        self.atom_off = np.ascontiguousarray(atom_off, dtype=np.int32)
        self.bond_off = np.ascontiguousarray(bond_off, dtype=np.int32)
        self.rot_off = np.ascontiguousarray(rot_off, dtype=np.int32)
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
        self.bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
        self.rot = np.ascontiguousarray(rot, dtype=np.int32).reshape(-1)
        self.id_base = int(id_base)

    @property
    def n(self) -> int:
        return len(self.atom_off) - 1

    def sizes(self):
        return np.diff(self.atom_off), np.diff(self.rot_off)

    def subset(self, idx):
        """Batch of the ligands idx (in that order); ids are not kept."""
        idx = np.asarray(idx, dtype=np.int64)
        l, t = self.sizes()
        nb = np.diff(self.bond_off)
        ao = np.concatenate([[0], np.cumsum(l[idx])])
        bo = np.concatenate([[0], np.cumsum(nb[idx])])
        ro = np.concatenate([[0], np.cumsum(t[idx])])
        xyz = np.concatenate([self.xyz[self.atom_off[i]:self.atom_off[i + 1]] for i in idx]) if len(idx) else \
            np.zeros((0, 3), np.float32)
        bonds = np.concatenate([self.bonds[self.bond_off[i]:self.bond_off[i + 1]] for i in idx]) if len(idx) else \
            np.zeros((0, 2), np.int32)
        rot = np.concatenate([self.rot[self.rot_off[i]:self.rot_off[i + 1]] for i in idx]) if len(idx) else \
            np.zeros((0,), np.int32)
        return LigandBatch(ao, bo, ro, xyz, bonds, rot, 0)


def ligand_sizes(seed: int, n: int, kind: int, prm, id0: int = 0):
    lib = _load()
    prm = np.ascontiguousarray(prm, dtype=np.float64)
    l = np.zeros(n, np.int32)
    t = np.zeros(n, np.int32)
    lib.synth_batch_sizes(seed, id0, n, kind, _p(prm, ctypes.c_double), _p(l, ctypes.c_int), _p(t, ctypes.c_int))
    return l, t


def ligand_batch(seed: int, l, t, id0: int = 0) -> LigandBatch:
    """Grow len(l) ligands with atom counts l and requested rotatable counts t."""
    lib = _load()
    l = np.ascontiguousarray(l, dtype=np.int32)
    t = np.ascontiguousarray(t, dtype=np.int32)
    n = len(l)
    na = int(l.sum())
    ao = np.zeros(n + 1, np.int32)
    bo = np.zeros(n + 1, np.int32)
    ro = np.zeros(n + 1, np.int32)
    xyz = np.zeros(3 * max(na, 1), np.float64)
    bonds = np.zeros(2 * max(na - n, 1), np.int32)
    rot = np.zeros(max(int(t.sum()), 1), np.int32)
    rc = lib.synth_batch(seed, id0, n, _p(l, ctypes.c_int), _p(t, ctypes.c_int), _p(ao, ctypes.c_int),
                         _p(bo, ctypes.c_int), _p(ro, ctypes.c_int), _p(xyz, ctypes.c_double),
                         _p(bonds, ctypes.c_int), _p(rot, ctypes.c_int))
    if rc != 0:
        raise RuntimeError(f"synth_batch failed ({rc})")
    return LigandBatch(ao, bo, ro, xyz[:3 * na].astype(np.float32), bonds[:2 * (na - n)], rot[:ro[-1]], id0)


class Pocket:
    """A pocket: probe points on voxel centres of an n^3 grid.

    pts: int32 [p, 3] voxel indices (x, y, z); h: voxel edge (Å);
    origin: centre of voxel (0,0,0) (Å); centre: probe centroid (Å).
    """

    def __init__(self, dims, h, origin, centre, pts):
        self.dims = tuple(int(d) for d in dims)
        self.h = float(h)
        self.origin = np.asarray(origin, np.float64)
        self.centre = np.asarray(centre, np.float64)
        self.pts = np.ascontiguousarray(pts, dtype=np.int32).reshape(-1, 3)


def pocket(seed: int, n: int, h: float, abc, sigma: float = 0.5, stride: int = 3) -> Pocket:
    lib = _load()
    cap = (n // stride + 1) ** 3
    pts = np.zeros(3 * cap, np.int32)
    npts = ctypes.c_int(0)
    origin = np.zeros(3, np.float64)
    centre = np.zeros(3, np.float64)
    rc = lib.synth_pocket(seed, n, h, abc[0], abc[1], abc[2], sigma, stride, _p(pts, ctypes.c_int), cap,
                          ctypes.byref(npts), _p(origin, ctypes.c_double), _p(centre, ctypes.c_double))
    if rc != 0:
        raise RuntimeError("synth_pocket failed")
    return Pocket((n, n, n), h, origin, centre, pts[:3 * npts.value])


def semi_axes(seed: int, pid: int, lo: float, hi: float):
    lib = _load()
    out = np.zeros(3, np.float64)
    lib.synth_semi_axes(seed, pid, lo, hi, _p(out, ctypes.c_double))
    return out
