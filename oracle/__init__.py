"""FP64 CPU oracle of batched pose evaluation (GeoDock-MA, Alg. 1/2, Eq. 1-3).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg load it; the CUDA path never does, and the two share no code.

The arithmetic lives in ``oracle.cpp`` (plain double-precision loops, built
on first use into ``_liboracle.so`` beside this file). This module marshals
numpy arrays into it. Every function cites the passage it follows in the C++
source. Parity of each function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_liboracle.so")
_SRC = os.path.join(_HERE, "oracle.cpp")
_lock = threading.Lock()
_lib = None

P = ctypes.POINTER


def build(force: bool = False) -> str:
    """Compile oracle.cpp (g++, -O2, no FP contraction so hosts round alike)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
                ("origin", ctypes.c_double * 3), ("centre", ctypes.c_double * 3), ("K", P(ctypes.c_uint16)),
                ("pts", P(ctypes.c_int32)), ("npts", ctypes.c_int)]


class Ligands(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("atom_off", P(ctypes.c_int32)), ("xyz", P(ctypes.c_float)),
                ("bond_off", P(ctypes.c_int32)), ("bonds", P(ctypes.c_int32)), ("rot_off", P(ctypes.c_int32)),
                ("rot", P(ctypes.c_int32)), ("id_base", ctypes.c_int64), ("ids", P(ctypes.c_int64))]


class Knobs(ctypes.Structure):
    _fields_ = [("hp_step", ctypes.c_double), ("lp_step", ctypes.c_double), ("threshold", ctypes.c_double),
                ("repetitions", ctypes.c_int), ("n_poses", ctypes.c_int), ("clip_box", ctypes.c_int),
                ("score_mode", ctypes.c_int), ("enable_refinement", ctypes.c_int), ("bump_thr", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("amb_delta", ctypes.c_double), ("amb_bump", ctypes.c_double)]


class Out(ctypes.Structure):
    _fields_ = [("best_score", P(ctypes.c_double)), ("best_pose", P(ctypes.c_int32)), ("status", P(ctypes.c_int32)),
                ("pose_S", P(ctypes.c_double)), ("pose_init_S", P(ctypes.c_double)),
                ("pose_init_lo", P(ctypes.c_double)), ("pose_init_hi", P(ctypes.c_double)),
                ("pose_status", P(ctypes.c_int32)), ("pose_xyz", P(ctypes.c_double)),
                ("init_xyz", P(ctypes.c_double)), ("sweep_base", P(ctypes.c_int64)), ("force_k", P(ctypes.c_int32)),
                ("chosen_k", P(ctypes.c_int32)), ("own_k", P(ctypes.c_int32)), ("pmax", ctypes.c_int32),
                ("cand_S", P(ctypes.c_double)), ("cand_lo", P(ctypes.c_double)), ("cand_hi", P(ctypes.c_double)),
                ("cand_status", P(ctypes.c_int32)), ("cand_amb", P(ctypes.c_int32))]


class RefineKnobs(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("clip_box", ctypes.c_int), ("bump_thr", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("lambda_max", ctypes.c_double), ("grow", ctypes.c_double),
                ("shrink", ctypes.c_double), ("amb_delta", ctypes.c_double), ("amb_bump", ctypes.c_double),
                ("amb_rel", ctypes.c_double)]


class RefineOut(ctypes.Structure):
    _fields_ = [("S_start", P(ctypes.c_double)), ("S_final", P(ctypes.c_double)), ("status", P(ctypes.c_int32)),
                ("xyz", P(ctypes.c_double)), ("gstride", ctypes.c_int32), ("G", P(ctypes.c_double)),
                ("D", P(ctypes.c_double)), ("lam", P(ctypes.c_double)), ("S_new", P(ctypes.c_double)),
                ("verdict", P(ctypes.c_int32)), ("accept", P(ctypes.c_int32)), ("flags", P(ctypes.c_int32)),
                ("force_accept", P(ctypes.c_int32)), ("force_G", P(ctypes.c_double))]


# Step-length rule of the local refinement (largest atom displacement, Å):
# start at LAMBDA0, times GROW after an accepted step (at most LAMBDA_MAX),
# times SHRINK after a rejected one.
LAMBDA0, LAMBDA_MAX, GROW, SHRINK = 0.25, 1.0, 1.5, 0.5


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_field.argtypes = [ctypes.c_int] * 3 + [P(ctypes.c_int32), ctypes.c_int, P(ctypes.c_uint16),
                                                              ctypes.c_int]
            lib.oracle_field.restype = ctypes.c_int
            lib.oracle_splitmix.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_splitmix.restype = ctypes.c_uint64
            lib.oracle_score.argtypes = [P(Grid), ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_int,
                                         P(ctypes.c_double), P(ctypes.c_int)]
            lib.oracle_score.restype = ctypes.c_int
            lib.oracle_term.argtypes = [P(Grid), ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_double,
                                        P(ctypes.c_double), P(ctypes.c_int)]
            lib.oracle_term.restype = ctypes.c_int
            lib.oracle_rotate.argtypes = [P(ctypes.c_double), ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                                          ctypes.c_double, P(ctypes.c_double)]
            lib.oracle_rotate.restype = None
            lib.oracle_n_angles.argtypes = [ctypes.c_double]
            lib.oracle_n_angles.restype = ctypes.c_int
            lib.oracle_peel_tile.argtypes = [ctypes.c_double]
            lib.oracle_peel_tile.restype = ctypes.c_int
            lib.oracle_pose_rotation.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, P(ctypes.c_double)]
            lib.oracle_pose_rotation.restype = None
            lib.oracle_dock.argtypes = [P(Grid), P(Ligands), P(Knobs), P(Out), ctypes.c_int]
            lib.oracle_dock.restype = ctypes.c_int
            D, I32 = P(ctypes.c_double), P(ctypes.c_int32)
            lib.oracle_trilinear_grad.argtypes = [P(Grid), ctypes.c_int, D, ctypes.c_int, D, D, P(ctypes.c_int)]
            lib.oracle_trilinear_grad.restype = ctypes.c_int
            lib.oracle_torsions.argtypes = [P(Ligands), ctypes.c_int, I32, I32, I32, P(ctypes.c_uint8), I32,
                                            P(ctypes.c_uint8)]
            lib.oracle_torsions.restype = ctypes.c_int
            lib.oracle_dof_apply.argtypes = [P(Ligands), ctypes.c_int, D, D, D]
            lib.oracle_dof_apply.restype = ctypes.c_int
            lib.oracle_dof_grad.argtypes = [P(Ligands), ctypes.c_int, D, D, D, D]
            lib.oracle_dof_grad.restype = ctypes.c_int
            lib.oracle_refine.argtypes = [P(Grid), P(Ligands), P(RefineKnobs), D, P(RefineOut), ctypes.c_int]
            lib.oracle_refine.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(P(t))


def field(dims, pts) -> np.ndarray:
    """Floored min-squared-distance field K (grid units), shape (nz, ny, nx), x fastest.

    Tabulates the inner minimum of Eq. 1 on voxel centres by brute force."""
    nx, ny, nz = (int(d) for d in dims)
    pts = np.ascontiguousarray(pts, dtype=np.int32).reshape(-1, 3)
    K = np.zeros(nx * ny * nz, np.uint16)
    rc = _load().oracle_field(nx, ny, nz, _ptr(pts, ctypes.c_int32), len(pts), _ptr(K, ctypes.c_uint16),
                              os.cpu_count() or 1)
    if rc != 0:
        raise ValueError("oracle_field: bad arguments")
    return K.reshape(nz, ny, nx)


class OraclePocket:
    """A pocket with its oracle field, ready to pass to the C structures."""

    def __init__(self, pk, K=None):
        self.dims = pk.dims
        self.h = pk.h
        self.origin = np.asarray(pk.origin, np.float64)
        self.centre = np.asarray(pk.centre, np.float64)
        self.pts = np.ascontiguousarray(pk.pts, np.int32)
        self.K = np.ascontiguousarray(field(pk.dims, pk.pts) if K is None else K, np.uint16)

    def cstruct(self) -> Grid:
        g = Grid()
        g.nx, g.ny, g.nz = self.dims
        g.h = self.h
        g.origin[:] = list(self.origin)
        g.centre[:] = list(self.centre)
        g.K = _ptr(self.K, ctypes.c_uint16)
        g.pts = _ptr(self.pts, ctypes.c_int32)
        g.npts = len(self.pts)
        return g


def score(opk: OraclePocket, xyz, mode=0, clip=1):
    """S (grid units) and the inside flag of one conformation; o = l / (h^2 S) is Eq. 1."""
    x = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
    S = ctypes.c_double(0)
    inside = ctypes.c_int(0)
    g = opk.cstruct()
    _load().oracle_score(ctypes.byref(g), mode, clip, _ptr(x, ctypes.c_double), len(x), ctypes.byref(S),
                         ctypes.byref(inside))
    return S.value, bool(inside.value)


def term(opk: OraclePocket, x, mode=0, clip=1, delta=0.0):
    """One atom's term of Eq. 1 (grid units) with its parity band.

    Returns (D, lo, hi, flags): lo and hi bound the term over the voxel-boundary alternatives of the
    nearest-voxel lookup within delta grid units; flags bit0 inside the box, bit1 box band (an
    alternative on the other side of the box edge), bit2 lo < hi."""
    x = np.ascontiguousarray(x, np.float64).reshape(3)
    out = np.zeros(3, np.float64)
    flags = ctypes.c_int(0)
    g = opk.cstruct()
    _load().oracle_term(ctypes.byref(g), int(mode), int(clip), _ptr(x, ctypes.c_double), float(delta),
                        _ptr(out, ctypes.c_double), ctypes.byref(flags))
    return float(out[0]), float(out[1]), float(out[2]), int(flags.value)


def rotate(xyz, c, b, theta):
    """Right-handed rotation by theta (rad) about the axis through c along (c - b)/|c - b| (Alg. 1)."""
    x = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
    out = np.zeros_like(x)
    c = np.ascontiguousarray(c, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    _load().oracle_rotate(_ptr(x, ctypes.c_double), len(x), _ptr(c, ctypes.c_double), _ptr(b, ctypes.c_double),
                          float(theta), _ptr(out, ctypes.c_double))
    return out


def splitmix(seed: int, ctr: int) -> int:
    """Raw SplitMix64 output number ctr+1 of the stream seeded with `seed` (pose generator)."""
    return int(_load().oracle_splitmix(seed, ctr))


def n_angles(step: float) -> int:
    return _load().oracle_n_angles(float(step))


def peel_tile(step: float) -> int:
    """Tile size x of tile peeling (Eq. 3 reading: divisor of 360, multiple of step, nearest sqrt(360 step))."""
    return _load().oracle_peel_tile(float(step))


def pose_rotation(seed: int, lig_id: int, p: int) -> np.ndarray:
    R = np.zeros(9, np.float64)
    _load().oracle_pose_rotation(seed, lig_id, p, _ptr(R, ctypes.c_double))
    return R.reshape(3, 3)


def pmax_of(kn) -> int:
    """Candidate slots per sweep in the trace layout (slot 0 is the incumbent)."""
    p = max(n_angles(kn["hp_step"]), n_angles(kn["lp_step"]))
    if kn.get("enable_refinement", 0):
        x = peel_tile(kn["hp_step"])
        p = max(p, 1 + 360 // x + int(round(x / kn["hp_step"])))
    return p


def sweep_layout(batch, kn):
    """Per-ligand sweep count R*2T and base index into the sweep trace (ligand-major, then pose, then sweep)."""
    _, t = batch.sizes()
    nsw = kn["repetitions"] * 2 * t.astype(np.int64)
    base = np.zeros(batch.n, np.int64)
    if batch.n:
        base[1:] = np.cumsum(nsw * kn["n_poses"])[:-1]
    return nsw, base, int((nsw * kn["n_poses"]).sum())


def _ligands(batch, ids=None, keep=None):
    L = Ligands()
    L.n = batch.n
    L.atom_off = _ptr(batch.atom_off, ctypes.c_int32)
    L.xyz = _ptr(batch.xyz, ctypes.c_float)
    L.bond_off = _ptr(batch.bond_off, ctypes.c_int32)
    L.bonds = _ptr(batch.bonds, ctypes.c_int32)
    L.rot_off = _ptr(batch.rot_off, ctypes.c_int32)
    L.rot = _ptr(batch.rot, ctypes.c_int32)
    L.id_base = batch.id_base
    if ids is not None:
        ids = np.ascontiguousarray(ids, np.int64)
        keep.append(ids)
        L.ids = _ptr(ids, ctypes.c_int64)
    return L


def dock(opk: OraclePocket, batch, kn, trace=False, force_k=None, amb_delta=0.0, amb_bump=0.0, nthreads=None,
         xyz_out=False, ids=None):
    """Run the greedy sweep of Alg. 2 for every (ligand, initial pose); returns a dict of arrays.

    trace: record per-sweep choices and per-candidate S with parity flags.
    force_k: replay these per-sweep choices (trace layout) instead of the own argmax.
    """
    lib = _load()
    n = batch.n
    N = int(kn["n_poses"])
    natoms = int(batch.atom_off[-1])
    res = {
        "best_score": np.zeros(n, np.float64), "best_pose": np.zeros(n, np.int32), "status": np.zeros(n, np.int32),
        "pose_S": np.zeros(n * N, np.float64), "pose_init_S": np.zeros(n * N, np.float64),
        "pose_init_lo": np.zeros(n * N, np.float64), "pose_init_hi": np.zeros(n * N, np.float64),
        "pose_status": np.zeros(n * N, np.int32),
    }
    if xyz_out:
        res["pose_xyz"] = np.zeros(natoms * N * 3, np.float64)
        res["init_xyz"] = np.zeros(natoms * N * 3, np.float64)
    o = Out()
    for k in ("best_score", "pose_S", "pose_init_S", "pose_init_lo", "pose_init_hi", "pose_xyz", "init_xyz"):
        if k in res:
            setattr(o, k, _ptr(res[k], ctypes.c_double))
    for k in ("best_pose", "status", "pose_status"):
        setattr(o, k, _ptr(res[k], ctypes.c_int32))
    keep = []
    if trace or force_k is not None:
        nsw, base, total = sweep_layout(batch, kn)
        pmax = pmax_of(kn)
        res.update(sweep_base=base, nsweep=nsw, pmax=pmax, chosen_k=np.zeros(total, np.int32),
                   own_k=np.zeros(total, np.int32), cand_S=np.zeros(total * pmax, np.float64),
                   cand_lo=np.zeros(total * pmax, np.float64), cand_hi=np.zeros(total * pmax, np.float64),
                   cand_status=np.zeros(total * pmax, np.int32), cand_amb=np.zeros(total * pmax, np.int32))
        o.sweep_base = _ptr(base, ctypes.c_int64)
        o.pmax = pmax
        for k in ("chosen_k", "own_k", "cand_status", "cand_amb"):
            setattr(o, k, _ptr(res[k], ctypes.c_int32))
        for k in ("cand_S", "cand_lo", "cand_hi"):
            setattr(o, k, _ptr(res[k], ctypes.c_double))
        if force_k is not None:
            fk = np.ascontiguousarray(force_k, np.int32)
            assert fk.shape == (total,)
            keep.append(fk)
            o.force_k = _ptr(fk, ctypes.c_int32)
    g = opk.cstruct()
    L = _ligands(batch, ids, keep)
    k = Knobs()
    k.hp_step, k.lp_step, k.threshold = float(kn["hp_step"]), float(kn["lp_step"]), float(kn["threshold"])
    k.repetitions, k.n_poses, k.clip_box = int(kn["repetitions"]), N, int(kn["clip_box"])
    k.score_mode, k.enable_refinement = int(kn["score_mode"]), int(kn.get("enable_refinement", 0))
    k.bump_thr, k.seed = float(kn["bump_thr"]), int(kn["seed"])
    k.amb_delta, k.amb_bump = float(amb_delta), float(amb_bump)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = lib.oracle_dock(ctypes.byref(g), ctypes.byref(L), ctypes.byref(k), ctypes.byref(o), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_dock: bad knobs ({rc})")
    res["threads"] = int(nthreads)
    return res


# ---------------------------------------------------------------- local refinement (not in the paper)

def trilinear_grad(opk: OraclePocket, xyz, clip=1):
    """Trilinear S (grid units), dS/dx (grid units per Å, shape (l, 3)) and the inside flag."""
    x = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
    dS = np.zeros_like(x)
    S = ctypes.c_double(0)
    inside = ctypes.c_int(0)
    g = opk.cstruct()
    _load().oracle_trilinear_grad(ctypes.byref(g), int(clip), _ptr(x, ctypes.c_double), len(x), ctypes.byref(S),
                                  _ptr(dS, ctypes.c_double), ctypes.byref(inside))
    return S.value, dS, bool(inside.value)


def torsions(batch, b):
    """Torsion layout of ligand b: dict of c, b, depth, mask (T, l), order (application), check (l, l)."""
    l = int(batch.atom_off[b + 1] - batch.atom_off[b])
    T = int(batch.rot_off[b + 1] - batch.rot_off[b])
    c, bb, depth, order = (np.zeros(max(T, 1), np.int32) for _ in range(4))
    mask = np.zeros(max(T, 1) * l, np.uint8)
    check = np.zeros(l * l, np.uint8)
    keep = []
    L = _ligands(batch, None, keep)
    r = _load().oracle_torsions(ctypes.byref(L), int(b), _ptr(c, ctypes.c_int32), _ptr(bb, ctypes.c_int32),
                                _ptr(depth, ctypes.c_int32), _ptr(mask, ctypes.c_uint8), _ptr(order, ctypes.c_int32),
                                _ptr(check, ctypes.c_uint8))
    if r < 0:
        raise ValueError("ring bond among the rotatable bonds")
    return dict(c=c[:T], b=bb[:T], depth=depth[:T], mask=mask[:T * l].reshape(T, l).astype(bool), order=order[:T],
                check=check.reshape(l, l).astype(bool))


def dof_apply(batch, b, x, q):
    """Pose z = g + R(omega)(tau(x) - g) + t for ligand b: q = (t, omega, theta_1..theta_T)."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, np.float64)
    z = np.zeros_like(x)
    keep = []
    L = _ligands(batch, None, keep)
    if _load().oracle_dof_apply(ctypes.byref(L), int(b), _ptr(x, ctypes.c_double), _ptr(q, ctypes.c_double),
                                _ptr(z, ctypes.c_double)) != 0:
        raise ValueError("ring bond among the rotatable bonds")
    return z


def dof_grad(batch, b, x, q, p):
    """d f / d q at z = dof_apply(x, q), given p = d f / d z (shape (l, 3))."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, np.float64)
    p = np.ascontiguousarray(p, np.float64).reshape(-1, 3)
    G = np.zeros(len(q), np.float64)
    keep = []
    L = _ligands(batch, None, keep)
    if _load().oracle_dof_grad(ctypes.byref(L), int(b), _ptr(x, ctypes.c_double), _ptr(q, ctypes.c_double),
                               _ptr(p, ctypes.c_double), _ptr(G, ctypes.c_double)) != 0:
        raise ValueError("ring bond among the rotatable bonds")
    return G


def refine(opk: OraclePocket, batch, xyz_in, steps=20, clip=1, bump_thr=2.0, force_accept=None, force_G=None,
           amb_delta=0.0, amb_bump=0.0, amb_rel=0.0, nthreads=None, lambda0=LAMBDA0, lambda_max=LAMBDA_MAX, grow=GROW,
           shrink=SHRINK):
    """Local refinement (trilinear Eq. 1, gradient ascent over rigid DOF and torsions) from xyz_in (Å).

    Replay: force_accept commits given decisions; force_G (n, steps, >= 6 + T) gives the step direction where
    an atom of the step's start pose lies within amb_delta of a cell face (flag bit 3), where the gradient of
    the trilinear score is one-sided and either side is valid."""
    n = batch.n
    natoms = int(batch.atom_off[-1])
    x = np.ascontiguousarray(xyz_in, np.float64).reshape(natoms, 3)
    _, t = batch.sizes()
    gstride = 6 + (int(t.max()) if n else 0)
    ns = n * steps
    res = dict(S_start=np.zeros(n), S_final=np.zeros(n), status=np.zeros(n, np.int32), xyz=np.zeros((natoms, 3)),
               G=np.zeros(ns * gstride), D=np.zeros(ns), lam=np.zeros(ns), S_new=np.zeros(ns),
               verdict=np.zeros(ns, np.int32), accept=np.zeros(ns, np.int32), flags=np.zeros(ns, np.int32),
               gstride=gstride)
    o = RefineOut()
    for k in ("S_start", "S_final", "xyz", "G", "D", "lam", "S_new"):
        setattr(o, k, _ptr(res[k], ctypes.c_double))
    for k in ("status", "verdict", "accept", "flags"):
        setattr(o, k, _ptr(res[k], ctypes.c_int32))
    o.gstride = gstride
    keep = []
    if force_accept is not None:
        fa = np.ascontiguousarray(force_accept, np.int32)
        assert fa.shape == (ns,)
        keep.append(fa)
        o.force_accept = _ptr(fa, ctypes.c_int32)
    if force_G is not None and ns:
        fg = np.zeros((n, steps, gstride))
        src = np.asarray(force_G, np.float64)
        fg[:, :, :min(gstride, src.shape[-1])] = src.reshape(n, steps, -1)[:, :, :gstride]
        fg = np.ascontiguousarray(fg.reshape(-1))
        keep.append(fg)
        o.force_G = _ptr(fg, ctypes.c_double)
    k = RefineKnobs(int(steps), int(clip), float(bump_thr), float(lambda0), float(lambda_max), float(grow),
                    float(shrink), float(amb_delta), float(amb_bump), float(amb_rel))
    g = opk.cstruct()
    L = _ligands(batch, None, keep)
    rc = _load().oracle_refine(ctypes.byref(g), ctypes.byref(L), ctypes.byref(k), _ptr(x, ctypes.c_double),
                               ctypes.byref(o), int(nthreads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("oracle_refine: bad knobs")
    res["G"] = res["G"].reshape(n, steps, gstride) if ns else res["G"]
    return res
