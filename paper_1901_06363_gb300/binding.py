"""ctypes binding of libgeodock.so (argument marshalling only).

Host inputs are numpy arrays; device outputs are torch CUDA tensors, whose
data pointers and the current torch stream are handed to the C calls. PyTorch
is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# GEODOCK_CHECKED=1 selects the checked build (index checks in every kernel, reported as call errors)
library_path = os.path.join(HERE, "libgeodock_checked.so" if os.environ.get("GEODOCK_CHECKED") == "1"
                            else "libgeodock.so")

DOCK_OK = 0
DOCK_ERR_INVALID_ARG = -1
DOCK_ERR_TOPOLOGY = -2
DOCK_ERR_OUT_OF_MEMORY = -3
DOCK_ERR_CUDA = -4
DOCK_ERR_TIMEOUT = -5
DOCK_ERR_UNSUPPORTED = -6

P = ctypes.POINTER


class dock_pocket(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
                ("origin", ctypes.c_double * 3), ("centre", ctypes.c_double * 3), ("K", P(ctypes.c_uint16)),
                ("pts", P(ctypes.c_int32)), ("npts", ctypes.c_int)]


class dock_ligand_batch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("atom_off", P(ctypes.c_int32)), ("xyz", P(ctypes.c_float)),
                ("bond_off", P(ctypes.c_int32)), ("bonds", P(ctypes.c_int32)), ("rot_off", P(ctypes.c_int32)),
                ("rot", P(ctypes.c_int32)), ("id_base", ctypes.c_int64), ("ids", P(ctypes.c_int64))]


class dock_knobs(ctypes.Structure):
    _fields_ = [("hp_step", ctypes.c_double), ("lp_step", ctypes.c_double), ("threshold", ctypes.c_double),
                ("repetitions", ctypes.c_int), ("n_poses", ctypes.c_int), ("enable_refinement", ctypes.c_int),
                ("clip_box", ctypes.c_int), ("bump_thr", ctypes.c_double), ("score_mode", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("seed", ctypes.c_uint64), ("plain_mode", ctypes.c_int)]


class dock_result(ctypes.Structure):
    _fields_ = [("score", ctypes.c_float), ("pose", ctypes.c_int32), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


RESULT_DTYPE = np.dtype([("score", np.float32), ("pose", np.int32), ("status", np.int32), ("reserved", np.int32)])


class dock_trace(ctypes.Structure):
    _fields_ = [("pmax", ctypes.c_int32), ("sweep_base", ctypes.c_void_p), ("chosen_k", ctypes.c_void_p),
                ("cand_S", ctypes.c_void_p), ("cand_status", ctypes.c_void_p), ("pose_S", ctypes.c_void_p),
                ("pose_init_S", ctypes.c_void_p), ("pose_status", ctypes.c_void_p), ("init_xyz", ctypes.c_void_p),
                ("pose_xyz", ctypes.c_void_p)]


class dock_tile(ctypes.Structure):
    _fields_ = [("lanes_per_pose", ctypes.c_int), ("angles_per_chunk", ctypes.c_int), ("warps_per_cta", ctypes.c_int)]


class dock_stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_uint64), ("atom_updates", ctypes.c_uint64), ("pair_bounds", ctypes.c_uint64),
                ("bump_pairs", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64), ("sweep_ms", ctypes.c_double),
                ("pose_reps_skipped", ctypes.c_uint64), ("lookups_skipped", ctypes.c_uint64)]


class dock_peaks(ctypes.Structure):
    _fields_ = [("fma_per_s", ctypes.c_double), ("ffma2_per_s", ctypes.c_double), ("tex_field_per_s", ctypes.c_double),
                ("tex_local_per_s", ctypes.c_double), ("l2_sectors_per_s", ctypes.c_double)]


class dock_refine_trace_buf(ctypes.Structure):
    _fields_ = [("gstride", ctypes.c_int32), ("G", ctypes.c_void_p), ("D", ctypes.c_void_p), ("lam", ctypes.c_void_p),
                ("S_new", ctypes.c_void_p), ("verdict", ctypes.c_void_p), ("accept", ctypes.c_void_p),
                ("S_start", ctypes.c_void_p), ("S_final", ctypes.c_void_p), ("status", ctypes.c_void_p)]


def _load():
    if not os.path.exists(library_path):
        raise ImportError(f"{library_path} is missing: build it with `python -m paper_1901_06363_gb300.build` "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(library_path)
    vp, i32p = ctypes.c_void_p, P(ctypes.c_int)
    sig = {
        "dock_create": ([P(vp), ctypes.c_int], ctypes.c_int),
        "dock_destroy": ([vp], None),
        "dock_last_error": ([vp], ctypes.c_char_p),
        "dock_init_pocket": ([vp, P(dock_pocket), i32p], ctypes.c_int),
        "dock_pocket_field": ([vp, ctypes.c_int, P(ctypes.c_uint16)], ctypes.c_int),
        "dock_upload_ligands": ([vp, P(dock_ligand_batch), i32p], ctypes.c_int),
        "dock_release_batch": ([vp, ctypes.c_int], ctypes.c_int),
        "dock_run": ([vp, ctypes.c_int, P(ctypes.c_int32), ctypes.c_int, P(dock_knobs), vp, vp, ctypes.c_int, vp],
                     ctypes.c_int),
        "dock_run_database": ([vp, P(dock_ligand_batch), P(ctypes.c_int32), ctypes.c_int, P(dock_knobs), ctypes.c_int,
                               vp, vp, vp], ctypes.c_int),
        "dock_run_trace": ([vp, ctypes.c_int, ctypes.c_int, P(dock_knobs), P(dock_trace), vp, vp], ctypes.c_int),
        "dock_trace_pmax": ([P(dock_knobs)], ctypes.c_int),
        "dock_set_tile": ([vp, P(dock_tile)], ctypes.c_int),
        "dock_get_tile": ([vp, P(dock_tile)], ctypes.c_int),
        "dock_autotune": ([vp, ctypes.c_int, ctypes.c_int, P(dock_knobs), P(dock_tile), vp], ctypes.c_int),
        "dock_last_stats": ([vp, P(dock_stats)], ctypes.c_int),
        "dock_measure_peaks": ([vp, ctypes.c_int, P(dock_peaks), vp], ctypes.c_int),
        "dock_run_static": ([vp, ctypes.c_int, ctypes.c_int, P(dock_knobs), vp, vp, vp], ctypes.c_int),
        "dock_batch_info": ([vp, ctypes.c_int, i32p, i32p, i32p, i32p], ctypes.c_int),
        "dock_score_trilinear": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "dock_score_trilinear_grad": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp], ctypes.c_int),
        "dock_dof_apply": ([vp, ctypes.c_int, vp, vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "dock_dof_grad": ([vp, ctypes.c_int, vp, vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "dock_refine": ([vp, ctypes.c_int, P(ctypes.c_int32), ctypes.c_int, P(dock_knobs), vp, vp, vp, ctypes.c_int,
                         vp], ctypes.c_int),
        "dock_refine_trace": ([vp, ctypes.c_int, ctypes.c_int, P(dock_knobs), vp, P(dock_refine_trace_buf), vp, vp],
                              ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


class DockError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def knobs_struct(kn) -> dock_knobs:
    """dock_knobs from a knob dict (keys as in synth.configs.knobs)."""
    k = dock_knobs()
    k.hp_step = float(kn["hp_step"])
    k.lp_step = float(kn.get("lp_step", kn["hp_step"]))
    k.threshold = float(kn.get("threshold", 0.0))
    k.repetitions = int(kn.get("repetitions", 1))
    k.n_poses = int(kn.get("n_poses", 1))
    k.enable_refinement = int(kn.get("enable_refinement", 0))
    k.clip_box = int(kn.get("clip_box", 1))
    k.bump_thr = float(kn.get("bump_thr", 2.0))
    k.score_mode = int(kn.get("score_mode", 0))
    k.refine_steps = int(kn.get("refine_steps", 0))
    k.seed = int(kn.get("seed", 0))
    k.plain_mode = int(kn.get("plain_mode", 0))
    return k


def _ptr(a, t):
    return a.ctypes.data_as(P(t))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Docker:
    """One dock_ctx on a CUDA device; methods mirror the C calls."""

    def __init__(self, device: int = 0):
        self._c = ctypes.c_void_p()
        rc = lib.dock_create(ctypes.byref(self._c), device)
        if rc != DOCK_OK:
            raise DockError(rc, f"dock_create(device={device}) failed")
        self._keep = []

    def close(self):
        if self._c:
            lib.dock_destroy(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != DOCK_OK:
            raise DockError(rc, f"{what}: {lib.dock_last_error(self._c).decode()}")

    # ---------------------------------------------------------------- inputs
    def init_pocket(self, pk, K=None) -> int:
        """dock_init_pocket: pk has dims, h, origin, centre, pts (voxel indices)."""
        p = dock_pocket()
        p.nx, p.ny, p.nz = (int(d) for d in pk.dims)
        p.h = float(pk.h)
        p.origin[:] = [float(v) for v in pk.origin]
        p.centre[:] = [float(v) for v in pk.centre]
        pts = np.ascontiguousarray(pk.pts, np.int32).reshape(-1, 3)
        p.pts = _ptr(pts, ctypes.c_int32)
        p.npts = len(pts)
        if K is not None:
            K = np.ascontiguousarray(K, np.uint16)
            p.K = _ptr(K, ctypes.c_uint16)
        pid = ctypes.c_int(-1)
        self._check(lib.dock_init_pocket(self._c, ctypes.byref(p), ctypes.byref(pid)), "dock_init_pocket")
        return pid.value

    def pocket_field(self, pid: int, dims) -> np.ndarray:
        nx, ny, nz = dims
        K = np.zeros(nx * ny * nz, np.uint16)
        self._check(lib.dock_pocket_field(self._c, pid, _ptr(K, ctypes.c_uint16)), "dock_pocket_field")
        return K.reshape(nz, ny, nx)

    @staticmethod
    def _batch_struct(batch, ids=None):
        """dock_ligand_batch over the batch's arrays; returns (struct, arrays to keep alive during the call)."""
        b = dock_ligand_batch()
        b.n = batch.n
        arrs = [np.ascontiguousarray(batch.atom_off, np.int32), np.ascontiguousarray(batch.xyz, np.float32),
                np.ascontiguousarray(batch.bond_off, np.int32), np.ascontiguousarray(batch.bonds, np.int32),
                np.ascontiguousarray(batch.rot_off, np.int32), np.ascontiguousarray(batch.rot, np.int32)]
        b.atom_off = _ptr(arrs[0], ctypes.c_int32)
        b.xyz = _ptr(arrs[1], ctypes.c_float)
        b.bond_off = _ptr(arrs[2], ctypes.c_int32)
        b.bonds = _ptr(arrs[3], ctypes.c_int32)
        b.rot_off = _ptr(arrs[4], ctypes.c_int32)
        b.rot = _ptr(arrs[5], ctypes.c_int32)
        b.id_base = int(batch.id_base)
        if ids is not None:
            ids = np.ascontiguousarray(ids, np.int64).reshape(-1)
            if len(ids) != batch.n:
                raise ValueError(f"ids: {len(ids)} values for {batch.n} ligands")
            b.ids = _ptr(ids, ctypes.c_int64)
            arrs.append(ids)
        return b, arrs

    def upload_ligands(self, batch, ids=None) -> int:
        b, keep = self._batch_struct(batch, ids)
        bid = ctypes.c_int(-1)
        self._check(lib.dock_upload_ligands(self._c, ctypes.byref(b), ctypes.byref(bid)), "dock_upload_ligands")
        del keep
        return bid.value

    def run_database(self, batch, pocket_ids, kn, chunk: int = 1024, xyz: bool = True, ids=None, stream=None):
        """dock_run_database: dock a host-memory ligand database chunk by chunk (host preparation of the next
        chunk overlapping the device sweep). Returns (results structured array, xyz array or None)."""
        pids = np.ascontiguousarray(pocket_ids, np.int32).reshape(-1)
        k = knobs_struct(kn)
        npk, n = len(pids), int(batch.n)
        natoms = int(batch.atom_off[-1]) if n else 0
        b, keep = self._batch_struct(batch, ids)
        out = np.zeros(npk * n, RESULT_DTYPE)
        xyz_out = np.zeros((npk, natoms, 3), np.float32) if xyz else None
        rc = lib.dock_run_database(self._c, ctypes.byref(b), _ptr(pids, ctypes.c_int32), npk, ctypes.byref(k), int(chunk),
                                   ctypes.c_void_p(out.ctypes.data),
                                   ctypes.c_void_p(xyz_out.ctypes.data) if xyz else None,
                                   _stream_ptr(stream) if stream is not None else None)
        del keep
        self._check(rc, "dock_run_database")
        return out, xyz_out

    def release_batch(self, bid: int):
        self._check(lib.dock_release_batch(self._c, bid), "dock_release_batch")

    # ------------------------------------------------------------------- runs
    def run(self, bid: int, pocket_ids, kn, n: int, natoms: int, xyz: bool = True, out=None, xyz_out=None,
            stream=None):
        """dock_run with host outputs (numpy) unless `out` is a torch CUDA tensor.

        Returns (results structured array or tensor, xyz array or tensor or None)."""
        pids = np.ascontiguousarray(pocket_ids, np.int32).reshape(-1)
        k = knobs_struct(kn)
        npk = len(pids)
        on_dev = out is not None and hasattr(out, "data_ptr")
        if on_dev:
            res_ptr = ctypes.c_void_p(out.data_ptr())
            xyz_ptr = ctypes.c_void_p(xyz_out.data_ptr()) if xyz_out is not None else None
            st = _stream_ptr(stream)
        else:
            out = np.zeros(npk * n, RESULT_DTYPE)
            res_ptr = ctypes.c_void_p(out.ctypes.data)
            if xyz:
                xyz_out = np.zeros((npk, natoms, 3), np.float32)
                xyz_ptr = ctypes.c_void_p(xyz_out.ctypes.data)
            else:
                xyz_out, xyz_ptr = None, None
            st = _stream_ptr(stream) if stream is not None else None
        rc = lib.dock_run(self._c, bid, _ptr(pids, ctypes.c_int32), npk, ctypes.byref(k), res_ptr, xyz_ptr,
                          1 if on_dev else 0, st)
        self._check(rc, "dock_run")
        return out, xyz_out

    def run_trace(self, bid: int, pid: int, kn, batch):
        """dock_run_trace: per-candidate trace (device buffers via torch), returned as numpy arrays."""
        bufs, sizes, pmax, out = self.run_trace_device(bid, pid, kn, batch)
        res = {name: tns.cpu().numpy()[:sizes[name]] for name, tns in bufs.items()}
        res["pmax"] = pmax
        res["result"] = out
        return res

    def run_trace_device(self, bid: int, pid: int, kn, batch):
        """dock_run_trace into torch CUDA tensors, left on the device.

        Returns (tensors by trace field, valid length of each, pmax, host results)."""
        import torch
        k = knobs_struct(kn)
        pmax = lib.dock_trace_pmax(ctypes.byref(k))
        N = int(kn["n_poses"])
        _, t = batch.sizes()
        nsw = int(kn["repetitions"]) * 2 * t.astype(np.int64)
        total = int((nsw * N).sum())
        natoms = int(batch.atom_off[-1])
        dev = torch.device("cuda")
        bufs = dict(chosen_k=torch.zeros(max(total, 1), dtype=torch.int32, device=dev),
                    cand_S=torch.zeros(max(total * pmax, 1), dtype=torch.float32, device=dev),
                    cand_status=torch.zeros(max(total * pmax, 1), dtype=torch.int32, device=dev),
                    pose_S=torch.zeros(max(batch.n * N, 1), dtype=torch.float32, device=dev),
                    pose_init_S=torch.zeros(max(batch.n * N, 1), dtype=torch.float32, device=dev),
                    pose_status=torch.zeros(max(batch.n * N, 1), dtype=torch.int32, device=dev),
                    init_xyz=torch.zeros(max(natoms * N * 3, 1), dtype=torch.float32, device=dev),
                    pose_xyz=torch.zeros(max(natoms * N * 3, 1), dtype=torch.float32, device=dev))
        tr = dock_trace()
        tr.pmax = pmax
        for name, tns in bufs.items():
            setattr(tr, name, tns.data_ptr())
        out = np.zeros(batch.n, RESULT_DTYPE)
        torch.cuda.synchronize()
        rc = lib.dock_run_trace(self._c, bid, pid, ctypes.byref(k), ctypes.byref(tr), ctypes.c_void_p(out.ctypes.data),
                                _stream_ptr(None))
        self._check(rc, "dock_run_trace")
        sizes = {"chosen_k": total, "cand_S": total * pmax, "cand_status": total * pmax, "pose_S": batch.n * N,
                 "pose_init_S": batch.n * N, "pose_status": batch.n * N, "init_xyz": natoms * N * 3,
                 "pose_xyz": natoms * N * 3}
        return bufs, sizes, pmax, out

    # ------------------------------------------------------------------ tiles
    def set_tile(self, lanes_per_pose=0, angles_per_chunk=0, warps_per_cta=0):
        t = dock_tile(lanes_per_pose, angles_per_chunk, warps_per_cta)
        self._check(lib.dock_set_tile(self._c, ctypes.byref(t)), "dock_set_tile")

    def autotune(self, bid: int, pid: int, kn, stream=None):
        k = knobs_struct(kn)
        t = dock_tile()
        self._check(lib.dock_autotune(self._c, bid, pid, ctypes.byref(k), ctypes.byref(t), _stream_ptr(stream)),
                    "dock_autotune")
        return (t.lanes_per_pose, t.angles_per_chunk, t.warps_per_cta)

    def stats(self):
        s = dock_stats()
        self._check(lib.dock_last_stats(self._c, ctypes.byref(s)), "dock_last_stats")
        return {name: getattr(s, name) for name, _ in dock_stats._fields_}

    def measure_peaks(self, pid: int, stream=None):
        """dock_measure_peaks: the device's measured FMA, texture-fetch and L2-sector rates (per second)."""
        p = dock_peaks()
        self._check(lib.dock_measure_peaks(self._c, pid, ctypes.byref(p),
                                           _stream_ptr(stream) if stream is not None else None),
                    "dock_measure_peaks")
        return {name: getattr(p, name) for name, _ in dock_peaks._fields_}

    # ------------------------------------------- refinement and differentiable score
    def batch_info(self, bid: int):
        """(ligands, atoms, largest ligand, largest torsion count) of a batch."""
        v = [ctypes.c_int(0) for _ in range(4)]
        self._check(lib.dock_batch_info(self._c, bid, *[ctypes.byref(x) for x in v]), "dock_batch_info")
        return tuple(x.value for x in v)

    def score_trilinear(self, bid: int, pid: int, xyz, clip: int = 1, out=None, stream=None):
        """o per ligand (torch CUDA tensor) of the poses xyz (CUDA float32, atom_off layout)."""
        import torch
        n = self.batch_info(bid)[0]
        xyz = xyz.contiguous()
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=xyz.device)
        self._check(lib.dock_score_trilinear(self._c, bid, pid, int(clip), ctypes.c_void_p(xyz.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
                    "dock_score_trilinear")
        return out

    def score_trilinear_grad(self, bid: int, pid: int, xyz, grad_o=None, clip: int = 1, stream=None):
        import torch
        xyz = xyz.contiguous()
        g = torch.empty_like(xyz)
        go = grad_o.contiguous() if grad_o is not None else None
        self._check(lib.dock_score_trilinear_grad(self._c, bid, pid, int(clip), ctypes.c_void_p(xyz.data_ptr()),
                                                  ctypes.c_void_p(go.data_ptr()) if go is not None else None,
                                                  ctypes.c_void_p(g.data_ptr()), _stream_ptr(stream)),
                    "dock_score_trilinear_grad")
        return g

    def dof_apply(self, bid: int, x, q, stream=None):
        """Pose z of x moved by q (CUDA float32, shape (n, qstride), qstride >= 6 + tmax)."""
        import torch
        x, q = x.contiguous(), q.contiguous()
        z = torch.empty_like(x)
        self._check(lib.dock_dof_apply(self._c, bid, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                       q.shape[-1], ctypes.c_void_p(z.data_ptr()), _stream_ptr(stream)),
                    "dock_dof_apply")
        return z

    def dof_grad(self, bid: int, x, q, grad_z, stream=None):
        import torch
        x, q, grad_z = x.contiguous(), q.contiguous(), grad_z.contiguous()
        g = torch.empty_like(q)
        self._check(lib.dock_dof_grad(self._c, bid, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                      q.shape[-1], ctypes.c_void_p(grad_z.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                      _stream_ptr(stream)), "dock_dof_grad")
        return g

    def refine(self, bid: int, pocket_ids, kn, xyz_in, out=None, xyz_out=None, stream=None):
        """dock_refine. xyz_in a CUDA tensor: device outputs (given or allocated); numpy: host outputs."""
        pids = np.ascontiguousarray(pocket_ids, np.int32).reshape(-1)
        k = knobs_struct(kn)
        n, natoms = self.batch_info(bid)[:2]
        npk = len(pids)
        if hasattr(xyz_in, "data_ptr"):
            import torch
            xyz_in = xyz_in.contiguous()
            if out is None:
                out = torch.empty(npk * n * 4, dtype=torch.int32, device=xyz_in.device)
            if xyz_out is None:
                xyz_out = torch.empty_like(xyz_in)
            rc = lib.dock_refine(self._c, bid, _ptr(pids, ctypes.c_int32), npk, ctypes.byref(k),
                                 ctypes.c_void_p(xyz_in.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(xyz_out.data_ptr()), 1, _stream_ptr(stream))
        else:
            xin = np.ascontiguousarray(xyz_in, np.float32)
            out = np.zeros(npk * n, RESULT_DTYPE)
            xyz_out = np.zeros((npk, natoms, 3), np.float32)
            rc = lib.dock_refine(self._c, bid, _ptr(pids, ctypes.c_int32), npk, ctypes.byref(k),
                                 ctypes.c_void_p(xin.ctypes.data), ctypes.c_void_p(out.ctypes.data),
                                 ctypes.c_void_p(xyz_out.ctypes.data), 0, None)
        self._check(rc, "dock_refine")
        return out, xyz_out

    def refine_trace(self, bid: int, pid: int, kn, xyz_in):
        """dock_refine_trace with host buffers; returns a dict of numpy arrays."""
        n, natoms, _, tmax = self.batch_info(bid)
        steps = int(kn["refine_steps"])
        gstride = 6 + tmax
        ns = max(n * steps, 1)
        bufs = dict(G=np.zeros(ns * gstride, np.float32), D=np.zeros(ns, np.float32), lam=np.zeros(ns, np.float32),
                    S_new=np.zeros(ns, np.float32), verdict=np.zeros(ns, np.int32), accept=np.zeros(ns, np.int32),
                    S_start=np.zeros(max(n, 1), np.float32), S_final=np.zeros(max(n, 1), np.float32),
                    status=np.zeros(max(n, 1), np.int32))
        tr = dock_refine_trace_buf()
        tr.gstride = gstride
        for name, a in bufs.items():
            setattr(tr, name, a.ctypes.data)
        xin = np.ascontiguousarray(xyz_in, np.float32)
        out = np.zeros(n, RESULT_DTYPE)
        xyz_out = np.zeros((natoms, 3), np.float32)
        k = knobs_struct(kn)
        rc = lib.dock_refine_trace(self._c, bid, pid, ctypes.byref(k), ctypes.c_void_p(xin.ctypes.data),
                                   ctypes.byref(tr), ctypes.c_void_p(out.ctypes.data),
                                   ctypes.c_void_p(xyz_out.ctypes.data))
        self._check(rc, "dock_refine_trace")
        res = {k2: (v[:n * steps] if v.shape[0] == ns and k2 not in ("S_start", "S_final", "status") else v[:n])
               for k2, v in bufs.items() if k2 != "G"}
        res["G"] = bufs["G"][:n * steps * gstride].reshape(n, steps, gstride)
        res["gstride"] = gstride
        res["result"] = out
        res["xyz"] = xyz_out
        return res
