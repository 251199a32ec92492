"""Independent restatements used to pin the oracle (test infrastructure).

Built from library routines rather than the oracle's own code: scipy's
rotation-vector rotations, csgraph shortest paths and connected components,
and numpy indexing. They are deliberately naive (all atom pairs at graph
distance >= 3 for the clash test) so that a restricted or reordered
computation in the oracle is checked against the plain definition.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components, shortest_path
from scipy.spatial.transform import Rotation


def ligand(batch, b):
    a0, a1 = batch.atom_off[b], batch.atom_off[b + 1]
    x = batch.xyz[a0:a1].astype(np.float64)
    bonds = batch.bonds[batch.bond_off[b]:batch.bond_off[b + 1]]
    rot = batch.rot[batch.rot_off[b]:batch.rot_off[b + 1]]
    return x, bonds, rot


def graph_distance(l, bonds):
    A = csr_matrix((np.ones(len(bonds)), (bonds[:, 0], bonds[:, 1])), shape=(l, l))
    return shortest_path(A, directed=False, unweighted=True)


def sides(l, bonds, rot):
    """(moving mask, c, b) for the left then right fragment of every rotatable bond."""
    out = []
    for r in rot:
        keep = np.ones(len(bonds), bool)
        keep[r] = False
        e = bonds[keep]
        A = csr_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(l, l))
        _, lab = connected_components(A, directed=False)
        u, v = sorted(bonds[r])
        left = lab == lab[u]
        out.append((left, u, v))
        out.append((~left, v, u))
    return out


def rotate_side(x, moving, c, b, theta):
    k = x[c] - x[b]
    k = k / np.linalg.norm(k)
    y = x.copy()
    rot = Rotation.from_rotvec(k * theta)
    y[moving] = rot.apply(x[moving] - x[c]) + x[c]
    return y


def nearest_S(K, origin, h, x, clip=True):
    """Sum of field values at the nearest voxels; (S, inside)."""
    t = (x - origin) / h
    v = np.floor(t + 0.5).astype(np.int64)
    nz, ny, nx = K.shape
    n = np.array([nx, ny, nz])
    inside = bool(np.all((v >= 0) & (v < n)))
    vc = np.clip(v, 0, n - 1)
    S = float(K[vc[:, 2], vc[:, 1], vc[:, 0]].astype(np.float64).sum())
    return S, inside


def clashes(x, gdist, thr):
    """True if any atom pair at graph distance >= 3 is closer than thr."""
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    mask = gdist >= 3
    return bool(np.any(d2[mask] < thr * thr))
