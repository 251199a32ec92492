"""The five workloads of the batched pose-evaluation path, as seeded recipes.

Each recipe returns plain inputs: a list of synth.Pocket, one
synth.LigandBatch and a knob dict. Sizes follow the paper's screening set
(Sec. 4.1: 28-153 atoms, 2-53 rotamers) scaled to the ranges below.

knob keys: hp_step, lp_step (degrees), threshold (relative fragment size),
repetitions, n_poses, enable_refinement, clip_box, bump_thr (Å), score_mode
(0 nearest, 1 trilinear), refine_steps, seed.
"""
from __future__ import annotations

import numpy as np

from . import ligand_batch, ligand_sizes, pocket, semi_axes

ELLIPSOID = (8.0, 6.0, 5.0)


def knobs(**kw):
    k = dict(hp_step=10.0, lp_step=10.0, threshold=0.0, repetitions=1, n_poses=8, enable_refinement=0,
             clip_box=1, bump_thr=2.0, score_mode=0, refine_steps=0, seed=0)
    k.update(kw)
    return k


def single(l=24, t=4, seed=0, n_grid=48, abc=ELLIPSOID, **kw):
    """One ligand x one pocket (24 atoms, 4 rotatable bonds, 48^3 grid, 8 poses, 10 degrees)."""
    pk = pocket(seed + 7, n_grid, 0.5, abc)
    b = ligand_batch(seed, np.array([l]), np.array([t]))
    return [pk], b, knobs(n_poses=8, hp_step=10.0, lp_step=10.0, repetitions=1, seed=seed, **kw)


def batched(n=1024, seed=1, n_grid=64, **kw):
    """1,024 ligands (16-64 atoms, 2-12 rotatable bonds) x one 64^3 pocket; 64 poses, 10 degrees, 4 repetitions."""
    pk = pocket(seed + 7, n_grid, 0.5, ELLIPSOID)
    l, t = ligand_sizes(seed, n, 0, [16, 64, 2, 12])
    b = ligand_batch(seed, l, t)
    k = dict(n_poses=64, hp_step=10.0, lp_step=10.0, repetitions=4, seed=seed)
    k.update(kw)
    return [pk], b, knobs(**k)


LOGNORMAL = [32.0, 0.4, 10, 80, 6.0, 15]


def sweep_batch(n=100_000, seed=3, id0=0):
    """Ligands with lognormal atom counts (median 32, clipped 10-80) and Poisson(6) rotatable bonds (<= 15)."""
    l, t = ligand_sizes(seed, n, 1, LOGNORMAL, id0=id0)
    return ligand_batch(seed, l, t, id0=id0)


SWEEP_STEPS = (5.0, 10.0, 20.0, 30.0, 45.0)
SWEEP_POSES = (8, 32, 128)
SWEEP_REPS = (1, 4, 16)


def knob_sweep(n=100_000, seed=3):
    """Knob sweep: 100,000 lognormal ligands x the 64^3 pocket, 45 (step, poses, repetitions) combinations."""
    pk = pocket(1 + 7, 64, 0.5, ELLIPSOID)
    b = sweep_batch(n, seed)
    combos = [knobs(hp_step=s, lp_step=s, n_poses=p, repetitions=r, seed=seed)
              for s in SWEEP_STEPS for p in SWEEP_POSES for r in SWEEP_REPS]
    return [pk], b, combos


def differentiation(n=4096, seed=4):
    """4,096 ligands (20-60 atoms, 3-10 rotatable bonds) x a 64^3 trilinear field; 20 refinement steps."""
    pk = pocket(1 + 7, 64, 0.5, ELLIPSOID)
    l, t = ligand_sizes(seed, n, 0, [20, 60, 3, 10])
    b = ligand_batch(seed, l, t)
    return [pk], b, knobs(n_poses=64, hp_step=10.0, lp_step=10.0, repetitions=4, score_mode=1,
                          refine_steps=20, seed=seed)


MULTI_SIDES = (48, 48, 48, 48, 64, 64, 64, 64, 96, 96, 96, 96, 128, 128, 128, 128)


def multi_pocket_pockets(seed=5):
    pks = []
    for i, n in enumerate(MULTI_SIDES):
        abc = semi_axes(seed, i, 5.0, 12.0)
        cap = n * 0.5 / 2.0 - 2.0  # keep the cavity 2 Å inside the box
        abc = np.minimum(abc, cap)
        pks.append(pocket(seed * 1000 + i, n, 0.5, abc))
    return pks


def multi_pocket(n=50_000, seed=5):
    """16 pockets (semi-axes 5-12 Å, 48^3-128^3 grids) x 50,000 lognormal ligands; 32 poses, 15 degrees, 2 reps."""
    return multi_pocket_pockets(seed), sweep_batch(n, seed), knobs(n_poses=32, hp_step=15.0, lp_step=15.0,
                                                                   repetitions=2, seed=seed)
