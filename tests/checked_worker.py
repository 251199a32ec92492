"""Docking cases run by both the library and its checked build (test infrastructure): the parity workloads'
shapes at small sizes, every entry point that launches kernels. `python tests/checked_worker.py OUT.npz` runs
them with whichever library the binding loads and saves the results."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def run_cases():
    import torch

    import synth
    import synth.configs as C
    from paper_1901_06363_gb300 import Docker

    out = {}
    dk = Docker(0)
    pk = synth.pocket(13, 64, 0.5, (6, 5, 4))
    pid = dk.init_pocket(pk)
    l, t = synth.ligand_sizes(13, 12, 0, [16, 64, 0, 10])
    b = synth.ligand_batch(13, l, t)
    natoms = int(b.atom_off[-1])
    bid = dk.upload_ligands(b)
    base = C.knobs(n_poses=12, hp_step=15.0, lp_step=15.0, repetitions=2, seed=3)
    variants = {"base": {}, "threshold": dict(threshold=0.5, lp_step=45.0, hp_step=10.0),
                "noclip": dict(clip_box=0), "peel": dict(enable_refinement=1, hp_step=5.0, lp_step=30.0, threshold=0.3),
                "trilinear": dict(score_mode=1), "exact": dict(score_mode=2), "plain": dict(plain_mode=1)}
    for name, kw in variants.items():
        res, xyz = dk.run(bid, [pid], dict(base, **kw), b.n, natoms)
        out["run_" + name] = res.view(np.int32).copy()
        out["xyz_" + name] = xyz.copy()
    g = dk.run_trace(bid, pid, base, b)
    out["trace_chosen"] = g["chosen_k"]
    out["trace_S"] = g["cand_S"]
    db, _ = dk.run_database(b, [pid], base, chunk=5)
    out["database"] = db.view(np.int32).copy()
    # refinement and the differentiable score from the docked poses
    kr = dict(base, refine_steps=8)
    x = torch.tensor(out["xyz_base"], dtype=torch.float32, device="cuda").reshape(-1)
    r, rx = dk.refine(bid, [pid], kr, x)
    out["refine"] = r.cpu().numpy()
    out["refine_xyz"] = rx.cpu().numpy()
    out["score"] = dk.score_trilinear(bid, pid, x).cpu().numpy()
    out["score_grad"] = dk.score_trilinear_grad(bid, pid, x).cpu().numpy()
    n, _, _, tmax = dk.batch_info(bid)
    q = torch.full((n, 6 + tmax), 0.1, dtype=torch.float32, device="cuda")
    out["dof_apply"] = dk.dof_apply(bid, x, q).cpu().numpy()
    out["dof_grad"] = dk.dof_grad(bid, x, q, torch.ones_like(x)).cpu().numpy()
    dk.release_batch(bid)
    dk.close()
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run_cases())
