"""Builds and saves the deformed-sphere FEM plan that ``tests/test_gpu_c3.py`` reads.

    python tests/c3_plan.py OUT.plan [EIG_DIR]

Icosphere level 6 with radius 1 + 0.2 h / max|h| (``workloads.deformed_icosphere``), P1
cotangent stiffness and lumped mass, the 4096 lowest generalized eigenpairs by the oracle's
spectral slicing (``oracle.fem.laplace_beltrami_basis``; about half an hour on eight cores;
cached as .npy files in EIG_DIR when given), then the library's host build (eps = 1e-6,
leaf 128, Algorithm 2's patch rule on the mesh, lumped-mass weights) and ``Plan.save``.
Test infrastructure: the eigenpairs are the oracle's, the plan the library's.
"""
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as W  # noqa: E402
from oracle import fem  # noqa: E402


def main(out: str, eig_dir: str | None = None) -> None:
    V, F = W.deformed_icosphere(6)
    files = [os.path.join(eig_dir, f) for f in ("c3_lam.npy", "c3_phi.npy", "c3_md.npy")] if eig_dir else []
    if files and all(os.path.exists(f) for f in files):
        lam, Phi, Md = (np.load(f) for f in files)
    else:
        t = time.time()
        lam, Phi, Md, _ = fem.laplace_beltrami_basis(V, F, 4096)
        print(f"eigenpairs {time.time() - t:.0f} s", flush=True)
        if files:
            for f, a in zip(files, (lam, Phi, Md)):
                np.save(f, a)
    from paper_2605_21828_gb300 import Plan
    t = time.time()
    plan = Plan.build(n=len(V), m=Phi.shape[1], eigenvalues=lam, evaluator="dense", dense=Phi, points=V, tris=F,
                      eps=1e-6, leaf_size=128, tree="mesh", weights=Md)
    info = plan.info()
    print(f"plan {time.time() - t:.0f} s: stored entries {info['stored_entries']}, max rank {info['max_rank']}, "
          f"levels {info['levels']}", flush=True)
    plan.save(out)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2] if len(sys.argv) > 2 else None)
