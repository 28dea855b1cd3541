"""Writes cube16_trajectory.txt: the float64 oracle's coloured CC trajectory on
the 16x16x16-cell jittered stretch cube (4 913 vertices, 24 576 tets; x = 0
face clamped, x = 1 face pulled to 1.5, 5% jitter, seed 0; stable Neo-Hookean,
nu = 0.3; 2-ring rest bases), 50 sweeps from the linear initial guess, for
E = 1e4 and E = 1e7: the energy and the free gradient norm after every sweep
and the final positions of 256 sampled vertices.  It calls only the oracle
(and the seeded input generator), so the stored values are the oracle's.

Run from the repository root:  python tests/golden/make_cube16_trajectory.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import meshgen  # noqa: E402
from oracle import fem, solvers, subspace, topology  # noqa: E402

SWEEPS = 50
E_VALUES = (1e4, 1e7)
SAMPLE_SEED = 16


def scene(E):
    return meshgen.stretch_box(16, 16, 16, E=E, nu=0.3, factor=1.5, jitter_amount=0.05, seed=0)


def sample_vertices(sc):
    free = np.flatnonzero(sc.pinned == 0)
    pick = (meshgen.uniform01(SAMPLE_SEED, np.arange(256)) * len(free)).astype(np.int64)
    return free[pick]


def main():
    out = ["# " + __doc__.strip().splitlines()[0], f"# sweeps {SWEEPS}"]
    for E in E_VALUES:
        sc = scene(E)
        pb = fem.problem_from_scene(sc)
        topo = topology.Topology(pb.n, pb.tets, pb.free)
        sup, U = subspace.build_local_bases(pb, topo, 2)
        x, hist = solvers.solve(pb, topo, sup, U, sc.x0, kind="cc", schedule="colored", tol=0.0,
                                max_iters=SWEEPS)
        assert hist.iterations == SWEEPS
        out.append(f"E {E:.17g}")
        out.append("energy " + " ".join(f"{v:.17g}" for v in hist.energy))
        out.append("gnorm " + " ".join(f"{v:.17g}" for v in hist.grad_norm))
        vs = sample_vertices(sc)
        out.append("sample " + " ".join(str(int(v)) for v in vs))
        out.append("x " + " ".join(f"{v:.17g}" for v in x[vs].ravel()))
        print(f"E={E:g}: rel residual after {SWEEPS} sweeps {hist.grad_norm[-1] / hist.grad_norm[0]:.3e}", flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "cube16_trajectory.txt"), "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
