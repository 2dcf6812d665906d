"""Writes tests/golden/oracle_tiny.json from the FP64 oracle only.

The paper prints no worked example beyond iteration counts (Sec. 4: 3 for
PP-PC with the multi-harmonic coarse solve, 5 for the fixed-point iteration,
19 for PP-IC, to a tolerance below 1e-6 on its own coax model, whose geometry
and materials it does not give).  Those counts are stored here as context.
The numeric values are the oracle's on the seeded tiny coax case, frozen so
that a later change to the oracle's arithmetic shows up as a failing
comparison (tests/test_golden.py) and must be justified.

Run from the repository root:  python tests/golden/make_golden.py
"""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.adjoint import loss_gradient  # noqa: E402
from oracle.fem import FEModel  # noqa: E402
from oracle.periodic import bruteforce_periodic  # noqa: E402
from oracle.pppc import ppic, pppc  # noqa: E402
from synth import REGION_SHEATH, workload  # noqa: E402


def main():
    prob = workload("tiny")
    m = FEModel(prob)
    traj = bruteforce_periodic(m, prob.N, prob.n_fine, prob.T, tol=1e-12, max_newton=80)
    P, grad = loss_gradient(m, traj, prob.T, REGION_SHEATH)
    a = pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-11, kmax=60)
    b = ppic(m, prob.N, prob.n_fine, prob.T, tol=1e-11, kmax=200)
    out = {
        "case": "synth.workload('tiny'): coax 5x8 mesh (33 unknowns), N=4, 3 fine steps, sheath sigma 5e6, "
                "Brauer steel with |B| cap 3 T, 10 A 50 Hz",
        "paper_iteration_counts_context_only": {
            "source": "Sec. 4 (its own coax model, tolerance < 1e-6)",
            "pppc_multiharmonic": 3, "fixed_point": 5, "ppic": 19},
        "periodic_solution": {
            "source": "oracle.periodic.bruteforce_periodic (Newton on all L levels with u^0 = u^L)",
            "norm_u_levels": float(np.linalg.norm(traj)),
            "u0_first_entries": [float(v) for v in traj[0, :4]]},
        "eddy_loss_and_gradient": {
            "source": "oracle.adjoint.loss_gradient (periodic adjoint), region = sheath",
            "loss_w_per_m": P, "grad_sigma_k1_k2_k3": [float(g) for g in grad]},
        "iterations_to_1e-11": {
            "source": "oracle.pppc.pppc (Eq. 4, multi-harmonic coarse solve) and oracle.pppc.ppic (Eq. 5)",
            "pppc": a.iterations, "ppic": b.iterations},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
