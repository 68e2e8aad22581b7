"""Writes the oracle's summaries of the 8^3-hex Kuhn cube (3072 tets): the
assembly to cube8_oracle.json, the stabilised velocity block to
cube8_stab_oracle.json.

Calls only the FP64 oracle and the seeded input generator.  The paper prints
no element values, so these numbers are the oracle's own (pinned by
tests/test_oracle_pins.py); they guard the oracle against silent drift.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import meshgen  # noqa: E402
import oracle  # noqa: E402


def summary():
    mesh, u = meshgen.config_mesh("cube8")
    rp, ci, A, G, rhs = oracle.assemble(mesh.coord, mesh.lnods, u, rho=meshgen.RHO, mu=meshgen.MU,
                                        dt=meshgen.DT)
    pick = [0, 1, 17, 4000, 9096]
    return {
        "workload": "Kuhn cube 8^3 hexes, 3072 tets, 729 nodes, natural numbering, seed 0",
        "rho": meshgen.RHO, "mu": meshgen.MU, "dt": meshgen.DT,
        "nnz": int(rp[-1]),
        "row_ptr_sum": int(rp.astype(np.int64).sum()),
        "col_idx_sum": int(ci.astype(np.int64).sum()),
        "A_sum": float(A.sum()), "A_abs_sum": float(np.abs(A).sum()),
        "G_sum": [float(x) for x in G.sum(axis=1)],
        "G_abs_sum": [float(x) for x in np.abs(G).sum(axis=1)],
        "rhs_sum": [float(x) for x in rhs.sum(axis=1)],
        "rhs_abs_sum": [float(x) for x in np.abs(rhs).sum(axis=1)],
        "A_at": {str(p): float(A[p]) for p in pick},
        "G_at": {str(p): [float(G[d, p]) for d in range(3)] for p in pick},
    }


def stab_summary():
    mesh, u = meshgen.config_mesh("cube8")
    rp, ci, Auu, G, rhs = oracle.assemble_stabilized(mesh.coord, mesh.lnods, u, rho=meshgen.RHO, mu=meshgen.MU,
                                                     dt=meshgen.DT)
    pick = [0, 1, 17, 4000, 9096]
    X, U = mesh.coord[mesh.lnods[0]], u[mesh.lnods[0]]
    t1, t2 = oracle.tau(X, U, meshgen.RHO, meshgen.MU)
    return {
        "workload": "Kuhn cube 8^3 hexes, 3072 tets, 729 nodes, natural numbering, seed 0: stabilised velocity block",
        "rho": meshgen.RHO, "mu": meshgen.MU, "dt": meshgen.DT,
        "nnz": int(rp[-1]),
        "Auu_sum": [float(x) for x in Auu.sum(axis=1)],
        "Auu_abs_sum": [float(x) for x in np.abs(Auu).sum(axis=1)],
        "Auu_at": {str(p): [float(Auu[c, p]) for c in range(9)] for p in pick},
        "tau_element0": [t1, t2],
    }


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    for name, fn in (("cube8_oracle.json", summary), ("cube8_stab_oracle.json", stab_summary)):
        out = os.path.join(here, name)
        with open(out, "w") as f:
            json.dump(fn(), f, indent=1)
        print("wrote", out)
