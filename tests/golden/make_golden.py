"""Write stored expected values for the GPU parity tests by running the FP64 oracle.

Only ``oracle/`` and the seeded input generators are called; nothing here touches
the CUDA library.  Each output JSON records the workload recipe it was made from.

    python tests/golden/make_golden.py inclusions128     # 3D 128^3 inclusion cell, ~1.5 h of CPU

Workload 'inclusions128': 3D 128^3 compressible neo-Hookean matrix (mu = 1) with
periodic spherical inclusions (mu = 10) of radius 6 voxels, seeded centres, 20 %
volume fraction, nu = 0.3 in both phases; Fbar = diag(0.9, 1, 1) (uniaxial
compression), rho = 10 fixed, tolerance 1e-8 on r_p and r_d (Section 2.1, eq.
check), Lambda_0 = W_F(Fbar).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2010_06697_gb300 import synth  # noqa: E402

WORKLOADS = {
    "inclusions128": dict(n=128, dim=3, kind="inclusion", seed=0, mu=(1.0, 10.0), nu=0.3,
                          Fbar=[[0.9, 0, 0], [0, 1, 0], [0, 0, 1]], rho=10.0, tol=1e-8, max_iter=1000),
}


def run(name):
    w = WORKLOADS[name]
    if w["kind"] == "inclusion":
        ph = synth.inclusion_phase(w["n"], w["dim"], w["seed"])
    else:
        ph = synth.laminate_phase(w["n"], w["dim"])
    par = synth.two_phase_params(w["mu"][0], w["mu"][1], w["nu"])
    t0 = time.time()
    r = oracle.admm_solve(ph, par, np.array(w["Fbar"], float), w["rho"], w["tol"], w["max_iter"])
    out = {
        "workload": name, "recipe": w,
        "source": "oracle.admm_solve (FP64 numpy), Section 2.1 Steps 1-4 with the Section 2.3 symbols",
        "phase_fraction": float(ph.mean()),
        "mu_ref": r["mu_ref"], "iters": r["iters"], "converged": r["converged"],
        "stress": r["stress"].tolist(),
        "history": [list(h) for h in r["history"]],
        "oracle_seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, r["iters"], r["converged"], r["stress"].tolist())


if __name__ == "__main__":
    for n in sys.argv[1:]:
        run(n)
