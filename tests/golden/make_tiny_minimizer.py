"""Write tests/golden/tiny_minimizer_<case>.json from oracle/ only.

Each fixture holds the minimiser of Eq. 5 + Eq. 6 for one 8 x 8 x 2 case of
tiny_problem.py, found by the dense ADMM of oracle/dense.py and confirmed by
the smoothed projected-gradient brute force of the same module (they must
agree to 1e-6).  Run:  python tests/golden/make_tiny_minimizer.py [case ...]
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, HERE)

from oracle import muffin_oracle as mo  # noqa: E402
from oracle import dense  # noqa: E402
from tiny_problem import tiny_inputs, CASES  # noqa: E402


def main():
    y, psf, _ = tiny_inputs()
    only = sys.argv[1:]
    for name, c in CASES.items():
        if only and name not in only:
            continue
        p = mo.make_problem(y, psf, c["J"], gen=c["gen"], mu_s=c["mu_s"], mu_l=c["mu_l"], tau=1.0,
                            dictionary=c.get("dictionary", "iuwt"))
        ops = dense.dense_operators(p)
        x_admm = dense.admm_minimize(p, 12000, 1.0, ops)
        x_pg = dense.smoothed_projected_gradient(p, ops)
        agree = float(np.linalg.norm(x_admm - x_pg) / np.linalg.norm(x_admm))
        print(name, "ADMM vs projected gradient rel diff", agree)
        assert agree < 1e-6, agree
        out = {
            "source": "oracle/dense.py admm_minimize (12000 passes, penalty 1), confirmed by "
                      "smoothed_projected_gradient; problem from tests/golden/tiny_problem.py",
            "case": c,
            "objective": dense.dense_objective(p, x_admm, ops),
            "pg_rel_diff": agree,
            "x": [float(v) for v in x_admm],
        }
        with open(os.path.join(HERE, f"tiny_minimizer_{name}.json"), "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
