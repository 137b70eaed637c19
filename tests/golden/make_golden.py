"""Write the stored oracle results under tests/golden/ (calls only the oracle).

The paper prints no worked example (its results are performance figures), so these
fixtures are regression anchors produced by the oracle from the seeded generator:
the SU(3) Landau workload of an 8^4 lattice, eps = 0.4, field seed 1, gauge seed 2,
overrelaxation omega = 1.7 until theta < 1e-12 or 500 sweeps, reunitarisation every
20 sweeps (the run settings of Section 3 with the overrelaxation parameter 1.7), and
its Coulomb counterpart on 8^3 x 8 with per-slice stop rule.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1412_1498_gb300 import fields  # noqa: E402


def run(gauge, name):
    U = fields.random_gauge_config((8, 8, 8, 8), 0.4, 1, 2)
    F0, th0, _, _ = oracle.measure(U, gauge)
    r = oracle.fix(U, 1e-12, 500, 1.7, gauge=gauge, reunit_interval=20)
    out = dict(
        workload=f"SU(3) {name}, 8^4, eps=0.4, seeds 1/2, omega=1.7, theta<1e-12 or 500 sweeps, reunit every 20",
        citation="Algorithm 1 and Eqs. (1)-(6); run settings Section 3",
        F0=F0, theta0=th0, rc=r["rc"], iters=r["iters"], F=r["F"], theta=r["theta"],
        theta_every_10=[float(x) for x in r["theta_hist"][::10]],
        slice_iters=[int(x) for x in r["slice_iters"]],
    )
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name.lower()}_8x4_seed1_2.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, r["iters"], r["F"], r["theta"])


if __name__ == "__main__":
    run(oracle.LANDAU, "Landau")
    run(oracle.COULOMB, "Coulomb")
