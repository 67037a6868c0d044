"""Writes cdr2d500_record.json: the oracle's full SIM-M run (Sec. 3.5, with the
multiplicity step of Sec. 3.4) on the 2-D convection–diffusion–reaction
workload at n = 250,000 — squares per level, shifts, cluster estimates and
multiplicities.  Calls only the oracle and the seeded workload generators.

    python tests/golden/make_cdr2d_record.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import simm as S  # noqa: E402
from workloads import config_cdr2d  # noqa: E402


def main():
    w = config_cdr2d()
    t0 = time.time()
    r = S.sim_m(w.A.to_scipy(), None, w.region, w.f, S.Options(**w.options))
    out = dict(
        workload=w.name,
        region=list(w.region),
        options=w.options,
        expected_count=w.expected_count,
        level_counts=[int(c) for c in r.level_counts],
        num_shifts=len(r.shifts),
        estimate_re=[float(x) for x in r.eigenvalues.real],
        estimate_im=[float(x) for x in r.eigenvalues.imag],
        multiplicity=[int(x) for x in r.multiplicities],
        inner_solves=int(r.n_inner_solves),
        oracle_seconds=round(time.time() - t0, 1),
    )
    with open(os.path.join(HERE, "cdr2d500_record.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("eigenvalues", len(out["estimate_re"]), "shifts", out["num_shifts"], "%.1fs" % out["oracle_seconds"])


if __name__ == "__main__":
    main()
