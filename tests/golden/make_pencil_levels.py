"""Writes pencil40064_levels.json: the oracle's location phase (Sec. 3.5 steps
1-6, no multiplicity) on the 40,064-row generalized pencil — squares evaluated
per level, shifts built, final squares, unresolvable final squares, and the
cluster estimates and sizes.  Calls only the oracle and the seeded workload
generators.

    python tests/golden/make_pencil_levels.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import simm as S  # noqa: E402
from workloads import config_pencil  # noqa: E402


def main():
    w = config_pencil()
    t0 = time.time()
    sm = S.SimM(w.A.to_scipy(), w.B.to_scipy(), S.Options(**w.options))
    sm.set_region(w.region, w.f)
    fix, fiy, fsid, fflag, s = sm.solve_levels()
    cl = sm.merge()
    out = dict(
        workload=w.name,
        region=list(w.region),
        options=w.options,
        level_counts=[int(c) for c in sm.level_counts],
        num_shifts=len(sm.spaces),
        final_squares=int(fix.size),
        unresolvable_final=int(np.sum(fflag)),
        clusters=int(cl["estimate"].size),
        estimate_re=[float(x) for x in cl["estimate"].real],
        estimate_im=[float(x) for x in cl["estimate"].imag],
        size=[int(x) for x in cl["size"]],
        oracle_seconds=round(time.time() - t0, 1),
    )
    with open(os.path.join(HERE, "pencil40064_levels.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("levels", out["level_counts"], "shifts", out["num_shifts"], "clusters", out["clusters"],
          "unresolvable", out["unresolvable_final"], "%.1fs" % out["oracle_seconds"])


if __name__ == "__main__":
    main()
