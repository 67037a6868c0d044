"""Writes batch_p12_record.json: the oracle's location phase (Sec. 3.5 steps
1-6) on pencil 12 of the 64-pencil batch workload (122x122 grid, Péclet 0.94,
194 eigenvalues), with new shifts at the levels (option
new_shifts_in_levels): without them a square left unresolvable at level 4
multiplies fourfold per level.  Calls only the oracle and the seeded workload
generators.

    python tests/golden/make_batch_p12_record.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import simm as S  # noqa: E402
from workloads.configs import config_batch  # noqa: E402

PENCIL = 12


def main():
    w = config_batch(64).pencils[PENCIL]
    t0 = time.time()
    sm = S.SimM(w.A.to_scipy(), None, S.Options(new_shifts_in_levels=1, **w.options))
    sm.set_region(w.region, w.f)
    init_shifts = len(sm.spaces)
    fix, fiy, fsid, fflag, s = sm.solve_levels()
    cl = sm.merge()
    out = dict(
        workload=w.name, pencil=PENCIL, region=list(w.region), options=dict(new_shifts_in_levels=1, **w.options),
        level_counts=[int(c) for c in sm.level_counts], initial_shifts=init_shifts, num_shifts=len(sm.spaces),
        final_squares=int(fix.size), unresolvable_final=int(fflag.sum()),
        estimate_re=[float(x) for x in cl["estimate"].real], estimate_im=[float(x) for x in cl["estimate"].imag],
        expected_count=w.expected_count, oracle_seconds=round(time.time() - t0, 1),
    )
    with open(os.path.join(HERE, "batch_p12_record.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("shifts", init_shifts, "->", out["num_shifts"], "clusters", len(out["estimate_re"]), "of",
          w.expected_count, "%.1fs" % out["oracle_seconds"])


if __name__ == "__main__":
    main()
