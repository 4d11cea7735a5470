"""The per-solve JSON record (host-side formatting; no GPU): fields and types
from a result dict of the shape combo.solve() returns."""
import json

import numpy as np


def test_solve_record_fields():
    from paper_2204_13624_gb300 import build, combo
    from paper_2204_13624_gb300 import microstructure as ms

    build.build()
    p = ms.centred_sphere((16, 8, 12), 0.2, 10.0, np.diag([1.05, 1.0, 1.0]), 2)
    result = dict(steps_done=2, iters=np.array([4, 3], np.int32), cg_iters=np.array([60, 52], np.int32),
                  resid=np.array([3e-9, 5e-9]), Pbar=np.arange(18.0).reshape(2, 9), nr_iters=17, n_backproj=2,
                  n_laminate_evals=40, n_operator=120)
    line = combo.solve_record(p, result, seconds=0.25, solver=combo.NEWTON_CG, kspace=combo.STAGGERED)
    assert "\n" not in line
    rec = json.loads(line)
    assert rec["grid"] == [16, 8, 12] and rec["voxels"] == 16 * 8 * 12
    assert rec["boxels"] == len(p["boxel_idx"]) > 0
    assert rec["solver"] == combo.NEWTON_CG and rec["kspace"] == combo.STAGGERED and rec["theory"] == 0
    assert rec["outer_iterations"] == [4, 3] and rec["cg_iterations"] == [60, 52]
    assert rec["Pbar"][1][8] == 17.0 and rec["residuals"] == [3e-9, 5e-9]
    assert rec["operator_applications"] == 120 and rec["back_projections"] == 2 and rec["seconds"] == 0.25
    # F (9 FP64 fields) and the half spectrum (9 complex FP64 per x-frequency, pitch rounded up to 4)
    assert rec["resident_field_bytes"] == 8 * 9 * 1536 + 16 * 9 * 12 * 8 * 12
