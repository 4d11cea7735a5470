"""Launch-shape autotuner: the first solve of a grid records a decision for
each FP32 Krylov pass, and every candidate shape of every pass gives the
result of the FP64 form (which the parity tests pin to the oracle)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cb():
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    yield combo
    for k in range(4):
        combo.autotune_force(k, -1)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def problem(n, seed):
    from paper_2204_13624_gb300 import microstructure as ms

    return ms.random_spheres(n, 5.0, 0.15, seed, 10.0, np.diag([1.03, 1.0, 1.0]) + 0.01, 1)


def test_first_solve_records_a_decision(cb):
    p = problem((64, 64, 128), 21)
    cb.solve(p, precision=cb.FP32_REFINED_DF, fixed_iterations=1, cg_fixed_iterations=2, fields=False)
    rep = cb.autotune_report()
    line = [l for l in rep.splitlines() if l.startswith("64x64x128 x1 FP32")]
    assert len(line) == 1
    for name in ("x-forward=", "y=", "z=", "x-inverse="):
        assert name in line[0]


@pytest.mark.parametrize("n", [(256, 128, 64), (128, 64, 256)])
def test_every_candidate_matches_the_fp64_form(cb, n):
    p = problem(n, 31)
    opts = dict(fixed_iterations=1, cg_fixed_iterations=10)
    ref = cb.solve(p, precision=cb.FP64, **opts)
    for k in range(4):
        for cand in (0, 1):
            cb.autotune_force(k, cand)
            g = cb.solve(p, precision=cb.FP32_REFINED_DF, **opts)
            cb.autotune_force(k, -1)
            assert rel(g["F"], ref["F"]) < 2e-5, (k, cand)
            assert rel(g["Pbar"], ref["Pbar"]) < 2e-5, (k, cand)
