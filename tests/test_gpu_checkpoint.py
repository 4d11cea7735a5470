"""GPU tests of checkpoint / resume (combo_state_export / combo_state_import)
and of the unit-level material entry points (combo_neohooke_eval,
combo_laminate_eval) against the FP64 oracle.

Resume: a solve run for k load steps, exported, imported into a fresh solve of
the same problem and options and finished must equal the uninterrupted solve
bit for bit (the same launch shapes: the autotuner's decision for the grid is
taken by the first solve and reused).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cb():
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    return combo


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


CASES = [dict(solver=1, precision=2), dict(solver=1, precision=0, theory=1),
         dict(solver=2, precision=0, kspace=3), dict(solver=0, precision=2, kspace=2)]


@pytest.mark.parametrize("o", CASES)
def test_resume_is_bitwise(cb, o):
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.centred_sphere((16, 16, 16), 0.2, 10.0, np.diag([1.06, 1.0, 0.98]), 4)
    full = cb.solve(p, tol=1e-8, **o)
    s1 = cb.Solve(p, tol=1e-8, **o)
    assert s1.advance_steps(2) is False
    blob = s1.export_state()
    s1.close()
    s2 = cb.Solve(p, tol=1e-8, **o)
    s2.import_state(blob)
    assert s2.advance(0) is True
    r = s2.finish()
    s2.close()
    assert np.array_equal(r["Pbar"], full["Pbar"])
    assert np.array_equal(r["F"], full["F"])
    assert np.array_equal(r["Pbar_phase"], full["Pbar_phase"])
    assert list(r["iters"]) == list(full["iters"])
    assert r["n_operator"] == full["n_operator"]
    if len(full["a"]):
        assert np.array_equal(r["a"], full["a"])


def test_checkpoint_misuse_is_rejected(cb):
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.centred_sphere((16, 16, 16), 0.2, 10.0, np.diag([1.06, 1.0, 0.98]), 4)
    q = ms.centred_sphere((16, 16, 16), 0.3, 10.0, np.diag([1.06, 1.0, 0.98]), 4)
    s = cb.Solve(p, tol=1e-8)
    s.advance_steps(1)
    blob = s.export_state()
    s.advance(3)  # stops inside a load step
    with pytest.raises(Exception):
        s.export_state()
    with pytest.raises(Exception):  # already advanced
        s.import_state(blob)
    s.close()
    t = cb.Solve(q, tol=1e-8)  # other boxel count
    with pytest.raises(Exception):
        t.import_state(blob)
    t.close()
    u = cb.Solve(p, tol=1e-8, solver=2)  # other options
    with pytest.raises(Exception):
        u.import_state(blob)
    u.close()
    w = cb.Solve(p, tol=1e-8)
    with pytest.raises(Exception):
        w.import_state(blob[:-8])
    w.import_state(blob)
    assert w.advance(0) is True
    w.close()


def test_unit_material_evaluations(cb, orc):
    rng = np.random.default_rng(12)
    for _ in range(6):
        F = (np.eye(3) + 0.2 * rng.uniform(-1, 1, (3, 3))).ravel()
        P, A = cb.neohooke_eval(F, 1.3, 2.1)
        Po, Ao = orc.neohooke(F, 1.3, 2.1)
        assert rel(P, Po) < 1e-13 and rel(A, Ao) < 1e-13
    with pytest.raises(Exception):
        cb.neohooke_eval(np.diag([1.0, 1.0, -1.0]).ravel(), 1.0, 2.0)
    mat = (1.0, 2.0, 10.0, 20.0)
    for k in range(6):
        N = rng.normal(size=3)
        N /= np.linalg.norm(N)
        c = 0.99625 if k == 0 else rng.uniform(0.05, 0.95)
        F = (np.eye(3) + 0.1 * rng.uniform(-1, 1, (3, 3))).ravel()
        g = cb.laminate_eval(F, N, c, mat)
        o = orc.laminate(F, N, c, mat)
        assert rel(g["P"], o["P"]) < 1e-12
        assert rel(g["A"], o["A"]) < 1e-10
        assert rel(g["a"], o["a"]) < 1e-9
        assert abs(g["iters"] - o["iters"]) <= 1
