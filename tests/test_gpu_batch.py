"""Batched solves (combo_solve_batch): independent problems on one grid,
stacked along z and solved together, give each problem the result of its own
solve (which the parity tests pin to the oracle).  Batches over several
grids: test_gpu_batch_mixed.py."""
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def batch_problems(n, count, seed=0):
    """Different microstructures, contrasts, loads and step counts on one grid."""
    from paper_2204_13624_gb300 import microstructure as ms

    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        Fb = np.eye(3) + np.diag(rng.uniform(-0.04, 0.04, 3)) + 0.03 * (rng.uniform(-1, 1, (3, 3)))
        steps = 1 + i % 3
        if i % 4 == 3:
            p = ms.homogeneous(n)  # no boxels at all
            p["Fbar"] = Fb.reshape(9)
            p["n_steps"] = steps
        elif i % 4 == 2:
            p = ms.random_boxels(n, seed=300 + i, contrast=5.0 + i, Fbar=Fb, n_steps=steps)
        else:
            p = ms.random_spheres(n, max(3.0, min(n) / 6), 0.08 + 0.04 * (i % 2), 400 + i, 10.0 * (1 + i % 2), Fb,
                                  steps)
        out.append(p)
    return out


@pytest.mark.parametrize("n", [(16, 16, 16), (24, 16, 12)])
def test_batch_equals_individual_solves_fp64(cb, n):
    probs = batch_problems(n, 5)
    alone = [cb.solve(p, precision=cb.FP64, tol=1e-8) for p in probs]
    batch = cb.solve_batch(probs, precision=cb.FP64, tol=1e-8)
    for p, a, b in zip(probs, alone, batch):
        assert b["steps_done"] == p["n_steps"]
        assert np.array_equal(a["iters"], b["iters"])
        assert np.all(np.abs(a["cg_iters"] - b["cg_iters"]) <= 1)
        assert rel(b["Pbar"], a["Pbar"]) < 1e-9
        assert rel(b["Pbar_phase"], a["Pbar_phase"]) < 1e-8
        assert rel(b["F"], a["F"]) < 1e-8
        assert rel(b["P"], a["P"]) < 1e-8
        assert np.all(b["resid"] <= 1e-8)


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_refined_at_compile_time_sizes(cb, prec):
    """64^3 problems: the batch runs the TMA-tiled y/z-passes and the streamed
    x-inverse over stacked problems."""
    probs = batch_problems((64, 64, 64), 3, seed=1)
    alone = [cb.solve(p, precision=prec, tol=1e-8) for p in probs]
    batch = cb.solve_batch(probs, precision=prec, tol=1e-8)
    for p, a, b in zip(probs, alone, batch):
        assert b["steps_done"] == p["n_steps"] and np.all(b["resid"] <= 1e-8)
        assert rel(b["Pbar"], a["Pbar"]) < 1e-6
        assert rel(b["Pbar_phase"], a["Pbar_phase"]) < 1e-5
        assert rel(b["F"], a["F"]) < 1e-4


def test_batch_rejects_the_fixed_point(cb):
    from paper_2204_13624_gb300 import microstructure as ms

    a = ms.homogeneous((8, 8, 8))
    b = ms.homogeneous((8, 8, 16))
    for probs in ([a, a], [a, b]):
        with pytest.raises(cb.ComboError) as e:
            cb.solve_batch(probs, solver=0)
        assert e.value.code == -1
    one = cb.solve_batch([a], solver=0, fixed_iterations=1)
    assert len(one) == 1 and one[0]["steps_done"] == a["n_steps"]
