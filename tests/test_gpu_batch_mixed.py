"""Batches over several grids (combo_solve_batch with unequal grids): the
problems of each grid form one stacked class, and every pass of every
operator application is one grouped launch over the work items of all
classes.  Each result must equal the oracle element by element (FP64 after
equal iterations: fields <= 1e-10, Pbar <= 1e-9) and its own single solve
(converged: FP64 Pbar <= 1e-9; refined forms at their stated tolerance, Pbar
<= 1e-5, F <= 1e-4: the Krylov iterations of another launch shape round
differently), and the oracle's converged state (refined: Pbar <= 1e-5, F <=
1e-4)."""
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


def mixed_problems(seed=0):
    """Grids covering the grouped kernels' bodies: 64^3 (compile-time x, y
    and z plans), 48 x 32 x 24 and 24 x 16 x 32 (generic plans, ragged), two
    problems on 16^3 (a stacked class), random boxels on 12 x 18 x 24;
    different contrasts, loads and load-step counts."""
    from paper_2204_13624_gb300 import microstructure as ms

    rng = np.random.default_rng(seed)

    def Fb():
        F = np.eye(3) + np.diag(rng.uniform(-0.04, 0.04, 3))
        F[0, 1] += rng.uniform(-0.04, 0.04)
        F[2, 1] += rng.uniform(-0.03, 0.03)
        return F

    return [
        ms.random_spheres((64, 64, 64), 6.0, 0.12, 11, 10.0, Fb(), 2),
        ms.random_spheres((48, 32, 24), 4.0, 0.1, 12, 20.0, Fb(), 1),
        ms.random_spheres((16, 16, 16), 3.0, 0.1, 13, 10.0, Fb(), 2),
        ms.random_boxels((12, 18, 24), seed=14, contrast=5.0, Fbar=Fb(), n_steps=1),
        ms.random_spheres((24, 16, 32), 3.5, 0.1, 15, 10.0, Fb(), 3),
        ms.random_spheres((16, 16, 16), 3.0, 0.12, 16, 30.0, Fb(), 1),
    ]


def test_mixed_batch_fp64_equal_iterations_against_oracle(cb, orc):
    probs = mixed_problems()
    out = cb.solve_batch(probs, precision=cb.FP64, solver=1, fixed_iterations=2, cg_fixed_iterations=8)
    for p, g in zip(probs, out):
        r = orc.solve(p, dict(solver=1, fixed_iter=2, cg_fixed_iter=8))
        assert g["steps_done"] == p["n_steps"]
        assert rel(g["F"], r["F"]) < 1e-10
        assert rel(g["P"], r["P"]) < 1e-10
        assert rel(g["Pbar"], r["Pbar"]) < 1e-9


def test_mixed_batch_fp64_converged_equals_single_solves(cb):
    probs = mixed_problems(1)
    alone = [cb.solve(p, precision=cb.FP64, tol=1e-8) for p in probs]
    out = cb.solve_batch(probs, precision=cb.FP64, tol=1e-8)
    for p, a, g in zip(probs, alone, out):
        assert g["steps_done"] == p["n_steps"] and np.all(g["resid"] <= 1e-8)
        assert np.array_equal(a["iters"], g["iters"])
        assert rel(g["Pbar"], a["Pbar"]) < 1e-9
        assert rel(g["Pbar_phase"], a["Pbar_phase"]) < 1e-8
        assert rel(g["F"], a["F"]) < 1e-8


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_batch_refined_against_single_solves_and_oracle(cb, orc, prec):
    probs = mixed_problems(2)
    alone = [cb.solve(p, precision=prec, tol=1e-8) for p in probs]
    out = cb.solve_batch(probs, precision=prec, tol=1e-8)
    for i, (p, a, g) in enumerate(zip(probs, alone, out)):
        assert g["steps_done"] == p["n_steps"] and np.all(g["resid"] <= 1e-8)
        # two tol-1e-8 solves whose Krylov iterations round differently (the
        # grouped bodies against the single solve's compile-time plans): the
        # stated refined tolerance
        assert rel(g["Pbar"], a["Pbar"]) < 1e-5
        assert rel(g["F"], a["F"]) < 1e-4
        if i in (1, 3):  # two of them against the converged oracle as well
            r = orc.solve(p, dict(solver=1, tol=1e-10, cg_tol=1e-4))
            assert rel(g["Pbar"], r["Pbar"]) < 1e-5
            assert rel(g["F"], r["F"]) < 1e-4


def test_mixed_batch_counts_and_errors(cb):
    from paper_2204_13624_gb300 import microstructure as ms

    probs = mixed_problems(3)[:3]
    out = cb.solve_batch(probs, precision=cb.FP32_REFINED_DF, tol=1e-8, fields=False)
    for p, g in zip(probs, out):
        assert g["n_operator"] > 0 and g["n_operator_fp64"] >= p["n_steps"]
    # a laminate failure in one problem names that problem
    with pytest.raises(cb.ComboError) as e:
        cb.solve_batch([ms.homogeneous((8, 8, 8)), ms.sphere_32(n_steps=1)], nr_max_iter=1)
    assert e.value.code == -4 and "problem 1" in str(e.value)


def test_large_class_runs_its_own_launches_beside_the_grouped_ones(cb):
    """A 192^3 problem fills the GPU on its own, so its class runs its own
    tuned launch sequences on a stream of its own while the small grids'
    classes share the grouped launches on another; every result still
    equals its single solve."""
    from paper_2204_13624_gb300 import microstructure as ms

    Fb = np.eye(3) + np.diag([0.03, -0.01, 0.0])
    probs = [ms.random_spheres((192, 192, 192), 9.0, 0.15, 21, 10.0, Fb, 2)] + mixed_problems(4)[1:4]
    for prec in (cb.FP64, cb.FP32_REFINED_DF):
        tol_pbar = 1e-9 if prec == cb.FP64 else 1e-5
        alone = [cb.solve(p, precision=prec, tol=1e-8, fields=True) for p in probs]
        out = cb.solve_batch(probs, precision=prec, tol=1e-8)
        for p, a, g in zip(probs, alone, out):
            assert g["steps_done"] == p["n_steps"] and np.all(g["resid"] <= 1e-8)
            assert rel(g["Pbar"], a["Pbar"]) < tol_pbar
            assert rel(g["F"], a["F"]) < 1e-4
