"""GPU parity of infinitesimal-strain ComBo (COMBO_INFINITESIMAL_STRAIN: isotropic
linear phases, closed-form composite boxels) against the FP64 oracle, through
the C ABI.

Tolerances (max-abs error relative to the max-abs reference value): the law
of a field <= 1e-12 (closed forms on both sides, arranged differently);
equal iterations in FP64 <= 1e-10 in F and P, <= 1e-9 in Pbar, the same CG
counts; the refined forms converged to tol 1e-8: Pbar <= 1e-6 of the FP64
oracle's converged state (the refined-form bound of the finite-strain path).
"""
import numpy as np
import pytest

from test_gpu_parity import problems, rel

pytestmark = pytest.mark.gpu
SMALL = 1


@pytest.fixture(scope="module")
def cb():
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    return combo


def solve_both(cb, orc, p, **o):
    g = cb.solve(p, theory=SMALL, **o)
    om = dict(solver=o.get("solver", 1), kspace=o.get("kspace", 0), tol=o.get("tol", 1e-8),
              fixed_iter=o.get("fixed_iterations", 0), cg_fixed_iter=o.get("cg_fixed_iterations", 0),
              cg_tol=o.get("cg_tol", 1e-3), max_iter=o.get("max_iter", 200 if o.get("solver", 1) == 1 else 100000),
              theory=SMALL)
    return g, orc.solve(p, om)


@pytest.mark.parametrize("n", [(12, 9, 18), (16, 16, 16), (64, 32, 8)])
def test_law_parity(cb, orc, n):
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.random_boxels(n, seed=sum(n) + 1, boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
    V = n[0] * n[1] * n[2]
    F = np.eye(3).reshape(9, 1) + 0.3 * np.random.default_rng(V).uniform(-1, 1, (9, V))
    Pg, ag = cb.constitutive(p, F, theory=SMALL)
    Po, ao = orc.constitutive_field(p, F, opts=dict(theory=SMALL))
    assert rel(Pg, Po) < 1e-12
    assert rel(ag, ao) < 1e-12
    S = Pg.reshape(3, 3, V)
    assert np.abs(S - S.transpose(1, 0, 2)).max() < 1e-13 * np.abs(S).max()


@pytest.mark.parametrize("kspace", [0, 2])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_newton_cg_parity(cb, orc, k, kspace):
    p = problems()[k]
    g, r = solve_both(cb, orc, p, solver=1, kspace=kspace, fixed_iterations=2, cg_fixed_iterations=12)
    assert rel(g["F"], r["F"]) < 1e-10
    assert rel(g["P"], r["P"]) < 1e-10
    assert rel(g["Pbar"], r["Pbar"]) < 1e-9
    assert list(g["cg_iters"]) == list(r["cg_iters"])
    pa = orc.phase_averages(p, r["F"], r["a"], theory=SMALL)
    assert rel(g["Pbar_phase"][-1], pa) < 1e-9


@pytest.mark.parametrize("solver", [0, 2])
def test_fixed_point_and_ncg_parity(cb, orc, solver):
    p = problems()[1]
    g, r = solve_both(cb, orc, p, solver=solver, fixed_iterations=6)
    assert rel(g["F"], r["F"]) < 1e-10
    assert rel(g["Pbar"], r["Pbar"]) < 1e-9
    assert list(g["iters"]) == list(r["iters"])


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_converged_sphere(cb, orc, precision):
    """The 32^3 ball: FP64 and both refined forms reach the oracle's converged
    state; the mean stress is symmetric and scales with the load."""
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.sphere_32(n_steps=2)
    g = cb.solve(p, theory=SMALL, precision=precision, tol=1e-8)
    r = orc.solve(p, dict(solver=1, tol=1e-10, cg_tol=1e-6, theory=SMALL))
    assert g["steps_done"] == 2 and np.all(g["resid"] <= 1e-8)
    assert rel(g["Pbar"], r["Pbar"]) < 1e-6
    S = g["Pbar"][-1].reshape(3, 3)
    assert np.abs(S - S.T).max() < 1e-7 * np.abs(S).max()
    assert rel(g["Pbar"][0], 0.5 * g["Pbar"][1]) < 1e-6
