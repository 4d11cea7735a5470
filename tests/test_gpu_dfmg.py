"""GPU parity of the doubly-fine material grid (App. A, Eq. constitutive_law)
against the FP64 oracle, through the C ABI (kspace COMBO_STAGGERED_DFMG).

Tolerances (max-abs error relative to the max-abs reference value): the law
of a field <= 1e-12 (the same FP64 formulas, summed in the same order; the
laminates converge to the same root within their NR tolerance, which the
jump vectors show at <= 1e-9); equal iterations of a solve <= 1e-10 in F,
<= 1e-9 in Pbar, the same iteration counts; converged solves <= 1e-8.
"""
import numpy as np
import pytest

from test_gpu_parity import problems, rel, solve_both

pytestmark = pytest.mark.gpu
DFMG = 3


@pytest.fixture(scope="module")
def cb():
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    return combo


@pytest.mark.parametrize("n", [(12, 9, 18), (16, 16, 16), (64, 32, 8), (8, 64, 6), (64, 48, 96), (2, 2, 2), (2, 4, 6)])
def test_law_parity(cb, orc, n):
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.random_boxels(n, seed=sum(n), boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
    V = n[0] * n[1] * n[2]
    rng = np.random.default_rng(V)
    F = np.eye(3).reshape(9, 1) + 0.08 * rng.uniform(-1, 1, (9, V))
    Pg, ag = cb.constitutive(p, F, kspace=DFMG)
    Po, ao = orc.constitutive_field(p, F, opts=dict(kspace=DFMG))
    assert rel(Pg, Po) < 1e-12
    if len(ao):
        assert rel(ag, ao) < 1e-9
    # the plain law differs: the gather is not the identity
    P2, _ = cb.constitutive(p, F, kspace=2)
    assert rel(P2, Po) > 1e-3


@pytest.mark.parametrize("solver", [0, 2])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_iteration_parity(cb, orc, k, solver):
    """Fixed point and nonlinear CG, iteration by iteration."""
    p = problems()[k]
    g, r = solve_both(cb, orc, p, solver=solver, kspace=DFMG, fixed_iterations=6)
    assert rel(g["F"], r["F"]) < 1e-10
    assert rel(g["P"], r["P"]) < 1e-10
    assert rel(g["Pbar"], r["Pbar"]) < 1e-9
    if len(r["a"]):
        assert rel(g["a"], r["a"]) < 1e-8
    assert list(g["iters"]) == list(r["iters"])
    assert g["n_operator"] == r["n_operator"]
    assert g["n_laminate_evals"] == r["n_lam_evals"]


def test_converged_sphere(cb, orc):
    """A 24^3 ball, two load steps, nonlinear CG to tol 1e-8: the oracle's
    state, its iteration counts within one, and its sub-cell phase averages;
    the fixed point reaches the same state."""
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.centred_sphere((24, 24, 24), 0.2, 10.0, np.diag([1.06, 1.0, 0.97]), 2)
    g, r = solve_both(cb, orc, p, solver=2, kspace=DFMG, tol=1e-8)
    assert g["steps_done"] == 2 and np.all(g["resid"] <= 1e-8)
    assert np.all(np.abs(np.asarray(g["iters"]) - np.asarray(r["iters"])) <= 1)
    assert rel(g["Pbar"], r["Pbar"]) < 1e-8
    assert rel(g["F"], r["F"]) < 1e-6
    pa = orc.phase_averages(p, r["F"], r["a"], kspace=DFMG)
    assert rel(g["Pbar_phase"][-1], pa) < 1e-7
    g0 = cb.solve(p, solver=0, kspace=DFMG, tol=1e-8)
    assert rel(g0["Pbar"][-1], g["Pbar"][-1]) < 1e-6
    assert g0["iters"].sum() > g["iters"].sum()
    # the double-float residual form reaches the same state
    gd = cb.solve(p, solver=2, kspace=DFMG, precision=2, tol=1e-8)
    assert np.all(gd["resid"] <= 1e-8)
    assert rel(gd["Pbar"], r["Pbar"]) < 1e-8
    assert rel(gd["Pbar_phase"][-1], pa) < 1e-7


@pytest.mark.parametrize("kspace", [0, DFMG])
@pytest.mark.parametrize("solver", [0, 2])
@pytest.mark.parametrize("k", [0, 1])
def test_double_float_residual_form(cb, orc, k, solver, kspace):
    """The fixed point and nonlinear CG with the double-float residual form
    (COMBO_FP32_REFINED_DF: the law -- the doubly-fine sub-cell laws and their
    gather included -- and the transforms in double-float, F in FP64):
    iteration by iteration within 1e-10 of the FP64 oracle."""
    p = problems()[k]
    g, r = solve_both(cb, orc, p, solver=solver, kspace=kspace, precision=2, fixed_iterations=6)
    assert rel(g["F"], r["F"]) < 1e-10
    assert rel(g["Pbar"], r["Pbar"]) < 1e-9
    assert list(g["iters"]) == list(r["iters"])


def test_refined_fp32_form_rejected_without_newton(cb):
    from paper_2204_13624_gb300 import microstructure as ms

    with pytest.raises(Exception):
        cb.solve(ms.homogeneous((8, 8, 8)), solver=2, precision=1)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_newton_cg_iteration_parity(cb, orc, k):
    """Newton-CG on the doubly-fine grid (the Hessian of the sub-cell energy
    in CG) in FP64 against the oracle's Newton-CG, equal iterations."""
    p = problems()[k]
    g, r = solve_both(cb, orc, p, solver=1, kspace=DFMG, fixed_iterations=2, cg_fixed_iterations=8)
    assert rel(g["F"], r["F"]) < 1e-10
    assert rel(g["P"], r["P"]) < 1e-10
    assert rel(g["Pbar"], r["Pbar"]) < 1e-9
    assert g["n_operator"] == r["n_operator"]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_newton_cg_converged(cb, orc, prec):
    """Converged Newton-CG on the doubly-fine grid in every precision form
    against the oracle's converged Newton-CG (FP64 Pbar <= 1e-8; refined
    forms Pbar <= 1e-5, F <= 1e-4), and against the GPU's nonlinear CG."""
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.random_spheres((24, 24, 24), 4.0, 0.15, 31, 10.0, np.diag([1.04, 1.0, 1.0]), 2)
    r = orc.solve(p, dict(solver=1, kspace=DFMG, tol=1e-10, cg_tol=1e-4))
    tol = 1e-10 if prec == 0 else 1e-8  # FP64: the oracle's tolerance
    g = cb.solve(p, solver=1, kspace=DFMG, precision=prec, tol=tol, cg_tol=1e-4 if prec == 0 else 1e-3)
    assert g["steps_done"] == 2 and np.all(g["resid"] <= tol)
    assert rel(g["Pbar"], r["Pbar"]) < (1e-9 if prec == 0 else 1e-5)
    assert rel(g["F"], r["F"]) < (1e-8 if prec == 0 else 1e-4)
    n = cb.solve(p, solver=2, kspace=DFMG, tol=1e-8)
    assert rel(g["Pbar"], n["Pbar"]) < 1e-5
    assert g["n_operator"] > 0 and g["n_operator_fp64"] < n["n_operator_fp64"]


def test_newton_cg_batch_rejected(cb):
    from paper_2204_13624_gb300 import microstructure as ms

    with pytest.raises(Exception):
        cb.solve_batch([ms.homogeneous((8, 8, 8))] * 2, solver=1, kspace=DFMG)


def test_double_float_log_accuracy(cb):
    """The double-float logarithm of the double-float forms against the FP64
    logarithm: absolute error <= 2^-46 max(1, |ln x|) over [1e-3, 1e3], where
    the inputs are first rounded to double-float (48-bit significand)."""
    rng = np.random.default_rng(9)
    x = np.concatenate([np.exp(rng.uniform(np.log(1e-3), np.log(1e3), 20000)),
                        1.0 + rng.uniform(-1e-3, 1e-3, 5000), [1.0, 2.0, 0.5, np.sqrt(2.0), 1 / np.sqrt(2.0)]])
    hi = x.astype(np.float32).astype(np.float64)
    xd = hi + (x - hi).astype(np.float32).astype(np.float64)  # the double-float value the kernel sees
    y = cb.df_log(x)
    ref = np.log(xd)
    err = np.abs(y - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() < 2.0 ** -46, err.max()
    assert y[-5] == 0.0
