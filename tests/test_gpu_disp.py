"""The displacement form of the rotated Green operator in the FP32 Krylov
passes (z-pass writing one nodal spectrum per row, y-inverse of three
components, x-inverse to the nodal fields, HEX8R gradient fused with the CG
update), against the oracle after equal iterations and against the
nine-component form of the same solve.

Tolerances (max-abs error relative to the max-abs reference value), as the
other FP32 Krylov parity tests: equal iterations F, Pbar <= 2e-5; converged
refined solves Pbar <= 1e-5, F <= 1e-4 (both forms at tol 1e-8: Pbar agree
<= 1e-6)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cb():
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    combo.krylov_displacement_form(True)
    yield combo
    combo.krylov_displacement_form(True)
    combo.autotune_force(2, -1)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def classes(cb, p, **o):
    """Kernel classes that one CG chunk of the solve launched."""
    s = cb.Solve(p, **o)
    try:
        s.profile(True)
        s.advance(10)
        return set(k for k, (ms, n) in s.profile_read().items() if n > 0)
    finally:
        s.close()


def balls(n, seed=19, r=3.0):
    from paper_2204_13624_gb300 import microstructure as ms

    return ms.random_spheres(n, r, 0.1, seed, 10.0, np.diag([1.03, 1.0, 1.0]) + 0.01, 1)


FIXED = dict(solver=1, fixed_iterations=1, cg_fixed_iterations=10)


def oracle_fixed(orc, p, kspace=0):
    return orc.solve(p, dict(solver=1, kspace=kspace, fixed_iter=1, cg_fixed_iter=10))


# grids of every x size the form takes (n1 = 128, 256, 512), compile-time y
# and z plans of both radix families, n2 = 108 (a multiple of 4, not of 8),
# and z = 512 (the 5-D tensor maps of the one-component store)
GRIDS = [(128, 48, 72), (256, 64, 48), (512, 48, 48), (256, 108, 48), (128, 48, 512), (128, 96, 144)]


@pytest.mark.parametrize("prec", [1, 2])
def test_displacement_form_against_oracle(cb, orc, prec):
    for n in GRIDS:
        p = balls(n)
        assert "grad_cg" in classes(cb, p, precision=prec, **FIXED), n
        g = cb.solve(p, precision=prec, **FIXED)
        r = oracle_fixed(orc, p)
        assert rel(g["F"], r["F"]) < 2e-5, n
        assert rel(g["Pbar"], r["Pbar"]) < 2e-5, n


@pytest.mark.parametrize("z", [72, 108, 216])
def test_displacement_form_second_z_tile_width(cb, orc, z):
    """The z-pass's second tile width, whose component group is not a whole
    number of warps for these lengths (the last warp of the inverse runs
    partly on a component that is not stored)."""
    cb.autotune_force(2, 1)
    try:
        p = balls((128, 48, z), seed=23)
        g = cb.solve(p, precision=1, **FIXED)
    finally:
        cb.autotune_force(2, -1)
    r = oracle_fixed(orc, p)
    assert rel(g["F"], r["F"]) < 2e-5
    assert rel(g["Pbar"], r["Pbar"]) < 2e-5


def test_displacement_form_in_stacked_batch(cb, orc):
    """Three problems on one grid stacked along z: the gradient wraps z
    within each problem, the reductions stay per problem."""
    from paper_2204_13624_gb300 import microstructure as ms

    probs = [balls((128, 48, 48), seed=31), ms.random_boxels((128, 48, 48), seed=32, contrast=5.0, n_steps=1),
             balls((128, 48, 48), seed=33, r=4.0)]
    out = cb.solve_batch(probs, precision=1, **FIXED)
    for p, g in zip(probs, out):
        r = oracle_fixed(orc, p)
        assert rel(g["F"], r["F"]) < 2e-5
        assert rel(g["Pbar"], r["Pbar"]) < 2e-5


@pytest.mark.parametrize("prec", [1, 2])
def test_displacement_form_equals_nine_component_form(cb, prec):
    p = balls((128, 64, 64), seed=41, r=5.0)
    p["n_steps"] = 2
    cb.krylov_displacement_form(False)
    try:
        assert "grad_cg" not in classes(cb, p, precision=prec, solver=1, tol=1e-8)
        a = cb.solve(p, precision=prec, solver=1, tol=1e-8)
    finally:
        cb.krylov_displacement_form(True)
    b = cb.solve(p, precision=prec, solver=1, tol=1e-8)
    assert np.all(a["resid"] <= 1e-8) and np.all(b["resid"] <= 1e-8)
    assert np.array_equal(a["iters"], b["iters"])
    assert rel(b["Pbar"], a["Pbar"]) < 1e-6
    assert rel(b["F"], a["F"]) < 1e-4


def test_displacement_form_converged_against_oracle(cb, orc):
    p = balls((128, 48, 48), seed=43, r=4.0)
    p["n_steps"] = 2
    g = cb.solve(p, precision=2, solver=1, tol=1e-8)
    r = orc.solve(p, dict(solver=1, tol=1e-10, cg_tol=1e-4))
    assert np.all(g["resid"] <= 1e-8)
    assert rel(g["Pbar"], r["Pbar"]) < 1e-5
    assert rel(g["F"], r["F"]) < 1e-4


def test_where_the_form_does_not_apply(cb):
    """Staggered grid, an x size without the form's kernels, a y side
    without a TMA-tiled plan and FP64 Krylov words keep the nine-component
    form."""
    for n, o in [((128, 48, 48), dict(kspace=2, precision=1)), ((96, 48, 48), dict(precision=1)),
                 ((128, 54, 48), dict(precision=1)), ((128, 48, 48), dict(precision=0))]:
        assert "grad_cg" not in classes(cb, balls(n), solver=1, **o), n
