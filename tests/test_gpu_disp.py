"""The reduced evaluation forms of the rotated Green operator in the FP32
Krylov passes, against the oracle after equal iterations and against the
nine-component form of the same solve:

* displacement form: the z-pass leaves one nodal spectrum per row, the
  y-inverse and x-inverse take three components, the HEX8R gradient is fused
  with the CG update (with the x-inverse too, where n2 allows its columns);
* nodal form: in addition the tangent pass assembles the nodal forces
  D^T (A : p) in real space (halo lines and planes, two direction buffers),
  the y-forward takes three components and the z-pass divides by |kr|^2.

Tolerances (max-abs error relative to the max-abs reference value), as the
other FP32 Krylov parity tests: equal iterations F, Pbar <= 2e-5; converged
refined solves Pbar <= 1e-5, F <= 1e-4 (two forms at tol 1e-8: Pbar agree
<= 1e-6)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DISP, NODAL = 1, 2


@pytest.fixture(scope="module")
def cb():
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    combo.krylov_form(combo.KRYLOV_NODAL)
    yield combo
    combo.krylov_form(combo.KRYLOV_NODAL)
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


def form_of(cls):
    return NODAL if "xfwd_nodal" in cls else (DISP if ("grad_cg" in cls or "xinv_grad_cg" in cls) else 0)


def balls(n, seed=19, r=3.0):
    from paper_2204_13624_gb300 import microstructure as ms

    return ms.random_spheres(n, r, 0.1, seed, 10.0, np.diag([1.03, 1.0, 1.0]) + 0.01, 1)


FIXED = dict(solver=1, fixed_iterations=1, cg_fixed_iterations=10)


def oracle_fixed(orc, p, kspace=0):
    return orc.solve(p, dict(solver=1, kspace=kspace, fixed_iter=1, cg_fixed_iter=10))


# grids of every x size the forms take (n1 = 128, 256, 512), compile-time y
# and z plans of both radix families, n2 = 108 (a multiple of 4, not of 8:
# the nodal pass's 4-line columns at n1 = 256, and the separate x-inverse and
# gradient kernels instead of the fused one), and z = 512 (the 5-D tensor
# maps of the one-component stores)
GRIDS = [(128, 48, 72), (256, 64, 48), (512, 48, 48), (256, 108, 48), (128, 48, 512), (128, 96, 144)]


@pytest.mark.parametrize("form", [DISP, NODAL])
@pytest.mark.parametrize("prec", [1, 2])
def test_reduced_form_against_oracle(cb, orc, form, prec):
    cb.krylov_form(form)
    try:
        for n in GRIDS:
            p = balls(n)
            assert form_of(classes(cb, p, precision=prec, **FIXED)) == form, n
            g = cb.solve(p, precision=prec, **FIXED)
            r = oracle_fixed(orc, p)
            assert rel(g["F"], r["F"]) < 2e-5, n
            assert rel(g["Pbar"], r["Pbar"]) < 2e-5, n
    finally:
        cb.krylov_form(NODAL)


@pytest.mark.parametrize("z", [72, 108, 216])
def test_displacement_form_second_z_tile_width(cb, orc, z):
    """The displacement z-pass's second tile width, whose component group is
    not a whole number of warps for these lengths (the last warp of the
    inverse runs partly on a component that is not stored)."""
    cb.krylov_form(DISP)
    cb.autotune_force(2, 1)
    try:
        p = balls((128, 48, z), seed=23)
        g = cb.solve(p, precision=1, **FIXED)
    finally:
        cb.autotune_force(2, -1)
        cb.krylov_form(NODAL)
    r = oracle_fixed(orc, p)
    assert rel(g["F"], r["F"]) < 2e-5
    assert rel(g["Pbar"], r["Pbar"]) < 2e-5


@pytest.mark.parametrize("form", [DISP, NODAL])
def test_reduced_form_in_stacked_batch(cb, orc, form):
    """Three problems on one grid stacked along z: the stencils wrap z within
    each problem, the reductions stay per problem."""
    from paper_2204_13624_gb300 import microstructure as ms

    probs = [balls((128, 48, 48), seed=31), ms.random_boxels((128, 48, 48), seed=32, contrast=5.0, n_steps=1),
             balls((128, 48, 48), seed=33, r=4.0)]
    cb.krylov_form(form)
    try:
        out = cb.solve_batch(probs, precision=1, **FIXED)
    finally:
        cb.krylov_form(NODAL)
    for p, g in zip(probs, out):
        r = oracle_fixed(orc, p)
        assert rel(g["F"], r["F"]) < 2e-5
        assert rel(g["Pbar"], r["Pbar"]) < 2e-5


def test_nodal_form_boxels_on_every_line(cb, orc):
    """Random boxels (random c+ and N at every voxel of a random half): the
    boxel tangents of halo lines and planes enter the nodal forces."""
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.random_boxels((128, 48, 48), seed=37, contrast=8.0, n_steps=1)
    assert form_of(classes(cb, p, precision=1, **FIXED)) == NODAL
    g = cb.solve(p, precision=1, **FIXED)
    r = oracle_fixed(orc, p)
    assert rel(g["F"], r["F"]) < 2e-5
    assert rel(g["Pbar"], r["Pbar"]) < 2e-5


@pytest.mark.parametrize("prec", [1, 2])
def test_reduced_forms_equal_nine_component_form(cb, prec):
    """Converged two-step solves (so CG runs both parities of iterations and
    the final update reads either direction buffer) in all three forms."""
    p = balls((128, 64, 64), seed=41, r=5.0)
    p["n_steps"] = 2
    res = {}
    try:
        for form in (0, DISP, NODAL):
            cb.krylov_form(form)
            assert form_of(classes(cb, p, precision=prec, solver=1, tol=1e-8)) == form
            res[form] = cb.solve(p, precision=prec, solver=1, tol=1e-8)
    finally:
        cb.krylov_form(NODAL)
    a = res[0]
    for form in (DISP, NODAL):
        b = res[form]
        assert np.all(a["resid"] <= 1e-8) and np.all(b["resid"] <= 1e-8)
        assert np.array_equal(a["iters"], b["iters"])
        assert rel(b["Pbar"], a["Pbar"]) < 1e-6
        assert rel(b["F"], a["F"]) < 1e-4


def test_nodal_form_converged_against_oracle(cb, orc):
    p = balls((128, 48, 48), seed=43, r=4.0)
    p["n_steps"] = 2
    g = cb.solve(p, precision=2, solver=1, tol=1e-8)
    r = orc.solve(p, dict(solver=1, tol=1e-10, cg_tol=1e-4))
    assert np.all(g["resid"] <= 1e-8)
    assert rel(g["Pbar"], r["Pbar"]) < 1e-5
    assert rel(g["F"], r["F"]) < 1e-4


def test_where_the_forms_do_not_apply(cb):
    """Staggered grid, an x size without the forms' kernels, a y side
    without a TMA-tiled plan and FP64 Krylov words keep the nine-component
    form; an unknown form is rejected."""
    for n, o in [((128, 48, 48), dict(kspace=2, precision=1)), ((96, 48, 48), dict(precision=1)),
                 ((128, 54, 48), dict(precision=1)), ((128, 48, 48), dict(precision=0))]:
        assert form_of(classes(cb, balls(n), solver=1, **o)) == 0, n
    with pytest.raises(cb.ComboError) as e:
        cb.krylov_form(3)
    assert e.value.code == -1
