"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (max-abs error relative to the max-abs reference value):
  FP64 fields after equal iterations  <= 1e-10, Pbar <= 1e-9
  FP32 Green operator                  <= 2e-6 (single-precision FFT rounding)
  FP32-refined converged solve: Pbar <= 1e-5, local F <= 1e-4
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


SHAPES = [(4, 4, 4), (2, 3, 4), (6, 9, 8), (8, 12, 18), (32, 16, 24), (24, 27, 6), (16, 32, 36), (64, 8, 16),
          (64, 64, 64), (128, 256, 16), (256, 64, 128), (32, 128, 512), (512, 16, 64), (16, 512, 16)]


@pytest.mark.parametrize("kspace", [0, 1, 2])
@pytest.mark.parametrize("n", SHAPES)
def test_green_operator_fp64(cb, orc, n, kspace):
    rng = np.random.default_rng(sum(n) + kspace)
    V = n[0] * n[1] * n[2]
    l = (1.0, 0.8, 1.3)
    X = rng.normal(size=(9, V))
    Yo, sso = orc.apply_G(X, n, l, kspace)
    Yg, ssg = cb.apply_G(X, n, l, kspace, cb.FP64)
    assert rel(Yg, Yo) < 1e-12
    assert abs(ssg - sso) <= 1e-11 * sso


@pytest.mark.parametrize("kspace", [0, 2])
@pytest.mark.parametrize("n", SHAPES)
def test_green_operator_fp32(cb, orc, n, kspace):
    rng = np.random.default_rng(sum(n))
    V = n[0] * n[1] * n[2]
    X = rng.normal(size=(9, V))
    Yo, sso = orc.apply_G(X, n, (1.0, 1.0, 1.0), kspace)
    Yg, ssg = cb.apply_G(X, n, (1.0, 1.0, 1.0), kspace, cb.FP32_REFINED)
    assert rel(Yg, Yo) < 2e-6
    assert abs(ssg - sso) <= 1e-5 * sso


@pytest.mark.parametrize("kspace", [0, 2])
@pytest.mark.parametrize("n", SHAPES)
def test_green_operator_double_float(cb, orc, n, kspace):
    """The double-float transforms of the refined residual: 48-bit significand,
    so G[X] agrees with the FP64 oracle far below the FP32 error."""
    rng = np.random.default_rng(sum(n) + 7)
    V = n[0] * n[1] * n[2]
    l = (1.0, 0.8, 1.3)
    X = rng.normal(size=(9, V))
    Yo, sso = orc.apply_G(X, n, l, kspace)
    Yg, ssg = cb.apply_G(X, n, l, kspace, cb.FP32_REFINED_DF)
    assert rel(Yg, Yo) < 1e-11
    assert abs(ssg - sso) <= 1e-5 * sso  # the norm is summed from the leading FP32 parts


def test_constitutive_matches_oracle(cb, orc):
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.random_boxels((8, 6, 12), seed=3, boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
    rng = np.random.default_rng(4)
    V = 8 * 6 * 12
    F = np.eye(3).reshape(9, 1) + 0.08 * rng.uniform(-1, 1, (9, V))
    a0 = 0.01 * rng.normal(size=(p["boxel_idx"].size, 3))
    Pg, ag = cb.constitutive(p, F, a=a0)
    Po, ao = orc.constitutive_field(p, F, a=a0)
    assert rel(Pg, Po) < 1e-13
    assert rel(ag, ao) < 1e-10


def solve_both(cb, orc, p, **o):
    g = cb.solve(p, **o)
    om = dict(solver=o.get("solver", 1), kspace=o.get("kspace", 0), tol=o.get("tol", 1e-8),
              fixed_iter=o.get("fixed_iterations", 0), cg_fixed_iter=o.get("cg_fixed_iterations", 0),
              cg_tol=o.get("cg_tol", 1e-3), max_iter=o.get("max_iter", 200 if o.get("solver", 1) else 100000))
    r = orc.solve(p, om)
    return g, r


def problems():
    from paper_2204_13624_gb300 import microstructure as ms

    return [
        ms.centred_sphere((12, 12, 12), 0.2, 10.0, np.diag([1.04, 1.0, 0.99]), 2),
        ms.random_boxels((12, 6, 9), seed=7, contrast=10.0, n_steps=2),
        ms.layered((8, 4, 6), axis=1, m_incl=1, c_boxel=0.3, n_steps=1),
    ]


@pytest.mark.parametrize("k", [0, 1, 2])
def test_fixed_point_parity(cb, orc, k):
    p = problems()[k]
    g, r = solve_both(cb, orc, p, solver=0, fixed_iterations=6)
    assert rel(g["F"], r["F"]) < 1e-10
    assert rel(g["Pbar"], r["Pbar"]) < 1e-9
    assert rel(g["a"], r["a"]) < 1e-9 if len(r["a"]) else True
    assert list(g["iters"]) == list(r["iters"])
    assert g["n_operator"] == r["n_operator"]


@pytest.mark.parametrize("k", [0, 1, 2])
def test_nonlinear_cg_parity(cb, orc, k):
    """Nonlinear CG (Fletcher-Reeves, basic-scheme step): iteration by
    iteration equal to the oracle."""
    p = problems()[k]
    g, r = solve_both(cb, orc, p, solver=2, fixed_iterations=7)
    assert rel(g["F"], r["F"]) < 1e-10
    assert rel(g["Pbar"], r["Pbar"]) < 1e-9
    assert list(g["iters"]) == list(r["iters"])


def test_nonlinear_cg_converged(cb, orc):
    """The 32^3 ball to tol 1e-8 by nonlinear CG: same iteration counts as the
    oracle, and the state Newton-CG reaches."""
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.sphere_32()
    g, r = solve_both(cb, orc, p, solver=2, tol=1e-8)
    assert g["steps_done"] == 5 and np.all(g["resid"] <= 1e-8)
    assert np.all(np.abs(np.asarray(g["iters"]) - np.asarray(r["iters"])) <= 1)
    assert rel(g["Pbar"], r["Pbar"]) < 1e-8
    gn = cb.solve(p, solver=1, tol=1e-10)
    assert rel(g["Pbar"][-1], gn["Pbar"][-1]) < 1e-7


@pytest.mark.parametrize("kspace", [0, 1, 2])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_newton_cg_parity(cb, orc, k, kspace):
    p = problems()[k]
    g, r = solve_both(cb, orc, p, solver=1, kspace=kspace, fixed_iterations=2, cg_fixed_iterations=12)
    assert rel(g["F"], r["F"]) < 1e-10
    assert rel(g["P"], r["P"]) < 1e-10
    assert rel(g["Pbar"], r["Pbar"]) < 1e-9
    assert list(g["cg_iters"]) == list(r["cg_iters"])
    # phase averages (Sec. 6.2) of the final state
    pa = orc.phase_averages(p, r["F"], r["a"])
    assert rel(g["Pbar_phase"][-1], pa) < 1e-9
    # laminate NR counts may differ where |f| sits on the stopping threshold
    # within rounding (the two sides form Delta and f differently)
    assert abs(g["nr_iters"] - r["nr_iters"]) <= max(2, 1e-3 * r["nr_iters"])
    assert abs(g["n_backproj"] - r["n_backproj"]) <= max(2, 1e-3 * r["n_backproj"])


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_newton_cg_parity_fast_sizes(cb, orc, prec):
    """Grids whose sides run the compile-time FFT plans in every pass, and the
    TMA-tiled FP32 y- and z-passes at n2, n3 = 64, 128, 256."""
    from paper_2204_13624_gb300 import microstructure as ms

    for n in [(64, 64, 64), (64, 32, 128), (128, 64, 256), (32, 128, 32), (16, 256, 16)]:
        p = ms.random_spheres(n, 5.0, 0.15, 11, 10.0, np.diag([1.03, 1.0, 1.0]) + 0.01, 1)
        g, r = solve_both(cb, orc, p, solver=1, precision=prec, fixed_iterations=1, cg_fixed_iterations=10)
        tol = 1e-10 if prec == 0 else 2e-5
        assert rel(g["F"], r["F"]) < tol
        assert rel(g["Pbar"], r["Pbar"]) < (1e-9 if prec == 0 else 2e-5)


@pytest.mark.parametrize("prec", [1, 2])
def test_newton_cg_parity_mixed_radix_plans(cb, orc, prec):
    """Every 2^a 3^b side with a compile-time plan in the FP32 passes (48, 72,
    96, 108, 144, 192, 216 along y and z through the TMA-tiled passes; half
    lengths 24 .. 108 in the x-passes), against the oracle after equal
    iterations."""
    from paper_2204_13624_gb300 import microstructure as ms

    for n in [(48, 72, 96), (72, 108, 48), (96, 48, 144), (108, 16, 192), (144, 216, 8), (192, 8, 216),
              (216, 144, 8)]:
        p = ms.random_spheres(n, 3.0, 0.1, 19, 10.0, np.diag([1.03, 1.0, 1.0]) + 0.01, 1)
        g, r = solve_both(cb, orc, p, solver=1, precision=prec, fixed_iterations=1, cg_fixed_iterations=10)
        assert rel(g["F"], r["F"]) < 2e-5, n
        assert rel(g["Pbar"], r["Pbar"]) < 2e-5, n


@pytest.mark.parametrize("prec", [1, 2])
def test_newton_cg_parity_tma_512(cb, orc, prec):
    """Sides of 512 along y and z: the TMA-tiled FP32 y- and z-passes through
    5-D tensor maps (the 512-long axis as 256 x 2), rotated and staggered
    grids, against the oracle after equal iterations."""
    from paper_2204_13624_gb300 import microstructure as ms

    for n, ks in [((8, 8, 512), 0), ((8, 512, 8), 0), ((8, 512, 64), 0), ((16, 64, 512), 0), ((8, 8, 512), 2)]:
        p = ms.random_spheres(n, 3.0, 0.12, 17, 10.0, np.diag([1.03, 1.0, 1.0]) + 0.01, 1)
        g, r = solve_both(cb, orc, p, solver=1, kspace=ks, precision=prec, fixed_iterations=1,
                          cg_fixed_iterations=10)
        assert rel(g["F"], r["F"]) < 2e-5
        assert rel(g["Pbar"], r["Pbar"]) < 2e-5


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_staggered_parity_fast_sizes(cb, orc, prec):
    """The staggered grid (App. A) through every z-pass variant: runtime
    plans, compile-time plans and the TMA-tiled FP32 pass."""
    from paper_2204_13624_gb300 import microstructure as ms

    for n in [(12, 9, 18), (64, 32, 128), (16, 256, 16)]:
        p = ms.random_spheres(n, 4.0, 0.15, 13, 10.0, np.diag([1.03, 1.0, 1.0]) + 0.01, 1)
        g, r = solve_both(cb, orc, p, solver=1, kspace=2, precision=prec, fixed_iterations=1,
                          cg_fixed_iterations=10)
        tol = 1e-10 if prec == 0 else 2e-5
        assert rel(g["F"], r["F"]) < tol
        assert rel(g["Pbar"], r["Pbar"]) < (1e-9 if prec == 0 else 2e-5)


def test_staggered_sphere_32_converged(cb, orc):
    """The 32^3 ball solved to tol 1e-8 on the staggered grid, against the oracle."""
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.sphere_32()
    g, r = solve_both(cb, orc, p, solver=1, kspace=2, tol=1e-8)
    assert g["steps_done"] == 5
    assert np.all(g["resid"] <= 1e-8)
    assert list(g["iters"]) == list(r["iters"])
    assert rel(g["Pbar"], r["Pbar"]) < 1e-9
    assert rel(g["F"], r["F"]) < 1e-9


def test_sphere_32_converged_fp64(cb, orc):
    """32^3 centred sphere, vf 0.2, contrast 10, Fbar = diag(1.05,1,1) in 5 steps, tol 1e-8."""
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.sphere_32()
    g, r = solve_both(cb, orc, p, solver=1, tol=1e-8)
    assert g["steps_done"] == 5
    assert np.all(g["resid"] <= 1e-8)
    assert list(g["iters"]) == list(r["iters"])
    assert list(g["cg_iters"]) == list(r["cg_iters"])
    assert rel(g["Pbar"], r["Pbar"]) < 1e-9
    assert rel(g["F"], r["F"]) < 1e-9
    assert rel(g["Pbar_phase"][-1], orc.phase_averages(p, r["F"], r["a"])) < 1e-9


@pytest.mark.parametrize("prec", [1, 2])
def test_sphere_32_refined_fp32(cb, orc, prec):
    """FP32 Krylov iterations with FP64 (1) or double-float (2) residual
    refinement against the FP64 oracle."""
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.sphere_32()
    g = cb.solve(p, solver=1, precision=prec, tol=1e-8)
    r = orc.solve(p, dict(solver=1, tol=1e-10, cg_tol=1e-4))
    assert g["steps_done"] == 5 and np.all(g["resid"] <= 1e-8)
    assert rel(g["Pbar"], r["Pbar"]) < 1e-5
    assert rel(g["F"], r["F"]) < 1e-4


def test_double_float_form_high_contrast(cb):
    """Contrast 100 under a 10 % stretch (thin, strongly compressed boxel
    phases): the double-float form converges to the state of the plain FP64
    form, which the parity tests above pin to the oracle."""
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.random_spheres((64, 64, 64), 6.0, 0.2, 5, 100.0, np.diag([1.10, 1.0, 1.0]), 2)
    g64 = cb.solve(p, solver=1, precision=cb.FP64, tol=1e-8)
    gdf = cb.solve(p, solver=1, precision=cb.FP32_REFINED_DF, tol=1e-8)
    assert gdf["steps_done"] == 2 and np.all(gdf["resid"] <= 1e-8)
    assert rel(gdf["Pbar"], g64["Pbar"]) < 1e-6
    assert rel(gdf["F"], g64["F"]) < 1e-4


def test_layered_laminate_exact_on_gpu(cb, orc):
    from paper_2204_13624_gb300 import microstructure as ms
    import test_oracle_solve as tos

    tos.orc_mod = orc
    p = ms.layered((4, 8, 4), axis=1, m_incl=3, c_boxel=0.37)
    g = cb.solve(p, solver=1, tol=1e-12, cg_tol=1e-8, max_iter=60)
    FA, FB, c, line = tos.exact_laminate(p, 1)
    F = g["F"].reshape(9, 4, 8, 4)
    for layer, ph in enumerate(line):
        want = FA if ph == 1 else (FB if ph == 0 else c * FA + (1 - c) * FB)
        assert np.allclose(F[:, :, layer, :].reshape(9, -1), want.reshape(9, 1), atol=1e-10)


def test_homogeneous_one_iteration_gpu(cb):
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.homogeneous((6, 4, 8))
    for solver in (0, 1):
        g = cb.solve(p, solver=solver, fixed_iterations=1)
        assert np.allclose(g["F"], p["Fbar"].reshape(9, 1), atol=1e-15)
        assert g["resid"][0] < 1e-14


def test_invalid_inputs_are_rejected(cb):
    from paper_2204_13624_gb300 import microstructure as ms

    base = ms.random_boxels((6, 4, 4), seed=1)
    bad = []
    q = dict(base)
    q["n"] = (7, 4, 4)
    bad.append(q)
    q = dict(base)
    q["n"] = (3, 4, 8)
    bad.append(q)
    q = dict(base)
    q["boxel_c"] = base["boxel_c"].copy()
    q["boxel_c"][0] = 1.5
    bad.append(q)
    q = dict(base)
    q["boxel_N"] = base["boxel_N"].copy()
    q["boxel_N"][0] = 0.0
    bad.append(q)
    q = dict(base)
    q["Fbar"] = np.diag([-1.0, 1.0, 1.0]).reshape(9)
    bad.append(q)
    q = dict(base)
    q["mu"] = (0.0, 1.0)
    bad.append(q)
    for q in bad:
        with pytest.raises(cb.ComboError) as e:
            cb.solve(q, fixed_iterations=1)
        assert e.value.code == -1


def test_full_size_256_sampled(cb, orc):
    """The 256^3 ball workload in the benchmark's launch configuration: after
    one refined Newton step, the stress at sampled voxels equals the oracle's
    per-voxel constitutive law evaluated at the GPU's F; the Green operator at
    that size is idempotent and keeps HEX8R gradients."""
    import torch

    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.spheres_256()
    s = cb.Solve(p, solver=1, precision=cb.FP32_REFINED, tol=1e-8)
    s.advance(40)
    out = s.finish(fields=True)
    s.close()
    F, P, a = out["F"], out["P"], out["a"]
    rng = np.random.default_rng(0)
    V = 256 ** 3
    vox = rng.integers(0, V, 3000)
    vb = {int(v): i for i, v in enumerate(p["boxel_idx"])}
    mat = (p["mu"][0], p["lam"][0], p["mu"][1], p["lam"][1])
    for v in vox:
        ph = int(p["phase"][v])
        if ph == 2:
            b = vb[int(v)]
            Po = orc.laminate(F[:, v], p["boxel_N"][b], p["boxel_c"][b], mat, a0=a[b])["P"]
        else:
            Po = orc.neohooke(F[:, v], p["mu"][ph], p["lam"][ph], False)
        assert np.allclose(P[:, v], Po, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(Po).max()))
    # Green operator at full size: idempotent, zero mean
    n = (256, 256, 256)
    X = torch.randn((9, V), dtype=torch.float64, device="cuda")
    for prec, tol in ((cb.FP64, 1e-12), (cb.FP32_REFINED, 2e-6)):
        Y, _ = cb.apply_G(X, n, precision=prec)
        Z, _ = cb.apply_G(Y, n, precision=prec)
        err = (Z - Y).abs().max().item() / Y.abs().max().item()
        assert err < tol
        assert Y.mean(dim=1).abs().max().item() < tol


def test_full_size_512_fibres_sampled(cb, orc):
    """The 512^3 z-fibre workload (134 M voxels, 10 M boxels) in the double-float
    refined form: after two Newton updates, the stress at sampled voxels
    equals the oracle's per-voxel constitutive law at the GPU's F, and the
    fluctuation F - <F> is compatible (G leaves it unchanged) and not zero."""
    import torch

    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.fibres_512()
    # short Newton steps (8 CG iterations) so that F has been updated twice
    s = cb.Solve(p, solver=1, precision=cb.FP32_REFINED_DF, tol=1e-8, cg_fixed_iterations=8)
    s.advance(20)
    out = s.finish(fields=True, device_results=True)
    s.close()
    F, P, a = out["F"], out["P"], out["a"].cpu().numpy()
    V = 512 ** 3
    rng = np.random.default_rng(1)
    vox = rng.integers(0, V, 1500)
    bvox = rng.choice(p["boxel_idx"], 500)  # boxels in particular
    vox = np.concatenate([vox, bvox])
    idx = torch.as_tensor(vox, device=F.device)
    Fs = F[:, idx].cpu().numpy()
    Ps = P[:, idx].cpu().numpy()
    # a is returned for the boxels kept after the c_min snap, in input order
    c = p["boxel_c"]
    cmin = cb.options().c_min
    kept = (c >= cmin) & (c <= 1.0 - cmin)
    kpos = np.cumsum(kept) - 1
    vb = {int(v): i for i, v in enumerate(p["boxel_idx"])}
    mat = (p["mu"][0], p["lam"][0], p["mu"][1], p["lam"][1])
    for j, v in enumerate(vox):
        ph = int(p["phase"][v])
        if ph == 2 and not kept[vb[int(v)]]:
            ph = 0 if c[vb[int(v)]] < cmin else 1
        if ph == 2:
            b = vb[int(v)]
            Po = orc.laminate(Fs[:, j], p["boxel_N"][b], c[b], mat, a0=a[kpos[b]])["P"]
        else:
            Po = orc.neohooke(Fs[:, j], p["mu"][ph], p["lam"][ph], False)
        assert np.allclose(Ps[:, j], Po, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(Po).max()))
    del P
    # compatibility of the solved fluctuation
    Fm = F - F.mean(dim=1, keepdim=True)
    del F
    assert Fm.abs().max().item() > 1e-3
    GF, _ = cb.apply_G(Fm, (512, 512, 512), precision=cb.FP32_REFINED_DF)
    err = (GF - Fm).abs().max().item() / Fm.abs().max().item()
    assert err < 1e-5
