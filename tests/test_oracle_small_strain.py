"""Pins of the oracle's infinitesimal-strain ComBo (cheat sheet, right column).

* an isotropic linear phase is the Neo-Hookean phase linearised at F = I:
  sigma(H) = A_NH(I) : H, and C = A_NH(I);
* the closed-form composite boxel is the small-load limit of the finite-strain
  laminate (Algorithm 1): at F = I + tH, P/t -> sigma_box(H), a/t -> a(H) as
  t -> 0, and the finite-strain boxel tangent at F = I is C_box;
* its jump balances tractions, (sigma+ - sigma-) N = 0, recomputed here from
  the returned a, and C_box is the exact derivative of sigma_box (linear);
* brute force on 4^3 grids: the displacement form (rotated and staggered
  gradients) is one linear solve; the FFT solve must reach its F;
* Hill-Mandel, a symmetric mean stress, and all solvers agree.
"""
import numpy as np
import pytest

from paper_2204_13624_gb300 import microstructure as ms
from test_oracle_fft_gamma import hex8r_gradient, staggered_gradient

SMALL = dict(theory=1)


def rand_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def test_pure_phase_is_the_linearised_neohooke(orc):
    rng = np.random.default_rng(1)
    _, A = orc.neohooke(np.eye(3).ravel(), 1.3, 2.1)
    for _ in range(5):
        H = rng.normal(size=9)
        S, Cm = orc.linear(np.eye(3).ravel() + H, 1.3, 2.1)
        assert np.allclose(S, A @ H, atol=1e-14)
        assert np.allclose(S.reshape(3, 3), S.reshape(3, 3).T, atol=1e-15)
        assert np.allclose(Cm, A, atol=1e-15)


def test_small_load_limit_of_the_finite_strain_laminate(orc):
    rng = np.random.default_rng(2)
    mat = (1.0, 2.0, 10.0, 20.0)
    for _ in range(6):
        N = rand_unit(rng)
        c = rng.uniform(0.05, 0.95)
        H = rng.uniform(-1, 1, 9)
        lin = orc.laminate_linear(np.eye(3).ravel() + H, N, c, mat)
        t = 1e-7
        fin = orc.laminate(np.eye(3).ravel() + t * H, N, c, mat)
        assert np.allclose(fin["P"] / t, lin["S"], rtol=0, atol=1e-5 * np.abs(lin["S"]).max())
        assert np.allclose(fin["a"] / t, lin["a"], rtol=0, atol=1e-5 * np.abs(lin["a"]).max())
        fin0 = orc.laminate(np.eye(3).ravel(), N, c, mat)
        assert np.allclose(fin0["A"], lin["C"], atol=1e-12 * np.abs(lin["C"]).max())


def test_jump_balances_tractions_and_tangent_is_exact(orc):
    rng = np.random.default_rng(3)
    mu_m, lam_m, mu_p, lam_p = mat = (1.0, 2.0, 7.0, 4.0)
    for _ in range(6):
        N = rand_unit(rng)
        c = rng.uniform(0.05, 0.95)
        H = rng.uniform(-1, 1, 9)
        out = orc.laminate_linear(np.eye(3).ravel() + H, N, c, mat)
        a = out["a"]
        eps = 0.5 * (H.reshape(3, 3) + H.reshape(3, 3).T)
        san = 0.5 * (np.outer(a, N) + np.outer(N, a))

        def sig(e, mu, lam):
            return lam * np.trace(e) * np.eye(3) + 2 * mu * e

        sp = sig(eps + san / c, mu_p, lam_p)
        sm = sig(eps - san / (1 - c), mu_m, lam_m)
        assert np.allclose((sp - sm) @ N, 0.0, atol=1e-13 * np.abs(sp).max())
        assert np.allclose(out["S"].reshape(3, 3), c * sp + (1 - c) * sm, atol=1e-13 * np.abs(sp).max())
        d = rng.uniform(-1, 1, 9)
        out2 = orc.laminate_linear(np.eye(3).ravel() + H + d, N, c, mat)
        assert np.allclose(out2["S"] - out["S"], out["C"] @ d, atol=1e-12 * np.abs(out["C"]).max())


@pytest.mark.parametrize("kind", ["rotated", "staggered"])
def test_brute_force_4cubed(orc, kind):
    p = ms.random_boxels((4, 4, 4), seed=51, boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
    n = p["n"]
    V = 64
    h = [p["l"][j] / n[j] for j in range(3)]
    grad = (lambda U: hex8r_gradient(U, h)) if kind == "rotated" else (lambda U: staggered_gradient(U, h))
    B = np.zeros((9 * V, 3 * V))
    for q in range(3 * V):
        e = np.zeros(3 * V)
        e[q] = 1.0
        B[:, q] = grad(e.reshape(3, n[2], n[1], n[0])).reshape(-1)
    Fb = np.tile(p["Fbar"].reshape(9, 1), (1, V))
    P0, _, A = orc.constitutive_field(p, Fb, opts=SMALL, tangent=True)
    Ab = np.zeros((9 * V, 9 * V))
    for i in range(9):
        for j in range(9):
            Ab[i * V:(i + 1) * V, j * V:(j + 1) * V] = np.diag(A[:, i, j])
    u = -np.linalg.lstsq(B.T @ Ab @ B, B.T @ P0.reshape(-1), rcond=1e-12)[0]
    F_bf = Fb + (B @ u).reshape(9, V)
    P_bf, _ = orc.constitutive_field(p, F_bf, opts=SMALL)
    assert np.linalg.norm(B.T @ P_bf.reshape(-1)) < 1e-12
    # (linear: one Newton step whose CG meets 1e-12 reaches tol; a further
    # step would run CG on a right-hand side at the rounding level)
    r = orc.solve(p, dict(solver=1, kspace=0 if kind == "rotated" else 2, tol=1e-10, cg_tol=1e-12, max_iter=20,
                          **SMALL))
    assert list(r["iters"]) == [1]
    assert np.allclose(r["F"], F_bf, atol=1e-10)
    assert np.allclose(r["Pbar"][-1], P_bf.mean(axis=1), atol=1e-12)


def test_solvers_agree_hill_mandel(orc):
    p = ms.centred_sphere((12, 12, 12), 0.2, 10.0, np.eye(3) + 0.01 * np.arange(9).reshape(3, 3) / 9, 2)
    r1 = orc.solve(p, dict(solver=1, tol=1e-12, cg_tol=1e-8, **SMALL))
    r0 = orc.solve(p, dict(solver=0, tol=1e-11, max_iter=20000, **SMALL))
    r2 = orc.solve(p, dict(solver=2, tol=1e-11, max_iter=20000, **SMALL))
    H = r1["F"] - np.eye(3).reshape(9, 1)
    Hb = p["Fbar"] - np.eye(3).ravel()
    assert abs(np.mean(np.sum(r1["P"] * H, axis=0)) - np.dot(r1["Pbar"][-1], Hb)) < 1e-12
    S = r1["Pbar"][-1].reshape(3, 3)
    assert np.allclose(S, S.T, atol=1e-14)
    assert np.allclose(r0["Pbar"], r1["Pbar"], atol=1e-10)
    assert np.allclose(r2["Pbar"], r1["Pbar"], atol=1e-10)
    # linear: the two load steps scale
    assert np.allclose(r1["Pbar"][0], 0.5 * r1["Pbar"][1], atol=1e-12)
    # one Newton step with an exact CG solves a linear problem
    assert r1["iters"][0] <= 4
