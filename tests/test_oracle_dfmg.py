"""Pins of the oracle's doubly-fine material grid (App. A, Eq. constitutive_law).

Every cell is cut into 8 sub-cells l in {0,1}^3.  Sub-cell l of cell c takes
the diagonal of F at c and each off-diagonal pair F_ab, F_ba from the staggered
position c + l_a e_a + l_b e_b (the edge nearest the sub-cell when F_ab[xi]
sits at xi - (e_a + e_b)/2, as the backward differences of the staggered
gradient put it).  The stress is the gradient of the sub-cell energy

    E(F) = 1/8 sum_c sum_l W_c(F_sub(c, l)),

W_c the Neo-Hookean energy of a pure cell, or c+ W+(F+) + c- W-(F-) at the
converged laminate jump of a composite boxel (Sec. 4.1).

* the oracle's stress equals central differences of E, assembled here with
  numpy shifts and the pinned Neo-Hookean energy, entry by entry;
* a uniform F gives the ordinary law on the diagonal and the mean of the four
  cells sharing an edge off it;
* the equilibrium of the staggered scheme with this law is the minimiser of E
  over staggered displacements: a displacement-based Newton (finite-difference
  Hessian of the oracle's own, pinned gradient) on a 4^3 grid must reach the
  F the FFT solve reaches;
* Hill-Mandel holds at convergence, and fixed point and nonlinear CG agree;
* the tangent (the sub-cell tangents applied to the assembled direction and
  gathered) is the derivative of the law and symmetric, and Newton-CG with it
  reaches the nonlinear-CG state.
"""
import numpy as np
import pytest

from paper_2204_13624_gb300 import microstructure as ms
from test_oracle_fft_gamma import staggered_gradient

DFMG = 3
SRC = {1: (0, 1), 3: (0, 1), 2: (0, 2), 6: (0, 2), 5: (1, 2), 7: (1, 2)}  # component -> axes (a, b)


def f_sub(F, n, l):
    """F_sub(c, l) for every cell c: [9][V].  F is [9][V] with V = n3*n2*n1, x fastest."""
    G = F.reshape(9, n[2], n[1], n[0])
    out = G.copy()
    axis_of = {0: 2, 1: 1, 2: 0}  # grid axis a -> numpy axis of [n3][n2][n1]
    for comp, (a, b) in SRC.items():
        shift = [0, 0, 0]
        shift[axis_of[a]] = -l[a]
        shift[axis_of[b]] = -l[b]
        out[comp] = np.roll(G[comp], shift, axis=(0, 1, 2))
    return out.reshape(9, -1)


def cell_energies(orc, p, F):
    """W_c(F_sub(c, l)) as [8][V]."""
    n = p["n"]
    V = n[0] * n[1] * n[2]
    phase = np.asarray(p["phase"]).ravel()
    box = -np.ones(V, np.int64)
    box[np.asarray(p["boxel_idx"], np.int64)] = np.arange(len(p["boxel_idx"]))
    mu, lam = p["mu"], p["lam"]
    mat = (mu[0], lam[0], mu[1], lam[1])
    W = np.zeros((8, V))
    for li in range(8):
        l = (li & 1, (li >> 1) & 1, (li >> 2) & 1)
        Fs = f_sub(F, n, l)
        for v in range(V):
            Fv = Fs[:, v]
            if phase[v] == 2:
                k = box[v]
                c = float(p["boxel_c"][k])
                N = np.asarray(p["boxel_N"][k], float)
                a = orc.laminate(Fv, N, c, mat)["a"]
                aN = np.outer(a, N).ravel()
                W[li, v] = (c * orc.neohooke_energy(Fv + aN / c, mu[1], lam[1])
                            + (1 - c) * orc.neohooke_energy(Fv - aN / (1 - c), mu[0], lam[0]))
            else:
                ph = int(phase[v])
                W[li, v] = orc.neohooke_energy(Fv, mu[ph], lam[ph])
    return W


def test_stress_is_the_gradient_of_the_subcell_energy(orc):
    p = ms.random_boxels((5, 4, 3), seed=41, boxel_frac=0.35, incl_frac=0.3, contrast=10.0)
    V = 60
    rng = np.random.default_rng(5)
    F = np.eye(3).reshape(9, 1) + 0.08 * rng.uniform(-1, 1, (9, V))
    P, _ = orc.constitutive_field(p, F, opts=dict(kspace=DFMG))
    phase = np.asarray(p["phase"]).ravel()
    picks = [(c, v) for c in range(9) for v in rng.choice(V, 4, replace=False)]
    picks += [(c, int(np.flatnonzero(phase == 2)[0])) for c in range(9)]
    h = 1e-5
    for comp, v in picks:
        Fp = F.copy()
        Fm = F.copy()
        Fp[comp, v] += h
        Fm[comp, v] -= h
        dE = (cell_energies(orc, p, Fp) - cell_energies(orc, p, Fm)).sum() / 8.0
        assert abs(dE / (2 * h) - P[comp, v]) < 1e-7, (comp, v, dE / (2 * h), P[comp, v])


def test_uniform_deformation(orc):
    p = ms.random_boxels((6, 5, 4), seed=42, boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
    n = p["n"]
    V = n[0] * n[1] * n[2]
    F = np.tile((np.eye(3) + 0.05 * np.arange(9).reshape(3, 3) / 9).reshape(9, 1), (1, V))
    P3, _ = orc.constitutive_field(p, F, opts=dict(kspace=DFMG))
    P0, _ = orc.constitutive_field(p, F)
    for comp in (0, 4, 8):
        assert np.allclose(P3[comp], P0[comp], atol=1e-12)
    axis_of = {0: 2, 1: 1, 2: 0}
    for comp, (a, b) in SRC.items():
        G = P0[comp].reshape(n[2], n[1], n[0])
        m = np.zeros_like(G)
        for la in (0, 1):
            for lb in (0, 1):
                shift = [0, 0, 0]
                shift[axis_of[a]] = la
                shift[axis_of[b]] = lb
                m += np.roll(G, shift, axis=(0, 1, 2))
        assert np.allclose(P3[comp], m.ravel() / 4, atol=1e-12), comp


@pytest.mark.slow
def test_displacement_minimiser_4cubed(orc):
    p = ms.random_boxels((4, 4, 4), seed=43, boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
    n = p["n"]
    V = 64
    h = [p["l"][j] / n[j] for j in range(3)]
    B = np.zeros((9 * V, 3 * V))
    for q in range(3 * V):
        e = np.zeros(3 * V)
        e[q] = 1.0
        B[:, q] = staggered_gradient(e.reshape(3, n[2], n[1], n[0]), h).reshape(-1)
    Fb = p["Fbar"].reshape(9, 1)
    opts = dict(kspace=DFMG)

    def grad(u):
        P, _ = orc.constitutive_field(p, Fb + (B @ u).reshape(9, V), opts=opts)
        return B.T @ P.reshape(-1)

    u = np.zeros(3 * V)
    eps = 1e-6
    for it in range(30):
        g = grad(u)
        if np.linalg.norm(g) < 1e-12:
            break
        H = np.zeros((3 * V, 3 * V))
        for q in range(3 * V):
            e = np.zeros(3 * V)
            e[q] = eps
            H[:, q] = (grad(u + e) - grad(u - e)) / (2 * eps)
        u -= np.linalg.lstsq(0.5 * (H + H.T), g, rcond=1e-10)[0]
    assert np.linalg.norm(grad(u)) < 1e-11
    F_bf = Fb + (B @ u).reshape(9, V)
    r = orc.solve(p, dict(solver=2, kspace=DFMG, tol=1e-13, max_iter=20000))
    assert np.allclose(r["F"], F_bf, atol=1e-9)


def test_fixed_point_and_ncg_agree_hill_mandel(orc):
    p = ms.centred_sphere((12, 12, 12), 0.2, 10.0, np.diag([1.04, 1.0, 0.99]) + 0.02 * np.eye(3)[[1, 0, 2]], 2)
    r2 = orc.solve(p, dict(solver=2, kspace=DFMG, tol=1e-11, max_iter=5000))
    r0 = orc.solve(p, dict(solver=0, kspace=DFMG, tol=1e-11, max_iter=20000))
    F, P = r2["F"], r2["P"]
    hm = np.mean(np.sum(P * F, axis=0))
    assert abs(hm - np.dot(r2["Pbar"][-1], p["Fbar"])) < 1e-10
    assert np.allclose(r0["F"], r2["F"], atol=1e-8)
    assert np.allclose(r0["Pbar"], r2["Pbar"], atol=1e-9)
    assert r2["iters"].sum() < r0["iters"].sum()
    # the plain staggered scheme gives a nearby but different state
    rs = orc.solve(p, dict(solver=2, kspace=2, tol=1e-11, max_iter=5000))
    d = np.abs(rs["Pbar"][-1] - r2["Pbar"][-1]).max()
    assert 1e-6 < d < 5e-2 * np.abs(r2["Pbar"][-1]).max()


def test_tangent_is_the_derivative_of_the_law(orc):
    """The doubly-fine tangent (the gather of the sub-cell tangents applied to
    the assembled direction) equals central differences of the pinned law,
    and it is symmetric (the Hessian of the sub-cell energy)."""
    p = ms.random_boxels((5, 4, 6), seed=45, boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
    V = 120
    rng = np.random.default_rng(6)
    F = np.eye(3).reshape(9, 1) + 0.08 * rng.uniform(-1, 1, (9, V))
    X1, X2 = rng.normal(size=(9, V)), rng.normal(size=(9, V))
    T1 = orc.dfmg_tangent_apply(p, F, X1)
    T2 = orc.dfmg_tangent_apply(p, F, X2)
    h = 1e-5
    Pp, _ = orc.constitutive_field(p, F + h * X1, opts=dict(kspace=DFMG))
    Pm, _ = orc.constitutive_field(p, F - h * X1, opts=dict(kspace=DFMG))
    fd = (Pp - Pm) / (2 * h)
    assert np.abs(fd - T1).max() < 1e-6 * np.abs(T1).max()
    assert abs(np.sum(X2 * T1) - np.sum(X1 * T2)) < 1e-10 * np.sqrt(np.sum(X1 * T1) * np.sum(X2 * T2))


def test_newton_reaches_the_nonlinear_cg_state(orc):
    p = ms.centred_sphere((12, 12, 12), 0.2, 10.0, np.diag([1.04, 1.0, 0.99]) + 0.02 * np.eye(3)[[1, 0, 2]], 2)
    rn = orc.solve(p, dict(solver=1, kspace=DFMG, tol=1e-11, cg_tol=1e-6))
    r2 = orc.solve(p, dict(solver=2, kspace=DFMG, tol=1e-11, max_iter=5000))
    assert np.allclose(rn["F"], r2["F"], atol=1e-8)
    assert np.allclose(rn["Pbar"], r2["Pbar"], atol=1e-10)
    assert rn["iters"].max() <= 8


def test_infinitesimal_strain_is_rejected(orc):
    p = ms.homogeneous((4, 4, 4))
    r = orc.solve(p, dict(solver=2, kspace=DFMG, theory=1), raise_on_error=False)
    assert r["status"] != 0


def test_phase_averages_split_the_mean_stress(orc):
    """Sub-cell phase averages: their volume-weighted sum is Pbar, since the
    gather moves every sub-cell stress component to exactly one cell."""
    p = ms.random_boxels((6, 5, 4), seed=44, boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
    r = orc.solve(p, dict(solver=2, kspace=DFMG, tol=1e-11, max_iter=5000))
    pa = orc.phase_averages(p, r["F"], r["a"], kspace=DFMG)
    phase = np.asarray(p["phase"]).ravel()
    c = np.asarray(p["boxel_c"])
    vol_p = (phase == 1).sum() + c.sum()
    vol_m = (phase == 0).sum() + (1 - c).sum()
    assert np.allclose((vol_m * pa[0] + vol_p * pa[1]) / phase.size, r["Pbar"][-1], atol=1e-11)
    assert np.allclose(r["P"].mean(axis=1), r["Pbar"][-1], atol=1e-13)
