"""Whole-solve pins of the oracle (paper Sec. 2 HOM, Sec. 3 Lippmann-Schwinger).

* homogeneous medium: F == Fbar after one iteration, zero residual;
* grid-aligned layered microstructure with one boxel layer: the solve must
  reproduce the exact rank-one laminate, computed here with scipy on the
  traction balance of the two pure phases (Sec. 4.1 jump conditions);
* brute force on 4^3 grids: the displacement-based discrete problem -- nodal
  displacements at voxel corners with the HEX8R gradient (rotated scheme) or
  a dense spectral gradient matrix (Moulinec-Suquet scheme) -- solved by a
  dense Newton with least squares; F must match the FFT solve;
* Hill-Mandel <P . F> = Pbar . Fbar at convergence (Sec. 2);
* fixed point and Newton-CG converge to the same state.
"""
import numpy as np
import pytest

from paper_2204_13624_gb300 import microstructure as ms
from test_oracle_fft_gamma import band_limit, hex8r_gradient, spectral_gradient, staggered_gradient

TIGHT = dict(tol=1e-12, cg_tol=1e-8, max_iter=60)


@pytest.mark.parametrize("solver", [0, 1])
def test_homogeneous_one_iteration(orc, solver):
    p = ms.homogeneous((6, 4, 8))
    r = orc.solve(p, dict(solver=solver, fixed_iter=1))
    Fb = p["Fbar"]
    assert np.allclose(r["F"], Fb[:, None], atol=1e-15)
    assert r["resid"][0] < 1e-14
    P = orc.neohooke(Fb, 1.0, 2.0, False)
    assert np.allclose(r["Pbar"][0], P, atol=1e-14)


def exact_laminate(p, axis):
    """Overall rank-one laminate of the layered problem: F_A (inclusion),
    F_B (matrix) with F_A - F_B = a (x) e_axis, mean Fbar, equal tractions."""
    n = p["n"]
    nax = n[axis]
    # count the inclusion layers from the phase field itself
    ph = p["phase"].reshape(n[2], n[1], n[0])
    line = np.moveaxis(ph, 2 - axis, 0)[:, 0, 0]
    m = int(np.sum(line == 1))
    c = float(p["boxel_c"][0])
    ct = (m + c) / nax
    N = np.zeros(3)
    N[axis] = 1.0
    Fb = p["Fbar"].reshape(3, 3)
    mu, lam = p["mu"], p["lam"]

    def F_AB(a):
        return Fb + (1 - ct) * np.outer(a, N), Fb - ct * np.outer(a, N)

    def res(a):
        FA, FB = F_AB(a)
        PA = orc_mod.neohooke(FA.ravel(), mu[1], lam[1], False).reshape(3, 3)
        PB = orc_mod.neohooke(FB.ravel(), mu[0], lam[0], False).reshape(3, 3)
        return (PA - PB) @ N

    # Newton on the 3 traction-balance equations with a central-difference
    # Jacobian, stopped on the residual itself (checked below)
    a = np.zeros(3)
    for _ in range(60):
        f = res(a)
        if np.linalg.norm(f) <= 1e-15 * max(1.0, np.linalg.norm(Fb)):
            break
        J = np.empty((3, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            J[:, k] = (res(a + e) - res(a - e)) / 2e-6
        a = a - np.linalg.solve(J, f)
    FA, FB = F_AB(a)
    PA = orc_mod.neohooke(FA.ravel(), mu[1], lam[1], False).reshape(3, 3)
    assert np.linalg.norm(res(a)) <= 1e-13 * np.linalg.norm(PA @ N), "exact laminate not traction balanced"
    return FA, FB, c, line


orc_mod = None


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("kspace", [0, 1])
def test_layered_laminate_is_exact(orc, axis, kspace):
    global orc_mod
    orc_mod = orc
    n = [4, 4, 4]
    # the spectral scheme drops Nyquist modes (k := 0 there), and a layered
    # field along an even axis has one: take an odd layer count for it
    n[axis] = 8 if kspace == 0 else 9
    p = ms.layered(tuple(n), axis=axis, m_incl=3, c_boxel=0.37)
    r = orc.solve(p, dict(solver=1, kspace=kspace, **TIGHT))
    FA, FB, c, line = exact_laminate(p, axis)
    F = r["F"].reshape(9, n[2], n[1], n[0])
    F = np.moveaxis(F, 3 - axis, 1)  # layer index first after component
    for layer, ph in enumerate(line):
        want = FA if ph == 1 else (FB if ph == 0 else c * FA + (1 - c) * FB)
        got = F[:, layer].reshape(9, -1)
        assert np.allclose(got, want.reshape(9, 1), atol=1e-10), (layer, ph)
    # boxel internal phases equal the laminate's pure phases
    N = np.zeros(3)
    N[axis] = 1.0
    a = r["a"][0]
    Fbox = c * FA + (1 - c) * FB
    assert np.allclose(Fbox + np.outer(a, N) / c, FA, atol=1e-9)
    ct = (3 + c) / n[axis]
    PA = orc.neohooke(FA.ravel(), p["mu"][1], p["lam"][1], False)
    PB = orc.neohooke(FB.ravel(), p["mu"][0], p["lam"][0], False)
    assert np.allclose(r["Pbar"][-1], ct * PA + (1 - ct) * PB, atol=1e-11)


def brute_force(orc, p, grad):
    """Newton with least squares on the displacement form: F = Fbar + B u,
    equilibrium B^T P(F) = 0."""
    n = p["n"]
    V = n[0] * n[1] * n[2]
    B = np.zeros((9 * V, 3 * V))
    for q in range(3 * V):
        e = np.zeros(3 * V)
        e[q] = 1.0
        B[:, q] = grad(e.reshape(3, n[2], n[1], n[0])).reshape(-1)
    u = np.zeros(3 * V)
    a = None
    Fb = p["Fbar"].reshape(9, 1)
    for it in range(40):
        F = Fb + (B @ u).reshape(9, V)
        P, a, A = orc.constitutive_field(p, F, a=a, tangent=True)
        r = B.T @ P.reshape(-1)
        if np.linalg.norm(r) < 1e-13:
            break
        # K = B^T blockdiag(A_v) B with field ordering [c][v]
        Ab = np.zeros((9 * V, 9 * V))
        for i in range(9):
            for j in range(9):
                Ab[i * V:(i + 1) * V, j * V:(j + 1) * V] = np.diag(A[:, i, j])
        K = B.T @ Ab @ B
        du = np.linalg.lstsq(K, -r, rcond=1e-12)[0]
        u += du
    F = Fb + (B @ u).reshape(9, V)
    P, a = orc.constitutive_field(p, F, a=a)
    return F, P


@pytest.mark.slow
@pytest.mark.parametrize("kspace", [0, 1, 2])
def test_brute_force_4cubed(orc, kspace):
    p = ms.random_boxels((4, 4, 4), seed=21, boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
    l = p["l"]
    n = p["n"]
    h = [l[j] / n[j] for j in range(3)]
    if kspace == 0:
        grad = lambda U: hex8r_gradient(U, h)
    elif kspace == 1:
        grad = lambda U: spectral_gradient(U, l)
    else:
        grad = lambda U: staggered_gradient(U, h)
    F_bf, P_bf = brute_force(orc, p, grad)
    r = orc.solve(p, dict(solver=1, kspace=kspace, **TIGHT))
    assert np.allclose(r["F"], F_bf, atol=1e-10)
    assert np.allclose(r["Pbar"][-1], P_bf.mean(axis=1), atol=1e-11)


def test_hill_mandel_and_solvers_agree(orc):
    p = ms.centred_sphere((12, 12, 12), 0.2, 10.0, np.diag([1.04, 1.0, 0.99]) + 0.02 * np.eye(3)[[1, 0, 2]], 2)
    r1 = orc.solve(p, dict(solver=1, **TIGHT))
    r0 = orc.solve(p, dict(solver=0, tol=1e-11, max_iter=5000))
    F, P = r1["F"], r1["P"]
    hm = np.mean(np.sum(P * F, axis=0))
    assert abs(hm - np.dot(r1["Pbar"][-1], p["Fbar"])) < 1e-11
    assert np.allclose(r0["Pbar"], r1["Pbar"], atol=1e-9)
    assert np.allclose(r0["F"], r1["F"], atol=1e-8)


def test_phase_averages_split_the_mean_stress(orc):
    """Sec. 6.2 phase averages: the volume-weighted sum of Pbar_- and Pbar_+ is
    Pbar (P_box = c+ P+ + c- P-); a layered laminate has the exact laminate
    phase stresses as its phase averages; with one phase, Pbar_+- = Pbar."""
    p = ms.random_boxels((6, 5, 4), seed=31, boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
    r = orc.solve(p, dict(solver=1, **TIGHT))
    pa = orc.phase_averages(p, r["F"], r["a"])
    phase = np.asarray(p["phase"]).ravel()
    c = np.asarray(p["boxel_c"])
    vol_p = (phase == 1).sum() + c.sum()
    vol_m = (phase == 0).sum() + (1 - c).sum()
    assert np.allclose((vol_m * pa[0] + vol_p * pa[1]) / phase.size, r["Pbar"][-1], atol=1e-12)
    # layered along x: every inclusion layer carries the same stress, so does every matrix layer
    q = ms.layered((8, 4, 4), axis=0, m_incl=3, c_boxel=0.4, contrast=10.0, Fbar=np.eye(3) + 0.05, n_steps=1)
    rq = orc.solve(q, dict(solver=1, **TIGHT))
    Pq = rq["P"].reshape(9, 4, 4, 8)
    paq = orc.phase_averages(q, rq["F"], rq["a"])
    ph = np.asarray(q["phase"]).reshape(4, 4, 8)
    assert np.allclose(paq[1], Pq[:, ph == 1].mean(1), atol=1e-11)
    assert np.allclose(paq[0], Pq[:, ph == 0].mean(1), atol=1e-11)
    h = ms.homogeneous((4, 4, 4), Fbar=np.eye(3) + 0.03)
    rh = orc.solve(h, dict(solver=1, **TIGHT))
    pah = orc.phase_averages(h, rh["F"], rh["a"])
    assert np.allclose(pah[0], rh["Pbar"][-1], atol=1e-13)
    assert np.all(pah[1] == 0)


@pytest.mark.parametrize("k", [0, 1])
def test_nonlinear_cg_reaches_the_newton_solution(orc, k):
    """Nonlinear CG (Sec. 3): its first iteration of a load step is the basic
    scheme's; converged, it reaches the state Newton-CG reaches (the discrete
    equilibrium is unique), in far fewer iterations than the basic scheme."""
    p = [ms.centred_sphere((12, 12, 12), 0.2, 10.0, np.diag([1.04, 1.0, 0.99]), 2),
         ms.random_boxels((12, 6, 9), seed=7, contrast=10.0, n_steps=2)][k]
    r0 = orc.solve(p, dict(solver=0, fixed_iter=1))
    r2 = orc.solve(p, dict(solver=2, fixed_iter=1))
    assert np.array_equal(r0["F"], r2["F"])
    rn = orc.solve(p, dict(solver=2, tol=1e-10, max_iter=5000))
    rN = orc.solve(p, dict(solver=1, tol=1e-10))
    rb = orc.solve(p, dict(solver=0, tol=1e-10, max_iter=20000))
    assert np.allclose(rn["F"], rN["F"], atol=1e-8)
    assert np.allclose(rn["Pbar"], rN["Pbar"], atol=1e-10)
    assert 3 * rn["iters"].sum() < rb["iters"].sum()
