"""Pins of the oracle's compressible Neo-Hookean law (paper Sec. 6.1).

The energy below is written from the paper's formula
W = lam/2 (ln J)^2 - mu ln J + mu/2 (tr C - 3); P and the tangent are checked
against its numerical derivatives, plus closed forms at F = I and objectivity.
"""
import numpy as np
import pytest


def W_paper(F, mu, lam):
    F = F.reshape(3, 3)
    J = np.linalg.det(F)
    return 0.5 * lam * np.log(J) ** 2 - mu * np.log(J) + 0.5 * mu * (np.trace(F.T @ F) - 3.0)


def rand_F(rng, s=0.3):
    while True:
        F = np.eye(3) + rng.uniform(-s, s, (3, 3))
        if np.linalg.det(F) > 0.3:
            return F


def test_zero_stress_at_identity(orc):
    P, A = orc.neohooke(np.eye(3).ravel(), 1.7, 2.3)
    assert np.max(np.abs(P)) == 0.0


def test_tangent_at_identity_is_isotropic(orc):
    mu, lam = 1.7, 2.3
    _, A = orc.neohooke(np.eye(3).ravel(), mu, lam)
    d = np.eye(3)
    ref = (lam * np.einsum("ij,kl->ijkl", d, d) + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))
    assert np.allclose(A, ref.reshape(9, 9), atol=1e-15)


def test_stress_is_energy_derivative(orc):
    rng = np.random.default_rng(1)
    for _ in range(10):
        F = rand_F(rng)
        mu, lam = rng.uniform(0.5, 5), rng.uniform(0.0, 10)
        P = orc.neohooke(F.ravel(), mu, lam, tangent=False)
        h = 1e-6
        Pfd = np.zeros(9)
        for q in range(9):
            e = np.zeros(9)
            e[q] = h
            Pfd[q] = (W_paper(F.ravel() + e, mu, lam) - W_paper(F.ravel() - e, mu, lam)) / (2 * h)
        assert np.allclose(P, Pfd, rtol=1e-7, atol=1e-8)
        # the oracle's own energy matches the paper formula
        assert abs(orc.neohooke_energy(F.ravel(), mu, lam) - W_paper(F, mu, lam)) < 1e-13


def test_tangent_is_stress_derivative_and_major_symmetric(orc):
    rng = np.random.default_rng(2)
    for _ in range(10):
        F = rand_F(rng)
        mu, lam = rng.uniform(0.5, 5), rng.uniform(0.0, 10)
        P, A = orc.neohooke(F.ravel(), mu, lam)
        h = 1e-6
        Afd = np.zeros((9, 9))
        for q in range(9):
            e = np.zeros(9)
            e[q] = h
            Afd[:, q] = (orc.neohooke(F.ravel() + e, mu, lam, False) - orc.neohooke(F.ravel() - e, mu, lam, False)) / (2 * h)
        assert np.allclose(A, Afd, rtol=1e-7, atol=1e-7)
        assert np.allclose(A, A.T, atol=1e-13)


def test_objectivity(orc):
    rng = np.random.default_rng(3)
    for _ in range(10):
        F = rand_F(rng)
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
        P = orc.neohooke(F.ravel(), 2.0, 3.0, False).reshape(3, 3)
        PQ = orc.neohooke((Q @ F).ravel(), 2.0, 3.0, False).reshape(3, 3)
        assert np.allclose(PQ, Q @ P, atol=1e-13)


def test_inadmissible_raises(orc):
    F = np.diag([-1.0, 1.0, 1.0])
    with pytest.raises(ValueError):
        orc.neohooke(F.ravel(), 1.0, 1.0)
