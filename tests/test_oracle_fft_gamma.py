"""Pins of the oracle's FFT and Green operator (paper Sec. 3, Eqs. nonlinearLSE, Gamma0).

* FFT: against the DFT written as a matrix, against numpy's FFT, Parseval
  and the round trip.
* G = mu0 Gamma0: zero at xi = 0, Hermitian and idempotent per frequency,
  compatible output (rows parallel to k), zero mean, and -- the strongest
  pin -- it leaves unchanged the real-space gradient of a periodic
  displacement: for the rotated (HEX8R) scheme the gradient is built here
  from the 8 voxel-corner displacements, for the spectral scheme from a band
  limited trigonometric polynomial.
"""
import numpy as np
import pytest


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 16, 18, 24, 27, 32, 36, 48, 64, 96])
def test_fft1_matches_dft_matrix(orc, n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    j = np.arange(n)
    Wm = np.exp(-2j * np.pi * np.outer(j, j) / n)
    assert np.allclose(orc.fft1(x, -1), Wm @ x, atol=1e-12 * n)
    assert np.allclose(orc.fft1(x, +1), np.conj(Wm) @ x, atol=1e-12 * n)


@pytest.mark.parametrize("shape", [(4, 6, 8), (3, 5, 2), (8, 8, 8), (12, 9, 16)])
def test_fft3_matches_numpy_parseval_roundtrip(orc, shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    X = orc.fft3(x, -1)
    assert np.allclose(X, np.fft.fftn(x), atol=1e-11)
    assert abs(np.sum(np.abs(X) ** 2) / x.size - np.sum(np.abs(x) ** 2)) < 1e-10 * np.sum(np.abs(x) ** 2)
    back = orc.fft3(X, +1) / x.size
    assert np.allclose(back, x, atol=1e-13)


def hex8r_gradient(U, h):
    """U[3][n3][n2][n1] nodal displacements at voxel corners (node (i,j,k) is
    the lower corner of voxel (i,j,k)).  Gradient at voxel centres = mean of
    the 4 edge differences parallel to each axis."""
    ax_of = {0: 3, 1: 2, 2: 1}  # x, y, z -> array axis
    H = np.zeros((3, 3) + U.shape[1:])
    for J in range(3):
        a = ax_of[J]
        D = (np.roll(U, -1, axis=a) - U) / h[J]
        o = [ax_of[m] for m in range(3) if m != J]
        H[:, J] = 0.25 * (D + np.roll(D, -1, axis=o[0]) + np.roll(D, -1, axis=o[1])
                          + np.roll(np.roll(D, -1, axis=o[0]), -1, axis=o[1]))
    return H.reshape(9, -1)


def spectral_gradient(U, l):
    n3, n2, n1 = U.shape[1:]
    Uh = np.fft.fftn(U, axes=(1, 2, 3))
    ks = []
    for n, L in ((n1, l[0]), (n2, l[1]), (n3, l[2])):
        f = np.fft.fftfreq(n, d=1.0 / n)
        k = 2 * np.pi * f / L
        if n % 2 == 0:
            k[n // 2] = 0.0
        ks.append(k)
    kx = ks[0][None, None, :]
    ky = ks[1][None, :, None]
    kz = ks[2][:, None, None]
    H = np.zeros((3, 3, n3, n2, n1))
    for i in range(3):
        for J, kk in enumerate((kx, ky, kz)):
            H[i, J] = np.real(np.fft.ifftn(1j * kk * Uh[i]))
    return H.reshape(9, -1)


def staggered_gradient(U, h):
    """App. A, Eq. gradient_operator: F_aa = D_a^+ U_a, F_aB = D_B^- U_a (B != a),
    D^+ phi[I] = (phi[I + e] - phi[I]) / h, D^- phi[I] = (phi[I] - phi[I - e]) / h,
    periodic; U[a][n3][n2][n1]."""
    ax_of = {0: 3, 1: 2, 2: 1}
    H = np.zeros((3, 3) + U.shape[1:])
    for a in range(3):
        for B in range(3):
            ax = ax_of[B] - 1  # axis of U[a]
            if a == B:
                H[a, B] = (np.roll(U[a], -1, axis=ax) - U[a]) / h[B]
            else:
                H[a, B] = (U[a] - np.roll(U[a], 1, axis=ax)) / h[B]
    return H.reshape(9, -1)


def band_limit(U):
    Uh = np.fft.fftn(U, axes=(1, 2, 3))
    for ax in (1, 2, 3):
        n = U.shape[ax]
        if n % 2 == 0:
            idx = [slice(None)] * 4
            idx[ax] = n // 2
            Uh[tuple(idx)] = 0.0
    return np.real(np.fft.ifftn(Uh, axes=(1, 2, 3)))


SHAPES = [((4, 4, 4), (1.0, 1.0, 1.0)), ((6, 4, 8), (1.0, 0.5, 2.0)), ((3, 6, 9), (0.3, 1.0, 1.5))]


@pytest.mark.parametrize("n,l", SHAPES)
def test_rotated_G_keeps_hex8r_gradients(orc, n, l):
    rng = np.random.default_rng(7)
    U = rng.normal(size=(3, n[2], n[1], n[0]))
    h = [l[j] / n[j] for j in range(3)]
    X = hex8r_gradient(U, h)
    Y, ss = orc.apply_G(X, n, l, orc.ROTATED)
    assert np.allclose(Y, X, atol=1e-12 * np.abs(X).max())
    assert abs(ss - np.sum(X * X)) < 1e-10 * np.sum(X * X)


@pytest.mark.parametrize("n,l", SHAPES)
def test_spectral_G_keeps_spectral_gradients(orc, n, l):
    rng = np.random.default_rng(8)
    U = band_limit(rng.normal(size=(3, n[2], n[1], n[0])))
    X = spectral_gradient(U, l)
    Y, _ = orc.apply_G(X, n, l, orc.SPECTRAL)
    assert np.allclose(Y, X, atol=1e-12 * np.abs(X).max())


@pytest.mark.parametrize("n,l", SHAPES)
def test_staggered_G_keeps_staggered_gradients(orc, n, l):
    rng = np.random.default_rng(11)
    U = rng.normal(size=(3, n[2], n[1], n[0]))
    h = [l[j] / n[j] for j in range(3)]
    X = staggered_gradient(U, h)
    Y, ss = orc.apply_G(X, n, l, orc.STAGGERED)
    assert np.allclose(Y, X, atol=1e-12 * np.abs(X).max())
    # and removes what is orthogonal to every staggered gradient: a field
    # whose rows have zero staggered divergence (adjoint of Grad) is mapped to 0
    Z = rng.normal(size=(9, n[0] * n[1] * n[2]))
    GZ, _ = orc.apply_G(Z, n, l, orc.STAGGERED)
    R = Z - GZ
    # R is orthogonal to all gradients: <R, Grad e_q> = 0 for unit displacements
    for q in rng.choice(3 * n[0] * n[1] * n[2], 12, replace=False):
        e = np.zeros(3 * n[0] * n[1] * n[2])
        e[q] = 1.0
        g = staggered_gradient(e.reshape(3, n[2], n[1], n[0]), h)
        assert abs(np.sum(R * g)) < 1e-10 * np.abs(Z).max()


@pytest.mark.parametrize("kspace", [0, 1, 2])
@pytest.mark.parametrize("n,l", SHAPES)
def test_G_is_zero_mean_projector(orc, kspace, n, l):
    rng = np.random.default_rng(9)
    V = n[0] * n[1] * n[2]
    X = rng.normal(size=(9, V))
    Y, _ = orc.apply_G(X, n, l, kspace)
    Z, _ = orc.apply_G(Y, n, l, kspace)
    assert np.allclose(Z, Y, atol=1e-12)
    assert np.allclose(Y.mean(axis=1), 0.0, atol=1e-13)
    # orthogonal projector: <X - GX, GX> = 0
    assert abs(np.sum((X - Y) * Y)) < 1e-10 * np.sum(X * X)
    # the same operator assembled here from numpy's FFT and the oracle's
    # per-frequency matrices: real output, equal values
    Xh = np.fft.fftn(X.reshape(9, n[2], n[1], n[0]), axes=(1, 2, 3))
    Yh = np.zeros_like(Xh)
    for k3 in range(n[2]):
        for k2 in range(n[1]):
            for k1 in range(n[0]):
                Gm = orc.gamma_matrix(kspace, n, l, (k1, k2, k3))
                Yh[:, k3, k2, k1] = Gm @ Xh[:, k3, k2, k1]
    y = np.fft.ifftn(Yh, axes=(1, 2, 3))
    assert np.max(np.abs(y.imag)) < 1e-13
    assert np.allclose(y.real.reshape(9, V), Y, atol=1e-13)


@pytest.mark.parametrize("kspace", [0, 1, 2])
def test_gamma_matrix_properties(orc, kspace):
    rng = np.random.default_rng(10)
    n, l = (6, 4, 8), (1.0, 0.7, 1.3)
    assert np.all(orc.gamma_matrix(kspace, n, l, (0, 0, 0)) == 0)
    for _ in range(20):
        xi = tuple(int(rng.integers(0, m)) for m in n)
        Gm = orc.gamma_matrix(kspace, n, l, xi)
        ks = [orc.kvec_row(kspace, n, l, xi, a) for a in range(3)]
        if kspace != 2:
            assert all(np.array_equal(ks[a], orc.kvec(kspace, n, l, xi)) for a in range(3))
        if np.all(ks[0] == 0):
            assert np.all(Gm == 0)
            continue
        assert np.allclose(Gm, Gm.conj().T, atol=1e-14)
        assert np.allclose(Gm @ Gm, Gm, atol=1e-13)
        x = rng.normal(size=9) + 1j * rng.normal(size=9)
        y = (Gm @ x).reshape(3, 3)
        # compatibility: y_iJ k_iK = y_iK k_iJ (row i is a multiple of k_i)
        for i in range(3):
            assert np.allclose(y[i][:, None] * ks[i][None, :], ks[i][:, None] * y[i][None, :], atol=1e-12)
        # Hermitian symmetry of the symbol: G(-xi) = conj G(xi)
        xm = tuple((-xi[j]) % n[j] for j in range(3))
        assert np.allclose(orc.gamma_matrix(kspace, n, l, xm), np.conj(Gm), atol=1e-14)


def test_rotated_nyquist_null_modes(orc):
    n, l = (4, 4, 4), (1.0, 1.0, 1.0)
    # two or more Nyquist indices -> k = 0 exactly
    for xi in [(2, 2, 0), (2, 0, 2), (0, 2, 2), (2, 2, 2), (2, 2, 1)]:
        assert np.all(orc.kvec(orc.ROTATED, n, l, xi) == 0)
    k = orc.kvec(orc.ROTATED, n, l, (2, 1, 0))
    assert k[0] != 0 and k[1] == 0 and k[2] == 0
