"""The identity behind the displacement form of the rotated Green operator
(the FP32 Krylov passes evaluate G that way): with the rotated symbol
k_J = (2 i / h_J) sin(theta_J / 2) e^{i (theta_1 + theta_2 + theta_3) / 2}
prod_{m != J} cos(theta_m / 2) (the cosine zero at a Nyquist index; Sec. 3,
the rotated scheme), row i of G X is the HEX8R gradient -- the difference
along each edge of a voxel parallel to axis J, averaged over its 4 such
edges, divided by h_J -- of the real nodal field u_i = IFFT(k^H X_i / |k|^2).

Written here with numpy's FFT and np.roll, independent of the oracle's code,
and compared with the oracle's Green operator (itself pinned in
test_oracle_fft_gamma.py) on even, odd and mixed grids with unequal cell sizes,
where a wrong phase sign, a dropped Nyquist rule or a stencil shifted the
wrong way fails."""
import numpy as np
import pytest


def disp_form(X, n, l):
    n1, n2, n3 = n
    Xh = np.fft.fftn(X.reshape(9, n3, n2, n1), axes=(1, 2, 3))
    idx = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    ax = [idx[2], idx[1], idx[0]]  # unsigned indices along x, y, z
    nn = [n1, n2, n3]
    h = [l[j] / nn[j] for j in range(3)]
    half = [np.pi * ax[j] / nn[j] for j in range(3)]  # theta / 2
    cos = [np.where(2 * ax[j] == nn[j], 0.0, np.cos(half[j])) for j in range(3)]
    P = np.exp(1j * (half[0] + half[1] + half[2]))
    k = []
    for J in range(3):
        kk = (2j / h[J]) * np.sin(half[J]) * P
        for m in range(3):
            if m != J:
                kk = kk * cos[m]
        k.append(kk)
    k2 = sum(np.abs(kk) ** 2 for kk in k)
    Y = np.zeros((9, n3, n2, n1))
    for i in range(3):
        s = sum(np.conj(k[L]) * Xh[3 * i + L] for L in range(3))
        s = np.where(k2 > 0, s / np.where(k2 > 0, k2, 1.0), 0.0)
        u = np.fft.ifftn(s)
        assert np.max(np.abs(u.imag)) <= 1e-12 * max(np.max(np.abs(u.real)), 1e-300)
        u = u.real

        def at(a):  # u at the corner offset a = (ax, ay, az)
            return np.roll(u, (-a[2], -a[1], -a[0]), axis=(0, 1, 2))

        for J in range(3):
            acc = 0.0
            for a in [(a0, a1, a2) for a0 in (0, 1) for a1 in (0, 1) for a2 in (0, 1)]:
                if a[J]:
                    continue
                b = list(a)
                b[J] = 1
                acc = acc + at(b) - at(a)
            Y[3 * i + J] = acc / (4 * h[J])
    return Y.reshape(9, -1)


@pytest.mark.parametrize("n", [(6, 5, 4), (8, 8, 8), (12, 9, 10), (7, 6, 3), (16, 4, 12)])
def test_rotated_operator_is_hex8r_gradient_of_nodal_field(orc, n):
    rng = np.random.default_rng(sum(n))
    l = (1.0, 0.8, 1.3)
    X = rng.standard_normal((9, int(np.prod(n))))
    Yo, _ = orc.apply_G(X, n, l, orc.ROTATED)
    Yd = disp_form(X, n, l)
    assert np.max(np.abs(Yd - Yo)) <= 1e-12 * np.max(np.abs(Yo))


def test_other_schemes_are_not_this_gradient(orc):
    """The identity is particular to the rotated scheme: the spectral and
    staggered operators differ from it (guards against a vacuous check)."""
    n, l = (8, 6, 10), (1.0, 1.0, 1.0)
    X = np.random.default_rng(5).standard_normal((9, int(np.prod(n))))
    Yd = disp_form(X, n, l)
    for ks in (1, 2):
        Yo, _ = orc.apply_G(X, n, l, ks)
        assert np.max(np.abs(Yd - Yo)) > 1e-3 * np.max(np.abs(Yo))


def hex8r_adjoint(X, n, l):
    """w_i(node) = sum over the 8 voxels v = node - b (b in {0,1}^3) of
    sum_J X_iJ(v) s(b_J) / (4 h_J), s(1) = +1, s(0) = -1: the adjoint of the
    HEX8R gradient (whose coefficient of u(v + b) in F_iJ(v) is s(b_J) / (4 h_J))."""
    n1, n2, n3 = n
    h = [l[j] / n[j] for j in range(3)]
    X = X.reshape(3, 3, n3, n2, n1)
    w = np.zeros((3, n3, n2, n1))
    for b in [(b0, b1, b2) for b0 in (0, 1) for b1 in (0, 1) for b2 in (0, 1)]:
        for J in range(3):
            s = 1.0 if b[J] else -1.0
            # X at v = node - b, seen from the node: roll by +b
            w += s / (4 * h[J]) * np.roll(X[:, J], (b[2], b[1], b[0]), axis=(1, 2, 3))
    return w


def div_form(X, n, l):
    """G X = D (D^T D)^+ D^T X with both stencils in real space and only the
    real scalar 1 / |kr|^2 in Fourier space (kr: the real rotated symbol)."""
    n1, n2, n3 = n
    w = hex8r_adjoint(X, n, l)
    idx = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    ax = [idx[2], idx[1], idx[0]]
    nn = [n1, n2, n3]
    h = [l[j] / nn[j] for j in range(3)]
    sa = [(2 / h[j]) * np.sin(np.pi * ax[j] / nn[j]) for j in range(3)]
    sb = [np.where(2 * ax[j] == nn[j], 0.0, np.cos(np.pi * ax[j] / nn[j])) for j in range(3)]
    kr2 = sum((sa[J] * np.prod([sb[m] for m in range(3) if m != J], axis=0)) ** 2 for J in range(3))
    inv = np.where(kr2 > 0, 1.0 / np.where(kr2 > 0, kr2, 1.0), 0.0)
    Y = np.zeros((9, n3, n2, n1))
    for i in range(3):
        u = np.fft.ifftn(np.fft.fftn(w[i]) * inv)
        assert np.max(np.abs(u.imag)) <= 1e-12 * max(np.max(np.abs(u.real)), 1e-300)
        u = u.real

        def at(a):
            return np.roll(u, (-a[2], -a[1], -a[0]), axis=(0, 1, 2))

        for J in range(3):
            acc = 0.0
            for a in [(a0, a1, a2) for a0 in (0, 1) for a1 in (0, 1) for a2 in (0, 1)]:
                acc = acc + (1.0 if a[J] else -1.0) * at(a)
            Y[3 * i + J] = acc / (4 * h[J])
    return Y.reshape(9, -1)


@pytest.mark.parametrize("n", [(6, 5, 4), (8, 8, 8), (12, 9, 10), (7, 6, 3), (16, 4, 12)])
def test_rotated_operator_is_gradient_of_inverse_laplacian_of_adjoint(orc, n):
    """G = D (D^T D)^+ D^T: the adjoint stencil in real space, then only a real
    scalar per frequency -- the form the tangent pass and scalar z-pass use."""
    rng = np.random.default_rng(3 + sum(n))
    l = (0.9, 1.2, 1.1)
    X = rng.standard_normal((9, int(np.prod(n))))
    Yo, _ = orc.apply_G(X, n, l, orc.ROTATED)
    assert np.max(np.abs(div_form(X, n, l) - Yo)) <= 1e-12 * np.max(np.abs(Yo))


def test_adjoint_stencil_is_the_adjoint(orc):
    """<D u, X> = <u, D^T X> for random u, X (the stencils are each other's
    transposes, so a sign or shift slip in either fails here)."""
    n, l = (6, 7, 5), (1.0, 0.8, 1.3)
    rng = np.random.default_rng(11)
    X = rng.standard_normal((9, int(np.prod(n))))
    u = rng.standard_normal((3, n[2], n[1], n[0]))
    h = [l[j] / n[j] for j in range(3)]
    Du = np.zeros((9, n[2], n[1], n[0]))
    for i in range(3):
        for J in range(3):
            for a in [(a0, a1, a2) for a0 in (0, 1) for a1 in (0, 1) for a2 in (0, 1)]:
                Du[3 * i + J] += (1.0 if a[J] else -1.0) / (4 * h[J]) * np.roll(u[i], (-a[2], -a[1], -a[0]),
                                                                               axis=(0, 1, 2))
    lhs = float(np.sum(Du.reshape(9, -1) * X))
    rhs = float(np.sum(u * hex8r_adjoint(X, n, l)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
