"""Pins of the coarse-graining oracle (normal detection, paper Sec. 5)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def nrm():
    from oracle import normals

    return normals


@pytest.fixture(scope="module")
def ball():
    from paper_2204_13624_gb300 import microstructure as ms

    return ms.fine_ball_image(256, 0.4)


def test_paper_composite_voxel_count(nrm, ball):
    # Sec. 6.2: the 256^3 ball coarse-grained to 32^3 has 2624 composite voxels
    phase, idx, c, N = nrm.block_normals(ball, (8, 8, 8), (1, 1, 1))
    assert int((phase == 2).sum()) == 2624 == idx.size


def test_volume_fractions_are_voxel_counts(nrm):
    rng = np.random.default_rng(0)
    chi = (rng.random((12, 16, 20)) < 0.3).astype(np.uint8)
    phase, idx, c, N = nrm.block_normals(chi, (4, 4, 3), (1, 1, 1))
    cnt = chi.reshape(4, 3, 4, 4, 5, 4).sum(axis=(1, 3, 5))  # [K, J, I] inclusion voxels per block
    frac = cnt / 48.0
    mixed = (cnt > 0) & (cnt < 48)
    assert np.array_equal(np.flatnonzero(mixed.ravel()), idx)
    assert np.allclose(c, frac.ravel()[idx], rtol=0, atol=1e-15)
    assert np.array_equal(phase.ravel() == 1, (cnt == 48).ravel())


def test_stencil_weights_equal_the_direct_periodic_stencil(nrm):
    rng = np.random.default_rng(1)
    chi = (rng.random((6, 8, 10)) < 0.5).astype(np.float64)
    h = (0.7, 1.3, 2.1)
    r = (h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2])
    direct = np.zeros_like(chi)
    for axis, ri in zip((2, 1, 0), r):
        direct += ri * (np.roll(chi, 1, axis) - 2 * chi + np.roll(chi, -1, axis))
    assert np.allclose(nrm.stencil_weights(chi, h), np.abs(direct), atol=1e-12)


@pytest.mark.parametrize("b,h", [((8, 8, 8), (1, 1, 1)), ((16, 8, 4), (1, 1, 1)), ((8, 8, 4), (1.0, 1.0, 2.0))])
def test_planar_interface_normal_is_recovered(nrm, b, h):
    from paper_2204_13624_gb300 import microstructure as ms

    nt = np.array([0.48, 0.6, 0.64])
    chi = ms.fine_plane_image((64, 64, 64), nt, 3.3, h)
    phase, idx, c, N = nrm.block_normals(chi, b, h)
    assert idx.size > 10
    # The half space is not periodic: its wrap at the faces of the box makes
    # further interfaces there, so only boxels off the box faces are checked.
    nc = (64 // b[0], 64 // b[1], 64 // b[2])
    I, J, K = idx % nc[0], (idx // nc[0]) % nc[1], idx // (nc[0] * nc[1])
    inner = (I > 0) & (I < nc[0] - 1) & (J > 0) & (J < nc[1] - 1) & (K > 0) & (K < nc[2] - 1)
    dots = N[inner] @ nt
    assert inner.sum() > 40
    assert np.all(dots > 0.75)  # out of the inclusion (the negative side)
    # Boxels the plane cuts across (not only at a corner, where a few staircase
    # voxels carry the weights) recover the normal to the staircase's accuracy.
    cut = inner & (c > 0.1) & (c < 0.9)
    assert cut.sum() > 20
    assert np.all(N[cut] @ nt > 0.998)
    assert np.mean(N[cut] @ nt) > 0.999
    if b == (16, 8, 4):
        # non-equiaxed boxels: the barycentre normal is far off (Fig. normal:kabel2)
        _, _, _, Nk = nrm.block_normals(chi, b, h, "kabel")
        assert np.mean(Nk[cut] @ nt) < 0.9


def test_ball_normals_point_out_and_beat_the_barycentre_normals(nrm, ball):
    """Sec. 5.2 / Sec. 6.2: the Laplacian normals are closer to the radial
    direction than the barycentre normals, for equiaxed voxels and more so for
    non-equiaxed boxels."""
    for b in [(8, 8, 8), (32, 16, 8)]:
        errs = {}
        for method in ("laplace", "kabel"):
            phase, idx, c, N = nrm.block_normals(ball, b, (1, 1, 1), method)
            nc = (256 // b[0], 256 // b[1], 256 // b[2])
            I, J, K = idx % nc[0], (idx // nc[0]) % nc[1], idx // (nc[0] * nc[1])
            cen = np.stack([(I + 0.5) * b[0], (J + 0.5) * b[1], (K + 0.5) * b[2]], 1) - 128.0
            radial = cen / np.linalg.norm(cen, axis=1)[:, None]
            cosang = np.clip(np.sum(N * radial, 1), -1, 1)
            assert np.all(cosang > 0)  # out of the ball
            errs[method] = float(np.mean(np.arccos(cosang)))
        assert errs["laplace"] < errs["kabel"]
        if b == (32, 16, 8):
            assert errs["laplace"] < 0.5 * errs["kabel"]


def test_normal_minimises_the_weighted_squared_distance(nrm, ball):
    """Brute force over directions: N minimises sum_w (N . x)^2 over unit
    vectors (the weighted least-squares plane of Sec. 5.2)."""
    b = (32, 16, 8)
    phase, idx, c, N = nrm.block_normals(ball, b, (1, 1, 1))
    w = nrm.stencil_weights(ball, (1, 1, 1))
    rng = np.random.default_rng(3)
    d = rng.normal(size=(20000, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    for t in rng.choice(idx.size, 6, replace=False):
        M = nrm.moment_tensor(ball, b, (1, 1, 1), int(idx[t]), w)
        q = np.einsum("ni,ij,nj->n", d, M, d)
        qn = float(N[t] @ M @ N[t])
        assert abs(np.linalg.norm(N[t]) - 1.0) < 1e-12
        assert qn <= q.min() * (1 + 1e-12)


def test_weights_count_the_neighbours_of_the_other_phase(nrm):
    """For a binary image every second difference of a voxel has the sign of
    -chi (or vanishes), so |S * chi| = sum_i r_i (number of the two
    neighbours along e_i in the other phase)."""
    rng = np.random.default_rng(4)
    chi = (rng.random((10, 12, 14)) < 0.4).astype(np.uint8)
    h = (0.9, 1.7, 0.6)
    r = (h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2])
    cnt = np.zeros(chi.shape)
    for axis, ri in zip((2, 1, 0), r):
        for sh in (1, -1):
            cnt += ri * (np.roll(chi, sh, axis) != chi)
    assert np.allclose(nrm.stencil_weights(chi, h), cnt, rtol=1e-13, atol=1e-12)


def test_barycentre_normal_and_its_degenerate_case(nrm):
    rng = np.random.default_rng(5)
    h = (1.0, 0.5, 2.0)
    chi = (rng.random((8, 16, 12)) < 0.5).astype(np.uint8)
    # coarse voxel 0 holds a centred 2x2x2 inclusion: the barycentres coincide
    chi[0:4, 0:4, 0:4] = 0
    chi[1:3, 1:3, 1:3] = 1
    b = (4, 4, 4)
    _, idx, _, Nk = nrm.block_normals(chi, b, h, "kabel")
    _, idx2, _, Nl = nrm.block_normals(chi, b, h, "laplace")
    assert np.array_equal(idx, idx2) and idx[0] == 0
    for t, ci in enumerate(idx):
        Nt = nrm.barycentre_normal(chi, b, h, int(ci))
        if np.any(Nt != 0):
            assert np.allclose(Nk[t], Nt, atol=1e-14)
    assert np.all(nrm.barycentre_normal(chi, b, h, 0) == 0)
    # undefined Ntilde: both methods give the Laplacian normal (up to sign),
    # an eigenvector of the smallest eigenvalue of M; for the centred cube M
    # is a multiple of the identity only when h is isotropic, not here
    M = nrm.moment_tensor(chi, b, h, 0)
    lam = np.linalg.eigvalsh(M)
    assert abs(abs(Nk[0] @ Nl[0]) - 1) < 1e-12
    assert Nl[0] @ M @ Nl[0] <= lam[0] * (1 + 1e-12)


@pytest.mark.parametrize("method", ["laplace", "kabel"])
def test_windowed_boxels_equal_the_whole_image_pass(nrm, method):
    """block_normals_at (direct stencil on each boxel's periodic halo) agrees
    with block_normals (Fourier-domain stencil over the image)."""
    rng = np.random.default_rng(6)
    chi = (rng.random((9, 12, 20)) < 0.45).astype(np.uint8) * 7  # any nonzero byte is inclusion
    b, h = (5, 4, 3), (1.2, 0.8, 1.0)
    phase, idx, c, N = nrm.block_normals(chi, b, h, method)
    allc = np.arange(phase.size)
    ph2, c2, N2 = nrm.block_normals_at(chi, b, h, allc, method)
    assert np.array_equal(ph2, phase.ravel())
    assert np.array_equal(c2[idx], c)
    assert np.allclose(N2[idx], N, atol=1e-12)


@pytest.mark.parametrize("b", [16, 32])
def test_coarser_composite_voxel_counts(nrm, ball, b):
    """The same ball coarse-grained to 16^3 and 8^3: the oracle's composite
    voxels (mixed blocks of the fine image) are the mixed blocks counted by the
    input generator's independent block-by-block scan (704 and 224)."""
    from paper_2204_13624_gb300 import microstructure as ms

    phase, idx, c, N = nrm.block_normals(ball, (b, b, b), (1, 1, 1))
    assert int((phase == 2).sum()) == idx.size == ms.fine_sphere_block_count(256, 256 // b, 0.4)
    assert idx.size == {16: 704, 32: 224}[b]
