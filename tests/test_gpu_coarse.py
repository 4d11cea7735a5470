"""GPU parity of the coarse-graining with the Sec. 5 normal detection
(combo_coarse_grain) against the oracle.

Phase codes, boxel indices and c+ are exact.  The normals are compared with a
tolerance from the eigenvalue gap of each boxel's M (Davis-Kahan: the angle
between computed and exact eigenvectors is at most the perturbation of M over
the gap).  The GPU forms M from exact integer sums; the oracle sums
nblock FP64 products, so its M is off by at most about nblock ulps of
sum w |x|^2 (the gamma_n bound of recursive summation); where the gap
is too small for that bound to mean anything, N is checked to be a unit
eigenvector of the smallest eigenvalue.  Where the barycentre normal is
undefined (coincident barycentres) the sign of the Laplacian normal is the
eigen-solver's, so the comparison is up to sign there.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def cb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    return combo


@pytest.fixture(scope="module")
def nrm():
    from oracle import normals

    return normals


def _boxel_window(chi, b, h, ci):
    """Weights, inclusion flags and positions of one boxel (direct periodic stencil)."""
    n3, n2, n1 = chi.shape
    b1, b2, b3 = b
    nc1, nc2 = n1 // b1, n2 // b2
    I, J, K = ci % nc1, (ci // nc1) % nc2, ci // (nc1 * nc2)
    xs = np.arange(I * b1 - 1, (I + 1) * b1 + 1) % n1
    ys = np.arange(J * b2 - 1, (J + 1) * b2 + 1) % n2
    zs = np.arange(K * b3 - 1, (K + 1) * b3 + 1) % n3
    win = (chi[np.ix_(zs, ys, xs)] != 0).astype(np.float64)
    c0 = win[1:-1, 1:-1, 1:-1]
    r = (h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2])
    w = np.abs(r[0] * (win[1:-1, 1:-1, :-2] + win[1:-1, 1:-1, 2:] - 2 * c0)
               + r[1] * (win[1:-1, :-2, 1:-1] + win[1:-1, 2:, 1:-1] - 2 * c0)
               + r[2] * (win[:-2, 1:-1, 1:-1] + win[2:, 1:-1, 1:-1] - 2 * c0)).ravel()
    qz, qy, qx = np.meshgrid(*(2 * np.arange(bb) + 1 - bb for bb in (b3, b2, b1)), indexing="ij")
    X = np.stack([qx.ravel() * 0.5 * h[0], qy.ravel() * 0.5 * h[1], qz.ravel() * 0.5 * h[2]], 1)
    return w, c0.ravel().astype(bool), X


def check_normals(chi, b, h, idx, N_gpu, N_or, method):
    """Per-boxel comparison of the GPU normals with the oracle's."""
    h = tuple(float(v) for v in h)
    assert N_gpu.shape == N_or.shape
    assert np.allclose(np.linalg.norm(N_gpu, axis=1), 1.0, atol=1e-13)
    worst = 0.0
    for t, ci in enumerate(np.asarray(idx)):
        w, inc, X = _boxel_window(chi, b, h, int(ci))
        dc = X[~inc].mean(0) - X[inc].mean(0)
        qsum = (np.round(2 * X[inc] / np.array(h))).sum(0)
        nt_defined = np.any(qsum != 0)
        if method == "kabel" and nt_defined:
            d = np.abs(N_gpu[t] - N_or[t]).max()
            assert d < 1e-14, (ci, N_gpu[t], N_or[t])
            continue
        P = X - (w @ X) / w.sum()
        M = (P * w[:, None]).T @ P
        scale = float(w @ (X * X).sum(1))  # sum w |x|^2 about the boxel centre
        lam = np.linalg.eigvalsh(M)
        gap = lam[1] - lam[0]
        # N is a unit eigenvector of the smallest eigenvalue (always)
        assert N_gpu[t] @ M @ N_gpu[t] - lam[0] <= 1e-12 * scale, ci
        tol = 1e-12 + (w.size + 64) * EPS * scale / max(gap, 1e-300)
        nt = dc / np.linalg.norm(dc) if nt_defined else np.zeros(3)
        undecided = (not nt_defined) or abs(nt @ N_or[t]) < 1e-9
        d = np.abs(N_gpu[t] - N_or[t]).max()
        if undecided:
            d = min(d, np.abs(N_gpu[t] + N_or[t]).max())
        if tol < 1e-3:
            assert d <= tol, (ci, d, tol, N_gpu[t], N_or[t])
            worst = max(worst, d / tol)
    return worst


def run_case(cb, nrm, chi, b, h, method, mem):
    import torch

    if mem == "device":
        out = cb.coarse_grain(torch.from_numpy(chi).cuda(), b, h, method)
        phase, idx, c, N, nb = (o.cpu().numpy() if hasattr(o, "cpu") else o for o in out)
    else:
        phase, idx, c, N, nb = cb.coarse_grain(chi, b, h, method)
    ophase, oidx, oc, oN = nrm.block_normals(chi, b, h, method)
    assert nb == oidx.size
    assert np.array_equal(phase, ophase)
    assert np.array_equal(idx, oidx)
    assert np.array_equal(c, oc)
    return check_normals(chi, b, h, idx, N, oN, method)


def _spheres(n, R, count, seed, h=(1.0, 1.0, 1.0)):
    from paper_2204_13624_gb300 import microstructure as ms

    return ms.fine_spheres_image(n, R, count, seed=seed, h=h)


CASES = [
    # (fine n, b, h, image)
    ((96, 80, 72), (8, 5, 6), (1.0, 1.5, 0.75), "spheres"),   # 16-byte loads, anisotropic h
    ((100, 48, 40), (10, 6, 8), (1.0, 1.0, 1.0), "spheres"),  # n1 % 32 != 0: byte loads
    ((160, 32, 32), (40, 8, 4), (0.5, 1.0, 1.0), "spheres"),  # boxel rows wider than a word
    ((256, 32, 16), (64, 4, 4), (1.0, 1.0, 1.0), "spheres"),  # word-aligned multi-word rows
    ((24, 16, 20), (4, 4, 5), (1.0, 1.0, 1.0), "noise"),      # many degenerate boxels
    ((12, 10, 8), (12, 10, 8), (1.0, 2.0, 3.0), "noise"),     # one coarse voxel
    ((2, 2, 2), (2, 1, 1), (1.0, 1.0, 1.0), "noise"),         # 2-voxel axes
    ((1, 4, 4), (1, 2, 2), (1.0, 1.0, 1.0), "noise"),         # 1-voxel axis
    ((64, 64, 64), (4, 4, 4), (1.0, 1.0, 1.0), "noise"),      # every coarse voxel a boxel
    ((96, 64, 48), (12, 8, 6), (1.0, 1.0, 1.0), "spheres"),   # fast path, spans across words
    ((128, 32, 24), (16, 16, 3), (1.0, 0.5, 2.0), "spheres"), # fast path, two table bytes
    ((96, 16, 16), (24, 2, 4), (1.0, 1.0, 1.0), "noise"),     # fast path, four bytes across words
    ((64, 8, 8), (1, 1, 1), (1.0, 1.0, 1.0), "noise"),        # one fine voxel per coarse voxel
]


@pytest.mark.parametrize("method", ["laplace", "kabel"])
@pytest.mark.parametrize("mem", ["host", "device"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_parity_with_the_oracle(cb, nrm, case, mem, method):
    n, b, h, kind = CASES[case]
    if kind == "spheres":
        chi = _spheres(n, 0.18 * min(n[0], n[1] * h[1] / h[0], n[2] * h[2] / h[0]), 6, seed=100 + case, h=h)
    else:
        rng = np.random.default_rng(200 + case)
        chi = (rng.random((n[2], n[1], n[0])) < 0.5).astype(np.uint8)
    run_case(cb, nrm, chi, b, h, method, mem)


@pytest.mark.parametrize("b", [(8, 8, 8), (32, 16, 8)])
@pytest.mark.parametrize("method", ["laplace", "kabel"])
def test_paper_ball_256(cb, nrm, b, method):
    """Sec. 5.2 / 6.2: the 256^3 ball of radius 0.4 L coarse-grained to 32^3
    voxels (2624 composite voxels) and to 8 x 16 x 32 boxels."""
    from paper_2204_13624_gb300 import microstructure as ms

    chi = ms.fine_ball_image(256, 0.4)
    run_case(cb, nrm, chi, b, (1.0, 1.0, 1.0), method, "device")
    if b == (8, 8, 8):
        _, idx, _, _, nb = cb.coarse_grain(chi, b)
        assert nb == 2624


def test_unaligned_device_image(cb, nrm):
    """A device image that does not start on 16 bytes takes the byte loads."""
    import torch

    chi = _spheres((64, 64, 64), 11, 5, seed=7)
    big = torch.zeros(chi.size + 1, dtype=torch.uint8, device="cuda")
    big[1:] = torch.from_numpy(chi.ravel()).cuda()
    view = big[1:].view(64, 64, 64)
    assert view.data_ptr() % 16 != 0
    phase, idx, c, N, nb = (o.cpu().numpy() if hasattr(o, "cpu") else o for o in cb.coarse_grain(view, (8, 8, 8)))
    ophase, oidx, oc, oN = nrm.block_normals(chi, (8, 8, 8), (1, 1, 1))
    assert np.array_equal(phase, ophase) and np.array_equal(idx, oidx) and np.array_equal(c, oc)
    check_normals(chi, (8, 8, 8), (1, 1, 1), idx, N, oN, "laplace")


def test_edge_cases(cb):
    z = np.zeros((16, 16, 16), np.uint8)
    phase, idx, c, N, nb = cb.coarse_grain(z, (4, 4, 4))
    assert nb == 0 and idx.size == 0 and not phase.any()
    phase, idx, c, N, nb = cb.coarse_grain(z + 3, (4, 4, 4))
    assert nb == 0 and np.all(phase == 1)
    chi = _spheres((32, 32, 32), 6, 4, seed=3)
    _, idx_all, c_all, N_all, nb = cb.coarse_grain(chi, (4, 4, 4))
    assert nb == idx_all.size > 10
    # cap = 0 counts only; a small cap keeps the first boxels
    _, idx0, _, _, nb0 = cb.coarse_grain(chi, (4, 4, 4), cap=0)
    assert nb0 == nb and idx0.size == 0
    _, idx5, c5, N5, nb5 = cb.coarse_grain(chi, (4, 4, 4), cap=5)
    assert nb5 == nb and np.array_equal(idx5, idx_all[:5]) and np.array_equal(N5, N_all[:5])
    # argument errors are status codes
    with pytest.raises(cb.ComboError):
        cb.coarse_grain(chi, (5, 4, 4))  # does not divide
    with pytest.raises(cb.ComboError):
        cb.coarse_grain(chi, (4, 4, 4), h=(1.0, 0.0, 1.0))
    with pytest.raises(cb.ComboError):
        cb.coarse_grain(np.zeros((128, 128, 128), np.uint8), (128, 128, 128))  # moments overflow int32
    with pytest.raises(cb.ComboError):
        cb.coarse_grain(np.zeros((64, 64, 4096), np.uint8), (8, 64, 64))  # slab exceeds shared memory


def test_full_size_spheres_1024_sampled(cb, nrm):
    """1024^3 spheres image (1 GiB) coarse-grained to 128^3 on the device, the
    configuration the benchmark times: phase counts and c+ are checked in
    full against host counts, the normals on a sample of boxels."""
    import torch

    from paper_2204_13624_gb300 import microstructure as ms

    chi = ms.fine_spheres_image((1024, 1024, 1024), 24, 4000, seed=ms.SEED_BASE + 5)
    d = torch.from_numpy(chi).cuda()
    phase, idx, c, N, nb = cb.coarse_grain(d, (8, 8, 8))
    del d
    phase, idx, c, N = (o.cpu().numpy() for o in (phase, idx, c, N))
    cnt = chi.reshape(128, 8, 128, 8, 128, 8).sum(axis=(1, 3, 5), dtype=np.int64).ravel()
    exp = np.where(cnt == 0, 0, np.where(cnt == 512, 1, 2)).astype(np.uint8)
    assert np.array_equal(phase.ravel(), exp)
    assert np.array_equal(idx, np.flatnonzero(exp == 2))
    assert np.array_equal(c, cnt[idx] / 512.0)
    rng = np.random.default_rng(11)
    pick = np.sort(rng.choice(idx.size, 400, replace=False))
    _, oc, oN = nrm.block_normals_at(chi, (8, 8, 8), (1, 1, 1), idx[pick])
    assert np.array_equal(oc, c[pick])
    check_normals(chi, (8, 8, 8), (1, 1, 1), idx[pick], N[pick], oN, "laplace")


def test_coarse_grained_ball_feeds_the_solver(cb, nrm):
    """Image -> composite boxels -> homogenization: the boxel list of the GPU
    coarse-graining and the oracle's give the same effective stress."""
    from paper_2204_13624_gb300 import microstructure as ms

    chi = ms.fine_ball_image(128, 0.4)
    phase, idx, c, N, nb = cb.coarse_grain(chi, (4, 4, 4))
    ophase, oidx, oc, oN = nrm.block_normals(chi, (4, 4, 4), (1, 1, 1))
    Fbar = np.eye(3).ravel() + np.array([0.02, 0.01, 0, 0, -0.01, 0, 0, 0, 0.01])
    out = []
    for (ph, ix, cc, NN) in ((phase, idx, c, N), (ophase, oidx, oc, oN)):
        prob = ms.make_problem((32, 32, 32), (1.0, 1.0, 1.0), ph.ravel(), ix, cc, NN, (1.0, 10.0), (2.0, 20.0),
                               Fbar, 2)
        out.append(cb.solve(prob, fields=False, precision=cb.FP64, tol=1e-10)["Pbar"])
    assert np.allclose(out[0], out[1], rtol=0, atol=1e-9 * np.abs(out[1]).max())
