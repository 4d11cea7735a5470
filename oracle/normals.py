"""FP64 CPU oracle of the composite-boxel coarse-graining with the paper's
normal detection (Sec. 5).

TEST INFRASTRUCTURE ONLY (see the package docstring): tests/ and the CPU legs
of bench.py use it; the CUDA library never does.  Plain numpy, following the
paper's steps in order; numpy's FFT and symmetric eigen-solver serve as
library steps.

Image conventions: chi[k, j, i] (x = i fastest) is 1 where the fine voxel
belongs to the inclusion phase, 0 in the matrix; fine voxel (i, j, k) has edge
lengths h = (hx, hy, hz) and centre ((i + 1/2) hx, (j + 1/2) hy, (k + 1/2) hz)
up to a common shift; the image is periodic.  A boxel is a block of
b = (b1, b2, b3) fine voxels; coarse voxel (I, J, K) holds the fine voxels
(b1 I + i', b2 J + j', b3 K + k').

Steps (Sec. 5.1, 5.2):
  [N.1] weights w = |S * chi| with the 3D stencil made of the 1D second
        difference chi[-e_i] - 2 chi + chi[+e_i] along each axis, weighted by
        r_i = h_j h_k / h_i (the 1/h_i^2 of the 1D Laplacian times the fine
        voxel volume); the convolution is carried out in the Fourier domain
        (periodic).
  [N.2] on every boxel holding both phases (0 < c+ < 1): the second moment
        M = sum_fine w x (x) x, x relative to the w-weighted barycentre of the
        interface voxels of the boxel (c_S of Fig. normal:new:1; the weighted
        least-squares plane through them); N = the
        eigenvector of the smallest eigenvalue of M, its sign chosen so that
        N . Ntilde > 0 (else -N) where Ntilde = (barycentre of the matrix
        voxels - barycentre of the inclusion voxels) normalised (Eq.
        normal:kabel), so that N points out of the inclusion (Eq.
        normal:flip).
  The barycentre normal alone (Eq. normal:kabel) is the "kabel" method.
"""
from __future__ import annotations

import numpy as np


def stencil_weights(chi, h):
    """[N.1]: w = |S * chi| by FFT convolution (periodic)."""
    chi = np.asarray(chi, dtype=np.float64)
    hx, hy, hz = (float(v) for v in h)
    r = (hy * hz / hx, hx * hz / hy, hx * hy / hz)  # r_i = h_j h_k / h_i
    n3, n2, n1 = chi.shape
    S = np.zeros_like(chi)
    # axis i of the stencil: r_i at -e_i and +e_i, -2 r_i at the centre
    for axis, ri in zip((2, 1, 0), r):  # x, y, z are the array axes 2, 1, 0
        idx_m = [0, 0, 0]
        idx_p = [0, 0, 0]
        idx_m[axis] = -1
        idx_p[axis] = 1 % chi.shape[axis]  # one voxel along the axis: its own neighbour
        S[tuple(idx_m)] += ri
        S[tuple(idx_p)] += ri
        S[0, 0, 0] -= 2.0 * ri
    conv = np.fft.ifftn(np.fft.fftn(chi) * np.fft.fftn(S)).real
    return np.abs(conv)


def block_normals(chi, b, h, method="laplace"):
    """Coarse-grain chi into boxels of b fine voxels.

    Returns (phase_c [nc3, nc2, nc1] uint8: 0 matrix, 1 inclusion, 2 boxel;
    boxel_idx (linear coarse index, increasing); c_plus; N [nb, 3]).

    Readings where the paper is silent (degenerate boxels):
      - Ntilde is undefined (taken as 0) when the two barycentres coincide;
        the sign rule keeps N only for Ntilde . N > 0, so N's sign is then
        the eigen-solver's;
      - the "kabel" method falls back to the Laplacian normal there;
      - the weights of a boxel holding both phases never all vanish: a fine
        voxel with a neighbour of the other phase has w > 0 (all its second
        differences share the sign of -chi), so M is well defined."""
    chi = (np.asarray(chi) != 0).astype(np.uint8)  # nonzero = inclusion
    n3, n2, n1 = chi.shape
    b1, b2, b3 = (int(v) for v in b)
    if n1 % b1 or n2 % b2 or n3 % b3:
        raise ValueError("block sizes must divide the fine grid")
    hv = np.array([float(v) for v in h])
    nc1, nc2, nc3 = n1 // b1, n2 // b2, n3 // b3
    w = stencil_weights(chi, h)
    # fine-voxel centre offsets from the boxel centre: x = q h / 2 with the
    # integer q = 2 i' + 1 - b (i' the position in the boxel)
    Q, P_all = _offsets((b1, b2, b3), hv)
    phase = np.zeros((nc3, nc2, nc1), np.uint8)
    idx, cs, Ns = [], [], []
    nblock = b1 * b2 * b3
    for K in range(nc3):
        for J in range(nc2):
            for I in range(nc1):
                blk = chi[K * b3:(K + 1) * b3, J * b2:(J + 1) * b2, I * b1:(I + 1) * b1]
                inc = blk.ravel().astype(bool)
                npl = int(inc.sum())
                if npl == 0:
                    continue
                if npl == nblock:
                    phase[K, J, I] = 1
                    continue
                phase[K, J, I] = 2
                wb = w[K * b3:(K + 1) * b3, J * b2:(J + 1) * b2, I * b1:(I + 1) * b1].ravel()
                idx.append(I + nc1 * (J + nc2 * K))
                cs.append(npl / nblock)
                Ns.append(_boxel_normal(inc, wb, Q, P_all, hv, method))
    return (phase, np.asarray(idx, np.int64), np.asarray(cs, np.float64),
            np.asarray(Ns, np.float64).reshape(-1, 3))


def _offsets(b, hv):
    """Integer offsets q = 2 i' + 1 - b of a boxel's fine voxels ([nblock, 3],
    x fastest) and their positions q h / 2 from the boxel centre."""
    b1, b2, b3 = b
    qx = 2 * np.arange(b1) + 1 - b1
    qy = 2 * np.arange(b2) + 1 - b2
    qz = 2 * np.arange(b3) + 1 - b3
    QZ, QY, QX = np.meshgrid(qz, qy, qx, indexing="ij")
    Q = np.stack([QX.ravel(), QY.ravel(), QZ.ravel()], 1)
    return Q, Q * (0.5 * hv)[None, :]


def _boxel_normal(inc, wb, Q, P_all, hv, method):
    """N of one boxel holding both phases: inc its inclusion flags, wb its
    Laplacian weights (both [nblock], x fastest)."""
    npl = int(inc.sum())
    nblock = inc.size
    # barycentres (Eq. normal:kabel) from the exact integer sums
    Qp = Q[inc].sum(0)
    Qm = Q[~inc].sum(0)
    cp = 0.5 * hv * Qp / npl
    cm = 0.5 * hv * Qm / (nblock - npl)
    dc = cm - cp
    Nt = dc / np.linalg.norm(dc) if np.any(dc != 0.0) else np.zeros(3)
    if method == "kabel" and np.any(Nt != 0.0):
        return Nt
    assert wb.sum() > 0.0
    P = P_all - (wb @ P_all) / wb.sum()  # relative to the weighted barycentre c_S
    M = (P * wb[:, None]).T @ P  # sum w x (x) x
    lam, vec = np.linalg.eigh(M)
    N = vec[:, 0]
    return N if float(Nt @ N) > 0.0 else -N  # Eq. normal:flip


def block_normals_at(chi, b, h, coarse_index, method="laplace"):
    """The boxels among the listed coarse voxels, for images too large for
    block_normals: the same steps, with the weights of each boxel from the
    periodic Laplacian stencil applied directly on its one-voxel halo (the
    direct evaluation Sec. 5.1 names as an alternative to the Fourier one;
    the two agree to rounding, pinned by the tests).  Returns (phase of each
    listed coarse voxel, c_plus, N) with c_plus = nan, N = nan for the pure
    ones."""
    chi = np.asarray(chi)
    n3, n2, n1 = chi.shape
    b1, b2, b3 = (int(v) for v in b)
    hv = np.array([float(v) for v in h])
    r = (hv[1] * hv[2] / hv[0], hv[0] * hv[2] / hv[1], hv[0] * hv[1] / hv[2])
    nc1, nc2 = n1 // b1, n2 // b2
    Q, P_all = _offsets((b1, b2, b3), hv)
    nblock = b1 * b2 * b3
    out_ph, out_c, out_N = [], [], []
    for ci in np.asarray(coarse_index, np.int64).ravel():
        I, J, K = int(ci % nc1), int((ci // nc1) % nc2), int(ci // (nc1 * nc2))
        xs = np.arange(I * b1 - 1, (I + 1) * b1 + 1) % n1
        ys = np.arange(J * b2 - 1, (J + 1) * b2 + 1) % n2
        zs = np.arange(K * b3 - 1, (K + 1) * b3 + 1) % n3
        win = (chi[np.ix_(zs, ys, xs)] != 0).astype(np.float64)
        c0 = win[1:-1, 1:-1, 1:-1]
        npl = int(c0.sum())
        if npl == 0 or npl == nblock:
            out_ph.append(0 if npl == 0 else 1)
            out_c.append(np.nan)
            out_N.append(np.full(3, np.nan))
            continue
        s = (r[0] * (win[1:-1, 1:-1, :-2] + win[1:-1, 1:-1, 2:] - 2 * c0)
             + r[1] * (win[1:-1, :-2, 1:-1] + win[1:-1, 2:, 1:-1] - 2 * c0)
             + r[2] * (win[:-2, 1:-1, 1:-1] + win[2:, 1:-1, 1:-1] - 2 * c0))
        out_ph.append(2)
        out_c.append(npl / nblock)
        out_N.append(_boxel_normal(c0.ravel().astype(bool), np.abs(s).ravel(), Q, P_all, hv, method))
    return np.asarray(out_ph, np.uint8), np.asarray(out_c), np.asarray(out_N).reshape(-1, 3)


def barycentre_normal(chi, b, h, coarse_index):
    """Ntilde of one boxel (Eq. normal:kabel), zeros when undefined."""
    chi = (np.asarray(chi) != 0).astype(np.uint8)  # nonzero = inclusion
    n3, n2, n1 = chi.shape
    b1, b2, b3 = (int(v) for v in b)
    nc1, nc2 = n1 // b1, n2 // b2
    I = coarse_index % nc1
    J = (coarse_index // nc1) % nc2
    K = coarse_index // (nc1 * nc2)
    blk = chi[K * b3:(K + 1) * b3, J * b2:(J + 1) * b2, I * b1:(I + 1) * b1].astype(bool)
    hv = np.array([float(v) for v in h])
    Z, Y, X = np.meshgrid(*(0.5 * hv[a] * (2 * np.arange(bb) + 1 - bb) for a, bb in ((2, b3), (1, b2), (0, b1))),
                          indexing="ij")
    cp = np.array([X[blk].mean(), Y[blk].mean(), Z[blk].mean()])
    cm = np.array([X[~blk].mean(), Y[~blk].mean(), Z[~blk].mean()])
    d = cm - cp
    nd = np.linalg.norm(d)
    return d / nd if nd > 0 else np.zeros(3)


def moment_tensor(chi, b, h, coarse_index, w=None):
    """M of one boxel (for the property checks of degenerate eigenvalues);
    w = stencil_weights(chi, h) when the caller has it already."""
    chi = (np.asarray(chi) != 0).astype(np.uint8)  # nonzero = inclusion
    n3, n2, n1 = chi.shape
    b1, b2, b3 = (int(v) for v in b)
    nc1, nc2 = n1 // b1, n2 // b2
    I = coarse_index % nc1
    J = (coarse_index // nc1) % nc2
    K = coarse_index // (nc1 * nc2)
    hx, hy, hz = (float(v) for v in h)
    if w is None:
        w = stencil_weights(chi, h)
    w = w[K * b3:(K + 1) * b3, J * b2:(J + 1) * b2, I * b1:(I + 1) * b1]
    ox = (np.arange(b1) + 0.5 - 0.5 * b1) * hx
    oy = (np.arange(b2) + 0.5 - 0.5 * b2) * hy
    oz = (np.arange(b3) + 0.5 - 0.5 * b3) * hz
    Z, Y, X = np.meshgrid(oz, oy, ox, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    wb = w.ravel()
    P = P - (wb @ P) / wb.sum()
    return (P * wb[:, None]).T @ P
