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
        idx_p[axis] = 1
        S[tuple(idx_m)] += ri
        S[tuple(idx_p)] += ri
        S[0, 0, 0] -= 2.0 * ri
    conv = np.fft.ifftn(np.fft.fftn(chi) * np.fft.fftn(S)).real
    return np.abs(conv)


def block_normals(chi, b, h, method="laplace"):
    """Coarse-grain chi into boxels of b fine voxels.

    Returns (phase_c [nc3, nc2, nc1] uint8: 0 matrix, 1 inclusion, 2 boxel;
    boxel_idx (linear coarse index, increasing); c_plus; N [nb, 3])."""
    chi = np.asarray(chi, dtype=np.uint8)
    n3, n2, n1 = chi.shape
    b1, b2, b3 = (int(v) for v in b)
    if n1 % b1 or n2 % b2 or n3 % b3:
        raise ValueError("block sizes must divide the fine grid")
    hx, hy, hz = (float(v) for v in h)
    nc1, nc2, nc3 = n1 // b1, n2 // b2, n3 // b3
    w = stencil_weights(chi, h) if method == "laplace" else None
    # fine-voxel centre offsets from the boxel centre, per axis
    ox = (np.arange(b1) + 0.5 - 0.5 * b1) * hx
    oy = (np.arange(b2) + 0.5 - 0.5 * b2) * hy
    oz = (np.arange(b3) + 0.5 - 0.5 * b3) * hz
    Z, Y, X = np.meshgrid(oz, oy, ox, indexing="ij")
    phase = np.zeros((nc3, nc2, nc1), np.uint8)
    idx, cs, Ns = [], [], []
    nblock = b1 * b2 * b3
    for K in range(nc3):
        for J in range(nc2):
            for I in range(nc1):
                blk = chi[K * b3:(K + 1) * b3, J * b2:(J + 1) * b2, I * b1:(I + 1) * b1]
                npl = int(blk.sum())
                if npl == 0:
                    continue
                if npl == nblock:
                    phase[K, J, I] = 1
                    continue
                phase[K, J, I] = 2
                inc = blk.astype(bool)
                cp = np.array([X[inc].mean(), Y[inc].mean(), Z[inc].mean()])
                cm = np.array([X[~inc].mean(), Y[~inc].mean(), Z[~inc].mean()])
                Nt = (cm - cp) / np.linalg.norm(cm - cp)  # Eq. normal:kabel
                if method == "kabel":
                    N = Nt
                else:
                    wb = w[K * b3:(K + 1) * b3, J * b2:(J + 1) * b2, I * b1:(I + 1) * b1].ravel()
                    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
                    P = P - (wb @ P) / wb.sum()  # relative to the weighted barycentre c_S
                    M = (P * wb[:, None]).T @ P  # sum w x (x) x
                    lam, vec = np.linalg.eigh(M)
                    N = vec[:, 0]
                    N = N if float(Nt @ N) > 0.0 else -N  # Eq. normal:flip
                idx.append(I + nc1 * (J + nc2 * K))
                cs.append(npl / nblock)
                Ns.append(N)
    return (phase, np.asarray(idx, np.int64), np.asarray(cs, np.float64),
            np.asarray(Ns, np.float64).reshape(-1, 3))


def moment_tensor(chi, b, h, coarse_index, w=None):
    """M of one boxel (for the property checks of degenerate eigenvalues);
    w = stencil_weights(chi, h) when the caller has it already."""
    chi = np.asarray(chi, dtype=np.uint8)
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
