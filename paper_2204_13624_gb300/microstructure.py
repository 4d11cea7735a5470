"""Seeded synthetic microstructures and load cases (input data only).

This module holds geometry, not the homogenization method: it places
inclusions, classifies voxels as matrix / inclusion / composite boxel, and
computes each boxel's inclusion volume fraction c+ and analytic interface
normal N.  Both the CUDA library's tests and the CPU oracle's tests take their
inputs from here; it imports neither.

Geometry conventions (paper Sec. 2 and App. A): the RVE is
Omega = prod_j [-l_j/2, l_j/2] on a grid of n1 x n2 x n3 voxels of edge
h_j = l_j / n_j; voxel (i, j, k) spans [-l/2 + i h, -l/2 + (i+1) h] per axis
and its linear index is i + n1 (j + n2 k).  The normal N of a composite voxel
points out of the inclusion ("+") into the matrix ("-") (paper Sec. 5.1); it
is the analytic surface normal at the projection of the voxel centre onto
the interface.

Volume fractions of voxels cut by a sphere are integrated along x of the
closed-form area of a disc clipped to a rectangle, with 24-point
Gauss-Legendre on every piece between the kinks of that area (tangencies and
corner crossings) after a smoothing substitution (host C helper
``csrc/geometry.c``; ``sphere_box_volume`` is the same integral in numpy);
for cylinders the clipped disc area is used directly.  The error is ~1e-12
per voxel (checked by tests/test_microstructure.py against the exact total
inclusion volume).

The problem dictionary (keys n, l, phase, boxel_idx, boxel_N, boxel_c, mu,
lam, Fbar, n_steps) is what ``combo.Problem`` and the oracle accept.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2204_13624

_GL_X, _GL_W = np.polynomial.legendre.leggauss(24)


# ----------------------------------------------------------------- areas
def _S(Y, rho):
    """Antiderivative of sqrt(rho^2 - Y^2) on [-rho, rho]."""
    Yc = np.clip(Y, -rho, rho)
    s = np.sqrt(np.maximum(rho * rho - Yc * Yc, 0.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        t = np.where(rho > 0, Yc / np.where(rho > 0, rho, 1.0), 0.0)
    return 0.5 * (Yc * s + rho * rho * np.arcsin(np.clip(t, -1.0, 1.0)))


def _quad_area(y, z, rho):
    """Area of the disc |(Y, Z)| < rho intersected with {Y <= y, Z <= z}."""
    y, z, rho = np.broadcast_arrays(np.asarray(y, float), np.asarray(z, float), np.asarray(rho, float))
    yp = np.clip(y, -rho, rho)
    w = np.sqrt(np.maximum(rho * rho - np.clip(z, -rho, rho) ** 2, 0.0))
    zpos = z >= 0
    # piece 1: [-rho, min(-w, y')] -> 2 s if z >= 0 else 0
    b1 = np.minimum(-w, yp)
    p1 = np.where(zpos & (b1 > -rho), 2.0 * (_S(b1, rho) - _S(-rho, rho)), 0.0)
    # piece 2: [-w, min(w, y')] -> z + s
    b2 = np.minimum(w, yp)
    p2 = np.where(b2 > -w, z * (b2 + w) + _S(b2, rho) - _S(-w, rho), 0.0)
    # piece 3: [w, y'] -> 2 s if z >= 0 else 0
    p3 = np.where(zpos & (yp > w), 2.0 * (_S(yp, rho) - _S(w, rho)), 0.0)
    out = p1 + p2 + p3
    out = np.where(z >= rho, 2.0 * (_S(yp, rho) - _S(-rho, rho)), out)
    out = np.where(z <= -rho, 0.0, out)
    return np.where(rho > 0, out, 0.0)


def disc_rect_area(rho, y0, y1, z0, z1):
    """Area of the disc of radius rho centred at the origin inside [y0,y1]x[z0,z1]."""
    return (_quad_area(y1, z1, rho) - _quad_area(y0, z1, rho) - _quad_area(y1, z0, rho)
            + _quad_area(y0, z0, rho))


def sphere_box_volume(R, x0, x1, y0, y1, z0, z1):
    """Volume of the ball |x| < R inside boxes [x0,x1]x[y0,y1]x[z0,z1] (arrays,
    coordinates relative to the centre)."""
    x0, x1, y0, y1, z0, z1 = (np.asarray(a, float) for a in (x0, x1, y0, y1, z0, z1))
    m = x0.shape[0]
    # kinks of the clipped-disc area as a function of x: rho(x) = |edge| or |corner|
    ds = [np.abs(y0), np.abs(y1), np.abs(z0), np.abs(z1)]
    for a in (y0, y1):
        for b in (z0, z1):
            ds.append(np.sqrt(a * a + b * b))
    bps = [x0, x1, np.full(m, -R), np.full(m, R)]
    for d in ds:
        h = np.sqrt(np.maximum(R * R - d * d, 0.0))
        bps += [h, -h]
    B = np.sort(np.clip(np.stack(bps, 1), x0[:, None], x1[:, None]), axis=1)
    a, b = B[:, :-1], B[:, 1:]
    # smoothing substitution x = a + (b - a) (3 t^2 - 2 t^3) removes the
    # (x - x*)^{1/2, 3/2} endpoint behaviour at the kinks
    t = 0.5 * (_GL_X + 1.0)
    wt = 0.5 * _GL_W
    u = 3 * t * t - 2 * t ** 3
    du = 6 * t - 6 * t * t
    X = a[..., None] + (b - a)[..., None] * u
    rho = np.sqrt(np.maximum(R * R - X * X, 0.0))
    Aq = disc_rect_area(rho, y0[:, None, None], y1[:, None, None], z0[:, None, None], z1[:, None, None])
    return np.sum(Aq * (b - a)[..., None] * du * wt, axis=(1, 2))


# ----------------------------------------------------------------- grids
def _edges(n, l):
    h = l / n
    lo = -0.5 * l + h * np.arange(n)
    return lo, lo + h


def _min_image(d, L):
    return d - L * np.round(d / L)


def _finish(n, l, phase, idx, c, N, c_min):
    """Mark inclusion / boxel voxels; snap boxels with c outside
    [c_min, 1 - c_min] to the pure phase."""
    full = c >= 1.0 - c_min
    empty = c <= c_min
    phase[idx[full]] = 1
    keep = ~(full | empty)
    idx, c, N = idx[keep], c[keep], N[keep]
    phase[idx] = 2
    return phase, idx, c, N


_geo = None


def _geometry_lib():
    """Build (once) and load the host C helper ``csrc/geometry.c``."""
    global _geo
    if _geo is None:
        import ctypes as C
        import os
        import subprocess

        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "csrc", "geometry.c")
        so = os.path.join(here, "_geometry.so")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = so + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"])
            os.replace(tmp, so)
        L = C.CDLL(so)
        vp = C.c_void_p
        L.geo_balls_count.argtypes = [vp, vp, C.c_int, vp, C.c_double, vp, vp]
        L.geo_balls_fill.argtypes = [vp, vp, C.c_int, vp, C.c_double, vp, C.c_int, vp, vp, vp, vp, vp]
        L.geo_ball_box_volume.argtypes = [C.c_double] * 7 + [C.c_int, vp, vp]
        L.geo_ball_box_volume.restype = C.c_double
        _geo = L
    return _geo


def spheres_geometry(n, l, centres, R, c_min=1e-6):
    """Phase field and boxels for non-overlapping periodic balls of radius R.

    Every voxel must be cut by at most one ball (callers keep a gap of
    >= 2 voxels between balls).  Returns (phase[V], boxel_idx, boxel_c,
    boxel_N)."""
    n = np.asarray([int(v) for v in n], np.int32)
    l = np.asarray([float(v) for v in l], np.float64)
    V = int(n[0]) * int(n[1]) * int(n[2])
    cen = np.ascontiguousarray(np.asarray(centres, float).reshape(-1, 3))
    nb = cen.shape[0]
    phase = np.zeros(V, np.uint8)
    counts = np.zeros(nb, np.int64)
    L = _geometry_lib()
    L.geo_balls_count(n.ctypes.data, l.ctypes.data, nb, cen.ctypes.data, float(R), phase.ctypes.data,
                      counts.ctypes.data)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    tot = int(offsets[-1])
    idx = np.zeros(tot, np.int64)
    c = np.zeros(tot)
    N = np.zeros((tot, 3))
    gx = np.ascontiguousarray(_GL_X)
    gw = np.ascontiguousarray(_GL_W)
    L.geo_balls_fill(n.ctypes.data, l.ctypes.data, nb, cen.ctypes.data, float(R), offsets.ctypes.data, gx.size,
                     gx.ctypes.data, gw.ctypes.data, idx.ctypes.data, c.ctypes.data, N.ctypes.data)
    order = np.argsort(idx, kind="stable")
    idx, c, N = idx[order], c[order], N[order]
    if idx.size and np.any(np.diff(idx) == 0):
        raise ValueError("a voxel is cut by two inclusions; increase the gap")
    return _finish(tuple(n), tuple(l), phase, idx, np.clip(c, 0.0, 1.0), N, c_min)


def fibres_geometry(n, l, centres_xy, R, c_min=1e-6):
    """Straight z-aligned periodic cylinders of radius R through centres (x, y)."""
    n = tuple(int(v) for v in n)
    l = tuple(float(v) for v in l)
    h = np.array([l[0] / n[0], l[1] / n[1], l[2] / n[2]])
    n1, n2, n3 = n
    col_phase = np.zeros(n1 * n2, np.uint8)
    cols, cs, Ns = [], [], []
    for cen in np.asarray(centres_xy, float).reshape(-1, 2):
        rng = []
        for ax in range(2):
            i0 = int(math.floor((cen[ax] - R + 0.5 * l[ax]) / h[ax])) - 1
            i1 = int(math.floor((cen[ax] + R + 0.5 * l[ax]) / h[ax])) + 1
            rng.append(np.arange(i0, i1 + 1))
        I, J = np.meshgrid(rng[0], rng[1], indexing="ij")
        I, J = I.ravel(), J.ravel()
        lox = -0.5 * l[0] + h[0] * I - cen[0]
        loy = -0.5 * l[1] + h[1] * J - cen[1]
        hix, hiy = lox + h[0], loy + h[1]
        dn = np.hypot(np.clip(0.0, lox, hix), np.clip(0.0, loy, hiy))
        df = np.hypot(np.maximum(np.abs(lox), np.abs(hix)), np.maximum(np.abs(loy), np.abs(hiy)))
        lin = (np.mod(I, n1) + n1 * np.mod(J, n2)).astype(np.int64)
        inside = df <= R
        cut = (~inside) & (dn < R)
        col_phase[lin[inside]] = 1
        if np.any(cut):
            area = disc_rect_area(np.full(cut.sum(), R), lox[cut], hix[cut], loy[cut], hiy[cut])
            cols.append(lin[cut])
            cs.append(area / (h[0] * h[1]))
            ctr = np.stack([0.5 * (lox[cut] + hix[cut]), 0.5 * (loy[cut] + hiy[cut])], 1)
            ctr /= np.linalg.norm(ctr, axis=1, keepdims=True)
            Ns.append(np.concatenate([ctr, np.zeros((ctr.shape[0], 1))], 1))
    if cols:
        col = np.concatenate(cols)
        cc = np.clip(np.concatenate(cs), 0.0, 1.0)
        NN = np.concatenate(Ns)
    else:
        col, cc, NN = np.zeros(0, np.int64), np.zeros(0), np.zeros((0, 3))
    order = np.argsort(col, kind="stable")
    col, cc, NN = col[order], cc[order], NN[order]
    if col.size and np.any(np.diff(col) == 0):
        raise ValueError("a column is cut by two fibres; increase the gap")
    full = cc >= 1.0 - c_min
    col_phase[col[full]] = 1
    keep = ~(full | (cc <= c_min))
    col, cc, NN = col[keep], cc[keep], NN[keep]
    col_phase[col] = 2
    phase = np.tile(col_phase, n3)
    nb_col = col.size
    idx = (col[None, :] + (n1 * n2) * np.arange(n3, dtype=np.int64)[:, None]).reshape(-1)
    c = np.tile(cc, n3)
    N = np.tile(NN, (n3, 1))
    assert idx.size == nb_col * n3
    return phase, idx, c, N


def rsa_centres(rng, count, dmin, box, dims=3, max_tries=400_000):
    """Random sequential addition of ``count`` points in a periodic box with
    minimum (periodic) distance ``dmin``."""
    box = np.asarray(box, float)[:dims]
    pts = np.zeros((count, dims))
    k = 0
    tries = 0
    while k < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("RSA did not place all inclusions")
        p = (rng.random(dims) - 0.5) * box
        if k:
            d = _min_image(pts[:k] - p, box)
            if np.min(np.sum(d * d, 1)) < dmin * dmin:
                continue
        pts[k] = p
        k += 1
    return pts


# ----------------------------------------------------------------- problems
def make_problem(n, l, phase, idx, c, N, mu, lam, Fbar, n_steps):
    return dict(n=tuple(int(v) for v in n), l=tuple(float(v) for v in l), phase=phase,
                boxel_idx=np.ascontiguousarray(idx, np.int64), boxel_c=np.ascontiguousarray(c, float),
                boxel_N=np.ascontiguousarray(N, float).reshape(-1, 3),
                mu=(float(mu[0]), float(mu[1])), lam=(float(lam[0]), float(lam[1])),
                Fbar=np.asarray(Fbar, float).reshape(9).copy(), n_steps=int(n_steps))


def centred_sphere(n=(32, 32, 32), vf=0.2, contrast=10.0, Fbar=None, n_steps=5, l=(1.0, 1.0, 1.0)):
    """One ball of volume fraction ``vf`` centred in the RVE (the 32^3 case:
    vf 0.2 -> radius 11.609 voxels).  Matrix mu=1, lam=2; inclusion x contrast."""
    vol = l[0] * l[1] * l[2]
    R = (3.0 * vf * vol / (4.0 * math.pi)) ** (1.0 / 3.0)
    phase, idx, c, N = spheres_geometry(n, l, [[0.0, 0.0, 0.0]], R)
    if Fbar is None:
        Fbar = np.diag([1.05, 1.0, 1.0])
    return make_problem(n, l, phase, idx, c, N, (1.0, contrast), (2.0, 2.0 * contrast), Fbar, n_steps)


def random_spheres(n, radius_vox, vf, seed, contrast, Fbar, n_steps, gap_vox=2.0):
    """Periodic random non-overlapping balls (RSA) of radius ``radius_vox``
    voxels at volume fraction ~vf; centre distance >= 2 r + gap."""
    n = tuple(int(v) for v in n)
    l = tuple(v / max(n) for v in n)
    h = 1.0 / max(n)
    R = radius_vox * h
    count = max(1, int(round(vf * l[0] * l[1] * l[2] / (4.0 / 3.0 * math.pi * R ** 3))))
    rng = np.random.default_rng(seed)
    cen = rsa_centres(rng, count, 2 * R + gap_vox * h, l, 3)
    phase, idx, c, N = spheres_geometry(n, l, cen, R)
    return make_problem(n, l, phase, idx, c, N, (1.0, contrast), (2.0, 2.0 * contrast), Fbar, n_steps)


def random_fibres(n, radius_vox, vf, seed, contrast, Fbar, n_steps, gap_vox=2.0):
    """Straight z-aligned cylinders of radius ``radius_vox`` voxels, placed
    randomly in xy (RSA, gap >= ``gap_vox``), fibre volume fraction ~vf."""
    n = tuple(int(v) for v in n)
    l = tuple(v / max(n) for v in n)
    h = 1.0 / max(n)
    R = radius_vox * h
    count = max(1, int(round(vf * l[0] * l[1] / (math.pi * R * R))))
    rng = np.random.default_rng(seed)
    cen = rsa_centres(rng, count, 2 * R + gap_vox * h, l, 2)
    phase, idx, c, N = fibres_geometry(n, l, cen, R)
    return make_problem(n, l, phase, idx, c, N, (1.0, contrast), (2.0, 2.0 * contrast), Fbar, n_steps)


def layered(n=(8, 4, 4), axis=0, m_incl=3, c_boxel=0.4, contrast=10.0, Fbar=None, n_steps=1, l=None):
    """Grid-aligned rank-one laminate: layers 0..m-1 along ``axis`` are
    inclusion, layer m is a composite boxel layer with c+ = c_boxel and normal
    +e_axis (pointing from the inclusion side into the matrix), the rest is
    matrix."""
    n = tuple(int(v) for v in n)
    l = tuple(v / max(n) for v in n) if l is None else tuple(float(v) for v in l)
    V = n[0] * n[1] * n[2]
    coords = np.indices((n[2], n[1], n[0])).reshape(3, -1)  # k, j, i
    pos = coords[2 - axis]
    phase = np.zeros(V, np.uint8)
    phase[pos < m_incl] = 1
    idx = np.nonzero(pos == m_incl)[0].astype(np.int64)
    phase[idx] = 2
    c = np.full(idx.size, float(c_boxel))
    N = np.zeros((idx.size, 3))
    N[:, axis] = 1.0
    if Fbar is None:
        Fbar = np.eye(3) + 0.05 * np.array([[1.0, 0.3, 0.0], [0.1, -0.2, 0.2], [0.0, 0.1, 0.15]])
    return make_problem(n, l, phase, idx, c, N, (1.0, contrast), (2.0, 2.0 * contrast), Fbar, n_steps)


def homogeneous(n=(8, 8, 8), mu=1.0, lam=2.0, phase_value=0, Fbar=None, n_steps=1):
    n = tuple(int(v) for v in n)
    V = n[0] * n[1] * n[2]
    phase = np.full(V, phase_value, np.uint8)
    if Fbar is None:
        Fbar = np.eye(3) + np.array([[0.05, 0.02, 0.0], [0.0, -0.01, 0.03], [0.01, 0.0, 0.02]])
    l = tuple(v / max(n) for v in n)
    return make_problem(n, l, phase, np.zeros(0, np.int64), np.zeros(0), np.zeros((0, 3)), (mu, mu), (lam, lam),
                        Fbar, n_steps)


def random_boxels(n, seed, boxel_frac=0.15, incl_frac=0.3, contrast=10.0, Fbar=None, n_steps=1, l=None):
    """Unstructured stress case: every voxel independently matrix / inclusion /
    boxel, boxels with random c+ in [0.02, 0.98] and random unit normals."""
    n = tuple(int(v) for v in n)
    V = n[0] * n[1] * n[2]
    rng = np.random.default_rng(seed)
    u = rng.random(V)
    phase = np.where(u < boxel_frac, 2, np.where(u < boxel_frac + incl_frac, 1, 0)).astype(np.uint8)
    idx = np.nonzero(phase == 2)[0].astype(np.int64)
    c = rng.uniform(0.02, 0.98, idx.size)
    N = rng.normal(size=(idx.size, 3))
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    if Fbar is None:
        Fbar = np.eye(3) + 0.04 * rng.uniform(-1, 1, (3, 3))
    l = tuple(v / max(n) for v in n) if l is None else l
    return make_problem(n, l, phase, idx, c, N, (1.0, contrast), (2.0, 2.0 * contrast), Fbar, n_steps)


# ----------------------------------------------------------------- named workloads
def sphere_32(n_steps=5):
    """32^3, one centred ball of volume fraction 0.2, contrast 10,
    Fbar = diag(1.05, 1, 1) in 5 load steps."""
    return centred_sphere((32, 32, 32), 0.2, 10.0, np.diag([1.05, 1.0, 1.0]), n_steps)


def spheres_256(n=256, n_steps=10, seed=SEED_BASE + 1, vf=0.25):
    """256^3 periodic random non-overlapping balls of radius 12 voxels at
    volume fraction 0.25 (centre distance >= 2 r + 2 voxels), contrast 100,
    uniaxial Fbar11 = 1.10 in 10 steps.  ``n`` < 256 keeps radius/n fixed
    (scaled copy for tests; pass a lower ``vf`` there, the 2-voxel gap is a
    larger share of a small radius)."""
    r = 12.0 * n / 256.0
    return random_spheres((n, n, n), r, vf, seed, 100.0, np.diag([1.10, 1.0, 1.0]), n_steps, gap_vox=2.0)


def fibres_512(n=512, n_steps=15, seed=SEED_BASE + 2, vf=0.3):
    """512^3 straight z-fibres of radius 10 voxels, fibre fraction 0.3,
    contrast 50, simple shear Fbar = I + 0.15 e1 (x) e2 in 15 steps."""
    r = 10.0 * n / 512.0
    Fb = np.eye(3)
    Fb[0, 1] = 0.15
    return random_fibres((n, n, n), r, vf, seed, 50.0, Fb, n_steps, gap_vox=2.0)


def batch_mix(count=64, seed=SEED_BASE + 3, sides=(32, 48, 64, 96, 128), n_steps=5, gap_vox=1.75):
    """``count`` independent random-sphere solves: side uniform from ``sides``,
    vf ~ U(0.1, 0.35), radius max(4, side/10) voxels, contrast 10, Fbar =
    I + diag(U(-.08,.08)^3) + off-diagonal U(-.10,.10).  The drawn vf is
    capped where random sequential addition with the gap that keeps every
    voxel cut by at most one ball would jam: (r + gap/2)^3 / r^3 * vf <= 0.3."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        side = int(rng.choice(sides))
        vf = float(rng.uniform(0.1, 0.35))
        r = max(4.0, side / 10.0)
        vf = min(vf, 0.3 * (r / (r + 0.5 * gap_vox)) ** 3)
        Fb = np.eye(3) + np.diag(rng.uniform(-0.08, 0.08, 3))
        off = rng.uniform(-0.10, 0.10, (3, 3))
        np.fill_diagonal(off, 0.0)
        Fb = Fb + off
        out.append(random_spheres((side,) * 3, r, vf, int(rng.integers(1 << 31)), 10.0, Fb, n_steps,
                                  gap_vox=gap_vox))
    return out


def lame(E, nu):
    """(mu, lambda) of Young's modulus E and Poisson ratio nu."""
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


# Sec. 6.1: inclusion E = 10, nu = 0.3; matrix E = 1, nu = 0 (GPa); 50 % shear F_xy
E1_MU = (lame(1.0, 0.0)[0], lame(10.0, 0.3)[0])
E1_LAM = (lame(1.0, 0.0)[1], lame(10.0, 0.3)[1])
E1_FBAR = np.array([[1.0, 0.5, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def sphere_e1_fine(fine=256, n_steps=5):
    """Sec. 6.2: the fine reference problem, the ball R = 0.4 of the unit RVE
    sampled at fine voxel centres, no composite voxels."""
    chi = fine_ball_image(fine, 0.4)
    n = (fine, fine, fine)
    return make_problem(n, (1.0, 1.0, 1.0), chi.ravel(), np.zeros(0, np.int64), np.zeros(0), np.zeros((0, 3)),
                        E1_MU, E1_LAM, E1_FBAR, n_steps)


def sphere_e1_coarse(phase, idx, c, N, n_steps=5):
    """Sec. 6.2: a coarse-grained problem from combo_coarse_grain's outputs
    (phase [nc3, nc2, nc1], boxel indices, c+, normals) on the unit RVE."""
    nc3, nc2, nc1 = phase.shape
    return make_problem((nc1, nc2, nc3), (1.0, 1.0, 1.0), np.ascontiguousarray(phase).ravel(), idx, c, N, E1_MU,
                        E1_LAM, E1_FBAR, n_steps)


def fine_ball_image(fine=256, R=0.4):
    """Binary fine image chi[k, j, i] (uint8, x fastest) of the ball |x| < R of
    the unit RVE [-0.5, 0.5]^3 sampled at the fine voxel centres (the paper's
    Sec. 6.2 sphere before coarse-graining)."""
    x = (np.arange(fine) + 0.5) / fine - 0.5
    r2 = x[None, None, :] ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2
    return (r2 < R * R).astype(np.uint8)


def fine_plane_image(n, normal, offset=0.0, h=(1.0, 1.0, 1.0)):
    """Binary fine image of the half space (x - c) . normal < offset (the
    inclusion), c the centre of the periodic box of n voxels of edges h,
    sampled at voxel centres; normal is normalised here."""
    n1, n2, n3 = (int(v) for v in n)
    nv = np.asarray(normal, float)
    nv = nv / np.linalg.norm(nv)
    x = (np.arange(n1) + 0.5 - 0.5 * n1) * h[0]
    y = (np.arange(n2) + 0.5 - 0.5 * n2) * h[1]
    z = (np.arange(n3) + 0.5 - 0.5 * n3) * h[2]
    d = nv[0] * x[None, None, :] + nv[1] * y[None, :, None] + nv[2] * z[:, None, None]
    return (d < offset).astype(np.uint8)


def fine_spheres_image(n, radius_vox, count, seed=SEED_BASE + 4, h=(1.0, 1.0, 1.0)):
    """Binary fine image chi[k, j, i] (uint8, x fastest) of `count` balls of
    radius radius_vox (in units of h[0]) at uniform random centres of the
    periodic box of n = (n1, n2, n3) voxels with edges h (balls may overlap;
    voxels are classified by their centres)."""
    n1, n2, n3 = (int(v) for v in n)
    hx, hy, hz = (float(v) for v in h)
    rng = np.random.default_rng(seed)
    L = np.array([n1 * hx, n2 * hy, n3 * hz])
    chi = np.zeros((n3, n2, n1), np.uint8)
    R = float(radius_vox) * hx
    for c in rng.random((int(count), 3)) * L:
        lo = np.floor((c - R) / [hx, hy, hz]).astype(int) - 1
        hi = np.ceil((c + R) / [hx, hy, hz]).astype(int) + 1
        ix = np.arange(lo[0], hi[0] + 1)
        iy = np.arange(lo[1], hi[1] + 1)
        iz = np.arange(lo[2], hi[2] + 1)
        dx = (ix + 0.5) * hx - c[0]
        dy = (iy + 0.5) * hy - c[1]
        dz = (iz + 0.5) * hz - c[2]
        inside = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2 < R * R
        sub = np.ix_(iz % n3, iy % n2, ix % n1)
        chi[sub] |= inside.astype(np.uint8)
    return chi


def fine_sphere_block_count(fine=256, coarse=32, R=0.4):
    """Number of coarse blocks that hold both phases when a ball of radius R
    (RVE [-0.5, 0.5]^3) is sampled at the fine voxel centres and the fine
    image is coarse-grained into ``coarse``^3 blocks (paper Sec. 6.2)."""
    x = (np.arange(fine) + 0.5) / fine - 0.5
    b = fine // coarse
    r2 = x[:, None] ** 2 + x[None, :] ** 2
    cnt = np.zeros((coarse, coarse, coarse), np.int64)
    for k in range(fine):
        inside = (r2 + x[k] ** 2) < R * R
        cnt[k // b] += inside.reshape(coarse, b, coarse, b).sum(axis=(1, 3))
    full = b ** 3
    return int(np.sum((cnt > 0) & (cnt < full)))
