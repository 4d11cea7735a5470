"""FP64 CPU oracle for the ComBo FFT homogenization hot path.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it; the
product path (``paper_2204_13624_gb300``) never imports it.

The oracle is plain C (``combo_oracle.c``) compiled with gcc and reached
through ctypes.  It shares no code with the CUDA library.  See the C file's
header for what each function computes and which part of the paper it
follows (Sec. 3 Lippmann-Schwinger / Green operator, Sec. 4 laminate
Algorithms 1 and 2, Sec. 6.1 Neo-Hookean material, App. A staggered grid and
doubly-fine material grid, the appendix cheat sheet's infinitesimal-strain
column).  ``normals.py`` (plain numpy) is the oracle of the coarse-graining
with the Sec. 5 normal detection.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force and the paper's printed facts.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "combo_oracle.c")
_LIB = os.path.join(_HERE, "libcombo_oracle.so")

ROTATED, SPECTRAL, STAGGERED, STAGGERED_DFMG = 0, 1, 2, 3
FIXED_POINT, NEWTON_CG, NONLINEAR_CG = 0, 1, 2

STATUS = {0: "ok", -1: "invalid", -3: "not converged", -4: "laminate NR failed",
          -5: "inadmissible (det F <= 0)", -6: "NaN"}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libcombo_oracle.so`` (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_neohooke.argtypes = [dp, C.c_double, C.c_double, dp, dp]
        L.orc_neohooke.restype = C.c_int
        L.orc_neohooke_energy.argtypes = [dp, C.c_double, C.c_double]
        L.orc_neohooke_energy.restype = C.c_double
        L.orc_laminate.argtypes = [dp, dp, C.c_double, dp, dp, C.c_double, C.c_double, C.c_int,
                                   dp, dp, ip, ip, dp]
        L.orc_laminate.restype = C.c_int
        L.orc_linear.argtypes = [dp, C.c_double, C.c_double, dp, dp]
        L.orc_linear.restype = C.c_int
        L.orc_laminate_linear.argtypes = [dp, dp, C.c_double, dp, dp, dp, dp]
        L.orc_laminate_linear.restype = C.c_int
        L.orc_fft1.argtypes = [C.c_int, C.c_int, dp, dp]
        L.orc_fft3.argtypes = [ip, C.c_int, dp]
        L.orc_kvec.argtypes = [C.c_int, ip, dp, ip, dp]
        L.orc_kvec_row.argtypes = [C.c_int, ip, dp, ip, C.c_int, dp]
        L.orc_gamma_matrix.argtypes = [C.c_int, ip, dp, ip, dp]
        L.orc_gamma_matrix.restype = C.c_int
        L.orc_apply_G.argtypes = [C.c_int, ip, dp, dp, dp]
        L.orc_apply_G.restype = C.c_double
        L.orc_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_solve.restype = C.c_int
        L.orc_constitutive_field.argtypes = [C.c_void_p, C.c_void_p, dp, dp, dp, dp]
        L.orc_dfmg_tangent_apply.argtypes = [C.c_void_p, C.c_void_p, dp, dp, dp]
        L.orc_dfmg_tangent_apply.restype = C.c_int
        L.orc_constitutive_field.restype = C.c_int
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(x, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- material
def neohooke(F, mu, lam, tangent=True):
    """P(F) and the 9x9 tangent A (row-major 2-tensors), Sec. 6.1."""
    F = _f64(F, (9,))
    P = np.zeros(9)
    A = np.zeros(81)
    rc = lib().orc_neohooke(_d(F), mu, lam, _d(P), _d(A) if tangent else None)
    if rc:
        raise ValueError(STATUS.get(rc, rc))
    return (P, A.reshape(9, 9)) if tangent else P


def neohooke_energy(F, mu, lam):
    F = _f64(F, (9,))
    return lib().orc_neohooke_energy(_d(F), mu, lam)


def laminate(F, N, c, mat, a0=None, tol_rel=1e-12, tol_abs=1e-14, max_iter=50, trace=False):
    """Algorithm 1 + Algorithm 2 for one boxel.  mat = (mu-, lam-, mu+, lam+).

    Returns dict(P, A, a, iters, nbp[, trace]).  Raises on failure."""
    F = _f64(F, (9,))
    N = _f64(N, (3,))
    m = _f64(mat, (4,))
    a = np.zeros(3) if a0 is None else _f64(a0, (3,)).copy()
    P = np.zeros(9)
    A = np.zeros(81)
    it = np.zeros(1, dtype=np.int32)
    nbp = np.zeros(1, dtype=np.int32)
    tr = np.full(4 * (max_iter + 1), np.nan) if trace else None
    rc = lib().orc_laminate(_d(F), _d(N), float(c), _d(m), _d(a), tol_rel, tol_abs, max_iter, _d(P), _d(A),
                            _i(it), _i(nbp), _d(tr) if trace else None)
    if rc:
        raise ValueError(STATUS.get(rc, rc))
    out = dict(P=P, A=A.reshape(9, 9), a=a, iters=int(it[0]), nbp=int(nbp[0]))
    if trace:
        k = int(it[0]) + 1
        out["trace"] = tr[: 4 * k].reshape(k, 4)
    return out


def linear(F, mu, lam):
    """Infinitesimal strain: sigma and C of an isotropic linear phase at F = I + H."""
    F = _f64(F, (9,))
    S = np.zeros(9)
    Cm = np.zeros(81)
    lib().orc_linear(_d(F), mu, lam, _d(S), _d(Cm))
    return S, Cm.reshape(9, 9)


def laminate_linear(F, N, c, mat):
    """Infinitesimal-strain composite boxel in closed form (cheat sheet):
    returns dict(S=sigma_box, C=C_box, a)."""
    F = _f64(F, (9,))
    N = _f64(N, (3,))
    m = _f64(mat, (4,))
    a = np.zeros(3)
    S = np.zeros(9)
    Cb = np.zeros(81)
    rc = lib().orc_laminate_linear(_d(F), _d(N), float(c), _d(m), _d(a), _d(S), _d(Cb))
    if rc:
        raise ValueError(STATUS.get(rc, rc))
    return dict(S=S, C=Cb.reshape(9, 9), a=a)


# ---------------------------------------------------------------- FFT / Gamma
def fft1(x, sign=-1):
    x = np.asarray(x, dtype=np.complex128)
    n = x.size
    ri = _f64(np.stack([x.real, x.imag], -1).ravel())
    out = np.zeros(2 * n)
    lib().orc_fft1(n, sign, _d(ri), _d(out))
    return out[0::2] + 1j * out[1::2]


def fft3(x, sign=-1):
    """3D transform of a complex array shaped [n3][n2][n1] (no normalisation)."""
    x = np.asarray(x, dtype=np.complex128)
    n = np.array([x.shape[2], x.shape[1], x.shape[0]], dtype=np.int32)
    ri = np.ascontiguousarray(np.stack([x.real, x.imag], -1))
    lib().orc_fft3(_i(n), sign, _d(ri))
    return ri[..., 0] + 1j * ri[..., 1]


def kvec(kspace, n, l, xi):
    n = np.asarray(n, dtype=np.int32)
    l = _f64(l)
    xi = np.asarray(xi, dtype=np.int32)
    out = np.zeros(6)
    lib().orc_kvec(kspace, _i(n), _d(l), _i(xi), _d(out))
    return out[0::2] + 1j * out[1::2]


def kvec_row(kspace, n, l, xi, a):
    """The derivative vector of row a of F (the staggered grid has one per row)."""
    n = np.asarray(n, dtype=np.int32)
    l = _f64(l)
    xi = np.asarray(xi, dtype=np.int32)
    out = np.zeros(6)
    lib().orc_kvec_row(kspace, _i(n), _d(l), _i(xi), int(a), _d(out))
    return out[0::2] + 1j * out[1::2]


def gamma_matrix(kspace, n, l, xi):
    n = np.asarray(n, dtype=np.int32)
    l = _f64(l)
    xi = np.asarray(xi, dtype=np.int32)
    out = np.zeros(162)
    lib().orc_gamma_matrix(kspace, _i(n), _d(l), _i(xi), _d(out))
    return (out[0::2] + 1j * out[1::2]).reshape(9, 9)


def apply_G(X, n, l=(1.0, 1.0, 1.0), kspace=ROTATED):
    """G[X] = mu0 Gamma0[X] for a real field X[9][n3][n2][n1]; returns (Y, sum |Y|^2)."""
    n = np.asarray(n, dtype=np.int32)
    X = _f64(X)
    Y = np.zeros_like(X)
    ss = lib().orc_apply_G(kspace, _i(n), _d(_f64(l)), _d(X), _d(Y))
    return Y, ss


# ---------------------------------------------------------------- solve
class _Problem(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("l", C.c_double * 3), ("phase", C.c_void_p), ("nb", C.c_int64),
                ("bidx", C.c_void_p), ("bN", C.c_void_p), ("bc", C.c_void_p), ("mu", C.c_double * 2),
                ("lam", C.c_double * 2), ("Fbar", C.c_double * 9), ("nsteps", C.c_int32)]


class _Options(C.Structure):
    _fields_ = [("solver", C.c_int32), ("kspace", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("fixed_iter", C.c_int32), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32),
                ("cg_fixed_iter", C.c_int32), ("nr_tol_rel", C.c_double), ("nr_tol_abs", C.c_double),
                ("nr_max_iter", C.c_int32), ("c_min", C.c_double), ("mu0", C.c_double), ("nthreads", C.c_int32),
                ("theory", C.c_int32)]


class _Result(C.Structure):
    _fields_ = [("Pbar", C.c_void_p), ("F", C.c_void_p), ("P", C.c_void_p), ("a", C.c_void_p),
                ("iters", C.c_void_p), ("cg_iters", C.c_void_p), ("resid", C.c_void_p), ("nr_iters", C.c_int64),
                ("n_backproj", C.c_int64), ("n_lam_evals", C.c_int64), ("n_operator", C.c_int64)]


DEFAULTS = dict(solver=NEWTON_CG, kspace=ROTATED, tol=1e-8, max_iter=200, fixed_iter=0, cg_tol=1e-3,
                cg_max_iter=2000, cg_fixed_iter=0, nr_tol_rel=1e-12, nr_tol_abs=1e-14, nr_max_iter=50,
                c_min=1e-6, mu0=0.0, nthreads=0, theory=0)


def _problem_struct(prob, keep):
    n = tuple(int(v) for v in prob["n"])
    V = n[0] * n[1] * n[2]
    phase = np.ascontiguousarray(prob["phase"], dtype=np.uint8).reshape(-1)
    assert phase.size == V
    bidx = np.ascontiguousarray(prob["boxel_idx"], dtype=np.int64)
    bN = _f64(prob["boxel_N"]).reshape(-1)
    bc = _f64(prob["boxel_c"]).reshape(-1)
    keep += [phase, bidx, bN, bc]
    s = _Problem()
    s.n = (C.c_int32 * 3)(*n)
    s.l = (C.c_double * 3)(*[float(v) for v in prob.get("l", (1.0, 1.0, 1.0))])
    s.phase = phase.ctypes.data
    s.nb = bidx.size
    s.bidx = bidx.ctypes.data if bidx.size else None
    s.bN = bN.ctypes.data if bidx.size else None
    s.bc = bc.ctypes.data if bidx.size else None
    s.mu = (C.c_double * 2)(*[float(v) for v in prob["mu"]])
    s.lam = (C.c_double * 2)(*[float(v) for v in prob["lam"]])
    s.Fbar = (C.c_double * 9)(*[float(v) for v in np.asarray(prob["Fbar"], dtype=np.float64).reshape(9)])
    s.nsteps = int(prob.get("n_steps", 1))
    return s, V


def _options_struct(opts):
    o = dict(DEFAULTS)
    o.update(opts or {})
    s = _Options()
    for k, v in o.items():
        setattr(s, k, v)
    return s


def solve(prob, opts=None, fields=True, raise_on_error=True):
    """Run the FP64 reference solve.  ``prob`` is the dict produced by
    ``paper_2204_13624_gb300.microstructure`` (keys n, l, phase, boxel_idx,
    boxel_N, boxel_c, mu, lam, Fbar, n_steps)."""
    keep = []
    ps, V = _problem_struct(prob, keep)
    os_ = _options_struct(opts)
    S = ps.nsteps
    nb = ps.nb
    out = dict(Pbar=np.zeros((S, 9)), iters=np.zeros(S, np.int32), cg_iters=np.zeros(S, np.int32),
               resid=np.zeros(S))
    if fields:
        out["F"] = np.zeros((9, V))
        out["P"] = np.zeros((9, V))
        out["a"] = np.zeros((max(nb, 1), 3))
    r = _Result()
    r.Pbar = out["Pbar"].ctypes.data
    r.iters = out["iters"].ctypes.data
    r.cg_iters = out["cg_iters"].ctypes.data
    r.resid = out["resid"].ctypes.data
    r.F = out["F"].ctypes.data if fields else None
    r.P = out["P"].ctypes.data if fields else None
    r.a = out["a"].ctypes.data if fields else None
    rc = lib().orc_solve(C.byref(ps), C.byref(os_), C.byref(r))
    out.update(status=rc, nr_iters=r.nr_iters, n_backproj=r.n_backproj, n_lam_evals=r.n_lam_evals,
               n_operator=r.n_operator)
    if fields:
        out["a"] = out["a"][:nb]
    if rc and raise_on_error:
        raise RuntimeError(f"oracle solve failed: {STATUS.get(rc, rc)}")
    return out


def constitutive_field(prob, F, a=None, opts=None, tangent=False):
    """P (and optionally the per-voxel 9x9 tangent) of a whole field F[9][V]."""
    keep = []
    ps, V = _problem_struct(prob, keep)
    os_ = _options_struct(opts)
    F = _f64(F).reshape(9, V)
    nb = ps.nb
    a = np.zeros((max(nb, 1), 3)) if a is None else _f64(a).reshape(-1, 3).copy()
    P = np.zeros((9, V))
    A = np.zeros((V, 81)) if tangent else None
    rc = lib().orc_constitutive_field(C.byref(ps), C.byref(os_), _d(F), _d(a), _d(P),
                                      _d(A) if tangent else None)
    if rc:
        raise RuntimeError(f"oracle constitutive failed: {STATUS.get(rc, rc)}")
    return (P, a[:nb], A.reshape(V, 9, 9)) if tangent else (P, a[:nb])


def dfmg_subcell_F(F, n, l):
    """F_sub(c, l) of every cell c under the doubly-fine material grid (App. A,
    Eq. constitutive_law): the diagonal of F at c, the off-diagonal pairs
    F_ab, F_ba at c + l_a e_a + l_b e_b.  F [9][V] (x fastest), l in {0,1}^3."""
    G = np.asarray(F, dtype=np.float64).reshape(9, n[2], n[1], n[0])
    out = G.copy()
    npax = {0: 2, 1: 1, 2: 0}
    for comp, (a_, b_) in ((1, (0, 1)), (3, (0, 1)), (2, (0, 2)), (6, (0, 2)), (5, (1, 2)), (7, (1, 2))):
        shift = [0, 0, 0]
        shift[npax[a_]] = -l[a_]
        shift[npax[b_]] = -l[b_]
        out[comp] = np.roll(G[comp], shift, axis=(0, 1, 2))
    return out.reshape(9, -1)


def dfmg_tangent_apply(prob, F, X, opts=None):
    """The tangent of the doubly-fine material grid law at F applied to X
    ([9][V] each): the Hessian of the sub-cell energy acting on X."""
    keep = []
    ps, V = _problem_struct(prob, keep)
    os_ = _options_struct(dict(opts or {}, kspace=STAGGERED_DFMG))
    F = _f64(F).reshape(9, V)
    X = _f64(X).reshape(9, V)
    Y = np.zeros((9, V))
    rc = lib().orc_dfmg_tangent_apply(C.byref(ps), C.byref(os_), _d(F), _d(X), _d(Y))
    if rc:
        raise RuntimeError(f"oracle doubly-fine tangent failed: {STATUS.get(rc, rc)}")
    return Y


def phase_averages(prob, F, a, c_min=1e-6, kspace=None, theory=0):
    """Phase averages Pbar_- (matrix) and Pbar_+ (inclusion) of a state (Sec. 6.2):
    the mean of P over the volume of each phase, where a pure voxel adds its P
    and its volume to its phase and a composite boxel adds c+- P+- and c+- to
    each, P+- the Neo-Hookean stresses at the laminate phase deformations
    F+- = F +- a (x) N / c+- (Sec. 4.1).  Boxels with c+ outside
    [c_min, 1 - c_min] count as pure voxels, as in the solve.  F [9][V],
    a [n_boxels][3] (the converged jump vectors).  Returns [2][9]."""
    phase = np.asarray(prob["phase"]).ravel().copy()
    F = np.asarray(F, dtype=np.float64).reshape(9, -1)
    mu, lam = prob["mu"], prob["lam"]
    if kspace == STAGGERED_DFMG:
        return _phase_averages_dfmg(prob, F, c_min)
    law = (lambda f, m, l: linear(f, m, l)[0]) if theory == 1 else (lambda f, m, l: neohooke(f, m, l, tangent=False))
    # infinitesimal strain: the jump enters symmetrised, eps+- = eps +- sym(a (x) N) / c+-;
    # sigma depends on sym(H) only, so a (x) N itself can be added to F
    sums = np.zeros((2, 9))
    vol = np.zeros(2)
    idx = np.asarray(prob["boxel_idx"], np.int64)
    cs = np.asarray(prob["boxel_c"], float)
    for k, v in enumerate(idx):
        if cs[k] < c_min:
            phase[v] = 0
        elif cs[k] > 1.0 - c_min:
            phase[v] = 1
    for v in np.flatnonzero(phase != 2):
        ph = int(phase[v])
        sums[ph] += law(F[:, v], mu[ph], lam[ph])
        vol[ph] += 1.0
    for k, v in enumerate(idx):
        if phase[v] != 2:
            continue
        c = float(cs[k])
        N = np.asarray(prob["boxel_N"][k], float)
        N = N / np.linalg.norm(N)
        Fb = F[:, v].reshape(3, 3)
        aN = np.outer(a[k], N)
        for ph, cph, Fph in ((1, c, Fb + aN / c), (0, 1.0 - c, Fb - aN / (1.0 - c))):
            sums[ph] += cph * law(Fph.reshape(9), mu[ph], lam[ph])
            vol[ph] += cph
    return np.where(vol[:, None] > 0, sums / np.maximum(vol, 1e-300)[:, None], 0.0)


def _phase_averages_dfmg(prob, F, c_min):
    """Phase averages under the doubly-fine material grid: every sub-cell has
    volume 1/8; a pure sub-cell adds P(F_sub) to its phase, a composite boxel's
    sub-cell adds c+- P+- at F_sub +- a (x) N / c+-, a the laminate jump at
    F_sub (Algorithm 1 solved afresh here)."""
    n = tuple(int(v) for v in prob["n"])
    phase = np.asarray(prob["phase"]).ravel().copy()
    mu, lam = prob["mu"], prob["lam"]
    idx = np.asarray(prob["boxel_idx"], np.int64)
    cs = np.asarray(prob["boxel_c"], float)
    box = {}
    for k, v in enumerate(idx):
        if cs[k] < c_min:
            phase[v] = 0
        elif cs[k] > 1.0 - c_min:
            phase[v] = 1
        else:
            box[int(v)] = k
    sums = np.zeros((2, 9))
    vol = np.zeros(2)
    mat = (mu[0], lam[0], mu[1], lam[1])
    for li in range(8):
        Fs = dfmg_subcell_F(F, n, (li & 1, (li >> 1) & 1, (li >> 2) & 1))
        for v in range(phase.size):
            if phase[v] != 2:
                ph = int(phase[v])
                sums[ph] += 0.125 * neohooke(Fs[:, v], mu[ph], lam[ph], tangent=False)
                vol[ph] += 0.125
                continue
            k = box[v]
            c = float(cs[k])
            N = np.asarray(prob["boxel_N"][k], float)
            N = N / np.linalg.norm(N)
            aN = np.outer(laminate(Fs[:, v], N, c, mat)["a"], N).ravel()
            sums[1] += 0.125 * c * neohooke(Fs[:, v] + aN / c, mu[1], lam[1], tangent=False)
            sums[0] += 0.125 * (1 - c) * neohooke(Fs[:, v] - aN / (1 - c), mu[0], lam[0], tangent=False)
            vol[1] += 0.125 * c
            vol[0] += 0.125 * (1 - c)
    return np.where(vol[:, None] > 0, sums / np.maximum(vol, 1e-300)[:, None], 0.0)


def num_threads():
    return lib().orc_num_threads()
