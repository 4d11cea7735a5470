"""Planted mistakes: a copy of the oracle with one plausible error must fail
the pin written for that part, so that the pins are known to bite.

Each case copies ``oracle/`` to a temporary directory, plants one mistake in
the C source by a textual substitution (the substituted text must occur
exactly once), builds the copy and runs the pin's check on it in a separate
interpreter; the check prints the pin's error measure, which must be far above
its tolerance (and the unmodified oracle passes the same pin in
``test_oracle_dfmg.py`` / ``test_oracle_small_strain.py``).
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the doubly-fine gather with the material taken at xi + l (the printed sign)
# instead of xi - l: the uniform-deformation pin (mean of the four cells that
# share the edge, on the minus side) must fail
GATHER = ("const long c12 = wrapi(i - l1, n1) + n1 * (wrapi(j - l2, n2) + n2 * k);",
          "const long c12 = wrapi(i + l1, n1) + n1 * (wrapi(j + l2, n2) + n2 * k);")
CHECK_GATHER = r"""
import numpy as np, oracle as orc
from paper_2204_13624_gb300 import microstructure as ms
p = ms.random_boxels((6, 5, 4), seed=42, boxel_frac=0.3, incl_frac=0.3, contrast=10.0)
n = p["n"]; V = n[0] * n[1] * n[2]
F = np.tile((np.eye(3) + 0.05 * np.arange(9).reshape(3, 3) / 9).reshape(9, 1), (1, V))
P3, _ = orc.constitutive_field(p, F, opts=dict(kspace=3))
P0, _ = orc.constitutive_field(p, F)
G = P0[1].reshape(n[2], n[1], n[0])
m = sum(np.roll(G, (0, lb, la), axis=(0, 1, 2)) for la in (0, 1) for lb in (0, 1)) / 4
print(np.abs(P3[1] - m.ravel()).max())
"""

# the small-strain jump with the wrong sign of the stiffness difference: the
# traction-balance pin must fail
JUMP = ("t += (Cm[9 * (3 * i + J) + q] - Cp[9 * (3 * i + J) + q]) * eps[q] * N[J];",
        "t += (Cp[9 * (3 * i + J) + q] - Cm[9 * (3 * i + J) + q]) * eps[q] * N[J];")
CHECK_JUMP = r"""
import numpy as np, oracle as orc
rng = np.random.default_rng(3)
N = rng.normal(size=3); N /= np.linalg.norm(N)
c = 0.4; H = rng.uniform(-1, 1, 9); mat = (1.0, 2.0, 7.0, 4.0)
out = orc.laminate_linear(np.eye(3).ravel() + H, N, c, mat)
a = out["a"]
eps = 0.5 * (H.reshape(3, 3) + H.reshape(3, 3).T)
san = 0.5 * (np.outer(a, N) + np.outer(N, a))
sig = lambda e, mu, lam: lam * np.trace(e) * np.eye(3) + 2 * mu * e
sp = sig(eps + san / c, 7.0, 4.0); sm = sig(eps - san / (1 - c), 1.0, 2.0)
print(np.abs((sp - sm) @ N).max() / np.abs(sp).max())
"""


# the Neo-Hookean stress with F^{-1} where F^{-T} belongs: the pin P = dW/dF
# (central differences of the paper's energy) must fail
NH = ("P[3 * i + Jx] = mu * F[3 * i + Jx] + (lam * lnJ - mu) * G[3 * Jx + i];",
      "P[3 * i + Jx] = mu * F[3 * i + Jx] + (lam * lnJ - mu) * G[3 * i + Jx];")
CHECK_NH = r"""
import numpy as np, oracle as orc
rng = np.random.default_rng(4)
F = (np.eye(3) + 0.2 * rng.uniform(-1, 1, (3, 3))).ravel()
P = orc.neohooke(F, 1.3, 2.1, tangent=False)
h = 1e-6
fd = np.array([(orc.neohooke_energy(F + h * e, 1.3, 2.1) - orc.neohooke_energy(F - h * e, 1.3, 2.1)) / (2 * h)
               for e in np.eye(9)])
print(np.abs(fd - P).max() / np.abs(P).max())
"""

# the staggered symbol with forward differences off the diagonal too: the
# pin that G leaves the printed staggered gradient unchanged must fail
STAG = ("for (int a = 0; a < 3; a++) kr[a][B] = (a == B) ? fwd : bwd;",
        "for (int a = 0; a < 3; a++) kr[a][B] = fwd;")
CHECK_STAG = r"""
import numpy as np, oracle as orc
from test_oracle_fft_gamma import staggered_gradient
n, l = (6, 4, 8), (1.0, 0.8, 1.3)
U = np.random.default_rng(11).normal(size=(3, n[2], n[1], n[0]))
X = staggered_gradient(U, [l[j] / n[j] for j in range(3)])
Y, _ = orc.apply_G(X, n, l, orc.STAGGERED)
print(np.abs(Y - X).max() / np.abs(X).max())
"""


# the rotated symbol without the cosine factors of the other axes (a plain
# central-difference symbol): the pin that G leaves the HEX8R gradient of
# random nodal displacements unchanged must fail
ROT = ("if (m != j) prod *= c[m];", "if (m != j) prod *= 1.0;")
CHECK_ROT = r"""
import numpy as np, oracle as orc
from test_oracle_fft_gamma import hex8r_gradient
n, l = (6, 4, 8), (1.0, 0.5, 2.0)
U = np.random.default_rng(7).normal(size=(3, n[2], n[1], n[0]))
X = hex8r_gradient(U, [l[j] / n[j] for j in range(3)])
Y, _ = orc.apply_G(X, n, l, orc.ROTATED)
print(np.abs(Y - X).max() / np.abs(X).max())
"""


# the laminate with the D matrix of the printed form (diag(N) in every block of
# rows: a -> N (x) a instead of a (x) N).  The residual f = (P+ - P-) N is
# formed without D, so Newton still finds the traction-balanced jump (with a
# wrong Hessian); the boxel tangent A_box = dP_box/dF_box (Eq. Peff:Seff, the
# pin by central differences) must fail
DMAT = ("D[(3 * i + Jx) * 3 + k] = (i == k) ? N[Jx] : 0.0;",
        "D[(3 * i + Jx) * 3 + k] = (Jx == k) ? N[i] : 0.0;")
CHECK_DMAT = r"""
import numpy as np, oracle as orc
rng = np.random.default_rng(5)
mat = (1.0, 2.0, 10.0, 20.0)
worst = 0.0
for _ in range(3):
    N = rng.normal(size=3); N /= np.linalg.norm(N)
    c = rng.uniform(0.2, 0.8)
    F = (np.eye(3) + 0.1 * rng.uniform(-1, 1, (3, 3))).ravel()
    try:
        A = orc.laminate(F, N, c, mat)["A"]
        h = 1e-6
        fd = np.array([(orc.laminate(F + h * e, N, c, mat)["P"] - orc.laminate(F - h * e, N, c, mat)["P"]) / (2 * h)
                       for e in np.eye(9)]).T
    except Exception:
        worst = 1e300
        continue
    worst = max(worst, np.abs(fd - A).max() / np.abs(A).max())
print(worst)
"""


# Sec. 5 normal detection (oracle/normals.py): the second moments taken about
# the boxel's plain centroid instead of the weighted barycentre of its interface
# voxels, or the 1D stencils without their weights r_i = h_j h_k / h_i on
# anisotropic voxels: the planar-interface pin (N . n >= 0.998 where the plane
# cuts across a boxel, for the centroid) or the direct-stencil pin (for the
# weights) must fail.
BARY = ("P = P_all - (wb @ P_all) / wb.sum()", "P = P_all - P_all.mean(axis=0)")
RW = ("r = (hy * hz / hx, hx * hz / hy, hx * hy / hz)", "r = (1.0, 1.0, 1.0)")
CHECK_PLANE = r"""
import numpy as np
from oracle import normals as nrm
from paper_2204_13624_gb300 import microstructure as ms
b, h = %s, %s
nt = np.array([0.48, 0.6, 0.64])
chi = ms.fine_plane_image((64, 64, 64), nt, 3.3, h)
phase, idx, c, N = nrm.block_normals(chi, b, h)
nc = (64 // b[0], 64 // b[1], 64 // b[2])
I, J, K = idx %% nc[0], (idx // nc[0]) %% nc[1], idx // (nc[0] * nc[1])
inner = (I > 0) & (I < nc[0] - 1) & (J > 0) & (J < nc[1] - 1) & (K > 0) & (K < nc[2] - 1)
cut = inner & (c > 0.1) & (c < 0.9)
print(1.0 - float(np.min(N[cut] @ nt)))
"""
CHECK_STENCIL = r"""
import numpy as np
from oracle import normals as nrm
chi = (np.random.default_rng(1).random((6, 8, 10)) < 0.5).astype(np.float64)
h = (0.7, 1.3, 2.1)
r = (h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2])
direct = sum(ri * (np.roll(chi, 1, ax) - 2 * chi + np.roll(chi, -1, ax)) for ax, ri in zip((2, 1, 0), r))
print(np.abs(nrm.stencil_weights(chi, h) - np.abs(direct)).max())
"""


def _mutant_run(tmp_path, old, new, check, fname="combo_oracle.c"):
    tmp_path.mkdir()
    dst = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    src = (dst / fname).read_text()
    assert src.count(old) == 1, "the planted text must occur exactly once"
    (dst / fname).write_text(src.replace(old, new))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT, os.path.join(ROOT, "tests")]))
    out = subprocess.run([sys.executable, "-c", check], env=env, cwd=str(tmp_path), capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    return float(out.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("case", ["gather", "jump", "neohooke", "staggered", "rotated", "dmatrix"])
def test_planted_mistake_fails_its_pin(tmp_path, case):
    old, new, check, tol = {"gather": (GATHER[0], GATHER[1], CHECK_GATHER, 1e-12),
                            "jump": (JUMP[0], JUMP[1], CHECK_JUMP, 1e-13),
                            "neohooke": (NH[0], NH[1], CHECK_NH, 1e-8),
                            "staggered": (STAG[0], STAG[1], CHECK_STAG, 1e-12),
                            "rotated": (ROT[0], ROT[1], CHECK_ROT, 1e-12),
                            "dmatrix": (DMAT[0], DMAT[1], CHECK_DMAT, 1e-6)}[case]
    ctrl = _mutant_run(tmp_path / "control", old, old, check)  # the unmodified oracle passes
    err = _mutant_run(tmp_path / "mutant", old, new, check)
    assert ctrl < tol, (case, ctrl)
    assert err > 1e3 * tol, (case, err)


@pytest.mark.parametrize("case", ["barycentre", "stencil_weights"])
def test_planted_mistake_in_the_normal_detection(tmp_path, case):
    """The moments about the plain centroid fail the planar-interface pin; the
    unweighted stencil (which still fits planes well) fails the direct-stencil
    pin on anisotropic voxels."""
    old, new, check, tol, worse = {
        "barycentre": (BARY[0], BARY[1], CHECK_PLANE % (repr((16, 8, 4)), repr((1, 1, 1))), 0.002, 0.01),
        "stencil_weights": (RW[0], RW[1], CHECK_STENCIL, 1e-12, 1e-3)}[case]
    ctrl = _mutant_run(tmp_path / "control", old, old, check, "normals.py")
    err = _mutant_run(tmp_path / "mutant", old, new, check, "normals.py")
    assert ctrl < tol, (case, ctrl)
    assert err > worse, (case, err)


# Algorithm 2 with the new beta a quarter of the way to the crossed bound
# instead of the midpoint: iterates stay admissible, but the pin that a
# projected step halves one phase Jacobian exactly (J affine in beta by the
# matrix determinant lemma) must fail.  The check prints the number of
# back-projected solves without as many halvings as projections.
BP = ("double bstar = 0.5 * (b0 + bc);", "double bstar = 0.75 * b0 + 0.25 * bc;")
CHECK_BP = r"""
import numpy as np, oracle as orc
from test_oracle_laminate import MAT, critical_cases
bad = 0
for F, N in critical_cases():
    try:
        r = orc.laminate(F.ravel(), N, 0.99625, MAT, trace=True)
    except ValueError:
        continue
    if r["nbp"] == 0:
        continue
    tr = r["trace"]
    halved = sum(abs(tr[k, col] - 0.5 * tr[k - 1, col]) < 1e-12 * max(1.0, tr[k - 1, col])
                 for k in range(1, tr.shape[0]) for col in (1, 2))
    bad += int(halved < r["nbp"])
print(bad)
"""


def test_planted_mistake_in_the_back_projection(tmp_path):
    ctrl = _mutant_run(tmp_path / "control", BP[0], BP[0], CHECK_BP)
    err = _mutant_run(tmp_path / "mutant", BP[0], BP[1], CHECK_BP)
    assert ctrl == 0
    assert err >= 3


# the doubly-fine assembly with the F_12 / F_21 pair taken at c - (l1, l2, 0)
# instead of c + (l1, l2, 0): the law is then no longer the gradient of the
# sub-cell energy, and the finite-difference pin must fail (the check prints
# the largest error relative to |P| over a few entries)
ASM = ("const long v12 = wrapi(i + l1, n1) + n1 * (wrapi(j + l2, n2) + n2 * k);",
       "const long v12 = wrapi(i - l1, n1) + n1 * (wrapi(j - l2, n2) + n2 * k);")
CHECK_ASM = r"""
import numpy as np, oracle as orc
from paper_2204_13624_gb300 import microstructure as ms
from test_oracle_dfmg import cell_energies
p = ms.random_boxels((5, 4, 3), seed=41, boxel_frac=0.35, incl_frac=0.3, contrast=10.0)
V = 60
rng = np.random.default_rng(5)
F = np.eye(3).reshape(9, 1) + 0.08 * rng.uniform(-1, 1, (9, V))
P, _ = orc.constitutive_field(p, F, opts=dict(kspace=3))
worst, h = 0.0, 1e-5
for comp, v in [(1, 7), (3, 30), (1, 44), (0, 12)]:
    Fp, Fm = F.copy(), F.copy()
    Fp[comp, v] += h
    Fm[comp, v] -= h
    dE = (cell_energies(orc, p, Fp) - cell_energies(orc, p, Fm)).sum() / 8.0
    worst = max(worst, abs(dE / (2 * h) - P[comp, v]) / np.abs(P).max())
print(worst)
"""


def test_planted_mistake_in_the_doubly_fine_assembly(tmp_path):
    ctrl = _mutant_run(tmp_path / "control", ASM[0], ASM[0], CHECK_ASM)
    err = _mutant_run(tmp_path / "mutant", ASM[0], ASM[1], CHECK_ASM)
    assert ctrl < 1e-7
    assert err > 1e-3


# the normal without the sign step of Eq. normal:flip: the pin that the ball's
# normals point out of the inclusion (N . x > 0, x from the ball's centre) must
# fail; the check prints the fraction of boxels whose normal points inwards
FLIP = ("return N if float(Nt @ N) > 0.0 else -N  # Eq. normal:flip", "return N")
CHECK_FLIP = r"""
import numpy as np
from oracle import normals as nrm
from paper_2204_13624_gb300 import microstructure as ms
chi = ms.fine_ball_image(64, 0.4)
b = (8, 8, 8)
phase, idx, c, N = nrm.block_normals(chi, b, (1, 1, 1))
nc = 8
I, J, K = idx % nc, (idx // nc) % nc, idx // (nc * nc)
x = np.stack([(I + 0.5) / nc - 0.5, (J + 0.5) / nc - 0.5, (K + 0.5) / nc - 0.5], axis=1)
print(float(np.mean(np.sum(N * x, axis=1) < 0.0)))
"""


def test_planted_mistake_in_the_normal_sign(tmp_path):
    ctrl = _mutant_run(tmp_path / "control", FLIP[0], FLIP[0], CHECK_FLIP, "normals.py")
    err = _mutant_run(tmp_path / "mutant", FLIP[0], FLIP[1], CHECK_FLIP, "normals.py")
    assert ctrl == 0.0
    assert err > 0.1


# nonlinear CG with the Fletcher-Reeves beta dropped (every step the basic
# scheme's): the pin that it needs fewer than a third of the basic scheme's
# iterations must fail; the check prints 3 x its iterations / the basic scheme's
NCG = ("const double beta = (it == 0) ? 0.0 : ss / gg_prev;", "const double beta = 0.0;")
CHECK_NCG = r"""
import numpy as np, oracle as orc
from paper_2204_13624_gb300 import microstructure as ms
p = ms.centred_sphere((12, 12, 12), 0.2, 10.0, np.diag([1.04, 1.0, 0.99]), 2)
rn = orc.solve(p, dict(solver=2, tol=1e-10, max_iter=20000))
rb = orc.solve(p, dict(solver=0, tol=1e-10, max_iter=20000))
print(3.0 * rn["iters"].sum() / rb["iters"].sum())
"""


def test_planted_mistake_in_the_nonlinear_cg(tmp_path):
    ctrl = _mutant_run(tmp_path / "control", NCG[0], NCG[0], CHECK_NCG)
    err = _mutant_run(tmp_path / "mutant", NCG[0], NCG[1], CHECK_NCG)
    assert ctrl < 1.0
    assert err > 2.0
