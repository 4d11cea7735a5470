"""Input generator checks (geometry only)."""
import math

import numpy as np

from paper_2204_13624_gb300 import microstructure as ms


def test_paper_sphere_block_count():
    # paper Sec. 6.2: the R = 0.4 ball on a 256^3 image coarse-grained to 32^3
    # gives 2624 composite voxels
    assert ms.fine_sphere_block_count(256, 32, 0.4) == 2624


def test_sphere_volume_is_exact():
    p = ms.sphere_32()
    V = 32 ** 3
    R = (3 * 0.2 / (4 * math.pi)) ** (1 / 3)
    vol = (np.sum(p["phase"] == 1) + p["boxel_c"].sum()) / V
    assert abs(vol - 4 / 3 * math.pi * R ** 3) < 1e-12
    assert np.all((p["boxel_c"] > 0) & (p["boxel_c"] < 1))
    assert np.allclose(np.linalg.norm(p["boxel_N"], axis=1), 1.0)
    assert np.all(p["phase"][p["boxel_idx"]] == 2)
    assert np.sum(p["phase"] == 2) == p["boxel_idx"].size
    assert np.all(np.diff(p["boxel_idx"]) > 0)


def test_normals_point_out_of_inclusion():
    p = ms.sphere_32()
    n = 32
    idx = p["boxel_idx"]
    i, j, k = idx % n, (idx // n) % n, idx // (n * n)
    ctr = (np.stack([i, j, k], 1) + 0.5) / n - 0.5
    assert np.all(np.sum(ctr * p["boxel_N"], 1) > 0)


def test_single_box_volume_against_sampling():
    v = ms.sphere_box_volume(1.0, *[np.array([x]) for x in (0.3, 0.9, -0.2, 0.5, 0.1, 0.8)])
    g = (np.arange(200) + 0.5) / 200
    X, Y, Z = np.meshgrid(0.3 + 0.6 * g, -0.2 + 0.7 * g, 0.1 + 0.7 * g, indexing="ij")
    mc = np.mean(X ** 2 + Y ** 2 + Z ** 2 < 1) * 0.6 * 0.7 * 0.7
    assert abs(v[0] - mc) < 2e-4


def test_random_spheres_and_fibres_small():
    p = ms.spheres_256(n=64, vf=0.1)
    assert p["boxel_idx"].size > 0 and np.all(p["phase"][p["boxel_idx"]] == 2)
    vf = (np.sum(p["phase"] == 1) + p["boxel_c"].sum()) / 64 ** 3
    assert abs(vf - 0.1) < 0.02
    q = ms.fibres_512(n=64, vf=0.08)
    vf = (np.sum(q["phase"] == 1) + q["boxel_c"].sum()) / 64 ** 3
    assert abs(vf - 0.08) < 0.03
    assert np.allclose(q["boxel_N"][:, 2], 0.0)
