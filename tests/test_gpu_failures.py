"""Failure detection without a GPU fault: every failure becomes a status code
that the call returns, and the context stays usable afterwards.

* a bounded wait that runs out (the bulk-copy kernels polled zero times on
  their tile barriers) -> COMBO_E_TIMEOUT;
* the laminate Newton iteration cap (Algorithm 1) set to one iteration ->
  COMBO_E_LAMINATE, with the failing boxel's state in the error text;
* a NaN planted on the host in one voxel of a checkpoint image ->
  COMBO_E_NAN from the residual evaluation;
* an allocation failure planted by the host-side hook -> COMBO_E_OOM, with
  nothing leaked.

After each failure the same problem solves normally on the same context.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

E_OOM, E_LAMINATE, E_NAN, E_TIMEOUT = -2, -4, -6, -7


@pytest.fixture(scope="module")
def cb():
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    return combo


def small_balls(n=(64, 64, 64), steps=1, radius=6.0):
    from paper_2204_13624_gb300 import microstructure as ms

    return ms.random_spheres(n, radius, 0.12, 77, 10.0, np.diag([1.04, 1.0, 1.0]), steps)


def test_wait_that_runs_out_returns_timeout(cb):
    # 64^3 in the refined form runs the TMA-tiled y- and z-passes, whose
    # tile waits poll their mbarrier; with no poll allowed every wait runs
    # out, the blocks drain their own copies and raise COMBO_E_TIMEOUT
    p = small_balls()
    with pytest.raises(cb.ComboError) as e:
        cb.solve(p, solver=1, precision=cb.FP32_REFINED, tol=1e-8, wait_poll_cap=-1)
    assert e.value.code == E_TIMEOUT
    g = cb.solve(p, solver=1, precision=cb.FP32_REFINED, tol=1e-8)
    assert g["steps_done"] == 1 and np.all(g["resid"] <= 1e-8)


def test_wait_cap_option_is_checked(cb):
    from paper_2204_13624_gb300 import microstructure as ms

    with pytest.raises(cb.ComboError) as e:
        cb.solve(ms.homogeneous((8, 8, 8)), wait_poll_cap=-2)
    assert e.value.code == -1


@pytest.mark.parametrize("prec", [0, 2])
def test_laminate_iteration_cap_returns_laminate_error(cb, prec):
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.sphere_32(n_steps=1)
    with pytest.raises(cb.ComboError) as e:
        cb.solve(p, solver=1, precision=prec, nr_max_iter=1)
    assert e.value.code == E_LAMINATE
    msg = str(e.value)
    assert "boxel" in msg and "iteration cap" in msg and "F_box" in msg
    g = cb.solve(p, solver=1, precision=prec)
    assert g["steps_done"] == 1


@pytest.mark.parametrize("prec", [0, 2])
def test_nan_in_an_imported_state_returns_nan(cb, prec):
    p = small_balls((16, 16, 16), steps=2, radius=3.0)
    V = 16 ** 3
    nb = int(p["boxel_idx"].size)
    s = cb.Solve(p, solver=1, precision=prec, tol=1e-8)
    s.advance_steps(1)
    img = bytearray(s.export_state())
    s.close()
    # the image ends with F [9][V] and the jump vectors [nb][3] (FP64)
    F = np.frombuffer(img, dtype=np.float64, count=9 * V, offset=len(img) - 8 * (9 * V + 3 * nb)).copy()
    pure = int(np.flatnonzero(np.asarray(p["phase"]) == 0)[5])
    F[4 * V + pure] = np.nan
    img[len(img) - 8 * (9 * V + 3 * nb):len(img) - 8 * 3 * nb] = F.tobytes()
    t = cb.Solve(p, solver=1, precision=prec, tol=1e-8)
    t.import_state(bytes(img))
    with pytest.raises(cb.ComboError) as e:
        t.advance()
    t.close()
    assert e.value.code == E_NAN
    g = cb.solve(p, solver=1, precision=prec, tol=1e-8)
    assert g["steps_done"] == 2


def test_allocation_failure_returns_oom_and_leaks_nothing(cb):
    import torch

    p = small_balls((32, 32, 32), steps=1, radius=4.0)
    cb.solve(p, solver=1, precision=cb.FP32_REFINED_DF)  # warm: tuner, module load
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for after in (0, 3, 9, 17, 25):
            cb.fault_inject_alloc(after)
            with pytest.raises(cb.ComboError) as e:
                cb.solve(p, solver=1, precision=cb.FP32_REFINED_DF)
            assert e.value.code == E_OOM, (after, str(e.value))
        cb.fault_inject_alloc(2)
        with pytest.raises(cb.ComboError) as e:
            cb.solve_batch([p, p], solver=1, precision=cb.FP32_REFINED_DF)
        assert e.value.code == E_OOM
    finally:
        cb.fault_inject_alloc(-1)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 4 << 20
    g = cb.solve(p, solver=1, precision=cb.FP32_REFINED_DF)
    assert g["steps_done"] == 1
