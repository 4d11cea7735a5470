"""The Green operator entry point that allocates no device memory.

combo_apply_G_noalloc serves callers that cannot call cudaMalloc (code
inside a memory pool or arena it does not own, loops that must not
allocate): its scratch is one fixed device array inside libcombo.so.  This
checks it through the C ABI against combo_apply_G, the allocating entry
point, on two calls in a row, within the FP64 parity tolerance used by the
other Green-operator tests, and against the oracle's Green operator (Sec. 3,
Eq. Gamma0: explicit 9x9 symbol matrices per frequency, its own complex FFT).
The file name sorts last so that a run stopping at the first failure has run
every other test before it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cb():
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    return combo


@pytest.mark.parametrize("n", [(32, 16, 24), (64, 8, 16), (16, 32, 36), (32, 32, 32), (2, 3, 4)])
@pytest.mark.parametrize("kspace", [0, 1])
def test_noalloc_matches_allocating_entry_point(cb, n, kspace):
    import torch

    V = n[0] * n[1] * n[2]
    l = (1.0, 0.8, 1.3)
    g = torch.Generator(device="cpu").manual_seed(sum(n) + kspace)
    X = torch.randn((9, V), dtype=torch.float64, generator=g).cuda()
    ref, ss_ref = cb.apply_G(X, n, l, kspace, cb.FP64)
    scale = ref.abs().max().item()
    for _ in range(2):  # two calls in a row share (and must clear) the scratch
        Y = torch.full_like(X, float("nan"))
        ss = cb.apply_G_noalloc(X, Y, n, l, kspace)
        torch.cuda.synchronize()
        assert (Y - ref).abs().max().item() <= 1e-12 * scale
        assert abs(ss - ss_ref) <= 1e-11 * ss_ref


@pytest.mark.parametrize("kspace", [0, 1])
def test_noalloc_matches_the_oracle(cb, kspace):
    """Y = G[X] of the entry point against the oracle's Green operator on a
    ragged grid (odd, mixed 2^a 3^b sides), on two calls in a row."""
    import torch

    import oracle

    n = (24, 9, 16)
    V = n[0] * n[1] * n[2]
    l = (1.0, 0.7, 1.2)
    rng = np.random.default_rng(11 + kspace)
    Xh = rng.standard_normal((9, V))
    ref, _ = oracle.apply_G(Xh.reshape(9, n[2], n[1], n[0]), n, l, kspace)
    ref = ref.reshape(9, V)
    X = torch.from_numpy(Xh).cuda()
    for _ in range(2):
        Y = torch.full_like(X, float("nan"))
        cb.apply_G_noalloc(X, Y, n, l, kspace)
        torch.cuda.synchronize()
        assert np.max(np.abs(Y.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_noalloc_rejects_the_staggered_grid(cb):
    import torch

    X = torch.zeros((9, 8 * 8 * 8), dtype=torch.float64, device="cuda")
    with pytest.raises(cb.ComboError) as e:
        cb.apply_G_noalloc(X, X, (8, 8, 8), kspace=cb.STAGGERED)
    assert e.value.code == -1 and "kspace" in str(e.value)


def test_noalloc_allocates_nothing_and_works_in_place(cb):
    import torch

    n = (32, 32, 32)
    V = 32 ** 3
    X = torch.randn((9, V), dtype=torch.float64, device="cuda")
    ref, _ = cb.apply_G(X, n)
    Y = torch.empty_like(X)
    cb.apply_G_noalloc(X, Y, n)  # first call on the device: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    cb.apply_G_noalloc(X, Y, n)
    Z = X.clone()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    cb.apply_G_noalloc(Z, Z, n, want_sumsq=False)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free2 == free1  # torch's caching allocator already holds Z's block
    assert free1 <= free0  # only torch's clone can have taken memory
    scale = ref.abs().max().item()
    assert (Y - ref).abs().max().item() <= 1e-12 * scale
    assert (Z - ref).abs().max().item() <= 1e-12 * scale


def test_noalloc_rejects_oversized_grids(cb):
    import torch

    X = torch.zeros((9, 64 * 64 * 64), dtype=torch.float64, device="cuda")
    with pytest.raises(cb.ComboError) as e:
        cb.apply_G_noalloc(X, X, (64, 64, 64))
    assert e.value.code == -1 and "too large" in str(e.value) and "259520" in str(e.value)
    with pytest.raises(cb.ComboError):
        cb.apply_G_noalloc(X, X, (128, 4, 4))
