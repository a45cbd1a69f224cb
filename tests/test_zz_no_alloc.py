"""The allocation-free Gram entry point (care_gram_noalloc), for callers that cannot
allocate device memory at call time, checked against the workspace-taking care_gram
through the C ABI.  Collected last on purpose (file name), so that a stop-at-first-
failure run has already run every other test."""
import numpy as np
import pytest

import care_inputs as ci
from oracle.lowrank import gram as oracle_gram

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_14742_b300 as m
    m.lib()
    return m


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,a,b", [(100, 3, 5), (300000, 12, 10), (20000, 130, 200), (4000, 1024, 1000)])
def test_gram_noalloc_matches_gram_on_two_calls(pb, dtype, n, a, b):
    tdt = torch.float64 if dtype == "f64" else torch.float32
    X = torch.tensor(ci.random_block(n, a, 71), dtype=tdt, device="cuda")
    Y = torch.tensor(ci.random_block(n, b, 72), dtype=tdt, device="cuda")
    ref = pb.gram(X, Y).cpu().numpy()
    Xh = X.double().cpu().numpy()
    Yh = Y.double().cpu().numpy()
    bound = (n + 2) * (U64 if dtype == "f64" else U32) * (np.abs(Xh).T @ np.abs(Yh))
    for _ in range(2):
        G = pb.gram_noalloc(X, Y).cpu().numpy()
        assert np.all(np.abs(G - ref) <= bound)


def test_gram_noalloc_scratch_reuse_across_shapes(pb):
    """The shared scratch keeps earlier contents: a small product after a large one,
    and the large one again, must not see stale partials."""
    Xa = torch.tensor(ci.random_block(50000, 40, 73), dtype=torch.float64, device="cuda")
    Xb = torch.tensor(ci.random_block(777, 3, 74), dtype=torch.float64, device="cuda")
    ga = pb.gram(Xa, Xa).cpu().numpy()
    gb = pb.gram(Xb, Xb).cpu().numpy()
    for _ in range(2):
        assert np.allclose(pb.gram_noalloc(Xa, Xa).cpu().numpy(), ga, rtol=1e-12, atol=1e-9)
        assert np.allclose(pb.gram_noalloc(Xb, Xb).cpu().numpy(), gb, rtol=1e-12, atol=1e-12)


def test_gram_noalloc_nonsymmetric_after_symmetric(pb):
    """A product X^T Y right after X^T X of the same shape: the symmetric call wrote
    only the upper tiles of the scratch, so the general call must not read any
    lower tile it left behind.  Checked against the oracle's FP64 product."""
    n, a = 30000, 96
    Xh = ci.random_block(n, a, 75)
    Yh = ci.random_block(n, a, 76)
    X = torch.tensor(Xh, device="cuda")
    Y = torch.tensor(Yh, device="cuda")
    bound = (n + 2) * U64 * (np.abs(Xh).T @ np.abs(Yh))
    ref_xy = oracle_gram(Xh, Yh)
    ref_xx = oracle_gram(Xh, Xh)
    for _ in range(2):
        Gs = pb.gram_noalloc(X, X).cpu().numpy()
        assert np.array_equal(Gs, Gs.T)
        assert np.all(np.abs(Gs - ref_xx) <= (n + 2) * U64 * (np.abs(Xh).T @ np.abs(Xh)))
        G = pb.gram_noalloc(X, Y).cpu().numpy()
        assert np.all(np.abs(G - ref_xy) <= bound)


def test_gram_noalloc_rejects_oversized_output(pb):
    cap = pb.GRAM_NOALLOC_SCRATCH_DOUBLES
    X = torch.zeros(8, 1100, dtype=torch.float64, device="cuda")
    Y = torch.zeros(8, cap // 1100 + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(pb.CareError) as e:
        pb.gram_noalloc(X, Y)
    assert e.value.status == 1  # CARE_ERR_INVALID_ARG
