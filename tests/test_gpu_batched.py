"""Batched solve of independent CAREs (care_solve_batched): every instance matches its
individual care_solve bitwise and meets the residual tolerance."""
import numpy as np
import pytest

import care_inputs as ci
from oracle import dense as od

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_14742_b300 as m
    m.lib()
    return m


def test_batched_matches_individual(pb):
    probs = ci.config_batched(count=6, side_lo=12, side_hi=28, mp_hi=3)
    dev = [(pb.CSR.from_arrays(p.n, p.A.rowptr, p.A.colind, p.A.val), p.B, p.C) for p in probs]
    Zb, infos, st = pb.care_solve_batched(dev, tol=1e-10, prec="mixed", r_cap=128, workers=3)
    assert st == 0
    for (A, B, C), p, Z, inf in zip(dev, probs, Zb, infos):
        Zi, ii = pb.care_solve(A, B, C, tol=1e-10, prec="mixed", r_cap=128)
        assert inf["status"] == "CARE_OK" and inf["res_rel_CtC"] <= 1e-10
        assert torch.equal(Z, Zi), p.name
        R = od.riccati_residual(p.A.to_dense(), p.B, p.C, Z.cpu().numpy() @ Z.cpu().numpy().T)
        assert np.linalg.norm(R) <= 2e-10 * np.linalg.norm(p.C @ p.C.T)


def test_batched_uneven_sizes_order_independent(pb):
    """Instances are scheduled largest-first; results do not depend on the worker count."""
    probs = ci.config_batched(count=5, side_lo=10, side_hi=30, mp_hi=4)
    dev = [(pb.CSR.from_arrays(p.n, p.A.rowptr, p.A.colind, p.A.val), p.B, p.C) for p in probs]
    Z1, _, _ = pb.care_solve_batched(dev, tol=1e-10, prec="mixed", r_cap=128, workers=1)
    Z4, _, _ = pb.care_solve_batched(dev, tol=1e-10, prec="mixed", r_cap=128, workers=4)
    for a, b in zip(Z1, Z4):
        assert torch.equal(a, b)
