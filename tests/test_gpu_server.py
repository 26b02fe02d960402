"""Request server: results in a concurrent mix equal the standalone solves.

Every right-hand side of a request runs as a column solve on its own workspace, with
the same kernels in the same order as amge_pcg_solve, so its result must be
identical (bit for bit) whatever else runs at the same time.  Faults are made on
the host: cancellation, a zero timeout, a budget too small for any workspace, a
non-finite right-hand side.
"""
import numpy as np
import pytest

from conftest import hierarchy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amge():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05613_gb300 import amge as mod

    return mod


@pytest.fixture(scope="module")
def hiers(amge):
    return {key: amge.amge_upload_levels(hierarchy(*key, True))
            for key in [("hcurl", 16, 2), ("hdiv", 24, 3), ("hcurl", 24, 3)]}


def _standalone(amge, h, B, prec):
    n, k = B.shape
    X = np.zeros_like(B)
    its = []
    for c in range(k):
        b = torch.from_numpy(np.ascontiguousarray(B[:, c])).cuda()
        x = torch.empty_like(b)
        st, info = amge.amge_pcg_solve(h, b, x, rtol=1e-8, precision=prec)
        assert st == amge.AMGE_OK
        X[:, c] = x.cpu().numpy()
        its.append(info[0]["iters"])
    return X, its


@pytest.mark.parametrize("prec", [0, 1])
def test_server_mix_equals_standalone(amge, hiers, prec):
    from paper_2107_05613_gb300.inputs import rhs_vector

    keys = list(hiers)
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(12):
        key = keys[i % len(keys)]
        h = hiers[key]
        k = int(rng.integers(1, 5))
        B = rhs_vector(1000 + i, h.n, k).reshape(h.n, k)
        reqs.append((h, B))
    sv = amge.amge_server_create(0, 6)
    tickets = []
    outs = []
    for h, B in reqs:
        X = np.zeros_like(B)
        outs.append(X)
        tickets.append(amge.amge_submit(sv, h, np.ascontiguousarray(B), X, nrhs=B.shape[1], precision=prec))
    results = [amge.amge_wait(sv, t) for t in tickets]
    stats = amge.amge_server_stats(sv)
    sv.destroy()
    assert stats["running_columns"] == 0 and stats["queued"] == 0
    for (h, B), X, (st, infos) in zip(reqs, outs, results):
        assert st == amge.AMGE_OK
        Xa, its = _standalone(amge, h, B, prec)
        assert np.array_equal(X, Xa)
        assert [i["iters"] for i in infos] == its
        assert all(i["true_relres"] <= 1e-8 and i["time_ms"] > 0 for i in infos)


def test_server_cancel_timeout_budget_nonfinite(amge, hiers):
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = hiers[("hcurl", 24, 3)]
    b = rhs_vector(7, h.n)
    sv = amge.amge_server_create(0, 1)                 # one slot: later requests queue
    x1 = np.zeros_like(b)
    t1 = amge.amge_submit(sv, h, b, x1, rtol=1e-30, maxit=400)   # runs all 400 iterations
    x2 = np.zeros_like(b)
    t2 = amge.amge_submit(sv, h, b, x2)
    st, _ = amge.amge_wait(sv, t1, timeout_ms=0)
    assert st == amge.AMGE_ETIMEOUT
    amge.amge_cancel(sv, t2)
    st2, _ = amge.amge_wait(sv, t2)
    assert st2 == amge.AMGE_ECANCELED
    st1, info1 = amge.amge_wait(sv, t1)
    assert st1 == amge.AMGE_ENOTCONV and info1[0]["iters"] == 400
    bad = np.stack([b, b], axis=1).copy()
    bad[5, 1] = np.nan
    xb = np.zeros_like(bad)
    tb = amge.amge_submit(sv, h, bad, xb, nrhs=2)
    stb, infob = amge.amge_wait(sv, tb)
    assert stb == amge.AMGE_ENONFINITE
    assert infob[0]["status"] == amge.AMGE_OK and infob[1]["status"] == amge.AMGE_ENONFINITE
    with pytest.raises(amge.AmgeError):
        amge.amge_cancel(sv, tb)                       # already collected
    sv.destroy()
    tiny = amge.amge_server_create(1 << 20, 4)        # 1 MiB: no workspace fits
    x3 = np.zeros_like(b)
    t3 = amge.amge_submit(tiny, h, b, x3)
    st3, _ = amge.amge_wait(tiny, t3)
    assert st3 == amge.AMGE_ENOMEM
    tiny.destroy()
