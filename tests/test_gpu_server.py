"""The request server (ttr_server_*) on the GPU: requests of different shapes, tolerances and
precisions in flight at once, each result equal to the oracle's rounding of the same sum; a budget
that admits one request at a time still completes every request, in order of arrival."""
import numpy as np
import pytest

import workloads as WL
from oracle import rounding as R
from oracle import tt as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_2511_03598_gb300 import build
    build.build()
    from paper_2511_03598_gb300 import binding
    assert torch.cuda.is_available()
    return binding


def requests():
    rng = np.random.default_rng(40)
    out = []
    x = WL.c1()
    out.append((x.summands, 1e-6, 2, 11, 0))
    out.append((x.summands, 1e-6, 0, 12, 1))
    for i, (d, n, rs, tol) in enumerate([(5, 6, [3, 4], 1e-3), (6, [4, 5, 3, 6, 4, 5], [2, 5, 3], 1e-5),
                                          (4, 9, [6], 1e-8), (7, 3, [2, 2, 2, 2], 1e-2)]):
        xs = [WL.random_tt(rng, d, n, r) for r in rs]
        for xx, c in zip(xs, rng.standard_normal(len(xs))):
            xx[0] = xx[0] * c
        out.append((xs, tol, i % 2 + 1, 20 + i, i % 2))
    return out


def check(B, srv, reqs):
    ids = []
    for xs, tol, block, seed, prec in reqs:
        ids.append(srv.submit(xs, tol, block, seed, B.options(precision=prec, slices=8)))
    for rid, (xs, tol, block, seed, prec) in zip(ids, reqs):
        got, info = srv.wait(rid)
        ref, rinfo = R.tt_round_adaptive_sum(xs, tol, seed, block=block)
        assert info["ranks"] == rinfo["ranks"], (rid, info["ranks"], rinfo["ranks"])
        rel = T.tt_dist(got, ref) / T.tt_norm(ref)
        assert rel <= (1e-10 if prec == 0 else 1e-9), (rid, rel)
        assert info["ms_run"] > 0.0 and info["footprint"] > 0


def test_server_mixed_requests(B):
    reqs = requests()
    with B.Server(workers=3, device_budget=8 << 30) as srv:
        check(B, srv, reqs)
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["in_use"] == 0


def test_server_budget_admits_one_at_a_time(B):
    reqs = requests()
    with B.Server(workers=3, device_budget=1 << 30) as srv:
        # the largest footprint decides: a budget just above it admits one request at a time
        ids = [srv.submit(xs, tol, block, seed, B.options(precision=prec, slices=8)) for xs, tol, block, seed, prec in reqs]
        infos = [srv.wait(i)[1] for i in ids]
        st = srv.stats()
    biggest = max(i["footprint"] for i in infos)
    assert st["peak_in_use"] <= 1 << 30
    with B.Server(workers=3, device_budget=biggest) as srv:
        ids = [srv.submit(xs, tol, block, seed, B.options(precision=prec, slices=8)) for xs, tol, block, seed, prec in reqs]
        infos = [srv.wait(i)[1] for i in ids]
        st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["peak_in_use"] <= biggest
    # first come, first served: requests are admitted in the order they were submitted
    assert [i["admit_order"] for i in infos] == list(range(len(reqs)))
