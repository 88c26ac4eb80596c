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


def serving_requests(ids):
    return [q for q in WL.c4_stream(count=max(ids) + 1, formal=False) if q.rid in ids]


def test_server_serving_stream_requests_alone_and_in_the_mix(B):
    """Two requests of the serving stream at their configured sizes (request 12: 2 summands of ranks
    93 and 31, d = 31, n = 112; request 16: ranks 98 and 77, d = 16, n = 75; both tol 1e-6, formal
    ranks 124 and 175), in the precision the serving measurement uses (sliced, slices from tol: 6,
    ~2.7e-12 per product), against the oracle's rounding of the same sum: identical ranks, the
    represented tensor within 1e-8 of the oracle's.  Each is rounded alone (one worker) and again in a
    mix with the small requests on three workers; the two results agree within the same bar (the
    block loop's SM share, hence its reduction order, differs)."""
    big = serving_requests({12, 16})
    opts = B.options(precision=B.TTR_PREC_SLICED)
    alone = {}
    with B.Server(workers=1, device_budget=16 << 30) as srv:
        for q in big:
            alone[q.rid] = srv.wait(srv.submit(q.tt.summands, q.tol, 0, 1000 + q.rid, opts))
    for q in big:
        got, info = alone[q.rid]
        ref, rinfo = R.tt_round_adaptive_sum(q.tt.summands, q.tol, 1000 + q.rid, block=0)
        assert info["ranks"] == rinfo["ranks"], (q.rid, info["ranks"], rinfo["ranks"])
        assert T.tt_dist(got, ref) <= 1e-8 * T.tt_norm(ref), q.rid
    small = requests()
    with B.Server(workers=3, device_budget=16 << 30) as srv:
        ids = []
        for i, q in enumerate(big):
            ids.append(("big", q, srv.submit(q.tt.summands, q.tol, 0, 1000 + q.rid, opts)))
            for xs, tol, block, seed, prec in small[3 * i:3 * i + 3]:
                ids.append(("small", (xs, tol, block, seed, prec),
                            srv.submit(xs, tol, block, seed, B.options(precision=prec, slices=8))))
        for kind, q, rid in ids:
            got, info = srv.wait(rid)
            if kind == "big":
                ref, rinfo = alone[q.rid]
                assert info["ranks"] == rinfo["ranks"]
                assert T.tt_dist(got, ref) <= 1e-8 * T.tt_norm(ref), q.rid
            else:
                xs, tol, block, seed, prec = q
                ref, rinfo = R.tt_round_adaptive_sum(xs, tol, seed, block=block)
                assert info["ranks"] == rinfo["ranks"]
                assert T.tt_dist(got, ref) <= (1e-10 if prec == 0 else 1e-9) * T.tt_norm(ref)
