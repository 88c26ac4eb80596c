"""Calls on different streams from different host threads, each with a share of the SMs, give the
same results as alone: every result is checked against the oracle within the parity bars of the
FP64 form (identical ranks, represented tensor within 1e-10)."""
import threading

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


def _cases():
    return [("c1", WL.c1(), 1e-6, 2, 5), ("c3s", WL.c3(d=6, n=16, r=10), 1e-8, 0, 7),
            ("ragged", WL.copies_plus_noise(8, 5, 7, 5, 3, 2, 1e-6, "ragged"), 1e-5, 3, 11),
            ("c1b", WL.c1(seed=4), 1e-7, 3, 13)]


def test_concurrent_streams_match_the_oracle(B):
    cases = _cases()
    refs = [R.tt_round_adaptive(x.cores, tol, seed=seed, block=blk, nrmx=x.norm) for _, x, tol, blk, seed in cases]
    dev = [[torch.from_numpy(np.ascontiguousarray(c)).to("cuda") for c in x.cores] for _, x, _, _, _ in cases]
    torch.cuda.synchronize()
    share = max(1, torch.cuda.get_device_properties(0).multi_processor_count // len(cases))
    out = [None] * len(cases)
    errs = []

    def run(i):
        try:
            _, x, tol, blk, seed = cases[i]
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                opts = B.options(nrmx=x.norm, max_sms=share)
                for rep in range(3):           # several rounds so that the calls overlap on the device
                    with B.round_adaptive(dev[i], tol, blk, seed, opts, stream=s) as y:
                        out[i] = (y.ranks, y.to_numpy())
        except Exception as e:                  # reported after the join
            errs.append((i, repr(e)))

    threads = [threading.Thread(target=run, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errs, errs
    for (name, x, tol, blk, seed), (ref, info), (ranks, cores) in zip(cases, refs, out):
        assert ranks == info["ranks"], name
        assert T.tt_dist(cores, ref) <= 1e-10 * T.tt_norm(ref), name
