"""ttr_partial_contractions_noalloc (scratch in a static device array, no allocation) against
ttr_partial_contractions, through the C ABI.  Named so that pytest collects it last; it must pass
in a fresh process and after the other tests alike (the static scratch keeps the previous call's
contents, which must not matter)."""
import ctypes

import numpy as np
import pytest

import workloads as WL

torch = pytest.importorskip("torch")

TOL = 1e-12          # the relative max-norm tolerance of the partial-contraction parity tests


@pytest.fixture(scope="module")
def B():
    from paper_2511_03598_gb300 import build
    build.build()
    from paper_2511_03598_gb300 import binding
    return binding


def _dev(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).to("cuda") for c in cores]


def _close(got, ref):
    assert set(got) == set(ref)
    for k in ref:
        g, e = got[k].cpu().numpy(), ref[k].cpu().numpy()
        assert g.shape == e.shape
        scale = max(np.abs(e).max(), 1e-300)
        assert np.abs(g - e).max() <= TOL * scale, (k, np.abs(g - e).max() / scale)


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_on_two_calls(B):
    assert torch.cuda.is_available()
    big = _dev(WL.c2().cores)                                    # d=20, n=50, r=210: 7.4 MB of scratch
    ragged = _dev(WL.random_tt(np.random.default_rng(3), 5, [3, 7, 1, 5, 4], [4, 9, 2, 6]))
    calls = [(big, 2024, 0, 80, 2), (ragged, 77, 3, 24, 2)]      # the second call is smaller: stale
    for cores, seed, c0, c1, t in calls:                         # scratch from the first is left over
        got = B.partial_contractions_noalloc(cores, seed, c0, c1, t)
        torch.cuda.synchronize()
        ref = B.partial_contractions(cores, seed, c0, c1, t, precision=B.TTR_PREC_FP64)
        _close(got, ref)


@pytest.mark.gpu
def test_noalloc_same_call_twice_into_the_same_outputs(B):
    cores = _dev(WL.c3(d=6, n=16, r=10).cores)
    ref = B.partial_contractions(cores, 5, 0, 40, 3, precision=B.TTR_PREC_FP64)
    out = {k: torch.full_like(v, float("nan")) for k, v in ref.items()}
    for _ in range(2):
        B.partial_contractions_noalloc(cores, 5, 0, 40, 3, out=out)
        torch.cuda.synchronize()
        _close(out, ref)


@pytest.mark.gpu
def test_noalloc_checks_caller_outputs(B):
    """The C side cannot check buffer sizes: the binding refuses a wrong `out` before any call."""
    cores = _dev(WL.c3(d=4, n=8, r=5).cores)
    good = {k: torch.empty((c.shape[0], 16), dtype=torch.float64, device="cuda") for k, c in
            zip(range(2, 5), cores[1:])}
    for k, bad in [(3, torch.empty((good[3].shape[0] + 1, 16), dtype=torch.float64, device="cuda")),
                   (4, torch.empty(good[4].shape, dtype=torch.float32, device="cuda")),
                   (2, torch.empty((16, good[2].shape[0]), dtype=torch.float64, device="cuda").t())]:
        with pytest.raises(ValueError):
            B.partial_contractions_noalloc(cores, 1, 0, 16, 2, out={**good, k: bad})
    with pytest.raises(ValueError):
        B.partial_contractions_noalloc(cores, 1, 0, 16, 2, out={k: v for k, v in good.items() if k != 3})


def test_noalloc_rejects_shapes_beyond_the_static_limit(B):
    """Host-side check, before any device work: runs without a GPU."""
    L = B.lib()
    d = 3
    n = (ctypes.c_int64 * d)(4, 4096, 4)
    r = (ctypes.c_int64 * (d + 1))(1, 512, 512, 1)
    p = (ctypes.c_void_p * d)(8, 16, 24)
    W = (ctypes.c_void_p * d)(0, 32, 40)
    st = L.ttr_partial_contractions_noalloc(d, n, r, p, ctypes.c_uint64(1), 0, 64, 2, W, None)
    assert st == 7                                               # TTR_ERR_UNSUPPORTED
    msg = L.ttr_last_error().decode()
    assert "TTR_STATIC_SCRATCH_BYTES" in msg and str(32 << 20) in msg
