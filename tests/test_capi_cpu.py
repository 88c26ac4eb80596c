"""The C-ABI library builds, loads without a GPU, and exports every function include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("defined", "if", "sizeof"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2511_03598_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("tt_round_fixed", "tt_round_adaptive", "tt_round_deterministic", "ttr_free",
                     "ttr_strerror", "ttr_default_options"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points_work_without_gpu(libpath):
    from paper_2511_03598_gb300 import binding as B
    L = B.lib()
    assert L.ttr_strerror(0) == b"ok"
    assert L.ttr_strerror(4) == b"CholeskyQR breakdown"
    o = B.Options()
    L.ttr_default_options(ctypes.byref(o))
    assert (o.precision, o.adap_r, o.f_init, o.f_inc, o.adap_r_tau_scale) == (0, 0, 0.1, 0.05, 1.0)


def test_argument_errors_are_reported_not_raised_on_host(libpath):
    """Argument checks run before any device work, so they work without a GPU."""
    from paper_2511_03598_gb300 import binding as B
    L = B.lib()
    res = B.Result()
    n = (ctypes.c_int64 * 2)(3, 3)
    r = (ctypes.c_int64 * 3)(2, 2, 1)          # r[0] != 1
    p = (ctypes.c_void_p * 2)(8, 16)
    st = L.tt_round_adaptive(2, n, r, p, 1e-6, 2, ctypes.c_uint64(1), None, None, ctypes.byref(res))
    assert st == 1 and res.status == 1
    assert b"r[0]" in L.ttr_last_error()
    r2 = (ctypes.c_int64 * 3)(1, 2, 1)
    st = L.tt_round_adaptive(2, n, r2, p, -1.0, 2, ctypes.c_uint64(1), None, None, ctypes.byref(res))
    assert st == 1
    st = L.tt_round_fixed(1, n, r2, p, 2, 0, ctypes.c_uint64(1), None, None, ctypes.byref(res))
    assert st == 1
    p_bad = (ctypes.c_void_p * 2)(8, 12)       # misaligned core pointer
    st = L.tt_round_deterministic(2, n, r2, p_bad, 1e-6, None, ctypes.byref(res))
    assert st == 1


def test_sum_argument_errors_on_host(libpath):
    """tt_round_adaptive_sum checks the summand count and every summand before any device work."""
    from paper_2511_03598_gb300 import binding as B
    L = B.lib()
    res = B.Result()
    P64 = ctypes.POINTER(ctypes.c_int64)
    PP = ctypes.POINTER(ctypes.c_void_p)
    n = (ctypes.c_int64 * 2)(3, 3)
    good = (ctypes.c_int64 * 3)(1, 2, 1)
    bad = (ctypes.c_int64 * 3)(1, 2, 2)            # r[d] != 1
    p = (ctypes.c_void_p * 2)(8, 16)
    rs = (P64 * 2)(ctypes.cast(good, P64), ctypes.cast(bad, P64))
    ps = (PP * 2)(ctypes.cast(p, PP), ctypes.cast(p, PP))
    st = L.tt_round_adaptive_sum(0, 2, n, rs, ps, 1e-6, 1, ctypes.c_uint64(1), None, None, ctypes.byref(res))
    assert st == 1 and b"summands" in L.ttr_last_error()
    st = L.tt_round_adaptive_sum(2, 2, n, rs, ps, 1e-6, 1, ctypes.c_uint64(1), None, None, ctypes.byref(res))
    assert st == 1 and b"r[d]" in L.ttr_last_error()
    st = L.tt_round_adaptive_sum(1, 2, n, rs, ps, 0.0, 1, ctypes.c_uint64(1), None, None, ctypes.byref(res))
    assert st == 1 and res.status == 1


def test_server_host_paths_without_gpu(libpath):
    """The request server starts and stops without a GPU; bad requests and requests larger than the
    whole budget are refused at submit, before any device work."""
    import numpy as np
    from paper_2511_03598_gb300 import binding as B
    import workloads as WL
    x = WL.c1()
    with B.Server(workers=2, device_budget=1 << 20, max_sms=10) as srv:
        with pytest.raises(B.TTRoundError) as e:
            srv.submit(x.summands, 1e-6, 2, 1)
        assert e.value.status == 7                       # TTR_ERR_UNSUPPORTED: over the budget
        with pytest.raises(B.TTRoundError) as e:
            srv.submit(x.summands, 0.0, 2, 1)
        assert e.value.status == 1
        bad = [[c.copy() for c in x.summands[0]]]
        bad[0][0] = np.ascontiguousarray(np.concatenate([bad[0][0], bad[0][0]], axis=0))   # r_0 = 2
        with pytest.raises(B.TTRoundError):
            srv.submit(bad, 1e-6, 2, 1)
        st = srv.stats()
        assert st["submitted"] == 0 and st["in_use"] == 0
        res = B.ServerResult()
        assert B.lib().ttr_server_wait(srv._h, 12345, ctypes.byref(res)) == 1   # unknown id
    cfg = B.ServerConfig(0, 0, 1 << 20, 0)
    h = ctypes.c_void_p()
    assert B.lib().ttr_server_create(ctypes.byref(cfg), ctypes.byref(h)) == 1   # no workers
