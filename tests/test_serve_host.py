"""Host-side parts of the request server that need no GPU: the device-memory
estimate used for admission and the validation of server configurations."""
import numpy as np
import pytest

from paper_2110_15676_gb300 import workloads as W


@pytest.fixture(scope="module")
def afc():
    from paper_2110_15676_gb300 import afc as A
    return A


def _req(afc, kind, elem, n, prec=0):
    wl = W.stationary_inflow(elem, n) if kind == afc.AFC_REQ_STATIONARY else W.rotating_transient(elem, n)
    return afc.Request(kind, elem, n, wl.eps, wl.c, wl.b, wl.u0, wl.dir_mask, wl.u_dir, f=wl.f,
                       opts=afc.default_opts(precision=prec), steps=5)


def test_estimate_grows_with_size_and_pattern(afc):
    for kind in (afc.AFC_REQ_TRANSIENT, afc.AFC_REQ_STATIONARY):
        small = _req(afc, kind, "p1", 6).estimate_bytes()
        big = _req(afc, kind, "p1", 9).estimate_bytes()
        q1 = _req(afc, kind, "q1", 9).estimate_bytes()
        assert 0 < small < big < q1
    # a stationary solve holds the MC pair data and a Krylov basis on top
    assert _req(afc, afc.AFC_REQ_STATIONARY, "q1", 8).estimate_bytes() > \
        _req(afc, afc.AFC_REQ_TRANSIENT, "q1", 8).estimate_bytes()
    # lower bound: the 27 diagonals of AA alone in FP64
    N = 9 ** 3
    assert _req(afc, afc.AFC_REQ_TRANSIENT, "q1", 9).estimate_bytes() > 27 * 8 * N


def test_bad_server_configurations_are_rejected_on_the_host(afc):
    for kw in ({"mode": 7}, {"max_active": 0}, {"hbm_budget": 0}, {"stationary_workers": 0},
               {"stationary_workers": 65}, {"max_chunk": 0}, {"builders": 0}, {"builders": 65}):
        with pytest.raises(afc.AfcError) as e:
            afc.Server(**kw)
        assert e.value.status == afc.AFC_E_INVALID
    c = afc.serve_config()
    assert c.mode == afc.AFC_SERVE_BATCHED and c.max_chunk >= 1 and c.hbm_budget > 0 and c.builders >= 1
