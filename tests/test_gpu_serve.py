"""Serving (continuous batching): results against the oracle, alone vs in a mix, memory-based admission."""
import numpy as np
import pytest

import oracle
from synthetic import ar_series, batch_shapes
from tests.helpers import coef_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tols():
    import paper_2112_12994_gb300 as t
    return t


def _requests(count, cfg):
    ns, ps = batch_shapes(count, config_id=cfg, n_lo=1_000, n_hi=200_000, p_lo=1, p_hi=120, p_log_uniform=True)
    return [(k, ar_series(int(n), int(p), config_id=cfg, series_index=k, max_log10_bound=6.0).y, int(p))
            for k, (n, p) in enumerate(zip(ns, ps))]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_served_results_match_oracle(tols, prec):
    reqs = _requests(20, 80)
    P = tols.TOLS_MIXED if prec == "mixed" else tols.TOLS_FP64
    with tols.Server(precision=P, arena_bytes=2 << 30) as srv:
        for rid, y, p in reqs:
            assert srv.submit(rid, y, p, 1e-12) == tols.TOLS_OK
        res = srv.run_until_idle()
        st = srv.stats()
    assert len(res) == len(reqs) and st["completed"] == len(reqs) and st["arena_used"] == 0
    tol = 1e-8 if prec == "fp64" else 1e-6
    by_id = {r["id"]: r for r in res}
    for rid, y, p in reqs:
        r = by_id[rid]
        assert r["status"] == tols.TOLS_OK, r["info"]
        assert r["latency_s"] > 0
        sol = oracle.ols_qr(y, p)
        if sol.forward_error_bound() <= tol / 10:
            assert coef_rel_err(r["phi"], sol.phi) <= tol
        assert r["info"]["rnorm"] == pytest.approx(sol.rnorm, rel=1e-11)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_result_is_the_same_alone_and_in_the_mix(tols, prec):
    # the probe's order (>= 16) takes the FFT products in float64, whose work units are fixed per request
    reqs = _requests(24, 81)
    probe = next(r for r in reqs if r[2] >= 16)
    P = tols.TOLS_MIXED if prec == "mixed" else tols.TOLS_FP64
    with tols.Server(precision=P, arena_bytes=2 << 30) as srv:
        srv.submit(1000, probe[1], probe[2], 1e-12)
        alone = srv.run_until_idle()[0]["phi"]
    with tols.Server(precision=P, arena_bytes=2 << 30, max_active=8) as srv:
        # requests arrive while others are on the GPU: submit in waves between steps
        for i, (rid, y, p) in enumerate(reqs):
            srv.submit(rid, y, p, 1e-12)
            if i % 5 == 4:
                srv.step()
        res = srv.run_until_idle()
        res_all = {r["id"]: r for r in res}
    # steps above may have retired some results before run_until_idle polled; they stay queued in the server
    assert probe[0] in res_all
    assert np.array_equal(res_all[probe[0]]["phi"], alone)


def test_admission_by_memory(tols):
    # an arena that holds about two of these requests at a time: the rest wait, all complete
    reqs = [(k, ar_series(100_000, 8, config_id=82, series_index=k).y, 8) for k in range(6)]
    # each request needs about 2.8 MB (float64 + float32 series, two float64 work vectors): 6.5 MiB holds two
    with tols.Server(precision=tols.TOLS_MIXED, arena_bytes=13 << 19) as srv:
        for rid, y, p in reqs:
            assert srv.submit(rid, y, p, 1e-12) == tols.TOLS_OK
        active, queued = srv.step()
        assert active <= 2 and queued == 4
        res = srv.run_until_idle()
        huge = srv.submit(99, np.zeros(10_000_000), 5, 1e-12)
        st = srv.stats()
    assert huge == tols.TOLS_ERR_OOM
    assert sorted(r["id"] for r in res) == list(range(6))
    assert all(r["status"] == tols.TOLS_OK for r in res)
    assert st["arena_used"] == 0
