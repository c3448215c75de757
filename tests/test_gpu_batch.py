"""Batched solves (one tile list over many series, per-series scalar steps) against the oracle and against
single-series solves, float64 and mixed precision."""
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


@pytest.fixture(scope="module", params=["fp64", "mixed"])
def prec(request):
    return request.param


@pytest.fixture(scope="module")
def ctx(tols, prec):
    c = tols.Context(precision=tols.TOLS_FP64 if prec == "fp64" else tols.TOLS_MIXED)
    yield c
    c.close()


def _batch(count, cfg, n_lo, n_hi, p_lo, p_hi):
    ns, ps = batch_shapes(count, config_id=cfg, n_lo=n_lo, n_hi=n_hi, p_lo=p_lo, p_hi=p_hi)
    ys = [ar_series(int(n), int(p), config_id=cfg, series_index=k, max_log10_bound=6.0).y
          for k, (n, p) in enumerate(zip(ns, ps))]
    return ys, [int(p) for p in ps]


def test_batch_matches_oracle(tols, ctx, prec):
    ys, ps = _batch(24, 40, 3_000, 120_000, 1, 120)
    phis, rn, infos, rc = tols.toeplitz_ols_solve_batched(ctx, ys, ps, 1e-12)
    assert rc == tols.TOLS_OK, [i["status"] for i in infos]
    tol = 1e-8 if prec == "fp64" else 1e-6
    for y, p, phi, r, info in zip(ys, ps, phis, rn, infos):
        sol = oracle.ols_qr(y, p)
        if sol.forward_error_bound() <= tol / 10:
            assert coef_rel_err(phi, sol.phi) <= tol, (p, info)
        assert r == pytest.approx(sol.rnorm, rel=1e-11)
        assert info["ne_ratio"] <= 1e-12


def test_series_result_does_not_depend_on_the_batch(tols, ctx):
    # a series' reduction order depends only on its own tiles, so alone or in any mix its phi is bitwise equal
    ys, ps = _batch(16, 41, 5_000, 300_000, 2, 80)
    phis, _, _, rc = tols.toeplitz_ols_solve_batched(ctx, ys, ps, 1e-12)
    assert rc == tols.TOLS_OK
    for k in (0, 7, 15):
        alone, _, _, rc1 = tols.toeplitz_ols_solve_batched(ctx, [ys[k]], [ps[k]], 1e-12)
        assert rc1 == tols.TOLS_OK
        assert np.array_equal(alone[0], phis[k]), k
    # and reordering the batch does not change anything either
    order = list(reversed(range(16)))
    phis_r, _, _, _ = tols.toeplitz_ols_solve_batched(ctx, [ys[k] for k in order], [ps[k] for k in order], 1e-12)
    for j, k in enumerate(order):
        assert np.array_equal(phis_r[j], phis[k])


def test_batch_per_series_errors(tols, ctx):
    good = ar_series(8_000, 6, config_id=42).y
    bad = good.copy()
    bad[100] = np.inf
    ys = [good, np.ones(4), bad, good]
    ps = [6, 4, 6, 6]
    # the binding raises on a negative batch status, so call the C ABI directly to see per-series codes
    phis, rn, infos, rc = _raw_batched(tols, ctx, ys, ps)
    assert rc == tols.TOLS_ERR_NONFINITE
    st = [i["status"] for i in infos]
    assert st[0] == tols.TOLS_OK and st[3] == tols.TOLS_OK
    assert st[1] == tols.TOLS_ERR_ARG
    assert st[2] == tols.TOLS_ERR_NONFINITE
    assert np.array_equal(phis[0], phis[3])


def _raw_batched(tols, ctx, ys, ps):
    import ctypes
    count = len(ys)
    ys = [np.ascontiguousarray(y, dtype=np.float64) for y in ys]
    phis = [np.zeros(int(p)) for p in ps]
    yp = (ctypes.c_void_p * count)(*[y.ctypes.data for y in ys])
    pp = (ctypes.c_void_p * count)(*[f.ctypes.data for f in phis])
    ns = np.array([y.size for y in ys], dtype=np.int64)
    pv = np.array(ps, dtype=np.int32)
    rn = np.zeros(count)
    infos = (tols.tols_info * count)()
    rc = tols.lib.toeplitz_ols_solve_batched(ctx.handle, count, ctypes.cast(yp, ctypes.c_void_p), ns.ctypes.data,
                                             pv.ctypes.data, 1e-12, ctypes.cast(pp, ctypes.c_void_p), rn.ctypes.data,
                                             ctypes.cast(infos, ctypes.c_void_p))
    return phis, rn, [i.as_dict() for i in infos], rc


def test_batch_rank_deficient_member_gets_min_norm(tols, ctx):
    ys = [np.full(700, 1.5), ar_series(9_000, 4, config_id=43).y]
    phis, rn, infos, rc = tols.toeplitz_ols_solve_batched(ctx, ys, [5, 4], 1e-12)
    assert np.allclose(phis[0], 0.2, atol=1e-10)
    assert coef_rel_err(phis[1], oracle.ols_qr(ys[1], 4).phi) <= 1e-6


def test_batched_device_equals_host_batched(tols, ctx):
    import torch
    ys, ps = _batch(10, 44, 2_000, 90_000, 1, 90)
    phis, rn, infos, rc = tols.toeplitz_ols_solve_batched(ctx, ys, ps, 1e-12)
    d_ys = [torch.tensor(y, dtype=torch.float64, device="cuda") for y in ys]
    d_phi = torch.empty(sum(ps), dtype=torch.float64, device="cuda")
    rn_d, infos_d, rc_d = tols.toeplitz_ols_solve_batched_device(ctx, d_ys, ps, d_phi, 1e-12)
    assert rc == rc_d == tols.TOLS_OK
    out = d_phi.cpu().numpy()
    off = 0
    for phi, p in zip(phis, ps):
        assert np.array_equal(out[off:off + p], phi)
        off += p


@pytest.mark.parametrize("product", ["auto", "fft", "direct"])
def test_batch_products_by_order(tols, prec, product):
    """Products per batched series: DIRECT forces the direct products; FFT takes the overlap-save float64 FFT
    products (N = 2,048) from pad16(p + 1) = 32 up; AUTO the choice timed per order class, which every context of
    the process shares (a second context plans alike). Whichever the choice, every series matches the oracle (a
    mixed series runs its Gram pass and checks in float64 too)."""
    ys, ps = _batch(12, 43, 5_000, 40_000, 2, 200)
    P = tols.TOLS_FP64 if prec == "fp64" else tols.TOLS_MIXED
    prod = {"auto": tols.TOLS_PRODUCT_AUTO, "fft": tols.TOLS_PRODUCT_FFT, "direct": tols.TOLS_PRODUCT_DIRECT}[product]
    with tols.Context(precision=P, product=prod) as c:
        phis, rn, infos, rc = tols.toeplitz_ols_solve_batched(c, ys, ps, 1e-12)
    with tols.Context(precision=P, product=prod) as c:
        _, _, infos2, _ = tols.toeplitz_ols_solve_batched(c, ys, ps, 1e-12)
    tol = 1e-8 if prec == "fp64" else 1e-6
    for k, (y, p, info) in enumerate(zip(ys, ps, infos)):
        pp = ((p + 1 + 15) // 16) * 16
        if product == "direct":
            assert info["product_used"] == tols.TOLS_PRODUCT_DIRECT, (p, info)
        elif product == "fft":
            want = tols.TOLS_PRODUCT_FFT if pp >= 32 else tols.TOLS_PRODUCT_DIRECT
            assert info["product_used"] == want, (p, info)
        else:
            assert info["product_used"] in (tols.TOLS_PRODUCT_FFT, tols.TOLS_PRODUCT_DIRECT), (p, info)
            assert infos2[k]["product_used"] == info["product_used"], (p, info, infos2[k])
        assert info["nfft"] == (2048 if info["product_used"] == tols.TOLS_PRODUCT_FFT else 0), info
        sol = oracle.ols_qr(y, p)
        if sol.forward_error_bound() <= tol / 10:
            assert coef_rel_err(phis[k], sol.phi) <= tol, (p, info)
        assert rn[k] == pytest.approx(sol.rnorm, rel=1e-11)


def test_profiled_batch_matches_graph_replays(tols, prec):
    """With the library's per-launch events on, a batch launches its passes one by one instead of replaying its
    CUDA graphs: the results are bitwise those of the graph replays, and the batched kernel classes record the
    launches (float64 FFT and direct passes for a batch with orders on both sides of the FFT threshold)."""
    ys, ps = _batch(10, 44, 5_000, 60_000, 2, 120)
    P = tols.TOLS_FP64 if prec == "fp64" else tols.TOLS_MIXED
    with tols.Context(precision=P) as c:
        phis, rn, infos, rc = tols.toeplitz_ols_solve_batched(c, ys, ps, 1e-12)
        tols.toeplitz_ols_profile(c, True)
        phis2, rn2, infos2, rc2 = tols.toeplitz_ols_solve_batched(c, ys, ps, 1e-12)
        names = tols.PROFILE_CLASS_NAMES
        counts = {names[k]: tols.toeplitz_ols_profile_read(c, k) for k in range(tols.TOLS_PROFILE_CLASSES)}
        tols.toeplitz_ols_profile(c, False)
    assert rc == rc2
    for a, b in zip(phis, phis2):
        assert np.array_equal(a, b)
    used = {i["product_used"] for i in infos}
    if tols.TOLS_PRODUCT_FFT in used:
        assert counts["batch_f64_fft"][0] > 0 and counts["batch_f64_fft"][1] > 0
    if tols.TOLS_PRODUCT_DIRECT in used:
        assert counts["batch_f64_direct"][0] > 0
    assert counts["precond"][0] > 0
