"""Algorithm LSAR on the device (toeplitz_ols_lsar) against the oracle's lsar on the same series and uniforms.

The random draws are inputs, so both sides sample the same rows: the sampled rows must agree exactly at every lag
(a draw could only differ if its uniform fell within rounding of a running-sum boundary, probability ~1e-16 per
draw), and the compressed estimates within 1e-9 of the coefficient norm (the GPU solves the sampled normal
equations by Cholesky plus one corrected semi-normal-equation step, the oracle by LAPACK least squares; both reach
the same minimiser, and these sampled problems have condition numbers below 1e3).
"""
import math

import numpy as np
import pytest

import oracle
from synthetic import ar_series, lsar_uniforms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tols():
    import paper_2112_12994_gb300 as t
    return t


def _run(tols, y, p_bar, c, unif):
    import torch
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_u = torch.tensor(unif, dtype=torch.float64, device="cuda")
    d_rows = torch.empty((p_bar, c), dtype=torch.int64, device="cuda")
    d_phi = torch.empty((p_bar, p_bar), dtype=torch.float64, device="cuda")
    with tols.Context() as ctx:
        tau, order, phi, rc = tols.toeplitz_ols_lsar(ctx, d_y, y.size, p_bar, c, d_u, d_rows, d_phi)
    return tau, order, phi, rc, d_rows.cpu().numpy(), d_phi.cpu().numpy()


# (n, generating order, p_bar, c): direct residual passes only; the FFT residual pass (rows >= 2^16, lags 33..40)
# over many sampling blocks with a ragged tail; the global-memory Cholesky (p_bar > 144); one block of rows
@pytest.mark.parametrize("n,p,p_bar,c,idx", [(20_000, 3, 10, 2000, 0), (70_000, 5, 40, 400, 1),
                                             (6_000, 2, 150, 600, 2), (100, 1, 4, 50, 3)])
def test_lsar_matches_oracle(tols, n, p, p_bar, c, idx):
    s = ar_series(n, p, config_id=90, series_index=idx, root_lo=1.2, root_hi=3.0)
    unif = lsar_uniforms(p_bar, c, config_id=90, series_index=idx)
    ref = oracle.lsar(s.y, p_bar, c, unif)
    tau, order, phi, rc, rows, phi_all = _run(tols, s.y, p_bar, c, unif)
    assert rc == tols.TOLS_OK
    assert np.array_equal(rows, ref.rows)
    for h in range(1, p_bar + 1):
        want = ref.phi[h - 1]
        got = phi_all[h - 1]
        assert np.linalg.norm(got[:h] - want) <= 1e-9 * np.linalg.norm(want) + 1e-12, h
        assert np.all(got[h:] == 0.0)
    assert np.max(np.abs(tau - ref.tau)) <= 1e-9 * np.max(np.abs(ref.tau)) + 1e-12
    thr = 1.96 / math.sqrt(c)
    if np.all(np.abs(np.abs(ref.tau) - thr) > 1e-6):
        assert order == ref.order
    if order:
        assert np.array_equal(phi[:order], phi_all[order - 1][:order]) and np.all(phi[order:] == 0.0)


def test_lsar_single_lag_single_draw(tols):
    # p_bar = 1, c = 1: one sampled row, phi_1 = y[i + 1] / y[i] (the lag-1 closed form with one draw)
    s = ar_series(500, 1, config_id=90, series_index=4)
    unif = lsar_uniforms(1, 1, config_id=90, series_index=4)
    tau, order, phi, rc, rows, _ = _run(tols, s.y, 1, 1, unif)
    i = int(rows[0, 0])
    assert rows[0, 0] == oracle.lsar(s.y, 1, 1, unif).rows[0, 0]
    assert tau[0] == pytest.approx(s.y[i + 1] / s.y[i], rel=1e-13)


def test_lsar_is_deterministic(tols):
    s = ar_series(70_000, 5, config_id=90, series_index=5)
    unif = lsar_uniforms(40, 400, config_id=90, series_index=5)
    a = _run(tols, s.y, 40, 400, unif)
    b = _run(tols, s.y, 40, 400, unif)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[4], b[4]) and np.array_equal(a[5], b[5])


def test_lsar_rejects_bad_arguments(tols):
    import torch
    y = torch.zeros(100, dtype=torch.float64, device="cuda")
    u = torch.zeros((10, 10), dtype=torch.float64, device="cuda")
    with tols.Context() as ctx:
        with pytest.raises(tols.TolsError):
            tols.toeplitz_ols_lsar(ctx, y, 100, 10, 5, u)       # c < p_bar
        with pytest.raises(tols.TolsError):
            tols.toeplitz_ols_lsar(ctx, y, 100, 300, 400, u)    # p_bar > 256
        with pytest.raises(tols.TolsError):
            tols.toeplitz_ols_lsar(ctx, y, 10, 10, 10, u)       # n <= p_bar


def test_lsar_with_outliers_matches_oracle(tols):
    # the outlier workload of Section 4.2 (0.05 % of the points), where the outliers carry large leverage
    from synthetic import with_outliers
    s = ar_series(40_000, 5, config_id=91, root_lo=1.2, root_hi=3.0)
    y = with_outliers(s.y, 20, config_id=91)
    unif = lsar_uniforms(12, 2000, config_id=91)
    ref = oracle.lsar(y, 12, 2000, unif)
    tau, order, phi, rc, rows, phi_all = _run(tols, y, 12, 2000, unif)
    assert rc == tols.TOLS_OK
    assert np.array_equal(rows, ref.rows)
    assert np.max(np.abs(tau - ref.tau)) <= 1e-9 * np.max(np.abs(ref.tau)) + 1e-12
