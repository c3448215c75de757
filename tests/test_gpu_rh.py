"""The Repeated Halving variant of LSAR on the device (toeplitz_ols_rh_lsar) against the oracle's repeated_halving
and rh_lsar on the same series and draws.

Level 0's scores must agree to 1e-7 relative: both sides solve with B^T B, whose condition number here reaches
about 1e6, by different factorisations (Cholesky on the GPU, LU in the oracle). The lags' sampled rows must agree
exactly (a draw could only move if its uniform fell within that relative distance of a running-sum boundary),
and tau to 1e-8 of its largest entry.
"""
import math

import numpy as np
import pytest

import oracle
from synthetic import ar_series, lsar_uniforms, rh_draws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tols():
    import paper_2112_12994_gb300 as t
    return t


def _run(tols, y, p_bar, c, k, keep, gauss, rh_unif, unif):
    import torch
    m = y.size - p_bar
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_sk = torch.tensor(np.concatenate([g.reshape(-1) for g in gauss]), dtype=torch.float64, device="cuda")
    d_rh = torch.tensor(np.stack(rh_unif), dtype=torch.float64, device="cuda")
    d_u = torch.tensor(unif, dtype=torch.float64, device="cuda")
    d_scores = torch.empty(m, dtype=torch.float64, device="cuda")
    d_rows = torch.empty((p_bar, c), dtype=torch.int64, device="cuda")
    with tols.Context() as ctx:
        tau, order, phi, rc = tols.toeplitz_ols_rh_lsar(ctx, d_y, y.size, p_bar, c, k, keep, d_sk, d_rh, d_u,
                                                        d_scores, d_rows)
    return tau, order, phi, rc, d_scores.cpu().numpy(), d_rows.cpu().numpy()


# (n, generating order, p_bar, c, k): six halvings; seven halvings over many sampling blocks; an order above the
# shared-memory Cholesky (p_bar + 1 > 144)
@pytest.mark.parametrize("n,p,p_bar,c,k,idx", [(20_000, 3, 10, 400, 16, 0), (70_000, 5, 40, 600, 8, 1),
                                               (6_000, 2, 150, 600, 8, 2)])
def test_rh_lsar_matches_oracle(tols, n, p, p_bar, c, k, idx):
    y = ar_series(n, p, config_id=92, series_index=idx, root_lo=1.2, root_hi=3.0).y
    X, b = oracle.lag_matrix(y, p_bar)
    C = np.column_stack([X, b])
    keep, gauss, rh_unif = rh_draws(C.shape[0], c, k, c, config_id=92, series_index=idx)
    unif = lsar_uniforms(p_bar, c, config_id=92, series_index=idx)
    rh = oracle.repeated_halving(C, c, c, keep, gauss, rh_unif)
    ref = oracle.rh_lsar(y, p_bar, c, rh, unif)
    tau, order, phi, rc, scores, rows = _run(tols, y, p_bar, c, k, keep, gauss, rh_unif, unif)
    assert rc == tols.TOLS_OK
    assert np.max(np.abs(scores - rh.scores) / rh.scores) <= 1e-7
    assert np.array_equal(rows, ref.rows)
    assert np.max(np.abs(tau - ref.tau)) <= 1e-8 * np.max(np.abs(ref.tau)) + 1e-12
    thr = 1.96 / math.sqrt(c)
    if np.all(np.abs(np.abs(ref.tau) - thr) > 1e-6):
        assert order == ref.order


def test_rh_lsar_rejects_bad_halvings(tols):
    import torch
    y = ar_series(3_000, 2, config_id=92, series_index=5).y
    p_bar, c, k = 4, 100, 4
    m = y.size - p_bar
    keep, gauss, rh_unif = rh_draws(m, c, k, c, config_id=92, series_index=5)
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_sk = torch.tensor(np.concatenate([g.reshape(-1) for g in gauss]), dtype=torch.float64, device="cuda")
    d_rh = torch.tensor(np.stack(rh_unif), dtype=torch.float64, device="cuda")
    d_u = torch.zeros((p_bar, c), dtype=torch.float64, device="cuda")
    bad = [kj.copy() for kj in keep]
    bad[1] = bad[1][::-1].copy()                                   # not increasing
    with tols.Context() as ctx:
        with pytest.raises(tols.TolsError):
            tols.toeplitz_ols_rh_lsar(ctx, d_y, y.size, p_bar, c, k, bad, d_sk, d_rh, d_u)
        bad = [kj.copy() for kj in keep]
        bad[0][-1] = m                                             # outside its level
        with pytest.raises(tols.TolsError):
            tols.toeplitz_ols_rh_lsar(ctx, d_y, y.size, p_bar, c, k, bad, d_sk, d_rh, d_u)
