"""Algorithm SRHT on the device (toeplitz_ols_srht) against the oracle's srht_ols on the same series and draws.

The Hadamard stages run in the order of the definition's recursion on both sides, so the transformed rows agree
closely; the GPU then solves the compressed problem through its normal equations (Cholesky), the oracle by
LAPACK least squares, so the coefficients agree to about kappa^2 u (below 1e-9 for these well-conditioned
series).
"""
import numpy as np
import pytest

import oracle
from synthetic import ar_series, srht_draws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tols():
    import paper_2112_12994_gb300 as t
    return t


def _run(tols, y, p, signs, rows):
    import torch
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_s = torch.tensor(signs, dtype=torch.float64, device="cuda")
    d_r = torch.tensor(np.asarray(rows, dtype=np.int64), device="cuda")
    d_phi = torch.empty(p, dtype=torch.float64, device="cuda")
    with tols.Context() as ctx:
        rc = tols.toeplitz_ols_srht(ctx, d_y, y.size, p, d_s, d_r, d_phi)
    return rc, d_phi.cpu().numpy()


# m2 = 512 (one shared-memory chunk), 4,096 (one full chunk), 32,768 (chunks plus three global stages)
@pytest.mark.parametrize("n,p,c,idx", [(500, 2, 100, 0), (3_000, 3, 300, 1), (20_000, 10, 1_000, 2)])
def test_srht_matches_oracle(tols, n, p, c, idx):
    y = ar_series(n, p, config_id=93, series_index=idx).y
    signs, rows = srht_draws(n - p, c, config_id=93, series_index=idx)
    ref = oracle.srht_ols(y, p, rows, signs)
    rc, phi = _run(tols, y, p, signs, rows)
    assert rc == tols.TOLS_OK
    assert np.linalg.norm(phi - ref) <= 1e-9 * np.linalg.norm(ref)


def test_srht_every_row_once_is_the_exact_fit(tols):
    # S takes each of the m2 padded rows once: S H D is orthogonal, so the fit is the exact OLS fit
    y = ar_series(3_000, 3, config_id=93, series_index=3).y
    signs, _ = srht_draws(2_997, 1, config_id=93, series_index=3)
    rows = np.random.default_rng(0).permutation(4096)
    rc, phi = _run(tols, y, 3, signs, rows)
    assert rc == tols.TOLS_OK
    exact = oracle.ols_qr(y, 3).phi
    assert np.linalg.norm(phi - exact) <= 1e-10 * np.linalg.norm(exact)


def test_srht_rejects_a_row_outside_the_padded_range(tols):
    y = ar_series(3_000, 3, config_id=93, series_index=4).y
    signs, rows = srht_draws(2_997, 50, config_id=93, series_index=4)
    rows = rows.copy()
    rows[7] = 4096
    with pytest.raises(tols.TolsError):
        _run(tols, y, 3, signs, rows)
