"""Order sweep / PACF (toeplitz_ols_pacf) against the oracle's fits of every order.

tau_h, the last coefficient of the AR(h) fit, is compared with the oracle's at each lag within the solve gate's
coefficient tolerance (the series are well conditioned at every order), and the order estimate is compared with
the one the oracle's taus give under the same rule.
"""
import numpy as np
import pytest

import oracle
from synthetic import ar_series

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tols():
    import paper_2112_12994_gb300 as t
    return t


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,p,h_max,idx", [(20_000, 3, 12, 0), (50_000, 8, 40, 1), (6_000, 1, 5, 2)])
def test_pacf_matches_oracle(tols, prec, n, p, h_max, idx):
    s = ar_series(n, p, config_id=80, series_index=idx, root_lo=1.5, root_hi=3.0)
    ref_tau, ref_order = oracle.pacf(s.y, h_max)
    P = tols.TOLS_FP64 if prec == "fp64" else tols.TOLS_MIXED
    with tols.Context(precision=P) as ctx:
        tau, order, infos, rc = tols.toeplitz_ols_pacf(ctx, s.y, h_max, 1e-12)
    assert rc in (tols.TOLS_OK, tols.TOLS_NOT_CONVERGED)
    scale = np.max(np.abs(ref_tau))
    assert np.all(np.abs(tau - ref_tau) <= 1e-7 * scale + 1e-9), np.max(np.abs(tau - ref_tau))
    thr = 1.96 / np.sqrt(n - np.arange(1, h_max + 1))
    if np.all(np.abs(np.abs(ref_tau) - thr) > 1e-6):      # no lag sits on the threshold
        assert order == ref_order
    if abs(ref_tau[p - 1]) > 2 * thr[p - 1]:
        assert order >= p                                 # the generating order is found when its lag is clear


def test_pacf_rejects_bad_arguments(tols):
    with tols.Context() as ctx:
        y = np.zeros(10)
        with pytest.raises(tols.TolsError):
            tols.toeplitz_ols_pacf(ctx, y, 10, 1e-12)     # needs n > h_max
        with pytest.raises(tols.TolsError):
            tols.toeplitz_ols_pacf(ctx, y, 0, 1e-12)
