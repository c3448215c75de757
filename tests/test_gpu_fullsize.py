"""Parity at the bench's full size and launch configuration: the AR(100), n = 2^22 series of the bench (float64,
product AUTO, which the autotuner resolves to the overlap-save FFT passes at this size).

The solve is graded by the gate of tests/helpers.py against the oracle's full QR (about 5 s on the host). The
fused pass is graded on sampled rows of u (each an explicit dot product of a row of X with v) and on every lag of
X^T u (an explicit dot product over all m rows per lag), with the normwise FFT error bound of test_gpu_fft.py.
"""
import math

import numpy as np
import pytest

import oracle
from synthetic import ar_series
from tests.helpers import assert_solve_parity

pytestmark = pytest.mark.gpu

N_FULL = 1 << 22
P = 100
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def tols():
    import paper_2112_12994_gb300 as t
    return t


@pytest.fixture(scope="module")
def series():
    # the bench workload: roots |r| in U[1.05, 2], Student-t(5) innovations scaled to unit variance
    return ar_series(N_FULL, P, config_id=2, root_lo=1.05, root_hi=2.0, noise="t5")


def test_bench_workload_solve(tols, series):
    sol = oracle.ols_qr(series.y, P)
    with tols.Context(precision=tols.TOLS_FP64) as ctx:
        phi, rnorm, info, rc = tols.toeplitz_ols_solve(ctx, series.y, P, 1e-10)
    assert rc == tols.TOLS_OK, info
    assert info["product_used"] == tols.TOLS_PRODUCT_FFT
    assert_solve_parity(series.y, P, phi, sol, 1e-8)


def test_bench_size_fused_pass_sampled(tols, series):
    import torch
    y = series.y
    n, m = y.size, y.size - P
    rng = np.random.default_rng(11)
    v = rng.standard_normal(P)
    u_old = rng.standard_normal(m)
    c = 0.375
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_v = torch.tensor(v, dtype=torch.float64, device="cuda")
    d_uo = torch.tensor(u_old, dtype=torch.float64, device="cuda")
    d_un = torch.empty(m, dtype=torch.float64, device="cuda")
    d_t = torch.empty(P, dtype=torch.float64, device="cuda")
    with tols.Context(precision=tols.TOLS_FP64, product=tols.TOLS_PRODUCT_FFT) as ctx:
        n2 = tols.toeplitz_ols_gk_pass(ctx, tols.TOLS_FP64, d_y, n, P, d_v, d_uo, c, d_un, d_t)
    u = d_un.cpu().numpy()
    t = d_t.cpu().numpy()
    k = 8 * U64 * math.log2(2048)
    win = math.sqrt(2048) * np.max(np.abs(y))
    # sampled rows of u = X v - c u_old (first, last and random rows, each tile position)
    rows = np.unique(np.concatenate([[0, 1, m - 2, m - 1], rng.integers(0, m, 256)]))
    for i in rows:
        xi = y[P + i - np.arange(P) - 1]
        ref = xi @ v - c * u_old[i]
        assert abs(u[i] - ref) <= k * win * np.linalg.norm(v) + 2 * U64 * abs(c * u_old[i]), i
    # every lag of X^T u (u as the GPU produced it)
    ref_t = np.array([np.dot(u, y[P - 1 - j: P - 1 - j + m]) for j in range(P)])
    tiles = math.ceil(m / (2048 - 112))
    bound = k * win * math.sqrt(tiles) * np.linalg.norm(u) + (m + P) * U64 * np.array(
        [np.dot(np.abs(u), np.abs(y[P - 1 - j: P - 1 - j + m])) for j in range(P)])
    assert np.all(np.abs(t - ref_t) <= bound)
    assert n2 == pytest.approx(float(u @ u), rel=64 * U64)


def test_bench_workload_lsar(tols, series):
    """Algorithm LSAR at the bench's size (p_bar = 120, c = 2000): lags 1 and 2 against the oracle on the full
    data (their scores need only y and phi_hat_1), every lag against the exact PACF within the sampling error, and
    a bitwise repeat."""
    import torch
    from synthetic import lsar_uniforms
    p_bar, c = 120, 2000
    y = series.y
    m = y.size - p_bar
    unif = lsar_uniforms(p_bar, c, config_id=2)
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_u = torch.tensor(unif, dtype=torch.float64, device="cuda")
    outs = []
    with tols.Context(precision=tols.TOLS_FP64) as ctx:
        for _ in range(2):
            d_rows = torch.empty((p_bar, c), dtype=torch.int64, device="cuda")
            d_phi = torch.empty((p_bar, p_bar), dtype=torch.float64, device="cuda")
            tau, order, phi, rc = tols.toeplitz_ols_lsar(ctx, d_y, y.size, p_bar, c, d_u, d_rows, d_phi)
            assert rc == tols.TOLS_OK
            outs.append((tau, d_rows.cpu().numpy(), d_phi.cpu().numpy()))
        tau_exact, _, _, _ = tols.toeplitz_ols_pacf(ctx, y, p_bar, 1e-10)
    tau, rows, phi_all = outs[0]
    assert np.array_equal(outs[1][0], tau) and np.array_equal(outs[1][1], rows) and np.array_equal(outs[1][2], phi_all)
    assert np.all((rows >= 0) & (rows < m))
    lev1 = oracle.leverage_p1(y[:m + 1])
    assert np.array_equal(rows[0], oracle.leverage_sample(lev1, unif[0]))
    phi1 = oracle.compressed_ols(y[:m + 1], 1, rows[0], lev1[rows[0]], c)
    assert phi_all[0, 0] == pytest.approx(phi1[0], rel=1e-11)
    lev2, pi2, _ = oracle.leverage_step(y[:m + 2], 2, phi_all[0, :1], lev1)
    assert np.array_equal(rows[1], oracle.leverage_sample(lev2, unif[1]))
    phi2 = oracle.compressed_ols(y[:m + 2], 2, rows[1], pi2[rows[1]], c)
    assert np.linalg.norm(phi_all[1, :2] - phi2) <= 1e-9 * np.linalg.norm(phi2)
    assert np.max(np.abs(tau - tau_exact)) <= 8.0 / math.sqrt(c)
