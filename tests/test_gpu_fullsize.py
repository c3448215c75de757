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
    assert info["product_used"] in (tols.TOLS_PRODUCT_FFT, tols.TOLS_PRODUCT_FFT4096), info
    assert info["nfft"] in (2048, 4096), info
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


@pytest.mark.parametrize("p,n", [(100, (1 << 25) + 3), (500, (1 << 24) + 3)])
def test_float_fft_pass_at_bench_lengths(tols, p, n):
    """The float overlap-save pass (register-blocked; window spectra and u_old rows arrive by bulk copies) over
    millions of rows: every CTA runs many tiles (at p = 100 more than one float flush of its spectral sums), and the
    last tile's rows are not a multiple of four (its last rows are read directly, not copied). Dense u: sampled
    rows of u_new against explicit dot products of rows of X, and every lag of X^T u normwise. Sparse u (v = 0,
    c = -1, so u_new = u_old exactly): X^T u against the explicit sum over the nonzero rows, which no tile can drop
    unnoticed."""
    import torch
    N, U32 = 4096, 2.0 ** -24
    y = ar_series(n, 3, config_id=54, series_index=p).y
    m = n - p
    yr = y.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(p)
    d_y = torch.tensor(y, dtype=torch.float32, device="cuda")
    d_t = torch.empty(p, dtype=torch.float64, device="cuda")
    L = N - ((p + 15) // 16) * 16
    tiles = math.ceil(m / L)
    assert (m - (tiles - 1) * L) % 4 != 0          # the ragged-tail case this test is about
    k = 8 * U32 * math.log2(N)
    win = math.sqrt(N) * np.max(np.abs(yr))
    with tols.Context(precision=tols.TOLS_MIXED, product=tols.TOLS_PRODUCT_FFT) as ctx:
        # dense
        v = rng.standard_normal(p)
        vr = v.astype(np.float32).astype(np.float64)
        u_old = rng.standard_normal(m).astype(np.float32)
        c = 0.375
        d_v = torch.tensor(v, dtype=torch.float64, device="cuda")
        d_uo = torch.tensor(u_old, device="cuda")
        d_un = torch.empty(m, dtype=torch.float32, device="cuda")
        n2 = tols.toeplitz_ols_gk_pass(ctx, tols.TOLS_MIXED, d_y, n, p, d_v, d_uo, c, d_un, d_t)
        u = d_un.cpu().numpy().astype(np.float64)
        t = d_t.cpu().numpy()
        rows = np.unique(np.concatenate([[0, 1, L - 1, L, m - 4, m - 3, m - 2, m - 1], rng.integers(0, m, 256)]))
        for i in rows:
            ref = yr[p + i - np.arange(p) - 1] @ vr - c * float(u_old[i])
            assert abs(u[i] - ref) <= k * win * np.linalg.norm(vr) + 2 * U32 * abs(c * u_old[i]), i
        ynorm = np.linalg.norm(yr)
        ref_t = np.array([np.dot(u, yr[p - 1 - j: p - 1 - j + m]) for j in range(p)])
        assert np.max(np.abs(t - ref_t)) <= 16 * U32 * math.log2(N) * math.sqrt(2.0) * np.linalg.norm(u) * ynorm
        assert n2 == pytest.approx(float(u @ u), rel=1e-5)
        # sparse: the first and last rows of tiles spread over the CTAs, the ragged tail, random rows
        nz = np.unique(np.concatenate([
            [0, m - 3, m - 2, m - 1],
            np.arange(0, tiles, 97) * L, np.minimum(np.arange(1, tiles, 89) * L - 1, m - 1),
            rng.integers(0, m, 64)]))
        us = np.zeros(m, dtype=np.float32)
        us[nz] = rng.standard_normal(nz.size).astype(np.float32)
        d_uo = torch.tensor(us, device="cuda")
        d_v.zero_()
        tols.toeplitz_ols_gk_pass(ctx, tols.TOLS_MIXED, d_y, n, p, d_v, d_uo, -1.0, d_un, d_t)
        assert np.array_equal(d_un.cpu().numpy(), us)
        t = d_t.cpu().numpy()
    usd = us[nz].astype(np.float64)
    ref_t = np.array([usd @ yr[p - 1 - j + nz] for j in range(p)])
    touched = np.unique(nz // L).size
    bound = k * win * math.sqrt(touched) * np.linalg.norm(usd) + 4 * U32 * np.array(
        [np.abs(usd) @ np.abs(yr[p - 1 - j + nz]) for j in range(p)])
    assert np.all(np.abs(t - ref_t) <= bound), np.max(np.abs(t - ref_t) / bound)
