"""Pins for the CPU oracle (no GPU): hand-written fixtures, exact rational solves, closed forms, invariants.

Each test would fail under a plausible mistake in the oracle (a shifted lag, a transposed operand, a dropped
term, a wrong sign); test_planted_mistakes_are_caught checks a few of those directly.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import tols
from synthetic import ar_series, coefficients_from_inverse_roots, draw_inverse_roots, rng_for, simulate
from tests.exact import normal_equations_exact, solve_spd_exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["xphi_n5_p2.json", "xphi_n7_p3.json"])
def test_lag_matrix_matches_hand_written_xphi(name):
    g = _golden(name)
    X, b = oracle.lag_matrix(np.array(g["y"], float), g["p"])
    assert X.tolist() == g["X"]
    assert b.tolist() == g["b"]


def _int_series(seed, n, lo=-9, hi=9):
    return np.random.default_rng(seed).integers(lo, hi + 1, size=n)


def _rows_from_definition(y, p):
    # independent index expression from the 1-based eq. (xphi): row i (1..n-p) = (y_{p+i-1}, ..., y_i)
    n = len(y)
    rows = [[int(y[(p + i - 1) - k - 1]) for k in range(p)] for i in range(1, n - p + 1)]
    rhs = [int(y[p + i - 1]) for i in range(1, n - p + 1)]
    return rows, rhs


@pytest.mark.parametrize("seed,n,p", [(1, 30, 3), (2, 41, 5), (3, 25, 1), (4, 60, 7)])
def test_oracle_equals_exact_rational_solution(seed, n, p):
    y = _int_series(seed, n)
    rows, rhs = _rows_from_definition(y, p)
    G, h = normal_equations_exact(rows, rhs)
    phi_exact = solve_spd_exact(G, h)
    sol = oracle.ols_qr(y.astype(float), p)
    ref = np.array([float(v) for v in phi_exact])
    assert np.linalg.norm(sol.phi - ref) <= 1e-12 * np.linalg.norm(ref)
    # residual norm against the exact rational residual
    r2 = sum((Fraction(bb) - sum(Fraction(r[j]) * phi_exact[j] for j in range(p))) ** 2 for r, bb in zip(rows, rhs))
    assert sol.rnorm == pytest.approx(math.sqrt(float(r2)), rel=1e-12)
    assert not sol.rank_deficient


def test_p1_closed_form():
    # p = 1: phi = sum_i y_i y_{i+1} / sum_i y_i^2 over the n-1 rows (exact rationals)
    y = _int_series(11, 200)
    num = sum(Fraction(int(y[i])) * int(y[i + 1]) for i in range(len(y) - 1))
    den = sum(Fraction(int(y[i])) ** 2 for i in range(len(y) - 1))
    sol = oracle.ols_qr(y.astype(float), 1)
    assert sol.phi[0] == pytest.approx(float(num / den), rel=1e-14)


def test_noise_free_recursion_is_recovered_exactly():
    # y_t = 1.5 y_{t-1} - 0.75 y_{t-2} + 0.125 y_{t-3}: dyadic coefficients and integer starts keep y exact
    phi = np.array([1.5, -0.75, 0.125])
    y = [3.0, -2.0, 5.0]
    for _ in range(37):
        y.append(phi[0] * y[-1] + phi[1] * y[-2] + phi[2] * y[-3])
    sol = oracle.ols_qr(np.array(y), 3)
    assert np.max(np.abs(sol.phi - phi)) < 1e-11
    assert sol.rnorm < 1e-9 * np.linalg.norm(y)


@pytest.mark.parametrize("p", [1, 3, 8])
def test_constant_series_gives_min_norm(p):
    # X = k * ones(m, p): every phi with sum(phi) = 1 fits exactly; the minimum-norm one is 1/p each
    sol = oracle.ols_qr(np.full(50, 3.0), p)
    assert sol.rank_deficient or p == 1
    assert np.allclose(sol.phi, 1.0 / p, atol=1e-12)
    assert sol.rnorm < 1e-12


def test_periodic_series_min_norm_matches_svd_lstsq():
    # period 3 with p = 6: rank 3; compare with LAPACK's SVD-based gelsd and check phi lies in the row space
    y = np.tile([1.0, -2.0, 0.5], 30)
    p = 6
    sol = oracle.ols_qr(y, p)
    X, b = oracle.lag_matrix(y, p)
    ref = scipy.linalg.lstsq(X, b, lapack_driver="gelsd")[0]
    assert sol.rank_deficient
    assert np.allclose(sol.phi, ref, atol=1e-10)
    _, s, Vt = np.linalg.svd(X)
    null = Vt[s < 1e-10 * s[0]]
    assert np.max(np.abs(null @ sol.phi)) < 1e-10


def test_blocked_qr_equals_single_block():
    s = ar_series(5000, 12, config_id=7)
    a = oracle.ols_qr(s.y, 12)
    b = oracle.ols_qr(s.y, 12, block_rows=333)
    assert np.max(np.abs(a.phi - b.phi)) < 1e-13 * np.max(np.abs(a.phi)) * 100
    assert a.rnorm == pytest.approx(b.rnorm, rel=1e-13)


def test_products_reduce_to_convolution_and_correlation():
    # (X v)[i] = sum_j y[p-1+i-j] v[j] is the 'valid' convolution of y[0..n-2] with v;
    # (X^T u)[j] is the 'valid' correlation of y[0..n-2] with u, read backwards.
    rng = np.random.default_rng(5)
    for n, p in [(40, 1), (57, 6), (300, 31)]:
        y = rng.standard_normal(n)
        v = rng.standard_normal(p)
        u = rng.standard_normal(n - p)
        assert np.allclose(oracle.matvec(y, p, v), np.convolve(y[:-1], v, mode="valid"), rtol=1e-13, atol=1e-13)
        assert np.allclose(oracle.rmatvec(y, p, u), np.correlate(y[:-1], u, mode="valid")[::-1], rtol=1e-12,
                           atol=1e-12)
        # adjoint identity <X v, u> = <v, X^T u>
        assert np.dot(oracle.matvec(y, p, v), u) == pytest.approx(np.dot(v, oracle.rmatvec(y, p, u)), rel=1e-12)


def test_normal_equation_invariant_and_loop_residual():
    s = ar_series(3000, 5, config_id=8)
    sol = oracle.ols_qr(s.y, 5)
    assert sol.ne_ratio < 1e-12
    # X^T r with plain loops, no matrix built
    y, p = s.y, 5
    g = [0.0] * p
    for i in range(len(y) - p):
        r = y[p + i] - sum(y[p + i - j - 1] * sol.phi[j] for j in range(p))
        for j in range(p):
            g[j] += y[p + i - j - 1] * r
    assert np.allclose(g, sol.g, atol=1e-8)
    assert np.linalg.norm(g) < 1e-9 * sol.norm2 * sol.rnorm


def test_residual_check_detects_wrong_phi():
    s = ar_series(2000, 4, config_id=9)
    sol = oracle.ols_qr(s.y, 4)
    bad = sol.phi.copy()
    bad[2] += 1e-3
    rn, _, ratio = oracle.residual_check(s.y, 4, bad, norm2=sol.norm2)
    assert ratio > 1e-6 and rn > sol.rnorm


def test_consistency_error_shrinks_like_inverse_sqrt_n():
    errs = {}
    for n in (2000, 20000, 200000):
        e = []
        for k in range(6):
            s = ar_series(n, 4, config_id=10, series_index=k)
            e.append(np.linalg.norm(oracle.ols_qr(s.y, 4).phi - s.phi_true))
        errs[n] = float(np.mean(e))
    slope = np.polyfit(np.log10(list(errs)), np.log10(list(errs.values())), 1)[0]
    assert -0.8 < slope < -0.3, errs


def test_gram_matches_exact_and_displacement_identity():
    y = _int_series(21, 35)
    p = 4
    rows, rhs = _rows_from_definition(y, p)
    Gx, hx = normal_equations_exact(rows, rhs)
    G, h = oracle.gram(y.astype(float), p)
    assert G.tolist() == [[float(v) for v in row] for row in Gx]
    assert h.tolist() == [float(v) for v in hx]
    # G[j+1,k+1] = G[j,k] + y[a-1] y[c-1] - y[a-1+m] y[c-1+m],  a = p-1-j, c = p-1-k, m = n-p
    m = len(y) - p
    for j in range(p - 1):
        for k in range(p - 1):
            a, c = p - 1 - j, p - 1 - k
            assert G[j + 1, k + 1] == G[j, k] + y[a - 1] * y[c - 1] - y[a - 1 + m] * y[c - 1 + m]


def test_row_norms_window_sum_and_trace():
    y = _int_series(31, 80).astype(float)
    p = 6
    rn, fro2 = oracle.row_norms(y, p)
    cs = np.concatenate([[0.0], np.cumsum(y * y)])
    assert rn.tolist() == [cs[i + p] - cs[i] for i in range(len(y) - p)]
    G, _ = oracle.gram(y, p)
    assert fro2 == pytest.approx(np.trace(G), rel=1e-15)


def test_leverage_p1_hand_written():
    g = _golden("leverage_p1_n4.json")
    lev = oracle.leverage_p1(np.array(g["y"], float))
    assert np.allclose(lev, np.array(g["lev_num"], float) / g["lev_den"], rtol=1e-15)
    # same thing from the general definition with p = 1
    assert np.allclose(oracle.exact_leverage(np.array(g["y"], float), 1), lev, rtol=1e-14)


def test_exact_leverage_properties():
    s = ar_series(400, 5, config_id=12)
    lev = oracle.exact_leverage(s.y, 5)
    assert lev.min() >= 0 and lev.max() <= 1
    assert lev.sum() == pytest.approx(5.0, rel=1e-12)
    X, _ = oracle.lag_matrix(s.y, 5)
    Q, _ = np.linalg.qr(X)
    assert np.allclose(lev, np.sum(Q * Q, axis=1), atol=1e-13)


@pytest.mark.parametrize("p", [2, 3, 6])
def test_leverage_step_with_exact_phi_gives_exact_leverage(p):
    # With phi_hat the exact OLS solution of the order-(p-1) problem, the update of eq. (FALS) is the exact
    # rank-one update of the hat-matrix diagonal, so it reproduces Def. "Leverage Score" for order p.
    s = ar_series(500, p, config_id=13)
    y = s.y
    prev = oracle.exact_leverage(y[:-1], p - 1)
    phi_hat = oracle.ols_qr(y[:-1], p - 1).phi
    lev, pi, _ = oracle.leverage_step(y, p, phi_hat, prev)
    assert np.allclose(lev, oracle.exact_leverage(y, p), atol=1e-12)
    assert pi.sum() == pytest.approx(1.0, rel=1e-12)


def test_generator_roots_stationary_and_coefficients():
    rng = rng_for(99, 0)
    inv = draw_inverse_roots(rng, 9, 1.2, 3.0)
    phi = coefficients_from_inverse_roots(inv)
    roots = np.roots(np.r_[1.0, -phi][::-1])
    assert np.min(np.abs(roots)) > 1.0
    # product form equals expanded polynomial at a few points
    for z in (0.3, -0.7 + 0.2j, 1.1j):
        assert abs(np.prod(1 - inv * z) - (1 - np.sum(phi * z ** np.arange(1, 10)))) < 1e-12


def test_generator_autocorrelation_matches_spectrum():
    s = ar_series(200_000, 3, config_id=14)
    y = s.y - 0.0
    n = y.size
    w = np.linspace(0, 2 * np.pi, 1 << 14, endpoint=False)
    z = np.exp(1j * w)
    S = 1.0 / np.abs(np.prod(1 - s.inv_roots[:, None] * z[None, :], axis=0)) ** 2
    acov = np.real(np.fft.ifft(S))
    rho_true = acov[:6] / acov[0]
    rho_hat = np.array([np.dot(y[: n - h], y[h:]) / np.dot(y, y) for h in range(6)])
    assert np.max(np.abs(rho_hat - rho_true)) < 3 / math.sqrt(n) * 3


def test_planted_mistakes_are_caught(monkeypatch):
    """Plant mistakes in the oracle (CPU only) and check the pins above notice them."""
    g = _golden("xphi_n5_p2.json")
    y = np.array(g["y"], float)
    real_lag = tols.lag_matrix

    def shifted(y_, p_, start=0, stop=None):          # off-by-one lag
        X, b = real_lag(y_, p_, start, stop)
        return np.roll(X, 1, axis=1), b

    monkeypatch.setattr(tols, "lag_matrix", shifted)
    X, _ = tols.lag_matrix(y, 2)
    assert X.tolist() != g["X"]
    yi = _int_series(1, 30)
    rows, rhs = _rows_from_definition(yi, 3)
    G, h = normal_equations_exact(rows, rhs)
    ref = np.array([float(v) for v in solve_spd_exact(G, h)])
    assert np.linalg.norm(tols.ols_qr(yi.astype(float), 3).phi - ref) > 1e-6
    monkeypatch.setattr(tols, "lag_matrix", real_lag)

    # transposed-product mistake: X^T u computed as a convolution instead of a correlation
    rng = np.random.default_rng(0)
    yy, v = rng.standard_normal(50), rng.standard_normal(45)
    wrong = np.convolve(yy[:-1], v, mode="valid")
    assert not np.allclose(wrong, oracle.rmatvec(yy, 5, v))


def test_pacf_pins():
    # lag 1 is the p = 1 closed form (in rationals); a noise-free AR(2) recursion with dyadic coefficients is fitted
    # exactly at lag 2, so tau_2 = phi_2
    from fractions import Fraction
    rng = np.random.default_rng(3)
    y = rng.standard_normal(400)
    tau, _ = oracle.pacf(y, 3)
    num = sum(Fraction(a) * Fraction(b) for a, b in zip(y[:-1], y[1:]))
    den = sum(Fraction(a) * Fraction(a) for a in y[:-1])
    assert tau[0] == pytest.approx(float(num / den), rel=1e-13)
    z = np.zeros(60)
    z[0], z[1] = 1.0, 0.5
    for t in range(2, z.size):
        z[t] = 0.75 * z[t - 1] - 0.25 * z[t - 2]
    tau2, _ = oracle.pacf(z, 2)
    assert tau2[1] == pytest.approx(-0.25, abs=1e-12)


# ---- Algorithm "LSAR" (Section 3.1) -------------------------------------------------------------------------
def test_leverage_sample_pins():
    # a linear scan over the running sum (brute force) on tiny inputs, with zero-score rows that can never be drawn
    rng = np.random.default_rng(11)
    lev = np.array([0.0, 0.5, 0.0, 1.25, 0.25, 0.0, 2.0])
    u = np.concatenate([[0.0, 0.999999], rng.random(500)])
    got = oracle.leverage_sample(lev, u)
    total = sum(lev)
    for uk, g in zip(u, got):
        run, want = 0.0, len(lev) - 1
        for i, v in enumerate(lev):
            run += v
            if run > uk * total:
                want = i
                break
        assert g == want
    assert not np.isin(got, [0, 2, 5]).any()
    # frequencies follow lev / sum(lev) (4 sigma over 200,000 draws)
    u = rng.random(200_000)
    counts = np.bincount(oracle.leverage_sample(lev, u), minlength=lev.size)
    prob = lev / total
    assert np.all(np.abs(counts - u.size * prob) <= 4 * np.sqrt(u.size * prob * (1 - prob)) + 1e-9)


def test_compressed_ols_pins():
    # hand-written rows of eq. (xphi) (golden n = 5, p = 2): rows 0 and 2 with equal pi give the plain LS fit of
    # those two rows, here an exactly determined 2x2 system
    g = _golden("xphi_n5_p2.json")
    y = np.array(g["y"], dtype=np.float64)
    X = np.array(g["X"], dtype=np.float64)[[0, 2]]
    b = np.array(g["b"], dtype=np.float64)[[0, 2]]
    phi = oracle.compressed_ols(y, 2, [0, 2], [0.5, 0.5], 2)
    assert phi == pytest.approx(np.linalg.solve(X, b), abs=1e-12)
    # the 1 / sqrt(c pi) rescale: row i drawn k_i times with pi_i = k_i / c makes S^T S = I, so the compressed
    # problem is the full one and its minimiser is the exact OLS fit (the QR oracle)
    s = ar_series(300, 3, config_id=5)
    m = s.y.size - 3
    k = np.random.default_rng(2).integers(1, 5, size=m)
    rows = np.repeat(np.arange(m), k)
    c = int(k.sum())
    phi = oracle.compressed_ols(s.y, 3, rows, k[rows] / c, c)
    assert phi == pytest.approx(oracle.ols_qr(s.y, 3).phi, rel=1e-10, abs=1e-12)
    # without the rescale the same rows give a different fit (the pin above depends on it)
    phi_unscaled = oracle.compressed_ols(s.y, 3, rows, np.full(rows.size, 1.0 / c), c)
    assert np.max(np.abs(phi_unscaled - phi)) > 1e-6


def test_lsar_pins():
    from synthetic import lsar_uniforms
    s = ar_series(20_000, 3, config_id=7, series_index=2, root_lo=1.1, root_hi=1.6)
    p_bar, c = 10, 2000
    u = lsar_uniforms(p_bar, c, config_id=7, series_index=2)
    r = oracle.lsar(s.y, p_bar, c, u)
    m = s.y.size - p_bar
    # eq. (FALS) adds r^2 / ||r||^2 (sum 1) per lag to the exact p = 1 scores (sum 1): the scores sum to p
    assert r.lev_sum == pytest.approx(np.arange(1, p_bar + 1), rel=1e-12)
    # lag 1 in closed form: with pi_i = y_i^2 / sum y^2 every weighted row has w^2 x^2 = sum y^2 / c, so
    # phi_1 = mean over the draws of y[i + 1] / y[i]
    rows = r.rows[0]
    assert r.tau[0] == pytest.approx(np.mean(s.y[rows + 1] / s.y[rows]), rel=1e-11)
    assert np.all((r.rows >= 0) & (r.rows < m))
    # the compressed fits track the exact PACF (oracle.pacf on the same series) within a few 1/sqrt(c)
    tau_exact, _ = oracle.pacf(s.y, p_bar)
    assert np.max(np.abs(r.tau - tau_exact)) <= 3.0 / math.sqrt(c)
    # the true order's coefficient is far above the threshold 1.96 / sqrt(c)
    assert abs(r.tau[2]) > 5 * 1.96 / math.sqrt(c) and r.order >= 3


def test_lsar_planted_mistakes_are_caught(monkeypatch):
    """Plant mistakes in the LSAR oracle (CPU only) and check the pins of test_lsar_pins notice them."""
    from synthetic import lsar_uniforms
    s = ar_series(5000, 2, config_id=7, series_index=3, root_lo=1.1, root_hi=1.6)
    u = lsar_uniforms(4, 500, config_id=7, series_index=3)
    real_ols, real_step = tols.compressed_ols, tols.leverage_step

    def shifted_ols(y, p, rows, pi_rows, c):           # sampled responses one row late
        phi_ = real_ols(y[1:], p, rows, pi_rows, c)
        return phi_

    monkeypatch.setattr(tols, "compressed_ols", shifted_ols)
    r = tols.lsar(s.y, 4, 500, u)
    assert abs(r.tau[0] - np.mean(s.y[r.rows[0] + 1] / s.y[r.rows[0]])) > 1e-6
    monkeypatch.setattr(tols, "compressed_ols", real_ols)

    def unnormalised_step(y, p, phi_hat, lev_prev):   # r^2 added without dividing by ||r||^2
        lev, pi, rr = real_step(y, p, phi_hat, lev_prev)
        return lev + (lev - lev_prev) * (rr - 1.0), pi, rr

    monkeypatch.setattr(tols, "leverage_step", unnormalised_step)
    r = tols.lsar(s.y, 4, 500, u)
    assert not np.allclose(r.lev_sum, np.arange(1, 5), rtol=1e-6)


def test_outlier_workload_generator():
    # Section 4.2: `count` distinct points replaced by y + U[-3, 3] + N(0, 100)
    from synthetic import with_outliers
    y = ar_series(20_000, 3, config_id=7).y
    z = with_outliers(y, 1000, config_id=7)
    assert np.array_equal(z, with_outliers(y, 1000, config_id=7))
    d = z - y
    changed = np.flatnonzero(d)
    assert changed.size == 1000
    dv = d[changed]
    assert abs(dv.mean()) < 4 * math.sqrt(103.0 / 1000)            # variance 100 + 36/12
    assert abs(dv.var() - 103.0) < 4 * 103.0 * math.sqrt(2.0 / 1000)
    assert np.all(z[np.setdiff1d(np.arange(y.size), changed)] == y[np.setdiff1d(np.arange(y.size), changed)])


# ---- Algorithm "SRHT" (Section 2.1) and Algorithm "Repeated Halving" (Section 3.2) --------------------------
@pytest.mark.parametrize("n", [1, 2, 8, 64, 1024])
def test_hadamard_transform_pins(n):
    # the normalised Sylvester matrix (scipy.linalg.hadamard / sqrt(n)); orthogonal and symmetric, so H H = I
    v = np.random.default_rng(n).standard_normal(n)
    Hv = oracle.hadamard_transform(v)
    assert np.allclose(Hv, scipy.linalg.hadamard(n) @ v / math.sqrt(n), rtol=0, atol=1e-13 * max(1.0, math.sqrt(n)))
    assert np.linalg.norm(Hv) == pytest.approx(np.linalg.norm(v), rel=1e-14)
    assert np.allclose(oracle.hadamard_transform(Hv), v, rtol=0, atol=1e-13)


def test_srht_pins():
    from synthetic import srht_draws
    s = ar_series(3000, 3, config_id=5)
    m, m2 = 3000 - 3, 4096
    exact = oracle.ols_qr(s.y, 3)
    # S takes every padded row once (c = m2, scale 1): S H D is orthogonal, so the fit is the exact OLS fit
    signs, _ = srht_draws(m, 1, config_id=5)
    perm = np.random.default_rng(0).permutation(m2)
    assert oracle.srht_ols(s.y, 3, perm, signs) == pytest.approx(exact.phi, rel=1e-11, abs=1e-13)
    # c = 300 uniform draws: the residual is within a few percent of the optimum (Theorem "Number of Rows to
    # Sample in SRHT Algorithm": (1 + eps) with probability >= 0.8)
    signs, rows = srht_draws(m, 300, config_id=5)
    phi = oracle.srht_ols(s.y, 3, rows, signs)
    rn = oracle.residual_check(s.y, 3, phi)[0]
    assert exact.rnorm <= rn <= 1.1 * exact.rnorm


def test_generalized_leverage_pins():
    rng = np.random.default_rng(4)
    C = rng.standard_normal((400, 5)) * np.array([1.0, 3.0, 0.2, 1.0, 5.0])
    Q, _ = np.linalg.qr(C)
    hat = np.sum(Q * Q, axis=1)                            # leverage scores: squared row norms of an orthonormal basis
    assert oracle.generalized_leverage(C, C) == pytest.approx(hat, rel=1e-10)
    B = C[rng.choice(400, 200, replace=False)]
    exact_B = oracle.generalized_leverage(C, B)
    assert oracle.generalized_leverage(C, B, np.eye(200)) == pytest.approx(exact_B, rel=1e-10)
    # Theorem "Leverage Score Approximation via Uniform Sampling": every generalised score w.r.t. an unscaled
    # row subset is at least the true score, and their total is about n d / m = 10
    assert np.all(exact_B >= hat * (1 - 1e-12))
    assert exact_B.sum() <= 2 * 400 * 5 / 200
    # the Gaussian sketch of eq. (glev) is unbiased: the mean over 400 sketches (N(0, 1/k) entries) is close
    k = 16
    est = np.mean([oracle.generalized_leverage(C, B, rng.standard_normal((k, 200)) / math.sqrt(k))
                   for _ in range(400)], axis=0)
    assert np.max(np.abs(est / exact_B - 1)) < 0.15


def test_repeated_halving_pins():
    from synthetic import rh_draws
    y = ar_series(20_000, 3, config_id=6).y
    X, b = oracle.lag_matrix(y, 8)
    C = np.column_stack([X, b])
    c = 400
    keep, gauss, unif = rh_draws(C.shape[0], c, 16, c, config_id=6)
    rh = oracle.repeated_halving(C, c, c, keep, gauss, unif)
    assert rh.sizes[0] == C.shape[0] and rh.sizes[-1] <= c < rh.sizes[-2]
    assert all(b_ == a_ // 2 for a_, b_ in zip(rh.sizes, rh.sizes[1:]))
    assert np.all(rh.scores > 0)
    prob = rh.scores[rh.rows] / math.fsum(rh.scores.tolist())
    assert np.allclose(rh.Xt, C[rh.rows] / np.sqrt(c * prob)[:, None], rtol=1e-14, atol=0)
    # a spectral approximation (Def. "lambda-Spectral Approximation"): x^T Xt^T Xt x / x^T C^T C x stays within a
    # small factor for every x
    Lc = np.linalg.cholesky(C.T @ C)
    M = np.linalg.solve(Lc, np.linalg.solve(Lc, rh.Xt.T @ rh.Xt).T)
    w = np.linalg.eigvalsh((M + M.T) / 2)
    assert 0.5 <= w.min() and w.max() <= 2.0
    # the scores track the true leverage of C (normalised) within a small factor for almost every row
    Q, _ = np.linalg.qr(C)
    ex = np.sum(Q * Q, axis=1)
    ratio = (rh.scores / rh.scores.sum()) / (ex / ex.sum())
    assert np.percentile(ratio, 1) > 0.25 and np.percentile(ratio, 99) < 4.0


def test_rh_lsar_pins():
    from synthetic import lsar_uniforms, rh_draws
    s = ar_series(20_000, 3, config_id=7, series_index=2, root_lo=1.1, root_hi=1.6)
    p_bar, c = 10, 2000
    X, b = oracle.lag_matrix(s.y, p_bar)
    C = np.column_stack([X, b])
    keep, gauss, unif = rh_draws(C.shape[0], c, 16, c, config_id=7)
    rh = oracle.repeated_halving(C, c, c, keep, gauss, unif)
    r = oracle.rh_lsar(s.y, p_bar, c, rh, lsar_uniforms(p_bar, c, config_id=7, series_index=2))
    tau_exact, _ = oracle.pacf(s.y, p_bar)
    assert np.max(np.abs(r.tau - tau_exact)) <= 3.0 / math.sqrt(c)
    assert abs(r.tau[2]) > 5 * 1.96 / math.sqrt(c) and r.order >= 3
    assert np.all((r.rows >= 0) & (r.rows < C.shape[0]))


def test_sketch_planted_mistakes_are_caught(monkeypatch):
    """Plant mistakes in the SRHT / Repeated Halving oracle (CPU only) and check the pins above notice them."""
    v = np.random.default_rng(1).standard_normal(64)
    real_h = tols.hadamard_transform

    def unnormalised(x):                                  # the 1/sqrt(2) of each stage dropped
        return real_h(x) * math.sqrt(len(x))

    monkeypatch.setattr(tols, "hadamard_transform", unnormalised)
    assert not np.isclose(np.linalg.norm(tols.hadamard_transform(v)), np.linalg.norm(v))
    monkeypatch.setattr(tols, "hadamard_transform", real_h)
    # generalised scores with B^T B in place of its inverse
    rng = np.random.default_rng(4)
    C = rng.standard_normal((100, 4))
    Q, _ = np.linalg.qr(C)
    wrong = np.einsum("ij,jk,ik->i", C, C.T @ C, C)
    assert not np.allclose(wrong, np.sum(Q * Q, axis=1))


def _rh_upsweep_expected():
    """Level-0 scores of Algorithm "Repeated Halving" (Section 3.2) on a hand-built 8 x 2 matrix, written out
    with explicit 2 x 2 Gram matrices (no oracle call). Halving keeps rows 0, 2, 5, 7 (level 1) and then level
    1's rows 1, 2 (level 2, the deepest: its own approximation, unscaled). Sketches are identities, so eq. (glev)
    gives the exact generalised scores x^T (B^T B)^{-1} x of Def. "Generalised Leverage Score"."""
    C = np.array([[1, 0], [0, 1], [1, 1], [2, -1], [1, 3], [-1, 2], [3, 1], [0, 2]], dtype=np.float64)
    lvl1 = C[[0, 2, 5, 7]]
    lvl2 = lvl1[[1, 2]]
    G2 = sum(np.outer(r, r) for r in lvl2)                  # [[2, -1], [-1, 5]], det 9
    s1 = np.array([r @ np.linalg.inv(G2) @ r for r in lvl1])
    assert np.allclose(s1 * 9, [5, 9, 9, 8])
    # three draws from level 1 by inverse CDF at u = 0.1, 0.5, 0.9 of the running sums 5, 14, 23, 31 (/ 9)
    picks = [0, 2, 3]
    pi = s1[picks] / s1.sum()                              # 5/31, 9/31, 8/31
    G1 = sum(np.outer(lvl1[k], lvl1[k]) / (3 * q) for k, q in zip(picks, pi))
    s0 = np.array([r @ np.linalg.inv(G1) @ r for r in C])
    return C, G1, s0


def test_repeated_halving_upsweep_pinned():
    """Level j is scored against the rescaled sample of level j+1 (its spectral approximation), not against the
    raw level j+1."""
    C, G1, s0 = _rh_upsweep_expected()
    keep = [np.array([0, 2, 5, 7]), np.array([1, 2])]
    gauss = [np.eye(3), np.eye(2)]
    unif = [np.array([0.3, 0.6, 0.95]), np.array([0.1, 0.5, 0.9])]
    rh = oracle.repeated_halving(C, 3, 2, keep, gauss, unif)
    assert rh.sizes == [8, 4, 2]
    assert np.allclose(rh.scores, s0, rtol=1e-13, atol=0)
    # scored against the raw level 1 instead, the scores differ by far more than rounding
    G_raw = C[[0, 2, 5, 7]].T @ C[[0, 2, 5, 7]]
    s_raw = np.array([r @ np.linalg.inv(G_raw) @ r for r in C])
    assert np.max(np.abs(s_raw - s0) / s0) > 0.1


def test_repeated_halving_raw_level_mistake_is_caught(monkeypatch):
    """Plant the raw-level mistake in the oracle (CPU only): the approximation step returns level j+1 itself."""
    C, _, s0 = _rh_upsweep_expected()

    def raw_level(A, scores, u, c):
        A = np.asarray(A, dtype=np.float64)
        return np.arange(A.shape[0]), A

    monkeypatch.setattr(tols, "spectral_approximation", raw_level)
    rh = oracle.repeated_halving(C, 3, 2, [np.array([0, 2, 5, 7]), np.array([1, 2])], [np.eye(4), np.eye(2)],
                                 [np.array([0.3, 0.6, 0.95]), np.array([0.1, 0.5, 0.9])])
    assert not np.allclose(rh.scores, s0, rtol=1e-6, atol=0)
