"""GPU parity of each hot-path step, element by element against the CPU oracle (through the C ABI).

Tolerances come from the arithmetic: a float64 sum of N terms is within N u sum|terms| of the exact sum
(u = 2^-53); the float32 kernels sum at most ~300 products per partial in float32 before the partials are
combined in float64, so 512 u32 sum|terms| bounds them (u32 = 2^-24). Sizes span several CTA tiles (2,048
rows in float64, 4,096 in float32) and end in a ragged tile.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    return _t


@pytest.fixture(scope="module")
def tols():
    import paper_2112_12994_gb300 as t
    return t


@pytest.fixture(scope="module")
def ctx(tols):
    # the direct (sliding-window) kernels; the FFT kernels are covered in test_gpu_fft.py
    c = tols.Context(precision=tols.TOLS_FP64, product=tols.TOLS_PRODUCT_DIRECT)
    yield c
    c.close()


def _series(seed, n):
    from synthetic import ar_series
    return ar_series(n, 3, config_id=50, series_index=seed).y


CASES = [(1, 3 * 4096 + 777 + 1), (5, 9000), (16, 12_345), (17, 4096 + 17), (100, 3 * 4096 + 100 + 5),
         (257, 20_000), (1024, 9_000)]


@pytest.mark.parametrize("p,n", CASES)
@pytest.mark.parametrize("with_old", [False, True])
def test_gk_pass_fp64(torch, tols, ctx, p, n, with_old):
    rng = np.random.default_rng(p * 7 + n)
    y = _series(p, n)
    m = n - p
    v = rng.standard_normal(p)
    u_old = rng.standard_normal(m) if with_old else None
    c = 0.731
    X, _ = oracle.lag_matrix(y, p)
    ref_u = X @ v - (c * u_old if with_old else 0.0)
    ref_t = X.T @ ref_u
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    d_y, d_v = dev(y), dev(v)
    d_uo = dev(u_old) if with_old else None
    d_un = torch.empty(m, dtype=torch.float64, device="cuda")
    d_t = torch.empty(p, dtype=torch.float64, device="cuda")
    n2 = tols.toeplitz_ols_gk_pass(ctx, tols.TOLS_FP64, d_y, n, p, d_v, d_uo, c, d_un, d_t)
    u = d_un.cpu().numpy()
    t = d_t.cpu().numpy()
    scale_u = np.abs(X) @ np.abs(v) + (abs(c) * np.abs(u_old) if with_old else 0.0)
    assert np.all(np.abs(u - ref_u) <= (p + 2) * U64 * scale_u + 1e-300)
    scale_t = np.abs(X.T) @ np.abs(ref_u)
    bound_t = (m + p) * U64 * scale_t + np.abs(X.T) @ ((p + 2) * U64 * scale_u)
    assert np.all(np.abs(t - ref_t) <= bound_t)
    assert n2 == pytest.approx(float(ref_u @ ref_u), rel=(m + 2 * p + 4) * U64 * 4)


@pytest.mark.parametrize("p,n", CASES)
def test_gk_pass_fp32(torch, tols, ctx, p, n):
    rng = np.random.default_rng(p * 11 + n)
    y = _series(p, n)
    m = n - p
    # the float32 kernel sees float32 inputs: the reference uses the same rounded values in float64
    y32 = y.astype(np.float32)
    v = rng.standard_normal(p)
    v32 = v.astype(np.float32).astype(np.float64)
    u_old = rng.standard_normal(m).astype(np.float32)
    c = 0.731
    c32 = float(np.float32(c))
    X, _ = oracle.lag_matrix(y32.astype(np.float64), p)
    ref_u = X @ v32 - c32 * u_old.astype(np.float64)
    d_y = torch.tensor(y32, device="cuda")
    d_v = torch.tensor(v, dtype=torch.float64, device="cuda")
    d_uo = torch.tensor(u_old, device="cuda")
    d_un = torch.empty(m, dtype=torch.float32, device="cuda")
    d_t = torch.empty(p, dtype=torch.float64, device="cuda")
    n2 = tols.toeplitz_ols_gk_pass(ctx, tols.TOLS_MIXED, d_y, n, p, d_v, d_uo, c, d_un, d_t)
    u = d_un.cpu().numpy().astype(np.float64)
    t = d_t.cpu().numpy()
    scale_u = np.abs(X) @ np.abs(v32) + abs(c32) * np.abs(u_old)
    assert np.all(np.abs(u - ref_u) <= (p + 3) * U32 * scale_u)
    # X^T is applied to the float32 u the kernel produced
    ref_t = X.T @ u
    scale_t = np.abs(X.T) @ np.abs(u)
    assert np.all(np.abs(t - ref_t) <= 512 * U32 * scale_t)
    assert n2 == pytest.approx(float(u @ u), rel=64 * U32)


@pytest.mark.parametrize("p,n", [(1, 5000), (10, 10_000), (100, 3 * 2048 + 333), (300, 7000), (1024, 6000)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gram(torch, tols, ctx, p, n, prec):
    y = _series(p + 1, n)
    G_ref, h_ref = oracle.gram(y, p)
    X, b = oracle.lag_matrix(y, p)
    Xa = np.abs(X)
    sG = Xa.T @ Xa
    sh = Xa.T @ np.abs(b)
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_G = torch.empty(p * p, dtype=torch.float64, device="cuda")
    d_h = torch.empty(p, dtype=torch.float64, device="cuda")
    P = tols.TOLS_FP64 if prec == "fp64" else tols.TOLS_MIXED
    b2 = tols.toeplitz_ols_gram(ctx, P, d_y, n, p, d_G, d_h)
    G = d_G.cpu().numpy().reshape(p, p)
    h = d_h.cpu().numpy()
    k = (n + 3 * p) * U64 if prec == "fp64" else 600 * U32
    assert np.all(np.abs(G - G_ref) <= k * sG)
    assert np.all(np.abs(h - h_ref) <= k * sh)
    assert b2 == pytest.approx(float(b @ b), rel=k)


@pytest.mark.parametrize("p,n", [(1, 5001), (7, 2048 * 3 + 7 + 1), (64, 10_000), (1024, 4000)])
def test_row_norms(torch, tols, ctx, p, n):
    y = _series(p + 2, n)
    rn_ref, fro_ref = oracle.row_norms(y, p)
    m = n - p
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_rn = torch.empty(m, dtype=torch.float64, device="cuda")
    fro = tols.toeplitz_ols_row_norms(ctx, d_y, n, p, d_rn)
    rn = d_rn.cpu().numpy()
    # tile-local float64 prefix sums: error within (2048 + p) u times the tile window's sum of squares
    win = (2048 + p) * U64 * np.sum(y * y)
    assert np.all(np.abs(rn - rn_ref) <= win)
    assert fro == pytest.approx(fro_ref, rel=(n + 2048) * U64 * 4)


@pytest.mark.parametrize("p,n", [(1, 3000), (12, 2048 * 2 + 12 + 99), (200, 9000)])
def test_residual_pass(torch, tols, ctx, p, n):
    y = _series(p + 3, n)
    sol = oracle.ols_qr(y, p)
    phi = sol.phi + 1e-3 * np.random.default_rng(p).standard_normal(p)
    X, b = oracle.lag_matrix(y, p)
    r = b - X @ phi
    g_ref = X.T @ r
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_phi = torch.tensor(phi, dtype=torch.float64, device="cuda")
    d_g = torch.empty(p, dtype=torch.float64, device="cuda")
    rn = tols.toeplitz_ols_residual(ctx, d_y, n, p, d_phi, d_g)
    g = d_g.cpu().numpy()
    Xa = np.abs(X)
    sr = np.abs(b) + Xa @ np.abs(phi)
    bound = (n + p) * U64 * (Xa.T @ np.abs(r)) + (p + 2) * U64 * (Xa.T @ sr)
    assert np.all(np.abs(g - g_ref) <= bound)
    assert rn == pytest.approx(float(np.linalg.norm(r)), rel=(n + p) * U64 * 4 + (p + 2) * U64 * np.max(sr / np.maximum(np.abs(r), 1e-300)))


@pytest.mark.parametrize("n", [2, 3, 5000, 4096 * 3 + 1])
def test_leverage_p1(torch, tols, ctx, n):
    y = _series(1, n)
    ref = oracle.leverage_p1(y)
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_l = torch.empty(n - 1, dtype=torch.float64, device="cuda")
    tols.toeplitz_ols_leverage_p1(ctx, d_y, n, d_l)
    assert np.allclose(d_l.cpu().numpy(), ref, rtol=(n + 8) * U64 * 4, atol=0)


@pytest.mark.parametrize("p,n", [(2, 3000), (3, 2048 * 2 + 3 + 17), (40, 12_000)])
def test_leverage_step(torch, tols, ctx, p, n):
    y = _series(p + 5, n)
    m = n - p
    prev = oracle.exact_leverage(y[:-1], p - 1) if m <= 3000 else np.full(m, (p - 1) / m)
    phi_hat = oracle.ols_qr(y[:-1], p - 1).phi * (1 + 1e-3)   # an approximate (sampled-style) solution
    lev_ref, pi_ref, s_ref = oracle.leverage_step(y, p, phi_hat, prev)
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    d_y, d_phi, d_prev = d(y), d(phi_hat), d(prev)
    d_lev = torch.empty(m, dtype=torch.float64, device="cuda")
    d_pi = torch.empty(m, dtype=torch.float64, device="cuda")
    s = tols.toeplitz_ols_leverage_step(ctx, d_y, n, p, d_phi, d_prev, d_lev, d_pi)
    Xp, bp = oracle.lag_matrix(y[:-1], p - 1)
    r = Xp @ phi_hat - bp
    er = (p + 2) * U64 * (np.abs(Xp) @ np.abs(phi_hat) + np.abs(bp))
    tol = (2 * np.abs(r) * er + r * r * (m + 8) * U64 * 4) / s_ref + 4 * U64 * lev_ref
    assert np.all(np.abs(d_lev.cpu().numpy() - lev_ref) <= tol)
    assert np.all(np.abs(d_pi.cpu().numpy() - pi_ref) <= tol / p + 4 * U64 * pi_ref)
    assert s == pytest.approx(s_ref, rel=(m + p) * U64 * 8)
