"""The overlap-save FFT product pass against the oracle (forced with TOLS_PRODUCT_FFT, or TOLS_PRODUCT_FFT4096 for
float64 transforms of length 4,096), and FFT solves.

FFT correlations are accurate normwise: for one tile the error of IDFT(DFT(a) . conj(DFT(b))) is within
c u log2(N) ||a||_2 ||b||_2 (c a small constant; 8 is used), with ||window||_2 <= sqrt(N) max|y|. Tiles have
N = 4096 (float32) or 2048 (float64) points and m spans several of them with a ragged tail.
"""
import math

import numpy as np
import pytest

import oracle
from synthetic import ar_series
from tests.helpers import assert_solve_parity

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


@pytest.fixture(scope="module", params=[2048, 4096], ids=["N2048", "N4096"])
def fctx(tols, request):
    """A context forcing FFT products; .nfft64 is the float64 transform length (float: 4,096 either way)."""
    c = tols.Context(precision=tols.TOLS_FP64,
                     product=tols.TOLS_PRODUCT_FFT if request.param == 2048 else tols.TOLS_PRODUCT_FFT4096)
    c.nfft64 = request.param
    yield c
    c.close()


CASES = [(1, 9 * 2048 + 77), (17, 3 * 4096 + 5), (100, 5 * 4096 + 333), (257, 20_000), (500, 30_000)]


@pytest.mark.parametrize("p,n", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("offset", [0, 1])
def test_fft_gk_pass(torch, tols, fctx, p, n, prec, offset):
    """offset 1: u_old and u_new are views one element into larger buffers (not 16-byte aligned), which the
    float pass serves with its shared-memory kernel instead of the bulk-copy one."""
    rng = np.random.default_rng(p * 13 + n)
    y = ar_series(n, 3, config_id=51, series_index=p).y
    m = n - p
    dt = torch.float64 if prec == "fp64" else torch.float32
    P = tols.TOLS_FP64 if prec == "fp64" else tols.TOLS_MIXED
    u_eps, N = (U64, fctx.nfft64) if prec == "fp64" else (U32, 4096)
    yr = y if prec == "fp64" else y.astype(np.float32).astype(np.float64)
    v = rng.standard_normal(p)
    vr = v if prec == "fp64" else v.astype(np.float32).astype(np.float64)
    u_old = rng.standard_normal(m)
    uor = u_old if prec == "fp64" else u_old.astype(np.float32).astype(np.float64)
    c = 0.731
    cr = c if prec == "fp64" else float(np.float32(c))
    X, _ = oracle.lag_matrix(yr, p)
    ref_u = X @ vr - cr * uor
    d_y = torch.tensor(y, dtype=dt, device="cuda")
    d_v = torch.tensor(v, dtype=torch.float64, device="cuda")
    d_uo = torch.tensor(np.concatenate([np.zeros(offset), u_old]), dtype=dt, device="cuda")[offset:]
    d_un = torch.empty(m + offset, dtype=dt, device="cuda")[offset:]
    d_t = torch.empty(p, dtype=torch.float64, device="cuda")
    n2 = tols.toeplitz_ols_gk_pass(fctx, P, d_y, n, p, d_v, d_uo, c, d_un, d_t)
    u = d_un.cpu().numpy().astype(np.float64)
    t = d_t.cpu().numpy()
    k = 8 * u_eps * math.log2(N)
    win = math.sqrt(N) * np.max(np.abs(yr))
    bound_u = k * win * np.linalg.norm(vr) + 2 * u_eps * np.abs(cr * uor)
    assert np.all(np.abs(u - ref_u) <= bound_u)
    ref_t = X.T @ u
    tiles = math.ceil(m / (N - ((p + 15) // 16) * 16))
    bound_t = k * win * math.sqrt(tiles) * np.linalg.norm(u) + (m + p) * u_eps * (np.abs(X.T) @ np.abs(u))
    assert np.all(np.abs(t - ref_t) <= bound_t)
    assert n2 == pytest.approx(float(u @ u), rel=64 * u_eps)


@pytest.mark.parametrize("p,n", [(10, 10_000), (20, 1000), (50, 2100), (100, 3 * 2048 + 333), (300, 20_000)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fft_gram(torch, tols, fctx, p, n, prec):
    y = ar_series(n, 4, config_id=52, series_index=p).y
    G_ref, h_ref = oracle.gram(y, p)
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_G = torch.empty(p * p, dtype=torch.float64, device="cuda")
    d_h = torch.empty(p, dtype=torch.float64, device="cuda")
    P = tols.TOLS_FP64 if prec == "fp64" else tols.TOLS_MIXED
    tols.toeplitz_ols_gram(fctx, P, d_y, n, p, d_G, d_h)
    G = d_G.cpu().numpy().reshape(p, p)
    u_eps, N = (U64, fctx.nfft64) if prec == "fp64" else (U32, 4096)
    m = n - p
    tiles = math.ceil(m / (N - ((p + 1 + 15) // 16) * 16))
    win = math.sqrt(N) * np.max(np.abs(y))
    bound = 8 * u_eps * math.log2(N) * win * win * tiles + (4 if prec == "mixed" else 0) * U32 * np.sum(y * y)
    assert np.max(np.abs(G - G_ref)) <= bound


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,p", [(10_000, 10), (300_000, 100), (60_000, 400)])
@pytest.mark.parametrize("nfft", [2048, 4096])
def test_fft_solve_matches_oracle(tols, prec, n, p, nfft):
    s = ar_series(n, p, config_id=53, series_index=p, root_lo=2.0, root_hi=4.0, max_log10_bound=6.0)
    sol = oracle.ols_qr(s.y, p)
    P = tols.TOLS_FP64 if prec == "fp64" else tols.TOLS_MIXED
    prod = tols.TOLS_PRODUCT_FFT if nfft == 2048 else tols.TOLS_PRODUCT_FFT4096
    with tols.Context(precision=P, product=prod) as ctx:
        phi, rnorm, info, rc = tols.toeplitz_ols_solve(ctx, s.y, p, 1e-12)
    assert rc == tols.TOLS_OK, info
    assert info["product_used"] == prod and info["nfft"] == nfft, info
    assert_solve_parity(s.y, p, phi, sol, 1e-8 if prec == "fp64" else 1e-6)


def test_wait_limit_gives_up_with_device_timeout(torch, tols):
    """The float FFT pass waits on its own bulk copies with a bounded poll count. With wait_polls = -1 every such
    wait gives up at once: the call reports TOLS_ERR_DEVICE_TIMEOUT instead of waiting (the kernel still lets the
    copies it issued land before it exits). The same context then runs a float64 pass (no bulk copies) to the
    right result, and a context with the default limit runs the float FFT pass to the right result."""
    n, p = 200_000, 100
    y = ar_series(n, 3, config_id=55).y
    m = n - p
    rng = np.random.default_rng(5)
    v = rng.standard_normal(p)
    d_v = torch.tensor(v, dtype=torch.float64, device="cuda")
    d_t = torch.empty(p, dtype=torch.float64, device="cuda")
    d_y32 = torch.tensor(y, dtype=torch.float32, device="cuda")
    d_uo32 = torch.tensor(rng.standard_normal(m), dtype=torch.float32, device="cuda")
    d_un32 = torch.empty(m, dtype=torch.float32, device="cuda")
    d_y64 = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_un64 = torch.empty(m, dtype=torch.float64, device="cuda")
    with tols.Context(precision=tols.TOLS_MIXED, product=tols.TOLS_PRODUCT_FFT, wait_polls=-1) as c:
        with pytest.raises(tols.TolsError) as e:
            tols.toeplitz_ols_gk_pass(c, tols.TOLS_MIXED, d_y32, n, p, d_v, d_uo32, 0.5, d_un32, d_t)
        assert e.value.code == tols.TOLS_ERR_DEVICE_TIMEOUT
        tols.toeplitz_ols_gk_pass(c, tols.TOLS_FP64, d_y64, n, p, d_v, None, 0.0, d_un64, d_t)
        u = d_un64.cpu().numpy()
        t = d_t.cpu().numpy()
    X, _ = oracle.lag_matrix(y, p)
    assert np.max(np.abs(u - X @ v)) <= 1e-12 * np.linalg.norm(v) * math.sqrt(2048) * np.max(np.abs(y)) * 100
    assert np.allclose(t, X.T @ u, rtol=0, atol=1e-10 * np.linalg.norm(u) * np.linalg.norm(y))
    with tols.Context(precision=tols.TOLS_MIXED, product=tols.TOLS_PRODUCT_FFT) as c:
        tols.toeplitz_ols_gk_pass(c, tols.TOLS_MIXED, d_y32, n, p, d_v, d_uo32, 0.5, d_un32, d_t)
        t32 = d_t.cpu().numpy()
    yr = y.astype(np.float32).astype(np.float64)
    u32 = d_un32.cpu().numpy().astype(np.float64)
    ref_t = np.array([np.dot(u32, yr[p - 1 - j: p - 1 - j + m]) for j in range(p)])
    assert np.max(np.abs(t32 - ref_t)) <= 1e-5 * np.linalg.norm(u32) * np.linalg.norm(yr)
