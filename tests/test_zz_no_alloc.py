"""The allocation-free fused pass against the context-based one, on two calls in a row.

toeplitz_ols_gk_pass_noalloc serves callers that cannot let the library allocate device memory (their memory
belongs to another allocator or a fixed pool, or their loop cannot afford cudaMalloc/cudaFree, which may
synchronise the device): it needs no context and keeps its cross-CTA partial sums in a fixed array inside the
library. Here it must reproduce toeplitz_ols_gk_pass on the same inputs: u_new exactly (each row is formed by the
same code), X^T u_new and ||u_new||^2 within the summation-order tolerances of tests/test_gpu_steps.py, and again
on a second call, which finds the first call's leftovers in the shared array.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p,n", [(1, 3 * 4096 + 777 + 1), (100, 3 * 4096 + 100 + 5), (256, 20_000)])
def test_noalloc_pass_matches_context_pass(prec, p, n):
    import torch

    import paper_2112_12994_gb300 as t
    from synthetic import ar_series

    rng = np.random.default_rng(p + n)
    y = ar_series(n, 3, config_id=70, series_index=p).y
    m = n - p
    dt = torch.float64 if prec == "fp64" else torch.float32
    P = t.TOLS_FP64 if prec == "fp64" else t.TOLS_MIXED
    d_y = torch.tensor(y, dtype=dt, device="cuda")
    d_v = torch.tensor(rng.standard_normal(p), dtype=torch.float64, device="cuda")
    d_uo = torch.tensor(rng.standard_normal(m), dtype=dt, device="cuda")
    c = 0.731

    # the existing entry point (context, arena) gives the reference, pinned to the same direct-product kernel
    ref_u = torch.empty(m, dtype=dt, device="cuda")
    ref_t = torch.empty(p, dtype=torch.float64, device="cuda")
    with t.Context(product=t.TOLS_PRODUCT_DIRECT) as ctx:
        ref_n2 = t.toeplitz_ols_gk_pass(ctx, P, d_y, n, p, d_v, d_uo, c, ref_u, ref_t)
    ref_u_h = ref_u.cpu().numpy().astype(np.float64)
    ref_t_h = ref_t.cpu().numpy()

    # tolerance on X^T u from the arithmetic: float64 sums within (m + p) u, float32 within 512 u32
    X, _ = oracle.lag_matrix(d_y.cpu().numpy().astype(np.float64), p)
    scale_t = np.abs(X.T) @ np.abs(ref_u_h)
    k = (m + p) * U64 if prec == "fp64" else 512 * U32

    stream = torch.cuda.current_stream()
    for call in range(2):
        out_u = torch.full((m,), float("nan"), dtype=dt, device="cuda")
        out_t = torch.full((p,), float("nan"), dtype=torch.float64, device="cuda")
        out_n2 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = t.toeplitz_ols_gk_pass_noalloc(P, d_y, n, p, d_v, d_uo, c, out_u, out_t, out_n2, stream.cuda_stream)
        assert rc == t.TOLS_OK, (call, rc)
        torch.cuda.synchronize()
        u = out_u.cpu().numpy().astype(np.float64)
        assert np.array_equal(u, ref_u_h), call
        assert np.all(np.abs(out_t.cpu().numpy() - ref_t_h) <= 2 * k * scale_t), call
        assert out_n2.item() == pytest.approx(ref_n2, rel=2 * k), call


def test_noalloc_rejects_orders_beyond_its_array():
    import torch

    import paper_2112_12994_gb300 as t

    p = t.TOLS_NOALLOC_MAX_P + 1
    n = 4 * p
    d_y = torch.zeros(n, dtype=torch.float64, device="cuda")
    d_v = torch.zeros(p, dtype=torch.float64, device="cuda")
    d_t = torch.zeros(p, dtype=torch.float64, device="cuda")
    d_n2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = t.toeplitz_ols_gk_pass_noalloc(t.TOLS_FP64, d_y, n, p, d_v, None, 0.0, None, d_t, d_n2, None)
    assert rc == t.TOLS_ERR_ARG


def test_noalloc_second_stream_ordered_by_event():
    """Calls on two streams share the one array; ordered by an event (the documented way to serialise them),
    the second call on another stream gives the first call's outputs bit for bit."""
    import torch

    import paper_2112_12994_gb300 as t
    from synthetic import ar_series

    p, n = 64, 5 * 4096 + 123
    m = n - p
    y = ar_series(n, 3, config_id=71).y
    rng = np.random.default_rng(7)
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_v = torch.tensor(rng.standard_normal(p), dtype=torch.float64, device="cuda")
    d_uo = torch.tensor(rng.standard_normal(m), dtype=torch.float64, device="cuda")
    s1 = torch.cuda.Stream()
    s2 = torch.cuda.Stream()
    outs = []
    done = torch.cuda.Event()
    for k, s in enumerate((s1, s2)):
        out_u = torch.empty(m, dtype=torch.float64, device="cuda")
        out_t = torch.empty(p, dtype=torch.float64, device="cuda")
        out_n2 = torch.empty(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()            # the outputs exist before either stream touches them
        if k == 1:
            s.wait_event(done)              # the second call waits for the first one's kernel
        rc = t.toeplitz_ols_gk_pass_noalloc(t.TOLS_FP64, d_y, n, p, d_v, d_uo, 0.25, out_u, out_t, out_n2,
                                            s.cuda_stream)
        assert rc == t.TOLS_OK
        if k == 0:
            done.record(s)
        outs.append((out_u, out_t, out_n2))
    torch.cuda.synchronize()
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
