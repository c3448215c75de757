"""Shared test helpers: the parity gate of a solve against the oracle."""
import numpy as np

import oracle


def coef_rel_err(phi, ref):
    return float(np.linalg.norm(np.asarray(phi) - ref) / max(np.linalg.norm(ref), 1e-300))


def assert_solve_parity(y, p, phi_gpu, sol, coef_tol, backward_tol=1e-12):
    """Gate of a GPU solve against the oracle.

    Coefficients must match to coef_tol where the oracle's own forward-error bound
    10 u (kappa + kappa^2 eta) is at most coef_tol / 10; otherwise (the oracle itself is not that accurate)
    the backward metrics are graded: relative residual-norm difference and the normal-equation ratio of the
    GPU phi, both recomputed by the oracle in float64.
    """
    rn, _, ne = oracle.residual_check(y, p, phi_gpu, norm2=sol.norm2)
    B = sol.forward_error_bound()
    rel = coef_rel_err(phi_gpu, sol.phi)
    if B <= coef_tol / 10:
        assert rel <= coef_tol, f"coef rel err {rel:.3e} > {coef_tol:.1e} (bound {B:.1e})"
    assert abs(rn - sol.rnorm) <= backward_tol * max(sol.rnorm, 1e-300) + 1e-14 * np.linalg.norm(y), \
        f"rnorm {rn!r} vs {sol.rnorm!r}"
    assert ne <= max(backward_tol, 10 * sol.ne_ratio), f"ne ratio {ne:.3e}"
    return rel, ne, B
