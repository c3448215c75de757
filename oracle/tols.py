"""Oracle for the Toeplitz OLS (TOLS) problem of an AR(p) fit — TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg may import, call or run this
module. The CUDA library never does, and this module imports nothing from it: the two share no code.

Everything here is plain float64 NumPy/LAPACK on the CPU, written to be checked against the paper by eye.
Notation (0-based, series y[0..n-1], order p, m = n - p rows):

    X[i, j] = y[p + i - j - 1],   b[i] = y[p + i],   i in [0, m), j in [0, p)

which is eq. (xphi) of Section 3 (1-based there: row 1 is (y_p ... y_1), response y_{p+1}).

Functions and the passage each follows:
  lag_matrix          eq. (xphi), Section 3 (the data matrix X_{n-p,p} and response y_{n-p,1}).
  matvec / rmatvec    explicit products X v and X^T u with the matrix of eq. (xphi).
  ols_qr              Def. "Ordinary Least Squares Problem" and Thm. "Solution to OLS problem" (Section 2):
                      the minimiser of ||X phi - b||, unique when X^T X is nonsingular, else the minimum-norm
                      one through the SVD. Computed by Householder QR (LAPACK dgeqrf through numpy) of the
                      explicit [X | b]; for large m the rows are fed in blocks and each block is stacked under
                      the previous triangle, because QR([R; X_2]) has the same R as QR([X_1; X_2]).
  residual_check      the normal equation of Thm. "Solution to OLS problem": g = X^T (b - X phi) and the ratio
                      ||g|| / (||X||_2 ||r||), with ||.|| the spectral norm as in the Notation paragraph
                      (Section 1).
  gram                X^T X and X^T b written out from eq. (xphi).
  row_norms           ||X(i,:)||^2 and ||X||_F^2 (Section 1 notation: X(i,:) is the i-th row).
  exact_leverage      Def. "Leverage Score" (Section 2.1.2): l(i) = e_i^T X (X^T X)^{-1} X^T e_i.
  leverage_p1         the exact scores for p = 1 printed after eq. (FASD) (Section 3.1):
                      l_{n,1}(i) = y_i^2 / sum_{t=1}^{n-1} y_t^2.
  leverage_step       eqs. (FALS), (FAR), (FASD), Section 3.1: l_{n,p} = l_{n-1,p-1} + r^2/||r||^2 with
                      r = X_{n-1,p-1} phi_hat - y_{n-1,p-1}, and pi = l / p.
  leverage_sample     the sampling step of Algorithm "LSAR" (Section 3.1): c rows drawn with replacement from the
                      distribution pi of eq. (FASD), by inverse CDF on the given uniforms.
  compressed_ols      the compressed OLS problem of Algorithm "LSAR": min ||S X phi - S b|| with S picking the
                      sampled rows of eq. (xphi), each scaled by 1 / sqrt(c pi_i); its minimiser by LAPACK lstsq.
  lsar                Algorithm "LSAR" (Section 3.1): for lags p = 1 .. p_bar on the same m = n - p_bar rows,
                      approximate leverage scores (Def. "Approximate Leverage Scores"), sampling, compressed
                      solve, PACF estimate tau_p = last coefficient, and the order estimate: the largest p with
                      |tau_p| >= 1.96 / sqrt(c).
  hadamard_transform  Def. "Hadamard Transform" (Section 2.1): H_m v by its recursion, normalised.
  srht_ols            Algorithm "SRHT" (Section 2.1, eq. (SRHT)): min ||S H D (X phi - b)|| with D random signs,
                      H the normalised Hadamard transform (rows zero-padded to a power of two) and S uniform
                      sampling with replacement scaled by sqrt(n/c).
  generalized_leverage  Def. "Generalised Leverage Score" (Section 3.2) and its Gaussian-sketch approximation,
                      eq. (glev).
  spectral_approximation  the sampling step of Algorithm "Repeated Halving" (Section 3.2): c rows drawn by their
                      scores, each scaled by 1 / sqrt(c p_i).
  repeated_halving    Algorithm "Repeated Halving" (Section 3.2): halve uniformly down to a small level, then
                      back up, sampling each level by its approximate generalised leverage scores with respect to
                      the spectral approximation of the level below.
  rh_lsar             the RH variant of LSAR (end of Section 3.2): Algorithm "LSAR" with the leverage scores
                      replaced by those Repeated Halving gives for the lag-p_bar matrix [X | b].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg

U64 = np.finfo(np.float64).eps / 2.0   # unit roundoff of float64


def _series(y, p: int) -> np.ndarray:
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
    if y.ndim != 1:
        raise ValueError("y must be one-dimensional")
    if p < 1 or y.size <= p:
        raise ValueError("need p >= 1 and n > p")
    return y


def lag_matrix(y, p: int, start: int = 0, stop: int | None = None):
    """Rows [start, stop) of X and b, eq. (xphi): X[i, j] = y[p+i-j-1], b[i] = y[p+i]."""
    y = _series(y, p)
    m = y.size - p
    stop = m if stop is None else min(stop, m)
    rows = np.arange(start, stop)
    cols = np.arange(p)
    X = y[p + rows[:, None] - cols[None, :] - 1]
    b = y[p + rows]
    return X, b


def matvec(y, p: int, v) -> np.ndarray:
    """(X v)[i] = sum_j X[i, j] v[j] with the explicit X of eq. (xphi)."""
    X, _ = lag_matrix(y, p)
    return X @ np.asarray(v, dtype=np.float64)


def rmatvec(y, p: int, u) -> np.ndarray:
    """(X^T u)[j] = sum_i X[i, j] u[i] with the explicit X of eq. (xphi)."""
    X, _ = lag_matrix(y, p)
    return X.T @ np.asarray(u, dtype=np.float64)


@dataclass
class OracleSolution:
    phi: np.ndarray          # the least-squares (or minimum-norm least-squares) coefficients
    rnorm: float             # ||b - X phi||_2 recomputed explicitly from phi
    R: np.ndarray            # p x p triangle of the QR of X
    c: np.ndarray            # first p entries of Q^T b
    sigma: np.ndarray        # singular values of R (= of X), descending
    rank_deficient: bool
    ne_ratio: float          # ||X^T r|| / (||X||_2 ||r||)
    g: np.ndarray            # X^T r

    @property
    def norm2(self) -> float:
        return float(self.sigma[0]) if self.sigma.size else 0.0

    @property
    def kappa(self) -> float:
        return float(self.sigma[0] / self.sigma[-1]) if self.sigma[-1] > 0 else math.inf

    @property
    def eta(self) -> float:
        nphi = float(np.linalg.norm(self.phi))
        return self.rnorm / (self.norm2 * nphi) if nphi > 0 and self.norm2 > 0 else math.inf

    def forward_error_bound(self) -> float:
        """First-order relative forward-error bound 10 u (kappa + kappa^2 eta) of a backward-stable LS solve."""
        k = self.kappa
        return 10.0 * U64 * (k + k * k * self.eta)


def _qr_triangle(y: np.ndarray, p: int, block_rows: int) -> np.ndarray:
    """The (p+1) x (p+1) triangle of the Householder QR of [X | b], rows streamed in blocks."""
    m = y.size - p
    tri = np.zeros((0, p + 1))
    for start in range(0, m, block_rows):
        X, b = lag_matrix(y, p, start, start + block_rows)
        stacked = np.vstack([tri, np.column_stack([X, b])])
        tri = np.linalg.qr(stacked, mode="r")
    if tri.shape[0] < p + 1:
        tri = np.vstack([tri, np.zeros((p + 1 - tri.shape[0], p + 1))])
    return tri


def residual_check(y, p: int, phi, norm2: float | None = None, block_rows: int = 65536):
    """r = b - X phi, g = X^T r, ||r|| and ||g|| / (||X||_2 ||r||), with explicit X in row blocks.

    ||r||^2 is a compensated (math.fsum) total of per-block sums. norm2 = ||X||_2 when known; otherwise it is
    taken from the singular values of the QR triangle.
    """
    y = _series(y, p)
    phi = np.asarray(phi, dtype=np.float64)
    m = y.size - p
    g = np.zeros(p)
    parts = []
    for start in range(0, m, block_rows):
        X, b = lag_matrix(y, p, start, start + block_rows)
        r = b - X @ phi
        parts.append(float(np.dot(r, r)))
        g += X.T @ r
    rnorm = math.sqrt(math.fsum(parts))
    if norm2 is None:
        tri = _qr_triangle(y, p, block_rows)
        norm2 = float(np.linalg.svd(tri[:p, :p], compute_uv=False)[0])
    ratio = float(np.linalg.norm(g)) / (norm2 * rnorm) if rnorm > 0 and norm2 > 0 else 0.0
    return rnorm, g, ratio


def ols_qr(y, p: int, block_rows: int = 65536, rank_tol: float | None = None) -> OracleSolution:
    """argmin_phi ||X phi - b||_2 (minimum-norm when rank deficient), Thm. "Solution to OLS problem".

    R phi = c by back substitution when R is numerically nonsingular
    (sigma_min / sigma_max > rank_tol, default 1e-13 * p); otherwise phi = R^+ c from the SVD of R, which is
    the minimum-norm solution because X^+ = R^+ Q^T when Q has orthonormal columns.
    """
    y = _series(y, p)
    tri = _qr_triangle(y, p, block_rows)
    R = tri[:p, :p]
    c = tri[:p, p]
    U, s, Vt = np.linalg.svd(R)
    tol = (1e-13 * p) if rank_tol is None else rank_tol
    deficient = not (s[0] > 0 and s[-1] > tol * s[0])
    if not deficient:
        phi = scipy.linalg.solve_triangular(R, c, lower=False)
    else:
        keep = s > (tol * s[0] if s[0] > 0 else 0.0)
        phi = Vt[keep].T @ ((U[:, keep].T @ c) / s[keep])
    rnorm, g, ratio = residual_check(y, p, phi, norm2=float(s[0]), block_rows=block_rows)
    return OracleSolution(phi=phi, rnorm=rnorm, R=R, c=c, sigma=s, rank_deficient=deficient, ne_ratio=ratio, g=g)


def gram(y, p: int, block_rows: int = 65536):
    """G = X^T X (p x p) and h = X^T b (p), summed over row blocks of the explicit X."""
    y = _series(y, p)
    m = y.size - p
    G = np.zeros((p, p))
    h = np.zeros(p)
    for start in range(0, m, block_rows):
        X, b = lag_matrix(y, p, start, start + block_rows)
        G += X.T @ X
        h += X.T @ b
    return G, h


def row_norms(y, p: int):
    """||X(i,:)||^2 for every row i, and ||X||_F^2 (compensated total)."""
    X, _ = lag_matrix(y, p)
    rn = np.sum(X * X, axis=1)
    return rn, math.fsum(rn.tolist())


def exact_leverage(y, p: int) -> np.ndarray:
    """Def. "Leverage Score": l(i) = x_i^T (X^T X)^{-1} x_i, the diagonal of the hat matrix (small m only)."""
    X, _ = lag_matrix(y, p)
    Ginv = np.linalg.inv(X.T @ X)
    return np.einsum("ij,jk,ik->i", X, Ginv, X)


def leverage_p1(y) -> np.ndarray:
    """l_{n,1}(i) = y_i^2 / sum_{t=1}^{n-1} y_t^2 for the n-1 rows of the AR(1) matrix (0-based: y[0..n-2])."""
    y = np.asarray(y, dtype=np.float64)
    head = y[:-1]
    return head * head / math.fsum((head * head).tolist())


def leverage_step(y, p: int, phi_hat, lev_prev):
    """One step of eqs. (FALS)/(FAR)/(FASD) for order p >= 2.

    The order-(p-1) problem lives on the first n-1 samples: X' = X_{n-1,p-1}, b' = y_{n-1,p-1}, both with
    m = n - p rows. Its matrix satisfies X_{n,p} = [b' | X'] (the lag-1 column of the order-p matrix is the
    order-(p-1) response), so with r = X' phi_hat - b':

        l_new(i) = lev_prev(i) + r(i)^2 / ||r||^2,   pi(i) = l_new(i) / p.

    Returns (l_new, pi, ||r||^2).
    """
    y = _series(y, p)
    phi_hat = np.asarray(phi_hat, dtype=np.float64)
    if phi_hat.size != p - 1:
        raise ValueError("phi_hat must have p-1 entries")
    Xp, bp = lag_matrix(y[:-1], p - 1)
    r = Xp @ phi_hat - bp
    s = math.fsum((r * r).tolist())
    lev = np.asarray(lev_prev, dtype=np.float64) + r * r / s
    return lev, lev / p, s


def pacf(y, h_max):
    """PACF estimates tau_h, h = 1 .. h_max (Def. "Partial Autocorrelation Function", Section 3): tau_h is the last
    coefficient of the AR(h) least-squares fit (ols_qr), and the order estimate is the largest h with
    |tau_h| >= 1.96 / sqrt(n - h), n - h the rows of that fit (0 if none).
    """
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    tau = np.array([ols_qr(y, h).phi[h - 1] for h in range(1, h_max + 1)])
    order = 0
    for h in range(1, h_max + 1):
        if abs(tau[h - 1]) >= 1.96 / np.sqrt(n - h):
            order = h
    return tau, order


def leverage_sample(lev, u) -> np.ndarray:
    """Rows drawn with replacement from pi(i) = lev(i) / p, eq. (FASD) (sum lev = p in exact arithmetic, so pi is
    lev normalised by its sum): draw k is the smallest row i with lev[0] + ... + lev[i] > u[k] * sum(lev), or the
    last row if rounding leaves no such i. u: uniforms in [0, 1)."""
    lev = np.asarray(lev, dtype=np.float64)
    cdf = np.cumsum(lev)
    t = np.asarray(u, dtype=np.float64) * cdf[-1]
    return np.minimum(np.searchsorted(cdf, t, side="right"), lev.size - 1).astype(np.int64)


def compressed_ols(y, p: int, rows, pi_rows, c: int) -> np.ndarray:
    """Minimiser of ||S X phi - S b|| (Algorithm "LSAR", Section 3.1): S takes row rows[k] of X and b of
    eq. (xphi) and scales it by 1 / sqrt(c pi_rows[k])."""
    y = _series(y, p)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.arange(p)
    Xs = y[p + rows[:, None] - cols[None, :] - 1]
    bs = y[p + rows]
    s = 1.0 / np.sqrt(c * np.asarray(pi_rows, dtype=np.float64))
    phi, *_ = np.linalg.lstsq(Xs * s[:, None], bs * s, rcond=None)
    return phi


@dataclass
class LsarResult:
    tau: np.ndarray          # PACF estimates tau_p, p = 1 .. p_bar
    order: int               # largest p with |tau_p| >= 1.96 / sqrt(c), 0 if none
    phi: list                # phi_hat at each lag (p coefficients at lag p)
    rows: np.ndarray         # (p_bar, c) sampled rows
    lev_sum: np.ndarray      # sum of the approximate leverage scores at each lag (p in exact arithmetic)
    rr: np.ndarray           # ||r||^2 of eq. (FAR) feeding lag p (nan at lag 1)


def lsar(y, p_bar: int, c: int, unif) -> LsarResult:
    """Algorithm "LSAR" (Section 3.1) with the c rows per lag drawn by leverage_sample from unif[p - 1].

    Every lag uses the same m = n - p_bar rows: at lag p the data are y[0 .. m + p) and its order-p matrix of
    eq. (xphi) has m rows. Lag 1 samples by the exact scores l_{.,1}; lag p >= 2 by l_p = l_{p-1} + r^2/||r||^2,
    eq. (FALS), with r the full-data residual of lag p-1's compressed estimate, eq. (FAR)."""
    y = _series(y, p_bar)
    unif = np.asarray(unif, dtype=np.float64)
    if unif.shape != (p_bar, c):
        raise ValueError("unif must have shape (p_bar, c)")
    m = y.size - p_bar
    tau = np.empty(p_bar)
    rows_all = np.empty((p_bar, c), dtype=np.int64)
    lev_sum = np.empty(p_bar)
    rr = np.full(p_bar, np.nan)
    phis = []
    lev = phi = None
    for p in range(1, p_bar + 1):
        yp = y[:m + p]
        if p == 1:
            lev = leverage_p1(yp)
        else:
            lev, _, rr[p - 1] = leverage_step(yp, p, phi, lev)
        pi = lev / p
        rows = leverage_sample(lev, unif[p - 1])
        phi = compressed_ols(yp, p, rows, pi[rows], c)
        tau[p - 1] = phi[p - 1]
        rows_all[p - 1] = rows
        lev_sum[p - 1] = math.fsum(lev.tolist())
        phis.append(phi)
    thr = 1.96 / math.sqrt(c)
    order = max([h for h in range(1, p_bar + 1) if abs(tau[h - 1]) >= thr], default=0)
    return LsarResult(tau=tau, order=order, phi=phis, rows=rows_all, lev_sum=lev_sum, rr=rr)


def hadamard_transform(v) -> np.ndarray:
    """H_m v, Def. "Hadamard Transform" (Section 2.1): H_0 = 1, H_m = [[H_{m-1}, H_{m-1}], [H_{m-1}, -H_{m-1}]] / sqrt(2),
    applied by that recursion (stage h combines the halves of every block of 2h entries). len(v) = 2^m."""
    v = np.array(v, dtype=np.float64, copy=True)
    n = v.size
    if n & (n - 1):
        raise ValueError("length must be a power of two")
    s = 1.0 / math.sqrt(2.0)
    h = 1
    while h < n:
        blocks = v.reshape(-1, 2, h)
        top = blocks[:, 0, :].copy()
        bot = blocks[:, 1, :].copy()
        blocks[:, 0, :] = (top + bot) * s
        blocks[:, 1, :] = (top - bot) * s
        h *= 2
    return v


def srht_ols(y, p: int, rows, signs) -> np.ndarray:
    """Algorithm "SRHT" (Section 2.1): phi minimising ||S H D (X phi - b)||, eq. (SRHT). The m rows of [X | b] are
    zero-padded to m2 = 2^ceil(log2 m); D = diag(signs) (m2 entries of +-1); H the normalised Hadamard transform
    of size m2; S takes rows[t] (drawn uniformly with replacement, c = len(rows) of them) scaled by sqrt(m2 / c)."""
    X, b = lag_matrix(y, p)
    m = X.shape[0]
    m2 = 1 << max(0, (m - 1).bit_length())
    signs = np.asarray(signs, dtype=np.float64)
    if signs.size != m2:
        raise ValueError("need one sign per padded row")
    Z = np.zeros((m2, p + 1))
    Z[:m, :p] = X
    Z[:m, p] = b
    Z *= signs[:, None]
    for j in range(p + 1):
        Z[:, j] = hadamard_transform(Z[:, j])
    rows = np.asarray(rows, dtype=np.int64)
    sc = math.sqrt(m2 / rows.size)
    phi, *_ = np.linalg.lstsq(sc * Z[rows, :p], sc * Z[rows, p], rcond=None)
    return phi


def generalized_leverage(C, B, G=None) -> np.ndarray:
    """Def. "Generalised Leverage Score" (Section 3.2): l^B(i) = C(i,:) (B^T B)^{-1} C(i,:)^T; with a sketch G
    (k x rows(B)), eq. (glev): ||G B (B^T B)^{-1} C(i,:)^T||^2."""
    C = np.asarray(C, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    K = np.linalg.solve(B.T @ B, C.T)            # (B^T B)^{-1} C^T, one column per row of C
    if G is None:
        return np.einsum("ij,ji->i", C, K)
    V = np.asarray(G, dtype=np.float64) @ (B @ K)   # G B (B^T B)^{-1} C(i,:)^T, one column per row
    return np.sum(V * V, axis=0)


@dataclass
class RHResult:
    scores: np.ndarray       # approximate generalised leverage scores of the rows of X (w.r.t. the level below)
    rows: np.ndarray         # the c rows of X sampled at the top level
    Xt: np.ndarray           # the spectral approximation: those rows, each scaled by 1 / sqrt(c p_i)
    sizes: list              # rows at each halving level, top first


def spectral_approximation(A, scores, u, c: int):
    """The sampling step of Algorithm "Repeated Halving" (Section 3.2): c rows of A drawn with replacement from
    p_i = scores_i / sum(scores) by leverage_sample on the uniforms u, each scaled by 1 / sqrt(c p_i). Returns the
    drawn row indices and the scaled rows (the approximation that the level above is scored against)."""
    rows = leverage_sample(scores, u)
    prob = scores[rows] / math.fsum(np.asarray(scores, dtype=np.float64).tolist())
    return rows, np.asarray(A, dtype=np.float64)[rows] / np.sqrt(c * prob)[:, None]


def repeated_halving(X, c: int, min_rows: int, keep, gauss, unif) -> RHResult:
    """Algorithm "Repeated Halving" (Section 3.2) with its random draws as inputs.

    Level 0 is X; while level j has more than min_rows rows, level j+1 is its rows keep[j] (floor(n_j / 2)
    distinct positions within level j, increasing: a uniform sample without replacement). The deepest level is
    its own spectral approximation. Going back up, level j's rows get the approximate generalised leverage scores of eq. (glev)
    with respect to the approximation of level j+1 (sketch gauss[j], k x rows of that approximation), and c rows
    are drawn with replacement by leverage_sample on unif[j], each scaled by 1 / sqrt(c p_i),
    p_i = score_i / sum(scores)."""
    X = np.asarray(X, dtype=np.float64)
    levels = [X]
    while levels[-1].shape[0] > min_rows:
        j = len(levels) - 1
        kj = np.asarray(keep[j], dtype=np.int64)
        if kj.size != levels[j].shape[0] // 2:
            raise ValueError("keep[j] must hold floor(n_j / 2) positions")
        levels.append(levels[j][kj])
    Xt = levels[-1]
    scores = rows = None
    for j in range(len(levels) - 2, -1, -1):
        scores = generalized_leverage(levels[j], Xt, gauss[j])
        rows, Xt = spectral_approximation(levels[j], scores, unif[j], c)
    if scores is None:                         # X itself is small: its exact scores, all of its rows
        scores = generalized_leverage(X, X)
        rows = np.arange(X.shape[0])
    return RHResult(scores=scores, rows=rows, Xt=Xt, sizes=[lv.shape[0] for lv in levels])


def rh_lsar(y, p_bar: int, c: int, rh: RHResult, unif) -> LsarResult:
    """The RH variant of Algorithm "LSAR" (end of Section 3.2): rh holds Repeated Halving run on [X | b] of order
    p_bar (m = n - p_bar rows); at every lag p the c rows are drawn by leverage_sample from rh.scores with
    unif[p - 1] and weighted by 1 / sqrt(c pi_i), pi = scores / sum(scores); the compressed fit, tau_p and the
    order estimate are those of lsar."""
    y = _series(y, p_bar)
    unif = np.asarray(unif, dtype=np.float64)
    if unif.shape != (p_bar, c):
        raise ValueError("unif must have shape (p_bar, c)")
    m = y.size - p_bar
    if rh.scores.size != m:
        raise ValueError("scores must cover the m = n - p_bar rows")
    pi = rh.scores / math.fsum(rh.scores.tolist())
    tau = np.empty(p_bar)
    rows_all = np.empty((p_bar, c), dtype=np.int64)
    phis = []
    for p in range(1, p_bar + 1):
        rows = leverage_sample(rh.scores, unif[p - 1])
        phi = compressed_ols(y[:m + p], p, rows, pi[rows], c)
        tau[p - 1] = phi[p - 1]
        rows_all[p - 1] = rows
        phis.append(phi)
    thr = 1.96 / math.sqrt(c)
    order = max([h for h in range(1, p_bar + 1) if abs(tau[h - 1]) >= thr], default=0)
    return LsarResult(tau=tau, order=order, phi=phis, rows=rows_all, lev_sum=np.full(p_bar, np.nan),
                      rr=np.full(p_bar, np.nan))
