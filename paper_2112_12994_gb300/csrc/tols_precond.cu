// Multi-CTA preconditioner of single-series solves: the factor R of LSQR on X R^{-1} (eq. (xphi), Section 3).
//
//   Gram path : G = X^T X from the Gram pass -> blocked Cholesky G = R^T R over 32 x 32 tiles (one launch for the
//               panel and one for the trailing update per tile column) -> M = R^{-1} (one warp per column) ->
//               kappa(R) = ||X||_2 ||M||_2 by power iteration.
//   QR path   : for float64 solves whose Gram factor is not trusted. c rows of X sampled evenly (the row-sampling
//               idea of Section 3.1, put to use as a preconditioner) and factored by shifted Cholesky QR
//               (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa 2020: a Cholesky factor of A^T A + s I, then
//               Q = A R^{-1}, repeated): two shifted stages and one plain one, R = R3 R2 R1. Every step is a tall
//               Gram product, a blocked Cholesky or a row-parallel triangular solve, so the whole GPU works on it;
//               a Householder QR of the sample spends its time in column-by-column reductions on one SM.
//
// GB300 runs float64 at 2 FMAs per clock per SM, so what counts is spreading the O(c p^2) and O(p^3) work over
// all 152 SMs. The host (tols_api.cu) launches the steps and reads PclInfo between factorisations.
#include <math.h>

#include "tols_internal.cuh"

namespace tols {
namespace {

constexpr int kT = 32;            // tile edge of the blocked kernels
constexpr int kTT = 256;          // threads of the tile kernels
constexpr int kOT = 1024;         // threads of the one-CTA kernels (power iterations)
constexpr int kInvWarps = 8;      // columns (warps) per CTA of the inverse
constexpr int kTrsmRows = 16;     // rows of the sample per CTA of the triangular solve

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float wsumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum (and max) over a CTA of kOT threads; every thread gets the result.
__device__ double bsum(double v, double* red) {
  v = wsum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += red[k];
  __syncthreads();
  return r;
}
__device__ double bmax(double v, double* red) {
  v = wmax(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, red[k]);
  __syncthreads();
  return r;
}

// Upper tile (a, b), a <= b, of an n x n tile grid from its index in row order: (0,0) (0,1) .. (0,n-1) (1,1) ...
__device__ __forceinline__ void upper_tile(int idx, int n, int& a, int& b) {
  a = 0;
  while (idx >= n - a) {
    idx -= n - a;
    ++a;
  }
  b = a + idx;
}

// ---- power iteration ------------------------------------------------------------------------------------
// lambda_max of the symmetric p x p matrix S (leading dimension ld; upper triangle read), its trace and largest
// diagonal entry (kept in info->lam_keep[keep] when keep >= 0; keep 0 also keeps the trace). 8 power iterations in float arithmetic on a copy scaled by 1 / max_j S_jj (two digits suffice:
// the result scales a shift or enters a ratio). With shift_rel > 0 the first p diagonal entries of S then get
// shift_rel * lambda_max added (a shifted Cholesky QR stage); info->shift records the amount.
__global__ void __launch_bounds__(kOT) pcl_lambda_kernel(double* S, int ld, int p, double shift_rel, int keep,
                                                          float* fb, PclInfo* info) {
  __shared__ float xs[TOLS_MAX_P], ys[TOLS_MAX_P];
  __shared__ double red[32];
  __shared__ float redf[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double tr = 0.0, dm = 0.0;
  for (int j = tid; j < p; j += blockDim.x) {
    const double d = S[(size_t)j * ld + j];
    tr += d;
    dm = fmax(dm, d);
  }
  tr = bsum(tr, red);
  dm = bmax(dm, red);
  const float inv = (dm > 0.0 && isfinite(dm)) ? (float)(1.0 / dm) : 1.0f;
  for (int i = warp; i < p; i += nw)
    for (int j = i + lane; j < p; j += 32) {
      const float g = (float)S[(size_t)i * ld + j] * inv;
      fb[(size_t)i * p + j] = g;
      fb[(size_t)j * p + i] = g;
    }
  for (int j = tid; j < p; j += blockDim.x) xs[j] = 1.0f;
  __syncthreads();
  float dot = 0.f, xx = 0.f;
  for (int it = 0; it < 8; ++it) {
    float d0 = 0.f, x0 = 0.f;
    for (int i = tid; i < p; i += blockDim.x) {          // ys = S xs, column i of the symmetric copy
      float a0 = 0.f, a1 = 0.f;
      int j = 0;
      for (; j + 1 < p; j += 2) {
        a0 = fmaf(fb[(size_t)j * p + i], xs[j], a0);
        a1 = fmaf(fb[(size_t)(j + 1) * p + i], xs[j + 1], a1);
      }
      if (j < p) a0 = fmaf(fb[(size_t)j * p + i], xs[j], a0);
      ys[i] = a0 + a1;
      d0 = fmaf(xs[i], a0 + a1, d0);
      x0 = fmaf(xs[i], xs[i], x0);
    }
    d0 = wsumf(d0);
    x0 = wsumf(x0);
    if (lane == 0) {
      redf[warp] = d0;
      redf[32 + warp] = x0;
    }
    __syncthreads();
    dot = 0.f;
    xx = 0.f;
    for (int k = 0; k < nw; ++k) {
      dot += redf[k];
      xx += redf[32 + k];
    }
    const float scale = dot > 0.f ? xx / dot : 0.f;
    for (int j = tid; j < p; j += blockDim.x) xs[j] = ys[j] * scale;
    __syncthreads();
  }
  const double lam = xx > 0.f ? (double)dot / (double)xx * dm : 0.0;
  if (tid == 0) {
    info->lam = lam;
    info->dmax = dm;
    info->trace = tr;
    info->shift = shift_rel > 0.0 ? shift_rel * lam : 0.0;
    if (keep >= 0) info->lam_keep[keep] = lam;
    if (keep == 0) info->trace_g = tr;
    if (!isfinite(tr) || !isfinite(lam)) info->nonfinite = 1;
  }
  if (shift_rel > 0.0)
    for (int j = tid; j < p; j += blockDim.x) S[(size_t)j * ld + j] += shift_rel * lam;
}

// Gp (P x P) <- G (p x p) plus shift on the diagonal, identity on the padding; Gsave (nullable) <- G.
__global__ void pcl_pad_kernel(const double* __restrict__ G, int p, double* __restrict__ Gp, int P, double shift,
                               double* __restrict__ Gsave) {
  const size_t tot = (size_t)P * P;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / P), j = (int)(q - (size_t)i * P);
    double v;
    if (i < p && j < p) {
      v = G[(size_t)i * p + j];
      if (Gsave) Gsave[(size_t)i * p + j] = v;
      if (i == j) v += shift;
    } else {
      v = i == j ? 1.0 : 0.0;
    }
    Gp[q] = v;
  }
}

// ---- blocked Cholesky G = R^T R (upper) over 32 x 32 tiles ------------------------------------------------
// Step k, panel: CTA b (tile column j = k + b) factors the diagonal tile (k, k) itself (11k FMAs: cheaper than a
// separate launch and a grid-wide wait), writes it (b = 0) or solves R_kk^T R_kj = A_kj for its tile of row k.
// A pivot at or below tiny = tiny_dmax max_j G_jj + tiny_shift (shift added), i.e. at rounding level, sets
// info->fail and every later step returns at once. Only the first p pivots are tested: the padding is an identity.
__global__ void __launch_bounds__(kTT) pcl_chol_panel_kernel(double* Gp, int P, int p, int k, double tiny_dmax,
                                                             double tiny_shift, PclInfo* info) {
  __shared__ double D[kT][kT + 1];
  __shared__ double X[kT][kT + 1];
  __shared__ double rinv[kT];
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  if (tid == 0) s_fail = *(volatile int*)&info->fail;
  __syncthreads();
  if (s_fail) return;
  const double tiny = tiny_dmax * info->dmax + tiny_shift * info->shift;
  const int j = k + blockIdx.x;
  const double* Dk = Gp + (size_t)k * kT * P + (size_t)k * kT;
  const double* Ak = Gp + (size_t)k * kT * P + (size_t)j * kT;
  for (int q = tid; q < kT * kT; q += kTT) {
    const int a = q >> 5, b = q & 31;
    D[a][b] = Dk[(size_t)a * P + b];
    if (j > k) X[a][b] = Ak[(size_t)a * P + b];
  }
  __syncthreads();
  for (int r = 0; r < kT; ++r) {
    if (tid == 0) {
      const double piv = D[r][r];
      // the padding (identity, never updated) has unit pivots: only the first p are tested
      if (!(piv > tiny) && (k * kT + r < p || !(piv > 0.0))) {
        s_fail = 1;
      } else {
        const double ri = rsqrt_newton(piv);
        rinv[r] = ri;
        D[r][r] = piv * ri;
      }
    }
    __syncthreads();
    if (s_fail) break;
    for (int c = r + 1 + tid; c < kT; c += kTT) D[r][c] *= rinv[r];
    __syncthreads();
    // trailing triangle a <= b of rows r+1..31
    for (int q = tid; q < kT * kT; q += kTT) {
      const int a = q >> 5, b = q & 31;
      if (a > r && b >= a) D[a][b] = fma(-D[r][a], D[r][b], D[a][b]);
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) atomicExch(&info->fail, 1);
    return;
  }
  if (j == k) {
    double* out = Gp + (size_t)k * kT * P + (size_t)k * kT;
    for (int q = tid; q < kT * kT; q += kTT) {
      const int a = q >> 5, b = q & 31;
      out[(size_t)a * P + b] = b >= a ? D[a][b] : 0.0;
    }
    return;
  }
  // R_kk^T X = A: row r of X is final once the earlier rows' parts are removed; then it is removed from the rows
  // below (right-looking)
  for (int r = 0; r < kT; ++r) {
    if (tid < kT) X[r][tid] *= rinv[r];
    __syncthreads();
    for (int q = tid; q < (kT - 1 - r) * kT; q += kTT) {
      const int a = r + 1 + (q >> 5), c = q & 31;
      X[a][c] = fma(-D[r][a], X[r][c], X[a][c]);
    }
    __syncthreads();
  }
  double* out = Gp + (size_t)k * kT * P + (size_t)j * kT;
  for (int q = tid; q < kT * kT; q += kTT) out[(size_t)(q >> 5) * P + (q & 31)] = X[q >> 5][q & 31];
}

// Step k, trailing update: A_ij -= R_ki^T R_kj for the tiles k < i <= j < nt (one CTA per tile, 2 x 2 entries per
// thread).
__global__ void __launch_bounds__(kTT) pcl_chol_update_kernel(double* Gp, int P, int k, const PclInfo* info) {
  __shared__ double Ri[kT][kT + 1];
  __shared__ double Rj[kT][kT + 1];
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  if (tid == 0) s_fail = *(volatile const int*)&info->fail;
  __syncthreads();
  if (s_fail) return;
  const int nt = P / kT;
  int a, b;
  upper_tile(blockIdx.x, nt - k - 1, a, b);
  const int ti = k + 1 + a, tj = k + 1 + b;
  const double* Rki = Gp + (size_t)k * kT * P + (size_t)ti * kT;
  const double* Rkj = Gp + (size_t)k * kT * P + (size_t)tj * kT;
  for (int q = tid; q < kT * kT; q += kTT) {
    const int r = q >> 5, c = q & 31;
    Ri[r][c] = Rki[(size_t)r * P + c];
    Rj[r][c] = Rkj[(size_t)r * P + c];
  }
  __syncthreads();
  const int r0 = (tid >> 4) * 2, c0 = (tid & 15) * 2;
  double a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
#pragma unroll 8
  for (int q = 0; q < kT; ++q) {
    const double x0 = Ri[q][r0], x1 = Ri[q][r0 + 1];
    const double z0 = Rj[q][c0], z1 = Rj[q][c0 + 1];
    a00 = fma(x0, z0, a00);
    a01 = fma(x0, z1, a01);
    a10 = fma(x1, z0, a10);
    a11 = fma(x1, z1, a11);
  }
  double* C = Gp + (size_t)ti * kT * P + (size_t)tj * kT;
  C[(size_t)r0 * P + c0] -= a00;
  C[(size_t)r0 * P + c0 + 1] -= a01;
  C[(size_t)(r0 + 1) * P + c0] -= a10;
  C[(size_t)(r0 + 1) * P + c0 + 1] -= a11;
}

// ---- M = R^{-1} (R: upper triangle of Rp, P x P; M: p x p row-major, zero below the diagonal) ------------
// One warp per column c: back substitution M[i][c] = (delta_ic - sum_{j=i+1..c} R[i][j] M[j][c]) / R[i][i],
// i = c .. 0, with the column in shared memory. Columns are independent, so p warps run at once.
__global__ void __launch_bounds__(kInvWarps * 32) pcl_inverse_kernel(const double* __restrict__ Rp, int P, int p,
                                                                    double* __restrict__ M, const PclInfo* info) {
  extern __shared__ double colbuf[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (*(volatile const int*)&info->fail) return;
  const int c = blockIdx.x * kInvWarps + warp;
  if (c >= p) return;
  double* col = colbuf + (size_t)warp * P;
  for (int i = c; i >= 0; --i) {
    const double* Ri = Rp + (size_t)i * P;
    double s = 0.0;
    for (int j = i + 1 + lane; j <= c; j += 32) s = fma(Ri[j], col[j], s);
    s = wsum(s);
    const double v = ((i == c) ? 1.0 : 0.0) - s;
    const double mi = v / Ri[i];
    __syncwarp();
    if (lane == 0) col[i] = mi;
    __syncwarp();
  }
  for (int i = lane; i < p; i += 32) M[(size_t)i * p + c] = i <= c ? col[i] : 0.0;
}

// kappa(R) = ||X||_2 ||R^{-1}||_2: lambda_max(M^T M) by 6 power iterations in float on a copy of M scaled by
// 1 / max_i |M_ii| (one CTA); ||X||_2^2 is info->lam_keep[slot] (slot 1: the sample's, for the QR path).
__global__ void __launch_bounds__(kOT) pcl_estimate_kernel(const double* __restrict__ M, int p, int slot,
                                                            float* fb, PclInfo* info) {
  __shared__ float xs[TOLS_MAX_P], ys[TOLS_MAX_P];
  __shared__ double red[32];
  __shared__ float redf[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (*(volatile const int*)&info->fail) return;
  double dm = 0.0;
  for (int j = tid; j < p; j += blockDim.x) dm = fmax(dm, fabs(M[(size_t)j * p + j]));
  dm = bmax(dm, red);
  const float inv = (dm > 0.0 && isfinite(dm)) ? (float)(1.0 / dm) : 1.0f;
  for (int i = warp; i < p; i += nw)
    for (int j = i + lane; j < p; j += 32) fb[(size_t)i * p + j] = (float)M[(size_t)i * p + j] * inv;
  for (int j = tid; j < p; j += blockDim.x) xs[j] = 1.0f;
  __syncthreads();
  float dot = 0.f, xx = 0.f;
  for (int it = 0; it < 6; ++it) {
    for (int i = warp; i < p; i += nw) {                 // ys = M xs: a warp per row, lanes along the row
      float a = 0.f;
      for (int j = i + lane; j < p; j += 32) a = fmaf(fb[(size_t)i * p + j], xs[j], a);
      a = wsumf(a);
      if (lane == 0) ys[i] = a;
    }
    __syncthreads();
    float d0 = 0.f, x0 = 0.f;
    for (int j = tid; j < p; j += blockDim.x) {          // zs = M^T ys: a thread per column
      float b0 = 0.f, b1 = 0.f;
      int i = 0;
      for (; i + 1 <= j; i += 2) {
        b0 = fmaf(fb[(size_t)i * p + j], ys[i], b0);
        b1 = fmaf(fb[(size_t)(i + 1) * p + j], ys[i + 1], b1);
      }
      if (i <= j) b0 = fmaf(fb[(size_t)i * p + j], ys[i], b0);
      const float z = b0 + b1;
      d0 = fmaf(xs[j], z, d0);
      x0 = fmaf(xs[j], xs[j], x0);
      xs[j] = z;     // only this thread reads xs[j] in this loop; rescaled after the reduction
    }
    d0 = wsumf(d0);
    x0 = wsumf(x0);
    if (lane == 0) {
      redf[warp] = d0;
      redf[32 + warp] = x0;
    }
    __syncthreads();
    dot = 0.f;
    xx = 0.f;
    for (int k = 0; k < nw; ++k) {
      dot += redf[k];
      xx += redf[32 + k];
    }
    const float scale = dot > 0.f ? xx / dot : 0.f;
    for (int j = tid; j < p; j += blockDim.x) xs[j] *= scale;
    __syncthreads();
  }
  if (tid == 0) {
    const double lamM = xx > 0.f ? (double)dot / (double)xx * dm * dm : 0.0;
    info->cond = sqrt(fmax(info->lam_keep[slot], 0.0)) * sqrt(fmax(lamM, 0.0));
  }
}

// M^T, and the float copies the mixed path reads.
__global__ void pcl_store_kernel(Work w, int mixed, const PclInfo* info) {
  if (*(volatile const int*)&info->fail) return;
  const int p = w.p;
  const size_t tot = (size_t)p * p;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / p), j = (int)(q - (size_t)i * p);
    const double mv = w.M[q];
    const double tv = w.M[(size_t)j * p + i];
    w.Mt[q] = tv;
    if (mixed) {
      w.M32[q] = (float)mv;
      w.Mt32[q] = (float)tv;
    }
  }
}

// The solve's state after the preconditioner (the fields precond_kernel sets).
__global__ void pcl_state_kernel(Work w, const PclInfo* info, int precond, int shifted, int trusted, int singular,
                                 double cond, double kappa_est) {
  DevState* st = w.st;
  const double b2 = *w.bnorm2;
  if (info->nonfinite || !isfinite(b2)) {
    st->status = TOLS_ERR_NONFINITE;
    st->phase = PH_DONE;
    st->done = 1;
    st->precond = 0;
    return;
  }
  st->bnorm = sqrt(fmax(b2, 0.0));
  st->anorm_f = sqrt(fmax(info->trace_g, 0.0));
  st->anorm_2 = sqrt(fmax(info->lam_keep[0], 0.0));
  if (!(st->anorm_2 > 0.0)) st->anorm_2 = st->anorm_f;
  if (singular) st->singular = 1;
  st->precond = precond;
  st->cond_est = precond ? cond : 0.0;
  st->kappa_est = precond ? kappa_est : 0.0;
  st->shifted = shifted;
  st->trusted = trusted;
}

// ---- sampled rows and shifted Cholesky QR ---------------------------------------------------------------
// A (c x p, row-major) <- rows floor((2i + 1) m / (2c)) of X: A[i][j] = y[p + row_i - j - 1].
__global__ void pcl_gather_kernel(const double* __restrict__ y, long long m, int p, long long c, double* __restrict__ A) {
  for (long long i = blockIdx.x; i < c; i += gridDim.x) {
    const long long row = ((2 * i + 1) * m) / (2 * c);
    const double* yr = y + p + row - 1;
    for (int j = threadIdx.x; j < p; j += blockDim.x) A[(size_t)i * p + j] = yr[-j];
  }
}

// Partial Gram tiles of a tall matrix: the upper tiles (a <= b) of A^T A over the rows of slice blockIdx.y (S
// slices), 2 x 2 entries per thread, rows staged 32 at a time; part[(slice * ntiles + tile) * 1024 + r * 32 + c].
__global__ void __launch_bounds__(kTT) pcl_tall_gram_kernel(const double* __restrict__ A, long long c, int p, int nt,
                                                            double* __restrict__ part) {
  __shared__ double Ai[kT][kT + 1];
  __shared__ double Aj[kT][kT + 1];
  const int tid = threadIdx.x;
  int ta, tb;
  upper_tile(blockIdx.x, nt, ta, tb);
  const int S = gridDim.y;
  const long long lo = c * blockIdx.y / S, hi = c * (blockIdx.y + 1) / S;
  const int r0 = (tid >> 4) * 2, c0 = (tid & 15) * 2;
  double a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
  for (long long rb = lo; rb < hi; rb += kT) {
    __syncthreads();
    for (int q = tid; q < kT * kT; q += kTT) {
      const int rr = q >> 5, cc = q & 31;
      const long long row = rb + rr;
      const int ci = ta * kT + cc, cj = tb * kT + cc;
      Ai[rr][cc] = (row < hi && ci < p) ? A[(size_t)row * p + ci] : 0.0;
      Aj[rr][cc] = (row < hi && cj < p) ? A[(size_t)row * p + cj] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < kT; ++q) {
      const double x0 = Ai[q][r0], x1 = Ai[q][r0 + 1];
      const double z0 = Aj[q][c0], z1 = Aj[q][c0 + 1];
      a00 = fma(x0, z0, a00);
      a01 = fma(x0, z1, a01);
      a10 = fma(x1, z0, a10);
      a11 = fma(x1, z1, a11);
    }
  }
  const int ntiles = nt * (nt + 1) / 2;
  double* out = part + ((size_t)blockIdx.y * ntiles + blockIdx.x) * (kT * kT);
  out[r0 * kT + c0] = a00;
  out[r0 * kT + c0 + 1] = a01;
  out[(r0 + 1) * kT + c0] = a10;
  out[(r0 + 1) * kT + c0 + 1] = a11;
}

// Gp tile (a, b) <- the sum of the S slices' partial tiles, in slice order; identity on the padding.
__global__ void __launch_bounds__(kTT) pcl_gram_reduce_kernel(const double* __restrict__ part, int nt, int S, int p,
                                                              double* __restrict__ Gp, int P) {
  int ta, tb;
  upper_tile(blockIdx.x, nt, ta, tb);
  const int ntiles = nt * (nt + 1) / 2;
  for (int q = threadIdx.x; q < kT * kT; q += kTT) {
    const int gi = ta * kT + (q >> 5), gj = tb * kT + (q & 31);
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += part[((size_t)s * ntiles + blockIdx.x) * (kT * kT) + q];
    if (gi >= p || gj >= p) v = gi == gj ? 1.0 : 0.0;
    Gp[(size_t)gi * P + gj] = v;
  }
}

// Q = A R^{-1} in place (A: c x p, row-major; R: upper triangle of Rp, P x P, identity on the padding). A CTA
// owns kTrsmRows rows and keeps their finished entries in shared memory; per column tile J:
// acc = A[:, J] - Q[:, <J] R[<J, J] (two entries per thread), then acc R_JJ^{-1} by substitution over the tile's
// 32 columns (right-looking), in shared memory.
__global__ void __launch_bounds__(kTT) pcl_trsm_kernel(double* __restrict__ A, long long c, int p,
                                                       const double* __restrict__ Rp, int P) {
  extern __shared__ double qs[];             // [kTrsmRows][P + 1]
  __shared__ double Rjj[kT][kT + 1];
  __shared__ double blk[kTrsmRows][kT + 1];
  __shared__ double rinv[kT];
  const int tid = threadIdx.x;
  const long long r0 = (long long)blockIdx.x * kTrsmRows;
  const int ld = P + 1;
  const int row = tid >> 4, cb = (tid & 15) * 2;
  const bool live = r0 + row < c;
  const int nt = P / kT;
  for (int J = 0; J < nt; ++J) {
    const int j0 = J * kT;
    for (int q = tid; q < kT * kT; q += kTT) Rjj[q >> 5][q & 31] = Rp[(size_t)(j0 + (q >> 5)) * P + j0 + (q & 31)];
    const int ca = j0 + cb, cbb = j0 + cb + 1;
    double a0 = (live && ca < p) ? A[(size_t)(r0 + row) * p + ca] : 0.0;
    double a1 = (live && cbb < p) ? A[(size_t)(r0 + row) * p + cbb] : 0.0;
    const double* qrow = qs + (size_t)row * ld;
#pragma unroll 4
    for (int q = 0; q < j0; ++q) {
      const double qv = qrow[q];
      a0 = fma(-qv, Rp[(size_t)q * P + ca], a0);
      a1 = fma(-qv, Rp[(size_t)q * P + cbb], a1);
    }
    blk[row][cb] = a0;
    blk[row][cb + 1] = a1;
    __syncthreads();
    if (tid < kT) rinv[tid] = 1.0 / Rjj[tid][tid];
    __syncthreads();
    for (int b = 0; b < kT; ++b) {
      if (tid < kTrsmRows) blk[tid][b] *= rinv[b];
      __syncthreads();
      const int wdt = kT - 1 - b;
      for (int q = tid; q < kTrsmRows * wdt; q += kTT) {
        const int rr = q / wdt, cc = b + 1 + (q - rr * wdt);
        blk[rr][cc] = fma(-blk[rr][b], Rjj[b][cc], blk[rr][cc]);
      }
      __syncthreads();
    }
    const double q0 = blk[row][cb], q1 = blk[row][cb + 1];
    qs[(size_t)row * ld + ca] = q0;
    qs[(size_t)row * ld + cbb] = q1;
    if (live && ca < p) A[(size_t)(r0 + row) * p + ca] = q0;
    if (live && cbb < p) A[(size_t)(r0 + row) * p + cbb] = q1;
    __syncthreads();
  }
}

// Z = X Y for upper-triangular P x P matrices (tile (a, b), a <= b: sum over tiles q = a .. b).
__global__ void __launch_bounds__(kTT) pcl_trmm_kernel(const double* __restrict__ X, const double* __restrict__ Y,
                                                       double* __restrict__ Z, int P) {
  __shared__ double Xs[kT][kT + 1];
  __shared__ double Ys[kT][kT + 1];
  const int tid = threadIdx.x, nt = P / kT;
  int ta, tb;
  upper_tile(blockIdx.x, nt, ta, tb);
  const int r0 = (tid >> 4) * 2, c0 = (tid & 15) * 2;
  double a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
  for (int tq = ta; tq <= tb; ++tq) {
    __syncthreads();
    for (int q = tid; q < kT * kT; q += kTT) {
      const int rr = q >> 5, cc = q & 31;
      const double xv = X[(size_t)(ta * kT + rr) * P + tq * kT + cc];
      const double yv = Y[(size_t)(tq * kT + rr) * P + tb * kT + cc];
      // the strictly lower part of a diagonal tile is not part of the triangle
      Xs[rr][cc] = (tq == ta && cc < rr) ? 0.0 : xv;
      Ys[rr][cc] = (tq == tb && cc < rr) ? 0.0 : yv;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < kT; ++q) {
      const double x0 = Xs[r0][q], x1 = Xs[r0 + 1][q];
      const double z0 = Ys[q][c0], z1 = Ys[q][c0 + 1];
      a00 = fma(x0, z0, a00);
      a01 = fma(x0, z1, a01);
      a10 = fma(x1, z0, a10);
      a11 = fma(x1, z1, a11);
    }
  }
  double* out = Z + (size_t)(ta * kT) * P + tb * kT;
  const bool diag = ta == tb;
  out[(size_t)r0 * P + c0] = (diag && c0 < r0) ? 0.0 : a00;
  out[(size_t)r0 * P + c0 + 1] = (diag && c0 + 1 < r0) ? 0.0 : a01;
  out[(size_t)(r0 + 1) * P + c0] = (diag && c0 < r0 + 1) ? 0.0 : a10;
  out[(size_t)(r0 + 1) * P + c0 + 1] = (diag && c0 + 1 < r0 + 1) ? 0.0 : a11;
}

}  // namespace

// ---- launches ----------------------------------------------------------------------------------------------
cudaError_t pcl_lambda(double* S, int ld, int p, double shift_rel, int keep, float* fb, PclInfo* info,
                       cudaStream_t s) {
  pcl_lambda_kernel<<<1, kOT, 0, s>>>(S, ld, p, shift_rel, keep, fb, info);
  return cudaGetLastError();
}
cudaError_t pcl_pad(const double* G, int p, double* Gp, int P, double shift, double* Gsave, cudaStream_t s) {
  const int grid = (int)(((size_t)P * P + 255) / 256);
  pcl_pad_kernel<<<grid < 1024 ? grid : 1024, 256, 0, s>>>(G, p, Gp, P, shift, Gsave);
  return cudaGetLastError();
}
cudaError_t pcl_chol_panel(double* Gp, int P, int p, int k, double tiny_dmax, double tiny_shift, PclInfo* info,
                           cudaStream_t s) {
  pcl_chol_panel_kernel<<<P / kT - k, kTT, 0, s>>>(Gp, P, p, k, tiny_dmax, tiny_shift, info);
  return cudaGetLastError();
}
cudaError_t pcl_chol_update(double* Gp, int P, int k, const PclInfo* info, cudaStream_t s) {
  const int r = P / kT - k - 1;
  if (r < 1) return cudaSuccess;
  pcl_chol_update_kernel<<<r * (r + 1) / 2, kTT, 0, s>>>(Gp, P, k, info);
  return cudaGetLastError();
}
cudaError_t pcl_inverse(const double* Rp, int P, int p, double* M, const PclInfo* info, cudaStream_t s) {
  const size_t smem = sizeof(double) * kInvWarps * (size_t)P;
  cudaError_t e = smem_opt_in((const void*)pcl_inverse_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  pcl_inverse_kernel<<<(p + kInvWarps - 1) / kInvWarps, kInvWarps * 32, smem, s>>>(Rp, P, p, M, info);
  return cudaGetLastError();
}
cudaError_t pcl_estimate(const double* M, int p, int slot, float* fb, PclInfo* info, cudaStream_t s) {
  pcl_estimate_kernel<<<1, kOT, 0, s>>>(M, p, slot, fb, info);
  return cudaGetLastError();
}
cudaError_t pcl_store(const Work& w, int mixed, const PclInfo* info, cudaStream_t s) {
  const int grid = (int)(((size_t)w.p * w.p + 255) / 256);
  pcl_store_kernel<<<grid < 1024 ? grid : 1024, 256, 0, s>>>(w, mixed, info);
  return cudaGetLastError();
}
cudaError_t pcl_state(const Work& w, const PclInfo* info, int precond, int shifted, int trusted, int singular,
                      double cond, double kappa_est, cudaStream_t s) {
  pcl_state_kernel<<<1, 1, 0, s>>>(w, info, precond, shifted, trusted, singular, cond, kappa_est);
  return cudaGetLastError();
}
cudaError_t pcl_gather(const double* y, long long m, int p, long long c, double* A, cudaStream_t s) {
  const long long grid = c < 4096 ? c : 4096;
  pcl_gather_kernel<<<(int)grid, 128, 0, s>>>(y, m, p, c, A);
  return cudaGetLastError();
}
// Row slices of the tall Gram product: enough CTAs for two per SM of a 152-SM part, at least 256 rows each.
int pcl_gram_slices(long long c, int P) {
  const int nt = P / kT, ntiles = nt * (nt + 1) / 2;
  long long s = (2 * 152 + ntiles - 1) / ntiles;
  const long long smax = c / 256 > 0 ? c / 256 : 1;
  if (s > smax) s = smax;
  if (s < 1) s = 1;
  return (int)s;
}
cudaError_t pcl_tall_gram(const double* A, long long c, int p, int P, int slices, double* part, cudaStream_t s) {
  const int nt = P / kT;
  dim3 grid(nt * (nt + 1) / 2, slices);
  pcl_tall_gram_kernel<<<grid, kTT, 0, s>>>(A, c, p, nt, part);
  return cudaGetLastError();
}
cudaError_t pcl_gram_reduce(const double* part, int P, int slices, int p, double* Gp, cudaStream_t s) {
  const int nt = P / kT;
  pcl_gram_reduce_kernel<<<nt * (nt + 1) / 2, kTT, 0, s>>>(part, nt, slices, p, Gp, P);
  return cudaGetLastError();
}
cudaError_t pcl_trsm(double* A, long long c, int p, const double* Rp, int P, cudaStream_t s) {
  const size_t smem = sizeof(double) * kTrsmRows * (size_t)(P + 1);
  cudaError_t e = smem_opt_in((const void*)pcl_trsm_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  pcl_trsm_kernel<<<(int)((c + kTrsmRows - 1) / kTrsmRows), kTT, smem, s>>>(A, c, p, Rp, P);
  return cudaGetLastError();
}
cudaError_t pcl_trmm(const double* X, const double* Y, double* Z, int P, cudaStream_t s) {
  const int nt = P / kT;
  pcl_trmm_kernel<<<nt * (nt + 1) / 2, kTT, 0, s>>>(X, Y, Z, P);
  return cudaGetLastError();
}

}  // namespace tols
