// Algorithm "LSAR" (Section 3.1) on the device: for each lag p, the approximate leverage scores of
// Def. "Approximate Leverage Scores" (eqs. (FALS), (FAR), (FASD)), c rows drawn with replacement by inverse CDF,
// the compressed OLS problem on those rows (each scaled by 1 / sqrt(c pi_i)) and its solution phi_hat_p, whose
// last coefficient is the PACF estimate tau_p.
//
// The full-data residual r = X' phi_hat_{p-1} - b' of eq. (FAR) comes from the product pass (pass_kernel or
// fft_pass_kernel with no lag sums, its ||r||^2 reduced by the pass's tail). The kernels here:
//   lsar_lev_kernel     lev += r^2 / ||r||^2 (eq. (FALS)) and the sum of every block of kLsarBlock rows;
//   lsar_prefix_kernel  exclusive prefix of the block sums (one CTA, fixed order);
//   lsar_sample_kernel  one warp per draw: the block by a 32-ary search of the prefix, then the row by a warp
//                       scan inside the block; the draw's weight p / (c lev_i) = 1 / (c pi_i);
//   lsar_gram_kernel    per-CTA partial Gram of the weighted sampled rows [b | X] (augmented, upper triangle);
//   lsar_reduce_kernel  the partials summed in CTA order;
//   lsar_solve_kernel   one CTA: Cholesky of the sampled X^T W X, then phi = (X^T W X)^-1 X^T W b with one step
//                       of the corrected semi-normal equations (residual of the sampled rows, second solve).
// Every sum runs in a fixed order, so a sweep is bitwise reproducible. Rows with score 0 are never drawn.
#include <math.h>

#include "tols_internal.cuh"

namespace tols {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Inclusive warp scan in a fixed order. The block sums and the sampler both use it, so the running sum at a
// block's last row equals the block's sum bit for bit.
__device__ __forceinline__ double warp_incl_scan(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Index of entry (q, q2), q <= q2, of an upper triangle stored column by column.
__host__ __device__ __forceinline__ long long tri_index(int q, int q2) { return (long long)q2 * (q2 + 1) / 2 + q; }

// Inverse of tri_index.
__device__ __forceinline__ void tri_unpack(long long e, int& q, int& q2) {
  int c2 = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((long long)(c2 + 1) * (c2 + 2) / 2 <= e) ++c2;
  while ((long long)c2 * (c2 + 1) / 2 > e) --c2;
  q2 = c2;
  q = (int)(e - (long long)c2 * (c2 + 1) / 2);
}

}  // namespace

// lev[i] += r[i]^2 / ||r||^2 (r == nullptr: lev unchanged), then bsum[b] = sum of block b's lev in the sampler's
// order. One warp per block of kLsarBlock rows.
__global__ void __launch_bounds__(256) lsar_lev_kernel(const double* __restrict__ r, const double* rr, double* lev,
                                                       long long m, long long nb, double* bsum, const int* status) {
  if (*status) return;
  const long long b = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (b >= nb) return;
  const int lane = threadIdx.x & 31;
  const double inv = r ? 1.0 / *rr : 0.0;
  const long long i0 = b * kLsarBlock;
  double carry = 0.0;
  for (int ch = 0; ch < kLsarBlock / 32; ++ch) {
    const long long i = i0 + ch * 32 + lane;
    double v = 0.0;
    if (i < m) {
      v = lev[i];
      if (r) {
        v = fma(r[i] * r[i], inv, v);
        lev[i] = v;
      }
    }
    carry += __shfl_sync(kFull, warp_incl_scan(v), 31);
  }
  if (lane == 0) bsum[b] = carry;
}

// bpre[b] = bsum[0] + ... + bsum[b-1], b <= nb (bpre[nb] is the total). One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) lsar_prefix_kernel(const double* __restrict__ bsum, long long nb,
                                                           double* bpre, const int* status) {
  if (*status) return;
  __shared__ double s_warp[32];
  __shared__ double s_tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double carry = 0.0;   // the same value in every thread
  for (long long base = 0; base < nb; base += 1024) {
    const long long i = base + threadIdx.x;
    const double v = i < nb ? bsum[i] : 0.0;
    const double incl = warp_incl_scan(v);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const double wi = warp_incl_scan(s_warp[lane]);
      const double ex = __shfl_up_sync(kFull, wi, 1);
      if (lane == 31) s_tot = wi;
      __syncwarp();
      s_warp[lane] = lane ? ex : 0.0;
    }
    __syncthreads();
    const double within = __shfl_up_sync(kFull, incl, 1);
    if (i < nb) bpre[i] = carry + ((lane ? within : 0.0) + s_warp[wid]);
    carry += s_tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) bpre[nb] = carry;
}

// Draw k (one warp): t = unif[k] * total; the row is the first i whose running sum exceeds t, or, if rounding
// leaves none, the last row with a positive score. rows[k] = i, w2[k] = p / (c lev[i]) = 1 / (c pi_i).
__global__ void __launch_bounds__(256) lsar_sample_kernel(const double* __restrict__ lev, long long m,
                                                          const double* __restrict__ bsum,
                                                          const double* __restrict__ bpre, long long nb,
                                                          const double* __restrict__ unif, int c, int p,
                                                          long long* rows, double* w2, const int* status) {
  if (*status) return;
  const int k = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (k >= c) return;
  const int lane = threadIdx.x & 31;
  const double t = unif[k] * bpre[nb];
  // the largest block b with bpre[b] <= t; the answer stays in [lo, hi)
  long long lo = 0, hi = nb;
  while (hi - lo > 1) {
    const long long step = (hi - lo + 31) / 32;
    const long long q = lo + (long long)lane * step;
    const unsigned bal = __ballot_sync(kFull, q < hi && bpre[q] <= t);
    const int last = bal ? 31 - __clz((int)bal) : 0;
    lo += (long long)last * step;
    hi = lo + step < hi ? lo + step : hi;
  }
  const long long b = lo;
  const double base = bpre[b];
  const long long i0 = b * kLsarBlock;
  long long pick = -1, last_pos = -1;
  double carry = 0.0;
  for (int ch = 0; ch < kLsarBlock / 32 && pick < 0; ++ch) {
    const long long i = i0 + ch * 32 + lane;
    const double v = i < m ? lev[i] : 0.0;
    const double incl = warp_incl_scan(v);
    const unsigned hit = __ballot_sync(kFull, i < m && base + (carry + incl) > t);
    const unsigned pos = __ballot_sync(kFull, i < m && v > 0.0);
    if (hit) pick = i0 + ch * 32 + (__ffs((int)hit) - 1);
    else if (pos) last_pos = i0 + ch * 32 + (31 - __clz((int)pos));
    carry += __shfl_sync(kFull, incl, 31);
  }
  if (pick < 0 && last_pos < 0) {
    // no positive score in block b (only past the last positive block): the last earlier block with a positive
    // sum, then its last positive row
    long long bb = -1;
    for (long long s = b - 1; s >= 0 && bb < 0; s -= 32) {
      const long long q = s - lane;
      const unsigned bal = __ballot_sync(kFull, q >= 0 && bsum[q] > 0.0);
      if (bal) bb = s - (__ffs((int)bal) - 1);
    }
    if (bb >= 0) {
      for (int ch = 0; ch < kLsarBlock / 32; ++ch) {
        const long long i = bb * kLsarBlock + ch * 32 + lane;
        const unsigned pos = __ballot_sync(kFull, i < m && lev[i] > 0.0);
        if (pos) last_pos = bb * kLsarBlock + ch * 32 + (31 - __clz((int)pos));
      }
    }
  }
  if (pick < 0) pick = last_pos >= 0 ? last_pos : m - 1;
  if (lane == 0) {
    rows[k] = pick;
    w2[k] = (double)p / ((double)c * lev[pick]);
  }
}

// CTA g: part[g][e(q, q2)] = sum over its draws k of w2_k a_k[q] a_k[q2], a_k[q] = y[p + rows[k] - q]
// (q = 0: the response b, q = 1 + j: column j of X), q <= q2 <= p.
__global__ void __launch_bounds__(256) lsar_gram_kernel(const double* __restrict__ y, int p,
                                                        const long long* __restrict__ rows,
                                                        const double* __restrict__ w2, int c, int per_cta,
                                                        double* part, long long tri, const int* status) {
  if (*status) return;
  extern __shared__ double lsm[];
  const int P1 = p + 1;
  double* A = lsm;
  double* WA = lsm + kLsarChunk * P1;
  const int k0 = blockIdx.x * per_cta;
  const int k1 = min(c, k0 + per_cta);
  double* out = part + (size_t)blockIdx.x * tri;
  if (k0 >= k1) {
    for (long long e = threadIdx.x; e < tri; e += blockDim.x) out[e] = 0.0;
    return;
  }
  for (int kc = k0; kc < k1; kc += kLsarChunk) {
    const int cnt = min(kLsarChunk, k1 - kc);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * P1; e += blockDim.x) {
      const int kk = e / P1, q = e - kk * P1;
      const double v = y[p + rows[kc + kk] - q];
      A[kk * P1 + q] = v;
      WA[kk * P1 + q] = w2[kc + kk] * v;
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < tri; e += blockDim.x) {
      int q, q2;
      tri_unpack(e, q, q2);
      double acc = kc == k0 ? 0.0 : out[e];
      for (int kk = 0; kk < cnt; ++kk) acc = fma(WA[kk * P1 + q], A[kk * P1 + q2], acc);
      out[e] = acc;
    }
  }
}

__global__ void lsar_reduce_kernel(const double* __restrict__ part, int ng, long long tri, double* G,
                                   const int* status) {
  if (*status) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tri; e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < ng; ++g) s += part[(size_t)g * tri + e];
    G[e] = s;
  }
}

namespace {

// z := L^-1 z (forward) then z := L^-T z (backward), L lower triangular row-major with leading dimension p and
// reciprocal diagonal rdiag. One warp.
__device__ void chol_solve_warp(const double* L, const double* rdiag, int p, double* z) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < p; ++k) {
    const double zk = z[k] * rdiag[k];
    __syncwarp();
    if (lane == 0) z[k] = zk;
    for (int i = k + 1 + lane; i < p; i += 32) z[i] = fma(-L[(size_t)i * p + k], zk, z[i]);
    __syncwarp();
  }
  for (int k = p - 1; k >= 0; --k) {
    const double xk = z[k] * rdiag[k];
    __syncwarp();
    if (lane == 0) z[k] = xk;
    for (int i = lane; i < k; i += 32) z[i] = fma(-L[(size_t)k * p + i], xk, z[i]);
    __syncwarp();
  }
}

}  // namespace

// One CTA of kLsarSolveThreads. H[j][l] = G[e(1 + j, 1 + l)] (the sampled X^T W X), h[j] = G[e(0, 1 + j)]
// (X^T W b). L: p x p scratch (shared memory when p <= kLsarSmemP, else Lg in global memory); rw: c doubles of
// global scratch. Writes phi (p doubles) and tau[lag - 1]; on a pivot that is not positive and finite, phi and
// tau are NaN and *status becomes lag (later lags are skipped).
__global__ void __launch_bounds__(kLsarSolveThreads, 1) lsar_solve_kernel(
    const double* __restrict__ G, int p, const double* __restrict__ y, const long long* __restrict__ rows,
    const double* __restrict__ w2, int c, double* Lg, double* rw, double* phi, double* tau, int lag, int* status) {
  if (*status) return;
  extern __shared__ double lsm[];
  __shared__ int s_fail;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int kWarps = kLsarSolveThreads / 32;
  const bool in_smem = p <= kLsarSmemP;
  double* L = in_smem ? lsm : Lg;
  double* vec = lsm + (in_smem ? (size_t)p * p : 0);
  double* z = vec;              // p
  double* x = vec + p;          // p
  double* rdiag = vec + 2 * p;  // p
  double* wpart = vec + 3 * p;  // kWarps x p
  if (tid == 0) s_fail = 0;
  for (int idx = tid; idx < p * p; idx += kLsarSolveThreads) {
    const int i = idx / p, j = idx - i * p;
    L[idx] = j <= i ? G[tri_index(1 + j, 1 + i)] : 0.0;
  }
  for (int j = tid; j < p; j += kLsarSolveThreads) z[j] = G[tri_index(0, 1 + j)];
  __syncthreads();
  // right-looking Cholesky H = L L^T
  for (int k = 0; k < p; ++k) {
    if (tid == 0) {
      const double d = L[(size_t)k * p + k];
      if (!(d > 0.0) || !isfinite(d)) {
        s_fail = 1;
      } else {
        const double l = sqrt(d);
        L[(size_t)k * p + k] = l;
        rdiag[k] = 1.0 / l;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const double r = rdiag[k];
    for (int i = k + 1 + tid; i < p; i += kLsarSolveThreads) L[(size_t)i * p + k] *= r;
    __syncthreads();
    const int t = p - k - 1;
    for (int idx = tid; idx < t * t; idx += kLsarSolveThreads) {
      const int ii = idx / t, jj = idx - ii * t;
      if (jj <= ii) {
        const int i = k + 1 + ii, j = k + 1 + jj;
        L[(size_t)i * p + j] = fma(-L[(size_t)i * p + k], L[(size_t)j * p + k], L[(size_t)i * p + j]);
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    for (int j = tid; j < p; j += kLsarSolveThreads) phi[j] = nan("");
    if (tid == 0) {
      tau[lag - 1] = nan("");
      *status = lag;
    }
    return;
  }
  // phi = H^-1 h
  if (wid == 0) chol_solve_warp(L, rdiag, p, z);
  __syncthreads();
  for (int j = tid; j < p; j += kLsarSolveThreads) x[j] = z[j];
  __syncthreads();
  // corrected semi-normal equations: rw_k = w2_k (b_k - x_k . phi), g = sum_k rw_k x_k, phi += H^-1 g
  for (int k = wid; k < c; k += kWarps) {
    const long long i = rows[k];
    double s = 0.0;
    for (int j = lane; j < p; j += 32) s = fma(y[p + i - 1 - j], x[j], s);
    s = warp_sum(s);
    if (lane == 0) rw[k] = w2[k] * (y[p + i] - s);
  }
  __syncthreads();
  for (int j = lane; j < p; j += 32) {
    double g = 0.0;
    for (int k = wid; k < c; k += kWarps) g = fma(rw[k], y[p + rows[k] - 1 - j], g);
    wpart[wid * p + j] = g;
  }
  __syncthreads();
  for (int j = tid; j < p; j += kLsarSolveThreads) {
    double g = 0.0;
    for (int w = 0; w < kWarps; ++w) g += wpart[w * p + j];
    z[j] = g;
  }
  __syncthreads();
  if (wid == 0) chol_solve_warp(L, rdiag, p, z);
  __syncthreads();
  for (int j = tid; j < p; j += kLsarSolveThreads) phi[j] = x[j] + z[j];
  if (tid == 0) tau[lag - 1] = x[p - 1] + z[p - 1];
}

size_t lsar_solve_smem(int p) {
  return sizeof(double) * ((p <= kLsarSmemP ? (size_t)p * p : 0) + (size_t)(3 + kLsarSolveThreads / 32) * p);
}

size_t lsar_gram_smem(int p) { return sizeof(double) * 2 * kLsarChunk * (size_t)(p + 1); }

cudaError_t launch_lsar_lev(const double* r, const double* rr, double* lev, long long m, double* bsum,
                            const int* status, cudaStream_t s) {
  const long long nb = (m + kLsarBlock - 1) / kLsarBlock;
  lsar_lev_kernel<<<(unsigned)((nb + 7) / 8), 256, 0, s>>>(r, rr, lev, m, nb, bsum, status);
  return cudaGetLastError();
}

cudaError_t launch_lsar_prefix(const double* bsum, long long nb, double* bpre, const int* status, cudaStream_t s) {
  lsar_prefix_kernel<<<1, 1024, 0, s>>>(bsum, nb, bpre, status);
  return cudaGetLastError();
}

cudaError_t launch_lsar_sample(const double* lev, long long m, const double* bsum, const double* bpre,
                               const double* unif, int c, int p, long long* rows, double* w2, const int* status,
                               cudaStream_t s) {
  const long long nb = (m + kLsarBlock - 1) / kLsarBlock;
  lsar_sample_kernel<<<(unsigned)((c + 7) / 8), 256, 0, s>>>(lev, m, bsum, bpre, nb, unif, c, p, rows, w2, status);
  return cudaGetLastError();
}

cudaError_t launch_lsar_gram(const double* y, int p, const long long* rows, const double* w2, int c, int ng,
                             double* part, double* G, const int* status, cudaStream_t s) {
  const long long tri = lsar_tri(p);
  const int per_cta = (c + ng - 1) / ng;
  const size_t smem = lsar_gram_smem(p);
  cudaError_t e = cudaFuncSetAttribute(lsar_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  lsar_gram_kernel<<<ng, 256, smem, s>>>(y, p, rows, w2, c, per_cta, part, tri, status);
  const int rb = (int)((tri + 255) / 256);
  lsar_reduce_kernel<<<rb < 1 ? 1 : rb, 256, 0, s>>>(part, ng, tri, G, status);
  return cudaGetLastError();
}

cudaError_t launch_lsar_solve(const double* G, int p, const double* y, const long long* rows, const double* w2,
                              int c, double* Lg, double* rw, double* phi, double* tau, int lag, int* status,
                              cudaStream_t s) {
  const size_t smem = lsar_solve_smem(p);
  cudaError_t e = cudaFuncSetAttribute(lsar_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  lsar_solve_kernel<<<1, kLsarSolveThreads, smem, s>>>(G, p, y, rows, w2, c, Lg, rw, phi, tau, lag, status);
  return cudaGetLastError();
}

}  // namespace tols
