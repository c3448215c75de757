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
//   lsar_chol_kernel    one CTA: Cholesky H = L L^T of the sampled H = X^T W X, phi0 = H^-1 X^T W b;
//   lsar_refine_kernel  per-CTA partial of g = X^T W (b - X phi0) over the sampled rows;
//   lsar_correct_kernel one CTA: phi = phi0 + H^-1 g (one step of the corrected semi-normal equations).
// Every sum runs in a fixed order, so a sweep is bitwise reproducible. Rows with score 0 are never drawn.
//
// The same file holds Algorithm "Repeated Halving" (Section 3.2: rh_* kernels, which reuse the sampler, the Gram
// kernel and the Cholesky kernel above on the augmented matrix [b | X] of order p_bar) and Algorithm "SRHT"
// (Section 2.1: srht_* and fwht_* kernels, whose sampled rows go through the same Gram layout and Cholesky).
#include <math.h>

#include "tols_internal.cuh"

namespace tols {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Inclusive warp scan in a fixed order.
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

// lev[i] += r[i]^2 / ||r||^2 (r == nullptr: lev unchanged), then bsum[b] = the sum of block b's lev (a warp sum:
// the sampler's running sums inside a block may differ from it in the last bit, which its fallback covers).
// One warp per block of kLsarBlock rows.
__global__ void __launch_bounds__(256) lsar_lev_kernel(const double* __restrict__ r, const double* rr, double* lev,
                                                       long long m, long long nb, double* bsum, const int* status) {
  if (*status) return;
  const long long b = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (b >= nb) return;
  const int lane = threadIdx.x & 31;
  const double inv = r ? 1.0 / *rr : 0.0;
  const long long i0 = b * kLsarBlock;
  double s = 0.0;
#pragma unroll 4
  for (int ch = 0; ch < kLsarBlock / 32; ++ch) {
    const long long i = i0 + ch * 32 + lane;
    if (i < m) {
      double v = lev[i];
      if (r) {
        v = fma(r[i] * r[i], inv, v);
        lev[i] = v;
      }
      s += v;
    }
  }
  s = warp_sum(s);
  if (lane == 0) bsum[b] = s;
}

// bpre[b] = bsum[0] + ... + bsum[b-1], b <= nb (bpre[nb] is the total). One CTA of 1024 threads: thread t sums
// its contiguous segment of the block sums, a block scan of the segment sums gives each segment's offset, then
// each thread writes its segment's running sums.
__global__ void __launch_bounds__(1024) lsar_prefix_kernel(const double* __restrict__ bsum, long long nb,
                                                           double* bpre, const int* status) {
  if (*status) return;
  __shared__ double s_warp[32];
  __shared__ double s_tot;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const long long seg = (nb + 1023) / 1024;
  const long long j0 = (long long)tid * seg;
  const long long j1 = j0 + seg < nb ? j0 + seg : nb;
  double s = 0.0;
  for (long long j = j0; j < j1; ++j) s += bsum[j];
  const double incl = warp_incl_scan(s);
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
  double run = (lane ? within : 0.0) + s_warp[wid];
  for (long long j = j0; j < j1; ++j) {
    bpre[j] = run;
    run += bsum[j];
  }
  if (tid == 0) bpre[nb] = s_tot;
}

// Draw k (one warp): t = unif[k] * total; the row is the first i whose running sum exceeds t, or, if rounding
// leaves none, the last row with a positive score. rows[k] = i, w2[k] = p / (c lev[i]) = 1 / (c pi_i); with
// p = 0 the scores are normalised by their sum instead, w2[k] = sum(lev) / (c lev[i]).
// The running sums are formed block prefix + lane-segment prefix + rows within the segment; they may differ
// from a plain left-to-right sum in the last bits, which matters only for a t within rounding of a boundary.
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
  // inside block b: lane l holds rows [i0 + 16 l, i0 + 16 l + 16); the crossing lane is the first whose running
  // sum exceeds t, and it walks its own rows
  constexpr int kSeg = kLsarBlock / 32;
  const long long s0 = b * kLsarBlock + (long long)lane * kSeg;
  double seg = 0.0;
  long long my_pos = -1;
#pragma unroll
  for (int r = 0; r < kSeg; ++r) {
    const long long i = s0 + r;
    const double v = i < m ? lev[i] : 0.0;
    seg += v;
    if (v > 0.0) my_pos = i;
  }
  const double incl = warp_incl_scan(seg);
  const double up = __shfl_up_sync(kFull, incl, 1);   // every lane takes part in the shuffle
  const double excl = lane ? up : 0.0;
  const unsigned hit = __ballot_sync(kFull, base + incl > t);
  long long pick = -1, last_pos = -1;
  if (hit) {
    const int L = __ffs((int)hit) - 1;
    if (lane == L) {
      double run = excl;
      for (int r = 0; r < kSeg && pick < 0; ++r) {
        const long long i = s0 + r;
        const double v = i < m ? lev[i] : 0.0;
        run += v;
        if (v > 0.0 && base + run > t) pick = i;
      }
      if (pick < 0) pick = my_pos;
    }
    pick = __shfl_sync(kFull, pick, L);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const long long other = __shfl_xor_sync(kFull, my_pos, o);
    my_pos = other > my_pos ? other : my_pos;
  }
  last_pos = my_pos;
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
  if (pick >= m) pick = m - 1;   // cannot happen; keeps every later read of y and lev in bounds
  if (lane == 0) {
    rows[k] = pick;
    w2[k] = (p > 0 ? (double)p : bpre[nb]) / ((double)c * lev[pick]);
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

// G[e] = the sum over the ng partials, in a fixed order: eight running sums over g = u mod 8, then combined
// pairwise (independent accumulators keep eight loads in flight).
__global__ void lsar_reduce_kernel(const double* __restrict__ part, int ng, long long tri, double* G,
                                   const int* status) {
  if (*status) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tri; e += (long long)gridDim.x * blockDim.x) {
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int g = 0;
    for (; g + 8 <= ng; g += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] += part[(size_t)(g + u) * tri + e];
    }
    for (int u = 0; g < ng; ++g, ++u) acc[u] += part[(size_t)g * tri + e];
    G[e] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  }
}

namespace {

// w := L^-1 h (h is overwritten), then x := L^-T w, for L lower triangular (row-major, leading dimension p) with
// reciprocal diagonal rdiag. The first four warps (one per SM sub-partition) do the work with one named barrier
// per step; the others wait at the closing __syncthreads. Callers have h, L, rdiag in place before it
// (visible to the first four warps through a __syncthreads).
__device__ void chol_solve_cta(const double* L, const double* rdiag, int p, double* h, double* w, double* x) {
  const int tid = threadIdx.x;
  if (tid < 128) {
    for (int k = 0; k < p; ++k) {
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const double zk = h[k] * rdiag[k];
      if (tid == 0) w[k] = zk;
      for (int i = k + 1 + tid; i < p; i += 128) h[i] = fma(-L[(size_t)i * p + k], zk, h[i]);
    }
    for (int k = p - 1; k >= 0; --k) {
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const double xk = w[k] * rdiag[k];
      if (tid == 0) x[k] = xk;
      for (int i = tid; i < k; i += 128) w[i] = fma(-L[(size_t)k * p + i], xk, w[i]);
    }
  }
  __syncthreads();
}

}  // namespace

// One CTA of kLsarSolveThreads. H[j][l] = G[e(1 + j, 1 + l)] (the sampled X^T W X), h[j] = G[e(0, 1 + j)]
// (X^T W b). Right-looking Cholesky H = L L^T with one barrier per step k: warps 1.. update their rows
// i >= k + 2 of the trailing triangle from a contiguous copy of column k (cur), write their rows of column k
// scaled, and copy the updated column k + 1 to the other buffer (nxt); meanwhile thread 0 updates the next
// pivot, entry (k + 1, k + 1), and forms its reciprocal square root. L works in shared memory when
// p <= kLsarSmemP, else in place in Lg. Writes L and its reciprocal diagonal to Lg, rdg (for
// lsar_correct_kernel) and, when phi is given, phi0 = H^-1 h to phi. off = 0 factors the whole augmented
// matrix instead (H[j][l] = G[e(j, l)], p = its order; Repeated Halving's B^T B). A pivot that is not positive
// and finite makes phi and tau[lag - 1] NaN (when given) and sets *status = lag, which skips every later
// kernel of the sweep.
__global__ void __launch_bounds__(kLsarSolveThreads, 1) lsar_chol_kernel(const double* __restrict__ G, int p,
                                                                         int off, double* Lg, double* rdg,
                                                                         double* phi, double* tau, int lag,
                                                                         int* status) {
  if (*status) return;
  extern __shared__ double lsm[];
  __shared__ int s_fail;
  __shared__ double s_piv[2][2];   // per step parity: 1/sqrt(d), 1/d
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int kWarps = kLsarSolveThreads / 32;
  const bool in_smem = p <= kLsarSmemP;
  double* L = in_smem ? lsm : Lg;
  double* v = lsm + (in_smem ? (size_t)p * p : 0);
  double* h = v + 2 * p;
  double* w = v + 3 * p;
  double* x = v + 4 * p;
  double* rdiag = v + 5 * p;
  for (int idx = tid; idx < p * p; idx += kLsarSolveThreads) {
    const int i = idx / p, j = idx - i * p;
    L[idx] = j <= i ? G[tri_index(off + j, off + i)] : 0.0;
  }
  for (int j = tid; j < p; j += kLsarSolveThreads) {
    if (phi) h[j] = G[tri_index(0, 1 + j)];
    v[j] = G[tri_index(off, off + j)];   // column 0 of H, the first column buffer
  }
  if (tid == 0) {
    const double d = G[tri_index(off, off)];
    s_fail = !(d > 0.0) || !isfinite(d);
    if (!s_fail) {
      const double r = rsqrt_newton(d);
      s_piv[0][0] = r;
      s_piv[0][1] = r * r;
      rdiag[0] = r;
    }
  }
  __syncthreads();
  if (tid == 0 && !s_fail) L[0] = G[tri_index(off, off)] * s_piv[0][0];
  for (int k = 0; k < p && !s_fail; ++k) {
    const double r = s_piv[k & 1][0], r2 = s_piv[k & 1][1];
    const double* cur = v + (k & 1) * p;   // column buffers: v[0, p) and v[p, 2p)
    double* nxt = v + ((k + 1) & 1) * p;
    if (wid == 0) {
      if (tid == 0 && k + 1 < p) {
        L[(size_t)(k + 1) * p + k] = cur[k + 1] * r;
        const double d = fma(-cur[k + 1] * r2, cur[k + 1], L[(size_t)(k + 1) * p + k + 1]);
        if (!(d > 0.0) || !isfinite(d)) {
          s_fail = 1;
        } else {
          const double rn = rsqrt_newton(d);
          s_piv[(k + 1) & 1][0] = rn;
          s_piv[(k + 1) & 1][1] = rn * rn;
          rdiag[k + 1] = rn;
          L[(size_t)(k + 1) * p + k + 1] = d * rn;
        }
      }
    } else {
      for (int i = k + 2 + (wid - 1); i < p; i += kWarps - 1) {
        const double ci = cur[i] * r2;
        for (int j = k + 1 + lane; j <= i; j += 32) {
          const double nv = fma(-ci, cur[j], L[(size_t)i * p + j]);
          L[(size_t)i * p + j] = nv;
          if (j == k + 1) nxt[i] = nv;
        }
        if (lane == 0) L[(size_t)i * p + k] = cur[i] * r;
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (phi)
      for (int j = tid; j < p; j += kLsarSolveThreads) phi[j] = nan("");
    if (tid == 0) {
      if (tau) tau[lag - 1] = nan("");
      *status = lag;
    }
    return;
  }
  if (phi) {
    chol_solve_cta(L, rdiag, p, h, w, x);
    for (int j = tid; j < p; j += kLsarSolveThreads) phi[j] = x[j];
  }
  for (int j = tid; j < p; j += kLsarSolveThreads) rdg[j] = rdiag[j];
  if (in_smem)
    for (int idx = tid; idx < p * p; idx += kLsarSolveThreads) Lg[idx] = L[idx];
}

// CTA g and its draws k (one warp each): rho_k = b_k - x_k . phi0, gpart[g][j] = sum_k w2_k rho_k x_k[j]
// (x_k[j] = y[p + rows[k] - 1 - j], b_k = y[p + rows[k]]).
__global__ void __launch_bounds__(256) lsar_refine_kernel(const double* __restrict__ y, int p,
                                                          const long long* __restrict__ rows,
                                                          const double* __restrict__ w2, int c, int per_cta,
                                                          const double* __restrict__ phi0, double* gpart,
                                                          const int* status) {
  if (*status) return;
  extern __shared__ double lsm[];
  double* ph = lsm;
  double* gw = lsm + p;   // 8 x p, one row per warp
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int j = tid; j < p; j += 256) ph[j] = phi0[j];
  for (int j = tid; j < 8 * p; j += 256) gw[j] = 0.0;
  __syncthreads();
  const int k0 = blockIdx.x * per_cta;
  const int k1 = min(c, k0 + per_cta);
  for (int k = k0 + wid; k < k1; k += 8) {
    const double* xr = y + p + rows[k] - 1;
    double s = 0.0;
    for (int j = lane; j < p; j += 32) s = fma(xr[-j], ph[j], s);
    s = warp_sum(s);
    const double rho = w2[k] * (xr[1] - s);
    for (int j = lane; j < p; j += 32) gw[wid * p + j] = fma(rho, xr[-j], gw[wid * p + j]);
  }
  __syncthreads();
  for (int j = tid; j < p; j += 256) {
    double g = 0.0;
    for (int q = 0; q < 8; ++q) g += gw[q * p + j];
    gpart[(size_t)blockIdx.x * p + j] = g;
  }
}

// One CTA of kLsarSolveThreads: g = the sum of the ng partials in CTA order, then phi += H^-1 g with the factor of
// lsar_chol_kernel (Lg, rdg); tau[lag - 1] = phi[p - 1].
__global__ void __launch_bounds__(kLsarSolveThreads, 1) lsar_correct_kernel(const double* __restrict__ Lg,
                                                                            const double* __restrict__ rdg, int p,
                                                                            const double* __restrict__ gpart, int ng,
                                                                            double* phi, double* tau, int lag,
                                                                            const int* status) {
  if (*status) return;
  extern __shared__ double lsm[];
  const int tid = threadIdx.x;
  const bool in_smem = p <= kLsarSmemP;
  double* Ls = lsm;
  double* v = lsm + (in_smem ? (size_t)p * p : 0);
  double* h = v;
  double* w = v + p;
  double* x = v + 2 * p;
  double* rdiag = v + 3 * p;
  double* red = v + 4 * p;   // kLsarSolveThreads
  if (in_smem)
    for (int idx = tid; idx < p * p; idx += kLsarSolveThreads) Ls[idx] = Lg[idx];
  for (int j = tid; j < p; j += kLsarSolveThreads) rdiag[j] = rdg[j];
  const int S = kLsarSolveThreads / p > 1 ? kLsarSolveThreads / p : 1;
  for (int t = tid; t < S * p; t += kLsarSolveThreads) {
    const int s = t / p, j = t - s * p;
    double acc = 0.0;
    for (int g = s; g < ng; g += S) acc += gpart[(size_t)g * p + j];
    red[t] = acc;
  }
  __syncthreads();
  for (int j = tid; j < p; j += kLsarSolveThreads) {
    double acc = 0.0;
    for (int s = 0; s < S; ++s) acc += red[s * p + j];
    h[j] = acc;
  }
  __syncthreads();
  chol_solve_cta(in_smem ? Ls : Lg, rdiag, p, h, w, x);
  for (int j = tid; j < p; j += kLsarSolveThreads) {
    const double v2 = phi[j] + x[j];
    phi[j] = v2;
    if (j == p - 1) tau[lag - 1] = v2;
  }
}

size_t lsar_chol_smem(int p) { return sizeof(double) * ((p <= kLsarSmemP ? (size_t)p * p : 0) + 6 * (size_t)p); }
size_t lsar_correct_smem(int p) {
  return sizeof(double) * ((p <= kLsarSmemP ? (size_t)p * p : 0) + 4 * (size_t)p + kLsarSolveThreads);
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
  const int rb = (int)((tri + 63) / 64);
  lsar_reduce_kernel<<<rb < 1 ? 1 : rb, 64, 0, s>>>(part, ng, tri, G, status);
  return cudaGetLastError();
}

cudaError_t launch_lsar_solve(const double* G, int p, const double* y, const long long* rows, const double* w2,
                              int c, int ng, double* Lg, double* rdg, double* gpart, double* phi, double* tau,
                              int lag, int* status, cudaStream_t s) {
  size_t smem = lsar_chol_smem(p);
  cudaError_t e = cudaFuncSetAttribute(lsar_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  lsar_chol_kernel<<<1, kLsarSolveThreads, smem, s>>>(G, p, 1, Lg, rdg, phi, tau, lag, status);
  const int per_cta = (c + ng - 1) / ng;
  lsar_refine_kernel<<<ng, 256, sizeof(double) * 9 * (size_t)p, s>>>(y, p, rows, w2, c, per_cta, phi, gpart, status);
  smem = lsar_correct_smem(p);
  e = cudaFuncSetAttribute(lsar_correct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  lsar_correct_kernel<<<1, kLsarSolveThreads, smem, s>>>(Lg, rdg, p, gpart, ng, phi, tau, lag, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------------
// Algorithm "Repeated Halving" (Section 3.2) on [X | b] of order pb (rows a_i[q] = y[pb + i - q], q <= pb, the
// augmented row order of the Gram kernel above; a column permutation changes no leverage score).

// out[e] = (in ? in[keep[e]] : keep[e]), e < cnt: the original rows of the next halving level.
__global__ void rh_map_kernel(const long long* __restrict__ in, const long long* __restrict__ keep, long long cnt,
                              long long* out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.x * blockDim.x)
    out[e] = in ? in[keep[e]] : keep[e];
}

__global__ void rh_fill_kernel(double* x, long long cnt, double v) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.x * blockDim.x)
    x[e] = v;
}

// CTA t: row t of M = S B (B^T B)^-1, eq. (glev), with B's rows sqrt(w2_r) a_{rows[r]} (r < cnt), S the k x cnt
// sketch (row-major) and B^T B = L L^T from lsar_chol_kernel (Lg, rdg; order P1 = pb + 1): first
// h = B^T S(t,:)^T, then M(t,:) = (L L^T)^-1 h.
__global__ void __launch_bounds__(kLsarSolveThreads, 1) rh_sketch_kernel(
    const double* __restrict__ y, int P1, const long long* __restrict__ rows, const double* __restrict__ w2, int cnt,
    const double* __restrict__ S, const double* __restrict__ Lg, const double* __restrict__ rdg, double* M,
    const int* status) {
  if (*status) return;
  extern __shared__ double lsm[];
  const int tid = threadIdx.x, t = blockIdx.x, pb = P1 - 1;
  const bool in_smem = P1 <= kLsarSmemP;
  double* Ls = lsm;
  double* v = lsm + (in_smem ? (size_t)P1 * P1 : 0);
  double* h = v;
  double* w = v + P1;
  double* x = v + 2 * P1;
  double* rdiag = v + 3 * P1;
  double* coef = v + 4 * P1;                                   // kLsarSolveThreads
  long long* rr = reinterpret_cast<long long*>(coef + kLsarSolveThreads);   // kLsarSolveThreads
  double acc = 0.0;                                            // h[q] for q = tid (tid < P1)
  for (int r0 = 0; r0 < cnt; r0 += kLsarSolveThreads) {
    const int nr = min(kLsarSolveThreads, cnt - r0);
    __syncthreads();
    if (tid < nr) {
      coef[tid] = S[(size_t)t * cnt + r0 + tid] * sqrt(w2[r0 + tid]);
      rr[tid] = rows[r0 + tid];
    }
    __syncthreads();
    if (tid < P1)
      for (int r = 0; r < nr; ++r) acc = fma(coef[r], y[pb + rr[r] - tid], acc);
  }
  if (tid < P1) h[tid] = acc;
  if (in_smem)
    for (int idx = tid; idx < P1 * P1; idx += kLsarSolveThreads) Ls[idx] = Lg[idx];
  for (int j = tid; j < P1; j += kLsarSolveThreads) rdiag[j] = rdg[j];
  __syncthreads();
  chol_solve_cta(in_smem ? Ls : Lg, rdiag, P1, h, w, x);
  for (int j = tid; j < P1; j += kLsarSolveThreads) M[(size_t)t * P1 + j] = x[j];
}

// score[e] = ||M a_i||^2, eq. (glev), for the row i = (list ? list[e] : e) of a halving level, e < cnt
// (M: k x P1 in shared memory).
__global__ void __launch_bounds__(256) rh_score_kernel(const double* __restrict__ y, int P1,
                                                       const double* __restrict__ M, int k,
                                                       const long long* __restrict__ list, long long cnt,
                                                       double* score, const int* status) {
  if (*status) return;
  extern __shared__ double lsm[];
  for (int idx = threadIdx.x; idx < k * P1; idx += blockDim.x) lsm[idx] = M[idx];
  __syncthreads();
  const int pb = P1 - 1;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.x * blockDim.x) {
    const long long i = list ? list[e] : e;
    const double* base = y + pb + i;
    double sc = 0.0;
    for (int t = 0; t < k; ++t) {
      const double* mt = lsm + t * P1;
      double s = 0.0;
      for (int q = 0; q < P1; ++q) s = fma(mt[q], base[-q], s);
      sc = fma(s, s, sc);
    }
    score[e] = sc;
  }
}

size_t rh_sketch_smem(int P1) {
  return sizeof(double) * ((P1 <= kLsarSmemP ? (size_t)P1 * P1 : 0) + 4 * (size_t)P1 + 2 * kLsarSolveThreads);
}

cudaError_t launch_rh_map(const long long* in, const long long* keep, long long cnt, long long* out,
                          cudaStream_t s) {
  const long long b = (cnt + 255) / 256;
  rh_map_kernel<<<(unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b)), 256, 0, s>>>(in, keep, cnt, out);
  return cudaGetLastError();
}

cudaError_t launch_rh_fill(double* x, long long cnt, double v, cudaStream_t s) {
  const long long b = (cnt + 255) / 256;
  rh_fill_kernel<<<(unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b)), 256, 0, s>>>(x, cnt, v);
  return cudaGetLastError();
}

cudaError_t launch_rh_factor(const double* G, int P1, double* Lg, double* rdg, int code, int* status,
                             cudaStream_t s) {
  const size_t smem = lsar_chol_smem(P1);
  cudaError_t e = cudaFuncSetAttribute(lsar_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  lsar_chol_kernel<<<1, kLsarSolveThreads, smem, s>>>(G, P1, 0, Lg, rdg, nullptr, nullptr, code, status);
  return cudaGetLastError();
}

cudaError_t launch_rh_sketch(const double* y, int P1, const long long* rows, const double* w2, int cnt,
                             const double* S, int k, const double* Lg, const double* rdg, double* M, int* status,
                             cudaStream_t s) {
  const size_t smem = rh_sketch_smem(P1);
  cudaError_t e = cudaFuncSetAttribute(rh_sketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  rh_sketch_kernel<<<k, kLsarSolveThreads, smem, s>>>(y, P1, rows, w2, cnt, S, Lg, rdg, M, status);
  return cudaGetLastError();
}

cudaError_t launch_rh_score(const double* y, int P1, const double* M, int k, const long long* list, long long cnt,
                            double* score, const int* status, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)k * P1;
  cudaError_t e = cudaFuncSetAttribute(rh_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long b = (cnt + 255) / 256;
  rh_score_kernel<<<(unsigned)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b)), 256, smem, s>>>(y, P1, M, k, list, cnt,
                                                                                         score, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------------
// Algorithm "SRHT" (Section 2.1, eq. (SRHT)) for the order-p problem: Z = H D [X | b] with the m rows zero-padded to
// m2 = 2^k (column-major, column j < p holds X(:, j), column p holds b), then the c sampled rows scaled by
// sqrt(m2 / c) go through the Gram kernel's layout (augmented order: b first) to lsar_chol_kernel.

// Z[j m2 + i] = signs[i] * (i < m ? C(i, j) : 0).
__global__ void srht_form_kernel(const double* __restrict__ y, int p, long long m, long long m2,
                                 const double* __restrict__ signs, double* Z) {
  const long long total = (long long)(p + 1) * m2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long j = e / m2, i = e - j * m2;
    double v = 0.0;
    if (i < m) v = j < p ? y[p - 1 + i - j] : y[p + i];
    Z[e] = signs[i] * v;
  }
}

// The Hadamard stages h = 1 .. blk/2 of Def. "Hadamard Transform" on chunks of blk entries (a power of two
// dividing m2), in shared memory: (a, b) -> ((a + b) / sqrt 2, (a - b) / sqrt 2) for the pairs (i, i + h) of
// every 2h-block.
__global__ void __launch_bounds__(256) fwht_block_kernel(double* Z, int lblk) {
  extern __shared__ double lsm[];
  const int blk = 1 << lblk;
  double* z = Z + (size_t)blockIdx.x * blk;
  for (int i = threadIdx.x; i < blk; i += blockDim.x) lsm[i] = z[i];
  const double s = 1.0 / sqrt(2.0);   // square root and quotient each rounded to double
  for (int lh = 0; lh < lblk; ++lh) {
    __syncthreads();
    const int h = 1 << lh;
    for (int t = threadIdx.x; t < blk / 2; t += blockDim.x) {
      const int i = ((t >> lh) << (lh + 1)) + (t & (h - 1));
      const double a = lsm[i], b = lsm[i + h];
      lsm[i] = (a + b) * s;
      lsm[i + h] = (a - b) * s;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < blk; i += blockDim.x) z[i] = lsm[i];
}

// One Hadamard stage with pair distance h = 2^lh over every column of length m2.
__global__ void fwht_stage_kernel(double* Z, int cols, long long m2, int lh) {
  const long long half = m2 / 2, total = (long long)cols * half, h = 1LL << lh;
  const double s = 1.0 / sqrt(2.0);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long col = t / half, tt = t - col * half;
    const long long i = col * m2 + ((tt >> lh) << (lh + 1)) + (tt & (h - 1));
    const double a = Z[i], b = Z[i + h];
    Z[i] = (a + b) * s;
    Z[i + h] = (a - b) * s;
  }
}

// CTA g: part[g][e(q, q2)] = sum over its draws k of a_k[q] a_k[q2], a_k = sc (Z(rows[k], p), Z(rows[k], 0 .. p-1)).
// A row index outside [0, m2) sets *status = -1 and reads row 0 instead.
__global__ void __launch_bounds__(256) srht_gram_kernel(const double* __restrict__ Z, long long m2, int p,
                                                        const long long* __restrict__ rows, int c, double sc,
                                                        int per_cta, double* part, long long tri, int* status) {
  extern __shared__ double lsm[];
  const int P1 = p + 1;
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
      long long r = rows[kc + kk];
      if (r < 0 || r >= m2) {
        *status = -1;
        r = 0;
      }
      const int col = q == 0 ? p : q - 1;
      lsm[kk * P1 + q] = sc * Z[(size_t)col * m2 + r];
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < tri; e += blockDim.x) {
      int q, q2;
      tri_unpack(e, q, q2);
      double acc = kc == k0 ? 0.0 : out[e];
      for (int kk = 0; kk < cnt; ++kk) acc = fma(lsm[kk * P1 + q], lsm[kk * P1 + q2], acc);
      out[e] = acc;
    }
  }
}

cudaError_t launch_srht_transform(const double* y, int p, long long m, long long m2, const double* signs, double* Z,
                                  cudaStream_t s) {
  const long long total = (long long)(p + 1) * m2;
  const long long b = (total + 255) / 256;
  srht_form_kernel<<<(unsigned)(b > 152 * 32 ? 152 * 32 : b), 256, 0, s>>>(y, p, m, m2, signs, Z);
  int lm2 = 0;
  while ((1LL << lm2) < m2) ++lm2;
  const int lblk = lm2 < 12 ? lm2 : 12;   // chunks of up to 4,096 entries in shared memory
  if (lblk > 0) {
    const size_t smem = sizeof(double) * ((size_t)1 << lblk);
    cudaError_t e = cudaFuncSetAttribute(fwht_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fwht_block_kernel<<<(unsigned)(total >> lblk), 256, smem, s>>>(Z, lblk);
  }
  for (int lh = lblk; lh < lm2; ++lh) {
    const long long half = total / 2;
    const long long bb = (half + 255) / 256;
    fwht_stage_kernel<<<(unsigned)(bb > 152 * 32 ? 152 * 32 : bb), 256, 0, s>>>(Z, p + 1, m2, lh);
  }
  return cudaGetLastError();
}

cudaError_t launch_srht_gram(const double* Z, long long m2, int p, const long long* rows, int c, double sc, int ng,
                             double* part, double* G, int* status, cudaStream_t s) {
  const long long tri = lsar_tri(p);
  const int per_cta = (c + ng - 1) / ng;
  const size_t smem = sizeof(double) * kLsarChunk * (size_t)(p + 1);
  srht_gram_kernel<<<ng, 256, smem, s>>>(Z, m2, p, rows, c, sc, per_cta, part, tri, status);
  const int rb = (int)((tri + 63) / 64);
  lsar_reduce_kernel<<<rb < 1 ? 1 : rb, 64, 0, s>>>(part, ng, tri, G, status);
  return cudaGetLastError();
}

cudaError_t launch_srht_solve(const double* G, int p, double* Lg, double* rdg, double* phi, int* status,
                              cudaStream_t s) {
  const size_t smem = lsar_chol_smem(p);
  cudaError_t e = cudaFuncSetAttribute(lsar_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  lsar_chol_kernel<<<1, kLsarSolveThreads, smem, s>>>(G, p, 1, Lg, rdg, phi, nullptr, 1, status);
  return cudaGetLastError();
}

}  // namespace tols
