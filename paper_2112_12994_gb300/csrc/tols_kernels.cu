// Kernels of the Toeplitz-OLS solver for sm_103a.
//
// One "pass" kernel carries the whole per-iteration hot path of LSQR on the structured matrix of
// eq. (xphi), Section 3 (X[i][j] = y[p+i-j-1], b[i] = y[p+i]):
//
//   u_new = X d - c * u_old        sliding-window dot products over a shared-memory tile of y
//   ||u_new||^2                    float64 accumulation
//   X^T u_new                      lag correlations of the fresh u tile against the same y tile
//
// so one iteration reads y once, reads u_old once and writes u_new once. The last CTA to finish (found with
// an atomic counter, no spinning) reduces the per-CTA partials in a fixed order and runs the scalar step of
// the solver (LSQR recurrence, correction solve or residual check) on the device, so the host never waits
// per iteration. FP64 products run in double; the mixed path runs the products in float with float64
// accumulation of every norm and every cross-tile sum.
#include <math.h>
#include <stdio.h>

#include <map>
#include <mutex>
#include <utility>

#include "tols_internal.cuh"

namespace tols {

__host__ __device__ inline long long lmin(long long a, long long b) { return a < b ? a : b; }

// Let a kernel launch with `bytes` of dynamic shared memory on the current device: its limit (at first the
// default, 48 KB less its static shared memory) is raised when needed, never lowered, since a launch is valid for
// any size up to the limit. The attribute belongs to the device, so the limit is recorded per (device, kernel);
// several host threads may call this.
cudaError_t smem_opt_in(const void* fn, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> limit;
  std::lock_guard<std::mutex> lock(mu);
  auto it = limit.find(std::make_pair(dev, fn));
  if (it == limit.end()) {
    cudaFuncAttributes attr;
    e = cudaFuncGetAttributes(&attr, fn);
    if (e != cudaSuccess) return e;
    it = limit.emplace(std::make_pair(dev, fn), attr.maxDynamicSharedSizeBytes).first;
  }
  int& cur = it->second;
  if (cur >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// ------------------------------------------------------------------------------------------------------
// shared-memory layout of the y window: 4 pad elements after every 16, so that 16-B vector loads by lanes
// 16 elements apart hit distinct banks.
__device__ __forceinline__ int phys(int i) { return i + ((i >> 4) << 2); }
__host__ __device__ inline int phys_size(int n) { return n + ((n + 15) >> 4) * 4 + 4; }

template <typename T>
struct TileCfg;
template <>
struct TileCfg<float> {
  static constexpr int RB = 16;    // consecutive rows per thread
  static constexpr int KC = 8;     // lags per inner step
  static constexpr int TILE = kThreads * RB;
  static constexpr int MINB = 3;   // resident CTAs per SM the register budget aims at
};
template <>
struct TileCfg<double> {
  static constexpr int RB = 8;
  static constexpr int KC = 8;
  static constexpr int TILE = kThreads * RB;
  static constexpr int MINB = 2;
};

template <typename T>
__device__ __forceinline__ void lds4(const T* s, int i, T* out);
template <>
__device__ __forceinline__ void lds4<float>(const float* s, int i, float* out) {
  float4 v = *reinterpret_cast<const float4*>(s + phys(i));
  out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <>
__device__ __forceinline__ void lds4<double>(const double* s, int i, double* out) {
  const double2* q = reinterpret_cast<const double2*>(s + phys(i));
  double2 a = q[0], b = q[1];
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}

template <typename T>
__device__ __forceinline__ void st4(T* g, const T* v);
template <>
__device__ __forceinline__ void st4<float>(float* g, const float* v) {
  *reinterpret_cast<float4*>(g) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st4<double>(double* g, const double* v) {
  reinterpret_cast<double2*>(g)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(g)[1] = make_double2(v[2], v[3]);
}

// Sum 8 values over the 32 lanes of a warp, scattered: afterwards every lane holds the full sum of value
// j = 4 [lane & 16] + 2 [lane & 8] + [lane & 4]. Fixed butterfly order, so the result is deterministic.
template <typename T>
__device__ __forceinline__ T warp_reduce_scatter8(const T* t, int lane) {
  const unsigned full = 0xffffffffu;
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  T a4[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const T keep = h16 ? t[4 + i] : t[i];
    const T send = h16 ? t[i] : t[4 + i];
    a4[i] = keep + __shfl_xor_sync(full, send, 16);
  }
  T a2[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const T keep = h8 ? a4[2 + i] : a4[i];
    const T send = h8 ? a4[i] : a4[2 + i];
    a2[i] = keep + __shfl_xor_sync(full, send, 8);
  }
  T a1 = (h4 ? a2[1] : a2[0]) + __shfl_xor_sync(full, h4 ? a2[0] : a2[1], 4);
  a1 += __shfl_xor_sync(full, a1, 2);
  a1 += __shfl_xor_sync(full, a1, 1);
  return a1;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the 256 threads of a CTA; every thread gets the result. scratch: >= 8 doubles of shared memory.
template <int NT = kThreads>
__device__ double block_sum(double v, double* scratch) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int k = 0; k < NT / 32; ++k) r += scratch[k];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------------------------------------------
// Preconditioner applications on p-vectors (M = R^{-1} upper triangular, Mt = M^T, both row-major).
// out = M^T in : out[j] = sum_{i<=j} M[i][j] in[i]
__device__ void apply_Mt(const Work& w, int precond, int mixed, const double* in, double* out) {
  const int p = w.p;
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    if (!precond) { out[j] = in[j]; continue; }
    if (mixed) {
      float acc = 0.f;
      for (int i = 0; i <= j; ++i) acc = fmaf(w.M32[(size_t)i * p + j], (float)in[i], acc);
      out[j] = acc;
    } else {
      double acc = 0.0;
      for (int i = 0; i <= j; ++i) acc = fma(w.M[(size_t)i * p + j], in[i], acc);
      out[j] = acc;
    }
  }
}
// out = M in : out[i] = sum_{j>=i} M[i][j] in[j] = sum_{j>=i} Mt[j][i] in[j]
__device__ void apply_M(const Work& w, int precond, int mixed, const double* in, double* out) {
  const int p = w.p;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    if (!precond) { out[i] = in[i]; continue; }
    if (mixed) {
      float acc = 0.f;
      for (int j = i; j < p; ++j) acc = fmaf(w.Mt32[(size_t)j * p + i], (float)in[j], acc);
      out[i] = acc;
    } else {
      double acc = 0.0;
      for (int j = i; j < p; ++j) acc = fma(w.Mt[(size_t)j * p + i], in[j], acc);
      out[i] = acc;
    }
  }
}
// out = M in with float64 arithmetic on whatever M the solve uses (float-rounded M in the mixed path).
__device__ void apply_M_exact(const Work& w, int precond, int mixed, const double* in, double* out) {
  const int p = w.p;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    if (!precond) { out[i] = in[i]; continue; }
    double acc = 0.0;
    for (int j = i; j < p; ++j)
      acc = fma(mixed ? (double)w.Mt32[(size_t)j * p + i] : w.Mt[(size_t)j * p + i], in[j], acc);
    out[i] = acc;
  }
}

__device__ double vec_norm2(const double* a, int p, double* scratch) {
  double s = 0.0;
  for (int j = threadIdx.x; j < p; j += blockDim.x) s += a[j] * a[j];
  return block_sum(s, scratch);
}

// ------------------------------------------------------------------------------------------------------
// Solver tails. Run by the last CTA of a pass with tk[k] = sum_i u_new[i] y[i+k] (k in [0, nlag)) in shared
// memory and n2 = ||u_new||^2. They update DevState and the p-vectors for the next launch.

// An inner solve (LSQR or the correction solve) stops when its stopping estimate has not halved for this many
// iterations: it has reached what the arithmetic (or the preconditioner) lets it reach, and the float64 check
// decides what comes next.
constexpr int kStallIters = 20;
// With the sampled-QR preconditioner kappa(X R^{-1}) is a small constant (about 3): a sweep that has not
// converged in this many iterations has met the limit of float64 arithmetic (kappa(X) u ~ 1).
constexpr int kQrIterCap = 100;

// After LSQR or the correction solve has finished: the next pass is a float64 residual check with
// d = -phi and u_old = b, c = -1, so that u_new = b - X phi.
__device__ void schedule_check(const Work& w, DevState* st, double* scratch) {
  for (int j = threadIdx.x; j < w.p; j += blockDim.x) w.d[j] = -w.phi[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    st->phase = PH_CHECK;
    st->coef = -1.0;
  }
}

// Start (or restart) LSQR on  min || A z - rhs ||,  A = X M, with beta1 = ||rhs|| and g = X^T rhs given.
// The correction M z is added to phi when LSQR stops.
__device__ void start_lsqr(const Work& w, DevState* st, const double* g, double beta1, double* scratch) {
  const int p = w.p;
  const int mixed = st->mixed;
  double* tmp = w.t;
  for (int j = threadIdx.x; j < p; j += blockDim.x) tmp[j] = beta1 > 0 ? g[j] / beta1 : 0.0;
  __syncthreads();
  apply_Mt(w, st->precond, mixed, tmp, w.v);
  __syncthreads();
  double alpha = sqrt(vec_norm2(w.v, p, scratch));
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    double vj = alpha > 0 ? w.v[j] / alpha : 0.0;
    w.v[j] = vj;
    w.w[j] = vj;
    w.z[j] = 0.0;
  }
  __syncthreads();
  apply_M(w, st->precond, mixed, w.v, w.d);
  __syncthreads();
  if (threadIdx.x == 0) {
    st->alpha = alpha;
    st->beta = beta1;
    st->beta1 = beta1;
    st->phibar = beta1;
    st->rhobar = alpha;
    st->anorm2 = 0.0;
    st->iter = 0;
    st->est_best = 1e300;
    st->iter_best = 0;
    st->phibar_mark = beta1;
    st->coef = beta1 > 0 ? alpha / beta1 : 0.0;
    st->phase = PH_LSQR;
  }
  __syncthreads();
  if (beta1 == 0.0 || alpha == 0.0) {
    // X^T rhs = 0: the correction is zero; go straight to the check.
    schedule_check(w, st, scratch);
  }
}

// Start the normal-equation correction solve (A^T A) zeta = M^T g, A = X M, by Golub-Kahan Bidiag 2.
__device__ void start_necorr(const Work& w, DevState* st, double* scratch) {
  const int p = w.p;
  apply_Mt(w, st->precond, 1, w.g, w.v);
  __syncthreads();
  double theta1 = sqrt(vec_norm2(w.v, p, scratch));
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    w.v[j] = theta1 > 0 ? w.v[j] / theta1 : 0.0;
    w.w[j] = 0.0;
    w.z[j] = 0.0;
  }
  __syncthreads();
  apply_M(w, st->precond, 1, w.v, w.d);
  __syncthreads();
  if (threadIdx.x == 0) {
    st->theta = theta1;
    st->theta1 = theta1;
    st->f = -1.0;
    st->coef = 0.0;
    st->anorm2 = 0.0;
    st->inner_iter = 0;
    st->est_best = 1e300;
    st->iter_best = 0;
    st->phase = PH_NECORR;
    if (w.f32_active) atomicAdd(w.f32_active, 1u);
  }
  __syncthreads();
}

// LSQR step (Paige & Saunders 1982, Bidiag 1 with Givens rotations), after the pass produced
// U_new = A v_i - alpha_i u_i (unnormalised, ||U_new|| = beta_{i+1}) and tk = X^T U_new in lag order.
__device__ void tail_lsqr(const Work& w, DevState* st, const double* tk, double n2, double* scratch) {
  const int p = w.p;
  const int mixed = st->mixed;
  double beta = sqrt(n2);
  // a beta at rounding level relative to ||B_k||_F means the Krylov space is exhausted: treat it as zero
  if (beta <= 1e-14 * sqrt(st->anorm2 + st->alpha * st->alpha)) beta = 0.0;
  double* tmp = w.t;
  for (int j = threadIdx.x; j < p; j += blockDim.x) tmp[j] = beta > 0 ? tk[p - 1 - j] / beta : 0.0;
  __syncthreads();
  double* s = w.g;  // scratch p-vector: A^T u_{i+1}
  apply_Mt(w, st->precond, mixed, tmp, s);
  __syncthreads();
  for (int j = threadIdx.x; j < p; j += blockDim.x) s[j] = s[j] - beta * w.v[j];
  __syncthreads();
  double alpha = sqrt(vec_norm2(s, p, scratch));
  if (beta == 0.0 || alpha <= 1e-14 * sqrt(st->anorm2 + alpha * alpha + beta * beta)) alpha = 0.0;
  const double rhobar = st->rhobar, phibar = st->phibar;
  const double rho = hypot(rhobar, beta);
  const double c = rho > 0 ? rhobar / rho : 1.0, sn = rho > 0 ? beta / rho : 0.0;
  const double theta = sn * alpha;
  const double phi_i = c * phibar;
  const double new_phibar = sn * phibar;
  const double new_rhobar = -c * alpha;
  const double step = rho > 0 ? phi_i / rho : 0.0, wscale = rho > 0 ? theta / rho : 0.0;
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const double wj = w.w[j];
    w.z[j] += step * wj;
    const double vj = alpha > 0 ? s[j] / alpha : 0.0;
    w.v[j] = vj;
    w.w[j] = vj - wscale * wj;
  }
  __syncthreads();
  const double anorm2 = st->anorm2 + alpha * alpha + beta * beta;
  const double arnorm = new_phibar * alpha * fabs(c);
  const double ratio = (new_phibar > 0 && anorm2 > 0) ? arnorm / (sqrt(anorm2) * new_phibar) : 0.0;
  const int iter = st->iter + 1;
  // the float64 floor of the ratio is about u sqrt(p) ||b|| / ||r|| (r = b - X phi carries an absolute error of
  // order u ||b||); LSQR's estimate of ||r|| is phibar
  const double floor64 = new_phibar > 0 ? 1e-15 * sqrt((double)p) * st->bnorm / new_phibar : 0.0;
  // with the sampled-QR preconditioner a sweep resolves the residual only to about kappa(X) u relative (each
  // later sweep starts from the float64 residual): asking LSQR for more spends iterations the next check would
  // not see
  const double floor_qr = st->precond == 2 ? 0.5 * st->kappa_est * 1.11e-16 : 0.0;
  const double tolA = st->mixed ? st->tol_inner : fmax(fmax(st->est_ratio, floor64), floor_qr);
  double est_best = st->est_best;
  int iter_best = st->iter_best;
  // progress: the ratio estimate halved, or the residual norm estimate still falls (relative 1e-10)
  const bool progress = ratio < 0.5 * est_best || new_phibar < (1.0 - 1e-10) * st->phibar_mark;
  if (progress) {
    est_best = fmin(ratio, est_best);
    iter_best = iter;
  }
  // Paige-Saunders stopping tests: ||A^T r|| <= tol ||A|| ||r||, or a compatible system ||r|| <= tol ||rhs||;
  // or no progress for kStallIters iterations
  const bool stop = (ratio <= tolA) || (new_phibar <= tolA * st->beta1) || (beta == 0.0) || (alpha == 0.0) ||
                    (iter >= st->iter_cap) || (iter - iter_best >= kStallIters) ||
                    (st->total_iter + 1 >= 64 * st->max_iter);
  __syncthreads();
  if (threadIdx.x == 0) {
    st->alpha = alpha;
    st->beta = beta;
    st->rhobar = new_rhobar;
    st->phibar = new_phibar;
    st->anorm2 = anorm2;
    st->iter = iter;
    st->est_best = est_best;
    st->iter_best = iter_best;
    if (progress) st->phibar_mark = new_phibar;
    st->total_iter += 1;
    if (mixed) st->f32_iter += 1;
    st->coef = beta > 0 ? alpha / beta : 0.0;
  }
  if (stop) {
    // phi += M z
    apply_M_exact(w, st->precond, mixed, w.z, tmp);
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x) w.phi[j] += tmp[j];
    __syncthreads();
    schedule_check(w, st, scratch);
  } else {
    apply_M(w, st->precond, mixed, w.v, w.d);
  }
}

// Bidiag 2 step (Paige & Saunders 1982) for (A^T A) zeta = s: after the pass produced
// P_i = A v_i - theta_i p_{i-1} (unnormalised, ||P_i|| = rho_i) and tk = X^T P_i.
__device__ void tail_necorr(const Work& w, DevState* st, const double* tk, double n2, double* scratch) {
  const int p = w.p;
  double rho = sqrt(n2);
  const double theta = st->theta;
  // rho at rounding level relative to ||R_k||_F: the Krylov space is exhausted, keep zeta as it is
  const bool rho_breakdown = rho <= 1e-14 * sqrt(st->anorm2 + theta * theta);
  if (rho_breakdown) rho = 0.0;
  const double f = rho > 0 ? -theta * st->f / rho : 0.0;
  double* tmp = w.t;
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const double wj = rho > 0 ? (w.v[j] - theta * w.w[j]) / rho : 0.0;
    w.w[j] = wj;
    w.z[j] += f * wj;
    tmp[j] = rho > 0 ? tk[p - 1 - j] / rho : 0.0;
  }
  __syncthreads();
  double* s = w.g;
  apply_Mt(w, st->precond, 1, tmp, s);
  __syncthreads();
  for (int j = threadIdx.x; j < p; j += blockDim.x) s[j] -= rho * w.v[j];
  __syncthreads();
  double theta_next = sqrt(vec_norm2(s, p, scratch));
  if (rho == 0.0 || theta_next <= 1e-14 * sqrt(st->anorm2 + theta * theta + rho * rho)) theta_next = 0.0;
  for (int j = threadIdx.x; j < p; j += blockDim.x) w.v[j] = theta_next > 0 ? s[j] / theta_next : 0.0;
  __syncthreads();
  const double resid = fabs(theta_next * f);
  const int it = st->inner_iter + 1;
  double est_best = st->est_best;
  int iter_best = st->iter_best;
  if (resid < 0.5 * est_best) {
    est_best = resid;
    iter_best = it;
  }
  const bool stop = rho == 0.0 || theta_next == 0.0 || resid <= st->tol_inner * st->theta1 ||
                    it >= st->iter_cap || (it - iter_best >= kStallIters) ||
                    (st->total_iter + 1 >= 64 * st->max_iter);
  __syncthreads();
  if (threadIdx.x == 0) {
    st->anorm2 += theta * theta + rho * rho;
    st->f = f;
    st->rho = rho;
    st->theta = theta_next;
    st->inner_iter = it;
    st->est_best = est_best;
    st->iter_best = iter_best;
    st->total_iter += 1;
    st->f32_iter += 1;
    st->coef = rho > 0 ? theta_next / rho : 0.0;
  }
  __syncthreads();
  if (stop) {
    if (threadIdx.x == 0 && w.f32_active) atomicSub(w.f32_active, 1u);
    apply_M_exact(w, st->precond, 1, w.z, tmp);
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x) w.phi[j] += tmp[j];
    __syncthreads();
    schedule_check(w, st, scratch);
  } else {
    apply_M(w, st->precond, 1, w.v, w.d);
  }
}

// float64 residual check: u_new = b - X phi was formed by the pass; tk = X^T r.
__device__ void tail_check(const Work& w, DevState* st, const double* tk, double n2, double* scratch) {
  const int p = w.p;
  const double rnorm = sqrt(n2);
  for (int j = threadIdx.x; j < p; j += blockDim.x) w.g[j] = tk[p - 1 - j];
  __syncthreads();
  const double gn = sqrt(vec_norm2(w.g, p, scratch));
  const double ne = (rnorm > 0 && st->anorm_2 > 0) ? gn / (st->anorm_2 * rnorm) : 0.0;
  const double prev = st->ne_ratio;
  // the residual norm still falls (by 1 % or more) since the last check: each sweep of LSQR on the residual can
  // resolve it only to about kappa(X) u relative, so an ill-conditioned solve needs several sweeps even while its
  // ratio stays high
  const bool r_progress = st->sweeps >= 1 && rnorm < 0.99 * st->rnorm;
  const int sweeps = st->sweeps + 1;
  const bool better = ne < st->ne_best;
  if (better)
    for (int j = threadIdx.x; j < p; j += blockDim.x) w.best[j] = w.phi[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    st->ne_ratio = ne;
    st->rnorm = rnorm;
    st->sweeps = sweeps;
    if (better) {
      st->ne_best = ne;
      st->rnorm_best = rnorm;
    }
  }
  __syncthreads();
  // Attainable ratio in float64: r = b - X phi carries an absolute error of order u ||b||, so the ratio cannot
  // go much below u sqrt(p) ||b|| / ||r||.
  const double floor64 = 1e-15 * sqrt((double)p) * fmax(1.0, rnorm > 0 ? st->bnorm / rnorm : 1.0);
  int next;
  if (threadIdx.x == 0 && rnorm <= st->tol * st->bnorm) st->compatible = 1;
  if (ne <= st->tol || rnorm <= st->tol * st->bnorm) next = 0;           // converged (or compatible)
  else if (sweeps >= st->max_sweeps || st->total_iter >= 64 * st->max_iter) next = 1;  // give up
  else if (sweeps >= 2 && ne > 0.7 * prev && !r_progress) {              // no progress since the last check
    next = (st->mixed && ne > 10.0 * floor64) ? 2 : 1;                   // mixed: float cannot refine it
  } else next = 3;                                                        // refine again
  if (next == 0 || next == 1 || next == 2) {
    if (threadIdx.x == 0) {
      st->status = next == 0 ? TOLS_OK : TOLS_NOT_CONVERGED;
      if (next == 2) st->mixed_ok = 0;
      st->phase = PH_DONE;
      st->done = 1;
    }
    return;
  }
  if (st->mixed) {
    start_necorr(w, st, scratch);
  } else {
    // LSQR on the residual: rhs = r, stored by this pass in U[0]; tighten the internal tolerance and cap the
    // restart at a few times the iterations the first run needed.
    if (threadIdx.x == 0) {
      st->est_ratio = fmax(st->est_ratio * 0.01, 1e-16);
      st->iter_cap = min(st->max_iter, max(2 * st->iter + 10, 20));
      if (st->precond == 2) st->iter_cap = min(st->iter_cap, kQrIterCap);
    }
    __syncthreads();
    start_lsqr(w, st, w.g, rnorm, scratch);
  }
}

// Gram matrix from c[h] = sum_{i<m} y[i] y[i+h], h in [0, p], plus the edge corrections
//   E_h(lo) = sum_{t<lo} (y[t+m] y[t+m+h] - y[t] y[t+h]):
//   G[j][k] = c[|j-k|] + E_|j-k|(p-1-max(j,k)),  h_j = (X^T b)_j = c[j+1] + E_{j+1}(p-1-j),
//   ||b||^2 = c[0] + E_0(p).
__device__ void tail_gram(const Work& w, const double* ck, double* bnorm2_out) {
  const int p = w.p;
  const long long m = w.m;
  const double* y = w.y64;
  for (int hh = threadIdx.x; hh <= p; hh += blockDim.x) {
    double E = 0.0;
    for (int lo = 0; lo <= p - hh; ++lo) {
      if (lo <= p - 1 - hh) {
        const int j = p - 1 - lo, k = j - hh;
        const double gv = ck[hh] + E;
        w.G[(size_t)j * p + k] = gv;
        w.G[(size_t)k * p + j] = gv;
      }
      if (lo == p - hh) {
        if (hh >= 1) w.h[hh - 1] = ck[hh] + E;
        else *bnorm2_out = ck[0] + E;
      } else {
        // term t = lo of the prefix; largest index read is y[p - 1 + m] = y[n - 1]
        E += y[lo + m] * y[lo + m + hh] - y[lo] * y[lo + hh];
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------------
// Pieces of the pass kernels (single series and batched).
//
// Shared memory (dynamic): ys[phys(TILE + p_pad + 16)] (T), us[phys(TILE)] (T), dr[p_pad] (T),
// wpart[kThreads/32][p_pad] (T), tacc[p_pad + 16] (double), scratch[16] (double).
template <typename T>
struct Smem {
  T *ys, *us, *dr, *wpart;
  double *tacc, *scratch;
  __device__ Smem(unsigned char* raw, int p_pad) {
    constexpr int TILE = TileCfg<T>::TILE;
    ys = reinterpret_cast<T*>(raw);
    us = ys + phys_size(TILE + p_pad + 16);      // u_old tile, padded layout
    dr = us + phys_size(TILE);                   // lag-reversed d
    wpart = dr + p_pad;                          // per-warp partial X^T u of a tile: [kThreads/32][p_pad]
    tacc = reinterpret_cast<double*>(wpart + (kThreads / 32) * p_pad);
    scratch = tacc + p_pad + 16;
  }
};

// For a solver-driven pass: which tail this kernel type runs for the series in state st, and its buffers
// (U[0]/U[1] ping-pong; b is y + p). Returns false when the phase belongs to the other precision or is done.
template <typename T>
__device__ bool select_phase(const DevState* st, const T* y, int p, const Work& w, int& tail, const T*& u_old,
                             T*& u_new, double& coef) {
  const int ph = st->phase;
  if (st->done || ph == PH_DONE) return false;
  if (sizeof(T) == 8) {
    if (ph == PH_CHECK) tail = TAIL_CHECK;
    else if (ph == PH_LSQR && !st->mixed) tail = TAIL_LSQR;
    else return false;
  } else {
    if (ph == PH_LSQR && st->mixed) tail = TAIL_LSQR;
    else if (ph == PH_NECORR) tail = TAIL_NECORR;
    else return false;
  }
  coef = st->coef;
  const int it = (tail == TAIL_NECORR) ? st->inner_iter : st->iter;
  if (tail == TAIL_CHECK) {
    u_old = y + p;                                   // b
    u_new = st->mixed ? nullptr : (T*)w.U[0];        // FP64: keep r for a restart
  } else if (tail == TAIL_NECORR) {
    u_old = it == 0 ? nullptr : (const T*)w.U[(it + 1) & 1];
    u_new = (T*)w.U[it & 1];
  } else {  // LSQR: the first pass reads the rhs (b on the first sweep, r stored in U[0] after a check)
    const int from_b = (st->sweeps == 0);
    if (it == 0) {
      u_old = from_b ? y + p : (const T*)w.U[0];
      u_new = (T*)w.U[1];
    } else {
      u_old = (const T*)w.U[(it & 1)];
      u_new = (T*)w.U[(it + 1) & 1];
    }
  }
  return true;
}

// Lag-reversed, scaled d into shared memory: dr[k] = d_scale * d[p-1-k], zero for k >= p.
template <typename T>
__device__ void load_dr(T* dr, const double* d, double d_scale, int p, int p_pad) {
  for (int k = threadIdx.x; k < p_pad; k += kThreads) dr[k] = k < p ? (T)(d_scale * d[p - 1 - k]) : (T)0;
}

// One tile of rows [i0, i0 + TILE): u_new = X d - c u_old (or u = y itself for the Gram lag sums), its squared
// norm (returned per thread) and the tile's X^T u contribution left in sm.wpart (per warp, lag order). The
// caller synchronises before reading wpart.
template <typename T>
__device__ double process_tile(const Smem<T>& sm, const T* __restrict__ y, long long n, long long m, int p_pad,
                               int nlag, int gram, const T* u_old, T* u_new, double coef, long long i0) {
  constexpr int RB = TileCfg<T>::RB;
  constexpr int KC = TileCfg<T>::KC;
  constexpr int TILE = TileCfg<T>::TILE;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jl = ((lane & 16) ? 4 : 0) + ((lane & 8) ? 2 : 0) + ((lane & 4) ? 1 : 0);
  const int r0 = tid * RB;                       // this thread's rows within the tile
  const int rows = (int)min((long long)TILE, m - i0);
  const int wlen = TILE + p_pad + 16;
  T* ys = sm.ys;
  T* us = sm.us;
  __syncthreads();                               // previous readers of ys / us / wpart are done
  for (int q = tid; q < wlen; q += kThreads) {
    const long long gi = i0 + q;
    ys[phys(q)] = gi < n ? y[gi] : (T)0;
  }
  if (!gram && u_old) {
    for (int q = tid; q < TILE; q += kThreads) us[phys(q)] = q < rows ? u_old[i0 + q] : (T)0;
  }
  __syncthreads();

  double n2 = 0.0;
  T uv[RB];
  if (gram) {
#pragma unroll
    for (int q = 0; q < RB / 4; ++q) lds4<T>(ys, r0 + 4 * q, uv + 4 * q);
#pragma unroll
    for (int r = 0; r < RB; ++r)
      if (r0 + r >= rows) uv[r] = (T)0;
  } else {
    // u_new = X d - c u_old : sliding window of y held in registers, KC lags per step
    T acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = (T)0;
    if (r0 < rows) {
      for (int k0 = 0; k0 < p_pad; k0 += KC) {
        T yv[RB + KC];
#pragma unroll
        for (int q = 0; q < (RB + KC) / 4; ++q) lds4<T>(ys, r0 + k0 + 4 * q, yv + 4 * q);
        T dv[KC];
#pragma unroll
        for (int q = 0; q < KC; ++q) dv[q] = sm.dr[k0 + q];
#pragma unroll
        for (int q = 0; q < KC; ++q)
#pragma unroll
          for (int r = 0; r < RB; ++r) acc[r] = fma(yv[r + q], dv[q], acc[r]);
      }
    }
    T uo[RB];
    if (u_old) {
#pragma unroll
      for (int q = 0; q < RB / 4; ++q) lds4<T>(us, r0 + 4 * q, uo + 4 * q);
    }
    T nn = (T)0;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      T u = (T)0;
      if (r0 + r < rows) {
        u = acc[r];
        if (u_old) u = fma((T)(-coef), uo[r], u);
      }
      nn = fma(u, u, nn);
      uv[r] = u;
    }
    n2 = (double)nn;
    if (u_new && r0 < rows) {
      T* dst = u_new + i0 + r0;
      if (((reinterpret_cast<uintptr_t>(dst) & 15) == 0) && r0 + RB <= rows) {
#pragma unroll
        for (int q = 0; q < RB / 4; ++q) st4<T>(dst + 4 * q, uv + 4 * q);
      } else {
#pragma unroll
        for (int r = 0; r < RB; ++r)
          if (r0 + r < rows) dst[r] = uv[r];
      }
    }
  }

  // tk[k] += sum_r u[r] y[r + k]: 8 lags at a time from the same conflict-free window loads, then a warp
  // reduce-scatter (9 shuffles) leaves lag k0 + jl on lanes with (lane & 3) == 0.
  for (int k0 = 0; k0 < nlag; k0 += 8) {
    T t8[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) t8[q] = (T)0;
    if (r0 < rows) {
      T yv[RB + 8];
#pragma unroll
      for (int q = 0; q < (RB + 8) / 4; ++q) lds4<T>(ys, r0 + k0 + 4 * q, yv + 4 * q);
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int r = 0; r < RB; ++r) t8[q] = fma(uv[r], yv[r + q], t8[q]);
    }
    const T v = warp_reduce_scatter8<T>(t8, lane);
    if ((lane & 3) == 0) sm.wpart[warp * p_pad + k0 + jl] = v;
  }
  return n2;
}

// Sum of the per-warp partials of lag k (fixed order).
template <typename T>
__device__ __forceinline__ double warp_parts_sum(const T* wpart, int p_pad, int k) {
  T sum = (T)0;
#pragma unroll
  for (int q = 0; q < kThreads / 32; ++q) sum += wpart[q * p_pad + k];
  return (double)sum;
}

// Two-level arrival of `nunits` partial results (unit u wrote part_t[u][.] and part_n2[u]): groups of kGroup
// units, then the groups. Returns true in the CTA that arrived last overall, which then holds the totals in
// tacc[0 .. nlag) and scratch[8], and has reset the counters it used. No waiting anywhere.
__device__ bool arrive(const Work& w, long long unit, long long nunits, int nlag, int p_pad, double* tacc,
                       double* scratch, int* s_last) {
  const int tid = threadIdx.x;
  const long long grp = unit / kGroup;
  const long long ngroups = (nunits + kGroup - 1) / kGroup;
  const int gsize = (int)min((long long)kGroup, nunits - grp * kGroup);
  __threadfence();
  __syncthreads();
  if (tid == 0) *s_last = (atomicAdd(&w.counters[grp], 1u) == (unsigned)(gsize - 1));
  __syncthreads();
  if (!*s_last) return false;
  __threadfence();
  for (int k = tid; k < nlag; k += kThreads) {
    double sum = 0.0;
    for (int q = 0; q < gsize; ++q) sum += __ldcg(&w.part_t[(size_t)(grp * kGroup + q) * p_pad + k]);
    w.grp_t[(size_t)grp * p_pad + k] = sum;
  }
  if (tid == 0) {
    double sum = 0.0;
    for (int q = 0; q < gsize; ++q) sum += __ldcg(&w.part_n2[grp * kGroup + q]);
    w.grp_n2[grp] = sum;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) *s_last = (atomicAdd(&w.counters[ngroups], 1u) == (unsigned)(ngroups - 1));
  __syncthreads();
  if (!*s_last) return false;
  __threadfence();
  for (int k = tid; k < nlag; k += kThreads) {
    double sum = 0.0;
    for (long long q = 0; q < ngroups; ++q) sum += __ldcg(&w.grp_t[(size_t)q * p_pad + k]);
    tacc[k] = sum;
  }
  if (tid == 0) {
    double sum = 0.0;
    for (long long q = 0; q < ngroups; ++q) sum += __ldcg(&w.grp_n2[q]);
    scratch[8] = sum;
    for (long long q = 0; q <= ngroups; ++q) w.counters[q] = 0u;
  }
  __syncthreads();
  return true;
}

// The scalar step after a pass (run by the last CTA with the totals in tacc / n2_all).
template <typename T>
__device__ void run_tail(int tail, const Work& w, int gram, int nlag, const double* tacc, double n2_all,
                         double* scratch, double* out_t, double* out_n2) {
  DevState* st = w.st;
  switch (tail) {
    case TAIL_STORE:
      if (out_t)
        for (int j = threadIdx.x; j < nlag; j += kThreads) out_t[j] = gram ? tacc[j] : tacc[nlag - 1 - j];
      if (threadIdx.x == 0 && out_n2) *out_n2 = n2_all;
      break;
    case TAIL_LSQR: tail_lsqr(w, st, tacc, n2_all, scratch); break;
    case TAIL_NECORR: tail_necorr(w, st, tacc, n2_all, scratch); break;
    case TAIL_CHECK: tail_check(w, st, tacc, n2_all, scratch); break;
    case TAIL_GRAM: tail_gram(w, tacc, out_n2); break;
    default: break;
  }
}

#include "tols_fft.cuh"

// ------------------------------------------------------------------------------------------------------
// Single-series pass kernel: each CTA accumulates its tiles, the CTAs then arrive.
template <typename T>
__global__ void __launch_bounds__(kThreads, TileCfg<T>::MINB) pass_kernel(PassArgs<T> a) {
  constexpr int TILE = TileCfg<T>::TILE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  int tail = a.tail;
  const T* u_old = a.u_old;
  T* u_new = a.u_new;
  double coef = a.coef_host;
  if (a.check_done) {
    if (!select_phase<T>(a.w.st, a.y, a.p, a.w, tail, u_old, u_new, coef)) return;
  } else if (a.coef_dev) {
    coef = *a.coef_dev;
  }
  const int p_pad = a.p_pad, nlag = a.nlag;
  Smem<T> sm(smem_raw, p_pad);
  const int tid = threadIdx.x;
  if (!a.gram) load_dr<T>(sm.dr, a.d, a.d_scale, a.p, p_pad);
  for (int k = tid; k < p_pad + 16; k += kThreads) sm.tacc[k] = 0.0;
  double n2 = 0.0;
  const long long ntiles = (a.m + TILE - 1) / TILE;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    n2 += process_tile<T>(sm, a.y, a.n, a.m, p_pad, nlag, a.gram, u_old, u_new, coef, tile * TILE);
    __syncthreads();
    for (int k = tid; k < nlag; k += kThreads) sm.tacc[k] += warp_parts_sum<T>(sm.wpart, p_pad, k);
  }
  __syncthreads();
  const double n2_cta = block_sum(n2, sm.scratch);
  for (int k = tid; k < nlag; k += kThreads) a.w.part_t[(size_t)blockIdx.x * p_pad + k] = sm.tacc[k];
  if (tid == 0) a.w.part_n2[blockIdx.x] = n2_cta;
  if (!arrive(a.w, blockIdx.x, gridDim.x, nlag, p_pad, sm.tacc, sm.scratch, &s_last)) return;
  const double n2_all = sm.scratch[8];
  __syncthreads();
  if (tid == 0 && a.worklog) a.worklog[a.work_slot] = 1 + tail + 5 * (int)(sizeof(T) == 8);
  run_tail<T>(tail, a.w, a.gram, nlag, sm.tacc, n2_all, sm.scratch, a.out_t, a.out_n2);
}

// ------------------------------------------------------------------------------------------------------
// Batched pass kernel: the CTAs stride over one tile list that concatenates the tiles of every series. Each
// tile leaves its own partials, the tiles of a series arrive in groups of kGroup, and the CTA that completes a
// series runs that series' scalar step. A series' reduction order depends only on its own tiles, so its result
// is the same whatever else is in the batch.
template <typename T>
__global__ void __launch_bounds__(kThreads, TileCfg<T>::MINB) batch_pass_kernel(BatchArgs a) {
  constexpr int TILE = TileCfg<T>::TILE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  __shared__ int s_skip;
  const int is_double = sizeof(T) == 8;
  const long long total = a.live ? a.live[is_double ? 1 : 0] : (is_double ? a.tiles_d : a.tiles_f);
  const int* tile_series = is_double ? a.tile_series_d : a.tile_series_f;
  const int tid = threadIdx.x;
  for (long long g = blockIdx.x; g < total; g += gridDim.x) {
    const int sidx = tile_series[g];
    const BatchSeries& S = a.series[sidx];
    const Work& w = S.w;
    const T* y = is_double ? (const T*)S.w.y64 : (const T*)S.w.y32;
    const long long local = g - (is_double ? S.tile0_d : S.tile0_f);
    const long long ntiles = (S.w.m + TILE - 1) / TILE;
    int tail = TAIL_GRAM;
    const T* u_old = nullptr;
    T* u_new = nullptr;
    double coef = 0.0;
    const int gram = a.gram;
    const int p = S.w.p;
    const int p_pad = gram ? pad_p(p + 1) : pad_p(p);
    const int nlag = gram ? p + 1 : p;
    if (tid == 0) {
      int skip = 0;
      if (gram) skip = !is_double;                            // Gram lag sums from float64 products
      else skip = !select_phase<T>(w.st, y, p, w, tail, u_old, u_new, coef);
      s_skip = skip;
    }
    __syncthreads();
    const int skip = s_skip;
    __syncthreads();
    if (skip) continue;
    if (!gram) select_phase<T>(w.st, y, p, w, tail, u_old, u_new, coef);
    Smem<T> sm(smem_raw, p_pad);
    if (!gram) load_dr<T>(sm.dr, w.d, 1.0, p, p_pad);
    const double n2t = process_tile<T>(sm, y, S.w.n, S.w.m, p_pad, nlag, gram, u_old, u_new, coef, local * TILE);
    __syncthreads();
    for (int k = tid; k < nlag; k += kThreads)
      w.part_t[(size_t)local * p_pad + k] = warp_parts_sum<T>(sm.wpart, p_pad, k);
    const double n2_tile = block_sum(n2t, sm.scratch);
    if (tid == 0) w.part_n2[local] = n2_tile;
    if (!arrive(w, local, ntiles, nlag, p_pad, sm.tacc, sm.scratch, &s_last)) continue;
    const double n2_all = sm.scratch[8];
    __syncthreads();
    run_tail<T>(tail, w, gram, nlag, sm.tacc, n2_all, sm.scratch, nullptr, w.bnorm2);
    __syncthreads();
    if (tid == 0 && !gram && w.st->done && a.done_count) atomicAdd(a.done_count, 1u);
  }
}

template <typename T>
static size_t pass_smem(int p_pad) {
  constexpr int TILE = TileCfg<T>::TILE;
  size_t b = sizeof(T) * ((size_t)phys_size(TILE + p_pad + 16) + phys_size(TILE) + p_pad +
                          (size_t)(kThreads / 32) * p_pad);
  b += sizeof(double) * ((size_t)p_pad + 16 + 16);
  return b;
}

// FFT length of a pass: PassArgs::fft is 0 (direct products) or N (1 also means the precision's default N).
template <typename T>
static int pass_nfft(const PassArgs<T>& a) { return a.fft == 0 ? 0 : a.fft == 1 ? FftCfg<T>::N : a.fft; }

template <typename T>
cudaError_t launch_pass(const PassArgs<T>& a, int grid, cudaStream_t s) {
  const int nfft = pass_nfft(a);
  if (nfft && nfft != FftCfg<T>::N && !(sizeof(T) == 8 && nfft == 4096)) return cudaErrorInvalidValue;
  const long long rows_per_tile = nfft ? (long long)(nfft - a.p_pad) : (long long)TileCfg<T>::TILE;
  if (rows_per_tile < 1) return cudaErrorInvalidValue;
  const long long ntiles = (a.m + rows_per_tile - 1) / rows_per_tile;
  int g = (int)lmin((long long)grid, ntiles);
  if (g < 1) g = 1;
  cudaError_t e;
  if constexpr (sizeof(T) == 4) {
    // float product passes take the register-blocked kernel, whose inputs arrive by bulk copies: 16-byte aligned
    // u vectors and spectra, and its float64 sum buffer
    const bool aligned = ((reinterpret_cast<uintptr_t>(a.u_old) | reinterpret_cast<uintptr_t>(a.u_new) |
                           reinterpret_cast<uintptr_t>(a.w.wspec32)) & 15) == 0;
    if (nfft && !a.gram && a.nlag > 0 && aligned && a.w.sacc32 && a.w.wspec32) {
      e = smem_opt_in((const void*)fft32_pass_kernel, 200 * 1024);
      if (e != cudaSuccess) return e;
      fft32_pass_kernel<<<g, kThreads, fft32_pass_smem(a.p_pad), s>>>(a);
      return cudaGetLastError();
    }
  } else {
    if (nfft == 4096) {
      e = smem_opt_in((const void*)fft_pass_kernel<double, 4096>, 200 * 1024);
      if (e != cudaSuccess) return e;
      fft_pass_kernel<double, 4096><<<g, kThreads, fft_pass_smem<double, 4096>(a.p_pad), s>>>(a);
      return cudaGetLastError();
    }
  }
  e = smem_opt_in(nfft ? (const void*)fft_pass_kernel<T> : (const void*)pass_kernel<T>, 200 * 1024);
  if (e != cudaSuccess) return e;
  if (nfft) fft_pass_kernel<T><<<g, kThreads, fft_pass_smem<T>(a.p_pad), s>>>(a);
  else pass_kernel<T><<<g, kThreads, pass_smem<T>(a.p_pad), s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_pass<float>(const PassArgs<float>&, int, cudaStream_t);
template cudaError_t launch_pass<double>(const PassArgs<double>&, int, cudaStream_t);

size_t pass_smem_bytes(int is_double, int p_pad, int nfft) {
  if (nfft) {
    if (!is_double) return fft32_pass_smem(p_pad);
    return nfft == 4096 ? fft_pass_smem<double, 4096>(p_pad) : fft_pass_smem<double>(p_pad);
  }
  return is_double ? pass_smem<double>(p_pad) : pass_smem<float>(p_pad);
}
// the kernel whose occupancy sizes the grid of FFT passes of length nfft (float: the register-blocked kernel)
const void* fft_kernel_ptr(int is_double, int nfft) {
  if (!is_double) return (const void*)fft32_pass_kernel;
  return nfft == 4096 ? (const void*)fft_pass_kernel<double, 4096> : (const void*)fft_pass_kernel<double>;
}
size_t fft32_sum_bytes() { return sizeof(float4) * (size_t)kMaxGrid * (FftCfg<float>::N / 2 + 1); }
int fft_size(int is_double) { return is_double ? FftCfg<double>::N : FftCfg<float>::N; }

template <typename T, int N>
static size_t spectra_bytes(long long m, int p_pad) {
  const long long L = N - p_pad;
  return sizeof(typename FftCfg<T>::V) * (size_t)((m + L - 1) / L) * FftCfg2<T, N>::WS;
}
size_t fft_spectra_bytes(int is_double, long long m, int p_pad, int nfft) {
  if (!is_double) return spectra_bytes<float, 4096>(m, p_pad);
  return nfft == 4096 ? spectra_bytes<double, 4096>(m, p_pad) : spectra_bytes<double, 2048>(m, p_pad);
}

template <typename T, int N>
static cudaError_t launch_spectra_t(const T* y, long long n, long long m, int p_pad, void* out, const void* tw,
                                    int grid, cudaStream_t s) {
  using V = typename FftCfg<T>::V;
  const size_t smem = round16(sizeof(V) * 2 * (size_t)FftCfg2<T, N>::PADDED);   // the work arrays A, B only
  cudaError_t e = smem_opt_in((const void*)spectrum_kernel<T, N>, 200 * 1024);
  if (e != cudaSuccess) return e;
  const int L = N - p_pad;
  const long long ntiles = (m + L - 1) / L;
  const int g = (int)lmin((long long)grid, ntiles);
  spectrum_kernel<T, N><<<g < 1 ? 1 : g, kThreads, smem, s>>>(y, n, m, L, (V*)out, (const V*)tw);
  return cudaGetLastError();
}
cudaError_t launch_spectra(int is_double, const void* y, long long n, long long m, int p_pad, void* out,
                           const void* tw, int grid, cudaStream_t s, int nfft) {
  if (!is_double) return launch_spectra_t<float, 4096>((const float*)y, n, m, p_pad, out, tw, grid, s);
  return nfft == 4096 ? launch_spectra_t<double, 4096>((const double*)y, n, m, p_pad, out, tw, grid, s)
                      : launch_spectra_t<double, 2048>((const double*)y, n, m, p_pad, out, tw, grid, s);
}
int pass_tile_rows(int is_double) { return is_double ? TileCfg<double>::TILE : TileCfg<float>::TILE; }
const void* pass_kernel_ptr(int is_double) {
  return is_double ? (const void*)pass_kernel<double> : (const void*)pass_kernel<float>;
}

template <typename T>
cudaError_t launch_batch_pass(const BatchArgs& a, int grid, int p_pad_max, cudaStream_t s) {
  const size_t smem = pass_smem<T>(p_pad_max);
  cudaError_t e = smem_opt_in((const void*)batch_pass_kernel<T>, 200 * 1024);
  if (e != cudaSuccess) return e;
  const long long total = sizeof(T) == 8 ? a.tiles_d : a.tiles_f;
  int g = (int)lmin((long long)grid, total);
  if (g < 1) g = 1;
  batch_pass_kernel<T><<<g, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}
size_t batch_fft_smem(int p_pad_max) { return fft_pass_smem<double>(p_pad_max); }
const void* batch_fft_kernel_ptr() { return (const void*)batch_fft_kernel; }
cudaError_t launch_batch_fft(const BatchArgs& a, int grid, int p_pad_max, cudaStream_t s) {
  cudaError_t e = smem_opt_in((const void*)batch_fft_kernel, 200 * 1024);
  if (e != cudaSuccess) return e;
  int g = (int)lmin((long long)grid, a.tiles_x);
  if (g < 1) return cudaSuccess;
  batch_fft_kernel<<<g, kThreads, batch_fft_smem(p_pad_max), s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_batch_dspec(const BatchSeries* series, int count, cudaStream_t s) {
  const size_t smem = FftSmem<double>::bytes(0);
  cudaError_t e = smem_opt_in((const void*)batch_dspec_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  if (count < 1) return cudaSuccess;
  batch_dspec_kernel<<<count, kThreads, smem, s>>>(series);
  return cudaGetLastError();
}
template cudaError_t launch_batch_pass<float>(const BatchArgs&, int, int, cudaStream_t);
template cudaError_t launch_batch_pass<double>(const BatchArgs&, int, int, cudaStream_t);
const void* batch_kernel_ptr(int is_double) {
  return is_double ? (const void*)batch_pass_kernel<double> : (const void*)batch_pass_kernel<float>;
}

// ------------------------------------------------------------------------------------------------------
// Preconditioner: ||X||_F, a power-iteration estimate of ||X||_2, Cholesky G = R^T R (upper R, in place),
// M = R^{-1} and M^T (float64 and float copies). One CTA; G is symmetric on entry.
__device__ __forceinline__ double* scratch_vec(const Work& w) { return w.t; }  // w.t, w.g: 2 p_pad doubles

// G and R^{-1} are worked on in shared memory when both fit (p <= kPrecondSmemP, tols_internal.cuh): the
// factorisation and the back substitutions are chains of dependent read-modify-writes, which would wait on L2
// round trips in global memory.

// s / d by multiplication with magic = ceil(2^32 / d) = (2^32 - 1) / d + 1 (division by an invariant integer,
// Granlund & Montgomery 1994): exact while s d < 2^32, integer instructions only (the general division
// sequence goes through float conversions, which are slow here).
// d = 1 has no 32-bit magic (2^32): its magic is 0 and small_div returns s itself.
__device__ __forceinline__ unsigned div_magic(unsigned d) { return d > 1u ? 0xffffffffu / d + 1u : 0u; }
__device__ __forceinline__ int small_div(int s, unsigned magic) {
  return magic ? (int)__umulhi((unsigned)s, magic) : s;
}

// The preconditioner runs one CTA per series; 16 warps (4 per SM sub-partition) hide the latency of its chains of
// dependent shared-memory and FP64 operations better than 8.
constexpr int kPcThreads = 512;

// Sampled-row QR (Section 3.1: a least-squares problem on sampled rows of X): c = kQrRowsPerP p rows of X,
// evenly spaced (row i_k = floor((k + 1/2) m / c)), gathered into w.qr (c x p, row-major), then Householder QR
// in float64. R (upper triangular, p x p, row-major) is written to R. Returns false when a column of the sample
// is (numerically) dependent on the others, i.e. R would be singular.
__device__ bool sampled_qr(const Work& w, double* R, double* qw, double* qpart, double* scratch) {
  const int p = w.p;
  const long long m = w.m;
  const int c = kQrRowsPerP * p;
  double* A = w.qr;
  double* qv = w.qr + (size_t)c * p;                   // the Householder vector (global scratch, L1-cached reads)
  const double* y = w.y64;
  // gather: one row per warp at a time, its lanes along the row (one 64-bit division per row, not per entry)
  for (int i = threadIdx.x >> 5; i < c; i += kPcThreads / 32) {
    const long long row = ((2LL * i + 1) * m) / (2LL * c);
    const double* yr = y + p + row - 1;              // X[row][j] = y[p + row - j - 1]
    for (int j = threadIdx.x & 31; j < p; j += 32) A[(size_t)i * p + j] = yr[-j];
  }
  for (int q = threadIdx.x; q < p * p; q += kPcThreads) R[q] = 0.0;
  __syncthreads();
  double amax = 0.0;   // largest |R_kk| so far, for the rank test
  bool full_rank = true;
  for (int k = 0; k < p; ++k) {
    // Householder vector of column k below the diagonal: v = x - alpha e_k, alpha = -sign(x_k) ||x||
    double s = 0.0;
    for (int i = k + threadIdx.x; i < c; i += kPcThreads) {
      const double a = A[(size_t)i * p + k];
      qv[i] = a;
      s = fma(a, a, s);
    }
    s = block_sum<kPcThreads>(s, scratch);                      // synchronises: qv complete
    const double x0 = qv[k];
    const double nrm = sqrt(s);
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    const double vk = x0 - alpha;
    const double vtv = s - x0 * x0 + vk * vk;
    amax = fmax(amax, nrm);
    if (!(nrm > 1e-13 * amax)) full_rank = false;
    const int ncol = p - k - 1;
    if (vtv > 0.0 && ncol > 0) {
      const double beta = 2.0 / vtv;
      __syncthreads();
      if (threadIdx.x == 0) qv[k] = vk;
      __syncthreads();
      // qw_j = beta sum_{i >= k} v_i A[i][j] for the trailing columns: (column, row-slice) pairs over the CTA
      const int nsplit = max(1, min(kPcThreads / ncol, c - k));
      for (int t = threadIdx.x; t < ncol * nsplit; t += kPcThreads) {
        const int r0 = t / ncol, jj = t - r0 * ncol;      // t < kPcThreads: one division per thread
        const int j = k + 1 + jj;
        // four independent accumulators: the loads of A (L2-resident) overlap instead of waiting one by one
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int i = k + r0;
        for (; i + 3 * nsplit < c; i += 4 * nsplit) {
          a0 = fma(qv[i], A[(size_t)i * p + j], a0);
          a1 = fma(qv[i + nsplit], A[(size_t)(i + nsplit) * p + j], a1);
          a2 = fma(qv[i + 2 * nsplit], A[(size_t)(i + 2 * nsplit) * p + j], a2);
          a3 = fma(qv[i + 3 * nsplit], A[(size_t)(i + 3 * nsplit) * p + j], a3);
        }
        for (; i < c; i += nsplit) a0 = fma(qv[i], A[(size_t)i * p + j], a0);
        qpart[t] = (a0 + a1) + (a2 + a3);
      }
      __syncthreads();
      for (int jj = threadIdx.x; jj < ncol; jj += kPcThreads) {
        double acc = 0.0;
        for (int r0 = 0; r0 < nsplit; ++r0) acc += qpart[r0 * ncol + jj];
        qw[jj] = beta * acc;
      }
      __syncthreads();
      // A[i][j] -= v_i qw_j over the trailing block ((c - k) ncol < 6 p^2 entries: q ncol < 2^32)
      const int tot = (c - k) * ncol;
      const unsigned nmag = div_magic((unsigned)ncol);
      // four entries per thread at a time: all four loads issue before the stores (the entries are distinct)
      for (int q0 = threadIdx.x; q0 < tot; q0 += 4 * kPcThreads) {
        size_t idx[4];
        double va[4], wb[4], av[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int q = q0 + s * kPcThreads;
          const int qq = q < tot ? q : q0;                  // out of range: a harmless duplicate of q0
          const int r = small_div(qq, nmag), jj = qq - r * ncol;
          idx[s] = (size_t)(k + r) * p + (k + 1 + jj);
          va[s] = qv[k + r];
          wb[s] = qw[jj];
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) av[s] = A[idx[s]];
#pragma unroll
        for (int s = 0; s < 4; ++s)
          if (q0 + s * kPcThreads < tot) A[idx[s]] = fma(-va[s], wb[s], av[s]);
      }
      __syncthreads();
    }
    // row k of R: alpha on the diagonal, the transformed row k beyond it
    for (int j = k + threadIdx.x; j < p; j += kPcThreads) R[(size_t)k * p + j] = j == k ? alpha : A[(size_t)k * p + j];
    __syncthreads();
  }
  return full_rank;
}

__device__ void precond_body(const Work& w, int want_precond, double* smem) {
  const int p = w.p;
  const unsigned pmag = div_magic((unsigned)p);   // q / p for q < p^2 (q p < 2^32 for p <= 1024)
  DevState* st = w.st;
  __shared__ double scratch[16];
  __shared__ int s_fail;
  __shared__ int s_shift;
  __shared__ double s_val[2];
  __shared__ float xs[TOLS_MAX_P], ys[TOLS_MAX_P], zs[TOLS_MAX_P];
  __shared__ float red2[2 * (kPcThreads / 32)];
  __shared__ unsigned s_mag[TOLS_MAX_P + 2];       // div_magic(d), d = 0 .. p + 1, formed once (a division each)
  for (int d = threadIdx.x; d <= p + 1; d += kPcThreads) s_mag[d] = d > 0 ? div_magic((unsigned)d) : 0u;
  __shared__ double qw[kQrMaxP], qpart[kPcThreads];
  const bool in_smem = smem && p <= kPrecondSmemP;
  double* G = in_smem ? smem : w.G;
  double* Mm = in_smem ? smem + (size_t)p * p : w.M;
  // the Gram matrix is kept for a refactorisation: in w.G when the work is in shared memory, else in w.Mt
  // (written only at the end)
  const double* Gsave = in_smem ? w.G : w.Mt;
  if (in_smem) {
#pragma unroll 4
    for (int q = threadIdx.x; q < p * p; q += kPcThreads) G[q] = w.G[q];
    __syncthreads();
  }
  // ||X||_F^2 = trace(G)
  double tr = 0.0, dmax = 0.0;
  for (int j = threadIdx.x; j < p; j += kPcThreads) {
    tr += G[(size_t)j * p + j];
    dmax = fmax(dmax, G[(size_t)j * p + j]);
  }
  tr = block_sum<kPcThreads>(tr, scratch);
  // block max of the diagonal
  {
    double v = dmax;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (int k = 0; k < kPcThreads / 32; ++k) r = fmax(r, scratch[k]);
      s_val[0] = r;
    }
    __syncthreads();
    dmax = s_val[0];
    __syncthreads();
  }
  // Sums over the CTA of two per-thread float values (every thread gets them).
  auto sum2 = [&](float& dot, float& xx) {
    for (int o = 16; o > 0; o >>= 1) {
      dot += __shfl_xor_sync(0xffffffffu, dot, o);
      xx += __shfl_xor_sync(0xffffffffu, xx, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red2[threadIdx.x >> 5] = dot;
      red2[(kPcThreads / 32) + (threadIdx.x >> 5)] = xx;
    }
    __syncthreads();
    dot = xx = 0.f;
    for (int q = 0; q < kPcThreads / 32; ++q) {
      dot += red2[q];
      xx += red2[(kPcThreads / 32) + q];
    }
  };
  // power iteration for lambda_max = ||X||_2^2 on a float copy of G (two digits suffice for the ratio's norm);
  // the copy lives in the M area, which is free until the factorisation
  double lam = 0.0;
  {
    float* Gf = reinterpret_cast<float*>(Mm);
    // G is symmetric: convert its upper triangle and mirror it (float64 -> float conversions use the FP64 pipe)
    for (int q = threadIdx.x; q < p * p; q += kPcThreads) {
      const int i = small_div(q, pmag), j = q - i * p;
      if (i <= j) {
        const float g = (float)G[q];
        Gf[q] = g;
        Gf[j * p + i] = g;
      }
    }
    for (int j = threadIdx.x; j < p; j += kPcThreads) xs[j] = 1.0f;
    __syncthreads();
    // float arithmetic throughout (FP64 instructions, divisions above all, are expensive here); the next
    // iterate is y scaled by xx / dot, the inverse Rayleigh quotient, which keeps its norm near the first one's
    float dot = 0.f, xx = 0.f;
    for (int it = 0; it < 8; ++it) {
      dot = 0.f;
      xx = 0.f;
      for (int i = threadIdx.x; i < p; i += kPcThreads) {      // ys = G xs (column i of the symmetric G)
        float a0 = 0.f, a1 = 0.f;
        int j = 0;
        for (; j + 1 < p; j += 2) {
          a0 = fmaf(Gf[j * p + i], xs[j], a0);
          a1 = fmaf(Gf[(j + 1) * p + i], xs[j + 1], a1);
        }
        if (j < p) a0 = fmaf(Gf[j * p + i], xs[j], a0);
        const float yi = a0 + a1;
        ys[i] = yi;
        dot = fmaf(xs[i], yi, dot);
        xx = fmaf(xs[i], xs[i], xx);
      }
      sum2(dot, xx);
      const float scale = dot > 0.f ? xx / dot : 0.f;
      for (int j = threadIdx.x; j < p; j += kPcThreads) xs[j] = ys[j] * scale;
      __syncthreads();
    }
    lam = xx > 0.f ? (double)dot / (double)xx : 0.0;
  }
  if (!isfinite(tr) || !isfinite(*w.bnorm2)) {
    if (threadIdx.x == 0) {
      st->status = TOLS_ERR_NONFINITE;
      st->phase = PH_DONE;
      st->done = 1;
      st->precond = 0;
    }
    return;
  }
  if (threadIdx.x == 0) {
    st->bnorm = sqrt(fmax(*w.bnorm2, 0.0));
    st->anorm_f = sqrt(fmax(tr, 0.0));
    st->anorm_2 = sqrt(fmax(lam, 0.0));
    if (!(st->anorm_2 > 0.0)) st->anorm_2 = st->anorm_f;
    s_fail = 0;
  }
  __syncthreads();

  // Cholesky G = R^T R on the upper triangle (right-looking), first without a shift, then M = R^{-1}. If a pivot
  // falls to rounding level (<= p u max_j G_jj, u of the precision G was formed in: G singular at working
  // precision), G is refactored with the shift lambda = 10 p u max_j G_jj, which bounds kappa(X R^{-1}) by about
  // sqrt(lambda) kappa(X). A singular G is flagged: if the solve then turns out compatible (an exactly
  // rank-deficient X), the host repeats it with plain LSQR from zero, which returns the minimum-norm solution
  // (Thm. "Solution to OLS problem"). kappa(R) = ||X||_2 ||R^{-1}||_2 is estimated by power iteration; a factor
  // with kappa(R)^2 u > 1/4 still preconditions LSQR (better than a shifted one) but is not trusted for the
  // semi-normal-equation start, nor for refinement with float products.
  const double ueps = 1.11e-16;   // G is formed from float64 products in every precision
  if (want_precond && !in_smem) {
    for (size_t q = threadIdx.x; q < (size_t)p * p; q += kPcThreads) w.Mt[q] = G[q];
    __syncthreads();
  }
  if (threadIdx.x == 0) s_shift = 0;
  __syncthreads();
  // ||R^{-1}||_2^2 = lambda_max(M^T M) (M in Mm): power iteration on a float copy of M's upper triangle in the
  // area of R (not needed any more), rows padded to p + 1 entries so that both row and column walks are free of
  // bank conflicts; returns kappa(R) = ||X||_2 ||R^{-1}||_2.
  auto estimate = [&]() -> double {
    float* Mf = reinterpret_cast<float*>(G);
    const int ld = p + 1;
    for (int q = threadIdx.x; q < p * p; q += kPcThreads) {
      const int i = small_div(q, pmag), j = q - i * p;
      if (i <= j) Mf[i * ld + j] = (float)Mm[q];
    }
    for (int j = threadIdx.x; j < p; j += kPcThreads) xs[j] = 1.0f;
    __syncthreads();
    float dot = 0.f, xx = 0.f;
    for (int it = 0; it < 6; ++it) {
      for (int i = threadIdx.x; i < p; i += kPcThreads) {        // ys = M xs (rows)
        float a0 = 0.f, a1 = 0.f;
        int j = i;
        for (; j + 1 < p; j += 2) {
          a0 = fmaf(Mf[i * ld + j], xs[j], a0);
          a1 = fmaf(Mf[i * ld + j + 1], xs[j + 1], a1);
        }
        if (j < p) a0 = fmaf(Mf[i * ld + j], xs[j], a0);
        ys[i] = a0 + a1;
      }
      __syncthreads();
      dot = 0.f;
      xx = 0.f;
      for (int j = threadIdx.x; j < p; j += kPcThreads) {        // zs = M^T ys (columns)
        float b0 = 0.f, b1 = 0.f;
        int i = 0;
        for (; i + 1 <= j; i += 2) {
          b0 = fmaf(Mf[i * ld + j], ys[i], b0);
          b1 = fmaf(Mf[(i + 1) * ld + j], ys[i + 1], b1);
        }
        if (i <= j) b0 = fmaf(Mf[i * ld + j], ys[i], b0);
        const float zj = b0 + b1;
        zs[j] = zj;
        dot = fmaf(xs[j], zj, dot);
        xx = fmaf(xs[j], xs[j], xx);
      }
      sum2(dot, xx);
      const float scale = dot > 0.f ? xx / dot : 0.f;
      for (int j = threadIdx.x; j < p; j += kPcThreads) xs[j] = zs[j] * scale;
      __syncthreads();
    }
    const double lamM = xx > 0.f ? (double)dot / (double)xx : 0.0;
    return sqrt(fmax(lam, 0.0)) * sqrt(fmax(lamM, 0.0));
  };
  // M = R^{-1} (R upper triangular in G), then kappa(R) = ||X||_2 ||R^{-1}||_2.
  auto invert_and_estimate = [&]() -> double {
    // M = R^{-1} from R M = I, right-looking: M starts as I; at step i (from p-1 down) row i is final up to the
    // factor 1/R_ii, and its contribution R_ri M_ic is removed from every row r < i (a rectangle of i x (p-i)
    // entries, spread evenly over every warp).
    // (used after the sampled QR, p <= kQrMaxP: the reciprocals of the diagonal go to qw, one division each)
    for (int q = threadIdx.x; q < p * p; q += kPcThreads) Mm[q] = (q == small_div(q, pmag) * (p + 1)) ? 1.0 : 0.0;
    for (int j = threadIdx.x; j < p; j += kPcThreads) qw[j] = 1.0 / G[j * p + j];
    __syncthreads();
    for (int i = p - 1; i >= 0; --i) {
      const double inv = qw[i];
      for (int c = i + threadIdx.x; c < p; c += kPcThreads) Mm[i * p + c] *= inv;
      __syncthreads();
      const int wd = p - i;
      const unsigned wmag = div_magic((unsigned)wd);
      for (int s2 = threadIdx.x; s2 < i * wd; s2 += kPcThreads) {
        const int r = small_div(s2, wmag), c = i + (s2 - r * wd);
        Mm[r * p + c] = fma(-G[r * p + i], Mm[i * p + c], Mm[r * p + c]);
      }
      __syncthreads();
    }
    return estimate();
  };
  // Copies of M into the float64 / float matrices the solve reads (M and M^T).
  // The float copies serve only the mixed path.
  auto store = [&]() {
    const bool mixed = st->mixed;
    for (int q = threadIdx.x; q < p * p; q += kPcThreads) {
      const int i = small_div(q, pmag), j = q - i * p;
      const double mv = Mm[q];                  // M[i][j]
      const double tv = Mm[j * p + i];          // M[j][i] = M^T[i][j]
      if (in_smem) w.M[q] = mv;
      w.Mt[q] = tv;
      if (mixed) {
        w.M32[q] = (float)mv;
        w.Mt32[q] = (float)tv;
      }
    }
    __syncthreads();
  };
  double cond = 0.0;
  for (int attempt = 0; attempt < 2 && want_precond && !st->no_precond; ++attempt) {
    double lambda = 0.0;
    if (attempt == 1) {
      if (threadIdx.x == 0) s_shift = 1;
      lambda = 10.0 * (double)p * ueps * dmax;
      for (size_t q = threadIdx.x; q < (size_t)p * p; q += kPcThreads) G[q] = Gsave[q];
      __syncthreads();
      for (int j = threadIdx.x; j < p; j += kPcThreads) G[(size_t)j * p + j] += lambda;
      if (threadIdx.x == 0) s_fail = 0;
      __syncthreads();
    }
    const double tiny = attempt == 0 ? (double)p * ueps * dmax : 1e-3 * lambda;
    // right-looking: every thread reads the pivot itself (no broadcast step), scales row k by the reciprocal,
    // then updates the trailing upper triangle. The same elimination applied to B = I (rows scaled by 1/R_kk,
    // row k subtracted R_ki times from every row i > k) leaves B = L^{-1} = (R^{-1})^T, lower triangular, in Mm:
    // the inverse comes out of the same p steps instead of p more.
    double* B = Mm;
    for (int q = threadIdx.x; q < p * p; q += kPcThreads) B[q] = (q == small_div(q, pmag) * (p + 1)) ? 1.0 : 0.0;
    // Thread 0 forms each pivot's square root and reciprocal once, one step ahead (it also owns the update of
    // the next diagonal entry): float64 square roots and divisions are long instruction sequences on the FP64
    // pipe, which every warp would otherwise repeat.
    if (threadIdx.x == 0) {
      const double piv = G[0];
      if (!(piv > tiny)) {
        s_fail = 1;
      } else {
        const double r = rsqrt_newton(piv);
        s_val[0] = piv * r;
        s_val[1] = r;
      }
    }
    __syncthreads();
    for (int k = 0; k < p; ++k) {
      if (s_fail) break;
      const double rkk = s_val[0];
      const double inv = s_val[1];
      for (int j = k + 1 + threadIdx.x; j < p; j += kPcThreads) G[k * p + j] *= inv;
      for (int c = threadIdx.x; c <= k; c += kPcThreads) B[k * p + c] *= inv;
      __syncthreads();
      if (threadIdx.x == 0) G[k * p + k] = rkk;
      // trailing update G[i][j] -= r_i r_j over k < i <= j < p, spread evenly over every warp: the triangle of
      // width w = p-k-1 is folded (row a paired with row w-1-a) into ceil(w/2) rows of exactly w+1 entries
      const double* __restrict__ rowk = G + k * p;
      const int wd = p - k - 1;
      const int half = (wd + 1) >> 1;
      // entry (k+1, k+1), the next pivot, is thread 0's (s2 = 0 of the fold)
      if (threadIdx.x == 0 && wd > 0) {
        const int d = (k + 1) * p + (k + 1);
        const double piv = fma(-rowk[k + 1], rowk[k + 1], G[d]);
        G[d] = piv;
        if (!(piv > tiny)) {
          s_fail = 1;
        } else {
          const double r = rsqrt_newton(piv);
          s_val[0] = piv * r;
          s_val[1] = r;
        }
      }
      // then every other entry of the fold, and the B rectangle B[i][c] -= R_ki B[k][c] (k < i < p, c <= k),
      // shared by warps 1 .. 15: warp 0 runs only thread 0's pivot chain (its other lanes would otherwise wait
      // behind that divergent branch before starting their share)
      const unsigned wmag = s_mag[wd + 1];
      const int t1 = (int)threadIdx.x - 32;
      for (int s2 = t1 < 0 ? 0x7fffffff : t1; s2 < half * (wd + 1); s2 += kPcThreads - 32) {
        if (s2 == 0) continue;
        const int a = small_div(s2, wmag), b = s2 - a * (wd + 1);
        int r, c;
        if (b < wd - a) {
          r = a;
          c = a + b;
        } else {
          r = wd - 1 - a;
          if (r <= a) continue;            // the middle row of an odd width is covered by its first half
          c = r + (b - (wd - a));
        }
        const int i = k + 1 + r, j = k + 1 + c;
        G[i * p + j] = fma(-rowk[i], rowk[j], G[i * p + j]);
      }
      const int kc = k + 1;
      const unsigned kmag = s_mag[kc];
      for (int s2 = t1 < 0 ? 0x7fffffff : t1; s2 < wd * kc; s2 += kPcThreads - 32) {
        const int r = small_div(s2, kmag), c = s2 - r * kc;
        const int i = k + 1 + r;
        B[i * p + c] = fma(-rowk[i], B[k * p + c], B[i * p + c]);
      }
      __syncthreads();
    }
    __syncthreads();
    if (s_fail) {
      if (attempt == 1) break;                     // even the shifted matrix failed: no preconditioner
      if (threadIdx.x == 0) st->singular = 1;      // singular at working precision: refactor with the shift
      __syncthreads();
      continue;
    }
    // M = B^T, in place (Mm then holds M = R^{-1}, upper triangular)
    for (int q = threadIdx.x; q < p * p; q += kPcThreads) {
      const int i = small_div(q, pmag), j = q - i * p;
      if (i < j) {
        Mm[i * p + j] = Mm[j * p + i];
        Mm[j * p + i] = 0.0;
      }
    }
    __syncthreads();
    cond = estimate();
    break;
  }
  const int ok = want_precond && !st->no_precond && !s_fail;
  const bool trusted = ok && !s_shift && cond * cond * ueps <= 0.25;
  if (ok) store();
  // A float64 solve whose Gram factor is not trusted (or that asks for it): precondition with the R factor of a
  // Householder QR of rows of X sampled evenly, the row-sampling idea of Section 3.1 put to use as a
  // preconditioner. R from QR carries errors of order kappa u, not kappa^2 u, so LSQR on X R^{-1} converges in
  // a few tens of iterations up to kappa(X) ~ 1/u. The Gram factor stays if the sample is rank deficient.
  bool qr_used = false;
  if (want_precond && !st->no_precond && (want_precond == 2 || (!trusted && want_precond != 3)) && w.qr &&
      p <= kQrMaxP && w.m >= (long long)kQrRowsPerP * p) {
    if (sampled_qr(w, G, qw, qpart, scratch)) {
      cond = invert_and_estimate();
      store();
      qr_used = true;
    }
  }
  if (threadIdx.x == 0) {
    if (ok || qr_used) {
      st->precond = qr_used ? 2 : 1;
      st->cond_est = cond;
      // the sampled R is about sqrt(c / m) times the full one, so ||X||_2 ||R_s^{-1}||_2 overstates kappa(X) by
      // sqrt(m / c)
      st->kappa_est = qr_used ? cond * sqrt((double)(kQrRowsPerP * p) / (double)w.m) : cond;
      st->shifted = qr_used ? 0 : s_shift;
      st->trusted = qr_used ? 0 : trusted;
    } else {
      st->precond = 0;
      st->cond_est = 0.0;
    }
  }
}

__global__ void __launch_bounds__(kPcThreads, 1) precond_kernel(Work w, int want_precond, int use_smem) {
  extern __shared__ double psm[];
  precond_body(w, want_precond, use_smem ? psm : nullptr);
}
__global__ void __launch_bounds__(kPcThreads, 1) precond_batch_kernel(const BatchSeries* series, int want_precond,
                                                                 int use_smem) {
  extern __shared__ double psm[];
  precond_body(series[blockIdx.x].w, want_precond, use_smem ? psm : nullptr);
}

static size_t precond_smem(int p_max) {
  const int q = p_max < kPrecondSmemP ? p_max : kPrecondSmemP;
  return sizeof(double) * 2 * (size_t)q * q;
}
static cudaError_t precond_config() {
  // dynamic plus static shared memory must stay within the per-CTA limit: ask for exactly the largest need
  const int bytes = (int)precond_smem(kPrecondSmemP);
  cudaError_t e = smem_opt_in((const void*)precond_kernel, bytes);
  if (e == cudaSuccess) e = smem_opt_in((const void*)precond_batch_kernel, bytes);
  return e;
}

cudaError_t launch_precond(Work w, int want_precond, cudaStream_t s) {
  cudaError_t e = precond_config();
  if (e != cudaSuccess) return e;
  const int use = w.p <= kPrecondSmemP;
  precond_kernel<<<1, kPcThreads, use ? precond_smem(w.p) : 0, s>>>(w, want_precond, use);
  return cudaGetLastError();
}
// Batched: series with p <= kPrecondSmemP work in shared memory sized for the largest such p in the batch.
cudaError_t launch_precond_batch(const BatchSeries* series, int count, int want_precond, cudaStream_t s,
                                 int p_max) {
  cudaError_t e = precond_config();
  if (e != cudaSuccess) return e;
  precond_batch_kernel<<<count, kPcThreads, precond_smem(p_max), s>>>(series, want_precond, 1);
  return cudaGetLastError();
}

// Start of a solve. With a trusted (unshifted, kappa(R)^2 u <= 1/4) Cholesky factor of the float64 Gram matrix:
// start from the semi-normal-equation solution phi0 = R^{-1} R^{-T} X^T b (O(p^2)) and let a float64 check pass
// decide whether more is needed. Otherwise LSQR from zero on b with float64 products.
// A mixed solve takes the same route. Its float products serve only the correction sweeps that may follow a
// check (Bidiag 2 on (X^T X) delta = g), and only when they can contract the error: a trusted factor and
// kappa(X) u32 <= 1e-2 (a sweep then gains about -log10(kappa(X) u32) digits). Otherwise the state drops its
// mixed flag and every later pass is a float64 one.
__device__ void start_solve(const Work& w, DevState* st, double* scratch) {
  for (int j = threadIdx.x; j < w.p; j += kThreads) w.phi[j] = 0.0;
  __syncthreads();
  if (st->precond == 2 && threadIdx.x == 0) st->iter_cap = min(st->iter_cap, kQrIterCap);
  if (st->mixed) {
    const bool float_ok = st->precond && st->trusted && !st->singular && st->kappa_est * 5.96e-8 <= 1e-2;
    __syncthreads();
    if (!float_ok && threadIdx.x == 0) {
      st->mixed = 0;
      st->iter_cap = st->max_iter;
    }
    __syncthreads();
  }
  if (st->precond && st->trusted) {
    apply_Mt(w, 1, 0, w.h, w.t);
    __syncthreads();
    apply_M_exact(w, 1, 0, w.t, w.phi);
    __syncthreads();
    schedule_check(w, st, scratch);
    return;
  }
  start_lsqr(w, st, w.h, st->bnorm, scratch);
}

__global__ void __launch_bounds__(kThreads) init_lsqr_kernel(Work w) {
  __shared__ double scratch[16];
  DevState* st = w.st;
  for (int j = threadIdx.x; j < w.p; j += kThreads) w.phi[j] = 0.0;
  __syncthreads();
  if (st->done) return;   // e.g. non-finite input found by the preconditioner
  start_solve(w, st, scratch);
}

// Warm start: phi already holds a guess; the first pass is a residual check.
__global__ void __launch_bounds__(kThreads) init_check_kernel(Work w) {
  __shared__ double scratch[16];
  schedule_check(w, w.st, scratch);
}

__global__ void __launch_bounds__(kThreads) init_lsqr_batch_kernel(const BatchSeries* series, unsigned int* done) {
  __shared__ double scratch[16];
  const Work& w = series[blockIdx.x].w;
  DevState* st = w.st;
  if (st->done) {  // e.g. non-finite input found by the preconditioner kernel
    if (threadIdx.x == 0 && done) atomicAdd(done, 1u);
    return;
  }
  for (int j = threadIdx.x; j < w.p; j += kThreads) w.phi[j] = 0.0;
  __syncthreads();
  start_solve(w, st, scratch);
}
cudaError_t launch_init_lsqr_batch(const BatchSeries* series, int count, unsigned int* done, cudaStream_t s) {
  init_lsqr_batch_kernel<<<count, kThreads, 0, s>>>(series, done);
  return cudaGetLastError();
}

cudaError_t launch_init_lsqr(Work w, int warm, cudaStream_t s) {
  if (warm) init_check_kernel<<<1, kThreads, 0, s>>>(w);
  else init_lsqr_kernel<<<1, kThreads, 0, s>>>(w);
  return cudaGetLastError();
}

// Copy the best iterate into phi when the solve did not converge.
__global__ void finish_kernel(Work w) {
  DevState* st = w.st;
  if (st->status != TOLS_OK && st->ne_best < st->ne_ratio) {
    for (int j = threadIdx.x; j < w.p; j += blockDim.x) w.phi[j] = w.best[j];
    __syncthreads();
    if (threadIdx.x == 0) { st->ne_ratio = st->ne_best; st->rnorm = st->rnorm_best; }
  }
}
__global__ void finish_batch_kernel(const BatchSeries* series) {
  const Work& w = series[blockIdx.x].w;
  DevState* st = w.st;
  if (st->status != TOLS_OK && st->ne_best < st->ne_ratio) {
    for (int j = threadIdx.x; j < w.p; j += blockDim.x) w.phi[j] = w.best[j];
    __syncthreads();
    if (threadIdx.x == 0) { st->ne_ratio = st->ne_best; st->rnorm = st->rnorm_best; }
  }
}
// Copy each series' state and phi into contiguous arrays (phi at stride `stride`).
__global__ void gather_batch_kernel(const BatchSeries* series, DevState* states, double* phis, int stride) {
  const Work& w = series[blockIdx.x].w;
  for (int j = threadIdx.x; j < w.p; j += blockDim.x) phis[(size_t)blockIdx.x * stride + j] = w.phi[j];
  if (threadIdx.x == 0) states[blockIdx.x] = *w.st;
}
cudaError_t launch_gather_batch(const BatchSeries* series, int count, DevState* states, double* phis, int stride,
                                cudaStream_t s) {
  gather_batch_kernel<<<count, 128, 0, s>>>(series, states, phis, stride);
  return cudaGetLastError();
}

// float copies of every series of a batch (one CTA per series)
__global__ void convert_batch_kernel(const BatchSeries* series) {
  const Work& w = series[blockIdx.x].w;
  for (long long i = threadIdx.x; i < w.n; i += blockDim.x) w.y32[i] = (float)w.y64[i];
}
cudaError_t launch_convert_batch(const BatchSeries* series, int count, cudaStream_t s) {
  convert_batch_kernel<<<count, 512, 0, s>>>(series);
  return cudaGetLastError();
}

cudaError_t launch_finish_batch(const BatchSeries* series, int count, cudaStream_t s) {
  finish_batch_kernel<<<count, kThreads, 0, s>>>(series);
  return cudaGetLastError();
}

cudaError_t launch_finish(Work w, cudaStream_t s) {
  finish_kernel<<<1, kThreads, 0, s>>>(w);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------------
__global__ void convert_f32_kernel(const double* __restrict__ y, float* __restrict__ y32, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y32[i] = (float)y[i];
}
cudaError_t launch_convert_f32(const double* y, float* y32, long long n, cudaStream_t s) {
  const int grid = (int)lmin((n + 255) / 256, 152 * 16);
  convert_f32_kernel<<<grid, 256, 0, s>>>(y, y32, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------------
// Row norms of X (a float64 scan of y^2 local to each tile, so that cancellation is bounded by the tile):
//   rn2[i] = sum_{t=i}^{i+p-1} y[t]^2,  ||X||_F^2 = sum_i rn2[i].
constexpr int kScanTile = 2048;
__global__ void __launch_bounds__(kThreads) row_norms_kernel(const double* __restrict__ y, long long n, int p,
                                                             double* __restrict__ rn2, double* part) {
  extern __shared__ double sq[];  // kScanTile + p + 1
  __shared__ double scratch[16];
  const long long m = n - p;
  const long long i0 = (long long)blockIdx.x * kScanTile;
  const int rows = (int)min((long long)kScanTile, m - i0);
  const int len = rows + p;  // y[i0 .. i0+rows+p-1]
  // inclusive prefix of y^2 over the window, in shared memory: sq[q+1] = sum_{s<=q} y[i0+s]^2
  const int per = (len + kThreads - 1) / kThreads;
  const int beg = threadIdx.x * per, end = min(len, beg + per);
  double run = 0.0;
  for (int q = beg; q < end; ++q) {
    const double v = y[i0 + q];
    run += v * v;
    sq[q + 1] = run;
  }
  // exclusive scan of per-thread totals
  __shared__ double tot[kThreads];
  tot[threadIdx.x] = run;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int k = 0; k < kThreads; ++k) { const double t = tot[k]; tot[k] = acc; acc += t; }
    sq[0] = 0.0;
  }
  __syncthreads();
  const double off = tot[threadIdx.x];
  for (int q = beg; q < end; ++q) sq[q + 1] += off;
  __syncthreads();
  double loc = 0.0;
  for (int r = threadIdx.x; r < rows; r += kThreads) {
    const double v = sq[r + p] - sq[r];
    if (rn2) rn2[i0 + r] = v;
    loc += v;
  }
  loc = block_sum(loc, scratch);
  if (threadIdx.x == 0) part[blockIdx.x] = loc;
}

__global__ void sum_parts_kernel(const double* part, int count, double* out) {
  __shared__ double scratch[16];
  double s = 0.0;
  // fixed order: each thread a contiguous chunk, then the block sum
  const int per = (count + kThreads - 1) / kThreads;
  for (int q = threadIdx.x * per; q < min(count, (int)(threadIdx.x + 1) * per); ++q) s += part[q];
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) *out = s;
}

cudaError_t launch_row_norms(const double* y, long long n, int p, double* rn2, double* fro2_dev, double* scratch,
                             cudaStream_t s) {
  const long long m = n - p;
  const int blocks = (int)((m + kScanTile - 1) / kScanTile);
  const size_t smem = sizeof(double) * (kScanTile + p + 2);
  cudaError_t e = cudaFuncSetAttribute(row_norms_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  if (e != cudaSuccess) return e;
  row_norms_kernel<<<blocks, kThreads, smem, s>>>(y, n, p, rn2, scratch);
  sum_parts_kernel<<<1, kThreads, 0, s>>>(scratch, blocks, fro2_dev);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------------
// Leverage scores (Section 3.1).
constexpr int kLevTile = 4096;
__global__ void __launch_bounds__(kThreads) sumsq_kernel(const double* __restrict__ y, long long cnt, double* part) {
  __shared__ double scratch[16];
  const long long i0 = (long long)blockIdx.x * kLevTile;
  double s = 0.0;
  for (long long i = i0 + threadIdx.x; i < min(cnt, i0 + kLevTile); i += kThreads) s = fma(y[i], y[i], s);
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void lev_p1_kernel(const double* __restrict__ y, long long cnt, const double* total, double* lev) {
  const double inv = 1.0 / *total;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x)
    lev[i] = y[i] * y[i] * inv;
}
cudaError_t launch_leverage_p1(const double* y, long long n, double* lev, double* scratch, cudaStream_t s) {
  const long long cnt = n - 1;
  const int blocks = (int)((cnt + kLevTile - 1) / kLevTile);
  sumsq_kernel<<<blocks, kThreads, 0, s>>>(y, cnt, scratch + 1);
  sum_parts_kernel<<<1, kThreads, 0, s>>>(scratch + 1, blocks, scratch);
  const int grid = (int)lmin((cnt + 255) / 256, 152 * 16);
  lev_p1_kernel<<<grid, 256, 0, s>>>(y, cnt, scratch, lev);
  return cudaGetLastError();
}

// lev[i] = lev_prev[i] + r[i]^2 / ||r||^2, pi[i] = lev[i] / p; r stored by a pass, ||r||^2 in *rr.
__global__ void lev_update_kernel(const double* __restrict__ r, long long m, const double* rr,
                                  const double* __restrict__ lev_prev, double* lev, double* pi, int p) {
  const double inv = 1.0 / *rr;
  const double invp = 1.0 / (double)p;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const double v = fma(r[i] * r[i], inv, lev_prev[i]);
    lev[i] = v;
    if (pi) pi[i] = v * invp;
  }
}
cudaError_t launch_leverage_step(const double* r, long long m, int p, const double* rr, const double* lev_prev,
                                 double* lev, double* pi, double* /*unused*/, cudaStream_t s) {
  const int grid = (int)lmin((m + 255) / 256, 152 * 16);
  lev_update_kernel<<<grid, 256, 0, s>>>(r, m, rr, lev_prev, lev, pi, p);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------------
__global__ void check_finite_kernel(const double* __restrict__ y, long long n, int* flag) {
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(y[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}
cudaError_t launch_check_finite(const double* y, long long n, int* flag, cudaStream_t s) {
  const int grid = (int)lmin((n + 255) / 256, 152 * 8);
  check_finite_kernel<<<grid, 256, 0, s>>>(y, n, flag);
  return cudaGetLastError();
}

}  // namespace tols
