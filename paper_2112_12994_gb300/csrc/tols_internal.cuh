// Internal declarations of the Toeplitz-OLS CUDA library (sm_103a).
//
// Notation (0-based): series y[0..n-1], order p, m = n - p rows,
//   X[i][j] = y[p + i - j - 1],  b[i] = y[p + i]                       (eq. (xphi), Section 3).
// The kernels index the lags by k = p - 1 - j, so that
//   (X d)[i]     = sum_k y[i + k] * d[p - 1 - k]
//   (X^T u)[j]   = sum_i u[i] * y[i + p - 1 - j] = tk[p - 1 - j],  tk[k] = sum_i u[i] * y[i + k].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/toeplitz_ols.h"

namespace tols {

constexpr int kThreads = 256;            // threads per CTA of every pass kernel
constexpr int kGroup = 16;               // CTAs per first-level reduction group
constexpr int kMaxGrid = 152 * 4;        // upper bound on pass grid size (partials buffer rows)
constexpr int kMaxGroups = (kMaxGrid + kGroup - 1) / kGroup;

// 1/sqrt(x) for x > 0 in float64 by Newton-Raphson for f(r) = 1/r^2 - x (r <- r (3 - x r^2) / 2), started from
// the float reciprocal square root: two steps take the 24-bit start to full float64 accuracy (quadratic
// convergence). A short chain of FP64 operations, where sqrt followed by a division is a long one.
// x is first scaled by an even power of two into [1, 4) (exponent arithmetic on the bits), so the float start
// never overflows or underflows.
__device__ __forceinline__ double rsqrt_newton(double x) {
  const long long bits = __double_as_longlong(x);
  const int ef = (int)((bits >> 52) & 0x7ff);
  if (ef == 0 || ef == 0x7ff) return 1.0 / sqrt(x);         // zero, subnormal, inf, nan: the plain way
  const int kk = (ef - 1023) >> 1;                           // x = xs 4^kk, xs in [1, 4)
  const double xs = __longlong_as_double(bits - ((long long)(2 * kk) << 52));
  double r = (double)rsqrtf((float)xs);
  r = r * fma(-0.5 * xs, r * r, 1.5);
  r = r * fma(-0.5 * xs, r * r, 1.5);
  return __longlong_as_double(__double_as_longlong(r) - ((long long)kk << 52));   // r 2^-kk
}

// Round p up to the lag-chunk granularity used by the direct kernels.
__host__ __device__ constexpr int pad_p(int p) { return (p + 15) & ~15; }

// One-CTA preconditioner (precond_kernel): it factors in shared memory up to this order, leaving G in global memory
// untouched. Its want_precond: 0 none, 1 the Gram factor (the sampled-row QR when that is not trusted), 2 the
// sampled-row QR, 3 the Gram factor only (no QR; the caller reads DevState::trusted).
constexpr int kPrecondSmemP = 112;

// Sampled-row QR preconditioner: orders it serves and rows sampled per coefficient; its scratch (doubles).
constexpr int kQrMaxP = 256;
constexpr int kQrRowsPerP = 8;
__host__ __device__ constexpr size_t qr_scratch_doubles(int p) {
  return p <= kQrMaxP ? (size_t)kQrRowsPerP * p * (p + 1) : 0;   // the sampled rows, then a Householder vector
}

// What the last CTA of a pass does after the grid-wide reduction (see tails in tols_kernels.cu).
enum TailMode : int {
  TAIL_STORE = 0,    // write the reduced X^T u and ||u||^2 to out_t / out_n2
  TAIL_LSQR = 1,     // LSQR (Golub-Kahan Bidiag 1 + Givens) scalar step
  TAIL_NECORR = 2,   // Golub-Kahan Bidiag 2 step for the normal-equation correction (X^T X) delta = g
  TAIL_CHECK = 3,    // float64 residual check: g = X^T r, ||r||, ne ratio; mixed: start the next correction
  TAIL_GRAM = 4,     // Gram matrix from lag sums plus edge corrections
};

// Phases of the device-driven solver state machine.
enum Phase : int {
  PH_LSQR = 0,       // iterating LSQR
  PH_CHECK = 1,      // a float64 residual check pass is due
  PH_NECORR = 2,     // iterating the correction solve
  PH_DONE = 3,
};

// Scalars of one solve, resident in device memory. Vectors live in the Work buffers.
struct DevState {
  // LSQR (Paige & Saunders 1982) scalars
  double alpha, beta, rhobar, phibar, anorm2, bnorm, beta1;
  // Bidiag 2 (correction solve) scalars
  double theta, rho, f, theta1;
  // coefficient for the next pass: u_new = X d - coef * u_old
  double coef;
  // norms
  double anorm_f, anorm_2, ne_ratio, rnorm, ne_best, rnorm_best;
  double tol, tol_inner, est_ratio, cond_est;
  double kappa_est;  // estimate of kappa(X) (sampled-QR preconditioner: cond_est sqrt(c / m), c the rows sampled)
  double est_best;   // best (halving) value of the inner solve's stopping estimate, at inner iteration iter_best
  double phibar_mark;  // LSQR residual-norm estimate at the last iteration that made progress
  int iter, max_iter, iter_cap, inner_iter, total_iter, sweeps, max_sweeps, iter_best;
  int phase, status, precond, mixed, mixed_ok;
  int done;          // 1 => every pass kernel returns at once
  int singular;      // the Gram matrix was singular at working precision
  int compatible;    // a check found ||r|| <= tol ||b||
  int shifted;       // the Cholesky factor needed the diagonal shift
  int trusted;       // unshifted factor with kappa(R)^2 u <= 1/4 (semi-normal-equation start, float refinement)
  int fft;           // a batched pass with overlap-save FFT products ran for this series
  int no_precond;    // set by the host: plain LSQR (minimum-norm repeat of a rank-deficient problem)
  int f32_iter;      // inner iterations run with float products (a mixed solve that needed correction sweeps)
  int dev_error;     // a kernel's bounded wait on its own copies gave up (the host reports TOLS_ERR_DEVICE_TIMEOUT)
};

// Device pointers of one solve's workspace.
struct Work {
  long long n, m;
  int p, p_pad;
  const double* y64;      // n doubles
  float* y32;             // n floats (mixed)
  void* U[2];             // ping-pong m-vectors (double in FP64 mode, float in mixed)
  double* part_t;         // [kMaxGrid][p_pad] per-CTA partial X^T u (lag order k)
  double* part_n2;        // [kMaxGrid]
  double* grp_t;          // [kMaxGroups][p_pad]
  double* grp_n2;         // [kMaxGroups]
  unsigned int* counters; // [kMaxGroups + 1]
  // p-vectors (each p_pad doubles)
  double *v, *w, *z, *d, *phi, *g, *h, *t, *best;
  double* G;              // p*p Gram matrix (row-major), later overwritten by R
  double* M;              // p*p upper-triangular R^{-1} (row-major)
  double* Mt;             // p*p its transpose (row-major)
  float* M32;             // float copies for the mixed path
  float* Mt32;
  double* bnorm2;         // device scalar ||b||^2 written by the Gram pass
  double* qr;             // (nullable) float64 scratch of the sampled-row QR preconditioner (p <= 256): the sampled
                          // rows (kQrRowsPerP p x p) and a Householder vector
  DevState* st;
  const void* tw32;       // FFT twiddles exp(-2 pi i t / 4096), t < 4096 (float2)
  const void* tw64;       // FFT twiddles exp(-2 pi i t / 2048), t < 2048 (double2)
  const void* tw64x;      // FFT twiddles exp(-2 pi i t / 4096), t < 4096 (double2): float64 passes with N = 4,096
  void* wspec32;          // doubled window spectra of the float FFT tiles ([tiles][N/2 + 1]; FFT passes only)
  void* wspec64;          // the same for the float64 FFT tiles
  void* sacc32;           // (float FFT passes) per-CTA sums of W . conj(U) as float pairs: [kMaxGrid][N/2 + 1] float4
  void* dspec64;          // (batched float64 FFT series) doubled spectrum of the lag-reversed d, N/2 + 1 entries
  unsigned int* f32_active;  // (batches, nullable) count of the batch's series in a float correction sweep
};

// Arguments of a pass kernel (passed by value).
template <typename T>
struct PassArgs {
  const T* y;             // series, n elements (the window of row i is y[i .. i+p-1])
  long long n, m;
  int p, p_pad;
  int nlag;               // number of lags in the correlation (p for X^T u, p+1 for the Gram lag sums)
  int gram;               // 1: correlation of y with itself (u := y[i]), no X d product
  const double* d;        // p-vector (device) for X d; lag-reversed internally
  double d_scale;         // the pass multiplies by d_scale * d
  const T* u_old;         // nullable
  T* u_new;               // nullable
  const double* coef_dev; // device scalar c (nullable => coef_host)
  double coef_host;
  int tail;               // TailMode
  Work w;                 // workspace (for the reduction buffers and the tails)
  double* out_t;          // TAIL_STORE: reduced X^T u (p, j order)
  double* out_n2;         // TAIL_STORE: reduced ||u||^2 (1)
  int check_done;         // 1: return at once when w.st->done is set
  int* worklog;           // nullable: the tail writes 1 + tail + 5 * (T == double) into worklog[work_slot]
  int work_slot;
  int fft;                // 0: direct products; N: overlap-save FFT products of length N (float 4,096; float64
                          // 2,048 or 4,096)
  int wait_polls;         // poll limit of the kernel's waits on its own bulk copies (0: the default, about 2 s;
                          // negative: none, every such wait gives up at once)
};

// One series of a batch (device array). Its Work points at the series' own slices of the batch buffers; its
// partial buffers hold one row per tile (of the float64 tile size, the larger count).
struct BatchSeries {
  Work w;
  long long tile0_f, tile0_d;   // first index of this series in the float / double tile lists
  long long tile0_x;            // first index in the float64 FFT unit list (series with w.dspec64 set)
};

// Arguments of a batched pass launch.
struct BatchArgs {
  const BatchSeries* series;
  const int* tile_series_f;     // float tile list: tile -> series
  const int* tile_series_d;     // double tile list: tile -> series
  long long tiles_f, tiles_d;
  const int* tile_series_x;     // float64 FFT unit list (kBatchFftUnit tiles each): unit -> series
  long long tiles_x;            // units in that list
  int gram;                     // 1: Gram lag-sum pass (TAIL_GRAM) instead of a solver pass
  unsigned int* done_count;     // incremented once per series that reaches PH_DONE
  const long long* live;        // (nullable) device counts {tiles_f, tiles_d, tiles_x} of the lists as they are now:
                                // the host compacts the lists to the unfinished series between graph replays, so
                                // a kernel reads its count at run time (tiles_f, tiles_d, tiles_x size the grid)
};

// Batched series with p_pad(p + 1) in [32, 1024) take the overlap-save float64 FFT products (N = 2,048, tiles of
// 2,048 - pad_p(p + 1) rows) for their Gram pass, checks and float64 iterations; the others the direct products.
// The float correction sweeps of mixed series use the direct float products.
constexpr int kBatchFftN = 2048;
__host__ __device__ constexpr bool batch_fft_series(int p) {
  return pad_p(p + 1) >= 32 && pad_p(p + 1) < kBatchFftN / 2;
}
__host__ __device__ constexpr long long batch_fft_tiles(long long m, int p) {
  return (m + (kBatchFftN - pad_p(p + 1)) - 1) / (kBatchFftN - pad_p(p + 1));
}
// Work unit of the batched FFT pass: up to kBatchFftUnit consecutive tiles of one series, whose X^T u spectra are
// summed and transformed back once (a fixed grouping per series, so results do not depend on the batch).
constexpr int kBatchFftUnit = 4;
__host__ __device__ constexpr long long batch_fft_units(long long m, int p) {
  return (batch_fft_tiles(m, p) + kBatchFftUnit - 1) / kBatchFftUnit;
}
__host__ __device__ constexpr size_t batch_fft_spectra_doubles(long long m, int p) {
  return (size_t)batch_fft_tiles(m, p) * (kBatchFftN / 2 + 1) * 2;
}

// Launch helpers (tols_kernels.cu).
cudaError_t smem_opt_in(const void* fn, int bytes);   // per-device dynamic shared-memory opt-in, set once
size_t pass_smem_bytes(int is_double, int p_pad, int nfft = 0);   // nfft: 0 (direct products) or the FFT length
const void* fft_kernel_ptr(int is_double, int nfft);
int fft_size(int is_double);              // default N of the real FFT per tile (float 4096, double 2048)
size_t fft_spectra_bytes(int is_double, long long m, int p_pad, int nfft);
size_t fft32_sum_bytes();                 // the float FFT pass's per-CTA float64 sum buffer (Work::sacc32)
cudaError_t launch_spectra(int is_double, const void* y, long long n, long long m, int p_pad, void* out,
                           const void* tw, int grid, cudaStream_t s, int nfft);
int pass_tile_rows(int is_double);
const void* pass_kernel_ptr(int is_double);
template <typename T>
cudaError_t launch_pass(const PassArgs<T>& a, int grid, cudaStream_t s);

template <typename T>
cudaError_t launch_batch_pass(const BatchArgs& a, int grid, int p_pad_max, cudaStream_t s);
const void* batch_kernel_ptr(int is_double);
cudaError_t launch_batch_fft(const BatchArgs& a, int grid, int p_pad_max, cudaStream_t s);
cudaError_t launch_batch_dspec(const BatchSeries* series, int count, cudaStream_t s);
const void* batch_fft_kernel_ptr();
size_t batch_fft_smem(int p_pad_max);
cudaError_t launch_precond_batch(const BatchSeries* series, int count, int want_precond, cudaStream_t s,
                                 int p_max);
cudaError_t launch_init_lsqr_batch(const BatchSeries* series, int count, unsigned int* done, cudaStream_t s);
cudaError_t launch_finish_batch(const BatchSeries* series, int count, cudaStream_t s);
cudaError_t launch_convert_batch(const BatchSeries* series, int count, cudaStream_t s);
cudaError_t launch_convert_f32(const double* y, float* y32, long long n, cudaStream_t s);
cudaError_t launch_precond(Work w, int mixed, cudaStream_t s);
cudaError_t launch_init_lsqr(Work w, int mixed, cudaStream_t s);
cudaError_t launch_finish(Work w, cudaStream_t s);
cudaError_t launch_prepare_check(Work w, cudaStream_t s);
cudaError_t launch_row_norms(const double* y, long long n, int p, double* rn2, double* fro2_dev, double* scratch,
                             cudaStream_t s);
cudaError_t launch_leverage_p1(const double* y, long long n, double* lev, double* scratch, cudaStream_t s);
cudaError_t launch_leverage_step(const double* r, long long m, int p, const double* rr, const double* lev_prev,
                                 double* lev, double* pi, double* unused, cudaStream_t s);
cudaError_t launch_check_finite(const double* y, long long n, int* flag, cudaStream_t s);

// Multi-CTA preconditioner of single-series solves (tols_precond.cu); the host runs its steps (tols_api.cu).
struct PclInfo {
  int fail;             // a pivot of the running factorisation fell to its floor
  int nonfinite;        // a trace or lambda_max was not finite
  double lam, dmax, trace, shift;   // the last power iteration: lambda_max, largest diagonal entry, trace, shift
  double lam_keep[2];   // lambda_max of G (||X||_2^2) and of the sample's Gram matrix (QR path)
  double trace_g;       // trace of G (||X||_F^2)
  double cond;          // the last kappa(R) estimate
};
constexpr int kPclTile = 32;
__host__ __device__ constexpr int pcl_pad_p(int p) { return (p + kPclTile - 1) / kPclTile * kPclTile; }
cudaError_t pcl_lambda(double* S, int ld, int p, double shift_rel, int keep, float* fb, PclInfo* info, cudaStream_t s);
cudaError_t pcl_pad(const double* G, int p, double* Gp, int P, double shift, double* Gsave, cudaStream_t s);
cudaError_t pcl_chol_panel(double* Gp, int P, int p, int k, double tiny_dmax, double tiny_shift, PclInfo* info,
                           cudaStream_t s);
cudaError_t pcl_chol_update(double* Gp, int P, int k, const PclInfo* info, cudaStream_t s);
cudaError_t pcl_inverse(const double* Rp, int P, int p, double* M, const PclInfo* info, cudaStream_t s);
cudaError_t pcl_estimate(const double* M, int p, int slot, float* fb, PclInfo* info, cudaStream_t s);
cudaError_t pcl_store(const Work& w, int mixed, const PclInfo* info, cudaStream_t s);
cudaError_t pcl_state(const Work& w, const PclInfo* info, int precond, int shifted, int trusted, int singular,
                      double cond, double kappa_est, cudaStream_t s);
cudaError_t pcl_gather(const double* y, long long m, int p, long long c, double* A, cudaStream_t s);
int pcl_gram_slices(long long c, int P);
cudaError_t pcl_tall_gram(const double* A, long long c, int p, int P, int slices, double* part, cudaStream_t s);
cudaError_t pcl_gram_reduce(const double* part, int P, int slices, int p, double* Gp, cudaStream_t s);
cudaError_t pcl_trsm(double* A, long long c, int p, const double* Rp, int P, cudaStream_t s);
cudaError_t pcl_trmm(const double* X, const double* Y, double* Z, int P, cudaStream_t s);

// Algorithm "LSAR" (Section 3.1), tols_lsar.cu.
constexpr int kLsarMaxP = 256;          // largest p_bar
constexpr int kLsarBlock = 512;         // rows per sampling block (one warp scans it in 16 chunks of 32)
constexpr int kLsarChunk = 16;          // sampled rows staged in shared memory at a time by the Gram kernel
constexpr int kLsarSolveThreads = 512;  // threads of the one-CTA Cholesky solve
constexpr int kLsarSmemP = 144;         // the solve keeps its Cholesky factor in shared memory up to this order
constexpr int kLsarFftMinOrder = 32;    // full-data residual by the FFT pass from this order (and 2^16 rows) up
__host__ __device__ constexpr long long lsar_tri(int p) { return (long long)(p + 1) * (p + 2) / 2; }
size_t lsar_chol_smem(int p);
size_t lsar_correct_smem(int p);
size_t lsar_gram_smem(int p);
cudaError_t launch_lsar_lev(const double* r, const double* rr, double* lev, long long m, double* bsum,
                            const int* status, cudaStream_t s);
cudaError_t launch_lsar_prefix(const double* bsum, long long nb, double* bpre, const int* status, cudaStream_t s);
cudaError_t launch_lsar_sample(const double* lev, long long m, const double* bsum, const double* bpre,
                               const double* unif, int c, int p, long long* rows, double* w2, const int* status,
                               cudaStream_t s);
cudaError_t launch_lsar_gram(const double* y, int p, const long long* rows, const double* w2, int c, int ng,
                             double* part, double* G, const int* status, cudaStream_t s);
cudaError_t launch_lsar_solve(const double* G, int p, const double* y, const long long* rows, const double* w2,
                              int c, int ng, double* Lg, double* rdg, double* gpart, double* phi, double* tau,
                              int lag, int* status, cudaStream_t s);
// Algorithm "Repeated Halving" (Section 3.2), tols_lsar.cu.
constexpr int kRhMaxSketch = 64;        // largest sketch height k
size_t rh_sketch_smem(int P1);
cudaError_t launch_rh_map(const long long* in, const long long* keep, long long cnt, long long* out, cudaStream_t s);
cudaError_t launch_rh_fill(double* x, long long cnt, double v, cudaStream_t s);
cudaError_t launch_rh_factor(const double* G, int P1, double* Lg, double* rdg, int code, int* status,
                             cudaStream_t s);
cudaError_t launch_rh_sketch(const double* y, int P1, const long long* rows, const double* w2, int cnt,
                             const double* S, int k, const double* Lg, const double* rdg, double* M, int* status,
                             cudaStream_t s);
cudaError_t launch_rh_score(const double* y, int P1, const double* M, int k, const long long* list, long long cnt,
                            double* score, const int* status, cudaStream_t s);
// Algorithm "SRHT" (Section 2.1), tols_lsar.cu.
cudaError_t launch_srht_transform(const double* y, int p, long long m, long long m2, const double* signs, double* Z,
                                  cudaStream_t s);
cudaError_t launch_srht_gram(const double* Z, long long m2, int p, const long long* rows, int c, double sc, int ng,
                             double* part, double* G, int* status, cudaStream_t s);
cudaError_t launch_srht_solve(const double* G, int p, double* Lg, double* rdg, double* phi, int* status,
                              cudaStream_t s);

}  // namespace tols
