/*
 * toeplitz_ols.h — C ABI of the GB300 (sm_103a) Toeplitz least-squares / AR(p) solver.
 *
 * Problem (eq. (xphi), Section 3; Def. "Ordinary Least Squares Problem", Section 2). For a series
 * y[0..n-1], an order p >= 1 and m = n - p rows,
 *
 *     X[i][j] = y[p + i - j - 1],   b[i] = y[p + i],   i in [0, m), j in [0, p),
 *
 *     phi* = argmin_phi || X phi - b ||_2     (minimum-norm when X is rank deficient, Thm. "Solution to OLS
 *                                              problem").
 *
 * X is never formed: a Toeplitz matrix is fixed by its first row and column (Section 3), here by y[0 .. n-2],
 * and b by y[p .. n-1].
 *
 * Conventions for every function below:
 *   - Return 0 (TOLS_OK) on success, TOLS_NOT_CONVERGED (> 0, a warning) or a negative TOLS_ERR_* code.
 *   - "host" pointers are ordinary CPU memory owned by the caller; the library copies what it needs and keeps
 *     no caller pointer after the call returns.
 *   - "device" pointers are global memory on the context's GPU (e.g. a torch tensor's data_ptr()); they are
 *     read/written on the context's stream, and the call returns after that stream work has completed.
 *   - All arrays are dense and contiguous; vectors of length p are indexed by j = 0..p-1 as in phi_{j+1}.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef TOEPLITZ_OLS_H
#define TOEPLITZ_OLS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------------------- */
#define TOLS_OK 0
#define TOLS_NOT_CONVERGED 1        /* warning: phi holds the last iterate, info holds the achieved ratio   */
#define TOLS_ERR_ARG (-1)           /* null pointer, n <= p, p < 1, p > TOLS_MAX_P, bad enum                 */
#define TOLS_ERR_NONFINITE (-2)     /* y holds NaN or Inf                                                    */
#define TOLS_ERR_OOM (-3)           /* device or pinned-host allocation failed, or mem_cap_bytes exceeded   */
#define TOLS_ERR_CUDA (-4)          /* a CUDA runtime call failed; the message is in toeplitz_ols_last_error */
#define TOLS_ERR_DEVICE_TIMEOUT (-5)/* a bounded device-side wait gave up                                   */
#define TOLS_ERR_NO_DEVICE (-6)     /* no CUDA device, or the device is not sm_103                          */
#define TOLS_ERR_BUSY (-7)          /* serving: no slot or memory free for this request right now           */

#define TOLS_MAX_P 1024             /* largest order handled                                                */

/* ---- configuration ------------------------------------------------------------------------------- */
typedef enum {
  TOLS_FP64 = 0,   /* every product of X in float64 on the GPU                                               */
  TOLS_MIXED = 1   /* the float64 route (float64 Gram pass, factor and checks) with float32 products in the
                      correction sweeps that follow a check, when kappa(X) u32 <= 1e-2 lets them contract the
                      error; float64 recurrence scalars throughout                                             */
} tols_precision;

typedef enum {
  TOLS_PRECOND_NONE = 0,      /* plain LSQR on X                                                           */
  TOLS_PRECOND_GRAM_CHOL = 1, /* LSQR on X R^{-1}, R the Cholesky factor of the Gram matrix X^T X. A       
                                 solve whose factor is not trustworthy (kappa(R)^2 u > 1/4) switches to
                                 TOLS_PRECOND_SAMPLED_QR by itself (n - p >= 8p)                                */
  TOLS_PRECOND_SAMPLED_QR = 2 /* LSQR on X R^{-1}, R from a float64 QR of 8p to 32p rows of X sampled evenly
                                 (the row-sampling idea of Section 3.1 used as a preconditioner; errors of order
                                 kappa u instead of kappa^2 u; see toeplitz_ols_preconditioner). n - p >= 8p;
                                 otherwise the Gram factor is used                                             */
} tols_precond;

typedef enum {
  TOLS_PRODUCT_AUTO = 0,      /* pick per (n, p, precision)                                               */
  TOLS_PRODUCT_DIRECT = 1,    /* sliding-window dot products                                              */
  TOLS_PRODUCT_FFT = 2,       /* overlap-save FFT blocks of the default length (float 4,096; float64 2,048)  */
  TOLS_PRODUCT_FFT4096 = 3    /* overlap-save FFT blocks of length 4,096 in both precisions               */
} tols_product;

typedef struct {
  int precision;          /* tols_precision                                                                 */
  int device;             /* CUDA device ordinal                                                            */
  size_t mem_cap_bytes;   /* cap on the context's device arena; 0 = no cap                                  */
  int max_iter;           /* cap on LSQR iterations per solve (FP64) / per inner solve (mixed); 0 = 4p+200 */
  int max_sweeps;         /* mixed: cap on float64 residual-correction passes; 0 = 6                        */
  int precond;            /* tols_precond                                                                   */
  int product;            /* tols_product                                                                   */
  void* cuda_stream;      /* cudaStream_t to run on; NULL = a stream owned by the context                   */
  int wait_polls;         /* poll limit of a kernel's wait on its own bulk copies (the float FFT pass); 0 = the
                             default, about two seconds; -1 = no polling, every such wait gives up at once (to
                             test the path). A wait that gives up ends the call with TOLS_ERR_DEVICE_TIMEOUT; the
                             kernel still lets its copies land before it exits, and the context stays usable   */
} tols_config;

/* Per-solve report. ne_ratio and rnorm always come from an explicit float64 pass over the data. */
typedef struct {
  int status;             /* same code the call returned (per series in batched calls)                      */
  int iters;              /* LSQR iterations (FP64) or inner iterations over all sweeps (mixed)             */
  int sweeps;             /* float64 residual passes made                                                   */
  int precision_used;     /* TOLS_MIXED when float32 products did part of the work, else TOLS_FP64          */
  int precond_used;       /* tols_precond actually used (SAMPLED_QR for an ill-conditioned float64 solve,
                             NONE if no factor could be formed)                                               */
  int product_used;       /* tols_product actually used                                                     */
  double ne_ratio;        /* ||X^T r|| / (||X||_2est ||r||), r = b - X phi, from a float64 pass             */
  double rnorm;           /* ||b - X phi||_2 from the same pass                                             */
  double bnorm;           /* ||b||_2                                                                        */
  double anorm_2;         /* estimate of ||X||_2 (power iteration on X^T X, a lower bound)                 */
  double anorm_f;         /* ||X||_F                                                                        */
  double cond_est;        /* max R_jj / min R_jj of the Cholesky factor (a rough lower bound of kappa(X))   */
  long long nfft;         /* FFT length N of the overlap-save product passes (tiles of N - pad16(p + 1) rows);
                             0 with direct products                                                           */
} tols_info;

typedef struct tols_ctx tols_ctx;

/* Fill *cfg with defaults: FP64, device 0, no cap, Gram-Cholesky preconditioner, AUTO product. */
void toeplitz_ols_config_default(tols_config* cfg);

/* Create a context on cfg->device (host pointer cfg, copied). *out receives an opaque handle owned by the
 * caller until toeplitz_ols_destroy. Errors: TOLS_ERR_ARG, TOLS_ERR_NO_DEVICE, TOLS_ERR_CUDA. */
int toeplitz_ols_create(tols_ctx** out, const tols_config* cfg);

/* Free every device and host resource of ctx. NULL is accepted. */
int toeplitz_ols_destroy(tols_ctx* ctx);

/* Text for a status code (static storage). */
const char* toeplitz_ols_strerror(int code);

/* Last detailed error message of ctx (static per context, overwritten by the next failing call). */
const char* toeplitz_ols_last_error(const tols_ctx* ctx);

/* ---- solves ----------------------------------------------------------------------------------------- */

/* Solve the AR(p) least-squares problem of eq. (xphi) for host series y[0..n-1].
 *   tol   : stop when ||X^T r|| <= tol ||X||_2 ||r|| (Thm. "Solution to OLS problem": the normal equation),
 *           checked by a float64 pass; 0 means 1e-12.
 *   phi   : host, p doubles, written on success and on TOLS_NOT_CONVERGED.
 *   rnorm : host, nullable; ||b - X phi||_2.
 *   info  : host, nullable.
 * Errors: TOLS_ERR_ARG, TOLS_ERR_NONFINITE, TOLS_ERR_OOM, TOLS_ERR_CUDA. */
int toeplitz_ols_solve(tols_ctx* ctx, const double* y, long long n, int p, double tol, double* phi,
                       double* rnorm, tols_info* info);

/* Same as toeplitz_ols_solve with y already on the device (d_y, n doubles) and phi written to device memory
 * d_phi (p doubles). Nothing crosses PCIe/C2C except p-sized results copied into *rnorm and *info. */
int toeplitz_ols_solve_device(tols_ctx* ctx, const double* d_y, long long n, int p, double tol, double* d_phi,
                              double* rnorm, tols_info* info);

/* Solve count independent problems (host series y[k][0..n[k]-1], orders p[k]) in one batched launch
 * sequence (each problem is eq. (xphi) for its own series, Section 3). Every pass kernel covers all
 * series at once. Products per series: under TOLS_PRODUCT_AUTO the overlap-save float64 FFT (N = 2,048) or the
 * direct products, chosen per order class pad16(p[k] + 1) by a timing made once per process and device and shared
 * by every context of the process; TOLS_PRODUCT_FFT (or FFT4096) takes the FFT from pad16(p[k] + 1) = 32 up,
 * TOLS_PRODUCT_DIRECT the direct products. The float correction sweeps of a mixed batch use the direct float
 * products. A series' result does not depend on the rest of the batch, nor on the context that solved it.
 * info[k].product_used and nfft report the products a series took.
 * phi[k] (host, p[k] doubles), rnorm (host, count, nullable), info (host, count, nullable).
 * Returns the worst status over the batch; info[k].status holds each series' own code. */
int toeplitz_ols_solve_batched(tols_ctx* ctx, int count, const double* const* y, const long long* n,
                               const int* p, double tol, double* const* phi, double* rnorm, tols_info* info);

/* Same as toeplitz_ols_solve_batched with every series already on the device: d_y is a host array of count
 * device pointers (series k: n[k] doubles), and the coefficients are written to the device array d_phi, series
 * k at d_phi + sum_{j<k} p[j] (zeros for a series rejected with TOLS_ERR_ARG). rnorm / info: host, nullable. */
int toeplitz_ols_solve_batched_device(tols_ctx* ctx, int count, const double* const* d_y, const long long* n,
                                      const int* p, double tol, double* d_phi, double* rnorm, tols_info* info);

/* Order sweep and PACF (Def. "Partial Autocorrelation Function", Section 3, with the order rule of the LSAR
 * algorithm's last step taken on the full data): fits AR(h) for h = 1 .. h_max to the one series y, as one batch;
 * tau[h-1] = the last coefficient of the AR(h) fit, the PACF estimate at lag h; *order = the largest h with
 * |tau[h-1]| >= 1.96 / sqrt(n - h) (n - h: the rows of that fit), 0 if there is none.
 * y: host, n doubles (copied in). tau: host, h_max doubles (caller-owned). order, info (h_max entries): host,
 * nullable. Requires 1 <= h_max <= TOLS_MAX_P and n > h_max (else TOLS_ERR_ARG). Returns, like the batched solve,
 * the worst per-fit code; a fit that failed contributes no lag to the order. */
int toeplitz_ols_pacf(tols_ctx* ctx, const double* y, long long n, int h_max, double tol, double* tau, int* order,
                      tols_info* info);

/* ---- serving: continuous batching of fit requests ----------------------------------------------------
 * A server owns a context and one device arena. Submitted requests (series copied in at submit) wait in FIFO
 * order; each toeplitz_ols_server_step admits waiting requests while fewer than max_active are active and the
 * request's device footprint (about 28 n bytes for a mixed request, 24 n for a float64 one, plus about 8.5 n
 * for the float64 FFT window spectra of a request with p >= 16, plus O(p^2)) fits in the
 * arena, sets the newcomers up, runs one burst of batched iterations over every active request, and retires the
 * finished ones (their memory is free for the next admission at once). A request's arithmetic depends only on
 * its own data, so its result is the same alone or among any other requests. */
typedef struct tols_server tols_server;

typedef struct {
  int precision;          /* tols_precision (default TOLS_MIXED)                                           */
  int device;             /* CUDA device ordinal                                                           */
  size_t arena_bytes;     /* device arena for active requests; 0 = half of the free device memory          */
  int max_active;         /* admission cap on concurrently active requests (default 1024)                  */
  int burst;              /* batched passes per step (default 4)                                           */
  int max_iter, max_sweeps;  /* as in tols_config                                                          */
  void* cuda_stream;      /* cudaStream_t, or NULL for a stream owned by the server                       */
} tols_server_config;

typedef struct {
  long long id;           /* the id given at submit                                                       */
  int status;             /* per-request status code                                                      */
  int p;
  double latency_s;       /* seconds from toeplitz_ols_server_submit to the step that retired it           */
  tols_info info;
} tols_result;

typedef struct {
  long long submitted, completed;
  int active, queued;
  size_t arena_bytes, arena_used;
} tols_server_stats;

void toeplitz_ols_server_config_default(tols_server_config* cfg);
/* Errors: TOLS_ERR_ARG, TOLS_ERR_NO_DEVICE, TOLS_ERR_OOM (the arena could not be allocated). */
int toeplitz_ols_server_create(tols_server** out, const tols_server_config* cfg);
int toeplitz_ols_server_destroy(tols_server* srv);
/* Queue a fit of host series y[0..n-1] at order p (copied; the caller keeps y). TOLS_ERR_OOM if the request
 * could never fit in the arena, TOLS_ERR_ARG for bad sizes. */
int toeplitz_ols_server_submit(tols_server* srv, long long id, const double* y, long long n, int p, double tol);
/* Admit, iterate once, retire (blocks for one burst). *active / *queued (nullable) report the counts after. */
int toeplitz_ols_server_step(tols_server* srv, int* active, int* queued);
/* Move up to max finished results into out[] (host) and their coefficients into phi_out (host, nullable,
 * max * TOLS_MAX_P doubles: result i at phi_out + i * TOLS_MAX_P). *got = number moved. */
int toeplitz_ols_server_poll(tols_server* srv, tols_result* out, double* phi_out, int max, int* got);
int toeplitz_ols_server_stats(tols_server* srv, tols_server_stats* st);

/* ---- streaming series: append samples and re-solve, warm-started from the previous phi ---------------- */
int toeplitz_ols_stream_open(tols_ctx* ctx, int p, double tol, int* handle);
int toeplitz_ols_stream_push(tols_ctx* ctx, int handle, const double* y_chunk, long long len);
int toeplitz_ols_stream_solve(tols_ctx* ctx, int handle, double* phi, double* rnorm, tols_info* info);
int toeplitz_ols_stream_close(tols_ctx* ctx, int handle);

/* ---- hot-path steps, exposed one by one -------------------------------------------------------------
 * Each runs the same kernels the solver runs. All pointers are device pointers unless marked host.
 * precision selects the element type of d_y / d_u_old / d_u_new: TOLS_FP64 -> double, TOLS_MIXED -> float.
 */

/* One fused Golub-Kahan product pass (the products of X used by every LSQR iteration):
 *     u_new = X v - c u_old           (m entries; u_old may be NULL, then the term is dropped)
 *     *unorm2 = ||u_new||^2           (host, accumulated in float64)
 *     xtu = X^T u_new                 (p doubles, device)
 * v: p doubles (device). d_u_new may be NULL (then u_new is only used for the norm and X^T u_new).
 * d_u_old and d_u_new may not alias. */
int toeplitz_ols_gk_pass(tols_ctx* ctx, int precision, const void* d_y, long long n, int p, const double* d_v,
                         const void* d_u_old, double c, void* d_u_new, double* d_xtu, double* unorm2);

/* Allocation-free variant of toeplitz_ols_gk_pass. The paper has no counterpart: this exists for callers that
 * cannot let the library allocate device memory — applications whose device memory is owned by another
 * allocator (a framework's caching allocator, or a pool reserved up front to a fixed budget), where an extra
 * cudaMalloc could fail or break the budget, and latency-critical loops that cannot afford cudaMalloc/cudaFree,
 * which can synchronise the device. It needs no context and calls no allocating routine.
 *   - Same operation and arguments as toeplitz_ols_gk_pass, always with the direct (sliding-window) products, as
 *     toeplitz_ols_gk_pass computes them under TOLS_PRODUCT_DIRECT, except: ||u_new||^2 is written to d_unorm2 (one
 *     double, device), and the call only enqueues work on cuda_stream (a cudaStream_t; NULL = the legacy default
 *     stream) of the current device and returns without waiting: synchronise the stream before reading outputs.
 *   - The cross-CTA partial sums live in one fixed array of about 660 KB inside the library image, present on
 *     every GPU that loads the library until the process exits. Its size limits p to TOLS_NOALLOC_MAX_P; larger
 *     p returns TOLS_ERR_ARG, as do n <= p, a bad precision and null d_y, d_v, d_xtu or d_unorm2.
 *   - The first call on a device looks up that array's device address (cudaGetSymbolAddress) with that device
 *     current; make this first call before any stream capture on that device. The address is kept for the life
 *     of the process and belongs to the device's primary context: do not call this entry point from another
 *     context on that device, nor after cudaDeviceReset.
 *   - Every call on a device shares the one array: calls whose work overlaps on the GPU (different streams, or
 *     different host threads) race and give wrong results. Serialise them (one stream, or events). Each call
 *     clears the arrival counters it relies on before its kernel runs.
 * Errors: TOLS_ERR_ARG, TOLS_ERR_NO_DEVICE (no current device), TOLS_ERR_CUDA (lookup or launch failed). */
#define TOLS_NOALLOC_MAX_P 256
int toeplitz_ols_gk_pass_noalloc(int precision, const void* d_y, long long n, int p, const double* d_v,
                                 const void* d_u_old, double c, void* d_u_new, double* d_xtu, double* d_unorm2,
                                 void* cuda_stream);

/* The Gram matrix G = X^T X (p*p doubles, row-major, device) and h = X^T b (p doubles, device) from one
 * correlation pass over y plus O(p^2) edge corrections; TOLS_MIXED forms the lag sums from float32 products. */
int toeplitz_ols_gram(tols_ctx* ctx, int precision, const double* d_y, long long n, int p, double* d_G,
                      double* d_h, double* bnorm2);

/* The preconditioner of a solve (the factor R of LSQR on X R^{-1}; the row-sampling idea of Section 3.1 supplies
 * the sampled-row variant): from a float64 Gram pass over d_y (n doubles, device); precision TOLS_MIXED gives the
 * same factor (a mixed solve also keeps float copies of it),
 *   kind = TOLS_PRECOND_GRAM_CHOL : R = the Cholesky factor of G = X^T X (shifted by 10 p u max_j G_jj when a pivot
 *                                   falls to rounding level);
 *   kind = TOLS_PRECOND_SAMPLED_QR: if the Gram factor is not trusted (kappa(R)^2 u > 1/4) or always
 *                                   when asked, R from shifted Cholesky QR of c rows of X sampled evenly (row
 *                                   floor((2k + 1) m / (2c)), k < c), c = 32p if m >= 256 p^2, 16p if m >= 128 p^2,
 *                                   else 8p; needs m >= 8p; the Gram factor if that fails.
 * From p = 64 up this runs on every SM (32 x 32 tiles); below, in one CTA (sampled-row Householder QR, p <= 256).
 * d_M (device, p x p doubles, row-major) receives M = R^{-1}, upper triangular. info (host, nullable): precond_used,
 * cond_est (kappa estimate: ||X||_2 ||R^{-1}||_2, or that of the sample for the QR), anorm_2, anorm_f, bnorm.
 * Returns TOLS_NOT_CONVERGED when no factor could be formed (d_M untouched). */
int toeplitz_ols_preconditioner(tols_ctx* ctx, int precision, const double* d_y, long long n, int p, int kind,
                                double* d_M, tols_info* info);

/* Row norms of X: d_rn2[i] = ||X(i,:)||^2 = sum_{t=i}^{i+p-1} y[t]^2 (m doubles, device, nullable) and
 * *fro2 = ||X||_F^2 (host), from a float64 prefix scan of y^2. */
int toeplitz_ols_row_norms(tols_ctx* ctx, const double* d_y, long long n, int p, double* d_rn2, double* fro2);

/* The float64 residual pass used for correction and for the final check:
 *     r = b - X phi (not stored),  d_g = X^T r (p doubles, device),  *rnorm = ||r||_2 (host). */
int toeplitz_ols_residual(tols_ctx* ctx, const double* d_y, long long n, int p, const double* d_phi, double* d_g,
                          double* rnorm);

/* Exact leverage scores for p = 1 (after eq. (FASD), Section 3.1): d_lev[i] = y[i]^2 / sum_{t<n-1} y[t]^2,
 * i in [0, n-1) (device, n-1 doubles). */
int toeplitz_ols_leverage_p1(tols_ctx* ctx, const double* d_y, long long n, double* d_lev);

/* One step of the approximate-leverage recursion, eqs. (FALS)-(FASD), Section 3.1, for order p >= 2:
 * with X', b' the order-(p-1) problem on y[0..n-2] (m = n-p rows) and phi_hat (p-1 doubles, device),
 *     r = X' phi_hat - b',   d_lev[i] = d_lev_prev[i] + r[i]^2 / ||r||^2,   d_pi[i] = d_lev[i] / p,
 * all m doubles on the device (d_lev may equal d_lev_prev; d_pi nullable); *rnorm2 = ||r||^2 (host). */
int toeplitz_ols_leverage_step(tols_ctx* ctx, const double* d_y, long long n, int p, const double* d_phi_hat,
                               const double* d_lev_prev, double* d_lev, double* d_pi, double* rnorm2);

/* Algorithm "LSAR" (Section 3.1): PACF estimates from compressed fits, lags p = 1 .. p_bar, on the device.
 * Every lag uses the same m = n - p_bar rows: lag p fits the order-p problem of eq. (xphi) on y[0 .. m + p).
 *   scores   lag 1: the exact l_1(i) = y[i]^2 / sum_{t<m} y[t]^2; lag p >= 2: eq. (FALS),
 *            l_p = l_{p-1} + r^2 / ||r||^2 with r the full-data residual of lag p-1's estimate, eq. (FAR);
 *   sampling c rows with replacement from pi = l_p / p, eq. (FASD): draw k takes the first row whose running sum of
 *            l_p exceeds d_unif[(p-1) c + k] * sum(l_p) (the last row with a positive score if rounding leaves
 *            none), and scales it by 1 / sqrt(c pi_i);
 *   solve    phi_hat_p = the minimiser of the compressed problem, by Cholesky of the sampled X^T W X and one
 *            corrected semi-normal-equation step; tau[p-1] = phi_hat_p[p-1], the PACF estimate at lag p.
 * The order estimate is the largest p with |tau[p-1]| >= 1.96 / sqrt(c) (0 if none).
 * d_y: n doubles (device). d_unif: p_bar x c uniforms in [0, 1) (device, row p-1 for lag p): the random draws are
 * inputs. tau: p_bar doubles (host). order: host, nullable. phi: host, nullable, p_bar doubles: phi_hat at the
 * order estimate, zero-padded (all zero if the order is 0). d_rows: device, nullable, p_bar x c sampled rows
 * (int64, row p-1 for lag p). d_phi_all: device, nullable, p_bar x p_bar: row p-1 holds phi_hat_p, zero-padded.
 * Needs 1 <= p_bar <= 256, c >= p_bar, n > p_bar. Returns TOLS_NOT_CONVERGED if a sampled X^T W X is not positive
 * definite (tau is NaN from that lag on; the message names the lag). Runs on the context's stream and returns
 * after it finishes. */
int toeplitz_ols_lsar(tols_ctx* ctx, const double* d_y, long long n, int p_bar, int c, const double* d_unif,
                      double* tau, int* order, double* phi, long long* d_rows, double* d_phi_all);

/* The Repeated Halving variant of Algorithm "LSAR" (end of Section 3.2): Algorithm "Repeated Halving" (Section 3.2)
 * runs once on C = [X | b] of order p_bar (m = n - p_bar rows: C(i,:) holds y[i .. i + p_bar]); its top-level
 * scores then replace eq. (FALS) at every lag of LSAR (same lags, sampling, compressed fits and order estimate as
 * toeplitz_ols_lsar; the draws at each lag are weighted by 1 / sqrt(c pi_i), pi = scores / sum(scores)).
 *   halving  levels >= 1 halvings: h_sizes[0] = m, h_sizes[j+1] = h_sizes[j] / 2 (host, levels + 1 entries);
 *            h_keep (host) holds, level after level, the h_sizes[j+1] increasing positions within level j that
 *            level j+1 keeps (the uniform subsets are inputs). The deepest level is its own approximation.
 *   upward   for j = levels-1 .. 0: B = the approximation of level j+1 (the deepest level's rows, unscaled, or c
 *            rows drawn from level j+1, each scaled by 1 / sqrt(c p_r)); the scores of level j's rows are
 *            ||S_j B (B^T B)^-1 C(i,:)^T||^2, eq. (glev), with the sketch S_j (k x rows(B), row-major; d_sketch
 *            holds S_0, S_1, ... in turn, rows(B) = h_sizes[levels] for the deepest level's sketch, else c);
 *            for j >= 1, c rows of level j are drawn from its scores with d_rh_unif[j c .. j c + c) (inverse CDF
 *            as in toeplitz_ols_lsar) to form level j's approximation. Level 0's scores are the result.
 * d_y: n doubles (device). d_unif: p_bar x c uniforms for the lags (device). tau (host, p_bar), order (host,
 * nullable), phi (host, nullable, p_bar doubles) as in toeplitz_ols_lsar. d_scores: device, nullable, m doubles
 * (level 0's scores). d_rows: device, nullable, p_bar x c sampled rows of the lags (int64).
 * Needs 1 <= p_bar <= 256, 1 <= k <= 64, c >= p_bar + 1, p_bar + 1 <= h_sizes[levels] <= 2^30. Returns TOLS_ERR_ARG on
 * malformed sizes or keep lists (checked before any device work), TOLS_NOT_CONVERGED if a B^T B or a sampled
 * Gram matrix is not positive definite (the message names the level or lag). Runs on the context's stream
 * and returns after it finishes. */
int toeplitz_ols_rh_lsar(tols_ctx* ctx, const double* d_y, long long n, int p_bar, int c, int k, int levels,
                         const long long* h_sizes, const long long* h_keep, const double* d_sketch,
                         const double* d_rh_unif, const double* d_unif, double* tau, int* order, double* phi,
                         double* d_scores, long long* d_rows);

/* Algorithm "SRHT" (Section 2.1): phi minimising ||S H D (X phi - b)||, eq. (SRHT), for the order-p problem of
 * eq. (xphi). The m = n - p rows of [X | b] are zero-padded to m2 = 2^ceil(log2 m); D = diag(d_signs) (m2 doubles,
 * +-1, device); H is the normalised Hadamard transform of Def. "Hadamard Transform" (m2 x m2), applied to every
 * column by its recursion; S takes the c rows d_rows[0 .. c) (int64 in [0, m2), device; drawn uniformly with
 * replacement by the caller) scaled by sqrt(m2 / c). The compressed problem is solved through its normal
 * equations (Cholesky). d_phi: p doubles (device). Needs 1 <= p <= 256, c >= p, n > p; holds (p + 1) m2
 * doubles of device memory while it runs. Returns TOLS_ERR_ARG for a row index outside [0, m2) (found on the
 * device; phi is then not written), TOLS_NOT_CONVERGED if the normal matrix is not positive definite. Returns
 * after the context's stream finishes. */
int toeplitz_ols_srht(tols_ctx* ctx, const double* d_y, long long n, int p, int c, const double* d_signs,
                      const long long* d_rows, double* d_phi);

/* ---- instrumentation (no counterpart in the paper: measurement of this library's own kernels) ----------
 * toeplitz_ols_profile(ctx, 1) clears the counters and starts timing every kernel the context launches with
 * a pair of CUDA events on the context's stream; 0 stops timing (counters are kept).
 * toeplitz_ols_profile_read returns, for one kernel class, the number of launches that did work and their
 * summed device time in milliseconds. Classes:
 *   0..4  float32 pass kernel with tail STORE, LSQR, NECORR, CHECK, GRAM
 *   5..9  float64 pass kernel with tail STORE, LSQR, NECORR, CHECK, GRAM
 *   10    preconditioner (Cholesky + inverse), 11 float32 conversion, 12 other small kernels
 *   13..16 batched solves: float64 FFT pass, float64 direct pass, float32 direct pass, d spectra (every launch,
 *         whether or not it found work; while profiling, batches launch their passes one by one instead of
 *         replaying CUDA graphs)
 *   -1    every kernel launch the context made since profiling was enabled (launches only; ms = 0),
 *         counted whether or not timing is on, including launches that found no work. */
#define TOLS_PROFILE_CLASSES 17
int toeplitz_ols_profile(tols_ctx* ctx, int enable);
int toeplitz_ols_profile_read(tols_ctx* ctx, int kind, long long* launches, double* total_ms);

#ifdef __cplusplus
}
#endif

#endif /* TOEPLITZ_OLS_H */
