// C ABI of the Toeplitz-OLS solver: context, device arena, the solve drivers and the step entry points.
//
// A solve (eq. (xphi), Section 3; Thm. "Solution to OLS problem", Section 2) runs as a device-resident state
// machine. The host launches pass kernels; the last CTA of each pass performs the scalar step and writes
// the next phase into DevState, so the host only polls a status word every few launches:
//
//   FP64  : Gram pass (float64 products) -> preconditioner (Cholesky factor of the Gram matrix, or the R of sampled
//           rows when that factor is not trusted) -> trusted factor: semi-normal-equation start
//           phi0 = R^-1 R^-T X^T b; else LSQR passes from zero -> float64 check pass
//           [-> LSQR on the stored residual -> check ...] until the ratio meets tol or a check stops improving
//   MIXED : the same route; after a check that misses tol, while the factor is trusted and kappa(X) u32 <= 1e-2,
//           the correction sweep uses float products (Golub-Kahan Bidiag 2 on the normal-equation correction,
//           float64 scalars) -> float64 check pass -> ...; float64 LSQR sweeps otherwise, and a warm-started
//           float64 repeat when the float sweeps stop contracting.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <math.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tols_internal.cuh"

using namespace tols;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct StreamSeries {
  int p;
  double tol;
  std::vector<double> y;
  std::vector<double> phi;  // last solution (warm start)
};

}  // namespace

constexpr size_t kStateBytes = (sizeof(tols::DevState) + 255) / 256 * 256;   // pinned state, then phi

struct tols_ctx {
  tols_config cfg{};
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t used = 0;
  DevBuf y64, y32, u0, u1, part, vecs, mats, state, scratch, rbuf, tune, tune_y, spec32, spec64, sacc32, b_spec, lsar,
      pcl;
  // batched solves: pooled per-series buffers
  DevBuf b_y64, b_y32, b_u0, b_u1, b_part, b_cnt, b_vecs, b_phi, b_mats, b_state, b_series, b_tiles;
  double* h_stage = nullptr;    // pinned staging of host series for one H2D copy
  size_t h_stage_cap = 0;
  DevState* h_state = nullptr;  // pinned copy of the device state, followed by a pinned phi (TOLS_MAX_P doubles)
  double* h_phi = nullptr;
  PclInfo* h_pcl = nullptr;     // pinned copy of the multi-CTA preconditioner's report (after h_phi)
  std::string err;
  std::map<int, StreamSeries> streams;
  int next_handle = 1;
  int grid[6] = {};                   // pass grid (float, double; direct, FFT of the default N, FFT of N = 4,096)
  size_t grid_pad[6] = {};            // p_pad the grid was computed for
  void* tw32 = nullptr;               // FFT twiddle tables (float2[4096], double2[2048], double2[4096])
  void* tw64 = nullptr;
  void* tw64x = nullptr;
  std::map<int, int> fft_choice;      // autotuner: key (is_double, p_pad, gram) -> FFT length N, or 0 (direct)
  int last_fft = 0;                   // FFT length of the last solve's iteration passes (0: direct)
  // instrumentation (toeplitz_ols_profile)
  bool prof = false;
  long long launch_total = 0;
  long long prof_launches[TOLS_PROFILE_CLASSES] = {};
  double prof_ms[TOLS_PROFILE_CLASSES] = {};
  struct Pending { cudaEvent_t e0, e1; int slot, kind; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_free;
  int* d_worklog = nullptr;
  int* h_worklog = nullptr;
};

namespace {

int fail(tols_ctx* c, int code, const char* what, cudaError_t e = cudaSuccess) {
  if (c) {
    char buf[512];
    if (e != cudaSuccess)
      snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    else
      snprintf(buf, sizeof buf, "%s", what);
    c->err = buf;
  }
  return code;
}

#define CK(expr)                                                          \
  do {                                                                    \
    cudaError_t e_ = (expr);                                              \
    if (e_ != cudaSuccess) return fail(ctx, TOLS_ERR_CUDA, #expr, e_);    \
  } while (0)

// Grow a device buffer to at least bytes (contents are not preserved), honouring the memory cap.
int ensure(tols_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.cap >= bytes) return TOLS_OK;
  if (b.p) {
    cudaFree(b.p);
    ctx->used -= b.cap;
    b.p = nullptr;
    b.cap = 0;
  }
  bytes = (bytes + 255) & ~size_t(255);
  if (ctx->cfg.mem_cap_bytes && ctx->used + bytes > ctx->cfg.mem_cap_bytes)
    return fail(ctx, TOLS_ERR_OOM, "device arena would exceed mem_cap_bytes");
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, TOLS_ERR_OOM, "cudaMalloc", e);
  }
  b.cap = bytes;
  ctx->used += bytes;
  return TOLS_OK;
}

void release(tols_ctx* ctx, DevBuf& b) {
  if (b.p) cudaFree(b.p);
  ctx->used -= b.cap;
  b = DevBuf{};
}

constexpr int kMaxPending = 512;

// Accumulate the timed launches recorded since the last call (the stream is synchronised here).
int flush_profile(tols_ctx* ctx) {
  if (ctx->pending.empty()) return TOLS_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(ctx->h_worklog, ctx->d_worklog, sizeof(int) * kMaxPending, cudaMemcpyDeviceToHost));
  for (const auto& q : ctx->pending) {
    const int kind = q.kind >= 0 ? q.kind : ctx->h_worklog[q.slot] - 1;
    if (kind >= 0 && kind < TOLS_PROFILE_CLASSES) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, q.e0, q.e1));
      ctx->prof_launches[kind] += 1;
      ctx->prof_ms[kind] += ms;
    }
    ctx->ev_free.push_back(q.e0);
    ctx->ev_free.push_back(q.e1);
  }
  ctx->pending.clear();
  CK(cudaMemsetAsync(ctx->d_worklog, 0, sizeof(int) * kMaxPending, ctx->stream));
  return TOLS_OK;
}

int take_event(tols_ctx* ctx, cudaEvent_t* e) {
  if (!ctx->ev_free.empty()) {
    *e = ctx->ev_free.back();
    ctx->ev_free.pop_back();
    return TOLS_OK;
  }
  CK(cudaEventCreate(e));
  return TOLS_OK;
}

// Launch a pass kernel (timed when profiling).
template <typename T>
int run_pass(tols_ctx* ctx, PassArgs<T> a, int grid) {
  ctx->launch_total++;
  a.wait_polls = ctx->cfg.wait_polls;
  if (!ctx->prof) {
    CK(launch_pass<T>(a, grid, ctx->stream));
    return TOLS_OK;
  }
  int rc;
  if ((int)ctx->pending.size() >= kMaxPending && (rc = flush_profile(ctx))) return rc;
  tols_ctx::Pending q;
  if ((rc = take_event(ctx, &q.e0)) || (rc = take_event(ctx, &q.e1))) return rc;
  q.slot = (int)ctx->pending.size();
  q.kind = -1;
  a.worklog = ctx->d_worklog;
  a.work_slot = q.slot;
  CK(cudaEventRecord(q.e0, ctx->stream));
  CK(launch_pass<T>(a, grid, ctx->stream));
  CK(cudaEventRecord(q.e1, ctx->stream));
  ctx->pending.push_back(q);
  return TOLS_OK;
}

// Launch one of the small kernels of class kind (timed when profiling).
template <typename F>
int run_small(tols_ctx* ctx, int kind, F launch) {
  ctx->launch_total++;
  if (!ctx->prof) {
    CK(launch());
    return TOLS_OK;
  }
  int rc;
  if ((int)ctx->pending.size() >= kMaxPending && (rc = flush_profile(ctx))) return rc;
  tols_ctx::Pending q;
  if ((rc = take_event(ctx, &q.e0)) || (rc = take_event(ctx, &q.e1))) return rc;
  q.slot = -1;
  q.kind = kind;
  CK(cudaEventRecord(q.e0, ctx->stream));
  CK(launch());
  CK(cudaEventRecord(q.e1, ctx->stream));
  ctx->pending.push_back(q);
  return TOLS_OK;
}

#define RUN(expr)                       \
  do {                                  \
    int rc_ = (expr);                   \
    if (rc_) return rc_;                \
  } while (0)

// fft: 0 (direct products) or the FFT length N (1: the precision's default N).
int pass_grid_for(tols_ctx* ctx, int is_double, int p_pad, int fft = 0) {
  if (fft == 1) fft = fft_size(is_double);
  const int slot = is_double + 2 * (fft == 0 ? 0 : fft == fft_size(is_double) ? 1 : 2);
  if (ctx->grid[slot] == 0 || ctx->grid_pad[slot] != (size_t)p_pad) {
    int nb = 0;
    const void* fn = fft ? fft_kernel_ptr(is_double, fft) : pass_kernel_ptr(is_double);
    const size_t smem = pass_smem_bytes(is_double, p_pad, fft);
    smem_opt_in(fn, 200 * 1024);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, smem) != cudaSuccess || nb < 1) nb = 1;
    // A float64 FFT pass keeps the FP64 pipe busy with two CTAs per SM already; a third adds one more closing
    // inverse transform per SM without raising the pipe's throughput (4M rows, p = 100: 0.471 ms at 2 per SM,
    // 0.497 ms at 3).
    const int per_sm = (fft && is_double) ? 2 : 4;
    ctx->grid[slot] = std::min(kMaxGrid, ctx->sms * std::min(nb, per_sm));
    ctx->grid_pad[slot] = p_pad;
  }
  return ctx->grid[slot];
}

// Doubled window spectra of series y (tiles of N - p_pad rows) in the context's buffer for that precision, which
// every FFT pass reads. form: transform them here (spectrum_kernel); else only make room (a Gram pass fills it).
// nfft: the FFT length N (0 or 1: the precision's default).
int fft_spectra(tols_ctx* ctx, Work& w, int is_double, const void* y, long long n, long long m, int p_pad, bool form,
                int nfft = 0) {
  if (nfft <= 1) nfft = fft_size(is_double);
  DevBuf& b = is_double ? ctx->spec64 : ctx->spec32;
  RUN(ensure(ctx, b, fft_spectra_bytes(is_double, m, p_pad, nfft)));
  if (is_double) {
    w.wspec64 = b.p;
  } else {
    w.wspec32 = b.p;
    RUN(ensure(ctx, ctx->sacc32, fft32_sum_bytes()));
    w.sacc32 = ctx->sacc32.p;
  }
  if (!form) return TOLS_OK;
  return run_small(ctx, 12, [&] {
    return launch_spectra(is_double, y, n, m, p_pad, b.p, is_double ? (nfft == 4096 ? w.tw64x : w.tw64) : w.tw32,
                          pass_grid_for(ctx, is_double, p_pad, nfft), ctx->stream, nfft);
  });
}

// Product kernel for a pass over series y (T = float or double): the sliding-window direct products or the
// overlap-save FFT, and its length N. DIRECT / FFT / FFT4096 force one; AUTO times the direct and the FFT pass of
// the default N once per (precision, p_pad) on the series at hand when it is long enough for the choice to matter
// (cached in the context), else picks by p. Float64 transforms of N = 4,096 serve the orders the default N = 2,048
// cannot (p_pad >= 1,024) and TOLS_PRODUCT_FFT4096; below that they were not faster on GB300 (one CTA per SM
// instead of two: 7.73 against 7.72 ms at p = 500, n = 2^26, and slower at smaller p) and their rounding error
// is larger (u log2 N sqrt(N) per window), which shows at the float64 floor of ill-conditioned series. Returns 0
// (direct) or N.
template <typename T>
int choose_fft(tols_ctx* ctx, const Work& w, const T* y, long long n, int p, int p_pad, int nlag, int gram) {
  const int is_double = sizeof(T) == 8;
  const int n_def = fft_size(is_double);
  const bool def_ok = p_pad < n_def / 2;                   // enough rows per FFT tile
  const bool long_ok = is_double && p_pad < 4096 / 2;
  if (ctx->cfg.product == TOLS_PRODUCT_DIRECT) return 0;
  if (ctx->cfg.product == TOLS_PRODUCT_FFT4096 && long_ok) return 4096;
  if (ctx->cfg.product == TOLS_PRODUCT_FFT || ctx->cfg.product == TOLS_PRODUCT_FFT4096)
    return def_ok ? n_def : long_ok ? 4096 : 0;
  if (!def_ok) return long_ok ? 4096 : 0;                   // only the long transforms fit these orders
  const long long m = n - p;
  const int key = is_double * 100000 + p_pad * 2 + gram;
  auto it = ctx->fft_choice.find(key);
  if (it != ctx->fft_choice.end()) return it->second;
  const int guess = p_pad >= (is_double ? 32 : 64) ? n_def : 0;
  if (m < (1 << 20) || ensure(ctx, ctx->tune, sizeof(double) * (4 * (size_t)p_pad + 64)) != TOLS_OK) return guess;
  double* sc = (double*)ctx->tune.p;
  PassArgs<T> a;
  memset(&a, 0, sizeof a);
  a.y = y;
  a.n = n;
  a.m = m;
  a.p = p;
  a.p_pad = p_pad;
  a.nlag = nlag;
  a.gram = gram;
  a.d = sc + 2 * p_pad;           // contents do not matter for timing
  a.d_scale = 1.0;
  a.tail = TAIL_STORE;
  a.out_t = sc;
  a.out_n2 = sc + p_pad + 8;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int cand[2] = {0, n_def};
  float best_ms = 0.f;
  int choice = guess;
  for (int c = 0; c < 2; ++c) {
    if (cand[c] < 0) continue;
    Work wf = w;                  // an FFT pass reads (or, for the Gram, writes) the window spectra of its N
    if (cand[c] && fft_spectra(ctx, wf, is_double, y, n, m, p_pad, !gram, cand[c]) != TOLS_OK) continue;
    a.fft = cand[c];
    a.w = wf;
    const int grid = pass_grid_for(ctx, is_double, p_pad, cand[c]);
    launch_pass<T>(a, grid, ctx->stream);                 // warm-up
    cudaEventRecord(e0, ctx->stream);
    launch_pass<T>(a, grid, ctx->stream);
    launch_pass<T>(a, grid, ctx->stream);
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (cudaGetLastError() != cudaSuccess) continue;
    if (c == 0 || ms < best_ms) {
      best_ms = ms;
      choice = cand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->fft_choice[key] = choice;
  return choice;
}

// Lay out one solve's workspace in the context buffers. y64 is the caller's (or staged) device series.
int prepare_work(tols_ctx* ctx, const double* y64, long long n, int p, bool mixed, bool need_u, Work& w) {
  memset(&w, 0, sizeof w);
  w.n = n;
  w.m = n - p;
  w.p = p;
  w.p_pad = pad_p(p + 1);
  w.y64 = y64;
  const size_t m = (size_t)w.m;
  int rc;
  if (mixed) {
    if ((rc = ensure(ctx, ctx->y32, sizeof(float) * (size_t)n))) return rc;
    w.y32 = (float*)ctx->y32.p;   // filled when the first float pass is due
  }
  if (need_u) {
    // float64 even for a mixed solve: it runs float64 iterations when float products cannot refine it (the float
    // passes use the first half)
    const size_t es = sizeof(double);
    if ((rc = ensure(ctx, ctx->u0, es * m))) return rc;
    if ((rc = ensure(ctx, ctx->u1, es * m))) return rc;
    w.U[0] = ctx->u0.p;
    w.U[1] = ctx->u1.p;
  }
  const size_t pp = (size_t)w.p_pad;
  // The arrival counters sit at a fixed offset at the head of the buffer, whatever p is: every pass leaves
  // them at zero, and they are zeroed whenever the buffer is (re)allocated.
  const size_t cnt_bytes = 256 * ((sizeof(unsigned int) * (kMaxGroups + 1) + 255) / 256);
  const size_t part_bytes = cnt_bytes + sizeof(double) * (kMaxGrid * pp + kMaxGrid + kMaxGroups * pp + kMaxGroups);
  const bool fresh_part = ctx->part.cap < part_bytes;
  if ((rc = ensure(ctx, ctx->part, part_bytes))) return rc;
  w.counters = (unsigned int*)ctx->part.p;
  double* q = (double*)((char*)ctx->part.p + cnt_bytes);
  w.part_n2 = q; q += kMaxGrid;
  w.grp_n2 = q; q += kMaxGroups;
  w.part_t = q; q += kMaxGrid * pp;
  w.grp_t = q; q += kMaxGroups * pp;
  if (fresh_part) CK(cudaMemsetAsync(ctx->part.p, 0, cnt_bytes, ctx->stream));
  if ((rc = ensure(ctx, ctx->vecs, sizeof(double) * (10 * pp + 8)))) return rc;
  q = (double*)ctx->vecs.p;
  w.v = q; q += pp;
  w.w = q; q += pp;
  w.z = q; q += pp;
  w.d = q; q += pp;
  w.phi = q; q += pp;
  w.g = q; q += pp;
  w.h = q; q += pp;
  w.t = q; q += pp;
  w.best = q; q += pp;
  w.bnorm2 = q; q += pp;
  const size_t pq = (size_t)p * p;
  const size_t qrd = qr_scratch_doubles(p);
  if ((rc = ensure(ctx, ctx->mats, sizeof(double) * (3 * pq + qrd) + sizeof(float) * 2 * pq + 1024))) return rc;
  q = (double*)ctx->mats.p;
  w.G = q; q += pq;
  w.M = q; q += pq;
  w.Mt = q; q += pq;
  w.qr = qrd ? q : nullptr;
  q += qrd;
  float* f = (float*)q;
  w.M32 = f; f += pq;
  w.Mt32 = f;
  if ((rc = ensure(ctx, ctx->state, sizeof(DevState)))) return rc;
  w.st = (DevState*)ctx->state.p;
  w.tw32 = ctx->tw32;
  w.tw64 = ctx->tw64;
  w.tw64x = ctx->tw64x;
  return TOLS_OK;
}

template <typename T>
PassArgs<T> base_args(const Work& w, const T* y, long long n, int p, int p_pad) {
  PassArgs<T> a;
  memset(&a, 0, sizeof a);
  a.y = y;
  a.n = n;
  a.m = n - p;
  a.p = p;
  a.p_pad = p_pad;
  a.nlag = p;
  a.d_scale = 1.0;
  a.w = w;
  return a;
}

int validate(tols_ctx* ctx, long long n, int p) {
  if (!ctx) return TOLS_ERR_ARG;
  if (p < 1 || p > TOLS_MAX_P) return fail(ctx, TOLS_ERR_ARG, "p out of range [1, TOLS_MAX_P]");
  if (n <= p) return fail(ctx, TOLS_ERR_ARG, "need n > p");
  return TOLS_OK;
}

// ------------------------------------------------------------------------------------------------------
// Multi-CTA preconditioner of single-series solves (tols_precond.cu), for orders from kPclMinP up.
constexpr int kPclMinP = 64;

// Rows of X sampled for the QR preconditioner: c = r p with r = 8, 16 or 32. More rows lower kappa(X R^{-1})
// (about 2.1, 1.6, 1.4 on the AR(500) bench series), which saves LSQR iterations, each a pass over all m rows;
// the sample's QR costs O(c p^2). r grows with m / (8 p^2), the ratio of the two.
long long pcl_sample_rows(long long m, int p) {
  const long long q = m / (8LL * p * p);
  const long long r = q >= 32 ? 32 : q >= 16 ? 16 : 8;
  return r * p;
}

int pcl_sync(tols_ctx* ctx, const PclInfo* d_info) {
  CK(cudaMemcpyAsync(ctx->h_pcl, d_info, sizeof(PclInfo), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return TOLS_OK;
}

// Every tile step of the blocked Cholesky of Gp (P x P).
int pcl_factor(tols_ctx* ctx, double* Gp, int P, int p, double tiny_dmax, double tiny_shift, PclInfo* d_info) {
  const int nt = P / kPclTile;
  for (int k = 0; k < nt; ++k) {
    RUN(run_small(ctx, 10, [&] { return pcl_chol_panel(Gp, P, p, k, tiny_dmax, tiny_shift, d_info, ctx->stream); }));
    if (k + 1 < nt) RUN(run_small(ctx, 10, [&] { return pcl_chol_update(Gp, P, k, d_info, ctx->stream); }));
  }
  return TOLS_OK;
}

// The preconditioner of one solve, with the state precond_kernel leaves: norms of X from G (trace, power
// iteration), the Cholesky factor of G (refactored with the shift 10 p u max_j G_jj if a pivot falls to rounding
// level, which flags G as singular), M = R^{-1}, kappa(R) and the trust test kappa(R)^2 u <= 1/4 (u of float64: G
// is formed from float64 products). A solve whose factor is not trusted (or that asks for it) is preconditioned
// instead by the R of c sampled rows of X from shifted Cholesky QR (two shifted stages, shift
// 11 (c p + p (p + 1)) u lambda_max, then one plain stage; R = R3 R2 R1). The host reads a small report after
// each factorisation.
int precond_large(tols_ctx* ctx, Work& w, int want, bool mixed) {
  const int p = w.p, P = pcl_pad_p(p), nt = P / kPclTile;
  const size_t PP = (size_t)P * P;
  const double ueps = 1.11e-16;                              // G comes from float64 products in every precision
  const bool qr_ok = want != 0 && w.m >= 8LL * p;
  const long long c = qr_ok ? pcl_sample_rows(w.m, p) : 0;
  const int slices = c ? pcl_gram_slices(c, P) : 0;
  const size_t ntiles = (size_t)nt * (nt + 1) / 2;
  const size_t head = 256;                                   // PclInfo
  const size_t fb_bytes = (sizeof(float) * (size_t)p * p + 255) / 256 * 256;
  size_t bytes = head + fb_bytes + sizeof(double) * PP;      // report, float copy, Gp
  if (c) bytes += sizeof(double) * (4 * PP + (size_t)c * p + (size_t)slices * ntiles * 1024);
  RUN(ensure(ctx, ctx->pcl, bytes));
  char* base = (char*)ctx->pcl.p;
  PclInfo* d_info = (PclInfo*)base;
  float* fb = (float*)(base + head);
  double* Gp = (double*)(base + head + fb_bytes);
  double* Rq[4] = {Gp + PP, Gp + 2 * PP, Gp + 3 * PP, Gp + 4 * PP};
  double* A = Gp + 5 * PP;
  double* part = A + (size_t)c * p;
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(d_info, 0, sizeof(PclInfo), st));
  RUN(run_small(ctx, 10, [&] { return pcl_lambda(w.G, p, p, 0.0, 0, fb, d_info, st); }));
  bool ok = false, shifted = false, singular = false;
  double cond = 0.0, g_shift = 0.0, g_tiny = (double)p * ueps;
  if (want) {
    RUN(run_small(ctx, 10, [&] { return pcl_pad(w.G, p, Gp, P, 0.0, nullptr, st); }));
    RUN(pcl_factor(ctx, Gp, P, p, (double)p * ueps, 0.0, d_info));
    RUN(pcl_sync(ctx, d_info));
    if (!ctx->h_pcl->nonfinite) {
      if (ctx->h_pcl->fail) {
        singular = true;
        g_shift = 10.0 * (double)p * ueps * ctx->h_pcl->dmax;
        g_tiny = 1e-3 * 10.0 * (double)p * ueps;
        CK(cudaMemsetAsync(&d_info->fail, 0, sizeof(int), st));
        RUN(run_small(ctx, 10, [&] { return pcl_pad(w.G, p, Gp, P, g_shift, nullptr, st); }));
        RUN(pcl_factor(ctx, Gp, P, p, g_tiny, 0.0, d_info));
        RUN(pcl_sync(ctx, d_info));
        shifted = !ctx->h_pcl->fail;
      }
      if (!ctx->h_pcl->fail) {
        RUN(run_small(ctx, 10, [&] { return pcl_inverse(Gp, P, p, w.M, d_info, st); }));
        RUN(run_small(ctx, 10, [&] { return pcl_estimate(w.M, p, 0, fb, d_info, st); }));
        RUN(pcl_sync(ctx, d_info));
        cond = ctx->h_pcl->cond;
        ok = true;
      }
    }
  }
  const bool nonfinite = ctx->h_pcl->nonfinite != 0 && want;
  bool trusted = ok && !shifted && cond * cond * ueps <= 0.25;
  int precond = ok ? 1 : 0;
  double kappa_est = cond;
  if (qr_ok && !nonfinite && (want == 2 || !trusted)) {
    const double shift_rel = 11.0 * ((double)c * p + (double)p * (p + 1)) * 1.11e-16;
    CK(cudaMemsetAsync(&d_info->fail, 0, sizeof(int), st));
    RUN(run_small(ctx, 10, [&] { return pcl_gather(w.y64, w.m, p, c, A, st); }));
    // stage s: Gram matrix of the current A (the sample, then Q1, Q2), its factor; A <- A R^{-1} after stages 0, 1
    auto stage = [&](int s, bool shift) -> int {
      RUN(run_small(ctx, 10, [&] { return pcl_tall_gram(A, c, p, P, slices, part, st); }));
      RUN(run_small(ctx, 10, [&] { return pcl_gram_reduce(part, P, slices, p, Gp, st); }));
      RUN(run_small(ctx, 10, [&] {
        return pcl_lambda(Gp, P, p, shift ? shift_rel : 0.0, s == 0 ? 1 : -1, fb, d_info, st);
      }));
      RUN(pcl_factor(ctx, Gp, P, p, shift ? 0.0 : (double)p * 1.11e-16, shift ? 1e-3 : 0.0, d_info));
      if (s < 2) {
        CK(cudaMemcpyAsync(Rq[s], Gp, sizeof(double) * PP, cudaMemcpyDeviceToDevice, st));
        RUN(run_small(ctx, 10, [&] { return pcl_trsm(A, c, p, Gp, P, st); }));
      }
      return TOLS_OK;
    };
    // R = R3 R2 R1, M = R^{-1} and its kappa estimate
    auto finish = [&]() -> int {
      RUN(run_small(ctx, 10, [&] { return pcl_trmm(Rq[1], Rq[0], Rq[2], P, st); }));   // R2 R1
      RUN(run_small(ctx, 10, [&] { return pcl_trmm(Gp, Rq[2], Rq[3], P, st); }));      // R3 R2 R1
      RUN(run_small(ctx, 10, [&] { return pcl_inverse(Rq[3], P, p, w.M, d_info, st); }));
      RUN(run_small(ctx, 10, [&] { return pcl_estimate(w.M, p, 1, fb, d_info, st); }));
      return pcl_sync(ctx, d_info);
    };
    RUN(stage(0, true));
    RUN(stage(1, true));
    RUN(stage(2, false));
    RUN(pcl_sync(ctx, d_info));
    bool qr_done = false, m_replaced = false;
    if (!ctx->h_pcl->fail && !ctx->h_pcl->nonfinite) {
      RUN(finish());
      qr_done = m_replaced = true;
    }
    // kappa(sample) beyond about 1e14: the plain last stage gives an R whose inverse float64 cannot apply (errors
    // of order kappa u). Shift the last stage too: R is then regularised at about 1e-13 sigma_max, LSQR resolves
    // the well-determined part fast and the near-null directions (no better determined in float64) slowly.
    if (!ctx->h_pcl->nonfinite && (!qr_done || ctx->h_pcl->cond * 1.11e-16 > 1e-2)) {
      CK(cudaMemsetAsync(&d_info->fail, 0, sizeof(int), st));
      RUN(stage(2, true));
      RUN(pcl_sync(ctx, d_info));
      qr_done = !ctx->h_pcl->fail && !ctx->h_pcl->nonfinite;
      if (qr_done) RUN(finish());
    }
    if (qr_done) {
      cond = ctx->h_pcl->cond;
      // ||A||_2 ||R^{-1}||_2 estimates kappa of the sample, which tracks kappa(X)
      kappa_est = cond;
      precond = 2;
      trusted = false;
      shifted = false;
    } else if (ok && m_replaced) {
      // the QR did not complete: the Gram factor stays; its inverse is formed again (the QR's overwrote it)
      CK(cudaMemsetAsync(&d_info->fail, 0, sizeof(int), st));
      RUN(run_small(ctx, 10, [&] { return pcl_pad(w.G, p, Gp, P, g_shift, nullptr, st); }));
      RUN(pcl_factor(ctx, Gp, P, p, g_tiny, 0.0, d_info));
      RUN(run_small(ctx, 10, [&] { return pcl_inverse(Gp, P, p, w.M, d_info, st); }));
    }
    CK(cudaMemsetAsync(&d_info->fail, 0, sizeof(int), st));
  }
  if (precond) RUN(run_small(ctx, 10, [&] { return pcl_store(w, mixed ? 1 : 0, d_info, st); }));
  RUN(run_small(ctx, 10, [&] {
    return pcl_state(w, d_info, precond, shifted ? 1 : 0, trusted ? 1 : 0, singular ? 1 : 0, cond, kappa_est, st);
  }));
  return TOLS_OK;
}

// Gram pass (float64 products, in every precision) + preconditioner for series w.y64. fft: the Gram pass uses the
// FFT kernel and writes the float64 window spectra (room made by fft_spectra). The float copy y32 of a mixed solve
// is made when its first float pass is due.
int run_setup(tols_ctx* ctx, Work& w, bool mixed, bool no_precond, int fft = 0, int want_override = -1) {
  const int pg = pad_p(w.p + 1);
  PassArgs<double> a = base_args<double>(w, w.y64, w.n, w.p, pg);
  a.gram = 1;
  a.nlag = w.p + 1;
  a.tail = TAIL_GRAM;
  a.out_n2 = w.bnorm2;
  a.fft = fft;
  RUN(run_pass<double>(ctx, a, pass_grid_for(ctx, 1, pg, a.fft)));
  const int want = no_precond ? 0 : want_override >= 0 ? want_override : ctx->cfg.precond;
  if (w.p >= kPclMinP) {
    // Orders whose Gram factor fits the one-CTA kernel's shared memory try that kernel first: one launch serves
    // the common case of a trusted factor, where the tiled multi-CTA steps spend their time in launches and in
    // host reads of the factorisation's report (AR(100), n = 2^22: 1.34 ms per solve with the tiled steps).
    // An untrusted factor goes on to the multi-CTA path: more sampled rows, and a regularised QR.
    if (want == TOLS_PRECOND_GRAM_CHOL && w.p <= kPrecondSmemP) {
      RUN(run_small(ctx, 10, [&] { return launch_precond(w, 3, ctx->stream); }));
      int trusted = 0;
      CK(cudaMemcpyAsync(&trusted, &w.st->trusted, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      if (trusted) return TOLS_OK;
    }
    return precond_large(ctx, w, want, mixed);
  }
  RUN(run_small(ctx, 10, [&] { return launch_precond(w, want, ctx->stream); }));
  return TOLS_OK;
}

void fill_info(tols_info* info, const DevState& s, int prec) {
  if (!info) return;
  info->status = s.status;
  info->iters = s.total_iter;
  info->sweeps = s.sweeps;
  info->precision_used = prec;
  info->precond_used = s.precond;
  info->product_used = s.fft ? TOLS_PRODUCT_FFT : TOLS_PRODUCT_DIRECT;  // single series: set after the call
  info->nfft = s.fft ? kBatchFftN : 0;
  info->ne_ratio = s.ne_ratio;
  info->rnorm = s.rnorm;
  info->bnorm = s.bnorm;
  info->anorm_2 = s.anorm_2;
  info->anorm_f = s.anorm_f;
  info->cond_est = s.cond_est;
}

// One complete solve of the series at d_y (device). phi0 (device, nullable) warm-starts. Leaves phi in w.phi
// and the final state in *ctx->h_state.
int solve_core(tols_ctx* ctx, const double* d_y, long long n, int p, double tol, bool mixed, const double* phi0,
               Work& w, bool no_precond = false, double* d_phi_out = nullptr, bool* phi_out_done = nullptr,
               double* h_phi_out = nullptr) {
  if (phi_out_done) *phi_out_done = false;
  int rc = prepare_work(ctx, d_y, n, p, mixed, true, w);
  if (rc) return rc;
  const int max_iter = ctx->cfg.max_iter > 0 ? ctx->cfg.max_iter : 4 * p + 200;
  const int max_sweeps = ctx->cfg.max_sweeps > 0 ? ctx->cfg.max_sweeps : 6;
  DevState hs;
  memset(&hs, 0, sizeof hs);
  hs.tol = tol;
  hs.tol_inner = 1e-5;
  hs.est_ratio = tol;
  hs.max_iter = max_iter;
  // float correction solves that need more than ~100 preconditioned iterations mean kappa(X) is too large for
  // float products; they stop early and the stall test hands the problem to the float64 path
  hs.iter_cap = mixed ? std::min(max_iter, 100) : max_iter;
  hs.max_sweeps = max_sweeps;
  hs.mixed = mixed ? 1 : 0;
  hs.mixed_ok = 1;
  hs.ne_ratio = 1e300;
  hs.ne_best = 1e300;
  hs.rnorm_best = 0.0;
  hs.status = TOLS_NOT_CONVERGED;
  hs.phase = PH_LSQR;
  *ctx->h_state = hs;
  CK(cudaMemcpyAsync(w.st, ctx->h_state, sizeof(DevState), cudaMemcpyHostToDevice, ctx->stream));
  // products: the direct or FFT kernel per precision. FFT passes use tiles of N - pad_p(p + 1) rows and read
  // the tile window spectra: the float64 Gram pass forms the float64 ones; the float ones (mixed solves that run
  // float correction sweeps) come from spectrum_kernel when first needed.
  const int pp = pad_p(p);
  const int pg = pad_p(p + 1);
  const int fft64 = choose_fft<double>(ctx, w, w.y64, n, p, pp, p, 0);
  if (fft64) RUN(fft_spectra(ctx, w, 1, w.y64, n, n - p, pg, false, fft64));
  if ((rc = run_setup(ctx, w, mixed, no_precond, fft64))) return rc;
  if (phi0) {
    CK(cudaMemcpyAsync(w.phi, phi0, sizeof(double) * p, cudaMemcpyDeviceToDevice, ctx->stream));
    RUN(run_small(ctx, 12, [&] { return launch_init_lsqr(w, 1, ctx->stream); }));
  } else {
    RUN(run_small(ctx, 12, [&] { return launch_init_lsqr(w, 0, ctx->stream); }));
  }
  PassArgs<double> ad = base_args<double>(w, w.y64, n, p, fft64 ? pg : pp);
  ad.check_done = 1;
  ad.d = w.d;
  ad.fft = fft64;
  PassArgs<float> af = base_args<float>(w, w.y32, n, p, pp);
  af.check_done = 1;
  af.d = w.d;
  ctx->last_fft = ad.fft;
  const int gd = pass_grid_for(ctx, 1, ad.p_pad, ad.fft);
  int gf = 0;
  bool f32_ready = false, f32_mode = false;
  const long long max_launch = (long long)(max_iter + 4) * (max_sweeps + 2) * 2 + 16;
  long long launched = 0;
  // a solve from a trusted factor usually ends with its first (check) pass: start with a burst of one
  int burst = 1;
  while (true) {
    if (f32_mode) {
      for (int k = 0; k < burst; ++k) RUN(run_pass<float>(ctx, af, gf));
      RUN(run_pass<double>(ctx, ad, gd));
      launched += burst + 1;
    } else {
      for (int k = 0; k < burst; ++k) RUN(run_pass<double>(ctx, ad, gd));
      launched += burst;
    }
    // phi goes out with every state read, so a converged solve needs no further round trip
    if (d_phi_out) CK(cudaMemcpyAsync(d_phi_out, w.phi, sizeof(double) * p, cudaMemcpyDeviceToDevice, ctx->stream));
    if (h_phi_out) CK(cudaMemcpyAsync(h_phi_out, w.phi, sizeof(double) * p, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    RUN(flush_profile(ctx));
    const DevState& cur = *ctx->h_state;
    if (cur.dev_error) return fail(ctx, TOLS_ERR_DEVICE_TIMEOUT, "a kernel's wait on its bulk copies gave up");
    if (cur.done || cur.phase == PH_DONE) break;
    if (launched > max_launch) return fail(ctx, TOLS_ERR_DEVICE_TIMEOUT, "solver did not reach a final state");
    // float passes are due while a mixed solve runs a correction sweep
    const bool want32 = mixed && cur.mixed && (cur.phase == PH_NECORR || cur.phase == PH_LSQR);
    if (want32 && !f32_ready) {
      RUN(run_small(ctx, 11, [&] { return launch_convert_f32(w.y64, w.y32, n, ctx->stream); }));
      const int fft32 = choose_fft<float>(ctx, w, w.y32, n, p, pp, p, 0);
      if (fft32) RUN(fft_spectra(ctx, w, 0, w.y32, n, n - p, pg, true));
      af.fft = fft32;
      af.p_pad = fft32 ? pg : pp;
      af.w = w;
      gf = pass_grid_for(ctx, 0, af.p_pad, af.fft);
      f32_ready = true;
    }
    if (want32 != f32_mode) {
      f32_mode = want32;
      burst = 4;
    } else {
      burst = burst == 1 ? 4 : std::min(burst * 2, 16);
    }
  }
  if (ctx->h_state->status == TOLS_OK) {
    if (phi_out_done) *phi_out_done = d_phi_out != nullptr;
    return TOLS_OK;                              // nothing for the finishing kernel to do
  }
  RUN(run_small(ctx, 12, [&] { return launch_finish(w, ctx->stream); }));
  CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  RUN(flush_profile(ctx));
  return TOLS_OK;
}

// Solve with precision fallback; phi (device) receives the result.
int solve_device_impl(tols_ctx* ctx, const double* d_y, long long n, int p, double tol, double* d_phi,
                      double* rnorm, tols_info* info, const double* phi0, int force_prec = -1,
                      double* h_phi = nullptr, bool* h_phi_done = nullptr) {
  if (tol <= 0) tol = 1e-12;
  bool mixed = force_prec >= 0 ? force_prec == TOLS_MIXED : ctx->cfg.precision == TOLS_MIXED;
  Work w;
  bool phi_done = false;
  if (h_phi_done) *h_phi_done = false;
  int rc = solve_core(ctx, d_y, n, p, tol, mixed, phi0, w, false, d_phi, &phi_done, h_phi);
  if (rc) return rc;
  if (mixed && ctx->h_state->mixed_ok == 0 && ctx->h_state->status != TOLS_ERR_NONFINITE &&
      ctx->h_state->status != TOLS_OK) {
    // the float correction sweeps stopped contracting: redo it in float64, warm-started from the best iterate
    // when that one is usable, else from zero
    const bool warm = ctx->h_state->ne_best < 1e-3;
    phi_done = false;
    if (warm) CK(cudaMemcpyAsync(d_phi, w.best, sizeof(double) * p, cudaMemcpyDeviceToDevice, ctx->stream));
    mixed = false;
    const int saved_iter = ctx->h_state->total_iter;
    rc = solve_core(ctx, d_y, n, p, tol, false, warm ? d_phi : nullptr, w);
    if (rc) return rc;
    ctx->h_state->total_iter += saved_iter;
  }
  if (ctx->h_state->singular && ctx->h_state->compatible && ctx->h_state->status >= 0) {
    // X is exactly rank deficient (singular Gram matrix, zero residual): the shifted preconditioner does not
    // give the minimum-norm solution, plain LSQR from zero does. Keep the first result if the repeat fails.
    phi_done = false;
    CK(cudaMemcpyAsync(d_phi, w.phi, sizeof(double) * p, cudaMemcpyDeviceToDevice, ctx->stream));
    const DevState first = *ctx->h_state;
    rc = solve_core(ctx, d_y, n, p, tol, false, nullptr, w, true);
    if (rc) return rc;
    if (!(ctx->h_state->status == TOLS_OK && ctx->h_state->compatible)) {
      *ctx->h_state = first;
      CK(cudaMemcpyAsync(w.phi, d_phi, sizeof(double) * p, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
      ctx->h_state->total_iter += first.total_iter;
      ctx->h_state->sweeps += first.sweeps;
      mixed = false;
    }
  }
  const DevState& s = *ctx->h_state;
  if (s.status == TOLS_ERR_NONFINITE) return fail(ctx, TOLS_ERR_NONFINITE, "y holds NaN or Inf");
  if (!phi_done) {   // (a converged first solve already delivered phi with its last state read)
    CK(cudaMemcpyAsync(d_phi, w.phi, sizeof(double) * p, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else if (h_phi_done) {
    *h_phi_done = h_phi != nullptr;
  }
  if (rnorm) *rnorm = s.rnorm;
  // a mixed request is reported as mixed only when float products did part of the work
  fill_info(info, s, mixed && s.f32_iter > 0 ? TOLS_MIXED : TOLS_FP64);
  if (info) {
    info->nfft = ctx->last_fft;
    if (ctx->last_fft) info->product_used = ctx->last_fft == 4096 ? TOLS_PRODUCT_FFT4096 : TOLS_PRODUCT_FFT;
  }
  return s.status;
}

int stage_y(tols_ctx* ctx, const double* y, long long n) {
  int rc = ensure(ctx, ctx->y64, sizeof(double) * (size_t)n);
  if (rc) return rc;
  CK(cudaMemcpyAsync(ctx->y64.p, y, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
  return TOLS_OK;
}

int host_solve(tols_ctx* ctx, const double* y, long long n, int p, double tol, double* phi, double* rnorm,
               tols_info* info, const double* phi0_host) {
  int rc = stage_y(ctx, y, n);
  if (rc) return rc;
  if ((rc = ensure(ctx, ctx->scratch, sizeof(double) * (2 * (size_t)p + 64)))) return rc;
  double* d_phi = (double*)ctx->scratch.p;
  double* d_phi0 = nullptr;
  if (phi0_host) {
    d_phi0 = d_phi + p;
    CK(cudaMemcpyAsync(d_phi0, phi0_host, sizeof(double) * p, cudaMemcpyHostToDevice, ctx->stream));
  }
  bool h_done = false;
  rc = solve_device_impl(ctx, (const double*)ctx->y64.p, n, p, tol, d_phi, rnorm, info, d_phi0, -1, ctx->h_phi,
                         &h_done);
  if (rc < 0) return rc;
  if (h_done) {      // phi came back with the last state read
    memcpy(phi, ctx->h_phi, sizeof(double) * p);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(phi, d_phi, sizeof(double) * p, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(ctx, TOLS_ERR_CUDA, "copy phi to host", e);
  return rc;
}


// ------------------------------------------------------------------------------------------------------
// Batched solves: every series gets its own slices of pooled buffers; one tile list per precision covers all
// series; burst launches of the batched pass kernel (captured once into a CUDA graph) run until every series has
// reached its final state.
constexpr int kTileF = 4096, kTileD = 2048;   // rows per tile of the float / double pass kernels

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct BatchPlan {
  std::vector<int> idx;                      // caller index of every valid series
  std::vector<const double*> y_dev;          // device series given by the caller (else packed in b_y64)
  std::vector<long long> n, m, off_y, off_u, off_part, off_cnt, ntd, ntf, ntx;
  std::vector<int> p;
  std::vector<char> fft;                     // float64 FFT products (batch_fft_series)
  std::vector<size_t> off_vec, off_phi, off_mat, off_spec;
  size_t y_elems = 0, u_elems = 0, part_doubles = 0, cnt_uints = 0, vec_doubles = 0, phi_doubles = 0,
         mat_bytes = 0, spec_doubles = 0;
  long long tiles_f = 0, tiles_d = 0, tiles_x = 0;
  int p_pad_max = 16, p_pad_max_x = 16;
};

// Partial-sum slots (and arrival units) of a batched series, enough for every kernel that may run a pass over it:
// one per tile of the direct float64 kernel, or one per unit of kBatchFftUnit tiles of the FFT kernel, and one per
// tile of the direct float kernel (the correction sweeps of a mixed series; its tiles can outnumber the FFT units).
long long batch_units(long long m, int p, bool fx) {
  const long long d = fx ? batch_fft_units(m, p) : (m + kTileD - 1) / kTileD;
  return std::max(d, (m + kTileF - 1) / kTileF);
}

// Batched products (a9): whether a series of order p runs its batched float64 passes on the overlap-save FFT
// products (N = 2,048, tiles of N - pad_p(p + 1) rows) or on the direct ones. DIRECT forces the direct products;
// FFT / FFT4096 take the FFT from pad_p(p + 1) = 32 up. AUTO measures, once per process, device and class
// pad_p(p + 1): one direct and one FFT pass (best of three launches each) over a synthetic series of
// kBatchTuneRows rows of that order (enough tiles for several waves of CTAs, so that the passes run at their
// steady rate), and takes the FFT only where it is at least 5 % faster. The choice is kept
// for every context of the process, so a series' products, and so its result, do not depend on the context (or
// server) that solved it. The float correction sweeps of mixed series use the direct float products.
constexpr long long kBatchTuneRows = 1 << 21;
std::mutex g_batch_tune_mu;
std::map<long long, int> g_batch_tune;   // key device * 4096 + pad_p(p + 1) -> 1 FFT, 0 direct

int batch_fft_choice(tols_ctx* ctx, int p) {
  const int pp = pad_p(p + 1);
  if (ctx->cfg.product == TOLS_PRODUCT_DIRECT || pp >= kBatchFftN / 2) return 0;
  if (ctx->cfg.product != TOLS_PRODUCT_AUTO) return batch_fft_series(p) ? 1 : 0;
  std::lock_guard<std::mutex> lock(g_batch_tune_mu);
  const long long key = (long long)ctx->device * 4096 + pp;
  auto it = g_batch_tune.find(key);
  if (it != g_batch_tune.end()) return it->second;
  const int guess = batch_fft_series(p) ? 1 : 0;
  // synthetic series of order pt = pp - 1 (a fixed pseudo-random sequence: timing does not depend on values)
  const int pt = pp - 1;
  const long long n = kBatchTuneRows + pt;
  // its own buffer for the series: a caller may hold a staged series in ctx->y64 (the PACF batch)
  if (ensure(ctx, ctx->tune_y, sizeof(double) * (size_t)n) != TOLS_OK ||
      ensure(ctx, ctx->tune, sizeof(double) * (4 * (size_t)pp + 64)) != TOLS_OK)
    return guess;
  std::vector<double> hy((size_t)n);
  unsigned long long x = 0x9e3779b97f4a7c15ull;
  for (auto& v : hy) {
    x = x * 6364136223846793005ull + 1442695040888963407ull;
    v = (double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
  const double* d_y = (const double*)ctx->tune_y.p;
  if (cudaMemcpyAsync((void*)d_y, hy.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, ctx->stream) !=
      cudaSuccess)
    return guess;
  Work w;
  if (prepare_work(ctx, d_y, n, pt, false, true, w) != TOLS_OK) return guess;
  double* sc = (double*)ctx->tune.p;
  PassArgs<double> a = base_args<double>(w, d_y, n, pt, pp);
  a.d = sc + 2 * pp;
  a.u_old = (const double*)w.U[0];
  a.u_new = (double*)w.U[1];
  a.coef_host = 0.5;
  a.tail = TAIL_STORE;
  a.out_t = sc;
  a.out_n2 = sc + pp + 8;
  cudaMemsetAsync(w.U[0], 0, sizeof(double) * (size_t)kBatchTuneRows, ctx->stream);
  cudaMemsetAsync(sc, 0, sizeof(double) * (4 * (size_t)pp + 64), ctx->stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best[2] = {0.f, 0.f};
  bool ok = true;
  for (int f = 0; f < 2 && ok; ++f) {
    Work wf = w;
    if (f && fft_spectra(ctx, wf, 1, d_y, n, kBatchTuneRows, pp, true, kBatchFftN) != TOLS_OK) {
      ok = false;
      break;
    }
    a.fft = f ? kBatchFftN : 0;
    a.w = wf;
    const int grid = pass_grid_for(ctx, 1, pp, a.fft);
    launch_pass<double>(a, grid, ctx->stream);           // warm-up
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(e0, ctx->stream);
      launch_pass<double>(a, grid, ctx->stream);
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r == 0 || ms < best[f]) best[f] = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok || cudaGetLastError() != cudaSuccess) return guess;
  const int choice = best[1] < 0.95f * best[0] ? 1 : 0;
  g_batch_tune[key] = choice;
  return choice;
}

void plan_batch(tols_ctx* ctx, BatchPlan& B, int count, const long long* n, const int* p, std::vector<int>& status,
                bool mixed) {
  for (int k = 0; k < count; ++k) {
    if (p[k] < 1 || p[k] > TOLS_MAX_P || n[k] <= p[k]) { status[k] = TOLS_ERR_ARG; continue; }
    const long long nn = n[k], mm = nn - p[k];
    const int pp1 = pad_p(p[k] + 1);
    B.idx.push_back(k);
    B.n.push_back(nn);
    B.m.push_back(mm);
    B.p.push_back(p[k]);
    B.off_y.push_back((long long)B.y_elems);
    B.y_elems += align_up((size_t)nn, 64);
    B.off_u.push_back((long long)B.u_elems);
    B.u_elems += align_up((size_t)mm, 64);
    const bool fx = batch_fft_choice(ctx, p[k]) != 0;
    const long long ntd = fx ? 0 : (mm + kTileD - 1) / kTileD, ntf = (mm + kTileF - 1) / kTileF;
    const long long ntx = fx ? batch_fft_units(mm, p[k]) : 0;
    const long long nun = batch_units(mm, p[k], fx);
    const long long ngr = (nun + kGroup - 1) / kGroup;
    B.fft.push_back(fx ? 1 : 0);
    B.ntd.push_back(ntd);
    B.ntf.push_back(ntf);
    B.ntx.push_back(ntx);
    B.off_spec.push_back(B.spec_doubles);
    if (fx) B.spec_doubles += batch_fft_spectra_doubles(mm, p[k]) + 2 * (kBatchFftN / 2 + 1);
    B.off_part.push_back((long long)B.part_doubles);
    B.part_doubles += (size_t)(nun * pp1 + nun + ngr * pp1 + ngr);
    B.off_cnt.push_back((long long)B.cnt_uints);
    B.cnt_uints += (size_t)align_up((size_t)ngr + 1, 4);
    B.off_vec.push_back(B.vec_doubles);
    B.vec_doubles += 10 * (size_t)pp1;
    B.off_phi.push_back(B.phi_doubles);
    B.phi_doubles += (size_t)p[k];
    B.off_mat.push_back(B.mat_bytes);
    B.mat_bytes += align_up(sizeof(double) * (3 * (size_t)p[k] * p[k] + qr_scratch_doubles(p[k])) +
                            sizeof(float) * 2 * (size_t)p[k] * p[k], 256);
    B.tiles_f += ntf;
    B.tiles_d += ntd;
    B.tiles_x += ntx;
    B.p_pad_max = std::max(B.p_pad_max, pp1);
    if (fx) B.p_pad_max_x = std::max(B.p_pad_max_x, pp1);
  }
}

int batch_grid(tols_ctx* ctx, int is_double, int p_pad) {
  int nb = 0;
  smem_opt_in(batch_kernel_ptr(is_double), 200 * 1024);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel_ptr(is_double), kThreads,
                                                    pass_smem_bytes(is_double, p_pad)) != cudaSuccess || nb < 1)
    nb = 1;
  return ctx->sms * std::min(nb, 4);
}

int batch_fft_grid(tols_ctx* ctx, int p_pad) {
  int nb = 0;
  smem_opt_in(batch_fft_kernel_ptr(), 200 * 1024);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_fft_kernel_ptr(), kThreads, batch_fft_smem(p_pad)) !=
          cudaSuccess || nb < 1)
    nb = 1;
  return ctx->sms * std::min(nb, 4);
}

// d_y_packed: device series packed at B.off_y. Results: phi (device, packed at B.off_phi), states (host).
int batch_core(tols_ctx* ctx, BatchPlan& B, double tol, bool mixed, std::vector<DevState>& states,
               bool no_precond = false) {
  const int cnt = (int)B.idx.size();
  if (cnt == 0) return TOLS_OK;
  int rc;
  if (mixed && (rc = ensure(ctx, ctx->b_y32, sizeof(float) * B.y_elems))) return rc;
  // float64 for mixed series too: they run float64 iterations when float products cannot refine them
  const size_t ues = sizeof(double);
  if ((rc = ensure(ctx, ctx->b_u0, ues * B.u_elems)) || (rc = ensure(ctx, ctx->b_u1, ues * B.u_elems))) return rc;
  if ((rc = ensure(ctx, ctx->b_part, sizeof(double) * B.part_doubles))) return rc;
  const bool fresh_cnt = ctx->b_cnt.cap < sizeof(unsigned) * (B.cnt_uints + 4);
  if ((rc = ensure(ctx, ctx->b_cnt, sizeof(unsigned) * (B.cnt_uints + 4)))) return rc;
  if ((rc = ensure(ctx, ctx->b_vecs, sizeof(double) * B.vec_doubles))) return rc;
  if ((rc = ensure(ctx, ctx->b_phi, sizeof(double) * B.phi_doubles))) return rc;
  if ((rc = ensure(ctx, ctx->b_mats, B.mat_bytes))) return rc;
  if ((rc = ensure(ctx, ctx->b_state, sizeof(DevState) * cnt))) return rc;
  if ((rc = ensure(ctx, ctx->b_series, sizeof(BatchSeries) * cnt))) return rc;
  const size_t tiles_bytes = align_up(sizeof(int) * (size_t)(B.tiles_f + B.tiles_d + B.tiles_x), 16);
  if ((rc = ensure(ctx, ctx->b_tiles, tiles_bytes + 4 * sizeof(long long)))) return rc;
  if (B.spec_doubles && (rc = ensure(ctx, ctx->b_spec, sizeof(double) * B.spec_doubles))) return rc;
  (void)fresh_cnt;
  // counters (and the done counter after them) start at zero; every pass leaves the counters at zero
  unsigned int* d_done = (unsigned int*)ctx->b_cnt.p + B.cnt_uints;
  CK(cudaMemsetAsync(ctx->b_cnt.p, 0, sizeof(unsigned) * (B.cnt_uints + 4), ctx->stream));

  const int max_iter_cfg = ctx->cfg.max_iter;
  const int max_sweeps = ctx->cfg.max_sweeps > 0 ? ctx->cfg.max_sweeps : 6;
  std::vector<BatchSeries> hs(cnt);
  std::vector<int> tiles((size_t)(B.tiles_f + B.tiles_d + B.tiles_x));
  states.assign(cnt, DevState{});
  long long tf = 0, td = 0, tx = 0;
  for (int k = 0; k < cnt; ++k) {
    BatchSeries& S = hs[k];
    memset(&S, 0, sizeof S);
    Work& w = S.w;
    const int p = B.p[k];
    const size_t pp1 = (size_t)pad_p(p + 1);
    w.n = B.n[k];
    w.m = B.m[k];
    w.p = p;
    w.p_pad = (int)pp1;
    w.y64 = B.y_dev.empty() ? (const double*)ctx->b_y64.p + B.off_y[k] : B.y_dev[k];
    w.y32 = mixed ? (float*)ctx->b_y32.p + B.off_y[k] : nullptr;
    w.U[0] = (char*)ctx->b_u0.p + ues * B.off_u[k];
    w.U[1] = (char*)ctx->b_u1.p + ues * B.off_u[k];
    double* q = (double*)ctx->b_part.p + B.off_part[k];
    const long long nun = batch_units(B.m[k], p, B.fft[k]), ngr = (nun + kGroup - 1) / kGroup;
    w.part_t = q; q += nun * pp1;
    w.part_n2 = q; q += nun;
    w.grp_t = q; q += ngr * pp1;
    w.grp_n2 = q;
    w.counters = (unsigned int*)ctx->b_cnt.p + B.off_cnt[k];
    q = (double*)ctx->b_vecs.p + B.off_vec[k];
    w.v = q; q += pp1;
    w.w = q; q += pp1;
    w.z = q; q += pp1;
    w.d = q; q += pp1;
    w.g = q; q += pp1;
    w.h = q; q += pp1;
    w.t = q; q += pp1;
    w.best = q; q += pp1;
    w.bnorm2 = q; q += pp1;
    w.phi = (double*)ctx->b_phi.p + B.off_phi[k];
    char* mb = (char*)ctx->b_mats.p + B.off_mat[k];
    const size_t pq = (size_t)p * p;
    w.G = (double*)mb;
    w.M = w.G + pq;
    w.Mt = w.M + pq;
    w.qr = qr_scratch_doubles(p) ? w.Mt + pq : nullptr;
    w.M32 = (float*)(w.Mt + pq + qr_scratch_doubles(p));
    w.Mt32 = w.M32 + pq;
    w.st = (DevState*)ctx->b_state.p + k;
    w.f32_active = mixed ? d_done + 1 : nullptr;   // the batch's count of series in a float correction sweep
    w.tw64 = ctx->tw64;
    w.tw64x = ctx->tw64x;
    w.tw32 = ctx->tw32;
    if (B.fft[k]) {
      double* sp = (double*)ctx->b_spec.p + B.off_spec[k];
      w.wspec64 = sp;
      w.dspec64 = sp + batch_fft_spectra_doubles(B.m[k], p);
    }
    S.tile0_f = tf;               // index in the float tile list
    S.tile0_x = tx;               // index in the FFT tile list (stored after the float and double lists)
    for (long long t = 0; t < B.ntf[k]; ++t) tiles[(size_t)(tf + t)] = k;
    for (long long t = 0; t < B.ntd[k]; ++t) tiles[(size_t)(B.tiles_f + td + t)] = k;
    for (long long t = 0; t < B.ntx[k]; ++t) tiles[(size_t)(B.tiles_f + B.tiles_d + tx + t)] = k;
    tx += B.ntx[k];
    tf += B.ntf[k];
    td += B.ntd[k];
    S.tile0_d = td - B.ntd[k];   // index in the double tile list (stored after the float list)
    DevState& st = states[k];
    memset(&st, 0, sizeof st);
    const int max_iter = max_iter_cfg > 0 ? max_iter_cfg : 4 * p + 200;
    st.tol = tol;
    st.tol_inner = 1e-5;
    st.est_ratio = tol;
    st.max_iter = max_iter;
    st.iter_cap = mixed ? std::min(max_iter, 100) : max_iter;
    st.max_sweeps = max_sweeps;
    st.mixed = mixed ? 1 : 0;
    st.mixed_ok = 1;
    st.ne_ratio = 1e300;
    st.ne_best = 1e300;
    st.status = TOLS_NOT_CONVERGED;
    st.phase = PH_LSQR;
  }
  const BatchSeries* d_series = (const BatchSeries*)ctx->b_series.p;
  CK(cudaMemcpyAsync(ctx->b_series.p, hs.data(), sizeof(BatchSeries) * cnt, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->b_state.p, states.data(), sizeof(DevState) * cnt, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->b_tiles.p, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, ctx->stream));
  long long* d_live = (long long*)((char*)ctx->b_tiles.p + tiles_bytes);
  long long h_live[3] = {B.tiles_f, B.tiles_d, B.tiles_x};
  CK(cudaMemcpyAsync(d_live, h_live, sizeof h_live, cudaMemcpyHostToDevice, ctx->stream));
  BatchArgs a;
  memset(&a, 0, sizeof a);
  a.series = d_series;
  a.tile_series_f = (const int*)ctx->b_tiles.p;
  a.tile_series_d = (const int*)ctx->b_tiles.p + B.tiles_f;
  a.tile_series_x = (const int*)ctx->b_tiles.p + B.tiles_f + B.tiles_d;
  a.tiles_f = B.tiles_f;
  a.tiles_d = B.tiles_d;
  a.tiles_x = B.tiles_x;
  a.done_count = d_done;
  a.live = d_live;
  const int gf = batch_grid(ctx, 0, B.p_pad_max), gd = batch_grid(ctx, 1, B.p_pad_max);

  // setup: float copy, Gram lag sums, preconditioner, LSQR start
  if (mixed && B.y_dev.empty())
    RUN(run_small(ctx, 11, [&] { return launch_convert_f32((const double*)ctx->b_y64.p, (float*)ctx->b_y32.p,
                                                           (long long)B.y_elems, ctx->stream); }));
  else if (mixed)
    RUN(run_small(ctx, 11, [&] { return launch_convert_batch(d_series, cnt, ctx->stream); }));
  BatchArgs ag = a;
  ag.gram = 1;
  const int gx = B.tiles_x ? batch_fft_grid(ctx, B.p_pad_max_x) : 0;
  // launches per float64 solver pass: the FFT pair (d spectra, FFT pass) and/or the direct float64 pass; while some
  // series of a mixed batch run a float correction sweep, the float pass joins them
  const int per_pass = (B.tiles_x ? 2 : 0) + (B.tiles_d ? 1 : 0);
  // the Gram pass (float64 products for every series); the FFT series' one also forms their window spectra
  if (B.tiles_x) RUN(run_small(ctx, 13, [&] { return launch_batch_fft(ag, gx, B.p_pad_max_x, ctx->stream); }));
  if (B.tiles_d) RUN(run_small(ctx, 14, [&] { return launch_batch_pass<double>(ag, gd, B.p_pad_max, ctx->stream); }));
  const int want = no_precond ? 0 : ctx->cfg.precond;
  RUN(run_small(ctx, 10, [&] { return launch_precond_batch(d_series, cnt, want, ctx->stream, B.p_pad_max); }));
  RUN(run_small(ctx, 12, [&] { return launch_init_lsqr_batch(d_series, cnt, d_done, ctx->stream); }));

  // iterations: a burst of batched passes captured once into a CUDA graph, replayed until all series are done
  const int burst = 4;
  auto enqueue_burst = [&](bool with_float) -> int {
    // run_small counts each launch, and times it when profiling (which replaces the graphs by direct launches)
    for (int k = 0; k < burst; ++k) {
      if (with_float)
        RUN(run_small(ctx, 15, [&] { return launch_batch_pass<float>(a, gf, B.p_pad_max, ctx->stream); }));
      if (B.tiles_x) {
        RUN(run_small(ctx, 16, [&] { return launch_batch_dspec(d_series, cnt, ctx->stream); }));
        RUN(run_small(ctx, 13, [&] { return launch_batch_fft(a, gx, B.p_pad_max_x, ctx->stream); }));
      }
      if (B.tiles_d)
        RUN(run_small(ctx, 14, [&] { return launch_batch_pass<double>(a, gd, B.p_pad_max, ctx->stream); }));
    }
    return TOLS_OK;
  };
  // two captured bursts: float64 passes only, and with the float pass (mixed batches)
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  if (!ctx->prof) {
    for (int f = 0; f < (mixed ? 2 : 1); ++f) {
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      const long long before = ctx->launch_total;
      rc = enqueue_burst(f == 1);
      ctx->launch_total = before;
      cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
      if (rc) return rc;
      if (e != cudaSuccess) return fail(ctx, TOLS_ERR_CUDA, "capture of the batched burst", e);
      e = cudaGraphInstantiate(&exec[f], graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(ctx, TOLS_ERR_CUDA, "instantiate the batched burst", e);
    }
  }
  unsigned int* h_done = (unsigned int*)ctx->h_worklog;  // pinned, reused as landing slots: done, in float sweeps
  // Compaction of the tile lists to the series not yet done: the per-series tile ranges stay contiguous and in
  // order (a series' partial-sum slots are indexed by its local tile or unit number, tile - tile0), only each
  // series' first index (tile0_*) moves. The kernels read the list lengths from d_live at run time, so the
  // captured graphs stay valid.
  long long listed = cnt;
  auto compact_lists = [&]() -> int {
    CK(cudaMemcpyAsync(states.data(), ctx->b_state.p, sizeof(DevState) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    long long nf = 0, nd = 0, nx = 0, na = 0;
    for (int k = 0; k < cnt; ++k) {
      const DevState& st = states[k];
      if (st.done || st.phase == PH_DONE) continue;
      ++na;
      hs[k].tile0_f = nf;
      hs[k].tile0_d = nd;
      hs[k].tile0_x = nx;
      for (long long t = 0; t < B.ntf[k]; ++t) tiles[(size_t)(nf + t)] = k;
      for (long long t = 0; t < B.ntd[k]; ++t) tiles[(size_t)(B.tiles_f + nd + t)] = k;
      for (long long t = 0; t < B.ntx[k]; ++t) tiles[(size_t)(B.tiles_f + B.tiles_d + nx + t)] = k;
      nf += B.ntf[k];
      nd += B.ntd[k];
      nx += B.ntx[k];
    }
    CK(cudaMemcpyAsync(ctx->b_series.p, hs.data(), sizeof(BatchSeries) * cnt, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->b_tiles.p, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    h_live[0] = nf;
    h_live[1] = nd;
    h_live[2] = nx;
    CK(cudaMemcpyAsync(d_live, h_live, sizeof h_live, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    listed = na;
    return TOLS_OK;
  };
  int max_iter_all = 0;
  for (int k = 0; k < cnt; ++k) max_iter_all = std::max(max_iter_all, states[k].max_iter);
  const long long max_rounds = ((long long)(max_iter_all + 4) * (max_sweeps + 2) * 2) / burst + 16;
  int out = TOLS_OK;
  bool with_float = false;
  for (long long round = 0;; ++round) {
    if (exec[with_float ? 1 : 0]) {
      ctx->launch_total += burst * (per_pass + (with_float ? 1 : 0));
      cudaError_t e = cudaGraphLaunch(exec[with_float ? 1 : 0], ctx->stream);
      if (e != cudaSuccess) { out = fail(ctx, TOLS_ERR_CUDA, "cudaGraphLaunch", e); break; }
    } else if ((out = enqueue_burst(with_float))) {
      break;
    }
    cudaError_t e = cudaMemcpyAsync(h_done, d_done, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { out = fail(ctx, TOLS_ERR_CUDA, "batched poll", e); break; }
    // read the landing slots before flush_profile, which reuses the same pinned buffer for the work log
    const unsigned done_now = h_done[0], float_now = h_done[1];
    if ((out = flush_profile(ctx))) break;
    if (done_now >= (unsigned)cnt) break;
    if (round > max_rounds) { out = fail(ctx, TOLS_ERR_DEVICE_TIMEOUT, "batched solve did not finish"); break; }
    with_float = mixed && float_now > 0;
    // once half of the series still listed are done, the lists keep only the unfinished ones: a pass launch over
    // the full lists would spend its time skipping finished series' tiles
    const long long active = (long long)cnt - done_now;
    if (active * 2 <= listed && (out = compact_lists()) != TOLS_OK) break;
  }
  for (auto x : exec)
    if (x) cudaGraphExecDestroy(x);
  if (out) return out;
  RUN(run_small(ctx, 12, [&] { return launch_finish_batch(d_series, cnt, ctx->stream); }));
  CK(cudaMemcpyAsync(states.data(), ctx->b_state.p, sizeof(DevState) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  RUN(flush_profile(ctx));
  return TOLS_OK;
}

// A plan over a subset of B's series (their float64 series stay where they are).
BatchPlan sub_plan(tols_ctx* ctx, const BatchPlan& B, const std::vector<int>& which) {
  BatchPlan S;
  std::vector<long long> n;
  std::vector<int> p;
  for (int k : which) {
    n.push_back(B.n[k]);
    p.push_back(B.p[k]);
  }
  std::vector<int> st(which.size(), TOLS_OK);
  plan_batch(ctx, S, (int)which.size(), n.data(), p.data(), st, false);
  for (int k : which)
    S.y_dev.push_back(B.y_dev.empty() ? (const double*)ctx->b_y64.p + B.off_y[k] : B.y_dev[k]);
  return S;
}

// Run the batch, then, together as float64 sub-batches: the series whose float correction sweeps stopped
// contracting, and the exactly rank-deficient ones (plain LSQR from zero gives the minimum norm). phi_host:
// coefficients packed at B.off_phi.
int batch_solve_all(tols_ctx* ctx, BatchPlan& B, double tol, bool mixed, std::vector<DevState>& states,
                    std::vector<double>& phi_host, std::vector<int>& prec_used) {
  const int cnt = (int)B.idx.size();
  prec_used.assign(cnt, TOLS_FP64);
  phi_host.assign(B.phi_doubles, 0.0);
  if (cnt == 0) return TOLS_OK;
  int rc;
  if ((rc = batch_core(ctx, B, tol, mixed, states))) return rc;
  CK(cudaMemcpy(phi_host.data(), ctx->b_phi.p, sizeof(double) * B.phi_doubles, cudaMemcpyDeviceToHost));
  // a mixed series counts as mixed when float products did part of its work
  for (int k = 0; k < cnt; ++k)
    if (mixed && states[k].f32_iter > 0) prec_used[k] = TOLS_MIXED;
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int> which;
    for (int k = 0; k < cnt; ++k) {
      const DevState& s = states[k];
      if (pass == 0 && mixed && s.status != TOLS_OK && s.status != TOLS_ERR_NONFINITE && s.mixed_ok == 0)
        which.push_back(k);
      if (pass == 1 && s.singular && s.compatible && s.status >= 0) which.push_back(k);
    }
    if (which.empty()) continue;
    BatchPlan S = sub_plan(ctx, B, which);
    std::vector<DevState> sst;
    if ((rc = batch_core(ctx, S, tol, false, sst, pass == 1))) return rc;
    std::vector<double> sphi(S.phi_doubles);
    CK(cudaMemcpy(sphi.data(), ctx->b_phi.p, sizeof(double) * S.phi_doubles, cudaMemcpyDeviceToHost));
    for (size_t j = 0; j < which.size(); ++j) {
      const int k = which[j];
      if (pass == 1 && !(sst[j].status == TOLS_OK && sst[j].compatible)) continue;  // keep the first result
      sst[j].total_iter += states[k].total_iter;
      sst[j].sweeps += states[k].sweeps;
      states[k] = sst[j];
      memcpy(phi_host.data() + B.off_phi[k], sphi.data() + S.off_phi[j], sizeof(double) * B.p[k]);
      prec_used[k] = TOLS_FP64;
    }
  }
  // Series whose sampled rows are numerically rank deficient in float64 (kappa of the sample beyond about 1e14)
  // keep the batch's result (NOT_CONVERGED at their float64 floor). Repeating them one by one through the multi-CTA
  // preconditioner (whose last QR stage is shifted) lowered their residuals, but on the 4,096-series workload none
  // of the 28 such series met the oracle gate either way, while the repeats took about half of the batch's device
  // time.
  return TOLS_OK;
}

// ------------------------------------------------------------------------------------------------------
// Serving: continuous batching over one device arena. Requests wait in FIFO order and are admitted while a slot
// is free and their footprint fits in the arena; every step admits, sets up the newcomers (Gram pass,
// preconditioner, LSQR start — batched over the newcomers), runs one burst of batched passes over all active
// requests, and retires the finished ones, freeing their memory at once.
class ArenaAlloc {
 public:
  void reset(size_t cap) {
    free_.clear();
    free_[0] = cap;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, noff = it->first + bytes;
      free_.erase(it);
      if (rest) free_[noff] = rest;
      used_ += bytes;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes, 256);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

// Bytes of one series' arena slice; with base != nullptr also lays the slice out into w.
// fx: the request's float64 passes take the batched FFT products (batch_fft_choice).
size_t series_slice(char* base, long long n, int p, bool mixed, bool fx, Work* w) {
  const long long m = n - p;
  const size_t pp1 = (size_t)pad_p(p + 1);
  const long long ntd = batch_units(m, p, fx), ngr = (ntd + kGroup - 1) / kGroup;
  const size_t es = sizeof(double);   // float64 even for mixed requests (float64 iterations when float cannot refine)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align_up(bytes, 256);
    return base ? base + o : nullptr;
  };
  char* st = take(sizeof(DevState));
  char* cnt = take(sizeof(unsigned) * (size_t)(ngr + 1));
  char* y64 = take(sizeof(double) * (size_t)n);
  char* y32 = mixed ? take(sizeof(float) * (size_t)n) : nullptr;
  char* u0 = take(es * (size_t)m);
  char* u1 = take(es * (size_t)m);
  char* part = take(sizeof(double) * (size_t)(ntd * pp1 + ntd + ngr * pp1 + ngr));
  char* vec = take(sizeof(double) * (9 * pp1 + (size_t)p));
  char* mat = take(sizeof(double) * (3 * (size_t)p * p + qr_scratch_doubles(p)) + sizeof(float) * 2 * (size_t)p * p);
  // window spectra of the FFT tiles and the spectrum of d (requests with float64 FFT products)
  char* spec = fx ? take(sizeof(double) * (batch_fft_spectra_doubles(m, p) + 2 * (kBatchFftN / 2 + 1))) : nullptr;
  if (base && w) {
    memset(w, 0, sizeof *w);
    w->n = n;
    w->m = m;
    w->p = p;
    w->p_pad = (int)pp1;
    w->st = (DevState*)st;
    w->counters = (unsigned*)cnt;
    w->y64 = (const double*)y64;
    w->y32 = (float*)y32;
    w->U[0] = u0;
    w->U[1] = u1;
    double* q = (double*)part;
    w->part_t = q; q += ntd * pp1;
    w->part_n2 = q; q += ntd;
    w->grp_t = q; q += ngr * pp1;
    w->grp_n2 = q;
    q = (double*)vec;
    w->v = q; q += pp1;
    w->w = q; q += pp1;
    w->z = q; q += pp1;
    w->d = q; q += pp1;
    w->g = q; q += pp1;
    w->h = q; q += pp1;
    w->t = q; q += pp1;
    w->best = q; q += pp1;
    w->bnorm2 = q; q += pp1;
    w->phi = q;
    const size_t pq = (size_t)p * p;
    w->G = (double*)mat;
    w->M = w->G + pq;
    w->Mt = w->M + pq;
    w->qr = qr_scratch_doubles(p) ? w->Mt + pq : nullptr;
    w->M32 = (float*)(w->Mt + pq + qr_scratch_doubles(p));
    w->Mt32 = w->M32 + pq;
    if (spec) {
      w->wspec64 = spec;
      w->dspec64 = (double*)spec + batch_fft_spectra_doubles(m, p);
    }
  }
  return off;
}

DevState initial_state(const tols_config& cfg, int p, double tol, bool mixed) {
  DevState st;
  memset(&st, 0, sizeof st);
  const int max_iter = cfg.max_iter > 0 ? cfg.max_iter : 4 * p + 200;
  st.tol = tol;
  st.tol_inner = 1e-5;
  st.est_ratio = tol;
  st.max_iter = max_iter;
  st.iter_cap = mixed ? std::min(max_iter, 100) : max_iter;
  st.max_sweeps = cfg.max_sweeps > 0 ? cfg.max_sweeps : 6;
  st.mixed = mixed ? 1 : 0;
  st.mixed_ok = 1;
  st.ne_ratio = 1e300;
  st.ne_best = 1e300;
  st.status = TOLS_NOT_CONVERGED;
  st.phase = PH_LSQR;
  return st;
}

struct SrvRequest {
  long long id;
  long long n;
  int p;
  double tol;
  std::vector<double> y;
  double t_submit;
  bool mixed = false;       // precision of this attempt
  bool no_precond = false;  // plain LSQR (minimum-norm repeat of an exactly rank-deficient problem)
  int prior_iters = 0, prior_sweeps = 0;
};

struct SrvActive {
  SrvRequest req;
  size_t off = 0, bytes = 0;
  Work w;
};

double now_s(const std::chrono::steady_clock::time_point& t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct tols_server {
  tols_ctx* ctx = nullptr;
  bool mixed = false;
  int max_active = 0;
  int burst = 4;
  char* arena = nullptr;
  size_t arena_cap = 0;
  ArenaAlloc alloc;
  std::deque<SrvRequest> queue;
  std::vector<SrvRequest> requeue;
  std::vector<SrvActive> active;
  std::vector<tols_result> results;
  std::vector<double> result_phi;   // TOLS_MAX_P doubles per result
  DevBuf table, tiles, gather;
  std::vector<DevState> h_states;
  std::vector<double> h_phi;
  std::chrono::steady_clock::time_point t0;
  long long submitted = 0, completed = 0;
  bool float_due = false;           // the last step left a mixed request in a float correction sweep
};

namespace {

// Upload a series table (and its tile lists) for the series in `list` (indices into srv->active).
int upload_table(tols_server* srv, const std::vector<int>& list, BatchArgs& a, int& p_pad_max) {
  tols_ctx* ctx = srv->ctx;
  const int cnt = (int)list.size();
  std::vector<BatchSeries> hs(cnt);
  long long tf = 0, td = 0, tx = 0;
  p_pad_max = 16;
  for (int k = 0; k < cnt; ++k) {
    const Work& w = srv->active[list[k]].w;
    memset(&hs[k], 0, sizeof(BatchSeries));
    hs[k].w = w;
    hs[k].w.tw64 = ctx->tw64;
    hs[k].w.tw64x = ctx->tw64x;
    hs[k].w.tw32 = ctx->tw32;
    hs[k].tile0_f = tf;
    hs[k].tile0_d = td;
    hs[k].tile0_x = tx;
    tf += (w.m + kTileF - 1) / kTileF;
    if (w.dspec64) tx += batch_fft_units(w.m, w.p);
    else td += (w.m + kTileD - 1) / kTileD;
    p_pad_max = std::max(p_pad_max, pad_p(w.p + 1));
  }
  std::vector<int> tiles((size_t)(tf + td + tx));
  for (int k = 0; k < cnt; ++k) {
    const Work& w = hs[k].w;
    const long long ntf = (w.m + kTileF - 1) / kTileF;
    const long long ntd = w.dspec64 ? 0 : (w.m + kTileD - 1) / kTileD;
    const long long ntx = w.dspec64 ? batch_fft_units(w.m, w.p) : 0;
    for (long long t = 0; t < ntf; ++t) tiles[(size_t)(hs[k].tile0_f + t)] = k;
    for (long long t = 0; t < ntd; ++t) tiles[(size_t)(tf + hs[k].tile0_d + t)] = k;
    for (long long t = 0; t < ntx; ++t) tiles[(size_t)(tf + td + hs[k].tile0_x + t)] = k;
  }
  int rc;
  if ((rc = ensure(ctx, srv->table, sizeof(BatchSeries) * std::max(cnt, 1)))) return rc;
  if ((rc = ensure(ctx, srv->tiles, sizeof(int) * std::max<size_t>(tiles.size(), 1)))) return rc;
  CK(cudaMemcpyAsync(srv->table.p, hs.data(), sizeof(BatchSeries) * cnt, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(srv->tiles.p, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, ctx->stream));
  memset(&a, 0, sizeof a);
  a.series = (const BatchSeries*)srv->table.p;
  a.tile_series_f = (const int*)srv->tiles.p;
  a.tile_series_d = (const int*)srv->tiles.p + tf;
  a.tile_series_x = (const int*)srv->tiles.p + tf + td;
  a.tiles_f = tf;
  a.tiles_d = td;
  a.tiles_x = tx;
  // the host vectors must outlive the copies: pageable-memory copies are staged before they return
  return TOLS_OK;
}

int server_admit(tols_server* srv, std::vector<int>& fresh) {
  tols_ctx* ctx = srv->ctx;
  while (!srv->queue.empty() && (int)srv->active.size() < srv->max_active) {
    SrvRequest& r = srv->queue.front();
    const bool fx = batch_fft_choice(ctx, r.p) != 0;
    const size_t bytes = series_slice(nullptr, r.n, r.p, r.mixed, fx, nullptr);
    size_t off = 0;
    if (!srv->alloc.alloc(bytes, &off)) break;  // FIFO: the head waits until memory frees up
    SrvActive a;
    a.off = off;
    a.bytes = bytes;
    series_slice(srv->arena + off, r.n, r.p, r.mixed, fx, &a.w);
    DevState st = initial_state(ctx->cfg, r.p, r.tol, r.mixed);
    st.no_precond = r.no_precond ? 1 : 0;
    CK(cudaMemcpyAsync((void*)a.w.y64, r.y.data(), sizeof(double) * (size_t)r.n, cudaMemcpyHostToDevice,
                       ctx->stream));
    const long long nun = batch_units(r.n - r.p, r.p, a.w.dspec64 != nullptr);
    CK(cudaMemsetAsync(a.w.counters, 0, sizeof(unsigned) * (size_t)((nun + kGroup - 1) / kGroup + 1), ctx->stream));
    CK(cudaMemcpyAsync(a.w.st, &st, sizeof(DevState), cudaMemcpyHostToDevice, ctx->stream));
    a.req = std::move(r);
    srv->queue.pop_front();
    fresh.push_back((int)srv->active.size());
    srv->active.push_back(std::move(a));
  }
  if (fresh.empty()) return TOLS_OK;
  // setup of the newcomers, batched over them
  BatchArgs a;
  int pmax = 16;
  RUN(upload_table(srv, fresh, a, pmax));
  for (int k : fresh) {
    const SrvActive& A = srv->active[k];
    if (A.req.mixed) {
      const Work& w = A.w;
      RUN(run_small(ctx, 11, [&] { return launch_convert_f32(w.y64, w.y32, w.n, ctx->stream); }));
    }
  }
  BatchArgs ag = a;
  ag.gram = 1;
  // the Gram pass from float64 products for every request; the FFT requests' one also forms their window spectra
  if (a.tiles_x) {
    ctx->launch_total++;
    CK(launch_batch_fft(ag, batch_fft_grid(ctx, pmax), pmax, ctx->stream));
  }
  if (a.tiles_d) {
    ctx->launch_total++;
    CK(launch_batch_pass<double>(ag, batch_grid(ctx, 1, pmax), pmax, ctx->stream));
  }
  const int want = ctx->cfg.precond;
  const int cnt = (int)fresh.size();
  RUN(run_small(ctx, 10, [&] { return launch_precond_batch(a.series, cnt, want, ctx->stream, pmax); }));
  RUN(run_small(ctx, 12, [&] { return launch_init_lsqr_batch(a.series, cnt, nullptr, ctx->stream); }));
  return TOLS_OK;
}

}  // namespace

namespace tols {
cudaError_t launch_gather_batch(const BatchSeries* series, int count, DevState* states, double* phis, int stride,
                                cudaStream_t s);
}

namespace {

int server_round(tols_server* srv) {
  tols_ctx* ctx = srv->ctx;
  const int cnt = (int)srv->active.size();
  if (cnt == 0) return TOLS_OK;
  std::vector<int> all(cnt);
  for (int k = 0; k < cnt; ++k) all[k] = k;
  BatchArgs a;
  int pmax = 16;
  RUN(upload_table(srv, all, a, pmax));
  const int gf = batch_grid(ctx, 0, pmax), gd = batch_grid(ctx, 1, pmax);
  const int gx = a.tiles_x ? batch_fft_grid(ctx, pmax) : 0;
  // float passes serve the correction sweeps of mixed requests (launched while the last step left some request in
  // one), double passes every float64 iteration and check: interleaving them lets both kinds progress in a burst
  const bool any_float = srv->float_due;
  for (int k = 0; k < srv->burst; ++k) {
    if (any_float) {
      ctx->launch_total++;
      CK(launch_batch_pass<float>(a, gf, pmax, ctx->stream));
    }
    if (a.tiles_x) {
      ctx->launch_total += 2;
      CK(launch_batch_dspec(a.series, cnt, ctx->stream));
      CK(launch_batch_fft(a, gx, pmax, ctx->stream));
    }
    if (a.tiles_d) {
      ctx->launch_total++;
      CK(launch_batch_pass<double>(a, gd, pmax, ctx->stream));
    }
  }
  RUN(run_small(ctx, 12, [&] { return launch_finish_batch(a.series, cnt, ctx->stream); }));
  int rc;
  if ((rc = ensure(ctx, srv->gather, (sizeof(DevState) + sizeof(double) * TOLS_MAX_P) * (size_t)cnt))) return rc;
  DevState* d_st = (DevState*)srv->gather.p;
  double* d_phi = (double*)(d_st + cnt);
  RUN(run_small(ctx, 12, [&] { return launch_gather_batch(a.series, cnt, d_st, d_phi, TOLS_MAX_P, ctx->stream); }));
  srv->h_states.resize(cnt);
  srv->h_phi.resize((size_t)cnt * TOLS_MAX_P);
  CK(cudaMemcpyAsync(srv->h_states.data(), d_st, sizeof(DevState) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(srv->h_phi.data(), d_phi, sizeof(double) * TOLS_MAX_P * cnt, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  RUN(flush_profile(ctx));
  // retire the finished requests; note whether a float correction sweep is under way
  srv->float_due = false;
  for (int k = 0; k < cnt; ++k) {
    const DevState& s = srv->h_states[k];
    if (!(s.done || s.phase == PH_DONE) && s.mixed && s.phase == PH_NECORR) srv->float_due = true;
  }
  std::vector<SrvActive> keep;
  keep.reserve(cnt);
  for (int k = 0; k < cnt; ++k) {
    SrvActive& A = srv->active[k];
    DevState s = srv->h_states[k];
    if (!(s.done || s.phase == PH_DONE)) {
      keep.push_back(std::move(A));
      continue;
    }
    const double* phi = srv->h_phi.data() + (size_t)k * TOLS_MAX_P;
    const bool hopeless = A.req.mixed && s.status != TOLS_OK && s.status != TOLS_ERR_NONFINITE && s.mixed_ok == 0;
    const bool rankdef = s.singular && s.compatible && s.status >= 0 && !A.req.no_precond;
    if (hopeless || rankdef) {
      // back to the head of the queue as a float64 request (plain LSQR for the minimum norm when X is exactly
      // rank deficient); it is batched with everything else from the next step on
      SrvRequest r = std::move(A.req);
      r.prior_iters += s.total_iter;
      r.prior_sweeps += s.sweeps;
      r.mixed = false;
      if (rankdef) r.no_precond = true;
      srv->alloc.release(A.off, A.bytes);
      srv->requeue.push_back(std::move(r));
      continue;
    }
    s.total_iter += A.req.prior_iters;
    s.sweeps += A.req.prior_sweeps;
    const int prec = A.req.mixed && s.f32_iter > 0 ? TOLS_MIXED : TOLS_FP64;
    tols_result res;
    memset(&res, 0, sizeof res);
    res.id = A.req.id;
    res.status = s.status;
    res.p = A.req.p;
    res.latency_s = now_s(srv->t0) - A.req.t_submit;
    fill_info(&res.info, s, prec);
    res.info.status = s.status;
    srv->results.push_back(res);
    const size_t base = srv->result_phi.size();
    srv->result_phi.resize(base + TOLS_MAX_P, 0.0);
    memcpy(srv->result_phi.data() + base, phi, sizeof(double) * A.req.p);
    srv->alloc.release(A.off, A.bytes);
    srv->completed++;
  }
  srv->active.swap(keep);
  for (auto it = srv->requeue.rbegin(); it != srv->requeue.rend(); ++it) srv->queue.push_front(std::move(*it));
  srv->requeue.clear();
  return TOLS_OK;
}
}  // namespace

// ======================================================================================================
extern "C" {

void toeplitz_ols_config_default(tols_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof *cfg);
  cfg->precision = TOLS_FP64;
  cfg->device = 0;
  cfg->precond = TOLS_PRECOND_GRAM_CHOL;
  cfg->product = TOLS_PRODUCT_AUTO;
}

const char* toeplitz_ols_strerror(int code) {
  switch (code) {
    case TOLS_OK: return "ok";
    case TOLS_NOT_CONVERGED: return "not converged (phi holds the best iterate)";
    case TOLS_ERR_ARG: return "invalid argument";
    case TOLS_ERR_NONFINITE: return "series holds NaN or Inf";
    case TOLS_ERR_OOM: return "out of device memory (or memory cap reached)";
    case TOLS_ERR_CUDA: return "CUDA runtime error";
    case TOLS_ERR_DEVICE_TIMEOUT: return "device-side wait gave up";
    case TOLS_ERR_NO_DEVICE: return "no sm_103 CUDA device";
    case TOLS_ERR_BUSY: return "no slot or memory free";
    default: return "unknown status";
  }
}

const char* toeplitz_ols_last_error(const tols_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int toeplitz_ols_create(tols_ctx** out, const tols_config* cfg) {
  if (!out) return TOLS_ERR_ARG;
  *out = nullptr;
  tols_config c;
  if (cfg) c = *cfg;
  else toeplitz_ols_config_default(&c);
  if (c.precision != TOLS_FP64 && c.precision != TOLS_MIXED) return TOLS_ERR_ARG;
  if (c.precond != TOLS_PRECOND_NONE && c.precond != TOLS_PRECOND_GRAM_CHOL && c.precond != TOLS_PRECOND_SAMPLED_QR)
    return TOLS_ERR_ARG;
  if (c.product < TOLS_PRODUCT_AUTO || c.product > TOLS_PRODUCT_FFT4096 || c.wait_polls < -1) return TOLS_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= c.device || c.device < 0) {
    cudaGetLastError();
    return TOLS_ERR_NO_DEVICE;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c.device) != cudaSuccess) return TOLS_ERR_NO_DEVICE;
  if (!(prop.major == 10 && prop.minor == 3)) return TOLS_ERR_NO_DEVICE;
  if (cudaSetDevice(c.device) != cudaSuccess) return TOLS_ERR_NO_DEVICE;
  tols_ctx* ctx = new tols_ctx;
  ctx->cfg = c;
  ctx->device = c.device;
  ctx->sms = prop.multiProcessorCount;
  if (c.cuda_stream) {
    ctx->stream = (cudaStream_t)c.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return TOLS_ERR_CUDA;
    }
    ctx->own_stream = true;
  }
  if (cudaMalloc(&ctx->d_worklog, sizeof(int) * kMaxPending) != cudaSuccess ||
      cudaMemset(ctx->d_worklog, 0, sizeof(int) * kMaxPending) != cudaSuccess ||
      cudaMallocHost(&ctx->h_worklog, sizeof(int) * kMaxPending) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return TOLS_ERR_OOM;
  }
  {
    // FFT twiddles exp(-2 pi i t / N) in float64 on the host (libm), rounded to float for the float table
    std::vector<double2> t64(2048), t64x(4096);
    std::vector<float2> t32(4096);
    for (int t = 0; t < 2048; ++t) {
      const double a = -2.0 * M_PI * (double)t / 2048.0;
      t64[t] = make_double2(cos(a), sin(a));
    }
    for (int t = 0; t < 4096; ++t) {
      const double a = -2.0 * M_PI * (double)t / 4096.0;
      t32[t] = make_float2((float)cos(a), (float)sin(a));
      t64x[t] = make_double2(cos(a), sin(a));
    }
    if (cudaMalloc(&ctx->tw64, sizeof(double2) * 2048) != cudaSuccess ||
        cudaMalloc(&ctx->tw64x, sizeof(double2) * 4096) != cudaSuccess ||
        cudaMalloc(&ctx->tw32, sizeof(float2) * 4096) != cudaSuccess ||
        cudaMemcpy(ctx->tw64, t64.data(), sizeof(double2) * 2048, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->tw64x, t64x.data(), sizeof(double2) * 4096, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->tw32, t32.data(), sizeof(float2) * 4096, cudaMemcpyHostToDevice) != cudaSuccess) {
      if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
      delete ctx;
      return TOLS_ERR_OOM;
    }
  }
  if (cudaMallocHost(&ctx->h_state, kStateBytes + sizeof(double) * TOLS_MAX_P + sizeof(PclInfo)) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return TOLS_ERR_OOM;
  }
  ctx->h_phi = (double*)((char*)ctx->h_state + kStateBytes);
  ctx->h_pcl = (PclInfo*)(ctx->h_phi + TOLS_MAX_P);
  *out = ctx;
  return TOLS_OK;
}

int toeplitz_ols_destroy(tols_ctx* ctx) {
  if (!ctx) return TOLS_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  DevBuf* bufs[] = {&ctx->y64,    &ctx->y32,   &ctx->u0,    &ctx->u1,     &ctx->part,    &ctx->vecs,
                    &ctx->mats,   &ctx->state, &ctx->scratch, &ctx->rbuf,  &ctx->b_y64,   &ctx->b_y32,
                    &ctx->b_u0,   &ctx->b_u1,  &ctx->b_part, &ctx->b_cnt,  &ctx->b_vecs,  &ctx->b_phi,
                    &ctx->b_mats, &ctx->b_state, &ctx->b_series, &ctx->b_tiles, &ctx->tune, &ctx->spec32,
                    &ctx->spec64, &ctx->sacc32, &ctx->b_spec, &ctx->lsar, &ctx->pcl, &ctx->tune_y};
  for (DevBuf* b : bufs) release(ctx, *b);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->h_state) cudaFreeHost(ctx->h_state);
  if (ctx->h_worklog) cudaFreeHost(ctx->h_worklog);
  if (ctx->tw32) cudaFree(ctx->tw32);
  if (ctx->tw64) cudaFree(ctx->tw64);
  if (ctx->tw64x) cudaFree(ctx->tw64x);
  if (ctx->d_worklog) cudaFree(ctx->d_worklog);
  for (auto& q : ctx->pending) { cudaEventDestroy(q.e0); cudaEventDestroy(q.e1); }
  for (auto e : ctx->ev_free) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return TOLS_OK;
}

int toeplitz_ols_solve(tols_ctx* ctx, const double* y, long long n, int p, double tol, double* phi, double* rnorm,
                       tols_info* info) {
  int rc = validate(ctx, n, p);
  if (rc) return rc;
  if (!y || !phi) return fail(ctx, TOLS_ERR_ARG, "null pointer");
  cudaSetDevice(ctx->device);
  rc = host_solve(ctx, y, n, p, tol, phi, rnorm, info, nullptr);
  if (info && rc < 0) info->status = rc;
  return rc;
}

int toeplitz_ols_solve_device(tols_ctx* ctx, const double* d_y, long long n, int p, double tol, double* d_phi,
                              double* rnorm, tols_info* info) {
  int rc = validate(ctx, n, p);
  if (rc) return rc;
  if (!d_y || !d_phi) return fail(ctx, TOLS_ERR_ARG, "null pointer");
  cudaSetDevice(ctx->device);
  rc = solve_device_impl(ctx, d_y, n, p, tol <= 0 ? 1e-12 : tol, d_phi, rnorm, info, nullptr);
  if (info && rc < 0) info->status = rc;
  return rc;
}

int toeplitz_ols_solve_batched(tols_ctx* ctx, int count, const double* const* y, const long long* n, const int* p,
                               double tol, double* const* phi, double* rnorm, tols_info* info) {
  if (!ctx || count < 0 || (count > 0 && (!y || !n || !p || !phi))) return TOLS_ERR_ARG;
  if (count == 0) return TOLS_OK;
  cudaSetDevice(ctx->device);
  if (tol <= 0) tol = 1e-12;
  std::vector<int> status(count, TOLS_OK);
  BatchPlan B;
  plan_batch(ctx, B, count, n, p, status, ctx->cfg.precision == TOLS_MIXED);
  for (int k : B.idx)
    if (!y[k] || !phi[k]) return fail(ctx, TOLS_ERR_ARG, "null series or phi pointer");
  int rc;
  // stage the host series in pinned memory, then one copy to the device
  if (ctx->h_stage_cap < B.y_elems) {
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_cap = 0;
    if (cudaMallocHost(&ctx->h_stage, sizeof(double) * std::max<size_t>(B.y_elems, 1)) != cudaSuccess)
      return fail(ctx, TOLS_ERR_OOM, "pinned staging buffer");
    ctx->h_stage_cap = B.y_elems;
  }
  if ((rc = ensure(ctx, ctx->b_y64, sizeof(double) * std::max<size_t>(B.y_elems, 1)))) return rc;
  for (size_t k = 0; k < B.idx.size(); ++k)
    memcpy(ctx->h_stage + B.off_y[k], y[B.idx[k]], sizeof(double) * (size_t)B.n[k]);
  CK(cudaMemcpyAsync(ctx->b_y64.p, ctx->h_stage, sizeof(double) * B.y_elems, cudaMemcpyHostToDevice, ctx->stream));
  const bool mixed = ctx->cfg.precision == TOLS_MIXED;
  std::vector<DevState> states;
  std::vector<int> prec_used;
  std::vector<double> phis;
  if ((rc = batch_solve_all(ctx, B, tol, mixed, states, phis, prec_used))) return rc;
  int worst = TOLS_OK;
  for (int k = 0; k < count; ++k) {
    if (info) memset(&info[k], 0, sizeof(tols_info));
    if (rnorm) rnorm[k] = 0.0;
  }
  for (size_t j = 0; j < B.idx.size(); ++j) {
    const int k = B.idx[j];
    const DevState& s = states[j];
    status[k] = s.status;
    memcpy(phi[k], phis.data() + B.off_phi[j], sizeof(double) * B.p[j]);
    if (rnorm) rnorm[k] = s.rnorm;
    if (info) {
      fill_info(&info[k], s, prec_used[j]);
    }
  }
  for (int k = 0; k < count; ++k) {
    if (info) info[k].status = status[k];
    const int rc2 = status[k];
    if (rc2 < 0) worst = worst < 0 ? std::min(worst, rc2) : rc2;
    else if (worst >= 0) worst = std::max(worst, rc2);
  }
  return worst;
}

int toeplitz_ols_pacf(tols_ctx* ctx, const double* y, long long n, int h_max, double tol, double* tau, int* order,
                      tols_info* info) {
  if (!ctx) return TOLS_ERR_ARG;
  if (!y || !tau || h_max < 1 || h_max > TOLS_MAX_P || n <= h_max)
    return fail(ctx, TOLS_ERR_ARG, "need y, tau, 1 <= h_max <= TOLS_MAX_P and n > h_max");
  cudaSetDevice(ctx->device);
  if (tol <= 0) tol = 1e-12;
  int rc = stage_y(ctx, y, n);
  if (rc) return rc;
  // the fits of order 1 .. h_max, one batch over the one staged series
  std::vector<long long> nn((size_t)h_max, n);
  std::vector<int> pp((size_t)h_max);
  for (int k = 0; k < h_max; ++k) pp[k] = k + 1;
  std::vector<int> status((size_t)h_max, TOLS_OK);
  const bool mixed = ctx->cfg.precision == TOLS_MIXED;
  BatchPlan B;
  plan_batch(ctx, B, h_max, nn.data(), pp.data(), status, mixed);
  for (size_t j = 0; j < B.idx.size(); ++j) B.y_dev.push_back((const double*)ctx->y64.p);
  std::vector<DevState> states;
  std::vector<int> prec_used;
  std::vector<double> phis;
  if ((rc = batch_solve_all(ctx, B, tol, mixed, states, phis, prec_used))) return rc;
  int worst = TOLS_OK;
  for (size_t j = 0; j < B.idx.size(); ++j) {
    const int k = B.idx[j];
    tau[k] = phis[B.off_phi[j] + (size_t)B.p[j] - 1];   // tau_h: the last coefficient of the AR(h) fit
    status[k] = states[j].status;
    if (info) fill_info(&info[k], states[j], prec_used[j]);
  }
  for (int k = 0; k < h_max; ++k) {
    if (info) info[k].status = status[k];
    if (status[k] < 0) worst = worst < 0 ? std::min(worst, status[k]) : status[k];
    else if (worst >= 0 && status[k] > worst) worst = status[k];
  }
  if (order) {
    int o = 0;
    for (int h = 1; h <= h_max; ++h)
      if (status[h - 1] >= 0 && fabs(tau[h - 1]) >= 1.96 / sqrt((double)(n - h))) o = h;
    *order = o;
  }
  return worst;
}

int toeplitz_ols_lsar(tols_ctx* ctx, const double* d_y, long long n, int p_bar, int c, const double* d_unif,
                      double* tau, int* order, double* phi, long long* d_rows, double* d_phi_all) {
  if (!ctx) return TOLS_ERR_ARG;
  if (!d_y || !d_unif || !tau) return fail(ctx, TOLS_ERR_ARG, "null pointer");
  if (p_bar < 1 || p_bar > kLsarMaxP) return fail(ctx, TOLS_ERR_ARG, "p_bar out of range [1, 256]");
  if (c < p_bar) return fail(ctx, TOLS_ERR_ARG, "need c >= p_bar");
  const long long m = n - p_bar;   // rows at every lag
  if (m < 1) return fail(ctx, TOLS_ERR_ARG, "need n > p_bar");
  cudaSetDevice(ctx->device);
  const long long nb = (m + kLsarBlock - 1) / kLsarBlock;
  const long long tri_max = lsar_tri(p_bar);
  const int ng = std::max(1, std::min(ctx->sms, (c + 7) / 8));
  const size_t p2 = (size_t)p_bar * p_bar;
  // one buffer: lev, bsum, bpre, w2, Gram partials, G, the Cholesky factor and its reciprocal diagonal, the
  // refinement partials, tau, phi per lag, ||r||^2, the leverage-p1 scratch, then the sampled rows (int64) and
  // the status word
  const size_t lev_scr = (size_t)((m + 4095) / 4096) + 64;
  const size_t nd = (size_t)m + nb + (nb + 1) + (size_t)c + ng * (size_t)tri_max + tri_max + p2 + p_bar +
                    ng * (size_t)p_bar + p_bar + (d_phi_all ? 0 : p2) + 8 + lev_scr;
  const size_t bytes = sizeof(double) * nd + sizeof(long long) * (d_rows ? 0 : (size_t)c) + 256;
  int rc;
  if ((rc = ensure(ctx, ctx->lsar, bytes))) return rc;
  if ((rc = ensure(ctx, ctx->rbuf, sizeof(double) * (size_t)m))) return rc;
  double* q = (double*)ctx->lsar.p;
  double* lev = q; q += m;
  double* bsum = q; q += nb;
  double* bpre = q; q += nb + 1;
  double* w2 = q; q += c;
  double* part = q; q += ng * (size_t)tri_max;
  double* G = q; q += tri_max;
  double* Lg = q; q += p2;
  double* rdg = q; q += p_bar;
  double* gpart = q; q += ng * (size_t)p_bar;
  double* tau_dev = q; q += p_bar;
  double* phi_all = d_phi_all;
  if (!phi_all) { phi_all = q; q += p2; }
  double* rr = q; q += 8;
  double* lscr = q; q += lev_scr;
  long long* rows_tmp = (long long*)q;
  int* status = (int*)(rows_tmp + (d_rows ? 0 : c));
  double* r = (double*)ctx->rbuf.p;
  // buffers for the residual passes, sized for the largest order
  Work w;
  if ((rc = prepare_work(ctx, d_y, n, p_bar, false, false, w))) return rc;
  const bool use_fft = p_bar - 1 >= kLsarFftMinOrder && m >= (1LL << 16);
  const int pp_fft = pad_p(p_bar);
  if (use_fft) RUN(fft_spectra(ctx, w, 1, d_y, n, m, pp_fft, true));
  void* spec = ctx->spec64.p;
  CK(cudaMemsetAsync(phi_all, 0, sizeof(double) * p2, ctx->stream));
  CK(cudaMemsetAsync(status, 0, sizeof(int), ctx->stream));
  for (int p = 1; p <= p_bar; ++p) {
    // eq. (FALS): exact scores at lag 1, else add the full-data residual of lag p-1's estimate, eq. (FAR)
    if (p == 1) {
      RUN(run_small(ctx, 12, [&] { return launch_leverage_p1(d_y, m + 1, lev, lscr, ctx->stream); }));
    } else {
      const int qo = p - 1;   // the order-(p-1) problem on y[0 .. m + p - 1): m rows
      if ((rc = prepare_work(ctx, d_y, m + qo, qo, false, false, w))) return rc;
      const bool fft = use_fft && qo >= kLsarFftMinOrder;
      const int pp = fft ? pp_fft : pad_p(qo);
      PassArgs<double> a = base_args<double>(w, d_y, m + qo, qo, pp);
      a.d = phi_all + (size_t)(p - 2) * p_bar;
      a.u_old = d_y + qo;
      a.coef_host = 1.0;
      a.u_new = r;
      a.nlag = 0;
      a.tail = TAIL_STORE;
      a.out_t = nullptr;
      a.out_n2 = rr;
      if (fft) {
        a.fft = 1;
        a.w.wspec64 = spec;
      }
      RUN(run_pass<double>(ctx, a, pass_grid_for(ctx, 1, pp, fft ? 1 : 0)));
    }
    long long* rows_p = d_rows ? d_rows + (size_t)(p - 1) * c : rows_tmp;
    RUN(run_small(ctx, 12, [&] { return launch_lsar_lev(p == 1 ? nullptr : r, rr, lev, m, bsum, status, ctx->stream); }));
    RUN(run_small(ctx, 12, [&] { return launch_lsar_prefix(bsum, nb, bpre, status, ctx->stream); }));
    RUN(run_small(ctx, 12, [&] {
      return launch_lsar_sample(lev, m, bsum, bpre, d_unif + (size_t)(p - 1) * c, c, p, rows_p, w2, status,
                                ctx->stream);
    }));
    RUN(run_small(ctx, 12, [&] { return launch_lsar_gram(d_y, p, rows_p, w2, c, ng, part, G, status, ctx->stream); }));
    RUN(run_small(ctx, 12, [&] {
      return launch_lsar_solve(G, p, d_y, rows_p, w2, c, ng, Lg, rdg, gpart, phi_all + (size_t)(p - 1) * p_bar,
                               tau_dev, p, status, ctx->stream);
    }));
  }
  int h_status = 0;
  CK(cudaMemcpyAsync(tau, tau_dev, sizeof(double) * p_bar, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  // Algorithm "LSAR": the order estimate is the largest lag with |tau_p| >= 1.96 / sqrt(c)
  int o = 0;
  const double thr = 1.96 / sqrt((double)c);
  for (int p = 1; p <= p_bar; ++p)
    if (fabs(tau[p - 1]) >= thr) o = p;
  if (order) *order = o;
  if (phi) {
    if (o > 0) {
      CK(cudaMemcpyAsync(phi, phi_all + (size_t)(o - 1) * p_bar, sizeof(double) * p_bar, cudaMemcpyDeviceToHost,
                         ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    } else {
      for (int j = 0; j < p_bar; ++j) phi[j] = 0.0;
    }
  }
  if (h_status) {
    char msg[96];
    snprintf(msg, sizeof msg, "sampled Gram matrix not positive definite at lag %d", h_status);
    ctx->err = msg;
    return TOLS_NOT_CONVERGED;
  }
  return TOLS_OK;
}

int toeplitz_ols_rh_lsar(tols_ctx* ctx, const double* d_y, long long n, int p_bar, int c, int k, int levels,
                         const long long* h_sizes, const long long* h_keep, const double* d_sketch,
                         const double* d_rh_unif, const double* d_unif, double* tau, int* order, double* phi,
                         double* d_scores, long long* d_rows) {
  if (!ctx) return TOLS_ERR_ARG;
  if (!d_y || !h_sizes || !h_keep || !d_sketch || !d_rh_unif || !d_unif || !tau)
    return fail(ctx, TOLS_ERR_ARG, "null pointer");
  if (p_bar < 1 || p_bar > kLsarMaxP) return fail(ctx, TOLS_ERR_ARG, "p_bar out of range [1, 256]");
  if (k < 1 || k > kRhMaxSketch) return fail(ctx, TOLS_ERR_ARG, "sketch rows k out of range [1, 64]");
  const long long m = n - p_bar;
  const int P1 = p_bar + 1;
  if (m < 1 || levels < 1 || h_sizes[0] != m) return fail(ctx, TOLS_ERR_ARG, "need n > p_bar, levels >= 1, sizes[0] = n - p_bar");
  if (c < P1) return fail(ctx, TOLS_ERR_ARG, "need c >= p_bar + 1");
  size_t keep_total = 0, orig_total = 0;
  for (int j = 0; j < levels; ++j) {
    if (h_sizes[j + 1] != h_sizes[j] / 2) return fail(ctx, TOLS_ERR_ARG, "sizes must halve");
    keep_total += (size_t)h_sizes[j + 1];
  }
  orig_total = keep_total;
  const long long deep = h_sizes[levels];
  if (deep < P1) return fail(ctx, TOLS_ERR_ARG, "the deepest level needs at least p_bar + 1 rows");
  if (deep > (1LL << 30)) return fail(ctx, TOLS_ERR_ARG, "the deepest level may hold at most 2^30 rows");
  {
    // each level's kept positions: increasing, inside the level above
    size_t off = 0;
    for (int j = 0; j < levels; ++j) {
      for (long long e = 0; e < h_sizes[j + 1]; ++e) {
        const long long v = h_keep[off + e];
        if (v < 0 || v >= h_sizes[j] || (e > 0 && v <= h_keep[off + e - 1]))
          return fail(ctx, TOLS_ERR_ARG, "keep lists must be increasing positions inside their level");
      }
      off += (size_t)h_sizes[j + 1];
    }
  }
  cudaSetDevice(ctx->device);
  const long long nb = (m + kLsarBlock - 1) / kLsarBlock;
  const long long tri_max = lsar_tri(p_bar);
  const long long bmax = std::max<long long>(c, deep);
  const int ng = std::max(1, std::min(ctx->sms, (int)((bmax + 7) / 8)));
  const size_t p2 = (size_t)p_bar * p_bar;
  // doubles: scores of level 0 and of the current level, block sums and prefix, the weights of B and of a lag's
  // draws, Gram partials, G, the Cholesky factor (order p_bar + 1) and its reciprocal diagonal, refinement
  // partials, M, tau, phi per lag; then int64: the original rows of levels 1.., the kept positions, the drawn
  // positions, B's rows, a lag's rows; then the status word
  const size_t nd = (size_t)m + (size_t)h_sizes[1] + nb + (nb + 1) + bmax + c + ng * (size_t)tri_max + tri_max +
                    (size_t)P1 * P1 + P1 + ng * (size_t)p_bar + (size_t)k * P1 + p_bar + p2;
  const size_t ni = orig_total + keep_total + 2 * (size_t)c + (size_t)bmax;
  int rc;
  if ((rc = ensure(ctx, ctx->lsar, sizeof(double) * nd + sizeof(long long) * ni + 256))) return rc;
  double* q = (double*)ctx->lsar.p;
  double* scores0 = q; q += m;
  double* scoresj = q; q += h_sizes[1];
  double* bsum = q; q += nb;
  double* bpre = q; q += nb + 1;
  double* bw2 = q; q += bmax;
  double* w2 = q; q += c;
  double* part = q; q += ng * (size_t)tri_max;
  double* G = q; q += tri_max;
  double* Lg = q; q += (size_t)P1 * P1;
  double* rdg = q; q += P1;
  double* gpart = q; q += ng * (size_t)p_bar;
  double* M = q; q += (size_t)k * P1;
  double* tau_dev = q; q += p_bar;
  double* phi_all = q; q += p2;
  long long* orig = (long long*)q;
  long long* keep = orig + orig_total;
  long long* drawn = keep + keep_total;
  long long* brows = drawn + c;
  long long* rows_tmp = brows + bmax;
  int* status = (int*)(rows_tmp + c);
  CK(cudaMemsetAsync(phi_all, 0, sizeof(double) * p2, ctx->stream));
  CK(cudaMemsetAsync(status, 0, sizeof(int), ctx->stream));
  CK(cudaMemcpyAsync(keep, h_keep, sizeof(long long) * keep_total, cudaMemcpyHostToDevice, ctx->stream));
  // original rows of every level below the top: orig_{j+1} = orig_j[keep_j] (orig_0 the identity)
  std::vector<size_t> orig_off((size_t)levels + 1, 0);
  for (int j = 1; j <= levels; ++j) orig_off[j] = (j == 1 ? 0 : orig_off[j - 1] + (size_t)h_sizes[j - 1]);
  {
    size_t koff = 0;
    for (int j = 0; j < levels; ++j) {
      const long long* in = j == 0 ? nullptr : orig + orig_off[j];
      RUN(run_small(ctx, 12, [&] {
        return launch_rh_map(in, keep + koff, h_sizes[j + 1], orig + orig_off[j + 1], ctx->stream);
      }));
      koff += (size_t)h_sizes[j + 1];
    }
  }
  // the deepest level is its own spectral approximation: its rows, weight 1
  const long long* b_rows = orig + orig_off[levels];
  long long b_cnt = deep;
  RUN(run_small(ctx, 12, [&] { return launch_rh_fill(bw2, deep, 1.0, ctx->stream); }));
  // S_0 .. S_{levels-2} are k x c each; the deepest level's k x deep sketch S_{levels-1} comes last
  std::vector<size_t> sk_off((size_t)levels, 0);
  for (int j = 1; j < levels; ++j) sk_off[j] = (size_t)k * (size_t)c * (size_t)j;
  for (int j = levels - 1; j >= 0; --j) {
    const int gj = std::max(1, std::min(ctx->sms, (int)((b_cnt + 7) / 8)));
    const long long* list = j == 0 ? nullptr : orig + orig_off[j];
    double* sc = j == 0 ? scores0 : scoresj;
    RUN(run_small(ctx, 12, [&] {
      return launch_lsar_gram(d_y, p_bar, b_rows, bw2, (int)b_cnt, gj, part, G, status, ctx->stream);
    }));
    RUN(run_small(ctx, 12, [&] { return launch_rh_factor(G, P1, Lg, rdg, 10000 + j, status, ctx->stream); }));
    RUN(run_small(ctx, 12, [&] {
      return launch_rh_sketch(d_y, P1, b_rows, bw2, (int)b_cnt, d_sketch + sk_off[j], k, Lg, rdg, M, status,
                              ctx->stream);
    }));
    RUN(run_small(ctx, 12, [&] { return launch_rh_score(d_y, P1, M, k, list, h_sizes[j], sc, status, ctx->stream); }));
    if (j > 0) {
      // draw the c rows of this level's approximation (weights sum / (c score)), as original rows
      RUN(run_small(ctx, 12, [&] { return launch_lsar_lev(nullptr, nullptr, sc, h_sizes[j], bsum, status, ctx->stream); }));
      const long long nbj = (h_sizes[j] + kLsarBlock - 1) / kLsarBlock;
      RUN(run_small(ctx, 12, [&] { return launch_lsar_prefix(bsum, nbj, bpre, status, ctx->stream); }));
      RUN(run_small(ctx, 12, [&] {
        return launch_lsar_sample(sc, h_sizes[j], bsum, bpre, d_rh_unif + (size_t)j * c, c, 0, drawn, bw2, status,
                                  ctx->stream);
      }));
      RUN(run_small(ctx, 12, [&] { return launch_rh_map(list, drawn, c, brows, ctx->stream); }));
      b_rows = brows;
      b_cnt = c;
    }
  }
  if (d_scores) CK(cudaMemcpyAsync(d_scores, scores0, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice, ctx->stream));
  // the LSAR lags with the level-0 scores in place of eq. (FALS)
  RUN(run_small(ctx, 12, [&] { return launch_lsar_lev(nullptr, nullptr, scores0, m, bsum, status, ctx->stream); }));
  RUN(run_small(ctx, 12, [&] { return launch_lsar_prefix(bsum, nb, bpre, status, ctx->stream); }));
  const int ngl = std::max(1, std::min(ctx->sms, (c + 7) / 8));
  for (int p = 1; p <= p_bar; ++p) {
    long long* rows_p = d_rows ? d_rows + (size_t)(p - 1) * c : rows_tmp;
    RUN(run_small(ctx, 12, [&] {
      return launch_lsar_sample(scores0, m, bsum, bpre, d_unif + (size_t)(p - 1) * c, c, 0, rows_p, w2, status,
                                ctx->stream);
    }));
    RUN(run_small(ctx, 12, [&] { return launch_lsar_gram(d_y, p, rows_p, w2, c, ngl, part, G, status, ctx->stream); }));
    RUN(run_small(ctx, 12, [&] {
      return launch_lsar_solve(G, p, d_y, rows_p, w2, c, ngl, Lg, rdg, gpart, phi_all + (size_t)(p - 1) * p_bar,
                               tau_dev, p, status, ctx->stream);
    }));
  }
  int h_status = 0;
  CK(cudaMemcpyAsync(tau, tau_dev, sizeof(double) * p_bar, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  int o = 0;
  const double thr = 1.96 / sqrt((double)c);
  for (int p = 1; p <= p_bar; ++p)
    if (fabs(tau[p - 1]) >= thr) o = p;
  if (order) *order = o;
  if (phi) {
    if (o > 0) {
      CK(cudaMemcpyAsync(phi, phi_all + (size_t)(o - 1) * p_bar, sizeof(double) * p_bar, cudaMemcpyDeviceToHost,
                         ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    } else {
      for (int j = 0; j < p_bar; ++j) phi[j] = 0.0;
    }
  }
  if (h_status) {
    char msg[112];
    if (h_status >= 10000)
      snprintf(msg, sizeof msg, "Repeated Halving: B^T B not positive definite at level %d", h_status - 10000);
    else
      snprintf(msg, sizeof msg, "sampled Gram matrix not positive definite at lag %d", h_status);
    ctx->err = msg;
    return TOLS_NOT_CONVERGED;
  }
  return TOLS_OK;
}

int toeplitz_ols_srht(tols_ctx* ctx, const double* d_y, long long n, int p, int c, const double* d_signs,
                      const long long* d_rows, double* d_phi) {
  if (!ctx) return TOLS_ERR_ARG;
  if (!d_y || !d_signs || !d_rows || !d_phi) return fail(ctx, TOLS_ERR_ARG, "null pointer");
  if (p < 1 || p > kLsarMaxP) return fail(ctx, TOLS_ERR_ARG, "p out of range [1, 256]");
  if (n <= p) return fail(ctx, TOLS_ERR_ARG, "need n > p");
  if (c < p) return fail(ctx, TOLS_ERR_ARG, "need c >= p");
  cudaSetDevice(ctx->device);
  const long long m = n - p;
  long long m2 = 1;
  while (m2 < m) m2 <<= 1;
  const long long tri = lsar_tri(p);
  const int ng = std::max(1, std::min(ctx->sms, (c + 7) / 8));
  const size_t nd = (size_t)(p + 1) * m2 + ng * (size_t)tri + tri + (size_t)p * p + p;
  int rc;
  if ((rc = ensure(ctx, ctx->lsar, sizeof(double) * nd + 256))) return rc;
  double* q = (double*)ctx->lsar.p;
  double* Z = q; q += (size_t)(p + 1) * m2;
  double* part = q; q += ng * (size_t)tri;
  double* G = q; q += tri;
  double* Lg = q; q += (size_t)p * p;
  double* rdg = q; q += p;
  int* status = (int*)q;
  CK(cudaMemsetAsync(status, 0, sizeof(int), ctx->stream));
  RUN(run_small(ctx, 12, [&] { return launch_srht_transform(d_y, p, m, m2, d_signs, Z, ctx->stream); }));
  const double sc = sqrt((double)m2 / (double)c);
  RUN(run_small(ctx, 12, [&] { return launch_srht_gram(Z, m2, p, d_rows, c, sc, ng, part, G, status, ctx->stream); }));
  RUN(run_small(ctx, 12, [&] { return launch_srht_solve(G, p, Lg, rdg, d_phi, status, ctx->stream); }));
  int h_status = 0;
  CK(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h_status < 0) return fail(ctx, TOLS_ERR_ARG, "a sampled row index is outside [0, m2)");
  if (h_status > 0) {
    ctx->err = "the sampled, transformed Gram matrix is not positive definite";
    return TOLS_NOT_CONVERGED;
  }
  return TOLS_OK;
}

int toeplitz_ols_solve_batched_device(tols_ctx* ctx, int count, const double* const* d_y, const long long* n,
                                      const int* p, double tol, double* d_phi, double* rnorm, tols_info* info) {
  if (!ctx || count < 0 || (count > 0 && (!d_y || !n || !p || !d_phi))) return TOLS_ERR_ARG;
  if (count == 0) return TOLS_OK;
  cudaSetDevice(ctx->device);
  if (tol <= 0) tol = 1e-12;
  std::vector<int> status(count, TOLS_OK);
  BatchPlan B;
  plan_batch(ctx, B, count, n, p, status, ctx->cfg.precision == TOLS_MIXED);
  for (int k : B.idx) {
    if (!d_y[k]) return fail(ctx, TOLS_ERR_ARG, "null device series pointer");
    B.y_dev.push_back(d_y[k]);
  }
  const bool mixed = ctx->cfg.precision == TOLS_MIXED;
  std::vector<DevState> states;
  std::vector<int> prec_used;
  std::vector<double> phis;
  int rc;
  if ((rc = batch_solve_all(ctx, B, tol, mixed, states, phis, prec_used))) return rc;
  // output: phi of series k at d_phi + sum_{j<k} p[j]
  std::vector<size_t> out_off(count + 1, 0);
  for (int k = 0; k < count; ++k) out_off[k + 1] = out_off[k] + (size_t)std::max(p[k], 0);
  std::vector<double> outv(out_off[count], 0.0);
  for (size_t j = 0; j < B.idx.size(); ++j)
    memcpy(outv.data() + out_off[B.idx[j]], phis.data() + B.off_phi[j], sizeof(double) * B.p[j]);
  CK(cudaMemcpyAsync(d_phi, outv.data(), sizeof(double) * outv.size(), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  int worst = TOLS_OK;
  for (int k = 0; k < count; ++k) {
    if (info) memset(&info[k], 0, sizeof(tols_info));
    if (rnorm) rnorm[k] = 0.0;
  }
  for (size_t j = 0; j < B.idx.size(); ++j) {
    const int k = B.idx[j];
    status[k] = states[j].status;
    if (rnorm) rnorm[k] = states[j].rnorm;
    if (info) fill_info(&info[k], states[j], prec_used[j]);
  }
  for (int k = 0; k < count; ++k) {
    if (info) info[k].status = status[k];
    if (status[k] < 0) worst = worst < 0 ? std::min(worst, status[k]) : status[k];
    else if (worst >= 0) worst = std::max(worst, status[k]);
  }
  return worst;
}

int toeplitz_ols_stream_open(tols_ctx* ctx, int p, double tol, int* handle) {
  if (!ctx || !handle || p < 1 || p > TOLS_MAX_P) return TOLS_ERR_ARG;
  StreamSeries s;
  s.p = p;
  s.tol = tol;
  *handle = ctx->next_handle++;
  ctx->streams[*handle] = s;
  return TOLS_OK;
}

int toeplitz_ols_stream_push(tols_ctx* ctx, int handle, const double* y_chunk, long long len) {
  if (!ctx || len < 0 || (len > 0 && !y_chunk)) return TOLS_ERR_ARG;
  auto it = ctx->streams.find(handle);
  if (it == ctx->streams.end()) return TOLS_ERR_ARG;
  it->second.y.insert(it->second.y.end(), y_chunk, y_chunk + len);
  return TOLS_OK;
}

int toeplitz_ols_stream_solve(tols_ctx* ctx, int handle, double* phi, double* rnorm, tols_info* info) {
  if (!ctx || !phi) return TOLS_ERR_ARG;
  auto it = ctx->streams.find(handle);
  if (it == ctx->streams.end()) return TOLS_ERR_ARG;
  StreamSeries& s = it->second;
  int rc = validate(ctx, (long long)s.y.size(), s.p);
  if (rc) return rc;
  cudaSetDevice(ctx->device);
  rc = host_solve(ctx, s.y.data(), (long long)s.y.size(), s.p, s.tol, phi, rnorm, info,
                  s.phi.empty() ? nullptr : s.phi.data());
  if (rc >= 0) s.phi.assign(phi, phi + s.p);
  if (info && rc < 0) info->status = rc;
  return rc;
}

int toeplitz_ols_stream_close(tols_ctx* ctx, int handle) {
  if (!ctx) return TOLS_ERR_ARG;
  return ctx->streams.erase(handle) ? TOLS_OK : TOLS_ERR_ARG;
}

// ---- step entry points ----------------------------------------------------------------------------
int toeplitz_ols_gk_pass(tols_ctx* ctx, int precision, const void* d_y, long long n, int p, const double* d_v,
                         const void* d_u_old, double c, void* d_u_new, double* d_xtu, double* unorm2) {
  int rc = validate(ctx, n, p);
  if (rc) return rc;
  if (!d_y || !d_v || !d_xtu || (precision != TOLS_FP64 && precision != TOLS_MIXED))
    return fail(ctx, TOLS_ERR_ARG, "bad argument");
  cudaSetDevice(ctx->device);
  Work w;
  if ((rc = prepare_work(ctx, nullptr, n, p, false, false, w))) return rc;
  if ((rc = ensure(ctx, ctx->scratch, sizeof(double) * (2 * (size_t)p + 64)))) return rc;
  double* d_n2 = (double*)ctx->scratch.p;
  const int pp = pad_p(p);
  CK(cudaMemsetAsync(&w.st->dev_error, 0, sizeof(int), ctx->stream));
  if (precision == TOLS_FP64) {
    PassArgs<double> a = base_args<double>(w, (const double*)d_y, n, p, pp);
    a.d = d_v;
    a.u_old = (const double*)d_u_old;
    a.coef_host = c;
    a.u_new = (double*)d_u_new;
    a.tail = TAIL_STORE;
    a.out_t = d_xtu;
    a.out_n2 = d_n2;
    a.fft = choose_fft<double>(ctx, w, (const double*)d_y, n, p, pp, p, 0);
    if (a.fft) {
      RUN(fft_spectra(ctx, w, 1, d_y, n, n - p, pp, true, a.fft));
      a.w.wspec64 = w.wspec64;
    }
    RUN(run_pass<double>(ctx, a, pass_grid_for(ctx, 1, pp, a.fft)));
  } else {
    PassArgs<float> a = base_args<float>(w, (const float*)d_y, n, p, pp);
    a.d = d_v;
    a.u_old = (const float*)d_u_old;
    a.coef_host = c;
    a.u_new = (float*)d_u_new;
    a.tail = TAIL_STORE;
    a.out_t = d_xtu;
    a.out_n2 = d_n2;
    a.fft = choose_fft<float>(ctx, w, (const float*)d_y, n, p, pp, p, 0);
    if (a.fft) {
      RUN(fft_spectra(ctx, w, 0, d_y, n, n - p, pp, true));
      a.w.wspec32 = w.wspec32;
      a.w.sacc32 = w.sacc32;
    }
    RUN(run_pass<float>(ctx, a, pass_grid_for(ctx, 0, pp, a.fft)));
  }
  double h = 0.0;
  int derr = 0;
  CK(cudaMemcpyAsync(&h, d_n2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&derr, &w.st->dev_error, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (derr) return fail(ctx, TOLS_ERR_DEVICE_TIMEOUT, "a kernel's wait on its bulk copies gave up");
  if (unorm2) *unorm2 = h;
  return TOLS_OK;
}

int toeplitz_ols_gram(tols_ctx* ctx, int precision, const double* d_y, long long n, int p, double* d_G, double* d_h,
                      double* bnorm2) {
  int rc = validate(ctx, n, p);
  if (rc) return rc;
  if (!d_y || !d_G || !d_h || (precision != TOLS_FP64 && precision != TOLS_MIXED))
    return fail(ctx, TOLS_ERR_ARG, "bad argument");
  cudaSetDevice(ctx->device);
  const bool mixed = precision == TOLS_MIXED;
  Work w;
  if ((rc = prepare_work(ctx, d_y, n, p, mixed, false, w))) return rc;
  w.G = d_G;
  w.h = d_h;
  const int pg = pad_p(p + 1);
  if (mixed) {
    RUN(run_small(ctx, 11, [&] { return launch_convert_f32(d_y, w.y32, n, ctx->stream); }));
    PassArgs<float> a = base_args<float>(w, w.y32, n, p, pg);
    a.gram = 1;
    a.nlag = p + 1;
    a.tail = TAIL_GRAM;
    a.out_n2 = w.bnorm2;
    a.fft = choose_fft<float>(ctx, w, w.y32, n, p, pg, p + 1, 1);
    if (a.fft) {
      RUN(fft_spectra(ctx, w, 0, w.y32, n, n - p, pg, false));
      a.w.wspec32 = w.wspec32;
    }
    RUN(run_pass<float>(ctx, a, pass_grid_for(ctx, 0, pg, a.fft)));
  } else {
    PassArgs<double> a = base_args<double>(w, d_y, n, p, pg);
    a.gram = 1;
    a.nlag = p + 1;
    a.tail = TAIL_GRAM;
    a.out_n2 = w.bnorm2;
    a.fft = choose_fft<double>(ctx, w, d_y, n, p, pg, p + 1, 1);
    if (a.fft) {
      RUN(fft_spectra(ctx, w, 1, d_y, n, n - p, pg, false, a.fft));
      a.w.wspec64 = w.wspec64;
    }
    RUN(run_pass<double>(ctx, a, pass_grid_for(ctx, 1, pg, a.fft)));
  }
  double h = 0.0;
  CK(cudaMemcpyAsync(&h, w.bnorm2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (bnorm2) *bnorm2 = h;
  return TOLS_OK;
}

int toeplitz_ols_preconditioner(tols_ctx* ctx, int precision, const double* d_y, long long n, int p, int kind,
                                double* d_M, tols_info* info) {
  int rc = validate(ctx, n, p);
  if (rc) return rc;
  if (!d_y || !d_M || (precision != TOLS_FP64 && precision != TOLS_MIXED) ||
      (kind != TOLS_PRECOND_GRAM_CHOL && kind != TOLS_PRECOND_SAMPLED_QR))
    return fail(ctx, TOLS_ERR_ARG, "bad argument");
  cudaSetDevice(ctx->device);
  const bool mixed = precision == TOLS_MIXED;
  Work w;
  if ((rc = prepare_work(ctx, d_y, n, p, mixed, false, w))) return rc;
  DevState hs;
  memset(&hs, 0, sizeof hs);
  hs.mixed = mixed ? 1 : 0;
  *ctx->h_state = hs;
  CK(cudaMemcpyAsync(w.st, ctx->h_state, sizeof(DevState), cudaMemcpyHostToDevice, ctx->stream));
  const int pg = pad_p(p + 1);
  const int fft = choose_fft<double>(ctx, w, d_y, n, p, pg, p + 1, 1);
  if (fft) RUN(fft_spectra(ctx, w, 1, nullptr, n, n - p, pg, false, fft));
  RUN(run_setup(ctx, w, mixed, false, fft, kind));
  CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const DevState& s = *ctx->h_state;
  if (s.status == TOLS_ERR_NONFINITE) return fail(ctx, TOLS_ERR_NONFINITE, "y holds NaN or Inf");
  if (s.precond) CK(cudaMemcpyAsync(d_M, w.M, sizeof(double) * (size_t)p * p, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (info) {
    memset(info, 0, sizeof *info);
    fill_info(info, s, mixed ? TOLS_MIXED : TOLS_FP64);
    info->status = s.precond ? TOLS_OK : TOLS_NOT_CONVERGED;
    info->cond_est = s.kappa_est;
  }
  return s.precond ? TOLS_OK : TOLS_NOT_CONVERGED;
}

int toeplitz_ols_row_norms(tols_ctx* ctx, const double* d_y, long long n, int p, double* d_rn2, double* fro2) {
  int rc = validate(ctx, n, p);
  if (rc) return rc;
  if (!d_y) return fail(ctx, TOLS_ERR_ARG, "null pointer");
  cudaSetDevice(ctx->device);
  const long long m = n - p;
  const size_t blocks = (size_t)((m + 2047) / 2048);
  if ((rc = ensure(ctx, ctx->scratch, sizeof(double) * (blocks + 64)))) return rc;
  double* s = (double*)ctx->scratch.p;
  RUN(run_small(ctx, 12, [&] { return launch_row_norms(d_y, n, p, d_rn2, s, s + 8, ctx->stream); }));
  double h = 0.0;
  CK(cudaMemcpyAsync(&h, s, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (fro2) *fro2 = h;
  return TOLS_OK;
}

int toeplitz_ols_residual(tols_ctx* ctx, const double* d_y, long long n, int p, const double* d_phi, double* d_g,
                          double* rnorm) {
  int rc = validate(ctx, n, p);
  if (rc) return rc;
  if (!d_y || !d_phi || !d_g) return fail(ctx, TOLS_ERR_ARG, "null pointer");
  cudaSetDevice(ctx->device);
  Work w;
  if ((rc = prepare_work(ctx, d_y, n, p, false, false, w))) return rc;
  if ((rc = ensure(ctx, ctx->scratch, sizeof(double) * 64))) return rc;
  double* d_n2 = (double*)ctx->scratch.p;
  const int pp = pad_p(p);
  PassArgs<double> a = base_args<double>(w, d_y, n, p, pp);
  a.d = d_phi;
  a.d_scale = -1.0;     // u = -X phi - (-1) b = b - X phi
  a.u_old = d_y + p;
  a.coef_host = -1.0;
  a.tail = TAIL_STORE;
  a.out_t = d_g;
  a.out_n2 = d_n2;
  a.fft = choose_fft<double>(ctx, w, d_y, n, p, pp, p, 0);
  if (a.fft) {
    RUN(fft_spectra(ctx, w, 1, d_y, n, n - p, pp, true, a.fft));
    a.w.wspec64 = w.wspec64;
  }
  RUN(run_pass<double>(ctx, a, pass_grid_for(ctx, 1, pp, a.fft)));
  double h = 0.0;
  CK(cudaMemcpyAsync(&h, d_n2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (rnorm) *rnorm = sqrt(h);
  return TOLS_OK;
}

int toeplitz_ols_leverage_p1(tols_ctx* ctx, const double* d_y, long long n, double* d_lev) {
  if (!ctx) return TOLS_ERR_ARG;
  if (!d_y || !d_lev || n < 2) return fail(ctx, TOLS_ERR_ARG, "bad argument");
  cudaSetDevice(ctx->device);
  const size_t blocks = (size_t)((n - 1 + 4095) / 4096);
  int rc = ensure(ctx, ctx->scratch, sizeof(double) * (blocks + 64));
  if (rc) return rc;
  RUN(run_small(ctx, 12, [&] { return launch_leverage_p1(d_y, n, d_lev, (double*)ctx->scratch.p, ctx->stream); }));
  CK(cudaStreamSynchronize(ctx->stream));
  return TOLS_OK;
}

int toeplitz_ols_leverage_step(tols_ctx* ctx, const double* d_y, long long n, int p, const double* d_phi_hat,
                               const double* d_lev_prev, double* d_lev, double* d_pi, double* rnorm2) {
  int rc = validate(ctx, n, p);
  if (rc) return rc;
  if (p < 2 || !d_y || !d_phi_hat || !d_lev_prev || !d_lev) return fail(ctx, TOLS_ERR_ARG, "bad argument");
  cudaSetDevice(ctx->device);
  const long long m = n - p;
  // the order-(p-1) problem on y[0..n-2]: X' phi_hat - b' with b' = y + (p-1)
  Work w;
  if ((rc = prepare_work(ctx, d_y, n - 1, p - 1, false, false, w))) return rc;
  if ((rc = ensure(ctx, ctx->rbuf, sizeof(double) * (size_t)m))) return rc;
  if ((rc = ensure(ctx, ctx->scratch, sizeof(double) * 64))) return rc;
  double* d_rr = (double*)ctx->scratch.p;
  const int pp = pad_p(p - 1);
  PassArgs<double> a = base_args<double>(w, d_y, n - 1, p - 1, pp);
  a.d = d_phi_hat;
  a.u_old = d_y + (p - 1);
  a.coef_host = 1.0;
  a.u_new = (double*)ctx->rbuf.p;
  a.nlag = 0;
  a.tail = TAIL_STORE;
  a.out_t = nullptr;
  a.out_n2 = d_rr;
  RUN(run_pass<double>(ctx, a, pass_grid_for(ctx, 1, pp)));
  RUN(run_small(ctx, 12, [&] {
    return launch_leverage_step((const double*)ctx->rbuf.p, m, p, d_rr, d_lev_prev, d_lev, d_pi, nullptr, ctx->stream);
  }));
  double h = 0.0;
  CK(cudaMemcpyAsync(&h, d_rr, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (rnorm2) *rnorm2 = h;
  return TOLS_OK;
}


void toeplitz_ols_server_config_default(tols_server_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof *cfg);
  cfg->precision = TOLS_MIXED;
  cfg->device = 0;
  cfg->max_active = 1024;
  cfg->burst = 4;
}

int toeplitz_ols_server_create(tols_server** out, const tols_server_config* cfg) {
  if (!out) return TOLS_ERR_ARG;
  *out = nullptr;
  tols_server_config c;
  if (cfg) c = *cfg;
  else toeplitz_ols_server_config_default(&c);
  if (c.precision != TOLS_FP64 && c.precision != TOLS_MIXED) return TOLS_ERR_ARG;
  tols_config cc;
  toeplitz_ols_config_default(&cc);
  cc.precision = c.precision;
  cc.device = c.device;
  cc.max_iter = c.max_iter;
  cc.max_sweeps = c.max_sweeps;
  cc.cuda_stream = c.cuda_stream;
  tols_ctx* ctx = nullptr;
  int rc = toeplitz_ols_create(&ctx, &cc);
  if (rc) return rc;
  tols_server* srv = new tols_server;
  srv->ctx = ctx;
  srv->mixed = c.precision == TOLS_MIXED;
  srv->max_active = c.max_active > 0 ? c.max_active : 1024;
  srv->burst = c.burst > 0 ? c.burst : 4;
  size_t cap = c.arena_bytes;
  if (cap == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    cap = fr / 2;
  }
  if (cudaMalloc(&srv->arena, cap) != cudaSuccess) {
    cudaGetLastError();
    toeplitz_ols_destroy(ctx);
    delete srv;
    return TOLS_ERR_OOM;
  }
  srv->arena_cap = cap;
  srv->alloc.reset(cap);
  srv->t0 = std::chrono::steady_clock::now();
  *out = srv;
  return TOLS_OK;
}

int toeplitz_ols_server_destroy(tols_server* srv) {
  if (!srv) return TOLS_OK;
  tols_ctx* ctx = srv->ctx;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  release(ctx, srv->table);
  release(ctx, srv->tiles);
  release(ctx, srv->gather);
  if (srv->arena) cudaFree(srv->arena);
  toeplitz_ols_destroy(ctx);
  delete srv;
  return TOLS_OK;
}

int toeplitz_ols_server_submit(tols_server* srv, long long id, const double* y, long long n, int p, double tol) {
  if (!srv || !y || p < 1 || p > TOLS_MAX_P || n <= p) return TOLS_ERR_ARG;
  // a mixed request may be re-run in float64, which needs the larger footprint
  if (align_up(series_slice(nullptr, n, p, false, batch_fft_choice(srv->ctx, p) != 0, nullptr), 256) >
      srv->arena_cap)
    return TOLS_ERR_OOM;
  SrvRequest r;
  r.id = id;
  r.n = n;
  r.p = p;
  r.tol = tol > 0 ? tol : 1e-12;
  r.y.assign(y, y + n);
  r.t_submit = now_s(srv->t0);
  r.mixed = srv->mixed;
  srv->queue.push_back(std::move(r));
  srv->submitted++;
  return TOLS_OK;
}

int toeplitz_ols_server_step(tols_server* srv, int* active, int* queued) {
  if (!srv) return TOLS_ERR_ARG;
  tols_ctx* ctx = srv->ctx;
  cudaSetDevice(ctx->device);
  std::vector<int> fresh;
  int rc = server_admit(srv, fresh);
  if (rc) return rc;
  if ((rc = server_round(srv))) return rc;
  if (active) *active = (int)srv->active.size();
  if (queued) *queued = (int)srv->queue.size();
  return TOLS_OK;
}

int toeplitz_ols_server_poll(tols_server* srv, tols_result* out, double* phi_out, int max, int* got) {
  if (!srv || !got || max < 0 || (max > 0 && !out)) return TOLS_ERR_ARG;
  const int k = std::min<int>(max, (int)srv->results.size());
  for (int i = 0; i < k; ++i) {
    out[i] = srv->results[i];
    if (phi_out) memcpy(phi_out + (size_t)i * TOLS_MAX_P, srv->result_phi.data() + (size_t)i * TOLS_MAX_P,
                        sizeof(double) * TOLS_MAX_P);
  }
  srv->results.erase(srv->results.begin(), srv->results.begin() + k);
  srv->result_phi.erase(srv->result_phi.begin(), srv->result_phi.begin() + (size_t)k * TOLS_MAX_P);
  *got = k;
  return TOLS_OK;
}

int toeplitz_ols_server_stats(tols_server* srv, tols_server_stats* st) {
  if (!srv || !st) return TOLS_ERR_ARG;
  st->submitted = srv->submitted;
  st->completed = srv->completed;
  st->active = (int)srv->active.size();
  st->queued = (int)srv->queue.size();
  st->arena_bytes = srv->arena_cap;
  st->arena_used = srv->alloc.used();
  return TOLS_OK;
}

int toeplitz_ols_profile(tols_ctx* ctx, int enable) {
  if (!ctx) return TOLS_ERR_ARG;
  cudaSetDevice(ctx->device);
  int rc = flush_profile(ctx);
  if (rc) return rc;
  if (enable) {
    ctx->launch_total = 0;
    for (int k = 0; k < TOLS_PROFILE_CLASSES; ++k) { ctx->prof_launches[k] = 0; ctx->prof_ms[k] = 0.0; }
  }
  ctx->prof = enable != 0;
  return TOLS_OK;
}

int toeplitz_ols_profile_read(tols_ctx* ctx, int kind, long long* launches, double* total_ms) {
  if (!ctx || kind < -1 || kind >= TOLS_PROFILE_CLASSES) return TOLS_ERR_ARG;
  cudaSetDevice(ctx->device);
  int rc = flush_profile(ctx);
  if (rc) return rc;
  if (kind == -1) {
    if (launches) *launches = ctx->launch_total;
    if (total_ms) *total_ms = 0.0;
  } else {
    if (launches) *launches = ctx->prof_launches[kind];
    if (total_ms) *total_ms = ctx->prof_ms[kind];
  }
  return TOLS_OK;
}

}  // extern "C"
