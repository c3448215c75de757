// Overlap-save FFT product pass (included by tols_kernels.cu: it shares the arrival and tail code).
//
// The same outputs as pass_kernel — u_new = X d - c u_old, ||u_new||^2, X^T u_new (or the Gram lag sums) — with
// the two structured products of eq. (xphi) done as circular correlations of length N per tile of L = N - p_pad
// rows, which never wrap inside the rows and lags used:
//   (X d)[i0 + r] = sum_{k<p} w[r + k] dr[k]          = IDFT(W . conj(DR))[r],   r < L
//   tk[k]         = sum_{r<L} u[r] w[r + k]             = IDFT(W . conj(U))[k],    k < nlag
// with w the window y[i0 .. i0+N) (zero past the end of y), dr the lag-reversed d, u the tile's fresh u (zero
// beyond its rows). The window spectra W of all tiles are formed once per solve (by the Gram pass, or by
// spectrum_kernel) and read from global memory. Per tile a pass runs one inverse transform (X d) and one forward
// transform (u). The X^T u products are linear in the spectra, so each CTA sums W . conj(U) over its tiles and
// transforms back once, at its end; the spectrum of dr is formed once per CTA and launch.
//
// A real N-point FFT is an N/2-point complex FFT of the packed pairs (w[2j], w[2j+1]) plus an O(N) split; the
// complex FFT is a radix-8 (then 4, 2) Stockham autosort in shared memory, one butterfly per thread per stage.
// Twiddles come from a table of exp(-2 pi i t / N), t < N, computed on the host in float64. Half spectra are
// kept doubled (2W, 2U, 2D): the split and merge then need no halving, and every product of two of them and its
// merge carry a factor 8, removed with the 1 / (8 M) scale of the inverse transform (all powers of two: exact).
#pragma once

// Index into the FFT work arrays: one pad element after every 8, so that the strided writes of the first
// Stockham stages (stride 8 complex values) land in distinct shared-memory banks.
__device__ __forceinline__ int pix(int i) { return i + (i >> 3); }

template <typename T>
struct FftCfg;
// N: real FFT length per tile. WS: entries per tile of the window-spectrum array (bins 0 .. N/2; the float
// tiles are padded to N/2 + 2 entries so that every tile starts on a 16-byte boundary, as bulk copies require).
template <>
struct FftCfg<float> {
  static constexpr int N = 4096;
  static constexpr int WS = N / 2 + 2;
  using V = float2;
};
template <>
struct FftCfg<double> {
  static constexpr int N = 2048;
  static constexpr int WS = N / 2 + 1;
  using V = double2;
};

template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// a * conj(b)
template <typename V>
__device__ __forceinline__ V cmulc(V a, V b) {
  V r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
// float2 sums and differences as packed two-lane instructions (sm_100 and later: one issue slot instead of two;
// per component the same rounding as a scalar add). a - b is fma(b, -1, a), exact before its one rounding.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
template <typename V>
__device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
template <typename V, typename S>
__device__ __forceinline__ V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }
// multiply by -i (forward) or +i (inverse)
template <typename V>
__device__ __forceinline__ V cmul_mi(V a, bool inv) {
  V r;
  if (inv) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// In-register DFT of R points, forward (exp(-2 pi i qr / R)) or inverse (exp(+...)), unnormalised.
template <typename V, typename S, int R>
__device__ __forceinline__ void dft_small(V* v, bool inv);
template <typename V, typename S>
__device__ __forceinline__ void dft2(V& a, V& b) {
  const V t = a;
  a = cadd(t, b);
  b = csub(t, b);
}
template <typename V, typename S, int R>
__device__ __forceinline__ void dft_small(V* v, bool inv) {
  if (R == 2) {
    dft2<V, S>(v[0], v[1]);
  } else if (R == 4) {
    V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    V t2 = cadd(v[1], v[3]), t3 = cmul_mi(csub(v[1], v[3]), inv);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  } else {  // R == 8: two 4-point DFTs of the even and odd points, then the radix-2 combination
    V e[4] = {v[0], v[2], v[4], v[6]};
    V o[4] = {v[1], v[3], v[5], v[7]};
    dft_small<V, S, 4>(e, inv);
    dft_small<V, S, 4>(o, inv);
    const S h = (S)0.70710678118654752440;  // 1/sqrt(2)
    // w8^q, q = 0..3, w8 = exp(-+ i pi / 4)
    V o1, o2, o3;
    o1.x = h * (o[1].x + (inv ? -o[1].y : o[1].y));
    o1.y = h * (o[1].y + (inv ? o[1].x : -o[1].x));
    o2 = cmul_mi(o[2], inv);
    o3.x = h * (-o[3].x + (inv ? -o[3].y : o[3].y));
    o3.y = h * (-o[3].y + (inv ? o[3].x : -o[3].x));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
}

// One Stockham radix-R stage over M points (in -> out): sub-transforms of length Ls grow to Ls * R.
// tw: exp(-2 pi i t / (2M)), t < 2M; omega_M^s = tw[2s]. The first stage (Ls = 1) has only unit twiddles.
template <typename V, typename S, int R, int M, int Ls>
__device__ __forceinline__ void fft_stage(const V* __restrict__ in, V* __restrict__ out,
                                          const V* __restrict__ tw, bool inv) {
  constexpr int stride = M / R;
  constexpr int Ln = Ls * R;
  constexpr int tstep = 2 * (M / Ln);
  for (int j = threadIdx.x; j < stride; j += kThreads) {
    const int k = j & (Ls - 1);
    const int g = j / Ls;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[pix(j + r * stride)];
    if (Ls > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        V t = tw[r * k * tstep];
        if (inv) t.y = -t.y;
        v[r] = cmul(v[r], t);
      }
    }
    dft_small<V, S, R>(v, inv);
#pragma unroll
    for (int q = 0; q < R; ++q) out[pix(g * Ln + k + q * Ls)] = v[q];
  }
  __syncthreads();
}

// Complex FFT of M points in a (b is scratch); the result ends in a (every plan here has an even stage count).
template <typename V, typename S, int M>
__device__ void fft_complex(V* a, V* b, const V* tw, bool inv) {
  static_assert(M == 2048 || M == 1024, "plans for M = 2048 (8,8,8,4) and M = 1024 (8,8,8,2)");
  fft_stage<V, S, 8, M, 1>(a, b, tw, inv);
  fft_stage<V, S, 8, M, 8>(b, a, tw, inv);
  fft_stage<V, S, 8, M, 64>(a, b, tw, inv);
  if (M == 2048) fft_stage<V, S, 4, M, 512>(b, a, tw, inv);
  else fft_stage<V, S, 2, M, 512>(b, a, tw, inv);
}

// Split of the packed complex transform Z of a real sequence into its doubled half spectrum, two bins at a time:
//   a = Z[f] + conj(Z[M-f]),  b = Z[f] - conj(Z[M-f]),  s = -i w^f b   (w = exp(-2 pi i / N), Z[M] = Z[0])
//   2X[f] = a + s,   2X[M-f] = conj(a - s).
template <typename V, typename S>
__device__ __forceinline__ void split2(V zf, V zmf, V twf, V& xf, V& xmf) {
  const S ax = zf.x + zmf.x, ay = zf.y - zmf.y;
  const S bx = zf.x - zmf.x, by = zf.y + zmf.y;
  const S tbx = twf.x * bx - twf.y * by;   // w^f b
  const S tby = twf.x * by + twf.y * bx;
  xf.x = ax + tby;                         // s = tby - i tbx
  xf.y = ay - tbx;
  xmf.x = ax - tby;
  xmf.y = -(ay + tbx);
}
// Inverse: from a doubled Hermitian half spectrum V (bins f and M-f) to the doubled packed input of an inverse
// M-point FFT:  a = V[f] + conj(V[M-f]),  b = V[f] - conj(V[M-f]),  q = i conj(w^f) b;
//   2Z[f] = a + q,   2Z[M-f] = conj(a - q).
template <typename V, typename S>
__device__ __forceinline__ void merge2(V vf, V vmf, V twf, V& zf, V& zmf) {
  const S ax = vf.x + vmf.x, ay = vf.y - vmf.y;
  const S bx = vf.x - vmf.x, by = vf.y + vmf.y;
  const S cbx = twf.x * bx + twf.y * by;   // conj(w^f) b
  const S cby = twf.x * by - twf.y * bx;
  zf.x = ax - cby;                         // q = -cby + i cbx
  zf.y = ay + cbx;
  zmf.x = ax + cby;
  zmf.y = -(ay - cbx);
}

template <typename T, int N = FftCfg<T>::N>
struct FftCfg2 {
  static constexpr int M = N / 2;
  static constexpr int PADDED = M + M / 8 + 8;   // entries of a padded work array (index pix(f), f <= M)
  // entries per tile of the window-spectrum array: bins 0 .. M, float tiles padded to a 16-byte multiple
  static constexpr int WS = sizeof(T) == 4 ? M + 2 : M + 1;
};

__host__ __device__ constexpr size_t round16(size_t b) { return (b + 15) & ~(size_t)15; }

// Gram pass: below this many multiply-adds per tile (p_pad x nlag) the lag sums come from |W|^2 plus direct
// corrections (one transform per tile); above it from W . conj(B) with B the tile's row block (two transforms).
template <typename T>
struct GramCfg {
  static constexpr long long kDirectMax = sizeof(T) == 8 ? 24576 : 65536;
};

// Shared memory of the FFT kernels: work arrays A, B (padded), the doubled spectrum D of the lag-reversed d,
// the CTA's accumulated spectrum S (float64), the Gram pass's window segments ext[2 p_pad], tacc, scratch.
template <typename T, int N = FftCfg<T>::N>
struct FftSmem {
  using V = typename FftCfg<T>::V;
  static constexpr int M = N / 2;
  static constexpr int PADDED = FftCfg2<T, N>::PADDED;
  V *A, *B, *D;
  double2* S;
  T* ext;
  double *tacc, *scratch;
  __host__ __device__ static size_t bytes(int p_pad) {
    return round16(sizeof(V) * (2 * (size_t)PADDED + (M + 1))) + sizeof(double2) * (M + 1) +
           round16(sizeof(T) * 2 * (size_t)p_pad) + sizeof(double) * ((size_t)p_pad + 16 + 16);
  }
  __device__ FftSmem(unsigned char* raw, int p_pad) {
    A = reinterpret_cast<V*>(raw);
    B = A + PADDED;
    D = B + PADDED;
    unsigned char* q = raw + round16(sizeof(V) * (2 * (size_t)PADDED + (M + 1)));
    S = reinterpret_cast<double2*>(q);
    q += sizeof(double2) * (M + 1);
    ext = reinterpret_cast<T*>(q);
    q += round16(sizeof(T) * 2 * (size_t)p_pad);
    tacc = reinterpret_cast<double*>(q);
    scratch = tacc + p_pad + 16;
  }
};

// Window y[i0 .. i0+N) (zero past n), packed in pairs, into sm.A; then its complex transform (result in sm.A).
template <typename T, int N = FftCfg<T>::N>
__device__ void fft_window(FftSmem<T, N>& sm, const T* __restrict__ y, long long n, long long i0,
                           const typename FftCfg<T>::V* tw) {
  using V = typename FftCfg<T>::V;
  constexpr int M = N / 2;
  for (int j = threadIdx.x; j < M; j += kThreads) {
    const long long g0 = i0 + 2 * j;
    V v;
    v.x = g0 < n ? y[g0] : (T)0;
    v.y = g0 + 1 < n ? y[g0 + 1] : (T)0;
    sm.A[pix(j)] = v;
  }
  __syncthreads();
  fft_complex<V, T, M>(sm.A, sm.B, tw, false);
}

// Doubled spectrum of the lag-reversed, scaled d, into sm.D.
template <typename T, int N = FftCfg<T>::N>
__device__ void fft_d_spectrum(FftSmem<T, N>& sm, const double* d, double d_scale, int p, const typename FftCfg<T>::V* tw) {
  using V = typename FftCfg<T>::V;
  constexpr int M = N / 2;
  for (int j = threadIdx.x; j < M; j += kThreads) {
    const int k0 = 2 * j, k1 = 2 * j + 1;
    V v;
    v.x = k0 < p ? (T)(d_scale * d[p - 1 - k0]) : (T)0;
    v.y = k1 < p ? (T)(d_scale * d[p - 1 - k1]) : (T)0;
    sm.A[pix(j)] = v;
  }
  __syncthreads();
  fft_complex<V, T, M>(sm.A, sm.B, tw, false);
  for (int f = threadIdx.x; f <= M / 2; f += kThreads) {
    V xf, xm;
    split2<V, T>(sm.A[pix(f)], sm.A[pix((M - f) & (M - 1))], tw[f], xf, xm);
    sm.D[f] = xf;
    sm.D[M - f] = xm;
  }
  __syncthreads();
}

template <typename V>
__device__ __forceinline__ void acc_add(double2& s, V v) {
  s.x += (double)v.x;
  s.y += (double)v.y;
}

// One tile of L rows starting at i0 of a product pass: u = X d - c u_old on the tile's rows (stored when u_new
// is given), and W . conj(U) added into the CTA's spectrum sm.S. wt: the tile's doubled window spectrum
// (M + 1 entries, global). Returns this thread's part of ||u||^2.
template <typename T, int N = FftCfg<T>::N>
__device__ double fft_tile(FftSmem<T, N>& sm, long long m, int L, const T* u_old, T* u_new, double coef, long long i0,
                           const typename FftCfg<T>::V* tw, const typename FftCfg<T>::V* __restrict__ wt,
                           bool lags) {
  using V = typename FftCfg<T>::V;
  constexpr int M = N / 2;
  const T sc = (T)(1.0 / (8.0 * M));
  const int rows = (int)min((long long)L, m - i0);
  // X d = IRFFT(W . conj(D)) on rows [0, L)
  for (int f = threadIdx.x; f <= M / 2; f += kThreads) {
    V zf, zm;
    merge2<V, T>(cmulc(wt[f], sm.D[f]), cmulc(wt[M - f], sm.D[M - f]), tw[f], zf, zm);
    sm.A[pix(f)] = zf;
    if (f != 0 && f != M / 2) sm.A[pix(M - f)] = zm;
  }
  __syncthreads();
  fft_complex<V, T, M>(sm.A, sm.B, tw, true);
  // u = X d - c u_old on the tile's rows, zero elsewhere; packed into B for its forward transform
  T nn = (T)0;
  for (int j = threadIdx.x; j < M; j += kThreads) {
    const int r0 = 2 * j, r1 = 2 * j + 1;
    const V z = sm.A[pix(j)];
    T u0 = (T)0, u1 = (T)0;
    if (r0 < rows) {
      u0 = z.x * sc;
      if (u_old) u0 = fma((T)(-coef), u_old[i0 + r0], u0);
      if (u_new) u_new[i0 + r0] = u0;
    }
    if (r1 < rows) {
      u1 = z.y * sc;
      if (u_old) u1 = fma((T)(-coef), u_old[i0 + r1], u1);
      if (u_new) u_new[i0 + r1] = u1;
    }
    nn = fma(u0, u0, fma(u1, u1, nn));
    V v;
    v.x = u0;
    v.y = u1;
    sm.B[pix(j)] = v;
  }
  __syncthreads();
  if (!lags) return (double)nn;   // no X^T u wanted (nlag == 0): u and ||u||^2 only
  fft_complex<V, T, M>(sm.B, sm.A, tw, false);
  // S += W . conj(U)
  for (int f = threadIdx.x; f <= M / 2; f += kThreads) {
    V uf, um;
    split2<V, T>(sm.B[pix(f)], sm.B[pix((M - f) & (M - 1))], tw[f], uf, um);
    acc_add(sm.S[f], cmulc(wt[f], uf));
    if (f != M / 2) acc_add(sm.S[M - f], cmulc(wt[M - f], um));
  }
  return (double)nn;
}

// One tile of the Gram pass: the tile's doubled window spectrum into wt (global), and the lag sums
// sum_{r < rows} y[i0 + r] y[i0 + r + k], k < nlag, into the CTA's state:
//   corr: S += |W|^2 (circular autocorrelation of the window) and tacc -= its pairs that start in the window's
//         last p_pad samples: sum_{j < p_pad} ext[j] ext[j + k], ext = (window tail, window head); the last
//         tile also drops its pairs that start at rows >= m.
//   else: S += W . conj(B), B the spectrum of the tile's row block (zero beyond its rows).
template <typename T, int N = FftCfg<T>::N>
__device__ void fft_gram_tile(FftSmem<T, N>& sm, const T* __restrict__ y, long long n, long long m, int L, int p_pad,
                              int nlag, long long i0, const typename FftCfg<T>::V* tw,
                              typename FftCfg<T>::V* __restrict__ wt, bool corr) {
  using V = typename FftCfg<T>::V;
  constexpr int M = N / 2;
  const int rows = (int)min((long long)L, m - i0);
  if (corr) {
    for (int j = threadIdx.x; j < 2 * p_pad; j += kThreads) {
      const long long g = j < p_pad ? i0 + L + j : i0 + (j - p_pad);
      sm.ext[j] = g < n ? y[g] : (T)0;
    }
  }
  fft_window<T, N>(sm, y, n, i0, tw);
  for (int f = threadIdx.x; f <= M / 2; f += kThreads) {
    V xf, xm;
    split2<V, T>(sm.A[pix(f)], sm.A[pix((M - f) & (M - 1))], tw[f], xf, xm);
    wt[f] = xf;
    wt[M - f] = xm;
    if (corr) {
      sm.S[f].x += (double)xf.x * xf.x + (double)xf.y * xf.y;
      if (f != M / 2) sm.S[M - f].x += (double)xm.x * xm.x + (double)xm.y * xm.y;
    }
  }
  if (corr) {
    for (int k = threadIdx.x; k < nlag; k += kThreads) {
      double c = 0.0;
      for (int j = 0; j < p_pad; ++j) c = fma((double)sm.ext[j], (double)sm.ext[j + k], c);
      if (rows < L) {
        const long long hi = min(i0 + L, n - k);
        for (long long i = m; i < hi; ++i) c = fma((double)y[i], (double)y[i + k], c);
      }
      sm.tacc[k] -= c;
    }
    return;
  }
  // row block spectrum B (sm.B is free: the window transform ended in sm.A)
  for (int j = threadIdx.x; j < M; j += kThreads) {
    const int r0 = 2 * j, r1 = 2 * j + 1;
    V v;
    v.x = r0 < rows ? y[i0 + r0] : (T)0;
    v.y = r1 < rows ? y[i0 + r1] : (T)0;
    sm.B[pix(j)] = v;
  }
  __syncthreads();
  fft_complex<V, T, M>(sm.B, sm.A, tw, false);
  for (int f = threadIdx.x; f <= M / 2; f += kThreads) {
    V bf, bm;
    split2<V, T>(sm.B[pix(f)], sm.B[pix((M - f) & (M - 1))], tw[f], bf, bm);
    acc_add(sm.S[f], cmulc(wt[f], bf));      // wt[f], wt[M - f]: written by this thread above
    if (f != M / 2) acc_add(sm.S[M - f], cmulc(wt[M - f], bm));
  }
}

// End of a CTA's tiles: tacc[k] += IRFFT(S)[k], k < nlag (S holds 4x the true spectrum: scale 1 / (8 M)).
template <typename T, int N = FftCfg<T>::N>
__device__ void fft_finish_lags(FftSmem<T, N>& sm, int nlag, const typename FftCfg<T>::V* tw) {
  using V = typename FftCfg<T>::V;
  constexpr int M = N / 2;
  for (int f = threadIdx.x; f <= M / 2; f += kThreads) {
    V vf, vm, zf, zm;
    vf.x = (T)sm.S[f].x;
    vf.y = (T)sm.S[f].y;
    vm.x = (T)sm.S[M - f].x;
    vm.y = (T)sm.S[M - f].y;
    merge2<V, T>(vf, vm, tw[f], zf, zm);
    sm.A[pix(f)] = zf;
    if (f != 0 && f != M / 2) sm.A[pix(M - f)] = zm;
  }
  __syncthreads();
  fft_complex<V, T, M>(sm.A, sm.B, tw, true);
  const double sc = 1.0 / (8.0 * M);
  for (int k = threadIdx.x; k < nlag; k += kThreads) {
    const V z = sm.A[pix(k >> 1)];
    sm.tacc[k] += (double)((k & 1) ? z.y : z.x) * sc;
  }
}

// Twiddle table of the N-point transforms: exp(-2 pi i t / N), t < N (float N = 4,096; float64 N = 2,048 or 4,096).
template <typename T, int N>
__device__ __forceinline__ const typename FftCfg<T>::V* fft_twiddles(const Work& w) {
  using V = typename FftCfg<T>::V;
  if (sizeof(T) == 4) return reinterpret_cast<const V*>(w.tw32);
  return reinterpret_cast<const V*>(N == 4096 ? w.tw64x : w.tw64);
}

template <typename T, int N = FftCfg<T>::N>
__global__ void __launch_bounds__(kThreads, 3) fft_pass_kernel(PassArgs<T> a) {
  using V = typename FftCfg<T>::V;
  constexpr int M = N / 2;
  constexpr int WS = FftCfg2<T, N>::WS;
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
  const int L = N - p_pad;
  const V* tw = fft_twiddles<T, N>(a.w);
  V* wspec = reinterpret_cast<V*>(sizeof(T) == 8 ? a.w.wspec64 : a.w.wspec32);
  FftSmem<T, N> sm(smem_raw, p_pad);
  const int tid = threadIdx.x;
  for (int k = tid; k < p_pad + 16; k += kThreads) sm.tacc[k] = 0.0;
  for (int f = tid; f <= M; f += kThreads) sm.S[f] = make_double2(0.0, 0.0);
  const long long ntiles = (a.m + L - 1) / L;
  const bool corr = a.gram && (long long)p_pad * nlag <= GramCfg<T>::kDirectMax;
  if (!a.gram && blockIdx.x < ntiles) fft_d_spectrum<T, N>(sm, a.d, a.d_scale, a.p, tw);
  double n2 = 0.0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    V* wt = wspec + (size_t)tile * WS;
    if (a.gram) fft_gram_tile<T, N>(sm, a.y, a.n, a.m, L, p_pad, nlag, tile * L, tw, wt, corr);
    else n2 += fft_tile<T, N>(sm, a.m, L, u_old, u_new, coef, tile * L, tw, wt, nlag > 0);
  }
  __syncthreads();
  if (blockIdx.x < ntiles && nlag > 0) fft_finish_lags<T, N>(sm, nlag, tw);
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

template <typename T, int N = FftCfg<T>::N>
static size_t fft_pass_smem(int p_pad) {
  return FftSmem<T, N>::bytes(p_pad);
}

// Doubled window spectra of every tile of a series (tiles of L = N - p_pad rows), for passes whose Gram pass did
// not form them (another precision's Gram pass, or a single product pass): y does not change between passes.
template <typename T, int N = FftCfg<T>::N>
__global__ void __launch_bounds__(kThreads) spectrum_kernel(const T* __restrict__ y, long long n, long long m, int L,
                                                           typename FftCfg<T>::V* __restrict__ out,
                                                           const typename FftCfg<T>::V* tw) {
  using V = typename FftCfg<T>::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int M = N / 2;
  FftSmem<T, N> sm(smem_raw, 0);
  const long long ntiles = (m + L - 1) / L;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    fft_window<T, N>(sm, y, n, tile * L, tw);
    V* wt = out + (size_t)tile * FftCfg2<T, N>::WS;
    for (int f = threadIdx.x; f <= M / 2; f += kThreads) {
      V xf, xm;
      split2<V, T>(sm.A[pix(f)], sm.A[pix((M - f) & (M - 1))], tw[f], xf, xm);
      wt[f] = xf;
      wt[M - f] = xm;
    }
  }
}

// Batched float64 overlap-save pass: the CTAs stride over one list of work units, each up to kBatchFftUnit
// consecutive FFT tiles of one series (tiles of L = N - pad_p(p + 1) rows; window spectra formed by the batch's
// Gram pass; the spectrum of the series' d formed before the pass by batch_dspec_kernel). A unit sums its tiles'
// X^T u spectra and transforms back once; the grouping depends only on the series, so a series' partials, and so
// its result, do not depend on the rest of the batch. The units of a series then arrive and its last CTA runs
// the series' scalar step.
__global__ void __launch_bounds__(kThreads, 3) batch_fft_kernel(BatchArgs a) {
  using T = double;
  using V = double2;
  constexpr int N = FftCfg<T>::N;
  constexpr int M = N / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const long long tiles_x = a.live ? a.live[2] : a.tiles_x;
  for (long long g = blockIdx.x; g < tiles_x; g += gridDim.x) {
    const int sidx = a.tile_series_x[g];
    const BatchSeries& S = a.series[sidx];
    const Work& w = S.w;
    const int p = w.p, pg = pad_p(p + 1), L = N - pg;
    const long long unit = g - S.tile0_x, ntiles = (w.m + L - 1) / L;
    const long long nunits = (ntiles + kBatchFftUnit - 1) / kBatchFftUnit;
    int tail = TAIL_GRAM;
    const T* u_old = nullptr;
    T* u_new = nullptr;
    double coef = 0.0;
    const int gram = a.gram;
    const int nlag = gram ? p + 1 : p;
    // every thread reads the series state itself: it cannot change while a unit of the series is pending
    if (!gram && !select_phase<T>(w.st, w.y64, p, w, tail, u_old, u_new, coef)) continue;
    __syncthreads();                                   // the previous unit is done with shared memory
    FftSmem<T> sm(smem_raw, pg);
    const V* tw = reinterpret_cast<const V*>(w.tw64);
    for (int k = tid; k < pg + 16; k += kThreads) sm.tacc[k] = 0.0;
    for (int f = tid; f <= M; f += kThreads) sm.S[f] = make_double2(0.0, 0.0);
    if (!gram) {
      const V* dsp = reinterpret_cast<const V*>(w.dspec64);
      for (int f = tid; f <= M; f += kThreads) sm.D[f] = dsp[f];
    }
    const bool corr = (long long)pg * nlag <= GramCfg<T>::kDirectMax;
    double n2 = 0.0;
    const long long t1 = lmin((unit + 1) * kBatchFftUnit, ntiles);
    for (long long t = unit * kBatchFftUnit; t < t1; ++t) {
      __syncthreads();
      V* wt = reinterpret_cast<V*>(w.wspec64) + (size_t)t * FftCfg<T>::WS;
      if (gram) fft_gram_tile<T>(sm, w.y64, w.n, w.m, L, pg, nlag, t * L, tw, wt, corr);
      else n2 += fft_tile<T>(sm, w.m, L, u_old, u_new, coef, t * L, tw, wt, true);
    }
    __syncthreads();
    fft_finish_lags<T>(sm, nlag, tw);
    __syncthreads();
    for (int k = tid; k < nlag; k += kThreads) w.part_t[(size_t)unit * pg + k] = sm.tacc[k];
    const double n2_unit = block_sum(n2, sm.scratch);
    if (tid == 0) w.part_n2[unit] = n2_unit;
    if (!arrive(w, unit, nunits, nlag, pg, sm.tacc, sm.scratch, &s_last)) continue;
    const double n2_all = sm.scratch[8];
    __syncthreads();
    if (tid == 0) w.st->fft = 1;
    run_tail<T>(tail, w, gram, nlag, sm.tacc, n2_all, sm.scratch, nullptr, w.bnorm2);
    __syncthreads();
    if (tid == 0 && !gram && w.st->done && a.done_count) atomicAdd(a.done_count, 1u);
  }
}

// Doubled spectrum of the lag-reversed d of every batched FFT series that has a float64 pass to run (one CTA per
// series), for the batch_fft_kernel launch that follows.
__global__ void __launch_bounds__(kThreads) batch_dspec_kernel(const BatchSeries* series) {
  using V = double2;
  constexpr int M = FftCfg<double>::N / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_go;
  const Work& w = series[blockIdx.x].w;
  if (!w.dspec64) return;
  if (threadIdx.x == 0) {
    int tail;
    const double* uo;
    double* un;
    double c;
    s_go = select_phase<double>(w.st, w.y64, w.p, w, tail, uo, un, c);
  }
  __syncthreads();
  if (!s_go) return;
  FftSmem<double> sm(smem_raw, 0);
  fft_d_spectrum<double>(sm, w.d, 1.0, w.p, reinterpret_cast<const V*>(w.tw64));
  V* out = reinterpret_cast<V*>(w.dspec64);
  for (int f = threadIdx.x; f <= M; f += kThreads) out[f] = sm.D[f];
}

// ------------------------------------------------------------------------------------------------------------
// Register-blocked float product pass (N = 4,096, M = 2,048; the float solver and step passes with X^T u, not the
// Gram pass). The same arithmetic as fft_pass_kernel<float>, arranged so that every pointwise step works on
// registers: thread j holds the points j + 256 r (r < 8) of a 2,048-point transform. The Stockham radix-8, 8, 8, 4
// transform reads its first stage's input from, and leaves its last stage's output in, exactly that set, so the
// spectral products before the inverse transform, the rows of u between the two transforms and the split after the
// forward transform need no shared-memory pass; three exchanges per transform remain. The split and merge pair bin
// f with bin M - f: lanes 0-15 of warp w take j = 16 w + l and lanes 16-31 the partners 256 - j (0 pairs with 128),
// so the pair sits on lanes l and l ^ 16 of one warp (a shuffle).
//
// A tile's inputs from HBM — its window spectrum (16,400 bytes) and its rows of u_old — arrive by bulk copies
// (cp.async.bulk, completion counted on an mbarrier) issued one tile ahead by thread 0: the spectrum into one of two
// shared buffers while the previous tile still reads the other, u_old into one buffer as soon as the previous
// tile's rows have been read. No thread waits on a global load of the main loop. Twiddles: each thread reads the
// base twiddle of each of its stages once per launch and forms the rest by products. The CTA's spectral sum
// W . conj(U) is kept per thread in float over at most kFft32Flush tiles and then added to the CTA's running sum, a
// float pair per bin in global memory (each thread owns its bins: no atomics); the CTA transforms its sum back once,
// at its end.
constexpr int kFft32Flush = 16;

// t * exp(-+2 pi i r / 8) (INV: +) for r = 1, 2, 3, without products by 0 or 1 (h = 1/sqrt(2)).
template <bool INV, int r>
__device__ __forceinline__ float2 mul_e8(float2 t) {
  const float h = 0.70710678118654752f;
  if (r == 1) return INV ? make_float2(h * (t.x - t.y), h * (t.x + t.y)) : make_float2(h * (t.x + t.y), h * (t.y - t.x));
  if (r == 2) return INV ? make_float2(-t.y, t.x) : make_float2(t.y, -t.x);
  return INV ? make_float2(-h * (t.x + t.y), h * (t.x - t.y)) : make_float2(h * (t.y - t.x), -h * (t.x + t.y));
}

__device__ __forceinline__ int fft32_j(int tid) {
  const int w = tid >> 5, l = tid & 31;
  const int a = 16 * w + (l & 15);
  return l < 16 ? a : (a == 0 ? 128 : 256 - a);
}

// pv[q] = the value of bin M - f at this thread's bin f = j + 256 q (bin M itself, the partner of bin 0, is the
// caller's business where it differs from bin 0).
__device__ __forceinline__ void fft32_partner(const float2* v, float2* pv, int j) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    pv[q].x = __shfl_xor_sync(0xffffffffu, v[7 - q].x, 16);
    pv[q].y = __shfl_xor_sync(0xffffffffu, v[7 - q].y, 16);
  }
  if (j == 128) {
#pragma unroll
    for (int q = 0; q < 8; ++q) pv[q] = v[7 - q];
  } else if (j == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) pv[q] = v[(8 - q) & 7];
  }
}

// Per-thread base twiddles of the register-blocked transform (forward sign; the inverse conjugates them): the
// second stage's w = exp(-2 pi i (j mod 8) / 64), the third's exp(-2 pi i (j mod 64) / 512) and the last stage's
// exp(-2 pi i j / 2048). They depend on j only, so a thread reads them once per launch and forms every other
// twiddle of its butterflies from them by products (each within a few ulp).
struct Fft32Tw {
  float2 s2, s3, s4;
};
__device__ __forceinline__ Fft32Tw fft32_base_twiddles(const float2* tw, int j) {
  Fft32Tw t;
  t.s2 = tw[64 * (j & 7)];
  t.s3 = tw[8 * (j & 63)];
  t.s4 = tw[2 * j];
  return t;
}

// One Stockham radix-8 stage between shared buffers for the thread's butterfly j (stride 256): in[j + 256 r],
// twiddles w^r (w the stage's base twiddle), out[g Ln + k + Ls q] with k = j mod Ls.
template <bool INV, int Ls>
__device__ __forceinline__ void fft32_stage8(float2* z, int j, const float2* in, float2* out, float2 w) {
  constexpr int Ln = Ls * 8;
  const int k = j & (Ls - 1), g = j / Ls;
#pragma unroll
  for (int r = 0; r < 8; ++r) z[r] = in[pix(j + 256 * r)];
  float2 t[8];
  t[1] = w;
  if (INV) t[1].y = -t[1].y;
  t[2] = cmul(t[1], t[1]);
  t[4] = cmul(t[2], t[2]);
  t[3] = cmul(t[1], t[2]);
  t[5] = cmul(t[4], t[1]);
  t[6] = cmul(t[4], t[2]);
  t[7] = cmul(t[4], t[3]);
#pragma unroll
  for (int r = 1; r < 8; ++r) z[r] = cmul(z[r], t[r]);
  dft_small<float2, float, 8>(z, INV);
#pragma unroll
  for (int q = 0; q < 8; ++q) out[pix(g * Ln + k + Ls * q)] = z[q];
}

// 2,048-point complex transform of the thread-held points z[r] = x[j + 256 r]; on return z[r] = X[j + 256 r].
// Stages radix 8 (Ls 1, from registers), 8 (Ls 8), 8 (Ls 64), 4 (Ls 512, into registers); bufA, bufB carry the
// three exchanges. The caller separates a later write of bufA from this call's last reads by a barrier.
// after_first_sync() runs in every thread right after the first barrier (every thread has then left the code
// before this call).
template <bool INV, typename F>
__device__ __forceinline__ void fft32_2048(float2* z, int j, float2* bufA, float2* bufB, const Fft32Tw& tw,
                                           F&& after_first_sync) {
  dft_small<float2, float, 8>(z, INV);
#pragma unroll
  for (int q = 0; q < 8; ++q) bufA[pix(8 * j + q)] = z[q];
  __syncthreads();
  after_first_sync();
  fft32_stage8<INV, 8>(z, j, bufA, bufB, tw.s2);
  __syncthreads();
  fft32_stage8<INV, 64>(z, j, bufB, bufA, tw.s3);
  __syncthreads();
  float2 a[4], b[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = bufA[pix(j + 512 * r)];
    b[r] = bufA[pix(j + 256 + 512 * r)];
  }
  // twiddles w^r of butterfly j (w = exp(-+2 pi i j / 2048)); those of j + 256 times exp(-+2 pi i r / 8)
  float2 ta[4];
  ta[1] = tw.s4;
  if (INV) ta[1].y = -ta[1].y;
  ta[2] = cmul(ta[1], ta[1]);
  ta[3] = cmul(ta[1], ta[2]);
#pragma unroll
  for (int r = 1; r < 4; ++r) {
    const float2 tb = r == 1 ? mul_e8<INV, 1>(ta[r]) : r == 2 ? mul_e8<INV, 2>(ta[r]) : mul_e8<INV, 3>(ta[r]);
    a[r] = cmul(a[r], ta[r]);
    b[r] = cmul(b[r], tb);
  }
  dft_small<float2, float, 4>(a, INV);
  dft_small<float2, float, 4>(b, INV);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    z[2 * q] = a[q];
    z[2 * q + 1] = b[q];
  }
}

// w^f for f = j + 256 q (N = 4,096): w^j exp(-i pi q / 8), one table entry and a product with a constant (for
// even q a multiple of exp(-i pi / 4): no products by 0 or 1).
__device__ __forceinline__ float2 fft32_twf(float2 base, int q) {
  if (q == 0) return base;
  if (q == 2) return mul_e8<false, 1>(base);
  if (q == 4) return mul_e8<false, 2>(base);
  if (q == 6) return mul_e8<false, 3>(base);
  const float c = q == 1 ? 0.92387953251128676f : q == 3 ? 0.38268343236508977f : q == 5 ? -0.38268343236508977f
                                                                                            : -0.92387953251128676f;
  const float sn = q == 1 ? 0.38268343236508977f : q == 3 ? 0.92387953251128676f : q == 5 ? 0.92387953251128676f
                                                                                           : 0.38268343236508977f;
  return cmul(base, make_float2(c, -sn));
}

// 2Z[f] of the packed input of an inverse transform from the doubled half spectrum V at bins f and M - f (merge2).
__device__ __forceinline__ float2 fft32_merge(float2 vf, float2 vmf, float2 twf) {
  const float ax = vf.x + vmf.x, ay = vf.y - vmf.y;
  const float bx = vf.x - vmf.x, by = vf.y + vmf.y;
  const float cbx = twf.x * bx + twf.y * by;
  const float cby = twf.x * by - twf.y * bx;
  return make_float2(ax - cby, ay + cbx);
}
// 2X[f] (and, for f = 0, 2X[M] in xm) of a real sequence from its packed transform Z at bins f and M - f (split2).
__device__ __forceinline__ float2 fft32_split(float2 zf, float2 zmf, float2 twf, float2* xm) {
  const float ax = zf.x + zmf.x, ay = zf.y - zmf.y;
  const float bx = zf.x - zmf.x, by = zf.y + zmf.y;
  const float tbx = twf.x * bx - twf.y * by;
  const float tby = twf.x * by + twf.y * bx;
  if (xm) *xm = make_float2(ax - tby, -(ay + tbx));
  return make_float2(ax + tby, ay - tbx);
}

// mbarrier and bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk; sm_90 and later).
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// One arrival on bar announcing `bytes` of transfer, then the copy global -> shared that completes them. dst, src
// 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Wait for the phase of parity `parity` of bar to complete, polling at most `polls` times (each poll suspends for
// up to about a microsecond); false if it gave up.
constexpr int kMbarPolls = 1 << 21;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int polls = kMbarPolls) {
  const unsigned a = smem_addr(bar);
  for (int i = 0; i < polls; ++i) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, 1000;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Shared memory of fft32_pass_kernel: exchange buffers A, B (padded), the spectrum D of the lag-reversed d, two
// staged window spectra, the staged u_old rows of a tile, three mbarriers, tacc, scratch.
struct Fft32Smem {
  static constexpr int M = FftCfg<float>::N / 2;
  static constexpr int PADDED = FftCfg2<float>::PADDED;
  static constexpr int WS = FftCfg<float>::WS;
  static constexpr int UROWS = FftCfg<float>::N;     // more than any tile's rows
  float2 *A, *B, *D, *W;     // W: the two spectrum buffers, WS entries apart
  float* U;
  unsigned long long* bar;   // [0], [1]: the spectrum buffers; [2]: the u_old buffer
  double *tacc, *scratch;
  __host__ __device__ static size_t bytes(int p_pad) {
    return sizeof(float2) * (2 * (size_t)PADDED + 3 * (size_t)WS) + sizeof(float) * UROWS + 32 +
           sizeof(double) * ((size_t)p_pad + 16 + 16);
  }
  __device__ Fft32Smem(unsigned char* raw) {
    A = reinterpret_cast<float2*>(raw);
    B = A + PADDED;
    D = B + PADDED;
    W = D + WS;
    U = reinterpret_cast<float*>(W + 2 * WS);
    bar = reinterpret_cast<unsigned long long*>(U + UROWS);
    tacc = reinterpret_cast<double*>(bar + 4);
    scratch = nullptr;   // set by the kernel (after tacc's p_pad + 16 entries)
  }
};
static_assert((sizeof(float2) * 2 * FftCfg2<float>::PADDED) % 16 == 0, "D, W, U must start 16-byte aligned");
static_assert((sizeof(float2) * FftCfg<float>::WS) % 16 == 0, "a spectrum tile must be a multiple of 16 bytes");

__global__ void __launch_bounds__(kThreads, 2) fft32_pass_kernel(PassArgs<float> a) {
  using V = float2;
  constexpr int N = FftCfg<float>::N;
  constexpr int M = N / 2;
  constexpr int WS = FftCfg<float>::WS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  int tail = a.tail;
  const float* u_old = a.u_old;
  float* u_new = a.u_new;
  double coef = a.coef_host;
  if (a.check_done) {
    if (!select_phase<float>(a.w.st, a.y, a.p, a.w, tail, u_old, u_new, coef)) return;
  } else if (a.coef_dev) {
    coef = *a.coef_dev;
  }
  const int p_pad = a.p_pad, nlag = a.nlag;
  const int L = N - p_pad;
  const V* tw = reinterpret_cast<const V*>(a.w.tw32);
  const V* wspec = reinterpret_cast<const V*>(a.w.wspec32);
  Fft32Smem sm(smem_raw);
  sm.scratch = sm.tacc + p_pad + 16;
  const int tid = threadIdx.x;
  const int j = fft32_j(tid);
  for (int k = tid; k < p_pad + 16; k += kThreads) sm.tacc[k] = 0.0;
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_init(&sm.bar[2], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const long long ntiles = (a.m + L - 1) / L;
  double n2 = 0.0;
  // a wait that gives up marks the thread failed: it waits no more, and thread 0 issues no further copy (a buffer
  // whose copy may still be landing is never the target of another), so the rest of the launch runs on stale data
  // and ends; the host reads the flag and reports TOLS_ERR_DEVICE_TIMEOUT
  const int polls = a.wait_polls > 0 ? a.wait_polls : a.wait_polls < 0 ? 0 : kMbarPolls;
  bool failed = false;
  unsigned iss_w0 = 0u, iss_w1 = 0u, iss_u = 0u;   // thread 0: copies issued on bar[0], bar[1], bar[2]
  // u_old rows of a tile that arrive by the bulk copy (a multiple of 4 rows; the rest are read directly)
  auto u_bytes = [&](long long t) -> unsigned {
    if (!u_old) return 0u;
    const long long rows = lmin((long long)L, a.m - t * L);
    return (unsigned)(rows * (long long)sizeof(float)) & ~15u;
  };
  auto issue_w = [&](long long t, int b) {
    bulk_load(sm.W + b * WS, wspec + (size_t)t * WS, (unsigned)(sizeof(V) * WS), &sm.bar[b]);
    if (b) ++iss_w1;
    else ++iss_w0;
  };
  auto issue_u = [&](long long t) {
    const unsigned nb = u_bytes(t);
    if (nb) {
      bulk_load(sm.U, u_old + t * L, nb, &sm.bar[2]);
      ++iss_u;
    }
  };
  if (blockIdx.x < ntiles) {
    if (tid == 0) {
      issue_w(blockIdx.x, 0);       // the first tile's inputs arrive while d's spectrum is formed
      issue_u(blockIdx.x);
    }
    const V twj = tw[j];
    const Fft32Tw twb = fft32_base_twiddles(tw, j);
    V z[8], pv[8];
    // doubled spectrum of the lag-reversed, scaled d (point i = j + 256 r holds d entries 2i, 2i + 1)
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int k0 = 2 * (j + 256 * r);
      z[r].x = k0 < a.p ? (float)(a.d_scale * a.d[a.p - 1 - k0]) : 0.f;
      z[r].y = k0 + 1 < a.p ? (float)(a.d_scale * a.d[a.p - 2 - k0]) : 0.f;
    }
    fft32_2048<false>(z, j, sm.A, sm.B, twb, [] {});
    fft32_partner(z, pv, j);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      V xm;
      sm.D[j + 256 * q] = fft32_split(z[q], pv[q], fft32_twf(twj, q), (q == 0 && j == 0) ? &xm : nullptr);
      if (q == 0 && j == 0) sm.D[M] = xm;
    }
    __syncthreads();     // D complete; sm.A / sm.B free for the tiles
    V Sq[8], Sm = make_float2(0.f, 0.f), nnq = make_float2(0.f, 0.f);
    float n2h = 0.f, n2l = 0.f;    // this thread's ||u||^2, a float pair (TwoSum per flush)
#pragma unroll
    for (int q = 0; q < 8; ++q) Sq[q] = make_float2(0.f, 0.f);
    // the CTA's running sum per bin as an unevaluated float pair {re, im, re lo, im lo}: each flush adds by Knuth's
    // TwoSum, so the pair keeps about twice float's precision with float instructions only (a float64 add here
    // costs a warp 64 issue cycles of GB300's FP64 pipe)
    float4* sacc = reinterpret_cast<float4*>(a.w.sacc32) + (size_t)blockIdx.x * (M + 1);
    bool first_flush = true;
    int pending = 0;
    auto two_sum_add = [](float4& s, float2 x) {
      const float hx = s.x + x.x, bx = hx - s.x, ex = (s.x - (hx - bx)) + (x.x - bx);
      const float hy = s.y + x.y, by = hy - s.y, ey = (s.y - (hy - by)) + (x.y - by);
      s = make_float4(hx, hy, s.z + ex, s.w + ey);
    };
    auto flush = [&]() {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float4 s = first_flush ? make_float4(0.f, 0.f, 0.f, 0.f) : sacc[j + 256 * q];
        two_sum_add(s, Sq[q]);
        sacc[j + 256 * q] = s;
        Sq[q] = make_float2(0.f, 0.f);
      }
      if (j == 0) {
        float4 s = first_flush ? make_float4(0.f, 0.f, 0.f, 0.f) : sacc[M];
        two_sum_add(s, Sm);
        sacc[M] = s;
        Sm = make_float2(0.f, 0.f);
      }
      {
        const float x = nnq.x + nnq.y, h = n2h + x, bb = h - n2h;
        n2l += (n2h - (h - bb)) + (x - bb);
        n2h = h;
      }
      nnq = make_float2(0.f, 0.f);
      first_flush = false;
      pending = 0;
    };
    const float sc = 1.0f / (8.0f * M);
    const float c = (float)coef;
    unsigned kw = 0, ku = 0;          // tiles consumed: spectrum buffer kw & 1 (phase kw >> 1), u_old phase ku
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++kw) {
      const int b = kw & 1;
      const long long i0 = tile * L;
      const int rows = (int)lmin((long long)L, a.m - i0);
      const long long nt = tile + gridDim.x;
      if (!failed && !mbar_wait(&sm.bar[b], (kw >> 1) & 1u, polls)) failed = true;
      const V* wt = sm.W + b * WS;
      // X d = IRFFT(W . conj(D)) on the tile's rows
#pragma unroll
      for (int q = 0; q < 8; ++q) z[q] = cmulc(wt[j + 256 * q], sm.D[j + 256 * q]);
      fft32_partner(z, pv, j);
      if (j == 0) pv[0] = cmulc(wt[M], sm.D[M]);      // the partner of bin 0 is bin M
#pragma unroll
      for (int q = 0; q < 8; ++q) z[q] = fft32_merge(z[q], pv[q], fft32_twf(twj, q));
      // past the first barrier every thread is done with the other spectrum buffer (the previous tile)
      fft32_2048<true>(z, j, sm.A, sm.B, twb, [&] {
        if (tid == 0 && !failed && nt < ntiles) issue_w(nt, b ^ 1);
      });
      // rows 2i, 2i + 1 of u_old for the thread's points i = j + 256 r (tile offsets are even: L is)
      const unsigned ub = u_bytes(tile);
      const int rows_al = (int)(ub / sizeof(float));
      if (ub) {
        if (!failed && !mbar_wait(&sm.bar[2], ku & 1u, polls)) failed = true;
        ++ku;
      }
      V uo[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int r0 = 2 * (j + 256 * r);
        uo[r] = make_float2(0.f, 0.f);
        if (u_old) {
          if (r0 + 1 < rows_al) {
            uo[r] = *reinterpret_cast<const V*>(sm.U + r0);
          } else {
            if (r0 < rows) uo[r].x = r0 < rows_al ? sm.U[r0] : u_old[i0 + r0];
            if (r0 + 1 < rows) uo[r].y = u_old[i0 + r0 + 1];
          }
        }
      }
      // u = X d - c u_old on the tile's rows, zero elsewhere; u_new stored; ||u||^2 summed in float over the
      // flush window, per lane pair
      const float2 sc2 = make_float2(sc, sc), mc2 = make_float2(-c, -c);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int r0 = 2 * (j + 256 * r);
        float2 u = __fmul2_rn(z[r], sc2);
        if (u_old) u = __ffma2_rn(uo[r], mc2, u);
        if (r0 >= rows) u.x = 0.f;
        if (r0 + 1 >= rows) u.y = 0.f;
        if (u_new) {
          if (r0 + 1 < rows) *reinterpret_cast<V*>(u_new + i0 + r0) = u;
          else if (r0 < rows) u_new[i0 + r0] = u.x;
        }
        nnq = __ffma2_rn(u, u, nnq);
        z[r] = u;
      }
      // S += W . conj(U), U the doubled half spectrum of u; past the first barrier u_old's buffer is free
      fft32_2048<false>(z, j, sm.B, sm.A, twb, [&] {
        if (tid == 0 && !failed && nt < ntiles) issue_u(nt);
      });
      fft32_partner(z, pv, j);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        V xm;
        const V x = fft32_split(z[q], pv[q], fft32_twf(twj, q), (q == 0 && j == 0) ? &xm : nullptr);
        Sq[q] = __fadd2_rn(Sq[q], cmulc(wt[j + 256 * q], x));
        if (q == 0 && j == 0) {
          const V tm = cmulc(wt[M], xm);
          Sm.x += tm.x;
          Sm.y += tm.y;
        }
      }
      if (++pending == kFft32Flush) flush();
    }
    {
      if (pending) flush();
      n2 = (double)n2h + (double)n2l;
      // tacc[k] = IRFFT(S)[k], k < nlag, from this thread's bins of the CTA's sum (S holds 4x the true spectrum:
      // scale 1 / (8 M))
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 s = sacc[j + 256 * q];
        z[q] = make_float2(s.x + s.z, s.y + s.w);
      }
      fft32_partner(z, pv, j);
      if (j == 0) {
        const float4 s = sacc[M];
        pv[0] = make_float2(s.x + s.z, s.y + s.w);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) z[q] = fft32_merge(z[q], pv[q], fft32_twf(twj, q));
      fft32_2048<true>(z, j, sm.A, sm.B, twb, [] {});
      const double scd = 1.0 / (8.0 * M);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int k0 = 2 * (j + 256 * r);
        if (k0 < nlag) sm.tacc[k0] = (double)z[r].x * scd;
        if (k0 + 1 < nlag) sm.tacc[k0 + 1] = (double)z[r].y * scd;
      }
    }
  }
  if (tid == 0) {
    // every copy this CTA issued has completed before it leaves (waits bounded, at the full limit)
    if (iss_w0 && !mbar_wait(&sm.bar[0], (iss_w0 - 1) & 1u)) failed = true;
    if (iss_w1 && !mbar_wait(&sm.bar[1], (iss_w1 - 1) & 1u)) failed = true;
    if (iss_u && !mbar_wait(&sm.bar[2], (iss_u - 1) & 1u)) failed = true;
  }
  if (failed && a.w.st) atomicExch(&a.w.st->dev_error, 1);
  __syncthreads();
  const double n2_cta = block_sum(n2, sm.scratch);
  for (int k = tid; k < nlag; k += kThreads) a.w.part_t[(size_t)blockIdx.x * p_pad + k] = sm.tacc[k];
  if (tid == 0) a.w.part_n2[blockIdx.x] = n2_cta;
  if (!arrive(a.w, blockIdx.x, gridDim.x, nlag, p_pad, sm.tacc, sm.scratch, &s_last)) return;
  const double n2_all = sm.scratch[8];
  __syncthreads();
  if (tid == 0 && a.worklog) a.worklog[a.work_slot] = 1 + tail;
  run_tail<float>(tail, a.w, a.gram, nlag, sm.tacc, n2_all, sm.scratch, a.out_t, a.out_n2);
}

static size_t fft32_pass_smem(int p_pad) { return Fft32Smem::bytes(p_pad); }
