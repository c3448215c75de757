// Overlap-save FFT product pass (included by tols_kernels.cu: it shares the arrival and tail code).
//
// The same outputs as pass_kernel — u_new = X d - c u_old, ||u_new||^2, X^T u_new (or the Gram lag sums) — with
// the two structured products of eq. (xphi) done as circular correlations of length N per tile of L = N - p_pad
// rows, which never wrap inside the rows and lags used:
//   (X d)[i0 + r] = sum_{k<p} w[r + k] dr[k]          = IDFT(W . conj(DR))[r],   r < L
//   tk[k]         = sum_{r<L} u[r] w[r + k]             = IDFT(W . conj(U))[k],    k < nlag
// with w the window y[i0 .. i0+N), dr the lag-reversed d, u the tile's fresh u (zero beyond its rows). Per tile:
// one forward real FFT of the window, one inverse for X d, one forward of u, one inverse for X^T u; the spectrum
// of dr is formed once per CTA and launch.
//
// A real N-point FFT is an N/2-point complex FFT of the packed pairs (w[2j], w[2j+1]) plus an O(N) split; the
// complex FFT is a radix-8 (then 4, 2) Stockham autosort in shared memory, one butterfly per thread per stage.
// Twiddles come from a table of exp(-2 pi i t / N), t < N, computed on the host in float64.
#pragma once

// Index into the FFT work arrays: one pad element after every 8, so that the strided writes of the first
// Stockham stages (stride 8 complex values) land in distinct shared-memory banks.
__device__ __forceinline__ int pix(int i) { return i + (i >> 3); }

template <typename T>
struct FftCfg;
template <>
struct FftCfg<float> {
  static constexpr int N = 4096;
  using V = float2;
};
template <>
struct FftCfg<double> {
  static constexpr int N = 2048;
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
// tw: exp(-2 pi i t / (2M)), t < 2M; omega_M^s = tw[2s].
template <typename V, typename S, int R, int M>
__device__ __forceinline__ void fft_stage(const V* __restrict__ in, V* __restrict__ out, int Ls,
                                          const V* __restrict__ tw, bool inv) {
  constexpr int stride = M / R;
  const int Ln = Ls * R;
  const int tstep = 2 * (M / Ln);
  for (int j = threadIdx.x; j < stride; j += kThreads) {
    const int k = j & (Ls - 1);
    const int g = j / Ls;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[pix(j + r * stride)];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      V t = tw[r * k * tstep];
      if (inv) t.y = -t.y;
      v[r] = cmul(v[r], t);
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
  fft_stage<V, S, 8, M>(a, b, 1, tw, inv);
  fft_stage<V, S, 8, M>(b, a, 8, tw, inv);
  fft_stage<V, S, 8, M>(a, b, 64, tw, inv);
  if (M == 2048) fft_stage<V, S, 4, M>(b, a, 512, tw, inv);
  else fft_stage<V, S, 2, M>(b, a, 512, tw, inv);
}

// Split of the packed complex transform Z of a real sequence into its half spectrum:
//   X[f] = (Z[f] + conj(Z[M-f])) / 2 - i w^f (Z[f] - conj(Z[M-f])) / 2,   w = exp(-2 pi i / N), Z[M] = Z[0].
template <typename V, typename S>
__device__ __forceinline__ V real_split(V zf, V zmf, V twf) {
  const V c = cconj(zmf);
  const V e = cscale(cadd(zf, c), (S)0.5);
  const V o = cscale(csub(zf, c), (S)0.5);
  return cadd(e, cmul(twf, cmul_mi(o, false)));
}
// Inverse: from a Hermitian half spectrum V (f in [0, M]) to the packed complex input of an inverse M-point FFT:
//   Z[f] = (V[f] + conj(V[M-f])) / 2 + i conj(w^f) (V[f] - conj(V[M-f])) / 2.
template <typename V, typename S>
__device__ __forceinline__ V real_merge(V vf, V vmf, V twf) {
  const V c = cconj(vmf);
  const V e = cscale(cadd(vf, c), (S)0.5);
  const V o = cscale(csub(vf, c), (S)0.5);
  return cadd(e, cmul_mi(cmul(cconj(twf), o), true));
}

template <typename T>
struct FftCfg2 {
  static constexpr int M = FftCfg<T>::N / 2;
  static constexpr int PADDED = M + M / 8 + 8;   // entries of a padded work array (index pix(f), f <= M)
};

template <typename T>
struct FftSmem {
  using V = typename FftCfg<T>::V;
  V *A, *B;               // work arrays, padded (pix)
  V *W, *D;               // half spectra, M + 1 entries each
  double *tacc, *scratch;
  __device__ FftSmem(unsigned char* raw, int p_pad) {
    constexpr int M = FftCfg<T>::N / 2;
    constexpr int PADDED = FftCfg2<T>::PADDED;
    A = reinterpret_cast<V*>(raw);
    B = A + PADDED;
    W = B + PADDED;
    D = W + (M + 1);
    tacc = reinterpret_cast<double*>(D + (M + 1));
    scratch = tacc + p_pad + 16;
  }
};

// Spectrum of the lag-reversed d (scaled), into sm.D.
template <typename T>
__device__ void fft_d_spectrum(FftSmem<T>& sm, const double* d, double d_scale, int p, const typename FftCfg<T>::V* tw) {
  using V = typename FftCfg<T>::V;
  constexpr int M = FftCfg<T>::N / 2;
  for (int j = threadIdx.x; j < M; j += kThreads) {
    const int k0 = 2 * j, k1 = 2 * j + 1;
    V v;
    v.x = k0 < p ? (T)(d_scale * d[p - 1 - k0]) : (T)0;
    v.y = k1 < p ? (T)(d_scale * d[p - 1 - k1]) : (T)0;
    sm.A[pix(j)] = v;
  }
  __syncthreads();
  fft_complex<V, T, M>(sm.A, sm.B, tw, false);
  for (int f = threadIdx.x; f <= M; f += kThreads)
    sm.D[f] = real_split<V, T>(sm.A[pix(f & (M - 1))], sm.A[pix((M - f) & (M - 1))], tw[f]);
  __syncthreads();
}

// One tile of L rows starting at i0. Accumulates X^T u (lag order) into sm.tacc; returns this thread's ||u||^2.
// Window spectrum W = RFFT(y[i0 .. i0 + N)) of one tile, into sm.W.
template <typename T>
__device__ void fft_window_spectrum(FftSmem<T>& sm, const T* __restrict__ y, long long n, long long i0,
                                    const typename FftCfg<T>::V* tw) {
  using V = typename FftCfg<T>::V;
  constexpr int M = FftCfg<T>::N / 2;
  for (int j = threadIdx.x; j < M; j += kThreads) {
    const long long g0 = i0 + 2 * j;
    V v;
    v.x = g0 < n ? y[g0] : (T)0;
    v.y = g0 + 1 < n ? y[g0 + 1] : (T)0;
    sm.A[pix(j)] = v;
  }
  __syncthreads();
  fft_complex<V, T, M>(sm.A, sm.B, tw, false);
  for (int f = threadIdx.x; f <= M; f += kThreads)
    sm.W[f] = real_split<V, T>(sm.A[pix(f & (M - 1))], sm.A[pix((M - f) & (M - 1))], tw[f]);
  __syncthreads();
}

// One tile of L rows starting at i0. Accumulates X^T u (lag order) into sm.tacc; returns this thread's ||u||^2.
// wsrc: the tile's window spectrum precomputed in global memory (M + 1 entries), or null to transform it here.
template <typename T>
__device__ double fft_tile(FftSmem<T>& sm, const T* __restrict__ y, long long n, long long m, int L, int nlag,
                           int gram, const T* u_old, T* u_new, double coef, long long i0,
                           const typename FftCfg<T>::V* tw, const typename FftCfg<T>::V* __restrict__ wsrc) {
  using V = typename FftCfg<T>::V;
  constexpr int M = FftCfg<T>::N / 2;
  const T invM = (T)1 / (T)M;
  const int rows = (int)min((long long)L, m - i0);
  if (wsrc) {
    for (int f = threadIdx.x; f <= M; f += kThreads) sm.W[f] = wsrc[f];
    __syncthreads();
  } else {
    fft_window_spectrum<T>(sm, y, n, i0, tw);
  }

  double n2 = 0.0;
  if (!gram) {
    // X d = IRFFT(W . conj(D)) on rows [0, L)
    for (int f = threadIdx.x; f <= M; f += kThreads) sm.B[pix(f)] = cmulc(sm.W[f], sm.D[f]);
    __syncthreads();
    for (int f = threadIdx.x; f < M; f += kThreads) sm.A[pix(f)] = real_merge<V, T>(sm.B[pix(f)], sm.B[pix(M - f)], tw[f]);
    __syncthreads();
    fft_complex<V, T, M>(sm.A, sm.B, tw, true);
    // u = X d - c u_old on the tile's rows, zero elsewhere; packed into B for its forward transform
    T nn = (T)0;
    for (int j = threadIdx.x; j < M; j += kThreads) {
      const int r0 = 2 * j, r1 = 2 * j + 1;
      const V z = sm.A[pix(j)];
      T u0 = (T)0, u1 = (T)0;
      if (r0 < rows) {
        u0 = z.x * invM;
        if (u_old) u0 = fma((T)(-coef), u_old[i0 + r0], u0);
        if (u_new) u_new[i0 + r0] = u0;
      }
      if (r1 < rows) {
        u1 = z.y * invM;
        if (u_old) u1 = fma((T)(-coef), u_old[i0 + r1], u1);
        if (u_new) u_new[i0 + r1] = u1;
      }
      nn = fma(u0, u0, fma(u1, u1, nn));
      V v;
      v.x = u0;
      v.y = u1;
      sm.B[pix(j)] = v;
    }
    n2 = (double)nn;
    __syncthreads();
    fft_complex<V, T, M>(sm.B, sm.A, tw, false);
  } else {
    // Gram lag sums: u = y itself on the tile's rows
    for (int j = threadIdx.x; j < M; j += kThreads) {
      const int r0 = 2 * j, r1 = 2 * j + 1;
      V v;
      v.x = r0 < rows ? y[i0 + r0] : (T)0;
      v.y = r1 < rows ? y[i0 + r1] : (T)0;
      sm.B[pix(j)] = v;
    }
    __syncthreads();
    fft_complex<V, T, M>(sm.B, sm.A, tw, false);
  }
  // X^T u = IRFFT(W . conj(U)) on lags [0, nlag)
  for (int f = threadIdx.x; f <= M; f += kThreads) {
    const V uf = real_split<V, T>(sm.B[pix(f & (M - 1))], sm.B[pix((M - f) & (M - 1))], tw[f]);
    sm.A[pix(f)] = cmulc(sm.W[f], uf);
  }
  __syncthreads();
  for (int f = threadIdx.x; f < M; f += kThreads) sm.B[pix(f)] = real_merge<V, T>(sm.A[pix(f)], sm.A[pix(M - f)], tw[f]);
  __syncthreads();
  fft_complex<V, T, M>(sm.B, sm.A, tw, true);
  for (int k = threadIdx.x; k < nlag; k += kThreads) {
    const V z = sm.B[pix(k >> 1)];
    sm.tacc[k] += (double)(((k & 1) ? z.y : z.x) * invM);
  }
  return n2;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 3) fft_pass_kernel(PassArgs<T> a) {
  using V = typename FftCfg<T>::V;
  constexpr int N = FftCfg<T>::N;
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
  const V* tw = reinterpret_cast<const V*>(sizeof(T) == 8 ? a.w.tw64 : a.w.tw32);
  FftSmem<T> sm(smem_raw, p_pad);
  const int tid = threadIdx.x;
  for (int k = tid; k < p_pad + 16; k += kThreads) sm.tacc[k] = 0.0;
  if (!a.gram) fft_d_spectrum<T>(sm, a.d, a.d_scale, a.p, tw);
  double n2 = 0.0;
  const long long ntiles = (a.m + L - 1) / L;
  const V* wspec = reinterpret_cast<const V*>(sizeof(T) == 8 ? a.w.wspec64 : a.w.wspec32);
  if (!a.use_wspec) wspec = nullptr;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    n2 += fft_tile<T>(sm, a.y, a.n, a.m, L, nlag, a.gram, u_old, u_new, coef, tile * L, tw,
                      wspec ? wspec + (size_t)tile * (FftCfg<T>::N / 2 + 1) : nullptr);
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

template <typename T>
static size_t fft_pass_smem(int p_pad) {
  using V = typename FftCfg<T>::V;
  constexpr int M = FftCfg<T>::N / 2;
  return sizeof(V) * (2 * (size_t)FftCfg2<T>::PADDED + 2 * (size_t)(M + 1)) + sizeof(double) * ((size_t)p_pad + 16 + 16);
}

// Window spectra of every tile of a series (tiles of L = N - p_pad rows), computed once per solve: y does not
// change between passes, so the passes read W from here instead of transforming the window again.
template <typename T>
__global__ void __launch_bounds__(kThreads) spectrum_kernel(const T* __restrict__ y, long long n, long long m, int L,
                                                           typename FftCfg<T>::V* __restrict__ out,
                                                           const typename FftCfg<T>::V* tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int M = FftCfg<T>::N / 2;
  FftSmem<T> sm(smem_raw, 0);
  const long long ntiles = (m + L - 1) / L;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    fft_window_spectrum<T>(sm, y, n, tile * L, tw);
    for (int f = threadIdx.x; f <= M; f += kThreads) out[(size_t)tile * (M + 1) + f] = sm.W[f];
  }
}
