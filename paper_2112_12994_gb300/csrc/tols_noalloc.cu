// Allocation-free variant of the fused product pass (toeplitz_ols_gk_pass_noalloc).
//
// Some callers cannot let this library allocate device memory: applications whose device memory is owned by
// another allocator (a framework's caching allocator, or a pool reserved up front to a fixed budget), where an
// extra cudaMalloc could fail or break the budget, and latency-critical loops where cudaMalloc / cudaFree are
// not acceptable because they can synchronise the device. For them this entry point needs no context and
// allocates nothing: the caller passes every input and output, and the cross-CTA partial sums and arrival
// counters the pass needs live in the fixed array below, part of the library image on every GPU that loads it
// (it stays resident until the process exits).
#include <string.h>

#include <mutex>

#include "tols_internal.cuh"

using namespace tols;

namespace {

constexpr int kNoAllocGrid = 304;                       // CTAs per launch (2 per SM on a 152-SM GB300)
constexpr int kNoAllocGroups = (kNoAllocGrid + kGroup - 1) / kGroup;
constexpr int kNoAllocPadP = pad_p(TOLS_NOALLOC_MAX_P);
// layout (doubles): counters (kMaxGroups + 1 unsigned ints, padded to 256 bytes), part_n2[kNoAllocGrid],
// grp_n2[kNoAllocGroups], part_t[kNoAllocGrid][p_pad], grp_t[kNoAllocGroups][p_pad]
constexpr size_t kCounterBytes = 256 * ((sizeof(unsigned int) * (kMaxGroups + 1) + 255) / 256);
constexpr size_t kScratchDoubles = kCounterBytes / sizeof(double) + kNoAllocGrid + kNoAllocGroups +
                                   (size_t)(kNoAllocGrid + kNoAllocGroups) * kNoAllocPadP + 1;  // ~660 KB

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

template <typename T>
int run(const void* d_y, long long n, int p, const double* d_v, const void* d_u_old, double c, void* d_u_new,
        double* d_xtu, double* d_unorm2, cudaStream_t stream, void* scratch) {
  const int pp = pad_p(p);
  Work w;
  memset(&w, 0, sizeof w);
  w.n = n;
  w.m = n - p;
  w.p = p;
  w.p_pad = pp;
  w.counters = reinterpret_cast<unsigned int*>(scratch);
  double* q = reinterpret_cast<double*>(reinterpret_cast<char*>(scratch) + kCounterBytes);
  w.part_n2 = q; q += kNoAllocGrid;
  w.grp_n2 = q; q += kNoAllocGroups;
  w.part_t = q; q += (size_t)kNoAllocGrid * pp;
  w.grp_t = q;
  // the arrival counters must start at zero (every pass also leaves them at zero)
  if (cudaMemsetAsync(scratch, 0, kCounterBytes, stream) != cudaSuccess) return TOLS_ERR_CUDA;
  PassArgs<T> a;
  memset(&a, 0, sizeof a);
  a.y = static_cast<const T*>(d_y);
  a.n = n;
  a.m = n - p;
  a.p = p;
  a.p_pad = pp;
  a.nlag = p;
  a.d = d_v;
  a.d_scale = 1.0;
  a.u_old = static_cast<const T*>(d_u_old);
  a.coef_host = c;
  a.u_new = static_cast<T*>(d_u_new);
  a.tail = TAIL_STORE;
  a.w = w;
  a.out_t = d_xtu;
  a.out_n2 = d_unorm2;
  return launch_pass<T>(a, kNoAllocGrid, stream) == cudaSuccess ? TOLS_OK : TOLS_ERR_CUDA;
}

}  // namespace

extern "C" int toeplitz_ols_gk_pass_noalloc(int precision, const void* d_y, long long n, int p, const double* d_v,
                                            const void* d_u_old, double c, void* d_u_new, double* d_xtu,
                                            double* d_unorm2, void* cuda_stream) {
  if (precision != TOLS_FP64 && precision != TOLS_MIXED) return TOLS_ERR_ARG;
  if (p < 1 || p > TOLS_NOALLOC_MAX_P || n <= p) return TOLS_ERR_ARG;
  if (!d_y || !d_v || !d_xtu || !d_unorm2) return TOLS_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TOLS_ERR_NO_DEVICE;
  void* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return TOLS_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (precision == TOLS_FP64) return run<double>(d_y, n, p, d_v, d_u_old, c, d_u_new, d_xtu, d_unorm2, s, scratch);
  return run<float>(d_y, n, p, d_v, d_u_old, c, d_u_new, d_xtu, d_unorm2, s, scratch);
}
