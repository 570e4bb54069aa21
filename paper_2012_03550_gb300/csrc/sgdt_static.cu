// std_rmse_static: the RMSE/MAE reduction for callers that cannot allocate
// device memory.
//
// Some callers cannot let a library call cudaMalloc: a serving process whose
// device memory is entirely reserved by its own pool allocator, or a
// latency-critical loop that must not pay for cudaMalloc/cudaFree (cudaFree
// synchronises the whole device).  For them this file offers one entry point
// that allocates nothing: the caller passes the model and the entries
// already in device memory plus a device output, and the only scratch (the
// per-block partial sums) lives in a file-scope __device__ array of fixed
// size, present on every GPU that loads the library until the process exits.
#include <cmath>
#include <mutex>
#include <string>

#include "sgdt_internal.cuh"

namespace sgdt {
namespace {

constexpr int kStaticThreads = 256;

// Per-block (sum of squares, sum of absolute values) partials: 2 doubles per
// block, STD_STATIC_RMSE_BLOCKS blocks (16 KiB).  Shared by every call.
static __device__ __align__(256) double g_rmse_scratch[2 * STD_STATIC_RMSE_BLOCKS];

struct StaticArgs {
  Geometry g;
  const float* A[kMaxN];   // caller's factor matrices, I_n x J_n row-major
  const float* B[kMaxN];   // caller's Kruskal matrices, J_n x R row-major
  const int32_t* coords;
  const float* values;
  int64_t k;
};

// Same arithmetic as the context's prediction/RMSE kernel: x-hat =
// sum_r prod_n <a(n)_{i_n}, b(n)_r>, FP64 sums of (x - x-hat)^2 and
// |x - x-hat| per block in a fixed tree order.  An index outside [0, I_n)
// contributes NaN to both sums (the bounds are checked before any read), so
// both results are NaN.
__global__ void __launch_bounds__(kStaticThreads)
k_rmse_static(StaticArgs a, double* __restrict__ scratch) {
  extern __shared__ float Bs[];
  const Geometry& g = a.g;
  for (int n = 0; n < g.N; ++n)
    for (int i = threadIdx.x; i < g.J[n] * g.R; i += blockDim.x) Bs[g.boff[n] + i] = a.B[n][i];
  __syncthreads();
  double se = 0.0, ae = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.k; i += (int64_t)gridDim.x * blockDim.x) {
    const float* rows[kMaxN];
    bool ok = true;
    for (int n = 0; n < g.N; ++n) {
      const int32_t v = a.coords[(size_t)i * g.N + n];
      if (v < 0 || (int64_t)v >= g.I[n]) { ok = false; rows[n] = nullptr; }
      else rows[n] = a.A[n] + (size_t)v * g.J[n];
    }
    if (!ok) {
      const double nan = __longlong_as_double(0x7ff8000000000000LL);
      se += nan;
      ae += nan;
      continue;
    }
    float xhat = 0.f;
    for (int r = 0; r < g.R; ++r) {
      float prod = 1.f;
      for (int n = 0; n < g.N; ++n) {
        const float* br = Bs + g.boff[n] + r;
        float dot = 0.f;
        for (int j = 0; j < g.J[n]; ++j) dot = fmaf(rows[n][j], br[j * g.R], dot);
        prod *= dot;
      }
      xhat += prod;
    }
    const double d = (double)a.values[i] - (double)xhat;
    se += d * d;
    ae += fabs(d);
  }
  __shared__ double red_se[kStaticThreads / 32], red_ae[kStaticThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    se += __shfl_down_sync(0xffffffffu, se, off);
    ae += __shfl_down_sync(0xffffffffu, ae, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red_se[warp] = se; red_ae[warp] = ae; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < kStaticThreads / 32; ++w) { s1 += red_se[w]; s2 += red_ae[w]; }
    scratch[2 * blockIdx.x] = s1;
    scratch[2 * blockIdx.x + 1] = s2;
  }
}

// Sums the `blocks` partials of this call in a fixed order; out = {rmse, mae}.
__global__ void k_rmse_static_finish(const double* __restrict__ scratch, int blocks, int64_t k,
                                     double* __restrict__ out) {
  __shared__ double s1[256], s2[256];
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < blocks; i += blockDim.x) { x += scratch[2 * i]; y += scratch[2 * i + 1]; }
  s1[threadIdx.x] = x;
  s2[threadIdx.x] = y;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) { s1[threadIdx.x] += s1[threadIdx.x + w]; s2[threadIdx.x] += s2[threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = k > 0 ? sqrt(s1[0] / (double)k) : 0.0;
    out[1] = k > 0 ? s2[0] / (double)k : 0.0;
  }
}

// Device address of g_rmse_scratch, looked up once per device with that
// device current (the host-side name of the array is only a stand-in).  The
// address is cached for the life of the process: it belongs to the device's
// primary context, so after cudaDeviceReset it is stale and this entry point
// must not be called again in that process.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

cudaError_t static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_rmse_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

int static_fail(int code, const std::string& msg) { return record_error(code, "std_rmse_static: " + msg); }

}  // namespace
}  // namespace sgdt

extern "C" int std_rmse_static(int32_t order, const int64_t* mode_sizes, const int32_t* ranks, int32_t r_core,
                               const float* const* A, const float* const* B, int64_t k, const int32_t* coords,
                               const float* values, double* out, void* stream) {
  using namespace sgdt;
  if (order < 2 || order > STD_MAX_ORDER) return static_fail(STD_EUNSUPPORTED, "order outside [2, STD_MAX_ORDER]");
  if (r_core < 1 || r_core > STD_MAX_RANK) return static_fail(STD_EUNSUPPORTED, "r_core outside [1, STD_MAX_RANK]");
  if (!mode_sizes || !ranks || !A || !B || !out) return static_fail(STD_EINVAL, "NULL argument");
  if (k < 0) return static_fail(STD_EINVAL, "k must be >= 0");
  if (k > 0 && (!coords || !values)) return static_fail(STD_EINVAL, "NULL coords or values");
  StaticArgs a{};
  a.g.N = order;
  a.g.R = r_core;
  int boff = 0;
  for (int n = 0; n < order; ++n) {
    if (ranks[n] < 1 || ranks[n] > STD_MAX_RANK) return static_fail(STD_EUNSUPPORTED, "rank outside [1, STD_MAX_RANK]");
    if (mode_sizes[n] < 1) return static_fail(STD_EINVAL, "mode size must be >= 1");
    if (!A[n] || !B[n]) return static_fail(STD_EINVAL, "NULL factor or Kruskal matrix");
    a.g.J[n] = ranks[n];
    a.g.I[n] = mode_sizes[n];
    a.g.boff[n] = boff;
    boff += ranks[n] * r_core;
    a.A[n] = A[n];
    a.B[n] = B[n];
  }
  a.coords = coords;
  a.values = values;
  a.k = k;
  double* scratch = nullptr;
  cudaError_t e = static_scratch(&scratch);
  if (e != cudaSuccess) return static_fail(STD_ECUDA, std::string("scratch address: ") + cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t want = (k + kStaticThreads - 1) / kStaticThreads;
  const int blocks = (int)(want < STD_STATIC_RMSE_BLOCKS ? want : STD_STATIC_RMSE_BLOCKS);
  if (blocks > 0) {
    k_rmse_static<<<blocks, kStaticThreads, (size_t)boff * sizeof(float), st>>>(a, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(STD_ECUDA, std::string("rmse kernel: ") + cudaGetErrorString(e));
  }
  k_rmse_static_finish<<<1, 256, 0, st>>>(scratch, blocks, k, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(STD_ECUDA, std::string("rmse finish: ") + cudaGetErrorString(e));
  return STD_OK;
}
