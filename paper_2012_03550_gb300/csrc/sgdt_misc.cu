// Small kernels around the epoch kernel: COO packing and index validation,
// parameter initialisation, the core rebuild of Eq. 4, and the prediction /
// RMSE-MAE reduction of Eq. 19.
#include <cmath>

#include <cuda_bf16.h>

#include "sgdt_internal.cuh"

namespace sgdt {

// COO (k x N int32 + float values) -> library layout: one record of `cs`
// 32-bit words per nonzero, [i_1 .. i_N, bits(value), padding], so that one
// nonzero is one aligned 16- or 32-byte load.  Indices outside [0, I_n) set
// *err and are clamped to 0 so no later kernel reads out of bounds.
__global__ void k_pack_coo(Geometry g, const int32_t* __restrict__ coords, const float* __restrict__ values,
                           int64_t k, uint32_t* __restrict__ coo, int cs, int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t* rec = coo + (size_t)i * cs;
    for (int n = 0; n < g.N; ++n) {
      int32_t v = coords[(size_t)i * g.N + n];
      if (v < 0 || (int64_t)v >= g.I[n]) {
        atomicExch(err, STD_EINVAL);
        v = 0;
      }
      rec[n] = (uint32_t)v;
    }
    rec[g.N] = __float_as_uint(values[i]);
    for (int w = g.N + 1; w < cs; ++w) rec[w] = 0u;
  }
}

__global__ void k_check_coords(Geometry g, const int32_t* __restrict__ coords, int64_t k, int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    for (int n = 0; n < g.N; ++n) {
      const int32_t v = coords[(size_t)i * g.N + n];
      if (v < 0 || (int64_t)v >= g.I[n]) atomicExch(err, STD_EINVAL);
    }
}

// Counter-based normal draws: SplitMix64 of (seed, stream, index) -> two
// uniforms in (0, 1] -> Box-Muller.
__device__ __forceinline__ double normal_draw(uint64_t seed, uint64_t stream, uint64_t idx) {
  const uint64_t z1 = splitmix_out(seed ^ splitmix_out(stream * 0x9E3779B97F4A7C15ULL + 2ULL * idx + 1ULL));
  const uint64_t z2 = splitmix_out(seed ^ splitmix_out(stream * 0x9E3779B97F4A7C15ULL + 2ULL * idx + 2ULL));
  const double u1 = ((double)(z1 >> 11) + 1.0) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(z2 >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

__global__ void k_init_factor(float* A, int64_t I, int J, int Jp, int mode, double mu, double sigma,
                              uint64_t seed, uint64_t stream) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I * Jp; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / Jp;
    const int j = (int)(i % Jp);
    float v = 0.f;
    if (j < J) {
      const double z = normal_draw(seed, stream, (uint64_t)(row * J + j));
      v = (float)(mode == 0 ? mu + sigma * z : z / sqrt((double)J));
    }
    A[i] = v;
  }
}

__global__ void k_init_kruskal(float* B, Geometry g, int mode, double mu, double sigma, uint64_t seed) {
  for (int n = 0; n < g.N; ++n)
    for (int i = threadIdx.x; i < g.J[n] * g.R; i += blockDim.x) {
      const double z = normal_draw(seed, 1000ULL + (uint64_t)n, (uint64_t)i);
      B[g.boff[n] + i] = (float)(mode == 0 ? mu + sigma * z : z / sqrt((double)g.J[n]));
    }
}

// G-hat = sum_r b(1)_r o ... o b(N)_r (Eq. 4), mode 1 fastest.
__global__ void k_build_core(Geometry g, const float* __restrict__ B, float* __restrict__ core) {
  for (int lin = blockIdx.x * blockDim.x + threadIdx.x; lin < g.prodJ; lin += gridDim.x * blockDim.x) {
    int jd[kMaxN];
    int t = lin;
    for (int k = 0; k < g.N; ++k) { jd[k] = t % g.J[k]; t /= g.J[k]; }
    float acc = 0.f;
    for (int r = 0; r < g.R; ++r) {
      float prod = 1.f;
      for (int k = 0; k < g.N; ++k) prod *= B[g.boff[k] + jd[k] * g.R + r];
      acc += prod;
    }
    core[lin] = acc;
  }
}

// Prediction x-hat = sum_r prod_n <a(n)_{i_n}, b(n)_r> at k coordinates — the
// Tucker model of Def. 6 with the Kruskal core of Eq. 4 contracted mode by
// mode.  With `values`, also the FP64 sums of (x - x-hat)^2 and |x - x-hat|
// per block (fixed tree order), finished by k_rmse_finish.
constexpr int kPredictThreads = 256;

__global__ void __launch_bounds__(kPredictThreads)
k_predict(Geometry g, AParams A, const float* __restrict__ B, const int32_t* __restrict__ coords,
          const float* __restrict__ values, int64_t k, float* __restrict__ out, double* __restrict__ partials,
          int* err) {
  extern __shared__ float Bs[];
  int sumJR = 0;
  for (int n = 0; n < g.N; ++n) sumJR += g.J[n] * g.R;
  for (int i = threadIdx.x; i < sumJR; i += blockDim.x) Bs[i] = B[i];
  __syncthreads();
  double se = 0.0, ae = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    const float* rows[kMaxN];
    bool ok = true;
    for (int n = 0; n < g.N; ++n) {
      const int32_t v = coords[(size_t)i * g.N + n];
      if (v < 0 || (int64_t)v >= g.I[n]) { ok = false; rows[n] = nullptr; }
      else rows[n] = A.A[n] + (size_t)v * g.Jp[n];
    }
    if (!ok) {
      atomicExch(err, STD_EINVAL);
      if (out) out[i] = __int_as_float(0x7fc00000);
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
    if (out) out[i] = xhat;
    if (values) {
      const double d = (double)values[i] - (double)xhat;
      se += d * d;
      ae += fabs(d);
    }
  }
  if (partials) {
    __shared__ double red_se[kPredictThreads / 32], red_ae[kPredictThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
      se += __shfl_down_sync(0xffffffffu, se, off);
      ae += __shfl_down_sync(0xffffffffu, ae, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red_se[warp] = se; red_ae[warp] = ae; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s1 = 0.0, s2 = 0.0;
      for (int w = 0; w < kPredictThreads / 32; ++w) { s1 += red_se[w]; s2 += red_ae[w]; }
      partials[2 * blockIdx.x] = s1;
      partials[2 * blockIdx.x + 1] = s2;
    }
  }
}

__global__ void k_rmse_finish(const double* __restrict__ partials, int blocks, double* __restrict__ result) {
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < blocks; i += blockDim.x) { a += partials[2 * i]; b += partials[2 * i + 1]; }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) { s1[threadIdx.x] += s1[threadIdx.x + w]; s2[threadIdx.x] += s2[threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { result[0] = s1[0]; result[1] = s2[0]; }
}

// BF16 mirror of an FP32 factor matrix (round to nearest even; padding 0).
__global__ void k_mirror_bf16(const float* __restrict__ A, uint16_t* __restrict__ Ab, int64_t I, int J, int Jp,
                              int Jb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I * Jb; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / Jb;
    const int j = (int)(i - row * Jb);
    Ab[i] = j < J ? __bfloat16_as_ushort(__float2bfloat16_rn(A[row * Jp + j])) : (uint16_t)0;
  }
}

static int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}

cudaError_t launch_pack_coo(const Geometry& g, const int32_t* coords, const float* values, int64_t k,
                            uint32_t* coo, int cs, int* err, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  k_pack_coo<<<grid_for(k, 256), 256, 0, st>>>(g, coords, values, k, coo, cs, err);
  return cudaGetLastError();
}

cudaError_t launch_check_coords(const Geometry& g, const int32_t* coords, int64_t k, int* err, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  k_check_coords<<<grid_for(k, 256), 256, 0, st>>>(g, coords, k, err);
  return cudaGetLastError();
}

cudaError_t launch_init_params(const Geometry& g, float* const* A, float* B, int mode, double mu,
                               double sigma, uint64_t seed, cudaStream_t st) {
  for (int n = 0; n < g.N; ++n) {
    k_init_factor<<<grid_for(g.I[n] * g.Jp[n], 256), 256, 0, st>>>(A[n], g.I[n], g.J[n], g.Jp[n], mode, mu,
                                                                   sigma, seed, (uint64_t)n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_init_kruskal<<<1, 256, 0, st>>>(B, g, mode, mu, sigma, seed);
  return cudaGetLastError();
}

cudaError_t launch_mirror_bf16(const Geometry& g, float* const* A, uint16_t* const* Ab, cudaStream_t st) {
  for (int n = 0; n < g.N; ++n) {
    if (!Ab[n]) continue;
    k_mirror_bf16<<<grid_for(g.I[n] * g.Jb[n], 256), 256, 0, st>>>(A[n], Ab[n], g.I[n], g.J[n], g.Jp[n], g.Jb[n]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_build_core(const Geometry& g, const float* B, float* core, cudaStream_t st) {
  k_build_core<<<grid_for(g.prodJ, 256), 256, 0, st>>>(g, B, core);
  return cudaGetLastError();
}

int predict_blocks(int64_t k) { return grid_for(k, kPredictThreads) > 1184 ? 1184 : grid_for(k, kPredictThreads); }

cudaError_t launch_predict(const Geometry& g, const AParams& A, const float* B, const int32_t* coords,
                           const float* values, int64_t k, float* out, double* partials, int blocks,
                           int* err, cudaStream_t st) {
  int sumJR = 0;
  for (int n = 0; n < g.N; ++n) sumJR += g.J[n] * g.R;
  k_predict<<<blocks, kPredictThreads, (size_t)sumJR * sizeof(float), st>>>(g, A, B, coords, values, k, out,
                                                                             partials, err);
  return cudaGetLastError();
}

// Predictions for several contexts in one launch: thread per query of the
// concatenated list, which finds its context by binary search over the
// items' offsets; the arithmetic is k_predict's, term for term, so each
// result equals that context's own std_predict.
__global__ void __launch_bounds__(kPredictThreads)
k_predict_multi(const PredictItem* __restrict__ items, int count, int64_t total, int* err) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].off <= q) lo = mid;
      else hi = mid - 1;
    }
    const PredictItem& it = items[lo];
    const Geometry& g = it.g;
    const int64_t i = q - it.off;
    const float* rows[kMaxN];
    bool ok = true;
    for (int n = 0; n < g.N; ++n) {
      const int32_t v = it.coords[(size_t)i * g.N + n];
      if (v < 0 || (int64_t)v >= g.I[n]) { ok = false; rows[n] = nullptr; }
      else rows[n] = it.A.A[n] + (size_t)v * g.Jp[n];
    }
    if (!ok) {
      atomicExch(err, STD_EINVAL);
      it.out[i] = __int_as_float(0x7fc00000);
      continue;
    }
    float xhat = 0.f;
    for (int r = 0; r < g.R; ++r) {
      float prod = 1.f;
      for (int n = 0; n < g.N; ++n) {
        const float* br = it.B + g.boff[n] + r;
        float dot = 0.f;
        for (int j = 0; j < g.J[n]; ++j) dot = fmaf(rows[n][j], br[j * g.R], dot);
        prod *= dot;
      }
      xhat += prod;
    }
    it.out[i] = xhat;
  }
}

cudaError_t launch_predict_multi(const PredictItem* items, int count, int64_t total, int* err, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  k_predict_multi<<<predict_blocks(total), kPredictThreads, 0, st>>>(items, count, total, err);
  return cudaGetLastError();
}

cudaError_t launch_rmse_finish(const double* partials, int blocks, double* result, cudaStream_t st) {
  k_rmse_finish<<<1, 256, 0, st>>>(partials, blocks, result);
  return cudaGetLastError();
}

}  // namespace sgdt
