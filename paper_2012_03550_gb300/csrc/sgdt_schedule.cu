// Minibatch sampler, COO gather and per-mode tiler (one CTA per minibatch).
//
// The paper draws each minibatch Psi at random from the nonzeros (Sec. 3.2,
// Eq. 3; input of Algorithm 1) and keeps a single COO copy of the tensor,
// grouping the samples of Psi that share a factor row when updating A(n)
// (Sec. 4.4.2).  Here every minibatch of the epoch is prepared up front, in
// parallel, because none of this depends on the model:
//   1. sampler: positions t of the minibatch -> training entries pi_e(t);
//   2. gather: the entries' coordinates and values from the library's COO;
//   3. tiler: for each mode n, a stable sort of the minibatch by i_n (keys
//      (i_n, batch position), unique, sorted by an in-shared-memory bitonic
//      network) and, for every sorted position, the first and last sorted
//      position of its run of equal i_n;
//   4. links: for every sorted position of the mode-n copy and every k < n,
//      the start of the mode-k run holding the same sample, i.e. the slot
//      under which the epoch kernel publishes that sample's updated mode-k
//      row during the minibatch.
// The sorted copies let each phase of the epoch kernel stream its samples
// contiguously and find the rows it owns without atomics.
#include "sgdt_internal.cuh"

namespace sgdt {

__global__ void __launch_bounds__(kScheduleThreads)
k_schedule(Geometry g, const uint32_t* __restrict__ coo, int cs, Feistel f, Schedule s, int64_t b0) {
  extern __shared__ unsigned long long sm_keys[];
  const int M = s.M;
  int L = 1;
  while (L < M) L <<= 1;
  unsigned long long* keys = sm_keys;                       // L entries
  int32_t* sid = reinterpret_cast<int32_t*>(keys + L);     // M entries

  const int64_t b = b0 + blockIdx.x;
  const int64_t t0 = b * (int64_t)M;
  const int64_t tb = s.b_first * (int64_t)M;   // storage index = position - tb
  const int m = (int)((s.n - t0) < (int64_t)M ? (s.n - t0) : (int64_t)M);

  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    const uint64_t y = feistel_perm(f, (uint64_t)(t0 + q));
    sid[q] = (int32_t)y;
    s.sid[t0 + q - tb] = (int32_t)y;
  }
  __syncthreads();

  for (int n = 0; n < g.N; ++n) {
    for (int q = threadIdx.x; q < L; q += blockDim.x) {
      if (q < m) {
        const uint32_t i = coo[(size_t)sid[q] * cs + n];
        keys[q] = ((unsigned long long)i << 32) | (unsigned long long)(uint32_t)q;
      } else {
        keys[q] = ~0ULL;
      }
    }
    __syncthreads();
    // Bitonic sorting network, ascending; keys are unique so the result is
    // the stable order by i_n.
    for (int k = 2; k <= L; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long x = keys[i], y = keys[ixj];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              keys[i] = y;
              keys[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
      const unsigned long long kq = keys[q];
      const uint32_t i = (uint32_t)(kq >> 32);
      const int pos = (int)(uint32_t)(kq & 0xffffffffULL);
      int lo = 0, hi = q;          // first sorted position with index i
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((uint32_t)(keys[mid] >> 32) < i) lo = mid + 1; else hi = mid;
      }
      const int start = lo;
      lo = q; hi = m - 1;          // last sorted position with index i
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((uint32_t)(keys[mid] >> 32) > i) hi = mid - 1; else lo = mid;
      }
      const int end = lo;
      const uint32_t* e = coo + (size_t)sid[pos] * cs;
      const size_t t = (size_t)(t0 + q - tb);
      for (int k = 0; k < g.N; ++k) s.crd[((size_t)n * g.N + k) * s.npad + t] = (int32_t)e[k];
      s.val[(size_t)n * s.npad + t] = __uint_as_float(e[g.N]);
      s.pos[(size_t)n * s.npad + t] = pos;
      s.seg[(size_t)n * s.npad + t] = (uint32_t)start | ((uint32_t)end << 16);
      if (n + 1 < g.N) s.rsp[(size_t)n * s.npad + (size_t)(t0 + pos - tb)] = start;
      // modes k < n were sorted in earlier passes of this CTA, which wrote
      // rsp[k]; the pass-ending __syncthreads orders those writes before
      // these reads
      for (int k = 0; k < n; ++k)
        s.link[(size_t)(n * (n - 1) / 2 + k) * s.npad + t] = s.rsp[(size_t)k * s.npad + (size_t)(t0 + pos - tb)];
    }
    __syncthreads();
  }
}

cudaError_t launch_schedule(const Geometry& g, const uint32_t* coo, int cs, const Feistel& f,
                            const Schedule& s, int64_t b0, int64_t b1, cudaStream_t st) {
  if (b1 <= b0) return cudaSuccess;
  int L = 1;
  while (L < s.M) L <<= 1;
  const size_t smem = (size_t)L * sizeof(unsigned long long) + (size_t)s.M * sizeof(int32_t);
  cudaError_t e = cudaFuncSetAttribute(k_schedule, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t nb = b1 - b0;
  for (int64_t off = 0; off < nb; off += 2147483647LL) {
    const int64_t cnt = (nb - off) < 2147483647LL ? (nb - off) : 2147483647LL;
    k_schedule<<<(unsigned)cnt, kScheduleThreads, smem, st>>>(g, coo, cs, f, s, b0 + off);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sgdt
