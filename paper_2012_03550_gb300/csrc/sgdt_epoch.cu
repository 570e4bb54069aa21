// Persistent epoch kernel: Algorithm 1 for every minibatch of a range.
//
// One cooperative launch holds G co-resident CTAs for the whole range.  Each
// minibatch (m samples) is split into G contiguous chunks of ceil(m/G) samples
// per phase; the phases are separated by grid barriers with a watchdog.
//
// Core phase (Algorithm 1 lines 1-15; Eq. 7, Eq. 15).  A is fixed during the
// phase, so each CTA gathers its samples' N factor rows once and keeps
//   p[s][k][r] = <a_k(s), b(k)_r>
// in shared memory.  For mode n the line-5 product W_r = H O_r has the closed
// form W_r[s] = a_n(s) * w[s][r], w[s][r] = prod_{k != n} p[s][k][r]
// (mixed-product property of the Kronecker product, Eq. 7), and the
// line-13 vector of column r after columns r' < r moved by Delta_{r'} is
//   V_r = g_r + sum_{r' < r} C_{r r'} Delta_{r'},
//   g_r = sum_s W_r[s] e_s,  C_{r r'} = sum_s W_r[s] W_{r'}[s]^T,
//   e_s = sum_r W_r[s].b_r - x_s at the start of the mode
// (exact algebra of lines 8-13: the residual of line 8-11 is e_s plus the
// moves already made).  So one grid-wide reduction of (g, C) per mode
// replaces R sequential reductions: every CTA writes its partial, CTA c sums
// a slice over all CTAs in a fixed order, and after a second barrier every
// CTA replays the R cyclic SGD steps (line 14) on the same numbers, so all
// CTAs hold bit-identical B without broadcasting it.
//
// Core rebuild (line 16, Eq. 4) is done redundantly by every CTA in shared
// memory.
//
// Factor phase (lines 17-25; Eqs. 10, 11, 18), mode after mode.  The samples
// come sorted by i_n (tiler), so each row's samples are one contiguous run.
// A warp per sample forms the Kronecker row S_s (Eq. 10, Def. 1 column order)
// and the contraction E_s = G_(n) S_s^T against the unfolded core, the
// residual e_s = a_n . E_s - x_s and the contribution e_s E_s (= the row's
// share of -X E^T + a E E^T, line 22).  Runs inside one chunk are summed and
// applied by the owning CTA; a run that crosses chunks is summed per chunk,
// and the last contributor (an atomic arrival count per run) adds the pieces
// in chunk order and applies the update, so the result does not depend on
// arrival order and no floating-point atomics are used.
#include "sgdt_internal.cuh"

namespace sgdt {

namespace {

struct SmemLayout {
  int B, G, GT, rows, p, w, e, v, x, red, delta, coords, seg, total_words;
};

__host__ __device__ inline SmemLayout smem_layout(const Geometry& g, int chunk_max, int payload_max) {
  SmemLayout L;
  int off = 0;
  auto take = [&](int words) {
    const int at = off;
    off += (words + 3) & ~3;   // 16-byte aligned sections
    return at;
  };
  int sumJR = 0;
  for (int n = 0; n < g.N; ++n) sumJR += g.J[n] * g.R;
  L.B = take(sumJR);
  L.G = take(g.prodJ);
  L.GT = take(g.prodJ);
  L.rows = take(chunk_max * g.sumJ);
  L.p = take(chunk_max * g.N * g.R);
  L.w = take(chunk_max * g.R);
  L.e = take(chunk_max);
  L.v = take(chunk_max * g.Jmax);
  L.x = take(chunk_max);
  L.red = take(payload_max);
  L.delta = take(g.R * kMaxJ);
  L.coords = take(chunk_max * g.N);
  L.seg = take(chunk_max);
  L.total_words = off;
  return L;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_int(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// Grid barrier over all CTAs of the cooperative launch.  The counter only
// grows; barrier k completes when it reaches k * G.  A wait longer than the
// watchdog budget (or an error raised by another CTA) makes every CTA return
// false; the host then reports STD_ETIMEOUT.
__device__ bool grid_barrier(const EpochArgs& a, unsigned long long& generation) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++generation;
    const unsigned long long target = generation * (unsigned long long)gridDim.x;
    __threadfence();
    atomicAdd(a.bar, 1ULL);
    const unsigned long long t0 = globaltimer_ns();
    int ok = 1;
    unsigned spins = 0;
    while (ld_acquire_u64(a.bar) < target) {
      if ((++spins & 63u) == 0u) {
        if (ld_volatile_int(a.err) != 0) { ok = 0; break; }
        if (globaltimer_ns() - t0 > a.watchdog_ns) {
          atomicCAS(a.err, 0, STD_ETIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Index (j <= jp) of the row-major upper triangle of a J x J matrix.
__device__ __forceinline__ int tri_index(int j, int jp, int J) {
  return j * J - (j * (j - 1)) / 2 + (jp - j);
}

}  // namespace

__global__ void __launch_bounds__(kEpochThreads)
k_epoch(EpochArgs a) {
  extern __shared__ __align__(16) float sm[];
  const Geometry& g = a.g;
  const int N = g.N, R = g.R;
  const SmemLayout L = smem_layout(g, a.chunk_max, a.payload_max);
  float* Bsm = sm + L.B;
  float* Gsm = sm + L.G;
  float* GT = sm + L.GT;
  float* rows = sm + L.rows;
  float* pbuf = sm + L.p;
  float* wbuf = sm + L.w;
  float* ebuf = sm + L.e;
  float* vbuf = sm + L.v;
  float* xbuf = sm + L.x;
  float* redsm = sm + L.red;
  float* delta = sm + L.delta;
  int* cbuf = reinterpret_cast<int*>(sm + L.coords);
  uint32_t* sgbuf = reinterpret_cast<uint32_t*>(sm + L.seg);

  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
  const int M = a.s.M;
  const int sumJ = g.sumJ, Jmax = g.Jmax;
  unsigned long long generation = 0;

  int sumJR = 0;
  for (int n = 0; n < N; ++n) sumJR += g.J[n] * R;
  for (int i = tid; i < sumJR; i += T) Bsm[i] = __ldcg(a.B + i);
  __syncthreads();

  for (int64_t b = a.b0; b < a.b1; ++b) {
    const int64_t t0 = b * (int64_t)M;
    const int m = (int)((a.s.n - t0) < (int64_t)M ? (a.s.n - t0) : (int64_t)M);
    const int chunk = (m + G - 1) / G;
    const int lo = c * chunk;
    const int hi = min(lo + chunk, m);
    const int cnt = hi > lo ? hi - lo : 0;
    const bool probe = (b == a.probe_batch);
    const float fm = (float)m;

    // ------------------------------------------------------------------
    // Core phase.  Samples: this CTA's chunk of the mode-1-sorted copy.
    // ------------------------------------------------------------------
    for (int i = tid; i < cnt * N; i += T) {
      const int s = i / N, k = i % N;
      cbuf[i] = __ldg(a.s.crd + ((size_t)0 * N + k) * a.s.npad + (size_t)(t0 + lo + s));
    }
    for (int s = tid; s < cnt; s += T) xbuf[s] = __ldg(a.s.val + (size_t)(t0 + lo + s));
    __syncthreads();
    for (int i = tid; i < cnt * sumJ; i += T) {
      const int s = i / sumJ;
      int jj = i % sumJ, k = 0;
      while (jj >= g.J[k]) { jj -= g.J[k]; ++k; }
      rows[i] = __ldcg(a.A[k] + (size_t)cbuf[s * N + k] * g.Jp[k] + jj);
    }
    __syncthreads();
    for (int i = tid; i < cnt * N * R; i += T) {
      const int s = i / (N * R), k = (i / R) % N, r = i % R;
      const float* ar = rows + s * sumJ + g.joff[k];
      const float* br = Bsm + g.boff[k] + r;
      float acc = 0.f;
      for (int j = 0; j < g.J[k]; ++j) acc = fmaf(ar[j], br[j * R], acc);
      pbuf[i] = acc;
    }
    __syncthreads();

    for (int n = 0; n < N; ++n) {
      const int Jn = g.J[n];
      const int Tn = Jn * (Jn + 1) / 2;
      const int P = R * Jn + (R * (R - 1) / 2) * Tn;
      // w[s][r] and the residual e_s at the start of mode n
      for (int s = tid; s < cnt; s += T) {
        float e = -xbuf[s];
        for (int r = 0; r < R; ++r) {
          float w = 1.f;
          for (int k = 0; k < N; ++k)
            if (k != n) w *= pbuf[(s * N + k) * R + r];
          wbuf[s * R + r] = w;
          e = fmaf(w, pbuf[(s * N + n) * R + r], e);
        }
        ebuf[s] = e;
      }
      __syncthreads();
      // CTA partial of (g, C)
      for (int o = tid; o < P; o += T) {
        float acc = 0.f;
        if (o < R * Jn) {
          const int r = o / Jn, j = o % Jn;
          for (int s = 0; s < cnt; ++s)
            acc = fmaf(ebuf[s] * wbuf[s * R + r], rows[s * sumJ + g.joff[n] + j], acc);
        } else {
          int q = o - R * Jn;
          int pair = q / Tn, t = q % Tn;
          int r = 1;
          while (pair >= r) { pair -= r; ++r; }
          const int rp = pair;
          int j = 0;
          while (t >= Jn - j) { t -= Jn - j; ++j; }
          const int jp = j + t;
          for (int s = 0; s < cnt; ++s) {
            const float* an = rows + s * sumJ + g.joff[n];
            acc = fmaf(wbuf[s * R + r] * wbuf[s * R + rp], an[j] * an[jp], acc);
          }
        }
        __stcg(a.part + (size_t)c * a.payload_max + o, acc);
      }
      if (!grid_barrier(a, generation)) return;
      // CTA c sums its slice of the payload over all CTAs (fixed order)
      {
        const int per = (P + G - 1) / G;
        const int o_lo = c * per, o_hi = min(o_lo + per, P);
        for (int o = o_lo + warp; o < o_hi; o += nwarps) {
          float acc = 0.f;
          for (int cc = lane; cc < G; cc += 32) acc += __ldcg(a.part + (size_t)cc * a.payload_max + o);
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
          if (lane == 0) __stcg(a.red + o, acc);
        }
      }
      if (!grid_barrier(a, generation)) return;
      for (int o = tid; o < P; o += T) redsm[o] = __ldcg(a.red + o);
      __syncthreads();
      // Cyclic SGD over the columns of B(n) (lines 7-14), replayed by every CTA
      if (warp == 0) {
        const float* gv = redsm;
        const float* Cv = redsm + R * Jn;
        float* Bn = Bsm + g.boff[n];
        for (int r = 0; r < R; ++r) {
          if (lane < Jn) {
            float V = gv[r * Jn + lane];
            for (int rp = 0; rp < r; ++rp) {
              const float* C = Cv + (r * (r - 1) / 2 + rp) * Tn;
              for (int jp = 0; jp < Jn; ++jp) {
                const int lo_j = min(lane, jp), hi_j = max(lane, jp);
                V = fmaf(C[tri_index(lo_j, hi_j, Jn)], delta[rp * kMaxJ + jp], V);
              }
            }
            const float bo = Bn[lane * R + r];
            const float bn = bo - a.lr_b * (V / fm + a.lam_b * bo);
            delta[r * kMaxJ + lane] = bn - bo;
            Bn[lane * R + r] = bn;
            if (probe && c == 0 && a.probeV) a.probeV[((size_t)n * R + r) * kMaxJ + lane] = V;
          }
          __syncwarp();
        }
      }
      __syncthreads();
      // p[s][n][r] with the new B(n)
      for (int i = tid; i < cnt * R; i += T) {
        const int s = i / R, r = i % R;
        const float* ar = rows + s * sumJ + g.joff[n];
        const float* br = Bsm + g.boff[n] + r;
        float acc = 0.f;
        for (int j = 0; j < Jn; ++j) acc = fmaf(ar[j], br[j * R], acc);
        pbuf[(s * N + n) * R + r] = acc;
      }
      __syncthreads();
    }

    // ------------------------------------------------------------------
    // G-hat from B (Eq. 4), mode 1 fastest.
    // ------------------------------------------------------------------
    for (int lin = tid; lin < g.prodJ; lin += T) {
      int jd[kMaxN];
      int t = lin;
      for (int k = 0; k < N; ++k) { jd[k] = t % g.J[k]; t /= g.J[k]; }
      float acc = 0.f;
      for (int r = 0; r < R; ++r) {
        float prod = 1.f;
        for (int k = 0; k < N; ++k) prod *= Bsm[g.boff[k] + jd[k] * R + r];
        acc += prod;
      }
      Gsm[lin] = acc;
    }
    __syncthreads();

    // ------------------------------------------------------------------
    // Factor phase, n = 1..N.
    // ------------------------------------------------------------------
    for (int n = 0; n < N; ++n) {
      const int Jn = g.J[n];
      const int Pn = g.prodJ / Jn;
      // G_(n) transposed: GT[c * Jn + j] = G-hat at (j_n = j, others = digits of column c)
      for (int i = tid; i < g.prodJ; i += T) {
        const int cc = i / Jn, j = i % Jn;
        int rem = cc, lin = j * g.gstride[n];
        for (int k = 0; k < N; ++k) {
          if (k == n) continue;
          lin += (rem % g.J[k]) * g.gstride[k];
          rem /= g.J[k];
        }
        GT[i] = Gsm[lin];
      }
      const size_t base = (size_t)(t0 + lo);
      for (int i = tid; i < cnt * N; i += T) {
        const int s = i / N, k = i % N;
        cbuf[i] = __ldg(a.s.crd + ((size_t)n * N + k) * a.s.npad + base + s);
      }
      for (int s = tid; s < cnt; s += T) {
        xbuf[s] = __ldg(a.s.val + (size_t)n * a.s.npad + base + s);
        sgbuf[s] = __ldg(a.s.seg + (size_t)n * a.s.npad + base + s);
      }
      __syncthreads();
      for (int i = tid; i < cnt * sumJ; i += T) {
        const int s = i / sumJ;
        int jj = i % sumJ, k = 0;
        while (jj >= g.J[k]) { jj -= g.J[k]; ++k; }
        rows[i] = __ldcg(a.A[k] + (size_t)cbuf[s * N + k] * g.Jp[k] + jj);
      }
      __syncthreads();
      // Gather-contract: one warp per sample
      for (int s = warp; s < cnt; s += nwarps) {
        const float* rs = rows + s * sumJ;
        float acc[kMaxJ];
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j) acc[j] = 0.f;
        for (int cc = lane; cc < Pn; cc += 32) {
          int rem = cc;
          float S = 1.f;
          for (int k = 0; k < N; ++k) {
            if (k == n) continue;
            S *= rs[g.joff[k] + rem % g.J[k]];
            rem /= g.J[k];
          }
          const float* gt = GT + cc * Jn;
#pragma unroll
          for (int j = 0; j < kMaxJ; ++j)
            if (j < Jn) acc[j] = fmaf(gt[j], S, acc[j]);
        }
        float e = -xbuf[s];
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j) {
          if (j < Jn) {
            float v = acc[j];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            v = __shfl_sync(0xffffffffu, v, 0);
            acc[j] = v;
            e = fmaf(rs[g.joff[n] + j], v, e);
          }
        }
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j)
          if (j < Jn && lane == j) vbuf[s * Jmax + j] = e * acc[j];
      }
      __syncthreads();
      // Segmented reduce of the contributions and the row updates (line 23)
      for (int s = warp; s < cnt; s += nwarps) {
        const uint32_t sg = sgbuf[s];
        const int st = (int)(sg & 0xffffu), en = (int)(sg >> 16);
        const int q = lo + s;
        if (!(q == lo || st == q)) continue;
        const int qend = min(en, hi - 1);
        float F = 0.f;
        if (lane < Jn)
          for (int q2 = q; q2 <= qend; ++q2) F += vbuf[(q2 - lo) * Jmax + lane];
        const int row = cbuf[s * N + n];
        bool apply = (st >= lo) && (en < hi);
        if (!apply) {
          const int slot = (st < lo) ? 0 : 1;
          if (lane < Jn) __stcg(a.bpart + ((size_t)c * 2 + slot) * kMaxJ + lane, F);
          __threadfence();
          __syncwarp();
          const int c0 = st / chunk, c1 = en / chunk;
          unsigned old = 0;
          if (lane == 0) old = atomicAdd(a.bcnt + c1, 1u);
          old = __shfl_sync(0xffffffffu, old, 0);
          if (old == (unsigned)(c1 - c0)) {
            __threadfence();
            if (lane < Jn) {
              F = __ldcg(a.bpart + ((size_t)c0 * 2 + 1) * kMaxJ + lane);
              for (int cc = c0 + 1; cc <= c1; ++cc) F += __ldcg(a.bpart + ((size_t)cc * 2 + 0) * kMaxJ + lane);
            }
            if (lane == 0) a.bcnt[c1] = 0u;
            apply = true;
          }
        }
        if (apply && lane < Jn) {
          const float denom = a.norm_mode == 1 ? (float)(en - st + 1) : fm;
          float* ap = a.A[n] + (size_t)row * g.Jp[n] + lane;
          const float av = __ldcg(ap);
          __stcg(ap, av - a.lr_a * (F / denom + a.lam_a * av));
          if (probe && a.probeF) a.probeF[((size_t)n * M + st) * kMaxJ + lane] = F;
        }
      }
      if (!grid_barrier(a, generation)) return;
    }
  }

  if (c == 0) {
    for (int i = tid; i < sumJR; i += T) a.B[i] = Bsm[i];
    for (int i = tid; i < g.prodJ; i += T) {
      int jd[kMaxN];
      int t = i;
      for (int k = 0; k < N; ++k) { jd[k] = t % g.J[k]; t /= g.J[k]; }
      float acc = 0.f;
      for (int r = 0; r < R; ++r) {
        float prod = 1.f;
        for (int k = 0; k < N; ++k) prod *= Bsm[g.boff[k] + jd[k] * R + r];
        acc += prod;
      }
      a.core[i] = acc;
    }
  }
}

size_t epoch_smem_bytes(const Geometry& g, int chunk_max, int payload_max) {
  return (size_t)smem_layout(g, chunk_max, payload_max).total_words * sizeof(float);
}

cudaError_t epoch_kernel_setup(size_t smem) {
  return cudaFuncSetAttribute(k_epoch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int epoch_max_ctas(size_t smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_epoch, kEpochThreads, smem) != cudaSuccess) return 0;
  return per * sms;
}

cudaError_t launch_epoch(const EpochArgs& a, int ctas, size_t smem, cudaStream_t st) {
  EpochArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)k_epoch, dim3(ctas), dim3(kEpochThreads), args, smem, st);
}

}  // namespace sgdt
