// Persistent epoch kernel: Algorithm 1 for every minibatch of a range.
//
// One cooperative launch holds G co-resident CTAs (one per SM) for the whole
// range.  Each minibatch (m samples) is split into G contiguous chunks of
// ceil(m/G) samples per phase; phases are separated by grid barriers with a
// watchdog.  The work inside a phase is organised for latency: few
// block-wide steps, per-sample reductions with warp shuffles, index tables
// built once per launch, and the next phase's schedule prefetched into a
// second shared-memory buffer while the current phase runs.
//
// Core phase (Algorithm 1 lines 1-15; Eq. 7, Eq. 15).  A is fixed during the
// phase: each CTA gathers its samples' N factor rows once and keeps
//   p[s][k][r] = <a_k(s), b(k)_r>.
// For mode n the line-5 product W_r = H O_r has the closed form
// W_r[s] = a_n(s) * w[s][r], w[s][r] = prod_{k != n} p[s][k][r] (mixed-product
// property of the Kronecker product, Eq. 7), and the line-13 vector of column
// r after columns r' < r moved by Delta_{r'} is
//   V_r = g_r + sum_{r' < r} C_{r r'} Delta_{r'},
//   g_r = sum_s W_r[s] e_s,  C_{r r'} = sum_s W_r[s] W_{r'}[s]^T,
//   e_s = sum_r W_r[s].b_r - x_s at the start of the mode,
// the exact algebra of lines 8-13 (the line 8-11 residual is e_s plus the moves
// already made).  One grid-wide reduction of (g, C) per mode replaces R
// sequential reductions: every CTA writes its partial, CTA c sums a slice
// over all CTAs in a fixed order, and after a second barrier every CTA
// replays the R cyclic SGD steps (line 14) as a block forward substitution on
// the same numbers, so all CTAs hold bit-identical B without a broadcast.
//
// Core rebuild (line 16, Eq. 4) is done redundantly by every CTA.
//
// Factor phase (lines 17-25; Eqs. 10, 11, 18), mode after mode, samples
// sorted by i_n (tiler) so that each row's samples form one run.  Per chunk:
// the Kronecker rows S_s (Eq. 10, Def. 1 column order) are built tile by
// tile in shared memory and contracted with the unfolded core,
// E_s = G_(n) S_s^T, by (sample, column-pair) register tiles; the residual
// e_s = a_n . E_s - x_s is reduced across each sample's lanes with shuffles,
// and the row sums F = sum_s e_s E_s (the row's -X E^T + a E E^T of line 22)
// come from segmented scans over the sorted samples.  Runs inside the chunk
// are applied by the owning CTA; a run that crosses chunks is summed per
// chunk and the last contributor (an acquire-release arrival count per run)
// adds the pieces in chunk order and applies the update, so the result does
// not depend on arrival order and no floating-point atomics are used.
#include "sgdt_internal.cuh"

namespace sgdt {

namespace {

constexpr int kCTile = 256;        // Kronecker-row columns per shared-memory tile
constexpr int kOutPerThread = 4;   // (sample, column-pair) tiles per thread

__host__ __device__ inline int pad4(int x) { return (x + 3) & ~3; }

__host__ __device__ inline int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

__host__ __device__ inline int max_pn(const Geometry& g) {
  int mx = 1;
  for (int n = 0; n < g.N; ++n) {
    const int pn = g.prodJ / g.J[n];
    if (pn > mx) mx = pn;
  }
  return mx;
}

__host__ __device__ inline int sum_pn(const Geometry& g) {
  int s = 0;
  for (int n = 0; n < g.N; ++n) s += g.prodJ / g.J[n];
  return s;
}

struct SmemLayout {
  int B, G, GT[2], ldig, coff, cdig, rowtab, rows, p, w, u, ww, aa, e, S, E, F, red, V, D;
  int crd[2], xs[2], seg[2], head, total_words;
};

__host__ __device__ inline SmemLayout smem_layout(const Geometry& g, int chunk, int payload) {
  SmemLayout L;
  int off = 0;
  auto take = [&](int words) {
    const int at = off;
    off += pad4(words);
    return at;
  };
  int sumJR = 0;
  for (int n = 0; n < g.N; ++n) sumJR += g.J[n] * g.R;
  const int Pmax = max_pn(g);
  const int tile = Pmax < kCTile ? pad4(Pmax) : kCTile;
  const int npairs = g.R * (g.R - 1) / 2;
  const int Tmax = g.Jmax * (g.Jmax + 1) / 2;
  const int gt = g.Jmax * pad4(Pmax);
  L.B = take(sumJR);
  L.G = take(g.prodJ);
  L.GT[0] = take(gt);
  L.GT[1] = take(gt);
  L.ldig = take(g.prodJ);
  L.coff = take(sum_pn(g));
  L.cdig = take(sum_pn(g));
  L.rowtab = take(g.sumJ);
  L.rows = take(chunk * g.sumJ);
  L.p = take(chunk * g.N * g.R);
  L.w = take(chunk * g.R);
  L.u = take(chunk * g.R);
  L.ww = take(chunk * (npairs > 0 ? npairs : 1));
  L.aa = take(chunk * Tmax);
  L.e = take(chunk);
  L.S = take(chunk * tile);
  L.E = take(chunk * g.Jmax);
  L.F = take(chunk * g.Jmax);
  L.red = take(payload);
  L.V = take(g.R * kMaxJ);
  L.D = take(kMaxJ);
  L.crd[0] = take(chunk * g.N);
  L.crd[1] = take(chunk * g.N);
  L.xs[0] = take(chunk);
  L.xs[1] = take(chunk);
  L.seg[0] = take(chunk);
  L.seg[1] = take(chunk);
  L.head = take(chunk + 1);
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

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_acq_rel_add_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ int ld_volatile_int(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

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
    red_release_add_u64(a.bar, 1ULL);
    int ok = 1;
    if (ld_acquire_u64(a.bar) < target) {
      const unsigned long long t0 = globaltimer_ns();
      unsigned spins = 0;
      while (ld_acquire_u64(a.bar) < target) {
        if ((++spins & 31u) == 0u) {
          if (ld_volatile_int(a.err) != 0) { ok = 0; break; }
          if (globaltimer_ns() - t0 > a.watchdog_ns) {
            atomicCAS(a.err, 0, STD_ETIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Index (j <= jp) of the row-major upper triangle of a J x J matrix.
__device__ __forceinline__ int tri_index(int j, int jp, int J) { return j * J - (j * (j - 1)) / 2 + (jp - j); }

struct Phase {
  int m, chunk, lo, hi, cnt;
};

__device__ __forceinline__ Phase phase_of(const EpochArgs& a, int64_t b) {
  Phase ph;
  const int M = a.s.M;
  const int64_t t0 = b * (int64_t)M;
  ph.m = (int)((a.s.n - t0) < (int64_t)M ? (a.s.n - t0) : (int64_t)M);
  ph.chunk = (ph.m + gridDim.x - 1) / gridDim.x;
  ph.lo = blockIdx.x * ph.chunk;
  ph.hi = min(ph.lo + ph.chunk, ph.m);
  ph.cnt = ph.hi > ph.lo ? ph.hi - ph.lo : 0;
  return ph;
}

// This CTA's chunk of the mode-`mode` sorted copy of minibatch b (coordinates
// [s][k], values, runs) into shared buffers.
__device__ __forceinline__ void load_schedule(const EpochArgs& a, int64_t b, int mode, int* crd, float* xs,
                                              uint32_t* seg) {
  const Phase ph = phase_of(a, b);
  const int N = a.g.N;
  const size_t base = (size_t)(b * (int64_t)a.s.M + ph.lo);
  for (int i = threadIdx.x; i < ph.cnt * N; i += blockDim.x) {
    const int k = i / ph.cnt, s = i - k * ph.cnt;
    crd[s * N + k] = __ldg(a.s.crd + ((size_t)mode * N + k) * a.s.npad + base + s);
  }
  for (int s = threadIdx.x; s < ph.cnt; s += blockDim.x) {
    xs[s] = __ldg(a.s.val + (size_t)mode * a.s.npad + base + s);
    seg[s] = __ldg(a.s.seg + (size_t)mode * a.s.npad + base + s);
  }
}

// The N factor rows of every sample of the chunk, with L2-coherent loads
// (rows may have been written by other CTAs in earlier phases).
__device__ __forceinline__ void load_rows(const EpochArgs& a, const int* crd, int cnt, const int* rowtab,
                                          float* rows) {
  const Geometry& g = a.g;
  const int N = g.N, sumJ = g.sumJ;
  for (int i = threadIdx.x; i < cnt * sumJ; i += blockDim.x) {
    const int s = i / sumJ, jj = i - s * sumJ;
    const int k = rowtab[jj] & 0xff, j = rowtab[jj] >> 8;
    rows[i] = __ldcg(a.A[k] + (size_t)crd[s * N + k] * g.Jp[k] + j);
  }
}

}  // namespace

__global__ void __launch_bounds__(kEpochThreads, 1)
k_epoch(EpochArgs a) {
  extern __shared__ __align__(16) float sm[];
  const Geometry& g = a.g;
  const int N = g.N, R = g.R;
  const SmemLayout L = smem_layout(g, a.chunk_max, a.payload_max);
  float* Bsm = sm + L.B;
  float* Gsm = sm + L.G;
  float* GTb[2] = {sm + L.GT[0], sm + L.GT[1]};
  uint32_t* ldig = reinterpret_cast<uint32_t*>(sm + L.ldig);
  int* coff = reinterpret_cast<int*>(sm + L.coff);
  uint32_t* cdig = reinterpret_cast<uint32_t*>(sm + L.cdig);
  int* rowtab = reinterpret_cast<int*>(sm + L.rowtab);
  float* rows = sm + L.rows;
  float* pbuf = sm + L.p;
  float* wbuf = sm + L.w;
  float* ubuf = sm + L.u;
  float* wwbuf = sm + L.ww;
  float* aabuf = sm + L.aa;
  float* ebuf = sm + L.e;
  float* Sbuf = sm + L.S;
  float* Ebuf = sm + L.E;
  float* Fbuf = sm + L.F;
  float* redsm = sm + L.red;
  float* Vsm = sm + L.V;
  float* Dsm = sm + L.D;
  int* crdb[2] = {reinterpret_cast<int*>(sm + L.crd[0]), reinterpret_cast<int*>(sm + L.crd[1])};
  float* xsb[2] = {sm + L.xs[0], sm + L.xs[1]};
  uint32_t* segb[2] = {reinterpret_cast<uint32_t*>(sm + L.seg[0]), reinterpret_cast<uint32_t*>(sm + L.seg[1])};
  int* head = reinterpret_cast<int*>(sm + L.head);

  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
  const int M = a.s.M;
  const int sumJ = g.sumJ, Jmax = g.Jmax;
  const int npairs = R * (R - 1) / 2;
  const int Rp = pow2_at_least(R);            // lanes per sample in the W step (<= 32)
  const int Pmax = max_pn(g);
  const int ctile_cap = Pmax < kCTile ? pad4(Pmax) : kCTile;
  unsigned long long generation = 0;

  // ---- tables built once per launch ----
  int sumJR = 0;
  for (int n = 0; n < N; ++n) sumJR += g.J[n] * R;
  for (int i = tid; i < sumJR; i += T) Bsm[i] = __ldcg(a.B + i);
  for (int lin = tid; lin < g.prodJ; lin += T) {
    int t = lin;
    uint32_t packed = 0;
    for (int k = 0; k < N; ++k) {
      packed |= (uint32_t)(t % g.J[k]) << (5 * k);
      t /= g.J[k];
    }
    ldig[lin] = packed;
  }
  {
    int base = 0;
    for (int n = 0; n < N; ++n) {
      const int Pn = g.prodJ / g.J[n];
      for (int cc = tid; cc < Pn; cc += T) {
        int rem = cc, off = 0, sh = 0;
        uint32_t packed = 0;
        for (int k = 0; k < N; ++k) {
          if (k == n) continue;
          const int d = rem % g.J[k];
          rem /= g.J[k];
          off += d * g.gstride[k];
          packed |= (uint32_t)d << sh;
          sh += 5;
        }
        coff[base + cc] = off;
        cdig[base + cc] = packed;
      }
      base += Pn;
    }
  }
  for (int jj = tid; jj < sumJ; jj += T) {
    int k = 0, j = jj;
    while (j >= g.J[k]) { j -= g.J[k]; ++k; }
    rowtab[jj] = k | (j << 8);
  }
  int buf = 0;
  if (a.b0 < a.b1) load_schedule(a, a.b0, 0, crdb[0], xsb[0], segb[0]);
  __syncthreads();

  for (int64_t b = a.b0; b < a.b1; ++b) {
    const Phase ph = phase_of(a, b);
    const int cnt = ph.cnt, lo = ph.lo, hi = ph.hi;
    const bool probe = (b == a.probe_batch);
    const float fm = (float)ph.m;

    // ------------------------------------------------------------------
    // Core phase on this CTA's chunk of the mode-1-sorted copy.
    // ------------------------------------------------------------------
    const int* crd = crdb[buf];
    const float* xs = xsb[buf];
    load_rows(a, crd, cnt, rowtab, rows);
    // factor mode 1's schedule does not depend on the model: fetch it now
    load_schedule(a, b, 0, crdb[buf ^ 1], xsb[buf ^ 1], segb[buf ^ 1]);
    __syncthreads();
    for (int i = tid; i < cnt * N * R; i += T) {
      const int s = i / (N * R), kr = i - s * (N * R), k = kr / R, r = kr - k * R;
      const float* ar = rows + s * sumJ + g.joff[k];
      const float* br = Bsm + g.boff[k] + r;
      float acc0 = 0.f, acc1 = 0.f;
      int j = 0;
      for (; j + 1 < g.J[k]; j += 2) {
        acc0 = fmaf(ar[j], br[j * R], acc0);
        acc1 = fmaf(ar[j + 1], br[(j + 1) * R], acc1);
      }
      if (j < g.J[k]) acc0 = fmaf(ar[j], br[j * R], acc0);
      pbuf[i] = acc0 + acc1;
    }
    __syncthreads();

    for (int n = 0; n < N; ++n) {
      const int Jn = g.J[n];
      const int Tn = Jn * (Jn + 1) / 2;
      const int P = R * Jn + npairs * Tn;
      // W step: lane group of Rp lanes per sample.  w[s][r], residual e_s
      // (segmented shuffle sum over r), u[s][r] = e_s w[s][r], ww = w_r w_r'.
      for (int i0 = 0; i0 < cnt * Rp; i0 += T) {
        const int i = i0 + tid;
        const int s = i / Rp, r = i - s * Rp;
        const bool live = (s < cnt) && (r < R);
        float w = 0.f, contrib = 0.f;
        if (live) {
          w = 1.f;
          for (int k = 0; k < N; ++k)
            if (k != n) w *= pbuf[(s * N + k) * R + r];
          contrib = w * pbuf[(s * N + n) * R + r];
        }
        for (int off = Rp >> 1; off > 0; off >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, off);
        if (live) {
          const float e = contrib - xs[s];
          wbuf[s * R + r] = w;
          ubuf[s * R + r] = e * w;
          if (r == 0) ebuf[s] = e;
        }
        // pairs (r, r') with r' < r: lane r pulls w_{r'} from its group
        for (int rp = 0; rp < Rp - 1; ++rp) {
          const float wr = __shfl_sync(0xffffffffu, w, (lane & ~(Rp - 1)) + rp);
          if (live && rp < r) wwbuf[s * npairs + r * (r - 1) / 2 + rp] = w * wr;
        }
      }
      for (int i = tid; i < cnt * Jn * Jn; i += T) {
        const int s = i / (Jn * Jn), jj = i - s * (Jn * Jn), j = jj / Jn, jp = jj - j * Jn;
        if (j <= jp) {
          const float* an = rows + s * sumJ + g.joff[n];
          aabuf[s * Tn + tri_index(j, jp, Jn)] = an[j] * an[jp];
        }
      }
      __syncthreads();
      // CTA partial of (g, C) in a fixed sample order
      for (int o = tid; o < P; o += T) {
        float acc0 = 0.f, acc1 = 0.f;
        if (o < R * Jn) {
          const int r = o / Jn, j = o - r * Jn;
          const float* an = rows + g.joff[n] + j;
          int s = 0;
          for (; s + 1 < cnt; s += 2) {
            acc0 = fmaf(ubuf[s * R + r], an[s * sumJ], acc0);
            acc1 = fmaf(ubuf[(s + 1) * R + r], an[(s + 1) * sumJ], acc1);
          }
          if (s < cnt) acc0 = fmaf(ubuf[s * R + r], an[s * sumJ], acc0);
        } else {
          const int q = o - R * Jn;
          const int pair = q / Tn, t = q - pair * Tn;
          int s = 0;
          for (; s + 1 < cnt; s += 2) {
            acc0 = fmaf(wwbuf[s * npairs + pair], aabuf[s * Tn + t], acc0);
            acc1 = fmaf(wwbuf[(s + 1) * npairs + pair], aabuf[(s + 1) * Tn + t], acc1);
          }
          if (s < cnt) acc0 = fmaf(wwbuf[s * npairs + pair], aabuf[s * Tn + t], acc0);
        }
        __stcg(a.part + (size_t)c * a.payload_max + o, acc0 + acc1);
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
      // Cyclic SGD over the columns of B(n) (lines 7-14) as a block forward
      // substitution in one warp: V_r starts at g_r; after column r moves by
      // Delta_r, every later V_r'' gains C_{r'' r} Delta_r.
      if (warp == 0) {
        float* Bn = Bsm + g.boff[n];
        const float* Cv = redsm + R * Jn;
        for (int i = lane; i < R * Jn; i += 32) Vsm[(i / Jn) * kMaxJ + i % Jn] = redsm[i];
        __syncwarp();
        for (int r = 0; r < R; ++r) {
          if (lane < Jn) {
            const float V = Vsm[r * kMaxJ + lane];
            const float bo = Bn[lane * R + r];
            const float bn = bo - a.lr_b * (V / fm + a.lam_b * bo);
            Dsm[lane] = bn - bo;
            Bn[lane * R + r] = bn;
            if (probe && c == 0 && a.probeV) a.probeV[((size_t)n * R + r) * kMaxJ + lane] = V;
          }
          __syncwarp();
          if (lane < Jn) {
            for (int r2 = r + 1; r2 < R; ++r2) {
              const float* C = Cv + (r2 * (r2 - 1) / 2 + r) * Tn;
              float acc0 = Vsm[r2 * kMaxJ + lane], acc1 = 0.f;
              int jp = 0;
              for (; jp + 1 < Jn; jp += 2) {
                acc0 = fmaf(C[tri_index(min(lane, jp), max(lane, jp), Jn)], Dsm[jp], acc0);
                acc1 = fmaf(C[tri_index(min(lane, jp + 1), max(lane, jp + 1), Jn)], Dsm[jp + 1], acc1);
              }
              if (jp < Jn) acc0 = fmaf(C[tri_index(min(lane, jp), max(lane, jp), Jn)], Dsm[jp], acc0);
              Vsm[r2 * kMaxJ + lane] = acc0 + acc1;
            }
          }
          __syncwarp();
        }
      }
      __syncthreads();
      // p[s][n][r] with the new B(n)
      for (int i = tid; i < cnt * R; i += T) {
        const int s = i / R, r = i - s * R;
        const float* ar = rows + s * sumJ + g.joff[n];
        const float* br = Bsm + g.boff[n] + r;
        float acc0 = 0.f, acc1 = 0.f;
        int j = 0;
        for (; j + 1 < Jn; j += 2) {
          acc0 = fmaf(ar[j], br[j * R], acc0);
          acc1 = fmaf(ar[j + 1], br[(j + 1) * R], acc1);
        }
        if (j < Jn) acc0 = fmaf(ar[j], br[j * R], acc0);
        pbuf[(s * N + n) * R + r] = acc0 + acc1;
      }
      __syncthreads();
    }
    buf ^= 1;

    // ------------------------------------------------------------------
    // G-hat from B (Eq. 4), mode 1 fastest, then G_(1) as [j][c].
    // ------------------------------------------------------------------
    for (int lin = tid; lin < g.prodJ; lin += T) {
      const uint32_t packed = ldig[lin];
      float acc = 0.f;
      for (int r = 0; r < R; ++r) {
        float prod = 1.f;
        for (int k = 0; k < N; ++k) prod *= Bsm[g.boff[k] + (int)((packed >> (5 * k)) & 31u) * R + r];
        acc += prod;
      }
      Gsm[lin] = acc;
    }
    __syncthreads();
    {
      const int Pn = g.prodJ / g.J[0], Pp = pad4(Pn);
      float* GT = GTb[0];
      for (int i = tid; i < g.J[0] * Pp; i += T) {
        const int j = i / Pp, cc = i - j * Pp;
        GT[i] = cc < Pn ? Gsm[coff[cc] + j * g.gstride[0]] : 0.f;
      }
    }
    __syncthreads();

    // ------------------------------------------------------------------
    // Factor phase, n = 1..N.
    // ------------------------------------------------------------------
    int toff = 0;   // offset of mode n's column tables
    for (int n = 0; n < N; ++n) {
      const int Jn = g.J[n];
      const int Pn = g.prodJ / Jn;
      const int Pp = pad4(Pn);
      const int* fcrd = crdb[buf];
      const float* fx = xsb[buf];
      const uint32_t* fseg = segb[buf];
      const float* GT = GTb[n & 1];
      const uint32_t* cdn = cdig + toff;
      // rows, and the run heads of this chunk compacted in order (warp 0)
      if (warp == 0) {
        int nh = 0;
        for (int s0 = 0; s0 < cnt; s0 += 32) {
          const int s = s0 + lane;
          bool is_head = false;
          if (s < cnt) is_head = (s == 0) || ((int)(fseg[s] & 0xffffu) == lo + s);
          const unsigned mask = __ballot_sync(0xffffffffu, is_head);
          if (is_head) head[nh + __popc(mask & ((1u << lane) - 1u))] = s;
          nh += __popc(mask);
        }
        if (lane == 0) head[cnt] = nh;
      }
      load_rows(a, fcrd, cnt, rowtab, rows);
      __syncthreads();
      const int nheads = head[cnt];
      // Gather-contract E_s = G_(n) S_s^T over Kronecker-row tiles.  Thread
      // tile (s, column pair); Tj lanes per sample.
      const int ntj = (Jn + 1) >> 1;
      const int Tj = pow2_at_least(ntj);
      const int nout = cnt * Tj;
      float acc[kOutPerThread][2];
#pragma unroll
      for (int q = 0; q < kOutPerThread; ++q) acc[q][0] = acc[q][1] = 0.f;
      for (int c0 = 0; c0 < Pp; c0 += ctile_cap) {
        const int ct = min(ctile_cap, Pp - c0);
        if (c0 > 0) __syncthreads();
        for (int i = tid; i < cnt * ct; i += T) {
          const int s = i / ct, cl = i - s * ct, cc = c0 + cl;
          float S = 0.f;
          if (cc < Pn) {
            const float* rs = rows + s * sumJ;
            uint32_t packed = cdn[cc];
            S = 1.f;
            for (int k = 0; k < N; ++k) {
              if (k == n) continue;
              S *= rs[g.joff[k] + (int)(packed & 31u)];
              packed >>= 5;
            }
          }
          Sbuf[s * ctile_cap + cl] = S;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kOutPerThread; ++q) {
          const int o = tid + q * T;
          const int s = o / Tj, jt = o - s * Tj;
          if (o < nout && jt < ntj) {
            const int j0 = 2 * jt;
            const float4* sv = reinterpret_cast<const float4*>(Sbuf + s * ctile_cap);
            const float4* g0 = reinterpret_cast<const float4*>(GT + j0 * Pp + c0);
            const float4* g1 = reinterpret_cast<const float4*>(GT + min(j0 + 1, Jn - 1) * Pp + c0);
            float a0 = acc[q][0], a1 = acc[q][1];
            for (int v = 0; v < (ct >> 2); ++v) {
              const float4 x = sv[v], y = g0[v], z = g1[v];
              a0 = fmaf(x.x, y.x, a0); a0 = fmaf(x.y, y.y, a0); a0 = fmaf(x.z, y.z, a0); a0 = fmaf(x.w, y.w, a0);
              a1 = fmaf(x.x, z.x, a1); a1 = fmaf(x.y, z.y, a1); a1 = fmaf(x.z, z.z, a1); a1 = fmaf(x.w, z.w, a1);
            }
            acc[q][0] = a0;
            acc[q][1] = a1;
          }
        }
      }
      // residual e_s = a_n . E_s - x_s (shuffle sum over the sample's Tj
      // lanes), then the contributions v = e_s E_s
#pragma unroll
      for (int q = 0; q < kOutPerThread; ++q) {
        const int o0 = q * T;
        if (o0 < nout) {   // uniform across the block
          const int o = tid + o0;
          const int s = o / Tj, jt = o - s * Tj;
          const bool live = (o < nout) && (jt < ntj);
          const int j0 = 2 * jt;
          float part = 0.f;
          if (live) {
            const float* an = rows + s * sumJ + g.joff[n];
            part = an[j0] * acc[q][0];
            if (j0 + 1 < Jn) part = fmaf(an[j0 + 1], acc[q][1], part);
          }
          for (int off = Tj >> 1; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
          if (live) {
            const float e = part - fx[s];
            Ebuf[s * Jmax + j0] = e * acc[q][0];
            if (j0 + 1 < Jn) Ebuf[s * Jmax + j0 + 1] = e * acc[q][1];
          }
        }
      }
      __syncthreads();
      // run sums: segmented inclusive scan of the contributions over the
      // sorted samples, one warp per column j, 32 samples at a time
      for (int j = warp; j < Jn; j += nwarps) {
        float carry = 0.f;
        int pieces = 0;
        for (int s0 = 0; s0 < cnt; s0 += 32) {
          const int s = s0 + lane;
          const bool valid = s < cnt;
          bool is_head = false;
          float x = 0.f;
          if (valid) {
            is_head = (s == 0) || ((int)(fseg[s] & 0xffffu) == lo + s);
            x = Ebuf[s * Jmax + j];
          }
          const unsigned hmask = __ballot_sync(0xffffffffu, is_head);
          const unsigned upto = hmask & (0xffffffffu >> (31 - lane));   // heads at lanes <= lane
          const int first = upto ? 31 - __clz(upto) : -1;              // latest head at or before lane
          if (lane == 0 && !is_head) x += carry;                       // run continued from the last block
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane - off >= (first < 0 ? 0 : first)) x += y;
          }
          // a piece ends at s when the next sample starts a run or the chunk ends
          bool ends = false;
          if (valid) {
            if (s + 1 >= cnt) ends = true;
            else ends = ((int)(fseg[s + 1] & 0xffffu) == lo + s + 1);
          }
          const int piece = pieces + __popc(upto) - 1;
          if (ends) Fbuf[piece * Jmax + j] = x;
          carry = __shfl_sync(0xffffffffu, x, 31);
          pieces += __popc(hmask);
        }
      }
      __syncthreads();
      // updates (line 23): runs inside the chunk directly; the first and last
      // pieces, when their runs cross chunk edges, through the arrival count
      for (int i = tid; i < nheads * Jn; i += T) {
        const int h = i / Jn, j = i - h * Jn;
        const int s0 = head[h];
        const uint32_t sg = fseg[s0];
        const int st = (int)(sg & 0xffffu), en = (int)(sg >> 16);
        if (st >= lo && en < hi) {
          const float F = Fbuf[h * Jmax + j];
          const float denom = a.norm_mode == 1 ? (float)(en - st + 1) : fm;
          float* ap = a.A[n] + (size_t)fcrd[s0 * N + n] * g.Jp[n] + j;
          const float av = __ldcg(ap);
          __stcg(ap, av - a.lr_a * (F / denom + a.lam_a * av));
          if (probe && a.probeF) a.probeF[((size_t)n * M + st) * kMaxJ + j] = F;
        }
      }
      if (warp < 2 && nheads > 0) {
        const int h = (warp == 0) ? 0 : nheads - 1;
        const int s0 = head[h];
        const uint32_t sg = fseg[s0];
        const int st = (int)(sg & 0xffffu), en = (int)(sg >> 16);
        const bool crosses = (st < lo) || (en >= hi);
        // warp 0 takes the first piece if its run began before the chunk;
        // warp 1 takes the last piece if its run began inside and continues
        const bool mine = crosses && ((warp == 0) ? (st < lo) : (st >= lo));
        if (mine) {
          const int slot = (st < lo) ? 0 : 1;
          if (lane < Jn) __stcg(a.bpart + ((size_t)c * 2 + slot) * kMaxJ + lane, Fbuf[h * Jmax + lane]);
          __threadfence();
          __syncwarp();
          const int c0 = st / ph.chunk, c1 = en / ph.chunk;
          unsigned old = 0;
          if (lane == 0) old = atom_acq_rel_add_u32(a.bcnt + c1, 1u);
          old = __shfl_sync(0xffffffffu, old, 0);
          if (old == (unsigned)(c1 - c0)) {
            __threadfence();
            if (lane < Jn) {
              float F = __ldcg(a.bpart + ((size_t)c0 * 2 + 1) * kMaxJ + lane);
              for (int cc = c0 + 1; cc <= c1; ++cc) F += __ldcg(a.bpart + ((size_t)cc * 2 + 0) * kMaxJ + lane);
              const float denom = a.norm_mode == 1 ? (float)(en - st + 1) : fm;
              float* ap = a.A[n] + (size_t)fcrd[s0 * N + n] * g.Jp[n] + lane;
              const float av = __ldcg(ap);
              __stcg(ap, av - a.lr_a * (F / denom + a.lam_a * av));
              if (probe && a.probeF) a.probeF[((size_t)n * M + st) * kMaxJ + lane] = F;
            }
            if (lane == 0) a.bcnt[c1] = 0u;
          }
        }
      }
      // meanwhile: the next phase's schedule and G_(n+1) as [j][c]
      if (warp >= 2 && n + 1 < N) {
        const int nt = T - 64, t2 = tid - 64;
        const int n1 = n + 1, Pn1 = g.prodJ / g.J[n1], Pp1 = pad4(Pn1);
        const int* cof1 = coff + toff + Pn;
        float* GT1 = GTb[n1 & 1];
        for (int i = t2; i < g.J[n1] * Pp1; i += nt) {
          const int j = i / Pp1, cc = i - j * Pp1;
          GT1[i] = cc < Pn1 ? Gsm[cof1[cc] + j * g.gstride[n1]] : 0.f;
        }
      }
      {
        const int64_t nb = (n + 1 < N) ? b : b + 1;
        const int nmode = (n + 1 < N) ? n + 1 : 0;
        if (nb < a.b1) load_schedule(a, nb, nmode, crdb[buf ^ 1], xsb[buf ^ 1], segb[buf ^ 1]);
      }
      buf ^= 1;
      toff += Pn;
      if (!grid_barrier(a, generation)) return;
    }
  }

  if (c == 0) {
    for (int i = tid; i < sumJR; i += T) a.B[i] = Bsm[i];
    for (int lin = tid; lin < g.prodJ; lin += T) {
      const uint32_t packed = ldig[lin];
      float acc = 0.f;
      for (int r = 0; r < R; ++r) {
        float prod = 1.f;
        for (int k = 0; k < N; ++k) prod *= Bsm[g.boff[k] + (int)((packed >> (5 * k)) & 31u) * R + r];
        acc += prod;
      }
      a.core[lin] = acc;
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
