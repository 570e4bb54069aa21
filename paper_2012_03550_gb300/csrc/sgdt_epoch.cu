// Persistent epoch kernel: Algorithm 1 for every minibatch of a range.
//
// One cooperative launch holds G co-resident CTAs (one per SM) for the whole
// range.  Each minibatch (m samples) is split into G contiguous chunks of
// ceil(m/G) samples per phase; phases are separated by grid barriers with a
// watchdog.  The kernel is instantiated per order N so that every loop over
// modes unrolls; the work inside a phase is a handful of block-wide steps
// (small register-tiled products over the chunk's samples, warp-shuffle
// reductions per sample), and the next phase's schedule is prefetched into a
// second shared-memory buffer while the current phase runs.
//
// Core phase (Algorithm 1 lines 1-15; Eq. 7, Eq. 15).  A is fixed during the
// phase: each CTA gathers its samples' N factor rows once and keeps
//   p[s][k][r] = <a_k(s), b(k)_r>.
// For mode n the line-5 product W_r = H O_r has the closed form
// W_r[s] = a_n(s) * w[s][r], w[s][r] = prod_{k != n} p[s][k][r] (mixed-product
// property of the Kronecker product, Eq. 7), i.e. the rows of all W_r together
// are Y_s = w_s (x) a_n(s) (length R*J_n).  The line-13 vector of column r
// after columns r' < r moved by Delta_{r'} is
//   V_r = g_r + sum_{r' < r} C_{r r'} Delta_{r'},
//   g_r = sum_s W_r[s] e_s,  C_{r r'} = sum_s W_r[s] W_{r'}[s]^T,
//   e_s = sum_r W_r[s].b_r - x_s at the start of the mode,
// the exact algebra of lines 8-13 (the line 8-11 residual is e_s plus the moves
// already made).  So g and the blocks C_{r r'} (r' < r) are parts of the Gram
// matrix of [Y | e] over the samples: one register-tiled product per CTA, one
// grid-wide reduction per mode (every CTA writes its partial, CTA c sums a
// slice over all CTAs in a fixed order), and after a second barrier every CTA
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
#include <cuda_bf16.h>

#include "sgdt_internal.cuh"

namespace sgdt {

namespace {

constexpr int kCTile = 256;        // Kronecker-row columns per shared-memory tile
constexpr int kOutPerThread = 2;   // (sample, column pair, half) tiles per thread

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

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Row stride (in BF16 elements) of the Kronecker-row and unfolded-core tiles
// of the tensor-core contraction: at least the K extent rounded up to 16, and
// congruent to 8 modulo 64 so that the eight rows a fragment load touches fall
// on distinct shared-memory banks.
__host__ __device__ inline int bf16_row_stride(int Pn) {
  const int p16 = round_up(Pn, 16);
  int q = (p16 - 8 + 63) / 64;
  if (q < 0) q = 0;
  int kp = 64 * q + 8;
  if (kp < p16) kp += 64;
  return kp;
}

// Row stride of Y' = [Y | e] in shared memory: R*Jmax + 1 columns plus one
// spare (2-wide tiles may read one column past the residual), even.
__host__ __device__ inline int ystride(const Geometry& g) { return (g.R * g.Jmax + 3) & ~1; }

struct SmemLayout {
  int B, G, GT[2], GTh[2], Sh, ldig, coff, cdig, rowtab, rows, p, w, Y, S, E, F, red, V, D;
  int crd[2], xs[2], seg[2], head, total_words;
};

__host__ __device__ inline SmemLayout smem_layout(const Geometry& g, int chunk, int payload, int precision) {
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
  const int gt = g.Jmax * pad4(Pmax);
  L.B = take(sumJR);
  L.G = take(g.prodJ);
  const bool bf = precision == 1;
  const int kpmax = bf16_row_stride(Pmax);
  const int jn16 = round_up(g.Jmax, 16);
  L.GT[0] = take(bf ? 0 : gt);
  L.GT[1] = take(bf ? 0 : gt);
  L.GTh[0] = take(bf ? jn16 * kpmax / 2 : 0);
  L.GTh[1] = take(bf ? jn16 * kpmax / 2 : 0);
  L.Sh = take(bf ? round_up(chunk, 16) * kpmax / 2 : 0);
  L.ldig = take(g.prodJ);
  L.coff = take(sum_pn(g));
  L.cdig = take(2 * sum_pn(g));
  L.rowtab = take(g.sumJ);
  L.rows = take(chunk * g.sumJ);
  L.p = take(chunk * g.N * g.R);
  L.w = take(chunk * g.R);
  L.Y = take(chunk * ystride(g));
  L.S = take(bf ? 0 : chunk * tile);
  L.E = take(chunk * g.Jmax);
  L.F = take(chunk * g.Jmax);
  L.red = take(payload);
  L.V = take(g.R * kMaxJ);
  L.D = take(g.R * kMaxJ);
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
template <int N>
__device__ __forceinline__ void load_schedule(const EpochArgs& a, int64_t b, int mode, int* crd, float* xs,
                                              uint32_t* seg) {
  const Phase ph = phase_of(a, b);
  const size_t base = (size_t)(b * (int64_t)a.s.M + ph.lo);
  for (int s = threadIdx.x; s < ph.cnt; s += blockDim.x) {
#pragma unroll
    for (int k = 0; k < N; ++k) crd[s * N + k] = __ldg(a.s.crd + ((size_t)mode * N + k) * a.s.npad + base + s);
    xs[s] = __ldg(a.s.val + (size_t)mode * a.s.npad + base + s);
    seg[s] = __ldg(a.s.seg + (size_t)mode * a.s.npad + base + s);
  }
}

// The N factor rows of every sample of the chunk, with L2-coherent loads
// (rows may have been written by other CTAs in earlier phases).
template <int N>
__device__ __forceinline__ void load_rows(const EpochArgs& a, const int* crd, int cnt, const int* rowtab,
                                          float* rows) {
  const Geometry& g = a.g;
  const int sumJ = g.sumJ;
  const int total = cnt * sumJ, T = blockDim.x;
  for (int i0 = threadIdx.x; i0 < total; i0 += 4 * T) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * T;
      v[u] = 0.f;
      if (i < total) {
        const int s = i / sumJ, jj = i - s * sumJ;
        const int k = rowtab[jj] & 0xff, j = rowtab[jj] >> 8;
        if (a.precision == 1) {
          const unsigned short h = __ldcg(reinterpret_cast<const unsigned short*>(a.Ab[k]) +
                                          (size_t)crd[s * N + k] * g.Jb[k] + j);
          v[u] = __uint_as_float((uint32_t)h << 16);
        } else {
          v[u] = __ldcg(a.A[k] + (size_t)crd[s * N + k] * g.Jp[k] + j);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u * T < total) rows[i0 + u * T] = v[u];
  }
}

// G_(n) as BF16 [j][c] with row stride bf16_row_stride(P_n); rows j >= J_n
// (up to a multiple of 16) and columns c >= P_n are zero.
__device__ __forceinline__ void build_gt_bf16(__nv_bfloat16* dst, const float* Gsm, const int* cof, int Jn, int Pn,
                                              int gsn, int t0, int nt) {
  const int KP = bf16_row_stride(Pn), J16 = round_up(Jn, 16);
  for (int i = t0; i < J16 * KP; i += nt) {
    const int j = i / KP, cc = i - j * KP;
    const float v = (j < Jn && cc < Pn) ? Gsm[cof[cc] + j * gsn] : 0.f;
    dst[i] = __float2bfloat16_rn(v);
  }
}

__device__ __forceinline__ void mma_bf16_16816(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

}  // namespace

template <int N>
__global__ void __launch_bounds__(kEpochThreads, 1)
k_epoch(EpochArgs a) {
  extern __shared__ __align__(16) float sm[];
  const Geometry& g = a.g;
  const int R = g.R;
  const SmemLayout L = smem_layout(g, a.chunk_max, a.payload_max, a.precision);
  float* Bsm = sm + L.B;
  float* Gsm = sm + L.G;
  float* GTb[2] = {sm + L.GT[0], sm + L.GT[1]};
  __nv_bfloat16* GThb[2] = {reinterpret_cast<__nv_bfloat16*>(sm + L.GTh[0]),
                            reinterpret_cast<__nv_bfloat16*>(sm + L.GTh[1])};
  __nv_bfloat16* Sh = reinterpret_cast<__nv_bfloat16*>(sm + L.Sh);
  const bool bf = a.precision == 1;
  uint32_t* ldig = reinterpret_cast<uint32_t*>(sm + L.ldig);
  int* coff = reinterpret_cast<int*>(sm + L.coff);
  unsigned long long* cdig = reinterpret_cast<unsigned long long*>(sm + L.cdig);
  int* rowtab = reinterpret_cast<int*>(sm + L.rowtab);
  float* rows = sm + L.rows;
  float* pbuf = sm + L.p;
  float* Ybuf = sm + L.Y;
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
  const int ys = ystride(g);
  int Jr[N], joff[N], boff[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    Jr[k] = g.J[k];
    joff[k] = g.joff[k];
    boff[k] = g.boff[k];
  }
  unsigned long long generation = 0;

  // ---- tables built once per launch ----
  int sumJR = 0;
#pragma unroll
  for (int n = 0; n < N; ++n) sumJR += Jr[n] * R;
  for (int i = tid; i < sumJR; i += T) Bsm[i] = __ldcg(a.B + i);
  for (int lin = tid; lin < g.prodJ; lin += T) {
    int t = lin;
    uint32_t packed = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      packed |= (uint32_t)(t % Jr[k]) << (5 * k);
      t /= Jr[k];
    }
    ldig[lin] = packed;
  }
  {
    int base = 0;
#pragma unroll
    for (int n = 0; n < N; ++n) {
      const int Pn = g.prodJ / Jr[n];
      for (int cc = tid; cc < Pn; cc += T) {
        int rem = cc, off = 0, sh = 0;
        unsigned long long packed = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          if (k == n) continue;
          const int d = rem % Jr[k];
          rem /= Jr[k];
          off += d * g.gstride[k];
          packed |= (unsigned long long)(joff[k] + d) << sh;   // element offset in a sample's rows
          sh += 8;
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
  if (a.b0 < a.b1) load_schedule<N>(a, a.b0, 0, crdb[0], xsb[0], segb[0]);
  __syncthreads();

  for (int64_t b = a.b0; b < a.b1; ++b) {
    const Phase ph = phase_of(a, b);
    const int cnt = ph.cnt, lo = ph.lo, hi = ph.hi;
    const bool probe = (b == a.probe_batch);
    const float fm = (float)ph.m;
    const float invm = 1.0f / fm;

    // ------------------------------------------------------------------
    // Core phase on this CTA's chunk of the mode-1-sorted copy.
    // ------------------------------------------------------------------
    const int* crd = crdb[buf];
    const float* xs = xsb[buf];
    load_rows<N>(a, crd, cnt, rowtab, rows);
    // factor mode 1's schedule does not depend on the model: fetch it now
    load_schedule<N>(a, b, 0, crdb[buf ^ 1], xsb[buf ^ 1], segb[buf ^ 1]);
    __syncthreads();
    // p[s][k][r]: thread per (s, r), all modes
    for (int i = tid; i < cnt * R; i += T) {
      const int s = i / R, r = i - s * R;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float* ar = rows + s * sumJ + joff[k];
        const float* br = Bsm + boff[k] + r;
        float acc0 = 0.f, acc1 = 0.f;
        int j = 0;
        for (; j + 1 < Jr[k]; j += 2) {
          acc0 = fmaf(ar[j], br[j * R], acc0);
          acc1 = fmaf(ar[j + 1], br[(j + 1) * R], acc1);
        }
        if (j < Jr[k]) acc0 = fmaf(ar[j], br[j * R], acc0);
        pbuf[(s * N + k) * R + r] = acc0 + acc1;
      }
    }
    __syncthreads();

#pragma unroll
    for (int n = 0; n < N; ++n) {
      const int Jn = Jr[n];
      const int K = R * Jn;
      const int P = K + npairs * Jn * Jn;
      // W step: Rp lanes per sample.  w[s][r], residual e_s (shuffle sum over r).
      for (int i0 = 0; i0 < cnt * Rp; i0 += T) {
        const int i = i0 + tid;
        const int s = i / Rp, r = i - s * Rp;
        const bool live = (s < cnt) && (r < R);
        float w = 0.f, contrib = 0.f;
        if (live) {
          w = 1.f;
#pragma unroll
          for (int k = 0; k < N; ++k)
            if (k != n) w *= pbuf[(s * N + k) * R + r];
          contrib = w * pbuf[(s * N + n) * R + r];
        }
        for (int off = Rp >> 1; off > 0; off >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, off);
        if (live) {
          // Y[s][r*Jn + j] = w[s][r] a_n(s)[j]; e_s in column K of Y'
          float* yrow = Ybuf + s * ys;
          const float* an = rows + s * sumJ + joff[n];
          for (int j = 0; j < Jn; ++j) yrow[r * Jn + j] = w * an[j];
          if (r == 0) yrow[K] = contrib - xs[s];
        }
      }
      __syncthreads();
      // Gram tiles of Y' (fixed sample order): g = Y'^T e (1 x 2 tiles) and
      // C_{r r'} = Y_r^T Y_r' for r' < r (2 x 2 tiles)
      {
        const int tj = (Jn + 1) >> 1;
        const int gtiles = (K + 1) >> 1;
        const int ntiles = gtiles + npairs * tj * tj;
        for (int t = tid; t < ntiles; t += T) {
          int ya, yb, rowsz, colsz, obase, ostride;
          if (t < gtiles) {
            ya = K;               // the residual column
            yb = 2 * t;
            rowsz = 1;
            colsz = min(2, K - yb);
            obase = yb;
            ostride = 0;
          } else {
            const int q = t - gtiles;
            int pair = q / (tj * tj);
            const int w2 = q - pair * tj * tj, ta = w2 / tj, tb = w2 - ta * tj;
            int r = 1;
            while (pair >= r) { pair -= r; ++r; }
            const int rp = pair;
            ya = r * Jn + 2 * ta;
            yb = rp * Jn + 2 * tb;
            rowsz = min(2, Jn - 2 * ta);
            colsz = min(2, Jn - 2 * tb);
            obase = K + ((r * (r - 1) / 2 + rp) * Jn + 2 * ta) * Jn + 2 * tb;
            ostride = Jn;
          }
          float c00 = 0.f, c01 = 0.f, c10 = 0.f, c11 = 0.f;
          float d00 = 0.f, d01 = 0.f, d10 = 0.f, d11 = 0.f;
          const float* ysp = Ybuf;
          int s = 0;
          for (; s + 1 < cnt; s += 2, ysp += 2 * ys) {
            const float a0 = ysp[ya], a1 = ysp[ya + 1], b0 = ysp[yb], b1 = ysp[yb + 1];
            const float e0 = ysp[ys + ya], e1 = ysp[ys + ya + 1], f0 = ysp[ys + yb], f1 = ysp[ys + yb + 1];
            c00 = fmaf(a0, b0, c00);
            c01 = fmaf(a0, b1, c01);
            c10 = fmaf(a1, b0, c10);
            c11 = fmaf(a1, b1, c11);
            d00 = fmaf(e0, f0, d00);
            d01 = fmaf(e0, f1, d01);
            d10 = fmaf(e1, f0, d10);
            d11 = fmaf(e1, f1, d11);
          }
          if (s < cnt) {
            const float a0 = ysp[ya], a1 = ysp[ya + 1], b0 = ysp[yb], b1 = ysp[yb + 1];
            c00 = fmaf(a0, b0, c00);
            c01 = fmaf(a0, b1, c01);
            c10 = fmaf(a1, b0, c10);
            c11 = fmaf(a1, b1, c11);
          }
          c00 += d00;
          c01 += d01;
          c10 += d10;
          c11 += d11;
          float* dst = a.part + (size_t)c * a.payload_max + obase;
          __stcg(dst, c00);
          if (colsz > 1) __stcg(dst + 1, c01);
          if (rowsz > 1) {
            __stcg(dst + ostride, c10);
            if (colsz > 1) __stcg(dst + ostride + 1, c11);
          }
        }
      }
      if (!grid_barrier(a, generation)) return;
      // CTA c sums its slice of the payload over all CTAs (fixed order)
      {
        const int per = (P + G - 1) / G;
        const int o_lo = c * per, o_hi = min(o_lo + per, P);
        for (int o = o_lo + warp; o < o_hi; o += nwarps) {
          float acc = 0.f;
          for (int cc0 = lane; cc0 < G; cc0 += 8 * 32) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int cc = cc0 + 32 * u;
              v[u] = cc < G ? __ldcg(a.part + (size_t)cc * a.payload_max + o) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += v[u];
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
          if (lane == 0) __stcg(a.red + o, acc);
        }
      }
      if (!grid_barrier(a, generation)) return;
      for (int o0 = tid; o0 < P; o0 += 4 * T) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (o0 + u * T < P) ? __ldcg(a.red + o0 + u * T) : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (o0 + u * T < P) redsm[o0 + u * T] = v[u];
      }
      __syncthreads();
      // Cyclic SGD over the columns of B(n) (lines 7-14) as a block forward
      // substitution: V_r starts at g_r; after column r moves by Delta_r,
      // every later V_r'' gains C_{r'' r} Delta_r.
      {
        // 8 lanes per (r'', j) share each dot product; the lane that
        // completes V_{r+1} also moves column r+1
        float* Bn = Bsm + boff[n];
        const float* Cv = redsm + K;
        for (int i = tid; i < K; i += T) {
          const int r = i / Jn;
          Vsm[r * kMaxJ + i - r * Jn] = redsm[i];
        }
        if (tid < Jn) {
          const float V = redsm[tid];
          const float bo = Bn[tid * R];
          const float bn = bo - a.lr_b * (V * invm + a.lam_b * bo);
          Dsm[tid] = bn - bo;
          Bn[tid * R] = bn;
          if (probe && c == 0 && a.probeV) a.probeV[((size_t)n * R) * kMaxJ + tid] = V;
        }
        __syncthreads();
        for (int r = 0; r + 1 < R; ++r) {
          const int Q = (R - 1 - r) * Jn;
          for (int base = 0; base < Q * 8; base += T) {
            const int t = base + tid, q = t >> 3, l = t & 7;
            const bool live = q < Q;
            int r2 = 0, j = 0;
            float sum = 0.f;
            if (live) {
              const int qr = q / Jn;
              r2 = r + 1 + qr;
              j = q - qr * Jn;
              const float* C = Cv + ((r2 * (r2 - 1) / 2 + r) * Jn + j) * Jn;
              const float* D = Dsm + r * kMaxJ;
              for (int jp = l; jp < Jn; jp += 8) sum = fmaf(C[jp], D[jp], sum);
            }
            sum += __shfl_xor_sync(0xffffffffu, sum, 4);
            sum += __shfl_xor_sync(0xffffffffu, sum, 2);
            sum += __shfl_xor_sync(0xffffffffu, sum, 1);
            if (live && l == 0) {
              const float V = Vsm[r2 * kMaxJ + j] + sum;
              Vsm[r2 * kMaxJ + j] = V;
              if (r2 == r + 1) {
                const float bo = Bn[j * R + r2];
                const float bn = bo - a.lr_b * (V * invm + a.lam_b * bo);
                Dsm[r2 * kMaxJ + j] = bn - bo;
                Bn[j * R + r2] = bn;
                if (probe && c == 0 && a.probeV) a.probeV[((size_t)n * R + r2) * kMaxJ + j] = V;
              }
            }
          }
          __syncthreads();
        }
      }
      // p[s][n][r] with the new B(n)
      for (int i = tid; i < cnt * R; i += T) {
        const int s = i / R, r = i - s * R;
        const float* ar = rows + s * sumJ + joff[n];
        const float* br = Bsm + boff[n] + r;
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
      const float* bp[N];
#pragma unroll
      for (int k = 0; k < N; ++k) bp[k] = Bsm + boff[k] + (int)((packed >> (5 * k)) & 31u) * R;
      float acc = 0.f;
      for (int r = 0; r < R; ++r) {
        float prod = bp[0][r];
#pragma unroll
        for (int k = 1; k < N; ++k) prod *= bp[k][r];
        acc += prod;
      }
      Gsm[lin] = acc;
    }
    __syncthreads();
    if (bf) {
      build_gt_bf16(GThb[0], Gsm, coff, Jr[0], g.prodJ / Jr[0], g.gstride[0], tid, T);
    } else {
      const int Pn = g.prodJ / Jr[0], Pp = pad4(Pn);
      float* GT = GTb[0];
      for (int i = tid; i < Jr[0] * Pp; i += T) {
        const int j = i / Pp, cc = i - j * Pp;
        GT[i] = cc < Pn ? Gsm[coff[cc] + j * g.gstride[0]] : 0.f;
      }
    }
    __syncthreads();

    // ------------------------------------------------------------------
    // Factor phase, n = 1..N.
    // ------------------------------------------------------------------
    int toff = 0;   // offset of mode n's column tables
#pragma unroll
    for (int n = 0; n < N; ++n) {
      const int Jn = Jr[n];
      const int Pn = g.prodJ / Jn;
      const int Pp = pad4(Pn);
      const int* fcrd = crdb[buf];
      const float* fx = xsb[buf];
      const uint32_t* fseg = segb[buf];
      const float* GT = GTb[n & 1];
      const unsigned long long* cdn = cdig + toff;
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
      load_rows<N>(a, fcrd, cnt, rowtab, rows);
      __syncthreads();
      const int nheads = head[cnt];
      if (bf) {
        // Tensor-core contraction: E (samples x J_n) = S (samples x P_n) .
        // G_(n)^T with BF16 operands and FP32 accumulation, mma.sync
        // m16n8k16 tiles (one warp per 16 x 8 output tile, full K).
        const int KP = bf16_row_stride(Pn);
        const int C16 = round_up(cnt, 16);
        const __nv_bfloat16* GTh = GThb[n & 1];
        {
          // thread per (Kronecker column, sample group); columns looped when
          // the row is wider than the block
          const int ngroups = max(1, T / KP);
          const int sg = tid / KP;
          if (sg < ngroups) {
            for (int cl = tid - sg * KP; cl < KP; cl += (KP > T ? T : KP)) {
              int off[N - 1];
              const bool colv = cl < Pn;
              if (colv) {
                const unsigned long long packed = cdn[cl];
#pragma unroll
                for (int k = 0; k < N - 1; ++k) off[k] = (int)((packed >> (8 * k)) & 0xffu);
              }
              for (int s = sg; s < C16; s += ngroups) {
                float S1 = 0.f;
                if (colv && s < cnt) {
                  const float* rs = rows + s * sumJ;
                  S1 = rs[off[0]];
#pragma unroll
                  for (int k = 1; k < N - 1; ++k) S1 *= rs[off[k]];
                }
                Sh[s * KP + cl] = __float2bfloat16_rn(S1);
              }
            }
          }
        }
        __syncthreads();
        {
          const int mt = C16 >> 4, ntile = (Jn + 7) >> 3, ksteps = round_up(Pn, 16) >> 4;
          const int gq = lane >> 2, tq = lane & 3;
          for (int w = warp; w < mt * ntile; w += nwarps) {
            const int mi = w / ntile, ni = w - mi * ntile;
            const uint32_t* A0 = reinterpret_cast<const uint32_t*>(Sh + (mi * 16 + gq) * KP);
            const uint32_t* A1 = reinterpret_cast<const uint32_t*>(Sh + (mi * 16 + gq + 8) * KP);
            const uint32_t* Bq = reinterpret_cast<const uint32_t*>(GTh + (ni * 8 + gq) * KP);
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            for (int ks = 0; ks < ksteps; ++ks) {
              const int kw = ks * 8 + tq;
              mma_bf16_16816(d, A0[kw], A1[kw], A0[kw + 4], A1[kw + 4], Bq[kw], Bq[kw + 4]);
            }
            const int s0 = mi * 16 + gq, j0 = ni * 8 + 2 * tq;
            if (s0 < cnt) {
              if (j0 < Jn) Ebuf[s0 * Jmax + j0] = d[0];
              if (j0 + 1 < Jn) Ebuf[s0 * Jmax + j0 + 1] = d[1];
            }
            if (s0 + 8 < cnt) {
              if (j0 < Jn) Ebuf[(s0 + 8) * Jmax + j0] = d[2];
              if (j0 + 1 < Jn) Ebuf[(s0 + 8) * Jmax + j0 + 1] = d[3];
            }
          }
        }
        __syncthreads();
        // residual e_s = a_n . E_s - x_s (8 lanes per sample), contributions in place
        for (int base = 0; base < cnt * 8; base += T) {
          const int t8 = base + tid, s = t8 >> 3, l = t8 & 7;
          const bool live = s < cnt;
          float part = 0.f;
          if (live) {
            const float* an = rows + s * sumJ + joff[n];
            for (int j = l; j < Jn; j += 8) part = fmaf(an[j], Ebuf[s * Jmax + j], part);
          }
          part += __shfl_xor_sync(0xffffffffu, part, 4);
          part += __shfl_xor_sync(0xffffffffu, part, 2);
          part += __shfl_xor_sync(0xffffffffu, part, 1);
          if (live) {
            const float e = part - fx[s];
            for (int j = l; j < Jn; j += 8) Ebuf[s * Jmax + j] *= e;
          }
        }
        __syncthreads();
      } else {
      // Gather-contract E_s = G_(n) S_s^T over Kronecker-row tiles.  Thread
        // tile (sample, column pair, half of the Kronecker columns); the two
        // halves are adjacent lanes; 2*Tj lanes per sample.
        const int ntj = (Jn + 1) >> 1;
        const int Tj = pow2_at_least(ntj);
        const int lg = 31 - __clz(2 * Tj);          // log2(2 * Tj)
        const int nout = cnt << lg;
        float acc[kOutPerThread][2];
#pragma unroll
        for (int q = 0; q < kOutPerThread; ++q) acc[q][0] = acc[q][1] = 0.f;
        for (int c0 = 0; c0 < Pp; c0 += ctile_cap) {
          const int ct = min(ctile_cap, Pp - c0);
          if (c0 > 0) __syncthreads();
          // column-major build: thread per (Kronecker column, sample group)
          {
            const int ngroups = max(1, T / ct);
            const int sg = tid / ct, cl = tid - sg * ct;
            if (sg < ngroups) {
              const int cc = c0 + cl;
              if (cc < Pn) {
                const unsigned long long packed = cdn[cc];
                int off[N - 1];
#pragma unroll
                for (int k = 0; k < N - 1; ++k) off[k] = (int)((packed >> (8 * k)) & 0xffu);
                for (int s = sg; s < cnt; s += ngroups) {
                  const float* rs = rows + s * sumJ;
                  float S1 = rs[off[0]];
#pragma unroll
                  for (int k = 1; k < N - 1; ++k) S1 *= rs[off[k]];
                  Sbuf[s * ctile_cap + cl] = S1;
                }
              } else {
                for (int s = sg; s < cnt; s += ngroups) Sbuf[s * ctile_cap + cl] = 0.f;
              }
            }
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < kOutPerThread; ++q) {
            const int o = tid + q * T;
            const int s = o >> lg, rem = o & ((1 << lg) - 1), jt = rem >> 1, h = rem & 1;
            if (o < nout && jt < ntj) {
              const int j0 = 2 * jt;
              const float4* sv = reinterpret_cast<const float4*>(Sbuf + s * ctile_cap);
              const float4* g0 = reinterpret_cast<const float4*>(GT + j0 * Pp + c0);
              const float4* g1 = reinterpret_cast<const float4*>(GT + min(j0 + 1, Jn - 1) * Pp + c0);
              float a0 = acc[q][0], a1 = acc[q][1], b0 = 0.f, b1 = 0.f;
              const int nv = ct >> 2;
              int v = h;
              for (; v + 2 < nv; v += 4) {
                const float4 x = sv[v], y = g0[v], z = g1[v];
                const float4 x2 = sv[v + 2], y2 = g0[v + 2], z2 = g1[v + 2];
                a0 = fmaf(x.x, y.x, a0); a0 = fmaf(x.y, y.y, a0); a0 = fmaf(x.z, y.z, a0); a0 = fmaf(x.w, y.w, a0);
                a1 = fmaf(x.x, z.x, a1); a1 = fmaf(x.y, z.y, a1); a1 = fmaf(x.z, z.z, a1); a1 = fmaf(x.w, z.w, a1);
                b0 = fmaf(x2.x, y2.x, b0); b0 = fmaf(x2.y, y2.y, b0); b0 = fmaf(x2.z, y2.z, b0); b0 = fmaf(x2.w, y2.w, b0);
                b1 = fmaf(x2.x, z2.x, b1); b1 = fmaf(x2.y, z2.y, b1); b1 = fmaf(x2.z, z2.z, b1); b1 = fmaf(x2.w, z2.w, b1);
              }
              if (v < nv) {
                const float4 x = sv[v], y = g0[v], z = g1[v];
                a0 = fmaf(x.x, y.x, a0); a0 = fmaf(x.y, y.y, a0); a0 = fmaf(x.z, y.z, a0); a0 = fmaf(x.w, y.w, a0);
                a1 = fmaf(x.x, z.x, a1); a1 = fmaf(x.y, z.y, a1); a1 = fmaf(x.z, z.z, a1); a1 = fmaf(x.w, z.w, a1);
              }
              acc[q][0] = a0 + b0;
              acc[q][1] = a1 + b1;
            }
          }
        }
        // combine the two halves, residual e_s = a_n . E_s - x_s (shuffle sum
        // over the sample's lanes), then the contributions e_s E_s
#pragma unroll
        for (int q = 0; q < kOutPerThread; ++q) {
          const int o0 = q * T;
          if (o0 < nout) {   // uniform across the block
            const int o = tid + o0;
            const int s = o >> lg, rem = o & ((1 << lg) - 1), jt = rem >> 1, h = rem & 1;
            const bool live = (o < nout) && (jt < ntj);
            const int j0 = 2 * jt;
            float e0 = acc[q][0] + __shfl_xor_sync(0xffffffffu, acc[q][0], 1);
            float e1 = acc[q][1] + __shfl_xor_sync(0xffffffffu, acc[q][1], 1);
            float part = 0.f;
            if (live && h == 0) {
              const float* an = rows + s * sumJ + joff[n];
              part = an[j0] * e0;
              if (j0 + 1 < Jn) part = fmaf(an[j0 + 1], e1, part);
            }
            for (int off = 1 << (lg - 1); off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if (live && h == 0) {
              const float e = part - fx[s];
              Ebuf[s * Jmax + j0] = e * e0;
              if (j0 + 1 < Jn) Ebuf[s * Jmax + j0 + 1] = e * e1;
            }
          }
        }
        __syncthreads();
      }
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
          const int start = first < 0 ? 0 : first;
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane - off >= start) x += y;
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
          const int row = fcrd[s0 * N + n];
          float* ap = a.A[n] + (size_t)row * g.Jp[n] + j;
          const float av = bf ? __ldcg(ap) : rows[s0 * sumJ + joff[n] + j];
          const float nv = av - a.lr_a * (F / denom + a.lam_a * av);
          __stcg(ap, nv);
          if (bf) __stcg(reinterpret_cast<unsigned short*>(a.Ab[n]) + (size_t)row * g.Jb[n] + j,
                         __bfloat16_as_ushort(__float2bfloat16_rn(nv)));
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
          // the warp barrier orders the lanes' piece stores before lane 0's
          // release; the acquire side is completed by a fence on the rare
          // last-arriver path
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
              const int row = fcrd[s0 * N + n];
              float* ap = a.A[n] + (size_t)row * g.Jp[n] + lane;
              const float av = bf ? __ldcg(ap) : rows[s0 * sumJ + joff[n] + lane];
              const float nv = av - a.lr_a * (F / denom + a.lam_a * av);
              __stcg(ap, nv);
              if (bf) __stcg(reinterpret_cast<unsigned short*>(a.Ab[n]) + (size_t)row * g.Jb[n] + lane,
                             __bfloat16_as_ushort(__float2bfloat16_rn(nv)));
              if (probe && a.probeF) a.probeF[((size_t)n * M + st) * kMaxJ + lane] = F;
            }
            if (lane == 0) a.bcnt[c1] = 0u;
          }
        }
      }
      // meanwhile: G_(n+1) as [j][c] and the next phase's schedule
      if (warp >= 2 && n + 1 < N) {
        const int nt = T - 64, t2 = tid - 64;
        const int n1 = n + 1, Pn1 = g.prodJ / Jr[n1], Pp1 = pad4(Pn1);
        const int* cof1 = coff + toff + Pn;
        if (bf) {
          build_gt_bf16(GThb[n1 & 1], Gsm, cof1, Jr[n1], Pn1, g.gstride[n1], t2, nt);
        } else {
          float* GT1 = GTb[n1 & 1];
          for (int i = t2; i < Jr[n1] * Pp1; i += nt) {
            const int j = i / Pp1, cc = i - j * Pp1;
            GT1[i] = cc < Pn1 ? Gsm[cof1[cc] + j * g.gstride[n1]] : 0.f;
          }
        }
      }
      {
        const int64_t nb = (n + 1 < N) ? b : b + 1;
        const int nmode = (n + 1 < N) ? n + 1 : 0;
        if (nb < a.b1) load_schedule<N>(a, nb, nmode, crdb[buf ^ 1], xsb[buf ^ 1], segb[buf ^ 1]);
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
#pragma unroll
        for (int k = 0; k < N; ++k) prod *= Bsm[boff[k] + (int)((packed >> (5 * k)) & 31u) * R + r];
        acc += prod;
      }
      a.core[lin] = acc;
    }
  }
}

namespace {

template <int N>
const void* epoch_fn() {
  return (const void*)k_epoch<N>;
}

const void* kernel_for(int N) {
  switch (N) {
    case 2: return epoch_fn<2>();
    case 3: return epoch_fn<3>();
    case 4: return epoch_fn<4>();
    case 5: return epoch_fn<5>();
    case 6: return epoch_fn<6>();
    default: return nullptr;
  }
}

}  // namespace

int epoch_chunk_cap(const Geometry& g) {
  const int lanes = 2 * pow2_at_least((g.Jmax + 1) >> 1);   // lanes per sample in the contraction
  int cap = kOutPerThread * kEpochThreads / lanes;
  return cap < kMaxChunk ? cap : kMaxChunk;
}

int epoch_payload_floats(const Geometry& g) {
  int mx = 0;
  for (int n = 0; n < g.N; ++n) {
    const int Jn = g.J[n];
    const int P = g.R * Jn + (g.R * (g.R - 1) / 2) * Jn * Jn;
    if (P > mx) mx = P;
  }
  return mx;
}

size_t epoch_smem_bytes(const Geometry& g, int chunk_max, int payload_max, int precision) {
  return (size_t)smem_layout(g, chunk_max, payload_max, precision).total_words * sizeof(float);
}

cudaError_t epoch_kernel_setup(int N, size_t smem) {
  const void* fn = kernel_for(N);
  if (!fn) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int epoch_max_ctas(int N, size_t smem) {
  const void* fn = kernel_for(N);
  int dev = 0, sms = 0, per = 0;
  if (!fn) return 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kEpochThreads, smem) != cudaSuccess) return 0;
  return per * sms;
}

cudaError_t launch_epoch(const EpochArgs& a, int ctas, size_t smem, cudaStream_t st) {
  const void* fn = kernel_for(a.g.N);
  if (!fn) return cudaErrorInvalidValue;
  EpochArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(kEpochThreads), args, smem, st);
}

}  // namespace sgdt
