// Persistent epoch kernel: Algorithm 1 for every minibatch of a range.
//
// One cooperative launch holds G co-resident CTAs (one per SM) for the whole
// range.  Each minibatch (m samples) is split into G contiguous chunks of
// ceil(m/G) samples.  The chain of dependent phases per minibatch (N core
// modes, the core rebuild, N factor modes) makes the kernel latency-bound, so
// it is built to shorten that chain:
//  - per minibatch there is one grid barrier, so that the next minibatch
//    gathers every row this one updated;
//  - everything exchanged between CTAs inside a minibatch travels as 64-bit
//    words (sequence tag << 32 | float bits), written with relaxed stores and
//    polled with relaxed loads until the tag of the current (minibatch, mode)
//    shows up.  A 64-bit access is single-copy atomic, so a reader that sees
//    the tag sees the value written with it: no fence and no barrier, and a
//    consumer waits only for the words it needs.  Every wait is bounded by a
//    watchdog (error word + early return);
//  - each CTA step is written for a short per-warp instruction stream:
//    compact code (mode loops are not unrolled, per-mode constants live in
//    shared memory), divisions by launch constants through multiply-high,
//    operand rows built once per minibatch, and register-tiled products.
//
// Core phase (Algorithm 1, core phase; Eq. 7, Eq. 15).  A is fixed during the
// phase: each CTA gathers its samples' N factor rows once and keeps
//   p[s][k][r] = <a_k(s), b(k)_r>.
// For mode n the product W_r = H O_r has the closed form
// W_r[s] = w[s][r] a_n(s), w[s][r] = prod_{k != n} p[s][k][r] (mixed-product
// property of the Kronecker product, Eq. 7).  The gradient bracket V of column r
// after columns r' < r moved by Delta_{r'} is
//   V_r = g_r + sum_{r' < r} C_{r r'} Delta_{r'},
//   g_r = sum_s e_s w[s][r] a_n(s),  C_{r r'} = sum_s w[s][r] w[s][r'] a_n(s) a_n(s)^T,
//   e_s = sum_r w[s][r] p[s][n][r] - x_s at the start of the mode,
// the exact algebra of Algorithm 1's residual and Gram steps (the residual
// against the other columns is e_s plus the moves already made).  Each C_{r r'} is symmetric, so the payload is g plus
// the upper triangles of the blocks r' < r.  Reduction over the CTAs in two
// tagged hops: every CTA publishes its partial payload; CTA c sums a slice of
// it over all CTAs in a fixed order and pushes the sums into every CTA's own
// copy of the payload (so each CTA then polls lines nobody else reads); every
// CTA replays the R cyclic SGD steps on identical numbers, so all
// CTAs hold bit-identical B without a broadcast.
//
// Core rebuild (Eq. 4) is done redundantly by every CTA.
//
// Factor phase (Algorithm 1, factor phase; Eqs. 10, 11, 18), mode after mode, samples
// sorted by i_n (tiler) so that each row's samples form one run.  Per chunk:
// the Kronecker rows S_s (Eq. 10, Def. 1 column order) are built in shared
// memory and contracted with the unfolded core, E_s = G_(n) S_s^T; the
// residual e_s = a_n . E_s - x_s is reduced across each sample's lanes with
// shuffles, and the row sums F = sum_s e_s E_s (the row's -X E^T + a E E^T,
// the bracket of Eq. 18) are summed per run in sorted order.  A run inside the chunk is
// applied by this CTA.  A run that continues from an earlier chunk is
// published as a tagged piece; the CTA where the run starts polls the pieces,
// adds them in chunk order and applies the update, so no floating-point
// atomics are used and the result does not depend on timing.  Each updated
// row is also published, tagged, under its run start; later modes of the
// same minibatch (which need the rows of modes k < n as updated, Gauss-Seidel
// order) poll those slots, found through the tiler's links.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "sgdt_internal.cuh"

namespace sgdt {

namespace {

constexpr int kRightBudget = 16384;  // floats of precomputed right Gram operands (all modes)
constexpr int kSBudget = 32768;      // floats of Kronecker rows materialised at once (FP32 form)
constexpr int kMaxSmemBytes = 227 * 1024;
constexpr int kDigitTable = 4096;    // core entries whose packed digits are tabulated in shared memory

__host__ __device__ inline int pad4(int x) { return (x + 3) & ~3; }

__host__ __device__ inline int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

__host__ __device__ inline int tri(int J) { return J * (J + 1) / 2; }

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

// Core-phase payload of mode n as exchanged (64-bit tagged words, moved two
// per 16-byte access): g (R rows of J_n, each padded to a multiple of 4) and
// the upper triangles of the R(R-1)/2 blocks C_{r r'}, r' < r (each padded to
// a multiple of 4); padding words carry zeros.
__host__ __device__ inline int core_payload(int Jn, int R) {
  return R * pad4(Jn) + (R * (R - 1) / 2) * pad4(tri(Jn));
}

__host__ __device__ inline int payload_max(const Geometry& g) {
  int mx = 0;
  for (int n = 0; n < g.N; ++n) mx = core_payload(g.J[n], g.R) > mx ? core_payload(g.J[n], g.R) : mx;
  return mx;
}

// The reduced payload in shared memory: g (R x J_n, padded to 4), then every
// block C_{r r'} unpacked to full J_n x pad4(J_n) rows.
__host__ __device__ inline int unpacked_payload(int Jn, int R) {
  return pad4(R * Jn) + (R * (R - 1) / 2) * Jn * pad4(Jn);
}

// Thread tiles (one left column x 4 right columns) of the core-phase Gram
// partial of a mode, and the sample slices each tile is split into.
constexpr int kGramSplitChunk = 48;
// K-snapshot chunks of at least this many samples form their left Gram
// operand rows with one thread per sample (a 16-lane group per sample below)
constexpr int kThreadPerSampleChunk = 96;
__host__ __device__ inline int gram_tiles(int Jn, int R) {
  return R * (pad4(Jn) >> 2) + (R * (R - 1) / 2) * (pad4(Jn * (Jn + 1) / 2) >> 2);
}
__host__ __device__ inline int gram_slices(int ntile) {
  const int q = kEpochThreads / ntile;
  return q < 1 ? 1 : (q > 3 ? 3 : q);
}

// Width of a sample's Gram operand rows: left = [w_r w_r' (pairs) | e w_r],
// right = [a_j a_j' (upper triangle, padded to 4) | a_j (padded to 4)].
__host__ __device__ inline int left_width(const Geometry& g) { return g.R * (g.R - 1) / 2 + g.R; }
__host__ __device__ inline int right_width(int Jn) { return pad4(tri(Jn)) + pad4(Jn); }

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

// Row stride (in floats) of the FP32 Kronecker-row and unfolded-core tiles:
// P_n padded to 4 and then to an odd number of 16-byte units, so that the
// eight 16-byte loads of a quarter warp from eight consecutive rows fall on
// distinct shared-memory banks.
__host__ __device__ inline int fp32_row_stride(int Pn) {
  const int p4 = pad4(Pn);
  return (p4 & 7) == 4 ? p4 : p4 + 4;
}

struct SmemLayout {
  int B, VB, Bs, G, GT, GTh, Sh, S, ldig, cdig, rowtab, trij, sc[2], rows, master, p, left, right, red, D, q,
      head, fown, pbuf, gsp, cred, total_words;
  int lw, rw, sfloats, rpre, ldig_on, gsplit, srows;
};

// Words of one phase's schedule chunk: coordinates [s][N], value, run
// bounds, links [s][N].
__host__ __device__ inline int sched_chunk_words(int N, int chunk) { return (2 * N + 2) * chunk; }

// Layout variant v: 0 = right Gram operands of all modes precomputed once per
// minibatch; 1 = right operands rebuilt per mode.  srows: Kronecker rows
// materialised at once (the factor-phase contraction walks the chunk in
// pieces of srows samples); 0 = Kronecker entries formed on the fly in the
// contraction (FP32 form only).
__host__ __device__ inline SmemLayout smem_layout_v(const Geometry& g, int chunk, int ctas, int precision, int v,
                                                    int srows, int cl) {
  SmemLayout L;
  int off = 0;
  auto take = [&](int words) {
    const int at = off;
    off += pad4(words);
    return at;
  };
  int sumJR = 0, rwmax = 0, rwall = 0, redmax = 0;
  for (int n = 0; n < g.N; ++n) {
    sumJR += g.J[n] * g.R;
    rwmax = right_width(g.J[n]) > rwmax ? right_width(g.J[n]) : rwmax;
    rwall += right_width(g.J[n]);
    redmax = unpacked_payload(g.J[n], g.R) > redmax ? unpacked_payload(g.J[n], g.R) : redmax;
  }
  const int Pmax = max_pn(g);
  const bool bf = precision == 1;
  L.lw = left_width(g);
  L.rpre = (v == 0 && chunk * rwall <= kRightBudget) ? 1 : 0;
  L.rw = L.rpre ? rwall : rwmax;
  const int spmax = fp32_row_stride(Pmax);
  if (!bf && srows * spmax > kSBudget) srows = kSBudget / spmax;
  L.srows = srows;
  L.sfloats = bf ? 0 : srows * spmax;
  const int kpmax = bf16_row_stride(Pmax);
  // the unfolded core of one mode at a time: J_n rows of P_n (padded) columns
  int gt32 = 0, gt16 = 0;
  for (int n = 0; n < g.N; ++n) {
    const int pn = g.prodJ / g.J[n];
    const int f = g.J[n] * fp32_row_stride(pn), h = round_up(g.J[n], 8) * bf16_row_stride(pn) / 2;
    gt32 = f > gt32 ? f : gt32;
    gt16 = h > gt16 ? h : gt16;
  }
  L.ldig_on = g.prodJ <= kDigitTable ? 1 : 0;
  L.B = take(sumJR);
  L.VB = take(sumJR);
  L.Bs = take(sumJR);
  L.G = take(g.prodJ);
  L.GT = take(bf ? 0 : gt32);
  L.GTh = take(bf ? gt16 : 0);
  L.Sh = take(bf ? round_up(srows, 16) * kpmax / 2 : 0);
  L.S = take(L.sfloats);
  L.ldig = take(L.ldig_on ? g.prodJ : 0);
  L.cdig = take(2 * sum_pn(g));
  L.rowtab = take(g.sumJ);
  L.trij = take(tri(g.Jmax));
  L.sc[0] = take(sched_chunk_words(g.N, chunk));
  L.sc[1] = take(sched_chunk_words(g.N, chunk));
  L.rows = take(chunk * g.sumJ);
  L.master = take(bf ? chunk * g.Jmax : 0);
  L.p = take(chunk * g.N * g.R);
  L.left = take(chunk * L.lw);
  L.right = take(chunk * L.rw);
  L.red = take(redmax);
  L.D = take(64);
  L.q = take(chunk * g.Jmax);
  L.head = take(chunk + 2);
  L.fown = take(32);
  L.pbuf = take(ctas * g.Jmax);
  // large chunks: each Gram tile of the core phase is summed over up to 3
  // sample slices by different threads, the slices' partials staged here
  L.gsplit = chunk >= kGramSplitChunk ? 1 : 0;
  int gneed = 0;
  if (L.gsplit)
    for (int n = 0; n < g.N; ++n) {
      const int nt = gram_tiles(g.J[n], g.R);
      const int nsl = gram_slices(nt);
      const int need = nsl > 1 ? nsl * nt * 4 : 0;
      gneed = need > gneed ? need : gneed;
    }
  L.gsp = take(gneed);
  // cluster form: this CTA's core-phase Gram partial, two copies (mode parity),
  // read by the other CTAs of the cluster through distributed shared memory
  L.cred = take(cl ? 2 * pad4(payload_max(g)) : 0);
  L.total_words = off;
  return L;
}

// The first variant whose shared memory fits a CTA.
__host__ __device__ inline SmemLayout smem_layout(const Geometry& g, int chunk, int ctas, int precision, int cl = 0) {
  SmemLayout L = smem_layout_v(g, chunk, ctas, precision, 0, chunk, cl);
  if (L.total_words * 4 > kMaxSmemBytes) L = smem_layout_v(g, chunk, ctas, precision, 1, chunk, cl);
  // fewer Kronecker rows at a time (multiples of 16), then none (FP32)
  for (int sr = (chunk / 2 + 15) / 16 * 16; sr >= 16 && L.total_words * 4 > kMaxSmemBytes; sr = sr / 2 / 16 * 16)
    L = smem_layout_v(g, chunk, ctas, precision, 1, sr, cl);
  if (L.total_words * 4 > kMaxSmemBytes && precision != 1) L = smem_layout_v(g, chunk, ctas, precision, 1, 0, cl);
  return L;
}

// Division of small non-negative integers (< 2^31) by a launch constant d
// with one multiply-high (Granlund & Montgomery 1994): q = (umulhi(x, mul) +
// x) >> shr with shr = ceil(log2 d), mul = 2^32 (2^shr - d) / d + 1.
struct FastDiv {
  uint32_t mul, shr;
};

__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t s = 0;
  while ((1ULL << s) < d) ++s;
  FastDiv f;
  f.shr = s;
  f.mul = (uint32_t)(((1ULL << 32) * ((1ULL << s) - d)) / d + 1);
  return f;
}

__device__ __forceinline__ int fdiv(int x, FastDiv f) {
  return (int)((__umulhi((uint32_t)x, f.mul) + (uint32_t)x) >> f.shr);
}

// ---------------------------------------------------------------------------
// Memory-model primitives.
// ---------------------------------------------------------------------------
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

__device__ __forceinline__ int ld_volatile_int(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Tagged exchange word: relaxed (strong, single-copy atomic) 64-bit accesses.
__device__ __forceinline__ void put_word(unsigned long long* p, uint32_t tag, float v) {
  const unsigned long long w = ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v);
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long get_word(const unsigned long long* p) {
  unsigned long long w;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return w;
}

__device__ __forceinline__ void put_pair(unsigned long long* p, uint32_t tag, float v0, float v1) {
  const unsigned long long w0 = ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v0);
  const unsigned long long w1 = ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v1);
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(w0), "l"(w1) : "memory");
}

// Two adjacent tagged words (16-byte aligned) in one access; each word is
// single-copy atomic and carries its own tag.
__device__ __forceinline__ ulonglong2 get_pair(const unsigned long long* p) {
  ulonglong2 w;
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(w.x), "=l"(w.y) : "l"(p) : "memory");
  return w;
}

__device__ __forceinline__ uint32_t tag_of(unsigned long long w) { return (uint32_t)(w >> 32); }

__device__ __forceinline__ float val_of(unsigned long long w) { return __uint_as_float((uint32_t)w); }

// Re-reads *p until it carries `tag` (back to back: a sleep between reads,
// 32 ns to 1 us, measured slower) and returns that word.  On watchdog
// expiry, or when another CTA raised an error, returns the last word read
// (its tag is not `tag`).  Kept out of line: it is only entered when the
// first read of a word came back early, and one shared copy keeps the
// per-minibatch code small.
__device__ __noinline__ unsigned long long spin_word(const unsigned long long* p, uint32_t tag, int* err,
                                                     unsigned long long budget) {
  const unsigned long long t0 = globaltimer_ns();
  unsigned spins = 0;
  unsigned long long w = get_word(p);
  while (tag_of(w) != tag) {
    ++spins;
    if ((spins & 15u) == 0u) {
      if (ld_volatile_int(err) != 0) break;
      if (globaltimer_ns() - t0 > budget) {
        atomicCAS(err, 0, STD_ETIMEOUT);
        break;
      }
    }
    w = get_word(p);
  }
  return w;
}

// The word at p once it carries `tag`, given a first read w; `ok` turns false
// when the wait gave up.
__device__ __forceinline__ unsigned long long settle(const unsigned long long* p, unsigned long long w, uint32_t tag,
                                                     bool& ok, const EpochArgs& a) {
  if (tag_of(w) != tag) {
    w = ok ? spin_word(p, tag, a.err, a.watchdog_ns) : w;
    ok = ok && tag_of(w) == tag;
  }
  return w;
}

// Waits until every live word w[u] (p[u] != nullptr) carries tag tg[u]: each
// round re-reads all the words still missing at once, so the waits overlap.
// Returns false when the watchdog expires or another CTA raised an error.
template <int K>
__device__ __forceinline__ bool wait_all(const unsigned long long* const (&p)[K], unsigned long long (&w)[K],
                                         const uint32_t (&tg)[K], const EpochArgs& a) {
  unsigned long long t0 = 0;
  unsigned spins = 0;
#pragma unroll 1
  while (true) {
    bool done = true;
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (p[u] && tag_of(w[u]) != tg[u]) {
        done = false;
        w[u] = get_word(p[u]);
      }
    if (done) return true;
    if (t0 == 0) t0 = globaltimer_ns();
    ++spins;
    if ((spins & 15u) == 0u) {
      if (ld_volatile_int(a.err) != 0) return false;
      if (globaltimer_ns() - t0 > a.watchdog_ns) {
        atomicCAS(a.err, 0, STD_ETIMEOUT);
        return false;
      }
    }
  }
}

// wait_all for word pairs: p[u] (16-byte aligned, nullptr = absent) must
// hold `tag` in both words.
template <int K>
__device__ __forceinline__ bool wait_pairs(const unsigned long long* const (&p)[K], ulonglong2 (&w)[K], uint32_t tag,
                                           const EpochArgs& a) {
  unsigned long long t0 = 0;
  unsigned spins = 0;
#pragma unroll 1
  while (true) {
    bool done = true;
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (p[u] && (tag_of(w[u].x) != tag || tag_of(w[u].y) != tag)) {
        done = false;
        w[u] = get_pair(p[u]);
      }
    if (done) return true;
    if (t0 == 0) t0 = globaltimer_ns();
    ++spins;
    if ((spins & 15u) == 0u) {
      if (ld_volatile_int(a.err) != 0) return false;
      if (globaltimer_ns() - t0 > a.watchdog_ns) {
        atomicCAS(a.err, 0, STD_ETIMEOUT);
        return false;
      }
    }
  }
}

// Barrier over the G CTAs that work on one tensor (all CTAs of a
// single-tensor launch, or one group of a batched launch; co-resident in a
// cooperative launch).  The counter only grows; barrier k completes when it
// reaches k * G.  A wait longer than the
// watchdog budget (or an error raised by another CTA) makes every CTA return
// false; the host then reports STD_ETIMEOUT.
__device__ bool grid_barrier(const EpochArgs& a, unsigned long long& generation, int G) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++generation;
    const unsigned long long target = generation * (unsigned long long)G;
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

// Named barrier over the first `threads` threads of the CTA (id 1; id 0 is
// __syncthreads).
__device__ __forceinline__ void named_sync(int threads) {
  asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory");
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Waits for this thread's cp.async groups but the most recent one.
__device__ __forceinline__ void cp_async_wait_but_last() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

struct Phase {
  int m, chunk, lo, hi, cnt;
};

__device__ __forceinline__ Phase phase_of(const EpochArgs& a, int64_t b, int G, int c) {
  Phase ph;
  const int M = a.s.M;
  const int64_t t0 = b * (int64_t)M;
  ph.m = (int)((a.s.n - t0) < (int64_t)M ? (a.s.n - t0) : (int64_t)M);
  ph.chunk = (ph.m + G - 1) / G;
  ph.lo = c * ph.chunk;
  ph.hi = min(ph.lo + ph.chunk, ph.m);
  ph.cnt = ph.hi > ph.lo ? ph.hi - ph.lo : 0;
  return ph;
}

// Asynchronous copy of this CTA's chunk of the mode-`mode` sorted copy of
// minibatch b into a shared schedule buffer (coordinates [s][N], values, run
// bounds, links [s][N]).
__device__ __forceinline__ void prefetch_schedule(const EpochArgs& a, int N, int64_t b, int mode, int* buf,
                                                  int chunk_max, FastDiv fper, int G, int c) {
  const Phase ph = phase_of(a, b, G, c);
  const size_t base = (size_t)((b - a.s.b_first) * (int64_t)a.s.M + ph.lo);
  int* crd = buf;
  int* xs = buf + N * chunk_max;
  int* seg = xs + chunk_max;
  int* lnk = seg + chunk_max;
  const int per = N + 2 + mode;
#pragma unroll 1
  for (int i = threadIdx.x; i < ph.cnt * per; i += blockDim.x) {
    const int s = fdiv(i, fper), f = i - s * per;
    const size_t t = base + s;
    if (f < N) cp_async4(crd + s * N + f, a.s.crd + ((size_t)mode * N + f) * a.s.npad + t);
    else if (f == N) cp_async4(xs + s, a.s.val + (size_t)mode * a.s.npad + t);
    else if (f == N + 1) cp_async4(seg + s, a.s.seg + (size_t)mode * a.s.npad + t);
    else {
      const int k = f - N - 2;
      cp_async4(lnk + s * N + k, a.s.link + (size_t)(mode * (mode - 1) / 2 + k) * a.s.npad + t);
    }
  }
}

__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ void mma_bf16_16816(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Product of a sample's N-1 row entries named by a packed Kronecker column
// (8-bit element offsets into the sample's concatenated rows).
__device__ __forceinline__ float kron_entry(const float* rs, unsigned long long packed, int nm1) {
  float v = rs[(int)(packed & 0xffu)];
  if (nm1 == 2) return v * rs[(int)((packed >> 8) & 0xffu)];   // 3-way tensors
#pragma unroll 1
  for (int k = 1; k < nm1; ++k) v *= rs[(int)((packed >> (8 * k)) & 0xffu)];
  return v;
}

// FP32 factor-phase contraction E_s = G_(n) S_s^T with the residual and the
// contributions: thread per (group of SG consecutive samples, j), JL lanes
// per group (J_n rounded up to a power of two), so that each unfolded-core
// load serves SG samples; e_s = a_n . E_s - x_s is a shuffle sum over the
// group's lanes, and qbuf[s][j] = e_s E_s[j].  Without materialised
// Kronecker rows (full_s false) the entries are formed on the fly.
template <int SG>
__device__ __forceinline__ void contract_fp32(int cnt, int Jn, int Pn, int Pp, bool full_s, const float* GT,
                                              const float* Sbuf, const float* rows, int sumJ, int an_off,
                                              const unsigned long long* cdn, int nm1, const float* fx, float* qbuf,
                                              int Jmax, int tid, int T) {
  const int JL = pow2_at_least(Jn);
  const int lg = 31 - __clz(JL);
  const int ngrp = (cnt + SG - 1) / SG;
  const int nitems = ngrp << lg;
#pragma unroll 1
  for (int o0 = 0; o0 < nitems; o0 += T) {
    const int o = o0 + tid;
    const int s0 = (o >> lg) * SG, j = o & (JL - 1);
    const bool livej = (o < nitems) && (j < Jn);
    float e[SG];
#pragma unroll
    for (int q = 0; q < SG; ++q) e[q] = 0.f;
    if (livej) {
      const float* gv = GT + j * Pp;
      if (full_s) {
        // two partial sums per sample (even and odd 4-column groups)
        const float4* g4 = reinterpret_cast<const float4*>(gv);
        const float4* s4 = reinterpret_cast<const float4*>(Sbuf);
        const int nv = Pp >> 2;
        int sr[SG];   // 4-column row offsets of the group's samples (the last sample repeated past cnt)
        float f[SG];
#pragma unroll
        for (int q = 0; q < SG; ++q) {
          sr[q] = (s0 + q < cnt ? s0 + q : cnt - 1) * nv;
          f[q] = 0.f;
        }
        int v = 0;
#pragma unroll 1
        for (; v + 1 < nv; v += 2) {
          const float4 y = g4[v], y2 = g4[v + 1];
#pragma unroll
          for (int q = 0; q < SG; ++q) {
            const float4 x = s4[sr[q] + v], x2 = s4[sr[q] + v + 1];
            e[q] = fmaf(x.x, y.x, e[q]);
            e[q] = fmaf(x.y, y.y, e[q]);
            e[q] = fmaf(x.z, y.z, e[q]);
            e[q] = fmaf(x.w, y.w, e[q]);
            f[q] = fmaf(x2.x, y2.x, f[q]);
            f[q] = fmaf(x2.y, y2.y, f[q]);
            f[q] = fmaf(x2.z, y2.z, f[q]);
            f[q] = fmaf(x2.w, y2.w, f[q]);
          }
        }
        if (v < nv) {
          const float4 y = g4[v];
#pragma unroll
          for (int q = 0; q < SG; ++q) {
            const float4 x = s4[sr[q] + v];
            e[q] = fmaf(x.x, y.x, e[q]);
            e[q] = fmaf(x.y, y.y, e[q]);
            e[q] = fmaf(x.z, y.z, e[q]);
            e[q] = fmaf(x.w, y.w, e[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < SG; ++q) e[q] += f[q];
      } else {
        // entries formed on the fly, added in exactly the order of the
        // materialised form (even 4-column groups into e, odd ones into f,
        // padding columns as zeros), so the result does not depend on which
        // form the shared-memory budget allowed
        const int nv = Pp >> 2;
#pragma unroll
        for (int q = 0; q < SG; ++q)
          if (s0 + q < cnt) {
            const float* rs = rows + (s0 + q) * sumJ;
            float acc = 0.f, acc2 = 0.f;
#pragma unroll 1
            for (int v = 0; v < nv; ++v) {
              float a4 = v & 1 ? acc2 : acc;
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                const int cc = 4 * v + h;
                const float x = cc < Pn ? kron_entry(rs, cdn[cc], nm1) : 0.f;
                a4 = fmaf(x, gv[cc], a4);
              }
              if (v & 1) acc2 = a4;
              else acc = a4;
            }
            e[q] = acc + acc2;
          }
      }
    }
#pragma unroll
    for (int q = 0; q < SG; ++q) {
      const int s = s0 + q;
      const bool live = livej && s < cnt;
      float part = live ? rows[s * sumJ + an_off + j] * e[q] : 0.f;
#pragma unroll 1
      for (int off = JL >> 1; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
      if (live) qbuf[s * Jmax + j] = (part - fx[s]) * e[q];
    }
  }
}

// Right Gram operand row of one sample for mode n (a_j a_j' packed, then a_j),
// written by the lanes of one warp.
__device__ __forceinline__ void right_row(float* dst, const float* an, int Jn, int tJ, int tJp, int rwn,
                                          const int* trij, int lane) {
#pragma unroll 1
  for (int qq = lane; qq < rwn; qq += 32) {
    float v = 0.f;
    if (qq < tJ) {
      const int t = trij[qq];
      v = an[t & 0xff] * an[t >> 8];
    } else if (qq >= tJp && qq < tJp + Jn) {
      v = an[qq - tJp];
    }
    dst[qq] = v;
  }
}

}  // namespace

// Barrier over the CTAs of this thread block cluster (release/acquire at
// cluster scope: global and shared memory written before it are visible to
// every CTA of the cluster after it).
__device__ __forceinline__ void cluster_sync_all() { cooperative_groups::this_cluster().sync(); }

// The epoch of one tensor on the G CTAs c = 0..G-1 that own it.  SNAP: the
// K-snapshot form, G CTAs per group and a.snap_k groups (see k_epoch_snap).
// CL: the G CTAs are one thread block cluster (G <= 16, see k_epoch_cl): the
// core-phase reduction reads the other CTAs' partials from their shared
// memory and adds them in the same order as the two-hop exchange (so both
// forms give the same bits), and every other exchange keeps its tagged words
// but is preceded by a cluster barrier instead of being polled for.
// PLAIN: the default options only (no momentum, no probe, the 1/M
// normaliser), whose code then leaves out the other options' branches.
template <bool BF, bool SNAP, bool CL, bool PLAIN>
__device__ __forceinline__ void epoch_body(const EpochArgs& a, const int G, const int c) {
  extern __shared__ __align__(16) float sm[];
  // per-mode constants, indexed by the (runtime) mode
  __shared__ int mJ[kMaxN], mJoff[kMaxN], mBoff[kMaxN], mJp[kMaxN], mJb[kMaxN], mPn[kMaxN], mToff[kMaxN],
      mGs[kMaxN], mRoff[kMaxN];
  __shared__ FastDiv mFna4[kMaxN], mFnq4[kMaxN], mFtJ[kMaxN], mFJ[kMaxN], mFper[kMaxN];
  __shared__ float* mA[kMaxN];
  __shared__ float* mvA[kMaxN];
  __shared__ unsigned short* mAb[kMaxN];
  __shared__ int s_nheads;
  __shared__ FastDiv mFrw[kMaxN], mFjo[kMaxN], mFtail[kMaxN];
  __shared__ int s_soff[65];   // K-snapshot form: offsets of the row lists (K <= 64)
  const int N = a.g.N, R = a.g.R;
  const int chunk_max = a.chunk_max;
  const SmemLayout L = smem_layout(a.g, chunk_max, G, BF ? 1 : 0, CL ? 1 : 0);
  float* credsm = sm + L.cred;
  int cpar = 0;   // parity of the core mode (cluster form: which partial buffer)
  float* Bsm = sm + L.B;
  float* VBsm = sm + L.VB;   // Kruskal-column velocities (momentum)
  float* Bsnap = sm + L.Bs;  // K-snapshot form: B at the start of the block (then the combined B)
  float* Gsm = sm + L.G;
  float* GT = sm + L.GT;
  __nv_bfloat16* GTh = reinterpret_cast<__nv_bfloat16*>(sm + L.GTh);
  __nv_bfloat16* Sh = reinterpret_cast<__nv_bfloat16*>(sm + L.Sh);
  float* Sbuf = sm + L.S;
  uint32_t* ldig = reinterpret_cast<uint32_t*>(sm + L.ldig);
  unsigned long long* cdig = reinterpret_cast<unsigned long long*>(sm + L.cdig);
  int* rowtab = reinterpret_cast<int*>(sm + L.rowtab);
  int* trij = reinterpret_cast<int*>(sm + L.trij);
  int* scb[2] = {reinterpret_cast<int*>(sm + L.sc[0]), reinterpret_cast<int*>(sm + L.sc[1])};
  float* rows = sm + L.rows;
  float* master = sm + L.master;
  float* pbuf = sm + L.p;
  float* left = sm + L.left;
  float* right = sm + L.right;
  float* redsm = sm + L.red;
  float* Dsm = sm + L.D;
  float* qbuf = sm + L.q;
  int* head = reinterpret_cast<int*>(sm + L.head);
  float* pieces_sm = sm + L.pbuf;

  const int tid = threadIdx.x, T = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
  const int M = a.s.M;
  const int sumJ = a.g.sumJ, Jmax = a.g.Jmax, prodJ = a.g.prodJ;
  const int npairs = R * (R - 1) / 2;
  const int NR = N * R;
  const int lw = L.lw, rw = L.rw;
  unsigned long long generation = 0;

  // ---- tables built once per launch ----
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < kMaxN; ++k) {
      mJ[k] = a.g.J[k];
      mJoff[k] = a.g.joff[k];
      mBoff[k] = a.g.boff[k];
      mJp[k] = a.g.Jp[k];
      mJb[k] = a.g.Jb[k];
      mGs[k] = a.g.gstride[k];
      mA[k] = a.A[k];
      mvA[k] = a.vA[k];
      mAb[k] = reinterpret_cast<unsigned short*>(a.Ab[k]);
    }
    int toff = 0, roff = 0;
    for (int k = 0; k < N; ++k) {
      const int Jk = mJ[k];
      mPn[k] = prodJ / Jk;
      mToff[k] = toff;
      toff += mPn[k];
      mRoff[k] = L.rpre ? roff : 0;
      roff += right_width(Jk);
      mFna4[k] = make_fastdiv((uint32_t)(pad4(Jk) >> 2));
      mFnq4[k] = make_fastdiv((uint32_t)(pad4(tri(Jk)) >> 2));
      mFtJ[k] = make_fastdiv((uint32_t)tri(Jk));
      mFJ[k] = make_fastdiv((uint32_t)Jk);
      mFper[k] = make_fastdiv((uint32_t)(N + 2 + k));
      mFrw[k] = make_fastdiv((uint32_t)right_width(Jk));
      mFjo[k] = make_fastdiv((uint32_t)(a.g.joff[k] > 0 ? a.g.joff[k] : 1));
      mFtail[k] = make_fastdiv((uint32_t)(a.g.sumJ - a.g.joff[k]));
    }
  }
  __syncthreads();   // thread 0's per-mode tables, read by every thread below
  const FastDiv f_sumJ = make_fastdiv((uint32_t)sumJ);
#pragma unroll 1
  for (int jj = tid; jj < sumJ; jj += T) {
    int k = 0, j = jj;
    while (j >= mJ[k]) { j -= mJ[k]; ++k; }
    rowtab[jj] = k | (j << 8);
  }
  __syncthreads();
  const FastDiv f_R = make_fastdiv((uint32_t)R);
  const FastDiv f_NR = make_fastdiv((uint32_t)(N * R));
  const FastDiv f_Jmax = make_fastdiv((uint32_t)Jmax);
  int sumJR = 0;
  for (int n = 0; n < N; ++n) sumJR += mJ[n] * R;
#pragma unroll 1
  for (int i = tid; i < sumJR; i += T) {
    Bsm[i] = __ldcg(a.B + i);
    VBsm[i] = a.momentum != 0.f ? __ldcg(a.vB + i) : 0.f;
    if (SNAP) Bsnap[i] = Bsm[i];
  }
  // packed digits (5 bits per mode, mode 1 lowest) of core entry lin, from
  // the table when it fits in shared memory
  auto core_digits = [&](int lin) -> uint32_t {
    if (L.ldig_on) return ldig[lin];
    uint32_t packed = 0;
    int t = lin;
    for (int k = 0; k < N; ++k) {
      const int q = fdiv(t, mFJ[k]);
      packed |= (uint32_t)(t - q * mJ[k]) << (5 * k);
      t = q;
    }
    return packed;
  };
  if (L.ldig_on)
#pragma unroll 1
    for (int lin = tid; lin < prodJ; lin += T) {
      int t = lin;
      uint32_t packed = 0;
      for (int k = 0; k < N; ++k) {
        packed |= (uint32_t)(t % mJ[k]) << (5 * k);
        t /= mJ[k];
      }
      ldig[lin] = packed;
    }
#pragma unroll 1
  for (int n = 0; n < N; ++n) {
#pragma unroll 1
    for (int cc = tid; cc < mPn[n]; cc += T) {
      int rem = cc, sh = 0;
      unsigned long long packed = 0;
      for (int k = 0; k < N; ++k) {
        if (k == n) continue;
        const int d = rem % mJ[k];
        rem /= mJ[k];
        packed |= (unsigned long long)(mJoff[k] + d) << sh;   // element offset in a sample's rows
        sh += 8;
      }
      cdig[mToff[n] + cc] = packed;
    }
  }
#pragma unroll 1
  for (int q = tid; q < tri(Jmax); q += T) {
    int jb = 0;
    while (tri(jb + 1) <= q) ++jb;
    trij[q] = (q - tri(jb)) | (jb << 8);   // packed upper-triangle index q = jb (jb + 1) / 2 + ja
  }
  int buf = 0;
  // minibatches b0 + it * stride + first, it = 0 .. iters-1 (the K-snapshot
  // form: group q takes minibatch q of every block of K)
  const int stride = SNAP ? a.snap_k : 1;
  const int64_t first = SNAP ? a.snap_grp : 0;
  const int64_t iters = (a.b1 - a.b0 + stride - 1) / stride;
  const int Gtot = SNAP ? a.snap_k * G : G;
  if (a.b0 + first < a.b1) prefetch_schedule(a, N, a.b0 + first, 0, scb[0], chunk_max, mFper[0], G, c);
  cp_async_commit();
  __syncthreads();

  // K-snapshot block boundary after block `blk`: every group has finished its
  // minibatch; the Kruskal-column changes are added to the block's B and the
  // factor-row changes to A, in minibatch order, and every CTA continues from
  // the combined model
  auto snap_boundary = [&](int64_t blk) -> bool {
    if (!grid_barrier(a, generation, Gtot)) return false;
    const int64_t bs = a.b0 + blk * stride;
    const int kq = (int)((a.b1 - bs) < (int64_t)stride ? (a.b1 - bs) : (int64_t)stride);
    // column changes, loaded eight minibatches at a time and added in order
#pragma unroll 1
    for (int i = tid; i < sumJR; i += T) {
      float v = Bsnap[i];
      if (a.lr_b != 0.f)
#pragma unroll 1
        for (int k0 = 0; k0 < kq; k0 += 8) {
          float dv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) dv[u] = k0 + u < kq ? __ldcg(a.snap_dB + (size_t)(k0 + u) * sumJR + i) : 0.f;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (k0 + u < kq) v = __fadd_rn(v, dv[u]);
        }
      Bsnap[i] = v;
      Bsm[i] = v;
    }
    // sizes of the kq lists of rows this CTA owns, and their offsets
    if (warp == 0) {
      const int* cp = a.snap_count + a.snap_cta * stride;
      const int c0 = lane < kq ? __ldcg(cp + lane) : 0;
      const int c1 = lane + 32 < kq ? __ldcg(cp + lane + 32) : 0;
      int x0 = c0, x1 = c1;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y0 = __shfl_up_sync(0xffffffffu, x0, off), y1 = __shfl_up_sync(0xffffffffu, x1, off);
        if (lane >= off) {
          x0 += y0;
          x1 += y1;
        }
      }
      const int t0 = __shfl_sync(0xffffffffu, x0, 31);
      x1 += t0;
      if (lane < kq) s_soff[lane] = x0 - c0;
      if (lane + 32 < kq) s_soff[lane + 32] = x1 - c1;
      if (lane == 31) s_soff[kq] = x1;
    }
    __syncthreads();
    const int total = s_soff[kq];
    // staging area: the buffers of one minibatch's phases (rows .. q), free
    // here: a hash table of the rows (open addressing, H >= 2 total slots),
    // then per entry its list entry, minibatch, previous entry of the same
    // row, "last of its row" flag, row change and row value
    int H = 64;
    while (H < 2 * total) H <<= 1;
    const int span = L.head - L.rows;
    if ((long long)3 * H + (long long)total * (5 + 2 * Jmax) <= span) {
      // Every list entry and its row change, and the row as A holds it, all
      // loads in flight at once.  Then, minibatch after minibatch in shared
      // memory, each entry finds the previous entry of its row (hash table)
      // and takes that entry's value, or A's, plus its change: a row touched
      // by several minibatches gets its changes in minibatch order (within
      // one minibatch the entries are distinct rows).  Finally the last
      // value of every row goes to A.
      unsigned long long* hkey = reinterpret_cast<unsigned long long*>(sm + L.rows);
      int* hidx = reinterpret_cast<int*>(hkey + H);
      int2* se = reinterpret_cast<int2*>(hidx + H);
      int* sk = reinterpret_cast<int*>(se + total);
      int* prv = sk + total;
      int* lastf = prv + total;
      float* sd = reinterpret_cast<float*>(lastf + total);   // [total][Jmax] change, then value
      float* sa = sd + (size_t)total * Jmax;                  // [total][Jmax] the row in A
      const int hbits = 31 - __clz(H);
#pragma unroll 1
      for (int i = tid; i < H; i += T) hkey[i] = ~0ULL;
#pragma unroll 1
      for (int t = tid; t < total; t += T) {
        int lo = 0, hi = kq - 1;   // the list holding entry t
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_soff[mid] <= t) lo = mid;
          else hi = mid - 1;
        }
        se[t] = __ldcg(a.snap_list + ((size_t)a.snap_cta * stride + lo) * (size_t)(N * M) + (t - s_soff[lo]));
        sk[t] = lo;
      }
      __syncthreads();
#pragma unroll 1
      for (int i0 = tid; i0 < total * Jmax; i0 += 2 * T) {
        float dv[2], av[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int i = i0 + u * T;
          dv[u] = 0.f;
          av[u] = 0.f;
          if (i < total * Jmax) {
            const int t = fdiv(i, f_Jmax), jj = i - t * Jmax;
            const int2 en = se[t];
            const int nn = en.y >> 16;
            if (jj < mJ[nn]) {
              dv[u] = __ldcg(a.snap_drow + (((size_t)sk[t] * N + nn) * M + (en.y & 0xffff)) * Jmax + jj);
              av[u] = __ldcg(mA[nn] + (unsigned)en.x * (unsigned)mJp[nn] + jj);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (i0 + u * T < total * Jmax) {
            sd[i0 + u * T] = dv[u];
            sa[i0 + u * T] = av[u];
          }
      }
      __syncthreads();
#pragma unroll 1
      for (int k = 0; k < kq; ++k) {
        const int t0 = s_soff[k], t1 = s_soff[k + 1];
#pragma unroll 1
        for (int t = t0 + tid; t < t1; t += T) {
          const int2 en = se[t];
          const unsigned long long key = ((unsigned long long)(en.y >> 16) << 32) | (unsigned)en.x;
          int h = (int)((key * 0x9E3779B97F4A7C15ULL) >> (64 - hbits));
          int p = -1;
#pragma unroll 1
          for (int tries = 0; tries < H; ++tries) {
            const unsigned long long old = atomicCAS(hkey + h, ~0ULL, key);
            if (old == ~0ULL) break;   // new row
            if (old == key) {          // seen in an earlier minibatch
              p = hidx[h];
              break;
            }
            h = (h + 1) & (H - 1);
          }
          hidx[h] = t;
          prv[t] = p;
          lastf[t] = 1;
          if (p >= 0) lastf[p] = 0;
        }
        __syncthreads();
#pragma unroll 1
        for (int i = t0 * Jmax + tid; i < t1 * Jmax; i += T) {
          const int t = fdiv(i, f_Jmax), jj = i - t * Jmax;
          const int p = prv[t];
          const float base = p >= 0 ? sd[p * Jmax + jj] : sa[i];
          sd[i] = __fadd_rn(base, sd[i]);
        }
        __syncthreads();
      }
#pragma unroll 1
      for (int i = tid; i < total * Jmax; i += T) {
        const int t = fdiv(i, f_Jmax), jj = i - t * Jmax;
        const int2 en = se[t];
        const int nn = en.y >> 16;
        if (lastf[t] && jj < mJ[nn]) {
          const float nv = sd[i];
          __stcg(mA[nn] + (unsigned)en.x * (unsigned)mJp[nn] + jj, nv);
          if (BF)
            __stcg(mAb[nn] + (unsigned)en.x * (unsigned)mJb[nn] + jj, __bfloat16_as_ushort(__float2bfloat16_rn(nv)));
        }
      }
      __syncthreads();
    } else {
      // lists larger than the staging area: list after list.  A warp takes
      // 32 / Jmax entries per pass, lane group g entry g, lane j column j,
      // two passes' loads in flight
      const int gpw = 32 / Jmax;
      const int sub = lane / Jmax, jj = lane - sub * Jmax;
#pragma unroll 1
      for (int k = 0; k < kq; ++k) {
        const int cnt_k = __ldcg(a.snap_count + a.snap_cta * stride + k);
        const int2* lst = a.snap_list + ((size_t)a.snap_cta * stride + k) * (size_t)(N * M);
#pragma unroll 1
        for (int e0 = warp * 2 * gpw; e0 < cnt_k; e0 += nwarps * 2 * gpw) {
          float d[2], av[2];
          float* ap[2];
          int nn[2];
          unsigned rw[2];
          bool live[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int e = e0 + u * gpw + sub;
            live[u] = sub < gpw && e < cnt_k;
            if (live[u]) {
              const int2 en = __ldcg(lst + e);
              nn[u] = en.y >> 16;
              rw[u] = (unsigned)en.x;
              live[u] = jj < mJ[nn[u]];
              if (live[u]) {
                d[u] = __ldcg(a.snap_drow + (((size_t)k * N + nn[u]) * M + (en.y & 0xffff)) * Jmax + jj);
                ap[u] = mA[nn[u]] + rw[u] * (unsigned)mJp[nn[u]] + jj;
                av[u] = __ldcg(ap[u]);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (live[u]) {
              const float nv = __fadd_rn(av[u], d[u]);
              __stcg(ap[u], nv);
              if (BF)
                __stcg(mAb[nn[u]] + rw[u] * (unsigned)mJb[nn[u]] + jj, __bfloat16_as_ushort(__float2bfloat16_rn(nv)));
            }
        }
        __syncthreads();
      }
    }
    if (tid < stride) a.snap_count[a.snap_cta * stride + tid] = 0;
    return grid_barrier(a, generation, Gtot);
  };

#pragma unroll 1
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t b = a.b0 + it * stride + first;
    if (SNAP) {
      if (it > 0 && !snap_boundary(it - 1)) return;
      if (b >= a.b1) continue;   // a group without a minibatch in the last block
    }
    const Phase ph = phase_of(a, b, G, c);
    const int cnt = ph.cnt, lo = ph.lo, hi = ph.hi;
    const bool probe = (b == a.probe_batch);
    const float fm = (float)ph.m;
    const float invm = 1.0f / fm;
    const uint32_t tag0 = a.tag_base + (uint32_t)((b - a.b0) * 8);

    // every row update of the previous minibatch is visible after this
    if (CL) {
      if (b > a.b0) cluster_sync_all();
    } else if (!SNAP && b > a.b0 && !grid_barrier(a, generation, G)) {
      return;
    }
    cp_async_wait_all();
    __syncthreads();
    // FP32: the chunk's factor rows copied straight into shared memory, all
    // in flight at once (one cp.async group, committed before the prefetch)
    if (!BF) {
      const int* crd0 = scb[buf];
#pragma unroll 1
      for (int i = tid; i < cnt * sumJ; i += T) {
        const int s = fdiv(i, f_sumJ), jj = i - s * sumJ;
        const int k = rowtab[jj] & 0xff, j = rowtab[jj] >> 8;
        cp_async4(rows + i, mA[k] + (unsigned)crd0[s * N + k] * (unsigned)mJp[k] + j);
      }
      cp_async_commit();
    }
    // factor mode 2's chunk arrives while the core phase runs
    prefetch_schedule(a, N, b, 1, scb[buf ^ 1], chunk_max, mFper[1], G, c);
    cp_async_commit();

    // ------------------------------------------------------------------
    // Core phase on this CTA's chunk of the mode-1-sorted copy; the rows
    // stay in shared memory for factor mode 1, which uses the same chunk.
    // ------------------------------------------------------------------
    const int* crd = scb[buf];
    const float* xs = reinterpret_cast<const float*>(scb[buf] + N * chunk_max);
    constexpr int UC = SNAP ? 4 : 2;   // row loads in flight per thread (K-snapshot chunks are larger)
    if (!BF) cp_async_wait_but_last();   // the rows, not the prefetch
#pragma unroll 1
    for (int i0 = tid; i0 < (BF ? cnt * sumJ : 0); i0 += UC * T) {
      float v[UC];
#pragma unroll
      for (int u = 0; u < UC; ++u) {
        const int i = i0 + u * T;
        v[u] = 0.f;
        if (i < cnt * sumJ) {
          const int s = fdiv(i, f_sumJ), jj = i - s * sumJ;
          const int k = rowtab[jj] & 0xff, j = rowtab[jj] >> 8;
          const unsigned row = (unsigned)crd[s * N + k];
          if (BF) v[u] = __uint_as_float((uint32_t)__ldcg(mAb[k] + row * (unsigned)mJb[k] + j) << 16);
          else v[u] = __ldcg(mA[k] + row * (unsigned)mJp[k] + j);
        }
      }
#pragma unroll
      for (int u = 0; u < UC; ++u)
        if (i0 + u * T < cnt * sumJ) rows[i0 + u * T] = v[u];
    }
    __syncthreads();
    // lr_b = 0 leaves B unchanged: the core phase is skipped
    if (a.lr_b != 0.f) {
      // p[s][k][r] (thread per (sample, k, r)) and, when they fit, the right
      // Gram operand rows of every mode (they depend on A only)
  #pragma unroll 1
      for (int i = tid; i < cnt * NR; i += T) {
        const int s = fdiv(i, f_NR), kr = i - s * NR;
        const int k = fdiv(kr, f_R), r = kr - k * R;
        const float* ar = rows + s * sumJ + mJoff[k];
        const float* br = Bsm + mBoff[k] + r;
        float acc0 = 0.f, acc1 = 0.f;
        int j = 0;
  #pragma unroll 1
        for (; j + 1 < mJ[k]; j += 2) {
          acc0 = fmaf(ar[j], br[j * R], acc0);
          acc1 = fmaf(ar[j + 1], br[(j + 1) * R], acc1);
        }
        if (j < mJ[k]) acc0 = fmaf(ar[j], br[j * R], acc0);
        pbuf[i] = acc0 + acc1;
      }
      if (L.rpre)
  #pragma unroll 1
        for (int s = warp; s < cnt; s += nwarps) {
          const float* rs = rows + s * sumJ;
  #pragma unroll 1
          for (int n = 0; n < N; ++n) {
            const int Jn = mJ[n];
            right_row(right + s * rw + mRoff[n], rs + mJoff[n], Jn, tri(Jn), pad4(tri(Jn)), right_width(Jn), trij,
                      lane);
          }
        }
      __syncthreads();

  #pragma unroll 1
      for (int n = 0; n < N; ++n) {
        const int Jn = mJ[n];
        const int tJ = tri(Jn);
        const int tJp = pad4(tJ);
        const int Jq = pad4(Jn);
        const int K = R * Jn;
        const int Kq = pad4(K);
        const int Kx = R * Jq;                  // exchanged g rows, padded
        const int P = Kx + npairs * tJp;        // exchanged payload (multiple of 4 words)
        const uint32_t tag = tag0 + (uint32_t)n;
        const int nq4 = tJp >> 2, na4 = Jq >> 2;
        const int ntile = R * na4 + npairs * nq4;
        const FastDiv f_na4 = mFna4[n], f_nq4 = mFnq4[n];
        // left Gram operand rows: w_r = prod_{k != n} p[s][k][r], the residual
        // e_s = sum_r w_r p[s][n][r] - x_s, e_s w_r and w_r w_r' (r' < r); one
        // sample per 16-lane group (R <= 16) or per warp, lane r forming w_r
        // and the residual a group sum, except in the large chunks of the
        // K-snapshot form, one sample per thread.  Then the right operand rows
        // of this mode unless built above.
        {
          const bool per_thread = SNAP && cnt >= kThreadPerSampleChunk;
          const int gl = R <= 16 ? 16 : 32;
          const int gpw = 32 / gl;
          const int sub = lane / gl, gla = lane - sub * gl;
          const int gbase = sub * gl;
  #pragma unroll 1
          for (int s0 = warp * gpw; s0 < (per_thread ? 0 : cnt); s0 += nwarps * gpw) {
            const int s = s0 + sub;
            const bool live = (s < cnt) && (gla < R);
            float w = 0.f, contrib = 0.f;
            if (live) {
              const float* ps = pbuf + s * NR + gla;
              w = 1.f;
  #pragma unroll 1
              for (int k = 0; k < N; ++k)
                if (k != n) w *= ps[k * R];
              contrib = w * ps[n * R];
            }
  #pragma unroll
            for (int off = 16; off > 0; off >>= 1)
              if (off < gl) contrib += __shfl_xor_sync(0xffffffffu, contrib, off);
            float* lrow = left + s * lw;
  #pragma unroll 1
            for (int rp = 0; rp + 1 < R; ++rp) {
              const float wp = __shfl_sync(0xffffffffu, w, gbase + rp);
              if (live && rp < gla) lrow[gla * (gla - 1) / 2 + rp] = w * wp;
            }
            if (live) lrow[npairs + gla] = (contrib - xs[s]) * w;
          }
          if (per_thread)
  #pragma unroll 1
            for (int s = tid; s < cnt; s += T) {
              const float* ps = pbuf + s * NR;
              float* lrow = left + s * lw;
              float contrib = 0.f;
  #pragma unroll 1
              for (int r = 0; r < R; ++r) {
                float w = 1.f;
  #pragma unroll 1
                for (int k = 0; k < N; ++k)
                  if (k != n) w *= ps[k * R + r];
                contrib = fmaf(w, ps[n * R + r], contrib);
                lrow[npairs + r] = w;
              }
              const float e = contrib - xs[s];
  #pragma unroll 1
              for (int r = 1; r < R; ++r) {
                const float wr = lrow[npairs + r];
  #pragma unroll 1
                for (int rp = 0; rp < r; ++rp) lrow[r * (r - 1) / 2 + rp] = wr * lrow[npairs + rp];
              }
  #pragma unroll 1
              for (int r = 0; r < R; ++r) lrow[npairs + r] *= e;
            }
          if (!L.rpre) {
            // thread per (sample, entry) of the right rows
            const int rwn = right_width(Jn);
            const FastDiv frw = mFrw[n];
  #pragma unroll 1
            for (int i = tid; i < cnt * rwn; i += T) {
              const int s = fdiv(i, frw), qq = i - s * rwn;
              const float* an = rows + s * sumJ + mJoff[n];
              float v = 0.f;
              if (qq < tJ) {
                const int t = trij[qq];
                v = an[t & 0xff] * an[t >> 8];
              } else if (qq >= tJp && qq < tJp + Jn) {
                v = an[qq - tJp];
              }
              right[s * rw + qq] = v;
            }
          }
        }
        __syncthreads();
        // Gram partial, thread tile = one left column x 4 right columns over
        // the chunk (or over one of up to 3 sample slices, added in slice
        // order), published as soon as it is summed
        {
          const float* rbase = right + mRoff[n];
          unsigned long long* dst = a.part + (unsigned)c * (unsigned)a.pstride;
          const int nsl = L.gsplit ? gram_slices(ntile) : 1;
          float4* gsp = reinterpret_cast<float4*>(sm + L.gsp);
          const int cs = (cnt + nsl - 1) / nsl;
  #pragma unroll 1
          for (int t0 = tid; t0 < nsl * ntile; t0 += T) {
            const int sl = t0 / ntile, t = t0 - sl * ntile;
            int li, rc;
            if (t < R * na4) {
              const int r = fdiv(t, f_na4), jg = t - r * na4;
              li = npairs + r;
              rc = tJp + 4 * jg;
            } else {
              const int t2 = t - R * na4;
              const int qi = fdiv(t2, f_nq4), jg = t2 - qi * nq4;
              li = qi;
              rc = 4 * jg;
            }
            const int obase = 4 * t;   // tiles are the payload's 4-word groups in order
            float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
            const float* lp = left + li;
            const float* rp = rbase + rc;
            const int se = min(cnt, (sl + 1) * cs);
            int s = sl * cs;
  #pragma unroll 1
            for (; s + 1 < se; s += 2) {
              const float l0 = lp[s * lw], l1 = lp[(s + 1) * lw];
              const float4 r0 = *reinterpret_cast<const float4*>(rp + s * rw);
              const float4 r1 = *reinterpret_cast<const float4*>(rp + (s + 1) * rw);
              x0.x = fmaf(l0, r0.x, x0.x); x0.y = fmaf(l0, r0.y, x0.y);
              x0.z = fmaf(l0, r0.z, x0.z); x0.w = fmaf(l0, r0.w, x0.w);
              x1.x = fmaf(l1, r1.x, x1.x); x1.y = fmaf(l1, r1.y, x1.y);
              x1.z = fmaf(l1, r1.z, x1.z); x1.w = fmaf(l1, r1.w, x1.w);
            }
            if (s < se) {
              const float l0 = lp[s * lw];
              const float4 r0 = *reinterpret_cast<const float4*>(rp + s * rw);
              x0.x = fmaf(l0, r0.x, x0.x); x0.y = fmaf(l0, r0.y, x0.y);
              x0.z = fmaf(l0, r0.z, x0.z); x0.w = fmaf(l0, r0.w, x0.w);
            }
            const float4 x = make_float4(x0.x + x1.x, x0.y + x1.y, x0.z + x1.z, x0.w + x1.w);
            if (nsl == 1) {
              if (CL) {
                *reinterpret_cast<float4*>(credsm + (cpar & 1) * pad4(payload_max(a.g)) + obase) = x;
              } else {
                put_pair(dst + obase, tag, x.x, x.y);
                put_pair(dst + obase + 2, tag, x.z, x.w);
              }
            } else if (sl > 0) {
              gsp[(sl - 1) * ntile + t] = x;
            } else {
              gsp[(nsl - 1) * ntile + t] = x;   // slice 0 parks its sum after the others
            }
          }
          if (nsl > 1) {
            __syncthreads();
  #pragma unroll 1
            for (int t = tid; t < ntile; t += T) {
              float4 x = gsp[(nsl - 1) * ntile + t];
  #pragma unroll 1
              for (int q = 1; q < nsl; ++q) {
                const float4 y = gsp[(q - 1) * ntile + t];
                x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w;
              }
              if (CL) {
                *reinterpret_cast<float4*>(credsm + (cpar & 1) * pad4(payload_max(a.g)) + 4 * t) = x;
              } else {
                put_pair(dst + 4 * t, tag, x.x, x.y);
                put_pair(dst + 4 * t + 2, tag, x.z, x.w);
              }
            }
          }
        }
        // payload word o of the reduced Gram into shared memory: g as R x J_n,
        // each block C_{r r'} unpacked to full rows of stride pad4(J_n)
        auto put_red = [&](int o, float v) {
          if (o < Kx) {
            const int r = fdiv(o >> 2, f_na4), j = o - r * Jq;
            if (j < Jn) redsm[r * Jn + j] = v;
          } else {
            const int t = o - Kx;
            const int q = fdiv(t >> 2, f_nq4), jj = t - q * tJp;
            if (jj < tJ) {
              const int ja = trij[jj] & 0xff, jb = trij[jj] >> 8;
              float* blk = redsm + Kq + q * Jn * Jq;
              blk[ja * Jq + jb] = v;
              blk[jb * Jq + ja] = v;
            }
          }
        };
        bool ok = true;
        if (CL) {
          // every CTA sums the cluster's partials itself, word by word, in the
          // order of the two-hop exchange's butterfly over GL = G rounded up
          // to a power of two lanes (missing CTAs contribute +0)
          cluster_sync_all();
          cooperative_groups::cluster_group cg_cl = cooperative_groups::this_cluster();
          const int GL = pow2_at_least(G);
          const float* mine = credsm + (cpar & 1) * pad4(payload_max(a.g));
  #pragma unroll 1
          for (int o = tid; o < P; o += T) {
            float t16[16];
  #pragma unroll
            for (int q = 0; q < 16; ++q)
              t16[q] = (q < G) ? *cg_cl.map_shared_rank(mine + o, (unsigned)q) : 0.f;
  #pragma unroll
            for (int off = 8; off > 0; off >>= 1)
              if (off < GL)
  #pragma unroll
                for (int q = 0; q < 8; ++q)
                  if (q < off) t16[q] = t16[q] + t16[q + off];
            put_red(o, t16[0]);
          }
        } else {
        // hop 1: CTA c sums its slice of the payload (word pairs) over all CTAs
        // (in CTA order within each lane, then a fixed butterfly across the
        // GL lanes of the pair) and pushes each sum into every CTA's copy of
        // the payload; with fewer than 32 CTAs a warp takes 32 / GL pairs at once
        // (a separate loop: the full-warp form is faster when every lane has a CTA)
        {
          const int P2 = P >> 1;
          const int per = (P2 + G - 1) / G;
          const int o_lo = c * per, o_hi = min(o_lo + per, P2);
          if (G >= 32) {
    #pragma unroll 1
            for (int o = o_lo + warp; o < o_hi; o += nwarps) {
              ulonglong2 w8[8];
              const unsigned long long* p8[8];
    #pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int cc = lane + 32 * u;
                p8[u] = cc < G ? a.part + (unsigned)cc * (unsigned)a.pstride + 2 * o : nullptr;
                w8[u] = p8[u] ? get_pair(p8[u]) : make_ulonglong2(0ULL, 0ULL);
              }
              if (ok) ok = wait_pairs<8>(p8, w8, tag, a);
              float s0 = 0.f, s1 = 0.f;
    #pragma unroll
              for (int u = 0; u < 8; ++u)
                if (p8[u]) {
                  s0 += val_of(w8[u].x);
                  s1 += val_of(w8[u].y);
                }
    #pragma unroll
              for (int off = 16; off > 0; off >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, off);
                s1 += __shfl_xor_sync(0xffffffffu, s1, off);
              }
              if (ok)
    #pragma unroll 1
                for (int cc = lane; cc < G; cc += 32) put_pair(a.inbox + (unsigned)cc * (unsigned)a.pstride + 2 * o, tag, s0, s1);
            }
          } else {
            // GL = G rounded up to a power of two lanes per pair, one CTA per lane
            const int GL = pow2_at_least(G);
            const int lgl = 31 - __clz(GL);
            const int sub = lane >> lgl, gl = lane & (GL - 1);
    #pragma unroll 1
            for (int ob = o_lo + (warp << (5 - lgl)); ob < o_hi; ob += nwarps << (5 - lgl)) {
              const int o = ob + sub;
              ulonglong2 w1[1];
              const unsigned long long* p1[1];
              p1[0] = (o < o_hi && gl < G) ? a.part + (unsigned)gl * (unsigned)a.pstride + 2 * o : nullptr;
              w1[0] = p1[0] ? get_pair(p1[0]) : make_ulonglong2(0ULL, 0ULL);
              if (ok) ok = wait_pairs<1>(p1, w1, tag, a);
              float s0 = p1[0] ? val_of(w1[0].x) : 0.f, s1 = p1[0] ? val_of(w1[0].y) : 0.f;
    #pragma unroll
              for (int off = 16; off > 0; off >>= 1)
                if (off < GL) {
                  s0 += __shfl_xor_sync(0xffffffffu, s0, off);
                  s1 += __shfl_xor_sync(0xffffffffu, s1, off);
                }
              if (ok && o < o_hi && gl < G)
                put_pair(a.inbox + (unsigned)gl * (unsigned)a.pstride + 2 * o, tag, s0, s1);
            }
          }
        }
        // hop 2: this CTA's copy of the reduced payload, into shared memory: g
        // as R x J_n, each block C_{r r'} unpacked to full rows of stride
        // pad4(J_n)
        {
          const unsigned long long* mine = a.inbox + (unsigned)c * (unsigned)a.pstride;
  #pragma unroll 1
          for (int o2 = tid; o2 < (P >> 1); o2 += T) {
            ulonglong2 w1[1];
            const unsigned long long* p1[1] = {mine + 2 * o2};
            w1[0] = get_pair(p1[0]);
            if (ok) ok = wait_pairs<1>(p1, w1, tag, a);
  #pragma unroll
            for (int u = 0; u < 2; ++u) put_red(2 * o2 + u, val_of(u == 0 ? w1[0].x : w1[0].y));
          }
        }
        }
        {
          // zero padding columns of the unpacked blocks
          if (Jq > Jn)
  #pragma unroll 1
            for (int i = tid; i < npairs * Jn; i += T)
  #pragma unroll 1
              for (int j = Jn; j < Jq; ++j) redsm[Kq + i * Jq + j] = 0.f;
        }
        if (!__syncthreads_and(ok) && !CL) return;
        // Cyclic SGD over the columns of B(n) (Algorithm 1's loop over r) as a block forward
        // substitution: warp w keeps V_w (lane j) and V_{w+16}; at step r the
        // owner of column r moves it, and every later V_r'' gains C_{r'' r}
        // Delta_r (Delta double-buffered by step parity, one named barrier per
        // step).
        {
          const int nrw = R < nwarps ? R : nwarps;
          if (warp < nrw) {
            float* Bn = Bsm + mBoff[n];
            const float* Cv = redsm + Kq;
            const bool lj = lane < Jn;
            const int ra = warp, rb = warp + nwarps;
            float Va = (lj && ra < R) ? redsm[ra * Jn + lane] : 0.f;
            float Vb = (lj && rb < R) ? redsm[rb * Jn + lane] : 0.f;
            const float boa = (lj && ra < R) ? Bn[lane * R + ra] : 0.f;
            const float bob = (lj && rb < R) ? Bn[lane * R + rb] : 0.f;
            const int nv4 = Jq >> 2;
  #pragma unroll 1
            for (int r = 0; r < R; ++r) {
              float* D = Dsm + (r & 1) * 32;
              if ((ra == r || rb == r) && lane < Jq) {
                float d = 0.f;
                if (lj) {
                  const float V = ra == r ? Va : Vb;
                  const float bo = ra == r ? boa : bob;
                  const float gb = V * invm + a.lam_b * bo;
                  float step = gb;
                  if (!PLAIN && a.momentum != 0.f) {
                    float* vb = VBsm + mBoff[n] + lane * R + r;
                    step = a.momentum * *vb + gb;
                    *vb = step;
                  }
                  float bn;
                  if (SNAP) {
                    // the change is recorded for the block's end (w + delta form)
                    const float dl = -__fmul_rn(a.lr_b, step);
                    bn = __fadd_rn(bo, dl);
                    if (c == 0) a.snap_dB[(size_t)a.snap_grp * sumJR + mBoff[n] + lane * R + r] = dl;
                  } else {
                    bn = bo - a.lr_b * step;
                  }
                  d = bn - bo;
                  Bn[lane * R + r] = bn;
                  if (!PLAIN && probe && c == 0 && a.probeV) a.probeV[((unsigned)n * R + r) * kMaxJ + lane] = V;
                }
                D[lane] = d;
              }
              named_sync(nrw * 32);
              if (lj) {
                const float4* D4 = reinterpret_cast<const float4*>(D);
  #pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                  const int r2 = h == 0 ? ra : rb;
                  if (r2 > r && r2 < R) {
                    const float4* C4 = reinterpret_cast<const float4*>(Cv + ((r2 * (r2 - 1) / 2 + r) * Jn + lane) * Jq);
                    float s0 = 0.f, s1 = 0.f;
  #pragma unroll   // (unrolled: the loads of C_{r'' r} issue together)
                    for (int v = 0; v < kMaxJ / 4; ++v) {
                      if (v >= nv4) break;
                      const float4 cv = C4[v], dv = D4[v];
                      s0 = fmaf(cv.x, dv.x, s0);
                      s1 = fmaf(cv.y, dv.y, s1);
                      s0 = fmaf(cv.z, dv.z, s0);
                      s1 = fmaf(cv.w, dv.w, s1);
                    }
                    if (h == 0) Va += s0 + s1;
                    else Vb += s0 + s1;
                  }
                }
              }
            }
          }
        }
        __syncthreads();
        // p[s][n][r] with the new B(n): thread per (sample, r)
  #pragma unroll 1
        for (int i = tid; i < cnt * R; i += T) {
          const int s = fdiv(i, f_R), r = i - s * R;
          const float* ar = rows + s * sumJ + mJoff[n];
          const float* br = Bsm + mBoff[n] + r;
          float acc0 = 0.f, acc1 = 0.f;
          int j = 0;
  #pragma unroll 1
          for (; j + 1 < Jn; j += 2) {
            acc0 = fmaf(ar[j], br[j * R], acc0);
            acc1 = fmaf(ar[j + 1], br[(j + 1) * R], acc1);
          }
          if (j < Jn) acc0 = fmaf(ar[j], br[j * R], acc0);
          pbuf[s * NR + n * R + r] = acc0 + acc1;
        }
        __syncthreads();
        ++cpar;
      }
    }

    // ------------------------------------------------------------------
    // G-hat from B (Eq. 4), mode 1 fastest.
    // ------------------------------------------------------------------
#pragma unroll 1
    for (int lin = tid; lin < prodJ; lin += T) {
      const uint32_t packed = core_digits(lin);
      float acc = 0.f;
#pragma unroll 1
      for (int r = 0; r < R; ++r) {
        float prod = Bsm[mBoff[0] + (int)(packed & 31u) * R + r];
#pragma unroll 1
        for (int k = 1; k < N; ++k) prod *= Bsm[mBoff[k] + (int)((packed >> (5 * k)) & 31u) * R + r];
        acc += prod;
      }
      Gsm[lin] = acc;
    }
    __syncthreads();

    // ------------------------------------------------------------------
    // Factor phase, n = 1..N.
    // ------------------------------------------------------------------
#pragma unroll 1
    for (int n = 0; n < N; ++n) {
      const int Jn = mJ[n];
      const int Pn = mPn[n];
      const int Pp = fp32_row_stride(Pn);
      const uint32_t tag = tag0 + (uint32_t)n;
      const unsigned long long* cdn = cdig + mToff[n];
      bool ok = true;
      if (n > 0) {
        cp_async_wait_all();
        __syncthreads();
        if (CL) cluster_sync_all();   // the previous mode's row slots
        buf ^= 1;
        // FP32: rows of modes k >= n from A straight into shared memory (one
        // cp.async group, committed before the prefetch)
        if (!BF) {
          const int* fc = scb[buf];
          const int tailJ = sumJ - mJoff[n];
          const FastDiv ft = mFtail[n];
#pragma unroll 1
          for (int i = tid; i < cnt * tailJ; i += T) {
            const int s = fdiv(i, ft), jj = mJoff[n] + (i - s * tailJ);
            const int k = rowtab[jj] & 0xff, j = rowtab[jj] >> 8;
            cp_async4(rows + s * sumJ + jj, mA[k] + (unsigned)fc[s * N + k] * (unsigned)mJp[k] + j);
          }
          cp_async_commit();
        }
        // the next phase's chunk: mode n+1 of this minibatch, or mode 1 of the next
        const int64_t nb = (n + 1 < N) ? b : b + stride;
        const int nmode = (n + 1 < N) ? n + 1 : 0;
        if (nb < a.b1) prefetch_schedule(a, N, nb, nmode, scb[buf ^ 1], chunk_max, mFper[nmode], G, c);
        cp_async_commit();
      }
      const int* fcrd = scb[buf];
      const float* fx = reinterpret_cast<const float*>(scb[buf] + N * chunk_max);
      const uint32_t* fseg = reinterpret_cast<const uint32_t*>(scb[buf] + (N + 1) * chunk_max);
      const int* fl = scb[buf] + (N + 2) * chunk_max;
      // rows: modes k < n as updated earlier in this minibatch (tagged slots,
      // through the links), modes k >= n from A; G_(n) and the run heads are
      // built while the first loads are in flight
      // FP32: only the rows of modes k < n (the first joff[n] entries of a
      // sample's rows) go through this loop
      const int width = BF ? sumJ : mJoff[n];
      const FastDiv fw = BF ? f_sumJ : mFjo[n];
      const int total = n > 0 ? cnt * width : 0;
      constexpr int UG = SNAP ? 4 : 2;   // row loads in flight per thread
      unsigned long long w2[UG];
      const unsigned long long* p2[UG];
      uint32_t t2[UG];
      float v2[UG];
      int i0 = tid;
#pragma unroll 1
      for (bool first = true; i0 < total || first; i0 += UG * T, first = false) {
#pragma unroll
        for (int u = 0; u < UG; ++u) {
          const int i = i0 + u * T;
          p2[u] = nullptr;
          w2[u] = 0ULL;
          t2[u] = 0u;
          v2[u] = 0.f;
          if (i < total) {
            const int s = fdiv(i, fw), jj = i - s * width;
            const int k = rowtab[jj] & 0xff, j = rowtab[jj] >> 8;
            if (k < n) {
              p2[u] = a.mail + ((unsigned)k * (unsigned)M + (unsigned)fl[s * N + k]) * (unsigned)(Jmax + (Jmax & 1)) + j;
              w2[u] = get_word(p2[u]);
              t2[u] = tag0 + (uint32_t)k;
            } else {
              const unsigned row = (unsigned)fcrd[s * N + k];
              if (BF) v2[u] = __uint_as_float((uint32_t)__ldcg(mAb[k] + row * (unsigned)mJb[k] + j) << 16);
              else v2[u] = __ldcg(mA[k] + row * (unsigned)mJp[k] + j);
            }
          }
        }
        if (first) {
          // G_(n) for the contraction, [j][c]: warp per j, lanes over c;
          // column c sits at the offset of its other-mode digits in G-hat
          // (BF16: the rows and columns the tensor-core tiles read, J_n
          // rounded up to 8 and P_n to 16)
          const int KP = BF ? bf16_row_stride(Pn) : Pp;
          const int Kext = BF ? round_up(Pn, 16) : Pp;
          const int Jrows = a.contraction == 1 ? 0 : (BF ? round_up(Jn, 8) : Jn);
#pragma unroll 1
          for (int j = warp; j < Jrows; j += nwarps)
#pragma unroll 1
            for (int cc0 = lane; cc0 < Kext; cc0 += 64) {
              float gv[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int cc = cc0 + 32 * h;
                gv[h] = 0.f;
                if (j < Jn && cc < Pn) {
                  const unsigned long long packed = cdn[cc];
                  int off = j * mGs[n], sh = 0;
#pragma unroll 1
                  for (int k = 0; k < N; ++k) {
                    if (k == n) continue;
                    off += ((int)((packed >> sh) & 0xffu) - mJoff[k]) * mGs[k];
                    sh += 8;
                  }
                  gv[h] = Gsm[off];
                }
              }
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int cc = cc0 + 32 * h;
                if (cc < Kext) {
                  if (BF) GTh[j * KP + cc] = __float2bfloat16_rn(gv[h]);
                  else GT[j * KP + cc] = gv[h];
                }
              }
            }
          // run heads of this chunk, compacted in order (last warp)
          if (warp == nwarps - 1) {
            int nh = 0;
#pragma unroll 1
            for (int s0 = 0; s0 < cnt; s0 += 32) {
              const int s = s0 + lane;
              bool is_head = false;
              if (s < cnt) is_head = (s == 0) || ((int)(fseg[s] & 0xffffu) == lo + s);
              const unsigned mask = __ballot_sync(0xffffffffu, is_head);
              if (is_head) head[nh + __popc(mask & ((1u << lane) - 1u))] = s;
              nh += __popc(mask);
            }
            if (lane == 0) {
              head[nh] = cnt;
              s_nheads = nh;
            }
          }
        }
        if (ok) ok = wait_all<UG>(p2, w2, t2, a);
#pragma unroll
        for (int u = 0; u < UG; ++u) {
          const int i = i0 + u * T;
          if (i < total) {
            const int s = fdiv(i, fw);
            rows[s * sumJ + (i - s * width)] = p2[u] ? (BF ? bf16_round(val_of(w2[u])) : val_of(w2[u])) : v2[u];
          }
        }
      }
      if (!BF && n > 0) cp_async_wait_but_last();   // the rows of modes >= n, not the prefetch
      if (!__syncthreads_and(ok) && !CL) return;
      const int nheads = s_nheads;
      // BF16 form: the FP32 master rows, fetched only for the runs this CTA
      // updates (run heads that start in this chunk), while the contraction runs
      if (BF) {
#pragma unroll 1
        for (int h = warp; h < nheads; h += nwarps) {
          const int s0 = head[h];
          if (lane < Jn && (int)(fseg[s0] & 0xffffu) >= lo)
            cp_async4(master + h * Jmax + lane, mA[n] + (unsigned)fcrd[s0 * N + n] * (unsigned)mJp[n] + lane);
        }
        cp_async_commit();
      }
      // Kronecker rows S_s (Eq. 10), warp per sample, lanes over columns
      const int nm1 = N - 1;
      const bool kru = a.contraction == 1;
      const bool full_s = BF || L.srows > 0;
      if (kru) {
        // Kruskal form of the same contraction (Eq. 4 in Eq. 11):
        // E_s = G_(n) S_s^T = B(n) w_s, w_s[r] = prod_{k != n} <a_k(s), b(k)_r>;
        // warp per sample, lane r forms w_r, lane j forms E_j, then the
        // residual e_s = a_n . E_s - x_s (warp sum) and the contributions
#pragma unroll 1
        for (int s = warp; s < cnt; s += nwarps) {
          const float* rs = rows + s * sumJ;
          float w = 0.f;
          if (lane < R) {
            w = 1.f;
#pragma unroll 1
            for (int k = 0; k < N; ++k) {
              if (k == n) continue;
              const float* ak = rs + mJoff[k];
              const float* bk = Bsm + mBoff[k] + lane;
              float d0 = 0.f, d1 = 0.f;
              int j = 0;
#pragma unroll 1
              for (; j + 1 < mJ[k]; j += 2) {
                d0 = fmaf(ak[j], bk[j * R], d0);
                d1 = fmaf(ak[j + 1], bk[(j + 1) * R], d1);
              }
              if (j < mJ[k]) d0 = fmaf(ak[j], bk[j * R], d0);
              w *= d0 + d1;
            }
          }
          float E = 0.f;
          const float* bn = Bsm + mBoff[n] + (lane < Jn ? lane : 0) * R;
#pragma unroll 1
          for (int r = 0; r < R; ++r) E = fmaf(bn[r], __shfl_sync(0xffffffffu, w, r), E);
          float part = lane < Jn ? rs[mJoff[n] + lane] * E : 0.f;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
          if (lane < Jn) qbuf[s * Jmax + lane] = (part - fx[s]) * E;
        }
      }
      if (kru) {
        __syncthreads();   // E_s and the contributions were formed above
      } else {
        // the chunk in pieces of srows samples (one piece when they all fit):
        // Kronecker rows of the piece, then its contraction
        const int piece = full_s ? (L.srows < cnt ? L.srows : cnt) : cnt;
#pragma unroll 1
        for (int sa = 0; sa < cnt || sa == 0; sa += (piece > 0 ? piece : 1)) {
          const int pc = cnt - sa < piece ? cnt - sa : piece;
          const float* prow = rows + sa * sumJ;
          const float* pfx = fx + sa;
          float* pq = qbuf + sa * Jmax;
          if (sa > 0) __syncthreads();   // the previous piece's tiles are no longer read
          if (BF) {
            // (the K extent P_n rounded up to 16 is all the tiles read)
            const int KP = bf16_row_stride(Pn);
            const int Kext = round_up(Pn, 16);
#pragma unroll 1
            for (int s = warp; s < round_up(pc, 16); s += nwarps) {
              const float* rs = prow + s * sumJ;
#pragma unroll 1
              for (int cc = lane; cc < Kext; cc += 64) {
                const int c2 = cc + 32;
                const float v0 = (s < pc && cc < Pn) ? kron_entry(rs, cdn[cc], nm1) : 0.f;
                const float v1 = (s < pc && c2 < Pn) ? kron_entry(rs, cdn[c2], nm1) : 0.f;
                Sh[s * KP + cc] = __float2bfloat16_rn(v0);
                if (c2 < Kext) Sh[s * KP + c2] = __float2bfloat16_rn(v1);
              }
            }
          } else if (full_s) {
#pragma unroll 1
            for (int s = warp; s < pc; s += nwarps) {
              const float* rs = prow + s * sumJ;
#pragma unroll 1
              for (int cc = lane; cc < Pp; cc += 64) {
                const int c2 = cc + 32;
                const float v0 = cc < Pn ? kron_entry(rs, cdn[cc], nm1) : 0.f;
                const float v1 = c2 < Pn ? kron_entry(rs, cdn[c2], nm1) : 0.f;
                Sbuf[s * Pp + cc] = v0;
                if (c2 < Pp) Sbuf[s * Pp + c2] = v1;
              }
            }
          }
          __syncthreads();
          if (BF) {
            // Tensor-core contraction: E (samples x J_n) = S (samples x P_n) .
            // G_(n)^T with BF16 operands and FP32 accumulation, mma.sync
            // m16n8k16 tiles (one warp per 16 x 8 output tile, full K).
            const int KP = bf16_row_stride(Pn);
            const int mt = round_up(pc, 16) >> 4, ntl = (Jn + 7) >> 3, ksteps = round_up(Pn, 16) >> 4;
            const int gq = lane >> 2, tq = lane & 3;
#pragma unroll 1
            for (int w = warp; w < mt * ntl; w += nwarps) {
              const int mi = w / ntl, ni = w - mi * ntl;
              const uint32_t* A0 = reinterpret_cast<const uint32_t*>(Sh + (mi * 16 + gq) * KP);
              const uint32_t* A1 = reinterpret_cast<const uint32_t*>(Sh + (mi * 16 + gq + 8) * KP);
              const uint32_t* Bq = reinterpret_cast<const uint32_t*>(GTh + (ni * 8 + gq) * KP);
              float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
              for (int ks = 0; ks < ksteps; ++ks) {
                const int kw = ks * 8 + tq;
                mma_bf16_16816(d, A0[kw], A1[kw], A0[kw + 4], A1[kw + 4], Bq[kw], Bq[kw + 4]);
              }
              const int s0 = mi * 16 + gq, j0 = ni * 8 + 2 * tq;
              if (s0 < pc) {
                if (j0 < Jn) pq[s0 * Jmax + j0] = d[0];
                if (j0 + 1 < Jn) pq[s0 * Jmax + j0 + 1] = d[1];
              }
              if (s0 + 8 < pc) {
                if (j0 < Jn) pq[(s0 + 8) * Jmax + j0] = d[2];
                if (j0 + 1 < Jn) pq[(s0 + 8) * Jmax + j0 + 1] = d[3];
              }
            }
            __syncthreads();
            // residual e_s = a_n . E_s - x_s (8 lanes per sample), contributions in place
#pragma unroll 1
            for (int base = 0; base < pc * 8; base += T) {
              const int t8 = base + tid, s = t8 >> 3, l = t8 & 7;
              const bool live = s < pc;
              float part = 0.f;
              if (live) {
                const float* an = prow + s * sumJ + mJoff[n];
#pragma unroll 1
                for (int j = l; j < Jn; j += 8) part = fmaf(an[j], pq[s * Jmax + j], part);
              }
              part += __shfl_xor_sync(0xffffffffu, part, 4);
              part += __shfl_xor_sync(0xffffffffu, part, 2);
              part += __shfl_xor_sync(0xffffffffu, part, 1);
              if (live) {
                const float e = part - pfx[s];
#pragma unroll 1
                for (int j = l; j < Jn; j += 8) pq[s * Jmax + j] *= e;
              }
            }
          } else {
            // four samples per thread when that still fills half the block,
            // else two when that fills a quarter (each sample's sums are
            // formed in the same order whatever the grouping)
            // (or the tile the caller or the batched tuner set)
            const int JL = pow2_at_least(Jn);
            const int sg = a.tile_sg > 0 ? a.tile_sg
                                         : (((pc + 3) >> 2) * JL >= (T >> 1) ? 4 : (((pc + 1) >> 1) * JL >= (T >> 2) ? 2 : 1));
            if (sg == 4)
              contract_fp32<4>(pc, Jn, Pn, Pp, full_s, GT, Sbuf, prow, sumJ, mJoff[n], cdn, nm1, pfx, pq, Jmax, tid, T);
            else if (sg == 2)
              contract_fp32<2>(pc, Jn, Pn, Pp, full_s, GT, Sbuf, prow, sumJ, mJoff[n], cdn, nm1, pfx, pq, Jmax, tid, T);
            else
              contract_fp32<1>(pc, Jn, Pn, Pp, full_s, GT, Sbuf, prow, sumJ, mJoff[n], cdn, nm1, pfx, pq, Jmax, tid, T);
          }
          if (pc <= 0) break;
        }
      }
      __syncthreads();
      // run sums (warp per run piece): the warp's 32 / J_n lane groups take
      // every sub-th sample of the run (lane j of a group sums column j), then
      // group 0 adds the groups' sums in group order; kept in the run head's
      // row of qbuf; the piece of a run begun in an earlier chunk is published
      {
        const int nsub = 32 / Jn;
        const int sub = lane / Jn, j = lane - sub * Jn;
#pragma unroll 1
        for (int h = warp; h < nheads; h += nwarps) {
          const int s0 = head[h], s1 = head[h + 1];
          float F = 0.f;
          if (sub < nsub)
#pragma unroll 1
            for (int s = s0 + sub; s < s1; s += nsub) F += qbuf[s * Jmax + j];
#pragma unroll 1
          for (int g = 1; g < nsub; ++g) {
            const float o = __shfl_sync(0xffffffffu, F, (lane + g * Jn) & 31);
            if (sub == 0) F += o;
          }
          if (lane < Jn) {
            qbuf[s0 * Jmax + lane] = F;
            if ((int)(fseg[s0] & 0xffffu) < lo) put_word(a.piece + ((unsigned)n * G + c) * (unsigned)Jmax + lane, tag, F);
          }
        }
      }
      if (CL) cluster_sync_all();   // every chunk's run pieces
      // a run begun here that continues: the pieces of chunks c+1 .. c1,
      // polled in parallel
      const uint32_t seg_last = cnt > 0 ? fseg[head[nheads - 1]] : 0u;
      const int st_last = (int)(seg_last & 0xffffu), en_last = (int)(seg_last >> 16);
      const bool owner = cnt > 0 && st_last >= lo && en_last >= hi;
      const int npc = owner ? (en_last / ph.chunk - c) * Jn : 0;
#pragma unroll 1
      for (int i = tid; i < npc; i += T) {
        const int pc = fdiv(i, mFJ[n]), j = i - pc * Jn;
        const unsigned long long* p = a.piece + ((unsigned)n * G + (unsigned)(c + 1 + pc)) * (unsigned)Jmax + j;
        pieces_sm[i] = val_of(settle(p, get_word(p), tag, ok, a));
      }
      if (BF) cp_async_wait_all();
      if (!__syncthreads_and(ok) && !CL) return;
      // the factor-row update of every run that starts in this chunk (pieces of
      // a continuing run added in chunk order), warp per run, lane j
#pragma unroll 1
      for (int h = warp; h < nheads; h += nwarps)
        if (lane < Jn) {
          const int s0 = head[h];
          const uint32_t sg = fseg[s0];
          const int st = (int)(sg & 0xffffu), en = (int)(sg >> 16);
          if (st >= lo) {
            float F = qbuf[s0 * Jmax + lane];
            if (en >= hi)
#pragma unroll 1
              for (int i = lane; i < npc; i += Jn) F += pieces_sm[i];
            const float denom = (!PLAIN && a.norm_mode == 1) ? (float)(en - st + 1) : fm;
            const unsigned row = (unsigned)fcrd[s0 * N + n];
            const float av = BF ? master[h * Jmax + lane] : rows[s0 * sumJ + mJoff[n] + lane];
            const float ga = F / denom + a.lam_a * av;
            float step = ga;
            if (!PLAIN && a.momentum != 0.f) {
              float* vp = mvA[n] + row * (unsigned)mJp[n] + lane;
              step = a.momentum * __ldcg(vp) + ga;
              if (!a.dry) __stcg(vp, step);
            }
            float nv;
            if (SNAP) {
              // the change goes to the block's end; this CTA's later modes
              // read the row as this minibatch left it (w + delta form)
              const float dl = -__fmul_rn(a.lr_a, step);
              nv = __fadd_rn(av, dl);
              a.snap_drow[(((size_t)a.snap_grp * N + n) * M + st) * Jmax + lane] = dl;
              if (lane == 0) {
                const unsigned owner = (row * 2654435761u + (unsigned)n * 40503u) % (unsigned)Gtot;
                const int at = atomicAdd(a.snap_count + owner * stride + a.snap_grp, 1);
                a.snap_list[((size_t)owner * stride + a.snap_grp) * (size_t)(N * M) + at] =
                    make_int2((int)row, (n << 16) | st);
              }
            } else {
              nv = av - a.lr_a * step;
              if (!a.dry) {
                __stcg(mA[n] + row * (unsigned)mJp[n] + lane, nv);
                if (BF) __stcg(mAb[n] + row * (unsigned)mJb[n] + lane, __bfloat16_as_ushort(__float2bfloat16_rn(nv)));
              }
            }
            if (n + 1 < N)
              put_word(a.mail + ((unsigned)n * (unsigned)M + st) * (unsigned)(Jmax + (Jmax & 1)) + lane, tag, nv);
            if (!PLAIN && probe && a.probeF) a.probeF[((unsigned)n * M + st) * kMaxJ + lane] = F;
          }
        }
    }
    buf ^= 1;
  }
  if (SNAP && iters > 0 && !snap_boundary(iters - 1)) return;

  if ((SNAP ? a.snap_cta == 0 : c == 0) && !a.dry) {
#pragma unroll 1
    for (int i = tid; i < sumJR; i += T) {
      a.B[i] = Bsm[i];
      if (a.momentum != 0.f) a.vB[i] = VBsm[i];
    }
#pragma unroll 1
    for (int lin = tid; lin < prodJ; lin += T) {
      const uint32_t packed = core_digits(lin);
      float acc = 0.f;
      for (int r = 0; r < R; ++r) {
        float prod = 1.f;
        for (int k = 0; k < N; ++k) prod *= Bsm[mBoff[k] + (int)((packed >> (5 * k)) & 31u) * R + r];
        acc += prod;
      }
      a.core[lin] = acc;
    }
  }
  // no CTA leaves (or starts its next tensor) while another may still read
  // its shared memory
  if (CL) cluster_sync_all();
}

// One tensor on the whole grid.
template <bool BF, bool PLAIN>
__global__ void __launch_bounds__(kEpochThreads, 1)
k_epoch(EpochArgs a) {
  epoch_body<BF, false, false, PLAIN>(a, gridDim.x, blockIdx.x);
}

// One tensor on one thread block cluster of gridDim.x <= 16 CTAs.
template <bool BF, bool PLAIN>
__global__ void __launch_bounds__(kEpochThreads, 1)
k_epoch_cl(EpochArgs a) {
  epoch_body<BF, false, true, PLAIN>(a, gridDim.x, (int)cooperative_groups::this_cluster().block_rank());
}

// K-snapshot form (a labelled variant of Algorithm 1's minibatch order): the
// grid is a.snap_k groups of a.snap_gk CTAs.  In every block of K consecutive
// minibatches, group q runs minibatch q of the block exactly as k_epoch would
// on snap_gk CTAs (its own exchange buffers, its own chain of core and factor
// phases), but from the model as it stood when the block began: it writes no
// parameter and records its changes.  At the block's end (two grid barriers)
// the Kruskal-column changes are added to B and the factor-row changes to A in
// minibatch order, each row by the one CTA its index hashes to, so the result
// does not depend on timing.  One chain of dependent phases per block instead
// of per minibatch.
template <bool BF, bool PLAIN>
__global__ void __launch_bounds__(kEpochThreads, 1)
k_epoch_snap(EpochArgs a) {
  __shared__ __align__(16) EpochArgs s_a;
  const int grp = (int)blockIdx.x / a.snap_gk, c = (int)blockIdx.x - grp * a.snap_gk;
  if (threadIdx.x == 0) {
    s_a = a;
    s_a.snap_grp = grp;
    s_a.snap_cta = (int)blockIdx.x;
    // this group's exchange buffers
    const size_t NJ = (size_t)a.g.N * a.g.Jmax;
    s_a.part = a.part + (size_t)grp * a.snap_gk * a.pstride;
    s_a.inbox = a.inbox + (size_t)grp * a.snap_gk * a.pstride;
    s_a.piece = a.piece + (size_t)grp * a.snap_gk * NJ;
    s_a.mail = a.mail + (size_t)grp * a.s.M * a.g.N * (a.g.Jmax + (a.g.Jmax & 1));
  }
  __syncthreads();
  epoch_body<BF, true, false, PLAIN>(s_a, a.snap_gk, c);
}

// Many independent tensors in one persistent launch: the grid is split into
// groups of CTAs [m.gstart[q], m.gstart[q+1]); group q runs the epochs of the
// tensors m.order[m.first[q] .. m.first[q+1]) one after the other, each on
// its own arguments (copied into shared memory) and exchange buffers.
template <bool BF, bool CL, bool PLAIN>
__global__ void __launch_bounds__(kEpochThreads, 1)
k_epoch_multi(MultiArgs m) {
  __shared__ __align__(16) EpochArgs s_a;
  int grp = 0;
#pragma unroll 1
  while (grp + 1 < m.groups && m.gstart[grp + 1] <= (int)blockIdx.x) ++grp;
  const int G = m.gstart[grp + 1] - m.gstart[grp], c = (int)blockIdx.x - m.gstart[grp];
#pragma unroll 1
  for (int q = m.first[grp]; q < m.first[grp + 1]; ++q) {
    const int* src = reinterpret_cast<const int*>(m.items + m.order[q]);
    int* dst = reinterpret_cast<int*>(&s_a);
#pragma unroll 1
    for (int i = threadIdx.x; i < (int)(sizeof(EpochArgs) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    epoch_body<BF, false, CL, PLAIN>(s_a, G, c);
    __syncthreads();
  }
}

#ifdef SGDT_EPOCH_PLAIN_TU
// This translation unit: the kernels specialised for the default options.
const void* epoch_plain_kernel(int kind, int precision) {
  const bool bf = precision == 1;
  switch (kind) {
    case 0: return bf ? (const void*)k_epoch<true, true> : (const void*)k_epoch<false, true>;
    case 1: return bf ? (const void*)k_epoch_cl<true, true> : (const void*)k_epoch_cl<false, true>;
    case 2: return bf ? (const void*)k_epoch_snap<true, true> : (const void*)k_epoch_snap<false, true>;
    case 3: return bf ? (const void*)k_epoch_multi<true, false, true> : (const void*)k_epoch_multi<false, false, true>;
    default: return bf ? (const void*)k_epoch_multi<true, true, true> : (const void*)k_epoch_multi<false, true, true>;
  }
}
#else
// One thread waits, through the epoch kernel's bounded wait, for a tag that
// nothing writes: the watchdog must expire and record STD_ETIMEOUT in *err.
__global__ void k_wait_probe(EpochArgs a, const unsigned long long* word) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long* p[1] = {word};
  unsigned long long w[1] = {get_word(word)};
  const uint32_t tg[1] = {1u};
  (void)wait_all<1>(p, w, tg, a);
}

bool epoch_args_plain(const EpochArgs& a) {
  return a.momentum == 0.f && a.norm_mode == 0 && (a.probe_batch < a.b0 || a.probe_batch >= a.b1);
}

namespace {

// The kernel of each form: the general one (every option) or the one
// specialised for the default options (compiled in its own translation unit).
const void* kernel_for(int precision, bool plain = false) {
  if (plain) return epoch_plain_kernel(0, precision);
  return precision == 1 ? (const void*)k_epoch<true, false> : (const void*)k_epoch<false, false>;
}

const void* multi_kernel_for(int precision, bool cl = false, bool plain = false) {
  if (plain) return epoch_plain_kernel(cl ? 4 : 3, precision);
  if (cl)
    return precision == 1 ? (const void*)k_epoch_multi<true, true, false> : (const void*)k_epoch_multi<false, true, false>;
  return precision == 1 ? (const void*)k_epoch_multi<true, false, false> : (const void*)k_epoch_multi<false, false, false>;
}

const void* cl_kernel_for(int precision, bool plain = false) {
  if (plain) return epoch_plain_kernel(1, precision);
  return precision == 1 ? (const void*)k_epoch_cl<true, false> : (const void*)k_epoch_cl<false, false>;
}

const void* snap_kernel_for(int precision, bool plain = false) {
  if (plain) return epoch_plain_kernel(2, precision);
  return precision == 1 ? (const void*)k_epoch_snap<true, false> : (const void*)k_epoch_snap<false, false>;
}

// Blocks of one kernel resident per SM at this shared memory.
int blocks_per_sm(const void* fn, size_t smem) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kEpochThreads, smem) != cudaSuccess) return 0;
  return per;
}

}  // namespace

int epoch_chunk_cap(const Geometry& g) {
  (void)g;
  return kMaxChunk;
}

int epoch_payload_floats(const Geometry& g) { return payload_max(g); }

bool epoch_gram_fits(const Geometry& g) {
  return g.sumJ < 256;   // Kronecker columns address a sample's rows with 8-bit offsets
}

size_t epoch_smem_bytes(const Geometry& g, int chunk_max, int ctas, int precision) {
  return (size_t)smem_layout(g, chunk_max, ctas, precision).total_words * sizeof(float);
}

// Attributes and occupancy cover both kernels of a form (general and
// specialised), so either can be launched on the same layout.
cudaError_t epoch_kernel_setup(int precision, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(kernel_for(precision), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel_for(precision, true), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

int epoch_max_ctas(int precision, size_t smem) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const int p0 = blocks_per_sm(kernel_for(precision), smem), p1 = blocks_per_sm(kernel_for(precision, true), smem);
  return (p0 < p1 ? p0 : p1) * sms;
}

cudaError_t launch_epoch(const EpochArgs& a, int ctas, size_t smem, cudaStream_t st) {
  EpochArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(kernel_for(a.precision, epoch_args_plain(a)), dim3(ctas), dim3(kEpochThreads),
                                     args, smem, st);
}

cudaError_t epoch_snap_setup(int precision, size_t smem) {
  cudaError_t e =
      cudaFuncSetAttribute(snap_kernel_for(precision), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(snap_kernel_for(precision, true), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

int epoch_snap_max_ctas(int precision, size_t smem) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const int p0 = blocks_per_sm(snap_kernel_for(precision), smem);
  const int p1 = blocks_per_sm(snap_kernel_for(precision, true), smem);
  return (p0 < p1 ? p0 : p1) * sms;
}

cudaError_t launch_epoch_snap(const EpochArgs& a, int ctas, size_t smem, cudaStream_t st) {
  EpochArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(snap_kernel_for(a.precision, epoch_args_plain(a)), dim3(ctas),
                                     dim3(kEpochThreads), args, smem, st);
}

cudaError_t launch_wait_probe(unsigned long long watchdog_ns, int* err, const unsigned long long* word,
                              cudaStream_t st) {
  EpochArgs a{};
  a.err = err;
  a.watchdog_ns = watchdog_ns;
  k_wait_probe<<<1, 32, 0, st>>>(a, word);
  return cudaGetLastError();
}

cudaError_t epoch_multi_setup(int precision, size_t smem) {
  cudaError_t e =
      cudaFuncSetAttribute(multi_kernel_for(precision), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(multi_kernel_for(precision, false, true), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  return e;
}

int epoch_multi_max_ctas(int precision, size_t smem) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const int p0 = blocks_per_sm(multi_kernel_for(precision), smem);
  const int p1 = blocks_per_sm(multi_kernel_for(precision, false, true), smem);
  return (p0 < p1 ? p0 : p1) * sms;
}

// Cooperative launch through the launch-attribute form, which stream capture
// records as a cooperative kernel node.
cudaError_t launch_epoch_multi(const MultiArgs& m, int precision, int ctas, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kEpochThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MultiArgs copy = m;
  void* args[] = {&copy};
  return cudaLaunchKernelExC(&cfg, multi_kernel_for(precision, false, m.plain != 0), args);
}

// ---------------------------------------------------------------------------
// Cluster form (groups of 2..16 CTAs as one thread block cluster).
// ---------------------------------------------------------------------------
namespace {

cudaError_t cl_attrs(const void* fn, size_t smem, int csize) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && csize > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaLaunchConfig_t cl_config(int ctas, int csize, size_t smem, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kEpochThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

bool epoch_cluster_size_ok(int csize) { return csize == 2 || csize == 4 || csize == 8 || csize == 16; }

size_t epoch_smem_bytes_cl(const Geometry& g, int chunk_max, int ctas, int precision) {
  return (size_t)smem_layout(g, chunk_max, ctas, precision, 1).total_words * sizeof(float);
}

// Clusters of csize CTAs that can be resident at once (0: none), for both
// kernels of the form.
int epoch_cl_max_clusters(int precision, bool multi, size_t smem, int csize) {
  int best = -1;
  for (int plain = 0; plain < 2; ++plain) {
    const void* fn = multi ? multi_kernel_for(precision, true, plain != 0) : cl_kernel_for(precision, plain != 0);
    if (cl_attrs(fn, smem, csize) != cudaSuccess) return 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cl_config(csize, csize, smem, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = best < 0 || n < best ? n : best;
  }
  return best;
}

cudaError_t launch_epoch_cl(const EpochArgs& a, int ctas, size_t smem, cudaStream_t st) {
  const void* fn = cl_kernel_for(a.precision, epoch_args_plain(a));
  cudaError_t e = cl_attrs(fn, smem, ctas);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cl_config(ctas, ctas, smem, st, attr);
  EpochArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// Groups of csize CTAs, each one cluster; gstart[q] = q * csize.  Not
// cooperative: clusters are independent, and a cluster's CTAs are resident
// together by construction.
cudaError_t launch_epoch_multi_cl(const MultiArgs& m, int precision, int csize, size_t smem, cudaStream_t st) {
  const void* fn = multi_kernel_for(precision, true, m.plain != 0);
  cudaError_t e = cl_attrs(fn, smem, csize);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cl_config(m.groups * csize, csize, smem, st, attr);
  MultiArgs copy = m;
  void* args[] = {&copy};
  return cudaLaunchKernelExC(&cfg, fn, args);
}
#endif  // SGDT_EPOCH_PLAIN_TU

}  // namespace sgdt
