// Host side of the C ABI declared in include/sgd_tucker.h: argument checks,
// device memory of a context, and the launch sequence of each call.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "sgdt_internal.cuh"

using namespace sgdt;

namespace {

thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(STD_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
  }
  return set_error(STD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define STD_CUDA(call, what)                       \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_error(e_, what); \
  } while (0)

}  // namespace

int sgdt::record_error(int code, const std::string& msg) { return set_error(code, msg); }

struct std_ctx {
  Geometry g{};
  std_options opt{};
  cudaStream_t stream = nullptr;
  int sms = 0;
  int64_t nnz = 0;
  int cs = 0;                       // 32-bit words per packed COO record
  uint32_t* coo = nullptr;
  float* A[kMaxN] = {};
  uint16_t* Ab[kMaxN] = {};   // BF16 mirrors (precision 1)
  float* vA[kMaxN] = {};      // momentum velocities of the factor rows (momentum != 0)
  float* vB = nullptr;        // momentum velocities of the Kruskal columns
  float* B = nullptr;
  float* core = nullptr;
  int* err = nullptr;
  unsigned long long* bar = nullptr;
  // schedule of the current epoch
  Schedule sched{};
  void* sched_mem = nullptr;
  size_t sched_bytes = 0;
  int64_t sched_epoch = -1;
  int sched_M = 0;
  int64_t sched_b0 = 0, sched_b1 = 0;   // minibatches the schedule buffer holds
  // epoch exchange words (tagged; see k_epoch)
  unsigned long long* part = nullptr;
  size_t part_words = 0;
  unsigned long long* inbox = nullptr;
  size_t inbox_words = 0;
  unsigned long long* piece = nullptr;
  size_t piece_words = 0;
  unsigned long long* mail = nullptr;
  size_t mail_words = 0;
  uint32_t tag_base = 1;
  // K-snapshot form: recorded changes and the per-CTA lists of rows to apply
  float* snap_dB = nullptr;
  size_t snap_dB_floats = 0;
  float* snap_drow = nullptr;
  size_t snap_drow_floats = 0;
  int2* snap_list = nullptr;
  size_t snap_list_items = 0;
  int* snap_count = nullptr;
  size_t snap_count_items = 0;
  // probe
  float* probe_mem = nullptr;
  size_t probe_floats = 0;
  // staging for host inputs of predict / rmse
  void* stage = nullptr;
  size_t stage_bytes = 0;
  double* rpart = nullptr;
  int rpart_blocks = 0;
  double* result = nullptr;
  int64_t epoch = 0;
  int64_t cursor = 0;               // next minibatch of the epoch in progress (batched steps); 0 = at a boundary
  int32_t cursor_M = 0;             // minibatch size of that epoch
  size_t allocated = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evm = nullptr;
  // per-segment timing of a timed call: before the sampler/tiler, between
  // it and the update kernel, after the update kernel (3 events a segment)
  std::vector<cudaEvent_t> seg_ev;
  int seg_count = 0;
};

namespace {

int dev_alloc(std_ctx* c, void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->opt.hbm_budget_bytes && c->allocated + bytes > c->opt.hbm_budget_bytes)
    return set_error(STD_ENOMEM, std::string(what) + ": HBM budget exceeded");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_error(e, what);
  }
  c->allocated += bytes;
  return STD_OK;
}

void dev_free(std_ctx* c, void* p, size_t bytes) {
  if (p) {
    cudaFree(p);
    c->allocated -= (bytes == 0 ? 16 : bytes);
  }
}

int read_err(std_ctx* c, const char* what) {
  int h = 0;
  STD_CUDA(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), what);
  STD_CUDA(cudaStreamSynchronize(c->stream), what);
  if (h != 0) {
    STD_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), what);
    STD_CUDA(cudaStreamSynchronize(c->stream), what);
    if (h == STD_EINVAL) return set_error(STD_EINVAL, std::string(what) + ": coordinate outside [0, I_n)");
    if (h == STD_ETIMEOUT) return set_error(STD_ETIMEOUT, std::string(what) + ": grid barrier watchdog expired");
    return set_error(h, std::string(what) + ": device error");
  }
  return STD_OK;
}

int ensure_stage(std_ctx* c, size_t bytes) {
  if (bytes <= c->stage_bytes) return STD_OK;
  dev_free(c, c->stage, c->stage_bytes);
  c->stage = nullptr;
  c->stage_bytes = 0;
  int rc = dev_alloc(c, &c->stage, bytes, "staging buffer");
  if (rc) return rc;
  c->stage_bytes = bytes;
  return STD_OK;
}

int payload_floats(const Geometry& g) { return epoch_payload_floats(g); }

// Schedules minibatches [bs, be) of the current epoch at minibatch size M
// (sampler and tiler) into the context's schedule buffer, unless it holds
// them already.  Position t is stored at index t - bs * M (Schedule.b_first).
int ensure_schedule_range(std_ctx* c, int M, int64_t bs, int64_t be) {
  if (c->sched_mem && c->sched_M == M && c->sched_epoch == c->epoch && c->sched_b0 <= bs && be <= c->sched_b1)
    return STD_OK;
  const int N = c->g.N;
  const int64_t npad = (be - bs) * M;
  const size_t words = (size_t)npad * schedule_words_per_position(N);
  const size_t bytes = words * 4;
  if (bytes > c->sched_bytes) {
    dev_free(c, c->sched_mem, c->sched_bytes);
    c->sched_mem = nullptr;
    c->sched_bytes = 0;
    c->sched_b0 = c->sched_b1 = 0;
    int rc = dev_alloc(c, &c->sched_mem, bytes, "epoch schedule");
    if (rc) return rc;
    c->sched_bytes = bytes;
  }
  int32_t* base = static_cast<int32_t*>(c->sched_mem);
  Schedule s{};
  s.crd = base;
  s.val = reinterpret_cast<float*>(base + (size_t)npad * N * N);
  s.pos = base + (size_t)npad * (N * N + N);
  s.seg = reinterpret_cast<uint32_t*>(base + (size_t)npad * (N * N + 2 * N));
  s.sid = base + (size_t)npad * (N * N + 3 * N);
  s.link = s.sid + (size_t)npad;
  s.rsp = s.link + (size_t)npad * (N * (N - 1) / 2);
  s.npad = npad;
  s.n = c->nnz;
  s.M = M;
  s.b_first = bs;
  const Feistel f = make_feistel((uint64_t)c->nnz, c->opt.seed_sched, (uint64_t)c->epoch);
  STD_CUDA(launch_schedule(c->g, c->coo, c->cs, f, s, bs, be, c->stream), "sampler/tiler launch");
  c->sched = s;
  c->sched_M = M;
  c->sched_epoch = c->epoch;
  c->sched_b0 = bs;
  c->sched_b1 = be;
  return STD_OK;
}

// The whole epoch's schedule (batched launches run whole epochs or long
// stretches of one).
int ensure_schedule(std_ctx* c, int M) {
  const int64_t nb = (c->nnz + M - 1) / M;
  return ensure_schedule_range(c, M, 0, nb);
}

// Minibatches per schedule segment of std_sgd_epoch / std_sgd_batches: about
// 2^22 sampled positions (the schedule of one segment is ~400 MB for a 3-order
// tensor instead of the epoch's; a segment of 1,024 minibatches of 4,096 keeps
// the sampler/tiler's one-CTA-per-minibatch launch several CTAs deep per SM),
// a multiple of K in the K-snapshot form so that blocks never straddle segments.
int64_t segment_batches(int M, int K) {
  int64_t S = (1LL << 22) / M;
  if (S < 1) S = 1;
  if (K >= 2) S = S < K ? K : S / K * K;
  return S;
}

cudaEvent_t seg_event(std_ctx* c, size_t i) {
  while (c->seg_ev.size() <= i) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->seg_ev.push_back(e);
  }
  return c->seg_ev[i];
}

int choose_ctas(std_ctx* c, int M, int* ctas, int* chunk_max, size_t* smem) {
  const int payload = payload_floats(c->g);
  if (payload > kMaxCorePayload)
    return set_error(STD_EUNSUPPORTED, "core reduction payload R*J + R(R-1)/2*J(J+1)/2 exceeds 8192 floats");
  if (!epoch_gram_fits(c->g))
    return set_error(STD_EUNSUPPORTED, "core reduction tiles exceed the epoch kernel's per-thread limit");
  const int cap = epoch_chunk_cap(c->g);
  int G = c->opt.ctas;
  if (G <= 0) {
    G = (M + 15) / 16;
    if (G > c->sms) G = c->sms;
    const int need = (M + cap - 1) / cap;
    if (G < need) G = need;
  }
  if (G < 1) G = 1;
  if (G > kMaxEpochCtas) {
    if (c->opt.ctas > 0) return set_error(STD_EINVAL, "requested CTA count exceeds the epoch kernel's limit (256)");
    G = kMaxEpochCtas;
  }
  int ch = (M + G - 1) / G;
  if (ch > cap) return set_error(STD_EUNSUPPORTED, "minibatch too large for the CTA count at these ranks");
  size_t sm = epoch_smem_bytes(c->g, ch, G, c->opt.precision);
  if (sm > 227 * 1024) return set_error(STD_EUNSUPPORTED, "shape needs more shared memory than a CTA has");
  STD_CUDA(epoch_kernel_setup(c->opt.precision, sm), "epoch kernel attributes");
  const int maxG = epoch_max_ctas(c->opt.precision, sm);
  if (maxG < 1) return set_error(STD_EUNSUPPORTED, "epoch kernel cannot be resident");
  if (G > maxG) {
    if (c->opt.ctas > 0) return set_error(STD_EINVAL, "requested CTA count exceeds co-resident capacity");
    G = maxG;
    ch = (M + G - 1) / G;
    if (ch > cap) return set_error(STD_EUNSUPPORTED, "minibatch too large for the co-resident CTAs at these ranks");
    sm = epoch_smem_bytes(c->g, ch, G, c->opt.precision);
    if (sm > 227 * 1024) return set_error(STD_EUNSUPPORTED, "shape needs more shared memory than a CTA has");
    STD_CUDA(epoch_kernel_setup(c->opt.precision, sm), "epoch kernel attributes");
  }
  *ctas = G;
  *chunk_max = ch;
  *smem = sm;
  return STD_OK;
}

// Grows one exchange buffer to at least `words` tagged words; a new buffer
// starts zeroed (tag 0, which no exchange uses).
int ensure_words(std_ctx* c, unsigned long long** p, size_t* have, size_t words, const char* what) {
  if (words <= *have) return STD_OK;
  dev_free(c, *p, *have * 8);
  *p = nullptr;
  *have = 0;
  int rc = dev_alloc(c, (void**)p, words * 8, what);
  if (rc) return rc;
  *have = words;
  STD_CUDA(cudaMemsetAsync(*p, 0, words * 8, c->stream), what);
  return STD_OK;
}

int exchange_pstride(int payload) { return (payload + 7) & ~7; }

int ensure_scratch(std_ctx* c, int G, int payload, int M) {
  const size_t ps = (size_t)exchange_pstride(payload);
  const size_t NJ = (size_t)c->g.N * c->g.Jmax;
  int rc = ensure_words(c, &c->part, &c->part_words, (size_t)G * ps, "core partials");
  if (!rc) rc = ensure_words(c, &c->inbox, &c->inbox_words, (size_t)G * ps, "core reduction copies");
  if (!rc) rc = ensure_words(c, &c->piece, &c->piece_words, (size_t)G * NJ, "run pieces");
  // row slots: a stride of Jmax rounded up to even keeps word pairs 16-byte aligned
  const size_t NJ2 = (size_t)c->g.N * (c->g.Jmax + (c->g.Jmax & 1));
  if (!rc) rc = ensure_words(c, &c->mail, &c->mail_words, (size_t)M * NJ2, "row slots");
  return rc;
}

// Tags of one launch over `batches` minibatches: tag_base + 8 (b - b0) + n.
// Before the 32-bit sequence would wrap, every exchange word is cleared and
// the sequence restarts at 1, so a stale word never carries a live tag.
int reserve_tags(std_ctx* c, int64_t batches, uint32_t* base) {
  const uint64_t span = (uint64_t)batches * 8ULL + 8ULL;
  if (span >= 0x80000000ULL) return set_error(STD_EUNSUPPORTED, "too many minibatches in one launch");
  if ((uint64_t)c->tag_base + span >= 0xFFFFFFF0ULL) {
    STD_CUDA(cudaMemsetAsync(c->part, 0, c->part_words * 8, c->stream), "exchange reset");
    STD_CUDA(cudaMemsetAsync(c->inbox, 0, c->inbox_words * 8, c->stream), "exchange reset");
    STD_CUDA(cudaMemsetAsync(c->piece, 0, c->piece_words * 8, c->stream), "exchange reset");
    STD_CUDA(cudaMemsetAsync(c->mail, 0, c->mail_words * 8, c->stream), "exchange reset");
    c->tag_base = 1;
  }
  *base = c->tag_base;
  c->tag_base += (uint32_t)span;
  return STD_OK;
}

int check_hyper(float lr_a, float lr_b, float lam_a, float lam_b, int32_t M) {
  if (!(std::isfinite(lr_a) && std::isfinite(lr_b) && std::isfinite(lam_a) && std::isfinite(lam_b)))
    return set_error(STD_EINVAL, "learning rates and lambdas must be finite");
  if (M < 1) return set_error(STD_EINVAL, "minibatch must be >= 1");
  if (M > STD_MAX_MINIBATCH) return set_error(STD_EUNSUPPORTED, "minibatch exceeds STD_MAX_MINIBATCH");
  return STD_OK;
}

// Kernel arguments of minibatches [b0, b1) of the context's current schedule.
EpochArgs epoch_args(std_ctx* c, float lr_a, float lr_b, float lam_a, float lam_b, int64_t b0, int64_t b1,
                     int chunk, uint32_t tag_base) {
  EpochArgs a{};
  a.g = c->g;
  for (int n = 0; n < c->g.N; ++n) {
    a.A[n] = c->A[n];
    a.Ab[n] = c->Ab[n];
    a.vA[n] = c->vA[n];
  }
  a.precision = c->opt.precision;
  a.B = c->B;
  a.core = c->core;
  a.s = c->sched;
  a.b0 = b0;
  a.b1 = b1;
  a.lr_a = lr_a;
  a.lr_b = lr_b;
  a.lam_a = lam_a;
  a.lam_b = lam_b;
  a.norm_mode = c->opt.norm_mode;
  a.contraction = c->opt.contraction;
  a.tile_sg = c->opt.tile;
  a.momentum = c->opt.momentum;
  a.vB = c->vB;
  a.chunk_max = chunk;
  a.tag_base = tag_base;
  a.part = c->part;
  a.inbox = c->inbox;
  a.piece = c->piece;
  a.mail = c->mail;
  a.pstride = exchange_pstride(payload_floats(c->g));
  a.bar = c->bar;
  a.err = c->err;
  a.watchdog_ns = c->opt.watchdog_ns ? c->opt.watchdog_ns : 2000000000ULL;
  a.probe_batch = -1;
  return a;
}

// CTAs per group of the K-snapshot form: K groups, each of the size the
// library would give one minibatch on 1/K of the GPU, at least enough for the
// kernel's chunk limit.
int choose_snap_ctas(std_ctx* c, int M, int K, int* gk, int* chunk_max, size_t* smem) {
  const int payload = payload_floats(c->g);
  if (payload > kMaxCorePayload)
    return set_error(STD_EUNSUPPORTED, "core reduction payload R*J + R(R-1)/2*J(J+1)/2 exceeds 8192 floats");
  if (!epoch_gram_fits(c->g))
    return set_error(STD_EUNSUPPORTED, "core reduction tiles exceed the epoch kernel's per-thread limit");
  // a group may take up to 256 samples per CTA (the strict form stops at
  // 128, where more CTAs always pay); shared memory is checked below
  const int cap = 2 * epoch_chunk_cap(c->g);
  const int need = (M + cap - 1) / cap;
  int G = c->opt.ctas > 0 ? c->opt.ctas / K : std::min(c->sms / K, (M + 15) / 16);
  if (G < need) G = need;
  if (G < 1) G = 1;
  if ((int64_t)G * K > kMaxEpochCtas || G * K > c->sms)
    return set_error(STD_EUNSUPPORTED, "K-snapshot: K groups of ceil(M/256) CTAs exceed the GPU");
  const int ch = (M + G - 1) / G;
  const size_t sm = epoch_smem_bytes(c->g, ch, G, c->opt.precision);
  if (sm > 227 * 1024) return set_error(STD_EUNSUPPORTED, "shape needs more shared memory than a CTA has");
  STD_CUDA(epoch_snap_setup(c->opt.precision, sm), "snapshot kernel attributes");
  if (epoch_snap_max_ctas(c->opt.precision, sm) < G * K)
    return set_error(STD_EUNSUPPORTED, "K-snapshot: the groups cannot all be resident");
  *gk = G;
  *chunk_max = ch;
  *smem = sm;
  return STD_OK;
}

template <typename T>
int ensure_items(std_ctx* c, T** p, size_t* have, size_t items, const char* what) {
  if (items <= *have) return STD_OK;
  dev_free(c, *p, *have * sizeof(T));
  *p = nullptr;
  *have = 0;
  int rc = dev_alloc(c, (void**)p, items * sizeof(T), what);
  if (rc) return rc;
  *have = items;
  return STD_OK;
}

// Runs minibatches [b0, b1) of the current epoch, Algorithm 1's order or the
// K-snapshot form (std_options.snapshot = K), segment after segment: the
// sampler/tiler schedules a segment, then one cooperative launch runs it.
// With `timed`, three events per segment are recorded (seg_ev).
int run_batches(std_ctx* c, float lr_a, float lr_b, float lam_a, float lam_b, int32_t M, int64_t b0, int64_t b1,
                bool probe, bool timed) {
  const int K = c->opt.snapshot >= 2 ? c->opt.snapshot : 1;
  const int N = c->g.N;
  int G = 0, Gk = 0, chunk = 0;
  size_t smem = 0;
  int rc = STD_OK;
  if (K >= 2) {
    rc = choose_snap_ctas(c, M, K, &Gk, &chunk, &smem);
    G = Gk * K;
  } else {
    rc = choose_ctas(c, M, &G, &chunk, &smem);
  }
  if (rc) return rc;
  // groups of 2..16 CTAs run as one thread block cluster (same results as the
  // cooperative form, exchanges through cluster barriers and shared memory)
  bool cl = false;
  if (K < 2 && epoch_cluster_size_ok(G)) {
    const size_t smc = epoch_smem_bytes_cl(c->g, chunk, G, c->opt.precision);
    if (smc <= 227 * 1024 && epoch_cl_max_clusters(c->opt.precision, false, smc, G) >= 1) {
      cl = true;
      smem = smc;
    }
  }
  rc = ensure_scratch(c, G, payload_floats(c->g), M * K);
  if (rc) return rc;
  if (K >= 2) {
    int sumJR = 0;
    for (int n = 0; n < N; ++n) sumJR += c->g.J[n] * c->g.R;
    rc = ensure_items(c, &c->snap_dB, &c->snap_dB_floats, (size_t)K * sumJR, "snapshot column changes");
    if (!rc)
      rc = ensure_items(c, &c->snap_drow, &c->snap_drow_floats, (size_t)K * N * M * c->g.Jmax, "snapshot row changes");
    if (!rc) rc = ensure_items(c, &c->snap_list, &c->snap_list_items, (size_t)G * K * N * M, "snapshot row lists");
    if (!rc) rc = ensure_items(c, &c->snap_count, &c->snap_count_items, (size_t)G * K, "snapshot list counts");
    if (rc) return rc;
  }
  float* pV = nullptr;
  float* pF = nullptr;
  if (probe) {
    const size_t need = (size_t)N * c->g.R * kMaxJ + (size_t)N * M * kMaxJ;
    rc = ensure_items(c, &c->probe_mem, &c->probe_floats, need, "gradient probe");
    if (rc) return rc;
    STD_CUDA(cudaMemsetAsync(c->probe_mem, 0, need * 4, c->stream), "probe clear");
    pV = c->probe_mem;
    pF = c->probe_mem + (size_t)N * c->g.R * kMaxJ;
  }
  const int64_t S = segment_batches(M, K);
  c->seg_count = 0;
  for (int64_t sb = b0; sb < b1; sb += S) {
    const int64_t se = b1 - sb < S ? b1 : sb + S;
    const size_t ei = 3 * (size_t)c->seg_count;
    if (timed) {
      cudaEvent_t e0 = seg_event(c, ei), e1 = seg_event(c, ei + 1), e2 = seg_event(c, ei + 2);
      if (!e0 || !e1 || !e2) return set_error(STD_ECUDA, "event create");
      STD_CUDA(cudaEventRecord(e0, c->stream), "event");
    }
    rc = ensure_schedule_range(c, M, sb, se);
    if (rc) return rc;
    if (timed) STD_CUDA(cudaEventRecord(c->seg_ev[ei + 1], c->stream), "event");
    uint32_t tag_base = 0;
    rc = reserve_tags(c, se - sb, &tag_base);
    if (rc) return rc;
    EpochArgs a = epoch_args(c, lr_a, lr_b, lam_a, lam_b, sb, se, chunk, tag_base);
    a.probe_batch = probe && sb == b0 ? b0 : -1;
    a.probeV = pV;
    a.probeF = pF;
    STD_CUDA(cudaMemsetAsync(c->bar, 0, sizeof(unsigned long long), c->stream), "barrier clear");
    if (K >= 2) {
      a.snap_k = K;
      a.snap_gk = Gk;
      a.snap_dB = c->snap_dB;
      a.snap_drow = c->snap_drow;
      a.snap_list = c->snap_list;
      a.snap_count = c->snap_count;
      STD_CUDA(cudaMemsetAsync(c->snap_count, 0, (size_t)G * K * sizeof(int), c->stream), "snapshot counts");
      STD_CUDA(launch_epoch_snap(a, G, smem, c->stream), "snapshot kernel launch");
    } else if (cl) {
      STD_CUDA(launch_epoch_cl(a, G, smem, c->stream), "cluster epoch kernel launch");
    } else {
      STD_CUDA(launch_epoch(a, G, smem, c->stream), "epoch kernel launch");
    }
    if (timed) STD_CUDA(cudaEventRecord(c->seg_ev[ei + 2], c->stream), "event");
    c->seg_count += 1;
  }
  return read_err(c, K >= 2 ? "snapshot kernel" : "epoch kernel");
}

const int32_t* stage_coords(std_ctx* c, const int32_t* coords, const float* values, int64_t k,
                            const float** dvalues, int* rc) {
  *rc = STD_OK;
  *dvalues = values;
  if (c->opt.ptr_kind == 1) return coords;
  const size_t cb = (size_t)k * c->g.N * 4;
  const size_t vb = values ? (size_t)k * 4 : 0;
  *rc = ensure_stage(c, cb + vb + 16);
  if (*rc) return nullptr;
  int32_t* dc = static_cast<int32_t*>(c->stage);
  cudaError_t e = cudaMemcpyAsync(dc, coords, cb, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess && values) {
    float* dv = reinterpret_cast<float*>(dc + (size_t)k * c->g.N);
    e = cudaMemcpyAsync(dv, values, vb, cudaMemcpyDefault, c->stream);
    *dvalues = dv;
  }
  if (e != cudaSuccess) {
    *rc = cuda_error(e, "staging copy");
    return nullptr;
  }
  return dc;
}

}  // namespace

extern "C" {

void std_default_options(std_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->r_core = 5;
  opt->precision = 0;
  opt->norm_mode = 0;
  opt->init_mode = 1;
  opt->init_mu = 0.5;
  opt->init_sigma = 0.1;
  opt->seed_init = 1;
  opt->seed_sched = 2;
  opt->ptr_kind = 0;
  opt->ctas = 0;
  opt->stream = nullptr;
  opt->watchdog_ns = 0;
  opt->hbm_budget_bytes = 0;
  opt->contraction = 0;
  opt->momentum = 0.f;
  opt->snapshot = 0;
}

const char* std_last_error(void) { return g_last_error.c_str(); }

int std_destroy(std_ctx* c) {
  if (!c) return STD_OK;
  cudaStreamSynchronize(c->stream);
  for (int n = 0; n < kMaxN; ++n) {
    if (c->A[n]) cudaFree(c->A[n]);
    if (c->Ab[n]) cudaFree(c->Ab[n]);
    if (c->vA[n]) cudaFree(c->vA[n]);
  }
  if (c->vB) cudaFree(c->vB);
  void* ptrs[] = {c->coo, c->B, c->core, c->err, c->bar, c->sched_mem, c->part, c->inbox,
                  c->piece, c->mail, c->probe_mem, c->stage, c->rpart, c->result,
                  c->snap_dB, c->snap_drow, c->snap_list, c->snap_count};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->evm) cudaEventDestroy(c->evm);
  for (cudaEvent_t e : c->seg_ev) cudaEventDestroy(e);
  delete c;
  return STD_OK;
}

int std_create(std_ctx** out, int32_t order, const int64_t* mode_sizes, const int32_t* ranks, int64_t nnz,
               const int32_t* indices, const float* values, const std_options* opt_in) {
  if (!out) return set_error(STD_EINVAL, "out is NULL");
  *out = nullptr;
  std_options opt;
  std_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (order < 2) return set_error(STD_EINVAL, "order must be >= 2");
  if (order > STD_MAX_ORDER) return set_error(STD_EUNSUPPORTED, "order exceeds STD_MAX_ORDER");
  if (!mode_sizes || !ranks || !indices || !values) return set_error(STD_EINVAL, "NULL array argument");
  if (nnz < 1 || nnz >= 2147483647LL) return set_error(STD_EINVAL, "nnz must be in [1, 2^31 - 1)");
  if (opt.r_core < 1) return set_error(STD_EINVAL, "r_core must be >= 1");
  if (opt.r_core > STD_MAX_RANK) return set_error(STD_EUNSUPPORTED, "r_core exceeds STD_MAX_RANK");
  if (opt.precision != 0 && opt.precision != 1) return set_error(STD_EINVAL, "precision must be 0 or 1");
  if (opt.norm_mode != 0 && opt.norm_mode != 1) return set_error(STD_EINVAL, "norm_mode must be 0 or 1");
  if (opt.init_mode != 0 && opt.init_mode != 1) return set_error(STD_EINVAL, "init_mode must be 0 or 1");
  if (opt.ptr_kind != 0 && opt.ptr_kind != 1) return set_error(STD_EINVAL, "ptr_kind must be 0 or 1");
  if (opt.ctas < 0) return set_error(STD_EINVAL, "ctas must be >= 0");
  if (opt.contraction != 0 && opt.contraction != 1) return set_error(STD_EINVAL, "contraction must be 0 or 1");
  if (!(opt.momentum >= 0.f && opt.momentum < 1.f)) return set_error(STD_EINVAL, "momentum must be in [0, 1)");
  if (opt.tile != 0 && opt.tile != 1 && opt.tile != 2 && opt.tile != 4)
    return set_error(STD_EINVAL, "tile must be 0, 1, 2 or 4");
  if (opt.snapshot < 0) return set_error(STD_EINVAL, "snapshot must be >= 0");
  if (opt.snapshot > 64) return set_error(STD_EUNSUPPORTED, "snapshot exceeds 64 minibatches per block");
  if (opt.snapshot >= 2 && opt.momentum != 0.f)
    return set_error(STD_EINVAL, "the K-snapshot form is defined without momentum");
  Geometry g{};
  g.N = order;
  g.R = opt.r_core;
  int64_t prodJ = 1;
  int sumJ = 0, Jmax = 0, boff = 0;
  for (int n = 0; n < order; ++n) {
    if (mode_sizes[n] < 1 || mode_sizes[n] >= 2147483647LL) return set_error(STD_EINVAL, "mode size out of range");
    if (ranks[n] < 1) return set_error(STD_EINVAL, "rank must be >= 1");
    if (ranks[n] > STD_MAX_RANK) return set_error(STD_EUNSUPPORTED, "rank exceeds STD_MAX_RANK");
    g.I[n] = mode_sizes[n];
    g.J[n] = ranks[n];
    g.Jp[n] = (ranks[n] + 3) & ~3;
    g.Jb[n] = (ranks[n] + 7) & ~7;
    g.boff[n] = boff;
    boff += ranks[n] * g.R;
    g.joff[n] = sumJ;
    sumJ += ranks[n];
    g.gstride[n] = (int)prodJ;
    prodJ *= ranks[n];
    if (ranks[n] > Jmax) Jmax = ranks[n];
    if (prodJ > STD_MAX_CORE) return set_error(STD_EUNSUPPORTED, "prod J_n exceeds STD_MAX_CORE");
  }
  g.sumJ = sumJ;
  g.prodJ = (int)prodJ;
  g.Jmax = Jmax;

  std_ctx* c = new std_ctx();
  c->g = g;
  c->opt = opt;
  c->stream = static_cast<cudaStream_t>(opt.stream);
  c->nnz = nnz;
  c->cs = (order + 1 <= 4) ? 4 : 8;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    int rc = cuda_error(e, "device query");
    delete c;
    return rc;
  }
  int rc = STD_OK;
#define TRY(x)                 \
  do {                         \
    rc = (x);                  \
    if (rc) {                  \
      std_destroy(c);          \
      return rc;               \
    }                          \
  } while (0)
  TRY(cudaEventCreate(&c->ev0) == cudaSuccess ? STD_OK : cuda_error(cudaGetLastError(), "event create"));
  TRY(cudaEventCreate(&c->ev1) == cudaSuccess ? STD_OK : cuda_error(cudaGetLastError(), "event create"));
  TRY(cudaEventCreate(&c->evm) == cudaSuccess ? STD_OK : cuda_error(cudaGetLastError(), "event create"));
  TRY(dev_alloc(c, (void**)&c->err, 16, "error word"));
  TRY(dev_alloc(c, (void**)&c->bar, 16, "barrier word"));
  TRY(dev_alloc(c, (void**)&c->result, 16, "result"));
  TRY(dev_alloc(c, (void**)&c->coo, (size_t)nnz * c->cs * 4, "COO"));
  for (int n = 0; n < order; ++n) TRY(dev_alloc(c, (void**)&c->A[n], (size_t)g.I[n] * g.Jp[n] * 4, "factor matrix"));
  if (opt.precision == 1)
    for (int n = 0; n < order; ++n)
      TRY(dev_alloc(c, (void**)&c->Ab[n], (size_t)g.I[n] * g.Jb[n] * 2, "BF16 factor mirror"));
  TRY(dev_alloc(c, (void**)&c->B, (size_t)boff * 4, "Kruskal matrices"));
  if (opt.momentum != 0.f) {
    for (int n = 0; n < order; ++n) {
      TRY(dev_alloc(c, (void**)&c->vA[n], (size_t)g.I[n] * g.Jp[n] * 4, "factor velocities"));
      TRY(cudaMemsetAsync(c->vA[n], 0, (size_t)g.I[n] * g.Jp[n] * 4, c->stream) == cudaSuccess
              ? STD_OK : cuda_error(cudaGetLastError(), "memset"));
    }
    TRY(dev_alloc(c, (void**)&c->vB, (size_t)boff * 4, "Kruskal velocities"));
    TRY(cudaMemsetAsync(c->vB, 0, (size_t)boff * 4, c->stream) == cudaSuccess
            ? STD_OK : cuda_error(cudaGetLastError(), "memset"));
  }
  TRY(dev_alloc(c, (void**)&c->core, (size_t)g.prodJ * 4, "core"));
  TRY(cudaMemsetAsync(c->err, 0, 16, c->stream) == cudaSuccess ? STD_OK : cuda_error(cudaGetLastError(), "memset"));
  const int32_t* dcoords = indices;
  const float* dvalues = values;
  if (opt.ptr_kind == 0) {
    TRY(ensure_stage(c, (size_t)nnz * (order + 1) * 4 + 16));
    int32_t* sc = static_cast<int32_t*>(c->stage);
    float* sv = reinterpret_cast<float*>(sc + (size_t)nnz * order);
    e = cudaMemcpyAsync(sc, indices, (size_t)nnz * order * 4, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv, values, (size_t)nnz * 4, cudaMemcpyDefault, c->stream);
    TRY(e == cudaSuccess ? STD_OK : cuda_error(e, "COO upload"));
    dcoords = sc;
    dvalues = sv;
  }
  e = launch_pack_coo(g, dcoords, dvalues, nnz, c->coo, c->cs, c->err, c->stream);
  TRY(e == cudaSuccess ? STD_OK : cuda_error(e, "COO pack"));
  e = launch_init_params(g, c->A, c->B, opt.init_mode, opt.init_mu, opt.init_sigma, opt.seed_init, c->stream);
  TRY(e == cudaSuccess ? STD_OK : cuda_error(e, "parameter init"));
  e = launch_build_core(g, c->B, c->core, c->stream);
  TRY(e == cudaSuccess ? STD_OK : cuda_error(e, "core build"));
  if (opt.precision == 1) {
    e = launch_mirror_bf16(g, c->A, c->Ab, c->stream);
    TRY(e == cudaSuccess ? STD_OK : cuda_error(e, "BF16 mirror"));
  }
  TRY(read_err(c, "std_create"));
  if (opt.ptr_kind == 0) {
    // the staging buffer held the whole COO; give it back
    dev_free(c, c->stage, c->stage_bytes);
    c->stage = nullptr;
    c->stage_bytes = 0;
  }
#undef TRY
  *out = c;
  return STD_OK;
}

int std_sgd_epoch(std_ctx* c, float lr_a, float lr_b, float lambda_a, float lambda_b, int32_t minibatch,
                  std_epoch_stats* out) {
  if (!c) return set_error(STD_EINVAL, "context is NULL");
  int rc = check_hyper(lr_a, lr_b, lambda_a, lambda_b, minibatch);
  if (rc) return rc;
  if (c->cursor != 0)
    return set_error(STD_EINVAL, "an epoch is in progress on this context (batched steps); finish it with std_batch_step");
  const int64_t nb = (c->nnz + minibatch - 1) / minibatch;
  // the epoch time covers the sampler/tiler and the update kernel of every segment
  rc = run_batches(c, lr_a, lr_b, lambda_a, lambda_b, minibatch, 0, nb, false, true);
  if (rc) return rc;
  float ms = 0.f, ms_sched = 0.f, ms_upd = 0.f;
  if (c->seg_count > 0)
    STD_CUDA(cudaEventElapsedTime(&ms, c->seg_ev[0], c->seg_ev[3 * (size_t)c->seg_count - 1]), "event time");
  for (int i = 0; i < c->seg_count; ++i) {
    float a = 0.f, b = 0.f;
    STD_CUDA(cudaEventElapsedTime(&a, c->seg_ev[3 * (size_t)i], c->seg_ev[3 * (size_t)i + 1]), "event time");
    STD_CUDA(cudaEventElapsedTime(&b, c->seg_ev[3 * (size_t)i + 1], c->seg_ev[3 * (size_t)i + 2]), "event time");
    ms_sched += a;
    ms_upd += b;
  }
  if (out) {
    out->seconds = ms * 1e-3;
    out->sched_seconds = ms_sched * 1e-3;
    out->update_seconds = ms_upd * 1e-3;
    out->nnz = c->nnz;
    out->batches = nb;
    out->nnz_per_s = ms > 0.f ? (double)c->nnz / (ms * 1e-3) : 0.0;
    out->epoch = c->epoch;
  }
  c->epoch += 1;
  return STD_OK;
}

int std_sgd_batches(std_ctx* c, float lr_a, float lr_b, float lambda_a, float lambda_b, int32_t minibatch,
                    int64_t batch_begin, int64_t batch_end, std_probe* probe) {
  if (!c) return set_error(STD_EINVAL, "context is NULL");
  int rc = check_hyper(lr_a, lr_b, lambda_a, lambda_b, minibatch);
  if (rc) return rc;
  const int64_t nb = (c->nnz + minibatch - 1) / minibatch;
  if (batch_begin < 0 || batch_end > nb || batch_begin > batch_end)
    return set_error(STD_EINVAL, "batch range outside the epoch");
  const bool want = probe && (probe->core_V || probe->factor_F || probe->nseg) && batch_end > batch_begin;
  rc = run_batches(c, lr_a, lr_b, lambda_a, lambda_b, minibatch, batch_begin, batch_end, want, false);
  if (rc || !want) return rc;
  const int N = c->g.N, R = c->g.R, M = minibatch;
  const int64_t t0 = batch_begin * (int64_t)M;
  const int m = (int)((c->nnz - t0) < M ? (c->nnz - t0) : M);
  // the probed minibatch's run bounds (its segment may have been replaced)
  rc = ensure_schedule_range(c, M, batch_begin, batch_begin + 1);
  if (rc) return rc;
  const int64_t ts = t0 - c->sched.b_first * (int64_t)M;
  std::vector<float> hv((size_t)N * R * kMaxJ), hf((size_t)N * M * kMaxJ);
  std::vector<uint32_t> seg((size_t)m);
  STD_CUDA(cudaMemcpy(hv.data(), c->probe_mem, hv.size() * 4, cudaMemcpyDeviceToHost), "probe copy");
  STD_CUDA(cudaMemcpy(hf.data(), c->probe_mem + hv.size(), hf.size() * 4, cudaMemcpyDeviceToHost), "probe copy");
  if (probe->core_V) std::memcpy(probe->core_V, hv.data(), hv.size() * 4);
  for (int n = 0; n < N; ++n) {
    STD_CUDA(cudaMemcpy(seg.data(), c->sched.seg + (size_t)n * c->sched.npad + ts, (size_t)m * 4,
                        cudaMemcpyDeviceToHost), "segment copy");
    int64_t u = 0;
    for (int q = 0; q < m; ++q) {
      const int st = (int)(seg[q] & 0xffffu);
      if (st != q) continue;
      if (probe->factor_F)
        std::memcpy(probe->factor_F + ((size_t)n * M + u) * kMaxJ, hf.data() + ((size_t)n * M + q) * kMaxJ,
                    kMaxJ * 4);
      ++u;
    }
    if (probe->factor_F)
      for (int64_t v = u; v < M; ++v) std::memset(probe->factor_F + ((size_t)n * M + v) * kMaxJ, 0, kMaxJ * 4);
    if (probe->nseg) probe->nseg[n] = u;
  }
  return STD_OK;
}

int std_schedule(std_ctx* c, int32_t minibatch, int64_t batch_begin, int64_t batch_end, int32_t* sample_ids,
                 int32_t* order, int32_t* seg_start, int32_t* seg_end) {
  if (!c) return set_error(STD_EINVAL, "context is NULL");
  if (minibatch < 1) return set_error(STD_EINVAL, "minibatch must be >= 1");
  if (minibatch > STD_MAX_MINIBATCH) return set_error(STD_EUNSUPPORTED, "minibatch exceeds STD_MAX_MINIBATCH");
  const int64_t nb = (c->nnz + minibatch - 1) / minibatch;
  if (batch_begin < 0 || batch_end > nb || batch_begin > batch_end)
    return set_error(STD_EINVAL, "batch range outside the epoch");
  if (batch_end <= batch_begin) return STD_OK;
  int rc = ensure_schedule_range(c, minibatch, batch_begin, batch_end);
  if (rc) return rc;
  const int64_t t0 = batch_begin * (int64_t)minibatch;
  int64_t t1 = batch_end * (int64_t)minibatch;
  if (t1 > c->nnz) t1 = c->nnz;
  const int64_t cnt = t1 - t0;
  if (cnt <= 0) return STD_OK;
  const int N = c->g.N;
  const int64_t ts = t0 - c->sched.b_first * (int64_t)minibatch;   // storage index of position t0
  if (sample_ids)
    STD_CUDA(cudaMemcpy(sample_ids, c->sched.sid + ts, (size_t)cnt * 4, cudaMemcpyDefault), "schedule copy");
  std::vector<uint32_t> seg;
  for (int n = 0; n < N; ++n) {
    if (order)
      STD_CUDA(cudaMemcpy(order + (size_t)n * cnt, c->sched.pos + (size_t)n * c->sched.npad + ts, (size_t)cnt * 4,
                          cudaMemcpyDefault), "schedule copy");
    if (seg_start || seg_end) {
      seg.resize((size_t)cnt);
      STD_CUDA(cudaMemcpy(seg.data(), c->sched.seg + (size_t)n * c->sched.npad + ts, (size_t)cnt * 4,
                          cudaMemcpyDeviceToHost), "schedule copy");
      for (int64_t q = 0; q < cnt; ++q) {
        if (seg_start) seg_start[(size_t)n * cnt + q] = (int32_t)(seg[q] & 0xffffu);
        if (seg_end) seg_end[(size_t)n * cnt + q] = (int32_t)(seg[q] >> 16);
      }
    }
  }
  return STD_OK;
}

int std_predict(std_ctx* c, int64_t k, const int32_t* coords, float* out) {
  if (!c) return set_error(STD_EINVAL, "context is NULL");
  if (k < 0) return set_error(STD_EINVAL, "k must be >= 0");
  if (k == 0) return STD_OK;
  if (!coords || !out) return set_error(STD_EINVAL, "NULL array argument");
  const int32_t* dc = coords;
  float* dout = out;
  if (c->opt.ptr_kind == 0) {
    const size_t cb = (size_t)k * c->g.N * 4;
    int rc = ensure_stage(c, cb + (size_t)k * 4 + 16);
    if (rc) return rc;
    int32_t* sc = static_cast<int32_t*>(c->stage);
    STD_CUDA(cudaMemcpyAsync(sc, coords, cb, cudaMemcpyDefault, c->stream), "predict staging");
    dc = sc;
    dout = reinterpret_cast<float*>(sc + (size_t)k * c->g.N);
  }
  AParams A{};
  for (int n = 0; n < c->g.N; ++n) A.A[n] = c->A[n];
  STD_CUDA(launch_predict(c->g, A, c->B, dc, nullptr, k, dout, nullptr, predict_blocks(k), c->err, c->stream),
           "predict launch");
  if (c->opt.ptr_kind == 0)
    STD_CUDA(cudaMemcpyAsync(out, dout, (size_t)k * 4, cudaMemcpyDefault, c->stream), "predict copy");
  return read_err(c, "std_predict");
}

int std_predict_many(int32_t count, std_ctx* const* ctxs, const int64_t* k, const int32_t* const* coords,
                     float* const* out) {
  if (count < 1 || !ctxs || !k || !coords || !out) return set_error(STD_EINVAL, "bad arguments");
  const int kind = ctxs[0] ? ctxs[0]->opt.ptr_kind : 0;
  int64_t total = 0;
  size_t cwords = 0;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return set_error(STD_EINVAL, "NULL context");
    if (ctxs[i]->opt.ptr_kind != kind) return set_error(STD_EINVAL, "contexts differ in ptr_kind");
    if (k[i] < 0) return set_error(STD_EINVAL, "k must be >= 0");
    if (k[i] > 0 && (!coords[i] || !out[i])) return set_error(STD_EINVAL, "NULL array argument");
    total += k[i];
    cwords += (size_t)k[i] * ctxs[i]->g.N;
  }
  if (total == 0) return STD_OK;
  cudaStream_t st = ctxs[0]->stream;
  // one stream-ordered allocation: items, error word, (host pointers) staged
  // coordinates and results
  const size_t items_b = (size_t)count * sizeof(PredictItem);
  const size_t err_off = (items_b + 15) & ~(size_t)15;
  const size_t crd_off = err_off + 16;
  const size_t out_off = (crd_off + (kind == 0 ? cwords * 4 : 0) + 15) & ~(size_t)15;
  const size_t bytes = out_off + (kind == 0 ? (size_t)total * 4 : 0);
  char* dev = nullptr;
  STD_CUDA(cudaMallocAsync((void**)&dev, bytes, st), "multi-predict staging");
  std::vector<PredictItem> h(count);
  int64_t off = 0;
  size_t cw = 0;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    std_ctx* c = ctxs[i];
    PredictItem& it = h[i];
    it.g = c->g;
    for (int n = 0; n < c->g.N; ++n) it.A.A[n] = c->A[n];
    it.B = c->B;
    it.k = k[i];
    it.off = off;
    if (kind == 0) {
      int32_t* dc = reinterpret_cast<int32_t*>(dev + crd_off) + cw;
      it.coords = dc;
      it.out = reinterpret_cast<float*>(dev + out_off) + off;
      if (k[i] > 0)
        e = cudaMemcpyAsync(dc, coords[i], (size_t)k[i] * c->g.N * 4, cudaMemcpyHostToDevice, st);
    } else {
      it.coords = coords[i];
      it.out = out[i];
    }
    off += k[i];
    cw += (size_t)k[i] * c->g.N;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(dev, h.data(), items_b, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev + err_off, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = launch_predict_multi(reinterpret_cast<const PredictItem*>(dev), count, total,
                             reinterpret_cast<int*>(dev + err_off), st);
  if (e == cudaSuccess && kind == 0)
    for (int i = 0; i < count && e == cudaSuccess; ++i)
      if (k[i] > 0)
        e = cudaMemcpyAsync(out[i], reinterpret_cast<float*>(dev + out_off) + h[i].off, (size_t)k[i] * 4,
                            cudaMemcpyDeviceToHost, st);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, dev + err_off, sizeof(int), cudaMemcpyDeviceToHost, st);
  const cudaError_t ef = cudaFreeAsync(dev, st);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "multi-predict");
  if (herr != 0) return set_error(STD_EINVAL, "std_predict_many: coordinate outside [0, I_n)");
  return STD_OK;
}

int std_rmse(std_ctx* c, int64_t k, const int32_t* coords, const float* values, double* rmse, double* mae) {
  if (!c) return set_error(STD_EINVAL, "context is NULL");
  if (k < 0 || !rmse) return set_error(STD_EINVAL, "bad arguments");
  if (k == 0) {
    *rmse = 0.0;
    if (mae) *mae = 0.0;
    return STD_OK;
  }
  if (!coords || !values) return set_error(STD_EINVAL, "NULL array argument");
  int rc = STD_OK;
  const float* dv = nullptr;
  const int32_t* dc = stage_coords(c, coords, values, k, &dv, &rc);
  if (rc) return rc;
  const int blocks = predict_blocks(k);
  if (blocks > c->rpart_blocks) {
    dev_free(c, c->rpart, (size_t)c->rpart_blocks * 16);
    c->rpart = nullptr;
    c->rpart_blocks = 0;
    rc = dev_alloc(c, (void**)&c->rpart, (size_t)blocks * 16, "rmse partials");
    if (rc) return rc;
    c->rpart_blocks = blocks;
  }
  AParams A{};
  for (int n = 0; n < c->g.N; ++n) A.A[n] = c->A[n];
  STD_CUDA(launch_predict(c->g, A, c->B, dc, dv, k, nullptr, c->rpart, blocks, c->err, c->stream), "rmse launch");
  STD_CUDA(launch_rmse_finish(c->rpart, blocks, c->result, c->stream), "rmse finish");
  double h[2] = {0.0, 0.0};
  STD_CUDA(cudaMemcpyAsync(h, c->result, 16, cudaMemcpyDeviceToHost, c->stream), "rmse copy");
  rc = read_err(c, "std_rmse");
  if (rc) return rc;
  if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return set_error(STD_ENUMERIC, "std_rmse: NaN or Inf in the sums");
  *rmse = std::sqrt(h[0] / (double)k);
  if (mae) *mae = h[1] / (double)k;
  return STD_OK;
}

int std_get_params(std_ctx* c, float* const* A, float* const* B, float* core, int64_t* epoch) {
  if (!c) return set_error(STD_EINVAL, "context is NULL");
  const Geometry& g = c->g;
  for (int n = 0; n < g.N; ++n) {
    if (A && A[n])
      STD_CUDA(cudaMemcpy2DAsync(A[n], (size_t)g.J[n] * 4, c->A[n], (size_t)g.Jp[n] * 4, (size_t)g.J[n] * 4,
                                 (size_t)g.I[n], cudaMemcpyDefault, c->stream), "get A");
    if (B && B[n])
      STD_CUDA(cudaMemcpyAsync(B[n], c->B + g.boff[n], (size_t)g.J[n] * g.R * 4, cudaMemcpyDefault, c->stream),
               "get B");
  }
  if (core) {
    STD_CUDA(launch_build_core(g, c->B, c->core, c->stream), "core build");
    STD_CUDA(cudaMemcpyAsync(core, c->core, (size_t)g.prodJ * 4, cudaMemcpyDefault, c->stream), "get core");
  }
  STD_CUDA(cudaStreamSynchronize(c->stream), "get params sync");
  if (epoch) *epoch = c->epoch;
  return STD_OK;
}

int std_set_params(std_ctx* c, const float* const* A, const float* const* B, int64_t epoch) {
  if (!c) return set_error(STD_EINVAL, "context is NULL");
  const Geometry& g = c->g;
  for (int n = 0; n < g.N; ++n) {
    if (A && A[n])
      STD_CUDA(cudaMemcpy2DAsync(c->A[n], (size_t)g.Jp[n] * 4, A[n], (size_t)g.J[n] * 4, (size_t)g.J[n] * 4,
                                 (size_t)g.I[n], cudaMemcpyDefault, c->stream), "set A");
    if (B && B[n])
      STD_CUDA(cudaMemcpyAsync(c->B + g.boff[n], B[n], (size_t)g.J[n] * g.R * 4, cudaMemcpyDefault, c->stream),
               "set B");
  }
  STD_CUDA(launch_build_core(g, c->B, c->core, c->stream), "core build");
  if (c->opt.precision == 1) STD_CUDA(launch_mirror_bf16(g, c->A, c->Ab, c->stream), "BF16 mirror");
  if (c->vB) {
    for (int n = 0; n < g.N; ++n)
      STD_CUDA(cudaMemsetAsync(c->vA[n], 0, (size_t)g.I[n] * g.Jp[n] * 4, c->stream), "velocity reset");
    STD_CUDA(cudaMemsetAsync(c->vB, 0, (size_t)g.boff[g.N - 1] * 4 + (size_t)g.J[g.N - 1] * g.R * 4, c->stream),
             "velocity reset");
  }
  STD_CUDA(cudaStreamSynchronize(c->stream), "set params sync");
  if (epoch >= 0) {
    c->epoch = epoch;
    c->cursor = 0;
  }
  return STD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched epochs: many independent tensors in one persistent launch.
// ---------------------------------------------------------------------------

struct std_batch {
  std::vector<std_ctx*> ctxs;
  cudaStream_t stream = nullptr;
  int precision = 0;
  int group = 0;          // CTAs per tensor (the base size); 0 until tuned
  int tile = 0;           // FP32 contraction tile of every tensor (0 = from its chunk size)
  bool tuned = false;
  bool promote = false;   // long tensors may get groups of 2^k x group CTAs
  std::vector<int> fixed_g; // per-tensor group sizes set by the caller (empty: none)
  std::vector<int> last_g; // CTAs each tensor had in the last launch
  int* err = nullptr;     // one error word shared by every tensor of a launch
  EpochArgs* d_items = nullptr;
  int* d_order = nullptr;
  int* d_first = nullptr;
  int* d_gstart = nullptr;
  int* d_gstart_cl = nullptr;   // cluster form: each size class's group starts, from 0
  size_t cap_items = 0, cap_groups = 0;
  // pinned host staging of the launch arguments (fixed addresses, so that a
  // captured graph copies their current contents at every replay)
  EpochArgs* h_items = nullptr;
  int* h_order = nullptr;
  int* h_first = nullptr;
  int* h_gstart = nullptr;
  int* h_gstart_cl = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evm = nullptr;
  // cluster form: one launch per group size, on forked streams of the capture
  cudaStream_t fork[8] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[8] = {};
  // the launch sequence (barrier resets, argument uploads, the cooperative
  // kernel) captured as a CUDA graph and replayed while its shape holds
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<std_ctx*> gkey_ctxs;
  int gkey_ctas = 0, gkey_groups = 0;
  size_t gkey_smem = 0;
  std::vector<std::pair<int, int>> gkey_classes;   // cluster form: (size, groups) per launch; empty = cooperative
  bool gkey_plain = false;                         // the captured launches use the specialised kernels
  const void* gkey_items = nullptr;
  bool replayed = false;   // the last launch replayed the graph
};

namespace {

// Smallest chunk a CTA of the batched kernel handles for tensor c at group
// size G, or 0 when the shape does not fit a CTA.
size_t batch_smem(std_ctx* c, int M, int G, bool cl = false) {
  const int chunk = (M + G - 1) / G;
  if (chunk > epoch_chunk_cap(c->g)) return 0;
  const size_t sm = cl ? epoch_smem_bytes_cl(c->g, chunk, G, c->opt.precision)
                       : epoch_smem_bytes(c->g, chunk, G, c->opt.precision);
  return sm > 227 * 1024 ? 0 : sm;
}

// One launch of minibatches range[t] = [b0, b1) of every tensor t; dry = no
// parameter writes (timing runs of the tuner).  Every tensor runs on a group
// of G CTAs, except, when promote is set, the tensors that would set the
// makespan: those get a group of their own of G * 2^k CTAs (up to 32 CTAs
// and chunks of at least 8 samples), doubled one at a time while the
// estimated makespan falls.  The other tensors go longest-first to the
// least-loaded base group.
int batch_launch(std_batch* bt, float lr_a, float lr_b, float lam_a, float lam_b, int32_t M,
                 const std::vector<std::pair<int64_t, int64_t>>& range, int G, bool dry, bool promote) {
  const int T = (int)bt->ctxs.size();
  size_t smem = 0;
  if ((size_t)T > bt->cap_items) {
    // grow every argument buffer (device and pinned host) to T tensors
    if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
    bt->gexec = nullptr;
    cudaFree(bt->d_items);
    cudaFree(bt->d_order);
    cudaFree(bt->d_first);
    cudaFree(bt->d_gstart);
    cudaFree(bt->d_gstart_cl);
    cudaFreeHost(bt->h_items);
    cudaFreeHost(bt->h_order);
    cudaFreeHost(bt->h_first);
    cudaFreeHost(bt->h_gstart);
    cudaFreeHost(bt->h_gstart_cl);
    bt->d_gstart_cl = nullptr;
    bt->h_gstart_cl = nullptr;
    bt->d_items = nullptr;
    bt->d_order = nullptr;
    bt->d_first = nullptr;
    bt->d_gstart = nullptr;
    bt->h_items = nullptr;
    bt->h_order = nullptr;
    bt->h_first = nullptr;
    bt->h_gstart = nullptr;
    bt->cap_items = 0;
    const size_t ci = (size_t)T, cg = (size_t)(T + 1);
    STD_CUDA(cudaMalloc((void**)&bt->d_items, ci * sizeof(EpochArgs)), "batch arguments");
    STD_CUDA(cudaMalloc((void**)&bt->d_order, ci * sizeof(int)), "batch order");
    STD_CUDA(cudaMalloc((void**)&bt->d_first, cg * sizeof(int)), "batch groups");
    STD_CUDA(cudaMalloc((void**)&bt->d_gstart, cg * sizeof(int)), "batch group starts");
    STD_CUDA(cudaMallocHost((void**)&bt->h_items, ci * sizeof(EpochArgs)), "batch arguments (host)");
    STD_CUDA(cudaMallocHost((void**)&bt->h_order, ci * sizeof(int)), "batch order (host)");
    STD_CUDA(cudaMallocHost((void**)&bt->h_first, cg * sizeof(int)), "batch groups (host)");
    STD_CUDA(cudaMallocHost((void**)&bt->h_gstart, cg * sizeof(int)), "batch group starts (host)");
    STD_CUDA(cudaMalloc((void**)&bt->d_gstart_cl, (cg + 8) * sizeof(int)), "batch cluster group starts");
    STD_CUDA(cudaMallocHost((void**)&bt->h_gstart_cl, (cg + 8) * sizeof(int)), "batch cluster group starts (host)");
    bt->cap_items = ci;
    bt->cap_groups = cg;
  }
  // work estimates and the base-size shared memory (a larger group has
  // smaller chunks, so the base size bounds every tensor's need)
  std::vector<int64_t> w(T), e0v(T), e1v(T);
  size_t smem_cl = 0;
  for (int t = 0; t < T; ++t) {
    std_ctx* c = bt->ctxs[t];
    int rc = ensure_schedule(c, M);
    if (rc) return rc;
    const int gown = bt->fixed_g.empty() ? G : bt->fixed_g[t];
    const size_t sm = batch_smem(c, M, gown);
    if (sm == 0) return set_error(STD_EUNSUPPORTED, "a tensor of the batch does not fit a CTA at this group size");
    smem = sm > smem ? sm : smem;
    const size_t smc = batch_smem(c, M, gown, true);
    smem_cl = smc == 0 ? (size_t)-1 : (smc > smem_cl ? smc : smem_cl);
    const int64_t nb = (c->nnz + M - 1) / M;
    e0v[t] = range[t].first < nb ? range[t].first : nb;
    e1v[t] = range[t].second < nb ? range[t].second : nb;
    // time per minibatch ~ a fixed chain of dependent steps plus a part that
    // grows with the per-sample work (fit of measured times at M = 256:
    // 34 us + 0.17 us x (sum J + prod J / max J))
    w[t] = (e1v[t] - e0v[t]) * (int64_t)(192 + c->g.sumJ + c->g.prodJ / c->g.Jmax);
  }
  STD_CUDA(epoch_multi_setup(bt->precision, smem), "batched kernel attributes");
  const int maxc = epoch_multi_max_ctas(bt->precision, smem);
  if (maxc / G < 1) return set_error(STD_EUNSUPPORTED, "batched kernel cannot be resident at this group size");
  // longest processing time first
  std::vector<int> byw(T);
  for (int t = 0; t < T; ++t) byw[t] = t;
  std::sort(byw.begin(), byw.end(), [&](int x, int y) { return w[x] != w[y] ? w[x] > w[y] : x < y; });
  std::vector<int> gt(T, G);
  int promoted_ctas = 0, promoted = 0;
  if (promote) {
    // greedy on the estimated makespan: a tensor's time at 2^k x G CTAs is
    // its work times kSpeed[k] (measured per-minibatch times at M = 256,
    // J in {4, 8, 16}: about 0.77 for the first doubling, 0.86 for the next);
    // the base groups finish after max(their mean load, their longest tensor)
    static const double kSpeed[6] = {1.0, 0.77, 0.66, 0.63, 0.62, 0.62};
    std::vector<int> lv(T, 0);
    auto makespan = [&](const std::vector<int>& lvl, int pctas) {
      const int nb0 = (maxc - pctas) / G;
      if (nb0 < 1) return 1e300;
      double base_sum = 0.0, base_max = 0.0, prom_max = 0.0;
      int nbase_t = 0;
      for (int t = 0; t < T; ++t) {
        if (lvl[t] == 0) {
          base_sum += (double)w[t];
          base_max = (double)w[t] > base_max ? (double)w[t] : base_max;
          ++nbase_t;
        } else {
          const double e = (double)w[t] * kSpeed[lvl[t]];
          prom_max = e > prom_max ? e : prom_max;
        }
      }
      const int ng = nb0 < nbase_t ? nb0 : nbase_t;
      const double base_span = nbase_t == 0 ? 0.0 : (base_sum / (ng > 0 ? ng : 1) > base_max ? base_sum / ng : base_max);
      return base_span > prom_max ? base_span : prom_max;
    };
    double cur = makespan(lv, 0);
    int pctas = 0;
#pragma unroll 1
    for (int it = 0; it < 4 * T; ++it) {
      // the tensor that sets the makespan: the longest at its current size
      int bt_t = -1;
      double bt_e = -1.0;
      for (int t = 0; t < T; ++t) {
        const double e = (double)w[t] * kSpeed[lv[t]];
        if (e > bt_e) {
          bt_e = e;
          bt_t = t;
        }
      }
      const int g_now = G << lv[bt_t], g_new = g_now * 2;
      if (g_new > 32 || M / g_new < 8 || lv[bt_t] >= 5) break;
      const int extra = lv[bt_t] == 0 ? g_new : g_now;
      if (pctas + extra > maxc - G) break;
      std::vector<int> nx = lv;
      nx[bt_t] += 1;
      const double e = makespan(nx, pctas + extra);
      if (!(e < cur)) break;
      lv = nx;
      pctas += extra;
      cur = e;
    }
    for (int t = 0; t < T; ++t)
      if (lv[t] > 0) {
        gt[t] = G << lv[t];
        promoted_ctas += gt[t];
        ++promoted;
      }
  }
  std::vector<std::vector<int>> lists;
  std::vector<int> gsize;
  if (!bt->fixed_g.empty()) {
    // caller-fixed sizes: one class of groups per distinct size; every class
    // starts with one group, then the class with the highest mean load per
    // group (time per size from the same speed model) gains a group while
    // CTAs remain, up to one group per tensor
    gt = bt->fixed_g;
    std::vector<int> sizes(gt.begin(), gt.end());
    std::sort(sizes.begin(), sizes.end());
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    const int S = (int)sizes.size();
    auto speed = [](int g) {
      // relative to 4 CTAs: doubling 0.77, 0.86, 0.95; halving 1.5 per step
      double f = 1.0;
      for (int x = 4; x < g; x *= 2) f *= x == 4 ? 0.77 : (x == 8 ? 0.86 : 0.95);
      for (int x = 4; x > g; x /= 2) f *= 1.5;
      return f;
    };
    std::vector<int> ng(S, 1), cnt(S, 0);
    std::vector<double> sum(S, 0.0), mx(S, 0.0);
    int used = 0;
    for (int k = 0; k < S; ++k) used += sizes[k];
    if (used > maxc) return set_error(STD_EUNSUPPORTED, "the fixed group sizes do not fit the co-resident CTAs");
    for (int t = 0; t < T; ++t) {
      const int k = (int)(std::lower_bound(sizes.begin(), sizes.end(), gt[t]) - sizes.begin());
      const double e = (double)w[t] * speed(gt[t]);
      sum[k] += e;
      mx[k] = e > mx[k] ? e : mx[k];
      ++cnt[k];
    }
#pragma unroll 1
    while (true) {
      int best = -1;
      double best_f = -1.0;
      for (int k = 0; k < S; ++k) {
        if (ng[k] >= cnt[k] || used + sizes[k] > maxc) continue;
        const double f = sum[k] / ng[k];
        if (f > best_f) {
          best_f = f;
          best = k;
        }
      }
      if (best < 0) break;
      ++ng[best];
      used += sizes[best];
    }
    std::vector<int> first_group(S, 0);
    int q0 = 0;
    for (int k = 0; k < S; ++k) {
      first_group[k] = q0;
      for (int i = 0; i < ng[k]; ++i) gsize.push_back(sizes[k]);
      q0 += ng[k];
    }
    lists.assign(q0, {});
    std::vector<double> load(q0, 0.0);
    for (int t : byw) {
      const int k = (int)(std::lower_bound(sizes.begin(), sizes.end(), gt[t]) - sizes.begin());
      int b = first_group[k];
      for (int q = first_group[k] + 1; q < first_group[k] + ng[k]; ++q)
        if (load[q] < load[b]) b = q;
      load[b] += (double)w[t];
      lists[b].push_back(t);
    }
  }
  int nbase = (maxc - promoted_ctas) / G;
  if (nbase > T - promoted) nbase = T - promoted;
  const int groups = bt->fixed_g.empty() ? promoted + nbase : (int)gsize.size();
  if (groups < 1) return set_error(STD_EUNSUPPORTED, "batched kernel cannot be resident at this group size");
  if (bt->fixed_g.empty()) {
    lists.assign(groups, {});
    gsize.assign(groups, G);
    int q = 0;
    for (int t : byw)
      if (gt[t] > G) {
        lists[q].push_back(t);
        gsize[q] = gt[t];
        ++q;
      }
    std::vector<int64_t> load(nbase, 0);
    for (int t : byw) {
      if (gt[t] > G) continue;
      int b = 0;
      for (int k = 1; k < nbase; ++k)
        if (load[k] < load[b]) b = k;
      load[b] += w[t];
      lists[promoted + b].push_back(t);
    }
  }
  bt->last_g = gt;
  bool plain = true;   // every tensor with the default options: the specialised kernels
  for (int t = 0; t < T; ++t) {
    std_ctx* c = bt->ctxs[t];
    int rc = ensure_scratch(c, gt[t], payload_floats(c->g), M);
    if (rc) return rc;
    uint32_t tag_base = 0;
    rc = reserve_tags(c, e1v[t] - e0v[t], &tag_base);
    if (rc) return rc;
    EpochArgs a = epoch_args(c, lr_a, lr_b, lam_a, lam_b, e0v[t], e1v[t], (M + gt[t] - 1) / gt[t], tag_base);
    a.err = bt->err;
    a.tile_sg = bt->tile;
    a.dry = dry ? 1 : 0;
    if (dry) a.momentum = 0.f;
    bt->h_items[t] = a;
    plain = plain && epoch_args_plain(a);
  }
  // cluster form: every group one thread block cluster (2..16 CTAs, or a
  // single CTA), one launch per group size; the groups are ordered by size so
  // that each size's groups are consecutive.  Same results as the cooperative
  // form, which takes over when a size is not a cluster size or clusters of
  // it cannot be resident.
  std::vector<std::pair<int, int>> classes;
  {
    bool ok = smem_cl <= (size_t)227 * 1024;
    for (int q = 0; q < groups && ok; ++q) ok = gsize[q] == 1 || epoch_cluster_size_ok(gsize[q]);
    if (ok) {
      std::vector<int> idx(groups);
      for (int q = 0; q < groups; ++q) idx[q] = q;
      std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return gsize[x] < gsize[y]; });
      std::vector<std::vector<int>> l2(groups);
      std::vector<int> g2(groups);
      for (int q = 0; q < groups; ++q) {
        l2[q] = lists[idx[q]];
        g2[q] = gsize[idx[q]];
      }
      for (int q = 0; q < groups; ++q)
        if (classes.empty() || classes.back().first != g2[q]) classes.push_back({g2[q], 1});
        else classes.back().second += 1;
      // only one size, and no more groups than clusters of it can be resident
      // at once: a cluster must fit inside one GPC, so fewer groups of a size
      // run side by side than CTAs would allow, and groups that wait for a
      // free slot would stretch the launch (measured on the batched workload:
      // 692 ms in the cluster form against 421 ms cooperative with groups of
      // 4 and 8)
      if (classes.size() != 1 || epoch_cl_max_clusters(bt->precision, true, smem_cl, classes[0].first) <
                                     classes[0].second)
        ok = false;
      if (ok) {
        lists.swap(l2);
        gsize.swap(g2);
      } else {
        classes.clear();
      }
    }
  }
  if (!classes.empty()) smem = smem_cl;
  int no = 0;
  bt->h_first[0] = 0;
  bt->h_gstart[0] = 0;
  for (int q = 0; q < groups; ++q) {
    for (int t : lists[q]) bt->h_order[no++] = t;
    bt->h_first[q + 1] = no;
    bt->h_gstart[q + 1] = bt->h_gstart[q] + gsize[q];
  }
  {
    int at = 0, q0 = 0;
    for (const auto& k : classes) {
      for (int j = 0; j <= k.second; ++j) bt->h_gstart_cl[at + j] = j * k.first;
      at += k.second + 1;
      q0 += k.second;
    }
  }
  const int ctas = bt->h_gstart[groups];
  // (re)capture the launch sequence when its shape changed: the tensors (their
  // barrier words), the group size, the group count, the shared memory and
  // the argument buffers; otherwise replay it (the copies read the pinned
  // staging, so the new ranges, order and flags reach the device)
  const bool same = bt->gexec && bt->gkey_ctxs == bt->ctxs && bt->gkey_ctas == ctas && bt->gkey_groups == groups &&
                    bt->gkey_smem == smem && bt->gkey_items == (const void*)bt->d_items &&
                    bt->gkey_classes == classes && bt->gkey_plain == plain;
  bt->replayed = same;
  if (!same) {
    if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
    bt->gexec = nullptr;
    if (!bt->cap_stream) STD_CUDA(cudaStreamCreateWithFlags(&bt->cap_stream, cudaStreamNonBlocking), "capture stream");
    cudaStream_t cs = bt->cap_stream;
    STD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "graph capture");
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < T && e == cudaSuccess; ++t)
      e = cudaMemsetAsync(bt->ctxs[t]->bar, 0, sizeof(unsigned long long), cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bt->d_items, bt->h_items, (size_t)T * sizeof(EpochArgs), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bt->d_order, bt->h_order, (size_t)T * sizeof(int), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bt->d_first, bt->h_first, (size_t)(groups + 1) * sizeof(int), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bt->d_gstart, bt->h_gstart, (size_t)(groups + 1) * sizeof(int), cudaMemcpyHostToDevice,
                          cs);
    if (e == cudaSuccess && !classes.empty())
      e = cudaMemcpyAsync(bt->d_gstart_cl, bt->h_gstart_cl, (size_t)(groups + classes.size()) * sizeof(int),
                          cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && classes.empty()) {
      MultiArgs m{};
      m.items = bt->d_items;
      m.order = bt->d_order;
      m.first = bt->d_first;
      m.gstart = bt->d_gstart;
      m.groups = groups;
      m.plain = plain ? 1 : 0;
      e = launch_epoch_multi(m, bt->precision, ctas, smem, cs);
    } else if (e == cudaSuccess) {
      // one cluster launch per group size, the sizes in parallel branches
      if (!bt->ev_fork) e = cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming);
      for (size_t k = 1; k < classes.size() && e == cudaSuccess; ++k) {
        if (!bt->fork[k]) e = cudaStreamCreateWithFlags(&bt->fork[k], cudaStreamNonBlocking);
        if (e == cudaSuccess && !bt->ev_join[k]) e = cudaEventCreateWithFlags(&bt->ev_join[k], cudaEventDisableTiming);
      }
      if (e == cudaSuccess) e = cudaEventRecord(bt->ev_fork, cs);
      int q0 = 0, at = 0;
      for (size_t k = 0; k < classes.size() && e == cudaSuccess; ++k) {
        cudaStream_t sk = k == 0 ? cs : bt->fork[k];
        if (k > 0) e = cudaStreamWaitEvent(sk, bt->ev_fork, 0);
        MultiArgs m{};
        m.items = bt->d_items;
        m.order = bt->d_order;
        m.first = bt->d_first + q0;
        m.gstart = bt->d_gstart_cl + at;
        m.groups = classes[k].second;
        m.plain = plain ? 1 : 0;
        if (e == cudaSuccess) e = launch_epoch_multi_cl(m, bt->precision, classes[k].first, smem, sk);
        if (e == cudaSuccess && k > 0) e = cudaEventRecord(bt->ev_join[k], sk);
        q0 += classes[k].second;
        at += classes[k].second + 1;
      }
      for (size_t k = 1; k < classes.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(cs, bt->ev_join[k], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bt->gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      bt->gexec = nullptr;
      return cuda_error(e, "batched launch graph");
    }
    bt->gkey_ctxs = bt->ctxs;
    bt->gkey_ctas = ctas;
    bt->gkey_groups = groups;
    bt->gkey_smem = smem;
    bt->gkey_items = bt->d_items;
    bt->gkey_classes = classes;
    bt->gkey_plain = plain;
  }
  STD_CUDA(cudaEventRecord(bt->evm, bt->stream), "event");
  STD_CUDA(cudaGraphLaunch(bt->gexec, bt->stream), "batched graph launch");
  STD_CUDA(cudaEventRecord(bt->ev1, bt->stream), "event");
  int h = 0;
  STD_CUDA(cudaMemcpyAsync(&h, bt->err, sizeof(int), cudaMemcpyDeviceToHost, bt->stream), "batch error read");
  STD_CUDA(cudaStreamSynchronize(bt->stream), "batch sync");
  if (h != 0) {
    STD_CUDA(cudaMemset(bt->err, 0, sizeof(int)), "batch error reset");
    if (h == STD_ETIMEOUT) return set_error(STD_ETIMEOUT, "batched epoch kernel: barrier watchdog expired");
    return set_error(h, "batched epoch kernel: device error");
  }
  return STD_OK;
}

}  // namespace

extern "C" {

int std_batch_create(std_batch** out, int32_t count, std_ctx* const* ctxs, int32_t ctas_per_tensor) {
  if (!out) return set_error(STD_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !ctxs) return set_error(STD_EINVAL, "a batch needs at least one context");
  if (ctas_per_tensor < -1) return set_error(STD_EINVAL, "ctas_per_tensor must be >= -1");
  for (int t = 0; t < count; ++t) {
    if (!ctxs[t]) return set_error(STD_EINVAL, "NULL context in the batch");
    if (ctxs[t]->opt.precision != ctxs[0]->opt.precision)
      return set_error(STD_EINVAL, "every context of a batch must use the same precision");
    if (ctxs[t]->stream != ctxs[0]->stream)
      return set_error(STD_EINVAL, "every context of a batch must use the same stream");
    if (ctxs[t]->opt.snapshot >= 2)
      return set_error(STD_EINVAL, "batched launches run Algorithm 1's order (snapshot 0 or 1)");
    for (int u = 0; u < t; ++u)
      if (ctxs[u] == ctxs[t]) return set_error(STD_EINVAL, "a context appears twice in the batch");
  }
  std_batch* bt = new std_batch();
  bt->ctxs.assign(ctxs, ctxs + count);
  bt->stream = ctxs[0]->stream;
  bt->precision = ctxs[0]->opt.precision;
  bt->group = ctas_per_tensor > 0 ? ctas_per_tensor : 0;
  bt->tuned = ctas_per_tensor > 0;
  bt->promote = ctas_per_tensor == 0;
  cudaError_t e = cudaMalloc((void**)&bt->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(bt->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&bt->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&bt->ev1);
  if (e == cudaSuccess) e = cudaEventCreate(&bt->evm);
  if (e != cudaSuccess) {
    std_batch_destroy(bt);
    return cuda_error(e, "batch setup");
  }
  *out = bt;
  return STD_OK;
}

int std_batch_destroy(std_batch* bt) {
  if (!bt) return STD_OK;
  cudaStreamSynchronize(bt->stream);
  if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
  if (bt->cap_stream) cudaStreamDestroy(bt->cap_stream);
  cudaFree(bt->err);
  cudaFree(bt->d_items);
  cudaFree(bt->d_order);
  cudaFree(bt->d_first);
  cudaFree(bt->d_gstart);
  cudaFree(bt->d_gstart_cl);
  cudaFreeHost(bt->h_items);
  cudaFreeHost(bt->h_order);
  cudaFreeHost(bt->h_first);
  cudaFreeHost(bt->h_gstart);
  cudaFreeHost(bt->h_gstart_cl);
  for (int k = 0; k < 8; ++k) {
    if (bt->fork[k]) cudaStreamDestroy(bt->fork[k]);
    if (bt->ev_join[k]) cudaEventDestroy(bt->ev_join[k]);
  }
  if (bt->ev_fork) cudaEventDestroy(bt->ev_fork);
  if (bt->ev0) cudaEventDestroy(bt->ev0);
  if (bt->ev1) cudaEventDestroy(bt->ev1);
  if (bt->evm) cudaEventDestroy(bt->evm);
  delete bt;
  return STD_OK;
}

int std_batch_step(std_batch* bt, float lr_a, float lr_b, float lambda_a, float lambda_b, int32_t minibatch,
                   int64_t max_batches, std_batch_stats* out) {
  if (!bt) return set_error(STD_EINVAL, "batch is NULL");
  int rc = check_hyper(lr_a, lr_b, lambda_a, lambda_b, minibatch);
  if (rc) return rc;
  if (max_batches < 1) return set_error(STD_EINVAL, "max_batches must be >= 1");
  for (std_ctx* c : bt->ctxs)
    if (c->cursor > 0 && c->cursor_M != minibatch)
      return set_error(STD_EINVAL, "a context has an epoch in progress with another minibatch size");
  if (!bt->tuned) {
    // autotuner: each group size that fits times a dry run (no parameter
    // writes) of 3% of every tensor's minibatches from its position, so that
    // the trial has the epoch's mix of long and short tensors; the fastest wins
    float best = -1.f;
    int best_g = 0;
    std::vector<std::pair<int64_t, int64_t>> trial;
    for (std_ctx* c : bt->ctxs) {
      const int64_t nb = (c->nnz + minibatch - 1) / minibatch;
      const int64_t k = (int64_t)std::ceil(0.03 * (double)nb);
      trial.push_back({c->cursor, c->cursor + (k < 1 ? 1 : k)});
    }
    for (int G = 1; G <= 32; G *= 2) {
      bool fits = true;
      for (std_ctx* c : bt->ctxs)
        if (batch_smem(c, minibatch, G) == 0) fits = false;
      if (!fits) continue;
      rc = batch_launch(bt, lr_a, lr_b, lambda_a, lambda_b, minibatch, trial, G, true, bt->promote);
      if (rc == STD_EUNSUPPORTED) continue;
      if (rc) return rc;
      float ms = 0.f;
      STD_CUDA(cudaEventElapsedTime(&ms, bt->evm, bt->ev1), "event time");
      if (best < 0.f || ms < best) {
        best = ms;
        best_g = G;
      }
    }
    if (best_g == 0) return set_error(STD_EUNSUPPORTED, "no group size fits every tensor of the batch");
    bt->group = best_g;
    // then the FP32 contraction tile on the same trial (same bits whatever
    // the tile; the per-chunk choice, 0, stays unless a fixed tile is faster)
    if (bt->precision == 0) {
      float best_t = -1.f;
      int best_tile = 0;
      for (int tile : {0, 1, 2, 4}) {
        bt->tile = tile;
        rc = batch_launch(bt, lr_a, lr_b, lambda_a, lambda_b, minibatch, trial, best_g, true, bt->promote);
        if (rc) return rc;
        float ms = 0.f;
        STD_CUDA(cudaEventElapsedTime(&ms, bt->evm, bt->ev1), "event time");
        if (best_t < 0.f || ms < best_t * 0.99f) {
          best_t = ms;
          best_tile = tile;
        }
      }
      bt->tile = best_tile;
    }
    bt->tuned = true;
  }
  STD_CUDA(cudaEventRecord(bt->ev0, bt->stream), "event");
  std::vector<std::pair<int64_t, int64_t>> range;
  int64_t nnz = 0;
  for (std_ctx* c : bt->ctxs) {
    const int64_t nb = (c->nnz + minibatch - 1) / minibatch;
    const int64_t e1 = (max_batches >= nb - c->cursor) ? nb : c->cursor + max_batches;
    range.push_back({c->cursor, e1});
    const int64_t t1 = e1 * (int64_t)minibatch < c->nnz ? e1 * (int64_t)minibatch : c->nnz;
    nnz += t1 - c->cursor * (int64_t)minibatch;
  }
  rc = batch_launch(bt, lr_a, lr_b, lambda_a, lambda_b, minibatch, range, bt->group, false, bt->promote);
  if (rc) return rc;
  for (size_t t = 0; t < bt->ctxs.size(); ++t) {
    std_ctx* c = bt->ctxs[t];
    const int64_t nb = (c->nnz + minibatch - 1) / minibatch;
    c->cursor = range[t].second;
    c->cursor_M = minibatch;
    if (c->cursor >= nb) {
      c->cursor = 0;
      c->epoch += 1;
    }
  }
  float ms = 0.f, ms_upd = 0.f;
  STD_CUDA(cudaEventElapsedTime(&ms, bt->ev0, bt->ev1), "event time");
  STD_CUDA(cudaEventElapsedTime(&ms_upd, bt->evm, bt->ev1), "event time");
  if (out) {
    out->seconds = ms * 1e-3;
    out->update_seconds = ms_upd * 1e-3;
    out->nnz = nnz;
    out->nnz_per_s = ms > 0.f ? (double)nnz / (ms * 1e-3) : 0.0;
    out->tensors = (int32_t)bt->ctxs.size();
    out->ctas_per_tensor = bt->group;
    out->graph_replayed = bt->replayed ? 1 : 0;
    out->reserved = 0;
  }
  return STD_OK;
}

int std_batch_reset(std_batch* bt, int32_t count, std_ctx* const* ctxs) {
  if (!bt) return set_error(STD_EINVAL, "batch is NULL");
  if (count < 1 || !ctxs) return set_error(STD_EINVAL, "a batch needs at least one context");
  for (int t = 0; t < count; ++t) {
    if (!ctxs[t]) return set_error(STD_EINVAL, "NULL context in the batch");
    if (ctxs[t]->opt.precision != bt->precision)
      return set_error(STD_EINVAL, "every context of a batch must use the batch's precision");
    if (ctxs[t]->stream != bt->stream) return set_error(STD_EINVAL, "every context of a batch must use its stream");
    if (ctxs[t]->opt.snapshot >= 2)
      return set_error(STD_EINVAL, "batched launches run Algorithm 1's order (snapshot 0 or 1)");
    for (int u = 0; u < t; ++u)
      if (ctxs[u] == ctxs[t]) return set_error(STD_EINVAL, "a context appears twice in the batch");
  }
  bt->ctxs.assign(ctxs, ctxs + count);
  if (!bt->fixed_g.empty()) {
    // per-tensor sizes belonged to the old members: back to the uniform base size
    bt->fixed_g.clear();
  }
  bt->last_g.clear();
  return STD_OK;
}

int std_batch_set_groups(std_batch* bt, const int32_t* ctas_per_tensor) {
  if (!bt || !ctas_per_tensor) return set_error(STD_EINVAL, "batch or sizes is NULL");
  std::vector<int> g(bt->ctxs.size());
  int mn = 0;
  for (size_t t = 0; t < g.size(); ++t) {
    if (ctas_per_tensor[t] < 1 || ctas_per_tensor[t] > 32)
      return set_error(STD_EINVAL, "a group size is outside [1, 32]");
    g[t] = ctas_per_tensor[t];
    mn = (mn == 0 || g[t] < mn) ? g[t] : mn;
  }
  bt->fixed_g = g;
  bt->group = mn;
  bt->tuned = true;
  bt->promote = false;
  return STD_OK;
}

int std_batch_tile(const std_batch* bt, int32_t* tile) {
  if (!bt || !tile) return set_error(STD_EINVAL, "batch or output is NULL");
  *tile = bt->tile;
  return STD_OK;
}

int std_batch_groups(const std_batch* bt, int32_t* ctas_per_tensor) {
  if (!bt || !ctas_per_tensor) return set_error(STD_EINVAL, "batch or output is NULL");
  for (size_t t = 0; t < bt->ctxs.size(); ++t)
    ctas_per_tensor[t] = t < bt->last_g.size() ? bt->last_g[t] : 0;
  return STD_OK;
}

int std_batch_epoch(std_batch* bt, float lr_a, float lr_b, float lambda_a, float lambda_b, int32_t minibatch,
                    std_batch_stats* out) {
  return std_batch_step(bt, lr_a, lr_b, lambda_a, lambda_b, minibatch, INT64_MAX, out);
}

int std_reserve(std_ctx* c, int32_t minibatch, int32_t ctas_per_tensor, int64_t max_query) {
  if (!c) return set_error(STD_EINVAL, "context is NULL");
  if (minibatch < 1) return set_error(STD_EINVAL, "minibatch must be >= 1");
  if (minibatch > STD_MAX_MINIBATCH) return set_error(STD_EUNSUPPORTED, "minibatch exceeds STD_MAX_MINIBATCH");
  if (ctas_per_tensor < 1 || ctas_per_tensor > kMaxEpochCtas)
    return set_error(STD_EINVAL, "ctas_per_tensor must be in [1, 256]");
  if (c->cursor > 0 && c->cursor_M != minibatch)
    return set_error(STD_EINVAL, "an epoch is in progress with another minibatch size");
  if (max_query < 0) return set_error(STD_EINVAL, "max_query must be >= 0");
  int rc = ensure_schedule(c, minibatch);
  if (!rc) rc = ensure_scratch(c, ctas_per_tensor, payload_floats(c->g), minibatch);
  if (!rc && c->opt.ptr_kind == 0 && max_query > 0)
    rc = ensure_stage(c, (size_t)max_query * c->g.N * 4 + (size_t)max_query * 4 + 16);
  if (rc) return rc;
  STD_CUDA(cudaStreamSynchronize(c->stream), "reserve sync");
  return STD_OK;
}

int std_device_bytes(const std_ctx* c, uint64_t* bytes) {
  if (!c || !bytes) return set_error(STD_EINVAL, "context or output is NULL");
  *bytes = (uint64_t)c->allocated;
  return STD_OK;
}

int std_watchdog_probe(uint64_t watchdog_ns, int32_t* status) {
  if (!status) return set_error(STD_EINVAL, "status is NULL");
  if (watchdog_ns < 1000ULL || watchdog_ns > 10000000000ULL)
    return set_error(STD_EINVAL, "watchdog_ns must be in [1e3, 1e10]");
  int* err = nullptr;
  unsigned long long* word = nullptr;
  cudaError_t e = cudaMalloc((void**)&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&word, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(word, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = launch_wait_probe(watchdog_ns, err, word, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  cudaFree(word);
  if (e != cudaSuccess) return cuda_error(e, "watchdog probe");
  *status = h;
  return STD_OK;
}

int std_progress(const std_ctx* c, int64_t* epoch, int64_t* next_batch) {
  if (!c) return set_error(STD_EINVAL, "context is NULL");
  if (epoch) *epoch = c->epoch;
  if (next_batch) *next_batch = c->cursor;
  return STD_OK;
}

}  // extern "C"
