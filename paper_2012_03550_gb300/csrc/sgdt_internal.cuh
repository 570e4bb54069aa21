// Internal declarations of the GB300 SGD_Tucker library (not part of the ABI).
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "sgd_tucker.h"

namespace sgdt {

constexpr int kMaxN = STD_MAX_ORDER;
constexpr int kMaxJ = STD_MAX_RANK;
constexpr int kEpochThreads = 512;
constexpr int kScheduleThreads = 512;
constexpr int kMaxChunk = 128;          // samples per CTA per phase in the epoch kernel
constexpr int kMaxCorePayload = 8192;   // floats of the per-mode core reduction
constexpr int kMaxEpochCtas = 256;     // CTAs of the epoch kernel (reductions poll 8 words per lane)

// ---------------------------------------------------------------------------
// Minibatch sampler: keyed permutation pi_e of [0, n) used to visit the
// training entries in epoch e.  Balanced Feistel network on 2h bits (Luby &
// Rackoff), 2h the smallest even width with 2^(2h) >= n (h >= 1), six rounds
// (L, R) -> (R, L ^ (F(R ^ K_i) & (2^h - 1))) with F the SplitMix64 output
// function (Steele, Lea & Flood 2014) and K_i = F(seed + (8 e + i + 1) * 0x9E3779B97F4A7C15);
// values >= n are re-encrypted until they fall in [0, n) (cycle walking,
// Black & Rogaway 2002).  Integer-only, so host and device agree bit for bit.
// ---------------------------------------------------------------------------
struct Feistel {
  uint64_t key[6];
  uint64_t n;
  int h;
};

__host__ __device__ __forceinline__ uint64_t splitmix_out(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

inline Feistel make_feistel(uint64_t n, uint64_t seed, uint64_t epoch) {
  Feistel f;
  f.n = n;
  int bits = 0;
  if (n > 1) {
    uint64_t v = n - 1;
    while (v) { ++bits; v >>= 1; }
  }
  f.h = (bits + 1) / 2;
  if (f.h < 1) f.h = 1;
  for (int i = 0; i < 6; ++i)
    f.key[i] = splitmix_out(seed + (8ULL * epoch + (uint64_t)i + 1ULL) * 0x9E3779B97F4A7C15ULL);
  return f;
}

__host__ __device__ __forceinline__ uint64_t feistel_encrypt(const Feistel& f, uint64_t x) {
  const uint64_t mask = (1ULL << f.h) - 1ULL;
  uint64_t L = x >> f.h, R = x & mask;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    uint64_t t = L ^ (splitmix_out(R ^ f.key[i]) & mask);
    L = R;
    R = t;
  }
  return (L << f.h) | R;
}

__host__ __device__ __forceinline__ uint64_t feistel_perm(const Feistel& f, uint64_t t) {
  uint64_t y = feistel_encrypt(f, t);
  while (y >= f.n) y = feistel_encrypt(f, y);
  return y;
}

// ---------------------------------------------------------------------------
// Geometry of a model shared by all kernels.
// ---------------------------------------------------------------------------
struct Geometry {
  int N;
  int R;
  int J[kMaxN];
  int Jp[kMaxN];        // row stride of the FP32 factor matrices (J_n rounded up to 4)
  int Jb[kMaxN];        // row stride of the BF16 factor mirrors (J_n rounded up to 8)
  int boff[kMaxN];      // offset of B(n) (J_n x R, row-major) in the concatenated B
  int joff[kMaxN];      // offset of mode n's row inside a sample's concatenated rows
  int gstride[kMaxN];   // stride of j_n in G-hat (mode 1 fastest)
  int sumJ;
  int prodJ;
  int Jmax;
  int64_t I[kMaxN];
};

// Sorted per-mode copies of one epoch's minibatches (output of the tiler).
// For mode n and epoch position t (minibatch b occupies [bM, bM+m)):
//   coord(n, k, t) = crd[((size_t)n * N + k) * npad + t]
//   val(n, t)      = val[(size_t)n * npad + t]
//   pos(n, t)      = pos[(size_t)n * npad + t]        (batch position before sorting)
//   seg(n, t)      = seg[(size_t)n * npad + t]        (run start | run end << 16, within the minibatch)
//   link(n, k, t)  = link[(size_t)(n * (n - 1) / 2 + k) * npad + t],  k < n:
//                    the start of the mode-k run that holds the same sample
//                    (sorted position in the mode-k copy of the minibatch)
// and sid[t] the training-entry index pi_e(t).  rsp[k][t] (k < N - 1) is the
// tiler's scratch: the mode-k run start of batch position t - bM.  The arrays
// hold the minibatches from b_first on: position t is stored at index
// t - b_first * M (npad positions in all).
struct Schedule {
  int32_t* crd;
  float* val;
  int32_t* pos;
  uint32_t* seg;
  int32_t* sid;
  int32_t* link;
  int32_t* rsp;
  int64_t npad;
  int64_t n;
  int M;
  int64_t b_first;
};

// Words per epoch position of a Schedule of order N.
inline size_t schedule_words_per_position(int N) {
  return (size_t)N * N + 3 * (size_t)N + 1 + (size_t)N * (N - 1) / 2 + (size_t)(N - 1);
}

struct EpochArgs {
  Geometry g;
  float* A[kMaxN];       // FP32 factor masters, I_n x Jp_n
  uint16_t* Ab[kMaxN];   // BF16 mirrors of A (precision 1), I_n x Jb_n
  int precision;         // 0 FP32; 1 BF16 gathers and tensor-core contraction
  float* B;              // concatenated Kruskal matrices (read at start, written at end)
  float* core;           // G-hat output (prod J), written at end
  Schedule s;
  int64_t b0, b1;        // minibatch range
  float lr_a, lr_b, lam_a, lam_b;
  int norm_mode;
  int contraction;       // 0 Kronecker rows x unfolded core; 1 Kruskal form E = B(n) w
  int tile_sg;          // FP32 contraction: samples per thread (1, 2, 4); 0 = from the chunk size
  float momentum;        // heavy-ball mu (0 = plain SGD)
  int dry;               // 1: compute everything, write no parameter (timing runs)
  float* vA[kMaxN];      // factor-row velocities, I_n x Jp_n (momentum != 0)
  float* vB;             // Kruskal-column velocities, concatenated like B (momentum != 0)
  int chunk_max;
  // cross-CTA exchange words: (sequence tag << 32) | float bits
  uint32_t tag_base;           // tag of (minibatch b, mode n) = tag_base + 8 (b - b0) + n
  unsigned long long* part;    // [G][pstride]   per-CTA core-phase Gram partials
  unsigned long long* inbox;   // [G][pstride]   reduced Gram payload, one copy per CTA
  unsigned long long* piece;   // [N][G][Jmax]   run pieces that continue a run begun in an earlier chunk
  unsigned long long* mail;    // [N][M][Jmax]   rows updated this minibatch, by mode-n run start
  int pstride;
  unsigned long long* bar;
  int* err;
  unsigned long long watchdog_ns;
  // probe
  int64_t probe_batch;
  float* probeV;         // [N][R][kMaxJ]
  float* probeF;         // [N][M][kMaxJ], indexed by the run's first sorted position
  // K-snapshot form (k_epoch_snap): snap_k groups of snap_gk CTAs; group q
  // runs minibatch b0 + iK + q of block i from the block's starting model and
  // records its changes; at the block's end they are added in minibatch order.
  int snap_k;
  int snap_gk;
  int snap_grp;          // this CTA's group (set per CTA in the kernel)
  int snap_cta;          // this CTA's index in the whole grid
  float* snap_dB;        // [K][sum_n J_n R] changes of the Kruskal columns
  float* snap_drow;      // [K][N][M][Jmax] changes of the factor rows, by mode-n run start
  int2* snap_list;       // [G][K][N M] (row, mode << 16 | run start) of the rows CTA g applies
  int* snap_count;       // [G][K] entries of each list
};

// A batched launch: EpochArgs of every tensor (device array), and for each
// group q of `group` CTAs the tensors order[first[q] .. first[q+1]).
struct MultiArgs {
  const EpochArgs* items;
  const int* order;
  const int* first;    // group q runs order[first[q] .. first[q+1])
  const int* gstart;   // group q owns CTAs [gstart[q], gstart[q+1])
  int groups;
  int plain;           // every tensor runs with the default options (see epoch_args_plain)
};

// Factor-matrix pointers passed to kernels by value.
struct AParams {
  float* A[kMaxN];
};

// One context's share of a multi-context prediction launch: queries
// [off, off + k) of the launch are its k coordinates (coords, k x N) and
// results (out).
struct PredictItem {
  Geometry g;
  AParams A;
  const float* B;
  const int32_t* coords;
  float* out;
  int64_t k;
  int64_t off;
};

// Launchers (host side, defined in the .cu files).
// The default options (no momentum, no probe minibatch in [b0, b1), the 1/M
// normaliser): the launchers then use the update kernels specialised for them.
bool epoch_args_plain(const EpochArgs& a);
// Those kernels (compiled in their own translation unit): kind 0 k_epoch,
// 1 k_epoch_cl, 2 k_epoch_snap, 3 k_epoch_multi, 4 its cluster form.
const void* epoch_plain_kernel(int kind, int precision);
cudaError_t launch_schedule(const Geometry& g, const uint32_t* coo, int cs, const Feistel& f,
                            const Schedule& s, int64_t b0, int64_t b1, cudaStream_t st);
int epoch_payload_floats(const Geometry& g);   // largest core-phase Gram payload over the modes
bool epoch_gram_fits(const Geometry& g);       // core-phase Gram tiles within the per-thread limit
cudaError_t launch_mirror_bf16(const Geometry& g, float* const* A, uint16_t* const* Ab, cudaStream_t st);
int epoch_chunk_cap(const Geometry& g);   // largest samples per CTA per phase the kernel takes
size_t epoch_smem_bytes(const Geometry& g, int chunk_max, int ctas, int precision);
cudaError_t epoch_kernel_setup(int precision, size_t smem);
int epoch_max_ctas(int precision, size_t smem);
cudaError_t launch_epoch(const EpochArgs& a, int ctas, size_t smem, cudaStream_t st);
cudaError_t epoch_snap_setup(int precision, size_t smem);
int epoch_snap_max_ctas(int precision, size_t smem);
cudaError_t launch_epoch_snap(const EpochArgs& a, int ctas, size_t smem, cudaStream_t st);
cudaError_t launch_wait_probe(unsigned long long watchdog_ns, int* err, const unsigned long long* word,
                              cudaStream_t st);
cudaError_t epoch_multi_setup(int precision, size_t smem);
int epoch_multi_max_ctas(int precision, size_t smem);
cudaError_t launch_epoch_multi(const MultiArgs& m, int precision, int ctas, size_t smem, cudaStream_t st);
// Cluster form of the update kernels: one tensor's group of 2, 4, 8 or 16
// CTAs as one thread block cluster (same results bit for bit as the
// cooperative form with that many CTAs).
bool epoch_cluster_size_ok(int csize);
size_t epoch_smem_bytes_cl(const Geometry& g, int chunk_max, int ctas, int precision);
int epoch_cl_max_clusters(int precision, bool multi, size_t smem, int csize);
cudaError_t launch_epoch_cl(const EpochArgs& a, int ctas, size_t smem, cudaStream_t st);
cudaError_t launch_epoch_multi_cl(const MultiArgs& m, int precision, int csize, size_t smem, cudaStream_t st);
cudaError_t launch_init_params(const Geometry& g, float* const* A, float* B, int mode, double mu,
                               double sigma, uint64_t seed, cudaStream_t st);
cudaError_t launch_check_coords(const Geometry& g, const int32_t* coords, int64_t k, int* err,
                                cudaStream_t st);
cudaError_t launch_pack_coo(const Geometry& g, const int32_t* coords, const float* values, int64_t k,
                            uint32_t* coo, int cs, int* err, cudaStream_t st);
cudaError_t launch_build_core(const Geometry& g, const float* B, float* core, cudaStream_t st);
int predict_blocks(int64_t k);
cudaError_t launch_predict(const Geometry& g, const AParams& A, const float* B, const int32_t* coords,
                           const float* values, int64_t k, float* out, double* partials, int blocks,
                           int* err, cudaStream_t st);
cudaError_t launch_rmse_finish(const double* partials, int blocks, double* result, cudaStream_t st);
cudaError_t launch_predict_multi(const PredictItem* items, int count, int64_t total, int* err, cudaStream_t st);

// Sets the thread-local message returned by std_last_error(); returns code.
int record_error(int code, const std::string& msg);

}  // namespace sgdt
