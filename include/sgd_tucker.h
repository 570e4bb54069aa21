/*
 * sgd_tucker.h — C ABI of the GB300 SGD_Tucker library (libsgdtucker.so).
 *
 * SGD_Tucker (Li et al., arXiv 2012.03550) decomposes a sparse N-order tensor
 * X (I_1 x ... x I_N, given as COO nonzeros) into factor matrices
 * A(n) in R^{I_n x J_n} and a core G-hat that is itself a Kruskal product of
 * matrices B(n) in R^{J_n x R_core} (Sec. 4.1, Eq. 4):
 *     G-hat = sum_r b(1)_{:,r} o ... o b(N)_{:,r},
 *     x-hat(i_1..i_N) = G-hat x_1 a(1)_{i_1,:} ... x_N a(N)_{i_N,:}   (Def. 6).
 * Training is the minibatch SGD of Algorithm 1 (Sec. 4.3, Eqs. 13-18): for
 * each minibatch Psi of M sampled nonzeros, a core phase that updates every
 * column b(n)_{:,r} cyclically (Eq. 15), the rebuild of G-hat (Eq. 4), and a
 * factor phase that updates every touched row a(n)_{i,:} (Eq. 18), mode after
 * mode.  All kernels run on one GPU (sm_103a).
 *
 * Conventions for every call:
 *  - Every function returns STD_OK (0) or a negative status; none aborts.
 *    std_last_error() returns a thread-local message for the last failure.
 *  - Indices are 0-based (the paper is 1-based).  Coordinates are int32,
 *    row-major [k][N].  Factor matrices cross the ABI dense row-major
 *    (I_n x J_n), Kruskal matrices row-major (J_n x R_core), the core as a
 *    vector of prod J_n floats with mode 1 fastest (Vec_1 of Def. 2).
 *  - Pointer arguments are host pointers when std_options.ptr_kind = 0 and
 *    device pointers (e.g. torch data_ptr()) when ptr_kind = 1.  The library
 *    never takes ownership of caller memory; buffers may be freed after the
 *    call returns.  Output buffers are owned by the caller.
 *  - A context owns all device memory it allocates and runs every kernel on
 *    std_options.stream.  Calls on one context must not overlap; distinct
 *    contexts are independent.  All calls are synchronous with respect to the
 *    host unless noted.
 */
#ifndef SGD_TUCKER_H
#define SGD_TUCKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define STD_OK            0
#define STD_EINVAL      (-1)  /* bad argument: N, I_n, J_n, M, index >= I_n, null pointer */
#define STD_ENOMEM      (-2)  /* device allocation failed or the HBM budget was exceeded */
#define STD_ECUDA       (-3)  /* a CUDA runtime call failed (message has the CUDA error) */
#define STD_ETIMEOUT    (-4)  /* a device grid barrier exceeded its watchdog budget */
#define STD_ENUMERIC    (-5)  /* NaN or Inf met in a reduction */
#define STD_EUNSUPPORTED (-6) /* shape beyond the kernels' compiled limits (see below) */

/* Kernel limits (checked by std_create / std_sgd_epoch, STD_EUNSUPPORTED):
 * 2 <= N <= STD_MAX_ORDER, 1 <= J_n <= STD_MAX_RANK, 1 <= R_core <= STD_MAX_RANK,
 * prod J_n <= STD_MAX_CORE, minibatch M <= STD_MAX_MINIBATCH. */
#define STD_MAX_ORDER     6
#define STD_MAX_RANK      32
#define STD_MAX_CORE      16384
#define STD_MAX_MINIBATCH 16384

typedef struct std_ctx std_ctx;

/* Options of a context; initialise with std_default_options(). */
typedef struct {
    int32_t  r_core;      /* R_core >= 1, Kruskal rank of the core (Eq. 4); default 5 (Sec. 5.3) */
    int32_t  precision;   /* 0: FP32 everywhere; 1: BF16 copies of A and G-hat for gathers and
                             the core contraction, FP32 accumulation and FP32 master A, B */
    int32_t  norm_mode;   /* factor-row normaliser: 0 = minibatch size M (Eq. 18, default),
                             1 = |Psi_i|, the row's sample count (Algorithm 1, factor update) */
    int32_t  init_mode;   /* initial A, B: 0 = N(init_mu, init_sigma^2) (Sec. 5.1: 0.5, 0.1),
                             1 = N(0, 1/J_n); drawn on the device from seed_init */
    double   init_mu;
    double   init_sigma;
    uint64_t seed_init;   /* initial-parameter stream */
    uint64_t seed_sched;  /* minibatch-sampler key: epoch e visits the training entries in the
                             order of a keyed permutation of [0, nnz) (see std_sgd_epoch) */
    int32_t  ptr_kind;    /* 0: pointers are host memory; 1: pointers are device memory */
    int32_t  ctas;        /* CTAs of the persistent epoch kernel; 0 = chosen by the library */
    void*    stream;      /* cudaStream_t for every kernel and copy; NULL = the legacy stream */
    uint64_t watchdog_ns; /* grid-barrier wait budget in ns; 0 = 2e9 (2 s) */
    uint64_t hbm_budget_bytes; /* cap on the context's device allocations; 0 = none */
    int32_t  contraction; /* factor-phase E_s = G-hat_(n) S_s^T (Eq. 11, Algorithm 1's
                             factor phase): 0 = Kronecker row S_s against the unfolded core (default);
                             1 = the same product through the core's Kruskal form (Eq. 4):
                             E_s = B(n) w_s, w_s[r] = prod_{k != n} <a(k)_{i_k,:}, b(k)_{:,r}>,
                             O(R sum_k J_k) instead of O(J_n prod_{k != n} J_k) per sample */
    float    momentum;    /* heavy-ball momentum mu in [0, 1) for every update of Algorithm 1
                             (Kruskal columns and factor rows): v <- mu v + g, w <- w - lr v, g the
                             regularised gradient; 0 = plain SGD (default).  The accelerated SGD
                             the paper names as future work (Sec. 6).  Velocities start at zero,
                             are kept per parameter on the device, and std_set_params resets them */
    int32_t  snapshot;    /* K-snapshot form, a labelled variant of Algorithm 1's minibatch order
                             (the paper has no counterpart; it amortises the chain of dependent
                             phases of Algorithm 1 over K minibatches): 0 or 1 = Algorithm 1's
                             order (default); K >= 2 = the minibatches of a call are taken in blocks
                             of K consecutive ones (the first block starting at the call's first
                             minibatch), every minibatch of a block runs Algorithm 1's step from the
                             model as it stood when the block began, and their changes
                             (w <- w + delta, delta = -lr * gradient) are added to that model in
                             minibatch order.  K groups of CTAs run a block's minibatches at once.
                             Limits: K <= 64, K * ceil(M / 256) CTAs resident, momentum 0
                             (STD_EINVAL otherwise); batched launches refuse such contexts */
    int32_t  tile;        /* register tile of the FP32 factor-phase contraction E_s = G-hat_(n) S_s^T
                             (Eqs. 10-11): samples per thread sharing each unfolded-core load,
                             1, 2 or 4; 0 = chosen from the chunk size (default).  Every sample's
                             sums are formed in the same order whatever the tile, so results are
                             the same bits.  Batched launches run every tensor with the batch's
                             tile instead (std_batch_tile).  Other values: STD_EINVAL */
} std_options;

/* Fill *opt with the defaults listed above. */
void std_default_options(std_options* opt);

/*
 * Create a context holding the training tensor and the model: the problem of
 * Sec. 3.2 (the sparse tensor X over the observed set Omega, Table 1 notation;
 * the low-rank model of Def. 6 with the core of Eq. 4, Sec. 4.1), with X held
 * as one COO copy on the device (Sec. 4.4.2).
 *   order        N (2..STD_MAX_ORDER)
 *   mode_sizes   I_n, n < N (each >= 1, < 2^31)
 *   ranks        J_n, n < N (1..STD_MAX_RANK)
 *   nnz          number of training nonzeros (>= 1, < 2^31)
 *   indices      nnz x N int32 coordinates, 0-based, row-major (host or device per ptr_kind)
 *   values       nnz float values
 *   opt          options (NULL = defaults)
 * The COO is copied into library-owned device memory (coordinates checked
 * against I_n: STD_EINVAL on an index outside [0, I_n)).  A and B are drawn
 * per init_mode.  Errors: STD_EINVAL, STD_EUNSUPPORTED, STD_ENOMEM, STD_ECUDA;
 * on error *out is NULL and nothing is leaked.
 */
int std_create(std_ctx** out, int32_t order, const int64_t* mode_sizes, const int32_t* ranks,
               int64_t nnz, const int32_t* indices, const float* values, const std_options* opt);

/* Release every resource of the context created by std_create (the COO copy
 * of Sec. 4.4.2 and the model of Def. 6 / Eq. 4) after the context's
 * stream drains; NULL is a no-op.  Returns STD_OK. */
int std_destroy(std_ctx* ctx);

/* Per-epoch statistics (nullable output of std_sgd_epoch). */
typedef struct {
    double  seconds;        /* device time of the epoch (sampler, tiler and update kernels) */
    double  sched_seconds;  /* device time of the sampler/tiler kernel alone */
    double  update_seconds; /* device time of the persistent update kernel alone */
    double  nnz_per_s;      /* nnz / seconds */
    int64_t nnz;         /* training nonzeros visited */
    int64_t batches;     /* minibatches in the epoch (the last one may be short) */
    int64_t epoch;       /* index of the epoch just run */
} std_epoch_stats;

/*
 * One training epoch (Algorithm 1 over every minibatch).  Epoch e visits the
 * training entries in the order pi_e(0), pi_e(1), ... where pi_e is a keyed
 * permutation of [0, nnz) (a balanced 6-round Feistel network with SplitMix64
 * rounds, restricted to [0, nnz) by cycle walking, keyed by seed_sched and e);
 * minibatch b is positions [bM, min(bM+M, nnz)), and a short last minibatch
 * uses its own size as M in every normaliser.  Per minibatch:
 *   core phase, n = 1..N, r = 1..R_core in order (Algorithm 1, core phase):
 *     b(n)_r <- b(n)_r - lr_b (V / M + lambda_b b(n)_r),  V of Eq. 15;
 *     lr_b = 0 leaves B unchanged and the core phase is skipped (the paper's
 *     schedule that updates B only in some epochs, Sec. 5.3);
 *   G-hat from B (Eq. 4);
 *   factor phase, n = 1..N in order (Algorithm 1): every row i touched by the
 *     minibatch, all rows of a mode reading the state before that mode's update:
 *     a(n)_i <- a(n)_i - lr_a (F / M_i + lambda_a a(n)_i),  F of Eq. 18,
 *     M_i = M (norm_mode 0) or the row's sample count (norm_mode 1).
 * minibatch: 1..STD_MAX_MINIBATCH.  The epoch counter then advances.
 * Errors: STD_EINVAL, STD_EUNSUPPORTED, STD_ENOMEM, STD_ECUDA, STD_ETIMEOUT.
 */
int std_sgd_epoch(std_ctx* ctx, float lr_a, float lr_b, float lambda_a, float lambda_b,
                  int32_t minibatch, std_epoch_stats* out);

/* Gradient probe of std_sgd_batches: host buffers filled for the first
 * minibatch of the range (any member may be NULL). */
typedef struct {
    float*   core_V;    /* [N][R_core][STD_MAX_RANK]: V of Algorithm 1's core phase (the bracket of
                           Eq. 15) for each mode n and column r, in update order */
    float*   factor_F;  /* [N][M][STD_MAX_RANK]: F of Algorithm 1's factor phase (the bracket of
                           Eq. 18) for each mode n and each touched row, rows ascending */
    int64_t* nseg;      /* [N]: touched rows per mode */
} std_probe;

/*
 * Minibatches [batch_begin, batch_end) of the current epoch's schedule (same
 * definition as std_sgd_epoch), without advancing the epoch counter.  With a
 * probe, the gradients of the first minibatch of the range are recorded.
 */
int std_sgd_batches(std_ctx* ctx, float lr_a, float lr_b, float lambda_a, float lambda_b,
                    int32_t minibatch, int64_t batch_begin, int64_t batch_end, std_probe* probe);

/*
 * The sampler and tiler output of the current epoch for minibatches
 * [batch_begin, batch_end): for the `count` positions t of those minibatches,
 *   sample_ids[t]            training-entry index pi_e(t)                 (int32[count])
 *   order[n][t]              batch position of the q-th entry after the stable
 *                            sort of the minibatch by i_n                  (int32[N][count])
 *   seg_start[n][t], seg_end[n][t]  first and last sorted position (within the
 *                            minibatch) of the run of equal i_n holding sorted
 *                            position q                                    (int32[N][count])
 * where t = (minibatch start) + q.  Any output may be NULL.  Host buffers.
 */
int std_schedule(std_ctx* ctx, int32_t minibatch, int64_t batch_begin, int64_t batch_end,
                 int32_t* sample_ids, int32_t* order, int32_t* seg_start, int32_t* seg_end);

/* x-hat at k coordinates (Def. 6 with the Kruskal core of Eq. 4); out[k]. */
int std_predict(std_ctx* ctx, int64_t k, const int32_t* coords, float* out);

/* std_predict for several contexts in ONE launch (Def. 6 with the core of
 * Eq. 4): k[i] coordinates coords[i] (k[i] x N_i int32, row-major) of
 * ctxs[i] into out[i].  Every context must have the same ptr_kind; host
 * buffers are staged through one stream-ordered allocation on ctxs[0]'s
 * stream.  Each result equals that context's own std_predict bit for bit.
 * Errors: STD_EINVAL (bad arguments, mixed ptr_kind, a coordinate outside
 * [0, I_n): its result is NaN), STD_ECUDA. */
int std_predict_many(int32_t count, std_ctx* const* ctxs, const int64_t* k, const int32_t* const* coords,
                     float* const* out);

/*
 * RMSE and MAE (Eq. 19) of the model over k entries (coords k x N, values k),
 * accumulated in FP64 in a fixed order (bit-reproducible).  mae may be NULL.
 * k = 0 gives 0.  STD_ENUMERIC when the sum is NaN or Inf.
 */
int std_rmse(std_ctx* ctx, int64_t k, const int32_t* coords, const float* values,
             double* rmse, double* mae);

/*
 * Copy the model out: A[n] (I_n x J_n), B[n] (J_n x R_core), core (prod J_n,
 * mode 1 fastest, built from B by Eq. 4) and the epoch counter.  Any array or
 * entry may be NULL.  Buffers per ptr_kind.
 */
int std_get_params(std_ctx* ctx, float* const* A, float* const* B, float* core, int64_t* epoch);

/* Overwrite the model parameters of Def. 6 and Eq. 4 (A[n] in R^{I_n x J_n},
 * B[n] in R^{J_n x R_core}, as in std_get_params; NULL entries are left
 * unchanged), rebuild G-hat from B (Eq. 4), and set the epoch counter
 * (ignored when < 0).  Heavy-ball velocities are reset to zero.  Errors:
 * STD_EINVAL (NULL context), STD_ECUDA. */
int std_set_params(std_ctx* ctx, const float* const* A, const float* const* B, int64_t epoch);

/* Thread-local description of the last error ("" if none). */
const char* std_last_error(void);

/*
 * Batched epochs: many independent decompositions (each its own std_ctx) in
 * one persistent launch.  The GPU's co-resident CTAs are split into groups of
 * `ctas_per_tensor` CTAs; each group runs the epoch of its tensors one after
 * the other (longest first onto the least-loaded group), so small tensors no
 * longer leave the GPU idle behind one tensor's chain of dependent phases
 * (Algorithm 1).  Each tensor's epoch is exactly the one std_sgd_epoch would
 * run with that many CTAs.  The launch sequence (barrier resets, argument
 * uploads from pinned staging, the cooperative kernel) is captured once as a
 * CUDA graph and replayed while the tensors, the group size and the group
 * count stay the same; samplers run before it only when a tensor starts an
 * epoch.
 *   count, ctxs       the contexts (same precision, same stream; each at most
 *                     once); they must outlive the batch, which does not own them
 *   ctas_per_tensor   CTAs per tensor, the same for every tensor; 0 = a base
 *                     size chosen on the first step by timing each power of
 *                     two up to 32 that fits on a run of 3% of every tensor's
 *                     minibatches that writes no parameter (the autotuner),
 *                     and, at every launch, a group of 2^k times the base
 *                     size (up to 32 CTAs, chunks of at least 8 samples) for
 *                     each tensor whose work alone exceeds the average load
 *                     of a base group (std_batch_groups reports the sizes);
 *                     -1 = the tuned size for every tensor, no larger groups
 * Errors: STD_EINVAL, STD_ECUDA.
 */
typedef struct std_batch std_batch;
int std_batch_create(std_batch** out, int32_t count, std_ctx* const* ctxs, int32_t ctas_per_tensor);

typedef struct {
    double  seconds;          /* device time of the batched epoch (samplers, tilers, update kernel) */
    double  update_seconds;   /* device time of the batched update kernel alone */
    double  nnz_per_s;        /* total training nonzeros / seconds */
    int64_t nnz;              /* total training nonzeros visited */
    int32_t tensors;
    int32_t ctas_per_tensor;  /* the base group size (std_batch_groups gives each tensor's) */
    int32_t graph_replayed;   /* 1: the launch replayed the captured graph; 0: it was (re)captured */
    int32_t reserved;
} std_batch_stats;

/* Up to max_batches minibatches of every tensor of the batch, each tensor
 * continuing its epoch in progress (a context keeps its position between
 * calls, so tensors can join and leave between steps); a tensor that
 * completes its epoch advances its epoch counter and starts the next epoch at
 * the next step.  Same hyperparameters and minibatch size for all; the
 * minibatch sequence is std_sgd_epoch's.  std_sgd_epoch refuses a context
 * whose epoch is in progress.  Errors: STD_EINVAL, STD_EUNSUPPORTED,
 * STD_ENOMEM, STD_ECUDA, STD_ETIMEOUT. */
int std_batch_step(std_batch* batch, float lr_a, float lr_b, float lambda_a, float lambda_b,
                   int32_t minibatch, int64_t max_batches, std_batch_stats* out);

/* Replace the batch's tensors (same rules as std_batch_create; same precision
 * and stream as the batch), keeping its buffers, its tuned group size and
 * its captured launch for reuse; per-tensor sizes from std_batch_set_groups
 * are dropped (set them again for the new members).  For a serving loop whose
 * set of jobs changes between steps.  Errors: STD_EINVAL. */
int std_batch_reset(std_batch* batch, int32_t count, std_ctx* const* ctxs);

/* Fix each tensor's group size (count entries in [1, 32], in the order of
 * std_batch_create): no tuner and no promotion; tensors of one size share
 * groups of that size, and the size class with the highest mean load per
 * group gains a group while CTAs remain, up to one group per tensor.  A tensor's result then depends only
 * on its own size, not on the other tensors (the serving loop sizes each job
 * from its own shape).  Errors: STD_EINVAL. */
int std_batch_set_groups(std_batch* batch, const int32_t* ctas_per_tensor);

/* CTAs each tensor of the batch had in the last launch (count entries, in
 * the order of std_batch_create; 0 before the first launch).  A tensor's
 * result equals std_sgd_epoch's with that many CTAs. */
int std_batch_groups(const std_batch* batch, int32_t* ctas_per_tensor);

/* The FP32 contraction tile the batch runs with (std_options.tile: 0 = from
 * each tensor's chunk size, else 1, 2 or 4 for every tensor).  With
 * ctas_per_tensor = 0 the tuner picks it on the first step, after the group
 * size, by timing each choice on the same dry run; results are the same bits
 * whatever the tile.  Until then, and with fixed group sizes, it is 0.
 * Errors: STD_EINVAL (NULL arguments). */
int std_batch_tile(const std_batch* batch, int32_t* tile);

/* std_batch_step without a limit: every tensor finishes its current epoch. */
int std_batch_epoch(std_batch* batch, float lr_a, float lr_b, float lambda_a, float lambda_b,
                    int32_t minibatch, std_batch_stats* out);

/* The context's epoch counter and the next minibatch of its epoch in
 * progress (0 at an epoch boundary). */
int std_progress(const std_ctx* ctx, int64_t* epoch, int64_t* next_batch);

/* Allocate now everything that batched steps at this minibatch size and a
 * group of ctas_per_tensor CTAs (or fewer) need: the current epoch's sample
 * schedule and the exchange scratch; for a host-pointer context also the
 * staging of std_predict / std_rmse calls of up to max_query coordinates.
 * Later calls of that shape allocate nothing, so std_device_bytes then gives
 * the context's whole footprint and a host-side admission rule can rely on
 * it.  Counted against hbm_budget_bytes.  Errors: STD_EINVAL,
 * STD_EUNSUPPORTED, STD_ENOMEM, STD_ECUDA. */
int std_reserve(std_ctx* ctx, int32_t minibatch, int32_t ctas_per_tensor, int64_t max_query);

/* Bytes of device memory the context holds (COO, parameters, schedule,
 * scratch). */
int std_device_bytes(const std_ctx* ctx, uint64_t* bytes);

/* Failure-detection check of the epoch kernels' bounded waits: one thread
 * waits, through the same wait routine, for a tagged exchange word that
 * nothing writes, with a watchdog of watchdog_ns (1e3..1e10).  *status gets
 * the error the device recorded: STD_ETIMEOUT when the watchdog expired as it
 * must.  Nothing faults and the device stays usable.  Errors: STD_EINVAL,
 * STD_ECUDA. */
int std_watchdog_probe(uint64_t watchdog_ns, int32_t* status);

/* Release the batch (not its contexts; NULL is a no-op). */
int std_batch_destroy(std_batch* batch);

/*
 * RMSE and MAE without any device allocation.  The paper has no counterpart:
 * this is for callers that cannot let a library allocate device memory, such
 * as a serving process whose device memory is all reserved by its own pool
 * allocator, or a latency-critical loop that cannot pay for cudaMalloc and
 * cudaFree (cudaFree synchronises the whole device).
 *
 * Same quantity as std_rmse (Eq. 19) for the model given by the caller:
 *   order, mode_sizes[N], ranks[N], r_core   host values (limits as std_create)
 *   A[N]     host array of device pointers; A[n] is I_n x J_n, row-major
 *   B[N]     host array of device pointers; B[n] is J_n x r_core, row-major
 *   coords   device, k x N int32 (0-based); values: device, k floats
 *   out      device, 2 doubles: {rmse, mae}; {0, 0} when k = 0
 *   stream   cudaStream_t (NULL = legacy stream)
 * The call only enqueues two kernels on `stream` and returns; read `out`
 * after synchronising the stream.  A coordinate outside [0, I_n) is never
 * read through: it makes both results NaN.  Sizes beyond the limits return
 * STD_EUNSUPPORTED.  The library cannot check the device pointers: A[n],
 * B[n], coords, values and out must be device memory of the stated sizes on
 * the current device (the Python binding checks this before the call).
 * Scratch: a fixed __device__ array of STD_STATIC_RMSE_BLOCKS x 2 doubles
 * (16 KiB) inside the library, held by every GPU that loads the library until
 * the process exits.  It is not zeroed: each call writes every slot it reads.
 * Every call shares it, so calls that overlap on the GPU (concurrent streams,
 * other threads) race and must be serialised by the caller.  The first call
 * on each device looks up the array's device address with that device
 * current; make that first call before any stream capture.  The address is
 * kept for the life of the process, so the call must not be used on a device
 * after cudaDeviceReset in the same process.
 */
#define STD_STATIC_RMSE_BLOCKS 1024
int std_rmse_static(int32_t order, const int64_t* mode_sizes, const int32_t* ranks, int32_t r_core,
                    const float* const* A, const float* const* B, int64_t k, const int32_t* coords,
                    const float* values, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SGD_TUCKER_H */
