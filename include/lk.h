/*
 * lk.h -- LightKernel-GB300: persistent-thread work dispatch for one GPU.
 *
 * The method is Burgio, "Enabling predictable parallelism in single-GPU
 * systems with persistent CUDA threads" (LightKernel, LK):
 *   - Sec. II.C: one CUDA kernel is spawned once; it holds exactly one block
 *     per SM, pinned at boot, and its threads spin-wait for work.
 *   - Sec. I / II.A: the host sends a persistent thread "a descriptor of the
 *     work and a reference to the in/out data items", and software maps work
 *     and data onto a chosen cluster of SMs.
 *   - Sec. II.D, Table 1: per-SM dual mailboxes (to_GPU / from_GPU) carry
 *     integer status codes between host and device.
 *   - Sec. III: the life cycle Init -> {Copyin, Trigger, Wait, Copyout}* ->
 *     Dispose.  lk_init = Init, lk_submit = Trigger, lk_wait / lk_poll =
 *     Wait, lk_dispose = Dispose.  Copyin / Copyout stay with the caller.
 *
 * A "cluster" here is a caller-chosen set of SMs (one pinned CTA each); the
 * paper's own case is one SM per cluster.  It is not a CUDA thread-block
 * cluster.
 *
 * Threading: lk_submit may be called from many host threads at once (each
 * cluster's mailbox is a multi-producer ring; FIFO order = the order in which
 * submissions obtained their ring ticket).  lk_poll / lk_wait / lk_status may
 * be called from any thread.  lk_init and lk_dispose must not race with other
 * calls on the same context.
 *
 * Errors: every call returns an int status (LK_OK or a negative LK_E* code);
 * nothing throws or aborts across this boundary.  lk_strerror names a code.
 *
 * Memory: the caller owns every in/out buffer (device memory, e.g. torch
 * tensors).  A buffer passed to lk_submit must stay allocated and untouched
 * by other writers until lk_poll / lk_wait has returned LK_OK for that
 * handle.  Outputs are complete and visible to device work the host issues
 * after that return.  The library owns its mailboxes, status words, execution
 * log and the persistent kernel; lk_dispose releases them.
 *
 * While a context runs, its CTAs occupy their SMs: a device-wide synchronise
 * (cudaDeviceSynchronize, torch.cuda.synchronize) blocks until the context is
 * disposed or its idle lease runs out, and so may a device allocation or free
 * (cudaMalloc / cudaFree, e.g. a caching allocator that grows).  Allocate
 * buffers before lk_init; wait on other streams only.
 */
#ifndef LK_H
#define LK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define LK_OK         0   /* success / descriptor finished                  */
#define LK_PENDING    1   /* lk_poll: descriptor not finished yet           */
#define LK_EINVAL    -1   /* bad argument (range, alignment, op, size)      */
#define LK_EAGAIN    -2   /* cluster mailbox ring full; retry later         */
#define LK_ETIMEDOUT -3   /* wait / dispose deadline passed                 */
#define LK_EDEVICE   -4   /* the persistent kernel reported an error, or a CUDA call failed */
#define LK_ESTATE    -5   /* context not running (exited, disposed, lease expired) */
#define LK_ENOMEM    -6   /* host or device allocation failed               */
#define LK_EBUSY     -7   /* lk_dispose: kernel still running after the abort; context kept */

/* ---- from_GPU status codes (Table 1, Sec. II.D) ------------------------ */
#define LK_ST_INIT      0  /* THREAD_INIT: booted, nothing run yet           */
#define LK_ST_FINISHED  1  /* THREAD_FINISHED: last descriptor completed     */
#define LK_ST_WORKING   2  /* THREAD_WORKING: a descriptor is running        */
#define LK_ST_NOP       4  /* THREAD_NOP: idle acknowledgement (one-deep mailbox) */
/* build-only statuses beyond Table 1 */
#define LK_ST_EXITED    8  /* the cluster's CTAs returned after EXIT         */
#define LK_ST_ERROR    32  /* the cluster stopped on a device-side error     */

/* ---- to_GPU command codes (Table 1, Sec. II.D) ------------------------- */
#define LK_CMD_NOP   4     /* THREAD_NOP                                      */
#define LK_CMD_EXIT  8     /* THREAD_EXIT: run everything posted before, then return */
#define LK_CMD_WORK 16     /* THREAD_WORK: 16 + operation code               */

/* ---- operations (the "work" a descriptor names) ----------------------- */
#define LK_OP_NOP        0 /* no data; measures the dispatch path alone      */
#define LK_OP_ADD_I32    1 /* out[i] = in0[i] + in1[i], int32, wraps mod 2^32; n elements */
#define LK_OP_HIST_U8    2 /* out[v] = #{i : in0[i] == v}; n bytes in, 256 int32 bins out (overwritten) */
#define LK_OP_SUM_F32    3 /* out[0] = sum of n float32 (fixed order for a given n and cluster size) */
#define LK_OP_GEMM64_F32 4 /* n tiles: out[t] = in0[t] x in1[t], 64x64 row-major float32 tiles;     */
                           /* float32 FFMA, or split-bf16 tensor-core MMAs for whole tiles (see   */
                           /* LK_INIT_GEMM_FFMA); per element within 1e-4 sum_k |a b|              */
#define LK_OP_COPY_I32   5 /* out[i] = in0[i], int32; n elements             */
#define LK_OP_COMBINE_SUM  6 /* out[0] = binary64 sum of n float32 partials, one at the start of each */
                             /* 16-byte slot of in0 (fixed order)            */
#define LK_OP_COMBINE_HIST 7 /* out[v] = sum over j < n of in0[256 j + v] (n int32 histograms) */
#define LK_OP_SPIN       8 /* the compute-bound loop of Sec. III: every thread t of CTA r iterates */
                           /* x <- 1664525 x + 1013904223 (mod 2^32) n times from 65536 r + t + 1; */
                           /* no memory traffic; out (optional, uint32 per CTA) receives the XOR    */
                           /* of the CTA's final values                                             */
#define LK_OP_COUNT      9
#define LK_OP_BATCH      9 /* a batch posted by lk_submit_batch (one descriptor, many items) */
#define LK_OP_SERVE     10 /* lk_serve's device queue: the cluster's CTAs claim work units until */
                           /* the queue closes (posted by lk_serve, LK_SERVE_QUEUE)             */

/* ---- device-side error reasons (lk_device_error) ---------------------- */
#define LK_DERR_NONE     0
#define LK_DERR_LEASE    1 /* no work and no heartbeat for idle_lease_ns: kernel returned */
#define LK_DERR_ABORT    2 /* host set the abort word                        */
#define LK_DERR_BOOT     3 /* boot barrier did not complete in time          */
#define LK_DERR_STALL    4 /* a CTA waited too long for its cluster master   */
#define LK_DERR_BADDESC  5 /* descriptor failed the device-side check        */
#define LK_DERR_STAGING  6 /* a shared-memory staging copy did not complete in time */
#define LK_DERR_BOUNDS   7 /* bounds-checking build (liblk_bounds.so) only: a body's index or   */
                           /* address fell outside its operand, share or shared-memory region; */
                           /* the access was skipped (see lk_bounds_violations)                 */

typedef struct lk_ctx lk_ctx;   /* opaque; owned by the library */

/* A handle names one submitted descriptor: (cluster << 48) | seq, seq >= 1
 * its 1-based position in the cluster's FIFO.  0 is never a valid handle. */
typedef uint64_t lk_handle;

/* lk_init parameters.  Zero-initialise, then set what you need. */
typedef struct {
  int device;                  /* CUDA device ordinal                                   */
  int num_clusters;            /* >= 1                                                  */
  const int* sms_per_cluster;  /* [num_clusters] CTAs of each cluster, each >= 1; total */
                               /* <= SM count x ctas_per_sm                             */
  const int* smids;            /* optional: the SM ids of cluster 0, then cluster 1, ... */
                               /* (total entries; an id appears at most ctas_per_sm     */
                               /* times, its k-th appearance naming the SM's k-th CTA); */
                               /* NULL = clusters are cut from the observed CTAs in     */
                               /* slot-major order: every SM's first CTA by ascending   */
                               /* SM id, then every SM's second CTA                     */
  int threads_per_cta;         /* multiple of 32 in [64, 1024]; 0 -> 256                 */
  int ring_depth;              /* descriptors queued per cluster, power of two; 0 -> 1024 */
  uint64_t backoff_base_ns;    /* first __nanosleep of a spin back-off (0 = pure spin)   */
  uint64_t backoff_cap_ns;     /* back-off ceiling; 0 -> 256 ns                          */
  uint64_t idle_lease_ns;      /* the kernel returns after this long with no work and    */
                               /* no heartbeat (lk_submit, lk_poll, lk_wait, lk_sync and */
                               /* lk_heartbeat beat); 0 -> 10 s                          */
  uint64_t boot_timeout_ns;    /* lk_init fails if the CTAs are not all up; 0 -> 10 s    */
  uint32_t exec_log_cap;       /* execution-log records kept per CTA (ring); 0 = no log  */
  uint32_t flags;              /* LK_INIT_* bits                                        */
  uint32_t max_batch_units;    /* work units one batch may hold (lk_submit_batch);      */
                               /* 0 -> 8192                                             */
  uint32_t ctas_per_sm;        /* persistent CTAs on each SM: 0 or 1 -> one (Sec. II.C); */
                               /* 2 -> two, each with half the shared memory (the      */
                               /* "multiple persistent threads" model Sec. II.C leaves  */
                               /* for later); 2 needs threads_per_cta <= 256            */
  uint32_t serve_units;        /* entries of lk_serve's device queue (LK_SERVE_QUEUE):  */
                               /* work units published and not yet read, and requests  */
                               /* completed and not yet retired; power of two in       */
                               /* [256, 2^22]; 0 -> 65536 (72 bytes of pinned host     */
                               /* memory each)                                         */
} lk_init_params;

/* lk_init_params.flags: how descriptors reach a cluster's CTAs.
 * Default: only the cluster's master thread (thread 0 of rank 0, the paper's
 * one master thread per mailbox, Sec. II.D) polls the host-mapped ring, and
 * relays each descriptor to the other CTAs through a tagged slot in device
 * memory.  LK_INIT_DIRECT: every CTA's thread 0 polls the ring itself (no
 * relay hop, but every extra reader of the ring's cache line delays the
 * host's stores to it). */
#define LK_INIT_DIRECT 1u
/* LK_INIT_MAILBOX: the paper's own one-deep mailbox pair per cluster
 * (Sec. II.D, Table 1) instead of the ring.  The host writes the descriptor's
 * words, then release-stores to_GPU = THREAD_WORK + op; the master answers
 * from_GPU = THREAD_WORKING, relays the descriptor to the other CTAs and, once
 * all have finished, writes THREAD_FINISHED.  The host that observes FINISHED
 * (in lk_poll, lk_wait, lk_sync or a later lk_submit) re-arms with
 * to_GPU = THREAD_NOP, and the master acknowledges with from_GPU = THREAD_NOP;
 * only then does the mailbox take the next descriptor.  So at most one
 * descriptor per cluster is in flight, and lk_submit returns LK_EAGAIN until
 * the previous one has finished and its re-arm was acknowledged.  Cannot be
 * combined with LK_INIT_DIRECT (LK_EINVAL). */
#define LK_INIT_MAILBOX 2u
/* LK_INIT_GEMM_FFMA: GEMM tiles always take the float32 FFMA path (k-order
 * fused multiply-adds, bit-reproducible).  Default: whole tiles at 256
 * threads with one CTA per SM run on the tensor cores with operands split
 * into two bf16 parts (each product formed to within 2^-15 |a||b|, inside
 * the GEMM bound 1e-4 sum_k |a b|); tiles split across CTAs always take FFMA. */
#define LK_INIT_GEMM_FFMA 4u

/* A work descriptor.  The in/out pointers travel beside it. */
typedef struct {
  uint32_t op;      /* LK_OP_*                                            */
  uint32_t flags;   /* reserved, 0                                        */
  uint64_t n;       /* elements (ADD/COPY: int32, SUM: float32, HIST: bytes, GEMM: tiles) */
  uint64_t aux;     /* load-rate cap of this descriptor in bytes per      */
                    /* microsecond (= MB/s) over the whole cluster, at     */
                    /* least LK_RATE_MIN; 0 = the cluster's default       */
                    /* (lk_set_rate).  Paces ADD, COPY, SUM, HIST, GEMM    */
                    /* and batches; other ops ignore it                   */
} lk_desc;

/* Smallest load-rate cap (bytes per microsecond = 1 GB/s). */
#define LK_RATE_MIN 1000ull

/* One execution-log record: one CTA's share of one descriptor. */
typedef struct {
  uint64_t seq;        /* descriptor's position in its cluster's FIFO (1-based)    */
  uint32_t cluster;
  uint32_t rank;       /* the CTA's rank inside its cluster (0 = master)           */
  uint32_t smid;       /* %smid read by the CTA when it wrote this record          */
  uint32_t op;         /* the operation it ran                                     */
  uint64_t order;      /* how many descriptors this CTA ran before this one        */
  uint64_t t_pick_ns;  /* %globaltimer: this CTA took the descriptor (from the     */
                       /* ring or mailbox, or a relayed member from the relay)    */
  uint64_t t_start_ns; /* %globaltimer: this CTA started its share                 */
  uint64_t t_end_ns;   /* %globaltimer: this CTA finished its share                */
  uint64_t t_done_ns;  /* %globaltimer of the completion store if this CTA was the */
                       /* last to arrive, else 0                                   */
} lk_exec_rec;         /* 64 bytes */

/* Init (Sec. III): allocate the mailboxes, launch the persistent kernel (one
 * CTA per SM, cooperative launch, enough shared memory that no second CTA
 * fits), and wait until every CTA has read its %smid and joined its cluster.
 * On success *out owns a running context.
 * Errors: LK_EINVAL (partition, sizes), LK_ENOMEM, LK_EDEVICE (CUDA failure,
 * launch refused), LK_ETIMEDOUT (boot did not finish; everything is freed). */
int lk_init(lk_ctx** out, const lk_init_params* p);

/* Trigger (Sec. III): post descriptor d with its data items to `cluster`.
 *   in[0..n_in-1]: device pointers to the inputs (ADD: 2, HIST/SUM/COPY: 1,
 *   GEMM: 2 = A tiles, B tiles, NOP: 0); out: device pointer to the output.
 *   Every non-null pointer must be 16-byte aligned and below 2^48; n must
 *   be at most 2^40 (HIST: below 2^31, GEMM: at most 2^28 tiles).  No CUDA call is made:
 *   the descriptor reaches the device through the mailbox ring only.
 *   Outputs are written while the descriptor runs (a histogram's bins are
 *   cleared by the cluster's first CTA and accumulated by every CTA), so an
 *   output must not be read until the descriptor has finished.  Descriptors
 *   posted to one cluster that write the same output leave the last one's
 *   result when they have the same n (histograms: always).
 * On success *h names the descriptor.
 * Errors: LK_EINVAL (cluster, op, n_in, alignment, n too large),
 * LK_EAGAIN (ring full, or with LK_INIT_MAILBOX the mailbox not idle yet:
 * nothing was posted), LK_ESTATE (context not running). */
int lk_submit(lk_ctx* ctx, int cluster, const lk_desc* d, const void* const* in, int n_in,
              void* out, lk_handle* h);

/* Not in the paper: cap the rate at which `cluster` loads its inputs, for
 * isolation of the other clusters' memory traffic.  Each CTA paces its TMA
 * loads with a token bucket as deep as its stage ring (the burst), so a
 * cluster of S CTAs moves at most about bytes_per_us (MB/s) once past the
 * burst; a paced body takes correspondingly longer.  Applies to
 * descriptors posted after the call whose own lk_desc.aux is 0.
 * bytes_per_us: 0 = unpaced, else >= LK_RATE_MIN and < 2^40.
 * Errors: LK_EINVAL (ctx, cluster, rate). */
int lk_set_rate(lk_ctx* ctx, int cluster, uint64_t bytes_per_us);

/* Not in the paper: load yielding between clusters, for isolation.  While a
 * cluster with role LK_ROLE_CRITICAL has a descriptor running (from its
 * pickup to its last CTA's completion), every cluster with role
 * LK_ROLE_YIELD stops issuing new input loads in its streaming bodies (add,
 * copy, sum, histogram; the loads already in flight complete, and one wait
 * lasts at most 1 ms), so a critical task meets less memory traffic while
 * the yielding work keeps full speed in between.  Roles apply to
 * descriptors posted after the call; a cluster may also keep a rate cap
 * (lk_set_rate).  role: LK_ROLE_NONE, LK_ROLE_CRITICAL or LK_ROLE_YIELD.
 * Errors: LK_EINVAL (ctx, cluster, role). */
#define LK_ROLE_NONE     0
#define LK_ROLE_CRITICAL 1
#define LK_ROLE_YIELD    2
int lk_set_role(lk_ctx* ctx, int cluster, int role);

/* Wait (Sec. III), non-blocking: LK_OK if h finished, LK_PENDING if not.
 * Errors: LK_EINVAL (bad handle), LK_EDEVICE (the cluster stopped on a device
 * error before finishing h), LK_ESTATE (context gone before h finished). */
int lk_poll(lk_ctx* ctx, lk_handle h);

/* Wait (Sec. III), blocking: spin until h finished or timeout_ns elapsed.
 * Returns LK_OK, LK_ETIMEDOUT, or lk_poll's errors. */
int lk_wait(lk_ctx* ctx, lk_handle h, uint64_t timeout_ns);

/* ---- batches: many descriptors in one mailbox post ---------------------- */
/* Not in the paper: one post hands a cluster a whole list of items.  Each
 * item is split into `parts` work units (a unit = one part of one item, run
 * by one CTA); the cluster's CTAs claim units from an atomic ticket, so
 * items of uneven size spread over the cluster.  Parts of a sum or histogram
 * item are combined by the last part to finish (sums: binary64 in part
 * order, so a result depends only on the item's n, its parts and the block
 * size).  One completion covers the whole batch. */
typedef struct {
  const void* in0;        /* device pointers, as lk_submit                        */
  const void* in1;
  void* out;
  uint32_t op;            /* LK_OP_NOP .. LK_OP_COPY_I32                          */
  uint32_t parts;         /* CTAs sharing the item: 1..8, or 0 = from the tune    */
  uint64_t n;             /* as lk_desc.n                                          */
} lk_batch_item;          /* 40 bytes */

typedef struct {
  uint32_t max_parts;     /* cap on parts of an item (1..8, and at most the       */
                          /* cluster size); 0 -> 8                                 */
  uint32_t reserved;
  uint64_t part_bytes;    /* an item with parts == 0 gets ceil(input bytes /       */
                          /* part_bytes) parts, capped; 0 -> 4 MiB                 */
} lk_batch_tune;

/* Post `count` items (host array; copied by the call, so it may be reused at
 * once) to `cluster` as one descriptor.  The expanded unit table lives in
 * library-owned pinned host-mapped memory until the batch finishes; the
 * items' data buffers follow lk_submit's ownership rule.  A batch starts
 * only after every earlier descriptor of its cluster has finished.
 * tune: NULL = defaults.  *h names the batch (lk_wait / lk_poll as usual).
 * Errors: LK_EINVAL (an item fails lk_submit's checks, too many units, too
 * many split sum / histogram items), LK_EAGAIN (ring or batch buffers busy),
 * LK_ESTATE. */
int lk_submit_batch(lk_ctx* ctx, int cluster, const lk_batch_item* items, uint32_t count,
                    const lk_batch_tune* tune, lk_handle* h);

/* The same items as one CUDA graph of ordinary launches (one kernel per item,
 * the same bodies; grid = clamp(ceil(input bytes / 256 KiB), 1, max_ctas)
 * CTAs of `threads` threads), captured once, then launched `reps` times with
 * a synchronise after each.  ms[r] receives launch-to-synchronise-return time
 * of repetition r (host clock).  Must not run while a full-chip context is
 * alive.  Returns LK_OK, LK_EINVAL, LK_EDEVICE. */
int lk_baseline_graph(int device, const lk_batch_item* items, uint32_t count, int max_ctas, int threads,
                      int reps, float* ms);

/* ---- serving: continuous admission of requests ------------------------- */
/* Not in the paper.  Requests arrive over time from several host producer
 * threads; one dispatcher admits them in arrival order while the bytes they
 * hold (inputs, outputs, scratch) fit in a device-memory budget.  Two ways to
 * run what is admitted (lk_serve_params.mode):
 *   LK_SERVE_QUEUE (device-resident queue): each admitted request is split
 *     into work units (see the split rule below), which the host
 *     publishes into a ring in pinned host-mapped memory, one unit of each
 *     admitted request in turn (so a request that arrives while large ones
 *     run is interleaved with them), at most window x (CTAs) units ahead of
 *     the completed requests.  One LK_OP_SERVE descriptor per cluster turns
 *     every CTA of every cluster into a worker: it claims the next unit index
 *     from one device counter, runs that part, and the request's last part
 *     combines it (sums in part order, histograms) and appends the request
 *     to a completion ring the host reads.  The host only admits, publishes
 *     and retires; no host round trip is spent per unit.
 *   LK_SERVE_CHUNKS (host dispatcher): each request is split into chunks of
 *     at most chunk_bytes of input, one descriptor each, which the host posts
 *     to every cluster as its in-flight window (window chunks) frees up; a
 *     split sum or histogram ends with one LK_OP_COMBINE_* descriptor.
 * Either way results do not depend on what else runs (all clusters must have
 * the same size). */
#define LK_SERVE_CHUNKS 0
#define LK_SERVE_QUEUE  1
typedef struct {
  uint64_t t_arrival_ns;  /* arrival time relative to the run's start         */
  uint32_t op;            /* LK_OP_ADD_I32 .. LK_OP_COPY_I32                  */
  uint32_t producer;      /* host producer thread that injects it             */
  uint64_t n;             /* as lk_desc.n                                      */
  const void* in0;        /* device pointers, resident for the whole run      */
  const void* in1;
  void* out;              /* device output, or NULL: taken from the arena      */
} lk_request;             /* 48 bytes */

typedef struct {
  uint64_t t_admit_ns;    /* admitted (budget granted), relative to start      */
  uint64_t t_complete_ns; /* last descriptor of the request observed finished  */
  void* out;              /* where the output was written                      */
  int32_t status;         /* LK_OK or an LK_E* code                            */
  uint32_t chunks;        /* descriptors the request ran as (without combine)  */
} lk_request_result;      /* 32 bytes */

typedef struct {
  int n_producers;            /* >= 1; request.producer < n_producers             */
  int window;                 /* CHUNKS: chunks each cluster may hold at once;     */
                              /* QUEUE: units published ahead of the completed     */
                              /* requests, per serving CTA; 0 -> 2                 */
  uint64_t chunk_bytes;       /* CHUNKS: input bytes per chunk; 0 -> 16 MiB        */
  uint64_t budget_bytes;      /* admission budget: bytes held by admitted,         */
                              /* unfinished requests                              */
  void* arena;                /* device memory (256-byte aligned) for outputs of    */
                              /* requests with out == NULL and for the per-chunk   */
                              /* partials of split sums and histograms; QUEUE: its */
                              /* first lk_serve_queue_state_bytes(max_inflight)    */
                              /* bytes hold the queue's device state               */
  uint64_t arena_bytes;
  uint64_t timeout_ns;        /* whole run; 0 -> 120 s                            */
  uint64_t coalesce_bytes;    /* requests of at most this many input bytes run as  */
                              /* items of batch posts (lk_submit_batch), many to a */
                              /* post, so that one dispatch serves them all; 0 =   */
                              /* off; at most chunk_bytes                          */
  uint32_t coalesce_max;      /* requests per coalesced post; 0 -> 256, <= 256     */
  uint32_t coalesce_part_bytes; /* input bytes per work unit of a coalesced item   */
                              /* (its CTAs: at most 8); 0 -> 256 KiB              */
  uint32_t mode;              /* LK_SERVE_CHUNKS or LK_SERVE_QUEUE                  */
  uint32_t max_inflight;      /* QUEUE: admitted, unfinished requests at most;     */
                              /* 0 -> 4096                                        */
  uint64_t part_bytes;        /* QUEUE: largest unit (input bytes); 0 -> 8 MiB;    */
                              /* at most 2^40                                      */
  uint64_t min_part_bytes;    /* QUEUE: smallest unit when a request is spread      */
                              /* wider; 0 -> 128 KiB; 64 KiB <= it <= part_bytes   */
} lk_serve_params;

/* How LK_SERVE_QUEUE splits a request of B input bytes into units (at most
 * 1024): at least ceil(B / part_bytes); a sum (whose float result depends
 * on its split) exactly
 *   max(ceil(B / part_bytes), min(S, ceil(B / min_part_bytes))),
 * S = the context's CTAs, so it is the same whatever else is served; any
 * other op as many as max(ceil(B / f), min(idle, ceil(B /
 * min_part_bytes))), where idle = S minus the backlog when it is admitted
 * (the admitted units no CTA has claimed yet; units already running do not
 * count) and f = part_bytes while that backlog holds at least S x
 * part_bytes input bytes (the queue is saturated), else
 * max(min_part_bytes, part_bytes / 8).  Their results do not depend on the
 * split, so a request spreads over the CTAs that no queued unit waits for,
 * in units of at most f. */

/* The rule above as a function: the units LK_SERVE_QUEUE gives a request of
 * `op` (ADD, HIST, SUM, GEMM or COPY) over n elements (bytes, tiles) on a
 * context of `ctas` CTAs, admitted while `backlog_units` units of
 * `backlog_bytes` input bytes wait unclaimed; part_bytes and
 * min_part_bytes as in lk_serve_params (0 -> the defaults).  Host-only:
 * no device or context is touched.  Returns 0 for an op outside that set,
 * ctas = 0 or parts sizes lk_serve would refuse (min_part_bytes below
 * 64 KiB or above part_bytes, part_bytes above 2^40). */
uint32_t lk_serve_parts(uint32_t op, uint64_t n, uint32_t ctas, uint64_t backlog_units, uint64_t backlog_bytes,
                        uint64_t part_bytes, uint64_t min_part_bytes);

/* Device bytes the queue's state takes at the start of the arena
 * (LK_SERVE_QUEUE) for `max_inflight` request slots (0 -> 4096). */
uint64_t lk_serve_queue_state_bytes(uint32_t max_inflight);

/* Run the requests through the context's clusters (all of one size) and
 * fill res[i] for each.  A request's result does not depend on the mix:
 * QUEUE, as the units the split rule above gives (res.chunks = units);
 * CHUNKS, as
 * chunks of at most chunk_bytes (one descriptor each, then one combine
 * descriptor for split sums and histograms), or, when it is at most
 * coalesce_bytes, as one item of a batch post split by coalesce_part_bytes
 * (coalescing applies to CHUNKS only).  Outputs taken from the arena are
 * released when the request completes (read them before the next call
 * reuses the arena).  In QUEUE mode the context must have been created live
 * (lk_init) and nothing else may be posted to it during the call.
 * Returns LK_OK if every request finished, LK_EINVAL, LK_ENOMEM (a request
 * needs more arena or budget than exists), or the first error. */
int lk_serve(lk_ctx* ctx, const lk_request* reqs, size_t count, const lk_serve_params* p,
             lk_request_result* res);

/* ---- the paper's life-cycle measurement (Sec. III, Tables 2-3) ---------- */
typedef struct {
  uint64_t init_ns;      /* LK: lk_init          | CUDA: cudaMalloc of the output  */
  uint64_t trigger_ns;   /* LK: lk_submit        | CUDA: cudaLaunchKernel          */
  uint64_t wait_ns;      /* LK: lk_wait          | CUDA: cudaStreamSynchronize     */
  uint64_t dispose_ns;   /* LK: lk_dispose       | CUDA: cudaFree                  */
} lk_phase_times;

/* `runs` times: Init a context of one cluster of `sms` CTAs (`threads` each),
 * Trigger one LK_OP_SPIN descriptor of `iters` iterations, Wait for it,
 * Dispose; host CLOCK_MONOTONIC time of each phase into out[run].  out_dev
 * (optional, device, `sms` uint32) receives the spin results of the last
 * run.  Returns LK_OK or the first error. */
int lk_phase_run(int device, int sms, int threads, uint64_t iters, int runs, void* out_dev, lk_phase_times* out);

/* The traditional life cycle of the same work: Alloc (cudaMalloc of the
 * output), Spawn (cudaLaunchKernel of the spin body, grid = sms CTAs of
 * `threads`), Wait (cudaStreamSynchronize), Dispose (cudaFree), `runs`
 * times.  out_dev as above. */
int lk_baseline_phase_run(int device, int sms, int threads, uint64_t iters, int runs, void* out_dev,
                          lk_phase_times* out);

/* Refresh the idle lease without posting work.  LK_OK or LK_EINVAL. */
int lk_heartbeat(lk_ctx* ctx);

/* Wait until every descriptor submitted so far, on every cluster, finished.
 * Returns LK_OK, LK_ETIMEDOUT, or lk_poll's errors. */
int lk_sync(lk_ctx* ctx, uint64_t timeout_ns);

/* Dispose (Sec. III): post EXIT (THREAD_EXIT, Table 1) behind everything
 * already queued, wait for the kernel to return, free everything.  If the
 * kernel has not returned after timeout_ns, set the abort word (every device
 * wait checks it) and wait up to timeout_ns + 2 s more.
 * Returns LK_OK (freed), LK_EDEVICE (kernel had reported an error; freed),
 * LK_ETIMEDOUT (kernel returned only after the abort; freed), LK_EBUSY (the
 * kernel is still running: nothing is freed under it and ctx stays valid, so
 * lk_dispose may be called again), LK_EINVAL (null ctx). */
int lk_dispose(lk_ctx* ctx, uint64_t timeout_ns);

/* The SM ids of `cluster`'s CTAs by rank (Sec. II.C: blocks are pinned to
 * SMs at boot).  Writes min(size, cap) ids; returns the cluster size, or
 * LK_EINVAL. */
int lk_cluster_info(lk_ctx* ctx, int cluster, int* smids, int cap);

/* from_GPU status of `cluster` (Table 1): LK_ST_INIT after boot until the
 * first post, LK_ST_WORKING while posted descriptors are unfinished,
 * LK_ST_FINISHED once all of them finished, LK_ST_EXITED / LK_ST_ERROR after
 * the cluster's CTAs returned.  With LK_INIT_MAILBOX the word the master
 * writes is returned as it is, LK_ST_NOP (re-arm acknowledged) included.
 * LK_EINVAL for a bad cluster. */
int lk_status(lk_ctx* ctx, int cluster);

/* First device-side error reason (LK_DERR_*), or LK_EINVAL. */
int lk_device_error(lk_ctx* ctx);

/* Number of SMs of the context's device and of CTAs in the context. */
int lk_num_sms(lk_ctx* ctx);
int lk_num_ctas(lk_ctx* ctx);

/* Copy the execution log out: up to `cap` records, grouped by CTA, each CTA's
 * records in the order it ran them (only the last exec_log_cap per CTA are
 * kept).  *n receives the count written; *dropped (optional) the number of
 * older records overwritten.  Safe while the context runs (the records of
 * descriptors still running may be absent) and after lk_dispose has stopped
 * the kernel.  Returns LK_OK, LK_EINVAL, LK_EDEVICE. */
int lk_exec_log(lk_ctx* ctx, lk_exec_rec* buf, size_t cap, size_t* n, uint64_t* dropped);

/* Human-readable name of an LK_* return code. */
const char* lk_strerror(int code);

/* ---- finite mode: one launch that runs a fixed list and returns -------- */
/* Runs `count` descriptors through a fresh persistent kernel whose mailbox
 * ring is pre-filled in device memory and ends with EXIT, so the kernel needs
 * no host interaction and can be timed with CUDA events or replayed by a
 * profiler.  cluster_of[i] names descriptor i's cluster; in0/in1/out are
 * per-descriptor device pointers (NULL where unused).  *elapsed_ms (optional)
 * receives the CUDA-event time of the launch.  If log_out is non-null it
 * receives up to log_cap execution-log records and *log_n their count.
 * Returns LK_OK or the lk_init / lk_dispose errors. */
int lk_run_finite(const lk_init_params* p, const lk_desc* descs, const int* cluster_of,
                  const void* const* in0, const void* const* in1, void* const* out, size_t count,
                  float* elapsed_ms, lk_exec_rec* log_out, size_t log_cap, size_t* log_n);

/* ---- trace runner: timed submission streams (native, no Python in the loop) */
typedef struct {
  uint64_t t_arrival_ns;  /* release time relative to the run's start               */
  int32_t cluster;        /* target cluster (LK) or stream slot (ordinary launches) */
  uint32_t op;            /* LK_OP_*                                                */
  uint64_t n;             /* as lk_desc.n                                           */
  const void* in0;        /* device pointers, as lk_submit                          */
  const void* in1;
  void* out;
  const void* h_in0;      /* LK_TRACE_E2E only: pinned host copies of the inputs    */
  const void* h_in1;      /* (copied to in0 / in1 before the item is released)      */
  void* h_out;            /* ... and the host buffer `out` is copied back to        */
  uint64_t in0_bytes;     /* bytes copied for each                                  */
  uint64_t in1_bytes;
  uint64_t out_bytes;
} lk_trace_item;          /* 96 bytes */

typedef struct {
  uint64_t t_submit_ns;   /* host CLOCK_MONOTONIC at submit entry (E2E: at the start */
                          /* of the input copy), relative to the run's start         */
  uint64_t t_complete_ns; /* host time the completion was observed (E2E: the output  */
                          /* copy finished)                                          */
  int32_t status;         /* LK_OK or the error the item hit                        */
  int32_t thread;         /* host thread that handled it                            */
  uint64_t t_post_ns;     /* the work was posted or launched (E2E: after the input  */
                          /* copy)                                                  */
  uint64_t t_observed_ns; /* its completion was observed (E2E: before the output    */
                          /* copy); E2E latency = copy in + dispatch + copy out     */
} lk_trace_result;        /* 40 bytes */

#define LK_TRACE_OPEN   0  /* release on arrival; several items in flight per cluster */
#define LK_TRACE_CLOSED 1  /* a thread releases its next item after the previous one finished */
#define LK_TRACE_E2E    2  /* closed loop with host->device input and device->host output copies */

/* Run a trace through a running context.  Items are split across n_threads
 * host threads by cluster (cluster % n_threads); each thread releases its
 * items in t_arrival order, no earlier than their arrival time, in the given
 * mode (LK_TRACE_*).  Latency = t_complete - t_submit.
 * pin_cpu_base >= 0 pins thread i to CPU pin_cpu_base + i.
 * Returns LK_OK if every item finished, else the first error. */
int lk_run_trace(lk_ctx* ctx, const lk_trace_item* items, size_t count, int n_threads,
                 int mode, int pin_cpu_base, uint64_t timeout_ns, lk_trace_result* res);

/* The same trace as ordinary kernel launches: per item, cudaLaunchKernel of
 * the same body with grid = ctas_of_slot[item.cluster] CTAs of `threads`
 * threads, then cudaStreamSynchronize; one non-blocking stream per slot.
 * mode LK_TRACE_E2E adds the same copies as lk_run_trace; other modes are
 * closed loop per thread (a launch returns only after its item finished).
 * Must not run while a full-chip context is alive (its CTAs hold the SMs). */
int lk_baseline_run_trace(int device, const lk_trace_item* items, size_t count, int n_slots,
                          const int* ctas_of_slot, int threads, int n_threads, int mode,
                          int pin_cpu_base, lk_trace_result* res);

/* Dispose (as lk_dispose) and report the persistent kernel's lifetime from
 * CUDA events recorded around its launch on its own stream (-1 if unknown). */
int lk_dispose_timed(lk_ctx* ctx, uint64_t timeout_ns, float* kernel_ms);

/* ---- one ordinary launch that allocates nothing ------------------------ */
/* The paper has no counterpart: this is a convenience of this library.
 * It runs one descriptor as an ordinary kernel launch (the same bodies and
 * split as lk_baseline_run_trace: `ctas` CTAs of `threads` threads) on the
 * caller's `stream` (a cudaStream_t; NULL = the legacy default stream) and
 * returns without waiting.  Unlike every other entry point it calls no
 * cudaMalloc, cudaFree or other allocating routine: the scratch that the sum
 * and histogram bodies use to combine per-CTA results is one file-scope
 * device array of 5,248 bytes, so it suits callers that cannot allocate --
 * a real-time loop that must not take the allocator's unbounded latency
 * after start-up, or a host thread sharing the GPU with a running persistent
 * context, where an allocation or free can block until that kernel returns.
 *   device: CUDA ordinal; in[0..n_in-1], out: device pointers, 16-byte
 *   aligned, as lk_submit.  ctas: 1..1024 (the array holds one partial sum per
 *   CTA: more is rejected with LK_EINVAL, nothing launched).
 * The argument checks are lk_submit's (op, inputs, n limits, alignment, the
 * pointers an op dereferences; d->aux is checked and then ignored), made
 * before any CUDA call.
 * The first call on a device looks up the array's device address and clears
 * it (an asynchronous memset on `stream`); make that first call before any
 * stream capture.  All calls on a device share the one array and each
 * launch's last CTA leaves it zeroed for the next, so calls whose launches
 * overlap on the GPU race on it: serialise them (one stream, or events).  A
 * launch that is refused (LK_EDEVICE) or that never starts (an earlier error
 * on the stream) does not touch the array; a launch whose CTAs run always
 * ends with its last CTA re-zeroing it, a body that gives up on a staging
 * copy included; only a fault that destroys the CUDA context leaves it
 * undefined, and the array goes with that context.
 * Returns LK_OK (launched), LK_EINVAL, LK_EDEVICE (CUDA error). */
int lk_launch_noalloc(int device, const lk_desc* d, const void* const* in, int n_in, void* out,
                      int ctas, int threads, void* stream);

/* ---- the bounds-checking build ---------------------------------------- */
/* The paper has no counterpart: this is a test aid of this library.
 * liblk_bounds.so is this library compiled with -DLK_DEBUG_BOUNDS: every
 * body checks, before each global-memory access path and shared-memory or
 * TMEM region it uses, that the index or address lies inside the operand
 * (as the descriptor's n sizes it), the CTA's or warp's share, and the
 * region, and that vector and TMA addresses are 16-byte aligned.  A failed
 * check skips the access (a skipped TMA copy completes its barrier phase
 * with no bytes), counts a violation, records the first site (LK_OOB_*
 * values of lk_device.cuh: 1 share, 2 staged load, 3 stage region, 4 store,
 * 5 histogram counter, 6 GEMM load, 7 GEMM store, 8 GEMM shared memory or
 * TMEM) and makes that descriptor end with LK_DERR_BOUNDS (lk_wait returns
 * LK_EDEVICE).  It stands in for a device memory checker.
 *   device: CUDA ordinal.  count, first_site: out.  Read it with no context
 *   running on the device (the read is an ordinary synchronous copy).
 * Returns LK_OK; LK_EINVAL in the product build (liblk.so) or for NULL
 * outputs; LK_EDEVICE (CUDA error). */
int lk_bounds_violations(int device, uint64_t* count, uint32_t* first_site);

/* Host-mapped round-trip floor: one host thread release-stores a counter, one
 * GPU thread acquire-spins on it and release-stores an echo, the host
 * acquire-spins on the echo.  Writes `iters` round-trip times (ns). */
int lk_pingpong(int device, int iters, uint64_t* rtt_ns);

#ifdef __cplusplus
}
#endif
#endif /* LK_H */
