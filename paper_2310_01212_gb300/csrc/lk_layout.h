/*
 * lk_layout.h -- memory layout shared by the host runtime and the persistent
 * kernel (internal; not part of the public ABI).
 *
 * Host-mapped pinned memory (the host<->device mailboxes of Sec. II.D):
 *   ring[c][R]      descriptor slots of cluster c (the to_GPU side), one
 *                   64-byte line each, published with a lap tag in every word
 *                   (lk_wire below).  Table 1's single to_GPU integer becomes
 *                   the slot's `cmd` (THREAD_WORK + op, THREAD_EXIT).
 *   rdone[..]       the from_GPU completion words: one per CTA, the seq of
 *                   the last descriptor that CTA finished (monotone); a
 *                   cluster's words are contiguous from rd_off[c], 16 to a
 *                   128-byte line, and the cluster has finished seq once
 *                   every one of its words reaches it.
 *   cword[c]        per-cluster from_GPU words: `done` (one-deep mailbox
 *                   mode: seq of the last finished descriptor), `status`
 *                   (Table 1 code), each on its own 128-byte line.
 *   ctrl            abort word, heartbeat, boot / exit counters, first error.
 *   info[g]         (cluster, rank, smid) of CTA g, written at boot.
 * Device memory (cluster-internal relay, L2-resident):
 *   dcl[c]          relay ring (D slots), generation, per-slot completion
 *                   words and arrival counters, per-rank finished counts
 *                   (one-deep mailbox mode), per-rank partial sums,
 *                   histogram-clear words.
 *   log[g][cap]     execution-log records (lk_exec_rec) of CTA g.
 */
#ifndef LK_LAYOUT_H
#define LK_LAYOUT_H
#include <stdint.h>
#include "../../include/lk.h"

#define LK_LINE 128
#define LK_BCAST_DEPTH 8          /* descriptors a cluster may have in flight */
#define LK_MAX_CTAS 1024          /* upper bound on CTAs per context          */
#define LK_MAX_CLUSTERS 256
#define LK_RDONE_ALIGN 16         /* completion words per 128-byte line        */

/* A descriptor as the device uses it (decoded; also the relay-ring format). */
typedef struct __attribute__((aligned(64))) {
  uint64_t seq;     /* 1-based FIFO position                           */
  uint32_t cmd;     /* LK_CMD_WORK + op, or LK_CMD_EXIT                 */
  uint32_t flags;
  uint64_t n;
  uint64_t in0;
  uint64_t in1;
  uint64_t out;
  uint64_t aux;
  uint64_t t_pick;  /* device-side: %globaltimer when the slot was taken */
} lk_slot;

/* A mailbox slot as it sits in the host-mapped ring: eight 8-byte words.
 * Words 0..5 each carry, in their top 16 bits, the slot's lap tag: for
 * ticket t of a ring of 2^L slots, tag = ((t >> L) + 1) mod 2^16.  The host
 * issues a release fence, then stores the words (8-byte single-copy atomic
 * stores); a reader loads all six words at once and accepts the slot only
 * when every tag equals the lap it waits for, then issues an acquire fence.
 * Pickup thus costs one round trip over the host link instead of two (flag,
 * then payload).  Addresses, n and aux must fit in 48 bits.
 *   w0 = tag | flags << 16 | cmd      w3 = tag | in1
 *   w1 = tag | n                      w4 = tag | out
 *   w2 = tag | in0                    w5 = tag | aux
 *   w6 = seq (t + 1)                  w7 = 0                              */
typedef struct __attribute__((aligned(64))) {
  uint64_t w[8];
} lk_wire;

#define LK_TAG_SHIFT 48
#define LK_LOW48 0x0000ffffffffffffull

#ifdef __CUDACC__
#define LK_HD __host__ __device__ __forceinline__
#else
#define LK_HD static inline
#endif

LK_HD uint64_t lk_lap_tag(uint64_t t, uint32_t ring_log2) { return ((t >> ring_log2) + 1) & 0xffffull; }

/* Decode words 0..5 into a descriptor (tags are checked by the caller). */
LK_HD void lk_wire_decode(const uint64_t w[6], uint64_t seq, lk_slot* d) {
  d->seq = seq;
  d->cmd = (uint32_t)(w[0] & 0xffffull);
  d->flags = (uint32_t)((w[0] >> 16) & 0xffffull);
  d->n = w[1] & LK_LOW48;
  d->in0 = w[2] & LK_LOW48;
  d->in1 = w[3] & LK_LOW48;
  d->out = w[4] & LK_LOW48;
  d->aux = w[5] & LK_LOW48;
  d->t_pick = 0;
}

typedef struct __attribute__((aligned(LK_LINE))) {
  uint64_t done;                 /* seq of the last finished descriptor (device writes) */
  uint8_t pad0[LK_LINE - 8];
  uint64_t status;               /* LK_ST_* (device writes)                             */
  uint64_t error;                /* LK_DERR_* that stopped this cluster, 0 = none       */
  uint8_t pad1[LK_LINE - 16];
} lk_cword;

/* The paper's one-deep to_GPU mailbox of a cluster (LK_INIT_MAILBOX).  The
 * host writes the descriptor's words, then release-stores `to_gpu`
 * (THREAD_NOP, THREAD_EXIT or THREAD_WORK + op, Table 1); the master acquires
 * `to_gpu` and only then reads the words.  The from_GPU side is the
 * cluster's `status` word (lk_cword). */
typedef struct __attribute__((aligned(LK_LINE))) {
  uint64_t n, in0;        /* word pairs on 16-byte boundaries: one vector load each */
  uint64_t in1, out;
  uint64_t aux, flags;
  uint64_t seq;           /* host's count of posts (diagnostic; the device counts its own) */
  uint64_t to_gpu;
  uint8_t pad[LK_LINE - 64];
} lk_mbox;

typedef struct __attribute__((aligned(LK_LINE))) {
  uint64_t abort;                /* host writes non-zero: every device wait returns     */
  uint8_t pad0[LK_LINE - 8];
  uint64_t heartbeat;            /* host increments; refreshes the idle lease           */
  uint8_t pad1[LK_LINE - 8];
  uint32_t booted;               /* CTAs that finished boot (device increments)         */
  uint32_t exited;               /* CTAs that returned                                  */
  uint32_t first_error;          /* first LK_DERR_* (device, atomic CAS from 0)         */
  uint32_t pad2;
  uint8_t pad3[LK_LINE - 16];
} lk_ctrl;

typedef struct {
  int32_t cluster;               /* -1: CTA not used (explicit SM lists)                */
  int32_t rank;
  int32_t smid;
  int32_t slot;                  /* 0, or 1 for the second CTA on its SM                */
} lk_cta_info;

/* Per-cluster state in device memory.  `flag[r]` is the number of
 * descriptors rank r has finished (monotone; one-deep mailbox mode, where
 * rank 0 gathers the flags and completes each descriptor).  In the ring
 * modes every CTA publishes its own completion word to the host instead;
 * descriptor k (0-based) uses slot k mod D of the relay ring, the partials
 * and the histogram-clear word, and its last CTA to arrive on
 * arrive[k mod D] (the one that also combines a sum) resets
 * the counter and release-stores slot_done[k mod D] = k + 1, which gates the
 * slot's reuse by descriptor k + D. */
typedef struct __attribute__((aligned(LK_LINE))) {
  uint32_t count;
  uint8_t pad[LK_LINE - 4];
} lk_line_counter;

typedef struct __attribute__((aligned(LK_LINE))) {
  uint64_t gen;                          /* LK_GEN_STOP once the master stopped         */
  uint8_t pad0[LK_LINE - 8];
  uint64_t slot_done[LK_BCAST_DEPTH];    /* seq of the last finished descriptor of slot */
  uint8_t pad1[LK_LINE - 8 * LK_BCAST_DEPTH];
  lk_line_counter arrive[LK_BCAST_DEPTH]; /* CTAs that finished the slot's descriptor   */
  uint64_t flag[LK_MAX_CTAS];            /* per-rank finished count (mailbox mode)      */
  lk_wire relay[LK_BCAST_DEPTH];         /* relay ring (lap-tagged like the host ring)  */
  uint64_t hzero[LK_BCAST_DEPTH];        /* seq whose histogram output rank 0 cleared   */
  uint8_t pad2[LK_LINE - 8 * LK_BCAST_DEPTH];
  float partial[LK_BCAST_DEPTH][LK_MAX_CTAS]; /* per-rank partial sums                  */
} lk_dcluster;

/* ---- batches (lk_submit_batch) ----------------------------------------- */
/* One work unit = one part of one item; the host expands a batch's items
 * into a unit table in pinned host-mapped memory (48 bytes per unit). */
typedef struct {
  uint64_t in0, in1, out;
  uint64_t n_op;     /* op << 56 | n (n < 2^48)                                 */
  uint64_t meta;     /* part (bits 0-7) | parts (8-15) | combine slot + 1 (16-47, */
                     /* 0 = none: single-part item, or an op needing no combine)   */
  uint64_t item;     /* index of the item in its batch                           */
} lk_unit;

#define LK_BATCH_SPLIT_SUMS 2048   /* multi-part sum items per batch        */
#define LK_BATCH_SPLIT_HISTS 256   /* multi-part histogram items per batch  */
#define LK_BATCH_BUFFERS 2         /* unit tables per cluster               */

typedef struct {
  uint32_t done;                   /* parts finished (the last one resets it) */
  uint32_t pad;
  float partial[8];
} lk_sum_state;

typedef struct {
  uint32_t done;
  uint32_t pad[3];
  uint32_t bins[256];              /* zero at rest                            */
} lk_hist_state;

typedef struct __attribute__((aligned(LK_LINE))) {
  unsigned long long ticket;       /* next unit to claim (rank 0 resets it)   */
  uint8_t pad[LK_LINE - 8];
  lk_sum_state sums[LK_BATCH_SPLIT_SUMS];
  lk_hist_state hists[LK_BATCH_SPLIT_HISTS];
} lk_bcluster;

/* ---- the serving queue (lk_serve, LK_SERVE_QUEUE) ------------------------
 * The host publishes work units (parts of admitted requests) into a ring in
 * pinned host-mapped memory; every CTA of the serving clusters claims the
 * next unit index from one device counter, waits for that entry to be
 * published, runs the part and acknowledges the entry.  The last part of a
 * request combines it (sums in part order, histograms) and appends the
 * request's slot to a completion ring in host-mapped memory.  The host only
 * admits, publishes and retires. */
/* Unit u sits in entry u mod Q.  Like the mailbox ring, every word the host
 * writes carries the lap tag (u >> log2 Q) + 1 in its top 16 bits, so the
 * claimer reads the whole entry in one probe and accepts it when all six
 * tags are current (unit indices below 2^32 per lk_serve call).
 *   w0 = tag | in0      w3 = tag | n
 *   w1 = tag | in1      w4 = tag | op << 32 | parts << 16 | part
 *   w2 = tag | out      w5 = tag | request slot                          */
typedef struct __attribute__((aligned(64))) {
  uint64_t w[6];
  uint64_t ack;      /* device: u + 1 once the claimer has read the entry          */
  uint64_t pad;
} lk_qunit;          /* 64 bytes */

#define LK_SERVE_MAX_PARTS 1024   /* work units of one request           */

typedef struct __attribute__((aligned(LK_LINE))) {
  uint32_t done;                  /* parts finished (the last one resets it)  */
  uint8_t pad[LK_LINE - 4];
  uint32_t bins[256];             /* histogram accumulator, zero at rest      */
  float partial[LK_SERVE_MAX_PARTS]; /* per-part sums                        */
} lk_qslot;

typedef struct __attribute__((aligned(LK_LINE))) {
  unsigned long long head;        /* next unit to claim (every serving CTA)   */
  uint8_t pad0[LK_LINE - 8];
  unsigned long long cq_tail;     /* completions appended                     */
  uint8_t pad1[LK_LINE - 8];
  lk_qunit* units;                /* host-mapped unit ring [qmask + 1]        */
  uint64_t* cq;                   /* host-mapped completion ring [qmask + 1]: */
                                  /* entry p = (p >> qlog2) + 1 << 32 | slot  */
  uint64_t* close;                /* host-mapped: 0 open, else 1 << 63 | units */
  lk_qslot* slots;                /* device: request slots                    */
  uint64_t qmask;
  uint32_t qlog2;
  uint32_t nslots;
} lk_qstate;                      /* device memory (the start of the arena)   */

/* Everything the persistent kernel needs; passed by value at launch. */
#define LK_KFLAG_DIRECT 1u       /* every CTA polls the ring; else the master relays  */
#define LK_KFLAG_MAILBOX 2u      /* the master takes work from lk_mbox, not the ring   */
#define LK_KFLAG_FINITE 4u       /* finite mode: ring pre-filled in device memory      */
#define LK_KFLAG_GEMM_FFMA 8u    /* GEMM tiles on the FFMA path only                   */

/* Descriptor flag bits the host sets in the posted wire (never user-set:
 * lk_desc.flags must be 0): the cluster's lk_set_role. */
#define LK_DFLAG_CRITICAL 1u      /* marks crit_active while it runs              */
#define LK_DFLAG_YIELD    2u      /* its loads wait while crit_active is non-zero */

typedef struct {
  lk_wire* ring;                 /* [C][R]; host-mapped (live) or device (finite mode)  */
  lk_cword* cword;               /* [C] host-mapped                                     */
  uint64_t* rdone;               /* host-mapped per-CTA completion words (rd_off[c] + r) */
  int32_t* rd_off;               /* [C] device: first completion word of each cluster   */
  lk_mbox* mbox;                 /* [C] host-mapped (LK_KFLAG_MAILBOX), else NULL       */
  lk_ctrl* ctrl;                 /* host-mapped                                         */
  lk_cta_info* info;             /* [G] host-mapped                                     */
  lk_dcluster* dcl;              /* [C] device                                          */
  int32_t* cl_start;             /* [C+1] device: prefix sums of cluster sizes          */
  int32_t* pin_smid;             /* [total] device, or NULL: explicit SM ids by (c, r)  */
  int32_t* boot_smid;            /* [G] device: boot exchange                           */
  uint32_t* boot_count;          /* device: boot barrier counter                        */
  lk_exec_rec* log;              /* [G][log_cap] device, or NULL                        */
  uint64_t* log_count;           /* [G] device: records written per CTA                 */
  lk_bcluster* bcl;              /* [C] device: batch tickets and combine state         */
  uint32_t* cta_hist;            /* [total][256] device: single-part histogram bins     */
  int32_t* crit_active;          /* device: critical descriptors running (lk_set_role)  */
  int32_t num_clusters;
  int32_t grid;
  int32_t total;                 /* CTAs that join clusters (= sum of sizes)            */
  uint32_t ring_mask;            /* R - 1                                               */
  uint32_t ring_log2;            /* log2 R                                              */
  uint32_t log_cap;
  uint32_t flags;
  int32_t ctas_per_sm;           /* 1, or 2: two persistent CTAs share each SM          */
  uint64_t backoff_base_ns;
  uint64_t backoff_cap_ns;
  uint64_t lease_ns;
  uint64_t boot_timeout_ns;
} lk_kargs;

#endif
