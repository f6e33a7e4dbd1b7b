/*
 * lk_layout.h -- memory layout shared by the host runtime and the persistent
 * kernel (internal; not part of the public ABI).
 *
 * Host-mapped pinned memory (the host<->device mailboxes of Sec. II.D):
 *   ring[c][R]      descriptor slots of cluster c (the to_GPU side).  A slot is
 *                   one 64-byte line; its `seq` word is written last, with
 *                   release order, and names the slot's position in the
 *                   cluster's FIFO (1-based).  Table 1's single to_GPU integer
 *                   becomes the slot's `cmd` (THREAD_WORK + op, THREAD_EXIT).
 *   cword[c]        per-cluster from_GPU words: `done` (seq of the last
 *                   finished descriptor, monotone), `status` (Table 1 code),
 *                   each on its own 128-byte line.
 *   ctrl            abort word, heartbeat, boot / exit counters, first error.
 *   info[g]         (cluster, rank, smid) of CTA g, written at boot.
 * Device memory (cluster-internal relay, L2-resident):
 *   dcl[c]          broadcast ring (D slots), generation, device-side done,
 *                   arrival counters, per-rank partial sums, histogram
 *                   accumulators.
 *   log[g][cap]     execution-log records (lk_exec_rec) of CTA g.
 */
#ifndef LK_LAYOUT_H
#define LK_LAYOUT_H
#include <stdint.h>
#include "../../include/lk.h"

#define LK_LINE 128
#define LK_BCAST_DEPTH 4          /* descriptors a cluster may have in flight */
#define LK_MAX_CTAS 1024          /* upper bound on CTAs per context          */
#define LK_MAX_CLUSTERS 256

/* One mailbox slot: 64 bytes, seq published last. */
typedef struct __attribute__((aligned(64))) {
  uint64_t seq;     /* 1-based FIFO position; written last (release)   */
  uint32_t cmd;     /* LK_CMD_WORK + op, or LK_CMD_EXIT                 */
  uint32_t flags;
  uint64_t n;
  uint64_t in0;
  uint64_t in1;
  uint64_t out;
  uint64_t aux;
  uint64_t t_pick;  /* device-side: %globaltimer when the master took it */
} lk_slot;

typedef struct __attribute__((aligned(LK_LINE))) {
  uint64_t done;                 /* seq of the last finished descriptor (device writes) */
  uint8_t pad0[LK_LINE - 8];
  uint64_t status;               /* LK_ST_* (device writes)                             */
  uint64_t error;                /* LK_DERR_* that stopped this cluster, 0 = none       */
  uint8_t pad1[LK_LINE - 16];
} lk_cword;

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
  int32_t pad;
} lk_cta_info;

/* Per-cluster relay state in device memory. */
typedef struct __attribute__((aligned(LK_LINE))) {
  uint64_t gen;                          /* descriptors relayed so far (master writes)  */
  uint8_t pad0[LK_LINE - 8];
  uint64_t dev_done;                     /* descriptors finished (last arriver writes)  */
  uint8_t pad1[LK_LINE - 8];
  uint32_t arrive[LK_BCAST_DEPTH];       /* CTAs done with relay slot d                 */
  uint8_t pad2[LK_LINE - 4 * LK_BCAST_DEPTH];
  lk_slot bcast[LK_BCAST_DEPTH];         /* relay ring                                  */
  uint32_t hist[LK_BCAST_DEPTH][256];    /* histogram accumulators, zero at rest        */
  float partial[LK_BCAST_DEPTH][LK_MAX_CTAS]; /* per-rank partial sums                  */
} lk_dcluster;

/* Everything the persistent kernel needs; passed by value at launch. */
typedef struct {
  lk_slot* ring;                 /* [C][R]; host-mapped (live) or device (finite mode)  */
  lk_cword* cword;               /* [C] host-mapped                                     */
  lk_ctrl* ctrl;                 /* host-mapped                                         */
  lk_cta_info* info;             /* [G] host-mapped                                     */
  lk_dcluster* dcl;              /* [C] device                                          */
  int32_t* cl_start;             /* [C+1] device: prefix sums of cluster sizes          */
  int32_t* pin_smid;             /* [total] device, or NULL: explicit SM ids by (c, r)  */
  int32_t* boot_smid;            /* [G] device: boot exchange                           */
  uint32_t* boot_count;          /* device: boot barrier counter                        */
  lk_exec_rec* log;              /* [G][log_cap] device, or NULL                        */
  uint64_t* log_count;           /* [G] device: records written per CTA                 */
  int32_t num_clusters;
  int32_t grid;
  int32_t total;                 /* CTAs that join clusters (= sum of sizes)            */
  uint32_t ring_mask;            /* R - 1                                               */
  uint32_t log_cap;
  uint32_t flags;
  uint64_t backoff_base_ns;
  uint64_t backoff_cap_ns;
  uint64_t lease_ns;
  uint64_t boot_timeout_ns;
} lk_kargs;

#endif
