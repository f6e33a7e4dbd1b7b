/*
 * lk_runtime.cpp -- host side of LightKernel-GB300 (the C ABI of lk.h).
 *
 * The host is the producer side of every cluster's mailbox (Sec. II.D).  A
 * mailbox is a ring of 64-byte slots in pinned host-mapped memory.  Posting
 * (Trigger, Sec. III) is: take a ticket t on the cluster's tail (a CAS that
 * also refuses when the ring is full), fill slot t mod R, then publish it by
 * release-storing seq = t + 1.  No CUDA call is on this path.  Waiting is an
 * acquire load of the cluster's `done` word, which the device release-stores
 * when the last CTA of the cluster finishes a descriptor.
 */
#include <errno.h>
#include <pthread.h>
#include <sched.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "lk_backend.h"
#include "lk_layout.h"
#include "lk_validate.h"

namespace {

inline uint64_t now_ns() {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

template <class T> inline T ld_acq(const T* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
template <class T> inline T ld_rlx(const T* p) { return __atomic_load_n(p, __ATOMIC_RELAXED); }
template <class T, class V> inline void st_rel(T* p, V v) { __atomic_store_n(p, (T)v, __ATOMIC_RELEASE); }
template <class T, class V> inline void st_rlx(T* p, V v) { __atomic_store_n(p, (T)v, __ATOMIC_RELAXED); }

struct alignas(LK_LINE) Tail {
  std::atomic<uint64_t> t{0};
};

constexpr uint64_t kSeqMask = (1ull << 48) - 1;

}  // namespace

struct lk_ctx {
  int device = 0;
  int C = 0;          /* clusters */
  int G = 0;          /* CTAs launched */
  int total = 0;      /* CTAs that join clusters */
  int T = 256;        /* threads per CTA */
  int per_sm = 1;     /* persistent CTAs per SM */
  uint32_t R = 1024;  /* ring depth */
  int sm_count = 0;
  bool finite = false;
  std::vector<int> sizes;
  std::vector<int> cl_start;

  void* mapped_h = nullptr;
  void* mapped_d = nullptr;
  lk_wire* ring_h = nullptr;     /* host view of the ring (live mode) */
  uint32_t R_log2 = 10;
  lk_cword* cword_h = nullptr;
  uint64_t* rdone_h = nullptr;   /* per-CTA completion words (ring modes) */
  std::vector<int> rd_off;       /* first completion word of each cluster */
  lk_ctrl* ctrl_h = nullptr;
  lk_cta_info* info_h = nullptr;

  void* dev_base = nullptr;
  lk_kargs args{};
  uint32_t log_cap = 0;

  Tail* tail = nullptr;          /* [C], host-only tickets */

  /* one-deep mailbox mode (LK_INIT_MAILBOX) */
  bool mailbox = false;
  lk_mbox* mbox_h = nullptr;     /* [C] host-mapped to_GPU mailboxes */
  Tail* rearmed = nullptr;       /* [C] descriptors whose FINISHED the host consumed */

  Tail* rate = nullptr;          /* [C] default load-rate cap (bytes/us), 0 = none */
  Tail* role = nullptr;          /* [C] lk_set_role value                         */

  /* batches: per cluster LK_BATCH_BUFFERS unit tables in host-mapped memory */
  uint32_t max_units = 0;
  lk_unit* units_h = nullptr;    /* [C][LK_BATCH_BUFFERS][max_units] */
  lk_unit* units_d = nullptr;
  struct BatchState {
    std::mutex mu;
    uint64_t next = 0;                          /* batches posted so far */
    uint64_t seq_of[LK_BATCH_BUFFERS] = {0};    /* batch seq that last used each table */
  };
  BatchState* batch = nullptr;   /* [C] */

  /* lk_serve's device queue (live contexts): host-mapped unit ring,
   * completion ring and close word */
  uint32_t qn = 0, qlog2 = 0;
  lk_qunit* q_units_h = nullptr;
  lk_qunit* q_units_d = nullptr;
  uint64_t* q_cq_h = nullptr;
  uint64_t* q_cq_d = nullptr;
  uint64_t* q_close_h = nullptr;
  uint64_t* q_close_d = nullptr;
  lkb_launch* launch = nullptr;
  std::atomic<int> running{0};
};

/* ---------------------------------------------------------------------- */
static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static void beat(lk_ctx* ctx) { st_rlx(&ctx->ctrl_h->heartbeat, now_ns()); }

static int device_err_to_rc(uint32_t e) {
  if (e == LK_DERR_NONE) return LK_OK;
  if (e == LK_DERR_LEASE || e == LK_DERR_ABORT) return LK_ESTATE;
  return LK_EDEVICE;
}

static int op_inputs(uint32_t op) { return lk_op_inputs(op); }

/* Argument checks shared by lk_submit and the finite / trace paths. */
static int validate(const lk_desc* d, const void* in0, const void* in1, int n_in, void* out) {
  return lk_validate_desc(d, in0, in1, n_in, out);
}

/* Publish ticket t into slot s (see lk_wire): a release fence orders every
 * earlier host write before the slot's words; each word carries the lap tag,
 * so a reader that sees all tags current has the whole descriptor. */
static void write_slot(lk_wire* s, uint64_t t, uint32_t R_log2, uint32_t cmd, const lk_desc* d,
                       const void* in0, const void* in1, void* out) {
  const uint64_t tag = lk_lap_tag(t, R_log2) << LK_TAG_SHIFT;
  const uint64_t flags = d ? d->flags : 0;
  __atomic_thread_fence(__ATOMIC_RELEASE);
  st_rlx(&s->w[0], tag | (flags & 0xffffull) << 16 | (uint64_t)(cmd & 0xffffu));
  st_rlx(&s->w[1], tag | ((d ? d->n : 0) & LK_LOW48));
  st_rlx(&s->w[2], tag | ((uint64_t)(uintptr_t)in0 & LK_LOW48));
  st_rlx(&s->w[3], tag | ((uint64_t)(uintptr_t)in1 & LK_LOW48));
  st_rlx(&s->w[4], tag | ((uint64_t)(uintptr_t)out & LK_LOW48));
  st_rlx(&s->w[5], tag | ((d ? d->aux : 0) & LK_LOW48));
  st_rlx(&s->w[6], t + 1);
  st_rlx(&s->w[7], (uint64_t)0);
}

/* Returns the first device-side error, or 0. */
static uint32_t dev_error(lk_ctx* ctx) { return ld_acq(&ctx->ctrl_h->first_error); }

static bool ctx_alive(lk_ctx* ctx) {
  if (!ctx->running.load(std::memory_order_acquire)) return false;
  if (dev_error(ctx) != 0) return false;
  if (ld_acq(&ctx->ctrl_h->exited) != 0) return false;
  return true;
}

/* One-deep mailbox (LK_INIT_MAILBOX): the host half of the four-phase
 * handshake (Sec. II.D, Table 1).  If the cluster's from_GPU word reads
 * THREAD_FINISHED for the newest post, consume that completion once (a CAS
 * on `rearmed`): publish it in the host-side `done` word that every wait
 * path reads, then re-arm with to_GPU = THREAD_NOP.  FINISHED can only mean
 * the newest post: the next post waits for the master's NOP acknowledgement
 * of this re-arm. */
static void mbox_observe(lk_ctx* ctx, int c) {
  const uint64_t t = ctx->tail[c].t.load(std::memory_order_acquire);
  uint64_t r = ctx->rearmed[c].t.load(std::memory_order_acquire);
  if (r >= t) return;
  if (ld_acq(&ctx->cword_h[c].status) != LK_ST_FINISHED) return;
  if (!ctx->rearmed[c].t.compare_exchange_strong(r, t, std::memory_order_acq_rel)) return;
  st_rel(&ctx->cword_h[c].done, t);
  st_rel(&ctx->mbox_h[c].to_gpu, (uint64_t)LK_CMD_NOP);
}

/* Finished descriptors of cluster c (FIFO: every seq <= the value).  Ring
 * modes: every CTA of the cluster publishes the seq of the last descriptor
 * it finished, so the cluster has finished the minimum of its words.  The
 * words are read with plain loads, all in flight together, and one acquire
 * fence follows (acquire loads would each wait for the one before). */
static uint64_t cl_done(lk_ctx* ctx, int c) {
  if (ctx->mailbox) {
    mbox_observe(ctx, c);
    return ld_acq(&ctx->cword_h[c].done);
  }
  const uint64_t* w = ctx->rdone_h + ctx->rd_off[c];
  const int S = ctx->sizes[c];
  uint64_t m = ld_rlx(&w[0]);
  for (int r = 1; r < S; ++r) {
    const uint64_t v = ld_rlx(&w[r]);
    m = v < m ? v : m;
  }
  __atomic_thread_fence(__ATOMIC_ACQUIRE);
  return m;
}

/* Mailbox post: only when the previous descriptor finished, was re-armed and
 * the master acknowledged the re-arm (from_GPU = THREAD_NOP); the CAS on the
 * tail makes one of several racing producers the owner.  The descriptor's
 * words are stored first; the release store of to_GPU publishes them. */
static int post_mailbox(lk_ctx* ctx, int c, uint32_t cmd, const lk_desc* d, const void* in0, const void* in1,
                        void* out, uint64_t* seq_out) {
  Tail& tl = ctx->tail[c];
  uint64_t t = tl.t.load(std::memory_order_acquire);
  for (;;) {
    if (t > 0) {
      if (cl_done(ctx, c) < t) return LK_EAGAIN;
      if (ld_acq(&ctx->cword_h[c].status) != LK_ST_NOP) return LK_EAGAIN;
    }
    if (tl.t.compare_exchange_weak(t, t + 1, std::memory_order_acq_rel, std::memory_order_acquire)) break;
  }
  lk_mbox* mb = &ctx->mbox_h[c];
  st_rlx(&mb->n, d ? d->n : 0);
  st_rlx(&mb->in0, (uint64_t)(uintptr_t)in0);
  st_rlx(&mb->in1, (uint64_t)(uintptr_t)in1);
  st_rlx(&mb->out, (uint64_t)(uintptr_t)out);
  st_rlx(&mb->aux, d ? d->aux : 0);
  st_rlx(&mb->flags, (uint64_t)(d ? d->flags : 0));
  st_rlx(&mb->seq, t + 1);
  st_rel(&mb->to_gpu, (uint64_t)cmd);
  *seq_out = t + 1;
  return LK_OK;
}

/* Ticket + publish.  Returns LK_OK / LK_EAGAIN.  A descriptor without its
 * own rate cap carries the cluster's default (lk_set_rate) in `aux`, and
 * every descriptor the cluster's role (lk_set_role) in its flag bits. */
static int post(lk_ctx* ctx, int c, uint32_t cmd, const lk_desc* d, const void* in0, const void* in1,
                void* out, uint64_t* seq_out) {
  lk_desc paced;
  const uint64_t role = ctx->role[c].t.load(std::memory_order_relaxed);
  if (d && (!d->aux || role)) {
    paced = *d;
    if (!paced.aux) paced.aux = ctx->rate[c].t.load(std::memory_order_relaxed);
    paced.flags |= role == LK_ROLE_CRITICAL ? LK_DFLAG_CRITICAL : role == LK_ROLE_YIELD ? LK_DFLAG_YIELD : 0u;
    d = &paced;
  }
  if (ctx->mailbox) return post_mailbox(ctx, c, cmd, d, in0, in1, out, seq_out);
  Tail& tl = ctx->tail[c];
  uint64_t t = tl.t.load(std::memory_order_relaxed);
  for (;;) {
    uint64_t done = cl_done(ctx, c);
    if (t - done >= ctx->R) return LK_EAGAIN;   /* slot t mod R still holds descriptor t-R+1 */
    if (tl.t.compare_exchange_weak(t, t + 1, std::memory_order_acq_rel, std::memory_order_relaxed)) break;
  }
  lk_wire* s = &ctx->ring_h[(size_t)c * ctx->R + (t & (ctx->R - 1))];
  write_slot(s, t, ctx->R_log2, cmd, d, in0, in1, out);
  *seq_out = t + 1;
  return LK_OK;
}

/* ---------------------------------------------------------------------- */
/* Build the memory layout.  live: ring in host-mapped memory, else device. */
static int setup(lk_ctx* ctx, const lk_init_params* p, bool live, uint32_t ring_depth_override) {
  if (!p || p->num_clusters < 1 || p->num_clusters > LK_MAX_CLUSTERS || !p->sms_per_cluster)
    return LK_EINVAL;
  lkb_props props;
  int rc = lkb_props_get(p->device, &props);
  if (rc != LK_OK) return rc;
  if (!props.can_map_host || !props.cooperative) return LK_EDEVICE;
  ctx->device = p->device;
  ctx->sm_count = props.sm_count;
  ctx->C = p->num_clusters;
  ctx->sizes.assign(p->sms_per_cluster, p->sms_per_cluster + p->num_clusters);
  ctx->cl_start.assign(ctx->C + 1, 0);
  for (int c = 0; c < ctx->C; ++c) {
    if (ctx->sizes[c] < 1) return LK_EINVAL;
    ctx->cl_start[c + 1] = ctx->cl_start[c] + ctx->sizes[c];
  }
  ctx->total = ctx->cl_start[ctx->C];
  if (p->ctas_per_sm > 2) return LK_EINVAL;
  ctx->per_sm = p->ctas_per_sm == 2 ? 2 : 1;
  if (ctx->total > ctx->per_sm * props.sm_count || ctx->total > LK_MAX_CTAS) return LK_EINVAL;
  if (p->smids) {
    std::vector<int> seen(props.sm_count, 0);
    for (int i = 0; i < ctx->total; ++i) {
      if (p->smids[i] < 0 || p->smids[i] >= props.sm_count || seen[p->smids[i]] >= ctx->per_sm) return LK_EINVAL;
      seen[p->smids[i]]++;
    }
    ctx->G = ctx->per_sm * props.sm_count;   /* every CTA slot of every SM; those not listed return at boot */
  } else {
    ctx->G = ctx->total;
  }
  ctx->T = p->threads_per_cta ? p->threads_per_cta : 256;
  if (ctx->T < 64 || ctx->T > 1024 || ctx->T % 32) return LK_EINVAL;
  if (ctx->per_sm == 2 && ctx->T > 256) return LK_EINVAL;
  uint32_t R = ring_depth_override ? ring_depth_override : (p->ring_depth ? (uint32_t)p->ring_depth : 1024u);
  if (R < 2 || (R & (R - 1)) || R > (1u << 24)) return LK_EINVAL;
  ctx->R = R;
  ctx->R_log2 = 0;
  while ((1u << ctx->R_log2) < R) ctx->R_log2++;
  ctx->log_cap = p->exec_log_cap;
  if (p->flags & ~(uint32_t)(LK_INIT_DIRECT | LK_INIT_MAILBOX | LK_INIT_GEMM_FFMA)) return LK_EINVAL;
  if ((p->flags & LK_INIT_DIRECT) && (p->flags & LK_INIT_MAILBOX)) return LK_EINVAL;
  ctx->mailbox = live && (p->flags & LK_INIT_MAILBOX);

  /* host-mapped block: [ring (live only)] cword[C] rdone[..] ctrl info[G] [unit tables, mailboxes,
   * serving queue (live only)] */
  ctx->max_units = live ? (p->max_batch_units ? p->max_batch_units : 8192u) : 0u;
  if (ctx->max_units > (1u << 22)) return LK_EINVAL;
  size_t off_ring = 0;
  size_t ring_bytes = (size_t)ctx->C * R * sizeof(lk_wire);
  size_t off_cw = live ? align_up(ring_bytes, LK_LINE) : 0;
  /* per-CTA completion words: each cluster's on lines of its own */
  ctx->rd_off.assign(ctx->C, 0);
  size_t rd_words = 0;
  for (int c = 0; c < ctx->C; ++c) {
    ctx->rd_off[c] = (int)rd_words;
    rd_words += align_up((size_t)ctx->sizes[c], LK_RDONE_ALIGN);
  }
  size_t off_rd = align_up(off_cw + ctx->C * sizeof(lk_cword), LK_LINE);
  size_t off_ctrl = align_up(off_rd + rd_words * sizeof(uint64_t), LK_LINE);
  size_t off_info = align_up(off_ctrl + sizeof(lk_ctrl), LK_LINE);
  size_t off_units = align_up(off_info + ctx->G * sizeof(lk_cta_info), LK_LINE);
  size_t units_bytes = (size_t)ctx->C * LK_BATCH_BUFFERS * ctx->max_units * sizeof(lk_unit);
  size_t off_mbox = align_up(off_units + units_bytes, LK_LINE);
  size_t mbox_bytes = ctx->mailbox ? ctx->C * sizeof(lk_mbox) : 0;
  /* the serving queue: unit ring, completion ring, close word (live only) */
  ctx->qn = live ? (p->serve_units ? p->serve_units : 65536u) : 0u;
  if (live && (ctx->qn < 256 || ctx->qn > (1u << 22) || (ctx->qn & (ctx->qn - 1)))) return LK_EINVAL;
  ctx->qlog2 = 0;
  while (ctx->qn && (1u << ctx->qlog2) < ctx->qn) ctx->qlog2++;
  size_t off_q = align_up(off_mbox + mbox_bytes, LK_LINE);
  size_t off_cq = align_up(off_q + (size_t)ctx->qn * sizeof(lk_qunit), LK_LINE);
  size_t off_close = align_up(off_cq + (size_t)ctx->qn * sizeof(uint64_t), LK_LINE);
  size_t mapped_bytes = align_up(off_close + (ctx->qn ? LK_LINE : 0), 4096);
  rc = lkb_alloc_mapped(ctx->device, mapped_bytes, &ctx->mapped_h, &ctx->mapped_d);
  if (rc != LK_OK) return rc;
  char* mh = (char*)ctx->mapped_h;
  char* md = (char*)ctx->mapped_d;
  ctx->cword_h = (lk_cword*)(mh + off_cw);
  ctx->rdone_h = (uint64_t*)(mh + off_rd);
  ctx->ctrl_h = (lk_ctrl*)(mh + off_ctrl);
  ctx->info_h = (lk_cta_info*)(mh + off_info);
  if (ctx->max_units) {
    ctx->units_h = (lk_unit*)(mh + off_units);
    ctx->units_d = (lk_unit*)(md + off_units);
  }
  if (ctx->qn) {
    ctx->q_units_h = (lk_qunit*)(mh + off_q);
    ctx->q_units_d = (lk_qunit*)(md + off_q);
    ctx->q_cq_h = (uint64_t*)(mh + off_cq);
    ctx->q_cq_d = (uint64_t*)(md + off_cq);
    ctx->q_close_h = (uint64_t*)(mh + off_close);
    ctx->q_close_d = (uint64_t*)(md + off_close);
  }
  if (ctx->mailbox) {
    ctx->mbox_h = (lk_mbox*)(mh + off_mbox);
    for (int c = 0; c < ctx->C; ++c) ctx->mbox_h[c].to_gpu = LK_CMD_NOP;   /* idle */
  }

  /* device block: [ring (finite only)] dcl[C] cl_start rd_off pin_smid boot_smid boot_count crit_active
   * log_count bcl chist log */
  size_t d_ring = 0;
  size_t d_dcl = live ? 0 : align_up(ring_bytes, LK_LINE);
  size_t d_start = align_up(d_dcl + ctx->C * sizeof(lk_dcluster), LK_LINE);
  size_t d_rdoff = align_up(d_start + (ctx->C + 1) * sizeof(int32_t), LK_LINE);
  size_t d_pin = align_up(d_rdoff + ctx->C * sizeof(int32_t), LK_LINE);
  size_t d_bsm = align_up(d_pin + (p->smids ? ctx->total : 0) * sizeof(int32_t), LK_LINE);
  size_t d_bcnt = align_up(d_bsm + ctx->G * sizeof(int32_t), LK_LINE);
  size_t d_crit = align_up(d_bcnt + sizeof(uint32_t), LK_LINE);
  size_t d_lcnt = align_up(d_crit + sizeof(int32_t), LK_LINE);
  size_t d_bcl = align_up(d_lcnt + ctx->G * sizeof(uint64_t), LK_LINE);
  size_t d_chist = align_up(d_bcl + ctx->C * sizeof(lk_bcluster), LK_LINE);
  size_t d_log = align_up(d_chist + (size_t)ctx->total * 256 * sizeof(uint32_t), LK_LINE);
  size_t dev_bytes = align_up(d_log + (size_t)ctx->G * ctx->log_cap * sizeof(lk_exec_rec), 4096);
  rc = lkb_alloc_device(ctx->device, dev_bytes, &ctx->dev_base);
  if (rc != LK_OK) return rc;
  char* db = (char*)ctx->dev_base;
  /* control state starts at zero; the log records need no clearing */
  rc = lkb_zero_device(ctx->device, db, d_log);
  if (rc != LK_OK) return rc;
  rc = lkb_copy_h2d(ctx->device, db + d_start, ctx->cl_start.data(), (ctx->C + 1) * sizeof(int32_t));
  if (rc == LK_OK) rc = lkb_copy_h2d(ctx->device, db + d_rdoff, ctx->rd_off.data(), ctx->C * sizeof(int32_t));
  if (rc == LK_OK && p->smids)
    rc = lkb_copy_h2d(ctx->device, db + d_pin, p->smids, ctx->total * sizeof(int32_t));
  if (rc != LK_OK) return rc;

  lk_kargs& a = ctx->args;
  memset(&a, 0, sizeof a);
  a.ring = (lk_wire*)(live ? (void*)(md + off_ring) : (void*)(db + d_ring));
  a.cword = (lk_cword*)(md + off_cw);
  a.rdone = (uint64_t*)(md + off_rd);
  a.rd_off = (int32_t*)(db + d_rdoff);
  a.mbox = ctx->mailbox ? (lk_mbox*)(md + off_mbox) : nullptr;
  a.ctrl = (lk_ctrl*)(md + off_ctrl);
  a.info = (lk_cta_info*)(md + off_info);
  a.dcl = (lk_dcluster*)(db + d_dcl);
  a.cl_start = (int32_t*)(db + d_start);
  a.pin_smid = p->smids ? (int32_t*)(db + d_pin) : nullptr;
  a.boot_smid = (int32_t*)(db + d_bsm);
  a.boot_count = (uint32_t*)(db + d_bcnt);
  a.log_count = (uint64_t*)(db + d_lcnt);
  a.log = ctx->log_cap ? (lk_exec_rec*)(db + d_log) : nullptr;
  a.bcl = (lk_bcluster*)(db + d_bcl);
  a.cta_hist = (uint32_t*)(db + d_chist);
  a.crit_active = (int32_t*)(db + d_crit);
  a.num_clusters = ctx->C;
  a.grid = ctx->G;
  a.total = ctx->total;
  a.ring_mask = R - 1;
  a.ring_log2 = ctx->R_log2;
  a.log_cap = ctx->log_cap;
  a.flags = ((p->flags & LK_INIT_DIRECT) ? LK_KFLAG_DIRECT : 0u) | (ctx->mailbox ? LK_KFLAG_MAILBOX : 0u);
  a.ctas_per_sm = ctx->per_sm;
  if (p->flags & LK_INIT_GEMM_FFMA) a.flags |= LK_KFLAG_GEMM_FFMA;
  if (!live) a.flags |= LK_KFLAG_FINITE;
  a.backoff_base_ns = p->backoff_base_ns;
  a.backoff_cap_ns = p->backoff_cap_ns ? p->backoff_cap_ns : 256;
  a.lease_ns = p->idle_lease_ns ? p->idle_lease_ns : 10000000000ull;
  a.boot_timeout_ns = p->boot_timeout_ns ? p->boot_timeout_ns : 10000000000ull;
  if (live) ctx->ring_h = (lk_wire*)(mh + off_ring);

  ctx->tail = new (std::nothrow) Tail[ctx->C];
  ctx->rearmed = new (std::nothrow) Tail[ctx->C];
  ctx->rate = new (std::nothrow) Tail[ctx->C];
  ctx->role = new (std::nothrow) Tail[ctx->C];
  ctx->batch = new (std::nothrow) lk_ctx::BatchState[ctx->C];
  if (!ctx->tail || !ctx->rearmed || !ctx->rate || !ctx->role || !ctx->batch) return LK_ENOMEM;
  return LK_OK;
}

static void teardown(lk_ctx* ctx) {
  if (ctx->launch) lkb_release(ctx->launch);
  if (ctx->dev_base) lkb_free_device(ctx->dev_base);
  if (ctx->mapped_h) lkb_free_mapped(ctx->mapped_h);
  delete[] ctx->tail;
  delete[] ctx->rearmed;
  delete[] ctx->rate;
  delete[] ctx->role;
  delete[] ctx->batch;
  delete ctx;
}

/* Wait for the kernel to return; on timeout set abort and wait again. */
static int join_kernel(lk_ctx* ctx, uint64_t timeout_ns) {
  uint64_t t0 = now_ns();
  for (;;) {
    int f = lkb_finished(ctx->launch);
    if (f < 0) return LK_EDEVICE;
    if (f == 1) return LK_OK;
    if (now_ns() - t0 > timeout_ns) break;
    std::this_thread::yield();
  }
  st_rel(&ctx->ctrl_h->abort, (uint64_t)1);
  t0 = now_ns();
  for (;;) {
    int f = lkb_finished(ctx->launch);
    if (f < 0) return LK_EDEVICE;
    if (f == 1) return LK_ETIMEDOUT;   /* returned, but only after the abort */
    if (now_ns() - t0 > timeout_ns + 2000000000ull) return LK_EBUSY;   /* still running */
    std::this_thread::yield();
  }
}

extern "C" {

int lk_init(lk_ctx** out, const lk_init_params* p) {
  if (!out || !p) return LK_EINVAL;
  *out = nullptr;
  lk_ctx* ctx = new (std::nothrow) lk_ctx();
  if (!ctx) return LK_ENOMEM;
  int rc = setup(ctx, p, true, 0);
  if (rc != LK_OK) { teardown(ctx); return rc; }
  beat(ctx);
  rc = lkb_launch_kernel(ctx->device, &ctx->args, ctx->T, &ctx->launch);
  if (rc != LK_OK) { ctx->launch = nullptr; teardown(ctx); return rc; }
  /* boot: every CTA read %smid, joined its cluster and counted itself */
  uint64_t t0 = now_ns();
  uint64_t limit = ctx->args.boot_timeout_ns + 1000000000ull;
  for (;;) {
    uint32_t b = ld_acq(&ctx->ctrl_h->booted);
    if (b >= (uint32_t)ctx->G) break;
    uint32_t e = dev_error(ctx);
    int f = lkb_finished(ctx->launch);
    if (e != 0 || f != 0 || now_ns() - t0 > limit) {
      int j = join_kernel(ctx, 0);
      if (j == LK_EBUSY) { *out = nullptr; return LK_ETIMEDOUT; }   /* leaked: kernel still up */
      teardown(ctx);
      return (f < 0) ? LK_EDEVICE : (e == LK_DERR_BOOT || e == 0 ? LK_ETIMEDOUT : LK_EDEVICE);
    }
    std::this_thread::yield();
  }
  ctx->running.store(1, std::memory_order_release);
  *out = ctx;
  return LK_OK;
}

int lk_submit(lk_ctx* ctx, int cluster, const lk_desc* d, const void* const* in, int n_in,
              void* out, lk_handle* h) {
  if (!ctx || !h || !d) return LK_EINVAL;
  if (cluster < 0 || cluster >= ctx->C) return LK_EINVAL;
  if (n_in < 0 || n_in > 2 || (n_in > 0 && !in)) return LK_EINVAL;
  const void* in0 = n_in > 0 ? in[0] : nullptr;
  const void* in1 = n_in > 1 ? in[1] : nullptr;
  int rc = validate(d, in0, in1, n_in, out);
  if (rc != LK_OK) return rc;
  if (!ctx_alive(ctx)) return LK_ESTATE;
  beat(ctx);
  uint64_t seq = 0;
  rc = post(ctx, cluster, LK_CMD_WORK + d->op, d, in0, in1, out, &seq);
  if (rc != LK_OK) return rc;
  *h = ((uint64_t)cluster << 48) | seq;
  return LK_OK;
}

static int poll_seq(lk_ctx* ctx, int c, uint64_t seq) {
  if (cl_done(ctx, c) >= seq) return LK_OK;
  uint32_t e = dev_error(ctx);
  if (e != 0) {
    /* the cluster may still have finished it before stopping */
    if (cl_done(ctx, c) >= seq) return LK_OK;
    return device_err_to_rc(e);
  }
  if (ld_acq(&ctx->ctrl_h->exited) != 0 || !ctx->running.load(std::memory_order_relaxed)) {
    if (cl_done(ctx, c) >= seq) return LK_OK;
    return LK_ESTATE;
  }
  return LK_PENDING;
}

static int decode(lk_ctx* ctx, lk_handle h, int* c, uint64_t* seq) {
  uint64_t cl = h >> 48;
  uint64_t s = h & kSeqMask;
  if (cl >= (uint64_t)ctx->C || s == 0) return LK_EINVAL;
  if (s > ctx->tail[cl].t.load(std::memory_order_acquire)) return LK_EINVAL;
  *c = (int)cl;
  *seq = s;
  return LK_OK;
}

int lk_poll(lk_ctx* ctx, lk_handle h) {
  if (!ctx) return LK_EINVAL;
  int c;
  uint64_t s;
  if (decode(ctx, h, &c, &s) != LK_OK) return LK_EINVAL;
  beat(ctx);
  return poll_seq(ctx, c, s);
}

int lk_set_rate(lk_ctx* ctx, int cluster, uint64_t bytes_per_us) {
  if (!ctx || cluster < 0 || cluster >= ctx->C) return LK_EINVAL;
  if (bytes_per_us >= (1ull << 40) || (bytes_per_us != 0 && bytes_per_us < LK_RATE_MIN)) return LK_EINVAL;
  ctx->rate[cluster].t.store(bytes_per_us, std::memory_order_relaxed);
  return LK_OK;
}

int lk_set_role(lk_ctx* ctx, int cluster, int role) {
  if (!ctx || cluster < 0 || cluster >= ctx->C) return LK_EINVAL;
  if (role != LK_ROLE_NONE && role != LK_ROLE_CRITICAL && role != LK_ROLE_YIELD) return LK_EINVAL;
  ctx->role[cluster].t.store((uint64_t)role, std::memory_order_relaxed);
  return LK_OK;
}

int lk_heartbeat(lk_ctx* ctx) {
  if (!ctx) return LK_EINVAL;
  beat(ctx);
  return LK_OK;
}

int lk_wait(lk_ctx* ctx, lk_handle h, uint64_t timeout_ns) {
  if (!ctx) return LK_EINVAL;
  int c;
  uint64_t s;
  if (decode(ctx, h, &c, &s) != LK_OK) return LK_EINVAL;
  if (cl_done(ctx, c) >= s) return LK_OK;
  beat(ctx);
  uint64_t t0 = now_ns();
  uint64_t last_beat = t0;
  for (uint32_t i = 0;; ++i) {
    if (cl_done(ctx, c) >= s) return LK_OK;
    if ((i & 255) == 255) {
      int rc = poll_seq(ctx, c, s);
      if (rc != LK_PENDING) return rc;
      uint64_t t = now_ns();
      if (t - t0 > timeout_ns) return LK_ETIMEDOUT;
      if (t - last_beat > 1000000ull) { beat(ctx); last_beat = t; }
    }
  }
}

int lk_sync(lk_ctx* ctx, uint64_t timeout_ns) {
  if (!ctx) return LK_EINVAL;
  uint64_t t0 = now_ns();
  for (int c = 0; c < ctx->C; ++c) {
    uint64_t s = ctx->tail[c].t.load(std::memory_order_acquire);
    if (s == 0) continue;
    uint64_t spent = now_ns() - t0;
    int rc = lk_wait(ctx, ((uint64_t)c << 48) | s, spent >= timeout_ns ? 0 : timeout_ns - spent);
    if (rc != LK_OK) return rc;
  }
  return LK_OK;
}

int lk_dispose(lk_ctx* ctx, uint64_t timeout_ns) { return lk_dispose_timed(ctx, timeout_ns, nullptr); }

int lk_dispose_timed(lk_ctx* ctx, uint64_t timeout_ns, float* kernel_ms) {
  if (kernel_ms) *kernel_ms = -1.f;
  if (!ctx) return LK_EINVAL;
  uint64_t t0 = now_ns();
  if (ctx->launch && ctx_alive(ctx)) {
    beat(ctx);
    for (int c = 0; c < ctx->C; ++c) {
      uint64_t seq;
      for (;;) {
        int rc = post(ctx, c, LK_CMD_EXIT, nullptr, nullptr, nullptr, nullptr, &seq);
        if (rc == LK_OK) break;
        if (!ctx_alive(ctx) || now_ns() - t0 > timeout_ns) break;
        std::this_thread::yield();
      }
    }
  }
  ctx->running.store(0, std::memory_order_release);
  int rc = LK_OK;
  if (ctx->launch) {
    uint64_t spent = now_ns() - t0;
    rc = join_kernel(ctx, spent >= timeout_ns ? 0 : timeout_ns - spent);
    if (rc == LK_EBUSY) return LK_EBUSY;   /* kernel still running: keep everything */
    if (kernel_ms) *kernel_ms = lkb_elapsed_ms(ctx->launch);
  }
  uint32_t e = dev_error(ctx);
  teardown(ctx);
  if (rc != LK_OK) return rc;
  if (e != 0 && e != LK_DERR_LEASE) return LK_EDEVICE;
  return LK_OK;
}

/* Input bytes of one item: what the split rule divides. */
static uint64_t item_input_bytes(uint32_t op, uint64_t n) {
  switch (op) {
    case LK_OP_ADD_I32: return 8 * n;
    case LK_OP_COPY_I32: return 4 * n;
    case LK_OP_SUM_F32: return 4 * n;
    case LK_OP_HIST_U8: return n;
    case LK_OP_GEMM64_F32: return 32768 * n;
    default: return 0;
  }
}

int lk_submit_batch(lk_ctx* ctx, int cluster, const lk_batch_item* items, uint32_t count,
                    const lk_batch_tune* tune, lk_handle* h) {
  if (!ctx || !h || (count > 0 && !items) || cluster < 0 || cluster >= ctx->C) return LK_EINVAL;
  if (!ctx->max_units) return LK_EINVAL;   /* finite-mode contexts take no batches */
  uint32_t cap = tune && tune->max_parts ? tune->max_parts : 8u;
  const uint64_t part_bytes = tune && tune->part_bytes ? tune->part_bytes : (4ull << 20);
  if (cap > 8) return LK_EINVAL;
  cap = std::min<uint32_t>(cap, (uint32_t)ctx->sizes[cluster]);
  /* validate and count units, split sums and split histograms */
  uint64_t units = 0;
  uint32_t sums = 0, hists = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const lk_batch_item& it = items[i];
    lk_desc d{it.op, 0, it.n, 0};
    int rc = validate(&d, it.in0, it.in1, op_inputs(it.op), it.out);
    if (rc != LK_OK) return rc;
    if (it.parts > 8) return LK_EINVAL;
    uint32_t parts = it.parts ? std::min(it.parts, cap)
                              : (uint32_t)std::min<uint64_t>(cap, std::max<uint64_t>(1, (item_input_bytes(it.op, it.n) + part_bytes - 1) / part_bytes));
    if (parts > 1 && it.op == LK_OP_SUM_F32) ++sums;
    if (parts > 1 && it.op == LK_OP_HIST_U8) ++hists;
    units += parts;
  }
  if (units > ctx->max_units || sums > LK_BATCH_SPLIT_SUMS || hists > LK_BATCH_SPLIT_HISTS) return LK_EINVAL;
  if (!ctx_alive(ctx)) return LK_ESTATE;
  beat(ctx);
  lk_ctx::BatchState& bs = ctx->batch[cluster];
  std::lock_guard<std::mutex> g(bs.mu);
  const uint32_t b = (uint32_t)(bs.next % LK_BATCH_BUFFERS);
  if (cl_done(ctx, cluster) < bs.seq_of[b]) return LK_EAGAIN;   /* table still in use */
  lk_unit* tab = ctx->units_h + ((size_t)cluster * LK_BATCH_BUFFERS + b) * ctx->max_units;
  uint64_t u = 0;
  uint32_t s_slot = 0, h_slot = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const lk_batch_item& it = items[i];
    uint32_t parts = it.parts ? std::min(it.parts, cap)
                              : (uint32_t)std::min<uint64_t>(cap, std::max<uint64_t>(1, (item_input_bytes(it.op, it.n) + part_bytes - 1) / part_bytes));
    uint64_t comb = 0;
    if (parts > 1 && it.op == LK_OP_SUM_F32) comb = ++s_slot;
    if (parts > 1 && it.op == LK_OP_HIST_U8) comb = ++h_slot;
    for (uint32_t p = 0; p < parts; ++p, ++u) {
      lk_unit& un = tab[u];
      un.in0 = (uint64_t)(uintptr_t)it.in0;
      un.in1 = (uint64_t)(uintptr_t)it.in1;
      un.out = (uint64_t)(uintptr_t)it.out;
      un.n_op = ((uint64_t)it.op << 56) | (it.n & LK_LOW48);
      un.meta = (uint64_t)p | ((uint64_t)parts << 8) | (comb << 16);
      un.item = i;
    }
  }
  /* the unit table is read by the device after it acquires the descriptor,
   * which write_slot publishes behind a release fence */
  lk_desc d{LK_OP_BATCH, 0, units, 0};
  uint64_t seq = 0;
  int rc = post(ctx, cluster, LK_CMD_WORK + LK_OP_BATCH, &d, ctx->units_d + (tab - ctx->units_h), nullptr, nullptr,
                &seq);
  if (rc != LK_OK) return rc;
  bs.seq_of[b] = seq;
  bs.next++;
  *h = ((uint64_t)cluster << 48) | seq;
  return LK_OK;
}

int lk_phase_run(int device, int sms, int threads, uint64_t iters, int runs, void* out_dev, lk_phase_times* out) {
  if (sms < 1 || runs < 1 || !out || iters > 0xffffffffull) return LK_EINVAL;
  for (int r = 0; r < runs; ++r) {
    lk_init_params p;
    memset(&p, 0, sizeof p);
    p.device = device;
    p.num_clusters = 1;
    p.sms_per_cluster = &sms;
    p.threads_per_cta = threads;
    p.ring_depth = 64;
    p.max_batch_units = 16;
    lk_ctx* ctx = nullptr;
    const uint64_t t0 = now_ns();
    int rc = lk_init(&ctx, &p);
    const uint64_t t1 = now_ns();
    if (rc != LK_OK) return rc;
    lk_desc d{LK_OP_SPIN, 0, iters, 0};
    lk_handle h = 0;
    rc = lk_submit(ctx, 0, &d, nullptr, 0, r == runs - 1 ? out_dev : nullptr, &h);
    const uint64_t t2 = now_ns();
    if (rc == LK_OK) rc = lk_wait(ctx, h, 60000000000ull);
    const uint64_t t3 = now_ns();
    int rd = lk_dispose(ctx, 30000000000ull);
    const uint64_t t4 = now_ns();
    if (rc != LK_OK) return rc;
    if (rd != LK_OK) return rd;
    out[r] = lk_phase_times{t1 - t0, t2 - t1, t3 - t2, t4 - t3};
  }
  return LK_OK;
}

int lk_cluster_info(lk_ctx* ctx, int cluster, int* smids, int cap) {
  if (!ctx || cluster < 0 || cluster >= ctx->C || cap < 0 || (cap > 0 && !smids)) return LK_EINVAL;
  int size = ctx->sizes[cluster];
  for (int g = 0; g < ctx->G; ++g) {
    lk_cta_info inf = ctx->info_h[g];
    if (inf.cluster == cluster && inf.rank >= 0 && inf.rank < size && inf.rank < cap) smids[inf.rank] = inf.smid;
  }
  return size;
}

int lk_status(lk_ctx* ctx, int cluster) {
  if (!ctx || cluster < 0 || cluster >= ctx->C) return LK_EINVAL;
  /* the device writes the status word only at boot and at exit; in between
   * Table 1's WORKING / FINISHED follow from the ring counters, which saves
   * the device two system-scope stores per descriptor */
  const uint64_t st = ld_acq(&ctx->cword_h[cluster].status);
  if (st == LK_ST_EXITED || st == LK_ST_ERROR || ctx->mailbox) return (int)st;
  const uint64_t tail = ctx->tail[cluster].t.load(std::memory_order_acquire);
  if (tail == 0) return LK_ST_INIT;
  return cl_done(ctx, cluster) >= tail ? LK_ST_FINISHED : LK_ST_WORKING;
}

int lk_device_error(lk_ctx* ctx) {
  if (!ctx) return LK_EINVAL;
  return (int)dev_error(ctx);
}

int lk_num_sms(lk_ctx* ctx) { return ctx ? ctx->sm_count : LK_EINVAL; }
int lk_num_ctas(lk_ctx* ctx) { return ctx ? ctx->total : LK_EINVAL; }

/* Gather the per-CTA logs (device memory) into caller order. */
static int read_log(lk_ctx* ctx, lk_exec_rec* buf, size_t cap, size_t* n, uint64_t* dropped) {
  *n = 0;
  if (dropped) *dropped = 0;
  if (!ctx->log_cap || !ctx->args.log) return LK_OK;
  std::vector<uint64_t> counts(ctx->G);
  int rc = lkb_copy_d2h(ctx->device, counts.data(), ctx->args.log_count, ctx->G * sizeof(uint64_t));
  if (rc != LK_OK) return rc;
  std::vector<lk_exec_rec> tmp((size_t)ctx->log_cap);
  uint64_t drop = 0;
  size_t w = 0;
  for (int g = 0; g < ctx->G; ++g) {
    uint64_t cnt = counts[g];
    if (cnt == 0) continue;
    uint64_t keep = cnt < ctx->log_cap ? cnt : ctx->log_cap;
    drop += cnt - keep;
    rc = lkb_copy_d2h(ctx->device, tmp.data(), ctx->args.log + (size_t)g * ctx->log_cap,
                      (size_t)ctx->log_cap * sizeof(lk_exec_rec));
    if (rc != LK_OK) return rc;
    uint64_t first = cnt - keep;
    for (uint64_t k = first; k < cnt && w < cap; ++k) buf[w++] = tmp[k % ctx->log_cap];
  }
  *n = w;
  if (dropped) *dropped = drop;
  return LK_OK;
}

int lk_exec_log(lk_ctx* ctx, lk_exec_rec* buf, size_t cap, size_t* n, uint64_t* dropped) {
  if (!ctx || !n || (cap > 0 && !buf)) return LK_EINVAL;
  return read_log(ctx, buf, cap, n, dropped);
}

const char* lk_strerror(int code) {
  switch (code) {
    case LK_OK: return "LK_OK";
    case LK_PENDING: return "LK_PENDING";
    case LK_EINVAL: return "LK_EINVAL: invalid argument";
    case LK_EAGAIN: return "LK_EAGAIN: cluster mailbox ring full";
    case LK_ETIMEDOUT: return "LK_ETIMEDOUT: deadline passed";
    case LK_EDEVICE: return "LK_EDEVICE: device-side or CUDA error";
    case LK_ESTATE: return "LK_ESTATE: context not running";
    case LK_ENOMEM: return "LK_ENOMEM: allocation failed";
    case LK_EBUSY: return "LK_EBUSY: kernel still running; context kept";
    default: return "LK_?: unknown code";
  }
}

/* ---------------------------------------------------------------------- */
int lk_run_finite(const lk_init_params* p, const lk_desc* descs, const int* cluster_of,
                  const void* const* in0, const void* const* in1, void* const* out, size_t count,
                  float* elapsed_ms, lk_exec_rec* log_out, size_t log_cap, size_t* log_n) {
  if (!p || (count > 0 && (!descs || !cluster_of))) return LK_EINVAL;
  if (log_n) *log_n = 0;
  std::vector<uint64_t> per(p->num_clusters > 0 ? p->num_clusters : 1, 0);
  for (size_t i = 0; i < count; ++i) {
    if (cluster_of[i] < 0 || cluster_of[i] >= p->num_clusters) return LK_EINVAL;
    const lk_desc* d = &descs[i];
    int rc = validate(d, in0 ? in0[i] : nullptr, in1 ? in1[i] : nullptr, op_inputs(d->op),
                      out ? out[i] : nullptr);
    if (rc != LK_OK) return rc;
    per[cluster_of[i]]++;
  }
  uint64_t mx = 0;
  for (uint64_t v : per) mx = std::max(mx, v);
  uint32_t R = 2;
  while (R < mx + 1) R <<= 1;
  lk_ctx* ctx = new (std::nothrow) lk_ctx();
  if (!ctx) return LK_ENOMEM;
  ctx->finite = true;
  int rc = setup(ctx, p, false, R);
  if (rc != LK_OK) { teardown(ctx); return rc; }
  /* fill the ring on the host, then copy it into device memory */
  std::vector<lk_wire> ring((size_t)ctx->C * R);
  memset(ring.data(), 0, ring.size() * sizeof(lk_wire));
  std::vector<uint64_t> t(ctx->C, 0);
  for (size_t i = 0; i < count; ++i) {
    int c = cluster_of[i];
    write_slot(&ring[(size_t)c * R + t[c]], t[c], ctx->R_log2, LK_CMD_WORK + descs[i].op, &descs[i],
               in0 ? in0[i] : nullptr, in1 ? in1[i] : nullptr, out ? out[i] : nullptr);
    ++t[c];
  }
  for (int c = 0; c < ctx->C; ++c) {
    write_slot(&ring[(size_t)c * R + t[c]], t[c], ctx->R_log2, LK_CMD_EXIT, nullptr, nullptr, nullptr, nullptr);
    ++t[c];
  }
  rc = lkb_copy_h2d(ctx->device, ctx->args.ring, ring.data(), ring.size() * sizeof(lk_wire));
  if (rc != LK_OK) { teardown(ctx); return rc; }
  beat(ctx);
  rc = lkb_launch_kernel(ctx->device, &ctx->args, ctx->T, &ctx->launch);
  if (rc != LK_OK) { ctx->launch = nullptr; teardown(ctx); return rc; }
  /* bounded: the lease ends an idle kernel; the abort ends a stuck one */
  uint64_t limit = ctx->args.lease_ns + ctx->args.boot_timeout_ns;
  rc = join_kernel(ctx, limit);
  if (rc == LK_EBUSY) return LK_ETIMEDOUT;   /* leaked: kernel still up */
  if (rc == LK_OK && elapsed_ms) *elapsed_ms = lkb_elapsed_ms(ctx->launch);
  if (rc == LK_OK && log_out && log_n) rc = read_log(ctx, log_out, log_cap, log_n, nullptr);
  uint32_t e = dev_error(ctx);
  teardown(ctx);
  if (rc != LK_OK) return rc;
  return e ? LK_EDEVICE : LK_OK;
}

/* ---------------------------------------------------------------------- */
static void pin_to(int cpu) {
#ifdef __linux__
  if (cpu < 0) return;
  int n = (int)std::thread::hardware_concurrency();
  if (n <= 0) return;
  cpu_set_t set;
  CPU_ZERO(&set);
  CPU_SET(cpu % n, &set);
  pthread_setaffinity_np(pthread_self(), sizeof set, &set);
#else
  (void)cpu;
#endif
}

int lk_run_trace(lk_ctx* ctx, const lk_trace_item* items, size_t count, int n_threads,
                 int mode, int pin_cpu_base, uint64_t timeout_ns, lk_trace_result* res) {
  if (!ctx || (count > 0 && (!items || !res)) || n_threads < 1 || n_threads > 256) return LK_EINVAL;
  if (mode < LK_TRACE_OPEN || mode > LK_TRACE_E2E) return LK_EINVAL;
  const bool closed_loop = mode != LK_TRACE_OPEN;
  const bool e2e = mode == LK_TRACE_E2E;
  for (size_t i = 0; i < count; ++i) {
    const lk_trace_item& it = items[i];
    if (it.cluster < 0 || it.cluster >= ctx->C) return LK_EINVAL;
    lk_desc d{it.op, 0, it.n, 0};
    int rc = validate(&d, it.in0, it.in1, op_inputs(it.op), it.out);
    if (rc != LK_OK) return rc;
    res[i] = lk_trace_result{0, 0, LK_PENDING, -1, 0, 0};
  }
  if (!ctx_alive(ctx)) return LK_ESTATE;
  /* per thread: its items in arrival order */
  std::vector<std::vector<size_t>> mine(n_threads);
  for (size_t i = 0; i < count; ++i) mine[items[i].cluster % n_threads].push_back(i);
  for (auto& v : mine)
    std::stable_sort(v.begin(), v.end(), [&](size_t a, size_t b) { return items[a].t_arrival_ns < items[b].t_arrival_ns; });
  std::atomic<int> ready{0};
  std::atomic<uint64_t> start{0};
  std::atomic<int> first_err{0};

  auto worker = [&](int w) {
    pin_to(pin_cpu_base >= 0 ? pin_cpu_base + w : -1);
    const std::vector<size_t>& v = mine[w];
    void* stream = nullptr;
    if (e2e && lkb_stream_create(ctx->device, &stream) != LK_OK) stream = nullptr;
    ready.fetch_add(1);
    uint64_t t0;
    while ((t0 = start.load(std::memory_order_acquire)) == 0) {}
    uint64_t deadline = t0 + timeout_ns;
    /* pending handles in submission order per cluster (completion is FIFO per cluster) */
    std::vector<std::vector<std::pair<uint64_t, size_t>>> pend(ctx->C);
    /* no allocation inside the timed loop: room for every item up front */
    {
      std::vector<size_t> per_cluster(ctx->C, 0);
      for (size_t k = 0; k < v.size(); ++k) per_cluster[items[v[k]].cluster]++;
      for (int c = 0; c < ctx->C; ++c) pend[c].reserve(per_cluster[c]);
    }
    std::vector<size_t> head(ctx->C, 0);
    size_t next = 0, finished = 0;
    while (finished < v.size()) {
      uint64_t now = now_ns();
      if (now > deadline) {
        for (size_t k = 0; k < v.size(); ++k)
          if (res[v[k]].status == LK_PENDING) res[v[k]].status = LK_ETIMEDOUT;
        int z = 0;
        first_err.compare_exchange_strong(z, LK_ETIMEDOUT);
        if (stream) lkb_stream_destroy(stream);
        return;
      }
      bool can_release = next < v.size() && now >= t0 + items[v[next]].t_arrival_ns &&
                         (!closed_loop || finished == next);
      if (can_release) {
        const lk_trace_item& it = items[v[next]];
        lk_desc d{it.op, 0, it.n, 0};
        uint64_t ts = now_ns();
        uint64_t seq = 0;
        int rc = LK_OK;
        if (e2e) {
          /* Copyin (Sec. III): inputs from pinned host memory, on this thread's stream */
          if (!stream) rc = LK_EDEVICE;
          if (rc == LK_OK && it.in0_bytes && it.h_in0)
            rc = lkb_memcpy_async(stream, (void*)it.in0, it.h_in0, it.in0_bytes, 1);
          if (rc == LK_OK && it.in1_bytes && it.h_in1)
            rc = lkb_memcpy_async(stream, (void*)it.in1, it.h_in1, it.in1_bytes, 1);
          if (rc == LK_OK) rc = lkb_stream_sync(stream);
        }
        if (rc == LK_OK) rc = post(ctx, it.cluster, LK_CMD_WORK + it.op, &d, it.in0, it.in1, it.out, &seq);
        while (rc == LK_EAGAIN && e2e) rc = post(ctx, it.cluster, LK_CMD_WORK + it.op, &d, it.in0, it.in1, it.out, &seq);
        if (rc == LK_OK) {
          res[v[next]].t_submit_ns = ts - t0;
          res[v[next]].t_post_ns = now_ns() - t0;
          res[v[next]].thread = w;
          pend[it.cluster].push_back({seq, v[next]});
          ++next;
        } else if (rc != LK_EAGAIN) {
          res[v[next]].status = rc;
          ++next;
          ++finished;
        }
      }
      /* completions */
      for (int c = w; c < ctx->C; c += n_threads) {
        auto& pq = pend[c];
        if (head[c] == pq.size()) continue;
        uint64_t done = cl_done(ctx, c);
        if (done < pq[head[c]].first) {
          if (dev_error(ctx) != 0 || ld_acq(&ctx->ctrl_h->exited) != 0) {
            int rc = device_err_to_rc(dev_error(ctx));
            if (rc == LK_OK) rc = LK_ESTATE;
            for (size_t k = head[c]; k < pq.size(); ++k) res[pq[k].second].status = rc;
            finished += pq.size() - head[c];
            head[c] = pq.size();
            int z = 0;
            first_err.compare_exchange_strong(z, rc);
          }
          continue;
        }
        uint64_t tc = now_ns() - t0;
        while (head[c] < pq.size() && pq[head[c]].first <= done) {
          const size_t idx = pq[head[c]].second;
          int st = LK_OK;
          res[idx].t_observed_ns = tc;
          if (e2e && items[idx].out_bytes && items[idx].h_out) {
            /* Copyout (Sec. III) */
            st = lkb_memcpy_async(stream, items[idx].h_out, items[idx].out, items[idx].out_bytes, 0);
            if (st == LK_OK) st = lkb_stream_sync(stream);
            tc = now_ns() - t0;
          }
          res[idx].t_complete_ns = tc;
          res[idx].status = st;
          ++head[c];
          ++finished;
        }
      }
      if ((next & 1023) == 0) beat(ctx);
    }
    if (stream) lkb_stream_destroy(stream);
  };
  std::vector<std::thread> th;
  for (int w = 0; w < n_threads; ++w) th.emplace_back(worker, w);
  while (ready.load() < n_threads) std::this_thread::yield();
  start.store(now_ns(), std::memory_order_release);
  for (auto& x : th) x.join();
  beat(ctx);
  int e = first_err.load();
  for (size_t i = 0; i < count && e == 0; ++i)
    if (res[i].status != LK_OK) e = res[i].status;
  return e;
}

}  // extern "C"

/* ---------------------------------------------------------------------- */
/* Serving: producers inject requests, one dispatcher admits, chunks and
 * completes them.                                                          */
namespace {

/* First-fit allocator over [0, size) with coalescing of freed blocks. */
class Arena {
 public:
  explicit Arena(uint64_t size) { if (size) free_[0] = size; }
  bool alloc(uint64_t bytes, uint64_t* off) {
    bytes = (bytes + 255) & ~255ull;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const uint64_t rest = it->second - bytes;
        const uint64_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = (bytes + 255) & ~255ull;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<uint64_t, uint64_t> free_;
};

struct ServeReq {
  uint64_t in_bytes = 0, out_bytes = 0, scratch_bytes = 0, held = 0;
  uint64_t unit = 1;          /* elements per alignment unit */
  uint64_t elem_bytes = 4;    /* input bytes per element (per input) */
  uint32_t chunks = 1, done_chunks = 0;
  bool needs_combine = false, arena_out = false;
  bool coalesced = false;     /* runs as one item of a batch post */
  uint64_t out_off = 0, scratch_off = 0;
  void* out = nullptr;
  void* scratch = nullptr;
};

}  // namespace

static uint64_t queue_state_bytes(uint32_t nslots) {
  return align_up(sizeof(lk_qstate), 256) + align_up((uint64_t)nslots * sizeof(lk_qslot), 256);
}

/* The queue's split rule (see lk.h, lk_serve_parts): units of a request of
 * op over n elements, given the context's CTAs and the backlog of admitted
 * units no CTA has claimed yet (count and input bytes). */
static uint32_t split_parts(uint32_t op, uint64_t n, uint64_t ctas, uint64_t backlog_units, uint64_t backlog_bytes,
                            uint64_t part_bytes, uint64_t min_part) {
  const uint64_t B = item_input_bytes(op, n);
  const uint64_t fine_part = std::max<uint64_t>(min_part, part_bytes / 8);
  auto ceil_parts = [&](uint64_t unit) {
    return std::min<uint64_t>(std::max<uint64_t>(1, (B + unit - 1) / unit), LK_SERVE_MAX_PARTS);
  };
  const uint64_t base = ceil_parts(part_bytes);
  uint64_t fine = ceil_parts(fine_part);
  uint64_t wide = std::min<uint64_t>((B + min_part - 1) / min_part, LK_SERVE_MAX_PARTS);
  if (op == LK_OP_GEMM64_F32) {   /* whole tiles */
    fine = std::min<uint64_t>(fine, n);
    wide = std::min<uint64_t>(wide, n);
  }
  /* a sum's float result depends on its split: a function of B and the CTAs alone */
  if (op == LK_OP_SUM_F32) return (uint32_t)std::max(base, std::min(ctas, wide));
  const uint64_t floor_parts = backlog_bytes >= ctas * part_bytes ? base : fine;   /* saturated? */
  const uint64_t idle = backlog_units < ctas ? ctas - backlog_units : 0;
  return (uint32_t)std::max(floor_parts, std::min(idle, wide));
}

extern "C" uint32_t lk_serve_parts(uint32_t op, uint64_t n, uint32_t ctas, uint64_t backlog_units,
                                   uint64_t backlog_bytes, uint64_t part_bytes, uint64_t min_part_bytes) {
  if (op < LK_OP_ADD_I32 || op > LK_OP_COPY_I32 || ctas == 0) return 0;
  const uint64_t part = part_bytes ? part_bytes : (8ull << 20);
  const uint64_t min_part = min_part_bytes ? min_part_bytes : (128ull << 10);
  if (min_part < 65536 || part < min_part || part > (1ull << 40)) return 0;
  return split_parts(op, n, ctas, backlog_units, backlog_bytes, part, min_part);
}

extern "C" uint64_t lk_serve_queue_state_bytes(uint32_t max_inflight) {
  return queue_state_bytes(max_inflight ? max_inflight : 4096u);
}

/* lk_serve, LK_SERVE_QUEUE: the device-resident queue (see lk.h).  The
 * host admits requests, publishes their units round-robin into the
 * host-mapped unit ring (lap-tagged words, as lk_qunit describes) while
 * fewer than `window` x CTAs published units are unclaimed, and retires
 * requests from the completion ring.  Units are claimed in index order, so
 * the claimed count is tracked by walking the entries' acknowledgements in
 * order; unit indices stay below 2^32 per call. */
static int serve_queue(lk_ctx* ctx, const lk_request* reqs, size_t count, const lk_serve_params* p,
                       lk_request_result* res) {
  if (!ctx->qn || ctx->mailbox) return LK_EINVAL;   /* live ring-mode contexts only */
  const uint32_t nslots = p->max_inflight ? p->max_inflight : 4096u;
  const uint64_t part_bytes = p->part_bytes ? p->part_bytes : (8ull << 20);
  const uint64_t min_part = p->min_part_bytes ? p->min_part_bytes : (128ull << 10);
  const uint64_t timeout = p->timeout_ns ? p->timeout_ns : 120000000000ull;
  const int window = p->window > 0 ? p->window : 2;
  const uint64_t W = std::min<uint64_t>((uint64_t)window * (uint64_t)ctx->total, ctx->qn / 2);
  if (nslots > ctx->qn || min_part < 65536 || part_bytes < min_part || part_bytes > (1ull << 40) ||
      ((uintptr_t)p->arena & 255u) || !p->arena)
    return LK_EINVAL;
  const uint64_t sbytes = queue_state_bytes(nslots);
  if (p->arena_bytes < sbytes) return LK_ENOMEM;
  struct QReq {
    uint64_t in_bytes = 0, out_bytes = 0, held = 0, out_off = 0;
    uint32_t parts = 1, published = 0, slot = 0;
    bool arena_out = false;
    void* out = nullptr;
  };
  std::vector<QReq> st(count);
  for (size_t i = 0; i < count; ++i) {
    const lk_request& r = reqs[i];
    if (r.producer >= (uint32_t)p->n_producers) return LK_EINVAL;
    if (r.op < LK_OP_ADD_I32 || r.op > LK_OP_COPY_I32) return LK_EINVAL;
    lk_desc d{r.op, 0, r.n, 0};
    int rc = validate(&d, r.in0, r.in1, op_inputs(r.op), r.out ? r.out : (void*)(uintptr_t)256);
    if (rc != LK_OK) return rc;
    QReq& q = st[i];
    q.in_bytes = item_input_bytes(r.op, r.n);
    q.out_bytes = r.op == LK_OP_ADD_I32 || r.op == LK_OP_COPY_I32 ? 4 * r.n
                  : r.op == LK_OP_SUM_F32                        ? 16
                  : r.op == LK_OP_HIST_U8                        ? 1024
                                                                 : 16384 * r.n;
    /* a sum's unit count is fixed now; other ops are split at admission */
    q.parts = split_parts(r.op, r.n, (uint64_t)ctx->total, 0, 0, part_bytes, min_part);
    q.arena_out = r.out == nullptr;
    q.held = q.in_bytes + q.out_bytes;
    if (q.held > p->budget_bytes || (q.arena_out && q.out_bytes + 256 > p->arena_bytes - sbytes)) return LK_ENOMEM;
    res[i] = lk_request_result{0, 0, nullptr, LK_PENDING, q.parts};
  }
  if (!ctx_alive(ctx)) return LK_ESTATE;

  /* device state at the start of the arena: zeroed (copy engine), then the
   * header the serving CTAs read; the host-mapped rings start empty */
  int rc = lkb_zero_device(ctx->device, p->arena, sbytes);
  lk_qstate hdr;
  memset(&hdr, 0, sizeof hdr);
  hdr.units = ctx->q_units_d;
  hdr.cq = ctx->q_cq_d;
  hdr.close = ctx->q_close_d;
  hdr.slots = (lk_qslot*)((char*)p->arena + align_up(sizeof(lk_qstate), 256));
  hdr.qmask = ctx->qn - 1;
  hdr.qlog2 = ctx->qlog2;
  hdr.nslots = nslots;
  if (rc == LK_OK) rc = lkb_copy_h2d(ctx->device, p->arena, &hdr, sizeof hdr);
  if (rc != LK_OK) return rc;
  memset(ctx->q_units_h, 0, (size_t)ctx->qn * sizeof(lk_qunit));
  memset(ctx->q_cq_h, 0, (size_t)ctx->qn * sizeof(uint64_t));
  st_rel(ctx->q_close_h, (uint64_t)0);
  beat(ctx);
  /* one LK_OP_SERVE per cluster: every CTA becomes a worker of the queue */
  std::vector<uint64_t> serve_seq(ctx->C, 0);
  for (int c = 0; c < ctx->C; ++c) {
    const lk_desc d{LK_OP_SERVE, 0, 0, 0};
    const uint64_t t0 = now_ns();
    for (;;) {
      rc = post(ctx, c, LK_CMD_WORK + LK_OP_SERVE, &d, p->arena, nullptr, nullptr, &serve_seq[c]);
      if (rc != LK_EAGAIN) break;
      if (!ctx_alive(ctx) || now_ns() - t0 > timeout) break;
      std::this_thread::yield();
    }
    if (rc != LK_OK) {
      /* the clusters that did get the descriptor leave at once when the queue closes */
      st_rel(ctx->q_close_h, (1ull << 63));
      for (int b = 0; b < c; ++b) lk_wait(ctx, ((uint64_t)b << 48) | serve_seq[b], 10000000000ull);
      return rc == LK_EAGAIN ? LK_ETIMEDOUT : rc;
    }
  }

  /* producers: each releases its own requests at their arrival times */
  std::mutex qmu;
  std::deque<size_t> arrived;
  std::atomic<uint64_t> start{0};
  std::atomic<int> ready{0};
  std::atomic<bool> stop{false};
  std::vector<std::vector<size_t>> mine(p->n_producers);
  for (size_t i = 0; i < count; ++i) mine[reqs[i].producer].push_back(i);
  for (auto& v : mine)
    std::stable_sort(v.begin(), v.end(), [&](size_t a, size_t b) { return reqs[a].t_arrival_ns < reqs[b].t_arrival_ns; });
  auto producer = [&](int w) {
    ready.fetch_add(1);
    uint64_t t0;
    while ((t0 = start.load(std::memory_order_acquire)) == 0) {}
    for (size_t i : mine[w]) {
      while (now_ns() < t0 + reqs[i].t_arrival_ns)
        if (stop.load(std::memory_order_relaxed)) return;
      std::lock_guard<std::mutex> g(qmu);
      arrived.push_back(i);
    }
  };
  std::vector<std::thread> th;
  for (int w = 0; w < p->n_producers; ++w) th.emplace_back(producer, w);
  while (ready.load() < p->n_producers) std::this_thread::yield();
  const uint64_t t0 = now_ns();
  start.store(t0, std::memory_order_release);

  Arena arena(p->arena_bytes - sbytes);
  std::vector<uint32_t> free_slots(nslots);
  for (uint32_t k = 0; k < nslots; ++k) free_slots[k] = nslots - 1 - k;
  std::vector<size_t> slot_req(nslots, 0);
  std::deque<size_t> waiting;    /* arrived, not admitted (FIFO) */
  std::deque<size_t> active;     /* admitted with units left to publish (round-robin) */
  uint64_t held = 0, next_u = 0, acked = 0, cq_head = 0, last_beat = t0;
  uint64_t unpublished = 0;         /* units of admitted requests not yet published */
  uint64_t unpublished_bytes = 0;   /* and their input bytes */
  uint64_t pub_bytes = 0;           /* input bytes of every published unit */
  /* input bytes published through unit u, at u mod qn: the bytes of the
   * published units no CTA has claimed yet are cum(next_u) - cum(acked) */
  std::vector<uint64_t> cum(ctx->qn, 0);
  size_t finished = 0;
  int first_err = LK_OK;
  char* const out_base = (char*)p->arena + sbytes;
  while (finished < count) {
    const uint64_t now = now_ns();
    if (now - t0 > timeout) {
      for (size_t i = 0; i < count; ++i)
        if (res[i].status == LK_PENDING) res[i].status = LK_ETIMEDOUT;
      first_err = LK_ETIMEDOUT;
      break;
    }
    if (!ctx_alive(ctx)) {
      int e = device_err_to_rc(dev_error(ctx));
      for (size_t i = 0; i < count; ++i)
        if (res[i].status == LK_PENDING) res[i].status = e ? e : LK_ESTATE;
      first_err = e ? e : LK_ESTATE;
      break;
    }
    if (now - last_beat > 1000000ull) {
      beat(ctx);
      last_beat = now;
    }
    {
      std::lock_guard<std::mutex> g(qmu);
      while (!arrived.empty()) {
        waiting.push_back(arrived.front());
        arrived.pop_front();
      }
    }
    /* admission in arrival order while the budget, a slot and the arena allow */
    while (!waiting.empty() && !free_slots.empty()) {
      const size_t i = waiting.front();
      QReq& q = st[i];
      if (held + q.held > p->budget_bytes) break;
      uint64_t oo = 0;
      if (q.arena_out && !arena.alloc(q.out_bytes, &oo)) break;
      q.out_off = oo;
      q.out = q.arena_out ? out_base + oo : reqs[i].out;
      q.slot = free_slots.back();
      free_slots.pop_back();
      slot_req[q.slot] = i;
      held += q.held;
      if (reqs[i].op != LK_OP_SUM_F32) {
        /* spread over the CTAs that no queued unit waits for: the backlog is
         * every admitted unit no CTA has claimed yet (published or not);
         * units already running do not count, their CTAs free up first */
        const uint64_t backlog = unpublished + (next_u - acked);
        const uint64_t claimed_bytes = acked ? cum[(acked - 1) & (ctx->qn - 1)] : 0;
        const uint64_t backlog_bytes = unpublished_bytes + (pub_bytes - claimed_bytes);
        q.parts = split_parts(reqs[i].op, reqs[i].n, (uint64_t)ctx->total, backlog, backlog_bytes, part_bytes,
                              min_part);
      }
      unpublished += q.parts;
      unpublished_bytes += q.in_bytes;
      res[i].chunks = q.parts;
      res[i].t_admit_ns = now_ns() - t0;
      active.push_back(i);
      waiting.pop_front();
    }
    /* claimed units: their entries are acknowledged in claim (index) order */
    while (acked < next_u && ld_acq(&ctx->q_units_h[acked & (ctx->qn - 1)].ack) == acked + 1) ++acked;
    /* publish one unit of each active request in turn, at most W unclaimed */
    while (!active.empty() && next_u - acked < W) {
      const size_t i = active.front();
      active.pop_front();
      QReq& q = st[i];
      const lk_request& r = reqs[i];
      lk_qunit* e = &ctx->q_units_h[next_u & (ctx->qn - 1)];
      const uint64_t tag = (((next_u >> ctx->qlog2) + 1) & 0xffffull) << LK_TAG_SHIFT;
      __atomic_thread_fence(__ATOMIC_RELEASE);   /* earlier host writes before the entry's words */
      st_rlx(&e->w[0], tag | ((uint64_t)(uintptr_t)r.in0 & LK_LOW48));
      st_rlx(&e->w[1], tag | ((uint64_t)(uintptr_t)r.in1 & LK_LOW48));
      st_rlx(&e->w[2], tag | ((uint64_t)(uintptr_t)q.out & LK_LOW48));
      st_rlx(&e->w[3], tag | (r.n & LK_LOW48));
      st_rlx(&e->w[4], tag | ((uint64_t)r.op << 32) | ((uint64_t)q.parts << 16) | (uint64_t)q.published);
      st_rlx(&e->w[5], tag | (uint64_t)q.slot);
      /* this unit's share of the input bytes, the request's split exactly */
      const uint64_t ub = q.in_bytes * (q.published + 1) / q.parts - q.in_bytes * q.published / q.parts;
      pub_bytes += ub;
      cum[next_u & (ctx->qn - 1)] = pub_bytes;
      ++next_u;
      --unpublished;
      unpublished_bytes -= ub;
      if (++q.published < q.parts) active.push_back(i);
    }
    /* retire completed requests */
    for (;;) {
      const uint64_t v = ld_acq(&ctx->q_cq_h[cq_head & (ctx->qn - 1)]);
      if ((v >> 32) != (cq_head >> ctx->qlog2) + 1) break;
      const uint32_t slot = (uint32_t)(v & 0xffffffffu);
      ++cq_head;
      if (slot >= nslots) {
        first_err = LK_EDEVICE;
        continue;
      }
      const size_t i = slot_req[slot];
      QReq& q = st[i];
      res[i].t_complete_ns = now_ns() - t0;
      res[i].status = LK_OK;
      res[i].out = q.out;
      if (q.arena_out) arena.release(q.out_off, q.out_bytes);
      held -= q.held;
      free_slots.push_back(slot);
      ++finished;
    }
  }
  stop.store(true);
  for (auto& x : th) x.join();
  /* close the queue: every worker whose claimed unit lies beyond the last
   * published one leaves, and each cluster's LK_OP_SERVE completes */
  st_rel(ctx->q_close_h, (1ull << 63) | next_u);
  beat(ctx);
  for (int c = 0; c < ctx->C; ++c) {
    const int w = lk_wait(ctx, ((uint64_t)c << 48) | serve_seq[c], 10000000000ull);
    if (w != LK_OK && first_err == LK_OK) first_err = w;
  }
  return first_err;
}

extern "C" int lk_serve(lk_ctx* ctx, const lk_request* reqs, size_t count, const lk_serve_params* p,
                        lk_request_result* res) {
  if (!ctx || !p || (count > 0 && (!reqs || !res)) || p->n_producers < 1 || p->n_producers > 256) return LK_EINVAL;
  for (int c = 1; c < ctx->C; ++c)
    if (ctx->sizes[c] != ctx->sizes[0]) return LK_EINVAL;   /* results must not depend on the cluster */
  if (p->mode == LK_SERVE_QUEUE) return serve_queue(ctx, reqs, count, p, res);
  if (p->mode != LK_SERVE_CHUNKS) return LK_EINVAL;
  const int window = p->window > 0 ? p->window : 2;
  const uint64_t chunk_bytes = p->chunk_bytes ? p->chunk_bytes : (16ull << 20);
  const uint64_t timeout = p->timeout_ns ? p->timeout_ns : 120000000000ull;
  if (chunk_bytes < 65536 || ((uintptr_t)p->arena & 255u)) return LK_EINVAL;
  const uint64_t coalesce_bytes = p->coalesce_bytes;
  const uint32_t coalesce_max = p->coalesce_max ? p->coalesce_max : 256u;
  lk_batch_tune ctune{8u, 0u, p->coalesce_part_bytes ? p->coalesce_part_bytes : (256u << 10)};
  if (coalesce_bytes > chunk_bytes || coalesce_max > 256 || (coalesce_bytes && !ctx->max_units) ||
      (coalesce_bytes && (uint64_t)coalesce_max * 8 > ctx->max_units))
    return LK_EINVAL;
  std::vector<ServeReq> st(count);
  for (size_t i = 0; i < count; ++i) {
    const lk_request& r = reqs[i];
    if (r.producer >= (uint32_t)p->n_producers) return LK_EINVAL;
    if (r.op < LK_OP_ADD_I32 || r.op > LK_OP_COPY_I32) return LK_EINVAL;
    lk_desc d{r.op, 0, r.n, 0};
    int rc = validate(&d, r.in0, r.in1, op_inputs(r.op), r.out ? r.out : (void*)(uintptr_t)256);
    if (rc != LK_OK) return rc;
    ServeReq& q = st[i];
    switch (r.op) {
      case LK_OP_ADD_I32: q.in_bytes = 8 * r.n; q.out_bytes = 4 * r.n; q.unit = 4; q.elem_bytes = 4; break;
      case LK_OP_COPY_I32: q.in_bytes = 4 * r.n; q.out_bytes = 4 * r.n; q.unit = 4; q.elem_bytes = 4; break;
      case LK_OP_SUM_F32: q.in_bytes = 4 * r.n; q.out_bytes = 16; q.unit = 4; q.elem_bytes = 4; break;
      case LK_OP_HIST_U8: q.in_bytes = r.n; q.out_bytes = 1024; q.unit = 16; q.elem_bytes = 1; break;
      default: q.in_bytes = 32768 * r.n; q.out_bytes = 16384 * r.n; q.unit = 1; q.elem_bytes = 32768; break;
    }
    /* elements per chunk: a whole number of alignment units */
    const uint64_t per_elem = r.op == LK_OP_ADD_I32 ? 8 : q.elem_bytes;
    uint64_t ce = std::max<uint64_t>(q.unit, chunk_bytes / per_elem / q.unit * q.unit);
    q.chunks = (uint32_t)std::max<uint64_t>(1, (r.n + ce - 1) / ce);
    q.coalesced = q.in_bytes <= coalesce_bytes;
    if (q.coalesced) q.chunks = 1;
    q.needs_combine = !q.coalesced && q.chunks > 1 && (r.op == LK_OP_SUM_F32 || r.op == LK_OP_HIST_U8);
    q.scratch_bytes = q.needs_combine ? (uint64_t)q.chunks * (r.op == LK_OP_SUM_F32 ? 16 : 1024) : 0;
    q.arena_out = r.out == nullptr;
    q.held = q.in_bytes + q.out_bytes + q.scratch_bytes;
    const uint64_t need = (q.arena_out ? q.out_bytes + 256 : 0) + (q.scratch_bytes ? q.scratch_bytes + 256 : 0);
    if (q.held > p->budget_bytes || need > p->arena_bytes) return LK_ENOMEM;
    res[i] = lk_request_result{0, 0, nullptr, LK_PENDING, q.chunks};
  }
  if (!ctx_alive(ctx)) return LK_ESTATE;

  /* producers: each releases its own requests at their arrival times */
  std::mutex qmu;
  std::deque<size_t> arrived;
  std::atomic<uint64_t> start{0};
  std::atomic<int> ready{0};
  std::atomic<bool> stop{false};
  std::vector<std::vector<size_t>> mine(p->n_producers);
  for (size_t i = 0; i < count; ++i) mine[reqs[i].producer].push_back(i);
  for (auto& v : mine)
    std::stable_sort(v.begin(), v.end(), [&](size_t a, size_t b) { return reqs[a].t_arrival_ns < reqs[b].t_arrival_ns; });
  auto producer = [&](int w) {
    ready.fetch_add(1);
    uint64_t t0;
    while ((t0 = start.load(std::memory_order_acquire)) == 0) {}
    for (size_t i : mine[w]) {
      while (now_ns() < t0 + reqs[i].t_arrival_ns)
        if (stop.load(std::memory_order_relaxed)) return;
      std::lock_guard<std::mutex> g(qmu);
      arrived.push_back(i);
    }
  };
  std::vector<std::thread> th;
  for (int w = 0; w < p->n_producers; ++w) th.emplace_back(producer, w);
  while (ready.load() < p->n_producers) std::this_thread::yield();
  const uint64_t t0 = now_ns();
  start.store(t0, std::memory_order_release);

  /* dispatcher */
  Arena arena(p->arena_bytes);
  uint64_t held = 0;
  std::deque<size_t> waiting;                      /* arrived, not admitted (FIFO) */
  std::deque<std::pair<size_t, uint32_t>> chunks;  /* admitted chunks to post     */
  std::deque<size_t> combines;                     /* requests whose combine is due */
  std::deque<size_t> smalls;                       /* admitted coalesced requests  */
  std::vector<std::vector<size_t>> posts;          /* members of each batch post   */
  std::vector<lk_batch_item> bitems;
  struct Fly { uint64_t seq; size_t req; int kind; };   /* kind 0 chunk, 1 combine, 2 batch (req = post) */
  std::vector<std::deque<Fly>> fly(ctx->C);
  size_t finished = 0;
  int first_err = LK_OK;
  int rr = 0;
  auto complete = [&](size_t i, int status) {
    ServeReq& q = st[i];
    res[i].t_complete_ns = now_ns() - t0;
    res[i].status = status;
    res[i].out = q.out;
    if (q.arena_out) arena.release(q.out_off, q.out_bytes);
    if (q.scratch_bytes) arena.release(q.scratch_off, q.scratch_bytes);
    held -= q.held;
    ++finished;
    if (status != LK_OK && first_err == LK_OK) first_err = status;
  };
  auto post_chunk = [&](int c, size_t i, uint32_t j, uint64_t* seq) -> int {
    const lk_request& r = reqs[i];
    ServeReq& q = st[i];
    const uint64_t per_elem = r.op == LK_OP_ADD_I32 ? 8 : q.elem_bytes;
    const uint64_t ce = std::max<uint64_t>(q.unit, chunk_bytes / per_elem / q.unit * q.unit);
    const uint64_t e0 = (uint64_t)j * ce, e1 = std::min<uint64_t>(r.n, e0 + ce);
    const uint64_t step = r.op == LK_OP_GEMM64_F32 ? 16384 : q.elem_bytes;   /* bytes per element of in0/in1/out */
    const char* a0 = (const char*)r.in0;
    const char* a1 = (const char*)r.in1;
    char* o = (char*)q.out;
    lk_desc d{r.op, 0, e1 - e0, 0};
    const void* in0 = a0 ? a0 + e0 * step : nullptr;
    const void* in1 = a1 ? a1 + e0 * step : nullptr;
    void* out;
    if (r.op == LK_OP_SUM_F32) out = q.needs_combine ? (char*)q.scratch + 16 * j : q.out;
    else if (r.op == LK_OP_HIST_U8) out = q.needs_combine ? (char*)q.scratch + 1024 * j : q.out;
    else out = o + e0 * (r.op == LK_OP_GEMM64_F32 ? 16384 : 4);
    return post(ctx, c, LK_CMD_WORK + r.op, &d, in0, in1, out, seq);
  };
  while (finished < count) {
    const uint64_t now = now_ns();
    if (now - t0 > timeout) {
      for (size_t i = 0; i < count; ++i)
        if (res[i].status == LK_PENDING) res[i].status = LK_ETIMEDOUT;
      if (first_err == LK_OK) first_err = LK_ETIMEDOUT;
      break;
    }
    if (!ctx_alive(ctx)) {
      int e = device_err_to_rc(dev_error(ctx));
      for (size_t i = 0; i < count; ++i)
        if (res[i].status == LK_PENDING) res[i].status = e ? e : LK_ESTATE;
      if (first_err == LK_OK) first_err = e ? e : LK_ESTATE;
      break;
    }
    {
      std::lock_guard<std::mutex> g(qmu);
      while (!arrived.empty()) {
        waiting.push_back(arrived.front());
        arrived.pop_front();
      }
    }
    /* admission in arrival order while the budget and the arena allow */
    while (!waiting.empty()) {
      const size_t i = waiting.front();
      ServeReq& q = st[i];
      if (held + q.held > p->budget_bytes) break;
      uint64_t oo = 0, so = 0;
      if (q.arena_out && !arena.alloc(q.out_bytes, &oo)) break;
      if (q.scratch_bytes && !arena.alloc(q.scratch_bytes, &so)) {
        if (q.arena_out) arena.release(oo, q.out_bytes);
        break;
      }
      q.out_off = oo;
      q.scratch_off = so;
      q.out = q.arena_out ? (char*)p->arena + oo : reqs[i].out;
      q.scratch = q.scratch_bytes ? (char*)p->arena + so : nullptr;
      held += q.held;
      res[i].t_admit_ns = now_ns() - t0;
      if (q.coalesced) smalls.push_back(i);
      else for (uint32_t j = 0; j < q.chunks; ++j) chunks.emplace_back(i, j);
      waiting.pop_front();
    }
    /* clusters pull: each takes work while its window has room; coalesced
     * requests go out many to a batch post, in arrival order against the
     * chunks of larger requests */
    for (int k = 0; k < ctx->C; ++k) {
      const int c = (rr + k) % ctx->C;
      while ((int)fly[c].size() < window && (!combines.empty() || !chunks.empty() || !smalls.empty())) {
        uint64_t seq = 0;
        if (!combines.empty()) {
          const size_t i = combines.front();
          ServeReq& q = st[i];
          lk_desc d{reqs[i].op == LK_OP_SUM_F32 ? (uint32_t)LK_OP_COMBINE_SUM : (uint32_t)LK_OP_COMBINE_HIST, 0,
                    q.chunks, 0};
          if (post(ctx, c, LK_CMD_WORK + d.op, &d, q.scratch, nullptr, q.out, &seq) != LK_OK) break;
          fly[c].push_back({seq, i, 1});
          combines.pop_front();
        } else if (!smalls.empty() &&
                   (chunks.empty() || reqs[smalls.front()].t_arrival_ns <= reqs[chunks.front().first].t_arrival_ns)) {
          const size_t take = std::min<size_t>(smalls.size(), coalesce_max);
          bitems.clear();
          for (size_t m = 0; m < take; ++m) {
            const size_t i = smalls[m];
            const lk_request& r = reqs[i];
            bitems.push_back(lk_batch_item{r.in0, r.in1, st[i].out, r.op, 0u, r.n});
          }
          lk_handle h = 0;
          if (lk_submit_batch(ctx, c, bitems.data(), (uint32_t)take, &ctune, &h) != LK_OK) break;
          posts.emplace_back(smalls.begin(), smalls.begin() + (long)take);
          smalls.erase(smalls.begin(), smalls.begin() + (long)take);
          fly[c].push_back({h & kSeqMask, posts.size() - 1, 2});
        } else if (!chunks.empty()) {
          const auto cj = chunks.front();
          if (post_chunk(c, cj.first, cj.second, &seq) != LK_OK) break;
          fly[c].push_back({seq, cj.first, 0});
          chunks.pop_front();
        } else {
          break;
        }
      }
    }
    rr = (rr + 1) % ctx->C;
    /* completions (FIFO per cluster) */
    for (int c = 0; c < ctx->C; ++c) {
      if (fly[c].empty()) continue;
      const uint64_t done = cl_done(ctx, c);
      while (!fly[c].empty() && fly[c].front().seq <= done) {
        const Fly f = fly[c].front();
        fly[c].pop_front();
        if (f.kind == 2) {
          for (size_t i : posts[f.req]) complete(i, LK_OK);
          posts[f.req].clear();
          posts[f.req].shrink_to_fit();
          continue;
        }
        ServeReq& q = st[f.req];
        if (f.kind == 1) {
          complete(f.req, LK_OK);
        } else if (++q.done_chunks == q.chunks) {
          if (q.needs_combine) combines.push_back(f.req);
          else complete(f.req, LK_OK);
        }
      }
    }
    if ((finished & 1023) == 0) beat(ctx);
  }
  stop.store(true);
  for (auto& x : th) x.join();
  beat(ctx);
  return first_err;
}
