/*
 * lk_kernel.cu -- the LightKernel persistent kernel for sm_103a, its CUDA
 * backend, the ordinary-launch baseline and the host-mapped ping-pong.
 *
 * Persistent kernel (Sec. II.C): spawned once, one CTA per SM (the dynamic
 * shared-memory request leaves no room for a second CTA, and the launch is
 * cooperative so all CTAs are resident or the launch fails).  At boot every
 * CTA reads %smid; the CTAs exchange their SM ids and each one joins the
 * cluster that its SM belongs to (clusters are cut from the sorted SM ids, or
 * given as explicit SM lists).  The paper's check that a block sits on the SM
 * it expects becomes a table built from the SM ids actually observed.
 *
 * Mailboxes (Sec. II.D, Table 1): rank 0's thread 0 -- the paper's master
 * thread -- polls its cluster's host-mapped ring and relays each descriptor
 * through a device ring (with LK_INIT_DIRECT every CTA's thread 0 polls the
 * ring itself; with LK_INIT_MAILBOX the master runs the paper's one-deep
 * to_GPU / from_GPU handshake instead of the ring), and every CTA runs its
 * share.  Each CTA then release-stores its own finished count; rank 0 gathers
 * the counts, combines partial results and publishes the descriptor's
 * sequence number in the host-mapped `done` word (from_GPU =
 * THREAD_FINISHED; the status word itself in mailbox mode).
 *
 * Every device-side wait is bounded: by an idle lease (refreshed by the
 * host's heartbeat), by the host's abort word, and by a stall deadline.  On
 * expiry the kernel records the reason and returns normally.
 */
#include <cuda_runtime.h>
#include <pthread.h>
#include <sched.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "lk_backend.h"
#include "lk_bodies.cuh"
#include "lk_layout.h"
#include "lk_validate.h"

using namespace lk;

#define LK_GEN_STOP 0xffffffffffffffffull

/* ======================================================================= */
/* device side                                                              */
/* ======================================================================= */

__device__ __forceinline__ void set_error(const lk_kargs& a, int c, uint32_t code) {
  cas_relaxed_sys(&a.ctrl->first_error, 0u, code);
  if (c >= 0) st_relaxed_sys(&a.cword[c].error, (uint64_t)code);
  __threadfence_system();
}

__device__ __forceinline__ void ld_relaxed_sys_v2(const uint64_t* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.relaxed.sys.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_sys() { asm volatile("fence.acq_rel.sys;" ::: "memory"); }

__device__ __forceinline__ bool tags_match(const uint64_t* w, uint64_t tag) {
  return (w[0] >> LK_TAG_SHIFT) == tag && (w[1] >> LK_TAG_SHIFT) == tag && (w[2] >> LK_TAG_SHIFT) == tag &&
         (w[3] >> LK_TAG_SHIFT) == tag && (w[4] >> LK_TAG_SHIFT) == tag && (w[5] >> LK_TAG_SHIFT) == tag;
}
/* One probe of a ring slot: three vector loads in flight together, the last
 * an acquire.  When every tag is current, that acquire load has read a word
 * the host stored after its release fence, so it synchronises with the
 * host's post and no system-scope fence is needed (measured on GB300: a
 * system-scope fence after relaxed system-scope loads cost 0.48 us of a
 * host round trip; an acquire load in the probe, nothing). */
__device__ __forceinline__ void probe(const lk_wire* s, uint64_t* w) {
  ld_relaxed_sys_v2(&s->w[0], w[0], w[1]);
  ld_relaxed_sys_v2(&s->w[2], w[2], w[3]);
  asm volatile("ld.acquire.sys.v2.u64 {%0, %1}, [%2];" : "=l"(w[4]), "=l"(w[5]) : "l"(&s->w[4]) : "memory");
}

/* Wait until ring slot `s` holds ticket k (every tagged word carries lap tag
 * `tag`), then decode it.  A probe loads the six tagged words at once, so it
 * costs one round trip over the host link.  One probe at a time, from one
 * thread: every extra read in flight on the slot's line makes the host's
 * stores to that line wait for ownership again.  The acquire fence after a
 * successful probe pairs with the host's release fence before its stores.
 * Each probe also loads *pre (device memory, relaxed, in flight beside the
 * probe, so it costs no extra time) into *pre_val: the completion word the
 * caller gates on next, read while it waits anyway; the GPU-scope fence
 * after success makes that load an acquire.  Returns 0 or an LK_DERR_*
 * reason (lease ran out, abort). */
__device__ __forceinline__ int take_from_ring(const lk_kargs& a, const lk_wire* s, uint64_t tag, uint64_t seq,
                                              lk_slot& out, const uint64_t* pre, uint64_t* pre_val) {
  Backoff bo(a.backoff_base_ns, a.backoff_cap_ns);
  uint64_t hb = ld_relaxed_sys(&a.ctrl->heartbeat);
  uint64_t t_last = gtime();
  uint64_t abort_v = 0, hb_v = hb;   /* loaded at the previous check, used at the next */
  uint64_t w[6];
  for (uint32_t it = 1;; ++it) {
    uint64_t pv;
    asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(pv) : "l"(pre) : "memory");
    probe(s, w);
    if (tags_match(w, tag)) {
      *pre_val = pv;
      break;
    }
    if ((it & 63) == 0) {
      if (abort_v) return LK_DERR_ABORT;
      const uint64_t now = gtime();
      if (now - t_last > a.lease_ns) {
        if (hb_v == hb) return LK_DERR_LEASE;
        hb = hb_v;
        t_last = now;
      }
      abort_v = ld_relaxed_sys(&a.ctrl->abort);
      hb_v = ld_relaxed_sys(&a.ctrl->heartbeat);
    }
    bo.pause();
  }
  /* the probe's acquire load synchronised with the host's post; this
   * GPU-scope fence orders the prefetched completion word (a relaxed load)
   * before everything this CTA does next, the relay included */
  fence_acq_rel_gpu();
  lk_wire_decode(w, seq, &out);
  return 0;
}

/* One-deep mailbox (LK_INIT_MAILBOX, Sec. II.D, Table 1), master thread
 * only.  Descriptor k+1 is taken in up to two steps:
 *   1. (k > 0) the re-arm of the four-phase handshake: wait for
 *      to_GPU = THREAD_NOP, which the host writes once it saw
 *      THREAD_FINISHED for descriptor k, and acknowledge with
 *      from_GPU = THREAD_NOP;
 *   2. wait for to_GPU = THREAD_EXIT or THREAD_WORK + op; after the acquire
 *      fence, read the descriptor's words (a second round trip over the host
 *      link: the ring's lap tags exist to save it) and answer
 *      from_GPU = THREAD_WORKING.
 * Both waits are bounded like take_from_ring's.  Returns 0 or LK_DERR_*. */
__device__ __noinline__ int wait_to_gpu(const lk_kargs& a, const uint64_t* p, bool want_nop, uint64_t* v_out) {
  Backoff bo(a.backoff_base_ns, a.backoff_cap_ns);
  uint64_t hb = ld_relaxed_sys(&a.ctrl->heartbeat);
  uint64_t t_last = gtime();
  uint64_t v;
  for (uint32_t it = 1;; ++it) {
    v = ld_acquire_sys(p);   /* an acquire load: the fence below is then nearly free */
    if (want_nop ? v == LK_CMD_NOP : (v == LK_CMD_EXIT || v >= LK_CMD_WORK)) break;
    if ((it & 63) == 0) {
      if (ld_relaxed_sys(&a.ctrl->abort)) return LK_DERR_ABORT;
      const uint64_t now = gtime();
      if (now - t_last > a.lease_ns) {
        const uint64_t h = ld_relaxed_sys(&a.ctrl->heartbeat);
        if (h == hb) return LK_DERR_LEASE;
        hb = h;
        t_last = now;
      }
    }
    bo.pause();
  }
  fence_acq_rel_sys();
  *v_out = v;
  return 0;
}

__device__ __noinline__ int take_from_mailbox(const lk_kargs& a, int c, uint64_t k, lk_slot& out) {
  lk_mbox* mb = a.mbox + c;
  uint64_t v = 0;
  if (k > 0) {
    const int err = wait_to_gpu(a, &mb->to_gpu, true, &v);
    if (err) return err;
    st_relaxed_sys(&a.cword[c].status, LK_ST_NOP);
  }
  const int err = wait_to_gpu(a, &mb->to_gpu, false, &v);
  if (err) return err;
  uint64_t w[6] = {0, 0, 0, 0, 0, 0};
  if (v != LK_CMD_EXIT) {
    ld_relaxed_sys_v2(&mb->n, w[0], w[1]);
    ld_relaxed_sys_v2(&mb->in1, w[2], w[3]);
    ld_relaxed_sys_v2(&mb->aux, w[4], w[5]);
  }
  out.seq = k + 1;
  out.cmd = (uint32_t)v;
  out.flags = (uint32_t)w[5];
  out.n = w[0];
  out.in0 = w[1];
  out.in1 = w[2];
  out.out = w[3];
  out.aux = w[4];
  out.t_pick = 0;
  if (v == LK_CMD_EXIT) return 0;
  st_relaxed_sys(&a.cword[c].status, LK_ST_WORKING);
  return 0;
}

/* Relay (the default delivery): the master copies descriptor k into relay slot
 * k mod D as six lap-tagged words (the host ring's format, tag = relay lap),
 * after the fence that followed its ring probe, so members need no separate
 * generation word: they probe the slot in L2 (one round trip, the last load
 * an acquire) and accept it when every tag is current.  No timestamp rides
 * in the slot: reading %globaltimer is slow, so no store waits on one. */
__device__ __forceinline__ void relay_publish(lk_wire* rs, uint64_t k, const lk_slot& d) {
  const uint64_t tag = ((k / LK_BCAST_DEPTH + 1) & 0xffffull) << LK_TAG_SHIFT;
  const uint64_t v[6] = {tag | ((uint64_t)(d.flags & 0xffffu) << 16) | (d.cmd & 0xffffu), tag | (d.n & LK_LOW48),
                         tag | (d.in0 & LK_LOW48), tag | (d.in1 & LK_LOW48), tag | (d.out & LK_LOW48),
                         tag | (d.aux & LK_LOW48)};
#pragma unroll
  for (int i = 0; i < 6; ++i) asm volatile("st.relaxed.gpu.u64 [%0], %1;" ::"l"(&rs->w[i]), "l"(v[i]) : "memory");
}

/* One probe of a relay slot: three vector loads, the last an acquire (when
 * every tag is current it read a word the master stored after its fence,
 * so it synchronises with the master; no separate fence follows). */
__device__ __forceinline__ void relay_probe(const lk_wire* rs, uint64_t* w) {
  asm volatile("ld.relaxed.gpu.v2.u64 {%0, %1}, [%2];" : "=l"(w[0]), "=l"(w[1]) : "l"(&rs->w[0]) : "memory");
  asm volatile("ld.relaxed.gpu.v2.u64 {%0, %1}, [%2];" : "=l"(w[2]), "=l"(w[3]) : "l"(&rs->w[2]) : "memory");
  asm volatile("ld.acquire.gpu.v2.u64 {%0, %1}, [%2];" : "=l"(w[4]), "=l"(w[5]) : "l"(&rs->w[4]) : "memory");
}

/* A relayed member waits for descriptor k in relay slot rs (L2).  One probe
 * at a time (measured: a second staggered probe in flight did not lower the
 * broadcast latency to 36 members, about 0.6 us).  The periodic checks
 * (abort word, master stop, lease) read their words without waiting on
 * them: each check uses the values loaded at the previous one.  Returns 0,
 * -1 (the master stopped) or an LK_DERR_* reason. */
__device__ __forceinline__ int take_from_relay(const lk_kargs& a, const lk_dcluster* dc, const lk_wire* rs, uint64_t k,
                                               lk_slot& out) {
  const uint64_t tag = (k / LK_BCAST_DEPTH + 1) & 0xffffull;
  Backoff bo(a.backoff_base_ns, a.backoff_cap_ns);
  uint64_t hb = ld_relaxed_sys(&a.ctrl->heartbeat);
  uint64_t t_last = gtime();
  const uint64_t limit = a.lease_ns + 1000000000ull;
  uint64_t abort_v = 0, gen_v = 0, hb_v = hb;
  uint64_t w[6];
  for (uint32_t it = 1;; ++it) {
    relay_probe(rs, w);
    if (tags_match(w, tag)) break;
    if ((it & 127) == 0) {
      /* act on the words loaded one check ago, then load them again */
      if (abort_v) return LK_DERR_ABORT;
      if (gen_v == LK_GEN_STOP) return -1;
      const uint64_t now = gtime();
      if (now - t_last > limit) {
        if (hb_v == hb) return LK_DERR_STALL;
        hb = hb_v;
        t_last = now;
      }
      abort_v = ld_relaxed_sys(&a.ctrl->abort);
      asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(gen_v) : "l"(&dc->gen) : "memory");
      hb_v = ld_relaxed_sys(&a.ctrl->heartbeat);
    }
    bo.pause();
  }
  lk_wire_decode(w, k + 1, &out);
  return 0;
}

/* Wait until *word >= want (GPU scope): relay generation, device-side done.
 * `stop_on_max` treats LK_GEN_STOP as the master's stop signal (returns -1).
 * *seen (optional) receives the value that satisfied the wait. */
__device__ __noinline__ int wait_word(const lk_kargs& a, const uint64_t* word, uint64_t want, bool stop_on_max,
                                      uint64_t* seen = nullptr) {
  Backoff bo(a.backoff_base_ns, a.backoff_cap_ns);
  uint64_t hb = ld_relaxed_sys(&a.ctrl->heartbeat);
  uint64_t t_last = gtime();
  const uint64_t limit = a.lease_ns + 1000000000ull;
  for (uint32_t it = 1;; ++it) {
    const uint64_t g = ld_acquire_gpu(word);
    if (stop_on_max && g == LK_GEN_STOP) return -1;
    if (g >= want) {
      if (seen) *seen = g;
      return 0;
    }
    if ((it & 255) == 0) {
      if (ld_relaxed_sys(&a.ctrl->abort)) return LK_DERR_ABORT;
      const uint64_t now = gtime();
      if (now - t_last > limit) {
        const uint64_t h = ld_relaxed_sys(&a.ctrl->heartbeat);
        if (h == hb) return LK_DERR_STALL;
        hb = h;
        t_last = now;
      }
    }
    bo.pause();
  }
}

/* Every warp of rank 0: wait until every rank of the cluster has finished
 * descriptor `want` (flag[q] >= want).  Lanes poll disjoint ranks in
 * parallel; the warps poll independently, each one round trip per pass, and
 * the first to see every flag raised tells the others through *found --
 * with their passes out of step, a raised flag is seen sooner than by one
 * warp alone.  Returns 0 or an LK_DERR_* reason (same bounds as wait_word). */
__device__ __noinline__ int gather_flags(const lk_kargs& a, const uint64_t* flag, int S, uint64_t want,
                                         volatile int* found) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t pending = 0;   /* bit j: rank lane + 32 j not seen yet */
  for (int j = 0; j < 32 && (int)lane + 32 * j < S; ++j) pending |= 1u << j;
  uint64_t hb = 0, t_last = 0;
  if (lane == 0) {
    hb = ld_relaxed_sys(&a.ctrl->heartbeat);
    t_last = gtime();
  }
  const uint64_t limit = a.lease_ns + 1000000000ull;
  for (uint32_t it = 1;; ++it) {
    if (__any_sync(0xffffffffu, *found != 0)) {   /* warp-uniform */
      fence_acq_rel_gpu();
      return 0;
    }
    /* relaxed loads can all be in flight at once (acquire loads would each
     * wait for the one before); one acquire fence follows success */
    for (int g = 0; g < 32 && (pending >> g); g += 8) {
      uint64_t v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (pending & (1u << (g + j)))
          asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(v[j]) : "l"(flag + lane + 32 * (g + j)) : "memory");
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if ((pending & (1u << (g + j))) && v[j] >= want) pending &= ~(1u << (g + j));
    }
    if (__all_sync(0xffffffffu, pending == 0)) {
      fence_acq_rel_gpu();
      if (lane == 0) *found = 1;
      return 0;
    }
    if ((it & 255) == 0) {
      int err = 0;
      if (lane == 0) {
        if (ld_relaxed_sys(&a.ctrl->abort)) {
          err = LK_DERR_ABORT;
        } else {
          const uint64_t now = gtime();
          if (now - t_last > limit) {
            const uint64_t h = ld_relaxed_sys(&a.ctrl->heartbeat);
            if (h == hb) err = LK_DERR_STALL;
            hb = h;
            t_last = now;
          }
        }
      }
      err = __shfl_sync(0xffffffffu, err, 0);
      if (err) return err;
    }
  }
}

/* Per-CTA pace of a descriptor whose `aux` caps the cluster's load rate
 * (bytes per microsecond over its S CTAs; 0 = none). */
__device__ __forceinline__ uint64_t cta_rate(uint64_t cluster_rate, int S) {
  if (!cluster_rate) return 0;
  const uint64_t r = cluster_rate / (uint64_t)S;
  return r ? r : 1;
}

/* This CTA's share of descriptor d (rank r of S).  Returns an LK_DERR_* code
 * or 0.  `partial_out` receives the sum body's per-CTA partial.  MAXT (the
 * largest block size of the calling kernel) sets how far the GEMM's k loop is
 * unrolled: fully at up to 256 threads with one CTA per SM, where the
 * registers allow it.  P (CTAs per SM) sets the shared-memory budget.
 * `rate` (bytes per microsecond for this CTA, 0 = unpaced) paces the loads
 * of the streaming and GEMM bodies; `tc` lets whole GEMM tiles use the
 * tensor cores. */
template <int MAXT, int P>
__device__ __forceinline__ int run_body(const lk_slot& d, int r, int S, unsigned char* dsm, uint64_t* bars,
                                        uint32_t& phase, float* red, float* partial_out, HistSink hist,
                                        uint64_t rate, const int32_t* gate, bool tc = true) {
  const uint32_t op = d.cmd - LK_CMD_WORK;
  const Pace deadline{gtime() + 2000000000ull, rate, gate};
  bool ok = true;
  switch (op) {
    case LK_OP_ADD_I32: ok = body_add<P, (MAXT <= 256 && P == 1)>(d, r, S, dsm, bars, phase, deadline); break;
    case LK_OP_COPY_I32: ok = body_copy<P>(d, r, S, dsm, bars, phase, deadline); break;
    case LK_OP_SUM_F32:
      ok = body_sum<P, (MAXT <= 256 && P == 1)>(d, r, S, dsm, bars, phase, deadline, red, partial_out);
      break;
    case LK_OP_HIST_U8: ok = body_hist<P>(d, r, S, dsm, bars, phase, deadline, hist); break;
    case LK_OP_GEMM64_F32:
      ok = body_gemm<(MAXT <= 256 && P == 1), P>(d, r, S, reinterpret_cast<float*>(dsm), bars, phase, deadline, tc);
      break;
    case LK_OP_COMBINE_SUM: body_combine_sum(d, r); break;
    case LK_OP_COMBINE_HIST: body_combine_hist(d, r); break;
    case LK_OP_SPIN: body_spin(d, r, reinterpret_cast<uint32_t*>(red)); break;
    case LK_OP_NOP: break;
    default: return LK_DERR_BADDESC;
  }
#ifdef LK_DEBUG_BOUNDS
  if (lk_oob_seen()) return LK_DERR_BOUNDS;
#endif
  return ok ? 0 : LK_DERR_STAGING;
}

/* Serving queue: thread 0 waits until unit u of the ring is published (all
 * six words of entry u mod Q carry u's lap tag), or the host closed the
 * queue below u.  The entry is this CTA's alone (units are claimed once), so
 * its probe delays no other reader; one probe reads the whole entry, its
 * last load an acquire.  The ack tells the host the entry may be rewritten.
 * Returns 0 (w[0..5] = in0, in1, out, n, op/parts/part, slot, tags
 * stripped), 1 (closed: no unit u) or an LK_DERR_* reason. */
__device__ __noinline__ int serve_take(const lk_kargs& a, uint32_t qlog2, lk_qunit* e, uint64_t u,
                                       const uint64_t* close, uint64_t* w) {
  Backoff bo(a.backoff_base_ns, a.backoff_cap_ns);
  uint64_t hb = ld_relaxed_sys(&a.ctrl->heartbeat);
  uint64_t t_last = gtime();
  uint64_t close_v = 0, abort_v = 0, hb_v = hb;   /* loaded at one check, used at the next */
  const uint64_t tag = ((u >> qlog2) + 1) & 0xffffull;
  for (uint32_t it = 1;; ++it) {
    ld_relaxed_sys_v2(&e->w[0], w[0], w[1]);
    ld_relaxed_sys_v2(&e->w[2], w[2], w[3]);
    asm volatile("ld.acquire.sys.v2.u64 {%0, %1}, [%2];" : "=l"(w[4]), "=l"(w[5]) : "l"(&e->w[4]) : "memory");
    if (tags_match(w, tag)) break;
    if ((it & 15) == 0) {
      if ((close_v >> 63) && u >= (close_v & ~(1ull << 63))) return 1;
      close_v = ld_relaxed_sys(close);
    }
    if ((it & 63) == 0) {
      if (abort_v) return LK_DERR_ABORT;
      const uint64_t now = gtime();
      if (now - t_last > a.lease_ns) {
        if (hb_v == hb) return LK_DERR_LEASE;
        hb = hb_v;
        t_last = now;
      }
      abort_v = ld_relaxed_sys(&a.ctrl->abort);
      hb_v = ld_relaxed_sys(&a.ctrl->heartbeat);
    }
    bo.pause();
  }
  for (int i = 0; i < 6; ++i) w[i] &= LK_LOW48;
  st_relaxed_sys(&e->ack, u + 1);
  return 0;
}

/* Work units, claimed one at a time by each CTA of the cluster, for two
 * descriptors (one loop, so the bodies are inlined once for both):
 *   LK_OP_BATCH (lk_submit_batch): units from the batch's table in pinned
 *     host-mapped memory, claimed with the cluster's ticket; the batch ends
 *     when the table is exhausted.  Parts of a split sum or histogram
 *     combine through per-item state in the cluster's batch state.
 *   LK_OP_SERVE (lk_serve's device queue): the CTAs of every serving
 *     cluster claim the next unit index from one device counter and wait
 *     for that entry of the host-mapped unit ring (serve_take), until the
 *     queue closes.  Parts combine through the request's slot; the last
 *     part also appends the request to the completion ring, after a
 *     system-scope fence.
 * A unit is one part of one item or request, run by this CTA with the
 * body's (part, parts) split, so a result depends only on the item and its
 * parts.  The last part to finish (an acquire-release counter) writes a
 * split result -- sums in binary64 by combine_sum, as a cluster of `parts`
 * CTAs would, so a split sum is bit-identical to it -- and returns the
 * state to zero.  Returns an LK_DERR_* code or 0. */
template <int MAXT, int P>
__device__ __forceinline__ int run_units(const lk_kargs& a, const lk_slot& d, int c, int r, unsigned char* dsm,
                                         uint64_t* bars, uint32_t& phase, float* red) {
  __shared__ uint64_t s_w[5];                    /* in0, in1, out, op << 56 | n, unused */
  __shared__ int s_take;                         /* 0 unit claimed, 1 none left, else LK_DERR_* */
  __shared__ uint32_t s_part, s_parts;
  __shared__ float* s_psum;                      /* per-part sums of a split item */
  __shared__ uint32_t* s_pbins;                  /* accumulator of a split histogram */
  __shared__ uint32_t* s_pdone;                  /* parts finished (split items) */
  __shared__ uint32_t s_rslot;                   /* serve: the request's slot */
  __shared__ float s_part_sum;
  __shared__ int s_lastp;
  const bool serve = d.cmd == LK_CMD_WORK + LK_OP_SERVE;
  uint32_t* my_hist = a.cta_hist + (size_t)(a.cl_start[c] + r) * 256u;
  /* batch */
  lk_bcluster* bc = a.bcl + c;
  const lk_unit* units = reinterpret_cast<const lk_unit*>(d.in0);
  const uint64_t nunits = d.n;
  /* serve */
  lk_qstate* qs = reinterpret_cast<lk_qstate*>(d.in0);
  lk_qunit* qunits = nullptr;
  uint64_t* cq = nullptr;
  const uint64_t* qclose = nullptr;
  lk_qslot* qslots = nullptr;
  uint64_t qmask = 0;
  uint32_t qlog2 = 0, nslots = 0;
  if (serve) {
    qunits = reinterpret_cast<lk_qunit*>(__ldcg(reinterpret_cast<const unsigned long long*>(&qs->units)));
    cq = reinterpret_cast<uint64_t*>(__ldcg(reinterpret_cast<const unsigned long long*>(&qs->cq)));
    qclose = reinterpret_cast<const uint64_t*>(__ldcg(reinterpret_cast<const unsigned long long*>(&qs->close)));
    qslots = reinterpret_cast<lk_qslot*>(__ldcg(reinterpret_cast<const unsigned long long*>(&qs->slots)));
    qmask = __ldcg(reinterpret_cast<const unsigned long long*>(&qs->qmask));
    qlog2 = __ldcg(&qs->qlog2);
    nslots = __ldcg(&qs->nslots);
  }
  const uint64_t rate = serve ? 0 : cta_rate(d.aux, a.cl_start[c + 1] - a.cl_start[c]);
  const int32_t* gate = (d.flags & LK_DFLAG_YIELD) ? a.crit_active : nullptr;
  for (;;) {
    if (threadIdx.x == 0) {
      uint64_t w[5] = {0, 0, 0, 0, 0};
      int take = 0;
      uint32_t part = 0, parts = 1;
      if (serve) {
        const unsigned long long u = atomicAdd(&qs->head, 1ull);
        uint64_t e[6];
        take = serve_take(a, qlog2, qunits + (u & qmask), u, qclose, e);
        part = (uint32_t)(e[4] & 0xffffu);
        parts = (uint32_t)((e[4] >> 16) & 0xffffu);
        const uint32_t rslot = (uint32_t)e[5];
        w[0] = e[0];
        w[1] = e[1];
        w[2] = e[2];
        w[3] = ((e[4] >> 32) & 0xffull) << 56 | e[3];   /* op << 56 | n, as a batch unit */
        if (!take && (rslot >= nslots || parts < 1 || parts > LK_SERVE_MAX_PARTS || part >= parts))
          take = LK_DERR_BADDESC;
        if (!take) {
          lk_qslot* sl = qslots + rslot;
          s_psum = sl->partial;
          s_pbins = sl->bins;
          s_pdone = &sl->done;
          s_rslot = rslot;
        }
      } else {
        const unsigned long long u = atomicAdd(&bc->ticket, 1ull);
        if (u < nunits) {
          const ulonglong2* p = reinterpret_cast<const ulonglong2*>(units + u);
          const ulonglong2 v0 = __ldcv(p), v1 = __ldcv(p + 1), v2 = __ldcv(p + 2);
          w[0] = v0.x; w[1] = v0.y; w[2] = v1.x; w[3] = v1.y;
          part = (uint32_t)(v2.x & 0xffu);
          parts = (uint32_t)((v2.x >> 8) & 0xffu);
          const uint64_t comb = v2.x >> 16;   /* combine slot + 1, 0 = none */
          const uint32_t op = (uint32_t)(w[3] >> 56);
          if (comb && op == LK_OP_SUM_F32) {
            s_psum = bc->sums[comb - 1].partial;
            s_pdone = &bc->sums[comb - 1].done;
          } else if (comb && op == LK_OP_HIST_U8) {
            s_pbins = bc->hists[comb - 1].bins;
            s_pdone = &bc->hists[comb - 1].done;
          }
        } else {
          take = 1;
        }
      }
      for (int i = 0; i < 5; ++i) s_w[i] = w[i];
      s_part = part;
      s_parts = parts;
      s_take = take;
    }
    __syncthreads();
    const int take = s_take;   /* CTA-uniform */
    if (take) return take == 1 ? 0 : take;
    const uint32_t op = (uint32_t)(s_w[3] >> 56);
    const uint32_t part = s_part, parts = s_parts;
    lk_slot it;
    it.seq = d.seq;
    it.cmd = LK_CMD_WORK + op;
    it.flags = 0;
    it.n = s_w[3] & LK_LOW48;
    it.in0 = s_w[0];
    it.in1 = s_w[1];
    it.out = s_w[2];
    it.aux = 0;
    it.t_pick = 0;
    const Pace deadline{gtime() + 2000000000ull, rate, gate};
    bool ok = true;
    if (op == LK_OP_SUM_F32) {
      float* pout = parts > 1 ? s_psum + part : &s_part_sum;
      ok = body_sum<P, (MAXT <= 256 && P == 1)>(it, (int)part, (int)parts, dsm, bars, phase, deadline, red, pout);
    } else if (op == LK_OP_HIST_U8) {
      ok = body_hist<P>(it, (int)part, (int)parts, dsm, bars, phase, deadline,
                        HistSink{parts > 1 ? s_pbins : my_hist, nullptr, 0, nullptr});
    } else {
      ok = run_body<MAXT, P>(it, (int)part, (int)parts, dsm, bars, phase, red, nullptr, HistSink{}, rate, gate,
                             (a.flags & LK_KFLAG_GEMM_FFMA) == 0) == 0;
    }
    __syncthreads();
    /* the last part of a split sum or histogram (a single part always is) finishes it */
    const bool split = parts > 1 && (op == LK_OP_SUM_F32 || op == LK_OP_HIST_U8 || serve);
    if (threadIdx.x == 0) {
      s_lastp = 1;
      if (split) {
        __threadfence();
        s_lastp = atomicAdd(s_pdone, 1u) == parts - 1;
        if (s_lastp) __threadfence();
      }
    }
    __syncthreads();
    if (s_lastp) {
      if (op == LK_OP_SUM_F32) {
        if (parts > 1) combine_sum(it, s_psum, (int)parts);
        else if (threadIdx.x == 0) *reinterpret_cast<float*>(it.out) = s_part_sum;
      } else if (op == LK_OP_HIST_U8) {
        combine_hist(it, parts > 1 ? s_pbins : my_hist);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        if (split) *s_pdone = 0;
        if (serve) {
          /* every output write of the request before its completion entry */
          fence_acq_rel_sys();
          const unsigned long long pos = atomicAdd(&qs->cq_tail, 1ull);
          st_relaxed_sys(cq + (pos & qmask), (((uint64_t)pos >> qlog2) + 1) << 32 | s_rslot);
        }
      }
    }
    __syncthreads();   /* the shared claim words are rewritten by the next claim */
    if (!ok) return LK_DERR_STAGING;
  }
}

template <int MAXT, int P>
__device__ __forceinline__ void persistent_main(const lk_kargs& a) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(64) lk_slot s_desc;
  __shared__ int32_t s_cl, s_rank, s_size, s_exit, s_err;
  __shared__ volatile int s_found;     /* rank 0: a warp saw every rank's flag (mailbox mode) */
  __shared__ int32_t s_last;           /* this CTA arrived last on the descriptor's slot */
  __shared__ uint64_t s_slot_seen;     /* the slot's completion word, read while probing */
  __shared__ uint64_t s_tpick, s_tstart; /* thread 0's stamps, for the execution log */
  __shared__ float s_red[32];
  __shared__ __align__(8) uint64_t s_bars[LK_ALL_BARS];
  const uint32_t tid = threadIdx.x;

  /* ---- boot: read %smid, exchange, join a cluster --------------------- */
  __shared__ int32_t s_sm, s_slot, s_pos;
  if (tid == 0) {
    s_err = 0;
    s_slot = 0;
    s_pos = 0;
    const uint32_t sm = smid();
    s_sm = (int32_t)sm;
    a.boot_smid[blockIdx.x] = (int32_t)sm;
    __threadfence();
    atomicAdd(a.boot_count, 1u);
    const uint64_t t0 = gtime();
    while (ld_acquire_gpu32(a.boot_count) < (uint32_t)a.grid) {
      if (gtime() - t0 > a.boot_timeout_ns) {
        s_err = LK_DERR_BOOT;
        break;
      }
    }
  }
  __syncthreads();
  /* Position of this CTA in the slot-major order of (slot, SM id): slot s of
   * an SM is the CTA with the s-th lowest block index among those that landed
   * on it, and every SM's slot 0 comes before any slot 1.  With one CTA per
   * SM this is the order of SM ids.  The whole CTA counts, over a copy of the
   * exchanged ids in shared memory (at most 2 x 152 of them). */
  if (!s_err) {
    int32_t* all = reinterpret_cast<int32_t*>(dsm);
    for (int j = (int)tid; j < a.grid; j += (int)blockDim.x) all[j] = __ldcg(a.boot_smid + j);
    __syncthreads();
    const int32_t my_sm = s_sm;
    int below = 0;
    for (int j = (int)tid; j < (int)blockIdx.x; j += (int)blockDim.x) below += all[j] == my_sm;
    if (below) atomicAdd(&s_slot, below);
    __syncthreads();
    const int my_slot = s_slot;
    if (!a.pin_smid) {
      int before = 0;
      for (int j = (int)tid; j < a.grid; j += (int)blockDim.x) {
        int sj = 0;
        for (int q = 0; q < j; ++q) sj += all[q] == all[j];
        before += (sj < my_slot) || (sj == my_slot && all[j] < my_sm);
      }
      if (before) atomicAdd(&s_pos, before);
    }
    __syncthreads();
  }
  if (tid == 0) {
    const int err = s_err;
    const uint32_t sm = (uint32_t)s_sm;
    int c = -1, rk = -1;
    if (!err) {
      int pos = -1;
      if (a.pin_smid) {
        /* slot s of an SM takes the (s+1)-th occurrence of its id in the list */
        int seen = 0;
        for (int i = 0; i < a.total; ++i)
          if (a.pin_smid[i] == (int32_t)sm && seen++ == s_slot) {
            pos = i;
            break;
          }
      } else {
        pos = s_pos < a.total ? s_pos : -1;
      }
      if (pos >= 0) {
        c = 0;
        while (a.cl_start[c + 1] <= pos) ++c;
        rk = pos - a.cl_start[c];
      }
    }
    s_cl = c;
    s_rank = rk;
    s_size = c >= 0 ? a.cl_start[c + 1] - a.cl_start[c] : 0;
    lk_cta_info* inf = a.info + blockIdx.x;
    st_relaxed_sys32(&inf->cluster, c);
    st_relaxed_sys32(&inf->rank, rk);
    st_relaxed_sys32(&inf->smid, (int32_t)sm);
    st_relaxed_sys32(&inf->slot, s_slot);
    if (err) {
      set_error(a, c, (uint32_t)err);
    } else if (rk == 0) {
      st_relaxed_sys(&a.cword[c].status, LK_ST_INIT);
    }
    for (uint32_t i = 0; i < LK_ALL_BARS; ++i) mbar_init(&s_bars[i], 1);
    fence_barrier_init();
    red_release_sys_add(&a.ctrl->booted, 1u);
  }
  __syncthreads();
  if (s_cl < 0 || s_err) return;

  const int c = s_cl, r = s_rank, S = s_size;
  const bool master = (r == 0);
  const bool relay = (a.flags & LK_KFLAG_DIRECT) == 0;
  const bool mailbox = (a.flags & LK_KFLAG_MAILBOX) != 0;   /* implies relay */
  lk_dcluster* dc = a.dcl + c;
  const lk_wire* ring = a.ring + (size_t)c * (a.ring_mask + 1);
  uint64_t* my_done = a.rdone + a.rd_off[c] + r;   /* this CTA's host-visible completion word */
  uint32_t phase = 0;
  int final_err = 0;
  uint64_t known_done = 0;   /* mailbox master: descriptors it completed */

  for (uint64_t k = 0;; ++k) {
    const uint32_t slot = (uint32_t)(k % LK_BCAST_DEPTH);
    /* ---- descriptor k+1: from the ring, or from the master's relay ------ */
    if (tid == 0) {
      int err = 0;
      lk_slot& dsc = s_desc;   /* written in place: no copy through local memory */
      const lk_wire* w = ring + (k & a.ring_mask);
      const uint64_t tag = lk_lap_tag(k, a.ring_log2);
      /* slot k mod D (relay copy, partials, histogram-clear word, arrival
       * counter) is free once descriptor k+1-D, its previous user, finished */
      const uint64_t need = k + 1 > LK_BCAST_DEPTH ? k + 1 - LK_BCAST_DEPTH : 0;
      s_slot_seen = 0;   /* shared, not local: the take functions write it through a pointer */
      if (master && mailbox) {
        err = take_from_mailbox(a, c, k, dsc);
        s_slot_seen = known_done;   /* the mailbox master completes each descriptor itself */
      } else if (!relay || master) {
        err = take_from_ring(a, w, tag, k + 1, dsc, &dc->slot_done[slot], &s_slot_seen);
      } else {
        err = take_from_relay(a, dc, &dc->relay[slot], k, dsc);
      }
      const uint64_t t_pick = gtime();   /* read now, stored below (the read is slow) */
      /* Who gates: the CTA that reads the ring or mailbox for the cluster --
       * the master, which relays descriptor k only once slot k mod D is free
       * (so a relayed member needs no check: the slot it reads was free when
       * the master wrote it), or, with LK_INIT_DIRECT, every CTA for itself
       * (EXIT uses no slot there). */
      const bool self_gate = relay ? master : (!err && dsc.cmd != LK_CMD_EXIT);
      if (!err && self_gate && need && s_slot_seen < need) {
        const int ww = wait_word(a, &dc->slot_done[slot], need, false);
        err = ww < 0 ? LK_DERR_STALL : ww;
      }
      /* a batch starts once every earlier descriptor of the cluster finished
       * (its ticket and combine state are then at rest): the latest user of
       * each slot */
      if (!err && self_gate && dsc.cmd == LK_CMD_WORK + LK_OP_BATCH) {
        for (uint64_t j = 1; j <= k && j <= LK_BCAST_DEPTH && !err; ++j) {
          const uint64_t q = k - j;
          const int ww = wait_word(a, &dc->slot_done[q % LK_BCAST_DEPTH], q + 1, false);
          err = ww < 0 ? LK_DERR_STALL : ww;
        }
      }
      /* a critical descriptor (lk_set_role) counts as running from here to
       * its last CTA's completion; yielding clusters read the count */
      if (!err && master && (dsc.flags & LK_DFLAG_CRITICAL) && dsc.cmd != LK_CMD_EXIT)
        red_relaxed_gpu_add_s32(a.crit_active, 1);
      if (relay && master) {
        if (!err) relay_publish(&dc->relay[slot], k, dsc);
        else st_release_gpu(&dc->gen, LK_GEN_STOP);
      }
      if (err) {
        if (err > 0) {
          set_error(a, c, (uint32_t)err);
          final_err = err;
        } else {
          final_err = LK_DERR_STALL;   /* master stopped; its reason is recorded */
        }
        s_exit = 1;
      } else {
        s_exit = (dsc.cmd == LK_CMD_EXIT);
      }
      s_err = 0;
      s_found = 0;
      s_last = 0;
      s_tpick = t_pick;
      s_tstart = gtime();
    }
    __syncthreads();
    if (s_exit) break;

    /* ---- run this CTA's share ------------------------------------------ */
    const lk_slot d = s_desc;
    const uint32_t op = d.cmd - LK_CMD_WORK;
    const int berr = (op == LK_OP_BATCH || op == LK_OP_SERVE)
                         ? run_units<MAXT, P>(a, d, c, r, dsm, s_bars, phase, s_red)
                         : run_body<MAXT, P>(d, r, S, dsm, s_bars, phase, s_red, &dc->partial[slot][r],
                                             HistSink{nullptr, &dc->hzero[slot], d.seq,
                                                      k > 0 && !mailbox ? &dc->slot_done[(k - 1) % LK_BCAST_DEPTH]
                                                                        : nullptr},
                                             cta_rate(d.aux, S), (d.flags & LK_DFLAG_YIELD) ? a.crit_active : nullptr,
                                             (a.flags & LK_KFLAG_GEMM_FFMA) == 0);
    if (berr && tid == 0) s_err = berr;
    __syncthreads();

    uint64_t t_end = 0, t_done = 0;
    if (tid == 0) t_end = gtime();
    if (mailbox) {
      /* ---- finish, one-deep mailbox: rank 0 gathers every rank's flag,
       * combines a sum, and answers THREAD_FINISHED ---------------------- */
      if (tid == 0 && S > 1) st_release_gpu(&dc->flag[r], k + 1);   /* orders this CTA's writes (after the barrier) */
      if (master) {
        if (S > 1) {
          const int gerr = gather_flags(a, dc->flag, S, k + 1, &s_found);
          if (gerr && (tid & 31) == 0) s_err = gerr;
        }
        __syncthreads();
        if (!s_err) {
          if (op == LK_OP_SUM_F32) combine_sum(d, dc->partial[slot], S);
          __syncthreads();
          if (tid == 0) {
            if (op == LK_OP_BATCH) a.bcl[c].ticket = 0;   /* every rank has left the claim loop */
            /* one system-scope fence orders every output write (this CTA's,
             * and the other ranks' through their flags) before the stores */
            fence_acq_rel_sys();
            asm volatile("st.relaxed.gpu.u64 [%0], %1;" ::"l"(&dc->slot_done[slot]), "l"(k + 1) : "memory");
            known_done = k + 1;
            st_relaxed_sys(&a.cword[c].status, LK_ST_FINISHED);   /* the host re-arms */
            if (d.flags & LK_DFLAG_CRITICAL) red_relaxed_gpu_add_s32(a.crit_active, -1);
            t_done = gtime();
          }
        }
      }
    } else {
      /* ---- finish, ring modes: every CTA publishes its own completion
       * word (the paper's per-SM from_GPU mailbox); the host takes the
       * minimum over the cluster's words, so nothing between the last CTA's
       * end and the host waits on another CTA.  A sum or batch needs one
       * CTA to finish the descriptor's shared state first: each CTA arrives
       * on the slot's counter before publishing, and the last arriver
       * combines (the host's minimum includes its word, published after the
       * combine).  Other ops -- a histogram too: every CTA adds its counts
       * into the output itself -- arrive after publishing, off the host's
       * path; their arrivals only pick the CTA that frees the slot. */
      const bool comb = op == LK_OP_SUM_F32 || op == LK_OP_BATCH;
      if (comb) {
        if (tid == 0 && !s_err)
          s_last = S == 1 || atom_add_acq_rel_gpu(&dc->arrive[slot].count, 1u) == (uint32_t)(S - 1);
        __syncthreads();
        if (s_last) {   /* CTA-uniform after the barrier */
          if (op == LK_OP_SUM_F32) combine_sum(d, dc->partial[slot], S);
          __syncthreads();   /* the combine's writes before thread 0's fence */
        }
      }
      if (tid == 0 && !s_err) {
        /* every output write of this CTA (and of the combine, when this CTA
         * ran it; the barrier above orders the other threads' writes) before
         * the host-visible word */
        fence_acq_rel_sys();
        st_relaxed_sys(my_done, k + 1);
        if (!comb) s_last = S == 1 || atom_add_acq_rel_gpu(&dc->arrive[slot].count, 1u) == (uint32_t)(S - 1);
        if (s_last) {
          /* every CTA has arrived: free the slot (the arrivals, acquire-
           * release, order their reads of the relay slot and their partials
           * before this release) */
          if (S > 1) dc->arrive[slot].count = 0;
          if (op == LK_OP_BATCH) a.bcl[c].ticket = 0;   /* every CTA has left the claim loop */
          st_release_gpu(&dc->slot_done[slot], k + 1);
          if (d.flags & LK_DFLAG_CRITICAL) red_relaxed_gpu_add_s32(a.crit_active, -1);
          t_done = gtime();
        }
      }
    }
    if (tid == 0 && a.log) {
      lk_exec_rec* rec = a.log + (size_t)blockIdx.x * a.log_cap + (k % a.log_cap);
      rec->seq = d.seq;
      rec->cluster = (uint32_t)c;
      rec->rank = (uint32_t)r;
      rec->smid = smid();
      rec->op = op;
      rec->order = k;
      rec->t_pick_ns = s_tpick;
      rec->t_start_ns = s_tstart;
      rec->t_end_ns = t_end;
      rec->t_done_ns = t_done;
      a.log_count[blockIdx.x] = k + 1;
    }
    __syncthreads();
    if (s_err) {
      if (tid == 0) {
        set_error(a, c, (uint32_t)s_err);
        final_err = s_err;
        if (master && relay) st_release_gpu(&dc->gen, LK_GEN_STOP);
      }
      break;
    }
  }
  if (tid == 0) {
    if (master && mailbox) {
      /* completions the host has not consumed through FINISHED yet stay
       * visible after the status word below overwrites it */
      st_relaxed_sys(&a.cword[c].done, known_done);
      fence_acq_rel_sys();
    }
    if (master) st_relaxed_sys(&a.cword[c].status, final_err ? LK_ST_ERROR : LK_ST_EXITED);
    red_release_sys_add(&a.ctrl->exited, 1u);
  }
}

/* The persistent kernel (live contexts: lk_init). */
template <int MAXT, int P>
__global__ void __launch_bounds__(MAXT, P) lk_persistent(const lk_kargs a) {
  persistent_main<MAXT, P>(a);
}

/* The same kernel under another name for finite mode (lk_run_finite, 256
 * threads, one CTA per SM), so that a profiler can select its launches
 * apart from live contexts, which wait on the host and cannot be replayed. */
__global__ void __launch_bounds__(256, 1) lk_finite(const lk_kargs a) { persistent_main<256, 1>(a); }

/* ---- ordinary-launch baseline: the same bodies, one launch per item ------ */
struct lk_scratch {
  uint32_t counter;
  uint32_t pad[31];
  uint32_t hist[256];
  float partial[LK_MAX_CTAS];
};

template <int MAXT>
__global__ void __launch_bounds__(MAXT) lk_ordinary(const lk_slot d, lk_scratch* sc) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ float s_red[32];
  __shared__ __align__(8) uint64_t s_bars[LK_ALL_BARS];
  __shared__ int32_t s_last;
  const int r = blockIdx.x, S = gridDim.x;
  const uint32_t op = d.cmd - LK_CMD_WORK;
  if (op == LK_OP_NOP) return;
  /* the shared stage barriers and those of this block's warps, one per thread */
  if (threadIdx.x < LK_NUM_BARS + (blockDim.x >> 5) * LK_STAGES) {
    mbar_init(&s_bars[threadIdx.x], 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  run_body<MAXT, 1>(d, r, S, dsm, s_bars, phase, s_red, &sc->partial[r], HistSink{sc->hist, nullptr, 0, nullptr}, 0, nullptr);
  if (op != LK_OP_SUM_F32 && op != LK_OP_HIST_U8) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atom_add_acq_rel_gpu(&sc->counter, 1u) == (uint32_t)(S - 1);
  }
  __syncthreads();
  if (s_last) {
    if (op == LK_OP_SUM_F32) combine_sum(d, sc->partial, S);
    else combine_hist(d, sc->hist);
    __syncthreads();
    if (threadIdx.x == 0) sc->counter = 0;
  }
}

/* ---- host-mapped ping-pong (the dispatch floor) ------------------------- */
__global__ void lk_pingpong_kernel(const uint64_t* ping, uint64_t* pong, int iters, uint64_t abort_after_ns) {
  if (threadIdx.x != 0) return;
  for (int i = 1; i <= iters; ++i) {
    const uint64_t t0 = gtime();
    while (ld_acquire_sys(ping) != (uint64_t)i) {
      if (gtime() - t0 > abort_after_ns) {
        st_release_sys(pong, ~0ull);
        return;
      }
    }
    st_release_sys(pong, (uint64_t)i);
  }
}

/* ======================================================================= */
/* host side: CUDA backend                                                  */
/* ======================================================================= */
namespace {

std::once_flag g_preload_once;
cudaError_t g_preload_err = cudaSuccess;

/* Load every kernel of this library up front: with lazy module loading, a
 * first launch while a persistent kernel holds the SMs could wait on it. */
void preload_all() {
  std::call_once(g_preload_once, [] {
    cudaFuncAttributes fa;
    const void* fns[] = {(const void*)lk_persistent<256, 1>,  (const void*)lk_persistent<512, 1>,
                         (const void*)lk_persistent<1024, 1>, (const void*)lk_persistent<256, 2>,
                         (const void*)lk_finite,
                         (const void*)lk_ordinary<256>,
                         (const void*)lk_ordinary<512>,    (const void*)lk_ordinary<1024>,
                         (const void*)lk_pingpong_kernel};
    for (const void* f : fns) {
      cudaError_t e = cudaFuncGetAttributes(&fa, f);
      if (e != cudaSuccess && g_preload_err == cudaSuccess) g_preload_err = e;
    }
    /* ordinary launches of the histogram / GEMM bodies take 64 KB of shared memory */
    const void* ord[] = {(const void*)lk_ordinary<256>, (const void*)lk_ordinary<512>, (const void*)lk_ordinary<1024>};
    for (int i = 0; i < 3; ++i) {
      cudaError_t e = cudaFuncSetAttribute(ord[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)lk::body_smem_bytes(1));
      if (e != cudaSuccess && g_preload_err == cudaSuccess) g_preload_err = e;
    }
  });
}

const void* persistent_fn(int threads, int per_sm, bool finite) {
  if (finite && per_sm == 1 && threads <= 256) return (const void*)lk_finite;
  if (per_sm == 2) return threads <= 256 ? (const void*)lk_persistent<256, 2> : nullptr;
  if (threads <= 256) return (const void*)lk_persistent<256, 1>;
  if (threads <= 512) return (const void*)lk_persistent<512, 1>;
  return (const void*)lk_persistent<1024, 1>;
}

/* Allocations are recycled, never returned to the driver while the process
 * runs: cudaFree / cudaFreeHost may wait for the whole device, which would
 * stall behind any other persistent kernel that is still resident. */
struct Block {
  void* host;
  void* dev;
  size_t bytes;
  int device;
  bool mapped;
};
std::mutex g_pool_mu;
std::vector<Block> g_free;
std::vector<Block> g_used;

cudaStream_t copy_stream(int device) {
  static std::mutex mu;
  static std::vector<cudaStream_t> streams;
  std::lock_guard<std::mutex> g(mu);
  if ((int)streams.size() <= device) streams.resize(device + 1, nullptr);
  if (!streams[device]) {
    cudaSetDevice(device);
    cudaStreamCreateWithFlags(&streams[device], cudaStreamNonBlocking);
  }
  return streams[device];
}

int take_block(int device, size_t bytes, bool mapped, Block* out) {
  std::lock_guard<std::mutex> g(g_pool_mu);
  size_t best = (size_t)-1;
  for (size_t i = 0; i < g_free.size(); ++i) {
    const Block& b = g_free[i];
    if (b.device == device && b.mapped == mapped && b.bytes >= bytes && b.bytes <= 2 * bytes + (1 << 20) &&
        (best == (size_t)-1 || b.bytes < g_free[best].bytes))
      best = i;
  }
  if (best != (size_t)-1) {
    *out = g_free[best];
    g_free.erase(g_free.begin() + best);
    g_used.push_back(*out);
    return LK_OK;
  }
  Block b{nullptr, nullptr, bytes, device, mapped};
  if (cudaSetDevice(device) != cudaSuccess) return LK_EDEVICE;
  if (mapped) {
    if (cudaHostAlloc(&b.host, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) return LK_ENOMEM;
    if (cudaHostGetDevicePointer(&b.dev, b.host, 0) != cudaSuccess) return LK_EDEVICE;
  } else {
    if (cudaMalloc(&b.dev, bytes) != cudaSuccess) return LK_ENOMEM;
  }
  g_used.push_back(b);
  *out = b;
  return LK_OK;
}

void give_back(void* key, bool mapped) {
  std::lock_guard<std::mutex> g(g_pool_mu);
  for (size_t i = 0; i < g_used.size(); ++i) {
    void* k = mapped ? g_used[i].host : g_used[i].dev;
    if (k == key) {
      g_free.push_back(g_used[i]);
      g_used.erase(g_used.begin() + i);
      return;
    }
  }
}

int zero_device(int device, void* dev, size_t bytes) {
  /* a host->device copy of zeros runs on a copy engine, not on the SMs */
  static std::vector<char> zeros;
  static std::mutex mu;
  std::lock_guard<std::mutex> g(mu);
  const size_t chunk = 4u << 20;
  if (zeros.size() < chunk) zeros.assign(chunk, 0);
  cudaStream_t s = copy_stream(device);
  for (size_t off = 0; off < bytes; off += chunk) {
    size_t nb = std::min(chunk, bytes - off);
    if (cudaMemcpyAsync((char*)dev + off, zeros.data(), nb, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return LK_EDEVICE;
  }
  return cudaStreamSynchronize(s) == cudaSuccess ? LK_OK : LK_EDEVICE;
}

}  // namespace

struct lkb_launch {
  int device;
  cudaStream_t s;
  cudaEvent_t e0, e1;
};

int lkb_props_get(int device, lkb_props* out) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return LK_EDEVICE;
  out->sm_count = p.multiProcessorCount;
  out->smem_per_sm = p.sharedMemPerMultiprocessor;
  out->smem_per_block_optin = p.sharedMemPerBlockOptin;
  out->max_threads_per_sm = p.maxThreadsPerMultiProcessor;
  out->can_map_host = p.canMapHostMemory;
  out->cooperative = p.cooperativeLaunch;
  return LK_OK;
}

int lkb_alloc_mapped(int device, size_t bytes, void** host, void** dev) {
  Block b;
  int rc = take_block(device, bytes, true, &b);
  if (rc != LK_OK) return rc;
  memset(b.host, 0, bytes);
  *host = b.host;
  *dev = b.dev;
  return LK_OK;
}
void lkb_free_mapped(void* host) { give_back(host, true); }

int lkb_alloc_device(int device, size_t bytes, void** dev) {
  Block b;
  int rc = take_block(device, bytes, false, &b);
  if (rc != LK_OK) return rc;
  *dev = b.dev;
  return LK_OK;
}
void lkb_free_device(void* dev) { give_back(dev, false); }

int lkb_zero_device(int device, void* dev, size_t bytes) { return zero_device(device, dev, bytes); }

int lkb_copy_h2d(int device, void* dst, const void* src, size_t bytes) {
  cudaStream_t s = copy_stream(device);
  if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return LK_EDEVICE;
  return cudaStreamSynchronize(s) == cudaSuccess ? LK_OK : LK_EDEVICE;
}
int lkb_copy_d2h(int device, void* dst, const void* src, size_t bytes) {
  cudaStream_t s = copy_stream(device);
  if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return LK_EDEVICE;
  return cudaStreamSynchronize(s) == cudaSuccess ? LK_OK : LK_EDEVICE;
}

int lkb_stream_create(int device, void** stream) {
  if (cudaSetDevice(device) != cudaSuccess) return LK_EDEVICE;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LK_EDEVICE;
  *stream = (void*)s;
  return LK_OK;
}
int lkb_memcpy_async(void* stream, void* dst, const void* src, size_t bytes, int host_to_device) {
  return cudaMemcpyAsync(dst, src, bytes, host_to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                         (cudaStream_t)stream) == cudaSuccess
             ? LK_OK
             : LK_EDEVICE;
}
int lkb_stream_sync(void* stream) {
  return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? LK_OK : LK_EDEVICE;
}
void lkb_stream_destroy(void* stream) {
  if (stream) cudaStreamDestroy((cudaStream_t)stream);
}

int lkb_launch_kernel(int device, const lk_kargs* a, int threads, lkb_launch** out) {
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return LK_EDEVICE;
  preload_all();
  if (g_preload_err != cudaSuccess) return LK_EDEVICE;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return LK_EDEVICE;
  const int want = a->ctas_per_sm == 2 ? 2 : 1;
  const void* fn = persistent_fn(threads, want, (a->flags & LK_KFLAG_FINITE) != 0);
  if (!fn) return LK_EINVAL;
  /* exactly `want` CTAs per SM: ask for more than 1/(want+1) of the SM's
   * shared memory (one CTA: more than half; two: more than a third) */
  size_t dyn = std::max<size_t>(lk::body_smem_bytes(want), p.sharedMemPerMultiprocessor / (want + 1) + 1);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
    return LK_EDEVICE;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, dyn) != cudaSuccess) return LK_EDEVICE;
  if (per_sm != want || a->grid > want * p.multiProcessorCount) return LK_EDEVICE;
  lkb_launch* l = new lkb_launch{device, nullptr, nullptr, nullptr};
  if (cudaStreamCreateWithFlags(&l->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&l->e0) != cudaSuccess || cudaEventCreate(&l->e1) != cudaSuccess) {
    lkb_release(l);
    return LK_EDEVICE;
  }
  lk_kargs args = *a;
  void* params[] = {&args};
  cudaEventRecord(l->e0, l->s);
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(a->grid), dim3(threads), params, dyn, l->s);
  if (e != cudaSuccess) {
    if (getenv("LK_LOG")) fprintf(stderr, "lk: cooperative launch failed: %s\n", cudaGetErrorString(e));
    lkb_release(l);
    return LK_EDEVICE;
  }
  cudaEventRecord(l->e1, l->s);
  *out = l;
  return LK_OK;
}

int lkb_finished(lkb_launch* l) {
  if (!l) return 1;
  cudaError_t e = cudaEventQuery(l->e1);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return -1;
}

float lkb_elapsed_ms(lkb_launch* l) {
  float ms = -1.f;
  if (!l || cudaEventElapsedTime(&ms, l->e0, l->e1) != cudaSuccess) return -1.f;
  return ms;
}

void lkb_release(lkb_launch* l) {
  if (!l) return;
  if (l->e0) cudaEventDestroy(l->e0);
  if (l->e1) cudaEventDestroy(l->e1);
  if (l->s) cudaStreamDestroy(l->s);
  delete l;
}

/* ======================================================================= */
/* ordinary-launch baseline and ping-pong (C ABI)                           */
/* ======================================================================= */
namespace {
inline uint64_t now_ns() {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}
void pin_cpu(int cpu) {
  if (cpu < 0) return;
  int n = (int)std::thread::hardware_concurrency();
  if (n <= 0) return;
  cpu_set_t set;
  CPU_ZERO(&set);
  CPU_SET(cpu % n, &set);
  pthread_setaffinity_np(pthread_self(), sizeof set, &set);
}
cudaError_t launch_ordinary(const lk_slot& d, int grid, int threads, lk_scratch* sc, cudaStream_t s) {
  const uint32_t op = d.cmd - LK_CMD_WORK;
  const size_t smem = (op == LK_OP_NOP || op == LK_OP_SPIN) ? 0 : lk::body_smem_bytes(1);
  if (threads <= 256) lk_ordinary<256><<<grid, threads, smem, s>>>(d, sc);
  else if (threads <= 512) lk_ordinary<512><<<grid, threads, smem, s>>>(d, sc);
  else lk_ordinary<1024><<<grid, threads, smem, s>>>(d, sc);
  return cudaGetLastError();
}
}  // namespace

extern "C" int lk_baseline_run_trace(int device, const lk_trace_item* items, size_t count, int n_slots,
                                     const int* ctas_of_slot, int threads, int n_threads, int mode,
                                     int pin_cpu_base, lk_trace_result* res) {
  if ((count > 0 && (!items || !res)) || n_slots < 1 || !ctas_of_slot || n_threads < 1 || threads < 64 ||
      threads > 1024 || threads % 32)
    return LK_EINVAL;
  for (int s = 0; s < n_slots; ++s)
    if (ctas_of_slot[s] < 1 || ctas_of_slot[s] > LK_MAX_CTAS) return LK_EINVAL;
  for (size_t i = 0; i < count; ++i) {
    if (items[i].cluster < 0 || items[i].cluster >= n_slots || items[i].op >= LK_OP_COUNT) return LK_EINVAL;
    res[i] = lk_trace_result{0, 0, LK_PENDING, -1, 0, 0};
  }
  if (cudaSetDevice(device) != cudaSuccess) return LK_EDEVICE;
  preload_all();
  std::vector<cudaStream_t> st(n_slots, nullptr);
  std::vector<lk_scratch*> sc(n_slots, nullptr);
  int rc = LK_OK;
  for (int s = 0; s < n_slots && rc == LK_OK; ++s) {
    if (cudaStreamCreateWithFlags(&st[s], cudaStreamNonBlocking) != cudaSuccess) rc = LK_EDEVICE;
    else if (cudaMalloc(&sc[s], sizeof(lk_scratch)) != cudaSuccess) rc = LK_ENOMEM;
    else if (cudaMemsetAsync(sc[s], 0, sizeof(lk_scratch), st[s]) != cudaSuccess) rc = LK_EDEVICE;
    else if (cudaStreamSynchronize(st[s]) != cudaSuccess) rc = LK_EDEVICE;
  }
  if (rc == LK_OK) {
    std::vector<std::vector<size_t>> mine(n_threads);
    for (size_t i = 0; i < count; ++i) mine[items[i].cluster % n_threads].push_back(i);
    for (auto& v : mine)
      std::stable_sort(v.begin(), v.end(),
                       [&](size_t a, size_t b) { return items[a].t_arrival_ns < items[b].t_arrival_ns; });
    std::atomic<int> ready{0};
    std::atomic<uint64_t> start{0};
    std::atomic<int> err{0};
    auto worker = [&](int w) {
      pin_cpu(pin_cpu_base >= 0 ? pin_cpu_base + w : -1);
      cudaSetDevice(device);
      ready.fetch_add(1);
      uint64_t t0;
      while ((t0 = start.load(std::memory_order_acquire)) == 0) {
      }
      for (size_t i : mine[w]) {
        const lk_trace_item& it = items[i];
        while (now_ns() < t0 + it.t_arrival_ns) {
        }
        lk_slot d;
        memset(&d, 0, sizeof d);
        d.cmd = LK_CMD_WORK + it.op;
        d.n = it.n;
        d.in0 = (uint64_t)(uintptr_t)it.in0;
        d.in1 = (uint64_t)(uintptr_t)it.in1;
        d.out = (uint64_t)(uintptr_t)it.out;
        const int s = it.cluster;
        const bool e2e = mode == LK_TRACE_E2E;
        const uint64_t ts = now_ns();
        cudaError_t e = cudaSuccess;
        if (e2e) {
          if (it.in0_bytes && it.h_in0)
            e = cudaMemcpyAsync((void*)it.in0, it.h_in0, it.in0_bytes, cudaMemcpyHostToDevice, st[s]);
          if (e == cudaSuccess && it.in1_bytes && it.h_in1)
            e = cudaMemcpyAsync((void*)it.in1, it.h_in1, it.in1_bytes, cudaMemcpyHostToDevice, st[s]);
          if (e == cudaSuccess) e = cudaStreamSynchronize(st[s]);
        }
        const uint64_t tp = now_ns();
        if (e == cudaSuccess) e = launch_ordinary(d, ctas_of_slot[s], threads, sc[s], st[s]);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st[s]);
        const uint64_t to = now_ns();
        if (e == cudaSuccess && e2e && it.out_bytes && it.h_out) {
          e = cudaMemcpyAsync(it.h_out, it.out, it.out_bytes, cudaMemcpyDeviceToHost, st[s]);
          if (e == cudaSuccess) e = cudaStreamSynchronize(st[s]);
        }
        const uint64_t tc = now_ns();
        res[i].t_submit_ns = ts - t0;
        res[i].t_complete_ns = tc - t0;
        res[i].t_post_ns = tp - t0;
        res[i].t_observed_ns = to - t0;
        res[i].thread = w;
        res[i].status = e == cudaSuccess ? LK_OK : LK_EDEVICE;
        if (e != cudaSuccess) {
          int z = 0;
          err.compare_exchange_strong(z, LK_EDEVICE);
          return;
        }
      }
    };
    std::vector<std::thread> th;
    for (int w = 0; w < n_threads; ++w) th.emplace_back(worker, w);
    while (ready.load() < n_threads) std::this_thread::yield();
    start.store(now_ns(), std::memory_order_release);
    for (auto& x : th) x.join();
    rc = err.load();
  }
  for (int s = 0; s < n_slots; ++s) {
    if (st[s]) cudaStreamSynchronize(st[s]);
    if (sc[s]) cudaFree(sc[s]);
    if (st[s]) cudaStreamDestroy(st[s]);
  }
  return rc;
}

/* ---- the traditional life cycle of the compute-bound loop (Sec. III) ------ */
extern "C" int lk_baseline_phase_run(int device, int sms, int threads, uint64_t iters, int runs, void* out_dev,
                                     lk_phase_times* out) {
  if (sms < 1 || sms > LK_MAX_CTAS || runs < 1 || !out || threads < 64 || threads > 1024 || threads % 32 ||
      iters > 0xffffffffull)
    return LK_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return LK_EDEVICE;
  preload_all();
  if (g_preload_err != cudaSuccess) return LK_EDEVICE;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LK_EDEVICE;
  int rc = LK_OK;
  for (int r = 0; r < runs && rc == LK_OK; ++r) {
    void* buf = nullptr;
    const uint64_t t0 = now_ns();
    if (cudaMalloc(&buf, (size_t)sms * sizeof(uint32_t)) != cudaSuccess) { rc = LK_ENOMEM; break; }
    const uint64_t t1 = now_ns();
    lk_slot d;
    memset(&d, 0, sizeof d);
    d.cmd = LK_CMD_WORK + LK_OP_SPIN;
    d.n = iters;
    d.out = (uint64_t)(uintptr_t)(r == runs - 1 && out_dev ? out_dev : buf);
    cudaError_t e = launch_ordinary(d, sms, threads, nullptr, s);
    const uint64_t t2 = now_ns();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const uint64_t t3 = now_ns();
    if (cudaFree(buf) != cudaSuccess && e == cudaSuccess) e = cudaErrorUnknown;
    const uint64_t t4 = now_ns();
    if (e != cudaSuccess) rc = LK_EDEVICE;
    out[r] = lk_phase_times{t1 - t0, t2 - t1, t3 - t2, t4 - t3};
  }
  cudaStreamDestroy(s);
  return rc;
}

/* ---- a batch as one CUDA graph of ordinary launches ---------------------- */
extern "C" int lk_baseline_graph(int device, const lk_batch_item* items, uint32_t count, int max_ctas, int threads,
                                 int reps, float* ms) {
  if ((count > 0 && !items) || max_ctas < 1 || max_ctas > LK_MAX_CTAS || threads < 64 || threads > 1024 ||
      threads % 32 || reps < 1 || !ms)
    return LK_EINVAL;
  for (uint32_t i = 0; i < count; ++i) {
    const lk_batch_item& it = items[i];
    const lk_desc d{it.op, 0, it.n, 0};
    const int need = lk_op_inputs(it.op);
    if (need < 0 || lk_validate_desc(&d, it.in0, it.in1, need, it.out) != LK_OK) return LK_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) return LK_EDEVICE;
  preload_all();
  if (g_preload_err != cudaSuccess) return LK_EDEVICE;
  cudaStream_t s = nullptr;
  lk_scratch* sc = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = LK_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) rc = LK_EDEVICE;
  if (rc == LK_OK && cudaMalloc(&sc, sizeof(lk_scratch)) != cudaSuccess) rc = LK_ENOMEM;
  if (rc == LK_OK && (cudaMemsetAsync(sc, 0, sizeof(lk_scratch), s) != cudaSuccess ||
                      cudaStreamSynchronize(s) != cudaSuccess))
    rc = LK_EDEVICE;
  if (rc == LK_OK) {
    /* the kernels run one after another, so they can share one scratch block */
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = LK_EDEVICE;
    for (uint32_t i = 0; i < count && rc == LK_OK; ++i) {
      const lk_batch_item& it = items[i];
      if (it.op == LK_OP_NOP) continue;
      uint64_t in_bytes = it.op == LK_OP_ADD_I32 ? 8 * it.n
                          : it.op == LK_OP_HIST_U8 ? it.n
                          : it.op == LK_OP_GEMM64_F32 ? 32768 * it.n
                                                      : 4 * it.n;
      int grid = (int)std::min<uint64_t>((uint64_t)max_ctas, std::max<uint64_t>(1, (in_bytes + 262143) / 262144));
      lk_slot d;
      memset(&d, 0, sizeof d);
      d.cmd = LK_CMD_WORK + it.op;
      d.n = it.n;
      d.in0 = (uint64_t)(uintptr_t)it.in0;
      d.in1 = (uint64_t)(uintptr_t)it.in1;
      d.out = (uint64_t)(uintptr_t)it.out;
      if (launch_ordinary(d, grid, threads, sc, s) != cudaSuccess) rc = LK_EDEVICE;
    }
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc == LK_OK && e != cudaSuccess) rc = LK_EDEVICE;
    if (rc == LK_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = LK_EDEVICE;
  }
  for (int r = 0; r < reps && rc == LK_OK; ++r) {
    const uint64_t t0 = now_ns();
    if (cudaGraphLaunch(exec, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) rc = LK_EDEVICE;
    ms[r] = (float)((now_ns() - t0) / 1e6);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (sc) cudaFree(sc);
  if (s) cudaStreamDestroy(s);
  return rc;
}

/* ---- one ordinary launch that allocates nothing --------------------------
 * The sum and histogram bodies combine per-CTA results through a small
 * scratch block (arrival counter, 256 histogram bins, one partial per CTA).
 * lk_baseline_run_trace takes that block from cudaMalloc; this entry point
 * takes it from the file-scope array below instead, so it never allocates.
 * Capacity: one lk_scratch (5,248 bytes), i.e. at most LK_MAX_CTAS CTAs per
 * launch.  Every GPU that loads this library keeps the array until exit.
 * State between calls: lk_ordinary ignores a body's staging failure and still
 * counts every CTA's arrival, so a launch whose CTAs run always ends with
 * its last CTA re-zeroing the counter and bins; a refused launch never
 * touches the array. */
static __device__ __align__(256) lk_scratch g_noalloc_scratch;

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256];   /* device address of g_noalloc_scratch, per device */
}  // namespace

extern "C" int lk_launch_noalloc(int device, const lk_desc* d, const void* const* in, int n_in, void* out,
                                 int ctas, int threads, void* stream) {
  /* the descriptor checks of lk_submit (op, inputs, sizes, alignment, the
   * pointers each op dereferences), then this entry point's own limits */
  if (!d || device < 0 || device >= 256 || n_in < 0 || n_in > 2 || (n_in > 0 && !in)) return LK_EINVAL;
  const int vrc = lk_validate_desc(d, n_in > 0 ? in[0] : nullptr, n_in > 1 ? in[1] : nullptr, n_in, out);
  if (vrc != LK_OK) return vrc;
  if (ctas < 1 || ctas > LK_MAX_CTAS) return LK_EINVAL;   /* beyond the static scratch */
  if (threads < 64 || threads > 1024 || threads % 32) return LK_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return LK_EDEVICE;
  preload_all();
  if (g_preload_err != cudaSuccess) return LK_EDEVICE;
  void* scratch;
  {
    /* set-up, once per device, with that device current: the array's name is
     * only a host-side stand-in, so look up its device address */
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LK_EDEVICE;
      /* the array starts zeroed at module load and every launch's last CTA
       * returns the counter and bins to zero; clear once more here anyway */
      if (cudaMemsetAsync(p, 0, sizeof(lk_scratch), (cudaStream_t)stream) != cudaSuccess) return LK_EDEVICE;
      g_noalloc_ptr[device] = p;
    }
    scratch = g_noalloc_ptr[device];
  }
  lk_slot sl;
  memset(&sl, 0, sizeof sl);
  sl.cmd = LK_CMD_WORK + d->op;
  sl.n = d->n;
  sl.in0 = n_in > 0 ? (uint64_t)(uintptr_t)in[0] : 0;
  sl.in1 = n_in > 1 ? (uint64_t)(uintptr_t)in[1] : 0;
  sl.out = (uint64_t)(uintptr_t)out;
  return launch_ordinary(sl, ctas, threads, (lk_scratch*)scratch, (cudaStream_t)stream) == cudaSuccess
             ? LK_OK
             : LK_EDEVICE;
}

extern "C" int lk_bounds_violations(int device, uint64_t* count, uint32_t* first_site) {
#ifdef LK_DEBUG_BOUNDS
  if (!count || !first_site) return LK_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return LK_EDEVICE;
  unsigned long long c = 0;
  unsigned int s = 0;
  if (cudaMemcpyFromSymbol(&c, lk::g_lk_oob_count, sizeof c) != cudaSuccess ||
      cudaMemcpyFromSymbol(&s, lk::g_lk_oob_site, sizeof s) != cudaSuccess)
    return LK_EDEVICE;
  *count = c;
  *first_site = s;
  return LK_OK;
#else
  (void)device;
  (void)count;
  (void)first_site;
  return LK_EINVAL;   /* the product build checks no bounds */
#endif
}

extern "C" int lk_pingpong(int device, int iters, uint64_t* rtt_ns) {
  if (iters < 1 || !rtt_ns) return LK_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return LK_EDEVICE;
  preload_all();
  void *h = nullptr, *dptr = nullptr;
  int rc = lkb_alloc_mapped(device, 4096, &h, &dptr);
  if (rc != LK_OK) return rc;
  uint64_t* ping = (uint64_t*)h;
  uint64_t* pong = (uint64_t*)h + 16;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    lkb_free_mapped(h);
    return LK_EDEVICE;
  }
  lk_pingpong_kernel<<<1, 32, 0, s>>>((const uint64_t*)dptr, (uint64_t*)dptr + 16, iters, 2000000000ull);
  if (cudaGetLastError() != cudaSuccess) rc = LK_EDEVICE;
  for (int i = 1; i <= iters && rc == LK_OK; ++i) {
    const uint64_t t0 = now_ns();
    __atomic_store_n(ping, (uint64_t)i, __ATOMIC_RELEASE);
    for (;;) {
      const uint64_t x = __atomic_load_n(pong, __ATOMIC_ACQUIRE);
      if (x == (uint64_t)i) break;
      if (x == ~0ull || now_ns() - t0 > 3000000000ull) {
        rc = LK_ETIMEDOUT;
        break;
      }
    }
    rtt_ns[i - 1] = now_ns() - t0;
  }
  if (rc != LK_OK) __atomic_store_n(ping, ~0ull, __ATOMIC_RELEASE);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == LK_OK) rc = LK_EDEVICE;
  cudaStreamDestroy(s);
  lkb_free_mapped(h);
  return rc;
}
