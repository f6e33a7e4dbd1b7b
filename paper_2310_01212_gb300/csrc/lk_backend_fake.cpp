/*
 * lk_backend_fake.cpp -- a host-thread stand-in for the GPU (test build
 * liblk_fake.so only).
 *
 * It plays the device's side of the mailbox protocol over the same memory
 * layout as the persistent kernel: per cluster, one thread acquires ring
 * slots in FIFO order (or, with LK_INIT_MAILBOX, runs the one-deep four-phase
 * mailbox handshake), reports WORKING / FINISHED in the from_GPU words,
 * release-stores every rank's completion word (mailbox mode: `done`), writes
 * execution-log records for every rank, honours
 * EXIT, the abort word and the idle lease.  Work bodies are not run: this
 * backend exists to test the host runtime (tickets, ring-full refusals,
 * handles, waits, timeouts, dispose) on a machine without a GPU.
 *
 * Fault knobs (read at launch):
 *   LK_FAKE_SMS=n          SM count the fake device reports (default 16)
 *   LK_FAKE_STALL_US=t     each descriptor takes t microseconds
 *   LK_FAKE_DROP_AFTER=m   completions after the m-th are never published
 *   LK_FAKE_FAIL_AFTER=m   after m descriptors the cluster stops with LK_DERR_BADDESC
 *   LK_FAKE_FAIL_CODE=e    ... or with device error e instead (e.g. 7, LK_DERR_BOUNDS)
 *   LK_FAKE_NO_BOOT=1      the CTAs never report boot
 */
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "lk_backend.h"

namespace {

uint64_t now_ns() {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}
uint64_t env_u64(const char* k, uint64_t dflt) {
  const char* v = getenv(k);
  return v && *v ? strtoull(v, nullptr, 10) : dflt;
}
template <class T> T ld_acq(const T* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
template <class T> void st_rel(T* p, T v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }

int fake_sms() { return (int)env_u64("LK_FAKE_SMS", 16); }

}  // namespace

struct lkb_launch {
  std::vector<std::thread> threads;
  std::atomic<int> alive{0};
  uint64_t t0 = 0, t1 = 0;
};

int lkb_props_get(int device, lkb_props* out) {
  if (device != 0) return LK_EDEVICE;
  out->sm_count = fake_sms();
  out->smem_per_sm = 233472;
  out->smem_per_block_optin = 232448;
  out->max_threads_per_sm = 2048;
  out->can_map_host = 1;
  out->cooperative = 1;
  return LK_OK;
}

int lkb_alloc_mapped(int, size_t bytes, void** host, void** dev) {
  void* p = aligned_alloc(4096, (bytes + 4095) / 4096 * 4096);
  if (!p) return LK_ENOMEM;
  memset(p, 0, bytes);
  *host = *dev = p;
  return LK_OK;
}
void lkb_free_mapped(void* host) { free(host); }
int lkb_alloc_device(int, size_t bytes, void** dev) {
  void* p = aligned_alloc(4096, (bytes + 4095) / 4096 * 4096);
  if (!p) return LK_ENOMEM;
  *dev = p;
  return LK_OK;
}
void lkb_free_device(void* dev) { free(dev); }
int lkb_zero_device(int, void* dev, size_t bytes) {
  memset(dev, 0, bytes);
  return LK_OK;
}
int lkb_copy_h2d(int, void* dst, const void* src, size_t bytes) {
  memcpy(dst, src, bytes);
  return LK_OK;
}
int lkb_copy_d2h(int, void* dst, const void* src, size_t bytes) {
  memcpy(dst, src, bytes);
  return LK_OK;
}

int lkb_stream_create(int, void** stream) {
  *stream = (void*)1;
  return LK_OK;
}
int lkb_memcpy_async(void*, void* dst, const void* src, size_t bytes, int) {
  memcpy(dst, src, bytes);
  return LK_OK;
}
int lkb_stream_sync(void*) { return LK_OK; }
void lkb_stream_destroy(void*) {}

static void set_error(const lk_kargs& a, int c, uint32_t code) {
  uint32_t z = 0;
  __atomic_compare_exchange_n(&a.ctrl->first_error, &z, code, false, __ATOMIC_ACQ_REL, __ATOMIC_RELAXED);
  if (c >= 0) st_rel(&a.cword[c].error, (uint64_t)code);
}

/* One thread per cluster: the master's loop, with every rank's log record. */
static void cluster_loop(lk_kargs a, int c, std::vector<int> ctas, std::vector<int> smids, lkb_launch* l) {
  const uint64_t stall = env_u64("LK_FAKE_STALL_US", 0) * 1000ull;
  const uint64_t drop_after = env_u64("LK_FAKE_DROP_AFTER", ~0ull);
  const uint64_t fail_after = env_u64("LK_FAKE_FAIL_AFTER", ~0ull);
  const int fail_code = (int)env_u64("LK_FAKE_FAIL_CODE", LK_DERR_BADDESC);
  const lk_wire* ring = a.ring + (size_t)c * (a.ring_mask + 1);
  const bool mailbox = (a.flags & LK_KFLAG_MAILBOX) != 0;
  const int32_t rd_off = a.rd_off[c];   /* "device" memory is host memory here */
  uint64_t finished = 0;
  int err = 0;
  /* bounded wait for `ready` (abort, idle lease), as the kernel's waits */
  auto wait_for = [&](auto ready) {
    uint64_t hb = ld_acq(&a.ctrl->heartbeat);
    uint64_t t_last = now_ns();
    while (!ready()) {
      if (ld_acq(&a.ctrl->abort)) return (int)LK_DERR_ABORT;
      uint64_t t = now_ns();
      if (t - t_last > a.lease_ns) {
        uint64_t h = ld_acq(&a.ctrl->heartbeat);
        if (h == hb) return (int)LK_DERR_LEASE;
        hb = h;
        t_last = t;
      }
      std::this_thread::yield();
    }
    return 0;
  };
  /* LK_OP_SERVE: claim units from the queue's device counter until it
   * closes, as every CTA of the cluster does on the GPU (here one thread
   * claims for the cluster); no body runs, the last part of a request
   * appends it to the completion ring */
  auto serve = [&](lk_qstate* qs) {
    for (;;) {
      const uint64_t u = __atomic_fetch_add(&qs->head, 1ull, __ATOMIC_ACQ_REL);
      lk_qunit* e = qs->units + (u & qs->qmask);
      bool closed = false;
      const uint64_t tag = ((u >> qs->qlog2) + 1) & 0xffffull;
      uint64_t ew[6];
      int w = wait_for([&] {
        for (int i = 0; i < 6; ++i) ew[i] = __atomic_load_n(&e->w[i], __ATOMIC_RELAXED);
        bool cur = true;
        for (int i = 0; i < 6; ++i) cur = cur && (ew[i] >> LK_TAG_SHIFT) == tag;
        if (cur) {
          __atomic_thread_fence(__ATOMIC_ACQUIRE);
          return true;
        }
        const uint64_t cl = ld_acq(qs->close);
        if ((cl >> 63) && u >= (cl & ~(1ull << 63))) {
          closed = true;
          return true;
        }
        return false;
      });
      if (w) return w;
      if (closed) return 0;
      st_rel(&e->ack, u + 1);
      const uint32_t parts = (uint32_t)((ew[4] >> 16) & 0xffffu), rslot = (uint32_t)(ew[5] & 0xffffffffu);
      if (rslot >= qs->nslots || parts < 1) return (int)LK_DERR_BADDESC;
      if (stall) std::this_thread::sleep_for(std::chrono::nanoseconds(stall));
      lk_qslot* sl = qs->slots + rslot;
      const bool last = parts == 1 || __atomic_fetch_add(&sl->done, 1u, __ATOMIC_ACQ_REL) == parts - 1;
      if (last) {
        if (parts > 1) __atomic_store_n(&sl->done, 0u, __ATOMIC_RELAXED);
        const uint64_t pos = __atomic_fetch_add(&qs->cq_tail, 1ull, __ATOMIC_ACQ_REL);
        st_rel(&qs->cq[pos & qs->qmask], ((pos >> qs->qlog2) + 1) << 32 | rslot);
      }
    }
  };
  for (uint64_t k = 0;; ++k) {
    uint32_t cmd = 0;
    uint64_t in0 = 0;
    if (mailbox) {
      /* the one-deep mailbox: acknowledge the host's re-arm, then take work */
      lk_mbox* mb = a.mbox + c;
      if (k > 0) {
        err = wait_for([&] { return ld_acq(&mb->to_gpu) == (uint64_t)LK_CMD_NOP; });
        if (err) break;
        st_rel(&a.cword[c].status, (uint64_t)LK_ST_NOP);
      }
      uint64_t v = 0;
      err = wait_for([&] {
        v = ld_acq(&mb->to_gpu);
        return v == (uint64_t)LK_CMD_EXIT || v >= (uint64_t)LK_CMD_WORK;
      });
      if (err) break;
      cmd = (uint32_t)v;
    } else {
      const lk_wire* s = ring + (k & a.ring_mask);
      const uint64_t tag = lk_lap_tag(k, a.ring_log2);
      uint64_t w[6];
      err = wait_for([&] {
        for (int i = 0; i < 6; ++i) w[i] = __atomic_load_n(&s->w[i], __ATOMIC_RELAXED);
        for (int i = 0; i < 6; ++i)
          if ((w[i] >> LK_TAG_SHIFT) != tag) return false;
        __atomic_thread_fence(__ATOMIC_ACQUIRE);
        return true;
      });
      if (err) break;
      lk_slot dsc;
      lk_wire_decode(w, k + 1, &dsc);
      cmd = dsc.cmd;
      in0 = dsc.in0;
    }
    if (cmd == LK_CMD_EXIT) break;
    if (k >= fail_after) { err = fail_code; break; }
    if (cmd == LK_CMD_WORK + LK_OP_SERVE) {
      err = serve(reinterpret_cast<lk_qstate*>(in0));
      if (err) break;
    }
    const uint64_t t_pick = now_ns();
    st_rel(&a.cword[c].status, (uint64_t)LK_ST_WORKING);
    if (stall) std::this_thread::sleep_for(std::chrono::nanoseconds(stall));
    const uint64_t t_end = now_ns();
    if (a.log) {
      for (size_t r = 0; r < ctas.size(); ++r) {
        const int g = ctas[r];
        lk_exec_rec* rec = a.log + (size_t)g * a.log_cap + (k % a.log_cap);
        rec->seq = k + 1;
        rec->cluster = (uint32_t)c;
        rec->rank = (uint32_t)r;
        rec->smid = (uint32_t)smids[r];
        rec->op = cmd - LK_CMD_WORK;
        rec->order = k;
        rec->t_pick_ns = t_pick;
        rec->t_start_ns = t_pick;
        rec->t_end_ns = t_end;
        rec->t_done_ns = r + 1 == ctas.size() ? t_end : 0;
        a.log_count[g] = k + 1;
      }
    }
    if (k < drop_after) {
      finished = k + 1;
      /* ring modes: every rank publishes its own completion word */
      if (!mailbox)
        for (size_t r = 0; r < ctas.size(); ++r) st_rel(&a.rdone[rd_off + r], k + 1);
      st_rel(&a.cword[c].status, (uint64_t)LK_ST_FINISHED);
    }
  }
  if (mailbox) st_rel(&a.cword[c].done, finished);
  if (err) set_error(a, c, (uint32_t)err);
  st_rel(&a.cword[c].status, (uint64_t)(err ? LK_ST_ERROR : LK_ST_EXITED));
  __atomic_fetch_add(&a.ctrl->exited, (uint32_t)ctas.size(), __ATOMIC_ACQ_REL);
  l->alive.fetch_sub(1);
}

int lkb_launch_kernel(int, const lk_kargs* ap, int threads, lkb_launch** out) {
  if (threads < 64) return LK_EDEVICE;
  const lk_kargs a = *ap;
  lkb_launch* l = new lkb_launch();
  l->t0 = now_ns();
  const int sms = fake_sms();
  /* boot: CTA g lands on SM (5g + 3) mod sms (CTAs g and g + sms share an
   * SM); clusters from the slot-major order of (slot, SM id), as on the GPU */
  if (a.grid > (a.ctas_per_sm == 2 ? 2 : 1) * sms) return LK_EDEVICE;
  std::vector<int> host_start(a.num_clusters + 1);
  memcpy(host_start.data(), a.cl_start, sizeof(int) * (a.num_clusters + 1));
  std::vector<int> sm_of(a.grid), slot_of(a.grid, 0);
  for (int g = 0; g < a.grid; ++g) {
    sm_of[g] = (5 * g + 3) % sms;
    for (int q = 0; q < g; ++q) slot_of[g] += sm_of[q] == sm_of[g];
  }
  std::vector<int> order(a.grid);
  for (int g = 0; g < a.grid; ++g) order[g] = g;
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    return slot_of[x] != slot_of[y] ? slot_of[x] < slot_of[y] : sm_of[x] < sm_of[y];
  });
  std::vector<std::vector<int>> ctas(a.num_clusters), smids(a.num_clusters);
  for (int g = 0; g < a.grid; ++g) {
    int pos = -1;
    if (a.pin_smid) {
      int seen = 0;
      for (int i = 0; i < a.total && pos < 0; ++i)
        if (a.pin_smid[i] == sm_of[g] && seen++ == slot_of[g]) pos = i;
    } else {
      pos = (int)(std::find(order.begin(), order.end(), g) - order.begin());
    }
    int c = -1, r = -1;
    if (pos >= 0) {
      c = 0;
      while (host_start[c + 1] <= pos) ++c;
      r = pos - host_start[c];
    }
    a.info[g].cluster = c;
    a.info[g].rank = r;
    a.info[g].smid = sm_of[g];
    a.info[g].slot = slot_of[g];
  }
  for (int c = 0; c < a.num_clusters; ++c) {
    int size = host_start[c + 1] - host_start[c];
    ctas[c].assign(size, -1);
    smids[c].assign(size, -1);
  }
  for (int g = 0; g < a.grid; ++g)
    if (a.info[g].cluster >= 0) {
      ctas[a.info[g].cluster][a.info[g].rank] = g;
      smids[a.info[g].cluster][a.info[g].rank] = sm_of[g];
    }
  if (env_u64("LK_FAKE_NO_BOOT", 0)) {
    /* never boots: the "kernel" just waits for the abort word */
    l->alive.store(1);
    l->threads.emplace_back([a, l] {
      while (!ld_acq(&a.ctrl->abort)) std::this_thread::yield();
      l->alive.fetch_sub(1);
    });
    *out = l;
    return LK_OK;
  }
  for (int c = 0; c < a.num_clusters; ++c) st_rel(&a.cword[c].status, (uint64_t)LK_ST_INIT);
  __atomic_store_n(&a.ctrl->booted, (uint32_t)a.grid, __ATOMIC_RELEASE);
  l->alive.store(a.num_clusters);
  for (int c = 0; c < a.num_clusters; ++c) l->threads.emplace_back(cluster_loop, a, c, ctas[c], smids[c], l);
  *out = l;
  return LK_OK;
}

int lkb_finished(lkb_launch* l) {
  if (!l) return 1;
  if (l->alive.load() == 0) {
    if (!l->t1) l->t1 = now_ns();
    return 1;
  }
  return 0;
}

float lkb_elapsed_ms(lkb_launch* l) { return l && l->t1 ? (float)((l->t1 - l->t0) / 1e6) : -1.f; }

void lkb_release(lkb_launch* l) {
  if (!l) return;
  for (auto& t : l->threads)
    if (t.joinable()) t.join();
  delete l;
}

/* The ordinary-launch and ping-pong entry points need a GPU. */
extern "C" int lk_baseline_run_trace(int, const lk_trace_item*, size_t, int, const int*, int, int, int, int,
                                     lk_trace_result*) {
  return LK_EDEVICE;
}
extern "C" int lk_pingpong(int, int, uint64_t*) { return LK_EDEVICE; }
extern "C" int lk_bounds_violations(int, uint64_t*, uint32_t*) { return LK_EINVAL; }
extern "C" int lk_baseline_phase_run(int, int, int, uint64_t, int, void*, lk_phase_times*) { return LK_EDEVICE; }
extern "C" int lk_baseline_graph(int, const lk_batch_item*, uint32_t, int, int, int, float*) { return LK_EDEVICE; }
extern "C" int lk_launch_noalloc(int, const lk_desc*, const void* const*, int, void*, int, int, void*) {
  return LK_EDEVICE;
}
