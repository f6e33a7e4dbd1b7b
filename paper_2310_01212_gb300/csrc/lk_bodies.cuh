/*
 * lk_bodies.cuh -- the work a descriptor names (Sec. I: "a descriptor of the
 * work and a reference to the in/out data items"), split across the S CTAs
 * of a cluster.  CTA `r` of S takes a contiguous, 16-byte-aligned share of
 * the data; the split depends only on (n, S), so a result does not depend on
 * which descriptors ran before or beside it.
 *
 * Streaming bodies (add, copy, sum, histogram) move a CTA's share through
 * shared memory: thread 0 issues TMA bulk copies (cp.async.bulk, 16-byte
 * granules, completion counted on an mbarrier per stage) into a ring of
 * LK_STAGES stages, so up to three stages (96 KB) per SM are in flight while
 * every warp consumes the fourth; registers no longer bound the bytes in
 * flight.  One CTA barrier per chunk both releases the consumed stage for
 * refill and makes every thread agree on whether the stage arrived in time.
 *
 * Bodies:
 *   add_i32   out[i] = a[i] + b[i] mod 2^32: both inputs staged, 128-bit
 *             streaming stores of the sums
 *   copy_i32  out[i] = in[i]: staged in, then a bulk store straight from the
 *             stage (no registers touched)
 *   hist_u8   per-CTA counts -> cluster accumulator (global atomics) -> copied
 *             out by rank 0.  Small shares count into per-warp bins with
 *             shared atomics; large shares count into lane-private 32-bit
 *             counters, which no two lanes of a warp ever share, so random
 *             bytes cause no shared-memory bank conflicts; with one CTA per
 *             SM every warp streams its part through a ring of its own.
 *   sum_f32   per-thread float accumulators, warp shuffles, per-CTA partial;
 *             rank 0 adds the partials in rank order in binary64
 *   gemm64    64x64x64 float32 tiles staged into shared memory by TMA bulk
 *             copies.  Whole tiles (one CTA per SM, 256 threads): tcgen05
 *             tensor cores on split-bf16 operands.  Row blocks and other
 *             shapes: six 32 KB stages (three with two CTAs per SM), 4x4
 *             register micro-tiles, FFMA in k order
 * Used by the persistent kernel and by the ordinary-launch baseline kernels.
 */
#ifndef LK_BODIES_CUH
#define LK_BODIES_CUH
#include "lk_device.cuh"
#include "lk_layout.h"

namespace lk {

/* Contiguous share [beg, end) of `units` for rank r of S. */
__device__ __forceinline__ void share(uint64_t units, int r, int S, uint64_t& beg, uint64_t& end) {
  beg = units * (uint64_t)r / (uint64_t)S;
  end = units * (uint64_t)(r + 1) / (uint64_t)S;
}

__device__ __forceinline__ int4 add4(int4 x, int4 y) {
  return make_int4((int)((unsigned)x.x + (unsigned)y.x), (int)((unsigned)x.y + (unsigned)y.y),
                   (int)((unsigned)x.z + (unsigned)y.z), (int)((unsigned)x.w + (unsigned)y.w));
}

/* ---- shared-memory layout of a CTA ------------------------------------- */
/* With one CTA per SM (P = 1) the streaming bodies use 192 KB of the CTA's
 * 224 KB: a 64 KB work region (histogram counters) and a 128 KB ring of
 * LK_STAGES streaming stages; the FFMA GEMM's stages span those 192 KB and
 * the tensor-core GEMM uses all 224 KB (LK_TC_SMEM).  With two CTAs per SM
 * (P = 2) each CTA owns half of every region, so the bytes in flight per SM
 * stay the same. */
#define LK_SMEM_WORK (64u * 1024u)     /* histogram counters or GEMM stages   */
#define LK_SMEM_STREAM (128u * 1024u)  /* streaming stages                    */
#define LK_SMEM_DYN (LK_SMEM_WORK + LK_SMEM_STREAM)
#define LK_STAGES 4u
#define LK_GEMM_STAGE_FLOATS 8192u     /* one GEMM stage: A rows 16 KB + B tile 16 KB */
#define LK_HIST_COPIES 2u              /* lane-private counter copies (32 KB each), P = 1 */
#define LK_NUM_BARS 8u                 /* mbarriers: one per stage; the tensor-core GEMM's MMA completion in 4-7 */
#define LK_WARP_BARS (32u * LK_STAGES)  /* then one per stage of each warp's own ring (histogram) */
#define LK_ALL_BARS (LK_NUM_BARS + LK_WARP_BARS)

template <int P>
struct SmemCfg {
  static_assert(P == 1 || P == 2, "one or two CTAs per SM");
  static constexpr uint32_t work_bytes = LK_SMEM_WORK / P;
  static constexpr uint32_t stream_bytes = LK_SMEM_STREAM / P;
  static constexpr uint32_t dyn_bytes = work_bytes + stream_bytes;
  static constexpr uint32_t gemm_stages = dyn_bytes / (LK_GEMM_STAGE_FLOATS * 4u);   /* 6 or 3 */
  static constexpr uint32_t hist_copies = LK_HIST_COPIES / P;
  static_assert(gemm_stages <= LK_NUM_BARS, "one mbarrier per stage");
};

/* Time limits of one body.  Every staging wait ends by `deadline`.  A
 * non-zero `rate` (bytes per microsecond for this CTA) paces the TMA loads:
 * a token bucket as deep as the stage ring, so the first stages load at once
 * and each later one no earlier than its bytes allow; the deadline then
 * moves out by the paced duration of the CTA's share. */
struct Pace {
  uint64_t deadline;
  uint64_t rate;
  const int32_t* gate;   /* non-null: yield to critical descriptors (lk_set_role) */
};

/* Thread 0: sleep until `due` (%globaltimer ns); bounded by `due` itself. */
__device__ __forceinline__ void sleep_until(uint64_t due) {
  for (uint64_t now = gtime(); now < due; now = gtime()) {
    const uint64_t left = due - now;
    __nanosleep(left > 2000u ? 2000u : (uint32_t)left);
  }
}

/* Load yielding of one issuing thread (lk_set_role): before each refill of
 * a stage it holds while the count of running critical descriptors is
 * positive.  The count tested is the one loaded at the previous refill (the
 * load's round trip overlaps the stage wait in between, so a refill never
 * waits on L2 for it); one hold lasts at most LK_YIELD_HOLD_NS and a body's
 * holds together at most LK_YIELD_BUDGET_NS, by which its stage deadline is
 * extended.  The count is a hint: a stale value only shifts a hold by one
 * stage. */
#define LK_YIELD_HOLD_NS 1000000ull
#define LK_YIELD_BUDGET_NS 8000000ull
struct Yield {
  const int32_t* gate;
  int32_t seen;
  uint64_t end;
  __device__ __forceinline__ explicit Yield(const int32_t* g) : gate(g), seen(0), end(0) {
    if (gate) {
      end = gtime() + LK_YIELD_BUDGET_NS;
      seen = ld_relaxed_gpu_s32(gate);
    }
  }
  __device__ __forceinline__ void hold() {
    if (!gate) return;
    if (seen > 0) {
      uint64_t now = gtime();
      const uint64_t lim = now + LK_YIELD_HOLD_NS < end ? now + LK_YIELD_HOLD_NS : end;
      while (now < lim && ld_relaxed_gpu_s32(gate) > 0) {
        __nanosleep(256);
        now = gtime();
      }
    }
    seen = ld_relaxed_gpu_s32(gate);
  }
};

/* Stream the 16-byte vectors [beg, end) of NIN inputs through the stages.
 * consume(v0, nv, s0, s1) runs on every thread for each chunk: vectors
 * v0 .. v0+nv-1 of the share sit at s0[0..nv) (and s1[0..nv) for a second
 * input).  With STORE, consume issues bulk stores from the stage (thread 0)
 * and a stage is refilled only after those stores have read it.  `phase`
 * holds one parity bit per mbarrier and persists across descriptors.
 * Returns false, on every thread alike, if a stage did not arrive before
 * the deadline; this CTA's copies in flight are allowed to land first. */
template <int NIN, bool STORE, int P, class F>
__device__ __forceinline__ bool stream(const uint4* in0, const uint4* in1, uint64_t beg, uint64_t end,
                                       unsigned char* stage_mem, uint64_t* bars, uint32_t& phase, Pace pace,
                                       F&& consume) {
  constexpr uint32_t stage_vec = SmemCfg<P>::stream_bytes / LK_STAGES / NIN / 16u;   /* vectors per input per chunk */
  const uint64_t total = end > beg ? end - beg : 0;
  const uint64_t nch = (total + stage_vec - 1) / stage_vec;
  if (nch == 0) return true;
  constexpr uint64_t chunk_bytes = (uint64_t)stage_vec * 16u * NIN;
  const uint64_t deadline = (pace.rate ? pace.deadline + total * 16u * NIN * 1000u / pace.rate : pace.deadline) +
                            (pace.gate ? LK_YIELD_BUDGET_NS : 0u);
  const uint64_t t_first = pace.rate && threadIdx.x == 0 ? gtime() : 0;
  Yield yield(threadIdx.x == 0 ? pace.gate : nullptr);
  auto sbuf = [&](uint32_t st, int which) {
    return reinterpret_cast<uint4*>(stage_mem + ((size_t)st * NIN + which) * stage_vec * 16u);
  };
  auto issue = [&](uint64_t ch) {   /* thread 0 only */
    const uint32_t st = (uint32_t)(ch % LK_STAGES);
    const uint64_t v0 = beg + ch * stage_vec;
    const uint32_t nv = (uint32_t)((end - v0) < stage_vec ? (end - v0) : stage_vec);
    if (!LK_INB(v0 >= beg && v0 + nv <= end && ((uintptr_t)(in0 + v0) & 15u) == 0 &&
                    (NIN == 1 || ((uintptr_t)(in1 + v0) & 15u) == 0), LK_OOB_STREAM_LOAD) ||
        !LK_INB(((size_t)st * NIN + NIN) * stage_vec * 16u <= SmemCfg<P>::stream_bytes, LK_OOB_STREAM_SMEM)) {
      mbar_expect_tx(&bars[st], 0u);   /* skipped: the phase completes with no bytes */
      return;
    }
    mbar_expect_tx(&bars[st], nv * 16u * NIN);
    bulk_g2s(sbuf(st, 0), in0 + v0, nv * 16u, &bars[st]);
    if (NIN > 1) bulk_g2s(sbuf(st, 1), in1 + v0, nv * 16u, &bars[st]);
  };
  if (threadIdx.x == 0) {
    yield.hold();
    fence_proxy_async_global();   /* earlier generic writes before these async reads */
    fence_proxy_async_smem();     /* earlier generic shared accesses before async writes */
    for (uint64_t ch = 0; ch < nch && ch < LK_STAGES; ++ch) issue(ch);
  }
  for (uint64_t ch = 0; ch < nch; ++ch) {
    const uint32_t st = (uint32_t)(ch % LK_STAGES);
    const bool ok = mbar_wait(&bars[st], (phase >> st) & 1u, deadline);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        for (uint64_t c2 = ch; c2 < nch && c2 < ch + LK_STAGES; ++c2) {
          const uint32_t s2 = (uint32_t)(c2 % LK_STAGES);
          mbar_wait(&bars[s2], (phase >> s2) & 1u, deadline + 1000000000ull);
        }
        if (STORE) bulk_wait_all();
      }
      __syncthreads();
      return false;
    }
    phase ^= 1u << st;
    /* every thread has finished chunk ch-1: refill its stage */
    if (threadIdx.x == 0 && ch >= 1 && ch - 1 + LK_STAGES < nch) {
      if (pace.rate) sleep_until(t_first + ch * chunk_bytes * 1000u / pace.rate);
      yield.hold();
      if (STORE) bulk_wait_read_all();
      fence_proxy_async_smem();
      issue(ch - 1 + LK_STAGES);
    }
    const uint64_t v0 = beg + ch * stage_vec;
    const uint32_t nv = (uint32_t)((end - v0) < stage_vec ? (end - v0) : stage_vec);
    consume(v0, nv, sbuf(st, 0), NIN > 1 ? sbuf(st, 1) : nullptr);
  }
  __syncthreads();   /* every consumer is done before a later body reuses the stages */
  if (STORE && threadIdx.x == 0) {
    bulk_wait_all();
    fence_proxy_async_global();   /* the stores' writes before this thread's later release */
  }
  return true;
}

/* Shares of at most K vectors per thread skip the stage ring: every thread
 * issues all of its 128-bit loads at once and then consumes them -- one
 * global round trip, with no TMA issue, mbarrier wait or CTA barrier, which
 * on a share of a few tens of KB cost more than they hide.  f(i, v, x) gets
 * the thread's i-th vector, index v of the input.  Used by the add and sum
 * bodies of kernels with registers to spare (DIRECT: at most 256 threads,
 * one CTA per SM); elsewhere the extra live registers would spill. */
template <int K, class F>
__device__ __forceinline__ void direct(const uint4* in, uint64_t beg, uint64_t total, F&& f) {
  const uint32_t T = blockDim.x;
  uint4 q[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const uint64_t v = threadIdx.x + (uint64_t)i * T;
    if (v < total) q[i] = ld_stream(in + beg + v);
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const uint64_t v = threadIdx.x + (uint64_t)i * T;
    if (v < total) f(i, beg + v, q[i]);
  }
}
#define LK_DIRECT_ADD 4u     /* vectors per thread per input: add  */
#define LK_DIRECT_ONE 8u     /* vectors per thread: sum, histogram */

/* ---- int32 add / copy -------------------------------------------------- */
template <int P, bool DIRECT = false>
__device__ __forceinline__ bool body_add(const lk_slot& d, int r, int S, unsigned char* dsm, uint64_t* bars,
                                         uint32_t& phase, Pace pace) {
  const uint64_t n = d.n, nv = n >> 2;
  uint64_t beg, end;
  share(nv, r, S, beg, end);
  if (!LK_INB(beg <= end && end <= nv, LK_OOB_SHARE)) end = beg;
  int4* o = reinterpret_cast<int4*>(d.out);
  const uint32_t T = blockDim.x;
  bool ok = true;
  if (DIRECT && end - beg <= (uint64_t)LK_DIRECT_ADD * T) {
    const int4* a = reinterpret_cast<const int4*>(d.in0);
    const int4* b = reinterpret_cast<const int4*>(d.in1);
    int4 x[LK_DIRECT_ADD], y[LK_DIRECT_ADD];
#pragma unroll
    for (uint32_t i = 0; i < LK_DIRECT_ADD; ++i) {
      const uint64_t v = beg + threadIdx.x + (uint64_t)i * T;
      if (v < end) {
        x[i] = ld_stream(a + v);
        y[i] = ld_stream(b + v);
      }
    }
#pragma unroll
    for (uint32_t i = 0; i < LK_DIRECT_ADD; ++i) {
      const uint64_t v = beg + threadIdx.x + (uint64_t)i * T;
      if (v < end) st_stream(o + v, add4(x[i], y[i]));
    }
  } else {
    ok = stream<2, false, P>(reinterpret_cast<const uint4*>(d.in0), reinterpret_cast<const uint4*>(d.in1),
                             beg, end, dsm + SmemCfg<P>::work_bytes, bars, phase, pace,
                             [&](uint64_t v0, uint32_t cnt, const uint4* s0, const uint4* s1) {
                               const int4* a = reinterpret_cast<const int4*>(s0);
                               const int4* b = reinterpret_cast<const int4*>(s1);
                               for (uint32_t v = threadIdx.x; v < cnt; v += T)
                                 if (LK_INB(v0 + v < end, LK_OOB_STORE)) st_stream(o + v0 + v, add4(a[v], b[v]));
                             });
  }
  if (r == S - 1) {
    const int32_t* as = reinterpret_cast<const int32_t*>(d.in0);
    const int32_t* bs = reinterpret_cast<const int32_t*>(d.in1);
    int32_t* os = reinterpret_cast<int32_t*>(d.out);
    for (uint64_t j = nv * 4 + threadIdx.x; j < n; j += T) os[j] = (int32_t)((uint32_t)as[j] + (uint32_t)bs[j]);
  }
  return ok;
}

template <int P>
__device__ __forceinline__ bool body_copy(const lk_slot& d, int r, int S, unsigned char* dsm, uint64_t* bars,
                                          uint32_t& phase, Pace pace) {
  const uint64_t n = d.n, nv = n >> 2;
  uint64_t beg, end;
  share(nv, r, S, beg, end);
  if (!LK_INB(beg <= end && end <= nv, LK_OOB_SHARE)) end = beg;
  uint4* o = reinterpret_cast<uint4*>(d.out);
  const bool ok = stream<1, true, P>(reinterpret_cast<const uint4*>(d.in0), nullptr, beg, end, dsm + SmemCfg<P>::work_bytes, bars,
                                  phase, pace, [&](uint64_t v0, uint32_t cnt, const uint4* s0, const uint4*) {
                                    if (threadIdx.x == 0 && LK_INB(v0 + cnt <= end, LK_OOB_STORE)) {
                                      bulk_s2g(o + v0, s0, cnt * 16u);
                                      bulk_commit();
                                    }
                                  });
  if (r == S - 1) {
    const int32_t* as = reinterpret_cast<const int32_t*>(d.in0);
    int32_t* os = reinterpret_cast<int32_t*>(d.out);
    for (uint64_t j = nv * 4 + threadIdx.x; j < n; j += blockDim.x) os[j] = as[j];
  }
  return ok;
}

/* ---- float32 sum: this CTA's partial (valid in thread 0) ---------------- */
template <int P, bool DIRECT = false>
__device__ __forceinline__ bool body_sum(const lk_slot& d, int r, int S, unsigned char* dsm, uint64_t* bars,
                                         uint32_t& phase, Pace pace, float* red, float* partial_out) {
  const uint64_t n = d.n, nv = n >> 2;
  uint64_t beg, end;
  share(nv, r, S, beg, end);
  if (!LK_INB(beg <= end && end <= nv, LK_OOB_SHARE)) end = beg;
  const uint32_t T = blockDim.x;
  float acc0 = 0.f, acc1 = 0.f;
  bool ok = true;
  if (DIRECT && end - beg <= (uint64_t)LK_DIRECT_ONE * T) {
    /* the thread's vectors alternate between the two accumulators, as in
     * the staged loop below over a single chunk */
    direct<LK_DIRECT_ONE>(reinterpret_cast<const uint4*>(d.in0), beg, end - beg, [&](int i, uint64_t, uint4 q) {
      const float4 p = make_float4(__uint_as_float(q.x), __uint_as_float(q.y), __uint_as_float(q.z), __uint_as_float(q.w));
      if (i & 1) acc1 += (p.x + p.y) + (p.z + p.w);
      else acc0 += (p.x + p.y) + (p.z + p.w);
    });
  } else ok = stream<1, false, P>(reinterpret_cast<const uint4*>(d.in0), nullptr, beg, end, dsm + SmemCfg<P>::work_bytes,
                                   bars, phase, pace, [&](uint64_t, uint32_t cnt, const uint4* s0, const uint4*) {
                                     const float4* x = reinterpret_cast<const float4*>(s0);
                                     uint32_t v = threadIdx.x;
                                     for (; v + T < cnt; v += 2 * T) {
                                       const float4 p = x[v], q = x[v + T];
                                       acc0 += (p.x + p.y) + (p.z + p.w);
                                       acc1 += (q.x + q.y) + (q.z + q.w);
                                     }
                                     if (v < cnt) {
                                       const float4 p = x[v];
                                       acc0 += (p.x + p.y) + (p.z + p.w);
                                     }
                                   });
  if (r == S - 1) {
    const float* xs = reinterpret_cast<const float*>(d.in0);
    for (uint64_t j = nv * 4 + threadIdx.x; j < n; j += T) acc0 += xs[j];
  }
  float s = acc0 + acc1;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (uint32_t w = 0; w < T / 32; ++w) t += red[w];
    *partial_out = t;
  }
  return ok;
}

/* Rank 0: out[0] = partials added in rank order (binary64). */
__device__ __forceinline__ void combine_sum(const lk_slot& d, const float* partial, int S) {
  if (threadIdx.x >= 32) return;
  const uint32_t lane = threadIdx.x;
  double s = 0.0;
  for (int q = (int)lane; q < S; q += 32) s += (double)__ldcg(partial + q);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) *reinterpret_cast<float*>(d.out) = (float)s;
}

/* ---- uint8 histogram ---------------------------------------------------- */
/* Shares below this many bytes per CTA use per-warp bins, whose set-up and
 * read-out are cheap; larger shares use the conflict-free lane-private path
 * (measured crossover on GB300: a 28 KB share counts in 2.5 us lane-private
 * against 2.9 us in per-warp bins; a 7 KB share in 1.9 against 1.7 us). */
#define LK_HIST_SMALL_BYTES (16u * 1024u)
/* With one CTA per SM, shares from this many bytes per CTA stream through
 * one ring per warp (measured on GB300 over 152 CTAs: from 0.4 MB per CTA
 * 3-4 % faster at 256 threads and 14 % at 512; below 0.2 MB 1-4 % slower,
 * where the CTA's single ring needs fewer copies and waits). */
#define LK_HIST_WARP_BYTES (256u * 1024u)

__device__ __forceinline__ void count4_warp(uint32_t* bins, uint32_t w) {
  atomicAdd(&bins[w & 0xffu], 1u);
  atomicAdd(&bins[(w >> 8) & 0xffu], 1u);
  atomicAdd(&bins[(w >> 16) & 0xffu], 1u);
  atomicAdd(&bins[w >> 24], 1u);
}

/* Lane-private counters: word (v << 5) | lane of a copy (8192 words, 32 KB)
 * counts bin v for this lane alone, so lane l only touches bank l, and one
 * byte costs an extract, an address and one shared reduction.  32-bit
 * counters cannot overflow: a share holds fewer than 2^31 bytes. */
__device__ __forceinline__ void count4_lane(uint32_t lane_addr, uint32_t w) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint32_t v = (w >> (8 * b)) & 0xffu;
    asm volatile("red.relaxed.cta.shared::cta.add.u32 [%0], 1;" ::"r"(lane_addr + (v << 7)) : "memory");
  }
}

/* Thread v (< 256) adds bin v over the 32 lanes of every copy.  The loads of
 * a row start at thread-dependent columns, so each 8-thread phase of a
 * 128-bit warp load touches all 32 banks once. */
template <int P>
__device__ __forceinline__ uint32_t hist_readout(const uint32_t* sh, uint32_t v) {
  uint32_t tot = 0;
  for (uint32_t c = 0; c < SmemCfg<P>::hist_copies; ++c) {
    const uint4* rw = reinterpret_cast<const uint4*>(sh + c * 8192u + v * 32u);
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
      const uint4 q = rw[(j + v) & 7u];
      tot += (q.x + q.y) + (q.z + q.w);
    }
  }
  return tot;
}

__device__ __forceinline__ void hist_zero(uint32_t* sh, uint32_t words) {
  uint4* z = reinterpret_cast<uint4*>(sh);
  for (uint32_t i = threadIdx.x; i < words / 4; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
}

/* ---- histogram of a large share, one CTA per SM ------------------------- */
/* Counters: word 64 v + 32 c + lane counts bin v for one lane of copy c
 * (two copies, 64 KB).  A bin's row is 256 bytes, so the byte offset of
 * bin v is v << 8: one byte permute moves byte b of a loaded word into
 * bits 8..15, and an add of the lane's base makes the address.  Lane l
 * still touches only bank l.  The 16 bytes of one vector: every address is
 * formed before the first reduction, so the reductions issue back to back. */
__device__ __forceinline__ void count16_row(uint32_t lane_addr, uint4 q) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
  uint32_t a[16];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int b = 0; b < 4; ++b) a[4 * i + b] = lane_addr + __byte_perm(w[i], 0u, 0x4404u | ((uint32_t)b << 4));
#pragma unroll
  for (int j = 0; j < 16; ++j) asm volatile("red.relaxed.cta.shared::cta.add.u32 [%0], 1;" ::"r"(a[j]) : "memory");
}

/* Thread v (< 256) adds row v (both copies, 32 lanes each); each 8-thread
 * phase of the 128-bit loads starts at thread-dependent columns and so
 * touches all 32 banks once. */
__device__ __forceinline__ uint32_t hist_row_readout(const uint32_t* sh, uint32_t v) {
  const uint4* rw = reinterpret_cast<const uint4*>(sh + v * 64u);
  uint32_t tot = 0;
#pragma unroll
  for (uint32_t j = 0; j < 16; ++j) {
    const uint4 q = rw[(j + v) & 15u];
    tot += (q.x + q.y) + (q.z + q.w);
  }
  return tot;
}

/* Every warp streams its own contiguous part of the CTA's share [beg, end)
 * (16-byte vectors) through a private ring of LK_STAGES stages -- its slice
 * of the streaming region -- which its lane 0 fills with TMA bulk copies and
 * all its lanes await on the warp's own mbarriers (bars[LK_NUM_BARS + 4 w
 * + s], phase bits LK_NUM_BARS + s of `phase`, which every lane of the warp
 * keeps alike).  A warp never waits for another between chunks (with one
 * ring per CTA, warps stalled about a fifth of their cycles at the per-chunk
 * barrier: random bytes make their counting times uneven).  Returns false,
 * on every thread alike, if a stage did not arrive before the deadline. */
template <int P, bool YIELD>
__device__ __forceinline__ bool hist_warp_streams(const uint4* in, uint64_t beg, uint64_t end, unsigned char* dsm,
                                                  uint64_t* bars, uint32_t& phase, uint32_t lane_addr, Pace pace) {
  static_assert(P == 1, "the counter rows take the whole 64 KB work region of one CTA per SM");
  const uint32_t W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t stage_vec = SmemCfg<P>::stream_bytes / W / LK_STAGES / 16u;
  uint4* ring = reinterpret_cast<uint4*>(dsm + SmemCfg<P>::work_bytes) + (size_t)warp * LK_STAGES * stage_vec;
  uint64_t* wb = bars + LK_NUM_BARS + warp * LK_STAGES;
  uint64_t wbeg, wend;
  share(end - beg, (int)warp, (int)W, wbeg, wend);
  wbeg += beg;
  wend += beg;
  /* the warp's part, its ring slice and barriers, and the farthest counter
   * address any byte can form (row 255 of this lane and copy) */
  if (!LK_INB(wbeg <= wend && wend <= end, LK_OOB_SHARE) ||
      !LK_INB((size_t)(warp + 1) * LK_STAGES * stage_vec * 16u <= SmemCfg<P>::stream_bytes &&
                  LK_NUM_BARS + (warp + 1) * LK_STAGES <= LK_ALL_BARS, LK_OOB_STREAM_SMEM) ||
      !LK_INB(lane_addr - smem_addr(dsm) + 0xff00u + 4u <= SmemCfg<P>::work_bytes, LK_OOB_HIST_COUNTER))
    wend = wbeg;
  const uint64_t total = wend - wbeg;
  const uint64_t nch = (total + stage_vec - 1) / stage_vec;
  /* the warp's rate: the CTA's, split evenly over its warps */
  const uint64_t rate = pace.rate ? (pace.rate / W ? pace.rate / W : 1) : 0;
  const uint64_t deadline =
      (rate ? pace.deadline + total * 16u * 1000u / rate : pace.deadline) + (YIELD ? LK_YIELD_BUDGET_NS : 0u);
  const uint64_t t_first = rate && lane == 0 ? gtime() : 0;
  /* compiled apart from the plain loop: its state would cost the counting
   * loop registers */
  Yield yield(YIELD && lane == 0 && nch ? pace.gate : nullptr);
  auto parity = [&](uint64_t ch) {
    return ((phase >> (LK_NUM_BARS + (uint32_t)(ch % LK_STAGES))) & 1u) ^ ((uint32_t)(ch / LK_STAGES) & 1u);
  };
  auto issue = [&](uint64_t ch) {   /* lane 0 only */
    const uint32_t st = (uint32_t)(ch % LK_STAGES);
    const uint64_t v0 = wbeg + ch * stage_vec;
    const uint32_t nv = (uint32_t)((wend - v0) < stage_vec ? (wend - v0) : stage_vec);
    if (!LK_INB(v0 + nv <= wend && ((uintptr_t)(in + v0) & 15u) == 0, LK_OOB_STREAM_LOAD)) {
      mbar_expect_tx(&wb[st], 0u);   /* skipped: the phase completes with no bytes */
      return;
    }
    mbar_expect_tx(&wb[st], nv * 16u);
    bulk_g2s(ring + (size_t)st * stage_vec, in + v0, nv * 16u, &wb[st]);
  };
  if (lane == 0 && nch) {
    if (YIELD) yield.hold();
    fence_proxy_async_global();   /* earlier generic writes before these async reads */
    fence_proxy_async_smem();     /* earlier generic shared accesses before async writes */
    for (uint64_t ch = 0; ch < nch && ch < LK_STAGES; ++ch) issue(ch);
  }
  bool failed = false;
  uint64_t ch = 0;
  for (; ch < nch; ++ch) {
    const uint32_t st = (uint32_t)(ch % LK_STAGES);
    const bool ok = mbar_wait(&wb[st], parity(ch), deadline);
    if (!__all_sync(0xffffffffu, ok)) {
      failed = true;
      break;
    }
    const uint64_t v0 = wbeg + ch * stage_vec;
    const uint32_t cnt = (uint32_t)((wend - v0) < stage_vec ? (wend - v0) : stage_vec);
    const uint4* s0 = ring + (size_t)st * stage_vec;
    /* four vectors loaded before their 64 reductions: the reductions are
     * ordered asm, so loads placed after them would wait for them */
    uint32_t v = lane;
    for (; v + 96 < cnt; v += 128) {
      uint4 q[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) q[i] = s0[v + 32 * i];
#pragma unroll
      for (int i = 0; i < 4; ++i) count16_row(lane_addr, q[i]);
    }
    for (; v < cnt; v += 32) count16_row(lane_addr, s0[v]);
    __syncwarp();   /* every lane has read the stage before it is refilled */
    if (lane == 0 && ch + LK_STAGES < nch) {
      /* token bucket as deep as the ring: chunk k >= LK_STAGES no earlier
       * than t_first + (k - LK_STAGES + 1) chunks' worth of time */
      if (rate) sleep_until(t_first + (ch + 1) * (uint64_t)stage_vec * 16u * 1000u / rate);
      if (YIELD) yield.hold();
      fence_proxy_async_smem();
      issue(ch + LK_STAGES);
    }
  }
  /* a failed wait leaves the copies issued after it in flight: let them land */
  const uint64_t issued = failed ? (ch + LK_STAGES < nch ? ch + LK_STAGES : nch) : nch;
  if (lane == 0)
    for (uint64_t c2 = ch; failed && c2 < issued; ++c2)
      mbar_wait(&wb[c2 % LK_STAGES], parity(c2), deadline + 1000000000ull);
  /* each issued chunk completed one phase of its stage's barrier */
  for (uint32_t st = 0; st < LK_STAGES; ++st) {
    const uint64_t uses = issued > st ? (issued - st + LK_STAGES - 1) / LK_STAGES : 0;
    phase ^= (uint32_t)(uses & 1u) << (LK_NUM_BARS + st);
  }
  return !__syncthreads_or(failed);
}

/* Where a histogram's counts go.  With `zero` null, every CTA adds its
 * counts into `acc` (zero at rest) and a combine copies it out afterwards
 * (split parts, ordinary launches).  With `zero` set (a descriptor on a
 * cluster), rank 0 clears the output itself and release-stores `seq` into
 * *zero, and every CTA adds its counts straight into the output once it has
 * acquired that word: no combine, and no CTA waits for another at the end.
 * Rank 0 clears only once the cluster's previous descriptor has finished on
 * every CTA (*prev_done >= seq - 1; null when there is none, or the cluster
 * runs one descriptor at a time), so a CTA still writing the same buffer
 * for an earlier descriptor cannot land after the clear: the output ends as
 * the last descriptor's result, as if the descriptors ran one by one. */
struct HistSink {
  uint32_t* acc;
  uint64_t* zero;
  uint64_t seq;
  const uint64_t* prev_done;
};

/* Thread 0 waits for rank 0's cleared output (with a sink that has one),
 * then the whole CTA synchronises; false, on every thread, if the word did
 * not arrive by `deadline`. */
__device__ __forceinline__ bool hist_out_ready(const HistSink& sink, uint64_t deadline) {
  __shared__ int s_ready;
  if (threadIdx.x == 0) {
    int ready = 1;
    if (sink.zero)
      for (uint32_t it = 0; ld_acquire_gpu(sink.zero) < sink.seq; ++it)
        if ((it & 63u) == 63u && gtime() > deadline) {
          ready = 0;
          break;
        }
    s_ready = ready;
  }
  __syncthreads();
  return s_ready != 0;
}

template <int P>
__device__ __forceinline__ bool body_hist(const lk_slot& d, int r, int S, unsigned char* dsm, uint64_t* bars,
                                          uint32_t& phase, Pace pace, HistSink sink) {
  const uint64_t nv = d.n >> 4;
  uint64_t beg, end;
  share(nv, r, S, beg, end);
  if (!LK_INB(beg <= end && end <= nv, LK_OOB_SHARE)) end = beg;
  const bool tail = (r == S - 1) && (d.n & 15);
  const uint32_t T = blockDim.x, W = T / 32, lane = threadIdx.x & 31;
  uint32_t* sh = reinterpret_cast<uint32_t*>(dsm);
  const uint8_t* xb = reinterpret_cast<const uint8_t*>(d.in0);
  bool ok = true;
  const uint64_t total = end - beg;
  uint32_t* acc = sink.acc;
  if (sink.zero) {
    acc = reinterpret_cast<uint32_t*>(d.out);
    if (r == 0) {
      /* the counters' targets start at zero; the others add once they see it */
      if (sink.prev_done && !hist_out_ready(HistSink{nullptr, const_cast<uint64_t*>(sink.prev_done), sink.seq - 1,
                                                     nullptr},
                                            pace.deadline))
        return false;
      for (uint32_t v = threadIdx.x; v < 256; v += T) acc[v] = 0;
      __syncthreads();
      if (threadIdx.x == 0) st_release_gpu(sink.zero, sink.seq);
    }
  }
  if (total * 16 < LK_HIST_SMALL_BYTES) {
    hist_zero(sh, W * 256);
    __syncthreads();
    uint32_t* bins = sh + (threadIdx.x >> 5) * 256;
    ok = stream<1, false, P>(reinterpret_cast<const uint4*>(d.in0), nullptr, beg, end, dsm + SmemCfg<P>::work_bytes, bars, phase,
                          pace, [&](uint64_t, uint32_t cnt, const uint4* s0, const uint4*) {
                            for (uint32_t v = threadIdx.x; v < cnt; v += T) {
                              const uint4 q = s0[v];
                              count4_warp(bins, q.x);
                              count4_warp(bins, q.y);
                              count4_warp(bins, q.z);
                              count4_warp(bins, q.w);
                            }
                          });
    if (tail)
      for (uint64_t j = nv * 16 + threadIdx.x; j < d.n; j += T) atomicAdd(&bins[xb[j]], 1u);
    const bool ready = hist_out_ready(sink, pace.deadline);
    for (uint32_t v = threadIdx.x; ready && v < 256; v += T) {
      uint32_t s = 0;
      for (uint32_t w = 0; w < W; ++w) s += sh[w * 256 + v];
      if (s) atomicAdd(&acc[v], s);
    }
    return ok && ready;
  }
  if constexpr (P == 1) {
    if (total * 16 >= LK_HIST_WARP_BYTES) {
      /* large share, one CTA per SM: rows of 2 x 32 lane-private counters,
       * warps w and w + 2 share copy w % 2 (their reductions are atomic) */
      const uint32_t lane_addr = smem_addr(sh) + ((threadIdx.x >> 5) & 1u) * 128u + lane * 4u;
      hist_zero(sh, 256u * 64u);
      __syncthreads();
      ok = pace.gate ? hist_warp_streams<P, true>(reinterpret_cast<const uint4*>(d.in0), beg, end, dsm, bars, phase,
                                                  lane_addr, pace)
                     : hist_warp_streams<P, false>(reinterpret_cast<const uint4*>(d.in0), beg, end, dsm, bars, phase,
                                                   lane_addr, pace);
      if (tail)
        for (uint64_t j = nv * 16 + threadIdx.x; j < d.n; j += T)
          asm volatile("red.relaxed.cta.shared::cta.add.u32 [%0], 1;" ::"r"(lane_addr + ((uint32_t)xb[j] << 8))
                       : "memory");
      const bool ready = hist_out_ready(sink, pace.deadline);
      for (uint32_t v = threadIdx.x; ready && v < 256; v += T) {
        const uint32_t tot = hist_row_readout(sh, v);
        if (tot) atomicAdd(&acc[v], tot);
      }
      return ok && ready;
    }
  }
  /* medium share, or two CTAs per SM: one ring for the CTA; lane-private
   * 32-bit counters, one set per copy; the W / copies warps of a copy share
   * its words (their reductions to a word are atomic) */
  constexpr uint32_t copies = SmemCfg<P>::hist_copies;
  const uint32_t copy = (threadIdx.x >> 5) % copies;
  const uint32_t lane_addr = smem_addr(sh + copy * 8192u + lane);
  hist_zero(sh, copies * 8192u);
  __syncthreads();
  ok = stream<1, false, P>(reinterpret_cast<const uint4*>(d.in0), nullptr, beg, end, dsm + SmemCfg<P>::work_bytes, bars, phase,
                        pace, [&](uint64_t, uint32_t cnt, const uint4* s0, const uint4*) {
                          /* four vectors loaded before their 64 reductions: the
                           * reductions are ordered asm, so loads placed after
                           * them would wait for them */
                          uint32_t v = threadIdx.x;
                          for (; v + 3 * T < cnt; v += 4 * T) {
                            uint4 q[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) q[i] = s0[v + i * T];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                              count4_lane(lane_addr, q[i].x);
                              count4_lane(lane_addr, q[i].y);
                              count4_lane(lane_addr, q[i].z);
                              count4_lane(lane_addr, q[i].w);
                            }
                          }
                          for (; v < cnt; v += T) {
                            const uint4 q = s0[v];
                            count4_lane(lane_addr, q.x);
                            count4_lane(lane_addr, q.y);
                            count4_lane(lane_addr, q.z);
                            count4_lane(lane_addr, q.w);
                          }
                        });
  if (tail)
    for (uint64_t j = nv * 16 + threadIdx.x; j < d.n; j += T)
      asm volatile("red.relaxed.cta.shared::cta.add.u32 [%0], 1;" ::"r"(lane_addr + ((uint32_t)xb[j] << 7)) : "memory");
  const bool ready = hist_out_ready(sink, pace.deadline);
  for (uint32_t v = threadIdx.x; ready && v < 256; v += T) {
    const uint32_t tot = hist_readout<P>(sh, v);
    if (tot) atomicAdd(&acc[v], tot);
  }
  return ok && ready;
}

/* Rank 0: copy the accumulator out and return it to zero for reuse. */
__device__ __forceinline__ void combine_hist(const lk_slot& d, uint32_t* acc) {
  int32_t* out = reinterpret_cast<int32_t*>(d.out);
  for (uint32_t v = threadIdx.x; v < 256; v += blockDim.x) {
    out[v] = (int32_t)__ldcg(acc + v);
    acc[v] = 0;
  }
}

/* ---- the compute-bound loop (Sec. III) ----------------------------------- */
__device__ __forceinline__ void body_spin(const lk_slot& d, int r, uint32_t* red) {
  uint32_t x = 65536u * (uint32_t)r + threadIdx.x + 1u;
  /* eight dependent steps per trip: a one-step trip spends most of its time
   * on the 64-bit counter and the back edge, not on the multiply-add chain */
  const uint64_t n = d.n;
  uint64_t i = 0;
#pragma unroll 1
  for (; i + 8 <= n; i += 8) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x = 1664525u * x + 1013904223u;
  }
#pragma unroll 1
  for (; i < n; ++i) x = 1664525u * x + 1013904223u;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x ^= __shfl_xor_sync(0xffffffffu, x, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0 && d.out) {
    uint32_t v = 0;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) v ^= red[w];
    reinterpret_cast<uint32_t*>(d.out)[r] = v;
  }
}

/* ---- combining chunk results (rank 0 of the cluster alone) ------------- */
/* out[0] = binary64 sum of n float32 partials, one per 16-byte slot, added
 * lane-strided then by a fixed shuffle tree: the order depends only on n. */
__device__ __forceinline__ void body_combine_sum(const lk_slot& d, int r) {
  if (r != 0 || threadIdx.x >= 32) return;
  const float* p = reinterpret_cast<const float*>(d.in0);
  double s = 0.0;
  for (uint64_t q = threadIdx.x; q < d.n; q += 32) s += (double)__ldcg(p + 4 * q);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (threadIdx.x == 0) *reinterpret_cast<float*>(d.out) = (float)s;
}

/* out[v] = sum over j < n of in0[256 j + v]: n int32 histograms. */
__device__ __forceinline__ void body_combine_hist(const lk_slot& d, int r) {
  if (r != 0) return;
  const int32_t* h = reinterpret_cast<const int32_t*>(d.in0);
  for (uint32_t v = threadIdx.x; v < 256; v += blockDim.x) {
    uint32_t s = 0;
    for (uint64_t j = 0; j < d.n; ++j) s += (uint32_t)__ldcg(h + 256 * j + v);
    reinterpret_cast<int32_t*>(d.out)[v] = (int32_t)s;
  }
}

/* ---- 64x64x64 float32 GEMM tiles ---------------------------------------- */
/* Work unit = (tile, block of 64/U rows).  U > 1 only when there are fewer
 * tiles than CTAs, so that one tile can spread over up to 8 CTAs. */
__device__ __forceinline__ uint32_t gemm_row_split(uint64_t tiles, int S) {
  uint32_t U = 1;
  if (tiles > 0 && tiles < (uint64_t)S) {
    uint64_t want = ((uint64_t)S + tiles - 1) / tiles;
    while (U < want && U < 8) U <<= 1;
  }
  return U;
}

/* Shared memory: SmemCfg<P>::gemm_stages stages of (A rows 16 KB, B tile
 * 16 KB) over the whole dynamic shared memory; one mbarrier per stage. */

/* ---- the GEMM tile on the 5th-generation tensor cores ------------------- */
/* C = A B for whole 64x64x64 float32 tiles, with tcgen05.mma kind::f16 on
 * bf16 operands (exact products, float32 accumulation in TMEM).  One bf16
 * (or TF32) product per element pair would miss the 1e-4 sum|a b| bound, so
 * every operand is split in two: x_hi = bf16(x) and x_lo = bf16(x - x_hi),
 * both rounded to nearest; x - x_hi is exact in float32, and x_hi + x_lo
 * differs from x by at most 2^-16 |x|, so each product a b is formed to
 * within about 2^-15 |a b| (3.1e-5, against the 1e-4 bound; accumulation
 * adds at most 64 float32 roundings).  The A operand stacks A_hi (rows 0-63)
 * on A_lo (rows 64-127) and the B operand B_hi (columns 0-63) on B_lo
 * (64-127), so one chain of four MMAs over K (M = 128, N = 128, K = 16;
 * TMEM rows are lanes 0-127, one to one) yields all four products in a
 * 128 x 128 block D, and
 * C[r][n] = D[r][n] + D[r][n+64] + D[r+64][n] + D[r+64][n+64].
 * Two pipelines, one per half of the CTA (warps 0-3 and 4-7, each with its
 * own named barrier), take alternate tiles.  Each half has two buffers
 * (operands in shared memory, a 128 x 128 block in TMEM, an MMA-completion
 * mbarrier) and alternates between them: it splits tile k into buffer
 * k mod 2, hands it to the tensor core, and finishes tile k-1 (TMEM read-out,
 * row exchange, stores) while those MMAs run, so the tensor core's latency
 * hides behind the epilogue.  The TMA stage ring is shared: tile u sits in
 * stage (u - first) mod 3, and the half that split tile u refills that stage
 * with tile u+3.
 * Shared memory (224 KB): three 32 KB TMA stages of raw tiles (A rows, B) at
 * 0; four 32 KB buffers at 96 KB, two per half: the operands (A' then B',
 * 16 KB each, in the K-major core-matrix layout the descriptors name), then
 * the epilogue's row exchange once the MMAs have read them.  TMEM: all 512
 * columns (four blocks of 128), allocated for the body and freed on every
 * path out of it. */
#define LK_TC_SMEM (224u * 1024u)
#define LK_TC_STAGES 3u
#define LK_TC_MMA_BAR 4u             /* bars 4-7: MMA completion of (half, buffer) 2 h + b */
#define LK_TC_OPS (96u * 1024u)
/* instruction descriptor: D float32 (bits 4-5 = 1), A and B bf16 (bits 7-9,
 * 10-12 = 1), both K-major, N = 128 (bits 17-22 = N/8), M = 128 (bits 24-28 = M/16) */
#define LK_TC_IDESC ((1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24))

/* (x0, x1) -> bf16 pairs hi = bf16(x), lo = bf16(x - hi), x0 in the low half */
__device__ __forceinline__ void bf16_split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x1 - h1), "f"(x0 - h0));
}

/* Eight consecutive k of one operand row (x0: k..k+3, x1: k+4..k+7) -> one
 * 16-byte core-matrix row of hi parts and one of lo parts. */
__device__ __forceinline__ void bf16_split8(float4 x0, float4 x1, uint4& hi, uint4& lo) {
  bf16_split2(x0.x, x0.y, hi.x, lo.x);
  bf16_split2(x0.z, x0.w, hi.y, lo.y);
  bf16_split2(x1.x, x1.y, hi.z, lo.z);
  bf16_split2(x1.z, x1.w, hi.w, lo.w);
}

/* Column e of the 4x4 block q[0..3] (rows k..k+3): the K-chunk of output column n = 4 n4 + e. */
__device__ __forceinline__ float4 column_of(const float4* q, uint32_t e) {
  float4 v;
  v.x = e == 0 ? q[0].x : e == 1 ? q[0].y : e == 2 ? q[0].z : q[0].w;
  v.y = e == 0 ? q[1].x : e == 1 ? q[1].y : e == 2 ? q[1].z : q[1].w;
  v.z = e == 0 ? q[2].x : e == 1 ? q[2].y : e == 2 ? q[2].z : q[2].w;
  v.w = e == 0 ? q[3].x : e == 1 ? q[3].y : e == 2 ? q[3].z : q[3].w;
  return v;
}

/* The 128 threads of one half (local index t): split the staged raw tile
 * (A rows at `raw`, B at raw + 16 KB) into an operand buffer.  A core matrix
 * is 8 rows of 8 bf16 (16 bytes); the offset of (row i, K-chunk kc = k/8) is
 * (i/8) 1024 + kc 128 + (i%8) 16 bytes.  The thread-to-chunk maps make each
 * 8-thread phase of a 128-bit access touch eight distinct 16-byte bank
 * groups, on the raw side and on the operand side. */
__device__ __forceinline__ void tc_split(const unsigned char* raw, unsigned char* ops, uint32_t t) {
#pragma unroll
  for (uint32_t q = 0; q < 4; ++q) {                 /* A: 512 chunks of 8 k */
    const uint32_t c = t + 128u * q;
    const uint32_t j = c & 7u, s = (c >> 3) & 7u, ig = c >> 6;
    const uint32_t i = ig * 8u + j, kc = (j + s) & 7u, h = (kc >> 2) & 1u;
    const unsigned char* src = raw + i * 256u + kc * 32u;
    /* the half at 16 h first: distinct bank groups across the phase */
    const float4 xa = *reinterpret_cast<const float4*>(src + h * 16u);
    const float4 xb = *reinterpret_cast<const float4*>(src + (h ^ 1u) * 16u);
    uint4 hi, lo;
    bf16_split8(h ? xb : xa, h ? xa : xb, hi, lo);
    const uint32_t off = ig * 1024u + kc * 128u + j * 16u;
    *reinterpret_cast<uint4*>(ops + off) = hi;                         /* A_hi: rows 0-63 */
    *reinterpret_cast<uint4*>(ops + 8192u + off) = lo;                 /* A_lo: rows 64-127 */
  }
  {                                                  /* B: 128 blocks of 8 k x 4 n, transposed */
    const uint32_t n4 = t & 15u, kb = t >> 4;
    const unsigned char* rb = raw + 16384u;
    float4 v[8];
#pragma unroll
    for (uint32_t m = 0; m < 8; ++m) v[m] = *reinterpret_cast<const float4*>(rb + (8u * kb + m) * 256u + n4 * 16u);
#pragma unroll
    for (uint32_t te = 0; te < 4; ++te) {
      const uint32_t e = (te + (n4 >> 1)) & 3u;      /* rotated: distinct bank groups per phase */
      const uint32_t n = 4u * n4 + e;
      uint4 hi, lo;
      bf16_split8(column_of(v, e), column_of(v + 4, e), hi, lo);
      const uint32_t off = (n >> 3) * 1024u + kb * 128u + (n & 7u) * 16u;
      *reinterpret_cast<uint4*>(ops + 16384u + off) = hi;              /* B_hi: rows 0-63 */
      *reinterpret_cast<uint4*>(ops + 24576u + off) = lo;              /* B_lo: rows 64-127 */
    }
  }
}

/* Barrier of one half (named barrier 1 or 2, 128 threads); the _and form
 * also returns the AND of every participant's `v`, so that all 128 threads
 * take the same branch afterwards. */
__device__ __forceinline__ void half_sync(uint32_t h) { asm volatile("bar.sync %0, 128;" ::"r"(1u + h) : "memory"); }
__device__ __forceinline__ bool half_sync_and(uint32_t h, bool v) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, %2, 128, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)v), "r"(1u + h)
      : "memory");
  return out != 0;
}

__device__ __forceinline__ bool body_gemm_tc(const lk_slot& d, int r, int S, unsigned char* dsm, uint64_t* bars,
                                             uint32_t& phase, Pace pace) {
  uint64_t beg, end;
  share(d.n, r, S, beg, end);
  if (!LK_INB(end <= d.n, LK_OOB_SHARE)) end = beg;
  if (beg >= end) return true;
  const float* A = reinterpret_cast<const float*>(d.in0);
  const float* B = reinterpret_cast<const float*>(d.in1);
  float* C = reinterpret_cast<float*>(d.out);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t h = warp >> 2, lt = threadIdx.x & 127u;   /* half, index within it */
  const bool leader = lt == 0;
  const uint64_t tiles = end - beg;
  constexpr uint64_t unit_bytes = 32768u;
  const uint64_t deadline = pace.rate ? pace.deadline + tiles * unit_bytes * 1000u / pace.rate : pace.deadline;
  const uint64_t t_first = pace.rate ? gtime() : 0;
  auto issue = [&](uint64_t u) {   /* a half's leader, or thread 0 at the start */
    const uint32_t st = (uint32_t)((u - beg) % LK_TC_STAGES);
    unsigned char* sa = dsm + st * 32768u;
    fence_proxy_async_smem();
    if (!LK_INB(u >= beg && u < end, LK_OOB_GEMM_LOAD) || !LK_INB((st + 1) * 32768u <= LK_TC_OPS, LK_OOB_GEMM_SMEM)) {
      mbar_expect_tx(&bars[st], 0u);   /* skipped: the phase completes with no bytes */
      return;
    }
    mbar_expect_tx(&bars[st], 32768u);
    bulk_g2s(sa, A + u * 4096, 16384u, &bars[st]);
    bulk_g2s(sa + 16384u, B + u * 4096, 16384u, &bars[st]);
  };
  /* parity of a barrier's k-th completion in this body, from its bit at entry */
  const uint32_t phase0 = phase;
  auto parity = [&](uint32_t bar, uint64_t k) { return ((phase0 >> bar) & 1u) ^ (uint32_t)(k & 1u); };
  __shared__ uint32_t s_tmem;
  /* loads issued into each stage so far: a parity wait is only sound one
   * phase ahead, so a half waits for a stage's next load to be issued (by
   * the other half, once it consumed the stage's previous tile) before it
   * waits for that load's phase */
  __shared__ uint32_t s_issued[LK_TC_STAGES];
  __syncthreads();          /* every stage is free: the previous use ended with a barrier */
  if (warp == 0) tmem_alloc(&s_tmem, 512);
  if (threadIdx.x == 0) {
    for (uint32_t sb = 0; sb < LK_TC_STAGES; ++sb) s_issued[sb] = 0;
    for (uint64_t u = beg; u < end && u < beg + LK_TC_STAGES; ++u) {
      issue(u);
      s_issued[u - beg] = 1;
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  /* this half's two buffers b: TMEM block dt0 + 128 b, shared memory
   * ops0 + 32 KB b (operands, then the epilogue's row exchange) */
  const uint32_t dt0 = s_tmem + 256u * h;
  unsigned char* ops0 = dsm + LK_TC_OPS + h * 65536u;
  /* both halves' two buffers inside the shared memory and the 512 TMEM columns */
  const bool bufs_ok = LK_INB(LK_TC_OPS + (h + 1) * 65536u <= LK_TC_SMEM && 256u * (h + 1) <= 512u, LK_OOB_GEMM_SMEM);
  /* epilogue: warp quarter q holds D rows 32q..32q+31 (rows 64-127 are the
   * A_lo products of output rows 0-63) */
  const uint32_t quarter = warp & 3u;
  const uint32_t drow = 32u * quarter + lane;
  /* Tile u, the kk-th of this half, in buffer b = kk & 1: wait for its MMAs,
   * fold each row's column halves (B_hi and B_lo products) into the buffer,
   * rows 0-63 at `part`, rows 64-127 at part + 64 x 64 (16-byte chunk c of
   * row i at position c ^ (i & 7): no bank conflicts on either side), then
   * add the two parts and store the tile in coalesced 128-bit stores.
   * Returns false, on all 128 threads alike, if the MMAs did not complete
   * in time; on return the buffer and its TMEM block are free again. */
  auto epilogue = [&](uint64_t u, uint64_t kk) -> bool {
    const uint32_t b = (uint32_t)(kk & 1u), bar = LK_TC_MMA_BAR + 2u * h + b;
    float* part = reinterpret_cast<float*>(ops0 + 32768u * b);
    bool done = mbar_wait(&bars[bar], parity(bar, kk >> 1), deadline + 1000000000ull);
    if (done) {
      tc_fence_after_sync();
      float* prow = part + drow * 64u;
      const uint32_t sw = drow & 7u;
#pragma unroll
      for (uint32_t c0 = 0; c0 < 64; c0 += 32) {
        float v[32], w[32];
        tmem_ld32(dt0 + 128u * b + ((32u * quarter) << 16) + c0, v);
        tmem_ld32(dt0 + 128u * b + ((32u * quarter) << 16) + c0 + 64u, w);
#pragma unroll
        for (uint32_t c = 0; c < 32; c += 4)
          *reinterpret_cast<float4*>(prow + ((((c0 + c) >> 2) ^ sw) << 2)) =
              make_float4(v[c] + w[c], v[c + 1] + w[c + 1], v[c + 2] + w[c + 2], v[c + 3] + w[c + 3]);
      }
    }
    tc_fence_before_sync();         /* these TMEM reads precede this block's next MMAs */
    if (half_sync_and(h, done)) {
      float* ct = C + u * 4096;
#pragma unroll
      for (uint32_t q = 0; q < 8; ++q) {
        const uint32_t f = lt + 128u * q, i = f >> 4, c4 = f & 15u, pos = (c4 ^ (i & 7u)) << 2;
        const float4 x = *reinterpret_cast<const float4*>(part + i * 64u + pos);
        const float4 y = *reinterpret_cast<const float4*>(part + (i + 64u) * 64u + pos);
        if (LK_INB(u < end && i * 64u + c4 * 4u + 4u <= 4096u, LK_OOB_GEMM_STORE))
          st_stream(reinterpret_cast<float4*>(ct + i * 64u + c4 * 4u), make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w));
      }
    } else {
      done = false;
    }
    return half_sync_and(h, done);
  };
  bool ok = true;
  uint64_t k = 0;                  /* tiles this half has split and handed to the tensor core */
  for (uint64_t u = beg + h; u < end; u += 2, ++k) {
    const uint32_t st = (uint32_t)((u - beg) % LK_TC_STAGES);
    const uint64_t use = (u - beg) / LK_TC_STAGES;   /* completions of stage st before this one */
    const uint32_t b = (uint32_t)(k & 1u);
    bool go = true;
    if (leader) {
      const volatile uint32_t* iss = s_issued;
      for (uint32_t it = 0; iss[st] < use + 1; ++it)
        if ((it & 15) == 15 && gtime() > deadline) {
          go = false;
          break;
        }
      __threadfence_block();
      if (go) {
        go = mbar_wait(&bars[st], parity(st, use), deadline);
        if (!go) mbar_wait(&bars[st], parity(st, use), deadline + 1000000000ull);   /* let it land */
      }
    }
    if (!half_sync_and(h, go)) {
      ok = false;
      break;
    }
    mbar_wait(&bars[st], parity(st, use), deadline + 1000000000ull);   /* complete: visibility */
    unsigned char* ops = ops0 + 32768u * b;
    tc_split(dsm + st * 32768u, ops, lt);
    fence_proxy_async_smem();       /* the operands, written by threads, are read by the tensor core */
    tc_fence_before_sync();
    half_sync(h);
    if (leader) {
      /* this half has split tile u: its stage takes tile u+3 */
      if (u + LK_TC_STAGES < end) {
        if (pace.rate) sleep_until(t_first + (u + 1 - beg) * unit_bytes * 1000u / pace.rate);
        issue(u + LK_TC_STAGES);
        __threadfence_block();
        atomicAdd(&s_issued[st], 1u);
      }
      tc_fence_after_sync();
      const uint32_t ah = smem_addr(ops), bh = ah + 16384u;
      if (bufs_ok) {
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j)
          umma_f16(dt0 + 128u * b, umma_desc(ah + 256u * j, 128u, 1024u), umma_desc(bh + 256u * j, 128u, 1024u),
                   LK_TC_IDESC, j > 0);
      }
      umma_commit(&bars[LK_TC_MMA_BAR + 2u * h + b]);
    }
    /* while the tensor core works on tile u, finish the previous tile */
    if (k > 0 && !epilogue(u - 2, k - 1)) {
      ok = false;
      ++k;
      break;
    }
  }
  if (ok && k > 0 && !epilogue(beg + h + 2 * (k - 1), k - 1)) ok = false;
  /* MMAs of an unfinished tile may still be in flight: the last commit
   * covers every earlier MMA, so let it complete (bounded) before TMEM is
   * freed */
  if (!ok && leader && k > 0) {
    const uint32_t bar = LK_TC_MMA_BAR + 2u * h + (uint32_t)((k - 1) & 1u);
    mbar_wait(&bars[bar], parity(bar, (k - 1) >> 1), deadline + 2000000000ull);
  }
  tc_fence_before_sync();
  __syncthreads();          /* both halves done: stages and operand buffers are free */
  tc_fence_after_sync();
  if (warp == 0) tmem_dealloc(s_tmem, 512);
  /* every thread advances every barrier's phase bit by its completions here */
  if (ok) {
    for (uint32_t sb = 0; sb < LK_TC_STAGES; ++sb) {
      const uint64_t uses = tiles > sb ? (tiles - sb + LK_TC_STAGES - 1) / LK_TC_STAGES : 0;
      phase ^= (uint32_t)(uses & 1u) << sb;
    }
    for (uint32_t hh = 0; hh < 2; ++hh) {
      const uint64_t mine = tiles > hh ? (tiles - hh + 1) / 2 : 0;
      for (uint32_t bb = 0; bb < 2; ++bb) {
        const uint64_t commits = mine > bb ? (mine - bb + 1) / 2 : 0;
        phase ^= (uint32_t)(commits & 1u) << (LK_TC_MMA_BAR + 2u * hh + bb);
      }
    }
  }
  return ok;
}

/* FFMA micro-tiles of one row block: `rows` rows of A (row-major, 64 k
 * each) times the 64 x 64 B tile, both in shared memory, into C (row-major,
 * 64 floats a row).  Thread t takes micro-tiles of MR rows x MC columns, t
 * and t + T ...; every output accumulates its 64 products in k order with
 * one fused multiply-add each, whatever the micro-tile shape, so a tile's
 * result does not depend on how it was split into row blocks. */
template <int MR, int MC, bool FULL_UNROLL>
__device__ __forceinline__ void ffma_block(const float* sA, const float* sB, float* cblk, uint32_t rows, bool store_ok) {
  constexpr uint32_t ncg = 64u / MC;
  const uint32_t nmt = rows / MR * ncg;
  for (uint32_t mt = threadIdx.x; mt < nmt; mt += blockDim.x) {
    const uint32_t r0 = mt / ncg * MR, c0 = mt % ncg * MC;
    float c[MR][MC];
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int j = 0; j < MC; ++j) c[i][j] = 0.f;
#pragma unroll(FULL_UNROLL ? 16 : 2)
    for (uint32_t k = 0; k < 64; k += 4) {
      float av[MR][4], bv[4][MC];
#pragma unroll
      for (int i = 0; i < MR; ++i) {
        const float4 q = *reinterpret_cast<const float4*>(sA + (r0 + i) * 64 + k);
        av[i][0] = q.x; av[i][1] = q.y; av[i][2] = q.z; av[i][3] = q.w;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (MC == 4) {
          const float4 b = *reinterpret_cast<const float4*>(sB + (k + q) * 64 + c0);
          bv[q][0] = b.x; bv[q][1] = b.y; bv[q][MC > 2 ? 2 : 0] = b.z; bv[q][MC > 3 ? 3 : 0] = b.w;
        } else {
          const float2 b = *reinterpret_cast<const float2*>(sB + (k + q) * 64 + c0);
          bv[q][0] = b.x; bv[q][1] = b.y;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
          for (int j = 0; j < MC; ++j) c[i][j] = fmaf(av[i][q], bv[q][j], c[i][j]);
    }
    if (store_ok && LK_INB(r0 + MR <= rows && c0 + MC <= 64u, LK_OOB_GEMM_STORE)) {
#pragma unroll
      for (int i = 0; i < MR; ++i) {
        float* crow = cblk + (r0 + i) * 64 + c0;
        if (MC == 4) *reinterpret_cast<float4*>(crow) = make_float4(c[i][0], c[i][1], c[i][MC > 2 ? 2 : 0], c[i][MC > 3 ? 3 : 0]);
        else *reinterpret_cast<float2*>(crow) = make_float2(c[i][0], c[i][1]);
      }
    }
  }
}

/* Returns false if a staging copy did not complete before the deadline.
 * `phase` holds one parity bit per stage and persists across descriptors;
 * `pace` paces the tile loads as in stream().  Whole tiles at 256 threads
 * with one CTA per SM run on the tensor cores (body_gemm_tc) unless
 * `tensor_cores` is false; row blocks of split tiles and other shapes take
 * the FFMA path below. */
template <bool FULL_UNROLL, int P>
__device__ __forceinline__ bool body_gemm(const lk_slot& d, int r, int S, float* sm, uint64_t* bars,
                                          uint32_t& phase, Pace pace, bool tensor_cores) {
  const uint64_t tiles = d.n;
  const uint32_t U = gemm_row_split(tiles, S);
  /* FULL_UNROLL holds only in the kernels built for 256 threads and one CTA
   * per SM, the only ones that can take the tensor-core path */
  if constexpr (FULL_UNROLL)
    if (P == 1 && tensor_cores && U == 1 && blockDim.x == 256)
      return body_gemm_tc(d, r, S, reinterpret_cast<unsigned char*>(sm), bars, phase, pace);
  const uint32_t rows = 64 / U;
  uint64_t beg, end;
  share(tiles * U, r, S, beg, end);
  if (!LK_INB(end <= tiles * U, LK_OOB_SHARE)) end = beg;
  if (beg >= end) return true;
  const float* A = reinterpret_cast<const float*>(d.in0);
  const float* B = reinterpret_cast<const float*>(d.in1);
  float* C = reinterpret_cast<float*>(d.out);
  constexpr uint32_t nstages = SmemCfg<P>::gemm_stages;
  const uint64_t unit_bytes = rows * 256u + 16384u;
  const uint64_t deadline = pace.rate ? pace.deadline + (end - beg) * unit_bytes * 1000u / pace.rate : pace.deadline;
  const uint64_t t_first = pace.rate && threadIdx.x == 0 ? gtime() : 0;
  auto issue = [&](uint64_t u) {   /* thread 0 */
    const uint32_t st = (uint32_t)((u - beg) % nstages);
    const uint64_t tile = u / U;
    const uint32_t rb = (uint32_t)(u % U);
    float* sA = sm + st * LK_GEMM_STAGE_FLOATS;
    fence_proxy_async_smem();
    if (!LK_INB(tile < tiles && rb < U && (uint64_t)(rb + 1) * rows <= 64u, LK_OOB_GEMM_LOAD) ||
        !LK_INB((st + 1) * LK_GEMM_STAGE_FLOATS * 4u <= SmemCfg<P>::dyn_bytes, LK_OOB_GEMM_SMEM)) {
      mbar_expect_tx(&bars[st], 0u);   /* skipped: the phase completes with no bytes */
      return;
    }
    mbar_expect_tx(&bars[st], rows * 256u + 16384u);
    bulk_g2s(sA, A + tile * 4096 + (uint64_t)rb * rows * 64, rows * 256u, &bars[st]);
    bulk_g2s(sA + 4096, B + tile * 4096, 16384u, &bars[st]);
  };
  __shared__ int s_staged;
  __syncthreads();          /* every stage is free: the previous use ended with a barrier */
  if (threadIdx.x == 0)
    for (uint64_t u = beg; u < end && u < beg + nstages; ++u) issue(u);
  bool ok = true;
  for (uint64_t u = beg; u < end; ++u) {
    const uint32_t st = (uint32_t)((u - beg) % nstages);
    /* thread 0 alone decides whether the stage arrived in time, so that every
     * thread takes the same path through the barriers below */
    if (threadIdx.x == 0) {
      int arrived = mbar_wait(&bars[st], (phase >> st) & 1u, deadline);
      if (!arrived) {
        /* let this CTA's own copies land before giving up */
        for (uint64_t v = u; v < end && v < u + nstages; ++v) {
          const uint32_t s2 = (uint32_t)((v - beg) % nstages);
          mbar_wait(&bars[s2], (phase >> s2) & 1u, deadline + 1000000000ull);
        }
      }
      s_staged = arrived;
    }
    __syncthreads();
    if (!s_staged) {
      ok = false;
      break;
    }
    /* every thread finished unit u-1: refill its stage with unit u-1+STAGES */
    if (threadIdx.x == 0 && u > beg && u - 1 + nstages < end) {
      if (pace.rate) sleep_until(t_first + (u - beg) * unit_bytes * 1000u / pace.rate);
      issue(u - 1 + nstages);
    }
    /* the phase is complete: this wait returns at once and makes the copied
     * bytes visible to this thread */
    mbar_wait(&bars[st], (phase >> st) & 1u, deadline + 1000000000ull);
    phase ^= 1u << st;
    const float* sA = sm + st * LK_GEMM_STAGE_FLOATS;
    const float* sB = sA + 4096;
    const uint64_t tile = u / U;
    const uint32_t rb = (uint32_t)(u % U);
    float* cblk = C + tile * 4096 + (uint64_t)rb * rows * 64;
    const bool cblk_ok = LK_INB(tile < tiles && (uint64_t)(rb + 1) * rows <= 64u, LK_OOB_GEMM_STORE);
    /* every thread takes a micro-tile: the smaller the row block, the fewer
     * outputs each (a one-tile item split 8 ways keeps all threads busy) */
    if (rows >= 64) ffma_block<4, 4, FULL_UNROLL>(sA, sB, cblk, rows, cblk_ok);
    else if (rows >= 32) ffma_block<2, 4, FULL_UNROLL>(sA, sB, cblk, rows, cblk_ok);
    else if (rows >= 16) ffma_block<2, 2, FULL_UNROLL>(sA, sB, cblk, rows, cblk_ok);
    else ffma_block<1, 2, FULL_UNROLL>(sA, sB, cblk, rows, cblk_ok);
  }
  __syncthreads();          /* every stage is free for the next body */
  return ok;
}

/* Dynamic shared memory a CTA asks for when P CTAs share an SM. */
__host__ __device__ constexpr uint32_t body_smem_bytes(int P) { return P == 2 ? SmemCfg<2>::dyn_bytes : LK_TC_SMEM; }

}  // namespace lk
#endif
