/*
 * lk_bodies.cuh -- the work a descriptor names (Sec. I: "a descriptor of the
 * work and a reference to the in/out data items"), split across the S CTAs
 * of a cluster.  CTA `r` of S takes a contiguous, 16-byte-aligned share of
 * the data; the split depends only on (n, S), so a result does not depend on
 * which descriptors ran before or beside it.
 *
 * Bodies:
 *   add_i32   out[i] = a[i] + b[i] mod 2^32          (128-bit streaming loads)
 *   copy_i32  out[i] = in[i]
 *   hist_u8   per-CTA counts -> cluster accumulator (global atomics) -> copied
 *             out by the last CTA.  Small shares count into per-warp bins with
 *             shared atomics; large shares count into lane-private packed
 *             16-bit counters, which no two lanes of a warp ever share, so
 *             random bytes cause no shared-memory bank conflicts.
 *   sum_f32   per-thread float accumulators, warp shuffles, per-CTA partial;
 *             the last CTA adds the partials in rank order in binary64
 *   gemm64    64x64x64 float32 tiles staged into shared memory by TMA bulk
 *             copies (cp.async.bulk + mbarrier, two stages so the next tile
 *             loads while this one computes), 4x4 register micro-tiles, FFMA
 *             in k order
 * Every streaming loop issues all of a thread's loads for one round (U per
 * thread, predicated on the share's end) before using any of them, so a
 * share of any size costs one memory round trip per round.
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

/* ---- int32 add / copy -------------------------------------------------- */
template <int U, bool ADD>
__device__ __forceinline__ void body_add_copy(const lk_slot& d, int r, int S) {
  const uint64_t n = d.n;
  const int4* a = reinterpret_cast<const int4*>(d.in0);
  const int4* b = reinterpret_cast<const int4*>(d.in1);
  int4* o = reinterpret_cast<int4*>(d.out);
  const uint64_t nv = n >> 2;
  uint64_t beg, end;
  share(nv, r, S, beg, end);
  const uint32_t T = blockDim.x;
  for (uint64_t base = beg + threadIdx.x; base < end; base += (uint64_t)U * T) {
    int4 x[U], y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = base + (uint64_t)u * T;
      if (i < end) {
        x[u] = ld_stream(a + i);
        if (ADD) y[u] = ld_stream(b + i);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = base + (uint64_t)u * T;
      if (i < end) st_stream(o + i, ADD ? add4(x[u], y[u]) : x[u]);
    }
  }
  if (r == S - 1) {
    const int32_t* as = reinterpret_cast<const int32_t*>(d.in0);
    const int32_t* bs = reinterpret_cast<const int32_t*>(d.in1);
    int32_t* os = reinterpret_cast<int32_t*>(d.out);
    for (uint64_t j = nv * 4 + threadIdx.x; j < n; j += T)
      os[j] = ADD ? (int32_t)((uint32_t)as[j] + (uint32_t)bs[j]) : as[j];
  }
}

/* ---- float32 sum: this CTA's partial (valid in thread 0) ---------------- */
template <int U>
__device__ __forceinline__ float body_sum_partial(const lk_slot& d, int r, int S, float* red) {
  const uint64_t n = d.n;
  const float4* x = reinterpret_cast<const float4*>(d.in0);
  const uint64_t nv = n >> 2;
  uint64_t beg, end;
  share(nv, r, S, beg, end);
  const uint32_t T = blockDim.x;
  float acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) acc[u] = 0.f;
  for (uint64_t base = beg + threadIdx.x; base < end; base += (uint64_t)U * T) {
    float4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = base + (uint64_t)u * T;
      v[u] = i < end ? ld_stream(x + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] += (v[u].x + v[u].y) + (v[u].z + v[u].w);
  }
  if (r == S - 1) {
    const float* xs = reinterpret_cast<const float*>(d.in0);
    for (uint64_t j = nv * 4 + threadIdx.x; j < n; j += T) acc[0] += xs[j];
  }
  float s = acc[0];
#pragma unroll
  for (int u = 1; u < U; ++u) s += acc[u];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (uint32_t w = 0; w < T / 32; ++w) t += red[w];
  return t;
}

/* Last CTA of the cluster: out[0] = partials added in rank order (binary64). */
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
/* Shares below this many bytes per CTA use the per-warp-bin path, whose set-up
 * and read-out are cheap; larger shares use the conflict-free path. */
#define LK_HIST_SMALL_BYTES (64u * 1024u)
#define LK_HIST_COPIES 4u      /* lane-private counter copies (16 KB each)   */

__device__ __forceinline__ void count4_warp(uint32_t* bins, uint32_t w) {
  atomicAdd(&bins[w & 0xffu], 1u);
  atomicAdd(&bins[(w >> 8) & 0xffu], 1u);
  atomicAdd(&bins[(w >> 16) & 0xffu], 1u);
  atomicAdd(&bins[w >> 24], 1u);
}

__device__ __forceinline__ void red_add_shared(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.cta.shared::cta.add.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

/* Lane-private counters: word ((v & 127) << 5) | lane of a copy holds bins v
 * (low 16 bits, v < 128) and v (high 16 bits, v >= 128) for this lane alone;
 * lane l only touches bank l. */
__device__ __forceinline__ void count4_lane(uint32_t* lane_base, uint32_t w) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint32_t v = (w >> (8 * b)) & 0xffu;
    red_add_shared(lane_base + ((v & 127u) << 5), 1u << ((v >> 7) << 4));
  }
}

template <int U>
__device__ __forceinline__ void hist_small(const lk_slot& d, uint64_t beg, uint64_t end, bool tail, uint32_t* sh,
                                           uint32_t* acc) {
  const uint32_t T = blockDim.x, W = T / 32;
  for (uint32_t i = threadIdx.x; i < W * 256; i += T) sh[i] = 0;
  __syncthreads();
  uint32_t* bins = sh + (threadIdx.x >> 5) * 256;
  const uint4* x = reinterpret_cast<const uint4*>(d.in0);
  for (uint64_t base = beg + threadIdx.x; base < end; base += (uint64_t)U * T) {
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = base + (uint64_t)u * T;
      if (i < end) v[u] = ld_stream(x + i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (base + (uint64_t)u * T < end) {
        count4_warp(bins, v[u].x);
        count4_warp(bins, v[u].y);
        count4_warp(bins, v[u].z);
        count4_warp(bins, v[u].w);
      }
    }
  }
  if (tail) {
    const uint8_t* xb = reinterpret_cast<const uint8_t*>(d.in0);
    for (uint64_t j = (d.n >> 4) * 16 + threadIdx.x; j < d.n; j += T) atomicAdd(&bins[xb[j]], 1u);
  }
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < 256; v += T) {
    uint32_t s = 0;
    for (uint32_t w = 0; w < W; ++w) s += sh[w * 256 + v];
    if (s) atomicAdd(&acc[v], s);
  }
}

template <int U>
__device__ __forceinline__ void hist_large(const lk_slot& d, uint64_t beg, uint64_t end, bool tail, uint32_t* sh,
                                           uint32_t* acc) {
  const uint32_t T = blockDim.x, W = T / 32;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t copy = (threadIdx.x >> 5) % LK_HIST_COPIES;
  uint32_t* lane_base = sh + copy * 4096u + lane;
  /* a 16-bit counter takes at most 65535 increments between read-outs: every
   * lane word is shared by ceil(W / copies) threads */
  const uint32_t sharers = (W + LK_HIST_COPIES - 1) / LK_HIST_COPIES;
  const uint64_t per_thread = 65535u / sharers / 16u;     /* vectors per thread per round */
  const uint64_t chunk = per_thread * T;
  const uint4* x = reinterpret_cast<const uint4*>(d.in0);
  uint32_t tot_lo = 0, tot_hi = 0;   /* bins row and row+128, rows owned by threads < 128 */
  uint64_t cbeg = beg;
  do {
    const uint64_t cend = (end - cbeg > chunk) ? cbeg + chunk : end;
    uint4* z = reinterpret_cast<uint4*>(sh);
    for (uint32_t i = threadIdx.x; i < LK_HIST_COPIES * 1024u; i += T) z[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (uint64_t base = cbeg + threadIdx.x; base < cend; base += (uint64_t)U * T) {
      uint4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t i = base + (uint64_t)u * T;
        if (i < cend) v[u] = ld_stream(x + i);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (base + (uint64_t)u * T < cend) {
          count4_lane(lane_base, v[u].x);
          count4_lane(lane_base, v[u].y);
          count4_lane(lane_base, v[u].z);
          count4_lane(lane_base, v[u].w);
        }
      }
    }
    if (tail && cend == end) {
      const uint8_t* xb = reinterpret_cast<const uint8_t*>(d.in0);
      for (uint64_t j = (d.n >> 4) * 16 + threadIdx.x; j < d.n; j += T) {
        const uint32_t v = xb[j];
        red_add_shared(lane_base + ((v & 127u) << 5), 1u << ((v >> 7) << 4));
      }
    }
    __syncthreads();
    /* read-out: thread `row` < 128 adds the 32 lane words of its row in every
     * copy, 16 bytes at a time, starting at a row-dependent column so that a
     * warp's loads spread over all banks */
    for (uint32_t row = threadIdx.x; row < 128; row += T) {
      for (uint32_t c = 0; c < LK_HIST_COPIES; ++c) {
        const uint4* rw = reinterpret_cast<const uint4*>(sh + c * 4096u + row * 32u);
#pragma unroll
        for (uint32_t j = 0; j < 8; ++j) {
          const uint4 q = rw[(j + row) & 7u];
          tot_lo += (q.x & 0xffffu) + (q.y & 0xffffu) + (q.z & 0xffffu) + (q.w & 0xffffu);
          tot_hi += (q.x >> 16) + (q.y >> 16) + (q.z >> 16) + (q.w >> 16);
        }
      }
    }
    __syncthreads();
    cbeg = cend;
  } while (cbeg < end);
  for (uint32_t row = threadIdx.x; row < 128; row += T) {
    if (tot_lo) atomicAdd(&acc[row], tot_lo);
    if (tot_hi) atomicAdd(&acc[row + 128], tot_hi);
  }
}

template <int U>
__device__ __forceinline__ void body_hist(const lk_slot& d, int r, int S, uint32_t* sh, uint32_t* acc) {
  const uint64_t nv = d.n >> 4;
  uint64_t beg, end;
  share(nv, r, S, beg, end);
  const bool tail = (r == S - 1) && (d.n & 15);
  if ((end - beg) * 16 < LK_HIST_SMALL_BYTES) hist_small<U>(d, beg, end, tail, sh, acc);
  else hist_large<U>(d, beg, end, tail, sh, acc);
}

/* Last CTA: copy the accumulator out and return it to zero for reuse. */
__device__ __forceinline__ void combine_hist(const lk_slot& d, uint32_t* acc) {
  int32_t* out = reinterpret_cast<int32_t*>(d.out);
  for (uint32_t v = threadIdx.x; v < 256; v += blockDim.x) {
    out[v] = (int32_t)__ldcg(acc + v);
    acc[v] = 0;
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

/* Shared memory: two stages of (A rows 16 KB, B tile 16 KB); bars[2]. */
#define LK_GEMM_STAGE_FLOATS 8192u

/* Returns false if a staging copy did not complete before `deadline`.
 * `phase` holds one parity bit per stage and persists across descriptors. */
__device__ __forceinline__ bool body_gemm(const lk_slot& d, int r, int S, float* sm, uint64_t* bars,
                                          uint32_t& phase, uint64_t deadline) {
  const uint64_t tiles = d.n;
  const uint32_t U = gemm_row_split(tiles, S);
  const uint32_t rows = 64 / U;
  uint64_t beg, end;
  share(tiles * U, r, S, beg, end);
  if (beg >= end) return true;
  const float* A = reinterpret_cast<const float*>(d.in0);
  const float* B = reinterpret_cast<const float*>(d.in1);
  float* C = reinterpret_cast<float*>(d.out);
  const uint32_t T = blockDim.x;
  auto issue = [&](uint64_t u, uint32_t st) {
    if (threadIdx.x == 0) {
      const uint64_t tile = u / U;
      const uint32_t rb = (uint32_t)(u % U);
      float* sA = sm + st * LK_GEMM_STAGE_FLOATS;
      fence_proxy_async_smem();
      mbar_expect_tx(&bars[st], rows * 256u + 16384u);
      bulk_g2s(sA, A + tile * 4096 + (uint64_t)rb * rows * 64, rows * 256u, &bars[st]);
      bulk_g2s(sA + 4096, B + tile * 4096, 16384u, &bars[st]);
    }
  };
  __shared__ int s_staged;
  __syncthreads();          /* both stages are free: the previous use ended with a barrier */
  issue(beg, 0);
  bool ok = true;
  for (uint64_t u = beg; u < end; ++u) {
    const uint32_t st = (uint32_t)((u - beg) & 1);
    if (u + 1 < end) issue(u + 1, st ^ 1u);
    /* thread 0 alone decides whether the stage arrived in time, so that every
     * thread takes the same path through the barriers below */
    if (threadIdx.x == 0) {
      int arrived = mbar_wait(&bars[st], (phase >> st) & 1u, deadline);
      if (!arrived) {
        /* let this CTA's own copies land before giving up */
        mbar_wait(&bars[st], (phase >> st) & 1u, deadline + 1000000000ull);
        if (u + 1 < end) mbar_wait(&bars[st ^ 1u], (phase >> (st ^ 1u)) & 1u, deadline + 1000000000ull);
      }
      s_staged = arrived;
    }
    __syncthreads();
    if (!s_staged) {
      ok = false;
      break;
    }
    /* the phase is complete: this wait returns at once and makes the copied
     * bytes visible to this thread */
    mbar_wait(&bars[st], (phase >> st) & 1u, deadline + 1000000000ull);
    phase ^= 1u << st;
    const float* sA = sm + st * LK_GEMM_STAGE_FLOATS;
    const float* sB = sA + 4096;
    const uint64_t tile = u / U;
    const uint32_t rb = (uint32_t)(u % U);
    const uint32_t nmt = rows * 4;   /* 4x4 micro-tiles: rows/4 row groups x 16 column groups */
    for (uint32_t mt = threadIdx.x; mt < nmt; mt += T) {
      const uint32_t r0 = (mt >> 4) << 2, c0 = (mt & 15u) << 2;
      float c[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[i][j] = 0.f;
#pragma unroll 2
      for (uint32_t k = 0; k < 64; k += 4) {
        float av[4][4], bv[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 q = *reinterpret_cast<const float4*>(sA + (r0 + i) * 64 + k);
          av[i][0] = q.x; av[i][1] = q.y; av[i][2] = q.z; av[i][3] = q.w;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 b = *reinterpret_cast<const float4*>(sB + (k + q) * 64 + c0);
          bv[q][0] = b.x; bv[q][1] = b.y; bv[q][2] = b.z; bv[q][3] = b.w;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) c[i][j] = fmaf(av[i][q], bv[q][j], c[i][j]);
      }
      float* crow = C + tile * 4096 + (uint64_t)(rb * rows + r0) * 64 + c0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4*>(crow + i * 64) = make_float4(c[i][0], c[i][1], c[i][2], c[i][3]);
    }
    __syncthreads();        /* stage st is free for unit u + 2 */
  }
  return ok;
}

/* Shared-memory bytes a body needs (histogram counters or GEMM stages). */
__host__ __device__ constexpr uint32_t body_smem_bytes(int threads) {
  return (uint32_t)(threads / 32) * 1024u > 65536u ? (uint32_t)(threads / 32) * 1024u : 65536u;
}

}  // namespace lk
#endif
