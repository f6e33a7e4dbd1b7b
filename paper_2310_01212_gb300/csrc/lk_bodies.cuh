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
 *   hist_u8   per-warp shared-memory bins -> per-CTA totals -> cluster
 *             accumulator (global atomics) -> copied out by the last CTA
 *   sum_f32   per-thread float accumulators, warp shuffles, per-CTA partial;
 *             the last CTA adds the partials in rank order in binary64
 *   gemm64    64x64x64 float32 tiles staged into shared memory by TMA bulk
 *             copies (cp.async.bulk + mbarrier), FFMA in k order
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
  uint64_t i = beg + threadIdx.x;
  for (; i + (uint64_t)(U - 1) * T < end; i += (uint64_t)U * T) {
    int4 x[U], y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      x[u] = ld_stream(a + i + (uint64_t)u * T);
      if (ADD) y[u] = ld_stream(b + i + (uint64_t)u * T);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) st_stream(o + i + (uint64_t)u * T, ADD ? add4(x[u], y[u]) : x[u]);
  }
  for (; i < end; i += T) {
    int4 x = ld_stream(a + i);
    st_stream(o + i, ADD ? add4(x, ld_stream(b + i)) : x);
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
  uint64_t i = beg + threadIdx.x;
  for (; i + (uint64_t)(U - 1) * T < end; i += (uint64_t)U * T) {
    float4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = ld_stream(x + i + (uint64_t)u * T);
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] += (v[u].x + v[u].y) + (v[u].z + v[u].w);
  }
  for (; i < end; i += T) {
    float4 v = ld_stream(x + i);
    acc[0] += (v.x + v.y) + (v.z + v.w);
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
__device__ __forceinline__ void count4(uint32_t* bins, uint32_t w) {
  atomicAdd(&bins[w & 0xffu], 1u);
  atomicAdd(&bins[(w >> 8) & 0xffu], 1u);
  atomicAdd(&bins[(w >> 16) & 0xffu], 1u);
  atomicAdd(&bins[w >> 24], 1u);
}

template <int U>
__device__ __forceinline__ void body_hist(const lk_slot& d, int r, int S, uint32_t* sh, uint32_t* acc) {
  const uint32_t T = blockDim.x, W = T / 32;
  for (uint32_t i = threadIdx.x; i < W * 256; i += T) sh[i] = 0;
  __syncthreads();
  uint32_t* bins = sh + (threadIdx.x >> 5) * 256;
  const uint64_t n = d.n;
  const uint4* x = reinterpret_cast<const uint4*>(d.in0);
  const uint64_t nv = n >> 4;
  uint64_t beg, end;
  share(nv, r, S, beg, end);
  uint64_t i = beg + threadIdx.x;
  for (; i + (uint64_t)(U - 1) * T < end; i += (uint64_t)U * T) {
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = ld_stream(x + i + (uint64_t)u * T);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      count4(bins, v[u].x);
      count4(bins, v[u].y);
      count4(bins, v[u].z);
      count4(bins, v[u].w);
    }
  }
  for (; i < end; i += T) {
    uint4 v = ld_stream(x + i);
    count4(bins, v.x);
    count4(bins, v.y);
    count4(bins, v.z);
    count4(bins, v.w);
  }
  if (r == S - 1) {
    const uint8_t* xb = reinterpret_cast<const uint8_t*>(d.in0);
    for (uint64_t j = nv * 16 + threadIdx.x; j < n; j += T) atomicAdd(&bins[xb[j]], 1u);
  }
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < 256; v += T) {
    uint32_t s = 0;
    for (uint32_t w = 0; w < W; ++w) s += sh[w * 256 + v];
    if (s) atomicAdd(&acc[v], s);
  }
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

/* Returns false if a staging copy did not complete before `deadline`. */
__device__ __forceinline__ bool body_gemm(const lk_slot& d, int r, int S, float* sA, float* sB, uint64_t* bar,
                                          uint32_t& phase, uint64_t deadline) {
  const uint64_t tiles = d.n;
  const uint32_t U = gemm_row_split(tiles, S);
  const uint32_t rows = 64 / U;
  uint64_t beg, end;
  share(tiles * U, r, S, beg, end);
  const float* A = reinterpret_cast<const float*>(d.in0);
  const float* B = reinterpret_cast<const float*>(d.in1);
  float* C = reinterpret_cast<float*>(d.out);
  const uint32_t T = blockDim.x;
  int64_t cur = -1;
  for (uint64_t u = beg; u < end; ++u) {
    const uint64_t tile = u / U;
    const uint32_t rb = (uint32_t)(u % U);
    const bool newB = (int64_t)tile != cur;
    __syncthreads();   /* everyone is done reading sA / sB */
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      mbar_expect_tx(bar, rows * 256u + (newB ? 16384u : 0u));
      bulk_g2s(sA, A + tile * 4096 + (uint64_t)rb * rows * 64, rows * 256u, bar);
      if (newB) bulk_g2s(sB, B + tile * 4096, 16384u, bar);
    }
    cur = (int64_t)tile;
    if (!mbar_wait(bar, phase, deadline)) {
      mbar_wait(bar, phase, deadline + 1000000000ull);   /* let our own copy land */
      return false;
    }
    phase ^= 1u;
    const uint32_t nmt = (rows / 2) * 16;   /* 2x4 micro-tiles */
    for (uint32_t mt = threadIdx.x; mt < nmt; mt += T) {
      const uint32_t r0 = (mt / 16) * 2, c0 = (mt % 16) * 4;
      float c[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll 4
      for (uint32_t k = 0; k < 64; k += 4) {
        const float4 a0 = *reinterpret_cast<const float4*>(sA + r0 * 64 + k);
        const float4 a1 = *reinterpret_cast<const float4*>(sA + (r0 + 1) * 64 + k);
        const float4 b0 = *reinterpret_cast<const float4*>(sB + (k + 0) * 64 + c0);
        const float4 b1 = *reinterpret_cast<const float4*>(sB + (k + 1) * 64 + c0);
        const float4 b2 = *reinterpret_cast<const float4*>(sB + (k + 2) * 64 + c0);
        const float4 b3 = *reinterpret_cast<const float4*>(sB + (k + 3) * 64 + c0);
        const float av[2][4] = {{a0.x, a0.y, a0.z, a0.w}, {a1.x, a1.y, a1.z, a1.w}};
        const float bv[4][4] = {{b0.x, b0.y, b0.z, b0.w}, {b1.x, b1.y, b1.z, b1.w},
                                {b2.x, b2.y, b2.z, b2.w}, {b3.x, b3.y, b3.z, b3.w}};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) c[i][j] = fmaf(av[i][q], bv[q][j], c[i][j]);
      }
      float* crow = C + tile * 4096 + (uint64_t)(rb * rows + r0) * 64 + c0;
      *reinterpret_cast<float4*>(crow) = make_float4(c[0][0], c[0][1], c[0][2], c[0][3]);
      *reinterpret_cast<float4*>(crow + 64) = make_float4(c[1][0], c[1][1], c[1][2], c[1][3]);
    }
  }
  return true;
}

/* Shared-memory bytes a body needs (hist bins or GEMM staging). */
__host__ __device__ constexpr uint32_t body_smem_bytes(int threads) {
  return (uint32_t)(threads / 32) * 1024u > 32768u ? (uint32_t)(threads / 32) * 1024u : 32768u;
}

}  // namespace lk
#endif
