/*
 * lk_oracle.c -- CPU oracle for the LightKernel hot path (test infrastructure
 * only; see lk_oracle.h).  Every routine is the plain definition, written for
 * a reader to check by eye: no blocking, no vectorisation, no reordering
 * beyond what the definition states.
 */
#include "lk_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* int32 vector add.  The descriptor carries two input items and one output
 * item (Sec. I: "a reference to the in/out data items").  Overflow wraps, as
 * two's-complement hardware adds do: the sum is taken modulo 2^32. */
void lko_add_i32(const int32_t* a, const int32_t* b, int32_t* out, size_t n) {
  for (size_t i = 0; i < n; ++i) {
    uint32_t s = (uint32_t)a[i] + (uint32_t)b[i]; /* unsigned add is mod 2^32 in C */
    out[i] = (int32_t)s;
  }
}

/* int32 copy: the identity on the data item. */
void lko_copy_i32(const int32_t* in, int32_t* out, size_t n) {
  for (size_t i = 0; i < n; ++i) out[i] = in[i];
}

/* 256-bin histogram of bytes: bins[v] counts the bytes equal to v. */
void lko_hist_u8(const uint8_t* x, size_t n, int64_t bins[256]) {
  for (int v = 0; v < 256; ++v) bins[v] = 0;
  for (size_t i = 0; i < n; ++i) bins[x[i]] += 1;
}

/* Pairwise (cascade) summation in binary64.  Each binary32 input is exact in
 * binary64; the error of pairwise summation is at most about
 * log2(n) * 2^-53 * sum|x|, far inside the 1e-4 * sum|x| acceptance bound. */
static double pairwise(const float* x, size_t n) {
  if (n <= 8) {
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += (double)x[i];
    return s;
  }
  size_t h = n / 2;
  return pairwise(x, h) + pairwise(x + h, n - h);
}

double lko_sum_f32(const float* x, size_t n) { return pairwise(x, n); }

double lko_abs_sum_f32(const float* x, size_t n) {
  double s = 0.0;
  for (size_t i = 0; i < n; ++i) s += fabs((double)x[i]);
  return s;
}

/* C = A B for `tiles` consecutive 64x64 row-major tiles:
 *   C[i][j] = sum_k A[i][k] * B[k][j].
 * Products of two binary32 values are exact in binary64; the k-sum is the
 * plain triple loop in binary64. */
void lko_gemm64_f32(const float* A, const float* B, double* C, size_t tiles) {
  for (size_t t = 0; t < tiles; ++t) {
    const float* a = A + t * 4096;
    const float* b = B + t * 4096;
    double* c = C + t * 4096;
    for (int i = 0; i < 64; ++i)
      for (int j = 0; j < 64; ++j) {
        double s = 0.0;
        for (int k = 0; k < 64; ++k) s += (double)a[i * 64 + k] * (double)b[k * 64 + j];
        c[i * 64 + j] = s;
      }
  }
}

/* bound[i][j] = sum_k |A[i][k] * B[k][j]|: the scale of the per-element
 * acceptance bound for a binary32 GEMM. */
void lko_gemm64_abs_bound(const float* A, const float* B, double* bound, size_t tiles) {
  for (size_t t = 0; t < tiles; ++t) {
    const float* a = A + t * 4096;
    const float* b = B + t * 4096;
    double* c = bound + t * 4096;
    for (int i = 0; i < 64; ++i)
      for (int j = 0; j < 64; ++j) {
        double s = 0.0;
        for (int k = 0; k < 64; ++k) s += fabs((double)a[i * 64 + k] * (double)b[k * 64 + j]);
        c[i * 64 + j] = s;
      }
  }
}

/* Affine map f(x) = a x + c (mod 2^32).  f applied k times is again affine;
 * composing g after f gives (a_g a_f, a_g c_f + c_g).  Square-and-multiply
 * over the bits of `iters` gives f^iters in O(log iters) compositions. */
uint32_t lko_lcg_jump(uint32_t x0, uint64_t iters) {
  uint32_t acc_a = 1u, acc_c = 0u;          /* identity map */
  uint32_t pa = 1664525u, pc = 1013904223u; /* f^(2^bit) */
  while (iters) {
    if (iters & 1u) {                       /* acc <- p after acc */
      acc_c = pa * acc_c + pc;
      acc_a = pa * acc_a;
    }
    pc = pa * pc + pc;                      /* p <- p after p */
    pa = pa * pa;
    iters >>= 1;
  }
  return acc_a * x0 + acc_c;
}

uint32_t lko_lcg_brute(uint32_t x0, uint64_t iters) {
  uint32_t x = x0;
  for (uint64_t i = 0; i < iters; ++i) x = 1664525u * x + 1013904223u;
  return x;
}

uint32_t lko_spin_xor(uint32_t rank, uint32_t threads, uint64_t iters) {
  uint32_t r = 0;
  for (uint32_t t = 0; t < threads; ++t) r ^= lko_lcg_jump(65536u * rank + t + 1u, iters);
  return r;
}

/* ---------------------------------------------------------------------------
 * Execution-log checker.
 *
 * The dispatch model (Sec. II.C-II.D): one persistent block is pinned on each
 * SM at boot; the host hands a cluster one descriptor at a time through that
 * cluster's mailbox; every block of the cluster takes part in it and the
 * cluster reports it finished.  Hence, for every cluster c and every posted
 * descriptor s of c, each rank r of c runs s exactly once, on the SM that r is
 * pinned to, and each rank runs c's descriptors in posting order: the k-th
 * descriptor a rank runs is descriptor k (sequence numbers start at 1).
 * ------------------------------------------------------------------------- */
static void flag(lko_check_result* r, int code, int64_t idx) {
  if (r->violations == 0) {
    r->first_code = code;
    r->first_index = idx;
  }
  r->violations += 1;
  r->counts[code] += 1;
}

int64_t lko_check_exec_log(size_t m, const uint64_t* seq, const int32_t* cluster,
                           const int32_t* rank, const int32_t* smid, const int32_t* op,
                           const uint64_t* order, int32_t n_clusters,
                           const int32_t* cluster_size, const int32_t* pinned_smid,
                           const uint64_t* n_posted, const int32_t* posted_op,
                           const uint64_t* t_end, const uint64_t* t_complete,
                           lko_check_result* out) {
  lko_check_result r;
  memset(&r, 0, sizeof r);
  r.first_index = -1;

  /* rank offsets and posted-descriptor offsets per cluster */
  int64_t* roff = (int64_t*)calloc((size_t)n_clusters + 1, sizeof(int64_t));
  int64_t* poff = (int64_t*)calloc((size_t)n_clusters + 1, sizeof(int64_t));
  int64_t* soff = (int64_t*)calloc((size_t)n_clusters + 1, sizeof(int64_t));
  for (int c = 0; c < n_clusters; ++c) {
    roff[c + 1] = roff[c] + cluster_size[c];
    poff[c + 1] = poff[c] + (int64_t)n_posted[c];
    soff[c + 1] = soff[c] + (int64_t)n_posted[c] * cluster_size[c];
  }
  /* one counter per (cluster, descriptor, rank) share */
  uint32_t* seen = (uint32_t*)calloc((size_t)soff[n_clusters] + 1, sizeof(uint32_t));

  for (size_t i = 0; i < m; ++i) {
    int32_t c = cluster[i];
    if (c < 0 || c >= n_clusters) { flag(&r, LKO_BAD_CLUSTER, (int64_t)i); continue; }
    if (rank[i] < 0 || rank[i] >= cluster_size[c]) { flag(&r, LKO_BAD_RANK, (int64_t)i); continue; }
    if (seq[i] < 1 || seq[i] > n_posted[c]) { flag(&r, LKO_BAD_SEQ, (int64_t)i); continue; }
    int64_t share = soff[c] + (int64_t)(seq[i] - 1) * cluster_size[c] + rank[i];
    seen[share] += 1;
    if (seen[share] == 2) flag(&r, LKO_DUPLICATE, (int64_t)i);
    /* FIFO: the k-th descriptor this CTA ran (k from 0) must be descriptor k+1 */
    if (seq[i] != order[i] + 1) flag(&r, LKO_FIFO, (int64_t)i);
    int32_t want = pinned_smid ? pinned_smid[roff[c] + rank[i]] : -1;
    if (want >= 0 && smid[i] != want) flag(&r, LKO_WRONG_SM, (int64_t)i);
    if (posted_op && op[i] != posted_op[poff[c] + (int64_t)seq[i] - 1]) flag(&r, LKO_WRONG_OP, (int64_t)i);
    if (t_end && t_complete && t_end[i] > t_complete[poff[c] + (int64_t)seq[i] - 1])
      flag(&r, LKO_EARLY_COMPLETE, (int64_t)i);
  }
  for (int c = 0; c < n_clusters; ++c)
    for (uint64_t s = 1; s <= n_posted[c]; ++s)
      for (int q = 0; q < cluster_size[c]; ++q)
        if (seen[soff[c] + (int64_t)(s - 1) * cluster_size[c] + q] == 0) flag(&r, LKO_MISSING, -1);

  free(seen);
  free(soff);
  free(poff);
  free(roff);
  if (out) *out = r;
  return r.violations;
}
