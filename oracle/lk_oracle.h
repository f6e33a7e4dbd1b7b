/*
 * lk_oracle.h -- CPU oracle for the LightKernel hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously
 * correct definition of what the GPU path computes.  Only the test-suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no header, helper, table or constant with the CUDA path.
 *
 * Work bodies (the descriptor's "work" applied to its "in/out data items",
 * Sec. I of Burgio, "Enabling predictable parallelism in single-GPU systems
 * with persistent CUDA threads"):
 *   add_i32   out[i] = a[i] + b[i], two's-complement wrap
 *   copy_i32  out[i] = in[i]
 *   hist_u8   bins[v] = #{ i : x[i] == v }, v in 0..255
 *   sum_f32   S = sum_i x[i], accumulated in binary64 (pairwise)
 *   gemm64    C = A B for 64x64 row-major binary32 tiles, accumulated in binary64
 *
 * Execution-log checker: the invariants the paper's dispatch model fixes
 * (Sec. II.C, II.D): every posted descriptor runs exactly once, in the order
 * its cluster received it, only on the SMs pinned to that cluster.
 */
#ifndef LK_ORACLE_H
#define LK_ORACLE_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

void   lko_add_i32(const int32_t* a, const int32_t* b, int32_t* out, size_t n);
void   lko_copy_i32(const int32_t* in, int32_t* out, size_t n);
void   lko_hist_u8(const uint8_t* x, size_t n, int64_t bins[256]);
double lko_sum_f32(const float* x, size_t n);
double lko_abs_sum_f32(const float* x, size_t n);
void   lko_gemm64_f32(const float* A, const float* B, double* C, size_t tiles);
void   lko_gemm64_abs_bound(const float* A, const float* B, double* bound, size_t tiles);

/* The compute-bound loop of Sec. III ("a loop of 20k iterations ... no memory
 * transfer or accesses"), made checkable: thread t of CTA r iterates the
 * linear congruential map x <- 1664525 x + 1013904223 (mod 2^32) `iters`
 * times from x0 = 65536 r + t + 1; a CTA's result is the XOR of its threads'
 * final values.  The oracle jumps ahead by composing the affine map with
 * itself (O(log iters)), never running the loop.
 *   lko_spin_xor(r, threads, iters) -> XOR over t < threads of x_iters(r, t)
 *   lko_lcg_brute(x0, iters)        -> the plain loop, for pinning small cases */
uint32_t lko_spin_xor(uint32_t rank, uint32_t threads, uint64_t iters);
uint32_t lko_lcg_jump(uint32_t x0, uint64_t iters);
uint32_t lko_lcg_brute(uint32_t x0, uint64_t iters);

/* Violation codes reported by lko_check_exec_log. */
enum {
  LKO_OK = 0,
  LKO_BAD_CLUSTER = 1,    /* cluster index outside the partition            */
  LKO_BAD_RANK = 2,       /* rank outside [0, size of its cluster)          */
  LKO_BAD_SEQ = 3,        /* sequence number never posted to that cluster   */
  LKO_DUPLICATE = 4,      /* a (cluster, seq, rank) share ran more than once */
  LKO_MISSING = 5,        /* a (cluster, seq, rank) share never ran          */
  LKO_FIFO = 6,           /* a CTA ran its cluster's descriptors out of order */
  LKO_WRONG_SM = 7,       /* share ran on an SM not pinned to that (cluster, rank) */
  LKO_WRONG_OP = 8,       /* share ran a different operation than was posted */
  LKO_EARLY_COMPLETE = 9  /* completion observed before a share had finished */
};

typedef struct {
  int64_t violations;     /* total number of violations found              */
  int64_t first_index;    /* record index of the first violation (-1 none) */
  int32_t first_code;     /* LKO_* code of the first violation             */
  int32_t counts[10];     /* violations per code                           */
} lko_check_result;

/*
 * Check an execution log of m records against the dispatch invariants.
 *   seq[i], cluster[i], rank[i], smid[i], op[i]: what record i says ran.
 *   order[i]: position of record i in the log of its (cluster, rank) CTA,
 *             0 for the first descriptor that CTA ran.
 *   n_clusters, cluster_size[c]: the partition.
 *   pinned_smid[off_c + r]: the SM that (cluster c, rank r) is pinned to,
 *             where off_c = sum of cluster_size[0..c-1]; -1 = any SM of c.
 *   n_posted[c]: descriptors posted to c, with sequence numbers 1..n_posted[c].
 *   posted_op[poff_c + s - 1]: operation of descriptor s of cluster c, where
 *             poff_c = sum of n_posted[0..c-1]; NULL skips the op check.
 *   t_end[i] / t_complete[poff_c + s - 1]: optional (NULL) timestamps on one
 *             clock; a share must end no later than its descriptor completes.
 * Returns the number of violations (0 = the log satisfies every invariant).
 */
int64_t lko_check_exec_log(size_t m, const uint64_t* seq, const int32_t* cluster,
                           const int32_t* rank, const int32_t* smid, const int32_t* op,
                           const uint64_t* order, int32_t n_clusters,
                           const int32_t* cluster_size, const int32_t* pinned_smid,
                           const uint64_t* n_posted, const int32_t* posted_op,
                           const uint64_t* t_end, const uint64_t* t_complete,
                           lko_check_result* out);

#ifdef __cplusplus
}
#endif
#endif
