/*
 * lk_validate.h -- the argument checks every entry point that accepts a
 * descriptor applies before anything reaches the device (internal; shared by
 * the host runtime and the ordinary-launch entry points, so that the limits
 * of include/lk.h are enforced in one place).
 */
#ifndef LK_VALIDATE_H
#define LK_VALIDATE_H
#include <stdint.h>
#include "lk_layout.h"

/* Inputs each op takes (-1: not an operation a descriptor may name). */
static inline int lk_op_inputs(uint32_t op) {
  switch (op) {
    case LK_OP_NOP: return 0;
    case LK_OP_ADD_I32: return 2;
    case LK_OP_HIST_U8: return 1;
    case LK_OP_SUM_F32: return 1;
    case LK_OP_GEMM64_F32: return 2;
    case LK_OP_COPY_I32: return 1;
    case LK_OP_COMBINE_SUM: return 1;
    case LK_OP_COMBINE_HIST: return 1;
    case LK_OP_SPIN: return 0;
    default: return -1;
  }
}

static inline int lk_aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

/* Descriptor d with inputs in0/in1 (n_in of them) and output out:
 * LK_OK, or LK_EINVAL for a bad op, input count, flags, size, rate,
 * alignment, an address above 2^48, or a missing pointer that the op
 * dereferences.  Limits: n <= 2^40; HIST n < 2^31 (int32 bins); GEMM
 * n <= 2^28 tiles; COMBINE_* n <= 2^20 and out required; SPIN n <= 2^32
 * (out optional); SUM / HIST always write out. */
static inline int lk_validate_desc(const lk_desc* d, const void* in0, const void* in1, int n_in, void* out) {
  if (!d) return LK_EINVAL;
  const int need = lk_op_inputs(d->op);
  if (need < 0 || n_in != need) return LK_EINVAL;
  if (d->flags != 0) return LK_EINVAL;
  if (d->n > (1ull << 40) || d->aux >= (1ull << 40) || (d->aux != 0 && d->aux < LK_RATE_MIN)) return LK_EINVAL;
  const void* ins[2] = {in0, in1};
  for (int i = 0; i < need; ++i) {
    if (!lk_aligned16(ins[i]) || (uintptr_t)ins[i] > LK_LOW48) return LK_EINVAL;
    if (d->n > 0 && !ins[i]) return LK_EINVAL;
  }
  if (!lk_aligned16(out) || (uintptr_t)out > LK_LOW48) return LK_EINVAL;
  switch (d->op) {
    case LK_OP_NOP: break;
    case LK_OP_SUM_F32:
      if (!out) return LK_EINVAL;
      break;
    case LK_OP_HIST_U8:
      if (!out) return LK_EINVAL;
      if (d->n > 0x7fffffffull) return LK_EINVAL;   /* bins are int32 */
      break;
    case LK_OP_GEMM64_F32:
      if (d->n > (1ull << 28)) return LK_EINVAL;
      if (d->n > 0 && !out) return LK_EINVAL;
      break;
    case LK_OP_COMBINE_SUM:
    case LK_OP_COMBINE_HIST:
      if (!out || d->n > (1ull << 20)) return LK_EINVAL;
      break;
    case LK_OP_SPIN:
      if (d->n > 0xffffffffull) return LK_EINVAL;   /* out is optional */
      break;
    default:
      if (d->n > 0 && !out) return LK_EINVAL;
  }
  return LK_OK;
}

#endif
