/*
 * lk_backend.h -- what the host runtime needs from the device side.
 *
 * liblk.so links the CUDA implementation (lk_kernel.cu).  The test build
 * liblk_fake.so links lk_backend_fake.cpp, where host threads play the
 * device's part of the same mailbox protocol over the same memory layout, so
 * that the host runtime can be exercised on a machine without a GPU.
 */
#ifndef LK_BACKEND_H
#define LK_BACKEND_H
#include <stddef.h>
#include <stdint.h>
#include "lk_layout.h"

typedef struct {
  int sm_count;
  size_t smem_per_sm;
  size_t smem_per_block_optin;
  int max_threads_per_sm;
  int can_map_host;
  int cooperative;
} lkb_props;

/* Opaque handle of a launched persistent kernel. */
typedef struct lkb_launch lkb_launch;

int  lkb_props_get(int device, lkb_props* out);                      /* LK_OK / LK_EDEVICE */
int  lkb_alloc_mapped(int device, size_t bytes, void** host, void** dev); /* zeroed */
void lkb_free_mapped(void* host);
int  lkb_alloc_device(int device, size_t bytes, void** dev);           /* zeroed */
void lkb_free_device(void* dev);
int  lkb_zero_device(int device, void* dev, size_t bytes);           /* copy engine, not SMs */
int  lkb_copy_h2d(int device, void* dst, const void* src, size_t bytes);
int  lkb_copy_d2h(int device, void* dst, const void* src, size_t bytes);
/* Streams for the end-to-end trace mode (copies beside a running kernel). */
int  lkb_stream_create(int device, void** stream);
int  lkb_memcpy_async(void* stream, void* dst, const void* src, size_t bytes, int host_to_device);
int  lkb_stream_sync(void* stream);
void lkb_stream_destroy(void* stream);
/* Launch the persistent kernel: a->grid CTAs of `threads` threads. */
int  lkb_launch_kernel(int device, const lk_kargs* a, int threads, lkb_launch** out);
/* 1 = kernel returned, 0 = still running, < 0 = LK_EDEVICE. */
int  lkb_finished(lkb_launch* l);
/* Elapsed CUDA-event time of the launch in ms (after it finished), or -1. */
float lkb_elapsed_ms(lkb_launch* l);
void lkb_release(lkb_launch* l);

#endif
