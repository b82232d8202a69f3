// Kernels of a user of this library, launched with genesys_launch.  Built by
// the GPU tests against include/ and libgenesys.so.
//
//   launch_demo_pwrite:  each block pwrites its `block_bytes` of `src` (pinned
//                        staging) at file offset base + b * block_bytes, at
//                        work-group grain (relaxed, blocking), or once for the
//                        whole grid at kernel grain with strong ordering (a
//                        cooperative launch).  The host relaunches it with new
//                        arguments through GENESYS_LAUNCH_GRAPH.
//   launch_demo_sites:   two relaxed kernel-grain calls in one kernel, each at
//                        its own site: a pread (consumer: the first block to
//                        arrive calls, every block receives the result) and a
//                        pwrite of the bytes read (producer: the last block to
//                        arrive calls).
//   launch_demo_reuse:   the same relaxed kernel-grain site reached twice by
//                        every block (a misuse the device code must report).
#include <cuda_runtime.h>

#include "genesys.h"
#include "genesys_device.cuh"

using namespace genesys;

__global__ void launch_demo_pwrite(genesys_dev g, int fd, const uint8_t *src, uint64_t block_bytes, uint64_t base,
                                   int kernel_grain, long long *ret) {
  if (kernel_grain) {
    const uint64_t n = block_bytes * gridDim.x;
    const int64_t r = call<KERNEL, STRONG, BLOCKING>(g, SYS_pwrite64, (uint64_t)fd, (uint64_t)src, n, base);
    if (threadIdx.x == 0) ret[blockIdx.x] = r;
    return;
  }
  const uint64_t off = (uint64_t)blockIdx.x * block_bytes;
  const int64_t r = call<GROUP, RELAXED, BLOCKING>(g, SYS_pwrite64, (uint64_t)fd, (uint64_t)(src + off), block_bytes,
                                                   base + off);
  if (threadIdx.x == 0) ret[blockIdx.x] = r;
}

__global__ void launch_demo_sites(genesys_dev g, int fd, uint8_t *buf, uint64_t len, long long *ret) {
  const int64_t r1 = call_at<KERNEL, RELAXED, BLOCKING>(g, 1, SYS_pread64, (uint64_t)fd, (uint64_t)buf, len, 0);
  const int64_t r2 = call_at<KERNEL, RELAXED, BLOCKING>(g, 2, SYS_pwrite64, (uint64_t)fd, (uint64_t)buf, len, len);
  if (threadIdx.x == 0) {
    ret[2 * blockIdx.x] = r1;
    ret[2 * blockIdx.x + 1] = r2;
  }
}

__global__ void launch_demo_reuse(genesys_dev g, long long *ret) {
  // getpid is neither producer nor consumer (relaxed would mean strong): the
  // consumer role is named, so the first block to arrive calls
  const int64_t a = call_at<KERNEL, RELAXED, BLOCKING, ROLE_CONSUMER>(g, 3, SYS_getpid);
  const int64_t b = call_at<KERNEL, RELAXED, BLOCKING, ROLE_CONSUMER>(g, 3, SYS_getpid);
  if (threadIdx.x == 0) {
    ret[2 * blockIdx.x] = a;
    ret[2 * blockIdx.x + 1] = b;
  }
}

extern "C" int launch_demo_pwrite_run(genesys_ctx *ctx, int fd, const uint8_t *src, uint64_t block_bytes,
                                      uint64_t base, uint32_t blocks, uint32_t threads, int kernel_grain,
                                      long long *ret_dev, uint32_t flags) {
  genesys_dev g;
  if (int rc = genesys_device_view(ctx, &g)) return rc;
  void *args[] = {&g, &fd, &src, &block_bytes, &base, &kernel_grain, &ret_dev};
  const uint32_t grid[3] = {blocks, 1, 1}, block[3] = {threads, 1, 1};
  const uint32_t gran = kernel_grain ? GENESYS_GRAN_KERNEL : (GENESYS_GRAN_GROUP | GENESYS_LAUNCH_RELAXED);
  return genesys_launch(ctx, (const void *)&launch_demo_pwrite, grid, block, 0, args,
                        gran | GENESYS_LAUNCH_SYNC | flags, nullptr);
}

extern "C" int launch_demo_sites_run(genesys_ctx *ctx, int fd, uint8_t *buf, uint64_t len, uint32_t blocks,
                                     long long *ret_dev, uint32_t flags) {
  genesys_dev g;
  if (int rc = genesys_device_view(ctx, &g)) return rc;
  void *args[] = {&g, &fd, &buf, &len, &ret_dev};
  const uint32_t grid[3] = {blocks, 1, 1}, block[3] = {128, 1, 1};
  return genesys_launch(ctx, (const void *)&launch_demo_sites, grid, block, 0, args, flags | GENESYS_LAUNCH_SYNC,
                        nullptr);
}

extern "C" int launch_demo_reuse_run(genesys_ctx *ctx, uint32_t blocks, long long *ret_dev) {
  genesys_dev g;
  if (int rc = genesys_device_view(ctx, &g)) return rc;
  void *args[] = {&g, &ret_dev};
  const uint32_t grid[3] = {blocks, 1, 1}, block[3] = {64, 1, 1};
  return genesys_launch(ctx, (const void *)&launch_demo_reuse, grid, block, 0, args,
                        GENESYS_GRAN_KERNEL | GENESYS_LAUNCH_RELAXED | GENESYS_LAUNCH_SYNC, nullptr);
}
