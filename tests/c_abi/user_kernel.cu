// A kernel of a user of this library: one pread per work-group through the
// device header, launched with genesys_launch.  Compiled (not run) by the host
// tests to show that the device header stands on its own.
#include <cuda_runtime.h>

#include "genesys.h"
#include "genesys_device.cuh"

__global__ void user_scan(genesys_dev g, int fd, uint8_t *staging, uint64_t chunk, unsigned long long *bytes) {
  uint8_t *buf = staging + blockIdx.x * chunk;
  // one pread per work-group, strong ordering, blocking (Sec. 4.1)
  const int64_t r = genesys::call<genesys::GROUP, genesys::STRONG, genesys::BLOCKING>(
      g, SYS_pread64, (uint64_t)fd, (uint64_t)buf, chunk, blockIdx.x * chunk);
  if (threadIdx.x == 0 && r > 0) atomicAdd(bytes, (unsigned long long)r);
}

extern "C" int user_launch(genesys_ctx *ctx, int fd, uint8_t *staging, uint64_t chunk, uint32_t blocks,
                           unsigned long long *bytes_dev) {
  genesys_dev g;
  if (int rc = genesys_device_view(ctx, &g)) return rc;
  void *args[] = {&g, &fd, &staging, &chunk, &bytes_dev};
  const uint32_t grid[3] = {blocks, 1, 1}, block[3] = {128, 1, 1};
  return genesys_launch(ctx, (const void *)&user_scan, grid, block, 0, args,
                        GENESYS_GRAN_GROUP | GENESYS_LAUNCH_SYNC, nullptr);
}
