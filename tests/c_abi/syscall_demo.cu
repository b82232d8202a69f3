// Device code that calls through genesys_syscall.cuh: every thread writes its
// own 64-byte record with a work-item pwrite (the plain form), then each
// block asks for the process id at work-group grain.  Built by the tests
// against include/ alone; the host half receives the context's device view.
#include "genesys_syscall.cuh"

__global__ void syscall_demo_kernel(int fd, const uint8_t *records, long long *item_ret, long long *group_ret) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  item_ret[i] = genesys_syscall(SYS_pwrite64, (uint64_t)fd, (uint64_t)(records + 64 * i), 64, 64 * i);
  const int64_t pid = genesys_syscall<genesys::GROUP>(SYS_getpid);
  if (threadIdx.x == 0) group_ret[blockIdx.x] = pid;
}

extern "C" int syscall_demo(const void *view, int fd, const uint8_t *records, uint32_t blocks, uint32_t threads,
                            long long *item_ret, long long *group_ret) {
  if (int rc = genesys_syscall_bind((const genesys_dev *)view)) return rc;
  syscall_demo_kernel<<<blocks, threads>>>(fd, records, item_ret, group_ret);
  return cudaDeviceSynchronize() == cudaSuccess ? GENESYS_OK : GENESYS_ECUDA;
}
