/* genesys_syscall(nr, args...): the device call without a context argument
 * (Sec. 4.1, Sec. 5).
 *
 * genesys::call<Gran, Order, Block>(dev, nr, ...) in genesys_device.cuh names
 * its context's device view in every call.  This header binds one view per
 * translation unit instead: the host passes the view (genesys_device_view) to
 * genesys_syscall_bind before it launches this file's kernels, and device
 * code calls genesys_syscall(nr, a0, ..., a5).  Without template arguments
 * that is the paper's plain form: the calling work-item alone, strong
 * ordering, blocking.  genesys_syscall<Gran, Order, Block>(...) chooses
 * another form, with genesys::call's rules: every thread of the group reaches
 * the call; a strongly ordered kernel-grain call needs every block resident
 * (a cooperative launch, as genesys_launch makes); work-item calls are always
 * strongly ordered.  The result is the call's return value, or -errno.
 */
#ifndef GENESYS_SYSCALL_CUH
#define GENESYS_SYSCALL_CUH

#include <cuda_runtime.h>

#include "genesys.h"
#include "genesys_device.cuh"

/* The bound device view: one copy per translation unit (constant memory). */
static __constant__ genesys_dev genesys_bound_dev;

/* Host: bind `view` for this translation unit's genesys_syscall calls (a
 * synchronous copy to constant memory; not while kernels of this unit that
 * make calls run).  GENESYS_OK, GENESYS_EINVAL for NULL, or GENESYS_ECUDA. */
static inline int genesys_syscall_bind(const genesys_dev *view) {
  if (!view) return GENESYS_EINVAL;
  return cudaMemcpyToSymbol(genesys_bound_dev, view, sizeof *view) == cudaSuccess ? GENESYS_OK : GENESYS_ECUDA;
}

template <int G = genesys::ITEM, int O = genesys::STRONG, int B = genesys::BLOCKING>
__device__ __forceinline__ int64_t genesys_syscall(uint32_t nr, uint64_t a0 = 0, uint64_t a1 = 0, uint64_t a2 = 0,
                                                   uint64_t a3 = 0, uint64_t a4 = 0, uint64_t a5 = 0) {
  static_assert(!(G == genesys::ITEM && O == genesys::RELAXED), "work-item calls are strongly ordered (Sec. 4.1)");
  return genesys::call<G, O, B>(genesys_bound_dev, nr, a0, a1, a2, a3, a4, a5);
}

/* The same call at kernel-grain site `site` (0 .. GENESYS_KSITES - 1; the
 * form above uses site 0).  A relaxed kernel-grain site serves one call per
 * block per launch (genesys_launch resets the sites before each launch): a
 * kernel that makes several relaxed kernel-grain calls gives each its own
 * site.  A site reused within a launch makes no further calls: the extra
 * arrivals return -EINVAL and the launch's status words record it.  Strongly
 * ordered kernel-grain calls may share a site. */
template <int G, int O, int B>
__device__ __forceinline__ int64_t genesys_syscall_at(uint32_t site, uint32_t nr, uint64_t a0 = 0, uint64_t a1 = 0,
                                                      uint64_t a2 = 0, uint64_t a3 = 0, uint64_t a4 = 0,
                                                      uint64_t a5 = 0) {
  static_assert(!(G == genesys::ITEM && O == genesys::RELAXED), "work-item calls are strongly ordered (Sec. 4.1)");
  return genesys::call_at<G, O, B>(genesys_bound_dev, site, nr, a0, a1, a2, a3, a4, a5);
}

#endif
