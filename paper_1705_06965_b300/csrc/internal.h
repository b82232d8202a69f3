// Internal helpers shared by the runtime and the workload entry points.
#pragma once

#include <stddef.h>
#include <time.h>

#include "genesys.h"

/* Host CLOCK_MONOTONIC in ns: the clock of every host-side deadline and host
 * timestamp of the library. */
static inline uint64_t genesys_mono_ns(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

#ifdef __cplusplus
extern "C" {
#endif

/* Record `msg` as the calling thread's last error (genesys_last_error) and
 * return `code`. */
int genesys_internal_error(int code, const char *msg);

struct genesys_ctx;
/* Device scratch arena owned by the context: returns (in *out) at least
 * `bytes` of device memory, growing the arena with cudaMalloc when needed.
 * The memory is reused by the next call; callers must be done with it (the
 * workload entry points synchronise before returning). */
int genesys_internal_scratch(struct genesys_ctx *ctx, size_t bytes, void **out);

/* Staging arena position, and giving back everything allocated after it. */
uint64_t genesys_internal_staging_mark(struct genesys_ctx *ctx);
void genesys_internal_staging_release(struct genesys_ctx *ctx, uint64_t mark);

/* Count of persistent server kernels (key-value, echo) running on the
 * context: +1 when one starts, -1 once it has finished.  genesys_shutdown
 * refuses while it is above 0. */
void genesys_internal_servers(struct genesys_ctx *ctx, int delta);

/* CUDA device ordinal of the context (-1 for NULL). */
int genesys_internal_device(struct genesys_ctx *ctx);

/* Host clock (CLOCK_MONOTONIC) minus device clock (%globaltimer), in ns, from
 * `rounds` GPU <-> host flag round trips: the estimate of the round with the
 * shortest trip, whose length goes to *rtt_ns (the error is at most half of
 * it).  Every wait is bounded by timeout_ns. */
int genesys_internal_clock_offset(int device, uint32_t rounds, uint64_t timeout_ns, int64_t *offset_ns,
                                  uint64_t *rtt_ns);

#ifdef __cplusplus
}

#include <stdio.h>

#include <exception>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

/* C++ exceptions must not cross the C ABI (a ctypes or C caller would be
 * terminated): an entry point whose body allocates host containers or starts
 * threads runs it through genesys_guard, which turns an exception into an
 * error code and a message.  bad_alloc and system_error (a thread that cannot
 * start) become GENESYS_ENOMEM, anything else GENESYS_EINVAL.  The message is
 * formatted into a fixed buffer: no allocation while handling. */
template <class Body>
static inline int genesys_guard(const char *where, Body &&body) noexcept {
  char msg[256];
  try {
    return body();
  } catch (const std::bad_alloc &) {
    snprintf(msg, sizeof msg, "%s: out of host memory", where);
    return genesys_internal_error(GENESYS_ENOMEM, msg);
  } catch (const std::system_error &e) {
    snprintf(msg, sizeof msg, "%s: %s", where, e.what());
    return genesys_internal_error(GENESYS_ENOMEM, msg);
  } catch (const std::exception &e) {
    snprintf(msg, sizeof msg, "%s: %s", where, e.what());
    return genesys_internal_error(GENESYS_EINVAL, msg);
  } catch (...) {
    snprintf(msg, sizeof msg, "%s: unexpected exception", where);
    return genesys_internal_error(GENESYS_EINVAL, msg);
  }
}

/* Joins the threads of `th` that are still joinable when it goes out of
 * scope, also when an exception or an early return leaves the scope:
 * destroying a joinable std::thread would terminate the process.  Every wait
 * of those threads is bounded, so the joins end. */
struct genesys_joiner {
  std::vector<std::thread> &th;
  ~genesys_joiner() {
    for (auto &t : th)
      if (t.joinable()) t.join();
  }
};
#endif
