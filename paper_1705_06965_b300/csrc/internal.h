// Internal helpers shared by the runtime and the workload entry points.
#pragma once

#include <stddef.h>

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
#endif
