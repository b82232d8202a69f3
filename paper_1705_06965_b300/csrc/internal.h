// Internal helpers shared by the runtime and the workload entry points.
#pragma once

#ifdef __cplusplus
extern "C" {
#endif

/* Record `msg` as the calling thread's last error (genesys_last_error) and
 * return `code`. */
int genesys_internal_error(int code, const char *msg);

#ifdef __cplusplus
}
#endif
