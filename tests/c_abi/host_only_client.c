/* A plain C client of libgenesys.so: the C ABI used without Python.
 *
 * A host-only context (no GPU) runs the whole request protocol with the
 * calling thread in the role of a GPU work-item: slot claim, publish,
 * doorbell, service thread, completion word.  The program makes a NOP round
 * trip, writes 64 neighbouring 64-byte pieces of a file with pwrite requests
 * (non-blocking, then drained) and reads them back with one pread request,
 * and checks the bytes and the service counters.  Exit status 0 on success.
 *
 * Build: gcc -I include host_only_client.c -L <pkg> -lgenesys -Wl,-rpath,<pkg>
 * Run:   ./host_only_client <scratch file>
 */
#define _GNU_SOURCE
#include <fcntl.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <sys/syscall.h>
#include <unistd.h>

#include "genesys.h"

#define CHECK(cond, ...)                              \
  do {                                                \
    if (!(cond)) {                                    \
      fprintf(stderr, "FAIL %s:%d: ", __FILE__, __LINE__); \
      fprintf(stderr, __VA_ARGS__);                   \
      fprintf(stderr, " (%s)\n", genesys_last_error()); \
      return 1;                                       \
    }                                                 \
  } while (0)

int main(int argc, char **argv) {
  if (argc != 2) {
    fprintf(stderr, "usage: %s <scratch file>\n", argv[0]);
    return 2;
  }
  genesys_config cfg;
  CHECK(genesys_config_default(&cfg) == 0, "config_default");
  cfg.flags = GENESYS_INIT_HOST_ONLY;
  cfg.n_slots = 256;
  cfg.n_service_threads = 2;
  cfg.staging_bytes = 1 << 20;
  genesys_ctx *ctx = NULL;
  CHECK(genesys_init(&cfg, 0, &ctx) == 0 && ctx, "init");

  int64_t ret = 0;
  uint64_t a[6] = {12345, 0, 0, 0, 0, 0};
  CHECK(genesys_emulate_call(ctx, GENESYS_NR_NOP, a, GENESYS_REQ_BLOCKING, &ret) == 0 && ret == 12345, "nop");

  uint8_t *buf = (uint8_t *)genesys_staging(ctx, 2 * 4096);
  CHECK(buf != NULL, "staging");
  for (int i = 0; i < 4096; ++i) buf[i] = (uint8_t)(i * 7 + 3);
  const int fd = open(argv[1], O_CREAT | O_TRUNC | O_RDWR, 0644);
  CHECK(fd >= 0, "open");
  for (int k = 0; k < 64; ++k) {  /* 64 work-items, one 64-byte pwrite each */
    const uint64_t w[6] = {(uint64_t)fd, (uint64_t)(uintptr_t)(buf + 64 * k), 64, (uint64_t)(64 * k), 0, 0};
    CHECK(genesys_emulate_call(ctx, SYS_pwrite64, w, 0, &ret) == 0, "pwrite %d", k);
  }
  CHECK(genesys_drain(ctx, 2000000000ull) == 0, "drain");
  const uint64_t r[6] = {(uint64_t)fd, (uint64_t)(uintptr_t)(buf + 4096), 4096, 0, 0, 0};
  CHECK(genesys_emulate_call(ctx, SYS_pread64, r, GENESYS_REQ_BLOCKING, &ret) == 0 && ret == 4096, "pread %lld",
        (long long)ret);
  CHECK(memcmp(buf, buf + 4096, 4096) == 0, "bytes read back differ");
  close(fd);

  genesys_stats_t st;
  CHECK(genesys_stats_get(ctx, &st) == 0, "stats");
  CHECK(st.requests == 66 && st.failed == 0, "requests %llu failed %llu", (unsigned long long)st.requests,
        (unsigned long long)st.failed);
  CHECK(genesys_shutdown(ctx) == 0, "shutdown");
  printf("ok requests=%llu os_calls=%llu\n", (unsigned long long)st.requests, (unsigned long long)st.os_calls);
  return 0;
}
