/* Doorbell ring choice of positional file calls (genesys_ring_of_file in
 * include/genesys_layout.h), as a plain C program: for a rounds of 64
 * consecutive 4 KiB preads (the C1 configuration: 64 blocks reading the
 * neighbouring chunks of one file) and 64 consecutive work-item pwrites of
 * 64 bytes, and the same for 64 KiB pwrites, print how many of `rings`
 * rings each set reaches.  Usage: ring_regions <rings>. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <sys/syscall.h>

#include "genesys_layout.h"

static unsigned rings_reached(uint64_t fd, uint64_t first_off, uint64_t len, unsigned n, unsigned rings,
                              int is_read) {
  unsigned char seen[64] = {0};
  unsigned reached = 0;
  for (unsigned i = 0; i < n; ++i) {
    const uint32_t r = genesys_ring_of_file(fd, first_off + (uint64_t)i * len, rings, is_read);
    if (r >= rings) return 0; /* out of range: reported as 0 */
    if (!seen[r]) {
      seen[r] = 1;
      ++reached;
    }
  }
  return reached;
}

int main(int argc, char **argv) {
  const unsigned rings = argc > 1 ? (unsigned)atoi(argv[1]) : 4;
  if (rings == 0 || rings > 64) return 2;
  unsigned worst_reads = rings, most_writes = 0, most_big_writes = 0;
  /* rounds of 64 neighbouring 4 KiB chunks, one round per 256 KiB of a 1 GiB
     file, on a few descriptors */
  for (uint64_t fd = 3; fd < 7; ++fd)
    for (uint64_t round = 0; round < 4096; ++round) {
      const unsigned r = rings_reached(fd, round << 18, 4096, 64, rings, 1);
      if (r < worst_reads) worst_reads = r;
    }
  /* 64 neighbouring 64-byte pwrites (two warps of a block), 4,096 of them */
  for (uint64_t fd = 3; fd < 7; ++fd)
    for (uint64_t blk = 0; blk < 4096; ++blk) {
      const unsigned w = rings_reached(fd, blk << 12, 64, 64, rings, 0);
      if (w > most_writes) most_writes = w;
      const unsigned b = rings_reached(fd, blk << 18, 65536, 4, rings, 0);
      if (b > most_big_writes) most_big_writes = b;
    }
  printf("reads_min_rings=%u writes_max_rings=%u big_writes_max_rings=%u\n", worst_reads, most_writes,
         most_big_writes);
  return 0;
}
