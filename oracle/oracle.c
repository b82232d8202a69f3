/*
 * CPU oracle for the GPU system-call workloads.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline/reference leg may load this library.  It shares no
 * code, header, table or constant generator with the CUDA path: it is a plain,
 * sequential program that issues the same Linux system calls (pread, pwrite,
 * ...) on the same seeded inputs and computes every result by its plain
 * definition, in exact integer arithmetic.
 *
 * Paper: Vesely et al., "GPU System Calls" (GENESYS), arXiv 1705.06965.
 */
#define _GNU_SOURCE
#include <errno.h>
#include <fcntl.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <netinet/in.h>
#include <sys/mman.h>
#include <sys/socket.h>
#include <time.h>
#include <unistd.h>

/* ------------------------------------------------------------------ common */

/* pread that keeps calling until `len` bytes or end of file (a short read is
 * legal for pread(2); the caller retries at the advanced offset). */
static int64_t pread_full(int fd, uint8_t *buf, uint64_t len, uint64_t off) {
  uint64_t got = 0;
  while (got < len) {
    ssize_t r = pread(fd, buf + got, len - got, (off_t)(off + got));
    if (r < 0) {
      if (errno == EINTR) continue;
      return -errno;
    }
    if (r == 0) break;                       /* end of file */
    got += (uint64_t)r;
  }
  return (int64_t)got;
}

static int64_t pwrite_full(int fd, const uint8_t *buf, uint64_t len, uint64_t off) {
  uint64_t put = 0;
  while (put < len) {
    ssize_t r = pwrite(fd, buf + put, len - put, (off_t)(off + put));
    if (r < 0) {
      if (errno == EINTR) continue;
      return -errno;
    }
    put += (uint64_t)r;
  }
  return (int64_t)put;
}

/* splitmix64 (Steele, Lea & Flood, OOPSLA 2014), written out from its
 * published definition: state advances by the golden gamma, the output is the
 * state passed through two xor-shift-multiply rounds and a final xor-shift.
 * oracle_splitmix64_at(seed, i) is the (i+1)-th output of a generator whose
 * state starts at `seed`. */
uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* ---------------------------------------------------------------------- C1
 * The pread microbenchmark of Sec. 6 (Fig. 5): a file on tmpfs is read with
 * pread in fixed-size chunks; here every byte read is counted into a 256-bin
 * histogram.  The sum over bins is order-free, so the assignment of chunks to
 * work-groups on the GPU cannot change the result.
 *
 * hist[b] = number of bytes of the file whose value is b, read chunk by chunk
 * at offsets 0, chunk, 2*chunk, ...  Returns the number of bytes read or -errno. */
int64_t oracle_c1_histogram(const char *path, uint64_t chunk, uint32_t *hist) {
  if (chunk == 0) return -EINVAL;
  int fd = open(path, O_RDONLY);
  if (fd < 0) return -errno;
  uint8_t *buf = (uint8_t *)malloc(chunk);
  if (!buf) { close(fd); return -ENOMEM; }
  for (int b = 0; b < 256; ++b) hist[b] = 0;
  uint64_t off = 0;
  int64_t ret = 0;
  for (;;) {
    int64_t r = pread_full(fd, buf, chunk, off);
    if (r < 0) { ret = r; break; }
    for (int64_t i = 0; i < r; ++i) hist[buf[i]] += 1;
    off += (uint64_t)r;
    if ((uint64_t)r < chunk) { ret = (int64_t)off; break; }
  }
  free(buf);
  close(fd);
  return ret;
}

/* ---------------------------------------------------------------------- C2
 * The pwrite microbenchmark (Sec. 4.1 "Invocation granularity", Sec. 6): each
 * of n_threads work-items owns the 64 bytes at file offset gid*64, filled with
 * the eight 64-bit little-endian words splitmix64_at(seed, gid*8 + k), k=0..7.
 * pwrite takes an absolute offset, so the file content does not depend on the
 * order or grouping of the calls (Sec. 4.1).  The oracle issues the calls the
 * way a group of `group` work-items does when one designated work-item calls
 * on behalf of the group (Sec. 5): one pwrite of the group's contiguous
 * group*64 bytes, in group order; group = 1 is the work-item grain.
 * The file is created/truncated first.  Returns the number of pwrite calls. */
int64_t oracle_c2_pwrite(const char *path, uint64_t n_threads, uint64_t group, uint64_t seed) {
  if (group == 0) return -EINVAL;
  int fd = open(path, O_CREAT | O_TRUNC | O_WRONLY, 0644);
  if (fd < 0) return -errno;
  uint8_t *buf = (uint8_t *)malloc(group * 64);
  if (!buf) { close(fd); return -ENOMEM; }
  int64_t calls = 0;
  for (uint64_t g0 = 0; g0 < n_threads; g0 += group) {
    uint64_t members = n_threads - g0 < group ? n_threads - g0 : group;
    for (uint64_t t = 0; t < members; ++t)
      for (uint64_t k = 0; k < 8; ++k) {
        uint64_t w = oracle_splitmix64_at(seed, (g0 + t) * 8 + k);
        for (int j = 0; j < 8; ++j) buf[t * 64 + k * 8 + j] = (uint8_t)(w >> (8 * j));
      }
    int64_t r = pwrite_full(fd, buf, members * 64, g0 * 64);
    if (r < 0) { calls = r; break; }
    ++calls;
  }
  free(buf);
  close(fd);
  return calls;
}

/* ---------------------------------------------------------------------- C3
 * Wordcount (Sec. 7.1): count the occurrences of query words in a list of
 * files.  Reading: a token is a maximal run of bytes that are neither ' ' nor
 * '\n'; an occurrence is a token equal, byte for byte and as a whole, to a
 * query.  Each file is read sequentially with pread in `chunk`-byte pieces;
 * a token cut by a chunk boundary is carried over to the next piece.
 *
 * counts[q] += occurrences of query q (queries16[q*16 .. +qlen[q]]) over all
 * files; if per_file is non-NULL, per_file[f*nq + q] gets the file's own count.
 * Returns total bytes read or -errno. */
static int is_sep(uint8_t c) { return c == ' ' || c == '\n'; }

#define TOKMAX 16

static void match_token(const uint8_t *tok, uint64_t len, const uint8_t *queries16,
                        const uint8_t *qlen, int nq, uint64_t *counts) {
  if (len == 0 || len > TOKMAX) return;       /* queries are at most 16 bytes */
  for (int q = 0; q < nq; ++q)
    if (qlen[q] == len && memcmp(queries16 + 16 * q, tok, len) == 0) { counts[q] += 1; return; }
}

static int64_t wordcount_file(const char *path, const uint8_t *queries16, const uint8_t *qlen, int nq,
                              uint64_t chunk, uint8_t *buf, uint64_t *counts) {
  int fd = open(path, O_RDONLY);
  if (fd < 0) return -errno;
  uint8_t tok[TOKMAX];
  uint64_t tlen = 0;                          /* may exceed TOKMAX: then the token cannot match */
  uint64_t off = 0;
  for (;;) {
    int64_t r = pread_full(fd, buf, chunk, off);
    if (r < 0) { close(fd); return r; }
    for (int64_t i = 0; i < r; ++i) {
      uint8_t c = buf[i];
      if (is_sep(c)) {
        match_token(tok, tlen, queries16, qlen, nq, counts);
        tlen = 0;
      } else {
        if (tlen < TOKMAX) tok[tlen] = c;
        ++tlen;
      }
    }
    off += (uint64_t)r;
    if ((uint64_t)r < chunk) break;
  }
  match_token(tok, tlen, queries16, qlen, nq, counts);   /* a token that ends at end of file */
  close(fd);
  return (int64_t)off;
}

int64_t oracle_c3_wordcount(const char **paths, int n_files, const uint8_t *queries16, const uint8_t *qlen,
                            int nq, uint64_t chunk, uint64_t *counts, uint64_t *per_file) {
  if (chunk == 0) return -EINVAL;
  uint8_t *buf = (uint8_t *)malloc(chunk);
  uint64_t *fc = (uint64_t *)calloc((size_t)nq, sizeof(uint64_t));
  if (!buf || !fc) { free(buf); free(fc); return -ENOMEM; }
  for (int q = 0; q < nq; ++q) counts[q] = 0;
  int64_t total = 0;
  for (int f = 0; f < n_files; ++f) {
    for (int q = 0; q < nq; ++q) fc[q] = 0;
    int64_t r = wordcount_file(paths[f], queries16, qlen, nq, chunk, buf, fc);
    if (r < 0) { total = r; break; }
    total += r;
    for (int q = 0; q < nq; ++q) {
      counts[q] += fc[q];
      if (per_file) per_file[(size_t)f * nq + q] = fc[q];
    }
  }
  free(buf);
  free(fc);
  return total;
}

/* The paper's CPU comparison for wordcount (Sec. 7.1): the same count with
 * OpenMP, files assigned to cores.  Same result as oracle_c3_wordcount. */
int64_t oracle_c3_wordcount_omp(const char **paths, int n_files, const uint8_t *queries16, const uint8_t *qlen,
                                int nq, uint64_t chunk, uint64_t *counts, int n_threads) {
  if (chunk == 0) return -EINVAL;
  for (int q = 0; q < nq; ++q) counts[q] = 0;
  int64_t total = 0;
  int err = 0;
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel num_threads(n_threads)
  {
    uint8_t *buf = (uint8_t *)malloc(chunk);
    uint64_t *fc = (uint64_t *)calloc((size_t)nq, sizeof(uint64_t));
    uint64_t *mine = (uint64_t *)calloc((size_t)nq, sizeof(uint64_t));
    int64_t my_total = 0;
#pragma omp for schedule(dynamic, 1)
    for (int f = 0; f < n_files; ++f) {
      if (!buf || !fc || !mine) { err = -ENOMEM; continue; }
      for (int q = 0; q < nq; ++q) fc[q] = 0;
      int64_t r = wordcount_file(paths[f], queries16, qlen, nq, chunk, buf, fc);
      if (r < 0) { err = (int)r; continue; }
      my_total += r;
      for (int q = 0; q < nq; ++q) mine[q] += fc[q];
    }
#pragma omp critical
    {
      total += my_total;
      if (mine) for (int q = 0; q < nq; ++q) counts[q] += mine[q];
    }
    free(buf); free(fc); free(mine);
  }
  return err ? err : total;
}

/* ---------------------------------------------------------------------- C5
 * Mixed trace of GPU kernels making file and memory system calls (Sec. 7:
 * the filesystem calls pread/pwrite and the memory calls mmap/munmap of the
 * paper's 11-call set, Sec. 8.1).  Each request is a list of operations, run
 * in order:
 *   kind 0  pread  `len` bytes of input file `file` at `off`; result: the
 *           checksum of the bytes read;
 *   kind 1  pwrite `len` bytes of the stream of `seed` to the output file at
 *           `out_off`; result: the byte count written;
 *   kind 2  mmap an anonymous `len`-byte region, fill word i with
 *           splitmix64_at(seed, i), checksum the region, munmap it; result:
 *           the checksum.
 * Checksum of a byte string (zero padded to whole 64-bit little-endian words
 * w_0, w_1, ...): the sum mod 2^64 of splitmix64's output function applied to
 * w_i + (i + 1) * 0x9E3779B97F4A7C15 - i.e. for an all-zero string, the sum of
 * the first outputs of splitmix64 started at 0.  A sum, so any partition of
 * the string can be checksummed in parallel. */
typedef struct oracle_c5_op {
  uint32_t kind, file;
  uint64_t off, len, seed, out_off;
} oracle_c5_op;

static uint64_t sm_out(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t oracle_c5_checksum(const uint8_t *buf, uint64_t len) {
  uint64_t s = 0;
  for (uint64_t i = 0; 8 * i < len; ++i) {
    uint64_t w = 0;
    for (uint64_t b = 0; b < 8 && 8 * i + b < len; ++b) w |= (uint64_t)buf[8 * i + b] << (8 * b);
    s += sm_out(w + (i + 1) * 0x9E3779B97F4A7C15ULL);
  }
  return s;
}

/* results[k] receives operation k's result (or -errno as uint64). */
int64_t oracle_c5_request(const oracle_c5_op *ops, uint32_t n_ops, const int32_t *in_fds, int32_t out_fd,
                          uint64_t *results) {
  for (uint32_t k = 0; k < n_ops; ++k) {
    const oracle_c5_op *op = &ops[k];
    if (op->kind == 0) {
      uint8_t *buf = (uint8_t *)malloc(op->len ? op->len : 1);
      if (!buf) return -ENOMEM;
      int64_t r = pread_full(in_fds[op->file], buf, op->len, op->off);
      results[k] = r < 0 ? (uint64_t)r : oracle_c5_checksum(buf, (uint64_t)r);
      free(buf);
    } else if (op->kind == 1) {
      uint8_t *buf = (uint8_t *)malloc(op->len ? op->len : 1);
      if (!buf) return -ENOMEM;
      for (uint64_t b = 0; b < op->len; ++b)
        buf[b] = (uint8_t)(oracle_splitmix64_at(op->seed, b >> 3) >> (8 * (b & 7)));
      int64_t r = pwrite_full(out_fd, buf, op->len, op->out_off);
      results[k] = (uint64_t)r;
      free(buf);
    } else if (op->kind == 2) {
      uint64_t *p = (uint64_t *)mmap(NULL, op->len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
      if (p == MAP_FAILED) { results[k] = (uint64_t)(int64_t)-errno; continue; }
      for (uint64_t i = 0; i < op->len / 8; ++i) p[i] = oracle_splitmix64_at(op->seed, i);
      results[k] = oracle_c5_checksum((const uint8_t *)p, op->len);
      munmap(p, op->len);
    } else {
      return -EINVAL;
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------- C4
 * Key-value service over UDP (Sec. 7.3 networking: the GPU receives and sends
 * datagrams with recvfrom/sendto at work-group grain).  The oracle is the
 * sequential server: a table of n_keys keys (16 bytes each) with their values,
 * requests applied one after the other in client sequence order.
 * Request datagram: op u8 (0 GET, 1 SET), pad u8, vlen u16, seq u32, key[16],
 *                   value[vlen] (SET only); little-endian.
 * Reply datagram:   op|0x80 u8, status u8 (0 ok, 1 no such key), vlen u16,
 *                   seq u32, value[vlen] (GET of a present key only).
 * `reqs` holds n requests back to back (each a datagram); replies are written
 * back to back into `out` (at most n * (8 + 1024) bytes) with their offsets in
 * `out_off[n + 1]`.  Values: vals[i * 1024 .. + vlens[i]] (updated by SETs). */
static int key_cmp(const uint8_t *a, const uint8_t *b) { return memcmp(a, b, 16); }

static int64_t find_key(const uint8_t *keys, const uint32_t *order, uint32_t n_keys, const uint8_t *key) {
  uint32_t lo = 0, hi = n_keys;
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo) / 2;
    int c = key_cmp(keys + 16 * (size_t)order[mid], key);
    if (c == 0) return order[mid];
    if (c < 0) lo = mid + 1; else hi = mid;
  }
  return -1;
}

static const uint8_t *sort_keys;
static int order_cmp(const void *x, const void *y) {
  return key_cmp(sort_keys + 16 * (size_t)*(const uint32_t *)x, sort_keys + 16 * (size_t)*(const uint32_t *)y);
}

/* Apply one request datagram q to the table and write its reply to rep;
 * returns the reply length. */
static uint64_t c4_apply(const uint8_t *keys, const uint32_t *order, uint32_t n_keys, uint8_t *vals, uint16_t *vlens,
                         const uint8_t *q, uint8_t *rep) {
  const uint8_t op = q[0];
  const uint16_t vlen = (uint16_t)(q[2] | (q[3] << 8));
  const int64_t k = find_key(keys, order, n_keys, q + 8);
  rep[0] = (uint8_t)(op | 0x80);
  memcpy(rep + 4, q + 4, 4);
  uint16_t rlen = 0;
  if (k < 0) {
    rep[1] = 1;
  } else if (op == 0) {
    rep[1] = 0;
    rlen = vlens[k];
    memcpy(rep + 8, vals + (size_t)k * 1024, rlen);
  } else {
    rep[1] = 0;
    vlens[k] = vlen;
    memcpy(vals + (size_t)k * 1024, q + 24, vlen);
  }
  rep[2] = (uint8_t)rlen;
  rep[3] = (uint8_t)(rlen >> 8);
  return 8 + (uint64_t)rlen;
}

/* order[i] = the key numbers sorted by key bytes (the lookup index). */
int64_t oracle_kv_index(const uint8_t *keys, uint32_t n_keys, uint32_t *order) {
  for (uint32_t i = 0; i < n_keys; ++i) order[i] = i;
  sort_keys = keys;
  qsort(order, n_keys, sizeof(uint32_t), order_cmp);
  return 0;
}

int64_t oracle_c4_replay(const uint8_t *keys, uint32_t n_keys, uint8_t *vals, uint16_t *vlens, const uint8_t *reqs,
                         uint64_t n, uint8_t *out, uint64_t *out_off) {
  uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * (n_keys ? n_keys : 1));
  if (!order) return -ENOMEM;
  oracle_kv_index(keys, n_keys, order);
  uint64_t pos = 0, o = 0;
  for (uint64_t r = 0; r < n; ++r) {
    const uint8_t *q = reqs + pos;
    out_off[r] = o;
    o += c4_apply(keys, order, n_keys, vals, vlens, q, out + o);
    pos += 24 + (q[0] == 1 ? (uint16_t)(q[2] | (q[3] << 8)) : 0);
  }
  out_off[n] = o;
  free(order);
  return (int64_t)o;
}

/* ------------------------------------------------------------ UDP servers
 * Plain CPU servers for the network workloads (Sec. 7.3: the echo server can
 * process packets on the CPU or on the GPU, both with recvfrom/sendto).  One
 * host thread answers the datagrams of the given sockets (bound by the
 * caller) one at a time: it polls them round robin with non-blocking
 * recvfrom and answers with sendto to the sender.  It returns when every
 * socket got its stop datagram, or when nothing arrived for idle_ns. */
static uint64_t mono_ns(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

/* Echo: each datagram goes back unchanged; a 4-byte datagram is the stop
 * datagram.  stats[2]: datagrams echoed, bytes echoed. */
int64_t oracle_udp_echo(const int32_t *fds, uint32_t n_fds, uint32_t max_packet, uint64_t idle_ns, uint64_t *stats) {
  uint8_t *buf = (uint8_t *)malloc(max_packet ? max_packet : 1);
  uint8_t *done = (uint8_t *)calloc(n_fds ? n_fds : 1, 1);
  if (!buf || !done) { free(buf); free(done); return -ENOMEM; }
  uint32_t open = n_fds;
  uint64_t last = mono_ns();
  stats[0] = stats[1] = 0;
  while (open > 0) {
    int got = 0;
    for (uint32_t i = 0; i < n_fds; ++i) {
      if (done[i]) continue;
      struct sockaddr_storage from;
      socklen_t flen = sizeof from;
      const ssize_t n = recvfrom(fds[i], buf, max_packet, MSG_DONTWAIT, (struct sockaddr *)&from, &flen);
      if (n < 0) continue;
      got = 1;
      if (n == 4) { done[i] = 1; --open; continue; }
      if (sendto(fds[i], buf, (size_t)n, 0, (struct sockaddr *)&from, flen) == n) {
        stats[0] += 1;
        stats[1] += (uint64_t)n;
      }
    }
    const uint64_t now = mono_ns();
    if (got) last = now;
    else if (now - last > idle_ns) break;
  }
  free(buf);
  free(done);
  return (int64_t)stats[0];
}

/* Key-value: each request datagram is applied in arrival order with the same
 * rule as oracle_c4_replay (order from oracle_kv_index); op 2 is the stop
 * datagram.  stats[2]: requests answered, reply bytes. */
int64_t oracle_kv_serve(const int32_t *fds, uint32_t n_fds, const uint8_t *keys, const uint32_t *order,
                        uint32_t n_keys, uint8_t *vals, uint16_t *vlens, uint64_t idle_ns, uint64_t *stats) {
  uint8_t q[24 + 1024 + 64], rep[8 + 1024];
  uint8_t *done = (uint8_t *)calloc(n_fds ? n_fds : 1, 1);
  if (!done) return -ENOMEM;
  uint32_t open = n_fds;
  uint64_t last = mono_ns();
  stats[0] = stats[1] = 0;
  while (open > 0) {
    int got = 0;
    for (uint32_t i = 0; i < n_fds; ++i) {
      if (done[i]) continue;
      struct sockaddr_storage from;
      socklen_t flen = sizeof from;
      const ssize_t n = recvfrom(fds[i], q, sizeof q, MSG_DONTWAIT, (struct sockaddr *)&from, &flen);
      if (n < 0) continue;
      got = 1;
      if (n >= 1 && q[0] == 2) { done[i] = 1; --open; continue; }
      if (n < 24) continue;
      const uint64_t r = c4_apply(keys, order, n_keys, vals, vlens, q, rep);
      if (sendto(fds[i], rep, r, 0, (struct sockaddr *)&from, flen) == (ssize_t)r) {
        stats[0] += 1;
        stats[1] += r;
      }
    }
    const uint64_t now = mono_ns();
    if (got) last = now;
    else if (now - last > idle_ns) break;
  }
  free(done);
  return (int64_t)stats[0];
}

/* ---------------------------------------------------------------------- C6
 * Block permutation (Sec. 6, "Blocking and ordering strategies", Fig. 6): the
 * input array is cut into 8 KiB blocks; each block is permuted `iters` times
 * with the same byte permutation (one step: out[i] = in[perm[i]], a gather
 * like the permutation steps of DES) and the result is written to the file at
 * the block's own offset with pwrite.  Returns the number of pwrite calls. */
int64_t oracle_c6_permute(const uint8_t *input, uint64_t n_blocks, const uint16_t *perm, uint32_t iters,
                          const char *path) {
  int fd = open(path, O_CREAT | O_TRUNC | O_WRONLY, 0644);
  if (fd < 0) return -errno;
  uint8_t a[8192], b[8192];
  int64_t calls = 0;
  for (uint64_t blk = 0; blk < n_blocks; ++blk) {
    memcpy(a, input + blk * 8192, 8192);
    for (uint32_t it = 0; it < iters; ++it) {
      for (int i = 0; i < 8192; ++i) b[i] = a[perm[i]];
      memcpy(a, b, 8192);
    }
    int64_t r = pwrite_full(fd, a, 8192, blk * 8192);
    if (r < 0) { close(fd); return r; }
    ++calls;
  }
  close(fd);
  return calls;
}
