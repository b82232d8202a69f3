/*
 * Seeded synthetic input generators for the GPU system-call workloads.
 *
 * This file holds no part of the method's arithmetic (no histogram, no
 * tokeniser, no matcher): it only writes input files and records what it
 * emitted.  Both the CUDA path and the CPU oracle read the files it writes.
 *
 * Random numbers: splitmix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used counter-based:
 * the i-th output (0-based) of a generator whose state starts at `seed` is
 *     mix(seed + (i + 1) * 0x9E3779B97F4A7C15)
 * with mix() the published splitmix64 output function.
 *
 * The word corpus stands in for the paper's wordcount input (the Linux source
 * tree searched for 64 strings, Sec. 7.1), which is not available here.
 */
#define _GNU_SOURCE
#include <errno.h>
#include <fcntl.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static inline uint64_t sm_at(uint64_t seed, uint64_t i) { return sm_mix(seed + (i + 1) * GAMMA); }

typedef struct { uint64_t seed, i; } stream_t;
static inline uint64_t st_next(stream_t *s) { return sm_at(s->seed, s->i++); }
/* uniform double in [0, 1) from the top 53 bits */
static inline double st_unif(stream_t *s) { return (double)(st_next(s) >> 11) * 0x1.0p-53; }

uint64_t gen_splitmix64_at(uint64_t seed, uint64_t i) { return sm_at(seed, i); }

/* Bytes [byte0, byte0 + n) of the little-endian byte stream formed by the
 * outputs of the generator started at `seed` (word k covers bytes 8k..8k+7). */
void gen_stream_bytes(uint64_t seed, uint64_t byte0, uint8_t *out, uint64_t n) {
  for (uint64_t b = 0; b < n; ++b) {
    uint64_t pos = byte0 + b;
    uint64_t w = sm_at(seed, pos >> 3);
    out[b] = (uint8_t)(w >> (8 * (pos & 7)));
  }
}

static int write_all(int fd, const uint8_t *p, size_t n) {
  while (n) {
    ssize_t r = write(fd, p, n);
    if (r < 0) { if (errno == EINTR) continue; return -errno; }
    p += r; n -= (size_t)r;
  }
  return 0;
}

/* Writes `nbytes` of the stream of `seed` to `path` (created/truncated). */
int gen_stream_file(const char *path, uint64_t seed, uint64_t nbytes) {
  int fd = open(path, O_CREAT | O_TRUNC | O_WRONLY, 0644);
  if (fd < 0) return -errno;
  const size_t B = 1 << 20;
  uint8_t *buf = (uint8_t *)malloc(B);
  if (!buf) { close(fd); return -ENOMEM; }
  int rc = 0;
  for (uint64_t off = 0; off < nbytes && rc == 0; off += B) {
    uint64_t n = nbytes - off < B ? nbytes - off : B;
    uint64_t w0 = off >> 3;                 /* off is a multiple of 8 */
    for (uint64_t k = 0; k < (n + 7) / 8; ++k) {
      uint64_t w = sm_at(seed, w0 + k);
      uint8_t tmp[8];
      for (int j = 0; j < 8; ++j) tmp[j] = (uint8_t)(w >> (8 * j));
      uint64_t m = n - 8 * k < 8 ? n - 8 * k : 8;
      memcpy(buf + 8 * k, tmp, m);
    }
    rc = write_all(fd, buf, n);
  }
  free(buf);
  close(fd);
  return rc;
}

/* ---------------------------------------------------------------- corpus */

#define MAXW 16

typedef struct {
  int n;
  char (*w)[MAXW];
  uint8_t *len;
  /* open-addressing set over the words, for duplicate rejection and lookup */
  int32_t *tab;
  uint64_t tabmask;
} vocab_t;

static uint64_t word_key(const char *s, int len) {
  uint64_t a = 0, b = 0;
  for (int i = 0; i < len && i < 8; ++i) a |= (uint64_t)(uint8_t)s[i] << (8 * i);
  for (int i = 8; i < len; ++i) b |= (uint64_t)(uint8_t)s[i] << (8 * (i - 8));
  return sm_mix(a ^ sm_mix(b ^ (uint64_t)len));
}

static int vocab_find(const vocab_t *v, const char *s, int len) {
  uint64_t h = word_key(s, len) & v->tabmask;
  for (;;) {
    int32_t id = v->tab[h];
    if (id < 0) return -1;
    if (v->len[id] == len && memcmp(v->w[id], s, (size_t)len) == 0) return id;
    h = (h + 1) & v->tabmask;
  }
}

static void vocab_insert(vocab_t *v, int id) {
  uint64_t h = word_key(v->w[id], v->len[id]) & v->tabmask;
  while (v->tab[h] >= 0) h = (h + 1) & v->tabmask;
  v->tab[h] = id;
}

static int vocab_build(vocab_t *v, int n, uint64_t seed) {
  v->n = n;
  v->w = calloc((size_t)n, MAXW);
  v->len = calloc((size_t)n, 1);
  uint64_t cap = 1;
  while (cap < (uint64_t)n * 4) cap <<= 1;
  v->tab = malloc(cap * sizeof(int32_t));
  v->tabmask = cap - 1;
  if (!v->w || !v->len || !v->tab) return -ENOMEM;
  for (uint64_t i = 0; i < cap; ++i) v->tab[i] = -1;
  stream_t s = {sm_at(seed, 1), 0};
  for (int id = 0; id < n; ++id) {
    for (;;) {
      int len = 3 + (int)(st_next(&s) % 10);       /* uniform 3..12 */
      char tmp[MAXW];
      for (int k = 0; k < len; ++k) tmp[k] = (char)('a' + st_next(&s) % 26);
      if (vocab_find(v, tmp, len) >= 0) continue;  /* redraw duplicates */
      memcpy(v->w[id], tmp, (size_t)len);
      v->len[id] = (uint8_t)len;
      vocab_insert(v, id);
      break;
    }
  }
  return 0;
}

static void vocab_free(vocab_t *v) { free(v->w); free(v->len); free(v->tab); }

/* Finite Zipf over ranks 1..n, p(r) proportional to r^-s; rank r is word r-1. */
static double *zipf_cdf(int n, double s) {
  double *c = malloc(sizeof(double) * (size_t)n);
  if (!c) return NULL;
  double acc = 0;
  for (int r = 1; r <= n; ++r) { acc += pow((double)r, -s); c[r - 1] = acc; }
  for (int r = 0; r < n; ++r) c[r] /= acc;
  c[n - 1] = 1.0;
  return c;
}

/* smallest index i with cdf[i] > u (u in [0,1)) */
static int zipf_draw(const double *cdf, int n, double u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cdf[mid] > u) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/*
 * Writes `n_files` text files dir/f00000.txt ... made of lowercase words drawn
 * Zipf(zipf_s) from a seeded `vocab_n`-word vocabulary, each word followed by a
 * newline (probability 1/16) or a space, every file truncated to its own
 * lognormal size (median `median_bytes`, log-sd `sigma`, capped at `cap_bytes`,
 * at least 1 byte).  Also picks `n_present` distinct vocabulary words at
 * log-uniform ranks and `n_absent` strings that are not vocabulary words as the
 * query list.
 *
 * Outputs (caller-allocated):
 *   sizes_out[n_files]            file sizes in bytes
 *   queries_out[nq * 16]          query strings, NUL padded (nq = n_present + n_absent)
 *   qlen_out[nq]                  query lengths
 *   truth_out[n_files * nq]       per file, how many emitted tokens equal each query
 *                                 (the final token of a file may be cut short by the
 *                                 truncation; it is counted as the string it became)
 *   tokens_out[n_files]           tokens per file
 * Returns 0 or -errno.
 */
int gen_corpus(const char *dir, int n_files, double median_bytes, double sigma, uint64_t cap_bytes,
               int vocab_n, double zipf_s, int n_present, int n_absent, uint64_t seed, int n_threads,
               uint64_t *sizes_out, char *queries_out, uint8_t *qlen_out, uint64_t *truth_out,
               uint64_t *tokens_out) {
  int nq = n_present + n_absent;
  if (n_present > vocab_n || nq <= 0 || n_files <= 0) return -EINVAL;
  vocab_t v;
  int rc = vocab_build(&v, vocab_n, seed);
  if (rc) return rc;
  double *cdf = zipf_cdf(vocab_n, zipf_s);
  if (!cdf) { vocab_free(&v); return -ENOMEM; }

  /* sizes */
  stream_t fs = {sm_at(seed, 2), 0};
  for (int f = 0; f < n_files; ++f) {
    double u1 = 1.0 - st_unif(&fs), u2 = st_unif(&fs);
    double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    double x = median_bytes * exp(sigma * z);
    uint64_t sz = x >= (double)cap_bytes ? cap_bytes : (uint64_t)llround(x);
    if (sz < 1) sz = 1;
    sizes_out[f] = sz;
  }

  /* queries */
  int32_t *qmap = malloc(sizeof(int32_t) * (size_t)vocab_n);
  if (!qmap) { free(cdf); vocab_free(&v); return -ENOMEM; }
  for (int i = 0; i < vocab_n; ++i) qmap[i] = -1;
  memset(queries_out, 0, (size_t)nq * 16);
  stream_t qs = {sm_at(seed, 3), 0};
  for (int q = 0; q < n_present; ++q) {
    for (;;) {
      int r = (int)floor(exp(st_unif(&qs) * log((double)vocab_n)));   /* 1..vocab_n-1 */
      if (r < 1) r = 1;
      int id = r - 1;
      if (qmap[id] >= 0) continue;
      qmap[id] = q;
      memcpy(queries_out + 16 * q, v.w[id], v.len[id]);
      qlen_out[q] = v.len[id];
      break;
    }
  }
  for (int q = n_present; q < nq; ++q) {
    for (;;) {
      int len = 3 + (int)(st_next(&qs) % 10);
      char tmp[MAXW] = {0};
      for (int k = 0; k < len; ++k) tmp[k] = (char)('a' + st_next(&qs) % 26);
      if (vocab_find(&v, tmp, len) >= 0) continue;
      int dup = 0;
      for (int p = n_present; p < q; ++p)
        if (qlen_out[p] == len && memcmp(queries_out + 16 * p, tmp, (size_t)len) == 0) dup = 1;
      if (dup) continue;
      memcpy(queries_out + 16 * q, tmp, (size_t)len);
      qlen_out[q] = (uint8_t)len;
      break;
    }
  }

  memset(truth_out, 0, sizeof(uint64_t) * (size_t)n_files * (size_t)nq);
  int err = 0;
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
  for (int f = 0; f < n_files; ++f) {
    if (err) continue;
    char path[4096];
    snprintf(path, sizeof path, "%s/f%05d.txt", dir, f);
    int fd = open(path, O_CREAT | O_TRUNC | O_WRONLY, 0644);
    if (fd < 0) { err = -errno; continue; }
    const size_t B = 1 << 20;
    uint8_t *buf = malloc(B + 64);
    uint64_t *truth = truth_out + (size_t)f * nq;
    stream_t ts = {sm_at(seed, 1000000ULL + (uint64_t)f), 0};
    uint64_t left = sizes_out[f], ntok = 0;
    size_t fill = 0;
    while (left > 0) {
      int id = zipf_draw(cdf, vocab_n, st_unif(&ts));
      char sep = (st_next(&ts) & 15) == 0 ? '\n' : ' ';
      int len = v.len[id];
      ++ntok;
      if ((uint64_t)len <= left) {
        memcpy(buf + fill, v.w[id], (size_t)len);
        fill += (size_t)len;
        left -= (uint64_t)len;
        if (qmap[id] >= 0) truth[qmap[id]]++;
        if (left > 0) { buf[fill++] = (uint8_t)sep; --left; }
      } else {
        /* the file ends inside this word: the token is the cut prefix */
        int cut = (int)left;
        memcpy(buf + fill, v.w[id], (size_t)cut);
        fill += (size_t)cut;
        left = 0;
        for (int q = 0; q < nq; ++q)
          if (qlen_out[q] == cut && memcmp(queries_out + 16 * q, v.w[id], (size_t)cut) == 0) truth[q]++;
      }
      if (fill >= B) {
        int w = write_all(fd, buf, fill);
        if (w) err = w;
        fill = 0;
      }
    }
    if (fill) { int w = write_all(fd, buf, fill); if (w) err = w; }
    tokens_out[f] = ntok;
    free(buf);
    close(fd);
  }
  free(qmap);
  free(cdf);
  vocab_free(&v);
  return err;
}

/* Vocabulary word `id` of the vocabulary seeded by `seed` (for tests). */
int gen_vocab_word(uint64_t seed, int vocab_n, int id, char *out16) {
  vocab_t v;
  int rc = vocab_build(&v, vocab_n, seed);
  if (rc) return rc;
  memset(out16, 0, 16);
  memcpy(out16, v.w[id], v.len[id]);
  rc = v.len[id];
  vocab_free(&v);
  return rc;
}
