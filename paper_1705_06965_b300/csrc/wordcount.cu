// C3: batched filesystem scan (wordcount, Sec. 7.1) on GPU system calls.
//
// The paper's wordcount reads a list of files with GPU-invoked file system
// calls at work-group granularity and counts occurrences of 64 search words
// (Sec. 7.1).  Here one persistent kernel (one block per resident slot) pulls
// (file, chunk) work items from a queue in device memory, reads each chunk
// with pread into host-mapped staging, streams it into shared memory and
// counts whole-token matches against the query list.  In the batched form the
// pread of the next item is a relaxed, non-blocking call that is in flight
// while the current item is scanned (double buffering; Sec. 4.1 suggests weak
// ordering with non-blocking reads for prefetching).  The plain form issues a
// blocking, strongly ordered pread per item.
//
// Token rule: a token is a maximal run of bytes other than ' ' and '\n'; a
// token belongs to the item holding its first byte.  Each read takes one byte
// before the item (does a token start at the item's first byte?) and
// GENESYS_C3_MAX_QUERY_LEN bytes after it (a token that starts inside may end there; a
// longer one cannot equal any query).
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "genesys.h"
#include "genesys_device.cuh"
#include "internal.h"

using namespace genesys;

namespace {

constexpr int kMaxQ = GENESYS_C3_MAX_QUERIES;
constexpr int kHalo = GENESYS_C3_MAX_QUERY_LEN;  // bytes read past an item
constexpr int kHash = 128;                        // query hash table entries

struct C3Item {
  int32_t fd;
  uint32_t len;     // bytes of the item
  uint64_t off;     // file offset of the item
  uint64_t fsize;   // size of the file
  uint64_t pad;
};
static_assert(sizeof(C3Item) == 32, "item layout");

struct C3Queries {
  uint64_t w[kMaxQ][2];  // query bytes, little-endian, zero padded to 16
  uint8_t len[kMaxQ];
  uint32_t nq;
};

int set_err(int code, const char *msg) { return genesys_internal_error(code, msg); }

// Shared-memory tile of a block: 64 bytes per thread (32 at 1024 threads),
// within the 48 KiB a launch gets without opting in.
inline uint32_t c3_tile_bytes(uint32_t threads) { return threads * 16 * (threads > 512 ? 2 : 4); }

__device__ __forceinline__ uint32_t qhash(uint64_t w0, uint64_t w1, uint32_t len) {
  uint64_t z = w0 * 0x9E3779B97F4A7C15ull ^ (w1 + len) * 0xC2B2AE3D27D4EB4Full;
  z ^= z >> 29;
  z *= 0xBF58476D1CE4E5B9ull;
  return (uint32_t)(z >> 57);  // 7 bits: kHash = 128
}

struct C3Smem {
  uint64_t qw[kMaxQ][2];
  unsigned long long cnt[kMaxQ];
  int16_t htab[kHash];
  uint8_t qlen[kMaxQ];
  uint32_t minlen;
  int64_t r;
  uint32_t item;
};

__device__ void c3_prologue(C3Smem &S, const C3Queries *Q) {
  const uint32_t nq = Q->nq;
  for (uint32_t i = threadIdx.x; i < kMaxQ; i += blockDim.x) {
    S.cnt[i] = 0;
    if (i < nq) {
      S.qw[i][0] = Q->w[i][0];
      S.qw[i][1] = Q->w[i][1];
      S.qlen[i] = Q->len[i];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t mn = 255;
    for (int h = 0; h < kHash; ++h) S.htab[h] = -1;
    for (uint32_t i = 0; i < nq; ++i) {
      uint32_t h = qhash(S.qw[i][0], S.qw[i][1], S.qlen[i]);
      while (S.htab[h] >= 0) h = (h + 1) & (kHash - 1);
      S.htab[h] = (int16_t)i;
      mn = S.qlen[i] < mn ? S.qlen[i] : mn;
    }
    S.minlen = mn;
  }
  __syncthreads();
}

// Separator bits of four bytes (bit i set when byte i is ' ' or '\n'): an
// exact zero-byte test on x ^ ' ' and x ^ '\n', then the four high bits
// gathered into the low nibble.
__device__ __forceinline__ uint32_t sep_bits4(uint32_t x) {
  const uint32_t t1 = x ^ 0x20202020u, t2 = x ^ 0x0A0A0A0Au;
  const uint32_t z1 = ~(((t1 & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t1 | 0x7F7F7F7Fu);
  const uint32_t z2 = ~(((t2 & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t2 | 0x7F7F7F7Fu);
  const uint32_t m = (z1 | z2) >> 7;        // 0 or 1 in bits 0, 8, 16, 24
  return (m * 0x01020408u) >> 24;            // bits 0..3
}

// Count the tokens that start at the 16 positions p0 .. p0 + 15 of an item,
// whose bytes b[p0 - 1] .. b[p0 + 46] are tile[base] .. tile[base + 47]: three
// 16-byte shared loads become a 48-bit separator mask (positions at or past
// `avail`, and b[-1] at the start of a file, count as separators).  Token
// starts are the non-separators after a separator; a token's length is the
// distance to the next separator bit, so only tokens of a query's length
// range are assembled byte by byte and looked up in the query hash table.
__device__ __noinline__ void c3_window(C3Smem &S, const uint8_t *tile, uint32_t base, uint32_t p0, uint32_t len,
                                       uint64_t avail, uint64_t off, uint32_t tile_bytes, const genesys_dev &g) {
  if (!dcheck(g, base + 48 <= tile_bytes + 48 && (base & 15) == 0)) return;
  uint64_t sep = 0;  // bit j: window byte j (= b[p0 - 1 + j]) is a separator
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const uint4 x = *reinterpret_cast<const uint4 *>(tile + base + 16 * v);
    const uint64_t bits = sep_bits4(x.x) | (sep_bits4(x.y) << 4) | (sep_bits4(x.z) << 8) | (sep_bits4(x.w) << 12);
    sep |= bits << (16 * v);
  }
  const uint64_t valid = avail - p0 + 1;  // window bytes before `avail` (>= 2, as p0 < len <= avail)
  if (valid < 48) sep |= ~0ull << valid;
  sep |= ~0ull << 48;
  if (p0 == 0 && off == 0) sep |= 1ull;  // the start of a file
  // token starts among window bytes 1 .. min(16, len - p0)
  const uint32_t last = len - p0 < 16 ? len - p0 : 16;
  uint64_t starts = ~sep & (sep << 1) & (((2ull << last) - 1) & ~1ull);
  while (starts) {
    const int j = __ffsll((long long)starts) - 1;
    starts &= starts - 1;
    const uint32_t L = (uint32_t)(__ffsll((long long)(sep >> j)) - 1);  // run of non-separators
    if (L > (uint32_t)kHalo || L < S.minlen) continue;
    const uint8_t *tok = tile + base + j;
    uint64_t w0 = 0, w1 = 0;
    for (uint32_t q = 0; q < L; ++q) {
      const uint64_t c = tok[q];
      if (q < 8) w0 |= c << (8 * q); else w1 |= c << (8 * (q - 8));
    }
    uint32_t h = qhash(w0, w1, L);
    for (int probe = 0; probe < kHash; ++probe) {
      const int qi = S.htab[h];
      if (qi < 0) break;
      if (S.qlen[qi] == L && S.qw[qi][0] == w0 && S.qw[qi][1] == w1) {
        atomicAdd(&S.cnt[qi], 1ull);
        break;
      }
      h = (h + 1) & (kHash - 1);
    }
  }
}

// Count the tokens that start in [0, len) of one item.  b[j] = buf[1 + j]
// holds file byte off + j for j in [-1, avail); b[-1] is meaningful only when
// off > 0.  tile: dynamic shared memory of tile_bytes + 48.  A tile is
// several 16-byte loads per thread, all in flight together (the bytes cross
// the host link: one load per round trip would leave the block waiting at the
// barrier); thread t then owns the 16-position windows t, t + threads, ...
__device__ void c3_scan(const genesys_dev &g, C3Smem &S, uint8_t *tile, uint32_t tile_bytes, const uint8_t *buf,
                        uint64_t buf_cap, uint64_t off, uint32_t len, uint64_t avail) {
  if (avail < len) len = (uint32_t)avail;
  const uint32_t span = tile_bytes + 32;  // s[i] = b[t0 + i - 1], i < span
  for (uint32_t t0 = 0; t0 < len; t0 += tile_bytes) {
    for (uint32_t i = threadIdx.x * 16; i < span; i += blockDim.x * 16) {
      if (t0 + i + 16 <= buf_cap)
        *reinterpret_cast<uint4 *>(tile + i) = *reinterpret_cast<const uint4 *>(buf + t0 + i);
    }
    __syncthreads();
    for (uint32_t base = threadIdx.x * 16; base < tile_bytes && t0 + base < len; base += blockDim.x * 16)
      c3_window(S, tile, base, t0 + base, len, avail, off, tile_bytes, g);
    __syncthreads();
  }
}

__device__ __forceinline__ void c3_read_args(const C3Item &it, uint8_t *buf, uint64_t *dst, uint64_t *n,
                                             uint64_t *foff) {
  // off > 0: read b[-1 ..] into buf[0 ..]; off == 0: read b[0 ..] into buf[1 ..]
  if (it.off > 0) {
    *dst = (uint64_t)buf;
    *foff = it.off - 1;
    *n = (uint64_t)it.len + 1 + kHalo;
  } else {
    *dst = (uint64_t)(buf + 1);
    *foff = 0;
    *n = (uint64_t)it.len + kHalo;
  }
}

__device__ __forceinline__ uint64_t c3_avail(const C3Item &it, int64_t r) {
  if (r <= 0) return 0;
  return it.off > 0 ? (uint64_t)r - 1 : (uint64_t)r;
}

__device__ void c3_flush(C3Smem &S, uint32_t nq, unsigned long long *counts) {
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nq; i += blockDim.x)
    if (S.cnt[i]) atomicAdd(&counts[i], S.cnt[i]);
}

// Plain form: each block pops an item, issues a blocking, strongly ordered
// work-group-grain pread, scans it, repeats.
__global__ void __launch_bounds__(1024, 1) c3_plain_kernel(genesys_dev g, const C3Item *items, uint32_t n_items,
                                                        uint32_t *head, const C3Queries *Q, uint8_t *staging,
                                                        uint64_t buf_bytes, uint32_t tile_bytes,
                                                        unsigned long long *counts) {
  extern __shared__ __align__(16) uint8_t tile[];
  __shared__ C3Smem S;
  c3_prologue(S, Q);
  uint8_t *buf = staging + (size_t)blockIdx.x * buf_bytes;
  for (;;) {
    if (threadIdx.x == 0) S.item = atomicAdd(head, 1u);
    __syncthreads();
    const uint32_t idx = S.item;
    if (idx >= n_items) break;
    const C3Item it = items[idx];
    uint64_t dst, n, foff;
    c3_read_args(it, buf, &dst, &n, &foff);
    // a short read is continued until the item and its halo are whole or the file ends
    const int64_t r = pread_full<GROUP, STRONG>(g, (uint64_t)it.fd, (uint8_t *)dst, n, foff);
    if (r < 0) break;
    c3_scan(g, S, tile, tile_bytes, buf, buf_bytes, it.off, it.len, c3_avail(it, r));
    __syncthreads();  // S.item is rewritten by the next pop
  }
  c3_flush(S, Q->nq, counts);
}

// Batched form: double-buffered, relaxed non-blocking preads (tickets).
__global__ void __launch_bounds__(1024, 1) c3_batched_kernel(genesys_dev g, const C3Item *items, uint32_t n_items,
                                                          uint32_t *head, const C3Queries *Q, uint8_t *staging,
                                                          uint64_t buf_bytes, uint32_t tile_bytes,
                                                          unsigned long long *counts) {
  extern __shared__ __align__(16) uint8_t tile[];
  __shared__ C3Smem S;
  c3_prologue(S, Q);
  uint8_t *bufs[2] = {staging + (size_t)(2 * blockIdx.x) * buf_bytes,
                      staging + (size_t)(2 * blockIdx.x + 1) * buf_bytes};
  const bool leader = threadIdx.x == 0;
  Ticket cur{0xFFFFFFFFu, 0, 0}, nxt{0xFFFFFFFFu, 0, 0};
  uint32_t cur_idx = 0xFFFFFFFFu, nxt_idx = 0xFFFFFFFFu;
  auto issue_item = [&](Ticket *t, uint32_t idx, uint8_t *buf) {
    const C3Item it = items[idx];
    uint64_t dst, n, foff;
    c3_read_args(it, buf, &dst, &n, &foff);
    issue(g, t, SYS_pread64, (uint64_t)it.fd, dst, n, foff);
  };
  // the prefetched read came back short of what it asked for: read the rest
  // (blocking) until the item and its halo are whole or the file ends
  auto finish_item = [&](int64_t r, uint32_t idx, uint8_t *buf) -> int64_t {
    const C3Item it = items[idx];
    uint64_t dst, n, foff;
    c3_read_args(it, buf, &dst, &n, &foff);
    uint64_t got = r > 0 ? ((uint64_t)r < n ? (uint64_t)r : n) : 0;
    while (r > 0 && got < n) {
      Ticket more;
      issue(g, &more, SYS_pread64, (uint64_t)it.fd, dst + got, n - got, foff + got);
      r = wait(g, more);
      if (r > 0) got += (uint64_t)r < n - got ? (uint64_t)r : n - got;
    }
    return r < 0 ? r : (int64_t)got;
  };
  if (leader) {
    cur_idx = atomicAdd(head, 1u);
    if (cur_idx < n_items) issue_item(&cur, cur_idx, bufs[0]);
  }
  for (uint32_t k = 0;; ++k) {
    if (leader) {
      int64_t r = -1;
      if (cur_idx < n_items) {
        nxt_idx = atomicAdd(head, 1u);
        if (nxt_idx < n_items) issue_item(&nxt, nxt_idx, bufs[(k + 1) & 1]);
        r = finish_item(wait(g, cur), cur_idx, bufs[k & 1]);
        if (r < 0 && nxt_idx < n_items) {  // stop: collect the prefetch, release its slot
          wait(g, nxt);
          nxt_idx = 0xFFFFFFFFu;
        }
      }
      S.r = r;
      S.item = cur_idx;
      cur = nxt;
      cur_idx = nxt_idx;
      nxt = Ticket{0xFFFFFFFFu, 0, 0};
      nxt_idx = 0xFFFFFFFFu;
    }
    __syncthreads();
    const uint32_t idx = S.item;
    const int64_t r = S.r;
    if (idx >= n_items || r < 0) break;
    const C3Item it = items[idx];
    c3_scan(g, S, tile, tile_bytes, bufs[k & 1], buf_bytes, it.off, it.len, c3_avail(it, r));
    __syncthreads();  // buffer k&1 is free for the prefetch two items ahead; S is rewritten next
  }
  c3_flush(S, Q->nq, counts);
}

}  // namespace

extern "C" {

int genesys_c3_wordcount(genesys_ctx *c, const int32_t *fds, const uint64_t *file_bytes, uint32_t n_files,
                         const uint8_t *queries16, const uint8_t *qlen, uint32_t nq, uint64_t chunk, uint32_t ctas,
                         uint32_t threads, uint32_t form, void *staging, uint64_t staging_bytes,
                         unsigned long long *counts_dev, void *stream) {
  return genesys_guard("genesys_c3_wordcount", [&]() -> int {
    if (!c || !fds || !file_bytes || !queries16 || !qlen || !staging || !counts_dev)
      return set_err(GENESYS_EINVAL, "NULL argument");
    if (nq == 0 || nq > (uint32_t)kMaxQ) return set_err(GENESYS_EINVAL, "1..64 queries");
    for (uint32_t q = 0; q < nq; ++q)
      if (qlen[q] == 0 || qlen[q] > kHalo) return set_err(GENESYS_EINVAL, "query length must be 1..16");
    if (chunk < 64 || chunk % 16 || chunk > (1u << 30)) return set_err(GENESYS_EINVAL, "chunk: multiple of 16, >= 64");
    if (ctas == 0 || threads < 32 || threads > 1024 || threads % 32) return set_err(GENESYS_EINVAL, "bad launch shape");
    if ((uintptr_t)staging % 16) return set_err(GENESYS_EINVAL, "staging must be 16-byte aligned");
    const uint64_t buf_bytes = chunk + 64;
    const uint64_t need = (uint64_t)ctas * buf_bytes * (form == GENESYS_FORM_BATCHED ? 2 : 1);
    if (staging_bytes < need) return set_err(GENESYS_EINVAL, "staging too small: ctas * (chunk + 64) per buffer");

    // work items: (file, chunk) pairs in file order
    std::vector<C3Item> items;
    for (uint32_t f = 0; f < n_files; ++f) {
      if (fds[f] < 0) return set_err(GENESYS_EINVAL, "bad fd");
      for (uint64_t off = 0; off < file_bytes[f]; off += chunk) {
        C3Item it{};
        it.fd = fds[f];
        it.len = (uint32_t)(file_bytes[f] - off < chunk ? file_bytes[f] - off : chunk);
        it.off = off;
        it.fsize = file_bytes[f];
        items.push_back(it);
      }
    }
    if (items.empty()) return 0;
    if (items.size() > 0xFFFFFFF0ull) return set_err(GENESYS_EINVAL, "too many work items");
    C3Queries q{};
    q.nq = nq;
    for (uint32_t i = 0; i < nq; ++i) {
      uint8_t tmp[16] = {0};
      memcpy(tmp, queries16 + 16 * i, qlen[i]);
      memcpy(&q.w[i][0], tmp, 8);
      memcpy(&q.w[i][1], tmp + 8, 8);
      q.len[i] = qlen[i];
    }
    // device scratch: [head u32 | pad to 256][queries][items]
    const size_t q_off = 256, items_off = (q_off + sizeof(C3Queries) + 255) & ~size_t(255);
    const size_t bytes = items_off + items.size() * sizeof(C3Item);
    void *scratch = nullptr;
    int rc = genesys_internal_scratch(c, bytes, &scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint8_t> pack(items_off, 0);
    memcpy(pack.data() + q_off, &q, sizeof q);
    if (cudaMemcpyAsync(scratch, pack.data(), pack.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync((uint8_t *)scratch + items_off, items.data(), items.size() * sizeof(C3Item),
                        cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      return set_err(GENESYS_ECUDA, "upload of work items failed");
    }
    genesys_dev g;
    genesys_device_view(c, &g);
    if (form == GENESYS_FORM_BATCHED && g.n_slots < 2ull * ctas)
      return set_err(GENESYS_EINVAL, "the batched form holds two slots per block: n_slots must be >= 2 * ctas");
    const C3Item *d_items = (const C3Item *)((uint8_t *)scratch + items_off);
    uint32_t n_items = (uint32_t)items.size();
    uint32_t *head = (uint32_t *)scratch;
    const C3Queries *d_q = (const C3Queries *)((uint8_t *)scratch + q_off);
    uint8_t *st = (uint8_t *)staging;
    uint64_t bb = buf_bytes;
    uint32_t tile_bytes = c3_tile_bytes(threads);
    void *args[] = {&g, &d_items, &n_items, &head, &d_q, &st, &bb, &tile_bytes, &counts_dev};
    const size_t smem = tile_bytes + 48;
    const void *k = form == GENESYS_FORM_BATCHED ? (const void *)&c3_batched_kernel : (const void *)&c3_plain_kernel;
    const uint32_t flags = form == GENESYS_FORM_BATCHED
                               ? (GENESYS_GRAN_GROUP | GENESYS_LAUNCH_RELAXED | GENESYS_LAUNCH_NONBLOCKING)
                               : GENESYS_GRAN_GROUP;
    const uint32_t g3[3] = {ctas, 1, 1}, b3[3] = {threads, 1, 1};
    rc = genesys_launch(c, k, g3, b3, smem, args, flags | GENESYS_LAUNCH_SYNC, stream);
    if (rc) return rc;
    int32_t stw[GENESYS_ST_WORDS];
    rc = genesys_status(c, stw, 1);
    if (rc) return rc;
    if (stw[GENESYS_ST_TIMEOUTS] || stw[GENESYS_ST_FAILED_CALLS] || stw[GENESYS_ST_FIRST_ERROR]) {
      char msg[160];
      snprintf(msg, sizeof msg, "device-side calls failed: first error %d, %d timeouts, %d failed calls",
               stw[GENESYS_ST_FIRST_ERROR], stw[GENESYS_ST_TIMEOUTS], stw[GENESYS_ST_FAILED_CALLS]);
      return set_err(GENESYS_EDEVICE, msg);
    }
    return 0;
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free wordcount.  Same kernels as genesys_c3_wordcount, but the
// per-call device scratch (queue head, query table, work-item list) lives in
// a fixed file-scope device array instead of memory obtained with cudaMalloc,
// for callers that must not allocate device memory while they run.
namespace {

constexpr uint32_t kStaticMaxItems = GENESYS_C3_NOALLOC_MAX_ITEMS;
constexpr size_t kStaticQOff = 256;
constexpr size_t kStaticItemsOff = (kStaticQOff + sizeof(C3Queries) + 255) & ~size_t(255);
constexpr size_t kStaticBytes = kStaticItemsOff + (size_t)kStaticMaxItems * sizeof(C3Item);
constexpr int kStaticMaxDevices = 64;
static_assert(kStaticBytes == GENESYS_C3_NOALLOC_SCRATCH_BYTES, "documented scratch size");

// Every device that loads this library holds this array until the process
// exits.  Host code must not pass `g_c3_noalloc_scratch` itself to a kernel:
// on the host it names a stand-in object, not the device address, which is
// looked up with cudaGetSymbolAddress (below) once per device.
static __device__ __align__(256) unsigned char g_c3_noalloc_scratch[kStaticBytes];

// Host image of the same layout, copied to the device array on each call.
static unsigned char g_c3_noalloc_host[kStaticBytes];
static std::mutex g_c3_noalloc_mu;
static void *g_c3_noalloc_dev_addr[kStaticMaxDevices];

}  // namespace

// The device address of the array on device `dev`, looked up once per device
// with that device current; the caller's current device is restored.
static int c3_noalloc_scratch_address(int dev, unsigned char **out) {
  if (!g_c3_noalloc_dev_addr[dev]) {
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      return set_err(GENESYS_ECUDA, "cudaGetDevice failed");
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      return set_err(GENESYS_ECUDA, "cudaSetDevice failed");
    }
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_c3_noalloc_scratch);
    if (prev != dev && cudaSetDevice(prev) != cudaSuccess) {
      cudaGetLastError();
      return set_err(GENESYS_ECUDA, "cudaSetDevice (restoring the caller's device) failed");
    }
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      char msg[160];
      snprintf(msg, sizeof msg, "cudaGetSymbolAddress(g_c3_noalloc_scratch): %s", cudaGetErrorString(e));
      return set_err(GENESYS_ECUDA, msg);
    }
    g_c3_noalloc_dev_addr[dev] = p;
  }
  *out = (unsigned char *)g_c3_noalloc_dev_addr[dev];
  return 0;
}

extern "C" int genesys_c3_wordcount_noalloc(genesys_ctx *c, const int32_t *fds, const uint64_t *file_bytes,
                                            uint32_t n_files, const uint8_t *queries16, const uint8_t *qlen,
                                            uint32_t nq, uint64_t chunk, uint32_t ctas, uint32_t threads,
                                            uint32_t form, void *staging, uint64_t staging_bytes,
                                            unsigned long long *counts_dev, void *stream) {
  return genesys_guard("genesys_c3_wordcount_noalloc", [&]() -> int {
    if (!c || !fds || !file_bytes || !queries16 || !qlen || !staging || !counts_dev)
      return set_err(GENESYS_EINVAL, "NULL argument");
    if (nq == 0 || nq > (uint32_t)kMaxQ) return set_err(GENESYS_EINVAL, "1..64 queries");
    for (uint32_t q = 0; q < nq; ++q)
      if (qlen[q] == 0 || qlen[q] > kHalo) return set_err(GENESYS_EINVAL, "query length must be 1..16");
    if (chunk < 64 || chunk % 16 || chunk > (1u << 30)) return set_err(GENESYS_EINVAL, "chunk: multiple of 16, >= 64");
    if (ctas == 0 || threads < 32 || threads > 1024 || threads % 32) return set_err(GENESYS_EINVAL, "bad launch shape");
    if ((uintptr_t)staging % 16) return set_err(GENESYS_EINVAL, "staging must be 16-byte aligned");
    const uint64_t buf_bytes = chunk + 64;
    const uint64_t need = (uint64_t)ctas * buf_bytes * (form == GENESYS_FORM_BATCHED ? 2 : 1);
    if (staging_bytes < need) return set_err(GENESYS_EINVAL, "staging too small: ctas * (chunk + 64) per buffer");
    uint64_t n_items = 0;
    for (uint32_t f = 0; f < n_files; ++f) {
      if (fds[f] < 0) return set_err(GENESYS_EINVAL, "bad fd");
      n_items += (file_bytes[f] + chunk - 1) / chunk;
    }
    if (n_items > kStaticMaxItems) {
      char msg[200];
      snprintf(msg, sizeof msg,
               "the files need %llu work items of %llu bytes; the allocation-free wordcount holds at most %u "
               "(use a larger chunk or genesys_c3_wordcount)",
               (unsigned long long)n_items, (unsigned long long)chunk, kStaticMaxItems);
      return set_err(GENESYS_EINVAL, msg);
    }
    if (n_items == 0) return 0;
    const int dev = genesys_internal_device(c);
    if (dev < 0 || dev >= kStaticMaxDevices) return set_err(GENESYS_EINVAL, "device ordinal out of range");

    std::lock_guard<std::mutex> lock(g_c3_noalloc_mu);
    unsigned char *scratch = nullptr;
    if (int rc0 = c3_noalloc_scratch_address(dev, &scratch)) return rc0;  // first call on the device only
    unsigned char *h = g_c3_noalloc_host;
    memset(h, 0, kStaticItemsOff);  // queue head starts at 0; unused query entries are 0
    C3Queries *q = reinterpret_cast<C3Queries *>(h + kStaticQOff);
    q->nq = nq;
    for (uint32_t i = 0; i < nq; ++i) {
      uint8_t tmp[16] = {0};
      memcpy(tmp, queries16 + 16 * i, qlen[i]);
      memcpy(&q->w[i][0], tmp, 8);
      memcpy(&q->w[i][1], tmp + 8, 8);
      q->len[i] = qlen[i];
    }
    C3Item *hi = reinterpret_cast<C3Item *>(h + kStaticItemsOff);
    uint32_t n = 0;
    for (uint32_t f = 0; f < n_files; ++f) {
      for (uint64_t off = 0; off < file_bytes[f]; off += chunk) {
        C3Item it{};
        it.fd = fds[f];
        it.len = (uint32_t)(file_bytes[f] - off < chunk ? file_bytes[f] - off : chunk);
        it.off = off;
        it.fsize = file_bytes[f];
        hi[n++] = it;
      }
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(scratch, h, kStaticItemsOff + (size_t)n * sizeof(C3Item), cudaMemcpyHostToDevice, s) !=
        cudaSuccess) {
      cudaGetLastError();
      return set_err(GENESYS_ECUDA, "upload of work items failed");
    }
    genesys_dev g;
    genesys_device_view(c, &g);
    if (form == GENESYS_FORM_BATCHED && g.n_slots < 2ull * ctas)
      return set_err(GENESYS_EINVAL, "the batched form holds two slots per block: n_slots must be >= 2 * ctas");
    const C3Item *d_items = (const C3Item *)(scratch + kStaticItemsOff);
    uint32_t *head = (uint32_t *)scratch;
    const C3Queries *d_q = (const C3Queries *)(scratch + kStaticQOff);
    uint8_t *st = (uint8_t *)staging;
    uint64_t bb = buf_bytes;
    uint32_t tile_bytes = c3_tile_bytes(threads);
    void *args[] = {&g, &d_items, &n, &head, &d_q, &st, &bb, &tile_bytes, &counts_dev};
    const size_t smem = tile_bytes + 48;
    const void *k = form == GENESYS_FORM_BATCHED ? (const void *)&c3_batched_kernel : (const void *)&c3_plain_kernel;
    const uint32_t flags = form == GENESYS_FORM_BATCHED
                               ? (GENESYS_GRAN_GROUP | GENESYS_LAUNCH_RELAXED | GENESYS_LAUNCH_NONBLOCKING)
                               : GENESYS_GRAN_GROUP;
    const uint32_t g3[3] = {ctas, 1, 1}, b3[3] = {threads, 1, 1};
    int rc = genesys_launch(c, k, g3, b3, smem, args, flags | GENESYS_LAUNCH_SYNC, stream);
    if (rc) return rc;
    int32_t stw[GENESYS_ST_WORDS];
    rc = genesys_status(c, stw, 1);
    if (rc) return rc;
    if (stw[GENESYS_ST_TIMEOUTS] || stw[GENESYS_ST_FAILED_CALLS] || stw[GENESYS_ST_FIRST_ERROR]) {
      char msg[160];
      snprintf(msg, sizeof msg, "device-side calls failed: first error %d, %d timeouts, %d failed calls",
               stw[GENESYS_ST_FIRST_ERROR], stw[GENESYS_ST_TIMEOUTS], stw[GENESYS_ST_FAILED_CALLS]);
      return set_err(GENESYS_EDEVICE, msg);
    }
    return 0;
  });
}
