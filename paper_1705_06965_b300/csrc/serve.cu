// C5: serving a trace of syscall-issuing GPU kernels with continuous
// admission.
//
// Each request is one GPU kernel (64 .. 65,536 threads) that runs a list of
// file and memory operations through GPU system calls - pread + checksum,
// pwrite of a seeded stream, mmap + fill + checksum + munmap - the
// filesystem and memory-allocation calls of the paper's implemented set
// (Sec. 5, Sec. 7, Sec. 8.1).  The server admits an arrived request as soon as
// a launch slot, syscall slots, staging bytes and HBM bytes are free for it,
// launches it on one of several streams (directly, or by relaunching a
// per-slot CUDA graph with updated parameters), and retires it when its
// completion event fires, so requests that arrive while others run overlap on
// the device.  Latency = retirement time - arrival time.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>
#include <sys/mman.h>
#include <time.h>

#include <algorithm>
#include <map>
#include <vector>

#include "genesys.h"
#include "genesys_device.cuh"
#include "internal.h"

using namespace genesys;

namespace {

constexpr uint32_t kSitesPerReq = 2 * GENESYS_C5_MAX_OPS;  // mmap + munmap per op
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
// Linux's MAP_UNINITIALIZED: the kernel overwrites the whole region, so a
// reused region need not be cleared first
constexpr uint64_t kMapUninitialized = 0x4000000;

int set_err(int code, const char *msg) { return genesys_internal_error(code, msg); }

// splitmix64 output function and counter-based value (Steele, Lea & Flood 2014)
__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t sm_at(uint64_t seed, uint64_t i) { return sm_mix(seed + (i + 1) * kGamma); }
// checksum term of 64-bit word `w` at word index `i` of a buffer
__device__ __forceinline__ uint64_t cs_term(uint64_t w, uint64_t i) { return sm_mix(w + (i + 1) * kGamma); }

__device__ __forceinline__ uint64_t block_sum(uint64_t v) {
  __shared__ uint64_t red[32];
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  const uint32_t w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  uint64_t s = 0;
  if (threadIdx.x == 0)
    for (uint32_t i = 0; i < (blockDim.x + 31) / 32; ++i) s += red[i];
  return s;  // valid in thread 0
}

// Parts of an operation of `len` bytes: `parts` blocks, each `share` bytes
// (a multiple of 16), the last one shorter.
__device__ __forceinline__ void split(uint64_t len, uint32_t nblocks, uint32_t min_part, uint32_t *parts,
                                      uint64_t *share) {
  uint64_t p = (len + min_part - 1) / min_part;
  if (p > nblocks) p = nblocks;
  if (p > GENESYS_C5_MAX_PARTS) p = GENESYS_C5_MAX_PARTS;
  if (p == 0) p = 1;
  uint64_t sh = (len + p - 1) / p;
  sh = (sh + 15) & ~uint64_t(15);
  *parts = (uint32_t)((len + sh - 1) / sh);
  *share = sh;
}

// Bytes an operation's parts occupy in staging (or HBM): the parts are
// share-aligned, and every operation has its own region because blocks run
// ahead of each other (nothing makes block A finish operation k before block
// B starts operation k + 1).
__host__ __device__ __forceinline__ uint64_t region_bytes(uint32_t parts, uint64_t share) {
  return ((uint64_t)parts * share + 16 + 255) & ~uint64_t(255);
}

// Block b of the nb blocks that run one request: it handles part b of each
// pread/pwrite; mmap'd regions are filled and checksummed by all threads of
// the nb blocks.  ks: the request's kernel-grain call sites (2 per op).  The
// blocks are the launch's grid (one kernel per request) or a virtual grid run
// by the persistent executor's blocks.
__device__ void c5_run_block(const genesys_dev &g, const genesys_c5_op *ops, uint32_t n_ops, const int32_t *in_fds,
                             int32_t out_fd, uint8_t *staging, uint8_t *landing, unsigned long long *results,
                             uint32_t min_part, uint32_t pread_to_hbm, uint32_t b, uint32_t nb, genesys_ksite *ks) {
  uint64_t st_off = 0, land_off = 0;  // this operation's region
  for (uint32_t k = 0; k < n_ops; ++k) {
    const genesys_c5_op op = ops[k];
    if (op.kind == GENESYS_C5_PREAD) {
      uint32_t parts;
      uint64_t share;
      split(op.len, nb, min_part, &parts, &share);
      uint8_t *region = pread_to_hbm ? landing + land_off : staging + st_off;
      if (pread_to_hbm) land_off += region_bytes(parts, share);
      if (b < parts) {
        const uint64_t p0 = (uint64_t)b * share;
        const uint64_t plen = op.len - p0 < share ? op.len - p0 : share;
        const uint64_t fd = (uint64_t)(int64_t)in_fds[op.file];
        // the pread lands in this part of the request's staging; with
        // pread_to_hbm the block then moves it to its HBM landing region
        // (the SMs copy it: a copy-engine transfer ordered on a stream could
        // queue behind this very kernel) and scans it there
        uint8_t *st_part = staging + st_off + p0;
        // a short read is continued until the part is whole or the file ends
        const int64_t r = pread_full<GROUP, RELAXED, ROLE_CONSUMER>(g, fd, st_part, plen, op.off + p0);
        uint8_t *dst = region + p0;
        // 16-byte loads, eight in flight per thread: the bytes cross the host
        // link, so a thread's loads must overlap to cover its latency
        if (pread_to_hbm && r > 0) {
          const uint4 *src = reinterpret_cast<const uint4 *>(st_part);
          uint4 *to = reinterpret_cast<uint4 *>(dst);
#pragma unroll 8
          for (uint64_t i = threadIdx.x; i < ((uint64_t)r + 15) / 16; i += blockDim.x) to[i] = src[i];
          __syncthreads();
        }
        uint64_t s = 0;
        if (r > 0) {
          const uint64_t n16 = (uint64_t)r >> 4;
          const uint4 *w4 = reinterpret_cast<const uint4 *>(dst);
#pragma unroll 8
          for (uint64_t i = threadIdx.x; i < n16; i += blockDim.x) {
            const uint4 v = w4[i];
            s += cs_term((uint64_t)v.x | ((uint64_t)v.y << 32), (p0 >> 3) + 2 * i) +
                 cs_term((uint64_t)v.z | ((uint64_t)v.w << 32), (p0 >> 3) + 2 * i + 1);
          }
          if (threadIdx.x == 0)  // the last 0-15 bytes: whole words, then a zero-padded one
            for (uint64_t wd = 2 * n16; wd * 8 < (uint64_t)r; ++wd) {
              uint64_t val = 0;
              for (uint64_t q = 0; q < 8 && wd * 8 + q < (uint64_t)r; ++q) val |= (uint64_t)dst[wd * 8 + q] << (8 * q);
              s += cs_term(val, (p0 >> 3) + wd);
            }
        }
        s = block_sum(s);
        if (threadIdx.x == 0) {
          if (r < 0) atomicExch(&results[GENESYS_C5_MAX_OPS + k], (unsigned long long)r);
          else atomicAdd(&results[k], (unsigned long long)s);
        }
      }
      st_off += region_bytes(parts, share);
      __syncthreads();
    } else if (op.kind == GENESYS_C5_PWRITE) {
      uint32_t parts;
      uint64_t share;
      split(op.len, nb, min_part, &parts, &share);
      uint8_t *region = staging + st_off;
      st_off += region_bytes(parts, share);
      if (b < parts) {
        const uint64_t p0 = (uint64_t)b * share;
        const uint64_t plen = op.len - p0 < share ? op.len - p0 : share;
        uint64_t *w = reinterpret_cast<uint64_t *>(region + p0);
        for (uint64_t i = threadIdx.x; i < (plen + 7) / 8; i += blockDim.x) w[i] = sm_at(op.seed, (p0 >> 3) + i);
        const int64_t r = call<GROUP, RELAXED, BLOCKING, ROLE_PRODUCER>(
            g, SYS_pwrite64, (uint64_t)(int64_t)out_fd, (uint64_t)(region + p0), plen, op.out_off + p0);
        if (threadIdx.x == 0) {
          if (r < 0) atomicExch(&results[GENESYS_C5_MAX_OPS + k], (unsigned long long)r);
          else atomicAdd(&results[k], (unsigned long long)r);
        }
      }
      __syncthreads();
    } else {
      // mmap at kernel grain (consumer: the first block to arrive calls, the
      // others wait for its result), fill + checksum by every thread, munmap at
      // kernel grain (producer: the last block to arrive calls)
      const int64_t p = call_vgrid<BLOCKING, ROLE_CONSUMER>(
          g, ks + 2 * k, nb, SYS_mmap, 0, op.len, PROT_READ | PROT_WRITE,
          MAP_PRIVATE | MAP_ANONYMOUS | kMapUninitialized, (uint64_t)-1, 0);
      if (p < 0 || p == 0) {
        if (b == 0 && threadIdx.x == 0) atomicExch(&results[GENESYS_C5_MAX_OPS + k], (unsigned long long)p);
        continue;
      }
      // fill with 16-byte stores, then read back what this thread wrote with
      // uncached loads (independent, so they overlap) and checksum it
      ulonglong2 *m = reinterpret_cast<ulonglong2 *>(p);
      const uint64_t pairs = op.len >> 4;
      const uint64_t stride = (uint64_t)nb * blockDim.x;
      const uint64_t first = (uint64_t)b * blockDim.x + threadIdx.x;
      for (uint64_t i = first; i < pairs; i += stride) m[i] = make_ulonglong2(sm_at(op.seed, 2 * i), sm_at(op.seed, 2 * i + 1));
      uint64_t s = 0;
#pragma unroll 8
      for (uint64_t i = first; i < pairs; i += stride) {
        const ulonglong2 v = __ldcv(m + i);
        s += cs_term(v.x, 2 * i) + cs_term(v.y, 2 * i + 1);
      }
      s = block_sum(s);
      if (threadIdx.x == 0) atomicAdd(&results[k], (unsigned long long)s);
      const int64_t u = call_vgrid<BLOCKING, ROLE_PRODUCER>(g, ks + 2 * k + 1, nb, SYS_munmap, (uint64_t)p, op.len);
      if (u < 0 && threadIdx.x == 0) atomicExch(&results[GENESYS_C5_MAX_OPS + k], (unsigned long long)u);
    }
  }
}

// One request as its own kernel: block b of the grid is block b of the request.
__global__ void __launch_bounds__(1024) c5_request_kernel(genesys_dev g, const genesys_c5_op *ops, uint32_t n_ops,
                                                          const int32_t *in_fds, int32_t out_fd, uint8_t *staging,
                                                          uint8_t *landing, unsigned long long *results,
                                                          uint32_t min_part, uint32_t pread_to_hbm) {
  c5_run_block(g, ops, n_ops, in_fds, out_fd, staging, landing, results, min_part, pread_to_hbm, blockIdx.x, gridDim.x,
               g.ksite);
}

// ------------------------------------------------------ persistent executor
// One kernel serves the whole trace: its blocks pop work units - block b of
// the request in launch slot si - from a ring the serve loop appends to as it
// admits requests, and run c5_run_block for them.  Requests of every size
// share the launch; a request's blocks run on whichever executor blocks take
// its units, so blocks of many requests are on the device at once.
//
// Host-written, pinned: the slot records (a request's operations and
// regions, written before its units are published) and the unit ring (entry
// = (position + 1):32 | slot:16 | block:16, release-stored by the host; the
// device acquires it).  Device memory: the ring's consumer position, each
// slot's results, call sites and count of finished blocks.  Device-written,
// pinned: each slot's results and the sequence number of its finished request
// (release-stored last), which the serve loop polls to retire requests.
constexpr uint32_t kExecStop = 0xFFFFu;  // unit slot field: the block leaves

struct alignas(64) ExecSlot {  // written by the host before the slot's units
  uint32_t n_ops, nb;
  uint64_t st_off, hbm_off;
  uint64_t seq;
  genesys_c5_op ops[GENESYS_C5_MAX_OPS];
};

struct alignas(64) ExecDone {  // written by the request's last block
  unsigned long long results[2 * GENESYS_C5_MAX_OPS];
  uint64_t seq;
};

// Wait (one thread) for ring entry `u`; returns it, or 0 if `deadline_ns`
// passed first (then the executor records -ETIMEDOUT in *err).
__device__ uint64_t exec_wait_unit(const uint64_t *units, uint32_t mask, uint32_t u, uint64_t deadline_ns,
                                   int32_t *err) {
  const uint64_t t0 = now_ns();
  uint32_t ns = 256;
  for (;;) {
    const uint64_t e = ld_acquire_sys(units + (u & mask));
    if ((uint32_t)(e >> 32) == u + 1u) return e;
    if (now_ns() - t0 > deadline_ns) {
      atomicCAS(err, 0, -(int32_t)kETIMEDOUT);
      return 0;
    }
    __nanosleep(ns);
    ns = ns < 32768 ? ns * 2 : ns;  // idle executor blocks poll the host rarely
  }
}

constexpr uint32_t kExecSlotWords = sizeof(ExecSlot) / 16;  // 16-byte pieces of a slot record
static_assert(sizeof(ExecSlot) % 16 == 0 && kExecSlotWords <= 32, "a slot record is read by one warp");

__global__ void __launch_bounds__(1024) c5_executor_kernel(
    genesys_dev g, const ExecSlot *slots, ExecDone *done, const uint64_t *units, uint32_t unit_mask, uint32_t *head,
    unsigned long long *results, genesys_ksite *ksites, uint32_t *finished, const int32_t *in_fds, int32_t out_fd,
    uint8_t *staging, uint8_t *landing, uint32_t min_part, uint32_t pread_to_hbm, uint64_t idle_deadline_ns,
    int32_t *err) {
  __shared__ ExecSlot rec_s;
  __shared__ uint32_t si_s, b_s;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t u = atomicAdd(head, 1u);
      const uint64_t e = exec_wait_unit(units, unit_mask, u, idle_deadline_ns, err);
      si_s = e ? (uint32_t)(e >> 16) & 0xFFFFu : kExecStop;
      b_s = (uint32_t)e & 0xFFFFu;
    }
    __syncthreads();
    const uint32_t si = si_s;
    if (si == kExecStop) break;
    // the slot record (written by the host before it released the entry that
    // thread 0 acquired), one 16-byte piece per thread of the first warp: a
    // single round trip over the host link, not one per field
    if (threadIdx.x < kExecSlotWords) {
      uint64_t lo, hi;
      asm volatile("ld.relaxed.sys.global.v2.u64 {%0, %1}, [%2];"
                   : "=l"(lo), "=l"(hi)
                   : "l"(reinterpret_cast<const uint64_t *>(slots + si) + 2 * threadIdx.x)
                   : "memory");
      reinterpret_cast<uint64_t *>(&rec_s)[2 * threadIdx.x] = lo;
      reinterpret_cast<uint64_t *>(&rec_s)[2 * threadIdx.x + 1] = hi;
    }
    __syncthreads();
    const uint32_t nb = rec_s.nb;
    unsigned long long *res = results + (size_t)si * 2 * GENESYS_C5_MAX_OPS;
    genesys_ksite *ks = ksites + (size_t)si * kSitesPerReq;
    c5_run_block(g, rec_s.ops, rec_s.n_ops, in_fds, out_fd, staging + rec_s.st_off, landing + rec_s.hbm_off, res,
                 min_part, pread_to_hbm, b_s, nb, ks);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(&finished[si], 1u) == nb - 1u) {
        // the request's last block: hand its results to the host and make
        // the slot's device state ready for the next request
        __threadfence();
        volatile ExecDone *d = done + si;
        for (uint32_t k = 0; k < 2 * GENESYS_C5_MAX_OPS; ++k) d->results[k] = atomicExch(res + k, 0ull);
        for (uint32_t k = 0; k < kSitesPerReq; ++k) {
          ks[k].arrive = 0;
          ks[k].ticket = 0;
          ks[k].flag = 0;
          ks[k].ret = 0;
        }
        finished[si] = 0;
        fence_acq_rel_sys();
        st_relaxed_sys((uint64_t *)&d->seq, rec_s.seq);
      }
    }
    __syncthreads();  // the shared request state is rewritten by the next unit
  }
}

// First-fit allocator over [0, size) with coalescing of freed ranges.
class RangeAlloc {
 public:
  explicit RangeAlloc(uint64_t size) { free_[0] = size; }
  bool alloc(uint64_t n, uint64_t *off) {
    n = (n + 255) & ~uint64_t(255);
    if (n == 0) { *off = 0; return true; }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const uint64_t rest = it->second - n, at = it->first + n;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t n) {
    n = (n + 255) & ~uint64_t(255);
    if (n == 0) return;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<uint64_t, uint64_t> free_;
};

struct Needs {
  uint64_t staging, hbm;
  uint32_t slots, blocks;
};

Needs needs_of(const genesys_c5_request &r, uint32_t bt, uint32_t min_part, uint32_t pread_to_hbm) {
  Needs n{0, 0, 0, 0};
  n.blocks = (r.threads + bt - 1) / bt;
  uint64_t parts_max = 1;
  for (uint32_t k = 0; k < r.n_ops; ++k) {
    const genesys_c5_op &op = r.ops[k];
    if (op.kind == GENESYS_C5_MMAP) continue;
    uint64_t p = (op.len + min_part - 1) / min_part;
    p = std::min<uint64_t>(std::min<uint64_t>(p ? p : 1, n.blocks), GENESYS_C5_MAX_PARTS);
    const uint64_t sh = ((op.len + p - 1) / p + 15) & ~uint64_t(15);
    const uint64_t span = region_bytes((uint32_t)((op.len + sh - 1) / sh), sh);
    n.staging += span;
    if (op.kind == GENESYS_C5_PREAD && pread_to_hbm) n.hbm += span;
    parts_max = std::max(parts_max, p);
  }
  n.slots = (uint32_t)parts_max + 1;  // each part's caller, or the kernel-grain caller
  return n;
}

struct Launch {
  bool busy = false;
  uint32_t req = 0;
  int stream = 0;
  Needs need{};
  uint64_t st_off = 0, hbm_off = 0;
  cudaEvent_t done = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t node = nullptr;
};

// GPU mmaps are served from regions mapped and registered before the first
// request, while no request kernel runs: per power-of-two size class, as many
// regions as the trace has mmaps of that class, at most two per request
// slot (blocks of a request can be one operation apart).
int reserve_trace_mmaps(genesys_ctx *c, const genesys_c5_request *reqs, uint32_t n_req, uint32_t K) {
  std::map<uint64_t, uint64_t> per_class;
  for (uint32_t r = 0; r < n_req; ++r)
    for (uint32_t k = 0; k < reqs[r].n_ops; ++k)
      if (reqs[r].ops[k].kind == GENESYS_C5_MMAP) {
        uint64_t cls = 4096;
        while (cls < reqs[r].ops[k].len) cls <<= 1;
        per_class[cls] += 1;
      }
  std::vector<uint64_t> sizes;
  for (auto &kv : per_class)
    for (uint64_t i = 0; i < std::min<uint64_t>(kv.second, 2ull * K); ++i) sizes.push_back(kv.first);
  return sizes.empty() ? 0 : genesys_mmap_reserve(c, sizes.data(), (uint32_t)sizes.size());
}

// System calls a request makes (each pread/pwrite part, mmap and munmap).
uint64_t calls_of(const genesys_c5_request &q, uint32_t blocks, uint32_t min_part) {
  uint64_t calls = 0;
  for (uint32_t k = 0; k < q.n_ops; ++k) {
    const genesys_c5_op &op = q.ops[k];
    if (op.kind == GENESYS_C5_MMAP) { calls += 2; continue; }
    uint64_t p = (op.len + min_part - 1) / min_part;
    p = std::min<uint64_t>(std::min<uint64_t>(p ? p : 1, blocks), GENESYS_C5_MAX_PARTS);
    const uint64_t sh = ((op.len + p - 1) / p + 15) & ~uint64_t(15);
    calls += (op.len + sh - 1) / sh;
  }
  return calls;
}

// genesys_c5_serve with cfg.persistent: the serve loop feeds one executor
// kernel (c5_executor_kernel) instead of launching a kernel per request.
int serve_persistent(genesys_ctx *c, const genesys_c5_request *reqs, uint32_t n_req, const int32_t *in_fds,
                     uint32_t n_in, int32_t out_fd, const genesys_serve_config &cfg, const genesys_dev &g0,
                     uint64_t *results, uint64_t *latency_ns, genesys_serve_stats *stats) {
  const uint32_t K = cfg.max_inflight, bt = cfg.block_threads;
  if (K >= kExecStop) return set_err(GENESYS_EINVAL, "persistent executor: max_inflight must be below 65535");
  uint32_t P = cfg.persistent_blocks;
  if (P == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c5_executor_kernel, (int)bt, 0) != cudaSuccess ||
        per_sm <= 0)
      return set_err(GENESYS_ECUDA, "occupancy query failed");
    P = (uint32_t)per_sm * g0.n_sms;
  }
  if (g0.n_slots < 2ull * P + 2ull * K)
    return set_err(GENESYS_EINVAL, "persistent executor: the slot area needs 2 slots per executor block and request");
  uint32_t max_nb = 1;
  for (uint32_t r = 0; r < n_req; ++r) max_nb = std::max(max_nb, (reqs[r].threads + bt - 1) / bt);
  if (max_nb > 0xFFFFu) return set_err(GENESYS_EINVAL, "persistent executor: at most 65535 blocks per request");
  uint32_t cap = 1;
  while (cap < (uint64_t)K * max_nb + P + 1) cap <<= 1;  // units of the requests in flight + the stops

  // device memory (the context's scratch): ring consumer position, per slot
  // results / call sites / finished blocks, the fd table, the HBM landing
  const size_t res_off = 256;
  const size_t ks_off = res_off + (size_t)K * 2 * GENESYS_C5_MAX_OPS * 8;
  const size_t fin_off = ks_off + (size_t)K * kSitesPerReq * sizeof(genesys_ksite);
  const size_t fds_off = (fin_off + (size_t)K * 4 + 255) & ~size_t(255);
  const size_t land_off = (fds_off + (size_t)n_in * 4 + 4095) & ~size_t(4095);
  void *scratch = nullptr;
  int rc = genesys_internal_scratch(c, land_off + cfg.hbm_budget + 4096, &scratch);
  if (rc) return rc;
  uint8_t *dbase = (uint8_t *)scratch;
  // pinned, host-mapped: slot records, results handed back, the unit ring, the error word
  const size_t h_slots = (size_t)K * sizeof(ExecSlot), h_done = (size_t)K * sizeof(ExecDone);
  const size_t h_units = (size_t)cap * 8, h_bytes = h_slots + h_done + h_units + 64;
  uint8_t *hp = nullptr;
  if (cudaHostAlloc((void **)&hp, h_bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    cudaGetLastError();
    return set_err(GENESYS_ECUDA, "persistent executor: pinned memory");
  }
  memset(hp, 0, h_bytes);
  ExecSlot *hslots = (ExecSlot *)hp;
  ExecDone *hdone = (ExecDone *)(hp + h_slots);
  uint64_t *units = (uint64_t *)(hp + h_slots + h_done);
  int32_t *herr = (int32_t *)(hp + h_slots + h_done + h_units);
  const uint64_t staging_mark = genesys_internal_staging_mark(c);
  uint8_t *staging = (uint8_t *)genesys_staging(c, cfg.staging_budget + 4096);
  cudaStream_t stream = nullptr;
  auto give_back = [&]() {
    if (stream) cudaStreamDestroy(stream);
    cudaFreeHost(hp);
    genesys_internal_staging_release(c, staging_mark);
  };
  if (!staging) {
    give_back();
    return set_err(GENESYS_ENOMEM, "staging arena too small for staging_budget");
  }
  staging = (uint8_t *)(((uintptr_t)staging + 255) & ~uintptr_t(255));
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMemsetAsync(dbase, 0, land_off, stream) != cudaSuccess ||
      cudaMemcpyAsync(dbase + fds_off, in_fds, (size_t)n_in * 4, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaGetLastError();
    give_back();
    return set_err(GENESYS_ECUDA, "persistent executor: set-up");
  }
  if (cfg.reserve_mmaps && (rc = reserve_trace_mmaps(c, reqs, n_req, K))) {
    give_back();
    return rc;
  }

  // the executor runs until it takes a stop unit (one per block), or its
  // blocks have waited cfg.timeout_ns for a unit
  {
    genesys_dev g = g0;
    uint32_t *head = (uint32_t *)dbase;
    unsigned long long *d_res = (unsigned long long *)(dbase + res_off);
    genesys_ksite *d_ks = (genesys_ksite *)(dbase + ks_off);
    uint32_t *d_fin = (uint32_t *)(dbase + fin_off);
    const int32_t *d_fds = (const int32_t *)(dbase + fds_off);
    uint8_t *land = dbase + land_off;
    const ExecSlot *slots_p = hslots;
    ExecDone *done_p = hdone;
    const uint64_t *units_p = units;
    uint32_t mask = cap - 1, mp = cfg.min_part, p2h = cfg.pread_to_hbm;
    int32_t ofd = out_fd;
    uint64_t idle = cfg.timeout_ns;
    int32_t *err_p = herr;
    void *args[] = {&g, &slots_p, &done_p, &units_p, &mask, &head, &d_res, &d_ks, &d_fin, &d_fds, &ofd,
                    &staging, &land, &mp, &p2h, &idle, &err_p};
    if (cudaLaunchKernel((const void *)&c5_executor_kernel, dim3(P), dim3(bt), args, 0, stream) != cudaSuccess) {
      cudaGetLastError();
      give_back();
      return set_err(GENESYS_ECUDA, "persistent executor: launch");
    }
  }

  struct Busy {
    bool busy = false;
    uint32_t req = 0;
    uint64_t seq = 0;
    Needs need{};
    uint64_t st_off = 0, hbm_off = 0;
  };
  std::vector<Busy> bs(K);
  RangeAlloc st_alloc(cfg.staging_budget), hbm_alloc(cfg.hbm_budget);
  uint64_t next = 0, retired = 0, calls = 0, admitted_wait_ns = 0, inflight = 0, max_inflight_seen = 0;
  uint32_t tail = 0;  // ring positions published
  int err = 0;
  const uint64_t t0 = genesys_mono_ns();
  std::vector<uint64_t> arrival_abs(n_req);
  for (uint32_t r = 0; r < n_req; ++r) arrival_abs[r] = cfg.honor_arrivals ? t0 + reqs[r].arrival_ns : t0;
  const uint64_t deadline = t0 + cfg.timeout_ns;
  auto publish = [&](uint32_t si, uint32_t b) {
    __atomic_store_n(&units[tail & (cap - 1)],
                     ((uint64_t)(tail + 1u) << 32) | ((uint64_t)si << 16) | (uint64_t)b, __ATOMIC_RELEASE);
    ++tail;
  };
  while (retired < n_req && !err) {
    bool progress = false;
    for (uint32_t si = 0; si < K; ++si) {  // retire finished requests
      Busy &B = bs[si];
      if (!B.busy || __atomic_load_n(&hdone[si].seq, __ATOMIC_ACQUIRE) != B.seq) continue;
      latency_ns[B.req] = genesys_mono_ns() - arrival_abs[B.req];
      const volatile unsigned long long *hr = hdone[si].results;
      for (uint32_t k = 0; k < GENESYS_C5_MAX_OPS; ++k)
        results[(size_t)B.req * GENESYS_C5_MAX_OPS + k] = hr[GENESYS_C5_MAX_OPS + k] ? hr[GENESYS_C5_MAX_OPS + k] : hr[k];
      st_alloc.release(B.st_off, B.need.staging);
      hbm_alloc.release(B.hbm_off, B.need.hbm);
      B.busy = false;
      --inflight;
      ++retired;
      progress = true;
    }
    while (next < n_req) {  // admit arrived requests, in arrival order, while budgets allow
      const uint64_t now = genesys_mono_ns();
      if (arrival_abs[next] > now) break;
      uint32_t si = 0;
      while (si < K && bs[si].busy) ++si;
      if (si == K) break;
      const Needs nd = needs_of(reqs[next], bt, cfg.min_part, cfg.pread_to_hbm);
      uint64_t so = 0, ho = 0;
      if (!st_alloc.alloc(nd.staging, &so)) break;
      if (!hbm_alloc.alloc(nd.hbm, &ho)) { st_alloc.release(so, nd.staging); break; }
      Busy &B = bs[si];
      B = Busy{true, (uint32_t)next, next + 1, nd, so, ho};
      ExecSlot &rec = hslots[si];
      rec.n_ops = reqs[next].n_ops;
      rec.nb = nd.blocks;
      rec.st_off = so;
      rec.hbm_off = ho;
      rec.seq = B.seq;
      memcpy(rec.ops, reqs[next].ops, sizeof rec.ops);
      for (uint32_t b = 0; b < nd.blocks; ++b) publish(si, b);  // each release-stored after the record
      admitted_wait_ns += now - arrival_abs[next];
      calls += calls_of(reqs[next], nd.blocks, cfg.min_part);
      ++inflight;
      max_inflight_seen = std::max(max_inflight_seen, inflight);
      ++next;
      progress = true;
    }
    if (!progress) {
      if (genesys_mono_ns() > deadline) { err = GENESYS_ETIMEDOUT; break; }
      if (cudaStreamQuery(stream) != cudaErrorNotReady) { err = GENESYS_EDEVICE; break; }  // executor left early
      timespec ts{0, 2000};
      nanosleep(&ts, nullptr);
    }
  }
  const uint64_t t_end = genesys_mono_ns();
  for (uint32_t b = 0; b < P; ++b) publish(kExecStop, 0);  // every executor block leaves
  const cudaError_t se = cudaStreamSynchronize(stream);
  if (se != cudaSuccess && !err) err = GENESYS_ECUDA;
  const int drc = genesys_drain(c, 10ull * g0.deadline_ns);
  genesys_reclaim(c);
  const int32_t exec_err = *(volatile int32_t *)herr;
  give_back();
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->requests = retired;
    stats->syscalls = calls;
    stats->makespan_ns = t_end - t0;
    stats->max_inflight = max_inflight_seen;
    stats->admission_wait_ns = admitted_wait_ns;
  }
  if (err == GENESYS_ETIMEDOUT) return set_err(err, "serve: trace did not finish within timeout_ns");
  if (err == GENESYS_EDEVICE || exec_err) return set_err(GENESYS_EDEVICE, "serve: the executor kernel left early");
  if (err) return set_err(err, "serve: a CUDA call failed");
  if (drc) return drc;
  int32_t stw[GENESYS_ST_WORDS];
  rc = genesys_status(c, stw, 1);
  if (rc) return rc;
  if (stw[GENESYS_ST_TIMEOUTS] || stw[GENESYS_ST_FIRST_ERROR]) {
    char msg[160];
    snprintf(msg, sizeof msg, "serve: device-side calls failed: first error %d, %d timeouts",
             stw[GENESYS_ST_FIRST_ERROR], stw[GENESYS_ST_TIMEOUTS]);
    return set_err(GENESYS_EDEVICE, msg);
  }
  return 0;
}

}  // namespace

extern "C" int genesys_serve_config_default(genesys_serve_config *cfg) {
  if (!cfg) return set_err(GENESYS_EINVAL, "cfg is NULL");
  memset(cfg, 0, sizeof *cfg);
  cfg->max_inflight = 64;
  cfg->n_streams = 64;
  cfg->staging_budget = 64ull << 20;
  cfg->hbm_budget = 64ull << 20;
  cfg->slot_budget = 16384;
  cfg->block_threads = 256;
  cfg->min_part = 16384;
  cfg->use_graphs = 1;
  cfg->pread_to_hbm = 0;
  cfg->honor_arrivals = 1;
  cfg->reserve_mmaps = 1;
  cfg->timeout_ns = 120000000000ull;
  return 0;
}

extern "C" int genesys_c5_serve(genesys_ctx *c, const genesys_c5_request *reqs, uint32_t n_req, const int32_t *in_fds,
                                uint32_t n_in, int32_t out_fd, const genesys_serve_config *cfg_in, uint64_t *results,
                                uint64_t *latency_ns, genesys_serve_stats *stats) {
  return genesys_guard("genesys_c5_serve", [&]() -> int {
    if (!c || (!reqs && n_req) || !in_fds || !results || !latency_ns) return set_err(GENESYS_EINVAL, "NULL argument");
    genesys_serve_config cfg;
    if (cfg_in) cfg = *cfg_in; else genesys_serve_config_default(&cfg);
    const uint32_t bt = cfg.block_threads;
    if (bt < 32 || bt > 1024 || bt % 32) return set_err(GENESYS_EINVAL, "block_threads: 32..1024, multiple of 32");
    if (cfg.max_inflight == 0 || cfg.n_streams == 0 || cfg.min_part < 16)
      return set_err(GENESYS_EINVAL, "max_inflight, n_streams >= 1; min_part >= 16");
    if (out_fd < 0 || n_in == 0) return set_err(GENESYS_EINVAL, "bad file descriptors");
    for (uint32_t r = 0; r < n_req; ++r) {
      if (reqs[r].threads == 0 || reqs[r].n_ops > GENESYS_C5_MAX_OPS) return set_err(GENESYS_EINVAL, "bad request");
      for (uint32_t k = 0; k < reqs[r].n_ops; ++k) {
        const genesys_c5_op &op = reqs[r].ops[k];
        if (op.kind > GENESYS_C5_MMAP || op.len == 0 || (op.kind == GENESYS_C5_PREAD && op.file >= n_in) ||
            (op.kind == GENESYS_C5_MMAP && op.len % 16))
          return set_err(GENESYS_EINVAL, "bad operation");
      }
      const Needs nd = needs_of(reqs[r], bt, cfg.min_part, cfg.pread_to_hbm);
      if (nd.staging > cfg.staging_budget || nd.hbm > cfg.hbm_budget || nd.slots > cfg.slot_budget)
        return set_err(GENESYS_EINVAL, "a request needs more than the whole budget");
    }
    memset(results, 0, sizeof(uint64_t) * GENESYS_C5_MAX_OPS * n_req);
    memset(latency_ns, 0, sizeof(uint64_t) * n_req);
    if (n_req == 0) return 0;

    genesys_dev g0;
    genesys_device_view(c, &g0);
    if (cfg.slot_budget > g0.n_slots) cfg.slot_budget = g0.n_slots;
    const int dev = genesys_internal_device(c);
    if (cudaSetDevice(dev) != cudaSuccess) return set_err(GENESYS_ECUDA, "cudaSetDevice");
    if (cfg.persistent)
      return serve_persistent(c, reqs, n_req, in_fds, n_in, out_fd, cfg, g0, results, latency_ns, stats);

    // device state: per launch slot its ops, results (+ error words) and
    // kernel-grain call records; the input fd table; the HBM landing arena
    const uint32_t K = cfg.max_inflight;
    const size_t per_ops = GENESYS_C5_MAX_OPS * sizeof(genesys_c5_op);
    const size_t per_res = 2 * GENESYS_C5_MAX_OPS * sizeof(unsigned long long);
    const size_t per_ks = kSitesPerReq * sizeof(genesys_ksite);
    const size_t per_slot = (per_ops + per_res + per_ks + 255) & ~size_t(255);
    const size_t fds_off = (size_t)K * per_slot;
    const size_t land_off = (fds_off + n_in * sizeof(int32_t) + 4095) & ~size_t(4095);
    void *scratch = nullptr;
    int rc = genesys_internal_scratch(c, land_off + cfg.hbm_budget + 4096, &scratch);
    if (rc) return rc;
    uint8_t *dbase = (uint8_t *)scratch;
    const uint64_t staging_mark = genesys_internal_staging_mark(c);
    uint8_t *staging = (uint8_t *)genesys_staging(c, cfg.staging_budget + 4096);
    if (!staging) return set_err(GENESYS_ENOMEM, "staging arena too small for staging_budget");
    staging = (uint8_t *)(((uintptr_t)staging + 255) & ~uintptr_t(255));

    std::vector<cudaStream_t> streams(cfg.n_streams, nullptr);
    for (auto &s : streams) {
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        for (auto made : streams)
          if (made) cudaStreamDestroy(made);
        genesys_internal_staging_release(c, staging_mark);
        return set_err(GENESYS_ECUDA, "stream");
      }
    }
    // pinned host mirrors of each slot's ops and results
    uint8_t *hmirror = nullptr;
    if (cudaHostAlloc((void **)&hmirror, (size_t)K * (per_ops + per_res), cudaHostAllocPortable) != cudaSuccess) {
      for (auto s : streams) cudaStreamDestroy(s);
      genesys_internal_staging_release(c, staging_mark);
      return set_err(GENESYS_ECUDA, "pinned mirror");
    }
    std::vector<Launch> slots(K);
    for (auto &L : slots) {
      if (cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) {
        for (auto &M : slots)
          if (M.done) cudaEventDestroy(M.done);
        for (auto s : streams) cudaStreamDestroy(s);
        cudaFreeHost(hmirror);
        genesys_internal_staging_release(c, staging_mark);
        return set_err(GENESYS_ECUDA, "events");
      }
    }
    cudaMemcpy(dbase + fds_off, in_fds, n_in * sizeof(int32_t), cudaMemcpyHostToDevice);

    if (cfg.reserve_mmaps && (rc = reserve_trace_mmaps(c, reqs, n_req, K))) {
      for (auto &L : slots) cudaEventDestroy(L.done);
      for (auto s : streams) cudaStreamDestroy(s);
      cudaFreeHost(hmirror);
      genesys_internal_staging_release(c, staging_mark);
      return rc;
    }

    RangeAlloc st_alloc(cfg.staging_budget), hbm_alloc(cfg.hbm_budget);
    uint32_t slots_free = cfg.slot_budget;
    uint64_t next = 0, retired = 0, launched = 0, calls = 0, admitted_wait_ns = 0;
    uint64_t max_inflight_seen = 0, inflight = 0, graph_launches = 0;
    int err = 0;
    const uint64_t t0 = genesys_mono_ns();
    std::vector<uint64_t> arrival_abs(n_req);
    for (uint32_t r = 0; r < n_req; ++r) arrival_abs[r] = cfg.honor_arrivals ? t0 + reqs[r].arrival_ns : t0;

    auto launch = [&](uint32_t si, uint32_t r) -> int {
      Launch &L = slots[si];
      const genesys_c5_request &q = reqs[r];
      cudaStream_t s = streams[L.stream];
      uint8_t *dslot = dbase + (size_t)si * per_slot;
      genesys_c5_op *d_ops = (genesys_c5_op *)dslot;
      unsigned long long *d_res = (unsigned long long *)(dslot + per_ops);
      genesys_ksite *d_ks = (genesys_ksite *)(dslot + per_ops + per_res);
      uint8_t *h = hmirror + (size_t)si * (per_ops + per_res);
      memcpy(h, q.ops, q.n_ops * sizeof(genesys_c5_op));
      if (cudaMemcpyAsync(d_ops, h, q.n_ops * sizeof(genesys_c5_op), cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaMemsetAsync(d_res, 0, per_res + per_ks, s) != cudaSuccess)
        return -1;
      genesys_dev g = g0;
      g.ksite = d_ks;
      const int32_t *d_fds = (const int32_t *)(dbase + fds_off);
      uint8_t *st = staging + L.st_off;
      uint8_t *land = dbase + land_off + L.hbm_off;
      uint32_t nops = q.n_ops, mp = cfg.min_part, p2h = cfg.pread_to_hbm;
      int32_t ofd = out_fd;
      void *args[] = {&g, &d_ops, &nops, &d_fds, &ofd, &st, &land, &d_res, &mp, &p2h};
      const dim3 grid(L.need.blocks), block(bt);
      if (cfg.use_graphs) {
        cudaKernelNodeParams kp{};
        kp.func = (void *)&c5_request_kernel;
        kp.gridDim = grid;
        kp.blockDim = block;
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        if (!L.exec) {
          // one single-kernel graph per launch slot, instantiated once; later
          // requests on the slot only update the node's parameters
          if (cudaGraphCreate(&L.graph, 0) != cudaSuccess) return -1;
          if (cudaGraphAddKernelNode(&L.node, L.graph, nullptr, 0, &kp) != cudaSuccess) return -1;
          if (cudaGraphInstantiate(&L.exec, L.graph, 0) != cudaSuccess) return -1;
        } else if (cudaGraphExecKernelNodeSetParams(L.exec, L.node, &kp) != cudaSuccess) {
          return -1;
        }
        if (cudaGraphLaunch(L.exec, s) != cudaSuccess) return -1;
        ++graph_launches;
      } else if (cudaLaunchKernel((const void *)&c5_request_kernel, grid, block, args, 0, s) != cudaSuccess) {
        return -1;
      }
      if (cudaMemcpyAsync(h + per_ops, d_res, per_res, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaEventRecord(L.done, s) != cudaSuccess)
        return -1;
      return 0;
    };

    const uint64_t deadline = t0 + cfg.timeout_ns;
    while (retired < n_req && !err) {
      bool progress = false;
      // retire finished requests
      for (uint32_t si = 0; si < K; ++si) {
        Launch &L = slots[si];
        if (!L.busy) continue;
        const cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) { err = GENESYS_ECUDA; break; }
        const uint64_t now = genesys_mono_ns();
        latency_ns[L.req] = now - arrival_abs[L.req];
        const uint64_t *hr = (const uint64_t *)(hmirror + (size_t)si * (per_ops + per_res) + per_ops);
        for (uint32_t k = 0; k < GENESYS_C5_MAX_OPS; ++k)
          results[(size_t)L.req * GENESYS_C5_MAX_OPS + k] = hr[GENESYS_C5_MAX_OPS + k] ? hr[GENESYS_C5_MAX_OPS + k]
                                                                                       : hr[k];
        st_alloc.release(L.st_off, L.need.staging);
        hbm_alloc.release(L.hbm_off, L.need.hbm);
        slots_free += L.need.slots;
        L.busy = false;
        --inflight;
        ++retired;
        progress = true;
      }
      // admit arrived requests, in arrival order, while budgets allow
      while (next < n_req && !err) {
        const uint64_t now = genesys_mono_ns();
        if (arrival_abs[next] > now) break;
        uint32_t si = 0;
        while (si < K && slots[si].busy) ++si;
        if (si == K) break;
        const Needs nd = needs_of(reqs[next], bt, cfg.min_part, cfg.pread_to_hbm);
        if (nd.slots > slots_free) break;
        uint64_t so = 0, ho = 0;
        if (!st_alloc.alloc(nd.staging, &so)) break;
        if (!hbm_alloc.alloc(nd.hbm, &ho)) { st_alloc.release(so, nd.staging); break; }
        Launch &L = slots[si];
        L.busy = true;
        L.req = (uint32_t)next;
        L.need = nd;
        L.st_off = so;
        L.hbm_off = ho;
        // launch slot si owns stream si mod n_streams: with as many streams as
        // launch slots a request never queues behind another on its stream
        L.stream = (int)(si % cfg.n_streams);
        slots_free -= nd.slots;
        admitted_wait_ns += now - arrival_abs[next];
        if (launch(si, (uint32_t)next) != 0) { err = GENESYS_ECUDA; break; }
        ++launched;
        ++inflight;
        max_inflight_seen = std::max(max_inflight_seen, inflight);
        calls += calls_of(reqs[next], nd.blocks, cfg.min_part);
        ++next;
        progress = true;
      }
      if (!progress) {
        if (genesys_mono_ns() > deadline) { err = GENESYS_ETIMEDOUT; break; }
        // nap between event polls: back-to-back cudaEventQuery calls contend
        // with the service threads' CUDA calls
        timespec ts{0, 2000};
        nanosleep(&ts, nullptr);
      }
    }
    const uint64_t t_end = genesys_mono_ns();
    // on failure: wait for what was launched before freeing its resources
    for (auto s : streams) cudaStreamSynchronize(s);
    int drc = genesys_drain(c, 10ull * g0.deadline_ns);
    genesys_reclaim(c);  // no request kernel runs any more: unpin released regions
    for (auto &L : slots) {
      if (L.exec) cudaGraphExecDestroy(L.exec);
      if (L.graph) cudaGraphDestroy(L.graph);
      cudaEventDestroy(L.done);
    }
    for (auto s : streams) cudaStreamDestroy(s);
    cudaFreeHost(hmirror);
    genesys_internal_staging_release(c, staging_mark);
    if (stats) {
      memset(stats, 0, sizeof *stats);
      stats->requests = retired;
      stats->syscalls = calls;
      stats->makespan_ns = t_end - t0;
      stats->max_inflight = max_inflight_seen;
      stats->admission_wait_ns = admitted_wait_ns;
      stats->graph_launches = graph_launches;
    }
    if (err == GENESYS_ETIMEDOUT) return set_err(err, "serve: trace did not finish within timeout_ns");
    if (err) return set_err(err, "serve: a CUDA call failed");
    if (drc) return drc;
    int32_t stw[GENESYS_ST_WORDS];
    rc = genesys_status(c, stw, 1);
    if (rc) return rc;
    if (stw[GENESYS_ST_TIMEOUTS] || stw[GENESYS_ST_FIRST_ERROR]) {
      char msg[160];
      snprintf(msg, sizeof msg, "serve: device-side calls failed: first error %d, %d timeouts",
               stw[GENESYS_ST_FIRST_ERROR], stw[GENESYS_ST_TIMEOUTS]);
      return set_err(GENESYS_EDEVICE, msg);
    }
    return 0;
  });
}
