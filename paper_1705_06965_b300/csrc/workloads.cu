// Data-parallel kernels that make GPU system calls and consume their results,
// and their C-ABI entry points (declared in genesys.h).
//
// Paper: Vesely et al., "GPU System Calls", arXiv 1705.06965.
//   C1  Sec. 6 / Fig. 5   pread microbenchmark (here: pread + byte histogram)
//   C2  Sec. 4.1 / Sec. 6 pwrite at work-item / warp / work-group / kernel grain
//   C6  Sec. 6 / Fig. 6   block permutation + work-group pwrite, 4 ordering x blocking modes
//   probe Sec. 4.1        strong ordering: stores before the call are complete
//   ping-pong             host-link round trip of a flag (the floor of a blocking call)
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "genesys.h"
#include "genesys_device.cuh"
#include "internal.h"

using namespace genesys;

namespace {

// splitmix64 (Steele, Lea & Flood 2014), counter-based: value i of the
// generator whose state starts at `seed`.
__device__ __forceinline__ uint64_t sm64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int set_err(int code, const char *msg) { return genesys_internal_error(code, msg); }

// Launch through the runtime (legality checks, kernel-grain state reset,
// synchronise + drain), then turn device-side failures into GENESYS_EDEVICE.
int run(genesys_ctx *c, const void *kernel, uint32_t grid, uint32_t block, size_t smem, void **args, uint32_t flags,
        void *stream) {
  const uint32_t g3[3] = {grid, 1, 1}, b3[3] = {block, 1, 1};
  int rc = genesys_launch(c, kernel, g3, b3, smem, args, flags | GENESYS_LAUNCH_SYNC, stream);
  if (rc) return rc;
  int32_t st[GENESYS_ST_WORDS];
  rc = genesys_status(c, st, 1);
  if (rc) return rc;
  if (st[GENESYS_ST_TIMEOUTS] || st[GENESYS_ST_FAILED_CALLS] || st[GENESYS_ST_FIRST_ERROR] ||
      st[GENESYS_ST_BAD_ARGS]) {
    char msg[160];
    snprintf(msg, sizeof msg, "device-side calls failed: first error %d, %d timeouts, %d failed calls",
             st[GENESYS_ST_FIRST_ERROR], st[GENESYS_ST_TIMEOUTS], st[GENESYS_ST_FAILED_CALLS]);
    return set_err(GENESYS_EDEVICE, msg);
  }
  return 0;
}

// ------------------------------------------------------------------- C1
// Byte histogram of `n` bytes at `buf` (host-mapped staging, 16-byte aligned)
// into the calling warp's shared-memory copy.  16-byte vector loads, up to
// four in flight per thread, so a block streams the chunk over the host link
// in few round trips.
__device__ __forceinline__ void hist_bytes(const uint8_t *buf, uint64_t n, uint32_t *my) {
  const uint4 *v = reinterpret_cast<const uint4 *>(buf);
  const uint64_t n16 = n >> 4;
#pragma unroll 4
  for (uint64_t i = threadIdx.x; i < n16; i += blockDim.x) {
    const uint4 x = v[i];
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int b = 0; b < 4; ++b) atomicAdd(&my[(w[k] >> (8 * b)) & 0xFFu], 1u);
    }
  }
  for (uint64_t i = (n16 << 4) + threadIdx.x; i < n; i += blockDim.x) atomicAdd(&my[buf[i]], 1u);
}

// The same for one warp: lanes stride the buffer, four loads in flight each.
__device__ __forceinline__ void hist_bytes_warp(const uint8_t *buf, uint64_t n, uint32_t *my, uint32_t lane) {
  const uint4 *v = reinterpret_cast<const uint4 *>(buf);
  const uint64_t n16 = n >> 4;
#pragma unroll 4
  for (uint64_t i = lane; i < n16; i += 32) {
    const uint4 x = v[i];
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int b = 0; b < 4; ++b) atomicAdd(&my[(w[k] >> (8 * b)) & 0xFFu], 1u);
    }
  }
  for (uint64_t i = (n16 << 4) + lane; i < n; i += 32) atomicAdd(&my[buf[i]], 1u);
}

__device__ __forceinline__ void hist_flush(uint32_t *sh, uint32_t *hist_out) {
  __syncthreads();
  const uint32_t nw = blockDim.x >> 5;
  for (uint32_t b = threadIdx.x; b < 256; b += blockDim.x) {
    uint32_t s = 0;
    for (uint32_t w = 0; w < nw; ++w) s += sh[w * 256 + b];
    if (s) atomicAdd(&hist_out[b], s);
  }
}

// Plain form: work-group grain, strong ordering, blocking (the combination
// the paper's microbenchmarks start from).  Block b reads chunks b, b+G, ...
__global__ void __launch_bounds__(1024, 1) c1_plain_kernel(genesys_dev g, int fd, uint64_t file_bytes, uint32_t chunk,
                                                        uint8_t *staging, uint32_t *hist_out) {
  extern __shared__ uint32_t sh[];
  for (uint32_t i = threadIdx.x; i < (blockDim.x >> 5) * 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  uint32_t *my = sh + (threadIdx.x >> 5) * 256;
  uint8_t *buf = staging + (size_t)blockIdx.x * chunk;
  const uint64_t n_chunks = (file_bytes + chunk - 1) / chunk;
  for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const uint64_t off = c * chunk;
    const uint64_t len = file_bytes - off < chunk ? file_bytes - off : chunk;
    // a short read is continued until the chunk is whole or the file ends
    const int64_t r = pread_full<GROUP, STRONG>(g, (uint64_t)fd, buf, len, off);
    if (r <= 0) break;  // r is the same in every thread (broadcast after the call)
    hist_bytes(buf, (uint64_t)r, my);
  }
  hist_flush(sh, hist_out);
}

// HBM form: as the plain form, but the block first moves each chunk from
// staging into its own landing buffer in HBM (16-byte loads over the host
// link, stores to HBM) and builds the histogram from the HBM copy.
__global__ void __launch_bounds__(1024, 1) c1_hbm_kernel(genesys_dev g, int fd, uint64_t file_bytes, uint32_t chunk,
                                                        uint8_t *staging, uint32_t *hist_out, uint8_t *landing) {
  extern __shared__ uint32_t sh[];
  for (uint32_t i = threadIdx.x; i < (blockDim.x >> 5) * 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  uint32_t *my = sh + (threadIdx.x >> 5) * 256;
  uint8_t *buf = staging + (size_t)blockIdx.x * chunk;
  uint8_t *land = landing + (size_t)blockIdx.x * chunk;
  const uint64_t n_chunks = (file_bytes + chunk - 1) / chunk;
  for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const uint64_t off = c * chunk;
    const uint64_t len = file_bytes - off < chunk ? file_bytes - off : chunk;
    const int64_t r = pread_full<GROUP, STRONG>(g, (uint64_t)fd, buf, len, off);
    if (r <= 0) break;  // r is the same in every thread (broadcast after the call)
    const uint64_t n = (uint64_t)r;
    const uint4 *src = reinterpret_cast<const uint4 *>(buf);
    uint4 *dst = reinterpret_cast<uint4 *>(land);
#pragma unroll 4
    for (uint64_t i = threadIdx.x; i < (n + 15) / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    hist_bytes(land, n, my);
    __syncthreads();  // the landing buffer is rewritten by the next chunk
  }
  hist_flush(sh, hist_out);
}

// Warp form: warp grain, strong ordering, blocking.  Every warp of the grid
// reads on its own: global warp w reads chunks w, w + W, ... (W warps in the
// grid) into its own staging piece and counts them into its own shared-memory
// histogram copy, with no block-wide barrier between chunks.
__global__ void __launch_bounds__(1024, 1) c1_warp_kernel(genesys_dev g, int fd, uint64_t file_bytes, uint32_t chunk,
                                                       uint8_t *staging, uint32_t *hist_out) {
  extern __shared__ uint32_t sh[];
  for (uint32_t i = threadIdx.x; i < (blockDim.x >> 5) * 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t *my = sh + wib * 256;
  const uint64_t n_warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  uint8_t *buf = staging + gw * chunk;
  const uint64_t n_chunks = (file_bytes + chunk - 1) / chunk;
  for (uint64_t c = gw; c < n_chunks; c += n_warps) {  // warp-uniform loop
    const uint64_t off = c * chunk;
    const uint64_t len = file_bytes - off < chunk ? file_bytes - off : chunk;
    const int64_t r = pread_full<WARP, STRONG>(g, (uint64_t)fd, buf, len, off);
    if (r <= 0) break;  // r is the same in every lane (broadcast after the call)
    hist_bytes_warp(buf, (uint64_t)r, my, lane);
  }
  hist_flush(sh, hist_out);
}

// Batched form: relaxed, non-blocking preads double-buffered per block - the
// read of chunk k+1 is in flight while chunk k is scanned (Sec. 4.1: weak
// ordering with non-blocking prefetching reads).
template <int D>
__global__ void __launch_bounds__(1024, 1) c1_batched_kernel(genesys_dev g, int fd, uint64_t file_bytes, uint32_t chunk,
                                                          uint8_t *staging, uint32_t *hist_out) {
  extern __shared__ uint32_t sh[];
  __shared__ int64_t r_s;
  for (uint32_t i = threadIdx.x; i < (blockDim.x >> 5) * 256; i += blockDim.x) sh[i] = 0;
  uint32_t *my = sh + (threadIdx.x >> 5) * 256;
  uint8_t *base = staging + (size_t)D * blockIdx.x * chunk;  // D buffers of this block
  const uint64_t n_chunks = (file_bytes + chunk - 1) / chunk;
  const uint64_t n_mine = blockIdx.x < n_chunks ? (n_chunks - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const bool leader = threadIdx.x == 0;
  Ticket t[D];  // the k-th chunk of this block uses ticket and buffer k % D
  auto chunk_off = [&](uint64_t k) { return (blockIdx.x + k * gridDim.x) * (uint64_t)chunk; };
  auto chunk_len = [&](uint64_t off) { return file_bytes - off < chunk ? file_bytes - off : (uint64_t)chunk; };
  auto issue_chunk = [&](uint64_t k) {
    const uint64_t off = chunk_off(k);
    issue(g, &t[k % D], SYS_pread64, (uint64_t)fd, (uint64_t)(base + (k % D) * (uint64_t)chunk), chunk_len(off), off);
  };
  uint64_t issued = 0;
  if (leader)
    for (; issued < D && issued < n_mine; ++issued) issue_chunk(issued);
  __syncthreads();
  for (uint64_t k = 0; k < n_mine; ++k) {
    if (leader) {
      int64_t r = wait(g, t[k % D]);
      // a short read is continued (blocking) until the chunk is whole or the file ends
      const uint64_t off = chunk_off(k), len = chunk_len(off);
      uint8_t *buf = base + (k % D) * (uint64_t)chunk;
      uint64_t got = r > 0 ? ((uint64_t)r < len ? (uint64_t)r : len) : 0;
      while (r > 0 && got < len) {
        Ticket more;
        issue(g, &more, SYS_pread64, (uint64_t)fd, (uint64_t)(buf + got), len - got, off + got);
        r = wait(g, more);
        if (r > 0) got += (uint64_t)r < len - got ? (uint64_t)r : len - got;
      }
      if (r >= 0) r = (int64_t)got;
      if (r <= 0)  // stop early: collect the reads still in flight so that their slots are released
        for (uint64_t j = k + 1; j < issued; ++j) wait(g, t[j % D]);
      r_s = r;
    }
    __syncthreads();  // consumer: barrier after the read completes
    const int64_t r = r_s;
    if (r <= 0) break;
    hist_bytes(base + (k % D) * (uint64_t)chunk, (uint64_t)r, my);
    __syncthreads();  // buffer k % D is free again
    if (leader && issued < n_mine) issue_chunk(issued++);
  }
  hist_flush(sh, hist_out);
}

// ------------------------------------------------------------------- C2
// Marshal: the warp writes its 32 threads' 64-byte patterns (2 KiB, contiguous
// in staging) with lane-interleaved 16-byte stores, so each store instruction
// covers 512 contiguous bytes.  splitmix64 is counter-based, so any lane can
// produce any thread's words.  Threads >= n write nothing.
__device__ __forceinline__ void c2_marshal_warp(uint64_t warp_gid0, uint64_t n, uint64_t seed, uint8_t *staging) {
  const uint32_t lane = lane_id();
  uint64_t *base = reinterpret_cast<uint64_t *>(staging + warp_gid0 * 64);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t w = j * 64 + lane * 2;           // word index within the warp's 256 words
    const uint64_t wi = warp_gid0 * 8 + w;          // global word index
    if (wi / 8 < n) st_v2(base + w, sm64_at(seed, wi), sm64_at(seed, wi + 1));
  }
}

template <int G, int O, int B>
__global__ void __launch_bounds__(1024) c2_pwrite_kernel(genesys_dev g, int fd, uint64_t n, uint64_t seed,
                                                         uint8_t *staging) {
  const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (G == KERNEL) {
    // grid-stride over warps' payloads (the grid may be smaller than n when the
    // launch is cooperative), then one call for the whole kernel
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = gid - lane_id(); t < n; t += stride) c2_marshal_warp(t, n, seed, staging);
    __syncwarp();
    call<KERNEL, O, B>(g, SYS_pwrite64, (uint64_t)fd, (uint64_t)staging, n * 64, 0);
    return;
  }
  const uint64_t warp0 = gid - lane_id();
  if (warp0 < n) c2_marshal_warp(warp0, n, seed, staging);
  __syncwarp();
  if (G == GROUP) {
    const uint64_t b0 = (uint64_t)blockIdx.x * blockDim.x;
    const uint64_t cnt = n - b0 < blockDim.x ? n - b0 : blockDim.x;
    call<GROUP, O, B>(g, SYS_pwrite64, (uint64_t)fd, (uint64_t)(staging + b0 * 64), cnt * 64, b0 * 64);
    return;
  }
  if (gid >= n) return;
  if (G == ITEM) {
    call<ITEM, STRONG, B>(g, SYS_pwrite64, (uint64_t)fd, (uint64_t)(staging + gid * 64), 64, gid * 64);
  } else {
    call_warp_coalesced<O, B>(g, SYS_pwrite64, fd, (uint64_t)(staging + gid * 64), 64, gid * 64);
  }
}

// ------------------------------------------------------- visibility probe
// Every thread stores its word, then the group's caller asks the CPU to check
// that all of the group's words are visible.  R = ROLE_PRODUCER puts the
// barrier before the call under relaxed ordering (the stores must be
// complete); R = ROLE_CONSUMER omits it, so stores may legitimately still be
// in flight (violations allowed).
template <int G, int O, int R>
__global__ void __launch_bounds__(1024) visibility_kernel(genesys_dev g, uint64_t n, uint64_t seed, uint64_t *probe,
                                                          unsigned long long *viol) {
  const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (G == KERNEL) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = gid; t < n; t += stride) probe[t] = sm64_at(seed, t);
    const int64_t r = call_at<KERNEL, O, BLOCKING, R>(g, 0, GENESYS_NR_CHECK_VISIBLE, (uint64_t)probe, n, seed, 0);
    if (r > 0) atomicAdd(viol, (unsigned long long)r);
    return;
  }
  if (gid < n) probe[gid] = sm64_at(seed, gid);
  if (G == ITEM) {
    if (gid >= n) return;
    const int64_t r = call<ITEM, STRONG, BLOCKING, R>(g, GENESYS_NR_CHECK_VISIBLE, (uint64_t)(probe + gid), 1, seed, gid);
    if (r > 0) atomicAdd(viol, (unsigned long long)r);
    return;
  }
  if (G == WARP) {
    if (gid >= n) return;
    const uint32_t active = __activemask();
    const uint64_t first = gid - lane_id();          // in-range lanes start at lane 0
    const uint64_t cnt = __popc(active);
    const int64_t r = call<WARP, O, BLOCKING, R>(g, GENESYS_NR_CHECK_VISIBLE, (uint64_t)(probe + first), cnt, seed, first);
    if (lane_id() == 0 && r > 0) atomicAdd(viol, (unsigned long long)r);
    return;
  }
  const uint64_t b0 = (uint64_t)blockIdx.x * blockDim.x;
  const uint64_t cnt = n - b0 < blockDim.x ? n - b0 : blockDim.x;
  const int64_t r = call<GROUP, O, BLOCKING, R>(g, GENESYS_NR_CHECK_VISIBLE, (uint64_t)(probe + b0), cnt, seed, b0);
  if (threadIdx.x == 0 && r > 0) atomicAdd(viol, (unsigned long long)r);
}

// ------------------------------------------------------------------- C6
// Block permutation (Sec. 6, Fig. 6): block b of the input (8 KiB) is staged
// in shared memory, permuted `iters` times with out[i] = in[perm[i]], written
// to host-mapped staging and then to the file with a work-group pwrite at
// offset b * 8 KiB.  Ordering and blocking of that pwrite are the four
// combinations the paper compares.
template <int O, int B>
__global__ void __launch_bounds__(1024) c6_permute_kernel(genesys_dev g, int fd, const uint8_t *input,
                                                          const uint16_t *perm, uint32_t iters, uint8_t *staging) {
  __shared__ __align__(16) uint8_t buf[2][8192];
  __shared__ __align__(16) uint16_t p[8192];
  const uint64_t blk = blockIdx.x;
  const uint4 *in4 = reinterpret_cast<const uint4 *>(input + blk * 8192);
  for (uint32_t i = threadIdx.x; i < 512; i += blockDim.x) reinterpret_cast<uint4 *>(buf[0])[i] = in4[i];
  for (uint32_t i = threadIdx.x; i < 1024; i += blockDim.x)
    reinterpret_cast<uint4 *>(p)[i] = reinterpret_cast<const uint4 *>(perm)[i];
  __syncthreads();
  uint32_t cur = 0;
  for (uint32_t it = 0; it < iters; ++it) {
    for (uint32_t i = threadIdx.x; i < 8192; i += blockDim.x) buf[cur ^ 1][i] = buf[cur][p[i]];
    __syncthreads();
    cur ^= 1;
  }
  uint8_t *dst = staging + blk * 8192;
  for (uint32_t i = threadIdx.x; i < 512; i += blockDim.x)
    reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(buf[cur])[i];
  call<GROUP, O, B>(g, SYS_pwrite64, (uint64_t)fd, (uint64_t)dst, 8192, blk * 8192);
}

// One system call made by GPU code: every thread of a `threads`-wide block
// takes part at the given granularity (the caller is the designated thread),
// and thread 0 stores the result.  Any call the context allows can be made
// this way (open, read, write, lseek, close, madvise, ...).
template <int G>
__global__ void one_call_kernel(genesys_dev g, uint32_t nr, uint64_t a0, uint64_t a1, uint64_t a2, uint64_t a3,
                                uint64_t a4, uint64_t a5, long long *ret) {
  const int64_t r = call<G, STRONG, BLOCKING>(g, nr, a0, a1, a2, a3, a4, a5);
  if (threadIdx.x == 0) *ret = r;
}

template <int G, int O, int B>
const void *c2_kernel_ptr() {
  return reinterpret_cast<const void *>(&c2_pwrite_kernel<G, O, B>);
}

const void *c2_select(uint32_t gran, bool relaxed, bool nonblocking) {
#define C2_CASE(G)                                                                      \
  if (gran == G) {                                                                      \
    if (!relaxed && !nonblocking) return c2_kernel_ptr<G, STRONG, BLOCKING>();          \
    if (!relaxed && nonblocking) return c2_kernel_ptr<G, STRONG, NONBLOCKING>();        \
    if (relaxed && !nonblocking) return c2_kernel_ptr<G, RELAXED, BLOCKING>();          \
    return c2_kernel_ptr<G, RELAXED, NONBLOCKING>();                                    \
  }
  if (gran == ITEM) {
    if (relaxed) return nullptr;
    return nonblocking ? c2_kernel_ptr<ITEM, STRONG, NONBLOCKING>() : c2_kernel_ptr<ITEM, STRONG, BLOCKING>();
  }
  C2_CASE(WARP)
  C2_CASE(GROUP)
  C2_CASE(KERNEL)
#undef C2_CASE
  return nullptr;
}

template <int G, int O, int R>
const void *vis_ptr() {
  return reinterpret_cast<const void *>(&visibility_kernel<G, O, R>);
}

// Host-link round trip: one GPU thread stores `r` to `ping` (host-mapped) and
// waits for the host to store `r` to `pong`, for r = 1 .. rounds; the wait is
// bounded by deadline_ns.  out[0] = elapsed ns, out[1] = rounds completed,
// out[2] = 1 if the deadline ended it.
__global__ void pingpong_kernel(uint64_t *ping, const uint64_t *pong, uint32_t rounds, uint64_t deadline_ns,
                                unsigned long long *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint64_t t0 = now_ns();
  uint32_t done = 0;
  bool late = false;
  for (uint32_t r = 1; r <= rounds && !late; ++r) {
    st_release_sys(ping, r);
    while (ld_acquire_sys(pong) != r) {
      if (now_ns() - t0 > deadline_ns) { late = true; break; }
    }
    if (!late) done = r;
  }
  out[0] = now_ns() - t0;
  out[1] = done;
  out[2] = late ? 1ull : 0ull;
}

// Zero-copy streaming over the host link: every thread of the grid reads
// (or writes) 16-byte words of pinned host memory, four independent accesses
// in flight per thread.  The reads fold into one word that is compared with a
// value it practically never takes, so they cannot be dropped.
__global__ void link_read_kernel(const uint4 *__restrict__ p, uint64_t n16, unsigned long long *sink) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x = 0;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const uint4 a = p[i], b = p[i + stride], c = p[i + 2 * stride], d = p[i + 3 * stride];
    x ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
  }
  for (; i < n16; i += stride) {
    const uint4 a = p[i];
    x ^= a.x ^ a.y ^ a.z ^ a.w;
  }
  if (x == 0x9E3779B9u) atomicAdd(sink, 1ull);
}

__global__ void link_write_kernel(uint4 *__restrict__ p, uint64_t n16) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
    p[i] = make_uint4((uint32_t)i, (uint32_t)(i >> 32), ~(uint32_t)i, 0x5EEDu);
}

// Both directions at once: the even blocks read the first n16_half words,
// the odd blocks write the next n16_half (as the two kernels above do).
__global__ void link_both_kernel(uint4 *__restrict__ p, uint64_t n16_half, unsigned long long *sink) {
  const uint64_t half_blocks = gridDim.x / 2;
  const uint64_t stride = half_blocks * blockDim.x;
  const uint64_t first = (uint64_t)(blockIdx.x / 2) * blockDim.x + threadIdx.x;
  if (blockIdx.x / 2 >= half_blocks) return;  // an odd grid's last block
  if (blockIdx.x % 2 == 0) {
    uint32_t x = 0;
    uint64_t i = first;
    for (; i + 3 * stride < n16_half; i += 4 * stride) {
      const uint4 a = p[i], b = p[i + stride], c = p[i + 2 * stride], d = p[i + 3 * stride];
      x ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
    }
    for (; i < n16_half; i += stride) {
      const uint4 a = p[i];
      x ^= a.x ^ a.y ^ a.z ^ a.w;
    }
    if (x == 0x9E3779B9u) atomicAdd(sink, 1ull);
  } else {
    uint4 *q = p + n16_half;
    for (uint64_t i = first; i < n16_half; i += stride)
      q[i] = make_uint4((uint32_t)i, (uint32_t)(i >> 32), ~(uint32_t)i, 0x5EEDu);
  }
}

// Clock alignment: round r, one GPU thread reads its clock, stores r to
// `ping`, waits for the host to answer r on `pong` and reads its clock again;
// t[2r], t[2r + 1] = the two readings.  Bounded by deadline_ns.
__global__ void clock_probe_kernel(uint64_t *ping, const uint64_t *pong, uint32_t rounds, uint64_t deadline_ns,
                                   unsigned long long *t, unsigned long long *late) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint64_t t0 = now_ns();
  for (uint32_t r = 1; r <= rounds; ++r) {
    const uint64_t a = now_ns();
    st_release_sys(ping, r);
    while (ld_acquire_sys(pong) != r) {
      if (now_ns() - t0 > deadline_ns) { *late = 1; return; }
    }
    t[2 * (r - 1)] = a;
    t[2 * (r - 1) + 1] = now_ns();
  }
}

}  // namespace

extern "C" {

int genesys_c1_histogram(genesys_ctx *c, int fd, uint64_t file_bytes, uint64_t chunk, uint32_t groups,
                         uint32_t threads, uint32_t form, void *staging, uint64_t staging_bytes, uint32_t *hist_dev,
                         void *stream) {
  if (!c || !staging || !hist_dev) return set_err(GENESYS_EINVAL, "NULL argument");
  if (fd < 0) return set_err(GENESYS_EINVAL, "bad fd");
  if (chunk == 0 || chunk % 16 || chunk > (1u << 30)) return set_err(GENESYS_EINVAL, "chunk must be a multiple of 16");
  if (groups == 0 || threads < 32 || threads > 1024 || threads % 32) return set_err(GENESYS_EINVAL, "bad launch shape");
  if ((uintptr_t)staging % 16) return set_err(GENESYS_EINVAL, "staging must be 16-byte aligned");
  if (form > GENESYS_FORM_HBM) return set_err(GENESYS_EINVAL, "form: GENESYS_FORM_PLAIN, _BATCHED, _WARP or _HBM");
  const uint64_t need = (uint64_t)groups * chunk *
                        (form == GENESYS_FORM_BATCHED ? 2 : form == GENESYS_FORM_WARP ? threads / 32 : 1);
  if (staging_bytes < need) return set_err(GENESYS_EINVAL, "staging too small");
  // the batched form keeps as many reads in flight per block as the staging
  // holds buffers for (2..4)
  uint32_t depth = (uint32_t)std::min<uint64_t>(4, staging_bytes / ((uint64_t)groups * chunk));
  if (file_bytes == 0) return 0;
  genesys_dev g;
  genesys_device_view(c, &g);
  if (form == GENESYS_FORM_BATCHED && g.n_slots < 2ull * groups)
    return set_err(GENESYS_EINVAL, "the batched form holds two slots per block: n_slots must be >= 2 * groups");
  while (depth > 2 && g.n_slots < (uint64_t)depth * groups) --depth;
  uint32_t ch = (uint32_t)chunk;
  uint8_t *st = (uint8_t *)staging;
  void *args[] = {&g, &fd, &file_bytes, &ch, &st, &hist_dev};
  const size_t smem = (size_t)(threads / 32) * 256 * 4;
  if (form == GENESYS_FORM_BATCHED) {
    const void *k = depth >= 4 ? (const void *)&c1_batched_kernel<4>
                  : depth == 3 ? (const void *)&c1_batched_kernel<3> : (const void *)&c1_batched_kernel<2>;
    return run(c, k, groups, threads, smem, args,
               GENESYS_GRAN_GROUP | GENESYS_LAUNCH_RELAXED | GENESYS_LAUNCH_NONBLOCKING, stream);
  }
  if (form == GENESYS_FORM_WARP)
    return run(c, (const void *)&c1_warp_kernel, groups, threads, smem, args, GENESYS_GRAN_WARP, stream);
  if (form == GENESYS_FORM_HBM) {
    void *landing = nullptr;  // the context's device scratch: one chunk per block
    const int rc = genesys_internal_scratch(c, (size_t)groups * chunk, &landing);
    if (rc) return rc;
    uint8_t *land = (uint8_t *)landing;
    void *hargs[] = {&g, &fd, &file_bytes, &ch, &st, &hist_dev, &land};
    return run(c, (const void *)&c1_hbm_kernel, groups, threads, smem, hargs, GENESYS_GRAN_GROUP, stream);
  }
  return run(c, (const void *)&c1_plain_kernel, groups, threads, smem, args, GENESYS_GRAN_GROUP, stream);
}

int genesys_c2_pwrite(genesys_ctx *c, int fd, uint64_t n, uint32_t gran, uint32_t bt, uint32_t relaxed,
                      uint32_t nonblocking, uint64_t seed, void *staging, uint64_t staging_bytes, void *stream) {
  if (!c || !staging) return set_err(GENESYS_EINVAL, "NULL argument");
  if (fd < 0) return set_err(GENESYS_EINVAL, "bad fd");
  if (gran > GENESYS_GRAN_KERNEL || bt < 32 || bt > 1024 || bt % 32) return set_err(GENESYS_EINVAL, "bad shape");
  if (staging_bytes < n * 64 || (uintptr_t)staging % 16) return set_err(GENESYS_EINVAL, "staging too small or unaligned");
  if (n == 0) return 0;
  const void *k = c2_select(gran, relaxed != 0, nonblocking != 0);
  if (!k) return set_err(GENESYS_EINVAL, "work-item grain calls are always strongly ordered (Sec. 4.1)");
  genesys_dev g;
  genesys_device_view(c, &g);
  uint64_t blocks = (n + bt - 1) / bt;
  if (gran == GENESYS_GRAN_KERNEL && !relaxed) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)bt, 0) != cudaSuccess || per_sm == 0)
      return set_err(GENESYS_ECUDA, "occupancy query failed");
    const uint64_t cap = (uint64_t)per_sm * g.n_sms;
    if (blocks > cap) blocks = cap;
  }
  if (blocks > 0x7FFFFFFFull) return set_err(GENESYS_EINVAL, "too many threads");
  uint8_t *st = (uint8_t *)staging;
  void *args[] = {&g, &fd, &n, &seed, &st};
  const uint32_t flags = gran | (relaxed ? GENESYS_LAUNCH_RELAXED : 0) | (nonblocking ? GENESYS_LAUNCH_NONBLOCKING : 0);
  return run(c, k, (uint32_t)blocks, bt, 0, args, flags, stream);
}

int genesys_c6_permute(genesys_ctx *c, int fd, const uint8_t *input_dev, const uint16_t *perm_dev, uint64_t n_blocks,
                       uint32_t iters, uint32_t relaxed, uint32_t nonblocking, void *staging, uint64_t staging_bytes,
                       void *stream) {
  if (!c || !input_dev || !perm_dev || !staging) return set_err(GENESYS_EINVAL, "NULL argument");
  if (fd < 0) return set_err(GENESYS_EINVAL, "bad fd");
  if (n_blocks == 0) return 0;
  if (n_blocks > 0x7FFFFFFFull) return set_err(GENESYS_EINVAL, "too many blocks");
  if (staging_bytes < n_blocks * 8192 || (uintptr_t)staging % 16 || (uintptr_t)input_dev % 16 ||
      (uintptr_t)perm_dev % 16)
    return set_err(GENESYS_EINVAL, "staging >= n_blocks * 8 KiB; 16-byte aligned buffers");
  const void *k = relaxed ? (nonblocking ? (const void *)&c6_permute_kernel<RELAXED, NONBLOCKING>
                                         : (const void *)&c6_permute_kernel<RELAXED, BLOCKING>)
                          : (nonblocking ? (const void *)&c6_permute_kernel<STRONG, NONBLOCKING>
                                         : (const void *)&c6_permute_kernel<STRONG, BLOCKING>);
  genesys_dev g;
  genesys_device_view(c, &g);
  uint8_t *st = (uint8_t *)staging;
  void *args[] = {&g, &fd, &input_dev, &perm_dev, &iters, &st};
  const uint32_t flags = GENESYS_GRAN_GROUP | (relaxed ? GENESYS_LAUNCH_RELAXED : 0) |
                         (nonblocking ? GENESYS_LAUNCH_NONBLOCKING : 0);
  return run(c, k, (uint32_t)n_blocks, 1024, 0, args, flags, stream);
}

int genesys_gpu_call(genesys_ctx *c, uint32_t nr, const uint64_t args[6], uint32_t gran, uint32_t threads,
                     long long *ret_dev, void *stream) {
  if (!c || !args || !ret_dev) return set_err(GENESYS_EINVAL, "NULL argument");
  if (threads == 0 || threads > 1024 || (gran == GENESYS_GRAN_WARP && threads > 32) || gran > GENESYS_GRAN_GROUP)
    return set_err(GENESYS_EINVAL, "one block of 1..1024 threads; work-item, warp (<= 32 threads) or work-group");
  if (gran == GENESYS_GRAN_ITEM && threads != 1) return set_err(GENESYS_EINVAL, "work-item grain: one thread");
  genesys_dev g;
  genesys_device_view(c, &g);
  uint64_t a0 = args[0], a1 = args[1], a2 = args[2], a3 = args[3], a4 = args[4], a5 = args[5];
  void *kargs[] = {&g, &nr, &a0, &a1, &a2, &a3, &a4, &a5, &ret_dev};
  const void *k = gran == GENESYS_GRAN_ITEM   ? (const void *)&one_call_kernel<ITEM>
                  : gran == GENESYS_GRAN_WARP ? (const void *)&one_call_kernel<WARP>
                                              : (const void *)&one_call_kernel<GROUP>;
  const uint32_t g3[3] = {1, 1, 1}, b3[3] = {threads, 1, 1};
  int rc = genesys_launch(c, k, g3, b3, 0, kargs, gran | GENESYS_LAUNCH_SYNC, stream);
  if (rc) return rc;
  int32_t st[GENESYS_ST_WORDS];
  rc = genesys_status(c, st, 1);
  if (rc) return rc;
  if (st[GENESYS_ST_TIMEOUTS] || st[GENESYS_ST_FIRST_ERROR]) return set_err(GENESYS_EDEVICE, "device wait timed out");
  return 0;
}

int genesys_visibility_probe(genesys_ctx *c, uint64_t n, uint32_t gran, uint32_t bt, uint32_t relaxed, uint64_t seed,
                             uint64_t *probe, unsigned long long *viol, void *stream) {
  if (!c || !probe || !viol) return set_err(GENESYS_EINVAL, "NULL argument");
  if (gran > GENESYS_GRAN_KERNEL || bt < 32 || bt > 1024 || bt % 32) return set_err(GENESYS_EINVAL, "bad shape");
  if (n == 0) return 0;
  const void *k = nullptr;
  // relaxed runs use the consumer role (no barrier before the call): the
  // configuration in which the check may legitimately see missing stores
  switch (gran) {
    case GENESYS_GRAN_ITEM: k = relaxed ? nullptr : vis_ptr<ITEM, STRONG, ROLE_PRODUCER>(); break;
    case GENESYS_GRAN_WARP: k = relaxed ? vis_ptr<WARP, RELAXED, ROLE_CONSUMER>() : vis_ptr<WARP, STRONG, ROLE_PRODUCER>(); break;
    case GENESYS_GRAN_GROUP: k = relaxed ? vis_ptr<GROUP, RELAXED, ROLE_CONSUMER>() : vis_ptr<GROUP, STRONG, ROLE_PRODUCER>(); break;
    default: k = relaxed ? vis_ptr<KERNEL, RELAXED, ROLE_CONSUMER>() : vis_ptr<KERNEL, STRONG, ROLE_PRODUCER>(); break;
  }
  if (!k) return set_err(GENESYS_EINVAL, "work-item grain calls are always strongly ordered (Sec. 4.1)");
  genesys_dev g;
  genesys_device_view(c, &g);
  uint64_t blocks = (n + bt - 1) / bt;
  if (gran == GENESYS_GRAN_KERNEL && !relaxed) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)bt, 0) != cudaSuccess || per_sm == 0)
      return set_err(GENESYS_ECUDA, "occupancy query failed");
    const uint64_t cap = (uint64_t)per_sm * g.n_sms;
    if (blocks > cap) blocks = cap;
  }
  void *args[] = {&g, &n, &seed, &probe, &viol};
  const uint32_t flags = gran | (relaxed ? GENESYS_LAUNCH_RELAXED : 0);
  return run(c, k, (uint32_t)blocks, bt, 0, args, flags, stream);
}

int genesys_internal_clock_offset(int device, uint32_t rounds, uint64_t timeout_ns, int64_t *offset_ns,
                                  uint64_t *rtt_ns) {
  return genesys_guard("genesys_internal_clock_offset", [&]() -> int {
    if (!offset_ns || rounds == 0) return set_err(GENESYS_EINVAL, "bad argument");
    if (cudaSetDevice(device) != cudaSuccess) return set_err(GENESYS_ECUDA, "cudaSetDevice");
    uint64_t *flags = nullptr;
    if (cudaHostAlloc((void **)&flags, 128, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
      return set_err(GENESYS_ECUDA, "cudaHostAlloc");
    memset(flags, 0, 128);
    uint64_t *d_flags = nullptr;
    unsigned long long *d_t = nullptr;
    cudaStream_t st = nullptr;
    int rc = 0;
    if (cudaHostGetDevicePointer((void **)&d_flags, flags, 0) != cudaSuccess ||
        cudaMalloc((void **)&d_t, (2ull * rounds + 1) * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(d_t, 0, (2ull * rounds + 1) * sizeof(unsigned long long)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
      rc = set_err(GENESYS_ECUDA, "clock probe set-up");
    if (rc == 0) {
      std::vector<uint64_t> host_t(rounds, 0);
      bool host_late = false;
      volatile uint64_t *ping = flags, *pong = flags + 8;
      std::thread echo([&] {
        const uint64_t until = genesys_mono_ns() + timeout_ns + 1000000000ull;
        for (uint32_t r = 1; r <= rounds; ++r) {
          while (__atomic_load_n(ping, __ATOMIC_ACQUIRE) != r) {
            if (genesys_mono_ns() > until) { host_late = true; return; }
            __builtin_ia32_pause();
          }
          host_t[r - 1] = genesys_mono_ns();
          __atomic_store_n(pong, (uint64_t)r, __ATOMIC_RELEASE);
        }
      });
      clock_probe_kernel<<<1, 32, 0, st>>>(d_flags, d_flags + 8, rounds, timeout_ns, d_t, d_t + 2ull * rounds);
      const cudaError_t e = cudaStreamSynchronize(st);
      echo.join();
      std::vector<unsigned long long> t(2ull * rounds + 1);
      if (e != cudaSuccess || cudaMemcpy(t.data(), d_t, t.size() * sizeof(t[0]), cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = set_err(GENESYS_ECUDA, "clock probe kernel");
      } else if (t[2ull * rounds] || host_late) {
        rc = set_err(GENESYS_ETIMEDOUT, "clock probe: rounds did not complete within the timeout");
      } else {
        uint64_t best = ~0ull;
        int64_t off = 0;
        for (uint32_t r = 0; r < rounds; ++r) {
          const uint64_t a = t[2 * r], b = t[2 * r + 1];
          if (b - a < best) {
            best = b - a;
            off = (int64_t)host_t[r] - (int64_t)(a + (b - a) / 2);
          }
        }
        *offset_ns = off;
        if (rtt_ns) *rtt_ns = best;
      }
    }
    if (st) cudaStreamDestroy(st);
    if (d_t) cudaFree(d_t);
    cudaFreeHost(flags);
    return rc;
  });
}

// Round-trip latency of a flag between a GPU thread and a host thread over
// the host link (the floor under any blocking GPU system call).
int genesys_link_pingpong(int device, uint32_t rounds, uint64_t timeout_ns, uint64_t *ns_per_round) {
  return genesys_guard("genesys_link_pingpong", [&]() -> int {
    if (!ns_per_round || rounds == 0) return set_err(GENESYS_EINVAL, "NULL argument or zero rounds");
    if (cudaSetDevice(device) != cudaSuccess) return set_err(GENESYS_ECUDA, "cudaSetDevice");
    uint64_t *flags = nullptr;  // ping in line 0, pong in line 1 (separate 64-byte lines)
    if (cudaHostAlloc((void **)&flags, 128, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
      return set_err(GENESYS_ECUDA, "cudaHostAlloc");
    memset(flags, 0, 128);
    uint64_t *d_flags = nullptr;
    unsigned long long *d_out = nullptr;
    cudaStream_t st = nullptr;
    int rc = 0;
    if (cudaHostGetDevicePointer((void **)&d_flags, flags, 0) != cudaSuccess ||
        cudaMalloc((void **)&d_out, 3 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      rc = set_err(GENESYS_ECUDA, "pingpong set-up");
    }
    bool host_late = false;
    if (rc == 0) {
      volatile uint64_t *ping = flags, *pong = flags + 8;
      std::thread echo([&] {
        const uint64_t until = genesys_mono_ns() + timeout_ns + 1000000000ull;
        for (uint32_t r = 1; r <= rounds; ++r) {
          while (__atomic_load_n(ping, __ATOMIC_ACQUIRE) != r) {
            if (genesys_mono_ns() > until) { host_late = true; return; }
            __builtin_ia32_pause();
          }
          __atomic_store_n(pong, (uint64_t)r, __ATOMIC_RELEASE);
        }
      });
      pingpong_kernel<<<1, 32, 0, st>>>(d_flags, d_flags + 8, rounds, timeout_ns, d_out);
      const cudaError_t e = cudaStreamSynchronize(st);
      echo.join();
      unsigned long long out[3] = {0, 0, 0};
      if (e != cudaSuccess || cudaMemcpy(out, d_out, sizeof out, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = set_err(GENESYS_ECUDA, "pingpong kernel");
      else if (out[2] || host_late || out[1] != rounds)
        rc = set_err(GENESYS_ETIMEDOUT, "pingpong: rounds did not complete within the timeout");
      else
        *ns_per_round = out[0] / rounds;
    }
    if (st) cudaStreamDestroy(st);
    if (d_out) cudaFree(d_out);
    cudaFreeHost(flags);
    return rc;
  });
}

// Zero-copy bandwidth of the SMs over the host link: the ceiling of a kernel
// that reads what the service copied into pinned staging (or writes what a
// pwrite will send).  Best of `reps` timed launches after one warm-up.
int genesys_link_stream(int device, void *host_buf, uint64_t bytes, int write, uint32_t blocks, uint32_t threads,
                        uint32_t reps, double *gb_per_s) {
  return genesys_guard("genesys_link_stream", [&]() -> int {
    if (!host_buf || !gb_per_s || bytes < 16 || bytes % 16 || (uintptr_t)host_buf % 16 || reps == 0)
      return set_err(GENESYS_EINVAL, "a 16-byte aligned buffer of a positive multiple of 16 bytes, reps >= 1");
    if (blocks == 0 || blocks > 65535 || threads == 0 || threads > 1024 || threads % 32)
      return set_err(GENESYS_EINVAL, "blocks 1..65535, threads a multiple of 32 up to 1024");
    if (write < 0 || write > 2 || (write == 2 && (blocks < 2 || bytes % 32)))
      return set_err(GENESYS_EINVAL, "write 0, 1 or 2 (both: at least 2 blocks and a multiple of 32 bytes)");
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return set_err(GENESYS_ECUDA, "cudaSetDevice");
    uint4 *d_buf = nullptr;
    unsigned long long *d_sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    if (cudaHostGetDevicePointer((void **)&d_buf, host_buf, 0) != cudaSuccess) {
      cudaGetLastError();
      rc = set_err(GENESYS_EINVAL, "host_buf is not pinned, host-mapped memory");
    } else if (cudaMalloc((void **)&d_sink, sizeof(unsigned long long)) != cudaSuccess ||
               cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
               cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = set_err(GENESYS_ECUDA, "link stream set-up");
    }
    const uint64_t n16 = bytes / 16;
    float best = 0.0f;
    for (uint32_t r = 0; rc == 0 && r <= reps; ++r) {
      cudaEventRecord(e0, st);
      if (write == 2) link_both_kernel<<<blocks, threads, 0, st>>>(d_buf, n16 / 2, d_sink);
      else if (write) link_write_kernel<<<blocks, threads, 0, st>>>(d_buf, n16);
      else link_read_kernel<<<blocks, threads, 0, st>>>(d_buf, n16, d_sink);
      cudaEventRecord(e1, st);
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = set_err(GENESYS_ECUDA, "link stream kernel");
      } else if (r > 0 && ms > 0.0f && (best == 0.0f || ms < best)) {
        best = ms;  // launch 0 is the warm-up
      }
    }
    if (rc == 0 && best <= 0.0f) rc = set_err(GENESYS_ECUDA, "link stream: no timed launch");
    if (rc == 0) *gb_per_s = (double)bytes / (best * 1e-3) / 1e9;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (d_sink) cudaFree(d_sink);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
  });
}

}  // extern "C"
