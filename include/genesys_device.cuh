/*
 * genesys_device.cuh - device side of GPU system calls (sm_103a).
 *
 * A GPU kernel invokes a Linux system call with function-like semantics
 * (Sec. 5, "Invoking GPU system calls"):
 *
 *     int64_t r = genesys::call<Gran, Order, Block>(dev, SYS_pread64, fd, buf, len, off);
 *
 *   Gran  - invocation granularity (Sec. 4.1): ITEM (every calling thread is its
 *           own caller), WARP (the active lanes of a warp; the lowest active
 *           lane calls for them), GROUP (the thread block, the paper's
 *           work-group; thread 0 calls) or KERNEL (the whole grid; one
 *           elected thread calls).  Every thread of the group must make the
 *           call (uniform control flow per group); the designated caller's
 *           arguments are used (Sec. 5).
 *   Order - STRONG: a group barrier before and after the call; RELAXED: a
 *           barrier only before a producer call (write/send-like) and only
 *           after a consumer call (read/recv-like) (Sec. 4.1, Sec. 5).  ITEM is
 *           always strong (Sec. 4.1).  KERNEL+STRONG needs a cooperative launch
 *           (the paper forbids it because a grid larger than the resident set
 *           would deadlock, Sec. 4.1; a cooperative launch caps the grid at the
 *           resident set, which removes that case).
 *   Block - BLOCKING: the caller waits for the result, which is then returned
 *           to every thread that passes the barrier after the call (a relaxed
 *           producer has no such barrier: only the caller waits, the paper's
 *           "one wavefront waits"); NONBLOCKING: returns 0 at once, the CPU
 *           processes the call later (Sec. 4.1 "Blocking versus non-blocking").
 *
 * Results follow the raw Linux convention: >= 0, or -errno.  No wait in this
 * file is unbounded: every spin gives up after dev.deadline_ns, returns
 * -ETIMEDOUT and records it in dev.status.
 *
 * Pointer arguments must be addresses the host can use: pinned host-mapped
 * memory (genesys_staging), or memory the GPU obtained through mmap.
 *
 * Checked builds (GENESYS_DEVICE_CHECKS defined) test the indices this file
 * and the workload kernels compute (slot, ring, buffer offsets) before using
 * them; a failed check counts in dev.status[GENESYS_ST_BAD_ARGS], records
 * -EINVAL as the first error and skips the access, so a bug shows as a status
 * word instead of a fault.
 */
#ifndef GENESYS_DEVICE_CUH
#define GENESYS_DEVICE_CUH

#include <stdint.h>
#include <sys/syscall.h>

#include "genesys_layout.h"

namespace genesys {

enum Gran { ITEM = 0, WARP = 1, GROUP = 2, KERNEL = 3 };
enum Order { STRONG = 0, RELAXED = 1 };
enum Block { BLOCKING = 0, NONBLOCKING = 1 };
/* Role of a call (Sec. 4.1 "System call ordering semantics"). */
enum Role { ROLE_AUTO = 0, ROLE_PRODUCER = 1, ROLE_CONSUMER = 2, ROLE_BOTH = 3 };

constexpr int64_t kETIMEDOUT = 110;

/* ------------------------------------------------------------ primitives */

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_sys(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(uint64_t *p, uint64_t v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_sys() { asm volatile("fence.acq_rel.sys;" ::: "memory"); }
__device__ __forceinline__ void st_relaxed_sys(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
/* 16-byte store to (host-mapped) memory */
__device__ __forceinline__ void st_v2(uint64_t *p, uint64_t a, uint64_t b) {
  asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ uint32_t lane_id() {
  uint32_t l;
  asm("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}

/* Hardware id of the calling lane: (SM, warp slot, lane).  The paper indexes
 * the syscall area by the hardware id of the active work-item (Sec. 5); here it
 * is the first slot a lane tries, so that concurrent callers rarely collide. */
__device__ __forceinline__ uint32_t hw_lane_id() {
  uint32_t sm, w;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
  asm volatile("mov.u32 %0, %%warpid;" : "=r"(w));
  return (sm * 64u + (w & 63u)) * 32u + lane_id();
}

__device__ __forceinline__ int role_of(uint32_t nr) {
  switch (nr) {
    case SYS_write: case SYS_pwrite64: case SYS_sendto: case SYS_sendmmsg:
    case SYS_munmap: case SYS_madvise: case SYS_close:
      return ROLE_PRODUCER;
    case SYS_read: case SYS_pread64: case SYS_recvfrom: case SYS_recvmmsg:
    case SYS_mmap: case SYS_open: case SYS_openat:
      return ROLE_CONSUMER;
    default:
      return ROLE_BOTH;
  }
}

__device__ __forceinline__ void note_error(const genesys_dev &g, int64_t code) {
  atomicCAS(reinterpret_cast<int *>(&g.status[GENESYS_ST_FIRST_ERROR]), 0, (int)code);
  if (code == -kETIMEDOUT) atomicAdd(reinterpret_cast<int *>(&g.status[GENESYS_ST_TIMEOUTS]), 1);
}

/* Checked builds: true if `ok`, else count the failure and return false. */
__device__ __forceinline__ bool dcheck(const genesys_dev &g, bool ok) {
#ifdef GENESYS_DEVICE_CHECKS
  if (!ok) {
    atomicAdd(reinterpret_cast<int *>(&g.status[GENESYS_ST_BAD_ARGS]), 1);
    atomicCAS(reinterpret_cast<int *>(&g.status[GENESYS_ST_FIRST_ERROR]), 0, -22);
  }
  return ok;
#else
  (void)g;
  return true || ok;
#endif
}

__device__ __forceinline__ void note_latency(const genesys_dev &g, uint64_t t0) {
  if (g.lat_cap == 0) return;
  uint32_t i = atomicAdd(g.lat_count, 1u);
  if (i < g.lat_cap) g.lat[i] = now_ns() - t0;
}

/* Per-call trace record (only when the context keeps a trace). */
__device__ __forceinline__ void trace_call(const genesys_dev &g, uint32_t s, uint32_t sq, uint32_t nr, uint32_t gran,
                                           uint64_t t_call, uint64_t t_pub, uint64_t t_done) {
  if (g.trace_cap == 0) return;
  const uint32_t i = atomicAdd(g.trace_count, 1u);
  if (i >= g.trace_cap) return;
  genesys_trace_dev *r = g.trace + i;
  r->slot = s;
  r->seq = sq;
  r->nr = nr;
  r->gran = gran;
  r->t_call = t_call;
  r->t_publish = t_pub;
  r->t_done = t_done;
}

__device__ __forceinline__ bool expired(const genesys_dev &g, uint64_t t0) {
  return now_ns() - t0 > g.deadline_ns;
}

__device__ __forceinline__ uint32_t ring_of(const genesys_dev &g, uint32_t slot) {
  return genesys_ring_of(slot, g.n_rings);
}

/* The doorbell ring of a request: by file region for pread/pwrite (file
 * neighbours from different blocks meet in one ring and merge), by slot
 * group for other calls. */
__device__ __forceinline__ uint32_t ring_for(const genesys_dev &g, uint32_t slot, uint32_t nr, uint64_t a0,
                                             uint64_t a3) {
  return (nr == SYS_pread64 || nr == SYS_pwrite64) ? genesys_ring_of_file(a0, a3, g.n_rings, nr == SYS_pread64)
                                                    : ring_of(g, slot);
}

/* Give up the claim lock of a slot this thread owns without using it. */
__device__ __forceinline__ void slot_release_lock(const genesys_dev &g, uint32_t s) {
  __threadfence();
  atomicExch(&g.owner[s], 0u);
}

/* ------------------------------------------------------ slot protocol
 * Wait (bounded) until the CPU has finished the previous request of slot `s`,
 * which the caller owns: sequence `sq` is the slot's last.  Returns 0, or
 * -ETIMEDOUT with the slot released. */
__device__ __forceinline__ int64_t slot_wait_previous(const genesys_dev &g, uint32_t s, uint32_t sq, uint64_t t0) {
  uint32_t ns = 128;
  while ((uint32_t)(ld_relaxed_sys(&g.done[s]) >> 32) != sq) {
    if (expired(g, t0)) {
      __threadfence();
      atomicExch(&g.owner[s], 0u);
      note_error(g, -kETIMEDOUT);
      return -kETIMEDOUT;
    }
    __nanosleep(ns);
    ns = ns < 2048 ? ns * 2 : ns;
  }
  fence_acq_rel_sys();
  st_relaxed_gpu(&g.known_done[s], sq);
  return 0;
}

/* One thread.  Try to claim a slot (device-side lock in HBM, never an RMW on
 * host memory): up to 32 slots from `hint` on.  A slot's previous request may
 * still be in flight (a non-blocking call releases its slot once published).
 * Without `skip_busy` the first free slot is taken and its previous request
 * waited for, bounded: a slot still held by an unfinished request delays the
 * new call (Sec. 5, Fig. 4).  With `skip_busy` (one caller claiming one slot)
 * a slot whose previous request is unfinished is passed over for a later one
 * of the 32 that is ready, one look at its completion word each; only when
 * none is does the caller wait, for the first it passed over (kept owned
 * meanwhile: the CPU finishes it whatever the GPU holds, so no hold-and-wait).
 * Returns 1 with *slot_out set, 0 if every slot tried is taken, or
 * -ETIMEDOUT. */
__device__ __forceinline__ int64_t slot_try_claim(const genesys_dev &g, uint32_t hint, uint32_t *slot_out,
                                                  uint64_t t0, bool skip_busy = false) {
  uint32_t s = hint % g.n_slots;
  uint32_t busy = 0xFFFFFFFFu, busy_sq = 0;  // the first owned slot with an unfinished request
  for (uint32_t probe = 0; probe < 32; ++probe) {
    if (!dcheck(g, s < g.n_slots)) {  // (checked builds; s stays below n_slots by construction)
      if (busy != 0xFFFFFFFFu) slot_release_lock(g, busy);
      return -kETIMEDOUT;
    }
    if (atomicCAS(&g.owner[s], 0u, 1u) == 0u) {
      __threadfence();
      const uint32_t sq = ld_relaxed_gpu(&g.seq[s]);
      bool ready = ld_relaxed_gpu(&g.known_done[s]) == sq;
      if (!ready && skip_busy && (uint32_t)(ld_relaxed_sys(&g.done[s]) >> 32) == sq) {
        fence_acq_rel_sys();
        st_relaxed_gpu(&g.known_done[s], sq);
        ready = true;
      }
      if (ready || !skip_busy) {
        if (busy != 0xFFFFFFFFu) slot_release_lock(g, busy);
        if (!ready) {
          const int64_t w = slot_wait_previous(g, s, sq, t0);
          if (w < 0) return w;
        }
        *slot_out = s;
        return 1;
      }
      if (busy == 0xFFFFFFFFu) {
        busy = s;
        busy_sq = sq;
      } else {
        slot_release_lock(g, s);
      }
    }
    s = (s + 1 == g.n_slots) ? 0 : s + 1;
  }
  if (busy != 0xFFFFFFFFu) {
    const int64_t w = slot_wait_previous(g, busy, busy_sq, t0);
    if (w < 0) return w;
    *slot_out = busy;
    return 1;
  }
  if (expired(g, t0)) {
    note_error(g, -kETIMEDOUT);
    return -kETIMEDOUT;
  }
  return 0;
}

/* One thread: claim a slot, waiting (bounded, with back-off) while all are
 * taken.  The caller must not hold anything other callers need meanwhile. */
__device__ __forceinline__ int64_t slot_claim(const genesys_dev &g, uint32_t hint, uint32_t *slot_out,
                                              uint64_t t0, bool skip_busy = false) {
  uint32_t ns = 32;
  for (uint32_t round = 0;; ++round) {
    const int64_t r = slot_try_claim(g, hint + round * 32u, slot_out, t0, skip_busy);
    if (r != 0) return r < 0 ? r : 0;
    __nanosleep(ns);
    ns = ns < 4096 ? ns * 2 : ns;
  }
}

/* Marshal the request into the slot with four 16-byte stores that cover its
 * whole 64-byte line (the arguments, then the request word beside a zeroed
 * result word), so the line crosses the host link as full writes rather than
 * a partial one; returns its sequence.  The result word is the CPU's only
 * while it serves the slot's previous request, which the claim has waited
 * for.  The caller fences (system scope) and rings the doorbell afterwards. */
__device__ __forceinline__ uint32_t slot_fill(const genesys_dev &g, uint32_t s, uint32_t nr, uint32_t flags,
                                              uint64_t a0, uint64_t a1, uint64_t a2, uint64_t a3, uint64_t a4,
                                              uint64_t a5) {
  const uint32_t sq = ld_relaxed_gpu(&g.seq[s]) + 1u;
  st_relaxed_gpu(&g.seq[s], sq);
  genesys_slot *sl = g.slots + s;
  st_v2(&sl->args[0], a0, a1);
  st_v2(&sl->args[2], a2, a3);
  st_v2(&sl->args[4], a4, a5);
  const uint64_t req = ((uint64_t)sq << 32) | ((uint64_t)(nr & 0xFFFFu) << 16) | (flags & 0xFFFFu);
  st_v2(&sl->req, req, 0);
  return sq;
}

/* The same marshalling for a whole warp whose 32 lanes claimed the 32
 * consecutive slots s0 .. s0 + 31 (s0 a multiple of 32): the warp's slots are
 * 2 KiB of contiguous lines, written with four lane-interleaved 16-byte
 * stores per lane, each store instruction covering 512 contiguous bytes
 * (eight whole slots), so the lines leave for the host as full writes instead
 * of 16-byte pieces at a 64-byte stride.  Store j, lane l writes quarter l % 4
 * of slot 8j + l / 4; the quarter's words come from the lane that owns the
 * slot, by shuffles.  Every lane of the warp calls it; returns the calling
 * lane's sequence. */
__device__ __forceinline__ uint32_t slot_fill_warp(const genesys_dev &g, uint32_t s, uint32_t nr, uint32_t flags,
                                                   uint64_t a0, uint64_t a1, uint64_t a2, uint64_t a3,
                                                   uint64_t a4, uint64_t a5) {
  const uint32_t sq = ld_relaxed_gpu(&g.seq[s]) + 1u;
  st_relaxed_gpu(&g.seq[s], sq);
  const uint64_t req = ((uint64_t)sq << 32) | ((uint64_t)(nr & 0xFFFFu) << 16) | (flags & 0xFFFFu);
  const uint32_t lane = lane_id(), q = lane & 3u;
  uint64_t *base = reinterpret_cast<uint64_t *>(g.slots + (s - lane));
#pragma unroll
  for (uint32_t j = 0; j < 4; ++j) {
    const uint32_t src = 8u * j + (lane >> 2);
    const uint64_t x0 = __shfl_sync(0xFFFFFFFFu, a0, src), y0 = __shfl_sync(0xFFFFFFFFu, a1, src);
    const uint64_t x1 = __shfl_sync(0xFFFFFFFFu, a2, src), y1 = __shfl_sync(0xFFFFFFFFu, a3, src);
    const uint64_t x2 = __shfl_sync(0xFFFFFFFFu, a4, src), y2 = __shfl_sync(0xFFFFFFFFu, a5, src);
    const uint64_t x3 = __shfl_sync(0xFFFFFFFFu, req, src);
    const uint64_t x = q == 0 ? x0 : q == 1 ? x1 : q == 2 ? x2 : x3;
    const uint64_t y = q == 0 ? y0 : q == 1 ? y1 : q == 2 ? y2 : 0ull;
    st_v2(base + 64u * j + 2u * lane, x, y);
  }
  return sq;
}

/* Doorbells.  The service thread takes a ring's entries in position order
 * and stops at the first one not yet written, so the time between taking a
 * position and writing its entry holds up every later entry of the ring.  The
 * system-scope fence that orders the slot stores before the entry (it waits
 * until the host link has acknowledged them, microseconds) therefore comes
 * first; the position is taken after it and the entry written at once.  A
 * fence followed by a relaxed system-scope store is a release pattern. */

/* Doorbell for one published slot on ring r (one thread); returns its ring
 * position. */
__device__ __forceinline__ uint32_t ring_one(const genesys_dev &g, uint32_t s, uint32_t r) {
  if (!dcheck(g, r < g.n_rings && s < g.n_slots)) return 0;
  fence_acq_rel_sys();
  const uint32_t pos = atomicAdd(&g.ring_tail[r * 32u], 1u);
  st_relaxed_sys(g.rings + (size_t)r * (g.ring_mask + 1u) + (pos & g.ring_mask), GENESYS_RING_ENTRY(pos, s));
  return pos;
}

/* Doorbell for the lanes of `mask` that each filled slot `s`.  After a warp
 * barrier (so that the fences below cover the slot stores of every lane, in
 * case lanes wrote parts of each other's slots) every lane fences (one
 * warp-wide instruction); the lanes going to the same ring (grouped with
 * __match_any_sync) then take consecutive positions with one atomic, and each
 * lane writes its own entry, so a warp's entries leave as one contiguous
 * store instead of one store per lane.  Returns the calling lane's ring
 * position (lane order within the group). */
__device__ __forceinline__ uint32_t ring_warp(const genesys_dev &g, uint32_t mask, uint32_t s, uint32_t r) {
  if (!dcheck(g, r < g.n_rings && s < g.n_slots)) r = 0;  // checked builds: counted, and kept in bounds
  __syncwarp(mask);
  fence_acq_rel_sys();
  const uint32_t peers = __match_any_sync(mask, r);
  const uint32_t lane = lane_id();
  const uint32_t leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&g.ring_tail[r * 32u], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  const uint32_t pos = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
  st_relaxed_sys(g.rings + (size_t)r * (g.ring_mask + 1u) + (pos & g.ring_mask), GENESYS_RING_ENTRY(pos, s));
  return pos;
}

/* Doorbell for a full warp whose lanes filled the 32 consecutive slots
 * s0 .. s0 + 31 (s0 a multiple of 32) with requests of ring r: one entry at
 * one ring position announces the 32 requests.  The warp barrier orders
 * every lane's slot stores before lane 0's system-scope fence, which orders
 * them before the entry (a release on behalf of the warp).  Every lane of
 * the warp calls; returns the ring position (the same for every lane). */
__device__ __forceinline__ uint32_t ring_run(const genesys_dev &g, uint32_t s0, uint32_t r) {
  if (!dcheck(g, r < g.n_rings && s0 + GENESYS_RING_MAX_RUN <= g.n_slots)) r = 0;  // counted, kept in bounds
  __syncwarp();
  uint32_t pos = 0;
  if (lane_id() == 0) {
    fence_acq_rel_sys();
    pos = atomicAdd(&g.ring_tail[r * 32u], 1u);
    st_relaxed_sys(g.rings + (size_t)r * (g.ring_mask + 1u) + (pos & g.ring_mask),
                   GENESYS_RING_ENTRY_RUN(pos, s0, GENESYS_RING_MAX_RUN));
  }
  return __shfl_sync(0xFFFFFFFFu, pos, 0);
}

/* Wait until the CPU finished request `sq` of slot `s`; returns its result.
 * Polls with relaxed loads and makes the acquire once, with a fence after the
 * load that saw the completion (an acquire pattern). */
__device__ __forceinline__ int64_t slot_wait(const genesys_dev &g, uint32_t s, uint32_t sq, uint64_t t0) {
  uint32_t ns = g.poll_min_ns;
  const uint32_t cap = g.poll_max_ns;
  uint64_t d;
  for (;;) {
    d = ld_relaxed_sys(&g.done[s]);
    if ((uint32_t)(d >> 32) == sq) break;
    if (expired(g, t0)) { note_error(g, -kETIMEDOUT); return -kETIMEDOUT; }
    __nanosleep(ns);
    ns = ns < cap ? ns + (ns >> 1) + 1 : cap;
  }
  fence_acq_rel_sys();
  st_relaxed_gpu(&g.known_done[s], sq);
  const uint32_t lo = (uint32_t)d;
  const int64_t ret = lo == GENESYS_RET_IN_SLOT ? (int64_t)ld_relaxed_sys(&g.slots[s].ret) : (int64_t)(int32_t)lo;
  if (ret < 0) atomicAdd(reinterpret_cast<int *>(&g.status[GENESYS_ST_FAILED_CALLS]), 1);
  return ret;
}

/* The same wait for a request published at position `pos` of ring `r`.  The
 * caller polls a count of the ring's finished entries instead of its own
 * completion word: one word for all the lanes of a warp, so a warp's polls
 * coalesce into one read, and GENESYS_RING_DONE_COPIES copies of it on
 * separate lines, one per group of warps, so that the grid's polls do not all
 * queue on one host-memory word.  It sleeps about as long as the entries still
 * ahead of it take at the rate it has seen the count advance (at most
 * kMaxNapNs at a time, so the deadline check stays prompt).  Once the count
 * has passed its position, one acquire fence and one read of its completion
 * word give the result. */
constexpr uint32_t kMaxNapNs = 100000;
/* Before a caller has seen its ring's count advance it does not know the
 * rate the entries ahead of it are served at: its first nap assumes this many
 * ns per entry (a lone request costs the service about that; a warp's entry
 * of 32 more), so a caller deep in a queue does not poll the host while the
 * entries ahead of it are still being served. */
constexpr uint32_t kPriorNsPerEntry = 64;

__device__ __forceinline__ int64_t slot_wait_ring(const genesys_dev &g, uint32_t s, uint32_t sq, uint32_t r,
                                                  uint32_t pos, uint64_t t0) {
  const uint32_t copy = (hw_lane_id() >> 5) % GENESYS_RING_DONE_COPIES;
  if (!dcheck(g, r < g.n_rings && s < g.n_slots)) return -kETIMEDOUT;
  const uint64_t *fin_word = g.ring_done + ((size_t)r * GENESYS_RING_DONE_COPIES + copy) * 8u;
  uint32_t ns = g.poll_min_ns;
  const uint32_t cap = g.poll_max_ns;
  uint32_t fin0 = 0;
  uint64_t when0 = 0;
  for (;;) {
    const uint32_t fin = (uint32_t)ld_relaxed_sys(fin_word);
    const int32_t ahead = (int32_t)(pos + 1u - fin);  // entries up to and including ours not finished
    if (ahead <= 0) break;
    const uint64_t now = now_ns();
    if (now - t0 > g.deadline_ns) { note_error(g, -kETIMEDOUT); return -kETIMEDOUT; }
    uint64_t nap = ns;
    if (when0 == 0) {
      when0 = now;
      fin0 = fin;
      const uint64_t prior = (uint64_t)ahead * kPriorNsPerEntry;
      nap = prior > nap ? prior : nap;
    } else if (fin != fin0) {
      const uint64_t est = (now - when0) / (uint32_t)(fin - fin0) * (uint64_t)ahead;  // ns per entry x ahead
      nap = est > nap ? est : nap;
    }
    __nanosleep(nap < kMaxNapNs ? (uint32_t)nap : kMaxNapNs);
    ns = ns < cap ? ns + (ns >> 1) + 1 : cap;
  }
  fence_acq_rel_sys();
  const uint64_t d = ld_relaxed_sys(&g.done[s]);
  if ((uint32_t)(d >> 32) != sq) return slot_wait(g, s, sq, t0);  // not expected once the count passed it
  st_relaxed_gpu(&g.known_done[s], sq);
  const uint32_t lo = (uint32_t)d;
  const int64_t ret = lo == GENESYS_RET_IN_SLOT ? (int64_t)ld_relaxed_sys(&g.slots[s].ret) : (int64_t)(int32_t)lo;
  if (ret < 0) atomicAdd(reinterpret_cast<int *>(&g.status[GENESYS_ST_FAILED_CALLS]), 1);
  return ret;
}

__device__ __forceinline__ void slot_release(const genesys_dev &g, uint32_t s) {
  __threadfence();
  atomicExch(&g.owner[s], 0u);
}

/* Whole request by one thread: claim, marshal, publish, optionally wait. */
__device__ __forceinline__ int64_t single_call(const genesys_dev &g, uint32_t nr, uint32_t flags, bool wait,
                                               uint64_t a0, uint64_t a1, uint64_t a2, uint64_t a3, uint64_t a4,
                                               uint64_t a5) {
  const uint64_t t0 = now_ns();
  uint32_t s;
  int64_t rc = slot_claim(g, hw_lane_id(), &s, t0, true);
  if (rc < 0) return rc;
  const uint32_t sq = slot_fill(g, s, nr, flags, a0, a1, a2, a3, a4, a5);
  const uint32_t r = ring_for(g, s, nr, a0, a3);
  const uint32_t pos = ring_one(g, s, r);  // fence first: the slot stores (and, through
                                           // the group's barrier, its earlier stores)
  const uint64_t t_pub = g.trace_cap ? now_ns() : 0;
  int64_t ret = 0;
  if (wait) {
    ret = slot_wait_ring(g, s, sq, r, pos, t0);
    trace_call(g, s, sq, nr, (flags >> GENESYS_REQ_GRAN_SHIFT) & 3u, t0, t_pub, ret == -kETIMEDOUT ? 0 : now_ns());
    if (ret == -kETIMEDOUT) {  /* the CPU may still finish it: keep the slot's
                                  sequence so the next claimer waits for it */
      slot_release(g, s);
      return ret;
    }
  } else {
    trace_call(g, s, sq, nr, (flags >> GENESYS_REQ_GRAN_SHIFT) & 3u, t0, t_pub, 0);
  }
  slot_release(g, s);
  note_latency(g, t0);
  return ret;
}

/* ------------------------------------------------ tickets (prefetching)
 * A non-blocking call whose result is collected later: the paper's relaxed,
 * non-blocking prefetching read (Sec. 4.1).  The slot stays owned by the
 * caller until genesys::wait, so the result cannot be overwritten. */
struct Ticket {
  uint32_t slot;
  uint32_t seq;
  uint64_t t0;
  uint32_t pos;   // ring position
  uint32_t ring;  // doorbell ring
};

__device__ __forceinline__ int64_t issue(const genesys_dev &g, Ticket *t, uint32_t nr, uint64_t a0 = 0,
                                         uint64_t a1 = 0, uint64_t a2 = 0, uint64_t a3 = 0, uint64_t a4 = 0,
                                         uint64_t a5 = 0) {
  t->t0 = now_ns();
  int64_t rc = slot_claim(g, hw_lane_id(), &t->slot, t->t0, true);
  if (rc < 0) { t->slot = 0xFFFFFFFFu; return rc; }
  t->seq = slot_fill(g, t->slot, nr, GENESYS_REQ_TICKET | GENESYS_REQ_RELAXED, a0, a1, a2, a3, a4, a5);
  t->ring = ring_for(g, t->slot, nr, a0, a3);
  t->pos = ring_one(g, t->slot, t->ring);
  return 0;
}

__device__ __forceinline__ int64_t wait(const genesys_dev &g, const Ticket &t) {
  if (t.slot == 0xFFFFFFFFu) return -kETIMEDOUT;
  const int64_t ret = slot_wait_ring(g, t.slot, t.seq, t.ring, t.pos, now_ns());
  trace_call(g, t.slot, t.seq, 0, GENESYS_GRAN_GROUP, t.t0, 0, ret == -kETIMEDOUT ? 0 : now_ns());
  slot_release(g, t.slot);
  if (ret != -kETIMEDOUT) note_latency(g, t.t0);
  return ret;
}

/* ------------------------------------------------------ group barriers */

/* Grid-wide barrier for cooperative launches (all CTAs co-resident).  Bounded:
 * returns false (and records -ETIMEDOUT) if the other CTAs do not arrive. */
__device__ __forceinline__ bool grid_sync(const genesys_dev &g) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
    const uint32_t nblocks = gridDim.x * gridDim.y * gridDim.z;
    uint32_t *count = g.grid_bar, *gen = g.grid_bar + 32;
    const uint32_t my_gen = ld_acquire_gpu(gen);
    __threadfence_system();
    const uint32_t arrived = atomicAdd(count, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      st_relaxed_gpu(count, 0u);
      st_release_gpu(gen, my_gen + 1u);
    } else {
      const uint64_t t0 = now_ns();
      uint32_t ns = 32;
      while (ld_acquire_gpu(gen) == my_gen) {
        if (expired(g, t0)) { note_error(g, -kETIMEDOUT); ok = 0; break; }
        __nanosleep(ns);
        ns = ns < 1024 ? ns * 2 : ns;
      }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <int G>
__device__ __forceinline__ void group_barrier(uint32_t warp_mask) {
  if (G == WARP) __syncwarp(warp_mask);
  if (G == GROUP) __syncthreads();
}

__device__ __forceinline__ bool is_block_leader() {
  return threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
}

/* A relaxed kernel-grain site reached more often than the grid has blocks
 * in one launch (see call_at): recorded as a bad argument, -EINVAL. */
__device__ __forceinline__ int64_t site_reused(const genesys_dev &g) {
  atomicAdd(reinterpret_cast<int *>(&g.status[GENESYS_ST_BAD_ARGS]), 1);
  atomicCAS(reinterpret_cast<int *>(&g.status[GENESYS_ST_FIRST_ERROR]), 0, -22);
  return -22;
}

/* Relaxed kernel-grain call over `nblocks` blocks at site record `ks` (every
 * thread of each block takes part).  producer: every block arrives and the
 * last one to arrive calls, so no block ever waits for another (no deadlock
 * whatever the number of blocks); only its caller receives the result.
 * consumer: the first block to arrive calls and the others wait for its
 * result (the caller is running by construction, so they cannot deadlock);
 * every thread receives it. */
__device__ __forceinline__ int64_t kernel_relaxed(const genesys_dev &g, genesys_ksite *ks, uint32_t nblocks,
                                                  bool producer, uint32_t nr, uint32_t flags, bool wait, uint64_t a0,
                                                  uint64_t a1, uint64_t a2, uint64_t a3, uint64_t a4, uint64_t a5) {
  __shared__ int64_t kret_s;
  if (producer) {
    __syncthreads();
    int64_t r = 0;
    if (is_block_leader()) {
      __threadfence_system();
      const uint32_t arrived = atomicAdd(&ks->arrive, 1u);
      if (arrived == nblocks - 1) {
        __threadfence_system();
        r = single_call(g, nr, flags, wait, a0, a1, a2, a3, a4, a5);
      } else if (arrived >= nblocks) {
        r = site_reused(g);
      }
    }
    return r;
  }
  if (is_block_leader()) {
    int64_t r;
    const uint32_t ticket = atomicAdd(&ks->ticket, 1u);
    if (ticket == 0u) {
      r = single_call(g, nr, flags, wait, a0, a1, a2, a3, a4, a5);
      ks->ret = r;
      __threadfence();
      st_release_gpu(&ks->flag, 1u);
    } else if (ticket >= nblocks) {
      r = site_reused(g);
    } else {
      const uint64_t t0 = now_ns();
      uint32_t ns = 64;
      r = 0;
      while (ld_acquire_gpu(&ks->flag) == 0u) {
        if (expired(g, t0)) { note_error(g, -kETIMEDOUT); r = -kETIMEDOUT; break; }
        __nanosleep(ns);
        ns = ns < 2048 ? ns * 2 : ns;
      }
      if (r == 0) r = *(volatile int64_t *)&ks->ret;
    }
    kret_s = r;
  }
  __syncthreads();
  const int64_t r = kret_s;
  __syncthreads();
  return r;
}

/* ------------------------------------------------------------- the call */

template <int G, int O, int B, int R = ROLE_AUTO>
__device__ __forceinline__ int64_t call_at(const genesys_dev &g, uint32_t site, uint32_t nr, uint64_t a0 = 0,
                                           uint64_t a1 = 0, uint64_t a2 = 0, uint64_t a3 = 0, uint64_t a4 = 0,
                                           uint64_t a5 = 0) {
  static_assert(G != ITEM || O == STRONG, "work-item grain is implicitly strong (Sec. 4.1)");
  const int role = R == ROLE_AUTO ? role_of(nr) : R;
  const bool pre = O == STRONG || (role & ROLE_PRODUCER);
  const bool post = O == STRONG || (role & ROLE_CONSUMER);
  const uint32_t flags = (B == BLOCKING ? GENESYS_REQ_BLOCKING : 0u) | ((uint32_t)G << GENESYS_REQ_GRAN_SHIFT) |
                         (O == RELAXED ? GENESYS_REQ_RELAXED : 0u);

  if (G == ITEM) {
    /* every calling lane is a caller; lanes of a warp that call together
     * share one doorbell atomic per ring.  Lanes claim in rounds: the lanes
     * that got a slot in a round publish together, complete and release it
     * before the next round, so no lane holds a slot while it waits for a
     * sibling that has none (with fewer slots than callers, holding and
     * waiting would deadlock). */
    const uint32_t active = __activemask();
    const uint64_t t0 = now_ns();
    const uint32_t hint = hw_lane_id();
    bool pending = true;
    int64_t rc = 0;
    uint32_t ns = 32;
    for (uint32_t round = 0; __ballot_sync(active, pending); ++round) {
      uint32_t s = 0;
      bool ok = false;
      if (pending) {
        const int64_t t = slot_try_claim(g, hint + round * 32u, &s, t0);
        if (t < 0) { rc = t; pending = false; }
        ok = t > 0;
      }
      const uint32_t okmask = __ballot_sync(active, ok);
      // a full warp on 32 consecutive slots (the usual case: each lane got the
      // slot of its hardware id) writes them as whole lines
      const uint32_t s0 = __shfl_sync(active, s, __ffs(active) - 1);
      const uint32_t r = ring_for(g, s, nr, a0, a3);
      const uint32_t r0 = __shfl_sync(active, r, __ffs(active) - 1);
      const bool lines = okmask == 0xFFFFFFFFu && (s0 & 31u) == 0 &&
                         __all_sync(0xFFFFFFFFu, s == s0 + lane_id() && r == r0) && dcheck(g, s0 + 32u <= g.n_slots);
      if (ok) {
        const uint32_t sq = lines ? slot_fill_warp(g, s, nr, flags, a0, a1, a2, a3, a4, a5)
                                  : slot_fill(g, s, nr, flags, a0, a1, a2, a3, a4, a5);
        const uint32_t pos = lines ? ring_run(g, s0, r) : ring_warp(g, okmask, s, r);
        const uint64_t t_pub = g.trace_cap ? now_ns() : 0;
        rc = B == BLOCKING ? slot_wait_ring(g, s, sq, r, pos, t0) : 0;
        trace_call(g, s, sq, nr, GENESYS_GRAN_ITEM, t0, t_pub,
                   (B == BLOCKING && rc != -kETIMEDOUT) ? now_ns() : 0);
        slot_release(g, s);
        if (rc != -kETIMEDOUT) note_latency(g, t0);
        pending = false;
      } else if (pending) {
        __nanosleep(ns);
        ns = ns < 4096 ? ns * 2 : ns;
      }
    }
    return rc;
  }

  if (G == WARP || G == GROUP) {
    const uint32_t active = G == WARP ? __activemask() : 0xFFFFFFFFu;
    const bool leader = G == WARP ? lane_id() == (uint32_t)(__ffs(active) - 1) : is_block_leader();
    if (pre) group_barrier<G>(active);
    int64_t ret = 0;
    if (leader) ret = single_call(g, nr, flags, B == BLOCKING, a0, a1, a2, a3, a4, a5);
    if (!post) return ret;            /* relaxed producer: only the caller waited */
    if (G == WARP) {
      __syncwarp(active);
      return __shfl_sync(active, ret, __ffs(active) - 1);
    }
    __shared__ int64_t ret_s;
    if (leader) ret_s = ret;
    __syncthreads();
    ret = ret_s;
    __syncthreads();                  /* ret_s may be rewritten by the next call */
    return ret;
  }

  /* KERNEL grain: one caller for the whole grid.  Strongly ordered calls
   * may be made at one site any number of times (grid barriers separate
   * them).  A relaxed call site serves one call per block per launch: its
   * arrival counters are reset before each launch (genesys_launch), and
   * nothing tells a block's second call at a site from another block's
   * first.  A site reached more often than the grid has blocks has been
   * reused: the extra arrivals make no call, return -EINVAL and record it
   * (status word GENESYS_ST_BAD_ARGS), so the launch reports the misuse;
   * give each relaxed kernel-grain call of a kernel its own site (call_at).
   * A relaxed call whose role is both producer and consumer (a call that is
   * neither, e.g. getpid, unless R names a role) is strongly ordered, so at
   * kernel grain it waits at grid barriers and needs every block resident. */
  genesys_ksite *ks = g.ksite + (site % GENESYS_KSITES);
  const uint32_t nblocks = gridDim.x * gridDim.y * gridDim.z;
  if (pre && post) {
    /* strong: grid barriers before and after (cooperative launch only) */
    if (!grid_sync(g)) return -kETIMEDOUT;
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && is_block_leader()) {
      const int64_t r = single_call(g, nr, flags, B == BLOCKING, a0, a1, a2, a3, a4, a5);
      ks->ret = r;
    }
    if (!grid_sync(g)) return -kETIMEDOUT;
    return *(volatile int64_t *)&ks->ret;
  }
  return kernel_relaxed(g, ks, nblocks, pre, nr, flags, B == BLOCKING, a0, a1, a2, a3, a4, a5);
}

/* A relaxed kernel-grain call over a group of `nblocks` thread blocks that
 * need not be the launch's grid - the virtual grid of a request that a
 * persistent kernel runs on whichever of its blocks pick it up - with its own
 * call-site record `ks` (zeroed before the group's first block arrives, and
 * by the group before it is used for another).  Every block of the group
 * makes the call once, with all its threads; the rules are call_at's relaxed
 * kernel grain: a producer (R = ROLE_PRODUCER) is issued by the last block to
 * arrive and only its caller waits, a consumer (ROLE_CONSUMER) by the first
 * block to arrive and every block receives the result.  Neither waits for a
 * block that has not started, so the group may be larger than what is
 * resident.  Arrivals beyond nblocks are a reused site: -EINVAL. */
template <int B, int R>
__device__ __forceinline__ int64_t call_vgrid(const genesys_dev &g, genesys_ksite *ks, uint32_t nblocks, uint32_t nr,
                                              uint64_t a0 = 0, uint64_t a1 = 0, uint64_t a2 = 0, uint64_t a3 = 0,
                                              uint64_t a4 = 0, uint64_t a5 = 0) {
  static_assert(R == ROLE_PRODUCER || R == ROLE_CONSUMER, "call_vgrid: a producer or a consumer call");
  const uint32_t flags = (B == BLOCKING ? GENESYS_REQ_BLOCKING : 0u) | (GENESYS_GRAN_KERNEL << GENESYS_REQ_GRAN_SHIFT) |
                         GENESYS_REQ_RELAXED;
  return kernel_relaxed(g, ks, nblocks, R == ROLE_PRODUCER, nr, flags, B == BLOCKING, a0, a1, a2, a3, a4, a5);
}

/* Warp grain with request coalescing.  Every active lane brings its own
 * positional transfer (pread/pwrite-like: fd, buf, len, off).  Lanes are
 * grouped by fd with __match_any_sync; within a group, lanes whose buffer and
 * file range continue the previous lane's form one run, and the lowest lane of
 * each run issues a single call covering the run.  Each lane gets the part of
 * the run's result that covers its own range - what its own call would have
 * returned.  Ordering and blocking as for call<WARP, O, B>. */
template <int O, int B>
__device__ __forceinline__ int64_t call_warp_coalesced(const genesys_dev &g, uint32_t nr, int fd, uint64_t buf,
                                                       uint64_t len, uint64_t off) {
  const int role = role_of(nr);
  const bool pre = O == STRONG || (role & ROLE_PRODUCER);
  const bool post = O == STRONG || (role & ROLE_CONSUMER);
  const uint32_t flags = (B == BLOCKING ? GENESYS_REQ_BLOCKING : 0u) | (GENESYS_GRAN_WARP << GENESYS_REQ_GRAN_SHIFT) |
                         (O == RELAXED ? GENESYS_REQ_RELAXED : 0u);
  const uint32_t active = __activemask();
  const uint32_t lane = lane_id();
  if (pre) __syncwarp(active);
  const uint32_t peers = __match_any_sync(active, fd);
  const uint32_t below = peers & ((1u << lane) - 1u);
  const int prev = below ? 31 - __clz(below) : (int)lane;
  const uint64_t pbuf_end = __shfl_sync(peers, buf + len, prev);
  const uint64_t poff_end = __shfl_sync(peers, off + len, prev);
  const bool starts_run = below == 0 || pbuf_end != buf || poff_end != off;
  const uint32_t starts = __ballot_sync(peers, starts_run);
  /* my run's leader: the highest run start at or below me */
  const uint32_t at_or_below = starts & ((2u << lane) - 1u);
  const int leader = 31 - __clz(at_or_below);
  /* my run's last lane: the highest peer below the next run start above me */
  const uint32_t above = peers & ~((2u << lane) - 1u);
  const uint32_t next_start = starts & above;
  const uint32_t limit = next_start ? ((1u << (__ffs(next_start) - 1)) - 1u) : 0xFFFFFFFFu;
  const int last = 31 - __clz(peers & limit);
  const uint64_t run_end = __shfl_sync(peers, off + len, last);
  const uint64_t run_off = __shfl_sync(peers, off, leader);
  int64_t ret = 0;
  if ((int)lane == leader) ret = single_call(g, nr, flags, B == BLOCKING, (uint64_t)fd, buf, run_end - off, off, 0, 0);
  if (!post && B == NONBLOCKING) return 0;
  if (post) __syncwarp(active);
  if (!post) {
    /* relaxed producer, blocking: only the run leaders waited */
    return (int)lane == leader ? (int64_t)(ret < 0 ? ret : (ret < (int64_t)len ? ret : (int64_t)len)) : 0;
  }
  const int64_t run_ret = __shfl_sync(peers, ret, leader);
  if (run_ret < 0) return run_ret;
  const uint64_t before = off - run_off;
  const uint64_t got = (uint64_t)run_ret > before ? (uint64_t)run_ret - before : 0;
  return (int64_t)(got < len ? got : len);
}

template <int G, int O, int B, int R = ROLE_AUTO>
__device__ __forceinline__ int64_t call(const genesys_dev &g, uint32_t nr, uint64_t a0 = 0, uint64_t a1 = 0,
                                        uint64_t a2 = 0, uint64_t a3 = 0, uint64_t a4 = 0, uint64_t a5 = 0) {
  return call_at<G, O, B, R>(g, 0u, nr, a0, a1, a2, a3, a4, a5);
}

/* pread of `len` bytes at `off` into `buf` that goes on after a short read,
 * as a reader's loop does: a pread may return fewer bytes than asked before
 * the end of the file (Linux allows it; the file system, a signal or the
 * host's service can cause it), so the group calls again for the rest until
 * it has `len` bytes or a read returns 0 (end of file).  Blocking; the group
 * and ordering of call<G, O, BLOCKING>, whose result every thread of the
 * group receives, so the loop is uniform across the group.  Returns the bytes
 * read, or the first -errno. */
template <int G, int O, int R = ROLE_AUTO>
__device__ __forceinline__ int64_t pread_full(const genesys_dev &g, uint64_t fd, uint8_t *buf, uint64_t len,
                                              uint64_t off) {
  static_assert(G == WARP || G == GROUP, "pread_full: warp or work-group grain (the result is broadcast)");
  uint64_t got = 0;
  while (got < len) {
    const int64_t r = call<G, O, BLOCKING, R>(g, SYS_pread64, fd, (uint64_t)(buf + got), len - got, off + got);
    if (r < 0) return r;
    if (r == 0) break;
    got += (uint64_t)r < len - got ? (uint64_t)r : len - got;
  }
  return (int64_t)got;
}

}  // namespace genesys

#endif /* GENESYS_DEVICE_CUH */
