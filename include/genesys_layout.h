/*
 * genesys_layout.h - memory layout shared by the device invocation code
 * (genesys_device.cuh) and the host service runtime.
 *
 * The syscall area (Sec. 5, "GPU to CPU communication", Fig. 3) is an array of
 * 64-byte slots in pinned, host-mapped system memory that both the GPU and
 * the CPU can reach.  A slot holds the system call number, the request state
 * and up to six arguments; the argument field is reused for the return value.
 *
 * Differences from the paper's layout, forced by a discrete GPU behind PCIe
 * without host-native atomics (device RMW on host memory is not atomic with
 * respect to the CPU):
 *   - every word has one writer at a time.  The request word and arguments
 *     are written only by the GPU, the completion word only by the CPU; the
 *     slot's result word is the CPU's while it serves a request and the GPU's
 *     (it zeroes it with the rest of the line) once the request has completed
 *     and the slot is claimed again.  No read-modify-write on host memory is
 *     ever needed;
 *   - the slot state of Fig. 4 is carried by sequence numbers instead of an
 *     atomically updated state field: a slot is FREE when its completion
 *     sequence equals its request sequence, READY/PROCESSING while the request
 *     sequence is ahead, FINISHED once the CPU writes the completion sequence;
 *   - completion words live in their own dense array, so that one warp polling
 *     32 neighbouring slots reads 256 contiguous bytes instead of 32 lines;
 *   - the CPU learns of new requests from doorbell rings (one per service
 *     thread, see genesys_ring_of) instead of an interrupt carrying the
 *     wavefront's hardware ID
 *     (Sec. 3 notes that interrupt versus polling is orthogonal to the design).
 *
 * All multi-byte fields are little-endian (x86-64 host, NVIDIA GPU).
 */
#ifndef GENESYS_LAYOUT_H
#define GENESYS_LAYOUT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GENESYS_SLOT_BYTES 64u

/* One request slot (Sec. 5, Fig. 3), one 64-byte line.  The GPU writes the
 * whole line when it fills the slot (the result word as 0), so the line
 * crosses the host link as full writes. */
typedef struct genesys_slot {
  uint64_t args[6];   /* Linux passes at most six arguments; 16-byte aligned
                         so the GPU writes them with three vector stores    */
  /* bits 63..32: request sequence number (1, 2, ... per slot)
   * bits 31..16: system call number (host SYS_* number, or a GENESYS_NR_* op)
   * bits 15..0 : GENESYS_REQ_* flags                                        */
  uint64_t req;
  uint64_t ret;       /* full 64-bit return value, written by the CPU when it
                         does not fit in the completion word (see below)     */
} genesys_slot;
#ifdef __cplusplus
static_assert(sizeof(genesys_slot) == GENESYS_SLOT_BYTES, "a slot is one 64-byte line");
#endif

/* Completion word, written by the CPU only:
 *   bits 63..32: sequence number of the last finished request of the slot
 *   bits 31..0 : its return value as int32, or GENESYS_RET_IN_SLOT when the
 *                value does not fit (then the full value is in slot.ret,
 *                written before the completion word).                      */
#define GENESYS_RET_IN_SLOT 0x80000000u

/* Request flags (low 16 bits of slot.req). */
#define GENESYS_REQ_BLOCKING   0x0001u  /* a GPU thread waits for the result          */
#define GENESYS_REQ_GRAN_SHIFT 1        /* 2 bits: GENESYS_GRAN_*                     */
#define GENESYS_REQ_RELAXED    0x0008u  /* relaxed ordering (Sec. 4.1)                */
#define GENESYS_REQ_TICKET     0x0010u  /* non-blocking call whose result is collected
                                           later with genesys_wait (slot stays owned) */

/* Invocation granularities (Sec. 4.1), plus the warp grain of this design. */
#define GENESYS_GRAN_ITEM   0u
#define GENESYS_GRAN_WARP   1u
#define GENESYS_GRAN_GROUP  2u
#define GENESYS_GRAN_KERNEL 3u

/* Operations that are not Linux system calls (numbers above any SYS_*). */
#define GENESYS_NR_NOP            0x7F00u  /* returns args[0]; measures the protocol alone   */
#define GENESYS_NR_CHECK_VISIBLE  0x7F01u  /* args: ptr, count, seed -> number of u64 words
                                              in [ptr, ptr+count) that differ from
                                              splitmix64_at(seed, i); the strong-ordering
                                              visibility probe                            */

#ifdef __CUDACC__
#define GENESYS_HD __host__ __device__
#else
#define GENESYS_HD
#endif

/* Doorbell ring of a slot, for calls other than positional file calls.
 * Slots are taken in groups of 256 (eight warps of one SM: the slot a lane
 * tries first is its hardware id), so the requests of one thread block meet
 * in one ring; the group number is hashed so that the callers of different
 * SMs and warp slots spread over all rings. */
#define GENESYS_RING_GROUP_SHIFT 8u
static inline GENESYS_HD uint32_t genesys_ring_of(uint32_t slot, uint32_t n_rings) {
  uint32_t g = slot >> GENESYS_RING_GROUP_SHIFT;
  g ^= g >> 7;
  g *= 0x9E3779B1u;
  g ^= g >> 15;
  return g % n_rings;
}

/* Doorbell ring of a positional file call (pread/pwrite): calls on the same
 * region of one file meet in one ring, whichever GPU threads make them, and
 * the regions of a file spread over all rings.  Any slot may therefore reach
 * any ring (each ring holds an entry for every slot).  Writes to one file
 * serialise on its inode lock whichever thread makes them, so for writes the
 * region is 256 KiB: the ring's service thread finds file neighbours in its
 * batches and merges them into fewer Linux calls.  Reads of one file take no
 * such lock and copy in parallel on several threads, so for reads the region
 * is 16 KiB: neighbouring small reads (4 KiB chunks of many blocks) spread
 * over the service threads instead of queueing on one. */
#define GENESYS_RING_REGION_SHIFT_WRITE 18u
#define GENESYS_RING_REGION_SHIFT_READ 14u
static inline GENESYS_HD uint32_t genesys_ring_of_file(uint64_t fd, uint64_t off, uint32_t n_rings, int is_read) {
  const uint32_t shift = is_read ? GENESYS_RING_REGION_SHIFT_READ : GENESYS_RING_REGION_SHIFT_WRITE;
  uint64_t z = (off >> shift) * 0x9E3779B97F4A7C15ull ^ (fd + 1) * 0xC2B2AE3D27D4EB4Full;
  z ^= z >> 29;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 32;
  return (uint32_t)(z % n_rings);
}

/* Doorbell ring entry: bits 63..32 = ring position + 1; bits 31..24 = the
 * number of requests it announces, minus 1; bits 23..0 = the slot of the
 * first.  An entry announces the requests of `count` consecutive slots: one
 * (a single caller), or a whole warp's 32 when its lanes filled 32 consecutive
 * slots (one ring position for the warp).  Slot numbers are below 2^24. */
#define GENESYS_RING_SLOT_BITS 24u
#define GENESYS_RING_MAX_RUN 32u
#define GENESYS_RING_ENTRY_RUN(pos, slot, count)                                             \
  ((((uint64_t)(uint32_t)((pos) + 1u)) << 32) | ((uint64_t)(((count) - 1u) & 0xFFu) << 24) | \
   (uint64_t)((slot) & 0xFFFFFFu))
#define GENESYS_RING_ENTRY(pos, slot) GENESYS_RING_ENTRY_RUN(pos, slot, 1u)

/* Copies of each ring's finished-entries count (callers poll the copy of
 * their warp, so that no single host-memory word takes every poll). */
#define GENESYS_RING_DONE_COPIES 16u

/* Kernel-grain call sites per launch (GENESYS_GRAN_KERNEL). */
#define GENESYS_KSITES 64u

/* Device status words (int32 each), in device memory. */
#define GENESYS_ST_FIRST_ERROR   0   /* first negative code seen by any device wait    */
#define GENESYS_ST_TIMEOUTS      1   /* device waits that gave up (deadline)           */
#define GENESYS_ST_FAILED_CALLS  2   /* calls that returned a negative value           */
#define GENESYS_ST_BAD_ARGS      3   /* device-side argument checks that failed        */
#define GENESYS_ST_WORDS         8

/* Per-kernel-grain-site state in device memory, reset before each launch. */
typedef struct genesys_ksite {
  uint32_t arrive;    /* CTAs that reached the call                              */
  uint32_t ticket;    /* first-arriver election (consumer role)                  */
  uint32_t flag;      /* set to 1 when the result is available                   */
  uint32_t pad;
  int64_t ret;
  uint64_t pad2;
} genesys_ksite;

/* Per-call trace records (genesys_trace_read): the device record is written
 * by the calling GPU thread (device clock, ns), the host record by the service
 * thread (CLOCK_MONOTONIC, ns); they are joined by (slot, seq). */
typedef struct genesys_trace_dev {
  uint32_t slot, seq, nr, gran;  /* gran: GENESYS_GRAN_*                         */
  uint64_t t_call;               /* the call began (before the slot claim)        */
  uint64_t t_publish;            /* its doorbell entry was written (0: unknown)   */
  uint64_t t_done;               /* the result was seen (0: non-blocking)         */
} genesys_trace_dev;
typedef struct genesys_trace_host {
  uint32_t slot, seq;
  uint64_t t_pickup;             /* the batch holding it was taken from the ring  */
  uint64_t t_done;               /* its completion word was written               */
} genesys_trace_host;

/* The device view of a context: a plain struct passed to kernels by value. */
typedef struct genesys_dev {
  genesys_slot *slots;        /* host-mapped, n_slots entries                       */
  uint64_t *done;             /* host-mapped, n_slots completion words              */
  uint64_t *rings;            /* host-mapped, n_rings * ring_cap doorbell entries   */
  uint64_t *ring_done;        /* host-mapped: leading entries of ring r the CPU has
                                 finished, GENESYS_RING_DONE_COPIES copies on separate
                                 64-byte lines (word 8 * (r * COPIES + c)), stored with
                                 release after the completion words they cover      */
  uint32_t *owner;            /* device memory: slot claim locks                    */
  uint32_t *seq;              /* device memory: last published sequence per slot    */
  uint32_t *known_done;       /* device memory: last sequence seen finished         */
  uint32_t *ring_tail;        /* device memory: producer positions, stride 32 words */
  genesys_ksite *ksite;       /* device memory: GENESYS_KSITES entries              */
  uint32_t *grid_bar;         /* device memory: {count, generation}                 */
  int32_t *status;            /* device memory: GENESYS_ST_WORDS                    */
  uint64_t *lat;              /* device memory: per-call latency samples (ns)       */
  uint32_t *lat_count;        /* device memory: samples written (may exceed cap)    */
  genesys_trace_dev *trace;   /* device memory: per-call trace records, or NULL    */
  uint32_t *trace_count;      /* device memory: trace records written (may exceed cap) */
  uint32_t trace_cap;         /* 0: tracing off                                     */
  uint32_t lat_cap;
  uint32_t n_slots;
  uint32_t n_rings;
  uint32_t ring_mask;         /* ring_cap - 1, ring_cap a power of two              */
  uint64_t deadline_ns;       /* every device wait gives up after this long         */
  uint32_t n_sms;
  uint32_t poll_min_ns;       /* completion polls: first back-off ...                */
  uint32_t poll_max_ns;       /* ... growing 1.5x per poll up to this                */
  uint32_t reserved;
} genesys_dev;

#ifdef __cplusplus
}
#endif

#endif /* GENESYS_LAYOUT_H */
