/*
 * genesys.h - C ABI of the B300 GPU system-call runtime.
 *
 * What it implements: the GENESYS mechanism of Vesely et al., "GPU System
 * Calls" (arXiv 1705.06965): GPU code invokes Linux system calls with
 * function-like semantics at a chosen invocation granularity, ordering and
 * blocking mode (Sec. 4.1); requests travel through a syscall area of 64-byte
 * slots in system memory visible to both processors (Sec. 5, Fig. 3, Fig. 4);
 * CPU-side workers carry out the calls, optionally coalescing several requests
 * into one unit of work (Sec. 4.2, Sec. 5), and write the results back; a
 * host function waits until every GPU call has completed (Sec. 8.3).
 *
 * Conventions for every function below:
 *   - return 0 (or a documented non-negative value) on success and a negative
 *     GENESYS_E* code on failure; nothing aborts the process;
 *     genesys_last_error() describes the last failure of the calling thread;
 *   - pointers are plain host or device addresses; "device pointer" means
 *     memory the GPU can address (cudaMalloc'd memory, or the host-mapped
 *     staging arena, whose addresses are valid on both sides);
 *   - a `stream` argument is a cudaStream_t passed as void* (NULL = the
 *     legacy default stream);
 *   - the context owns the syscall area, the doorbell rings, the staging arena
 *     and the service threads; the caller owns file descriptors, sockets and
 *     the device buffers it passes in.
 */
#ifndef GENESYS_H
#define GENESYS_H

#include <stddef.h>
#include <stdint.h>

#include "genesys_layout.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define GENESYS_OK          0
#define GENESYS_EINVAL    (-22)   /* bad argument or illegal flag combination        */
#define GENESYS_ENOMEM    (-12)   /* allocation failed, or staging arena exhausted  */
#define GENESYS_ETIMEDOUT (-110)  /* a bounded wait gave up                          */
#define GENESYS_ENODEV    (-19)   /* no usable CUDA device                           */
#define GENESYS_EDEVICE   (-1001) /* the GPU reported failed or timed-out calls     */
#define GENESYS_ECUDA     (-1000) /* a CUDA runtime call failed                      */
/* Every entry point returns one of these codes (0 on success) and records a
 * message for genesys_last_error.  No C++ exception leaves the library: a host
 * allocation that fails, or a thread that cannot start, becomes
 * GENESYS_ENOMEM, and whatever the call had set up is given back. */

/* ------------------------------------------------------------ configuration */
#define GENESYS_INIT_HOST_ONLY   0x1u /* no GPU: host memory only; requests come from
                                         genesys_emulate_call (protocol tests)        */
#define GENESYS_INIT_NO_THREADS  0x2u /* spawn no service threads: the caller drives
                                         them with genesys_service                    */
#define GENESYS_INIT_ANY_SYSCALL 0x4u /* pass any system call number to the kernel
                                         (default: the supported set only)            */

typedef struct genesys_config {
  uint32_t n_slots;            /* syscall-area slots; 0 = one per resident GPU thread
                                  (SMs x 2048), the paper's one-slot-per-active-
                                  work-item sizing (Sec. 5); at most 2^24              */
  uint32_t n_service_threads;  /* CPU service threads, one doorbell ring each (>= 1)   */
  const int32_t *service_cpus; /* CPU to pin each service thread to, or NULL           */
  uint64_t staging_bytes;      /* pinned host-mapped staging arena                      */
  uint64_t coalesce_window_ns; /* Sec. 4.2: how long a service thread waits after the
                                  first request of a batch for more to arrive (0 = take
                                  what is ready)                                       */
  uint32_t coalesce_max;       /* Sec. 4.2: requests processed as one batch (>= 1); the
                                  requests of one doorbell entry (up to a warp's 32)
                                  are never split, so a batch may hold up to 31 more  */
  uint32_t merge;              /* 1: a batch's pread/pwrite requests that are
                                  contiguous in the file are merged into one Linux call
                                  (pread/pwrite or preadv/pwritev)                    */
  uint64_t device_deadline_ns; /* every device-side wait gives up after this long      */
  uint32_t lat_samples;        /* capacity of the per-call latency sample buffer       */
  uint32_t flags;              /* GENESYS_INIT_*                                       */
  uint64_t idle_spin_ns;       /* a service thread busy-polls this long after its last
                                  request before it starts napping                     */
  uint32_t poll_min_ns;        /* GPU completion polls: first back-off (ns) ...         */
  uint32_t poll_max_ns;        /* ... growing 1.5x per poll up to this; more polls cost
                                  host-link read requests, fewer add latency           */
  uint32_t trace_capacity;     /* per-call trace records kept on each side (device and
                                  host); 0 = tracing off (genesys_trace_read)          */
  uint32_t reserved0;
} genesys_config;

typedef struct genesys_stats {  /* genesys_stats_t */
  uint64_t requests;           /* GPU requests retired by the service threads          */
  uint64_t os_calls;           /* Linux calls made for them (fewer when merged)        */
  uint64_t failed;             /* requests whose result was negative                   */
  uint64_t nonblocking_failed; /* of those, requests nobody waited for (Sec. 4.1)      */
  uint64_t bytes;              /* bytes moved by read/write-like calls                 */
  uint64_t batches;            /* batches processed (Sec. 4.2 coalescing units)        */
  uint64_t busy_ns;            /* service-thread time spent processing batches         */
  uint64_t by_op[8];           /* requests per op: pread, pwrite, sendto, recvfrom,
                                  mmap, munmap, internal ops, other                    */
  uint64_t op_ns[8];           /* service time per op (unmerged requests)              */
  uint64_t op_max_ns[8];       /* longest single request per op                        */
  uint64_t mmap_new;           /* GPU mmaps served by mmap(2) + registration           */
  uint64_t mmap_reused;        /* GPU mmaps served by a released region                */
  uint64_t service_cpu_ns;     /* CPU time of the service threads (their per-thread CPU
                                  clocks)                                              */
  uint64_t protocol_errors;    /* checked builds (GENESYS_DEVICE_CHECKS): requests whose
                                  sequence number was not the slot's previous one + 1,
                                  or whose ring entry named a slot out of range; always
                                  0 in other builds                                    */
  uint64_t pickup_ns;          /* service-thread time taking batches: reading the slots
                                  of the ready ring entries (and any coalescing window) */
  uint64_t order_ns;           /* ... ordering a batch so that file neighbours merge   */
  uint64_t complete_ns;        /* ... writing results, completion words and the rings'
                                  finished counts (the Linux calls are op_ns)           */
  uint64_t empty_polls;        /* ring polls that found no new request at the head     */
  uint64_t hole_polls;         /* of those, polls where a later entry was already
                                  written: a position taken whose entry had not yet
                                  arrived held the ring up                            */
} genesys_stats_t;

typedef struct genesys_ctx genesys_ctx;

/* Fill *cfg with defaults (Sec. 5 sizes the syscall area by the hardware
 * threads that can be active at once): slots = SMs x 2048 (or 65536 without a
 * GPU), 4 service threads, 256 MiB staging, no coalescing window, coalesce_max
 * 64, merge on, 2 s device deadline, 1 M latency samples, polls 256 ns .. 2
 * us. */
int genesys_config_default(genesys_config *cfg);

/* Create a context on CUDA device `device`: allocates the syscall area, the
 * completion words and the doorbell rings in pinned host-mapped memory, the
 * device-side slot state in device memory, the staging arena, and starts the
 * service threads.  *out receives the context.  Sec. 5. */
int genesys_init(const genesys_config *cfg, int device, genesys_ctx **out);

/* Tear the context down (no counterpart in the paper).  Wait for the device's work in flight (kernels that still
 * make calls keep being served; every device-side wait is bounded), stop the
 * service threads after draining for up to 1 s, and free everything the
 * context owns.  Returns GENESYS_EINVAL and leaves the context untouched while
 * a key-value or echo server started on it still runs (stop it first); on any
 * other return the context is gone.  Idempotent for a NULL context. */
int genesys_shutdown(genesys_ctx *ctx);

/* The device view of the context: the syscall area and its rings (Sec. 5,
 * Fig. 3) as a plain struct, pass it to kernels by value;
 * genesys_device.cuh reads it; genesys_syscall.cuh binds it for the
 * handle-less genesys_syscall). */
int genesys_device_view(genesys_ctx *ctx, genesys_dev *out);

/* ------------------------------------------------------------ launching */
#define GENESYS_LAUNCH_GRAN_MASK   0x3u   /* GENESYS_GRAN_* the kernel uses            */
#define GENESYS_LAUNCH_RELAXED     0x10u  /* the kernel's calls use relaxed ordering   */
#define GENESYS_LAUNCH_NONBLOCKING 0x20u  /* the kernel's calls are non-blocking       */
#define GENESYS_LAUNCH_COOPERATIVE 0x100u /* force a cooperative launch                */
#define GENESYS_LAUNCH_SYNC        0x200u /* wait for the kernel, then drain its calls */
#define GENESYS_LAUNCH_GRAPH       0x400u /* launch through a CUDA graph built once per
                                             launch shape and relaunched               */

/* Launch a kernel that makes GPU system calls.  `kernel` is the kernel's host
 * stub (a __global__ function pointer from a library linked against the shared
 * CUDA runtime); grid/block are 3 sizes each; args as for cudaLaunchKernel.
 * `flags` declares the granularity/ordering/blocking the kernel uses so that
 * the legality rules of Sec. 4.1 are checked before launch:
 *   - work-item grain with relaxed ordering -> GENESYS_EINVAL (always strong);
 *   - kernel grain with strong ordering -> cooperative launch; a grid larger
 *     than the resident set -> GENESYS_EINVAL (this is the deadlock of Sec. 4.1).
 * The kernel-grain call sites are reset on `stream` before every kernel
 * (whatever grain `flags` declares): a relaxed kernel-grain site serves one
 * call per block per launch (genesys_device.cuh, call_at).
 * GENESYS_LAUNCH_GRAPH (no counterpart in the paper, which launches kernels
 * directly; it cuts the launch cost of kernels relaunched with new
 * arguments): the first launch of a (kernel, grid, block, smem_bytes,
 * cooperative) shape builds a graph of that one kernel node and instantiates
 * it; later launches of the shape set the node's arguments to `args` on the
 * instantiated graph and launch it (cudaGraphExecKernelNodeSetParams +
 * cudaGraphLaunch), so the kernel is not set up again.  The graphs belong to
 * the context (freed by genesys_shutdown); queued launches keep the arguments
 * they were given.  Set-up or launch failures are GENESYS_ECUDA. */
int genesys_launch(genesys_ctx *ctx, const void *kernel, const uint32_t grid[3], const uint32_t block[3],
                   size_t smem_bytes, void **args, uint32_t flags, void *stream);

/* Measurement only (no counterpart in the paper).  Device time (ms) of the
 * kernel of the most recent genesys_launch, from CUDA events recorded
 * immediately before and after it on its stream.  For non-blocking calls the
 * kernel can end before the CPU has processed them; genesys_drain covers the
 * rest. */
int genesys_last_launch_ms(genesys_ctx *ctx, float *ms);

/* CPU-side system call processing (Sec. 5) on the caller's thread.  With
 * GENESYS_INIT_NO_THREADS: process ready requests on the calling thread for up
 * to timeout_ns; returns the number of requests processed.  With service
 * threads: waits up to timeout_ns for all published requests to be processed;
 * returns 0 or GENESYS_ETIMEDOUT. */
int genesys_service(genesys_ctx *ctx, uint64_t timeout_ns);

/* Sec. 8.3: wait until every request published so far (non-blocking ones
 * included) has completed.  Call it after the kernels that made the calls
 * have finished (e.g. after a stream synchronize).  0 or GENESYS_ETIMEDOUT. */
int genesys_drain(genesys_ctx *ctx, uint64_t timeout_ns);

/* GPU mmap/munmap support (Sec. 5, Table 1's memory calls).  Unregister and
 * unmap the regions GPU code released with munmap.  A GPU munmap cannot do
 * this itself: cudaHostUnregister waits until no kernel is running, and the
 * calling kernel is running.  Released regions stay pinned until this call (or
 * genesys_shutdown) and are reused by later GPU mmaps of a size they fit.
 * Call it when no kernel that makes calls on this context is running. */
int genesys_reclaim(genesys_ctx *ctx);

/* GPU mmap support (Sec. 5).  Map (mmap(2), anonymous) and register n regions
 * of the given sizes (rounded up to pages) ahead of time, into the pool GPU
 * mmaps are served from. cudaHostRegister can stall while the GPU is busy with
 * other kernels (on a B300 a registration waited tens of seconds behind a
 * stream of kernels), and a kernel waiting for its mmap keeps the GPU busy:
 * reserving before the kernels start keeps registration off the path. */
int genesys_mmap_reserve(genesys_ctx *ctx, const uint64_t *sizes, uint32_t n);

/* Measurement of the service side (Sec. 4.2 coalescing, Sec. 7).  Copy the
 * service counters (genesys_stats: requests, Linux calls, batches, bytes,
 * failures, per-call-type time, the service threads' CPU time) into *out (host
 * memory, caller-owned).  GENESYS_EINVAL for NULL arguments. */
int genesys_stats_get(genesys_ctx *ctx, genesys_stats_t *out);
/* The same as genesys_stats_get, under the boundary's own name (Sec. 4.2,
 * Sec. 7: the service counters). */
int genesys_stats(genesys_ctx *ctx, genesys_stats_t *out);
/* Measurement only (no counterpart in the paper): launches made through
 * GENESYS_LAUNCH_GRAPH on this context so far, into *out. */
int genesys_graph_launches(genesys_ctx *ctx, uint64_t *out);
/* Zero the service counters; the service threads' CPU time counts from
 * here on.  Call between measurements, with no calls in flight. */
int genesys_stats_reset(genesys_ctx *ctx);

/* Copy the device status words (GENESYS_ST_*: timeouts and the first error,
 * including those of non-blocking calls nobody waits for, Sec. 4.1) into out;
 * clear them if `clear`. */
int genesys_status(genesys_ctx *ctx, int32_t out[GENESYS_ST_WORDS], int clear);

/* Invocation latency as Sec. 7 measures it.  Copy up to `cap` per-call latency
 * samples (ns, caller-side invocation latency) into out (host memory); *n_out
 * = samples recorded (may exceed cap); clears the buffer if `clear`. */
int genesys_latency(genesys_ctx *ctx, uint64_t *out, uint32_t cap, uint32_t *n_out, int clear);

/* Buffers GPU calls can name (Sec. 5 relies on shared virtual memory; here
 * pinned host-mapped memory stands in).  Bump-allocate `bytes` (256-byte
 * aligned) from the staging arena: pinned, host-mapped memory whose address is
 * valid on the host and on the GPU, so GPU code can pass it to
 * pread/pwrite/sendto/recvfrom.  NULL if exhausted. */
void *genesys_staging(genesys_ctx *ctx, size_t bytes);
/* Give the whole staging arena back (every earlier genesys_staging address
 * becomes free for reuse).  Only when no kernel or server uses staging. */
int genesys_staging_reset(genesys_ctx *ctx);

/* Message of the calling thread's last failure (interface plumbing, no
 * counterpart in the paper). */
const char *genesys_last_error(void);

/* Per-call trace (the timeline of a call, Sec. 5: publish, CPU pickup, CPU
 * completion, result seen), kept when genesys_config.trace_capacity > 0.
 * Device records are written by the calling GPU thread (device clock, ns);
 * host records by the service thread (CLOCK_MONOTONIC, ns).  A record pair
 * is joined by (slot, seq). */
/* (genesys_trace_dev and genesys_trace_host are defined in genesys_layout.h) */
/* Measurement only (where a call's time goes; no counterpart in the paper).
 * Copy out and clear the trace (call it with no kernel running on the
 * context): up to dev_cap / host_cap records (the rest is dropped and counted
 * in *n_dev / *n_host, which return the totals recorded).
 * *host_minus_device_ns (if non-NULL) = host clock - device clock, from a
 * round-trip calibration (the sample with the shortest round trip; error <=
 * half of it). */
int genesys_trace_read(genesys_ctx *ctx, genesys_trace_dev *dev, uint32_t dev_cap, uint32_t *n_dev,
                       genesys_trace_host *host, uint32_t host_cap, uint32_t *n_host, int64_t *host_minus_device_ns);

/* Interface check (no counterpart in the paper).  Size in bytes of a structure
 * of this interface, so that a binding built against another version of this
 * header can refuse to run instead of misreading memory: which =
 * GENESYS_SIZEOF_*; 0 for an unknown value. */
#define GENESYS_SIZEOF_CONFIG       0
#define GENESYS_SIZEOF_STATS        1
#define GENESYS_SIZEOF_SERVE_CONFIG 2
#define GENESYS_SIZEOF_SERVE_STATS  3
#define GENESYS_SIZEOF_TRACE_DEV    4
#define GENESYS_SIZEOF_TRACE_HOST   5
#define GENESYS_SIZEOF_C5_REQUEST   6
#define GENESYS_SIZEOF_DEV          7
uint32_t genesys_sizeof(int which);

/* Failure detection on the host (no counterpart in the paper; a watchdog's
 * probe): *stalled_mask gets bit r
 * set for every doorbell ring r (r < 64) that has requests waiting but whose
 * service has finished no batch for stall_ns (a stopped, paused or stuck
 * service thread, or a NO_THREADS context nobody services); *pending (if
 * non-NULL) = requests published and not yet finished over all rings.  Cheap
 * enough to call periodically while kernels run. */
int genesys_service_health(genesys_ctx *ctx, uint64_t stall_ns, uint64_t *stalled_mask, uint64_t *pending);

/* Failure handling on the host (no counterpart in the paper): stop the service
 * thread of doorbell ring `ring` (it finishes the batch it holds), leave the
 * ring unserved for pause_ns, then start a new thread that continues from the
 * same ring position.  Requests published meanwhile wait in the ring; a caller
 * whose wait passes device_deadline_ns gives up with -ETIMEDOUT, and its
 * request is still carried out later.  GENESYS_EINVAL without service threads
 * or for a bad ring.  Blocks for pause_ns. */
int genesys_service_restart(genesys_ctx *ctx, uint32_t ring, uint64_t pause_ns);

/* Failure injection on the host for tests (no counterpart in the paper).
 * Checked builds only (GENESYS_DEVICE_CHECKS, libgenesys_checked.so): from now
 * on every pread the service threads make for GPU requests asks for at most
 * cap_bytes (0 = no cap), merged or not, so that GPU callers receive short
 * reads in the middle of a file, which Linux allows at any time (Sec. 5: the
 * CPU carries out the call and returns its result).  Callers that need whole
 * chunks go on reading (genesys::pread_full).  Other builds: GENESYS_EINVAL. */
int genesys_check_pread_cap(genesys_ctx *ctx, uint64_t cap_bytes);

/* Protocol testing without a GPU (no counterpart in the paper; the steps are
 * Sec. 5's).  GENESYS_INIT_HOST_ONLY contexts: make one call through the full
 * protocol from a CPU thread standing in for a GPU lane (claim a slot,
 * marshal, publish, ring the doorbell, wait if GENESYS_REQ_BLOCKING is in
 * flags). Safe to call from many threads at once.  *ret receives the result. */
int genesys_emulate_call(genesys_ctx *ctx, uint32_t nr, const uint64_t args[6], uint32_t flags, int64_t *ret);

/* ------------------------------------------------------------ workloads
 * Data-parallel kernels that make GPU system calls and consume their results.
 * Each returns 0, a negative GENESYS_E* code, or GENESYS_EDEVICE when a
 * device-side call failed or timed out (details via genesys_status).  All
 * launch on `stream` and return after the kernel finished and its calls
 * were drained. */

/* Forms of a workload. */
#define GENESYS_FORM_PLAIN   0u  /* work-group grain, strong ordering, blocking      */
#define GENESYS_FORM_BATCHED 1u  /* relaxed, non-blocking, double-buffered prefetch  */
#define GENESYS_FORM_WARP    2u  /* warp grain, strong ordering, blocking (C1)       */
#define GENESYS_FORM_HBM     3u  /* plain, each chunk copied to HBM and scanned there (C1) */

/* C1, Sec. 6 pread microbenchmark (Fig. 5): `groups` thread blocks of `threads`
 * threads read `file_bytes` bytes of `fd` with pread in `chunk`-byte pieces
 * (chunk i by block i mod groups) at work-group granularity and build a
 * 256-bin byte histogram, added into hist_dev[256] (device pointer, uint32).
 * form GENESYS_FORM_WARP reads at warp granularity instead: chunk i by warp
 * i mod (groups * threads / 32); GENESYS_FORM_HBM is the plain form with each
 * chunk moved from staging into an HBM landing buffer (the context's device
 * scratch, groups * chunk bytes) and counted there.  staging: host-mapped,
 * >= groups * chunk * (BATCHED: 2, WARP: threads / 32, PLAIN and HBM: 1)
 * bytes, 16-byte aligned; chunk a multiple of 16, threads a multiple of 32;
 * another form is GENESYS_EINVAL.  The batched form keeps up to
 * min(4, staging_bytes / (groups * chunk)) reads in flight per block (at
 * least 2; fewer if the slot area cannot hold that many per block). */
int genesys_c1_histogram(genesys_ctx *ctx, int fd, uint64_t file_bytes, uint64_t chunk, uint32_t groups,
                         uint32_t threads, uint32_t form, void *staging, uint64_t staging_bytes,
                         uint32_t *hist_dev, void *stream);

/* C2, the pwrite microbenchmark (Sec. 4.1 "Invocation granularity", Sec. 6):
 * n_threads GPU threads each write the 64 bytes splitmix64_at(seed, gid*8+k),
 * k = 0..7 (little-endian) to `fd` at offset gid*64.  `gran` (GENESYS_GRAN_*)
 * and `group_threads` (threads per block, 32..1024, multiple of 32) set the
 * invocation granularity: one pwrite per thread, per warp, per block, or one
 * for the whole kernel; `order_relaxed`/`nonblocking` the semantics.
 * staging: host-mapped, >= n_threads * 64 bytes.  Work-item grain with relaxed
 * ordering is GENESYS_EINVAL (Sec. 4.1); kernel grain with strong ordering runs
 * as a cooperative launch (grid-stride over the threads).  Per-call
 * latencies go to the context's sample buffer (genesys_latency). */
int genesys_c2_pwrite(genesys_ctx *ctx, int fd, uint64_t n_threads, uint32_t gran, uint32_t group_threads,
                      uint32_t order_relaxed, uint32_t nonblocking, uint64_t seed, void *staging,
                      uint64_t staging_bytes, void *stream);

/* C3, wordcount (Sec. 7.1): count whole-token occurrences of nq query words
 * (queries16[q*16 ..], qlen[q] bytes, 1..16 bytes, at most 64 queries; host
 * arrays) in n_files open files (fds[f], file_bytes[f]; host arrays).  A token
 * is a maximal run of bytes other than ' ' and '\n'.  One persistent kernel of
 * `ctas` blocks x `threads` pulls (file, chunk)-sized work items from a queue
 * and reads each with pread at work-group grain: GENESYS_FORM_PLAIN blocking
 * and strongly ordered, GENESYS_FORM_BATCHED relaxed and non-blocking with the
 * next item's read in flight while the current one is scanned.  Counts are
 * added into counts_dev[nq] (device, uint64).  staging: host-mapped,
 * >= ctas * (chunk + 64) * (BATCHED ? 2 : 1) bytes; chunk a multiple of 16.
 * The work-item list lives in a context-owned device scratch buffer. */
#define GENESYS_C3_MAX_QUERIES   64
#define GENESYS_C3_MAX_QUERY_LEN 16
int genesys_c3_wordcount(genesys_ctx *ctx, const int32_t *fds, const uint64_t *file_bytes, uint32_t n_files,
                         const uint8_t *queries16, const uint8_t *qlen, uint32_t nq, uint64_t chunk, uint32_t ctas,
                         uint32_t threads, uint32_t form, void *staging, uint64_t staging_bytes,
                         unsigned long long *counts_dev, void *stream);

/* Allocation-free variant of genesys_c3_wordcount (the paper has no
 * counterpart; this is a service for callers).  Some callers cannot allocate
 * device memory while they run: a process that must keep a fixed device
 * footprint after start-up, or a code path where a cudaMalloc/cudaFree - which
 * can synchronise the whole device - is not acceptable.  This entry point
 * makes no cudaMalloc, cudaFree or other allocating call: its per-call device
 * scratch (queue head, query table, work-item list) is a file-scope device
 * array of GENESYS_C3_NOALLOC_SCRATCH_BYTES (about 1 MiB) that every GPU which
 * loads the library holds until the process exits.  The caller still passes
 * all inputs and outputs, with the same meaning as for genesys_c3_wordcount.
 *   - Limit: at most GENESYS_C3_NOALLOC_MAX_ITEMS work items, where a file of
 *     n bytes takes ceil(n / chunk) of them; more returns GENESYS_EINVAL with
 *     a message saying so.
 *   - Set-up: the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current, keeps it, and makes the
 *     caller's current device current again; make that first call before any
 *     stream capture.
 *   - Sharing: every call uses the same array, which keeps the last call's
 *     contents (each call rewrites the part it reads, queue head included).
 *     Calls are serialised on the host and each waits for its kernel, but
 *     calls whose kernels overlap on the GPU would race on the array. */
#define GENESYS_C3_NOALLOC_MAX_ITEMS 32768u
#define GENESYS_C3_NOALLOC_SCRATCH_BYTES (1536u + GENESYS_C3_NOALLOC_MAX_ITEMS * 32u)
int genesys_c3_wordcount_noalloc(genesys_ctx *ctx, const int32_t *fds, const uint64_t *file_bytes,
                                 uint32_t n_files, const uint8_t *queries16, const uint8_t *qlen, uint32_t nq,
                                 uint64_t chunk, uint32_t ctas, uint32_t threads, uint32_t form, void *staging,
                                 uint64_t staging_bytes, unsigned long long *counts_dev, void *stream);

/* C5: serving a trace of syscall-issuing GPU kernels.  Each request is one
 * kernel of `threads` threads (blocks of block_threads) that runs up to
 * GENESYS_C5_MAX_OPS operations in order (Sec. 7 filesystem and memory calls):
 *   GENESYS_C5_PREAD  pread `len` bytes of in_fds[file] at `off`, split over
 *                     blocks (work-group grain, relaxed, blocking); result =
 *                     checksum of the bytes (see below);
 *   GENESYS_C5_PWRITE write `len` bytes of the splitmix64 stream of `seed` to
 *                     out_fd at `out_off` (work-group grain parts); result =
 *                     bytes written;
 *   GENESYS_C5_MMAP   mmap `len` (a multiple of 16) anonymous bytes at kernel grain (registered
 *                     for device access), fill word i with
 *                     splitmix64_at(seed, i), checksum it, munmap it at kernel
 *                     grain; result = checksum.
 * Checksum of a byte string: sum mod 2^64 over its little-endian 64-bit words
 * w_i (zero padded) of splitmix64's output function applied to
 * w_i + (i + 1) * 0x9E3779B97F4A7C15.
 * The server admits requests in arrival order once they have arrived
 * (arrival_ns after the call starts, if honor_arrivals) and a launch slot,
 * syscall slots, staging bytes and HBM bytes are free; launches them on
 * n_streams streams (launch slot i on stream i mod n_streams; as relaunched
 * single-kernel CUDA graphs if use_graphs);
 * retires them when their completion event fires.  With cfg.persistent, one
 * executor kernel of persistent_blocks blocks (block_threads each) runs for
 * the whole trace instead: admitting a request appends its blocks as work
 * units (request, block) to a ring in pinned host memory, the executor's
 * blocks take units in ring order and run them, the request's last block
 * writes its results to pinned memory, and the loop retires the request when
 * it sees them; uneven requests share the one launch and no launch is made
 * per request (max_inflight <= 65534; n_streams and use_graphs do not apply).
 * Outputs (host arrays): results[n_req * 8] (negative errno on failure),
 * latency_ns[n_req] (retirement - arrival); *stats if non-NULL. */
#define GENESYS_C5_MAX_OPS 8u
#define GENESYS_C5_MAX_PARTS 256u
#define GENESYS_C5_PREAD 0u
#define GENESYS_C5_PWRITE 1u
#define GENESYS_C5_MMAP 2u

typedef struct genesys_c5_op {
  uint32_t kind, file;
  uint64_t off, len, seed, out_off;
} genesys_c5_op;

typedef struct genesys_c5_request {
  uint64_t arrival_ns;
  uint32_t threads, n_ops;
  genesys_c5_op ops[GENESYS_C5_MAX_OPS];
} genesys_c5_request;

typedef struct genesys_serve_config {
  uint32_t max_inflight;    /* launch slots: requests on the GPU at once          */
  uint32_t n_streams;
  uint64_t staging_budget;  /* pinned bytes for in-flight requests' pwrite data    */
  uint64_t hbm_budget;      /* device bytes for in-flight requests' pread landing  */
  uint32_t slot_budget;     /* syscall-area slots in-flight requests may hold      */
  uint32_t block_threads;
  uint32_t min_part;        /* smallest per-block share of a pread/pwrite (bytes): the
                               invocation granularity knob the autotuner sets      */
  uint32_t use_graphs;
  uint32_t pread_to_hbm;    /* 1: pread data is moved to HBM and scanned there     */
  uint32_t honor_arrivals;  /* 1: open loop on arrival_ns; 0: all present at start */
  uint32_t reserve_mmaps;   /* 1: map and register the trace's mmap regions before
                               the first request (genesys_mmap_reserve)            */
  uint64_t timeout_ns;      /* give up (GENESYS_ETIMEDOUT) after this long         */
  uint32_t persistent;      /* 1: one persistent executor kernel serves the whole
                               trace (below); 0: one kernel launch per request     */
  uint32_t persistent_blocks; /* executor blocks (0: as many as can be resident)   */
} genesys_serve_config;

typedef struct genesys_serve_stats {
  uint64_t requests, syscalls, makespan_ns, max_inflight, admission_wait_ns, graph_launches;
} genesys_serve_stats;

/* Fill *cfg with the defaults: 64 launch slots on 64 streams; budgets of
 * 64 MiB staging, 64 MiB HBM and 16,384 syscall slots; 256-thread blocks;
 * min_part 16 KiB; graphs on; pread data scanned where it lands; arrivals
 * honoured; mmaps reserved; 120 s timeout. */
int genesys_serve_config_default(genesys_serve_config *cfg);
int genesys_c5_serve(genesys_ctx *ctx, const genesys_c5_request *reqs, uint32_t n_req, const int32_t *in_fds,
                     uint32_t n_in, int32_t out_fd, const genesys_serve_config *cfg, uint64_t *results,
                     uint64_t *latency_ns, genesys_serve_stats *stats);

/* C4, key-value service over UDP (Sec. 7.3 networking): the server is a
 * persistent GPU kernel, one block per UDP socket on 127.0.0.1:port_base + w,
 * that receives request batches with recvmmsg and answers them with sendmmsg
 * (work-group grain GPU system calls; non-blocking receive polls).  The table
 * lives in device memory: n_keys 16-byte keys (keys[16 * i]) in an
 * open-addressing index, values in GENESYS_KV_VALUE_MAX-byte slots, preloaded
 * with value i = the first vlen0[i] bytes of the splitmix64 stream of seed
 * vseed0[i] (host arrays).  Requests for one key must all go to one socket
 * (the client sends to (first four key bytes, little-endian) mod n_sockets);
 * a block applies a batch's requests in arrival order per key.
 * Request: op u8 (GENESYS_KV_GET/SET/STOP), pad u8, vlen u16, seq u32,
 * key[16], value[vlen] (SET).  Reply: op|0x80 u8, status u8 (0 ok, 1 no such
 * key), vlen u16, seq u32, value[vlen] (GET of a present key).  A block leaves
 * on a STOP datagram, when genesys_kv_stop sets the stop flag and it is idle,
 * or after idle_timeout_ns without datagrams. */
#define GENESYS_KV_VALUE_MAX 1024u
#define GENESYS_KV_MAX_BATCH 64u
#define GENESYS_KV_GET 0u
#define GENESYS_KV_SET 1u
#define GENESYS_KV_STOP 2u
typedef struct genesys_kv_server genesys_kv_server;
int genesys_kv_start(genesys_ctx *ctx, const uint8_t *keys, const uint16_t *vlen0, const uint64_t *vseed0,
                     uint32_t n_keys, uint32_t n_sockets, uint32_t batch, uint32_t threads, uint16_t port_base,
                     uint64_t idle_timeout_ns, genesys_kv_server **out);
/* Stop the server (bounded by timeout_ns), drain its calls, free it; *served
 * (if non-NULL) = replies sent.  On an error (GENESYS_ETIMEDOUT: the kernel
 * has not left, or its calls did not drain) the server is kept and the call
 * can be repeated; the context cannot be shut down until one succeeds. */
int genesys_kv_stop(genesys_kv_server *srv, uint64_t timeout_ns, uint64_t *served);
/* C4 (Sec. 7.3; lost datagrams are read this way: the server logs the
 * requests it received and the oracle replays exactly those).  Bit j of
 * out[j / 32] (host array of (n_seqs + 31) / 32 words) is set when the
 * request whose seq field is j reached the server, for j < n_seqs <=
 * GENESYS_KV_SEQ_LOG (requests with larger seq are not logged).  Call it
 * after the load has ended, before genesys_kv_stop.  GENESYS_EINVAL for NULL
 * arguments or n_seqs too large. */
#define GENESYS_KV_SEQ_LOG (1u << 24)
int genesys_kv_received(genesys_kv_server *srv, uint32_t *out, uint64_t n_seqs);
/* C4 (Sec. 7.3).  Current value of key k (copied to out, GENESYS_KV_VALUE_MAX
 * bytes room); returns its length. */
int genesys_kv_value(genesys_kv_server *srv, uint32_t k, uint8_t *out);
/* C4's load generator (Sec. 7.3 measures its network workloads with a client
 * on the host).  Open-loop UDP load generator on up to 8 host threads (no
 * more than the CPUs the calling thread may run on: restricting the caller's
 * CPU set gives the generator its own cores), each with its own socket: request j (reqs + req_off[j], req_off[n] = end) is sent
 * arrival_ns[j] after start to the socket its key maps to, by the thread that
 * owns that socket (so one key's requests leave in order), and its reply comes
 * back to that thread; replies are matched by seq into replies[seq * (8 +
 * VALUE_MAX)], reply_len[seq], latency_ns[seq] (send to receive).  Then sends
 * STOP to every socket.  stats[6]: received, duplicates, malformed, send
 * errors, largest send lateness (ns), first send to last reply (ns).
 * GENESYS_ETIMEDOUT if replies are still missing timeout_ns after the last
 * arrival. */
int genesys_kv_client(const uint8_t *reqs, const uint64_t *req_off, uint64_t n, const uint64_t *arrival_ns,
                      uint16_t port_base, uint32_t n_sockets, uint64_t timeout_ns, uint8_t *replies,
                      uint32_t *reply_len, uint64_t *latency_ns, uint64_t *stats);

/* UDP echo server (Sec. 7.3, Fig. 10: bandwidth versus packet size; the GPU
 * part of the paper's echo server calls recvfrom/sendto at work-group grain,
 * blocking, weak ordering).  A persistent GPU kernel, one block per UDP
 * socket on 127.0.0.1:port_base + w.  form GENESYS_ECHO_SINGLE: a block
 * receives one datagram with recvfrom; GENESYS_ECHO_BATCH: up to `batch`
 * (1..GENESYS_ECHO_MAX_BATCH) with recvmmsg.  The block copies each datagram
 * through its SMs from a receive buffer to a send buffer (both in the
 * context's host-mapped staging, 2 * batch * max_packet bytes per socket plus
 * headers) and sends it back to its sender (sendto / sendmmsg).  Datagrams
 * are at most max_packet (8..GENESYS_ECHO_PACKET_MAX) bytes; a datagram of
 * GENESYS_ECHO_STOP_BYTES bytes ends its block, as do genesys_echo_stop and
 * idle_timeout_ns without datagrams (0 = 10 s).  Errors: GENESYS_EINVAL
 * (argument ranges, bind failure), GENESYS_ENOMEM (staging too small). */
#define GENESYS_ECHO_PACKET_MAX 65504u
#define GENESYS_ECHO_MAX_BATCH 64u
#define GENESYS_ECHO_STOP_BYTES 4u
#define GENESYS_ECHO_SINGLE 0u
#define GENESYS_ECHO_BATCH 1u
typedef struct genesys_echo_server genesys_echo_server;
int genesys_echo_start(genesys_ctx *ctx, uint32_t n_sockets, uint32_t max_packet, uint32_t form, uint32_t batch,
                       uint32_t threads, uint16_t port_base, uint64_t idle_timeout_ns, genesys_echo_server **out);
/* Stop the echo server (bounded by timeout_ns), drain its calls and free it;
 * stats[2] (if non-NULL): datagrams echoed, bytes echoed.  On an error the
 * server is kept and the call can be repeated, as for genesys_kv_stop. */
int genesys_echo_stop(genesys_echo_server *srv, uint64_t timeout_ns, uint64_t *stats);
/* Fig. 10's client side.  Closed-loop UDP echo load generator on n_threads
 * host threads (each with its own socket and the server sockets s = t, t +
 * n_threads, ...): `window` datagrams of packet_bytes
 * (8..GENESYS_ECHO_PACKET_MAX) in flight per server socket (fewer if the
 * replies would not fit in half of the thread's receive buffer), n_packets in
 * total.  A datagram is lane u32, generation u32, then seeded bytes; a reply
 * counts as echoed when it equals the datagram byte for byte.  Ends when every
 * datagram is answered or no reply came for stall_ns (0 = 200 ms); then, if
 * send_stop, sends a GENESYS_ECHO_STOP_BYTES datagram to every server socket.
 * stats[7]: sent, echoed, bad replies, lost (no reply), first send to last
 * reply (ns), echoed bytes, send errors. */
int genesys_echo_client(uint16_t port_base, uint32_t n_sockets, uint32_t packet_bytes, uint64_t n_packets,
                        uint32_t window, uint32_t n_threads, uint64_t seed, uint64_t stall_ns, uint32_t send_stop,
                        uint64_t *stats);

/* Service-rate ceiling for work-item pwrites (Sec. 5, CPU-side system call
 * processing): the calling host thread publishes n_calls requests
 * pwrite(fd, payload + i * bytes_per_call, bytes_per_call, i * bytes_per_call)
 * into the slot area, one slot each, as a work-item-grain blocking launch
 * would (slots filled first, in rounds of n_slots; one doorbell entry for 32
 * consecutive slots that start at a multiple of 32, as a full warp rings),
 * and *elapsed_ns is the
 * time from the first doorbell entry to the last completion, summed over the
 * rounds: the service threads' time alone, with no GPU in the loop.  payload
 * is a host address.  The context must be idle (no kernel running, no slot
 * claimed: GENESYS_EINVAL otherwise); its device-side sequence numbers and
 * ring tails are updated so that kernels can continue to use it.  A call that
 * wrote fewer bytes than asked makes it return GENESYS_EINVAL. */
int genesys_service_probe(genesys_ctx *ctx, int fd, const void *payload, uint32_t bytes_per_call, uint64_t n_calls,
                          uint64_t *elapsed_ns);
/* The same probe with the doorbells rung out of file order, as GPU
 * work-items ring them: the calls are cut into runs of `run` consecutive ones
 * (32: a warp's), and run k is rung in pass k % stride of each round, so
 * neighbouring runs land a 1/stride of the round apart and rarely meet in one
 * batch (stride 8: the eight warps of a 256-thread block).  run = stride = 1
 * is genesys_service_probe.  GENESYS_EINVAL for run or stride 0, otherwise
 * as genesys_service_probe. */
int genesys_service_probe_order(genesys_ctx *ctx, int fd, const void *payload, uint32_t bytes_per_call,
                                uint64_t n_calls, uint32_t run, uint32_t stride, uint64_t *elapsed_ns);

/* C6, block permutation (Sec. 6, Fig. 6): n_blocks thread blocks of 1024
 * threads each take one 8 KiB block of input_dev (device), permute it `iters`
 * times with out[i] = in[perm_dev[i]] (perm_dev: 8192 uint16, device), copy it
 * to staging + b * 8 KiB (host-mapped, >= n_blocks * 8 KiB) and pwrite it to
 * fd at offset b * 8 KiB at work-group grain, strong or relaxed, blocking or
 * non-blocking - the four combinations of Fig. 6. */
int genesys_c6_permute(genesys_ctx *ctx, int fd, const uint8_t *input_dev, const uint16_t *perm_dev, uint64_t n_blocks,
                       uint32_t iters, uint32_t relaxed, uint32_t nonblocking, void *staging, uint64_t staging_bytes,
                       void *stream);

/* One system call made from GPU code (Sec. 5: any system call, function-like):
 * one block of `threads` threads calls `nr` with args[6] at work-item (1
 * thread), warp or work-group grain, strong and blocking; the result (>= 0 or
 * -errno) is stored to *ret_dev (device, int64).  Pointer arguments must be
 * host-usable addresses (staging).  A failed call is a result, not an error
 * of this function; a device-side timeout is GENESYS_EDEVICE. */
int genesys_gpu_call(genesys_ctx *ctx, uint32_t nr, const uint64_t args[6], uint32_t gran, uint32_t threads,
                     long long *ret_dev, void *stream);

/* Strong-ordering visibility probe (Sec. 4.1: strong ordering means every
 * store before the call has completed): n_threads threads each store their
 * 8-byte word splitmix64_at(seed, gid) into probe[gid] (host-mapped), then a
 * group of the given grain calls GENESYS_NR_CHECK_VISIBLE on the group's
 * words; the CPU counts the words that are not yet visible.  The sum over
 * calls is written to *violations_dev (device pointer, uint64). */
int genesys_visibility_probe(genesys_ctx *ctx, uint64_t n_threads, uint32_t gran, uint32_t group_threads,
                             uint32_t order_relaxed, uint64_t seed, uint64_t *probe,
                             unsigned long long *violations_dev, void *stream);

/* Host-link round trip (the latency floor of a blocking GPU system call,
 * Sec. 5: the GPU publishes a request and waits for the CPU's answer): one GPU
 * thread on `device` stores r to a flag in pinned host-mapped memory and waits
 * for a host thread to store r to a second flag, r = 1 .. rounds.
 * *ns_per_round = GPU-timed nanoseconds per round trip.  Every wait, on both
 * sides, ends after timeout_ns (GENESYS_ETIMEDOUT); no context is needed. */
int genesys_link_pingpong(int device, uint32_t rounds, uint64_t timeout_ns, uint64_t *ns_per_round);

/* Zero-copy host-link bandwidth of the SMs (the ceiling of a consumer kernel
 * that reads what a pread landed in pinned staging, Sec. 7.1, or of a kernel
 * writing what a pwrite sends): blocks x threads GPU threads on `device`
 * stream over `bytes` of pinned, host-mapped memory at host address
 * `host_buf` (the caller's; for example a context's staging, or any memory
 * pinned by cudaHostAlloc or cudaHostRegister with mapping) with 16-byte
 * loads (write = 0) or 16-byte stores (write = 1) that cover every word
 * once, or both at once (write = 2: the even blocks read the first half of
 * the buffer while the odd blocks write the second half).  *gb_per_s = bytes
 * (both directions together for write = 2) / the fastest of `reps` launches
 * (CUDA events) after one warm-up.  Use more bytes than the GPU's L2 holds, or reads may be
 * served from it.  GENESYS_EINVAL: NULL pointers, a buffer not 16-byte aligned
 * or not a positive multiple of 16 bytes, reps 0, blocks outside 1..65535,
 * threads not a multiple of 32 up to 1024, write outside 0..2 (2: fewer than
 * 2 blocks or bytes not a multiple of 32), or memory that is not pinned and
 * mapped.  The caller's current device is unchanged. */
int genesys_link_stream(int device, void *host_buf, uint64_t bytes, int write, uint32_t blocks, uint32_t threads,
                        uint32_t reps, double *gb_per_s);

#ifdef __cplusplus
}
#endif

#endif /* GENESYS_H */
