// Host side of GPU system calls: context, syscall area, doorbell rings and the
// CPU service threads that carry out the GPU's requests.
//
// Paper: Vesely et al., "GPU System Calls", arXiv 1705.06965.
//   Sec. 5 "CPU-side system call processing": a CPU worker scans the syscall
//   area for ready requests, marks them as processing, executes the call and
//   writes the result back (Fig. 4); coalescing batches several requests into
//   one unit of work, bounded by a time window and a maximum count (Sec. 4.2).
//   Sec. 8.3: a host function waits until all GPU calls have completed.
//
// B300 design (x86-64 host, PCIe Gen6, no host-native atomics): the service
// threads are user-mode pollers (the model of the paper's related work, Sec. 9;
// Sec. 3 calls interrupt vs polling orthogonal).  Each owns one doorbell ring
// that GPU callers append slot numbers to, so a thread reads only the slots
// that have work instead of scanning the whole syscall area.
#include <cuda_runtime.h>
#include <errno.h>
#include <fcntl.h>
#include <pthread.h>
#include <sched.h>
#include <string.h>
#include <sys/mman.h>
#include <sys/socket.h>
#include <sys/syscall.h>
#include <sys/uio.h>
#include <time.h>
#include <unistd.h>

#include <algorithm>
#include <cstdarg>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <thread>
#include <map>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "genesys.h"
#include "internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return fail(GENESYS_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

inline void cpu_relax() { __builtin_ia32_pause(); }

inline uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// splitmix64 output function (Steele, Lea & Flood 2014), counter-based:
// value i of the generator started at `seed`.  Used only by the visibility
// probe op, which checks GPU stores of this pattern.
inline uint64_t sm64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

enum OpIdx { OP_PREAD = 0, OP_PWRITE, OP_SENDTO, OP_RECVFROM, OP_MMAP, OP_MUNMAP, OP_INTERNAL, OP_OTHER };

// Each ring's counters are written by its service thread only (or under the
// service mutex), so an increment is a relaxed load and store, not a locked
// read-modify-write; genesys_stats_get reads them with relaxed loads.
inline void bump(std::atomic<uint64_t> &a, uint64_t v) {
  a.store(a.load(std::memory_order_relaxed) + v, std::memory_order_relaxed);
}

struct alignas(64) Counters {
  std::atomic<uint64_t> requests{0}, os_calls{0}, failed{0}, nb_failed{0}, bytes{0}, batches{0}, busy_ns{0};
  std::atomic<uint64_t> by_op[8] = {};
  std::atomic<uint64_t> op_ns[8] = {}, op_max_ns[8] = {};
  std::atomic<uint64_t> last_batch_ns{0};  // when the ring's last batch was finished
  // where a batch's time goes: taking it (slot reads, any coalescing window),
  // ordering it for merging, and writing its results back; the Linux calls
  // themselves are op_ns
  std::atomic<uint64_t> pickup_ns{0}, order_ns{0}, complete_ns{0};
  // polls that found the entry at the ring's head not yet written; of those,
  // the ones where a later entry was already written (a position taken on
  // the GPU whose entry had not arrived: a hole that holds up the ring)
  std::atomic<uint64_t> empty_polls{0}, hole_polls{0};
};

struct Request {
  uint32_t slot, seq, nr, flags;
  uint64_t a[6];
  int64_t ret;
  uint32_t entry;  // index, within its batch, of the ring entry that announced it
};

// One service batch and the scratch its processing needs (owned by one
// service thread, or by the caller of genesys_service / genesys_drain).
struct Batch {
  std::vector<Request> req;
  std::vector<Request *> ptr;      // processing order
  std::vector<uint32_t> run;       // first request of each run, then n
  std::vector<int32_t> next;       // run that continues this one in its file, or -1
  std::vector<uint8_t> has_pred;
  std::vector<uint32_t> hidx, hgen;  // open-addressing table: (call, fd, offset) -> run
  std::vector<uint32_t> slot_ids;    // slots of the ready ring entries
  std::vector<uint32_t> entry_of;    // ring entry (index within the batch) of each request
  std::vector<uint32_t> left;        // per ring entry: its requests not yet completed
  std::vector<uint64_t> done_ns;     // per request: when its completion word was written
  uint32_t n_entries = 0, prefix = 0;  // entries taken; leading entries wholly completed
  uint64_t head = 0;                 // ring position of the batch's first entry
  uint32_t gen = 0;
  size_t target;                     // requests a batch takes (coalesce_max)
  // room for the target and one more ring entry's requests (entries are taken whole)
  explicit Batch(size_t want)
      : req(want + GENESYS_RING_MAX_RUN - 1), ptr(req.size()), run(req.size() + 1), next(req.size()),
        has_pred(req.size()), slot_ids(req.size()), entry_of(req.size()), left(req.size()),
        done_ns(req.size()), target(want) {
    size_t cap = 16;
    while (cap < 2 * req.size()) cap <<= 1;
    hidx.assign(cap, 0);
    hgen.assign(cap, 0);
  }
};

}  // namespace

struct genesys_ctx {
  genesys_config cfg{};
  int device = -1;
  bool host_only = false;
  uint32_t n_sms = 0;

  // host-mapped (or plain host memory in host-only mode)
  genesys_slot *slots = nullptr;
  uint64_t *done = nullptr;
  uint64_t *rings = nullptr;
  uint64_t *ring_done = nullptr;  // per ring: GENESYS_RING_DONE_COPIES copies of the finished count
  uint32_t ring_cap = 0;
  uint8_t *staging = nullptr;
  std::atomic<uint64_t> staging_used{0};

  // device-side state (device memory; host memory in host-only mode)
  uint32_t *owner = nullptr, *seq = nullptr, *known_done = nullptr, *ring_tail = nullptr;
  genesys_ksite *ksite = nullptr;
  uint32_t *grid_bar = nullptr;
  int32_t *status = nullptr;
  uint64_t *lat = nullptr;
  uint32_t *lat_count = nullptr;

  // service side
  std::vector<std::thread> threads;
  std::atomic<bool> stop{false};
  std::atomic<int> servers{0};  // persistent server kernels running on the context
  std::unique_ptr<std::atomic<bool>[]> ring_stop;  // per ring: its thread should leave
  std::mutex restart_mu;
  std::vector<uint64_t> head;                       // per ring, touched by its thread only
  std::unique_ptr<std::atomic<uint64_t>[]> retired;  // per ring: positions fully processed
  std::unique_ptr<Counters[]> counters;             // per ring
  std::mutex svc_mu;                                // NO_THREADS mode: one caller at a time

  // Regions the GPU mapped with mmap, registered for device access.
  // cudaHostUnregister waits until no kernel is running, so a GPU munmap
  // cannot unregister while its own kernel waits for the answer: the region
  // moves to `released` (still mapped and pinned) and is unregistered and
  // unmapped at the next genesys_reclaim / shutdown; a later GPU mmap of a
  // size it fits reuses it instead of mapping and pinning new memory.
  struct Mapping {
    void *host;
    size_t region;     // bytes mapped and registered
    size_t len;        // bytes the GPU asked for
  };
  std::mutex map_mu;
  std::unordered_map<uintptr_t, Mapping> maps;      // live: device address -> mapping
  std::multimap<size_t, std::pair<uintptr_t, Mapping>> released;  // by region size
  std::atomic<uint64_t> mmap_new{0}, mmap_reused{0};

  cudaStream_t aux = nullptr;  // private stream for small copies
  // pinned landing buffers of the small device-to-host reads made after every
  // launch (ring positions, status words): a copy into pageable memory is
  // staged by the driver and takes about twice as long
  uint32_t *tails_host = nullptr;
  int32_t *status_host = nullptr;
  std::mutex small_mu;  // one such read at a time
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // around the last launched kernel

  void *scratch = nullptr;  // device scratch arena for workload entry points
  size_t scratch_bytes = 0;

  // per-call trace (cfg.trace_capacity > 0): device records in device memory,
  // host records per ring (written by that ring's service thread only)
  genesys_trace_dev *trace = nullptr;
  uint32_t *trace_count = nullptr;
  std::vector<std::vector<genesys_trace_host>> trace_host;
  std::unique_ptr<std::atomic<uint32_t>[]> trace_n;  // host records written per ring (may exceed capacity)

  // CPU time of service threads that have left (restarts), and the total at
  // the last genesys_stats_reset
  std::atomic<uint64_t> cpu_retired_ns{0};
  uint64_t cpu_reset_ns = 0;

  // checked builds: the last sequence number the service saw per slot (each
  // slot's requests go through one ring, so one thread writes each entry)
  std::vector<uint32_t> last_seq;
  std::atomic<uint64_t> protocol_errors{0};
  uint64_t created_ns = 0;
  // checked builds: every pread made for GPU requests asks for at most this
  // many bytes (0 = no cap), so that callers meet short reads mid-file
  uint64_t pread_cap = 0;

  // GENESYS_LAUNCH_GRAPH: one single-kernel graph per launch shape, relaunched
  // with each call's arguments
  struct GraphKey {
    const void *kernel;
    uint32_t grid[3], block[3];
    size_t smem;
    bool coop;
    bool operator<(const GraphKey &o) const {
      return std::tie(kernel, grid[0], grid[1], grid[2], block[0], block[1], block[2], smem, coop) <
             std::tie(o.kernel, o.grid[0], o.grid[1], o.grid[2], o.block[0], o.block[1], o.block[2], o.smem, o.coop);
    }
  };
  struct GraphExec {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
  };
  std::mutex graph_mu;
  std::map<GraphKey, GraphExec> graphs;
  std::atomic<uint64_t> graph_launches{0};
};

namespace {

// -------------------------------------------------------------- requests

void complete(genesys_ctx *c, const Request &r, Counters &k) {
  const bool fits = r.ret >= INT32_MIN + 1 && r.ret <= INT32_MAX;
  uint64_t word = (uint64_t)r.seq << 32;
  if (fits) {
    word |= (uint32_t)(int32_t)r.ret;
  } else {
    __atomic_store_n(&c->slots[r.slot].ret, (uint64_t)r.ret, __ATOMIC_RELAXED);
    word |= GENESYS_RET_IN_SLOT;
  }
  if (r.ret < 0) {
    bump(k.failed, 1);
    if (!(r.flags & GENESYS_REQ_BLOCKING) && !(r.flags & GENESYS_REQ_TICKET))
      bump(k.nb_failed, 1);
  }
  __atomic_store_n(&c->done[r.slot], word, __ATOMIC_RELEASE);
}

int op_index(uint32_t nr) {
  switch (nr) {
    case SYS_pread64: return OP_PREAD;
    case SYS_pwrite64: return OP_PWRITE;
    case SYS_sendto: case SYS_sendmmsg: return OP_SENDTO;
    case SYS_recvfrom: case SYS_recvmmsg: return OP_RECVFROM;
    case SYS_mmap: return OP_MMAP;
    case SYS_munmap: return OP_MUNMAP;
    default: return nr >= 0x7F00u ? OP_INTERNAL : OP_OTHER;
  }
}

bool allowed(const genesys_ctx *c, uint32_t nr) {
  if (c->cfg.flags & GENESYS_INIT_ANY_SYSCALL) return true;
  switch (nr) {
    case SYS_read: case SYS_write: case SYS_pread64: case SYS_pwrite64: case SYS_open: case SYS_openat:
    case SYS_close: case SYS_lseek: case SYS_sendto: case SYS_recvfrom: case SYS_sendmmsg:
    case SYS_recvmmsg: case SYS_madvise: case SYS_getpid: case SYS_fsync:
      return true;
    default:
      return false;
  }
}

inline int64_t sys_ret(long r) { return r < 0 ? -(int64_t)errno : (int64_t)r; }

// mmap from the GPU: an anonymous private mapping is served from a released
// region of a fitting size when there is one (zeroed, unless the caller passed
// MAP_UNINITIALIZED because it overwrites the whole region), otherwise mapped
// with mmap(2) and registered for device access.  Other mappings go straight
// to mmap(2) + registration.  Returns the device address.
#ifndef MAP_UNINITIALIZED
#define MAP_UNINITIALIZED 0x4000000
#endif
int64_t do_mmap(genesys_ctx *c, const uint64_t *a) {
  const size_t len = (size_t)a[1];
  const int prot = (int)a[2], flags = (int)a[3], fd = (int)a[4];
  if (len == 0) return -EINVAL;
  const bool anon = a[0] == 0 && (flags & MAP_ANONYMOUS) && (flags & MAP_PRIVATE) && a[5] == 0;
  if (anon && !c->host_only) {
    std::lock_guard<std::mutex> g(c->map_mu);
    auto it = c->released.lower_bound(len);
    if (it != c->released.end() && it->first <= 2 * len) {
      auto m = it->second;
      c->released.erase(it);
      if (!(flags & MAP_UNINITIALIZED)) memset(m.second.host, 0, m.second.region);
      m.second.len = len;
      c->maps[m.first] = m.second;
      c->mmap_reused.fetch_add(1, std::memory_order_relaxed);
      return (int64_t)m.first;
    }
  }
  void *p = mmap((void *)a[0], len, prot, flags & ~MAP_UNINITIALIZED, fd, (off_t)a[5]);
  if (p == MAP_FAILED) return -(int64_t)errno;
  uintptr_t dev = (uintptr_t)p;
  if (!c->host_only) {
    if (cudaHostRegister(p, len, cudaHostRegisterMapped | cudaHostRegisterPortable) != cudaSuccess) {
      cudaGetLastError();
      munmap(p, len);
      return -ENOMEM;
    }
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) {
      cudaGetLastError();
      c->released.emplace(len, std::make_pair((uintptr_t)p, genesys_ctx::Mapping{p, len, len}));
      return -ENOMEM;
    }
    dev = (uintptr_t)d;
  }
  c->mmap_new.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> g(c->map_mu);
  c->maps[dev] = {p, len, len};
  return (int64_t)dev;
}

// munmap from the GPU (whole GPU-made mappings only): the region is released
// for reuse; genesys_reclaim unregisters and unmaps it once no kernel runs.
int64_t do_munmap(genesys_ctx *c, const uint64_t *a) {
  std::lock_guard<std::mutex> g(c->map_mu);
  auto it = c->maps.find((uintptr_t)a[0]);
  if (it == c->maps.end()) return -EINVAL;
  if ((size_t)a[1] != it->second.len) return -EINVAL;
  if (c->host_only) {
    const int r = munmap(it->second.host, it->second.region);
    c->maps.erase(it);
    return r == 0 ? 0 : -(int64_t)errno;
  }
  c->released.emplace(it->second.region, std::make_pair(it->first, it->second));
  c->maps.erase(it);
  return 0;
}

// Unregister and unmap released regions (and, at shutdown, live ones).
void reclaim(genesys_ctx *c, bool all) {
  std::lock_guard<std::mutex> g(c->map_mu);
  for (auto &kv : c->released) {
    if (!c->host_only) cudaHostUnregister(kv.second.second.host);
    munmap(kv.second.second.host, kv.second.second.region);
  }
  c->released.clear();
  if (all) {
    for (auto &kv : c->maps) {
      if (!c->host_only) cudaHostUnregister(kv.second.host);
      munmap(kv.second.host, kv.second.region);
    }
    c->maps.clear();
  }
}

// One positional read or write for one request, as its own Linux call would
// be made (pread asks for at most pread_cap bytes when a cap is set).
int64_t rw_one(const genesys_ctx *c, const Request &r) {
  void *buf = (void *)r.a[1];
  uint64_t len = r.a[2];
  if (r.nr == SYS_pread64) {
    if (c->pread_cap && len > c->pread_cap) len = c->pread_cap;
    return sys_ret(pread((int)r.a[0], buf, len, (off_t)r.a[3]));
  }
  return sys_ret(pwrite((int)r.a[0], buf, len, (off_t)r.a[3]));
}

int64_t execute_one(genesys_ctx *c, Request &r, Counters &k) {
  const uint64_t *a = r.a;
  bump(k.os_calls, 1);
  switch (r.nr) {
    case GENESYS_NR_NOP:
      bump(k.os_calls, (uint64_t)-1);
      return (int64_t)a[0];
    case GENESYS_NR_CHECK_VISIBLE: {
      bump(k.os_calls, (uint64_t)-1);
      const volatile uint64_t *p = (const volatile uint64_t *)a[0];
      int64_t bad = 0;
      for (uint64_t i = 0; i < a[1]; ++i) bad += p[i] != sm64_at(a[2], a[3] + i);
      return bad;
    }
    case SYS_mmap:
      return do_mmap(c, a);
    case SYS_munmap:
      return do_munmap(c, a);
    case SYS_pread64:
    case SYS_pwrite64:
      return rw_one(c, r);
    default:
      if (!allowed(c, r.nr)) return -ENOSYS;
      return sys_ret(syscall((long)r.nr, a[0], a[1], a[2], a[3], a[4], a[5]));
  }
}

// Merge a run of pread/pwrite requests that continue each other in the file
// (same fd, offset of each = offset + length of the previous) into one Linux
// call.  Contiguous buffers become one pread/pwrite, others one
// preadv/pwritev.  Each request then receives the part of the merged result
// that covers its own range - the value its own call would have returned.
// A merged call can come back short of the run's total (a short read or
// write, or a fault in one request's buffer after earlier bytes were moved)
// or fail: the requests it covered in full keep their share, the one it
// covered in part keeps that part (a short count its own call could have
// returned), and every later request is made again as a call of its own, so
// that no request receives 0 or another's error for bytes its own call would
// have moved.
size_t merge_run(const genesys_ctx *c, Request *const *reqs, size_t i, size_t n, Counters &k) {
  const uint32_t nr = reqs[i]->nr;
  const int fd = (int)reqs[i]->a[0];
  size_t j = i + 1;
  bool contiguous_buf = true;
  while (j < n && j - i < IOV_MAX && reqs[j]->nr == nr && (int)reqs[j]->a[0] == fd &&
         reqs[j]->a[3] == reqs[j - 1]->a[3] + reqs[j - 1]->a[2]) {
    if (reqs[j]->a[1] != reqs[j - 1]->a[1] + reqs[j - 1]->a[2]) contiguous_buf = false;
    ++j;
  }
  const size_t m = j - i;
  const uint64_t off = reqs[i]->a[3];
  uint64_t total = 0;
  for (size_t t = i; t < j; ++t) total += reqs[t]->a[2];
  int64_t res;
  bump(k.os_calls, 1);
  const uint64_t e0 = genesys_mono_ns();
  if (m == 1) {
    res = rw_one(c, *reqs[i]);
  } else if (contiguous_buf) {
    void *buf = (void *)reqs[i]->a[1];
    const uint64_t ask = nr == SYS_pread64 && c->pread_cap ? std::min<uint64_t>(total, c->pread_cap) : total;
    long r = nr == SYS_pread64 ? pread(fd, buf, ask, (off_t)off) : pwrite(fd, buf, ask, (off_t)off);
    res = sys_ret(r);
  } else {
    iovec iov[IOV_MAX];
    size_t niov = m;
    for (size_t t = 0; t < m; ++t) iov[t] = {(void *)reqs[i + t]->a[1], (size_t)reqs[i + t]->a[2]};
    if (nr == SYS_pread64 && c->pread_cap && total > c->pread_cap) {  // ask for at most the cap
      uint64_t left = c->pread_cap;
      for (niov = 0; niov < m && left; ++niov) {
        if (iov[niov].iov_len > left) iov[niov].iov_len = (size_t)left;
        left -= iov[niov].iov_len;
      }
    }
    long r = nr == SYS_pread64 ? preadv(fd, iov, (int)niov, (off_t)off) : pwritev(fd, iov, (int)niov, (off_t)off);
    res = sys_ret(r);
  }
  uint64_t moved = res > 0 ? (uint64_t)res : 0;
  // requests the merged call covered (in full, or the one it covered in part)
  size_t t = i;
  uint64_t prefix = 0;
  if (m == 1) {
    reqs[t++]->ret = res;
  } else if (res >= 0) {
    for (; t < j; ++t) {
      const uint64_t len = reqs[t]->a[2];
      if ((uint64_t)res < prefix + len) break;
      reqs[t]->ret = (int64_t)len;
      prefix += len;
    }
    if (t < j && (uint64_t)res > prefix) {
      reqs[t]->ret = (int64_t)((uint64_t)res - prefix);
      ++t;
    }
  }
  // the rest: each as its own call
  for (; t < j; ++t) {
    bump(k.os_calls, 1);
    reqs[t]->ret = rw_one(c, *reqs[t]);
    if (reqs[t]->ret > 0) moved += (uint64_t)reqs[t]->ret;
  }
  const uint64_t dt = genesys_mono_ns() - e0;
  const int oi = nr == SYS_pread64 ? OP_PREAD : OP_PWRITE;
  bump(k.op_ns[oi], dt);
  if (dt > k.op_max_ns[oi].load(std::memory_order_relaxed)) k.op_max_ns[oi].store(dt, std::memory_order_relaxed);
  if (moved) bump(k.bytes, moved);
  return j;
}

inline bool is_rw(uint32_t nr) { return nr == SYS_pread64 || nr == SYS_pwrite64; }

// Requests p[0..m) of the batch are carried out: write their completion
// words now, and advance the ring's finished count past every leading entry
// whose requests are all complete.  A caller waits for the count to pass its
// entry, so completing call by call (instead of once the whole batch is done)
// lets the first requests of a batch go on while the service still works on
// the rest.
void finish(genesys_ctx *c, uint32_t ri, Batch &b, Request *const *p, size_t m, Counters &k) {
  const uint64_t now = c->cfg.trace_capacity ? genesys_mono_ns() : 0;
  for (size_t i = 0; i < m; ++i) {
    complete(c, *p[i], k);
    --b.left[p[i]->entry];
    b.done_ns[(size_t)(p[i] - b.req.data())] = now;
  }
  const uint32_t before = b.prefix;
  while (b.prefix < b.n_entries && b.left[b.prefix] == 0) ++b.prefix;
  if (b.prefix != before)
    for (uint32_t q = 0; q < GENESYS_RING_DONE_COPIES; ++q)
      __atomic_store_n(&c->ring_done[((size_t)ri * GENESYS_RING_DONE_COPIES + q) * 8], b.head + b.prefix,
                       __ATOMIC_RELEASE);
}

// Returns the time it finished (genesys_mono_ns).
uint64_t process_batch(genesys_ctx *c, uint32_t ri, Batch &b, size_t n, Counters &k) {
  const uint64_t t0 = genesys_mono_ns();
  Request *const req = b.req.data();
  Request **p = b.ptr.data();
  for (size_t i = 0; i < n; ++i) p[i] = req + i;
  if (c->cfg.merge && n > 1) {
    // The requests of a batch are concurrent, so any order is a legal
    // schedule.  A batch arrives as runs of requests that already continue
    // each other in their file (a warp's lanes publish in lane order).  Each
    // run is chained to the run of the same call and fd that starts where it
    // ends (a hash table keyed by call, fd and start offset; a run gets at
    // most one predecessor), and the chains are laid out one after the other,
    // so that neighbours in a file become adjacent and merge into one Linux
    // call.  Linear in the batch; the hashing is per run, not per request.
    auto continues = [](const Request &prev, const Request &r) {
      return is_rw(r.nr) && r.nr == prev.nr && (int)r.a[0] == (int)prev.a[0] && r.a[3] == prev.a[3] + prev.a[2];
    };
    uint32_t k = 0;
    b.run[k++] = 0;
    for (size_t i = 1; i < n; ++i)
      if (!continues(req[i - 1], req[i])) b.run[k++] = (uint32_t)i;
    b.run[k] = (uint32_t)n;
    if (k > 1) {
      const uint32_t mask = (uint32_t)b.hidx.size() - 1;
      if (++b.gen == 0) {
        std::fill(b.hgen.begin(), b.hgen.end(), 0u);
        b.gen = 1;
      }
      const uint32_t gen = b.gen;
      auto slot_of = [&](uint32_t nr, int fd, uint64_t off) {
        const uint64_t z =
            (off * 0x9E3779B97F4A7C15ull) ^ ((((uint64_t)(uint32_t)fd << 16) | nr) * 0xC2B2AE3D27D4EB4Full);
        return (uint32_t)(z >> 32) & mask;
      };
      auto starts = [&](uint32_t r, uint32_t nr, int fd, uint64_t off) {
        const Request &q = req[b.run[r]];
        return q.nr == nr && (int)q.a[0] == fd && q.a[3] == off;
      };
      for (uint32_t r = 0; r < k; ++r) {
        b.next[r] = -1;
        b.has_pred[r] = 0;
        const Request &q = req[b.run[r]];
        if (!is_rw(q.nr)) continue;
        uint32_t h = slot_of(q.nr, (int)q.a[0], q.a[3]);
        while (b.hgen[h] == gen && !starts(b.hidx[h], q.nr, (int)q.a[0], q.a[3])) h = (h + 1) & mask;
        if (b.hgen[h] != gen) {
          b.hgen[h] = gen;
          b.hidx[h] = r;
        }
      }
      for (uint32_t r = 0; r < k; ++r) {
        const Request &last = req[b.run[r + 1] - 1];
        if (!is_rw(last.nr) || last.a[2] == 0) continue;
        const uint64_t end = last.a[3] + last.a[2];
        uint32_t h = slot_of(last.nr, (int)last.a[0], end);
        while (b.hgen[h] == gen) {
          const uint32_t r2 = b.hidx[h];
          if (starts(r2, last.nr, (int)last.a[0], end)) {
            if (!b.has_pred[r2] && r2 != r) {
              b.next[r] = (int32_t)r2;
              b.has_pred[r2] = 1;
            }
            break;
          }
          h = (h + 1) & mask;
        }
      }
      size_t o = 0;
      for (uint32_t r = 0; r < k; ++r)
        if (!b.has_pred[r])
          for (int32_t q = (int32_t)r; q >= 0 && o < n; q = b.next[q])
            for (uint32_t i = b.run[q]; i < b.run[q + 1] && o < n; ++i) p[o++] = req + i;
      if (o != n)  // not reachable (offsets grow along a chain), kept as a guard
        for (size_t i = 0; i < n; ++i) p[i] = req + i;
    }
  }
  bump(k.order_ns, genesys_mono_ns() - t0);
  uint64_t cpl_ns = 0;  // time spent completing (writing completion words and the count)
  for (size_t i = 0; i < n;) {
    Request &r = *p[i];
    if (c->cfg.merge && (r.nr == SYS_pread64 || r.nr == SYS_pwrite64)) {
      const size_t j = merge_run(c, p, i, n, k);
      const uint64_t f0 = genesys_mono_ns();
      finish(c, ri, b, p + i, j - i, k);
      cpl_ns += genesys_mono_ns() - f0;
      i = j;
      continue;
    }
    const uint64_t e0 = genesys_mono_ns();
    r.ret = execute_one(c, r, k);
    const uint64_t e1 = genesys_mono_ns();
    const uint64_t dt = e1 - e0;
    const int oi = op_index(r.nr);
    bump(k.op_ns[oi], dt);
    if (dt > k.op_max_ns[oi].load(std::memory_order_relaxed)) k.op_max_ns[oi].store(dt, std::memory_order_relaxed);
    if (r.ret > 0 && (r.nr == SYS_pread64 || r.nr == SYS_pwrite64 || r.nr == SYS_read || r.nr == SYS_write ||
                      r.nr == SYS_sendto || r.nr == SYS_recvfrom))
      bump(k.bytes, (uint64_t)r.ret);
    finish(c, ri, b, p + i, 1, k);
    cpl_ns += genesys_mono_ns() - e1;
    ++i;
  }
  const uint64_t t_cpl = genesys_mono_ns();
  uint64_t per_op[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (size_t i = 0; i < n; ++i) ++per_op[op_index(req[i].nr)];
  if (c->cfg.trace_capacity) {
    std::vector<genesys_trace_host> &tr = c->trace_host[ri];
    const uint32_t at = c->trace_n[ri].load(std::memory_order_relaxed);
    for (size_t i = 0; i < n; ++i)
      if (at + i < tr.size()) tr[at + i] = genesys_trace_host{req[i].slot, req[i].seq, t0, b.done_ns[i]};
    c->trace_n[ri].store(at + (uint32_t)n, std::memory_order_release);
  }
  for (int o = 0; o < 8; ++o)
    if (per_op[o]) bump(k.by_op[o], per_op[o]);
  bump(k.requests, n);
  bump(k.batches, 1);
  const uint64_t t_end = genesys_mono_ns();
  bump(k.complete_ns, cpl_ns + (t_end - t_cpl));
  k.last_batch_ns.store(t_end, std::memory_order_relaxed);
  bump(k.busy_ns, t_end - t0);
  return t_end;
}

// Ring entry `pos` if written: the first slot and the number of requests it
// announces (consecutive slots; see GENESYS_RING_ENTRY_RUN).
inline bool entry_ready(const uint64_t *ring, uint32_t mask, uint64_t pos, uint32_t *slot, uint32_t *count) {
  const uint64_t e = __atomic_load_n(&ring[pos & mask], __ATOMIC_ACQUIRE);
  if ((uint32_t)(e >> 32) != (uint32_t)(pos + 1)) return false;
  *slot = (uint32_t)e & ((1u << GENESYS_RING_SLOT_BITS) - 1u);
  *count = (((uint32_t)e >> GENESYS_RING_SLOT_BITS) & 0xFFu) + 1u;
  return true;
}

inline void read_request(genesys_ctx *c, uint32_t s, Request *r) {
#ifdef GENESYS_DEVICE_CHECKS
  if (s >= c->cfg.n_slots) {  // a doorbell entry naming no slot: count it and serve slot 0's request instead
    c->protocol_errors.fetch_add(1);
    s = 0;
  }
#endif
  const genesys_slot *sl = &c->slots[s];
  const uint64_t req = __atomic_load_n(&sl->req, __ATOMIC_ACQUIRE);
  r->slot = s;
  r->seq = (uint32_t)(req >> 32);
#ifdef GENESYS_DEVICE_CHECKS
  // a slot's requests are numbered 1, 2, 3, ... and each waits for the one
  // before it, so the service must see them in that order
  if (r->seq != c->last_seq[s] + 1u) c->protocol_errors.fetch_add(1);
  c->last_seq[s] = r->seq;
#endif
  r->nr = (uint32_t)(req >> 16) & 0xFFFFu;
  r->flags = (uint32_t)req & 0xFFFFu;
  for (int i = 0; i < 6; ++i) r->a[i] = __atomic_load_n(&sl->args[i], __ATOMIC_RELAXED);
  r->ret = 0;
}

// Take ready entries from ring `ri` until the batch holds coalesce_max
// requests (an entry's requests are taken whole, so a batch may hold up to
// GENESYS_RING_MAX_RUN - 1 more) and process them as one batch (Sec. 4.2).
// Returns the number of requests processed.
size_t poll_ring(genesys_ctx *c, uint32_t ri, Batch &b) {
  const uint64_t *ring = c->rings + (size_t)ri * c->ring_cap;
  const uint32_t mask = c->ring_cap - 1;
  const uint64_t h = c->head[ri];
  std::vector<Request> &batch = b.req;
  const size_t target = b.target;
  size_t n = 0, e = 0;  // requests, entries
  uint32_t s, cnt;
  // take the ready entries first and prefetch their slots (written by the GPU,
  // so their lines are not in the CPU's caches), then read the slots
  uint32_t *slots = b.slot_ids.data();
  uint32_t *ent = b.entry_of.data();
  while (n < target && entry_ready(ring, mask, h + e, &s, &cnt)) {
    for (uint32_t q = 0; q < cnt; ++q) {
      slots[n + q] = s + q;
      ent[n + q] = (uint32_t)e;
      __builtin_prefetch(&c->slots[s + q], 0, 0);
    }
    b.left[e] = cnt;
    n += cnt;
    ++e;
  }
  Counters &k = c->counters[ri];
  if (n == 0) {
    bump(k.empty_polls, 1);
    uint32_t t, tc;
    for (uint32_t ahead : {1u, 8u, 32u, 64u})
      if (entry_ready(ring, mask, h + ahead, &t, &tc)) {
        bump(k.hole_polls, 1);
        break;
      }
    return 0;
  }
  const uint64_t t_pick = genesys_mono_ns();
  for (size_t i = 0; i < n; ++i) {
    read_request(c, slots[i], &batch[i]);
    batch[i].entry = ent[i];
  }
  if (n < target && c->cfg.coalesce_window_ns) {
    const uint64_t until = genesys_mono_ns() + c->cfg.coalesce_window_ns;
    while (n < target && genesys_mono_ns() < until) {
      if (entry_ready(ring, mask, h + e, &s, &cnt)) {
        for (uint32_t q = 0; q < cnt; ++q) {
          read_request(c, s + q, &batch[n + q]);
          batch[n + q].entry = (uint32_t)e;
        }
        b.left[e] = cnt;
        n += cnt;
        ++e;
      } else {
        cpu_relax();
      }
    }
  }
  b.head = h;
  b.n_entries = (uint32_t)e;
  b.prefix = 0;
  bump(k.pickup_ns, genesys_mono_ns() - t_pick);
  const uint64_t t_done = process_batch(c, ri, b, n, k);
  c->head[ri] = h + e;
  c->retired[ri].store(h + e, std::memory_order_release);
  for (uint32_t q = 0; q < GENESYS_RING_DONE_COPIES; ++q)
    __atomic_store_n(&c->ring_done[((size_t)ri * GENESYS_RING_DONE_COPIES + q) * 8], h + e, __ATOMIC_RELEASE);
  bump(k.complete_ns, genesys_mono_ns() - t_done);
  return n;
}

void service_main(genesys_ctx *c, uint32_t ri) {
  if (c->cfg.service_cpus) {
    cpu_set_t set;
    CPU_ZERO(&set);
    CPU_SET(c->cfg.service_cpus[ri], &set);
    pthread_setaffinity_np(pthread_self(), sizeof set, &set);
  }
  if (!c->host_only) cudaSetDevice(c->device);
  Batch batch(std::max<uint32_t>(1, c->cfg.coalesce_max));
  uint64_t last_work = genesys_mono_ns();
  uint32_t idle_polls = 0;
  while (!c->stop.load(std::memory_order_relaxed) && !c->ring_stop[ri].load(std::memory_order_relaxed)) {
    if (poll_ring(c, ri, batch)) {
      last_work = 0;
      idle_polls = 0;
      continue;
    }
    if (++idle_polls < 64) { cpu_relax(); continue; }
    idle_polls = 0;
    const uint64_t now = genesys_mono_ns();
    if (last_work == 0) last_work = now;
    if (now - last_work < c->cfg.idle_spin_ns) {
      cpu_relax();
    } else {
      timespec ts{0, 20000};  // nap 20 us while idle
      nanosleep(&ts, nullptr);
    }
  }
}

template <class T>
int dev_alloc(genesys_ctx *c, T **p, size_t count) {
  const size_t bytes = std::max<size_t>(count * sizeof(T), 256);
  if (c->host_only) {
    *p = (T *)aligned_alloc(256, (bytes + 255) & ~size_t(255));
    if (!*p) return fail(GENESYS_ENOMEM, "host allocation of %zu bytes failed", bytes);
    memset(*p, 0, bytes);
    return 0;
  }
  CUDA_TRY(cudaMalloc((void **)p, bytes));
  CUDA_TRY(cudaMemset(*p, 0, bytes));
  return 0;
}

template <class T>
int host_alloc(genesys_ctx *c, T **p, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  if (c->host_only) {
    *p = (T *)aligned_alloc(4096, (bytes + 4095) & ~size_t(4095));
    if (!*p) return fail(GENESYS_ENOMEM, "host allocation of %zu bytes failed", bytes);
    memset(*p, 0, bytes);
    return 0;
  }
  CUDA_TRY(cudaHostAlloc((void **)p, bytes, cudaHostAllocMapped | cudaHostAllocPortable));
  memset(*p, 0, bytes);
  return 0;
}

template <class T>
void dev_free(genesys_ctx *c, T *p) {
  if (!p) return;
  if (c->host_only) free(p); else cudaFree(p);
}
template <class T>
void host_free(genesys_ctx *c, T *p) {
  if (!p) return;
  if (c->host_only) free(p); else cudaFreeHost(p);
}

void free_all(genesys_ctx *c) {
  host_free(c, c->slots);
  host_free(c, c->done);
  host_free(c, c->rings);
  host_free(c, c->ring_done);
  host_free(c, c->staging);
  host_free(c, c->tails_host);
  host_free(c, c->status_host);
  dev_free(c, c->owner);
  dev_free(c, c->seq);
  dev_free(c, c->known_done);
  dev_free(c, c->ring_tail);
  dev_free(c, c->ksite);
  dev_free(c, c->grid_bar);
  dev_free(c, c->status);
  dev_free(c, c->lat);
  dev_free(c, c->lat_count);
  dev_free(c, c->trace);
  dev_free(c, c->trace_count);
  if (c->scratch && !c->host_only) cudaFree(c->scratch);
  for (auto &kv : c->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  c->graphs.clear();
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->ev_start) cudaEventDestroy(c->ev_start);
  if (c->ev_end) cudaEventDestroy(c->ev_end);
  reclaim(c, true);
}

// Ring positions published so far, per ring.  Device memory: read after the
// kernels have finished.
int read_tails(genesys_ctx *c, std::vector<uint32_t> &tails) {
  const uint32_t n = c->cfg.n_service_threads;
  if (c->host_only) {
    for (uint32_t r = 0; r < n; ++r) tails[r] = __atomic_load_n(&c->ring_tail[r * 32], __ATOMIC_ACQUIRE);
    return 0;
  }
  std::lock_guard<std::mutex> g(c->small_mu);
  CUDA_TRY(cudaMemcpyAsync(c->tails_host, c->ring_tail, (size_t)n * 32 * 4, cudaMemcpyDeviceToHost, c->aux));
  CUDA_TRY(cudaStreamSynchronize(c->aux));
  for (uint32_t r = 0; r < n; ++r) tails[r] = c->tails_host[(size_t)r * 32];
  return 0;
}

// GENESYS_LAUNCH_GRAPH: the first launch of a (kernel, grid, block, shared
// memory, cooperative) shape builds and instantiates a graph holding that one
// kernel node; later launches of the shape set the node's arguments on the
// instantiated graph and launch it, without rebuilding it.  Launches already
// queued keep the arguments they were given.
int launch_graph(genesys_ctx *c, const void *kernel, const uint32_t grid[3], const uint32_t block[3], size_t smem,
                 void **args, bool coop, cudaStream_t s) {
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void *>(kernel);
  kp.gridDim = dim3(grid[0], grid[1], grid[2]);
  kp.blockDim = dim3(block[0], block[1], block[2]);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  genesys_ctx::GraphKey key{kernel, {grid[0], grid[1], grid[2]}, {block[0], block[1], block[2]}, smem, coop};
  std::lock_guard<std::mutex> lock(c->graph_mu);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    genesys_ctx::GraphExec ge;
    cudaError_t e = cudaGraphCreate(&ge.graph, 0);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&ge.node, ge.graph, nullptr, 0, &kp);
    if (e == cudaSuccess && coop) {
      cudaKernelNodeAttrValue v{};
      v.cooperative = 1;
      e = cudaGraphKernelNodeSetAttribute(ge.node, cudaKernelNodeAttributeCooperative, &v);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge.exec, ge.graph, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (ge.exec) cudaGraphExecDestroy(ge.exec);
      if (ge.graph) cudaGraphDestroy(ge.graph);
      return fail(GENESYS_ECUDA, "graph launch set-up: %s", cudaGetErrorString(e));
    }
    it = c->graphs.emplace(key, ge).first;
  } else {
    CUDA_TRY(cudaGraphExecKernelNodeSetParams(it->second.exec, it->second.node, &kp));
  }
  CUDA_TRY(cudaGraphLaunch(it->second.exec, s));
  c->graph_launches.fetch_add(1, std::memory_order_relaxed);
  return 0;
}

}  // namespace

// ===================================================================== C ABI

extern "C" {

const char *genesys_last_error(void) { return g_last_error.c_str(); }

int genesys_internal_error(int code, const char *msg) { return fail(code, "%s", msg); }

int genesys_internal_device(genesys_ctx *c) { return c ? c->device : -1; }

void genesys_internal_servers(genesys_ctx *c, int delta) {
  if (c) c->servers.fetch_add(delta);
}

uint64_t genesys_internal_staging_mark(genesys_ctx *c) { return c ? c->staging_used.load() : 0; }

void genesys_internal_staging_release(genesys_ctx *c, uint64_t mark) {
  if (c) c->staging_used.store(mark);
}

int genesys_internal_scratch(genesys_ctx *c, size_t bytes, void **out) {
  if (!c || !out) return fail(GENESYS_EINVAL, "NULL argument");
  if (c->host_only) return fail(GENESYS_EINVAL, "host-only context has no device scratch");
  if (bytes > c->scratch_bytes) {
    if (c->scratch) {
      CUDA_TRY(cudaDeviceSynchronize());
      CUDA_TRY(cudaFree(c->scratch));
      c->scratch = nullptr;
      c->scratch_bytes = 0;
    }
    const size_t grow = std::max<size_t>(bytes, 1u << 20);
    CUDA_TRY(cudaMalloc(&c->scratch, grow));
    c->scratch_bytes = grow;
  }
  *out = c->scratch;
  return 0;
}

int genesys_config_default(genesys_config *cfg) {
  if (!cfg) return fail(GENESYS_EINVAL, "cfg is NULL");
  memset(cfg, 0, sizeof *cfg);
  cfg->n_slots = 0;
  cfg->n_service_threads = 4;
  cfg->staging_bytes = 256ull << 20;
  cfg->coalesce_window_ns = 0;
  cfg->coalesce_max = 64;
  cfg->merge = 1;
  cfg->device_deadline_ns = 2000000000ull;
  cfg->lat_samples = 1u << 20;
  cfg->idle_spin_ns = 200000000ull;
  cfg->poll_min_ns = 256;
  cfg->poll_max_ns = 2048;
  return 0;
}

int genesys_init(const genesys_config *cfg_in, int device, genesys_ctx **out) {
  return genesys_guard("genesys_init", [&]() -> int {
    if (!out) return fail(GENESYS_EINVAL, "out is NULL");
    *out = nullptr;
    genesys_config cfg;
    if (cfg_in) cfg = *cfg_in; else genesys_config_default(&cfg);
    if (cfg.n_service_threads == 0 || cfg.n_service_threads > 256)
      return fail(GENESYS_EINVAL, "n_service_threads must be 1..256");
    if (cfg.coalesce_max == 0) cfg.coalesce_max = 1;
    if (cfg.device_deadline_ns == 0) return fail(GENESYS_EINVAL, "device_deadline_ns must be > 0");
    if (cfg.poll_min_ns == 0) cfg.poll_min_ns = 256;
    if (cfg.poll_max_ns < cfg.poll_min_ns) cfg.poll_max_ns = cfg.poll_min_ns;
    if (cfg.poll_max_ns > 1000000) return fail(GENESYS_EINVAL, "poll_max_ns above 1 ms");

    auto c = std::make_unique<genesys_ctx>();
    // whatever was set up is given back on every failure path (an early
    // return or an exception) until the context is handed out
    struct FreeOnFail {
      genesys_ctx *c;
      bool armed = true;
      ~FreeOnFail() { if (armed) free_all(c); }
    } free_on_fail{c.get()};
    c->host_only = (cfg.flags & GENESYS_INIT_HOST_ONLY) != 0;
    c->device = device;
    if (!c->host_only) {
      int ndev = 0;
      if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(GENESYS_ENODEV, "no CUDA device");
      }
      if (device < 0 || device >= ndev) return fail(GENESYS_EINVAL, "device %d out of range", device);
      CUDA_TRY(cudaSetDevice(device));
      int sms = 0, mapped = 0;
      CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
      CUDA_TRY(cudaDeviceGetAttribute(&mapped, cudaDevAttrCanMapHostMemory, device));
      if (!mapped) return fail(GENESYS_ENODEV, "device cannot map host memory");
      c->n_sms = (uint32_t)sms;
      CUDA_TRY(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
      CUDA_TRY(cudaEventCreate(&c->ev_start));
      CUDA_TRY(cudaEventCreate(&c->ev_end));
    } else {
      c->n_sms = 0;
    }
    if (cfg.n_slots == 0) cfg.n_slots = c->host_only ? 65536u : c->n_sms * 2048u;
    if (cfg.n_slots < 32) cfg.n_slots = 32;
    if (cfg.n_slots > (1u << GENESYS_RING_SLOT_BITS))
      return fail(GENESYS_EINVAL, "n_slots above 2^24 (doorbell entries name slots in 24 bits)");
    c->cfg = cfg;

    // doorbell rings: a slot has at most one request outstanding, announced by
    // one entry in one ring (any ring: positional file calls go by file
    // region), so a ring with an entry for every slot can never overflow
    c->ring_cap = (uint32_t)next_pow2(std::max<uint64_t>(cfg.n_slots, 64));

    int rc;
    if ((rc = host_alloc(c.get(), &c->slots, (size_t)cfg.n_slots * sizeof(genesys_slot)))) return rc;
    if ((rc = host_alloc(c.get(), &c->done, (size_t)cfg.n_slots * 8))) return rc;
    if ((rc = host_alloc(c.get(), &c->rings, (size_t)cfg.n_service_threads * c->ring_cap * 8))) return rc;
    if ((rc = host_alloc(c.get(), &c->ring_done, (size_t)cfg.n_service_threads * GENESYS_RING_DONE_COPIES * 64)))
      return rc;
    if (cfg.staging_bytes && (rc = host_alloc(c.get(), &c->staging, cfg.staging_bytes))) return rc;
    if ((rc = dev_alloc(c.get(), &c->owner, cfg.n_slots))) return rc;
    if ((rc = dev_alloc(c.get(), &c->seq, cfg.n_slots))) return rc;
    if ((rc = dev_alloc(c.get(), &c->known_done, cfg.n_slots))) return rc;
    if ((rc = dev_alloc(c.get(), &c->ring_tail, (size_t)cfg.n_service_threads * 32))) return rc;
    if ((rc = dev_alloc(c.get(), &c->ksite, GENESYS_KSITES))) return rc;
    if ((rc = dev_alloc(c.get(), &c->grid_bar, 64))) return rc;
    if ((rc = dev_alloc(c.get(), &c->status, GENESYS_ST_WORDS))) return rc;
    if (!c->host_only) {
      if ((rc = host_alloc(c.get(), &c->tails_host, (size_t)cfg.n_service_threads * 32 * 4))) return rc;
      if ((rc = host_alloc(c.get(), &c->status_host, GENESYS_ST_WORDS * 4))) return rc;
    }
    if ((rc = dev_alloc(c.get(), &c->lat, std::max<uint32_t>(cfg.lat_samples, 1)))) return rc;
    if ((rc = dev_alloc(c.get(), &c->lat_count, 1))) return rc;
    if (cfg.trace_capacity) {
      if ((rc = dev_alloc(c.get(), &c->trace, cfg.trace_capacity))) return rc;
      if ((rc = dev_alloc(c.get(), &c->trace_count, 1))) return rc;
    }

    const uint32_t nr = cfg.n_service_threads;
    c->head.assign(nr, 0);
    c->retired.reset(new std::atomic<uint64_t>[nr]);
    for (uint32_t r = 0; r < nr; ++r) c->retired[r].store(0);
    c->counters.reset(new Counters[nr]);
    c->ring_stop.reset(new std::atomic<bool>[nr]);
    for (uint32_t r = 0; r < nr; ++r) c->ring_stop[r].store(false);
  #ifdef GENESYS_DEVICE_CHECKS
    c->last_seq.assign(cfg.n_slots, 0);
  #endif
    c->created_ns = genesys_mono_ns();
    c->trace_n.reset(new std::atomic<uint32_t>[nr]);
    for (uint32_t r = 0; r < nr; ++r) c->trace_n[r].store(0);
    if (cfg.trace_capacity) c->trace_host.assign(nr, std::vector<genesys_trace_host>((cfg.trace_capacity + nr - 1) / nr));
    if (!(cfg.flags & GENESYS_INIT_NO_THREADS)) {
      try {
        for (uint32_t r = 0; r < nr; ++r) c->threads.emplace_back(service_main, c.get(), r);
      } catch (...) {  // a thread could not start: stop the ones that did
        c->stop.store(true);
        for (auto &t : c->threads) t.join();
        c->threads.clear();
        throw;
      }
    }
    free_on_fail.armed = false;
    *out = c.release();
    return 0;
  });
}

// How long genesys_drain spins before it sleeps between looks.
constexpr uint64_t kDrainSpinNs = 50000;

int genesys_drain(genesys_ctx *c, uint64_t timeout_ns) {
  return genesys_guard("genesys_drain", [&]() -> int {
    if (!c) return fail(GENESYS_EINVAL, "ctx is NULL");
    std::vector<uint32_t> tails(c->cfg.n_service_threads);
    int rc = read_tails(c, tails);
    if (rc) return rc;
    std::unique_ptr<Batch> batch;  // NO_THREADS mode: the caller services the rings
    const uint64_t start = genesys_mono_ns(), until = start + timeout_ns;
    // After a blocking launch its last requests retire within microseconds of
    // its end: spin briefly before sleeping, since a sleep costs tens of
    // microseconds of timer slack (once per launch when a step runs many).  The
    // spin stays short so that a long drain (non-blocking calls still being
    // served) does not take a core from the service threads.
    const uint64_t spin_until = start + kDrainSpinNs;
    for (uint32_t r = 0; r < c->cfg.n_service_threads; ++r) {
      for (;;) {
        // positions are 32-bit on the device: compare modulo 2^32
        const uint32_t got = (uint32_t)c->retired[r].load(std::memory_order_acquire);
        if ((int32_t)(got - tails[r]) >= 0) break;
        if (c->cfg.flags & GENESYS_INIT_NO_THREADS) {
          std::lock_guard<std::mutex> g(c->svc_mu);
          if (!batch) batch.reset(new Batch(std::max<uint32_t>(1, c->cfg.coalesce_max)));
          poll_ring(c, r, *batch);
        } else if (genesys_mono_ns() < spin_until) {
          for (int i = 0; i < 32; ++i) cpu_relax();
        } else {
          std::this_thread::sleep_for(std::chrono::microseconds(5));
        }
        if (genesys_mono_ns() > until)
          return fail(GENESYS_ETIMEDOUT, "drain: ring %u retired %u of %u requests", r, got, tails[r]);
      }
    }
    return 0;
  });
}

// CPU time a running service thread has used so far (0 if unavailable).
static uint64_t thread_cpu_ns(std::thread &t) {
  clockid_t cid;
  timespec ts;
  if (!t.joinable() || pthread_getcpuclockid(t.native_handle(), &cid) != 0 || clock_gettime(cid, &ts) != 0) return 0;
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

static uint64_t service_cpu_total(genesys_ctx *c) {
  uint64_t t = c->cpu_retired_ns.load();
  for (auto &th : c->threads) t += thread_cpu_ns(th);
  return t;
}

uint32_t genesys_sizeof(int which) {
  switch (which) {
    case GENESYS_SIZEOF_CONFIG: return sizeof(genesys_config);
    case GENESYS_SIZEOF_STATS: return sizeof(genesys_stats_t);
    case GENESYS_SIZEOF_SERVE_CONFIG: return sizeof(genesys_serve_config);
    case GENESYS_SIZEOF_SERVE_STATS: return sizeof(genesys_serve_stats);
    case GENESYS_SIZEOF_TRACE_DEV: return sizeof(genesys_trace_dev);
    case GENESYS_SIZEOF_TRACE_HOST: return sizeof(genesys_trace_host);
    case GENESYS_SIZEOF_C5_REQUEST: return sizeof(genesys_c5_request);
    case GENESYS_SIZEOF_DEV: return sizeof(genesys_dev);
    default: return 0;
  }
}

int genesys_service_health(genesys_ctx *c, uint64_t stall_ns, uint64_t *stalled_mask, uint64_t *pending) {
  return genesys_guard("genesys_service_health", [&]() -> int {
    if (!c || !stalled_mask) return fail(GENESYS_EINVAL, "NULL argument");
    std::vector<uint32_t> tails(c->cfg.n_service_threads);
    int rc = read_tails(c, tails);
    if (rc) return rc;
    const uint64_t now = genesys_mono_ns();
    uint64_t mask = 0, total = 0;
    for (uint32_t r = 0; r < c->cfg.n_service_threads; ++r) {
      // positions are 32-bit on the device: the distance modulo 2^32; the
      // service may have passed the tails read above (requests published and
      // finished since), which counts as nothing waiting
      const int32_t d = (int32_t)(tails[r] - (uint32_t)c->retired[r].load(std::memory_order_acquire));
      const uint32_t waiting = d > 0 ? (uint32_t)d : 0u;
      total += waiting;
      const uint64_t last = c->counters[r].last_batch_ns.load(std::memory_order_relaxed);
      if (waiting && now - std::max(last, c->created_ns) > stall_ns && r < 64) mask |= 1ull << r;
    }
    *stalled_mask = mask;
    if (pending) *pending = total;
    return 0;
  });
}

int genesys_service_restart(genesys_ctx *c, uint32_t ring, uint64_t pause_ns) {
  return genesys_guard("genesys_service_restart", [&]() -> int {
    if (!c) return fail(GENESYS_EINVAL, "ctx is NULL");
    if (c->threads.empty()) return fail(GENESYS_EINVAL, "the context has no service threads");
    if (ring >= c->cfg.n_service_threads) return fail(GENESYS_EINVAL, "no ring %u", ring);
    std::lock_guard<std::mutex> g(c->restart_mu);
    // the thread finishes the batch it has and leaves; its ring position (head)
    // stays with the context, so the new thread continues where it stopped
    c->ring_stop[ring].store(true);
    const uint64_t used = thread_cpu_ns(c->threads[ring]);  // read before it leaves: its clock goes with it
    c->threads[ring].join();
    c->cpu_retired_ns.fetch_add(used);
    if (pause_ns) std::this_thread::sleep_for(std::chrono::nanoseconds(pause_ns));
    c->ring_stop[ring].store(false);
    c->threads[ring] = std::thread(service_main, c, ring);
    return 0;
  });
}

int genesys_shutdown(genesys_ctx *c) {
  if (!c) return 0;
  if (const int n = c->servers.load())
    return fail(GENESYS_EINVAL, "%d server kernel(s) still run on this context: stop them first", n);
  int rc = 0;
  // kernels still in flight use the slot area and may wait on calls: let them
  // finish (every device wait is bounded) while the service threads still run
  if (!c->host_only && cudaSetDevice(c->device) == cudaSuccess && cudaDeviceSynchronize() != cudaSuccess)
    rc = fail(GENESYS_ECUDA, "shutdown: %s", cudaGetErrorString(cudaGetLastError()));
  std::unique_lock<std::mutex> restarting(c->restart_mu);  // no thread is being replaced meanwhile
  if (!c->threads.empty()) {
    if (const int d = genesys_drain(c, 1000000000ull)) rc = rc ? rc : d;
    c->stop.store(true);
    for (auto &t : c->threads) t.join();
    c->threads.clear();
  }
  restarting.unlock();
  free_all(c);
  delete c;
  return rc;
}

int genesys_device_view(genesys_ctx *c, genesys_dev *d) {
  if (!c || !d) return fail(GENESYS_EINVAL, "NULL argument");
  memset(d, 0, sizeof *d);
  d->slots = c->slots;
  d->done = c->done;
  d->rings = c->rings;
  d->ring_done = c->ring_done;
  d->owner = c->owner;
  d->seq = c->seq;
  d->known_done = c->known_done;
  d->ring_tail = c->ring_tail;
  d->ksite = c->ksite;
  d->grid_bar = c->grid_bar;
  d->status = c->status;
  d->lat = c->lat;
  d->lat_count = c->lat_count;
  d->lat_cap = c->cfg.lat_samples;
  d->trace = c->trace;
  d->trace_count = c->trace_count;
  d->trace_cap = c->cfg.trace_capacity;
  d->n_slots = c->cfg.n_slots;
  d->n_rings = c->cfg.n_service_threads;
  d->ring_mask = c->ring_cap - 1;
  d->deadline_ns = c->cfg.device_deadline_ns;
  d->n_sms = c->n_sms;
  d->poll_min_ns = c->cfg.poll_min_ns;
  d->poll_max_ns = c->cfg.poll_max_ns;
  return 0;
}

int genesys_launch(genesys_ctx *c, const void *kernel, const uint32_t grid[3], const uint32_t block[3],
                   size_t smem, void **args, uint32_t flags, void *stream) {
  if (!c || !kernel || !grid || !block) return fail(GENESYS_EINVAL, "NULL argument");
  if (c->host_only) return fail(GENESYS_EINVAL, "host-only context cannot launch kernels");
  const uint32_t gran = flags & GENESYS_LAUNCH_GRAN_MASK;
  const bool relaxed = flags & GENESYS_LAUNCH_RELAXED;
  if (gran == GENESYS_GRAN_ITEM && relaxed)
    return fail(GENESYS_EINVAL, "work-item grain calls are always strongly ordered (Sec. 4.1)");
  bool coop = (flags & GENESYS_LAUNCH_COOPERATIVE) || (gran == GENESYS_GRAN_KERNEL && !relaxed);
  const dim3 g(grid[0], grid[1], grid[2]), b(block[0], block[1], block[2]);
  const uint64_t nblocks = (uint64_t)grid[0] * grid[1] * grid[2];
  const uint64_t nthreads = (uint64_t)block[0] * block[1] * block[2];
  if (nblocks == 0 || nthreads == 0) return fail(GENESYS_EINVAL, "empty grid or block");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaSetDevice(c->device));
  if (coop) {
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, (int)nthreads, smem));
    if (nblocks > (uint64_t)per_sm * c->n_sms)
      return fail(GENESYS_EINVAL,
                  "kernel-grain strong ordering needs every block resident: grid %llu > %d x %u (Sec. 4.1)",
                  (unsigned long long)nblocks, per_sm, c->n_sms);
  }
  // kernel-grain call sites start every launch reset, whatever grain the
  // flags declare (a kernel may mix grains)
  CUDA_TRY(cudaMemsetAsync(c->ksite, 0, GENESYS_KSITES * sizeof(genesys_ksite), s));
  CUDA_TRY(cudaEventRecord(c->ev_start, s));
  if (flags & GENESYS_LAUNCH_GRAPH) {
    int rc = launch_graph(c, kernel, grid, block, smem, args, coop, s);
    if (rc) return rc;
  } else if (coop) {
    CUDA_TRY(cudaLaunchCooperativeKernel(kernel, g, b, args, smem, s));
  } else {
    CUDA_TRY(cudaLaunchKernel(kernel, g, b, args, smem, s));
  }
  CUDA_TRY(cudaEventRecord(c->ev_end, s));
  if (flags & GENESYS_LAUNCH_SYNC) {
    CUDA_TRY(cudaStreamSynchronize(s));
    return genesys_drain(c, 10ull * c->cfg.device_deadline_ns);
  }
  return 0;
}

int genesys_last_launch_ms(genesys_ctx *c, float *ms) {
  if (!c || !ms) return fail(GENESYS_EINVAL, "NULL argument");
  if (c->host_only) return fail(GENESYS_EINVAL, "host-only context has no launches");
  CUDA_TRY(cudaEventSynchronize(c->ev_end));
  CUDA_TRY(cudaEventElapsedTime(ms, c->ev_start, c->ev_end));
  return 0;
}

int genesys_service(genesys_ctx *c, uint64_t timeout_ns) {
  return genesys_guard("genesys_service", [&]() -> int {
    if (!c) return fail(GENESYS_EINVAL, "ctx is NULL");
    const uint64_t until = genesys_mono_ns() + timeout_ns;
    if (c->cfg.flags & GENESYS_INIT_NO_THREADS) {
      std::lock_guard<std::mutex> g(c->svc_mu);
      Batch batch(std::max<uint32_t>(1, c->cfg.coalesce_max));
      int total = 0;
      do {
        size_t n = 0;
        for (uint32_t r = 0; r < c->cfg.n_service_threads; ++r) n += poll_ring(c, r, batch);
        total += (int)n;
        if (n == 0) cpu_relax();
      } while (genesys_mono_ns() < until);
      return total;
    }
    return genesys_drain(c, timeout_ns);
  });
}

int genesys_mmap_reserve(genesys_ctx *c, const uint64_t *sizes, uint32_t n) {
  return genesys_guard("genesys_mmap_reserve", [&]() -> int {
    if (!c || (!sizes && n)) return fail(GENESYS_EINVAL, "NULL argument");
    if (c->host_only) return fail(GENESYS_EINVAL, "host-only context");
    for (uint32_t i = 0; i < n; ++i) {
      const size_t len = (size_t)((sizes[i] + 4095) & ~uint64_t(4095));
      if (len == 0) continue;
      void *p = mmap(nullptr, len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
      if (p == MAP_FAILED) return fail(GENESYS_ENOMEM, "mmap of %zu bytes failed", len);
      if (cudaHostRegister(p, len, cudaHostRegisterMapped | cudaHostRegisterPortable) != cudaSuccess) {
        cudaGetLastError();
        munmap(p, len);
        return fail(GENESYS_ECUDA, "cudaHostRegister of %zu bytes failed", len);
      }
      void *d = nullptr;
      if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaHostUnregister(p);
        munmap(p, len);
        return fail(GENESYS_ECUDA, "cudaHostGetDevicePointer failed");
      }
      std::lock_guard<std::mutex> g(c->map_mu);
      c->released.emplace(len, std::make_pair((uintptr_t)d, genesys_ctx::Mapping{p, len, len}));
    }
    return 0;
  });
}

int genesys_reclaim(genesys_ctx *c) {
  if (!c) return fail(GENESYS_EINVAL, "ctx is NULL");
  reclaim(c, false);
  return 0;
}

int genesys_stats_get(genesys_ctx *c, genesys_stats_t *o) {
  return genesys_guard("genesys_stats_get", [&]() -> int {
    if (!c || !o) return fail(GENESYS_EINVAL, "NULL argument");
    memset(o, 0, sizeof *o);
    for (uint32_t r = 0; r < c->cfg.n_service_threads; ++r) {
      Counters &k = c->counters[r];
      o->requests += k.requests.load();
      o->os_calls += k.os_calls.load();
      o->failed += k.failed.load();
      o->nonblocking_failed += k.nb_failed.load();
      o->bytes += k.bytes.load();
      o->batches += k.batches.load();
      o->busy_ns += k.busy_ns.load();
      o->pickup_ns += k.pickup_ns.load();
      o->order_ns += k.order_ns.load();
      o->complete_ns += k.complete_ns.load();
      o->empty_polls += k.empty_polls.load();
      o->hole_polls += k.hole_polls.load();
      for (int i = 0; i < 8; ++i) {
        o->by_op[i] += k.by_op[i].load();
        o->op_ns[i] += k.op_ns[i].load();
        o->op_max_ns[i] = std::max<uint64_t>(o->op_max_ns[i], k.op_max_ns[i].load());
      }
    }
    o->mmap_new = c->mmap_new.load();
    o->mmap_reused = c->mmap_reused.load();
    {
      std::lock_guard<std::mutex> g(c->restart_mu);  // the thread list is stable
      const uint64_t cpu = service_cpu_total(c);
      o->service_cpu_ns = cpu > c->cpu_reset_ns ? cpu - c->cpu_reset_ns : 0;
    }
    o->protocol_errors = c->protocol_errors.load();
    return 0;
  });
}

int genesys_stats_reset(genesys_ctx *c) {
  if (!c) return fail(GENESYS_EINVAL, "ctx is NULL");
  for (uint32_t r = 0; r < c->cfg.n_service_threads; ++r) {
    Counters &k = c->counters[r];
    k.requests = 0; k.os_calls = 0; k.failed = 0; k.nb_failed = 0; k.bytes = 0; k.batches = 0; k.busy_ns = 0;
    k.pickup_ns = 0; k.order_ns = 0; k.complete_ns = 0; k.empty_polls = 0; k.hole_polls = 0;
    for (int i = 0; i < 8; ++i) k.by_op[i] = 0, k.op_ns[i] = 0, k.op_max_ns[i] = 0;
  }
  std::lock_guard<std::mutex> g(c->restart_mu);
  c->cpu_reset_ns = service_cpu_total(c);
  return 0;
}

int genesys_stats(genesys_ctx *c, genesys_stats_t *out) { return genesys_stats_get(c, out); }

int genesys_graph_launches(genesys_ctx *c, uint64_t *out) {
  if (!c || !out) return fail(GENESYS_EINVAL, "NULL argument");
  *out = c->graph_launches.load();
  return 0;
}

int genesys_check_pread_cap(genesys_ctx *c, uint64_t cap_bytes) {
  if (!c) return fail(GENESYS_EINVAL, "ctx is NULL");
#ifdef GENESYS_DEVICE_CHECKS
  c->pread_cap = cap_bytes;
  return 0;
#else
  (void)cap_bytes;
  return fail(GENESYS_EINVAL, "genesys_check_pread_cap: only the checked build (GENESYS_DEVICE_CHECKS) caps preads");
#endif
}

int genesys_trace_read(genesys_ctx *c, genesys_trace_dev *dev, uint32_t dev_cap, uint32_t *n_dev,
                       genesys_trace_host *host, uint32_t host_cap, uint32_t *n_host, int64_t *host_minus_device_ns) {
  return genesys_guard("genesys_trace_read", [&]() -> int {
    if (!c || (dev_cap && !dev) || (host_cap && !host)) return fail(GENESYS_EINVAL, "NULL argument");
    if (!c->cfg.trace_capacity) return fail(GENESYS_EINVAL, "the context keeps no trace (trace_capacity 0)");
    uint32_t nd = 0;
    if (!c->host_only) {
      CUDA_TRY(cudaMemcpy(&nd, c->trace_count, 4, cudaMemcpyDeviceToHost));
      const uint32_t k = std::min({nd, c->cfg.trace_capacity, dev_cap});
      if (k) CUDA_TRY(cudaMemcpy(dev, c->trace, (size_t)k * sizeof(genesys_trace_dev), cudaMemcpyDeviceToHost));
      CUDA_TRY(cudaMemset(c->trace_count, 0, 4));
    }
    if (n_dev) *n_dev = nd;
    uint32_t nh = 0, out = 0;
    for (uint32_t r = 0; r < c->cfg.n_service_threads; ++r) {
      const uint32_t n = c->trace_n[r].load(std::memory_order_acquire);
      const uint32_t have = std::min<uint32_t>(n, (uint32_t)c->trace_host[r].size());
      for (uint32_t i = 0; i < have && out < host_cap; ++i) host[out++] = c->trace_host[r][i];
      nh += n;
      c->trace_n[r].store(0, std::memory_order_release);
    }
    if (n_host) *n_host = nh;
    if (host_minus_device_ns) {
      if (c->host_only) {
        *host_minus_device_ns = 0;
      } else {
        int rc = genesys_internal_clock_offset(c->device, 200, 2000000000ull, host_minus_device_ns, nullptr);
        if (rc) return rc;
      }
    }
    return 0;
  });
}

int genesys_status(genesys_ctx *c, int32_t out[GENESYS_ST_WORDS], int clear) {
  if (!c || !out) return fail(GENESYS_EINVAL, "NULL argument");
  if (c->host_only) {
    memcpy(out, c->status, GENESYS_ST_WORDS * 4);
    if (clear) memset(c->status, 0, GENESYS_ST_WORDS * 4);
    return 0;
  }
  std::lock_guard<std::mutex> g(c->small_mu);
  CUDA_TRY(cudaMemcpyAsync(c->status_host, c->status, GENESYS_ST_WORDS * 4, cudaMemcpyDeviceToHost, c->aux));
  if (clear) CUDA_TRY(cudaMemsetAsync(c->status, 0, GENESYS_ST_WORDS * 4, c->aux));
  CUDA_TRY(cudaStreamSynchronize(c->aux));
  memcpy(out, c->status_host, GENESYS_ST_WORDS * 4);
  return 0;
}

int genesys_latency(genesys_ctx *c, uint64_t *out, uint32_t cap, uint32_t *n_out, int clear) {
  return genesys_guard("genesys_latency", [&]() -> int {
    if (!c || !n_out) return fail(GENESYS_EINVAL, "NULL argument");
    uint32_t n = 0;
    if (c->host_only) {
      n = *c->lat_count;
    } else {
      CUDA_TRY(cudaMemcpyAsync(&n, c->lat_count, 4, cudaMemcpyDeviceToHost, c->aux));
      CUDA_TRY(cudaStreamSynchronize(c->aux));
    }
    *n_out = n;
    const uint32_t m = std::min(std::min(n, cap), c->cfg.lat_samples);
    if (out && m) {
      if (c->host_only) memcpy(out, c->lat, (size_t)m * 8);
      else CUDA_TRY(cudaMemcpyAsync(out, c->lat, (size_t)m * 8, cudaMemcpyDeviceToHost, c->aux));
    }
    if (clear) {
      if (c->host_only) *c->lat_count = 0;
      else CUDA_TRY(cudaMemsetAsync(c->lat_count, 0, 4, c->aux));
    }
    if (!c->host_only) CUDA_TRY(cudaStreamSynchronize(c->aux));
    return 0;
  });
}

void *genesys_staging(genesys_ctx *c, size_t bytes) {
  if (!c || !c->staging) { fail(GENESYS_EINVAL, "no staging arena"); return nullptr; }
  const uint64_t need = (bytes + 255) & ~uint64_t(255);
  uint64_t cur = c->staging_used.load();
  do {
    if (cur + need > c->cfg.staging_bytes) {
      fail(GENESYS_ENOMEM, "staging arena exhausted (%llu + %llu > %llu)", (unsigned long long)cur,
           (unsigned long long)need, (unsigned long long)c->cfg.staging_bytes);
      return nullptr;
    }
  } while (!c->staging_used.compare_exchange_weak(cur, cur + need));
  return c->staging + cur;
}

int genesys_staging_reset(genesys_ctx *c) {
  if (!c) return fail(GENESYS_EINVAL, "ctx is NULL");
  c->staging_used.store(0);
  return 0;
}

// Host emulation of one GPU lane making a call (GENESYS_INIT_HOST_ONLY): the
// same claim / marshal / publish / doorbell / wait steps as genesys_device.cuh,
// with CPU atomics on the host copies of the device-side state.
// Host-side ceiling of the service path for work-item pwrites: the requests
// a GPU work-item launch would publish (one slot each), published by this
// thread instead, so that the time is the service threads' alone.  Slots are
// filled first; the clock runs from the first doorbell entry to the last
// completion word.  The context's device-side claim state (sequence numbers,
// ring tails) is read before and written back after, so the context stays
// usable by kernels.  No kernel may be running on the context meanwhile.
int genesys_service_probe(genesys_ctx *c, int fd, const void *payload, uint32_t bytes_per_call, uint64_t n_calls,
                          uint64_t *elapsed_ns) {
  return genesys_service_probe_order(c, fd, payload, bytes_per_call, n_calls, 1, 1, elapsed_ns);
}

int genesys_service_probe_order(genesys_ctx *c, int fd, const void *payload, uint32_t bytes_per_call,
                                uint64_t n_calls, uint32_t run, uint32_t stride, uint64_t *elapsed_ns) {
  return genesys_guard("genesys_service_probe", [&]() -> int {
    if (!c || !payload || !elapsed_ns || bytes_per_call == 0) return fail(GENESYS_EINVAL, "NULL argument");
    if (run == 0 || stride == 0) return fail(GENESYS_EINVAL, "service probe: run and stride must be >= 1");
    if (c->threads.empty()) return fail(GENESYS_EINVAL, "genesys_service_probe needs service threads");
    const uint32_t S = c->cfg.n_slots, R = c->cfg.n_service_threads;
    std::vector<uint32_t> seq(S), kd(S), owner(S), tails_raw((size_t)R * 32);
    auto copy = [&](void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) -> int {
      if (c->host_only) { memcpy(dst, src, bytes); return 0; }
      CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, kind, c->aux));
      CUDA_TRY(cudaStreamSynchronize(c->aux));
      return 0;
    };
    int rc;
    if ((rc = copy(seq.data(), c->seq, 4ull * S, cudaMemcpyDeviceToHost)) ||
        (rc = copy(kd.data(), c->known_done, 4ull * S, cudaMemcpyDeviceToHost)) ||
        (rc = copy(owner.data(), c->owner, 4ull * S, cudaMemcpyDeviceToHost)) ||
        (rc = copy(tails_raw.data(), c->ring_tail, tails_raw.size() * 4, cudaMemcpyDeviceToHost)))
      return rc;
    for (uint32_t s = 0; s < S; ++s) {
      if (owner[s] != 0) return fail(GENESYS_EINVAL, "service probe: slot %u is claimed (a kernel is running?)", s);
      if ((uint32_t)(__atomic_load_n(&c->done[s], __ATOMIC_ACQUIRE) >> 32) != seq[s])
        return fail(GENESYS_EINVAL, "service probe: slot %u has a request in flight", s);
    }
    const uint64_t deadline = c->cfg.device_deadline_ns;
    const uint16_t flags = GENESYS_REQ_BLOCKING | (GENESYS_GRAN_ITEM << GENESYS_REQ_GRAN_SHIFT);
    const uint8_t *base = (const uint8_t *)payload;
    uint64_t total = 0, bad = 0;
    for (uint64_t i0 = 0; i0 < n_calls;) {
      const uint32_t m = (uint32_t)std::min<uint64_t>(S, n_calls - i0);
      for (uint32_t s = 0; s < m; ++s) {
        const uint64_t i = i0 + s;
        genesys_slot *sl = &c->slots[s];
        const uint64_t a[6] = {(uint64_t)fd, (uint64_t)(uintptr_t)(base + i * bytes_per_call), bytes_per_call,
                               i * bytes_per_call, 0, 0};
        for (int k = 0; k < 6; ++k) __atomic_store_n(&sl->args[k], a[k], __ATOMIC_RELAXED);
        ++seq[s];
        __atomic_store_n(&sl->req, ((uint64_t)seq[s] << 32) | ((uint64_t)(SYS_pwrite64 & 0xFFFF) << 16) | flags,
                         __ATOMIC_RELEASE);
      }
      const uint64_t t0 = genesys_mono_ns();
      // doorbells: runs of `run` consecutive slots; run k is rung in pass
      // k % stride, so neighbouring runs are a 1/stride of the round apart.
      // As a GPU warp does, 32 consecutive slots starting at a multiple of 32
      // (always one ring) are announced by one entry, other slots one by one.
      const uint32_t n_runs = (m + run - 1) / run;
      auto ring_at = [&](uint32_t s) {
        return genesys_ring_of_file((uint64_t)(int64_t)fd, (i0 + s) * (uint64_t)bytes_per_call, R, 0);
      };
      auto ring_entry = [&](uint32_t s, uint32_t count) {
        const uint32_t r = ring_at(s);  // the ring a GPU pwrite of this request rings: by file region
        const uint32_t pos = tails_raw[(size_t)r * 32]++;
        __atomic_store_n(&c->rings[(size_t)r * c->ring_cap + (pos & (c->ring_cap - 1))],
                         GENESYS_RING_ENTRY_RUN(pos, s, count), __ATOMIC_RELEASE);
      };
      for (uint32_t pass = 0; pass < stride; ++pass)
        for (uint32_t k = pass; k < n_runs; k += stride) {
          const uint32_t end = std::min(m, (k + 1) * run);
          for (uint32_t s = k * run; s < end;) {
            if (s % GENESYS_RING_MAX_RUN == 0 && s + GENESYS_RING_MAX_RUN <= end &&
                ring_at(s) == ring_at(s + GENESYS_RING_MAX_RUN - 1)) {
              ring_entry(s, GENESYS_RING_MAX_RUN);
              s += GENESYS_RING_MAX_RUN;
            } else {
              ring_entry(s, 1);
              ++s;
            }
          }
        }
      for (uint32_t s = 0; s < m; ++s) {
        uint64_t d;
        while ((uint32_t)((d = __atomic_load_n(&c->done[s], __ATOMIC_ACQUIRE)) >> 32) != seq[s]) {
          if (genesys_mono_ns() - t0 > deadline) {
            rc = fail(GENESYS_ETIMEDOUT, "service probe: slot %u not completed within the deadline", s);
            break;
          }
          cpu_relax();
        }
        if (rc) break;
        if ((int32_t)(uint32_t)d != (int32_t)bytes_per_call) ++bad;
        kd[s] = seq[s];
      }
      total += genesys_mono_ns() - t0;
      if (rc) break;
      i0 += m;
    }
    // the device-side state the kernels continue from
    if (c->host_only) {
      memcpy(c->seq, seq.data(), 4ull * S);
      memcpy(c->known_done, kd.data(), 4ull * S);
      for (uint32_t r = 0; r < R; ++r) __atomic_store_n(&c->ring_tail[r * 32], tails_raw[(size_t)r * 32], __ATOMIC_RELEASE);
    } else {
      int wrc;
      if ((wrc = copy(c->seq, seq.data(), 4ull * S, cudaMemcpyHostToDevice)) ||
          (wrc = copy(c->known_done, kd.data(), 4ull * S, cudaMemcpyHostToDevice)) ||
          (wrc = copy(c->ring_tail, tails_raw.data(), tails_raw.size() * 4, cudaMemcpyHostToDevice)))
        return wrc;
    }
    if (rc) return rc;
    *elapsed_ns = total;
    if (bad) return fail(GENESYS_EINVAL, "service probe: %llu calls returned a short count", (unsigned long long)bad);
    return 0;
  });
}

int genesys_emulate_call(genesys_ctx *c, uint32_t nr, const uint64_t args[6], uint32_t flags, int64_t *ret) {
  return genesys_guard("genesys_emulate_call", [&]() -> int {
    if (!c || !args || !ret) return fail(GENESYS_EINVAL, "NULL argument");
    if (!c->host_only) return fail(GENESYS_EINVAL, "genesys_emulate_call needs a host-only context");
    const uint64_t t0 = genesys_mono_ns();
    const uint64_t deadline = c->cfg.device_deadline_ns;
    static std::atomic<uint32_t> hint_ctr{0};
    uint32_t s = hint_ctr.fetch_add(1) % c->cfg.n_slots;
    for (uint32_t probes = 0;; ++probes) {
      uint32_t expect = 0;
      if (__atomic_compare_exchange_n(&c->owner[s], &expect, 1u, false, __ATOMIC_ACQUIRE, __ATOMIC_RELAXED)) break;
      s = (s + 1) % c->cfg.n_slots;
      if (probes % 64 == 63) {
        if (genesys_mono_ns() - t0 > deadline) return fail(GENESYS_ETIMEDOUT, "no free slot");
        std::this_thread::yield();
      }
    }
    const uint32_t sq = __atomic_load_n(&c->seq[s], __ATOMIC_RELAXED);
    if (__atomic_load_n(&c->known_done[s], __ATOMIC_RELAXED) != sq) {
      while ((uint32_t)(__atomic_load_n(&c->done[s], __ATOMIC_ACQUIRE) >> 32) != sq) {
        if (genesys_mono_ns() - t0 > deadline) {
          __atomic_store_n(&c->owner[s], 0u, __ATOMIC_RELEASE);
          return fail(GENESYS_ETIMEDOUT, "slot %u still busy", s);
        }
        cpu_relax();
      }
      __atomic_store_n(&c->known_done[s], sq, __ATOMIC_RELAXED);
    }
    const uint32_t nsq = sq + 1;
    __atomic_store_n(&c->seq[s], nsq, __ATOMIC_RELAXED);
    genesys_slot *sl = &c->slots[s];
    for (int i = 0; i < 6; ++i) __atomic_store_n(&sl->args[i], args[i], __ATOMIC_RELAXED);
    __atomic_store_n(&sl->req, ((uint64_t)nsq << 32) | ((uint64_t)(nr & 0xFFFFu) << 16) | (flags & 0xFFFFu),
                     __ATOMIC_RELEASE);
    // the ring the device would choose: by file region for pread/pwrite
    const uint32_t r = (nr == SYS_pread64 || nr == SYS_pwrite64)
                           ? genesys_ring_of_file(args[0], args[3], c->cfg.n_service_threads, nr == SYS_pread64)
                           : genesys_ring_of(s, c->cfg.n_service_threads);
    const uint32_t pos = __atomic_fetch_add(&c->ring_tail[r * 32], 1u, __ATOMIC_ACQ_REL);
    __atomic_store_n(&c->rings[(size_t)r * c->ring_cap + (pos & (c->ring_cap - 1))], GENESYS_RING_ENTRY(pos, s),
                     __ATOMIC_RELEASE);
    int64_t result = 0;
    if (flags & GENESYS_REQ_BLOCKING) {
      uint64_t d;
      for (;;) {
        d = __atomic_load_n(&c->done[s], __ATOMIC_ACQUIRE);
        if ((uint32_t)(d >> 32) == nsq) break;
        if (genesys_mono_ns() - t0 > deadline) {
          __atomic_store_n(&c->owner[s], 0u, __ATOMIC_RELEASE);
          return fail(GENESYS_ETIMEDOUT, "call not completed within the deadline");
        }
        if (c->cfg.flags & GENESYS_INIT_NO_THREADS) std::this_thread::yield(); else cpu_relax();
      }
      __atomic_store_n(&c->known_done[s], nsq, __ATOMIC_RELAXED);
      const uint32_t lo = (uint32_t)d;
      result = lo == GENESYS_RET_IN_SLOT ? (int64_t)__atomic_load_n(&sl->ret, __ATOMIC_RELAXED) : (int64_t)(int32_t)lo;
    }
    __atomic_store_n(&c->owner[s], 0u, __ATOMIC_RELEASE);
    *ret = result;
    return 0;
  });
}

}  // extern "C"
