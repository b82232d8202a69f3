// UDP echo server whose packet processing runs on the GPU (Sec. 7.3, Fig. 10:
// bandwidth versus packet size; the GPU part calls recvfrom/sendto at
// work-group grain, blocking, weak ordering).
//
// One persistent block per UDP socket (127.0.0.1:port_base + w).  A block
// receives one datagram with recvfrom (GENESYS_ECHO_SINGLE, the paper's form)
// or up to `batch` datagrams with recvmmsg (GENESYS_ECHO_BATCH), copies the
// bytes through its SMs from the receive buffer to the send buffer (both in
// host-mapped staging: the data crosses the host link in both directions), and
// sends each datagram back to its sender with sendto / sendmmsg.  Receives are
// non-blocking (MSG_DONTWAIT) and the block naps while its socket is idle, so
// that a quiet socket never holds a service thread inside the kernel.
//
// The load generator (genesys_echo_client) is closed loop: `window` packets in
// flight per server socket, each reply checked byte for byte against what was
// sent, and a new packet sent in its place.
#include <arpa/inet.h>
#include <cuda_runtime.h>
#include <errno.h>
#include <netinet/in.h>
#include <string.h>
#include <sys/socket.h>
#include <time.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "genesys.h"
#include "genesys_device.cuh"
#include "internal.h"

using namespace genesys;

namespace {

constexpr uint32_t kMaxBatch = GENESYS_ECHO_MAX_BATCH;
constexpr uint32_t kHeader = 8;  // client packet header: lane u32, generation u32

int set_err(int code, const char *msg) { return genesys_internal_error(code, msg); }

// Message headers of one block, at the start of its staging area; the receive
// buffers (batch x stride) and send buffers (batch x stride) follow.
struct EchoHeaders {
  mmsghdr rhdr[kMaxBatch];
  mmsghdr shdr[kMaxBatch];
  iovec riov[kMaxBatch];
  iovec siov[kMaxBatch];
  sockaddr_in6 addr[kMaxBatch];
  socklen_t alen;
};
constexpr uint64_t kHeadersBytes = (sizeof(EchoHeaders) + 255) & ~uint64_t(255);

inline void set_buffers(int fd) {
  const int want = 64 << 20;
  // SO_RCVBUFFORCE / SO_SNDBUFFORCE pass the system cap when permitted
  if (setsockopt(fd, SOL_SOCKET, SO_RCVBUFFORCE, &want, sizeof want) != 0)
    setsockopt(fd, SOL_SOCKET, SO_RCVBUF, &want, sizeof want);
  if (setsockopt(fd, SOL_SOCKET, SO_SNDBUFFORCE, &want, sizeof want) != 0)
    setsockopt(fd, SOL_SOCKET, SO_SNDBUF, &want, sizeof want);
}

// Copy n messages (len[i] bytes from src + i * stride to dst + i * stride)
// with the whole block: the 16-byte chunks of all messages are spread over
// the threads, four loads in flight per thread.  Receive buffers are read
// with ld.global.cv (the host rewrote them since the last batch).
__device__ void copy_messages(const genesys_dev &g, const uint8_t *src, uint8_t *dst, uint32_t stride,
                              const uint32_t *len, uint32_t n, uint32_t *prefix /* smem, kMaxBatch + 1 */) {
  if (threadIdx.x == 0) {
    uint32_t c = 0;
    for (uint32_t i = 0; i < n; ++i) { prefix[i] = c; c += (len[i] + 15) >> 4; }
    prefix[n] = c;
  }
  __syncthreads();
  const uint32_t total = prefix[n];
  constexpr int U = 4;
  for (uint32_t base = threadIdx.x; base < total; base += U * blockDim.x) {
    uint4 v[U];
    uint32_t at[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t c = base + u * blockDim.x;
      at[u] = ~0u;
      if (c < total) {
        uint32_t lo = 0, hi = n;  // message m with prefix[m] <= c < prefix[m + 1]
        while (hi - lo > 1) { const uint32_t mid = (lo + hi) >> 1; if (prefix[mid] <= c) lo = mid; else hi = mid; }
        at[u] = lo * stride + ((c - prefix[lo]) << 4);
        if (!dcheck(g, lo < n && ((c - prefix[lo]) << 4) + 16 <= stride)) { at[u] = ~0u; continue; }
        v[u] = __ldcv(reinterpret_cast<const uint4 *>(src + at[u]));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (at[u] != ~0u) *reinterpret_cast<uint4 *>(dst + at[u]) = v[u];
  }
}

template <bool kBatch>
__global__ void __launch_bounds__(1024) echo_server_kernel(genesys_dev g, const int32_t *fds, uint8_t *areas,
                                                           uint64_t area_bytes, uint32_t batch, uint32_t stride,
                                                           volatile int32_t *stop_flag, uint64_t idle_timeout_ns,
                                                           unsigned long long *counters) {
  __shared__ uint32_t s_len[kMaxBatch];
  __shared__ uint32_t s_prefix[kMaxBatch + 1];
  __shared__ int s_leave;
  uint8_t *area = areas + blockIdx.x * area_bytes;
  EchoHeaders *H = reinterpret_cast<EchoHeaders *>(area);
  uint8_t *rbuf = area + kHeadersBytes;
  uint8_t *sbuf = rbuf + (uint64_t)batch * stride;
  const int fd = fds[blockIdx.x];
  if (kBatch) {
    for (uint32_t i = threadIdx.x; i < batch; i += blockDim.x) {
      H->riov[i].iov_base = rbuf + (uint64_t)i * stride;
      H->riov[i].iov_len = stride;
      memset(&H->rhdr[i], 0, sizeof(mmsghdr));
      H->rhdr[i].msg_hdr.msg_name = &H->addr[i];
      H->rhdr[i].msg_hdr.msg_iov = &H->riov[i];
      H->rhdr[i].msg_hdr.msg_iovlen = 1;
      memset(&H->shdr[i], 0, sizeof(mmsghdr));
      H->shdr[i].msg_hdr.msg_name = &H->addr[i];
      H->shdr[i].msg_hdr.msg_iov = &H->siov[i];
      H->shdr[i].msg_hdr.msg_iovlen = 1;
      H->siov[i].iov_base = sbuf + (uint64_t)i * stride;
    }
  }
  uint64_t idle_since = now_ns();
  uint32_t nap = 256;
  unsigned long long packets = 0, bytes = 0;
  for (;;) {
    int64_t n;
    if (kBatch) {
      for (uint32_t i = threadIdx.x; i < batch; i += blockDim.x)
        H->rhdr[i].msg_hdr.msg_namelen = sizeof(sockaddr_in6);
      __syncthreads();  // the consumer-role call has no barrier before it
      n = call<GROUP, RELAXED, BLOCKING, ROLE_CONSUMER>(g, SYS_recvmmsg, (uint64_t)fd, (uint64_t)H->rhdr, batch,
                                                       MSG_DONTWAIT, 0);
    } else {
      if (threadIdx.x == 0) H->alen = sizeof(sockaddr_in6);  // the calling thread's own store
      n = call<GROUP, RELAXED, BLOCKING, ROLE_CONSUMER>(g, SYS_recvfrom, (uint64_t)fd, (uint64_t)rbuf, stride,
                                                       MSG_DONTWAIT, (uint64_t)&H->addr[0], (uint64_t)&H->alen);
    }
    if (n == -EAGAIN || n == 0) {
      // thread 0 decides for the block, so that every thread leaves together
      if (threadIdx.x == 0) s_leave = *stop_flag || now_ns() - idle_since > idle_timeout_ns;
      __syncthreads();
      const int leave = s_leave;
      __syncthreads();
      if (leave) break;
      __nanosleep(nap);
      nap = nap < 16384 ? nap * 2 : nap;
      continue;
    }
    if (n < 0) break;
    idle_since = now_ns();
    nap = 256;
    const uint32_t m = kBatch ? (uint32_t)n : 1u;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x)
      s_len[i] = kBatch ? *(volatile unsigned int *)&H->rhdr[i].msg_len : (uint32_t)n;
    __syncthreads();
    // a GENESYS_ECHO_STOP_BYTES datagram is the last one its socket gets
    const bool stop = s_len[m - 1] == GENESYS_ECHO_STOP_BYTES;
    const uint32_t echo = stop ? m - 1 : m;
    copy_messages(g, rbuf, sbuf, stride, s_len, echo, s_prefix);
    if (kBatch) {
      for (uint32_t i = threadIdx.x; i < echo; i += blockDim.x) {
        H->siov[i].iov_len = s_len[i];
        H->shdr[i].msg_hdr.msg_namelen = *(volatile socklen_t *)&H->rhdr[i].msg_hdr.msg_namelen;
      }
    }
    // the barrier before the call publishes the copies; the one after it
    // gives every thread the result (the loop runs in step on all threads)
    uint32_t sent = 0;
    while (sent < echo) {
      int64_t r;
      if (kBatch)
        r = call<GROUP, RELAXED, BLOCKING, ROLE_BOTH>(g, SYS_sendmmsg, (uint64_t)fd, (uint64_t)(H->shdr + sent),
                                                      echo - sent, 0);
      else
        r = call<GROUP, RELAXED, BLOCKING, ROLE_BOTH>(g, SYS_sendto, (uint64_t)fd, (uint64_t)sbuf, s_len[0], 0,
                                                      (uint64_t)&H->addr[0],
                                                      (uint64_t)*(volatile socklen_t *)&H->alen) >= 0 ? 1 : -1;
      if (r <= 0) break;
      sent += (uint32_t)r;
    }
    for (uint32_t i = 0; i < sent; ++i) bytes += s_len[i];
    packets += sent;
    if (stop) break;
    __syncthreads();  // s_len and the buffers are reused by the next receive
  }
  if (threadIdx.x == 0) {
    atomicAdd(&counters[0], packets);
    atomicAdd(&counters[1], bytes);
  }
}

}  // namespace

struct genesys_echo_server {
  genesys_ctx *ctx = nullptr;
  std::vector<int> socks;
  cudaStream_t stream = nullptr, ctl = nullptr;
  void *dmem = nullptr;  // fds | stop flag | counters[2]
  int32_t *d_stop = nullptr;
  unsigned long long *d_counters = nullptr;
  uint64_t staging_mark = 0;
  bool running = false;
};

extern "C" int genesys_echo_start(genesys_ctx *c, uint32_t n_sockets, uint32_t max_packet, uint32_t form,
                                  uint32_t batch, uint32_t threads, uint16_t port_base, uint64_t idle_timeout_ns,
                                  genesys_echo_server **out) {
  return genesys_guard("genesys_echo_start", [&]() -> int {
    if (!c || !out) return set_err(GENESYS_EINVAL, "NULL argument");
    if (n_sockets == 0 || n_sockets > 1024 || max_packet < kHeader || max_packet > GENESYS_ECHO_PACKET_MAX ||
        form > GENESYS_ECHO_BATCH || threads < 32 || threads > 1024 || threads % 32)
      return set_err(GENESYS_EINVAL, "n_sockets 1..1024, max_packet 8..GENESYS_ECHO_PACKET_MAX, form SINGLE/BATCH, "
                                     "threads 32..1024 (multiple of 32)");
    if (form == GENESYS_ECHO_SINGLE) batch = 1;
    if (batch == 0 || batch > kMaxBatch) return set_err(GENESYS_EINVAL, "batch 1..GENESYS_ECHO_MAX_BATCH");
    const uint32_t stride = (max_packet + 255) & ~255u;
    const uint64_t area_bytes = kHeadersBytes + 2ull * batch * stride;
    auto s = new genesys_echo_server();
    s->ctx = c;
    auto fail_cleanup = [&](int code, const char *msg) {
      for (int fd : s->socks) close(fd);
      if (s->dmem) cudaFree(s->dmem);
      if (s->stream) cudaStreamDestroy(s->stream);
      if (s->ctl) cudaStreamDestroy(s->ctl);
      genesys_internal_staging_release(c, s->staging_mark);
      delete s;
      return set_err(code, msg);
    };
    s->staging_mark = genesys_internal_staging_mark(c);
    for (uint32_t w = 0; w < n_sockets; ++w) {
      int fd = socket(AF_INET, SOCK_DGRAM, 0);
      if (fd < 0) return fail_cleanup(GENESYS_EINVAL, "socket failed");
      s->socks.push_back(fd);
      set_buffers(fd);
      sockaddr_in a{};
      a.sin_family = AF_INET;
      a.sin_port = htons((uint16_t)(port_base + w));
      a.sin_addr.s_addr = htonl(INADDR_LOOPBACK);
      if (bind(fd, (sockaddr *)&a, sizeof a) != 0) return fail_cleanup(GENESYS_EINVAL, "bind failed (port in use?)");
    }
    const int dev = genesys_internal_device(c);
    if (cudaSetDevice(dev) != cudaSuccess) return fail_cleanup(GENESYS_ECUDA, "cudaSetDevice");
    const size_t o_stop = (4ull * n_sockets + 15) & ~size_t(15), o_cnt = o_stop + 16, bytes = o_cnt + 16;
    if (cudaMalloc(&s->dmem, bytes) != cudaSuccess) return fail_cleanup(GENESYS_ENOMEM, "device memory");
    uint8_t *d = (uint8_t *)s->dmem;
    std::vector<int32_t> fds(s->socks.begin(), s->socks.end());
    if (cudaMemset(d, 0, bytes) != cudaSuccess ||
        cudaMemcpy(d, fds.data(), 4ull * n_sockets, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail_cleanup(GENESYS_ECUDA, "upload");
    s->d_stop = (int32_t *)(d + o_stop);
    s->d_counters = (unsigned long long *)(d + o_cnt);
    uint8_t *areas = (uint8_t *)genesys_staging(c, area_bytes * n_sockets);
    if (!areas) return fail_cleanup(GENESYS_ENOMEM, "staging arena too small for the echo buffers");
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->ctl, cudaStreamNonBlocking) != cudaSuccess)
      return fail_cleanup(GENESYS_ECUDA, "streams");
    genesys_dev g;
    genesys_device_view(c, &g);
    const int32_t *d_fds = (const int32_t *)d;
    uint64_t ab = area_bytes;
    uint32_t bt = batch, st = stride;
    volatile int32_t *stop = s->d_stop;
    uint64_t idle = idle_timeout_ns ? idle_timeout_ns : 10000000000ull;
    unsigned long long *cnt = s->d_counters;
    void *args[] = {&g, &d_fds, &areas, &ab, &bt, &st, &stop, &idle, &cnt};
    const uint32_t g3[3] = {n_sockets, 1, 1}, b3[3] = {threads, 1, 1};
    const void *k = form == GENESYS_ECHO_BATCH ? (const void *)&echo_server_kernel<true>
                                               : (const void *)&echo_server_kernel<false>;
    const int rc = genesys_launch(c, k, g3, b3, 0, args, GENESYS_GRAN_GROUP | GENESYS_LAUNCH_RELAXED, s->stream);
    if (rc) return fail_cleanup(rc, genesys_last_error());
    s->running = true;
    genesys_internal_servers(c, +1);
    *out = s;
    return 0;
  });
}

extern "C" int genesys_echo_stop(genesys_echo_server *s, uint64_t timeout_ns, uint64_t *stats) {
  return genesys_guard("genesys_echo_stop", [&]() -> int {
    if (!s) return set_err(GENESYS_EINVAL, "NULL server");
    int rc = 0;
    if (s->running) {
      const int32_t one = 1;
      cudaMemcpyAsync(s->d_stop, &one, 4, cudaMemcpyHostToDevice, s->ctl);
      cudaStreamSynchronize(s->ctl);
      const uint64_t until = genesys_mono_ns() + timeout_ns;
      while (cudaStreamQuery(s->stream) == cudaErrorNotReady) {
        if (genesys_mono_ns() > until) { rc = set_err(GENESYS_ETIMEDOUT, "echo server did not stop"); break; }
        std::this_thread::sleep_for(std::chrono::microseconds(100));
      }
      if (rc == 0) {  // the kernel has finished (else it stays running: a later stop waits again)
        cudaStreamSynchronize(s->stream);
        s->running = false;
        genesys_internal_servers(s->ctx, -1);
      }
    }
    if (rc == 0) rc = genesys_drain(s->ctx, timeout_ns);  // its last calls, also on a repeated stop
    if (stats) {
      unsigned long long v[2] = {0, 0};
      cudaMemcpy(v, s->d_counters, sizeof v, cudaMemcpyDeviceToHost);
      stats[0] = v[0];
      stats[1] = v[1];
    }
    if (rc) return rc;  // the kernel may still run (or calls are pending): keep its memory
    for (int fd : s->socks) close(fd);
    cudaFree(s->dmem);
    cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->ctl);
    genesys_internal_staging_release(s->ctx, s->staging_mark);
    delete s;
    return 0;
  });
}

// ---------------------------------------------------------------- client
namespace {

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct EchoLane {
  uint32_t server;        // server socket index
  uint32_t gen = 0;       // generation of the packet in flight
  bool busy = false;
  std::vector<uint8_t> pkt;
};

struct EchoTally {
  uint64_t sent = 0, echoed = 0, bad = 0, lost = 0, bytes = 0, send_err = 0, first = ~0ull, last = 0;
};

void echo_client_thread(uint32_t t, uint32_t n_threads, uint16_t port_base, uint32_t n_sockets, uint32_t P,
                        uint64_t quota, uint32_t window, uint64_t seed, uint64_t stall_ns, EchoTally *out) {
  EchoTally T;
  int fd = socket(AF_INET, SOCK_DGRAM, 0);
  if (fd < 0) { T.send_err = quota; *out = T; return; }
  set_buffers(fd);
  sockaddr_in me{};
  me.sin_family = AF_INET;
  me.sin_addr.s_addr = htonl(INADDR_LOOPBACK);
  bind(fd, (sockaddr *)&me, sizeof me);
  int rcv = 0;
  socklen_t rl = sizeof rcv;
  getsockopt(fd, SOL_SOCKET, SO_RCVBUF, &rcv, &rl);
  // lanes: `window` per server socket this thread owns, capped so that the
  // replies in flight fit in half of this socket's receive buffer
  std::vector<uint32_t> mine;
  for (uint32_t s = t; s < n_sockets; s += n_threads) mine.push_back(s);
  const uint64_t fit = std::max<uint64_t>(1, (uint64_t)rcv / 2 / ((uint64_t)P + 256));
  uint32_t w = window;
  while (w > 1 && (uint64_t)w * mine.size() > fit) --w;
  std::vector<EchoLane> lanes;
  for (uint32_t s : mine)
    for (uint32_t k = 0; k < w; ++k) {
      EchoLane L;
      L.server = s;
      L.pkt.resize(P);
      const uint32_t id = (uint32_t)lanes.size();
      memcpy(L.pkt.data(), &id, 4);
      for (uint32_t b = kHeader; b < P; ++b)
        L.pkt[b] = (uint8_t)(mix64(seed ^ ((uint64_t)t << 48) ^ ((uint64_t)id << 32) ^ (b >> 3)) >> (8 * (b & 7)));
      lanes.push_back(std::move(L));
    }
  constexpr int kB = 32;
  std::vector<mmsghdr> sh(kB), rh(kB);
  std::vector<iovec> siov(kB), riov(kB);
  std::vector<sockaddr_in> to(kB);
  std::vector<uint8_t> rbuf((size_t)kB * (P + 64));
  int ns = 0;
  uint64_t busy = 0;  // lanes with a packet in flight
  auto queue = [&](uint32_t id) {
    EchoLane &L = lanes[id];
    ++L.gen;
    memcpy(L.pkt.data() + 4, &L.gen, 4);
    L.busy = true;
    ++busy;
    to[ns] = sockaddr_in{};
    to[ns].sin_family = AF_INET;
    to[ns].sin_port = htons((uint16_t)(port_base + L.server));
    to[ns].sin_addr.s_addr = htonl(INADDR_LOOPBACK);
    siov[ns] = {L.pkt.data(), P};
    memset(&sh[ns], 0, sizeof(mmsghdr));
    sh[ns].msg_hdr.msg_name = &to[ns];
    sh[ns].msg_hdr.msg_namelen = sizeof(sockaddr_in);
    sh[ns].msg_hdr.msg_iov = &siov[ns];
    sh[ns].msg_hdr.msg_iovlen = 1;
    ++ns;
    ++T.sent;
  };
  auto flush = [&] {
    int done = 0;
    while (done < ns) {
      const int r = sendmmsg(fd, sh.data() + done, ns - done, 0);
      if (r <= 0) {
        for (int i = done; i < ns; ++i) {
          uint32_t id;
          memcpy(&id, siov[i].iov_base, 4);
          lanes[id].busy = false;
          --busy;
        }
        T.send_err += ns - done;
        break;
      }
      done += r;
    }
    ns = 0;
  };
  T.first = genesys_mono_ns();
  for (uint32_t id = 0; id < lanes.size() && T.sent < quota; ++id) {
    queue(id);
    if (ns == kB) flush();
  }
  flush();
  uint64_t last_reply = genesys_mono_ns();
  while (busy) {
    for (int i = 0; i < kB; ++i) {
      riov[i] = {rbuf.data() + (size_t)i * (P + 64), P + 64};
      memset(&rh[i], 0, sizeof(mmsghdr));
      rh[i].msg_hdr.msg_iov = &riov[i];
      rh[i].msg_hdr.msg_iovlen = 1;
    }
    const int m = recvmmsg(fd, rh.data(), kB, MSG_DONTWAIT, nullptr);
    const uint64_t now = genesys_mono_ns();
    if (m <= 0) {
      if (now - last_reply > stall_ns) break;
      continue;
    }
    last_reply = now;
    for (int i = 0; i < m; ++i) {
      const uint8_t *r = rbuf.data() + (size_t)i * (P + 64);
      uint32_t id = ~0u, gen = 0;
      if (rh[i].msg_len >= kHeader) { memcpy(&id, r, 4); memcpy(&gen, r + 4, 4); }
      if (id >= lanes.size() || !lanes[id].busy || gen != lanes[id].gen) { ++T.bad; continue; }
      EchoLane &L = lanes[id];
      L.busy = false;
      --busy;
      if (rh[i].msg_len != P || memcmp(r, L.pkt.data(), P) != 0) {
        ++T.bad;
      } else {
        ++T.echoed;
        T.bytes += P;
      }
      if (T.sent < quota) queue(id);
    }
    T.last = now;
    flush();
  }
  T.lost = busy;
  close(fd);
  *out = T;
}

}  // namespace

extern "C" int genesys_echo_client(uint16_t port_base, uint32_t n_sockets, uint32_t packet_bytes, uint64_t n_packets,
                                   uint32_t window, uint32_t n_threads, uint64_t seed, uint64_t stall_ns,
                                   uint32_t send_stop, uint64_t *stats) {
  return genesys_guard("genesys_echo_client", [&]() -> int {
    if (!stats || n_sockets == 0 || packet_bytes < kHeader || packet_bytes > GENESYS_ECHO_PACKET_MAX || window == 0 ||
        n_threads == 0)
      return set_err(GENESYS_EINVAL, "bad argument");
    n_threads = std::min(n_threads, n_sockets);
    std::vector<EchoTally> tally(n_threads);
    std::vector<std::thread> th;
    genesys_joiner join_all{th};
    for (uint32_t t = 0; t < n_threads; ++t) {
      const uint64_t quota = n_packets / n_threads + (t < n_packets % n_threads ? 1 : 0);
      th.emplace_back(echo_client_thread, t, n_threads, port_base, n_sockets, packet_bytes, quota, window, seed,
                      stall_ns ? stall_ns : 200000000ull, &tally[t]);
    }
    for (auto &x : th) x.join();
    EchoTally S;
    for (auto &T : tally) {
      S.sent += T.sent; S.echoed += T.echoed; S.bad += T.bad; S.lost += T.lost; S.bytes += T.bytes;
      S.send_err += T.send_err;
      S.first = std::min(S.first, T.first);
      S.last = std::max(S.last, T.last);
    }
    if (send_stop) {
      int fd = socket(AF_INET, SOCK_DGRAM, 0);
      if (fd >= 0) {
        for (uint32_t w = 0; w < n_sockets; ++w) {
          const uint8_t stop[GENESYS_ECHO_STOP_BYTES] = {0};
          sockaddr_in to{};
          to.sin_family = AF_INET;
          to.sin_port = htons((uint16_t)(port_base + w));
          to.sin_addr.s_addr = htonl(INADDR_LOOPBACK);
          sendto(fd, stop, sizeof stop, 0, (sockaddr *)&to, sizeof to);
        }
        close(fd);
      }
    }
    stats[0] = S.sent;
    stats[1] = S.echoed;
    stats[2] = S.bad;
    stats[3] = S.lost;
    stats[4] = S.last > S.first ? S.last - S.first : 0;
    stats[5] = S.bytes;
    stats[6] = S.send_err;
    return 0;
  });
}
