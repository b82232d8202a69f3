// C4: a key-value service whose server runs on the GPU and talks UDP through
// GPU system calls (Sec. 7.3: the GPU part of the echo server calls
// recvfrom/sendto at work-group granularity; here batched as recvmmsg /
// sendmmsg, one batch per call).
//
// The table lives in HBM: n_keys 16-byte keys in an open-addressing index,
// values in fixed 1024-byte slots.  One persistent block per UDP socket
// (port_base + w); a client sends each key's requests to socket
// (first four key bytes, little-endian) mod n_sockets, so the requests of one
// key arrive at one block in the order they were sent.  A block receives a
// batch, orders same-key requests of the batch into waves (a request runs
// after the previous request of its key), applies GET/SET one request per
// warp, writes the replies and sends them back as one batch.
//
// Wire format (little-endian).  Request: op u8 (0 GET, 1 SET, 2 STOP), pad u8,
// vlen u16, seq u32, key[16], value[vlen] (SET).  Reply: op|0x80 u8, status u8
// (0 ok, 1 no such key), vlen u16, seq u32, value[vlen] (GET of a present key).
#include <arpa/inet.h>
#include <cuda_runtime.h>
#include <sched.h>
#include <errno.h>
#include <netinet/in.h>
#include <pthread.h>
#include <stdio.h>
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

constexpr uint32_t kVal = GENESYS_KV_VALUE_MAX;       // value slot bytes
constexpr uint32_t kReq = 24 + kVal;                  // largest request datagram
constexpr uint32_t kRep = 8 + kVal;                   // largest reply datagram
constexpr uint32_t kBufStride = (kReq + 63) & ~63u;   // per-message buffer
constexpr uint32_t kMaxBatch = GENESYS_KV_MAX_BATCH;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

int set_err(int code, const char *msg) { return genesys_internal_error(code, msg); }

__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t key_hash(uint64_t k0, uint64_t k1) {
  uint64_t z = k0 * 0x9E3779B97F4A7C15ull ^ k1 * 0xC2B2AE3D27D4EB4Full;
  return z ^ (z >> 29);
}

// Per-block layout in host-mapped staging.
struct KvBlockArea {
  mmsghdr rhdr[kMaxBatch];
  mmsghdr shdr[kMaxBatch];
  iovec riov[kMaxBatch];
  iovec siov[kMaxBatch];
  sockaddr_in6 addr[kMaxBatch];  // senders' addresses, from recvmmsg
  uint8_t rbuf[kMaxBatch][kBufStride];
  uint8_t sbuf[kMaxBatch][kBufStride];
};

// Table build: values of the preload (value i = stream of seed vseed[i]) and
// the key index (slot -> key number + 1).
__global__ void kv_build_kernel(const uint8_t *keys, const uint16_t *vlen0, const uint64_t *vseed0, uint32_t n_keys,
                                uint32_t *index, uint32_t index_mask, uint8_t *vals, uint16_t *vlens) {
  const uint32_t i = blockIdx.x;
  if (i >= n_keys) return;
  const uint32_t words = (vlen0[i] + 7) / 8;
  uint64_t *v = reinterpret_cast<uint64_t *>(vals + (size_t)i * kVal);
  for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) v[w] = sm_mix(vseed0[i] + (w + 1) * kGamma);
  if (threadIdx.x == 0) {
    vlens[i] = vlen0[i];
    const uint64_t *k = reinterpret_cast<const uint64_t *>(keys + 16 * (size_t)i);
    uint32_t h = (uint32_t)key_hash(k[0], k[1]) & index_mask;
    for (uint32_t probe = 0; probe <= index_mask; ++probe) {
      if (atomicCAS(&index[h], 0u, i + 1) == 0u) break;
      h = (h + 1) & index_mask;
    }
  }
}

__device__ __forceinline__ int32_t kv_lookup(const uint8_t *keys, const uint32_t *index, uint32_t index_mask,
                                             uint64_t k0, uint64_t k1) {
  uint32_t h = (uint32_t)key_hash(k0, k1) & index_mask;
  for (uint32_t probe = 0; probe <= index_mask; ++probe) {
    const uint32_t e = index[h];
    if (e == 0) return -1;
    const uint64_t *k = reinterpret_cast<const uint64_t *>(keys + 16 * (size_t)(e - 1));
    if (k[0] == k0 && k[1] == k1) return (int32_t)(e - 1);
    h = (h + 1) & index_mask;
  }
  return -1;
}

struct KvShared {
  int32_t ki[kMaxBatch];     // key number or -1
  int32_t pred[kMaxBatch];   // previous request of the same key in the batch, or -1
  uint8_t level[kMaxBatch];
  uint32_t rep_len[kMaxBatch];
  uint32_t n_levels;
  int stop;
};

__global__ void __launch_bounds__(1024) kv_server_kernel(genesys_dev g, const int32_t *fds, KvBlockArea *areas,
                                                         uint32_t batch, const uint8_t *keys, const uint32_t *index,
                                                         uint32_t index_mask, uint8_t *vals, uint16_t *vlens,
                                                         volatile int32_t *stop_flag, uint64_t idle_timeout_ns,
                                                         unsigned long long *served, uint32_t *seen) {
  __shared__ KvShared S;
  KvBlockArea *A = areas + blockIdx.x;
  const int fd = fds[blockIdx.x];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // one-time set-up of the message headers (host-mapped memory)
  for (uint32_t i = threadIdx.x; i < batch; i += blockDim.x) {
    A->riov[i].iov_base = A->rbuf[i];
    A->riov[i].iov_len = kReq;
    memset(&A->rhdr[i], 0, sizeof(mmsghdr));
    A->rhdr[i].msg_hdr.msg_name = &A->addr[i];
    A->rhdr[i].msg_hdr.msg_iov = &A->riov[i];
    A->rhdr[i].msg_hdr.msg_iovlen = 1;
    memset(&A->shdr[i], 0, sizeof(mmsghdr));
    A->shdr[i].msg_hdr.msg_name = &A->addr[i];
    A->shdr[i].msg_hdr.msg_iov = &A->siov[i];
    A->shdr[i].msg_hdr.msg_iovlen = 1;
    A->siov[i].iov_base = A->sbuf[i];
  }
  uint64_t idle_since = now_ns();
  uint32_t nap = 256;
  unsigned long long my_served = 0;
  for (;;) {
    for (uint32_t i = threadIdx.x; i < batch; i += blockDim.x) A->rhdr[i].msg_hdr.msg_namelen = sizeof(sockaddr_in6);
    // the consumer-role call has no barrier before it: these stores of other
    // threads reach the host ahead of the request through this barrier and
    // the caller's release
    __syncthreads();
    const int64_t n = call<GROUP, RELAXED, BLOCKING, ROLE_CONSUMER>(g, SYS_recvmmsg, (uint64_t)fd, (uint64_t)A->rhdr,
                                                                    batch, MSG_DONTWAIT, 0);
    if (n == -EAGAIN || n == 0) {
      // thread 0 decides for the block, so that every thread leaves together
      if (threadIdx.x == 0) S.stop = *stop_flag || now_ns() - idle_since > idle_timeout_ns;
      __syncthreads();
      const int leave = S.stop;
      __syncthreads();
      if (leave) break;
      __nanosleep(nap);
      nap = nap < 16384 ? nap * 2 : nap;
      continue;
    }
    if (n < 0) break;
    idle_since = now_ns();
    nap = 256;
    // parse: key lookup, same-key predecessor in the batch
    if (threadIdx.x == 0) S.stop = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < (uint32_t)n; i += blockDim.x) {
      const uint8_t *q = A->rbuf[i];
      const uint64_t *k = reinterpret_cast<const uint64_t *>(q + 8);
      if (q[0] == GENESYS_KV_STOP) {
        S.ki[i] = -2;
        S.stop = 1;
      } else {
        S.ki[i] = kv_lookup(keys, index, index_mask, k[0], k[1]);
        // the log of received requests (genesys_kv_received)
        const uint32_t seq = (uint32_t)q[4] | ((uint32_t)q[5] << 8) | ((uint32_t)q[6] << 16) | ((uint32_t)q[7] << 24);
        if (seq < GENESYS_KV_SEQ_LOG) atomicOr(&seen[seq >> 5], 1u << (seq & 31));
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < (uint32_t)n; i += blockDim.x) {
      int32_t p = -1;
      if (S.ki[i] >= 0)
        for (int32_t j = (int32_t)i - 1; j >= 0; --j)
          if (S.ki[j] == S.ki[i]) { p = j; break; }
      S.pred[i] = p;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t mx = 0;
      for (uint32_t i = 0; i < (uint32_t)n; ++i) {
        S.level[i] = S.pred[i] < 0 ? 0 : (uint8_t)(S.level[S.pred[i]] + 1);
        mx = S.level[i] > mx ? S.level[i] : mx;
      }
      S.n_levels = mx + 1;
    }
    __syncthreads();
    // apply in waves; one warp per request
    for (uint32_t lv = 0; lv < S.n_levels; ++lv) {
      for (uint32_t i = warp; i < (uint32_t)n; i += nwarps) {
        if (S.level[i] != lv) continue;
        const uint8_t *q = A->rbuf[i];
        uint8_t *rep = A->sbuf[i];
        const int32_t ki = S.ki[i];
        if (ki == -2) {
          if (lane == 0) S.rep_len[i] = 0;
          continue;
        }
        const uint8_t op = q[0];
        uint32_t rlen = 0;
        uint8_t status = 1;
        if (ki >= 0 && op == GENESYS_KV_GET) {
          status = 0;
          rlen = vlens[ki];
          const uint8_t *src = vals + (size_t)ki * kVal;
          for (uint32_t b = lane * 8; b < rlen; b += 256)
            *reinterpret_cast<uint64_t *>(rep + 8 + b) = *reinterpret_cast<const uint64_t *>(src + b);
        } else if (ki >= 0 && op == GENESYS_KV_SET) {
          status = 0;
          uint32_t vlen = q[2] | (q[3] << 8);
          if (vlen > kVal) vlen = kVal;
          uint8_t *dst = vals + (size_t)ki * kVal;
          for (uint32_t b = lane * 8; b < vlen; b += 256)
            *reinterpret_cast<uint64_t *>(dst + b) = *reinterpret_cast<const uint64_t *>(q + 24 + b);
          if (lane == 0) vlens[ki] = (uint16_t)vlen;
        }
        if (lane == 0) {
          rep[0] = (uint8_t)(op | 0x80);
          rep[1] = status;
          rep[2] = (uint8_t)rlen;
          rep[3] = (uint8_t)(rlen >> 8);
          rep[4] = q[4]; rep[5] = q[5]; rep[6] = q[6]; rep[7] = q[7];
          S.rep_len[i] = 8 + rlen;
        }
        __syncwarp();
      }
      __syncthreads();
    }
    // send the replies of this batch (the STOP message gets none)
    uint32_t m = 0;
    for (uint32_t i = threadIdx.x; i < (uint32_t)n; i += blockDim.x) {
      A->siov[i].iov_len = S.rep_len[i];
      A->shdr[i].msg_hdr.msg_namelen = A->rhdr[i].msg_hdr.msg_namelen;
    }
    if (S.stop) m = (uint32_t)n - 1; else m = (uint32_t)n;   // STOP is the last message of its socket
    uint32_t sent = 0;
    while (sent < m) {
      const int64_t r = call<GROUP, RELAXED, BLOCKING, ROLE_BOTH>(g, SYS_sendmmsg, (uint64_t)fd,
                                                                 (uint64_t)(A->shdr + sent), m - sent, 0);
      if (r <= 0) break;
      sent += (uint32_t)r;
    }
    my_served += sent;
    if (S.stop) break;
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(served, my_served);
}

}  // namespace

struct genesys_kv_server {
  genesys_ctx *ctx = nullptr;
  uint32_t n_sockets = 0, batch = 0, n_keys = 0;
  std::vector<int> socks;
  cudaStream_t stream = nullptr, ctl = nullptr;
  void *dmem = nullptr;          // device: fds, index, keys, vals, vlens, stop flag, served
  int32_t *d_stop = nullptr;
  unsigned long long *d_served = nullptr;
  uint32_t *d_seen = nullptr;    // received-request log, GENESYS_KV_SEQ_LOG bits
  uint8_t *d_vals = nullptr;
  uint16_t *d_vlens = nullptr;
  uint64_t staging_mark = 0;
  bool running = false;
};

extern "C" int genesys_kv_start(genesys_ctx *c, const uint8_t *keys, const uint16_t *vlen0, const uint64_t *vseed0,
                                uint32_t n_keys, uint32_t n_sockets, uint32_t batch, uint32_t threads,
                                uint16_t port_base, uint64_t idle_timeout_ns, genesys_kv_server **out) {
  return genesys_guard("genesys_kv_start", [&]() -> int {
    if (!c || !keys || !vlen0 || !vseed0 || !out || n_keys == 0) return set_err(GENESYS_EINVAL, "NULL argument");
    if (n_sockets == 0 || n_sockets > 1024 || batch == 0 || batch > kMaxBatch || threads < 32 || threads > 1024 ||
        threads % 32)
      return set_err(GENESYS_EINVAL, "n_sockets 1..1024, batch 1..64, threads 32..1024 (multiple of 32)");
    for (uint32_t i = 0; i < n_keys; ++i)
      if (vlen0[i] > kVal) return set_err(GENESYS_EINVAL, "value longer than GENESYS_KV_VALUE_MAX");
    auto s = new genesys_kv_server();
    s->ctx = c;
    s->n_sockets = n_sockets;
    s->batch = batch;
    s->n_keys = n_keys;
    auto fail_cleanup = [&](int code, const char *msg) {
      for (int fd : s->socks) close(fd);
      if (s->dmem) cudaFree(s->dmem);
      if (s->stream) cudaStreamDestroy(s->stream);
      if (s->ctl) cudaStreamDestroy(s->ctl);
      genesys_internal_staging_release(c, s->staging_mark);
      delete s;
      return set_err(code, msg);
    };
    // sockets: 127.0.0.1:port_base + w, large receive buffers
    for (uint32_t w = 0; w < n_sockets; ++w) {
      int fd = socket(AF_INET, SOCK_DGRAM, 0);
      if (fd < 0) return fail_cleanup(GENESYS_EINVAL, "socket failed");
      s->socks.push_back(fd);
      // SO_RCVBUFFORCE / SO_SNDBUFFORCE pass the system cap (net.core.rmem_max,
      // often a few hundred KiB) when permitted: bursts of requests then wait in
      // the socket instead of being dropped
      int buf = 64 << 20;
      if (setsockopt(fd, SOL_SOCKET, SO_RCVBUFFORCE, &buf, sizeof buf) != 0)
        setsockopt(fd, SOL_SOCKET, SO_RCVBUF, &buf, sizeof buf);
      if (setsockopt(fd, SOL_SOCKET, SO_SNDBUFFORCE, &buf, sizeof buf) != 0)
        setsockopt(fd, SOL_SOCKET, SO_SNDBUF, &buf, sizeof buf);
      sockaddr_in a{};
      a.sin_family = AF_INET;
      a.sin_port = htons((uint16_t)(port_base + w));
      a.sin_addr.s_addr = htonl(INADDR_LOOPBACK);
      if (bind(fd, (sockaddr *)&a, sizeof a) != 0) return fail_cleanup(GENESYS_EINVAL, "bind failed (port in use?)");
    }
    const int dev = genesys_internal_device(c);
    if (cudaSetDevice(dev) != cudaSuccess) return fail_cleanup(GENESYS_ECUDA, "cudaSetDevice");
    uint32_t index_size = 1;
    while (index_size < 2 * n_keys) index_size <<= 1;
    // device memory: fds | stop | served | index | keys | vals | vlens | vlen0 | vseed0
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (off + bytes + 255) & ~size_t(255); return o; };
    const size_t o_fds = take(4 * n_sockets), o_stop = take(4), o_served = take(8),
                 o_seen = take(GENESYS_KV_SEQ_LOG / 8), o_index = take(4ull * index_size),
                 o_keys = take(16ull * n_keys), o_vals = take((size_t)kVal * n_keys), o_vlens = take(2ull * n_keys),
                 o_vlen0 = take(2ull * n_keys), o_vseed0 = take(8ull * n_keys);
    if (cudaMalloc(&s->dmem, off) != cudaSuccess) return fail_cleanup(GENESYS_ENOMEM, "device memory for the table");
    uint8_t *d = (uint8_t *)s->dmem;
    std::vector<int32_t> fds(s->socks.begin(), s->socks.end());
    if (cudaMemset(d, 0, o_keys) != cudaSuccess ||
        cudaMemcpy(d + o_fds, fds.data(), 4 * n_sockets, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + o_keys, keys, 16ull * n_keys, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + o_vlen0, vlen0, 2ull * n_keys, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + o_vseed0, vseed0, 8ull * n_keys, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail_cleanup(GENESYS_ECUDA, "upload of the table");
    s->d_stop = (int32_t *)(d + o_stop);
    s->d_served = (unsigned long long *)(d + o_served);
    s->d_seen = (uint32_t *)(d + o_seen);  // zeroed with the rest of [0, o_keys) above
    s->d_vals = d + o_vals;
    s->d_vlens = (uint16_t *)(d + o_vlens);
    kv_build_kernel<<<n_keys, 128>>>(d + o_keys, (const uint16_t *)(d + o_vlen0), (const uint64_t *)(d + o_vseed0),
                                     n_keys, (uint32_t *)(d + o_index), index_size - 1, d + o_vals, s->d_vlens);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail_cleanup(GENESYS_ECUDA, "table build");
    // staging: one message area per block
    s->staging_mark = genesys_internal_staging_mark(c);
    KvBlockArea *areas = (KvBlockArea *)genesys_staging(c, sizeof(KvBlockArea) * n_sockets);
    if (!areas) return fail_cleanup(GENESYS_ENOMEM, "staging arena too small for the message areas");
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->ctl, cudaStreamNonBlocking) != cudaSuccess)
      return fail_cleanup(GENESYS_ECUDA, "streams");
    genesys_dev g;
    genesys_device_view(c, &g);
    const int32_t *d_fds = (const int32_t *)(d + o_fds);
    const uint8_t *d_keys = d + o_keys;
    const uint32_t *d_index = (const uint32_t *)(d + o_index);
    uint32_t imask = index_size - 1, bt = batch;
    uint8_t *vals = s->d_vals;
    uint16_t *vl = s->d_vlens;
    volatile int32_t *stop = s->d_stop;
    uint64_t idle = idle_timeout_ns ? idle_timeout_ns : 10000000000ull;
    unsigned long long *served = s->d_served;
    uint32_t *seen = s->d_seen;
    void *args[] = {&g, &d_fds, &areas, &bt, &d_keys, &d_index, &imask, &vals, &vl, &stop, &idle, &served, &seen};
    const uint32_t g3[3] = {n_sockets, 1, 1}, b3[3] = {threads, 1, 1};
    int rc = genesys_launch(c, (const void *)&kv_server_kernel, g3, b3, 0, args,
                            GENESYS_GRAN_GROUP | GENESYS_LAUNCH_RELAXED, s->stream);
    if (rc) return fail_cleanup(rc, genesys_last_error());
    s->running = true;
    genesys_internal_servers(c, +1);
    *out = s;
    return 0;
  });
}

extern "C" int genesys_kv_stop(genesys_kv_server *s, uint64_t timeout_ns, uint64_t *served) {
  return genesys_guard("genesys_kv_stop", [&]() -> int {
    if (!s) return set_err(GENESYS_EINVAL, "NULL server");
    int rc = 0;
    if (s->running) {
      // ask the blocks to leave once idle (they also leave on a STOP message)
      const int32_t one = 1;
      cudaMemcpyAsync(s->d_stop, &one, 4, cudaMemcpyHostToDevice, s->ctl);
      cudaStreamSynchronize(s->ctl);
      const uint64_t until = genesys_mono_ns() + timeout_ns;
      while (cudaStreamQuery(s->stream) == cudaErrorNotReady) {
        if (genesys_mono_ns() > until) { rc = set_err(GENESYS_ETIMEDOUT, "kv server did not stop"); break; }
        std::this_thread::sleep_for(std::chrono::microseconds(100));
      }
      if (rc == 0) {  // the kernel has finished (else it stays running: a later stop waits again)
        cudaStreamSynchronize(s->stream);
        s->running = false;
        genesys_internal_servers(s->ctx, -1);
      }
    }
    if (rc == 0) rc = genesys_drain(s->ctx, timeout_ns);  // its last calls, also on a repeated stop
    if (served) {
      unsigned long long v = 0;
      cudaMemcpy(&v, s->d_served, 8, cudaMemcpyDeviceToHost);
      *served = v;
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

// The received-request log (for checks): bit j of out[j / 32] is set when
// the request with sequence number j has reached the server.
extern "C" int genesys_kv_received(genesys_kv_server *s, uint32_t *out, uint64_t n_seqs) {
  return genesys_guard("genesys_kv_received", [&]() -> int {
    if (!s || !out) return set_err(GENESYS_EINVAL, "NULL argument");
    if (n_seqs > GENESYS_KV_SEQ_LOG) return set_err(GENESYS_EINVAL, "the log holds GENESYS_KV_SEQ_LOG requests");
    const size_t words = (size_t)(n_seqs + 31) / 32;
    if (words && (cudaMemcpyAsync(out, s->d_seen, words * 4, cudaMemcpyDeviceToHost, s->ctl) != cudaSuccess ||
                  cudaStreamSynchronize(s->ctl) != cudaSuccess)) {
      cudaGetLastError();
      return set_err(GENESYS_ECUDA, "copy of the received-request log");
    }
    return 0;
  });
}

// Copy the current value of key `k` (for checks): returns its length.
extern "C" int genesys_kv_value(genesys_kv_server *s, uint32_t k, uint8_t *out) {
  return genesys_guard("genesys_kv_value", [&]() -> int {
    if (!s || !out || k >= s->n_keys) return set_err(GENESYS_EINVAL, "bad argument");
    uint16_t len = 0;
    if (cudaMemcpy(&len, s->d_vlens + k, 2, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(out, s->d_vals + (size_t)k * kVal, len, cudaMemcpyDeviceToHost) != cudaSuccess)
      return set_err(GENESYS_ECUDA, "copy");
    return len;
  });
}

// ---------------------------------------------------------------- client
// Open-loop load generator on host threads.  Thread w owns the server
// sockets s with s % n_threads == w and its own client socket: it sends its
// requests (those whose key maps to one of its sockets) in sequence order at
// their arrival times, batching every request that is due into one sendmmsg,
// and receives their replies on its socket (the server answers the sender),
// matching them by sequence number.  Requests of one key therefore leave in
// sequence order from one thread, and every reply is handled by the thread
// that sent its request.
namespace {

struct KvClientTally {
  uint64_t received = 0, dup = 0, bad = 0, send_err = 0, late_max = 0;
  bool timed_out = false;
};

void kv_client_thread(int fd, const std::vector<uint64_t> &mine, const uint8_t *reqs, const uint64_t *req_off,
                      uint64_t n, const uint64_t *arrival_ns, uint64_t t0, uint16_t port_base, uint32_t n_sockets,
                      uint64_t deadline, uint8_t *replies, uint32_t *reply_len, uint64_t *latency_ns,
                      uint64_t *t_send, KvClientTally *out) {
  KvClientTally T;
  constexpr int kB = 64;
  std::vector<mmsghdr> sh(kB), rh(kB);
  std::vector<iovec> siov(kB), riov(kB);
  std::vector<sockaddr_in> to(kB);
  std::vector<uint8_t> rb((size_t)kB * kRep);
  size_t i = 0;  // next request of `mine` to send
  uint64_t pending = mine.size();
  while (pending > 0) {
    // replies first: they free the server's buffers
    for (int q = 0; q < kB; ++q) {
      riov[q] = {rb.data() + (size_t)q * kRep, kRep};
      memset(&rh[q], 0, sizeof(mmsghdr));
      rh[q].msg_hdr.msg_iov = &riov[q];
      rh[q].msg_hdr.msg_iovlen = 1;
    }
    const int got = recvmmsg(fd, rh.data(), kB, MSG_DONTWAIT, nullptr);
    uint64_t now = genesys_mono_ns();
    for (int q = 0; q < got; ++q) {
      const uint8_t *r = rb.data() + (size_t)q * kRep;
      const uint32_t len = rh[q].msg_len;
      uint32_t seq = ~0u;
      if (len >= 8) memcpy(&seq, r + 4, 4);
      if (len < 8 || seq >= n || t_send[seq] == 0) { ++T.bad; continue; }
      if (reply_len[seq]) { ++T.dup; continue; }
      memcpy(replies + (size_t)seq * kRep, r, len);
      reply_len[seq] = len;
      latency_ns[seq] = now - t_send[seq];
      ++T.received;
      --pending;
    }
    // then every request that is due
    int m = 0;
    while (m < kB && i + m < mine.size() && t0 + arrival_ns[mine[i + m]] <= now) {
      const uint64_t j = mine[i + m];
      const uint8_t *q = reqs + req_off[j];
      uint32_t k0;
      memcpy(&k0, q + 8, 4);
      to[m] = sockaddr_in{};
      to[m].sin_family = AF_INET;
      to[m].sin_port = htons((uint16_t)(port_base + k0 % n_sockets));
      to[m].sin_addr.s_addr = htonl(INADDR_LOOPBACK);
      siov[m] = {(void *)q, (size_t)(req_off[j + 1] - req_off[j])};
      memset(&sh[m], 0, sizeof(mmsghdr));
      sh[m].msg_hdr.msg_name = &to[m];
      sh[m].msg_hdr.msg_namelen = sizeof(sockaddr_in);
      sh[m].msg_hdr.msg_iov = &siov[m];
      sh[m].msg_hdr.msg_iovlen = 1;
      T.late_max = std::max(T.late_max, now - (t0 + arrival_ns[j]));
      t_send[j] = now;
      ++m;
    }
    int sent = 0;
    while (sent < m) {
      const int r = sendmmsg(fd, sh.data() + sent, m - sent, 0);
      if (r <= 0) {
        T.send_err += m - sent;
        pending -= m - sent;
        break;
      }
      sent += r;
    }
    i += m;
    if (got <= 0 && m == 0) {
      if (now > deadline) { T.timed_out = true; break; }
      __builtin_ia32_pause();
    }
  }
  *out = T;
}

}  // namespace

extern "C" int genesys_kv_client(const uint8_t *reqs, const uint64_t *req_off, uint64_t n, const uint64_t *arrival_ns,
                                 uint16_t port_base, uint32_t n_sockets, uint64_t timeout_ns, uint8_t *replies,
                                 uint32_t *reply_len, uint64_t *latency_ns, uint64_t *stats) {
  return genesys_guard("genesys_kv_client", [&]() -> int {
    if (!reqs || !req_off || !arrival_ns || !replies || !reply_len || !latency_ns || n_sockets == 0)
      return set_err(GENESYS_EINVAL, "NULL argument");
    // one thread per CPU the caller may run on (it restricts the generator to
    // its share of the host's cores that way), at most 8, at most one per socket
    cpu_set_t allowed;
    uint32_t cpus = 1;
    if (sched_getaffinity(0, sizeof allowed, &allowed) == 0) cpus = std::max(1, CPU_COUNT(&allowed));
    const uint32_t n_threads = std::min<uint32_t>(std::min<uint32_t>(n_sockets, 8), cpus);
    std::vector<uint64_t> t_send(n, 0);  // before any socket is opened: this may throw
    std::vector<int> fds;
    for (uint32_t w = 0; w < n_threads; ++w) {
      int fd = socket(AF_INET, SOCK_DGRAM, 0);
      if (fd < 0) break;
      int want = 64 << 20;
      if (setsockopt(fd, SOL_SOCKET, SO_RCVBUFFORCE, &want, sizeof want) != 0)
        setsockopt(fd, SOL_SOCKET, SO_RCVBUF, &want, sizeof want);
      if (setsockopt(fd, SOL_SOCKET, SO_SNDBUFFORCE, &want, sizeof want) != 0)
        setsockopt(fd, SOL_SOCKET, SO_SNDBUF, &want, sizeof want);
      sockaddr_in me{};
      me.sin_family = AF_INET;
      me.sin_addr.s_addr = htonl(INADDR_LOOPBACK);
      if (bind(fd, (sockaddr *)&me, sizeof me) != 0) { close(fd); break; }
      fds.push_back(fd);
    }
    if (fds.size() != n_threads) {
      for (int fd : fds) close(fd);
      return set_err(GENESYS_EINVAL, "client socket or bind failed");
    }
    memset(reply_len, 0, sizeof(uint32_t) * n);
    std::vector<std::vector<uint64_t>> owned(n_threads);
    for (uint64_t j = 0; j < n; ++j) {
      uint32_t k0;
      memcpy(&k0, reqs + req_off[j] + 8, 4);
      owned[(k0 % n_sockets) % n_threads].push_back(j);
    }
    std::vector<KvClientTally> tally(n_threads);
    const uint64_t t0 = genesys_mono_ns() + 2000000;  // start in 2 ms, once the threads run
    const uint64_t deadline = t0 + (n ? arrival_ns[n - 1] : 0) + timeout_ns;
    std::vector<std::thread> th;
    genesys_joiner join_all{th};
    for (uint32_t w = 0; w < n_threads; ++w)
      th.emplace_back(kv_client_thread, fds[w], std::cref(owned[w]), reqs, req_off, n, arrival_ns, t0, port_base,
                      n_sockets, deadline, replies, reply_len, latency_ns, t_send.data(), &tally[w]);
    for (auto &t : th) t.join();
    // STOP to every socket (no reply)
    for (uint32_t w = 0; w < n_sockets; ++w) {
      uint8_t stop[24] = {GENESYS_KV_STOP};
      sockaddr_in to{};
      to.sin_family = AF_INET;
      to.sin_port = htons((uint16_t)(port_base + w));
      to.sin_addr.s_addr = htonl(INADDR_LOOPBACK);
      sendto(fds[0], stop, sizeof stop, 0, (sockaddr *)&to, sizeof to);
    }
    for (int fd : fds) close(fd);
    KvClientTally S;
    for (auto &T : tally) {
      S.received += T.received;
      S.dup += T.dup;
      S.bad += T.bad;
      S.send_err += T.send_err;
      S.late_max = std::max(S.late_max, T.late_max);
      S.timed_out |= T.timed_out;
    }
    if (stats) {
      stats[0] = S.received;
      stats[1] = S.dup;
      stats[2] = S.bad;
      stats[3] = S.send_err;
      stats[4] = S.late_max;
      uint64_t first = ~0ull, last = 0;
      for (uint64_t j = 0; j < n; ++j) {
        if (!reply_len[j]) continue;
        first = std::min(first, t_send[j]);
        last = std::max(last, t_send[j] + latency_ns[j]);
      }
      stats[5] = last > first ? last - first : 0;  // first send to last reply
    }
    if (S.timed_out) return set_err(GENESYS_ETIMEDOUT, "kv client: replies missing at the deadline");
    return 0;
  });
}
