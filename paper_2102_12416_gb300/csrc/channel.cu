// Intra-device channels between two blocks (Sec. 3.2.2, Channel API; tag
// scheme of Sec. 3.1).
//
// The paper's channel pairs two chares under a program-unique id and matches
// each send with a receive through a 64-bit UCX tag whose low 32 bits are a
// counter kept by each endpoint and bumped on every send or receive, so no
// host-side metadata message is needed.  Here both endpoints live on one GPU:
// a send copies the payload into the peer's preallocated receive slot and
// publishes the message's sequence number with a release store; a receive
// acquire-waits (bounded) for that number, copies the payload out (or leaves
// it in place) and publishes "consumed".  The per-endpoint host counters play
// the role of the tag counters: message n of a direction always uses slot
// parity n & 1 and sequence number n + 1, so messages match in order and
// exactly once.
//
// A receive posted before its send (in host program order) with a
// destination buffer is the Channel API's expected message: the receive only
// registers the buffer, and the matching send copies the payload straight
// into it in one launch, without the slot.  A zero-copy receive leaves the
// message in its slot and holds the slot until the next receive at that
// endpoint or channel_release, so the sender cannot overwrite it while the
// receiver still reads it.
#include <cstdlib>
#include <cstring>
#include <deque>

#include "runtime.h"

using namespace jgb;

// Device counters of one channel (one 256-byte block).
struct ChanCtr {
  uint32_t delivered[2];  // messages delivered to endpoint e (seq of the last one)
  uint32_t consumed[2];   // messages endpoint e has consumed
  uint32_t done[2];       // copy CTAs finished for the message in flight to e
  uint32_t err;
  uint32_t pad0;
  uint64_t size[2][2];    // payload size of the message in slot [e][parity]
  uint32_t pp_arrive[2];  // ping-pong: CTA arrivals for messages to endpoint e
  uint32_t rdone[2];      // copy-out CTAs finished for the receive in flight at e
  uint32_t bw_arrive[2];  // bandwidth test: CTA arrivals of windows sent to endpoint e
  uint32_t bw_ack[2];     // bandwidth test: CTA arrivals of acknowledgements to e
};

// Host-side metadata message of the GPU Messaging form.
struct MsgMeta {
  const void* src;
  size_t bytes;
  uint64_t seq;
};

struct channel_s {
  jacobi_t* h = nullptr;
  uint32_t id = 0;
  int64_t block[2] = {-1, -1};
  size_t max_bytes = 0;
  char* mem = nullptr;     // slots + counters (library-owned)
  void* slot[2][2] = {};   // [endpoint][parity]
  ChanCtr* ctr = nullptr;
  uint32_t* h_err = nullptr;
  uint64_t sent[2] = {0, 0};   // device-channel messages sent BY endpoint e
  uint64_t recvd[2] = {0, 0};  // device-channel messages received BY endpoint e
                               // (the host-staged and Messaging forms keep out of these)
  bool held[2] = {false, false};  // endpoint e holds its last message in the slot (zero-copy)
  struct Posted {                 // receive posted before its send: payload goes straight to dst
    uint64_t n;
    void* dst;
    size_t bytes;
  };
  std::deque<Posted> posted[2];   // per receiving endpoint, in message order
  // the last message delivered straight into a posted receive at endpoint e,
  // and the stream its send was issued on (-1: none yet)
  int64_t direct_n[2] = {-1, -1};
  void* direct_stream[2] = {nullptr, nullptr};
  void* hstage[2] = {nullptr, nullptr};  // pinned host staging of the host-staged form, per receiver
  std::deque<MsgMeta> mailbox[2];        // metadata messages waiting at endpoint e
  uint64_t msg_seq[2] = {0, 0};
};

namespace {

constexpr int kChanThreads = 256;

__device__ __forceinline__ void copy16(void* __restrict__ dst, const void* __restrict__ src, size_t bytes, size_t tid,
                                       size_t nthreads) {
  // bytes is a multiple of 16 for the vector part; the tail is copied bytewise.
  const size_t nv = bytes / 16;
  const uint4* s4 = (const uint4*)src;
  uint4* d4 = (uint4*)dst;
  for (size_t q = tid; q < nv; q += nthreads) d4[q] = __ldcg(s4 + q);
  const unsigned char* s1 = (const unsigned char*)src;
  unsigned char* d1 = (unsigned char*)dst;
  for (size_t q = nv * 16 + tid; q < bytes; q += nthreads) d1[q] = s1[q];
}

// Send message n (0-based) from endpoint `from` to endpoint `to`.
__global__ void k_chan_send(ChanCtr* c, int to, uint32_t n, const void* src, void* slot, size_t bytes,
                            uint64_t wait_ns) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    // The slot of parity n & 1 is free once message n - 2 has been consumed.
    ok = (n < 2) ? 1 : (wait_seq_ge(&c->consumed[to], n - 1, &c->err, wait_ns) ? 1 : 0);
  }
  __syncthreads();
  if (!ok) return;
  copy16(slot, src, bytes, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(&c->done[to], 1u);
    if (prev == gridDim.x - 1) {  // last CTA: publish the message
      c->done[to] = 0;
      c->size[to][n & 1] = bytes;
      __threadfence();
      st_release_u32(&c->delivered[to], n + 1);
    }
  }
}

// Send message n straight into the receiver's pre-posted buffer: wait until
// every earlier message to that endpoint has been consumed (so "consumed"
// stays in order), copy, then publish the message as delivered and consumed
// (it never occupies a slot).
// With ordered set the host has shown that message n - 1 was itself delivered
// straight into a posted receive by a send earlier on the same stream, which
// published consumed = n before this launch: the poll is skipped.
__global__ void k_chan_send_direct(ChanCtr* c, int to, uint32_t n, const void* src, void* dst, size_t bytes,
                                   uint64_t wait_ns, int ordered) {
  __shared__ int ok;
  if (threadIdx.x == 0)
    ok = (n < 1 || ordered) ? 1 : (wait_seq_ge(&c->consumed[to], n, &c->err, wait_ns) ? 1 : 0);
  __syncthreads();
  if (!ok) return;
  copy16(dst, src, bytes, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    // one CTA: its barrier already orders every copy before the release
    // store; several: the last CTA to finish publishes
    bool last = gridDim.x == 1;
    if (!last) {
      __threadfence();
      last = atomicAdd(&c->done[to], 1u) == gridDim.x - 1;
      if (last) {
        c->done[to] = 0;
        __threadfence();
      }
    }
    if (last) {
      st_release_u32(&c->delivered[to], n + 1);
      st_release_u32(&c->consumed[to], n + 1);
    }
  }
}

// Release a slot held by a zero-copy receive: consumed[at] = value.
__global__ void k_chan_release(ChanCtr* c, int at, uint32_t value) { st_release_u32(&c->consumed[at], value); }

// Receive message n at endpoint `at` (dst may be null: zero-copy).  release
// > 0 first publishes consumed = release for the message this endpoint held;
// with hold set the message stays in its slot (consumed is not published).
__global__ void k_chan_recv(ChanCtr* c, int at, uint32_t n, void* dst, const void* slot, size_t bytes,
                            uint64_t wait_ns, uint32_t* done_ctr, uint32_t release, int hold) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    if (release && blockIdx.x == 0) st_release_u32(&c->consumed[at], release);
    int good = wait_seq_ge(&c->delivered[at], n + 1, &c->err, wait_ns) ? 1 : 0;
    if (good && c->size[at][n & 1] != bytes) {
      atomicCAS(&c->err, (uint32_t)DEV_OK, (uint32_t)DEV_SEQ);
      good = 0;
    }
    ok = good;
  }
  __syncthreads();
  if (!ok) return;
  if (dst) copy16(dst, slot, bytes, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(done_ctr, 1u);
    if (prev == gridDim.x - 1) {
      *done_ctr = 0;
      __threadfence();
      if (!hold) st_release_u32(&c->consumed[at], n + 1);
    }
  }
}

// OSU-style ping-pong (Sec. 4.2.1) inside one cooperative launch.  CTAs
// [0, G) are endpoint 0, [G, 2G) endpoint 1.  Round r: endpoint 0 copies
// `bytes` from its source buffer into endpoint 1's slot; each of its CTAs
// then bumps pp_arrive[1]; endpoint 1 waits until pp_arrive[1] == G*(r+1),
// then replies the same way.  All waits are bounded.
__global__ void k_pingpong(ChanCtr* c, void* slot0, void* slot1, const void* src0, const void* src1, size_t bytes,
                           int64_t rounds, int G, uint64_t wait_ns) {
  const int side = blockIdx.x < (unsigned)G ? 0 : 1;
  const int cta = side == 0 ? blockIdx.x : blockIdx.x - G;
  const size_t tid = (size_t)cta * blockDim.x + threadIdx.x, nthr = (size_t)G * blockDim.x;
  __shared__ int ok;
  for (int64_t r = 0; r < rounds; ++r) {
    // endpoint 0 sends, endpoint 1 receives; then the reverse.
    for (int leg = 0; leg < 2; ++leg) {
      const int sender = leg;  // leg 0: 0 -> 1, leg 1: 1 -> 0
      const int to = 1 - sender;
      if (side == sender) {
        copy16(to == 1 ? slot1 : slot0, sender == 0 ? src0 : src1, bytes, tid, nthr);
        __syncthreads();
        if (threadIdx.x == 0) {
          __threadfence();
          atomicAdd(&c->pp_arrive[to], 1u);
        }
      } else {
        if (threadIdx.x == 0) {
          const uint32_t target = (uint32_t)G * (uint32_t)(r + 1);
          ok = wait_seq_ge(&c->pp_arrive[side], target, &c->err, wait_ns) ? 1 : 0;
        }
        __syncthreads();
        if (!ok) return;
      }
    }
  }
}

// Plain multi-CTA device copy (the data movement of the GPU Messaging form).
__global__ void k_msg_copy(void* dst, const void* src, size_t bytes) {
  copy16(dst, src, bytes, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

// OSU-style bandwidth test (Sec. 4.2.2) inside one cooperative launch.  CTAs
// [0, G) are endpoint 0, [G, 2G) endpoint 1.  Each iteration the sender copies
// `window` messages of `bytes` back to back into the peer's slot, then each of
// its CTAs bumps the peer's arrival counter; the receiver waits for G arrivals
// per iteration and (one-directional form) acknowledges with its own G
// arrivals, which the sender waits for before the next window.  With
// bidirectional set both endpoints send a window each iteration and the
// arrivals double as acknowledgements.  All waits are bounded.
__global__ void k_bandwidth(ChanCtr* c, void* slot0, void* slot1, const void* src0, const void* src1, size_t bytes,
                            int window, int64_t iters, int G, int bidir, uint64_t wait_ns) {
  const int side = blockIdx.x < (unsigned)G ? 0 : 1;
  const int peer = 1 - side;
  const int cta = side == 0 ? blockIdx.x : blockIdx.x - G;
  const size_t tid = (size_t)cta * blockDim.x + threadIdx.x, nthr = (size_t)G * blockDim.x;
  __shared__ int ok;
  for (int64_t it = 0; it < iters; ++it) {
    const uint32_t target = (uint32_t)G * (uint32_t)(it + 1);
    if (side == 0 || bidir) {
      for (int w = 0; w < window; ++w) copy16(peer == 1 ? slot1 : slot0, side == 0 ? src0 : src1, bytes, tid, nthr);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&c->bw_arrive[peer], 1u);
      }
    }
    if (side == 1 || bidir) {
      if (threadIdx.x == 0) ok = wait_seq_ge(&c->bw_arrive[side], target, &c->err, wait_ns) ? 1 : 0;
      __syncthreads();
      if (!ok) return;
    }
    if (!bidir) {
      if (side == 1) {
        if (threadIdx.x == 0) {
          __threadfence();
          atomicAdd(&c->bw_ack[0], 1u);
        }
      } else {
        if (threadIdx.x == 0) ok = wait_seq_ge(&c->bw_ack[0], target, &c->err, wait_ns) ? 1 : 0;
        __syncthreads();
        if (!ok) return;
      }
    }
  }
}

cudaStream_t S(void* s) { return (cudaStream_t)s; }

int endpoint_of(const channel_s* ch, int64_t block) {
  if (block == ch->block[0]) return 0;
  if (block == ch->block[1]) return 1;
  return -1;
}

int copy_ctas(size_t bytes) {
  const size_t per = (size_t)kChanThreads * 16 * 4;  // ~16 KB per CTA
  size_t n = (bytes + per - 1) / per;
  if (n < 1) n = 1;
  if (n > 1024) n = 1024;
  return (int)n;
}

}  // namespace

extern "C" {

int channel_open(jacobi_t* h, uint32_t channel_id, int64_t block_a, int64_t block_b, size_t max_bytes,
                 channel_t** out) {
  if (!h || !out) return set_error(JACOBI_EINVAL, "null argument");
  *out = nullptr;
  const int64_t nb = (int64_t)h->plan.blocks.size();
  if (block_a < 0 || block_a >= nb || block_b < 0 || block_b >= nb || block_a == block_b)
    return set_error(JACOBI_EINVAL, "channel endpoints must be two distinct blocks of the handle");
  if (max_bytes == 0 || max_bytes > ((size_t)1 << 34)) return set_error(JACOBI_EINVAL, "bad max_bytes");
  for (channel_s* c : h->channels)
    if (c->id == channel_id) return set_error(JACOBI_EINVAL, "channel id %u already open", channel_id);
  channel_s* ch = new (std::nothrow) channel_s();
  if (!ch) return set_error(JACOBI_ENOMEM, "host allocation failed");
  ch->h = h;
  ch->id = channel_id;
  ch->block[0] = block_a;
  ch->block[1] = block_b;
  ch->max_bytes = max_bytes;
  const size_t sb = align_up(max_bytes, 256);
  const size_t total = 4 * sb + 256;
  if (cudaMalloc((void**)&ch->mem, total) != cudaSuccess || cudaMallocHost((void**)&ch->h_err, 64) != cudaSuccess) {
    if (ch->mem) cudaFree(ch->mem);
    delete ch;
    return set_error(JACOBI_ENOMEM, "channel allocation of %zu bytes failed", total);
  }
  for (int e = 0; e < 2; ++e)
    for (int p = 0; p < 2; ++p) ch->slot[e][p] = ch->mem + (2 * e + p) * sb;
  ch->ctr = (ChanCtr*)(ch->mem + 4 * sb);
  cudaError_t e = cudaMemset(ch->mem, 0, total);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(ch->mem);
    cudaFreeHost(ch->h_err);
    delete ch;
    return set_error(JACOBI_ECUDA, "channel init failed: %s", cudaGetErrorString(e));
  }
  h->channels.push_back(ch);
  *out = ch;
  return JACOBI_OK;
}

int channel_send(channel_t* ch, int64_t from_block, const void* src, size_t bytes, void* stream) {
  if (!ch || !src) return set_error(JACOBI_EINVAL, "null argument");
  const int from = endpoint_of(ch, from_block);
  if (from < 0) return set_error(JACOBI_EINVAL, "block %lld is not an endpoint of channel %u", (long long)from_block, ch->id);
  if (bytes > ch->max_bytes) return set_error(JACOBI_EINVAL, "message of %zu bytes exceeds max_bytes", bytes);
  if ((uintptr_t)src % 16) return set_error(JACOBI_EINVAL, "src must be 16-byte aligned");
  const int to = 1 - from;
  const uint32_t n = (uint32_t)ch->sent[from];
  if (!ch->posted[to].empty() && ch->posted[to].front().n == ch->sent[from]) {
    const channel_s::Posted pr = ch->posted[to].front();
    if (pr.bytes != bytes)
      return set_error(JACOBI_ESEQ, "channel %u: message %llu has %zu bytes, the posted receive expects %zu", ch->id,
                       (unsigned long long)pr.n, bytes, pr.bytes);
    const int ordered = ch->direct_n[to] + 1 == (int64_t)ch->sent[from] && ch->direct_stream[to] == stream;
    k_chan_send_direct<<<copy_ctas(bytes), kChanThreads, 0, S(stream)>>>(ch->ctr, to, n, src, pr.dst, bytes,
                                                                         ch->h->wait_ns, ordered);
    JGB_CUDA(cudaGetLastError());
    ch->posted[to].pop_front();
    ch->direct_n[to] = (int64_t)ch->sent[from];
    ch->direct_stream[to] = stream;
  } else {
    k_chan_send<<<copy_ctas(bytes), kChanThreads, 0, S(stream)>>>(ch->ctr, to, n, src, ch->slot[to][n & 1], bytes,
                                                                    ch->h->wait_ns);
    JGB_CUDA(cudaGetLastError());
  }
  ch->sent[from] += 1;
  return JACOBI_OK;
}

int channel_recv(channel_t* ch, int64_t at_block, void* dst, size_t bytes, void* stream) {
  if (!ch) return set_error(JACOBI_EINVAL, "null channel");
  const int at = endpoint_of(ch, at_block);
  if (at < 0) return set_error(JACOBI_EINVAL, "block %lld is not an endpoint of channel %u", (long long)at_block, ch->id);
  if (bytes > ch->max_bytes) return set_error(JACOBI_EINVAL, "message of %zu bytes exceeds max_bytes", bytes);
  if (dst && (uintptr_t)dst % 16) return set_error(JACOBI_EINVAL, "dst must be 16-byte aligned");
  const uint32_t n = (uint32_t)ch->recvd[at];
  const uint32_t release = ch->held[at] ? n : 0u;  // the held message is n - 1: consumed = n
  if (dst && ch->recvd[at] >= ch->sent[1 - at]) {
    // posted before its send: the send will deliver straight into dst
    if (release) {
      k_chan_release<<<1, 1, 0, S(stream)>>>(ch->ctr, at, release);
      JGB_CUDA(cudaGetLastError());
    }
    ch->posted[at].push_back(channel_s::Posted{ch->recvd[at], dst, bytes});
  } else {
    const int ctas = dst ? copy_ctas(bytes) : 1;
    k_chan_recv<<<ctas, kChanThreads, 0, S(stream)>>>(ch->ctr, at, n, dst, ch->slot[at][n & 1], bytes,
                                                      ch->h->wait_ns, &ch->ctr->rdone[at], release, dst ? 0 : 1);
    JGB_CUDA(cudaGetLastError());
  }
  ch->held[at] = dst == nullptr;
  ch->recvd[at] += 1;
  return JACOBI_OK;
}

int channel_release(channel_t* ch, int64_t at_block, void* stream) {
  if (!ch) return set_error(JACOBI_EINVAL, "null channel");
  const int at = endpoint_of(ch, at_block);
  if (at < 0) return set_error(JACOBI_EINVAL, "block %lld is not an endpoint of channel %u", (long long)at_block, ch->id);
  if (!ch->held[at]) return JACOBI_OK;
  k_chan_release<<<1, 1, 0, S(stream)>>>(ch->ctr, at, (uint32_t)ch->recvd[at]);
  JGB_CUDA(cudaGetLastError());
  ch->held[at] = false;
  return JACOBI_OK;
}

int channel_slot(channel_t* ch, int64_t at_block, int32_t parity, void** slot) {
  if (!ch || !slot || (parity != 0 && parity != 1)) return set_error(JACOBI_EINVAL, "bad arguments");
  const int at = endpoint_of(ch, at_block);
  if (at < 0) return set_error(JACOBI_EINVAL, "block is not an endpoint of the channel");
  *slot = ch->slot[at][parity];
  return JACOBI_OK;
}

int channel_sync(channel_t* ch, void* stream) {
  if (!ch) return set_error(JACOBI_EINVAL, "null channel");
  JGB_CUDA(cudaStreamSynchronize(S(stream)));
  JGB_CUDA(cudaMemcpy(ch->h_err, &ch->ctr->err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  const uint32_t e = *ch->h_err;
  if (e == DEV_OK) {
    for (int at = 0; at < 2; ++at)
      if (!ch->posted[at].empty())
        return set_error(JACOBI_EAGAIN, "channel %u: a receive posted at block %lld still waits for its send", ch->id,
                         (long long)ch->block[at]);
    return JACOBI_OK;
  }
  JGB_CUDA(cudaMemset(&ch->ctr->err, 0, sizeof(uint32_t)));
  if (e == DEV_TIMEOUT) return set_error(JACOBI_ETIMEDOUT, "channel %u: a device-side wait timed out", ch->id);
  return set_error(JACOBI_ESEQ, "channel %u: message size or sequence mismatch", ch->id);
}

int channel_pingpong(channel_t* ch, size_t bytes, int64_t round_trips, int32_t ctas_per_side, void* stream) {
  if (!ch || round_trips < 0 || ctas_per_side < 1) return set_error(JACOBI_EINVAL, "bad arguments");
  if (bytes > ch->max_bytes) return set_error(JACOBI_EINVAL, "message exceeds max_bytes");
  int dev = 0, sms = 0, per_sm = 0;
  JGB_CUDA(cudaGetDevice(&dev));
  JGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  JGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pingpong, kChanThreads, 0));
  if (2 * ctas_per_side > per_sm * sms) return set_error(JACOBI_EINVAL, "too many CTAs for a co-resident launch");
  const cudaStream_t s = S(stream);
  JGB_CUDA(cudaMemsetAsync(ch->ctr->pp_arrive, 0, sizeof(ch->ctr->pp_arrive), s));
  // Each side sends from its own parity-1 slot into the peer's parity-0 slot.
  void* slot0 = ch->slot[0][0];
  void* slot1 = ch->slot[1][0];
  const void* src0 = ch->slot[0][1];
  const void* src1 = ch->slot[1][1];
  ChanCtr* c = ch->ctr;
  int G = ctas_per_side;
  uint64_t wn = ch->h->wait_ns;
  void* args[] = {&c, &slot0, &slot1, (void*)&src0, (void*)&src1, &bytes, &round_trips, &G, &wn};
  JGB_CUDA(cudaLaunchCooperativeKernel((const void*)k_pingpong, dim3(2 * G), dim3(kChanThreads), args, 0, s));
  return JACOBI_OK;
}

int channel_send_host(channel_t* ch, int64_t from_block, const void* src, size_t bytes, void* stream) {
  if (!ch || !src) return set_error(JACOBI_EINVAL, "null argument");
  const int from = endpoint_of(ch, from_block);
  if (from < 0) return set_error(JACOBI_EINVAL, "block is not an endpoint of the channel");
  if (bytes > ch->max_bytes) return set_error(JACOBI_EINVAL, "message exceeds max_bytes");
  const int to = 1 - from;
  if (!ch->hstage[to]) JGB_CUDA(cudaMallocHost(&ch->hstage[to], ch->max_bytes));
  // Device -> host into the staging buffer, then wait: only then may the host
  // hand the message on.
  JGB_CUDA(cudaMemcpyAsync(ch->hstage[to], src, bytes, cudaMemcpyDeviceToHost, S(stream)));
  JGB_CUDA(cudaStreamSynchronize(S(stream)));
  return JACOBI_OK;
}

int channel_recv_host(channel_t* ch, int64_t at_block, void* dst, size_t bytes, void* stream) {
  if (!ch || !dst) return set_error(JACOBI_EINVAL, "null argument");
  const int at = endpoint_of(ch, at_block);
  if (at < 0) return set_error(JACOBI_EINVAL, "block is not an endpoint of the channel");
  if (bytes > ch->max_bytes || !ch->hstage[at]) return set_error(JACOBI_EINVAL, "no host-staged message");
  JGB_CUDA(cudaMemcpyAsync(dst, ch->hstage[at], bytes, cudaMemcpyHostToDevice, S(stream)));
  JGB_CUDA(cudaStreamSynchronize(S(stream)));
  return JACOBI_OK;
}

int channel_send_msg(channel_t* ch, int64_t from_block, const void* src, size_t bytes, void* stream) {
  (void)stream;
  if (!ch || !src) return set_error(JACOBI_EINVAL, "null argument");
  const int from = endpoint_of(ch, from_block);
  if (from < 0) return set_error(JACOBI_EINVAL, "block is not an endpoint of the channel");
  if (bytes > ch->max_bytes) return set_error(JACOBI_EINVAL, "message exceeds max_bytes");
  const int to = 1 - from;
  ch->mailbox[to].push_back(MsgMeta{src, bytes, ch->msg_seq[to]++});
  return JACOBI_OK;
}

int channel_recv_msg(channel_t* ch, int64_t at_block, void* dst, size_t bytes, void* stream) {
  if (!ch || !dst) return set_error(JACOBI_EINVAL, "null argument");
  const int at = endpoint_of(ch, at_block);
  if (at < 0) return set_error(JACOBI_EINVAL, "block is not an endpoint of the channel");
  if (ch->mailbox[at].empty()) return set_error(JACOBI_EAGAIN, "no metadata message has arrived yet");
  const MsgMeta m = ch->mailbox[at].front();
  if (m.bytes != bytes) return set_error(JACOBI_ESEQ, "message %llu has %zu bytes, receive expects %zu",
                                         (unsigned long long)m.seq, m.bytes, bytes);
  if ((uintptr_t)dst % 16 || (uintptr_t)m.src % 16) return set_error(JACOBI_EINVAL, "buffers must be 16-byte aligned");
  ch->mailbox[at].pop_front();
  // The receive is posted only now that the metadata is here: issue the copy
  // and wait for its completion.
  k_msg_copy<<<copy_ctas(bytes), kChanThreads, 0, S(stream)>>>(dst, m.src, bytes);
  JGB_CUDA(cudaGetLastError());
  JGB_CUDA(cudaStreamSynchronize(S(stream)));
  return JACOBI_OK;
}

int channel_bandwidth(channel_t* ch, size_t bytes, int32_t window, int64_t iterations, int32_t ctas_per_side,
                      int32_t bidirectional, void* stream) {
  if (!ch || window < 1 || iterations < 0 || ctas_per_side < 1) return set_error(JACOBI_EINVAL, "bad arguments");
  if (bytes > ch->max_bytes) return set_error(JACOBI_EINVAL, "message exceeds max_bytes");
  int dev = 0, sms = 0, per_sm = 0;
  JGB_CUDA(cudaGetDevice(&dev));
  JGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  JGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bandwidth, kChanThreads, 0));
  if (2 * ctas_per_side > per_sm * sms) return set_error(JACOBI_EINVAL, "too many CTAs for a co-resident launch");
  const cudaStream_t s = S(stream);
  JGB_CUDA(cudaMemsetAsync(ch->ctr->bw_arrive, 0, sizeof(ch->ctr->bw_arrive) + sizeof(ch->ctr->bw_ack), s));
  void* slot0 = ch->slot[0][0];
  void* slot1 = ch->slot[1][0];
  const void* src0 = ch->slot[0][1];
  const void* src1 = ch->slot[1][1];
  ChanCtr* c = ch->ctr;
  int G = ctas_per_side, W = window, bidir = bidirectional ? 1 : 0;
  uint64_t wn = ch->h->wait_ns;
  void* args[] = {&c, &slot0, &slot1, (void*)&src0, (void*)&src1, &bytes, &W, &iterations, &G, &bidir, &wn};
  JGB_CUDA(cudaLaunchCooperativeKernel((const void*)k_bandwidth, dim3(2 * G), dim3(kChanThreads), args, 0, s));
  return JACOBI_OK;
}

int channel_close(channel_t* ch) {
  if (!ch) return JACOBI_OK;
  cudaDeviceSynchronize();
  for (int e = 0; e < 2; ++e)
    if (ch->hstage[e]) cudaFreeHost(ch->hstage[e]);
  jacobi_t* h = ch->h;
  for (size_t q = 0; q < h->channels.size(); ++q)
    if (h->channels[q] == ch) {
      h->channels.erase(h->channels.begin() + q);
      break;
    }
  cudaFree(ch->mem);
  cudaFreeHost(ch->h_err);
  delete ch;
  return JACOBI_OK;
}

}  // extern "C"
