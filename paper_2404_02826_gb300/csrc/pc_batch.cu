// Many snapshots on one GPU: batched compression / decompression and a
// serving loop.  Host code only; every item runs the same kernels as a plain
// call (pc_api.cu), on one of several CUDA streams.
//
// Lanes.  A lane is a host thread with its own CUDA stream and its own slice
// of device scratch.  Compression reads a few bytes back twice per snapshot
// (the value range, then the final size), and small snapshots are dominated by
// launch and read-back latency; with several lanes those latencies overlap and
// the kernels of different snapshots share the GPU.
//
// Server.  Requests queue in arrival order.  A free lane admits the oldest one
// when a first-fit allocator over the caller's arena can hold its scratch and
// its output; scratch is returned when the request completes, the output when
// the caller releases it.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "pc_internal.cuh"

namespace {

constexpr uint64_t kArenaAlign = 256;

uint64_t align_up(uint64_t x) { return (x + kArenaAlign - 1) / kArenaAlign * kArenaAlign; }

uint32_t pick_lanes(uint32_t lanes, uint32_t count) {
  if (lanes == 0) lanes = 8;
  if (lanes > count) lanes = count;
  return lanes ? lanes : 1;
}

uint64_t compress_scratch(uint64_t n, int dtype, uint32_t leaf_size, uint32_t flags, uint64_t *bytes) {
  pc_config cfg = {leaf_size, flags};
  return uint64_t(pc_compress_workspace_size(n, dtype, &cfg, 0, bytes));
}

// Runs fn(lane, stream, item) for every item over `lanes` host threads, items
// in the given order; the lane streams start after the work already queued on
// `caller` and the call returns when every item is done.
template <typename Fn>
int run_lanes(uint32_t lanes, const std::vector<uint32_t> &order, cudaStream_t caller, Fn fn) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PC_ERR_CUDA;
  cudaEvent_t start;
  if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) return PC_ERR_CUDA;
  if (cudaEventRecord(start, caller) != cudaSuccess) {
    cudaEventDestroy(start);
    return PC_ERR_CUDA;
  }
  std::atomic<uint32_t> next{0};
  std::atomic<int> cuda_fail{0};
  auto worker = [&](uint32_t lane) {
    if (cudaSetDevice(dev) != cudaSuccess) {
      cuda_fail = 1;
      return;
    }
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cuda_fail = 1;
      return;
    }
    cudaStreamWaitEvent(s, start, 0);
    for (;;) {
      const uint32_t k = next.fetch_add(1);
      if (k >= order.size()) break;
      fn(lane, s, order[k]);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) cuda_fail = 1;
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> threads;
  for (uint32_t l = 1; l < lanes; ++l) threads.emplace_back(worker, l);
  worker(0);
  for (auto &t : threads) t.join();
  cudaEventDestroy(start);
  return cuda_fail ? PC_ERR_CUDA : PC_OK;
}

double now_seconds() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) in kArenaAlign units.
class Arena {
 public:
  explicit Arena(uint64_t size) : size_(size / kArenaAlign * kArenaAlign) {
    if (size_) free_[0] = size_;
  }
  bool alloc(uint64_t bytes, uint64_t *off) {
    bytes = align_up(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const uint64_t rest = it->second - bytes;
        const uint64_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_[*off] = bytes;
        in_use_ += bytes;
        return true;
      }
    }
    return false;
  }
  bool release(uint64_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return false;
    uint64_t start = off, len = u->second;
    in_use_ -= len;
    used_.erase(u);
    auto nx = free_.lower_bound(start);
    if (nx != free_.end() && start + len == nx->first) {
      len += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == start) {
        start = pv->first;
        len += pv->second;
        free_.erase(pv);
      }
    }
    free_[start] = len;
    return true;
  }
  uint64_t size() const { return size_; }
  uint64_t in_use() const { return in_use_; }

 private:
  uint64_t size_;
  uint64_t in_use_ = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> length
  std::map<uint64_t, uint64_t> used_;  // offset -> length
};

}  // namespace

struct pc_server {
  struct Job {
    pc_request req;
    double t_submit;
  };
  uint8_t *base = nullptr;
  Arena arena;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // lanes wait for admissible work
  std::condition_variable cv_done;  // pollers wait for completions
  std::deque<Job> queue;
  std::deque<pc_completion> done;
  uint32_t running = 0;
  bool stopping = false;
  std::vector<std::thread> lanes;

  pc_server(void *a, uint64_t bytes) : base(static_cast<uint8_t *>(a)), arena(bytes) {}

  // Whether scratch and output would fit the arena now (tries, then gives back).
  bool fits(uint64_t sbytes, uint64_t obytes) {
    uint64_t a = 0, b = 0;
    if (!arena.alloc(obytes, &a)) return false;
    const bool ok = arena.alloc(sbytes, &b);
    if (ok) arena.release(b);
    arena.release(a);
    return ok;
  }

  // Arena bytes a request needs while it runs (scratch) and after (output).
  static int needs(const pc_request &r, uint64_t *scratch, uint64_t *output) {
    if (r.kind == PC_REQ_COMPRESS) {
      pc_config cfg = {r.leaf_size, r.flags};
      int rc = pc_compress_workspace_size(r.n, r.dtype, &cfg, 0, scratch);
      if (rc) return rc;
      return pc_compress_bound(r.n, r.dtype, &cfg, output);
    }
    if (r.kind == PC_REQ_DECOMPRESS) {
      if (r.dtype != PC_F32 && r.dtype != PC_F64) return PC_ERR_ARG;
      int rc = pc_decompress_workspace_size(r.n, scratch);
      if (rc) return rc;
      *output = 3 * (r.dtype == PC_F32 ? 4 : 8) * r.n;
      return PC_OK;
    }
    return PC_ERR_ARG;
  }

  void lane_main() {
    cudaSetDevice(device);
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      // admit the oldest request when its scratch and output fit
      uint64_t soff = 0, ooff = 0, sbytes = 0, obytes = 0;
      int rc = PC_OK;
      bool have = false;
      Job job;
      while (!have) {
        if (!queue.empty()) {
          job = queue.front();
          rc = needs(job.req, &sbytes, &obytes);
          // can never run (or, while stopping, nothing running will free room): complete it with an error
          const bool never = rc || align_up(sbytes) + align_up(obytes) > arena.size();
          const bool starved = stopping && running == 0 && !fits(sbytes, obytes);
          if (never || starved) {
            queue.pop_front();
            pc_completion c = {};
            c.tag = job.req.tag;
            c.kind = job.req.kind;
            c.status = rc ? rc : PC_ERR_CAPACITY;  // the arena cannot hold it
            c.t_submit = job.t_submit;
            c.t_start = c.t_done = now_seconds();
            done.push_back(c);
            cv_done.notify_all();
            continue;
          }
          if (arena.alloc(obytes, &ooff)) {
            if (arena.alloc(sbytes, &soff)) {
              queue.pop_front();
              have = true;
              break;
            }
            arena.release(ooff);
          }
        }
        if (stopping && queue.empty()) {
          lk.unlock();
          cudaStreamDestroy(s);
          return;
        }
        cv_work.wait(lk);
      }
      ++running;
      lk.unlock();
      pc_completion c = {};
      c.tag = job.req.tag;
      c.kind = job.req.kind;
      c.t_submit = job.t_submit;
      c.t_start = now_seconds();
      c.output = base + ooff;
      const pc_request &r = job.req;
      if (r.kind == PC_REQ_COMPRESS) {
        pc_config cfg = {r.leaf_size, r.flags};
        uint64_t size = 0;
        c.status = pcx::compress_device(r.input, r.n, r.dtype, r.eb_mode, r.eb, &cfg, base + ooff, obytes, &size,
                                        base + soff, sbytes, s);
        c.output_bytes = size;
      } else {
        c.status = pc_decompress(r.input, r.input_bytes, base + ooff, obytes, base + soff, sbytes, s);
        c.output_bytes = obytes;
      }
      if (cudaStreamSynchronize(s) != cudaSuccess && c.status == PC_OK) c.status = PC_ERR_CUDA;
      c.t_done = now_seconds();
      lk.lock();
      arena.release(soff);
      if (c.status != PC_OK) {
        arena.release(ooff);
        c.output = nullptr;
        c.output_bytes = 0;
      }
      --running;
      done.push_back(c);
      cv_done.notify_all();
      cv_work.notify_all();  // scratch came back: waiting requests may fit now
    }
  }
};

extern "C" {

int pc_compress_batch_workspace_size(const pc_compress_item *items, uint32_t count, uint32_t lanes,
                                     uint64_t *out_bytes) {
  if (!out_bytes || (count && !items)) return PC_ERR_ARG;
  uint64_t slice = kArenaAlign;
  for (uint32_t i = 0; i < count; ++i) {
    uint64_t b = 0;
    int rc = int(compress_scratch(items[i].n, items[i].dtype, items[i].leaf_size, items[i].flags, &b));
    if (rc) return rc;
    slice = std::max(slice, align_up(b));
  }
  *out_bytes = slice * pick_lanes(lanes, count);
  return PC_OK;
}

int pc_compress_batch(pc_compress_item *items, uint32_t count, uint32_t lanes, void *workspace,
                      uint64_t workspace_bytes, void *stream) {
  if (count == 0) return PC_OK;
  if (!items || !workspace || reinterpret_cast<uintptr_t>(workspace) % kArenaAlign) return PC_ERR_ARG;
  lanes = pick_lanes(lanes, count);
  uint64_t need = 0;
  int rc = pc_compress_batch_workspace_size(items, count, lanes, &need);
  if (rc) return rc;
  if (workspace_bytes < need) return PC_ERR_CAPACITY;
  const uint64_t slice = need / lanes;
  std::vector<uint32_t> order(count);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return items[a].n > items[b].n; });
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  rc = run_lanes(lanes, order, static_cast<cudaStream_t>(stream), [&](uint32_t lane, cudaStream_t s, uint32_t i) {
    pc_compress_item &it = items[i];
    pc_config cfg = {it.leaf_size, it.flags};
    uint64_t size = 0;
    it.status = pcx::compress_device(it.positions, it.n, it.dtype, it.eb_mode, it.eb, &cfg, it.out, it.out_capacity,
                                     &size, ws + lane * slice, slice, s);
    it.out_size = it.status == PC_OK ? size : 0;
  });
  if (rc) return rc;
  for (uint32_t i = 0; i < count; ++i)
    if (items[i].status != PC_OK) return items[i].status;
  return PC_OK;
}

int pc_decompress_batch_workspace_size(const pc_decompress_item *items, uint32_t count, uint32_t lanes,
                                       uint64_t *out_bytes) {
  if (!out_bytes || (count && !items)) return PC_ERR_ARG;
  uint64_t slice = kArenaAlign;
  for (uint32_t i = 0; i < count; ++i) {
    uint64_t b = 0;
    int rc = pc_decompress_workspace_size(items[i].n, &b);
    if (rc) return rc;
    slice = std::max(slice, align_up(b));
  }
  *out_bytes = slice * pick_lanes(lanes, count);
  return PC_OK;
}

int pc_decompress_batch(pc_decompress_item *items, uint32_t count, uint32_t lanes, void *workspace,
                        uint64_t workspace_bytes, void *stream) {
  if (count == 0) return PC_OK;
  if (!items || !workspace || reinterpret_cast<uintptr_t>(workspace) % kArenaAlign) return PC_ERR_ARG;
  lanes = pick_lanes(lanes, count);
  uint64_t need = 0;
  int rc = pc_decompress_batch_workspace_size(items, count, lanes, &need);
  if (rc) return rc;
  if (workspace_bytes < need) return PC_ERR_CAPACITY;
  const uint64_t slice = need / lanes;
  std::vector<uint32_t> order(count);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return items[a].n > items[b].n; });
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  rc = run_lanes(lanes, order, static_cast<cudaStream_t>(stream), [&](uint32_t lane, cudaStream_t s, uint32_t i) {
    pc_decompress_item &it = items[i];
    it.status = pc_decompress(it.stream_data, it.stream_bytes, it.out_positions, it.out_capacity_bytes,
                              ws + lane * slice, slice, s);
  });
  if (rc) return rc;
  for (uint32_t i = 0; i < count; ++i)
    if (items[i].status != PC_OK) return items[i].status;
  return PC_OK;
}

double pc_server_now(void) { return now_seconds(); }

int pc_server_create(void *arena, uint64_t arena_bytes, uint32_t lanes, pc_server **out) {
  if (!out || !arena || reinterpret_cast<uintptr_t>(arena) % kArenaAlign || lanes == 0 || lanes > 64)
    return PC_ERR_ARG;
  pc_server *s = new pc_server(arena, arena_bytes);
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return PC_ERR_CUDA;
  }
  for (uint32_t l = 0; l < lanes; ++l) s->lanes.emplace_back([s] { s->lane_main(); });
  *out = s;
  return PC_OK;
}

int pc_server_submit(pc_server *server, const pc_request *request) {
  if (!server || !request) return PC_ERR_ARG;
  if (request->kind != PC_REQ_COMPRESS && request->kind != PC_REQ_DECOMPRESS) return PC_ERR_ARG;
  const double t = now_seconds();
  std::lock_guard<std::mutex> lk(server->mu);
  if (server->stopping) return PC_ERR_ARG;
  server->queue.push_back(pc_server::Job{*request, t});
  server->cv_work.notify_one();
  return PC_OK;
}

int pc_server_poll(pc_server *server, pc_completion *out, uint32_t max, uint32_t *got, int wait) {
  if (!server || !got || (max && !out)) return PC_ERR_ARG;
  std::unique_lock<std::mutex> lk(server->mu);
  if (wait)
    server->cv_done.wait(lk, [&] {
      return !server->done.empty() || (server->queue.empty() && server->running == 0);
    });
  uint32_t k = 0;
  while (k < max && !server->done.empty()) {
    out[k++] = server->done.front();
    server->done.pop_front();
  }
  *got = k;
  return PC_OK;
}

int pc_server_release(pc_server *server, void *output) {
  if (!server || !output) return PC_ERR_ARG;
  std::lock_guard<std::mutex> lk(server->mu);
  const uint8_t *p = static_cast<const uint8_t *>(output);
  if (p < server->base || p >= server->base + server->arena.size()) return PC_ERR_ARG;
  if (!server->arena.release(uint64_t(p - server->base))) return PC_ERR_ARG;
  server->cv_work.notify_all();
  return PC_OK;
}

int pc_server_stats(pc_server *server, uint64_t *pending, uint64_t *arena_in_use) {
  if (!server) return PC_ERR_ARG;
  std::lock_guard<std::mutex> lk(server->mu);
  if (pending) *pending = server->queue.size() + server->running;
  if (arena_in_use) *arena_in_use = server->arena.in_use();
  return PC_OK;
}

int pc_server_destroy(pc_server *server) {
  if (!server) return PC_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(server->mu);
    server->stopping = true;
  }
  server->cv_work.notify_all();
  for (auto &t : server->lanes) t.join();
  delete server;
  return PC_OK;
}

}  // extern "C"
