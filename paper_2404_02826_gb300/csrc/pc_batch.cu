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

// Workspace of a batched decompression: the stream pointers and headers, one
// 64-byte error word and code bounds per item, the items' launch records, their
// leaf starts, every item's chunk descriptors (planned from the item's particle
// count) and one code table per item.
struct DecBatchLayout {
  uint64_t off_ptrs = 0, off_headers = 0, off_err = 0, off_items = 0, off_leaf_start = 0, off_chunks = 0,
           off_tables = 0, table_stride = 0, total = 0;
};

int decode_batch_layout(const pc_decompress_item *items, uint32_t count, DecBatchLayout &L) {
  uint64_t chunk_bytes = 0;
  for (uint32_t i = 0; i < count; ++i) {
    if (items[i].n > PC_MAX_PARTICLES) return PC_ERR_ARG;
    chunk_bytes += pcx::decode_chunk_bytes(items[i].n);
  }
  uint64_t o = 0;
  L.off_ptrs = o;
  o = align_up(o + 8ull * count);
  L.off_headers = o;
  o = align_up(o + uint64_t(PC_HEADER_BYTES) * count);
  L.off_err = o;  // 64 bytes per item, then the batch's own error word
  o = align_up(o + 64ull * (count + 1));
  L.off_items = o;
  o = align_up(o + sizeof(pcx::DecItem) * count);
  L.off_leaf_start = o;
  o = align_up(o + 8ull * (count + 1));
  L.off_chunks = o;
  o = align_up(o + chunk_bytes);
  L.table_stride = align_up(pcx::decode_table_bytes());
  L.off_tables = o;
  o += L.table_stride * count;
  L.total = o;
  return PC_OK;
}

// The batched decompression proper: every item's status is set; returns
// PC_ERR_CUDA when a CUDA call failed, else PC_OK.
//  1. the headers of all streams: one gather kernel and one read-back;
//  2. the plain call's checks per item, on the host, in its order;
//  3. one validation launch over all streams' leaves, one table launch, one
//     persistent decode launch per kind of stream (streams with lossless axes
//     one launch each);
//  4. every item's error word: one read-back.
int decode_batch_run(pc_decompress_item *items, uint32_t count, const DecBatchLayout &L, uint8_t *ws,
                     cudaStream_t st) {
  std::vector<const uint8_t *> ptrs(count, nullptr);
  std::vector<uint8_t> live(count, 0);
  uint32_t first_live = count;
  for (uint32_t i = 0; i < count; ++i) {
    const pc_decompress_item &it = items[i];
    items[i].status = PC_OK;
    if (!it.stream_data || reinterpret_cast<uintptr_t>(it.stream_data) % 16) {
      items[i].status = PC_ERR_ARG;
    } else if (it.stream_bytes < PC_HEADER_BYTES) {
      items[i].status = PC_ERR_CORRUPT;
    } else {
      live[i] = 1;
      if (first_live == count) first_live = i;
    }
    ptrs[i] = static_cast<const uint8_t *>(it.stream_data);
  }
  if (first_live == count) return PC_OK;
  for (uint32_t i = 0; i < count; ++i)
    if (!live[i]) ptrs[i] = ptrs[first_live];  // a header that is not used: read from a valid stream
  std::vector<uint8_t> headers(uint64_t(count) * PC_HEADER_BYTES);
  if (cudaMemcpyAsync(ws + L.off_ptrs, ptrs.data(), 8ull * count, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      pcx::launch_gather_headers(reinterpret_cast<const uint8_t *const *>(ws + L.off_ptrs), count,
                                 ws + L.off_headers, st) != cudaSuccess ||
      cudaMemcpyAsync(headers.data(), ws + L.off_headers, headers.size(), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemsetAsync(ws + L.off_err, 0, 64ull * (count + 1), st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PC_ERR_CUDA;

  std::vector<pcx::DecItem> dev;  // the streams that decode, in item order
  std::vector<uint32_t> which;    // their item index
  std::vector<int> kind;
  for (uint32_t i = 0; i < count; ++i) {
    if (!live[i]) continue;
    const pc_decompress_item &it = items[i];
    pc_info I;
    int s = pc_stream_info(headers.data() + uint64_t(i) * PC_HEADER_BYTES, PC_HEADER_BYTES, &I);
    const uint64_t esz = I.dtype == PC_F32 ? 4 : 8;
    if (!s && I.total_bytes > it.stream_bytes) s = PC_ERR_CORRUPT;
    if (!s && it.out_capacity_bytes < 3 * esz * I.n) s = PC_ERR_CAPACITY;
    if (!s && I.n == 0) continue;  // nothing to decode: PC_OK
    if (!s && (!it.out_positions || reinterpret_cast<uintptr_t>(it.out_positions) % esz)) s = PC_ERR_ARG;
    if (!s && I.n > it.n) s = PC_ERR_CAPACITY;  // the workspace was planned for it.n particles
    if (s) {
      items[i].status = s;
      continue;
    }
    pcx::DecItem d = {};
    pcx::DecodeLaunch &a = d.a;
    a.stream = static_cast<const uint8_t *>(it.stream_data);
    a.n = I.n;
    a.dtype = int(I.dtype);
    a.num_leaves = I.num_leaves;
    a.payload_words = I.payload_words;
    a.s = I.s;
    bool exact_o = true;
    for (int k = 0; k < 3; ++k) {
      a.o[k] = I.o[k];
      a.of[k] = float(I.o[k]);
      exact_o = exact_o && double(a.of[k]) == I.o[k];
    }
    a.sh = float(I.s);
    a.sl = float(I.s - double(a.sh));
    a.fast = I.dtype == PC_F32 && exact_o && I.s > 0x1p-100 && I.s < 0x1p100;
    a.out = it.out_positions;
    a.vec = reinterpret_cast<uintptr_t>(it.out_positions) % 16 == 0;
    a.err = reinterpret_cast<uint32_t *>(ws + L.off_err + 64ull * i);
    a.qb = reinterpret_cast<int32_t *>(ws + L.off_err + 64ull * i + 32);
    a.tab = ws + L.off_tables + L.table_stride * i;
    a.raw = I.lossless_axes;
    dev.push_back(d);
    which.push_back(i);
    kind.push_back(a.raw ? pcx::kDecKinds
                         : (a.dtype == 0 ? (a.fast ? pcx::kDecKindF32Fast : pcx::kDecKindF32) : pcx::kDecKindF64));
  }
  const uint32_t nd = uint32_t(dev.size());
  if (nd == 0) return PC_OK;
  // chunk descriptors: each kind's streams one after another (lossless streams last)
  uint64_t at = 0;
  uint64_t kind_first[pcx::kDecKinds + 1] = {}, kind_chunks[pcx::kDecKinds + 1] = {};
  bool kind_vec[pcx::kDecKinds] = {true, true, true};
  for (int k = 0; k <= pcx::kDecKinds; ++k) {
    kind_first[k] = at;
    for (uint32_t j = 0; j < nd; ++j) {
      if (kind[j] != k) continue;
      dev[j].a.chunks = ws + L.off_chunks + 32ull * at;
      dev[j].chunk0 = at - kind_first[k];
      at += pcx::decode_chunks(dev[j].a.n);
      if (k < pcx::kDecKinds) kind_vec[k] = kind_vec[k] && dev[j].a.vec;
    }
    kind_chunks[k] = at - kind_first[k];
  }
  // leaves: every stream from a multiple of 32
  std::vector<uint64_t> leaf_start(nd + 1);
  uint64_t leaves = 0;
  for (uint32_t j = 0; j < nd; ++j) {
    dev[j].leaf0 = leaves;
    leaf_start[j] = leaves;
    leaves += (dev[j].a.num_leaves + 31) / 32 * 32;
  }
  leaf_start[nd] = leaves;
  pcx::DecItem *items_dev = reinterpret_cast<pcx::DecItem *>(ws + L.off_items);
  uint64_t *leaf_dev = reinterpret_cast<uint64_t *>(ws + L.off_leaf_start);
  if (cudaMemcpyAsync(items_dev, dev.data(), sizeof(pcx::DecItem) * nd, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(leaf_dev, leaf_start.data(), 8ull * (nd + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      pcx::launch_validate_batch(items_dev, leaf_dev, nd, leaves, st) != cudaSuccess ||
      pcx::launch_dtable_batch(items_dev, nd, st) != cudaSuccess)
    return PC_ERR_CUDA;
  uint32_t *berr = reinterpret_cast<uint32_t *>(ws + L.off_err + 64ull * count);
  for (int k = 0; k < pcx::kDecKinds; ++k)
    if (pcx::launch_decode_batch(k, kind_vec[k], items_dev, ws + L.off_chunks + 32ull * kind_first[k],
                                 kind_chunks[k], berr, st) != cudaSuccess)
      return PC_ERR_CUDA;
  for (uint32_t j = 0; j < nd; ++j)
    if (kind[j] == pcx::kDecKinds && pcx::launch_decode_lossless(dev[j].a, st) != cudaSuccess) return PC_ERR_CUDA;
  // every item's error word and the batch's: one read-back
  std::vector<uint32_t> errs(16ull * (count + 1));
  if (cudaMemcpyAsync(errs.data(), ws + L.off_err, 64ull * (count + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PC_ERR_CUDA;
  pcx::trace_flush();
  const uint32_t batch_err = errs[16ull * count];  // a wait gave up: no item's output can be trusted
  for (uint32_t j = 0; j < nd; ++j) {
    const uint32_t e = errs[16ull * which[j]] | batch_err;
    items[which[j]].status = (e & pcx::kErrCorrupt)   ? PC_ERR_CORRUPT
                             : (e & pcx::kErrTimeout) ? PC_ERR_TIMEOUT
                             : e                      ? PC_ERR_CUDA
                                                      : PC_OK;
  }
  return PC_OK;
}

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
  (void)lanes;  // one set of launches serves every item
  if (!out_bytes || (count && !items)) return PC_ERR_ARG;
  DecBatchLayout L;
  const int rc = decode_batch_layout(items, count, L);
  if (rc) return rc;
  *out_bytes = L.total;
  return PC_OK;
}

int pc_decompress_batch(pc_decompress_item *items, uint32_t count, uint32_t lanes, void *workspace,
                        uint64_t workspace_bytes, void *stream) {
  (void)lanes;  // one set of launches serves every item
  if (count == 0) return PC_OK;
  if (!items || !workspace || reinterpret_cast<uintptr_t>(workspace) % kArenaAlign) return PC_ERR_ARG;
  DecBatchLayout L;
  const int rc = decode_batch_layout(items, count, L);
  if (rc) return rc;
  if (workspace_bytes < L.total) return PC_ERR_CAPACITY;
  const int cuda = decode_batch_run(items, count, L, static_cast<uint8_t *>(workspace),
                                    static_cast<cudaStream_t>(stream));
  if (cuda) return cuda;
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
