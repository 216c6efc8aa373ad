// A serving loop over the grouped Stream-K launch: requests (independent
// GEMMs of any shape) are queued as they arrive; a worker thread admits them
// into batches, bounded by a problem count and by the HBM their operands
// pin, plans each batch as one Stream-K iteration space (the grouped
// schedule), and launches it on one of a few streams, so that a batch admitted
// while others run overlaps them on the device.  Completion is observed with
// events; each request's latency runs from submission to that observation.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/streamk.h"
#include "host_util.h"
#include "launch.h"
#include "planner.h"
#include "sk_args.h"

using namespace sk::host;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t id;
  int64_t m, n, k;
  const void* A;
  const void* B;
  void* C;
  const float* scale_a;  // E4M3 requests: block scales; else null
  const float* scale_b;
  float alpha, beta;
  int64_t bytes;
  int64_t tiles;  // 128 x 128 output tiles: at least the SM count fills the GPU alone
  bool f8;
  Clock::time_point submitted;
};

// One batch in flight: its stream, buffers and requests.
struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  // One device block and its pinned staging copy, uploaded with one copy per
  // batch: the problem table, the walk table, the per-CTA start problems.
  char* d_block = nullptr;
  char* h_block = nullptr;
  size_t off_walk = 0, off_start = 0;
  sk::GroupProblem* d_probs = nullptr;
  sk::GroupWalk* d_walk = nullptr;
  int32_t* d_start = nullptr;
  sk::GroupProblem* h_probs = nullptr;
  sk::GroupWalk* h_walk = nullptr;
  int32_t* h_start = nullptr;
  int32_t* d_err = nullptr;
  char* ws = nullptr;
  // mapped pinned word a failing launch writes its status into (host view,
  // device view); cleared before each launch
  int32_t* h_status = nullptr;
  int32_t* d_status = nullptr;
  std::vector<Request> reqs;
  int64_t bytes = 0;
  bool busy = false;
};

}  // namespace

struct sk_server_s {
  int ab_type = 0, c_type = 0, max_batch = 1, num_sms = 0;
  int64_t budget = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  // queued requests by input type (0: the server's 16-bit type, 1: E4M3);
  // a batch takes one type, the one whose oldest request is older
  std::deque<Request> pending[2];
  bool none_pending() const { return pending[0].empty() && pending[1].empty(); }
  // id -> (state, latency_us, status): state 0 queued, 1 running, 2 done
  struct Entry {
    int state = 0;
    int status = SK_OK;
    double latency_us = 0.0;
  };
  std::unordered_map<uint64_t, Entry> entries;
  std::condition_variable done_cv;
  int64_t inflight_bytes = 0;
  uint64_t next_id = 1;
  int64_t submitted = 0, completed = 0, batches = 0, max_batch_seen = 0, problems_launched = 0;
  bool stop = false;
  std::atomic<int64_t> queued{0};  // submissions not yet admitted (read without the lock)
  // Tensor maps encoded before, keyed by (kind, pointer, dtype, rows, cols,
  // box rows); used by the worker only.
  struct MapKey {
    const void* ptr;
    int64_t rows, cols;
    int32_t kind, dtype, box;
    bool operator==(const MapKey& o) const {
      return ptr == o.ptr && rows == o.rows && cols == o.cols && kind == o.kind &&
             dtype == o.dtype && box == o.box;
    }
  };
  struct MapHash {
    size_t operator()(const MapKey& k) const {
      uint64_t h = reinterpret_cast<uintptr_t>(k.ptr) * 0x9E3779B97F4A7C15ull;
      h ^= static_cast<uint64_t>(k.rows) * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
      h ^= static_cast<uint64_t>(k.cols) * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
      h ^= static_cast<uint64_t>(k.kind * 1024 + k.dtype * 512 + k.box) + (h << 6) + (h >> 2);
      return static_cast<size_t>(h);
    }
  };
  struct MapEntry {
    CUtensorMap map;
    int status;  // SK_OK, or the encode failure (kind 2: 1 = TMA store possible)
  };
  std::unordered_map<MapKey, MapEntry, MapHash> map_cache;
  // single-GEMM plans for lone requests, per (m, n, k, input type); they all
  // run on the fifo stream, so their workspaces are never used concurrently;
  // used by the worker only, destroyed with the server
  struct PlanKey {
    int64_t m, n, k;
    int32_t ab;
    bool operator==(const PlanKey& o) const { return m == o.m && n == o.n && k == o.k && ab == o.ab; }
  };
  struct PlanHash {
    size_t operator()(const PlanKey& k) const {
      uint64_t h = static_cast<uint64_t>(k.m) * 0x9E3779B97F4A7C15ull;
      h ^= static_cast<uint64_t>(k.n) * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
      h ^= static_cast<uint64_t>(k.k) * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
      return static_cast<size_t>(h ^ static_cast<uint64_t>(k.ab));
    }
  };
  std::unordered_map<PlanKey, sk_plan_t, PlanHash> single_plans;
  // A launch whose CTAs wait on one another (split tiles) must find every
  // CTA of its grid resident, so it runs alone: it waits for every slot's
  // work in flight, and every later launch waits for this event, recorded
  // after it.  Data-parallel launches between split ones overlap freely.
  cudaEvent_t split_done = nullptr;
  // Lone requests run on one stream in arrival order, as plain launches do
  // (with their plans' own launch form: programmatic dependent launch, CTA
  // pairs); batches run on their slots' streams.
  cudaStream_t fifo = nullptr;
  int device = 0;
  std::thread worker;
};

namespace {

constexpr size_t kMapCacheEntries = 16384;
constexpr size_t kSinglePlanCap = 256;  // cached single-GEMM plans (each owns a workspace)
constexpr int kIdleSpinUs = 200;  // idle worker: spin before sleeping

void free_slot(Slot& s) {
  if (s.d_block) cudaFree(s.d_block);
  if (s.d_err) cudaFree(s.d_err);
  if (s.ws) cudaFree(s.ws);
  if (s.h_block) cudaFreeHost(s.h_block);
  if (s.h_status) cudaFreeHost(s.h_status);
  if (s.done) cudaEventDestroy(s.done);
  if (s.stream) cudaStreamDestroy(s.stream);
  s = Slot();
}

cudaError_t alloc_slot(Slot& s, int max_batch, int num_sms) {
  cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
  const size_t ws = static_cast<size_t>(sk::kFlagBytes) + static_cast<size_t>(num_sms) * sk::kBlkM * 256 * 4;
  auto up = [](size_t v) { return (v + 127) / 128 * 128; };
  s.off_walk = up(static_cast<size_t>(max_batch) * sizeof(sk::GroupProblem));
  s.off_start = s.off_walk + up(static_cast<size_t>(max_batch + 1) * sizeof(sk::GroupWalk));
  const size_t block = s.off_start + static_cast<size_t>(2 * num_sms) * sizeof(int32_t);
  if (e == cudaSuccess) e = cudaMalloc(&s.d_block, block);
  if (e == cudaSuccess) e = cudaMallocHost(&s.h_block, block);
  if (e == cudaSuccess) {
    s.d_probs = reinterpret_cast<sk::GroupProblem*>(s.d_block);
    s.d_walk = reinterpret_cast<sk::GroupWalk*>(s.d_block + s.off_walk);
    s.d_start = reinterpret_cast<int32_t*>(s.d_block + s.off_start);
    s.h_probs = reinterpret_cast<sk::GroupProblem*>(s.h_block);
    s.h_walk = reinterpret_cast<sk::GroupWalk*>(s.h_block + s.off_walk);
    s.h_start = reinterpret_cast<int32_t*>(s.h_block + s.off_start);
  }
  if (e == cudaSuccess) e = cudaMalloc(&s.d_err, 4 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(s.d_err, 0, 4 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&s.ws, ws);
  if (e == cudaSuccess) e = cudaMemset(s.ws, 0, ws);
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&s.h_status), 4 * sizeof(int32_t), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s.d_status), s.h_status, 0);
  if (e == cudaSuccess) s.h_status[0] = 0;
  return e;
}

// Plan and launch the requests of a slot as one grouped launch.  Returns an
// sk_status; on failure nothing is in flight on the slot.  Runs without the
// server lock: it reads only the slot (owned by the worker while busy) and
// the server's immutable settings.
// Tensor map through the server's cache: kind 0 = 2-D operand, 1 = 3-D
// operand view, 2 = output (status 1 when C can be stored by TMA, else 0).
int cached_map(sk_server_s* sv, CUtensorMap* out, int kind, const void* ptr, int dtype,
               int64_t rows, int64_t cols, int box) {
  const sk_server_s::MapKey key{ptr, rows, cols, kind, dtype, box};
  auto it = sv->map_cache.find(key);
  if (it == sv->map_cache.end()) {
    sk_server_s::MapEntry e{};
    if (kind == 0)
      e.status = encode_operand(&e.map, ptr, dtype, rows, cols, cols, box);
    else if (kind == 1)
      e.status = encode_operand_3d(&e.map, ptr, dtype, rows, cols, cols, box);
    else
      e.status = encode_output(&e.map, const_cast<void*>(ptr), dtype, rows, cols, cols) ? 1 : 0;
    if (sv->map_cache.size() >= kMapCacheEntries) sv->map_cache.clear();
    it = sv->map_cache.emplace(key, e).first;
  }
  *out = it->second.map;
  return it->second.status;
}

// Orders a launch of slot s on `stream`: after the last split launch, and
// (for a split launch) after all other slots' work in flight.
cudaError_t order_launch(sk_server_s* sv, Slot& s, cudaStream_t stream, bool split) {
  cudaError_t e = cudaStreamWaitEvent(stream, sv->split_done, 0);
  if (split)
    for (Slot& o : sv->slots)
      if (&o != &s && o.busy && e == cudaSuccess) e = cudaStreamWaitEvent(stream, o.done, 0);
  return e;
}

// A lone request runs as a single GEMM from a plan cached per shape and input
// type, on the fifo stream: its arguments travel by value with the launch, so
// nothing is uploaded first.
int launch_single(sk_server_s* sv, Slot& s) {
  const Request& r = s.reqs[0];
  const int ab_type = r.f8 ? SK_E4M3 : sv->ab_type;
  const sk_server_s::PlanKey key{r.m, r.n, r.k, ab_type};
  auto it = sv->single_plans.find(key);
  if (it == sv->single_plans.end()) {
    if (sv->single_plans.size() >= kSinglePlanCap) {
      // every plan's launches are on the fifo stream: once it has drained,
      // none is in use
      const cudaError_t e = cudaStreamSynchronize(sv->fifo);
      if (e != cudaSuccess) return cuda_status(e);
      for (auto& kv : sv->single_plans) sk_plan_destroy(kv.second);
      sv->single_plans.clear();
    }
    sk_plan_t p = nullptr;
    // The plan's own launch form (CTA pairs, programmatic dependent launch)
    // is safe here: within one stream a kernel's CTAs only wait for SMs that
    // earlier kernels of the stream free on their own, and a split launch
    // runs alone with respect to the slots' streams (order_launch).
    int st = sk_plan(&p, r.m, r.n, r.k, static_cast<sk_dtype>(ab_type),
                     static_cast<sk_dtype>(ab_type), static_cast<sk_dtype>(sv->c_type), SK_F32,
                     SK_ROW_MAJOR, SK_COL_MAJOR, SK_ROW_MAJOR, SK_MODE_AUTO);
    if (st != SK_OK) {
      sk_plan_destroy(p);
      return st;
    }
    it = sv->single_plans.emplace(key, p).first;
  }
  int64_t ws = 0;
  sk_plan_get(it->second, SK_ATTR_WORKSPACE_BYTES, &ws);
  const bool split = ws > 0;
  {
    const cudaError_t e = order_launch(sv, s, sv->fifo, split);
    if (e != cudaSuccess) return cuda_status(e);
  }
  s.h_status[0] = 0;
  int st = sk::gemm_reporting(it->second, r.A, r.B, r.scale_a, r.scale_b, r.C, r.alpha, r.beta,
                              sv->fifo, s.d_status);
  if (st != SK_OK) return st;
  if (split) {
    const cudaError_t e = cudaEventRecord(sv->split_done, sv->fifo);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return cuda_status(cudaEventRecord(s.done, sv->fifo));
}

int launch_slot(sk_server_s* sv, Slot& s) {
  const int count = static_cast<int>(s.reqs.size());
  if (count == 1) return launch_single(sv, s);
  const bool f8 = s.reqs[0].f8;  // a batch holds one input type
  const int ab_type = f8 ? SK_E4M3 : sv->ab_type;
  // E4M3 problems are planned as 16-bit problems of k/2 (the same bytes per row)
  std::vector<int64_t> m(count), n(count), k(count);
  for (int i = 0; i < count; ++i) {
    m[i] = s.reqs[i].m;
    n[i] = s.reqs[i].n;
    k[i] = f8 ? s.reqs[i].k / 2 : s.reqs[i].k;
  }
  // A batch packs requests below a wave each (larger ones run alone) and is
  // launched as data-parallel waves over the problems' tiles, planned in
  // O(count + grid) with no segment records: the worker's planning time is
  // on every request's path, and a data-parallel launch never has to run
  // alone (split launches wait for all other work in flight).  128-wide tiles
  // while the batch has fewer than two waves of them, for parallelism.
  int64_t tiles128 = 0;
  for (int i = 0; i < count; ++i) tiles128 += s.reqs[i].tiles;
  const int tile_n = f8 || tiles128 < 2 * static_cast<int64_t>(sv->num_sms) ? 128 : 0;
  auto plan = std::make_shared<sk::GroupPlan>();
  {
    const int st = sk::describe_grouped_dp(count, m.data(), n.data(), k.data(), tile_n,
                                           sv->num_sms, plan.get());
    if (st != SK_OK) return st;
  }
  const sk::GroupPlan& gp = *plan;
  int st = SK_OK;
  for (int i = 0; i < count; ++i) {
    const Request& r = s.reqs[i];
    sk::GroupProblem& pr = s.h_probs[i];
    std::memset(static_cast<void*>(&pr), 0, sizeof(pr));
    // E4M3 rows go to TMA as 16-bit rows of k/2 elements
    const int tt = f8 ? SK_BF16 : ab_type;
    const int64_t tk = f8 ? r.k / 2 : r.k;
    st = cached_map(sv, &pr.tmA, 0, r.A, tt, r.m, tk, sk::kBlkM);
    if (st == SK_OK) st = cached_map(sv, &pr.tmB, 0, r.B, tt, r.n, tk, gp.tile_n);
    const bool use3d = gp.tile_n <= 128 && tk / sk::kBlkK >= 2;
    if (st == SK_OK && use3d) st = cached_map(sv, &pr.tmA3, 1, r.A, tt, r.m, tk, sk::kBlkM);
    if (st == SK_OK && use3d) st = cached_map(sv, &pr.tmB3, 1, r.B, tt, r.n, tk, gp.tile_n);
    if (st != SK_OK) return st;
    if (!use3d) {
      pr.tmA3 = pr.tmA;
      pr.tmB3 = pr.tmB;
    }
    const bool c_tma = cached_map(sv, &pr.tmC, 2, r.C, sv->c_type, r.m, r.n, 0) == 1;
    if (!c_tma) pr.tmC = pr.tmA;
    pr.C = r.C;
    pr.ldc = r.n;
    pr.m = static_cast<int32_t>(r.m);
    pr.n = static_cast<int32_t>(r.n);
    pr.c_tma = c_tma ? store_path(0) : 0;
    pr.c_vec = (r.n * static_cast<int64_t>(dtype_size(sv->c_type))) % 16 == 0 ? 1 : 0;
    pr.alpha = r.alpha;
    pr.beta = r.beta;
    pr.scale_a = r.scale_a;
    pr.scale_b = r.scale_b;
    pr.ld_scale = static_cast<int32_t>((r.k + 127) / 128);
  }
  std::memcpy(s.h_walk, gp.walk.data(), gp.walk.size() * sizeof(sk::GroupWalk));
  std::memcpy(s.h_start, gp.gstart.data(), gp.gstart.size() * sizeof(int32_t));
  cudaError_t e = cudaMemcpyAsync(s.d_block, s.h_block,
                                  s.off_start + gp.gstart.size() * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s.stream);
  if (e != cudaSuccess) return cuda_status(e);
  sk::SkArgs a{};
  sk::set_group_walk_args(a, gp);
  a.idesc = make_idesc(ab_type, gp.tile_n, 1);
  const bool split = gp.workspace_bytes > 0;
  a.flags = split ? reinterpret_cast<uint32_t*>(s.ws) : nullptr;
  a.partials = split ? reinterpret_cast<float*>(s.ws + sk::kFlagBytes) : nullptr;
  a.epoch = next_epoch();
  a.err = s.d_err;
  a.err_host = s.d_status;
  a.trace_cap = gp.max_segments;
  a.debug_skip_signal = -1;
  a.timeout_ns = kDefaultTimeoutNs;
  a.pdl = 0;
  a.gwalk = s.d_walk;
  a.gstart = s.d_start;
  a.gprobs = s.d_probs;
  const CUtensorMap& any = s.h_probs[0].tmA;
  e = order_launch(sv, s, s.stream, split);
  if (e != cudaSuccess) return cuda_status(e);
  s.h_status[0] = 0;
  e = f8                ? sk::launch_grouped_f8(sv->c_type, gp.tile_n, any, a, split, s.stream)
      : gp.tile_n == 256 ? sk::launch_grouped_bn256(sv->c_type, 1, any, a, split, s.stream)
      : gp.tile_n == 64  ? sk::launch_grouped_bn64(sv->c_type, 1, any, a, split, s.stream)
                         : sk::launch_grouped_bn128(sv->c_type, 1, any, a, split, s.stream);
  if (e == cudaSuccess && split) e = cudaEventRecord(sv->split_done, s.stream);
  if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
  if (e != cudaSuccess) return cuda_status(e);
  return SK_OK;
}

void finish(sk_server_s* sv, Slot& s, int status) {
  const auto now = Clock::now();
  for (const Request& r : s.reqs) {
    auto& e = sv->entries[r.id];
    e.state = 2;
    e.status = status;
    e.latency_us = std::chrono::duration<double, std::micro>(now - r.submitted).count();
    ++sv->completed;
  }
  sv->inflight_bytes -= s.bytes;
  s.reqs.clear();
  s.bytes = 0;
  s.busy = false;
}

void worker_loop(sk_server_s* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    // retire finished batches
    bool any_busy = false;
    for (Slot& s : sv->slots) {
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) {
        any_busy = true;
        continue;
      }
      int status = q == cudaSuccess ? SK_OK : SK_ERR_CUDA;
      if (status == SK_OK && *reinterpret_cast<volatile int32_t*>(s.h_status) != 0) {
        status = SK_ERR_TIMEOUT;
        cudaMemset(s.d_err, 0, 4 * sizeof(int32_t));
        cudaMemset(s.ws, 0, static_cast<size_t>(sk::kFlagBytes));
      }
      finish(sv, s, status);
      sv->done_cv.notify_all();
    }
    if (sv->stop && sv->none_pending() && !any_busy) break;
    // admit a batch into a free slot
    Slot* free_slot_p = nullptr;
    for (Slot& s : sv->slots)
      if (!s.busy) {
        free_slot_p = &s;
        break;
      }
    if (free_slot_p != nullptr && !sv->none_pending()) {
      Slot& s = *free_slot_p;
      const int t = sv->pending[0].empty()   ? 1
                    : sv->pending[1].empty() ? 0
                    : (sv->pending[1].front().id < sv->pending[0].front().id ? 1 : 0);
      std::deque<Request>& q = sv->pending[t];
      // Batch only under backlog: with as many free slots as queued
      // requests each runs alone (a single launch); otherwise the queue is
      // spread over the free slots.
      int free_slots = 0;
      for (const Slot& o : sv->slots) free_slots += o.busy ? 0 : 1;
      const int queued = static_cast<int>(q.size());
      const int cap = std::min(sv->max_batch, (queued + free_slots - 1) / free_slots);
      // A request with at least a wave of tiles fills the GPU on its own:
      // sharing a launch gains it nothing and would cost it its own plan's
      // configuration (CTA pairs, 256-wide tiles), so it runs alone; only
      // requests below a wave are packed together.
      const int64_t wave = sv->num_sms;
      while (!q.empty() && static_cast<int>(s.reqs.size()) < cap) {
        const Request& r = q.front();
        if (!s.reqs.empty() && r.tiles >= wave) break;
        const bool nothing_else = s.reqs.empty() && sv->inflight_bytes == 0;
        if (!nothing_else && sv->inflight_bytes + s.bytes + r.bytes > sv->budget) break;
        s.bytes += r.bytes;
        s.reqs.push_back(r);
        sv->entries[r.id].state = 1;
        q.pop_front();
        sv->queued.fetch_sub(1, std::memory_order_relaxed);
        if (r.tiles >= wave) break;
      }
      if (!s.reqs.empty()) {
        sv->inflight_bytes += s.bytes;
        s.busy = true;
        lk.unlock();  // planning and encoding do not block submitters
        const int st = launch_slot(sv, s);
        lk.lock();
        if (st != SK_OK) {
          finish(sv, s, st);
          sv->done_cv.notify_all();
        } else {
          const int64_t count = static_cast<int64_t>(s.reqs.size());
          ++sv->batches;
          sv->problems_launched += count;
          sv->max_batch_seen = std::max<int64_t>(sv->max_batch_seen, count);
        }
        continue;
      }
    }
    // Nothing to launch now.  With batches in flight, poll their events
    // (yielding the core between polls: a timed sleep would round up to the
    // kernel's timer slack, tens of microseconds).  Idle, spin a while for a
    // submission before blocking on the condition variable.
    lk.unlock();
    if (any_busy) {
      std::this_thread::yield();
    } else {
      const auto t0 = Clock::now();
      while (sv->queued.load(std::memory_order_relaxed) == 0 &&
             Clock::now() - t0 < std::chrono::microseconds(kIdleSpinUs))
        std::this_thread::yield();
    }
    lk.lock();
    if (!any_busy)
      sv->cv.wait_for(lk, std::chrono::milliseconds(5),
                      [&] { return sv->stop || !sv->none_pending(); });
  }
}

}  // namespace

extern "C" {

int sk_server_create(sk_server_t* out, sk_dtype ab_type, sk_dtype c_type, int max_batch, int slots,
                     int64_t hbm_budget_bytes) {
  if (out == nullptr) return SK_ERR_INVALID;
  *out = nullptr;
  if (max_batch < 1 || max_batch > 4096 || slots < 1 || slots > 8 || hbm_budget_bytes <= 0)
    return SK_ERR_INVALID;
  if (!(ab_type == SK_F16 || ab_type == SK_BF16)) return SK_ERR_UNSUPPORTED;
  if (!(c_type == SK_F32 || c_type == SK_BF16 || c_type == SK_F16)) return SK_ERR_UNSUPPORTED;
  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SK_ERR_CUDA;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SK_ERR_CUDA;
  if (major != 10 || minor != 3) return SK_ERR_DEVICE;
  size_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  cudaError_t e = sk::prepare_bn128(&s1);
  if (e == cudaSuccess) e = sk::prepare_bn64(&s0);
  if (e == cudaSuccess) e = sk::prepare_bn256(&s2);
  if (e == cudaSuccess) e = sk::prepare_f8(&s3);
  if (e != cudaSuccess) return cuda_status(e);
  sk_server_s* sv = new (std::nothrow) sk_server_s();
  if (sv == nullptr) return SK_ERR_NOMEM;
  sv->ab_type = ab_type;
  sv->c_type = c_type;
  sv->max_batch = max_batch;
  sv->num_sms = sms;
  sv->budget = hbm_budget_bytes;
  sv->device = dev;
  e = cudaEventCreateWithFlags(&sv->split_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->fifo, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (sv->split_done) cudaEventDestroy(sv->split_done);
    delete sv;
    return cuda_status(e);
  }
  sv->slots.resize(static_cast<size_t>(slots));
  for (Slot& s : sv->slots) {
    e = alloc_slot(s, max_batch, sms);
    if (e != cudaSuccess) {
      for (Slot& t : sv->slots) free_slot(t);
      cudaEventDestroy(sv->split_done);
      cudaStreamDestroy(sv->fifo);
      delete sv;
      return cuda_status(e);
    }
  }
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return SK_OK;
}

}  // extern "C"

namespace {

int submit(sk_server_t sv, int64_t m, int64_t n, int64_t k, const void* A, const void* B,
           const float* scale_a, const float* scale_b, void* C, float alpha, float beta,
           uint64_t* ticket) {
  const bool f8 = scale_a != nullptr;
  if (sv == nullptr || ticket == nullptr || m < 1 || n < 1 || k < 1 || k % (f8 ? 16 : 8) != 0 ||
      m > INT32_MAX || n > INT32_MAX || k > INT32_MAX || A == nullptr || B == nullptr ||
      C == nullptr || (reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(B) & 15u) ||
      (reinterpret_cast<uintptr_t>(C) & 15u))
    return SK_ERR_INVALID;
  if (f8 && (scale_b == nullptr || (reinterpret_cast<uintptr_t>(scale_a) & 3u) ||
             (reinterpret_cast<uintptr_t>(scale_b) & 3u)))
    return SK_ERR_INVALID;
  Request r{};
  r.m = m;
  r.n = n;
  r.k = k;
  r.A = A;
  r.B = B;
  r.C = C;
  r.scale_a = scale_a;
  r.scale_b = scale_b;
  r.f8 = f8;
  r.alpha = alpha;
  r.beta = beta;
  const int64_t in_bytes = f8 ? 1 : 2;
  r.bytes = in_bytes * (m * k + n * k) + m * n * static_cast<int64_t>(dtype_size(sv->c_type));
  r.tiles = ((m + 127) / 128) * ((n + 127) / 128);
  r.submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return SK_ERR_INVALID;
    r.id = sv->next_id++;
    sv->entries[r.id] = sk_server_s::Entry{};
    sv->pending[f8 ? 1 : 0].push_back(r);
    ++sv->submitted;
    sv->queued.fetch_add(1, std::memory_order_relaxed);
  }
  sv->cv.notify_one();
  *ticket = r.id;
  return SK_OK;
}

}  // namespace

extern "C" {

int sk_server_submit(sk_server_t sv, int64_t m, int64_t n, int64_t k, const void* A, const void* B,
                     void* C, float alpha, float beta, uint64_t* ticket) {
  return submit(sv, m, n, k, A, B, nullptr, nullptr, C, alpha, beta, ticket);
}

int sk_server_submit_scaled(sk_server_t sv, int64_t m, int64_t n, int64_t k, const void* A,
                            const void* B, const float* scale_a, const float* scale_b, void* C,
                            float alpha, float beta, uint64_t* ticket) {
  if (scale_a == nullptr || scale_b == nullptr) return SK_ERR_INVALID;
  return submit(sv, m, n, k, A, B, scale_a, scale_b, C, alpha, beta, ticket);
}

int sk_server_poll(sk_server_t sv, uint64_t ticket, int* state, double* latency_us) {
  if (sv == nullptr || state == nullptr) return SK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->entries.find(ticket);
  if (it == sv->entries.end()) return SK_ERR_INVALID;
  *state = it->second.state;
  if (latency_us) *latency_us = it->second.latency_us;
  if (it->second.state == 2) {
    const int st = it->second.status;
    sv->entries.erase(it);
    return st;
  }
  return SK_OK;
}

int sk_server_wait(sk_server_t sv, uint64_t ticket, double* latency_us) {
  if (sv == nullptr) return SK_ERR_INVALID;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->entries.find(ticket);
  if (it == sv->entries.end()) return SK_ERR_INVALID;
  sv->done_cv.wait(lk, [&] {
    auto e = sv->entries.find(ticket);
    return e == sv->entries.end() || e->second.state == 2;
  });
  it = sv->entries.find(ticket);
  if (it == sv->entries.end()) return SK_ERR_INVALID;  // retired by a concurrent poll
  const int st = it->second.status;
  if (latency_us) *latency_us = it->second.latency_us;
  sv->entries.erase(it);
  return st;
}

int sk_server_stats(sk_server_t sv, int64_t* stats) {
  if (sv == nullptr || stats == nullptr) return SK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  const int64_t v[6] = {sv->submitted, sv->completed, sv->batches, sv->max_batch_seen,
                        sv->problems_launched,
                        static_cast<int64_t>(sv->pending[0].size() + sv->pending[1].size())};
  for (int i = 0; i < 6; ++i) stats[i] = v[i];
  return SK_OK;
}

int sk_server_destroy(sk_server_t sv) {
  if (sv == nullptr) return SK_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  if (sv->fifo) cudaStreamSynchronize(sv->fifo);
  for (Slot& s : sv->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    free_slot(s);
  }
  if (sv->fifo) cudaStreamDestroy(sv->fifo);
  for (auto& kv : sv->single_plans) sk_plan_destroy(kv.second);
  if (sv->split_done) cudaEventDestroy(sv->split_done);
  delete sv;
  return SK_OK;
}

}  // extern "C"
