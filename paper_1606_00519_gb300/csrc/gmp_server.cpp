// gmp_server.cpp - serving loop of libgmp: continuous batching of
// decompression requests under a device-memory budget.
//
// A request is a compressed stream in host memory.  At submit the host
// builds its block index.  A scheduler thread admits pending requests in
// arrival order as soon as the device arena has room for the request's
// compressed bytes, index and output; it packs the admitted requests into a
// batch and launches it on the first idle lane (a decoder context with its own
// CUDA stream), so batches formed while others run overlap on the GPU.  A host
// function enqueued after each batch stamps its completion time; outputs stay
// in device memory until the caller releases the request.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gmp.h"
#include "gmp_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one device allocation (offsets, 256-byte units).
class Arena {
 public:
  bool init(uint64_t bytes) {
    if (cudaMalloc(&base_, bytes) != cudaSuccess) return false;
    size_ = bytes;
    free_[0] = bytes;
    return true;
  }
  ~Arena() {
    if (base_) cudaFree(base_);
  }
  static uint64_t round(uint64_t n) { return (n + 255) & ~uint64_t(255); }
  // returns offset or UINT64_MAX
  uint64_t alloc(uint64_t n) {
    n = round(std::max<uint64_t>(n, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        uint64_t off = it->first, rem = it->second - n;
        free_.erase(it);
        if (rem) free_[off + n] = rem;
        used_ += n;
        return off;
      }
    }
    return UINT64_MAX;
  }
  void release(uint64_t off, uint64_t n) {
    n = round(std::max<uint64_t>(n, 1));
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint8_t* ptr(uint64_t off) const { return base_ + off; }
  uint64_t size() const { return size_; }
  uint64_t used() const { return used_; }

 private:
  uint8_t* base_ = nullptr;
  uint64_t size_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> free_;
};

struct Request {
  uint64_t id;
  const uint8_t* host;
  uint64_t bytes;
  std::vector<gmp_block_ref> index;
  gmp_stream_info info;
  uint64_t need;        // arena bytes
  uint64_t off = UINT64_MAX;
  uint64_t comp_off = 0, index_off = 0, out_off = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  int32_t status = 0;
};

struct Lane {
  gmp_context* ctx = nullptr;
  cudaStream_t stream = nullptr;
  gmp_file_desc* h_table = nullptr;  // pinned
  gmp_file_desc* d_table = nullptr;
  int32_t* h_status = nullptr;       // pinned
  int32_t* d_status = nullptr;
  std::vector<std::shared_ptr<Request>> batch;
  std::atomic<bool> done{false};
  double t_done = 0;
  bool busy = false;
  // the batch's decode: next on the stream (inputs copied in), and ended
  cudaEvent_t ev_ready = nullptr, ev_done = nullptr;
};

}  // namespace

struct gmp_server {
  int device = 0;
  gmp_server_opts opts{};
  Arena arena;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;   // submitted, not admitted
  std::deque<std::shared_ptr<Request>> admitted;  // memory reserved, not launched
  std::unordered_map<uint64_t, std::shared_ptr<Request>> live;  // until released
  std::vector<gmp_completion> completed;
  uint64_t next_id = 1, in_system = 0;
  int error = 0;
  bool stop = false;
  Clock::time_point t0 = Clock::now();
  cudaEvent_t base = nullptr;  // device-clock origin of the completions' device times
  std::thread sched;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void loop();
  int launch(Lane& L, std::vector<std::shared_ptr<Request>>& reqs);
};

// Runs on the driver's callback thread when the lane's stream reaches the end
// of its batch.  It takes no lock (a later copy on the same stream may wait
// for this callback while the scheduler holds the mutex); the scheduler's
// timed wait picks the flag up if this notification races its wait.
static void CUDART_CB lane_done_cb(void* arg) {
  auto* pr = static_cast<std::pair<gmp_server*, Lane*>*>(arg);
  Lane* L = pr->second;
  L->t_done = pr->first->now();
  L->done.store(true, std::memory_order_release);
  pr->first->cv_work.notify_all();
  delete pr;
}

int gmp_server::launch(Lane& L, std::vector<std::shared_ptr<Request>>& reqs) {
  const size_t n = reqs.size();
  double ts = now();
  for (size_t i = 0; i < n; i++) {
    Request& r = *reqs[i];
    r.t_start = ts;
    if (cudaMemcpyAsync(arena.ptr(r.comp_off), r.host, r.bytes, cudaMemcpyHostToDevice, L.stream) != cudaSuccess)
      return GMP_ERR_CUDA;
    if (!r.index.empty() &&
        cudaMemcpyAsync(arena.ptr(r.index_off), r.index.data(), r.index.size() * sizeof(gmp_block_ref),
                        cudaMemcpyHostToDevice, L.stream) != cudaSuccess)
      return GMP_ERR_CUDA;
    gmp_file_desc& f = L.h_table[i];
    f.comp = arena.ptr(r.comp_off);
    f.comp_bytes = r.bytes;
    f.index = reinterpret_cast<const gmp_block_ref*>(arena.ptr(r.index_off));
    f.n_blocks = r.index.size();
    f.out = arena.ptr(r.out_off);
    f.out_cap = std::max<uint64_t>(r.info.orig_size, 1);
  }
  if (cudaMemcpyAsync(L.d_table, L.h_table, n * sizeof(gmp_file_desc), cudaMemcpyHostToDevice, L.stream) !=
      cudaSuccess)
    return GMP_ERR_CUDA;
  if (cudaEventRecord(L.ev_ready, L.stream) != cudaSuccess) return GMP_ERR_CUDA;
  int rc = gmp_decompress_batch(L.ctx, L.d_table, n, L.d_status, L.stream);
  if (rc) return rc;
  if (cudaEventRecord(L.ev_done, L.stream) != cudaSuccess) return GMP_ERR_CUDA;
  if (cudaMemcpyAsync(L.h_status, L.d_status, n * sizeof(int32_t), cudaMemcpyDeviceToHost, L.stream) != cudaSuccess)
    return GMP_ERR_CUDA;
  L.batch = reqs;
  L.busy = true;
  L.done.store(false);
  auto* arg = new std::pair<gmp_server*, Lane*>(this, &L);
  if (cudaLaunchHostFunc(L.stream, lane_done_cb, arg) != cudaSuccess) {
    delete arg;
    return GMP_ERR_CUDA;
  }
  return GMP_OK;
}

void gmp_server::loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    bool progressed = false;
    // 1. completions
    for (auto& Lp : lanes) {
      Lane& L = *Lp;
      if (L.busy && L.done.load(std::memory_order_acquire)) {
        // device times of the batch (both events completed before the
        // lane's completion function ran)
        float ms_ready = 0.f, ms_done = 0.f;
        cudaEventElapsedTime(&ms_ready, base, L.ev_ready);
        cudaEventElapsedTime(&ms_done, base, L.ev_done);
        for (size_t i = 0; i < L.batch.size(); i++) {
          Request& r = *L.batch[i];
          r.status = L.h_status[i];
          r.t_done = L.t_done;
          gmp_completion c;
          c.id = r.id;
          c.status = r.status;
          c.d_out = arena.ptr(r.out_off);
          c.out_bytes = r.info.orig_size;
          c.t_submit = r.t_submit;
          c.t_start = r.t_start;
          c.t_done = r.t_done;
          c.t_gpu_ready = ms_ready * 1e-3;
          c.t_gpu_done = ms_done * 1e-3;
          completed.push_back(c);
          in_system--;
        }
        L.batch.clear();
        L.busy = false;
        progressed = true;
        cv_done.notify_all();
      }
    }
    // 2. admission in arrival order while the arena has room
    while (!pending.empty()) {
      auto r = pending.front();
      uint64_t off = arena.alloc(r->need);
      if (off == UINT64_MAX) break;
      r->off = off;
      r->comp_off = off;
      r->index_off = off + Arena::round(r->bytes);
      r->out_off = r->index_off + Arena::round(std::max<size_t>(r->index.size(), 1) * sizeof(gmp_block_ref));
      admitted.push_back(r);
      pending.pop_front();
      progressed = true;
    }
    // 3. launch admitted requests on idle lanes (lanes are touched only by
    // this thread, so the copies and the launch run without the lock)
    for (auto& Lp : lanes) {
      if (admitted.empty()) break;
      Lane& L = *Lp;
      if (L.busy) continue;
      std::vector<std::shared_ptr<Request>> reqs;
      while (!admitted.empty() && reqs.size() < opts.max_batch) {
        reqs.push_back(admitted.front());
        admitted.pop_front();
      }
      lk.unlock();
      int rc = launch(L, reqs);
      lk.lock();
      progressed = true;
      if (rc) {
        error = rc;
        stop = true;
        cv_done.notify_all();
      }
    }
    if (stop) break;
    if (progressed) continue;
    // nothing to do right now: sleep (releasing the lock) until a submit, a
    // release, a lane completion or a short timeout
    bool any_busy = false;
    for (auto& Lp : lanes) any_busy |= Lp->busy;
    if (any_busy) cv_work.wait_for(lk, std::chrono::microseconds(200));
    else if (pending.empty() && admitted.empty())
      cv_work.wait(lk, [&] { return stop || !pending.empty() || !admitted.empty(); });
    else
      cv_work.wait_for(lk, std::chrono::milliseconds(2));  // waiting for memory to be released
    if (stop) break;
  }
  // drain in-flight work before exit
  lk.unlock();
  for (auto& Lp : lanes) cudaStreamSynchronize(Lp->stream);
}

extern "C" {

void gmp_server_opts_default(gmp_server_opts* o) {
  o->budget_bytes = 32ull << 30;
  // 8 lanes of up to 64 requests: with 4 lanes of 256 the lanes copied their
  // inputs in and then decoded in step with each other, so the host link and
  // the SMs took turns (closed-loop peak 220-228 GB/s against 256-261)
  o->n_lanes = 8;
  o->max_batch = 64;
  o->max_block_out = 256u << 10;
  o->warps_per_cta = 0;
}

int gmp_server_create(gmp_server** out, int device, const gmp_server_opts* opts) {
  if (!out) return GMP_ERR_INVALID_ARG;
  *out = nullptr;
  gmp_server_opts o;
  if (opts) o = *opts;
  else gmp_server_opts_default(&o);
  if (o.n_lanes == 0 || o.n_lanes > 64 || o.max_batch == 0 || o.budget_bytes == 0) return GMP_ERR_INVALID_ARG;
  std::unique_ptr<gmp_server> S(new (std::nothrow) gmp_server());
  if (!S) return GMP_ERR_NOMEM;
  S->device = device;
  S->opts = o;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  int rc = GMP_OK;
  if (!S->arena.init(o.budget_bytes)) rc = GMP_ERR_CUDA;
  for (uint32_t i = 0; i < o.n_lanes && rc == GMP_OK; i++) {
    auto L = std::make_unique<Lane>();
    gmp_context_opts co;
    gmp_context_opts_default(&co);
    co.max_block_out = o.max_block_out;
    co.warps_per_cta = o.warps_per_cta;
    co.max_files = o.max_batch;
    co.concurrent = 1;  // the lanes' batches overlap on the GPU
    rc = gmp_context_create(&L->ctx, device, &co);
    if (rc) break;
    if (cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&L->h_table, o.max_batch * sizeof(gmp_file_desc)) != cudaSuccess ||
        cudaMalloc(&L->d_table, o.max_batch * sizeof(gmp_file_desc)) != cudaSuccess ||
        cudaMallocHost(&L->h_status, o.max_batch * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&L->d_status, o.max_batch * sizeof(int32_t)) != cudaSuccess ||
        cudaEventCreate(&L->ev_ready) != cudaSuccess || cudaEventCreate(&L->ev_done) != cudaSuccess)
      rc = GMP_ERR_CUDA;
    S->lanes.push_back(std::move(L));
  }
  if (rc == GMP_OK &&
      (cudaEventCreate(&S->base) != cudaSuccess || cudaEventRecord(S->base, S->lanes[0]->stream) != cudaSuccess ||
       cudaEventSynchronize(S->base) != cudaSuccess))
    rc = GMP_ERR_CUDA;
  cudaSetDevice(prev);
  if (rc) {
    gmp_server_destroy(S.release());
    return rc;
  }
  gmp_server* raw = S.release();
  raw->sched = std::thread([raw] { raw->loop(); });
  *out = raw;
  return GMP_OK;
}

int gmp_server_submit(gmp_server* S, const void* host_stream, size_t bytes, uint64_t* id) {
  if (!S || !host_stream || !id) return GMP_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
  size_t nb = 0;
  int rc = gmp_index_build(host_stream, bytes, nullptr, 0, &nb, &r->info);
  if (rc) return rc;
  r->index.resize(nb);
  rc = gmp_index_build(host_stream, bytes, r->index.data(), nb, &nb, &r->info);
  if (rc) return rc;
  if (r->info.max_block_out > S->opts.max_block_out) return GMP_ERR_CAPACITY;
  r->host = static_cast<const uint8_t*>(host_stream);
  r->bytes = bytes;
  r->need = Arena::round(bytes) + Arena::round(std::max<size_t>(nb, 1) * sizeof(gmp_block_ref)) +
            Arena::round(std::max<uint64_t>(r->info.orig_size, 1));
  if (r->need > S->arena.size()) return GMP_ERR_CAPACITY;
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->error) return S->error;
    r->id = S->next_id++;
    r->t_submit = S->now();
    S->pending.push_back(r);
    S->live[r->id] = r;
    S->in_system++;
    *id = r->id;
  }
  S->cv_work.notify_all();
  return GMP_OK;
}

int gmp_server_poll(gmp_server* S, gmp_completion* out, size_t cap, size_t* n, int wait_ms) {
  if (!S || !n || (cap && !out)) return GMP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->completed.empty() && wait_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->completed.empty() || S->error; });
  size_t k = std::min(cap, S->completed.size());
  std::copy(S->completed.begin(), S->completed.begin() + k, out);
  S->completed.erase(S->completed.begin(), S->completed.begin() + k);
  *n = k;
  return S->error;
}

int gmp_server_release(gmp_server* S, uint64_t id) {
  if (!S) return GMP_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->live.find(id);
    if (it == S->live.end()) return GMP_ERR_INVALID_ARG;
    Request& r = *it->second;
    if (r.t_done == 0) return GMP_ERR_INVALID_ARG;  // not completed yet
    S->arena.release(r.off, r.need);
    S->live.erase(it);
  }
  S->cv_work.notify_all();
  return GMP_OK;
}

int gmp_server_drain(gmp_server* S) {
  if (!S) return GMP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv_done.wait(lk, [&] { return S->in_system == 0 || S->error; });
  return S->error;
}

int gmp_server_copy_out(gmp_server* S, uint64_t id, void* dst, size_t cap, int dst_is_device) {
  if (!S || (!dst && cap)) return GMP_ERR_INVALID_ARG;
  const uint8_t* src = nullptr;
  uint64_t n = 0;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->live.find(id);
    if (it == S->live.end() || it->second->t_done == 0) return GMP_ERR_INVALID_ARG;
    src = S->arena.ptr(it->second->out_off);
    n = std::min<uint64_t>(it->second->info.orig_size, cap);
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  cudaError_t e = n ? cudaMemcpy(dst, src, n, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost)
                    : cudaSuccess;
  cudaSetDevice(prev);
  return e == cudaSuccess ? GMP_OK : GMP_ERR_CUDA;
}

double gmp_server_now(gmp_server* S) { return S ? S->now() : 0.0; }

uint64_t gmp_server_bytes_in_use(gmp_server* S) {
  if (!S) return 0;
  std::lock_guard<std::mutex> g(S->mu);
  return S->arena.used();
}

void gmp_server_destroy(gmp_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->sched.joinable()) S->sched.join();
  for (auto& Lp : S->lanes) {
    Lane& L = *Lp;
    if (L.stream) cudaStreamSynchronize(L.stream);
    if (L.ctx) gmp_context_destroy(L.ctx);
    if (L.stream) cudaStreamDestroy(L.stream);
    if (L.h_table) cudaFreeHost(L.h_table);
    if (L.d_table) cudaFree(L.d_table);
    if (L.h_status) cudaFreeHost(L.h_status);
    if (L.d_status) cudaFree(L.d_status);
    if (L.ev_ready) cudaEventDestroy(L.ev_ready);
    if (L.ev_done) cudaEventDestroy(L.ev_done);
  }
  if (S->base) cudaEventDestroy(S->base);
  delete S;
}

}  // extern "C"
