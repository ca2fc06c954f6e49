// Served form: a request loop that keeps each request's system resident on
// the device, admits requests by their device footprint and overlaps the
// work of the admitted ones.
//
// One device pool of `budget` bytes is reserved at start; requests are taken
// in arrival order and admitted as soon as a contiguous block of their
// footprint (selm_mg_footprint) is free in the pool and a worker slot is
// idle, so memory released by a finishing request admits the next one while
// others are still running.  Each worker owns a CUDA stream and runs its
// request (selm_mg_step_host: copy in, nsteps Euler-Maruyama steps, copy
// out) independently of the others; the GPU overlaps the streams.  No device
// allocation or device-wide synchronisation happens in the loop (handles take
// their workspace from the pool), so one request's set-up or teardown does
// not stall the others.

#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/selm_mg.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
  uint64_t id;
  selm_request req;
  size_t bytes;
  double t_submit;
};

}  // namespace

struct selm_server {
  int device = 0;
  size_t budget = 0;
  char* pool = nullptr;
  std::map<size_t, size_t> free_blocks;   // offset -> size
  size_t in_use = 0, peak_in_use = 0;
  int max_slots = 1, busy = 0, peak_busy = 0;
  std::deque<Pending> queue;
  std::vector<selm_result> done;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv;         // queue / pool / slot changes
  std::condition_variable cv_done;    // a request finished
  bool stop = false;
  uint64_t next_id = 1;
  size_t outstanding = 0;
  Clock::time_point t0;
  std::string err;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  // first-fit sub-allocation from the pool (mu held)
  size_t largest_free() const {
    size_t m = 0;
    for (const auto& kv : free_blocks) m = kv.second > m ? kv.second : m;
    return m;
  }
  void* take(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, sz = it->second;
      free_blocks.erase(it);
      if (sz > bytes) free_blocks[off + bytes] = sz - bytes;
      in_use += bytes;
      peak_in_use = in_use > peak_in_use ? in_use : peak_in_use;
      return pool + off;
    }
    return nullptr;
  }
  void give(void* p, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    size_t off = (size_t)((char*)p - pool);
    in_use -= bytes;
    auto it = free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);   // merge with the next block
    if (nx != free_blocks.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_blocks.erase(nx);
    }
    if (it != free_blocks.begin()) {   // merge with the previous block
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_blocks.erase(it);
      }
    }
  }
};

namespace {

// Allocation hooks handed to the handles: one allocation per handle (its
// workspace), served from the pool block reserved at admission.
struct Grant {
  void* ptr;
  size_t bytes;
  bool used;
};

void* grant_alloc(size_t bytes, void* ctx) {
  Grant* g = (Grant*)ctx;
  if (g->used || bytes > g->bytes) return nullptr;
  g->used = true;
  return g->ptr;
}

void grant_free(void*, void*) {}

void worker_loop(selm_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Pending job;
    void* block = nullptr;
    double t_admit = 0.0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] {
        return s->stop || (!s->queue.empty() && s->largest_free() >= ((s->queue.front().bytes + 255) & ~(size_t)255));
      });
      if (s->stop && s->queue.empty()) break;
      if (s->stop && s->largest_free() < ((s->queue.front().bytes + 255) & ~(size_t)255)) break;
      job = s->queue.front();
      s->queue.pop_front();
      block = s->take(job.bytes);
      s->busy += 1;
      s->peak_busy = s->busy > s->peak_busy ? s->busy : s->peak_busy;
      t_admit = s->now();
    }
    s->cv.notify_all();
    selm_result res{};
    res.id = job.id;
    res.user = job.req.user;
    res.t_submit = job.t_submit;
    res.t_admit = t_admit;
    Grant g{block, job.bytes, false};
    selm_mg_desc d = job.req.desc;
    d.alloc = grant_alloc;
    d.free = grant_free;
    d.alloc_ctx = &g;
    if (d.max_particles < job.req.np) d.max_particles = job.req.np;
    selm_mg* h = nullptr;
    res.status = selm_mg_create(&d, st, &h);
    if (res.status == SELM_OK) {
      // a request's handle lives for a few steps (capturing graphs would not pay
      // off) and shares the GPU with the other slots (a mispredicted V-cycle
      // costs them)
      res.status = selm_mg_set_option(h, SELM_OPT_GRAPHS, 0);
      if (res.status == SELM_OK) res.status = selm_mg_set_option(h, SELM_OPT_SPECULATE, 0);
      if (res.status == SELM_OK)
        res.status = selm_mg_step_host(h, job.req.np, job.req.X, job.req.F, job.req.dt, job.req.nsteps,
                                       job.req.ncycles_per_step, st);
      long long total = 0;
      selm_mg_stats(h, nullptr, nullptr, &total);
      res.vcycles = (int)total;
      cudaStreamSynchronize(st);
      selm_mg_destroy(h);
    }
    res.t_done = s->now();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->give(block, job.bytes);
      s->busy -= 1;
      s->done.push_back(res);
      s->outstanding -= 1;
    }
    s->cv.notify_all();
    s->cv_done.notify_all();
  }
  cudaStreamDestroy(st);
}

size_t request_bytes(const selm_request* r) {
  selm_mg_desc d = r->desc;
  if (d.max_particles < r->np) d.max_particles = r->np;
  return selm_mg_footprint(&d);
}

}  // namespace

extern "C" {

selm_status selm_server_create(size_t budget_bytes, int max_slots, selm_server** out) {
  if (!out || budget_bytes < 4096 || max_slots < 1 || max_slots > 256) return SELM_EINVAL;
  *out = nullptr;
  selm_server* s = new (std::nothrow) selm_server();
  if (!s) return SELM_ENOMEM;
  cudaGetDevice(&s->device);
  s->budget = budget_bytes & ~(size_t)255;
  if (cudaMalloc((void**)&s->pool, s->budget) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return SELM_ENOMEM;
  }
  s->free_blocks[0] = s->budget;
  s->max_slots = max_slots;
  s->t0 = Clock::now();
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker_loop, s);
  *out = s;
  return SELM_OK;
}

selm_status selm_server_submit(selm_server* s, const selm_request* r, uint64_t* id) {
  if (!s || !r || r->np < 0 || r->nsteps < 0 || (r->np > 0 && (!r->X || !r->F))) return SELM_EINVAL;
  const size_t bytes = request_bytes(r);
  if (bytes == 0) return SELM_EINVAL;
  if (((bytes + 255) & ~(size_t)255) > s->budget) return SELM_EBUSY;   // could never be admitted
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Pending p{s->next_id++, *r, bytes, s->now()};
    if (id) *id = p.id;
    s->queue.push_back(p);
    s->outstanding += 1;
  }
  s->cv.notify_all();
  return SELM_OK;
}

int selm_server_poll(selm_server* s, selm_result* out, int max) {
  if (!s || !out || max <= 0) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  int n = 0;
  while (n < max && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.erase(s->done.begin());
  }
  return n;
}

selm_status selm_server_drain(selm_server* s) {
  if (!s) return SELM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->outstanding == 0; });
  return SELM_OK;
}

selm_status selm_server_stats(selm_server* s, size_t* peak_bytes, int* peak_slots, size_t* bytes_in_use,
                              int* queued) {
  if (!s) return SELM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (peak_bytes) *peak_bytes = s->peak_in_use;
  if (peak_slots) *peak_slots = s->peak_busy;
  if (bytes_in_use) *bytes_in_use = s->in_use;
  if (queued) *queued = (int)s->queue.size();
  return SELM_OK;
}

double selm_server_clock(selm_server* s) { return s ? s->now() : 0.0; }

selm_status selm_server_destroy(selm_server* s) {
  if (!s) return SELM_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  for (auto& t : s->workers) t.join();
  cudaFree(s->pool);
  delete s;
  return SELM_OK;
}

}  // extern "C"
