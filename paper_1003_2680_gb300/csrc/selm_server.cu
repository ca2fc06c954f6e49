// Served form: a request loop that keeps each request's system resident on
// the device, admits requests by their device footprint and overlaps the
// work of the admitted ones.  Two loops share the queue, the pool and the
// admission rule:
//   * streams (selm_server_create): one worker thread and CUDA stream per
//     slot, each running its request alone;
//   * continuous batching (selm_server_create_batched): one scheduler runs
//     every admitted request's next Euler-Maruyama step as one batched step
//     (selm_batch over the requests' handles: shared graph launches, or the
//     persistent batched FAC launch whose work list holds one slot per
//     request).  Between steps finished requests leave and waiting ones are
//     admitted, and the batch is rebuilt over the new membership.
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
#include "selm_batch_internal.h"
#include "selm_handle.h"

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
  bool batched = false;               // continuous batching instead of per-slot streams
  bool persistent = true;             // batched: the persistent launch where the systems qualify
  long long batch_steps = 0, batch_rebuilds = 0;
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

// Continuous batching: one scheduler, one stream.  A tick admits waiting
// requests (arrival order, footprint in the pool, a free slot, the batch's
// dt and chain cycles per step), runs one Euler-Maruyama step of every
// active request as one batched step, and retires the requests whose steps
// are done.  A request's handle, particles and chain stay on the device from
// admission to retirement; the batch is rebuilt only when the membership
// changes.
struct Active {
  Pending job;
  void* block = nullptr;
  selm_mg* h = nullptr;
  int left = 0;
  double t_admit = 0.0;
};

void batched_loop(selm_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::vector<Active> active;
  selm_batch* batch = nullptr;
  bool changed = false;
  auto finish = [&](Active& a, selm_status status) {
    selm_result res{};
    res.id = a.job.id;
    res.user = a.job.req.user;
    res.t_submit = a.job.t_submit;
    res.t_admit = a.t_admit;
    res.status = status;
    if (a.h) {
      if (status == SELM_OK && a.job.req.np > 0) {
        const size_t bytes = (size_t)a.job.req.np * a.job.req.desc.dim * sizeof(double);
        if (cudaMemcpyAsync(a.job.req.X, a.h->Xs, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
          res.status = SELM_ECUDA;
      }
      long long total = 0;
      selm_mg_stats(a.h, nullptr, nullptr, &total);
      res.vcycles = (int)total;
    }
    res.t_done = s->now();
    if (a.h) selm_mg_destroy(a.h);
    a.h = nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    s->give(a.block, a.job.bytes);
    s->busy -= 1;
    s->done.push_back(res);
    s->outstanding -= 1;
  };
  for (;;) {
    std::vector<Active> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // the batch's first request fixes its dt and chain cycles per step
      auto ref = [&]() -> const selm_request* {
        if (!active.empty()) return &active.front().job.req;
        return admitted.empty() ? nullptr : &admitted.front().job.req;
      };
      auto fits = [&](const Pending& p) {
        if ((int)(active.size() + admitted.size()) >= s->max_slots) return false;
        if (s->largest_free() < ((p.bytes + 255) & ~(size_t)255)) return false;
        const selm_request* r0 = ref();
        return !r0 || (p.req.dt == r0->dt && p.req.ncycles_per_step == r0->ncycles_per_step);
      };
      if (active.empty())
        s->cv.wait(lk, [&] { return s->stop || (!s->queue.empty() && fits(s->queue.front())); });
      if (active.empty() && s->stop && (s->queue.empty() || !fits(s->queue.front()))) break;
      while (!s->queue.empty() && fits(s->queue.front())) {
        Active a;
        a.job = s->queue.front();
        s->queue.pop_front();
        a.block = s->take(a.job.bytes);
        a.left = a.job.req.nsteps;
        a.t_admit = s->now();
        s->busy += 1;
        s->peak_busy = s->busy > s->peak_busy ? s->busy : s->peak_busy;
        admitted.push_back(a);
      }
    }
    // set up the admitted requests' handles and particles (outside the lock)
    for (Active& a : admitted) {
      Grant g{a.block, a.job.bytes, false};
      selm_mg_desc d = a.job.req.desc;
      d.alloc = grant_alloc;
      d.free = grant_free;
      d.alloc_ctx = &g;
      if (d.max_particles < a.job.req.np) d.max_particles = a.job.req.np;
      selm_status status = selm_mg_create(&d, st, &a.h);
      if (status == SELM_OK && a.job.req.np > 0) {
        const size_t bytes = (size_t)a.job.req.np * d.dim * sizeof(double);
        if (cudaMemcpyAsync(a.h->Xs, a.job.req.X, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(a.h->Fs, a.job.req.F, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
          status = SELM_ECUDA;
      }
      if (status != SELM_OK || a.left == 0) {   // failed set-up, or no step to run
        finish(a, status);
        continue;
      }
      active.push_back(a);
      changed = true;
    }
    s->cv.notify_all();
    s->cv_done.notify_all();
    if (active.empty()) continue;
    if (changed || !batch) {
      if (batch) selm_batch_destroy(batch);
      batch = nullptr;
      std::vector<selm_mg*> hs;
      for (Active& a : active) hs.push_back(a.h);
      selm_status st_b = selm::batch_adopt((int)hs.size(), hs.data(), false, st, &batch);
      if (st_b == SELM_OK && !s->persistent) st_b = selm_batch_set_persistent(batch, 0);
      if (st_b != SELM_OK) {
        if (batch) selm_batch_destroy(batch);
        batch = nullptr;
        for (Active& a : active) finish(a, st_b);
        active.clear();
        s->cv.notify_all();
        s->cv_done.notify_all();
        continue;
      }
      changed = false;
      std::lock_guard<std::mutex> lk(s->mu);
      s->batch_rebuilds += 1;
    }
    std::vector<int> np;
    std::vector<double*> X;
    std::vector<const double*> F;
    for (Active& a : active) {
      np.push_back(a.job.req.np);
      X.push_back(a.h->Xs);
      F.push_back(a.h->Fs);
    }
    const selm_request& r0 = active.front().job.req;
    selm_status step = selm_batch_step(batch, np.data(), X.data(), F.data(), r0.dt, 1, r0.ncycles_per_step,
                                       nullptr, st);
    if (step == SELM_OK && cudaStreamSynchronize(st) != cudaSuccess) step = SELM_ECUDA;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->batch_steps += 1;
    }
    std::vector<Active> keep;
    for (Active& a : active) {
      a.left -= 1;
      if (step != SELM_OK || a.left == 0) {
        if (batch) {
          selm_batch_destroy(batch);   // the batch borrows the handles: release it first
          batch = nullptr;
        }
        finish(a, step);
        changed = true;
      } else {
        keep.push_back(a);
      }
    }
    active.swap(keep);
    s->cv.notify_all();
    s->cv_done.notify_all();
  }
  if (batch) selm_batch_destroy(batch);
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

selm_status selm_server_create_batched(size_t budget_bytes, int max_slots, int persistent, selm_server** out) {
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
  s->batched = true;
  s->persistent = persistent != 0;
  s->t0 = Clock::now();
  s->workers.emplace_back(batched_loop, s);
  *out = s;
  return SELM_OK;
}

selm_status selm_server_batch_stats(selm_server* s, long long* steps, long long* rebuilds) {
  if (!s) return SELM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (steps) *steps = s->batch_steps;
  if (rebuilds) *rebuilds = s->batch_rebuilds;
  return SELM_OK;
}

selm_status selm_server_submit(selm_server* s, const selm_request* r, uint64_t* id) {
  if (!s || !r || r->np < 0 || r->nsteps < 0 || (r->np > 0 && (!r->X || !r->F))) return SELM_EINVAL;
  if (s->batched && r->desc.projection != SELM_PROJ_NONE) return SELM_EINVAL;   // the batched form's systems
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
