// Batched form: many independent channel systems of uneven sizes advanced
// together (Algorithm 4 for each system).
//
// Each phase of an Euler-Maruyama step is captured once as a CUDA graph whose
// branches are the systems (one forked stream per system during capture), so
// one graph launch runs that phase for every system and the GPU schedules the
// systems' kernels -- in particular their cluster-resident coarse engines,
// each of which fills only part of the GPU -- side by side.  The FAC solve
// (Algorithm 1) runs one graph launch per V-cycle for all systems; that graph
// ends with each system's next residual norm copied to pinned host memory,
// from which the host decides whether another cycle is needed.  Systems that
// have already met their tolerance take the extra cycles of the slowest
// system (their iterates only get more accurate).
//
// The engine's thread-block cluster size is chosen by an autotuner that times
// the batched V-cycle graph for each candidate.
//
// Persistent form (the default when every system qualifies: one inner
// precision, the exact coarsest step, level-0 rows in 8-wide segments): each
// FAC cycle of all systems -- a solve cycle or a chain cycle -- is one
// cooperative launch that walks the cycle's phases for every system with grid
// barriers between phases (batch_persist_launch); the solve's per-cycle graph
// is that launch plus one strided copy of all residual norms, and the chain
// graph holds the step's chain cycles.  Its autotuner times the launch over
// tile shapes (z rows per level-0 column item, co-resident blocks per SM).

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "../../include/selm_mg.h"
#include "selm_batch_internal.h"
#include "selm_handle.h"
#include "selm_launch.h"
#include "selm_prof.h"

using namespace selm;

struct selm_batch {
  int n = 0;
  std::vector<selm_mg*> sys;
  std::vector<cudaStream_t> branch;   // capture branches, one per system
  cudaStream_t origin = nullptr;      // capture origin
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  double* host_norm = nullptr;        // pinned [n][2]: ||r||^2, ||b||^2
  // captured graphs
  cudaGraphExec_t g_start = nullptr;  // spread + initial residual and norms
  cudaGraphExec_t g_cycle = nullptr;  // one V-cycle + update + next residual norm
  cudaGraphExec_t g_chain = nullptr;  // k stochastic cycles of every chain
  cudaGraphExec_t g_finish = nullptr; // combine, interpolate, move particles
  // kernels each graph holds: recorded at capture (where nothing runs) and
  // credited to the launch counter on every replay
  long long k_start = 0, k_cycle = 0, k_chain = 0, k_finish = 0;
  // arguments baked into the graphs
  std::vector<int> np;
  std::vector<double*> X;
  std::vector<const double*> F;
  double dt = -1.0;
  int kchain = -1;
  int cluster = 0;
  BatchPersist* bp = nullptr;   // persistent form (null: per-system graphs only)
  bool persistent = false;
  unsigned* host_flag = nullptr;  // pinned copy of the persistent launches' timeout word
  bool owns = true;               // false: the systems are borrowed (batch_adopt) and outlive the batch
  std::string err;
};

namespace {

#define BCK(call)                                                 \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) {                                      \
      b->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return SELM_ECUDA;                                          \
    }                                                             \
  } while (0)

#define BST(expr)                      \
  do {                                 \
    selm_status s_ = (expr);           \
    if (s_ != SELM_OK) return s_;      \
  } while (0)

// Inside capture lambdas: record the failing call on the batch.
#define LCK(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      b->err = std::string(#call) + " (system " + std::to_string(i) + "): " + cudaGetErrorString(e_); \
      return SELM_ECUDA;                                                            \
    }                                                                               \
  } while (0)
#define LST(expr)                                                                     \
  do {                                                                                \
    selm_status s_ = (expr);                                                          \
    if (s_ != SELM_OK) {                                                              \
      b->err = std::string(#expr) + " (system " + std::to_string(i) + "): " + b->sys[i]->err; \
      return s_;                                                                      \
    }                                                                                 \
  } while (0)

void drop_graphs(selm_batch* b) {
  for (cudaGraphExec_t* g : {&b->g_start, &b->g_cycle, &b->g_chain, &b->g_finish}) {
    if (*g) cudaGraphExecDestroy(*g);
    *g = nullptr;
  }
}

// Captures fn(i, stream_i) for every system as parallel branches of one graph.
template <typename Fn>
selm_status capture(selm_batch* b, Fn fn, cudaGraphExec_t* out, long long* kernels) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  const long long l0 = prof::g_launches.load();
  BCK(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
  selm_status st = SELM_OK;
  cudaError_t ce = cudaEventRecord(b->fork, b->origin);
  for (int i = 0; i < b->n && ce == cudaSuccess && st == SELM_OK; ++i) {
    ce = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
    if (ce != cudaSuccess) break;
    st = fn(i, b->branch[i]);
    if (st != SELM_OK) break;
    ce = cudaEventRecord(b->join[i], b->branch[i]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->origin, b->join[i], 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t ce2 = cudaStreamEndCapture(b->origin, &graph);
  *kernels = prof::g_launches.load() - l0;
  prof::g_launches.fetch_sub(*kernels);   // recorded, not run
  if (st != SELM_OK || ce != cudaSuccess || ce2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (st == SELM_OK) {
      b->err = std::string("graph capture failed: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ce2);
      st = SELM_ECUDA;
    }
    return st;
  }
  ce = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    b->err = std::string("graph instantiation failed: ") + cudaGetErrorString(ce);
    return SELM_ECUDA;
  }
  return SELM_OK;
}

// Residual of system i's solve and its squared norm copied to pinned memory.
selm_status residual_norm(selm_batch* b, int i, cudaStream_t s) {
  selm_mg* h = b->sys[i];
  LCK(cudaMemsetAsync(h->red + 1, 0, sizeof(double), s));
  LST(outer_residual(h, h->vel, h->u, h->bvel, h->vel.b[0], h->red + 1, s));
  LCK(cudaMemcpyAsync(b->host_norm + 2 * i, h->red + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  return SELM_OK;
}

// Captures fn(stream) on the origin stream alone (the persistent form).
template <typename Fn>
selm_status capture_single(selm_batch* b, Fn fn, cudaGraphExec_t* out, long long* kernels) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  const long long l0 = prof::g_launches.load();
  BCK(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
  const cudaError_t ce = fn(b->origin);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce2 = cudaStreamEndCapture(b->origin, &graph);
  *kernels = prof::g_launches.load() - l0;
  prof::g_launches.fetch_sub(*kernels);   // recorded, not run
  if (ce != cudaSuccess || ce2 != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    b->err = std::string("graph capture failed: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ce2);
    return SELM_ECUDA;
  }
  const cudaError_t ce3 = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (ce3 != cudaSuccess) {
    b->err = std::string("graph instantiation failed: ") + cudaGetErrorString(ce3);
    return SELM_ECUDA;
  }
  return SELM_OK;
}

selm_status build_cycle_graph(selm_batch* b) {
  if (b->persistent) {
    // one pipelined solve cycle of every system, then all residual norms to
    // host_norm[2 i]
    return capture_single(
        b,
        [&](cudaStream_t s) -> cudaError_t {
          cudaError_t e = batch_persist_launch(b->bp, 1, s);
          if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(b->host_norm, 2 * sizeof(double), batch_persist_norms(b->bp), sizeof(double),
                                  sizeof(double), b->n, cudaMemcpyDeviceToHost, s);
          if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->host_flag, batch_persist_bar(b->bp) + 2, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                s);
          return e;
        },
        &b->g_cycle, &b->k_cycle);
  }
  return capture(
      b,
      [&](int i, cudaStream_t s) -> selm_status {
        selm_mg* h = b->sys[i];
        const size_t inner = (size_t)h->vel.lev[0].size * h->esize;
        LCK(cudaMemsetAsync(h->vel.v[0], 0, inner, s));
        LST(vcycle(h, h->vel, h->vel.v[0], h->vel.b[0], false, h->cyc + 1, s));
        LST(outer_update(h, h->vel, h->u, h->vel.v[0], s));
        return residual_norm(b, i, s);
      },
      &b->g_cycle, &b->k_cycle);
}

selm_status build_graphs(selm_batch* b, const int* np, double* const* X, const double* const* F, double dt,
                         int kchain) {
  drop_graphs(b);
  for (int i = 0; i < b->n; ++i) {
    b->np[i] = np[i];
    b->X[i] = X[i];
    b->F[i] = F[i];
  }
  b->dt = dt;
  b->kchain = kchain;
  BST(capture(
      b,
      [&](int i, cudaStream_t s) -> selm_status {
        selm_mg* h = b->sys[i];
        const size_t nv = (size_t)h->vel.lev[0].size * sizeof(double);
        LCK(cudaMemsetAsync(h->bvel, 0, nv, s));
        LCK(launch_spread(h->vel.lev[0], h->d.n, h->d.dim, np[i], X[i], F[i], h->bvel, s));
        LCK(cudaMemsetAsync(h->u, 0, nv, s));
        LCK(cudaMemsetAsync(h->vel.v[0], 0, (size_t)h->vel.lev[0].size * h->esize, s));
        LCK(cudaMemsetAsync(h->red, 0, sizeof(double), s));
        LCK(launch_norm2(h->vel.lev[0].size, h->bvel, h->red, s));
        LCK(cudaMemcpyAsync(b->host_norm + 2 * i + 1, h->red, sizeof(double), cudaMemcpyDeviceToHost, s));
        return residual_norm(b, i, s);
      },
      &b->g_start, &b->k_start));
  BST(build_cycle_graph(b));
  if (b->persistent)
    BST(capture_single(
        b,
        [&](cudaStream_t s) -> cudaError_t {
          for (int q = 0; q < kchain; ++q) {
            cudaError_t e = batch_persist_launch(b->bp, 0, s);
            // a timed-out barrier of any chain cycle stays visible until the
            // next step's first read-back
            if (e == cudaSuccess)
              e = cudaMemcpyAsync(b->host_flag + 1, batch_persist_bar(b->bp) + 2, sizeof(unsigned),
                                  cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return e;
          }
          return cudaSuccess;
        },
        &b->g_chain, &b->k_chain));
  else
  BST(capture(
      b,
      [&](int i, cudaStream_t s) -> selm_status {
        selm_mg* h = b->sys[i];
        const size_t inner = (size_t)h->vel.lev[0].size * h->esize;
        for (int q = 0; q < kchain; ++q) {
          LST(outer_residual(h, h->vel, h->xi, nullptr, h->vel.b[0], nullptr, s));
          LCK(cudaMemsetAsync(h->vel.v[0], 0, inner, s));
          LST(vcycle(h, h->vel, h->vel.v[0], h->vel.b[0], true, h->cyc + 0, s));
          LST(outer_update(h, h->vel, h->xi, h->vel.v[0], s));
          LCK(launch_inc_u64(h->cyc + 0, s));
        }
        return SELM_OK;
      },
      &b->g_chain, &b->k_chain));
  BST(capture(
      b,
      [&](int i, cudaStream_t s) -> selm_status {
        selm_mg* h = b->sys[i];
        const long long nv = h->vel.lev[0].size;
        LCK(launch_axpby(nv, dt, h->u, std::sqrt(2.0 * h->d.kT * dt), h->xi, h->wcomb, s));
        LCK(launch_interp(h->vel.lev[0], h->d.n, h->d.dim, np[i], X[i], h->wcomb, h->V, s));
        LCK(launch_em(np[i], h->d.dim, X[i], h->V, s));
        return SELM_OK;
      },
      &b->g_finish, &b->k_finish));
  return SELM_OK;
}

bool same_args(const selm_batch* b, const int* np, double* const* X, const double* const* F, double dt,
               int kchain) {
  if (!b->g_start || b->dt != dt || b->kchain != kchain) return false;
  for (int i = 0; i < b->n; ++i)
    if (b->np[i] != np[i] || b->X[i] != X[i] || b->F[i] != F[i]) return false;
  return true;
}

// A grid barrier of a persistent launch that gave up (its bounded wait ran
// out) leaves that launch's results undefined: reported once, then cleared.
selm_status check_timeout(selm_batch* b) {
  if (!b->persistent || !b->host_flag || (b->host_flag[0] == 0u && b->host_flag[1] == 0u)) return SELM_OK;
  b->host_flag[0] = b->host_flag[1] = 0u;
  b->err = "a grid barrier of the persistent batched launch timed out";
  return SELM_ECUDA;
}

bool all_converged(const selm_batch* b, std::vector<int>& cycles, int cyc) {
  bool all = true;
  for (int i = 0; i < b->n; ++i) {
    const double rn2 = b->host_norm[2 * i], bn2 = b->host_norm[2 * i + 1];
    const bool ok = bn2 == 0.0 || std::sqrt(rn2) <= b->sys[i]->d.tol * std::sqrt(bn2);
    if (ok && cycles[i] < 0) cycles[i] = cyc;
    all = all && ok;
  }
  return all;
}

}  // namespace

namespace selm {

selm_status batch_adopt(int nsys, selm_mg* const* hs, bool owns, void* stream, selm_batch** out) {
  if (nsys < 1 || !hs || !out) return SELM_EINVAL;
  *out = nullptr;
  for (int i = 0; i < nsys; ++i)
    if (!hs[i] || hs[i]->d.projection != SELM_PROJ_NONE) return SELM_EINVAL;
  selm_batch* b = new (std::nothrow) selm_batch();
  if (!b) return SELM_ENOMEM;
  b->owns = false;   // until set-up succeeds the caller keeps the systems
  b->n = nsys;
  b->np.assign(nsys, 0);
  b->X.assign(nsys, nullptr);
  b->F.assign(nsys, nullptr);
  for (int i = 0; i < nsys; ++i) {
    selm_mg* h = hs[i];
    // The systems' graph branches run side by side: each keeps its levels in
    // its own cluster engine (cooperative launches would take every SM).
    h->vel.use_coop = false;
    h->pres.use_coop = false;
    b->sys.push_back(h);
    selm_status st = selm::replan_engine(h, 0, stream ? (cudaStream_t)stream : nullptr);
    if (st != SELM_OK) {
      selm_batch_destroy(b);
      return st;
    }
  }
  bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaMallocHost((void**)&b->host_norm, 2 * sizeof(double) * nsys) == cudaSuccess;
  for (int i = 0; i < nsys && ok; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    b->branch.push_back(s);
    b->join.push_back(e);
  }
  if (!ok) {
    cudaGetLastError();
    selm_batch_destroy(b);
    return SELM_ENOMEM;
  }
  // persistent form, when every system qualifies
  {
    std::vector<BatchSysHost> hb(nsys);
    bool same = true;
    for (int i = 0; i < nsys; ++i) {
      selm_mg* h = b->sys[i];
      BatchSysHost& q = hb[i];
      q.levels = h->vel.levels;
      q.esize = h->esize;
      q.cholesky = h->d.coarse_mode == SELM_COARSE_CHOLESKY;
      q.lev = h->vel.lev;
      q.v = h->vel.v;
      q.b = h->vel.b;
      q.t = h->vel.t;
      q.key = h->key;
      q.cyc = h->cyc;
      q.u = h->u;
      q.xi = h->xi;
      q.bvel = h->bvel;
      same = same && h->mu1 == b->sys[0]->mu1 && h->mu2 == b->sys[0]->mu2;
    }
    if (same && batch_persist_eligible(nsys, hb.data()) &&
        cudaMallocHost((void**)&b->host_flag, 2 * sizeof(unsigned)) == cudaSuccess) {
      b->host_flag[0] = b->host_flag[1] = 0u;
      cudaStreamSynchronize(stream ? (cudaStream_t)stream : nullptr);
      if (batch_persist_create(nsys, hb.data(), b->sys[0]->mu1, b->sys[0]->mu2, &b->bp) == cudaSuccess)
        b->persistent = true;
      cudaGetLastError();
    }
  }
  b->owns = owns;
  *out = b;
  return SELM_OK;
}

}  // namespace selm

extern "C" {

selm_status selm_batch_create(int nsys, const selm_mg_desc* descs, void* stream, selm_batch** out) {
  if (nsys < 1 || !descs || !out) return SELM_EINVAL;
  *out = nullptr;
  for (int i = 0; i < nsys; ++i)
    if (descs[i].projection != SELM_PROJ_NONE) {
      std::fprintf(stderr, "selm_batch_create: the batched form runs SELM_PROJ_NONE systems\n");
      return SELM_EINVAL;
    }
  std::vector<selm_mg*> hs;
  for (int i = 0; i < nsys; ++i) {
    selm_mg* h = nullptr;
    selm_status st = selm_mg_create(&descs[i], stream, &h);
    if (st != SELM_OK) {
      for (selm_mg* q : hs) selm_mg_destroy(q);
      return st;
    }
    hs.push_back(h);
  }
  selm_status st = selm::batch_adopt(nsys, hs.data(), true, stream, out);
  if (st != SELM_OK)
    for (selm_mg* q : hs) selm_mg_destroy(q);
  return st;
}

selm_status selm_batch_destroy(selm_batch* b) {
  if (!b) return SELM_EINVAL;
  cudaDeviceSynchronize();
  drop_graphs(b);
  if (b->owns)
    for (selm_mg* h : b->sys) selm_mg_destroy(h);
  for (cudaStream_t s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->host_norm) cudaFreeHost(b->host_norm);
  batch_persist_destroy(b->bp);
  if (b->host_flag) cudaFreeHost(b->host_flag);
  delete b;
  return SELM_OK;
}

selm_mg* selm_batch_system(selm_batch* b, int i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->sys[i];
}

const char* selm_batch_last_error(const selm_batch* b) { return b ? b->err.c_str() : "null batch"; }

selm_status selm_batch_step(selm_batch* b, const int* np, double* const* X, const double* const* F, double dt,
                            int nsteps, int ncycles_per_step, int* solve_cycles, void* stream) {
  if (!b || !np || !X || !F || nsteps < 0 || ncycles_per_step < 0 || !(dt >= 0.0)) return SELM_EINVAL;
  for (int i = 0; i < b->n; ++i)
    if (np[i] < 0 || np[i] > b->sys[i]->d.max_particles || (np[i] > 0 && (!X[i] || !F[i]))) return SELM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!same_args(b, np, X, F, dt, ncycles_per_step)) BST(build_graphs(b, np, X, F, dt, ncycles_per_step));
  int max_cycles = 0;
  for (selm_mg* h : b->sys) max_cycles = max_cycles > h->d.max_cycles ? max_cycles : h->d.max_cycles;
  std::vector<int> cycles(b->n, -1);
  for (int step = 0; step < nsteps; ++step) {
    std::fill(cycles.begin(), cycles.end(), -1);
    BCK(cudaGraphLaunch(b->g_start, st));
    prof::g_launches.fetch_add(b->k_start);
    BCK(cudaStreamSynchronize(st));
    BST(check_timeout(b));
    int cyc = 0;
    while (!all_converged(b, cycles, cyc)) {
      if (cyc >= max_cycles) {
        b->err = "batched FAC solve did not converge";
        return SELM_ENOCONV;
      }
      BCK(cudaGraphLaunch(b->g_cycle, st));
      prof::g_launches.fetch_add(b->k_cycle);
      BCK(cudaStreamSynchronize(st));
      BST(check_timeout(b));
      ++cyc;
      for (selm_mg* h : b->sys) h->total_vcycles += 1;
    }
    if (ncycles_per_step > 0) {
      BCK(cudaGraphLaunch(b->g_chain, st));
      prof::g_launches.fetch_add(b->k_chain);
      for (selm_mg* h : b->sys) {
        h->cycle += ncycles_per_step;
        h->total_vcycles += ncycles_per_step;
      }
    }
    BCK(cudaGraphLaunch(b->g_finish, st));
    prof::g_launches.fetch_add(b->k_finish);
    for (int i = 0; i < b->n; ++i) b->sys[i]->last_solve_cycles = cycles[i];
  }
  if (solve_cycles)
    for (int i = 0; i < b->n; ++i) solve_cycles[i] = cycles[i];
  return SELM_OK;
}

selm_status selm_batch_cycle(selm_batch* b, int mode, void* stream) {
  if (!b || (mode != SELM_BATCH_SOLVE && mode != SELM_BATCH_SAMPLE)) return SELM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (b->persistent) {
    BCK(batch_persist_launch(b->bp, mode == SELM_BATCH_SAMPLE ? 0 : 2, st));
    for (selm_mg* h : b->sys) {
      if (mode == SELM_BATCH_SAMPLE) h->cycle += 1;
      h->total_vcycles += 1;
    }
    return SELM_OK;
  }
  BCK(cudaEventRecord(b->fork, st));
  for (int i = 0; i < b->n; ++i) {
    selm_mg* h = b->sys[i];
    cudaStream_t s = b->branch[i];
    const size_t inner = (size_t)h->vel.lev[0].size * h->esize;
    BCK(cudaStreamWaitEvent(s, b->fork, 0));
    if (mode == SELM_BATCH_SAMPLE) {
      LST(outer_residual(h, h->vel, h->xi, nullptr, h->vel.b[0], nullptr, s));
      LCK(cudaMemsetAsync(h->vel.v[0], 0, inner, s));
      LST(vcycle(h, h->vel, h->vel.v[0], h->vel.b[0], true, h->cyc + 0, s));
      LST(outer_update(h, h->vel, h->xi, h->vel.v[0], s));
      LCK(launch_inc_u64(h->cyc + 0, s));
      h->cycle += 1;
    } else {
      LST(outer_residual(h, h->vel, h->u, h->bvel, h->vel.b[0], nullptr, s));
      LCK(cudaMemsetAsync(h->vel.v[0], 0, inner, s));
      LST(vcycle(h, h->vel, h->vel.v[0], h->vel.b[0], false, h->cyc + 1, s));
      LST(outer_update(h, h->vel, h->u, h->vel.v[0], s));
    }
    BCK(cudaEventRecord(b->join[i], s));
    BCK(cudaStreamWaitEvent(st, b->join[i], 0));
  }
  return SELM_OK;
}

selm_status selm_batch_autotune(selm_batch* b, int* chosen_cluster, void* stream) {
  if (!b) return SELM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  BCK(cudaStreamSynchronize(st));   // no batched graph may still be running
  float best_p = -1.0f;
  if (b->bp) {
    // tile shapes of the persistent launch: z rows per level-0 column item x
    // co-resident blocks per SM, each timed over solve cycles of every system
    // (the iterates u are reset at the start of every step)
    const int kcs[3] = {8, 16, 32}, bpss[2] = {1, 2};
    int best_kc = 16, best_bps = 1;
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    for (int kc : kcs)
      for (int bps : bpss) {
        BCK(batch_persist_configure(b->bp, kc, bps));
        int got_kc = 0, got_bps = 0;
        batch_persist_shape(b->bp, &got_kc, &got_bps);
        if (got_bps != bps) continue;   // that many blocks do not fit on an SM
        BCK(batch_persist_launch(b->bp, 2, st));   // warm-up
        BCK(cudaEventRecord(e0, st));
        for (int r = 0; r < 3; ++r) BCK(batch_persist_launch(b->bp, 2, st));
        prof::g_launches.fetch_add(4);
        BCK(cudaEventRecord(e1, st));
        BCK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        BCK(cudaEventElapsedTime(&ms, e0, e1));
        if (best_p < 0.0f || ms < best_p) {
          best_p = ms;
          best_kc = kc;
          best_bps = bps;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BCK(batch_persist_configure(b->bp, best_kc, best_bps));
    BST(check_timeout(b));
  }
  // the per-system graph form over engine cluster sizes; the faster form wins
  b->persistent = false;
  const int cands[3] = {16, 8, 4};
  float best = -1.0f;
  int best_c = 0;
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  for (int c : cands) {
    for (selm_mg* h : b->sys) BST(replan_engine(h, c, nullptr));
    BST(build_cycle_graph(b));
    BCK(cudaGraphLaunch(b->g_cycle, st));   // warm-up
    BCK(cudaEventRecord(e0, st));
    for (int r = 0; r < 3; ++r) BCK(cudaGraphLaunch(b->g_cycle, st));
    prof::g_launches.fetch_add(4 * b->k_cycle);
    BCK(cudaEventRecord(e1, st));
    BCK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    BCK(cudaEventElapsedTime(&ms, e0, e1));
    if (best < 0.0f || ms < best) {
      best = ms;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (selm_mg* h : b->sys) BST(replan_engine(h, best_c, nullptr));
  drop_graphs(b);   // graphs are rebuilt with the chosen plans on the next step
  b->cluster = best_c;
  if (chosen_cluster) *chosen_cluster = best_c;
  // both forms were timed over 3 solve cycles of every system
  b->persistent = b->bp && (best_p >= 0.0f && best_p < best);
  return SELM_OK;
}

selm_status selm_batch_set_persistent(selm_batch* b, int on) {
  if (!b) return SELM_EINVAL;
  if (on && !b->bp) return SELM_EINVAL;
  cudaDeviceSynchronize();
  drop_graphs(b);
  b->persistent = on != 0;
  return SELM_OK;
}

selm_status selm_batch_info(const selm_batch* b, int* persistent, int* kc, int* blocks_per_sm, int* cluster) {
  if (!b) return SELM_EINVAL;
  int k = 0, bps = 0;
  batch_persist_shape(b->bp, &k, &bps);
  if (persistent) *persistent = b->persistent ? 1 : 0;
  if (kc) *kc = k;
  if (blocks_per_sm) *blocks_per_sm = bps;
  if (cluster) *cluster = b->cluster;
  return SELM_OK;
}

selm_status selm_batch_phase_times(selm_batch* b, int mode, int max_phases, int* types, int* levels, double* us,
                                   int* nphases, void* stream) {
  if (!b || !b->bp || (mode != SELM_BATCH_SOLVE && mode != SELM_BATCH_SAMPLE) || max_phases < 0) return SELM_EINVAL;
  const int kind = mode == SELM_BATCH_SAMPLE ? 0 : 2;
  const int n = batch_persist_phases(b->bp, kind, nullptr, nullptr);
  if (nphases) *nphases = n;
  if (!types || !levels || !us) return SELM_OK;   // count query
  if (n > max_phases) return SELM_EINVAL;
  std::vector<int> t(n), l(n);
  batch_persist_phases(b->bp, kind, t.data(), l.data());
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* d = nullptr;
  BCK(cudaMalloc(&d, (n + 1) * sizeof(unsigned long long)));
  std::vector<unsigned long long> h(n + 1, 0ull);
  cudaError_t e = batch_persist_launch(b->bp, kind, st, d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, (n + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) {
    b->err = std::string("phase timing: ") + cudaGetErrorString(e);
    return SELM_ECUDA;
  }
  prof::g_launches.fetch_add(1);
  if (mode == SELM_BATCH_SAMPLE)
    for (selm_mg* hh : b->sys) hh->cycle += 1;
  for (int p = 0; p < n; ++p) {
    types[p] = t[p];
    levels[p] = l[p];
    us[p] = 1e-3 * (double)(h[p + 1] - h[p]);
  }
  return check_timeout(b);
}

}  // extern "C"
