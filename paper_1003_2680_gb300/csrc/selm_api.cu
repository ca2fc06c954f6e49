// C ABI of the stochastic multigrid SELM library: handle management and the
// host orchestration of Algorithms 1, 3 and 4 on a caller-given stream.
//
// All device state of a handle (Galerkin tables, level fields, FP64 outer
// fields, reduction slots, particle scratch) lives in one workspace block
// whose layout is computed on the host; the block comes from the caller's
// allocator hooks or cudaMalloc.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/selm_mg.h"
#include "selm_coarse.h"
#include "selm_handle.h"
#include "selm_prof.h"
#include "selm_internal.h"
#include "selm_launch.h"

using namespace selm;

namespace {

void fill_desc_defaults(selm_mg_desc* d) {
  if (d->levels == 0) d->levels = default_levels(d->n);
  if (d->nu_pre == 0) d->nu_pre = 2;
  if (d->nu_post == 0) d->nu_post = 2;
  if (d->tol == 0.0) d->tol = 1e-10;
  if (d->max_cycles == 0) d->max_cycles = 100;
  if (d->proj_tol == 0.0) d->proj_tol = 1e-10;
  if (d->max_particles == 0) d->max_particles = 4096;
}

std::string validate(const selm_mg_desc& d) {
  if (d.dim != 2 && d.dim != 3) return "dim must be 2 or 3";
  if (d.n < 4) return "n must be at least 4";
  if (!(d.mu > 0.0)) return "mu must be positive";
  if (!(d.kT >= 0.0)) return "kT must be non-negative";
  if (d.nu_pre < 0 || d.nu_post < 0 || d.nu_pre + d.nu_post > 64) return "invalid smoothing counts";
  if (d.precision != SELM_FP64 && d.precision != SELM_FP32_REFINE64) return "invalid precision";
  if (d.projection != SELM_PROJ_NONE && d.projection != SELM_PROJ_MAC) return "invalid projection";
  if (d.coarse_mode != SELM_COARSE_CHOLESKY && d.coarse_mode != SELM_COARSE_SMOOTH) return "invalid coarse_mode";
  if (!(d.tol > 0.0) || !(d.proj_tol > 0.0)) return "tolerances must be positive";
  if (d.max_cycles < 1 || d.max_particles < 1) return "max_cycles and max_particles must be positive";
  return "";
}

std::string build_systems(const selm_mg_desc& d, Sys* vel, Sys* pres, bool* has_pres) {
  std::string e = build_velocity_system(d.dim, d.n, d.levels, d.mu, &vel->host);
  if (!e.empty()) return "velocity system: " + e;
  *has_pres = d.projection == SELM_PROJ_MAC;
  if (*has_pres) {
    e = build_pressure_system(d.dim, d.n, d.levels, &pres->host);
    if (!e.empty()) return "pressure system: " + e;
  }
  if (d.coarse_mode == SELM_COARSE_SMOOTH) {
    const HostSystem* ss[2] = {&vel->host, *has_pres ? &pres->host : nullptr};
    for (const HostSystem* s : ss) {
      if (!s) continue;
      for (const auto& c : s->lev[s->levels - 1])
        for (int a = 0; a < 2; ++a)
          if (c.dims[a] > 1 && c.dims[a] % c.mods[a] != 0)
            return "coarsest level too small for a valid colouring in smooth mode";
    }
  }
  return "";
}

struct TableOffsets {
  size_t S64, S32, rzw64, rzw32, pzw64, pzw32, rzi, pzi, Linv, zb64, zb32;
};

// Workspace plan: tables + fields.  When `base` is null only sizes are computed.
struct Plan {
  Layout lay;
  std::vector<double> dbl;
  std::vector<float> flt;
  std::vector<int> ints;
  size_t dbl_off = 0, flt_off = 0, int_off = 0;
  std::vector<TableOffsets> toff[2][kMaxLevels];
  size_t field_off[3][kMaxLevels][3];   // velocity, pressure, the chain's velocity copy
  size_t u_off = 0, xi_off = 0, bvel_off = 0, wcomb_off = 0, phi_off = 0, prhs_off = 0, red_off = 0,
         cyc_off = 0, V_off = 0, Xs_off = 0, Fs_off = 0, eng_off[3] = {0, 0, 0}, spec_off = 0, spec_bytes = 0;
};

void plan_tables(const HostSystem& hs, int si, Plan* p) {
  for (int l = 0; l < hs.levels; ++l) {
    p->toff[si][l].clear();
    for (const auto& c : hs.lev[l]) {
      TableOffsets t{};
      t.S64 = p->dbl.size();
      p->dbl.insert(p->dbl.end(), c.S.begin(), c.S.end());
      t.S32 = p->flt.size();
      for (double x : c.S) p->flt.push_back((float)x);
      t.rzw64 = p->dbl.size();
      p->dbl.insert(p->dbl.end(), c.rz_w.begin(), c.rz_w.end());
      t.rzw32 = p->flt.size();
      for (double x : c.rz_w) p->flt.push_back((float)x);
      t.pzw64 = p->dbl.size();
      p->dbl.insert(p->dbl.end(), c.pz_w.begin(), c.pz_w.end());
      t.pzw32 = p->flt.size();
      for (double x : c.pz_w) p->flt.push_back((float)x);
      t.rzi = p->ints.size();
      p->ints.insert(p->ints.end(), c.rz_idx.begin(), c.rz_idx.end());
      t.pzi = p->ints.size();
      p->ints.insert(p->ints.end(), c.pz_idx.begin(), c.pz_idx.end());
      t.Linv = p->dbl.size();
      p->dbl.insert(p->dbl.end(), c.Linv.begin(), c.Linv.end());
      t.zb64 = p->dbl.size();
      p->dbl.insert(p->dbl.end(), c.zb.begin(), c.zb.end());
      t.zb32 = p->flt.size();
      for (double x : c.zb) p->flt.push_back((float)x);
      p->toff[si][l].push_back(t);
    }
  }
}

// vcycle_only: V-cycle scratch only.  caller_level0: the caller passes the
// level-0 v and b of every V-cycle, so level 0 reserves its residual buffer
// alone (v and b stay unbound).
void make_plan(const selm_mg_desc& d, const Sys& vel, const Sys* pres, int esize, Plan* p,
               bool vcycle_only = false, bool caller_level0 = false) {
  plan_tables(vel.host, 0, p);
  if (pres) plan_tables(pres->host, 1, p);
  p->dbl_off = p->lay.add(p->dbl.size() * sizeof(double) + 8);
  p->flt_off = p->lay.add(p->flt.size() * sizeof(float) + 8);
  p->int_off = p->lay.add(p->ints.size() * sizeof(int) + 8);
  const HostSystem* hs[2] = {&vel.host, pres ? &pres->host : nullptr};
  for (int si = 0; si < 2; ++si) {
    if (!hs[si]) continue;
    for (int l = 0; l < hs[si]->levels; ++l)
      for (int f = 0; f < 3; ++f) {
        if (caller_level0 && l == 0 && f < 2) continue;
        p->field_off[si][l][f] = p->lay.add((size_t)hs[si]->level_size(l) * esize);
      }
  }
  if (vcycle_only) {   // V-cycle scratch only: tables, level fields, counters, engine plan
    p->eng_off[0] = p->lay.add(kEngParamBytes);
    p->red_off = p->lay.add(16 * sizeof(double));
    p->cyc_off = p->lay.add(4 * sizeof(unsigned long long));
    return;
  }
  const size_t nv = (size_t)vel.host.level_size(0);
  p->u_off = p->lay.add(nv * 8);
  p->xi_off = p->lay.add(nv * 8);
  p->bvel_off = p->lay.add(nv * 8);
  p->wcomb_off = p->lay.add(nv * 8);
  if (pres) {
    const size_t np_ = (size_t)pres->host.level_size(0);
    p->phi_off = p->lay.add(3 * np_ * 8);
    p->prhs_off = p->lay.add(np_ * 8);
    // spectral inner solves of the projection (FP32 inner precision, uniform
    // channel with nx == ny a power of two <= 128)
    const HostComp& pc = pres->host.lev[0][0];
    const int n = pc.dims[0];
    if (esize == 4 && pres->host.ncomp == 1 && d.dim == 3 && pc.dims[1] == n && n >= 4 && n <= 128 &&
        (n & (n - 1)) == 0 && pc.dims[2] >= 2 && pc.kind[2] == kAxisCellNeu) {
      p->spec_bytes = (size_t)n * n * pc.dims[2] * 8;
      p->spec_off = p->lay.add(p->spec_bytes);
    }
  }
  p->eng_off[0] = p->lay.add(kEngParamBytes);
  if (pres) p->eng_off[1] = p->lay.add(kEngParamBytes);
  if (pres) {   // the chain's level fields and engine plan (it runs beside the solve)
    for (int l = 0; l < vel.host.levels; ++l)
      for (int f = 0; f < 3; ++f) p->field_off[2][l][f] = p->lay.add((size_t)vel.host.level_size(l) * esize);
    p->eng_off[2] = p->lay.add(kEngParamBytes);
  }
  p->red_off = p->lay.add(16 * sizeof(double));
  p->cyc_off = p->lay.add(4 * sizeof(unsigned long long));
  p->V_off = p->lay.add((size_t)d.max_particles * 3 * sizeof(double));
  p->Xs_off = p->lay.add((size_t)d.max_particles * 3 * sizeof(double));
  p->Fs_off = p->lay.add((size_t)d.max_particles * 3 * sizeof(double));
}

// Binds system s to the tables of system si and the level fields of slot fsi
// (fsi < 0: slot si).
void bind_system(Sys* s, int si, const Plan& p, char* ws, int fsi = -1) {
  const HostSystem& hs = s->host;
  s->levels = hs.levels;
  s->ncomp = hs.ncomp;
  double* dbl = (double*)(ws + p.dbl_off);
  float* flt = (float*)(ws + p.flt_off);
  int* ints = (int*)(ws + p.int_off);
  for (int l = 0; l < hs.levels; ++l) {
    LevelDev& L = s->lev[l];
    std::memset(&L, 0, sizeof L);
    L.level = l;
    L.ncomp = hs.ncomp;
    long long off = 0;
    for (int ci = 0; ci < hs.ncomp; ++ci) {
      const HostComp& hc = hs.lev[l][ci];
      const TableOffsets& t = p.toff[si][l][ci];
      CompDev& c = L.c[ci];
      c.nx = hc.dims[0];
      c.ny = hc.dims[1];
      c.nz = hc.dims[2];
      c.off = off;
      off += hc.size();
      c.comp_id = hc.comp_id;
      c.zkind = hc.kind[2];
      c.mx = hc.mods[0];
      c.my = hc.mods[1];
      c.mz = hc.mods[2];
      c.ncol = c.mx * c.my * c.mz;
      c.s = hs.scale;
      c.S64 = dbl + t.S64;
      c.S32 = flt + t.S32;
      c.rz_w64 = hc.rz_w.empty() ? nullptr : dbl + t.rzw64;
      c.rz_w32 = hc.rz_w.empty() ? nullptr : flt + t.rzw32;
      c.pz_w64 = hc.pz_w.empty() ? nullptr : dbl + t.pzw64;
      c.pz_w32 = hc.pz_w.empty() ? nullptr : flt + t.pzw32;
      c.rz_idx = hc.rz_idx.empty() ? nullptr : ints + t.rzi;
      c.pz_idx = hc.pz_idx.empty() ? nullptr : ints + t.pzi;
      c.Linv = hc.Linv.empty() ? nullptr : dbl + t.Linv;
      c.zb64 = dbl + t.zb64;
      c.zb32 = flt + t.zb32;
      for (int q = 0; q < 9; ++q) {
        c.w1[q] = hc.w1[q];
        c.w2[q] = hc.w2[q];
        c.w1f[q] = (float)hc.w1[q];
        c.w2f[q] = (float)hc.w2[q];
      }
    }
    L.size = off;
    L.flow = 0;
    if (l >= 1) {
      L.flow = 1;
      for (int ci = 0; ci < hs.ncomp; ++ci)
        if (!coop_flow_ok(hs.lev[l][ci])) L.flow = 0;
    }
    const int f = fsi < 0 ? si : fsi;
    s->v[l] = ws + p.field_off[f][l][0];
    s->b[l] = ws + p.field_off[f][l][1];
    s->t[l] = ws + p.field_off[f][l][2];
  }
}

#define CK(call)                                                        \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                            \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);      \
      return SELM_ECUDA;                                                \
    }                                                                   \
  } while (0)

inline cudaStream_t S(void* st) { return (cudaStream_t)st; }

Sys* sys_of(selm_mg* h, int system) {
  if (system == SELM_SYS_VELOCITY) return &h->vel;
  if (system == SELM_SYS_PRESSURE && h->has_pres) return &h->pres;
  return nullptr;
}

}  // namespace

namespace selm {

// ---- V-cycle (Algorithm 3) -------------------------------------------------
template <typename T>
selm_status vcycle_t(selm_mg* h, Sys& s, int l, T* v0, const T* b0, bool noise, const unsigned long long* cyc,
                     cudaStream_t st) {
  T* v = l == 0 ? v0 : (T*)s.v[l];
  const T* b = l == 0 ? b0 : (const T*)s.b[l];
  const LevelDev& L = s.lev[l];
  const bool last = l == s.levels - 1;
  const EnginePlanT<T>& eng = eng_of<T>(s);
  // A level above the engine with at most 2^20 sites per component: each half
  // of its V-cycle in one cooperative launch (one or a few site updates per
  // thread per pass).  Larger levels keep one GPU-wide launch per colour pass,
  // whose parallelism then beats the launch overhead.
  bool coop_size = true;
  for (int c = 0; c < L.ncomp; ++c)
    if ((long long)L.c[c].nx * L.c[c].ny * L.c[c].nz > (1ll << 20)) coop_size = false;
  if (l > 0 && !last && !L.rb && coop_size && s.use_engine && s.use_coop && eng.valid && l < eng.params.l0 &&
      s.coop_bar && level_coop_supported<T>(L)) {
    const LevelDev& Lc = s.lev[l + 1];
    CK(launch_level_coop<T>(L, Lc, 0, h->mu1, h->mu2, v, b, (T*)s.t[l], (T*)s.b[l + 1], (T*)s.v[l + 1], s.coop_bar,
                            s.coop_flow, noise, h->key, cyc, st));
    selm_status r = vcycle_t<T>(h, s, l + 1, v0, b0, noise, cyc, st);
    if (r != SELM_OK) return r;
    CK(launch_level_coop<T>(L, Lc, 1, h->mu1, h->mu2, v, b, (T*)s.t[l], (T*)s.b[l + 1], (T*)s.v[l + 1], s.coop_bar,
                            s.coop_flow, noise, h->key, cyc, st));
    return SELM_OK;
  }
  if (l > 0 && s.use_engine && eng.valid && l == eng.params.l0) {
    // levels l..L-1 in one cluster launch: reads s.b[l], writes s.v[l]
    CK(launch_coarse_engine<T>(eng, h->mu1, h->mu2, h->d.coarse_mode, noise, h->key, cyc, st));
    return SELM_OK;
  }
  if (last && h->d.coarse_mode == SELM_COARSE_CHOLESKY) {
    CK(launch_coarsest<T>(L, v, b, noise, h->key, cyc, st));
    return SELM_OK;
  }
  for (int q = 0; q < h->mu1; ++q) CK(launch_smooth<T>(L, v, b, q, noise, h->key, cyc, st));
  if (!last) {
    const LevelDev& Lc = s.lev[l + 1];
    CK(launch_residual<T>(L, v, b, (T*)s.t[l], st));
    CK(launch_restrict<T>(L, Lc, (const T*)s.t[l], (T*)s.b[l + 1], st));
    CK(cudaMemsetAsync(s.v[l + 1], 0, (size_t)Lc.size * sizeof(T), st));
    selm_status r = vcycle_t<T>(h, s, l + 1, v0, b0, noise, cyc, st);
    if (r != SELM_OK) return r;
    CK(launch_prolong<T>(L, Lc, v, (const T*)s.v[l + 1], st));
  }
  for (int q = 0; q < h->mu2; ++q) CK(launch_smooth<T>(L, v, b, h->mu1 + q, noise, h->key, cyc, st));
  return SELM_OK;
}

selm_status vcycle(selm_mg* h, Sys& s, void* v0, const void* b0, bool noise, const unsigned long long* cyc,
                   cudaStream_t st) {
  h->total_vcycles += 1;
  if (h->esize == 4) return vcycle_t<float>(h, s, 0, (float*)v0, (const float*)b0, noise, cyc, st);
  return vcycle_t<double>(h, s, 0, (double*)v0, (const double*)b0, noise, cyc, st);
}

selm_status outer_residual(selm_mg* h, Sys& s, const double* z, const double* b, void* r, double* norm2,
                           cudaStream_t st) {
  if (h->esize == 4)
    CK(launch_outer_residual<float>(s.lev[0], z, b, (float*)r, norm2, st));
  else
    CK(launch_outer_residual<double>(s.lev[0], z, b, (double*)r, norm2, st));
  return SELM_OK;
}

selm_status outer_update(selm_mg* h, Sys& s, double* z, const void* d, cudaStream_t st) {
  if (h->esize == 4)
    CK(launch_outer_update<float>(s.lev[0].size, z, (const float*)d, st));
  else
    CK(launch_outer_update<double>(s.lev[0].size, z, (const double*)d, st));
  return SELM_OK;
}

}  // namespace selm

namespace {

void drop_graphs(selm_mg* h) {
  for (auto& g : h->vg) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = selm_mg::VGraph{};
  }
}

// One V-cycle on the system's level-0 buffers (s.v[0] += ..., rhs s.b[0]) as
// a replay of a captured CUDA graph: the same launches with the same
// arguments, without their per-launch host and launch-gap cost.  A key runs
// directly once first (lazy one-time setup stays out of the capture); with
// profiling on, or when capture fails, the V-cycle runs directly.
selm_status vcycle_internal(selm_mg* h, Sys& s, bool noise, const unsigned long long* cyc, cudaStream_t st) {
  if (!h->graphs || !h->cap || prof::g_on) return vcycle(h, s, s.v[0], s.b[0], noise, cyc, st);
  selm_mg::VGraph* g = nullptr;
  for (auto& e : h->vg)
    if (e.sys == &s && e.noise == noise && e.cyc == cyc) g = &e;
  if (!g) {
    for (auto& e : h->vg)
      if (!e.sys) {
        g = &e;
        break;
      }
    if (!g) return vcycle(h, s, s.v[0], s.b[0], noise, cyc, st);
    g->sys = &s;
    g->noise = noise;
    g->cyc = cyc;
  }
  if (!g->exec && g->uses++ == 0) return vcycle(h, s, s.v[0], s.b[0], noise, cyc, st);
  if (!g->exec) {
    const long long l0 = prof::g_launches.load();
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->graphs = false;
      return vcycle(h, s, s.v[0], s.b[0], noise, cyc, st);
    }
    const selm_status r = vcycle(h, s, s.v[0], s.b[0], noise, cyc, h->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    h->total_vcycles -= 1;   // the capture recorded the V-cycle; nothing ran
    g->launches = prof::g_launches.load() - l0;
    prof::g_launches.fetch_sub(g->launches);
    if (r != SELM_OK || e != cudaSuccess || !graph || cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      g->exec = nullptr;
      h->graphs = false;   // direct launches from now on
      return vcycle(h, s, s.v[0], s.b[0], noise, cyc, st);
    }
    cudaGraphDestroy(graph);
  }
  CK(cudaGraphLaunch(g->exec, st));
  h->total_vcycles += 1;
  prof::g_launches.fetch_add(g->launches);
  return SELM_OK;
}

// One FAC iteration (Algorithm 1) with the internal level-0 buffers.
selm_status fac_cycle(selm_mg* h, Sys& s, double* z, const double* b, bool noise, const unsigned long long* cyc,
                      cudaStream_t st) {
  selm_status r = outer_residual(h, s, z, b, s.b[0], nullptr, st);
  if (r != SELM_OK) return r;
  CK(cudaMemsetAsync(s.v[0], 0, (size_t)s.lev[0].size * h->esize, st));
  r = vcycle_internal(h, s, noise, cyc, st);
  if (r != SELM_OK) return r;
  return outer_update(h, s, z, s.v[0], st);
}

// Reads the reduction slots copied by a norm read-back issued on the copy
// stream after h->ev_norm (the work stream may already run later launches):
// out_b / out_r receive slots 0 / 1 (null: not wanted).  The same copy brings
// back the grid-barrier words of the systems (red[8..13]: velocity, pressure,
// the chain's copy); a timed-out wait of a cooperative level launch is
// reported here and its words are cleared.
selm_status read_norms_after_event(selm_mg* h, double* out_b, double* out_r, cudaStream_t st) {
  CK(cudaStreamWaitEvent(h->xfer, h->ev_norm, 0));
  CK(cudaMemcpyAsync(h->host_red, h->red, 14 * sizeof(double), cudaMemcpyDeviceToHost, h->xfer));
  CK(cudaStreamSynchronize(h->xfer));
  if (out_b) *out_b = h->host_red[0];
  if (out_r) *out_r = h->host_red[1];
  const unsigned* words = (const unsigned*)(h->host_red + 8);
  if (words[2] != 0u || words[6] != 0u || words[10] != 0u) {
    CK(cudaStreamSynchronize(st));
    if (h->side) CK(cudaStreamSynchronize(h->side));
    CK(cudaMemsetAsync(h->red + 8, 0, 6 * sizeof(double), st));
    CK(cudaStreamSynchronize(st));
    h->err = "a grid barrier of a cooperative level launch timed out";
    return SELM_ECUDA;
  }
  return SELM_OK;
}

// Deterministic FAC iteration until ||b - Az|| <= tol ||b||.
selm_status fac_solve(selm_mg* h, Sys& s, double* z, const double* b, double tol, int max_cycles, int* cycles,
                      double* rel_out, cudaStream_t st) {
  // Each cycle's residual norm comes back through the copy stream.  When the
  // previous residual and the observed contraction predict that the cycle
  // will not meet the tolerance, its V-cycle is enqueued before the norm is
  // read, so the device does not idle during the read-back; the correction is
  // added to z only once the norm says so.  Iterates and cycle counts are
  // those of the plain loop: a wrong guess costs one discarded V-cycle.
  double* nb = h->red + 0;
  double* nr = h->red + 1;
  CK(cudaMemsetAsync(nb, 0, 2 * sizeof(double), st));
  CK(launch_norm2(s.lev[0].size, b, nb, st));
  *cycles = 0;
  double bn = 0.0, rel_prev = -1.0, rho = 0.5;
  for (int cyc = 0;; ++cyc) {
    if (cyc > 0) CK(cudaMemsetAsync(nr, 0, sizeof(double), st));
    selm_status r = outer_residual(h, s, z, b, s.b[0], nr, st);
    if (r != SELM_OK) return r;
    CK(cudaEventRecord(h->ev_norm, st));
    const bool spec = h->speculate && cyc < max_cycles && (rel_prev < 0.0 || rel_prev * rho > 5.0 * tol);
    if (spec) {
      CK(cudaMemsetAsync(s.v[0], 0, (size_t)s.lev[0].size * h->esize, st));
      r = vcycle_internal(h, s, false, h->cyc + 1, st);
      if (r != SELM_OK) return r;
    }
    double bn2 = 0.0, rn2 = 0.0;
    r = read_norms_after_event(h, cyc == 0 ? &bn2 : nullptr, &rn2, st);
    if (r != SELM_OK) return r;
    if (cyc == 0) {
      if (bn2 == 0.0) {
        CK(cudaMemsetAsync(z, 0, (size_t)s.lev[0].size * sizeof(double), st));
        if (rel_out) *rel_out = 0.0;
        return SELM_OK;
      }
      bn = std::sqrt(bn2);
    }
    const double rel = std::sqrt(rn2) / bn;
    if (rel_out) *rel_out = rel;
    if (rel <= tol) {
      *cycles = cyc;
      return SELM_OK;
    }
    if (cyc >= max_cycles) {
      *cycles = cyc;
      h->err = "FAC solve did not converge";
      return SELM_ENOCONV;
    }
    if (!spec) {
      CK(cudaMemsetAsync(s.v[0], 0, (size_t)s.lev[0].size * h->esize, st));
      r = vcycle_internal(h, s, false, h->cyc + 1, st);
      if (r != SELM_OK) return r;
    }
    r = outer_update(h, s, z, s.v[0], st);
    if (r != SELM_OK) return r;
    if (rel_prev > 0.0) rho = std::min(1.0, std::max(1e-3, rel / rel_prev));
    rel_prev = rel;
  }
}

// The projection's pressure problem by FP64 iterative refinement around the
// spectral inner solve (Algorithm 1's iteration with the exact FP32 solve of
// the uniform channel's Neumann operator in place of the V-cycle): residual
// r = b - A phi in FP64, delta = A^-1 r in FP32 (FFT along x, y; Thomas along
// z), phi += delta, until ||r|| <= tol ||b||.
selm_status spectral_fac_solve(selm_mg* h, double* phi, const double* b, double tol, int max_cycles, int* cycles,
                               double* rel_out, cudaStream_t st) {
  Sys& s = h->pres;
  double* nb = h->red + 0;
  double* nr = h->red + 1;
  CK(cudaMemsetAsync(nb, 0, 2 * sizeof(double), st));
  CK(launch_norm2(s.lev[0].size, b, nb, st));
  *cycles = 0;
  double bn = 0.0;
  for (int cyc = 0;; ++cyc) {
    if (cyc > 0) CK(cudaMemsetAsync(nr, 0, sizeof(double), st));
    selm_status r = outer_residual(h, s, phi, b, s.b[0], nr, st);
    if (r != SELM_OK) return r;
    CK(cudaEventRecord(h->ev_norm, st));
    double bn2 = 0.0, rn2 = 0.0;
    r = read_norms_after_event(h, cyc == 0 ? &bn2 : nullptr, &rn2, st);
    if (r != SELM_OK) return r;
    if (cyc == 0) {
      if (bn2 == 0.0) {
        CK(cudaMemsetAsync(phi, 0, (size_t)s.lev[0].size * sizeof(double), st));
        if (rel_out) *rel_out = 0.0;
        return SELM_OK;
      }
      bn = std::sqrt(bn2);
    }
    const double rel = std::sqrt(rn2) / bn;
    if (rel_out) *rel_out = rel;
    if (rel <= tol) {
      *cycles = cyc;
      return SELM_OK;
    }
    if (cyc >= max_cycles) {
      *cycles = cyc;
      h->err = "spectral pressure solve did not converge";
      return SELM_ENOCONV;
    }
    CK(spectral_pressure_solve(s.lev[0], (const float*)s.b[0], (float*)s.v[0], h->spec, st));
    r = outer_update(h, s, phi, s.v[0], st);
    if (r != SELM_OK) return r;
  }
}

// w <- P~ w.  The pressure Poisson problem (D^ D^T) phi = D^ w is solved by
// the FAC iteration from an initial value (Algorithm 1 takes one): slot < 0
// starts from zero; slots 0..2 start from that slot's previous pressure.  On
// the uniform channel the iteration's inner solve is spectral by default
// (SELM_OPT_PRESSURE_SPECTRAL), else the pressure system's V-cycle.
selm_status project(selm_mg* h, double* w, int* cycles, cudaStream_t st, int slot = -1) {
  *cycles = 0;
  if (!h->has_pres) return SELM_OK;
  const long long np_ = h->pres.lev[0].size;
  double* phi = h->phi + (size_t)(slot < 0 ? 0 : slot) * np_;
  CK(cudaMemsetAsync(h->red + 2, 0, sizeof(double), st));
  CK(launch_divergence(h->vel.lev[0], w, h->prhs, h->red + 2, st));
  CK(launch_sub_mean(np_, h->prhs, h->red + 2, st));
  if (slot < 0) CK(cudaMemsetAsync(phi, 0, (size_t)np_ * sizeof(double), st));
  double rel = 0.0;
  selm_status r = h->spectral && h->spec
                      ? spectral_fac_solve(h, phi, h->prhs, h->d.proj_tol, h->d.max_cycles, cycles, &rel, st)
                      : fac_solve(h, h->pres, phi, h->prhs, h->d.proj_tol, h->d.max_cycles, cycles, &rel, st);
  if (r != SELM_OK) return r;
  CK(launch_grad_sub(h->vel.lev[0], w, phi, st));
  return SELM_OK;
}

selm_status chain_cycles(selm_mg* h, int ncycles, cudaStream_t st) {
  Sys& s = h->has_chain ? h->chn : h->vel;
  for (int q = 0; q < ncycles; ++q) {
    selm_status r = fac_cycle(h, s, h->xi, nullptr, true, h->cyc + 0, st);
    if (r != SELM_OK) return r;
    CK(launch_inc_u64(h->cyc + 0, st));
    h->cycle += 1;
  }
  return SELM_OK;
}

bool check_particles(selm_mg* h, int np, const void* X) {
  if (np < 0 || (np > 0 && !X)) {
    h->err = "invalid particle arguments";
    return false;
  }
  return true;
}

}  // namespace

namespace {

// First level of a system's coarse engine.  An explicit option wins; else
// level 1 goes to cooperative launches when it is large (a pass of level 1
// then spreads over every SM instead of one cluster per component, which
// pays once a component holds 2^17 sites or more) and the engine starts at
// level 2; otherwise the engine takes every level from 1.
int engine_first_level(const selm_mg* h, const Sys& s) {
  if (s.engine_level > 0) return s.engine_level;
  if (!s.use_coop || s.levels < 4) return 1;
  long long big = 0;
  for (int c = 0; c < s.lev[1].ncomp; ++c) {
    const CompDev& d = s.lev[1].c[c];
    const long long n = (long long)d.nx * d.ny * d.nz;
    big = n > big ? n : big;
  }
  if (big < (1ll << 17)) return 1;
  const bool ok = h->esize == 4 ? level_coop_supported<float>(s.lev[1]) : level_coop_supported<double>(s.lev[1]);
  return ok ? 2 : 1;
}

}  // namespace

namespace selm {

selm_status chain_advance(selm_mg* h, int ncycles, cudaStream_t st) { return chain_cycles(h, ncycles, st); }

size_t footprint_with_host(const selm_mg_desc& d, const HostSystem& host, size_t extra_bytes) {
  Sys vel;
  vel.host = host;
  Plan p;
  make_plan(d, vel, nullptr, d.precision == SELM_FP64 ? 8 : 4, &p, true);
  p.lay.add(extra_bytes);
  return p.lay.total;
}

selm_status create_with_host(const selm_mg_desc& d, const HostSystem& host, int engine_level, bool use_coop,
                             int rb_level, size_t extra_bytes, cudaStream_t st, selm_mg** out, size_t* extra_off) {
  *out = nullptr;
  selm_mg* h = new (std::nothrow) selm_mg();
  if (!h) return SELM_ENOMEM;
  h->d = d;
  h->vel.host = host;
  h->has_pres = false;
  h->mu1 = d.nu_pre;
  h->mu2 = d.nu_post;
  h->esize = d.precision == SELM_FP64 ? 8 : 4;
  h->key.k0 = (uint32_t)(d.seed & 0xffffffffu) ^ (uint32_t)(d.instance >> 32);
  h->key.k1 = (uint32_t)(d.seed >> 32) ^ (uint32_t)(d.instance & 0xffffffffu);
  h->vel.engine_level = engine_level;
  h->vel.use_coop = use_coop;
  Plan p;
  make_plan(d, h->vel, nullptr, h->esize, &p, true);
  const size_t xoff = p.lay.add(extra_bytes);
  h->ws_bytes = p.lay.total;
  void* ws = nullptr;
  if (d.alloc) {
    ws = d.alloc(h->ws_bytes, d.alloc_ctx);
    if (!ws) {
      delete h;
      return SELM_ENOMEM;
    }
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) {   // vector accesses need the documented alignment
      if (d.free) d.free(ws, d.alloc_ctx);
      delete h;
      return SELM_EINVAL;
    }
  } else if (cudaMalloc(&ws, h->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return SELM_ENOMEM;
  }
  h->ws = (char*)ws;
  h->host_red = new (std::nothrow) double[16];
  if (!h->host_red || cudaStreamCreateWithFlags(&h->xfer, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_norm, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    selm_mg_destroy(h);
    return SELM_ENOMEM;
  }
  cudaError_t ce = cudaSuccess;
  if (!p.dbl.empty())
    ce = cudaMemcpyAsync(h->ws + p.dbl_off, p.dbl.data(), p.dbl.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && !p.flt.empty())
    ce = cudaMemcpyAsync(h->ws + p.flt_off, p.flt.data(), p.flt.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && !p.ints.empty())
    ce = cudaMemcpyAsync(h->ws + p.int_off, p.ints.data(), p.ints.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  bind_system(&h->vel, 0, p, h->ws);
  if (rb_level >= 0 && rb_level < h->vel.levels) h->vel.lev[rb_level].rb = 1;
  h->red = (double*)(h->ws + p.red_off);
  h->vel.coop_bar = (unsigned*)(h->red + 8);
  h->cyc = (unsigned long long*)(h->ws + p.cyc_off);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->red, 0, 16 * sizeof(double), st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->cyc, 0, 4 * sizeof(unsigned long long), st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);   // host tables must outlive the copies
  if (ce != cudaSuccess) {
    std::fprintf(stderr, "create_with_host: %s\n", cudaGetErrorString(ce));
    selm_mg_destroy(h);
    return SELM_ECUDA;
  }
  h->vel.eng_dev = h->ws + p.eng_off[0];
  const int first = engine_first_level(h, h->vel);
  if (h->esize == 4)
    plan_coarse_engine<float>(h->vel.lev, h->vel.levels, h->vel.b, h->vel.v, h->vel.t, h->vel.eng_dev, st,
                              &h->vel.engf, 0, first);
  else
    plan_coarse_engine<double>(h->vel.lev, h->vel.levels, h->vel.b, h->vel.v, h->vel.t, h->vel.eng_dev, st,
                               &h->vel.engd, 0, first);
  cudaGetLastError();   // without a plan the per-pass path runs
  *extra_off = xoff;
  *out = h;
  return SELM_OK;
}

selm_status vcycle_level(selm_mg* h, Sys& s, int level, bool noise, const unsigned long long* cyc, cudaStream_t st) {
  h->total_vcycles += 1;
  if (h->esize == 4) return vcycle_t<float>(h, s, level, nullptr, nullptr, noise, cyc, st);
  return vcycle_t<double>(h, s, level, nullptr, nullptr, noise, cyc, st);
}

selm_status replan_engine(selm_mg* h, int cluster, cudaStream_t st) {
  for (Sys* sy : {&h->vel, h->has_pres ? &h->pres : (Sys*)nullptr, h->has_chain ? &h->chn : (Sys*)nullptr}) {
    if (!sy || !sy->eng_dev) continue;
    CK(cudaStreamSynchronize(st));   // no launch may still read the old plan
    sy->engine_cluster = cluster;
    // without a plan (returns false) the per-pass path runs
    if (h->esize == 4)
      plan_coarse_engine<float>(sy->lev, sy->levels, sy->b, sy->v, sy->t, sy->eng_dev, st, &sy->engf, cluster,
                                engine_first_level(h, *sy));
    else
      plan_coarse_engine<double>(sy->lev, sy->levels, sy->b, sy->v, sy->t, sy->eng_dev, st, &sy->engd, cluster,
                                 engine_first_level(h, *sy));
    cudaGetLastError();
  }
  return SELM_OK;
}
}  // namespace selm

extern "C" {

size_t selm_mg_footprint(const selm_mg_desc* desc) {
  if (!desc) return 0;
  selm_mg_desc d = *desc;
  fill_desc_defaults(&d);
  if (!validate(d).empty()) return 0;
  Sys vel, pres;
  bool has_pres = false;
  if (!build_systems(d, &vel, &pres, &has_pres).empty()) return 0;
  Plan p;
  make_plan(d, vel, has_pres ? &pres : nullptr, d.precision == SELM_FP64 ? 8 : 4, &p);
  return p.lay.total;
}

selm_status selm_mg_create(const selm_mg_desc* desc, void* stream, selm_mg** out) {
  if (!desc || !out) return SELM_EINVAL;
  *out = nullptr;
  selm_mg* h = new (std::nothrow) selm_mg();
  if (!h) return SELM_ENOMEM;
  h->d = *desc;
  fill_desc_defaults(&h->d);
  std::string e = validate(h->d);
  if (e.empty()) e = build_systems(h->d, &h->vel, &h->pres, &h->has_pres);
  if (e.empty() && h->vel.host.level_size(0) >= (1ll << 31)) e = "grid too large (level field >= 2^31 elements)";
  if (!e.empty()) {
    std::fprintf(stderr, "selm_mg_create: %s\n", e.c_str());
    delete h;
    return SELM_EINVAL;
  }
  h->mu1 = h->d.nu_pre;
  h->mu2 = h->d.nu_post;
  h->esize = h->d.precision == SELM_FP64 ? 8 : 4;
  const uint64_t seed = h->d.seed, inst = h->d.instance;
  h->key.k0 = (uint32_t)(seed & 0xffffffffu) ^ (uint32_t)(inst >> 32);
  h->key.k1 = (uint32_t)(seed >> 32) ^ (uint32_t)(inst & 0xffffffffu);
  Plan p;
  make_plan(h->d, h->vel, h->has_pres ? &h->pres : nullptr, h->esize, &p);
  h->ws_bytes = p.lay.total;
  void* ws = nullptr;
  if (h->d.alloc) {
    ws = h->d.alloc(h->ws_bytes, h->d.alloc_ctx);
    if (!ws) {
      delete h;
      return SELM_ENOMEM;
    }
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) {   // vector accesses need the documented alignment
      if (h->d.free) h->d.free(ws, h->d.alloc_ctx);
      delete h;
      return SELM_EINVAL;
    }
  } else if (cudaMalloc(&ws, h->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return SELM_ENOMEM;
  }
  h->ws = (char*)ws;
  // Host word for norm read-backs: ordinary host memory (the read is
  // followed by a stream synchronisation anyway), so that creating and
  // destroying handles never synchronises the device.
  h->host_red = new (std::nothrow) double[16];
  if (!h->host_red || cudaStreamCreateWithFlags(&h->xfer, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_norm, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    selm_mg_destroy(h);
    return SELM_ENOMEM;
  }
  cudaStream_t st = S(stream);
  cudaError_t ce = cudaSuccess;
  if (!p.dbl.empty())
    ce = cudaMemcpyAsync(h->ws + p.dbl_off, p.dbl.data(), p.dbl.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && !p.flt.empty())
    ce = cudaMemcpyAsync(h->ws + p.flt_off, p.flt.data(), p.flt.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && !p.ints.empty())
    ce = cudaMemcpyAsync(h->ws + p.int_off, p.ints.data(), p.ints.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  bind_system(&h->vel, 0, p, h->ws);
  if (h->has_pres) bind_system(&h->pres, 1, p, h->ws);
  if (h->has_pres) {
    h->chn.host = h->vel.host;
    bind_system(&h->chn, 0, p, h->ws, 2);
    h->has_chain = true;
  }
  for (int si = 0; si < 3; ++si) {
    Sys* sy = si == 0 ? &h->vel : si == 1 ? (h->has_pres ? &h->pres : nullptr) : (h->has_chain ? &h->chn : nullptr);
    if (!sy) continue;
    void* dp = h->ws + p.eng_off[si];
    sy->eng_dev = dp;
    const int first = engine_first_level(h, *sy);
    if (h->esize == 4)
      plan_coarse_engine<float>(sy->lev, sy->levels, sy->b, sy->v, sy->t, dp, st, &sy->engf, 0, first);
    else
      plan_coarse_engine<double>(sy->lev, sy->levels, sy->b, sy->v, sy->t, dp, st, &sy->engd, 0, first);
    cudaGetLastError();
  }
  h->u = (double*)(h->ws + p.u_off);
  h->xi = (double*)(h->ws + p.xi_off);
  h->bvel = (double*)(h->ws + p.bvel_off);
  h->wcomb = (double*)(h->ws + p.wcomb_off);
  if (h->has_pres) {
    h->phi = (double*)(h->ws + p.phi_off);
    h->prhs = (double*)(h->ws + p.prhs_off);
    if (p.spec_bytes > 0 && spectral_pressure_supported(h->pres.lev[0])) {
      h->spec = h->ws + p.spec_off;
      h->spectral = true;
    }
  }
  h->red = (double*)(h->ws + p.red_off);
  h->vel.coop_bar = (unsigned*)(h->red + 8);
  if (h->has_pres) h->pres.coop_bar = (unsigned*)(h->red + 10);
  if (h->has_chain) h->chn.coop_bar = (unsigned*)(h->red + 12);
  h->cyc = (unsigned long long*)(h->ws + p.cyc_off);
  h->V = (double*)(h->ws + p.V_off);
  h->Xs = (double*)(h->ws + p.Xs_off);
  h->Fs = (double*)(h->ws + p.Fs_off);
  const size_t nv = (size_t)h->vel.lev[0].size * sizeof(double);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->xi, 0, nv, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->u, 0, nv, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->bvel, 0, nv, st);
  if (ce == cudaSuccess && h->has_pres)
    ce = cudaMemsetAsync(h->phi, 0, 3 * (size_t)h->pres.lev[0].size * sizeof(double), st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->cyc, 0, 4 * sizeof(unsigned long long), st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->red, 0, 16 * sizeof(double), st);
  if (ce == cudaSuccess && h->has_pres) {
    ce = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    int least = 0, greatest = 0;
    if (ce == cudaSuccess) ce = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (ce == cudaSuccess && greatest < least)
      ce = cudaStreamCreateWithPriority(&h->prio, cudaStreamNonBlocking, greatest);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);  // host tables must outlive the copies
  if (ce != cudaSuccess) {
    std::fprintf(stderr, "selm_mg_create: %s\n", cudaGetErrorString(ce));
    selm_mg_destroy(h);
    return SELM_ECUDA;
  }
  *out = h;
  return SELM_OK;
}

selm_status selm_mg_destroy(selm_mg* h) {
  if (!h) return SELM_EINVAL;
  if (h->side) {
    cudaStreamSynchronize(h->side);   // nothing of the handle's may still read the workspace
    cudaStreamDestroy(h->side);
  }
  if (h->prio) {
    cudaStreamSynchronize(h->prio);
    cudaStreamDestroy(h->prio);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->xfer) {
    cudaStreamSynchronize(h->xfer);
    cudaStreamDestroy(h->xfer);
  }
  if (h->ev_norm) cudaEventDestroy(h->ev_norm);
  drop_graphs(h);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->ws) {
    if (h->d.free)
      h->d.free(h->ws, h->d.alloc_ctx);
    else
      cudaFree(h->ws);
  }
  stokes_release(h);
  delete[] h->host_red;
  delete h;
  return SELM_OK;
}

const char* selm_mg_last_error(const selm_mg* h) { return h ? h->err.c_str() : "null handle"; }

int selm_mg_levels(const selm_mg* h, int system) {
  if (!h) return 0;
  if (system == SELM_SYS_VELOCITY) return h->vel.levels;
  if (system == SELM_SYS_PRESSURE && h->has_pres) return h->pres.levels;
  return 0;
}

int selm_mg_ncomp(const selm_mg* h, int system) {
  if (!h) return 0;
  if (system == SELM_SYS_VELOCITY) return h->vel.ncomp;
  if (system == SELM_SYS_PRESSURE && h->has_pres) return h->pres.ncomp;
  return 0;
}

selm_status selm_mg_layout(const selm_mg* h, int system, int level, int comp, int* dims3, long long* offset,
                           long long* level_size) {
  if (!h) return SELM_EINVAL;
  const Sys* s = system == SELM_SYS_VELOCITY ? &h->vel : (system == SELM_SYS_PRESSURE && h->has_pres ? &h->pres : nullptr);
  if (!s || level < 0 || level >= s->levels || comp < 0 || comp >= s->ncomp) return SELM_EINVAL;
  const CompDev& c = s->lev[level].c[comp];
  if (dims3) {
    dims3[0] = c.nx;
    dims3[1] = c.ny;
    dims3[2] = c.nz;
  }
  if (offset) *offset = c.off;
  if (level_size) *level_size = s->lev[level].size;
  return SELM_OK;
}

int selm_mg_inner_bytes(const selm_mg* h) { return h ? h->esize : 0; }

selm_status selm_mg_chain(selm_mg* h, double** xi, uint64_t* cycle) {
  if (!h) return SELM_EINVAL;
  if (xi) *xi = h->xi;
  if (cycle) *cycle = h->cycle;
  return SELM_OK;
}

selm_status selm_mg_velocity(selm_mg* h, double** u) {
  if (!h || !u) return SELM_EINVAL;
  *u = h->u;
  return SELM_OK;
}

selm_status selm_mg_fail_waits(selm_mg* h, int system, void* stream) {
  if (!h) return SELM_EINVAL;
  Sys* s = sys_of(h, system);
  if (!s || !s->coop_bar) return SELM_EINVAL;
  CK(cudaMemsetAsync(s->coop_bar + 2, 0x01, sizeof(unsigned), S(stream)));   // any non-zero word
  return SELM_OK;
}

selm_status selm_mg_set_cycle(selm_mg* h, uint64_t cycle) {
  if (!h) return SELM_EINVAL;
  CK(launch_set_u64(h->cyc + 0, cycle, nullptr));
  CK(cudaDeviceSynchronize());
  h->cycle = cycle;
  return SELM_OK;
}


selm_status selm_mg_set_option(selm_mg* h, int option, int value) {
  if (!h) return SELM_EINVAL;
  // every option changes the V-cycle's launches: drop the captured graphs
  // (after the device finished any launch of them)
  bool captured = false;
  for (const auto& g : h->vg) captured = captured || g.exec != nullptr;
  if (captured) {
    CK(cudaDeviceSynchronize());
    drop_graphs(h);
  }
  if (option == SELM_OPT_GRAPHS) {
    h->graphs = value != 0;
    return SELM_OK;
  }
  if (option == SELM_OPT_SPECULATE) {
    h->speculate = value != 0;
    return SELM_OK;
  }
  if (option == SELM_OPT_COARSE_ENGINE) {
    h->vel.use_engine = h->pres.use_engine = h->chn.use_engine = value != 0;
    return SELM_OK;
  }
  if (option == SELM_OPT_ENGINE_CLUSTER) {
    if (value < 0 || value > 16) return SELM_EINVAL;
    return replan_engine(h, value, nullptr);
  }
  if (option == SELM_OPT_LEVEL_COOP) {
    if (value < 0 || value > 2) return SELM_EINVAL;
    h->vel.use_coop = h->pres.use_coop = h->chn.use_coop = value != 0;
    h->vel.coop_flow = h->pres.coop_flow = h->chn.coop_flow = value == 1;
    return replan_engine(h, h->vel.engine_cluster, nullptr);   // the automatic first level depends on it
  }
  if (option == SELM_OPT_PRESSURE_SPECTRAL) {
    if (value != 0 && !h->spec) return SELM_EINVAL;
    h->spectral = value != 0;
    return SELM_OK;
  }
  if (option == SELM_OPT_ENGINE_LEVEL) {
    if (value < 0 || value > kMaxLevels) return SELM_EINVAL;
    h->vel.engine_level = h->pres.engine_level = h->chn.engine_level = value;
    return replan_engine(h, h->vel.engine_cluster, nullptr);
  }
  return SELM_EINVAL;
}

selm_status selm_mg_engine_info(const selm_mg* h, int system, int* first_level, int* cluster_size,
                                size_t* smem_bytes) {
  if (!h) return SELM_EINVAL;
  const Sys* s = system == SELM_SYS_VELOCITY ? &h->vel : (system == SELM_SYS_PRESSURE && h->has_pres ? &h->pres : nullptr);
  if (!s) return SELM_EINVAL;
  const bool v = h->esize == 4 ? s->engf.valid : s->engd.valid;
  if (first_level) *first_level = v ? (h->esize == 4 ? s->engf.params.l0 : s->engd.params.l0) : -1;
  if (cluster_size) *cluster_size = v ? (h->esize == 4 ? s->engf.cluster : s->engd.cluster) : 0;
  if (smem_bytes) *smem_bytes = v ? (h->esize == 4 ? s->engf.smem_bytes : s->engd.smem_bytes) : 0;
  return SELM_OK;
}

int selm_mg_pressure_spectral(const selm_mg* h) { return h && h->spectral && h->spec ? 1 : 0; }

selm_status selm_mg_stats(const selm_mg* h, int* last_solve_cycles, int* last_proj_cycles, long long* total) {
  if (!h) return SELM_EINVAL;
  if (last_solve_cycles) *last_solve_cycles = h->last_solve_cycles;
  if (last_proj_cycles) *last_proj_cycles = h->last_proj_cycles;
  if (total) *total = h->total_vcycles;
  return SELM_OK;
}

// ---- stage entry points ------------------------------------------------------

selm_status selm_mg_smooth(selm_mg* h, int system, int level, void* v, const void* b, int sweep, uint64_t cycle,
                           int noise, void* stream) {
  if (!h) return SELM_EINVAL;
  Sys* s = sys_of(h, system);
  if (!s || level < 0 || level >= s->levels || !v || !b || sweep < 0 || sweep > 255) return SELM_EINVAL;
  cudaStream_t st = S(stream);
  CK(launch_set_u64(h->cyc + 1, cycle, st));
  if (h->esize == 4)
    CK(launch_smooth<float>(s->lev[level], (float*)v, (const float*)b, sweep, noise != 0, h->key, h->cyc + 1, st));
  else
    CK(launch_smooth<double>(s->lev[level], (double*)v, (const double*)b, sweep, noise != 0, h->key, h->cyc + 1, st));
  return SELM_OK;
}

selm_status selm_mg_residual_restrict(selm_mg* h, int system, int level, const void* v, const void* b,
                                      void* b_coarse, void* stream) {
  if (!h) return SELM_EINVAL;
  Sys* s = sys_of(h, system);
  if (!s || level < 0 || level + 1 >= s->levels || !v || !b || !b_coarse) return SELM_EINVAL;
  cudaStream_t st = S(stream);
  if (h->esize == 4) {
    CK(launch_residual<float>(s->lev[level], (const float*)v, (const float*)b, (float*)s->t[level], st));
    CK(launch_restrict<float>(s->lev[level], s->lev[level + 1], (const float*)s->t[level], (float*)b_coarse, st));
  } else {
    CK(launch_residual<double>(s->lev[level], (const double*)v, (const double*)b, (double*)s->t[level], st));
    CK(launch_restrict<double>(s->lev[level], s->lev[level + 1], (const double*)s->t[level], (double*)b_coarse, st));
  }
  return SELM_OK;
}

selm_status selm_mg_prolong_correct(selm_mg* h, int system, int level, void* v, const void* v_coarse, void* stream) {
  if (!h) return SELM_EINVAL;
  Sys* s = sys_of(h, system);
  if (!s || level < 0 || level + 1 >= s->levels || !v || !v_coarse) return SELM_EINVAL;
  cudaStream_t st = S(stream);
  if (h->esize == 4)
    CK(launch_prolong<float>(s->lev[level], s->lev[level + 1], (float*)v, (const float*)v_coarse, st));
  else
    CK(launch_prolong<double>(s->lev[level], s->lev[level + 1], (double*)v, (const double*)v_coarse, st));
  return SELM_OK;
}

selm_status selm_mg_coarsest(selm_mg* h, int system, void* v, const void* b, uint64_t cycle, int noise, void* stream) {
  if (!h) return SELM_EINVAL;
  Sys* s = sys_of(h, system);
  if (!s || !v || !b || h->d.coarse_mode != SELM_COARSE_CHOLESKY) return SELM_EINVAL;
  cudaStream_t st = S(stream);
  CK(launch_set_u64(h->cyc + 1, cycle, st));
  const LevelDev& L = s->lev[s->levels - 1];
  if (h->esize == 4)
    CK(launch_coarsest<float>(L, (float*)v, (const float*)b, noise != 0, h->key, h->cyc + 1, st));
  else
    CK(launch_coarsest<double>(L, (double*)v, (const double*)b, noise != 0, h->key, h->cyc + 1, st));
  return SELM_OK;
}

selm_status selm_mg_vcycle(selm_mg* h, int system, void* v, const void* b, uint64_t cycle, int noise, void* stream) {
  if (!h) return SELM_EINVAL;
  Sys* s = sys_of(h, system);
  if (!s || !v || !b) return SELM_EINVAL;
  cudaStream_t st = S(stream);
  CK(launch_set_u64(h->cyc + 1, cycle, st));
  return vcycle(h, *s, v, b, noise != 0, h->cyc + 1, st);
}

selm_status selm_mg_outer_residual(selm_mg* h, int system, const double* z, const double* b64, void* r,
                                   double* norm2, void* stream) {
  if (!h) return SELM_EINVAL;
  Sys* s = sys_of(h, system);
  if (!s || !z || !r) return SELM_EINVAL;
  return outer_residual(h, *s, z, b64, r, norm2, S(stream));
}

selm_status selm_mg_outer_update(selm_mg* h, int system, double* z, const void* d, void* stream) {
  if (!h) return SELM_EINVAL;
  Sys* s = sys_of(h, system);
  if (!s || !z || !d) return SELM_EINVAL;
  return outer_update(h, *s, z, d, S(stream));
}

selm_status selm_mg_fac_cycle(selm_mg* h, int system, double* z, const double* b64, uint64_t cycle, int noise,
                              void* stream) {
  if (!h) return SELM_EINVAL;
  Sys* s = sys_of(h, system);
  if (!s || !z) return SELM_EINVAL;
  cudaStream_t st = S(stream);
  CK(launch_set_u64(h->cyc + 1, cycle, st));
  return fac_cycle(h, *s, z, b64, noise != 0, h->cyc + 1, st);
}

selm_status selm_mg_fac_solve(selm_mg* h, int system, double* z, const double* b64, double tol, int max_cycles,
                              int* cycles_out, double* resid_out, void* stream) {
  if (!h) return SELM_EINVAL;
  Sys* s = sys_of(h, system);
  if (!s || !z || !b64 || !(tol > 0.0) || max_cycles < 0) return SELM_EINVAL;
  int cycles = 0;
  double rel = 0.0;
  selm_status r = fac_solve(h, *s, z, b64, tol, max_cycles, &cycles, &rel, S(stream));
  if (cycles_out) *cycles_out = cycles;
  if (resid_out) *resid_out = rel;
  return r;
}

selm_status selm_mg_spread(selm_mg* h, int np, const double* X, const double* F, double* b, void* stream) {
  if (!h || !b || !check_particles(h, np, X) || (np > 0 && !F)) return SELM_EINVAL;
  cudaStream_t st = S(stream);
  CK(cudaMemsetAsync(b, 0, (size_t)h->vel.lev[0].size * sizeof(double), st));
  CK(launch_spread(h->vel.lev[0], h->d.n, h->d.dim, np, X, F, b, st));
  return SELM_OK;
}

selm_status selm_mg_interp(selm_mg* h, int np, const double* X, const double* u, double* U, void* stream) {
  if (!h || !u || !check_particles(h, np, X) || (np > 0 && !U)) return SELM_EINVAL;
  CK(launch_interp(h->vel.lev[0], h->d.n, h->d.dim, np, X, u, U, S(stream)));
  return SELM_OK;
}

selm_status selm_mg_project(selm_mg* h, double* w, int* cycles_out, void* stream) {
  if (!h || !w) return SELM_EINVAL;
  int cycles = 0;
  selm_status r = project(h, w, &cycles, S(stream));
  if (cycles_out) *cycles_out = cycles;
  return r;
}

selm_status selm_mg_em_update(selm_mg* h, int np, double* X, const double* V, void* stream) {
  if (!h || !check_particles(h, np, X) || (np > 0 && !V)) return SELM_EINVAL;
  CK(launch_em(np, h->d.dim, X, V, S(stream)));
  return SELM_OK;
}

// ---- SELM operations (Algorithm 4) ----------------------------------------------

selm_status selm_mg_solve(selm_mg* h, int np, const double* X, const double* F, double* U, int* cycles_out,
                          double* resid_out, void* stream) {
  if (!h || !check_particles(h, np, X) || (np > 0 && (!F || !U))) return SELM_EINVAL;
  cudaStream_t st = S(stream);
  const long long nv = h->vel.lev[0].size;
  CK(cudaMemsetAsync(h->bvel, 0, (size_t)nv * sizeof(double), st));
  CK(launch_spread(h->vel.lev[0], h->d.n, h->d.dim, np, X, F, h->bvel, st));
  int pc = 0, pc2 = 0;
  selm_status r = project(h, h->bvel, &pc, st, 0);
  if (r != SELM_OK) return r;
  CK(cudaMemsetAsync(h->u, 0, (size_t)nv * sizeof(double), st));
  int cycles = 0;
  double rel = 0.0;
  r = fac_solve(h, h->vel, h->u, h->bvel, h->d.tol, h->d.max_cycles, &cycles, &rel, st);
  h->last_solve_cycles = cycles;
  if (cycles_out) *cycles_out = cycles;
  if (resid_out) *resid_out = rel;
  if (r != SELM_OK) return r;
  const double* field = h->u;
  if (h->has_pres) {
    CK(cudaMemcpyAsync(h->wcomb, h->u, (size_t)nv * sizeof(double), cudaMemcpyDeviceToDevice, st));
    r = project(h, h->wcomb, &pc2, st, 1);
    if (r != SELM_OK) return r;
    field = h->wcomb;
  }
  h->last_proj_cycles = pc + pc2;
  CK(launch_interp(h->vel.lev[0], h->d.n, h->d.dim, np, X, field, U, st));
  return SELM_OK;
}

selm_status selm_mg_sample(selm_mg* h, int np, const double* X, int ncycles, double* g, double* xi_out,
                           void* stream) {
  if (!h || ncycles < 0 || !check_particles(h, np, X) || (np > 0 && !g)) return SELM_EINVAL;
  cudaStream_t st = S(stream);
  selm_status r = chain_cycles(h, ncycles, st);
  if (r != SELM_OK) return r;
  const long long nv = h->vel.lev[0].size;
  if (xi_out) CK(cudaMemcpyAsync(xi_out, h->xi, (size_t)nv * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(launch_axpby(nv, std::sqrt(2.0 * h->d.kT), h->xi, 0.0, h->xi, h->wcomb, st));
  int pc = 0;
  r = project(h, h->wcomb, &pc, st, 2);
  if (r != SELM_OK) return r;
  CK(launch_interp(h->vel.lev[0], h->d.n, h->d.dim, np, X, h->wcomb, g, st));
  return SELM_OK;
}

}  // extern "C"

namespace {

selm_status step_on(selm_mg* h, int np, double* X, const double* F, double dt, int nsteps, int ncycles_per_step,
                    cudaStream_t st) {
  const long long nv = h->vel.lev[0].size;
  // With the projection, the chain cycles run on the side stream (on the
  // chain's own level fields) beside the spread, the first projection and the
  // velocity solve; the combination of u and the chain state waits for them.
  const bool overlap = h->side != nullptr && h->has_chain && ncycles_per_step > 0;
  for (int step = 0; step < nsteps; ++step) {
    bool joined = true;
    auto join = [&]() -> selm_status {
      if (!joined) {
        joined = true;
        CK(cudaStreamWaitEvent(st, h->ev_join, 0));
      }
      return SELM_OK;
    };
    auto fail = [&](selm_status r) {
      join();
      return r;
    };
    selm_status r = SELM_OK;
    if (overlap) {
      CK(cudaEventRecord(h->ev_fork, st));
      CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
      joined = false;
      r = chain_cycles(h, ncycles_per_step, h->side);
      if (cudaEventRecord(h->ev_join, h->side) != cudaSuccess) {
        h->err = "event record on the side stream failed";
        cudaStreamSynchronize(h->side);
        return SELM_ECUDA;
      }
      if (r != SELM_OK) return fail(r);
    }
    if (cudaMemsetAsync(h->bvel, 0, (size_t)nv * sizeof(double), st) != cudaSuccess ||
        launch_spread(h->vel.lev[0], h->d.n, h->d.dim, np, X, F, h->bvel, st) != cudaSuccess) {
      h->err = cudaGetErrorString(cudaGetLastError());
      return fail(SELM_ECUDA);
    }
    int pc = 0, pc2 = 0, cycles = 0;
    double rel = 0.0;
    r = project(h, h->bvel, &pc, st, 0);
    if (r != SELM_OK) return fail(r);
    if (cudaMemsetAsync(h->u, 0, (size_t)nv * sizeof(double), st) != cudaSuccess) {
      h->err = cudaGetErrorString(cudaGetLastError());
      return fail(SELM_ECUDA);
    }
    r = fac_solve(h, h->vel, h->u, h->bvel, h->d.tol, h->d.max_cycles, &cycles, &rel, st);
    h->last_solve_cycles = cycles;
    if (r != SELM_OK) return fail(r);
    r = join();
    if (r != SELM_OK) return r;
    if (!overlap) {
      r = chain_cycles(h, ncycles_per_step, st);
      if (r != SELM_OK) return r;
    }
    CK(launch_axpby(nv, dt, h->u, std::sqrt(2.0 * h->d.kT * dt), h->xi, h->wcomb, st));
    r = project(h, h->wcomb, &pc2, st, 1);
    if (r != SELM_OK) return r;
    h->last_proj_cycles = pc + pc2;
    CK(launch_interp(h->vel.lev[0], h->d.n, h->d.dim, np, X, h->wcomb, h->V, st));
    CK(launch_em(np, h->d.dim, X, h->V, st));
  }
  return SELM_OK;
}

}  // namespace

extern "C" {

selm_status selm_mg_step(selm_mg* h, int np, double* X, const double* F, double dt, int nsteps, int ncycles_per_step,
                         void* stream) {
  if (!h || nsteps < 0 || ncycles_per_step < 0 || !(dt >= 0.0) || !check_particles(h, np, X) || (np > 0 && !F))
    return SELM_EINVAL;
  if (np > h->d.max_particles) {
    h->err = "np exceeds max_particles";
    return SELM_EINVAL;
  }
  cudaStream_t user = S(stream);
  // When the chain runs beside the step's main path, the main path (the
  // critical one) runs on the handle's high-priority stream, so that the
  // block scheduler gives it the SMs first and the chain fills what it
  // leaves idle; the caller's stream waits for the step at the end.
  if (!h->prio || !h->has_chain || ncycles_per_step <= 0 || nsteps <= 0)
    return step_on(h, np, X, F, dt, nsteps, ncycles_per_step, user);
  CK(cudaEventRecord(h->ev_in, user));
  CK(cudaStreamWaitEvent(h->prio, h->ev_in, 0));
  const selm_status r = step_on(h, np, X, F, dt, nsteps, ncycles_per_step, h->prio);
  if (cudaEventRecord(h->ev_out, h->prio) != cudaSuccess || cudaStreamWaitEvent(user, h->ev_out, 0) != cudaSuccess) {
    cudaStreamSynchronize(h->prio);
    h->err = "joining the step's stream failed";
    return SELM_ECUDA;
  }
  return r;
}

selm_status selm_mg_step_host(selm_mg* h, int np, double* X_host, const double* F_host, double dt, int nsteps,
                              int ncycles_per_step, void* stream) {
  if (!h || !check_particles(h, np, X_host) || (np > 0 && !F_host)) return SELM_EINVAL;
  if (np > h->d.max_particles) {
    h->err = "np exceeds max_particles";
    return SELM_EINVAL;
  }
  cudaStream_t st = S(stream);
  const size_t bytes = (size_t)np * h->d.dim * sizeof(double);
  if (np > 0) {
    CK(cudaMemcpyAsync(h->Xs, X_host, bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->Fs, F_host, bytes, cudaMemcpyHostToDevice, st));
  }
  selm_status r = selm_mg_step(h, np, h->Xs, h->Fs, dt, nsteps, ncycles_per_step, stream);
  if (r != SELM_OK) return r;
  if (np > 0) CK(cudaMemcpyAsync(X_host, h->Xs, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SELM_OK;
}

selm_status selm_philox4x32_10(const uint32_t* ctr, uint32_t key0, uint32_t key1, uint32_t* out, int n,
                               void* stream) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return SELM_EINVAL;
  Key k{key0, key1};
  if (launch_philox(ctr, k, out, n, S(stream)) != cudaSuccess) return SELM_ECUDA;
  return SELM_OK;
}

}  // extern "C"


// ---------------------------------------------------------------------------
// V-cycle without device allocation.
//
// For callers that cannot allocate device memory themselves or through us at
// run time -- for example a service that fixes its device memory budget up
// front and forbids allocation while it runs, or a thread that cannot reach
// the allocator of the framework owning the device -- this entry point runs
// one V-cycle with all of its scratch (Galerkin tables, coarse-level fields,
// the level-0 residual buffer, counters, the coarse-engine plan) in the fixed
// device array below.  Every device that loads this library holds the array
// until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;   // 16 MiB per device
constexpr int kStaticMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticSlot {
  bool ready = false;
  selm_mg_desc key{};
  selm_mg* h = nullptr;   // host-side bookkeeping; its workspace is g_static_scratch
};
StaticSlot g_static_slots[kStaticMaxDevices];
// Host bookkeeping of a slot (its tables, plans and key) is rebuilt in place;
// one lock per device serialises the host side of concurrent calls.
std::mutex g_static_locks[kStaticMaxDevices];

bool same_vcycle_desc(const selm_mg_desc& a, const selm_mg_desc& b) {
  return a.dim == b.dim && a.n == b.n && a.mu == b.mu && a.levels == b.levels && a.nu_pre == b.nu_pre &&
         a.nu_post == b.nu_post && a.precision == b.precision && a.coarse_mode == b.coarse_mode &&
         a.seed == b.seed && a.instance == b.instance;
}

// Builds the hierarchy of descriptor d inside the static array (the set-up of
// create_with_host, without an allocation).  Synchronises st.
selm_status static_setup(StaticSlot& slot, const selm_mg_desc& d, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    std::fprintf(stderr,
                 "selm_mg_vcycle_static: set-up for a new descriptor copies tables and synchronises the stream; "
                 "make the first call with this descriptor outside stream capture\n");
    return SELM_EINVAL;
  }
  selm_mg* h = slot.h ? slot.h : new (std::nothrow) selm_mg();
  if (!h) return SELM_ENOMEM;
  slot.h = h;
  slot.ready = false;
  h->d = d;
  h->vel = Sys();
  h->pres = Sys();
  h->has_pres = false;
  std::string e = build_systems(d, &h->vel, &h->pres, &h->has_pres);
  if (!e.empty()) {
    std::fprintf(stderr, "selm_mg_vcycle_static: %s\n", e.c_str());
    return SELM_EINVAL;
  }
  h->mu1 = d.nu_pre;
  h->mu2 = d.nu_post;
  h->esize = d.precision == SELM_FP64 ? 8 : 4;
  h->key.k0 = (uint32_t)(d.seed & 0xffffffffu) ^ (uint32_t)(d.instance >> 32);
  h->key.k1 = (uint32_t)(d.seed >> 32) ^ (uint32_t)(d.instance & 0xffffffffu);
  Plan p;
  make_plan(d, h->vel, nullptr, h->esize, &p, true, true);
  if (p.lay.total > kStaticScratchBytes) {
    std::fprintf(stderr,
                 "selm_mg_vcycle_static: this grid needs %zu bytes of scratch, above the static limit of %zu bytes\n",
                 p.lay.total, kStaticScratchBytes);
    return SELM_EINVAL;
  }
  // In host code g_static_scratch names a host-side stand-in; the device
  // address must come from the runtime, with this device current.
  void* base = nullptr;
  cudaError_t ce = cudaGetSymbolAddress(&base, g_static_scratch);
  if (ce != cudaSuccess || !base) {
    std::fprintf(stderr, "selm_mg_vcycle_static: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(ce));
    cudaGetLastError();
    return SELM_ECUDA;
  }
  h->ws = (char*)base;
  h->ws_bytes = kStaticScratchBytes;
  if (!p.dbl.empty())
    ce = cudaMemcpyAsync(h->ws + p.dbl_off, p.dbl.data(), p.dbl.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && !p.flt.empty())
    ce = cudaMemcpyAsync(h->ws + p.flt_off, p.flt.data(), p.flt.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && !p.ints.empty())
    ce = cudaMemcpyAsync(h->ws + p.int_off, p.ints.data(), p.ints.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  bind_system(&h->vel, 0, p, h->ws);
  h->vel.v[0] = nullptr;   // level 0 works on the caller's v and b
  h->vel.b[0] = nullptr;
  h->red = (double*)(h->ws + p.red_off);
  h->vel.coop_bar = (unsigned*)(h->red + 8);
  h->cyc = (unsigned long long*)(h->ws + p.cyc_off);
  // a previous descriptor's bytes may sit at these offsets
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->red, 0, 16 * sizeof(double), st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->cyc, 0, 4 * sizeof(unsigned long long), st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);   // the host tables are temporaries
  if (ce != cudaSuccess) {
    std::fprintf(stderr, "selm_mg_vcycle_static: %s\n", cudaGetErrorString(ce));
    return SELM_ECUDA;
  }
  h->vel.eng_dev = h->ws + p.eng_off[0];
  const int first = engine_first_level(h, h->vel);
  // Without an engine plan (no cluster shape fits) the per-pass path runs; a
  // CUDA error while planning is an error.
  if (h->esize == 4)
    plan_coarse_engine<float>(h->vel.lev, h->vel.levels, h->vel.b, h->vel.v, h->vel.t, h->vel.eng_dev, st,
                              &h->vel.engf, 0, first);
  else
    plan_coarse_engine<double>(h->vel.lev, h->vel.levels, h->vel.b, h->vel.v, h->vel.t, h->vel.eng_dev, st,
                               &h->vel.engd, 0, first);
  ce = cudaStreamSynchronize(st);
  if (ce == cudaSuccess) ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    std::fprintf(stderr, "selm_mg_vcycle_static: planning the coarse levels failed: %s\n", cudaGetErrorString(ce));
    return SELM_ECUDA;
  }
  slot.key = d;
  slot.ready = true;
  return SELM_OK;
}

}  // namespace

extern "C" selm_status selm_mg_vcycle_static(const selm_mg_desc* desc, void* v, const void* b, uint64_t cycle,
                                             int noise, void* stream) {
  if (!desc || !v || !b) return SELM_EINVAL;
  selm_mg_desc d = *desc;
  d.projection = SELM_PROJ_NONE;
  d.alloc = nullptr;
  d.free = nullptr;
  fill_desc_defaults(&d);
  std::string e = validate(d);
  int dev = 0;
  if (e.empty() && cudaGetDevice(&dev) != cudaSuccess) e = "no current CUDA device";
  if (e.empty() && (dev < 0 || dev >= kStaticMaxDevices)) e = "device index out of range";
  if (!e.empty()) {
    std::fprintf(stderr, "selm_mg_vcycle_static: %s\n", e.c_str());
    return SELM_EINVAL;
  }
  cudaStream_t st = S(stream);
  std::lock_guard<std::mutex> lock(g_static_locks[dev]);
  StaticSlot& slot = g_static_slots[dev];
  if (!slot.ready || !same_vcycle_desc(slot.key, d)) {
    const selm_status r = static_setup(slot, d, st);
    if (r != SELM_OK) return r;
  }
  selm_mg* h = slot.h;
  // The counter slot keeps the previous call's value: set it for this call.
  if (launch_set_u64(h->cyc + 1, cycle, st) != cudaSuccess) return SELM_ECUDA;
  return vcycle(h, h->vel, v, b, noise != 0, h->cyc + 1, st);
}
