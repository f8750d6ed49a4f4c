// C ABI of the HOT library (include/hot_mpm.h) and the host side of Alg. 3.
//
// The host issues kernels and takes the solver's scalar decisions (loop
// termination, line-search acceptance, L-BFGS pair acceptance); every vector
// and particle operation runs on the device.
#include <chrono>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <thread>

#include "internal.h"

namespace hot {

static thread_local std::string g_last_error;
static mpm_alloc_fn g_alloc = nullptr;
static mpm_free_fn g_free = nullptr;
static void *g_ctx = nullptr;

static std::atomic<long long> g_launches{0};

void fail(mpm_status code, const std::string &msg) { throw Error{code, msg}; }

void set_thread_error(const std::string &msg) { g_last_error = msg; }

void note_launch(const char *what) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  check_cuda(cudaGetLastError(), what);
}

// kernels run by a graph launch (counted once per executed kernel node)
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// `only`: empty (every name) or a comma-separated list of names
bool prof_selected(const std::string &only, const char *name) {
  if (only.empty()) return true;
  const std::string n(name);
  size_t a = 0;
  while (a <= only.size()) {
    size_t b = only.find(',', a);
    if (b == std::string::npos) b = only.size();
    if (only.compare(a, b - a, n) == 0 && b - a == n.size()) return true;
    a = b + 1;
  }
  return false;
}

static cudaEvent_t take_event(Scene &s) {
  if (!s.ev_pool.empty()) {
    cudaEvent_t e = s.ev_pool.back();
    s.ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  HOT_CUDA(cudaEventCreate(&e));
  return e;
}

ProfScope::ProfScope(Scene &sc, const char *name) : s(&sc), id(-1) {
  if (!sc.prof) return;
  // no events inside a stream capture (conditional graph bodies refuse them)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(sc.st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  if (!prof_selected(sc.prof_only, name)) return;
  for (size_t k = 0; k < sc.prof_names.size(); ++k)
    if (sc.prof_names[k] == name) id = (int)k;
  if (id < 0) {
    id = (int)sc.prof_names.size();
    sc.prof_names.push_back(name);
  }
  a = take_event(sc);
  b = take_event(sc);
  HOT_CUDA(cudaEventRecord(a, sc.st));
}

ProfScope::~ProfScope() {
  if (id < 0) return;
  cudaEventRecord(b, s->st);
  s->prof_ids.push_back(id);
  s->prof_ev.push_back(a);
  s->prof_ev.push_back(b);
}

void check_cuda(cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    fail(MPM_ERR_CUDA, m);
  }
}

void *dev_alloc(size_t bytes, cudaStream_t st) {
  void *p = nullptr;
  if (g_alloc) {
    p = g_alloc(bytes, (void *)st, g_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) fail(MPM_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  return p;
}

void dev_free(void *p, cudaStream_t st) {
  if (!p) return;
  if (g_free) g_free(p, (void *)st, g_ctx);
  else cudaFree(p);
}

int read_errflag(Scene &s) {
  int e = 0;
  HOT_CUDA(cudaMemcpyAsync(&e, s.errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  return e;
}

size_t Scene::bytes() const {
  size_t b = pd.bytes() + pd_alt.bytes() + pmat.bytes() + pmat_alt.bytes() + pid.bytes() + pid_alt.bytes() +
             mat_table.bytes() + bc_dev.bytes() + key.bytes() + slot.bytes() + perm.bytes() + tmp.bytes() +
             cell_count.bytes() + cell_start.bytes() + cell_first.bytes() + cell_n.bytes() + cell_key.bytes() +
             blk_first.bytes() + blk_end.bytes() + blk_key.bytes() + flags.bytes() + flag_scan.bytes() + m.bytes() +
             v.bytes() + xi.bytes() + fixed.bytes() + mv.bytes() + mxi.bytes() + dv.bytes() + g.bytes() +
             pdir.bytes() + q.bytes() + g_new.bytes() + dv_new.bytes() + vtmp.bytes() + hist_s.bytes() +
             hist_y.bytes() + Lv.bytes() + Lp.bytes() + Le.bytes() + dv_e.bytes() + g_e.bytes() + gscr.bytes() +
             part.bytes() + tr_alpha.bytes() + tr_int.bytes() + lstate.bytes() + cg_r.bytes() + cg_z.bytes() +
             cg_p.bytes() + cg_Ap.bytes() + cgs.bytes() +
             scal.bytes() + errflag.bytes() + scan.block_sums.bytes() + scan.total.bytes() + hd.bytes() + hf.bytes();
  for (auto &t : topo) b += t.bytes();
  return b;
}

void Scene::release() {
  for (auto *b : {&pd, &pd_alt, &m, &v, &xi, &mv, &mxi, &dv, &g, &pdir, &q, &g_new, &dv_new, &vtmp, &hist_s,
                  &hist_y, &Lv, &Lp, &part, &scal, &Le, &dv_e, &g_e, &gscr, &tr_alpha})
    b->release();
  lstate.release();
  for (auto *b : {&cg_r, &cg_z, &cg_p, &cg_Ap}) b->release();
  cgs.release();
  for (auto *b : {&pmat, &pmat_alt, &pid, &pid_alt, &slot, &perm, &tmp, &cell_count, &cell_start, &cell_first,
                  &cell_n, &cell_key, &blk_first, &blk_end, &blk_key, &flags, &flag_scan, &errflag, &tr_int})
    b->release();
  key.release();
  fixed.release();
  mat_table.release();
  bc_dev.release();
  scan.block_sums.release();
  scan.total.release();
  for (auto &t : topo) t.release();
  hd.release();
  hf.release();
  for (auto e : prof_ev) cudaEventDestroy(e);
  for (auto e : ev_pool) cudaEventDestroy(e);
  prof_ev.clear();
  ev_pool.clear();
}

namespace {

// material table, boundary boxes and the status word on the device (scene
// creation, and again when a parked scene comes back)
void upload_tables(Scene &s) {
  std::vector<MatParams> mt(s.mats.size());
  for (size_t k = 0; k < s.mats.size(); ++k) {
    double E = s.mats[k].E, nu = s.mats[k].nu;
    mt[k].mu = E / (2.0 * (1.0 + nu));
    mt[k].lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    mt[k].xi = std::sqrt(3.0 * (2.0 * mt[k].mu + mt[k].lam) * (2.0 * mt[k].mu + mt[k].lam) +
                         6.0 * mt[k].lam * mt[k].lam);
    mt[k].model = s.mats[k].model;
    mt[k].plastic = s.mats[k].plasticity;
    mt[k].yield = s.mats[k].yield_stress;
  }
  s.mat_table.ensure(mt.size(), 1.0);
  HOT_CUDA(cudaMemcpyAsync(s.mat_table.p, mt.data(), sizeof(MatParams) * mt.size(), cudaMemcpyHostToDevice, s.st));
  s.bc_dev.ensure(std::max<size_t>(1, s.bcs.size()), 1.0);
  if (!s.bcs.empty())
    HOT_CUDA(cudaMemcpyAsync(s.bc_dev.p, s.bcs.data(), sizeof(mpm_bc) * s.bcs.size(), cudaMemcpyHostToDevice, s.st));
  s.errflag.ensure(4, 1.0);
  HOT_CUDA(cudaMemsetAsync(s.errflag.p, 0, sizeof(int) * 4, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));   // the host vectors above are released on return
}

}  // namespace

void park_scene(Scene &s) {
  if (s.parked) return;
  HOT_CUDA(cudaStreamSynchronize(s.st));
  s.peak_bytes = std::max(s.peak_bytes, s.bytes());
  const size_t np = (size_t)s.np;
  s.host_pd.resize((size_t)PF_COUNT * np);
  s.host_pmat.resize(np);
  s.host_pid.resize(np);
  if (np > 0) {
    HOT_CUDA(cudaMemcpyAsync(s.host_pd.data(), s.pd.p, sizeof(double) * PF_COUNT * np, cudaMemcpyDeviceToHost, s.st));
    HOT_CUDA(cudaMemcpyAsync(s.host_pmat.data(), s.pmat.p, sizeof(int) * np, cudaMemcpyDeviceToHost, s.st));
    HOT_CUDA(cudaMemcpyAsync(s.host_pid.data(), s.pid.p, sizeof(int) * np, cudaMemcpyDeviceToHost, s.st));
  }
  HOT_CUDA(cudaStreamSynchronize(s.st));
  s.drop_graph();
  pn_release(s);
  s.release();
  s.hd.cl_level = s.hf.cl_level = -1;
  s.nlev = 0;
  s.phase = PH_IDLE;
  s.has_grid = s.has_solution = false;
  s.parked = true;
}

void ensure_resident(Scene &s) {
  if (!s.parked) return;
  const size_t np = (size_t)s.np;
  try {
    upload_tables(s);
    s.pd.ensure((size_t)PF_COUNT * np + 1, 1.0);
    s.pmat.ensure(np + 1, 1.0);
    s.pid.ensure(np + 1, 1.0);
  } catch (...) {
    s.release();   // stays parked, nothing half-resident
    throw;
  }
  if (np > 0) {
    HOT_CUDA(cudaMemcpyAsync(s.pd.p, s.host_pd.data(), sizeof(double) * PF_COUNT * np, cudaMemcpyHostToDevice, s.st));
    HOT_CUDA(cudaMemcpyAsync(s.pmat.p, s.host_pmat.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s.st));
    HOT_CUDA(cudaMemcpyAsync(s.pid.p, s.host_pid.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s.st));
  }
  HOT_CUDA(cudaStreamSynchronize(s.st));
  std::vector<double>().swap(s.host_pd);
  std::vector<int>().swap(s.host_pmat);
  std::vector<int>().swap(s.host_pid);
  s.parked = false;
}

namespace {

void validate_opts(const mpm_solver_opts *o) {
  if (!o) fail(MPM_ERR_INVALID_ARG, "opts is NULL");
  if (!(o->eps > 0.0)) fail(MPM_ERR_INVALID_ARG, "eps must be > 0");
  if (o->cn_mode != 0 && o->cn_mode != 1) fail(MPM_ERR_INVALID_ARG, "cn_mode must be 0 or 1");
  if (o->lbfgs_m < 1 || o->lbfgs_m > MAX_HIST) fail(MPM_ERR_INVALID_ARG, "lbfgs_m must be in 1..16");
  if (o->levels < 1 || o->levels > MAX_LEVELS) fail(MPM_ERR_INVALID_ARG, "levels must be in 1..8");
  if (o->precision != 0 && o->precision != 1) fail(MPM_ERR_INVALID_ARG, "precision must be 0 or 1");
  if (o->max_iters < 1 || o->max_ls < 1) fail(MPM_ERR_INVALID_ARG, "max_iters and max_ls must be >= 1");
  if (o->max_coarse_cg < 0) fail(MPM_ERR_INVALID_ARG, "max_coarse_cg must be >= 0");
  if (o->solver < 0 || o->solver > 2) fail(MPM_ERR_INVALID_ARG, "solver must be 0 (HOT), 1 (PN-PCG) or 2 (PN-MGPCG)");
  if (o->refresh_every < 0) fail(MPM_ERR_INVALID_ARG, "refresh_every must be >= 0");
  if (o->fallback_after < 0) fail(MPM_ERR_INVALID_ARG, "fallback_after must be >= 0");
  if (o->dt <= 0.0 && !(o->fps > 0.0 && o->cfl > 0.0)) fail(MPM_ERR_INVALID_ARG, "need dt > 0 or fps, cfl > 0");
}

}  // namespace

// Refresh extension (not in Alg. 3): rebuild the hierarchy at the top of
// iteration it > 0 every refresh_every iterations.
bool refresh_due(const mpm_solver_opts &o, int it) { return o.refresh_every > 0 && it > 0 && it % o.refresh_every == 0; }

namespace {

void compute_dt(Scene &s) {
  if (s.opts.dt > 0.0) {
    s.dt = s.opts.dt;
    return;
  }
  double vmax = s.np ? max_particle_speed(s) : 0.0;
  double dt = 1.0 / s.opts.fps;
  if (vmax > 0.0) dt = std::min(dt, s.opts.cfl * s.geo.dx / vmax);
  s.dt = dt;
}

void do_p2g(Scene &s) {
  ensure_resident(s);
  s.drop_graph();
  HOT_CUDA(cudaMemsetAsync(s.errflag.p, 0, sizeof(int), s.st));
  compute_dt(s);
  if (s.np > 0) {
    bin_and_sort(s);
    int e = read_errflag(s);
    if (e & DEV_ERR_DOMAIN) fail(MPM_ERR_DOMAIN, "a particle stencil leaves the grid (3 cells from the walls)");
  } else {
    s.n_cells = s.n_blocks = 0;
  }
  build_level0_nodes(s);
  p2g_transfer(s);
  s.nlev = 0;
  s.phase = PH_P2G;
  s.has_grid = true;
  s.has_solution = false;
}

template <class T>
void build_hier(Scene &s, Hier<T> &h) {
  const int64_t n = s.nn();
  h.cl_level = -1;   // re-plan the coarsest solve for the new hierarchy
  s.Lv.ensure(9 * (size_t)s.np + 9);
  velocity_gradient(s, s.v.p, nullptr, s.Lv.p);      // F at dv = 0
  build_pattern0(s);
  build_colors(s, 0);
  particle_stiffness<T>(s, h);
  hessian_assemble<T>(s, h);
  finalize_values<T>(s, h, 0);
  int M = 1;
  const int levels = s.opts.solver == 1 ? 1 : s.opts.levels;   // PN-PCG needs the fine matrix only
  for (int m = 0; m + 1 < levels; ++m) {
    build_coarse_topology(s, m);
    build_colors(s, m + 1);
    rap<T>(s, h, m);
    finalize_values<T>(s, h, m + 1);
    M = m + 2;
  }
  s.nlev = M;
  (void)n;
}

void do_build(Scene &s) {
  if (s.phase < PH_P2G) fail(MPM_ERR_STATE, "mpm_p2g must run before the hierarchy is built");
  s.drop_graph();
  if (s.opts.precision == 0) build_hier<double>(s, s.hd);
  else build_hier<float>(s, s.hf);
  s.phase = PH_HIER;
}

void run_vcycle(Scene &s, const double *b, double *u, bool use_graph) {
  if (s.opts.precision == 0) vcycle<double>(s, s.hd, b, u, use_graph);
  else vcycle<float>(s, s.hf, b, u, use_graph);
}
void reset_log(Scene &s) {
  if (s.opts.precision == 0) reset_cg_log<double>(s, s.hd);
  else reset_cg_log<float>(s, s.hf);
}
std::vector<int> read_log(Scene &s) {
  return s.opts.precision == 0 ? read_cg_log<double>(s, s.hd) : read_cg_log<float>(s, s.hf);
}

// Alg. 1 (the comparison solvers): Newton iterations with the projected
// Hessian rebuilt at every iterate, the inexact CG solve (newton.cu), the
// same backtracking line search and termination test as the L-BFGS loop.
void pn_loop(Scene &s, double &E, double norms[2], double thr, double &nrm, int &it, int &trials_total,
             int &inner_total, mpm_status &status) {
  const int64_t n3 = 3 * s.nn();
  if (s.nn() == 0) return;
  pn_prepare(s);
  while (true) {
    if (!std::isfinite(norms[0]) || !std::isfinite(norms[1]) || !std::isfinite(E)) {
      status = MPM_ERR_NUMERIC;
      break;
    }
    nrm = std::sqrt(s.opts.cn_mode == 0 ? norms[1] : norms[0]);
    if (nrm <= thr) break;
    if (it >= s.opts.max_iters) {
      status = MPM_ERR_NOT_CONVERGED;
      break;
    }
    if (it > 0) pn_rebuild_values(s);   // the hierarchy built for this step is the one at dv = 0
    const int cg = pn_cg_run(s);        // s.pdir <- p, H p ~ -g
    s.trace.inner.push_back(cg);
    inner_total += cg;
    velocity_gradient(s, s.pdir.p, nullptr, s.Lp.p);
    double alpha = 1.0, E1 = E;
    int t = 0;
    bool ok = false;
    for (t = 1; t <= s.opts.max_ls; ++t) {
      E1 = energy(s, s.Lv.p, s.Lp.p, alpha, s.dv.p, s.pdir.p);
      if (E1 <= E) {
        ok = true;
        break;
      }
      alpha *= 0.5;
    }
    trials_total += ok ? t : s.opts.max_ls;
    if (!ok) {
      status = MPM_ERR_LINESEARCH;
      break;
    }
    s.trace.alphas.push_back(alpha);
    s.trace.ls_trials.push_back(t);
    lincomb(s, s.dv_new.p, 1.0, s.dv.p, alpha, s.pdir.p, n3);
    axpy(s, s.Lv.p, alpha, s.Lp.p, 9 * s.np);
    std::swap(s.dv, s.dv_new);
    gradient(s, s.Lv.p, s.dv.p, s.g.p, norms);
    E = E1;
    ++it;
  }
  pn_release(s);
}

mpm_status do_solve(Scene &s, mpm_step_stats *st) {
  if (s.phase < PH_P2G) fail(MPM_ERR_STATE, "mpm_p2g must run before mpm_solve_step");
  // The projected Hessian and its hierarchy serve the iterations only: they
  // are built once the termination test at dv = 0 has asked for a first
  // iteration (a scene at rest under the tolerance skips the build).
  const bool had_hier = s.phase >= PH_HIER;
  const int64_t n = s.nn(), n3 = 3 * n;
  const int w = s.opts.lbfgs_m;
  for (auto *b : {&s.dv, &s.g, &s.pdir, &s.q, &s.g_new, &s.dv_new, &s.vtmp}) b->ensure(n3 + 3);
  s.hist_s.ensure((size_t)w * n3 + 3);
  s.hist_y.ensure((size_t)w * n3 + 3);
  s.Lv.ensure(9 * (size_t)s.np + 9);
  s.Lp.ensure(9 * (size_t)s.np + 9);
  HOT_CUDA(cudaMemsetAsync(s.dv.p, 0, sizeof(double) * n3, s.st));
  HOT_CUDA(cudaMemsetAsync(s.errflag.p, 0, sizeof(int), s.st));
  velocity_gradient(s, s.v.p, nullptr, s.Lv.p);
  s.trace.clear();
  s.graph_launches = 0;
  reset_log(s);
  s.hist_n = 0;
  s.hist_head = 0;
  const int64_t nfree = count_free(s);
  double norms[2];
  gradient(s, s.Lv.p, s.dv.p, s.g.p, norms);
  const double g1n = std::sqrt(norms[0]);
  double E = energy(s, s.Lv.p, nullptr, 0.0, s.dv.p, nullptr);
  mpm_status status = MPM_OK;
  int it = 0, trials_total = 0, cg_total = 0, inner_total = 0;
  double nrm = 0.0;
  const double thr = s.opts.cn_mode == 0 ? s.opts.eps * std::sqrt((double)nfree) : s.opts.eps * g1n;
  const bool finite0 = std::isfinite(norms[0]) && std::isfinite(norms[1]) && std::isfinite(E);
  const double nrm0 = std::sqrt(s.opts.cn_mode == 0 ? norms[1] : norms[0]);
  const bool need_iter = finite0 && !(nrm0 <= thr);
  if (need_iter && !had_hier) do_build(s);
  if (s.opts.solver != 0) {
    if (need_iter) {
      pn_loop(s, E, norms, thr, nrm, it, trials_total, inner_total, status);
    } else {
      nrm = nrm0;
      if (!finite0) status = MPM_ERR_NUMERIC;
    }
  }
  const bool on_device =
      s.opts.solver == 0 && need_iter && solve_loop_graph(s, E, norms, thr, E, nrm, it, trials_total, status);
  bool to_newton = false;   // fallback_after reached (extension)
  while (s.opts.solver == 0 && !on_device) {
    if (!std::isfinite(norms[0]) || !std::isfinite(norms[1]) || !std::isfinite(E)) {
      status = MPM_ERR_NUMERIC;
      break;
    }
    bool done;
    if (s.opts.cn_mode == 0) {
      nrm = std::sqrt(norms[1]);
      done = nrm <= s.opts.eps * std::sqrt((double)nfree);
    } else {
      nrm = std::sqrt(norms[0]);
      done = nrm <= s.opts.eps * g1n;
    }
    if (done) break;
    if (it >= s.opts.max_iters) {
      status = MPM_ERR_NOT_CONVERGED;
      break;
    }
    if (s.opts.fallback_after > 0 && it >= s.opts.fallback_after) {
      to_newton = true;
      break;
    }
    if (refresh_due(s.opts, it)) {
      // extension: the hierarchy at the current iterate, a fresh history
      pn_rebuild_values(s);
      s.hist_n = 0;
    }
    // two-loop recursion around the V-cycle initializer (Alg. 3)
    scale_copy(s, s.q.p, -1.0, s.g.p, n3);
    two_loop_first(s, s.q.p, n3);
    run_vcycle(s, s.q.p, s.pdir.p, true);
    two_loop_second(s, s.pdir.p, n3);
    int fb = 0;
    double pg = dot(s, s.pdir.p, s.g.p, n3);
    if (!(pg < 0.0)) {
      // not a descent direction: drop the history, use the V-cycle alone
      fb = 1;
      s.hist_n = 0;
      scale_copy(s, s.q.p, -1.0, s.g.p, n3);
      run_vcycle(s, s.q.p, s.pdir.p, true);
      pg = dot(s, s.pdir.p, s.g.p, n3);
      if (!(pg < 0.0)) {
        // still none (or not finite): steepest descent
        fb = 2;
        scale_copy(s, s.pdir.p, -1.0, s.g.p, n3);
      }
    }
    s.trace.fallback.push_back(fb);
    // backtracking line search on E(dv + alpha p)
    velocity_gradient(s, s.pdir.p, nullptr, s.Lp.p);
    double alpha = 1.0, E1 = E;
    int t = 0;
    bool ok = false;
    for (t = 1; t <= s.opts.max_ls; ++t) {
      E1 = energy(s, s.Lv.p, s.Lp.p, alpha, s.dv.p, s.pdir.p);
      if (E1 <= E) {
        ok = true;
        break;
      }
      alpha *= 0.5;
    }
    trials_total += ok ? t : s.opts.max_ls;
    if (!ok) {
      status = MPM_ERR_LINESEARCH;
      break;
    }
    s.trace.alphas.push_back(alpha);
    s.trace.ls_trials.push_back(t);
    const int slot = s.hist_head;
    double *sv = s.hist_s.p + (size_t)slot * n3;
    double *yv = s.hist_y.p + (size_t)slot * n3;
    lincomb(s, s.dv_new.p, 1.0, s.dv.p, alpha, s.pdir.p, n3);
    lincomb(s, sv, 1.0, s.dv_new.p, -1.0, s.dv.p, n3);
    axpy(s, s.Lv.p, alpha, s.Lp.p, 9 * s.np);
    std::swap(s.dv, s.dv_new);
    gradient(s, s.Lv.p, s.dv.p, s.g_new.p, norms);
    lincomb(s, yv, 1.0, s.g_new.p, -1.0, s.g.p, n3);
    double d3[3];
    dots3(s, yv, sv, n3, d3);   // y.s, y.y, s.s
    int skip = !(d3[0] > 1e-14 * std::sqrt(d3[1] * d3[2]));
    s.trace.skipped.push_back(skip);
    if (!skip) {
      s.hist_rho[slot] = 1.0 / d3[0];
      s.hist_head = (s.hist_head + 1) % w;
      s.hist_n = std::min(s.hist_n + 1, w);
    }
    std::swap(s.g, s.g_new);
    E = E1;
    ++it;
  }
  if (to_newton) {
    // extension: finish the step with PN-MGPCG from the current iterate
    const int solver = s.opts.solver;
    s.opts.solver = 2;
    try {
      pn_loop(s, E, norms, thr, nrm, it, trials_total, inner_total, status);
    } catch (...) {
      s.opts.solver = solver;
      throw;
    }
    s.opts.solver = solver;
  }
  int e = read_errflag(s);
  if (e & DEV_ERR_TIMEOUT) status = MPM_ERR_TIMEOUT;
  s.trace.cg_counts = read_log(s);
  for (int c : s.trace.cg_counts) cg_total += c > 0 ? c : 0;
  s.trace.iters = it;
  s.phase = PH_SOLVED;
  s.has_solution = true;
  mpm_step_stats out;
  std::memset(&out, 0, sizeof(out));
  out.iters = it;
  out.ls_trials = trials_total;
  out.coarse_cg_iters = cg_total;
  out.vcycles = (int)s.trace.cg_counts.size();
  out.final_norm = nrm;
  out.energy = E;
  out.dt_used = s.dt;
  out.n_particles = s.np;
  out.n_levels = s.nlev;
  for (int m = 0; m < s.nlev && m < 8; ++m) {
    out.n_nodes[m] = s.topo[m].n;
    out.nnz_blocks[m] = s.topo[m].nnzb;
  }
  out.status = status;
  out.graph_vcycles = s.graph_launches;
  out.device_loop = on_device ? 1 : 0;
  s.last_iters = it;
  s.last_stats = out;
  if (st) *st = out;
  return status;
}

void do_g2p(Scene &s) {
  if (s.phase != PH_SOLVED) fail(MPM_ERR_STATE, "mpm_g2p needs a solved step");
  const int64_t n3 = 3 * s.nn();
  s.vtmp.ensure(n3 + 3);
  lincomb(s, s.vtmp.p, 1.0, s.v.p, 1.0, s.dv.p, n3);
  g2p_transfer(s, s.vtmp.p);
  HOT_CUDA(cudaStreamSynchronize(s.st));
  s.phase = PH_IDLE;
}

template <class F>
mpm_status guarded(Scene *s, F &&f) {
  try {
    return f();
  } catch (const Error &e) {
    if (s) s->last_error = e.msg;
    g_last_error = e.msg;
    return e.code;
  } catch (const std::exception &e) {
    if (s) s->last_error = e.what();
    g_last_error = e.what();
    return MPM_ERR_INVALID_ARG;
  }
}

template <class T>
void hier_to_host(Scene &s, Hier<T> &h, int level, double *vals) {
  Topo &t = s.topo[level];
  std::vector<T> hv(9 * (size_t)t.nnzb);
  std::vector<int> rp(t.n + 1);
  HOT_CUDA(cudaMemcpyAsync(hv.data(), h.L[level].vals.p, sizeof(T) * hv.size(), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaMemcpyAsync(rp.data(), t.row_ptr.p, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  for (int64_t i = 0; i < t.n; ++i) {
    int b0 = rp[i], nb = rp[i + 1] - rp[i];
    for (int k = 0; k < nb; ++k)
      for (int e = 0; e < 9; ++e) vals[9 * (size_t)(b0 + k) + e] = (double)hv[9 * (size_t)b0 + (size_t)e * nb + k];
  }
}

}  // namespace
}  // namespace hot

using namespace hot;

extern "C" {

mpm_status mpm_set_allocator(mpm_alloc_fn alloc, mpm_free_fn free_fn, void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) {
    g_last_error = "alloc and free must both be set or both be NULL";
    return MPM_ERR_INVALID_ARG;
  }
  g_alloc = alloc;
  g_free = free_fn;
  g_ctx = ctx;
  return MPM_OK;
}

const char *mpm_last_error(mpm_scene_t s) {
  if (s) return reinterpret_cast<Scene *>(s)->last_error.c_str();
  return g_last_error.c_str();
}

mpm_status mpm_create_scene(const mpm_scene_desc *d, const mpm_solver_opts *o, mpm_scene_t *out) {
  return guarded(nullptr, [&]() -> mpm_status {
    if (!d || !out) fail(MPM_ERR_INVALID_ARG, "desc and out must not be NULL");
    *out = nullptr;
    validate_opts(o);
    if (d->n_particles < 0 || d->n_particles > (int64_t)INT32_MAX / 2) fail(MPM_ERR_INVALID_ARG, "bad n_particles");
    const int64_t np = d->n_particles;
    if (np > 0 && (!d->x || !d->v || !d->F || !d->vol || !d->mass))
      fail(MPM_ERR_INVALID_ARG, "x, v, F, vol and mass are required");
    if (d->n_materials < 1 || !d->materials) fail(MPM_ERR_INVALID_ARG, "at least one material is required");
    if (d->n_bcs < 0 || (d->n_bcs > 0 && !d->bcs)) fail(MPM_ERR_INVALID_ARG, "bad bcs");
    if (!(d->dx > 0.0)) fail(MPM_ERR_INVALID_ARG, "dx must be > 0");
    for (int k = 0; k < 3; ++k)
      if (d->grid_dims[k] < 8 || d->grid_dims[k] > 4096) fail(MPM_ERR_INVALID_ARG, "grid_dims must be in 8..4096");
    for (int k = 0; k < d->n_materials; ++k) {
      const mpm_material &m = d->materials[k];
      if (!(m.E > 0.0) || !(m.nu > -1.0 && m.nu < 0.5) || (m.model != 0 && m.model != 1) ||
          m.plasticity < 0 || m.plasticity > 2 || (m.plasticity == 1 && !(m.yield_stress > 0.0)))
        fail(MPM_ERR_INVALID_ARG, "bad material " + std::to_string(k));
    }
    Scene *s = new Scene();
    try {
      s->np = np;
      s->opts = *o;
      s->mats.assign(d->materials, d->materials + d->n_materials);
      if (d->n_bcs > 0) s->bcs.assign(d->bcs, d->bcs + d->n_bcs);
      s->geo.dx = d->dx;
      s->geo.inv_dx = 1.0 / d->dx;
      for (int k = 0; k < 3; ++k) {
        s->geo.dims[k] = d->grid_dims[k];
        s->geo.origin[k] = d->origin[k];
        s->geo.nb[k] = (d->grid_dims[k] + 3) / 4;
        s->gravity[k] = d->gravity[k];
      }
      s->ncell_dense = (int64_t)s->geo.nb[0] * s->geo.nb[1] * s->geo.nb[2] * 64;
      cudaStream_t st = (cudaStream_t)d->cuda_stream;
      if (st == nullptr) {
        // a private stream: the legacy default stream cannot be captured into graphs
        HOT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        s->own_stream = true;
      }
      s->set_stream(st);
      int dev = 0;
      HOT_CUDA(cudaGetDevice(&dev));
      HOT_CUDA(cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev));
      upload_tables(*s);
      s->pd.ensure((size_t)PF_COUNT * np + 1, 1.0);
      s->pmat.ensure(np + 1, 1.0);
      s->pid.ensure(np + 1, 1.0);
      if (np > 0) {
        std::vector<int> ids(np);
        for (int64_t i = 0; i < np; ++i) ids[i] = (int)i;
        HOT_CUDA(cudaMemcpyAsync(s->pid.p, ids.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s->st));
        cudaMemcpyKind kind = d->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        HOT_CUDA(cudaMemsetAsync(s->pd.p + (size_t)PF_C * np, 0, sizeof(double) * 9 * np, s->st));
        HOT_CUDA(cudaMemcpyAsync(s->pd.p + (size_t)PF_VOL * np, d->vol, sizeof(double) * np, kind, s->st));
        HOT_CUDA(cudaMemcpyAsync(s->pd.p + (size_t)PF_MASS * np, d->mass, sizeof(double) * np, kind, s->st));
        if (d->material_id) {
          if (!d->inputs_on_device) {
            for (int64_t i = 0; i < np; ++i)
              if (d->material_id[i] < 0 || d->material_id[i] >= d->n_materials)
                fail(MPM_ERR_INVALID_ARG, "material_id out of range");
          }
          HOT_CUDA(cudaMemcpyAsync(s->pmat.p, d->material_id, sizeof(int) * np, kind, s->st));
        } else {
          HOT_CUDA(cudaMemsetAsync(s->pmat.p, 0, sizeof(int) * np, s->st));
        }
        load_state_from_user_order(*s, d->x, d->v, d->F, d->C, d->inputs_on_device != 0);
      }
      HOT_CUDA(cudaStreamSynchronize(s->st));
    } catch (...) {
      s->release();
      if (s->own_stream) cudaStreamDestroy(s->st);
      delete s;
      throw;
    }
    *out = reinterpret_cast<mpm_scene_t>(s);
    return MPM_OK;
  });
}

mpm_status mpm_destroy_scene(mpm_scene_t sc) {
  if (!sc) return MPM_OK;
  Scene *s = reinterpret_cast<Scene *>(sc);
  cudaStreamSynchronize(s->st);
  s->drop_graph();
  pn_release(*s);
  s->release();
  for (auto a : s->aux_st)
    if (a) cudaStreamDestroy(a);
  if (s->own_stream) cudaStreamDestroy(s->st);
  delete s;
  return MPM_OK;
}

mpm_status mpm_set_options(mpm_scene_t sc, const mpm_solver_opts *o) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    validate_opts(o);
    bool rebuild = o->precision != s->opts.precision || o->levels != s->opts.levels;
    if (o->flags != s->opts.flags) s->drop_graph();   // launch modes are baked into the V-cycle graph
    s->opts = *o;
    if (rebuild && s->phase >= PH_HIER) s->phase = PH_P2G;
    return MPM_OK;
  });
}

mpm_status mpm_p2g(mpm_scene_t sc) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    do_p2g(*s);
    return MPM_OK;
  });
}

mpm_status mpm_build_hierarchy(mpm_scene_t sc) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    do_build(*s);
    HOT_CUDA(cudaStreamSynchronize(s->st));
    return MPM_OK;
  });
}

mpm_status mpm_solve_step(mpm_scene_t sc, mpm_step_stats *st) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    mpm_status r = do_solve(*s, st);
    if (r != MPM_OK) s->last_error = "solve ended with status " + std::to_string((int)r);
    return r;
  });
}

mpm_status mpm_g2p(mpm_scene_t sc) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    do_g2p(*s);
    return MPM_OK;
  });
}

mpm_status mpm_step(mpm_scene_t sc, mpm_step_stats *st) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    do_p2g(*s);
    mpm_status r = do_solve(*s, st);
    if (r == MPM_OK || r == MPM_ERR_NOT_CONVERGED || r == MPM_ERR_LINESEARCH) do_g2p(*s);
    if (r != MPM_OK) s->last_error = "solve ended with status " + std::to_string((int)r);
    return r;
  });
}

// Worker threads of mpm_step_batch: set by mpm_batch_autotune, else one per
// host core (a step blocks its thread in stream synchronisations, and more
// threads than cores only spin against each other).
static std::atomic<int> g_batch_workers{0};

static int batch_workers(int n) {
  int w = g_batch_workers.load();
  if (w <= 0) {
    const unsigned hc = std::thread::hardware_concurrency();
    w = hc ? (int)hc : 8;
  }
  return std::max(1, std::min(n, w));
}

mpm_status mpm_step_batch(mpm_scene_t *scenes, int32_t n, mpm_step_stats *stats) {
  if (n < 0 || (n > 0 && !scenes)) {
    g_last_error = "bad batch";
    return MPM_ERR_INVALID_ARG;
  }
  std::vector<mpm_status> res(n, MPM_OK);
  const int workers = batch_workers(n);
  // longest previous step first: a long step that starts last would set the
  // batch's end (scenes not yet stepped keep their order)
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const Scene *sa = reinterpret_cast<const Scene *>(scenes[a]), *sb = reinterpret_cast<const Scene *>(scenes[b]);
    return (sa ? sa->last_step_s : 0.0) > (sb ? sb->last_step_s : 0.0);
  });
  std::atomic<int> next{0};
  std::vector<std::thread> th;
  th.reserve(workers);
  int dev = 0;
  cudaGetDevice(&dev);
  for (int k = 0; k < workers; ++k)
    th.emplace_back([&]() {
      cudaSetDevice(dev);
      for (int q = next.fetch_add(1); q < n; q = next.fetch_add(1)) {
        const int i = order[q];
        const auto t0 = std::chrono::steady_clock::now();
        res[i] = mpm_step(scenes[i], stats ? &stats[i] : nullptr);
        if (Scene *si = reinterpret_cast<Scene *>(scenes[i]))
          si->last_step_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      }
    });
  for (auto &t : th) t.join();
  for (int i = 0; i < n; ++i)
    if (res[i] != MPM_OK) {
      g_last_error = "scene " + std::to_string(i) + ": " + reinterpret_cast<Scene *>(scenes[i])->last_error;
      return res[i];
    }
  return MPM_OK;
}

// Launch configurations tried by mpm_batch_autotune: V-cycle as a CUDA graph
// with one cooperative launch per Gauss-Seidel sweep (the single-scene
// default); V-cycle launched eagerly (no per-step graph capture, which
// serialises host threads); eager with one launch per color (no cooperative
// launches, whose co-residency requirement keeps small scenes' kernels from
// overlapping); eager with one launch per color on the finest level only (the
// coarser levels of small scenes then sweep as 16-CTA cluster launches, which
// overlap with other scenes' kernels).  None changes the arithmetic.
static const int32_t kTuneModes[4] = {0, 1, 5, 9};

mpm_status mpm_batch_autotune(mpm_scene_t *scenes, int32_t n, int32_t steps, int32_t *flags_out,
                              int32_t *workers_out, double *rate_out, int32_t *steps_run_out) {
  if (n <= 0 || !scenes || steps < 1) {
    g_last_error = "bad batch";
    return MPM_ERR_INVALID_ARG;
  }
  int64_t particles = 0;
  for (int i = 0; i < n; ++i) {
    if (!scenes[i]) {
      g_last_error = "NULL scene in batch";
      return MPM_ERR_INVALID_ARG;
    }
    particles += reinterpret_cast<Scene *>(scenes[i])->np;
  }
  const unsigned hc = std::thread::hardware_concurrency();
  const int cores = hc ? (int)hc : 8;
  std::vector<int> wl = {std::max(1, cores / 2), cores, 2 * cores};
  if (wl[0] == wl[1]) wl.erase(wl.begin());
  // candidates: launch mode (bits 0, 2) x rows per block of the per-color
  // sweeps (bits 8-9, only where those launches run) x worker threads
  std::vector<int> cand;
  for (int mode : kTuneModes) {
    if (mode & 12)
      for (int wb = 0; wb < 4; ++wb) cand.push_back(mode | (wb << 8));
    else
      cand.push_back(mode);
  }
  const int kTuned = 1 | 4 | 8 | (3 << 8);
  double best = -1.0;
  int best_mode = 0, best_w = cores, runs = 0;
  for (int mode : cand) {
    for (int w : wl) {
      for (int i = 0; i < n; ++i) {
        Scene *s = reinterpret_cast<Scene *>(scenes[i]);
        s->opts.flags = (s->opts.flags & ~kTuned) | mode;
      }
      g_batch_workers.store(w);
      const auto t0 = std::chrono::steady_clock::now();
      for (int k = 0; k < steps; ++k) {
        const mpm_status r = mpm_step_batch(scenes, n, nullptr);
        if (r != MPM_OK) return r;
        ++runs;
      }
      const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      const double rate = (double)particles * steps / secs;
      if (rate > best) {
        best = rate;
        best_mode = mode;
        best_w = w;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    Scene *s = reinterpret_cast<Scene *>(scenes[i]);
    s->opts.flags = (s->opts.flags & ~kTuned) | best_mode;
  }
  g_batch_workers.store(best_w);
  if (flags_out) *flags_out = best_mode;
  if (workers_out) *workers_out = best_w;
  if (rate_out) *rate_out = best;
  if (steps_run_out) *steps_run_out = runs;
  return MPM_OK;
}

mpm_status mpm_get_state(mpm_scene_t sc, double *x, double *v, double *F, double *C, int32_t to_device) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    ensure_resident(*s);
    scatter_state_to_user_order(*s, x, v, F, C, to_device != 0);
    return MPM_OK;
  });
}

mpm_status mpm_set_state(mpm_scene_t sc, const double *x, const double *v, const double *F, const double *C,
                         int32_t from_device) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    ensure_resident(*s);
    load_state_from_user_order(*s, x, v, F, C, from_device != 0);
    s->phase = PH_IDLE;
    s->has_grid = s->has_solution = false;
    return MPM_OK;
  });
}

mpm_status mpm_get_grid(mpm_scene_t sc, int64_t *n_nodes, int32_t *node_ijk, double *m, double *v, double *xi,
                        int32_t *fixed, double *dv) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    if (!s->has_grid && (node_ijk || m || v || xi || fixed || dv)) fail(MPM_ERR_STATE, "no grid before mpm_p2g");
    const int64_t n = s->has_grid ? s->nn() : 0;
    if (n_nodes) *n_nodes = n;
    if (n == 0) return MPM_OK;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
      HOT_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->st));
    };
    if (node_ijk) cp(node_ijk, s->topo[0].coords.p, sizeof(int) * 3 * n);
    if (m) cp(m, s->m.p, sizeof(double) * n);
    if (v) cp(v, s->v.p, sizeof(double) * 3 * n);
    if (xi) cp(xi, s->xi.p, sizeof(double) * n);
    std::vector<uint8_t> fx;
    if (fixed) {
      fx.resize(n);
      cp(fx.data(), s->fixed.p, n);
    }
    if (dv) {
      if (s->has_solution) cp(dv, s->dv.p, sizeof(double) * 3 * n);
      else std::memset(dv, 0, sizeof(double) * 3 * n);
    }
    HOT_CUDA(cudaStreamSynchronize(s->st));
    if (fixed)
      for (int64_t i = 0; i < n; ++i) fixed[i] = fx[i];
    return MPM_OK;
  });
}

mpm_status mpm_eval_energy(mpm_scene_t sc, const double *dvh, double *E) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s || !dvh || !E) fail(MPM_ERR_INVALID_ARG, "NULL argument");
    if (s->phase < PH_P2G) fail(MPM_ERR_STATE, "mpm_p2g must run first");
    const int64_t n3 = 3 * s->nn();
    s->dv_e.ensure(n3 + 3);
    s->Le.ensure(9 * (size_t)s->np + 9);
    HOT_CUDA(cudaMemcpyAsync(s->dv_e.p, dvh, sizeof(double) * n3, cudaMemcpyHostToDevice, s->st));
    velocity_gradient(*s, s->v.p, s->dv_e.p, s->Le.p);
    *E = energy(*s, s->Le.p, nullptr, 0.0, s->dv_e.p, nullptr);
    return MPM_OK;
  });
}

mpm_status mpm_eval_gradient(mpm_scene_t sc, const double *dvh, double *gh) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s || !dvh || !gh) fail(MPM_ERR_INVALID_ARG, "NULL argument");
    if (s->phase < PH_P2G) fail(MPM_ERR_STATE, "mpm_p2g must run first");
    const int64_t n3 = 3 * s->nn();
    s->dv_e.ensure(n3 + 3);
    s->g_e.ensure(n3 + 3);
    s->Le.ensure(9 * (size_t)s->np + 9);
    HOT_CUDA(cudaMemcpyAsync(s->dv_e.p, dvh, sizeof(double) * n3, cudaMemcpyHostToDevice, s->st));
    velocity_gradient(*s, s->v.p, s->dv_e.p, s->Le.p);
    double norms[2];
    gradient(*s, s->Le.p, s->dv_e.p, s->g_e.p, norms);
    HOT_CUDA(cudaMemcpyAsync(gh, s->g_e.p, sizeof(double) * n3, cudaMemcpyDeviceToHost, s->st));
    HOT_CUDA(cudaStreamSynchronize(s->st));
    return MPM_OK;
  });
}

mpm_status mpm_get_hessian(mpm_scene_t sc, int32_t level, int64_t *n_rows, int64_t *nnz_blocks, int32_t *row_ptr,
                           int32_t *cols, double *vals, int32_t *coords) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    if (s->phase < PH_HIER || s->nlev == 0)
      fail(MPM_ERR_STATE, "no hierarchy: call mpm_build_hierarchy (or mpm_solve_step on a scene that iterates)");
    if (level < 0 || level >= s->nlev) fail(MPM_ERR_INVALID_ARG, "level out of range");
    Topo &t = s->topo[level];
    if (n_rows) *n_rows = t.n;
    if (nnz_blocks) *nnz_blocks = t.nnzb;
    if (row_ptr) HOT_CUDA(cudaMemcpyAsync(row_ptr, t.row_ptr.p, sizeof(int) * (t.n + 1), cudaMemcpyDeviceToHost, s->st));
    if (cols) HOT_CUDA(cudaMemcpyAsync(cols, t.cols.p, sizeof(int) * t.nnzb, cudaMemcpyDeviceToHost, s->st));
    if (coords) HOT_CUDA(cudaMemcpyAsync(coords, t.coords.p, sizeof(int) * 3 * t.n, cudaMemcpyDeviceToHost, s->st));
    HOT_CUDA(cudaStreamSynchronize(s->st));
    if (vals) {
      if (s->opts.precision == 0) hier_to_host<double>(*s, s->hd, level, vals);
      else hier_to_host<float>(*s, s->hf, level, vals);
    }
    return MPM_OK;
  });
}

mpm_status mpm_apply_vcycle(mpm_scene_t sc, const double *b, double *u, int32_t *cg_iters) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s || !b || !u) fail(MPM_ERR_INVALID_ARG, "NULL argument");
    if (s->phase < PH_HIER || s->nlev == 0) fail(MPM_ERR_STATE, "no hierarchy: call mpm_build_hierarchy first");
    const int64_t n3 = 3 * s->nn();
    s->dv_e.ensure(n3 + 3);
    s->g_e.ensure(n3 + 3);
    HOT_CUDA(cudaMemsetAsync(s->errflag.p, 0, sizeof(int), s->st));
    HOT_CUDA(cudaMemcpyAsync(s->dv_e.p, b, sizeof(double) * n3, cudaMemcpyHostToDevice, s->st));
    reset_log(*s);
    run_vcycle(*s, s->dv_e.p, s->g_e.p, false);
    HOT_CUDA(cudaMemcpyAsync(u, s->g_e.p, sizeof(double) * n3, cudaMemcpyDeviceToHost, s->st));
    HOT_CUDA(cudaStreamSynchronize(s->st));
    std::vector<int> lg = read_log(*s);
    if (cg_iters) *cg_iters = lg.empty() ? 0 : lg.back();
    if (read_errflag(*s) & DEV_ERR_TIMEOUT) fail(MPM_ERR_TIMEOUT, "a device-side barrier of the V-cycle timed out");
    return MPM_OK;
  });
}

mpm_status mpm_scene_park(mpm_scene_t sc) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    park_scene(*s);
    return MPM_OK;
  });
}

mpm_status mpm_scene_unpark(mpm_scene_t sc) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    ensure_resident(*s);
    return MPM_OK;
  });
}

mpm_status mpm_set_wait_limit(mpm_scene_t sc, int64_t polls) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    if (polls < 1) fail(MPM_ERR_INVALID_ARG, "polls must be >= 1");
    HOT_CUDA(cudaStreamSynchronize(s->st));
    s->spin_limit = polls;
    s->drop_graph();   // captured launches carry the old limit
    return MPM_OK;
  });
}

mpm_status mpm_get_inner_iters(mpm_scene_t sc, int32_t capacity, int32_t *n, int32_t *cg_iters) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s || !n) fail(MPM_ERR_INVALID_ARG, "NULL argument");
    const std::vector<int> &v = s->trace.inner;
    *n = (int32_t)v.size();
    const int k = std::min<int>(capacity, (int)v.size());
    for (int i = 0; i < k; ++i)
      if (cg_iters) cg_iters[i] = v[i];
    return MPM_OK;
  });
}

mpm_status mpm_get_trace(mpm_scene_t sc, int32_t capacity, int32_t *n_iters, double *alphas, int32_t *ls_trials,
                         int32_t *skipped, int32_t *fallback, int32_t *n_vcycles, int32_t *cg_counts) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    const Trace &t = s->trace;
    if (n_iters) *n_iters = t.iters;
    if (n_vcycles) *n_vcycles = (int)t.cg_counts.size();
    int ni = std::min<int>(capacity, (int)t.alphas.size());
    for (int i = 0; i < ni; ++i) {
      if (alphas) alphas[i] = t.alphas[i];
      if (ls_trials) ls_trials[i] = t.ls_trials[i];
    }
    int nf = std::min<int>(capacity, (int)t.fallback.size());
    for (int i = 0; i < nf; ++i)
      if (fallback) fallback[i] = t.fallback[i];
    int ns = std::min<int>(capacity, (int)t.skipped.size());
    for (int i = 0; i < ns; ++i)
      if (skipped) skipped[i] = t.skipped[i];
    int nc = std::min<int>(capacity, (int)t.cg_counts.size());
    for (int i = 0; i < nc; ++i)
      if (cg_counts) cg_counts[i] = t.cg_counts[i];
    return MPM_OK;
  });
}

mpm_status mpm_profile(mpm_scene_t sc, int32_t enable, const char *only) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s) fail(MPM_ERR_INVALID_ARG, "scene is NULL");
    HOT_CUDA(cudaStreamSynchronize(s->st));
    if (enable) {
      for (auto e : s->prof_ev) s->ev_pool.push_back(e);
      s->prof_ev.clear();
      s->prof_ids.clear();
      s->prof_names.clear();
    }
    s->prof = enable != 0;
    s->prof_only = only ? only : "";
    return MPM_OK;
  });
}

mpm_status mpm_profile_read(mpm_scene_t sc, int32_t capacity, int32_t *count, char *names, double *total_ms,
                            int64_t *launches) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  return guarded(s, [&]() -> mpm_status {
    if (!s || !count) fail(MPM_ERR_INVALID_ARG, "NULL argument");
    HOT_CUDA(cudaStreamSynchronize(s->st));
    const int nk = (int)s->prof_names.size();
    std::vector<double> ms(nk, 0.0);
    std::vector<int64_t> cnt(nk, 0);
    for (size_t k = 0; k < s->prof_ids.size(); ++k) {
      float t = 0.f;
      HOT_CUDA(cudaEventElapsedTime(&t, s->prof_ev[2 * k], s->prof_ev[2 * k + 1]));
      ms[s->prof_ids[k]] += t;
      cnt[s->prof_ids[k]] += 1;
    }
    *count = nk;
    for (int k = 0; k < nk && k < capacity; ++k) {
      if (names) {
        std::memset(names + 32 * k, 0, 32);
        std::strncpy(names + 32 * k, s->prof_names[k].c_str(), 31);
      }
      if (total_ms) total_ms[k] = ms[k];
      if (launches) launches[k] = cnt[k];
    }
    return MPM_OK;
  });
}

int64_t mpm_kernel_launch_count(void) { return (int64_t)g_launches.load(); }

mpm_status mpm_scene_footprint(mpm_scene_t sc, int64_t *bytes) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  if (!s || !bytes) return MPM_ERR_INVALID_ARG;
  *bytes = (int64_t)s->bytes();
  return MPM_OK;
}

mpm_status mpm_scene_residency(mpm_scene_t sc, int32_t *parked, int64_t *peak_bytes) {
  Scene *s = reinterpret_cast<Scene *>(sc);
  if (!s) return MPM_ERR_INVALID_ARG;
  if (parked) *parked = s->parked ? 1 : 0;
  if (peak_bytes) *peak_bytes = (int64_t)std::max(s->peak_bytes, s->bytes());
  return MPM_OK;
}

}  // extern "C"
