// Alg. 3's L-BFGS iterations as one CUDA graph.
//
// Every decision the host-driven loop takes between kernels -- the
// termination test (Sec. 5.2), the restarts of a non-descent direction, the
// line search's halvings, the pair-skip rule and the history ring -- is taken
// here by a one-thread kernel from the same partial sums, summed in the same
// order, and steers conditional graph nodes: WHILE for the iterations and for
// the line search, IF for the two restarts and for the update after an
// accepted step.  The two loops give bitwise the same iterates; this one
// needs no host round trip per iteration (one per step).
#include "graph_capture.h"
#include "internal.h"

namespace hot {
namespace {

// part[stride * b + off] for b = 0..n-1, summed in order (the host loop's order)
__device__ double seq_sum(const double *part, int n, int stride, int off) {
  double s = 0.0;
  for (int b = 0; b < n; ++b) s += part[stride * b + off];
  return s;
}

// termination test at the top of an iteration; thr = eps sqrt(n_free) (CN)
// or eps |g^1| (relative)
__global__ void k_loop_check(LoopState *st, int cn_mode, double thr, int max_iters, cudaGraphConditionalHandle h) {
  int go = 0;
  if (st->status == MPM_OK) {
    const double n0 = st->n0, n1 = st->n1;
    if (!isfinite(n0) || !isfinite(n1) || !isfinite(st->E)) {
      st->status = MPM_ERR_NUMERIC;
    } else {
      const double nrm = sqrt(cn_mode == 0 ? n1 : n0);
      st->nrm = nrm;
      if (!(nrm <= thr)) {
        if (st->it >= max_iters)
          st->status = MPM_ERR_NOT_CONVERGED;
        else
          go = 1;
      }
    }
  }
  cudaGraphSetConditional(h, go);
}

// p^T g from its partials; level 1: a non-descent direction drops the history
// and restarts from the V-cycle alone; level 2: then from -g
__global__ void k_pg_decide(const double *part, int G, LoopState *st, int level, cudaGraphConditionalHandle h) {
  const double pg = seq_sum(part, G, 3, 0);
  st->pg = pg;
  const int bad = !(pg < 0.0);
  if (level == 1) {
    st->fb = bad ? 1 : 0;
    if (bad) st->hist_n = 0;
  } else if (bad) {
    st->fb = 2;
  }
  cudaGraphSetConditional(h, bad);
}

__global__ void k_ls_init(LoopState *st, cudaGraphConditionalHandle h) {
  st->alpha = 1.0;
  st->t = 1;
  st->ok = 0;
  cudaGraphSetConditional(h, 1);
}

// one backtracking trial: accept if E(dv + alpha p) <= E(dv), else halve
__global__ void k_ls_decide(const double *part, int n, LoopState *st, int max_ls, cudaGraphConditionalHandle h) {
  const double E1 = seq_sum(part, n, 1, 0);
  st->E1 = E1;
  int go = 0;
  if (E1 <= st->E) {
    st->ok = 1;
  } else {
    st->alpha *= 0.5;
    if (st->t < max_ls) {
      st->t += 1;
      go = 1;
    }
  }
  cudaGraphSetConditional(h, go);
}

// trace of the iteration; the update runs only after an accepted step
__global__ void k_ls_after(LoopState *st, int max_ls, double *tr_alpha, int *tr_int, int cap,
                           cudaGraphConditionalHandle h) {
  const int it = st->it;
  if (it < cap) tr_int[2 * cap + it] = st->fb;
  if (st->ok) {
    st->trials_total += st->t;
    if (it < cap) {
      tr_alpha[it] = st->alpha;
      tr_int[it] = st->t;
    }
  } else {
    st->trials_total += max_ls;
    st->status = MPM_ERR_LINESEARCH;
  }
  cudaGraphSetConditional(h, st->ok);
}

// hierarchy refresh (an extension of Alg. 3): every `every` iterations the
// projected Hessian and its hierarchy are rebuilt at the current iterate and
// the history restarts, as in the host-driven loop
__global__ void k_refresh_decide(LoopState *st, int every, cudaGraphConditionalHandle h) {
  const int go = st->it > 0 && st->it % every == 0;   // the host loop's rule (refresh_due)
  if (go) st->hist_n = 0;
  cudaGraphSetConditional(h, go);
}

__global__ void k_norms(const double *part, int nb, LoopState *st) {
  st->n0 = seq_sum(part, nb, 2, 0);
  st->n1 = seq_sum(part, nb, 2, 1);
}

// the pair (s, y) enters the history unless y^T s <= 1e-14 |y| |s|
__global__ void k_pair_decide(const double *part, int G, LoopState *st, int w, int *tr_int, int cap) {
  const double d0 = seq_sum(part, G, 3, 0), d1 = seq_sum(part, G, 3, 1), d2 = seq_sum(part, G, 3, 2);
  const int skip = !(d0 > 1e-14 * sqrt(d1 * d2));
  const int it = st->it;
  if (it < cap) tr_int[cap + it] = skip;
  if (!skip) {
    const int slot = st->head;
    st->rho[slot] = 1.0 / d0;
    st->head = (slot + 1) % w;
    st->hist_n = min(st->hist_n + 1, w);
  }
  st->E = st->E1;
  st->it = it + 1;
}


void vc_ready(Scene &s) {
  if (s.opts.precision == 0) vcycle_ready<double>(s, s.hd);
  else vcycle_ready<float>(s, s.hf);
}
void vc_emit(Scene &s, const double *b, double *u) {
  if (s.opts.precision == 0) vcycle_emit<double>(s, s.hd, b, u);
  else vcycle_emit<float>(s, s.hf, b, u);
}

// kernels captured into each part of the graph, to count the ones it runs
struct Counts {
  long long top = 0, body = 0, fb1 = 0, fb2 = 0, ls = 0, upd = 0, refresh = 0;
};

}  // namespace

bool solve_loop_graph(Scene &s, double E0, double norms0[2], double thr, double &E, double &nrm, int &it,
                      int &trials_total, mpm_status &status) {
  if (!s.loop_graph_ok || !s.graphs_ok || s.prof || (s.opts.flags & 17) || s.nn() == 0 ||
      s.opts.fallback_after > 0)
    return false;
  const int refresh = s.opts.refresh_every;
  // building the graph costs about as much host time as a handful of host-
  // driven iterations: by default it is used once the scene's previous solve
  // took at least DEVICE_LOOP_MIN_ITERS iterations (bit 5 forces it)
  if (!(s.opts.flags & 32) && s.last_iters < DEVICE_LOOP_MIN_ITERS) return false;
  const int64_t n3 = 3 * s.nn();
  const int w = s.opts.lbfgs_m, cap = s.opts.max_iters + 1, max_ls = s.opts.max_ls;
  const int cn = s.opts.cn_mode, max_iters = s.opts.max_iters;
  // every buffer the graph touches, sized before the capture (no allocation inside)
  s.lstate.ensure(1);
  s.tr_alpha.ensure(cap);
  s.tr_int.ensure(3 * (size_t)cap);
  s.part.ensure(4096);
  s.scal.ensure(64);
  s.gscr.ensure((size_t)54 * s.np, 1.0);   // the gradient's factor tables
  for (auto &a : s.aux_st)
    if (!a) HOT_CUDA(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
  vc_ready(s);
  LoopState *st = s.lstate.p;
  double *tra = s.tr_alpha.p;
  int *tri = s.tr_int.p;

  cudaGraph_t top = nullptr;
  cudaGraphExec_t exec = nullptr;
  Counts c;
  const long long c_start = launch_count();
  try {
    HOT_CUDA(cudaGraphCreate(&top, 0));
    HOT_CUDA(cudaStreamBeginCaptureToGraph(s.st, top, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const cudaGraphConditionalHandle h_it = new_handle(s.st);
    k_loop_check<<<1, 1, 0, s.st>>>(st, cn, thr, max_iters, h_it);
    HOT_LAUNCH("k_loop_check");
    cudaGraph_t body = add_conditional(s.st, h_it, cudaGraphCondTypeWhile);
    {
      cudaGraph_t g = nullptr;
      HOT_CUDA(cudaStreamEndCapture(s.st, &g));
    }
    c.top = launch_count() - c_start;

    // one iteration of Alg. 3
    const long long b0 = launch_count();
    HOT_CUDA(cudaStreamBeginCaptureToGraph(s.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (refresh > 0) {
      const cudaGraphConditionalHandle h_rf = new_handle(s.st);
      k_refresh_decide<<<1, 1, 0, s.st>>>(st, refresh, h_rf);
      HOT_LAUNCH("k_refresh_decide");
      cudaGraph_t rf = add_conditional(s.st, h_rf, cudaGraphCondTypeIf);
      const long long r0 = launch_count();
      capture_into(s, 0, rf, [&] { pn_rebuild_values(s); });
      c.refresh = launch_count() - r0;
    }
    scale_copy(s, s.q.p, -1.0, s.g.p, n3);
    two_loop_first_dev(s, s.q.p, n3, st);
    vc_emit(s, s.q.p, s.pdir.p);
    two_loop_second_dev(s, s.pdir.p, n3, st);
    {
      const int G = dot_launch(s, s.pdir.p, s.g.p, n3, 0, s.part.p);
      const cudaGraphConditionalHandle h_fb1 = new_handle(s.st);
      k_pg_decide<<<1, 1, 0, s.st>>>(s.part.p, G, st, 1, h_fb1);
      HOT_LAUNCH("k_pg_decide");
      cudaGraph_t fb1 = add_conditional(s.st, h_fb1, cudaGraphCondTypeIf);
      const long long f0 = launch_count();
      capture_into(s, 0, fb1, [&] {
        scale_copy(s, s.q.p, -1.0, s.g.p, n3);
        vc_emit(s, s.q.p, s.pdir.p);
        const int G2 = dot_launch(s, s.pdir.p, s.g.p, n3, 0, s.part.p);
        const cudaGraphConditionalHandle h_fb2 = new_handle(s.st);
        k_pg_decide<<<1, 1, 0, s.st>>>(s.part.p, G2, st, 2, h_fb2);
        HOT_LAUNCH("k_pg_decide");
        cudaGraph_t fb2 = add_conditional(s.st, h_fb2, cudaGraphCondTypeIf);
        const long long f2 = launch_count();
        capture_into(s, 1, fb2, [&] { scale_copy(s, s.pdir.p, -1.0, s.g.p, n3); });
        c.fb2 = launch_count() - f2;
      });
      c.fb1 = launch_count() - f0 - c.fb2;
    }
    velocity_gradient(s, s.pdir.p, nullptr, s.Lp.p);
    {
      const cudaGraphConditionalHandle h_ls = new_handle(s.st);
      k_ls_init<<<1, 1, 0, s.st>>>(st, h_ls);
      HOT_LAUNCH("k_ls_init");
      cudaGraph_t lsb = add_conditional(s.st, h_ls, cudaGraphCondTypeWhile);
      const long long l0 = launch_count();
      capture_into(s, 0, lsb, [&] {
        const int np = energy_launch(s, s.Lv.p, s.Lp.p, 0.0, &st->alpha, s.dv.p, s.pdir.p);
        k_ls_decide<<<1, 1, 0, s.st>>>(s.part.p, np, st, max_ls, h_ls);
        HOT_LAUNCH("k_ls_decide");
      });
      c.ls = launch_count() - l0;
    }
    {
      const cudaGraphConditionalHandle h_upd = new_handle(s.st);
      k_ls_after<<<1, 1, 0, s.st>>>(st, max_ls, tra, tri, cap, h_upd);
      HOT_LAUNCH("k_ls_after");
      cudaGraph_t upd = add_conditional(s.st, h_upd, cudaGraphCondTypeIf);
      const long long u0 = launch_count();
      capture_into(s, 0, upd, [&] {
        lincomb_alpha(s, s.dv_new.p, s.dv.p, s.pdir.p, n3, st);   // dv + alpha p
        hist_diff(s, s.hist_s.p, s.dv_new.p, s.dv.p, n3, st);     // s = new - old
        axpy_alpha(s, s.Lv.p, s.Lp.p, 9 * s.np, st);
        HOT_CUDA(cudaMemcpyAsync(s.dv.p, s.dv_new.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s.st));
        const int nb = gradient_launch(s, s.Lv.p, s.dv.p, s.g_new.p);
        k_norms<<<1, 1, 0, s.st>>>(s.part.p, nb, st);
        HOT_LAUNCH("k_norms");
        hist_diff(s, s.hist_y.p, s.g_new.p, s.g.p, n3, st);      // y = g_new - g
        const int G3 = dots3_hist_launch(s, n3, st, s.part.p);
        k_pair_decide<<<1, 1, 0, s.st>>>(s.part.p, G3, st, w, tri, cap);
        HOT_LAUNCH("k_pair_decide");
        HOT_CUDA(cudaMemcpyAsync(s.g.p, s.g_new.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s.st));
      });
      c.upd = launch_count() - u0;
    }
    k_loop_check<<<1, 1, 0, s.st>>>(st, cn, thr, max_iters, h_it);
    HOT_LAUNCH("k_loop_check");
    {
      cudaGraph_t g = nullptr;
      HOT_CUDA(cudaStreamEndCapture(s.st, &g));
    }
    c.body = launch_count() - b0 - c.fb1 - c.fb2 - c.ls - c.upd - c.refresh;
    HOT_CUDA(cudaGraphInstantiate(&exec, top, 0));
  } catch (const Error &) {
    end_any_capture(s.aux_st[1]);
    end_any_capture(s.aux_st[0]);
    end_any_capture(s.st);
    if (top) cudaGraphDestroy(top);
    cudaGetLastError();
    note_launches(-(launch_count() - c_start));
    s.loop_graph_ok = false;   // the host-driven loop from now on
    return false;
  }
  note_launches(-(launch_count() - c_start));   // captured, not run

  LoopState init = {};
  init.E = E0;
  init.n0 = norms0[0];
  init.n1 = norms0[1];
  HOT_CUDA(cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, s.st));
  HOT_CUDA(cudaGraphLaunch(exec, s.st));
  LoopState out;
  HOT_CUDA(cudaMemcpyAsync(&out, st, sizeof(out), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(top);

  it = out.it;
  trials_total = out.trials_total;
  E = out.E;
  nrm = out.nrm;
  status = (mpm_status)out.status;
  const int runs = it + (status == MPM_ERR_LINESEARCH ? 1 : 0);   // iterations that reached the line search
  std::vector<double> ta(cap);
  std::vector<int> ti(3 * (size_t)cap);
  if (runs > 0) {
    HOT_CUDA(cudaMemcpyAsync(ta.data(), tra, sizeof(double) * cap, cudaMemcpyDeviceToHost, s.st));
    HOT_CUDA(cudaMemcpyAsync(ti.data(), tri, sizeof(int) * 3 * (size_t)cap, cudaMemcpyDeviceToHost, s.st));
    HOT_CUDA(cudaStreamSynchronize(s.st));
  }
  s.trace.alphas.assign(ta.begin(), ta.begin() + it);
  s.trace.ls_trials.assign(ti.begin(), ti.begin() + it);
  s.trace.skipped.assign(ti.begin() + cap, ti.begin() + cap + it);
  s.trace.fallback.assign(ti.begin() + 2 * cap, ti.begin() + 2 * cap + runs);
  long long n_fb1 = 0, n_fb2 = 0;
  for (int f : s.trace.fallback) {
    n_fb1 += f >= 1;
    n_fb2 += f == 2;
  }
  s.graph_launches = (int)(runs + n_fb1);   // V-cycles run inside the graph
  long long n_refresh = 0;   // refreshes taken
  for (int k = 1; k < runs; ++k) n_refresh += refresh_due(s.opts, k) ? 1 : 0;
  note_launches(c.top + runs * c.body + n_fb1 * c.fb1 + n_fb2 * c.fb2 + (long long)trials_total * c.ls +
                (long long)it * c.upd + n_refresh * c.refresh);
  return true;
}

}  // namespace hot
