// The paper's comparison solvers (Alg. 1, inexact projected Newton): the
// inner conjugate-gradient solve of each Newton iteration, preconditioned by
// the scalar diagonal (PN-PCG) or by one V-cycle of a hierarchy rebuilt at
// every Newton iterate (PN-MGPCG, Sec. 4.3), stopped by the inexact
// criterion of Sec. 5.3:
//   k = min(1/2, sqrt(max(sqrt(r0^T P r0), tau))),  stop when
//   sqrt(r^T P r) <= k sqrt(r0^T P r0),  r^T P r = r^T z with z = P r.
// The CG loop runs as one CUDA graph per Newton iteration (a WHILE node over
// the iterations, an IF node that skips the update when p^T H p <= 0), so a
// solve costs one host round trip, not two per CG iteration.
#include "graph_capture.h"
#include "internal.h"

namespace hot {
namespace {

constexpr int NT = 256;
constexpr int WPB = NT / 32;

__device__ double seq_sum(const double *part, int n, int stride, int off) {
  double s = 0.0;
  for (int b = 0; b < n; ++b) s += part[stride * b + off];
  return s;
}

// y = H x for the level-0 block matrix (values in T, vectors in float64),
// one warp per row
template <class T>
__global__ void k_spmv(int64_t n, const int *__restrict__ row_ptr, const int *__restrict__ cols,
                       const T *__restrict__ vals, const double *__restrict__ x, double *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
  if (i >= n) return;   // warp-uniform
  const int lane = threadIdx.x & 31;
  const int rp = row_ptr[i], nb = row_ptr[i + 1] - rp;
  const T *v = vals + 9 * (int64_t)rp;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int b = lane; b < nb; b += 32) {
    const int j = cols[rp + b];
    const double x0 = x[3 * j], x1 = x[3 * j + 1], x2 = x[3 * j + 2];
    a0 = fma((double)v[b], x0, a0);
    a1 = fma((double)v[3 * nb + b], x0, a1);
    a2 = fma((double)v[6 * nb + b], x0, a2);
    a0 = fma((double)v[nb + b], x1, a0);
    a1 = fma((double)v[4 * nb + b], x1, a1);
    a2 = fma((double)v[7 * nb + b], x1, a2);
    a0 = fma((double)v[2 * nb + b], x2, a0);
    a1 = fma((double)v[5 * nb + b], x2, a1);
    a2 = fma((double)v[8 * nb + b], x2, a2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) {
    y[3 * i] = a0;
    y[3 * i + 1] = a1;
    y[3 * i + 2] = a2;
  }
}

// z = D^-1 r with D the scalar diagonal of H
template <class T>
__global__ void k_jacobi(double *__restrict__ z, const double *__restrict__ r, const T *__restrict__ diag, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT)
    z[k] = r[k] / (double)diag[k];
}

__global__ void k_cg_init(const double *part, int G, CgState *cs, double tau, int cap, cudaGraphConditionalHandle h) {
  const double rz = seq_sum(part, G, 3, 0);
  const double bn = sqrt(fmax(rz, 0.0));
  cs->rz = rz;
  cs->bn = bn;
  cs->k = fmin(0.5, sqrt(fmax(bn, tau)));
  cs->it = 0;
  cs->stop = 0;
  cudaGraphSetConditional(h, !(sqrt(fmax(rz, 0.0)) <= cs->k * bn) && cap > 0);
}

__global__ void k_cg_alpha(const double *part, int G, CgState *cs, cudaGraphConditionalHandle h) {
  const double pAp = seq_sum(part, G, 3, 0);
  cs->pAp = pAp;
  int go = 1;
  if (pAp <= 0.0) {
    cs->stop = 1;
    go = 0;
  } else {
    cs->alpha = cs->rz / pAp;
  }
  cudaGraphSetConditional(h, go);
}

__global__ void k_cg_xr(double *x, double *r, const double *__restrict__ p, const double *__restrict__ Ap, int64_t n,
                        const CgState *__restrict__ cs) {
  const double a = cs->alpha;
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT) {
    x[k] = fma(a, p[k], x[k]);
    r[k] = fma(-a, Ap[k], r[k]);
  }
}

__global__ void k_cg_beta(const double *part, int G, CgState *cs) {
  const double rz = seq_sum(part, G, 3, 0);
  cs->beta = rz / cs->rz;
  cs->rz = rz;
  cs->it += 1;
}

__global__ void k_cg_p(double *p, const double *__restrict__ z, int64_t n, const CgState *__restrict__ cs) {
  const double b = cs->beta;
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT)
    p[k] = fma(b, p[k], z[k]);
}

__global__ void k_cg_cond(const CgState *cs, int cap, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, !cs->stop && !(sqrt(fmax(cs->rz, 0.0)) <= cs->k * cs->bn) && cs->it < cap);
}


template <class T>
void precondition(Scene &s, Hier<T> &h, const double *r, double *z, int64_t n3) {
  if (s.opts.solver == 2) {
    vcycle_emit<T>(s, h, r, z);
    return;
  }
  k_jacobi<T><<<2 * s.nsm, NT, 0, s.st>>>(z, r, h.L[0].diag.p, n3);
  HOT_LAUNCH("k_jacobi");
}

template <class T>
void build_cg_graph(Scene &s, Hier<T> &h) {
  const int64_t n = s.nn(), n3 = 3 * n;
  const int cap = MPM_PN_MAX_CG;
  const double tau = s.opts.eps;
  Topo &t = s.topo[0];
  CgState *cs = s.cgs.p;
  double *x = s.pdir.p, *r = s.cg_r.p, *z = s.cg_z.p, *p = s.cg_p.p, *Ap = s.cg_Ap.p, *part = s.part.p;
  cudaGraph_t top = nullptr;
  const long long c0 = launch_count();
  PnGraph &gr = s.pn_graph;
  try {
    HOT_CUDA(cudaGraphCreate(&top, 0));
    HOT_CUDA(cudaStreamBeginCaptureToGraph(s.st, top, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    scale_copy(s, r, -1.0, s.g.p, n3);   // r0 = b = -g, x0 = 0
    HOT_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n3, s.st));
    precondition<T>(s, h, r, z, n3);
    HOT_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s.st));
    int G = dot_launch(s, r, z, n3, 0, part);
    const cudaGraphConditionalHandle h_while = new_handle(s.st);
    k_cg_init<<<1, 1, 0, s.st>>>(part, G, cs, tau, cap, h_while);
    HOT_LAUNCH("k_cg_init");
    cudaGraph_t body = add_conditional(s.st, h_while, cudaGraphCondTypeWhile);
    {
      cudaGraph_t g = nullptr;
      HOT_CUDA(cudaStreamEndCapture(s.st, &g));
    }
    gr.top_kernels = launch_count() - c0;
    const long long b0 = launch_count();
    HOT_CUDA(cudaStreamBeginCaptureToGraph(s.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    k_spmv<T><<<(unsigned)((n + WPB - 1) / WPB), NT, 0, s.st>>>(n, t.row_ptr.p, t.cols.p, h.L[0].vals.p, p, Ap);
    HOT_LAUNCH("k_spmv");
    G = dot_launch(s, p, Ap, n3, 0, part);
    const cudaGraphConditionalHandle h_go = new_handle(s.st);
    k_cg_alpha<<<1, 1, 0, s.st>>>(part, G, cs, h_go);
    HOT_LAUNCH("k_cg_alpha");
    cudaGraph_t upd = add_conditional(s.st, h_go, cudaGraphCondTypeIf);
    const long long u0 = launch_count();
    capture_into(s, 0, upd, [&] {
      k_cg_xr<<<2 * s.nsm, NT, 0, s.st>>>(x, r, p, Ap, n3, cs);
      HOT_LAUNCH("k_cg_xr");
      precondition<T>(s, h, r, z, n3);
      const int G2 = dot_launch(s, r, z, n3, 0, part);
      k_cg_beta<<<1, 1, 0, s.st>>>(part, G2, cs);
      HOT_LAUNCH("k_cg_beta");
      k_cg_p<<<2 * s.nsm, NT, 0, s.st>>>(p, z, n3, cs);
      HOT_LAUNCH("k_cg_p");
    });
    gr.upd_kernels = launch_count() - u0;
    k_cg_cond<<<1, 1, 0, s.st>>>(cs, cap, h_while);
    HOT_LAUNCH("k_cg_cond");
    {
      cudaGraph_t g = nullptr;
      HOT_CUDA(cudaStreamEndCapture(s.st, &g));
    }
    gr.body_kernels = launch_count() - b0 - gr.upd_kernels;
    HOT_CUDA(cudaGraphInstantiate(&gr.exec, top, 0));
    gr.graph = top;
  } catch (...) {
    end_any_capture(s.aux_st[0]);
    end_any_capture(s.st);
    if (top) cudaGraphDestroy(top);
    cudaGetLastError();
    note_launches(-(launch_count() - c0));
    throw;
  }
  note_launches(-(launch_count() - c0));   // captured, not run
}

}  // namespace

void pn_prepare(Scene &s) {
  const int64_t n3 = 3 * s.nn();
  for (auto *b : {&s.cg_r, &s.cg_z, &s.cg_p, &s.cg_Ap}) b->ensure(n3 + 3);
  s.cgs.ensure(1);
  s.part.ensure(4096);
  for (auto &a : s.aux_st)
    if (!a) HOT_CUDA(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
  pn_release(s);
  if (s.opts.precision == 0) {
    if (s.opts.solver == 2) vcycle_ready<double>(s, s.hd);
    build_cg_graph<double>(s, s.hd);
  } else {
    if (s.opts.solver == 2) vcycle_ready<float>(s, s.hf);
    build_cg_graph<float>(s, s.hf);
  }
}

int pn_cg_run(Scene &s) {
  HOT_CUDA(cudaGraphLaunch(s.pn_graph.exec, s.st));
  CgState out;
  HOT_CUDA(cudaMemcpyAsync(&out, s.cgs.p, sizeof(out), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  const PnGraph &gr = s.pn_graph;
  note_launches(gr.top_kernels + (long long)(out.it + out.stop) * gr.body_kernels +
                (long long)out.it * gr.upd_kernels);
  return out.it;
}

void pn_release(Scene &s) {
  if (s.pn_graph.exec) cudaGraphExecDestroy(s.pn_graph.exec);
  if (s.pn_graph.graph) cudaGraphDestroy(s.pn_graph.graph);
  s.pn_graph.exec = nullptr;
  s.pn_graph.graph = nullptr;
}

// the projected Hessian (and, but for PN-PCG, its Galerkin hierarchy) at the
// current iterate: the stiffness is taken at F from s.Lv, the velocity
// gradient of v^n + dv
void pn_rebuild_values(Scene &s) {
  if (s.opts.precision == 0) {
    particle_stiffness<double>(s, s.hd);
    hessian_assemble<double>(s, s.hd);
    finalize_values<double>(s, s.hd, 0);
    if (s.opts.solver != 1)   // PN-PCG uses the fine matrix only
      for (int m = 0; m + 1 < s.nlev; ++m) {
        rap<double>(s, s.hd, m);
        finalize_values<double>(s, s.hd, m + 1);
      }
  } else {
    particle_stiffness<float>(s, s.hf);
    hessian_assemble<float>(s, s.hf);
    finalize_values<float>(s, s.hf, 0);
    if (s.opts.solver != 1)
      for (int m = 0; m + 1 < s.nlev; ++m) {
        rap<float>(s, s.hf, m);
        finalize_values<float>(s, s.hf, m + 1);
      }
  }
}

}  // namespace hot
