// Node-vector operations in float64 for the L-BFGS loop of Alg. 3.  Every
// reduction uses a fixed grid and sums its partials in a fixed order, so
// results are bitwise reproducible run to run.
#include "internal.h"

namespace hot {

namespace {
constexpr int NT = 256;

__global__ void k_dot3(const double *__restrict__ x, const double *__restrict__ y, int64_t n, int mode,
                       double *__restrict__ part) {
  __shared__ double sh[NT];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT) {
    double xv = x[k], yv = y[k];
    a = __fma_rn(xv, yv, a);
    if (mode) {
      b = __fma_rn(xv, xv, b);
      c = __fma_rn(yv, yv, c);
    }
  }
  a = block_sum<NT>(a, sh);
  if (mode) {
    b = block_sum<NT>(b, sh);
    c = block_sum<NT>(c, sh);
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = a;
    part[3 * blockIdx.x + 1] = b;
    part[3 * blockIdx.x + 2] = c;
  }
}

// the rounding of these is spelled out so that the device-driven loop's
// versions (scalars read on the device) give the same bits
__global__ void k_axpy(double *__restrict__ y, double a, const double *__restrict__ x, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT)
    y[k] = __fma_rn(a, x[k], y[k]);
}
__global__ void k_lincomb(double *z, double a, const double *x, double b, const double *y, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT)
    z[k] = y ? __fma_rn(b, y[k], __dmul_rn(a, x[k])) : __dmul_rn(a, x[k]);
}

// Two-loop steps with the scalar coefficient formed on the device from the
// previous step's partials:
//   first loop : alpha_a = rho_a s_a^T q;  q <- q - alpha_a y_a
//   second loop: beta = rho_a y_a^T r;     r <- r + (alpha_a - beta) s_a
// Each launch applies the update for one pair (if upd) and emits the partial
// dot of the next pair (if nxt).
__device__ __forceinline__ void twoloop_body(double *v, const double *__restrict__ upd_vec,
                                             const double *__restrict__ part_in, int nin, double rho,
                                             double *__restrict__ alpha_store, int second,
                                             const double *__restrict__ alpha_prev, const double *__restrict__ nxt,
                                             double *__restrict__ part_out, int64_t n, double *sh) {
  double coef = 0.0;
  if (upd_vec) {
    double S = sum_partials<NT>(part_in, nin, sh);
    if (!second) {
      double a = __dmul_rn(rho, S);
      coef = -a;
      if (blockIdx.x == 0 && threadIdx.x == 0) *alpha_store = a;
    } else {
      coef = __fma_rn(-rho, S, *alpha_prev);
    }
  }
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT) {
    double vk = v[k];
    if (upd_vec) {
      vk = __fma_rn(coef, upd_vec[k], vk);
      v[k] = vk;
    }
    if (nxt) acc = __fma_rn(nxt[k], vk, acc);
  }
  if (nxt) {
    acc = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) part_out[blockIdx.x] = acc;
  }
}

__global__ void k_twoloop_step(double *v, const double *__restrict__ upd_vec, const double *__restrict__ part_in,
                               int nin, double rho, double *__restrict__ alpha_store, int second,
                               const double *__restrict__ alpha_prev, const double *__restrict__ nxt,
                               double *__restrict__ part_out, int64_t n) {
  __shared__ double sh[NT];
  twoloop_body(v, upd_vec, part_in, nin, rho, alpha_store, second, alpha_prev, nxt, part_out, n, sh);
}

// The same step with its pair taken from the device state: launch j of a
// fixed sequence of w + 1 (j = -1 only emits the first partial); steps past
// the current pair count do nothing.  Slot of the k-th newest pair:
// (head - 1 - k) mod w, as on the host.
__global__ void k_twoloop_dev(double *v, const double *__restrict__ upd_base, const double *__restrict__ nxt_base,
                              int64_t n, int w, const LoopState *__restrict__ st, int j, int second,
                              const double *__restrict__ part_in, int nin, double *__restrict__ part_out,
                              double *__restrict__ alpha_base) {
  __shared__ double sh[NT];
  const int m = st->hist_n, head = st->head;
  if (m == 0 || j >= m) return;
  auto slot = [&](int k) { return ((head - 1 - k) % w + w) % w; };
  const double *upd = nullptr, *nxt = nullptr;
  double rho = 0.0;
  int a = 0;
  if (!second) {
    if (j < 0) {
      nxt = nxt_base + (int64_t)slot(0) * n;
    } else {
      a = slot(j);
      upd = upd_base + (int64_t)a * n;
      nxt = j + 1 < m ? nxt_base + (int64_t)slot(j + 1) * n : nullptr;
      rho = st->rho[a];
    }
  } else {
    if (j < 0) {
      nxt = nxt_base + (int64_t)slot(m - 1) * n;
    } else {
      const int k = m - 1 - j;
      a = slot(k);
      upd = upd_base + (int64_t)a * n;
      nxt = k - 1 >= 0 ? nxt_base + (int64_t)slot(k - 1) * n : nullptr;
      rho = st->rho[a];
    }
  }
  twoloop_body(v, upd, part_in, nin, rho, second ? nullptr : alpha_base + a, second, alpha_base + a, nxt, part_out,
               n, sh);
}

__global__ void k_dot3_hist(const double *__restrict__ ys, const double *__restrict__ ss, int64_t n,
                            const LoopState *__restrict__ st, double *__restrict__ part) {
  __shared__ double sh[NT];
  const int64_t off = (int64_t)st->head * n;
  const double *x = ys + off, *y = ss + off;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT) {
    double xv = x[k], yv = y[k];
    a = __fma_rn(xv, yv, a);
    b = __fma_rn(xv, xv, b);
    c = __fma_rn(yv, yv, c);
  }
  a = block_sum<NT>(a, sh);
  b = block_sum<NT>(b, sh);
  c = block_sum<NT>(c, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = a;
    part[3 * blockIdx.x + 1] = b;
    part[3 * blockIdx.x + 2] = c;
  }
}

// z = 1 x + alpha y, y += alpha x, slot(head) of base = 1 x + (-1) y: the
// host path's k_lincomb / k_axpy arithmetic with the scalar read on the device
__global__ void k_lincomb_alpha(double *z, const double *x, const double *y, int64_t n,
                                const LoopState *__restrict__ st) {
  const double b = st->alpha;
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT)
    z[k] = __fma_rn(b, y[k], __dmul_rn(1.0, x[k]));
}
__global__ void k_axpy_alpha(double *__restrict__ y, const double *__restrict__ x, int64_t n,
                             const LoopState *__restrict__ st) {
  const double a = st->alpha;
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT)
    y[k] = __fma_rn(a, x[k], y[k]);
}
__global__ void k_hist_diff(double *base, const double *x, const double *y, int64_t n,
                            const LoopState *__restrict__ st) {
  double *z = base + (int64_t)st->head * n;
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT)
    z[k] = __fma_rn(-1.0, y[k], __dmul_rn(1.0, x[k]));
}

__global__ void k_count_free(const uint8_t *__restrict__ fixed, int64_t n, int *__restrict__ out) {
  int c = 0;
  for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n; k += (int64_t)gridDim.x * NT) c += fixed[k] == 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

int grid_for(const Scene &s) { return 2 * s.nsm; }
}  // namespace

int64_t count_free(Scene &s) {
  int64_t n = s.nn();
  if (n == 0) return 0;
  s.scan.total.ensure(1);
  HOT_CUDA(cudaMemsetAsync(s.scan.total.p, 0, sizeof(int), s.st));
  k_count_free<<<grid_for(s), NT, 0, s.st>>>(s.fixed.p, n, s.scan.total.p);
  HOT_LAUNCH("k_count_free");
  return read_scan_total(s.scan, s.st);
}

double dot(Scene &s, const double *x, const double *y, int64_t n) {
  double o[3];
  int G = grid_for(s);
  s.part.ensure(4096);
  k_dot3<<<G, NT, 0, s.st>>>(x, y, n, 0, s.part.p);
  HOT_LAUNCH("k_dot3");
  std::vector<double> h(3 * G);
  HOT_CUDA(cudaMemcpyAsync(h.data(), s.part.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  o[0] = 0.0;
  for (int b = 0; b < G; ++b) o[0] += h[3 * b];
  return o[0];
}

void dots3(Scene &s, const double *x, const double *y, int64_t n, double out[3]) {
  int G = grid_for(s);
  s.part.ensure(4096);
  k_dot3<<<G, NT, 0, s.st>>>(x, y, n, 1, s.part.p);
  HOT_LAUNCH("k_dot3");
  std::vector<double> h(3 * G);
  HOT_CUDA(cudaMemcpyAsync(h.data(), s.part.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  out[0] = out[1] = out[2] = 0.0;
  for (int b = 0; b < G; ++b) {
    out[0] += h[3 * b];
    out[1] += h[3 * b + 1];
    out[2] += h[3 * b + 2];
  }
}

void axpy(Scene &s, double *y, double a, const double *x, int64_t n) {
  k_axpy<<<grid_for(s), NT, 0, s.st>>>(y, a, x, n);
  HOT_LAUNCH("k_axpy");
}
void lincomb(Scene &s, double *z, double a, const double *x, double b, const double *y, int64_t n) {
  k_lincomb<<<grid_for(s), NT, 0, s.st>>>(z, a, x, b, y, n);
  HOT_LAUNCH("k_lincomb");
}
void scale_copy(Scene &s, double *dst, double a, const double *src, int64_t n) {
  k_lincomb<<<grid_for(s), NT, 0, s.st>>>(dst, a, src, 0.0, nullptr, n);
  HOT_LAUNCH("k_lincomb");
}

// history slot of the k-th newest pair (k = 0 newest)
static inline int hist_slot(const Scene &s, int k) {
  int w = s.opts.lbfgs_m;
  return ((s.hist_head - 1 - k) % w + w) % w;
}

void two_loop_first(Scene &s, double *q, int64_t n) {
  const int G = grid_for(s);
  const int m = s.hist_n;
  if (m == 0) return;
  s.part.ensure(4096);
  s.scal.ensure(64);
  double *pa = s.part.p, *pb = s.part.p + 2048;
  // partial of s_newest^T q
  int sl = hist_slot(s, 0);
  k_twoloop_step<<<G, NT, 0, s.st>>>(q, nullptr, nullptr, 0, 0.0, nullptr, 0, nullptr, s.hist_s.p + sl * n, pa, n);
  HOT_LAUNCH("k_twoloop_step");
  for (int k = 0; k < m; ++k) {
    int a = hist_slot(s, k);
    const double *nxt = (k + 1 < m) ? s.hist_s.p + hist_slot(s, k + 1) * n : nullptr;
    k_twoloop_step<<<G, NT, 0, s.st>>>(q, s.hist_y.p + a * n, pa, G, s.hist_rho[a], s.scal.p + a, 0, nullptr, nxt, pb,
                                       n);
    HOT_LAUNCH("k_twoloop_step");
    std::swap(pa, pb);
  }
}

void two_loop_second(Scene &s, double *r, int64_t n) {
  const int G = grid_for(s);
  const int m = s.hist_n;
  if (m == 0) return;
  double *pa = s.part.p, *pb = s.part.p + 2048;
  int sl = hist_slot(s, m - 1);
  k_twoloop_step<<<G, NT, 0, s.st>>>(r, nullptr, nullptr, 0, 0.0, nullptr, 1, nullptr, s.hist_y.p + sl * n, pa, n);
  HOT_LAUNCH("k_twoloop_step");
  for (int k = m - 1; k >= 0; --k) {
    int a = hist_slot(s, k);
    const double *nxt = (k - 1 >= 0) ? s.hist_y.p + hist_slot(s, k - 1) * n : nullptr;
    k_twoloop_step<<<G, NT, 0, s.st>>>(r, s.hist_s.p + a * n, pa, G, s.hist_rho[a], nullptr, 1, s.scal.p + a, nxt,
                                       pb, n);
    HOT_LAUNCH("k_twoloop_step");
    std::swap(pa, pb);
  }
}

void two_loop_first_dev(Scene &s, double *q, int64_t n, const LoopState *st) {
  const int G = grid_for(s), w = s.opts.lbfgs_m;
  double *pa = s.part.p, *pb = s.part.p + 2048;
  k_twoloop_dev<<<G, NT, 0, s.st>>>(q, nullptr, s.hist_s.p, n, w, st, -1, 0, nullptr, 0, pa, s.scal.p);
  HOT_LAUNCH("k_twoloop_dev");
  for (int j = 0; j < w; ++j) {
    k_twoloop_dev<<<G, NT, 0, s.st>>>(q, s.hist_y.p, s.hist_s.p, n, w, st, j, 0, pa, G, pb, s.scal.p);
    HOT_LAUNCH("k_twoloop_dev");
    std::swap(pa, pb);
  }
}

void two_loop_second_dev(Scene &s, double *r, int64_t n, const LoopState *st) {
  const int G = grid_for(s), w = s.opts.lbfgs_m;
  double *pa = s.part.p, *pb = s.part.p + 2048;
  k_twoloop_dev<<<G, NT, 0, s.st>>>(r, nullptr, s.hist_y.p, n, w, st, -1, 1, nullptr, 0, pa, s.scal.p);
  HOT_LAUNCH("k_twoloop_dev");
  for (int j = 0; j < w; ++j) {
    k_twoloop_dev<<<G, NT, 0, s.st>>>(r, s.hist_s.p, s.hist_y.p, n, w, st, j, 1, pa, G, pb, s.scal.p);
    HOT_LAUNCH("k_twoloop_dev");
    std::swap(pa, pb);
  }
}

int dot_launch(Scene &s, const double *x, const double *y, int64_t n, int mode, double *part) {
  const int G = grid_for(s);
  k_dot3<<<G, NT, 0, s.st>>>(x, y, n, mode, part);
  HOT_LAUNCH("k_dot3");
  return G;
}

int dots3_hist_launch(Scene &s, int64_t n, const LoopState *st, double *part) {
  const int G = grid_for(s);
  k_dot3_hist<<<G, NT, 0, s.st>>>(s.hist_y.p, s.hist_s.p, n, st, part);
  HOT_LAUNCH("k_dot3_hist");
  return G;
}

void lincomb_alpha(Scene &s, double *z, const double *x, const double *y, int64_t n, const LoopState *st) {
  k_lincomb_alpha<<<grid_for(s), NT, 0, s.st>>>(z, x, y, n, st);
  HOT_LAUNCH("k_lincomb_alpha");
}
void axpy_alpha(Scene &s, double *y, const double *x, int64_t n, const LoopState *st) {
  k_axpy_alpha<<<grid_for(s), NT, 0, s.st>>>(y, x, n, st);
  HOT_LAUNCH("k_axpy_alpha");
}
void hist_diff(Scene &s, double *base, const double *x, const double *y, int64_t n, const LoopState *st) {
  k_hist_diff<<<grid_for(s), NT, 0, s.st>>>(base, x, y, n, st);
  HOT_LAUNCH("k_hist_diff");
}

}  // namespace hot

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe: eight independent dependent chains per thread,
// enough resident warps per SM to hide the pipe latency.  Measures the rate
// that bounds the FP64 kernels (velocity gradient, gradient scatter, the
// FP64 Gauss-Seidel sweeps).
// ---------------------------------------------------------------------------
namespace hot {
__global__ void __launch_bounds__(256) k_fma_probe(double *__restrict__ out, int iters, double a, double b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 1e-3 * (double)(t & 1023) + 0.125 * j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[t] = s;
}
}  // namespace hot

extern "C" mpm_status mpm_probe_fp64_fma(void *cuda_stream, double *tflops) {
  using namespace hot;
  if (!tflops) return MPM_ERR_INVALID_ARG;
  *tflops = 0.0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MPM_ERR_CUDA;
  const int blocks = nsm * 8, threads = 256, iters = 4096;
  double *out = nullptr;
  try {
    out = static_cast<double *>(dev_alloc(sizeof(double) * blocks * threads, st));
  } catch (const Error &e) {
    return e.code;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  mpm_status status = MPM_OK;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, st);
    k_fma_probe<<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      status = MPM_ERR_CUDA;
      break;
    }
    note_launches(1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);   // the first launch is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dev_free(out, st);
  if (status == MPM_OK) *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return status;
}
