// Eq. 1 incremental potential: per-particle velocity gradients, energy,
// gradient (the nodal force of Sec. 4.1), projected per-particle stiffness
// and the cell-wise assembly of the fine-level 3x3-block Hessian.
#include "internal.h"

namespace hot {

namespace {
constexpr int NT = 256;

struct G {
  int dims[3], nb[3], nd[3];
  double dx, inv_dx, o[3];
};
G geo(const Scene &s) {
  G g;
  for (int k = 0; k < 3; ++k) {
    g.dims[k] = s.geo.dims[k];
    g.nb[k] = s.geo.nb[k];
    g.nd[k] = s.geo.dims[k] + 1;
    g.o[k] = s.geo.origin[k];
  }
  g.dx = s.geo.dx;
  g.inv_dx = s.geo.inv_dx;
  return g;
}

__device__ __forceinline__ int64_t nlin(int x, int y, int z, const int *nd) {
  return ((int64_t)z * nd[1] + y) * nd[0] + x;
}

// stencil of particle p: base node, per-axis weights and derivatives
__device__ __forceinline__ void stencil(const double *pd, int64_t np, int64_t p, const G &g, int b[3],
                                        double fx[3], double w[3][3], double dw[3][3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    b[k] = clampi(base_axis(pd[(PF_X + k) * np + p], g.o[k], g.inv_dx, &fx[k]), 0, g.dims[k] - 2);
    bspline_axis<double>(fx[k], g.inv_dx, w[k], dw[k]);
  }
}

// L_p = sum_i u_i grad w_ip^T (u2 added when present).  grad w_ip factors
// over the axes, (dw_x w_y w_z, w_x dw_y w_z, w_x w_y dw_z), so the stencil
// sum is taken one axis at a time (x, then y, then z): 270 FMA per particle
// instead of 405 for the node-by-node form (the FP64 pipe bounds this kernel).
__global__ void k_velgrad(const double *__restrict__ pd, int64_t np, G g, const int *__restrict__ map,
                          const double *__restrict__ u, const double *__restrict__ u2, double *__restrict__ L) {
  int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (p >= np) return;
  int b[3];
  double fx[3], w[3][3], dw[3][3];
  stencil(pd, np, p, g, b, fx, w, dw);
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // acc[3a + c] = L_ac
#pragma unroll
  for (int kz = 0; kz < 3; ++kz) {
    double tww[3] = {0, 0, 0}, twd[3] = {0, 0, 0}, tdw[3] = {0, 0, 0};
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      double sw[3] = {0, 0, 0}, sd[3] = {0, 0, 0};
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int idx = map[nlin(b[0] + kx, b[1] + ky, b[2] + kz, g.nd)];
        double ui[3] = {u[3 * idx], u[3 * idx + 1], u[3 * idx + 2]};
        if (u2) {
          ui[0] += u2[3 * idx];
          ui[1] += u2[3 * idx + 1];
          ui[2] += u2[3 * idx + 2];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          sw[a] = fma(ui[a], w[0][kx], sw[a]);
          sd[a] = fma(ui[a], dw[0][kx], sd[a]);
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        tww[a] = fma(sw[a], w[1][ky], tww[a]);
        twd[a] = fma(sw[a], dw[1][ky], twd[a]);
        tdw[a] = fma(sd[a], w[1][ky], tdw[a]);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[3 * a] = fma(tdw[a], w[2][kz], acc[3 * a]);
      acc[3 * a + 1] = fma(twd[a], w[2][kz], acc[3 * a + 1]);
      acc[3 * a + 2] = fma(tww[a], dw[2][kz], acc[3 * a + 2]);
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) L[k * np + p] = acc[k];
}

// F = (I + dt (Lv + alpha Lp)) F^n
__device__ __forceinline__ void deformed(const double *pd, int64_t np, int64_t p, const double *Lv,
                                         const double *Lp, double alpha, double dt, double F[9]) {
  double M[9], Fn[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    M[k] = Lv[k * np + p];
    if (Lp) M[k] += alpha * Lp[k * np + p];
    Fn[k] = pd[(PF_F + k) * np + p];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      F[3 * a + c] = Fn[3 * a + c] + dt * (M[3 * a] * Fn[c] + M[3 * a + 1] * Fn[3 + c] + M[3 * a + 2] * Fn[6 + c]);
}

// blocks [0, nbp): particle energies V_p psi(F_p); blocks [nbp, nbp+nbn): node
// terms 1/2 m |dv + a p|^2 - dt m g.(dv + a p).  One partial per block.
__global__ void k_energy(const double *__restrict__ pd, const int *__restrict__ pmat, const MatParams *__restrict__ mt,
                         int64_t np, const double *__restrict__ Lv, const double *__restrict__ Lp, double alpha,
                         const double *__restrict__ alpha_dev, double dt, int nbp, int64_t nn,
                         const double *__restrict__ m, const double *__restrict__ dv, const double *__restrict__ pdir,
                         double g0, double g1, double g2, double *__restrict__ part) {
  __shared__ double sh[NT];
  if (alpha_dev) alpha = *alpha_dev;   // step length held on the device (device-driven loop)
  double acc = 0.0;
  if ((int)blockIdx.x < nbp) {
    for (int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x; p < np; p += (int64_t)nbp * NT) {
      double F[9];
      deformed(pd, np, p, Lv, Lp, alpha, dt, F);
      const MatParams mp = mt[pmat[p]];
      acc += pd[PF_VOL * np + p] * psi_density<double>(F, mp.mu, mp.lam, mp.model);
    }
  } else {
    int nbn = gridDim.x - nbp;
    for (int64_t i = (int64_t)(blockIdx.x - nbp) * NT + threadIdx.x; i < nn; i += (int64_t)nbn * NT) {
      double d0 = dv[3 * i], d1 = dv[3 * i + 1], d2 = dv[3 * i + 2];
      if (pdir) {
        d0 += alpha * pdir[3 * i];
        d1 += alpha * pdir[3 * i + 1];
        d2 += alpha * pdir[3 * i + 2];
      }
      double mi = m[i];
      acc += 0.5 * mi * (d0 * d0 + d1 * d1 + d2 * d2) - dt * mi * (g0 * d0 + g1 * d1 + g2 * d2);
    }
  }
  double t = block_sum<NT>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Two-phase gradient.  The force on node i = b + (kx, ky, kz) of particle p
// is f_i = K_p grad w_ip with K_p = dt V_p P(F_p) F^n_p^T; by the axis
// factorization of grad w it is, per component a,
//   f_i[a] = A0[a][kx] P0[ky][kz] + A1[a][kx] P1[ky][kz] + A2[a][kx] P2[ky][kz]
// with A0 = K[a][0] dw_x, A1 = K[a][1] w_x, A2 = K[a][2] w_x and P0 = w_y w_z,
// P1 = dw_y w_z, P2 = w_y dw_z.  Phase 1, one thread per particle: the 27 A
// and 27 P values into scratch (SoA).  Phase 2, one warp per occupied cell:
// lane k < 27 owns stencil node k of the cell and sums f over the cell's
// particles in registers (9 FMA per particle), then adds to the grid once.
// No shared-memory atomics, full warps in both phases.
constexpr int GS_A = 0, GS_P = 27, GS_N = 54;
__global__ void k_grad_particles(const double *__restrict__ pd, const int *__restrict__ pmat,
                                 const MatParams *__restrict__ mt, int64_t np, const double *__restrict__ Lv,
                                 double dt, G g, double *__restrict__ scr) {
  int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (p >= np) return;
  int b[3];
  double fx[3], w[3][3], dw[3][3];
  stencil(pd, np, p, g, b, fx, w, dw);
#pragma unroll
  for (int ky = 0; ky < 3; ++ky)
#pragma unroll
    for (int kz = 0; kz < 3; ++kz) {
      scr[(GS_P + 3 * ky + kz) * np + p] = w[1][ky] * w[2][kz];
      scr[(GS_P + 9 + 3 * ky + kz) * np + p] = dw[1][ky] * w[2][kz];
      scr[(GS_P + 18 + 3 * ky + kz) * np + p] = w[1][ky] * dw[2][kz];
    }
  double F[9], P[9];
  deformed(pd, np, p, Lv, nullptr, 0.0, dt, F);
  const MatParams mp = mt[pmat[p]];
  piola<double>(F, mp.mu, mp.lam, mp.model, P);
  const double sc = dt * pd[PF_VOL * np + p];
  double K[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      K[3 * a + c] = sc * (P[3 * a] * pd[(PF_F + 3 * c) * np + p] + P[3 * a + 1] * pd[(PF_F + 3 * c + 1) * np + p] +
                           P[3 * a + 2] * pd[(PF_F + 3 * c + 2) * np + p]);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
      scr[(GS_A + 3 * a + kx) * np + p] = K[3 * a] * dw[0][kx];
      scr[(GS_A + 9 + 3 * a + kx) * np + p] = K[3 * a + 1] * w[0][kx];
      scr[(GS_A + 18 + 3 * a + kx) * np + p] = K[3 * a + 2] * w[0][kx];
    }
}

__global__ void k_grad_cells(const double *__restrict__ scr, int64_t np, const int *__restrict__ cell_first,
                             const int *__restrict__ cell_n, const int *__restrict__ cell_key, int64_t ncell, G g,
                             const int *__restrict__ map, double *__restrict__ gout) {
  const int64_t c = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= ncell || lane >= 27) return;
  const int kx = lane % 3, ky = (lane / 3) % 3, kz = lane / 9;
  const int yz = 3 * ky + kz;
  const int first = cell_first[c], cnt = cell_n[c];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int q = 0; q < cnt; ++q) {
    const int64_t p = first + q;
    const double p0 = scr[(GS_P + yz) * np + p], p1 = scr[(GS_P + 9 + yz) * np + p],
                 p2 = scr[(GS_P + 18 + yz) * np + p];
    a0 = fma(scr[(GS_A + kx) * np + p], p0, a0);
    a1 = fma(scr[(GS_A + 3 + kx) * np + p], p0, a1);
    a2 = fma(scr[(GS_A + 6 + kx) * np + p], p0, a2);
    a0 = fma(scr[(GS_A + 9 + kx) * np + p], p1, a0);
    a1 = fma(scr[(GS_A + 12 + kx) * np + p], p1, a1);
    a2 = fma(scr[(GS_A + 15 + kx) * np + p], p1, a2);
    a0 = fma(scr[(GS_A + 18 + kx) * np + p], p2, a0);
    a1 = fma(scr[(GS_A + 21 + kx) * np + p], p2, a1);
    a2 = fma(scr[(GS_A + 24 + kx) * np + p], p2, a2);
  }
  const unsigned key = (unsigned)cell_key[c];
  const unsigned B = key >> 6, l = key & 63u;
  const int x = (int)(B % g.nb[0]) * 4 + (l & 3) + kx;
  const int y = (int)((B / g.nb[0]) % g.nb[1]) * 4 + ((l >> 2) & 3) + ky;
  const int z = (int)(B / (g.nb[0] * g.nb[1])) * 4 + (l >> 4) + kz;
  const int idx = map[nlin(x, y, z, g.nd)];
  atomicAdd(gout + 3 * idx, a0);
  atomicAdd(gout + 3 * idx + 1, a1);
  atomicAdd(gout + 3 * idx + 2, a2);
}

// node terms m_i (dv_i - dt g), projection, and the two termination norms
__global__ void k_grad_nodes(int64_t nn, const double *__restrict__ m, const double *__restrict__ xi,
                             const uint8_t *__restrict__ fixed, const double *__restrict__ dv, double dt, double g0,
                             double g1, double g2, double cn_scale, double *__restrict__ gout,
                             double *__restrict__ part) {
  __shared__ double sh[NT];
  double a2 = 0.0, c2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < nn; i += (int64_t)gridDim.x * NT) {
    double r[3];
    if (fixed[i]) {
      r[0] = r[1] = r[2] = 0.0;
    } else {
      double mi = m[i];
      r[0] = gout[3 * i] + mi * (dv[3 * i] - dt * g0);
      r[1] = gout[3 * i + 1] + mi * (dv[3 * i + 1] - dt * g1);
      r[2] = gout[3 * i + 2] + mi * (dv[3 * i + 2] - dt * g2);
      double sq = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      a2 += sq;
      double den = cn_scale * xi[i];
      c2 += sq / (den * den);
    }
    gout[3 * i] = r[0];
    gout[3 * i + 1] = r[1];
    gout[3 * i + 2] = r[2];
  }
  double t = block_sum<NT>(a2, sh);
  double u = block_sum<NT>(c2, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t;
    part[2 * blockIdx.x + 1] = u;
  }
}

template <class T>
__global__ void k_stiffness(const double *__restrict__ pd, const int *__restrict__ pmat,
                            const MatParams *__restrict__ mt, int64_t np, const double *__restrict__ Lv, double dt,
                            T *__restrict__ A45) {
  int64_t p = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (p >= np) return;
  double Fd[9];
  deformed(pd, np, p, Lv, nullptr, 0.0, dt, Fd);
  T F[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) F[k] = (T)Fd[k];
  const MatParams mp = mt[pmat[p]];
  T A[45];
  projected_stiffness<T>(F, (T)mp.mu, (T)mp.lam, mp.model, A);
#pragma unroll
  for (int k = 0; k < 45; ++k) A45[k * np + p] = A[k];
}

// ---------------------------------------------------------------------------
// Fine Hessian: one CTA per occupied cell.  All particles of a cell share the
// same 27 stencil nodes, so each of the 378 node pairs (i <= l) is summed over
// the cell's particles in a register and added to the matrix once:
//   H_il += dt^2 V_p sum_{g,d} A_p[(a,g),(b,d)] d_ig d_ld,  d_i = F^n^T grad w_ip
// via B_i[a][b][d] = sum_g A_p[(a,g),(b,d)] d_ig (27 x 27 values per particle).
// ---------------------------------------------------------------------------
constexpr int HNT = 384;
constexpr int NPAIR = 378;

template <class T>
__global__ void __launch_bounds__(HNT) k_hessian_cells(const double *__restrict__ pd, int64_t np,
                                                      const T *__restrict__ A45, const int *__restrict__ cell_first,
                                                      const int *__restrict__ cell_n, const int *__restrict__ cell_key,
                                                      G g, double dt2, const int *__restrict__ map,
                                                      const int *__restrict__ row_ptr,
                                                      const int *__restrict__ slotpos, T *__restrict__ vals) {
  __shared__ T sA[81];
  __shared__ T sd[27 * 3];
  __shared__ T sB[27 * 27];
  __shared__ int snode[27];
  const int c = blockIdx.x;
  const int first = cell_first[c], cnt = cell_n[c];
  int cb[3];
  {
    unsigned key = (unsigned)cell_key[c];
    unsigned B = key >> 6, l = key & 63u;
    cb[0] = (int)(B % g.nb[0]) * 4 + (l & 3);
    cb[1] = (int)((B / g.nb[0]) % g.nb[1]) * 4 + ((l >> 2) & 3);
    cb[2] = (int)(B / (g.nb[0] * g.nb[1])) * 4 + (l >> 4);
  }
  if (threadIdx.x < 27) {
    int k = threadIdx.x;
    snode[k] = map[nlin(cb[0] + k % 3, cb[1] + (k / 3) % 3, cb[2] + k / 9, g.nd)];
  }
  // this thread's pair (i <= l) in stencil order
  int pi = 0, pl = 0;
  const bool has_pair = threadIdx.x < NPAIR;
  if (has_pair) {
    int t = threadIdx.x, i = 0;
    while (t >= 27 - i) {
      t -= 27 - i;
      ++i;
    }
    pi = i;
    pl = i + t;
  }
  T acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = T(0);
  for (int q = 0; q < cnt; ++q) {
    const int p = first + q;
    __syncthreads();
    if (threadIdx.x < 81) {
      int r = threadIdx.x / 9, cc = threadIdx.x % 9;
      const T sc = (T)(dt2 * pd[PF_VOL * np + p]);
      sA[threadIdx.x] = sc * A45[sym45(r, cc) * np + p];
    } else if (threadIdx.x >= 96 && threadIdx.x < 128) {
      // one warp: lanes 0-8 evaluate the weights of (axis lane/3, node lane%3)
      // and hold entry `lane` of F^n, then lanes 0-26 form node k's d = F^T grad w
      // from shuffles.  In T: the FP32 Hessian takes FP32 weights (the base
      // node stays exact in FP64).  FP64 instructions are scarce (2 FMA per
      // clock per SM), so no lane repeats another's axis.
      const int lane = threadIdx.x - 96;
      T wv = T(0), dwv = T(0), Fv = T(0);
      if (lane < 9) {
        const int a = lane / 3, kk = lane % 3;
        double fx;
        base_axis(pd[(PF_X + a) * np + p], g.o[a], g.inv_dx, &fx);
        T w[3], dw[3];
        bspline_axis<T>((T)fx, (T)g.inv_dx, w, dw);
        wv = kk == 0 ? w[0] : (kk == 1 ? w[1] : w[2]);
        dwv = kk == 0 ? dw[0] : (kk == 1 ? dw[1] : dw[2]);
        Fv = (T)pd[(PF_F + lane) * np + p];
      }
      const int k = lane < 27 ? lane : 0;
      const int kx = k % 3, ky = (k / 3) % 3, kz = k / 9;
      const T wx = __shfl_sync(0xffffffffu, wv, kx), dwx = __shfl_sync(0xffffffffu, dwv, kx);
      const T wy = __shfl_sync(0xffffffffu, wv, 3 + ky), dwy = __shfl_sync(0xffffffffu, dwv, 3 + ky);
      const T wz = __shfl_sync(0xffffffffu, wv, 6 + kz), dwz = __shfl_sync(0xffffffffu, dwv, 6 + kz);
      const T gw[3] = {dwx * wy * wz, wx * dwy * wz, wx * wy * dwz};
      T d[3];
#pragma unroll
      for (int b = 0; b < 3; ++b)     // d_a = sum_b F_ba gw_b, b in order
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T Fba = __shfl_sync(0xffffffffu, Fv, 3 * b + a);
          d[a] = b == 0 ? Fba * gw[0] : d[a] + Fba * gw[b];
        }
      if (lane < 27) {
#pragma unroll
        for (int a = 0; a < 3; ++a) sd[3 * k + a] = d[a];
      }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < 27 * 27; o += HNT) {
      int i = o / 27, abd = o % 27;
      int a = abd / 9, b = (abd / 3) % 3, d = abd % 3;
      sB[o] = sA[(3 * a) * 9 + 3 * b + d] * sd[3 * i] + sA[(3 * a + 1) * 9 + 3 * b + d] * sd[3 * i + 1] +
              sA[(3 * a + 2) * 9 + 3 * b + d] * sd[3 * i + 2];
    }
    __syncthreads();
    if (has_pair) {
      const T *Bi = sB + 27 * pi;
      const T dl0 = sd[3 * pl], dl1 = sd[3 * pl + 1], dl2 = sd[3 * pl + 2];
      // three FMA into the accumulator (a product summed apart, then added,
      // would cost a fourth FP64 instruction per entry)
#pragma unroll
      for (int ab = 0; ab < 9; ++ab)
        acc[ab] = fma(Bi[3 * ab + 2], dl2, fma(Bi[3 * ab + 1], dl1, fma(Bi[3 * ab], dl0, acc[ab])));
    }
  }
  __syncthreads();
  if (!has_pair) return;
  const int ri = snode[pi], rl = snode[pl];
  const int s = (pl % 3 - pi % 3 + 2) + 5 * ((pl / 3) % 3 - (pi / 3) % 3 + 2) + 25 * (pl / 9 - pi / 9 + 2);
  {
    int rp = row_ptr[ri], nb = row_ptr[ri + 1] - rp;
    int pos = slotpos[(int64_t)ri * NSLOT + s] - rp;
    T *base = vals + 9 * (int64_t)rp + pos;
#pragma unroll
    for (int e = 0; e < 9; ++e) atomicAdd(base + e * nb, acc[e]);
  }
  // the transposed block (rl, ri) is filled by k_hessian_mirror
}

// Lower half from the upper: a cell adds pair (i, l) of its stencil only for
// stencil index i <= l, i.e. for block offsets o = l - i with
// o_x + 3 o_y + 9 o_z >= 0 (the same sign in every cell), so the blocks with
// a negative index offset get the transpose of their mirror.  One warp per
// row; only reads of finished blocks, no atomics.
template <class T>
__global__ void k_hessian_mirror(int64_t nn, const int *__restrict__ row_ptr, const int *__restrict__ cols,
                                 const int *__restrict__ slotpos, T *vals) {
  const int64_t i = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  if (i >= nn) return;
  const int lane = threadIdx.x & 31;
  const int rp = row_ptr[i], nb = row_ptr[i + 1] - rp;
  for (int s = lane; s < NSLOT; s += 32) {
    const int o[3] = {s % 5 - 2, (s / 5) % 5 - 2, s / 25 - 2};
    if (o[0] + 3 * o[1] + 9 * o[2] >= 0) continue;
    const int pos = slotpos[i * NSLOT + s];
    if (pos < 0) continue;
    const int j = cols[pos];
    const int rpj = row_ptr[j], nbj = row_ptr[j + 1] - rpj;
    const int posj = slotpos[(int64_t)j * NSLOT + (NSLOT - 1 - s)] - rpj;
    const T *src = vals + 9 * (int64_t)rpj + posj;
    T *dst = vals + 9 * (int64_t)rp + (pos - rp);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) dst[(3 * a + b) * nb] = src[(3 * b + a) * nbj];
  }
}

// mass term and Dirichlet projection: held rows/columns zeroed, held
// diagonal m_i I (I when m_i = 0), free diagonal + m_i I.  One warp per row.
template <class T>
__global__ void k_hessian_finish(int64_t nn, const int *__restrict__ row_ptr, const int *__restrict__ cols,
                                 const uint8_t *__restrict__ fixed, const double *__restrict__ m,
                                 T *__restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (i >= nn) return;
  int rp = row_ptr[i], nb = row_ptr[i + 1] - rp;
  bool fi = fixed[i];
  T *base = vals + 9 * (int64_t)rp;
  for (int b = lane; b < nb; b += 32) {
    int j = cols[rp + b];
    if (fi || fixed[j]) {
#pragma unroll
      for (int e = 0; e < 9; ++e) base[e * nb + b] = T(0);
    }
    if (j == i) {
      double mi = m[i];
      T d = fi ? (T)(mi > 0.0 ? mi : 1.0) : (T)mi;
      base[0 * nb + b] += d;
      base[4 * nb + b] += d;
      base[8 * nb + b] += d;
    }
  }
}
}  // namespace

void velocity_gradient(Scene &s, const double *u, const double *u2, double *L) {
  if (s.np == 0) return;
  ProfScope prof_(s, "velgrad");
  k_velgrad<<<(unsigned)((s.np + NT - 1) / NT), NT, 0, s.st>>>(s.pd.p, s.np, geo(s), s.topo[0].map.p, u, u2, L);
  HOT_LAUNCH("k_velgrad");
}

int energy_launch(Scene &s, const double *L1, const double *L2, double alpha, const double *alpha_dev,
                  const double *dvv, const double *pv) {
  const int nbp = 2 * s.nsm, nbn = s.nsm;
  s.part.ensure(4096);
  ProfScope prof_(s, "energy");
  k_energy<<<nbp + nbn, NT, 0, s.st>>>(s.pd.p, s.pmat.p, s.mat_table.p, s.np, L1, L2, alpha, alpha_dev, s.dt, nbp,
                                       s.nn(), s.m.p, dvv, pv, s.gravity[0], s.gravity[1], s.gravity[2], s.part.p);
  HOT_LAUNCH("k_energy");
  return nbp + nbn;
}

double energy(Scene &s, const double *L1, const double *L2, double alpha, const double *dvv, const double *pv) {
  if (alpha == 0.0) {
    L2 = nullptr;
    pv = nullptr;
  }
  const int np = energy_launch(s, L1, L2, alpha, nullptr, dvv, pv);
  std::vector<double> h(np);
  HOT_CUDA(cudaMemcpyAsync(h.data(), s.part.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  double e = 0.0;
  for (double x : h) e += x;   // fixed order (the device-driven loop sums in the same order)
  return e;
}

int gradient_launch(Scene &s, const double *Lcur, const double *dvec, double *gout) {
  const int64_t nn = s.nn();
  HOT_CUDA(cudaMemsetAsync(gout, 0, sizeof(double) * 3 * nn, s.st));
  if (s.n_cells > 0) {
    s.gscr.ensure((size_t)GS_N * s.np, 1.0);
    ProfScope prof_(s, "grad_scatter");
    k_grad_particles<<<(unsigned)((s.np + NT - 1) / NT), NT, 0, s.st>>>(s.pd.p, s.pmat.p, s.mat_table.p, s.np,
                                                                        Lcur, s.dt, geo(s), s.gscr.p);
    HOT_LAUNCH("k_grad_particles");
    k_grad_cells<<<(unsigned)((s.n_cells + NT / 32 - 1) / (NT / 32)), NT, 0, s.st>>>(
        s.gscr.p, s.np, s.cell_first.p, s.cell_n.p, s.cell_key.p, s.n_cells, geo(s), s.topo[0].map.p, gout);
    HOT_LAUNCH("k_grad_cells");
  }
  const int nb = s.nsm;
  s.part.ensure(4096);
  double cn_scale = 24.0 * s.geo.dx * s.geo.dx * s.dt;
  k_grad_nodes<<<nb, NT, 0, s.st>>>(nn, s.m.p, s.xi.p, s.fixed.p, dvec, s.dt, s.gravity[0], s.gravity[1],
                                    s.gravity[2], cn_scale, gout, s.part.p);
  HOT_LAUNCH("k_grad_nodes");
  return nb;
}

void gradient(Scene &s, const double *Lcur, const double *dvec, double *gout, double norms[2]) {
  const int nb = gradient_launch(s, Lcur, dvec, gout);
  std::vector<double> h(2 * nb);
  HOT_CUDA(cudaMemcpyAsync(h.data(), s.part.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  norms[0] = norms[1] = 0.0;
  for (int b = 0; b < nb; ++b) {   // fixed order (the device-driven loop sums in the same order)
    norms[0] += h[2 * b];
    norms[1] += h[2 * b + 1];
  }
}

template <class T>
void particle_stiffness(Scene &s, Hier<T> &h) {
  h.A45.ensure((size_t)45 * s.np, 1.0);
  if (s.np == 0) return;
  ProfScope prof_(s, "stiffness");
  k_stiffness<T><<<(unsigned)((s.np + 127) / 128), 128, 0, s.st>>>(s.pd.p, s.pmat.p, s.mat_table.p, s.np, s.Lv.p,
                                                                  s.dt, h.A45.p);
  HOT_LAUNCH("k_stiffness");
}

template <class T>
void hessian_assemble(Scene &s, Hier<T> &h) {
  Topo &t = s.topo[0];
  Vals<T> &L = h.L[0];
  L.vals.ensure(9 * (size_t)t.nnzb);
  HOT_CUDA(cudaMemsetAsync(L.vals.p, 0, sizeof(T) * 9 * t.nnzb, s.st));
  if (s.n_cells > 0) {
    ProfScope prof_(s, "hessian_cells");
    k_hessian_cells<T><<<(unsigned)s.n_cells, HNT, 0, s.st>>>(s.pd.p, s.np, h.A45.p, s.cell_first.p, s.cell_n.p,
                                                             s.cell_key.p, geo(s), s.dt * s.dt, t.map.p, t.row_ptr.p,
                                                             t.slotpos.p, L.vals.p);
    HOT_LAUNCH("k_hessian_cells");
  }
  if (t.n > 0) {
    k_hessian_mirror<T><<<(unsigned)((t.n + NT / 32 - 1) / (NT / 32)), NT, 0, s.st>>>(t.n, t.row_ptr.p, t.cols.p,
                                                                                     t.slotpos.p, L.vals.p);
    HOT_LAUNCH("k_hessian_mirror");
    k_hessian_finish<T><<<(unsigned)((t.n + NT / 32 - 1) / (NT / 32)), NT, 0, s.st>>>(t.n, t.row_ptr.p, t.cols.p,
                                                                                     s.fixed.p, s.m.p, L.vals.p);
    HOT_LAUNCH("k_hessian_finish");
  }
}

template void particle_stiffness<double>(Scene &, Hier<double> &);
template void particle_stiffness<float>(Scene &, Hier<float> &);
template void hessian_assemble<double>(Scene &, Hier<double> &);
template void hessian_assemble<float>(Scene &, Hier<float> &);

}  // namespace hot
