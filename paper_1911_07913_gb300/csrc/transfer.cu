// Particle binning (bit-exact cell keys, deterministic stable counting sort),
// active-node construction, APIC P2G and G2P (Sec. 3.1, Jiang et al. 2015).
#include "internal.h"

namespace hot {

namespace {
constexpr int NT = 256;

__device__ __forceinline__ unsigned cell_key_of(int bx, int by, int bz, const int *nb) {
  unsigned B = ((unsigned)(bz >> 2) * (unsigned)nb[1] + (unsigned)(by >> 2)) * (unsigned)nb[0] + (unsigned)(bx >> 2);
  return B * 64u + (unsigned)(((bz & 3) << 4) | ((by & 3) << 2) | (bx & 3));
}
__device__ __forceinline__ void cell_of_key(unsigned key, const int *nb, int *c) {
  unsigned B = key >> 6, l = key & 63u;
  int Bx = B % nb[0], By = (B / nb[0]) % nb[1], Bz = B / (nb[0] * nb[1]);
  c[0] = Bx * 4 + (l & 3);
  c[1] = By * 4 + ((l >> 2) & 3);
  c[2] = Bz * 4 + (l >> 4);
}

struct GeoArgs {
  int dims[3];
  int nb[3];
  int ndims[3];     // node map extent = dims + 1
  double dx, inv_dx;
  double o[3];
};

GeoArgs geo_args(const Scene &s) {
  GeoArgs g;
  for (int k = 0; k < 3; ++k) {
    g.dims[k] = s.geo.dims[k];
    g.nb[k] = s.geo.nb[k];
    g.ndims[k] = s.geo.dims[k] + 1;
    g.o[k] = s.geo.origin[k];
  }
  g.dx = s.geo.dx;
  g.inv_dx = s.geo.inv_dx;
  return g;
}

__device__ __forceinline__ int64_t node_lin(int x, int y, int z, const int *nd) {
  return ((int64_t)z * nd[1] + y) * nd[0] + x;
}

__global__ void k_keys(const double *__restrict__ pd, int64_t np, GeoArgs g, unsigned *__restrict__ key,
                       int *__restrict__ slot, int *__restrict__ cell_count, int *__restrict__ err) {
  int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (p >= np) return;
  int b[3];
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double fx;
    b[k] = base_axis(pd[(PF_X + k) * np + p], g.o[k], g.inv_dx, &fx);
    if (b[k] < 0 || b[k] + 2 > g.dims[k] || !(fx == fx)) {
      bad = true;
      b[k] = b[k] < 0 ? 0 : (b[k] + 2 > g.dims[k] ? g.dims[k] - 2 : b[k]);
      if (b[k] < 0) b[k] = 0;
    }
  }
  if (bad) atomicOr(err, DEV_ERR_DOMAIN);
  unsigned kk = cell_key_of(b[0], b[1], b[2], g.nb);
  key[p] = kk;
  slot[p] = atomicAdd(&cell_count[kk], 1);
}

__global__ void k_place(const unsigned *__restrict__ key, const int *__restrict__ slot, const int *__restrict__ cell_start,
                        int64_t np, int *__restrict__ tmp) {
  int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (p >= np) return;
  tmp[cell_start[key[p]] + slot[p]] = (int)p;
}

// rank each particle inside its cell by its previous index: a stable order
__global__ void k_stable_rank(const int *__restrict__ tmp, const unsigned *__restrict__ key,
                              const int *__restrict__ cell_start, const int *__restrict__ cell_count, int64_t np,
                              int *__restrict__ perm, int *__restrict__ skey) {
  int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (q >= np) return;
  int src = tmp[q];
  unsigned k = key[src];
  int st = cell_start[k], cnt = cell_count[k];
  int rank = 0;
  for (int j = st; j < st + cnt; ++j) rank += tmp[j] < src;
  perm[st + rank] = src;
  skey[st + rank] = (int)k;
}

__global__ void k_gather(const double *__restrict__ pd, const int *__restrict__ pmat, const int *__restrict__ pid,
                         const int *__restrict__ perm, int64_t np, double *__restrict__ pd2, int *__restrict__ pmat2,
                         int *__restrict__ pid2) {
  int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (q >= np) return;
  int src = perm[q];
#pragma unroll 2
  for (int f = 0; f < PF_COUNT; ++f) pd2[f * np + q] = pd[f * np + src];
  pmat2[q] = pmat[src];
  pid2[q] = pid[src];
}

// segment heads: cells (shift 0) or 4^3-cell blocks (shift 6)
__global__ void k_heads(const int *__restrict__ skey, int64_t np, int shift, int *__restrict__ flag) {
  int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (q >= np) return;
  flag[q] = (q == 0) || ((skey[q] >> shift) != (skey[q - 1] >> shift));
}

__global__ void k_emit_segments(const int *__restrict__ skey, const int *__restrict__ flag, const int *__restrict__ idx,
                                int64_t np, int shift, int *__restrict__ first, int *__restrict__ segkey) {
  int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (q >= np || !flag[q]) return;
  int c = idx[q];
  first[c] = (int)q;
  segkey[c] = skey[q] >> shift;
}

__global__ void k_segment_ends(const int *__restrict__ first, int64_t nseg, int64_t np, int *__restrict__ out_n,
                               int as_count) {
  int64_t c = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (c >= nseg) return;
  int e = (c + 1 < nseg) ? first[c + 1] : (int)np;
  out_n[c] = as_count ? e - first[c] : e;
}

__global__ void k_mark_nodes(const int *__restrict__ cell_key, int64_t ncell, GeoArgs g, uint8_t *__restrict__ flag) {
  int64_t c = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (c >= ncell || lane >= 27) return;
  int b[3];
  cell_of_key((unsigned)cell_key[c], g.nb, b);
  int x = b[0] + lane % 3, y = b[1] + (lane / 3) % 3, z = b[2] + lane / 9;
  flag[node_lin(x, y, z, g.ndims)] = 1;
}

}  // namespace

// dense flags -> compact map and coordinates (shared by every level)
__global__ void k_finalize_map(const uint8_t *__restrict__ flag, int *map, int64_t ntot, int nx, int ny,
                               int *__restrict__ coords) {
  int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (k >= ntot) return;
  if (flag[k]) {
    int idx = map[k];
    int x = (int)(k % nx), y = (int)((k / nx) % ny), z = (int)(k / ((int64_t)nx * ny));
    coords[3 * idx] = x;
    coords[3 * idx + 1] = y;
    coords[3 * idx + 2] = z;
  } else {
    map[k] = -1;
  }
}

void compact_dense(Scene &s, Topo &T) {
  int64_t ntot = (int64_t)T.dims[0] * T.dims[1] * T.dims[2];
  exclusive_scan_u8(T.flag.p, T.map.p, ntot, s.scan, s.st);
  int n = read_scan_total(s.scan, s.st);
  T.n = n;
  T.coords.ensure(3 * (size_t)n + 3);
  k_finalize_map<<<(unsigned)((ntot + NT - 1) / NT), NT, 0, s.st>>>(T.flag.p, T.map.p, ntot, T.dims[0], T.dims[1],
                                                                    T.coords.p);
  HOT_LAUNCH("k_finalize_map");
}

void bin_and_sort(Scene &s) {
  const int64_t np = s.np;
  GeoArgs g = geo_args(s);
  s.key.ensure(np);
  s.slot.ensure(np);
  s.perm.ensure(np);
  s.tmp.ensure(np);
  s.cell_count.ensure(s.ncell_dense);
  s.cell_start.ensure(s.ncell_dense);
  HOT_CUDA(cudaMemsetAsync(s.cell_count.p, 0, sizeof(int) * s.ncell_dense, s.st));
  unsigned nbk = (unsigned)((np + NT - 1) / NT);
  k_keys<<<nbk, NT, 0, s.st>>>(s.pd.p, np, g, s.key.p, s.slot.p, s.cell_count.p, s.errflag.p);
  HOT_LAUNCH("k_keys");
  exclusive_scan(s.cell_count.p, s.cell_start.p, s.ncell_dense, s.scan, s.st);
  k_place<<<nbk, NT, 0, s.st>>>(s.key.p, s.slot.p, s.cell_start.p, np, s.tmp.p);
  HOT_LAUNCH("k_place");
  // sorted keys go to `slot` (free after k_place)
  k_stable_rank<<<nbk, NT, 0, s.st>>>(s.tmp.p, s.key.p, s.cell_start.p, s.cell_count.p, np, s.perm.p, s.slot.p);
  HOT_LAUNCH("k_stable_rank");
  s.pd_alt.ensure((size_t)PF_COUNT * np, 1.0);
  s.pmat_alt.ensure(np, 1.0);
  s.pid_alt.ensure(np, 1.0);
  k_gather<<<nbk, NT, 0, s.st>>>(s.pd.p, s.pmat.p, s.pid.p, s.perm.p, np, s.pd_alt.p, s.pmat_alt.p, s.pid_alt.p);
  HOT_LAUNCH("k_gather");
  std::swap(s.pd, s.pd_alt);
  std::swap(s.pmat, s.pmat_alt);
  std::swap(s.pid, s.pid_alt);

  // occupied cells and blocks
  s.flags.ensure(np);
  s.flag_scan.ensure(np);
  for (int pass = 0; pass < 2; ++pass) {
    int shift = pass == 0 ? 0 : 6;
    k_heads<<<nbk, NT, 0, s.st>>>(s.slot.p, np, shift, s.flags.p);
    HOT_LAUNCH("k_heads");
    exclusive_scan(s.flags.p, s.flag_scan.p, np, s.scan, s.st);
    int nseg = read_scan_total(s.scan, s.st);
    DBuf<int> &first = pass == 0 ? s.cell_first : s.blk_first;
    DBuf<int> &skey = pass == 0 ? s.cell_key : s.blk_key;
    DBuf<int> &cnt = pass == 0 ? s.cell_n : s.blk_end;
    first.ensure(nseg);
    skey.ensure(nseg);
    cnt.ensure(nseg);
    k_emit_segments<<<nbk, NT, 0, s.st>>>(s.slot.p, s.flags.p, s.flag_scan.p, np, shift, first.p, skey.p);
    HOT_LAUNCH("k_emit_segments");
    k_segment_ends<<<(unsigned)((nseg + NT - 1) / NT), NT, 0, s.st>>>(first.p, nseg, np, cnt.p, pass == 0);
    HOT_LAUNCH("k_segment_ends");
    if (pass == 0) s.n_cells = nseg;
    else s.n_blocks = nseg;
  }
}

void build_level0_nodes(Scene &s) {
  GeoArgs g = geo_args(s);
  Topo &T = s.topo[0];
  for (int k = 0; k < 3; ++k) T.dims[k] = s.geo.dims[k] + 1;
  int64_t ntot = (int64_t)T.dims[0] * T.dims[1] * T.dims[2];
  T.flag.ensure(ntot, 1.0);
  T.map.ensure(ntot, 1.0);
  HOT_CUDA(cudaMemsetAsync(T.flag.p, 0, ntot, s.st));
  unsigned nbc = (unsigned)((s.n_cells + NT / 32 - 1) / (NT / 32));
  if (s.n_cells > 0) {
    k_mark_nodes<<<nbc, NT, 0, s.st>>>(s.cell_key.p, s.n_cells, g, T.flag.p);
    HOT_LAUNCH("k_mark_nodes");
  }
  compact_dense(s, T);
}

// ---------------------------------------------------------------------------
// P2G: one CTA per occupied 4^3-cell block; its 6^3 node neighbourhood is
// accumulated in shared memory, then added to the grid with one atomic per
// touched node and component.
// ---------------------------------------------------------------------------
namespace {
constexpr int NB6 = 216;

__global__ void __launch_bounds__(NT) k_p2g(const double *__restrict__ pd, const int *__restrict__ pmat,
                                            const MatParams *__restrict__ mt, int64_t np,
                                            const int *__restrict__ blk_first, const int *__restrict__ blk_end,
                                            const int *__restrict__ blk_key, GeoArgs g, const int *__restrict__ map,
                                            double *__restrict__ m, double *__restrict__ mv,
                                            double *__restrict__ mxi) {
  __shared__ double acc[NB6 * 5];
  for (int i = threadIdx.x; i < NB6 * 5; i += NT) acc[i] = 0.0;
  __syncthreads();
  const int blk = blockIdx.x;
  const int key = blk_key[blk];
  const int Bx = key % g.nb[0], By = (key / g.nb[0]) % g.nb[1], Bz = key / (g.nb[0] * g.nb[1]);
  const int o0 = Bx * 4, o1 = By * 4, o2 = Bz * 4;
  const int pe = blk_end[blk];
  for (int p = blk_first[blk] + threadIdx.x; p < pe; p += NT) {
    double fx[3], w[3][3], dw[3][3];
    int b[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      b[k] = base_axis(pd[(PF_X + k) * np + p], g.o[k], g.inv_dx, &fx[k]);
      bspline_axis<double>(fx[k], g.inv_dx, w[k], dw[k]);
    }
    const double mp = pd[PF_MASS * np + p];
    const double xip = mt[pmat[p]].xi;
    double vp[3], C[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) vp[k] = pd[(PF_V + k) * np + p];
#pragma unroll
    for (int k = 0; k < 9; ++k) C[k] = pd[(PF_C + k) * np + p];
    const int l0 = b[0] - o0, l1 = b[1] - o1, l2 = b[2] - o2;
#pragma unroll
    for (int kz = 0; kz < 3; ++kz)
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const double wm = w[0][kx] * w[1][ky] * w[2][kz] * mp;
          const double r0 = (kx - fx[0]) * g.dx, r1 = (ky - fx[1]) * g.dx, r2 = (kz - fx[2]) * g.dx;
          const int li = ((l2 + kz) * 6 + (l1 + ky)) * 6 + (l0 + kx);
          double *a = acc + li * 5;
          atomicAdd(a, wm);
          atomicAdd(a + 1, wm * (vp[0] + C[0] * r0 + C[1] * r1 + C[2] * r2));
          atomicAdd(a + 2, wm * (vp[1] + C[3] * r0 + C[4] * r1 + C[5] * r2));
          atomicAdd(a + 3, wm * (vp[2] + C[6] * r0 + C[7] * r1 + C[8] * r2));
          atomicAdd(a + 4, wm * xip);
        }
  }
  __syncthreads();
  for (int li = threadIdx.x; li < NB6; li += NT) {
    const double *a = acc + li * 5;
    if (a[0] == 0.0) continue;
    int x = o0 + li % 6, y = o1 + (li / 6) % 6, z = o2 + li / 36;
    if (x >= g.ndims[0] || y >= g.ndims[1] || z >= g.ndims[2]) continue;
    int idx = map[node_lin(x, y, z, g.ndims)];
    if (idx < 0) continue;
    atomicAdd(m + idx, a[0]);
    atomicAdd(mv + 3 * idx, a[1]);
    atomicAdd(mv + 3 * idx + 1, a[2]);
    atomicAdd(mv + 3 * idx + 2, a[3]);
    atomicAdd(mxi + idx, a[4]);
  }
}

// v_i = (m v)_i / m_i, xi_i = (m xi)_i / m_i, Dirichlet nodes (walls within
// three cells, then the boxes in order, then zero-mass nodes)
__global__ void k_grid_finalize(int64_t n, const int *__restrict__ coords, GeoArgs g, const mpm_bc *__restrict__ bcs,
                                int nbc, double *__restrict__ m, const double *__restrict__ mv,
                                const double *__restrict__ mxi, double *__restrict__ v, double *__restrict__ xi,
                                uint8_t *__restrict__ fixed) {
  int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (i >= n) return;
  int c[3] = {coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]};
  double pos[3];
  bool fx = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    pos[k] = __dadd_rn(g.o[k], __dmul_rn((double)c[k], g.dx));
    if (c[k] < 3 || c[k] > g.dims[k] - 3) fx = true;
  }
  double vf[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < nbc; ++b) {
    const mpm_bc &bc = bcs[b];
    bool in = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) in = in && pos[k] >= bc.lo[k] && pos[k] <= bc.hi[k];
    if (in && bc.radius > 0.0) {
      // distance from the rotation axis, each operation rounded separately
      double r0 = __dadd_rn(pos[0], -bc.center[0]), r1 = __dadd_rn(pos[1], -bc.center[1]);
      double r2 = __dadd_rn(pos[2], -bc.center[2]);
      double t = __dadd_rn(__dadd_rn(__dmul_rn(r0, bc.axis[0]), __dmul_rn(r1, bc.axis[1])), __dmul_rn(r2, bc.axis[2]));
      double q0 = __dadd_rn(r0, -__dmul_rn(t, bc.axis[0])), q1 = __dadd_rn(r1, -__dmul_rn(t, bc.axis[1]));
      double q2 = __dadd_rn(r2, -__dmul_rn(t, bc.axis[2]));
      double d2 = __dadd_rn(__dadd_rn(__dmul_rn(q0, q0), __dmul_rn(q1, q1)), __dmul_rn(q2, q2));
      in = d2 <= __dmul_rn(bc.radius, bc.radius);
    }
    if (!in) continue;
    fx = true;
    if (bc.type == 0) {
      vf[0] = vf[1] = vf[2] = 0.0;
    } else {
      double w0 = bc.omega * bc.axis[0], w1 = bc.omega * bc.axis[1], w2 = bc.omega * bc.axis[2];
      double r0 = pos[0] - bc.center[0], r1 = pos[1] - bc.center[1], r2 = pos[2] - bc.center[2];
      vf[0] = w1 * r2 - w2 * r1;
      vf[1] = w2 * r0 - w0 * r2;
      vf[2] = w0 * r1 - w1 * r0;
    }
  }
  double mi = m[i];
  if (!(mi > 0.0)) fx = true;
  fixed[i] = fx ? 1 : 0;
  xi[i] = mi > 0.0 ? mxi[i] / mi : 0.0;
  if (fx) {
    v[3 * i] = vf[0];
    v[3 * i + 1] = vf[1];
    v[3 * i + 2] = vf[2];
  } else {
    v[3 * i] = mv[3 * i] / mi;
    v[3 * i + 1] = mv[3 * i + 1] / mi;
    v[3 * i + 2] = mv[3 * i + 2] / mi;
  }
}

__global__ void k_speed_max(const double *__restrict__ pd, int64_t np, double *__restrict__ part) {
  __shared__ double sh[NT];
  double mx = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x; p < np; p += (int64_t)gridDim.x * NT) {
    double a = pd[PF_V * np + p], b = pd[(PF_V + 1) * np + p], c = pd[(PF_V + 2) * np + p];
    double s2 = a * a + b * b + c * c;
    mx = s2 > mx ? s2 : mx;
  }
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_g2p(double *__restrict__ pd, const int *__restrict__ pmat, const MatParams *__restrict__ mt,
                      int64_t np, GeoArgs g, const int *__restrict__ map, const double *__restrict__ vn,
                      double dt) {
  int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (p >= np) return;
  double fx[3], w[3][3], dw[3][3];
  int b[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    b[k] = clampi(base_axis(pd[(PF_X + k) * np + p], g.o[k], g.inv_dx, &fx[k]), 0, g.dims[k] - 2);
    bspline_axis<double>(fx[k], g.inv_dx, w[k], dw[k]);
  }
  double vp[3] = {0, 0, 0}, B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, L[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int kz = 0; kz < 3; ++kz)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        int idx = map[node_lin(b[0] + kx, b[1] + ky, b[2] + kz, g.ndims)];
        double vi[3] = {vn[3 * idx], vn[3 * idx + 1], vn[3 * idx + 2]};
        double wgt = w[0][kx] * w[1][ky] * w[2][kz];
        double gw[3] = {dw[0][kx] * w[1][ky] * w[2][kz], w[0][kx] * dw[1][ky] * w[2][kz],
                        w[0][kx] * w[1][ky] * dw[2][kz]};
        double r[3] = {(kx - fx[0]) * g.dx, (ky - fx[1]) * g.dx, (kz - fx[2]) * g.dx};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          vp[a] += wgt * vi[a];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            B[3 * a + c] += wgt * vi[a] * r[c];
            L[3 * a + c] += vi[a] * gw[c];
          }
        }
      }
  double F[9], Fn[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) F[k] = pd[(PF_F + k) * np + p];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      Fn[3 * a + c] = F[3 * a + c] + dt * (L[3 * a] * F[c] + L[3 * a + 1] * F[3 + c] + L[3 * a + 2] * F[6 + c]);
  const MatParams mp = mt[pmat[p]];
  plastic_project(Fn, mp.mu, mp.yield, mp.plastic);
  const double Dinv = 4.0 * g.inv_dx * g.inv_dx;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    pd[(PF_F + k) * np + p] = Fn[k];
    pd[(PF_C + k) * np + p] = Dinv * B[k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    pd[(PF_V + k) * np + p] = vp[k];
    pd[(PF_X + k) * np + p] += dt * vp[k];
  }
}

// user AoS <-> library SoA in the caller's order
__global__ void k_soa_to_user(const double *__restrict__ pd, const int *__restrict__ pid, int64_t np,
                              double *__restrict__ x, double *__restrict__ v, double *__restrict__ F,
                              double *__restrict__ C) {
  int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (q >= np) return;
  int64_t o = pid[q];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    x[3 * o + k] = pd[(PF_X + k) * np + q];
    v[3 * o + k] = pd[(PF_V + k) * np + q];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    F[9 * o + k] = pd[(PF_F + k) * np + q];
    C[9 * o + k] = pd[(PF_C + k) * np + q];
  }
}

__global__ void k_user_to_soa(double *__restrict__ pd, const int *__restrict__ pid, int64_t np,
                              const double *__restrict__ x, const double *__restrict__ v,
                              const double *__restrict__ F, const double *__restrict__ C, int mask) {
  int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (q >= np) return;
  int64_t o = pid[q];
  if (mask & 1)
#pragma unroll
    for (int k = 0; k < 3; ++k) pd[(PF_X + k) * np + q] = x[3 * o + k];
  if (mask & 2)
#pragma unroll
    for (int k = 0; k < 3; ++k) pd[(PF_V + k) * np + q] = v[3 * o + k];
  if (mask & 4)
#pragma unroll
    for (int k = 0; k < 9; ++k) pd[(PF_F + k) * np + q] = F[9 * o + k];
  if (mask & 8)
#pragma unroll
    for (int k = 0; k < 9; ++k) pd[(PF_C + k) * np + q] = C[9 * o + k];
}
}  // namespace

void p2g_transfer(Scene &s) {
  GeoArgs g = geo_args(s);
  const int64_t n = s.topo[0].n;
  s.m.ensure(n);
  s.v.ensure(3 * n);
  s.xi.ensure(n);
  s.mv.ensure(3 * n);
  s.mxi.ensure(n);
  s.fixed.ensure(n);
  HOT_CUDA(cudaMemsetAsync(s.m.p, 0, sizeof(double) * n, s.st));
  HOT_CUDA(cudaMemsetAsync(s.mv.p, 0, sizeof(double) * 3 * n, s.st));
  HOT_CUDA(cudaMemsetAsync(s.mxi.p, 0, sizeof(double) * n, s.st));
  if (s.n_blocks > 0) {
    ProfScope prof_(s, "p2g");
    k_p2g<<<(unsigned)s.n_blocks, NT, 0, s.st>>>(s.pd.p, s.pmat.p, s.mat_table.p, s.np, s.blk_first.p, s.blk_end.p,
                                                 s.blk_key.p, g, s.topo[0].map.p, s.m.p, s.mv.p, s.mxi.p);
    HOT_LAUNCH("k_p2g");
  }
  if (n > 0) {
    k_grid_finalize<<<(unsigned)((n + NT - 1) / NT), NT, 0, s.st>>>(n, s.topo[0].coords.p, g, s.bc_dev.p,
                                                                    (int)s.bcs.size(), s.m.p, s.mv.p, s.mxi.p,
                                                                    s.v.p, s.xi.p, s.fixed.p);
    HOT_LAUNCH("k_grid_finalize");
  }
}

double max_particle_speed(Scene &s) {
  int nb = 2 * s.nsm;
  s.part.ensure(4096);
  k_speed_max<<<nb, NT, 0, s.st>>>(s.pd.p, s.np, s.part.p);
  HOT_LAUNCH("k_speed_max");
  std::vector<double> h(nb);
  HOT_CUDA(cudaMemcpyAsync(h.data(), s.part.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  double mx = 0.0;
  for (double x : h) mx = x > mx ? x : mx;
  return std::sqrt(mx);
}

void g2p_transfer(Scene &s, const double *vnew) {
  GeoArgs g = geo_args(s);
  if (s.np == 0) return;
  ProfScope prof_(s, "g2p");
  k_g2p<<<(unsigned)((s.np + NT - 1) / NT), NT, 0, s.st>>>(s.pd.p, s.pmat.p, s.mat_table.p, s.np, g,
                                                           s.topo[0].map.p, vnew, s.dt);
  HOT_LAUNCH("k_g2p");
}

void scatter_state_to_user_order(Scene &s, double *x, double *v, double *F, double *C, bool to_device) {
  const int64_t np = s.np;
  if (np == 0) return;
  s.pd_alt.ensure((size_t)PF_COUNT * np, 1.0);
  double *sx = s.pd_alt.p, *sv = sx + 3 * np, *sF = sv + 3 * np, *sC = sF + 9 * np;
  k_soa_to_user<<<(unsigned)((np + NT - 1) / NT), NT, 0, s.st>>>(s.pd.p, s.pid.p, np, sx, sv, sF, sC);
  HOT_LAUNCH("k_soa_to_user");
  cudaMemcpyKind kind = to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (x) HOT_CUDA(cudaMemcpyAsync(x, sx, sizeof(double) * 3 * np, kind, s.st));
  if (v) HOT_CUDA(cudaMemcpyAsync(v, sv, sizeof(double) * 3 * np, kind, s.st));
  if (F) HOT_CUDA(cudaMemcpyAsync(F, sF, sizeof(double) * 9 * np, kind, s.st));
  if (C) HOT_CUDA(cudaMemcpyAsync(C, sC, sizeof(double) * 9 * np, kind, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
}

void load_state_from_user_order(Scene &s, const double *x, const double *v, const double *F, const double *C,
                                bool from_device) {
  const int64_t np = s.np;
  if (np == 0) return;
  s.pd_alt.ensure((size_t)PF_COUNT * np, 1.0);
  double *sx = s.pd_alt.p, *sv = sx + 3 * np, *sF = sv + 3 * np, *sC = sF + 9 * np;
  cudaMemcpyKind kind = from_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  int mask = 0;
  if (x) { HOT_CUDA(cudaMemcpyAsync(sx, x, sizeof(double) * 3 * np, kind, s.st)); mask |= 1; }
  if (v) { HOT_CUDA(cudaMemcpyAsync(sv, v, sizeof(double) * 3 * np, kind, s.st)); mask |= 2; }
  if (F) { HOT_CUDA(cudaMemcpyAsync(sF, F, sizeof(double) * 9 * np, kind, s.st)); mask |= 4; }
  if (C) { HOT_CUDA(cudaMemcpyAsync(sC, C, sizeof(double) * 9 * np, kind, s.st)); mask |= 8; }
  k_user_to_soa<<<(unsigned)((np + NT - 1) / NT), NT, 0, s.st>>>(s.pd.p, s.pid.p, np, sx, sv, sF, sC, mask);
  HOT_LAUNCH("k_user_to_soa");
  HOT_CUDA(cudaStreamSynchronize(s.st));
}

}  // namespace hot
