// Node-embedding Galerkin multigrid (Sec. 4) and the V-cycle of Alg. 2.
//
// Storage: each level keeps its 3x3 blocks in block-CSR with at most 125
// blocks per row (offsets within +-2 per axis at every level, Sec. 6 "Sparse
// matrix storage"); row i stores entry e (3a+b) of its k-th block at
// vals[9*row_ptr[i] + e*nb_i + k], so that a warp reading one entry of 32
// consecutive blocks touches 32 consecutive words.
#include <atomic>
#include "internal.h"

#include <cooperative_groups.h>

#include <mutex>

namespace hot {

namespace {
constexpr int NT = 256;
constexpr int WPB = NT / 32;

__device__ __forceinline__ int64_t lin(int x, int y, int z, const int *nd) { return ((int64_t)z * nd[1] + y) * nd[0] + x; }

struct Dims {
  int d[3];
};
Dims dims_of(const Topo &t) {
  Dims r;
  for (int k = 0; k < 3; ++k) r.d[k] = t.dims[k];
  return r;
}

// cell occupancy lookup (block-major keys of the particle sort)
__device__ __forceinline__ bool cell_occupied(const int *cell_count, int x, int y, int z, const int *nb) {
  unsigned B = ((unsigned)(z >> 2) * (unsigned)nb[1] + (unsigned)(y >> 2)) * (unsigned)nb[0] + (unsigned)(x >> 2);
  unsigned key = B * 64u + (unsigned)(((z & 3) << 4) | ((y & 3) << 2) | (x & 3));
  return cell_count[key] > 0;
}

// Level-0 pattern: block (i, l) exists iff some occupied cell has both nodes
// in its 3^3 stencil, i.e. a cell c with max(i,l) - 2 <= c <= min(i,l) per axis.
__global__ void k_pattern0(int64_t n, const int *__restrict__ coords, const int *__restrict__ map, Dims nd,
                           const int *__restrict__ cell_count, int nb0, int nb1, int nb2, int cd0, int cd1, int cd2,
                           uint32_t *__restrict__ mask, int *__restrict__ rowcnt) {
  int64_t i = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int nb[3] = {nb0, nb1, nb2};
  const int cd[3] = {cd0, cd1, cd2};
  int ci[3] = {coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]};
  int count = 0;
  for (int r = 0; r < 4; ++r) {
    int s = r * 32 + lane;
    bool present = false;
    if (s < NSLOT) {
      int o[3] = {s % 5 - 2, (s / 5) % 5 - 2, s / 25 - 2};
      int cl[3];
      bool ok = true;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cl[k] = ci[k] + o[k];
        ok = ok && cl[k] >= 0 && cl[k] < nd.d[k];
      }
      if (ok && map[lin(cl[0], cl[1], cl[2], nd.d)] >= 0) {
        int lo[3], hi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          lo[k] = max(max(ci[k], cl[k]) - 2, 0);
          hi[k] = min(min(ci[k], cl[k]), cd[k] - 1);
        }
        for (int z = lo[2]; z <= hi[2] && !present; ++z)
          for (int y = lo[1]; y <= hi[1] && !present; ++y)
            for (int x = lo[0]; x <= hi[0] && !present; ++x) present = cell_occupied(cell_count, x, y, z, nb);
      }
    }
    unsigned bal = __ballot_sync(0xffffffffu, present);
    if (lane == 0) mask[4 * i + r] = bal;
    count += __popc(bal);
  }
  if (lane == 0) rowcnt[i] = count;
}

// cols / slotpos from the slot masks (columns in ascending slot order, which
// is ascending node order for (z, y, x)-lexicographic numbering)
// 27-coloring of the Gauss-Seidel sweeps: c = (x mod 3) + 3 (y mod 3) + 9 (z mod 3)
__device__ __forceinline__ int node_color(int x, int y, int z) { return x % 3 + 3 * (y % 3) + 9 * (z % 3); }

// cols / slotpos of each row from its offset mask.  A row keeps first the
// blocks of neighbours colored before the row's own color, then the others
// (the diagonal among them), each part in offset-slot order (which keeps
// spatial neighbours adjacent for the gathers of u).  The first part, of
// length nlow[i], is all that a Gauss-Seidel sweep starting from u = 0 needs
// in its forward half: the other neighbours are still zero.  A stable
// two-way partition with warp ballots; one warp per row.
__global__ void k_fill_pattern(int64_t n, const int *__restrict__ coords, const int *__restrict__ map, Dims nd,
                               const uint32_t *__restrict__ mask, const int *__restrict__ row_ptr,
                               int *__restrict__ cols, int *__restrict__ slotpos, int *__restrict__ nlow) {
  const int lane = threadIdx.x & 31;
  int64_t i = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
  if (i >= n) return;   // warp-uniform
  const int ci[3] = {coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]};
  const int own = node_color(ci[0], ci[1], ci[2]);
  unsigned lowb[4], highb[4];
  int nlo = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int s = r * 32 + lane;
    const bool on = s < NSLOT && ((mask[4 * i + r] >> lane) & 1u);
    const int o[3] = {s % 5 - 2, (s / 5) % 5 - 2, s / 25 - 2};
    const bool lo = on && node_color(ci[0] + o[0], ci[1] + o[1], ci[2] + o[2]) < own;
    lowb[r] = __ballot_sync(0xffffffffu, lo);
    highb[r] = __ballot_sync(0xffffffffu, on && !lo);
    nlo += __popc(lowb[r]);
  }
  const int base = row_ptr[i];
  const unsigned below = (1u << lane) - 1u;
  int lo_before = 0, hi_before = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int s = r * 32 + lane;
    if (s < NSLOT) {
      int rank = -1;
      if ((lowb[r] >> lane) & 1u) rank = lo_before + __popc(lowb[r] & below);
      else if ((highb[r] >> lane) & 1u) rank = nlo + hi_before + __popc(highb[r] & below);
      if (rank >= 0) {
        const int o[3] = {s % 5 - 2, (s / 5) % 5 - 2, s / 25 - 2};
        cols[base + rank] = map[lin(ci[0] + o[0], ci[1] + o[1], ci[2] + o[2], nd.d)];
        slotpos[i * NSLOT + s] = base + rank;
      } else {
        slotpos[i * NSLOT + s] = -1;
      }
    }
    lo_before += __popc(lowb[r]);
    hi_before += __popc(highb[r]);
  }
  if (lane == 0) nlow[i] = nlo;
}

// coarse node candidates of every fine node: |a - 2A| <= 1 per axis
__global__ void k_mark_coarse(int64_t n, const int *__restrict__ coords, Dims cd, uint8_t *__restrict__ flag) {
  int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (i >= n) return;
  int a[3] = {coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]};
  int lo[3], cnt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = (a[k] & 1) ? (a[k] - 1) >> 1 : a[k] >> 1;
    cnt[k] = (a[k] & 1) ? 2 : 1;
  }
  for (int z = 0; z < cnt[2]; ++z)
    for (int y = 0; y < cnt[1]; ++y)
      for (int x = 0; x < cnt[0]; ++x) flag[lin(lo[0] + x, lo[1] + y, lo[2] + z, cd.d)] = 1;
}

// symbolic Galerkin product: coarse (J, K) exists iff some fine a embedded in J
// has a block (a, c) with c embedded in K.  One warp per coarse row.
__global__ void k_pattern_rap(int64_t nc, const int *__restrict__ ccoords, const int *__restrict__ fmap, Dims fd,
                              const int *__restrict__ fcoords, const int *__restrict__ frow_ptr,
                              const int *__restrict__ fcols, uint32_t *__restrict__ mask, int *__restrict__ rowcnt) {
  __shared__ uint32_t smask[WPB][4];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t J = (int64_t)blockIdx.x * WPB + w;
  if (lane < 4) smask[w][lane] = 0u;
  __syncwarp();
  if (J < nc) {
    int cj[3] = {ccoords[3 * J], ccoords[3 * J + 1], ccoords[3 * J + 2]};
    for (int o = 0; o < 27; ++o) {
      int a[3] = {2 * cj[0] + o % 3 - 1, 2 * cj[1] + (o / 3) % 3 - 1, 2 * cj[2] + o / 9 - 1};
      if (a[0] < 0 || a[1] < 0 || a[2] < 0 || a[0] >= fd.d[0] || a[1] >= fd.d[1] || a[2] >= fd.d[2]) continue;
      int ia = fmap[lin(a[0], a[1], a[2], fd.d)];
      if (ia < 0) continue;
      for (int b = frow_ptr[ia] + lane; b < frow_ptr[ia + 1]; b += 32) {
        int c = fcols[b];
        int cc[3] = {fcoords[3 * c], fcoords[3 * c + 1], fcoords[3 * c + 2]};
        int lo[3], cnt[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          lo[k] = (cc[k] & 1) ? (cc[k] - 1) >> 1 : cc[k] >> 1;
          cnt[k] = (cc[k] & 1) ? 2 : 1;
        }
        for (int z = 0; z < cnt[2]; ++z)
          for (int y = 0; y < cnt[1]; ++y)
            for (int x = 0; x < cnt[0]; ++x) {
              int s = (lo[0] + x - cj[0] + 2) + 5 * (lo[1] + y - cj[1] + 2) + 25 * (lo[2] + z - cj[2] + 2);
              atomicOr(&smask[w][s >> 5], 1u << (s & 31));
            }
      }
    }
  }
  __syncwarp();
  if (J < nc && lane < 4) {
    uint32_t mk = smask[w][lane];
    mask[4 * J + lane] = mk;
    int c = __popc(mk);
    c += __shfl_down_sync(0xfu, c, 2, 4);
    c += __shfl_down_sync(0xfu, c, 1, 4);
    if (lane == 0) rowcnt[J] = c;
  }
}

__device__ __forceinline__ float embed_w(int d) { return d == 0 ? 1.0f : 0.5f; }

// Numeric Galerkin product H^{m+1} = R H^m R^T in two gathers, no atomics
// (every sum has one owner and a fixed order, so the hierarchy is bitwise
// reproducible):
//   T_aK   = sum_c H_ac R_Kc   for each fine row a and the coarse nodes K of
//            its window: fine couplings reach c in a +- 2 per axis, whose
//            parents K (|c - 2K| <= 1) lie in [floor(a/2) - 1, floor(a/2) + 2],
//            a 4^3 window; stored entry-major, T[a][e][window slot];
//   H_JK   = sum_a R_Ja T_aK   over the 27 fine children a of J.
// Weights of the linear embedding: 1 on a coarse node, 1/2 between two.
constexpr int RAP_WIN = 64;

// one warp per fine row a; lane l owns window slots l and l + 32
template <class T>
__global__ void k_rap_t(int64_t nf, const int *__restrict__ fcoords, const int *__restrict__ frow_ptr,
                        const int *__restrict__ fslotpos, const T *__restrict__ fvals, T *__restrict__ tout) {
  const int64_t a = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
  if (a >= nf) return;
  const int lane = threadIdx.x & 31;
  const int ca[3] = {fcoords[3 * a], fcoords[3 * a + 1], fcoords[3 * a + 2]};
  const int rp = frow_ptr[a], nb = frow_ptr[a + 1] - rp;
  const T *v = fvals + 9 * (int64_t)rp;
  const int *sp = fslotpos + a * NSLOT;
  T *to = tout + a * (9 * RAP_WIN);
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int q = lane + 32 * half;
    const int K[3] = {(ca[0] >> 1) - 1 + (q & 3), (ca[1] >> 1) - 1 + ((q >> 2) & 3), (ca[2] >> 1) - 1 + (q >> 4)};
    int lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {   // children c = 2K + oc of K within a +- 2
      lo[k] = max(-1, ca[k] - 2 * K[k] - 2);
      hi[k] = min(1, ca[k] - 2 * K[k] + 2);
    }
    T acc[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[e] = T(0);
    for (int oz = lo[2]; oz <= hi[2]; ++oz)
      for (int oy = lo[1]; oy <= hi[1]; ++oy)
        for (int ox = lo[0]; ox <= hi[0]; ++ox) {
          const int ex = 2 * K[0] + ox - ca[0], ey = 2 * K[1] + oy - ca[1], ez = 2 * K[2] + oz - ca[2];
          const int pos = sp[(ex + 2) + 5 * (ey + 2) + 25 * (ez + 2)];
          if (pos < 0) continue;
          const T w = (T)(embed_w(ox) * embed_w(oy) * embed_w(oz));
          const int k = pos - rp;
#pragma unroll
          for (int e = 0; e < 9; ++e) acc[e] = fma(w, v[e * nb + k], acc[e]);
        }
#pragma unroll
    for (int e = 0; e < 9; ++e) to[e * RAP_WIN + q] = acc[e];
  }
  (void)nb;
}

// one thread per coarse block (J, K = J + d) of coarse row J
template <class T>
__global__ void __launch_bounds__(128) k_rap_r(int64_t nc, const int *__restrict__ ccoords,
                                               const int *__restrict__ crow_ptr, const int *__restrict__ cslotpos,
                                               T *__restrict__ cvals, const int *__restrict__ fmap, Dims fd,
                                               const T *__restrict__ tin) {
  const int64_t J = blockIdx.x;
  const int s = threadIdx.x;
  if (J >= nc || s >= NSLOT) return;
  const int cpos = cslotpos[J * NSLOT + s];
  if (cpos < 0) return;
  const int d[3] = {s % 5 - 2, (s / 5) % 5 - 2, s / 25 - 2};
  const int cj[3] = {ccoords[3 * J], ccoords[3 * J + 1], ccoords[3 * J + 2]};
  T acc[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) acc[e] = T(0);
  for (int o = 0; o < 27; ++o) {
    const int oa[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
    int q = 0;
    bool in = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int a = 2 * cj[k] + oa[k];
      const int qk = d[k] - (oa[k] < 0 ? -1 : 0) + 1;   // K - (floor(a/2) - 1)
      in = in && a >= 0 && a < fd.d[k] && qk >= 0 && qk < 4;
      q += qk << (2 * k);
    }
    if (!in) continue;
    const int ia = fmap[lin(2 * cj[0] + oa[0], 2 * cj[1] + oa[1], 2 * cj[2] + oa[2], fd.d)];
    if (ia < 0) continue;
    const T w = (T)(embed_w(oa[0]) * embed_w(oa[1]) * embed_w(oa[2]));
    const T *tr = tin + (int64_t)ia * (9 * RAP_WIN) + q;
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[e] = fma(w, tr[e * RAP_WIN], acc[e]);
  }
  const int rp = crow_ptr[J], nb = crow_ptr[J + 1] - rp;
  T *cv = cvals + 9 * (int64_t)rp;
#pragma unroll
  for (int e = 0; e < 9; ++e) cv[e * nb + (cpos - rp)] = acc[e];
}

// Inverse of each diagonal block (formed in float64) and the scalar diagonal.
// A block that is not safely positive definite in the level's precision (its
// Cholesky pivots fail, or in float32 the smallest pivot is below 1e-6 of the
// largest, where rounding of a stiffness-dominated block swamps the mass
// term) is shifted by a multiple of its mean diagonal until it is.  In float64
// the assembled blocks are positive definite and the shift stays zero.
template <class T>
__global__ void k_diag(int64_t n, const int *__restrict__ row_ptr, const int *__restrict__ slotpos,
                       const T *__restrict__ vals, T *__restrict__ dinv, T *__restrict__ diag) {
  int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (i >= n) return;
  int rp = row_ptr[i], nb = row_ptr[i + 1] - rp;
  int pos = slotpos[i * NSLOT + DIAG_SLOT] - rp;
  double D[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) D[e] = (double)vals[9 * (int64_t)rp + e * nb + pos];
  const double mean = fabs(D[0] + D[4] + D[8]) / 3.0 + 1e-300;
  const double ratio = sizeof(T) == 4 ? 1e-6 : 0.0;
  double shift = 0.0;
  for (int attempt = 0; attempt < 12; ++attempt) {
    // Cholesky pivots of the symmetric part of D + shift I
    double a00 = D[0] + shift, a11 = D[4] + shift, a22 = D[8] + shift;
    double a01 = 0.5 * (D[1] + D[3]), a02 = 0.5 * (D[2] + D[6]), a12 = 0.5 * (D[5] + D[7]);
    double p0 = a00;
    bool ok = p0 > 0.0;
    double l10 = ok ? a01 / p0 : 0.0, l20 = ok ? a02 / p0 : 0.0;
    double p1 = a11 - l10 * a01;
    ok = ok && p1 > 0.0;
    double l21 = ok ? (a12 - l20 * a01) / p1 : 0.0;
    double p2 = a22 - l20 * a02 - l21 * l21 * p1;
    ok = ok && p2 > 0.0;
    if (ok) {
      double pmax = fmax(p0, fmax(p1, p2)), pmin = fmin(p0, fmin(p1, p2));
      if (pmin >= ratio * pmax) break;
    }
    shift = (shift == 0.0 ? (sizeof(T) == 4 ? 1e-6 : 1e-12) : 10.0 * shift / mean) * mean;
  }
  D[0] += shift;
  D[4] += shift;
  D[8] += shift;
  double c[9];
  cofactor3(D, c);
  double inv = 1.0 / (D[0] * c[0] + D[1] * c[1] + D[2] * c[2]);
  // inverse = cof^T / det
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) dinv[9 * i + 3 * a + b] = (T)(c[3 * b + a] * inv);
  diag[3 * i] = (T)D[0];
  diag[3 * i + 1] = (T)D[4];
  diag[3 * i + 2] = (T)D[8];
}

// 27-coloring c = (x mod 3) + 3 (y mod 3) + 9 (z mod 3)
__global__ void k_color_count(int64_t n, const int *__restrict__ coords, int *__restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (i >= n) return;
  int c = node_color(coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]);
  atomicAdd(&cnt[c], 1);
}
__global__ void k_color_fill(int64_t n, const int *__restrict__ coords, int *__restrict__ cursor,
                             int *__restrict__ list) {
  int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (i >= n) return;
  int c = node_color(coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]);
  list[atomicAdd(&cursor[c], 1)] = (int)i;
}

// one 16-byte record per entry of the color list: the row, where its blocks
// start and how many there are (one load instead of a chain of three)
__global__ void k_color_records(int64_t n, const int *__restrict__ list, const int *__restrict__ row_ptr,
                                const int *__restrict__ nlow, int4 *__restrict__ rec) {
  int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e >= n) return;
  const int i = list[e], rp = row_ptr[i];
  rec[e] = make_int4(i, rp, row_ptr[i + 1] - rp, nlow[i]);
}

// ---------------------------------------------------------------------------
// smoothing kernels: a group of RL consecutive lanes per row.  Lanes of a
// group read consecutive blocks of the row (entry-major storage keeps each of
// the 9 entry streams contiguous), then the group reduces its 3 sums with
// log2(RL) shuffles.
// ---------------------------------------------------------------------------
constexpr int RL = 32;
constexpr int RPW = 32 / RL;   // rows per warp

// Partial sums of (H u)_i over the blocks this lane visits, as explicit FMA
// chains (the FP64 pipe is the bound of these kernels: 9 FMA per block).
// matrix values of type T, vector and sums of type U (U = T, or double over
// a float matrix on the coarsest level)
template <class T, class U = T>
__device__ __forceinline__ void row_partial(int64_t i, bool valid, int lane, const int *__restrict__ row_ptr,
                                            const int *__restrict__ cols, const T *__restrict__ vals,
                                            const U *u, bool skip_diag, U acc[3]) {
  acc[0] = acc[1] = acc[2] = U(0);
  if (!valid) return;
  const int rp = row_ptr[i], nb = row_ptr[i + 1] - rp;
  const T *v = vals + 9 * (int64_t)rp;
#pragma unroll 2
  for (int b = lane; b < nb; b += RL) {
    int j = cols[rp + b];
    U h[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) h[e] = (U)v[e * nb + b];
    if (skip_diag && j == i) continue;
    const U u0 = u[3 * j], u1 = u[3 * j + 1], u2 = u[3 * j + 2];
    acc[0] = fma(h[0], u0, acc[0]);
    acc[1] = fma(h[3], u0, acc[1]);
    acc[2] = fma(h[6], u0, acc[2]);
    acc[0] = fma(h[1], u1, acc[0]);
    acc[1] = fma(h[4], u1, acc[1]);
    acc[2] = fma(h[7], u1, acc[2]);
    acc[0] = fma(h[2], u2, acc[0]);
    acc[1] = fma(h[5], u2, acc[1]);
    acc[2] = fma(h[8], u2, acc[2]);
  }
}

// (H u)_i summed over the warp, result in every lane (all three components).
template <class T>
__device__ __forceinline__ void row_product(int64_t i, bool valid, int lane, const int *__restrict__ row_ptr,
                                            const int *__restrict__ cols, const T *__restrict__ vals,
                                            const T *u, bool skip_diag, T acc[3]) {
  row_partial<T>(i, valid, lane, row_ptr, cols, vals, u, skip_diag, acc);
#pragma unroll
  for (int o = RL / 2; o > 0; o >>= 1) {
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
    acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], o);
    acc[2] += __shfl_xor_sync(0xffffffffu, acc[2], o);
  }
}

// Warp sum of three per-lane values with 6 additions instead of 15: the
// halves first trade components (lanes 0-15 keep 0 and 1, lanes 16-31 keep
// 2), then lanes 0-7 / 8-15 split 0 and 1.  Lanes 0-7 return the sum of
// component 0, lanes 8-15 of component 1, lanes 16-31 of component 2.
template <class T>
__device__ __forceinline__ T warp_sum3_split(const T a[3], int lane) {
  const bool up = lane & 16, b3 = lane & 8;
  const T r0 = __shfl_xor_sync(0xffffffffu, up ? a[0] : a[2], 16);
  const T r1 = __shfl_xor_sync(0xffffffffu, a[1], 16);
  const T x = (up ? a[2] : a[0]) + r0;   // lanes 0-15: component 0; 16-31: component 2
  const T y = a[1] + r1;                 // lanes 0-15: component 1
  T keep = (!up && b3) ? y : x;
  const T send = (!up && !b3) ? y : x;
  keep += __shfl_xor_sync(0xffffffffu, send, 8);
  keep += __shfl_xor_sync(0xffffffffu, keep, 4);
  keep += __shfl_xor_sync(0xffffffffu, keep, 2);
  keep += __shfl_xor_sync(0xffffffffu, keep, 1);
  return keep;
}

// A row of the block matrix held in registers: every load of the row (its
// blocks, D_i^-1 and b_i) is issued at once, so a row costs one memory round
// trip for the matrix and one for the gathered u_j.
constexpr int SW_PRE = 4;   // blocks of a row held in registers per lane (rows have <= 125)

template <class T>
struct RowRegs {
  int j[SW_PRE];
  T h[SW_PRE][9];
  T bv;      // lanes 0, 8, 16: component lane/8 of b_i
  T d[3];    // lanes 0-2: row `lane` of D_i^-1
};

// nb: blocks in the row (the stride of its entry streams); nuse: the leading
// blocks to use (nb, or the prefix of neighbours colored before the row when
// the others are still zero)
template <class T>
__device__ __forceinline__ void load_row(RowRegs<T> &R, int64_t i, int rp, int nb, int nuse, int lane,
                                         const int *__restrict__ cols, const T *__restrict__ vals,
                                         const T *__restrict__ dinv, const T *__restrict__ b) {
  const T *v = vals + 9 * (int64_t)rp;
#pragma unroll
  for (int q = 0; q < SW_PRE; ++q) {
    const int e0 = lane + 32 * q;
    R.j[q] = e0 < nuse ? cols[rp + e0] : -1;
#pragma unroll
    for (int e = 0; e < 9; ++e) R.h[q][e] = e0 < nuse ? v[e * nb + e0] : T(0);
  }
  R.bv = ((lane & 7) == 0 && lane < 24) ? b[3 * i + (lane >> 3)] : T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) R.d[c] = lane < 3 ? dinv[9 * i + 3 * lane + c] : T(0);
}

// u_i from a row held in registers (LDCG: u read through L2, for launches in
// which other SMs write it)
template <class T, bool LDCG>
__device__ __forceinline__ T ld_u(const T *p) {
  if (LDCG) return __ldcg(p);
  return *p;
}

// the new u_i of a row held in registers, on lanes 0-2 (component `lane`)
template <class T, bool LDCG>
__device__ __forceinline__ T row_new_u(const RowRegs<T> &R, int64_t i, int rp, int nb, int nuse, int lane,
                                       const int *__restrict__ cols, const T *__restrict__ vals, const T *u) {
  T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < SW_PRE; ++q) {
    // FP64: a warp-wide FP64 instruction holds the SM's FP64 pipe whether or
    // not its lanes are predicated on, so chunks past the used blocks are
    // skipped by a warp-uniform branch.  FP32: no branch, so the u gathers of
    // every chunk issue together.
    if (sizeof(T) == 8 && 32 * q >= nuse) break;
    const int j = R.j[q];
    if (j < 0 || j == i) continue;
    const T u0 = ld_u<T, LDCG>(u + 3 * j), u1 = ld_u<T, LDCG>(u + 3 * j + 1), u2 = ld_u<T, LDCG>(u + 3 * j + 2);
    acc[0] = fma(R.h[q][0], u0, acc[0]);
    acc[1] = fma(R.h[q][3], u0, acc[1]);
    acc[2] = fma(R.h[q][6], u0, acc[2]);
    acc[0] = fma(R.h[q][1], u1, acc[0]);
    acc[1] = fma(R.h[q][4], u1, acc[1]);
    acc[2] = fma(R.h[q][7], u1, acc[2]);
    acc[0] = fma(R.h[q][2], u2, acc[0]);
    acc[1] = fma(R.h[q][5], u2, acc[1]);
    acc[2] = fma(R.h[q][8], u2, acc[2]);
  }
  // rows longer than the register window (not produced by the 5^3 stencil)
  const T *v = vals + 9 * (int64_t)rp;
  for (int e0 = lane + 32 * SW_PRE; e0 < nuse; e0 += 32) {
    const int j = cols[rp + e0];
    if (j == i) continue;
    const T u0 = ld_u<T, LDCG>(u + 3 * j), u1 = ld_u<T, LDCG>(u + 3 * j + 1), u2 = ld_u<T, LDCG>(u + 3 * j + 2);
    acc[0] = fma(v[e0], u0, acc[0]);
    acc[1] = fma(v[3 * nb + e0], u0, acc[1]);
    acc[2] = fma(v[6 * nb + e0], u0, acc[2]);
    acc[0] = fma(v[nb + e0], u1, acc[0]);
    acc[1] = fma(v[4 * nb + e0], u1, acc[1]);
    acc[2] = fma(v[7 * nb + e0], u1, acc[2]);
    acc[0] = fma(v[2 * nb + e0], u2, acc[0]);
    acc[1] = fma(v[5 * nb + e0], u2, acc[1]);
    acc[2] = fma(v[8 * nb + e0], u2, acc[2]);
  }
  const T sum = warp_sum3_split<T>(acc, lane);
  const T y = ((lane & 7) == 0 && lane < 24) ? R.bv - sum : T(0);
  const T y0 = __shfl_sync(0xffffffffu, y, 0), y1 = __shfl_sync(0xffffffffu, y, 8),
          y2 = __shfl_sync(0xffffffffu, y, 16);
  return fma(R.d[2], y2, fma(R.d[1], y1, R.d[0] * y0));
}

template <class T, bool LDCG = true>
__device__ __forceinline__ void update_row(const RowRegs<T> &R, int64_t i, int rp, int nb, int nuse, int lane,
                                           const int *__restrict__ cols, const T *__restrict__ vals, T *u) {
  const T val = row_new_u<T, LDCG>(R, i, rp, nb, nuse, lane, cols, vals, u);
  if (lane < 3) u[3 * i + lane] = val;
}

// One row of a Gauss-Seidel color: u_i <- D_i^{-1} (b_i - sum_{j != i} H_ij u_j)
// (one warp per row; lanes 0, 8, 16 form the three residual components and
// lanes 0-2 apply the three rows of D_i^{-1}).
// one color of a sweep, one launch (rows given by their color records)
// (low: only the prefix of neighbours colored before the row, r.w blocks)
template <class T>
__global__ void k_sgs_color(const int4 *__restrict__ rec, int nrows, const int *__restrict__ cols,
                            const T *__restrict__ vals, const T *__restrict__ dinv, const T *__restrict__ b, T *u,
                            int low) {
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);   // one warp per row
  if (g >= nrows) return;   // warp-uniform
  const int lane = threadIdx.x & 31;
  const int4 r = rec[g];
  const int nuse = low ? r.w : r.z;
  RowRegs<T> R;
  load_row<T>(R, r.x, r.y, r.z, nuse, lane, cols, vals, dinv, b);
  update_row<T, false>(R, r.x, r.y, r.z, nuse, lane, cols, vals, u);
}

// r = b - H u
template <class T>
__global__ void k_residual(int64_t n, const int *__restrict__ row_ptr, const int *__restrict__ cols,
                           const T *__restrict__ vals, const T *__restrict__ b, const T *__restrict__ u,
                           T *__restrict__ r) {
  const int64_t i = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
  if (i >= n) return;   // warp-uniform
  const int lane = threadIdx.x & 31;
  const int rp = row_ptr[i], nb = row_ptr[i + 1] - rp;
  const T *v = vals + 9 * (int64_t)rp;
  int j[SW_PRE];
  T h[SW_PRE][9];
#pragma unroll
  for (int q = 0; q < SW_PRE; ++q) {
    const int e0 = lane + 32 * q;
    j[q] = e0 < nb ? cols[rp + e0] : -1;
#pragma unroll
    for (int e = 0; e < 9; ++e) h[q][e] = e0 < nb ? v[e * nb + e0] : T(0);
  }
  T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < SW_PRE; ++q) {
    if (sizeof(T) == 8 && 32 * q >= nb) break;   // FP64: skip unused chunks (warp-uniform)
    if (j[q] < 0) continue;
    const T u0 = u[3 * j[q]], u1 = u[3 * j[q] + 1], u2 = u[3 * j[q] + 2];
    acc[0] = fma(h[q][0], u0, acc[0]);
    acc[1] = fma(h[q][3], u0, acc[1]);
    acc[2] = fma(h[q][6], u0, acc[2]);
    acc[0] = fma(h[q][1], u1, acc[0]);
    acc[1] = fma(h[q][4], u1, acc[1]);
    acc[2] = fma(h[q][7], u1, acc[2]);
    acc[0] = fma(h[q][2], u2, acc[0]);
    acc[1] = fma(h[q][5], u2, acc[1]);
    acc[2] = fma(h[q][8], u2, acc[2]);
  }
  for (int e0 = lane + 32 * SW_PRE; e0 < nb; e0 += 32) {   // rows longer than the register window
    const int jj = cols[rp + e0];
    const T u0 = u[3 * jj], u1 = u[3 * jj + 1], u2 = u[3 * jj + 2];
    acc[0] = fma(v[e0], u0, acc[0]);
    acc[1] = fma(v[3 * nb + e0], u0, acc[1]);
    acc[2] = fma(v[6 * nb + e0], u0, acc[2]);
    acc[0] = fma(v[nb + e0], u1, acc[0]);
    acc[1] = fma(v[4 * nb + e0], u1, acc[1]);
    acc[2] = fma(v[7 * nb + e0], u1, acc[2]);
    acc[0] = fma(v[2 * nb + e0], u2, acc[0]);
    acc[1] = fma(v[5 * nb + e0], u2, acc[1]);
    acc[2] = fma(v[8 * nb + e0], u2, acc[2]);
  }
  const T sum = warp_sum3_split<T>(acc, lane);
  if ((lane & 7) == 0 && lane < 24) {
    const int64_t k = 3 * i + (lane >> 3);
    r[k] = b[k] - sum;
  }
}

// Residual from half of the symmetric matrix (option, flag bit 7): every
// off-diagonal coupling sits in the earlier-colored prefix of exactly one of
// its two rows, so the prefixes plus the diagonal blocks hold the matrix
// once.  r = b - D u first; then each prefix block H_ij of row i gives
// -H_ij u_j to r_i and, transposed, -H_ij^T u_i to r_j (atomic adds).  Half
// the matrix bytes of the full residual, three atomics per block.
template <class T>
__global__ void k_residual_diag(int64_t n, const int *__restrict__ row_ptr, const int *__restrict__ slotpos,
                                const T *__restrict__ vals, const T *__restrict__ b, const T *__restrict__ u,
                                T *__restrict__ r) {
  const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (i >= n) return;
  const int rp = row_ptr[i], nb = row_ptr[i + 1] - rp, k = slotpos[NSLOT * i + DIAG_SLOT] - rp;
  const T *v = vals + 9 * (int64_t)rp + k;
  const T u0 = u[3 * i], u1 = u[3 * i + 1], u2 = u[3 * i + 2];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    r[3 * i + c] = b[3 * i + c] - (v[(3 * c) * nb] * u0 + v[(3 * c + 1) * nb] * u1 + v[(3 * c + 2) * nb] * u2);
}

template <class T>
__global__ void k_residual_half(int64_t n, const int *__restrict__ row_ptr, const int *__restrict__ cols,
                                const int *__restrict__ nlow, const T *__restrict__ vals, const T *__restrict__ u,
                                T *r) {
  const int64_t i = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
  if (i >= n) return;   // warp-uniform
  const int lane = threadIdx.x & 31;
  const int rp = row_ptr[i], nb = row_ptr[i + 1] - rp, nl = nlow[i];
  const T *v = vals + 9 * (int64_t)rp;
  const T ui0 = u[3 * i], ui1 = u[3 * i + 1], ui2 = u[3 * i + 2];
  T acc[3] = {T(0), T(0), T(0)};
  for (int e0 = lane; e0 < nl; e0 += 32) {
    const int j = cols[rp + e0];
    T h[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) h[e] = v[e * nb + e0];
    const T u0 = u[3 * j], u1 = u[3 * j + 1], u2 = u[3 * j + 2];
    acc[0] = fma(h[0], u0, fma(h[1], u1, fma(h[2], u2, acc[0])));
    acc[1] = fma(h[3], u0, fma(h[4], u1, fma(h[5], u2, acc[1])));
    acc[2] = fma(h[6], u0, fma(h[7], u1, fma(h[8], u2, acc[2])));
    atomicAdd(r + 3 * j, -(h[0] * ui0 + h[3] * ui1 + h[6] * ui2));
    atomicAdd(r + 3 * j + 1, -(h[1] * ui0 + h[4] * ui1 + h[7] * ui2));
    atomicAdd(r + 3 * j + 2, -(h[2] * ui0 + h[5] * ui1 + h[8] * ui2));
  }
  const T sum = warp_sum3_split<T>(acc, lane);
  if ((lane & 7) == 0 && lane < 24) atomicAdd(r + 3 * i + (lane >> 3), -sum);
}

// b^{m+1}_J = sum_a R_Ja r_a over the 27 fine nodes a = 2J + o
template <class T>
__global__ void k_restrict(int64_t nc, const int *__restrict__ ccoords, const int *__restrict__ fmap, Dims fd,
                           const T *__restrict__ r, T *__restrict__ bc) {
  int64_t J = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (J >= nc) return;
  int cj[3] = {ccoords[3 * J], ccoords[3 * J + 1], ccoords[3 * J + 2]};
  T acc[3] = {T(0), T(0), T(0)};
  for (int o = 0; o < 27; ++o) {
    int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
    int a[3] = {2 * cj[0] + ox, 2 * cj[1] + oy, 2 * cj[2] + oz};
    if (a[0] < 0 || a[1] < 0 || a[2] < 0 || a[0] >= fd.d[0] || a[1] >= fd.d[1] || a[2] >= fd.d[2]) continue;
    int ia = fmap[lin(a[0], a[1], a[2], fd.d)];
    if (ia < 0) continue;
    T w = (T)(embed_w(ox) * embed_w(oy) * embed_w(oz));
    acc[0] += w * r[3 * ia];
    acc[1] += w * r[3 * ia + 1];
    acc[2] += w * r[3 * ia + 2];
  }
  bc[3 * J] = acc[0];
  bc[3 * J + 1] = acc[1];
  bc[3 * J + 2] = acc[2];
}

// u^m_a += sum_J R_Ja u^{m+1}_J over the 1..8 coarse parents of a
template <class T>
__global__ void k_prolong_add(int64_t nf, const int *__restrict__ fcoords, const int *__restrict__ cmap, Dims cd,
                              const T *__restrict__ uc, T *__restrict__ uf) {
  int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (i >= nf) return;
  int a[3] = {fcoords[3 * i], fcoords[3 * i + 1], fcoords[3 * i + 2]};
  int lo[3], cnt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = (a[k] & 1) ? (a[k] - 1) >> 1 : a[k] >> 1;
    cnt[k] = (a[k] & 1) ? 2 : 1;
  }
  T w = (T)(embed_w(cnt[0] - 1) * embed_w(cnt[1] - 1) * embed_w(cnt[2] - 1));
  T acc[3] = {T(0), T(0), T(0)};
  for (int z = 0; z < cnt[2]; ++z)
    for (int y = 0; y < cnt[1]; ++y)
      for (int x = 0; x < cnt[0]; ++x) {
        int J = cmap[lin(lo[0] + x, lo[1] + y, lo[2] + z, cd.d)];
        acc[0] += uc[3 * J];
        acc[1] += uc[3 * J + 1];
        acc[2] += uc[3 * J + 2];
      }
  uf[3 * i] += w * acc[0];
  uf[3 * i + 1] += w * acc[1];
  uf[3 * i + 2] += w * acc[2];
}

template <class T>
__global__ void k_load_rhs(int64_t n, const double *__restrict__ src, const uint8_t *__restrict__ fixed,
                           T *__restrict__ dst) {
  int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (k >= 3 * n) return;
  dst[k] = fixed[k / 3] ? T(0) : (T)src[k];
}
template <class T>
__global__ void k_store_out(int64_t n, const T *__restrict__ src, const uint8_t *__restrict__ fixed,
                            double *__restrict__ dst) {
  int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (k >= 3 * n) return;
  dst[k] = fixed[k / 3] ? 0.0 : (double)src[k];
}

// ---------------------------------------------------------------------------
// Coarsest level: Jacobi-preconditioned CG in one cooperative launch.  The
// stopping rule is the adaptive one of Sec. 5.3 read as
//   k = min(1/2, sqrt(max(sqrt(b^T D^-1 b), tau))),  stop when
//   sqrt(r^T D^-1 r) <= k sqrt(b^T D^-1 b),
// with D the scalar diagonal.  Every block sums the same partials in the same
// order, so all blocks take the same branch.  The grid barrier gives up after
// a bounded number of polls and reports DEV_ERR_TIMEOUT.
// ---------------------------------------------------------------------------
// every spin wait gives up after the scene's poll limit (mpm_set_wait_limit;
// default 1 << 24 polls), sets DEV_ERR_TIMEOUT and returns
__device__ bool grid_sync(unsigned *bar, unsigned &gen, int *err, long long spin_limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    unsigned arrived = atomicAdd(&bar[0], 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      long long spins = 0;
      while (*((volatile unsigned *)&bar[1]) == gen) {
        if (!keep_waiting(spins, spin_limit)) {
          ok = 0;
          atomicOr(err, DEV_ERR_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
  }
  gen += 1;
  __syncthreads();
  return ok != 0;
}

// ---------------------------------------------------------------------------
// A whole symmetric Gauss-Seidel smoothing of one level (forward colors, then
// backward) in one cooperative launch, with a grid barrier between colors.
// The color order and the per-row arithmetic are those of the one-launch-
// per-color path (the results are bitwise the same); only the launch
// boundaries become barriers.  On levels with few rows per color the time of
// a color is a chain of memory latencies, not work, so:
//  - rows are dealt round-robin over the blocks first (one SM per row while
//    there are fewer rows than SMs);
//  - each warp's first row of every color is found (list, row_ptr) once, at
//    the start, and kept in shared memory;
//  - the barrier is split: a block signals its arrival, loads the matrix
//    row, D_i^-1 and b_i of its next color (they do not depend on u), and
//    only then waits, so those loads overlap the other blocks' arrival.
// ---------------------------------------------------------------------------
struct SweepPlan {
  int off[54];   // first entry of each step's rows in the color list
  int nr[54];    // rows of each step
  int steps;
  int low_steps; // leading steps whose rows use only their lower-colored prefix (sweep from u = 0)
};

constexpr int SW_NT = 512;
constexpr int SW_WARPS = SW_NT / 32;
__device__ __forceinline__ void bar_arrive_release(unsigned *bar) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
}
__device__ __forceinline__ unsigned bar_load_acquire(const unsigned *bar) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
  return v;
}

// MULTI: some color has more rows than the grid has warps (further rounds).
// CLUSTER: the grid is one thread-block cluster and the barrier between colors
// is the hardware cluster barrier, split the same way (arrive with release
// semantics, load the next row, wait with acquire semantics); for levels whose
// colors have few rows, where the grid-wide barrier's latency, not the rows'
// work, sets the time of a color.
template <class T, bool MULTI, bool CLUSTER = false>
__global__ void __launch_bounds__(SW_NT, 1) k_sgs_persistent(SweepPlan plan, const int4 *__restrict__ rec,
                                                             const int *__restrict__ cols, const T *__restrict__ vals,
                                                             const T *__restrict__ dinv, const T *__restrict__ b, T *u,
                                                             unsigned *bar, int *err, long long spin_limit) {
  __shared__ int4 s_rec[54][SW_WARPS];
  __shared__ int s_ok;
  const int G = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int first = blockIdx.x + G * warp;   // this warp's first-round row of every step
  // .w becomes the number of leading blocks this step uses (the earlier-colored
  // prefix while u is zero beyond it, else the whole row)
  for (int k = lane; k < plan.steps; k += 32) {
    int4 rr = first < plan.nr[k] ? rec[plan.off[k] + first] : make_int4(-1, 0, 0, 0);
    if (k >= plan.low_steps) rr.w = rr.z;
    s_rec[k][warp] = rr;
  }
  if (threadIdx.x == 0) s_ok = 1;
  __syncthreads();
  RowRegs<T> R;
  {
    const int4 r0 = s_rec[0][warp];
    if (r0.x >= 0) load_row<T>(R, r0.x, r0.y, r0.z, r0.w, lane, cols, vals, dinv, b);
  }
  unsigned target = 0;
  for (int k = 0; k < plan.steps; ++k) {
    const int4 r = s_rec[k][warp];
    if (r.x >= 0) update_row<T, true>(R, r.x, r.y, r.z, r.w, lane, cols, vals, u);
    // further rounds (more rows in this color than warps in the grid)
    if (MULTI) {
      for (int g = first + G * SW_WARPS; g < plan.nr[k]; g += G * SW_WARPS) {
        const int4 r2 = rec[plan.off[k] + g];
        const int nuse2 = k < plan.low_steps ? r2.w : r2.z;
        // the registers of the row just updated are free: reuse them
        load_row<T>(R, r2.x, r2.y, r2.z, nuse2, lane, cols, vals, dinv, b);
        update_row<T, true>(R, r2.x, r2.y, r2.z, nuse2, lane, cols, vals, u);
      }
    }
    if (k + 1 == plan.steps) break;
    if (CLUSTER) {
      // every thread releases its own stores of u; all wait for all
      __syncwarp();
      asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
      const int4 rn = s_rec[k + 1][warp];
      if (rn.x >= 0) load_row<T>(R, rn.x, rn.y, rn.z, rn.w, lane, cols, vals, dinv, b);
      asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
      continue;
    }
    __syncthreads();   // the block's updates of this color precede its arrival
    if (threadIdx.x == 0) bar_arrive_release(bar);
    target += (unsigned)G;
    const int4 rn = s_rec[k + 1][warp];
    if (rn.x >= 0) load_row<T>(R, rn.x, rn.y, rn.z, rn.w, lane, cols, vals, dinv, b);
    if (threadIdx.x == 0) {
      long long spins = 0;
      while (bar_load_acquire(bar) < target) {
        if (!keep_waiting(spins, spin_limit)) {
          s_ok = 0;
          atomicOr(err, DEV_ERR_TIMEOUT);
          break;
        }
      }
    }
    __syncthreads();
    if (!s_ok) return;
  }
}

// A whole symmetric sweep of a small level on one thread-block cluster with
// the level's u held in shared memory: every CTA keeps a copy of all of u,
// gathers the neighbours' u_j from its own copy, and writes each new u_i into
// every CTA's copy (distributed shared memory).  The hardware cluster barrier
// between colors (arrive with release, wait with acquire, at cluster scope)
// orders those writes; u goes back to global memory once, after the last
// color.  A color then costs the barrier and on-chip latencies instead of two
// round trips through L2.  Rows, color order and per-row arithmetic are those
// of k_sgs_persistent, so the result is bitwise the same.
template <class T>
__global__ void __launch_bounds__(SW_NT, 1) k_sgs_cluster_smem(SweepPlan plan, const int4 *__restrict__ rec,
                                                               const int *__restrict__ cols,
                                                               const T *__restrict__ vals,
                                                               const T *__restrict__ dinv, const T *__restrict__ b,
                                                               T *u, int n) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ int4 s_rec[54][SW_WARPS];
  extern __shared__ __align__(16) unsigned char sw_dyn[];
  T *su = reinterpret_cast<T *>(sw_dyn);
  const int G = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster.block_rank();
  const int first = blockIdx.x + G * warp;
  for (int k = lane; k < plan.steps; k += 32) {
    int4 rr = first < plan.nr[k] ? rec[plan.off[k] + first] : make_int4(-1, 0, 0, 0);
    if (k >= plan.low_steps) rr.w = rr.z;
    s_rec[k][warp] = rr;
  }
  for (int k = threadIdx.x; k < 3 * n; k += SW_NT) su[k] = u[k];
  // every copy is loaded (and every CTA is running) before any remote write
  cluster.sync();
  RowRegs<T> R;
  {
    const int4 r0 = s_rec[0][warp];
    if (r0.x >= 0) load_row<T>(R, r0.x, r0.y, r0.z, r0.w, lane, cols, vals, dinv, b);
  }
  for (int k = 0; k < plan.steps; ++k) {
    const int4 r = s_rec[k][warp];
    if (r.x >= 0) {   // warp-uniform
      const T val = row_new_u<T, false>(R, r.x, r.y, r.z, r.w, lane, cols, vals, su);
      const T w0 = __shfl_sync(0xffffffffu, val, 0), w1 = __shfl_sync(0xffffffffu, val, 1),
              w2 = __shfl_sync(0xffffffffu, val, 2);
      if (lane < G) {
        T *dst = cluster.map_shared_rank(su, lane) + 3 * (int64_t)r.x;
        dst[0] = w0;
        dst[1] = w1;
        dst[2] = w2;
      }
    }
    if (k + 1 == plan.steps) break;
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    const int4 rn = s_rec[k + 1][warp];
    if (rn.x >= 0) load_row<T>(R, rn.x, rn.y, rn.z, rn.w, lane, cols, vals, dinv, b);
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
  // every copy is final; no CTA writes another's shared memory after this
  cluster.sync();
  for (int k = rank * SW_NT + threadIdx.x; k < 3 * n; k += G * SW_NT) u[k] = su[k];
}

// Distributed-shared-memory helpers (PTX): 32-bit shared-window addresses,
// their image in another CTA of the cluster, mbarriers with transaction
// counts, and remote stores that report their bytes to the receiving CTA's
// mbarrier.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// waits in hardware (the thread is suspended, up to about `hint_ns`, so it
// takes no issue slots from warps still computing) for the phase of the
// given parity; false if it has not completed by then
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ void st_async_tx(uint32_t addr, float v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
               "r"(__float_as_uint(v)), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_async_tx(uint32_t addr, double v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr),
               "l"(__double_as_longlong(v)), "r"(bar)
               : "memory");
}

// The same sweep as k_sgs_cluster_smem without a cluster-wide barrier between
// colors.  Each CTA owns two mbarriers, used by alternate colors.  A row's
// warp sends the row's new u_i to every CTA's copy with remote stores that
// count their bytes on the receiving CTA's mbarrier of that color; each CTA
// expects exactly (rows of the color) x 3 values and waits only for them, so
// no CTA waits for a fence of all outstanding stores.  Ordering: a CTA starts
// color k+1 only after every row of color k, from every CTA, has arrived; the
// rows of color k were computed (and their neighbours read) before they were
// sent, so no value of color k+1 can overwrite one still to be read for
// color k, and a CTA is at most one color ahead of another, which the two
// alternating mbarriers cover.  Waits are bounded: past the scene's poll
// limit the timeout is recorded and the wait goes on (the bytes of a color
// always arrive), and past max(limit, 2^22) polls (each a hardware wait of
// about a microsecond at most) the CTA stops.
template <class T>
__global__ void __launch_bounds__(SW_NT, 1) k_sgs_cluster_tx(SweepPlan plan, const int4 *__restrict__ rec,
                                                             const int *__restrict__ cols, const T *__restrict__ vals,
                                                             const T *__restrict__ dinv, const T *__restrict__ b,
                                                             T *u, int n, int *err, long long spin_limit) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ int4 s_rec[54][SW_WARPS];
  __shared__ __align__(8) unsigned long long s_bar[2];
  extern __shared__ __align__(16) unsigned char sw_dyn[];
  T *su = reinterpret_cast<T *>(sw_dyn);
  const int G = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster.block_rank();
  const int first = blockIdx.x + G * warp;
  for (int k = lane; k < plan.steps; k += 32) {
    int4 rr = first < plan.nr[k] ? rec[plan.off[k] + first] : make_int4(-1, 0, 0, 0);
    if (k >= plan.low_steps) rr.w = rr.z;
    s_rec[k][warp] = rr;
  }
  for (int k = threadIdx.x; k < 3 * n; k += SW_NT) su[k] = u[k];
  const uint32_t bar0 = smem_addr(&s_bar[0]), bar1 = smem_addr(&s_bar[1]);
  if (threadIdx.x == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    mbar_init_fence();
  }
  // every CTA's barriers are initialised and its copy loaded before any remote store
  cluster.sync();
  // lanes < G send to CTA `lane`: its copy of u and its two barriers
  uint32_t dst_u = 0, dst_b0 = 0, dst_b1 = 0;
  if (lane < G) {
    dst_u = cluster_addr(smem_addr(su), (uint32_t)lane);
    dst_b0 = cluster_addr(bar0, (uint32_t)lane);
    dst_b1 = cluster_addr(bar1, (uint32_t)lane);
  }
  const long long hard = spin_limit > (1ll << 22) ? spin_limit : (1ll << 22);
  bool live = true;
  RowRegs<T> R;
  {
    const int4 r0 = s_rec[0][warp];
    if (r0.x >= 0) load_row<T>(R, r0.x, r0.y, r0.z, r0.w, lane, cols, vals, dinv, b);
  }
  for (int k = 0; k < plan.steps; ++k) {
    const uint32_t bar = (k & 1) ? bar1 : bar0;
    if (threadIdx.x == 0 && live) mbar_expect_tx(bar, (uint32_t)(plan.nr[k] * 3 * (int)sizeof(T)));
    const int4 r = s_rec[k][warp];
    if (r.x >= 0) {   // warp-uniform
      const T val = row_new_u<T, false>(R, r.x, r.y, r.z, r.w, lane, cols, vals, su);
      const T w0 = __shfl_sync(0xffffffffu, val, 0), w1 = __shfl_sync(0xffffffffu, val, 1),
              w2 = __shfl_sync(0xffffffffu, val, 2);
      if (lane < G && live) {
        const uint32_t a = dst_u + (uint32_t)(3 * r.x * (int)sizeof(T)), mb = (k & 1) ? dst_b1 : dst_b0;
        st_async_tx(a, w0, mb);
        st_async_tx(a + (uint32_t)sizeof(T), w1, mb);
        st_async_tx(a + 2u * (uint32_t)sizeof(T), w2, mb);
      }
    }
    if (k + 1 < plan.steps) {   // the next color's row does not depend on u: load it while waiting
      const int4 rn = s_rec[k + 1][warp];
      if (rn.x >= 0) load_row<T>(R, rn.x, rn.y, rn.z, rn.w, lane, cols, vals, dinv, b);
    }
    if (live) {
      const uint32_t parity = (uint32_t)((k >> 1) & 1);
      long long spins = 0;
      while (!mbar_try_wait_cluster(bar, parity, 1000u)) {
        ++spins;
        if (spins == spin_limit && threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
        if (spins > hard) {
          live = false;
          atomicOr(err, DEV_ERR_TIMEOUT);
          break;
        }
      }
    }
  }
  // every CTA has received every value (no store is in flight); no CTA
  // touches another's shared memory after this
  cluster.sync();
  for (int k = rank * SW_NT + threadIdx.x; k < 3 * n; k += G * SW_NT) u[k] = su[k];
}

template <class T>
__global__ void __launch_bounds__(NT) k_coarse_pcg(int64_t n, const int *__restrict__ row_ptr, const int *__restrict__ cols,
                                                   const T *__restrict__ vals, const T *__restrict__ diag,
                                                   const T *__restrict__ b, T *x, T *r, T *z, T *p, T *Ap,
                                                   double *part, unsigned *bar, int *log, int *log_idx, int log_cap,
                                                   int *err, double tau, int max_iter, long long spin_limit) {
  __shared__ double sh[NT];
  unsigned gen = 0;
  const int64_t n3 = 3 * n;
  const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x, gstride = (int64_t)gridDim.x * NT;
  const int G = gridDim.x;
  double *partA = part, *partB = part + G;
  // x = 0, r = b, z = D^-1 r, p = z, partial r^T z
  double acc = 0.0;
  for (int64_t k = gtid; k < n3; k += gstride) {
    T bk = b[k];
    x[k] = T(0);
    r[k] = bk;
    T zk = bk / diag[k];
    z[k] = zk;
    p[k] = zk;
    acc += (double)bk * (double)zk;
  }
  double t = block_sum<NT>(acc, sh);
  if (threadIdx.x == 0) partA[blockIdx.x] = t;
  if (!grid_sync(bar, gen, err, spin_limit)) return;
  double rz = sum_partials<NT>(partA, G, sh);
  const double bn = sqrt(fmax(rz, 0.0));
  // in float32 a relative residual below ~1e-3 is not reliably reachable;
  // the floor keeps the (preconditioning) coarse solve from running to its cap
  const double kk = fmax(fmin(0.5, sqrt(fmax(bn, tau))), sizeof(T) == 4 ? 1e-3 : 0.0);
  int it = 0;
  while (true) {
    if (sqrt(fmax(rz, 0.0)) <= kk * bn || it >= max_iter) break;
    // Ap = H p, partial p^T Ap
    acc = 0.0;
    const int64_t warps = (int64_t)G * (NT / 32);
    for (int64_t w0 = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5); w0 * RPW < n; w0 += warps) {
      const int64_t i = w0 * RPW + ((threadIdx.x & 31) / RL);
      const bool valid = i < n;
      T a3[3];
      row_product<T>(i, valid, threadIdx.x % RL, row_ptr, cols, vals, p, false, a3);
      if (valid && (threadIdx.x % RL) == 0) {
        Ap[3 * i] = a3[0];
        Ap[3 * i + 1] = a3[1];
        Ap[3 * i + 2] = a3[2];
        acc += (double)p[3 * i] * (double)a3[0] + (double)p[3 * i + 1] * (double)a3[1] +
               (double)p[3 * i + 2] * (double)a3[2];
      }
    }
    t = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) partB[blockIdx.x] = t;
    if (!grid_sync(bar, gen, err, spin_limit)) return;
    double pAp = sum_partials<NT>(partB, G, sh);
    if (!(pAp > 0.0)) break;
    const double alpha = rz / pAp;
    acc = 0.0;
    for (int64_t k = gtid; k < n3; k += gstride) {
      T xk = x[k] + (T)alpha * p[k];
      T rk = r[k] - (T)alpha * Ap[k];
      x[k] = xk;
      r[k] = rk;
      T zk = rk / diag[k];
      z[k] = zk;
      acc += (double)rk * (double)zk;
    }
    t = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) partA[blockIdx.x] = t;
    if (!grid_sync(bar, gen, err, spin_limit)) return;
    double rz_new = sum_partials<NT>(partA, G, sh);
    const double beta = rz_new / rz;
    rz = rz_new;
    for (int64_t k = gtid; k < n3; k += gstride) p[k] = z[k] + (T)beta * p[k];
    ++it;
    if (!grid_sync(bar, gen, err, spin_limit)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int k = *log_idx;
    if (k < log_cap) log[k] = it;
    *log_idx = k + 1;
  }
}

// ---------------------------------------------------------------------------
// Coarsest level on one thread-block cluster of `cl` CTAs (16 where the part
// allows a non-portable cluster of that size, else 8): the level's rows are
// split over the CTAs by block count and kept in their shared memory.  Same
// Jacobi-PCG iteration and stopping rule as k_coarse_pcg, two hardware cluster
// barriers per iteration:
//   1. each CTA forms Ap and the partial p^T Ap of its rows and writes the
//      partial into every CTA's shared memory (distributed shared memory);
//   2. after the barrier, each CTA updates x, r, z of its rows, writes its
//      slice of z and its partial r^T z into every CTA; after the second
//      barrier every CTA forms the whole of p = z + beta p locally.
// The scalar arithmetic (sums of the cluster's partials in rank order, alpha,
// beta, the stopping test) runs in one thread and is read from shared
// memory: FP64 instructions are scarce on this part (2 FMA per clock per SM),
// and repeating them in every thread cost more than the iteration's work.
// Reductions skip the warps whose lanes hold no term.
// ---------------------------------------------------------------------------
constexpr int CLMAX = 16;
constexpr int CNT = 512;
constexpr int CNW = CNT / 32;
constexpr size_t CL_SMEM_MAX = 200 * 1024;
struct ClusterPlan {
  int bounds[CLMAX + 1];
};

// Sum over the CTA of per-warp values held in lane 0 of each warp; the total
// is returned to every lane of warp 0 (fixed order, so bitwise reproducible).
__device__ __forceinline__ double cta_sum_lane0(double v, double *ws) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < CNW ? ws[lane] : 0.0;
#pragma unroll
    for (int o = CNW / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    t = __shfl_sync(0xffffffffu, t, 0);
  }
  return t;
}

// Sum over the CTA of per-thread values that are zero in threads >= nz.
__device__ __forceinline__ double cta_sum_first(double v, int nz, double *ws) {
  const int warp = threadIdx.x >> 5;
  if (warp * 32 < nz) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  } else {
    v = 0.0;
  }
  return cta_sum_lane0(v, ws);
}

template <class T, class V>
__global__ void __launch_bounds__(CNT) k_coarse_pcg_cluster(int R, const int *__restrict__ row_ptr,
                                                            const int *__restrict__ gcols,
                                                            const T *__restrict__ gvals,
                                                            const T *__restrict__ gdiag, const T *__restrict__ b,
                                                            T *__restrict__ xout, ClusterPlan plan, int rows_max,
                                                            int nb_max, double tau, int max_iter, int *log,
                                                            int *log_idx, int log_cap) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ double ws[CNW];
  __shared__ double s_alpha, s_beta;
  __shared__ int s_stop;
  extern __shared__ __align__(16) unsigned char sm[];
  const int cl = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  double *redP = reinterpret_cast<double *>(sm);   // partials p^T Ap, by rank
  double *redR = redP + CLMAX;                     // partials r^T z, by rank
  V *pfull = reinterpret_cast<V *>(redR + CLMAX);
  V *zfull = pfull + 3 * R;
  V *x = zfull + 3 * R;
  V *r = x + 3 * rows_max;
  V *Ap = r + 3 * rows_max;
  V *dg = Ap + 3 * rows_max;
  V *vals = dg + 3 * rows_max;   // converted to V once, as the level is staged
  int *rptr = reinterpret_cast<int *>(vals + 9 * (int64_t)nb_max);
  int *cols = rptr + rows_max + 1;
  const int r0 = plan.bounds[rank], r1 = plan.bounds[rank + 1], nr = r1 - r0;
  const int g0 = row_ptr[r0], nbl = row_ptr[r1] - g0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cluster.sync();   // every CTA of the cluster is running before any remote access
  for (int k = threadIdx.x; k <= nr; k += CNT) rptr[k] = row_ptr[r0 + k] - g0;
#pragma unroll 4
  for (int k = threadIdx.x; k < nbl; k += CNT) cols[k] = gcols[g0 + k];
#pragma unroll 8
  for (int k = threadIdx.x; k < 9 * nbl; k += CNT) vals[k] = (V)gvals[9 * (int64_t)g0 + k];
  // x = 0, r = b, z = D^-1 r (slices to every CTA), partial r^T z
  double acc = 0.0;
  for (int k = threadIdx.x; k < 3 * nr; k += CNT) {
    const V d = (V)gdiag[3 * r0 + k], bk = (V)b[3 * r0 + k];
    dg[k] = d;
    x[k] = V(0);
    r[k] = bk;
    const V zk = bk / d;
    for (int dst = 0; dst < cl; ++dst) cluster.map_shared_rank(zfull, dst)[3 * r0 + k] = zk;
    acc += (double)bk * (double)zk;
  }
  double t = cta_sum_first(acc, 3 * nr, ws);
  if (warp == 0 && lane < cl) cluster.map_shared_rank(redR, lane)[rank] = t;
  cluster.sync();
  // rz, |b|_D, the tolerance k and the stopping test: one thread
  double rz = 0.0, bn = 0.0, kk = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < cl; ++k) rz += redR[k];
    bn = sqrt(fmax(rz, 0.0));
    // in float32 arithmetic a relative residual below ~1e-3 is not reliably reachable
    kk = fmax(fmin(0.5, sqrt(fmax(bn, tau))), sizeof(V) == 4 ? 1e-3 : 0.0);
    s_stop = (sqrt(fmax(rz, 0.0)) <= kk * bn || max_iter <= 0) ? 1 : 0;
  }
  for (int k = threadIdx.x; k < 3 * R; k += CNT) pfull[k] = zfull[k];   // p = z
  __syncthreads();
  int it = 0;
  while (!s_stop) {
    // Ap = H p on this CTA's rows, partial p^T Ap (lanes 0, 8, 16 hold the
    // three components of a row after the split warp sum)
    double accw = 0.0;
    for (int i = warp; i < nr; i += CNW) {
      V a3[3];
      row_partial<V, V>(i, true, lane, rptr, cols, vals, pfull, false, a3);
      const V sc = warp_sum3_split<V>(a3, lane);
      if ((lane & 7) == 0 && lane < 24) {
        const int c = lane >> 3;
        Ap[3 * i + c] = sc;
        accw += (double)pfull[3 * (r0 + i) + c] * (double)sc;
      }
    }
    if (warp < nr) accw += __shfl_down_sync(0xffffffffu, accw, 8) + __shfl_down_sync(0xffffffffu, accw, 16);
    t = cta_sum_lane0(accw, ws);
    if (warp == 0 && lane < cl) cluster.map_shared_rank(redP, lane)[rank] = t;
    cluster.sync();
    if (threadIdx.x == 0) {
      double pAp = 0.0;
      for (int k = 0; k < cl; ++k) pAp += redP[k];
      s_stop = (pAp > 0.0) ? 0 : 1;
      s_alpha = rz / pAp;
    }
    __syncthreads();
    if (s_stop) break;
    const V alpha = (V)s_alpha;
    acc = 0.0;
    for (int k = threadIdx.x; k < 3 * nr; k += CNT) {
      x[k] += alpha * pfull[3 * r0 + k];
      const V rk = r[k] - alpha * Ap[k];
      r[k] = rk;
      const V zk = rk / dg[k];
      for (int dst = 0; dst < cl; ++dst) cluster.map_shared_rank(zfull, dst)[3 * r0 + k] = zk;
      acc += (double)rk * (double)zk;
    }
    t = cta_sum_first(acc, 3 * nr, ws);
    if (warp == 0 && lane < cl) cluster.map_shared_rank(redR, lane)[rank] = t;
    cluster.sync();
    ++it;
    if (threadIdx.x == 0) {
      double rz_new = 0.0;
      for (int k = 0; k < cl; ++k) rz_new += redR[k];
      s_beta = rz_new / rz;
      rz = rz_new;
      s_stop = (sqrt(fmax(rz, 0.0)) <= kk * bn || it >= max_iter) ? 1 : 0;
    }
    __syncthreads();
    const V beta = (V)s_beta;
    for (int k = threadIdx.x; k < 3 * R; k += CNT) pfull[k] = zfull[k] + beta * pfull[k];
    __syncthreads();
  }
  for (int k = threadIdx.x; k < 3 * nr; k += CNT) xout[3 * r0 + k] = (T)x[k];
  if (rank == 0 && threadIdx.x == 0) {
    int k = *log_idx;
    if (k < log_cap) log[k] = it;
    *log_idx = k + 1;
  }
  cluster.sync();   // no CTA leaves while another may still address its shared memory
}

template <class T>
int coop_blocks() {
  static std::atomic<int> cached{-1};
  int c = cached.load();
  if (c < 0) {
    int per_sm = 0;
    HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_pcg<T>, NT, 0));
    int dev = 0, nsm = 0;
    HOT_CUDA(cudaGetDevice(&dev));
    HOT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    c = std::max(1, per_sm * nsm);
    cached.store(c);
  }
  return c;
}
}  // namespace

// ---------------------------------------------------------------------------
void build_pattern0(Scene &s) {
  Topo &t = s.topo[0];
  const int64_t n = t.n;
  t.mask.ensure(4 * (size_t)n + 4);
  t.rowcnt.ensure(n + 1);
  t.nlow.ensure(n + 1);
  t.row_ptr.ensure(n + 1);
  t.slotpos.ensure((size_t)NSLOT * n + NSLOT);
  if (n == 0) {
    t.nnzb = 0;
    HOT_CUDA(cudaMemsetAsync(t.row_ptr.p, 0, sizeof(int), s.st));
    return;
  }
  unsigned nbw = (unsigned)((n + WPB - 1) / WPB);
  k_pattern0<<<nbw, NT, 0, s.st>>>(n, t.coords.p, t.map.p, dims_of(t), s.cell_count.p, s.geo.nb[0], s.geo.nb[1],
                                   s.geo.nb[2], s.geo.dims[0], s.geo.dims[1], s.geo.dims[2], t.mask.p, t.rowcnt.p);
  HOT_LAUNCH("k_pattern0");
  HOT_CUDA(cudaMemsetAsync(t.rowcnt.p + n, 0, sizeof(int), s.st));
  exclusive_scan(t.rowcnt.p, t.row_ptr.p, n + 1, s.scan, s.st);
  t.nnzb = read_scan_total(s.scan, s.st);
  t.cols.ensure(t.nnzb);
  k_fill_pattern<<<nbw, NT, 0, s.st>>>(n, t.coords.p, t.map.p, dims_of(t), t.mask.p, t.row_ptr.p, t.cols.p,
                                       t.slotpos.p, t.nlow.p);
  HOT_LAUNCH("k_fill_pattern");
}

void build_coarse_topology(Scene &s, int m) {
  Topo &F = s.topo[m];
  Topo &C = s.topo[m + 1];
  for (int k = 0; k < 3; ++k) C.dims[k] = F.dims[k] / 2 + 1;
  int64_t ntot = (int64_t)C.dims[0] * C.dims[1] * C.dims[2];
  C.flag.ensure(ntot, 1.0);
  C.map.ensure(ntot, 1.0);
  HOT_CUDA(cudaMemsetAsync(C.flag.p, 0, ntot, s.st));
  if (F.n > 0) {
    k_mark_coarse<<<(unsigned)((F.n + NT - 1) / NT), NT, 0, s.st>>>(F.n, F.coords.p, dims_of(C), C.flag.p);
    HOT_LAUNCH("k_mark_coarse");
  }
  compact_dense(s, C);
  const int64_t n = C.n;
  C.mask.ensure(4 * (size_t)n + 4);
  C.rowcnt.ensure(n + 1);
  C.nlow.ensure(n + 1);
  C.row_ptr.ensure(n + 1);
  C.slotpos.ensure((size_t)NSLOT * n + NSLOT);
  if (n == 0) {
    C.nnzb = 0;
    return;
  }
  unsigned nbw = (unsigned)((n + WPB - 1) / WPB);
  k_pattern_rap<<<nbw, NT, 0, s.st>>>(n, C.coords.p, F.map.p, dims_of(F), F.coords.p, F.row_ptr.p, F.cols.p, C.mask.p,
                                      C.rowcnt.p);
  HOT_LAUNCH("k_pattern_rap");
  HOT_CUDA(cudaMemsetAsync(C.rowcnt.p + n, 0, sizeof(int), s.st));
  exclusive_scan(C.rowcnt.p, C.row_ptr.p, n + 1, s.scan, s.st);
  C.nnzb = read_scan_total(s.scan, s.st);
  C.cols.ensure(C.nnzb);
  k_fill_pattern<<<nbw, NT, 0, s.st>>>(n, C.coords.p, C.map.p, dims_of(C), C.mask.p, C.row_ptr.p, C.cols.p,
                                       C.slotpos.p, C.nlow.p);
  HOT_LAUNCH("k_fill_pattern");
}

void build_colors(Scene &s, int m) {
  Topo &t = s.topo[m];
  t.color_cnt.ensure(28);
  t.color_list.ensure(t.n + 1);
  t.color_rec.ensure(t.n + 1);
  HOT_CUDA(cudaMemsetAsync(t.color_cnt.p, 0, sizeof(int) * 28, s.st));
  if (t.n == 0) {
    for (int c = 0; c < 28; ++c) t.color_off[c] = 0;
    return;
  }
  unsigned nb = (unsigned)((t.n + NT - 1) / NT);
  k_color_count<<<nb, NT, 0, s.st>>>(t.n, t.coords.p, t.color_cnt.p);
  HOT_LAUNCH("k_color_count");
  int cnt[28];
  HOT_CUDA(cudaMemcpyAsync(cnt, t.color_cnt.p, sizeof(int) * 27, cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  t.color_off[0] = 0;
  for (int c = 0; c < 27; ++c) t.color_off[c + 1] = t.color_off[c] + cnt[c];
  HOT_CUDA(cudaMemcpyAsync(t.color_cnt.p, t.color_off, sizeof(int) * 27, cudaMemcpyHostToDevice, s.st));
  k_color_fill<<<nb, NT, 0, s.st>>>(t.n, t.coords.p, t.color_cnt.p, t.color_list.p);
  HOT_LAUNCH("k_color_fill");
  k_color_records<<<nb, NT, 0, s.st>>>(t.n, t.color_list.p, t.row_ptr.p, t.nlow.p, t.color_rec.p);
  HOT_LAUNCH("k_color_records");
  HOT_CUDA(cudaStreamSynchronize(s.st));   // color_off (host) must outlive the async copy
}

template <class T>
void rap(Scene &s, Hier<T> &h, int m) {
  Topo &F = s.topo[m];
  Topo &C = s.topo[m + 1];
  Vals<T> &VC = h.L[m + 1];
  VC.vals.ensure(9 * (size_t)C.nnzb + 9);
  if (C.n == 0) return;
  h.rap_t.ensure((size_t)9 * RAP_WIN * F.n + 9 * RAP_WIN);
  ProfScope prof_(s, "rap");
  k_rap_t<T><<<(unsigned)((F.n + WPB - 1) / WPB), NT, 0, s.st>>>(F.n, F.coords.p, F.row_ptr.p, F.slotpos.p,
                                                                h.L[m].vals.p, h.rap_t.p);
  HOT_LAUNCH("k_rap_t");
  k_rap_r<T><<<(unsigned)C.n, 128, 0, s.st>>>(C.n, C.coords.p, C.row_ptr.p, C.slotpos.p, VC.vals.p, F.map.p,
                                              dims_of(F), h.rap_t.p);
  HOT_LAUNCH("k_rap_r");
}

template <class T>
void finalize_values(Scene &s, Hier<T> &h, int m) {
  Topo &t = s.topo[m];
  Vals<T> &V = h.L[m];
  V.dinv.ensure(9 * (size_t)t.n + 9);
  V.diag.ensure(3 * (size_t)t.n + 3);
  V.u.ensure(3 * (size_t)t.n + 3);
  V.b.ensure(3 * (size_t)t.n + 3);
  V.r.ensure(3 * (size_t)t.n + 3);
  if (t.n == 0) return;
  k_diag<T><<<(unsigned)((t.n + NT - 1) / NT), NT, 0, s.st>>>(t.n, t.row_ptr.p, t.slotpos.p, V.vals.p, V.dinv.p,
                                                              V.diag.p);
  HOT_LAUNCH("k_diag");
}

namespace {
const char *const SWEEP_SCOPE[8] = {"sgs_l0", "sgs_l1", "sgs_l2", "sgs_l3", "sgs_l4", "sgs_l5", "sgs_l6", "sgs_l7"};

template <class T>
int persistent_blocks() {
  static std::atomic<int> cached{-1};
  int c = cached.load();
  if (c < 0) {
    int per_sm = 0, dev = 0, nsm = 0;
    int per_sm_multi = 0;
    HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sgs_persistent<T, false>, SW_NT, 0));
    HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_multi, k_sgs_persistent<T, true>, SW_NT, 0));
    per_sm = std::min(per_sm, per_sm_multi);
    HOT_CUDA(cudaGetDevice(&dev));
    HOT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    c = std::max(1, std::min(per_sm, 1) * nsm);   // one block per SM
    cached.store(c);
  }
  return c;
}

// CTAs of the cluster that runs the sweeps of small levels: 16 where a
// non-portable cluster of that size can be resident, else 8 (0: none).
// Row limits (largest color of the level), measured per level on the two-bar
// scenes against the grid-barrier sweep: with u in global memory the cluster
// sweep wins up to a few dozen FP64 rows per color; with u in shared memory
// and byte counts between colors (k_sgs_cluster_tx) FP64 levels win up to
// ~160 rows per color (135: 20% faster; 234: 50% slower, the FP64 pipe of 16
// SMs) and FP32 levels up to the cluster's 256 warps (234: 15% faster); with
// the cluster barrier between colors (k_sgs_cluster_smem) FP32 levels win up
// to ~200 rows (135: 11% faster; 234: 6% slower).
constexpr int CLUSTER_SWEEP_ROWS = 64;
constexpr int CLUSTER_SWEEP_ROWS_SMEM = 160;      // FP64, u in shared memory
constexpr int CLUSTER_SWEEP_ROWS_FP32 = 192;
constexpr int CLUSTER_SWEEP_ROWS_FP32_TX = 256;   // FP32, u in shared memory, byte counts between colors
template <class T>
int sweep_cluster_size() {
  static std::atomic<int> cached{-1};
  int c = cached.load();
  if (c < 0) {
    c = 0;
    if (cudaFuncSetAttribute(k_sgs_persistent<T, false, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess)
      cudaGetLastError();
    for (int cl : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cl);
      cfg.blockDim = dim3(SW_NT);
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cl;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_sgs_persistent<T, false, true>, &cfg) == cudaSuccess && n >= 1) {
        c = cl;
        break;
      }
      cudaGetLastError();
    }
    cached.store(c);
  }
  return c;
}

// Largest level vector (bytes of shared memory) that k_sgs_cluster_smem can
// hold with a cluster of sweep_cluster_size<T>() CTAs resident; 0: none.
template <class T>
size_t sweep_smem_limit() {
  static std::atomic<long long> cached{-1};
  long long c = cached.load();
  if (c < 0) {
    c = 0;
    const int cl = sweep_cluster_size<T>();
    // both shared-memory sweeps (barrier and transaction-count forms) must fit
    const void *kern[2] = {(const void *)k_sgs_cluster_smem<T>, (const void *)k_sgs_cluster_tx<T>};
    if (cl > 0) {
      for (const void *f : kern)
        if (cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
          cudaGetLastError();
      for (int kb : {192, 160, 128, 96, 64, 48}) {
        const int bytes = kb * 1024;
        bool fits = true;
        for (const void *f : kern) {
          if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
            cudaGetLastError();
            fits = false;
            break;
          }
          cudaLaunchConfig_t cfg = {};
          cfg.gridDim = dim3(cl);
          cfg.blockDim = dim3(SW_NT);
          cfg.dynamicSmemBytes = bytes;
          cudaLaunchAttribute attr[1];
          attr[0].id = cudaLaunchAttributeClusterDimension;
          attr[0].val.clusterDim.x = cl;
          attr[0].val.clusterDim.y = 1;
          attr[0].val.clusterDim.z = 1;
          cfg.attrs = attr;
          cfg.numAttrs = 1;
          int nc = 0;
          if (cudaOccupancyMaxActiveClusters(&nc, f, &cfg) != cudaSuccess || nc < 1) {
            cudaGetLastError();
            fits = false;
            break;
          }
        }
        if (fits) {
          c = bytes;
          break;
        }
      }
    }
    cached.store(c);
  }
  return (size_t)c;
}

template <class T>
void launch_sgs_persistent(Scene &s, Topo &t, Vals<T> &V, Hier<T> &h, const SweepPlan &plan, int max_rows) {
  // levels whose colors have few rows (the limits above): one cluster,
  // hardware cluster barriers between colors (flag bit 6 turns this off)
  const int CLR = sweep_cluster_size<T>();
  // the level's u in shared memory unless it does not fit (or flag bit 10)
  const size_t smem = 3 * (size_t)t.n * sizeof(T);
  const bool in_smem = !(s.opts.flags & 1024) && smem <= sweep_smem_limit<T>();
  const bool tx = in_smem && !(s.opts.flags & 2048);
  const int row_limit = sizeof(T) == 4 ? (tx ? CLUSTER_SWEEP_ROWS_FP32_TX : CLUSTER_SWEEP_ROWS_FP32)
                                       : in_smem ? CLUSTER_SWEEP_ROWS_SMEM : CLUSTER_SWEEP_ROWS;
  if (CLR > 0 && !(s.opts.flags & 64) && max_rows <= std::min(row_limit, CLR * SW_WARPS)) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CLR);
    cfg.blockDim = dim3(SW_NT);
    cfg.stream = s.st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CLR;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (in_smem) {
      cfg.dynamicSmemBytes = smem;
      if (!tx) {   // hardware cluster barrier between colors
        HOT_CUDA(cudaLaunchKernelEx(&cfg, k_sgs_cluster_smem<T>, plan, (const int4 *)t.color_rec.p,
                                    (const int *)t.cols.p, (const T *)V.vals.p, (const T *)V.dinv.p,
                                    (const T *)V.b.p, V.u.p, (int)t.n));
        note_launch("k_sgs_cluster_smem");
      } else {   // per-CTA transaction counts between colors
        HOT_CUDA(cudaLaunchKernelEx(&cfg, k_sgs_cluster_tx<T>, plan, (const int4 *)t.color_rec.p,
                                    (const int *)t.cols.p, (const T *)V.vals.p, (const T *)V.dinv.p,
                                    (const T *)V.b.p, V.u.p, (int)t.n, s.errflag.p, s.spin_limit));
        note_launch("k_sgs_cluster_tx");
      }
      return;
    }
    HOT_CUDA(cudaLaunchKernelEx(&cfg, k_sgs_persistent<T, false, true>, plan, (const int4 *)t.color_rec.p,
                                (const int *)t.cols.p, (const T *)V.vals.p, (const T *)V.dinv.p, (const T *)V.b.p,
                                V.u.p, (unsigned *)nullptr, s.errflag.p, s.spin_limit));
    note_launch("k_sgs_persistent");
    return;
  }
  // one block per SM at most, and no more blocks than the largest color has rows
  const int G = std::max(1, std::min(persistent_blocks<T>(), max_rows));
  unsigned *bar = h.bar.p + 2;
  HOT_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), s.st));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(SW_NT);
  cfg.stream = s.st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (max_rows > G * SW_WARPS)
    HOT_CUDA(cudaLaunchKernelEx(&cfg, k_sgs_persistent<T, true>, plan, (const int4 *)t.color_rec.p,
                                (const int *)t.cols.p, (const T *)V.vals.p, (const T *)V.dinv.p, (const T *)V.b.p,
                                V.u.p, bar, s.errflag.p, s.spin_limit));
  else
    HOT_CUDA(cudaLaunchKernelEx(&cfg, k_sgs_persistent<T, false>, plan, (const int4 *)t.color_rec.p,
                                (const int *)t.cols.p, (const T *)V.vals.p, (const T *)V.dinv.p, (const T *)V.b.p,
                                V.u.p, bar, s.errflag.p, s.spin_limit));
  note_launch("k_sgs_persistent");
}

// Symmetric Gauss-Seidel (Alg. 2): colors 0..26, then 26..0.  The backward
// sweep leaves out its first non-empty color: it is the forward sweep's last,
// and rows of one color are not coupled, so a second update in a row
// recomputes the same values from the same inputs.  Each sweep is one
// cooperative launch (one cluster launch on levels whose colors fit a
// cluster's warps); flag bit 2 makes it one launch per color on every
// level, bit 3 on the finest level only.
// from_zero: u = 0 on entry (pre-smoothing), so in the forward half a row's
// neighbours of later colors are still zero and only its prefix of earlier-
// colored neighbours is read; the skipped terms are exact zeros, so the result
// is bitwise that of the full rows.
template <class T>
void sgs_symmetric(Scene &s, Topo &t, Vals<T> &V, Hier<T> &h, int m, bool from_zero) {
  ProfScope sweep_(s, SWEEP_SCOPE[m & 7]);
  SweepPlan plan;
  plan.steps = 0;
  plan.low_steps = 0;
  int max_rows = 0;
  bool skipped = false;
  for (int k = 0; k < 54; ++k) {
    const bool forward = k < 27;
    const int c = forward ? k : 53 - k;
    const int nr = t.color_off[c + 1] - t.color_off[c];
    if (nr == 0) continue;
    if (!forward && !skipped) {
      skipped = true;
      continue;
    }
    plan.off[plan.steps] = t.color_off[c];
    plan.nr[plan.steps] = nr;
    plan.steps += 1;
    if (forward && from_zero) plan.low_steps = plan.steps;
    max_rows = std::max(max_rows, nr);
  }
  if (plan.steps == 0) return;
  const bool persistent = !(s.opts.flags & 4) && (m > 0 || !(s.opts.flags & 8));
  if (persistent) {
    ProfScope prof_(s, "sgs");
    launch_sgs_persistent<T>(s, t, V, h, plan, max_rows);
    return;
  }
  // rows (warps) per block of the per-color launches: options flag bits 8-9
  // (0: 8, 1: 2, 2: 4, 3: 16), picked by the batch autotuner
  const int wpb = sgs_color_warps(s.opts.flags);
  for (int k = 0; k < plan.steps; ++k) {
    ProfScope prof_(s, "sgs");
    k_sgs_color<T><<<(unsigned)((plan.nr[k] + wpb - 1) / wpb), 32 * wpb, 0, s.st>>>(
        t.color_rec.p + plan.off[k], plan.nr[k], t.cols.p, V.vals.p, V.dinv.p, V.b.p, V.u.p,
        k < plan.low_steps ? 1 : 0);
    HOT_LAUNCH("k_sgs_color");
  }
}

// Partition of the coarsest level over one cluster, computed once per
// hierarchy: 16 CTAs where a non-portable cluster of that size can be
// resident, else 8; cl_smem = 0 when the level does not fit either
// (cooperative fallback).
template <class T>
void plan_cluster(Scene &s, Hier<T> &h, int m) {
  Topo &t = s.topo[m];
  h.cl_level = m;
  h.cl_smem = 0;
  h.cl_size = 0;
  const int R = (int)t.n;
  if (R == 0) return;
  std::vector<int> rp(R + 1);
  HOT_CUDA(cudaMemcpyAsync(rp.data(), t.row_ptr.p, sizeof(int) * (R + 1), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  // set once, to the maximum: scenes planned on other threads launch the same kernel
  static std::once_flag once;
  std::call_once(once, [] {
    HOT_CUDA(cudaFuncSetAttribute(k_coarse_pcg_cluster<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CL_SMEM_MAX));
    if (cudaFuncSetAttribute(k_coarse_pcg_cluster<T, double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess)
      cudaGetLastError();
  });
  const int64_t B = rp[R];
  for (int cl : {CLMAX, 8}) {
    int bounds[CLMAX + 1];
    int r = 0;
    bounds[0] = 0;
    for (int c = 1; c < cl; ++c) {
      const int64_t target = B * c / cl;
      while (r < R && rp[r] < target) ++r;
      bounds[c] = r;
    }
    bounds[cl] = R;
    int rows_max = 0, nb_max = 0;
    for (int c = 0; c < cl; ++c) {
      rows_max = std::max(rows_max, bounds[c + 1] - bounds[c]);
      nb_max = std::max(nb_max, rp[bounds[c + 1]] - rp[bounds[c]]);
    }
    // vectors and the staged matrix values in FP64 whatever the hierarchy's precision
    const size_t bytes = 2 * CLMAX * sizeof(double) +
                         sizeof(double) * (6 * (size_t)R + 4 * 3 * (size_t)rows_max + 9 * (size_t)nb_max) +
                         sizeof(int) * ((size_t)rows_max + 1 + nb_max) + 64;
    if (bytes > CL_SMEM_MAX) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(CNT);
    cfg.dynamicSmemBytes = bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_pcg_cluster<T, double>, &cfg) != cudaSuccess ||
        nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    for (int c = 0; c <= cl; ++c) h.cl_bounds[c] = bounds[c];
    h.cl_size = cl;
    h.cl_rows_max = rows_max;
    h.cl_nb_max = nb_max;
    h.cl_smem = bytes;
    return;
  }
}

template <class T>
void coarse_solve(Scene &s, Hier<T> &h, int m) {
  Topo &t = s.topo[m];
  Vals<T> &V = h.L[m];
  int64_t nn = t.n;
  const int cap = (int)h.cg_log.cap;
  // Float32 coarse matrices of stiff scenes can lose definiteness to rounding,
  // where CG stalls short of its tolerance.  The cluster solver works in FP64
  // on the float32 matrix (its level is a few hundred rows in shared memory),
  // capped at 200 iterations; the cooperative fallback computes in float32,
  // capped at 100.
  const bool cluster = h.cl_smem > 0 && !(s.opts.flags & 2);
  const int max_iter = s.opts.max_coarse_cg > 0
                           ? s.opts.max_coarse_cg
                           : (int)(sizeof(T) == 4 ? std::min<int64_t>(3 * nn, cluster ? 200 : 100) : 3 * nn);
  if (cluster) {
    ClusterPlan plan;
    for (int c = 0; c <= h.cl_size; ++c) plan.bounds[c] = h.cl_bounds[c];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h.cl_size);
    cfg.blockDim = dim3(CNT);
    cfg.dynamicSmemBytes = h.cl_smem;
    cfg.stream = s.st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = h.cl_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ProfScope prof_(s, "coarse_pcg");
    HOT_CUDA(cudaLaunchKernelEx(&cfg, k_coarse_pcg_cluster<T, double>, (int)nn, (const int *)t.row_ptr.p,
                                (const int *)t.cols.p, (const T *)V.vals.p, (const T *)V.diag.p, (const T *)V.b.p,
                                V.u.p, plan, h.cl_rows_max, h.cl_nb_max, s.opts.eps, max_iter, h.cg_log.p,
                                h.cg_log.p + (cap - 1), cap - 1));
    note_launch("k_coarse_pcg_cluster");
    return;
  }
  int G = (int)((nn + WPB * RPW - 1) / (WPB * RPW));
  int maxb = coop_blocks<T>();
  if (G > maxb) G = maxb;
  if (G < 1) G = 1;
  HOT_CUDA(cudaMemsetAsync(h.bar.p, 0, 2 * sizeof(unsigned), s.st));
  double tau = s.opts.eps;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(NT);
  cfg.stream = s.st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ProfScope prof_(s, "coarse_pcg");
  HOT_CUDA(cudaLaunchKernelEx(&cfg, k_coarse_pcg<T>, nn, (const int *)t.row_ptr.p, (const int *)t.cols.p,
                              (const T *)V.vals.p, (const T *)V.diag.p, (const T *)V.b.p, V.u.p, h.r.p, h.z.p,
                              h.p.p, h.Ap.p, h.part.p, h.bar.p, h.cg_log.p, h.cg_log.p + (cap - 1), cap - 1,
                              s.errflag.p, tau, max_iter, s.spin_limit));
  note_launch("k_coarse_pcg");
}

template <class T>
void vcycle_launches(Scene &s, Hier<T> &h, const double *b_in, double *u_out) {
  const int M = s.nlev;
  Topo &t0 = s.topo[0];
  k_load_rhs<T><<<(unsigned)((3 * t0.n + NT - 1) / NT), NT, 0, s.st>>>(t0.n, b_in, s.fixed.p, h.L[0].b.p);
  HOT_LAUNCH("k_load_rhs");
  for (int m = 0; m < M - 1; ++m) {
    Topo &t = s.topo[m];
    Vals<T> &V = h.L[m];
    HOT_CUDA(cudaMemsetAsync(V.u.p, 0, sizeof(T) * 3 * t.n, s.st));
    sgs_symmetric<T>(s, t, V, h, m, true);
    if (s.opts.flags & 128) {
      ProfScope prof_(s, "residual");
      k_residual_diag<T><<<(unsigned)((t.n + NT - 1) / NT), NT, 0, s.st>>>(t.n, t.row_ptr.p, t.slotpos.p, V.vals.p,
                                                                          V.b.p, V.u.p, V.r.p);
      HOT_LAUNCH("k_residual_diag");
      k_residual_half<T><<<(unsigned)((t.n + WPB - 1) / WPB), NT, 0, s.st>>>(t.n, t.row_ptr.p, t.cols.p, t.nlow.p,
                                                                           V.vals.p, V.u.p, V.r.p);
      HOT_LAUNCH("k_residual_half");
    } else {
      ProfScope prof_(s, "residual");
      k_residual<T><<<(unsigned)((t.n + WPB - 1) / WPB), NT, 0, s.st>>>(
          t.n, t.row_ptr.p, t.cols.p, V.vals.p, V.b.p, V.u.p, V.r.p);
      HOT_LAUNCH("k_residual");
    }
    Topo &c = s.topo[m + 1];
    k_restrict<T><<<(unsigned)((c.n + NT - 1) / NT), NT, 0, s.st>>>(c.n, c.coords.p, t.map.p, dims_of(t), V.r.p,
                                                                     h.L[m + 1].b.p);
    HOT_LAUNCH("k_restrict");
  }
  coarse_solve<T>(s, h, M - 1);
  for (int m = M - 2; m >= 0; --m) {
    Topo &t = s.topo[m];
    Topo &c = s.topo[m + 1];
    Vals<T> &V = h.L[m];
    k_prolong_add<T><<<(unsigned)((t.n + NT - 1) / NT), NT, 0, s.st>>>(t.n, t.coords.p, c.map.p, dims_of(c),
                                                                       h.L[m + 1].u.p, V.u.p);
    HOT_LAUNCH("k_prolong_add");
    sgs_symmetric<T>(s, t, V, h, m, false);
  }
  k_store_out<T><<<(unsigned)((3 * t0.n + NT - 1) / NT), NT, 0, s.st>>>(t0.n, h.L[0].u.p, s.fixed.p, u_out);
  HOT_LAUNCH("k_store_out");
}
}  // namespace

// buffers the V-cycle touches, sized before any launch (and before capture)
template <class T>
void vcycle_prepare(Scene &s, Hier<T> &h) {
  const int64_t n = s.topo[s.nlev - 1].n;
  h.r.ensure(3 * n + 3);
  h.z.ensure(3 * n + 3);
  h.p.ensure(3 * n + 3);
  h.Ap.ensure(3 * n + 3);
  h.bar.ensure(4);
  h.cg_log.ensure(4097, 1.0);
  h.part.ensure(2 * (size_t)coop_blocks<T>() + 2);
  persistent_blocks<T>();   // occupancy queries and function attributes before any capture
  sweep_cluster_size<T>();
  sweep_smem_limit<T>();
  if (h.cl_level != s.nlev - 1) plan_cluster<T>(s, h, s.nlev - 1);
}

// Alg. 2 on b_in -> u_out.  The coarsest PCG appends its iteration count to
// the device log h.cg_log (read back with read_cg_log).  When the scene's
// stream allows it, the launch sequence (fixed for a hierarchy) is captured
// once into a CUDA graph and replayed.
template <class T>
void vcycle(Scene &s, Hier<T> &h, const double *b_in, double *u_out, bool use_graph) {
  if (s.topo[0].n == 0) return;
  vcycle_prepare<T>(s, h);
  ProfScope prof_(s, "vcycle");
  // profiling of kernels inside the V-cycle needs its eager launches
  const bool inner_prof = s.prof && (s.prof_only.empty() || prof_selected(s.prof_only, "sgs") ||
                                     prof_selected(s.prof_only, "residual") || prof_selected(s.prof_only, "coarse_pcg") ||
                                     prof_selected(s.prof_only, "sgs_l0"));
  if (use_graph && s.graphs_ok && !(s.opts.flags & 1) && !inner_prof) {
    if (s.vgraph && (s.vgraph_b != b_in || s.vgraph_u != u_out)) {
      cudaGraphExecDestroy(s.vgraph);
      s.vgraph = nullptr;
    }
    if (!s.vgraph) {
      cudaGraph_t g = nullptr;
      const long long c0 = launch_count();
      bool ok = cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        try {
          vcycle_launches<T>(s, h, b_in, u_out);
        } catch (const Error &) {
          ok = false;
        }
        cudaError_t e = cudaStreamEndCapture(s.st, &g);
        ok = ok && e == cudaSuccess && g != nullptr;
        if (ok) ok = cudaGraphInstantiate(&s.vgraph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();
      s.vgraph_kernels = launch_count() - c0;
      note_launches(-s.vgraph_kernels);   // captured, not run
      if (!ok) {
        s.vgraph = nullptr;
        s.graphs_ok = false;   // run eagerly from now on
      } else {
        s.vgraph_b = b_in;
        s.vgraph_u = u_out;
      }
    }
    if (s.vgraph) {
      HOT_CUDA(cudaGraphLaunch(s.vgraph, s.st));
      note_launches(s.vgraph_kernels);
      ++s.graph_launches;
      return;
    }
  }
  vcycle_launches<T>(s, h, b_in, u_out);
}

// The V-cycle's launches alone, into whatever the stream is doing (a
// capture of a larger graph included); vcycle_ready sizes its buffers and
// plans the coarsest solve beforehand (it may synchronize).
template <class T>
void vcycle_ready(Scene &s, Hier<T> &h) {
  if (s.topo[0].n > 0) vcycle_prepare<T>(s, h);
}
template <class T>
void vcycle_emit(Scene &s, Hier<T> &h, const double *b_in, double *u_out) {
  if (s.topo[0].n > 0) vcycle_launches<T>(s, h, b_in, u_out);
}

template <class T>
void reset_cg_log(Scene &s, Hier<T> &h) {
  h.cg_log.ensure(4097, 1.0);
  HOT_CUDA(cudaMemsetAsync(h.cg_log.p + (h.cg_log.cap - 1), 0, sizeof(int), s.st));
}

template <class T>
std::vector<int> read_cg_log(Scene &s, Hier<T> &h) {
  int cap = (int)h.cg_log.cap;
  int cnt = 0;
  HOT_CUDA(cudaMemcpyAsync(&cnt, h.cg_log.p + (cap - 1), sizeof(int), cudaMemcpyDeviceToHost, s.st));
  HOT_CUDA(cudaStreamSynchronize(s.st));
  int k = cnt < cap - 1 ? cnt : cap - 1;
  std::vector<int> out(k);
  if (k > 0) {
    HOT_CUDA(cudaMemcpyAsync(out.data(), h.cg_log.p, sizeof(int) * k, cudaMemcpyDeviceToHost, s.st));
    HOT_CUDA(cudaStreamSynchronize(s.st));
  }
  out.resize(cnt, -1);   // entries beyond the log capacity are unknown
  return out;
}

template void rap<double>(Scene &, Hier<double> &, int);
template void rap<float>(Scene &, Hier<float> &, int);
template void finalize_values<double>(Scene &, Hier<double> &, int);
template void finalize_values<float>(Scene &, Hier<float> &, int);
template void vcycle<double>(Scene &, Hier<double> &, const double *, double *, bool);
template void vcycle<float>(Scene &, Hier<float> &, const double *, double *, bool);
template void vcycle_ready<double>(Scene &, Hier<double> &);
template void vcycle_ready<float>(Scene &, Hier<float> &);
template void vcycle_emit<double>(Scene &, Hier<double> &, const double *, double *);
template void vcycle_emit<float>(Scene &, Hier<float> &, const double *, double *);
template void reset_cg_log<double>(Scene &, Hier<double> &);
template void reset_cg_log<float>(Scene &, Hier<float> &);
template std::vector<int> read_cg_log<double>(Scene &, Hier<double> &);
template std::vector<int> read_cg_log<float>(Scene &, Hier<float> &);

}  // namespace hot
