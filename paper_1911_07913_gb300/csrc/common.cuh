// Shared device helpers and internal declarations of the HOT library.
//
// Nothing here is exported; the C ABI lives in include/hot_mpm.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/hot_mpm.h"

namespace hot {

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
struct Error {
  mpm_status code;
  std::string msg;
};
[[noreturn]] void fail(mpm_status code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);
void note_launch(const char *what);   // error check + launch counter
#define HOT_CUDA(x) ::hot::check_cuda((x), #x)
#define HOT_LAUNCH(what) ::hot::note_launch(what)

// device-side status bits written by kernels, read by the host
enum : int {
  DEV_ERR_DOMAIN = 1,
  DEV_ERR_TIMEOUT = 2,
  DEV_ERR_NUMERIC = 4,
};

// ---------------------------------------------------------------------------
// device memory through the allocator hook
// ---------------------------------------------------------------------------
void *dev_alloc(size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);

template <class T>
struct DBuf {
  T *p = nullptr;
  size_t cap = 0;
  cudaStream_t st = nullptr;
  // grow to at least n elements (contents are not kept)
  void ensure(size_t n, double headroom = 1.25) {
    if (n <= cap && p) return;
    release();
    size_t want = n < 16 ? 16 : (size_t)(n * headroom) + 16;
    p = static_cast<T *>(dev_alloc(want * sizeof(T), st));
    cap = want;
  }
  void release() {
    if (p) dev_free(p, st);
    p = nullptr;
    cap = 0;
  }
  size_t bytes() const { return cap * sizeof(T); }
};

// ---------------------------------------------------------------------------
// scans and reductions (scan.cu)
// ---------------------------------------------------------------------------
struct ScanScratch {
  DBuf<int> block_sums;
  DBuf<int> total;
};
// exclusive prefix sum of n inputs (int or uint8) into out; *d_total (device)
// receives the sum.  out may alias in only for int input.
void exclusive_scan(const int *in, int *out, int64_t n, ScanScratch &sc, cudaStream_t st);
void exclusive_scan_u8(const uint8_t *in, int *out, int64_t n, ScanScratch &sc, cudaStream_t st);
int read_scan_total(ScanScratch &sc, cudaStream_t st);

constexpr int RED_THREADS = 256;

// ---------------------------------------------------------------------------
// kernel weights: quadratic B-spline along one axis (Sec. 3.1), fx in [1/2, 3/2)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void bspline_axis(T fx, T inv_dx, T w[3], T dw[3]) {
  T a = T(1.5) - fx, b = fx - T(1), c = fx - T(0.5);
  w[0] = T(0.5) * a * a;
  w[1] = T(0.75) - b * b;
  w[2] = T(0.5) * c * c;
  dw[0] = -a * inv_dx;
  dw[1] = T(-2) * b * inv_dx;
  dw[2] = c * inv_dx;
}

// Lowest stencil node along one axis: floor((x - o) * inv_dx - 1/2) with each
// operation rounded separately, so that every implementation agrees bit for bit.
__device__ __forceinline__ int base_axis(double x, double o, double inv_dx, double *fx) {
  double u = __dmul_rn(__dadd_rn(x, -o), inv_dx);
  double t = floor(__dadd_rn(u, -0.5));
  *fx = u - t;
  return (int)t;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ---------------------------------------------------------------------------
// small dense linear algebra
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void matmul3(const T *A, const T *B, T *C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

template <class T>
__device__ __forceinline__ T det3(const T *F) {
  return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
         F[2] * (F[3] * F[7] - F[4] * F[6]);
}

// cofactor matrix dJ/dF
template <class T>
__device__ __forceinline__ void cofactor3(const T *F, T *c) {
  c[0] = F[4] * F[8] - F[5] * F[7];
  c[1] = F[5] * F[6] - F[3] * F[8];
  c[2] = F[3] * F[7] - F[4] * F[6];
  c[3] = F[2] * F[7] - F[1] * F[8];
  c[4] = F[0] * F[8] - F[2] * F[6];
  c[5] = F[1] * F[6] - F[0] * F[7];
  c[6] = F[1] * F[5] - F[2] * F[4];
  c[7] = F[2] * F[3] - F[0] * F[5];
  c[8] = F[0] * F[4] - F[1] * F[3];
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (Golub & Van
// Loan, Sec. 8.5).  S (row-major, symmetric) is overwritten; on return
// ev[k] are eigenvalues and Q[:,k] (row-major Q[3*i+k]) the eigenvectors.
template <class T>
__device__ void jacobi_eig3(T *S, T ev[3], T *Q) {
#pragma unroll
  for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? T(1) : T(0);
  for (int sweep = 0; sweep < 12; ++sweep) {
    T off = S[1] * S[1] + S[2] * S[2] + S[5] * S[5];
    T diag = S[0] * S[0] + S[4] * S[4] + S[8] * S[8];
    if (off <= diag * T(sizeof(T) == 8 ? 1e-34 : 1e-16) || off == T(0)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      T apq = S[3 * p + q];
      if (apq == T(0)) continue;
      T app = S[3 * p + p], aqq = S[3 * q + q];
      T theta = (aqq - app) / (T(2) * apq);
      T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
      T c = T(1) / sqrt(t * t + T(1));
      T s = t * c;
      // S <- J^T S J with J the rotation in the (p, q) plane
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T skp = S[3 * k + p], skq = S[3 * k + q];
        S[3 * k + p] = c * skp - s * skq;
        S[3 * k + q] = s * skp + c * skq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T spk = S[3 * p + k], sqk = S[3 * q + k];
        S[3 * p + k] = c * spk - s * sqk;
        S[3 * q + k] = s * spk + c * sqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T qkp = Q[3 * k + p], qkq = Q[3 * k + q];
        Q[3 * k + p] = c * qkp - s * qkq;
        Q[3 * k + q] = s * qkp + c * qkq;
      }
    }
  }
  ev[0] = S[0];
  ev[1] = S[4];
  ev[2] = S[8];
}

template <class T>
__device__ __forceinline__ void swap_cols(T *Q, T *ev, int a, int b) {
  T t = ev[a];
  ev[a] = ev[b];
  ev[b] = t;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T q = Q[3 * k + a];
    Q[3 * k + a] = Q[3 * k + b];
    Q[3 * k + b] = q;
  }
}

// Signed SVD F = U diag(s) V^T with det U = det V = +1 and s0 >= s1 >= |s2|;
// s2 carries the sign of det F.  V from the eigenvectors of F^T F, U from a
// Gram-Schmidt QR of F V (the approach of McAdams et al. 2011 without their
// quaternion arithmetic).
template <class T>
__device__ void svd3(const T *F, T *U, T s[3], T *V) {
  T S[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) S[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
  T ev[3];
  jacobi_eig3(S, ev, V);
  if (ev[0] < ev[1]) swap_cols(V, ev, 0, 1);
  if (ev[0] < ev[2]) swap_cols(V, ev, 0, 2);
  if (ev[1] < ev[2]) swap_cols(V, ev, 1, 2);
  if (det3(V) < T(0)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) V[3 * k + 2] = -V[3 * k + 2];
  }
  T B[9];
  matmul3(F, V, B);
  const T tiny = T(sizeof(T) == 8 ? 1e-150 : 1e-30);
  // column 0
  T n0 = sqrt(B[0] * B[0] + B[3] * B[3] + B[6] * B[6]);
  T u0[3];
  if (n0 > tiny) {
    u0[0] = B[0] / n0; u0[1] = B[3] / n0; u0[2] = B[6] / n0;
  } else {
    u0[0] = T(1); u0[1] = T(0); u0[2] = T(0);
  }
  // column 1, orthogonalised against u0
  T d01 = u0[0] * B[1] + u0[1] * B[4] + u0[2] * B[7];
  T w1[3] = {B[1] - d01 * u0[0], B[4] - d01 * u0[1], B[7] - d01 * u0[2]};
  T n1 = sqrt(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2]);
  T u1[3];
  if (n1 > tiny) {
    u1[0] = w1[0] / n1; u1[1] = w1[1] / n1; u1[2] = w1[2] / n1;
  } else {
    // any unit vector orthogonal to u0
    T a[3] = {T(0), T(0), T(0)};
    int k = (fabs(u0[0]) < fabs(u0[1])) ? ((fabs(u0[0]) < fabs(u0[2])) ? 0 : 2) : ((fabs(u0[1]) < fabs(u0[2])) ? 1 : 2);
    a[k] = T(1);
    T d = u0[0] * a[0] + u0[1] * a[1] + u0[2] * a[2];
    T t[3] = {a[0] - d * u0[0], a[1] - d * u0[1], a[2] - d * u0[2]};
    T nt = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    u1[0] = t[0] / nt; u1[1] = t[1] / nt; u1[2] = t[2] / nt;
  }
  T u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2], u0[0] * u1[1] - u0[1] * u1[0]};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    U[3 * k + 0] = u0[k];
    U[3 * k + 1] = u1[k];
    U[3 * k + 2] = u2[k];
  }
  s[0] = u0[0] * B[0] + u0[1] * B[3] + u0[2] * B[6];
  s[1] = u1[0] * B[1] + u1[1] * B[4] + u1[2] * B[7];
  s[2] = u2[0] * B[2] + u2[1] * B[5] + u2[2] * B[8];
}

// ---------------------------------------------------------------------------
// materials
// ---------------------------------------------------------------------------
struct MatParams {
  double mu, lam, xi, yield;
  int model;    // 0 FCR, 1 NH
  int plastic;  // 0 none, 1 von Mises, 2 snow clamp
};

// Lagged plastic projection of F after the F update (once per step):
// 1 von Mises on the principal Hencky strains e = ln s, deviatoric part d
//   scaled onto 2 mu |d| = yield when it exceeds it (det F unchanged);
// 2 singular values clamped into [0.99, 1.001].  F unchanged otherwise.
__device__ inline void plastic_project(double *F, double mu, double yield, int type) {
  if (type == 0) return;
  double U[9], s[3], V[9];
  svd3<double>(F, U, s, V);
  double sn[3];
  if (type == 1) {
    double e[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) e[k] = log(fmax(s[k], 1e-300));
    const double mean = (e[0] + e[1] + e[2]) / 3.0;
    const double d0 = e[0] - mean, d1 = e[1] - mean, d2 = e[2] - mean;
    const double nd = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (!(2.0 * mu * nd > yield)) return;
    const double sc = yield / fmax(2.0 * mu * nd, 1e-300);
    sn[0] = exp(mean + d0 * sc);
    sn[1] = exp(mean + d1 * sc);
    sn[2] = exp(mean + d2 * sc);
  } else {
    bool changed = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sn[k] = fmin(fmax(s[k], 0.99), 1.001);
      changed = changed || sn[k] != s[k];
    }
    if (!changed) return;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      F[3 * i + j] = U[3 * i] * sn[0] * V[3 * j] + U[3 * i + 1] * sn[1] * V[3 * j + 1] + U[3 * i + 2] * sn[2] * V[3 * j + 2];
}

// energy density; +inf for Neo-Hookean with J <= 0
template <class T>
__device__ T psi_density(const T *F, T mu, T lam, int model) {
  T J = det3(F);
  if (model == 0) {
    T U[9], s[3], V[9];
    svd3(F, U, s, V);
    T a = s[0] - T(1), b = s[1] - T(1), c = s[2] - T(1);
    return mu * (a * a + b * b + c * c) + T(0.5) * lam * (J - T(1)) * (J - T(1));
  }
  if (!(J > T(0))) return T(INFINITY);
  T lnJ = log(J);
  T tr = T(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) tr += F[k] * F[k];
  return T(0.5) * mu * (tr - T(3)) - mu * lnJ + T(0.5) * lam * lnJ * lnJ;
}

// first Piola-Kirchhoff stress
template <class T>
__device__ void piola(const T *F, T mu, T lam, int model, T *P) {
  T c[9];
  cofactor3(F, c);
  T J = det3(F);
  if (model == 0) {
    T U[9], s[3], V[9];
    svd3(F, U, s, V);
    T k = lam * (J - T(1));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T r = U[3 * i] * V[3 * j] + U[3 * i + 1] * V[3 * j + 1] + U[3 * i + 2] * V[3 * j + 2];
        P[3 * i + j] = T(2) * mu * (F[3 * i + j] - r) + k * c[3 * i + j];
      }
    return;
  }
  T lnJ = log(J);
  T k = (lam * lnJ - mu) / J;
#pragma unroll
  for (int i = 0; i < 9; ++i) P[i] = mu * F[i] + k * c[i];
}

// Projected stiffness d^2 psi/dF^2 (Teran et al. 2005): in the SVD frame the
// 9x9 matrix splits into a 3x3 block over the singular values and three 2x2
// blocks whose eigenvectors are the "flip" (E_ij + E_ji)/sqrt2 and "twist"
// (E_ij - E_ji)/sqrt2 directions; every eigenvalue is clamped at zero and the
// matrix rebuilt.  Output: the 45 entries of the upper triangle, row-major
// over the 9x9 index (3a+b).
template <class T>
__device__ void projected_stiffness(const T *F, T mu, T lam, int model, T *A45) {
  T U[9], s[3], V[9];
  svd3(F, U, s, V);
  T J = s[0] * s[1] * s[2];
  T Hs[9], lam_flip[3], lam_twist[3];
  const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2}, pk[3] = {2, 1, 0};
  if (model == 0) {
    // psi^ = mu sum (s - 1)^2 + lam/2 (J - 1)^2
    T dJ[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T v = lam * dJ[i] * dJ[j];
        if (i == j) v += T(2) * mu;
        else v += lam * (J - T(1)) * s[3 - i - j];
        Hs[3 * i + j] = v;
      }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      T sk = s[pk[q]];
      lam_flip[q] = T(2) * mu - lam * (J - T(1)) * sk;
      T den = s[pi[q]] + s[pj[q]];
      T floor_den = T(sizeof(T) == 8 ? 1e-12 : 1e-6);
      if (den < floor_den) den = floor_den;
      lam_twist[q] = T(2) * mu - T(4) * mu / den + lam * (J - T(1)) * sk;
    }
  } else {
    // psi^ = mu/2 (sum s^2 - 3) - mu ln J + lam/2 (ln J)^2
    T lnJ = J > T(0) ? log(J) : T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T v = lam / (s[i] * s[j]);
        if (i == j) v += mu + (mu - lam * lnJ) / (s[i] * s[i]);
        Hs[3 * i + j] = v;
      }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      T ss = s[pi[q]] * s[pj[q]];
      lam_flip[q] = mu + (mu - lam * lnJ) / ss;
      lam_twist[q] = mu + (lam * lnJ - mu) / ss;
    }
  }
  T ev[3], Q[9];
  jacobi_eig3(Hs, ev, Q);
#pragma unroll
  for (int k = 0; k < 45; ++k) A45[k] = T(0);
  T D[9];
  // 3x3 block modes: D = U diag(Q[:,k]) V^T
  for (int k = 0; k < 3; ++k) {
    T l = ev[k] > T(0) ? ev[k] : T(0);
    if (l == T(0)) continue;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        D[3 * a + b] = U[3 * a] * Q[k] * V[3 * b] + U[3 * a + 1] * Q[3 + k] * V[3 * b + 1] +
                       U[3 * a + 2] * Q[6 + k] * V[3 * b + 2];
    int idx = 0;
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
      for (int c = r; c < 9; ++c) A45[idx++] += l * D[r] * D[c];
  }
  const T inv_sqrt2 = T(0.70710678118654752440);
  for (int q = 0; q < 3; ++q) {
    int i = pi[q], j = pj[q];
    for (int mode = 0; mode < 2; ++mode) {
      T l = mode == 0 ? lam_flip[q] : lam_twist[q];
      if (!(l > T(0))) continue;
      T sg = mode == 0 ? T(1) : T(-1);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          D[3 * a + b] = (U[3 * a + i] * V[3 * b + j] + sg * U[3 * a + j] * V[3 * b + i]) * inv_sqrt2;
      int idx = 0;
#pragma unroll
      for (int r = 0; r < 9; ++r)
#pragma unroll
        for (int c = r; c < 9; ++c) A45[idx++] += l * D[r] * D[c];
    }
  }
}

// index of (r, c), r <= c, in the 45-entry upper triangle
__host__ __device__ __forceinline__ int sym45(int r, int c) {
  if (r > c) { int t = r; r = c; c = t; }
  return r * 9 - r * (r - 1) / 2 + (c - r);
}

// ---------------------------------------------------------------------------
// deterministic block reduction of doubles (fixed order within a block)
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// sum of n partials in fixed order by one block; returns the total to all threads
template <int NT>
__device__ __forceinline__ double sum_partials(const double *part, int n, double *sh) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) acc += part[i];
  return block_sum<NT>(acc, sh);
}

// bounded wait helper: true while the caller should keep waiting
__device__ __forceinline__ bool keep_waiting(long long &spins, long long limit) {
  ++spins;
  if (spins > limit) return false;
  if ((spins & 63) == 0) __nanosleep(256);
  return true;
}

}  // namespace hot
