// Allocation-free evaluation of the particles' elastic energy.
//
// Some callers cannot allocate device memory at the moment they need this
// value: real-time loops that must not hit the implicit device
// synchronisation of cudaMalloc/cudaFree, hosts whose device memory budget is
// fixed up front by their own pool, and code paths that may not enter an
// allocator at all.  This file serves them with one entry point whose only
// scratch is a fixed array in the library's own device memory, reserved on a
// device when the library's module is first loaded there (with lazy module
// loading, at the first use of the module on that device).
#include <mutex>

#include "internal.h"

namespace hot {
void set_thread_error(const std::string &msg);   // api.cu: message for mpm_last_error(NULL)

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_BLOCK = 2048;             // particles per block
constexpr int NA_MAX_PARTIALS = 65536;         // scratch: 65,536 + 1 doubles = 512 KiB
constexpr int NA_MAX_MATERIALS = 16;
constexpr int64_t NA_MAX_PARTICLES = (int64_t)NA_MAX_PARTIALS * NA_PER_BLOCK;   // 134,217,728

// Shared by every call on a device, for the life of the process.  Slots
// [0, nblocks) take the per-block partial sums, slot NA_MAX_PARTIALS the
// total.  Every slot a call reads is written earlier in the same call, so
// nothing needs clearing between calls; calls that overlap on the GPU race
// on it.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_PARTIALS + 1];

struct MatTable {
  MatParams m[NA_MAX_MATERIALS];
};

__global__ void k_energy_partials_noalloc(const double *__restrict__ F, const double *__restrict__ vol,
                                          const int32_t *__restrict__ mat, int64_t n, MatTable mt,
                                          int nmat, double *__restrict__ partial) {
  __shared__ double sh[NA_THREADS];
  double acc = 0.0;
  const int64_t base = (int64_t)blockIdx.x * NA_PER_BLOCK;
  for (int k = threadIdx.x; k < NA_PER_BLOCK; k += NA_THREADS) {
    const int64_t p = base + k;
    if (p >= n) break;
    double Fp[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) Fp[e] = F[9 * p + e];
    const int id = mat ? mat[p] : 0;
    if (id < 0 || id >= nmat) {   // an id outside the table makes the result NaN
      acc += nan("");
      continue;
    }
    const MatParams &mp = mt.m[id];
    acc += vol[p] * psi_density<double>(Fp, mp.mu, mp.lam, mp.model);
  }
  double t = block_sum<NA_THREADS>(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_energy_total_noalloc(const double *__restrict__ partial, int nblocks, double *total,
                                       double *out_device) {
  __shared__ double sh[NA_THREADS];
  double t = sum_partials<NA_THREADS>(partial, nblocks, sh);
  if (threadIdx.x == 0) {
    *total = t;
    if (out_device) *out_device = t;
  }
}

// Device address of the scratch array, looked up once per CUDA context.  The
// cache is keyed on the context's unique id (cuCtxGetId, reached through the
// runtime's driver entry points, so the library needs no link to the driver
// library): after a cudaDeviceReset the device gets a new primary context,
// the module is loaded again and the array is looked up again, so no address
// from a destroyed context is ever used.  Where the driver entry points are
// not available the key falls back to the device ordinal.
using PfnCtxGetCurrent = int (*)(void **ctx);
using PfnCtxGetId = int (*)(void *ctx, unsigned long long *id);

std::mutex g_na_mutex;
std::once_flag g_na_once;
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;
struct NaEntry {
  unsigned long long key;
  double *ptr;
};
constexpr int NA_CACHE = 64;   // contexts remembered (fixed size: no allocation here either)
NaEntry g_na_cache[NA_CACHE];
int g_na_cached = 0;

void resolve_driver_entry_points() {
  void *f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(f);
  f = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(f);
  cudaGetLastError();
}

// key of the current context: its unique id, else (1 << 63) | device ordinal
bool current_context_key(unsigned long long &key) {
  if (g_ctx_get_current && g_ctx_get_id) {
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) == 0 && ctx && g_ctx_get_id(ctx, &id) == 0) {
      key = id;
      return true;
    }
    return false;   // no current context yet
  }
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  key = (1ull << 63) | (unsigned long long)dev;
  return true;
}

double *scratch_for_current_device() {
  std::call_once(g_na_once, resolve_driver_entry_points);
  std::lock_guard<std::mutex> lock(g_na_mutex);
  unsigned long long key = 0;
  const bool have_key = current_context_key(key);
  if (have_key)
    for (int k = 0; k < g_na_cached; ++k)
      if (g_na_cache[k].key == key) return g_na_cache[k].ptr;
  double *p = nullptr;   // (this lookup makes the device's context current if none was)
  check_cuda(cudaGetSymbolAddress((void **)&p, g_noalloc_scratch), "cudaGetSymbolAddress(g_noalloc_scratch)");
  if (!have_key && !current_context_key(key)) return p;   // not cached: looked up again next call
  if (g_na_cached < NA_CACHE) g_na_cache[g_na_cached++] = NaEntry{key, p};
  return p;
}

}  // namespace
}  // namespace hot

extern "C" mpm_status mpm_particle_energy_noalloc(const double *F, const double *vol, const int32_t *material_id,
                                                  const mpm_material *materials, int32_t n_materials,
                                                  int64_t n_particles, double *energy, int32_t energy_on_device,
                                                  void *cuda_stream) {
  using namespace hot;
  try {
    if (n_particles < 0) fail(MPM_ERR_INVALID_ARG, "n_particles must be >= 0");
    if (n_particles > NA_MAX_PARTICLES)
      fail(MPM_ERR_INVALID_ARG, "n_particles exceeds the allocation-free limit of 134,217,728 particles "
                                "(512 KiB of partial sums); use mpm_eval_energy");
    if (n_materials < 1 || n_materials > NA_MAX_MATERIALS || !materials)
      fail(MPM_ERR_INVALID_ARG, "between 1 and 16 materials are required");
    if (!energy || (n_particles > 0 && (!F || !vol))) fail(MPM_ERR_INVALID_ARG, "NULL argument");
    MatTable mt;
    for (int k = 0; k < NA_MAX_MATERIALS; ++k) mt.m[k] = MatParams{0.0, 0.0, 0.0, 0.0, 0, 0};
    for (int k = 0; k < n_materials; ++k) {
      const double E = materials[k].E, nu = materials[k].nu;
      if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5) || (materials[k].model != 0 && materials[k].model != 1))
        fail(MPM_ERR_INVALID_ARG, "bad material " + std::to_string(k));
      mt.m[k].mu = E / (2.0 * (1.0 + nu));
      mt.m[k].lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
      mt.m[k].model = materials[k].model;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double *scratch = scratch_for_current_device();
    const int nblocks = (int)((n_particles + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
    if (nblocks > 0) {
      k_energy_partials_noalloc<<<nblocks, NA_THREADS, 0, st>>>(F, vol, material_id, n_particles, mt, n_materials,
                                                                scratch);
      check_cuda(cudaGetLastError(), "k_energy_partials_noalloc");
    }
    k_energy_total_noalloc<<<1, NA_THREADS, 0, st>>>(scratch, nblocks, scratch + NA_MAX_PARTIALS,
                                                     energy_on_device ? energy : nullptr);
    check_cuda(cudaGetLastError(), "k_energy_total_noalloc");
    if (!energy_on_device) {
      check_cuda(cudaMemcpyAsync(energy, scratch + NA_MAX_PARTIALS, sizeof(double), cudaMemcpyDeviceToHost, st),
                 "cudaMemcpyAsync");
      check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    }
    return MPM_OK;
  } catch (const Error &e) {
    set_thread_error(e.msg);   // surfaced through mpm_last_error(NULL)
    return e.code;
  }
}
