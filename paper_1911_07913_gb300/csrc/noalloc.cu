// Allocation-free evaluation of the particles' elastic energy.
//
// Some callers cannot allocate device memory at the moment they need this
// value: code that runs while a CUDA stream is being captured into a graph
// (cudaMalloc is not a stream operation and is refused or breaks the
// capture), real-time loops that must not hit the implicit device
// synchronisation of cudaMalloc/cudaFree, and hosts whose memory budget is
// fixed up front by their own pool.  This file serves them with one entry
// point whose only scratch is a fixed array in the library's own device
// memory, reserved when the library is loaded.
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

// device address of the scratch array, looked up once per device
std::mutex g_na_mutex;
double *g_na_ptr[64] = {nullptr};

double *scratch_for_current_device() {
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) fail(MPM_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    double *p = nullptr;
    check_cuda(cudaGetSymbolAddress((void **)&p, g_noalloc_scratch), "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_na_ptr[dev] = p;
  }
  return g_na_ptr[dev];
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
