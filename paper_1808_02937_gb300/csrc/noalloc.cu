// hfsem_apply_noalloc: the operator product y = A x of hfsem_apply, for
// callers that must not allocate device memory during the call (for example
// a host thread that runs inside a memory-capped or allocation-free section
// of an application, or code that owns every allocation itself).  Its
// temporaries live in one file-scope device array instead of cudaMalloc'd
// buffers; the system handle itself was allocated earlier by hfsem_assemble.
#include <cstring>
#include <mutex>

#include "hfsem_internal.h"

namespace hf {
// kernels of the operator product (defined in system.cu)
__global__ void k_perm(const InstDev* __restrict__ inst, const double* __restrict__ in,
                       double* out, int nrhs, int to_elem);
__global__ void k_gather_z(const InstDev* __restrict__ inst, const double* arena,
                           const double* __restrict__ x, double* z, int nrhs, int lift,
                           const int* __restrict__ gate);
__global__ void k_scatter_out(const InstDev* __restrict__ inst, const double* arena,
                              const double* __restrict__ w, const double* __restrict__ x,
                              double* y, int nrhs, int lift, const int* __restrict__ gate);
__global__ void k_dense_rows(const InstDev* __restrict__ inst, const double* arena,
                             const double* __restrict__ z, double* ylow, double* T, int nrhs);
__global__ void k_dense_cols(const InstDev* __restrict__ inst, const double* ylow,
                             const double* T, double* w, int nrhs);
__global__ void k_toep_fwd(const InstDev* __restrict__ inst, const double* arena,
                           const double* __restrict__ z, double2* F, const double2* tw,
                           int Lmax, int nrhs, const int* __restrict__ gate);
__global__ void k_toep_freq(const InstDev* __restrict__ inst, const double2* spec, double2* F,
                            int nrhs, const int* __restrict__ gate);
__global__ void k_toep_inv(const InstDev* __restrict__ inst, const double* arena,
                           const double2* F, double* w, const double2* tw, int Lmax, int nrhs,
                           const int* __restrict__ gate);
}  // namespace hf

namespace {

// Scratch of the no-allocation entry point: 32 MiB per device, held by every
// GPU that loads the library until the process exits.
constexpr size_t kNoAllocBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_na_mu;
void* g_na_ptr[128] = {nullptr};   // device address of the array, per device

// Device address of the scratch array on the current device, looked up once
// per device (the array's name is only a host-side stand-in in host code).
void* scratch_address() {
  int dev = 0;
  HF_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) throw hf::Error(HFSEM_ERR_DEVICE, "device index out of range");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    HF_CHECK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_na_ptr[dev] = p;
  }
  return g_na_ptr[dev];
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

bool g_na_loaded[128] = {false};   // kernels of the product loaded, per device

dim3 grid_of(long long n, int bs, int y, int z) {
  long long g = (n + bs - 1) / bs;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return dim3((unsigned)g, (unsigned)y, (unsigned)z);
}

void set_smem_attr(const void* fn, size_t bytes) { hf::allow_dyn_smem(fn, bytes); }

}  // namespace

namespace hf {

// Called by hfsem_assemble: the module holding the scratch array and the
// kernels launched below are loaded on first use (CUDA's lazy loading), which
// reserves device memory.  Doing it here, where allocation is expected,
// leaves nothing to load in hfsem_apply_noalloc itself.
void noalloc_prepare() {
  scratch_address();
  int dev = 0;
  HF_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (g_na_loaded[dev]) return;
  const void* fns[] = {(const void*)k_perm,      (const void*)k_gather_z,
                       (const void*)k_scatter_out, (const void*)k_dense_rows,
                       (const void*)k_dense_cols, (const void*)k_toep_fwd,
                       (const void*)k_toep_freq,  (const void*)k_toep_inv};
  for (const void* f : fns) {
    cudaFuncAttributes fa;
    HF_CHECK(cudaFuncGetAttributes(&fa, f));
  }
  g_na_loaded[dev] = true;
}

}  // namespace hf

using namespace hf;

extern "C" int hfsem_apply_noalloc(hfsem_system* s, int32_t nrhs, const double* x, double* y) {
  try {
    if (!s || !x || !y || nrhs < 1 || nrhs > 64)
      throw Error(HFSEM_ERR_INVALID_ARG, "hfsem_apply_noalloc: bad arguments");
    if (!is_device_ptr(x) || !is_device_ptr(y))
      throw Error(HFSEM_ERR_INVALID_ARG, "hfsem_apply_noalloc: x and y must be device pointers");
    if (s->any_hmat)
      throw Error(HFSEM_ERR_INVALID_ARG,
                  "hfsem_apply_noalloc: dense and Toeplitz operators only (not HFSEM_MATVEC_HMATRIX)");
    // carve the scratch: x and y in element-major order, z, w, ylow, the
    // dense column partials and the FFT buffers
    const size_t nd = (size_t)s->total_nd * nrhs, nz = (size_t)s->total_nz * nrhs;
    size_t off[7], need = 0;
    const size_t sizes[7] = {nd * 8, nd * 8, nz * 8, nz * 8, nz * 8,
                             s->any_dense ? (size_t)s->total_T * nrhs * 8 : 0,
                             s->any_toep ? (size_t)s->total_fft * 2 * nrhs * 16 : 0};
    for (int i = 0; i < 7; ++i) {
      off[i] = need;
      need += round256(sizes[i]);
    }
    if (need > kNoAllocBytes)
      throw Error(HFSEM_ERR_INVALID_ARG,
                  "hfsem_apply_noalloc: needs " + std::to_string(need >> 20) +
                      " MiB of scratch, more than the 32 MiB it has; use hfsem_apply");
    unsigned char* base = static_cast<unsigned char*>(scratch_address());
    double* xe = reinterpret_cast<double*>(base + off[0]);
    double* ye = reinterpret_cast<double*>(base + off[1]);
    double* z = reinterpret_cast<double*>(base + off[2]);
    double* w = reinterpret_cast<double*>(base + off[3]);
    double* ylow = reinterpret_cast<double*>(base + off[4]);
    double* T = reinterpret_cast<double*>(base + off[5]);
    double2* F = reinterpret_cast<double2*>(base + off[6]);
    // every scratch element read below is written first in the same call,
    // so nothing has to be cleared
    const int ni = s->n_inst;
    const InstDev* di = s->d_inst.p;
    const long long nmp = (long long)s->max_N * s->max_P;
    k_perm<<<grid_of(nmp, 256, ni, nrhs), 256, 0, s->st>>>(di, x, xe, nrhs, 1);
    HF_LAUNCH_CHECK();
    k_gather_z<<<grid_of(nmp, 256, ni, nrhs), 256, 0, s->st>>>(di, s->arena.p, xe, z, nrhs, 0, nullptr);
    HF_LAUNCH_CHECK();
    if (s->any_dense) {
      int W = (s->max_P > 16) ? 4 : 8;
      size_t sm = (size_t)(W * 2 * s->max_P * s->max_P + W * s->max_P * nrhs) * sizeof(double);
      set_smem_attr((const void*)k_dense_rows, sm);
      k_dense_rows<<<dim3(s->max_N, ni), W * 32, sm, s->st>>>(di, s->arena.p, z, ylow, T, nrhs);
      HF_LAUNCH_CHECK();
      k_dense_cols<<<grid_of(nmp, 128, ni, nrhs), 128, 0, s->st>>>(di, ylow, T, w, nrhs);
      HF_LAUNCH_CHECK();
    }
    if (s->any_toep) {
      size_t sm = (size_t)s->max_L * sizeof(double2);
      set_smem_attr((const void*)k_toep_fwd, sm);
      set_smem_attr((const void*)k_toep_inv, sm);
      k_toep_fwd<<<dim3(2 * s->max_P, ni, nrhs), 256, sm, s->st>>>(di, s->arena.p, z, F, s->tw.p,
                                                                   s->tw_L, nrhs, nullptr);
      HF_LAUNCH_CHECK();
      k_toep_freq<<<grid_of(s->max_L, 128, ni, nrhs), 128, 0, s->st>>>(di, s->spec.p, F, nrhs, nullptr);
      HF_LAUNCH_CHECK();
      k_toep_inv<<<dim3(s->max_P, ni, nrhs), 256, sm, s->st>>>(di, s->arena.p, F, w, s->tw.p,
                                                               s->tw_L, nrhs, nullptr);
      HF_LAUNCH_CHECK();
    }
    k_scatter_out<<<grid_of(nmp, 256, ni, nrhs), 256, 0, s->st>>>(di, s->arena.p, w, xe, ye, nrhs,
                                                                  0, nullptr);
    HF_LAUNCH_CHECK();
    k_perm<<<grid_of(nmp, 256, ni, nrhs), 256, 0, s->st>>>(di, ye, y, nrhs, 0);
    HF_LAUNCH_CHECK();
    HF_CHECK(cudaStreamSynchronize(s->st));
    return HFSEM_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return HFSEM_ERR_OOM;
  } catch (...) {
    set_last_error("unknown error");
    return HFSEM_ERR_DEVICE;
  }
}
