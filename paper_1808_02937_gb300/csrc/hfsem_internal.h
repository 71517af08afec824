// Internal declarations shared by the translation units of the hfsem library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "hfsem.h"

namespace hf {

struct Error : public std::exception {
  int code;
  std::string msg;
  Error(int c, std::string m) : code(c), msg(std::move(m)) {}
  const char* what() const noexcept override { return msg.c_str(); }
};

inline void cuda_check(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    throw Error(HFSEM_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  if (e != cudaSuccess)
    throw Error(HFSEM_ERR_DEVICE, std::string(what) + ": " + cudaGetErrorString(e));
}
#define HF_CHECK(x) ::hf::cuda_check((x), #x)
extern std::atomic<long long> g_launches;   // kernels launched by this library (process-wide)
#define HF_LAUNCH_CHECK() \
  do {                    \
    ++::hf::g_launches;   \
    ::hf::cuda_check(cudaGetLastError(), "kernel launch"); \
  } while (0)

void set_last_error(const std::string& m);

// Owning device buffer.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  bool pooled = false;         // allocated stream-ordered (cudaMallocAsync) on st
  cudaStream_t st = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      if (pooled) cudaFreeAsync(p, st);
      else cudaFree(p);
    }
    p = nullptr;
    n = 0;
    pooled = false;
  }
  // allocates on the calling thread's allocation stream when one is set
  // (AllocStream below): stream-ordered from the device's memory pool, so a
  // factorisation repeated on the same stream reuses its memory without a
  // device synchronisation; otherwise cudaMalloc
  void alloc(size_t count);
  void ensure(size_t count) {
    if (count > n) alloc(count);
  }
};

// The stream that DevBuf::alloc allocates on for the calling thread (RAII).
cudaStream_t& alloc_stream();
struct AllocStream {
  cudaStream_t prev;
  explicit AllocStream(cudaStream_t s) : prev(alloc_stream()) { alloc_stream() = s; }
  ~AllocStream() { alloc_stream() = prev; }
};
// keep freed pool memory cached for reuse (once per device)
void pool_keep_memory();
// Lets kernel fn take up to `bytes` of dynamic shared memory.  The attribute
// is process-wide, so it is raised once per device to the most the function
// can have and never lowered: concurrent callers (other host threads) can
// then never see a limit below what they launch with.
void allow_dyn_smem(const void* fn, size_t bytes);

template <class T>
void DevBuf<T>::alloc(size_t count) {
  release();
  if (count == 0) return;
  cudaStream_t s = alloc_stream();
  if (s != reinterpret_cast<cudaStream_t>(-1)) {
    pool_keep_memory();
    HF_CHECK(cudaMallocAsync(reinterpret_cast<void**>(&p), count * sizeof(T), s));
    pooled = true;
    st = s;
  } else {
    HF_CHECK(cudaMalloc(&p, count * sizeof(T)));
  }
  n = count;
}

// Gauss rules (host): weight (1-x)^a (1+x)^b on [-1, 1].
void gauss_jacobi_rule(int n, double a, double b, std::vector<double>& x,
                       std::vector<double>& w);
void gauss_legendre_rule(int n, std::vector<double>& x, std::vector<double>& w);

// Largest Gauss-Legendre rule kept in the device table.
constexpr int kMaxGL = 96;
constexpr int kMaxP = 32;

// Kinds of operator storage.
constexpr int kDense = 0;
constexpr int kToeplitz = 1;
constexpr int kHmat = 2;     // FP64 H-matrix operator over a near-field band of pairs

// Options of the H-matrix operator (kHmat): Taylor rank, admissibility
// parameter (min-diameter rule) and leaf size in unknowns.  At rank 24 the
// Lemma's bound (1/3)^24 is below the FP64 rounding of the entries.
constexpr int kHopRank = 24;
constexpr double kHopLambda = 1.0;
constexpr int kHopLeafDofs = 128;

// Per-instance descriptor as seen by the kernels (plain data).
struct InstDev {
  int N, P, Nd, kind;
  int L, logL;          // FFT length (Toeplitz), power of two >= 2N
  int uniform;          // Toeplitz with constant row/column scalings
  int n_gj;             // points of the Gauss-Jacobi (0, 2-alpha) rule
  double alpha, theta, rho, c1, c2, g0;
  long long o_h, o_dl, o_dr;   // arena offsets (doubles)
  long long o_M;               // dense: packed lower blocks; Toeplitz: lags
  long long o_D;               // P x P self-block reference matrix
  long long o_gj;              // Gauss-Jacobi nodes then weights
  long long o_rs, o_cs;        // Toeplitz row / column scalings (N each)
  long long o_spec;            // Toeplitz symbol offset (complex entries)
  long long o_vec;             // sum of N_d over earlier instances
  long long o_z;               // sum of N*P over earlier instances
  long long o_T;               // dense: sum of N(N+1)/2 * P over earlier
  long long o_fft;             // Toeplitz: sum of L*P over earlier instances
  long long o_N;               // sum of N over earlier instances
  long long o_flo, o_off;      // kHmat: first stored f of row e; pair offsets (N+1)
  long long o_c0, o_rN;        // kHmat: column f = 0 (mode 0) and row e = N-1 (mode 0)
  long long band;              // kHmat: stored pairs
};

struct InstHost {
  int N, P, Nd, kind;
  double a, b, alpha, theta, rho, c1, c2, g0;
  std::vector<double> h, dl, dr;   // lengths; node distances to a and to b
  bool uniform = false;
  double q = 1.0;
  std::vector<int> flo;            // kHmat: first stored trial element of row e
  double node_diff(int i, int j) const {  // x_i - x_j, i >= j
    return (dl[i] <= dr[j]) ? dl[i] - dl[j] : dr[j] - dr[i];
  }
};

// Per-column BiCGSTAB scalars (one column = one instance x one rhs).
struct KCol {
  double rho, rho_old, alpha, omega, beta, bnorm2, res, snorm, true_res;
  int status, iters, restarts, checks;
};

// Kernels of a region the host enqueued ahead of knowing whether it is
// needed (a Krylov iteration after every column may already have stopped)
// take a device flag and return at once while it is 0; nullptr: always run.
#define HF_GATE(g)                       \
  do {                                   \
    if ((g) != nullptr && *(g) == 0) return; \
  } while (0)

struct KrylovWork {
  DevBuf<double> vecs, partial, bx;
  DevBuf<long long> coff;
  DevBuf<int> clen, flag;
  DevBuf<int> gates;   // one flag per region of an iteration block
  DevBuf<KCol> cols;
  ~KrylovWork();
};

// Preconditioner interface: y = M^{-1} r on element-major vectors.
struct Precond {
  virtual ~Precond() {}
  virtual void apply(int nrhs, const double* r_em, double* y_em) = 0;
  // HFSEM_OK, or the status of a failure the device recorded during the
  // applies so far (a copy that missed its wait limit: HFSEM_ERR_TIMEOUT)
  virtual int device_status() { return HFSEM_OK; }
};

}  // namespace hf

struct hfsem_system_s {
  cudaStream_t st = nullptr;
  int n_inst = 0;
  std::vector<hf::InstHost> ih;
  std::vector<hf::InstDev> idv;
  hf::DevBuf<hf::InstDev> d_inst;
  hf::DevBuf<double> arena;
  hf::DevBuf<double2> spec;
  hf::DevBuf<double> gl;          // Gauss-Legendre table: rule n at gl_off(n)
  long long total_nd = 0, total_nz = 0, total_T = 0, total_fft = 0, total_N = 0;
  int max_P = 0, max_N = 0, max_L = 0;
  bool any_dense = false, any_toep = false, any_hmat = false;
  hfsem_factor* hop = nullptr;    // the H-matrix operator of the kHmat instances
  const int* gate = nullptr;      // device flag of the region being enqueued (HF_GATE)
  // scratch, grown on demand
  hf::DevBuf<double> w_x, w_y, w_z, w_w, w_T, w_ylow, w_mom;
  hf::DevBuf<double2> w_fa, w_fb;
  hf::DevBuf<double> w_rhsdata;
  hf::DevBuf<double> w_hop;       // H-matrix operator: low-rank projections
  hf::DevBuf<double2> tw;         // FFT twiddles exp(-2 pi i j / tw_L)
  int tw_L = 0;
  hf::KrylovWork kry;
};

namespace hf {
// offset of the n-point rule in the Gauss-Legendre table (nodes, then weights)
__host__ __device__ inline long long gl_off(int n) { return (long long)n * (n - 1); }

// device-side pieces used by other translation units
void apply_operator(hfsem_system* s, int nrhs, const double* x_em, double* y_em,
                    int lift);
void ensure_work(hfsem_system* s, int nrhs);
void perm_to_elem(hfsem_system* s, int nrhs, const double* x_paper, double* x_em);
void perm_to_paper(hfsem_system* s, int nrhs, const double* x_em, double* x_paper);
void load_vector_em(hfsem_system* s, const hfsem_rhs* rhs, int lifted, double* G_em);
bool is_device_ptr(const void* p);
// kernel timing: Tick t(stream, "tag", work) ... ~Tick records the end event
bool timing_on();
struct Tick {
  int id = -1;
  cudaStream_t st;
  Tick(cudaStream_t s, const char* tag, double work = 0.0);
  ~Tick();
};
void timing_add_work(const char* tag, double work);
// Timing groups: the launches timed on this thread between begin and end
// form a group that can be dropped from the records later, once the host
// learns that the device skipped the region they belong to.
long long timing_group_begin();
void timing_group_end();
void timing_drop_group(long long g);
hf::Precond* precond_of(hfsem_system* s, hfsem_factor* f);
void bicgstab(hfsem_system* s, Precond* M, int nrhs, const double* b_em, double* x_em,
              double tol, int max_iter, std::vector<KCol>& out);
// Moves a system and its factor (may be NULL) to another stream: later calls
// issue their work there.  The caller makes sure no work of theirs is still
// running on the old stream.
void rebind_stream(hfsem_system* s, hfsem_factor* f, cudaStream_t st);
// After a failed call: wait for whatever the call already queued on the
// system's stream (errors ignored), so that no work of a failed call is
// still in flight when the caller moves on or frees the handles.
inline void drain_after_error(hfsem_system* s);
// Device bytes a system, a factor hold (their buffers as grown so far).
size_t system_bytes(const hfsem_system* s);
size_t factor_bytes(const hfsem_factor* f);
// The H-matrix operator of the kHmat instances of s (built at assembly from
// the band of pair blocks) and its product y += A x on element-major vectors.
void build_operator(hfsem_system* s);
void hop_apply(hfsem_system* s, int nrhs, const double* x_em, double* y_em);
// Near-field band of the kHmat operator: for every element e the first
// trial element f of the pairs (e, f <= e) its dense blocks need.
void hop_band(const InstHost& I, std::vector<int>& flo);
// Leaf size (unknowns) the autotuner chose for I's class under a requested
// precision; 0 if none.
int tune_leaf_dofs(const InstHost& I, int precision);
// Loads, on the current device, the scratch array and the kernels of
// hfsem_apply_noalloc (once per device), so that its calls allocate nothing.
void noalloc_prepare();
}  // namespace hf

inline void hf::drain_after_error(hfsem_system* s) {
  if (s) cudaStreamSynchronize(s->st);
  cudaGetLastError();
}
