// Right-preconditioned BiCGSTAB (Sec. 4.2, eq. (precondsys)) for a batch of
// columns (instance, right-hand side), all in FP64.
//
// Every column carries its own scalars, status and iteration count on the
// device.  The host enqueues iterations in blocks (2, 4, 8, then 16 at a
// time) and reads the column states back once per block: before each
// iteration a one-CTA kernel sets a device flag saying whether any column is
// still running, and the operator, preconditioner and vector kernels of the
// iteration return at once while it is 0.  A column whose recursive residual
// meets tol waits (no work, no count) until the block ends; the host then runs
// the true-residual check for all such columns at once.  A solve of i
// iterations costs about log2(i) + 2 host synchronisations, and iterations
// enqueued past the last one cost empty launches only.
// Inner products are reduced in a fixed order (per-CTA tree, then a fixed
// sweep over CTAs), so results are bitwise reproducible run to run.
//
// Convergence is decided on the true residual.  The recursively updated
// residual r drifts from b - A x in finite precision (the more so, the more
// iterations a weak preconditioner needs), so a column whose recursive
// residual reaches tol is only a candidate: its true residual b - A x is
// formed, and the column is accepted when that is within kTrueSlack * tol.
// Otherwise the iteration restarts from the true residual (residual
// replacement: r = rh = b - A x, p = v = 0).  A restart cycle shrinks the
// drift with the residual it starts from, so when one fails to halve the
// true residual of the previous check, the true residual sits at the floor
// the FP64 product A x allows (it grows with N_d and with the operator's
// rounding) and the column is accepted there; stats report that value.
#include "hfsem_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace hf {

constexpr int kChunk = 2048;   // elements per CTA in the reductions
constexpr int kDotThreads = 256;

enum : int {
  ST_RUN = 0,      // iterating
  ST_CONV = 1,     // true residual accepted
  ST_BREAK = 2,    // rho, omega or (rh, v) vanished
  ST_MAXIT = 3,    // iteration budget spent
  ST_CHECK = 4,    // recursive residual <= tol: true residual pending
  ST_RESTART = 5,  // true residual too large: restart from it
  ST_FLOOR = 6,    // accepted: restarts no longer reduce the true residual
};
// a candidate is accepted when ||b - A x|| <= kTrueSlack * tol * ||b||: the
// recursive and true residuals of FP64 BiCGSTAB may part by a modest factor
// even when nothing went wrong
constexpr double kTrueSlack = 100.0;
constexpr int kMaxRestarts = 8;

// fixed-order CTA reduction of up to 3 sums
template <int K>
__device__ void block_reduce(double (&v)[K], double* out) {
  __shared__ double red[K][kDotThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) s += red[threadIdx.x][w];
    out[threadIdx.x] = s;
  }
}

// Fused vector updates and partial inner products.
enum : int {
  M_INIT = 0,      // r = b - Ax (Ax given in v), rh = r, p = v = 0; dots (r,r)
  M_P = 1,         // p = r + beta (p - omega v)
  M_RV = 2,        // dot (rh, v)
  M_S = 3,         // s = r - alpha v; dot (s, s)
  M_TS = 4,        // dots (t, s), (t, t)
  M_X = 5,         // x += alpha ph + omega sh; r = s - omega t; dots (r,r), (rh,r)
  M_XS = 6,        // x += alpha ph  (early exit on small s)
  M_RES = 7,       // r = b - Ax (Ax in v); dots (r,r)
  M_TRUE = 8,      // candidates: s = b - Ax (Ax in t); dot (s,s)
  M_RESTART = 9,   // restarting columns: r = rh = s, p = v = 0; dot (r,r)
};

struct Vecs {
  double *b, *x, *r, *rh, *p, *ph, *v, *s, *sh, *t;
};

__global__ void k_bicg_vec(int mode, Vecs V, const long long* __restrict__ coff,
                           const int* __restrict__ clen, KCol* cols, double* partial,
                           int maxchunk) {
  const int c = blockIdx.y;
  const KCol k = cols[c];
  const int len = clen[c];
  const long long o = coff[c];
  const int chunk = blockIdx.x;
  if (chunk * kChunk >= len) return;
  const bool live = mode == M_INIT || mode == M_RES ? true
                    : mode == M_TRUE                ? k.status == ST_CHECK
                    : mode == M_RESTART             ? k.status == ST_RESTART
                                                    : k.status == ST_RUN;
  double acc[2] = {0.0, 0.0};
  if (live) {
    const int e0 = chunk * kChunk, e1 = min(len, e0 + kChunk);
    for (int j = e0 + threadIdx.x; j < e1; j += blockDim.x) {
      long long i = o + j;
      switch (mode) {
        case M_INIT: {
          double r = V.b[i] - V.v[i];
          V.r[i] = r;
          V.rh[i] = r;
          V.p[i] = 0.0;
          V.v[i] = 0.0;
          acc[0] += r * r;
          acc[1] += V.b[i] * V.b[i];
          break;
        }
        case M_P:
          V.p[i] = V.r[i] + k.beta * (V.p[i] - k.omega * V.v[i]);
          break;
        case M_RV:
          acc[0] += V.rh[i] * V.v[i];
          break;
        case M_S: {
          double s = V.r[i] - k.alpha * V.v[i];
          V.s[i] = s;
          acc[0] += s * s;
          break;
        }
        case M_TS:
          acc[0] += V.t[i] * V.s[i];
          acc[1] += V.t[i] * V.t[i];
          break;
        case M_X: {
          V.x[i] += k.alpha * V.ph[i] + k.omega * V.sh[i];
          double r = V.s[i] - k.omega * V.t[i];
          V.r[i] = r;
          acc[0] += r * r;
          acc[1] += V.rh[i] * r;
          break;
        }
        case M_XS:
          V.x[i] += k.alpha * V.ph[i];
          break;
        case M_RES: {
          double r = V.b[i] - V.v[i];
          acc[0] += r * r;
          break;
        }
        case M_TRUE: {
          double r = V.b[i] - V.t[i];
          V.s[i] = r;
          acc[0] += r * r;
          break;
        }
        case M_RESTART: {
          double r = V.s[i];
          V.r[i] = r;
          V.rh[i] = r;
          V.p[i] = 0.0;
          V.v[i] = 0.0;
          acc[0] += r * r;
          break;
        }
      }
    }
  }
  __shared__ double out[2];
  block_reduce<2>(acc, out);
  if (threadIdx.x < 2) partial[((size_t)c * maxchunk + chunk) * 2 + threadIdx.x] = out[threadIdx.x];
}

// Sum the chunk partials in order and advance the per-column scalars.
__global__ void k_bicg_scalar(int mode, const int* __restrict__ clen, KCol* cols,
                              const double* partial, int maxchunk, int ncols, double tol,
                              int iter, int max_iter) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  KCol k = cols[c];
  int nch = (clen[c] + kChunk - 1) / kChunk;
  double s0 = 0.0, s1 = 0.0;
  for (int j = 0; j < nch; ++j) {
    s0 += partial[((size_t)c * maxchunk + j) * 2];
    s1 += partial[((size_t)c * maxchunk + j) * 2 + 1];
  }
  switch (mode) {
    case M_INIT:
      k.checks = 0;
      k.bnorm2 = s1;
      k.rho = s0;
      k.rho_old = 1.0;
      k.alpha = 1.0;
      k.omega = 1.0;
      k.iters = 0;
      k.restarts = 0;
      k.true_res = INFINITY;
      k.res = (s1 > 0.0) ? sqrt(s0 / s1) : 0.0;
      k.status = (clen[c] == 0 || s1 == 0.0 || k.res <= tol) ? ST_CONV : ST_RUN;
      k.beta = 0.0;
      break;
    case M_RV:
      if (k.status != ST_RUN) break;
      if (s0 == 0.0 || !isfinite(s0)) {
        k.status = ST_BREAK;
        break;
      }
      k.alpha = k.rho / s0;
      break;
    case M_S:
      if (k.status != ST_RUN) break;
      k.snorm = sqrt(s0 / k.bnorm2);
      break;
    case M_TS:
      if (k.status != ST_RUN) break;
      if (s1 == 0.0 || !isfinite(s1)) {
        k.status = ST_BREAK;
        break;
      }
      k.omega = s0 / s1;
      if (k.omega == 0.0) k.status = ST_BREAK;
      break;
    case M_X:
      if (k.status != ST_RUN) break;
      k.iters += 1;   // per column: a column waiting for its check does not count
      k.res = sqrt(s0 / k.bnorm2);
      k.rho_old = k.rho;
      k.rho = s1;
      if (k.res <= tol) {
        k.status = ST_CHECK;
      } else if (k.rho == 0.0 || !isfinite(k.res)) {
        k.status = ST_BREAK;
      } else {
        k.beta = (k.rho / k.rho_old) * (k.alpha / k.omega);
        if (k.iters >= max_iter) k.status = ST_MAXIT;
      }
      break;
    case M_RES:
      k.true_res = (k.bnorm2 > 0.0) ? sqrt(s0 / k.bnorm2) : 0.0;
      break;
    case M_TRUE: {
      if (k.status != ST_CHECK) break;
      k.checks += 1;
      const double t = sqrt(s0 / k.bnorm2);
      if (t <= kTrueSlack * tol) {
        k.status = ST_CONV;
      } else if (!isfinite(t)) {
        k.status = ST_BREAK;
      } else if (k.restarts > 0 && !(t < 0.5 * k.true_res)) {
        k.status = ST_FLOOR;          // the last restart did not pay
      } else if (k.restarts >= kMaxRestarts || k.iters >= max_iter) {
        k.status = ST_MAXIT;
      } else {
        k.status = ST_RESTART;
      }
      k.true_res = t;
      break;
    }
    case M_RESTART:
      if (k.status != ST_RESTART) break;
      k.rho = s0;
      k.rho_old = 1.0;
      k.alpha = 1.0;
      k.omega = 1.0;
      k.beta = 0.0;
      k.res = sqrt(s0 / k.bnorm2);
      k.restarts += 1;
      k.status = ST_RUN;
      break;
  }
  cols[c] = k;
}

// Columns whose recursive residual was already small after s take the
// half step (x += alpha ph) and stop.
__global__ void k_bicg_smallS(KCol* cols, int ncols, double tol, int* flag) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  KCol k = cols[c];
  flag[c] = 0;
  if (k.status == ST_RUN && k.snorm <= tol) flag[c] = 1;
}

__global__ void k_bicg_xs(Vecs V, const long long* coff, const int* clen, KCol* cols,
                          const int* flag, int iter) {
  const int c = blockIdx.y;
  if (!flag[c]) return;
  const long long o = coff[c];
  const int len = clen[c];
  const KCol k = cols[c];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < len; j += gridDim.x * blockDim.x)
    V.x[o + j] += k.alpha * V.ph[o + j];
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // the scalar update is done by k_bicg_xs_fin after all blocks ran
  }
}

__global__ void k_bicg_xs_fin(KCol* cols, const int* flag, int ncols, int iter) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols || !flag[c]) return;
  cols[c].status = ST_CHECK;
  cols[c].res = cols[c].snorm;
  cols[c].iters += 1;
}

// gate = 1 if any column has status `which`, else 0 (one CTA)
__global__ void k_bicg_flags(const KCol* __restrict__ cols, int ncols, int which, int* gate) {
  int any = 0;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) any |= cols[c].status == which;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) *gate = any;
}

KrylovWork::~KrylovWork() = default;

namespace {
constexpr int kBlockFirst = 2;   // iterations enqueued before the first read
constexpr int kBlockMax = 16;

// Scope of one gated region: the kernels launched inside read `gate`, and
// the launches timed inside form one timing group.
struct Region {
  hfsem_system* s;
  long long group;
  Region(hfsem_system* sys, const int* gate) : s(sys) {
    s->gate = gate;
    group = timing_group_begin();
  }
  ~Region() {
    s->gate = nullptr;
    timing_group_end();
  }
};
}  // namespace

void bicgstab(hfsem_system* s, Precond* M, int nrhs, const double* b_em, double* x_em,
              double tol, int max_iter, std::vector<KCol>& out) {
  const int ni = s->n_inst;
  KrylovWork& W = s->kry;
  const int ncols = ni * nrhs;
  std::vector<long long> coff(ncols);
  std::vector<int> clen(ncols);
  int maxchunk = 1;
  for (int i = 0; i < ni; ++i)
    for (int r = 0; r < nrhs; ++r) {
      int c = i * nrhs + r;
      coff[c] = s->idv[i].o_vec * nrhs + (long long)r * s->ih[i].Nd;
      clen[c] = s->ih[i].Nd;
      maxchunk = std::max(maxchunk, (clen[c] + kChunk - 1) / kChunk);
    }
  size_t nv = (size_t)s->total_nd * nrhs;
  W.vecs.ensure(nv * 9 + 1);
  W.coff.ensure(ncols);
  W.clen.ensure(ncols);
  W.cols.ensure(ncols);
  W.partial.ensure((size_t)ncols * maxchunk * 2);
  W.flag.ensure(ncols);
  W.gates.ensure(kBlockMax);
  HF_CHECK(cudaMemcpyAsync(W.coff.p, coff.data(), ncols * sizeof(long long),
                           cudaMemcpyHostToDevice, s->st));
  HF_CHECK(cudaMemcpyAsync(W.clen.p, clen.data(), ncols * sizeof(int), cudaMemcpyHostToDevice,
                           s->st));
  Vecs V;
  V.b = const_cast<double*>(b_em);
  V.x = x_em;
  double* base = W.vecs.p;
  V.r = base + 0 * nv;
  V.rh = base + 1 * nv;
  V.p = base + 2 * nv;
  V.ph = base + 3 * nv;
  V.v = base + 4 * nv;
  V.s = base + 5 * nv;
  V.sh = base + 6 * nv;
  V.t = base + 7 * nv;
  if (!M) {
    V.ph = V.p;
    V.sh = V.s;
  }
  dim3 gv(maxchunk, ncols), bv(kDotThreads);
  int sb = (ncols + 127) / 128;
  // the vector passes' algorithmic bytes are added once the per-column
  // iteration counts are known (below): only live columns touch memory
  auto vec = [&](int mode) {
    Tick tk(s->st, "krylov_vec");
    k_bicg_vec<<<gv, bv, 0, s->st>>>(mode, V, W.coff.p, W.clen.p, W.cols.p, W.partial.p,
                                     maxchunk);
    HF_LAUNCH_CHECK();
  };
  auto scal = [&](int mode, int it) {
    k_bicg_scalar<<<sb, 128, 0, s->st>>>(mode, W.clen.p, W.cols.p, W.partial.p, maxchunk,
                                         ncols, tol, it, max_iter);
    HF_LAUNCH_CHECK();
  };
  // r0 = b - A x0
  apply_operator(s, nrhs, x_em, V.v, 0);
  vec(M_INIT);
  scal(M_INIT, 0);
  std::vector<KCol> hc(ncols);
  // candidates: true residual from t = A x (t is free between iterations);
  // accepted, restarted from it, or stopped
  auto check_phase = [&](int it) {
    apply_operator(s, nrhs, x_em, V.t, 0);
    vec(M_TRUE);
    scal(M_TRUE, it);
    vec(M_RESTART);
    scal(M_RESTART, it);
  };
  auto iteration = [&](int it) {
    vec(M_P);
    if (M) M->apply(nrhs, V.p, V.ph);
    apply_operator(s, nrhs, V.ph, V.v, 0);
    vec(M_RV);
    scal(M_RV, it);
    vec(M_S);
    scal(M_S, it);
    k_bicg_smallS<<<sb, 128, 0, s->st>>>(W.cols.p, ncols, tol, W.flag.p);
    HF_LAUNCH_CHECK();
    k_bicg_xs<<<dim3(8, ncols), 256, 0, s->st>>>(V, W.coff.p, W.clen.p, W.cols.p, W.flag.p, it);
    HF_LAUNCH_CHECK();
    k_bicg_xs_fin<<<sb, 128, 0, s->st>>>(W.cols.p, W.flag.p, ncols, it);
    HF_LAUNCH_CHECK();
    if (M) M->apply(nrhs, V.s, V.sh);
    apply_operator(s, nrhs, V.sh, V.t, 0);
    vec(M_TS);
    scal(M_TS, it);
    vec(M_X);
    scal(M_X, it);
  };
  std::vector<long long> groups;
  std::vector<int> gate_h(kBlockMax);
  int remaining = max_iter;   // the most iterations a running column may still take
  auto read_back = [&](bool& running, bool& check) {
    HF_CHECK(cudaMemcpyAsync(hc.data(), W.cols.p, ncols * sizeof(KCol), cudaMemcpyDeviceToHost,
                             s->st));
    if (!groups.empty())
      HF_CHECK(cudaMemcpyAsync(gate_h.data(), W.gates.p, groups.size() * sizeof(int),
                               cudaMemcpyDeviceToHost, s->st));
    HF_CHECK(cudaStreamSynchronize(s->st));
    if (timing_on()) timing_add_work("krylov_host_reads", 1.0);
    for (size_t r = 0; r < groups.size(); ++r)
      if (gate_h[r] == 0) timing_drop_group(groups[r]);
    groups.clear();
    running = check = false;
    remaining = 0;
    for (auto& k : hc) {
      if (k.status == ST_RUN) {
        running = true;
        remaining = std::max(remaining, max_iter - k.iters);
      }
      check = check || k.status == ST_CHECK;
    }
  };
  bool running = true, check = false;   // after init: enqueue a first block
  int it = 0;                           // iterations enqueued so far
  // every enqueued iteration advances each running column's own count, and
  // restarts are bounded, so this cap is never the one that stops the loop
  const long long it_cap = (long long)(kMaxRestarts + 2) * max_iter;
  for (int block = kBlockFirst;; block = std::min(2 * block, kBlockMax)) {
    if (check) {
      check_phase(it);
      read_back(running, check);
      if (running) block = kBlockFirst;   // restarted columns: short blocks again
    }
    if (!running || it >= it_cap) break;
    const int nb = std::min(block, std::max(remaining, 1));
    for (int k = 0; k < nb; ++k, ++it) {
      int* g = W.gates.p + groups.size();
      k_bicg_flags<<<1, 256, 0, s->st>>>(W.cols.p, ncols, ST_RUN, g);
      HF_LAUNCH_CHECK();
      Region rg(s, g);
      iteration(it);
      groups.push_back(rg.group);
    }
    read_back(running, check);
  }
  // true residual
  apply_operator(s, nrhs, x_em, V.v, 0);
  vec(M_RES);
  scal(M_RES, 0);
  out.resize(ncols);
  HF_CHECK(cudaMemcpyAsync(out.data(), W.cols.p, ncols * sizeof(KCol), cudaMemcpyDeviceToHost,
                           s->st));
  HF_CHECK(cudaStreamSynchronize(s->st));
  if (timing_on()) timing_add_work("krylov_host_reads", 1.0);
  for (auto& k : out)
    if (k.status == ST_RUN || k.status == ST_CHECK || k.status == ST_RESTART)
      k.status = ST_MAXIT;
  if (timing_on()) {
    // algorithmic bytes of the vector passes, 8 per vector element read or
    // written: init 6, per iteration 19 (p 4, (rh, v) 2, s 3, (t, s) 2,
    // x and r 8), per true-residual check 3, per restart 5, final residual 2
    double bytes = 0.0;
    for (int c = 0; c < ncols; ++c)
      bytes += 8.0 * clen[c] *
               (6.0 + 19.0 * out[c].iters + 3.0 * out[c].checks + 5.0 * out[c].restarts + 2.0);
    timing_add_work("krylov_vec", bytes);
  }
}

int status_code(const KCol& k) {
  switch (k.status) {
    case ST_CONV:
    case ST_FLOOR: return HFSEM_OK;
    case ST_BREAK: return HFSEM_ERR_BREAKDOWN;
    default: return HFSEM_ERR_NOT_CONVERGED;
  }
}

}  // namespace hf

using namespace hf;

extern "C" int hfsem_solve(hfsem_system* sys, hfsem_factor* fac, const hfsem_rhs* rhs,
                           double tol, int32_t max_iter, double* X, hfsem_stats* stats) {
  try {
    if (!sys || !rhs || !X || !stats) throw Error(HFSEM_ERR_INVALID_ARG, "NULL argument");
    if (!(tol > 0.0) || max_iter < 1) throw Error(HFSEM_ERR_INVALID_ARG, "tol > 0, max_iter >= 1");
    Precond* M = precond_of(sys, fac);
    int nrhs = rhs[0].nrhs;
    if (nrhs < 1 || nrhs > 64) throw Error(HFSEM_ERR_INVALID_ARG, "nrhs must be in [1, 64]");
    AllocStream as(sys->st);   // work buffers come stream-ordered from the pool
    ensure_work(sys, nrhs);
    size_t nv = (size_t)sys->total_nd * nrhs;
    KrylovWork& W = sys->kry;
    W.bx.ensure(2 * nv);
    double* b = W.bx.p;
    double* x = W.bx.p + nv;
    load_vector_em(sys, rhs, 1, b);
    HF_CHECK(cudaMemsetAsync(x, 0, nv * sizeof(double), sys->st));
    std::vector<KCol> cols;
    bicgstab(sys, M, nrhs, b, x, tol, max_iter, cols);
    perm_to_paper(sys, nrhs, x, sys->w_y.p);
    HF_CHECK(cudaMemcpyAsync(X, sys->w_y.p, nv * sizeof(double),
                             is_device_ptr(X) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             sys->st));
    HF_CHECK(cudaStreamSynchronize(sys->st));
    int worst = M ? M->device_status() : HFSEM_OK;
    if (worst != HFSEM_OK) set_last_error("the preconditioner's device work missed a wait limit");
    for (size_t c = 0; c < cols.size(); ++c) {
      stats[c].iters = cols[c].iters;
      stats[c].status = status_code(cols[c]);
      stats[c].rel_residual = cols[c].res;
      stats[c].rel_true_residual = cols[c].true_res;
      if (stats[c].status != HFSEM_OK && worst == HFSEM_OK) {
        worst = stats[c].status;
        char msg[160];
        snprintf(msg, sizeof(msg), "column %zu: %s after %d iterations (true residual %.3g)", c,
                 worst == HFSEM_ERR_BREAKDOWN ? "breakdown" : "not converged", cols[c].iters,
                 cols[c].true_res);
        set_last_error(msg);
      }
    }
    return worst;
  } catch (const Error& e) {
    set_last_error(e.msg);
    drain_after_error(sys);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    drain_after_error(sys);
    return HFSEM_ERR_OOM;
  } catch (...) {
    set_last_error("unknown error");
    drain_after_error(sys);
    return HFSEM_ERR_DEVICE;
  }
}
