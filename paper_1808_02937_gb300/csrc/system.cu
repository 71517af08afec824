// Assembly of the SEM operator (Sec. 2.2) and its application, dense
// (Sec. 4.2) or block-Toeplitz through FFTs (Sec. 4.3), plus the load vector.
//
// Representation.  On element e (0-based, [x_e, x_{e+1}], length h_e) the
// derivative of u_N^P is a polynomial of degree P-1; its Legendre
// coefficients z_e[m] follow from the unknowns by psi_p' = -(2p+1) L_p and the
// chain rule:
//     z_e[0] = (u(x_{e+1}) - u(x_e)) / h_e,
//     z_e[p] = -(2p+1) (2/h_e) uhat_e^p,            p = 1..P-1.
// Writing z = Pi x, the left-sided stiffness is S_l = Pi^T Mb Pi with the
// block lower-triangular element-pair matrix
//     Mb_ef[m][n] = gamma0 int_{I_e} L_m(xi_e(t)) int_{I_f, s<t}
//                    (t-s)^(1-alpha) L_n(xi_f(s)) ds dt,          f <= e,
// so A x = rho M x + Pi^T (theta Mb + (1-theta) Mb^T) Pi x.  Every block is
// read once per product and used for both Mb and Mb^T.
//
// Internal vector ordering is element-major: element e owns its P-1 bubbles
// followed by the hat at its right node (dof e*P + p - 1, hat j at j*P - 1).
#include <atomic>

#include "hfsem_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

namespace hf {

std::atomic<long long> g_launches{0};
static thread_local std::string g_last_error;
void set_last_error(const std::string& m) { g_last_error = m; }
const std::string& last_error() { return g_last_error; }

// ---------------------------------------------------------------------------
// kernel timing registry
// ---------------------------------------------------------------------------
namespace {
struct TimerRec {
  double ms = 0.0;
  long long launches = 0;
  double work = 0.0;
};
struct Pending {
  cudaEvent_t a, b;
  std::string tag;
  double work;
  long long group;   // timing group the launch belongs to (0: none)
  bool dropped;      // its region was skipped on the device: not counted
};
std::mutex g_tmu;
bool g_timing = false;
std::map<std::string, TimerRec> g_tim;
std::vector<Pending> g_pend;
std::vector<cudaEvent_t> g_evpool;

cudaEvent_t get_event() {
  if (!g_evpool.empty()) {
    cudaEvent_t e = g_evpool.back();
    g_evpool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void flush_pending() {
  for (auto& p : g_pend) {
    cudaEventSynchronize(p.b);
    if (p.dropped) {
      g_evpool.push_back(p.a);
      g_evpool.push_back(p.b);
      continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    TimerRec& r = g_tim[p.tag];
    r.ms += ms;
    r.launches += 1;
    r.work += p.work;
    g_evpool.push_back(p.a);
    g_evpool.push_back(p.b);
  }
  g_pend.clear();
}
}  // namespace

bool timing_on() { return g_timing; }

namespace {
thread_local long long t_group = 0;
std::atomic<long long> g_next_group{1};
}  // namespace

long long timing_group_begin() {
  t_group = g_next_group.fetch_add(1);
  return t_group;
}

void timing_group_end() { t_group = 0; }

void timing_drop_group(long long g) {
  if (g <= 0) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  for (auto& p : g_pend)
    if (p.group == g) p.dropped = true;
}

cudaStream_t& alloc_stream() {
  thread_local cudaStream_t s = reinterpret_cast<cudaStream_t>(-1);   // none: cudaMalloc
  return s;
}

void pool_keep_memory() {
  static std::mutex mu;
  static bool done[128] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;   // a process-local attribute of the pool
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[dev] = true;
}

Tick::Tick(cudaStream_t s, const char* tag, double work) : st(s) {
  if (!g_timing) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  Pending p;
  p.a = get_event();
  p.b = get_event();
  p.tag = tag;
  p.work = work;
  p.group = t_group;
  p.dropped = false;
  cudaEventRecord(p.a, s);
  g_pend.push_back(p);
  id = (int)g_pend.size() - 1;
}

Tick::~Tick() {
  if (id < 0) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  cudaEventRecord(g_pend[id].b, st);
}

void timing_add_work(const char* tag, double work) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_tim[tag].work += work;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Legendre three-term recurrence L_{k+1} = a_k x L_k - b_k L_{k-1} with
// a_k = (2k+1)/(k+1), b_k = k/(k+1), tabulated so that the quadrature loops
// carry no FP64 division (a costly sequence on this GPU's FP64 pipe)
constexpr int kRecMax = 128;
struct LegRec {
  double a[kRecMax], b[kRecMax];
};
constexpr LegRec make_legrec() {
  LegRec r{};
  for (int k = 0; k < kRecMax; ++k) {
    r.a[k] = (2.0 * k + 1.0) / (k + 1.0);
    r.b[k] = k / (k + 1.0);
  }
  return r;
}
__constant__ LegRec c_leg = make_legrec();

__device__ __forceinline__ double leg_next(int k, double x, double pk, double pkm1) {
  return c_leg.a[k] * x * pk - c_leg.b[k] * pkm1;
}

// Legendre values L_0..L_{n-1} at x into out[k*stride]
__device__ __forceinline__ void legendre_strided(int n, double x, double* out,
                                                 int stride, double scale) {
  double p0 = 1.0, p1 = x;
  if (n > 0) out[0] = scale * p0;
  if (n > 1) out[stride] = scale * p1;
  for (int k = 1; k + 1 < n; ++k) {
    double p2 = leg_next(k, x, p1, p0);
    out[(k + 1) * stride] = scale * p2;
    p0 = p1;
    p1 = p2;
  }
}

// Gauss points needed in one direction of a box whose distance to the
// kernel's singular line is r times its length (Bernstein ellipse argument:
// the error of an n-point rule on the kernel times degree-(P-1) polynomials
// falls like rhoB^-(2n - P + 1), kept near 1e-15 per box, below the rounding
// of the FP64 sums it enters).
__device__ __forceinline__ int box_points(int P, double r) {
  double t = 1.0 + 2.0 * r;
  double rhoB = t + sqrt(t * t - 1.0);
  int n = (int)ceil(0.5 * (P - 1) + 17.3 / log(rhoB)) + 1;
  n = max(n, (P + 2) / 2);
  return min(n, 40);
}

// Per-warp scratch of the pair quadrature
struct PairScratch {
  double* acc;  // P*P
  double* A;    // P*NQ   basis x weight at outer nodes
  double* B;    // P*NQ   basis x weight at inner nodes
  double* T;    // P*NQ   partial contraction
  double* su;   // NQ
  double* sv;   // NQ
  double* sk;   // NQ     per-node factors
  double* K;    // KCH    kernel values of a chunk of box rows
};
constexpr int NQ = 40;
constexpr int KCH = 256;
__host__ __device__ inline int pair_scratch_doubles(int P) { return P * P + 3 * P * NQ + 3 * NQ + KCH; }

__device__ inline PairScratch carve(double* base, int P) {
  PairScratch s;
  s.acc = base;
  s.A = s.acc + P * P;
  s.B = s.A + P * NQ;
  s.T = s.B + P * NQ;
  s.su = s.T + P * NQ;
  s.sv = s.su + NQ;
  s.sk = s.sv + NQ;
  s.K = s.sk + NQ;
  return s;
}

// acc[m][n] += sum_ij wu_i wv_j L_m(xi(u_i)) (g+u_i+v_j)^(1-alpha) L_n(eta(v_j))
// over the box [u0,u1] x [v0,v1]; xi = -1 + 2u/he, eta = 1 - 2v/hf; the
// weights are divided by he and hf (the block is stored scaled, see
// pair_block).
__device__ void box_quad(PairScratch& s, int P, double alpha, double he,
                         double hf, double g, double u0, double u1, double v0,
                         double v1, int nq, const double* gl, int lane) {
  const double* X = gl + gl_off(nq);
  const double* Wt = X + nq;
  double lu = u1 - u0, lv = v1 - v0;
  for (int i = lane; i < nq; i += 32) {
    double u = u0 + 0.5 * lu * (1.0 + X[i]);
    double v = v0 + 0.5 * lv * (1.0 + X[i]);
    s.su[i] = u;
    s.sv[i] = v;
    legendre_strided(P, -1.0 + 2.0 * u / he, s.A + i, NQ, 0.5 * (lu / he) * Wt[i]);
    legendre_strided(P, 1.0 - 2.0 * v / hf, s.B + i, NQ, 0.5 * (lv / hf) * Wt[i]);
  }
  __syncwarp();
  const double ex = 1.0 - alpha;
  // (g+u+v)^(1-alpha) = d^(1-alpha) exp((1-alpha) log y), y = (g+u+v)/d, with
  // d = g + u0 + v0 > 0 the box corner nearest the singular line: every box
  // is no longer than its distance to that line, so y lies in [1, 3] and the
  // logarithm stays small (a few ulp, at a fraction of the cost of pow)
  const double d = g + u0 + v0;
  const double dinv = 1.0 / d, dex = pow(d, ex);
  // T[n][i] = sum_j K(u_i, v_j) B[n][j], a chunk of rows i at a time: every
  // lane evaluates kernel values (nq^2 per box, the costly part), then every
  // lane forms sums of the chunk
  const int ib = max(1, min(nq, KCH / nq));
  for (int i0 = 0; i0 < nq; i0 += ib) {
    const int ni = min(ib, nq - i0);
    for (int t = lane; t < ni * nq; t += 32) {
      const int ii = t / nq, j = t - ii * nq;
      s.K[t] = dex * exp(ex * log((g + s.su[i0 + ii] + s.sv[j]) * dinv));
    }
    __syncwarp();
    for (int t = lane; t < ni * P; t += 32) {
      const int n = t / ni, ii = t - n * ni;
      const double* kr = s.K + ii * nq;
      const double* br = s.B + n * NQ;
      double a = 0.0;
      for (int j = 0; j < nq; ++j) a += kr[j] * br[j];
      s.T[n * NQ + i0 + ii] = a;
    }
    __syncwarp();
  }
  for (int e = lane; e < P * P; e += 32) {
    int m = e / P, n = e % P;
    double a = 0.0;
    for (int i = 0; i < nq; ++i) a += s.A[m * NQ + i] * s.T[n * NQ + i];
    s.acc[e] += a;
  }
  __syncwarp();
}

// One Duffy triangle of the square [0,c]^2 next to the common corner of a
// touching pair, kernel (u+v)^(1-alpha):
//   variant 0: u = c rho, v = c rho w;  variant 1: v = c rho, u = c rho w.
// rho: Gauss-Jacobi weight rho^(2-alpha) (rule gj on [-1,1], weight
// (1+x)^(2-alpha)), w: Gauss-Legendre with nw points.
__device__ void duffy_tri(PairScratch& s, int P, double alpha, double he,
                          double hf, double c, int variant, const double* gjx,
                          const double* gjw, int ngj, int nw, const double* gl,
                          int lane) {
  const double* X = gl + gl_off(nw);
  const double* Wt = X + nw;
  const double ex = 1.0 - alpha;
  // c^(3-alpha) 2^(alpha-3) / (he hf), in factors that stay in range
  const double cfac = pow(c, 1.0 - alpha) * (c / he) * (c / hf) * exp2(alpha - 3.0);
  // the inner weights with the kernel factor (1 + w_j)^(1-alpha), once
  for (int j = lane; j < nw; j += 32) s.K[j] = 0.5 * Wt[j] * pow(1.0 + 0.5 * (1.0 + X[j]), ex);
  __syncwarp();
  // per outer node k: T[q][k] = sum_j K_kj * basis_q(inner point (k, j))
  for (int k = lane; k < ngj; k += 32) {
    double rho = 0.5 * (1.0 + gjx[k]);
    double wk = cfac * gjw[k];
    for (int q = 0; q < P; ++q) s.T[q * NQ + k] = 0.0;
    // outer-only basis: variant 0 -> L_m(xi(c rho)); variant 1 -> L_n(eta(c rho))
    if (variant == 0)
      legendre_strided(P, -1.0 + 2.0 * c * rho / he, s.A + k, NQ, wk);
    else
      legendre_strided(P, 1.0 - 2.0 * c * rho / hf, s.A + k, NQ, wk);
    for (int j = 0; j < nw; ++j) {
      double w = 0.5 * (1.0 + X[j]);
      double kw = s.K[j];
      double y = (variant == 0) ? 1.0 - 2.0 * c * rho * w / hf
                                : -1.0 + 2.0 * c * rho * w / he;
      double p0 = 1.0, p1 = y;
      s.T[k] += kw;
      if (P > 1) s.T[NQ + k] += kw * p1;
      for (int q = 1; q + 1 < P; ++q) {
        double p2 = leg_next(q, y, p1, p0);
        s.T[(q + 1) * NQ + k] += kw * p2;
        p0 = p1;
        p1 = p2;
      }
    }
  }
  __syncwarp();
  for (int e = lane; e < P * P; e += 32) {
    int m = e / P, n = e % P;
    double a = 0.0;
    if (variant == 0)
      for (int k = 0; k < ngj; ++k) a += s.A[m * NQ + k] * s.T[n * NQ + k];
    else
      for (int k = 0; k < ngj; ++k) a += s.T[m * NQ + k] * s.A[n * NQ + k];
    s.acc[e] += a;
  }
  __syncwarp();
}

// Element-pair block (unscaled by gamma0) for test element e right of (or
// equal to) trial element f, divided by he hf: the block of the
// derivative-coefficient operator scales like he hf (distance)^(1-alpha),
// (h/2)^(3-alpha) for the self pair, which leaves the FP64 range for
// elements below ~1e-160; divided it scales like (distance)^(1-alpha) and
// pairs with the scale-free coefficient map of k_gather_z.
// kind: 0 self, 1 touching, 2 separated (gap g).
__device__ void pair_block(PairScratch& s, int P, double alpha, double he,
                           double hf, double g, int kind, const double* D,
                           const double* gjx, const double* gjw, int ngj,
                           const double* gl, int lane) {
  for (int e = lane; e < P * P; e += 32) s.acc[e] = 0.0;
  __syncwarp();
  if (kind == 0) {
    double sc = 0.25 * pow(0.5 * he, 1.0 - alpha);   // (he/2)^(3-alpha) / he^2
    for (int e = lane; e < P * P; e += 32) s.acc[e] = sc * D[e];
    __syncwarp();
    return;
  }
  if (kind == 1) {
    // u = t - x_e in [0, he], v = x_e - s in [0, hf], t - s = u + v
    double c = fmin(he, hf);
    int nw = (P + 1) / 2 + 12;
    duffy_tri(s, P, alpha, he, hf, c, 0, gjx, gjw, ngj, nw, gl, lane);
    duffy_tri(s, P, alpha, he, hf, c, 1, gjx, gjw, ngj, nw, gl, lane);
    int nq = box_points(P, 1.0);
    for (double u0 = c; u0 < he * (1.0 - 1e-15);) {       // remainder in u
      double u1 = fmin(2.0 * u0, he);
      box_quad(s, P, alpha, he, hf, 0.0, u0, u1, 0.0, c, nq, gl, lane);
      u0 = u1;
    }
    for (double v0 = c; v0 < hf * (1.0 - 1e-15);) {       // remainder in v
      double v1 = fmin(2.0 * v0, hf);
      box_quad(s, P, alpha, he, hf, 0.0, 0.0, c, v0, v1, nq, gl, lane);
      v0 = v1;
    }
    return;
  }
  // separated: geometric pieces in u and in v, each no longer than its
  // distance to the singular line u + v = -g
  for (double u0 = 0.0; u0 < he * (1.0 - 1e-15);) {
    double u1 = fmin(u0 + (g + u0), he);
    for (double v0 = 0.0; v0 < hf * (1.0 - 1e-15);) {
      double v1 = fmin(v0 + (g + v0), hf);
      double len = fmax(u1 - u0, v1 - v0);
      int nq = box_points(P, (g + u0 + v0) / len);
      box_quad(s, P, alpha, he, hf, g, u0, u1, v0, v1, nq, gl, lane);
      v0 = v1;
    }
    u0 = u1;
  }
}

// ---------------------------------------------------------------------------
// assembly kernels
// ---------------------------------------------------------------------------

// Self-block reference matrix D[m][n] = int_{-1}^{1} L_m(xi)
//   int_{-1}^{xi} (xi-eta)^(1-alpha) L_n(eta) deta dxi, from the fractional
// integral of a Legendre polynomial,
//   int_{-1}^{xi} (xi-eta)^(1-alpha) L_n = Gamma(2-alpha) n!/Gamma(n+3-alpha)
//        (1+xi)^(2-alpha) P_n^(alpha-2, 2-alpha)(xi),
// integrated with the Gauss-Jacobi rule for the weight (1+xi)^(2-alpha).
__global__ void k_selfblock(const InstDev* __restrict__ inst, double* arena) {
  const InstDev I = inst[blockIdx.x];
  const int P = I.P;
  const double* gx = arena + I.o_gj;
  const double* gw = gx + I.n_gj;
  const double a = I.alpha - 2.0;   // Jacobi parameters (a, -a)
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
    int m = e / P, n = e % P;
    double coef = 1.0 / (2.0 - I.alpha);   // Gamma(2-alpha) 0!/Gamma(3-alpha)
    for (int k = 1; k <= n; ++k) coef *= (double)k / (k + 2.0 - I.alpha);
    double acc = 0.0;
    for (int q = 0; q < I.n_gj; ++q) {
      double x = gx[q];
      // Jacobi P_n^(a,-a)(x): (k+1) P_{k+1} = (2k+1) x P_k - (k+a)(k-a)/k P_{k-1}
      double p0 = 1.0, p1 = x + a, pn = (n == 0) ? p0 : p1;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2 * k + 1) * x * p1 - (k + a) * (k - a) / k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
        pn = p2;
      }
      // Legendre L_m(x)
      double l0 = 1.0, l1 = x, lm = (m == 0) ? l0 : l1;
      for (int k = 1; k < m; ++k) {
        double l2 = ((2 * k + 1) * x * l1 - k * l0) / (k + 1);
        l0 = l1;
        l1 = l2;
        lm = l2;
      }
      acc += gw[q] * lm * pn;
    }
    arena[I.o_D + e] = coef * acc;
  }
}

// All element-pair blocks (dense instances: every f <= e; Toeplitz
// instances: the lags (e = k, f = 0), stored divided by r_k c_0).
__global__ void k_pairs(const InstDev* __restrict__ inst, double* arena,
                        const double* __restrict__ gl, int wpc, int stride) {
  extern __shared__ double smem[];
  const InstDev I = inst[blockIdx.y];
  const int P = I.P;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  PairScratch s = carve(smem + (size_t)warp * stride, P);
  const double* h = arena + I.o_h;
  const double* dl = arena + I.o_dl;
  const double* dr = arena + I.o_dr;
  const double* D = arena + I.o_D;
  const double* gjx = arena + I.o_gj;
  const double* gjw = gjx + I.n_gj;
  // kHmat: the boundary column and row only serve the lifting of c1, c2
  const bool lift = I.c1 != 0.0 || I.c2 != 0.0;
  const long long np = (I.kind == kDense)  ? (long long)I.N * (I.N + 1) / 2
                       : (I.kind == kHmat) ? I.band + (lift ? 2LL * I.N : 0LL)
                                           : I.N;
  const double* off = arena + I.o_off;   // kHmat: pairs before row e
  for (long long p = (long long)blockIdx.x * wpc + warp; p < np;
       p += (long long)gridDim.x * wpc) {
    int e, f;
    int out_kind = 0;   // 0: block at p; 1: column f = 0 (c0); 2: row e = N-1 (rN)
    if (I.kind == kDense) {
      e = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
      while ((long long)e * (e + 1) / 2 > p) --e;
      while ((long long)(e + 1) * (e + 2) / 2 <= p) ++e;
      f = (int)(p - (long long)e * (e + 1) / 2);
    } else if (I.kind == kHmat) {
      if (p < I.band) {
        int lo = 0, hi = I.N - 1;   // the row e with off[e] <= p < off[e+1]
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if ((long long)off[mid] <= p) lo = mid;
          else hi = mid - 1;
        }
        e = lo;
        f = (int)arena[I.o_flo + e] + (int)(p - (long long)off[e]);
      } else if (p < I.band + I.N) {
        e = (int)(p - I.band);
        f = 0;
        out_kind = 1;
      } else {
        e = I.N - 1;
        f = (int)(p - I.band - I.N);
        out_kind = 2;
      }
    } else {
      e = (int)p;
      f = 0;
    }
    int kind = (e == f) ? 0 : (e == f + 1 ? 1 : 2);
    double g = 0.0;
    if (kind == 2) {  // x_e - x_{f+1} from the closer endpoint
      g = (dl[e] <= dr[f + 1]) ? dl[e] - dl[f + 1] : dr[f + 1] - dr[e];
    }
    pair_block(s, P, I.alpha, h[e], h[f], g, kind, D, gjx, gjw, I.n_gj, gl, lane);
    double sc = I.g0;
    if (I.kind == kToeplitz) sc /= arena[I.o_rs + e] * arena[I.o_cs + f];
    if (out_kind == 0) {
      double* out = arena + I.o_M + p * P * P;
      for (int k = lane; k < P * P; k += 32) out[k] = sc * s.acc[k];
    } else if (out_kind == 1) {   // mode n = 0 of block (e, 0): c0[e][m]
      for (int m = lane; m < P; m += 32) arena[I.o_c0 + (long long)e * P + m] = sc * s.acc[m * P];
    } else {                      // mode m = 0 of block (N-1, f): rN[f][n]
      for (int n = lane; n < P; n += 32) arena[I.o_rN + (long long)f * P + n] = sc * s.acc[n];
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// FFT (radix-2, in shared memory, one sequence per CTA)
// ---------------------------------------------------------------------------
__global__ void k_twiddles(double2* tw, int Lmax) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Lmax / 2;
       j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)Lmax, &s, &c);
    tw[j] = make_double2(c, s);
  }
}

// in-place iterative FFT of a[] given in bit-reversed order;
// sign -1: forward (exp(-2 pi i jk/L)), +1: inverse (unnormalised)
__device__ void fft_core(double2* a, int L, int logL, const double2* __restrict__ tw,
                         int Lmax, int inverse) {
  for (int st = 1; st <= logL; ++st) {
    int half = 1 << (st - 1);
    int twstep = Lmax >> st;
    for (int t = threadIdx.x; t < L / 2; t += blockDim.x) {
      int j = t & (half - 1);
      int i0 = ((t >> (st - 1)) << st) + j;
      int i1 = i0 + half;
      double2 w = tw[j * twstep];
      if (inverse) w.y = -w.y;
      double2 x0 = a[i0], x1 = cmul(w, a[i1]);
      a[i0] = make_double2(x0.x + x1.x, x0.y + x1.y);
      a[i1] = make_double2(x0.x - x1.x, x0.y - x1.y);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int k, int logL) {
  return (int)(__brev((unsigned)k) >> (32 - logL));
}

// Toeplitz symbol: spectrum[(m*P+n)*L + w] = sum_k mu_k[m][n] exp(-2 pi i k w / L)
__global__ void k_symbol(const InstDev* __restrict__ inst, const double* arena,
                         double2* spec, const double2* tw, int Lmax) {
  extern __shared__ double2 fbuf[];
  const InstDev I = inst[blockIdx.y];
  if (I.kind != kToeplitz) return;
  const int P = I.P;
  int mn = blockIdx.x;
  if (mn >= P * P) return;
  const double* mu = arena + I.o_M;
  for (int k = threadIdx.x; k < I.L; k += blockDim.x) {
    double v = (k < I.N) ? mu[(size_t)k * P * P + mn] : 0.0;
    fbuf[bitrev(k, I.logL)] = make_double2(v, 0.0);
  }
  __syncthreads();
  fft_core(fbuf, I.L, I.logL, tw, Lmax, 0);
  double2* out = spec + I.o_spec + (size_t)mn * I.L;
  for (int k = threadIdx.x; k < I.L; k += blockDim.x) out[k] = fbuf[k];
}

// ---------------------------------------------------------------------------
// operator application
// ---------------------------------------------------------------------------

// z = Pi x, Pi scaled by the element length (z_e = h_e times the Legendre
// coefficients of u' on element e): z_e[0] = u(x_{e+1}) - u(x_e),
// z_e[m] = -2(2m+1) (coefficient of psi_m); the pair blocks carry the
// matching 1/(h_e h_f).  (lift: boundary hats carry c1, c2 instead of 0)
__global__ void k_gather_z(const InstDev* __restrict__ inst, const double* arena,
                           const double* __restrict__ x, double* z, int nrhs,
                           int lift, const int* __restrict__ gate) {
  HF_GATE(gate);
  const InstDev I = inst[blockIdx.y];
  const int r = blockIdx.z;
  const int P = I.P, N = I.N;
  const double* xv = x + I.o_vec * nrhs + (size_t)r * I.Nd;
  double* zv = z + I.o_z * nrhs + (size_t)r * N * P;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * P;
       t += gridDim.x * blockDim.x) {
    int e = t / P, m = t % P;
    // kHmat instances: the boundary values only (the H-matrix operator adds
    // the interior unknowns' product itself)
    const bool bnd_only = I.kind == kHmat;
    double val;
    if (m == 0) {
      double uL = (e == 0) ? (lift ? I.c1 : 0.0) : (bnd_only ? 0.0 : xv[e * P - 1]);
      double uR = (e == N - 1) ? (lift ? I.c2 : 0.0) : (bnd_only ? 0.0 : xv[(e + 1) * P - 1]);
      val = uR - uL;
    } else {
      val = bnd_only ? 0.0 : -2.0 * (2.0 * m + 1.0) * xv[e * P + m - 1];
    }
    zv[t] = val;
  }
}

// y = Pi^T w + rho M x (lift: the boundary hats' values enter the mass term)
__global__ void k_scatter_out(const InstDev* __restrict__ inst, const double* arena,
                              const double* __restrict__ w, const double* __restrict__ x,
                              double* y, int nrhs, int lift, const int* __restrict__ gate) {
  HF_GATE(gate);
  const InstDev I = inst[blockIdx.y];
  const int r = blockIdx.z;
  const int P = I.P, N = I.N;
  const double* h = arena + I.o_h;
  const double* xv = x + I.o_vec * nrhs + (size_t)r * I.Nd;
  // kHmat instances: the mass of the boundary hats only (the H-matrix
  // operator holds rho M on the interior unknowns)
  const bool bnd_only = I.kind == kHmat;
  const double* wv = w + I.o_z * nrhs + (size_t)r * N * P;
  double* yv = y + I.o_vec * nrhs + (size_t)r * I.Nd;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.Nd;
       i += gridDim.x * blockDim.x) {
    int e = i / P, p = i % P + 1;    // p == P: the hat at node e+1
    double out;
    if (p < P) {
      double he = h[e];
      out = -2.0 * (2.0 * p + 1.0) * wv[e * P + p];
      if (I.rho != 0.0) {
        // local mass on [L, R, psi_1..]: scaled by h/2
        double uL = (e == 0) ? (lift ? I.c1 : 0.0) : (bnd_only ? 0.0 : xv[e * P - 1]);
        double uR = (e == N - 1) ? (lift ? I.c2 : 0.0) : (bnd_only ? 0.0 : xv[(e + 1) * P - 1]);
        double acc = 0.0;
        if (p == 1) acc += uL + uR;
        if (p == 2) acc += (-uL + uR) / 3.0;
        acc += (2.0 / (2 * p - 1) + 2.0 / (2 * p + 3)) * (bnd_only ? 0.0 : xv[e * P + p - 1]);
        if (p + 2 < P) acc += -2.0 / (2 * p + 3) * (bnd_only ? 0.0 : xv[e * P + p + 1]);
        if (p - 2 >= 1) acc += -2.0 / (2 * p - 1) * (bnd_only ? 0.0 : xv[e * P + p - 3]);
        out += I.rho * 0.5 * he * acc;
      }
    } else {
      // hat at node j = e+1: right hat of element e, left hat of element e+1
      int j = e + 1;
      double hl = h[j - 1], hr = h[j];
      out = wv[(j - 1) * P] - wv[j * P];
      if (I.rho != 0.0) {
        double uj = (bnd_only ? 0.0 : xv[i]);
        double ul = (j - 1 == 0) ? (lift ? I.c1 : 0.0) : (bnd_only ? 0.0 : xv[(j - 1) * P - 1]);
        double ur = (j + 1 == N) ? (lift ? I.c2 : 0.0) : (bnd_only ? 0.0 : xv[(j + 1) * P - 1]);
        // element j-1 (local R): RR = 2/3, RL = 1/3, R psi_1 = 1, R psi_2 = 1/3
        double accl = (2.0 / 3.0) * uj + (1.0 / 3.0) * ul;
        if (P > 1) accl += (bnd_only ? 0.0 : xv[(j - 1) * P + 0]);
        if (P > 2) accl += (bnd_only ? 0.0 : xv[(j - 1) * P + 1]) / 3.0;
        // element j (local L): LL = 2/3, LR = 1/3, L psi_1 = 1, L psi_2 = -1/3
        double accr = (2.0 / 3.0) * uj + (1.0 / 3.0) * ur;
        if (P > 1) accr += (bnd_only ? 0.0 : xv[j * P + 0]);
        if (P > 2) accr -= (bnd_only ? 0.0 : xv[j * P + 1]) / 3.0;
        out += I.rho * (0.5 * hl * accl + 0.5 * hr * accr);
      }
    }
    yv[i] = out;
  }
}

// Dense rows: CTA per (row e, instance).  Each warp takes blocks f = warp,
// warp + W, ... of row e; the lower product accumulates into ylow[e], and
// Mb_ef^T z_e goes to T[(e,f)] for the column reduction.
__global__ void k_dense_rows(const InstDev* __restrict__ inst, const double* arena,
                             const double* __restrict__ z, double* ylow, double* T,
                             int nrhs) {
  extern __shared__ double sm[];
  const InstDev I = inst[blockIdx.y];
  if (I.kind != kDense) return;
  const int e = blockIdx.x;
  if (e >= I.N) return;
  const int P = I.P, PP = P * P;
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* prod = sm + (size_t)warp * 2 * PP;     // per warp: products
  double* yacc = sm + (size_t)W * 2 * PP;        // W * P * nrhs partial sums
  for (int k = threadIdx.x; k < W * P * nrhs; k += blockDim.x) yacc[k] = 0.0;
  __syncthreads();
  const double* Mrow = arena + I.o_M + ((long long)e * (e + 1) / 2) * PP;
  const double* zb = z + I.o_z * nrhs;
  const long long NP = (long long)I.N * P;
  for (int f = warp; f <= e; f += W) {
    const double* Mb = Mrow + (size_t)f * PP;
    double mv[32];
    int cnt = 0;
    for (int k = lane; k < PP; k += 32) mv[cnt++] = Mb[k];
    for (int r = 0; r < nrhs; ++r) {
      const double* zr = zb + r * NP;
      cnt = 0;
      for (int k = lane; k < PP; k += 32) {
        int m = k / P, n = k % P;
        prod[k] = mv[cnt] * zr[(size_t)f * P + n];        // row m of the product
        prod[PP + k] = mv[cnt] * zr[(size_t)e * P + m];   // column n of Mb^T z_e
        ++cnt;
      }
      __syncwarp();
      if (lane < P) {
        double sy = 0.0, st = 0.0;
        for (int n = 0; n < P; ++n) sy += prod[lane * P + n];
        for (int m = 0; m < P; ++m) st += prod[PP + m * P + lane];
        yacc[(warp * nrhs + r) * P + lane] += sy;
        T[I.o_T * nrhs + (size_t)r * ((long long)I.N * (I.N + 1) / 2) * P +
          ((long long)e * (e + 1) / 2 + f) * P + lane] = st;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < P * nrhs; k += blockDim.x) {
    int r = k / P, m = k % P;
    double s = 0.0;
    for (int w = 0; w < W; ++w) s += yacc[(w * nrhs + r) * P + m];
    ylow[I.o_z * nrhs + r * NP + (size_t)e * P + m] = s;
  }
}

// Boundary columns of a kHmat instance (lifting): z holds only the boundary
// values (z_0[0] = -c1, z_{N-1}[0] = c2; c2 - c1 for N = 1), and
//   w = theta M z + (1 - theta) M^T z
// needs of the stored pairs only the column f = 0 and the row e = N-1 (plus
// the diagonal pairs (0,0) and (N-1,N-1) of the band).
__global__ void k_lift_hmat(const InstDev* __restrict__ inst, const double* __restrict__ arena,
                            const double* __restrict__ z, double* w, int nrhs,
                            const int* __restrict__ gate) {
  HF_GATE(gate);
  const InstDev I = inst[blockIdx.y];
  if (I.kind != kHmat) return;
  const int P = I.P, N = I.N, r = blockIdx.z;
  const double* zv = z + I.o_z * nrhs + (size_t)r * N * P;
  double* wv = w + I.o_z * nrhs + (size_t)r * N * P;
  const double a0 = zv[0];
  const double aN = (N > 1) ? zv[(size_t)(N - 1) * P] : 0.0;
  const double* c0 = arena + I.o_c0;
  const double* rN = arena + I.o_rN;
  const double* M = arena + I.o_M;
  const long long PP = (long long)P * P;
  const long long d0 = (long long)arena[I.o_off];                       // pair (0, 0)
  const long long dN = (long long)arena[I.o_off + N] - 1;               // pair (N-1, N-1)
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * P; t += gridDim.x * blockDim.x) {
    const int e = t / P, m = t % P;
    double lo = a0 * c0[t];                                   // (M z)_e[m], column 0
    double up = (e == 0) ? a0 * M[d0 * PP + m] : 0.0;         // (M^T z)_e[m], row 0
    if (N > 1) {
      if (e == N - 1) lo += aN * M[dN * PP + (long long)m * P];
      up += aN * rN[t];                                       // row N-1
    }
    wv[t] = I.theta * lo + (1.0 - I.theta) * up;
  }
}

// Dense operator, two passes over the packed lower blocks M_ef (f <= e,
// row-major P x P, contiguous along f for fixed e), no temporaries:
//   row pass:     w[e][m] = theta       sum_{f <= e} sum_n M_ef[m][n] z[f][n]
//   column pass:  w[f][n] += (1-theta)  sum_{e >= f} sum_m M_ef[m][n] z[e][m]
// One warp per block-row (block-column); its lanes are (block, index) pairs,
// 32 / P blocks at a time, so that a lane keeps a fixed column n (row m) of
// the blocks it visits and accumulates all P outputs of its row (column)
// for RB right-hand sides in registers; one warp reduction at the end.
// Every FP64 multiply-add of the pass is one entry times one z value: the
// FP64 pipe, not memory, bounds it (4 flops per entry and right-hand side
// against 8 bytes per entry and pass).
template <int PT, int RB>
__global__ void __launch_bounds__(256) k_dense_rowpass(const InstDev* __restrict__ inst,
                                                       const double* __restrict__ arena,
                                                       const double* __restrict__ z, double* w,
                                                       int nrhs, const int* __restrict__ gate) {
  HF_GATE(gate);
  const InstDev I = inst[blockIdx.y];
  if (I.kind != kDense) return;
  const int P = I.P, N = I.N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = N - 1 - (int)(blockIdx.x * (blockDim.x >> 5) + warp);   // long rows first
  if (e < 0) return;
  const int r0 = blockIdx.z * RB;
  const long long NP = (long long)N * P;
  const double* zb = z + I.o_z * nrhs;
  double* wb = w + I.o_z * nrhs;
  double acc[PT][RB];
#pragma unroll
  for (int m = 0; m < PT; ++m)
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[m][r] = 0.0;
  if (I.theta != 0.0) {
    const int F = 32 / P;                   // blocks per step
    const int fo = lane / P, n = lane - fo * P;
    const long long PP = (long long)P * P;
    const double* strip = arena + I.o_M + ((long long)e * (e + 1) / 2) * PP;
    if (fo < F) {
      for (int f = fo; f <= e; f += F) {
        double zr[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r)
          zr[r] = (r0 + r < nrhs) ? __ldg(zb + (long long)(r0 + r) * NP + (long long)f * P + n) : 0.0;
        const double* blk = strip + (long long)f * PP + n;
#pragma unroll
        for (int m = 0; m < PT; ++m) {
          if (m < P) {
            const double v = __ldg(blk + m * P);
#pragma unroll
            for (int r = 0; r < RB; ++r) acc[m][r] = fma(v, zr[r], acc[m][r]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < PT; ++m) {
    if (m >= P) break;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      double x = acc[m][r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0 && r0 + r < nrhs) wb[(long long)(r0 + r) * NP + (long long)e * P + m] = I.theta * x;
    }
  }
}

template <int PT, int RB>
__global__ void __launch_bounds__(256) k_dense_colpass(const InstDev* __restrict__ inst,
                                                       const double* __restrict__ arena,
                                                       const double* __restrict__ z, double* w,
                                                       int nrhs, const int* __restrict__ gate) {
  HF_GATE(gate);
  const InstDev I = inst[blockIdx.y];
  if (I.kind != kDense || I.theta == 1.0) return;
  const int P = I.P, N = I.N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = (int)(blockIdx.x * (blockDim.x >> 5) + warp);          // long columns first
  if (f >= N) return;
  const int r0 = blockIdx.z * RB;
  const long long NP = (long long)N * P;
  const double* zb = z + I.o_z * nrhs;
  double* wb = w + I.o_z * nrhs;
  double acc[PT][RB];
#pragma unroll
  for (int n = 0; n < PT; ++n)
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[n][r] = 0.0;
  const int F = 32 / P;
  const int eo = lane / P, m = lane - eo * P;
  const long long PP = (long long)P * P;
  const double* base = arena + I.o_M;
  if (eo < F) {
    for (int e = f + eo; e < N; e += F) {
      double zr[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r)
        zr[r] = (r0 + r < nrhs) ? __ldg(zb + (long long)(r0 + r) * NP + (long long)e * P + m) : 0.0;
      const double* blk = base + ((long long)e * (e + 1) / 2 + f) * PP + (long long)m * P;
#pragma unroll
      for (int n = 0; n < PT; ++n) {
        if (n < P) {
          const double v = __ldg(blk + n);
#pragma unroll
          for (int r = 0; r < RB; ++r) acc[n][r] = fma(v, zr[r], acc[n][r]);
        }
      }
    }
  }
  const double c = 1.0 - I.theta;
#pragma unroll
  for (int n = 0; n < PT; ++n) {
    if (n >= P) break;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      double x = acc[n][r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0 && r0 + r < nrhs) wb[(long long)(r0 + r) * NP + (long long)f * P + n] += c * x;
    }
  }
}

// Launch both passes with the register tile PT >= max P of the batch.
template <int PT, int RB>
static void dense_passes(const InstDev* di, const double* arena, const double* z, double* w,
                         int nrhs, int ni, int maxN, cudaStream_t st, const int* gate) {
  dim3 g((maxN + 7) / 8, ni, (nrhs + RB - 1) / RB);
  k_dense_rowpass<PT, RB><<<g, 256, 0, st>>>(di, arena, z, w, nrhs, gate);
  HF_LAUNCH_CHECK();
  k_dense_colpass<PT, RB><<<g, 256, 0, st>>>(di, arena, z, w, nrhs, gate);
  HF_LAUNCH_CHECK();
}

void dense_operator(const InstDev* di, const double* arena, const double* z, double* w, int nrhs,
                    int ni, int maxN, int maxP, cudaStream_t st, const int* gate) {
  if (maxP <= 4)
    dense_passes<4, 8>(di, arena, z, w, nrhs, ni, maxN, st, gate);
  else if (maxP <= 8)
    dense_passes<8, 4>(di, arena, z, w, nrhs, ni, maxN, st, gate);
  else if (maxP <= 12)
    dense_passes<12, 4>(di, arena, z, w, nrhs, ni, maxN, st, gate);
  else if (maxP <= 16)
    dense_passes<16, 4>(di, arena, z, w, nrhs, ni, maxN, st, gate);
  else if (maxP <= 24)
    dense_passes<24, 2>(di, arena, z, w, nrhs, ni, maxN, st, gate);
  else
    dense_passes<32, 2>(di, arena, z, w, nrhs, ni, maxN, st, gate);
}

// Dense columns: w[f][n] = theta ylow[f][n] + (1-theta) sum_{e >= f} T[(e,f)][n]
__global__ void k_dense_cols(const InstDev* __restrict__ inst, const double* ylow,
                             const double* T, double* w, int nrhs) {
  const InstDev I = inst[blockIdx.y];
  if (I.kind != kDense) return;
  const int r = blockIdx.z;
  const int P = I.P;
  const long long NP = (long long)I.N * P;
  const long long npair = (long long)I.N * (I.N + 1) / 2;
  const double* Tr = T + I.o_T * nrhs + (size_t)r * npair * P;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < NP;
       t += (long long)gridDim.x * blockDim.x) {
    int f = (int)(t / P), n = (int)(t % P);
    double s = 0.0;
    for (int e = f; e < I.N; ++e) s += Tr[((long long)e * (e + 1) / 2 + f) * P + n];
    long long o = I.o_z * nrhs + r * NP + t;
    w[o] = I.theta * ylow[o] + (1.0 - I.theta) * s;
  }
}

// Toeplitz forward: CTA per (component n, slot, instance * nrhs).  Slot 0
// carries c_k z_k[n] (for theta T C z), slot 1 carries r_k z_k[n] (for
// (1-theta) Tt R z); uniform meshes use slot 0 only.
__global__ void k_toep_fwd(const InstDev* __restrict__ inst, const double* arena,
                           const double* __restrict__ z, double2* F,
                           const double2* tw, int Lmax, int nrhs, const int* __restrict__ gate) {
  extern __shared__ double2 fbuf[];
  HF_GATE(gate);
  const InstDev I = inst[blockIdx.y];
  if (I.kind != kToeplitz) return;
  const int P = I.P;
  const int n = blockIdx.x >> 1, slot = blockIdx.x & 1;
  const int r = blockIdx.z;
  if (n >= P || (slot == 1 && I.uniform)) return;
  const double* zr = z + I.o_z * nrhs + (size_t)r * I.N * P;
  const double* sc = arena + (slot == 0 ? I.o_cs : I.o_rs);
  for (int k = threadIdx.x; k < I.L; k += blockDim.x) {
    double v = 0.0;
    if (k < I.N) v = zr[(size_t)k * P + n] * (I.uniform ? 1.0 : sc[k]);
    fbuf[bitrev(k, I.logL)] = make_double2(v, 0.0);
  }
  __syncthreads();
  fft_core(fbuf, I.L, I.logL, tw, Lmax, 0);
  double2* out = F + (I.o_fft * 2 * nrhs + (size_t)(r * 2 + slot) * P * I.L) + (size_t)n * I.L;
  for (int k = threadIdx.x; k < I.L; k += blockDim.x) out[k] = fbuf[k];
}

// Frequency mixing, in place: slot 0 <- S(w) a(w); slot 1 <- S(w)^H b(w);
// uniform: slot 0 <- (theta S + (1-theta) S^H) a.
__global__ void k_toep_freq(const InstDev* __restrict__ inst, const double2* spec,
                            double2* F, int nrhs, const int* __restrict__ gate) {
  HF_GATE(gate);
  const InstDev I = inst[blockIdx.y];
  if (I.kind != kToeplitz) return;
  const int P = I.P, L = I.L;
  const int r = blockIdx.z;
  const double2* S = spec + I.o_spec;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < L; w += gridDim.x * blockDim.x) {
    double2* F0 = F + I.o_fft * 2 * nrhs + (size_t)(r * 2) * P * L;
    double2* F1 = F0 + (size_t)P * L;
    double2 a[kMaxP], b[kMaxP];
    for (int n = 0; n < P; ++n) a[n] = F0[(size_t)n * L + w];
    if (!I.uniform)
      for (int n = 0; n < P; ++n) b[n] = F1[(size_t)n * L + w];
    for (int m = 0; m < P; ++m) {
      double2 acc0 = make_double2(0.0, 0.0), acc1 = make_double2(0.0, 0.0);
      for (int n = 0; n < P; ++n) {
        double2 smn = S[(size_t)(m * P + n) * L + w];
        double2 snm = S[(size_t)(n * P + m) * L + w];
        double2 snmc = make_double2(snm.x, -snm.y);
        if (I.uniform) {
          double2 c = make_double2(I.theta * smn.x + (1.0 - I.theta) * snmc.x,
                                   I.theta * smn.y + (1.0 - I.theta) * snmc.y);
          double2 t = cmul(c, a[n]);
          acc0.x += t.x;
          acc0.y += t.y;
        } else {
          double2 t0 = cmul(smn, a[n]);
          double2 t1 = cmul(snmc, b[n]);
          acc0.x += t0.x;
          acc0.y += t0.y;
          acc1.x += t1.x;
          acc1.y += t1.y;
        }
      }
      F0[(size_t)m * L + w] = acc0;
      if (!I.uniform) F1[(size_t)m * L + w] = acc1;
    }
  }
}

// Toeplitz inverse: CTA per (component m, instance, rhs); writes w in z-space.
__global__ void k_toep_inv(const InstDev* __restrict__ inst, const double* arena,
                           const double2* F, double* w, const double2* tw,
                           int Lmax, int nrhs, const int* __restrict__ gate) {
  extern __shared__ double2 fbuf[];
  HF_GATE(gate);
  const InstDev I = inst[blockIdx.y];
  if (I.kind != kToeplitz) return;
  const int P = I.P, L = I.L, N = I.N;
  const int m = blockIdx.x, r = blockIdx.z;
  if (m >= P) return;
  double* wr = w + I.o_z * nrhs + (size_t)r * N * P;
  const double* rs = arena + I.o_rs;
  const double* cs = arena + I.o_cs;
  const double invL = 1.0 / L;
  for (int slot = 0; slot < (I.uniform ? 1 : 2); ++slot) {
    const double2* in = F + I.o_fft * 2 * nrhs + (size_t)(r * 2 + slot) * P * L + (size_t)m * L;
    for (int k = threadIdx.x; k < L; k += blockDim.x) fbuf[bitrev(k, I.logL)] = in[k];
    __syncthreads();
    fft_core(fbuf, L, I.logL, tw, Lmax, 1);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      double v = fbuf[k].x * invL;
      if (I.uniform)
        wr[(size_t)k * P + m] = rs[0] * cs[0] * v;
      else if (slot == 0)
        wr[(size_t)k * P + m] = I.theta * rs[k] * v;
      else
        wr[(size_t)k * P + m] += (1.0 - I.theta) * cs[k] * v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// load vector
// ---------------------------------------------------------------------------
// Legendre moments g_e[m] = int_{I_e} f L_m(xi_e) dx, m = 0..P, per
// (element, rhs) thread.  rhs layout: per instance, nrhs blocks of `stride`
// doubles starting at roff[inst].
__global__ void k_load_moments(const InstDev* __restrict__ inst, const double* arena,
                               const double* __restrict__ gl, const double* rhsdata,
                               const long long* roff, int kind, int n_terms,
                               int nrhs, double* mom) {
  const InstDev I = inst[blockIdx.y];
  const int r = blockIdx.z;
  const int P = I.P, N = I.N;
  const double* h = arena + I.o_h;
  const double* dl = arena + I.o_dl;
  const double* dr = arena + I.o_dr;
  const double Lab = dl[N];
  n_terms = (int)roff[2 * blockIdx.y + 1];
  const int stride = (kind == HFSEM_RHS_FRAC_POWERS) ? 3 * n_terms : n_terms;
  const double* rd = rhsdata + roff[2 * blockIdx.y] + (size_t)r * stride;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    double g[kMaxP + 1];
    for (int m = 0; m <= P; ++m) g[m] = 0.0;
    const double he = h[e];
    if (kind == HFSEM_RHS_LEGENDRE_AB) {
      int K = n_terms - 1;
      int nq = min((K + P) / 2 + 2, kMaxGL);
      const double* X = gl + gl_off(nq);
      const double* Wt = X + nq;
      for (int q = 0; q < nq; ++q) {
        double y = dl[e] + 0.5 * he * (1.0 + X[q]);   // x - a
        double s = -1.0 + 2.0 * y / Lab;
        double p0 = 1.0, p1 = s, fv = rd[0];
        if (K >= 1) fv += rd[1] * s;
        for (int k = 1; k < K; ++k) {
          double p2 = leg_next(k, s, p1, p0);
          fv += rd[k + 1] * p2;
          p0 = p1;
          p1 = p2;
        }
        double wq = 0.5 * he * Wt[q] * fv;
        double l0 = 1.0, l1 = X[q];
        g[0] += wq;
        if (P >= 1) g[1] += wq * l1;
        for (int k = 1; k < P; ++k) {
          double l2 = leg_next(k, X[q], l1, l0);
          g[k + 1] += wq * l2;
          l0 = l1;
          l1 = l2;
        }
      }
    } else {  // fractional powers
      // Terms whose element lies at least half its length from their
      // endpoint share one Gauss-Legendre rule per side, with enough points
      // for the Bernstein ellipse through the singularity 2 d0 / h beyond
      // the end of the reference interval (error ~ rho^-(2n - P), kept below
      // 1e-16): (d0 + o)^mu = d0^mu (1 + o/d0)^mu, the power of d0 once per
      // term and element, the second factor exp(mu log1p(o/d0)) per point
      // with log1p(o/d0) in [0, log 3] (a few ulp), and the Legendre values
      // once per point for a chunk of terms.
      constexpr int kTermChunk = 8;
      for (int side = 0; side < 2; ++side) {
        const double d0 = (side == 0) ? dl[e] : dr[e + 1];
        if (!(d0 >= 0.5 * he)) continue;
        const double tt = 1.0 + 2.0 * d0 / he;
        const double rho = tt + sqrt(tt * tt - 1.0);
        const int nq = min((int)ceil(0.5 * P + 18.5 / log(rho)) + 2, kMaxGL);
        const double* X = gl + gl_off(nq);
        const double* Wt = X + nq;
        const double id0 = 1.0 / d0;
        for (int t0 = 0; t0 < n_terms; t0 += kTermChunk) {
          double cp[kTermChunk], mu[kTermChunk];
          int nt = 0;
          for (int t = t0; t < min(n_terms, t0 + kTermChunk); ++t)
            if ((int)rd[3 * t + 2] == side) {
              mu[nt] = rd[3 * t + 1];
              cp[nt] = rd[3 * t] * pow(d0, mu[nt]);
              ++nt;
            }
          if (nt == 0) continue;
          for (int q = 0; q < nq; ++q) {
            const double o = 0.5 * he * (1.0 + X[q]);   // offset from the node nearest the end
            const double lg = log1p(o * id0);
            double S = 0.0;
            for (int j = 0; j < nt; ++j) S += cp[j] * exp(mu[j] * lg);
            const double wq = 0.5 * he * Wt[q] * S;
            const double xi = (side == 0) ? X[q] : -X[q];
            double l0 = 1.0, l1 = xi;
            g[0] += wq;
            if (P >= 1) g[1] += wq * l1;
            for (int k = 1; k < P; ++k) {
              double l2 = leg_next(k, xi, l1, l0);
              g[k + 1] += wq * l2;
              l0 = l1;
              l1 = l2;
            }
          }
        }
      }
      for (int t = 0; t < n_terms; ++t) {
        double coef = rd[3 * t], mu = rd[3 * t + 1];
        int side = (int)rd[3 * t + 2];
        double d0 = (side == 0) ? dl[e] : dr[e + 1];
        if (d0 == 0.0) {
          // end element: int (1 +- xi)^mu L_m dxi by the ratio recurrence
          // c_0 = 2^(mu+1)/(mu+1), c_{m+1} = c_m (mu - m)/(mu + m + 2)
          double scale = coef * pow(0.5 * he, mu + 1.0);
          double c = exp2(mu + 1.0) / (mu + 1.0);
          for (int m = 0; m <= P; ++m) {
            double sgn = (side == 1 && (m & 1)) ? -1.0 : 1.0;
            g[m] += scale * sgn * c;
            c *= (mu - m) / (mu + m + 2.0);
          }
        } else if (d0 >= 0.5 * he) {
          continue;   // done above
        } else {
          // offset o from the node nearest the endpoint, distance d0 + o;
          // exponential map o = d0((1+h/d0)^s - 1), s in [0,1], makes the
          // integrand smooth whatever h/d0 is
          int nq = min(24 + 2 * P, kMaxGL);
          const double* X = gl + gl_off(nq);
          const double* Wt = X + nq;
          double lr = log1p(he / d0);
          for (int q = 0; q < nq; ++q) {
            double sq = 0.5 * (1.0 + X[q]);
            double ex = exp(sq * lr);
            double dist = d0 * ex;                 // d0 + o
            double o = d0 * expm1(sq * lr);
            double jac = 0.5 * Wt[q] * d0 * lr * ex;  // do = d0 lr e^{s lr} ds
            double wq = coef * jac * pow(dist, mu);
            double xi = (side == 0) ? -1.0 + 2.0 * o / he : 1.0 - 2.0 * o / he;
            double l0 = 1.0, l1 = xi;
            g[0] += wq;
            if (P >= 1) g[1] += wq * l1;
            for (int k = 1; k < P; ++k) {
              double l2 = leg_next(k, xi, l1, l0);
              g[k + 1] += wq * l2;
              l0 = l1;
              l1 = l2;
            }
          }
        }
      }
    }
    // moments of instance i: (o_z + o_N) * nrhs + r N (P+1) + e (P+1)
    double* gout = mom + (size_t)(I.o_z + I.o_N) * nrhs + (size_t)r * N * (P + 1) +
                   (size_t)e * (P + 1);
    for (int m = 0; m <= P; ++m) gout[m] = g[m];
  }
}

// G from the moments: bubble (e,p): g_e[p-1] - g_e[p+1];
// hat j: (g_{j-1}[0] + g_{j-1}[1])/2 + (g_j[0] - g_j[1])/2.
__global__ void k_load_scatter(const InstDev* __restrict__ inst, const double* mom,
                               double* G, int nrhs) {
  const InstDev I = inst[blockIdx.y];
  const int r = blockIdx.z;
  const int P = I.P, N = I.N;
  const double* g = mom + (size_t)(I.o_z + I.o_N) * nrhs + (size_t)r * N * (P + 1);
  double* Gv = G + I.o_vec * nrhs + (size_t)r * I.Nd;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.Nd; i += gridDim.x * blockDim.x) {
    int e = i / P, p = i % P + 1;
    double v;
    if (p < P) {
      v = g[e * (P + 1) + p - 1] - g[e * (P + 1) + p + 1];
    } else {
      int j = e + 1;
      v = 0.5 * (g[(j - 1) * (P + 1)] + g[(j - 1) * (P + 1) + 1]) +
          0.5 * (g[j * (P + 1)] - g[j * (P + 1) + 1]);
    }
    Gv[i] = v;
  }
}

// ---------------------------------------------------------------------------
// orderings: X of Sec. 2.2 <-> element-major
// ---------------------------------------------------------------------------
__device__ __forceinline__ int paper_index(int i, int N, int P) {
  int e = i / P, p = i % P + 1;
  return (p < P) ? e * (P - 1) + p - 1 : N * (P - 1) + e;   // hat j = e+1 -> N(P-1) + j-1
}

__global__ void k_perm(const InstDev* __restrict__ inst, const double* __restrict__ in,
                       double* out, int nrhs, int to_elem) {
  const InstDev I = inst[blockIdx.y];
  const int r = blockIdx.z;
  const size_t base = I.o_vec * nrhs + (size_t)r * I.Nd;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.Nd; i += gridDim.x * blockDim.x) {
    int pi = paper_index(i, I.N, I.P);
    if (to_elem)
      out[base + i] = in[base + pi];
    else
      out[base + pi] = in[base + i];
  }
}

__global__ void k_axpy_sub(double* y, const double* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] -= x[i];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int ceil_log2(long long v) {
  int l = 0;
  while ((1LL << l) < v) ++l;
  return l;
}

static dim3 grid1(long long n, int bs, int y, int z) {
  long long g = (n + bs - 1) / bs;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return dim3((unsigned)g, (unsigned)y, (unsigned)z);
}

static std::vector<double>& gl_table_host() {
  static std::vector<double> tab;
  static std::once_flag once;
  std::call_once(once, [] {
    tab.assign((size_t)gl_off(kMaxGL + 1), 0.0);
    for (int n = 1; n <= kMaxGL; ++n) {
      std::vector<double> x, w;
      gauss_legendre_rule(n, x, w);
      for (int i = 0; i < n; ++i) {
        tab[gl_off(n) + i] = x[i];
        tab[gl_off(n) + n + i] = w[i];
      }
    }
  });
  return tab;
}

void ensure_work(hfsem_system* s, int nrhs) {
  size_t nd = (size_t)s->total_nd * nrhs, nz = (size_t)s->total_nz * nrhs;
  s->w_x.ensure(nd);
  s->w_y.ensure(nd);
  s->w_z.ensure(nz);
  s->w_w.ensure(nz);

  if (s->any_toep) s->w_fa.ensure((size_t)s->total_fft * 2 * nrhs);
}

static void launch_twiddles(hfsem_system* s) {
  if (s->tw_L >= s->max_L) return;
  s->tw_L = s->max_L;
  s->tw.alloc((size_t)s->tw_L / 2);
  k_twiddles<<<64, 256, 0, s->st>>>(s->tw.p, s->tw_L);
  HF_LAUNCH_CHECK();
}

static void set_smem(const void* fn, size_t bytes) { allow_dyn_smem(fn, bytes); }

void allow_dyn_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;   // (device, kernel) -> set
  int dev = 0;
  HF_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_pair(dev, fn);
  auto it = limit.find(key);
  if (it != limit.end() && it->second >= bytes) return;
  int optin = 0;
  HF_CHECK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  HF_CHECK(cudaFuncGetAttributes(&fa, fn));
  const size_t most = (size_t)optin - fa.sharedSizeBytes;
  if (bytes > most) throw Error(HFSEM_ERR_UNSUPPORTED, "kernel needs more shared memory than the device has");
  HF_CHECK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most));
  limit[key] = most;
}

void apply_operator(hfsem_system* s, int nrhs, const double* x, double* y, int lift) {
  ensure_work(s, nrhs);
  const int ni = s->n_inst;
  const InstDev* di = s->d_inst.p;
  double* z = s->w_z.p;
  double* w = s->w_w.p;
  k_gather_z<<<grid1((long long)s->max_N * s->max_P, 256, ni, nrhs), 256, 0, s->st>>>(
      di, s->arena.p, x, z, nrhs, lift, s->gate);
  HF_LAUNCH_CHECK();
  if (s->any_dense) {
    // algorithmic work: 2 multiply-adds per stored entry and right-hand side
    double flops = 0.0;
    for (auto& I : s->ih)
      if (I.kind == kDense) flops += 4.0 * I.P * I.P * I.N * (I.N + 1) / 2.0 * nrhs;
    Tick tk(s->st, "dense_mv", flops);
    dense_operator(di, s->arena.p, z, w, nrhs, ni, s->max_N, s->max_P, s->st, s->gate);
  }
  if (s->any_toep) {
    double bytes = 0.0;   // symbol read + z in + w out
    for (auto& D : s->idv)
      if (D.kind == kToeplitz) bytes += 16.0 * D.L * D.P * D.P + 2.0 * 8.0 * nrhs * D.N * D.P;
    Tick tk(s->st, "toeplitz_mv", bytes);
    size_t sm = (size_t)s->max_L * sizeof(double2);
    set_smem((const void*)k_toep_fwd, sm);
    set_smem((const void*)k_toep_inv, sm);
    k_toep_fwd<<<dim3(2 * s->max_P, ni, nrhs), 256, sm, s->st>>>(di, s->arena.p, z, s->w_fa.p,
                                                                 s->tw.p, s->tw_L, nrhs, s->gate);
    HF_LAUNCH_CHECK();
    k_toep_freq<<<grid1(s->max_L, 128, ni, nrhs), 128, 0, s->st>>>(di, s->spec.p, s->w_fa.p,
                                                                    nrhs, s->gate);
    HF_LAUNCH_CHECK();
    k_toep_inv<<<dim3(s->max_P, ni, nrhs), 256, sm, s->st>>>(di, s->arena.p, s->w_fa.p, w,
                                                             s->tw.p, s->tw_L, nrhs, s->gate);
    HF_LAUNCH_CHECK();
  }
  if (s->any_hmat) {
    k_lift_hmat<<<grid1((long long)s->max_N * s->max_P, 256, ni, nrhs), 256, 0, s->st>>>(
        di, s->arena.p, z, w, nrhs, s->gate);
    HF_LAUNCH_CHECK();
  }
  k_scatter_out<<<grid1((long long)s->max_N * s->max_P, 256, ni, nrhs), 256, 0, s->st>>>(
      di, s->arena.p, w, x, y, nrhs, lift, s->gate);
  HF_LAUNCH_CHECK();
  if (s->any_hmat) hop_apply(s, nrhs, x, y);   // y += A x on the kHmat instances
}

void perm_to_elem(hfsem_system* s, int nrhs, const double* xp, double* xe) {
  k_perm<<<grid1((long long)s->max_N * s->max_P, 256, s->n_inst, nrhs), 256, 0, s->st>>>(
      s->d_inst.p, xp, xe, nrhs, 1);
  HF_LAUNCH_CHECK();
}

void perm_to_paper(hfsem_system* s, int nrhs, const double* xe, double* xp) {
  k_perm<<<grid1((long long)s->max_N * s->max_P, 256, s->n_inst, nrhs), 256, 0, s->st>>>(
      s->d_inst.p, xe, xp, nrhs, 0);
  HF_LAUNCH_CHECK();
}

// Check rhs structs; returns nrhs.
static int check_rhs(hfsem_system* s, const hfsem_rhs* rhs) {
  if (!rhs) throw Error(HFSEM_ERR_INVALID_ARG, "rhs is NULL");
  int nrhs = rhs[0].nrhs;
  if (nrhs < 1 || nrhs > 64) throw Error(HFSEM_ERR_INVALID_ARG, "nrhs must be in [1, 64]");
  for (int i = 0; i < s->n_inst; ++i) {
    const hfsem_rhs& R = rhs[i];
    if (R.nrhs != nrhs) throw Error(HFSEM_ERR_INVALID_ARG, "nrhs differs between instances");
    if (R.kind != rhs[0].kind)
      throw Error(HFSEM_ERR_INVALID_ARG, "rhs kind differs between instances");
    if (!R.data) throw Error(HFSEM_ERR_INVALID_ARG, "rhs data is NULL");
    if (R.kind == HFSEM_RHS_FRAC_POWERS) {
      if (R.n_terms < 1 || R.n_terms > 4096)
        throw Error(HFSEM_ERR_INVALID_ARG, "FRAC_POWERS: 1 <= n_terms <= 4096");
      for (int k = 0; k < R.n_terms * nrhs; ++k) {
        double mu = R.data[3 * k + 1], side = R.data[3 * k + 2];
        if (!(mu > -1.0) || !(side == 0.0 || side == 1.0))
          throw Error(HFSEM_ERR_INVALID_ARG, "FRAC_POWERS: exponent > -1, side 0 or 1");
      }
    } else if (R.kind == HFSEM_RHS_LEGENDRE_AB) {
      if (R.n_terms < 1 || R.n_terms > 128)
        throw Error(HFSEM_ERR_INVALID_ARG, "LEGENDRE_AB: 1 <= K+1 <= 128");
    } else if (R.kind != HFSEM_RHS_LOAD_VECTOR) {
      throw Error(HFSEM_ERR_INVALID_ARG, "unknown rhs kind");
    }
  }
  return nrhs;
}

void load_vector_em(hfsem_system* s, const hfsem_rhs* rhs, int lifted, double* G_em) {
  int nrhs = check_rhs(s, rhs);
  ensure_work(s, nrhs);
  const int ni = s->n_inst;
  const int kind = rhs[0].kind;
  if (kind == HFSEM_RHS_LOAD_VECTOR) {
    // host data in X's ordering -> device -> element-major
    std::vector<double> buf((size_t)s->total_nd * nrhs);
    size_t off = 0;
    for (int i = 0; i < ni; ++i) {
      size_t cnt = (size_t)s->ih[i].Nd * nrhs;
      std::memcpy(buf.data() + off, rhs[i].data, cnt * sizeof(double));
      off += cnt;
    }
    HF_CHECK(cudaMemcpyAsync(s->w_y.p, buf.data(), buf.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s->st));
    HF_CHECK(cudaStreamSynchronize(s->st));
    perm_to_elem(s, nrhs, s->w_y.p, G_em);
  } else {
    std::vector<double> buf;
    std::vector<long long> roff(2 * ni);   // per instance: data offset, n_terms
    for (int i = 0; i < ni; ++i) {
      int stride = (kind == HFSEM_RHS_FRAC_POWERS) ? 3 * rhs[i].n_terms : rhs[i].n_terms;
      roff[2 * i] = (long long)buf.size();
      roff[2 * i + 1] = rhs[i].n_terms;
      buf.insert(buf.end(), rhs[i].data, rhs[i].data + (size_t)stride * nrhs);
    }
    size_t nb = buf.size() + (size_t)2 * ni + 2;
    s->w_rhsdata.ensure(nb);
    HF_CHECK(cudaMemcpyAsync(s->w_rhsdata.p, buf.data(), buf.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s->st));
    long long* d_roff = reinterpret_cast<long long*>(s->w_rhsdata.p + buf.size());
    HF_CHECK(cudaMemcpyAsync(d_roff, roff.data(), 2 * ni * sizeof(long long),
                             cudaMemcpyHostToDevice, s->st));
    const int n_terms = 0;   // per instance, from the table
    // moments: sum over instances of N (P+1) = total_nz + sum N, per rhs
    s->w_mom.ensure((size_t)(s->total_nz + s->total_N) * nrhs);
    Tick tk(s->st, "load_vector");
    k_load_moments<<<grid1(s->max_N, 128, ni, nrhs), 128, 0, s->st>>>(
        s->d_inst.p, s->arena.p, s->gl.p, s->w_rhsdata.p, d_roff, kind, n_terms, nrhs,
        s->w_mom.p);
    HF_LAUNCH_CHECK();
    k_load_scatter<<<grid1((long long)s->max_N * s->max_P, 256, ni, nrhs), 256, 0, s->st>>>(
        s->d_inst.p, s->w_mom.p, G_em, nrhs);
    HF_LAUNCH_CHECK();
    HF_CHECK(cudaStreamSynchronize(s->st));   // host staging buffer lifetime
  }
  if (lifted) {
    bool any = false;
    for (auto& I : s->ih) any = any || I.c1 != 0.0 || I.c2 != 0.0;
    if (any) {
      HF_CHECK(cudaMemsetAsync(s->w_x.p, 0, (size_t)s->total_nd * nrhs * sizeof(double), s->st));
      apply_operator(s, nrhs, s->w_x.p, s->w_y.p, 1);
      long long n = s->total_nd * nrhs;
      k_axpy_sub<<<grid1(n, 256, 1, 1), 256, 0, s->st>>>(G_em, s->w_y.p, n);
      HF_LAUNCH_CHECK();
    }
  }
}

static void validate(const hfsem_problem& p) {
  if (p.matvec < HFSEM_MATVEC_AUTO || p.matvec > HFSEM_MATVEC_HMATRIX)
    throw Error(HFSEM_ERR_INVALID_ARG, "unknown matvec kind");
  if (p.n_elem < 1) throw Error(HFSEM_ERR_INVALID_ARG, "n_elem must be >= 1");
  if (p.P < 1 || p.P > kMaxP) throw Error(HFSEM_ERR_INVALID_ARG, "P must be in [1, 32]");
  if (!(p.alpha > 1.0 && p.alpha < 2.0)) throw Error(HFSEM_ERR_INVALID_ARG, "alpha must be in (1, 2)");
  if (!(p.theta >= 0.0 && p.theta <= 1.0)) throw Error(HFSEM_ERR_INVALID_ARG, "theta must be in [0, 1]");
  if (!(p.rho >= 0.0) || !std::isfinite(p.rho)) throw Error(HFSEM_ERR_INVALID_ARG, "rho must be >= 0");
  if (!std::isfinite(p.c1) || !std::isfinite(p.c2)) throw Error(HFSEM_ERR_INVALID_ARG, "c1, c2 finite");
  if (!(p.b > p.a) || !std::isfinite(p.a) || !std::isfinite(p.b))
    throw Error(HFSEM_ERR_INVALID_ARG, "need a < b");
  if (!p.h) throw Error(HFSEM_ERR_INVALID_ARG, "h is NULL");
  double sum = 0.0;
  for (int i = 0; i < p.n_elem; ++i) {
    if (!(p.h[i] > 0.0) || !std::isfinite(p.h[i]))
      throw Error(HFSEM_ERR_INVALID_ARG, "element lengths must be positive");
    sum += p.h[i];
  }
  if (std::fabs(sum - (p.b - p.a)) > 1e-12 * (p.b - p.a))
    throw Error(HFSEM_ERR_INVALID_ARG, "sum of h differs from b - a");
}

static hfsem_system* assemble(int n, const hfsem_problem* probs, void* stream) {
  if (n < 1 || !probs) throw Error(HFSEM_ERR_INVALID_ARG, "n_inst >= 1 and probs required");
  for (int i = 0; i < n; ++i) validate(probs[i]);
  auto* s = new hfsem_system();
  try {
    s->st = (cudaStream_t)stream;
    AllocStream as(s->st);   // the system's buffers come stream-ordered from the pool
    s->n_inst = n;
    s->ih.resize(n);
    s->idv.resize(n);
    long long arena = 0, spec = 0;
    for (int i = 0; i < n; ++i) {
      const hfsem_problem& p = probs[i];
      InstHost& I = s->ih[i];
      InstDev& D = s->idv[i];
      std::memset(&D, 0, sizeof(D));
      I.N = p.n_elem;
      I.P = p.P;
      I.Nd = I.N * I.P - 1;
      I.a = p.a;
      I.b = p.b;
      I.alpha = p.alpha;
      I.theta = p.theta;
      I.rho = p.rho;
      I.c1 = p.c1;
      I.c2 = p.c2;
      I.g0 = 1.0 / std::tgamma(2.0 - p.alpha);
      I.h.assign(p.h, p.h + I.N);
      I.dl.assign(I.N + 1, 0.0);
      I.dr.assign(I.N + 1, 0.0);
      for (int k = 0; k < I.N; ++k) I.dl[k + 1] = I.dl[k] + I.h[k];
      for (int k = I.N - 1; k >= 0; --k) I.dr[k] = I.dr[k + 1] + I.h[k];
      // constant ratio h_{i+1}/h_i ?
      bool geo = true;
      double q = (I.N > 1) ? I.h[1] / I.h[0] : 1.0;
      for (int k = 1; k < I.N; ++k)
        if (std::fabs(I.h[k] / I.h[k - 1] - q) > 1e-12 * q) geo = false;
      double hmax = *std::max_element(I.h.begin(), I.h.end());
      double hmin = *std::min_element(I.h.begin(), I.h.end());
      I.uniform = geo && (hmax - hmin) <= 1e-13 * hmax;
      I.q = q;
      if (p.matvec == HFSEM_MATVEC_TOEPLITZ && !geo)
        throw Error(HFSEM_ERR_INVALID_ARG, "Toeplitz operator needs h_{i+1}/h_i constant");
      bool toep = (p.matvec == HFSEM_MATVEC_TOEPLITZ) ||
                  (p.matvec == HFSEM_MATVEC_AUTO && geo && hmax <= 16.0 * hmin && I.N >= 2);
      I.kind = toep ? kToeplitz : (p.matvec == HFSEM_MATVEC_HMATRIX ? kHmat : kDense);
      D.N = I.N;
      D.P = I.P;
      D.Nd = I.Nd;
      D.kind = I.kind;
      D.alpha = I.alpha;
      D.theta = I.theta;
      D.rho = I.rho;
      D.c1 = I.c1;
      D.c2 = I.c2;
      D.g0 = I.g0;
      D.uniform = I.uniform ? 1 : 0;
      D.n_gj = I.P + 1;
      D.o_h = arena;
      arena += I.N;
      D.o_dl = arena;
      arena += I.N + 1;
      D.o_dr = arena;
      arena += I.N + 1;
      D.o_D = arena;
      arena += (long long)I.P * I.P;
      D.o_gj = arena;
      arena += 2 * D.n_gj;
      D.o_rs = arena;
      arena += I.N;
      D.o_cs = arena;
      arena += I.N;
      if (I.kind == kHmat) {
        // the pairs the operator's near field needs (a band per row e), the
        // boundary column f = 0 and row e = N-1 (lifting), and their tables
        hop_band(I, I.flo);
        long long band = 0;
        for (int e = 0; e < I.N; ++e) band += e - I.flo[e] + 1;
        D.band = band;
        D.o_flo = arena;
        arena += I.N;
        D.o_off = arena;
        arena += I.N + 1;
        D.o_c0 = arena;
        arena += (long long)I.N * I.P;
        D.o_rN = arena;
        arena += (long long)I.N * I.P;
        D.o_M = arena;
        arena += band * I.P * I.P;
      } else {
        D.o_M = arena;
        long long nblk = (I.kind == kDense) ? (long long)I.N * (I.N + 1) / 2 : I.N;
        arena += nblk * I.P * I.P;
      }
      D.o_vec = s->total_nd;
      D.o_z = s->total_nz;
      D.o_N = s->total_N;
      s->total_N += I.N;
      s->total_nd += I.Nd;
      s->total_nz += (long long)I.N * I.P;
      if (I.kind == kDense) {
        D.o_T = s->total_T;
        s->total_T += (long long)I.N * (I.N + 1) / 2 * I.P;
        s->any_dense = true;
      } else if (I.kind == kHmat) {
        s->any_hmat = true;
      } else {
        D.logL = ceil_log2(2LL * I.N);
        D.L = 1 << D.logL;
        D.o_spec = spec;
        spec += (long long)D.L * I.P * I.P;
        D.o_fft = s->total_fft;
        s->total_fft += (long long)D.L * I.P;
        s->any_toep = true;
        s->max_L = std::max(s->max_L, D.L);
      }
      s->max_P = std::max(s->max_P, I.P);
      s->max_N = std::max(s->max_N, I.N);
    }
    s->arena.alloc((size_t)arena);
    if (spec) s->spec.alloc((size_t)spec);
    // host staging of geometry, rules and scalings
    std::vector<double> host((size_t)arena, 0.0);
    for (int i = 0; i < n; ++i) {
      InstHost& I = s->ih[i];
      InstDev& D = s->idv[i];
      std::copy(I.h.begin(), I.h.end(), host.begin() + D.o_h);
      std::copy(I.dl.begin(), I.dl.end(), host.begin() + D.o_dl);
      std::copy(I.dr.begin(), I.dr.end(), host.begin() + D.o_dr);
      std::vector<double> x, w;
      gauss_jacobi_rule(D.n_gj, 0.0, 2.0 - I.alpha, x, w);
      std::copy(x.begin(), x.end(), host.begin() + D.o_gj);
      std::copy(w.begin(), w.end(), host.begin() + D.o_gj + D.n_gj);
      // Toeplitz row / column scalings of the stored (divided) blocks:
      // M_ef / (h_e h_f) = (1/2) (g0/2 h_f^(1-alpha)) m_{e-f}
      for (int k = 0; k < I.N; ++k) {
        host[D.o_rs + k] = 0.5;
        host[D.o_cs + k] = I.g0 * 0.5 * std::pow(I.h[k], 1.0 - I.alpha);
      }
      if (I.kind == kHmat) {
        long long off = 0;
        for (int e = 0; e < I.N; ++e) {
          host[D.o_flo + e] = I.flo[e];
          host[D.o_off + e] = (double)off;
          off += e - I.flo[e] + 1;
        }
        host[D.o_off + I.N] = (double)off;
      }
    }
    HF_CHECK(cudaMemcpyAsync(s->arena.p, host.data(), host.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s->st));
    s->d_inst.alloc(n);
    HF_CHECK(cudaMemcpyAsync(s->d_inst.p, s->idv.data(), n * sizeof(InstDev),
                             cudaMemcpyHostToDevice, s->st));
    std::vector<double>& tab = gl_table_host();
    s->gl.alloc(tab.size());
    HF_CHECK(cudaMemcpyAsync(s->gl.p, tab.data(), tab.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s->st));
    k_selfblock<<<n, 128, 0, s->st>>>(s->d_inst.p, s->arena.p);
    HF_LAUNCH_CHECK();
    int wpc = (s->max_P <= 16) ? 4 : 2;
    int stride = pair_scratch_doubles(s->max_P);
    size_t sm = (size_t)wpc * stride * sizeof(double);
    set_smem((const void*)k_pairs, sm);
    long long maxpairs = 1;
    for (size_t i = 0; i < s->ih.size(); ++i) {
      const InstHost& I = s->ih[i];
      const long long np = I.kind == kDense  ? (long long)I.N * (I.N + 1) / 2
                           : I.kind == kHmat ? s->idv[i].band + 2LL * I.N
                                             : (long long)I.N;
      maxpairs = std::max(maxpairs, np);
    }
    long long gx = std::min<long long>((maxpairs + wpc - 1) / wpc, 65535);
    Tick tk(s->st, "pairs");
    k_pairs<<<dim3((unsigned)gx, n), wpc * 32, sm, s->st>>>(s->d_inst.p, s->arena.p, s->gl.p,
                                                           wpc, stride);
    HF_LAUNCH_CHECK();
    if (s->any_toep) {
      launch_twiddles(s);
      size_t fsm = (size_t)s->max_L * sizeof(double2);
      set_smem((const void*)k_symbol, fsm);
      k_symbol<<<dim3(s->max_P * s->max_P, n), 256, fsm, s->st>>>(s->d_inst.p, s->arena.p,
                                                                  s->spec.p, s->tw.p, s->tw_L);
      HF_LAUNCH_CHECK();
    }
    if (s->any_hmat) build_operator(s);
    HF_CHECK(cudaStreamSynchronize(s->st));
  } catch (...) {
    drain_after_error(s);
    delete s;
    throw;
  }
  return s;
}

// Run body with exceptions turned into status codes.
template <class F>
static int guarded(F&& body) {
  try {
    body();
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

// Copy a caller vector (host or device) into a device buffer.
static void stage_in(hfsem_system* s, const double* src, double* dst, size_t count) {
  HF_CHECK(cudaMemcpyAsync(dst, src, count * sizeof(double),
                           is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s->st));
}
static void stage_out(hfsem_system* s, const double* src, double* dst, size_t count) {
  HF_CHECK(cudaMemcpyAsync(dst, src, count * sizeof(double),
                           is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           s->st));
}

}  // namespace hf

using namespace hf;

namespace hf {
size_t system_bytes(const hfsem_system* s) {
  auto b = [](const auto& d) { return d.n * sizeof(*d.p); };
  return b(s->d_inst) + b(s->arena) + b(s->spec) + b(s->gl) + b(s->w_x) + b(s->w_y) + b(s->w_z) +
         b(s->w_w) + b(s->w_T) + b(s->w_ylow) + b(s->w_mom) + b(s->w_fa) + b(s->w_fb) +
         b(s->w_rhsdata) + b(s->tw) + b(s->kry.vecs) + b(s->kry.partial) + b(s->kry.bx) +
         b(s->kry.coff) + b(s->kry.clen) + b(s->kry.flag) + b(s->kry.cols) + b(s->w_hop) +
         (s->hop ? factor_bytes(s->hop) : 0);
}
}  // namespace hf

extern "C" {

int hfsem_assemble(int32_t n_inst, const hfsem_problem* probs, void* stream,
                   hfsem_system** out) {
  return guarded([&] {
    if (!out) throw Error(HFSEM_ERR_INVALID_ARG, "out is NULL");
    hfsem_system* s = assemble(n_inst, probs, stream);
    try {
      noalloc_prepare();
    } catch (...) {
      drain_after_error(s);
      delete s;
      throw;
    }
    *out = s;
  });
}

int hfsem_ndof(const hfsem_system* sys, int32_t inst, int32_t* nd) {
  return guarded([&] {
    if (!sys || !nd || inst < 0 || inst >= sys->n_inst)
      throw Error(HFSEM_ERR_INVALID_ARG, "bad system / instance");
    *nd = sys->ih[inst].Nd;
  });
}

int hfsem_apply(hfsem_system* sys, int32_t nrhs, const double* x, double* y) {
  return guarded([&] {
    if (!sys || !x || !y || nrhs < 1 || nrhs > 64)
      throw Error(HFSEM_ERR_INVALID_ARG, "bad arguments to hfsem_apply");
    AllocStream as(sys->st);
    ensure_work(sys, nrhs);
    size_t cnt = (size_t)sys->total_nd * nrhs;
    DevBuf<double> xe, ye;
    xe.alloc(cnt);
    ye.alloc(cnt);
    stage_in(sys, x, sys->w_y.p, cnt);
    perm_to_elem(sys, nrhs, sys->w_y.p, xe.p);
    apply_operator(sys, nrhs, xe.p, ye.p, 0);
    perm_to_paper(sys, nrhs, ye.p, sys->w_y.p);
    stage_out(sys, sys->w_y.p, y, cnt);
    HF_CHECK(cudaStreamSynchronize(sys->st));
  });
}

int hfsem_load_vector(hfsem_system* sys, const hfsem_rhs* rhs, int32_t lifted, double* G) {
  return guarded([&] {
    if (!sys || !rhs || !G) throw Error(HFSEM_ERR_INVALID_ARG, "bad arguments");
    int nrhs = rhs[0].nrhs;
    if (nrhs < 1 || nrhs > 64) throw Error(HFSEM_ERR_INVALID_ARG, "nrhs must be in [1, 64]");
    size_t cnt = (size_t)sys->total_nd * nrhs;
    AllocStream as(sys->st);
    DevBuf<double> ge;
    ge.alloc(cnt);
    load_vector_em(sys, rhs, lifted, ge.p);
    perm_to_paper(sys, nrhs, ge.p, sys->w_y.p);
    stage_out(sys, sys->w_y.p, G, cnt);
    HF_CHECK(cudaStreamSynchronize(sys->st));
  });
}


void hfsem_system_free(hfsem_system* sys) {
  if (!sys) return;
  cudaStreamSynchronize(sys->st);
  if (sys->hop) hfsem_factor_free(sys->hop);
  sys->hop = nullptr;
  delete sys;
}

const char* hfsem_status_str(int status) {
  switch (status) {
    case HFSEM_OK: return "ok";
    case HFSEM_ERR_INVALID_ARG: return "invalid argument";
    case HFSEM_ERR_OOM: return "out of device memory";
    case HFSEM_ERR_NOT_CONVERGED: return "not converged";
    case HFSEM_ERR_BREAKDOWN: return "Krylov breakdown";
    case HFSEM_ERR_TIMEOUT: return "device wait limit reached";
    case HFSEM_ERR_DEVICE: return "CUDA device error";
    case HFSEM_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* hfsem_last_error(void) { return hf::g_last_error.c_str(); }

int hfsem_timing_enable(int32_t on) {
  return guarded([&] {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_timing = on != 0;
  });
}

int hfsem_timing_reset(void) {
  return guarded([&] {
    std::lock_guard<std::mutex> lk(g_tmu);
    flush_pending();
    g_tim.clear();
  });
}

int hfsem_timing_read(const char* tag, double* total_ms, int64_t* launches, double* work) {
  return guarded([&] {
    if (!tag) throw Error(HFSEM_ERR_INVALID_ARG, "hfsem_timing_read: tag is NULL");
    std::lock_guard<std::mutex> lk(g_tmu);
    flush_pending();
    if (std::string(tag) == "launches") {   // kernels launched so far
      if (total_ms) *total_ms = 0.0;
      if (launches) *launches = g_launches;
      if (work) *work = 0.0;
      return;
    }
    auto it = g_tim.find(tag);
    TimerRec r = (it == g_tim.end()) ? TimerRec() : it->second;
    if (total_ms) *total_ms = r.ms;
    if (launches) *launches = r.launches;
    if (work) *work = r.work;
  });
}

}  // extern "C"
