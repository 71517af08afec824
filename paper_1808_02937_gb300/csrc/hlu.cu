// H-matrix approximation A~ (Sec. 3), H-LU factorisation and H-triangular
// solves (Sec. 4.1) on the GPU.
//
//  * k_diag / k_nearfield: the inadmissible leaves keep the exact entries of
//    A = rho M + theta S_l + (1-theta) S_l^T (end of Sec. 3.2), symmetrically
//    scaled by powers of two (D A D, D_i = 2^-round(log2(A_ii)/2)) before the
//    cast to the working precision.
//  * k_lowrank: every admissible pair (tau right of sigma) gets the Taylor
//    factors of eq. (eqn:Lexpan), Q_{i,nu} = gamma0 int h_nu phi_i',
//    W_{j,nu} = int g_nu phi_j' (Sec. 3.2); the lower block is theta Q W^T,
//    the mirrored upper block (1-theta) W Q^T.  The expansion is in s about
//    the centre of sigma, or in t about the centre of tau when tau is the
//    smaller cluster (Remark after the Lemma).
//  * k_hprog: one CTA per instance runs the op program the host planner
//    compiled from the recursive H-LU (or the forward/backward substitution).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <array>
#include <list>
#include <exception>
#include <map>
#include <thread>
#include <unordered_map>
#include <mutex>
#include <memory>
#include <string>

#include "hfsem_internal.h"
#include "hplan.h"

namespace hf {

struct SlotDev {
  long long off;   // U at off (m x kcap), V at off + m*kcap (n x kcap)
  int m, n, kcap, kmax;
};

struct DenseDev {   // one dense block of the near field
  long long off;
  int d0r, m, d0c, n;
};

struct LRPairDev {  // an admissible pair: tau (rows of the lower block) right of sigma
  int lower_slot, upper_slot;
  int te0, te1, se0, se1;       // element ranges
  int tlo, thi, slo, shi;       // support nodes
  int td0, tm, sd0, sn;         // unknown ranges
  long long toff;               // rows of Q (tm x R) then W (sn x R) in the FP64 row buffer
};

constexpr int kCluster = 8;   // CTAs (one thread-block cluster) per instance
// factorisations of at most kWideMaxInst instances, one of at least kWideNd
// unknowns, run the H-LU program on clusters of kWideCluster CTAs (a
// non-portable cluster size, used when the device can hold one)
constexpr int kWideCluster = 16;
constexpr int kWideMaxInst = 2;
constexpr int kWideNd = 8192;
// factorisations of at least kNarrowMinInst instances run it on clusters of
// kNarrowCluster CTAs: the instances, not the ops of one program, fill the
// device then, and small clusters pack its SMs more densely
constexpr int kNarrowCluster = 4;
constexpr int kNarrowMinInst = 32;

struct HInstDev {
  long long arena;   // offset of the instance arena (elements)
  long long rk0;     // offset into the rank array
  long long slot0;   // offset into the slot table
  long long dense0;  // offset into the dense-block table
  long long pair0;   // offset into the pair table
  long long ops0;
  int nops, ndense, npairs, n_slots;
  long long ws_off, rhs_off, ws_size;
  long long fw0;     // offset into the wave table
  int nfw;           // number of waves
  long long d_off;   // scaling D (FP64) offset
  int sys_inst;      // index into the system's instances
  int R;
  int nd;            // unknowns (leading dimension of the rhs area)
  long long ptask0;  // low-rank build: task offsets of the pairs (npairs + 1)
  long long gmax0;   // low-rank build: this instance's first pair in the maxima
  long long lrt0;    // low-rank build: this instance's FP64 row buffer
  long long st0, job0;  // leaf-solve tables: steps, jobs
  long long pk0;     // this instance's first job in the solve pack
  int jcap;          // jobs per part of the leaf solve
  int nst;           // steps (2 x leaves)
  int njob;          // jobs of the instance's plan
};

// right-hand sides per pass of the leaf solve
template <class T>
__host__ __device__ constexpr int solve_w() {
  return sizeof(T) == 4 ? 4 : 2;
}

constexpr int kHThreads = 256;

// ---------------------------------------------------------------------------
// entries of A in element-major unknowns
// ---------------------------------------------------------------------------
struct Term {
  int e, m;
  double a;
};

// contributions of unknown i to the Legendre coefficients of u' (z = Pi x)
__device__ __forceinline__ int terms_of(const InstDev& I, const double* h, int i, Term* t) {
  const int P = I.P;
  int e = i / P, p = i % P + 1;
  // coefficients of the length-scaled map z = h Pi x (the system's pair
  // blocks are stored divided by h_e h_f)
  (void)h;
  if (p < P) {
    t[0] = Term{e, p, -2.0 * (2.0 * p + 1.0)};
    return 1;
  }
  int j = e + 1;   // hat at node j: right hat of element j-1, left hat of element j
  t[0] = Term{j - 1, 0, 1.0};
  t[1] = Term{j, 0, -1.0};
  return 2;
}

// Mb_ef[m][n] for f <= e
__device__ __forceinline__ double mb_entry(const InstDev& I, const double* arena, int e, int f,
                                           int m, int n) {
  const int P = I.P;
  if (I.kind == kDense)
    return arena[I.o_M + ((long long)e * (e + 1) / 2 + f) * P * P + m * P + n];
  if (I.kind == kHmat) {   // the band: pairs (e, flo[e] .. e), checked on the host
    const long long q = (long long)arena[I.o_off + e] + (f - (int)arena[I.o_flo + e]);
    return arena[I.o_M + q * P * P + m * P + n];
  }
  return arena[I.o_rs + e] * arena[I.o_cs + f] * arena[I.o_M + (long long)(e - f) * P * P + m * P + n];
}

// S_l[r][c] = sum over terms a b Mb_ef[m][n], f <= e
__device__ double sl_entry(const InstDev& I, const double* arena, int r, int c) {
  const double* h = arena + I.o_h;
  Term tr[2], tc[2];
  int nr = terms_of(I, h, r, tr), nc = terms_of(I, h, c, tc);
  double s = 0.0;
  for (int a = 0; a < nr; ++a)
    for (int b = 0; b < nc; ++b) {
      int e = tr[a].e, f = tc[b].e;
      if (f > e || e < 0 || e >= I.N || f < 0 || f >= I.N) continue;
      s += tr[a].a * tc[b].a * mb_entry(I, arena, e, f, tr[a].m, tc[b].m);
    }
  return s;
}

// local index of unknown i on element e (0 left hat, 1 right hat, 1+p bubble) or -1
__device__ __forceinline__ int local_of(int P, int i, int e) {
  int ei = i / P, p = i % P + 1;
  if (p < P) return (ei == e) ? 1 + p : -1;
  int j = ei + 1;
  if (e == j - 1) return 1;
  if (e == j) return 0;
  return -1;
}

__device__ __forceinline__ double ref_mass(int a, int b) {
  if (a > b) {
    int t = a;
    a = b;
    b = t;
  }
  if (a <= 1 && b <= 1) return (a == b) ? 2.0 / 3.0 : 1.0 / 3.0;
  if (a <= 1) {
    int p = b - 1;
    if (p == 1) return 1.0;
    if (p == 2) return (a == 0) ? -1.0 / 3.0 : 1.0 / 3.0;
    return 0.0;
  }
  int p = a - 1, q = b - 1;
  if (p == q) return 2.0 / (2 * p - 1) + 2.0 / (2 * p + 3);
  if (q == p + 2) return -2.0 / (2 * p + 3);
  return 0.0;
}

__device__ double mass_entry(const InstDev& I, const double* h, int r, int c) {
  const int P = I.P;
  int er = r / P;
  double s = 0.0;
  for (int e = er; e <= er + 1 && e < I.N; ++e) {
    int a = local_of(P, r, e), b = local_of(P, c, e);
    if (a >= 0 && b >= 0) s += 0.5 * h[e] * ref_mass(a, b);
  }
  return s;
}

__device__ double a_entry(const InstDev& I, const double* arena, int r, int c) {
  double v = I.theta * sl_entry(I, arena, r, c) + (1.0 - I.theta) * sl_entry(I, arena, c, r);
  if (I.rho != 0.0) v += I.rho * mass_entry(I, arena + I.o_h, r, c);
  return v;
}

__global__ void k_diag(const HInstDev* __restrict__ hi, const InstDev* __restrict__ inst,
                       const double* arena, double* D) {
  const HInstDev H = hi[blockIdx.y];
  const InstDev I = inst[H.sys_inst];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.Nd; i += gridDim.x * blockDim.x) {
    double a = fabs(a_entry(I, arena, i, i));
    D[H.d_off + i] = (a > 0.0 && isfinite(a)) ? exp2(-rint(0.5 * log2(a))) : 1.0;
  }
}

// Near-field dense blocks of D A D.  One CTA per block and 128 x 128 tile:
// the derivative terms of the tile's rows and columns (z = Pi x, at most two
// per unknown) are formed once, so an entry costs only its moment products.
template <class T>
__global__ void __launch_bounds__(256) k_nearfield(const HInstDev* __restrict__ hi,
                                                   const InstDev* __restrict__ inst,
                                                   const double* arena,
                                                   const DenseDev* __restrict__ dens,
                                                   const double* D, T* har) {
  __shared__ Term rt[128][2], ct[128][2];
  __shared__ int rn[128], cn[128];
  const HInstDev H = hi[blockIdx.y];
  const InstDev I = inst[H.sys_inst];
  T* ar = har + H.arena;
  const double* Dv = D + H.d_off;
  const double* h = arena + I.o_h;
  for (int b = blockIdx.x; b < H.ndense; b += gridDim.x) {
    const DenseDev d = dens[H.dense0 + b];
    for (int i0 = 0; i0 < d.m; i0 += 128)
      for (int j0 = 0; j0 < d.n; j0 += 128) {
        const int mi = min(128, d.m - i0), nj = min(128, d.n - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < 256; t += blockDim.x) {
          if (t < 128) {
            if (t < mi) rn[t] = terms_of(I, h, d.d0r + i0 + t, rt[t]);
          } else if (t - 128 < nj) {
            cn[t - 128] = terms_of(I, h, d.d0c + j0 + t - 128, ct[t - 128]);
          }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < mi * nj; t += blockDim.x) {
          const int i = t % mi, j = t / mi;
          const int r = d.d0r + i0 + i, c = d.d0c + j0 + j;
          double sl = 0.0, su = 0.0;   // S_l[r][c] and S_l[c][r]
          for (int a = 0; a < rn[i]; ++a)
            for (int q = 0; q < cn[j]; ++q) {
              const Term A = rt[i][a], B = ct[j][q];
              if (A.e < 0 || A.e >= I.N || B.e < 0 || B.e >= I.N) continue;
              const double ab = A.a * B.a;
              if (B.e <= A.e) sl += ab * mb_entry(I, arena, A.e, B.e, A.m, B.m);
              if (A.e <= B.e) su += ab * mb_entry(I, arena, B.e, A.e, B.m, A.m);
            }
          double v = I.theta * sl + (1.0 - I.theta) * su;
          if (I.rho != 0.0) v += I.rho * mass_entry(I, h, r, c);
          ar[d.off + (long long)(j0 + j) * d.m + i0 + i] = (T)(Dv[r] * v * Dv[c]);
        }
      }
  }
}

// shared memory of k_lowrank: per CTA the quadrature (points, weights,
// Legendre values) and the recurrence coefficients, per warp the expansion
// functions and the moment block (16-byte multiples)
__host__ __device__ inline size_t lowrank_cta_bytes(int nq, int P, int R, size_t csize) {
  return ((size_t)(nq * (2 + P) + R) * csize + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t lowrank_warp_bytes(int nq, int P, int R, size_t csize) {
  return ((size_t)(nq * R + P * R + R) * csize + 15) & ~(size_t)15;
}

// Taylor low-rank factors of every admissible pair (tau right of sigma).
// One warp per task: a task is one element e of one side of one pair; it
// forms the element's moment block (the Legendre modes of the element against
// the R expansion functions of the side, by Gauss-Legendre quadrature) and
// writes the factor rows of the bubbles of e and of the hat at its left node
// (which also needs mode 0 of element e-1).  Tasks of pair k are [ptask[k],
// ptask[k+1]): the elements te0..elast of side 0, then of side 1; a warp
// takes a contiguous run of tasks.
// The per-point work runs in the precision of the factors (C = T): the
// geometry is formed in FP64 once per element, and the singular side is
// written as rr^(1-alpha) [u^(1-alpha) c_nu (sg / u)^nu] with d = rr u
// (u >= 1 on an admissible pair), the FP64 scale rr^(1-alpha) joining the
// row scales.  With the moments of the bubble p, 0.5 h_e acc, the h_e of the
// quadrature cancels the 2 / h_e of the derivative, and the hat row is
// 0.5 (acc_{e-1} - acc_e).
// Pass 0 finds, per term nu, the largest |Q| and |W| entries (after the D
// scaling); pass 1 writes the factors with every rank-one term balanced
// (|U_nu| and |V_nu| scaled to equal maxima): the products are unchanged and
// each factor stays inside the FP32 range on meshes whose element sizes span
// 10^80.
template <class T>
__global__ void __launch_bounds__(256) k_lowrank(const HInstDev* __restrict__ hi,
                                                 const InstDev* __restrict__ inst,
                                                 const double* arena, const double* __restrict__ gl,
                                                 const LRPairDev* __restrict__ pairs,
                                                 const SlotDev* __restrict__ slots,
                                                 const int* __restrict__ ptask, const double* D,
                                                 double* lrt, unsigned long long* gmax) {
  using C = T;
  extern __shared__ __align__(16) unsigned char lsm_raw[];
  const HInstDev H = hi[blockIdx.y];
  const InstDev I = inst[H.sys_inst];
  const int P = I.P, R = H.R;
  const int nq = min((P + R) / 2 + 13, kMaxGL);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  C* sX = reinterpret_cast<C*>(lsm_raw);   // [nq] Gauss-Legendre points
  C* sW = sX + nq;                         // [nq] weights
  C* sL = sW + nq;                         // [nq][P] Legendre polynomials
  C* sCo = sL + nq * P;                    // [R] (2 - alpha - nu) / nu
  unsigned char* wb = lsm_raw + lowrank_cta_bytes(nq, P, R, sizeof(C)) +
                      (size_t)warp * lowrank_warp_bytes(nq, P, R, sizeof(C));
  C* sF = reinterpret_cast<C*>(wb);        // [nq][R] expansion functions (scaled)
  C* sQ = sF + nq * R;                     // [P][R] quadrature sums of the element
  C* sQ0 = sQ + P * R;                     // [R] mode-0 sums of element e-1
  const double* X = gl + gl_off(nq);
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const double xq = X[q];
    sX[q] = (C)xq;
    sW[q] = (C)X[nq + q];
    double l0 = 1.0, l1 = xq;
    sL[q * P] = (C)1;
    if (P > 1) sL[q * P + 1] = (C)xq;
    for (int k = 1; k + 1 < P; ++k) {
      const double l2 = ((2 * k + 1) * xq * l1 - k * l0) / (k + 1);
      sL[q * P + k + 1] = (C)l2;
      l0 = l1;
      l1 = l2;
    }
  }
  for (int nu = threadIdx.x; nu < R; nu += blockDim.x)
    sCo[nu] = nu ? (C)((2.0 - I.alpha - nu) / nu) : (C)0;
  __syncthreads();
  const double* h = arena + I.o_h;
  const double* dl = arena + I.o_dl;
  const double* dr = arena + I.o_dr;
  auto ndiff = [&](int a, int b) {   // x_a - x_b, a >= b
    return (dl[a] <= dr[b]) ? dl[a] - dl[b] : dr[b] - dr[a];
  };
  const int* pt = ptask + H.ptask0;   // npairs + 1 task offsets
  const int ntask = pt[H.npairs];
  const double* Dv = D + H.d_off;
  double* rows = lrt + H.lrt0;
  const double ex = 1.0 - I.alpha;
  const C exc = (C)ex;
  // each warp takes a contiguous run of tasks: one search for the first
  // pair, then the pairs follow in order
  const int gw = blockIdx.x * nw + warp, nwarps = gridDim.x * nw;
  const int chunk = (ntask + nwarps - 1) / nwarps;
  const int t_begin = gw * chunk, t_end = min(ntask, t_begin + chunk);
  int lo = 0;
  if (t_begin < t_end) {
    int hi_ = H.npairs;
    while (hi_ - lo > 1) {
      const int mid = (lo + hi_) >> 1;
      if (pt[mid] <= t_begin) lo = mid; else hi_ = mid;
    }
  }
  int next_start = (t_begin < t_end) ? pt[lo + 1] : 0;
  for (int task = t_begin; task < t_end; ++task) {
    while (task >= next_start) {
      ++lo;
      next_start = pt[lo + 1];
    }
    const LRPairDev pr = pairs[H.pair0 + lo];
    const int tl = task - pt[lo];
    const int elast_t = (pr.te1 < I.N) ? pr.te1 : pr.te1 - 1;   // element e1 only feeds the hat at node e1
    const int nt = elast_t - pr.te0 + 1;
    const int side = tl < nt ? 0 : 1;
    const int e0 = side == 0 ? pr.te0 : pr.se0, e1 = side == 0 ? pr.te1 : pr.se1;
    const int e = e0 + (side == 0 ? tl : tl - nt);
    const int d0 = side == 0 ? pr.td0 : pr.sd0;
    const double r_s = 0.5 * ndiff(pr.shi, pr.slo);
    const double r_t = 0.5 * ndiff(pr.thi, pr.tlo);
    const bool sexp = (r_s <= r_t);
    const bool singular = (side == 0) == sexp;
    const double rr = sexp ? r_s : r_t;
    const double inv_rr = 1.0 / rr;
    const double fsc = singular ? pow(rr, ex) : 1.0;
    // expansion functions of element ee at the Gauss points: the argument is
    // A + B (1 +- x) with A, B from the FP64 geometry of the element
    auto fill_f = [&](int ee) {
      double A, B;
      const C sg = sexp ? (C)-1 : (C)1;
      if (singular) {
        if (sexp) A = (ndiff(ee, pr.shi) + r_s) * inv_rr;        // (t - s0) / r_s, t = left end
        else A = (r_t + ndiff(pr.tlo, ee + 1)) * inv_rr;         // (t0 - s) / r_t, s = right end
      } else {
        A = sexp ? (ndiff(ee, pr.slo) - r_s) * inv_rr             // (s - s0) / r_s
                 : (ndiff(ee, pr.tlo) - r_t) * inv_rr;            // (t - t0) / r_t
      }
      B = 0.5 * h[ee] * inv_rr;
      const C Ac = (C)A, Bc = (C)B;
      const bool rev = singular && !sexp;   // the argument falls as x rises
      for (int q = lane; q < nq; q += 32) {
        const C xq = sX[q];
        const C u = Ac + Bc * (rev ? ((C)1 - xq) : ((C)1 + xq));
        C* F = sF + q * R;
        if (singular) {
          const C iu = sg / u;
          C f = pow(u, exc);
          F[0] = f;
          for (int nu = 1; nu < R; ++nu) {
            f *= sCo[nu] * iu;
            F[nu] = f;
          }
        } else {
          C f = (C)1;
          for (int nu = 0; nu < R; ++nu) {
            F[nu] = f;
            f *= u;
          }
        }
      }
      __syncwarp();
    };
    const bool hat = e > e0, bub = e < e1;
    if (hat) {   // mode 0 of element e-1 (the Legendre mode 0 is 1)
      fill_f(e - 1);
      for (int nu = lane; nu < R; nu += 32) {
        C acc = (C)0;
        for (int q = 0; q < nq; ++q) acc += sW[q] * sF[q * R + nu];
        sQ0[nu] = acc;
      }
      __syncwarp();
    }
    fill_f(e);
    for (int t = lane; t < P * R; t += 32) {
      const int m = t / R, nu = t % R;
      C acc = (C)0;
      for (int q = 0; q < nq; ++q) acc += sW[q] * sL[q * P + m] * sF[q * R + nu];
      sQ[m * R + nu] = acc;
    }
    __syncwarp();
    // rows: the hat at node e (elements e-1 and e) when e > e0, the bubbles
    // of e when e < e1
    const double scale_side = ((side == 0) ? I.g0 : 1.0) * fsc;   // gamma0 sits with Q
    const int nb = bub ? P - 1 : 0, nh = hat ? 1 : 0;
    unsigned long long* gm = gmax + ((size_t)H.gmax0 + lo) * 64;
    // FP64 factor rows (before balancing): Q rows of tau then W rows of sigma
    double* out = rows + pr.toff + (side == 0 ? 0LL : (long long)pr.tm * R);
    const int nrow = side == 0 ? pr.tm : pr.sn;
    // lane k holds row k (P <= 32 rows per element)
    const int k = lane;
    const bool has = k < nb + nh;
    int row = 0, pp = 0;
    double rs = 0.0;
    if (has) {
      int dof;
      if (k < nh) {
        dof = e * P - 1;
        rs = 0.5 * scale_side * Dv[dof];
      } else {
        pp = k - nh + 1;
        dof = e * P + pp - 1;
        rs = -(2.0 * pp + 1.0) * scale_side * Dv[dof];
      }
      row = dof - d0;
    }
    for (int nu = 0; nu < R; ++nu) {
      double v = 0.0;
      if (has) {
        v = rs * (double)((k < nh) ? (sQ0[nu] - sQ[nu]) : sQ[pp * R + nu]);
        out[row + (long long)nu * nrow] = v;
      }
      double vmax = fabs(v);
      for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      if (lane == 0 && vmax > 0.0)
        atomicMax(&gm[side * 32 + nu], (unsigned long long)__double_as_longlong(vmax));
    }
    __syncwarp();
  }
}

// Balance and store the low-rank factors: per pair and term nu the Q column
// is scaled by c = sqrt(max|W| / max|Q|) and the W column by 1 / c (the
// product is unchanged; each factor stays inside the FP32 range on meshes
// whose element sizes span 10^80), then written to the slots: lower
// U = theta D Q, V = D W; upper U = D W, V = (1 - theta) D Q.
template <class T>
__global__ void k_lowrank_write(const HInstDev* __restrict__ hi, const InstDev* __restrict__ inst,
                                const LRPairDev* __restrict__ pairs,
                                const SlotDev* __restrict__ slots, const double* lrt,
                                const unsigned long long* gmax, T* har, int* ranks) {
  const HInstDev H = hi[blockIdx.y];
  const InstDev I = inst[H.sys_inst];
  const int R = H.R;
  T* ar = har + H.arena;
  for (int pi = blockIdx.x; pi < H.npairs; pi += gridDim.x) {
    const LRPairDev pr = pairs[H.pair0 + pi];
    const SlotDev slo = slots[H.slot0 + pr.lower_slot];
    const SlotDev sup = slots[H.slot0 + pr.upper_slot];
    const unsigned long long* gm = gmax + ((size_t)H.gmax0 + pi) * 64;
    const double* rows = lrt + H.lrt0 + pr.toff;
    const int nq = pr.tm * R, nw = pr.sn * R;
    for (int t = threadIdx.x; t < nq + nw; t += blockDim.x) {
      const int side = t < nq ? 0 : 1;
      const int tt = side == 0 ? t : t - nq;
      const int nrow = side == 0 ? pr.tm : pr.sn;
      const int row = tt % nrow, nu = tt / nrow;
      const double mq = __longlong_as_double((long long)gm[nu]);
      const double mw = __longlong_as_double((long long)gm[32 + nu]);
      double sc = (mq > 0.0 && mw > 0.0) ? sqrt(mw) / sqrt(mq) : 1.0;   // Q *= sc, W /= sc
      sc = (isfinite(sc) && sc > 0.0) ? sc : 1.0;
      const double v = rows[t];
      if (side == 0) {
        const double q = v * sc;
        ar[slo.off + row + (long long)nu * slo.m] = (T)(I.theta * q);
        ar[sup.off + (long long)sup.m * sup.kcap + row + (long long)nu * sup.n] = (T)((1.0 - I.theta) * q);
      } else {
        const double w = v / sc;
        ar[slo.off + (long long)slo.m * slo.kcap + row + (long long)nu * slo.n] = (T)w;
        ar[sup.off + row + (long long)nu * sup.m] = (T)w;
      }
    }
    if (threadIdx.x == 0) {
      ranks[H.rk0 + pr.lower_slot] = (I.theta != 0.0) ? R : 0;
      ranks[H.rk0 + pr.upper_slot] = (I.theta != 1.0) ? R : 0;
    }
  }
}

// ---------------------------------------------------------------------------
// interpreter
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dimv(int d, const int* rk) { return d >= 0 ? d : rk[-1 - d]; }
__device__ __forceinline__ long long vidx(const View& v, int i, int j) {
  return v.tr ? v.off + j + (long long)i * v.ld : v.off + i + (long long)j * v.ld;
}

// --- asynchronous element copies, global -> shared (cp.async): every
// thread issues its copies without waiting, so a whole operand is in flight
// at once; cp_async_wait_all + a barrier make it visible ---
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
template <class T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// --- mbarriers (completion of asynchronous copies and tensor-core MMAs) ---
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// --- 5th-generation tensor cores (tcgen05): accumulators in tensor memory ---
// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (16-byte units), descriptor version 1, no swizzle.  Operands are
// K-major in core matrices of 8 rows x 16 bytes (8 x 8 bf16), stored
// contiguously; SBO steps 8 rows, LBO steps 8 elements of K.
__device__ __forceinline__ unsigned long long tc_sdesc(const void* smem, unsigned lbo, unsigned sbo) {
  unsigned long long d = (unsigned long long)((smem_u32(smem) >> 4) & 0x3FFFu);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ULL << 46;
  return d;
}
// instruction descriptor: kind::f16, A and B bf16 (K-major), D f32, M x N
__device__ __forceinline__ unsigned tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_alloc(unsigned* slot, int ncols) {   // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(unsigned taddr, int ncols) {   // one whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_mma(unsigned dtmem, unsigned long long ad, unsigned long long bd,
                                       unsigned idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
// the commit names the mbarrier by its shared::cluster address (this CTA's rank)
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  unsigned rank, a;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(bar)), "r"(rank));
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(a)
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
// 16 consecutive 32-bit columns of this warp's 32 lanes
__device__ __forceinline__ void tc_ld16(unsigned taddr, float* v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = __uint_as_float(r[t]);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// dst[i + j ldd] <- view(i, j), i < m, j < n; 16-byte copies when the view is
// column-major and every column run starts on a 16-byte boundary on both sides
template <class T>
__device__ __forceinline__ void stage_view(T* dst, int ldd, const T* ar, const View& v, int m, int n) {
  if constexpr (sizeof(T) == 4) {
    if (!v.tr && (m & 3) == 0 && (ldd & 3) == 0 && (v.off & 3) == 0 && (v.ld & 3) == 0 &&
        ((smem_u32(dst) & 15u) == 0) && ((reinterpret_cast<unsigned long long>(ar) & 15ULL) == 0)) {
      const int m4 = m >> 2, total4 = m4 * n;
      for (int t = threadIdx.x; t < total4; t += blockDim.x) {
        const int i4 = t % m4, j = t / m4;
        cp_async16(dst + 4 * i4 + (long long)j * ldd, ar + v.off + 4LL * i4 + (long long)j * v.ld);
      }
      return;
    }
  }
  const int total = m * n;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int i = t % m, j = t / m;
    cp_async_elem(dst + i + j * ldd, ar + vidx(v, i, j));
  }
}

template <class T>
struct HCtx {
  T* ar;
  int* rk;
  const SlotDev* sl;
  T* ws;
  T* sm;
  long long smcap;   // elements of T in the dynamic shared memory
  unsigned long long* tprof;   // optional: recompression phase times (profiling)
  int tc;                      // dense leaf contractions on the tensor cores (BF16 in, FP32 out)
  unsigned tmem;               // tensor-memory accumulator (256 columns)
  unsigned long long* tcbar;   // mbarrier the MMAs commit to
  unsigned* tcphase;           // its phase
  unsigned long long* tcdbg;   // diagnostics of a tensor-core wait that ran out
  double tol;
  int* err;
  int leaf32;   // leaf LUs in FP32 arithmetic (FP64 arena kept for its range)
};

template <class T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// BF16x3 tensor-core tile: D (128 x N) = A (128 x K) B (K x N) with FP32
// accumulation in tensor memory (tcgen05).  A and B are read from FP32 views
// and split into a BF16 head and a BF16 tail (x = hi + lo, lo the rounded
// remainder), each stored in shared memory as K-major core matrices; three
// MMAs per K step (hi hi, hi lo, lo hi) give the products to about 2^-16
// relative, close to FP32 operands.  Then C = beta C + alpha D, with C stored
// 128 x N (ctr = 0) or N x 128 (ctr = 1).
// K a multiple of 16, N a multiple of 16 in [16, 256].  One thread issues the
// MMAs; all threads wait on the mbarrier they commit to (bounded), then read
// the accumulators back, warp w covering rows 32 (w mod 4) ...
__device__ bool tc_gemm128(HCtx<float>& c, const View& A, const View& B, const View& Cv, int ctr, int N,
                           int K, float alpha, float beta) {
  float* ar = c.ar;
  // operands on 1024-byte boundaries
  const unsigned base = smem_u32(c.sm);
  const unsigned pad = ((base + 1023u) & ~1023u) - base;
  // heads and tails of A (128 x K) and B (N x K), each on a 1024-byte boundary
  const size_t sa = ((size_t)128 * K + 511) & ~(size_t)511, sb = ((size_t)N * K + 511) & ~(size_t)511;
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(c.sm) + pad);
  __nv_bfloat16* Al = As + sa;
  __nv_bfloat16* Bs = Al + sa;
  __nv_bfloat16* Bl = Bs + sb;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nc8 = N >> 3;
  for (int t = tid; t < 128 * K; t += nt) {
    const int m = t & 127, k = t >> 7;
    const float x = ar[vidx(A, m, k)];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const int i = ((k >> 3) * 16 + (m >> 3)) * 64 + (m & 7) * 8 + (k & 7);
    As[i] = h;
    Al[i] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
  for (int t = tid; t < K * N; t += nt) {
    const int k = t % K, n = t / K;
    const float x = ar[vidx(B, k, n)];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const int i = ((k >> 3) * nc8 + (n >> 3)) * 64 + (n & 7) * 8 + (k & 7);
    Bs[i] = h;
    Bl[i] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    tc_fence_after();
    const unsigned idesc = tc_idesc_bf16(128, N);
    for (int s = 0; s < K / 16; ++s) {
      const unsigned long long ah = tc_sdesc(As + s * 2 * 16 * 64, 16 * 64 * 2, 128);
      const unsigned long long al = tc_sdesc(Al + s * 2 * 16 * 64, 16 * 64 * 2, 128);
      const unsigned long long bh = tc_sdesc(Bs + s * 2 * nc8 * 64, nc8 * 64 * 2, 128);
      const unsigned long long bl = tc_sdesc(Bl + s * 2 * nc8 * 64, nc8 * 64 * 2, 128);
      tc_mma(c.tmem, ah, bh, idesc, s > 0);
      tc_mma(c.tmem, ah, bl, idesc, 1);
      tc_mma(c.tmem, al, bh, idesc, 1);
    }
    tc_commit(c.tcbar);
  }
  // wait for the MMAs, at most ~2 ms of wall time; every thread must agree
  bool ok = true;
  {
    const unsigned ph = *c.tcphase;
    unsigned long long t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (!mbar_try_wait(c.tcbar, ph)) {
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
      if (t1 - t0 > 2000000ULL) {
        ok = false;
        break;
      }
    }
  }
  ok = __syncthreads_and(ok) != 0;
  tc_fence_after();
  if (!ok) {
    // record the barrier word and the descriptors, and stop using the
    // tensor cores in this CTA (the op is lost; the flag fails the factor)
    if (tid == 0) {
      atomicExch(c.err, 4);
      if (c.tcdbg) {
        unsigned long long w;
        asm volatile("ld.shared.b64 %0, [%1];" : "=l"(w) : "r"(smem_u32(c.tcbar)) : "memory");
        c.tcdbg[0] = w;
        c.tcdbg[1] = tc_sdesc(As, 16 * 64 * 2, 128);
        c.tcdbg[2] = tc_sdesc(Bs, nc8 * 64 * 2, 128);
        c.tcdbg[3] = tc_idesc_bf16(128, N);
        c.tcdbg[4] = c.tmem;
        c.tcdbg[5] = ((unsigned long long)N << 32) | (unsigned)K;
      }
    }
    c.tc = 0;
    __syncthreads();
    return true;
  }
  *c.tcphase ^= 1u;   // every thread tracks the barrier's phase
  const int warp = tid >> 5, lane = tid & 31, rw = warp & 3, h = warp >> 2;
  const int row = 32 * rw + lane;
  for (int col = 16 * h; col < N; col += 32) {
    float v[16];
    tc_ld16(c.tmem + ((unsigned)(32 * rw) << 16) + (unsigned)col, v);
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const long long ci = ctr ? vidx(Cv, col + t, row) : vidx(Cv, row, col + t);
      ar[ci] = (beta == 0.f ? 0.f : beta * ar[ci]) + alpha * v[t];
    }
  }
  tc_fence_before();
  __syncthreads();
  return true;
}

// FP32 arithmetic on an FP64 arena (the FP64 part of a mixed-precision
// factor keeps FP64 storage for the range of its entries; its products keep
// the mode's FP32 arithmetic): operands converted to FP32 on their way into
// shared memory, sums in FP32, results converted back.
// C = beta C + alpha A B, 64 x 64 output tiles, k in chunks of 16, 4 x 4 per thread.
__device__ void gemm_f32_on_f64(const HOp& o, HCtx<double>& c, int m, int n, int k, float alpha,
                                float beta) {
  double* ar = c.ar;
  float* As = reinterpret_cast<float*>(c.sm);   // [16][64]
  float* Bs = As + 16 * 64;                     // [16][64]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int m0 = 0; m0 < m; m0 += 64)
    for (int n0 = 0; n0 < n; n0 += 64) {
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
      for (int k0 = 0; k0 < k; k0 += 16) {
        for (int t = tid; t < 16 * 64; t += nt) {
          const int kk = t / 64, ii = t % 64;
          const int gi = m0 + ii, gk = k0 + kk, gj = n0 + ii;
          As[kk * 64 + ii] = (gi < m && gk < k) ? (float)ar[vidx(o.A, gi, gk)] : 0.f;
          Bs[kk * 64 + ii] = (gj < n && gk < k) ? (float)ar[vidx(o.B, gk, gj)] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          float a[4], b[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            a[q] = As[kk * 64 + ty * 4 + q];
            b[q] = Bs[kk * 64 + tx * 4 + q];
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
        }
        __syncthreads();
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int gi = m0 + ty * 4 + p, gj = n0 + tx * 4 + q;
          if (gi < m && gj < n) {
            const long long ci = vidx(o.C, gi, gj);
            const float cv = beta == 0.f ? 0.f : beta * (float)ar[ci];
            ar[ci] = (double)(cv + alpha * acc[p][q]);
          }
        }
    }
}

// C <- A C (A n x n, n <= 128) in FP32 arithmetic on an FP64 arena: A and a
// 32-column panel of C staged as FP32.
__device__ void trmm_l_f32_on_f64(const HOp& o, HCtx<double>& c, int n, int cc) {
  double* ar = c.ar;
  float* As = reinterpret_cast<float*>(c.sm);   // n x n, [i + k n]
  float* Pn = As + n * n;                       // n x 32, [k * 33 + j]
  const int tid = threadIdx.x;
  for (int t = tid; t < n * n; t += blockDim.x) As[t] = (float)ar[vidx(o.A, t % n, t / n)];
  const int tx = tid & 7, ty = tid >> 3;
  for (int c0 = 0; c0 < cc; c0 += 32) {
    const int cp = min(32, cc - c0);
    __syncthreads();
    for (int t = tid; t < n * cp; t += blockDim.x) {
      const int i = t % n, j = t / n;
      Pn[i * 33 + j] = (float)ar[vidx(o.C, i, c0 + j)];
    }
    __syncthreads();
    for (int rb = ty * 4; rb < n; rb += 128) {
      float acc[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
      for (int k = 0; k < n; ++k) {
        float a[4], b[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) a[p] = (rb + p < n) ? As[rb + p + k * n] : 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = Pn[k * 33 + tx + 8 * q];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (rb + p < n && tx + 8 * q < cp) ar[vidx(o.C, rb + p, c0 + tx + 8 * q)] = (double)acc[p][q];
    }
  }
  __syncthreads();
}

// C <- C A (A n x n, n <= 128) in FP32 arithmetic on an FP64 arena: A (row-
// major, padded row) and a 32-row panel of C staged as FP32.
__device__ void trmm_r_f32_on_f64(const HOp& o, HCtx<double>& c, int m, int n) {
  double* ar = c.ar;
  const int lda = n + 1;
  float* As = reinterpret_cast<float*>(c.sm);   // n x n, [k lda + j]
  float* Pn = As + n * lda;                     // 32 x n, [i + k * 32]
  const int tid = threadIdx.x;
  for (int t = tid; t < n * n; t += blockDim.x) As[(t % n) * lda + t / n] = (float)ar[vidx(o.A, t % n, t / n)];
  const int tx = tid & 31, ty = tid >> 5;
  for (int r0 = 0; r0 < m; r0 += 32) {
    const int rp = min(32, m - r0);
    __syncthreads();
    for (int t = tid; t < rp * n; t += blockDim.x)
      Pn[(t % rp) + (t / rp) * 32] = (float)ar[vidx(o.C, r0 + t % rp, t / rp)];
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
    for (int k = 0; k < n; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) a[p] = Pn[ty * 4 + p + k * 32];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = (tx + 32 * q < n) ? As[k * lda + tx + 32 * q] : 0.f;
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (ty * 4 + p < rp && tx + 32 * q < n)
          ar[vidx(o.C, r0 + ty * 4 + p, tx + 32 * q)] = (double)acc[p][q];
  }
  __syncthreads();
}

template <class T>
__device__ void op_gemm(const HOp& o, HCtx<T>& c) {
  const int m = dimv(o.C.r, c.rk), n = dimv(o.C.c, c.rk), k = dimv(o.A.c, c.rk);
  if (m <= 0 || n <= 0) return;
  T* ar = c.ar;
  const T alpha = (T)o.alpha, beta = (T)o.beta;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (k <= 0) {
    for (int t = tid; t < m * n; t += nt) {
      long long ci = vidx(o.C, t % m, t / m);
      ar[ci] = (beta == (T)0) ? (T)0 : beta * ar[ci];
    }
    return;
  }
  if constexpr (sizeof(T) == 8) {
    // FP64 part of a mixed factor: products of any size in FP32 arithmetic
    // (the small ones stay on their latency-bound FP64 paths)
    if (c.leaf32 && m >= 16 && n >= 16 && k >= 16) {
      gemm_f32_on_f64(o, c, m, n, k, (float)o.alpha, (float)o.beta);
      return;
    }
  }
  if constexpr (sizeof(T) == 4) {
    // dense leaf products on the tensor cores
    if (c.tc && m == 128 && n >= 16 && n <= 256 && (n & 15) == 0 && k >= 64 && (k & 15) == 0 &&
        (long long)(128 + n) * k + 1024 <= c.smcap) {
      if (tc_gemm128(c, o.A, o.B, o.C, 0, n, k, alpha, beta)) return;
    }
  }
  if constexpr (sizeof(T) == 4) {
    // rank-k update of an aligned column-major C (k <= 16): A and B staged,
    // C moved with 16-byte accesses, eight in flight per thread
    if (k <= 16 && m >= 64 && n >= 32 && !o.C.tr && (m & 3) == 0 && (o.C.off & 3) == 0 &&
        (o.C.ld & 3) == 0 && (long long)m * k + (long long)k * n + 64 <= c.smcap) {
      float* As = c.sm;                    // [i + kk m]
      float* Bs = As + (long long)m * k;   // [kk + j k]
      stage_view(As, m, ar, o.A, m, k);
      stage_view(Bs, k, ar, o.B, k, n);
      cp_async_wait_all();
      __syncthreads();
      const int m4 = m >> 2, items = m4 * n;
      const long long ldc = o.C.ld;
      for (int u0 = tid; u0 < items; u0 += 8 * nt) {
        float4 cv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int u = u0 + q * nt;
          if (u < items && beta != 0.f)
            cv[q] = *reinterpret_cast<const float4*>(ar + o.C.off + 4LL * (u % m4) + (long long)(u / m4) * ldc);
          else
            cv[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int u = u0 + q * nt;
          if (u < items) {
            const int i4 = u % m4, j = u / m4;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int kk = 0; kk < k; ++kk) {
              const float4 a4 = *reinterpret_cast<const float4*>(As + 4 * i4 + (long long)kk * m);
              const float b = Bs[kk + (long long)j * k];
              acc.x += a4.x * b;
              acc.y += a4.y * b;
              acc.z += a4.z * b;
              acc.w += a4.w * b;
            }
            float4 out;
            out.x = beta * cv[q].x + alpha * acc.x;
            out.y = beta * cv[q].y + alpha * acc.y;
            out.z = beta * cv[q].z + alpha * acc.z;
            out.w = beta * cv[q].w + alpha * acc.w;
            *reinterpret_cast<float4*>(ar + o.C.off + 4LL * i4 + (long long)j * ldc) = out;
          }
        }
      }
      __syncthreads();
      return;
    }
  }
  {
    // staged: A and B reach shared memory in one pass of asynchronous copies;
    // the outputs run in column-major order (coalesced C, four loads of C in
    // flight per thread), the inner dimension split over idle threads when
    // the output is small
    const long long mn = (long long)m * n;
    const long long need = (long long)m * k + (long long)k * n;
    if ((mn <= 4096 || k <= 32) && need + 16 * 256 <= c.smcap) {
      T* As = c.sm;                    // [i + kk m]
      T* Bs = As + (long long)m * k;   // [kk + j k]
      T* red = Bs + (long long)k * n;  // partials of the split inner dimension
      stage_view(As, m, ar, o.A, m, k);
      stage_view(Bs, k, ar, o.B, k, n);
      cp_async_wait_all();
      __syncthreads();
      const int imn = (int)mn;
      const int S = (imn >= nt) ? 1 : min(nt / imn, 16);
      if (S == 1) {
        for (int t0 = tid; t0 < imn; t0 += 4 * nt) {
          long long ci[4];
          T cv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = t0 + u * nt;
            ci[u] = -1;
            cv[u] = (T)0;
            if (t < imn) {
              ci[u] = vidx(o.C, t % m, t / m);
              if (beta != (T)0) cv[u] = ar[ci[u]];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = t0 + u * nt;
            if (t < imn) {
              const int i = t % m, j = t / m;
              const T* a = As + i;
              const T* b = Bs + (long long)j * k;
              T acc = 0;
              for (int kk = 0; kk < k; ++kk) acc += a[(long long)kk * m] * b[kk];
              ar[ci[u]] = beta * cv[u] + alpha * acc;
            }
          }
        }
      } else {
        const int t = tid % imn, sl = tid / imn;
        if (sl < S) {
          const int i = t % m, j = t / m;
          const int kc = (k + S - 1) / S, k0 = sl * kc, k1 = min(k, k0 + kc);
          T acc = 0;
          for (int kk = k0; kk < k1; ++kk) acc += As[i + (long long)kk * m] * Bs[kk + (long long)j * k];
          red[sl * imn + t] = acc;
        }
        __syncthreads();
        for (int t2 = tid; t2 < imn; t2 += nt) {
          T acc = 0;
          for (int q = 0; q < S; ++q) acc += red[q * imn + t2];
          const int i = t2 % m, j = t2 / m;
          const long long ci = vidx(o.C, i, j);
          ar[ci] = (beta == (T)0 ? (T)0 : beta * ar[ci]) + alpha * acc;
        }
      }
      __syncthreads();
      return;
    }
  }
  if ((long long)m * n <= 2048 && k >= 32) {
    // small output, long inner dimension: one warp per output, lanes split k
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (int oi = warp; oi < m * n; oi += nw) {
      int i = oi % m, j = oi / m;
      T acc = 0;
      for (int kk = lane; kk < k; kk += 32) acc += ar[vidx(o.A, i, kk)] * ar[vidx(o.B, kk, j)];
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
      if (lane == 0) {
        long long ci = vidx(o.C, i, j);
        ar[ci] = (beta == (T)0 ? (T)0 : beta * ar[ci]) + alpha * acc;
      }
    }
    return;
  }
  if (n <= 8) {
    // tall and narrow: rows in parallel; idle threads split k (partials
    // combined in shared memory); four independent loads in flight
    const int rows_per = (m >= nt) ? nt : m;
    const int S = (m >= nt) ? 1 : min(nt / m, 16);
    T* red = c.sm;   // S x rows_per x 8
    for (int i0 = 0; i0 < m; i0 += rows_per) {
      const int r = tid % rows_per, part = tid / rows_per, i = i0 + r;
      const int kc = (k + S - 1) / S, k0 = part * kc, k1 = min(k, k0 + kc);
      T acc[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = 0;
      if (part < S && i < m) {
        int kk = k0;
        for (; kk + 4 <= k1; kk += 4) {
          T a0 = ar[vidx(o.A, i, kk)], a1 = ar[vidx(o.A, i, kk + 1)];
          T a2 = ar[vidx(o.A, i, kk + 2)], a3 = ar[vidx(o.A, i, kk + 3)];
          for (int j = 0; j < n; ++j)
            acc[j] += a0 * ar[vidx(o.B, kk, j)] + a1 * ar[vidx(o.B, kk + 1, j)] +
                      a2 * ar[vidx(o.B, kk + 2, j)] + a3 * ar[vidx(o.B, kk + 3, j)];
        }
        for (; kk < k1; ++kk) {
          T a = ar[vidx(o.A, i, kk)];
          for (int j = 0; j < n; ++j) acc[j] += a * ar[vidx(o.B, kk, j)];
        }
      }
      if (S > 1) {
        if (part < S)
          for (int j = 0; j < n; ++j) red[(part * rows_per + r) * 8 + j] = acc[j];
        __syncthreads();
        if (part == 0 && i < m)
          for (int j = 0; j < n; ++j) {
            T v = 0;
            for (int q = 0; q < S; ++q) v += red[(q * rows_per + r) * 8 + j];
            long long ci = vidx(o.C, i, j);
            ar[ci] = (beta == (T)0 ? (T)0 : beta * ar[ci]) + alpha * v;
          }
        __syncthreads();
      } else if (i < m) {
        for (int j = 0; j < n; ++j) {
          long long ci = vidx(o.C, i, j);
          ar[ci] = (beta == (T)0 ? (T)0 : beta * ar[ci]) + alpha * acc[j];
        }
      }
    }
    return;
  }
  if (m <= 8) {
    for (int j = tid; j < n; j += nt) {
      T acc[8];
      for (int i = 0; i < 8; ++i) acc[i] = 0;
      for (int kk = 0; kk < k; ++kk) {
        T b = ar[vidx(o.B, kk, j)];
        for (int i = 0; i < m; ++i) acc[i] += ar[vidx(o.A, i, kk)] * b;
      }
      for (int i = 0; i < m; ++i) {
        long long ci = vidx(o.C, i, j);
        ar[ci] = (beta == (T)0 ? (T)0 : beta * ar[ci]) + alpha * acc[i];
      }
    }
    return;
  }
  if (m >= 96 && n >= 96) {
    // 128 x 128 C tiles, 8 x 8 outputs per thread, k in chunks of 8; the
    // next chunk is loaded into registers while the current one is used
    T* As = c.sm;             // [8][128]
    T* Bs = c.sm + 8 * 128;   // [8][128]
    const int tx = tid & 15, ty = tid >> 4;
    for (int m0 = 0; m0 < m; m0 += 128)
      for (int n0 = 0; n0 < n; n0 += 128) {
        T acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = 0;
        T ra[4], rb[4];
        auto fetch = [&](int k0) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int t = tid + q * 256;
            // A by rows (consecutive threads, consecutive rows), B by k
            // (eight threads read the eight k of one column)
            int kk = t >> 7, ii = t & 127;
            int gi = m0 + ii, gk = k0 + kk;
            ra[q] = (gi < m && gk < k) ? ar[vidx(o.A, gi, gk)] : (T)0;
            int kb = t & 7, jb = t >> 3;
            int gj = n0 + jb, gkb = k0 + kb;
            rb[q] = (gj < n && gkb < k) ? ar[vidx(o.B, gkb, gj)] : (T)0;
          }
        };
        fetch(0);
        for (int k0 = 0; k0 < k; k0 += 8) {
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int t = tid + q * 256;
            As[t] = ra[q];
            Bs[(t & 7) * 128 + (t >> 3)] = rb[q];
          }
          __syncthreads();
          if (k0 + 8 < k) fetch(k0 + 8);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            T a[8], b[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              a[q] = As[kk * 128 + ty * 4 + q];
              a[q + 4] = As[kk * 128 + 64 + ty * 4 + q];
              b[q] = Bs[kk * 128 + tx * 4 + q];
              b[q + 4] = Bs[kk * 128 + 64 + tx * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 8; ++p)
#pragma unroll
              for (int q = 0; q < 8; ++q) acc[p][q] += a[p] * b[q];
          }
        }
        // the tile goes through shared memory so that C is read and written
        // in column-major order (coalesced)
        T* Ct = c.sm + 2 * 8 * 128;   // [128][129]
        __syncthreads();
#pragma unroll
        for (int p = 0; p < 8; ++p)
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int li = p < 4 ? ty * 4 + p : 64 + ty * 4 + p - 4;
            const int lj = q < 4 ? tx * 4 + q : 64 + tx * 4 + q - 4;
            Ct[li + lj * 129] = acc[p][q];
          }
        __syncthreads();
        const int mt = min(128, m - m0), ntl = min(128, n - n0);
        for (int t = tid; t < mt * ntl; t += nt) {
          const int li = t % mt, lj = t / mt;
          const long long ci = vidx(o.C, m0 + li, n0 + lj);
          ar[ci] = (beta == (T)0 ? (T)0 : beta * ar[ci]) + alpha * Ct[li + lj * 129];
        }
      }
    __syncthreads();
    return;
  }
  // tiled: 64 x 64 C tiles, k in chunks of 16, 4 x 4 per thread
  T* As = c.sm;            // [16][64]
  T* Bs = c.sm + 16 * 64;  // [16][64]
  const int tx = tid & 15, ty = tid >> 4;
  for (int m0 = 0; m0 < m; m0 += 64)
    for (int n0 = 0; n0 < n; n0 += 64) {
      T acc[4][4];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
      for (int k0 = 0; k0 < k; k0 += 16) {
        for (int t = tid; t < 16 * 64; t += nt) {
          int kk = t / 64, ii = t % 64;
          int gi = m0 + ii, gk = k0 + kk;
          As[kk * 64 + ii] = (gi < m && gk < k) ? ar[vidx(o.A, gi, gk)] : (T)0;
          int gj = n0 + ii;
          Bs[kk * 64 + ii] = (gj < n && gk < k) ? ar[vidx(o.B, gk, gj)] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          T a[4], b[4];
          for (int q = 0; q < 4; ++q) {
            a[q] = As[kk * 64 + ty * 4 + q];
            b[q] = Bs[kk * 64 + tx * 4 + q];
          }
          for (int p = 0; p < 4; ++p)
            for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
        }
        __syncthreads();
      }
      for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
          int gi = m0 + ty * 4 + p, gj = n0 + tx * 4 + q;
          if (gi < m && gj < n) {
            long long ci = vidx(o.C, gi, gj);
            ar[ci] = (beta == (T)0 ? (T)0 : beta * ar[ci]) + alpha * acc[p][q];
          }
        }
    }
}

// C <- A C (A n x n, n <= 128): A (column-major) and a 32-column panel of C
// (row-major, ld 33) staged in shared memory; thread (ty, tx) computes rows
// 4ty..4ty+3 and columns tx, tx+8, tx+16, tx+24 of the panel.  Every shared
// load is a broadcast or hits 8 distinct banks.
template <class T>
__device__ void op_trmm_l(const HOp& o, HCtx<T>& c) {
  const int n = dimv(o.C.r, c.rk), cc = dimv(o.C.c, c.rk);
  if (n <= 0 || cc <= 0) return;
  T* ar = c.ar;
  if constexpr (sizeof(T) == 8) {
    if (c.leaf32 && cc > 4) {   // FP64 part of a mixed factor: FP32 arithmetic
      trmm_l_f32_on_f64(o, c, n, cc);
      return;
    }
  }
  if constexpr (sizeof(T) == 4) {
    // C <- A C on the tensor cores (C staged before it is overwritten)
    if (c.tc && n == 128 && cc >= 16 && cc <= 256 && (cc & 15) == 0 &&
        (long long)(128 + cc) * 128 + 1024 <= c.smcap) {
      if (tc_gemm128(c, o.A, o.C, o.C, 0, cc, 128, 1.f, 0.f)) return;
    }
  }
  if (cc <= 4 && !o.A.tr) {
    // a few right-hand sides (the H-solves): 2 threads per row split k, four
    // independent loads in flight per thread, A read from L2 (consecutive
    // threads, consecutive rows), partial sums combined in shared memory
    T* Pv = c.sm;            // n x cc
    T* red = c.sm + n * cc;  // 128 x cc partials of the second half
    for (int t = threadIdx.x; t < n * cc; t += blockDim.x) Pv[t] = ar[vidx(o.C, t % n, t / n)];
    __syncthreads();
    const int r = threadIdx.x & 127, part = threadIdx.x >> 7;
    const int kh = (n + 1) / 2, k0 = part * kh, k1 = min(n, k0 + kh);
    const T* Ac = ar + o.A.off + r;
    const long long ld = o.A.ld;
    T acc[4] = {0, 0, 0, 0};
    if (r < n) {
      int k = k0;
      for (; k + 4 <= k1; k += 4) {
        T a0 = Ac[k * ld], a1 = Ac[(k + 1) * ld], a2 = Ac[(k + 2) * ld], a3 = Ac[(k + 3) * ld];
        for (int j = 0; j < cc; ++j)
          acc[j] += a0 * Pv[k + j * n] + a1 * Pv[k + 1 + j * n] + a2 * Pv[k + 2 + j * n] +
                    a3 * Pv[k + 3 + j * n];
      }
      for (; k < k1; ++k) {
        T a = Ac[k * ld];
        for (int j = 0; j < cc; ++j) acc[j] += a * Pv[k + j * n];
      }
    }
    if (part == 1 && r < n)
      for (int j = 0; j < cc; ++j) red[r + j * 128] = acc[j];
    __syncthreads();
    if (part == 0 && r < n)
      for (int j = 0; j < cc; ++j) ar[vidx(o.C, r, j)] = acc[j] + red[r + j * 128];
    __syncthreads();
    return;
  }
  T* As = c.sm;            // n x n, [i + k n]
  T* Pn = c.sm + n * n;    // n x 32, [k * 33 + j]
  const int tid = threadIdx.x;
  stage_view(As, n, ar, o.A, n, n);
  const int tx = tid & 7, ty = tid >> 3;
  for (int c0 = 0; c0 < cc; c0 += 32) {
    const int cp = min(32, cc - c0);
    __syncthreads();
    for (int t = tid; t < n * cp; t += blockDim.x) {
      int i = t % n, j = t / n;
      cp_async_elem(Pn + i * 33 + j, ar + vidx(o.C, i, c0 + j));
    }
    cp_async_wait_all();
    __syncthreads();
    for (int rb = ty * 4; rb < n; rb += 128) {
      T acc[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0;
      for (int k = 0; k < n; ++k) {
        T a[4], b[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) a[p] = (rb + p < n) ? As[rb + p + k * n] : (T)0;
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = Pn[k * 33 + tx + 8 * q];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (rb + p < n && tx + 8 * q < cp) ar[vidx(o.C, rb + p, c0 + tx + 8 * q)] = acc[p][q];
    }
  }
  __syncthreads();
}

// C <- C A (A n x n, n <= 128): A (row-major) and a 32-row panel of C
// (column-major) in shared memory; thread (ty, tx) computes rows
// 4ty..4ty+3 and columns tx, tx+32, tx+64, tx+96.
template <class T>
__device__ void op_trmm_r(const HOp& o, HCtx<T>& c) {
  const int m = dimv(o.C.r, c.rk), n = dimv(o.C.c, c.rk);
  if (m <= 0 || n <= 0) return;
  T* ar = c.ar;
  if constexpr (sizeof(T) == 8) {
    if (c.leaf32) {   // FP64 part of a mixed factor: FP32 arithmetic
      trmm_r_f32_on_f64(o, c, m, n);
      return;
    }
  }
  if constexpr (sizeof(T) == 4) {
    // (C A)^T = A^T C^T on the tensor cores: M = n = 128, N = m, stored back transposed
    if (c.tc && n == 128 && m >= 16 && m <= 256 && (m & 15) == 0 &&
        (long long)(128 + m) * 128 + 1024 <= c.smcap) {
      const View At{o.A.off, o.A.c, o.A.r, o.A.ld, !o.A.tr};
      const View Ct{o.C.off, o.C.c, o.C.r, o.C.ld, !o.C.tr};
      if (tc_gemm128(c, At, Ct, o.C, 1, m, 128, 1.f, 0.f)) return;
    }
  }
  // A row-major with a padded row (lda = n + 1: the staging stores meet 4-way
  // bank conflicts at most, the row reads none)
  const int lda = n + 1;
  T* As = c.sm;                                 // n x n, [k lda + j]
  T* Pn = c.sm + (((long long)n * lda + 3) & ~3LL);   // 32 x n, [i + k * 32] (16-byte aligned)
  const int tid = threadIdx.x;
  bool vec = false;
  if constexpr (sizeof(T) == 4)
    vec = !o.A.tr && (n & 3) == 0 && (o.A.off & 3) == 0 && (o.A.ld & 3) == 0;
  if (vec) {
    // A (column-major, aligned) read with 16-byte loads, stored row-major
    const int n4 = n >> 2, tot = n4 * n;
    for (int t0 = tid; t0 < tot; t0 += 4 * blockDim.x) {
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = t0 + q * blockDim.x;
        if (t < tot)
          v[q] = *reinterpret_cast<const float4*>(ar + o.A.off + 4LL * (t % n4) + (long long)(t / n4) * o.A.ld);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = t0 + q * blockDim.x;
        if (t < tot) {
          const int i = 4 * (t % n4), j = t / n4;
          As[(i + 0) * lda + j] = v[q].x;
          As[(i + 1) * lda + j] = v[q].y;
          As[(i + 2) * lda + j] = v[q].z;
          As[(i + 3) * lda + j] = v[q].w;
        }
      }
    }
  } else {
    for (int t = tid; t < n * n; t += blockDim.x)
      cp_async_elem(As + (t % n) * lda + t / n, ar + vidx(o.A, t % n, t / n));
  }
  const int tx = tid & 31, ty = tid >> 5;
  for (int r0 = 0; r0 < m; r0 += 32) {
    const int rp = min(32, m - r0);
    __syncthreads();
    if (rp == 32) {
      View Cr = o.C;   // rows r0 .. r0 + 31
      Cr.off = vidx(o.C, r0, 0);
      stage_view(Pn, 32, ar, Cr, 32, n);
    } else {
      for (int t = tid; t < rp * n; t += blockDim.x)
        cp_async_elem(Pn + (t % rp) + (t / rp) * 32, ar + vidx(o.C, r0 + t % rp, t / rp));
    }
    cp_async_wait_all();
    __syncthreads();
    T acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = 0;
    for (int k = 0; k < n; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) a[p] = Pn[ty * 4 + p + k * 32];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = (tx + 32 * q < n) ? As[k * lda + tx + 32 * q] : (T)0;
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (ty * 4 + p < rp && tx + 32 * q < n) ar[vidx(o.C, r0 + ty * 4 + p, tx + 32 * q)] = acc[p][q];
  }
  __syncthreads();
}

// Unpivoted LU of C (n x n, n <= 128) in shared memory, returning L^-1 and
// U^-1 (L itself is never needed).  Step k of the elimination updates the
// trailing block and, in the same pass, X <- E_k X with E_k the k-th
// elimination matrix, so X ends as L^-1; every value a step reads is left
// untouched by that step, hence one barrier per step.  U^-1 = (D^-1 U)^-1 D^-1
// with D = diag(U), again one barrier per step.
// named barriers of the leaf LU (ids 1 and 2, all threads of the CTA)
__device__ __forceinline__ void nbar_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"((int)blockDim.x) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"((int)blockDim.x) : "memory");
}

// FP32 leaves (n <= 128), register resident: thread (tx, ty) holds rows
// tx + 32 r (r < 4) and columns ty + 8 q (q < 16) of the matrix and of the
// inverse being built.  Forward elimination (S -> U, X -> L^-1): row k of a
// warp's own columns comes from lane k mod 32 of the same warp (shuffles);
// only column k (the multipliers) crosses warps.  Its owner computes it one
// step ahead (look-ahead: it applies step k - 1 to column k first), publishes
// it in a double-buffered shared vector and arrives at a named barrier (ids
// alternate), on which the other warps wait; the owner goes on with the rest
// of step k - 1 meanwhile.  Backward ((D^-1 U)^-1): the scaled upper factor
// is published once, after which each warp eliminates its own columns
// without any barrier.  The outer loop over column blocks of 8 is unrolled so
// that every register index is static.
template <class T>
__device__ void getrf_inv_reg(const HOp& o, HCtx<T>& c) {
  const int n = o.C.r;
  T* ar = c.ar;                  // FP32 arithmetic whatever the arena's type
  float* colb = reinterpret_cast<float*>(c.sm);   // [2][128] multipliers of a step
  float* Ut = colb + 256;        // [128][129] scaled upper factor (row-major, padded)
  float* diag = Ut + 128 * 129;  // [128]
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  unsigned long long tq = 0;
  auto tmk = [&](int k) {   // profiling: phase times in tprof[11..14]
    if (!c.tprof || tid != 0) return;
    unsigned long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (k >= 0) atomicAdd(c.tprof + 11 + k, t1 - tq);
    tq = t1;
  };
  tmk(-1);
  float S[4][16], X[4][16];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = tx + 32 * r, j = ty + 8 * q;
      S[r][q] = (i < n && j < n) ? (float)ar[vidx(o.C, i, j)] : 0.f;
      X[r][q] = (i == j && i < n) ? 1.f : 0.f;
    }
  // publish the multipliers of step kn from local column cc, pivot in
  // register row rr of lane kn mod 32
  auto publish = [&](const float (&col)[4], float pv, int kn) {
    if (tx == 0 && (pv == 0.f || !isfinite(pv))) atomicExch(c.err, 1);
    const float inv = 1.f / pv;
    float* cb_ = colb + 128 * (kn & 1);
#pragma unroll
    for (int r = 0; r < 4; ++r) cb_[tx + 32 * r] = col[r] * inv;
    nbar_arrive(1 + (kn & 1));
  };
  tmk(0);
  if (n > 0 && ty == 0) {   // step 0: column 0 is owned by warp 0 (local column 0)
    const float col[4] = {S[0][0], S[1][0], S[2][0], S[3][0]};
    publish(col, __shfl_sync(0xffffffffu, S[0][0], 0), 0);
  }
#pragma unroll
  for (int cb = 0; cb < 16; ++cb) {
    const int rb = cb >> 2;   // register row block of rows 8 cb .. 8 cb + 7
    if (8 * cb >= n) break;
    for (int q = 0; q < 8; ++q) {
      const int k = 8 * cb + q;
      if (k >= n) break;
      if (ty != q) nbar_sync(1 + (k & 1));
      const float* col = colb + 128 * (k & 1);
      float l[4], rs[16], rx[16];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = tx + 32 * r;
        l[r] = (r >= rb && i > k) ? col[i] : 0.f;
      }
      // look-ahead first (it is on the critical path): the owner of column
      // k + 1 applies step k to it and publishes the multipliers of step k + 1
      const int kn = k + 1;
      bool la = false;
      if (kn < n) {
        if (q < 7) {   // column 8 cb + q + 1: warp q + 1, local column cb, pivot row block rb
          if (ty == q + 1) {
            const float rk = __shfl_sync(0xffffffffu, S[rb][cb], k & 31);
#pragma unroll
            for (int r = rb; r < 4; ++r) S[r][cb] -= l[r] * rk;
            const float cl[4] = {S[0][cb], S[1][cb], S[2][cb], S[3][cb]};
            publish(cl, __shfl_sync(0xffffffffu, S[rb][cb], kn & 31), kn);
            la = true;
          }
        } else if (cb + 1 < 16) {   // column 8 (cb + 1): warp 0, local column cb + 1
          if (ty == 0) {
            const int rn = (cb + 1) >> 2;
            const float rk = __shfl_sync(0xffffffffu, S[rb][cb + 1], k & 31);
#pragma unroll
            for (int r = rb; r < 4; ++r) S[r][cb + 1] -= l[r] * rk;
            const float cl[4] = {S[0][cb + 1], S[1][cb + 1], S[2][cb + 1], S[3][cb + 1]};
            float pv;
            if (rn == 0) pv = __shfl_sync(0xffffffffu, S[0][cb + 1], kn & 31);
            else if (rn == 1) pv = __shfl_sync(0xffffffffu, S[1][cb + 1], kn & 31);
            else if (rn == 2) pv = __shfl_sync(0xffffffffu, S[2][cb + 1], kn & 31);
            else pv = __shfl_sync(0xffffffffu, S[3][cb + 1], kn & 31);
            publish(cl, pv, kn);
            la = true;
          }
        }
      }
      // row k of this warp's columns (lane k mod 32)
#pragma unroll
      for (int c2 = 0; c2 < 16; ++c2) {
        rs[c2] = (c2 >= cb) ? __shfl_sync(0xffffffffu, S[rb][c2], k & 31) : 0.f;
        rx[c2] = (c2 <= cb) ? __shfl_sync(0xffffffffu, X[rb][c2], k & 31) : 0.f;
      }
      const int lac = (q < 7) ? cb : cb + 1;   // the look-ahead column, when la
#pragma unroll
      for (int r = rb; r < 4; ++r)
#pragma unroll
        for (int c2 = 0; c2 < 16; ++c2) {
          if (la && c2 == lac) continue;
          if (c2 > cb) S[r][c2] -= l[r] * rs[c2];
          else if (c2 < cb) X[r][c2] -= l[r] * rx[c2];
          else if (ty > q) S[r][c2] -= l[r] * rs[c2];
          else X[r][c2] -= l[r] * rx[c2];
        }
    }
  }
  tmk(1);
  // L^-1 out; diagonal of U to shared memory
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = tx + 32 * r, j = ty + 8 * q;
      if (i < n && j < n) ar[vidx(o.A, i, j)] = (T)X[r][q];
      if (i == j && i < n) diag[i] = S[r][q];
    }
  __syncthreads();
  // the scaled upper factor D^-1 U (strict upper part) to shared memory
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = tx + 32 * r;
    const float ri = (i < n) ? 1.f / diag[i] : 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int j = ty + 8 * q;
      if (i < n && j < n && j > i) Ut[i * 129 + j] = S[r][q] * ri;
      X[r][q] = (i == j && i < n) ? 1.f : 0.f;
    }
  }
  __syncthreads();
  tmk(2);
  if (c.tprof && tid == 0) atomicAdd(c.tprof + 15, 1ULL);
  // backward: X[i][j] -= Ut[i][k] X[k][j] for i < k <= j, each warp alone
#pragma unroll
  for (int cb = 15; cb >= 0; --cb) {
    const int rb = cb >> 2;
    if (8 * cb < n) {
      for (int q = 7; q >= 0; --q) {
        const int k = 8 * cb + q;
        if (k >= n || k == 0) continue;
        float u[4], rv[16];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int i = tx + 32 * r;
          u[r] = (r <= rb && i < k) ? Ut[i * 129 + k] : 0.f;
        }
#pragma unroll
        for (int c2 = 0; c2 < 16; ++c2) rv[c2] = (c2 >= cb) ? __shfl_sync(0xffffffffu, X[rb][c2], k & 31) : 0.f;
#pragma unroll
        for (int r = 0; r <= rb; ++r)
#pragma unroll
          for (int c2 = cb; c2 < 16; ++c2) X[r][c2] -= u[r] * rv[c2];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int j = ty + 8 * q;
    if (j >= n) continue;
    const float cj = 1.f / diag[j];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = tx + 32 * r;
      if (i < n) ar[vidx(o.B, i, j)] = (T)(X[r][q] * cj);
    }
  }
  tmk(3);
}

template <class T>
__device__ void op_getrf_inv(const HOp& o, HCtx<T>& c) {
  const int n = o.C.r;
  if (n <= 0) return;
  if (n <= 128 && (sizeof(T) == 4 || c.leaf32)) {
    getrf_inv_reg(o, c);
    return;
  }
  T* ar = c.ar;
  T* S = c.sm;             // n x n, [i + j n]
  T* X = c.sm + n * n;     // n x n
  const int tid = threadIdx.x;
  const int tx = tid & 31, ty = tid >> 5;   // a warp covers 32 consecutive rows of one column
  for (int t = tid; t < n * n; t += blockDim.x) {
    S[t] = ar[vidx(o.C, t % n, t / n)];
    X[t] = (t % n == t / n) ? (T)1 : (T)0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const T piv = S[k + k * n];
    if (tid == 0 && (piv == (T)0 || !isfinite((double)piv))) atomicExch(c.err, 1);
    const T inv = (T)1 / piv;
    // this thread's rows i = k+1+tx+32r (n <= 128: at most 4): multipliers
    // in registers, then columns j > k of S and j <= k of X (n in all)
    T l[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int i = k + 1 + tx + 32 * r;
      l[r] = (i < n) ? S[i + k * n] * inv : (T)0;
    }
    for (int j = ty; j < n; j += 8) {
      const bool lu = j > k;
      const T rk = lu ? S[k + j * n] : X[k + j * n];
      T* dst = (lu ? S : X) + j * n;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int i = k + 1 + tx + 32 * r;
        if (i < n) dst[i] -= l[r] * rk;
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < n * n; t += blockDim.x) ar[vidx(o.A, t % n, t / n)] = X[t];
  // (D^-1 U)^-1 by backward elimination of the unit upper factor: first
  // scale the strict upper part of S row by row (one division per entry)
  __syncthreads();
  for (int t = tid; t < n * n; t += blockDim.x) {
    int i = t % n, j = t / n;
    X[t] = (i == j) ? (T)1 : (T)0;
    if (j > i) S[t] = S[t] / S[i + i * n];
  }
  __syncthreads();
  for (int k = n - 1; k > 0; --k) {
    T u[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int i = tx + 32 * r;
      u[r] = (i < k) ? S[i + k * n] : (T)0;
    }
    for (int j = k + ty; j < n; j += 8) {
      const T xkj = X[k + j * n];
      T* dst = X + j * n;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int i = tx + 32 * r;
        if (i < k) dst[i] -= u[r] * xkj;
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < n * n; t += blockDim.x) {
    int i = t % n, j = t / n;
    ar[vidx(o.B, i, j)] = X[t] / S[j + j * n];
  }
}

// Householder QR of A (m x K, ld m) in place: R in the upper trapezoid,
// reflectors v (v_0 = 1 implied) below, tau[j]; kr = min(m, K) reflectors.
// Warp w owns the columns l = w mod (warps).  Step j: every warp forms the
// reflector of column j itself (x0 = A[j][j], sigma = sum_{i>j} A[i][j]^2),
// then applies it to its own columns l > j (w_l = A[j][l] + d_l / v0 with
// d_l = sum_{i>j} A[i][j] A[i][l]); the owner of column j scales its
// reflector at the start of step j + 1, when no warp reads it any more.  One
// barrier per step.
// barrier of the warps [w0, w0 + nw) (the whole CTA when nw covers it)
__device__ __forceinline__ void group_sync(int nw, int bar_id) {
  if (nw * 32 == (int)blockDim.x) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nw * 32) : "memory");
  }
}

template <class T>
__device__ void house_qr(T* A, int m, int K, T* tau, int w0 = 0, int nw_ = 0, int bar_id = 0) {
  const int kr = min(m, K);
  const int nw = nw_ ? nw_ : (int)(blockDim.x >> 5);
  const int lane = threadIdx.x & 31, warp = (int)(threadIdx.x >> 5) - w0;
  T pv0 = (T)0;   // v0 of the previous step (used by the owner of its column)
  for (int j = 0; j < kr; ++j) {
    // the owner of column j - 1 turns it into its reflector
    if (j > 0 && ((j - 1) % nw) == warp && pv0 != (T)0) {
      T* col = A + (long long)(j - 1) * m;
      const T inv = (T)1 / pv0;
      for (int i = j + lane; i < m; i += 32) col[i] *= inv;
    }
    const T* cj = A + (long long)j * m;
    T sg = (T)0;
    for (int i = j + 1 + lane; i < m; i += 32) sg += cj[i] * cj[i];
    for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
    const T x0 = cj[j];
    const T sn = sqrt(x0 * x0 + sg);
    const T alpha = (x0 >= (T)0) ? -sn : sn;
    const T v0 = x0 - alpha;
    const bool trivial = (sn == (T)0) || (v0 == (T)0) || sg == (T)0;
    const T tj = trivial ? (T)0 : (alpha - x0) / alpha;
    if (!trivial) {
      const T iv0 = (T)1 / v0;
      for (int l = j + 1 + ((warp - (j + 1)) % nw + nw) % nw; l < K; l += nw) {
        T* cl = A + (long long)l * m;
        T d = (T)0;
        for (int i = j + 1 + lane; i < m; i += 32) d += cj[i] * cl[i];
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        const T w = (cl[j] + d * iv0) * tj;
        __syncwarp();
        if (lane == 0) cl[j] -= w;
        const T wv = w * iv0;
        for (int i = j + 1 + lane; i < m; i += 32) cl[i] -= wv * cj[i];
      }
    }
    group_sync(nw, bar_id);
    if ((j % nw) == warp && lane == 0) {
      tau[j] = tj;
      if (!trivial) A[j + (long long)j * m] = alpha;
    }
    pv0 = trivial ? (T)0 : v0;
  }
  // the last reflector
  if (kr > 0 && ((kr - 1) % nw) == warp && pv0 != (T)0) {
    T* col = A + (long long)(kr - 1) * m;
    const T inv = (T)1 / pv0;
    for (int i = kr + lane; i < m; i += 32) col[i] *= inv;
  }
  group_sync(nw, bar_id);
}

// Y (m x r, ld ldy) <- Q Y with Q = H_0 ... H_{kr-1} stored in A (m x K)
template <class T>
__device__ void apply_q(const T* A, int m, int K, const T* tau, T* Y, int ldy, int r, int w0 = 0,
                        int nw_ = 0, int bar_id = 0) {
  const int kr = min(m, K);
  const int nw = nw_ ? nw_ : (int)(blockDim.x >> 5);
  const int lane = threadIdx.x & 31, warp = (int)(threadIdx.x >> 5) - w0;
  for (int j = kr - 1; j >= 0; --j) {
    T tj = tau[j];
    if (tj != (T)0) {
      for (int col = warp; col < r; col += nw) {
        T w = 0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + (long long)j * m] * Y[i + (long long)col * ldy];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        w = __shfl_sync(0xffffffffu, w, 0);
        w = (w + Y[j + (long long)col * ldy]) * tj;
        if (lane == 0) Y[j + (long long)col * ldy] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) Y[i + (long long)col * ldy] -= w * A[i + (long long)j * m];
      }
    }
    group_sync(nw, bar_id);
  }
}

// house_qr of A (m x K, global) run on a shared-memory copy when m K <= cap
template <class T>
__device__ void qr_staged(T* A, int m, int K, T* tau, T* red, T* stage, long long cap) {
  const long long mk = (long long)m * K;
  if (mk > cap) {
    house_qr(A, m, K, tau);
    return;
  }
  for (long long t = threadIdx.x; t < mk; t += blockDim.x) stage[t] = A[t];
  __syncthreads();
  house_qr(stage, m, K, tau);
  for (long long t = threadIdx.x; t < mk; t += blockDim.x) A[t] = stage[t];
  __syncthreads();
}

// Y (m x r, ld m, global) <- Q Y, with Q and Y copied to shared memory when
// m (K + r) <= cap
template <class T>
__device__ void apply_q_staged(const T* A, int m, int K, const T* tau, T* Y, int r, T* stage,
                               long long cap) {
  const long long mk = (long long)m * K, mr = (long long)m * r;
  if (mk + mr > cap) {
    apply_q(A, m, K, tau, Y, m, r);
    return;
  }
  T* Ys = stage + mk;
  for (long long t = threadIdx.x; t < mk; t += blockDim.x) stage[t] = A[t];
  for (long long t = threadIdx.x; t < mr; t += blockDim.x) Ys[t] = Y[t];
  __syncthreads();
  apply_q(stage, m, K, tau, Ys, m, r);
  for (long long t = threadIdx.x; t < mr; t += blockDim.x) Y[t] = Ys[t];
  __syncthreads();
}

// Column-pivoted Householder QR of the core M (ku x kv, ld K), M Pi = Q_M R_M,
// stopped at the first pivot below tol |R_M(0,0)| or after rmax steps; then
// Z = Q_M [I_r; 0] (ku x r, ld K).  On return M holds R_M above its diagonal
// and the reflectors below, piv the column permutation.  Returns r (the same
// in every thread).  Called by the whole CTA.
template <class T, class F>
__device__ int core_rrqr(T* M, int K, int ku, int kv, int rmax, double tol, T* tauM, T* cn, int* piv,
                         T* Z, F tmk3) {
  for (int j = threadIdx.x; j < kv; j += blockDim.x) piv[j] = j;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int r = 0;
  __shared__ int s_stop;
  __shared__ T s_r0;
  for (int st = 0; st < rmax; ++st) {
    // exact norms of the remaining parts of the columns (a warp per column)
    for (int j = st + warp; j < kv; j += nw) {
      T a = 0;
      for (int i = st + lane; i < ku; i += 32) a += M[i + j * K] * M[i + j * K];
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) cn[j] = a;
    }
    __syncthreads();
    // warp 0: pivot (largest remaining norm), stop test, swap, reflector
    if (warp == 0) {
      T best = (T)-1;
      int p = st;
      for (int j = st + lane; j < kv; j += 32)
        if (cn[j] > best) {
          best = cn[j];
          p = j;
        }
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) {
          best = ob;
          p = op;
        }
      }
      const T nrm = sqrt(fmax(best, (T)0));
      if (st == 0 && lane == 0) s_r0 = nrm;
      __syncwarp();
      const int stop = (nrm == (T)0 || (st > 0 && nrm <= (T)tol * s_r0)) ? 1 : 0;
      if (lane == 0) s_stop = stop;
      if (!stop) {
        if (p != st) {
          for (int i = lane; i < ku; i += 32) {
            const T a = M[i + st * K];
            M[i + st * K] = M[i + p * K];
            M[i + p * K] = a;
          }
          if (lane == 0) {
            const int a = piv[st];
            piv[st] = piv[p];
            piv[p] = a;
          }
        }
        __syncwarp();
        T a = 0;
        for (int i = st + 1 + lane; i < ku; i += 32) a += M[i + st * K] * M[i + st * K];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        const T x0 = M[st + st * K];
        const T sn = sqrt(x0 * x0 + a);
        const T alpha = (x0 >= (T)0) ? -sn : sn;
        const T v0 = x0 - alpha;
        const bool trivial = (sn == (T)0) || (v0 == (T)0) || a == (T)0;
        __syncwarp();
        if (!trivial) {
          const T iv = (T)1 / v0;
          for (int i = st + 1 + lane; i < ku; i += 32) M[i + st * K] *= iv;
        }
        __syncwarp();
        if (lane == 0) {
          tauM[st] = trivial ? (T)0 : (alpha - x0) / alpha;
          if (!trivial) M[st + st * K] = alpha;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const T tj = tauM[st];
    if (tj != (T)0)
      for (int l = st + 1 + warp; l < kv; l += nw) {
        T w = 0;
        for (int i = st + 1 + lane; i < ku; i += 32) w += M[i + st * K] * M[i + l * K];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w = (w + M[st + l * K]) * tj;
        __syncwarp();
        if (lane == 0) M[st + l * K] -= w;
        for (int i = st + 1 + lane; i < ku; i += 32) M[i + l * K] -= w * M[i + st * K];
      }
    __syncthreads();
    r = st + 1;
  }
  // (all threads agree on r: every exit is uniform)
  tmk3();
  // Z = Q_M [I_r; 0] (ku x r): apply the r reflectors of M in reverse
  for (int t = threadIdx.x; t < ku * r; t += blockDim.x) Z[(t % ku) + (t / ku) * K] = (t % ku == t / ku) ? (T)1 : (T)0;
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    T tj = tauM[j];
    if (tj != (T)0)
      for (int col = warp; col < r; col += nw) {
        T w = 0;
        for (int i = j + 1 + lane; i < ku; i += 32) w += M[i + j * K] * Z[i + col * K];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        w = __shfl_sync(0xffffffffu, w, 0);
        w = (w + Z[j + col * K]) * tj;
        if (lane == 0) Z[j + col * K] -= w;
        for (int i = j + 1 + lane; i < ku; i += 32) Z[i + col * K] -= w * M[i + j * K];
      }
    __syncthreads();
  }
  return r;
}

// x y added to the double-float sum (hi, lo): the product is split exactly
// (x y = p + e by fma), the sum by TwoSum; explicit rounding intrinsics keep
// the compiler from contracting the error terms away.
__device__ __forceinline__ void df_add_prod(float& hi, float& lo, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float e = __fmaf_rn(x, y, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float h2, float l2) {
  const float s = __fadd_rn(hi, h2);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, l2));
}

// 1/sqrt(d) for d > 0 in FP64 by Newton-Raphson, y <- y (3 - d y^2) / 2, from
// the FP32 estimate rsqrtf (~2^-22 relative error): one step when d is well
// inside FP32 range; otherwise on the mantissa m of d scaled to [0.5, 2) with
// an even exponent, two steps (below FP64 rounding), then the exponent is
// put back.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (d > 1e-30 && d < 1e30) {
    // in FP32 range: one step from the FP32 estimate leaves ~3e-13 relative
    // error, far below what the FP32 factors built from it can hold
    double y = (double)rsqrtf((float)d);
    return y * (1.5 - 0.5 * d * y * y);
  }
  int e;
  double mt = frexp(d, &e);   // d = mt 2^e, mt in [0.5, 1)
  if (e & 1) {
    mt *= 2.0;
    e -= 1;
  }
  double y = (double)rsqrtf((float)mt);
  y = y * (1.5 - 0.5 * mt * y * y);
  y = y * (1.5 - 0.5 * mt * y * y);
  return ldexp(y, -e / 2);
}

// Pivoted Cholesky of the symmetric K x K matrix G (row-major, K <= 32, FP64)
// by one warp: Pi^T G Pi = R^T R + E, stopped when the largest remaining
// diagonal falls to thr times the first pivot.  R (rank x K, pivoted column
// order) overwrites the upper triangle of G's first rank rows; piv[q] is the
// original column of pivoted column q; invd[q] = 1 / R[q][q] (FP32).
// Returns the rank (in every lane).  The pivot is chosen on FP32 copies of
// the remaining diagonal (FP64 instructions are the scarce resource here).
__device__ int pchol_warp(double* G, int K, int* piv, float* invd, double thr) {
  const int lane = threadIdx.x & 31;
  if (lane < K) piv[lane] = lane;
  __syncwarp();
  double d0 = 0.0;
  int r = 0;
  for (int k = 0; k < K; ++k) {
    float best = -1.f;
    int p = k;
    if (lane >= k && lane < K) {
      best = (float)G[lane * K + lane];
      if (!(best >= 0.f)) best = -1.f;   // NaN or negative: never a pivot
      p = lane;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, p, o);
      if (ob > best || (ob == best && op < p)) {
        best = ob;
        p = op;
      }
    }
    const double dp = G[p * K + p];
    if (k == 0) d0 = dp;
    if (!(dp > 0.0) || !(dp > thr * d0)) break;
    if (p != k) {   // symmetric swap of k and p (columns across every row: R's too)
      if (lane < K) {
        const double a = G[k * K + lane];
        G[k * K + lane] = G[p * K + lane];
        G[p * K + lane] = a;
      }
      __syncwarp();
      if (lane < K) {
        const double a = G[lane * K + k];
        G[lane * K + k] = G[lane * K + p];
        G[lane * K + p] = a;
      }
      if (lane == 0) {
        const int a = piv[k];
        piv[k] = piv[p];
        piv[p] = a;
      }
      __syncwarp();
    }
    const double inv = rsqrt_newton(dp);   // dp = G[k][k] after the swap
    __syncwarp();
    if (lane > k && lane < K) G[k * K + lane] *= inv;
    if (lane == 0) {
      G[k * K + k] = dp * inv;
      invd[k] = (float)inv;
    }
    __syncwarp();
    if (lane > k && lane < K) {
      const double rkj = G[k * K + lane];
      for (int i = k + 1; i < K; ++i) G[i * K + lane] -= G[k * K + i] * rkj;
    }
    __syncwarp();
    r = k + 1;
  }
  return r;
}

// c = R11^-1 z by one warp in FP32 (backward stable): R11 the leading n x n
// upper triangle of R (row-major, ld K), invd its inverse diagonal; z and out
// are vectors (out may be z)
__device__ void backsub_warp(const float* R, const float* invd, int K, int n, const float* z,
                             float* out) {
  const int lane = threadIdx.x & 31;
  float cq = 0.f;
  for (int i = n - 1; i >= 0; --i) {
    float part = (lane > i && lane < n) ? R[i * K + lane] * cq : 0.f;
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == i) cq = (z[i] - part) * invd[i];
  }
  __syncwarp();   // every z[i] is read before out (which may be z) is written
  if (lane < n) out[lane] = cq;
}

// Shared-memory floats in front of the staged factors in trunc_gram
// (Gram matrices in FP64, the small FP32 work arrays, pivots)
__host__ __device__ __forceinline__ long long gram_small(int K) {
  return ((long long)(12 * K * K + 7 * K) + 3) & ~3LL;
}

// n consecutive floats global -> shared as asynchronous copies (16-byte ones
// when both sides are aligned), every copy in flight at once; the caller
// waits (cp_async_wait_all) and synchronises
__device__ __forceinline__ void cp_async_range(float* dst, const float* src, long long n) {
  long long t0 = 0;
  if (((smem_u32(dst) & 15u) == 0) && ((reinterpret_cast<unsigned long long>(src) & 15ULL) == 0)) {
    const long long n4 = n >> 2;
    for (long long t = threadIdx.x; t < n4; t += blockDim.x) cp_async16(dst + 4 * t, src + 4 * t);
    t0 = n4 << 2;
  }
  for (long long t = t0 + threadIdx.x; t < n; t += blockDim.x) cp_async_elem(dst + t, src + t);
}

// Recompression of FP32 factors from their Gram matrices (K <= 32): G_U = U^T U
// and G_V = V^T V summed exactly in double-float from the FP32 entries, pivoted
// Cholesky in FP64, U Pi_U = Q_U R_U with Q_U = (U Pi_U)[:, :r_u] R_U11^-1
// (directions whose remaining diagonal falls below 2^-40 of the first are
// dropped: singular values under ~1e-6 of the largest, the FP32 rounding
// level of the factors); then the core RRQR of the Householder path on
// M = (R_U Pi_U^T)(R_V Pi_V^T)^T and
//   U_new = (U Pi_U)[:, :r_u] (R_U11^-1 Z),  V_new = (V Pi_V)[:, :r_v] (R_V11^-1 Pi_M R_M[:r, :]^T).
// The same truncated product as the Householder path, with a handful of CTA
// barriers instead of several per column.
// staged: the factors are already in shared memory at c.sm + gram_small(K)
// (U, m x K, then V, n x K); else they are read from Ut, Vt (staged here when
// they fit).
__device__ void trunc_gram(HCtx<float>& c, int slot, const float* Ut, const float* Vt, int K,
                           bool staged) {
  const SlotDev s = c.sl[slot];
  const int m = s.m, n = s.n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double* GU = reinterpret_cast<double*>(c.sm);        // K x K
  double* GV = GU + K * K;                             // K x K
  float* RUo = reinterpret_cast<float*>(GV + K * K);   // r_u x K (original columns)
  float* RVo = RUo + K * K;
  float* M = RVo + K * K;                              // core, ld K
  float* Z = M + K * K;
  float* WU = Z + K * K;                               // r_u x r, ld K
  float* WV = WU + K * K;                              // r_v x r (Y_V first), ld K
  float* RUp = WV + K * K;                             // R_U11, R_V11 in FP32 (pivoted order)
  float* RVp = RUp + K * K;
  float* tauM = RVp + K * K;
  float* cn = tauM + K;
  float* invdU = cn + K;
  float* invdV = invdU + K;
  int* pivU = reinterpret_cast<int*>(invdV + K);
  int* pivV = pivU + K;
  int* piv = pivV + K;
  const long long small = gram_small(K);
  float* stage = c.sm + small;
  const long long cap = c.smcap - small;
  __shared__ int s_ru, s_rv;
  unsigned long long tq = 0;
  auto tmk = [&](int k) {
    if (!c.tprof || tid != 0) return;
    unsigned long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (k >= 0) atomicAdd(c.tprof + k, t1 - tq);
    tq = t1;
  };
  tmk(-1);
  // the tall factors, staged when they fit
  const float* SU = Ut;
  const float* SV = Vt;
  if (staged) {
    SU = stage;
    SV = stage + (long long)m * K;
  } else if ((long long)(m + n) * K <= cap) {
    float* su = stage;
    float* sv = stage + (long long)m * K;
    cp_async_range(su, Ut, (long long)m * K);
    cp_async_range(sv, Vt, (long long)n * K);
    cp_async_wait_all();
    SU = su;
    SV = sv;
    __syncthreads();
  }
  // Gram matrices: a warp per 2 x 2 block (block row <= block column) of G_U,
  // then of G_V; four independent double-float sums per lane
  const int nb = (K + 1) / 2;
  const int EB = nb * (nb + 1) / 2;
  for (int task = warp; task < 2 * EB; task += nw) {
    const bool isv = task >= EB;
    int e = isv ? task - EB : task;
    int bi = 0;
    while (e >= nb - bi) {
      e -= nb - bi;
      ++bi;
    }
    const int bj = bi + e;
    const int i0 = 2 * bi, i1 = min(2 * bi + 1, K - 1), j0 = 2 * bj, j1 = min(2 * bj + 1, K - 1);
    const float* A = isv ? SV : SU;
    const int rows = isv ? n : m;
    const float* a0 = A + (long long)i0 * rows;
    const float* a1 = A + (long long)i1 * rows;
    const float* b0 = A + (long long)j0 * rows;
    const float* b1 = A + (long long)j1 * rows;
    float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = lane; t < rows; t += 32) {
      const float x0 = a0[t], x1 = a1[t], y0 = b0[t], y1 = b1[t];
      df_add_prod(h[0], l[0], x0, y0);
      df_add_prod(h[1], l[1], x0, y1);
      df_add_prod(h[2], l[2], x1, y0);
      df_add_prod(h[3], l[3], x1, y1);
    }
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float h2 = __shfl_xor_sync(0xffffffffu, h[q], o);
        const float l2 = __shfl_xor_sync(0xffffffffu, l[q], o);
        df_add(h[q], l[q], h2, l2);
      }
    }
    if (lane == 0) {
      double* G = isv ? GV : GU;
      const int ri[4] = {i0, i0, i1, i1}, cj[4] = {j0, j1, j0, j1};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double g = (double)h[q] + (double)l[q];
        G[ri[q] * K + cj[q]] = g;
        G[cj[q] * K + ri[q]] = g;
      }
    }
  }
  __syncthreads();
  tmk(0);
  // pivoted Cholesky of both, one warp each
  const double thr = 0x1p-40;
  if (warp == 0) {
    const int r = pchol_warp(GU, K, pivU, invdU, thr);
    if (lane == 0) s_ru = min(r, m);
  } else if (warp == 1) {
    const int r = pchol_warp(GV, K, pivV, invdV, thr);
    if (lane == 0) s_rv = min(r, n);
  }
  __syncthreads();
  tmk(1);
  const int ru = s_ru, rv = s_rv;
  float* Ud = c.ar + s.off;
  float* Vd = c.ar + s.off + (long long)m * s.kcap;
  if (ru == 0 || rv == 0) {
    if (tid == 0) c.rk[slot] = 0;
    __syncthreads();
    return;
  }
  // R in original column order, then the core M = RUo RVo^T (ru x rv, ld K)
  for (int t = tid; t < ru * K; t += nt) {
    const int i = t / K, q = t % K;
    const float v = (q >= i) ? (float)GU[i * K + q] : 0.f;
    RUo[i * K + pivU[q]] = v;
    RUp[i * K + q] = v;
  }
  for (int t = tid; t < rv * K; t += nt) {
    const int i = t / K, q = t % K;
    const float v = (q >= i) ? (float)GV[i * K + q] : 0.f;
    RVo[i * K + pivV[q]] = v;
    RVp[i * K + q] = v;
  }
  __syncthreads();
  for (int t = tid; t < ru * rv; t += nt) {
    const int i = t % ru, j = t / ru;
    float acc = 0.f;
    for (int l = 0; l < K; ++l) acc += RUo[i * K + l] * RVo[j * K + l];
    M[i + j * K] = acc;
  }
  tmk(2);
  const int rmax = min(min(ru, rv), s.kmax);
  const int r = core_rrqr(M, K, ru, rv, rmax, c.tol, tauM, cn, piv, Z, [&]() { tmk(3); });
  // Y_V = Pi_M R_M[:r, :]^T (rv x r), then the two triangular solves
  for (int t = tid; t < rv * r; t += nt) WV[(t % rv) + (t / rv) * K] = 0.f;
  __syncthreads();
  for (int t = tid; t < rv * r; t += nt) {
    const int j = t % rv, i = t / rv;   // R_M[i][j], j >= i
    if (j >= i) WV[piv[j] + i * K] = M[i + j * K];
  }
  __syncthreads();
  for (int task = warp; task < 2 * r; task += nw) {
    if (task < r) backsub_warp(RUp, invdU, K, ru, Z + task * K, WU + task * K);
    else backsub_warp(RVp, invdV, K, rv, WV + (task - r) * K, WV + (task - r) * K);
  }
  __syncthreads();
  tmk(4);
  // U_new = (U Pi_U)[:, :ru] W_U, V_new = (V Pi_V)[:, :rv] W_V
  for (long long t = tid; t < (long long)m * r; t += nt) {
    const int i = (int)(t % m), j = (int)(t / m);
    float acc = 0.f;
    for (int q = 0; q < ru; ++q) acc += SU[i + (long long)pivU[q] * m] * WU[q + j * K];
    Ud[i + (long long)j * m] = acc;
  }
  tmk(5);
  for (long long t = tid; t < (long long)n * r; t += nt) {
    const int i = (int)(t % n), j = (int)(t / n);
    float acc = 0.f;
    for (int q = 0; q < rv; ++q) acc += SV[i + (long long)pivV[q] * n] * WV[q + j * K];
    Vd[i + (long long)j * n] = acc;
  }
  tmk(6);
  if (c.tprof && tid == 0) {
    atomicAdd(c.tprof + 8, 1ULL);
    atomicAdd(c.tprof + 9, (unsigned long long)K);
    atomicAdd(c.tprof + 10, (unsigned long long)(m + n));
  }
  if (tid == 0) c.rk[slot] = r;
  __syncthreads();
}

// Recompress U V^T given as Ut (m x K) and Vt (n x K) in the workspace into
// LR slot `slot`.  U = Q_U R_U, V = Q_V R_V (Householder), then a column-
// pivoted QR of the small core M = R_U R_V^T, M Pi = Q_M R_M, stopped at the
// first pivot below tol |R_M(0,0)| (or at kmax):
//   U V^T ~ (Q_U Q_M[:, :r]) (Q_V Pi R_M[:r, :]^T)^T.
template <class T>
__device__ void trunc_core(HCtx<T>& c, int slot, T* Ut, T* Vt, int K) {
  if constexpr (sizeof(T) == 4) {
    if (K <= 32) {
      trunc_gram(c, slot, Ut, Vt, K, false);
      return;
    }
  }
  const SlotDev s = c.sl[slot];
  const int m = s.m, n = s.n;
  T* tauU = c.sm;
  T* tauV = tauU + K;
  T* red = tauV + K;                 // 32
  T* M = red + 32;                   // ku x kv, ld K
  T* tauM = M + K * K;               // K
  T* cn = tauM + K;                  // K column norms^2
  T* Z = cn + K;                     // K x K work (ld K)
  int* piv = reinterpret_cast<int*>(Z + K * K);   // K
  // the rest of the shared memory stages the tall factors (16-byte aligned)
  const long long small = ((2LL * K + 32 + 2LL * K * K + 3LL * K + K + 8) + 3) & ~3LL;
  T* stage = c.sm + small;
  const long long cap = c.smcap - small;
  // Householder QR of the tall factors, in shared memory when they fit (the
  // reflector loops are latency bound), written back for the final products
  unsigned long long tq = 0;
  auto tmk = [&](int k) {
    if (!c.tprof || threadIdx.x != 0) return;
    unsigned long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (k >= 0) atomicAdd(c.tprof + k, t1 - tq);
    tq = t1;
  };
  tmk(-1);
  const int nwt = (int)(blockDim.x >> 5), nwh = nwt / 2;
  const int wid = (int)(threadIdx.x >> 5);
  // both factors and their outputs fit: the two halves of the CTA factor U
  // and V at the same time (named barriers 1 and 2) and keep the reflectors
  const bool both = (long long)(m + n) * K * 2 <= cap && nwh > 0;
  T* SU = stage;
  T* SV = stage + (long long)m * K;
  if (both) {
    for (long long t = threadIdx.x; t < (long long)m * K; t += blockDim.x) SU[t] = Ut[t];
    for (long long t = threadIdx.x; t < (long long)n * K; t += blockDim.x) SV[t] = Vt[t];
    __syncthreads();
    if (wid < nwh) house_qr(SU, m, K, tauU, 0, nwh, 1);
    else if (wid < 2 * nwh) house_qr(SV, n, K, tauV, nwh, nwh, 2);
    __syncthreads();
    tmk(0);
  } else {
    qr_staged(Ut, m, K, tauU, red, stage, cap);
    tmk(0);
    qr_staged(Vt, n, K, tauV, red, stage, cap);
  }
  tmk(1);
  const int ku = min(m, K), kv = min(n, K);
  // core M = R_U R_V^T from the two triangles, staged
  T* RU = Ut;
  T* RV = Vt;
  long long ldu = m, ldv = n;
  if (both) {
    RU = SU;
    RV = SV;
  } else if ((long long)2 * K * K <= cap) {
    RU = stage;
    RV = stage + (long long)K * K;
    for (int t = threadIdx.x; t < K * K; t += blockDim.x) {
      int i = t % K, l = t / K;
      RU[t] = (i < ku && i <= l) ? Ut[i + (long long)l * m] : (T)0;
      RV[t] = (i < kv && i <= l) ? Vt[i + (long long)l * n] : (T)0;
    }
    ldu = ldv = K;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < ku * kv; t += blockDim.x) {
    int i = t % ku, j = t / ku;
    T acc = 0;
    for (int l = max(i, j); l < K; ++l) acc += RU[i + l * ldu] * RV[j + l * ldv];
    M[i + j * K] = acc;
  }
  const int rmax = min(min(ku, kv), s.kmax);
  tmk(2);
  const int r = core_rrqr(M, K, ku, kv, rmax, c.tol, tauM, cn, piv, Z, [&]() { tmk(3); });
  T* Ud = c.ar + s.off;
  T* Vd = c.ar + s.off + (long long)m * s.kcap;
  // U_new = Q_U [Z; 0], V_new = Q_V [Pi R_M[:r,:]^T; 0] (row piv[j] of the
  // core factor is R_M[:, j]); built in shared memory when both fit
  T* YU = both ? SV + (long long)n * K : Ud;
  T* YV = both ? YU + (long long)m * r : Vd;
  for (int t = threadIdx.x; t < m * r; t += blockDim.x) {
    int i = t % m, j = t / m;
    YU[t] = (i < ku) ? Z[i + j * K] : (T)0;
  }
  for (int t = threadIdx.x; t < n * r; t += blockDim.x) YV[t] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < kv * r; t += blockDim.x) {
    int j = t % kv, i = t / kv;   // R_M[i][j], j >= i
    YV[piv[j] + (long long)i * n] = (j >= i) ? M[i + j * K] : (T)0;
  }
  __syncthreads();
  tmk(4);
  if (both) {
    if (wid < nwh) apply_q(SU, m, K, tauU, YU, m, r, 0, nwh, 1);
    else if (wid < 2 * nwh) apply_q(SV, n, K, tauV, YV, n, r, nwh, nwh, 2);
    __syncthreads();
    tmk(5);
    for (int t = threadIdx.x; t < m * r; t += blockDim.x) Ud[t] = YU[t];
    for (int t = threadIdx.x; t < n * r; t += blockDim.x) Vd[t] = YV[t];
    __syncthreads();
  } else {
    apply_q_staged(Ut, m, K, tauU, Ud, r, stage, cap);
    tmk(5);
    apply_q_staged(Vt, n, K, tauV, Vd, r, stage, cap);
  }
  tmk(6);
  if (c.tprof && threadIdx.x == 0) {
    atomicAdd(c.tprof + 8, 1ULL);
    atomicAdd(c.tprof + 9, (unsigned long long)K);
    atomicAdd(c.tprof + 10, (unsigned long long)(m + n));
  }
  if (threadIdx.x == 0) c.rk[slot] = r;
  __syncthreads();
}

template <class T>
// returns true when the append overflowed the capacity and recompressed
__device__ bool op_append(const HOp& o, HCtx<T>& c) {
  const int slot = o.slot;
  const SlotDev s = c.sl[slot];
  const int k = dimv(o.A.c, c.rk);
  const int r0 = c.rk[slot];
  __syncthreads();
  if (k <= 0) return false;
  const bool ident = o.B.off < 0;                 // V_p = columns of I from ioff
  const long long ioff = ident ? (-1 - o.B.off) : 0;
  const T alpha = (T)o.alpha;
  T* ar = c.ar;
  if (r0 + k <= s.kcap) {
    T* Ud = ar + s.off;
    T* Vd = ar + s.off + (long long)s.m * s.kcap;
    for (int t = threadIdx.x; t < s.m * k; t += blockDim.x) {
      int i = t % s.m, j = t / s.m;
      Ud[i + (long long)(r0 + j) * s.m] = alpha * ar[vidx(o.A, i, j)];
    }
    for (int t = threadIdx.x; t < s.n * k; t += blockDim.x) {
      int i = t % s.n, j = t / s.n;
      Vd[i + (long long)(r0 + j) * s.n] = ident ? (T)(i == ioff + j ? 1 : 0) : ar[vidx(o.B, i, j)];
    }
    __syncthreads();
    if (threadIdx.x == 0) c.rk[slot] = r0 + k;
    __syncthreads();
    return false;
  }
  const int K = r0 + k;
  T* Ut = c.ws;
  T* Vt = c.ws + (long long)s.m * K;
  const T* Us = ar + s.off;
  const T* Vs = ar + s.off + (long long)s.m * s.kcap;
  if constexpr (sizeof(T) == 4) {
    // the concatenated factors go straight into the Gram recompression's
    // shared memory (asynchronous copies), not through the workspace
    const long long small = gram_small(K);
    if (K <= 32 && (long long)(s.m + s.n) * K <= c.smcap - small) {
      float* su = c.sm + small;
      float* sv = su + (long long)s.m * K;
      const long long mr = (long long)s.m * r0, nr = (long long)s.n * r0;
      cp_async_range(su, Us, mr);
      for (int t = threadIdx.x; t < s.m * k; t += blockDim.x)
        cp_async_elem(su + mr + t, ar + vidx(o.A, t % s.m, t / s.m));
      cp_async_range(sv, Vs, nr);
      if (ident) {
        for (int t = threadIdx.x; t < s.n * k; t += blockDim.x) {
          const int i = t % s.n, j = t / s.n;
          sv[nr + t] = (i == ioff + j) ? 1.f : 0.f;
        }
      } else {
        for (int t = threadIdx.x; t < s.n * k; t += blockDim.x)
          cp_async_elem(sv + nr + t, ar + vidx(o.B, t % s.n, t / s.n));
      }
      cp_async_wait_all();
      __syncthreads();
      if (alpha != (T)1)
        for (int t = threadIdx.x; t < s.m * k; t += blockDim.x) su[mr + t] *= alpha;
      __syncthreads();
      trunc_gram(c, slot, nullptr, nullptr, K, true);
      return true;
    }
  }
  for (int t = threadIdx.x; t < s.m * K; t += blockDim.x) {
    int i = t % s.m, j = t / s.m;
    Ut[t] = (j < r0) ? Us[i + (long long)j * s.m] : alpha * ar[vidx(o.A, i, j - r0)];
  }
  for (int t = threadIdx.x; t < s.n * K; t += blockDim.x) {
    int i = t % s.n, j = t / s.n;
    Vt[t] = (j < r0) ? Vs[i + (long long)j * s.n]
                     : (ident ? (T)(i == ioff + j - r0 ? 1 : 0) : ar[vidx(o.B, i, j - r0)]);
  }
  __syncthreads();
  trunc_core(c, slot, Ut, Vt, K);
  return true;
}

template <class T>
__device__ void op_trunc(const HOp& o, HCtx<T>& c) {
  const int slot = o.slot;
  const SlotDev s = c.sl[slot];
  const int K = c.rk[slot];
  __syncthreads();
  if (K <= 0) return;
  T* Ut = c.ws;
  T* Vt = c.ws + (long long)s.m * K;
  const T* Us = c.ar + s.off;
  const T* Vs = c.ar + s.off + (long long)s.m * s.kcap;
  if constexpr (sizeof(T) == 4) {
    const long long small = gram_small(K);
    if (K <= 32 && (long long)(s.m + s.n) * K <= c.smcap - small) {
      float* su = c.sm + small;
      cp_async_range(su, Us, (long long)s.m * K);
      cp_async_range(su + (long long)s.m * K, Vs, (long long)s.n * K);
      cp_async_wait_all();
      __syncthreads();
      trunc_gram(c, slot, nullptr, nullptr, K, true);
      return;
    }
  }
  for (int t = threadIdx.x; t < s.m * K; t += blockDim.x) Ut[t] = Us[t];
  for (int t = threadIdx.x; t < s.n * K; t += blockDim.x) Vt[t] = Vs[t];
  __syncthreads();
  trunc_core(c, slot, Ut, Vt, K);
}

struct HProgArgs {
  const HInstDev* inst;
  const int* waves;  // op offsets of the waves
  const HOp* ops;
  const SlotDev* slots;
  int* ranks;
  int* err;
  double tol;
  unsigned long long* prof;   // optional: per instance, 16 op types x (cycles, count)
  double* flops;              // per instance: algorithmic flops of the executed ops
  unsigned long long* wprof;  // optional: per instance and wave, wall ns then per CTA
                              // (busy ns, longest op ns, longest op index)
  int wstride;                // waves per instance in wprof
  long long smem_elems;       // dynamic shared memory, in elements of the factor type
  int n_inst_prof;            // instances in prof (the recompression phases follow them)
  int tc;                     // dense leaf contractions on the tensor cores
  unsigned long long* tcdbg;  // 8 words of diagnostics for a tensor-core wait that ran out
  int ncl;                    // CTAs per instance (the cluster size of the launch)
  int leaf32;                 // FP64 factor: leaf LUs in FP32 arithmetic
};

// algorithmic flops of one op with its run-time shapes
// (integer arithmetic: the thread that counts also claims the next op, and
// FP64 instructions are slow on this GPU's FP64 pipe)
__device__ unsigned long long op_flops(const HOp& o, const int* rk, const SlotDev* sl) {
  using u64 = unsigned long long;
  switch (o.type) {
    case OP_GEMM: {
      const u64 m = dimv(o.C.r, rk), n = dimv(o.C.c, rk), k = dimv(o.A.c, rk);
      return 2ull * m * n * k;
    }
    case OP_GETRF_INV: {   // LU and the two triangular inverses: 4/3 n^3
      const u64 n = o.C.r;
      return 4ull * n * n * n / 3ull;
    }
    case OP_TRMM_L: {
      const u64 n = dimv(o.C.r, rk), c = dimv(o.C.c, rk);
      return 2ull * n * n * c;
    }
    case OP_TRMM_R: {
      const u64 m = dimv(o.C.r, rk), n = dimv(o.C.c, rk);
      return 2ull * m * n * n;
    }
    case OP_TRUNC: {
      const u64 K = rk[o.slot], m = sl[o.slot].m, n = sl[o.slot].n;
      return 4ull * (m + n) * K * K + 2ull * K * K * K;
    }
    default:
      return 0ull;
  }
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
// hardware barrier of all threads of the cluster; release/acquire at cluster
// scope makes every global write before it visible to every CTA after it
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One thread-block cluster of a.ncl CTAs (8, or 16 for a few large
// instances) per instance runs the instance's H-LU program wave by wave: the ops of a wave are independent; a CTA that
// becomes free takes the next op of the wave from a counter in the shared
// memory of CTA 0 (distributed shared memory atomics; the planner orders a
// wave's ops longest first), and a cluster barrier separates consecutive
// waves.
template <class T>
__global__ void __launch_bounds__(kHThreads) k_hprog(HProgArgs a, T* har) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const unsigned crank = cluster_rank();
  const unsigned cid = cluster_id();
  const HInstDev H = a.inst[cid];
  HCtx<T> c;
  c.ar = har + H.arena;
  c.rk = a.ranks + H.rk0;
  c.sl = a.slots + H.slot0;
  c.ws = c.ar + H.ws_off + (long long)crank * H.ws_size;
  c.sm = reinterpret_cast<T*>(smraw);
  c.smcap = a.smem_elems;
  c.tprof = a.prof ? a.prof + (size_t)a.n_inst_prof * 32 : nullptr;
  c.tol = a.tol;
  c.err = a.err + cid;
  c.leaf32 = a.leaf32;
  // tensor memory (256 columns of FP32 accumulators) and the MMA mbarrier
  __shared__ unsigned s_tmem;
  __shared__ __align__(8) unsigned long long s_tcbar;
  unsigned tcphase = 0;
  c.tc = a.tc;
  c.tmem = 0;
  c.tcbar = &s_tcbar;
  c.tcphase = &tcphase;
  c.tcdbg = a.tcdbg;
  if (a.tc) {
    if ((threadIdx.x >> 5) == 0) tc_alloc(&s_tmem, 256);
    if (threadIdx.x == 0) {
      mbar_init(&s_tcbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    c.tmem = s_tmem;
  }
  const HOp* ops = a.ops + H.ops0;
  const int* waves = a.waves + H.fw0;
  const int nw = H.nfw;
  // per-wave op counters (two, alternating), used in CTA 0
  __shared__ unsigned s_ctr[2];
  __shared__ int s_next[2];   // claimed op index, double-buffered by op parity
  if (threadIdx.x == 0) s_ctr[0] = s_ctr[1] = 0u;
  const unsigned ctr_base = smem_u32(&s_ctr[0]);
  unsigned ctr0;   // the counters of CTA 0 in the cluster's shared window
  asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(ctr0) : "r"(ctr_base));
  cluster_barrier();
  unsigned long long fl = 0ull;
  const bool wp = a.wprof && threadIdx.x == 0;
  for (int w = 0; w < nw; ++w) {
    const int i0 = waves[w], n_w = waves[w + 1] - i0;
    // the other counter is idle (every CTA passed the barrier after wave
    // w - 1): reset it for wave w + 1
    if (crank == 0 && threadIdx.x == 0) s_ctr[(w + 1) & 1] = 0u;
    unsigned long long tw0 = 0, busy = 0, lmax = 0, ltype = 0;
    if (wp) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tw0));
    // thread 0 claims ops from CTA 0's counter; the first of the wave here,
    // each later one just before the barrier that closes the previous op,
    // into the other index slot: one barrier per op, and no thread can see
    // the index of the op it is executing change
    const unsigned ctr_w = ctr0 + 4u * (unsigned)(w & 1);
    int par = 0;
    if (threadIdx.x == 0) {
      unsigned k;
      asm volatile("atom.shared::cluster.add.u32 %0, [%1], 1;" : "=r"(k) : "r"(ctr_w) : "memory");
      s_next[0] = (int)k;
    }
    __syncthreads();
    for (;; par ^= 1) {
      const int kk = s_next[par];
      if (kk >= n_w) break;
      const int i = i0 + kk;
      const HOp o = ops[i];
      if (threadIdx.x == 0) fl += op_flops(o, c.rk, c.sl);
      unsigned long long t0 = 0;
      if ((a.prof && threadIdx.x == 0) || wp) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      int ptype = o.type;
      switch (o.type) {
        case OP_GEMM: op_gemm(o, c); break;
        case OP_GETRF_INV: op_getrf_inv(o, c); break;
        case OP_TRMM_L: op_trmm_l(o, c); break;
        case OP_TRMM_R: op_trmm_r(o, c); break;
        case OP_APPEND:
          if (op_append(o, c)) ptype = 9;   // the append recompressed (profile bucket)
          break;
        case OP_TRUNC: op_trunc(o, c); break;
        case OP_ZERO: {
          int m = dimv(o.C.r, c.rk), n = dimv(o.C.c, c.rk);
          for (int t = threadIdx.x; t < m * n; t += blockDim.x) c.ar[vidx(o.C, t % m, t / m)] = 0;
          break;
        }
        case OP_AXPY: {
          int m = dimv(o.C.r, c.rk), n = dimv(o.C.c, c.rk);
          for (int t = threadIdx.x; t < m * n; t += blockDim.x) {
            int ii = t % m, j = t / m;
            c.ar[vidx(o.C, ii, j)] += (T)o.alpha * c.ar[vidx(o.A, ii, j)];
          }
          break;
        }
        default: break;
      }
      if (threadIdx.x == 0) {
        unsigned k;
        asm volatile("atom.shared::cluster.add.u32 %0, [%1], 1;" : "=r"(k) : "r"(ctr_w) : "memory");
        s_next[par ^ 1] = (int)k;
      }
      __syncthreads();
      if (a.prof && threadIdx.x == 0) {   // all CTAs of the instance, summed
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        unsigned long long* pr = a.prof + (size_t)cid * 32 + 2 * (ptype & 15);
        atomicAdd(pr, t1 - t0);
        atomicAdd(pr + 1, 1ULL);
        if (o.type == OP_GEMM) {   // GEMM time by shape class (m, n, k: <=8, <=64, >64)
          auto cls = [](int d) { return d <= 8 ? 0 : (d <= 64 ? 1 : 2); };
          const int key = cls(dimv(o.C.r, c.rk)) * 9 + cls(dimv(o.C.c, c.rk)) * 3 + cls(dimv(o.A.c, c.rk));
          unsigned long long* g = a.prof + (size_t)a.n_inst_prof * 32 + 16 + 2 * key;
          atomicAdd(g, t1 - t0);
          atomicAdd(g + 1, 1ULL);
        }
      }
      if (wp) {
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        busy += t1 - t0;
        if (t1 - t0 > lmax) {
          lmax = t1 - t0;
          ltype = (unsigned long long)i;
        }
      }
    }
    cluster_barrier();
    if (wp) {
      unsigned long long t1;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
      unsigned long long* q = a.wprof + ((size_t)cid * a.wstride + w) * (1 + 3 * a.ncl);
      if (crank == 0) q[0] = t1 - tw0;
      q[1 + 3 * crank] = busy;
      q[2 + 3 * crank] = lmax;
      q[3 + 3 * crank] = ltype;
    }
  }
  if (threadIdx.x == 0) a.flops[((size_t)cid * a.ncl + crank) * 2] += (double)fl;
  if (a.tc) {   // every tensor-core op has completed and been read back
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tc_dealloc(c.tmem, 256);
  }
}

// Check of the BF16 tensor-core tile on its own: one cluster of kCluster CTAs,
// each set up as the factorisation sets itself up (tensor memory, MMA
// barrier, context), computes C_r = A B reps times on one barrier; CTA r
// writes its own C_r.  err[r] = 4 when a wait ran out.
__global__ void __launch_bounds__(kHThreads) k_tc_tile_check(float* ar, int N, int K, int reps, int* err,
                                                              unsigned long long* dbg) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ unsigned s_tmem;
  __shared__ __align__(8) unsigned long long s_tcbar;
  const unsigned crank = cluster_rank();
  HCtx<float> c;
  c.ar = ar;
  c.rk = nullptr;
  c.sl = nullptr;
  c.ws = nullptr;
  c.sm = reinterpret_cast<float*>(smraw);
  c.smcap = 0;
  c.tprof = nullptr;
  c.tol = 0.0;
  c.err = err + crank;
  c.leaf32 = 0;
  unsigned tcphase = 0;
  c.tc = 1;
  c.tcbar = &s_tcbar;
  c.tcphase = &tcphase;
  c.tcdbg = dbg;
  if ((threadIdx.x >> 5) == 0) tc_alloc(&s_tmem, 256);
  if (threadIdx.x == 0) {
    mbar_init(&s_tcbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tmem = s_tmem;
  const View A{0, 128, K, 128, 0};
  const View B{128LL * K, K, N, K, 0};
  const View C{128LL * K + (long long)K * N + (long long)crank * 128 * N, 128, N, 128, 0};
  for (int r = 0; r < reps && c.tc; ++r) tc_gemm128(c, A, B, C, 0, N, K, 1.f, 0.f);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tc_dealloc(c.tmem, 256);
}

// --- asynchronous bulk copies and distributed shared memory (inline PTX) ---
// global -> this CTA's shared memory, completion counted on bar (bytes)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ float ld_dsmem(const float* p, unsigned rank) {
  unsigned a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ double ld_dsmem(const double* p, unsigned rank) {
  unsigned a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}

// The solve pack: after the factorisation, every job's column segment is
// copied to its own slot of slot_elems entries (16-byte aligned) in job
// order, and its fields to a 16-byte record {x, active | kind << 9 | ldw <<
// 12} (a low-rank column is active below its block's current rank; the
// slot of an inactive one is zeroed).  The jobs of one CTA in one step are
// contiguous, so a step reaches shared memory in two bulk copies.
template <class T>
__global__ void k_solve_pack(const HInstDev* __restrict__ hi, const SolJob* __restrict__ jobs,
                             const T* har, const int* __restrict__ ranks, T* pack, int4* meta,
                             int slot_elems, int* err) {
  const HInstDev H = hi[blockIdx.y];
  const T* ar = har + H.arena;
  const int* rk = ranks + H.rk0;
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long j = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); j < H.njob;
       j += nw) {
    const SolJob J = jobs[H.job0 + j];
    const int act = (J.slot < 0 || J.l < rk[J.slot]) ? 1 : 0;
    // a rank above the columns the solve reads would lose part of the block
    if (lane == 0 && J.slot >= 0 && rk[J.slot] > J.lmax) atomicExch(err + blockIdx.y, 3);
    if (lane == 0)
      meta[H.pk0 + j] = make_int4(J.x, (act << 8) | ((int)J.kind << 9) | (J.ldw << 12), 0, 0);
    T* dst = pack + (H.pk0 + j) * slot_elems;
    for (int i = lane; i < J.n; i += 32) dst[i] = act ? ar[J.src + i] : (T)0;
  }
}

// one thread issues the two bulk copies of the jobs [a, a + nj)
template <class T>
__device__ __forceinline__ void solve_prefetch(int a, int nj, long long pk0, const T* pack,
                                               const int4* meta, int slot_elems, T* buf,
                                               int4* mbuf, unsigned long long* bar) {
  const unsigned bd = (unsigned)((long long)nj * slot_elems * sizeof(T));
  const unsigned bm = (unsigned)(nj * sizeof(int4));
  mbar_expect_tx(bar, bd + bm);
  if (nj > 0) {
    bulk_g2s(buf, pack + (pk0 + a) * slot_elems, bd, bar);
    bulk_g2s(mbuf, meta + pk0 + a, bm, bar);
  }
}

// Both triangular solves of an instance by its cluster of kCluster CTAs,
// one leaf step after another.  A CTA's jobs of a step reach shared memory in
// parts of jcap jobs (bulk copies, two buffers: the next part streams in
// while the current one is used).  Each CTA owns a fixed share of the
// low-rank columns and keeps their w in its own shared memory, every CTA
// keeps the solutions of the last kRing leaves, and the partial sums of the
// gathers and of the inverse product meet through distributed shared memory:
// two cluster barriers per step.  The right-hand sides go in chunks of
// solve_w<T>() columns; nsplit clusters share an instance, each taking a
// contiguous range of its chunks (they read the same factor and write
// disjoint columns of the right-hand-side area).
template <class T>
__global__ void __launch_bounds__(kHThreads) k_hsolve_cl(const HInstDev* __restrict__ hi,
                                                        const StepInfo* __restrict__ sinfo,
                                                        const StepCta* __restrict__ scta,
                                                        const T* __restrict__ pack,
                                                        const int4* __restrict__ meta, T* har,
                                                        int nrhs, int jmax, int slot_elems,
                                                        int wcols, int* err, double* flops,
                                                        unsigned long long* sprof,
                                                        const int* __restrict__ gate, int nsplit) {
  extern __shared__ __align__(16) unsigned char smraw[];
  HF_GATE(gate);   // every CTA of the cluster returns, before any barrier
  constexpr int kSolveW = solve_w<T>();
  constexpr int V = 128 * kSolveW;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smraw);   // [2]
  T* colb = reinterpret_cast<T*>(smraw + 16);                              // [2][jmax][slot]
  T* pr = colb + 2LL * jmax * slot_elems;   // [V] gather partial (read remotely)
  T* px = pr + V;                           // [V] inverse partial (read remotely)
  T* tmp = px + V;                          // [V] half sums
  T* r = tmp + V;                           // [V] leaf right-hand side
  T* bb = r + V;                            // [V] b of the leaf
  T* xs = bb + V;                           // [V] x of the leaf
  T* ring = xs + V;                         // [kRing][V] x of the last leaves
  T* wl = ring + kRing * V;                 // [wcols][W] w of this CTA's columns
  T* sx = wl + (long long)wcols * kSolveW;  // [jmax][W] scalars of the gathers
  int4* mbb = reinterpret_cast<int4*>(sx + (long long)jmax * kSolveW);   // [2][jmax]
  const unsigned crank = cluster_rank();
  const unsigned cid = cluster_id();
  const unsigned inst = cid / (unsigned)nsplit, part = cid % (unsigned)nsplit;
  const HInstDev H = hi[inst];
  T* ar = har + H.arena;
  const StepInfo* si = sinfo + H.st0;
  const StepCta* sc = scta + H.st0 * kCluster;
  const int jcap = H.jcap;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long ld = H.nd;
  const int nst = H.nst;
  const int nchunk = (nrhs + kSolveW - 1) / kSolveW;
  const int ch0 = (int)(part * nchunk / nsplit), ch1 = (int)((part + 1) * nchunk / nsplit);
  const int total = nst * (ch1 - ch0);
  unsigned long long fl = 0ull;   // integer: FP64 instructions are slow here
  bool ok = true;
  long long qfail = -1;   // part whose copy did not arrive in time
  // optional phase timer (cluster 0, CTA 0): waits, A, barrier, B, barrier, C
  const bool tp = sprof && cid == 0 && crank == 0 && tid == 0;
  unsigned long long tq = 0;
  auto tmark = [&](int k) {
    if (!tp) return;
    unsigned long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (k >= 0) sprof[k] += t1 - tq;
    tq = t1;
  };
  auto nparts = [&](const StepCta& C) { return max(1, (C.a3 - C.a0 + jcap - 1) / jcap); };
  auto prefetch = [&](const StepCta& C, int k, int b) {
    const int a = C.a0 + k * jcap;
    const int nj = max(0, min(C.a3 - a, jcap));
    solve_prefetch(a, nj, H.pk0, pack, meta, slot_elems, colb + (long long)b * jmax * slot_elems,
                   mbb + b * jmax, &bar[b]);
  };
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && total > 0) prefetch(sc[crank], 0, 0);
  // parts are begun in the order (step, k); qn counts them; the part begun
  // last is resident in buffer cb
  long long qn = 0;
  int ck = -1, cb = 0;
  auto begin = [&](int g, const StepCta& C, int k) {
    __syncthreads();   // the buffer about to be refilled is no longer read
    const int b = (int)(qn & 1);
    if (ok) {
      long long spins = 0;
      while (!mbar_try_wait(&bar[b], (unsigned)((qn >> 1) & 1))) {
        if (++spins > (1LL << 24)) {
          ok = false;
          qfail = qn;
          break;
        }
      }
    }
    if (tid == 0 && ok) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (k + 1 < nparts(C)) prefetch(C, k + 1, b ^ 1);
      else if (g + 1 < total) prefetch(sc[(long long)((g + 1) % nst) * kCluster + crank], 0, b ^ 1);
    }
    ck = k;
    cb = b;
    ++qn;
  };
  for (int g = 0; g < total; ++g) {
    const int s = g % nst, c0 = (ch0 + g / nst) * kSolveW;
    const int nc = min(kSolveW, nrhs - c0);
    T* b = ar + H.rhs_off + (long long)c0 * ld;
    if (s == 0) {   // a new chunk of right-hand sides: clear this CTA's w
      __syncthreads();
      for (int t = tid; t < wcols * kSolveW; t += blockDim.x) wl[t] = (T)0;
    }
    tmark(-1);
    const StepInfo S = si[s];
    const StepCta C = sc[(long long)s * kCluster + crank];
    const int n = S.n;
    const int i = tid & 127, h = tid >> 7;
    // b of the leaf (read now, used after the first barrier)
    for (int t = tid; t < n * nc; t += blockDim.x) {
      const int ii = t % n, c = t / n;
      bb[c * 128 + ii] = b[S.d0 + ii + c * ld];
    }
    begin(g, C, 0);
    tmark(0);
    // A: gathers, summed over this CTA's columns
    T acc[kSolveW];
#pragma unroll
    for (int c = 0; c < kSolveW; ++c) acc[c] = (T)0;
    for (int x = C.a0; x < C.a1;) {
      const int k = (x - C.a0) / jcap;
      if (k != ck) begin(g, C, k);
      const int pa = C.a0 + k * jcap, e = min(C.a1, pa + jcap);
      const T* buf = colb + (long long)cb * jmax * slot_elems;
      const int4* mb = mbb + cb * jmax;
      for (int t = tid; t < (e - x) * kSolveW; t += blockDim.x) {
        const int jl = x - pa + t / kSolveW, c = t % kSolveW;
        const int4 m = mb[jl];
        const int f = m.y, kind = (f >> 9) & 7;
        T v = (T)0;
        if (c < nc && ((f >> 8) & 1)) {
          if (kind == 0) v = ring[(m.x >> 7) * V + (m.x & 127) + c * 128];
          else if (kind == 4) v = b[m.x + c * ld];
          else v = wl[m.x * kSolveW + c];
        }
        sx[t] = v;
      }
      __syncthreads();
      if (i < n)
        for (int jl = h; jl < e - x; jl += 2) {
          const T a = buf[(long long)(x - pa + jl) * slot_elems + i];
#pragma unroll
          for (int c = 0; c < kSolveW; ++c) acc[c] += a * sx[jl * kSolveW + c];
        }
      if (tid == 0) fl += 2ull * (unsigned long long)n * nc * (e - x);
      __syncthreads();
      x = e;
    }
    if (h == 1)
#pragma unroll
      for (int c = 0; c < kSolveW; ++c) tmp[c * 128 + i] = acc[c];
    __syncthreads();
    if (h == 0)
#pragma unroll
      for (int c = 0; c < kSolveW; ++c) pr[c * 128 + i] = acc[c] + tmp[c * 128 + i];
    tmark(1);
    cluster_barrier();
    tmark(2);
    // B: r = b - sum of the partials; partial product of the inverse columns
    for (int t = tid; t < n * nc; t += blockDim.x) {
      const int ii = t % n, c = t / n;
      T v = bb[c * 128 + ii];
      for (unsigned qq = 0; qq < kCluster; ++qq) v -= ld_dsmem(&pr[c * 128 + ii], qq);
      r[c * 128 + ii] = v;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kSolveW; ++c) acc[c] = (T)0;
    for (int x = C.a1; x < C.a2;) {
      const int k = (x - C.a0) / jcap;
      if (k != ck) begin(g, C, k);
      const int pa = C.a0 + k * jcap, e = min(C.a2, pa + jcap);
      const T* buf = colb + (long long)cb * jmax * slot_elems;
      const int4* mb = mbb + cb * jmax;
      if (i < n)
        for (int jl = x - pa + h; jl < e - pa; jl += 2) {
          const T a = buf[(long long)jl * slot_elems + i];
          const int kk = mb[jl].x;
#pragma unroll
          for (int c = 0; c < kSolveW; ++c) acc[c] += a * r[c * 128 + kk];
        }
      if (tid == 0) fl += 2ull * (unsigned long long)n * nc * (e - x);
      x = e;
    }
    if (h == 1)
#pragma unroll
      for (int c = 0; c < kSolveW; ++c) tmp[c * 128 + i] = acc[c];
    __syncthreads();
    if (h == 0)
#pragma unroll
      for (int c = 0; c < kSolveW; ++c) px[c * 128 + i] = acc[c] + tmp[c * 128 + i];
    tmark(3);
    cluster_barrier();
    tmark(4);
    // C: x = sum of the partials (every CTA); w += V^T x over this CTA's columns
    T* rg = ring + (long long)S.ring * V;
    for (int t = tid; t < n * nc; t += blockDim.x) {
      const int ii = t % n, c = t / n;
      T v = (T)0;
      for (unsigned qq = 0; qq < kCluster; ++qq) v += ld_dsmem(&px[c * 128 + ii], qq);
      xs[c * 128 + ii] = v;
      rg[c * 128 + ii] = v;
      if (crank == 0) b[S.d0 + ii + c * ld] = v;
    }
    __syncthreads();
    for (int x = C.a2; x < C.a3;) {
      const int k = (x - C.a0) / jcap;
      if (k != ck) begin(g, C, k);
      const int pa = C.a0 + k * jcap, e = min(C.a3, pa + jcap);
      const T* buf = colb + (long long)cb * jmax * slot_elems;
      const int4* mb = mbb + cb * jmax;
      for (int jl = x - pa + warp; jl < e - pa; jl += (int)(blockDim.x >> 5)) {
        const int4 m = mb[jl];
        if (!((m.y >> 8) & 1)) continue;
        const T* col = buf + (long long)jl * slot_elems;
        T pa_[kSolveW];
#pragma unroll
        for (int c = 0; c < kSolveW; ++c) pa_[c] = (T)0;
        for (int ii = lane; ii < n; ii += 32) {
          const T a = col[ii];
#pragma unroll
          for (int c = 0; c < kSolveW; ++c) pa_[c] += a * xs[c * 128 + ii];
        }
#pragma unroll
        for (int c = 0; c < kSolveW; ++c)
          if (c < nc)
            for (int o = 16; o > 0; o >>= 1) pa_[c] += __shfl_xor_sync(0xffffffffu, pa_[c], o);
        if (lane == 0)
          for (int c = 0; c < nc; ++c) wl[m.x * kSolveW + c] += pa_[c];
      }
      if (tid == 0) fl += 2ull * (unsigned long long)n * nc * (e - x);
      x = e;
    }
    // every part of the step is begun (keeps the prefetch chain in order)
    for (int k = ck + 1; k < nparts(C); ++k) begin(g, C, k);
    tmark(5);
  }
  // no CTA may leave while another can still read its shared memory
  cluster_barrier();
  if (!ok) {
    // a copy never arrived: flag it and give the copies in flight a bounded
    // time to land before the shared memory is released
    if (tid == 0) atomicExch(err + inst, 2);
    if (qfail >= 0) {
      long long spins = 0;
      while (!mbar_try_wait(&bar[qfail & 1], (unsigned)((qfail >> 1) & 1)) && ++spins < (1LL << 20)) {
      }
    }
  }
  if (tid == 0) atomicAdd(&flops[((size_t)inst * kCluster + crank) * 2 + 1], (double)fl);
}

// rhs area <- D r (element-major FP64 -> T); rank slot n_slots <- nrhs
template <class T>
__global__ void k_hsolve_in(const HInstDev* __restrict__ hi, const InstDev* __restrict__ inst,
                            const double* __restrict__ r, const double* D, T* har, int* ranks,
                            int nrhs, const int* __restrict__ gate) {
  HF_GATE(gate);
  const HInstDev H = hi[blockIdx.y];
  const InstDev I = inst[H.sys_inst];
  T* rhs = har + H.arena + H.rhs_off;
  const double* rv = r + I.o_vec * nrhs;
  const long long n = (long long)I.Nd * nrhs;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    rhs[t] = (T)(D[H.d_off + t % I.Nd] * rv[t]);
  if (blockIdx.x == 0 && threadIdx.x == 0) ranks[H.rk0 + H.n_slots] = nrhs;
}

template <class T>
__global__ void k_hsolve_out(const HInstDev* __restrict__ hi, const InstDev* __restrict__ inst,
                             const double* D, const T* har, double* y, int nrhs,
                             const int* __restrict__ gate) {
  HF_GATE(gate);
  const HInstDev H = hi[blockIdx.y];
  const InstDev I = inst[H.sys_inst];
  const T* rhs = har + H.arena + H.rhs_off;
  double* yv = y + I.o_vec * nrhs;
  const long long n = (long long)I.Nd * nrhs;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    yv[t] = D[H.d_off + t % I.Nd] * (double)rhs[t];
}

// Dense expansion of the (unfactored) H-matrix, unscaled, element-major.
template <class T>
__global__ void k_expand(const HInstDev* __restrict__ hi, const DenseDev* dens,
                         const LRPairDev* pairs, const SlotDev* slots, const int* ranks,
                         const double* D, const T* har, double* out, int Nd) {
  const HInstDev H = hi[0];
  const T* ar = har + H.arena;
  const double* Dv = D + H.d_off;
  const int nb = H.ndense + 2 * H.npairs;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    if (b < H.ndense) {
      DenseDev d = dens[H.dense0 + b];
      for (int t = threadIdx.x; t < d.m * d.n; t += blockDim.x) {
        int i = t % d.m, j = t / d.m;
        int r = d.d0r + i, c = d.d0c + j;
        out[r + (long long)c * Nd] = (double)ar[d.off + t] / (Dv[r] * Dv[c]);
      }
    } else {
      int pi = (b - H.ndense) / 2, up = (b - H.ndense) % 2;
      LRPairDev pr = pairs[H.pair0 + pi];
      int slot = up ? pr.upper_slot : pr.lower_slot;
      SlotDev s = slots[H.slot0 + slot];
      int k = ranks[H.rk0 + slot];
      int rr0 = up ? pr.sd0 : pr.td0, cc0 = up ? pr.td0 : pr.sd0;
      for (int t = threadIdx.x; t < s.m * s.n; t += blockDim.x) {
        int i = t % s.m, j = t / s.m;
        double acc = 0.0;
        for (int l = 0; l < k; ++l)
          acc += (double)ar[s.off + i + (long long)l * s.m] *
                 (double)ar[s.off + (long long)s.m * s.kcap + j + (long long)l * s.n];
        int r = rr0 + i, c = cc0 + j;
        out[r + (long long)c * Nd] = acc / (Dv[r] * Dv[c]);
      }
    }
  }
}

__global__ void k_perm_mat(const double* in, double* out, int Nd, int N, int P) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)Nd * Nd;
       t += (long long)gridDim.x * blockDim.x) {
    int r = (int)(t % Nd), c = (int)(t / Nd);
    auto pidx = [&](int i) {
      int e = i / P, p = i % P + 1;
      return (p < P) ? e * (P - 1) + p - 1 : N * (P - 1) + e;
    };
    out[pidx(r) + (long long)pidx(c) * Nd] = in[t];
  }
}

// ---------------------------------------------------------------------------
// host: factor object
// ---------------------------------------------------------------------------
struct PlanBundle {
  HPlan plan;
  std::vector<DenseDev> dense;
  std::vector<LRPairDev> pairs;
  std::vector<int> ptask;        // low-rank build tasks per pair (prefix sums)
  long long lrrows = 0;          // entries of the FP64 row buffer of the low-rank build
  std::vector<SlotDev> slots;
  LeafSolve ls;                  // tables of the leaf solves
};


}  // namespace hf

namespace hf {
// Product tables of the H-matrix operator (kHmat instances), see hop_apply.
struct HopRow {        // one leaf row cluster of one instance
  int inst;            // factor instance
  int d0, nr;          // its unknowns [d0, d0 + nr) (instance-local)
  int it0, it1;        // its items
};
struct HopItem {       // one block whose rows contain the leaf
  long long off;       // element offset of the block in the factor arena
  int kind;            // 0 dense (m x n, column-major), 1 low-rank (U: m x kcap)
  int ld;              // rows of the block
  int roff;            // the leaf's first row inside the block
  int c0;              // dense: first column (instance-local); low-rank: slot record
  int nc;              // dense: columns
};
struct HopSlot {       // one low-rank block: w = V^T x~ over its columns
  long long offV;      // element offset of V (n x kcap, column-major)
  long long w0;        // offset of its w in the projection buffer
  int inst, c0, n, kcap, rk;   // factor instance, first column, columns, capacity, rank index
};
}  // namespace hf

struct hfsem_factor_s : public hf::Precond {
  hfsem_system* sys = nullptr;
  cudaStream_t st = nullptr;   // copy of the system's stream (free never touches sys)
  int precision = HFSEM_PREC_MIXED;
  // the system instances this factor covers, in its own order (factor
  // instance j is system instance insts[j]); the kernels index instances
  // by factor instance and reach the system's data through sys_inst
  std::vector<int> insts;
  int nfi = 0;
  // a batch whose meshes need different arithmetic is factored in parts
  // (FP32 and FP64); the object holding them owns no device data itself
  std::vector<std::unique_ptr<hfsem_factor_s>> parts;
  int build_only = 0;
  double tol = 1e-3;
  int R = 8;
  size_t tsize = 4;
  std::vector<std::shared_ptr<hf::PlanBundle>> plans;   // per instance (shared)
  std::vector<hf::HInstDev> hidev;
  hf::DevBuf<hf::HInstDev> d_hi;
  hf::DevBuf<int> d_waves;
  hf::DevBuf<hf::HOp> d_ops;
  hf::DevBuf<hf::SlotDev> d_slots;
  hf::DevBuf<hf::DenseDev> d_dense;
  hf::DevBuf<hf::LRPairDev> d_pairs;
  hf::DevBuf<int> d_ptask;                  // low-rank build tasks
  hf::DevBuf<unsigned long long> d_gmax;    // low-rank build: per pair and term, the largest entries
  hf::DevBuf<double> d_lrt;                 // low-rank build: factor rows before balancing (FP64)
  hf::DevBuf<hf::StepInfo> d_steps;   // leaf solve tables
  hf::DevBuf<hf::StepCta> d_step_cta;
  hf::DevBuf<hf::SolJob> d_jobs;
  hf::DevBuf<unsigned char> d_pack;    // solve pack: column segments in job order
  hf::DevBuf<int4> d_meta;             // and the jobs' records
  int sol_jmax = 1, sol_slot = 1, sol_wcols = 1;
  hf::DevBuf<unsigned long long> d_sprof;   // HFSEM_PROFILE=2: leaf-solve phase times
  size_t sol_smem = 0;
  void run_leaf_solve(int nrhs);
  void run_pack();
  hf::DevBuf<int> d_ranks, d_err;
  hf::DevBuf<double> d_D;
  hf::DevBuf<unsigned char> d_arena;
  size_t smem = 0;
  long long total_ops = 0;
  hf::DevBuf<unsigned long long> d_prof;   // HFSEM_PROFILE=1: time per op type
  hf::DevBuf<double> d_flops;               // per instance: factor / solve flops
  hf::DevBuf<unsigned long long> d_wprof;   // HFSEM_PROFILE=2: per-wave records
  hf::DevBuf<unsigned long long> d_tcdbg;   // tensor-core wait diagnostics (8 words)
  // operator use (build_only factors of kHmat instances): product tables
  hf::DevBuf<hf::HopRow> d_hrow;
  hf::DevBuf<hf::HopItem> d_hitem;
  hf::DevBuf<hf::HopSlot> d_hslot;
  int hop_nrows = 0, hop_nslots = 0, hop_kmax = 1;
  long long hop_wsize = 0;        // projection entries per right-hand side
  double hop_flops = 0.0;         // per right-hand side
  int wstride = 0;
  int ncl = hf::kCluster;   // CTAs per instance in the H-LU program (plans hold ncl workspaces)
  int leaf32 = 0;           // FP64 part of a mixed factor: leaf LUs in FP32 arithmetic
  void report(const char* what);
  void report_waves(const char* what);
  void apply(int nrhs, const double* r_em, double* y_em) override;
  int device_status() override;
  void collect_flops();
  void run_prog();
};

namespace hf {

// Whether the device can hold one cluster of ncl CTAs of the H-LU program
// (cluster sizes above 8 are non-portable and must be allowed on the kernel
// first); decided once per device and kernel.
static bool wide_clusters_fit(const void* fn, size_t smem, int ncl) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, bool> ok;
  int dev = 0;
  HF_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_pair(dev, fn);
  auto it = ok.find(key);
  if (it != ok.end()) return it->second;
  bool fit = false;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ncl);
    cfg.blockDim = dim3(kHThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ncl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    fit = cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) == cudaSuccess && nc >= 1;
  }
  cudaGetLastError();   // a refused query leaves no error behind
  ok[key] = fit;
  return fit;
}

template <class T>
static void set_prog_smem(size_t bytes) {
  allow_dyn_smem((const void*)k_hprog<T>, bytes);
}

static size_t prog_smem(const HPlan& p, size_t ts) {
  size_t leaf = (size_t)2 * p.leaf_max * p.leaf_max;
  size_t K = (size_t)std::max(p.kconcat_max, 1);
  size_t trunc = 2 * K + 32 + 2 * K * K + 3 * K + 8;
  size_t trmm = (size_t)p.leaf_max * (p.leaf_max + 1) + 4 + (size_t)std::max(p.leaf_max, 1) * 33;
  size_t gemm = 2 * 8 * 128 + 128 * 129;   // tiled GEMM: k chunks and the C tile
  return std::max(std::max(leaf, trunc), std::max(trmm, gemm)) * ts + 64;
}

// Plans depend on the mesh and the options only, so they are kept across
// factorisations (least recently used first out, bounded in count and in
// host bytes): refactoring the same meshes with new alpha, theta or rho, or
// the same batch again, skips the host planning.
constexpr size_t kPlanCacheMax = 4096;
constexpr size_t kPlanCacheBytes = size_t(4) << 30;
static std::mutex g_plan_mu;
static std::list<std::pair<std::string, std::shared_ptr<PlanBundle>>> g_plan_lru;
static std::unordered_map<std::string, decltype(g_plan_lru)::iterator> g_plan_idx;
static size_t g_plan_bytes = 0;

static size_t plan_bytes(const PlanBundle& pb) {
  const HPlan& p = pb.plan;
  return p.fac.size() * sizeof(HOp) + p.fac_waves.size() * sizeof(int) + p.B.size() * sizeof(Block) +
         p.C.size() * sizeof(Cluster) + pb.dense.size() * sizeof(DenseDev) +
         pb.slots.size() * sizeof(SlotDev) + pb.pairs.size() * sizeof(LRPairDev) +
         pb.ptask.size() * sizeof(int) + pb.ls.steps.size() * sizeof(StepInfo) +
         pb.ls.step_cta.size() * sizeof(StepCta) + pb.ls.jobs.size() * sizeof(SolJob) + 256;
}

static std::shared_ptr<PlanBundle> plan_cache_get(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_plan_idx.find(key);
  if (it == g_plan_idx.end()) return nullptr;
  g_plan_lru.splice(g_plan_lru.begin(), g_plan_lru, it->second);
  return g_plan_lru.front().second;
}

static void plan_cache_put(const std::string& key, std::shared_ptr<PlanBundle> pb) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  if (g_plan_idx.count(key)) return;
  g_plan_bytes += plan_bytes(*pb);
  g_plan_lru.emplace_front(key, std::move(pb));
  g_plan_idx[key] = g_plan_lru.begin();
  while (g_plan_lru.size() > 1 &&
         (g_plan_lru.size() > kPlanCacheMax || g_plan_bytes > kPlanCacheBytes)) {
    g_plan_bytes -= plan_bytes(*g_plan_lru.back().second);
    g_plan_idx.erase(g_plan_lru.back().first);
    g_plan_lru.pop_back();
  }
}

static std::string plan_key(const InstHost& I, const PlanOpts& o) {
  std::string k(reinterpret_cast<const char*>(I.h.data()), I.h.size() * sizeof(double));
  char buf[128];
  snprintf(buf, sizeof(buf), "|%d|%d|%.17g|%d|%d|%d|%d|%d|%d|%d", I.N, I.P, o.lambda, o.leaf_elems, o.R,
           o.kmax, o.max_concat, o.adm_min, o.structure_only, o.ncta);
  return k + buf;
}

// For every element e, the first trial element f of the pairs (e, f <= e)
// that the dense blocks of plan p read (entries of A in rows and columns of
// a cluster involve the elements of its bubbles and of its hats' supports).
static void band_need(const HPlan& p, int N, std::vector<int>& flo) {
  flo.resize(N);
  for (int e = 0; e < N; ++e) flo[e] = e;
  auto lo_of = [&](const Cluster& c) { return c.e0; };
  auto hi_of = [&](const Cluster& c) { return std::min(c.e1, N - 1); };
  for (int bi : p.dense_blocks) {
    const Cluster &t = p.C[p.B[bi].t], &c = p.C[p.B[bi].s];
    for (int pass = 0; pass < 2; ++pass) {
      const Cluster& a = pass ? c : t;   // test side
      const Cluster& b = pass ? t : c;   // trial side
      const int blo = lo_of(b);
      for (int e = std::max(lo_of(a), blo); e <= hi_of(a); ++e) flo[e] = std::min(flo[e], blo);
    }
  }
}

// Factor the system instances in `list` with one arithmetic (`precision`).
static hfsem_factor* factor_part(hfsem_system* s, const hfsem_hopts& opt, const std::vector<int>& list,
                                 int precision) {
  auto* f = new hfsem_factor();
  try {
    f->sys = s;
    f->st = s->st;
    f->precision = precision;
    f->insts = list;
    f->nfi = (int)list.size();
    // the FP64 part of a mixed-precision factor is in FP64 for the range of
    // its meshes' entries; its leaf LUs keep the FP32 arithmetic of the mode
    f->leaf32 = (precision == HFSEM_PREC_FP64 && opt.precision != HFSEM_PREC_FP64) ? 1 : 0;
    f->build_only = opt.build_only;
    f->tol = opt.tol_hlu;
    f->R = opt.R;
    const bool fp32 = f->precision != HFSEM_PREC_FP64;
    f->tsize = fp32 ? sizeof(float) : sizeof(double);
    size_t sol_budget = 0;   // shared memory the leaf solve may take
    {
      int dev = 0, optin = 0;
      HF_CHECK(cudaGetDevice(&dev));
      HF_CHECK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      sol_budget = (size_t)optin - 1024;
    }
    const int max_leaf = fp32 ? 128 : 96;
    std::map<std::string, std::shared_ptr<PlanBundle>> cache;
    const int ni = f->nfi;
    {
      // a part of one or two large instances (a request of the serving loop)
      // runs its H-LU program on clusters of 16 CTAs: its waves hold tens of
      // ops, and 8 CTAs would leave most of the GPU idle
      int maxnd = 0;
      for (int i : list) maxnd = std::max(maxnd, s->ih[i].Nd);
      f->ncl = (!opt.build_only && ni <= kWideMaxInst && maxnd >= kWideNd) ? kWideCluster
               : (ni >= kNarrowMinInst ? kNarrowCluster : kCluster);
    }
    std::vector<std::string> keys(ni);
    f->plans.resize(ni);
    f->hidev.resize(ni);
    std::vector<PlanOpts> popts(ni);
    for (int i = 0; i < ni; ++i) {
      const InstHost& I = s->ih[list[i]];
      PlanOpts o;
      o.lambda = opt.lambda;
      o.adm_min = opt.admissibility == HFSEM_ADM_MIN ? 1 : 0;
      const int kmax_eff = opt.kmax ? opt.kmax : opt.R;
      const int max_concat = fp32 ? 160 : 112;   // shared memory of the recompression
      // a dense product appended to a low-rank block adds one leaf's worth of rank
      // (in slices of 32 columns) to a block holding up to kKcapMult kmax
      const int leaf_cap = std::min(max_leaf, max_concat - kKcapMult * kmax_eff);
      int leaf = opt.leaf_elems ? opt.leaf_elems : std::max(1, leaf_cap / I.P);
      if (!opt.leaf_elems && !opt.build_only) {   // a tuned size for the instance's class
        const int d = tune_leaf_dofs(I, opt.precision);
        if (d > 0) leaf = std::max(1, d / I.P);
      }
      if (opt.build_only) {
        // an H-matrix built, never factored: no shared-memory limit on its
        // leaves (128 unknowns by default)
        leaf = opt.leaf_elems ? opt.leaf_elems : std::max(1, 128 / I.P);
        o.structure_only = 1;
      } else {
        leaf = std::min(leaf, std::max(1, leaf_cap / I.P));
      }
      o.leaf_elems = leaf;
      o.R = opt.R;
      o.kmax = kmax_eff;
      o.nrhs_max = 64;
      o.max_concat = max_concat;
      o.max_leaf = max_leaf;
      o.unique_tmp = 1;
      o.ncta = f->ncl;
      popts[i] = o;
      keys[i] = plan_key(I, o) + (fp32 ? "|f32|" : "|f64|") + std::to_string(sol_budget);
    }
    // plans not cached yet, one per distinct key, built on all host cores
    std::vector<int> todo;
    for (int i = 0; i < ni; ++i) {
      if (cache.count(keys[i])) continue;
      if (auto hit = plan_cache_get(keys[i])) {
        cache.emplace(keys[i], hit);
        continue;
      }
      cache.emplace(keys[i], nullptr);
      todo.push_back(i);
    }
    auto make_bundle = [&](int i) {
      const InstHost& I = s->ih[list[i]];
      const PlanOpts& o = popts[i];
      auto pb = std::make_shared<PlanBundle>();
      make_plan(I, o, pb->plan);
      HPlan& p = pb->plan;
      for (int bi : p.dense_blocks) {
        const Block& b = p.B[bi];
        pb->dense.push_back(DenseDev{b.off, p.C[b.t].d0, b.m, p.C[b.s].d0, b.n});
      }
      for (int bi : p.lr_blocks) {
        const Block& b = p.B[bi];
        pb->slots.push_back(SlotDev{b.off, b.m, b.n, b.kcap, b.kmax});
      }
      // pair lower blocks (t right of s) with their mirrors
      std::map<std::pair<int, int>, int> slot_of;
      for (int bi : p.lr_blocks) slot_of[{p.B[bi].t, p.B[bi].s}] = p.B[bi].slot;
      for (int bi : p.lr_blocks) {
        const Block& b = p.B[bi];
        if (!b.lower) continue;
        auto mi = slot_of.find({b.s, b.t});
        if (mi == slot_of.end()) throw Error(HFSEM_ERR_DEVICE, "block tree is not symmetric");
        const Cluster &ct = p.C[b.t], &cs = p.C[b.s];
        pb->pairs.push_back(LRPairDev{b.slot, mi->second, ct.e0, ct.e1, cs.e0, cs.e1, ct.lo,
                                      ct.hi, cs.lo, cs.hi, ct.d0, b.m, cs.d0, b.n, pb->lrrows});
        pb->lrrows += (long long)(b.m + b.n) * opt.R;
      }
      // one task per element of each side (element e1 only feeds the hat at
      // node e1 and is left out when it is past the last element)
      pb->ptask.assign(1, 0);
      for (const LRPairDev& q : pb->pairs) {
        const int nt = ((q.te1 < I.N) ? q.te1 : q.te1 - 1) - q.te0 + 1;
        const int ns = ((q.se1 < I.N) ? q.se1 : q.se1 - 1) - q.se0 + 1;
        pb->ptask.push_back(pb->ptask.back() + nt + ns);
      }
      if (!o.structure_only)
        build_leaf_solve(pb->plan, kCluster, sol_budget, (int)f->tsize,
                         fp32 ? solve_w<float>() : solve_w<double>(), pb->ls);
      return pb;
    };
    {
      std::vector<std::shared_ptr<PlanBundle>> built(todo.size());
      std::vector<std::exception_ptr> errs(todo.size());
      std::atomic<size_t> next{0};
      auto worker = [&] {
        for (size_t w; (w = next.fetch_add(1)) < todo.size();) {
          try {
            built[w] = make_bundle(todo[w]);
          } catch (...) {
            errs[w] = std::current_exception();
          }
        }
      };
      const size_t nth = std::min<size_t>(todo.size(),
                                          std::max(1u, std::min(32u, std::thread::hardware_concurrency())));
      std::vector<std::thread> pool;
      for (size_t t = 1; t < nth; ++t) pool.emplace_back(worker);
      worker();
      for (auto& t : pool) t.join();
      for (auto& e : errs)
        if (e) std::rethrow_exception(e);
      for (size_t w = 0; w < todo.size(); ++w) {
        plan_cache_put(keys[todo[w]], built[w]);
        cache[keys[todo[w]]] = built[w];
      }
    }
    for (int i = 0; i < ni; ++i) f->plans[i] = cache[keys[i]];
    // an instance assembled with the H-matrix operator stores only the pairs
    // of the operator's near field: this factor's must lie inside it
    for (int i = 0; i < ni; ++i) {
      const InstHost& I = s->ih[list[i]];
      if (I.kind != kHmat) continue;
      std::vector<int> need;
      band_need(f->plans[i]->plan, I.N, need);
      for (int e = 0; e < I.N; ++e)
        if (need[e] < I.flo[e])
          throw Error(HFSEM_ERR_UNSUPPORTED,
                      "the H-LU near field reaches pairs the H-matrix operator does not store: "
                      "factor with HFSEM_ADM_MIN, lambda >= 1 and automatic leaves, or assemble "
                      "with HFSEM_MATVEC_DENSE");
    }
    // one solve kernel serves every plan: cut the parts of each plan for the
    // largest leaf and the most owned low-rank columns of all of them
    {
      int nm = 1, wc = 1;
      for (auto& kv : cache) {
        nm = std::max(nm, kv.second->ls.nmax);
        wc = std::max(wc, kv.second->ls.wcols);
      }
      // a private copy for each plan cut for less: the shared plan keeps the
      // tables cut for itself (on all host cores, as above)
      std::vector<std::shared_ptr<PlanBundle>*> recut;
      for (auto& kv : cache)
        if (!opt.build_only && (kv.second->ls.nmax < nm || kv.second->ls.wcols < wc))
          recut.push_back(&kv.second);
      std::vector<std::exception_ptr> errs(recut.size());
      std::atomic<size_t> next{0};
      auto worker = [&] {
        for (size_t w; (w = next.fetch_add(1)) < recut.size();) {
          try {
            auto cp = std::make_shared<PlanBundle>(**recut[w]);
            build_leaf_solve(cp->plan, kCluster, sol_budget, (int)f->tsize,
                             fp32 ? solve_w<float>() : solve_w<double>(), cp->ls, nm, wc);
            *recut[w] = cp;
          } catch (...) {
            errs[w] = std::current_exception();
          }
        }
      };
      const size_t nth = std::min<size_t>(recut.size(),
                                          std::max(1u, std::min(32u, std::thread::hardware_concurrency())));
      std::vector<std::thread> pool;
      for (size_t t = 1; t < nth; ++t) pool.emplace_back(worker);
      if (!recut.empty()) worker();
      for (auto& t : pool) t.join();
      for (auto& e : errs)
        if (e) std::rethrow_exception(e);
      for (int i = 0; i < ni; ++i) f->plans[i] = cache[keys[i]];
    }
    // concatenate tables
    std::vector<HOp> ops;
    std::vector<int> waves;
    std::vector<SlotDev> slots;
    std::vector<DenseDev> dense;
    std::vector<LRPairDev> pairs;
    std::map<const PlanBundle*, std::array<long long, 7>> placed;
    std::vector<StepInfo> steps;
    std::vector<StepCta> step_cta;
    std::vector<SolJob> jobs;
    std::map<const PlanBundle*, std::array<long long, 2>> placed_leaf;
    std::map<const PlanBundle*, long long> placed_task;
    std::vector<int> ptask;
    long long gmax_n = 0, max_tasks = 0, lrt_n = 0;
    int jmax = 1, nmax = 1, wcols = 1;
    long long arena = 0, rk = 0, doff = 0, pkoff = 0;
    size_t smem = 0;
    for (int i = 0; i < ni; ++i) {
      const PlanBundle* pb = f->plans[i].get();
      auto pi = placed.find(pb);
      if (pi == placed.end()) {
        std::array<long long, 7> a{(long long)ops.size(), 0, (long long)slots.size(),
                                   (long long)dense.size(), (long long)pairs.size(),
                                   (long long)waves.size(), 0};
        waves.insert(waves.end(), pb->plan.fac_waves.begin(), pb->plan.fac_waves.end());
        ops.insert(ops.end(), pb->plan.fac.begin(), pb->plan.fac.end());
        slots.insert(slots.end(), pb->slots.begin(), pb->slots.end());
        dense.insert(dense.end(), pb->dense.begin(), pb->dense.end());
        pairs.insert(pairs.end(), pb->pairs.begin(), pb->pairs.end());
        placed_task[pb] = (long long)ptask.size();
        ptask.insert(ptask.end(), pb->ptask.begin(), pb->ptask.end());
        pi = placed.emplace(pb, a).first;
        smem = std::max(smem, prog_smem(pb->plan, f->tsize));
        placed_leaf[pb] = {(long long)steps.size(), (long long)jobs.size()};
        steps.insert(steps.end(), pb->ls.steps.begin(), pb->ls.steps.end());
        step_cta.insert(step_cta.end(), pb->ls.step_cta.begin(), pb->ls.step_cta.end());
        jobs.insert(jobs.end(), pb->ls.jobs.begin(), pb->ls.jobs.end());
        jmax = std::max(jmax, pb->ls.jcap);
        wcols = std::max(wcols, pb->ls.wcols);
        nmax = std::max(nmax, pb->ls.nmax);
      }
      HInstDev& H = f->hidev[i];
      std::memset(&H, 0, sizeof(H));
      const HPlan& p = pb->plan;
      H.arena = arena;
      arena += p.arena;
      arena = (arena + 31) & ~31LL;
      H.rk0 = rk;
      rk += p.n_slots + 1;
      H.slot0 = pi->second[2];
      H.dense0 = pi->second[3];
      H.pair0 = pi->second[4];
      H.ptask0 = placed_task[pb];
      H.gmax0 = gmax_n;
      gmax_n += (long long)pb->pairs.size();
      H.lrt0 = lrt_n;
      lrt_n += pb->lrrows;
      max_tasks = std::max<long long>(max_tasks, pb->ptask.back());
      H.ops0 = pi->second[0];

      H.nops = (int)p.fac.size();

      H.ndense = (int)pb->dense.size();
      H.npairs = (int)pb->pairs.size();
      H.n_slots = p.n_slots;
      H.ws_off = p.ws_off;
      H.ws_size = p.ws_size;
      H.rhs_off = p.rhs_off;
      H.fw0 = pi->second[5];

      H.nfw = (int)p.fac_waves.size() - 1;

      H.d_off = doff;
      doff += s->ih[list[i]].Nd;
      H.sys_inst = list[i];
      H.R = opt.R;
      H.nd = s->ih[list[i]].Nd;
      H.st0 = placed_leaf[pb][0];
      H.job0 = placed_leaf[pb][1];
      H.jcap = pb->ls.jcap;
      H.nst = (int)pb->ls.steps.size();
      H.njob = (int)pb->ls.jobs.size();
      H.pk0 = pkoff;
      pkoff += (long long)pb->ls.jobs.size();
      f->total_ops += H.nops;

    }
    // every CTA of the cluster sits alone on its SM (register bound), so the
    // kernel takes all the shared memory it may have: the recompression
    // stages its tall factors in what the other ops leave free
    {
      int dev = 0, optin = 0;
      HF_CHECK(cudaGetDevice(&dev));
      HF_CHECK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      cudaFuncAttributes fa;
      if (fp32)
        HF_CHECK(cudaFuncGetAttributes(&fa, k_hprog<float>));
      else
        HF_CHECK(cudaFuncGetAttributes(&fa, k_hprog<double>));
      const size_t avail = (size_t)optin - fa.sharedSizeBytes - 1024;
      if (smem > avail && !opt.build_only)
        throw Error(HFSEM_ERR_UNSUPPORTED, "H-LU kernel needs too much shared memory");
      smem = avail & ~(size_t)15;
    }
    f->smem = smem;
    f->d_hi.alloc(ni);
    HF_CHECK(cudaMemcpyAsync(f->d_hi.p, f->hidev.data(), ni * sizeof(HInstDev), cudaMemcpyHostToDevice, s->st));
    f->d_waves.alloc(std::max<size_t>(waves.size(), 1));
    if (!waves.empty())
      HF_CHECK(cudaMemcpyAsync(f->d_waves.p, waves.data(), waves.size() * sizeof(int), cudaMemcpyHostToDevice, s->st));
    f->d_ops.alloc(std::max<size_t>(ops.size(), 1));
    if (!ops.empty())
      HF_CHECK(cudaMemcpyAsync(f->d_ops.p, ops.data(), ops.size() * sizeof(HOp), cudaMemcpyHostToDevice, s->st));
    f->d_slots.alloc(std::max<size_t>(slots.size(), 1));
    if (!slots.empty())
      HF_CHECK(cudaMemcpyAsync(f->d_slots.p, slots.data(), slots.size() * sizeof(SlotDev), cudaMemcpyHostToDevice, s->st));
    f->d_dense.alloc(std::max<size_t>(dense.size(), 1));
    if (!dense.empty())
      HF_CHECK(cudaMemcpyAsync(f->d_dense.p, dense.data(), dense.size() * sizeof(DenseDev), cudaMemcpyHostToDevice, s->st));
    f->d_pairs.alloc(std::max<size_t>(pairs.size(), 1));
    if (!pairs.empty())
      HF_CHECK(cudaMemcpyAsync(f->d_pairs.p, pairs.data(), pairs.size() * sizeof(LRPairDev), cudaMemcpyHostToDevice, s->st));
    f->d_ptask.alloc(std::max<size_t>(ptask.size(), 1));
    if (!ptask.empty())
      HF_CHECK(cudaMemcpyAsync(f->d_ptask.p, ptask.data(), ptask.size() * sizeof(int), cudaMemcpyHostToDevice, s->st));
    f->d_gmax.alloc((size_t)std::max<long long>(gmax_n, 1) * 64);
    f->d_lrt.alloc((size_t)std::max<long long>(lrt_n, 1));
    HF_CHECK(cudaMemsetAsync(f->d_gmax.p, 0, f->d_gmax.n * sizeof(unsigned long long), s->st));
    f->d_steps.alloc(std::max<size_t>(steps.size(), 1));
    if (!steps.empty())
      HF_CHECK(cudaMemcpyAsync(f->d_steps.p, steps.data(), steps.size() * sizeof(StepInfo), cudaMemcpyHostToDevice, s->st));
    f->d_step_cta.alloc(std::max<size_t>(step_cta.size(), 1));
    if (!step_cta.empty())
      HF_CHECK(cudaMemcpyAsync(f->d_step_cta.p, step_cta.data(), step_cta.size() * sizeof(StepCta), cudaMemcpyHostToDevice, s->st));
    f->d_jobs.alloc(std::max<size_t>(jobs.size(), 1));
    if (!jobs.empty())
      HF_CHECK(cudaMemcpyAsync(f->d_jobs.p, jobs.data(), jobs.size() * sizeof(SolJob), cudaMemcpyHostToDevice, s->st));
    // leaf-solve shared memory: two buffers of jmax column slots, seven 128 x W
    // vectors, the ring, the CTA's w columns, the gather scalars and two
    // buffers of job records
    f->sol_jmax = jmax;
    f->sol_slot = (int)(((size_t)nmax * f->tsize + 15) / 16 * 16 / f->tsize);
    f->sol_wcols = wcols;
    const int sw = fp32 ? solve_w<float>() : solve_w<double>();
    f->sol_smem = solve_smem(jmax, nmax, wcols, (int)f->tsize, sw);
    f->d_pack.alloc((size_t)std::max<long long>(pkoff, 1) * f->sol_slot * f->tsize);
    f->d_meta.alloc((size_t)std::max<long long>(pkoff, 1));
    if (!opt.build_only) {
      if (f->sol_smem > sol_budget)
        throw Error(HFSEM_ERR_UNSUPPORTED, "leaf solve needs too much shared memory");
      if (fp32)
        allow_dyn_smem((const void*)k_hsolve_cl<float>, f->sol_smem);
      else
        allow_dyn_smem((const void*)k_hsolve_cl<double>, f->sol_smem);
    }
    f->d_ranks.alloc(std::max<long long>(rk, 1));
    HF_CHECK(cudaMemsetAsync(f->d_ranks.p, 0, std::max<long long>(rk, 1) * sizeof(int), s->st));
    f->d_err.alloc(ni);
    HF_CHECK(cudaMemsetAsync(f->d_err.p, 0, ni * sizeof(int), s->st));
    f->d_D.alloc(std::max<long long>(doff, 1));
    f->d_arena.alloc((size_t)std::max<long long>(arena, 1) * f->tsize);
    HF_CHECK(cudaMemsetAsync(f->d_arena.p, 0, (size_t)std::max<long long>(arena, 1) * f->tsize, s->st));
    // build A~
    int maxnd = 1, maxdense = 1, maxnpairs = 1;
    for (auto& H : f->hidev) {
      maxnd = std::max(maxnd, s->ih[H.sys_inst].Nd);
      maxdense = std::max(maxdense, H.ndense);
      maxnpairs = std::max(maxnpairs, H.npairs);
    }
    const bool prof = getenv("HFSEM_PROFILE") != nullptr;
    cudaEvent_t ev[5];
    if (prof)
      for (auto& e : ev) cudaEventCreate(&e);
    if (prof) cudaEventRecord(ev[0], s->st);
    dim3 gd((maxnd + 255) / 256, ni);
    k_diag<<<gd, 256, 0, s->st>>>(f->d_hi.p, s->d_inst.p, s->arena.p, f->d_D.p);
    HF_LAUNCH_CHECK();
    dim3 gn(std::min(maxdense, 1024), ni);
    // low-rank build: warps per CTA as the per-warp quadrature tables allow
    const int Pm = s->max_P, Rr = opt.R;
    const int nqm = std::min((Pm + Rr) / 2 + 13, kMaxGL);
    const size_t per_warp = lowrank_warp_bytes(nqm, Pm, Rr, f->tsize);
    const size_t per_cta = lowrank_cta_bytes(nqm, Pm, Rr, f->tsize);
    const int lr_warps = (int)std::max<size_t>(1, std::min<size_t>(8, (160 * 1024 - per_cta) / per_warp));
    const size_t lr_smem = per_cta + lr_warps * per_warp;
    dim3 gp((unsigned)std::max<long long>(1, std::min<long long>((max_tasks + lr_warps - 1) / lr_warps, 2048)), ni);
    if (fp32) {
      float* ar = reinterpret_cast<float*>(f->d_arena.p);
      k_nearfield<float><<<gn, 256, 0, s->st>>>(f->d_hi.p, s->d_inst.p, s->arena.p, f->d_dense.p, f->d_D.p, ar);
      HF_LAUNCH_CHECK();
      if (prof) cudaEventRecord(ev[1], s->st);
      if (lr_smem > 48 * 1024)
        allow_dyn_smem((const void*)k_lowrank<float>, lr_smem);
      k_lowrank<float><<<gp, lr_warps * 32, lr_smem, s->st>>>(f->d_hi.p, s->d_inst.p, s->arena.p, s->gl.p,
                                                          f->d_pairs.p, f->d_slots.p, f->d_ptask.p,
                                                          f->d_D.p, f->d_lrt.p, f->d_gmax.p);
      HF_LAUNCH_CHECK();
      k_lowrank_write<float><<<dim3(std::max(1, std::min(maxnpairs, 1024)), ni), 256, 0, s->st>>>(
          f->d_hi.p, s->d_inst.p, f->d_pairs.p, f->d_slots.p, f->d_lrt.p, f->d_gmax.p, ar, f->d_ranks.p);
      HF_LAUNCH_CHECK();
      set_prog_smem<float>(smem);
    } else {
      double* ar = reinterpret_cast<double*>(f->d_arena.p);
      k_nearfield<double><<<gn, 256, 0, s->st>>>(f->d_hi.p, s->d_inst.p, s->arena.p, f->d_dense.p, f->d_D.p, ar);
      HF_LAUNCH_CHECK();
      if (prof) cudaEventRecord(ev[1], s->st);
      if (lr_smem > 48 * 1024)
        allow_dyn_smem((const void*)k_lowrank<double>, lr_smem);
      k_lowrank<double><<<gp, lr_warps * 32, lr_smem, s->st>>>(f->d_hi.p, s->d_inst.p, s->arena.p, s->gl.p,
                                                          f->d_pairs.p, f->d_slots.p, f->d_ptask.p,
                                                          f->d_D.p, f->d_lrt.p, f->d_gmax.p);
      HF_LAUNCH_CHECK();
      k_lowrank_write<double><<<dim3(std::max(1, std::min(maxnpairs, 1024)), ni), 256, 0, s->st>>>(
          f->d_hi.p, s->d_inst.p, f->d_pairs.p, f->d_slots.p, f->d_lrt.p, f->d_gmax.p, ar, f->d_ranks.p);
      HF_LAUNCH_CHECK();
      set_prog_smem<double>(smem);
    }
    if (prof) cudaEventRecord(ev[2], s->st);
    if (!f->build_only) {
      f->run_prog();
      f->run_pack();
    }
    if (prof) cudaEventRecord(ev[3], s->st);
    HF_CHECK(cudaStreamSynchronize(s->st));
    if (prof) {
      float a = 0, b = 0, c = 0;
      cudaEventElapsedTime(&a, ev[0], ev[1]);
      cudaEventElapsedTime(&b, ev[1], ev[2]);
      cudaEventElapsedTime(&c, ev[2], ev[3]);
      fprintf(stderr, "[hfsem phases] diag+nearfield %.3f ms  lowrank %.3f ms  hlu %.3f ms\n", a, b, c);
      for (auto& e : ev) cudaEventDestroy(e);
    }
    if (getenv("HFSEM_PROFILE")) {
      const HPlan& p0 = f->plans[0]->plan;
      fprintf(stderr, "[hfsem plan] N=%d P=%d blocks=%zu dense=%zu lr=%zu fac_ops=%zu waves=%zu "
              "leaf_max=%d kconcat_max=%d hh_lr=%d arena=%lld\n", p0.N, p0.P, p0.B.size(),
              p0.dense_blocks.size(), p0.lr_blocks.size(), p0.fac.size(), (size_t)p0.fac_waves.size() - 1, p0.leaf_max,
              p0.kconcat_max, p0.hh_lr, p0.arena);
      f->report("factorisation");
      f->report_waves("factorisation");
    }
    std::vector<int> err(ni);
    HF_CHECK(cudaMemcpyAsync(err.data(), f->d_err.p, ni * sizeof(int), cudaMemcpyDeviceToHost, s->st));
    HF_CHECK(cudaStreamSynchronize(s->st));
    for (int e : err) {
      if (e == 3) throw Error(HFSEM_ERR_DEVICE, "low-rank block above the rank bound of the solves");
      if (e == 4) {
        unsigned long long d[8] = {0};
        if (f->d_tcdbg.p && cudaMemcpyAsync(d, f->d_tcdbg.p, sizeof(d), cudaMemcpyDeviceToHost,
                                            s->st) == cudaSuccess)
          cudaStreamSynchronize(s->st);
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "a tensor-core product did not complete within its wait limit (mbarrier %llx, "
                 "a-desc %llx, b-desc %llx, idesc %llx, tmem %llx, N|K %llx)",
                 d[0], d[1], d[2], d[3], d[4], d[5]);
        throw Error(HFSEM_ERR_TIMEOUT, msg);
      }
      if (e) throw Error(HFSEM_ERR_BREAKDOWN, "zero or non-finite pivot in an H-LU leaf");
    }
  } catch (...) {
    delete f;
    throw;
  }
  return f;
}

static hfsem_factor* factor(hfsem_system* s, const hfsem_hopts& opt) {
  AllocStream as(s->st);   // the factor's buffers come stream-ordered from the pool
  if (opt.R < 1 || opt.R > 32) throw Error(HFSEM_ERR_INVALID_ARG, "R must be in [1, 32]");
  if (!(opt.lambda > 0.0)) throw Error(HFSEM_ERR_INVALID_ARG, "lambda must be > 0");
  if (!(opt.tol_hlu >= 0.0)) throw Error(HFSEM_ERR_INVALID_ARG, "tol_hlu must be >= 0");
  if (opt.precision != HFSEM_PREC_FP64 && opt.precision != HFSEM_PREC_MIXED &&
      opt.precision != HFSEM_PREC_MIXED_TC)
    throw Error(HFSEM_ERR_INVALID_ARG, "unknown precision");
  if (opt.leaf_elems < 0 || opt.kmax < 0) throw Error(HFSEM_ERR_INVALID_ARG, "leaf_elems, kmax >= 0");
  if (opt.admissibility != HFSEM_ADM_MAX && opt.admissibility != HFSEM_ADM_MIN)
    throw Error(HFSEM_ERR_INVALID_ARG, "admissibility: HFSEM_ADM_MAX or HFSEM_ADM_MIN");
  // FP32 cannot factor the equilibrated H-matrix of meshes whose element
  // sizes span more than ~1e45 (the preconditioner then loses all digits):
  // those instances are factored in FP64, the others in the requested mode
  std::vector<int> lo, hi;
  for (int i = 0; i < s->n_inst; ++i) {
    const InstHost& I = s->ih[i];
    const double hmax = *std::max_element(I.h.begin(), I.h.end());
    const double hmin = *std::min_element(I.h.begin(), I.h.end());
    (opt.precision != HFSEM_PREC_FP64 && !(hmax > 1e45 * hmin) ? lo : hi).push_back(i);
  }
  if (hi.empty()) return factor_part(s, opt, lo, opt.precision);
  if (lo.empty()) return factor_part(s, opt, hi, HFSEM_PREC_FP64);
  auto* f = new hfsem_factor();
  try {
    f->sys = s;
    f->st = s->st;
    f->precision = opt.precision;
    f->build_only = opt.build_only;
    f->tol = opt.tol_hlu;
    f->R = opt.R;
    f->nfi = s->n_inst;
    for (int i = 0; i < s->n_inst; ++i) f->insts.push_back(i);
    f->parts.emplace_back(factor_part(s, opt, lo, opt.precision));
    f->parts.emplace_back(factor_part(s, opt, hi, HFSEM_PREC_FP64));
  } catch (...) {
    delete f;
    throw;
  }
  return f;
}

// ---------------------------------------------------------------------------
// H-matrix operator (kHmat instances): A~ in FP64 at rank kHopRank with the
// min-diameter rule (Sec. 3 at a rank where the Lemma's bound is below the
// rounding of FP64), built by the same kernels as the preconditioner's
// H-matrix, applied as y += D^-1 (D A~ D) D^-1 x.
// ---------------------------------------------------------------------------
static PlanOpts hop_plan_opts(int P) {
  PlanOpts o{};
  o.lambda = kHopLambda;
  o.leaf_elems = std::max(1, kHopLeafDofs / P);
  o.R = kHopRank;
  o.kmax = kHopRank;
  o.nrhs_max = 64;
  o.max_concat = 112;
  o.max_leaf = kHopLeafDofs;
  o.unique_tmp = 1;
  o.ncta = kCluster;
  o.structure_only = 1;
  o.adm_min = 1;
  return o;
}

void hop_band(const InstHost& I, std::vector<int>& flo) {
  HPlan p;
  make_plan(I, hop_plan_opts(I.P), p);
  band_need(p, I.N, flo);
}

void build_operator(hfsem_system* s) {
  std::vector<int> list;
  for (int i = 0; i < s->n_inst; ++i)
    if (s->ih[i].kind == kHmat) list.push_back(i);
  if (list.empty()) return;
  hfsem_hopts o{};
  o.R = kHopRank;
  o.lambda = kHopLambda;
  o.tol_hlu = 0.0;
  o.precision = HFSEM_PREC_FP64;
  o.leaf_elems = 0;
  o.kmax = 0;
  o.build_only = 1;
  o.admissibility = HFSEM_ADM_MIN;
  hfsem_factor* f = factor_part(s, o, list, HFSEM_PREC_FP64);
  s->hop = f;
  // product tables: per leaf row cluster, the blocks whose rows hold it
  std::vector<HopRow> rows;
  std::vector<HopItem> items;
  std::vector<HopSlot> slots;
  long long w0 = 0;
  double flops = 0.0;
  int kmax = 1;
  for (int j = 0; j < f->nfi; ++j) {
    const HPlan& p = f->plans[j]->plan;
    const HInstDev& H = f->hidev[j];
    const int nc = (int)p.C.size();
    std::vector<std::vector<int>> at(nc);   // blocks by row cluster
    for (int bi : p.dense_blocks) at[p.B[bi].t].push_back(bi);
    std::vector<int> slot_rec(p.n_slots, -1);
    for (int bi : p.lr_blocks) {
      const Block& b = p.B[bi];
      at[b.t].push_back(bi);
      slot_rec[b.slot] = (int)slots.size();
      const int k = std::min(kHopRank, std::min(b.m, b.n));
      slots.push_back(HopSlot{H.arena + b.off + (long long)b.m * b.kcap, w0, j, p.C[b.s].d0, b.n,
                              b.kcap, (int)(H.rk0 + b.slot)});
      w0 += b.kcap;
      kmax = std::max(kmax, b.kcap);
      flops += 2.0 * (b.m + b.n) * k;
    }
    for (int bi : p.dense_blocks) flops += 2.0 * p.B[bi].m * p.B[bi].n;
    // leaves, with the chain of their ancestors
    std::vector<int> parent(nc, -1);
    for (int c = 0; c < nc; ++c)
      for (int k = 0; k < 2; ++k)
        if (p.C[c].kid[k] >= 0) parent[p.C[c].kid[k]] = c;
    for (int c = 0; c < nc; ++c) {
      if (p.C[c].kid[0] >= 0 || p.C[c].d1 <= p.C[c].d0) continue;
      HopRow r{j, p.C[c].d0, p.C[c].d1 - p.C[c].d0, (int)items.size(), 0};
      for (int a = c; a >= 0; a = parent[a])
        for (int bi : at[a]) {
          const Block& b = p.B[bi];
          const int roff = p.C[c].d0 - p.C[b.t].d0;
          if (b.type == B_DENSE)
            items.push_back(HopItem{H.arena + b.off, 0, b.m, roff, p.C[b.s].d0, b.n});
          else
            items.push_back(HopItem{H.arena + b.off, 1, b.m, roff, slot_rec[b.slot], b.kcap});
        }
      r.it1 = (int)items.size();
      rows.push_back(r);
    }
  }
  f->hop_nrows = (int)rows.size();
  f->hop_nslots = (int)slots.size();
  f->hop_wsize = w0;
  f->hop_kmax = kmax;
  f->hop_flops = flops;
  f->d_hrow.alloc(std::max<size_t>(rows.size(), 1));
  f->d_hitem.alloc(std::max<size_t>(items.size(), 1));
  f->d_hslot.alloc(std::max<size_t>(slots.size(), 1));
  if (!rows.empty())
    HF_CHECK(cudaMemcpyAsync(f->d_hrow.p, rows.data(), rows.size() * sizeof(HopRow),
                             cudaMemcpyHostToDevice, s->st));
  if (!items.empty())
    HF_CHECK(cudaMemcpyAsync(f->d_hitem.p, items.data(), items.size() * sizeof(HopItem),
                             cudaMemcpyHostToDevice, s->st));
  if (!slots.empty())
    HF_CHECK(cudaMemcpyAsync(f->d_hslot.p, slots.data(), slots.size() * sizeof(HopSlot),
                             cudaMemcpyHostToDevice, s->st));
  HF_CHECK(cudaStreamSynchronize(s->st));   // host tables go out of scope
}

constexpr int kHopRB = 4;   // right-hand sides per pass

// x~ = D^-1 x on the kHmat instances (instance-local unknowns, rhs-major).
__global__ void k_hop_scale(const HInstDev* __restrict__ hi, const InstDev* __restrict__ inst,
                            const double* __restrict__ D, const double* __restrict__ x, double* xt,
                            int nrhs, const int* __restrict__ gate) {
  HF_GATE(gate);
  const HInstDev H = hi[blockIdx.y];
  const InstDev I = inst[H.sys_inst];
  const int r = blockIdx.z;
  const double* xv = x + I.o_vec * nrhs + (long long)r * I.Nd;
  double* tv = xt + I.o_vec * nrhs + (long long)r * I.Nd;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.Nd; i += gridDim.x * blockDim.x)
    tv[i] = xv[i] / D[H.d_off + i];
}

// w_b[k] = sum_j V_b[j][k] x~[c0 + j] for k below the block's rank (0 above),
// one warp per (block, column k).
__global__ void k_hop_proj(const HInstDev* __restrict__ hi, const InstDev* __restrict__ inst,
                           const HopSlot* __restrict__ slots, const int* __restrict__ ranks,
                           const double* __restrict__ ar, const double* __restrict__ xt, double* w,
                           long long wsize, int nrhs, const int* __restrict__ gate) {
  HF_GATE(gate);
  const HopSlot S = slots[blockIdx.x];
  const HInstDev H = hi[S.inst];
  const InstDev I = inst[H.sys_inst];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rank = ranks[S.rk];
  for (int k = warp; k < S.kcap; k += nw) {
    for (int r0 = 0; r0 < nrhs; r0 += kHopRB) {
      double acc[kHopRB];
#pragma unroll
      for (int q = 0; q < kHopRB; ++q) acc[q] = 0.0;
      if (k < rank) {
        const double* v = ar + S.offV + (long long)k * S.n;
        for (int j = lane; j < S.n; j += 32) {
          const double vj = v[j];
#pragma unroll
          for (int q = 0; q < kHopRB; ++q)
            if (r0 + q < nrhs) acc[q] = fma(vj, xt[I.o_vec * nrhs + (long long)(r0 + q) * I.Nd + S.c0 + j], acc[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < kHopRB; ++q) {
        double t = acc[q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0 && r0 + q < nrhs) w[(long long)(r0 + q) * wsize + S.w0 + k] = t;
      }
    }
  }
}

// y_i += D_i^-1 sum over the leaf's blocks (dense: row of D A~ D times x~;
// low-rank: row of U times w), a thread per row of the leaf.
__global__ void __launch_bounds__(128) k_hop_rows(const HInstDev* __restrict__ hi,
                                                  const InstDev* __restrict__ inst,
                                                  const HopRow* __restrict__ rows,
                                                  const HopItem* __restrict__ items,
                                                  const HopSlot* __restrict__ slots,
                                                  const int* __restrict__ ranks,
                                                  const double* __restrict__ D,
                                                  const double* __restrict__ ar,
                                                  const double* __restrict__ xt,
                                                  const double* __restrict__ w, long long wsize,
                                                  double* y, int nrhs,
                                                  const int* __restrict__ gate) {
  HF_GATE(gate);
  const HopRow Rw = rows[blockIdx.x];
  const HInstDev H = hi[Rw.inst];
  const InstDev I = inst[H.sys_inst];
  const int r0 = blockIdx.y * kHopRB;
  const double* xb = xt + I.o_vec * nrhs;
  for (int i = threadIdx.x; i < Rw.nr; i += blockDim.x) {
    double acc[kHopRB];
#pragma unroll
    for (int q = 0; q < kHopRB; ++q) acc[q] = 0.0;
    for (int t = Rw.it0; t < Rw.it1; ++t) {
      const HopItem It = items[t];
      if (It.kind == 0) {
        const double* a = ar + It.off + It.roff + i;
        for (int j = 0; j < It.nc; ++j) {
          const double aj = a[(long long)j * It.ld];
#pragma unroll
          for (int q = 0; q < kHopRB; ++q)
            if (r0 + q < nrhs) acc[q] = fma(aj, xb[(long long)(r0 + q) * I.Nd + It.c0 + j], acc[q]);
        }
      } else {
        const HopSlot S = slots[It.c0];
        const int rank = ranks[S.rk];
        const double* u = ar + It.off + It.roff + i;
        for (int k = 0; k < rank; ++k) {
          const double uk = u[(long long)k * It.ld];
#pragma unroll
          for (int q = 0; q < kHopRB; ++q)
            if (r0 + q < nrhs) acc[q] = fma(uk, w[(long long)(r0 + q) * wsize + S.w0 + k], acc[q]);
        }
      }
    }
    const double di = D[H.d_off + Rw.d0 + i];
#pragma unroll
    for (int q = 0; q < kHopRB; ++q)
      if (r0 + q < nrhs) y[I.o_vec * nrhs + (long long)(r0 + q) * I.Nd + Rw.d0 + i] += acc[q] / di;
  }
}

void hop_apply(hfsem_system* s, int nrhs, const double* x, double* y) {
  hfsem_factor* f = s->hop;
  if (!f || f->nfi == 0) return;
  Tick tk(s->st, "hmat_mv", f->hop_flops * nrhs);
  const long long nx = s->total_nd * nrhs;
  s->w_hop.ensure((size_t)(nx + f->hop_wsize * nrhs + 1));
  double* xt = s->w_hop.p;
  double* w = s->w_hop.p + nx;
  const double* ar = reinterpret_cast<const double*>(f->d_arena.p);
  int maxnd = 1;
  for (int i : f->insts) maxnd = std::max(maxnd, s->ih[i].Nd);
  k_hop_scale<<<dim3(std::min(1024, (maxnd + 255) / 256), f->nfi, nrhs), 256, 0, s->st>>>(
      f->d_hi.p, s->d_inst.p, f->d_D.p, x, xt, nrhs, s->gate);
  HF_LAUNCH_CHECK();
  if (f->hop_nslots > 0) {
    k_hop_proj<<<f->hop_nslots, 256, 0, s->st>>>(f->d_hi.p, s->d_inst.p, f->d_hslot.p, f->d_ranks.p,
                                                 ar, xt, w, f->hop_wsize, nrhs, s->gate);
    HF_LAUNCH_CHECK();
  }
  k_hop_rows<<<dim3(f->hop_nrows, (nrhs + kHopRB - 1) / kHopRB), 128, 0, s->st>>>(
      f->d_hi.p, s->d_inst.p, f->d_hrow.p, f->d_hitem.p, f->d_hslot.p, f->d_ranks.p, f->d_D.p, ar,
      xt, w, f->hop_wsize, y, nrhs, s->gate);
  HF_LAUNCH_CHECK();
}

}  // namespace hf

void hfsem_factor_s::collect_flops() {
  for (auto& q : parts) q->collect_flops();
  // move the device flop counters into the timing registry
  if (!d_flops.p || !hf::timing_on()) return;
  std::vector<double> h(d_flops.n);
  if (cudaMemcpyAsync(h.data(), d_flops.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return;
  double f0 = 0, f1 = 0;
  for (size_t i = 0; i < h.size(); i += 2) {
    f0 += h[i];
    f1 += h[i + 1];
  }
  hf::timing_add_work("hlu_factor", f0);
  hf::timing_add_work("hlu_solve", f1);
  cudaMemsetAsync(d_flops.p, 0, d_flops.n * sizeof(double), st);
}

void hfsem_factor_s::report(const char* what) {
  if (!d_prof.p) return;
  std::vector<unsigned long long> h(d_prof.n);
  cudaMemcpy(h.data(), d_prof.p, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  static const char* names[16] = {"?", "GEMM", "GETRF_INV", "TRMM_L", "TRMM_R", "APPEND",
                                  "TRUNC", "ZERO", "AXPY", "APPEND+TR", "?", "?", "?", "?", "?", "?"};
  // the instance with the most op time
  int worst = 0;
  unsigned long long wt = 0;
  const size_t ninst = (h.size() - 16 - 64) / 32;
  for (size_t c = 0; c < ninst; ++c) {
    unsigned long long t = 0;
    for (int k = 0; k < 16; ++k) t += h[c * 32 + 2 * k];
    if (t > wt) {
      wt = t;
      worst = (int)c;
    }
  }
  fprintf(stderr, "[hfsem profile] %s (instance %d, all CTAs; ns, ops)\n", what, worst);
  for (int t = 0; t < 16; ++t) {
    const unsigned long long ns = h[worst * 32 + 2 * t], n = h[worst * 32 + 2 * t + 1];
    if (n) fprintf(stderr, "  %-10s %14llu ns %8llu ops %10.0f ns/op\n", names[t], ns, n, (double)ns / n);
  }
  {
    const unsigned long long* q = &h[ninst * 32];
    if (q[8]) {
      static const char* ph[7] = {"qr U", "qr V", "core", "rrqr", "Z+rows", "apply U", "apply V"};
      if (q[15])
        fprintf(stderr, "[hfsem leaf LU] %llu calls, us per call: load %.1f forward %.1f out+scale %.1f backward+out %.1f\n",
                q[15], q[11] * 1e-3 / q[15], q[12] * 1e-3 / q[15], q[13] * 1e-3 / q[15], q[14] * 1e-3 / q[15]);
      fprintf(stderr, "[hfsem recompression] %llu calls (all instances), mean K %.1f, mean m+n %.0f; us/call:",
              q[8], (double)q[9] / q[8], (double)q[10] / q[8]);
      for (int k = 0; k < 7; ++k) fprintf(stderr, " %s %.1f", ph[k], q[k] * 1e-3 / q[8]);
      fprintf(stderr, "\n");
    }
  }
  {
    const unsigned long long* g = &h[ninst * 32 + 16];
    static const char* cl[3] = {"<=8", "<=64", ">64"};
    fprintf(stderr, "[hfsem gemm shapes] (all instances; m x n x k classes)\n");
    for (int key = 0; key < 27; ++key)
      if (g[2 * key + 1])
        fprintf(stderr, "  m%-4s n%-4s k%-4s %10.3f ms %7llu ops %8.0f ns/op\n", cl[key / 9], cl[(key / 3) % 3],
                cl[key % 3], g[2 * key] * 1e-6, g[2 * key + 1], (double)g[2 * key] / g[2 * key + 1]);
  }
  cudaMemset(d_prof.p, 0, d_prof.n * sizeof(unsigned long long));
}

// Critical-path view of one program run, for the instance whose run took
// longest: per wave the CTA with the most busy time decides, and the type
// of its longest op takes the wave's time.
void hfsem_factor_s::report_waves(const char* what) {
  if (!d_wprof.p) return;
  const int rec = 1 + 3 * ncl;
  std::vector<unsigned long long> h(d_wprof.n);
  cudaMemcpy(h.data(), d_wprof.p, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  int worst = 0;
  double wworst = -1;
  for (size_t c = 0; c < hidev.size(); ++c) {
    const int nw = hidev[c].nfw;
    double wall = 0;
    for (int w = 0; w < nw; ++w) wall += h[((size_t)c * wstride + w) * rec];
    if (wall > wworst) {
      wworst = wall;
      worst = (int)c;
    }
  }
  const hf::HPlan& P = plans[worst]->plan;
  const std::vector<hf::HOp>& prog = P.fac;
  const int nw = hidev[worst].nfw;
  static const char* names[16] = {"?", "GEMM", "GETRF_INV", "TRMM_L", "TRMM_R", "APPEND",
                                  "TRUNC", "ZERO", "AXPY", "?", "?", "?", "?", "?", "?", "?"};
  double wall = 0, crit = 0, sumbusy = 0, bytype[16] = {0}, ntype[16] = {0};
  std::map<std::string, std::pair<double, int>> shapes;
  for (int w = 0; w < nw; ++w) {
    const unsigned long long* q = &h[((size_t)worst * wstride + w) * rec];
    wall += q[0];
    int cm = 0;
    for (int k = 0; k < ncl; ++k) {
      sumbusy += q[1 + 3 * k];
      if (q[1 + 3 * k] > q[1 + 3 * cm]) cm = k;
    }
    crit += q[1 + 3 * cm];
    const size_t oi = (size_t)q[3 + 3 * cm];
    const hf::HOp& o = prog[std::min(oi, prog.size() - 1)];
    bytype[o.type & 15] += q[1 + 3 * cm];
    ntype[o.type & 15] += 1;
    char key[96];
    snprintf(key, sizeof(key), "%-9s C %4dx%-4d A.c %4d  wave ops %4d", names[o.type & 15], o.C.r,
             o.C.c, o.A.c, P.fac_waves[w + 1] - P.fac_waves[w]);
    auto& e = shapes[key];
    e.first += q[1 + 3 * cm];
    e.second += 1;
  }
  fprintf(stderr, "[hfsem waves] %s (instance %d): %d waves  wall %.3f ms  max-busy %.3f ms  mean CTA busy %.3f ms\n",
          what, worst, nw, wall * 1e-6, crit * 1e-6, sumbusy * 1e-6 / ncl);
  for (int t = 0; t < 16; ++t)
    if (ntype[t] > 0)
      fprintf(stderr, "  waves led by %-10s %6.0f  %.3f ms\n", names[t], ntype[t], bytype[t] * 1e-6);
  std::vector<std::pair<double, std::string>> top;
  for (auto& kv : shapes) top.push_back({kv.second.first, kv.first + "  x" + std::to_string(kv.second.second)});
  std::sort(top.rbegin(), top.rend());
  for (size_t t = 0; t < top.size() && t < 12; ++t)
    fprintf(stderr, "    %8.3f ms  %s\n", top[t].first * 1e-6, top[t].second.c_str());
}

void hfsem_factor_s::run_prog() {
  if (!d_prof.p && getenv("HFSEM_PROFILE")) {
    hf::AllocStream plain(reinterpret_cast<cudaStream_t>(-1));
    d_prof.alloc((size_t)nfi * 32 + 16 + 64);
    cudaMemset(d_prof.p, 0, d_prof.n * sizeof(unsigned long long));
  }
  if (!d_flops.p) {
    d_flops.alloc((size_t)nfi * std::max(ncl, hf::kCluster) * 2);
    cudaMemsetAsync(d_flops.p, 0, d_flops.n * sizeof(double), sys->st);
  }
  const void* fn = tsize == sizeof(float) ? (const void*)hf::k_hprog<float> : (const void*)hf::k_hprog<double>;
  if (ncl > hf::kCluster && !hf::wide_clusters_fit(fn, smem, ncl)) ncl = hf::kCluster;
  if (!d_tcdbg.p && precision == HFSEM_PREC_MIXED_TC) {
    d_tcdbg.alloc(8);
    HF_CHECK(cudaMemsetAsync(d_tcdbg.p, 0, 8 * sizeof(unsigned long long), sys->st));
  }
  const char* pe = getenv("HFSEM_PROFILE");
  if (!d_wprof.p && pe && atoi(pe) >= 2) {
    hf::AllocStream plain(reinterpret_cast<cudaStream_t>(-1));
    int nwmax = 1;
    for (auto& H : hidev) nwmax = std::max(nwmax, H.nfw);
    wstride = nwmax;
    d_wprof.alloc((size_t)nwmax * hidev.size() * (1 + 3 * ncl));
  }
  if (d_wprof.p) cudaMemsetAsync(d_wprof.p, 0, d_wprof.n * sizeof(unsigned long long), sys->st);
  hf::HProgArgs a{d_hi.p, d_waves.p, d_ops.p, d_slots.p, d_ranks.p, d_err.p, tol, d_prof.p, d_flops.p,
                  d_wprof.p, wstride, (long long)(smem / tsize) - 8, nfi,
                  precision == HFSEM_PREC_MIXED_TC ? 1 : 0, d_tcdbg.p, ncl, leaf32};
  hf::Tick tk(sys->st, "hlu_factor");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nfi * ncl));
  cfg.blockDim = dim3(hf::kHThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = sys->st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ncl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (getenv("HFSEM_PROFILE")) {
    // diagnostic: how many clusters of 8 and of 16 CTAs fit at once
    cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int cs : {8, 16}) {
      cudaLaunchConfig_t c2 = cfg;
      cudaLaunchAttribute a2[1];
      a2[0].id = cudaLaunchAttributeClusterDimension;
      a2[0].val.clusterDim.x = cs;
      a2[0].val.clusterDim.y = 1;
      a2[0].val.clusterDim.z = 1;
      c2.attrs = a2;
      c2.numAttrs = 1;
      c2.gridDim = dim3(cs * 16);
      int nc = -1;
      cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, fn, &c2);
      fprintf(stderr, "[hfsem] max active clusters of %d CTAs (smem %zu): %d (%s)\n", cs, smem, nc,
              cudaGetErrorString(e));
    }
    cudaGetLastError();
  }
  if (tsize == sizeof(float))
    HF_CHECK(cudaLaunchKernelEx(&cfg, hf::k_hprog<float>, a, reinterpret_cast<float*>(d_arena.p)));
  else
    HF_CHECK(cudaLaunchKernelEx(&cfg, hf::k_hprog<double>, a, reinterpret_cast<double*>(d_arena.p)));
  HF_LAUNCH_CHECK();
}

void hfsem_factor_s::run_pack() {
  // algorithmic bytes: every packed column read from the arena and written
  hf::Tick tk(sys->st, "solve_pack", 2.0 * (double)d_pack.n);
  // a warp per job column, about four jobs per warp: enough warps in flight
  // to keep the copy memory-bound for one large instance as for many small
  int maxjob = 1;
  for (const auto& H : hidev) maxjob = std::max(maxjob, H.njob);
  dim3 g((unsigned)std::min(8192, std::max(1, (maxjob + 31) / 32)), nfi);
  if (tsize == sizeof(float))
    hf::k_solve_pack<float><<<g, 256, 0, sys->st>>>(d_hi.p, d_jobs.p, reinterpret_cast<const float*>(d_arena.p),
                                                    d_ranks.p, reinterpret_cast<float*>(d_pack.p), d_meta.p, sol_slot,
                                                    d_err.p);
  else
    hf::k_solve_pack<double><<<g, 256, 0, sys->st>>>(d_hi.p, d_jobs.p, reinterpret_cast<const double*>(d_arena.p),
                                                     d_ranks.p, reinterpret_cast<double*>(d_pack.p), d_meta.p, sol_slot,
                                                     d_err.p);
  HF_LAUNCH_CHECK();
}

void hfsem_factor_s::run_leaf_solve(int nrhs) {
  const char* pe = getenv("HFSEM_PROFILE");
  if (!d_sprof.p && pe && atoi(pe) >= 2) {
    hf::AllocStream plain(reinterpret_cast<cudaStream_t>(-1));
    d_sprof.alloc(8);
    cudaMemset(d_sprof.p, 0, 8 * sizeof(unsigned long long));
  }
  hf::Tick tk(sys->st, "hlu_solve");
  cudaLaunchConfig_t cfg = {};
  // a few instances with several chunks of right-hand sides: the chunks are
  // split over clusters (at most ~15 clusters of 8 fit the device at once)
  const int nchunk = (nrhs + (tsize == sizeof(float) ? hf::solve_w<float>() : hf::solve_w<double>()) - 1) /
                     (tsize == sizeof(float) ? hf::solve_w<float>() : hf::solve_w<double>());
  const int nsplit = std::max(1, std::min(nchunk, 15 / std::max(nfi, 1)));
  cfg.gridDim = dim3((unsigned)(nfi * nsplit * hf::kCluster));
  cfg.blockDim = dim3(hf::kHThreads);
  cfg.dynamicSmemBytes = sol_smem;
  cfg.stream = sys->st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = hf::kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (tsize == sizeof(float))
    HF_CHECK(cudaLaunchKernelEx(&cfg, hf::k_hsolve_cl<float>, (const hf::HInstDev*)d_hi.p,
                                (const hf::StepInfo*)d_steps.p, (const hf::StepCta*)d_step_cta.p,
                                (const float*)d_pack.p, (const int4*)d_meta.p,
                                reinterpret_cast<float*>(d_arena.p), nrhs, sol_jmax, sol_slot, sol_wcols,
                                d_err.p, d_flops.p, d_sprof.p, sys->gate, nsplit));
  else
    HF_CHECK(cudaLaunchKernelEx(&cfg, hf::k_hsolve_cl<double>, (const hf::HInstDev*)d_hi.p,
                                (const hf::StepInfo*)d_steps.p, (const hf::StepCta*)d_step_cta.p,
                                (const double*)d_pack.p, (const int4*)d_meta.p,
                                reinterpret_cast<double*>(d_arena.p), nrhs, sol_jmax, sol_slot, sol_wcols,
                                d_err.p, d_flops.p, d_sprof.p, sys->gate, nsplit));
  HF_LAUNCH_CHECK();
  if (d_sprof.p) {
    unsigned long long h[8];
    cudaMemcpy(h, d_sprof.p, sizeof(h), cudaMemcpyDeviceToHost);
    static const char* nm[7] = {"wait", "gather", "barrier1", "inverse", "barrier2", "scatter", "barrier3"};
    fprintf(stderr, "[hfsem leaf solve] instance 0, CTA 0 (ms):");
    for (int k = 0; k < 7; ++k) fprintf(stderr, " %s %.3f", nm[k], h[k] * 1e-6);
    fprintf(stderr, "\n");
    cudaMemset(d_sprof.p, 0, sizeof(h));
  }
}

void hfsem_factor_s::apply(int nrhs, const double* r_em, double* y_em) {
  if (build_only) throw hf::Error(HFSEM_ERR_INVALID_ARG, "factor was built with build_only");
  if (nrhs > 64) throw hf::Error(HFSEM_ERR_INVALID_ARG, "nrhs > 64");
  if (!parts.empty()) {
    // each part writes the solutions of its own instances
    for (auto& q : parts) q->apply(nrhs, r_em, y_em);
    return;
  }
  if (!d_flops.p) {
    d_flops.alloc((size_t)nfi * std::max(ncl, hf::kCluster) * 2);
    cudaMemsetAsync(d_flops.p, 0, d_flops.n * sizeof(double), sys->st);
  }
  int maxnd = 1;
  for (int i : insts) maxnd = std::max(maxnd, sys->ih[i].Nd);
  dim3 g(std::min(1024, (maxnd * nrhs + 255) / 256), nfi);
  if (tsize == sizeof(float)) {
    float* ar = reinterpret_cast<float*>(d_arena.p);
    hf::k_hsolve_in<float><<<g, 256, 0, sys->st>>>(d_hi.p, sys->d_inst.p, r_em, d_D.p, ar, d_ranks.p, nrhs,
                                                      sys->gate);
    HF_LAUNCH_CHECK();
    run_leaf_solve(nrhs);
    hf::k_hsolve_out<float><<<g, 256, 0, sys->st>>>(d_hi.p, sys->d_inst.p, d_D.p, ar, y_em, nrhs, sys->gate);
  } else {
    double* ar = reinterpret_cast<double*>(d_arena.p);
    hf::k_hsolve_in<double><<<g, 256, 0, sys->st>>>(d_hi.p, sys->d_inst.p, r_em, d_D.p, ar, d_ranks.p, nrhs,
                                                      sys->gate);
    HF_LAUNCH_CHECK();
    run_leaf_solve(nrhs);
    hf::k_hsolve_out<double><<<g, 256, 0, sys->st>>>(d_hi.p, sys->d_inst.p, d_D.p, ar, y_em, nrhs, sys->gate);
  }
  HF_LAUNCH_CHECK();
}

namespace hf {
}  // namespace hf

int hfsem_factor_s::device_status() {
  if (!parts.empty()) {
    int worst = HFSEM_OK;
    for (auto& q : parts) {
      int e = q->device_status();
      if (e != HFSEM_OK) worst = e;
    }
    return worst;
  }
  std::vector<int> err(nfi);
  HF_CHECK(cudaMemcpyAsync(err.data(), d_err.p, err.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  HF_CHECK(cudaStreamSynchronize(st));
  for (int e : err)
    if (e == 2) return HFSEM_ERR_TIMEOUT;
  return HFSEM_OK;
}

namespace hf {

void rebind_stream(hfsem_system* s, hfsem_factor* f, cudaStream_t st) {
  s->st = st;
  if (s->hop) s->hop->st = st;
  if (!f) return;
  f->st = st;
  for (auto& q : f->parts) q->st = st;
}

size_t factor_bytes(const hfsem_factor* f) {
  auto b = [](const auto& d) { return d.n * sizeof(*d.p); };
  size_t t = b(f->d_hi) + b(f->d_waves) + b(f->d_ops) + b(f->d_slots) + b(f->d_dense) +
             b(f->d_pairs) + b(f->d_ptask) + b(f->d_gmax) + b(f->d_lrt) + b(f->d_steps) +
             b(f->d_step_cta) + b(f->d_jobs) + b(f->d_pack) + b(f->d_meta) + b(f->d_sprof) +
             b(f->d_ranks) + b(f->d_err) + b(f->d_D) + b(f->d_arena) + b(f->d_prof) +
             b(f->d_flops) + b(f->d_wprof) + b(f->d_tcdbg) + b(f->d_hrow) + b(f->d_hitem) +
             b(f->d_hslot);
  for (auto& q : f->parts) t += factor_bytes(q.get());
  return t;
}

Precond* precond_of(hfsem_system* s, hfsem_factor* f) {
  if (!f) return nullptr;
  if (f->sys != s) throw Error(HFSEM_ERR_INVALID_ARG, "factor belongs to another system");
  if (f->build_only) throw Error(HFSEM_ERR_INVALID_ARG, "factor was built with build_only");
  return f;
}
}  // namespace hf

using namespace hf;

extern "C" {

int hfsem_hlu_factor(hfsem_system* sys, const hfsem_hopts* opts, hfsem_factor** out) {
  try {
    if (!sys || !opts || !out) throw Error(HFSEM_ERR_INVALID_ARG, "NULL argument");
    *out = factor(sys, *opts);
    return HFSEM_OK;
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

int hfsem_hmatrix_dense(const hfsem_factor* fac, int32_t inst, double* out) {
  try {
    if (!fac || !out || inst < 0 || inst >= fac->sys->n_inst)
      throw Error(HFSEM_ERR_INVALID_ARG, "bad arguments");
    if (!fac->build_only) throw Error(HFSEM_ERR_INVALID_ARG, "only for factors built with build_only");
    hfsem_system* s = fac->sys;
    const InstHost& I = s->ih[inst];
    // the part holding this instance, and its index there
    const hfsem_factor* part = fac;
    for (auto& q : fac->parts)
      if (std::find(q->insts.begin(), q->insts.end(), inst) != q->insts.end()) part = q.get();
    fac = part;
    inst = (int32_t)(std::find(fac->insts.begin(), fac->insts.end(), inst) - fac->insts.begin());
    size_t nn = (size_t)I.Nd * I.Nd;
    DevBuf<double> em, pp;
    em.alloc(std::max<size_t>(nn, 1));
    pp.alloc(std::max<size_t>(nn, 1));
    HF_CHECK(cudaMemsetAsync(em.p, 0, nn * sizeof(double), s->st));
    const HInstDev* hsel = fac->d_hi.p + inst;
    int nb = fac->hidev[inst].ndense + 2 * fac->hidev[inst].npairs;
    if (fac->tsize == sizeof(float))
      k_expand<float><<<std::max(1, std::min(nb, 4096)), 256, 0, s->st>>>(
          hsel, fac->d_dense.p, fac->d_pairs.p, fac->d_slots.p, fac->d_ranks.p, fac->d_D.p,
          reinterpret_cast<const float*>(fac->d_arena.p), em.p, I.Nd);
    else
      k_expand<double><<<std::max(1, std::min(nb, 4096)), 256, 0, s->st>>>(
          hsel, fac->d_dense.p, fac->d_pairs.p, fac->d_slots.p, fac->d_ranks.p, fac->d_D.p,
          reinterpret_cast<const double*>(fac->d_arena.p), em.p, I.Nd);
    HF_LAUNCH_CHECK();
    k_perm_mat<<<1024, 256, 0, s->st>>>(em.p, pp.p, I.Nd, I.N, I.P);
    HF_LAUNCH_CHECK();
    HF_CHECK(cudaMemcpyAsync(out, pp.p, nn * sizeof(double),
                             is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->st));
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

int hfsem_hlu_solve(hfsem_system* sys, hfsem_factor* fac, const hfsem_rhs* rhs, double* X) {
  try {
    if (!sys || !fac || !rhs || !X) throw Error(HFSEM_ERR_INVALID_ARG, "NULL argument");
    if (fac->sys != sys) throw Error(HFSEM_ERR_INVALID_ARG, "factor belongs to another system");
    if (fac->build_only) throw Error(HFSEM_ERR_INVALID_ARG, "factor was built with build_only");
    const int nrhs = rhs[0].nrhs;
    if (nrhs < 1 || nrhs > 64) throw Error(HFSEM_ERR_INVALID_ARG, "nrhs must be in [1, 64]");
    AllocStream as(sys->st);
    ensure_work(sys, nrhs);
    const size_t cnt = (size_t)sys->total_nd * nrhs;
    DevBuf<double> g, y;
    g.alloc(std::max<size_t>(cnt, 1));
    y.alloc(std::max<size_t>(cnt, 1));
    load_vector_em(sys, rhs, 1, g.p);          // G with the boundary lifting
    fac->apply(nrhs, g.p, y.p);                // (L_H U_H)^-1 G
    perm_to_paper(sys, nrhs, y.p, sys->w_y.p);
    HF_CHECK(cudaMemcpyAsync(X, sys->w_y.p, cnt * sizeof(double),
                             is_device_ptr(X) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             sys->st));
    HF_CHECK(cudaStreamSynchronize(sys->st));
    if (fac->device_status() == HFSEM_ERR_TIMEOUT)
      throw Error(HFSEM_ERR_TIMEOUT, "an H-solve copy did not complete within its wait limit");
    return HFSEM_OK;
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

int hfsem_precond_apply(hfsem_factor* fac, int32_t nrhs, const double* r, double* y) {
  try {
    if (!fac || !r || !y || nrhs < 1 || nrhs > 64) throw Error(HFSEM_ERR_INVALID_ARG, "bad arguments");
    hfsem_system* s = fac->sys;
    AllocStream as(s->st);
    ensure_work(s, nrhs);
    size_t cnt = (size_t)s->total_nd * nrhs;
    DevBuf<double> a, b;
    a.alloc(cnt);
    b.alloc(cnt);
    HF_CHECK(cudaMemcpyAsync(s->w_y.p, r, cnt * sizeof(double),
                             is_device_ptr(r) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
    perm_to_elem(s, nrhs, s->w_y.p, a.p);
    fac->apply(nrhs, a.p, b.p);
    perm_to_paper(s, nrhs, b.p, s->w_y.p);
    HF_CHECK(cudaMemcpyAsync(y, s->w_y.p, cnt * sizeof(double),
                             is_device_ptr(y) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->st));
    HF_CHECK(cudaStreamSynchronize(s->st));
    if (fac->device_status() == HFSEM_ERR_TIMEOUT)
      throw Error(HFSEM_ERR_TIMEOUT, "an H-solve copy did not complete within its wait limit");
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

void hfsem_factor_free(hfsem_factor* f) {
  if (!f) return;
  cudaStreamSynchronize(f->st);
  f->collect_flops();
  delete f;
}

}  // extern "C"

// The tensor-core tile check (hfsem.h).
extern "C" int hfsem_tc_tile_check(int32_t N, int32_t K, int32_t reps, double* max_rel_err) {
  using namespace hf;
  try {
    if (N < 16 || N > 128 || (N & 15) || K < 64 || K > 128 || (K & 15) || reps < 1 || reps > 8 ||
        !max_rel_err)
      throw Error(HFSEM_ERR_INVALID_ARG, "hfsem_tc_tile_check: bad arguments");
    const size_t nab = (size_t)128 * K + (size_t)K * N;
    const size_t na = nab + (size_t)kCluster * 128 * N;
    std::vector<float> h(na, 0.f);
    for (size_t i = 0; i < nab; ++i) h[i] = (float)(((i * 37) % 101) / 101.0 - 0.5);
    DevBuf<float> d;
    DevBuf<int> de;
    DevBuf<unsigned long long> dd;
    d.alloc(na);
    de.alloc(kCluster);
    dd.alloc(8);
    HF_CHECK(cudaMemcpy(d.p, h.data(), na * sizeof(float), cudaMemcpyHostToDevice));
    HF_CHECK(cudaMemset(de.p, 0, kCluster * sizeof(int)));
    HF_CHECK(cudaMemset(dd.p, 0, 8 * sizeof(unsigned long long)));
    const int smem = 160 * 1024;   // heads and tails of the operands, (128 + N) x K bf16 each
    allow_dyn_smem((const void*)k_tc_tile_check, smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCluster);
    cfg.blockDim = dim3(kHThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HF_CHECK(cudaLaunchKernelEx(&cfg, k_tc_tile_check, d.p, (int)N, (int)K, (int)reps, de.p, dd.p));
    HF_CHECK(cudaDeviceSynchronize());
    int herr[kCluster] = {0};
    HF_CHECK(cudaMemcpy(h.data(), d.p, na * sizeof(float), cudaMemcpyDeviceToHost));
    HF_CHECK(cudaMemcpy(herr, de.p, sizeof(herr), cudaMemcpyDeviceToHost));
    for (int r = 0; r < kCluster; ++r)
      if (herr[r]) throw Error(HFSEM_ERR_TIMEOUT, "hfsem_tc_tile_check: a tensor-core product did not complete within its wait limit");
    // |C - A B| relative to sum_k |a_mk| |b_kn|, per entry, against FP64
    double mx = 0.0;
    for (int r = 0; r < kCluster; ++r)
      for (int n = 0; n < N; ++n)
        for (int m = 0; m < 128; ++m) {
          double ref = 0.0, mag = 0.0;
          for (int k = 0; k < K; ++k) {
            const double a = h[(size_t)m + (size_t)k * 128], b = h[(size_t)128 * K + k + (size_t)n * K];
            ref += a * b;
            mag += std::fabs(a * b);
          }
          const double got = h[nab + (size_t)r * 128 * N + m + (size_t)n * 128];
          if (mag > 0.0) mx = std::max(mx, std::fabs(ref - got) / mag);
        }
    *max_rel_err = mx;
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
