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
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <array>
#include <map>
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
};

constexpr int kCluster = 8;   // CTAs (one thread-block cluster) per instance

struct HInstDev {
  long long arena;   // offset of the instance arena (elements)
  long long rk0;     // offset into the rank array
  long long slot0;   // offset into the slot table
  long long dense0;  // offset into the dense-block table
  long long pair0;   // offset into the pair table
  long long ops0, sops0;
  int nops, nsops, ndense, npairs, n_slots;
  long long ws_off, rhs_off, ws_size;
  long long fw0, sw0;   // offsets into the wave table (factor, solve)
  int nfw, nsw;         // number of waves
  long long d_off;   // scaling D (FP64) offset
  int sys_inst;      // index into the system's instances
  int R;
};

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
  if (p < P) {
    t[0] = Term{e, p, -(2.0 * p + 1.0) * (2.0 / h[e])};
    return 1;
  }
  int j = e + 1;   // hat at node j: right hat of element j-1, left hat of element j
  t[0] = Term{j - 1, 0, 1.0 / h[j - 1]};
  t[1] = Term{j, 0, -1.0 / h[j]};
  return 2;
}

// Mb_ef[m][n] for f <= e
__device__ __forceinline__ double mb_entry(const InstDev& I, const double* arena, int e, int f,
                                           int m, int n) {
  const int P = I.P;
  if (I.kind == kDense)
    return arena[I.o_M + ((long long)e * (e + 1) / 2 + f) * P * P + m * P + n];
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

template <class T>
__global__ void k_nearfield(const HInstDev* __restrict__ hi, const InstDev* __restrict__ inst,
                            const double* arena, const DenseDev* __restrict__ dens,
                            const double* D, T* har) {
  const HInstDev H = hi[blockIdx.y];
  const InstDev I = inst[H.sys_inst];
  T* ar = har + H.arena;
  const double* Dv = D + H.d_off;
  for (int b = blockIdx.x; b < H.ndense; b += gridDim.x) {
    const DenseDev d = dens[H.dense0 + b];
    for (int t = threadIdx.x; t < d.m * d.n; t += blockDim.x) {
      int i = t % d.m, j = t / d.m;
      int r = d.d0r + i, c = d.d0c + j;
      ar[d.off + t] = (T)(Dv[r] * a_entry(I, arena, r, c) * Dv[c]);
    }
  }
}

// Taylor low-rank factors of every admissible pair.  CTA per pair.
template <class T>
__global__ void k_lowrank(const HInstDev* __restrict__ hi, const InstDev* __restrict__ inst,
                          const double* arena, const double* __restrict__ gl,
                          const LRPairDev* __restrict__ pairs, const SlotDev* __restrict__ slots,
                          const double* D, T* har, int* ranks) {
  __shared__ double sQ[kMaxP * 32];     // moments of the current element, P x R
  __shared__ double sX[64], sW[64];
  const HInstDev H = hi[blockIdx.y];
  const InstDev I = inst[H.sys_inst];
  if ((int)blockIdx.x >= H.npairs) return;
  const LRPairDev pr = pairs[H.pair0 + blockIdx.x];
  const int P = I.P, R = H.R;
  const double* h = arena + I.o_h;
  const double* dl = arena + I.o_dl;
  const double* dr = arena + I.o_dr;
  auto ndiff = [&](int a, int b) {   // x_a - x_b, a >= b
    return (dl[a] <= dr[b]) ? dl[a] - dl[b] : dr[b] - dr[a];
  };
  const double r_s = 0.5 * ndiff(pr.shi, pr.slo);
  const double r_t = 0.5 * ndiff(pr.thi, pr.tlo);
  const bool sexp = (r_s <= r_t);
  const double ex = 1.0 - I.alpha;
  const int nq = min((P + R) / 2 + 13, kMaxGL);
  const double* X = gl + gl_off(nq);
  const double* Wt = X + nq;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    sX[q] = X[q];
    sW[q] = Wt[q];
  }
  __syncthreads();
  const SlotDev lo = slots[H.slot0 + pr.lower_slot];
  const SlotDev up = slots[H.slot0 + pr.upper_slot];
  T* ar = har + H.arena;
  const double* Dv = D + H.d_off;
  // expansion functions at the Gauss points of element e, one pow per point:
  // sF[q*R + nu] = f_nu(x_q); side 0 varies t (tau), side 1 varies s (sigma)
  __shared__ double sF[64 * 32];
  __shared__ double sL[64 * kMaxP];
  __shared__ double sPrev[32];
  auto fill = [&](int side, int e) {
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      double xq = sX[q];
      double loc = 0.5 * h[e] * (1.0 + xq);
      double* F = sF + q * R;
      bool singular = (side == 0) == sexp;
      if (singular) {
        double d, rr, sg;
        if (sexp) {            // h_nu(t) = (-1)^nu c_nu r_s^nu (t - s0)^(1-alpha-nu)
          d = ndiff(e, pr.shi) + loc + r_s;
          rr = r_s;
          sg = -1.0;
        } else {               // h~_nu(s) = c_nu r_t^nu (t0 - s)^(1-alpha-nu)
          d = r_t + ndiff(pr.tlo, e + 1) + 0.5 * h[e] * (1.0 - xq);
          rr = r_t;
          sg = 1.0;
        }
        double f = pow(d, ex);
        F[0] = f;
        for (int nu = 1; nu < R; ++nu) {
          f *= sg * (2.0 - I.alpha - nu) / nu * rr / d;
          F[nu] = f;
        }
      } else {
        double y = sexp ? (ndiff(e, pr.slo) + loc - r_s) / r_s     // (s - s0)/r_s
                        : (ndiff(e, pr.tlo) + loc - r_t) / r_t;    // (t - t0)/r_t
        double f = 1.0;
        for (int nu = 0; nu < R; ++nu) {
          F[nu] = f;
          f *= y;
        }
      }
      double* Lq = sL + q * kMaxP;
      double l0 = 1.0, l1 = xq;
      Lq[0] = 1.0;
      if (P > 1) Lq[1] = xq;
      for (int k = 1; k + 1 < P; ++k) {
        double l2 = ((2 * k + 1) * xq * l1 - k * l0) / (k + 1);
        Lq[k + 1] = l2;
        l0 = l1;
        l1 = l2;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < P * R; t += blockDim.x) {
      int m = t / R, nu = t % R;
      double acc = 0.0;
      for (int q = 0; q < nq; ++q) acc += sW[q] * sL[q * kMaxP + m] * sF[q * R + nu];
      sQ[m * R + nu] = 0.5 * h[e] * acc;
    }
    __syncthreads();
  };
  // Two passes over the elements: the first finds, per term nu, the largest
  // |Q| and |W| row entries (after the D scaling), the second writes the
  // factors with every rank-one term balanced (|U_nu| and |V_nu| scaled to
  // equal maxima).  The products are unchanged; the balance keeps each factor
  // inside the FP32 range on meshes whose element sizes span 10^80.
  __shared__ unsigned long long smax[2][32];
  __shared__ double sscale[32];
  for (int t = threadIdx.x; t < 64; t += blockDim.x) smax[t / 32][t % 32] = 0ULL;
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      for (int nu = threadIdx.x; nu < R; nu += blockDim.x) {
        double mq = __longlong_as_double((long long)smax[0][nu]);
        double mw = __longlong_as_double((long long)smax[1][nu]);
        double sc = (mq > 0.0 && mw > 0.0) ? sqrt(mw) / sqrt(mq) : 1.0;   // Q *= s, W /= s
        sscale[nu] = (isfinite(sc) && sc > 0.0) ? sc : 1.0;
      }
      __syncthreads();
    }
    for (int side = 0; side < 2; ++side) {
      int e0 = side == 0 ? pr.te0 : pr.se0, e1 = side == 0 ? pr.te1 : pr.se1;
      int d0 = side == 0 ? pr.td0 : pr.sd0;
      double scale_side = (side == 0) ? I.g0 : 1.0;   // gamma0 sits with Q
      int elast = (e1 < I.N) ? e1 : e1 - 1;            // element e1 only feeds the hat at node e1
      for (int e = e0; e <= elast; ++e) {
        fill(side, e);
        // rows: the hat at node e (from elements e-1 and e) when e > e0, the
        // bubbles of e when e < e1
        int nb = (e < e1) ? P - 1 : 0;
        int nh = (e > e0) ? 1 : 0;
        for (int t = threadIdx.x; t < (nb + nh) * R; t += blockDim.x) {
          int k = t / R, nu = t % R;
          double v;
          int dof;
          if (k < nh) {
            v = sPrev[nu] / h[e - 1] - sQ[nu] / h[e];
            dof = e * P - 1;
          } else {
            int p = k - nh + 1;
            v = -(2.0 * p + 1.0) * (2.0 / h[e]) * sQ[p * R + nu];
            dof = e * P + p - 1;
          }
          v *= scale_side * Dv[dof];
          if (pass == 0) {
            atomicMax(&smax[side][nu], (unsigned long long)__double_as_longlong(fabs(v)));
            continue;
          }
          int row = dof - d0;
          if (side == 0) {
            v *= sscale[nu];
            // Q row: lower U = theta D Q, upper V = (1-theta) D Q
            ar[lo.off + row + (long long)nu * lo.m] = (T)(I.theta * v);
            ar[up.off + (long long)up.m * up.kcap + row + (long long)nu * up.n] =
                (T)((1.0 - I.theta) * v);
          } else {
            v /= sscale[nu];
            // W row: lower V = D W, upper U = D W
            ar[lo.off + (long long)lo.m * lo.kcap + row + (long long)nu * lo.n] = (T)v;
            ar[up.off + row + (long long)nu * up.m] = (T)v;
          }
        }
        __syncthreads();
        for (int nu = threadIdx.x; nu < R; nu += blockDim.x) sPrev[nu] = sQ[nu];
        __syncthreads();
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ranks[H.rk0 + pr.lower_slot] = (I.theta != 0.0) ? R : 0;
    ranks[H.rk0 + pr.upper_slot] = (I.theta != 1.0) ? R : 0;
  }
}

// ---------------------------------------------------------------------------
// interpreter
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dimv(int d, const int* rk) { return d >= 0 ? d : rk[-1 - d]; }
__device__ __forceinline__ long long vidx(const View& v, int i, int j) {
  return v.tr ? v.off + j + (long long)i * v.ld : v.off + i + (long long)j * v.ld;
}

template <class T>
struct HCtx {
  T* ar;
  int* rk;
  const SlotDev* sl;
  T* ws;
  T* sm;
  double tol;
  int* err;
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
            int kk = t >> 7, ii = t & 127;
            int gi = m0 + ii, gj = n0 + ii, gk = k0 + kk;
            ra[q] = (gi < m && gk < k) ? ar[vidx(o.A, gi, gk)] : (T)0;
            rb[q] = (gj < n && gk < k) ? ar[vidx(o.B, gk, gj)] : (T)0;
          }
        };
        fetch(0);
        for (int k0 = 0; k0 < k; k0 += 8) {
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int t = tid + q * 256;
            As[t] = ra[q];
            Bs[t] = rb[q];
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
#pragma unroll
        for (int p = 0; p < 8; ++p)
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            int gi = m0 + (p < 4 ? ty * 4 + p : 64 + ty * 4 + p - 4);
            int gj = n0 + (q < 4 ? tx * 4 + q : 64 + tx * 4 + q - 4);
            if (gi < m && gj < n) {
              long long ci = vidx(o.C, gi, gj);
              ar[ci] = (beta == (T)0 ? (T)0 : beta * ar[ci]) + alpha * acc[p][q];
            }
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
  for (int t = tid; t < n * n; t += blockDim.x) As[t] = ar[vidx(o.A, t % n, t / n)];
  const int tx = tid & 7, ty = tid >> 3;
  for (int c0 = 0; c0 < cc; c0 += 32) {
    const int cp = min(32, cc - c0);
    __syncthreads();
    for (int t = tid; t < n * cp; t += blockDim.x) {
      int i = t % n, j = t / n;
      Pn[i * 33 + j] = ar[vidx(o.C, i, c0 + j)];
    }
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
  T* As = c.sm;            // n x n, [k n + j]
  T* Pn = c.sm + n * n;    // 32 x n, [i + k * 32]
  const int tid = threadIdx.x;
  for (int t = tid; t < n * n; t += blockDim.x) As[(t % n) * n + t / n] = ar[vidx(o.A, t % n, t / n)];
  const int tx = tid & 31, ty = tid >> 5;
  for (int r0 = 0; r0 < m; r0 += 32) {
    const int rp = min(32, m - r0);
    __syncthreads();
    for (int t = tid; t < rp * n; t += blockDim.x) Pn[(t % rp) + (t / rp) * 32] = ar[vidx(o.C, r0 + t % rp, t / rp)];
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
      for (int q = 0; q < 4; ++q) b[q] = (tx + 32 * q < n) ? As[k * n + tx + 32 * q] : (T)0;
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
template <class T>
__device__ void op_getrf_inv(const HOp& o, HCtx<T>& c) {
  const int n = o.C.r;
  if (n <= 0) return;
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
template <class T>
__device__ void house_qr(T* A, int m, int K, T* tau, T* red) {
  const int kr = min(m, K);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < kr; ++j) {
    T part = 0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) part += A[i + (long long)j * m] * A[i + (long long)j * m];
    T s2 = block_sum<T>(part, red);
    T x0 = A[j + (long long)j * m];
    T s = sqrt(s2);
    T alpha = (x0 >= (T)0) ? -s : s;
    T v0 = x0 - alpha;
    bool trivial = (s == (T)0) || (v0 == (T)0);
    if (!trivial)
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[i + (long long)j * m] /= v0;
    __syncthreads();
    if (threadIdx.x == 0) {
      tau[j] = trivial ? (T)0 : (alpha - x0) / alpha;
      if (!trivial) A[j + (long long)j * m] = alpha;
    }
    __syncthreads();
    T tj = tau[j];
    if (tj != (T)0) {
      for (int l = j + 1 + warp; l < K; l += nw) {
        T w = 0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + (long long)j * m] * A[i + (long long)l * m];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        w = __shfl_sync(0xffffffffu, w, 0);
        w = (w + A[j + (long long)l * m]) * tj;
        if (lane == 0) A[j + (long long)l * m] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) A[i + (long long)l * m] -= w * A[i + (long long)j * m];
      }
    }
    __syncthreads();
  }
}

// Y (m x r, ld ldy) <- Q Y with Q = H_0 ... H_{kr-1} stored in A (m x K)
template <class T>
__device__ void apply_q(const T* A, int m, int K, const T* tau, T* Y, int ldy, int r) {
  const int kr = min(m, K);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
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
    __syncthreads();
  }
}

// Recompress U V^T given as Ut (m x K) and Vt (n x K) in the workspace into
// LR slot `slot`.  U = Q_U R_U, V = Q_V R_V (Householder), then a column-
// pivoted QR of the small core M = R_U R_V^T, M Pi = Q_M R_M, stopped at the
// first pivot below tol |R_M(0,0)| (or at kmax):
//   U V^T ~ (Q_U Q_M[:, :r]) (Q_V Pi R_M[:r, :]^T)^T.
template <class T>
__device__ void trunc_core(HCtx<T>& c, int slot, T* Ut, T* Vt, int K) {
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
  __shared__ int s_p, s_stop;
  __shared__ T s_r0;
  house_qr(Ut, m, K, tauU, red);
  house_qr(Vt, n, K, tauV, red);
  const int ku = min(m, K), kv = min(n, K);
  for (int t = threadIdx.x; t < ku * kv; t += blockDim.x) {
    int i = t % ku, j = t / ku;
    T acc = 0;
    for (int l = max(i, j); l < K; ++l) acc += Ut[i + (long long)l * m] * Vt[j + (long long)l * n];
    M[i + j * K] = acc;
  }
  for (int j = threadIdx.x; j < kv; j += blockDim.x) piv[j] = j;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rmax = min(min(ku, kv), s.kmax);
  int r = 0;
  for (int st = 0; st < rmax; ++st) {
    // exact norms of the remaining parts of the columns
    for (int j = st + threadIdx.x; j < kv; j += blockDim.x) {
      T a = 0;
      for (int i = st; i < ku; ++i) a += M[i + j * K] * M[i + j * K];
      cn[j] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int p = st;
      for (int j = st + 1; j < kv; ++j)
        if (cn[j] > cn[p]) p = j;
      T nrm = sqrt(cn[p]);
      if (st == 0) s_r0 = nrm;
      s_stop = (nrm == (T)0 || (st > 0 && nrm <= (T)c.tol * s_r0)) ? 1 : 0;
      s_p = p;
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    if (p != st) {
      for (int i = threadIdx.x; i < ku; i += blockDim.x) {
        T a = M[i + st * K];
        M[i + st * K] = M[i + p * K];
        M[i + p * K] = a;
      }
      if (threadIdx.x == 0) {
        int a = piv[st];
        piv[st] = piv[p];
        piv[p] = a;
      }
    }
    __syncthreads();
    // Householder on M[st:ku, st] (one warp), stored as in house_qr
    if (warp == 0) {
      T a = 0;
      for (int i = st + lane; i < ku; i += 32) a += M[i + st * K] * M[i + st * K];
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      T x0 = M[st + st * K];
      T sn = sqrt(a);
      T alpha = (x0 >= (T)0) ? -sn : sn;
      T v0 = x0 - alpha;
      bool trivial = (sn == (T)0) || (v0 == (T)0);
      __syncwarp();
      if (!trivial)
        for (int i = st + 1 + lane; i < ku; i += 32) M[i + st * K] /= v0;
      __syncwarp();
      if (lane == 0) {
        tauM[st] = trivial ? (T)0 : (alpha - x0) / alpha;
        if (!trivial) M[st + st * K] = alpha;
      }
    }
    __syncthreads();
    const T tj = tauM[st];
    if (tj != (T)0)
      for (int l = st + 1 + warp; l < kv; l += nw) {
        T w = 0;
        for (int i = st + 1 + lane; i < ku; i += 32) w += M[i + st * K] * M[i + l * K];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        w = __shfl_sync(0xffffffffu, w, 0);
        w = (w + M[st + l * K]) * tj;
        if (lane == 0) M[st + l * K] -= w;
        for (int i = st + 1 + lane; i < ku; i += 32) M[i + l * K] -= w * M[i + st * K];
      }
    __syncthreads();
    r = st + 1;
  }
  // (all threads agree on r: every exit is uniform)
  T* Ud = c.ar + s.off;
  T* Vd = c.ar + s.off + (long long)m * s.kcap;
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
  // U_new = Q_U [Z; 0]
  for (int t = threadIdx.x; t < m * r; t += blockDim.x) {
    int i = t % m, j = t / m;
    Ud[t] = (i < ku) ? Z[i + j * K] : (T)0;
  }
  // V_new = Q_V [Pi R_M[:r,:]^T; 0]: row piv[j] of the core factor is R_M[:, j]
  for (int t = threadIdx.x; t < n * r; t += blockDim.x) Vd[t] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < kv * r; t += blockDim.x) {
    int j = t % kv, i = t / kv;   // R_M[i][j], j >= i
    Vd[piv[j] + (long long)i * n] = (j >= i) ? M[i + j * K] : (T)0;
  }
  __syncthreads();
  apply_q(Ut, m, K, tauU, Ud, m, r);
  apply_q(Vt, n, K, tauV, Vd, n, r);
  if (threadIdx.x == 0) c.rk[slot] = r;
  __syncthreads();
}

template <class T>
__device__ void op_append(const HOp& o, HCtx<T>& c) {
  const int slot = o.slot;
  const SlotDev s = c.sl[slot];
  const int k = dimv(o.A.c, c.rk);
  const int r0 = c.rk[slot];
  __syncthreads();
  if (k <= 0) return;
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
    return;
  }
  const int K = r0 + k;
  T* Ut = c.ws;
  T* Vt = c.ws + (long long)s.m * K;
  const T* Us = ar + s.off;
  const T* Vs = ar + s.off + (long long)s.m * s.kcap;
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
  for (int t = threadIdx.x; t < s.m * K; t += blockDim.x) Ut[t] = Us[t];
  for (int t = threadIdx.x; t < s.n * K; t += blockDim.x) Vt[t] = Vs[t];
  __syncthreads();
  trunc_core(c, slot, Ut, Vt, K);
}

struct HProgArgs {
  const HInstDev* inst;
  const int* waves;
  const HOp* ops;
  const SlotDev* slots;
  int* ranks;
  int* err;
  double tol;
  unsigned long long* prof;   // optional: per instance, 16 op types x (cycles, count)
  double* flops;              // per instance: algorithmic flops of the executed ops
};

// algorithmic flops of one op with its run-time shapes
__device__ double op_flops(const HOp& o, const int* rk, const SlotDev* sl) {
  switch (o.type) {
    case OP_GEMM: {
      double m = dimv(o.C.r, rk), n = dimv(o.C.c, rk), k = dimv(o.A.c, rk);
      return 2.0 * m * n * k;
    }
    case OP_GETRF_INV: {
      double n = o.C.r;
      return (2.0 / 3.0) * n * n * n + (2.0 / 3.0) * n * n * n;
    }
    case OP_TRMM_L: {
      double n = dimv(o.C.r, rk), c = dimv(o.C.c, rk);
      return 2.0 * n * n * c;
    }
    case OP_TRMM_R: {
      double m = dimv(o.C.r, rk), n = dimv(o.C.c, rk);
      return 2.0 * m * n * n;
    }
    case OP_TRUNC: {
      double K = rk[o.slot], m = sl[o.slot].m, n = sl[o.slot].n;
      return 4.0 * (m + n) * K * K + 2.0 * K * K * K;
    }
    default:
      return 0.0;
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

// One thread-block cluster of kCluster CTAs per instance runs the instance's
// op program wave by wave: the ops of a wave are independent and spread
// round-robin over the CTAs, a cluster barrier separates consecutive waves.
template <class T>
__global__ void __launch_bounds__(kHThreads) k_hprog(HProgArgs a, T* har, int which) {
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
  c.tol = a.tol;
  c.err = a.err + cid;
  const HOp* ops = a.ops + (which ? H.sops0 : H.ops0);
  const int* waves = a.waves + (which ? H.sw0 : H.fw0);
  const int nw = which ? H.nsw : H.nfw;
  double fl = 0.0;
  for (int w = 0; w < nw; ++w) {
    const int i1 = waves[w + 1];
    for (int i = waves[w] + (int)crank; i < i1; i += kCluster) {
      const HOp o = ops[i];
      if (threadIdx.x == 0) fl += op_flops(o, c.rk, c.sl);
      unsigned long long t0 = 0;
      if (a.prof && crank == 0 && threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      switch (o.type) {
        case OP_GEMM: op_gemm(o, c); break;
        case OP_GETRF_INV: op_getrf_inv(o, c); break;
        case OP_TRMM_L: op_trmm_l(o, c); break;
        case OP_TRMM_R: op_trmm_r(o, c); break;
        case OP_APPEND: op_append(o, c); break;
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
      __syncthreads();
      if (a.prof && crank == 0 && threadIdx.x == 0) {
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        unsigned long long* pr = a.prof + (size_t)cid * 32 + 2 * (o.type & 15);
        pr[0] += t1 - t0;
        pr[1] += 1ULL;
      }
    }
    cluster_barrier();
  }
  if (threadIdx.x == 0) a.flops[((size_t)cid * kCluster + crank) * 2 + which] += fl;
}

// rhs area <- D r (element-major FP64 -> T); rank slot n_slots <- nrhs
template <class T>
__global__ void k_hsolve_in(const HInstDev* __restrict__ hi, const InstDev* __restrict__ inst,
                            const double* __restrict__ r, const double* D, T* har, int* ranks,
                            int nrhs) {
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
                             const double* D, const T* har, double* y, int nrhs) {
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
  std::vector<SlotDev> slots;
};

}  // namespace hf

struct hfsem_factor_s : public hf::Precond {
  hfsem_system* sys = nullptr;
  cudaStream_t st = nullptr;   // copy of the system's stream (free never touches sys)
  int precision = HFSEM_PREC_MIXED;
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
  hf::DevBuf<int> d_ranks, d_err;
  hf::DevBuf<double> d_D;
  hf::DevBuf<unsigned char> d_arena;
  size_t smem = 0;
  long long total_ops = 0, total_sops = 0;
  hf::DevBuf<unsigned long long> d_prof;   // HFSEM_PROFILE=1: time per op type
  hf::DevBuf<double> d_flops;               // per instance: factor / solve flops
  void report(const char* what);
  void apply(int nrhs, const double* r_em, double* y_em) override;
  void collect_flops();
  void run_prog(int which);
};

namespace hf {

template <class T>
static void set_prog_smem(size_t bytes) {
  HF_CHECK(cudaFuncSetAttribute((const void*)k_hprog<T>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

static size_t prog_smem(const HPlan& p, size_t ts) {
  size_t leaf = (size_t)2 * p.leaf_max * p.leaf_max;
  size_t K = (size_t)std::max(p.kconcat_max, 1);
  size_t trunc = 2 * K + 32 + 2 * K * K + 3 * K + 8;
  size_t trmm = (size_t)p.leaf_max * p.leaf_max + (size_t)std::max(p.leaf_max, 1) * 33;
  size_t gemm = 2 * 16 * 64;
  return std::max(std::max(leaf, trunc), std::max(trmm, gemm)) * ts + 64;
}

static std::string plan_key(const InstHost& I, const PlanOpts& o) {
  std::string k(reinterpret_cast<const char*>(I.h.data()), I.h.size() * sizeof(double));
  char buf[128];
  snprintf(buf, sizeof(buf), "|%d|%d|%.17g|%d|%d|%d|%d", I.N, I.P, o.lambda, o.leaf_elems, o.R,
           o.kmax, o.max_concat);
  return k + buf;
}

static hfsem_factor* factor(hfsem_system* s, const hfsem_hopts& opt) {
  if (opt.R < 1 || opt.R > 32) throw Error(HFSEM_ERR_INVALID_ARG, "R must be in [1, 32]");
  if (!(opt.lambda > 0.0)) throw Error(HFSEM_ERR_INVALID_ARG, "lambda must be > 0");
  if (!(opt.tol_hlu >= 0.0)) throw Error(HFSEM_ERR_INVALID_ARG, "tol_hlu must be >= 0");
  if (opt.precision != HFSEM_PREC_FP64 && opt.precision != HFSEM_PREC_MIXED)
    throw Error(HFSEM_ERR_INVALID_ARG, "unknown precision");
  if (opt.leaf_elems < 0 || opt.kmax < 0) throw Error(HFSEM_ERR_INVALID_ARG, "leaf_elems, kmax >= 0");
  auto* f = new hfsem_factor();
  try {
    f->sys = s;
    f->st = s->st;
    f->precision = opt.precision;
    // FP32 cannot factor the equilibrated H-matrix of meshes whose element
    // sizes span more than ~1e45 (the preconditioner then loses all digits);
    // such batches are factored in FP64 on the GPU
    if (f->precision == HFSEM_PREC_MIXED)
      for (const InstHost& I : s->ih) {
        double hmax = *std::max_element(I.h.begin(), I.h.end());
        double hmin = *std::min_element(I.h.begin(), I.h.end());
        if (hmax > 1e45 * hmin) f->precision = HFSEM_PREC_FP64;
      }
    f->build_only = opt.build_only;
    f->tol = opt.tol_hlu;
    f->R = opt.R;
    const bool fp32 = f->precision == HFSEM_PREC_MIXED;
    f->tsize = fp32 ? sizeof(float) : sizeof(double);
    const int max_leaf = fp32 ? 128 : 96;
    std::map<std::string, std::shared_ptr<PlanBundle>> cache;
    const int ni = s->n_inst;
    f->plans.resize(ni);
    f->hidev.resize(ni);
    for (int i = 0; i < ni; ++i) {
      const InstHost& I = s->ih[i];
      PlanOpts o;
      o.lambda = opt.lambda;
      const int kmax_eff = opt.kmax ? opt.kmax : opt.R;
      const int max_concat = fp32 ? 160 : 112;   // shared memory of the recompression
      // a dense product appended to a low-rank block adds one leaf's worth of rank
      const int leaf_cap = std::min(max_leaf, max_concat - 2 * kmax_eff);
      int leaf = opt.leaf_elems ? opt.leaf_elems : std::max(1, leaf_cap / I.P);
      leaf = std::min(leaf, std::max(1, leaf_cap / I.P));
      o.leaf_elems = leaf;
      o.R = opt.R;
      o.kmax = kmax_eff;
      o.nrhs_max = 64;
      o.max_concat = max_concat;
      o.max_leaf = max_leaf;
      o.unique_tmp = 1;
      o.ncta = kCluster;
      std::string key = plan_key(I, o);
      auto it = cache.find(key);
      if (it == cache.end()) {
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
                                        ct.hi, cs.lo, cs.hi, ct.d0, b.m, cs.d0, b.n});
        }
        it = cache.emplace(key, pb).first;
      }
      f->plans[i] = it->second;
    }
    // concatenate tables
    std::vector<HOp> ops;
    std::vector<int> waves;
    std::vector<SlotDev> slots;
    std::vector<DenseDev> dense;
    std::vector<LRPairDev> pairs;
    std::map<const PlanBundle*, std::array<long long, 7>> placed;
    long long arena = 0, rk = 0, doff = 0;
    size_t smem = 0;
    for (int i = 0; i < ni; ++i) {
      const PlanBundle* pb = f->plans[i].get();
      auto pi = placed.find(pb);
      if (pi == placed.end()) {
        std::array<long long, 7> a{(long long)ops.size(), (long long)(ops.size() + pb->plan.fac.size()),
                                   (long long)slots.size(), (long long)dense.size(),
                                   (long long)pairs.size(), (long long)waves.size(),
                                   (long long)(waves.size() + pb->plan.fac_waves.size())};
        waves.insert(waves.end(), pb->plan.fac_waves.begin(), pb->plan.fac_waves.end());
        waves.insert(waves.end(), pb->plan.sol_waves.begin(), pb->plan.sol_waves.end());
        ops.insert(ops.end(), pb->plan.fac.begin(), pb->plan.fac.end());
        ops.insert(ops.end(), pb->plan.sol.begin(), pb->plan.sol.end());
        slots.insert(slots.end(), pb->slots.begin(), pb->slots.end());
        dense.insert(dense.end(), pb->dense.begin(), pb->dense.end());
        pairs.insert(pairs.end(), pb->pairs.begin(), pb->pairs.end());
        pi = placed.emplace(pb, a).first;
        smem = std::max(smem, prog_smem(pb->plan, f->tsize));
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
      H.ops0 = pi->second[0];
      H.sops0 = pi->second[1];
      H.nops = (int)p.fac.size();
      H.nsops = (int)p.sol.size();
      H.ndense = (int)pb->dense.size();
      H.npairs = (int)pb->pairs.size();
      H.n_slots = p.n_slots;
      H.ws_off = p.ws_off;
      H.ws_size = p.ws_size;
      H.rhs_off = p.rhs_off;
      H.fw0 = pi->second[5];
      H.sw0 = pi->second[6];
      H.nfw = (int)p.fac_waves.size() - 1;
      H.nsw = (int)p.sol_waves.size() - 1;
      H.d_off = doff;
      doff += s->ih[i].Nd;
      H.sys_inst = i;
      H.R = opt.R;
      f->total_ops += H.nops;
      f->total_sops += H.nsops;
    }
    if (smem > 227 * 1024) throw Error(HFSEM_ERR_UNSUPPORTED, "H-LU kernel needs too much shared memory");
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
    f->d_ranks.alloc(std::max<long long>(rk, 1));
    HF_CHECK(cudaMemsetAsync(f->d_ranks.p, 0, std::max<long long>(rk, 1) * sizeof(int), s->st));
    f->d_err.alloc(ni);
    HF_CHECK(cudaMemsetAsync(f->d_err.p, 0, ni * sizeof(int), s->st));
    f->d_D.alloc(std::max<long long>(doff, 1));
    f->d_arena.alloc((size_t)std::max<long long>(arena, 1) * f->tsize);
    HF_CHECK(cudaMemsetAsync(f->d_arena.p, 0, (size_t)std::max<long long>(arena, 1) * f->tsize, s->st));
    // build A~
    int maxnd = 1, maxdense = 1, maxpairs = 1;
    for (auto& H : f->hidev) {
      maxnd = std::max(maxnd, s->ih[H.sys_inst].Nd);
      maxdense = std::max(maxdense, H.ndense);
      maxpairs = std::max(maxpairs, H.npairs);
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
    dim3 gp(maxpairs, ni);
    if (fp32) {
      float* ar = reinterpret_cast<float*>(f->d_arena.p);
      k_nearfield<float><<<gn, 256, 0, s->st>>>(f->d_hi.p, s->d_inst.p, s->arena.p, f->d_dense.p, f->d_D.p, ar);
      HF_LAUNCH_CHECK();
      if (prof) cudaEventRecord(ev[1], s->st);
      k_lowrank<float><<<gp, 128, 0, s->st>>>(f->d_hi.p, s->d_inst.p, s->arena.p, s->gl.p, f->d_pairs.p,
                                              f->d_slots.p, f->d_D.p, ar, f->d_ranks.p);
      HF_LAUNCH_CHECK();
      set_prog_smem<float>(smem);
    } else {
      double* ar = reinterpret_cast<double*>(f->d_arena.p);
      k_nearfield<double><<<gn, 256, 0, s->st>>>(f->d_hi.p, s->d_inst.p, s->arena.p, f->d_dense.p, f->d_D.p, ar);
      HF_LAUNCH_CHECK();
      if (prof) cudaEventRecord(ev[1], s->st);
      k_lowrank<double><<<gp, 128, 0, s->st>>>(f->d_hi.p, s->d_inst.p, s->arena.p, s->gl.p, f->d_pairs.p,
                                               f->d_slots.p, f->d_D.p, ar, f->d_ranks.p);
      HF_LAUNCH_CHECK();
      set_prog_smem<double>(smem);
    }
    if (prof) cudaEventRecord(ev[2], s->st);
    if (!f->build_only) f->run_prog(0);
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
      fprintf(stderr, "[hfsem plan] N=%d P=%d blocks=%zu dense=%zu lr=%zu fac_ops=%zu sol_ops=%zu "
              "leaf_max=%d kconcat_max=%d hh_lr=%d arena=%lld\n", p0.N, p0.P, p0.B.size(),
              p0.dense_blocks.size(), p0.lr_blocks.size(), p0.fac.size(), p0.sol.size(), p0.leaf_max,
              p0.kconcat_max, p0.hh_lr, p0.arena);
      f->report("factorisation");
    }
    std::vector<int> err(ni);
    HF_CHECK(cudaMemcpy(err.data(), f->d_err.p, ni * sizeof(int), cudaMemcpyDeviceToHost));
    for (int e : err)
      if (e) throw Error(HFSEM_ERR_BREAKDOWN, "zero or non-finite pivot in an H-LU leaf");
  } catch (...) {
    delete f;
    throw;
  }
  return f;
}

}  // namespace hf

void hfsem_factor_s::collect_flops() {
  // move the device flop counters into the timing registry
  if (!d_flops.p || !hf::timing_on()) return;
  std::vector<double> h(d_flops.n);
  cudaMemcpy(h.data(), d_flops.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost);
  double f0 = 0, f1 = 0;
  for (size_t i = 0; i < h.size(); i += 2) {
    f0 += h[i];
    f1 += h[i + 1];
  }
  hf::timing_add_work("hlu_factor", f0);
  hf::timing_add_work("hlu_solve", f1);
  cudaMemset(d_flops.p, 0, d_flops.n * sizeof(double));
}

void hfsem_factor_s::report(const char* what) {
  if (!d_prof.p) return;
  std::vector<unsigned long long> h(d_prof.n);
  cudaMemcpy(h.data(), d_prof.p, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  static const char* names[16] = {"?", "GEMM", "GETRF_INV", "TRMM_L", "TRMM_R", "APPEND",
                                  "TRUNC", "ZERO", "AXPY", "?", "?", "?", "?", "?", "?", "?"};
  fprintf(stderr, "[hfsem profile] %s (instance 0; ns, ops)\n", what);
  for (int t = 0; t < 16; ++t)
    if (h[2 * t + 1])
      fprintf(stderr, "  %-10s %14llu ns %8llu ops %10.0f ns/op\n", names[t], h[2 * t], h[2 * t + 1],
              (double)h[2 * t] / h[2 * t + 1]);
  cudaMemset(d_prof.p, 0, d_prof.n * sizeof(unsigned long long));
}

void hfsem_factor_s::run_prog(int which) {
  if (!d_prof.p && getenv("HFSEM_PROFILE")) {
    d_prof.alloc((size_t)sys->n_inst * 32);
    cudaMemset(d_prof.p, 0, d_prof.n * sizeof(unsigned long long));
  }
  if (!d_flops.p) {
    d_flops.alloc((size_t)sys->n_inst * hf::kCluster * 2);
    cudaMemsetAsync(d_flops.p, 0, d_flops.n * sizeof(double), sys->st);
  }
  hf::HProgArgs a{d_hi.p, d_waves.p, d_ops.p, d_slots.p, d_ranks.p, d_err.p, tol, d_prof.p, d_flops.p};
  hf::Tick tk(sys->st, which ? "hlu_solve" : "hlu_factor");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(sys->n_inst * hf::kCluster));
  cfg.blockDim = dim3(hf::kHThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = sys->st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = hf::kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (tsize == sizeof(float))
    HF_CHECK(cudaLaunchKernelEx(&cfg, hf::k_hprog<float>, a, reinterpret_cast<float*>(d_arena.p), which));
  else
    HF_CHECK(cudaLaunchKernelEx(&cfg, hf::k_hprog<double>, a, reinterpret_cast<double*>(d_arena.p), which));
  HF_LAUNCH_CHECK();
}

void hfsem_factor_s::apply(int nrhs, const double* r_em, double* y_em) {
  if (build_only) throw hf::Error(HFSEM_ERR_INVALID_ARG, "factor was built with build_only");
  if (nrhs > 64) throw hf::Error(HFSEM_ERR_INVALID_ARG, "nrhs > 64");
  int maxnd = 1;
  for (auto& I : sys->ih) maxnd = std::max(maxnd, I.Nd);
  dim3 g(std::min(1024, (maxnd * nrhs + 255) / 256), sys->n_inst);
  if (tsize == sizeof(float)) {
    float* ar = reinterpret_cast<float*>(d_arena.p);
    hf::k_hsolve_in<float><<<g, 256, 0, sys->st>>>(d_hi.p, sys->d_inst.p, r_em, d_D.p, ar, d_ranks.p, nrhs);
    HF_LAUNCH_CHECK();
    run_prog(1);
    if (d_prof.p) {
      cudaStreamSynchronize(sys->st);
      report("H-solve apply");
    }
    hf::k_hsolve_out<float><<<g, 256, 0, sys->st>>>(d_hi.p, sys->d_inst.p, d_D.p, ar, y_em, nrhs);
  } else {
    double* ar = reinterpret_cast<double*>(d_arena.p);
    hf::k_hsolve_in<double><<<g, 256, 0, sys->st>>>(d_hi.p, sys->d_inst.p, r_em, d_D.p, ar, d_ranks.p, nrhs);
    HF_LAUNCH_CHECK();
    run_prog(1);
    hf::k_hsolve_out<double><<<g, 256, 0, sys->st>>>(d_hi.p, sys->d_inst.p, d_D.p, ar, y_em, nrhs);
  }
  HF_LAUNCH_CHECK();
}

namespace hf {
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
    return e.code;
  } catch (...) {
    set_last_error("unknown error");
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
  }
}

int hfsem_precond_apply(hfsem_factor* fac, int32_t nrhs, const double* r, double* y) {
  try {
    if (!fac || !r || !y || nrhs < 1 || nrhs > 64) throw Error(HFSEM_ERR_INVALID_ARG, "bad arguments");
    hfsem_system* s = fac->sys;
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
    std::vector<int> err(s->n_inst);
    HF_CHECK(cudaMemcpy(err.data(), fac->d_err.p, err.size() * sizeof(int), cudaMemcpyDeviceToHost));
    return HFSEM_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.code;
  }
}

void hfsem_factor_free(hfsem_factor* f) {
  if (!f) return;
  cudaStreamSynchronize(f->st);
  f->collect_flops();
  delete f;
}

}  // extern "C"
