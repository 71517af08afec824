// Host planner: cluster tree, block tree with the admissibility condition of
// eq. (admis), storage layout, and the H-LU / H-solve programs (Sec. 4.1).
//
// Clusters are element ranges split in halves down to `leaf_elems` elements
// (the paper does not say how its cluster tree is built).  A cluster owns the
// bubbles of its elements and the hats at their right nodes, so its unknowns
// are contiguous in the element-major ordering; its support (Sec. 3.2) is
// [x_e0, x_min(e1+1, N)].
//
// The H-LU is the usual recursive block LU on the block tree,
//   LU(A11); U12 = L11^-1 A12; L21 = A21 U11^-1; A22 -= L21 U12; LU(A22),
// with every product and solve carried out in the formats of its operands
// (dense, low rank U V^T, hierarchical) and every update of a low-rank block
// appended to its factors and recompressed to the tolerance Tol_HLU.  The
// recursion is unrolled here into a flat list of dense kernels (GEMM,
// triangular multiplies with the inverted diagonal leaves, append and
// truncate), which the device interpreter runs in order.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <unordered_map>
#include <string>

#include "hplan.h"

namespace hf {
namespace {

// every allocation of the arena starts on a multiple of 4 entries (16 bytes
// in FP32), so columns of blocks whose leading dimension is a multiple of 4
// can be moved with 16-byte accesses
inline long long align4(long long x) { return (x + 3) & ~3LL; }

View vT(View v) {
  std::swap(v.r, v.c);
  v.tr ^= 1;
  return v;
}
View vrows(View v, int i0, int i1) {
  v.off += v.tr ? (long long)i0 * v.ld : i0;
  v.r = i1 - i0;
  return v;
}
View vcols(View v, int j0, int j1) {
  v.off += v.tr ? j0 : (long long)j0 * v.ld;
  v.c = j1 - j0;
  return v;
}

struct Builder {
  const InstHost& I;
  const PlanOpts& o;
  HPlan& p;
  long long top = 0;
  long long tmp_base = 0, tmp_top = 0, tmp_peak = 0;
  std::vector<HOp>* prog = nullptr;
  int max_m = 0;
  std::vector<char> dirty;   // LR block received updates since its last recompression
  std::vector<int> rank_est; // per LR slot: estimated current rank (Taylor rank R at first)

  Builder(const InstHost& i, const PlanOpts& op, HPlan& pl) : I(i), o(op), p(pl) {}

  // ---------------- structure ----------------
  int cluster(int e0, int e1) {
    Cluster c;
    c.e0 = e0;
    c.e1 = e1;
    c.d0 = e0 * I.P;
    c.d1 = std::min(e1 * I.P, I.Nd);
    c.lo = e0;
    c.hi = std::min(e1 + 1, I.N);
    c.kid[0] = c.kid[1] = -1;
    int id = (int)p.C.size();
    p.C.push_back(c);
    if (e1 - e0 > o.leaf_elems) {
      int mid = (e0 + e1) / 2;
      int a = cluster(e0, mid);
      int b = cluster(mid, e1);
      p.C[id].kid[0] = a;
      p.C[id].kid[1] = b;
    }
    return id;
  }
  bool leaf(int c) const { return p.C[c].kid[0] < 0; }

  double diam(int c) const { return I.node_diff(p.C[c].hi, p.C[c].lo); }
  double dist(int a, int b) const {
    const Cluster &x = p.C[a], &y = p.C[b];
    if (x.hi < y.lo) return I.node_diff(y.lo, x.hi);
    if (y.hi < x.lo) return I.node_diff(x.lo, y.hi);
    return 0.0;
  }
  bool admissible(int t, int s) const {
    double d = dist(t, s);
    const double dm = o.adm_min ? std::min(diam(t), diam(s)) : std::max(diam(t), diam(s));
    return d > 0.0 && dm <= o.lambda * d;
  }

  int block(int t, int s) {
    Block b;
    b.t = t;
    b.s = s;
    b.m = p.C[t].d1 - p.C[t].d0;
    b.n = p.C[s].d1 - p.C[s].d0;
    b.kid[0] = b.kid[1] = b.kid[2] = b.kid[3] = -1;
    b.off = b.inv = -1;
    b.slot = -1;
    b.kcap = b.kmax = 0;
    b.lower = (p.C[s].hi < p.C[t].lo) ? 1 : 0;
    if (admissible(t, s) && b.m > 0 && b.n > 0) {
      b.type = B_LR;
    } else if (leaf(t) || leaf(s)) {
      b.type = B_DENSE;
    } else {
      b.type = B_HIER;
    }
    int id = (int)p.B.size();
    p.B.push_back(b);
    if (b.type == B_HIER) {
      int k[4];
      k[0] = block(p.C[t].kid[0], p.C[s].kid[0]);
      k[1] = block(p.C[t].kid[0], p.C[s].kid[1]);
      k[2] = block(p.C[t].kid[1], p.C[s].kid[0]);
      k[3] = block(p.C[t].kid[1], p.C[s].kid[1]);
      for (int i = 0; i < 4; ++i) p.B[id].kid[i] = k[i];
    }
    return id;
  }

  void storage() {
    for (size_t i = 0; i < p.B.size(); ++i) {
      Block& b = p.B[i];
      max_m = std::max(max_m, std::max(b.m, b.n));
      if (b.type == B_DENSE) {
        b.off = top;
        top = align4(top + (long long)b.m * b.n);
        p.dense_blocks.push_back((int)i);
        if (b.t == b.s && !o.structure_only) {   // room for the inverted factors
          if (b.m > o.max_leaf)
            throw Error(HFSEM_ERR_UNSUPPORTED, "diagonal leaf larger than the kernel supports");
          p.leaf_max = std::max(p.leaf_max, b.m);
          b.inv = top;
          top = align4(top + 2LL * b.m * b.m);
        }
      } else if (b.type == B_LR) {
        int mn = std::min(b.m, b.n);
        b.kmax = std::min(o.kmax, mn);
        b.kcap = std::max(o.R, std::min(mn, kKcapMult * o.kmax));
        b.off = top;
        top = align4(top + (long long)(b.m + b.n) * b.kcap);
        b.slot = p.n_slots++;
        p.lr_blocks.push_back((int)i);
      }
    }
  }

  // ---------------- views ----------------
  View dense(int bi) const {
    const Block& b = p.B[bi];
    return View{b.off, b.m, b.n, std::max(b.m, 1), 0};
  }
  View linv(int bi) const {
    const Block& b = p.B[bi];
    return View{b.inv, b.m, b.m, std::max(b.m, 1), 0};
  }
  View uinv(int bi) const {
    const Block& b = p.B[bi];
    return View{b.inv + (long long)b.m * b.m, b.m, b.m, std::max(b.m, 1), 0};
  }
  View lrU(int bi) const {
    const Block& b = p.B[bi];
    return View{b.off, b.m, -1 - b.slot, b.m, 0};
  }
  View lrV(int bi) const {
    const Block& b = p.B[bi];
    return View{b.off + (long long)b.m * b.kcap, b.n, -1 - b.slot, b.n, 0};
  }
  int rank_cap(int bi) const { return p.B[bi].kcap; }
  // static upper bound of a (possibly runtime) dimension
  int bound(int d) const {
    if (d >= 0) return d;
    if (-1 - d == p.n_slots) return p.nrhs_max;   // rhs width of the solve program
    return p.B[p.lr_blocks[-1 - d]].kcap;
  }
  void release(long long mark) {
    if (!o.unique_tmp) tmp_top = mark;
  }
  View tmp(int r, int c_bound, int c_dim) {
    View v{tmp_top, r, c_dim, std::max(r, 1), 0};
    p.tmps.push_back({tmp_top, (long long)std::max(r, 1) * std::max(c_bound, 1), std::max(r, 1)});
    tmp_top = align4(tmp_top + (long long)std::max(r, 1) * std::max(c_bound, 1));
    tmp_peak = std::max(tmp_peak, tmp_top - tmp_base);
    return v;
  }
  // row range of child cluster c inside parent cluster par
  int r0(int par, int c) const { return p.C[c].d0 - p.C[par].d0; }
  int r1(int par, int c) const { return p.C[c].d1 - p.C[par].d0; }

  // ---------------- op emission ----------------
  static bool empty(const View& v) { return v.r == 0 || v.c == 0; }
  void op(int type, View A, View B, View C, double alpha, double beta, int slot = -1, int kest = 0) {
    HOp h;
    h.type = type;
    h.slot = slot;
    h.alpha = alpha;
    h.beta = beta;
    h.A = A;
    h.B = B;
    h.C = C;
    h.kest = kest;
    h.pad = 0;
    prog->push_back(h);
  }
  // estimated run-time value of a (possibly runtime) dimension: a rank is
  // taken at the estimate the planner keeps for its slot
  int est(int d) const {
    if (d >= 0) return d;
    if (-1 - d == p.n_slots) return p.nrhs_max;
    return rank_est[-1 - d];
  }
  void gemm(View C, View A, View B, double alpha, double beta) {
    if (empty(C)) return;
    if (A.c == 0) {
      if (beta == 0.0) zero(C);
      return;
    }
    op(OP_GEMM, A, B, C, alpha, beta);
  }
  void zero(View C) {
    if (!empty(C)) op(OP_ZERO, View{}, View{}, C, 0, 0);
  }
  void append(int cb, View U, View V, double alpha) {
    const Block& b = p.B[cb];
    if (U.r == 0 || V.r == 0 || U.c == 0) return;
    int kin = bound(U.c);
    p.kconcat_max = std::max(p.kconcat_max, b.kcap + kin);
    if (b.kcap + kin > o.max_concat)
      throw Error(HFSEM_ERR_UNSUPPORTED, "low-rank update larger than the recompression kernel");
    // the append overflows (and recompresses) when the estimate passes kcap
    const int kest = rank_est[b.slot] + est(U.c);
    op(OP_APPEND, U, V, lrU(cb), alpha, 0.0, b.slot, kest);
    rank_est[b.slot] = (kest > b.kcap) ? b.kmax : kest;
    dirty[cb] = 1;
  }
  void trunc(int cb) {
    // blocks that still hold their Taylor factors (rank R <= kmax) are used as
    // they are; updated blocks are recompressed before they become factors
    if (!dirty[cb]) return;
    dirty[cb] = 0;
    const Block& b = p.B[cb];
    p.kconcat_max = std::max(p.kconcat_max, b.kcap);
    op(OP_TRUNC, View{}, View{}, lrU(cb), 0.0, 0.0, b.slot, rank_est[b.slot]);
    rank_est[b.slot] = std::min(rank_est[b.slot], b.kmax);
  }

  // C += alpha U V^T, C any format
  void add_lr(int cb, View U, View V, double alpha) {
    const Block& c = p.B[cb];
    if (c.m == 0 || c.n == 0) return;
    if (c.type == B_DENSE) {
      gemm(dense(cb), U, vT(V), alpha, 1.0);
    } else if (c.type == B_LR) {
      append(cb, U, V, alpha);
    } else {
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          int k = c.kid[2 * i + j];
          int ti = p.C[c.t].kid[i], sj = p.C[c.s].kid[j];
          add_lr(k, vrows(U, r0(c.t, ti), r1(c.t, ti)), vrows(V, r0(c.s, sj), r1(c.s, sj)),
                 alpha);
        }
    }
  }

  // C += alpha Z, Z dense view, C any format
  void add_dense(int cb, View Z, double alpha) {
    const Block& c = p.B[cb];
    if (c.m == 0 || c.n == 0) return;
    if (c.type == B_DENSE) {
      op(OP_AXPY, Z, View{}, dense(cb), alpha, 1.0);
    } else if (c.type == B_LR) {
      // Z = Z I: append 32-column slices with identity right factors
      // (B.off = -1 - first column), each followed by a recompression
      p.hh_lr++;
      for (int c0 = 0; c0 < c.n; c0 += 32) {
        int c1 = std::min(c.n, c0 + 32);
        View Iv{-1 - (long long)c0, c.n, c1 - c0, c.n, 0};
        append(cb, vcols(Z, c0, c1), Iv, alpha);
      }
    } else {
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          int k = c.kid[2 * i + j];
          int ti = p.C[c.t].kid[i], sj = p.C[c.s].kid[j];
          add_dense(k, vcols(vrows(Z, r0(c.t, ti), r1(c.t, ti)), r0(c.s, sj), r1(c.s, sj)),
                    alpha);
        }
    }
  }

  // D += alpha A E  (A block, E dense)
  void gemm_hd(View D, int ab, View E, double alpha) {
    const Block& a = p.B[ab];
    if (a.m == 0 || a.n == 0 || empty(D)) return;
    if (a.type == B_DENSE) {
      gemm(D, dense(ab), E, alpha, 1.0);
    } else if (a.type == B_LR) {
      long long mark = tmp_top;
      View T = tmp(a.kcap, bound(E.c), E.c);
      T.r = lrU(ab).c;   // runtime rank rows
      gemm(T, vT(lrV(ab)), E, 1.0, 0.0);
      gemm(D, lrU(ab), T, alpha, 1.0);
      release(mark);
    } else {
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          int ti = p.C[a.t].kid[i], sj = p.C[a.s].kid[j];
          gemm_hd(vrows(D, r0(a.t, ti), r1(a.t, ti)), a.kid[2 * i + j],
                  vrows(E, r0(a.s, sj), r1(a.s, sj)), alpha);
        }
    }
  }

  // D += alpha E B  (E dense, B block)
  void gemm_dh(View D, View E, int bb, double alpha) {
    const Block& b = p.B[bb];
    if (b.m == 0 || b.n == 0 || empty(D)) return;
    if (b.type == B_DENSE) {
      gemm(D, E, dense(bb), alpha, 1.0);
    } else if (b.type == B_LR) {
      long long mark = tmp_top;
      View T = tmp(bound(E.r), b.kcap, lrU(bb).c);
      T.r = E.r;
      gemm(T, E, lrU(bb), 1.0, 0.0);
      gemm(D, T, vT(lrV(bb)), alpha, 1.0);
      release(mark);
    } else {
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          int ti = p.C[b.t].kid[i], sj = p.C[b.s].kid[j];
          gemm_dh(vcols(D, r0(b.s, sj), r1(b.s, sj)), vcols(E, r0(b.t, ti), r1(b.t, ti)),
                  b.kid[2 * i + j], alpha);
        }
    }
  }

  // D += alpha A B (A, B blocks; D dense view)
  void gemm_dab(View D, int ab, int bb, double alpha) {
    const Block &a = p.B[ab], &b = p.B[bb];
    if (a.m == 0 || a.n == 0 || b.n == 0 || empty(D)) return;
    if (a.type == B_DENSE) {
      gemm_dh(D, dense(ab), bb, alpha);
    } else if (b.type == B_DENSE) {
      gemm_hd(D, ab, dense(bb), alpha);
    } else if (a.type == B_LR) {
      long long mark = tmp_top;
      View T = tmp(a.kcap, b.n, b.n);
      T.r = lrU(ab).c;
      zero(T);
      gemm_dh(T, vT(lrV(ab)), bb, 1.0);
      gemm(D, lrU(ab), T, alpha, 1.0);
      release(mark);
    } else if (b.type == B_LR) {
      long long mark = tmp_top;
      View Z = tmp(a.m, b.kcap, lrU(bb).c);
      zero(Z);
      gemm_hd(Z, ab, lrU(bb), 1.0);
      gemm(D, Z, vT(lrV(bb)), alpha, 1.0);
      release(mark);
    } else {
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int k = 0; k < 2; ++k) {
            int ti = p.C[a.t].kid[i], sj = p.C[b.s].kid[j];
            gemm_dab(vcols(vrows(D, r0(a.t, ti), r1(a.t, ti)), r0(b.s, sj), r1(b.s, sj)),
                     a.kid[2 * i + k], b.kid[2 * k + j], alpha);
          }
    }
  }

  // C -= A B, blocks
  void gemm_sub(int cb, int ab, int bb) {
    const Block &c = p.B[cb], &a = p.B[ab], &b = p.B[bb];
    if (c.m == 0 || c.n == 0 || a.n == 0) return;
    if (c.type == B_HIER && a.type == B_HIER && b.type == B_HIER) {
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int k = 0; k < 2; ++k)
            gemm_sub(c.kid[2 * i + j], a.kid[2 * i + k], b.kid[2 * k + j]);
      return;
    }
    if (c.type == B_DENSE) {
      gemm_dab(dense(cb), ab, bb, -1.0);
      return;
    }
    if (a.type == B_LR) {
      // A B = U_A (B^T V_A)^T
      long long mark = tmp_top;
      View W = tmp(b.n, a.kcap, lrU(ab).c);      // n x k
      zero(W);
      gemm_dh(vT(W), vT(lrV(ab)), bb, 1.0);      // W^T += V_A^T B
      add_lr(cb, lrU(ab), W, -1.0);
      release(mark);
      return;
    }
    if (b.type == B_LR) {
      long long mark = tmp_top;
      View Z = tmp(a.m, b.kcap, lrU(bb).c);      // m x k
      zero(Z);
      gemm_hd(Z, ab, lrU(bb), 1.0);
      add_lr(cb, Z, lrV(bb), -1.0);
      release(mark);
      return;
    }
    if (a.type == B_DENSE && b.type == B_DENSE) {
      // rank at most the inner (leaf) cluster size
      add_lr(cb, dense(ab), vT(dense(bb)), -1.0);
      return;
    }
    // remaining: C LR / H with a hierarchical factor: form the product densely
    long long mark = tmp_top;
    View Z = tmp(a.m, b.n, b.n);
    zero(Z);
    gemm_dab(Z, ab, bb, 1.0);
    add_dense(cb, Z, -1.0);
    release(mark);
  }

  // X <- L^-1 X for a dense view, L the diagonal block lb
  void trsm_ll_d(int lb, View D) {
    const Block& l = p.B[lb];
    if (l.m == 0 || empty(D)) return;
    if (l.type == B_DENSE) {
      op(OP_TRMM_L, linv(lb), View{}, D, 1.0, 0.0);
      return;
    }
    int t1 = p.C[l.t].kid[0], t2 = p.C[l.t].kid[1];
    View D1 = vrows(D, r0(l.t, t1), r1(l.t, t1)), D2 = vrows(D, r0(l.t, t2), r1(l.t, t2));
    trsm_ll_d(l.kid[0], D1);
    gemm_hd(D2, l.kid[2], D1, -1.0);
    trsm_ll_d(l.kid[3], D2);
  }
  // X <- X U^-1 for a dense view
  void trsm_ru_d(int ub, View D) {
    const Block& u = p.B[ub];
    if (u.m == 0 || empty(D)) return;
    if (u.type == B_DENSE) {
      op(OP_TRMM_R, uinv(ub), View{}, D, 1.0, 0.0);
      return;
    }
    int s1 = p.C[u.s].kid[0], s2 = p.C[u.s].kid[1];
    View D1 = vcols(D, r0(u.s, s1), r1(u.s, s1)), D2 = vcols(D, r0(u.s, s2), r1(u.s, s2));
    trsm_ru_d(u.kid[0], D1);
    gemm_dh(D2, D1, u.kid[1], -1.0);
    trsm_ru_d(u.kid[3], D2);
  }

  void trsm_ll(int lb, int xb) {
    const Block& x = p.B[xb];
    if (x.m == 0 || x.n == 0) return;
    if (x.type == B_DENSE) {
      trsm_ll_d(lb, dense(xb));
    } else if (x.type == B_LR) {
      trunc(xb);
      trsm_ll_d(lb, lrU(xb));
    } else {
      const Block& l = p.B[lb];
      trsm_ll(l.kid[0], x.kid[0]);
      trsm_ll(l.kid[0], x.kid[1]);
      gemm_sub(x.kid[2], l.kid[2], x.kid[0]);
      gemm_sub(x.kid[3], l.kid[2], x.kid[1]);
      trsm_ll(l.kid[3], x.kid[2]);
      trsm_ll(l.kid[3], x.kid[3]);
    }
  }

  void trsm_ru(int ub, int xb) {
    const Block& x = p.B[xb];
    if (x.m == 0 || x.n == 0) return;
    if (x.type == B_DENSE) {
      trsm_ru_d(ub, dense(xb));
    } else if (x.type == B_LR) {
      trunc(xb);
      trsm_ru_d(ub, vT(lrV(xb)));   // V^T <- V^T U^-1
    } else {
      const Block& u = p.B[ub];
      trsm_ru(u.kid[0], x.kid[0]);
      trsm_ru(u.kid[0], x.kid[2]);
      gemm_sub(x.kid[1], x.kid[0], u.kid[1]);
      gemm_sub(x.kid[3], x.kid[2], u.kid[1]);
      trsm_ru(u.kid[3], x.kid[1]);
      trsm_ru(u.kid[3], x.kid[3]);
    }
  }

  void hlu(int bb) {
    const Block& b = p.B[bb];
    if (b.m == 0) return;
    if (b.type == B_DENSE) {
      op(OP_GETRF_INV, linv(bb), uinv(bb), dense(bb), 1.0, 0.0);
      return;
    }
    int k0 = b.kid[0], k1 = b.kid[1], k2 = b.kid[2], k3 = b.kid[3];
    hlu(k0);
    trsm_ll(k0, k1);
    trsm_ru(k0, k2);
    gemm_sub(k3, k2, k1);
    hlu(k3);
  }
};

}  // namespace

void make_plan(const InstHost& I, const PlanOpts& o, HPlan& p) {
  p = HPlan();
  p.N = I.N;
  p.P = I.P;
  p.Nd = I.Nd;
  p.nrhs_max = o.nrhs_max;
  p.R = o.R;
  Builder b(I, o, p);
  int root = b.cluster(0, I.N);
  b.block(root, root);
  b.storage();
  if (o.structure_only) {   // an H-matrix to be built, never factored
    p.arena = align4(b.top);
    p.fac_waves.assign(1, 0);
    p.ncta = std::max(o.ncta, 1);
    return;
  }
  b.dirty.assign(p.B.size(), 0);
  b.rank_est.assign(p.n_slots, o.R);
  // right-hand-side area, then temporaries, then the truncation workspace
  p.rhs_off = b.top;
  b.top = align4(b.top + (long long)std::max(I.Nd, 1) * o.nrhs_max);
  b.tmp_base = b.tmp_top = b.top;
  b.prog = &p.fac;
  b.hlu(0);
  long long ws_off = b.tmp_base + b.tmp_peak;
  p.tmp_base = b.tmp_base;
  p.tmp_size = b.tmp_peak;
  p.ws_off = ws_off;
  p.ws_size = (long long)2 * std::max(b.max_m, 1) * std::max(p.kconcat_max, 1);
  p.ncta = std::max(o.ncta, 1);
  p.arena = ws_off + p.ws_size * p.ncta;
  schedule_program(p, p.fac, p.fac_waves);
}

}  // namespace hf

namespace hf {
namespace {

// storage rectangle touched by a view: [r0, r1) x [c0, c1) of the column-major
// matrix starting at `base` with leading dimension ld (rank dims -> capacity)
struct Rect {
  long long base;
  int bucket;   // index of the access history the rectangle belongs to
  int ld;
  long long r0, r1, c0, c1;
  int slot;   // LR slot whose rank is read (-1 none)
};

struct Access {
  Rect rc;
  bool write;
};

}  // namespace

int program_levels(const HPlan& p, const std::vector<HOp>& prog, std::vector<int>& level) {
  // map storage offsets to the allocation that holds them
  struct Alloc {
    long long off, size;
    int ld;
    int slot;
  };
  std::vector<Alloc> al;
  for (const Block& b : p.B) {
    if (b.type == B_DENSE) {
      al.push_back({b.off, (long long)b.m * b.n, std::max(b.m, 1), -1});
      if (b.inv >= 0) {
        al.push_back({b.inv, (long long)b.m * b.m, std::max(b.m, 1), -1});
        al.push_back({b.inv + (long long)b.m * b.m, (long long)b.m * b.m, std::max(b.m, 1), -1});
      }
    } else if (b.type == B_LR) {
      al.push_back({b.off, (long long)b.m * b.kcap, b.m, b.slot});
      al.push_back({b.off + (long long)b.m * b.kcap, (long long)b.n * b.kcap, b.n, b.slot});
    }
  }
  for (const auto& t : p.tmps) al.push_back({t.off, t.size, t.ld, -1});
  std::sort(al.begin(), al.end(), [](const Alloc& a, const Alloc& b) { return a.off < b.off; });
  // coarse index: for every 4096-element bucket of the arena, the number of
  // allocations that start before the bucket (a lookup then scans the few
  // allocations that start inside it)
  constexpr int kShift = 12;
  long long top = 0;
  for (const Alloc& a : al) top = std::max(top, a.off + a.size);
  std::vector<int> first((size_t)(top >> kShift) + 2, 0);
  {
    size_t k = 0;
    for (size_t bk = 0; bk < first.size(); ++bk) {
      while (k < al.size() && al[k].off < ((long long)bk << kShift)) ++k;
      first[bk] = (int)k;
    }
  }
  auto find = [&](long long off) -> const Alloc* {
    if (off < 0 || al.empty()) return nullptr;
    const size_t bk = std::min((size_t)(off >> kShift), first.size() - 2);
    // allocations [0, first[bk]) start before the bucket, [first[bk],
    // first[bk + 1]) inside it: the last one starting at or before off
    size_t lo = first[bk], hi = std::max<size_t>(first[bk + 1], lo);
    while (lo < hi) {
      const size_t mid = (lo + hi) / 2;
      if (al[mid].off <= off) lo = mid + 1;
      else hi = mid;
    }
    while (lo < al.size() && al[lo].off <= off) ++lo;   // off past the last bucket
    if (lo == 0) return nullptr;
    const Alloc& a = al[lo - 1];
    return (off < a.off + a.size) ? &a : nullptr;
  };
  auto rect_of = [&](const View& v, int ncol_cap) -> Rect {
    // rows/cols in storage coordinates
    int sr = v.tr ? v.c : v.r, sc = v.tr ? v.r : v.c;
    Rect r;
    const Alloc* a = find(v.off);
    int slot = -1;
    if (sr < 0) slot = -1 - sr;
    if (sc < 0) slot = -1 - sc;
    if (a && a->slot >= 0) {   // LR factor: whole factor, rank read
      r.base = a->off;
      r.bucket = 2 + (int)(a - al.data());
      r.ld = a->ld;
      r.r0 = 0;
      r.r1 = a->ld;
      r.c0 = 0;
      r.c1 = a->size / a->ld;
      r.slot = a->slot;
      return r;
    }
    long long rows = sr < 0 ? ncol_cap : sr, cols = sc < 0 ? ncol_cap : sc;
    if (a) {
      long long rel = v.off - a->off;
      r.base = a->off;
      r.bucket = 2 + (int)(a - al.data());
      r.ld = a->ld;
      r.r0 = rel % a->ld;
      r.c0 = rel / a->ld;
    } else if (v.off >= p.rhs_off && v.off < p.rhs_off + (long long)std::max(p.Nd, 1) * p.nrhs_max) {
      long long rel = v.off - p.rhs_off;
      int ldr = std::max(p.Nd, 1);
      r.base = p.rhs_off;
      r.bucket = 1;
      r.ld = ldr;
      r.r0 = rel % ldr;
      r.c0 = rel / ldr;
    } else {   // temporaries: by raw address
      r.base = -1;
      r.bucket = 0;
      r.ld = v.ld;
      r.r0 = v.off % std::max(v.ld, 1);
      r.c0 = v.off / std::max(v.ld, 1);
      // treat as an interval [off, off + ld*cols)
      r.r0 = v.off;
      r.r1 = v.off + (long long)std::max(v.ld, 1) * (cols - 1) + rows;
      r.c0 = 0;
      r.c1 = 1;
      r.slot = slot;
      return r;
    }
    r.r1 = r.r0 + rows;
    r.c1 = r.c0 + cols;
    r.slot = slot;
    return r;
  };
  auto overlap = [](const Rect& a, const Rect& b) {
    if (a.base != b.base) return false;
    return a.r0 < b.r1 && b.r0 < a.r1 && a.c0 < b.c1 && b.c0 < a.c1;
  };
  const int cap = 64;
  level.assign(prog.size(), 0);
  // Per storage region (allocation base) the accesses that can still decide
  // a later op's level: a write dominates every earlier access it covers
  // (any later access that meets the covered one meets the write, whose
  // level is higher), so covered records are dropped; reads of the same
  // rectangle keep one record with their highest level; a read looks at
  // writes only.
  struct Rec {
    Rect rc;
    int lvl;
  };
  struct Hist {
    std::vector<Rec> wr, rd;
  };
  auto same = [](const Rect& a, const Rect& b) {
    return a.r0 == b.r0 && a.r1 == b.r1 && a.c0 == b.c0 && a.c1 == b.c1;
  };
  auto covers = [](const Rect& a, const Rect& b) {   // a contains b
    return a.r0 <= b.r0 && b.r1 <= a.r1 && a.c0 <= b.c0 && b.c1 <= a.c1;
  };
  // access histories: 0 raw addresses, 1 the right-hand-side area, 2 + k
  // allocation k
  std::vector<Hist> hist(al.size() + 2);
  // slot -> (last write level, max read level); 0: none yet
  std::vector<std::pair<int, int>> slot_state((size_t)std::max(p.n_slots, 0) + 1, {0, 0});
  int nlev = 0;
  std::vector<Access> acc;
  for (size_t i = 0; i < prog.size(); ++i) {
    const HOp& o = prog[i];
    acc.clear();
    auto add = [&](const View& v, bool w) {
      if (v.r == 0 || v.c == 0) return;
      acc.push_back({rect_of(v, cap), w});
    };
    int slot_w = -1;
    switch (o.type) {
      case OP_GEMM: add(o.A, false); add(o.B, false); add(o.C, true); break;
      case OP_GETRF_INV: add(o.C, true); add(o.A, true); add(o.B, true); break;
      case OP_TRMM_L: case OP_TRMM_R: add(o.A, false); add(o.C, true); break;
      case OP_APPEND: add(o.A, false); if (o.B.off >= 0) add(o.B, false); add(o.C, true); slot_w = o.slot; break;
      case OP_TRUNC: add(o.C, true); slot_w = o.slot; break;
      case OP_ZERO: add(o.C, true); break;
      case OP_AXPY: add(o.A, false); add(o.C, true); break;
    }
    int lv = 0;
    for (auto& a : acc) {
      const Hist& hh = hist[a.rc.bucket];
      for (auto& r : hh.wr)
        if (overlap(a.rc, r.rc)) lv = std::max(lv, r.lvl);
      if (a.write)
        for (auto& r : hh.rd)
          if (overlap(a.rc, r.rc)) lv = std::max(lv, r.lvl);
      if (a.rc.slot >= 0) lv = std::max(lv, slot_state[a.rc.slot].first);   // reads the slot's rank
    }
    if (slot_w >= 0) lv = std::max(lv, std::max(slot_state[slot_w].first, slot_state[slot_w].second));
    lv += 1;
    level[i] = lv;
    nlev = std::max(nlev, lv);
    for (auto& a : acc) {
      Hist& h = hist[a.rc.bucket];
      if (a.write) {
        auto dominated = [&](const Rec& r) { return covers(a.rc, r.rc); };
        h.wr.erase(std::remove_if(h.wr.begin(), h.wr.end(), dominated), h.wr.end());
        h.rd.erase(std::remove_if(h.rd.begin(), h.rd.end(), dominated), h.rd.end());
        h.wr.push_back({a.rc, lv});
      } else {
        bool merged = false;
        for (auto& r : h.rd)
          if (same(r.rc, a.rc)) {
            r.lvl = std::max(r.lvl, lv);
            merged = true;
            break;
          }
        if (!merged) h.rd.push_back({a.rc, lv});
      }
      if (a.rc.slot >= 0) {   // only APPEND / TRUNC change a rank (slot_w below)
        auto& st = slot_state[a.rc.slot];
        st.second = std::max(st.second, lv);
      }
    }
    if (slot_w >= 0) {
      auto& st = slot_state[slot_w];
      st.first = std::max(st.first, lv);
    }
  }
  return nlev;
}

}  // namespace hf

namespace hf {

// recompression of an m x K and an n x K factor: K Householder steps on each,
// a pivoted QR of the K x K core and two applications of the reflectors
static double trunc_cost(int m, int n, int K) { return 8.0 + K * (1.5 + (m + n) / 400.0); }

// Estimated run time (microseconds) of an op on one CTA, runtime ranks taken
// as the Taylor rank (or the planner's estimate for appends and
// recompressions): a fixed cost for the op's latencies plus its work at the
// rates the interpreter's kernels reach.
static double op_cost(const HPlan& p, const HOp& o) {
  auto dim = [&](int d) -> double {
    if (d >= 0) return d;
    const int sl = -1 - d;
    if (sl >= p.n_slots) return p.nrhs_max;
    return std::min(p.B[p.lr_blocks[sl]].kcap, std::max(p.R, 1));
  };
  switch (o.type) {
    case OP_GEMM: return 2.0 + 2.0 * dim(o.C.r) * dim(o.C.c) * dim(o.A.c) / 3e5;
    case OP_TRMM_L: return 2.0 + 2.0 * dim(o.C.r) * dim(o.C.r) * dim(o.C.c) / 2e5;
    case OP_TRMM_R: return 2.0 + 2.0 * dim(o.C.r) * dim(o.C.c) * dim(o.C.c) / 2e5;
    case OP_GETRF_INV: {
      const double n = dim(o.C.r) / 128.0;
      return 5.0 + 100.0 * n * n * n;
    }
    case OP_TRUNC: {
      const Block& b = p.B[p.lr_blocks[o.slot]];
      return trunc_cost(b.m, b.n, std::max(o.kest, 1));
    }
    case OP_APPEND: {
      const Block& b = p.B[p.lr_blocks[o.slot]];
      if (o.kest > b.kcap) return trunc_cost(b.m, b.n, o.kest);   // overflow: recompression
      return 2.0 + (b.m + b.n) * dim(o.A.c) / 2e4;
    }
    default: return 0.5 + dim(o.C.r) * dim(o.C.c) / 1e5;
  }
}

void schedule_program(const HPlan& p, std::vector<HOp>& prog, std::vector<int>& waves) {
  // 1. split big ops into independent pieces
  std::vector<HOp> out;
  out.reserve(prog.size() * 2);
  for (const HOp& o : prog) {
    if (o.type == OP_GEMM && o.C.r > 128) {
      for (int r0 = 0; r0 < o.C.r; r0 += 128) {
        int r1 = std::min(o.C.r, r0 + 128);
        HOp q = o;
        q.C = vrows(o.C, r0, r1);
        q.A = vrows(o.A, r0, r1);
        out.push_back(q);
      }
    } else if (o.type == OP_TRMM_L && o.C.c > 32) {
      for (int c0 = 0; c0 < o.C.c; c0 += 32) {
        HOp q = o;
        q.C = vcols(o.C, c0, std::min(o.C.c, c0 + 32));
        out.push_back(q);
      }
    } else if (o.type == OP_TRMM_R && o.C.r > 32) {
      for (int r0 = 0; r0 < o.C.r; r0 += 32) {
        HOp q = o;
        q.C = vrows(o.C, r0, std::min(o.C.r, r0 + 32));
        out.push_back(q);
      }
    } else {
      out.push_back(o);
    }
  }
  // 2. dependency levels, 3. stable order by level
  std::vector<int> lv;
  int nl = program_levels(p, out, lv);
  std::vector<int> cnt(nl + 2, 0);
  for (int l : lv) cnt[l]++;
  waves.assign(nl + 1, 0);
  for (int l = 1; l <= nl; ++l) waves[l] = waves[l - 1] + cnt[l];
  // op indices by level, in program order within a level
  std::vector<int> pos(waves.begin(), waves.end());
  std::vector<int> idx(out.size());
  for (size_t i = 0; i < out.size(); ++i) idx[pos[lv[i] - 1]++] = (int)i;
  // 4. within a wave, the longest ops first: the CTAs take ops in this order
  // as they become free (a counter per wave), longest-processing-time first
  // (ties keep program order)
  std::vector<double> cost(out.size());
  for (size_t i = 0; i < out.size(); ++i) cost[i] = op_cost(p, out[i]);
  for (int w = 0; w < nl; ++w)
    std::stable_sort(idx.begin() + waves[w], idx.begin() + waves[w + 1],
                     [&](int x, int y) { return cost[x] > cost[y]; });
  prog.resize(out.size());
  for (size_t k = 0; k < out.size(); ++k) prog[k] = out[idx[k]];
}

}  // namespace hf

namespace hf {
// Tables of the leaf solves: the leaf clusters in the order of their
// unknowns; for each leaf and direction the column jobs of the blocks in its
// block row (left of the diagonal forward, right of it backward), of its
// inverse diagonal block, and of the low-rank blocks whose column cluster
// holds it (the leaf's rows of V).  Column l of low-rank slot k belongs to
// CTA (k + l) mod ncta for both its gathers and its scatters; dense and
// inverse columns go to the CTA with the fewest jobs in the step so far.
size_t solve_smem(int jmax, int nmax, int wcols, int ts, int sw) {
  // mbarriers, two buffers of jmax column slots (nmax entries rounded to 16
  // bytes), six 128 x sw vectors and the ring, the CTA's w columns, the
  // gather scalars, two buffers of 16-byte job records
  const size_t slot = ((size_t)nmax * ts + 15) / 16 * 16;
  return 16 + 2 * (size_t)jmax * slot + (size_t)(6 + kRing) * 128 * sw * ts +
         (size_t)wcols * sw * ts + (size_t)jmax * sw * ts + 2 * (size_t)jmax * 16;
}

void build_leaf_solve(const HPlan& p, int ncta, size_t budget, int ts, int sw, LeafSolve& pb,
                      int nmax_min, int wcols_min) {
  std::vector<int> lf;
  for (size_t c = 0; c < p.C.size(); ++c)
    if (p.C[c].kid[0] < 0 && p.C[c].d1 > p.C[c].d0) lf.push_back((int)c);
  std::sort(lf.begin(), lf.end(), [&](int a, int b) { return p.C[a].d0 < p.C[b].d0; });
  const int nl = (int)lf.size();
  std::vector<long long> inv(p.C.size(), -1);
  for (const Block& b : p.B)
    if (b.type == B_DENSE && b.t == b.s) inv[b.t] = b.inv;
  // a factored low-rank block holds its Taylor rank R or a rank <= kmax after
  // recompression (every updated block is recompressed before it is used),
  // so columns from max(R, kmax) on are never active in the solves
  auto lmax = [&](const Block& b) { return std::min(b.kcap, std::max(p.R, b.kmax)); };
  // owner CTA and local w column of every low-rank column
  std::vector<std::vector<int>> wloc(p.n_slots);
  std::vector<int> wcnt(ncta, 0);
  for (int sl = 0; sl < p.n_slots; ++sl) {
    const Block& b = p.B[p.lr_blocks[sl]];
    wloc[sl].resize(lmax(b));
    for (int l = 0; l < lmax(b); ++l) wloc[sl][l] = wcnt[(sl + l) % ncta]++;
  }
  pb.wcols = 1;
  for (int c = 0; c < ncta; ++c) pb.wcols = std::max(pb.wcols, wcnt[c]);
  auto leaves_in = [&](int c, int& q0, int& q1) {
    const int d0 = p.C[c].d0, d1 = p.C[c].d1;
    q0 = (int)(std::lower_bound(lf.begin(), lf.end(), d0,
                                [&](int a, int v) { return p.C[a].d0 < v; }) - lf.begin());
    q1 = q0;
    while (q1 < nl && p.C[lf[q1]].d1 <= d1) ++q1;
  };
  auto leaf_of = [&](int d) {   // leaf holding unknown d
    int q = (int)(std::upper_bound(lf.begin(), lf.end(), d,
                                   [&](int v, int a) { return v < p.C[a].d0; }) - lf.begin()) - 1;
    return q;
  };
  // per leaf and direction: gather and scatter jobs, with their owner (-1: free)
  struct OJ {
    SolJob j;
    int owner;
  };
  std::vector<std::vector<OJ>> gat[2], sca[2];
  for (int d = 0; d < 2; ++d) {
    gat[d].assign(nl, {});
    sca[d].assign(nl, {});
  }
  for (const Block& b : p.B) {
    if (b.m == 0 || b.n == 0 || b.t == b.s) continue;
    if (b.type != B_DENSE && b.type != B_LR) continue;
    const Cluster &ct = p.C[b.t], &cs = p.C[b.s];
    const int d = (cs.d1 <= ct.d0) ? 0 : 1;   // block of L (forward) or of U (backward)
    int q0, q1;
    leaves_in(b.t, q0, q1);
    for (int q = q0; q < q1; ++q) {
      const long long ro = p.C[lf[q]].d0 - ct.d0;
      const int nq = p.C[lf[q]].d1 - p.C[lf[q]].d0;
      if (b.type == B_DENSE) {
        for (int k = 0; k < b.n; ++k) {
          const int row = cs.d0 + k, qs = leaf_of(row);
          const int dist = d == 0 ? q - qs : qs - q;
          SolJob J{b.off + ro + (long long)k * b.m, row, -1, 0, 4, 0, nq, 0};
          if (dist >= 1 && dist <= kRing) {
            J.kind = 0;
            J.x = (qs % kRing) * 128 + (row - p.C[lf[qs]].d0);
          }
          gat[d][q].push_back({J, -1});
        }
      } else {
        for (int l = 0; l < lmax(b); ++l)
          gat[d][q].push_back({SolJob{b.off + ro + (long long)l * b.m, wloc[b.slot][l], b.slot,
                                      (short)l, 1, 0, nq, lmax(b)},
                               (b.slot + l) % ncta});
      }
    }
    if (b.type == B_LR) {
      leaves_in(b.s, q0, q1);
      const long long v0 = b.off + (long long)b.m * b.kcap;
      for (int q = q0; q < q1; ++q) {
        const long long ro = p.C[lf[q]].d0 - cs.d0;
        const int nq = p.C[lf[q]].d1 - p.C[lf[q]].d0;
        for (int l = 0; l < lmax(b); ++l)
          sca[d][q].push_back({SolJob{v0 + ro + (long long)l * b.n, wloc[b.slot][l], b.slot,
                                      (short)l, 3, 0, nq, lmax(b)},
                               (b.slot + l) % ncta});
      }
    }
  }
  pb.steps.clear();
  pb.step_cta.clear();
  pb.jobs.clear();
  pb.nmax = 1;
  for (int q = 0; q < nl; ++q) pb.nmax = std::max(pb.nmax, p.C[lf[q]].d1 - p.C[lf[q]].d0);
  // the largest part that fits the budget
  const int nm = std::max(pb.nmax, nmax_min), wc = std::max(pb.wcols, wcols_min);
  int jcap = 1;
  while (jcap < 4096 && solve_smem(jcap + 1, nm, wc, ts, sw) <= budget) ++jcap;
  if (solve_smem(jcap, nm, wc, ts, sw) > budget)
    throw Error(HFSEM_ERR_UNSUPPORTED, "leaf solve does not fit in shared memory");
  pb.jcap = jcap;
  {
    size_t total = 0;
    for (int d = 0; d < 2; ++d)
      for (int q = 0; q < nl; ++q)
        total += gat[d][q].size() + sca[d][q].size() + (size_t)(p.C[lf[q]].d1 - p.C[lf[q]].d0);
    pb.jobs.reserve(total);
    pb.steps.reserve(2 * (size_t)nl);
    pb.step_cta.reserve(2 * (size_t)nl * ncta);
  }
  // per-CTA job lists of a step (kept across steps: capacity reused)
  std::vector<std::array<std::vector<SolJob>, 3>> per(ncta);
  std::vector<int> load(ncta, 0);
  for (int st = 0; st < 2 * nl; ++st) {
    const int d = st < nl ? 0 : 1;
    const int q = d == 0 ? st : 2 * nl - 1 - st;
    const Cluster& c = p.C[lf[q]];
    const int n = c.d1 - c.d0;
    if (inv[lf[q]] < 0) throw Error(HFSEM_ERR_DEVICE, "leaf without a dense diagonal block");
    if (n > 128) throw Error(HFSEM_ERR_UNSUPPORTED, "leaf larger than the solve kernel supports");
    pb.steps.push_back(StepInfo{c.d0, n, q % kRing});
    const long long dinv = inv[lf[q]] + (d ? (long long)n * n : 0LL);
    for (auto& a : per)
      for (auto& v : a) v.clear();
    std::fill(load.begin(), load.end(), 0);
    for (const OJ& o : gat[d][q])
      if (o.owner >= 0) {
        per[o.owner][0].push_back(o.j);
        load[o.owner]++;
      }
    for (const OJ& o : sca[d][q]) load[o.owner]++;
    auto least = [&]() {
      int c0 = 0;
      for (int k = 1; k < ncta; ++k)
        if (load[k] < load[c0]) c0 = k;
      return c0;
    };
    for (const OJ& o : gat[d][q])
      if (o.owner < 0) {
        const int c0 = least();
        per[c0][0].push_back(o.j);
        load[c0]++;
      }
    for (int k = 0; k < n; ++k) {
      const int c0 = least();
      per[c0][1].push_back(SolJob{dinv + (long long)k * n, k, -1, 0, 2, 0, n, 0});
      load[c0]++;
    }
    for (const OJ& o : sca[d][q]) per[o.owner][2].push_back(o.j);
    for (int cr = 0; cr < ncta; ++cr) {
      StepCta sc{};
      sc.a0 = (int)pb.jobs.size();
      pb.jobs.insert(pb.jobs.end(), per[cr][0].begin(), per[cr][0].end());
      sc.a1 = (int)pb.jobs.size();
      pb.jobs.insert(pb.jobs.end(), per[cr][1].begin(), per[cr][1].end());
      sc.a2 = (int)pb.jobs.size();
      pb.jobs.insert(pb.jobs.end(), per[cr][2].begin(), per[cr][2].end());
      sc.a3 = (int)pb.jobs.size();
      pb.step_cta.push_back(sc);
    }
  }
}
}  // namespace hf
