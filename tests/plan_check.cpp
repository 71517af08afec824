// Host-side check of the planner's output, independent of its own conflict
// model (which works on rectangles): for one mesh read from stdin,
//   * the leaf blocks of the block tree cover the N_d x N_d matrix exactly
//     once, and every low-rank block is admissible in the sense of Sec. 3.1,
//     max (or min) (diam tau, diam sigma) <= lambda dist(tau, sigma), with the supports
//     of the clusters' basis functions derived here from their unknowns;
//   * within each wave of the H-LU program (ops that the CTAs of a cluster
//     run concurrently) no op writes an arena element, or the rank of a
//     low-rank slot, that another op of the wave reads or writes, every
//     footprint taken element by element with runtime ranks at the slot's
//     capacity;
//   * the waves partition the program;
//   * the leaf-solve tables stay inside the arena and the shared-memory budget.
// Input: N P leaf_elems R lambda mode rule, then N element lengths (rule 0:
// max(diam) <= lambda dist, rule 1: min(diam) <= lambda dist); mode 1 checks
// the whole program as if it were one wave (the verifier's own test: the H-LU
// has dependencies, so that must fail).  Prints "OK ..." or the first
// violation ("FAIL ...") and exits non-zero.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <unordered_map>
#include <vector>

#include "hplan.h"

using namespace hf;

namespace {

int fail(const char* what, long long a = 0, long long b = 0, long long c = 0) {
  std::printf("FAIL %s %lld %lld %lld\n", what, a, b, c);
  std::exit(1);
}

long long dim_bound(const HPlan& p, int d) {
  if (d >= 0) return d;
  const int s = -1 - d;
  if (s == p.n_slots) return p.nrhs_max;
  return p.B[p.lr_blocks[s]].kcap;
}

struct Foot {
  std::vector<long long> rd, wr;   // arena elements
  std::vector<int> rrk, wrk;       // slot ranks
};

void view(const HPlan& p, const View& v, std::vector<long long>& out, std::vector<int>& rk) {
  if (v.r < 0) rk.push_back(-1 - v.r);
  if (v.c < 0) rk.push_back(-1 - v.c);
  const long long r = dim_bound(p, v.r), c = dim_bound(p, v.c);
  for (long long j = 0; j < c; ++j)
    for (long long i = 0; i < r; ++i) out.push_back(v.tr ? v.off + j + i * v.ld : v.off + i + j * v.ld);
}

void slot_storage(const HPlan& p, int slot, std::vector<long long>& out) {
  const Block& b = p.B[p.lr_blocks[slot]];
  const long long n = (long long)(b.m + b.n) * b.kcap;
  for (long long t = 0; t < n; ++t) out.push_back(b.off + t);
}

Foot footprint(const HPlan& p, const HOp& o) {
  Foot f;
  switch (o.type) {
    case OP_GEMM:
      view(p, o.A, f.rd, f.rrk);
      view(p, o.B, f.rd, f.rrk);
      if (o.beta != 0.0) view(p, o.C, f.rd, f.rrk);
      view(p, o.C, f.wr, f.rrk);
      break;
    case OP_GETRF_INV:
      view(p, o.C, f.rd, f.rrk);
      view(p, o.C, f.wr, f.rrk);
      view(p, o.A, f.wr, f.rrk);
      view(p, o.B, f.wr, f.rrk);
      break;
    case OP_TRMM_L:
    case OP_TRMM_R:
      view(p, o.A, f.rd, f.rrk);
      view(p, o.C, f.rd, f.rrk);
      view(p, o.C, f.wr, f.rrk);
      break;
    case OP_APPEND:
      view(p, o.A, f.rd, f.rrk);
      if (o.B.off >= 0) view(p, o.B, f.rd, f.rrk);
      slot_storage(p, o.slot, f.rd);
      slot_storage(p, o.slot, f.wr);
      f.rrk.push_back(o.slot);
      f.wrk.push_back(o.slot);
      break;
    case OP_TRUNC:
      slot_storage(p, o.slot, f.rd);
      slot_storage(p, o.slot, f.wr);
      f.rrk.push_back(o.slot);
      f.wrk.push_back(o.slot);
      break;
    case OP_ZERO:
      view(p, o.C, f.wr, f.rrk);
      break;
    case OP_AXPY:
      view(p, o.A, f.rd, f.rrk);
      view(p, o.C, f.rd, f.rrk);
      view(p, o.C, f.wr, f.rrk);
      break;
    default:
      fail("unknown op type", o.type);
  }
  for (long long e : f.rd)
    if (e < 0 || e >= p.arena) fail("read outside the arena", e, p.arena);
  for (long long e : f.wr)
    if (e < 0 || e >= p.arena) fail("write outside the arena", e, p.arena);
  return f;
}

}  // namespace

int main() {
  int N, P, leaf, R, mode, rule;
  double lambda;
  if (std::scanf("%d %d %d %d %lf %d %d", &N, &P, &leaf, &R, &lambda, &mode, &rule) != 7)
    return fail("input");
  InstHost I{};
  I.N = N;
  I.P = P;
  I.Nd = N * P - 1;
  I.h.resize(N);
  for (int i = 0; i < N; ++i)
    if (std::scanf("%lf", &I.h[i]) != 1) return fail("input h");
  I.dl.assign(N + 1, 0.0);
  I.dr.assign(N + 1, 0.0);
  for (int k = 0; k < N; ++k) I.dl[k + 1] = I.dl[k] + I.h[k];
  for (int k = N - 1; k >= 0; --k) I.dr[k] = I.dr[k + 1] + I.h[k];
  PlanOpts o{lambda, leaf, R, R, 64, 160, 128};
  o.unique_tmp = 1;
  o.ncta = 8;
  o.adm_min = rule;
  HPlan p;
  make_plan(I, o, p);

  // ---- block tree: exact cover and admissibility ----
  const int Nd = I.Nd;
  // node positions as distances to a (prefix sums) and to b (suffix sums):
  // a difference of nodes is taken from whichever is smaller, so meshes
  // refined far below the rounding of 1 keep their element sizes
  std::vector<double> da(N + 1, 0.0), db(N + 1, 0.0);
  for (int k = 0; k < N; ++k) da[k + 1] = da[k] + I.h[k];
  for (int k = N - 1; k >= 0; --k) db[k] = db[k + 1] + I.h[k];
  auto diff = [&](int i, int j) {   // x_i - x_j, i >= j
    return (da[i] <= db[j]) ? da[i] - da[j] : db[j] - db[i];
  };
  auto support = [&](const Cluster& c, int& lo, int& hi) {   // node indices
    lo = N + 1;
    hi = -1;
    for (int u = c.d0; u < c.d1; ++u) {
      const int e = u / P, q = u % P;
      lo = std::min(lo, e);
      hi = std::max(hi, (q < P - 1) ? e + 1 : std::min(e + 2, N));
    }
  };
  std::vector<unsigned char> cover((size_t)Nd * Nd, 0);
  int n_lr = 0;
  for (const Block& b : p.B) {
    if (b.type == B_HIER) continue;
    const Cluster &t = p.C[b.t], &s = p.C[b.s];
    if (b.m != t.d1 - t.d0 || b.n != s.d1 - s.d0) fail("block size", b.m, b.n);
    for (int i = t.d0; i < t.d1; ++i)
      for (int j = s.d0; j < s.d1; ++j)
        if (cover[(size_t)i * Nd + j]++) fail("entry covered twice", i, j);
    if (b.type == B_LR) {
      ++n_lr;
      int tl, th, sl, sh;
      support(t, tl, th);
      support(s, sl, sh);
      const double dist = (sl > th) ? diff(sl, th) : (tl > sh) ? diff(tl, sh) : 0.0;
      const double dt = diff(th, tl), ds = diff(sh, sl);
      const double diam = rule ? std::min(dt, ds) : std::max(dt, ds);
      if (!(dist > 0.0) || diam > lambda * dist * (1.0 + 1e-9)) fail("inadmissible low-rank block", b.t, b.s);
    }
  }
  for (size_t k = 0; k < cover.size(); ++k)
    if (!cover[k]) fail("entry not covered", (long long)(k / Nd), (long long)(k % Nd));

  // ---- waves: partition and no conflicts within a wave ----
  const std::vector<int> w = (mode == 1) ? std::vector<int>{0, (int)p.fac.size()} : p.fac_waves;
  if (w.empty() || w.front() != 0 || w.back() != (int)p.fac.size()) fail("waves do not span the program");
  for (size_t k = 1; k < w.size(); ++k)
    if (w[k] <= w[k - 1]) fail("empty or unordered wave", (long long)k);
  long long checked = 0;
  for (size_t k = 0; k + 1 < w.size(); ++k) {
    std::unordered_map<long long, int> writer;
    std::unordered_map<int, int> rank_writer;
    std::vector<Foot> fs;
    for (int i = w[k]; i < w[k + 1]; ++i) fs.push_back(footprint(p, p.fac[i]));
    for (size_t a = 0; a < fs.size(); ++a) {
      for (long long e : fs[a].wr) {
        auto it = writer.find(e);
        if (it != writer.end() && it->second != (int)a) fail("two writers in one wave", (long long)k, e);
        writer[e] = (int)a;
      }
      for (int s : fs[a].wrk) {
        auto it = rank_writer.find(s);
        if (it != rank_writer.end() && it->second != (int)a) fail("two rank writers in one wave", (long long)k, s);
        rank_writer[s] = (int)a;
      }
    }
    for (size_t a = 0; a < fs.size(); ++a) {
      for (long long e : fs[a].rd) {
        auto it = writer.find(e);
        if (it != writer.end() && it->second != (int)a) fail("read of an element written in the same wave", (long long)k, e);
        ++checked;
      }
      for (int s : fs[a].rrk) {
        auto it = rank_writer.find(s);
        if (it != rank_writer.end() && it->second != (int)a) fail("rank read while written in the same wave", (long long)k, s);
      }
    }
  }

  // ---- leaf-solve tables ----
  const size_t budget = 232448 - 1024;
  LeafSolve ls;
  build_leaf_solve(p, 8, budget, 4, 4, ls);
  if (ls.step_cta.size() != ls.steps.size() * 8) fail("step table size");
  for (const StepCta& sc : ls.step_cta)
    if (!(0 <= sc.a0 && sc.a0 <= sc.a1 && sc.a1 <= sc.a2 && sc.a2 <= sc.a3 && sc.a3 <= (int)ls.jobs.size()))
      fail("step job range", sc.a0, sc.a3);
  for (const SolJob& j : ls.jobs) {
    if (j.kind < 0 || j.kind > 4) fail("job kind", j.kind);
    if (j.n < 0 || j.n > ls.nmax) fail("job length", j.n);
    if (j.src < 0 || j.src + j.n > p.arena) fail("job outside the arena", j.src, j.n);
  }
  for (const StepInfo& st : ls.steps)
    if (st.d0 < 0 || st.n < 0 || st.d0 + st.n > Nd) fail("step rows", st.d0, st.n);
  if (solve_smem(ls.jcap, ls.nmax, ls.wcols, 4, 4) > budget) fail("leaf solve over the budget");

  std::printf("OK blocks %zu lr %d ops %zu waves %zu reads %lld jobs %zu\n", p.B.size(), n_lr,
              p.fac.size(), w.size() - 1, checked, ls.jobs.size());
  return 0;
}
