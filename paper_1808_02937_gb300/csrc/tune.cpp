// Autotuner of the H-LU leaf size.  Sec. 4.1 builds the H-matrix on a
// cluster tree whose leaf size it leaves open; the kernels here take leaves
// of up to 128 unknowns (96 in FP64).  Small leaves mean more low-rank
// blocks and longer op programs (the factorisation is latency-bound), large
// ones more dense work per op and larger leaf LUs; which is faster depends on
// the mesh, P and the arithmetic.  The tuner times the candidates on the
// caller's own instances and keeps the winner per class in a process-wide
// table that the factorisation consults when leaf_elems is 0.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "hfsem_internal.h"

namespace hf {
namespace {

using Key = std::tuple<int, int, int>;   // (fp64, kind, P)

std::mutex g_mu;
std::map<Key, int> g_table;   // class -> leaf size in unknowns

// the factor arithmetic an instance gets for a requested precision (meshes
// whose element sizes span more than 1e45 are factored in FP64)
int fp64_of(const InstHost& I, int precision) {
  const double hmax = *std::max_element(I.h.begin(), I.h.end());
  const double hmin = *std::min_element(I.h.begin(), I.h.end());
  return (precision == HFSEM_PREC_FP64 || hmax > 1e45 * hmin) ? 1 : 0;
}

Key key_of(const InstHost& I, int precision) {
  return Key{fp64_of(I, precision), I.uniform ? 0 : 1, I.P};
}

int matvec_of(const InstHost& I) {
  return I.kind == kToeplitz ? HFSEM_MATVEC_TOEPLITZ
                             : (I.kind == kHmat ? HFSEM_MATVEC_HMATRIX : HFSEM_MATVEC_DENSE);
}

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    HF_CHECK(cudaEventCreate(&a));
    HF_CHECK(cudaEventCreate(&b));
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  void start() { HF_CHECK(cudaEventRecord(a, st)); }
  float stop() {
    HF_CHECK(cudaEventRecord(b, st));
    HF_CHECK(cudaEventSynchronize(b));
    float ms = 0.f;
    HF_CHECK(cudaEventElapsedTime(&ms, a, b));
    return ms;
  }
};

void write_table(const char* path) {
  FILE* fp = std::fopen(path, "w");
  if (!fp) throw Error(HFSEM_ERR_INVALID_ARG, "cannot write the tuning table");
  std::fprintf(fp, "# hfsem leaf-size table: fp64 kind(0 uniform, 1 other) P leaf_unknowns\n");
  for (auto& kv : g_table)
    std::fprintf(fp, "%d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), kv.second);
  std::fclose(fp);
}

}  // namespace

int tune_leaf_dofs(const InstHost& I, int precision) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(key_of(I, precision));
  return it == g_table.end() ? 0 : it->second;
}

}  // namespace hf

using namespace hf;

extern "C" int hfsem_tune(hfsem_system* sys, const hfsem_hopts* opts, const hfsem_rhs* rhs, double tol,
                          int32_t max_iter, const char* path, hfsem_tune_entry* out, int32_t cap,
                          int32_t* n_out) {
  try {
    if (!sys || !opts || !rhs) throw Error(HFSEM_ERR_INVALID_ARG, "NULL argument");
    if (opts->build_only) throw Error(HFSEM_ERR_INVALID_ARG, "build_only factors cannot be tuned");
    if (cap < 0 || (cap > 0 && !out)) throw Error(HFSEM_ERR_INVALID_ARG, "out must hold cap entries");
    const int nrhs = rhs[0].nrhs;
    for (int i = 0; i < sys->n_inst; ++i)
      if (rhs[i].nrhs != nrhs) throw Error(HFSEM_ERR_INVALID_ARG, "every instance needs the same nrhs");
    // classes and their instances: kTuneInst per class, the class's own
    // instances in order, repeated when it has fewer, so that every timing
    // run launches the way a large batch does (clusters of 4 CTAs for the
    // H-LU program, one cluster per instance for the H-solves)
    constexpr int kTuneInst = 32;
    std::map<Key, std::vector<int>> cls;
    for (int i = 0; i < sys->n_inst; ++i) {
      auto& v = cls[key_of(sys->ih[i], opts->precision)];
      if ((int)v.size() < kTuneInst) v.push_back(i);
    }
    for (auto& kv : cls)
      for (size_t k = 0, n0 = kv.second.size(); kv.second.size() < (size_t)kTuneInst; ++k)
        kv.second.push_back(kv.second[k % n0]);
    std::vector<hfsem_tune_entry> res;
    Timer tm(sys->st);
    for (auto& kv : cls) {
      const int fp64 = std::get<0>(kv.first), P = std::get<2>(kv.first);
      const std::vector<int>& ids = kv.second;
      std::vector<hfsem_problem> probs(ids.size());
      std::vector<hfsem_rhs> rs(ids.size());
      for (size_t k = 0; k < ids.size(); ++k) {
        const InstHost& I = sys->ih[ids[k]];
        hfsem_problem& p = probs[k];
        std::memset(&p, 0, sizeof(p));
        p.n_elem = I.N;
        p.P = I.P;
        p.a = I.a;
        p.b = I.b;
        p.h = I.h.data();
        p.alpha = I.alpha;
        p.theta = I.theta;
        p.rho = I.rho;
        p.c1 = I.c1;
        p.c2 = I.c2;
        p.matvec = matvec_of(I);
        rs[k] = rhs[ids[k]];
      }
      hfsem_system* sub = nullptr;
      int e = hfsem_assemble((int32_t)probs.size(), probs.data(), sys->st, &sub);
      if (e != HFSEM_OK) return e;
      // the tuning system is freed on every way out of this class
      std::unique_ptr<hfsem_system, void (*)(hfsem_system*)> own(sub, hfsem_system_free);
      int nd = 0;
      for (int i : ids) nd += sys->ih[i].Nd;
      std::vector<double> X((size_t)nd * nrhs);
      std::vector<hfsem_stats> st(ids.size() * nrhs);
      // candidates in unknowns per leaf; the automatic size is the largest
      const int cap_dofs = fp64 ? 96 : 128;
      std::vector<int> cand;
      for (int d : {32, 48, 64, 96, 128})
        if (d <= cap_dofs) {
          const int el = std::max(1, d / P);
          if (cand.empty() || std::max(1, cand.back() / P) != el) cand.push_back(d);
        }
      int best = 0, best_it = 1 << 30;
      double best_ms = 1e300, auto_ms = 0.0;
      std::vector<std::pair<int, std::pair<double, int>>> tried;
      for (int d : cand) {
        hfsem_hopts o = *opts;
        o.leaf_elems = std::max(1, d / P);
        double ms = 0.0;
        int iters = 0;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {   // the first builds the plans
          hfsem_factor* f = nullptr;
          tm.start();
          int ef = hfsem_hlu_factor(sub, &o, &f);
          float fms = tm.stop();
          if (ef != HFSEM_OK) {
            ok = false;
            break;
          }
          std::unique_ptr<hfsem_factor, void (*)(hfsem_factor*)> fown(f, hfsem_factor_free);
          tm.start();
          int es = hfsem_solve(sub, f, rs.data(), tol, max_iter, X.data(), st.data());
          float sms = tm.stop();
          fown.reset();
          if (es != HFSEM_OK) {
            ok = false;
            break;
          }
          ms = fms + sms;
          iters = 0;
          for (auto& s : st) iters = std::max(iters, (int)s.iters);
        }
        if (!ok) continue;   // a size the kernels cannot take, or no convergence
        tried.push_back({d, {ms, iters}});
        if (d == cand.back()) auto_ms = ms;
        best_it = std::min(best_it, iters);
      }
      // fastest among the sizes within one iteration of the fewest
      for (auto& t : tried)
        if (t.second.second <= best_it + 1 && t.second.first < best_ms) {
          best_ms = t.second.first;
          best = t.first;
        }
      own.reset();
      if (best > 0) {
        {
          std::lock_guard<std::mutex> lk(g_mu);
          g_table[kv.first] = best;
        }
        hfsem_tune_entry te;
        te.fp64 = fp64;
        te.kind = std::get<1>(kv.first);
        te.P = P;
        te.leaf_dofs = best;
        te.n_inst = (int32_t)ids.size();
        te.ms = best_ms;
        te.ms_default = auto_ms;
        res.push_back(te);
      }
    }
    if (path) {
      std::lock_guard<std::mutex> lk(g_mu);
      write_table(path);
    }
    if (n_out) *n_out = (int32_t)res.size();
    for (int k = 0; k < cap && k < (int)res.size(); ++k) out[k] = res[k];
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

extern "C" int hfsem_tune_load(const char* path) {
  try {
    if (!path) throw Error(HFSEM_ERR_INVALID_ARG, "NULL path");
    FILE* fp = std::fopen(path, "r");
    if (!fp) throw Error(HFSEM_ERR_INVALID_ARG, "cannot read the tuning table");
    std::map<Key, int> t;
    char line[256];
    bool bad = false;
    while (std::fgets(line, sizeof(line), fp)) {
      if (line[0] == '#' || line[0] == '\n') continue;
      int a, k, P, d;
      if (std::sscanf(line, "%d %d %d %d", &a, &k, &P, &d) != 4 || (a != 0 && a != 1) ||
          (k != 0 && k != 1) || P < 1 || P > kMaxP || d < 1 || d > 128) {
        bad = true;
        break;
      }
      t[Key{a, k, P}] = d;
    }
    std::fclose(fp);
    if (bad) throw Error(HFSEM_ERR_INVALID_ARG, "malformed tuning table");
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : t) g_table[kv.first] = kv.second;
    return HFSEM_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.code;
  }
}

extern "C" int hfsem_tune_lookup(int32_t fp64, int32_t kind, int32_t P, int32_t* leaf_dofs) {
  if (!leaf_dofs) {
    set_last_error("NULL leaf_dofs");
    return HFSEM_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(Key{fp64 ? 1 : 0, kind ? 1 : 0, P});
  *leaf_dofs = it == g_table.end() ? 0 : it->second;
  return HFSEM_OK;
}

extern "C" int hfsem_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
  return HFSEM_OK;
}
