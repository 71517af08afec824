// Serving loop: many solve requests (one problem instance each, with its own
// right-hand sides) admitted into concurrent slots on one GPU, with resident
// factorisations reused across requests of the same problem.  The scheduling
// rules are in serve_sched.h; this file is the CUDA side of it: one host
// worker and one non-blocking CUDA stream per slot, so the work of requests
// that run at the same time overlaps on the device, and the C entry points.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "hfsem_internal.h"
#include "serve_sched.h"

namespace hf {
namespace {

struct Payload {
  std::vector<double> h, rhsdata;
  hfsem_problem prob;
  hfsem_rhs rhs;
  double* X = nullptr;
  hfsem_stats* stats = nullptr;
};

struct Handle {
  hfsem_system* sys = nullptr;
  hfsem_factor* fac = nullptr;
};

class CudaExec : public serve::Executor {
 public:
  CudaExec(int dev, int slots, const hfsem_hopts& o, double tol, int max_iter)
      : dev_(dev), hopts_(o), tol_(tol), max_iter_(max_iter), streams_(slots, nullptr) {}
  ~CudaExec() override {
    cudaSetDevice(dev_);
    for (auto s : streams_)
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
  }
  void thread_init(int slot) override {
    cudaSetDevice(dev_);
    cudaStreamCreateWithFlags(&streams_[slot], cudaStreamNonBlocking);
  }
  int build(int slot, serve::Request& r, void** handle, size_t* bytes) override {
    auto* p = static_cast<Payload*>(r.payload);
    auto* h = new Handle;
    int st = hfsem_assemble(1, &p->prob, streams_[slot], &h->sys);
    if (st == HFSEM_OK) st = hfsem_hlu_factor(h->sys, &hopts_, &h->fac);
    if (st != HFSEM_OK) {
      r.msg = hfsem_last_error();
      release(h);
      return st;
    }
    *handle = h;
    *bytes = system_bytes(h->sys) + factor_bytes(h->fac);
    return HFSEM_OK;
  }
  int solve(int slot, serve::Request& r, void* handle, size_t* bytes) override {
    auto* p = static_cast<Payload*>(r.payload);
    auto* h = static_cast<Handle*>(handle);
    rebind_stream(h->sys, h->fac, streams_[slot]);
    int st = hfsem_solve(h->sys, h->fac, &p->rhs, tol_, max_iter_, p->X, p->stats);
    if (st != HFSEM_OK) r.msg = hfsem_last_error();
    *bytes = system_bytes(h->sys) + factor_bytes(h->fac);
    return st;
  }
  void release(void* handle) override {
    auto* h = static_cast<Handle*>(handle);
    if (!h) return;
    cudaSetDevice(dev_);
    if (h->fac) hfsem_factor_free(h->fac);
    if (h->sys) hfsem_system_free(h->sys);
    delete h;
  }
  bool reusable_after(int status) override {
    return status == HFSEM_OK || status == HFSEM_ERR_NOT_CONVERGED || status == HFSEM_ERR_BREAKDOWN;
  }
  void release_payload(serve::Request& r) override {
    delete static_cast<Payload*>(r.payload);
    r.payload = nullptr;
  }

 private:
  int dev_;
  hfsem_hopts hopts_;
  double tol_;
  int max_iter_;
  std::vector<cudaStream_t> streams_;
};

// FNV-1a over the signature's bytes.
uint64_t hash_sig(const std::vector<double>& v) {
  uint64_t h = 1469598103934665603ull;
  const unsigned char* b = reinterpret_cast<const unsigned char*>(v.data());
  for (size_t i = 0; i < v.size() * sizeof(double); ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Device bytes a request is expected to need, from its sizes: the system
// (element-pair blocks of the dense operator or the Toeplitz symbol), the
// FP32 or FP64 H-matrix factor (leaf blocks, their inverses, low-rank
// factors, the update temporaries and the solve pack) and the solve's work
// vectors.  Used for admission only; resident factorisations are then
// charged what they actually hold.
void estimate(const hfsem_problem& p, int nrhs, const hfsem_hopts& o, bool uniform,
              size_t* build, size_t* work) {
  const double N = p.n_elem, P = p.P, Nd = N * P - 1;
  const double ts = o.precision == HFSEM_PREC_FP64 ? 8.0 : 4.0;
  double L = 1;
  while (L < 2 * N) L *= 2;
  const double leaf = std::min(128.0, std::max(P, std::floor(128.0 / P) * P));
  const double lg = std::max(1.0, std::log2(std::max(2.0, Nd / leaf)));
  // H-matrix operator: near-field pairs plus an FP64 H-matrix of rank 24
  const double hop = 8.0 * Nd * (6.0 * leaf + 6.0 * kHopRank * lg * 2.0) + 16.0 * N * P * P;
  const double sys = uniform                           ? 8.0 * N * P * P + 16.0 * (L + 1) * P * P + 64.0 * N
                     : p.matvec == HFSEM_MATVEC_HMATRIX ? hop
                                                        : 8.0 * P * P * N * (N + 1) / 2 + 64.0 * N;
  const double fac = ts * Nd * (4.0 * leaf + 6.0 * o.R * lg * 4.0) + 4.0 * Nd * 64 + (1 << 20);
  const double vec = 8.0 * Nd * nrhs * 14 + 8.0 * N * P * nrhs * 4;
  const double op = uniform ? 16.0 * 2 * L * P * nrhs : 0.0;   // FFT buffers
  *build = (size_t)(sys + fac);
  *work = (size_t)(vec + op);
}

bool is_uniform(const std::vector<double>& h) {
  for (double x : h)
    if (std::fabs(x - h[0]) > 1e-12 * h[0]) return false;
  return true;
}

}  // namespace
}  // namespace hf

struct hfsem_server_s {
  std::unique_ptr<hf::CudaExec> ex;
  std::unique_ptr<hf::serve::Scheduler> sched;
  hfsem_hopts hopts;
};

using namespace hf;

namespace {
template <class F>
int guard(F&& body) {
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
}  // namespace

extern "C" {

int hfsem_server_create(const hfsem_server_opts* o, hfsem_server** out) {
  return guard([&] {
    if (!o || !out) throw Error(HFSEM_ERR_INVALID_ARG, "NULL argument");
    if (o->slots < 1 || o->slots > 64) throw Error(HFSEM_ERR_INVALID_ARG, "slots must be in [1, 64]");
    if (o->budget_bytes < 0 || o->cache_factors < 0)
      throw Error(HFSEM_ERR_INVALID_ARG, "budget_bytes, cache_factors >= 0");
    if (!(o->tol > 0.0) || o->max_iter < 1) throw Error(HFSEM_ERR_INVALID_ARG, "tol > 0, max_iter >= 1");
    if (o->hopts.R < 1 || o->hopts.R > 32 || !(o->hopts.lambda > 0.0) || !(o->hopts.tol_hlu >= 0.0) ||
        o->hopts.build_only ||
        (o->hopts.admissibility != HFSEM_ADM_MAX && o->hopts.admissibility != HFSEM_ADM_MIN))
      throw Error(HFSEM_ERR_INVALID_ARG, "bad H-LU options");
    int dev = 0;
    HF_CHECK(cudaGetDevice(&dev));
    size_t budget = (size_t)o->budget_bytes;
    if (budget == 0) {
      size_t fr = 0, tot = 0;
      HF_CHECK(cudaMemGetInfo(&fr, &tot));
      budget = (size_t)(0.8 * (double)fr);
    }
    auto* s = new hfsem_server_s;
    s->hopts = o->hopts;
    s->ex.reset(new CudaExec(dev, o->slots, o->hopts, o->tol, o->max_iter));
    s->sched.reset(new serve::Scheduler(s->ex.get(), o->slots, budget, o->cache_factors, HFSEM_ERR_OOM));
    *out = s;
  });
}

int hfsem_server_submit(hfsem_server* s, const hfsem_request* q, int64_t* id) {
  return guard([&] {
    if (!s || !q || !q->prob || !q->rhs || !q->X || !q->stats || !id)
      throw Error(HFSEM_ERR_INVALID_ARG, "NULL argument");
    const hfsem_problem& p = *q->prob;
    const hfsem_rhs& r = *q->rhs;
    if (p.n_elem < 1 || p.n_elem > (1 << 20) || p.P < 1 || p.P > kMaxP || !p.h)
      throw Error(HFSEM_ERR_INVALID_ARG, "bad problem sizes");
    if (r.nrhs < 1 || r.nrhs > 64 || !r.data) throw Error(HFSEM_ERR_INVALID_ARG, "bad right-hand sides");
    size_t count = 0;
    const size_t nd = (size_t)p.n_elem * p.P - 1;
    if (r.kind == HFSEM_RHS_LOAD_VECTOR) {
      count = nd * r.nrhs;
    } else if (r.kind == HFSEM_RHS_FRAC_POWERS) {
      if (r.n_terms < 1 || r.n_terms > 4096) throw Error(HFSEM_ERR_INVALID_ARG, "FRAC_POWERS n_terms");
      count = (size_t)3 * r.n_terms * r.nrhs;
    } else if (r.kind == HFSEM_RHS_LEGENDRE_AB) {
      if (r.n_terms < 1 || r.n_terms > 128) throw Error(HFSEM_ERR_INVALID_ARG, "LEGENDRE_AB n_terms");
      count = (size_t)r.n_terms * r.nrhs;
    } else {
      throw Error(HFSEM_ERR_INVALID_ARG, "unknown rhs kind");
    }
    auto pay = std::make_unique<Payload>();
    pay->h.assign(p.h, p.h + p.n_elem);
    pay->rhsdata.assign(r.data, r.data + count);
    pay->prob = p;
    pay->prob.h = pay->h.data();
    pay->rhs = r;
    pay->rhs.data = pay->rhsdata.data();
    pay->X = q->X;
    pay->stats = q->stats;
    auto req = std::make_unique<serve::Request>();
    // everything the operator and the factorisation depend on (the boundary
    // values only enter the right-hand side)
    req->sig = {(double)p.n_elem, (double)p.P, p.a, p.b, p.alpha, p.theta, p.rho, (double)p.matvec};
    req->sig.insert(req->sig.end(), pay->h.begin(), pay->h.end());
    req->key = hash_sig(req->sig);
    estimate(p, r.nrhs, s->hopts, is_uniform(pay->h), &req->est_build, &req->est_work);
    req->payload = pay.release();
    *id = s->sched->submit(std::move(req));
  });
}

int hfsem_server_poll(hfsem_server* s, int32_t max, hfsem_done* out, int32_t* n) {
  return guard([&] {
    if (!s || !out || !n || max < 1) throw Error(HFSEM_ERR_INVALID_ARG, "bad arguments");
    auto d = s->sched->poll(max);
    for (size_t i = 0; i < d.size(); ++i) {
      hfsem_done& o = out[i];
      o.id = d[i].id;
      o.status = d[i].status;
      o.reused = d[i].reused;
      o.t_submit = d[i].t_submit;
      o.t_start = d[i].t_start;
      o.t_done = d[i].t_done;
      std::strncpy(o.msg, d[i].msg.c_str(), sizeof(o.msg) - 1);
      o.msg[sizeof(o.msg) - 1] = '\0';
    }
    *n = (int32_t)d.size();
  });
}

int hfsem_server_drain(hfsem_server* s) {
  return guard([&] {
    if (!s) throw Error(HFSEM_ERR_INVALID_ARG, "NULL server");
    s->sched->drain();
  });
}

int hfsem_server_counters_read(hfsem_server* s, hfsem_server_counters* c) {
  return guard([&] {
    if (!s || !c) throw Error(HFSEM_ERR_INVALID_ARG, "NULL argument");
    auto k = s->sched->counters();
    c->resident_bytes = (int64_t)k.resident;
    c->inflight_bytes = (int64_t)k.inflight;
    c->budget_bytes = (int64_t)k.budget;
    c->peak_bytes = (int64_t)k.peak_bytes;
    c->running = k.running;
    c->peak_running = k.peak_running;
    c->cached = k.cached;
    c->queued = k.queued;
    c->builds = k.builds;
    c->reuses = k.reuses;
    c->evictions = k.evictions;
    c->rejected = k.rejected;
  });
}

void hfsem_server_free(hfsem_server* s) {
  if (!s) return;
  try {
    s->sched->drain();
    s->sched->shutdown();
    s->sched.reset();
    s->ex.reset();
  } catch (...) {
  }
  delete s;
}

}  // extern "C"
