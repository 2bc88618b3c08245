// extern "C" boundary of the TDDFT-ris engine (declared in include/ris.h).
#include <string.h>

#include <atomic>
#include <mutex>
#include <memory>

#include "engine.cuh"

struct ris_ctx {
  ris::Engine eng;
};

namespace ris {
std::atomic<long long> g_launches{0};
std::atomic<long long> g_allocs{0};

namespace {
struct Rec {
  int cls;
  cudaStream_t st;
  cudaEvent_t a, b;
  double work;
};
// Profiling is per context: a context created with the profile option
// registers the streams it launches on, kernel classes are timed only on
// registered streams, and a context collects only its own streams' records.
std::mutex g_prof_mu;
std::atomic<int> g_prof_n{0};  // registered streams
std::vector<cudaStream_t> g_prof_streams;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  RIS_CUDA(cudaEventCreate(&e));
  return e;
}
bool profiled(cudaStream_t st) {
  for (cudaStream_t s : g_prof_streams)
    if (s == st) return true;
  return false;
}
// Takes the records of the given streams out of the list (events waited on).
void take_recs(const cudaStream_t* sts, int n, double* ms, double* work) {
  std::vector<Rec> keep;
  for (auto& r : g_recs) {
    bool mine = false;
    for (int i = 0; i < n; i++) mine = mine || (sts[i] && r.st == sts[i]);
    if (!mine) {
      keep.push_back(r);
      continue;
    }
    RIS_CUDA(cudaEventSynchronize(r.a));
    if (r.b) {
      RIS_CUDA(cudaEventSynchronize(r.b));
      float t = 0.f;
      RIS_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
      if (ms) ms[r.cls] += t;
      if (work) work[r.cls] += r.work;
      g_pool.push_back(r.b);
    }
    g_pool.push_back(r.a);
  }
  g_recs.swap(keep);
}
}  // namespace

void prof_attach(cudaStream_t st) {
  if (!st) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_streams.push_back(st);
  ++g_prof_n;
}
void prof_detach(cudaStream_t st) {
  if (!st) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto it = g_prof_streams.begin(); it != g_prof_streams.end(); ++it)
    if (*it == st) {
      g_prof_streams.erase(it);
      --g_prof_n;
      break;
    }
  if (!profiled(st)) {
    try {
      take_recs(&st, 1, nullptr, nullptr);
    } catch (const Error&) {
    }
  }
}
void prof_begin(int cls, cudaStream_t st) {
  if (g_prof_n.load() == 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!profiled(st)) return;
  Rec r{cls, st, take_event(), nullptr, 0.0};
  RIS_CUDA(cudaEventRecord(r.a, st));
  g_recs.push_back(r);
}
void prof_end(int cls, cudaStream_t st, double work) {
  if (g_prof_n.load() == 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto it = g_recs.rbegin(); it != g_recs.rend(); ++it)
    if (it->cls == cls && it->st == st && it->b == nullptr) {
      it->b = take_event();
      it->work = work;
      RIS_CUDA(cudaEventRecord(it->b, st));
      return;
    }
}
void prof_collect(const cudaStream_t* sts, int n, double* ms, double* work) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int c = 0; c < kProfN; c++) ms[c] = work[c] = 0.0;
  take_recs(sts, n, ms, work);
}
}  // namespace ris

namespace {

template <class F>
ris_status guarded(ris_ctx* ctx, F&& f) {
  if (!ctx) return RIS_ERR_ARG;
  struct TrackScope {  // route this thread's allocations to the context
    ris::MemTrack* prev;
    explicit TrackScope(ris::MemTrack* t) : prev(ris::t_track) { ris::t_track = t; }
    ~TrackScope() { ris::t_track = prev; }
  } scope(&ctx->eng.mem);
  try {
    RIS_CUDA(cudaSetDevice(ctx->eng.device));
    f();
    ctx->eng.err.clear();
    return RIS_OK;
  } catch (const ris::Error& e) {
    ctx->eng.err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    ctx->eng.err = e.what();
    return RIS_ERR_ARG;
  }
}

struct StageTimer {
  ris::Engine& e;
  int slot;
  StageTimer(ris::Engine& e_, int s) : e(e_), slot(s) { RIS_CUDA(cudaEventRecord(e.ev0, e.st)); }
  void stop() {
    RIS_CUDA(cudaEventRecord(e.ev1, e.st));
    RIS_CUDA(cudaEventSynchronize(e.ev1));
    float ms = 0.f;
    RIS_CUDA(cudaEventElapsedTime(&ms, e.ev0, e.ev1));
    e.stats[slot] = ms;
  }
};

}  // namespace

extern "C" {

ris_status ris_options_default(ris_options* opt) {
  if (!opt) return RIS_ERR_ARG;
  memset(opt, 0, sizeof(*opt));
  opt->precision = RIS_FP64;
  opt->rpa = 0;
  opt->cx = 0.25;
  opt->conv_tol = 1e-10;
  opt->max_iter = 100;
  opt->max_subspace = 0;
  opt->screen_thr = 1e-14;
  opt->mem_budget = 0;
  opt->occ_block = 0;
  opt->cuda_stream = nullptr;
  opt->device = 0;
  opt->profile = 0;
  opt->mixed_tol = 1e-6;
  opt->refine = 0;
  opt->precond = 0;
  opt->mo_window = 0.0;
  opt->deriv_prefetch = 1;
  opt->emu_f64 = 1;
  opt->eig_fp32 = 0;
  opt->stream = 0;
  opt->stream_block = 0;
  opt->subspace_ff = 1;
  return RIS_OK;
}

ris_status ris_create(ris_ctx** out, const ris_options* opt) {
  if (!out) return RIS_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<ris_ctx> c(new (std::nothrow) ris_ctx());
  if (!c) return RIS_ERR_OOM;
  ris_options o;
  ris_options_default(&o);
  if (opt) o = *opt;
  if (o.precision != RIS_FP64 && o.precision != RIS_MIXED) return RIS_ERR_ARG;
  if (!(o.conv_tol > 0) || o.max_iter <= 0 || !(o.screen_thr >= 0)) return RIS_ERR_ARG;
  if (o.precision == RIS_MIXED && !(o.mixed_tol > 0)) return RIS_ERR_ARG;
  if (o.precond != 0 && o.precond != 1) return RIS_ERR_ARG;
  if (!(o.mo_window >= 0.0)) return RIS_ERR_ARG;
  if (o.deriv_prefetch != 0 && o.deriv_prefetch != 1) return RIS_ERR_ARG;
  if (o.emu_f64 != 0 && o.emu_f64 != 1) return RIS_ERR_ARG;
  if (o.eig_fp32 != 0 && o.eig_fp32 != 1) return RIS_ERR_ARG;
  c->eng.opt = o;
  c->eng.device = o.device;
  ris_status s = guarded(c.get(), [&] {
    if (o.cuda_stream) {
      c->eng.st = (cudaStream_t)o.cuda_stream;
      c->eng.own_stream = false;
    } else {
      RIS_CUDA(cudaStreamCreateWithFlags(&c->eng.st, cudaStreamNonBlocking));
      c->eng.own_stream = true;
    }
    // keep freed stream-ordered allocations in the pool between calls
    cudaMemPool_t pool;
    RIS_CUDA(cudaDeviceGetDefaultMemPool(&pool, o.device));
    uint64_t thr = UINT64_MAX;
    RIS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    RIS_CUDA(cudaEventCreate(&c->eng.ev0));
    RIS_CUDA(cudaEventCreate(&c->eng.ev1));
    if (o.deriv_prefetch) {
      int lo = 0, hi = 0;
      RIS_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      RIS_CUDA(cudaStreamCreateWithPriority(&c->eng.st2, cudaStreamNonBlocking, lo));
      RIS_CUDA(cudaEventCreateWithFlags(&c->eng.evA, cudaEventDisableTiming));
      RIS_CUDA(cudaEventCreateWithFlags(&c->eng.evD, cudaEventDisableTiming));
    }
    if (o.profile) {
      ris::prof_attach(c->eng.st);
      ris::prof_attach(c->eng.st2);
    }
  });
  if (s != RIS_OK) return s;
  *out = c.release();
  return RIS_OK;
}

ris_status ris_build_aux(ris_ctx* ctx, int natm, const double* coords, int nshell,
                         const ris_shell* ao, int nJ, const ris_shell* auxJ, int nK,
                         const ris_shell* auxK) {
  return guarded(ctx, [&] {
    StageTimer t(ctx->eng, 0);
    ctx->eng.build_aux(natm, coords, nshell, ao, nJ, auxJ, nK, auxK);
    t.stop();
  });
}

ris_status ris_build_B(ris_ctx* ctx, int nao, int nmo, int nocc, const double* C,
                       const double* mo_energy) {
  return guarded(ctx, [&] {
    StageTimer t(ctx->eng, 1);
    ctx->eng.build_B(nao, nmo, nocc, C, mo_energy);
    t.stop();
  });
}

ris_status ris_excite(ris_ctx* ctx, int nstates, double* omega, double* X, double* Y) {
  return guarded(ctx, [&] {
    StageTimer t(ctx->eng, 2);
    ctx->eng.excite(nstates, omega, X, Y);
    t.stop();
  });
}

ris_status ris_apply(ris_ctx* ctx, int nvec, const double* X, double* out, double* out2) {
  return guarded(ctx, [&] { ctx->eng.apply(nvec, X, out, out2); });
}

ris_status ris_excite_guess(ris_ctx* ctx, int nstates, const double* X_guess, double* omega,
                            double* X, double* Y) {
  return guarded(ctx, [&] {
    RIS_REQUIRE(X_guess, RIS_ERR_ARG, "X_guess is NULL");
    StageTimer t(ctx->eng, 2);
    ctx->eng.excite(nstates, omega, X, Y, X_guess);
    t.stop();
  });
}

ris_status ris_phase_align(ris_ctx* ctx, int nstates, const double* X_prev, int* sign,
                           double* X_out) {
  return guarded(ctx, [&] { ctx->eng.phase_align(nstates, X_prev, sign, X_out); });
}

ris_status ris_time_coupling(ris_ctx* ctx, int npair, const double* nac, const double* velocity,
                             double* T) {
  return guarded(ctx, [&] { ctx->eng.time_coupling(npair, nac, velocity, T); });
}

ris_status ris_zvector(ris_ctx* ctx, int nrhs, const double* rhs, double* Z) {
  return guarded(ctx, [&] {
    StageTimer t(ctx->eng, 2);
    ctx->eng.zvector(nrhs, rhs, Z);
    t.stop();
  });
}

ris_status ris_gradient(ris_ctx* ctx, int n, const int* states, int nx, const double* X_in,
                        const double* Y_in, double* grad) {
  return guarded(ctx, [&] {
    ris::Engine& e = ctx->eng;
    RIS_REQUIRE(n >= 1 && states && grad, RIS_ERR_ARG, "bad gradient arguments");
    StageTimer t(e, 3);
    std::vector<int> pairs(2 * n);
    for (int k = 0; k < n; k++) pairs[2 * k] = pairs[2 * k + 1] = states[k];
    ris::SBuf<double> out((size_t)n * e.natm * 3, e.st);
    e.pair_derivs(n, pairs.data(), nx, X_in, Y_in, out.p);
    RIS_CUDA(cudaMemcpyAsync(grad, out.p, sizeof(double) * n * e.natm * 3, cudaMemcpyDefault, e.st));
    t.stop();
  });
}

ris_status ris_nac(ris_ctx* ctx, int npair, const int* pairs, int nx, const double* X_in,
                   const double* Y_in, const double* omega_in, double* nac, double* numerator) {
  bool degenerate = false;
  ris_status s = guarded(ctx, [&] {
    ris::Engine& e = ctx->eng;
    RIS_REQUIRE(npair >= 1 && pairs && nac, RIS_ERR_ARG, "bad coupling arguments");
    std::vector<double> om;
    if (X_in) {
      RIS_REQUIRE(omega_in, RIS_ERR_ARG, "omega_in is required with X_in");
      om.resize(nx);
      ris::copy_to_host(om.data(), omega_in, nx, e.st);
    } else {
      RIS_REQUIRE(e.stage >= 3, RIS_ERR_STATE, "no amplitudes: call ris_excite or pass X_in");
      om = e.h_omega;
      nx = e.nstates;
    }
    std::vector<double> den(npair);
    for (int g = 0; g < npair; g++) {
      const int I = pairs[2 * g], J = pairs[2 * g + 1];
      RIS_REQUIRE(I >= 0 && I < nx && J >= 0 && J < nx, RIS_ERR_ARG, "state index out of range");
      den[g] = om[J] - om[I];
      if (!(fabs(den[g]) >= 1e-8)) degenerate = true;
    }
    StageTimer t(e, 3);
    const size_t per = (size_t)e.natm * 3;
    ris::SBuf<double> num(npair * per, e.st), res(npair * per, e.st), dd(npair, e.st);
    e.pair_derivs(npair, pairs, nx, X_in, Y_in, num.p);
    if (numerator)
      RIS_CUDA(cudaMemcpyAsync(numerator, num.p, sizeof(double) * npair * per, cudaMemcpyDefault, e.st));
    if (!degenerate) {
      RIS_CUDA(cudaMemcpyAsync(dd.p, den.data(), sizeof(double) * npair, cudaMemcpyHostToDevice, e.st));
      ris::divide_pairs(res.p, num.p, dd.p, npair, (int)per, e.st);
      RIS_CUDA(cudaMemcpyAsync(nac, res.p, sizeof(double) * npair * per, cudaMemcpyDefault, e.st));
    }
    t.stop();
  });
  if (s == RIS_OK && degenerate) {
    ctx->eng.err = "|omega_J - omega_I| < 1e-8 for a requested pair";
    return RIS_ERR_DEGENERATE;
  }
  return s;
}

ris_status ris_get_mo_window(const ris_ctx* ctx, int* first_occ, int* nocc_act, int* nvir_act) {
  if (!ctx) return RIS_ERR_ARG;
  const ris::Engine& e = ctx->eng;
  if (first_occ) *first_occ = e.first_occ;
  if (nocc_act) *nocc_act = e.nocc;
  if (nvir_act) *nvir_act = e.nvir;
  return RIS_OK;
}

ris_status ris_get_dims(const ris_ctx* ctx, int* natm, int* nao, int* nocc, int* nauxJ,
                        int* nauxK, int* npairs) {
  if (!ctx) return RIS_ERR_ARG;
  const ris::Engine& e = ctx->eng;
  if (natm) *natm = e.natm;
  if (nao) *nao = e.ao.nfun;
  if (nocc) *nocc = e.nocc;
  if (nauxJ) *nauxJ = e.nJ;
  if (nauxK) *nauxK = e.nK;
  if (npairs) *npairs = e.pl.npair;
  return RIS_OK;
}

ris_status ris_get_stats(const ris_ctx* ctx, double* out, int n) {
  if (!ctx || !out || n < 0 || n > 34) return RIS_ERR_ARG;
  double all[34] = {0};
  for (int i = 0; i < 16; i++) all[i] = ctx->eng.stats[i];
  all[15] = (double)ris::g_launches.load();
  try {
    RIS_CUDA(cudaSetDevice(ctx->eng.device));
    double ms[ris::kProfN], work[ris::kProfN];
    const cudaStream_t sts[2] = {ctx->eng.st, ctx->eng.st2};
    ris::prof_collect(sts, 2, ms, work);
    for (int c = 0; c < ris::kProfN; c++) {
      const int slot = c == ris::kProfEmuGemm ? 30 : c == ris::kProfFF ? 32 : 16 + 2 * c;
      all[slot] = ms[c];
      all[slot + 1] = work[c];
    }
  } catch (const ris::Error& e) {
    ctx->eng.err = e.msg;
    return e.code;
  }
  all[28] = (double)ctx->eng.mem.cur;
  all[29] = (double)ctx->eng.mem.peak;
  for (int i = 0; i < n; i++) out[i] = all[i];
  return RIS_OK;
}

ris_status ris_trim(ris_ctx* ctx) {
  return guarded(ctx, [&] {
    ctx->eng.trim();
    RIS_CUDA(cudaStreamSynchronize(ctx->eng.st));
  });
}

long long ris_debug_alloc_count(void) { return ris::g_allocs.load(); }

const char* ris_last_error(const ris_ctx* ctx) { return ctx ? ctx->eng.err.c_str() : "null context"; }

void ris_destroy(ris_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->eng.device);
  if (ctx->eng.st) cudaStreamSynchronize(ctx->eng.st);
  if (ctx->eng.opt.profile) {
    ris::prof_detach(ctx->eng.st);
    ris::prof_detach(ctx->eng.st2);
  }
  delete ctx;
}

}  // extern "C"
