// C ABI of the bkrylov library: handle, workspace, operators, single-kernel
// entry points and the device-resident solver drivers.
//
// A solver keeps every n x s block and every s x s coefficient on the device.
// Each iteration is a fixed sequence of kernel launches; data-dependent
// branches (re-orthonormalise or not, converged, breakdown) are decided on
// the device and read by the later kernels from the control block, so the
// host enqueues `sync_every` iterations at a time and only then reads the
// stop flag.  Kernels of iterations past the stop return immediately.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "bk_common.cuh"
#include "bk_internal.h"

using namespace bk;

struct bkrylov_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 152;
  void* ws[2] = {nullptr, nullptr};   // [0] solver internals, [1] refinement / host staging
  size_t ws_cap[2] = {0, 0};
  Ctrl* host_ctrl = nullptr;          // pinned staging of the control block
  Prof prof;                          // per-phase timing of profiled solves
  cudaStream_t cap_stream = nullptr;  // private stream for capturing iteration graphs (lazy)
};

const char* const bk::kPhaseNames[kNumPhases] = {
    "spmm_alpha", "small_1", "update_rho", "tsqr_leaf_factor", "tsqr_tree", "tsqr_leaf_apply",
    "tsqr_rho_gram", "small_2", "p_update", "precond_rho", "gmres_orthogonalise", "localized_tree",
    "localized_assemble", "cholqr"};

struct bkrylov_op_s {
  bkrylov_handle h = nullptr;
  OpDesc d;
};

namespace {

#define BK_TRY(x)                                   \
  do {                                              \
    cudaError_t _e = (x);                           \
    if (_e != cudaSuccess) return BK_ERR_CUDA;      \
  } while (0)

struct Bump {
  char* base;
  size_t off = 0, cap;
  Bump(void* b, size_t c) : base((char*)b), cap(c) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = (T*)(base + off);
    off += sizeof(T) * count;
    return p;
  }
};

int ensure_ws(bkrylov_handle h, int which, size_t bytes) {
  if (h->ws_cap[which] >= bytes) return BK_OK;
  if (h->ws[which]) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BK_ERR_CUDA;
    cudaFree(h->ws[which]);
    h->ws[which] = nullptr;
    h->ws_cap[which] = 0;
  }
  if (cudaMalloc(&h->ws[which], bytes) != cudaSuccess) return BK_ERR_ALLOC;
  h->ws_cap[which] = bytes;
  return BK_OK;
}

Launch launch_of(bkrylov_handle h) {
  Launch L;
  L.stream = h->stream;
  L.sms = h->sms;
  return L;
}

bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

size_t gpart_count(const Launch& L, const TsqrPlan&) {
  // largest grid of a reducing row kernel (every reducing kernel, the TSQR
  // apply included, caps its grid at sms x kCtasPerSm) x largest partial
  // record (two Grams + 2)
  return (size_t)L.sms * kCtasPerSm * (kMM + kMM + 8);
}

// The options of one solve: the caller's bkrylov_opts plus the tolerance and the
// iteration limit, which the solve entry points take as arguments of their own.
struct SolveOpts : bkrylov_opts {
  double tol = 1e-8;
  int maxit = 1000;
};

void opts_or_default(const bkrylov_opts* o, bkrylov_opts* out) {
  if (o) *out = *o; else bkrylov_opts_default(out);
}

// The stopping measure of the refinement's outer test (reading c2): max_i rel_i, or
// the Frobenius ratio sqrt(sum (rel_i nb_i)^2 / sum nb_i^2) for norm_mode 1.
double host_stop_measure(int norm_mode, const double* rel, const double* nb, int s) {
  if (norm_mode != 1) {
    double mx = 0.0;
    for (int i = 0; i < s; ++i) mx = std::isnan(rel[i]) ? rel[i] : std::fmax(mx, rel[i]);
    return mx;
  }
  double num = 0.0, den = 0.0;
  for (int i = 0; i < s; ++i) {
    num += (rel[i] * nb[i]) * (rel[i] * nb[i]);
    den += nb[i] * nb[i];
  }
  return den > 0.0 ? std::sqrt(num / den) : 0.0;
}

// ---- control block upload / download ------------------------------------------
int ctrl_upload(bkrylov_handle h, Ctrl* dev, int s, const SolveOpts& o, double eps) {
  Ctrl* c = h->host_ctrl;
  std::memset(c, 0, sizeof(Ctrl));
  c->s = s;
  c->maxit = o.maxit;
  c->tol = o.tol;
  c->eta = o.eta;
  c->eps = eps;
  c->n_forced = (o.forced_reortho && o.n_forced > 0) ? o.n_forced : 0;
  c->sub_p = (o.subalgebra_p > 0 && o.subalgebra_p < s) ? o.subalgebra_p : s;
  c->has_prec = o.precond != nullptr;
  c->one_r = o.one_reduction != 0;
  c->norm_mode = o.norm_mode;
  c->replace_every = o.one_reduction ? o.replace_every : 0;
  for (int i = 0; i < s; ++i) c->sigma[i * kMaxS + i] = 1.0;
  BK_TRY(cudaMemcpyAsync(dev, c, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
  // the pinned staging buffer is reused: wait for the copy before returning
  BK_TRY(cudaStreamSynchronize(h->stream));
  return BK_OK;
}

int ctrl_download(bkrylov_handle h, const Ctrl* dev) {
  BK_TRY(cudaMemcpyAsync(h->host_ctrl, dev, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  BK_TRY(cudaStreamSynchronize(h->stream));
  return BK_OK;
}

int ctrl_peek(bkrylov_handle h, const Ctrl* dev) {
  // first 16 bytes: done, status, iter, reorths
  BK_TRY(cudaMemcpyAsync(h->host_ctrl, dev, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  BK_TRY(cudaStreamSynchronize(h->stream));
  return BK_OK;
}

int finish_info(bkrylov_handle h, const Ctrl* dev, int s, const double* hist_dev,
                const uint8_t* dec_dev, int nrec, bkrylov_info* info, float ms) {
  int rc = ctrl_download(h, dev);
  if (rc) return rc;
  const Ctrl* c = h->host_ctrl;
  const int status = c->done == kDoneRunning ? BK_NOT_CONVERGED : c->status;
  if (info) {
    info->iters = c->iter;
    info->reorths = c->reorths;
    info->converged = c->done == kDoneConverged;
    info->status = status;
    double mx = 0.0;
    for (int i = 0; i < s; ++i) mx = std::fmax(mx, c->relres[i]);
    info->relres_max = mx;
    if (info->relres) std::memcpy(info->relres, c->relres, sizeof(double) * s);
    const int nh = c->iter < info->history_len ? c->iter : info->history_len;
    if (info->history && hist_dev && nh > 0)
      BK_TRY(cudaMemcpy(info->history, hist_dev, sizeof(double) * nh, cudaMemcpyDeviceToHost));
    if (info->decisions && dec_dev && nh > 0)
      BK_TRY(cudaMemcpy(info->decisions, dec_dev, nh, cudaMemcpyDeviceToHost));
    info->elapsed_ms = ms;
    info->reorths_cholqr = c->cholqr_count;
    info->replacements = c->replacements;
    (void)nrec;
  }
  return status;
}

// ---------------------------------------------------------------- BCG ----
template <typename T>
struct BcgBufs {
  T *R, *P, *Q;
  T* Z = nullptr;              // M^{-1} R-bar (preconditioned solves only)
  T* U = nullptr;              // A Z (the one-reduction schedule only)
  const OpDesc* M = nullptr;   // the preconditioner M^{-1}, or null (M = I)
  void* tsqr;
  double* gpart;
  Ctrl* ctrl;
  double* hist;
  uint8_t* dec;
  uint8_t* forced;
  bool cholqr = false;         // FP64 block case: CholeskyQR2 normaliser, TSQR the fallback
  bool replace = false;        // 1R-BCG with the replacement of Q and alpha
};

template <typename T, typename Alloc>
void bcg_layout(Alloc& a, int64_t n, int s, int maxit, const TsqrPlan& tp, const Launch& L,
                BcgBufs<T>* b, bool prec, bool one_r) {
  const size_t ns = (size_t)n * s;
  auto r = a.template take<T>(ns);
  auto p = a.template take<T>(ns);
  auto q = a.template take<T>(ns);
  b->Z = prec ? a.template take<T>(ns) : nullptr;
  b->U = one_r ? a.template take<T>(ns) : nullptr;
  auto t = a.template take<char>(tp.bytes);
  auto g = a.template take<double>(gpart_count(L, tp));
  auto c = a.template take<Ctrl>(1);
  auto hs = a.template take<double>((size_t)maxit + 1);
  auto dc = a.template take<uint8_t>((size_t)maxit + 1);
  auto fc = a.template take<uint8_t>((size_t)maxit + 1);
  b->R = r; b->P = p; b->Q = q; b->tsqr = t; b->gpart = g; b->ctrl = c; b->hist = hs;
  b->dec = dc; b->forced = fc;
}

// Normaliser of S_BP^p (Def. "normalizer"): one TSQR per p-column group of the
// n x s block (row stride s), its R factor and Gram into the group's diagonal
// block of gamma / rho (s x s, row stride 32).  p = s: one TSQR of the block.
template <typename T>
cudaError_t tsqr_groups(const Launch& L, const TsqrPlan& tp, int s, T* X, double* gamma, double* rho,
                        void* scratch, double* gpart, unsigned* counter, const int* done,
                        const int* flag) {
  const int p = tp.s;
  if (p == s) return tsqr<T>(L, tp, X, X, gamma, rho, scratch, gpart, counter, done, flag);
  // per-phase profiling covers the groups as one normaliser phase
  Launch Lg = L;
  Lg.prof = nullptr;
  prof_begin(L, kPhTsqrLeaf);
  for (int c0 = 0; c0 < s; c0 += p) {
    const size_t d = (size_t)c0 * (kMaxS + 1);
    cudaError_t e = tsqr<T>(Lg, tp, X + c0, X + c0, gamma + d, rho ? rho + d : nullptr, scratch, gpart,
                            counter, done, flag, s);
    if (e != cudaSuccess) return e;
  }
  prof_end(L, kPhTsqrLeaf, (s / p) * tsqr_launches(tp));
  return cudaSuccess;
}

// One BCG-ARO iteration (Alg. "2R-CG"): two grid-wide reductions (alpha with
// the SpMM, rho with the update or after the normaliser).
template <typename T>
cudaError_t bcg_iteration(const Launch& L, const OpDesc& A, int s, T* X, const BcgBufs<T>& b,
                          const TsqrPlan& tp) {
  Ctrl* c = b.ctrl;
  cudaError_t e;
  Epi<T> ep;
  ep.left = b.P; ep.sym = 1; ep.gram_out = c->alpha; ep.gpart = b.gpart;
  ep.counter = c->counters[kCntA]; ep.done = &c->done;
  ep.status_out = &c->status; ep.stop_out = &c->done;
  // S_BP^p (tp.s = p < s): the FP64 steps restricted to the column groups
  const int gp = tp.s;
  constexpr bool kF64 = sizeof(T) == 8;
  prof_begin(L, kPhSpmm);
  if constexpr (kF64) {
    if (gp < s) e = spmm_groups(L, A, s, gp, (const double*)b.P, (double*)b.Q, *(const Epi<double>*)&ep);
    else e = spmm<T>(L, A, s, b.P, b.Q, nullptr, ep);
  } else {
    e = spmm<T>(L, A, s, b.P, b.Q, nullptr, ep);
  }
  if (e != cudaSuccess) return e;
  prof_end(L, kPhSpmm, 1);
  prof_begin(L, kPhSmall1);
  if ((e = small_bcg_1(L, c, b.forced)) != cudaSuccess) return e;
  prof_end(L, kPhSmall1, 1);
  prof_begin(L, kPhUpdate);
  if constexpr (kF64) {
    if (gp < s) e = bcg_update_groups(L, A.n, s, gp, (const double*)b.P, (const double*)b.Q, (double*)X,
                                      (double*)b.R, c, b.gpart, 1);
    else e = bcg_update<T>(L, A.n, s, b.P, b.Q, X, b.R, c, b.gpart, b.cholqr ? 2 : 1);
  } else {
    e = bcg_update<T>(L, A.n, s, b.P, b.Q, X, b.R, c, b.gpart, 1);
  }
  if (e != cudaSuccess) return e;
  prof_end(L, kPhUpdate, b.cholqr ? 1 : 2);
  if constexpr (kF64) {
    if (b.cholqr) {
      // CholeskyQR2 of R-tilde from the update's Gram; the device declines nearly
      // dependent blocks (then tsqr_now is set and the TSQR below normalises).  Without
      // a preconditioner the second row pass is folded into the direction update.
      prof_begin(L, kPhCholqr);
      if ((e = small_cholqr(L, c, 1)) != cudaSuccess) return e;
      if ((e = cholqr_pass(L, A.n, s, (double*)b.R, c, b.gpart, true)) != cudaSuccess) return e;
      if ((e = small_cholqr(L, c, 2)) != cudaSuccess) return e;
      if (b.M && (e = cholqr_pass(L, A.n, s, (double*)b.R, c, b.gpart, false)) != cudaSuccess) return e;
      prof_end(L, kPhCholqr, b.M ? 4 : 3);
    }
  }
  // preconditioned: after a re-orthonormalisation only rho = <Z, R-bar> is needed
  if ((e = tsqr_groups<T>(L, tp, s, b.R, c->gamma, b.M ? nullptr : c->rho_new, b.tsqr, b.gpart,
                          c->counters[kCntC], &c->done, b.cholqr ? &c->tsqr_now : &c->reortho_now)) !=
      cudaSuccess)
    return e;
  if (b.M) {
    // Z = M^{-1} R-bar and rho_m = R-bar^T Z in one fused operator pass
    Epi<T> pz;
    pz.left = b.R; pz.sym = 1; pz.gram_out = c->rho_m; pz.gpart = b.gpart;
    pz.counter = c->counters[kCntA]; pz.done = &c->done;
    pz.status_out = &c->status; pz.stop_out = &c->done;
    prof_begin(L, kPhPrec);
    if constexpr (kF64) {
      if (gp < s) e = spmm_groups(L, *b.M, s, gp, (const double*)b.R, (double*)b.Z, *(const Epi<double>*)&pz);
      else e = spmm<T>(L, *b.M, s, b.R, b.Z, nullptr, pz);
    } else {
      e = spmm<T>(L, *b.M, s, b.R, b.Z, nullptr, pz);
    }
    if (e != cudaSuccess) return e;
    prof_end(L, kPhPrec, 1);
  }
  const T* Zn = b.M ? b.Z : b.R;     // P = Z + P beta
  prof_begin(L, kPhSmall2);
  if ((e = small_bcg_2(L, c, b.hist, b.dec)) != cudaSuccess) return e;
  prof_end(L, kPhSmall2, 1);
  prof_begin(L, kPhPupdate);
  if constexpr (kF64) {
    if (gp < s) e = bcg_pupdate_groups(L, A.n, s, gp, (const double*)Zn, (double*)b.P, c);
    else if (b.cholqr && !b.M) e = cholqr_pupdate(L, A.n, s, (double*)b.R, (double*)b.P, c);
    else e = bcg_pupdate<T>(L, A.n, s, Zn, b.P, c);
  } else {
    e = bcg_pupdate<T>(L, A.n, s, Zn, b.P, c);
  }
  prof_end(L, kPhPupdate, 1);
  return e;
}

// One iteration of Alg. "1R-CG" (block case): the operator is applied to Z
// after the preconditioner, fused with delta = Z^T U, and alpha comes from the
// recursion alpha = delta - beta^T alpha beta in the small kernel; Q is
// updated like P (Q = U + Q beta) instead of being recomputed.
template <typename T>
cudaError_t bcg_iteration_1r(const Launch& L, const OpDesc& A, int s, T* X, const BcgBufs<T>& b,
                             const TsqrPlan& tp) {
  Ctrl* c = b.ctrl;
  cudaError_t e;
  prof_begin(L, kPhSmall1);
  if ((e = small_bcg_1(L, c, b.forced)) != cudaSuccess) return e;
  prof_end(L, kPhSmall1, 1);
  prof_begin(L, kPhUpdate);
  if ((e = bcg_update<T>(L, A.n, s, b.P, b.Q, X, b.R, c, b.gpart, 1)) != cudaSuccess) return e;
  prof_end(L, kPhUpdate, 2);
  if ((e = tsqr_groups<T>(L, tp, s, b.R, c->gamma, b.M ? nullptr : c->rho_new, b.tsqr, b.gpart,
                          c->counters[kCntC], &c->done, &c->reortho_now)) != cudaSuccess) return e;
  if (b.M) {
    Epi<T> pz;
    pz.left = b.R; pz.sym = 1; pz.gram_out = c->rho_m; pz.gpart = b.gpart;
    pz.counter = c->counters[kCntA]; pz.done = &c->done;
    pz.status_out = &c->status; pz.stop_out = &c->done;
    prof_begin(L, kPhPrec);
    if ((e = spmm<T>(L, *b.M, s, b.R, b.Z, nullptr, pz)) != cudaSuccess) return e;
    prof_end(L, kPhPrec, 1);
  }
  const T* Zn = b.M ? b.Z : b.R;
  Epi<T> ed;                                      // U = A Z, delta = Z^T U
  ed.left = Zn; ed.sym = 1; ed.gram_out = c->delta; ed.gpart = b.gpart;
  ed.counter = c->counters[kCntA]; ed.done = &c->done;
  prof_begin(L, kPhSpmm);
  if ((e = spmm<T>(L, A, s, Zn, b.U, nullptr, ed)) != cudaSuccess) return e;
  prof_end(L, kPhSpmm, 1);
  prof_begin(L, kPhSmall2);
  if ((e = small_bcg_2(L, c, b.hist, b.dec)) != cudaSuccess) return e;
  prof_end(L, kPhSmall2, 1);
  prof_begin(L, kPhPupdate);
  if ((e = bcg_pupdate<T>(L, A.n, s, Zn, b.P, c)) != cudaSuccess) return e;    // P = Z + P beta
  e = bcg_pupdate<T>(L, A.n, s, b.U, b.Q, c);                                  // Q = U + Q beta
  prof_end(L, kPhPupdate, 2);
  if (e != cudaSuccess || !b.replace) return e;
  // replacement (the small kernel decided): Q = A P and alpha = P^T Q as in Alg. "2R-CG"
  Epi<T> er;
  er.left = b.P; er.sym = 1; er.gram_out = c->alpha; er.gpart = b.gpart;
  er.counter = c->counters[kCntA]; er.done = &c->done; er.only_if = &c->replace_now;
  er.status_out = &c->status; er.stop_out = &c->done;
  prof_begin(L, kPhSpmm);
  e = spmm<T>(L, A, s, b.P, b.Q, nullptr, er);
  prof_end(L, kPhSpmm, 1);
  return e;
}

// A batch of solver iterations captured as one CUDA graph (destroyed with the
// object).  capture(h, k, step) records k calls of step(Launch) on the
// handle's private capture stream; nothing runs until the graph is launched.
struct GraphBatch {
  cudaGraphExec_t exec = nullptr;
  bool failed = false;
  ~GraphBatch() { if (exec) cudaGraphExecDestroy(exec); }
  template <typename Step>
  int capture(bkrylov_handle h, int k, Step step) {
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return BK_ERR_CUDA;
    Launch Lc;
    Lc.stream = h->cap_stream;
    Lc.sms = h->sms;
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return BK_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < k && e == cudaSuccess; ++i) e = step(Lc);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess || ee != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();          // clear the capture error; nothing was enqueued
      return BK_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { exec = nullptr; return BK_ERR_CUDA; }
    return BK_OK;
  }
};

// launches of one two-reduction iteration (the TSQR has 3 * levels + 4 launches): the
// SpMM, two s x s kernels, the update (lean and Gram-carrying, or the Gram-carrying one
// alone with CholeskyQR2, which adds two s x s kernels and one row pass, two with M) and
// the direction update, plus the preconditioner pass
int bcg_launches_per_iter(const TsqrPlan& tp, bool cholqr, bool prec) {
  return (cholqr ? (prec ? 9 : 8) : 6) + (prec ? 1 : 0) + tsqr_launches(tp);
}

// The CholeskyQR2 normaliser serves FP64 two-reduction BCG in the block case
bool use_cholqr(const bkrylov_opts& o, int s, bool f64) {
  return f64 && o.qr_mode == 0 && (o.subalgebra_p == 0 || o.subalgebra_p == s) && !o.one_reduction;
}

template <typename T>
int bcg_device(bkrylov_handle h, const OpDesc& A, int s, const T* B, T* X, const SolveOpts& o,
               double eps, bkrylov_info* info) {
  const Launch L = launch_of(h);
  const OpDesc* M = o.precond ? &o.precond->d : nullptr;
  if (M && sizeof(T) == 4) BK_TRY(op_make_fp32(L, o.precond->d));
  const int64_t n = A.n;
  // S_BP^p normalises p-column groups: the TSQR plan is for width p
  const int gp = (o.subalgebra_p > 0 && o.subalgebra_p < s) ? o.subalgebra_p : s;
  const TsqrPlan tp = tsqr_plan(n, gp, (int)sizeof(T));
  const int maxit = o.maxit > 0 ? o.maxit : 0;
  BcgBufs<T> b;
  Bump probe(nullptr, 0);
  const bool one_r = o.one_reduction != 0;
  bcg_layout<T>(probe, n, s, maxit, tp, L, &b, M != nullptr, one_r);
  int rc = ensure_ws(h, 0, probe.off + 4096);
  if (rc) return rc;
  Bump bump(h->ws[0], h->ws_cap[0]);
  bcg_layout<T>(bump, n, s, maxit, tp, L, &b, M != nullptr, one_r);
  b.M = M;
  b.cholqr = use_cholqr(o, s, sizeof(T) == 8);
  b.replace = one_r && o.replace_every > 0;
  if ((rc = ctrl_upload(h, b.ctrl, s, o, eps))) return rc;
  if (o.forced_reortho && o.n_forced > 0) {
    const int nf = o.n_forced < maxit + 1 ? o.n_forced : maxit + 1;
    BK_TRY(cudaMemcpy(b.forced, o.forced_reortho, nf, cudaMemcpyHostToDevice));
  }
  cudaEvent_t e0, e1;
  BK_TRY(cudaEventCreate(&e0));
  BK_TRY(cudaEventCreate(&e1));
  BK_TRY(cudaEventRecord(e0, L.stream));
  Ctrl* c = b.ctrl;
  // setup: R = B - A X ; n0 ; normalise ; P = R ; rho = R^T R
  Epi<T> none;
  BK_TRY(spmm<T>(L, A, s, X, b.R, B, none));
  Epi<T> g;
  g.sym = 1; g.gram_out = c->rho_new; g.gpart = b.gpart; g.counter = c->counters[kCntA];
  BK_TRY(gram<T>(L, n, s, b.R, b.R, g));
  BK_TRY(diag_sqrt(L, s, c->rho_new, c->n0));
  if (o.eta > 0) {
    BK_TRY(tsqr_groups<T>(L, tp, s, b.R, c->sigma, nullptr, b.tsqr, b.gpart, nullptr, nullptr, nullptr));
  }
  g.gram_out = c->rho;
  BK_TRY(gram<T>(L, n, s, b.R, b.R, g));
  if (M) {
    // P^0 = M^{-1} R-bar^0 and rho_m = R-bar^T P^0 (the init kernel takes rho from it
    // after the norms test, which uses the Euclidean Gram above)
    Epi<T> pz;
    pz.left = b.R; pz.sym = 1; pz.gram_out = c->rho_m; pz.gpart = b.gpart; pz.counter = c->counters[kCntA];
    BK_TRY(spmm<T>(L, *M, s, b.R, b.P, nullptr, pz));
  } else {
    BK_TRY(cudaMemcpyAsync(b.P, b.R, sizeof(T) * (size_t)n * s, cudaMemcpyDeviceToDevice, L.stream));
  }
  if (one_r) {
    // Alg. "1R-CG": Q^0 = A P^0 and alpha^0 = <P^0, Q^0> before the loop
    Epi<T> pa;
    pa.left = b.P; pa.sym = 1; pa.gram_out = c->alpha; pa.gpart = b.gpart; pa.counter = c->counters[kCntA];
    BK_TRY(spmm<T>(L, A, s, b.P, b.Q, nullptr, pa));
  }
  BK_TRY(small_bcg_init(L, c, o.eta > 0));
  Launch Lp = L;
  if (o.profile) Lp.prof = &h->prof;
  int batch = o.sync_every > 0 ? o.sync_every : (n >= (1 << 20) ? 4 : 16);
  // After the first batch (which also settles every kernel's launch attributes),
  // a batch of iterations is captured once as a CUDA graph on a private stream
  // and replayed on the handle's stream: small problems are bound by kernel
  // launches, and at every size the kernels that a device flag turns into
  // no-ops (the gated TSQR) cost a launch each.  The iteration has no host-side
  // branch (every decision is in the control block), so the replay is the same
  // kernel sequence.  Profiled solves launch directly (per-phase events).
  const bool use_graph = !o.profile && maxit > 2 * batch;
  GraphBatch gb;
  int enq = 0;
  while (true) {
    if ((rc = ctrl_peek(h, c))) return rc;
    if (h->host_ctrl->done != kDoneRunning || enq >= maxit) break;
    const int todo = (maxit - enq) < batch ? (maxit - enq) : batch;
    if (gb.exec && todo == batch) {
      BK_TRY(cudaGraphLaunch(gb.exec, L.stream));
    } else {
      for (int i = 0; i < todo; ++i) {
        BK_TRY((one_r ? bcg_iteration_1r<T>(Lp, A, s, X, b, tp) : bcg_iteration<T>(Lp, A, s, X, b, tp)));
        prof_collect(Lp.prof);
      }
    }
    enq += todo;
    // capture the graph while the device runs the first batch (the capture only
    // records launches); a capture that the runtime refuses leaves the direct
    // launches in charge
    if (use_graph && !gb.failed && !gb.exec && maxit - enq >= batch) {
      if (gb.capture(h, batch, [&](const Launch& Lc) { return (one_r ? bcg_iteration_1r<T>(Lc, A, s, X, b, tp) : bcg_iteration<T>(Lc, A, s, X, b, tp)); }))
        gb.failed = true;
    }
  }
  BK_TRY(cudaEventRecord(e1, L.stream));
  BK_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return finish_info(h, c, s, b.hist, b.dec, maxit, info, ms);
}

// ------------------------------------------------ iterative refinement ----
int bcg_ir_device(bkrylov_handle h, bkrylov_op Aop, int s, const double* B, double* X,
                  const SolveOpts& o, bkrylov_info* info, void* outer_ws, size_t outer_off) {
  const Launch L = launch_of(h);
  OpDesc& A = Aop->d;
  BK_TRY(op_make_fp32(L, A));
  const int64_t n = A.n;
  const size_t ns = (size_t)n * s;
  Bump bump((char*)outer_ws + outer_off, h->ws_cap[1] - outer_off);
  double* R = bump.take<double>(ns);
  float* R32 = bump.take<float>(ns);
  float* D32 = bump.take<float>(ns);
  double* nrm = bump.take<double>(2 * kMaxS);
  double* gp = bump.take<double>((size_t)L.sms * 4 * kMaxS + 64);
  unsigned* cnt = bump.take<unsigned>(kTicketWords);
  BK_TRY(cudaMemsetAsync(cnt, 0, kTicketWords * sizeof(unsigned), L.stream));
  cudaEvent_t e0, e1;
  BK_TRY(cudaEventCreate(&e0));
  BK_TRY(cudaEventCreate(&e1));
  BK_TRY(cudaEventRecord(e0, L.stream));
  double nb[kMaxS], nr[kMaxS];
  BK_TRY(ir_colnorms(L, n, s, B, nrm + kMaxS, gp, cnt));
  BK_TRY(cudaMemcpyAsync(nb, nrm + kMaxS, sizeof(double) * s, cudaMemcpyDeviceToHost, L.stream));
  BK_TRY(cudaStreamSynchronize(L.stream));
  for (int i = 0; i < s; ++i) nb[i] = std::sqrt(nb[i]);
  int outer = 0, inner_total = 0, reorth_total = 0, repl_total = 0, status = BK_NOT_CONVERGED;
  double relmax = 0.0, rel[kMaxS];
  const int max_outer = o.ir_max_outer > 0 ? o.ir_max_outer : 30;
  std::vector<double> hist;
  for (;;) {
    Epi<double> none;
    BK_TRY(spmm<double>(L, A, s, X, R, B, none));        // R = B - A X in FP64
    BK_TRY(ir_colnorms(L, n, s, R, nrm, gp, cnt));
    BK_TRY(cudaMemcpyAsync(nr, nrm, sizeof(double) * s, cudaMemcpyDeviceToHost, L.stream));
    BK_TRY(cudaStreamSynchronize(L.stream));
    relmax = 0.0;
    bool finite = true;
    for (int i = 0; i < s; ++i) {
      rel[i] = nb[i] > 0 ? std::sqrt(nr[i]) / nb[i] : 0.0;
      if (!std::isfinite(rel[i])) finite = false;
      relmax = std::fmax(relmax, rel[i]);
    }
    const double stopv = host_stop_measure(o.norm_mode, rel, nb, s);
    hist.push_back(stopv);
    if (!finite) { status = BK_NONFINITE; break; }
    if (stopv <= o.tol) { status = BK_OK; break; }
    if (outer >= max_outer) { status = BK_NOT_CONVERGED; break; }
    BK_TRY(ir_to_fp32(L, n, s, R, nrm, R32));
    BK_TRY(cudaMemsetAsync(D32, 0, sizeof(float) * ns, L.stream));
    SolveOpts io = o;
    io.tol = o.ir_inner_tol;
    io.norm_mode = 0;             // the inner solves test every column (reading c19)
    io.forced_reortho = nullptr;
    io.n_forced = 0;
    bkrylov_info ii;
    std::memset(&ii, 0, sizeof(ii));
    const int irc = bcg_device<float>(h, A, s, R32, D32, io, std::ldexp(1.0, -23), &ii);
    inner_total += ii.iters;
    reorth_total += ii.reorths;
    repl_total += ii.replacements;
    if (irc != BK_OK && irc != BK_NOT_CONVERGED) { status = irc; break; }
    BK_TRY(ir_accumulate(L, n, s, D32, nrm, X));
    ++outer;
  }
  BK_TRY(cudaEventRecord(e1, L.stream));
  BK_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->iters = inner_total;
    info->reorths = reorth_total;
    info->replacements = repl_total;
    info->reorths_cholqr = 0;
    info->outer = outer;
    info->converged = status == BK_OK;
    info->status = status;
    info->relres_max = relmax;
    if (info->relres) std::memcpy(info->relres, rel, sizeof(double) * s);
    if (info->history)
      for (int i = 0; i < (int)hist.size() && i < info->history_len; ++i) info->history[i] = hist[i];
    info->elapsed_ms = ms;
  }
  return status;
}

// ---------------------------------------------------------- BBiCGStab ----
int bicg_device(bkrylov_handle h, const OpDesc& A, int s, const double* B, double* X,
                const SolveOpts& o, bkrylov_info* info) {
  const Launch L = launch_of(h);
  const int64_t n = A.n;
  const size_t ns = (size_t)n * s;
  const TsqrPlan tp = tsqr_plan(n, s);
  const int maxit = o.maxit > 0 ? o.maxit : 0;
  auto layout = [&](auto& a, double** R, double** P, double** Q, double** U, double** R0,
                    void** ts, double** gp, Ctrl** c, double** hs, uint8_t** dc, uint8_t** fc) {
    *R = a.template take<double>(ns); *P = a.template take<double>(ns);
    *Q = a.template take<double>(ns); *U = a.template take<double>(ns);
    *R0 = a.template take<double>(ns); *ts = a.template take<char>(tp.bytes);
    *gp = a.template take<double>(gpart_count(L, tp)); *c = a.template take<Ctrl>(1);
    *hs = a.template take<double>((size_t)maxit + 1); *dc = a.template take<uint8_t>((size_t)maxit + 1);
    *fc = a.template take<uint8_t>((size_t)maxit + 1);
  };
  double *R, *P, *Q, *U, *R0, *gp, *hs;
  void* ts;
  Ctrl* c;
  uint8_t *dc, *fc;
  {
    Bump probe(nullptr, 0);
    layout(probe, &R, &P, &Q, &U, &R0, &ts, &gp, &c, &hs, &dc, &fc);
    int rc = ensure_ws(h, 0, probe.off + 4096);
    if (rc) return rc;
  }
  Bump bump(h->ws[0], h->ws_cap[0]);
  layout(bump, &R, &P, &Q, &U, &R0, &ts, &gp, &c, &hs, &dc, &fc);
  int rc = ctrl_upload(h, c, s, o, std::ldexp(1.0, -52));
  if (rc) return rc;
  if (o.forced_reortho && o.n_forced > 0) {
    const int nf = o.n_forced < maxit + 1 ? o.n_forced : maxit + 1;
    BK_TRY(cudaMemcpy(fc, o.forced_reortho, nf, cudaMemcpyHostToDevice));
  }
  cudaEvent_t e0, e1;
  BK_TRY(cudaEventCreate(&e0));
  BK_TRY(cudaEventCreate(&e1));
  BK_TRY(cudaEventRecord(e0, L.stream));
  Epi<double> none;
  BK_TRY(spmm<double>(L, A, s, X, R, B, none));
  Epi<double> g;
  g.sym = 1; g.gram_out = c->rho_new; g.gpart = gp; g.counter = c->counters[kCntA];
  BK_TRY(gram<double>(L, n, s, R, R, g));
  BK_TRY(diag_sqrt(L, s, c->rho_new, c->n0));
  if (o.eta != 0) BK_TRY(tsqr<double>(L, tp, R, R, c->sigma, nullptr, ts, gp, nullptr, nullptr, nullptr));
  BK_TRY(cudaMemcpyAsync(P, R, sizeof(double) * ns, cudaMemcpyDeviceToDevice, L.stream));
  BK_TRY(cudaMemcpyAsync(R0, R, sizeof(double) * ns, cudaMemcpyDeviceToDevice, L.stream));
  g.gram_out = c->rho;
  BK_TRY(gram<double>(L, n, s, R, R, g));
  Epi<double> g2;
  g2.sym = 0; g2.gram_out = c->g2; g2.gpart = gp; g2.counter = c->counters[kCntA];
  BK_TRY(gram<double>(L, n, s, R0, R, g2));
  if (maxit <= 0) {
    // nothing to iterate: report the initial state as not converged
  }
  const int batch = o.sync_every > 0 ? o.sync_every : (n >= (1 << 20) ? 4 : 16);
  int enq = 0;
  while (true) {
    if ((rc = ctrl_peek(h, c))) return rc;
    if (h->host_ctrl->done != kDoneRunning || enq >= maxit) break;
    const int todo = (maxit - enq) < batch ? (maxit - enq) : batch;
    for (int i = 0; i < todo; ++i) {
      Epi<double> e1p;
      e1p.left = R0; e1p.sym = 0; e1p.gram_out = c->alpha; e1p.gpart = gp;
      e1p.counter = c->counters[kCntA]; e1p.done = &c->done;
      BK_TRY(spmm<double>(L, A, s, P, Q, nullptr, e1p));                 // Q = A P, R0^T Q
      BK_TRY(small_bicg_1(L, c, fc));
      BK_TRY(bcg_update<double>(L, n, s, P, Q, X, R, c, gp, 0));         // X += P lx ; S = R - Q lam
      BK_TRY(tsqr<double>(L, tp, R, R, c->gamma, nullptr, ts, gp, nullptr, &c->done, &c->reortho_now));
      Epi<double> e3;
      e3.left = R0; e3.sym = 0; e3.gram_out = c->g3; e3.frob = R; e3.frob_out = c->frob;
      e3.gpart = gp; e3.counter = c->counters[kCntB]; e3.done = &c->done;
      BK_TRY(spmm<double>(L, A, s, R, U, nullptr, e3));                  // U = A S, R0^T U, <U,S>, <U,U>
      BK_TRY(small_bicg_2(L, c));
      BK_TRY(bicg_final(L, n, s, R, U, X, P, Q, R0, c, gp));
      BK_TRY(small_bicg_3(L, c, hs, dc));
    }
    enq += todo;
  }
  BK_TRY(cudaEventRecord(e1, L.stream));
  BK_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return finish_info(h, c, s, hs, dc, maxit, info, ms);
}

// ------------------------------------------------------------- BGMRes ----
int gmres_device(bkrylov_handle h, const OpDesc& A, int s, const double* B, double* X,
                 const SolveOpts& o, bkrylov_info* info) {
  Launch L = launch_of(h);
  if (o.profile) L.prof = &h->prof;
  const int64_t n = A.n;
  const size_t ns = (size_t)n * s;
  const int m = o.restart > 0 ? o.restart : 30;
  const int maxit = o.maxit > 0 ? o.maxit : 0;
  const TsqrPlan tp = tsqr_plan(n, s);
  const size_t ss = (size_t)s * s;
  const size_t gmg = (size_t)L.sms * 4 * kMM + (size_t)8 * (m + 1) * kMM;
  // localized Arnoldi (ortho 2): the local bases (m + 1 more blocks) and the tree
  const bool loc = o.ortho == 2;
  LocalArnoldi la;
  size_t la_bytes = 0;
  if (loc) {
    la_bytes = local_arnoldi_bytes(n, s, m, tp.tile, &la);
    const int64_t last = n - (la.tiles - 1) * (int64_t)tp.tile;
    if (s > 16 || last < s || m + 1 > 72 || la.reduce_smem > 200 * 1024) return BK_ERR_UNSUPPORTED;
  }
  char* la_base = nullptr;
  double* Pbase = nullptr;
  auto layout = [&](auto& a, double** V, double** Hc, double** Ht, double** H, double** Gq,
                    double** sig, double** zeta, double*** Vp, void** ts, double** gp,
                    double** gmp, Ctrl** c, double** hs) {
    if (loc) {
      Pbase = a.template take<double>(ns * (m + 1));
      la_base = a.template take<char>(la_bytes);
    }
    *V = a.template take<double>(ns * (m + 1));
    *Hc = a.template take<double>((size_t)(m + 1) * kMM);
    *Ht = a.template take<double>((size_t)(m + 1) * kMM);
    *H = a.template take<double>((size_t)(m + 1) * s * m * s);
    *Gq = a.template take<double>((size_t)m * (2 * ss + s));
    *sig = a.template take<double>((size_t)(m + 1) * ss);
    *zeta = a.template take<double>((size_t)m * kMM);
    *Vp = a.template take<double*>((size_t)m + 1);
    *ts = a.template take<char>(tp.bytes);
    *gp = a.template take<double>(gpart_count(L, tp));
    *gmp = a.template take<double>(gmg);
    *c = a.template take<Ctrl>(1);
    *hs = a.template take<double>((size_t)maxit + 1);
  };
  double *V, *Hc, *Ht, *H, *Gq, *sig, *zeta, *gp, *gmp, *hs;
  double** Vp;
  void* ts;
  Ctrl* c;
  {
    Bump probe(nullptr, 0);
    layout(probe, &V, &Hc, &Ht, &H, &Gq, &sig, &zeta, &Vp, &ts, &gp, &gmp, &c, &hs);
    int rc = ensure_ws(h, 0, probe.off + 4096);
    if (rc) return rc;
  }
  Bump bump(h->ws[0], h->ws_cap[0]);
  layout(bump, &V, &Hc, &Ht, &H, &Gq, &sig, &zeta, &Vp, &ts, &gp, &gmp, &c, &hs);
  int rc = ctrl_upload(h, c, s, o, std::ldexp(1.0, -52));
  if (rc) return rc;
  std::vector<double*> vp(m + 1);
  for (int j = 0; j <= m; ++j) vp[j] = V + ns * j;
  BK_TRY(cudaMemcpyAsync(Vp, vp.data(), sizeof(double*) * (m + 1), cudaMemcpyHostToDevice, L.stream));
  BK_TRY(cudaStreamSynchronize(L.stream));
  if (loc) {
    std::vector<double*> pb(m + 1);
    for (int j = 0; j <= m; ++j) pb[j] = Pbase + ns * j;
    if ((rc = local_arnoldi_layout(la_base, &la, pb.data(), L.stream))) return rc;
  }
  cudaEvent_t e0, e1;
  BK_TRY(cudaEventCreate(&e0));
  BK_TRY(cudaEventCreate(&e1));
  BK_TRY(cudaEventRecord(e0, L.stream));
  Epi<double> none;
  BK_TRY(spmm<double>(L, A, s, X, V, B, none));
  Epi<double> g;
  g.sym = 1; g.gram_out = c->rho_new; g.gpart = gp; g.counter = c->counters[kCntA];
  BK_TRY(gram<double>(L, n, s, V, V, g));
  BK_TRY(diag_sqrt(L, s, c->rho_new, c->n0));
  int total = 0;
  bool first = true;
  int status = BK_NOT_CONVERGED;
  while (total < maxit) {
    if (!first) BK_TRY(spmm<double>(L, A, s, X, V, B, none));     // restart residual
    first = false;
    if (loc) {                                     // V^0 sigma^0 = R^0 as a distributed S-QR
      BK_TRY(local_arnoldi_begin(L, la));
      BK_TRY(local_arnoldi_extend(L, la, tp, ts, 0, V, V, Hc, c->gamma));
    } else {
      BK_TRY(tsqr<double>(L, tp, V, V, c->gamma, nullptr, ts, gp, nullptr, nullptr, nullptr));
    }
    BK_TRY(init_sig(L, s, c->gamma, sig, m + 1));
    int k_done = 0;
    bool conv = false;
    for (int k = 0; k < m && total < maxit; ++k) {
      double* W = vp[k + 1];
      prof_begin(L, kPhSpmm);
      BK_TRY(spmm<double>(L, A, s, vp[k], W, nullptr, none));
      prof_end(L, kPhSpmm, 1);
      if (loc) {                                   // localized Arnoldi (Ch. 9.3)
        BK_TRY(local_arnoldi_extend(L, la, tp, ts, k + 1, W, W, Hc, c->gamma));
      } else if (o.ortho == 1) {                   // block MGS (Alg. "block-arnoldi")
        prof_begin(L, kPhOrtho);
        for (int j = 0; j <= k; ++j) {
          Epi<double> gj;
          gj.sym = 0; gj.gram_out = Hc + (size_t)j * kMM; gj.gpart = gp; gj.counter = c->counters[kCntA];
          BK_TRY(gram<double>(L, n, s, vp[j], W, gj));
          BK_TRY(block_axpy<double>(L, n, s, vp[j], Hc + (size_t)j * kMM, -1.0, W, 1.0, nullptr));
        }
        prof_end(L, kPhOrtho, 2 * (k + 1));
      } else {                                     // CGS2 (Ch. 9.1, #it = 2)
        prof_begin(L, kPhOrtho);
        BK_TRY(multi_gram(L, n, s, Vp, k + 1, W, Hc, 0, gmp, nullptr, nullptr));
        BK_TRY(multi_axpy(L, n, s, Vp, k + 1, Hc, W, -1.0, nullptr));
        BK_TRY(multi_gram(L, n, s, Vp, k + 1, W, Ht, 0, gmp, nullptr, nullptr));
        BK_TRY(multi_axpy(L, n, s, Vp, k + 1, Ht, W, -1.0, nullptr));
        BK_TRY(vec_add(L, (int64_t)(k + 1) * kMM, Ht, Hc, nullptr));
        prof_end(L, kPhOrtho, 5);
      }
      if (!loc) BK_TRY(tsqr<double>(L, tp, W, W, c->gamma, nullptr, ts, gp, nullptr, nullptr, nullptr));
      prof_begin(L, kPhSmall2);
      BK_TRY(small_gmres_step(L, c, Hc, H, Gq, sig, k, m, hs, total));
      prof_end(L, kPhSmall2, 1);
      prof_collect(L.prof);
      ++total;
      k_done = k + 1;
      if ((rc = ctrl_peek(h, c))) return rc;
      if (h->host_ctrl->done == kDoneConverged) { conv = true; break; }
      if (h->host_ctrl->done != kDoneRunning) break;
    }
    BK_TRY(small_gmres_backsub(L, c, H, sig, zeta, k_done, m));
    BK_TRY(multi_axpy(L, n, s, Vp, k_done, zeta, X, 1.0, nullptr));
    if (conv) { status = BK_OK; break; }
    if (h->host_ctrl->done != kDoneRunning) { status = h->host_ctrl->status; break; }
  }
  BK_TRY(cudaEventRecord(e1, L.stream));
  BK_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int st = finish_info(h, c, s, hs, nullptr, maxit, info, ms);
  if (info) info->status = status;
  (void)st;
  return status;
}

// Stage host B/X into device buffers when needed, run, copy X back (T: the element
// type of the blocks).
template <typename T, typename F>
int with_device_blocks(bkrylov_handle h, int64_t n, int s, const T* B, T* X, size_t extra_outer, F&& run) {
  const bool hb = is_host_ptr(B), hx = is_host_ptr(X);
  const size_t ns = (size_t)n * s;
  size_t need = 256 + extra_outer + (hb ? sizeof(T) * ns + 256 : 0) + (hx ? sizeof(T) * ns + 256 : 0);
  int rc = ensure_ws(h, 1, need);
  if (rc) return rc;
  Bump bump(h->ws[1], h->ws_cap[1]);
  const T* dB = B;
  T* dX = X;
  if (hb) {
    T* t = bump.take<T>(ns);
    BK_TRY(cudaMemcpyAsync(t, B, sizeof(T) * ns, cudaMemcpyHostToDevice, h->stream));
    dB = t;
  }
  if (hx) {
    T* t = bump.take<T>(ns);
    BK_TRY(cudaMemcpyAsync(t, X, sizeof(T) * ns, cudaMemcpyHostToDevice, h->stream));
    dX = t;
  }
  const size_t off = (bump.off + 255) & ~(size_t)255;
  const int status = run(dB, dX, off);
  if (hx) {
    BK_TRY(cudaMemcpyAsync(X, dX, sizeof(T) * ns, cudaMemcpyDeviceToHost, h->stream));
    BK_TRY(cudaStreamSynchronize(h->stream));
  }
  return status;
}

bool valid_s(int s) { return s >= 1 && s <= kMaxS; }

// ctrl layout (row stride 32) -> dense row-major s x s
__global__ void compact_kernel(int s, const double* __restrict__ in, double* __restrict__ out) {
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) out[i] = in[(i / s) * kMaxS + (i % s)];
}

}  // namespace

// =============================================================== C ABI ====
extern "C" {

const char* bkrylov_status_string(int st) {
  switch (st) {
    case BK_OK: return "ok";
    case BK_ERR_ARG: return "invalid argument";
    case BK_ERR_CUDA: return "CUDA error";
    case BK_ERR_ALLOC: return "device allocation failed";
    case BK_NOT_CONVERGED: return "not converged";
    case BK_BREAKDOWN: return "breakdown";
    case BK_NONFINITE: return "non-finite value";
    case BK_TIMEOUT: return "timeout";
    case BK_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

int bkrylov_version(void) { return BKRYLOV_VERSION; }

void bkrylov_opts_default(bkrylov_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eta = INFINITY;
  o->restart = 30;
  o->ortho = 1;
  o->prec = BK_FP64;
  o->ir_inner_tol = 1e-5;
  o->ir_max_outer = 30;
}

int bkrylov_create(bkrylov_handle* out, int device, void* stream) {
  if (!out) return BK_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return BK_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return BK_ERR_CUDA;
  bkrylov_ctx* h = new (std::nothrow) bkrylov_ctx();
  if (!h) return BK_ERR_ALLOC;
  h->device = device;
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreate(&h->stream) != cudaSuccess) { delete h; return BK_ERR_CUDA; }
    h->own_stream = true;
  }
  for (int i = 0; i < Prof::kMax; ++i) {
    cudaEventCreate(&h->prof.b[i]);
    cudaEventCreate(&h->prof.e[i]);
  }
  if (cudaMallocHost(&h->host_ctrl, sizeof(Ctrl)) != cudaSuccess) {
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return BK_ERR_ALLOC;
  }
  *out = h;
  return BK_OK;
}

int bkrylov_destroy(bkrylov_handle h) {
  if (!h) return BK_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  for (int i = 0; i < 2; ++i) if (h->ws[i]) cudaFree(h->ws[i]);
  if (h->host_ctrl) cudaFreeHost(h->host_ctrl);
  for (int i = 0; i < Prof::kMax; ++i) {
    if (h->prof.b[i]) cudaEventDestroy(h->prof.b[i]);
    if (h->prof.e[i]) cudaEventDestroy(h->prof.e[i]);
  }
  if (h->own_stream) cudaStreamDestroy(h->stream);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
  return BK_OK;
}

int bkrylov_set_stream(bkrylov_handle h, void* stream) {
  if (!h) return BK_ERR_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BK_ERR_CUDA;
  if (h->own_stream) { cudaStreamDestroy(h->stream); h->own_stream = false; }
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreate(&h->stream) != cudaSuccess) return BK_ERR_CUDA;
    h->own_stream = true;
  }
  return BK_OK;
}

int bkrylov_op_csr(bkrylov_handle h, int64_t n, int64_t nnz, const int32_t* row_ptr,
                   const int32_t* col, const void* val, int val_prec, bkrylov_op* A) {
  if (!h || !A || n <= 0 || nnz < 0 || !row_ptr || (nnz > 0 && (!col || !val))) return BK_ERR_ARG;
  if (nnz > INT32_MAX || (val_prec != BK_FP64 && val_prec != BK_FP32)) return BK_ERR_ARG;
  bkrylov_op op = new (std::nothrow) bkrylov_op_s();
  if (!op) return BK_ERR_ALLOC;
  op->h = h;
  op->d.kind = kOpCsr;
  op->d.n = n;
  op->d.nnz = nnz;
  op->d.row_ptr = row_ptr;
  op->d.col = col;
  if (val_prec == BK_FP64) {
    op->d.val = static_cast<const double*>(val);
  } else {
    // FP32 values are borrowed for the FP32 products; FP64 products (the FP64 solvers,
    // the refinement's outer residual) use an owned exact widening of them
    op->d.val32 = const_cast<float*>(static_cast<const float*>(val));
    op->d.val32_borrowed = true;
    double* v64 = nullptr;
    if (cudaMalloc(&v64, sizeof(double) * (size_t)(nnz > 0 ? nnz : 1)) != cudaSuccess) {
      delete op;
      return BK_ERR_ALLOC;
    }
    op->d.val64_owned = v64;
    op->d.val = v64;
    if (widen_block(launch_of(h), nnz, op->d.val32, v64) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
      cudaFree(v64);
      delete op;
      return BK_ERR_CUDA;
    }
  }
  *A = op;
  return BK_OK;
}

int bkrylov_op_stencil(bkrylov_handle h, int kind, int nx, int ny, int nz, const double* coeffs,
                       bkrylov_op* A) {
  if (!h || !A || nx <= 0 || ny <= 0 || nz <= 0 || !coeffs) return BK_ERR_ARG;
  if ((int64_t)nx * ny * nz > (int64_t)UINT32_MAX) return BK_ERR_ARG;   // 32-bit grid indexing
  bkrylov_op op = new (std::nothrow) bkrylov_op_s();
  if (!op) return BK_ERR_ALLOC;
  op->h = h;
  OpDesc& d = op->d;
  d.nx = nx; d.ny = ny; d.nz = nz;
  d.n = (int64_t)nx * ny * nz;
  const Launch L = launch_of(h);
  if (kind == BK_STENCIL_CONST7) {
    d.kind = kOpConst7;
    std::memcpy(d.c7, coeffs, sizeof(double) * 7);
    const int64_t plane = (int64_t)nx * ny;
    d.nnz = d.n + 2 * ((int64_t)(nx - 1) * ny * nz + (int64_t)nx * (ny - 1) * nz + plane * (nz - 1));
  } else if (kind == BK_STENCIL_VAR7) {
    d.kind = kOpVar7;
    d.coef_len = 4 * d.n;
    if (cudaMalloc(&d.coef, sizeof(double) * (size_t)d.coef_len) != cudaSuccess) { delete op; return BK_ERR_ALLOC; }
    if (op_prepare_stencil(L, d, coeffs) != cudaSuccess) { cudaFree(d.coef); delete op; return BK_ERR_CUDA; }
    const int64_t plane = (int64_t)nx * ny;
    d.nnz = d.n + 2 * ((int64_t)(nx - 1) * ny * nz + (int64_t)nx * (ny - 1) * nz + plane * (nz - 1));
  } else if (kind == BK_STENCIL_EDGE5 || kind == BK_STENCIL_EDGE5_LOG) {
    if (nz != 1) { delete op; return BK_ERR_ARG; }
    d.kind = kOpEdge5;
    d.edges = coeffs;
    if (kind == BK_STENCIL_EDGE5_LOG) {      // a_e = exp(theta_e), owned by the operator
      const int64_t ne = (int64_t)ny * (nx + 1) + (int64_t)(ny + 1) * nx;
      if (cudaMalloc(&d.edges_owned, sizeof(double) * (size_t)ne) != cudaSuccess) { delete op; return BK_ERR_ALLOC; }
      if (exp_block(L, ne, coeffs, d.edges_owned) != cudaSuccess) {
        cudaFree(d.edges_owned); delete op; return BK_ERR_CUDA;
      }
      d.edges = d.edges_owned;
      coeffs = d.edges_owned;
    }
    d.coef_len = d.n;
    if (cudaMalloc(&d.coef, sizeof(double) * (size_t)d.coef_len) != cudaSuccess) {
      cudaFree(d.edges_owned); delete op; return BK_ERR_ALLOC;
    }
    if (op_prepare_stencil(L, d, coeffs) != cudaSuccess) {
      cudaFree(d.coef); cudaFree(d.edges_owned); delete op; return BK_ERR_CUDA;
    }
    d.nnz = d.n + 2 * ((int64_t)(nx - 1) * ny + (int64_t)nx * (ny - 1));
  } else {
    delete op;
    return BK_ERR_ARG;
  }
  *A = op;
  return BK_OK;
}

int bkrylov_op_diag(bkrylov_handle h, int64_t n, const double* d, bkrylov_op* M) {
  if (!h || !M || n <= 0 || !d) return BK_ERR_ARG;
  bkrylov_op op = new (std::nothrow) bkrylov_op_s();
  if (!op) return BK_ERR_ALLOC;
  op->h = h;
  OpDesc& o = op->d;
  o.kind = kOpDiag;
  o.n = n;
  o.nnz = n;
  o.coef_len = n;
  if (cudaMalloc(&o.coef, sizeof(double) * (size_t)n) != cudaSuccess) { delete op; return BK_ERR_ALLOC; }
  if (cudaMemcpyAsync(o.coef, d, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, h->stream) !=
      cudaSuccess) {
    cudaFree(o.coef); delete op; return BK_ERR_CUDA;
  }
  *M = op;
  return BK_OK;
}

int bkrylov_op_jacobi(bkrylov_handle h, bkrylov_op A, bkrylov_op* M) {
  if (!h || !A || !M) return BK_ERR_ARG;
  const Launch L = launch_of(h);
  bkrylov_op op = new (std::nothrow) bkrylov_op_s();
  if (!op) return BK_ERR_ALLOC;
  op->h = h;
  OpDesc& o = op->d;
  o.kind = kOpDiag;
  o.n = A->d.n;
  o.nnz = o.n;
  o.coef_len = o.n;
  int* bad = nullptr;
  int bad_h = 0;
  auto fail = [&](int rc) { if (bad) cudaFree(bad); if (o.coef) cudaFree(o.coef); delete op; return rc; };
  if (cudaMalloc(&o.coef, sizeof(double) * (size_t)o.n) != cudaSuccess) { o.coef = nullptr; return fail(BK_ERR_ALLOC); }
  if (cudaMalloc(&bad, sizeof(int)) != cudaSuccess) { bad = nullptr; return fail(BK_ERR_ALLOC); }
  if (cudaMemsetAsync(bad, 0, sizeof(int), L.stream) != cudaSuccess) return fail(BK_ERR_CUDA);
  if (jacobi_inverse_diagonal(L, A->d, o.coef, bad) != cudaSuccess) return fail(BK_ERR_CUDA);
  if (cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, L.stream) != cudaSuccess ||
      cudaStreamSynchronize(L.stream) != cudaSuccess)
    return fail(BK_ERR_CUDA);
  cudaFree(bad);
  bad = nullptr;
  if (bad_h) return fail(BK_ERR_ARG);
  *M = op;
  return BK_OK;
}

int bkrylov_op_transpose(bkrylov_handle h, bkrylov_op A, bkrylov_op* At) {
  if (!h || !A || !At) return BK_ERR_ARG;
  bkrylov_op op = new (std::nothrow) bkrylov_op_s();
  if (!op) return BK_ERR_ALLOC;
  op->h = h;
  if (A->d.kind == kOpCsr) {
    const cudaError_t e = csr_transpose(launch_of(h), A->d, op->d);
    if (e != cudaSuccess) {
      delete op;
      return e == cudaErrorMemoryAllocation ? BK_ERR_ALLOC : BK_ERR_CUDA;
    }
  } else if (A->d.kind == kOpConst7) {
    // the transpose of a constant 7-point stencil swaps each -/+ pair
    op->d = OpDesc();
    op->d.kind = kOpConst7;
    op->d.n = A->d.n; op->d.nnz = A->d.nnz;
    op->d.nx = A->d.nx; op->d.ny = A->d.ny; op->d.nz = A->d.nz;
    const double* c = A->d.c7;   // (centre, -x, +x, -y, +y, -z, +z)
    const double ct[7] = {c[0], c[2], c[1], c[4], c[3], c[6], c[5]};
    std::memcpy(op->d.c7, ct, sizeof(ct));
  } else {
    delete op;
    return BK_ERR_UNSUPPORTED;
  }
  *At = op;
  return BK_OK;
}

int bkrylov_op_destroy(bkrylov_op A) {
  if (!A) return BK_ERR_ARG;
  if (A->h) cudaStreamSynchronize(A->h->stream);
  if (A->d.val32 && !A->d.val32_borrowed) cudaFree(A->d.val32);
  if (A->d.val64_owned) cudaFree(A->d.val64_owned);
  if (A->d.coef) cudaFree(A->d.coef);
  if (A->d.coef32) cudaFree(A->d.coef32);
  if (A->d.edges32) cudaFree(A->d.edges32);
  if (A->d.coef4) cudaFree(A->d.coef4);
  if (A->d.edges_owned) cudaFree(A->d.edges_owned);
  if (A->d.rp_owned) cudaFree(A->d.rp_owned);
  if (A->d.col_owned) cudaFree(A->d.col_owned);
  if (A->d.val_owned) cudaFree(A->d.val_owned);
  delete A;
  return BK_OK;
}

int bkrylov_op_size(bkrylov_op A, int64_t* n, int64_t* nnz) {
  if (!A) return BK_ERR_ARG;
  if (n) *n = A->d.n;
  if (nnz) *nnz = A->d.nnz;
  return BK_OK;
}

int bkrylov_spmm(bkrylov_handle h, bkrylov_op A, int s, const void* P, void* Q, int prec) {
  if (!h || !A || !valid_s(s) || !P || !Q || P == Q) return BK_ERR_ARG;
  const Launch L = launch_of(h);
  if (prec == BK_FP64) {
    Epi<double> none;
    BK_TRY(spmm<double>(L, A->d, s, (const double*)P, (double*)Q, nullptr, none));
  } else if (prec == BK_FP32) {
    BK_TRY(op_make_fp32(L, A->d));
    Epi<float> none;
    BK_TRY(spmm<float>(L, A->d, s, (const float*)P, (float*)Q, nullptr, none));
  } else {
    return BK_ERR_ARG;
  }
  return BK_OK;
}

int bkrylov_residual(bkrylov_handle h, bkrylov_op A, int s, const void* B, const void* X, void* R,
                     int prec) {
  if (!h || !A || !valid_s(s) || !B || !X || !R || X == R) return BK_ERR_ARG;
  const Launch L = launch_of(h);
  if (prec == BK_FP64) {
    Epi<double> none;
    BK_TRY(spmm<double>(L, A->d, s, (const double*)X, (double*)R, (const double*)B, none));
  } else if (prec == BK_FP32) {
    BK_TRY(op_make_fp32(L, A->d));
    Epi<float> none;
    BK_TRY(spmm<float>(L, A->d, s, (const float*)X, (float*)R, (const float*)B, none));
  } else {
    return BK_ERR_ARG;
  }
  return BK_OK;
}

// Scratch of the single-kernel entry points: grid partials + ticket words +
// a ctrl-layout result matrix, in workspace 1.
static int small_scratch(bkrylov_handle h, double** gp, unsigned** cnt, double** res) {
  const Launch L = launch_of(h);
  const size_t gpn = (size_t)L.sms * kCtasPerSm * (kMM + kMM + 8);
  int rc = ensure_ws(h, 1, sizeof(double) * (gpn + kMM) + sizeof(unsigned) * kTicketWords + 1024);
  if (rc) return rc;
  Bump b(h->ws[1], h->ws_cap[1]);
  *gp = b.take<double>(gpn);
  *res = b.take<double>(kMM);
  *cnt = b.take<unsigned>(kTicketWords);
  BK_TRY(cudaMemsetAsync(*cnt, 0, kTicketWords * sizeof(unsigned), h->stream));
  return BK_OK;
}

int bkrylov_spmm_gram(bkrylov_handle h, bkrylov_op A, int s, const void* P, void* Q, double* G, int sym,
                      int prec) {
  if (!h || !A || !valid_s(s) || !P || !Q || !G || P == Q) return BK_ERR_ARG;
  if (prec != BK_FP64 && prec != BK_FP32) return BK_ERR_ARG;
  double *gp, *res;
  unsigned* cnt;
  int rc = small_scratch(h, &gp, &cnt, &res);
  if (rc) return rc;
  const Launch L = launch_of(h);
  if (prec == BK_FP64) {
    Epi<double> e;
    e.left = (const double*)P; e.sym = sym ? 1 : 0; e.gram_out = res; e.gpart = gp; e.counter = cnt;
    BK_TRY(spmm<double>(L, A->d, s, (const double*)P, (double*)Q, nullptr, e));
  } else {
    BK_TRY(op_make_fp32(L, A->d));
    Epi<float> e;
    e.left = (const float*)P; e.sym = sym ? 1 : 0; e.gram_out = res; e.gpart = gp; e.counter = cnt;
    BK_TRY(spmm<float>(L, A->d, s, (const float*)P, (float*)Q, nullptr, e));
  }
  compact_kernel<<<1, 256, 0, h->stream>>>(s, res, G);
  BK_TRY(cudaGetLastError());
  return BK_OK;
}

int bkrylov_bdot(bkrylov_handle h, int64_t n, int s, const void* X, const void* Y, double* G, int sym,
                 int prec) {
  if (!h || n <= 0 || !valid_s(s) || !X || !Y || !G) return BK_ERR_ARG;
  double *gp, *res;
  unsigned* cnt;
  int rc = small_scratch(h, &gp, &cnt, &res);
  if (rc) return rc;
  const Launch L = launch_of(h);
  if (prec == BK_FP64) {
    Epi<double> e;
    e.sym = sym ? 1 : 0; e.gram_out = res; e.gpart = gp; e.counter = cnt;
    BK_TRY(gram<double>(L, n, s, (const double*)X, (const double*)Y, e));
  } else if (prec == BK_FP32) {
    Epi<float> e;
    e.sym = sym ? 1 : 0; e.gram_out = res; e.gpart = gp; e.counter = cnt;
    BK_TRY(gram<float>(L, n, s, (const float*)X, (const float*)Y, e));
  } else {
    return BK_ERR_ARG;
  }
  compact_kernel<<<1, 256, 0, h->stream>>>(s, res, G);
  BK_TRY(cudaGetLastError());
  return BK_OK;
}

int bkrylov_tsqr(bkrylov_handle h, int64_t n, int s, const void* X, void* Y, double* sigma, int prec) {
  if (!h || !valid_s(s) || n < s || !X || !Y || !sigma) return BK_ERR_ARG;
  const Launch L = launch_of(h);
  const TsqrPlan tp = tsqr_plan(n, s, prec == BK_FP32 ? 4 : 8);
  const size_t gpn = gpart_count(L, tp);
  int rc = ensure_ws(h, 1, tp.bytes + sizeof(double) * (gpn + kMM) + 2048);
  if (rc) return rc;
  Bump b(h->ws[1], h->ws_cap[1]);
  void* sc = b.take<char>(tp.bytes);
  double* res = b.take<double>(kMM);
  if (prec == BK_FP64) {
    BK_TRY(tsqr<double>(L, tp, (const double*)X, (double*)Y, res, nullptr, sc, nullptr, nullptr,
                        nullptr, nullptr));
  } else if (prec == BK_FP32) {
    BK_TRY(tsqr<float>(L, tp, (const float*)X, (float*)Y, res, nullptr, sc, nullptr, nullptr,
                       nullptr, nullptr));
  } else {
    return BK_ERR_ARG;
  }
  compact_kernel<<<1, 256, 0, h->stream>>>(s, res, sigma);
  BK_TRY(cudaGetLastError());
  return BK_OK;
}

static int check_solve_args(bkrylov_handle h, bkrylov_op A, int s, const void* B, void* X,
                            const SolveOpts& o) {
  if (!h || !A || !valid_s(s) || !B || !X || B == (const void*)X) return BK_ERR_ARG;
  if (A->d.n < s) return BK_ERR_ARG;
  if (!(o.tol >= 0.0) || o.maxit < 0 || !(o.eta >= 0.0)) return BK_ERR_ARG;
  if (o.norm_mode != 0 && o.norm_mode != 1) return BK_ERR_ARG;
  if (o.qr_mode != 0 && o.qr_mode != 1) return BK_ERR_ARG;
  if (o.replace_every < 0) return BK_ERR_ARG;
  if (o.subalgebra_p < 0 || (o.subalgebra_p > 0 && s % o.subalgebra_p != 0)) return BK_ERR_ARG;
  if (o.precond && o.precond->d.n != A->d.n) return BK_ERR_ARG;
  return BK_OK;
}

// the block-parallel subalgebra is a BCG option
static bool block_case(const bkrylov_opts& o, int s) {
  return o.subalgebra_p == 0 || o.subalgebra_p == s;
}

static SolveOpts solve_opts(const bkrylov_opts* opts, double tol, int maxit) {
  SolveOpts o;
  opts_or_default(opts, &o);
  o.tol = tol;
  o.maxit = maxit;
  return o;
}

int bkrylov_solve_bcg(bkrylov_handle h, bkrylov_op A, int s, const void* B, void* X, double tol, int maxit,
                      const bkrylov_opts* opts, bkrylov_info* info) {
  const SolveOpts o = solve_opts(opts, tol, maxit);
  int rc = check_solve_args(h, A, s, B, X, o);
  if (rc) return rc;
  if (o.one_reduction && !block_case(o, s)) return BK_ERR_UNSUPPORTED;
  const int64_t n = A->d.n;
  if (o.prec == BK_FP64) {
    return with_device_blocks<double>(h, n, s, static_cast<const double*>(B), static_cast<double*>(X), 0,
                                      [&](const double* dB, double* dX, size_t) {
      return bcg_device<double>(h, A->d, s, dB, dX, o, std::ldexp(1.0, -52), info);
    });
  }
  if (o.prec == BK_FP32) {
    // the raw FP32 solve: FP32 blocks and products, every s x s quantity in FP64
    BK_TRY(op_make_fp32(launch_of(h), A->d));
    return with_device_blocks<float>(h, n, s, static_cast<const float*>(B), static_cast<float*>(X), 0,
                                     [&](const float* dB, float* dX, size_t) {
      return bcg_device<float>(h, A->d, s, dB, dX, o, std::ldexp(1.0, -23), info);
    });
  }
  if (o.prec == BK_FP32_IR) {
    const size_t ns = (size_t)n * s;
    const size_t extra = sizeof(double) * ns + 2 * sizeof(float) * ns +
                         sizeof(double) * ((size_t)h->sms * 4 * kMaxS + 2 * kMaxS + 64) +
                         sizeof(unsigned) * kTicketWords + 4096;
    return with_device_blocks<double>(h, n, s, static_cast<const double*>(B), static_cast<double*>(X), extra,
                                      [&](const double* dB, double* dX, size_t off) {
      return bcg_ir_device(h, A, s, dB, dX, o, info, h->ws[1], off);
    });
  }
  return BK_ERR_ARG;
}

int bkrylov_solve_bbicgstab(bkrylov_handle h, bkrylov_op A, int s, const void* B, void* X, double tol,
                            int maxit, const bkrylov_opts* opts, bkrylov_info* info) {
  const SolveOpts o = solve_opts(opts, tol, maxit);
  int rc = check_solve_args(h, A, s, B, X, o);
  if (rc) return rc;
  if (!block_case(o, s) || o.precond || o.one_reduction) return BK_ERR_UNSUPPORTED;
  if (o.prec != BK_FP64) return BK_ERR_UNSUPPORTED;
  return with_device_blocks<double>(h, A->d.n, s, static_cast<const double*>(B), static_cast<double*>(X), 0,
                                    [&](const double* dB, double* dX, size_t) {
    return bicg_device(h, A->d, s, dB, dX, o, info);
  });
}

int bkrylov_solve_bgmres(bkrylov_handle h, bkrylov_op A, int s, const void* B, void* X, double tol, int maxit,
                         const bkrylov_opts* opts, bkrylov_info* info) {
  const SolveOpts o = solve_opts(opts, tol, maxit);
  int rc = check_solve_args(h, A, s, B, X, o);
  if (rc) return rc;
  if (!block_case(o, s) || o.precond || o.one_reduction) return BK_ERR_UNSUPPORTED;
  if (o.prec != BK_FP64) return BK_ERR_UNSUPPORTED;
  if (o.restart < 1 || o.restart > 64 || o.ortho < 0 || o.ortho > 2) return BK_ERR_ARG;
  return with_device_blocks<double>(h, A->d.n, s, static_cast<const double*>(B), static_cast<double*>(X), 0,
                                    [&](const double* dB, double* dX, size_t) {
    return gmres_device(h, A->d, s, dB, dX, o, info);
  });
}

int bkrylov_profile_count(void) { return kNumPhases; }

int bkrylov_profile_get(bkrylov_handle h, int i, const char** name, double* total_ms,
                        long long* launches) {
  if (!h || i < 0 || i >= kNumPhases) return BK_ERR_ARG;
  if (name) *name = kPhaseNames[i];
  if (total_ms) *total_ms = h->prof.ms[i];
  if (launches) *launches = h->prof.launches[i];
  return BK_OK;
}

int bkrylov_profile_reset(bkrylov_handle h) {
  if (!h) return BK_ERR_ARG;
  for (int i = 0; i < Prof::kMax; ++i) { h->prof.ms[i] = 0.0; h->prof.launches[i] = 0; }
  return BK_OK;
}

int bkrylov_kappa_d(bkrylov_handle h, int s, const double* A, double* kappa) {
  if (!h || !valid_s(s) || !A || !kappa) return BK_ERR_ARG;
  BK_TRY(small_kappa_d(launch_of(h), s, A, kappa));
  return BK_OK;
}

int bkrylov_reortho_decision(bkrylov_handle h, int s, const double* A, double eta, double eps, int* decision) {
  if (!h || !valid_s(s) || !A || !decision || !(eta >= 0.0) || !(eps > 0.0)) return BK_ERR_ARG;
  BK_TRY(small_criterion(launch_of(h), s, eta, eps, A, decision));
  return BK_OK;
}

int bkrylov_bcg_launches_per_iteration(int64_t n, int s, const bkrylov_opts* opts) {
  if (n < 1 || s < 1 || s > kMaxS) return -1;
  bkrylov_opts o;
  opts_or_default(opts, &o);
  const TsqrPlan tp = tsqr_plan(n, s);
  if (o.one_reduction)   // small 1, update (2), TSQR, preconditioner, U = A Z, small 2, two updates, replacement
    return 7 + tsqr_launches(tp) + (o.precond ? 1 : 0) + (o.replace_every > 0 ? 1 : 0);
  return bcg_launches_per_iter(tp, use_cholqr(o, s, o.prec == BK_FP64), o.precond != nullptr);
}

int bkrylov_adjoint_scatter(bkrylov_handle h, bkrylov_op A, int s, const double* Lam,
                            const double* X, double* g) {
  if (!h || !A || !valid_s(s) || !Lam || !X || !g) return BK_ERR_ARG;
  if (A->d.kind != kOpCsr) return BK_ERR_ARG;
  BK_TRY(adjoint_scatter(launch_of(h), A->d, s, Lam, X, g));
  return BK_OK;
}

int bkrylov_edge_theta_grad(bkrylov_handle h, bkrylov_op A, int s, const double* Lam,
                            const double* X, double* g) {
  if (!h || !A || !valid_s(s) || !Lam || !X || !g) return BK_ERR_ARG;
  if (A->d.kind != kOpEdge5) return BK_ERR_ARG;
  BK_TRY(edge_theta_grad(launch_of(h), A->d, s, Lam, X, g));
  return BK_OK;
}

}  // extern "C"
