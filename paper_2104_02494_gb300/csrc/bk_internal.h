// Host-side internal interfaces of the bkrylov library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bkrylov.h"

namespace bk {

struct Ctrl;

enum OpKind { kOpCsr = 0, kOpConst7 = 1, kOpVar7 = 2, kOpEdge5 = 3, kOpDiag = 4 };

struct OpDesc {
  int kind = kOpCsr;
  int64_t n = 0, nnz = 0;
  // CSR (borrowed) + owned float copy of the values
  const int32_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  float* val32 = nullptr;
  bool val32_borrowed = false;     // FP32 values given by the caller (not freed)
  double* val64_owned = nullptr;   // owned FP64 widening of caller-given FP32 values
  int32_t* rp_owned = nullptr;     // owned CSR arrays of a transposed operator
  int32_t* col_owned = nullptr;
  double* val_owned = nullptr;
  // stencils
  int nx = 0, ny = 0, nz = 0;
  double c7[7] = {0, 0, 0, 0, 0, 0, 0};
  // VAR7: owned diag + faces to the +x/+y/+z neighbour (0 at the boundary), 4 arrays of n.
  // EDGE5: owned diag (n); borrowed edge coefficients (ny*(nx+1) + (ny+1)*nx).
  // DIAG: owned entries (n) of the diagonal operator.
  double* coef = nullptr;          // owned double coefficient arrays
  float* coef32 = nullptr;         // owned float copy (lazy)
  const double* edges = nullptr;   // EDGE5 borrowed (or edges_owned)
  double* edges_owned = nullptr;   // EDGE5 from log-coefficients: a_e = exp(theta_e), owned
  float* edges32 = nullptr;        // EDGE5 owned float copy (lazy)
  float* coef4 = nullptr;          // VAR7 / EDGE5: per-cell float quadruples of the marching
                                   // kernel (owned, lazy; bk_march.cu)
  int64_t coef_len = 0;
};

// Fused epilogue of a row kernel: Gram  left^T out  and Frobenius sums <out, frob>_F, <out,out>_F.
template <typename T>
struct Epi {
  const T* left = nullptr;     // Gram G = left^T out (null: no Gram)
  int sym = 0;                 // upper triangle only, mirrored
  const T* frob = nullptr;     // Frobenius partner (null: none)
  double* gram_out = nullptr;  // s x s result, row stride 32 (device)
  double* frob_out = nullptr;  // [2]: <out,frob>, <out,out> (device)
  double* gpart = nullptr;     // grid partials scratch
  unsigned* counter = nullptr; // kTicketWords ticket words (0 on entry)
  const int* done = nullptr;   // optional stop flag: kernel exits when *done != 0
  const int* only_if = nullptr;  // optional: kernel exits unless *only_if != 0
  int* status_out = nullptr;     // pipelined kernels: BK_TIMEOUT written here if a bounded wait gave up
  int* stop_out = nullptr;       // ... and a non-zero stop flag here (the following kernels return)
};

// Optional per-phase device timing (CUDA events on the launching stream).
enum Phase : int {
  kPhSpmm = 0, kPhSmall1, kPhUpdate, kPhTsqrLeaf, kPhTsqrTree, kPhTsqrApply, kPhTsqrGram,
  kPhSmall2, kPhPupdate, kPhPrec, kPhOrtho, kPhLaTree, kPhLaAssemble, kPhCholqr, kNumPhases
};
struct Prof {
  static constexpr int kMax = 16;
  cudaEvent_t b[kMax] = {}, e[kMax] = {};
  bool used[kMax] = {};
  int nl[kMax] = {};          // launches in the pending phase
  double ms[kMax] = {};
  long long launches[kMax] = {};
};
extern const char* const kPhaseNames[kNumPhases];

struct Launch {
  cudaStream_t stream = nullptr;
  int sms = 152;
  Prof* prof = nullptr;
};

inline void prof_begin(const Launch& L, int id) {
  if (L.prof) cudaEventRecord(L.prof->b[id], L.stream);
}
inline void prof_end(const Launch& L, int id, int nlaunch) {
  if (L.prof) {
    cudaEventRecord(L.prof->e[id], L.stream);
    L.prof->used[id] = true;
    L.prof->nl[id] = nlaunch;
  }
}
// Wait for the recorded phases and add their durations (device time).
inline void prof_collect(Prof* p) {
  if (!p) return;
  for (int i = 0; i < Prof::kMax; ++i) {
    if (!p->used[i]) continue;
    float ms = 0.f;
    cudaEventSynchronize(p->e[i]);
    cudaEventElapsedTime(&ms, p->b[i], p->e[i]);
    p->ms[i] += ms;
    p->launches[i] += p->nl[i];
    p->used[i] = false;
  }
}

// ---- operator products (bk_spmm.cu) ----
// out = A in  (or out = sub - A in when sub != null), with optional fused epilogue.
template <typename T>
cudaError_t spmm(const Launch& L, const OpDesc& A, int s, const T* in, T* out, const T* sub,
                 const Epi<T>& ep);
cudaError_t op_prepare_stencil(const Launch& L, OpDesc& A, const double* coeffs);
cudaError_t op_make_fp32(const Launch& L, OpDesc& A);
// out[i] = (double)in[i]
cudaError_t widen_block(const Launch& L, int64_t count, const float* in, double* out);
// out[i] = exp(in[i])
cudaError_t exp_block(const Launch& L, int64_t count, const double* in, double* out);
// At = A^T of a CSR operator, columns sorted within every row; At owns its arrays
// (rp_owned, col_owned, val_owned).  Synchronises the stream (the row pointers are
// an exclusive scan of the column counts, formed on the host).
cudaError_t csr_transpose(const Launch& L, const OpDesc& A, OpDesc& At);

// ---- pipelined FP32 kernels (bk_march.cu), s % 4 == 0; cudaErrorNotSupported when a
// request is outside what they cover (the caller then uses the row kernels) ----
// out = A in for CONST7 / VAR7 / EDGE5 stencils, optionally with the symmetric Gram
// in^T out (ep.left == in, ep.sym).
cudaError_t march_spmm4(const Launch& L, const OpDesc& A, int s, const float* in, float* out,
                        const Epi<float>& ep);
// G = X^T Y (Y may equal X).
cudaError_t stream_gram4(const Launch& L, int64_t n, int s, const float* X, const float* Y,
                         const Epi<float>& ep);
// Z = diag(w) X with the symmetric Gram X^T Z (ep.left == X, ep.sym).
cudaError_t stream_diag4(const Launch& L, int64_t n, int s, const float* w, const float* X, float* Z,
                         const Epi<float>& ep);
// Per-cell float quadruples of VAR7 / EDGE5 operators (needs the FP32 copies).
cudaError_t op_make_coef4(const Launch& L, OpDesc& A);
// out[i] = 1 / a_ii of A (point Jacobi, M = diag(A)); *bad = 1 when some a_ii is
// zero or not finite (that entry is written as 0).
cudaError_t jacobi_inverse_diagonal(const Launch& L, const OpDesc& A, double* out, int* bad);
int spmm_grid(const Launch& L, int64_t n, int s);

// ---- row kernels (bk_rows.cu) ----
// G = X^T Y reduced deterministically into gram_out (row stride 32).
template <typename T>
cudaError_t gram(const Launch& L, int64_t n, int s, const T* X, const T* Y, const Epi<T>& ep);
// BCG fused update: X += P*lx ; R = R - Q*lam ; if (!reortho) rho_new = R^T R.
template <typename T>
cudaError_t bcg_update(const Launch& L, int64_t n, int s, const T* P, const T* Q, T* X, T* R,
                       Ctrl* ctrl, double* gpart, int use_fp64_x);
// BCG direction update P = R + P*beta.
template <typename T>
cudaError_t bcg_pupdate(const Launch& L, int64_t n, int s, const T* R, T* P, Ctrl* ctrl);
// The same two updates for FP32 blocks in the quad layout (s % 4 == 0), bk_quad.cu.
cudaError_t bcg_update4(const Launch& L, int64_t n, int s, const float* P, const float* Q, float* X,
                        float* R, Ctrl* ctrl, double* gpart, int rho_mode);
cudaError_t bcg_pupdate4(const Launch& L, int64_t n, int s, const float* R, float* P, Ctrl* ctrl);
// Generic Y = alpha*X*M + beta*Y (M s x s row stride 32 on device), optional fused Gram.
template <typename T>
cudaError_t block_axpy(const Launch& L, int64_t n, int s, const T* X, const double* M,
                       double alpha, T* Y, double beta, const int* done);
cudaError_t adjoint_scatter(const Launch& L, const OpDesc& A, int s, const double* Lam,
                            const double* X, double* g);
cudaError_t edge_theta_grad(const Launch& L, const OpDesc& A, int s, const double* Lam,
                            const double* X, double* g);

// ---- block-parallel subalgebra S_BP^p, FP64 (bk_group.cu): the same steps with
// every s x s coefficient block diagonal (p x p blocks): work O(s p) per row ----
cudaError_t spmm_groups(const Launch& L, const OpDesc& A, int s, int p, const double* P, double* Q,
                        const Epi<double>& ep);
cudaError_t bcg_update_groups(const Launch& L, int64_t n, int s, int p, const double* P, const double* Q,
                              double* X, double* R, Ctrl* ctrl, double* gpart, int rho_mode);
cudaError_t bcg_pupdate_groups(const Launch& L, int64_t n, int s, int p, const double* R, double* P,
                               Ctrl* ctrl);

// ---- TSQR (bk_tsqr.cu) ----
struct TsqrPlan {
  int64_t n = 0;
  int s = 0;
  int tile = 256;              // rows per leaf tile
  int fanin = 8;               // children per tree node
  int levels = 0;              // number of tree levels above the leaves
  int64_t nodes[16] = {0};     // tiles per level (level 0 = the block's row tiles)
  int64_t rows[16] = {0};      // rows per level (level l + 1 = stacked R factors of level l)
  size_t bytes = 0;            // scratch bytes
};
int tsqr_launches(const TsqrPlan& p);
// elem_bytes: 8 for FP64 blocks, 4 for FP32 ones (larger leaf tiles)
TsqrPlan tsqr_plan(int64_t n, int s, int elem_bytes = 8);
// Leaf tiles of X (FP64) factored on their own: Y_t = Q_t explicit, R_t (s x s) at Rloc + t * ldr.
cudaError_t tsqr_local_q(const Launch& L, const TsqrPlan& p, const double* X, double* Y, double* Rloc,
                         int64_t ldr, void* scratch);
// ---- localized Arnoldi (bk_local.cu) ----
// Device layout of the distributed S-QR decomposition of one BGMRes cycle (see bk_local.cu).
struct LocalArnoldi {
  int s = 0, m1 = 0, mx = 0;         // block size, max basis vectors, max blocks per vector
  int64_t n = 0, tiles = 0;
  int tile_rows = 0;
  int levels = 0;                    // tree levels above the tiles
  int fanin = 2;                     // children per tree node
  int64_t nodes[24] = {0};           // nodes per level (level 0 = tiles)
  double** Pb = nullptr;             // device array of m1 local-basis block pointers
  double* Pbh[72] = {nullptr};       // the same pointers on the host (m1 <= 65)
  double* Zt = nullptr;              // [tiles][mx s][s]  local R-factors of the newest block
  double* Zl = nullptr;              // [tiles][mx s][s]  coefficients of the newest basis vector
  double* NB[24] = {nullptr};        // level l: [nodes][m1][fanin][mx s][s] node bases
  double* Rout[24] = {nullptr};      // level l: [nodes][mx s][s] R-factors passed up
  double* Cin[24] = {nullptr};       // level l: [nodes][mx s][s] coefficients passed down
  size_t nb_bytes[24] = {0};
  size_t reduce_smem = 0;
};
size_t local_arnoldi_bytes(int64_t n, int s, int m, int tile_rows, LocalArnoldi* la);
// Lay out `la` in `base` (local_arnoldi_bytes of it); Pb gets its device pointer array.
int local_arnoldi_layout(void* base, LocalArnoldi* la, double* const* pb_host, cudaStream_t st);
// Start a cycle: node bases zeroed.
cudaError_t local_arnoldi_begin(const Launch& L, const LocalArnoldi& la);
// Extend by W (overwritten): k1 basis vectors so far (0 at the cycle start).  Writes
// the new basis vector into V, the projections into Hc (k1 blocks, row stride 32)
// and the normalisation factor into gamma (row stride 32).
cudaError_t local_arnoldi_extend(const Launch& L, const LocalArnoldi& la, const TsqrPlan& tp, void* tsqr_scratch,
                                 int k1, double* W, double* V, double* Hc, double* gamma);
// Y, gamma = Norm(X) (Y may alias X).  gamma -> ctrl-layout s x s (row stride 32).
// If rho_out != null, also the Gram Y^T Y (row stride 32) is produced.
// done: optional stop flag (skip when *done); reortho_flag: optional, skip unless *flag.
template <typename T>
// ld: row stride of X and Y (0: plan.s); a column group of a wider block is
// normalised with X, Y pointing at its first column and ld = the block width.
cudaError_t tsqr(const Launch& L, const TsqrPlan& plan, const T* X, T* Y, double* gamma_out,
                 double* rho_out, void* scratch, double* gpart, unsigned* counter,
                 const int* done, const int* reortho_flag, int ld = 0);

// ---- small s x s kernels (bk_small.cu) ----
cudaError_t small_bcg_init(const Launch& L, Ctrl* ctrl, int eta_positive);
cudaError_t small_bcg_1(const Launch& L, Ctrl* ctrl, const uint8_t* forced);
cudaError_t small_bcg_2(const Launch& L, Ctrl* ctrl, double* history, uint8_t* decisions);
// CholeskyQR2 normaliser of BCG (FP64 block case): the s x s factor of pass 1 or 2
// (pass 1 declines nearly dependent blocks, pass 2 falls back to the TSQR on failure),
// the row pass Y <- Y U^{-1} (with rho_new = Y^T Y when gram), and the direction update
// P <- R-bar + P beta with the second pass R-bar = Y1 U2^{-1} folded in.
cudaError_t small_cholqr(const Launch& L, Ctrl* ctrl, int pass);
cudaError_t cholqr_pass(const Launch& L, int64_t n, int s, double* Y, Ctrl* ctrl, double* gpart, bool gram);
cudaError_t cholqr_pupdate(const Launch& L, int64_t n, int s, double* R, double* P, Ctrl* ctrl);
cudaError_t small_bicg_1(const Launch& L, Ctrl* ctrl, const uint8_t* forced);
cudaError_t small_bicg_2(const Launch& L, Ctrl* ctrl);
cudaError_t small_bicg_3(const Launch& L, Ctrl* ctrl, double* history, uint8_t* decisions);
cudaError_t small_set_identity(const Launch& L, double* M, int s);
// kappa_D of an s x s symmetric matrix A (row stride s, device) into *out (device).
cudaError_t small_kappa_d(const Launch& L, int s, const double* A, double* out);
// The re-orthonormalisation decision eta kappa_D(A) > 1/sqrt(eps) as the solvers take it.
cudaError_t small_criterion(const Launch& L, int s, double eta, double eps, const double* A, int* out);
cudaError_t small_colnorms_from_gram(const Launch& L, Ctrl* ctrl);

// BGMRes small kernels
cudaError_t small_gmres_step(const Launch& L, Ctrl* ctrl, const double* Hc, double* H, double* Gq,
                             double* sig, int k, int m, double* history, int hist_index);
cudaError_t small_gmres_backsub(const Launch& L, Ctrl* ctrl, const double* H, const double* sig,
                                double* zeta, int k_done, int m);

// multi-block tall-skinny kernels (bk_rows.cu)
// H_j[a][c] (+)= sum_r V_j[r][a] W[r][c] for j < nb; H_j = H + j*1024, row stride 32
cudaError_t multi_gram(const Launch& L, int64_t n, int s, const double* const* V, int nb,
                       const double* W, double* H, int accumulate, double* gpart,
                       unsigned* counter, const int* done);
// W[r][c] += sign * sum_j sum_a V_j[r][a] H_j[a][c]   (H_j as above)
cudaError_t multi_axpy(const Launch& L, int64_t n, int s, const double* const* V, int nb,
                       const double* H, double* W, double sign, const int* done);

cudaError_t bicg_final(const Launch& L, int64_t n, int s, double* S, const double* U, double* X,
                       double* P, const double* Q, const double* R0s, Ctrl* ctrl, double* gpart);
cudaError_t vec_add(const Launch& L, int64_t count, const double* x, double* y, const int* done);
cudaError_t diag_sqrt(const Launch& L, int s, const double* G, double* out);
cudaError_t init_sig(const Launch& L, int s, const double* G, double* sig, int nblk);
int multi_gram_grid(const Launch& L, int64_t n, int s, int nb);

// IR helpers (bk_rows.cu)
cudaError_t ir_colnorms(const Launch& L, int64_t n, int s, const double* R, double* norms2,
                        double* gpart, unsigned* counter);
cudaError_t ir_to_fp32(const Launch& L, int64_t n, int s, const double* R, const double* norms,
                       float* R32);
cudaError_t ir_accumulate(const Launch& L, int64_t n, int s, const float* D32,
                          const double* norms, double* X);
cudaError_t cast_block(const Launch& L, int64_t count, const double* in, float* out);

}  // namespace bk
