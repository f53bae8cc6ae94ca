// Row-local block kernels: the BAXPY family of Ch. 3.3 (Table "kernels") as
// used by the solvers, with the block inner products that follow them fused in
// the same pass, plus the tall-skinny multi-block products of block GMRes,
// the iterative-refinement helpers and the adjoint scatter kernels.
//
// s x s coefficient matrices come from the control block (double, row stride
// 32) and are staged in shared memory; lane c of a row's sub-warp reads column
// c of them, the row's own values travel by __shfl_sync.
#include "bk_common.cuh"
#include "bk_internal.h"

namespace bk {

static int row_grid(const Launch& L, int64_t n, int s, int per_sm = kCtasPerSm) {
  const int rpw = 32 / next_pow2_s(s);
  const int64_t rows_per_cta = (int64_t)rpw * kWarps;
  int64_t need = (n + rows_per_cta - 1) / rows_per_cta;
  const int64_t cap = (int64_t)L.sms * per_sm;
  if (need > cap) need = cap;
  return (int)(need < 1 ? 1 : need);
}

template <typename T>
__device__ inline void stage_matrix(T* dst, const double* src, int s) {
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) dst[i] = (T)src[(i / s) * kMaxS + (i % s)];
}

// ---------------------------------------------------------------------------
// BCG fused update (Alg. "2R-CG", the lines after lambda):
//   X      <- X + P * lx            (lx = lambda sigma)
//   R      <- R - Q * lambda        (R-tilde)
//   rho_new = R^T R  (upper, mirrored) when no re-orthonormalisation follows.
template <typename T, int SW>
__global__ void __launch_bounds__(kThreads, min_ctas<T>())
bcg_update_kernel(int64_t n, int s, const T* __restrict__ P, const T* __restrict__ Q,
                  T* __restrict__ X, T* __restrict__ R, Ctrl* ctrl, double* gpart, int rho_mode) {
  if (ctrl->done) return;
  if (ctrl->reortho_now && rho_mode != 2) return;   // then the lean kernel updates, TSQR gives rho
  extern __shared__ double smem[];
  T* lx = reinterpret_cast<T*>(smem);
  T* lam = lx + kMM;
  double* red = reinterpret_cast<double*>(lam + kMM);   // after the two staged matrices
  stage_matrix(lx, ctrl->lx, s);
  stage_matrix(lam, ctrl->lam, s);
  const bool want_rho = rho_mode == 2 || (rho_mode != 0 && ctrl->reortho_now == 0);
  __syncthreads();
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31, c = lane & (SW - 1), rs = lane / SW;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  constexpr bool kPair = (sizeof(T) == 8) && (SW >= 2);
  double acc[SW];
#pragma unroll
  for (int a = 0; a < SW; ++a) acc[a] = 0.0;
  T acc_t[SW];
#pragma unroll
  for (int a = 0; a < SW; ++a) acc_t[a] = T(0);
  SymGramPair<kPair ? SW : 2> pg;
  pg.zero();
  int since = 0;
  auto do_row = [&](int64_t r) -> T {
    const bool ok = (r < n) && (c < s);
    const T p = ok ? P[r * s + c] : T(0);
    const T q = ok ? Q[r * s + c] : T(0);
    T dx = T(0), rq = T(0);
#pragma unroll
    for (int a = 0; a < SW; ++a) {
      const T pa = sw_bcast<SW>(p, a);
      const T qa = sw_bcast<SW>(q, a);
      if (a < s && c < s) {
        dx = fma(pa, lx[a * s + c], dx);
        rq = fma(qa, lam[a * s + c], rq);
      }
    }
    T rt = T(0);
    if (ok) {
      X[r * s + c] += dx;
      rt = R[r * s + c] - rq;
      R[r * s + c] = rt;
    }
    return rt;
  };
  auto accum_row = [&](T rt) {
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int a = 0; a < SW; ++a) {
        const T ra = sw_bcast<SW>(rt, a);
        if (a <= c) acc[a] = fma((double)ra, (double)rt, acc[a]);
      }
    } else {
#pragma unroll
      for (int a = 0; a < SW; ++a) {
        const T ra = sw_bcast<SW>(rt, a);
        if (a <= c) acc_t[a] = fma(ra, rt, acc_t[a]);
      }
      if (++since == kF32Window) {
#pragma unroll
        for (int a = 0; a < SW; ++a) { acc[a] += (double)acc_t[a]; acc_t[a] = T(0); }
        since = 0;
      }
    }
  };
  for (int64_t base = gw * RPW; base < n; base += 2 * nw * RPW) {
    const T rA = do_row(base + rs);
    const T rB = do_row(base + nw * RPW + rs);
    if (want_rho) {
      if constexpr (kPair) pg.add((double)rA, (double)rA, (double)rB, (double)rB);
      else { accum_row(rA); accum_row(rB); }
    }
  }
  if (!want_rho) return;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int a = 0; a < SW; ++a) acc[a] += (double)acc_t[a];
  }
  const int cnt = ut_count(s);
  double* part = red;
  double* scratch = red + cnt + 1;
  if constexpr (kPair) pg.cta_reduce(s, scratch, part);
  else cta_reduce_gram<SW>(acc, s, true, scratch, part);
  if (!grid_reduce_last(part, cnt, gpart, ctrl->counters[kCntB])) return;
  unpack_gram(part, s, true, ctrl->rho_new);
}

// The same update without a Gram (iterations that re-orthonormalise, where the
// normaliser produces rho, and BBiCGStab's S = R - Q lambda):  X <- X + P lx,
// R <- R - Q lam.  Few registers, both rows' loads issued before the shuffles.
template <typename T, int SW>
__global__ void __launch_bounds__(kThreads, 4)
bcg_update_lean_kernel(int64_t n, int s, const T* __restrict__ P, const T* __restrict__ Q,
                       T* __restrict__ X, T* __restrict__ R, Ctrl* ctrl, int only_if_reortho) {
  if (ctrl->done) return;
  if (only_if_reortho && !ctrl->reortho_now) return;
  __shared__ T lx[kMM];
  __shared__ T lam[kMM];
  stage_matrix(lx, ctrl->lx, s);
  stage_matrix(lam, ctrl->lam, s);
  __syncthreads();
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31, c = lane & (SW - 1), rs = lane / SW;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  for (int64_t base = gw * RPW; base < n; base += 2 * nw * RPW) {
    const int64_t rA = base + rs, rB = base + nw * RPW + rs;
    const bool okA = (rA < n) && (c < s), okB = (rB < n) && (c < s);
    const T pA = okA ? P[rA * s + c] : T(0), pB = okB ? P[rB * s + c] : T(0);
    const T qA = okA ? Q[rA * s + c] : T(0), qB = okB ? Q[rB * s + c] : T(0);
    const T xA = okA ? X[rA * s + c] : T(0), xB = okB ? X[rB * s + c] : T(0);
    const T zA = okA ? R[rA * s + c] : T(0), zB = okB ? R[rB * s + c] : T(0);
    T dxA = T(0), dxB = T(0), rqA = T(0), rqB = T(0);
#pragma unroll
    for (int a = 0; a < SW; ++a) {
      const T paA = sw_bcast<SW>(pA, a), paB = sw_bcast<SW>(pB, a);
      const T qaA = sw_bcast<SW>(qA, a), qaB = sw_bcast<SW>(qB, a);
      if (a < s && c < s) {
        const T l1 = lx[a * s + c], l2 = lam[a * s + c];
        dxA = fma(paA, l1, dxA); dxB = fma(paB, l1, dxB);
        rqA = fma(qaA, l2, rqA); rqB = fma(qaB, l2, rqB);
      }
    }
    if (okA) { X[rA * s + c] = xA + dxA; R[rA * s + c] = zA - rqA; }
    if (okB) { X[rB * s + c] = xB + dxB; R[rB * s + c] = zB - rqB; }
  }
}

// BCG direction update (Eq. "cg_update_p" with M = I):  P <- R + P * beta.
template <typename T, int SW>
__global__ void __launch_bounds__(kThreads, 4)
bcg_pupdate_kernel(int64_t n, int s, const T* __restrict__ R, T* __restrict__ P, Ctrl* ctrl) {
  if (ctrl->done) return;
  __shared__ T beta[kMM];
  stage_matrix(beta, ctrl->beta, s);
  __syncthreads();
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31, c = lane & (SW - 1), rs = lane / SW;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  // two row groups per trip: both rows' loads are issued before the shuffles
  for (int64_t base = gw * RPW; base < n; base += 2 * nw * RPW) {
    const int64_t rA = base + rs, rB = base + nw * RPW + rs;
    const bool okA = (rA < n) && (c < s), okB = (rB < n) && (c < s);
    const T pA = okA ? P[rA * s + c] : T(0);
    const T pB = okB ? P[rB * s + c] : T(0);
    const T xA = okA ? R[rA * s + c] : T(0);
    const T xB = okB ? R[rB * s + c] : T(0);
    T accA = T(0), accB = T(0);
#pragma unroll
    for (int a = 0; a < SW; ++a) {
      const T paA = sw_bcast<SW>(pA, a);
      const T paB = sw_bcast<SW>(pB, a);
      if (a < s && c < s) {
        const T b = beta[a * s + c];
        accA = fma(paA, b, accA);
        accB = fma(paB, b, accB);
      }
    }
    if (okA) P[rA * s + c] = xA + accA;
    if (okB) P[rB * s + c] = xB + accB;
  }
}

template <typename T, int SW>
static cudaError_t launch_update(const Launch& L, int64_t n, int s, const T* P, const T* Q, T* X,
                                 T* R, Ctrl* ctrl, double* gpart, int rho_mode) {
  const size_t sm = 2 * kMM * sizeof(T) + sizeof(double) * (ut_count(s) + 2 + kWarps * ut_count(s));
  auto k = bcg_update_kernel<T, SW>;
  if (sm > 44 * 1024) {   // 48 KB default includes the static reduction buffers
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const int grid = row_grid(L, n, s, resident_ctas(k, sm));
  k<<<grid, kThreads, sm, L.stream>>>(n, s, P, Q, X, R, ctrl, gpart, rho_mode);
  return cudaGetLastError();
}

#define BK_SW_DISPATCH(s, ...)                         \
  switch (next_pow2_s(s)) {                            \
    case 1: { constexpr int SW = 1; __VA_ARGS__; }     \
    case 2: { constexpr int SW = 2; __VA_ARGS__; }     \
    case 4: { constexpr int SW = 4; __VA_ARGS__; }     \
    case 8: { constexpr int SW = 8; __VA_ARGS__; }     \
    case 16: { constexpr int SW = 16; __VA_ARGS__; }   \
    case 32: { constexpr int SW = 32; __VA_ARGS__; }   \
    default: return cudaErrorInvalidValue;             \
  }

// rho_mode 1 (BCG): the lean kernel runs when the iteration re-orthonormalises,
// the Gram-carrying kernel otherwise (the device flag picks; the other returns).
// rho_mode 0 (BBiCGStab): the lean kernel always.
// rho_mode 2 (FP64 BCG with the CholeskyQR2 normaliser): the Gram-carrying kernel
// always, its rho_new = R-tilde^T R-tilde being the normaliser's first Gram.
template <typename T>
cudaError_t bcg_update(const Launch& L, int64_t n, int s, const T* P, const T* Q, T* X, T* R,
                       Ctrl* ctrl, double* gpart, int rho_mode) {
  if constexpr (sizeof(T) == 4) {
    if (s % 4 == 0) return bcg_update4(L, n, s, P, Q, X, R, ctrl, gpart, rho_mode);
  }
  if (rho_mode == 2) BK_SW_DISPATCH(s, return launch_update<T, SW>(L, n, s, P, Q, X, R, ctrl, gpart, rho_mode));
  BK_SW_DISPATCH(s, {
    const int grid = row_grid(L, n, s, resident_ctas(bcg_update_lean_kernel<T, SW>, 0));
    bcg_update_lean_kernel<T, SW><<<grid, kThreads, 0, L.stream>>>(n, s, P, Q, X, R, ctrl, rho_mode);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || rho_mode == 0) return e;
    return launch_update<T, SW>(L, n, s, P, Q, X, R, ctrl, gpart, rho_mode);
  });
}

template <typename T>
cudaError_t bcg_pupdate(const Launch& L, int64_t n, int s, const T* R, T* P, Ctrl* ctrl) {
  if constexpr (sizeof(T) == 4) {
    if (s % 4 == 0) return bcg_pupdate4(L, n, s, R, P, ctrl);
  }
  BK_SW_DISPATCH(s, bcg_pupdate_kernel<T, SW><<<row_grid(L, n, s, resident_ctas(bcg_pupdate_kernel<T, SW>, 0)),
                                                 kThreads, 0, L.stream>>>(n, s, R, P, ctrl);
                 return cudaGetLastError());
}

// Upper-triangular product of TWO rows per sub-warp without idle lanes (FP64):
// y_c = sum_{a <= c} x_a U_ac (U s x s, row stride s, upper triangular).  Lane c takes
// column c of row A (c + 1 terms) and column SW - 1 - c of row B (SW - c terms), SW + 1
// FMAs per lane whatever c is; the terms of every entry are added in the order a = 0, 1,
// ...  On exit lane c holds y_A[c] and y_B[c] (row B's values moved back by a shuffle).
template <int SW>
__device__ __forceinline__ void tri_pair(double xA, double xB, const double* U, int s, double& yA,
                                         double& yB) {
  const int c = threadIdx.x & (SW - 1);
  const int cB = SW - 1 - c;
  double accA = 0.0, accB = 0.0;
#pragma unroll
  for (int t = 0; t <= SW; ++t) {
    const bool first = t <= c;
    const int a = first ? t : t - c - 1;
    const double va = __shfl_sync(0xffffffffu, xA, a, SW);
    const double vb = __shfl_sync(0xffffffffu, xB, a, SW);
    const int col = first ? c : cB;
    const double u = (a < s && col < s) ? U[a * s + col] : 0.0;
    const double r = fma(first ? va : vb, u, first ? accA : accB);
    if (first) accA = r; else accB = r;
  }
  yA = accA;
  yB = __shfl_sync(0xffffffffu, accB, cB, SW);
}

// CholeskyQR2 row pass (FP64): Y <- Y U^{-1} in place with U^{-1} = ctrl->cq_inv (upper
// triangular), and with kGram rho_new = Y^T Y (upper, mirrored) through the last-CTA grid
// reduction.  Runs only while ctrl->qr_fast == 1.
template <int SW, bool kGram>
__global__ void __launch_bounds__(kThreads, 1)
cholqr_pass_kernel(int64_t n, int s, double* __restrict__ Y, Ctrl* ctrl, double* gpart) {
  if (ctrl->done || ctrl->qr_fast != 1) return;
  extern __shared__ double smem[];
  double* ui = smem;
  double* red = smem + kMM;
  stage_matrix(ui, ctrl->cq_inv, s);
  __syncthreads();
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31, c = lane & (SW - 1), rs = lane / SW;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  constexpr bool kPair = SW >= 2;
  double acc[SW];
#pragma unroll
  for (int a = 0; a < SW; ++a) acc[a] = 0.0;
  SymGramPair<kPair ? SW : 2> pg;
  pg.zero();
  for (int64_t base = gw * RPW; base < n; base += 2 * nw * RPW) {
    const int64_t rA = base + rs, rB = base + nw * RPW + rs;
    const bool okA = (rA < n) && (c < s), okB = (rB < n) && (c < s);
    const double xA = okA ? Y[rA * s + c] : 0.0, xB = okB ? Y[rB * s + c] : 0.0;
    double yA, yB;
    tri_pair<SW>(xA, xB, ui, s, yA, yB);
    if (okA) Y[rA * s + c] = yA;
    if (okB) Y[rB * s + c] = yB;
    if constexpr (kGram) {
      if constexpr (kPair) {
        pg.add(yA, yA, yB, yB);
      } else {
        acc[0] = fma(yA, yA, acc[0]);
        acc[0] = fma(yB, yB, acc[0]);
      }
    }
  }
  if constexpr (!kGram) return;
  const int cnt = ut_count(s);
  double* part = red;
  double* scratch = red + cnt + 1;
  if constexpr (kPair) pg.cta_reduce(s, scratch, part);
  else cta_reduce_gram<SW>(acc, s, true, scratch, part);
  if (!grid_reduce_last(part, cnt, gpart, ctrl->counters[kCntC])) return;
  unpack_gram(part, s, true, ctrl->rho_new);
}

cudaError_t cholqr_pass(const Launch& L, int64_t n, int s, double* Y, Ctrl* ctrl, double* gpart, bool gram) {
  const size_t sm = sizeof(double) * (kMM + ut_count(s) + 2 + kWarps * ut_count(s));
  BK_SW_DISPATCH(s, {
    auto k = gram ? cholqr_pass_kernel<SW, true> : cholqr_pass_kernel<SW, false>;
    if (sm > 44 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    k<<<row_grid(L, n, s, resident_ctas(k, sm)), kThreads, sm, L.stream>>>(n, s, Y, ctrl, gpart);
    return cudaGetLastError();
  });
}

// BCG direction update with the second CholeskyQR2 pass folded in (FP64, M = I): where
// the iteration's normaliser was CholeskyQR2 (ctrl->qr_fast == 1), R-bar = Y1 U2^{-1} is
// formed here (written back) and P <- R-bar + P beta uses it from registers; otherwise
// this is P <- R + P beta.
template <int SW>
__global__ void __launch_bounds__(kThreads, 2)
cholqr_pupdate_kernel(int64_t n, int s, double* __restrict__ R, double* __restrict__ P, Ctrl* ctrl) {
  if (ctrl->done) return;
  __shared__ double beta[kMM];
  __shared__ double ui[kMM];
  const bool fq = ctrl->qr_fast == 1;
  stage_matrix(beta, ctrl->beta, s);
  if (fq) stage_matrix(ui, ctrl->cq_inv, s);
  __syncthreads();
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31, c = lane & (SW - 1), rs = lane / SW;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  for (int64_t base = gw * RPW; base < n; base += 2 * nw * RPW) {
    const int64_t rA = base + rs, rB = base + nw * RPW + rs;
    const bool okA = (rA < n) && (c < s), okB = (rB < n) && (c < s);
    const double pA = okA ? P[rA * s + c] : 0.0, pB = okB ? P[rB * s + c] : 0.0;
    double xA = okA ? R[rA * s + c] : 0.0, xB = okB ? R[rB * s + c] : 0.0;
    if (fq) {
      double yA, yB;
      tri_pair<SW>(xA, xB, ui, s, yA, yB);
      xA = yA;
      xB = yB;
      if (okA) R[rA * s + c] = xA;
      if (okB) R[rB * s + c] = xB;
    }
    double accA = 0.0, accB = 0.0;
#pragma unroll
    for (int a = 0; a < SW; ++a) {
      const double paA = sw_bcast<SW>(pA, a), paB = sw_bcast<SW>(pB, a);
      if (a < s && c < s) {
        const double b = beta[a * s + c];
        accA = fma(paA, b, accA);
        accB = fma(paB, b, accB);
      }
    }
    if (okA) P[rA * s + c] = xA + accA;
    if (okB) P[rB * s + c] = xB + accB;
  }
}

cudaError_t cholqr_pupdate(const Launch& L, int64_t n, int s, double* R, double* P, Ctrl* ctrl) {
  BK_SW_DISPATCH(s, cholqr_pupdate_kernel<SW><<<row_grid(L, n, s, resident_ctas(cholqr_pupdate_kernel<SW>, 0)),
                                                kThreads, 0, L.stream>>>(n, s, R, P, ctrl);
                 return cudaGetLastError());
}

template cudaError_t bcg_update<double>(const Launch&, int64_t, int, const double*, const double*,
                                        double*, double*, Ctrl*, double*, int);
template cudaError_t bcg_update<float>(const Launch&, int64_t, int, const float*, const float*,
                                       float*, float*, Ctrl*, double*, int);
template cudaError_t bcg_pupdate<double>(const Launch&, int64_t, int, const double*, double*, Ctrl*);
template cudaError_t bcg_pupdate<float>(const Launch&, int64_t, int, const float*, float*, Ctrl*);

// ---------------------------------------------------------------------------
// Generic Y <- alpha * X * M + beta * Y  (M: s x s, row stride 32, device double).
template <typename T, int SW>
__global__ void __launch_bounds__(kThreads)
block_axpy_kernel(int64_t n, int s, const T* __restrict__ X, const double* __restrict__ Mg,
                  double alpha, T* __restrict__ Y, double beta, const int* done) {
  if (done && *done) return;
  __shared__ T M[kMM];
  stage_matrix(M, Mg, s);
  __syncthreads();
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31, c = lane & (SW - 1), rs = lane / SW;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  for (int64_t base = gw * RPW; base < n; base += nw * RPW) {
    const int64_t r = base + rs;
    const bool ok = (r < n) && (c < s);
    const T x = ok ? X[r * s + c] : T(0);
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < SW; ++a) {
      const T xa = sw_bcast<SW>(x, a);
      if (a < s && c < s) acc = fma(xa, M[a * s + c], acc);
    }
    if (ok) Y[r * s + c] = (beta == 0.0 ? T(0) : (T)beta * Y[r * s + c]) + (T)alpha * acc;
  }
}

template <typename T>
cudaError_t block_axpy(const Launch& L, int64_t n, int s, const T* X, const double* M, double alpha,
                       T* Y, double beta, const int* done) {
  const int grid = row_grid(L, n, s);
  BK_SW_DISPATCH(s, block_axpy_kernel<T, SW><<<grid, kThreads, 0, L.stream>>>(n, s, X, M, alpha, Y,
                                                                               beta, done);
                 return cudaGetLastError());
}
template cudaError_t block_axpy<double>(const Launch&, int64_t, int, const double*, const double*,
                                        double, double*, double, const int*);
template cudaError_t block_axpy<float>(const Launch&, int64_t, int, const float*, const double*,
                                       double, float*, double, const int*);

// ---------------------------------------------------------------------------
// Block GMRes projections (Ch. 9.1, classical block Gram-Schmidt): for the
// basis blocks V_0..V_{nb-1} and the new block W,
//   partial[cta][j][a][c] = sum over the CTA's rows of V_j[r][a] W[r][c],
// then a second kernel sums the CTA partials in CTA order (deterministic).
__global__ void __launch_bounds__(kThreads)
multi_gram_partial(int64_t n, int s, const double* const* __restrict__ V, int nb,
                   const double* __restrict__ W, double* __restrict__ gpart, const int* done) {
  if (done && *done) return;
  const int j = blockIdx.y;
  const double* __restrict__ Vj = V[j];
  const int ss = s * s;
  const int G = gridDim.x;
  const int64_t r0 = n * blockIdx.x / G, r1 = n * (blockIdx.x + 1) / G;
  __shared__ double red[kThreads];
  if (ss >= kThreads) {
    for (int o = threadIdx.x; o < ss; o += kThreads) {
      const int a = o / s, c = o % s;
      double acc = 0.0;
      for (int64_t r = r0; r < r1; ++r) acc = fma(Vj[r * s + a], W[r * s + c], acc);
      gpart[((size_t)blockIdx.x * nb + j) * ss + o] = acc;
    }
  } else {
    const int Rq = kThreads / ss;      // row subsets per output
    const int o = threadIdx.x % ss, q = threadIdx.x / ss;
    const int a = o / s, c = o % s;
    double acc = 0.0;
    if (q < Rq)
      for (int64_t r = r0 + q; r < r1; r += Rq) acc = fma(Vj[r * s + a], W[r * s + c], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < ss) {
      double t = 0.0;
      for (int k = 0; k < Rq; ++k) t += red[k * ss + threadIdx.x];
      gpart[((size_t)blockIdx.x * nb + j) * ss + threadIdx.x] = t;
    }
  }
}

__global__ void multi_gram_reduce(int G, int nb, int s, const double* __restrict__ gpart,
                                  double* __restrict__ H, int accumulate, const int* done) {
  if (done && *done) return;
  const int ss = s * s, total = nb * ss;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < G; ++b) t += gpart[(size_t)b * total + i];
    const int j = i / ss, a = (i % ss) / s, c = i % s;
    double* h = H + (size_t)j * kMM + a * kMaxS + c;
    *h = accumulate ? *h + t : t;
  }
}

int multi_gram_grid(const Launch& L, int64_t n, int s, int nb) {
  int64_t g = (int64_t)L.sms * 2 / (nb > 0 ? nb : 1);
  if (g < 8) g = 8;
  const int64_t rows_min = 64;
  if (g * rows_min > n) g = (n + rows_min - 1) / rows_min;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t multi_gram(const Launch& L, int64_t n, int s, const double* const* V, int nb,
                       const double* W, double* H, int accumulate, double* gpart, unsigned*,
                       const int* done) {
  const int G = multi_gram_grid(L, n, s, nb);
  dim3 grid(G, nb);
  multi_gram_partial<<<grid, kThreads, 0, L.stream>>>(n, s, V, nb, W, gpart, done);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int total = nb * s * s;
  multi_gram_reduce<<<(total + 255) / 256, 256, 0, L.stream>>>(G, nb, s, gpart, H, accumulate, done);
  return cudaGetLastError();
}

// W[r][c] += sign * sum_j sum_a V_j[r][a] H[j*s + a][c]   (H row stride s).
template <int SW>
__global__ void __launch_bounds__(kThreads)
multi_axpy_kernel(int64_t n, int s, const double* const* __restrict__ V, int nb,
                  const double* __restrict__ H, double* __restrict__ W, double sign, const int* done) {
  if (done && *done) return;
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31, c = lane & (SW - 1), rs = lane / SW;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  for (int64_t base = gw * RPW; base < n; base += nw * RPW) {
    const int64_t r = base + rs;
    const bool ok = (r < n) && (c < s);
    double acc = 0.0;
    for (int j = 0; j < nb; ++j) {
      const double v = ok ? V[j][r * s + c] : 0.0;
      const double* Hj = H + (size_t)j * kMM;
#pragma unroll
      for (int a = 0; a < SW; ++a) {
        const double va = sw_bcast<SW>(v, a);
        if (a < s && c < s) acc = fma(va, __ldg(Hj + a * kMaxS + c), acc);
      }
    }
    if (ok) W[r * s + c] += sign * acc;
  }
}

cudaError_t multi_axpy(const Launch& L, int64_t n, int s, const double* const* V, int nb,
                       const double* H, double* W, double sign, const int* done) {
  const int grid = row_grid(L, n, s);
  BK_SW_DISPATCH(s, multi_axpy_kernel<SW><<<grid, kThreads, 0, L.stream>>>(n, s, V, nb, H, W, sign,
                                                                            done);
                 return cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Iterative refinement helpers.
// Column sums of squares (norms2[c] = sum_r R[r][c]^2), deterministic.
template <int SW>
__global__ void __launch_bounds__(kThreads)
colnorm_kernel(int64_t n, int s, const double* __restrict__ R, double* __restrict__ norms2,
               double* gpart, unsigned* counter) {
  __shared__ double red[kWarps * kMaxS + kMaxS];
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31, c = lane & (SW - 1), rs = lane / SW, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  double acc = 0.0;
  for (int64_t base = gw * RPW; base < n; base += nw * RPW) {
    const int64_t r = base + rs;
    if (r < n && c < s) { const double v = R[r * s + c]; acc = fma(v, v, acc); }
  }
#pragma unroll
  for (int off = SW; off < 32; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane < SW && c < s) red[warp * kMaxS + c] = acc;
  __syncthreads();
  double* part = red + kWarps * kMaxS;
  if (threadIdx.x < s) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[w * kMaxS + threadIdx.x];
    part[threadIdx.x] = t;
  }
  __syncthreads();
  if (!grid_reduce_last(part, s, gpart, counter)) return;
  if (threadIdx.x < s) norms2[threadIdx.x] = part[threadIdx.x];
}

cudaError_t ir_colnorms(const Launch& L, int64_t n, int s, const double* R, double* norms2,
                        double* gpart, unsigned* counter) {
  const int grid = row_grid(L, n, s, 2);
  BK_SW_DISPATCH(s, colnorm_kernel<SW><<<grid, kThreads, 0, L.stream>>>(n, s, R, norms2, gpart,
                                                                         counter);
                 return cudaGetLastError());
}

// R32 = R / norm (column scaling, norm = sqrt(norms2), zero columns left unscaled).
// Element-wise over the row-major n x s block with a block size and grid stride
// that are multiples of s, so that every thread stays on one column and forms
// its scale factor once (FP64 square roots and divisions per element would make
// these passes FP64-bound).
__global__ void ir_to_fp32_kernel(int64_t total, int s, const double* __restrict__ R,
                                  const double* __restrict__ norms2, float* __restrict__ R32) {
  const double n2 = norms2[threadIdx.x % s];
  const double sc = n2 > 0.0 ? 1.0 / sqrt(n2) : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    R32[i] = (float)(R[i] * sc);
}

// X += D32 * norm (undo the column scaling), same launch shape.
__global__ void ir_accumulate_kernel(int64_t total, int s, const float* __restrict__ D32,
                                     const double* __restrict__ norms2, double* __restrict__ X) {
  const double n2 = norms2[threadIdx.x % s];
  const double sc = n2 > 0.0 ? sqrt(n2) : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    X[i] += (double)D32[i] * sc;
}

static int elem_grid2(const Launch& L, int64_t count) {
  int64_t g = (count + 255) / 256;
  const int64_t cap = (int64_t)L.sms * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// Block size (256 / s) * s: a multiple of s, so the column of element i is threadIdx.x % s.
static int col_block(int s) { return (256 / s) * s; }

static int col_grid(const Launch& L, int64_t total, int bs) {
  int64_t g = (total + bs - 1) / bs;
  const int64_t cap = (int64_t)L.sms * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t ir_to_fp32(const Launch& L, int64_t n, int s, const double* R, const double* norms2,
                       float* R32) {
  const int64_t total = n * s;
  const int bs = col_block(s);
  ir_to_fp32_kernel<<<col_grid(L, total, bs), bs, 0, L.stream>>>(total, s, R, norms2, R32);
  return cudaGetLastError();
}

cudaError_t ir_accumulate(const Launch& L, int64_t n, int s, const float* D32, const double* norms2,
                          double* X) {
  const int64_t total = n * s;
  const int bs = col_block(s);
  ir_accumulate_kernel<<<col_grid(L, total, bs), bs, 0, L.stream>>>(total, s, D32, norms2, X);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adjoint scatter on the CSR pattern: g[e] = -sum_k Lam[i][k] X[col[e]][k].
// One thread per stored entry; the row index comes from a binary search in
// row_ptr (entries of a warp mostly share one row, so Lam's row is reused).
__global__ void adjoint_scatter_kernel(int64_t n, int64_t nnz, int s, const int32_t* __restrict__ row_ptr,
                                       const int32_t* __restrict__ col, const double* __restrict__ Lam,
                                       const double* __restrict__ X, double* __restrict__ g) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n - 1;           // find i with row_ptr[i] <= e < row_ptr[i+1]
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const double* li = Lam + lo * s;
    const double* xj = X + (int64_t)col[e] * s;
    double acc = 0.0;
    for (int k = 0; k < s; ++k) acc = fma(li[k], xj[k], acc);
    g[e] = -acc;
  }
}

cudaError_t adjoint_scatter(const Launch& L, const OpDesc& A, int s, const double* Lam,
                            const double* X, double* g) {
  if (A.kind != kOpCsr) return cudaErrorInvalidValue;
  if (A.nnz == 0) return cudaSuccess;
  adjoint_scatter_kernel<<<elem_grid2(L, A.nnz), 256, 0, L.stream>>>(A.n, A.nnz, s, A.row_ptr, A.col,
                                                                     Lam, X, g);
  return cudaGetLastError();
}

// dL/dtheta_e for the per-edge 2D operator with a_e = exp(theta_e):
//   interior edge (i, j): -a_e sum_k (Lam_ik - Lam_jk)(X_ik - X_jk)
//   boundary edge (i):    -a_e sum_k Lam_ik X_ik
__global__ void edge_grad_kernel(int nx, int ny, int s, const double* __restrict__ edges,
                                 const double* __restrict__ Lam, const double* __restrict__ X,
                                 double* __restrict__ g) {
  const int64_t nh = (int64_t)ny * (nx + 1);
  const int64_t total = nh + (int64_t)(ny + 1) * nx;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = -1, j = -1;                       // the two cells (j = -1: boundary)
    if (e < nh) {
      const int y = (int)(e / (nx + 1)), x = (int)(e % (nx + 1));
      if (x > 0 && x < nx) { i = (int64_t)y * nx + x - 1; j = i + 1; }
      else i = (int64_t)y * nx + (x == 0 ? 0 : nx - 1);
    } else {
      const int64_t f = e - nh;
      const int y = (int)(f / nx), x = (int)(f % nx);
      if (y > 0 && y < ny) { i = (int64_t)(y - 1) * nx + x; j = i + nx; }
      else i = (int64_t)(y == 0 ? 0 : ny - 1) * nx + x;
    }
    const double* li = Lam + i * s;
    const double* xi = X + i * s;
    double acc = 0.0;
    if (j < 0) {
      for (int k = 0; k < s; ++k) acc = fma(li[k], xi[k], acc);
    } else {
      const double* lj = Lam + j * s;
      const double* xj = X + j * s;
      for (int k = 0; k < s; ++k) acc = fma(li[k] - lj[k], xi[k] - xj[k], acc);
    }
    g[e] = -edges[e] * acc;
  }
}

cudaError_t edge_theta_grad(const Launch& L, const OpDesc& A, int s, const double* Lam,
                            const double* X, double* g) {
  if (A.kind != kOpEdge5) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)A.ny * (A.nx + 1) + (int64_t)(A.ny + 1) * A.nx;
  edge_grad_kernel<<<elem_grid2(L, total), 256, 0, L.stream>>>(A.nx, A.ny, s, A.edges, Lam, X, g);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Last row pass of a BBiCGStab iteration (Alg. "BlockBiCGStab_with_reortho",
// M = I, T-hat = S-hat):
//   X <- X + S * lx          (lx = omega sigma^{k+1})
//   R <- S - omega U         (R-hat^{k+1}, written over S)
//   P <- R + (P - omega Q) beta
// with the Grams R^T R (upper, mirrored; kappa_D and residual norms) and
// R0s^T R (next lambda) accumulated in the same pass.
template <int SW>
__global__ void __launch_bounds__(kThreads)
bicg_final_kernel(int64_t n, int s, double* __restrict__ S, const double* __restrict__ U,
                  double* __restrict__ X, double* __restrict__ P, const double* __restrict__ Q,
                  const double* __restrict__ R0s, Ctrl* ctrl, double* gpart) {
  if (ctrl->done) return;
  extern __shared__ double smem[];
  double* lx = smem;
  double* beta = smem + kMM;
  double* red = smem + 2 * kMM;
  stage_matrix(lx, ctrl->lx, s);
  stage_matrix(beta, ctrl->beta, s);
  const double omega = ctrl->omega;
  __syncthreads();
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31, c = lane & (SW - 1), rs = lane / SW;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  double a1[SW], a2[SW];
#pragma unroll
  for (int a = 0; a < SW; ++a) { a1[a] = 0.0; a2[a] = 0.0; }
  for (int64_t base = gw * RPW; base < n; base += nw * RPW) {
    const int64_t r = base + rs;
    const bool ok = (r < n) && (c < s);
    const double sv = ok ? S[r * s + c] : 0.0;
    const double u = ok ? U[r * s + c] : 0.0;
    const double pq = ok ? fma(-omega, Q[r * s + c], P[r * s + c]) : 0.0;
    const double rn = fma(-omega, u, sv);
    double dx = 0.0, pb = 0.0;
#pragma unroll
    for (int a = 0; a < SW; ++a) {
      const double sa = sw_bcast<SW>(sv, a);
      const double pa = sw_bcast<SW>(pq, a);
      if (a < s && c < s) { dx = fma(sa, lx[a * s + c], dx); pb = fma(pa, beta[a * s + c], pb); }
    }
    const double l0 = ok ? R0s[r * s + c] : 0.0;
    if (ok) {
      X[r * s + c] += dx;
      S[r * s + c] = rn;
      P[r * s + c] = rn + pb;
    }
    const double rv = ok ? rn : 0.0;
#pragma unroll
    for (int a = 0; a < SW; ++a) {
      const double ra = sw_bcast<SW>(rv, a);
      const double la = sw_bcast<SW>(l0, a);
      if (a <= c) a1[a] = fma(ra, rv, a1[a]);
      a2[a] = fma(la, rv, a2[a]);
    }
  }
  const int c1 = ut_count(s), c2 = s * s;
  double* part = red;                       // c1 + c2
  double* scratch = red + c1 + c2 + 1;      // kWarps * c2
  cta_reduce_gram<SW>(a1, s, true, scratch, part);
  cta_reduce_gram<SW>(a2, s, false, scratch, part + c1);
  if (!grid_reduce_last(part, c1 + c2, gpart, ctrl->counters[kCntD])) return;
  unpack_gram(part, s, true, ctrl->rho);
  unpack_gram(part + c1, s, false, ctrl->g2);
}

cudaError_t bicg_final(const Launch& L, int64_t n, int s, double* S, const double* U, double* X,
                       double* P, const double* Q, const double* R0s, Ctrl* ctrl, double* gpart) {
  const int grid = row_grid(L, n, s, 2);
  const size_t sm = sizeof(double) * (2 * kMM + ut_count(s) + s * s + 2 + kWarps * s * s);
  BK_SW_DISPATCH(s, {
    auto k = bicg_final_kernel<SW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<grid, kThreads, sm, L.stream>>>(n, s, S, U, X, P, Q, R0s, ctrl, gpart);
    return cudaGetLastError();
  });
}

// y += x (count doubles), skipped when *done.
__global__ void vec_add_kernel(int64_t count, const double* __restrict__ x, double* __restrict__ y,
                               const int* done) {
  if (done && *done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}
cudaError_t vec_add(const Launch& L, int64_t count, const double* x, double* y, const int* done) {
  vec_add_kernel<<<elem_grid2(L, count), 256, 0, L.stream>>>(count, x, y, done);
  return cudaGetLastError();
}

// n0[i] = sqrt(G[i][i]) for a ctrl-layout Gram G.
__global__ void diag_sqrt_kernel(int s, const double* __restrict__ G, double* __restrict__ out) {
  if (threadIdx.x < s) out[threadIdx.x] = sqrt(G[threadIdx.x * kMaxS + threadIdx.x]);
}
cudaError_t diag_sqrt(const Launch& L, int s, const double* G, double* out) {
  diag_sqrt_kernel<<<1, 32, 0, L.stream>>>(s, G, out);
  return cudaGetLastError();
}

// Copy a ctrl-layout s x s matrix into block 0 of a stride-s block array and
// zero blocks 1..nblk-1.
__global__ void init_sig_kernel(int s, const double* __restrict__ G, double* __restrict__ sig, int nblk) {
  for (int i = threadIdx.x; i < nblk * s * s; i += blockDim.x)
    sig[i] = (i < s * s) ? G[(i / s) * kMaxS + (i % s)] : 0.0;
}
cudaError_t init_sig(const Launch& L, int s, const double* G, double* sig, int nblk) {
  init_sig_kernel<<<1, 256, 0, L.stream>>>(s, G, sig, nblk);
  return cudaGetLastError();
}

}  // namespace bk
