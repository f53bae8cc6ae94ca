// FP64 row kernels of BCG in the block-parallel *-subalgebra S_BP^p (Def.
// "subalgebras", Ch. 3.1; block CG over it, Ch. 4): every s x s coefficient is
// block diagonal with p x p blocks, so a row's column c only meets the columns
// of its own group [c0, c0 + p), c0 = p floor(c / p).  These kernels loop over
// the group only -- O(s p) FP64 work per row instead of O(s^2) -- and form only
// the groups' Gram entries.  Same scalar row layout as the block-case kernels
// (a sub-warp of SW = next_pow2(s) lanes per row, lane c owns column c); the
// group loop runs to the uniform bound p, so no lane diverges.
#include "bk_common.cuh"
#include "bk_internal.h"
#include "bk_ops.cuh"

namespace bk {

// Gram entries (c0 + j, c), j < p, c0 + j <= c, accumulated per lane in acc[j]
// (j compile-time): CTA sums into part[ut_index(a, c)]; entries outside the
// groups are zero.  scratch holds kWarps * ut_count(s) doubles.
template <int SW>
__device__ void cta_reduce_group(const double (&acc)[SW], int s, int p, double* scratch, double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane & (SW - 1);
  const int cnt = ut_count(s);
  for (int i = threadIdx.x; i < kWarps * cnt; i += blockDim.x) scratch[i] = 0.0;
  __syncthreads();
  // the sub-warps of a warp are summed first (lanes c, c + SW, ...)
  double v[SW];
#pragma unroll
  for (int j = 0; j < SW; ++j) {
    v[j] = acc[j];
#pragma unroll
    for (int off = SW; off < 32; off <<= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
  }
  if (lane < SW && c < s) {
    const int c0 = (c / p) * p;
#pragma unroll
    for (int j = 0; j < SW; ++j) {
      const int a = c0 + j;
      if (j < p && a <= c) scratch[warp * cnt + ut_index(a, c)] = v[j];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += scratch[w * cnt + i];
    part[i] = t;
  }
  __syncthreads();
}

// Q = A P and alpha = P^T Q on the groups' diagonal blocks (upper triangle).
template <int SW, class RowOp>
__global__ void __launch_bounds__(kThreads, 2)
spmm_grp_kernel(RowOp op, int64_t n, int s, int p, const double* __restrict__ P, double* __restrict__ Q,
                Epi<double> ep) {
  if (ep.done && *ep.done) return;
  extern __shared__ double smem[];
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31;
  const int c = lane & (SW - 1), rs = lane / SW;
  const int c0 = (c / p) * p;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  double acc[SW];
#pragma unroll
  for (int j = 0; j < SW; ++j) acc[j] = 0.0;
  for (int64_t base = gw * RPW; base < n; base += nw * RPW) {
    const int64_t r = base + rs;
    const bool ok = (r < n) && (c < s);
    double q = 0.0, l = 0.0;
    if (ok) {
      q = op(r, c, s, P);
      Q[r * s + c] = q;
      l = P[r * s + c];
    }
#pragma unroll
    for (int j = 0; j < SW; ++j) {
      if (j < p) acc[j] = fma(sw_bcast<SW>(l, c0 + j), q, acc[j]);
    }
  }
  const int cnt = ut_count(s);
  double* part = smem;
  double* scratch = smem + ((cnt + 1) & ~1);
  cta_reduce_group<SW>(acc, s, p, scratch, part);
  if (!grid_reduce_last(part, cnt, ep.gpart, ep.counter)) return;
  unpack_gram(part, s, true, ep.gram_out);
}

// X <- X + P lx, R <- R - Q lam over the groups; with kRho also the groups'
// rho_new = R^T R (runs when the iteration does not re-orthonormalise).
template <int SW, bool kRho>
__global__ void __launch_bounds__(kThreads, 2)
update_grp_kernel(int64_t n, int s, int p, const double* __restrict__ P, const double* __restrict__ Q,
                  double* __restrict__ X, double* __restrict__ R, Ctrl* ctrl, double* gpart,
                  int only_if_reortho) {
  if (ctrl->done) return;
  if constexpr (kRho) {
    if (ctrl->reortho_now) return;
  } else {
    if (only_if_reortho && !ctrl->reortho_now) return;
  }
  extern __shared__ double smem[];
  double* lx = smem;                 // s x s, row stride s
  double* lam = lx + s * s;
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    lx[i] = ctrl->lx[(i / s) * kMaxS + (i % s)];
    lam[i] = ctrl->lam[(i / s) * kMaxS + (i % s)];
  }
  __syncthreads();
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31;
  const int c = lane & (SW - 1), rs = lane / SW;
  const int c0 = (c / p) * p;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  double acc[SW];
#pragma unroll
  for (int j = 0; j < SW; ++j) acc[j] = 0.0;
  for (int64_t base = gw * RPW; base < n; base += nw * RPW) {
    const int64_t r = base + rs;
    const bool ok = (r < n) && (c < s);
    const double pv = ok ? P[r * s + c] : 0.0, qv = ok ? Q[r * s + c] : 0.0;
    double dx = 0.0, rq = 0.0;
#pragma unroll
    for (int j = 0; j < SW; ++j) {
      if (j < p) {
        const int a = c0 + j;
        const double pa = sw_bcast<SW>(pv, a), qa = sw_bcast<SW>(qv, a);
        if (c < s) {
          dx = fma(pa, lx[a * s + c], dx);
          rq = fma(qa, lam[a * s + c], rq);
        }
      }
    }
    double rt = 0.0;
    if (ok) {
      X[r * s + c] += dx;
      rt = R[r * s + c] - rq;
      R[r * s + c] = rt;
    }
    if constexpr (kRho) {
#pragma unroll
      for (int j = 0; j < SW; ++j) {
        if (j < p) acc[j] = fma(sw_bcast<SW>(rt, c0 + j), rt, acc[j]);
      }
    }
  }
  if constexpr (kRho) {
    const int cnt = ut_count(s);
    double* part = lam + s * s;
    double* scratch = part + ((cnt + 1) & ~1);
    __syncthreads();
    cta_reduce_group<SW>(acc, s, p, scratch, part);
    if (!grid_reduce_last(part, cnt, gpart, ctrl->counters[kCntB])) return;
    unpack_gram(part, s, true, ctrl->rho_new);
  }
}

// P <- R + P beta over the groups.
template <int SW>
__global__ void __launch_bounds__(kThreads, 2)
pupdate_grp_kernel(int64_t n, int s, int p, const double* __restrict__ R, double* __restrict__ P,
                   Ctrl* ctrl) {
  if (ctrl->done) return;
  extern __shared__ double smem[];
  double* beta = smem;
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) beta[i] = ctrl->beta[(i / s) * kMaxS + (i % s)];
  __syncthreads();
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31;
  const int c = lane & (SW - 1), rs = lane / SW;
  const int c0 = (c / p) * p;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  for (int64_t base = gw * RPW; base < n; base += nw * RPW) {
    const int64_t r = base + rs;
    const bool ok = (r < n) && (c < s);
    const double pv = ok ? P[r * s + c] : 0.0;
    const double zv = ok ? R[r * s + c] : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < SW; ++j) {
      if (j < p) {
        const int a = c0 + j;
        const double pa = sw_bcast<SW>(pv, a);
        if (c < s) acc = fma(pa, beta[a * s + c], acc);
      }
    }
    if (ok) P[r * s + c] = zv + acc;
  }
}

static int grp_grid(const Launch& L, int64_t n, int s) {
  const int rpw = 32 / next_pow2_s(s);
  const int64_t rows_per_cta = (int64_t)rpw * kWarps;
  int64_t need = (n + rows_per_cta - 1) / rows_per_cta;
  const int64_t cap = (int64_t)L.sms * kCtasPerSm;
  if (need > cap) need = cap;
  return (int)(need < 1 ? 1 : need);
}

template <typename K>
static cudaError_t grp_smem(K kern, size_t bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define BK_GRP_SW(s, ...)                              \
  switch (next_pow2_s(s)) {                            \
    case 2: { constexpr int SW = 2; __VA_ARGS__; }     \
    case 4: { constexpr int SW = 4; __VA_ARGS__; }     \
    case 8: { constexpr int SW = 8; __VA_ARGS__; }     \
    case 16: { constexpr int SW = 16; __VA_ARGS__; }   \
    case 32: { constexpr int SW = 32; __VA_ARGS__; }   \
    default: return cudaErrorInvalidValue;             \
  }

template <class RowOp>
static cudaError_t spmm_grp_op(const Launch& L, const RowOp& op, int64_t n, int s, int p, const double* P,
                               double* Q, const Epi<double>& ep) {
  const int cnt = ut_count(s);
  const size_t sm = sizeof(double) * ((size_t)((cnt + 1) & ~1) + (size_t)kWarps * cnt);
  BK_GRP_SW(s, {
    auto k = spmm_grp_kernel<SW, RowOp>;
    cudaError_t e = grp_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<grp_grid(L, n, s), kThreads, sm, L.stream>>>(op, n, s, p, P, Q, ep);
    return cudaGetLastError();
  });
}

cudaError_t spmm_groups(const Launch& L, const OpDesc& A, int s, int p, const double* P, double* Q,
                        const Epi<double>& ep) {
  if (p < 1 || s % p != 0 || !ep.left || !ep.sym) return cudaErrorInvalidValue;
  const int64_t n = A.n;
  switch (A.kind) {
    case kOpCsr: {
      CsrRow<double> op{A.row_ptr, A.col, A.val};
      return spmm_grp_op(L, op, n, s, p, P, Q, ep);
    }
    case kOpConst7: {
      Const7Row<double> op{A.nx, A.ny, A.nz, FastDiv((uint32_t)A.nx), FastDiv((uint32_t)A.ny), A.c7[0],
                           A.c7[1], A.c7[2], A.c7[3], A.c7[4], A.c7[5], A.c7[6]};
      return spmm_grp_op(L, op, n, s, p, P, Q, ep);
    }
    case kOpVar7: {
      Var7Row<double> op{A.nx, A.ny, A.nz, FastDiv((uint32_t)A.nx), FastDiv((uint32_t)A.ny), A.coef,
                         A.coef + n, A.coef + 2 * n, A.coef + 3 * n};
      return spmm_grp_op(L, op, n, s, p, P, Q, ep);
    }
    case kOpEdge5: {
      Edge5Row<double> op{A.nx, A.ny, FastDiv((uint32_t)A.nx), A.coef, A.edges,
                          A.edges + (int64_t)A.ny * (A.nx + 1)};
      return spmm_grp_op(L, op, n, s, p, P, Q, ep);
    }
    case kOpDiag: {
      DiagRow<double> op{A.coef};
      return spmm_grp_op(L, op, n, s, p, P, Q, ep);
    }
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t bcg_update_groups(const Launch& L, int64_t n, int s, int p, const double* P, const double* Q,
                              double* X, double* R, Ctrl* ctrl, double* gpart, int rho_mode) {
  if (p < 1 || s % p != 0) return cudaErrorInvalidValue;
  const int cnt = ut_count(s);
  const size_t sm_lean = sizeof(double) * 2 * s * s;
  const size_t sm_rho = sm_lean + sizeof(double) * ((size_t)((cnt + 1) & ~1) + (size_t)kWarps * cnt);
  const int grid = grp_grid(L, n, s);
  BK_GRP_SW(s, {
    auto kl = update_grp_kernel<SW, false>;
    cudaError_t e = grp_smem(kl, sm_lean);
    if (e != cudaSuccess) return e;
    kl<<<grid, kThreads, sm_lean, L.stream>>>(n, s, p, P, Q, X, R, ctrl, gpart, rho_mode);
    if ((e = cudaGetLastError()) != cudaSuccess || rho_mode == 0) return e;
    auto kh = update_grp_kernel<SW, true>;
    if ((e = grp_smem(kh, sm_rho)) != cudaSuccess) return e;
    kh<<<grid, kThreads, sm_rho, L.stream>>>(n, s, p, P, Q, X, R, ctrl, gpart, rho_mode);
    return cudaGetLastError();
  });
}

cudaError_t bcg_pupdate_groups(const Launch& L, int64_t n, int s, int p, const double* R, double* P,
                               Ctrl* ctrl) {
  if (p < 1 || s % p != 0) return cudaErrorInvalidValue;
  const size_t sm = sizeof(double) * s * s;
  BK_GRP_SW(s, {
    auto k = pupdate_grp_kernel<SW>;
    cudaError_t e = grp_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<grp_grid(L, n, s), kThreads, sm, L.stream>>>(n, s, p, R, P, ctrl);
    return cudaGetLastError();
  });
}

}  // namespace bk
