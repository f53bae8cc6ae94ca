// The s x s part of every iteration, on one CTA in FP64 (s <= 32):
// Cholesky / LU solves for the block coefficients lambda and beta, the
// diagonally scaled condition number kappa_D of the adaptive
// re-orthonormalisation test, the residual-transformation sigma, per-column
// residual norms, the stopping test and the block Givens step of block GMRes.
// All matrices live in shared memory with row stride 32 (kMaxS).
#include <math.h>

#include <type_traits>

#include "bk_common.cuh"
#include "bk_hh.cuh"
#include "bk_internal.h"

namespace bk {

constexpr int kST = 256;   // threads of the small-solve CTA
constexpr double kCholQrMinSine2 = 1e-10;   // CholeskyQR2 decline threshold (squared sine)
#define IDX(i, j) ((i) * kMaxS + (j))

__device__ void sm_copy(double* dst, const double* src, int s) {
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, c = i % s;
    dst[IDX(a, c)] = src[IDX(a, c)];
  }
}

__device__ void sm_identity(double* dst, int s) {
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, c = i % s;
    dst[IDX(a, c)] = (a == c) ? 1.0 : 0.0;
  }
}

// C = op(A) B with op(A) = A or A^T (C must not alias A or B).
// A thread forms up to four entries at once (independent FMA chains).
__device__ void sm_matmul(double* C, const double* A, bool transA, const double* B, int s) {
  const int n = s * s, nt = blockDim.x;
  for (int i0 = threadIdx.x; i0 < n; i0 += 4 * nt) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int a[4], c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * nt;
      a[u] = i < n ? i / s : 0;
      c[u] = i < n ? i % s : 0;
    }
    const int per = (n - i0 + nt - 1) / nt;          // this thread's entries (<= 4), no idle FMAs
    if (per >= 4) {
      for (int k = 0; k < s; ++k) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          acc[u] = fma(transA ? A[IDX(k, a[u])] : A[IDX(a[u], k)], B[IDX(k, c[u])], acc[u]);
      }
    } else {
      for (int u = 0; u < per; ++u)
        for (int k = 0; k < s; ++k)
          acc[u] = fma(transA ? A[IDX(k, a[u])] : A[IDX(a[u], k)], B[IDX(k, c[u])], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u * nt < n) C[IDX(a[u], c[u])] = acc[u];
  }
}

__device__ bool sm_all_finite(const double* A, int s, int* flag) {
  if (threadIdx.x == 0) *flag = 1;
  __syncthreads();
  for (int i = threadIdx.x; i < s * s; i += blockDim.x)
    if (!isfinite(A[IDX(i / s, i % s)])) *flag = 0;
  __syncthreads();
  const bool ok = *flag != 0;
  __syncthreads();
  return ok;
}

// In-place Cholesky A = L L^T (lower triangle of A overwritten by L).
// Fails (returns false) on a non-positive or non-finite pivot, which is the
// LAPACK potrf criterion.  Every thread forms the pivot's square root itself
// (no barrier between the pivot and the column scaling).
__device__ bool sm_cholesky(double* A, int s, int* flag) {
  if (threadIdx.x == 0) *flag = 1;
  __syncthreads();
  for (int k = 0; k < s; ++k) {
    const double d = A[IDX(k, k)];
    if (!(d > 0.0) || !isfinite(d)) return false;      // uniform: every thread read the same pivot
    const double lkk = sqrt(d);
    for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) A[IDX(i, k)] /= lkk;
    __syncthreads();
    if (threadIdx.x == 0) A[IDX(k, k)] = lkk;
    const int r = s - k - 1;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int i = k + 1 + e / r, j = k + 1 + e % r;
      if (j <= i) A[IDX(i, j)] = fma(-A[IDX(i, k)], A[IDX(j, k)], A[IDX(i, j)]);
    }
    __syncthreads();
  }
  return true;
}

// In-place Cholesky A = L L^T with a relative pivot floor: fails unless every pivot
// d_k (the Schur complement's diagonal entry, d_k = L_kk^2) keeps d_k > floor G_kk
// with G the matrix on entry (G_kk > 0).  d_k / G_kk is the squared sine between
// column k of a block whose Gram is G and the span of the columns before it, so a
// floor rejects nearly dependent blocks.  gd: kMaxS doubles of scratch.
__device__ bool sm_cholesky_floor(double* A, int s, double floor, double* gd, int* flag) {
  for (int i = threadIdx.x; i < s; i += blockDim.x) gd[i] = A[IDX(i, i)];
  if (threadIdx.x == 0) *flag = 1;
  __syncthreads();
  for (int k = 0; k < s; ++k) {
    const double d = A[IDX(k, k)], g = gd[k];
    if (!(g > 0.0) || !(d > floor * g) || !isfinite(d)) return false;   // uniform
    const double lkk = sqrt(d);
    for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) A[IDX(i, k)] /= lkk;
    __syncthreads();
    if (threadIdx.x == 0) A[IDX(k, k)] = lkk;
    const int r = s - k - 1;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int i = k + 1 + e / r, j = k + 1 + e % r;
      if (j <= i) A[IDX(i, j)] = fma(-A[IDX(i, k)], A[IDX(j, k)], A[IDX(i, j)]);
    }
    __syncthreads();
  }
  return true;
}

// U = L^T and Uinv = L^{-T} (both upper triangular, zeros below the diagonal) from the
// lower factor L of sm_cholesky (its strict upper triangle is ignored).  One warp per
// column c of L^{-1}: forward substitution L z = e_c with lane i holding z_i.
__device__ void sm_upper_and_inverse(const double* L, double* U, double* Uinv, int s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double dinv = (lane < s) ? 1.0 / L[IDX(lane, lane)] : 0.0;
  for (int c = warp; c < s; c += nw) {
    double v = (lane == c) ? 1.0 : 0.0;
    for (int i = c; i < s; ++i) {
      const double zi = __shfl_sync(0xffffffffu, v * dinv, i);
      if (lane > i && lane < s) v = fma(-L[IDX(lane, i)], zi, v);
      if (lane == i) v = zi;
    }
    if (lane < s) {
      Uinv[IDX(c, lane)] = v;                           // (L^{-1})_{lane c}, zero for lane < c
      U[IDX(c, lane)] = (lane >= c) ? L[IDX(lane, c)] : 0.0;
    }
  }
  __syncthreads();
}

// X = (L L^T)^{-1} B (X may alias B).  One warp per right-hand-side column,
// lane i holding row i; column-oriented substitution: once x_i is final it is
// broadcast by a shuffle and every later row subtracts its term, so the
// dependent chain per column is 2 s steps (the terms are subtracted in the
// same order k = 0, 1, ... as a row-oriented sweep).
__device__ void sm_chol_solve(const double* L, const double* B, double* X, int s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double dinv = (lane < s) ? 1.0 / L[IDX(lane, lane)] : 0.0;
  for (int c = warp; c < s; c += nw) {
    double v = (lane < s) ? B[IDX(lane, c)] : 0.0;
    for (int i = 0; i < s; ++i) {                      // forward: L y = b
      const double yi = __shfl_sync(0xffffffffu, v * dinv, i);
      if (lane > i && lane < s) v = fma(-L[IDX(lane, i)], yi, v);
      if (lane == i) v = yi;
    }
    for (int i = s - 1; i >= 0; --i) {                 // backward: L^T x = y
      const double xi = __shfl_sync(0xffffffffu, v * dinv, i);
      if (lane < i) v = fma(-L[IDX(i, lane)], xi, v);
      if (lane == i) v = xi;
    }
    if (lane < s) X[IDX(lane, c)] = v;
  }
  __syncthreads();
}

// In-place LU with partial pivoting (row interchanges recorded in piv).
// Fails on an exactly zero or non-finite pivot.
__device__ bool sm_lu(double* A, int* piv, int s, int* flag) {
  __shared__ int s_p;
  if (threadIdx.x == 0) *flag = 1;
  __syncthreads();
  for (int k = 0; k < s; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(A[IDX(k, k)]);
      for (int i = k + 1; i < s; ++i) {
        const double v = fabs(A[IDX(i, k)]);
        if (v > best) { best = v; p = i; }
      }
      piv[k] = p;
      s_p = p;
      if (!(best > 0.0) || !isfinite(best)) *flag = 0;
    }
    __syncthreads();
    if (!*flag) return false;
    const int p = s_p;
    if (p != k)
      for (int j = threadIdx.x; j < s; j += blockDim.x) {
        const double t = A[IDX(k, j)]; A[IDX(k, j)] = A[IDX(p, j)]; A[IDX(p, j)] = t;
      }
    __syncthreads();
    const double pk = A[IDX(k, k)];
    for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) A[IDX(i, k)] /= pk;
    __syncthreads();
    const int r = s - k - 1;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int i = k + 1 + e / r, j = k + 1 + e % r;
      A[IDX(i, j)] = fma(-A[IDX(i, k)], A[IDX(k, j)], A[IDX(i, j)]);
    }
    __syncthreads();
  }
  return true;
}

// X = A^{-1} B from the LU factors (X may alias B), one thread per column.
__device__ void sm_lu_solve(const double* LU, const int* piv, const double* B, double* X, int s) {
  const int c = threadIdx.x;
  if (c < s) {
    if (X != B) for (int i = 0; i < s; ++i) X[IDX(i, c)] = B[IDX(i, c)];
    for (int k = 0; k < s; ++k) {
      const int p = piv[k];
      if (p != k) { const double t = X[IDX(k, c)]; X[IDX(k, c)] = X[IDX(p, c)]; X[IDX(p, c)] = t; }
    }
    for (int i = 0; i < s; ++i) {
      double v = X[IDX(i, c)];
      for (int k = 0; k < i; ++k) v = fma(-LU[IDX(i, k)], X[IDX(k, c)], v);
      X[IDX(i, c)] = v;
    }
    for (int i = s - 1; i >= 0; --i) {
      double v = X[IDX(i, c)];
      for (int k = i + 1; k < s; ++k) v = fma(-LU[IDX(i, k)], X[IDX(k, c)], v);
      X[IDX(i, c)] = v / LU[IDX(i, i)];
    }
  }
  __syncthreads();
}

// Bit-level constants of the two precisions the eigenvalue bracketing runs in.
template <typename R> struct KBits;
template <> struct KBits<double> {
  using I = long long;
  static constexpr int kMant = 52, kExpMask = 0x7ff, kBias = 1023, kShift = 400;
  static __device__ __forceinline__ I bits(double v) { return __double_as_longlong(v); }
  static __device__ __forceinline__ double tiny() { return 0x1p-600; }
  static __device__ __forceinline__ double up() { return 0x1p400; }
  static __device__ __forceinline__ double down() { return 0x1p-400; }
  static __device__ __forceinline__ double stop() { return 0x1p-49; }   // 8 eps
};
template <> struct KBits<float> {
  using I = int;
  static constexpr int kMant = 23, kExpMask = 0xff, kBias = 127, kShift = 60;
  static __device__ __forceinline__ I bits(float v) { return __float_as_int(v); }
  static __device__ __forceinline__ float tiny() { return 0x1p-100f; }
  static __device__ __forceinline__ float up() { return 0x1p60f; }
  static __device__ __forceinline__ float down() { return 0x1p-60f; }
  static __device__ __forceinline__ float stop() { return 0x1p-20f; }   // 8 eps
};

// Number of eigenvalues of the symmetric tridiagonal T = tridiag(e, d, e)
// below x: the sign changes of the Sturm sequence of T - x I's leading
// principal minors p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (Wilkinson,
// "The Algebraic Eigenvalue Problem", 1965, Ch. 5).  No division: the two
// latest terms are rescaled together when they leave [2^-K, 2^K] (K = 400 in
// double, 60 in float), which keeps their signs and ratio; an exact zero takes
// the sign opposite to its predecessor (x moved off the root of that minor).
// Signs, zeros and exponents are read from the bit pattern (integer ALU): the
// floating-point pipe only carries the recurrence itself.
template <typename R>
__device__ int sturm_count(const R* d, const R* e2, int s, R x) {
  using B = KBits<R>;
  using I = typename B::I;
  constexpr int kSignShift = 8 * (int)sizeof(R) - 1;
  int cnt = 0;
  I sprev = 0;                          // sign bit of the previous term (1: negative)
  R pm1 = R(1), p = d[0] - x;
  for (int i = 0;; ++i) {
    I b = B::bits(p);
    if (((typename std::make_unsigned<I>::type)b << 1) == 0) {   // +-0: the sign opposite to the predecessor
      p = sprev ? B::tiny() : -B::tiny();
      b = B::bits(p);
    }
    const I sg = (I)((typename std::make_unsigned<I>::type)b >> kSignShift);
    cnt += (int)(sg != sprev);
    sprev = sg;
    const int ex = (int)((b >> B::kMant) & B::kExpMask);
    if (ex > B::kBias + B::kShift) { p *= B::down(); pm1 *= B::down(); }
    else if (ex < B::kBias - B::kShift) { p *= B::up(); pm1 *= B::up(); }
    if (i + 1 >= s) break;
    const R pn = fma(d[i + 1] - x, p, -e2[i] * pm1);
    pm1 = p;
    p = pn;
  }
  return cnt;
}

template <typename R>
__device__ inline R warp_sum(R v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// kappa_D(A) = kappa_2(D^-1/2 A D^-1/2), D = diag(A)  (Def. in Ch. 4.3): the
// ratio of the extreme eigenvalues of the scaled matrix M.  M is reduced to a
// symmetric tridiagonal T = Q^T M Q by s - 2 Householder reflections (Golub &
// Van Loan, "Matrix Computations", Alg. 8.3.1: p = tau M' v, w = p -
// (tau p^T v / 2) v, M' -= v w^T + w v^T, with the two products of each entry
// added in an order that keeps M' exactly symmetric), and T's smallest and
// largest eigenvalues are bracketed from its Gershgorin interval by
// multisection on Sturm counts (64 points per round: the bracket shrinks by 65
// per round, until it is within 8 eps ||T||, the accuracy to which the
// eigenvalues of M are determined at all, or after 12 rounds).
// +inf when a diagonal entry of A or the smallest
// eigenvalue is <= 0.  M and M2 are shared work matrices.
template <typename R>
__device__ double sm_kappa_d_t(const double* A, int s, R* M, R* M2, int* flag, double* lo_hi = nullptr) {
  __shared__ R s_tau, s_lo[2], s_hi[2];
  if (threadIdx.x == 0) *flag = 1;
  __syncthreads();
  for (int i = threadIdx.x; i < s; i += blockDim.x)
    if (!(A[IDX(i, i)] > 0.0)) *flag = 0;
  __syncthreads();
  if (!*flag) return INFINITY;
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, c = i % s;
    M[IDX(a, c)] = (R)(A[IDX(a, c)] / sqrt(A[IDX(a, a)] * A[IDX(c, c)]));
  }
  __syncthreads();
  if (s == 1) {
    if (lo_hi && threadIdx.x == 0) { lo_hi[0] = 1.0; lo_hi[1] = 1.0; }
    __syncthreads();
    return 1.0;
  }
  R* v = M2;                 // Householder vector (entries k+1 .. s-1 at 0 .. m-1)
  R* w = M2 + 32;            // w = p - K v
  R* dd = M2 + 64;           // diagonal of T
  R* e2 = M2 + 96;           // squared off-diagonal of T
  R* ee = M2 + 128;          // off-diagonal of T
  R* part = M2 + 160;        // 8 warps x 32 partial sums of M' v
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  for (int k = 0; k + 2 < s; ++k) {
    const int m = s - k - 1;
    if (warp == 0) {
      const R x = lane < m ? M[IDX(k + 1 + lane, k)] : R(0);
      const R x0 = __shfl_sync(0xffffffffu, x, 0);
      const R tail = warp_sum<R>(lane > 0 ? x * x : R(0));
      R tau = R(0), alpha = x0;
      if (tail > R(0)) {
        const R sig = sqrt(fma(x0, x0, tail));
        alpha = x0 >= R(0) ? -sig : sig;
        const R v0 = x0 - alpha;
        tau = R(2) / fma(v0, v0, tail);
        if (lane < m) v[lane] = lane == 0 ? v0 : x;
      }
      if (lane == 0) { dd[k] = M[IDX(k, k)]; ee[k] = alpha; s_tau = tau; }
    }
    __syncthreads();
    const R tau = s_tau;
    if (tau == R(0)) {                        // column already reduced
      __syncthreads();                        // every thread has read s_tau
      continue;
    }
    R acc = R(0);
    if (lane < m)
      for (int i = warp; i < m; i += nw) acc = fma(M[IDX(k + 1 + i, k + 1 + lane)], v[i], acc);
    part[warp * 32 + lane] = acc;
    __syncthreads();
    if (warp == 0) {
      R pj = R(0);
      for (int q = 0; q < nw; ++q) pj += part[q * 32 + lane];
      pj = lane < m ? tau * pj : R(0);
      const R vj = lane < m ? v[lane] : R(0);
      const R K = R(0.5) * tau * warp_sum<R>(pj * vj);
      if (lane < m) w[lane] = fma(-K, vj, pj);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e / m, j = e % m;
      R u;
      if constexpr (sizeof(R) == 8) u = __dadd_rn(__dmul_rn(v[i], w[j]), __dmul_rn(w[i], v[j]));
      else u = __fadd_rn(__fmul_rn(v[i], w[j]), __fmul_rn(w[i], v[j]));
      M[IDX(k + 1 + i, k + 1 + j)] -= u;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    dd[s - 2] = M[IDX(s - 2, s - 2)];
    ee[s - 2] = M[IDX(s - 1, s - 2)];
    dd[s - 1] = M[IDX(s - 1, s - 1)];
  }
  __syncthreads();
  // Gershgorin interval of T (warp 0), then multisection: threads 0..63 bracket
  // the smallest eigenvalue (first point with count >= 1), 64..127 the largest
  // (first point with count >= s).
  if (warp == 0) {
    R lo = R(INFINITY), hi = R(-INFINITY);
    if (lane < s) {
      const R r = (lane > 0 ? fabs(ee[lane - 1]) : R(0)) + (lane < s - 1 ? fabs(ee[lane]) : R(0));
      lo = dd[lane] - r;
      hi = dd[lane] + r;
      if (lane < s - 1) e2[lane] = ee[lane] * ee[lane];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, off));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if (lane < 2) { s_lo[lane] = lo; s_hi[lane] = hi; }
  }
  __syncthreads();
  __shared__ int s_first[4];
  // stop when both brackets are within 8 eps ||T|| (the accuracy to which
  // the eigenvalues of M are determined at all), after 12 rounds at most
  const R gnorm = fmax(fabs(s_lo[0]), fabs(s_hi[0]));
  for (int round = 0; round < 12; ++round) {
    bool done = true;              // uniform: every thread reads the same brackets
    for (int q = 0; q < 2; ++q) done = done && (s_hi[q] - s_lo[q] <= KBits<R>::stop() * gnorm);
    if (done) break;
    const int g = (threadIdx.x >> 6) & 1, t = threadIdx.x & 63;
    const R lo = s_lo[g], hi = s_hi[g];
    const R step = (hi - lo) / R(65);
    bool in = false;
    if (threadIdx.x < 128) in = sturm_count<R>(dd, e2, s, lo + step * R(t + 1)) >= (g == 0 ? 1 : s);
    // first point (per group of two warps) at or above the eigenvalue; 64: none
    const unsigned bal = __ballot_sync(0xffffffffu, in);
    if (threadIdx.x < 128 && lane == 0) s_first[warp] = bal ? (warp & 1) * 32 + __ffs(bal) - 1 : 64;
    __syncthreads();
    if (threadIdx.x < 128 && t == 0) {
      const int f = min(s_first[2 * g], s_first[2 * g + 1]);
      // the eigenvalue lies in (x_{f-1}, x_f], x_{-1} = lo, x_64 = hi
      s_lo[g] = f == 0 ? lo : lo + step * R(f);
      s_hi[g] = f == 64 ? hi : lo + step * R(f + 1);
    }
    __syncthreads();
  }
  const double lmin = 0.5 * ((double)s_lo[0] + (double)s_hi[0]);
  const double lmax = 0.5 * ((double)s_lo[1] + (double)s_hi[1]);
  if (lo_hi && threadIdx.x == 0) { lo_hi[0] = lmin; lo_hi[1] = lmax; }
  __syncthreads();
  return (lmin > 0.0 && s_hi[0] > R(0)) ? lmax / lmin : INFINITY;
}

__device__ double sm_kappa_d(const double* A, int s, double* M, double* M2, int* flag) {
  return sm_kappa_d_t<double>(A, s, M, M2, flag);
}

// max that propagates NaN (fmax would drop it)
__device__ inline double nanmax(double a, double b) { return (isnan(b) || b > a) ? b : a; }

__device__ inline void stop(Ctrl* c, int status) {
  if (threadIdx.x == 0) { c->done = kDoneStopped; c->status = status; }
}

// re-orthonormalisation decision (Eq. "reortho_criterion", read as
// eta * kappa_D > 1/sqrt(eps); eta = 0 never, eta = inf always)
__device__ int criterion(double eta, double eps, int s, const double* A, double* M, double* M2, int* flag) {
  if (eta == 0.0) return 0;
  if (isinf(eta)) return 1;
  const double thr = 1.0 / sqrt(eps);
  // first in FP32: where kappa_D < 2^10 the FP32 eigenvalues fix it to ~0.1 %
  // (absolute error ~ s eps_32 ||M||), so a decision more than 1 % off the
  // threshold is the FP64 one; otherwise (and for every larger kappa_D) FP64
  __shared__ double lh[2];
  const double k32 = sm_kappa_d_t<float>(A, s, reinterpret_cast<float*>(M), reinterpret_cast<float*>(M2),
                                         flag, lh);
  if (lh[0] > 0.0 && lh[0] > lh[1] * 0x1p-10 && isfinite(k32)) {
    const double x = eta * k32;
    if (x < 0.99 * thr) return 0;
    if (x > 1.01 * thr) return 1;
  }
  const double kap = sm_kappa_d(A, s, M, M2, flag);
  return (eta * kap > thr) ? 1 : 0;
}

__device__ int decide(Ctrl* c, const uint8_t* forced, const double* A, double* M, double* M2, int* flag) {
  const int k = c->iter;
  if (forced && k < c->n_forced) return forced[k] ? 1 : 0;
  return criterion(c->eta, c->eps, c->s, A, M, M2, flag);
}

// Orthogonal projection onto S_BP^p (Def. "subalgebras", Ch. 3.1): entries
// outside the p x p diagonal blocks become zero (p = s: nothing changes).
__device__ inline void sm_project(double* M, int s, int p) {
  if (p >= s) return;
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, b = i % s;
    if (a / p != b / p) M[IDX(a, b)] = 0.0;
  }
}

struct SmallSmem {
  double A[kMM], B[kMM], C[kMM], D[kMM], E[kMM], F[kMM];
  double red[kST];
  double w[kMaxS], tau[kMaxS];
  int flag;
};

// Stopping measure of the current relres[] (reading c2): the largest column ratio, or
// for norm_mode 1 the Frobenius ratio ||R||_F / ||R0||_F = sqrt(sum_i (relres_i n0_i)^2 /
// sum_i n0_i^2).  NaN in any column propagates.
__device__ inline double stop_measure(const Ctrl* c, int s) {
  if (c->norm_mode != 1) {
    double mx = 0.0;
    for (int i = 0; i < s; ++i) mx = nanmax(mx, c->relres[i]);
    return mx;
  }
  double num = 0.0, den = 0.0;
  for (int i = 0; i < s; ++i) {
    const double r = c->relres[i] * c->n0[i];
    num = fma(r, r, num);
    den = fma(c->n0[i], c->n0[i], den);
  }
  return den > 0.0 ? sqrt(num / den) : (isnan(num) ? num : 0.0);
}

// ---------------------------------------------------------------- BCG ----
// Initial test: relres_i = sqrt((sigma^T rho sigma)_ii) / ||R0_i||.
__global__ void __launch_bounds__(kST) small_bcg_init_k(Ctrl* c) {
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  const int s = c->s;
  sm_copy(S.A, c->rho, s);
  sm_copy(S.B, c->sigma, s);
  __syncthreads();
  sm_project(S.A, s, c->sub_p);
  __syncthreads();
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) c->rho[IDX(i / s, i % s)] = S.A[IDX(i / s, i % s)];
  sm_matmul(S.C, S.A, false, S.B, s);     // rho sigma
  __syncthreads();
  if (threadIdx.x < s) {
    const int i = threadIdx.x;
    double v = 0.0;
    for (int k = 0; k < s; ++k) v = fma(S.B[IDX(k, i)], S.C[IDX(k, i)], v);
    const double n0 = c->n0[i];
    c->relres[i] = !isfinite(n0) ? NAN : (n0 > 0.0 ? sqrt(fmax(v, 0.0)) / n0 : 0.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double mx = stop_measure(c, s);
    if (!isfinite(mx)) { c->done = kDoneStopped; c->status = BK_NONFINITE; }
    else if (mx <= c->tol) { c->done = kDoneConverged; c->status = BK_OK; }
    else if (c->maxit <= 0) { c->done = kDoneStopped; c->status = BK_NOT_CONVERGED; }
  }
  if (c->has_prec) {
    // preconditioned: rho^0 = <P^0, R-bar^0> (the Euclidean Gram above only gave the norms)
    __syncthreads();
    sm_copy(S.A, c->rho_m, s);
    __syncthreads();
    sm_project(S.A, s, c->sub_p);
    __syncthreads();
    for (int i = threadIdx.x; i < s * s; i += blockDim.x) c->rho[IDX(i / s, i % s)] = S.A[IDX(i / s, i % s)];
  }
}

// lambda = alpha^{-1} rho, the re-orthonormalisation decision, lx = lambda sigma.
__global__ void __launch_bounds__(kST) small_bcg_1_k(Ctrl* c, const uint8_t* forced) {
  if (c->done) return;
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  const int s = c->s;
  sm_copy(S.A, c->alpha, s);
  sm_copy(S.B, c->rho, s);
  sm_copy(S.E, c->sigma, s);
  __syncthreads();
  sm_project(S.A, s, c->sub_p);            // S_BP^p: alpha block diagonal
  __syncthreads();
  if (!sm_all_finite(S.A, s, &S.flag)) { stop(c, BK_NONFINITE); return; }
  sm_copy(S.C, S.A, s);
  __syncthreads();
  if (!sm_cholesky(S.C, s, &S.flag)) { stop(c, BK_BREAKDOWN); return; }
  sm_chol_solve(S.C, S.B, S.D, s);            // D = lambda
  const int reo = decide(c, forced, S.A, S.B, S.C, &S.flag);   // clobbers B, C
  __syncthreads();
  sm_matmul(S.B, S.D, false, S.E, s);          // lx = lambda sigma
  __syncthreads();
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, b = i % s;
    c->lam[IDX(a, b)] = S.D[IDX(a, b)];
    c->lx[IDX(a, b)] = S.B[IDX(a, b)];
  }
  if (threadIdx.x == 0) c->reortho_now = reo;
}

// sigma update, residual norms, stopping test, beta = rho^{-1} gamma^T rho_new.
__global__ void __launch_bounds__(kST) small_bcg_2_k(Ctrl* c, double* history, uint8_t* decisions) {
  if (c->done) return;
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  const int s = c->s;
  const int reo = c->reortho_now;
  const int k = c->iter;
  const int pre = c->has_prec;
  // A: the Euclidean Gram for the norms (not needed after a re-orthonormalisation
  // when preconditioned; then rho_new was not formed and A takes rho_m at once)
  sm_copy(S.A, (pre && reo) ? c->rho_m : c->rho_new, s);
  sm_copy(S.B, c->sigma, s);
  if (reo) sm_copy(S.C, c->gamma, s); else sm_identity(S.C, s);
  __syncthreads();
  if (reo && c->qr_fast == 2) {
    // CholeskyQR2 whose second factor failed: the TSQR factored Y1 = R-tilde U1^{-1},
    // so R-tilde = Y gamma' U1 and gamma = gamma' U1
    sm_copy(S.E, c->cq_u1, s);
    __syncthreads();
    sm_matmul(S.F, S.C, false, S.E, s);
    __syncthreads();
    sm_copy(S.C, S.F, s);
    for (int i = threadIdx.x; i < s * s; i += blockDim.x) c->gamma[IDX(i / s, i % s)] = S.F[IDX(i / s, i % s)];
    __syncthreads();
  }
  sm_project(S.A, s, c->sub_p);            // S_BP^p: rho block diagonal
  __syncthreads();
  if (!sm_all_finite(S.A, s, &S.flag)) { stop(c, BK_NONFINITE); return; }
  sm_matmul(S.D, S.C, false, S.B, s);          // sigma_new = gamma sigma
  __syncthreads();
  if (!reo) {
    sm_matmul(S.F, S.A, false, S.D, s);        // rho sigma_new
    __syncthreads();
  }
  {
    // column norms ||R-bar sigma e_i||^2 = (sigma^T rho sigma)_ii (sigma_i^T sigma_i after a
    // re-orthonormalisation): one warp per column, a shuffle sum over the rows
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = threadIdx.x >> 5; i < s; i += nw) {
      double v = 0.0;
      if (lane < s) v = S.D[IDX(lane, i)] * (reo ? S.D[IDX(lane, i)] : S.F[IDX(lane, i)]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) {
        const double n0 = c->n0[i];
        c->relres[i] = (!isfinite(n0) || isnan(v)) ? NAN : (n0 > 0.0 ? sqrt(fmax(v, 0.0)) / n0 : 0.0);
      }
    }
  }
  __syncthreads();
  __shared__ int s_conv;
  if (threadIdx.x == 0) {
    const double mx = stop_measure(c, s);
    if (history) history[k] = mx;
    if (decisions) decisions[k] = (uint8_t)reo;
    c->iter = k + 1;
    c->reorths += reo;
    c->cholqr_count += (reo && c->qr_fast == 1) ? 1 : 0;
    s_conv = !isfinite(mx) ? -1 : (mx <= c->tol ? 1 : 0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) c->sigma[IDX(i / s, i % s)] = S.D[IDX(i / s, i % s)];
  if (s_conv < 0) { stop(c, BK_NONFINITE); return; }
  if (s_conv > 0) {
    if (threadIdx.x == 0) { c->done = kDoneConverged; c->status = BK_OK; }
    return;
  }
  if (pre && !reo) {
    // the new rho = <Z, R-bar> replaces the Euclidean Gram used for the norms
    sm_copy(S.A, c->rho_m, s);
    __syncthreads();
    sm_project(S.A, s, c->sub_p);
    __syncthreads();
    if (!sm_all_finite(S.A, s, &S.flag)) { stop(c, BK_NONFINITE); return; }
  }
  // beta = rho_old^{-1} gamma^T rho_new
  sm_matmul(S.E, S.C, true, S.A, s);
  sm_copy(S.D, c->rho, s);
  __syncthreads();
  if (!sm_cholesky(S.D, s, &S.flag)) { stop(c, BK_BREAKDOWN); return; }
  sm_chol_solve(S.D, S.E, S.E, s);
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, b = i % s;
    c->beta[IDX(a, b)] = S.E[IDX(a, b)];
    c->rho[IDX(a, b)] = S.A[IDX(a, b)];
  }
  if (c->one_r) {
    // Alg. "1R-CG": alpha^{k+1} = delta^{k+1} - beta^T alpha^k beta (upper triangle, mirrored)
    sm_copy(S.B, c->alpha, s);
    __syncthreads();
    sm_matmul(S.F, S.B, false, S.E, s);        // alpha beta
    __syncthreads();
    sm_matmul(S.C, S.E, true, S.F, s);         // beta^T alpha beta
    __syncthreads();
    for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
      const int a = i / s, b = i % s;
      const int u = a < b ? a : b, v = a < b ? b : a;
      const double al = c->delta[IDX(u, v)] - S.C[IDX(u, v)];
      c->alpha[IDX(a, b)] = al;
      S.D[IDX(a, b)] = al;
    }
    if (c->replace_every > 0) {
      // replacement after every m-th iteration and whenever the recursive alpha has a
      // non-positive Cholesky pivot (the next lambda needs its Cholesky factor)
      __syncthreads();
      const bool due = (k + 1) % c->replace_every == 0;
      const bool ok = due || sm_cholesky(S.D, s, &S.flag);
      __syncthreads();
      if (threadIdx.x == 0) {
        c->replace_now = ok && !due ? 0 : 1;
        c->replacements += c->replace_now;
      }
    }
  }
  if (threadIdx.x == 0 && c->iter >= c->maxit) { c->done = kDoneStopped; c->status = BK_NOT_CONVERGED; }
}

// CholeskyQR2 normaliser of the re-orthonormalising iterations (Fukaya, Nakatsukasa,
// Yanagisawa, Yamamoto 2014), the s x s steps; the row passes Y <- Y U^{-1} with the
// Gram Y^T Y fused run between them.
// Pass 1: G1 = rho_new = R-tilde^T R-tilde from the update kernel.  G1 = U1^T U1 is taken
// only when every pivot keeps U1_kk^2 > 1e-10 G1_kk (every column's squared sine to
// the span of the columns before it); otherwise the Householder TSQR normalises.
__global__ void __launch_bounds__(kST) small_cholqr_1_k(Ctrl* c) {
  if (c->done) return;
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  const int s = c->s;
  if (!c->reortho_now) {
    if (threadIdx.x == 0) { c->qr_fast = 0; c->tsqr_now = 0; }
    return;
  }
  sm_copy(S.A, c->rho_new, s);
  __syncthreads();
  const bool ok = sm_all_finite(S.A, s, &S.flag) && sm_cholesky_floor(S.A, s, kCholQrMinSine2, S.w, &S.flag);
  __syncthreads();
  if (!ok) {
    if (threadIdx.x == 0) { c->qr_fast = 0; c->tsqr_now = 1; }
    return;
  }
  sm_upper_and_inverse(S.A, S.B, S.C, s);
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, b = i % s;
    c->cq_u1[IDX(a, b)] = S.B[IDX(a, b)];
    c->cq_inv[IDX(a, b)] = S.C[IDX(a, b)];
  }
  if (threadIdx.x == 0) { c->qr_fast = 1; c->tsqr_now = 0; }
}

// Pass 2: G2 = Y1^T Y1 (close to I) = U2^T U2 with every pivot above G2_kk / 2, then
// gamma = U2 U1 and the inverse U2^{-1} for the second row pass, and rho_new = I: the
// normalised block R-bar = Y1 U2^{-1} has orthonormal columns (Def. "normalizer"), so
// its Gram is not formed.  A failure leaves Y1 to the TSQR (qr_fast = 2; the small BCG
// kernel multiplies its factor by U1).
__global__ void __launch_bounds__(kST) small_cholqr_2_k(Ctrl* c) {
  if (c->done || c->qr_fast != 1) return;
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  const int s = c->s;
  sm_copy(S.A, c->rho_new, s);
  sm_copy(S.D, c->cq_u1, s);
  __syncthreads();
  const bool ok = sm_all_finite(S.A, s, &S.flag) && sm_cholesky_floor(S.A, s, 0.5, S.w, &S.flag);
  __syncthreads();
  if (!ok) {
    if (threadIdx.x == 0) { c->qr_fast = 2; c->tsqr_now = 1; }
    return;
  }
  sm_upper_and_inverse(S.A, S.B, S.C, s);
  sm_matmul(S.E, S.B, false, S.D, s);          // gamma = U2 U1
  __syncthreads();
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, b = i % s;
    c->gamma[IDX(a, b)] = S.E[IDX(a, b)];
    c->cq_inv[IDX(a, b)] = S.C[IDX(a, b)];
    c->rho_new[IDX(a, b)] = (a == b) ? 1.0 : 0.0;
  }
}

cudaError_t small_cholqr(const Launch& L, Ctrl* c, int pass) {
  auto k = pass == 1 ? small_cholqr_1_k : small_cholqr_2_k;
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k<<<1, kST, sm, L.stream>>>(c);
  return cudaGetLastError();
}

static cudaError_t launch_small(void (*k)(Ctrl*), const Launch& L, Ctrl* c) {
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k<<<1, kST, sm, L.stream>>>(c);
  return cudaGetLastError();
}

cudaError_t small_bcg_init(const Launch& L, Ctrl* c, int) { return launch_small(small_bcg_init_k, L, c); }

// The adaptive criterion's kappa_D on its own (the same device routine).
__global__ void __launch_bounds__(kST) small_kappa_d_k(int s, const double* A, double* out) {
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) S.A[IDX(i / s, i % s)] = A[i];
  __syncthreads();
  const double k = sm_kappa_d(S.A, s, S.B, S.C, &S.flag);
  if (threadIdx.x == 0) *out = k;
}

// The re-orthonormalisation criterion on its own (the solvers' decision routine).
__global__ void __launch_bounds__(kST) small_criterion_k(int s, double eta, double eps, const double* A, int* out) {
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) S.A[IDX(i / s, i % s)] = A[i];
  __syncthreads();
  const int d = criterion(eta, eps, s, S.A, S.B, S.C, &S.flag);
  if (threadIdx.x == 0) *out = d;
}

cudaError_t small_criterion(const Launch& L, int s, double eta, double eps, const double* A, int* out) {
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(small_criterion_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  small_criterion_k<<<1, kST, sm, L.stream>>>(s, eta, eps, A, out);
  return cudaGetLastError();
}

cudaError_t small_kappa_d(const Launch& L, int s, const double* A, double* out) {
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(small_kappa_d_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  small_kappa_d_k<<<1, kST, sm, L.stream>>>(s, A, out);
  return cudaGetLastError();
}

cudaError_t small_bcg_1(const Launch& L, Ctrl* c, const uint8_t* forced) {
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(small_bcg_1_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  small_bcg_1_k<<<1, kST, sm, L.stream>>>(c, forced);
  return cudaGetLastError();
}

cudaError_t small_bcg_2(const Launch& L, Ctrl* c, double* history, uint8_t* decisions) {
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(small_bcg_2_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  small_bcg_2_k<<<1, kST, sm, L.stream>>>(c, history, decisions);
  return cudaGetLastError();
}

// ---------------------------------------------------------- BBiCGStab ----
// (Alg. "BlockBiCGStab_with_reortho", M = I.)  alpha holds R0s^T Q-hat, g2
// holds R0s^T R-hat, rho holds R-hat^T R-hat.
// 1: LU of R0s^T Q-hat, lambda-hat = (R0s^T Q-hat)^{-1} R0s^T R-hat, decision
//    from kappa_D(R-hat^T R-hat), lx = lambda-hat sigma.
__global__ void __launch_bounds__(kST) small_bicg_1_k(Ctrl* c, const uint8_t* forced) {
  if (c->done) return;
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  const int s = c->s;
  sm_copy(S.A, c->alpha, s);
  sm_copy(S.B, c->g2, s);
  sm_copy(S.E, c->sigma, s);
  __syncthreads();
  if (!sm_all_finite(S.A, s, &S.flag)) { stop(c, BK_NONFINITE); return; }
  __shared__ int piv[kMaxS];
  if (!sm_lu(S.A, piv, s, &S.flag)) { stop(c, BK_BREAKDOWN); return; }
  sm_lu_solve(S.A, piv, S.B, S.D, s);          // D = lambda-hat
  sm_copy(S.C, c->rho, s);
  __syncthreads();
  const int reo = decide(c, forced, S.C, S.B, S.F, &S.flag);
  __syncthreads();
  sm_matmul(S.B, S.D, false, S.E, s);          // lx = lambda-hat sigma
  __syncthreads();
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, b = i % s;
    c->lu[IDX(a, b)] = S.A[IDX(a, b)];
    c->lam[IDX(a, b)] = S.D[IDX(a, b)];
    c->lx[IDX(a, b)] = S.B[IDX(a, b)];
  }
  if (threadIdx.x < s) c->piv[threadIdx.x] = piv[threadIdx.x];
  if (threadIdx.x == 0) c->reortho_now = reo;
}

// 2: omega-hat = <U,S>_F / <U,U>_F, beta-hat = -(R0s^T Q-hat)^{-1} R0s^T U-hat,
//    sigma^{k+1} = gamma sigma^k (or sigma^k), lx = omega sigma^{k+1}.
__global__ void __launch_bounds__(kST) small_bicg_2_k(Ctrl* c) {
  if (c->done) return;
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  const int s = c->s;
  const double uu = c->frob[1];
  if (!(uu > 0.0) || !isfinite(uu) || !isfinite(c->frob[0])) { stop(c, BK_BREAKDOWN); return; }
  const double omega = c->frob[0] / uu;
  sm_copy(S.A, c->lu, s);
  sm_copy(S.B, c->g3, s);
  sm_copy(S.E, c->sigma, s);
  if (c->reortho_now) sm_copy(S.C, c->gamma, s); else sm_identity(S.C, s);
  __shared__ int piv[kMaxS];
  if (threadIdx.x < s) piv[threadIdx.x] = c->piv[threadIdx.x];
  __syncthreads();
  sm_lu_solve(S.A, piv, S.B, S.D, s);          // D = (R0s^T Q)^{-1} R0s^T U
  sm_matmul(S.B, S.C, false, S.E, s);          // sigma_new
  __syncthreads();
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, b = i % s;
    c->beta[IDX(a, b)] = -S.D[IDX(a, b)];
    c->sigma_new[IDX(a, b)] = S.B[IDX(a, b)];
    c->lx[IDX(a, b)] = omega * S.B[IDX(a, b)];
  }
  if (threadIdx.x == 0) { c->omega = omega; c->reorths += c->reortho_now; }
}

// 3: residual norms sqrt(diag(sigma_new^T (R^T R) sigma_new)), stopping test.
__global__ void __launch_bounds__(kST) small_bicg_3_k(Ctrl* c, double* history, uint8_t* decisions) {
  if (c->done) return;
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  const int s = c->s;
  const int k = c->iter;
  sm_copy(S.A, c->rho, s);
  sm_copy(S.B, c->sigma_new, s);
  __syncthreads();
  if (!sm_all_finite(S.A, s, &S.flag)) { stop(c, BK_NONFINITE); return; }
  sm_matmul(S.C, S.A, false, S.B, s);
  __syncthreads();
  if (threadIdx.x < s) {
    const int i = threadIdx.x;
    double v = 0.0;
    for (int r = 0; r < s; ++r) v = fma(S.B[IDX(r, i)], S.C[IDX(r, i)], v);
    const double n0 = c->n0[i];
    c->relres[i] = (!isfinite(n0) || isnan(v)) ? NAN : (n0 > 0.0 ? sqrt(fmax(v, 0.0)) / n0 : 0.0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) c->sigma[IDX(i / s, i % s)] = S.B[IDX(i / s, i % s)];
  if (threadIdx.x == 0) {
    const double mx = stop_measure(c, s);
    if (history) history[k] = mx;
    if (decisions) decisions[k] = (uint8_t)c->reortho_now;
    c->iter = k + 1;
    if (!isfinite(mx)) { c->done = kDoneStopped; c->status = BK_NONFINITE; }
    else if (mx <= c->tol) { c->done = kDoneConverged; c->status = BK_OK; }
    else if (c->iter >= c->maxit) { c->done = kDoneStopped; c->status = BK_NOT_CONVERGED; }
  }
}

cudaError_t small_bicg_1(const Launch& L, Ctrl* c, const uint8_t* forced) {
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(small_bicg_1_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  small_bicg_1_k<<<1, kST, sm, L.stream>>>(c, forced);
  return cudaGetLastError();
}
cudaError_t small_bicg_2(const Launch& L, Ctrl* c) { return launch_small(small_bicg_2_k, L, c); }
cudaError_t small_bicg_3(const Launch& L, Ctrl* c, double* history, uint8_t* decisions) {
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(small_bicg_3_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  small_bicg_3_k<<<1, kST, sm, L.stream>>>(c, history, decisions);
  return cudaGetLastError();
}

// ------------------------------------------------------------- helpers ----
__global__ void set_identity_k(double* M, int s) {
  for (int i = threadIdx.x; i < kMM; i += blockDim.x) M[i] = ((i / kMaxS) == (i % kMaxS) && (i / kMaxS) < s) ? 1.0 : 0.0;
}
cudaError_t small_set_identity(const Launch& L, double* M, int s) {
  set_identity_k<<<1, 256, 0, L.stream>>>(M, s);
  return cudaGetLastError();
}

// ------------------------------------------------------------- BGMRes ----
// One block Givens step of Alg. "bgmres" for Arnoldi step k (Ch. 5.1):
//   Hc:  the new Hessenberg column, (k+1) blocks h_jk (row stride s) from the
//        projections, gamma (ctrl->gamma) below it;
//   rotate it by Q_0^T .. Q_{k-1}^T (their reflectors stored in Gq: 2s x s
//   reflectors + s taus per step), factor [h_kk; gamma] = Q_k [r; 0] by
//   Householder, store r and Q_k, update [sigma_k; sigma_k+1] <- Q_k^T [sigma_k; 0]
//   and test max_i ||sigma_{k+1} e_i|| / ||R0_i|| <= tol.
// H: (m+1)s x ms, row stride ms: column block k gets the rotated column.
__global__ void __launch_bounds__(kST)
small_gmres_step_k(Ctrl* c, const double* __restrict__ Hc, double* __restrict__ H, double* __restrict__ Gq,
                   double* __restrict__ sig, int k, int m, double* history, int hist_index) {
  if (c->done) return;
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  const int s = c->s;
  const int ld = m * s;
  // stage the 2s x s pair [h_j; h_{j+1}] in A (row stride s) and rotate
  double* P = S.A;                 // 2s x s  (fits: 2*32*32 = 2 kMM)
  double* V = S.C;                 // 2s x s reflectors
  double* tau = S.tau;
  // working column in global H column block k
  for (int i = threadIdx.x; i < (k + 1) * s * s; i += blockDim.x) {
    const int row = i / s, col = i % s;
    H[(size_t)row * ld + k * s + col] = Hc[(size_t)(row / s) * kMM + (row % s) * kMaxS + col];
  }
  for (int i = threadIdx.x; i < s * s; i += blockDim.x)
    H[(size_t)((k + 1) * s + i / s) * ld + k * s + (i % s)] = c->gamma[IDX(i / s, i % s)];
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    for (int i = threadIdx.x; i < 2 * s * s; i += blockDim.x) {
      P[i] = H[(size_t)(j * s + i / s) * ld + k * s + (i % s)];
      V[i] = Gq[(size_t)j * (2 * s * s + s) + i];
    }
    if (threadIdx.x < s) tau[threadIdx.x] = Gq[(size_t)j * (2 * s * s + s) + 2 * s * s + threadIdx.x];
    __syncthreads();
    cta_apply_qt<double>(V, tau, 2 * s, s, P, s, S.red, S.w);
    for (int i = threadIdx.x; i < 2 * s * s; i += blockDim.x)
      H[(size_t)(j * s + i / s) * ld + k * s + (i % s)] = P[i];
    __syncthreads();
  }
  // factor [h_kk; gamma]
  for (int i = threadIdx.x; i < 2 * s * s; i += blockDim.x) P[i] = H[(size_t)(k * s + i / s) * ld + k * s + (i % s)];
  __syncthreads();
  cta_geqr2<double>(P, 2 * s, s, tau, S.red, S.w);
  for (int i = threadIdx.x; i < 2 * s * s; i += blockDim.x) {
    const int row = i / s, col = i % s;
    Gq[(size_t)k * (2 * s * s + s) + i] = P[i];
    H[(size_t)(k * s + row) * ld + k * s + col] = (row < s && col >= row) ? P[i] : 0.0;
  }
  if (threadIdx.x < s) Gq[(size_t)k * (2 * s * s + s) + 2 * s * s + threadIdx.x] = tau[threadIdx.x];
  __syncthreads();
  // sigma update: [sigma_k; sigma_{k+1}] <- Q_k^T [sigma_k; 0]
  for (int i = threadIdx.x; i < 2 * s * s; i += blockDim.x) V[i] = (i < s * s) ? sig[(size_t)k * s * s + i] : 0.0;
  __syncthreads();
  cta_apply_qt<double>(P, tau, 2 * s, s, V, s, S.red, S.w);
  for (int i = threadIdx.x; i < 2 * s * s; i += blockDim.x) sig[(size_t)k * s * s + i] = V[i];
  __syncthreads();
  if (threadIdx.x < s) {
    const int i = threadIdx.x;
    double v = 0.0;
    for (int r = 0; r < s; ++r) { const double x = V[(s + r) * s + i]; v = fma(x, x, v); }
    const double n0 = c->n0[i];
    c->relres[i] = (!isfinite(n0) || isnan(v)) ? NAN : (n0 > 0.0 ? sqrt(v) / n0 : 0.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double mx = stop_measure(c, s);
    if (history) history[hist_index] = mx;
    c->iter = c->iter + 1;
    if (!isfinite(mx)) { c->done = kDoneStopped; c->status = BK_NONFINITE; }
    else if (mx <= c->tol) { c->done = kDoneConverged; c->status = BK_OK; }
  }
}

cudaError_t small_gmres_step(const Launch& L, Ctrl* c, const double* Hc, double* H, double* Gq,
                              double* sig, int k, int m, double* history, int hist_index) {
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(small_gmres_step_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  small_gmres_step_k<<<1, kST, sm, L.stream>>>(c, Hc, H, Gq, sig, k, m, history, hist_index);
  return cudaGetLastError();
}

// Block back-substitution R zeta = sigma over k_done steps (Alg. "bgmres"):
// zeta_l = r_ll^{-1} (sigma_l - sum_{j>l} r_lj zeta_j).  zeta: k_done blocks of
// 32 x 32 doubles (row stride 32).  Runs even when the solve has stopped (it is
// the final update).
__global__ void __launch_bounds__(kST)
small_gmres_backsub_k(Ctrl* c, const double* __restrict__ H, const double* __restrict__ sig,
                      double* __restrict__ zeta, int k_done, int m) {
  extern __shared__ double smraw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
  const int s = c->s;
  const int ld = m * s;
  for (int l = k_done - 1; l >= 0; --l) {
    for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
      const int a = i / s, b = i % s;
      double v = sig[(size_t)l * s * s + i];
      for (int j = l + 1; j < k_done; ++j)
        for (int q = 0; q < s; ++q)
          v = fma(-H[(size_t)(l * s + a) * ld + j * s + q], zeta[(size_t)j * kMM + q * kMaxS + b], v);
      S.B[IDX(a, b)] = v;
      S.A[IDX(a, b)] = H[(size_t)(l * s + a) * ld + l * s + b];
    }
    __syncthreads();
    if (threadIdx.x < s) {                     // upper-triangular solve, column threadIdx.x
      const int b = threadIdx.x;
      for (int a = s - 1; a >= 0; --a) {
        double v = S.B[IDX(a, b)];
        for (int q = a + 1; q < s; ++q) v = fma(-S.A[IDX(a, q)], S.B[IDX(q, b)], v);
        const double d = S.A[IDX(a, a)];
        S.B[IDX(a, b)] = (d != 0.0) ? v / d : 0.0;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < s * s; i += blockDim.x)
      zeta[(size_t)l * kMM + (i / s) * kMaxS + (i % s)] = S.B[IDX(i / s, i % s)];
    __syncthreads();
  }
}

cudaError_t small_gmres_backsub(const Launch& L, Ctrl* c, const double* H, const double* sig,
                                double* zeta, int k_done, int m) {
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(small_gmres_backsub_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  small_gmres_backsub_k<<<1, kST, sm, L.stream>>>(c, H, sig, zeta, k_done, m);
  return cudaGetLastError();
}

// ||R0_i|| from squared column norms (ctrl->n0 holds squares on entry).
__global__ void sqrt_n0_k(Ctrl* c) {
  if (threadIdx.x < c->s) c->n0[threadIdx.x] = sqrt(c->n0[threadIdx.x]);
}
cudaError_t small_colnorms_from_gram(const Launch& L, Ctrl* c) {
  sqrt_n0_k<<<1, 32, 0, L.stream>>>(c);
  return cudaGetLastError();
}

}  // namespace bk
