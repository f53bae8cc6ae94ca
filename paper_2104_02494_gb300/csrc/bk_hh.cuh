// CTA-level Householder QR and Q application in shared memory (used by the
// TSQR normalizer and by the block Givens step of block GMRes).
#pragma once
#include "bk_common.cuh"

namespace bk {

// Sum of one value per thread over the CTA (fixed order).  red: >= 32 doubles.
template <typename A>
__device__ A cta_sum(A v, A* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  A t = A(0);
  const int nw = blockDim.x >> 5;
  for (int w = 0; w < nw; ++w) t += red[w];
  __syncthreads();
  return t;
}

// In-place Householder QR of the m x s matrix A (shared memory, row stride s).
// On exit: R in the upper triangle, reflector j below the diagonal of column j
// (its diagonal entry 1 is implicit), tau[j] in shared memory.  Reflector j
// maps column j onto beta_j e_j with beta_j = -sign(alpha) ||x|| (identity
// when the sub-diagonal part is zero).  Column-parallel inner products:
// thread (k, q) sums rows q, q+P, ... of column k, then the P partials are
// added in order q = 0..P-1.
template <typename A>
__device__ void cta_geqr2(A* M, int m, int s, A* tau, A* red, A* w) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < s; ++j) {
    A part = A(0);
    for (int t = j + 1 + tid; t < m; t += nt) { const A a = M[t * s + j]; part = fma(a, a, part); }
    const A tail = cta_sum(part, red);
    const A alpha = M[j * s + j];
    A beta, tj, scale;
    if (tail == A(0)) { tj = A(0); beta = alpha; scale = A(0); }
    else {
      const A nrm = sqrt(alpha * alpha + tail);
      beta = alpha >= A(0) ? -nrm : nrm;
      tj = (beta - alpha) / beta;
      scale = A(1) / (alpha - beta);
    }
    if (tid == 0) tau[j] = tj;
    const int L = s - j - 1;
    if (tj != A(0)) {
      for (int t = j + 1 + tid; t < m; t += nt) M[t * s + j] *= scale;
      __syncthreads();
      if (L > 0) {
        const int P = nt / L, k = tid % L, q = tid / L;
        A acc = A(0);
        if (q < P)
          for (int t = j + q; t < m; t += P) {
            const A v = (t == j) ? A(1) : M[t * s + j];
            acc = fma(v, M[t * s + j + 1 + k], acc);
          }
        red[tid] = acc;
        __syncthreads();
        if (tid < L) {
          A sacc = A(0);
          for (int qq = 0; qq < P; ++qq) sacc += red[qq * L + tid];
          w[tid] = tj * sacc;
        }
        __syncthreads();
        if (q < P)
          for (int t = j + q; t < m; t += P) {
            const A v = (t == j) ? A(1) : M[t * s + j];
            M[t * s + j + 1 + k] = fma(-w[k], v, M[t * s + j + 1 + k]);
          }
      }
    }
    __syncthreads();
    if (tid == 0) M[j * s + j] = beta;
    __syncthreads();
  }
}

// C <- H_0 H_1 ... H_{s-1} C for the reflectors stored below the diagonal of V
// (m x s, row stride s) and C (m x s, row stride s): reflectors applied last
// to first.
template <typename A>
__device__ void cta_apply_q(const A* V, const A* tau, int m, int s, A* C, A* red, A* w) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int L = s, P = nt / L, k = tid % L, q = tid / L;
  for (int j = s - 1; j >= 0; --j) {
    const A tj = tau[j];
    if (tj == A(0)) continue;
    A acc = A(0);
    if (q < P)
      for (int t = j + q; t < m; t += P) {
        const A v = (t == j) ? A(1) : V[t * s + j];
        acc = fma(v, C[t * s + k], acc);
      }
    red[tid] = acc;
    __syncthreads();
    if (tid < L) {
      A sacc = A(0);
      for (int qq = 0; qq < P; ++qq) sacc += red[qq * L + tid];
      w[tid] = tj * sacc;
    }
    __syncthreads();
    if (q < P)
      for (int t = j + q; t < m; t += P) {
        const A v = (t == j) ? A(1) : V[t * s + j];
        C[t * s + k] = fma(-w[k], v, C[t * s + k]);
      }
    __syncthreads();
  }
}

// C <- H_{s-1} ... H_1 H_0 C  (= Q^T C): reflectors applied first to last.
template <typename A>
__device__ void cta_apply_qt(const A* V, const A* tau, int m, int s, A* C, int sc, A* red, A* w) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int L = sc, P = nt / L, k = tid % L, q = tid / L;
  for (int j = 0; j < s; ++j) {
    const A tj = tau[j];
    if (tj == A(0)) continue;
    A acc = A(0);
    if (q < P)
      for (int t = j + q; t < m; t += P) {
        const A v = (t == j) ? A(1) : V[t * s + j];
        acc = fma(v, C[t * sc + k], acc);
      }
    red[tid] = acc;
    __syncthreads();
    if (tid < L) {
      A sacc = A(0);
      for (int qq = 0; qq < P; ++qq) sacc += red[qq * L + tid];
      w[tid] = tj * sacc;
    }
    __syncthreads();
    if (q < P)
      for (int t = j + q; t < m; t += P) {
        const A v = (t == j) ? A(1) : V[t * s + j];
        C[t * sc + k] = fma(-w[k], v, C[t * sc + k]);
      }
    __syncthreads();
  }
}

}  // namespace bk
