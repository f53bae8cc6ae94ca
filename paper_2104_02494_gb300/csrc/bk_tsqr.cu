// Normalizer of the block case by TSQR (Ch. 7.3): X = Y sigma with Y^T Y = I,
// sigma upper triangular with diag(sigma) >= 0, defined for rank-deficient X
// (Def. "normalizer": Householder at every level, never Gram-Schmidt).
//
// The thesis splits the rows over MPI processes; here the "processes" are
// row tiles of one GPU:
//   1. leaf factor   one CTA per tile of 256 rows: Householder QR of the
//                    tile in shared memory; the reflectors overwrite the tile
//                    in Y, the tile's R factor goes to scratch;
//   2. tree factor   one CTA per tree node: Householder QR of the stacked R
//                    factors of its F = max(2, 256/s) children (FP64);
//   3. root          sign fix: gamma = D R_root with D = sign(diag R_root);
//   4. tree apply    top-down, each node turns its scatter factor sigma~ into
//                    those of its children: Q_node [sigma~; 0];
//   5. leaf apply    Y_tile = Q_tile [sigma~_tile; 0].
// Every sum inside a CTA runs in a fixed order, so the result is bitwise
// reproducible for a given n, s and device.
#include "bk_common.cuh"
#include "bk_internal.h"
#include "bk_hh.cuh"

namespace bk {

constexpr int kTile = 256;       // rows per leaf tile (>= s)
constexpr int kTT = 256;         // threads per TSQR CTA

TsqrPlan tsqr_plan(int64_t n, int s) {
  TsqrPlan p;
  p.n = n; p.s = s; p.tile = kTile;
  p.fanin = (kTile / s) < 2 ? 2 : kTile / s;
  if (p.fanin * s > kTile) p.fanin = kTile / s;
  p.nodes[0] = (n + kTile - 1) / kTile;
  int l = 0;
  while (p.nodes[l] > 1 && l < 15) {
    p.nodes[l + 1] = (p.nodes[l] + p.fanin - 1) / p.fanin;
    ++l;
  }
  p.levels = l;
  // scratch: per level l: R/sigma~ slots nodes_l*s*s, taus nodes_l*s; reflectors for l >= 1.
  size_t b = 0;
  for (int i = 0; i <= p.levels; ++i) {
    b += sizeof(double) * (size_t)p.nodes[i] * s * s;           // R / sigma~
    b += sizeof(double) * (size_t)p.nodes[i] * s;               // taus
    if (i >= 1) b += sizeof(double) * (size_t)p.nodes[i] * p.fanin * s * s;  // reflectors
  }
  p.bytes = b + 256;
  return p;
}

struct TsqrPtrs {
  double* R[16];
  double* tau[16];
  double* V[16];
};

static TsqrPtrs tsqr_ptrs(const TsqrPlan& p, void* scratch) {
  TsqrPtrs q{};
  char* c = (char*)scratch;
  const int s = p.s;
  for (int i = 0; i <= p.levels; ++i) {
    q.R[i] = (double*)c; c += sizeof(double) * (size_t)p.nodes[i] * s * s;
    q.tau[i] = (double*)c; c += sizeof(double) * (size_t)p.nodes[i] * s;
    if (i >= 1) { q.V[i] = (double*)c; c += sizeof(double) * (size_t)p.nodes[i] * p.fanin * s * s; }
  }
  return q;
}

__device__ __forceinline__ bool tsqr_skip(const int* done, const int* flag) {
  return (done && *done) || (flag && !*flag);
}

// ---- 1. leaf factor -------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kTT)
leaf_factor(int64_t n, int s, const T* __restrict__ X, T* __restrict__ Y, double* __restrict__ R0,
            double* __restrict__ tau0, const int* done, const int* flag) {
  if (tsqr_skip(done, flag)) return;
  extern __shared__ double smem_d[];
  T* M = reinterpret_cast<T*>(smem_d);
  T* red = M + kTile * s;
  T* w = red + kTT;
  T* tau = w + kMaxS;
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  const int m = (int)((n - r0) < kTile ? (n - r0) : kTile);
  for (int i = threadIdx.x; i < kTile * s; i += blockDim.x) {
    const int t = i / s;
    M[i] = (t < m) ? X[(r0 + t) * s + (i % s)] : T(0);
  }
  __syncthreads();
  const int mm = m > s ? m : s;       // a short tile is padded with zero rows up to s
  cta_geqr2<T>(M, mm, s, tau, red, w);
  for (int i = threadIdx.x; i < m * s; i += blockDim.x) Y[r0 * s + i] = M[i];
  double* Rb = R0 + (size_t)blockIdx.x * s * s;
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, c = i % s;
    Rb[i] = (c >= a && a < mm) ? (double)M[a * s + c] : 0.0;
  }
  if (threadIdx.x < s) tau0[(size_t)blockIdx.x * s + threadIdx.x] = (double)tau[threadIdx.x];
}

// ---- 2. tree factor -------------------------------------------------------------
__global__ void __launch_bounds__(kTT)
tree_factor(int64_t nchild, int F, int s, const double* __restrict__ Rc, double* __restrict__ Rn,
            double* __restrict__ Vn, double* __restrict__ taun, const int* done, const int* flag) {
  if (tsqr_skip(done, flag)) return;
  extern __shared__ double smem_d[];
  const int m = F * s;
  double* M = smem_d;
  double* red = M + m * s;
  double* w = red + kTT;
  double* tau = w + kMaxS;
  const int64_t c0 = (int64_t)blockIdx.x * F;
  for (int i = threadIdx.x; i < m * s; i += blockDim.x) {
    const int g = i / (s * s);
    M[i] = (c0 + g < nchild) ? Rc[(size_t)(c0 + g) * s * s + (i % (s * s))] : 0.0;
  }
  __syncthreads();
  cta_geqr2<double>(M, m, s, tau, red, w);
  double* V = Vn + (size_t)blockIdx.x * m * s;
  for (int i = threadIdx.x; i < m * s; i += blockDim.x) V[i] = M[i];
  double* Rb = Rn + (size_t)blockIdx.x * s * s;
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, c = i % s;
    Rb[i] = (c >= a) ? M[a * s + c] : 0.0;
  }
  if (threadIdx.x < s) taun[(size_t)blockIdx.x * s + threadIdx.x] = tau[threadIdx.x];
}

// ---- 3. root: gamma = D R, sigma~_root = D ------------------------------------------
__global__ void root_fix(int s, double* __restrict__ Rroot, double* __restrict__ gamma_out,
                         const int* done, const int* flag) {
  if (tsqr_skip(done, flag)) return;
  __shared__ double d[kMaxS];
  if (threadIdx.x < s) d[threadIdx.x] = (Rroot[threadIdx.x * s + threadIdx.x] < 0.0) ? -1.0 : 1.0;
  __syncthreads();
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, c = i % s;
    gamma_out[a * kMaxS + c] = d[a] * Rroot[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int a = i / s, c = i % s;
    Rroot[i] = (a == c) ? d[a] : 0.0;        // scatter factor of the root
  }
}

// ---- 4. tree apply --------------------------------------------------------------
__global__ void __launch_bounds__(kTT)
tree_apply(int64_t nchild, int F, int s, const double* __restrict__ Vn, const double* __restrict__ taun,
           const double* __restrict__ Sn, double* __restrict__ Sc, const int* done, const int* flag) {
  if (tsqr_skip(done, flag)) return;
  extern __shared__ double smem_d[];
  const int m = F * s;
  double* V = smem_d;
  double* C = V + m * s;
  double* red = C + m * s;
  double* w = red + kTT;
  double* tau = w + kMaxS;
  const double* Vb = Vn + (size_t)blockIdx.x * m * s;
  for (int i = threadIdx.x; i < m * s; i += blockDim.x) {
    V[i] = Vb[i];
    C[i] = (i < s * s) ? Sn[(size_t)blockIdx.x * s * s + i] : 0.0;
  }
  if (threadIdx.x < s) tau[threadIdx.x] = taun[(size_t)blockIdx.x * s + threadIdx.x];
  __syncthreads();
  cta_apply_q<double>(V, tau, m, s, C, red, w);
  const int64_t c0 = (int64_t)blockIdx.x * F;
  for (int i = threadIdx.x; i < m * s; i += blockDim.x) {
    const int g = i / (s * s);
    if (c0 + g < nchild) Sc[(size_t)(c0 + g) * s * s + (i % (s * s))] = C[i];
  }
}

// ---- 5. leaf apply ----------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kTT)
leaf_apply(int64_t n, int s, T* __restrict__ Y, const double* __restrict__ S0,
           const double* __restrict__ tau0, const int* done, const int* flag) {
  if (tsqr_skip(done, flag)) return;
  extern __shared__ double smem_d[];
  T* V = reinterpret_cast<T*>(smem_d);
  T* C = V + kTile * s;
  T* red = C + kTile * s;
  T* w = red + kTT;
  T* tau = w + kMaxS;
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  const int m = (int)((n - r0) < kTile ? (n - r0) : kTile);
  const int mm = m > s ? m : s;
  for (int i = threadIdx.x; i < mm * s; i += blockDim.x) {
    const int t = i / s;
    V[i] = (t < m) ? Y[(r0 + t) * s + (i % s)] : T(0);
    C[i] = (i < s * s) ? (T)S0[(size_t)blockIdx.x * s * s + i] : T(0);
  }
  if (threadIdx.x < s) tau[threadIdx.x] = (T)tau0[(size_t)blockIdx.x * s + threadIdx.x];
  __syncthreads();
  cta_apply_q<T>(V, tau, mm, s, C, red, w);
  for (int i = threadIdx.x; i < m * s; i += blockDim.x) Y[r0 * s + i] = C[i];
}

template <typename K>
static cudaError_t set_smem(K kern, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
cudaError_t tsqr(const Launch& L, const TsqrPlan& p, const T* X, T* Y, double* gamma_out,
                 double* rho_out, void* scratch, double* gpart, unsigned* counter, const int* done,
                 const int* flag) {
  const int s = p.s;
  const int64_t n = p.n;
  TsqrPtrs q = tsqr_ptrs(p, scratch);
  cudaError_t e;
  // 1. leaves
  prof_begin(L, kPhTsqrLeaf);
  {
    const size_t sm = sizeof(T) * ((size_t)kTile * s + kTT + 2 * kMaxS) + 64;
    auto k = leaf_factor<T>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    k<<<(unsigned)p.nodes[0], kTT, sm, L.stream>>>(n, s, X, Y, q.R[0], q.tau[0], done, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  prof_end(L, kPhTsqrLeaf, 1);
  // 2. tree up
  prof_begin(L, kPhTsqrTree);
  const int F = p.fanin;
  const size_t smf = sizeof(double) * ((size_t)F * s * s + kTT + 2 * kMaxS) + 64;
  if ((e = set_smem(tree_factor, smf)) != cudaSuccess) return e;
  for (int l = 1; l <= p.levels; ++l) {
    tree_factor<<<(unsigned)p.nodes[l], kTT, smf, L.stream>>>(p.nodes[l - 1], F, s, q.R[l - 1], q.R[l],
                                                               q.V[l], q.tau[l], done, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 3. root
  root_fix<<<1, 256, 0, L.stream>>>(s, q.R[p.levels], gamma_out, done, flag);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 4. tree down
  const size_t sma = sizeof(double) * (2 * (size_t)F * s * s + kTT + 2 * kMaxS) + 64;
  if ((e = set_smem(tree_apply, sma)) != cudaSuccess) return e;
  for (int l = p.levels; l >= 1; --l) {
    tree_apply<<<(unsigned)p.nodes[l], kTT, sma, L.stream>>>(p.nodes[l - 1], F, s, q.V[l], q.tau[l],
                                                              q.R[l], q.R[l - 1], done, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  prof_end(L, kPhTsqrTree, 2 * p.levels + 1);
  // 5. leaves
  prof_begin(L, kPhTsqrApply);
  {
    const size_t sm = sizeof(T) * (2 * (size_t)kTile * s + kTT + 2 * kMaxS) + 64;
    auto k = leaf_apply<T>;
    if ((e = set_smem(k, sm)) != cudaSuccess) return e;
    k<<<(unsigned)p.nodes[0], kTT, sm, L.stream>>>(n, s, Y, q.R[0], q.tau[0], done, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  prof_end(L, kPhTsqrApply, 1);
  if (rho_out) {
    Epi<T> ep;
    ep.sym = 1;
    ep.gram_out = rho_out;
    ep.gpart = gpart;
    ep.counter = counter;
    ep.done = done;
    ep.only_if = flag;          // a skipped normalisation also skips its Gram
    prof_begin(L, kPhTsqrGram);
    e = gram<T>(L, n, s, Y, Y, ep);
    prof_end(L, kPhTsqrGram, 1);
    return e;
  }
  return cudaSuccess;
}

template cudaError_t tsqr<double>(const Launch&, const TsqrPlan&, const double*, double*, double*,
                                  double*, void*, double*, unsigned*, const int*, const int*);
template cudaError_t tsqr<float>(const Launch&, const TsqrPlan&, const float*, float*, double*,
                                 double*, void*, double*, unsigned*, const int*, const int*);

}  // namespace bk
