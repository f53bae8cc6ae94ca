// Localized Arnoldi orthonormalisation for block GMRes (Ch. 9.3, Alg.
// "localized-arnoldi" with Algs. "reduction-localized" and
// "back-propagation-localized").
//
// The thesis's processes are the TSQR leaf tiles of one GPU (tile_rows rows
// each).  The Arnoldi basis is kept as a distributed S-QR decomposition
// (Def. "Distributed S-QR decomposition"): every tile t has a local
// orthonormal basis P_t^0, P_t^1, ... (the blocks Pb[j] restricted to the
// tile's rows) and the global basis vector k is V^k_t = sum_j P_t^j (zeta_t^k)_j.
// Extending the basis by W = A V^k:
//   1. la_mgs: per tile (one CTA, the tile of W in shared memory) block modified
//      Gram-Schmidt against P_t^0 .. P_t^k, every projection an s x s CTA sum:
//      the local coefficients go to Zt[t][j];
//   2. the rest of the tile is normalised by the tile Householder QR of the
//      TSQR normaliser (tsqr_local_q): P_t^{k+1} explicit, its R to Zt[t][k+1];
//   3. la_reduce, one launch per tree level, one CTA per node (a tree of
//      `fanin` children per node over the tiles, the same in every step; the
//      thesis prints the binary one): the children's vectors are
//      stacked, orthonormalised against the node's own basis by modified
//      Gram-Schmidt and normalised by a CTA Householder QR (diag(R) >= 0);
//      the node stores the new basis vector and passes its R-factor up; the
//      root's R-factor is the new Hessenberg column (projections and gamma);
//   4. la_backprop, one launch per level from the root down: a node that
//      receives the coefficients rho~ hands sum_i [zeta^i_c; 0] rho~_i to its
//      child c (the root receives the unit vector of its newest basis vector);
//      the tiles receive zeta_t;
//   5. la_assemble: V^{k+1}_t = sum_j P_t^j (zeta_t)_j.
// The local work of a step is 6 (k + 1) n s^2 flops (k + 1 projections and
// updates, k + 2 assembly terms) against 8 (k + 1) n s^2 for classical
// Gram-Schmidt repeated twice; the tree works on s x s blocks only.
#include <cstring>

#include "bk_common.cuh"
#include "bk_hh.cuh"
#include "bk_internal.h"

namespace bk {

// values of the tile held per thread in the row layout: tile_rows * SW / 256
// (tile_rows = 256 * leaf rows per thread of the FP64 TSQR: 64 / SW, 32 / SW at SW <= 4)
template <int SW>
__host__ __device__ constexpr int la_nt() { return (SW <= 4 ? 32 : 64); }

constexpr int kLocMaxS = 16;                   // widest block of the localized method

// ---- 1. local block modified Gram-Schmidt ---------------------------------------
// One CTA per tile; the tile of W is held in shared memory in the row layout
// (row stride SW: a warp's 32 / SW rows are 32 consecutive doubles).
template <int SW>
__global__ void __launch_bounds__(kThreads)
la_mgs(int64_t n, int s, int tile_rows, int k1, const double* const* __restrict__ Pb, double* __restrict__ W,
       double* __restrict__ Zt, int64_t ldz) {
  constexpr int NT = la_nt<SW>();
  constexpr int RPW = 32 / SW;                 // rows per warp per trip
  constexpr int RPC = kWarps * RPW;            // rows per CTA per trip
  extern __shared__ double Wt[];               // [tile_rows][SW]
  __shared__ double red[kWarps][SW][SW];
  __shared__ double G[SW][SW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = lane % SW, sub = lane / SW;
  const int64_t t0 = (int64_t)blockIdx.x * tile_rows;
  const int64_t tend = (t0 + tile_rows < n) ? t0 + tile_rows : n;
  for (int q = 0; q < NT; ++q) {
    const int lr = q * RPC + warp * RPW + sub;          // row within the tile
    const int64_t r = t0 + lr;
    Wt[lr * SW + c] = (r < tend && c < s) ? W[r * s + c] : 0.0;
  }
  for (int j = 0; j < k1; ++j) {
    const double* P = Pb[j];
    double acc[SW];
#pragma unroll
    for (int a = 0; a < SW; ++a) acc[a] = 0.0;
#pragma unroll 4
    for (int q = 0; q < NT; ++q) {
      const int lr = q * RPC + warp * RPW + sub;
      const int64_t r = t0 + lr;
      const double p = (r < tend && c < s) ? P[r * s + c] : 0.0;
      const double wv = Wt[lr * SW + c];
#pragma unroll
      for (int a = 0; a < SW; ++a) acc[a] = fma(sw_bcast<SW>(p, a), wv, acc[a]);      // P[r][a] W[r][c]
    }
#pragma unroll
    for (int a = 0; a < SW; ++a)
#pragma unroll
      for (int off = SW; off < 32; off <<= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], off);
    if (sub == 0) {
#pragma unroll
      for (int a = 0; a < SW; ++a) red[warp][a][c] = acc[a];
    }
    __syncthreads();
    if (tid < SW * SW) {
      const int a = tid / SW, b = tid % SW;
      double v = 0.0;
      for (int ww = 0; ww < kWarps; ++ww) v += red[ww][a][b];
      G[a][b] = v;
      if (a < s && b < s) Zt[(int64_t)blockIdx.x * ldz + (int64_t)j * s * s + a * s + b] = v;
    }
    __syncthreads();
    double g[SW];
#pragma unroll
    for (int a = 0; a < SW; ++a) g[a] = G[a][c];
#pragma unroll 4
    for (int q = 0; q < NT; ++q) {
      const int lr = q * RPC + warp * RPW + sub;
      const int64_t r = t0 + lr;
      const double p = (r < tend && c < s) ? P[r * s + c] : 0.0;
      double wv = Wt[lr * SW + c];
#pragma unroll
      for (int a = 0; a < SW; ++a) wv = fma(-sw_bcast<SW>(p, a), g[a], wv);            // W -= P G
      Wt[lr * SW + c] = wv;
    }
  }
  // each thread rewrites exactly the entries it updated
  for (int q = 0; q < NT; ++q) {
    const int lr = q * RPC + warp * RPW + sub;
    const int64_t r = t0 + lr;
    if (r < tend && c < s) W[r * s + c] = Wt[lr * SW + c];
  }
}

// ---- 5. assembly of the new global basis vector ----------------------------------
// V_t = sum_{j < k2} P_t^j Zl[t][j]; the tile's coefficients in shared memory.
template <int SW>
__global__ void __launch_bounds__(kThreads)
la_assemble(int64_t n, int s, int tile_rows, int k2, const double* const* __restrict__ Pb,
            const double* __restrict__ Zl, int64_t ldz, double* __restrict__ V) {
  constexpr int NT = la_nt<SW>();
  constexpr int RPW = 32 / SW;
  constexpr int RPC = kWarps * RPW;
  extern __shared__ double Z[];                // [k2][SW][SW]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = lane % SW, sub = lane / SW;
  const int64_t t0 = (int64_t)blockIdx.x * tile_rows;
  const int64_t tend = (t0 + tile_rows < n) ? t0 + tile_rows : n;
  for (int i = tid; i < k2 * SW * SW; i += kThreads) {
    const int j = i / (SW * SW), a = (i / SW) % SW, b = i % SW;
    Z[i] = (a < s && b < s) ? Zl[(int64_t)blockIdx.x * ldz + (int64_t)j * s * s + a * s + b] : 0.0;
  }
  __syncthreads();
  // four trips at a time: four independent accumulation chains per thread
  for (int q0 = 0; q0 < NT; q0 += 4) {
    int64_t r[4];
    bool ok[4];
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      r[u] = t0 + (int64_t)(q0 + u) * RPC + warp * RPW + sub;
      ok[u] = r[u] < tend && c < s;
      v[u] = 0.0;
    }
    for (int j = 0; j < k2; ++j) {
      const double* P = Pb[j];
      double p[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) p[u] = ok[u] ? P[r[u] * s + c] : 0.0;
#pragma unroll
      for (int a = 0; a < SW; ++a) {
        const double z = Z[(j * SW + a) * SW + c];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = fma(sw_bcast<SW>(p[u], a), z, v[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (ok[u]) V[r[u] * s + c] = v[u];
  }
}

// ---- 3. tree reduction, one CTA per node ----------------------------------------
// child_out: [nchild][mx s][s] (K2 = k1 + 1 blocks valid); NB: [nodes][m1][F][mx s][s];
// Rout: [nodes][mx s][s].  Shared memory: S (F mx s x s), C (as S, at least 256 s),
// rho (s x s), red (256), w, tau (32 each), the sign vector (32).  256 threads.
__global__ void __launch_bounds__(256)
la_reduce(int64_t nchild, int s, int k1, int mx, int m1, int F, const double* __restrict__ child_out,
          double* __restrict__ NB, double* __restrict__ Rout) {
  extern __shared__ double sm[];
  const int K2 = k1 + 1, Lr = K2 * s;
  const int64_t node = blockIdx.x;
  const int64_t c0 = (int64_t)F * node;
  const int nc = (int)((nchild - c0) < F ? (nchild - c0) : F);
  const int mrows = nc * Lr;
  const size_t cap = (size_t)F * mx * s * s;
  const size_t capc = cap > (size_t)256 * s ? cap : (size_t)256 * s;   // C also holds 256 s partials
  double* S = sm;
  double* C = S + cap;
  double* rho = C + capc;
  double* red = rho + s * s;
  double* w = red + 256;
  double* tau = w + 32;
  double* dsg = tau + 32;
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t vec = (size_t)mx * s * s;                 // one component / one vector
  for (int i = tid; i < mrows * s; i += nt) {
    const int row = i / s, col = i % s, q = row / Lr, rr = row % Lr;
    S[i] = child_out[(c0 + q) * vec + (size_t)rr * s + col];
  }
  __syncthreads();
  double* nbn = NB + (size_t)node * m1 * F * vec;
  double* rout = Rout + (size_t)node * vec;
  for (int i = 0; i < k1; ++i) {
    const double* Zi = nbn + (size_t)i * F * vec;         // [F][mx s][s], rows < (i + 1) s non-zero
    const int li = (i + 1) * s;
    {
      // thread (a, part): rho_i[a][:] over the rows part, part + np, ... (s chains
      // per thread); the np partial rows go to C (free until the normaliser)
      const int np = nt / s, a = tid % s, part = tid / s;
      if (part < np) {
        double acc[kLocMaxS];
#pragma unroll
        for (int b = 0; b < kLocMaxS; ++b) acc[b] = 0.0;
        for (int row = part; row < nc * li; row += np) {
          const int q = row / li, rr = row % li;
          const double z = Zi[q * vec + (size_t)rr * s + a];
          const double* Sr = S + (q * Lr + rr) * s;
#pragma unroll
          for (int b = 0; b < kLocMaxS; ++b)
            if (b < s) acc[b] = fma(z, Sr[b], acc[b]);
        }
#pragma unroll
        for (int b = 0; b < kLocMaxS; ++b)
          if (b < s) C[((size_t)part * s + a) * s + b] = acc[b];
      }
      __syncthreads();
      for (int e = tid; e < s * s; e += nt) {
        double v = 0.0;
        for (int pp = 0; pp < np; ++pp) v += C[(size_t)pp * s * s + e];
        rho[e] = v;
      }
    }
    __syncthreads();
    for (int e = tid; e < nc * li * s; e += nt) {
      const int col = e % s, row2 = e / s, q = row2 / li, rr = row2 % li;
      double v = S[(q * Lr + rr) * s + col];
      for (int a = 0; a < s; ++a) v = fma(-Zi[q * vec + (size_t)rr * s + a], rho[a * s + col], v);
      S[(q * Lr + rr) * s + col] = v;
    }
    for (int e = tid; e < s * s; e += nt) rout[(size_t)i * s * s + e] = rho[e];
    __syncthreads();
  }
  // normalise the stacked rest: S = Q R (Householder), Q explicit in C, diag(R) >= 0
  cta_geqr2(S, mrows, s, tau, red, w);
  for (int i = tid; i < mrows * s; i += nt) C[i] = ((i / s) == (i % s)) ? 1.0 : 0.0;
  __syncthreads();
  cta_apply_q(S, tau, mrows, s, C, red, w);
  if (tid < s) dsg[tid] = (S[tid * s + tid] < 0.0) ? -1.0 : 1.0;
  __syncthreads();
  double* nbk = nbn + (size_t)k1 * F * vec;
  for (int i = tid; i < mrows * s; i += nt) {
    const int row = i / s, col = i % s, q = row / Lr, rr = row % Lr;
    nbk[q * vec + (size_t)rr * s + col] = C[i] * dsg[col];
  }
  for (int e = tid; e < s * s; e += nt) {
    const int a = e / s, b = e % s;
    rout[(size_t)k1 * s * s + e] = (b >= a) ? dsg[a] * S[a * s + b] : 0.0;
  }
}

// ---- 4. back-propagation, one CTA per node --------------------------------------
// cin: [nodes][mx s][s] (K2 blocks valid); cout: [nchild][mx s][s].
__global__ void __launch_bounds__(256)
la_backprop(int64_t nchild, int s, int k1, int mx, int m1, int F, const double* __restrict__ cin,
            const double* __restrict__ NB, double* __restrict__ cout) {
  extern __shared__ double rt[];                          // K2 s x s
  const int K2 = k1 + 1, Lr = K2 * s;
  const int64_t node = blockIdx.x;
  const int64_t c0 = (int64_t)F * node;
  const int nc = (int)((nchild - c0) < F ? (nchild - c0) : F);
  const size_t vec = (size_t)mx * s * s;
  for (int i = threadIdx.x; i < Lr * s; i += blockDim.x) rt[i] = cin[node * vec + i];
  __syncthreads();
  const double* nbn = NB + (size_t)node * m1 * F * vec;
  // one output row per thread, its s columns as independent chains
  for (int row = threadIdx.x; row < nc * Lr; row += blockDim.x) {
    const int q = row / Lr, rr = row % Lr;
    double acc[kLocMaxS];
#pragma unroll
    for (int b = 0; b < kLocMaxS; ++b) acc[b] = 0.0;
    for (int ii = rr / s; ii <= k1; ++ii) {                // zeta^ii_q is zero below (ii + 1) s rows
      const double* Z = nbn + (size_t)ii * F * vec + q * vec + (size_t)rr * s;
      for (int a = 0; a < s; ++a) {
        const double z = Z[a];
        const double* R = rt + (ii * s + a) * s;
#pragma unroll
        for (int b = 0; b < kLocMaxS; ++b)
          if (b < s) acc[b] = fma(z, R[b], acc[b]);
      }
    }
#pragma unroll
    for (int b = 0; b < kLocMaxS; ++b)
      if (b < s) cout[(c0 + q) * vec + (size_t)rr * s + b] = acc[b];
  }
}

// The root's R-factor (K2 blocks) to the Hessenberg column (blocks 0 .. k1-1, row
// stride 32) and gamma (block k1); the unit coefficient vector e_k1 into unit.
__global__ void la_root_out(int s, int k1, const double* __restrict__ R, double* __restrict__ Hc,
                            double* __restrict__ gamma, double* __restrict__ unit) {
  const int K2 = k1 + 1;
  for (int i = threadIdx.x; i < K2 * s * s; i += blockDim.x) {
    const int j = i / (s * s), a = (i / s) % s, b = i % s;
    if (j < k1) Hc[(size_t)j * kMM + a * kMaxS + b] = R[i];
    else gamma[a * kMaxS + b] = R[i];
    unit[i] = (j == k1 && a == b) ? 1.0 : 0.0;
  }
}

// ---- host side ------------------------------------------------------------------
static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t local_arnoldi_bytes(int64_t n, int s, int m, int tile_rows, LocalArnoldi* la) {
  LocalArnoldi& a = *la;
  a.s = s; a.n = n; a.m1 = m + 1; a.mx = m + 1; a.tile_rows = tile_rows;
  a.tiles = (n + tile_rows - 1) / tile_rows;
  // fan-in: the widest of 8, 4, 2 whose node fits 200 KB of shared memory
  auto smem_of = [&](int F) {
    const size_t cap = (size_t)F * a.mx * s * s;
    return sizeof(double) * (cap + (cap > (size_t)256 * s ? cap : (size_t)256 * s) + (size_t)s * s + 256 + 96);
  };
  a.fanin = 2;
  for (int F : {8, 4}) {
    if (smem_of(F) <= 200 * 1024) { a.fanin = F; break; }
  }
  a.reduce_smem = smem_of(a.fanin);
  a.nodes[0] = a.tiles;
  a.levels = 0;
  while (a.nodes[a.levels] > 1 && a.levels < 23) {
    a.nodes[a.levels + 1] = (a.nodes[a.levels] + a.fanin - 1) / a.fanin;
    ++a.levels;
  }
  const size_t vec = (size_t)a.mx * s * s * sizeof(double);
  size_t b = al256(sizeof(double*) * (size_t)a.m1) + 2 * al256(vec * (size_t)a.tiles);
  for (int l = 1; l <= a.levels; ++l) {
    a.nb_bytes[l] = (size_t)a.nodes[l] * a.m1 * a.fanin * vec;
    b += al256(a.nb_bytes[l]) + 2 * al256(vec * (size_t)a.nodes[l]);
  }
  return b;
}

int local_arnoldi_layout(void* base, LocalArnoldi* la, double* const* pb_host, cudaStream_t st) {
  LocalArnoldi& a = *la;
  char* p = (char*)base;
  const size_t vec = (size_t)a.mx * a.s * a.s * sizeof(double);
  a.Pb = (double**)p; p += al256(sizeof(double*) * (size_t)a.m1);
  a.Zt = (double*)p; p += al256(vec * (size_t)a.tiles);
  a.Zl = (double*)p; p += al256(vec * (size_t)a.tiles);
  for (int l = 1; l <= a.levels; ++l) {
    a.NB[l] = (double*)p; p += al256(a.nb_bytes[l]);
    a.Rout[l] = (double*)p; p += al256(vec * (size_t)a.nodes[l]);
    a.Cin[l] = (double*)p; p += al256(vec * (size_t)a.nodes[l]);
  }
  if (a.m1 > 72) return BK_ERR_ARG;
  for (int j = 0; j < a.m1; ++j) a.Pbh[j] = pb_host[j];
  if (cudaMemcpyAsync(a.Pb, pb_host, sizeof(double*) * (size_t)a.m1, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return BK_ERR_CUDA;
  return BK_OK;
}

cudaError_t local_arnoldi_begin(const Launch& L, const LocalArnoldi& la) {
  for (int l = 1; l <= la.levels; ++l) {
    cudaError_t e = cudaMemsetAsync(la.NB[l], 0, la.nb_bytes[l], L.stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename K>
static cudaError_t raise_smem(K kern, size_t bytes) {
  if (bytes <= 44 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int SW>
static cudaError_t la_local(const Launch& L, const LocalArnoldi& la, int k1, double* W) {
  if (k1 == 0) return cudaSuccess;
  const int64_t ldz = (int64_t)la.mx * la.s * la.s;
  const size_t sm = sizeof(double) * (size_t)la.tile_rows * SW;
  cudaError_t e = raise_smem(la_mgs<SW>, sm);
  if (e != cudaSuccess) return e;
  la_mgs<SW><<<(unsigned)la.tiles, kThreads, sm, L.stream>>>(la.n, la.s, la.tile_rows, k1, la.Pb, W, la.Zt, ldz);
  return cudaGetLastError();
}

template <int SW>
static cudaError_t la_assemble_launch(const Launch& L, const LocalArnoldi& la, int k2, double* V) {
  const int64_t ldz = (int64_t)la.mx * la.s * la.s;
  const size_t sm = sizeof(double) * (size_t)k2 * SW * SW;
  cudaError_t e = raise_smem(la_assemble<SW>, sm);
  if (e != cudaSuccess) return e;
  la_assemble<SW><<<(unsigned)la.tiles, kThreads, sm, L.stream>>>(la.n, la.s, la.tile_rows, k2, la.Pb, la.Zl,
                                                                 ldz, V);
  return cudaGetLastError();
}

cudaError_t local_arnoldi_extend(const Launch& L, const LocalArnoldi& la, const TsqrPlan& tp, void* tsqr_scratch,
                                 int k1, double* W, double* V, double* Hc, double* gamma) {
  const int s = la.s;
  const int sw = next_pow2_s(s);
  if (tp.tile != la.tile_rows || tp.tile * sw != 256 * (sw <= 4 ? 32 : 64) || k1 >= la.m1)
    return cudaErrorInvalidValue;
  cudaError_t e;
  const int64_t ldz = (int64_t)la.mx * s * s;
  // 1. local MGS
  prof_begin(L, kPhOrtho);
  switch (sw) {
    case 1: e = la_local<1>(L, la, k1, W); break;
    case 2: e = la_local<2>(L, la, k1, W); break;
    case 4: e = la_local<4>(L, la, k1, W); break;
    case 8: e = la_local<8>(L, la, k1, W); break;
    case 16: e = la_local<16>(L, la, k1, W); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  prof_end(L, kPhOrtho, k1 > 0 ? 1 : 0);
  // 2. local normaliser: P_t^{k1} and its R-factor into Zt[t][k1]
  prof_begin(L, kPhTsqrLeaf);
  if ((e = tsqr_local_q(L, tp, W, la.Pbh[k1], la.Zt + (size_t)k1 * s * s, ldz, tsqr_scratch)) != cudaSuccess)
    return e;
  prof_end(L, kPhTsqrLeaf, 4);
  prof_begin(L, kPhLaTree);
  // 3. reduction up the tree, 4. back-propagation
  const int K2 = k1 + 1;
  if (la.levels == 0) {
    la_root_out<<<1, 256, 0, L.stream>>>(s, k1, la.Zt, Hc, gamma, la.Zl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    if ((e = raise_smem(la_reduce, la.reduce_smem)) != cudaSuccess) return e;
    for (int l = 1; l <= la.levels; ++l) {
      const double* child = (l == 1) ? la.Zt : la.Rout[l - 1];
      la_reduce<<<(unsigned)la.nodes[l], 256, la.reduce_smem, L.stream>>>(la.nodes[l - 1], s, k1, la.mx, la.m1,
                                                                          la.fanin, child, la.NB[l], la.Rout[l]);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    la_root_out<<<1, 256, 0, L.stream>>>(s, k1, la.Rout[la.levels], Hc, gamma, la.Cin[la.levels]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t bsm = sizeof(double) * (size_t)K2 * s * s;
    if ((e = raise_smem(la_backprop, bsm)) != cudaSuccess) return e;
    for (int l = la.levels; l >= 1; --l) {
      double* out = (l == 1) ? la.Zl : la.Cin[l - 1];
      la_backprop<<<(unsigned)la.nodes[l], 256, bsm, L.stream>>>(la.nodes[l - 1], s, k1, la.mx, la.m1,
                                                                  la.fanin, la.Cin[l], la.NB[l], out);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  prof_end(L, kPhLaTree, la.levels == 0 ? 1 : 2 * la.levels + 1);
  // 5. the new global basis vector
  prof_begin(L, kPhLaAssemble);
  switch (sw) {
    case 1: e = la_assemble_launch<1>(L, la, K2, V); break;
    case 2: e = la_assemble_launch<2>(L, la, K2, V); break;
    case 4: e = la_assemble_launch<4>(L, la, K2, V); break;
    case 8: e = la_assemble_launch<8>(L, la, K2, V); break;
    case 16: e = la_assemble_launch<16>(L, la, K2, V); break;
    default: return cudaErrorInvalidValue;
  }
  prof_end(L, kPhLaAssemble, 1);
  return e;
}

}  // namespace bk
