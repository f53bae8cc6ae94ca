// Normalizer of the block case by TSQR (Ch. 7.3): X = Y sigma with Y^T Y = I,
// sigma upper triangular with diag(sigma) >= 0, defined for rank-deficient X
// (Def. "normalizer": Householder at every level, never Gram-Schmidt).
//
// The thesis splits the rows over MPI processes; here the "processes" are
// row tiles of one GPU:
//   1. leaf factor   one CTA per tile of 256 x RPT rows (RPT = 64 / next_pow2(s);
//                    32 / next_pow2(s) for FP64 blocks of width <= 4),
//                    the rows in registers: Householder QR of the tile; the reflectors
//                    overwrite the tile in Y; the tile's R factor and the factor
//                    F = strict_upper(V^T V) + diag(tau) of its compact WY form
//                    H_0 ... H_{s-1} = I - V T V^T (T^{-1} = diag(1/tau) +
//                    strict_upper(V^T V)) go to scratch;
//   2. tree factor   the same kernel, one row per thread, on tiles of 256 rows
//                    of the stacked R factors of the level below (stored in
//                    FP64, arithmetic in the block's precision);
//   3. root          sign fix: gamma = D R_root with D = sign(diag R_root);
//   4. tree apply    top-down, each node turns its scatter factor sigma~ into
//                    those of its children: Q_node [sigma~; 0];
//   5. leaf apply    Y_tile = Q_tile [sigma~; 0] = [sigma~; 0] - V (T V_1^T sigma~)
//                    (V_1 = the tile's top s x s reflector block): one
//                    n x s by s x s product, with the Gram Y^T Y fused.
// Every sum runs in a fixed order, so the result is bitwise reproducible for
// a given n, s and device.
#include "bk_common.cuh"
#include "bk_internal.h"
#include "bk_hh.cuh"
#include "bk_quad.cuh"

namespace bk {

constexpr int kTT = 256;                 // threads per TSQR CTA

// Rows per leaf tile: 256 threads x RPT rows each, RPT = 64 / next_pow2(s),
// i.e. 64 row values per thread, except FP64 blocks of width <= 4, which keep
// 32 values (measured on a 128^3 BCG iteration against 32 values: s = 32
// 37.5 -> 33.9 ms, s = 16 and 8 about 1.5 % faster, s = 4 3 % slower).
// Larger tiles also shrink the tree.
constexpr int leaf_rpt(int sw, int elem_bytes) { return (elem_bytes == 8 && sw <= 4 ? 32 : 64) / sw; }
inline int leaf_tile_rows(int s, int elem_bytes) { return kTT * leaf_rpt(next_pow2_s(s), elem_bytes); }

TsqrPlan tsqr_plan(int64_t n, int s, int elem_bytes) {
  TsqrPlan p;
  p.n = n; p.s = s; p.tile = leaf_tile_rows(s, elem_bytes);
  p.fanin = p.tile / s;
  p.rows[0] = n;
  int l = 0;
  for (;;) {
    const int tl = (l == 0) ? p.tile : kTT;     // tree levels: one row per thread
    p.nodes[l] = (p.rows[l] + tl - 1) / tl;
    if (p.nodes[l] <= 1 || l == 15) break;
    p.rows[l + 1] = p.nodes[l] * s;       // the stacked R factors of level l
    ++l;
  }
  p.levels = l;
  size_t b = 0;
  for (int i = 0; i <= p.levels; ++i) b += 2 * sizeof(double) * (size_t)p.nodes[i] * s * s + 512;
  p.bytes = b + 256;
  return p;
}

struct TsqrPtrs {
  double* R[16];       // stacked R factors of level l (later: the scatter factors sigma~)
  double* Tf[16];      // WY factors T of the tiles of level l
};

static TsqrPtrs tsqr_ptrs(const TsqrPlan& p, void* scratch) {
  TsqrPtrs q{};
  char* c = (char*)scratch;
  const int s = p.s;
  for (int i = 0; i <= p.levels; ++i) {
    q.R[i] = (double*)c; c += (sizeof(double) * (size_t)p.nodes[i] * s * s + 255) & ~(size_t)255;
    q.Tf[i] = (double*)c; c += (sizeof(double) * (size_t)p.nodes[i] * s * s + 255) & ~(size_t)255;
  }
  return q;
}

__device__ __forceinline__ bool tsqr_skip(const int* done, const int* flag) {
  return (done && *done) || (flag && !*flag);
}

// Sum the V-vector v over the 32 lanes of a warp by recursive halving: after
// log2(V) exchange steps every lane holds one component, whose index it
// returns; the remaining steps add that component over the lanes that share
// it.  V (a power of two <= 32) shuffles instead of 5 V.
template <int V, typename A>
__device__ __forceinline__ int warp_reduce_scatter(A (&v)[V]) {
  const int lane = threadIdx.x & 31;
  int comp = 0;
  int len = V;
#pragma unroll
  for (int o = 16, step = 0; (1 << step) < V; o >>= 1, ++step) {
    const int half = V >> (step + 1);
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const A send = upper ? v[i] : v[i + half];
      const A recv = __shfl_xor_sync(0xffffffffu, send, o);
      v[i] = (upper ? v[i + half] : v[i]) + recv;
    }
    if (upper) comp += half;
    len = half;
  }
  (void)len;
#pragma unroll
  for (int o = 16 / V; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  return comp;
}

// ---- 1. leaf factor -------------------------------------------------------------
// Thread t owns tile rows t, t + 256, ... in registers (RPT rows of
// next_pow2(s) values); the column loop is unrolled so every register index is
// a compile-time constant.  Column j of the Householder QR needs one CTA vector
// sum: q[c] = sum_{g > j} M[g][j] M[g][c] for every c (q[j] is the squared
// norm below the diagonal).  With alpha = M[j][j]:
//   beta = -sign(alpha) sqrt(alpha^2 + q[j]),  tau = (beta - alpha) / beta,
//   scale = 1 / (alpha - beta),  v_g = scale M[g][j] (g > j), v_j = 1;
//   v^T M[:, c] = scale q[c] + M[j][c]:
//     c > j: w_c = tau (scale q[c] + M[j][c]), trailing update M[g][c] -= w_c v_g;
//     c < j: y_c = scale q[c] + M[j][c] = V[:, c]^T v_j.
// The compact WY form H_0 ... H_{s-1} = I - V T V^T has T upper triangular
// with T^{-1} = diag(1 / tau) + strict_upper(V^T V), so the tile stores
// F = strict_upper(V^T V) + diag(tau) (entry (c, j) = y_c, (j, j) = tau_j)
// and never forms T: the apply solves with T^{-1} instead (tile_w).  This
// keeps the column loop free of the serial T recursion.  The scalars are
// computed once per column, by warp 0, and published in shared memory
// (on GB300's narrow FP64 pipe this beats every warp forming them itself).
template <typename TIn, typename T, int SW, int RPT>
__global__ void __launch_bounds__(kTT)
leaf_factor(int64_t n, int s, int ld, const TIn* __restrict__ X, TIn* __restrict__ Y, double* __restrict__ R0,
            double* __restrict__ T0, const int* done, const int* flag) {
  if (tsqr_skip(done, flag)) return;
  constexpr int tile = kTT * RPT;
  __shared__ double Tm[SW * SW];
  __shared__ T red_w[2][kWarps][SW];
  __shared__ T rowj[2][SW];
  __shared__ T wy[2][SW];
  __shared__ T sc[2][4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * tile;
  const int m = (int)((n - r0) < tile ? (n - r0) : tile);
  T row[RPT][SW];
  // FP32 tiles with s % 4 == 0 move their rows as float4 quads
  constexpr bool kVec = sizeof(TIn) == 4 && sizeof(T) == 4 && SW >= 4;
  const bool vec = kVec && (s % 4 == 0) && (ld % 4 == 0) &&
                   ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15) == 0;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int g = tid + k * kTT;
    if constexpr (kVec) {
      if (vec) {
#pragma unroll
        for (int qq = 0; qq < SW / 4; ++qq) {
          const float4 v = (g < m && 4 * qq < s) ? ld4((const float*)X + (r0 + g) * ld + 4 * qq) : zero4();
          row[k][4 * qq] = v.x; row[k][4 * qq + 1] = v.y; row[k][4 * qq + 2] = v.z; row[k][4 * qq + 3] = v.w;
        }
        continue;
      }
    }
#pragma unroll
    for (int c = 0; c < SW; ++c) row[k][c] = (g < m && c < s) ? (T)X[(r0 + g) * ld + c] : T(0);
  }
  for (int i = tid; i < SW * SW; i += kTT) Tm[i] = 0.0;
#pragma unroll
  for (int j = 0; j < SW; ++j) {
    if (j >= s) break;
    const int par = j & 1;
    T q[SW];
#pragma unroll
    for (int c = 0; c < SW; ++c) {
      q[c] = T(0);
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int g = tid + k * kTT;
        if (g > j) q[c] = fma(row[k][j], row[k][c], q[c]);
      }
    }
    if (tid == j) {
#pragma unroll
      for (int c = 0; c < SW; ++c) rowj[par][c] = row[0][c];
    }
    const int comp = warp_reduce_scatter<SW, T>(q);
    if ((lane & (32 / SW - 1)) == 0) red_w[par][warp][comp] = q[0];
    __syncthreads();
    if (warp == 0) {
      T qc = T(0);
      if (lane < SW) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) qc += red_w[par][w][lane];
      }
      const T tail = __shfl_sync(0xffffffffu, qc, j);
      const T alpha = rowj[par][j];
      T beta, tj, scale;
      if (tail == T(0)) { tj = T(0); beta = alpha; scale = T(0); }
      else {
        const T nrm = sqrt(alpha * alpha + tail);
        beta = alpha >= T(0) ? -nrm : nrm;
        tj = (beta - alpha) / beta;
        scale = T(1) / (alpha - beta);
      }
      if (lane < SW) {
        const T vc = fma(scale, qc, rowj[par][lane]);       // v^T M[:, lane]
        wy[par][lane] = tj * vc;                            // read for lane > j only
        if (lane < j) Tm[lane * SW + j] = (double)vc;       // V_lane^T v_j
        else if (lane == j) Tm[j * SW + j] = (double)tj;    // tau_j
      }
      if (lane == 0) { sc[par][0] = beta; sc[par][1] = tj; sc[par][2] = scale; }
    }
    __syncthreads();
    const T tj = sc[par][1];
    if (tj != T(0)) {
      const T scale = sc[par][2];
      T v[RPT];
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int g = tid + k * kTT;
        if (g > j) { row[k][j] *= scale; v[k] = row[k][j]; }
        else v[k] = (g == j) ? T(1) : T(0);
      }
#pragma unroll
      for (int c = j + 1; c < SW; ++c) {
        const T w = wy[par][c];
#pragma unroll
        for (int k = 0; k < RPT; ++k) row[k][c] = fma(-w, v[k], row[k][c]);
      }
    }
    if (tid == j) row[0][j] = sc[par][0];
  }
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int g = tid + k * kTT;
    if (g < m) {
      if constexpr (kVec) {
        if (vec) {
#pragma unroll
          for (int qq = 0; qq < SW / 4; ++qq)
            if (4 * qq < s)
              st4((float*)Y + (r0 + g) * ld + 4 * qq,
                  make_float4(row[k][4 * qq], row[k][4 * qq + 1], row[k][4 * qq + 2], row[k][4 * qq + 3]));
          continue;
        }
      }
#pragma unroll
      for (int c = 0; c < SW; ++c) if (c < s) Y[(r0 + g) * ld + c] = (TIn)row[k][c];
    }
  }
  double* Rb = R0 + (size_t)blockIdx.x * s * s;
  if (tid < s) {
#pragma unroll
    for (int c = 0; c < SW; ++c) if (c < s) Rb[tid * s + c] = (c >= tid) ? (double)row[0][c] : 0.0;
  }
  __syncthreads();
  double* Tb = T0 + (size_t)blockIdx.x * s * s;
  for (int i = tid; i < s * s; i += kTT) Tb[i] = Tm[(i / s) * SW + (i % s)];
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

// ---- 5. leaf apply ----------------------------------------------------------------
// Y_tile = [sigma~; 0] - V W with W = T (V_1^T sigma~): V is the tile's unit
// lower trapezoidal reflector block (stored below the diagonal in Y, implicit
// unit diagonal, zero above), V_1 its top s x s block.
//
// (a) tile_w: one CTA per tile forms W (s x s, FP64) and stores it over the
// tile's factor F.
template <typename T>
__global__ void __launch_bounds__(kTT)
tile_w(int64_t n, int s, int ld, int tile, const T* __restrict__ Y, const double* __restrict__ S0,
       double* __restrict__ TW, const int* done, const int* flag) {
  if (tsqr_skip(done, flag)) return;
  __shared__ double Sg[kMM], Tt[kMM], Zm[kMM], V1[kMM];
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * tile;
  const int m = (int)((n - r0) < tile ? (n - r0) : tile);
  for (int i = tid; i < s * s; i += kTT) {
    const int a = i / s, c = i - a * s;
    Sg[a * kMaxS + c] = S0[(size_t)blockIdx.x * s * s + i];
    Tt[a * kMaxS + c] = TW[(size_t)blockIdx.x * s * s + i];
    V1[a * kMaxS + c] = (c == a) ? 1.0 : ((c < a && a < m) ? (double)Y[(r0 + a) * ld + c] : 0.0);
  }
  __syncthreads();
  for (int i = tid; i < s * s; i += kTT) {          // Z = V_1^T sigma~
    const int a = i / s, c = i - a * s;
    double acc = 0.0;
    for (int g = a; g < s; ++g) acc = fma(V1[g * kMaxS + a], Sg[g * kMaxS + c], acc);
    Zm[a * kMaxS + c] = acc;
  }
  __syncthreads();
  // W = T Z, i.e. T^{-1} W = Z with T^{-1} = diag(1 / tau) + strict_upper(V^T V):
  // back substitution W[a] = tau_a (Z[a] - sum_{b > a} (V^T V)[a][b] W[b]),
  // exact also for tau_a = 0 (then row a and column a of T vanish)
  double* Wm = Sg;                                   // sigma~ is no longer needed
  __syncthreads();
  for (int c = tid; c < s; c += kTT) {
    for (int a = s - 1; a >= 0; --a) {
      double acc = Zm[a * kMaxS + c];
      for (int b = a + 1; b < s; ++b) acc = fma(-Tt[a * kMaxS + b], Wm[b * kMaxS + c], acc);
      Wm[a * kMaxS + c] = Tt[a * kMaxS + a] * acc;
    }
  }
  __syncthreads();
  for (int i = tid; i < s * s; i += kTT) TW[(size_t)blockIdx.x * s * s + i] = Wm[(i / s) * kMaxS + (i % s)];
}

// (a') the same for FP32 leaf tiles, in FP32 arithmetic: one warp per tile,
// lane c forms column c of Z = V_1^T sigma~ and of W (registers).
template <typename TIn, int SW>
__global__ void __launch_bounds__(kThreads)
tile_w_f32(int64_t n, int s, int ld, int tile, int64_t tiles, const TIn* __restrict__ Y,
           const double* __restrict__ S0, double* __restrict__ TW, const int* done, const int* flag) {
  if (tsqr_skip(done, flag)) return;
  const int lane = threadIdx.x & 31;
  const int64_t tl = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (tl >= tiles) return;
  const int64_t r0 = tl * tile;
  const int m = (int)((n - r0) < tile ? (n - r0) : tile);
  const double* S = S0 + (size_t)tl * s * s;
  double* F = TW + (size_t)tl * s * s;
  const int c = lane;
  const bool cok = c < s;
  float sig[SW], w[SW];
#pragma unroll
  for (int g = 0; g < SW; ++g) sig[g] = (g < s && cok) ? (float)S[g * s + c] : 0.f;
  float z[SW];
#pragma unroll
  for (int a = 0; a < SW; ++a) {            // Z[a][c] = sum_{g >= a} V_1[g][a] sigma~[g][c]
    float acc = 0.f;
#pragma unroll
    for (int g = a; g < SW; ++g) {
      const float v = (g >= s || a >= s) ? 0.f
                    : (g == a ? 1.f : (g < m ? (float)Y[(r0 + g) * ld + a] : 0.f));
      acc = fmaf(v, sig[g], acc);
    }
    z[a] = acc;
  }
#pragma unroll
  for (int a = SW - 1; a >= 0; --a) {       // W[a] = tau_a (Z[a] - sum_{b > a} F[a][b] W[b])
    if (a >= s) { w[a] = 0.f; continue; }
    float acc = z[a];
#pragma unroll
    for (int b = a + 1; b < SW; ++b)
      if (b < s) acc = fmaf(-(float)F[a * s + b], w[b], acc);
    w[a] = (float)F[a * s + a] * acc;
  }
  __syncwarp();                             // every lane has read F before W overwrites it
  if (cok) {
#pragma unroll
    for (int a = 0; a < SW; ++a)
      if (a < s) F[a * s + c] = (double)w[a];
  }
}

// (b) apply_rows: every warp takes a contiguous chunk of rows (two row groups
// per trip), so consecutive trips stay inside one tile and lane c keeps
// column c of that tile's W in registers.  Lane c computes Y[r][c]; the Gram
// Y^T Y (upper, mirrored) is accumulated in the same pass when rho_out is given.
template <typename TIn, typename T, int SW>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? (SW >= 32 ? 2 : 4) : 1)
apply_rows(int64_t n, int s, int ld, int tile_shift, TIn* __restrict__ Y, const double* __restrict__ S0,
           const double* __restrict__ W, double* rho_out, double* gpart, unsigned* counter,
           const int* done, const int* flag) {
  if (tsqr_skip(done, flag)) return;
  extern __shared__ double smem_d[];
  constexpr int RPW = 32 / SW;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = lane & (SW - 1), rs = lane / SW;
  const bool want_rho = rho_out != nullptr;
  constexpr bool kPair = (sizeof(T) == 8) && (SW >= 2);
  const int cnt = ut_count(s);
  double* part = smem_d;
  double* scratch = smem_d + cnt + 1;
  double* lacc = scratch + kWarps * (cnt > 2 ? cnt : 2);
  double acc[SW];
#pragma unroll
  for (int a = 0; a < SW; ++a) acc[a] = 0.0;
  T acc_t[SW];
#pragma unroll
  for (int a = 0; a < SW; ++a) acc_t[a] = T(0);
  SymGramPair<kPair ? SW : 2> pg;
  pg.zero();
  int since = 0;
  if constexpr (sizeof(T) == 4) {
    if (want_rho)
      for (int a = 0; a < lacc_stride(SW); ++a) lacc[tid * lacc_stride(SW) + a] = 0.0;
  }
  // contiguous chunk of this warp, a multiple of 2 * RPW rows
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gwarp = (int64_t)blockIdx.x * kWarps + warp;
  int64_t chunk = (n + nwarps - 1) / nwarps;
  chunk = (chunk + 2 * RPW - 1) / (2 * RPW) * (2 * RPW);
  const int64_t lo = gwarp * chunk;
  const int64_t hi = (lo + chunk < n) ? lo + chunk : n;
  const int64_t tmask = ((int64_t)1 << tile_shift) - 1;
  int64_t cur_tile = -1;
  T wcol[SW];
#pragma unroll
  for (int a = 0; a < SW; ++a) wcol[a] = T(0);
  // a trip (2 * RPW rows starting at a multiple of 2 * RPW) never straddles a
  // tile (tiles are powers of two >= 256 rows), so the tile is warp-uniform
  auto do_row = [&](int64_t r, int64_t tl) -> T {
    const int g = (int)(r & tmask);
    const bool ok = (r < hi) && (c < s);
    T v = T(0), y = T(0);
    if (ok) {
      v = (g < s) ? (c == g ? T(1) : (c < g ? (T)Y[r * ld + c] : T(0))) : (T)Y[r * ld + c];
      if (g < s) y = (T)S0[(size_t)tl * s * s + g * s + c];
    }
#pragma unroll
    for (int a = 0; a < SW; ++a) {
      const T va = sw_bcast<SW>(v, a);
      y = fma(-va, wcol[a], y);
    }
    if (ok) Y[r * ld + c] = (TIn)y;
    return ok ? y : T(0);
  };
  auto accum_row = [&](T yv) {
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int a = 0; a < SW; ++a) {
        const T ya = sw_bcast<SW>(yv, a);
        if (a <= c) acc[a] = fma((double)ya, (double)yv, acc[a]);
      }
    } else {
#pragma unroll
      for (int a = 0; a < SW; ++a) {
        const T ya = sw_bcast<SW>(yv, a);
        if (a <= c) acc_t[a] = fma(ya, yv, acc_t[a]);
      }
      if (++since == kF32Window) {
        lacc_flush<SW>(lacc, acc_t);
        since = 0;
      }
    }
  };
  for (int64_t base = lo; base < hi; base += 2 * RPW) {
    const int64_t tl = base >> tile_shift;
    if (tl != cur_tile) {
      cur_tile = tl;
#pragma unroll
      for (int a = 0; a < SW; ++a)
        wcol[a] = (a < s && c < s) ? (T)W[(size_t)tl * s * s + a * s + c] : T(0);
    }
    const T yA = do_row(base + rs, tl);
    const T yB = do_row(base + RPW + rs, tl);
    if (want_rho) {
      if constexpr (kPair) pg.add((double)yA, (double)yA, (double)yB, (double)yB);
      else { accum_row(yA); accum_row(yB); }
    }
  }
  if (!want_rho) return;
  if constexpr (sizeof(T) == 4) {
    lacc_flush<SW>(lacc, acc_t);
    __syncthreads();
    lacc_reduce<SW>(lacc, s, true, part);
  } else if constexpr (kPair) {
    pg.cta_reduce(s, scratch, part);
  } else {
    cta_reduce_gram<SW>(acc, s, true, scratch, part);
  }
  if (!grid_reduce_last(part, cnt, gpart, counter)) return;
  unpack_gram(part, s, true, rho_out);
}

// (b') the same apply for FP32 blocks with s % 4 == 0 in the quad layout:
// lane (row, quad i) forms Y[r][4i .. 4i + 3]; the warp stages its rows of V
// and keeps the current tile's W (float, row stride SW) in shared memory; the
// Gram Y^T Y accumulates in 4 x 4 register blocks.  Same terms, same order
// as apply_rows for every output.
template <int SW>
__global__ void __launch_bounds__(kThreads, 2)
apply4(int64_t n, int s, int ld, int tile_shift, float* __restrict__ Y, const double* __restrict__ S0,
       const double* __restrict__ W, double* rho_out, double* gpart, unsigned* counter,
       const int* done, const int* flag) {
  if (tsqr_skip(done, flag)) return;
  using S = QuadShape<SW>;
  extern __shared__ double smem_d[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qi = lane % S::LPR, rho = lane / S::LPR;
  const bool qok = 4 * qi < s;
  const bool want_rho = rho_out != nullptr;
  const int cnt = ut_count(s);
  const GramPtrs<SW> sp(smem_d, cnt);
  // extra: per warp the tile's W (SW = 32) and the staged V rows
  float* ws = sp.extra + warp * (SW * SW + S::STAGE);
  float* stv = ws + SW * SW;
  GramOf<SW> g;
  if (want_rho) g.init(sp.slots);
  // contiguous chunk of this warp, a multiple of RW rows; a trip never
  // straddles a tile (tiles are powers of two >= 256 rows)
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gwarp = (int64_t)blockIdx.x * kWarps + warp;
  int64_t chunk = (n + nwarps - 1) / nwarps;
  chunk = (chunk + S::RW - 1) / S::RW * S::RW;
  const int64_t lo = gwarp * chunk;
  const int64_t hi = (lo + chunk < n) ? lo + chunk : n;
  const int64_t tmask = ((int64_t)1 << tile_shift) - 1;
  int64_t cur_tile = -1;
  // SW <= 16: the lane's four columns of W in registers, rows by shuffles;
  // SW = 32: W in shared memory, rows staged
  constexpr bool kRegW = SW <= 16;
  float4 cf[kRegW ? SW : 1];
  for (int64_t base = lo; base < hi; base += S::RW) {
    const int64_t tl = base >> tile_shift;
    if (tl != cur_tile) {
      cur_tile = tl;
      if constexpr (kRegW) {
        load_coef<SW>(cf, W + (size_t)tl * s * s, s, s, qi);
      } else {
        __syncwarp();
        for (int i = lane; i < SW * SW; i += 32) {
          const int a = i / SW, c = i % SW;
          ws[i] = (a < s && c < s) ? (float)W[(size_t)tl * s * s + a * s + c] : 0.f;
        }
        __syncwarp();
      }
    }
    const int64_t r = base + rho;
    const int gr = (int)(r & tmask);
    const bool ok = (r < hi) && qok;
    float4 v = ok ? ld4(Y + r * ld + 4 * qi) : zero4();
    float4 y = zero4();
    if (ok && gr < s) {
      // top rows of the tile: V = unit lower triangle there; [sigma~; 0] term
      const double* sg = S0 + (size_t)tl * s * s + (size_t)gr * s + 4 * qi;
      float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int a = 4 * qi + t;
        vv[t] = (a == gr) ? 1.f : (a < gr ? vv[t] : 0.f);
      }
      v = make_float4(vv[0], vv[1], vv[2], vv[3]);
      y = make_float4((float)sg[0], (float)sg[1], (float)sg[2], (float)sg[3]);
    }
    if constexpr (kRegW) {
      // y + sum_a (-v_a) w_a: the same roundings as y = fma(-v_a, w_a, y)
      y = row_times<SW>(make_float4(-v.x, -v.y, -v.z, -v.w), cf, y);
      if (ok) st4(Y + r * ld + 4 * qi, y);
    } else {
      st4(stv + rho * SW + 4 * qi, v);
      __syncwarp();
#pragma unroll 4
      for (int k = 0; k < S::NQ; ++k) {
        const float4 vk = ld4(stv + rho * SW + 4 * k);
#pragma unroll
        for (int t = 0; t < 4; ++t) y = fma4(-comp4(vk, t), ld4(ws + (4 * k + t) * SW + 4 * qi), y);
      }
      if (ok) st4(Y + r * ld + 4 * qi, y);
      __syncwarp();
    }
    if (want_rho) {
      const float4 yy = ok ? y : zero4();
      g.row(yy, yy, sp.stl, sp.stl);
    }
  }
  if (!want_rho) return;
  g.cta_reduce(s, true, sp.slots, sp.part, sp.stl, sp.stl);
  if (!grid_reduce_last(sp.part, cnt, gpart, counter)) return;
  unpack_gram(sp.part, s, true, rho_out);
}

template <int SW>
static cudaError_t launch_apply4(const Launch& L, int64_t rows, int s, int ld, int shift, float* Y,
                                 const double* Rst, const double* Tf, double* rho_out, double* gpart,
                                 unsigned* counter, const int* done, const int* flag) {
  auto k = apply4<SW>;
  const int cnt = ut_count(s);
  const size_t sm = gram_smem_bytes<SW>(cnt, (size_t)kWarps * (SW * SW + QuadShape<SW>::STAGE));
  cudaError_t err = cudaSuccess;
  const int occ = quad_occupancy(k, sm, &err);
  if (!occ) return err;
  k<<<quad_grid(L, occ, rows, QuadShape<SW>::RW), kThreads, sm, L.stream>>>(
      rows, s, ld, shift, Y, Rst, Tf, rho_out, gpart, counter, done, flag);
  return cudaGetLastError();
}

template <typename K>
static cudaError_t set_smem(K kern, size_t bytes) {
  if (bytes <= 44 * 1024) return cudaSuccess;   // 48 KB default includes static buffers
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// TIn: storage of the tiles (the block's type at level 0, double in the tree);
// T: arithmetic (the block's precision at every level).
template <typename TIn, typename T, int SW, int RPT>
static cudaError_t launch_leaves(const Launch& L, int64_t rows, int s, int ld, int64_t tiles,
                                 const TIn* X, TIn* Y, double* Rst, double* Tf, double* rho_out,
                                 double* gpart, unsigned* counter, const int* done, const int* flag,
                                 bool factor) {
  if (factor) {
    leaf_factor<TIn, T, SW, RPT><<<(unsigned)tiles, kTT, 0, L.stream>>>(rows, s, ld, X, Y, Rst, Tf, done,
                                                                        flag);
    return cudaGetLastError();
  }
  const int tile = kTT * RPT;
  if constexpr (sizeof(T) == 4) {
    tile_w_f32<TIn, SW><<<(unsigned)((tiles + kWarps - 1) / kWarps), kThreads, 0, L.stream>>>(
        rows, s, ld, tile, tiles, Y, Rst, Tf, done, flag);
  } else {
    tile_w<TIn><<<(unsigned)tiles, kTT, 0, L.stream>>>(rows, s, ld, tile, Y, Rst, Tf, done, flag);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int shift = 0;
  while ((1 << shift) < tile) ++shift;
  if constexpr (sizeof(TIn) == 4 && sizeof(T) == 4 && SW >= 4) {
    // the quad layout needs 16-byte aligned rows
    if (s % 4 == 0 && ld % 4 == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0)
      return launch_apply4<SW>(L, rows, s, ld, shift, Y, Rst, Tf, rho_out, gpart, counter, done, flag);
  }
  const int cnt = ut_count(s);
  const size_t lanes = (sizeof(T) == 4) ? (size_t)kThreads * lacc_stride(SW) : 0;
  const size_t sm = sizeof(double) * (cnt + 1 + kWarps * (cnt > 2 ? cnt : 2) + lanes) + 64;
  auto k = apply_rows<TIn, T, SW>;
  if ((e = set_smem(k, sm)) != cudaSuccess) return e;
  int64_t grid = (rows + 2 * kWarps - 1) / (2 * kWarps);
  const int64_t cap = (int64_t)L.sms * kCtasPerSm;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  k<<<(unsigned)grid, kThreads, sm, L.stream>>>(rows, s, ld, shift, Y, Rst, Tf, rho_out, gpart,
                                                 counter, done, flag);
  return cudaGetLastError();
}

// Level 0 tiles hold leaf_rpt rows per thread; the tree levels (stacked R
// factors, few rows) use one row per thread so that more CTAs share the work.
template <typename TIn, typename T>
static cudaError_t leaves(const Launch& L, int64_t rows, int s, int ld, int64_t tiles, const TIn* X,
                          TIn* Y,
                          double* Rst, double* Tf, double* rho_out, double* gpart, unsigned* counter,
                          const int* done, const int* flag, bool factor, bool bottom) {
#define BK_LEAVES(SWV)                                                                                 \
  return bottom ? launch_leaves<TIn, T, SWV, leaf_rpt(SWV, sizeof(T))>(L, rows, s, ld, tiles, X, Y,   \
                                                                      Rst, Tf, rho_out, gpart,        \
                                                                      counter, done, flag, factor)    \
                : launch_leaves<TIn, T, SWV, 1>(L, rows, s, ld, tiles, X, Y, Rst, Tf, rho_out, gpart,  \
                                                counter, done, flag, factor)
  switch (next_pow2_s(s)) {
    case 1: BK_LEAVES(1);
    case 2: BK_LEAVES(2);
    case 4: BK_LEAVES(4);
    case 8: BK_LEAVES(8);
    case 16: BK_LEAVES(16);
    case 32: BK_LEAVES(32);
    default: return cudaErrorInvalidValue;
  }
#undef BK_LEAVES
}

// Launches of one TSQR: a factor launch per level, the root's sign fix, and per level an
// apply of two launches (the WY product W = T (V1^T sigma~), then the rows).
int tsqr_launches(const TsqrPlan& p) { return 3 * (p.levels + 1) + 1; }

// X = Y gamma (Y may alias X).  Level 0 tiles the n x s block; level l + 1
// tiles the stacked R factors of level l (stored in FP64, factored in the
// block's precision: an FP32 block's leaf R factors carry FP32 rounding, so
// an FP64 tree would add nothing but FP64 work) until one tile remains,
// whose R is the root (sign fix in FP64).  The scatter factors then travel down: the apply of level l
// turns the sigma~ of its tiles into the stacked sigma~ of level l - 1.
template <typename T>
cudaError_t tsqr(const Launch& L, const TsqrPlan& p, const T* X, T* Y, double* gamma_out,
                 double* rho_out, void* scratch, double* gpart, unsigned* counter, const int* done,
                 const int* flag, int ld) {
  const int s = p.s;
  if (ld <= 0) ld = s;
  if (ld < s) return cudaErrorInvalidValue;
  TsqrPtrs q = tsqr_ptrs(p, scratch);
  cudaError_t e;
  if (rho_out && !counter) return cudaErrorInvalidValue;
  prof_begin(L, kPhTsqrLeaf);
  if ((e = leaves<T, T>(L, p.n, s, ld, p.nodes[0], X, Y, q.R[0], q.Tf[0], nullptr, nullptr, nullptr,
                        done, flag, true, true)) != cudaSuccess) return e;
  prof_end(L, kPhTsqrLeaf, 1);
  prof_begin(L, kPhTsqrTree);
  for (int l = 1; l <= p.levels; ++l)
    if ((e = leaves<double, T>(L, p.rows[l], s, s, p.nodes[l], q.R[l - 1], q.R[l - 1], q.R[l], q.Tf[l],
                               nullptr, nullptr, nullptr, done, flag, true, false)) != cudaSuccess) return e;
  root_fix<<<1, 256, 0, L.stream>>>(s, q.R[p.levels], gamma_out, done, flag);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int l = p.levels; l >= 1; --l)
    if ((e = leaves<double, T>(L, p.rows[l], s, s, p.nodes[l], nullptr, q.R[l - 1], q.R[l], q.Tf[l],
                               nullptr, nullptr, nullptr, done, flag, false, false)) != cudaSuccess) return e;
  prof_end(L, kPhTsqrTree, 3 * p.levels + 1);
  prof_begin(L, kPhTsqrApply);
  e = leaves<T, T>(L, p.n, s, ld, p.nodes[0], nullptr, Y, q.R[0], q.Tf[0], rho_out, gpart, counter,
                   done, flag, false, true);
  prof_end(L, kPhTsqrApply, 2);
  return e;
}

// Row tiles factored on their own (the local normaliser of the localized
// Arnoldi method): every leaf tile t of X gets its Householder QR X_t = Q_t R_t;
// Y_t = Q_t (explicit, s orthonormal columns on the tile) and R_t goes to
// Rloc + t * ldr (s x s, row-major).  No tree: the level-0 scatter factors
// are set to the identity before the apply.
__global__ void tile_r_out(int64_t tiles, int s, double* __restrict__ Rst, double* __restrict__ Rloc,
                           int64_t ldr) {
  const int64_t ss = (int64_t)s * s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tiles * ss;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = i / ss;
    const int e = (int)(i % ss);
    Rloc[t * ldr + e] = Rst[i];
    Rst[i] = (e / s == e % s) ? 1.0 : 0.0;
  }
}

cudaError_t tsqr_local_q(const Launch& L, const TsqrPlan& p, const double* X, double* Y, double* Rloc,
                         int64_t ldr, void* scratch) {
  const int s = p.s;
  TsqrPtrs q = tsqr_ptrs(p, scratch);
  cudaError_t e;
  if ((e = leaves<double, double>(L, p.n, s, s, p.nodes[0], X, Y, q.R[0], q.Tf[0], nullptr, nullptr,
                                  nullptr, nullptr, nullptr, true, true)) != cudaSuccess) return e;
  int64_t g = (p.nodes[0] * s * s + 255) / 256;
  if (g > (int64_t)L.sms * 8) g = (int64_t)L.sms * 8;
  tile_r_out<<<(unsigned)(g < 1 ? 1 : g), 256, 0, L.stream>>>(p.nodes[0], s, q.R[0], Rloc, ldr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return leaves<double, double>(L, p.n, s, s, p.nodes[0], nullptr, Y, q.R[0], q.Tf[0], nullptr, nullptr,
                                nullptr, nullptr, nullptr, false, true);
}

template cudaError_t tsqr<double>(const Launch&, const TsqrPlan&, const double*, double*, double*,
                                  double*, void*, double*, unsigned*, const int*, const int*, int);
template cudaError_t tsqr<float>(const Launch&, const TsqrPlan&, const float*, float*, double*,
                                 double*, void*, double*, unsigned*, const int*, const int*, int);

}  // namespace bk
