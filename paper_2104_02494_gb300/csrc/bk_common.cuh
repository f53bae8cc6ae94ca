// Internal definitions shared by the bkrylov CUDA sources (sm_103a).
//
// Thread mapping used by every row-local kernel on an n x s row-major block:
// a warp is split into 32/SW "sub-warps" of SW = next_pow2(s) lanes; one
// sub-warp owns one row and lane c < s owns column c.  A warp therefore
// touches 32/SW consecutive rows = one contiguous span of memory, and the s
// values of a row can be exchanged with __shfl_sync(width = SW).  Loops over
// rows advance a whole warp at a time so that every lane of the warp takes
// part in every shuffle.
#pragma once

#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "../../include/bkrylov.h"

namespace bk {

constexpr int kMaxS = BKRYLOV_MAX_S;   // 32
constexpr int kThreads = 256;          // threads per CTA of the row kernels
constexpr int kWarps = kThreads / 32;
// CTAs per SM launched by the row kernels (8 x 256 threads = full residency),
// so that enough loads are in flight to cover HBM latency.
constexpr int kCtasPerSm = 8;

// CTAs of a kThreads-thread kernel with `smem` dynamic bytes that stay resident on one SM
// (its registers and shared memory decide), at most kCtasPerSm.  A grid-stride kernel
// launched with sms x this many CTAs runs as one full wave: a compute-bound kernel
// loses no partial last wave.
template <class K>
inline int resident_ctas(K kern, size_t smem) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    occ = 0;
  }
  return occ < 1 ? 1 : (occ > kCtasPerSm ? kCtasPerSm : occ);
}

// ---- per-solve device control block --------------------------------------------
// s x s matrices are stored with row stride kMaxS: M[i][j] at i * kMaxS + j.
enum : int { kDoneRunning = 0, kDoneConverged = 1, kDoneStopped = 2 };
enum : int { kCntA = 0, kCntB = 1, kCntC = 2, kCntD = 3, kNumCounters = 8 };
// Ticket words behind every grid-reduction counter (zero on entry, zero again on exit):
// word 0 the final ticket, word 1 + g the ticket of CTA group g.
constexpr int kTicketWords = 128;
constexpr int kGroupCtas = 16;
constexpr int kMM = kMaxS * kMaxS;

struct Ctrl {
  int done;          // kDone*
  int status;        // bkrylov_status
  int iter;          // completed iterations
  int reorths;
  int reortho_now;   // decision of the current iteration
  int maxit;
  int s;
  int n_forced;
  int sub_p;         // block size of S_BP^p (s: the block case S_B)
  int has_prec;      // BCG with a preconditioner M^{-1} (rho_m carries rho)
  int one_r;         // BCG with one reduction (Alg. "1R-CG"): alpha from delta
  int norm_mode;     // stopping measure: 0 max_i ||R_i|| / ||R0_i||, 1 ||R||_F / ||R0||_F
  int qr_fast;       // CholeskyQR2 normaliser of this iteration: 0 not taken (declined or no
                     // re-orthonormalisation), 1 taken, 2 second factor failed (TSQR of Y1)
  int tsqr_now;      // the Householder TSQR runs in this iteration
  int cholqr_count;  // re-orthonormalisations normalised by CholeskyQR2
  int replace_every; // 1R-BCG: form Q = A P and alpha = <P, Q> after every m-th iteration
  int replace_now;   // ... after this iteration (set by the small kernel)
  int replacements;
  double tol;
  double eta;
  double eps;        // machine epsilon of the working precision
  double omega;      // BBiCGStab scalar
  double frob[4];    // Frobenius sums (BBiCGStab: <U,S>, <U,U>)
  unsigned counters[kNumCounters][kTicketWords];   // grid-reduction tickets
  double n0[kMaxS];      // ||R0_i||
  double relres[kMaxS];
  double alpha[kMM];     // BCG alpha = P^T Q        | BBiCGStab R0s^T Q
  double rho[kMM];       // BCG rho   = Rb^T Rb      | BBiCGStab R^T R (kappa_D, norms)
  double rho_new[kMM];   // BCG: R-bar^T R-bar of the new residual block (Euclidean)
  double rho_m[kMM];     // BCG with M: <Z, R-bar> = R-bar^T M^{-1} R-bar
  double delta[kMM];     // 1R-BCG: <Z, U> = Z^T A Z
  double sigma[kMM];
  double gamma[kMM];     // normalizer R factor of the last TSQR (diag >= 0)
  double lam[kMM];       // lambda
  double lx[kMM];        // lambda sigma  (X update)
  double beta[kMM];
  double g2[kMM];        // BBiCGStab R0s^T R
  double g3[kMM];        // BBiCGStab R0s^T U
  double lu[kMM];        // BBiCGStab LU factors of R0s^T Q
  double sigma_new[kMM]; // BBiCGStab sigma^{k+1}
  double cq_u1[kMM];     // CholeskyQR2: first upper Cholesky factor U1 (G1 = U1^T U1)
  double cq_inv[kMM];    // CholeskyQR2: inverse of the factor of the current pass
  int piv[kMaxS];
  double nb[kMaxS];      // refinement: ||B_i||
};

// ---- division by a loop-invariant integer ---------------------------------------
// Unsigned 32-bit division by an invariant divisor d >= 1 with one high
// multiply (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Fig. 4.1): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1,  q = (t + ((x - t) >> sh1)) >> sh2,
// t = mulhi(m, x), sh1 = min(l, 1), sh2 = max(l - 1, 0); exact for all 32-bit x.
struct FastDiv {
  uint32_t d = 1, m = 1, sh1 = 0, sh2 = 0;
  FastDiv() = default;
  __host__ explicit FastDiv(uint32_t div) : d(div) {
    uint32_t l = 0;
    while ((1ull << l) < div) ++l;
    m = (uint32_t)((((1ull << 32) * ((1ull << l) - div)) / div) + 1);
    sh1 = l < 1 ? l : 1;
    sh2 = l > 0 ? l - 1 : 0;
  }
  __device__ __forceinline__ uint32_t div(uint32_t x) const {
    const uint32_t t = __umulhi(m, x);
    return (t + ((x - t) >> sh1)) >> sh2;
  }
};

// ---- small helpers --------------------------------------------------------------
__host__ __device__ inline int next_pow2_s(int s) {
  int w = 1;
  while (w < s) w <<= 1;
  return w;
}

template <int SW, typename T>
__device__ __forceinline__ T sw_bcast(T v, int src) {
  return __shfl_sync(0xffffffffu, v, src, SW);
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// Upper-triangle packed index of (a, c), a <= c.
__host__ __device__ inline int ut_index(int a, int c) { return c * (c + 1) / 2 + a; }
__host__ __device__ inline int ut_count(int s) { return s * (s + 1) / 2; }

// ---- deterministic grid reduction ----------------------------------------------
// Sums gpart[(first + k * step) * cnt + j] over k < count into part[j] (shared memory)
// in a fixed order: R chunks of k per output (R = blockDim / cnt, at most 8, R * cnt at
// most kThreads), the chunk sums then added in chunk order.  Ends with a CTA barrier.
__device__ inline void sum_slots(double* part, int cnt, const double* gpart, int first, int step,
                                 int count) {
  __shared__ double s_acc[kThreads];
  int R = (int)blockDim.x / cnt;
  if (R > 8) R = 8;
  if (R * cnt > kThreads) R = kThreads / cnt;
  if (R >= 2) {
    double acc = 0.0;
    const int i = threadIdx.x % cnt;
    const int q = threadIdx.x / cnt;
    if (q < R) {
      const int k0 = (int)((long long)count * q / R), k1 = (int)((long long)count * (q + 1) / R);
#pragma unroll 4
      for (int k = k0; k < k1; ++k) acc += ldcg(gpart + (size_t)(first + k * step) * cnt + i);
      s_acc[threadIdx.x] = acc;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
      for (int k = 0; k < R; ++k) t += s_acc[k * cnt + threadIdx.x];
      part[threadIdx.x] = t;
    }
  } else {
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      double t = 0.0;
#pragma unroll 4
      for (int k = 0; k < count; ++k) t += ldcg(gpart + (size_t)(first + k * step) * cnt + j);
      part[j] = t;
    }
  }
  __syncthreads();
}

// Below this many partial values one level is faster: the second level adds a fence
// and an atomic round trip (measured on GB300: 152 CTAs x 36 values 8.2 us per launch
// with one level, 9.2 with two; 152 x 136: 15.4 / 10.2; 152 x 528: 41.0 / 16.4).
constexpr long long kTreeMinValues = 8192;

// Every CTA stores its `cnt` partial sums (already reduced inside the CTA, in
// shared memory `part`) to gpart[blockIdx.x * cnt + i].  One level: the last CTA
// to arrive (atomic ticket) sums the partials of CTA 0, 1, 2, ... in fixed chunks.
// Two levels, for large grids x cnt: the last CTA of each group of kGroupCtas
// consecutive CTAs sums its group's partials (in CTA order) into the slot of the
// group's first CTA, and the last group to finish sums the group sums in group
// order.  The last CTA's additions run on one SM's FP64 pipe (two per clock on
// GB300), so a single level of G x cnt additions is the cost the tree splits.
// Either way the order depends on the grid only: the result is bitwise
// reproducible for a given grid.  No thread ever waits for another CTA.
// Returns true in the last CTA only; the reduced values are then in `part`.
// `counter` points to kTicketWords words, zero on entry; the CTAs that use a
// word reset it for the next use.  kTree = false keeps one level (for kernels
// whose registers are at their cap, where the second level's state spills).
template <bool kTree = true>
__device__ inline bool grid_reduce_last(double* part, int cnt, double* gpart,
                                        unsigned* counter) {
  __shared__ unsigned s_ticket;
  const int G = gridDim.x;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) gpart[(size_t)blockIdx.x * cnt + i] = part[i];
  __threadfence();
  __syncthreads();
  const int ng = (G + kGroupCtas - 1) / kGroupCtas;
  const bool tree = kTree && ng >= 2 && ng < kTicketWords && (long long)G * cnt >= kTreeMinValues;
  // level 1 of the tree: this CTA's group; otherwise the whole grid
  const int g = tree ? (int)blockIdx.x / kGroupCtas : -1;
  int first = tree ? g * kGroupCtas : 0, step = 1;
  int count = tree ? ((G - first < kGroupCtas) ? G - first : kGroupCtas) : G;
  unsigned* ticket = counter + 1 + g;
  for (;;) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1u);
    __syncthreads();
    if (s_ticket != (unsigned)count - 1) return false;
    __threadfence();
    sum_slots(part, cnt, gpart, first, step, count);
    if (threadIdx.x == 0) *ticket = 0u;
    if (ticket == counter) break;
    // the group's sum replaces its first CTA's partial; then the ticket of the groups
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) gpart[(size_t)first * cnt + i] = part[i];
    __threadfence();
    __syncthreads();
    ticket = counter;
    first = 0;
    step = kGroupCtas;
    count = ng;
  }
  __syncthreads();
  return true;
}

// Reduce per-lane Gram accumulators of a CTA into shared memory.
// On entry lane c (< s) of every sub-warp holds acc[a] = partial of G[a][c].
// `sym`: only a <= c are meaningful; the packed upper triangle is produced.
// On exit part[0..cnt) holds the CTA's sums (cnt = ut_count(s) or s*s);
// `scratch` must hold kWarps * cnt doubles.
template <int SW>
__device__ inline void cta_reduce_gram(double (&acc)[SW], int s, bool sym, double* scratch,
                                       double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane & (SW - 1);
#pragma unroll
  for (int a = 0; a < SW; ++a) {
#pragma unroll
    for (int off = SW; off < 32; off <<= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], off);
  }
  const int cnt = sym ? ut_count(s) : s * s;
  if (lane < SW && c < s) {
#pragma unroll
    for (int a = 0; a < SW; ++a) {
      if (a < s && (!sym || a <= c)) scratch[warp * cnt + (sym ? ut_index(a, c) : a * s + c)] = acc[a];
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

// Symmetric Gram  l^T q  (upper triangle) of TWO rows per sub-warp, FP64,
// without idle lanes.  Lane c of a sub-warp (SW >= 2 lanes) holds column c
// of row A (la, qa) and of row B (lb, qb).  A row's upper triangle has
// SW(SW+1)/2 entries; lane cc = c mod SW/2 takes the column pair (cc, SW-1-cc),
// i.e. the entries (a, cc), a <= cc, and (a, SW-1-cc), a <= SW-1-cc: SW + 1
// entries, the same count for every lane.  Lanes c < SW/2 do this for row A,
// lanes c >= SW/2 for row B.  acc[t] is entry (t, cc) for t <= cc and
// (t - cc - 1, SW-1-cc) otherwise.  Columns >= s hold zeros in la/qa/lb/qb,
// so their entries vanish.
template <int SW>
struct SymGramPair {
  double acc[SW + 1];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int t = 0; t <= SW; ++t) acc[t] = 0.0;
  }
  __device__ __forceinline__ void add(double la, double qa, double lb, double qb) {
    const int c = threadIdx.x & (SW - 1);
    const bool hi = c >= SW / 2;
    const int cc = hi ? c - SW / 2 : c;
    const int c2 = SW - 1 - cc;
    const double q1a = __shfl_sync(0xffffffffu, qa, cc, SW), q1b = __shfl_sync(0xffffffffu, qb, cc, SW);
    const double q2a = __shfl_sync(0xffffffffu, qa, c2, SW), q2b = __shfl_sync(0xffffffffu, qb, c2, SW);
    const double q1 = hi ? q1b : q1a, q2 = hi ? q2b : q2a;
#pragma unroll
    for (int t = 0; t <= SW; ++t) {
      const bool first = t <= cc;
      const int a = first ? t : t - cc - 1;
      const double va = __shfl_sync(0xffffffffu, la, a, SW);
      const double vb = __shfl_sync(0xffffffffu, lb, a, SW);
      acc[t] = fma(hi ? vb : va, first ? q1 : q2, acc[t]);
    }
  }
  // CTA sum into the packed upper triangle part[0..s(s+1)/2); scratch holds
  // kWarps * s(s+1)/2 doubles.  Every entry with column < s is written by
  // exactly one lane of every warp.
  __device__ void cta_reduce(int s, double* scratch, double* part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t <= SW; ++t) {
      acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], SW / 2);
#pragma unroll
      for (int off = SW; off < 32; off <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], off);
    }
    const int cnt = ut_count(s);
    if (lane < SW / 2) {
      const int cc = lane, c2 = SW - 1 - lane;
#pragma unroll
      for (int t = 0; t <= SW; ++t) {
        const bool first = t <= cc;
        const int a = first ? t : t - cc - 1;
        const int col = first ? cc : c2;
        if (col < s) scratch[warp * cnt + ut_index(a, col)] = acc[t];
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
};

// FP32 Gram partials: every lane accumulates its column's products in float
// registers over a window of rows and then adds them into its own FP64 slots
// in shared memory, lacc[tid * lacc_stride(SW) + a] (no two lanes share a
// slot).  This keeps the FP64 work at 1/window of the products and the
// registers at SW floats per lane.
__host__ __device__ constexpr int lacc_stride(int SW) { return SW == 1 ? 1 : SW + 1; }
// rows per FP32 accumulation window: the float partial of one window carries a
// relative error of at most kF32Window * 2^-24; beyond it the sums are FP64.
constexpr int kF32Window = 64;
// CTAs per SM the row kernels are compiled for: FP32 instantiations are capped
// at 64 registers (4 CTAs of 256 threads) so that enough loads are in flight.
template <typename T> constexpr int min_ctas() { return sizeof(T) == 4 ? 4 : 1; }

template <int SW>
__device__ __forceinline__ void lacc_flush(double* lacc, float (&acc_t)[SW]) {
  double* mine = lacc + threadIdx.x * lacc_stride(SW);
#pragma unroll
  for (int a = 0; a < SW; ++a) { mine[a] += (double)acc_t[a]; acc_t[a] = 0.f; }
}

// CTA sum of the lacc slots into part[] (packed upper triangle when sym, else
// s x s row-major), in the fixed order warp 0..7, sub-warp 0..32/SW-1.
template <int SW>
__device__ void lacc_reduce(const double* lacc, int s, bool sym, double* part) {
  const int cnt = sym ? ut_count(s) : s * s;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    int a, c;
    if (sym) {
      c = 0;
      while ((c + 1) * (c + 2) / 2 <= i) ++c;
      a = i - c * (c + 1) / 2;
    } else {
      a = i / s;
      c = i - a * s;
    }
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w)
      for (int rs = 0; rs < 32 / SW; ++rs) t += lacc[(w * 32 + rs * SW + c) * lacc_stride(SW) + a];
    part[i] = t;
  }
  __syncthreads();
}

// Unpack a reduced Gram (packed upper or full s x s) into a ctrl-layout matrix.
__device__ inline void unpack_gram(const double* part, int s, bool sym, double* M) {
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    int a = i / s, c = i % s;
    double v;
    if (sym) v = (a <= c) ? part[ut_index(a, c)] : part[ut_index(c, a)];
    else v = part[i];
    M[a * kMaxS + c] = v;
  }
}

}  // namespace bk
