// Vectorised FP32 row layout ("quad layout") for blocks whose width s is a
// multiple of 4.  A row of s floats is s/4 float4 quads.  In the row phase
// every lane owns one quad: LPR = SW/4 lanes per row, RW = 32/LPR rows per
// warp per trip, so one warp instruction moves 512 contiguous bytes.
//
// Block inner products L^T M (Ch. 3.3, BDOT) are accumulated as 4 x 4
// register blocks: the warp stages its RW rows of both operands in shared
// memory, then lane (b, g) adds the outer products of Gram block b over the
// staged rows g, g + G, g + 2G, ...  A lane therefore keeps 16 (s = 32: 32)
// float accumulators instead of one per Gram column, and every staged value
// is read with 16-byte shared-memory loads.
//
// Precision: each lane sums 32 rows in float registers, adds that window
// into its own float slot in shared memory, and the slots of all lanes,
// warps and CTAs are added in double, in a fixed order (bitwise
// reproducible for a given grid).
#pragma once

#include <mutex>
#include <type_traits>
#include <vector>

#include "bk_internal.h"
#include "bk_ops.cuh"

namespace bk {

// Q = A P (or sub - A P) with an optional fused Gram, FP32 quad layout
// (s % 4 == 0, no Frobenius sums); bk_quad.cu.
template <class RowOp>
cudaError_t spmm4(const Launch& L, const RowOp& op, int64_t n, int s, const float* in, float* out,
                  const float* sub, const Epi<float>& ep);

// CTAs per SM the quad kernels are compiled for (register cap 255 / 85 / 128).
template <int SW>
constexpr int quad_min_ctas() { return SW >= 32 ? 2 : 3; }

// Resident CTAs per SM of a kernel at a given dynamic shared memory (capped
// at kCtasPerSm, the grid-partials budget), cached per device, kernel and
// shared-memory size; the dynamic shared-memory attribute is set on first use.
struct OccEntry {
  int dev;
  const void* kern;
  size_t smem;
  int occ;
};

template <typename K>
inline int quad_occupancy(K kern, size_t smem, cudaError_t* err) {
  static std::mutex g_occ_mu;
  static std::vector<OccEntry> g_occ;
  int dev = 0;
  if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return 0;
  const void* key = reinterpret_cast<const void*>(kern);
  std::lock_guard<std::mutex> lock(g_occ_mu);
  for (const OccEntry& e : g_occ)
    if (e.dev == dev && e.kern == key && e.smem == smem) return e.occ;
  // static shared memory counts against the 48 KB default too: always opt in
  if (smem > 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { *err = e; return 0; }
  }
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
  if (e != cudaSuccess) { *err = e; return 0; }
  if (occ < 1) occ = 1;
  if (occ > kCtasPerSm) occ = kCtasPerSm;
  g_occ.push_back({dev, key, smem, occ});
  return occ;
}

inline int quad_grid(const Launch& L, int occ, int64_t n, int rw) {
  const int64_t rows_per_cta = (int64_t)rw * kWarps;
  int64_t need = (n + rows_per_cta - 1) / rows_per_cta;
  const int64_t cap = (int64_t)L.sms * occ;
  if (need > cap) need = cap;
  return (int)(need < 1 ? 1 : need);
}

template <int SW>
struct QuadShape {
  static_assert(SW >= 4 && SW <= 32, "the quad layout needs 4 <= SW <= 32");
  static constexpr int NQ = SW / 4;                 // quads per row
  static constexpr int LPR = NQ;                    // lanes per row (row phase)
  static constexpr int RW = 32 / LPR;               // rows per warp per trip
  static constexpr int NB = NQ * NQ;                // 4 x 4 blocks of an SW x SW Gram
  static constexpr int NBL = NB > 32 ? NB / 32 : 1; // blocks per lane
  static constexpr int G = NB >= 32 ? 1 : 32 / NB;  // lanes sharing one block (row groups)
  static constexpr int RPL = RW / G;                // staged rows per lane per trip
  static constexpr int STAGE = RW * SW;             // floats of one staged operand per warp
  static constexpr int TPF = RPL >= 32 ? 1 : 32 / RPL;  // trips per 32-row register window
  static constexpr int NACC = 16 * NBL;             // float accumulators per lane
};

__device__ __forceinline__ float comp4(const float4& v, int t) {
  return t == 0 ? v.x : (t == 1 ? v.y : (t == 2 ? v.z : v.w));
}

// Stage an s x s control-block matrix (double, row stride 32) as float with
// row stride SW, zero beyond s, so that row a, columns 4i .. 4i + 3 is one
// aligned float4.
template <int SW>
__device__ inline void stage_quad_matrix(float* dst, const double* src, int s) {
  for (int i = threadIdx.x; i < SW * SW; i += blockDim.x) {
    const int a = i / SW, c = i % SW;
    dst[i] = (a < s && c < s) ? (float)src[a * kMaxS + c] : 0.f;
  }
}

template <int SW>
struct QuadGram {
  using S = QuadShape<SW>;
  float acc[S::NBL][16];
  int trips;
  float* slot;   // this thread's level-2 slots: slot[e * kThreads]

  __device__ __forceinline__ void init(float* l2) {
#pragma unroll
    for (int m = 0; m < S::NBL; ++m)
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[m][e] = 0.f;
    trips = 0;
    slot = l2 + threadIdx.x;
#pragma unroll
    for (int e = 0; e < S::NACC; ++e) slot[e * kThreads] = 0.f;
  }

  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int m = 0; m < S::NBL; ++m)
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        slot[(m * 16 + e) * kThreads] += acc[m][e];
        acc[m][e] = 0.f;
      }
    trips = 0;
  }

  // Outer products of the warp's staged rows: stl holds the left operand,
  // stm the right one (RW rows of SW floats each; may be the same buffer).
  __device__ __forceinline__ void trip(const float* stl, const float* stm) {
    const int lane = threadIdx.x & 31;
    const int b0 = S::NB >= 32 ? lane : lane % S::NB;
    const int g = S::NB >= 32 ? 0 : lane / S::NB;
#pragma unroll
    for (int k = 0; k < S::RPL; ++k) {
      const int rr = g + k * S::G;
#pragma unroll
      for (int m = 0; m < S::NBL; ++m) {
        const int b = b0 + 32 * m;
        const int bi = b / S::NQ, bj = b % S::NQ;
        const float4 a = ld4(stl + rr * SW + 4 * bi);
        const float4 q = ld4(stm + rr * SW + 4 * bj);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float at = comp4(a, t);
          acc[m][4 * t + 0] = fmaf(at, q.x, acc[m][4 * t + 0]);
          acc[m][4 * t + 1] = fmaf(at, q.y, acc[m][4 * t + 1]);
          acc[m][4 * t + 2] = fmaf(at, q.z, acc[m][4 * t + 2]);
          acc[m][4 * t + 3] = fmaf(at, q.w, acc[m][4 * t + 3]);
        }
      }
    }
    if (++trips == S::TPF) flush();
  }

  // CTA sums of entry (a, c) for a <= c (sym, packed by ut_index) or all
  // (a, c) (row-major), in double, into part[0 .. cnt).  Every thread of the
  // CTA calls this; l2 is the CTA's slot array.
  __device__ void cta_reduce(int s, bool sym, const float* l2, double* part) {
    flush();
    __syncthreads();
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
      const int b = (a / 4) * S::NQ + c / 4, e = (a % 4) * 4 + (c % 4);
      const int m = S::NB >= 32 ? b / 32 : 0;
      const int lb = S::NB >= 32 ? b % 32 : b;
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w)
        for (int g = 0; g < S::G; ++g)
          t += (double)l2[(m * 16 + e) * kThreads + w * 32 + lb + g * S::NB];
      part[i] = t;
    }
    __syncthreads();
  }
};

// Shared-memory floats of the Gram machinery: per-warp staging of two
// operands plus the level-2 slots.
template <int SW>
constexpr size_t quad_gram_floats() {
  return (size_t)kWarps * 2 * QuadShape<SW>::STAGE + (size_t)QuadShape<SW>::NACC * kThreads;
}

// Quad k of the calling lane's row: the LPR lanes of a row exchange their
// quads by shuffles (s shuffles per lane for the whole row).
template <int SW>
__device__ __forceinline__ float4 row_quad(const float4& mine, int k) {
  constexpr int LPR = QuadShape<SW>::LPR;
  if constexpr (LPR == 1) {
    return mine;
  } else {
    return make_float4(__shfl_sync(0xffffffffu, mine.x, k, LPR), __shfl_sync(0xffffffffu, mine.y, k, LPR),
                       __shfl_sync(0xffffffffu, mine.z, k, LPR), __shfl_sync(0xffffffffu, mine.w, k, LPR));
  }
}

// Row-owner Gram for SW <= 16: lane (row, quad i) adds L[r][a] M[r][4i + t]
// for every a (the row's L quads arrive by shuffles) into SW x 4 float
// accumulators: no shared-memory traffic per row.  Windows of kRowWin rows
// per lane go to float slots in shared memory; the CTA sums are in double.
template <int SW>
struct RowGram {
  using S = QuadShape<SW>;
  static_assert(SW <= 16, "RowGram keeps SW x 4 accumulators per lane");
  static constexpr int kRowWin = 32;
  float acc[SW][4];
  int rows;
  float* slot;   // slot[(a * 4 + t) * kThreads]

  __device__ __forceinline__ void init(float* l2) {
#pragma unroll
    for (int a = 0; a < SW; ++a)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[a][t] = 0.f;
    rows = 0;
    slot = l2 + threadIdx.x;
#pragma unroll
    for (int e = 0; e < 4 * SW; ++e) slot[e * kThreads] = 0.f;
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int a = 0; a < SW; ++a)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        slot[(a * 4 + t) * kThreads] += acc[a][t];
        acc[a][t] = 0.f;
      }
    rows = 0;
  }
  // l, m: this lane's quads of the current row (zero for rows past n)
  __device__ __forceinline__ void row(const float4& l, const float4& m) {
#pragma unroll
    for (int k = 0; k < S::NQ; ++k) {
      const float4 lk = row_quad<SW>(l, k);
#pragma unroll
      for (int t2 = 0; t2 < 4; ++t2) {
        const float la = comp4(lk, t2);
        float* r = acc[4 * k + t2];
        r[0] = fmaf(la, m.x, r[0]);
        r[1] = fmaf(la, m.y, r[1]);
        r[2] = fmaf(la, m.z, r[2]);
        r[3] = fmaf(la, m.w, r[3]);
      }
    }
    if (++rows == kRowWin) flush();
  }
  __device__ void cta_reduce(int s, bool sym, const float* l2, double* part) {
    flush();
    __syncthreads();
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
      const int qi = c / 4, t = c % 4;
      double sum = 0.0;
      for (int w = 0; w < kWarps; ++w)
        for (int rr = 0; rr < S::RW; ++rr)
          sum += (double)l2[(a * 4 + t) * kThreads + w * 32 + rr * S::LPR + qi];
      part[i] = sum;
    }
    __syncthreads();
  }
  static constexpr size_t smem_floats() { return (size_t)4 * SW * kThreads; }
};

// The block Gram with the staging interface of RowGram: row(l, m, stl, stm)
// stages the lane's quads and adds the warp's trip (used for SW = 32).
template <int SW>
struct StagedGram : QuadGram<SW> {
  using S = QuadShape<SW>;
  __device__ __forceinline__ void row(const float4& l, const float4& m, float* stl, float* stm) {
    const int lane = threadIdx.x & 31;
    const int qi = lane % S::LPR, rho = lane / S::LPR;
    st4(stl + rho * SW + 4 * qi, l);
    if (stm != stl) st4(stm + rho * SW + 4 * qi, m);
    __syncwarp();
    this->trip(stl, stm);
    __syncwarp();
  }
  static constexpr size_t smem_floats() { return quad_gram_floats<SW>(); }
};

template <int SW>
struct RowGramStaged : RowGram<SW> {
  __device__ __forceinline__ void row(const float4& l, const float4& m, float*, float*) {
    RowGram<SW>::row(l, m);
  }
};

// Columns 4i .. 4i + 3 of an s x s double matrix (row stride ld), every row a
// < SW, as floats in registers (zero beyond s): 4 SW registers.
template <int SW>
__device__ __forceinline__ void load_coef(float4 (&cf)[SW], const double* M, int s, int ld, int qi) {
#pragma unroll
  for (int a = 0; a < SW; ++a) {
    float v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int c = 4 * qi + t;
      v[t] = (a < s && c < s) ? (float)M[a * ld + c] : 0.f;
    }
    cf[a] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// acc + sum_a row[a] cf[a] over the quads of the lane's row (a ascending).
template <int SW>
__device__ __forceinline__ float4 row_times(const float4& mine, const float4 (&cf)[SW], float4 acc) {
#pragma unroll
  for (int k = 0; k < QuadShape<SW>::NQ; ++k) {
    const float4 rk = row_quad<SW>(mine, k);
#pragma unroll
    for (int t = 0; t < 4; ++t) acc = fma4(comp4(rk, t), cf[4 * k + t], acc);
  }
  return acc;
}

// Gram policy per width: shuffles for SW <= 8 (at most 32 accumulators),
// staged 4 x 4 blocks for 16 and 32 (16 or 32 accumulators).
template <int SW>
using GramOf = typename std::conditional<(SW <= 8), RowGramStaged<SW>, StagedGram<SW>>::type;

}  // namespace bk
