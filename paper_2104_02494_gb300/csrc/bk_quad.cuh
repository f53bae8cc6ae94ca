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
// Precision: each lane sums 16 rows in float registers, adds that window
// into its own float slot in shared memory, and the slots of all lanes,
// warps and CTAs are added in double, in a fixed order (bitwise
// reproducible for a given grid).
#pragma once

#include <mutex>
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
  static constexpr int TPF = RPL >= 16 ? 1 : 16 / RPL;  // trips per 16-row register window
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

}  // namespace bk
