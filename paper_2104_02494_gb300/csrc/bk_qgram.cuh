// FP32 block inner products L^T M (Ch. 3.3, BDOT) on CUDA-core FMAs for the
// pipelined kernels, whose left operand L is already in shared memory.
//
// Quad layout: a row of s floats is LPR = SW / 4 quads; a warp holds 32 lanes =
// (32 / LPR) row slots x LPR quads, and every lane handles one pair of rows per
// step (r0 in the first half of the step's rows, r1 in the second half).
//
// Symmetric Gram (kPair): the upper triangle in 4 x 4 blocks (aq, cq), aq <= cq.
// Lane quad q has the pair class p = min(q, LPR - 1 - q); it owns the column
// quad q of r0 and the column quad LPR - 1 - q of r1, i.e. one row with column
// quad p ("low row") and one with column quad LPR - 1 - p ("high row").  Its
// LPR + 1 accumulator slots are
//   slot k <= p:  block (k, p)          from the low row,
//   slot k >  p:  block (k - p - 1, LPR - 1 - p) from the high row,
// (q + 1) + (LPR - q) = LPR + 1 blocks per lane and row pair, the same for every
// lane; over the pair classes every block (aq <= cq) has exactly one slot.
// Full Gram (!kPair): lane quad q owns blocks (k, q), k < LPR, of both rows.
//
// Precision: every product goes into an FP32 accumulator for at most W1 row
// pairs, then (for SW <= 16) into a second FP32 level for at most W2 such
// windows, then the warp adds its lanes by a fixed shuffle tree (L levels) and
// one lane adds the result into the warp's FP64 slots; CTA and grid sums are
// FP64 in a fixed order.  With at most W1 products per level-1 window and W2
// windows per level-2 sum, every entry is within (W1 - 1 + W2 - 1 + L) 2^-24
// sum_r |L_ra M_rc| of the exact sum: at most 33 2^-24 (W1 <= 15, W2 = 15,
// L <= 5; SW = 32: W1 <= 28 in one level, L <= 3: 30 2^-24).
#pragma once

#include "bk_ops.cuh"

namespace bk {

template <int SW, bool kPair>
struct QuadGram {
  static constexpr int LPR = SW / 4;                         // quads (lanes) per row
  static constexpr int RS = 32 / LPR;                        // row slots per warp
  static constexpr int NSLOT = kPair ? (LPR == 1 ? 2 : LPR + 1) : LPR;
  static constexpr int NCLS = kPair ? (LPR == 1 ? 1 : LPR / 2) : LPR;   // lane classes
  static constexpr bool kTwo = SW <= 16;                     // second FP32 level
  static constexpr int kStep = kPair ? 1 : 2;                // products per entry and add()
  static constexpr int W1 = (kTwo ? 15 : 28) / kStep;        // add() calls per level-1 window
  static constexpr int W2 = 15;
  static constexpr int kWarpDoubles = NCLS * NSLOT * 16;     // FP64 slots per warp

  float a1[NSLOT][16];
  float a2[kTwo ? NSLOT : 1][kTwo ? 16 : 1];
  int n1, n2;
  int cls;        // pair class p (kPair) or column quad q
  bool high;      // kPair: the lane's r0 is the high row
  double* ws;     // this warp's FP64 slots [NCLS][NSLOT][16]

  __device__ __forceinline__ void zero1() {
#pragma unroll
    for (int k = 0; k < NSLOT; ++k)
#pragma unroll
      for (int e = 0; e < 16; ++e) a1[k][e] = 0.f;
  }
  // warp_slots: kWarpDoubles doubles of this warp (zeroed here, warp-wide).
  __device__ __forceinline__ void init(double* warp_slots) {
    const int lane = threadIdx.x & 31, q = lane % LPR;
    cls = kPair ? (q < LPR - 1 - q ? q : LPR - 1 - q) : q;
    high = kPair && LPR > 1 && q > LPR - 1 - q;
    ws = warp_slots;
    for (int i = lane; i < kWarpDoubles; i += 32) ws[i] = 0.0;
    __syncwarp();
    zero1();
    if constexpr (kTwo) {
#pragma unroll
      for (int k = 0; k < NSLOT; ++k)
#pragma unroll
        for (int e = 0; e < 16; ++e) a2[k][e] = 0.f;
    }
    n1 = 0;
    n2 = 0;
  }

  // Warp sum of acc over the lanes of the same class (fixed shuffle tree), added
  // in FP64 by the class's lane of row slot 0; acc is zeroed.
  template <int NS>
  __device__ __forceinline__ void to_fp64(float (&acc)[NS][16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        float v = acc[k][e];
#pragma unroll
        for (int off = LPR; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if constexpr (kPair && LPR > 1) v += __shfl_xor_sync(0xffffffffu, v, LPR - 1);
        acc[k][e] = v;
      }
    const int q = lane % LPR;
    if (lane < LPR && (!kPair || q == cls)) {
      double* w = ws + cls * NSLOT * 16;
#pragma unroll
      for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int e = 0; e < 16; ++e) w[k * 16 + e] += (double)acc[k][e];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[k][e] = 0.f;
  }

  __device__ __forceinline__ void flush1() {
    if constexpr (kTwo) {
#pragma unroll
      for (int k = 0; k < NSLOT; ++k)
#pragma unroll
        for (int e = 0; e < 16; ++e) a2[k][e] += a1[k][e];
      zero1();
      if (++n2 == W2) {
        to_fp64(a2);
        n2 = 0;
      }
    } else {
      to_fp64(a1);
    }
    n1 = 0;
  }

  __device__ __forceinline__ static void outer(float (&acc)[16], const float4& l, const float4& m) {
    const float lv[4] = {l.x, l.y, l.z, l.w};
    const float2 mlo = make_float2(m.x, m.y), mhi = make_float2(m.z, m.w);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 aa = make_float2(lv[t], lv[t]);
      const float2 lo = fma2(aa, mlo, make_float2(acc[4 * t + 0], acc[4 * t + 1]));
      const float2 hi = fma2(aa, mhi, make_float2(acc[4 * t + 2], acc[4 * t + 3]));
      acc[4 * t + 0] = lo.x; acc[4 * t + 1] = lo.y;
      acc[4 * t + 2] = hi.x; acc[4 * t + 3] = hi.y;
    }
  }

  // One row pair, called by all 32 lanes.  l0, l1: the left rows of r0 and r1 in
  // shared memory (s floats each; any readable row when the row is absent, whose
  // right quad is then zero); m0, m1: the lane's right quads of r0 (quad q) and r1
  // (quad LPR - 1 - q for kPair, q otherwise), zero for absent rows and for
  // columns >= s.  Left quads at columns >= s count as zero.
  __device__ __forceinline__ void add(const float* l0, const float* l1, const float4& m0, const float4& m1, int s) {
    if constexpr (kPair) {
      const float* lo = high ? l1 : l0;
      const float* hi = high ? l0 : l1;
      const float4 mlo = high ? m1 : m0, mhi = high ? m0 : m1;
#pragma unroll
      for (int k = 0; k < NSLOT; ++k) {
        const bool first = LPR == 1 ? k == 0 : k <= cls;
        const int aq = first ? k : (LPR == 1 ? 0 : k - cls - 1);
        float4 a = zero4();
        if (4 * aq < s) a = ld4((first ? lo : hi) + 4 * aq);
        outer(a1[k], a, first ? mlo : mhi);
      }
    } else {
#pragma unroll
      for (int k = 0; k < NSLOT; ++k) {
        float4 a0 = zero4(), b0 = zero4();
        if (4 * k < s) {
          a0 = ld4(l0 + 4 * k);
          b0 = ld4(l1 + 4 * k);
        }
        outer(a1[k], a0, m0);
        outer(a1[k], b0, m1);
      }
    }
    if (++n1 == W1) flush1();
  }

  // Flush every level into the warp's FP64 slots (all 32 lanes).
  __device__ __forceinline__ void finish() {
    if constexpr (kTwo) {
#pragma unroll
      for (int k = 0; k < NSLOT; ++k)
#pragma unroll
        for (int e = 0; e < 16; ++e) a2[k][e] += a1[k][e];
      to_fp64(a2);
    } else {
      to_fp64(a1);
    }
  }

  // CTA sum (after every warp's finish and a CTA barrier; any number of threads) of
  // the nwarps warps' slots into part: the packed upper triangle (sym) or s x s.
  __device__ static void sum(int s, bool sym, const double* slots, int nwarps, double* part) {
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
      const int aq = a / 4, cq = c / 4, e = 4 * (a % 4) + (c % 4);
      double t = 0.0;
      for (int w = 0; w < nwarps; ++w) {
        const double* ws = slots + (size_t)w * kWarpDoubles;
        if constexpr (kPair) {
          if (LPR == 1) {
            t += ws[0 * 16 + e];
            t += ws[1 * 16 + e];
          } else if (cq < LPR / 2) {
            t += ws[(cq * NSLOT + aq) * 16 + e];
          } else {
            const int p = LPR - 1 - cq;
            t += ws[(p * NSLOT + aq + p + 1) * 16 + e];
          }
        } else {
          t += ws[(cq * NSLOT + aq) * 16 + e];
        }
      }
      part[i] = t;
    }
    __syncthreads();
  }
};

}  // namespace bk
