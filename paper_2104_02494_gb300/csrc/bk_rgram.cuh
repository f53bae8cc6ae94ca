// FP32 block inner products L^T M (Ch. 3.3, BDOT) with one row per lane, for the
// pipelined kernels whose operands sit in shared memory in rows of s = SW floats
// (SW = 4, 8, 16), written by swizzled tensor copies.
//
// Swizzle: a stage of rows of SW floats is copied with the 32-, 64- or 128-byte
// swizzle whose span is one row (SW = 8, 16, 32; none for SW = 4, whose 16-byte
// rows are already bank-distinct): the 16-byte chunk q of row r lies at chunk
// q ^ ((r >> shift) & mask) of that row.  Eight lanes reading one logical chunk
// of eight consecutive rows then touch eight different bank groups.
//
// Gram blocks: the s x s Gram in 4 x 4 blocks (aq, cq) (the upper triangle aq <=
// cq when symmetric) is split into NCLS classes of at most MB blocks; a warp
// computes the blocks of one class for the rows it is given, each lane one row at
// a time, with every block index a compile-time constant.
//
// Precision: a lane's products go into an FP32 accumulator for at most W1 rows,
// then into a second FP32 level for at most W2 such windows, then the warp's 32
// lanes are added by a fixed shuffle tree (5 levels) and lane 0 adds the result
// into the warp's FP64 slots; CTA and grid sums are FP64 in a fixed order.  Every
// entry is within (W1 - 1 + W2 - 1 + 5) 2^-24 sum_r |L_ra M_rc| = 33 2^-24 of the
// exact sum (W1 = W2 = 15).
#pragma once

#include "bk_ops.cuh"

namespace bk {

template <int SW>
struct Swz {
  // chunk q of row r of a stage (the stage base 1024-byte aligned)
  static constexpr int kMask = SW == 32 ? 7 : (SW == 16 ? 3 : (SW == 8 ? 1 : 0));
  static constexpr int kShift = SW == 32 ? 0 : (SW == 16 ? 1 : 2);
  __device__ __forceinline__ static int chunk(int r, int q) { return q ^ ((r >> kShift) & kMask); }
  __device__ __forceinline__ static const float* at(const float* base, int r, int q) {
    return base + r * SW + 4 * chunk(r, q);
  }
  __device__ __forceinline__ static float* at(float* base, int r, int q) { return base + r * SW + 4 * chunk(r, q); }
  // For rows r = 32 g + lane the swizzle bits of r are those of the lane: the
  // float offset of chunk q within the row is a per-lane constant.
  __device__ __forceinline__ static int lane_off(int lane, int q) { return 4 * chunk(lane, q); }
};

// A class's blocks packed 4 bits each (aq in bits 0-1, cq in bits 2-3), block 0 lowest.
__host__ __device__ constexpr uint64_t blk4(int aq, int cq, int b) { return (uint64_t)(aq | (cq << 2)) << (4 * b); }

template <int SW, bool kSym>
struct GramClasses;
template <> struct GramClasses<4, true> {
  static constexpr int NCLS = 1, MB = 1;
  __host__ __device__ static constexpr int nb(int) { return 1; }
  __host__ __device__ static constexpr uint64_t code(int) { return blk4(0, 0, 0); }
};
template <> struct GramClasses<4, false> : GramClasses<4, true> {};
template <> struct GramClasses<8, true> {
  static constexpr int NCLS = 1, MB = 3;
  __host__ __device__ static constexpr int nb(int) { return 3; }
  __host__ __device__ static constexpr uint64_t code(int) { return blk4(0, 0, 0) | blk4(0, 1, 1) | blk4(1, 1, 2); }
};
template <> struct GramClasses<8, false> {
  static constexpr int NCLS = 1, MB = 4;
  __host__ __device__ static constexpr int nb(int) { return 4; }
  __host__ __device__ static constexpr uint64_t code(int) {
    return blk4(0, 0, 0) | blk4(0, 1, 1) | blk4(1, 0, 2) | blk4(1, 1, 3);
  }
};
template <> struct GramClasses<16, true> {
  static constexpr int NCLS = 3, MB = 4;
  __host__ __device__ static constexpr int nb(int c) { return c == 0 ? 4 : 3; }
  __host__ __device__ static constexpr uint64_t code(int c) {
    return c == 0 ? blk4(0, 0, 0) | blk4(0, 1, 1) | blk4(1, 1, 2) | blk4(0, 2, 3)
           : c == 1 ? blk4(1, 2, 0) | blk4(2, 2, 1) | blk4(0, 3, 2)
                    : blk4(1, 3, 0) | blk4(2, 3, 1) | blk4(3, 3, 2);
  }
};
template <> struct GramClasses<16, false> {
  static constexpr int NCLS = 3, MB = 6;
  __host__ __device__ static constexpr int nb(int c) { return c == 0 ? 6 : 5; }
  __host__ __device__ static constexpr uint64_t code(int c) {
    return c == 0 ? blk4(0, 0, 0) | blk4(0, 1, 1) | blk4(0, 2, 2) | blk4(0, 3, 3) | blk4(1, 0, 4) | blk4(1, 1, 5)
           : c == 1 ? blk4(1, 2, 0) | blk4(1, 3, 1) | blk4(2, 0, 2) | blk4(2, 1, 3) | blk4(2, 2, 4)
                    : blk4(2, 3, 0) | blk4(3, 0, 1) | blk4(3, 1, 2) | blk4(3, 2, 3) | blk4(3, 3, 4);
  }
};
template <class C>
__host__ __device__ constexpr int blk_aq(int c, int b) { return (int)((C::code(c) >> (4 * b)) & 3); }
template <class C>
__host__ __device__ constexpr int blk_cq(int c, int b) { return (int)((C::code(c) >> (4 * b + 2)) & 3); }

// Accumulators of one class CLS (compile time) for one lane.
template <int SW, bool kSym, int CLS>
struct RowGram2 {
  using C = GramClasses<SW, kSym>;
  static constexpr int NB = C::nb(CLS);
  static constexpr int kWarpDoubles = C::MB * 16;   // FP64 slots per warp
  static constexpr int W1 = 15, W2 = 15;
  float a1[NB][16];
  float a2[NB][16];
  int n1, n2;
  double* ws;

  __device__ __forceinline__ void init(double* warp_slots) {
    ws = warp_slots;
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < kWarpDoubles; i += 32) ws[i] = 0.0;
    __syncwarp();
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int e = 0; e < 16; ++e) { a1[b][e] = 0.f; a2[b][e] = 0.f; }
    n1 = n2 = 0;
  }
  __device__ __forceinline__ void to_fp64() {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        float v = a2[b][e];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        a2[b][e] = 0.f;
        if (lane == 0) ws[b * 16 + e] += (double)v;
      }
    __syncwarp();
  }
  __device__ __forceinline__ void flush1() {
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int e = 0; e < 16; ++e) { a2[b][e] += a1[b][e]; a1[b][e] = 0.f; }
    n1 = 0;
    if (++n2 == W2) {
      to_fp64();
      n2 = 0;
    }
  }
  // one row: l[q], m[q] the row's quads of the left and the right operand
  __device__ __forceinline__ void row(const float4 (&l)[SW / 4], const float4 (&m)[SW / 4]) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const float4 a = l[blk_aq<C>(CLS, b)];
      const float4 c = m[blk_cq<C>(CLS, b)];
      const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        a1[b][4 * t + 0] = fmaf(av[t], c.x, a1[b][4 * t + 0]);
        a1[b][4 * t + 1] = fmaf(av[t], c.y, a1[b][4 * t + 1]);
        a1[b][4 * t + 2] = fmaf(av[t], c.z, a1[b][4 * t + 2]);
        a1[b][4 * t + 3] = fmaf(av[t], c.w, a1[b][4 * t + 3]);
      }
    }
    if (++n1 == W1) flush1();
  }
  __device__ __forceinline__ void finish() {
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int e = 0; e < 16; ++e) { a2[b][e] += a1[b][e]; a1[b][e] = 0.f; }
    to_fp64();
  }
};

// CTA sum of the warps' FP64 slots (warp w computed class w % NCLS) into part: the
// packed upper triangle (kSym) or s x s.  After a CTA barrier; any number of threads.
template <int SW, bool kSym>
__device__ void row_gram_sum(int s, const double* slots, int nwarps, double* part) {
  using C = GramClasses<SW, kSym>;
  const int cnt = kSym ? ut_count(s) : s * s;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    int a, c;
    if (kSym) {
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
      const int cls = w % C::NCLS;
      for (int b = 0; b < C::nb(cls); ++b)
        if (blk_aq<C>(cls, b) == aq && blk_cq<C>(cls, b) == cq) t += slots[(size_t)w * C::MB * 16 + b * 16 + e];
    }
    part[i] = t;
  }
  __syncthreads();
}

}  // namespace bk
