// Vectorised FP32 row layout ("quad layout") for blocks whose width s is a
// multiple of 4.  A row of s floats is s/4 float4 quads.  In the row phase
// every lane owns one quad: LPR = SW/4 lanes per row, RW = 32/LPR rows per
// warp per trip, so one warp instruction moves 512 contiguous bytes.
//
// Block inner products L^T M (Ch. 3.3, BDOT) fused into these kernels are a
// dense tall-skinny contraction and run on the tensor cores (MmaGram: TF32
// mma with the three-term split that keeps FP32 accuracy) for SW >= 8; for
// SW = 4 the row's quads are exchanged by shuffles (RowGram).
//
// Precision: partial sums are FP32 over windows of at most 32 rows per
// accumulator (then a second FP32 level), every partial beyond is added in
// double, and the CTA and grid sums run in a fixed order (bitwise
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
// shared-memory size.  The kernel's dynamic shared-memory limit is an
// attribute of the kernel, not of a launch: it is only ever raised (to the
// largest size requested so far), so that every cached size stays valid.
struct OccEntry {
  int dev;
  const void* kern;
  size_t smem;
  int occ;
};
struct AttrEntry {
  int dev;
  const void* kern;
  size_t smem_max;
};

template <typename K>
inline int quad_occupancy(K kern, size_t smem, cudaError_t* err) {
  static std::mutex g_occ_mu;
  static std::vector<OccEntry> g_occ;
  static std::vector<AttrEntry> g_attr;
  int dev = 0;
  if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return 0;
  const void* key = reinterpret_cast<const void*>(kern);
  std::lock_guard<std::mutex> lock(g_occ_mu);
  AttrEntry* at = nullptr;
  for (AttrEntry& a : g_attr)
    if (a.dev == dev && a.kern == key) at = &a;
  if (!at) {
    g_attr.push_back({dev, key, 0});
    at = &g_attr.back();
  }
  // static shared memory counts against the 48 KB default too: always opt in
  if (smem > at->smem_max) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { *err = e; return 0; }
    at->smem_max = smem;
  }
  for (const OccEntry& e : g_occ)
    if (e.dev == dev && e.kern == key && e.smem == smem) return e.occ;
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
    sum(s, sym, l2, part);
  }
  // CTA sum of the slots in double (after every lane's flush and a CTA barrier);
  // any number of threads may take part.
  __device__ void sum(int s, bool sym, const float* l2, double* part) const {
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

// Gram policies share one interface: slot_floats() (CTA-wide slot array),
// stage_floats() (per warp, two operands), init(slots), row(l, m, stl, stm)
// once per trip, cta_reduce(s, sym, slots, part, stl, stm).

template <int SW>
struct RowGramStaged : RowGram<SW> {
  __host__ __device__ static constexpr size_t slot_floats() { return (size_t)4 * SW * kThreads; }
  __host__ __device__ static constexpr size_t stage_floats() { return 0; }
  __device__ __forceinline__ void row(const float4& l, const float4& m, float*, float*) {
    RowGram<SW>::row(l, m);
  }
  __device__ void cta_reduce(int s, bool sym, const float* slots, double* part, float*, float*) {
    RowGram<SW>::cta_reduce(s, sym, slots, part);
  }
  __device__ void finish(float*, float*) { RowGram<SW>::flush(); }
  __device__ void sum(int s, bool sym, const float* slots, double* part, float*, float*) const {
    RowGram<SW>::sum(s, sym, slots, part);
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

// Tensor-core Gram (FP32 blocks, SW >= 8): the warp stages k = 8 rows of
// both operands, and L^T M accumulates through mma.m16n8k8 TF32 tiles (a
// 16 x 8 tile of the Gram per instruction, FP32 accumulation).  Each FP32
// operand x is split into x = big + small, big = tf32(x), small =
// tf32(x - big), and the product is big*big' + big*small' + small*big'
// (relative error ~ 2^-21 per product, dropped term small*small' <= 2^-22).
// Tile (mi, nj) covers Gram rows 16 mi .. 16 mi + 15 and columns 8 nj ..
// 8 nj + 7.  Fragment layout of mma.m16n8k8 (.tf32): with g = lane / 4 and
// t = lane % 4, A holds (g, t), (g + 8, t), (g, t + 4), (g + 8, t + 4), B
// holds (t, g), (t + 4, g), C holds (g, 2t), (g, 2t + 1), (g + 8, 2t),
// (g + 8, 2t + 1).  Windows: the tensor-core accumulators take 32 rows, a
// float register level takes 32 windows, then double slots in shared memory.
__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float* d, const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// NTH: threads of the CTA (every thread owns 4 NTILE double slots; the CTA sum runs
// over NTH / 32 warps).  kRegSlots: the double slots live in registers until dump()
// writes them to a slot array for the CTA sum (no shared memory while streaming).
template <int SW, int NTH = kThreads, bool kRegSlots = false>
struct MmaGram {
  using S = QuadShape<SW>;
  static_assert(SW >= 8, "MmaGram needs at least 8 columns");
  static constexpr int MT = SW >= 16 ? SW / 16 : 1;   // m tiles (SW = 8: rows 8..15 are zero)
  static constexpr int NT = SW / 8;                    // n tiles
  static constexpr int NTILE = MT * NT;
  static constexpr int STR = SW <= 16 ? 24 : 40;       // staged row stride, = 8 or 24 mod 32
  static constexpr int BUFROWS = S::RW >= 8 ? S::RW : 8;
  static constexpr int TRIPS_PER_K = S::RW >= 8 ? 1 : 8 / S::RW;
  static constexpr int KSTEPS = S::RW >= 8 ? S::RW / 8 : 1;
  static constexpr int WIN1 = 4;                       // k-steps per accumulator window (32 rows)
  static constexpr int WIN2 = 32;                      // windows per float register level
  float c[NTILE][4];
  float c2[NTILE][4];
  double sreg[kRegSlots ? NTILE : 1][4];
  int ks, wins, trip_in_k;
  double* slot;                                        // slot[e * NTH], e < 4 NTILE

  __host__ __device__ static constexpr size_t slot_floats() { return (size_t)2 * 4 * NTILE * NTH; }
  __host__ __device__ static constexpr size_t stage_floats() { return (size_t)2 * BUFROWS * STR; }   // per warp

  __device__ __forceinline__ void init(float* slots) {
    slot = kRegSlots ? nullptr : reinterpret_cast<double*>(slots) + threadIdx.x;
#pragma unroll
    for (int i = 0; i < NTILE; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        c[i][e] = 0.f;
        c2[i][e] = 0.f;
        if constexpr (kRegSlots) sreg[i][e] = 0.0;
        else slot[(4 * i + e) * NTH] = 0.0;
      }
    ks = 0; wins = 0; trip_in_k = 0;
  }
  __device__ __forceinline__ void flush2() {
#pragma unroll
    for (int i = 0; i < NTILE; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if constexpr (kRegSlots) sreg[i][e] += (double)c2[i][e];
        else slot[(4 * i + e) * NTH] += (double)c2[i][e];
        c2[i][e] = 0.f;
      }
    wins = 0;
  }
  // kRegSlots: the thread's double slots into the slot array (slot_floats() floats)
  __device__ __forceinline__ void dump(float* slots) const {
    if constexpr (kRegSlots) {
      double* d = reinterpret_cast<double*>(slots) + threadIdx.x;
#pragma unroll
      for (int i = 0; i < NTILE; ++i)
#pragma unroll
        for (int e = 0; e < 4; ++e) d[(4 * i + e) * NTH] = sreg[i][e];
    }
  }
  __device__ __forceinline__ void flush1() {
#pragma unroll
    for (int i = 0; i < NTILE; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) { c2[i][e] += c[i][e]; c[i][e] = 0.f; }
    ks = 0;
    if (++wins == WIN2) flush2();
  }
  // one k-step over staged rows kb .. kb + 7 (row stride STR)
  __device__ __forceinline__ void kstep(const float* stl, const float* stm, int kb) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t bb[NT][2], bs[NT][2];
#pragma unroll
    for (int nj = 0; nj < NT; ++nj) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float x = stm[(kb + t + 4 * h) * STR + 8 * nj + g];
        bb[nj][h] = tf32_of(x);
        bs[nj][h] = tf32_of(x - __uint_as_float(bb[nj][h]));
      }
    }
#pragma unroll
    for (int mi = 0; mi < MT; ++mi) {
      uint32_t ab[4], as[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = kb + t + ((e & 2) ? 4 : 0);
        const int col = 16 * mi + g + ((e & 1) ? 8 : 0);
        const float x = (col < SW) ? stl[row * STR + col] : 0.f;
        ab[e] = tf32_of(x);
        as[e] = tf32_of(x - __uint_as_float(ab[e]));
      }
#pragma unroll
      for (int nj = 0; nj < NT; ++nj) {
        mma_tf32(c[mi * NT + nj], ab, bb[nj]);
        mma_tf32(c[mi * NT + nj], ab, bs[nj]);
        mma_tf32(c[mi * NT + nj], as, bb[nj]);
      }
    }
    if (++ks == WIN1) flush1();
  }
  // Ring-fed k-steps: a ring stage holds rows of SW floats stored with the swizzle SWZ
  // (chunk q of row r at SWZ::chunk(r, q)) and the k-steps start at multiples of 8 rows,
  // where the swizzle term depends on the row within the k-step only: every fragment
  // element of a k-step is at a per-lane constant offset from the k-step's first row.
  // The B fragments read the same (row, column) pairs as the A fragments (B[nj][h] =
  // A[nj / 2][2 h + nj % 2]), so they share the offsets, and the values when the two
  // operands are one block.
  int ring_off[MT][4];
  template <class SWZ>
  __device__ __forceinline__ void init_ring() {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = t + ((e & 2) ? 4 : 0);
        const int col = 16 * mi + g + ((e & 1) ? 8 : 0);
        ring_off[mi][e] = r * SW + 4 * SWZ::chunk(r, col >> 2) + (col & 3);
      }
  }
  // One k-step over rows r0 .. r0 + 7 (r0 a multiple of 8) of the left operand (the
  // Gram's rows, sx) and the right one (sy; kSame: the same block).
  template <bool kSame>
  __device__ __forceinline__ void kstep_ring(const float* sx, const float* sy, int r0) {
    static_assert(NT == 2 * MT, "ring-fed k-steps need SW = 16 or 32");
    const float* bx = sx + r0 * SW;
    const float* by = sy + r0 * SW;
    uint32_t ab[MT][4], as[MT][4];
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float x = bx[ring_off[mi][e]];
        ab[mi][e] = tf32_of(x);
        as[mi][e] = tf32_of(x - __uint_as_float(ab[mi][e]));
      }
    uint32_t bb[NT][2], bs[NT][2];
#pragma unroll
    for (int nj = 0; nj < NT; ++nj)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int mi = nj >> 1, e = 2 * h + (nj & 1);
        if constexpr (kSame) {
          bb[nj][h] = ab[mi][e];
          bs[nj][h] = as[mi][e];
        } else {
          const float y = by[ring_off[mi][e]];
          bb[nj][h] = tf32_of(y);
          bs[nj][h] = tf32_of(y - __uint_as_float(bb[nj][h]));
        }
      }
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
      for (int nj = 0; nj < NT; ++nj) {
        mma_tf32(c[mi * NT + nj], ab[mi], bb[nj]);
        mma_tf32(c[mi * NT + nj], ab[mi], bs[nj]);
        mma_tf32(c[mi * NT + nj], as[mi], bb[nj]);
      }
    if (++ks == WIN1) flush1();
  }
  // The preconditioner pass on a ring k-step: Z = diag(w) X for rows r0 .. r0 + 7 of the
  // stage (w0, w1: w of the lane's rows r0 + t and r0 + t + 4; rows zr0 + ... of Z, stored
  // only below n) and the Gram X^T Z.  The A fragments cover each element of the k-step
  // once, so each lane stores its 4 MT elements of Z; the B values are those elements.
  __device__ __forceinline__ void kstep_ring_diag(const float* sx, int r0, float w0, float w1, float* z,
                                                  int64_t zr0, int64_t n) {
    static_assert(NT == 2 * MT, "ring-fed k-steps need SW = 16 or 32");
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float* bx = sx + r0 * SW;
    uint32_t ab[MT][4], as[MT][4];
    float zv[MT][4];
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float x = bx[ring_off[mi][e]];
        ab[mi][e] = tf32_of(x);
        as[mi][e] = tf32_of(x - __uint_as_float(ab[mi][e]));
        zv[mi][e] = ((e & 2) ? w1 : w0) * x;
      }
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t row = zr0 + t + ((e & 2) ? 4 : 0);
        const int col = 16 * mi + g + ((e & 1) ? 8 : 0);
        if (row < n) z[row * SW + col] = zv[mi][e];
      }
    uint32_t bb[NT][2], bs[NT][2];
#pragma unroll
    for (int nj = 0; nj < NT; ++nj)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float y = zv[nj >> 1][2 * h + (nj & 1)];
        bb[nj][h] = tf32_of(y);
        bs[nj][h] = tf32_of(y - __uint_as_float(bb[nj][h]));
      }
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
      for (int nj = 0; nj < NT; ++nj) {
        mma_tf32(c[mi * NT + nj], ab[mi], bb[nj]);
        mma_tf32(c[mi * NT + nj], ab[mi], bs[nj]);
        mma_tf32(c[mi * NT + nj], as[mi], bb[nj]);
      }
    if (++ks == WIN1) flush1();
  }
  // Flush every level (the ring-fed use: no partial k-step).
  __device__ __forceinline__ void finish_ring() {
    flush1();
    flush2();
  }
  // Stage the lane's quads of this trip's rows (zero for rows past n) into the
  // warp's buffers stl / stm (BUFROWS x STR floats each; stm may equal stl)
  // and run the k-steps that became complete.
  __device__ __forceinline__ void row(const float4& l, const float4& m, float* stl, float* stm) {
    const int lane = threadIdx.x & 31;
    const int qi = lane % S::LPR, rho = lane / S::LPR;
    const int rb = (S::RW >= 8) ? 0 : trip_in_k * S::RW;
    __syncwarp();                              // the last k-step has read the buffers
    st4(stl + (rb + rho) * STR + 4 * qi, l);
    if (stm != stl) st4(stm + (rb + rho) * STR + 4 * qi, m);
    __syncwarp();
    if (++trip_in_k == TRIPS_PER_K) {
      trip_in_k = 0;
#pragma unroll
      for (int kk = 0; kk < KSTEPS; ++kk) kstep(stl, stm, 8 * kk);
    }
  }
  // Completes a partial k-step (rows not staged in it are zeroed), then sums
  // entry (a, c) over the CTA in double into part (ut_index order if sym).
  __device__ void cta_reduce(int s, bool sym, const float* slots, double* part, float* stl, float* stm) {
    finish(stl, stm);
    __syncthreads();
    sum(s, sym, slots, part, stl, stm);
  }
  // The warp's part of cta_reduce: complete the partial k-step and flush every
  // accumulator level into the lane's double slots.
  __device__ void finish(float* stl, float* stm) {
    if constexpr (TRIPS_PER_K > 1) {
      if (trip_in_k != 0) {
        const int lane = threadIdx.x & 31;
        __syncwarp();
        for (int i = trip_in_k * S::RW * STR + lane; i < 8 * STR; i += 32) {
          stl[i] = 0.f;
          stm[i] = 0.f;
        }
        __syncwarp();
        kstep(stl, stm, 0);
      }
    }
    flush1();
    flush2();
  }
  // CTA sum of the double slots (after every warp's finish and a CTA barrier);
  // any number of threads may take part.
  __device__ void sum(int s, bool sym, const float* slots, double* part, float*, float*) const {
    const double* sl = reinterpret_cast<const double*>(slots);
    const int cnt = sym ? ut_count(s) : s * s;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      int a, cc;
      if (sym) {
        cc = 0;
        while ((cc + 1) * (cc + 2) / 2 <= i) ++cc;
        a = i - cc * (cc + 1) / 2;
      } else {
        a = i / s;
        cc = i - a * s;
      }
      const int tile = (a / 16) * NT + cc / 8;
      const int r = a % 16, q = cc % 8;
      const int ln = (r % 8) * 4 + q / 2;
      const int e = 4 * tile + (r / 8) * 2 + (q % 2);
      double sum = 0.0;
      for (int w = 0; w < NTH / 32; ++w) sum += sl[e * NTH + w * 32 + ln];
      part[i] = sum;
    }
    __syncthreads();
  }
};

// Gram policy per width: tensor cores for SW >= 8, shuffles for SW = 4.
template <int SW>
using GramOf = typename std::conditional<(SW >= 8), MmaGram<SW>, RowGramStaged<SW>>::type;

// Dynamic shared memory of a quad kernel with a Gram of cnt packed entries:
// part (doubles) | slots | per-warp staging; extra_floats follow.
template <int SW>
inline size_t gram_smem_bytes(int cnt, size_t extra_floats = 0) {
  using G = GramOf<SW>;
  return sizeof(double) * (size_t)((cnt + 1) & ~1) +
         sizeof(float) * (G::slot_floats() + (size_t)kWarps * G::stage_floats() + extra_floats);
}
template <int SW>
struct GramPtrs {
  double* part;
  float* slots;
  float* stl;
  float* stm;
  float* extra;
  __device__ __forceinline__ GramPtrs(double* smem, int cnt) {
    using G = GramOf<SW>;
    part = smem;
    slots = reinterpret_cast<float*>(smem + ((cnt + 1) & ~1));
    float* stage = slots + G::slot_floats();
    stl = stage + (threadIdx.x >> 5) * G::stage_floats();
    stm = stl + G::stage_floats() / 2;
    extra = stage + kWarps * G::stage_floats();
  }
};

}  // namespace bk
