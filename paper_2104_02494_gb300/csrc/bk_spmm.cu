// BOP: operator applied to an n x s row-major block (Ch. 3.3, Table "kernels"),
// for an assembled CSR matrix and three matrix-free stencils, with an optional
// fused epilogue that accumulates a block inner product left^T Q (the alpha of
// Alg. "bcg", Eq. "cg_alpha") and Frobenius sums in the same pass.
//
// Mapping: one sub-warp of SW = next_pow2(s) lanes per row, lane c computes
// Q[r][c].  CSR: the lanes of a row read the same val/col entries (broadcast)
// and the s contiguous values P[col][0..s) (one coalesced segment).  Stencils:
// the neighbour rows r +- 1, r +- nx, r +- nx*ny are contiguous s-value
// segments; their reuse across rows is served by L1/L2 (a 128^2 plane of a
// 32-column FP64 block is 4 MB, far below the 129 MB L2).
#include "bk_common.cuh"
#include <vector>

#include "bk_internal.h"
#include "bk_ops.cuh"
#include "bk_quad.cuh"

namespace bk {

// ------------------------------------------------------------------- kernel ----
// FP32 blocks: Gram products are accumulated in float over kFlush row groups
// and then added into double accumulators, so the double-precision work is
// 1/kFlush of the product count while every Gram partial sum beyond one flush
// window is carried in double.
constexpr int kFlush = kF32Window;

// Epilogue kinds (compile time, so that each instantiation carries only its
// own accumulators): none; symmetric Gram left^T Q; full Gram left^T Q and/or
// the Frobenius sums <Q, frob>_F, <Q, Q>_F.
enum : int { kEpiNone = 0, kEpiSym = 1, kEpiFull = 2 };

template <typename T, int SW, class RowOp, int kEpi>
__global__ void __launch_bounds__(kThreads, min_ctas<T>())
spmm_kernel(RowOp op, int64_t n, int s, const T* __restrict__ P, T* __restrict__ Q,
            const T* __restrict__ sub, Epi<T> ep) {
  if (ep.done && *ep.done) return;
  if (ep.only_if && !*ep.only_if) return;
  extern __shared__ double smem[];
  constexpr int RPW = 32 / SW;
  const int lane = threadIdx.x & 31;
  const int c = lane & (SW - 1);
  const int rs = lane / SW;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  const bool has_gram = (kEpi != kEpiNone) && ep.left != nullptr;
  const bool has_frob = (kEpi == kEpiFull) && ep.frob != nullptr;
  constexpr bool kSym = kEpi == kEpiSym;
  // FP64 symmetric Grams use the idle-lane-free pairing of two rows per
  // sub-warp; FP32 Grams accumulate in float and flush to shared memory.
  constexpr bool kPair = kSym && (sizeof(T) == 8) && (SW >= 2);
  constexpr bool kRegAcc = (kEpi != kEpiNone) && (sizeof(T) == 8) && !kPair;
  constexpr int NACC = kRegAcc ? SW : 1;
  constexpr int NACCT = (kEpi != kEpiNone && sizeof(T) == 4) ? SW : 1;
  double acc[NACC];
#pragma unroll
  for (int a = 0; a < NACC; ++a) acc[a] = 0.0;
  T acc_t[NACCT];
#pragma unroll
  for (int a = 0; a < NACCT; ++a) acc_t[a] = T(0);
  SymGramPair<kPair ? SW : 2> pg;
  if constexpr (kPair) pg.zero();
  int since_flush = 0;
  double f_qf = 0.0, f_qq = 0.0;
  // shared-memory layout of the epilogue: part | scratch | FP32 lane slots
  const int gcnt = has_gram ? (kSym ? ut_count(s) : s * s) : 0;
  const int cnt = gcnt + (has_frob ? 2 : 0);
  double* part = smem;
  double* scratch = smem + ((cnt + 1) & ~1);
  double* lacc = scratch + kWarps * (gcnt > 2 ? gcnt : 2);
  if constexpr (sizeof(T) == 4 && kEpi != kEpiNone) {
    if (has_gram)
      for (int a = 0; a < lacc_stride(SW); ++a) lacc[threadIdx.x * lacc_stride(SW) + a] = 0.0;
  }

  auto accum_row = [&](T l, T q) {
    if constexpr (kEpi != kEpiNone) {
      if constexpr (sizeof(T) == 8) {
        if constexpr (kRegAcc) {
#pragma unroll
          for (int a = 0; a < SW; ++a) {
            const T la = sw_bcast<SW>(l, a);
            if (!kSym || a <= c) acc[a] = fma((double)la, (double)q, acc[a]);
          }
        }
      } else {
#pragma unroll
        for (int a = 0; a < SW; ++a) {
          const T la = sw_bcast<SW>(l, a);
          if (!kSym || a <= c) acc_t[a] = fma(la, q, acc_t[a]);
        }
        if (++since_flush == kFlush) {
          lacc_flush<SW>(lacc, acc_t);
          since_flush = 0;
        }
      }
    }
  };

  // two row groups per trip (rows A and B of every sub-warp)
  for (int64_t base = gw * RPW; base < n; base += 2 * nw * RPW) {
    const int64_t rA = base + rs, rB = base + nw * RPW + rs;
    const bool okA = (rA < n) && (c < s), okB = (rB < n) && (c < s);
    T qA = T(0), qB = T(0);
    if (okA) {
      qA = op(rA, c, s, P);
      if (sub) qA = sub[rA * s + c] - qA;
      if (Q) Q[rA * s + c] = qA;
    }
    if (okB) {
      qB = op(rB, c, s, P);
      if (sub) qB = sub[rB * s + c] - qB;
      if (Q) Q[rB * s + c] = qB;
    }
    if constexpr (kEpi != kEpiNone) {
      if (has_gram) {
        const T lA = okA ? ep.left[rA * s + c] : T(0);
        const T lB = okB ? ep.left[rB * s + c] : T(0);
        if constexpr (kPair) {
          pg.add((double)lA, (double)qA, (double)lB, (double)qB);
        } else {
          accum_row(lA, qA);
          accum_row(lB, qB);
        }
      }
      if (has_frob) {
        if (okA) {
          const double f = (double)ep.frob[rA * s + c];
          f_qf = fma((double)qA, f, f_qf);
          f_qq = fma((double)qA, (double)qA, f_qq);
        }
        if (okB) {
          const double f = (double)ep.frob[rB * s + c];
          f_qf = fma((double)qB, f, f_qf);
          f_qq = fma((double)qB, (double)qB, f_qq);
        }
      }
    }
  }
  if constexpr (kEpi == kEpiNone) {
    return;
  } else {
    if (!has_gram && !has_frob) return;
    // ---- CTA reduction of the epilogue sums into part[0..cnt) ----
    if (has_gram) {
      if constexpr (sizeof(T) == 4) {
        lacc_flush<SW>(lacc, acc_t);
        __syncthreads();
        lacc_reduce<SW>(lacc, s, kSym, part);
      } else if constexpr (kPair) {
        pg.cta_reduce(s, scratch, part);
      } else {
        cta_reduce_gram<SW>(acc, s, kSym, scratch, part);
      }
    }
    if (has_frob) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        f_qf += __shfl_xor_sync(0xffffffffu, f_qf, off);
        f_qq += __shfl_xor_sync(0xffffffffu, f_qq, off);
      }
      if (lane == 0) { scratch[2 * (threadIdx.x >> 5)] = f_qf; scratch[2 * (threadIdx.x >> 5) + 1] = f_qq; }
      __syncthreads();
      if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += scratch[2 * w + threadIdx.x];
        part[gcnt + threadIdx.x] = t;
      }
      __syncthreads();
    }
    if (!grid_reduce_last(part, cnt, ep.gpart, ep.counter)) return;
    if (has_gram) unpack_gram(part, s, kSym, ep.gram_out);
    if (has_frob && threadIdx.x < 2) ep.frob_out[threadIdx.x] = part[gcnt + threadIdx.x];
  }
}

int spmm_grid(const Launch& L, int64_t n, int s) {
  const int rpw = 32 / next_pow2_s(s);
  const int64_t rows_per_cta = (int64_t)rpw * kWarps;
  int64_t need = (n + rows_per_cta - 1) / rows_per_cta;
  const int64_t cap = (int64_t)L.sms * kCtasPerSm;
  if (need > cap) need = cap;
  if (need < 1) need = 1;
  return (int)need;
}

static size_t epi_smem(int s, bool gram, bool sym, bool frob, bool f32) {
  const int gcnt = gram ? (sym ? ut_count(s) : s * s) : 0;
  const int cnt = gcnt + (frob ? 2 : 0);
  const int sc = gcnt > 2 ? gcnt : 2;
  const size_t lanes = (f32 && gram) ? (size_t)kThreads * lacc_stride(next_pow2_s(s)) : 0;
  return sizeof(double) * ((size_t)(((cnt + 1) & ~1) + kWarps * sc) + lanes);
}

template <typename T, int SW, class RowOp>
static cudaError_t launch_sw(const Launch& L, const RowOp& op, int64_t n, int s, const T* in,
                             T* out, const T* sub, const Epi<T>& ep) {
  const bool g = ep.left != nullptr, f = ep.frob != nullptr;
  const int grid_max = spmm_grid(L, n, s);
  size_t sm = (g || f) ? epi_smem(s, g, ep.sym != 0, f, sizeof(T) == 4) : 0;
  auto launch = [&](auto kern) -> cudaError_t {
    if (sm > 44 * 1024) {   // 48 KB default includes the static reduction buffers
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    // one resident wave (FP64 rows are bound by the FP64 pipe: no partial last wave)
    const int wave = L.sms * resident_ctas(kern, sm);
    const int grid = grid_max < wave ? grid_max : wave;
    kern<<<grid, kThreads, sm, L.stream>>>(op, n, s, in, out, sub, ep);
    return cudaGetLastError();
  };
  if (!g && !f) return launch(spmm_kernel<T, SW, RowOp, kEpiNone>);
  if (g && !f && ep.sym) return launch(spmm_kernel<T, SW, RowOp, kEpiSym>);
  return launch(spmm_kernel<T, SW, RowOp, kEpiFull>);
}

template <typename T, class RowOp>
static cudaError_t launch_op(const Launch& L, const RowOp& op, int64_t n, int s, const T* in,
                             T* out, const T* sub, const Epi<T>& ep) {
  // FP32 blocks of width 4, 8, 12, ... use the vectorised quad layout
  if constexpr (sizeof(T) == 4) {
    if (s % 4 == 0 && !ep.frob) return spmm4<RowOp>(L, op, n, s, in, out, sub, ep);
  }
  switch (next_pow2_s(s)) {
    case 1: return launch_sw<T, 1>(L, op, n, s, in, out, sub, ep);
    case 2: return launch_sw<T, 2>(L, op, n, s, in, out, sub, ep);
    case 4: return launch_sw<T, 4>(L, op, n, s, in, out, sub, ep);
    case 8: return launch_sw<T, 8>(L, op, n, s, in, out, sub, ep);
    case 16: return launch_sw<T, 16>(L, op, n, s, in, out, sub, ep);
    case 32: return launch_sw<T, 32>(L, op, n, s, in, out, sub, ep);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T> static const T* pick(const double* d, const float* f);
template <> const double* pick<double>(const double* d, const float*) { return d; }
template <> const float* pick<float>(const double*, const float* f) { return f; }

template <typename T>
cudaError_t spmm(const Launch& L, const OpDesc& A, int s, const T* in, T* out, const T* sub,
                 const Epi<T>& ep) {
  const int64_t n = A.n;
  // FP32 blocks of width 4, 8, 12, ...: the pipelined kernels (bulk copies into a
  // shared-memory ring) for the stencils and the diagonal operator
  if constexpr (sizeof(T) == 4) {
    if (!sub && s % 4 == 0 && !ep.frob) {
      cudaError_t e = cudaErrorNotSupported;
      if (A.kind == kOpConst7 || A.kind == kOpVar7 || A.kind == kOpEdge5)
        e = march_spmm4(L, A, s, in, out, ep);
      else if (A.kind == kOpDiag && A.coef32 && ep.left == in && ep.sym)
        e = stream_diag4(L, n, s, A.coef32, in, out, ep);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  switch (A.kind) {
    case kOpCsr: {
      CsrRow<T> op{A.row_ptr, A.col, pick<T>(A.val, A.val32)};
      if (!op.val) return cudaErrorInvalidValue;
      return launch_op<T>(L, op, n, s, in, out, sub, ep);
    }
    case kOpConst7: {
      Const7Row<T> op{A.nx, A.ny, A.nz, FastDiv((uint32_t)A.nx), FastDiv((uint32_t)A.ny), (T)A.c7[0],
                      (T)A.c7[1], (T)A.c7[2], (T)A.c7[3], (T)A.c7[4], (T)A.c7[5], (T)A.c7[6]};
      return launch_op<T>(L, op, n, s, in, out, sub, ep);
    }
    case kOpVar7: {
      const T* base = pick<T>(A.coef, A.coef32);
      if (!base) return cudaErrorInvalidValue;
      Var7Row<T> op{A.nx, A.ny, A.nz, FastDiv((uint32_t)A.nx), FastDiv((uint32_t)A.ny), base, base + n,
                    base + 2 * n, base + 3 * n};
      return launch_op<T>(L, op, n, s, in, out, sub, ep);
    }
    case kOpEdge5: {
      const T* dg = pick<T>(A.coef, A.coef32);
      const T* e = pick<T>(A.edges, A.edges32);
      if (!dg || !e) return cudaErrorInvalidValue;
      Edge5Row<T> op{A.nx, A.ny, FastDiv((uint32_t)A.nx), dg, e, e + (int64_t)A.ny * (A.nx + 1)};
      return launch_op<T>(L, op, n, s, in, out, sub, ep);
    }
    case kOpDiag: {
      DiagRow<T> op{pick<T>(A.coef, A.coef32)};
      if (!op.w) return cudaErrorInvalidValue;
      return launch_op<T>(L, op, n, s, in, out, sub, ep);
    }
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t gram(const Launch& L, int64_t n, int s, const T* X, const T* Y, const Epi<T>& ep) {
  if constexpr (sizeof(T) == 4) {
    if (s % 4 == 0 && !ep.frob) {
      const cudaError_t r = stream_gram4(L, n, s, X, Y, ep);
      if (r != cudaErrorNotSupported) return r;
    }
  }
  Epi<T> e = ep;
  e.left = X;
  return launch_op<T>(L, IdRow<T>{}, n, s, Y, (T*)nullptr, (const T*)nullptr, e);
}
template cudaError_t gram<double>(const Launch&, int64_t, int, const double*, const double*,
                                  const Epi<double>&);
template cudaError_t gram<float>(const Launch&, int64_t, int, const float*, const float*,
                                 const Epi<float>&);

template cudaError_t spmm<double>(const Launch&, const OpDesc&, int, const double*, double*,
                                  const double*, const Epi<double>&);
template cudaError_t spmm<float>(const Launch&, const OpDesc&, int, const float*, float*,
                                 const float*, const Epi<float>&);

// ------------------------------------------------- operator preparation ----
// VAR7: diag and +x/+y/+z face coefficients from the cell field k (h = 1).
// Interior face 2 k_i k_j / (k_i + k_j); boundary face 2 k_i; the diagonal is
// the sum of the six faces taken in the order -x, +x, -y, +y, -z, +z.
__global__ void var7_prepare(int nx, int ny, int nz, const double* __restrict__ k,
                             double* __restrict__ out) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t plane = (int64_t)nx * ny;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(r % nx), y = (int)((r / nx) % ny), z = (int)(r / plane);
    const double ki = k[r];
    auto face = [&](bool in, int64_t j) {
      if (!in) return 2.0 * ki;
      const double kj = k[j];
      return 2.0 * ki * kj / (ki + kj);
    };
    const double fxm = face(x > 0, r - 1), fxp = face(x < nx - 1, r + 1);
    const double fym = face(y > 0, r - nx), fyp = face(y < ny - 1, r + nx);
    const double fzm = face(z > 0, r - plane), fzp = face(z < nz - 1, r + plane);
    double d = 0.0;
    d += fxm; d += fxp; d += fym; d += fyp; d += fzm; d += fzp;
    out[r] = d;
    out[n + r] = (x < nx - 1) ? fxp : 0.0;
    out[2 * n + r] = (y < ny - 1) ? fyp : 0.0;
    out[3 * n + r] = (z < nz - 1) ? fzp : 0.0;
  }
}

// EDGE5: diag[y][x] = ax[y][x] + ax[y][x+1] + ay[y][x] + ay[y+1][x].
__global__ void edge5_prepare(int nx, int ny, const double* __restrict__ e, double* __restrict__ diag) {
  const int64_t n = (int64_t)nx * ny;
  const double* ax = e;
  const double* ay = e + (int64_t)ny * (nx + 1);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(r % nx), y = (int)(r / nx);
    diag[r] = ax[(int64_t)y * (nx + 1) + x] + ax[(int64_t)y * (nx + 1) + x + 1] +
              ay[(int64_t)y * nx + x] + ay[(int64_t)(y + 1) * nx + x];
  }
}

__global__ void cast_kernel(int64_t count, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

static int elem_grid(const Launch& L, int64_t count) {
  int64_t g = (count + 255) / 256;
  const int64_t cap = (int64_t)L.sms * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t cast_block(const Launch& L, int64_t count, const double* in, float* out) {
  if (count <= 0) return cudaSuccess;
  cast_kernel<<<elem_grid(L, count), 256, 0, L.stream>>>(count, in, out);
  return cudaGetLastError();
}

__global__ void widen_kernel(int64_t count, const float* __restrict__ in, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

cudaError_t widen_block(const Launch& L, int64_t count, const float* in, double* out) {
  if (count <= 0) return cudaSuccess;
  widen_kernel<<<elem_grid(L, count), 256, 0, L.stream>>>(count, in, out);
  return cudaGetLastError();
}

__global__ void exp_kernel(int64_t count, const double* __restrict__ in, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = exp(in[i]);
}

cudaError_t exp_block(const Launch& L, int64_t count, const double* in, double* out) {
  if (count <= 0) return cudaSuccess;
  exp_kernel<<<elem_grid(L, count), 256, 0, L.stream>>>(count, in, out);
  return cudaGetLastError();
}

// ---- CSR transpose: entries per column, row pointers, scatter, then a sort of
// every row by column index (the scatter's order within a row depends on the
// order of the atomic increments; the sort makes the result deterministic).
__global__ void csr_count_cols(int64_t nnz, const int32_t* __restrict__ col, int32_t* __restrict__ cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[e]], 1);
}
__global__ void csr_scatter_t(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const int32_t* __restrict__ rpt,
                              int32_t* __restrict__ fill, int32_t* __restrict__ colt, double* __restrict__ valt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int32_t j = col[e];
      const int32_t pos = rpt[j] + atomicAdd(&fill[j], 1);
      colt[pos] = (int32_t)i;
      valt[pos] = val[e];
    }
}
__global__ void csr_sort_rows(int64_t n, const int32_t* __restrict__ rp, int32_t* __restrict__ col,
                              double* __restrict__ val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int32_t a = rp[i] + 1; a < rp[i + 1]; ++a) {   // insertion sort (rows are short)
      const int32_t c = col[a];
      const double v = val[a];
      int32_t b = a - 1;
      while (b >= rp[i] && col[b] > c) {
        col[b + 1] = col[b];
        val[b + 1] = val[b];
        --b;
      }
      col[b + 1] = c;
      val[b + 1] = v;
    }
}

cudaError_t csr_transpose(const Launch& L, const OpDesc& A, OpDesc& At) {
  if (A.kind != kOpCsr || !A.val) return cudaErrorInvalidValue;
  const int64_t n = A.n, nnz = A.nnz;
  cudaError_t e;
  int32_t *rpt = nullptr, *colt = nullptr, *fill = nullptr;
  double* valt = nullptr;
  auto fail = [&](cudaError_t r) {
    cudaFree(rpt); cudaFree(colt); cudaFree(fill); cudaFree(valt);
    return r;
  };
  if ((e = cudaMalloc(&rpt, sizeof(int32_t) * (size_t)(n + 1))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&colt, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&valt, sizeof(double) * (size_t)(nnz > 0 ? nnz : 1))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&fill, sizeof(int32_t) * (size_t)n)) != cudaSuccess) return fail(e);
  if ((e = cudaMemsetAsync(fill, 0, sizeof(int32_t) * (size_t)n, L.stream)) != cudaSuccess) return fail(e);
  if (nnz > 0) csr_count_cols<<<elem_grid(L, nnz), 256, 0, L.stream>>>(nnz, A.col, fill);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  std::vector<int32_t> cnt((size_t)n), rp((size_t)n + 1);
  if ((e = cudaMemcpyAsync(cnt.data(), fill, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, L.stream)) !=
      cudaSuccess)
    return fail(e);
  if ((e = cudaStreamSynchronize(L.stream)) != cudaSuccess) return fail(e);
  rp[0] = 0;
  for (int64_t j = 0; j < n; ++j) rp[j + 1] = rp[j] + cnt[j];
  if ((e = cudaMemcpyAsync(rpt, rp.data(), sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, L.stream)) !=
      cudaSuccess)
    return fail(e);
  if ((e = cudaMemsetAsync(fill, 0, sizeof(int32_t) * (size_t)n, L.stream)) != cudaSuccess) return fail(e);
  csr_scatter_t<<<elem_grid(L, n), 256, 0, L.stream>>>(n, A.row_ptr, A.col, A.val, rpt, fill, colt, valt);
  csr_sort_rows<<<elem_grid(L, n), 256, 0, L.stream>>>(n, rpt, colt, valt);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  if ((e = cudaStreamSynchronize(L.stream)) != cudaSuccess) return fail(e);
  cudaFree(fill);
  At.kind = kOpCsr;
  At.n = n;
  At.nnz = nnz;
  At.rp_owned = rpt; At.col_owned = colt; At.val_owned = valt;
  At.row_ptr = rpt; At.col = colt; At.val = valt;
  return cudaSuccess;
}

cudaError_t op_prepare_stencil(const Launch& L, OpDesc& A, const double* coeffs) {
  if (A.kind == kOpVar7) {
    var7_prepare<<<elem_grid(L, A.n), 256, 0, L.stream>>>(A.nx, A.ny, A.nz, coeffs, A.coef);
    return cudaGetLastError();
  }
  if (A.kind == kOpEdge5) {
    edge5_prepare<<<elem_grid(L, A.n), 256, 0, L.stream>>>(A.nx, A.ny, coeffs, A.coef);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// Point Jacobi: the diagonal a_ii of every operator kind, inverted.  CSR sums
// the stored entries with column == row (none stored: a_ii = 0).
__global__ void jacobi_kernel(OpDesc A, double* __restrict__ out, int* __restrict__ bad) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.n;
       r += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    switch (A.kind) {
      case kOpCsr:
        for (int32_t j = A.row_ptr[r]; j < A.row_ptr[r + 1]; ++j)
          if (A.col[j] == r) d += A.val[j];
        break;
      case kOpConst7: d = A.c7[0]; break;
      case kOpVar7:
      case kOpEdge5: d = A.coef[r]; break;
      case kOpDiag: d = A.coef[r]; break;
      default: break;
    }
    const bool ok = d != 0.0 && isfinite(d);
    out[r] = ok ? 1.0 / d : 0.0;
    if (!ok) *bad = 1;
  }
}

cudaError_t jacobi_inverse_diagonal(const Launch& L, const OpDesc& A, double* out, int* bad) {
  if (A.kind == kOpCsr && A.nnz > 0 && (!A.col || !A.val)) return cudaErrorInvalidValue;
  jacobi_kernel<<<elem_grid(L, A.n), 256, 0, L.stream>>>(A, out, bad);
  return cudaGetLastError();
}

cudaError_t op_make_fp32(const Launch& L, OpDesc& A) {
  cudaError_t e = cudaSuccess;
  if (A.kind == kOpCsr && !A.val32) {
    if ((e = cudaMalloc(&A.val32, sizeof(float) * (size_t)(A.nnz > 0 ? A.nnz : 1))) != cudaSuccess) return e;
    return cast_block(L, A.nnz, A.val, A.val32);
  }
  if ((A.kind == kOpVar7 || A.kind == kOpEdge5 || A.kind == kOpDiag) && !A.coef32) {
    if ((e = cudaMalloc(&A.coef32, sizeof(float) * (size_t)A.coef_len)) != cudaSuccess) return e;
    if ((e = cast_block(L, A.coef_len, A.coef, A.coef32)) != cudaSuccess) return e;
  }
  if (A.kind == kOpEdge5 && !A.edges32) {
    const int64_t ne = (int64_t)A.ny * (A.nx + 1) + (int64_t)(A.ny + 1) * A.nx;
    if ((e = cudaMalloc(&A.edges32, sizeof(float) * (size_t)ne)) != cudaSuccess) return e;
    if ((e = cast_block(L, ne, A.edges, A.edges32)) != cudaSuccess) return e;
  }
  return op_make_coef4(L, A);
}

}  // namespace bk
