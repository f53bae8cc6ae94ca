// FP32 row kernels in the quad layout (one float4 per lane, s a multiple of
// 4): the operator product with its fused Gram (BOP + BDOT, Ch. 3.3), the
// BCG block updates with the fused rho Gram (Alg. "2R-CG") and the direction
// update P = R + P beta (Eq. "cg_update_p", M = I).  They compute the same
// sums as the scalar-layout kernels, term for term in the same order for the
// row outputs; only the Gram summation order differs.
#include "bk_internal.h"
#include "bk_quad.cuh"

namespace bk {

enum : int { kQEpiNone = 0, kQEpiSym = 1, kQEpiFull = 2 };

// ------------------------------------------------------------------ BOP ----
// Q = A P (or Q = sub - A P), optional fused Gram left^T Q (upper triangle or
// full), reduced deterministically over the grid into ep.gram_out.
template <int SW, class RowOp, int kEpi>
__global__ void __launch_bounds__(kThreads, (kEpi != kQEpiNone && SW <= 8) ? 2 : quad_min_ctas<SW>())
spmm4_kernel(RowOp op, int64_t n, int s, const float* __restrict__ P, float* __restrict__ Q,
             const float* __restrict__ sub, Epi<float> ep) {
  if (ep.done && *ep.done) return;
  if (ep.only_if && !*ep.only_if) return;
  using S = QuadShape<SW>;
  using Gram = GramOf<SW>;
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qi = lane % S::LPR, rho = lane / S::LPR;
  const bool qok = 4 * qi < s;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  constexpr bool kGram = kEpi != kQEpiNone;
  const int cnt = kGram ? (kEpi == kQEpiSym ? ut_count(s) : s * s) : 0;
  const GramPtrs<SW> sp(smem, cnt);
  Gram g;
  if constexpr (kGram) g.init(sp.slots);
  // For a plain Gram (IdRow) both operands' rows are read first from DRAM:
  // they are loaded two trips ahead into a register ring, so that every warp
  // keeps three trips of DRAM reads in flight (operators with kLead off load
  // as they go).
  const int64_t stride = nw * S::RW;
  const int64_t off = op.lead_off();
  constexpr bool kLeftLead = kGram && RowOp::kLead && std::is_same<RowOp, IdRow<float>>::value;
  auto lead_at = [&](int64_t rr) -> float4 {
    if constexpr (RowOp::kLead) {
      const int64_t rl = rr + off;
      return (rr < n && qok && rl < n) ? ld4(P + rl * s + 4 * qi) : zero4();
    } else {
      return zero4();
    }
  };
  auto left_at = [&](int64_t rr) -> float4 {
    if constexpr (kLeftLead) return (rr < n && qok) ? ld4(ep.left + rr * s + 4 * qi) : zero4();
    else return zero4();
  };
  const int64_t b0 = gw * S::RW;
  float4 L0 = lead_at(b0 + rho), L1 = lead_at(b0 + stride + rho);
  float4 M0 = left_at(b0 + rho), M1 = left_at(b0 + stride + rho);
  for (int64_t base = b0; base < n; base += stride) {
    const float4 L2 = lead_at(base + 2 * stride + rho);
    const float4 M2 = left_at(base + 2 * stride + rho);
    const int64_t r = base + rho;
    const bool ok = (r < n) && qok;
    float4 q = zero4(), l = zero4();
    if (ok) {
      if constexpr (RowOp::kLead) q = op.quad_lead(r, qi, s, P, L0);
      else q = op.quad(r, qi, s, P);
      if (sub) q = sub4(ld4(sub + r * s + 4 * qi), q);
      if (Q) st4(Q + r * s + 4 * qi, q);
      if constexpr (kGram) l = kLeftLead ? M0 : ld4(ep.left + r * s + 4 * qi);
    }
    if constexpr (kGram) g.row(l, q, sp.stl, sp.stm);
    L0 = L1; L1 = L2;
    M0 = M1; M1 = M2;
  }
  if constexpr (kGram) {
    g.cta_reduce(s, kEpi == kQEpiSym, sp.slots, sp.part, sp.stl, sp.stm);
    if (!grid_reduce_last(sp.part, cnt, ep.gpart, ep.counter)) return;
    unpack_gram(sp.part, s, kEpi == kQEpiSym, ep.gram_out);
  }
}

template <int SW>
static size_t spmm4_smem(int s, int epi) {
  if (epi == kQEpiNone) return 0;
  return gram_smem_bytes<SW>(epi == kQEpiSym ? ut_count(s) : s * s);
}

template <int SW, class RowOp, int kEpi>
static cudaError_t spmm4_launch(const Launch& L, const RowOp& op, int64_t n, int s, const float* in,
                                float* out, const float* sub, const Epi<float>& ep) {
  auto k = spmm4_kernel<SW, RowOp, kEpi>;
  const size_t sm = spmm4_smem<SW>(s, kEpi);
  cudaError_t err = cudaSuccess;
  const int occ = quad_occupancy(k, sm, &err);
  if (!occ) return err;
  k<<<quad_grid(L, occ, n, QuadShape<SW>::RW), kThreads, sm, L.stream>>>(op, n, s, in, out, sub, ep);
  return cudaGetLastError();
}

template <int SW, class RowOp>
static cudaError_t spmm4_sw(const Launch& L, const RowOp& op, int64_t n, int s, const float* in,
                            float* out, const float* sub, const Epi<float>& ep) {
  if (!ep.left) return spmm4_launch<SW, RowOp, kQEpiNone>(L, op, n, s, in, out, sub, ep);
  if (ep.sym) return spmm4_launch<SW, RowOp, kQEpiSym>(L, op, n, s, in, out, sub, ep);
  return spmm4_launch<SW, RowOp, kQEpiFull>(L, op, n, s, in, out, sub, ep);
}

template <class RowOp>
cudaError_t spmm4(const Launch& L, const RowOp& op, int64_t n, int s, const float* in, float* out,
                  const float* sub, const Epi<float>& ep) {
  if (s % 4 != 0 || ep.frob) return cudaErrorInvalidValue;
  switch (next_pow2_s(s)) {
    case 4: return spmm4_sw<4>(L, op, n, s, in, out, sub, ep);
    case 8: return spmm4_sw<8>(L, op, n, s, in, out, sub, ep);
    case 16: return spmm4_sw<16>(L, op, n, s, in, out, sub, ep);
    case 32: return spmm4_sw<32>(L, op, n, s, in, out, sub, ep);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t spmm4<CsrRow<float>>(const Launch&, const CsrRow<float>&, int64_t, int,
                                          const float*, float*, const float*, const Epi<float>&);
template cudaError_t spmm4<Const7Row<float>>(const Launch&, const Const7Row<float>&, int64_t, int,
                                             const float*, float*, const float*, const Epi<float>&);
template cudaError_t spmm4<Var7Row<float>>(const Launch&, const Var7Row<float>&, int64_t, int,
                                           const float*, float*, const float*, const Epi<float>&);
template cudaError_t spmm4<Edge5Row<float>>(const Launch&, const Edge5Row<float>&, int64_t, int,
                                            const float*, float*, const float*, const Epi<float>&);
template cudaError_t spmm4<IdRow<float>>(const Launch&, const IdRow<float>&, int64_t, int,
                                         const float*, float*, const float*, const Epi<float>&);
template cudaError_t spmm4<DiagRow<float>>(const Launch&, const DiagRow<float>&, int64_t, int,
                                           const float*, float*, const float*, const Epi<float>&);

// -------------------------------------------------------- BCG updates ----
// X <- X + P lx, R <- R - Q lam (lx = lambda sigma); with kRho also
// rho_new = R^T R (upper, mirrored).  kRho runs in iterations that do not
// re-orthonormalise; the lean form in those that do (or always, when
// only_if_reortho == 0).
template <int SW, bool kRho>
__global__ void __launch_bounds__(kThreads, quad_min_ctas<SW>())
update4_kernel(int64_t n, int s, const float* __restrict__ P, const float* __restrict__ Q,
               float* __restrict__ X, float* __restrict__ R, Ctrl* ctrl, double* gpart,
               int only_if_reortho) {
  if (ctrl->done) return;
  if constexpr (kRho) {
    if (ctrl->reortho_now) return;
  } else {
    if (only_if_reortho && !ctrl->reortho_now) return;
  }
  using S = QuadShape<SW>;
  extern __shared__ double smem[];
  const int cnt = kRho ? ut_count(s) : 0;
  const GramPtrs<SW> sp(smem, cnt);
  float* lx = kRho ? sp.extra : reinterpret_cast<float*>(smem);   // s x s, row stride SW
  float* lam = lx + SW * SW;
  float* ustage = lam + SW * SW;           // per warp: RW rows of P, then of Q
  stage_quad_matrix<SW>(lx, ctrl->lx, s);
  stage_quad_matrix<SW>(lam, ctrl->lam, s);
  GramOf<SW> g;
  if constexpr (kRho) g.init(sp.slots);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qi = lane % S::LPR, rho = lane / S::LPR;
  const bool qok = 4 * qi < s;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  float* stp = ustage + warp * 2 * S::STAGE;
  float* stq = stp + S::STAGE;
  for (int64_t base = gw * S::RW; base < n; base += nw * S::RW) {
    const int64_t r = base + rho;
    const bool ok = (r < n) && qok;
    float4 p4 = zero4(), q4 = zero4(), x4 = zero4(), z4 = zero4();
    if (ok) {
      p4 = ld4(P + r * s + 4 * qi);
      q4 = ld4(Q + r * s + 4 * qi);
      x4 = ld4(X + r * s + 4 * qi);
      z4 = ld4(R + r * s + 4 * qi);
    }
    st4(stp + rho * SW + 4 * qi, p4);
    st4(stq + rho * SW + 4 * qi, q4);
    __syncwarp();
    float4 dx = zero4(), rq = zero4();
#pragma unroll 4
    for (int k = 0; k < S::NQ; ++k) {
      const float4 pk = ld4(stp + rho * SW + 4 * k);
      const float4 qk = ld4(stq + rho * SW + 4 * k);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int a = 4 * k + t;
        dx = fma4(comp4(pk, t), ld4(lx + a * SW + 4 * qi), dx);
        rq = fma4(comp4(qk, t), ld4(lam + a * SW + 4 * qi), rq);
      }
    }
    x4 = add4(x4, dx);
    z4 = sub4(z4, rq);
    if (ok) {
      st4(X + r * s + 4 * qi, x4);
      st4(R + r * s + 4 * qi, z4);
    }
    __syncwarp();
    if constexpr (kRho) {
      const float4 zz = ok ? z4 : zero4();
      g.row(zz, zz, sp.stl, sp.stl);
    }
  }
  if constexpr (kRho) {
    g.cta_reduce(s, true, sp.slots, sp.part, sp.stl, sp.stl);
    if (!grid_reduce_last(sp.part, cnt, gpart, ctrl->counters[kCntB])) return;
    unpack_gram(sp.part, s, true, ctrl->rho_new);
  }
}

// The same updates for SW <= 16 with the s x s coefficients in registers
// (each lane holds its four columns of lx, then of lam: 4 SW floats) and the
// rows exchanged by shuffles, in two phases: X <- X + P lx over all rows,
// then R <- R - Q lam (and the rho Gram, staged 4 x 4 blocks).  Two row
// groups per trip keep more loads in flight.
template <int SW, bool kRho>
__global__ void __launch_bounds__(kThreads, 2)
update4r_kernel(int64_t n, int s, const float* __restrict__ P, const float* __restrict__ Q,
                float* __restrict__ X, float* __restrict__ R, Ctrl* ctrl, double* gpart,
                int only_if_reortho) {
  if (ctrl->done) return;
  if constexpr (kRho) {
    if (ctrl->reortho_now) return;
  } else {
    if (only_if_reortho && !ctrl->reortho_now) return;
  }
  using S = QuadShape<SW>;
  extern __shared__ double smem[];
  const int cnt = kRho ? ut_count(s) : 0;
  const GramPtrs<SW> sp(smem, cnt);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qi = lane % S::LPR, rho = lane / S::LPR;
  const bool qok = 4 * qi < s;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  GramOf<SW> g;
  if constexpr (kRho) g.init(sp.slots);
  float4 cf[SW];
  load_coef<SW>(cf, ctrl->lx, s, kMaxS, qi);
  for (int64_t base = gw * S::RW; base < n; base += 2 * nw * S::RW) {
    if (lane == 0) {
      const int64_t pb = base + 4 * nw * S::RW;     // two trips ahead, both row groups
      l2_prefetch_rows(P, n, s, pb, S::RW);
      l2_prefetch_rows(P, n, s, pb + nw * S::RW, S::RW);
      l2_prefetch_rows(X, n, s, pb, S::RW);
      l2_prefetch_rows(X, n, s, pb + nw * S::RW, S::RW);
    }
    const int64_t rA = base + rho, rB = base + nw * S::RW + rho;
    const bool okA = (rA < n) && qok, okB = (rB < n) && qok;
    const float4 pA = okA ? ld4(P + rA * s + 4 * qi) : zero4();
    const float4 pB = okB ? ld4(P + rB * s + 4 * qi) : zero4();
    const float4 xA = okA ? ld4(X + rA * s + 4 * qi) : zero4();
    const float4 xB = okB ? ld4(X + rB * s + 4 * qi) : zero4();
    const float4 dA = row_times<SW>(pA, cf, zero4());
    const float4 dB = row_times<SW>(pB, cf, zero4());
    if (okA) st4(X + rA * s + 4 * qi, add4(xA, dA));
    if (okB) st4(X + rB * s + 4 * qi, add4(xB, dB));
  }
  load_coef<SW>(cf, ctrl->lam, s, kMaxS, qi);
  for (int64_t base = gw * S::RW; base < n; base += 2 * nw * S::RW) {
    if (lane == 0) {
      const int64_t pb = base + 4 * nw * S::RW;
      l2_prefetch_rows(Q, n, s, pb, S::RW);
      l2_prefetch_rows(Q, n, s, pb + nw * S::RW, S::RW);
      l2_prefetch_rows(R, n, s, pb, S::RW);
      l2_prefetch_rows(R, n, s, pb + nw * S::RW, S::RW);
    }
    const int64_t rA = base + rho, rB = base + nw * S::RW + rho;
    const bool okA = (rA < n) && qok, okB = (rB < n) && qok;
    const float4 qA = okA ? ld4(Q + rA * s + 4 * qi) : zero4();
    const float4 qB = okB ? ld4(Q + rB * s + 4 * qi) : zero4();
    const float4 zA = okA ? ld4(R + rA * s + 4 * qi) : zero4();
    const float4 zB = okB ? ld4(R + rB * s + 4 * qi) : zero4();
    const float4 tA = sub4(zA, row_times<SW>(qA, cf, zero4()));
    const float4 tB = sub4(zB, row_times<SW>(qB, cf, zero4()));
    if (okA) st4(R + rA * s + 4 * qi, tA);
    if (okB) st4(R + rB * s + 4 * qi, tB);
    if constexpr (kRho) {
      const float4 gA = okA ? tA : zero4(), gB = okB ? tB : zero4();
      g.row(gA, gA, sp.stl, sp.stl);
      g.row(gB, gB, sp.stl, sp.stl);
    }
  }
  if constexpr (kRho) {
    g.cta_reduce(s, true, sp.slots, sp.part, sp.stl, sp.stl);
    if (!grid_reduce_last(sp.part, cnt, gpart, ctrl->counters[kCntB])) return;
    unpack_gram(sp.part, s, true, ctrl->rho_new);
  }
}

// P <- R + P beta with beta's columns in registers (SW <= 16).  Every lane
// reads its own quad of P before the row's quads are exchanged, so P is
// updated in place safely.
template <int SW>
__global__ void __launch_bounds__(kThreads, 2)
pupdate4r_kernel(int64_t n, int s, const float* __restrict__ R, float* __restrict__ P, Ctrl* ctrl) {
  if (ctrl->done) return;
  using S = QuadShape<SW>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qi = lane % S::LPR, rho = lane / S::LPR;
  const bool qok = 4 * qi < s;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  float4 cf[SW];
  load_coef<SW>(cf, ctrl->beta, s, kMaxS, qi);
  for (int64_t base = gw * S::RW; base < n; base += 2 * nw * S::RW) {
    if (lane == 0) {
      const int64_t pb = base + 4 * nw * S::RW;
      l2_prefetch_rows(P, n, s, pb, S::RW);
      l2_prefetch_rows(P, n, s, pb + nw * S::RW, S::RW);
      l2_prefetch_rows(R, n, s, pb, S::RW);
      l2_prefetch_rows(R, n, s, pb + nw * S::RW, S::RW);
    }
    const int64_t rA = base + rho, rB = base + nw * S::RW + rho;
    const bool okA = (rA < n) && qok, okB = (rB < n) && qok;
    const float4 pA = okA ? ld4(P + rA * s + 4 * qi) : zero4();
    const float4 pB = okB ? ld4(P + rB * s + 4 * qi) : zero4();
    const float4 zA = okA ? ld4(R + rA * s + 4 * qi) : zero4();
    const float4 zB = okB ? ld4(R + rB * s + 4 * qi) : zero4();
    const float4 aA = row_times<SW>(pA, cf, zero4());
    const float4 aB = row_times<SW>(pB, cf, zero4());
    if (okA) st4(P + rA * s + 4 * qi, add4(zA, aA));
    if (okB) st4(P + rB * s + 4 * qi, add4(zB, aB));
  }
}

// P <- R + P beta.  The warp stages its rows of P before any lane writes P.
template <int SW>
__global__ void __launch_bounds__(kThreads, quad_min_ctas<SW>())
pupdate4_kernel(int64_t n, int s, const float* __restrict__ R, float* __restrict__ P, Ctrl* ctrl) {
  if (ctrl->done) return;
  using S = QuadShape<SW>;
  __shared__ __align__(16) float beta[SW * SW];
  __shared__ __align__(16) float stage[kWarps * S::STAGE];
  stage_quad_matrix<SW>(beta, ctrl->beta, s);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qi = lane % S::LPR, rho = lane / S::LPR;
  const bool qok = 4 * qi < s;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  float* stp = stage + warp * S::STAGE;
  for (int64_t base = gw * S::RW; base < n; base += nw * S::RW) {
    const int64_t r = base + rho;
    const bool ok = (r < n) && qok;
    float4 p4 = zero4(), z4 = zero4();
    if (ok) {
      p4 = ld4(P + r * s + 4 * qi);
      z4 = ld4(R + r * s + 4 * qi);
    }
    st4(stp + rho * SW + 4 * qi, p4);
    __syncwarp();
    float4 acc = zero4();
#pragma unroll 4
    for (int k = 0; k < S::NQ; ++k) {
      const float4 pk = ld4(stp + rho * SW + 4 * k);
#pragma unroll
      for (int t = 0; t < 4; ++t) acc = fma4(comp4(pk, t), ld4(beta + (4 * k + t) * SW + 4 * qi), acc);
    }
    __syncwarp();
    if (ok) st4(P + r * s + 4 * qi, add4(z4, acc));
  }
}

template <int SW>
static cudaError_t update4r_sw(const Launch& L, int64_t n, int s, const float* P, const float* Q,
                               float* X, float* R, Ctrl* ctrl, double* gpart, int rho_mode) {
  using S = QuadShape<SW>;
  cudaError_t err = cudaSuccess;
  {
    auto k = update4r_kernel<SW, false>;
    const int occ = quad_occupancy(k, 0, &err);
    if (!occ) return err;
    k<<<quad_grid(L, occ, n, 2 * S::RW), kThreads, 0, L.stream>>>(n, s, P, Q, X, R, ctrl, gpart, rho_mode);
    if ((err = cudaGetLastError()) != cudaSuccess || rho_mode == 0) return err;
  }
  auto k = update4r_kernel<SW, true>;
  const size_t sm = gram_smem_bytes<SW>(ut_count(s));
  const int occ = quad_occupancy(k, sm, &err);
  if (!occ) return err;
  k<<<quad_grid(L, occ, n, 2 * S::RW), kThreads, sm, L.stream>>>(n, s, P, Q, X, R, ctrl, gpart, rho_mode);
  return cudaGetLastError();
}

template <int SW>
static cudaError_t update4s_sw(const Launch& L, int64_t n, int s, const float* P, const float* Q,
                               float* X, float* R, Ctrl* ctrl, double* gpart, int rho_mode) {
  using S = QuadShape<SW>;
  cudaError_t err = cudaSuccess;
  {
    auto k = update4_kernel<SW, false>;
    const size_t sm = sizeof(float) * (2 * SW * SW + (size_t)kWarps * 2 * S::STAGE);
    const int occ = quad_occupancy(k, sm, &err);
    if (!occ) return err;
    k<<<quad_grid(L, occ, n, S::RW), kThreads, sm, L.stream>>>(n, s, P, Q, X, R, ctrl, gpart, rho_mode);
    if ((err = cudaGetLastError()) != cudaSuccess || rho_mode == 0) return err;
  }
  auto k = update4_kernel<SW, true>;
  const size_t sm = gram_smem_bytes<SW>(ut_count(s), 2 * SW * SW + (size_t)kWarps * 2 * S::STAGE);
  const int occ = quad_occupancy(k, sm, &err);
  if (!occ) return err;
  k<<<quad_grid(L, occ, n, S::RW), kThreads, sm, L.stream>>>(n, s, P, Q, X, R, ctrl, gpart, rho_mode);
  return cudaGetLastError();
}

template <int SW>
static cudaError_t update4_sw(const Launch& L, int64_t n, int s, const float* P, const float* Q,
                              float* X, float* R, Ctrl* ctrl, double* gpart, int rho_mode) {
  if constexpr (SW <= 16) return update4r_sw<SW>(L, n, s, P, Q, X, R, ctrl, gpart, rho_mode);
  else return update4s_sw<SW>(L, n, s, P, Q, X, R, ctrl, gpart, rho_mode);
}

cudaError_t bcg_update4(const Launch& L, int64_t n, int s, const float* P, const float* Q, float* X,
                        float* R, Ctrl* ctrl, double* gpart, int rho_mode) {
  if (s % 4 != 0) return cudaErrorInvalidValue;
  switch (next_pow2_s(s)) {
    case 4: return update4_sw<4>(L, n, s, P, Q, X, R, ctrl, gpart, rho_mode);
    case 8: return update4_sw<8>(L, n, s, P, Q, X, R, ctrl, gpart, rho_mode);
    case 16: return update4_sw<16>(L, n, s, P, Q, X, R, ctrl, gpart, rho_mode);
    case 32: return update4_sw<32>(L, n, s, P, Q, X, R, ctrl, gpart, rho_mode);
    default: return cudaErrorInvalidValue;
  }
}

template <int SW>
static cudaError_t pupdate4_sw(const Launch& L, int64_t n, int s, const float* R, float* P, Ctrl* ctrl) {
  cudaError_t err = cudaSuccess;
  if constexpr (SW <= 16) {
    auto k = pupdate4r_kernel<SW>;
    const int occ = quad_occupancy(k, 0, &err);
    if (!occ) return err;
    k<<<quad_grid(L, occ, n, 2 * QuadShape<SW>::RW), kThreads, 0, L.stream>>>(n, s, R, P, ctrl);
  } else {
    auto k = pupdate4_kernel<SW>;
    const int occ = quad_occupancy(k, 0, &err);
    if (!occ) return err;
    k<<<quad_grid(L, occ, n, QuadShape<SW>::RW), kThreads, 0, L.stream>>>(n, s, R, P, ctrl);
  }
  return cudaGetLastError();
}

cudaError_t bcg_pupdate4(const Launch& L, int64_t n, int s, const float* R, float* P, Ctrl* ctrl) {
  if (s % 4 != 0) return cudaErrorInvalidValue;
  switch (next_pow2_s(s)) {
    case 4: return pupdate4_sw<4>(L, n, s, R, P, ctrl);
    case 8: return pupdate4_sw<8>(L, n, s, R, P, ctrl);
    case 16: return pupdate4_sw<16>(L, n, s, R, P, ctrl);
    case 32: return pupdate4_sw<32>(L, n, s, R, P, ctrl);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bk
