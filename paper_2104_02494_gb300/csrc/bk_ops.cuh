// Row operators of the BOP kernels (Ch. 3.3, Table "kernels"): an assembled
// CSR matrix and three matrix-free stencils.  operator() gives entry (r, c)
// of A P for the scalar row layout (one lane per column); quad() gives the
// four entries (r, 4i .. 4i + 3) of an FP32 block for the vectorised layout
// (one float4 per lane, s a multiple of 4).  Both sum the terms of a row in
// ascending column order, the order of a column-sorted CSR row.
#pragma once

#include "bk_common.cuh"

namespace bk {

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Bulk prefetch of bytes [p, p + bytes) into L2 (no registers, no shared
// memory).  Issued only when p and bytes are multiples of 16; the range must
// lie inside one allocation: callers clip it to their arrays.
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  if (bytes && ((reinterpret_cast<uintptr_t>(p) | bytes) & 15u) == 0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// Rows [r0, r0 + count) of an n x s float block, clipped to [0, n); s % 4 == 0.
__device__ __forceinline__ void l2_prefetch_rows(const float* base, int64_t n, int s, int64_t r0, int count) {
  int64_t a = r0 < 0 ? 0 : r0, b = r0 + count > n ? n : r0 + count;
  if (a < b) l2_prefetch(base + a * s, (uint32_t)((b - a) * s * sizeof(float)));
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
// Packed FP32 FMAs (two lanes of a register pair per instruction on sm_100 and later),
// rounded per component exactly as fmaf.
__device__ __forceinline__ float2 fma2(float2 a, float2 x, float2 y) { return __ffma2_rn(a, x, y); }
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  const float2 aa = make_float2(a, a);
  const float2 lo = fma2(aa, make_float2(x.x, x.y), make_float2(y.x, y.y));
  const float2 hi = fma2(aa, make_float2(x.z, x.w), make_float2(y.z, y.w));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 sub4(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

template <typename T>
struct CsrRow {
  const int32_t* __restrict__ row_ptr;
  const int32_t* __restrict__ col;
  const T* __restrict__ val;
  __device__ __forceinline__ T operator()(int64_t r, int c, int s, const T* __restrict__ P) const {
    const int b = row_ptr[r], e = row_ptr[r + 1];
    T q = T(0);
    for (int j = b; j < e; ++j) q = fma(val[j], P[(int64_t)col[j] * s + c], q);
    return q;
  }
  static constexpr bool kLead = false;        // the column pattern is data
  __device__ __forceinline__ int64_t lead_off() const { return 0; }
  __device__ __forceinline__ float4 quad_lead(int64_t r, int i, int s, const float* __restrict__ P,
                                              float4) const {
    return quad(r, i, s, P);
  }
  __device__ __forceinline__ float4 quad(int64_t r, int i, int s, const float* __restrict__ P) const {
    const int b = row_ptr[r], e = row_ptr[r + 1];
    float4 q = zero4();
    for (int j = b; j < e; ++j) q = fma4(val[j], ld4(P + (int64_t)col[j] * s + 4 * i), q);
    return q;
  }
};

// 7-point constant coefficients; terms summed in ascending column order
// (-z, -y, -x, centre, +x, +y, +z), the order of a column-sorted CSR row.
// Grid coordinates of row r (x fastest) with two divisions by invariants.
__device__ __forceinline__ void grid_xyz(int64_t r, const FastDiv& dx, const FastDiv& dy, int& x, int& y,
                                         int& z) {
  const uint32_t u = (uint32_t)r;
  const uint32_t q1 = dx.div(u);
  x = (int)(u - q1 * dx.d);
  const uint32_t q2 = dy.div(q1);
  y = (int)(q1 - q2 * dy.d);
  z = (int)q2;
}

template <typename T>
struct Const7Row {
  int nx, ny, nz;
  FastDiv dx, dy;
  T c0, cxm, cxp, cym, cyp, czm, czp;
  __device__ __forceinline__ T operator()(int64_t r, int c, int s, const T* __restrict__ P) const {
    const int64_t plane = (int64_t)nx * ny;
    int x, y, z;
    grid_xyz(r, dx, dy, x, y, z);
    const T* p = P + r * s + c;
    T q = T(0);
    if (z > 0) q = fma(czm, p[-plane * s], q);
    if (y > 0) q = fma(cym, p[-(int64_t)nx * s], q);
    if (x > 0) q = fma(cxm, p[-s], q);
    q = fma(c0, p[0], q);
    if (x < nx - 1) q = fma(cxp, p[s], q);
    if (y < ny - 1) q = fma(cyp, p[(int64_t)nx * s], q);
    if (z < nz - 1) q = fma(czp, p[plane * s], q);
    return q;
  }
  __device__ __forceinline__ float4 quad(int64_t r, int i, int s, const float* __restrict__ P) const {
    const int64_t plane = (int64_t)nx * ny;
    int x, y, z;
    grid_xyz(r, dx, dy, x, y, z);
    const float* p = P + r * s + 4 * i;
    float4 q = zero4();
    if (z > 0) q = fma4(czm, ld4(p - plane * s), q);
    if (y > 0) q = fma4(cym, ld4(p - (int64_t)nx * s), q);
    if (x > 0) q = fma4(cxm, ld4(p - s), q);
    q = fma4(c0, ld4(p), q);
    if (x < nx - 1) q = fma4(cxp, ld4(p + s), q);
    if (y < ny - 1) q = fma4(cyp, ld4(p + (int64_t)nx * s), q);
    if (z < nz - 1) q = fma4(czp, ld4(p + plane * s), q);
    return q;
  }
  // In a row sweep the +z neighbour (row r + nx ny) is the row read first
  // from DRAM; a caller may load it ahead ("lead") and pass it in.  The
  // stencils keep kLead off: on GB300 the ring's registers cost more
  // occupancy than the lead latency it hides.
  static constexpr bool kLead = false;
  __device__ __forceinline__ int64_t lead_off() const { return (int64_t)nx * ny; }
  __device__ __forceinline__ float4 quad_lead(int64_t r, int i, int s, const float* __restrict__ P,
                                              float4 lead) const {
    const int64_t plane = (int64_t)nx * ny;
    int x, y, z;
    grid_xyz(r, dx, dy, x, y, z);
    const float* p = P + r * s + 4 * i;
    float4 q = zero4();
    if (z > 0) q = fma4(czm, ld4(p - plane * s), q);
    if (y > 0) q = fma4(cym, ld4(p - (int64_t)nx * s), q);
    if (x > 0) q = fma4(cxm, ld4(p - s), q);
    q = fma4(c0, ld4(p), q);
    if (x < nx - 1) q = fma4(cxp, ld4(p + s), q);
    if (y < ny - 1) q = fma4(cyp, ld4(p + (int64_t)nx * s), q);
    if (z < nz - 1) q = fma4(czp, lead, q);
    return q;
  }
};

// Variable-coefficient 7-point FV operator with precomputed coefficients:
// diag[r], fx[r] (face to r+1), fy[r] (face to r+nx), fz[r] (face to r+nx*ny).
template <typename T>
struct Var7Row {
  int nx, ny, nz;
  FastDiv dx, dy;
  const T* __restrict__ diag;
  const T* __restrict__ fx;
  const T* __restrict__ fy;
  const T* __restrict__ fz;
  __device__ __forceinline__ T operator()(int64_t r, int c, int s, const T* __restrict__ P) const {
    const int64_t plane = (int64_t)nx * ny;
    int x, y, z;
    grid_xyz(r, dx, dy, x, y, z);
    const T* p = P + r * s + c;
    T q = T(0);
    if (z > 0) q = fma(-fz[r - plane], p[-plane * s], q);
    if (y > 0) q = fma(-fy[r - nx], p[-(int64_t)nx * s], q);
    if (x > 0) q = fma(-fx[r - 1], p[-s], q);
    q = fma(diag[r], p[0], q);
    if (x < nx - 1) q = fma(-fx[r], p[s], q);
    if (y < ny - 1) q = fma(-fy[r], p[(int64_t)nx * s], q);
    if (z < nz - 1) q = fma(-fz[r], p[plane * s], q);
    return q;
  }
  __device__ __forceinline__ float4 quad(int64_t r, int i, int s, const float* __restrict__ P) const {
    const int64_t plane = (int64_t)nx * ny;
    int x, y, z;
    grid_xyz(r, dx, dy, x, y, z);
    const float* p = P + r * s + 4 * i;
    float4 q = zero4();
    if (z > 0) q = fma4(-fz[r - plane], ld4(p - plane * s), q);
    if (y > 0) q = fma4(-fy[r - nx], ld4(p - (int64_t)nx * s), q);
    if (x > 0) q = fma4(-fx[r - 1], ld4(p - s), q);
    q = fma4(diag[r], ld4(p), q);
    if (x < nx - 1) q = fma4(-fx[r], ld4(p + s), q);
    if (y < ny - 1) q = fma4(-fy[r], ld4(p + (int64_t)nx * s), q);
    if (z < nz - 1) q = fma4(-fz[r], ld4(p + plane * s), q);
    return q;
  }
  static constexpr bool kLead = false;
  __device__ __forceinline__ int64_t lead_off() const { return (int64_t)nx * ny; }
  __device__ __forceinline__ float4 quad_lead(int64_t r, int i, int s, const float* __restrict__ P,
                                              float4 lead) const {
    const int64_t plane = (int64_t)nx * ny;
    int x, y, z;
    grid_xyz(r, dx, dy, x, y, z);
    const float* p = P + r * s + 4 * i;
    float4 q = zero4();
    if (z > 0) q = fma4(-fz[r - plane], ld4(p - plane * s), q);
    if (y > 0) q = fma4(-fy[r - nx], ld4(p - (int64_t)nx * s), q);
    if (x > 0) q = fma4(-fx[r - 1], ld4(p - s), q);
    q = fma4(diag[r], ld4(p), q);
    if (x < nx - 1) q = fma4(-fx[r], ld4(p + s), q);
    if (y < ny - 1) q = fma4(-fy[r], ld4(p + (int64_t)nx * s), q);
    if (z < nz - 1) q = fma4(-fz[r], lead, q);
    return q;
  }
};

// 2D per-edge diffusion: ax[y][x] (ny x (nx+1)) joins (x-1,y),(x,y); ay[y][x]
// ((ny+1) x nx) joins (x,y-1),(x,y); diag precomputed.
template <typename T>
struct Edge5Row {
  int nx, ny;
  FastDiv dx;
  const T* __restrict__ diag;
  const T* __restrict__ ax;
  const T* __restrict__ ay;
  __device__ __forceinline__ T operator()(int64_t r, int c, int s, const T* __restrict__ P) const {
    const uint32_t u = (uint32_t)r;
    const uint32_t q1 = dx.div(u);
    const int x = (int)(u - q1 * dx.d);
    const int y = (int)q1;
    const T* p = P + r * s + c;
    T q = T(0);
    if (y > 0) q = fma(-ay[(int64_t)y * nx + x], p[-(int64_t)nx * s], q);
    if (x > 0) q = fma(-ax[(int64_t)y * (nx + 1) + x], p[-s], q);
    q = fma(diag[r], p[0], q);
    if (x < nx - 1) q = fma(-ax[(int64_t)y * (nx + 1) + x + 1], p[s], q);
    if (y < ny - 1) q = fma(-ay[(int64_t)(y + 1) * nx + x], p[(int64_t)nx * s], q);
    return q;
  }
  __device__ __forceinline__ float4 quad(int64_t r, int i, int s, const float* __restrict__ P) const {
    const uint32_t u = (uint32_t)r;
    const uint32_t q1 = dx.div(u);
    const int x = (int)(u - q1 * dx.d);
    const int y = (int)q1;
    const float* p = P + r * s + 4 * i;
    float4 q = zero4();
    if (y > 0) q = fma4(-ay[(int64_t)y * nx + x], ld4(p - (int64_t)nx * s), q);
    if (x > 0) q = fma4(-ax[(int64_t)y * (nx + 1) + x], ld4(p - s), q);
    q = fma4(diag[r], ld4(p), q);
    if (x < nx - 1) q = fma4(-ax[(int64_t)y * (nx + 1) + x + 1], ld4(p + s), q);
    if (y < ny - 1) q = fma4(-ay[(int64_t)(y + 1) * nx + x], ld4(p + (int64_t)nx * s), q);
    return q;
  }
  static constexpr bool kLead = false;
  __device__ __forceinline__ int64_t lead_off() const { return nx; }
  __device__ __forceinline__ float4 quad_lead(int64_t r, int i, int s, const float* __restrict__ P,
                                              float4 lead) const {
    const uint32_t u = (uint32_t)r;
    const uint32_t q1 = dx.div(u);
    const int x = (int)(u - q1 * dx.d);
    const int y = (int)q1;
    const float* p = P + r * s + 4 * i;
    float4 q = zero4();
    if (y > 0) q = fma4(-ay[(int64_t)y * nx + x], ld4(p - (int64_t)nx * s), q);
    if (x > 0) q = fma4(-ax[(int64_t)y * (nx + 1) + x], ld4(p - s), q);
    q = fma4(diag[r], ld4(p), q);
    if (x < nx - 1) q = fma4(-ax[(int64_t)y * (nx + 1) + x + 1], ld4(p + s), q);
    if (y < ny - 1) q = fma4(-ay[(int64_t)(y + 1) * nx + x], lead, q);
    return q;
  }
};

// Diagonal operator out_r = w_r in_r (a diagonal preconditioner M^{-1}, e.g.
// point Jacobi w = 1 / diag(A)); one coefficient per row.
template <typename T>
struct DiagRow {
  const T* __restrict__ w;
  __device__ __forceinline__ T operator()(int64_t r, int c, int s, const T* __restrict__ P) const {
    return w[r] * P[r * s + c];
  }
  __device__ __forceinline__ float4 quad(int64_t r, int i, int s, const float* __restrict__ P) const {
    const float d = w[r];
    const float4 v = ld4(P + r * s + 4 * i);
    return make_float4(d * v.x, d * v.y, d * v.z, d * v.w);
  }
  static constexpr bool kLead = false;
  __device__ __forceinline__ int64_t lead_off() const { return 0; }
  __device__ __forceinline__ float4 quad_lead(int64_t r, int i, int s, const float* __restrict__ P,
                                              float4) const {
    return quad(r, i, s, P);
  }
};

// Identity "operator": the row kernel then just streams Y, which turns the
// fused epilogue into a stand-alone block inner product X^T Y (BDOT).
template <typename T>
struct IdRow {
  __device__ __forceinline__ T operator()(int64_t r, int c, int s, const T* __restrict__ P) const {
    return P[r * s + c];
  }
  __device__ __forceinline__ float4 quad(int64_t r, int i, int s, const float* __restrict__ P) const {
    return ld4(P + r * s + 4 * i);
  }
  static constexpr bool kLead = true;
  __device__ __forceinline__ int64_t lead_off() const { return 0; }
  __device__ __forceinline__ float4 quad_lead(int64_t, int, int, const float*, float4 lead) const {
    return lead;
  }
};

}  // namespace bk
