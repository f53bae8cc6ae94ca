// Pipelined FP32 operator and block-inner-product kernels (BOP and BDOT of
// Ch. 3.3, Table "kernels"), for blocks whose width s is a multiple of 4.
//
// The kernels separate data movement from arithmetic: the lanes of one producer
// warp keep a ring of shared-memory stages filled with asynchronous tensor or bulk
// copies (completion counted in bytes on mbarriers; every wait bounded), and the
// consumer warps compute from shared memory.  A CTA therefore keeps tens of KB of
// HBM reads in flight without holding them in registers.
//
// march4_kernel: Q = A P for the matrix-free stencils, optionally with the
// symmetric Gram P^T Q fused (the alpha of Eq. "cg_alpha").  The grid is seen
// as (gx, gy, gz) (a 2D grid as (nx, 1, ny)); every CTA owns one xy-tile of
// Tx x Ty cells and one segment of z-planes and marches through the segment.
// Per plane one tiled tensor copy brings the tile with a one-cell halo in x
// and y ((Tx + 2) x (Ty + 2) cells x s floats, zero-filled outside the grid:
// the homogeneous Dirichlet boundary needs no branch) and, for variable
// coefficients, the same box of per-cell coefficients.  Planes z - 1, z and
// z + 1 stay in the ring while plane z is computed, so every P value is read
// from HBM once per tile; the halos of neighbouring tiles are read by CTAs
// that run at the same time and come from L2.  Consumers work in the quad
// layout (one float4 of a row per lane); the Gram is the tensor-core MmaGram at
// s = 16, 32 and the CUDA-core QuadGram at s = 4, 8.
//
// mstream_kernel (s = 16, 32): G = X^T Y (or X^T X), or Z = diag(w) X with X^T Z,
// over stages of 192-row tensor-copy boxes in a swizzled ring, the products on
// the tensor cores read straight from the ring.  rstream_kernel (s = 4, 8, 16)
// and stream4_kernel (other widths): the same on CUDA cores, row per lane or in
// the quad layout.
//
// Results: the row outputs are the same sums, term by term in the same
// order, as the scalar and quad kernels (the ascending column order of a
// column-sorted CSR row); the Gram sums differ only in summation order.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "bk_internal.h"
#include "bk_pipe.cuh"
#include "bk_qgram.cuh"
#include "bk_rgram.cuh"
#include "bk_quad.cuh"

namespace bk {

namespace {

// Streaming kernels: 7 consumer warps and one producer warp, 256 threads, so that a
// thread may hold up to 255 registers (the FP32 Gram accumulators of 32-column blocks).
constexpr int kConsumers = 7;
constexpr int kPipeThreads = (kConsumers + 1) * 32;
// Producer lanes of the producer warp.  The copies one thread issues do not
// overlap one another (measured on GB300: one issuing thread moves about 4.5
// TB/s over the whole GPU with 16 KB copies, two or more about 6.2 TB/s), so
// four lanes issue in turn; lane p owns the ring slots k with k % 4 == p (the
// stage count is a multiple of 4) and knows the last use of each of them.
constexpr int kProducers = 4;
constexpr size_t kDynSmemMax = 220 * 1024;            // dynamic shared memory per CTA
constexpr int kMaxStages = 12;
// Dynamic shared memory asked for at least, so that no two CTAs of a pipelined
// kernel share an SM (every CTA then has an SM's load bandwidth to itself).
constexpr size_t kOneCtaSmem = 120 * 1024;
// The ring starts on a 1024-byte boundary (the swizzle atoms of the row copies);
// every shared-memory size below reserves that much for the alignment.
constexpr size_t kRingAlign = 1024;
enum : int { kQEpiNone = 0, kQEpiSym = 1, kQEpiFull = 2 };

enum : int { kMConst7 = 0, kMVar7 = 1, kMEdge5 = 2 };

// Marching operator kernels (s <= 32): without a Gram, 11 consumer warps and the
// producer warp (384 threads of at most 168 registers: more warps hide the latency of
// the stencil's shared-memory loads; measured 0.55 -> 0.74 of HBM at s = 16).  With the
// Gram: 11 at s = 16 (tensor-core Gram), 7 at s = 32 (its 8 tiles need the 255-register
// budget) and at s = 4; at s = 8 11 for the constant stencil (0.274 -> 0.301 of HBM on the
// 128^3 Laplacian) and 7 for the coefficient stencils, whose extra registers spill at 168
// (VAR7: 0.372 with 7 against 0.361 with 11).
template <int kEpi, int SW, int kOp>
__host__ __device__ constexpr int march_consumers() {
  return (kEpi == kQEpiNone || SW == 16 || (SW == 8 && kOp == kMConst7)) ? 11 : 7;
}
template <int kEpi, int SW, int kOp>
__host__ __device__ constexpr int march_threads() { return (march_consumers<kEpi, SW, kOp>() + 1) * 32; }
// The fused Gram of the marching kernel: for s = 16 and 32 the tensor-core MmaGram
// (TF32 products with the three-term split, 16 x 8 tiles of mma.sync; at s = 16 few
// accumulator registers per lane, so 11 consumer warps fit; at s = 32 its 8 tiles take
// 128 registers per lane and 7 consumers keep the 255-register budget), for s = 4 and
// 8 the CUDA-core pair scheme QuadGram (at s = 8 half of every 16-row tensor-core tile
// would be empty; measured: 0.372 of HBM with QuadGram against 0.338 on the 192^3 VAR7
// operator).
// MmaGram keeps its double slots in registers while streaming and dumps them into the
// ring's memory (free once the pipeline has drained) for the CTA sum.
template <int SW, int kEpi, int kOp>
using MarchGram = typename std::conditional<(SW >= 16), MmaGram<SW, march_threads<kEpi, SW, kOp>(), true>,
                                            QuadGram<SW, true>>::type;
// Bytes of the Gram region at the start of the dynamic shared memory: the packed sums,
// then the Gram's slots (QuadGram) or the per-warp staging buffers (MmaGram).
template <int SW, int kEpi, int kOp>
__host__ __device__ constexpr size_t march_gram_bytes(int cnt) {
  if constexpr (SW >= 16) {
    using G = MarchGram<SW, kEpi, kOp>;
    return sizeof(double) * (size_t)((cnt + 1) & ~1) +
           sizeof(float) * ((size_t)(march_threads<kEpi, SW, kOp>() / 32) * G::stage_floats());
  } else {
    return sizeof(double) * ((size_t)((cnt + 1) & ~1) +
                             (size_t)march_consumers<kEpi, SW, kOp>() * QuadGram<SW, true>::kWarpDoubles);
  }
}

// ------------------------------------------------------------ host helpers ----
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of a row-major float array viewed as [gz][gy][gx][w] (w innermost),
// box {w, bx, by, 1}, zero fill outside.
cudaError_t make_map4(CUtensorMap* m, const float* base, int w, int gx, int gy, int gz, int bx, int by) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[4] = {(cuuint64_t)w, (cuuint64_t)gx, (cuuint64_t)gy, (cuuint64_t)gz};
  const cuuint64_t strides[3] = {(cuuint64_t)w * 4, (cuuint64_t)w * 4 * gx, (cuuint64_t)w * 4 * gx * gy};
  const cuuint32_t box[4] = {(cuuint32_t)w, (cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map of an n x s row-major float block, box {s, box_rows}, with the swizzle
// whose span is one row (s = 8, 16, 32; none for s = 4), zero fill past n.
cudaError_t make_map_rows(CUtensorMap* m, const float* base, int s, int64_t n, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)s, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)s * 4};
  const cuuint32_t box[2] = {(cuuint32_t)s, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUtensorMapSwizzle sw = s == 32 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : s == 16 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : s == 8 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE;
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The dynamic shared-memory limit of a kernel is raised once per device to
// the largest size asked for.
template <typename K>
cudaError_t smem_attr(K kern, size_t bytes) {
  static std::mutex mu;
  static std::vector<AttrEntry> seen;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const void* key = reinterpret_cast<const void*>(kern);
  std::lock_guard<std::mutex> lock(mu);
  for (AttrEntry& a : seen)
    if (a.dev == dev && a.kern == key) {
      if (bytes <= a.smem_max) return cudaSuccess;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e == cudaSuccess) a.smem_max = bytes;
      return e;
    }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) seen.push_back({dev, key, bytes});
  return e;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

// ------------------------------------------------------------------ plans ----
struct MarchArgs {
  int gx, gy, gz, hy;     // grid (2D grids: (nx, 1, ny)); hy = 1 when gy > 1
  int Tx, Ty, zlen;       // tile and z-segment length
  int tiles_x, ntiles;
  int ns, bx, by;         // ring stages, box extent (Tx + 2, Ty + 2 hy)
  int stage_floats;       // floats per ring stage (P box, then the coefficient box)
  int pfl;                // offset (floats) of the coefficient box: the P box rounded up to 128 bytes
  uint32_t stage_bytes;   // bytes copied per stage
  int gram_bytes;         // offset of the barriers in dynamic shared memory
  float c[7];             // CONST7: (-z, -y, -x, centre, +x, +y, +z) in the (gx, gy, gz) grid
  FastDiv fdx;            // division of a tile's cell index by Tx
};

struct MarchPlanEntry {
  int dev, gx, gy, gz, s, cf, sms;
  size_t gram;
  MarchArgs a;
  int grid;
  size_t smem;
};

// Tile and segment choice: every CTA owns one (tile, z-segment) item, all items
// are resident at once (one per SM), and the largest item bounds the time.
// Cost of an item: its cells times its planes, weighted lightly by the halo
// share of the copied boxes (read again from L2 by the neighbouring tiles),
// plus a fixed cost per plane (the consumer warps' barrier waits and ring
// bookkeeping, about the work of 160 cells: small tiles with a few steps per
// warp and plane ran well below their bandwidth).  Odd segments march downwards, so the two
// segments on either side of a segment boundary copy the planes next to it at
// the same time (both at their start or both at their end): the two halo
// planes of a segment are L2 hits too and cost little.
static bool plan_march(int gx, int gy, int gz, int s, int cf, int sms, size_t gram_bytes, MarchArgs* out,
                       int* grid, size_t* smem) {
  static std::mutex mu;
  static std::vector<MarchPlanEntry> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (const MarchPlanEntry& e : cache)
      if (e.dev == dev && e.gx == gx && e.gy == gy && e.gz == gz && e.s == s && e.cf == cf && e.sms == sms &&
          e.gram == gram_bytes) {
        *out = e.a;
        *grid = e.grid;
        *smem = e.smem;
        return true;
      }
  }
  const int hy = gy > 1 ? 1 : 0;
  const size_t bar_bytes = 2 * kMaxStages * sizeof(uint64_t);
  const size_t fixed = align_up(gram_bytes, 16) + bar_bytes + kRingAlign;
  if (fixed >= kDynSmemMax) return false;
  const size_t avail = kDynSmemMax - fixed;
  double best = 1e300;
  MarchArgs ba{};
  int bgrid = 0;
  int prev_tx = -1;
  for (int kx = 1; kx <= gx; ++kx) {
    const int Tx = (gx + kx - 1) / kx;
    if (Tx == prev_tx) continue;
    prev_tx = Tx;
    if (Tx + 2 > 256) continue;
    const int tx_n = (gx + Tx - 1) / Tx;
    int prev_ty = -1;
    for (int ky = 1; ky <= gy; ++ky) {
      const int Ty = (gy + ky - 1) / ky;
      if (Ty == prev_ty) continue;
      prev_ty = Ty;
      if (Ty + 2 * hy > 256) continue;
      const int tiles = tx_n * ((gy + Ty - 1) / Ty);
      if (tiles > sms) continue;
      const int bx = Tx + 2, by = Ty + 2 * hy;
      // the coefficient box starts on a 128-byte boundary inside the stage
      const size_t pbytes = align_up((size_t)bx * by * s * 4, 128);
      const size_t stage = align_up(pbytes + (size_t)bx * by * cf * 4, 128);
      int ns = (int)(avail / stage);
      if (ns > kMaxStages) ns = kMaxStages;
      ns -= ns % kProducers;      // every producer lane owns the same number of slots
      if (ns < 4) continue;
      for (int nseg = 1; nseg <= gz && tiles * nseg <= sms; ++nseg) {
        const int zlen = (gz + nseg - 1) / nseg;
        if ((int64_t)(nseg - 1) * zlen >= gz) continue;
        const double cells = (double)Tx * Ty;
        const double halo = (double)bx * by / cells - 1.0;
        double cost = cells * zlen * (1.0 + 0.15 * halo) + cells * (nseg > 1 ? 0.6 : 0.0) + 160.0 * (zlen + 2);
        if (ns < 6) cost *= 1.0 + 0.1 * (6 - ns);
        if (cost < best) {
          best = cost;
          ba = MarchArgs{};
          ba.gx = gx; ba.gy = gy; ba.gz = gz; ba.hy = hy;
          ba.Tx = Tx; ba.Ty = Ty; ba.zlen = zlen;
          ba.tiles_x = tx_n; ba.ntiles = tiles;
          ba.ns = ns; ba.bx = bx; ba.by = by;
          ba.pfl = (int)(pbytes / 4);
          ba.stage_floats = (int)(stage / 4);
          ba.stage_bytes = (uint32_t)((size_t)bx * by * (s + cf) * 4);
          ba.gram_bytes = (int)align_up(gram_bytes, 16);
          bgrid = tiles * nseg;
        }
      }
    }
  }
  if (!bgrid) return false;
  size_t sm = (size_t)ba.gram_bytes + bar_bytes + kRingAlign + (size_t)ba.ns * ba.stage_floats * 4;
  if (sm < kOneCtaSmem) sm = kOneCtaSmem;   // one CTA per SM
  *out = ba;
  *grid = bgrid;
  *smem = sm;
  std::lock_guard<std::mutex> lock(mu);
  cache.push_back({dev, gx, gy, gz, s, cf, sms, gram_bytes, ba, bgrid, sm});
  return true;
}

// --------------------------------------------------------------- kernels ----
// Shared-memory layout of both kernels: [Gram: part (cnt doubles, even) | the
// consumer warps' FP64 slots | mbarriers full[kMaxStages], empty[kMaxStages] |
// ring, 128-byte aligned].
__device__ __forceinline__ float* ring_base(unsigned char* smem, int bar_off) {
  const uintptr_t p = reinterpret_cast<uintptr_t>(smem + bar_off + 2 * kMaxStages * sizeof(uint64_t));
  return reinterpret_cast<float*>((p + kRingAlign - 1) & ~(uintptr_t)(kRingAlign - 1));
}
template <int SW, bool kPair>
__host__ __device__ constexpr size_t qgram_bytes(int cnt, int nconsumers) {
  return sizeof(double) * ((size_t)((cnt + 1) & ~1) + (size_t)nconsumers * QuadGram<SW, kPair>::kWarpDoubles);
}

// Grid-wide end of a fused Gram: every thread of the CTA takes part.  A CTA
// whose pipeline gave up contributes NaN, so the result shows it.
template <int SW, bool kPair, int NC, bool kTree = true>
__device__ __forceinline__ void gram_epilogue(QuadGram<SW, kPair>& g, double* part, const double* wslots,
                                              int s, bool sym, bool consumer, bool aborted,
                                              const Epi<float>& ep) {
  const int cnt = sym ? ut_count(s) : s * s;
  if (consumer) g.finish();
  __syncthreads();
  QuadGram<SW, kPair>::sum(s, sym, wslots, NC, part);
  if (aborted)
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) part[i] = __longlong_as_double(0x7ff8000000000000ll);
  __syncthreads();
  if (!grid_reduce_last<kTree>(part, cnt, ep.gpart, ep.counter)) return;
  unpack_gram(part, s, sym, ep.gram_out);
}

// One stencil quad (columns 4 qi .. 4 qi + 3) of the cell at box index cidx,
// summed in the ascending column order of a column-sorted CSR row.
template <int kOp, bool kHY>
__device__ __forceinline__ float4 stencil_quad(const MarchArgs& a, int s, const float* sm, const float* sc,
                                               const float* spp, int cidx, int qi) {
  const int o = cidx * s + 4 * qi;
  const int dy = a.bx * s;
  float4 q = zero4();
  if constexpr (kOp == kMConst7) {
    q = fma4(a.c[0], ld4(sm + o), q);
    if constexpr (kHY) q = fma4(a.c[1], ld4(sc + o - dy), q);
    q = fma4(a.c[2], ld4(sc + o - s), q);
    q = fma4(a.c[3], ld4(sc + o), q);
    q = fma4(a.c[4], ld4(sc + o + s), q);
    if constexpr (kHY) q = fma4(a.c[5], ld4(sc + o + dy), q);
    q = fma4(a.c[6], ld4(spp + o), q);
  } else if constexpr (kOp == kMVar7) {
    // per cell (diag, fx, fy, fz): faces to the +x, +y, +z neighbour
    const float* cm = sm + a.pfl;
    const float* cc = sc + a.pfl;
    const int oc = cidx * 4;
    const float4 own = ld4(cc + oc);
    q = fma4(-cm[oc + 3], ld4(sm + o), q);
    if constexpr (kHY) q = fma4(-cc[oc - a.bx * 4 + 2], ld4(sc + o - dy), q);
    q = fma4(-cc[oc - 4 + 1], ld4(sc + o - s), q);
    q = fma4(own.x, ld4(sc + o), q);
    q = fma4(-own.y, ld4(sc + o + s), q);
    if constexpr (kHY) q = fma4(-own.z, ld4(sc + o + dy), q);
    q = fma4(-own.w, ld4(spp + o), q);
  } else {
    // 2D per-edge operator, grid (nx, 1, ny): per cell (diag, a of the -x edge,
    // a of the -y edge, 0); the +x / +y edges are the neighbours'
    const float* cc = sc + a.pfl;
    const float* cp = spp + a.pfl;
    const int oc = cidx * 4;
    const float4 own = ld4(cc + oc);
    q = fma4(-own.z, ld4(sm + o), q);
    q = fma4(-own.y, ld4(sc + o - s), q);
    q = fma4(own.x, ld4(sc + o), q);
    q = fma4(-cc[oc + 4 + 1], ld4(sc + o + s), q);
    q = fma4(-cp[oc + 2], ld4(spp + o), q);
  }
  return q;
}

template <int SW, int kOp, int kEpi, bool kHY>
__global__ void __launch_bounds__(march_threads<kEpi, SW, kOp>(), 1)
march4_kernel(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmC,
              const MarchArgs a, int s_in, float* __restrict__ Q, const Epi<float> ep) {
  // the block width is the compile-time SW (the launcher takes s == SW only): row offsets,
  // the Gram's width and the quad tests fold into constants
  constexpr int s = SW;
  (void)s_in;
  if (ep.done && *ep.done) return;
  if (ep.only_if && !*ep.only_if) return;
  constexpr int LPR = SW / 4, RS = 32 / LPR;
  using Gram = MarchGram<SW, kEpi, kOp>;
  constexpr bool kGram = kEpi != kQEpiNone;
  constexpr bool kMma = SW >= 16;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kNC = march_consumers<kEpi, SW, kOp>();
  const bool consumer = warp < kNC;
  const int cnt = kGram ? ut_count(s) : 0;
  double* part = reinterpret_cast<double*>(smem);
  double* wslots = part + ((cnt + 1) & ~1);
  // MmaGram: two staging buffers per warp (its double slots are registers, dumped at
  // the end into the ring's memory)
  float* stl = nullptr;
  float* stm = nullptr;
  if constexpr (kMma) {
    stl = reinterpret_cast<float*>(wslots) + (size_t)warp * Gram::stage_floats();
    stm = stl + Gram::stage_floats() / 2;
  }
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.gram_bytes);
  uint64_t* empty = full + kMaxStages;
  float* ring = ring_base(smem, a.gram_bytes);
  const int ns = a.ns;
  if (threadIdx.x == 0) {
    for (int k = 0; k < ns; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kNC);
    }
    s_abort = 0;
    mbar_fence_init();
  }
  Gram g;
  if constexpr (kGram) {
    if constexpr (kMma) g.init(nullptr);   // every thread zeroes its register slots
    else if (consumer) g.init(wslots + (size_t)warp * Gram::kWarpDoubles);
  }
  __syncthreads();

  const int tile = blockIdx.x % a.ntiles, seg = blockIdx.x / a.ntiles;
  const int tx0 = (tile % a.tiles_x) * a.Tx, ty0 = (tile / a.tiles_x) * a.Ty;
  const int z_lo = seg * a.zlen;
  const int z_hi = min(a.gz, z_lo + a.zlen);
  const int nplanes = z_hi - z_lo;
  // ring index i holds plane z_lo - 1 + i (even segments) or z_hi - i (odd ones)
  const bool down = (seg & 1) != 0;
  bool aborted = false;

  if (!consumer) {
    // ---- producers: planes z_lo - 1 .. z_hi (ring indices 0 .. nplanes + 1), ring
    // index i issued by lane i % kProducers ----
    if (lane < kProducers) {
      int last[kMaxStages];
      for (int k = 0; k < kMaxStages; ++k) last[k] = -1;
      if (lane == 0) {
        tma_prefetch_desc(&tmP);
        if (kOp != kMConst7) tma_prefetch_desc(&tmC);
      }
      for (int i = lane; i < nplanes + 2; i += kProducers) {
        const int slot = i % ns;
        if (i >= ns && !mbar_wait(&empty[slot], (uint32_t)((i / ns) - 1) & 1u, &s_abort)) {
          report_timeout(ep.status_out, ep.stop_out);
          s_abort = 1;
          break;
        }
        float* st = ring + (size_t)slot * a.stage_floats;
        mbar_arrive_expect_tx(&full[slot], a.stage_bytes);
        const int z = down ? z_hi - i : z_lo - 1 + i;
        tma_load_4d(st, &tmP, 0, tx0 - 1, ty0 - a.hy, z, &full[slot]);
        if (kOp != kMConst7) tma_load_4d(st + a.pfl, &tmC, 0, tx0 - 1, ty0 - a.hy, z, &full[slot]);
        last[slot] = i;
      }
      // no copy may be in flight when the CTA ends: wait (bounded) for the last use of
      // each of this lane's slots
      volatile int never = 0;
      for (int k = lane; k < ns; k += kProducers)
        if (last[k] >= 0) mbar_wait(&full[k], (uint32_t)(last[k] / ns) & 1u, &never);
    }
    __syncwarp();
  } else {
    // ---- consumers: per step a warp takes 2 RS cells of the tile; the lane of row
    // slot ps and quad q computes quad q of cell c0 = base + ps and quad q1 of cell
    // c1 = c0 + RS (two independent chains): q1 = q for the tensor-core Gram, which
    // stages both cells' rows; q1 = LPR - 1 - q for the pair scheme of QuadGram ----
    const int ps = lane / LPR, q = lane % LPR, qb = kMma ? q : LPR - 1 - q;
    const bool qok0 = 4 * q < s, qok1 = 4 * qb < s;
    const int cells = a.Tx * a.Ty;
    const int nsteps = (cells + 2 * RS - 1) / (2 * RS);
    const int64_t plane = (int64_t)a.gx * a.gy;
    bool alive = mbar_wait(&full[0], 0, &s_abort) && mbar_wait(&full[1], 0, &s_abort);
    // slots of ring indices i - 1, i, i + 1 and the phase parity of index i + 1,
    // advanced without divisions
    int sl_prev = 0, sl_cur = 1, sl_next = 2 % ns;
    uint32_t ph_next = 0;
    for (int i = 1; i <= nplanes && alive; ++i) {   // ring index of the computed plane
      const int z = down ? z_hi - i : z_lo - 1 + i;
      if (!mbar_wait(&full[sl_next], ph_next, &s_abort)) {
        alive = false;
        break;
      }
      const float* prev = ring + (size_t)sl_prev * a.stage_floats;
      const float* sc = ring + (size_t)sl_cur * a.stage_floats;
      const float* next = ring + (size_t)sl_next * a.stage_floats;
      const float* sm = down ? next : prev;    // plane z - 1
      const float* spp = down ? prev : next;   // plane z + 1
      float* Qz = Q + (int64_t)z * plane * s;
      for (int st = warp; st < nsteps; st += kNC) {
        const int c0 = st * 2 * RS + ps, c1 = c0 + RS;
        const int ty0c = (int)a.fdx.div((uint32_t)c0), ty1c = (int)a.fdx.div((uint32_t)c1);
        const int tx0c = c0 - ty0c * a.Tx, tx1c = c1 - ty1c * a.Tx;
        const bool in0 = c0 < cells && tx0 + tx0c < a.gx && ty0 + ty0c < a.gy;
        const bool in1 = c1 < cells && tx0 + tx1c < a.gx && ty0 + ty1c < a.gy;
        // box index of the cell (an interior one for absent cells: readable, not used)
        const int b0 = in0 ? (ty0c + a.hy) * a.bx + tx0c + 1 : a.hy * a.bx + 1;
        const int b1 = in1 ? (ty1c + a.hy) * a.bx + tx1c + 1 : a.hy * a.bx + 1;
        float4 v0 = zero4(), v1 = zero4();
        if (in0 && qok0) v0 = stencil_quad<kOp, kHY>(a, s, sm, sc, spp, b0, q);
        if (in1 && qok1) v1 = stencil_quad<kOp, kHY>(a, s, sm, sc, spp, b1, qb);
        if (in0 && qok0) st4(Qz + ((int64_t)(ty0 + ty0c) * a.gx + tx0 + tx0c) * s + 4 * q, v0);
        if (in1 && qok1) st4(Qz + ((int64_t)(ty0 + ty1c) * a.gx + tx0 + tx1c) * s + 4 * qb, v1);
        if constexpr (kGram) {
          if constexpr (kMma) {
            const float4 l0 = (in0 && qok0) ? ld4(sc + b0 * s + 4 * q) : zero4();
            const float4 l1 = (in1 && qok1) ? ld4(sc + b1 * s + 4 * qb) : zero4();
            g.row(l0, v0, stl, stm);
            g.row(l1, v1, stl, stm);
          } else {
            g.add(sc + b0 * s, sc + b1 * s, v0, v1, s);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sl_prev]);   // ring index i - 1 is no longer read
      sl_prev = sl_cur;
      sl_cur = sl_next;
      if (++sl_next == ns) {
        sl_next = 0;
        ph_next ^= 1u;
      }
    }
    if (!alive) {
      report_timeout(ep.status_out, ep.stop_out);
      s_abort = 1;
    }
  }
  if constexpr (kGram) {
    __syncthreads();
    aborted = s_abort != 0;
    if constexpr (kMma) {
      // the ring is idle here: every consumer has passed its last stage and the
      // producer lanes have waited for their last copies
      if (consumer) g.finish(stl, stm);
      g.dump(ring);
      __syncthreads();
      g.sum(s, true, ring, part, stl, stm);
      if (aborted)
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) part[i] = __longlong_as_double(0x7ff8000000000000ll);
      __syncthreads();
      if (!grid_reduce_last(part, cnt, ep.gpart, ep.counter)) return;
      unpack_gram(part, s, true, ep.gram_out);
    } else {
      // s <= 8: at most 36 values per CTA, where one level is as fast
      gram_epilogue<SW, true, kNC, false>(g, part, wslots, s, true, consumer, aborted, ep);
    }
  }
}

struct StreamArgs {
  int64_t n;
  int64_t nchunks;
  int s;
  int cr;              // rows per chunk
  int ns;
  int two;             // Y staged separately (X != Y)
  int stage_floats;
  int op_floats;       // floats of one operand's chunk (cr * s)
  int gram_bytes;
};

// kMode 0: G = X^T Y (Y = X when !two).  kMode 1: Z = diag(w) X and G = X^T Z.
// kEpi: symmetric (kPair Gram) or full.
template <int SW, int kMode, int kEpi>
__global__ void __launch_bounds__(kPipeThreads, 1)
stream4_kernel(const float* __restrict__ X, const float* __restrict__ Y, const float* __restrict__ w,
               float* __restrict__ Z, const StreamArgs a, const Epi<float> ep) {
  if (ep.done && *ep.done) return;
  if (ep.only_if && !*ep.only_if) return;
  constexpr int LPR = SW / 4, RS = 32 / LPR;
  constexpr bool kSym = kEpi == kQEpiSym;
  using Gram = QuadGram<SW, kSym>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool consumer = warp < kConsumers;
  const int s = a.s;
  const int cnt = kSym ? ut_count(s) : s * s;
  double* part = reinterpret_cast<double*>(smem);
  double* wslots = part + ((cnt + 1) & ~1);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.gram_bytes);
  uint64_t* empty = full + kMaxStages;
  float* ring = ring_base(smem, a.gram_bytes);
  const int ns = a.ns;
  if (threadIdx.x == 0) {
    for (int k = 0; k < ns; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kConsumers);
    }
    s_abort = 0;
    mbar_fence_init();
  }
  Gram g;
  if (consumer) g.init(wslots + (size_t)warp * Gram::kWarpDoubles);
  __syncthreads();
  const int64_t my_chunks =
      (int64_t)blockIdx.x < a.nchunks ? (a.nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  bool aborted = false;
  if (!consumer) {
    // producers: chunk i (of this CTA) issued by lane i % kProducers
    if (lane < kProducers) {
      int64_t last[kMaxStages];
      for (int k = 0; k < kMaxStages; ++k) last[k] = -1;
      for (int64_t i = lane; i < my_chunks; i += kProducers) {
        const int slot = (int)(i % ns);
        if (i >= ns && !mbar_wait(&empty[slot], (uint32_t)((i / ns) - 1) & 1u, &s_abort)) {
          report_timeout(ep.status_out, ep.stop_out);
          s_abort = 1;
          break;
        }
        const int64_t c = blockIdx.x + i * gridDim.x;
        const int64_t r0 = c * a.cr;
        const int rows = (int)min((int64_t)a.cr, a.n - r0);
        const uint32_t bytes = (uint32_t)rows * s * 4;
        float* st = ring + (size_t)slot * a.stage_floats;
        mbar_arrive_expect_tx(&full[slot], a.two ? 2 * bytes : bytes);
        bulk_g2s(st, X + r0 * s, bytes, &full[slot]);
        if (a.two) bulk_g2s(st + a.op_floats, Y + r0 * s, bytes, &full[slot]);
        last[slot] = i;
      }
      volatile int never = 0;
      for (int k = lane; k < ns; k += kProducers)
        if (last[k] >= 0) mbar_wait(&full[k], (uint32_t)(last[k] / ns) & 1u, &never);
    }
    __syncwarp();
  } else {
    // per step a warp takes 2 RS rows of the chunk: the lane of row slot ps and quad q
    // handles rows r0 = base + ps and r1 = r0 + RS (its right quads: q of r0 and, for
    // the symmetric Gram, LPR - 1 - q of r1, else q of r1)
    const int ps = lane / LPR, q = lane % LPR;
    const int q1 = kSym ? LPR - 1 - q : q;
    const bool qok0 = 4 * q < s, qok1 = 4 * q1 < s;
    bool alive = true;
    for (int64_t i = 0; i < my_chunks; ++i) {
      const int slot = (int)(i % ns);
      if (!mbar_wait(&full[slot], (uint32_t)(i / ns) & 1u, &s_abort)) {
        alive = false;
        break;
      }
      const int64_t c = blockIdx.x + i * gridDim.x;
      const int64_t base = c * a.cr;
      const int rows = (int)min((int64_t)a.cr, a.n - base);
      const float* sx = ring + (size_t)slot * a.stage_floats;
      const float* sy = a.two ? sx + a.op_floats : sx;
      const int nsteps = (rows + 2 * RS - 1) / (2 * RS);
      for (int st = warp; st < nsteps; st += kConsumers) {
        const int r0 = st * 2 * RS + ps, r1 = r0 + RS;
        const bool in0 = r0 < rows, in1 = r1 < rows;
        const int e0 = in0 ? r0 : 0, e1 = in1 ? r1 : 0;
        float4 m0 = zero4(), m1 = zero4();
        if constexpr (kMode == 0) {
          if (in0 && qok0) m0 = ld4(sy + e0 * s + 4 * q);
          if (in1 && qok1) m1 = ld4(sy + e1 * s + 4 * q1);
        } else {
          if (in0 && qok0) {
            const float d = w[base + r0];
            const float4 x = ld4(sx + e0 * s + 4 * q);
            m0 = make_float4(d * x.x, d * x.y, d * x.z, d * x.w);
            st4(Z + (base + r0) * s + 4 * q, m0);
          }
          if (in1 && qok1) {
            const float d = w[base + r1];
            const float4 x = ld4(sx + e1 * s + 4 * q1);
            m1 = make_float4(d * x.x, d * x.y, d * x.z, d * x.w);
            st4(Z + (base + r1) * s + 4 * q1, m1);
          }
        }
        g.add(sx + e0 * s, sx + e1 * s, m0, m1, s);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
    }
    if (!alive) {
      report_timeout(ep.status_out, ep.stop_out);
      s_abort = 1;
    }
  }
  __syncthreads();
  aborted = s_abort != 0;
  gram_epilogue<SW, kSym, kConsumers>(g, part, wslots, s, kSym, consumer, aborted, ep);
}

// ------------------------------------------------- row-per-lane streaming ----
// G = X^T Y (Y = X when !two), or Z = diag(w) X with G = X^T Z (kMode 1), for
// s = 4, 8, 16.  A stage is R = 192 nbox rows of each operand, copied as nbox
// swizzled boxes of 192 rows (rows past n arrive as zeros); six consumer warps
// take the stage's 32-row groups, warp w computing Gram class w % NCLS.
// Consumer warps: 9 (three warps of each of three Gram classes at s = 16, or one
// class), 6 for the full 16-column Gram, whose larger classes need the registers
// of fewer warps.
template <int SW, bool kSym>
__host__ __device__ constexpr int rconsumers() { return (SW == 16 && !kSym) ? 6 : 9; }
constexpr int kBoxRows = 192;

struct RStreamArgs {
  int64_t n;
  int64_t nchunks;
  int s;
  int R;               // rows per stage
  int nbox;            // boxes per operand and stage
  int ns;
  int two;
  int stage_floats;
  int op_floats;       // floats of one operand's rows in a stage (R s)
  int gram_bytes;
};

template <int SW, int kMode, bool kSym, int CLS>
__device__ __forceinline__ bool rstream_consume(const RStreamArgs& a, const float* ring, uint64_t* full,
                                                uint64_t* empty, double* wslots, const float* __restrict__ w,
                                                float* __restrict__ Z, int64_t my_chunks, volatile int* abort) {
  using C = GramClasses<SW, kSym>;
  constexpr int LPR = SW / 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kNC = rconsumers<SW, kSym>();
  const int wpc = kNC / C::NCLS, wic = warp / C::NCLS;
  RowGram2<SW, kSym, CLS> g;
  g.init(wslots + (size_t)warp * C::MB * 16);
  bool alive = true;
  const int ngroups = a.R / 32;
  int off[LPR];
#pragma unroll
  for (int q = 0; q < LPR; ++q) off[q] = Swz<SW>::lane_off(lane, q);
  for (int64_t i = 0; i < my_chunks; ++i) {
    const int slot = (int)(i % a.ns);
    if (!mbar_wait(&full[slot], (uint32_t)(i / a.ns) & 1u, abort)) {
      alive = false;
      break;
    }
    const int64_t base = (blockIdx.x + i * gridDim.x) * (int64_t)a.R;
    const float* sx = ring + (size_t)slot * a.stage_floats;
    const float* sy = a.two ? sx + a.op_floats : sx;
    for (int grp = wic; grp < ngroups; grp += wpc) {
      const int r = grp * 32 + lane;
      float4 l[LPR], m[LPR];
#pragma unroll
      for (int q = 0; q < LPR; ++q) l[q] = ld4(sx + r * SW + off[q]);
      if constexpr (kMode == 0) {
#pragma unroll
        for (int q = 0; q < LPR; ++q) m[q] = a.two ? ld4(sy + r * SW + off[q]) : l[q];
      } else {
        const int64_t row = base + r;
        const float d = row < a.n ? w[row] : 0.f;
#pragma unroll
        for (int q = 0; q < LPR; ++q) {
          m[q] = make_float4(d * l[q].x, d * l[q].y, d * l[q].z, d * l[q].w);
          if (row < a.n) st4(Z + row * SW + 4 * q, m[q]);
        }
      }
      g.row(l, m);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);
  }
  g.finish();
  return alive;
}

// The producer warp of the streaming kernels: lane i (< kProducers) issues the stages
// i, i + kProducers, ... of this CTA's chunks (nbox boxes of kBoxRows rows of each
// operand), each after its slot was released, then waits (bounded) for its last copies.
template <int SW>
__device__ __forceinline__ void rstream_produce(const CUtensorMap& tmX, const CUtensorMap& tmY, const RStreamArgs& a,
                                                float* ring, uint64_t* full, uint64_t* empty, int64_t my_chunks,
                                                volatile int* s_abort, const Epi<float>& ep) {
  const int lane = threadIdx.x & 31;
  const int ns = a.ns;
  if (lane < kProducers) {
    int64_t last[kMaxStages];
    for (int k = 0; k < kMaxStages; ++k) last[k] = -1;
    const uint32_t box_bytes = (uint32_t)kBoxRows * SW * 4;
    const uint32_t bytes = box_bytes * a.nbox * (a.two ? 2 : 1);
    for (int64_t i = lane; i < my_chunks; i += kProducers) {
      const int slot = (int)(i % ns);
      if (i >= ns && !mbar_wait(&empty[slot], (uint32_t)((i / ns) - 1) & 1u, s_abort)) {
        report_timeout(ep.status_out, ep.stop_out);
        *s_abort = 1;
        break;
      }
      const int64_t r0 = (blockIdx.x + i * gridDim.x) * (int64_t)a.R;
      float* st = ring + (size_t)slot * a.stage_floats;
      mbar_arrive_expect_tx(&full[slot], bytes);
      for (int b = 0; b < a.nbox; ++b) {
        tma_load_2d(st + b * kBoxRows * SW, &tmX, 0, (int)(r0 + b * kBoxRows), &full[slot]);
        if (a.two) tma_load_2d(st + a.op_floats + b * kBoxRows * SW, &tmY, 0, (int)(r0 + b * kBoxRows), &full[slot]);
      }
      last[slot] = i;
    }
    volatile int never = 0;
    for (int k = lane; k < ns; k += kProducers)
      if (last[k] >= 0) mbar_wait(&full[k], (uint32_t)(last[k] / ns) & 1u, &never);
  }
  __syncwarp();
}

template <int SW, int kMode, bool kSym>
__global__ void __launch_bounds__((rconsumers<SW, kSym>() + 1) * 32, 1)
rstream_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
               const float* __restrict__ w, float* __restrict__ Z, const RStreamArgs a, const Epi<float> ep) {
  if (ep.done && *ep.done) return;
  if (ep.only_if && !*ep.only_if) return;
  using C = GramClasses<SW, kSym>;
  constexpr int kNC = rconsumers<SW, kSym>();
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_abort;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool consumer = warp < kNC;
  const int cnt = kSym ? ut_count(SW) : SW * SW;
  double* part = reinterpret_cast<double*>(smem);
  double* wslots = part + ((cnt + 1) & ~1);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.gram_bytes);
  uint64_t* empty = full + kMaxStages;
  float* ring = ring_base(smem, a.gram_bytes);
  const int ns = a.ns;
  if (threadIdx.x == 0) {
    for (int k = 0; k < ns; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kNC);
    }
    s_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();
  const int64_t my_chunks =
      (int64_t)blockIdx.x < a.nchunks ? (a.nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (!consumer) {
    rstream_produce<SW>(tmX, tmY, a, ring, full, empty, my_chunks, &s_abort, ep);
  } else {
    bool alive = true;
    switch (warp % C::NCLS) {
      case 0: alive = rstream_consume<SW, kMode, kSym, 0>(a, ring, full, empty, wslots, w, Z, my_chunks, &s_abort); break;
      case 1:
        if constexpr (C::NCLS > 1)
          alive = rstream_consume<SW, kMode, kSym, 1 % C::NCLS>(a, ring, full, empty, wslots, w, Z, my_chunks, &s_abort);
        break;
      default:
        if constexpr (C::NCLS > 2)
          alive = rstream_consume<SW, kMode, kSym, 2 % C::NCLS>(a, ring, full, empty, wslots, w, Z, my_chunks, &s_abort);
        break;
    }
    if (!alive) {
      report_timeout(ep.status_out, ep.stop_out);
      s_abort = 1;
    }
  }
  __syncthreads();
  const bool aborted = s_abort != 0;
  row_gram_sum<SW, kSym>(SW, wslots, kNC, part);
  if (aborted)
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) part[i] = __longlong_as_double(0x7ff8000000000000ll);
  __syncthreads();
  if (!grid_reduce_last(part, cnt, ep.gpart, ep.counter)) return;
  unpack_gram(part, SW, kSym, ep.gram_out);
}

// Streaming G = X^T Y (Y = X when !two) for s = 16, 32 with the products on the tensor
// cores: the consumer warps take the stage's 8-row k-steps w, w + NC, ... and read them
// as mma.m16n8k8 TF32 fragments straight from the swizzled ring (MmaGram::kstep_ring:
// three-term split, FP32 over 32-row windows and 32 windows, FP64 in registers); the
// slots are dumped into the idle ring for the CTA sum.  12 consumers at s = 16 (48
// k-steps per stage of 384 rows); 7 at s = 32 (256 threads, so that the 8 accumulator
// tiles fit the 255-register budget), the k-steps dealt round-robin across stages.
template <int SW>
__host__ __device__ constexpr int mconsumers() { return SW == 16 ? 12 : 7; }
template <int SW>
using StreamMma = MmaGram<SW, (mconsumers<SW>() + 1) * 32, true>;

// kDiag: the diagonal preconditioner pass, Z = diag(w) X written out and G = X^T Z.
template <int SW, bool kSym, bool kDiag>
__global__ void __launch_bounds__((mconsumers<SW>() + 1) * 32, 1)
mstream_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
               const RStreamArgs a, const float* __restrict__ w, float* __restrict__ Z, const Epi<float> ep) {
  if (ep.done && *ep.done) return;
  if (ep.only_if && !*ep.only_if) return;
  constexpr int kNC = mconsumers<SW>();
  using G = StreamMma<SW>;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_abort;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool consumer = warp < kNC;
  const int cnt = kSym ? ut_count(SW) : SW * SW;
  double* part = reinterpret_cast<double*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.gram_bytes);
  uint64_t* empty = full + kMaxStages;
  float* ring = ring_base(smem, a.gram_bytes);
  const int ns = a.ns;
  if (threadIdx.x == 0) {
    for (int k = 0; k < ns; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kNC);
    }
    s_abort = 0;
    mbar_fence_init();
  }
  G g;
  g.init(nullptr);
  g.template init_ring<Swz<SW>>();
  __syncthreads();
  const int64_t my_chunks =
      (int64_t)blockIdx.x < a.nchunks ? (a.nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (!consumer) {
    rstream_produce<SW>(tmX, tmY, a, ring, full, empty, my_chunks, &s_abort, ep);
  } else {
    bool alive = true;
    const int nk = a.R / 8;
    const bool same = !a.two;
    int slot = 0;
    uint32_t ph = 0;
    // kDiag: a warp takes at most kMaxK k-steps of a stage (48 / 12 at s = 16, 24 / 7 at 32)
    constexpr int kMaxK = 4;
    for (int64_t i = 0; i < my_chunks; ++i) {
      // k-steps dealt round-robin over the chunk's stages: warp w takes the global k-step
      // indices w, w + NC, ...
      const int k0 = (warp - (int)((i * nk) % kNC) + kNC) % kNC;
      float wv[kMaxK][2];
      const int64_t base = (blockIdx.x + i * gridDim.x) * (int64_t)a.R;
      if constexpr (kDiag) {
        // the scaling of the warp's rows, loaded before the stage wait (it does not come
        // through the ring)
#pragma unroll
        for (int j = 0; j < kMaxK; ++j) {
          const int64_t r = base + 8 * (k0 + j * kNC) + (lane & 3);
          const bool ok = k0 + j * kNC < nk;
          wv[j][0] = ok && r < a.n ? w[r] : 0.f;
          wv[j][1] = ok && r + 4 < a.n ? w[r + 4] : 0.f;
        }
      }
      if (!mbar_wait(&full[slot], ph, &s_abort)) {
        alive = false;
        break;
      }
      const float* sx = ring + (size_t)slot * a.stage_floats;
      const float* sy = a.two ? sx + a.op_floats : sx;
      if constexpr (kDiag) {
#pragma unroll
        for (int j = 0; j < kMaxK; ++j) {
          const int k = k0 + j * kNC;
          if (k < nk) g.kstep_ring_diag(sx, 8 * k, wv[j][0], wv[j][1], Z, base + 8 * k, a.n);
        }
      } else if (same) {
        for (int k = k0; k < nk; k += kNC) g.template kstep_ring<true>(sx, sx, 8 * k);
      } else {
        for (int k = k0; k < nk; k += kNC) g.template kstep_ring<false>(sx, sy, 8 * k);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
      if (++slot == ns) {
        slot = 0;
        ph ^= 1u;
      }
    }
    g.finish_ring();
    if (!alive) {
      report_timeout(ep.status_out, ep.stop_out);
      s_abort = 1;
    }
  }
  // the ring is idle: every consumer has released its last stage and the producer lanes
  // have waited for their last copies
  __syncthreads();
  const bool aborted = s_abort != 0;
  g.dump(ring);
  __syncthreads();
  g.sum(SW, kSym, ring, part, nullptr, nullptr);
  if (aborted)
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) part[i] = __longlong_as_double(0x7ff8000000000000ll);
  __syncthreads();
  if (!grid_reduce_last(part, cnt, ep.gpart, ep.counter)) return;
  unpack_gram(part, SW, kSym, ep.gram_out);
}

// ------------------------------------------------------------- launchers ----
namespace {

// Grid of an operator for the marching kernel: 2D grids (nz = 1) run as (nx, 1, ny).
void march_grid(const OpDesc& A, int* gx, int* gy, int* gz) {
  if (A.kind == kOpEdge5 || A.nz == 1) {
    *gx = A.nx; *gy = 1; *gz = A.ny;
  } else {
    *gx = A.nx; *gy = A.ny; *gz = A.nz;
  }
}

template <int SW, int kOp, int kEpi>
cudaError_t march_launch(const Launch& L, const OpDesc& A, int s, const float* in, float* out,
                         const Epi<float>& ep) {
  int gx, gy, gz;
  march_grid(A, &gx, &gy, &gz);
  const int cf = kOp == kMConst7 ? 0 : 4;
  const size_t gb = kEpi == kQEpiNone ? 0 : march_gram_bytes<SW, kEpi, kOp>(ut_count(s));
  MarchArgs a;
  int grid = 0;
  size_t smem = 0;
  if (!plan_march(gx, gy, gz, s, cf, L.sms, gb, &a, &grid, &smem)) return cudaErrorNotSupported;
  if constexpr (SW >= 16 && kEpi != kQEpiNone) {
    // the Gram's slots are dumped into the ring at the end
    if ((size_t)a.ns * a.stage_floats < MarchGram<SW, kEpi, kOp>::slot_floats()) return cudaErrorNotSupported;
  }
  a.fdx = FastDiv((uint32_t)a.Tx);
  if (kOp == kMConst7) {
    const double* c = A.c7;   // (centre, -x, +x, -y, +y, -z, +z)
    if (A.nz == 1) {          // 2D: the grid's y is the marching axis
      const float v[7] = {(float)c[3], 0.f, (float)c[1], (float)c[0], (float)c[2], 0.f, (float)c[4]};
      for (int k = 0; k < 7; ++k) a.c[k] = v[k];
    } else {
      const float v[7] = {(float)c[5], (float)c[3], (float)c[1], (float)c[0], (float)c[2], (float)c[4], (float)c[6]};
      for (int k = 0; k < 7; ++k) a.c[k] = v[k];
    }
  }
  CUtensorMap tmP, tmC;
  cudaError_t e = make_map4(&tmP, in, s, gx, gy, gz, a.bx, a.by);
  if (e != cudaSuccess) return e;
  if (kOp != kMConst7) {
    if (!A.coef4) return cudaErrorNotSupported;
    if ((e = make_map4(&tmC, A.coef4, 4, gx, gy, gz, a.bx, a.by)) != cudaSuccess) return e;
  } else {
    tmC = tmP;
  }
  auto k = a.hy ? march4_kernel<SW, kOp, kEpi, true> : march4_kernel<SW, kOp, kEpi, false>;
  if ((e = smem_attr(k, smem)) != cudaSuccess) return e;
  k<<<grid, march_threads<kEpi, SW, kOp>(), smem, L.stream>>>(tmP, tmC, a, s, out, ep);
  return cudaGetLastError();
}

template <int SW, int kOp>
cudaError_t march_epi(const Launch& L, const OpDesc& A, int s, const float* in, float* out, const Epi<float>& ep) {
  if (!ep.left) return march_launch<SW, kOp, kQEpiNone>(L, A, s, in, out, ep);
  if (ep.sym) return march_launch<SW, kOp, kQEpiSym>(L, A, s, in, out, ep);
  return cudaErrorNotSupported;
}

// Widths that are powers of two only (the kernel takes s as the compile-time SW); s = 12,
// 20, 24, 28 use the quad kernels.
template <int kOp>
cudaError_t march_sw(const Launch& L, const OpDesc& A, int s, const float* in, float* out, const Epi<float>& ep) {
  if (s != next_pow2_s(s)) return cudaErrorNotSupported;
  switch (next_pow2_s(s)) {
    case 4: return march_epi<4, kOp>(L, A, s, in, out, ep);
    case 8: return march_epi<8, kOp>(L, A, s, in, out, ep);
    case 16: return march_epi<16, kOp>(L, A, s, in, out, ep);
    case 32: return march_epi<32, kOp>(L, A, s, in, out, ep);
    default: return cudaErrorNotSupported;
  }
}

// Rows per chunk of the streaming kernel: about 16 KB per operand, a multiple of 32.
int stream_rows(int s) {
  int cr = 16384 / (4 * s);
  cr -= cr % 32;
  return cr < 32 ? 32 : cr;
}

template <int SW, int kMode, int kEpi>
cudaError_t stream_launch(const Launch& L, int64_t n, int s, const float* X, const float* Y, const float* w,
                          float* Z, const Epi<float>& ep) {
  const int cnt = kEpi == kQEpiSym ? ut_count(s) : s * s;
  const size_t gb = align_up(qgram_bytes<SW, kEpi == kQEpiSym>(cnt, kConsumers), 16);
  StreamArgs a;
  a.n = n;
  a.s = s;
  a.cr = stream_rows(s);
  a.nchunks = (n + a.cr - 1) / a.cr;
  a.two = (kMode == 0 && X != Y) ? 1 : 0;
  a.op_floats = a.cr * s;
  a.stage_floats = (int)(align_up((size_t)a.op_floats * 4 * (a.two ? 2 : 1), 128) / 4);
  a.gram_bytes = (int)gb;
  const size_t fixed = gb + 2 * kMaxStages * sizeof(uint64_t) + kRingAlign;
  int nsg = (int)((kDynSmemMax - fixed) / ((size_t)a.stage_floats * 4));
  a.ns = nsg > 8 ? 8 : nsg;
  a.ns -= a.ns % kProducers;   // every producer lane owns the same number of slots
  if (a.ns < kProducers) return cudaErrorNotSupported;
  size_t smem = fixed + (size_t)a.ns * a.stage_floats * 4;
  if (smem < kOneCtaSmem) smem = kOneCtaSmem;
  int64_t grid = a.nchunks < L.sms ? a.nchunks : L.sms;
  auto k = stream4_kernel<SW, kMode, kEpi>;
  cudaError_t e = smem_attr(k, smem);
  if (e != cudaSuccess) return e;
  k<<<(int)grid, kPipeThreads, smem, L.stream>>>(X, Y, w, Z, a, ep);
  return cudaGetLastError();
}

template <int kMode, int kEpi>
cudaError_t stream_sw(const Launch& L, int64_t n, int s, const float* X, const float* Y, const float* w, float* Z,
                      const Epi<float>& ep) {
  switch (next_pow2_s(s)) {
    case 4: return stream_launch<4, kMode, kEpi>(L, n, s, X, Y, w, Z, ep);
    case 8: return stream_launch<8, kMode, kEpi>(L, n, s, X, Y, w, Z, ep);
    case 16: return stream_launch<16, kMode, kEpi>(L, n, s, X, Y, w, Z, ep);
    default: return cudaErrorNotSupported;    // s > 16: the row kernels (see march_sw)
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <int SW, int kMode, bool kSym>
cudaError_t rstream_launch(const Launch& L, int64_t n, const float* X, const float* Y, const float* w, float* Z,
                           const Epi<float>& ep) {
  using C = GramClasses<SW, kSym>;
  const int cnt = kSym ? ut_count(SW) : SW * SW;
  RStreamArgs a;
  a.n = n;
  a.s = SW;
  // 18-24 KB of each operand per stage, its 6 nbox 32-row groups a multiple of the
  // warps of a class (3 with three classes, 9 with one, 2 for the full 16-column Gram)
  a.nbox = SW == 4 ? 6 : (SW == 8 ? 3 : 2);
  a.R = kBoxRows * a.nbox;
  a.nchunks = (n + a.R - 1) / a.R;
  a.two = (kMode == 0 && X != Y) ? 1 : 0;
  a.op_floats = a.R * SW;
  a.stage_floats = a.op_floats * (a.two ? 2 : 1);
  constexpr int kNC = rconsumers<SW, kSym>();
  a.gram_bytes = (int)align_up(sizeof(double) * ((size_t)((cnt + 1) & ~1) + (size_t)kNC * C::MB * 16), 16);
  const size_t fixed = a.gram_bytes + 2 * kMaxStages * sizeof(uint64_t) + kRingAlign;
  int nsg = (int)((kDynSmemMax - fixed) / ((size_t)a.stage_floats * 4));
  a.ns = nsg > 8 ? 8 : nsg;
  a.ns -= a.ns % kProducers;
  if (a.ns < kProducers) return cudaErrorNotSupported;
  size_t smem = fixed + (size_t)a.ns * a.stage_floats * 4;
  if (smem < kOneCtaSmem) smem = kOneCtaSmem;
  CUtensorMap tx, ty;
  cudaError_t e = make_map_rows(&tx, X, SW, n, kBoxRows);
  if (e != cudaSuccess) return e;
  if (a.two) {
    if ((e = make_map_rows(&ty, Y, SW, n, kBoxRows)) != cudaSuccess) return e;
  } else {
    ty = tx;
  }
  const int64_t grid = a.nchunks < L.sms ? a.nchunks : L.sms;
  auto k = rstream_kernel<SW, kMode, kSym>;
  if ((e = smem_attr(k, smem)) != cudaSuccess) return e;
  k<<<(int)grid, (kNC + 1) * 32, smem, L.stream>>>(tx, ty, w, Z, a, ep);
  return cudaGetLastError();
}

template <int SW, bool kSym, bool kDiag>
cudaError_t mstream_launch(const Launch& L, int64_t n, const float* X, const float* Y, const float* w, float* Z,
                           const Epi<float>& ep) {
  const int cnt = kSym ? ut_count(SW) : SW * SW;
  RStreamArgs a;
  a.n = n;
  a.s = SW;
  a.nbox = SW == 16 ? 2 : 1;               // 384 or 192 rows (24 KB of each operand) per stage
  a.R = kBoxRows * a.nbox;
  a.nchunks = (n + a.R - 1) / a.R;
  a.two = (!kDiag && X != Y) ? 1 : 0;
  a.op_floats = a.R * SW;
  a.stage_floats = a.op_floats * (a.two ? 2 : 1);
  a.gram_bytes = (int)align_up(sizeof(double) * (size_t)((cnt + 1) & ~1), 16);
  const size_t fixed = a.gram_bytes + 2 * kMaxStages * sizeof(uint64_t) + kRingAlign;
  int nsg = (int)((kDynSmemMax - fixed) / ((size_t)a.stage_floats * 4));
  a.ns = nsg > 8 ? 8 : nsg;
  a.ns -= a.ns % kProducers;
  if (a.ns < kProducers) return cudaErrorNotSupported;
  // the Gram's double slots are dumped into the ring at the end
  if ((size_t)a.ns * a.stage_floats < StreamMma<SW>::slot_floats()) return cudaErrorNotSupported;
  // the diagonal pass preloads at most 4 k-steps' scalings per warp and stage
  if (kDiag && (a.R / 8 + mconsumers<SW>() - 1) / mconsumers<SW>() > 4) return cudaErrorNotSupported;
  size_t smem = fixed + (size_t)a.ns * a.stage_floats * 4;
  if (smem < kOneCtaSmem) smem = kOneCtaSmem;
  CUtensorMap tx, ty;
  cudaError_t e = make_map_rows(&tx, X, SW, n, kBoxRows);
  if (e != cudaSuccess) return e;
  if (a.two) {
    if ((e = make_map_rows(&ty, Y, SW, n, kBoxRows)) != cudaSuccess) return e;
  } else {
    ty = tx;
  }
  const int64_t grid = a.nchunks < L.sms ? a.nchunks : L.sms;
  auto k = mstream_kernel<SW, kSym, kDiag>;
  if ((e = smem_attr(k, smem)) != cudaSuccess) return e;
  k<<<(int)grid, (mconsumers<SW>() + 1) * 32, smem, L.stream>>>(tx, ty, a, w, Z, ep);
  return cudaGetLastError();
}

template <int kMode, bool kSym>
cudaError_t rstream_sw(const Launch& L, int64_t n, int s, const float* X, const float* Y, const float* w, float* Z,
                       const Epi<float>& ep) {
  switch (s) {
    case 4: return rstream_launch<4, kMode, kSym>(L, n, X, Y, w, Z, ep);
    case 8: return rstream_launch<8, kMode, kSym>(L, n, X, Y, w, Z, ep);
    case 16: return rstream_launch<16, kMode, kSym>(L, n, X, Y, w, Z, ep);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t march_spmm4(const Launch& L, const OpDesc& A, int s, const float* in, float* out,
                        const Epi<float>& ep) {
  if (s % 4 != 0 || ep.frob || !out || !aligned16(in) || !aligned16(out)) return cudaErrorNotSupported;
  if (ep.left && (ep.left != in || !ep.sym)) return cudaErrorNotSupported;
  switch (A.kind) {
    case kOpConst7: return march_sw<kMConst7>(L, A, s, in, out, ep);
    case kOpVar7: return march_sw<kMVar7>(L, A, s, in, out, ep);
    case kOpEdge5: return march_sw<kMEdge5>(L, A, s, in, out, ep);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t stream_gram4(const Launch& L, int64_t n, int s, const float* X, const float* Y,
                         const Epi<float>& ep) {
  if (s % 4 != 0 || n < 1 || !aligned16(X) || !aligned16(Y)) return cudaErrorNotSupported;
  if (s == 16 || s == 32) {
    cudaError_t e;
    if (s == 16)
      e = ep.sym ? mstream_launch<16, true, false>(L, n, X, Y, nullptr, nullptr, ep)
                 : mstream_launch<16, false, false>(L, n, X, Y, nullptr, nullptr, ep);
    else
      e = ep.sym ? mstream_launch<32, true, false>(L, n, X, Y, nullptr, nullptr, ep)
                 : mstream_launch<32, false, false>(L, n, X, Y, nullptr, nullptr, ep);
    if (e != cudaErrorNotSupported) return e;
  }
  if (s == 4 || s == 8 || s == 16) {
    if (ep.sym) return rstream_sw<0, true>(L, n, s, X, Y, nullptr, nullptr, ep);
    return rstream_sw<0, false>(L, n, s, X, Y, nullptr, nullptr, ep);
  }
  if (ep.sym) return stream_sw<0, kQEpiSym>(L, n, s, X, Y, nullptr, nullptr, ep);
  return stream_sw<0, kQEpiFull>(L, n, s, X, Y, nullptr, nullptr, ep);
}

cudaError_t stream_diag4(const Launch& L, int64_t n, int s, const float* w, const float* X, float* Z,
                         const Epi<float>& ep) {
  if (s % 4 != 0 || n < 1 || !ep.sym || ep.left != X || !aligned16(X) || !aligned16(Z))
    return cudaErrorNotSupported;
  if (s == 16 || s == 32) {
    const cudaError_t e = s == 16 ? mstream_launch<16, true, true>(L, n, X, X, w, Z, ep)
                                  : mstream_launch<32, true, true>(L, n, X, X, w, Z, ep);
    if (e != cudaErrorNotSupported) return e;
  }
  if (s == 4 || s == 8 || s == 16) return rstream_sw<1, true>(L, n, s, X, nullptr, w, Z, ep);
  return stream_sw<1, kQEpiSym>(L, n, s, X, nullptr, w, Z, ep);
}

// Per-cell coefficient quadruples of the marching kernel (FP32): VAR7
// (diag, face to +x, face to +y, face to +z); EDGE5 (diag, edge to -x, edge
// to -y, 0).
__global__ void coef4_var7_kernel(int64_t n, const float* __restrict__ c32, float4* __restrict__ out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    out[r] = make_float4(c32[r], c32[n + r], c32[2 * n + r], c32[3 * n + r]);
}
__global__ void coef4_edge5_kernel(int nx, int ny, const float* __restrict__ diag, const float* __restrict__ e,
                                   float4* __restrict__ out) {
  const int64_t n = (int64_t)nx * ny;
  const float* ax = e;
  const float* ay = e + (int64_t)ny * (nx + 1);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(r % nx), y = (int)(r / nx);
    out[r] = make_float4(diag[r], ax[(int64_t)y * (nx + 1) + x], ay[(int64_t)y * nx + x], 0.f);
  }
}

cudaError_t op_make_coef4(const Launch& L, OpDesc& A) {
  if (A.coef4 || (A.kind != kOpVar7 && A.kind != kOpEdge5)) return cudaSuccess;
  if (!A.coef32 || (A.kind == kOpEdge5 && !A.edges32)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMalloc(&A.coef4, sizeof(float4) * (size_t)A.n);
  if (e != cudaSuccess) return e;
  const int grid = L.sms * 4;
  if (A.kind == kOpVar7)
    coef4_var7_kernel<<<grid, 256, 0, L.stream>>>(A.n, A.coef32, reinterpret_cast<float4*>(A.coef4));
  else
    coef4_edge5_kernel<<<grid, 256, 0, L.stream>>>(A.nx, A.ny, A.coef32, A.edges32,
                                                   reinterpret_cast<float4*>(A.coef4));
  return cudaGetLastError();
}

}  // namespace bk
