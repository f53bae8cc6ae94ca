// Block inner product G = X^T Y that allocates nothing.
//
// bkrylov_bdot needs a handle, and a handle grows a device workspace with
// cudaMalloc.  Some callers cannot allocate device memory at the point where
// they need a Gram matrix: code that runs under a fixed device-memory budget
// (a host framework that reserved all device memory up front and hands out
// only its own buffers), or a latency-critical loop in which an allocation
// could block or fail.  This entry point serves them: the caller passes the
// inputs, the output and a stream, and every piece of scratch (per-CTA
// partial sums, the reduced s x s matrix, the ticket words of the
// last-CTA reduction) lives in the file-scope device array below, which every
// GPU that loads the library keeps until the process exits (4.2 MB).
#include <mutex>

#include "bk_common.cuh"
#include "bk_internal.h"

namespace {

using namespace bk;

constexpr int kNaMaxCtas = 512;                               // reduction grid limit
constexpr size_t kNaPartials = (size_t)kNaMaxCtas * kMM;      // partial Grams (<= s*s each)
constexpr size_t kNaResult = kNaPartials;                     // reduced Gram, row stride 32
constexpr size_t kNaCounter = kNaPartials + kMM;              // ticket words (kTicketWords)
constexpr size_t kNaDoubles = kNaPartials + kMM + kTicketWords / 2;

static __device__ __align__(256) double g_bdot_scratch[kNaDoubles];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
double* g_na_addr[kNaMaxDevices] = {};

// Device address of g_bdot_scratch on the current device, looked up once per
// device (the host-side name of the array is only a stand-in, never a device
// address).
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return BK_ERR_CUDA;
  if (dev < 0 || dev >= kNaMaxDevices) return BK_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bdot_scratch) != cudaSuccess || !p) return BK_ERR_CUDA;
    g_na_addr[dev] = static_cast<double*>(p);
  }
  *out = g_na_addr[dev];
  return BK_OK;
}

__global__ void na_compact(int s, const double* __restrict__ in, double* __restrict__ out) {
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) out[i] = in[(i / s) * kMaxS + (i % s)];
}

}  // namespace

extern "C" int bkrylov_bdot_noalloc(int64_t n, int s, const void* X, const void* Y, double* G,
                                    int sym, int prec, void* cuda_stream) {
  if (n <= 0 || s < 1 || s > kMaxS || !X || !Y || !G) return BK_ERR_ARG;
  if (prec != BK_FP64 && prec != BK_FP32) return BK_ERR_ARG;
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != BK_OK) return rc;
  Launch L;
  L.stream = static_cast<cudaStream_t>(cuda_stream);
  L.sms = kNaMaxCtas / kCtasPerSm;   // the row kernels launch at most kCtasPerSm * sms CTAs
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNaCounter);
  // the ticket words must start at zero; the previous call's CTAs reset them,
  // but a call that failed mid-way might not have
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned) * kTicketWords, L.stream) != cudaSuccess) return BK_ERR_CUDA;
  cudaError_t e;
  if (prec == BK_FP64) {
    Epi<double> ep;
    ep.sym = sym ? 1 : 0; ep.gram_out = scratch + kNaResult; ep.gpart = scratch; ep.counter = counter;
    e = gram<double>(L, n, s, static_cast<const double*>(X), static_cast<const double*>(Y), ep);
  } else {
    Epi<float> ep;
    ep.sym = sym ? 1 : 0; ep.gram_out = scratch + kNaResult; ep.gpart = scratch; ep.counter = counter;
    e = gram<float>(L, n, s, static_cast<const float*>(X), static_cast<const float*>(Y), ep);
  }
  if (e != cudaSuccess) return BK_ERR_CUDA;
  na_compact<<<1, 256, 0, L.stream>>>(s, scratch + kNaResult, G);
  return cudaGetLastError() == cudaSuccess ? BK_OK : BK_ERR_CUDA;
}
