// Normal operator that allocates no device memory.
//
// sqcg_normal_op keeps its odd-parity intermediate (D_oe x) in the context's
// solver workspace, which the library allocates with cudaMalloc on first use.
// Some callers must not allocate at that point: host applications that hand
// the whole device memory to their own allocator or pool up front (a new
// cudaMalloc then fails or breaks their budget), and latency-bound loops that
// cannot accept a cudaMalloc, which may synchronise the device. For them
// sqcg_normal_op_noalloc keeps the intermediate in a fixed array compiled into
// this library instead (g_noalloc_scratch below, 8 MiB, present on every GPU
// that loads the library until the process exits).
#include <mutex>

#include "sqcg_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;

// Scratch for the intermediate colour vector. Shared by every call on a device:
// it keeps the contents of the last call, and calls that overlap on the GPU
// (other streams, other host threads) race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch for each device (host-side name of the
// array is only a stand-in and must never be given to a kernel).
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

int scratch_address(void** out) {
  int dev = 0;
  SQCG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return SQCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    SQCG_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return SQCG_OK;
}

}  // namespace

extern "C" int sqcg_normal_op_noalloc(sqcg_ctx* ctx, double sigma, int prec, const void* x, void* y) {
  if (!ctx || !x || !y || x == y) return SQCG_ERR_INVALID_ARG;
  if (prec != SQCG_F64 && prec != SQCG_F32) return SQCG_ERR_INVALID_ARG;
  const size_t need = (size_t)ctx->g.Vh * 3 * (prec == SQCG_F64 ? sizeof(double2) : sizeof(float2));
  if (need > kScratchBytes) return SQCG_ERR_SCRATCH_TOO_SMALL;
  if (!ctx->have_links) return SQCG_ERR_NO_LINKS;
  void* tmp = nullptr;
  SQCG_TRY(scratch_address(&tmp));
  DslashLaunch L = {};
  L.out_parity = 1;
  L.prec = L.out_prec = prec;
  L.epi = EPI_PLAIN;
  L.in = x;
  L.out = tmp;
  SQCG_TRY(launch_dslash(ctx, L, ctx->stream));
  L.out_parity = 0;
  L.epi = EPI_NORMAL;
  L.in = tmp;
  L.out = y;
  L.y = x;
  L.sigma = sigma;
  return launch_dslash(ctx, L, ctx->stream);
}
