// bt_precond_grad_noalloc: the preconditioner-network gradient of
// bt_precond_eval for callers that cannot allocate device memory -- code under
// a framework that owns every device allocation (a caching allocator or a
// fixed memory budget that cudaMalloc would bypass), or a service that forbids
// allocation after start-up because cudaMalloc/cudaFree synchronise the device.
// It uses no cudaMalloc/cudaFree and no allocating library routine: its scratch
// is the file-scope array below, whose device address is looked up once per
// device.  That address belongs to the device's primary context; after a
// cudaDeviceReset the cached address is stale, so a process that resets a
// device must not call this entry point on it again.
#include <mutex>

#include "bt_kernels.cuh"

using namespace bt;

namespace {

constexpr int NA_MAX_SAMPLES = BT_NOALLOC_MAX_SAMPLES;
constexpr int NA_ACT = MLP_IN + 4 * MLP_H + MLP_OUT;  // per-sample scratch floats
// layout (in floats): activations [NA_MAX_SAMPLES][NA_ACT], sample indices
// [NA_MAX_SAMPLES] (int), bfloat16 weights [MLP_NPARAM / 2 + 1]
constexpr size_t NA_FLOATS = (size_t)NA_MAX_SAMPLES * NA_ACT + NA_MAX_SAMPLES + MLP_NPARAM / 2 + 1;

// Every call on a device shares this array (about 2.2 MB, held by every GPU
// that loads the library until the process exits).
static __device__ __align__(256) float g_noalloc_scratch[NA_FLOATS];

std::mutex g_mu;
void* g_addr[64] = {};  // device address of g_noalloc_scratch, per device

__global__ void k_prepare(const float* __restrict__ w, __nv_bfloat16* __restrict__ w16, int* __restrict__ idx, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < MLP_NPARAM) w16[i] = __float2bfloat16_rn(w[i]);
  if (i < n) idx[i] = i;
}

}  // namespace

extern "C" bt_status bt_precond_grad_noalloc(const float* w, int32_t n, const float* feat, const float* G,
                                             const float* h, double* grad, float* loss, void* stream) {
  if (n < 1 || n > NA_MAX_SAMPLES || !w || !feat || !G || !h || !grad || !loss) return BT_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BT_ECUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      // first call on this device: resolve the symbol's device address
      if (cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch) != cudaSuccess) {
        g_addr[dev] = nullptr;
        return BT_ECUDA;
      }
    }
    base = g_addr[dev];
  }
  float* s = static_cast<float*>(base);
  const size_t A = (size_t)NA_MAX_SAMPLES;
  MlpTrainArgs a{};
  a.sx = s;
  a.sa1 = s + A * MLP_IN;
  a.sa2 = a.sa1 + A * MLP_H;
  a.sd1 = a.sa2 + A * MLP_H;
  a.sd2 = a.sd1 + A * MLP_H;
  a.sdc = a.sd2 + A * MLP_H;
  int* idx = reinterpret_cast<int*>(a.sdc + A * MLP_OUT);
  __nv_bfloat16* w16 = reinterpret_cast<__nv_bfloat16*>(idx + A);
  cudaStream_t st = (cudaStream_t)stream;
  // a launch error left pending by the caller's own earlier work would be
  // indistinguishable from ours: refuse to run on top of it (it stays pending)
  if (cudaPeekAtLastError() != cudaSuccess) return BT_ECUDA;
  // nothing in the scratch has to start at zero: every value the kernels read
  // is written earlier in the same call
  k_prepare<<<(MLP_NPARAM > n ? MLP_NPARAM : n) / 256 + 1, 256, 0, st>>>(w, w16, idx, n);
  if (cudaGetLastError() != cudaSuccess) return BT_ECUDA;
  a.w32 = nullptr;
  a.w16 = w16;
  a.m = a.v = nullptr;
  a.feat = feat;
  a.G = G;
  a.h = h;
  a.idx = idx;
  a.B = n;
  a.loss = loss;
  a.grad_out = grad;
  a.apply = 0;
  launch_mlp_train(a, st);
  return cudaGetLastError() == cudaSuccess ? BT_OK : BT_ECUDA;  // only this call's launches since the check above
}
