// Allocation-free variant of the 3x3 weight-gradient op.
//
// Some callers cannot allocate device memory at the point where they need a weight
// gradient: a real-time receiver or training loop whose memory is planned once at start-up
// (no allocator calls on the latency-critical path), code running while a CUDA graph is
// being captured around it, or embedding code that only ever sees the caller's own
// buffers.  conet_conv3x3_wgrad_noalloc serves them: it takes only inputs and outputs and
// keeps its split partial sums in a fixed array compiled into this library.
//
// That array is a file-scope static __device__ variable of NOALLOC_SCRATCH_FLOATS floats
// (4 MiB of split partials plus 256 KiB of bias partials, about 4.25 MiB): every GPU that
// loads the library holds it until the process exits.  Host code cannot use the array's
// name as a device address, so the first call on each device, with that device current,
// resolves the address once through cudaGetSymbolAddress and caches it; make that first
// call before any stream capture.  The cached address outlives a device reset
// (cudaDeviceReset unloads the module that holds the array), so the entry point must not be
// called on a device after it was reset in the same process.  All calls share the array and it keeps the last call's
// contents: every element a call reads is written by that same call first, and two calls
// that overlap on the GPU (different streams, or different host threads) race on it.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace conet {
namespace {

constexpr size_t NOALLOC_SPLIT_FLOATS = (size_t)1 << 20;                 // 4 MiB of split partials
constexpr size_t NOALLOC_BIAS_FLOATS = (size_t)EW_PART_CTAS * 128;       // bias partial sums
constexpr size_t NOALLOC_SCRATCH_FLOATS = NOALLOC_SPLIT_FLOATS + NOALLOC_BIAS_FLOATS;
constexpr int MAX_DEVICES = 64;

}  // namespace

static __device__ __align__(256) float g_wgrad_scratch[NOALLOC_SCRATCH_FLOATS];

namespace {

float* g_scratch_dev[MAX_DEVICES] = {};
std::mutex g_scratch_mu;

int scratch_address(float** out) {
  int dev = 0;
  CONET_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(CONET_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, MAX_DEVICES);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_wgrad_scratch);
    if (e != cudaSuccess) return check_cuda(e, "cudaGetSymbolAddress(g_wgrad_scratch)");
    g_scratch_dev[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_dev[dev];
  return CONET_OK;
}

}  // namespace
}  // namespace conet

using namespace conet;

extern "C" int conet_conv3x3_wgrad_noalloc(const float* x, const float* dz, int B, int T, int F, int cin, int cout,
                                           float* dW, float* db, void* stream) {
  if (!x || !dz || !dW) return fail(CONET_ERR_ARG, "NULL argument");
  if (B < 1 || T < 1 || F < 1) return fail(CONET_ERR_SHAPE, "empty grid B=%d T=%d F=%d", B, T, F);
  if (cin < 4 || cin > 128 || cin % 4 || cout < 4 || cout > 128 || cout % 4)
    return fail(CONET_ERR_SHAPE, "cin=%d cout=%d: multiples of 4 in 4..128 required", cin, cout);
  const long long M = (long long)B * T * F;
  const size_t need = wgrad_partial_floats(M, cin, cout, 1);
  if (need > NOALLOC_SPLIT_FLOATS)
    return fail(CONET_ERR_SHAPE, "weight gradient needs %zu scratch floats, the static array holds %zu", need,
                NOALLOC_SPLIT_FLOATS);
  float* scratch = nullptr;
  CONET_TRY(scratch_address(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  WgradArgs a = {};
  a.x[0] = x;
  a.g[0] = dz;
  a.dW[0] = dW;
  a.cin_src[0] = cin;
  a.part = scratch;
  a.cin = cin;
  a.cout = cout;
  a.n_br = 1;
  a.T = T;
  a.F = F;
  a.M = M;
  CONET_TRY(launch_wgrad(a, s));
  if (db) {
    float* ew = scratch + NOALLOC_SPLIT_FLOATS;
    CONET_TRY(launch_channel_sums(dz, M, cout, ew, s));
    CONET_TRY(launch_reduce_partials(ew, ew_grid(M), cout, db, 0, s));
  }
  return CONET_OK;
}
