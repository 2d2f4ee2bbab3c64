// Failure-detection self-test: a kernel whose pipeline-style wait can never complete, so
// that callers (and the library's tests) can watch a bounded device wait give up and
// surface through conet_sync as CONET_ERR_TIMEOUT, with the context still usable.
#include "common.cuh"
#include "net.cuh"
#include "tc.cuh"

namespace conet {
namespace {

constexpr int SELFTEST_SITE = 100;   // the site number conet_sync reports for this wait

// One thread initialises an mbarrier that expects one arrival and waits for its first phase
// with the same bounded wait the tensor-core pipelines use; nothing ever arrives, so the
// wait gives up after limit_ns, records the site and the kernel returns.
__global__ void selftest_timeout_kernel(int* err, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  tc::fence_mbar_init();
  tc::mbar_wait_for(&bar, 0u, err, SELFTEST_SITE, limit_ns);
}

}  // namespace
}  // namespace conet

using namespace conet;

extern "C" int conet_selftest_timeout(conet_t h, double limit_s, void* stream) {
  if (!h) return fail(CONET_ERR_ARG, "handle is NULL");
  if (!(limit_s >= 1e-6) || !(limit_s <= 1.0)) return fail(CONET_ERR_ARG, "limit %g s outside [1e-6, 1]", limit_s);
  selftest_timeout_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(h->d_err, (uint64_t)(limit_s * 1e9));
  return check_launch("selftest_timeout_kernel");
}
