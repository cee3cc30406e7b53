// selfcheck.cu — the bounded device wait, made to run out on purpose.
//
// Every wait of this library's kernels (a packet's TMA copy landing on its
// mbarrier) is bounded: after its limit the kernel records THAPI_E_TIMEOUT in
// a status word the host reads, and the context stays usable.  Here one warp
// waits on an mbarrier that nothing ever completes (no copy is issued, no
// thread arrives), so the wait gives up after `limit` tries and the status
// comes back as THAPI_E_TIMEOUT: the failure path, exercised without a fault.
#include "device_util.cuh"
#include "internal.cuh"

namespace thapi {

namespace {

__global__ void k_wait_runs_out(uint32_t limit, unsigned *status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    dev::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const bool landed = dev::mbar_wait_limit(&bar, 0u, limit);  // phase 0 never completes
  if (threadIdx.x == 0) *status = landed ? (unsigned)THAPI_OK : (unsigned)THAPI_E_TIMEOUT;
}

}  // namespace

cudaError_t launch_wait_check(uint32_t limit, unsigned *status, cudaStream_t s) {
  k_wait_runs_out<<<1, 32, 0, s>>>(limit, status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace thapi
