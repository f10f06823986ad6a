// fptc_check_bounded_wait (include/fptc.h): the bounded mbarrier wait that
// every tensor-core and TMA completion wait of the decoder uses
// (warp_tile.cuh mbar_wait), run on its own, so that its give-up path can be
// exercised on a GPU without a fault: one CTA waits on an mbarrier in its
// shared memory that either one of its threads arrives on (the wait
// completes) or nothing arrives on (the wait gives up after its 1 s bound and
// the kernel sets FPTC_FLAG_TIMEOUT in a status word, as the decode kernels
// do).  No other work is in flight, so giving up leaves nothing behind.
#include "fptc.h"
#include "fptc_internal.h"
#include "host_util.h"
#include "warp_tile.cuh"

namespace fptc {
namespace {

using namespace wt;

__global__ void __launch_bounds__(32) k_wait_check(uint32_t *flags, int arrive) {
  __shared__ uint64_t bar;
  const uint32_t a = smem_addr(&bar);
  if (threadIdx.x == 0) {
    mbar_init(a, 1u);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (arrive && threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
  const bool done = mbar_wait(a, 0u);
  if (!done && threadIdx.x == 0) atomicOr(flags, FPTC_FLAG_TIMEOUT);
  __syncwarp();
}

}  // namespace
}  // namespace fptc

using namespace fptc;

extern "C" fptc_status fptc_check_bounded_wait(int device, int arrive, uint32_t *flags) {
  return guarded([&]() -> fptc_status {
    clear_error();
    if (!flags) {
      set_error("flags is NULL");
      return FPTC_ERR_INVALID_ARGUMENT;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaError_t e = cudaSetDevice(device);
    uint32_t *d_flags = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_flags, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(d_flags, 0, sizeof(uint32_t));
    if (e == cudaSuccess) {
      k_wait_check<<<1, 32>>>(d_flags, arrive);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(flags, d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    cudaFree(d_flags);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
      set_error("bounded-wait check: %s", cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? FPTC_ERR_OUT_OF_MEMORY : FPTC_ERR_CUDA;
    }
    return FPTC_OK;
  });
}
