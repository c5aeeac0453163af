// dvm_selftest.cu -- self-test of the device-side failure detection: the
// bounded waits of the library's kernels give up with DVM_ERR_TIMEOUT in the
// status word instead of hanging, and the context stays usable.  Each case
// runs the library's own wait on something that never happens:
//   DVM_SELFTEST_GRID_BARRIER: the grid barrier of the Euler launches, with
//     one of two blocks leaving without arriving (about 1 s);
//   DVM_SELFTEST_MBARRIER: the mbarrier wait of the tensor-core kernels on a
//     barrier nobody arrives at (about 1 s).
#include "dvm_internal.cuh"
#include "dvm_math.cuh"
#include "dvm_tc.cuh"

namespace dvm {
namespace {

__global__ void k_selftest_grid(unsigned long long* bar, int* status) {
  if (blockIdx.x == 1) return;  // never arrives
  grid_sync(bar, status);
}

__global__ void k_selftest_mbar(int* status) {
  __shared__ uint64_t mbar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&mbar, 0)) set_status(status, DVM_ERR_TIMEOUT);
}

}  // namespace
}  // namespace dvm

extern "C" int dvm_selftest_timeout(int which, void* cuda_stream, int* status) {
  using namespace dvm;
  if (!status || (which != DVM_SELFTEST_GRID_BARRIER && which != DVM_SELFTEST_MBARRIER)) return DVM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned* scratch = nullptr;  // barrier count (2 words), status
  if (cudaMalloc((void**)&scratch, 4 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return DVM_ERR_OOM;
  }
  int rc = 0;
  int* st = reinterpret_cast<int*>(scratch + 2);
  if (cudaMemsetAsync(scratch, 0, 4 * sizeof(unsigned), s) != cudaSuccess) rc = DVM_ERR_CUDA;
  if (!rc) {
    if (which == DVM_SELFTEST_GRID_BARRIER) k_selftest_grid<<<2, 64, 0, s>>>(reinterpret_cast<unsigned long long*>(scratch), st);
    else k_selftest_mbar<<<1, 32, 0, s>>>(st);
    int host = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&host, st, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = DVM_ERR_CUDA;
    else
      *status = host;
  }
  cudaGetLastError();
  cudaFree(scratch);
  return rc;
}
