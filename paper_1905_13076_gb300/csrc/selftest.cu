// Failure detection self-test (pppc_selftest_wait_timeout): one block waits,
// with the library's bounded spin, on a flag that nothing sets, so the wait
// runs out and the timeout status comes back to the host.  Also the build
// query pppc_binary_version.
#include <cuda_runtime.h>

#include "../../include/pppc.h"
#include "args.h"
#include "common.cuh"

namespace pppc {
namespace {

__global__ void wait_selftest_kernel(const unsigned int* flag, int* status) {
    if (threadIdx.x == 0) spin_until([&] { return ld_acquire_u32(flag) != 0u; }, status);
}

}  // namespace
}  // namespace pppc

extern "C" pppc_status pppc_binary_version(int32_t* out) {
    if (!out) return PPPC_ERR_INVALID_ARG;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, pppc::wait_selftest_kernel) != cudaSuccess) {
        cudaGetLastError();
        return PPPC_ERR_CUDA;
    }
    *out = fa.binaryVersion;
    return PPPC_OK;
}

extern "C" pppc_status pppc_selftest_wait_timeout(void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* mem = nullptr;
    if (cudaMalloc(&mem, 8) != cudaSuccess) {
        cudaGetLastError();
        return PPPC_ERR_NOMEM;
    }
    unsigned int* flag = static_cast<unsigned int*>(mem);
    int* status = reinterpret_cast<int*>(flag + 1);
    int code = -1;
    bool ok = cudaMemsetAsync(mem, 0, 8, st) == cudaSuccess;
    if (ok) {
        pppc::wait_selftest_kernel<<<1, 32, 0, st>>>(flag, status);
        ok = cudaGetLastError() == cudaSuccess &&
             cudaMemcpyAsync(&code, status, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
             cudaStreamSynchronize(st) == cudaSuccess;
    }
    cudaFree(mem);
    if (!ok) {
        cudaGetLastError();
        return PPPC_ERR_CUDA;
    }
    return code == pppc::DEV_ERR_TIMEOUT ? PPPC_ERR_TIMEOUT : PPPC_ERR_CUDA;
}
