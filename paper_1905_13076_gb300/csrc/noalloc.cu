// Allocation-free variant of the batched harmonic solve.
//
// Some callers cannot allocate device memory: plugins that only receive
// buffers from a host application owning every allocation, or loops where
// cudaMalloc's implicit device synchronisation is not acceptable.  This
// entry point runs the same batched COCG kernel as the PP-PC coarse solve on
// a caller-supplied sparse pattern, with all of its work vectors taken from
// one file-scope device array instead of from cudaMalloc.
//
// The array is a fixed kNoAllocScratchBytes.  Every GPU that loads this
// library holds that much memory until the process exits.  All calls share
// it and it keeps the contents of the last call, so everything that must
// start at zero is cleared by each call, and calls that overlap on the GPU
// (different streams, or different host threads on one device) race.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/pppc.h"
#include "args.h"
#include "common.cuh"
#include "kernels.h"

namespace pppc {
namespace {

constexpr size_t kNoAllocScratchBytes = PPPC_NOALLOC_SCRATCH_BYTES;  // 12 MiB
constexpr int kNoAllocMaxN = PPPC_NOALLOC_MAX_N;
constexpr long long kNoAllocMaxUnknowns = PPPC_NOALLOC_MAX_UNKNOWNS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

// Host-side device addresses of g_scratch, looked up once per device.
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

inline size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// Pass 1 over the caller's pattern: rowptr must start at 0 and never
// decrease.  Only rowptr[0..n] is read.  Until this has passed, the row
// ranges cannot be trusted to stay inside col[], so nothing reads col.
__global__ void noalloc_check_rowptr_kernel(int n, const int* rowptr, int* status) {
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int a = rowptr[i], b = rowptr[i + 1];
        if ((i == 0 && a != 0) || b < a) atomicCAS(status, 0, 1);
    }
}

// Pass 2, once rowptr is known to be valid: every column index must lie in
// [0, n) and every row must hold its diagonal.  An out-of-range index is
// only compared, never used to address memory.
__global__ void noalloc_setup_kernel(int n, int N, const int* rowptr, const int* col, int* row_slot,
                                     int* sp_index, int* diag_k, double* tw, int* status) {
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        row_slot[i] = rowptr[i];
        sp_index[i] = i;
        int dk = -1;
        bool ok = true;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int c = col[k];
            if (c < 0 || c >= n) ok = false;
            if (c == i) dk = k;
        }
        if (dk < 0 || !ok) {
            atomicCAS(status, 0, 1);
            dk = rowptr[i];  // never used: the host stops on the status
        }
        diag_k[i] = dk;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += stride) {
        double s, c;
        sincospi(2.0 * (double)k / (double)N, &s, &c);
        tw[2 * k] = c;
        tw[2 * k + 1] = -s;
    }
}

}  // namespace
}  // namespace pppc

using namespace pppc;

extern "C" pppc_status pppc_harmonic_solve_noalloc(int32_t n, const int32_t* rowptr, const int32_t* col,
                                                   const double* kval, const double* cval, int32_t N,
                                                   const double* b, double* x, double tol, int32_t max_it,
                                                   void* stream, int32_t* iters_out) {
    if (n < 1 || !rowptr || !col || !kval || !cval || !b || !x) return PPPC_ERR_INVALID_ARG;
    if (N < 2 || (N % 2) != 0 || N > kNoAllocMaxN) return PPPC_ERR_INVALID_ARG;
    if (!(tol > 0.0) || max_it < 1) return PPPC_ERR_INVALID_ARG;
    const int H = N / 2 + 1;
    if ((long long)n * H > kNoAllocMaxUnknowns) return PPPC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PPPC_ERR_CUDA;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return PPPC_ERR_CUDA;
            }
            g_scratch_addr[dev] = ptr;
        }
        base = g_scratch_addr[dev];
    }

    LaunchCfg cfg;
    if (cocg_config(false, H, &cfg) != cudaSuccess) return PPPC_ERR_CUDA;

    // carve the scratch array
    const size_t vec = (size_t)n * H * 2 * sizeof(double);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void* p = static_cast<unsigned char*>(base) + off;
        off += align_up(bytes);
        return p;
    };
    int* row_slot = static_cast<int*>(take((size_t)n * sizeof(int)));
    int* sp_index = static_cast<int*>(take((size_t)n * sizeof(int)));
    int* diag_k = static_cast<int*>(take((size_t)n * sizeof(int)));
    double* tw = static_cast<double*>(take(2 * (size_t)N * sizeof(double)));
    void* r = take(vec);
    void* z = take(vec);
    void* w = take(vec);
    void* p = take(vec);
    void* s = take(vec);
    void* invd = take(vec);
    double* part = static_cast<double*>(take(2 * (size_t)cfg.blocks * 5 * H * sizeof(double)));
    GridBarrier* bar = static_cast<GridBarrier*>(take(sizeof(GridBarrier)));
    int* status = static_cast<int*>(take(sizeof(int)));
    long long* counters = static_cast<long long*>(take(3 * sizeof(long long)));
    if (off > kNoAllocScratchBytes) return PPPC_ERR_INVALID_ARG;

    // state that must start at zero
    if (cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(counters, 0, 3 * sizeof(long long), st) != cudaSuccess)
        return PPPC_ERR_CUDA;
    // validate the caller's pattern in two passes (rowptr, then col), each
    // read back before anything depends on it
    const int vblocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    int code = 0;
    noalloc_check_rowptr_kernel<<<vblocks, 256, 0, st>>>(n, rowptr, status);
    if (cudaGetLastError() != cudaSuccess) return PPPC_ERR_CUDA;
    if (cudaMemcpyAsync(&code, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PPPC_ERR_CUDA;
    if (code != 0) return PPPC_ERR_INVALID_ARG;  // rowptr does not start at 0 or decreases
    noalloc_setup_kernel<<<vblocks, 256, 0, st>>>(n, N, rowptr, col, row_slot, sp_index, diag_k, tw, status);
    if (cudaGetLastError() != cudaSuccess) return PPPC_ERR_CUDA;
    if (cudaMemcpyAsync(&code, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PPPC_ERR_CUDA;
    if (code != 0) return PPPC_ERR_INVALID_ARG;  // a column outside [0, n) or a row without its diagonal

    // every row is "special": its values are kval + c_p * cval, slot = CSR index
    CocgArgs a{};
    a.mesh.ndof = n;
    a.mesh.nnz = 0;
    a.mesh.n_slots = 0;
    a.mesh.n_sp = n;
    a.mesh.rowptr = rowptr;
    a.mesh.col = col;
    a.mesh.diag_k = diag_k;
    a.mesh.row_slot = row_slot;
    a.mesh.sp_index = sp_index;
    a.mesh.Klin = kval;
    a.mesh.invdiag_lin = kval;
    a.mesh.Mslot = cval;
    a.N = N;
    a.H = H;
    a.inv_dT = 1.0;
    a.tol = tol;
    a.max_it = max_it;
    a.Kbar = kval;
    a.tw = tw;
    a.b = b;
    a.x = x;
    a.r = r;
    a.z = z;
    a.w = w;
    a.p = p;
    a.s = s;
    a.invd_sp = invd;
    a.part = part;
    a.bar = bar;
    a.status = status;
    a.counters = counters;
    if (launch_cocg(a, false, cfg, st) != cudaSuccess) return PPPC_ERR_CUDA;
    long long its[3] = {0, 0, 0};
    if (cudaMemcpyAsync(&code, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(its, counters, sizeof its, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PPPC_ERR_CUDA;
    if (iters_out) *iters_out = (int32_t)its[2];
    switch (code) {
        case 0: return PPPC_OK;
        case DEV_ERR_LINEAR: return PPPC_ERR_LINEAR;
        case DEV_ERR_BREAKDOWN: return PPPC_ERR_BREAKDOWN;
        case DEV_ERR_NAN: return PPPC_ERR_NAN;
        case DEV_ERR_TIMEOUT: return PPPC_ERR_TIMEOUT;
        default: return PPPC_ERR_CUDA;
    }
}
