// Allocation-free CSR -> CSC transpose (FP32 values).
//
// Same stable counting sort as open_cf_csr_to_csc, for callers that must not
// allocate device memory themselves or through this library: programs whose
// host framework owns every device allocation through its own pool and forbids
// direct cudaMalloc, services that cannot afford the implicit device-wide
// synchronisation of cudaMalloc/cudaFree on their latency path, and code
// started with a fixed device-memory budget.  The counting sort's scratch (the
// per-row-block column counters and the column totals) lives in one
// file-scope device array of fixed size instead of a handle workspace.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "open_cf.h"

namespace {

constexpr size_t kScratchBytes = OPEN_CF_NOALLOC_SCRATCH_BYTES;

// Every device that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch on the current device.  The host-side symbol
// is only a stand-in, so the address is looked up on every call (a host-side
// query that allocates nothing), which stays right after a device reset; the
// sort kernels' shared-memory limit is raised on every call for the same
// reason.  The first call on a device also loads the library's module there.
int scratch_address(void **scratch) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return OPEN_CF_CUDA_ERROR;
    }
    e = ocf::prepare_csr_to_csc(ocf::CSC_MAX_N);   // the same limit a handle sets
    if (e != cudaSuccess) {
        cudaGetLastError();
        return OPEN_CF_CUDA_ERROR;
    }
    *scratch = p;
    return OPEN_CF_OK;
}

}  // namespace

extern "C" int open_cf_csr_to_csc_noalloc(int64_t m, int64_t n, int64_t nnz,
                                          const int64_t *row_ptr, const int32_t *col,
                                          const float *val, int64_t *col_ptr, int32_t *row_idx,
                                          float *cval, void *stream) {
    if (m < 0 || nnz < 0 || n <= 0) return OPEN_CF_INVALID_ARG;
    if ((m > 0 && !row_ptr) || !col_ptr) return OPEN_CF_INVALID_ARG;
    if (nnz > 0 && (!col || !val || !row_idx || !cval)) return OPEN_CF_INVALID_ARG;
    // The column totals (8 bytes per column) and at least one row block of
    // counters (4 bytes per column) must fit the fixed scratch; the sort's
    // shared-memory counters bound n as they do for the handle path.
    if (n > OPEN_CF_NOALLOC_MAX_COLUMNS) return OPEN_CF_UNSUPPORTED;
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != OPEN_CF_OK) return rc;

    int64_t *tot = reinterpret_cast<int64_t *>(scratch);
    const size_t tot_bytes = ((sizeof(int64_t) * (size_t)n + 255) / 256) * 256;
    int32_t *cnt = reinterpret_cast<int32_t *>(static_cast<unsigned char *>(scratch) + tot_bytes);
    const int64_t max_nb = (int64_t)((kScratchBytes - tot_bytes) / (sizeof(int32_t) * (size_t)n));
    if (max_nb < 1) return OPEN_CF_UNSUPPORTED;
    // Fewer row blocks than the handle path would use when n is large
    // (max_nb = 254 at n = 4096, 39 at n = 25,000): each block then walks
    // more rows, so the sort is slower there, never wrong.
    const ocf::CscPlan plan = ocf::csc_plan(m, n, nnz, max_nb);
    // Every counter and total the kernels read is written earlier in the same
    // call, so nothing left from a previous call needs clearing.
    cudaError_t e = ocf::launch_csr_to_csc<float>(m, n, nnz, row_ptr, col, val, col_ptr, row_idx,
                                                  cval, cnt, tot, plan,
                                                  reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return OPEN_CF_CUDA_ERROR;
    }
    return OPEN_CF_OK;
}
