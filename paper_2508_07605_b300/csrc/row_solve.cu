// Fused masked-Gram + Cholesky row solve (one ALS half-step).
//
// For every row i of a CSR matrix (a new application, an offline application,
// or -- on the CSC copy -- a setting), with F the fixed other factor:
//     A_i = sum_{j in Omega_i} f_j f_j^T + lambda I,   b_i = sum_{j in Omega_i} R_ij f_j,
//     A_i = L L^T,  L y = b_i,  L^T x_i = y.
// This is the per-row ridge solve of alternating least squares (the matrix
// factorisation model of collaborative filtering the paper builds on, Sec.
// "Collaborative Filtering Model"; the online fold-in of new rows of Sec.
// "Online Performance Prediction").
//
// Mapping (WPS warps per system; WPS = 1 for short rows, 4 for long rows):
//   * Staging: each warp takes 32 observations at a time; lane t loads
//     (j_t, R_t) and the whole factor row f_{j_t} (KP elements, 16-byte loads)
//     into a padded, bank-conflict-free shared-memory tile.  All 32 rows are
//     in flight at once, so global latency is paid once per 32 observations.
//   * Gram: the warp is G = 32/KP groups of KP lanes; group g takes the staged
//     observations t = g, g+G, ...; lane q of a group owns row q of A (KP
//     registers) and adds f_t[q] * f_t from 16-byte broadcast shared loads.
//     Groups (and, for WPS = 4, warps through shared memory in a fixed order)
//     are summed at the end.
//   * Cholesky: right-looking, fully unrolled over the pivot p; column p of L
//     is exchanged through a double-buffered shared vector, the rank-1 update
//     stays in registers.  Forward substitution by shuffles, back substitution
//     from a shared copy of L (stride KP+1, conflict-free).
// A never touches HBM: per row the kernel reads the CSR row and s factor rows
// and writes one factor row.
#include "common.cuh"
#include "kernels.h"
#include "solve_warp.cuh"

namespace ocf {

template <typename TV, typename TC, int KP, int WPS>
__global__ void __launch_bounds__(WPS == 1 ? 256 : 32 * WPS)
k_row_solve(SolveArgs<TV> a) {
    const int WARPS = (WPS == 1) ? (int)(blockDim.x >> 5) : WPS;   // WPS = 1: 1 .. 8 warps
    using WS = WarpSmem<TV, TC, KP>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WS *smem = reinterpret_cast<WS *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    // WPS == 1: one system per warp; WPS > 1: one system per CTA.
    const int64_t sys0 = (WPS == 1) ? (int64_t)blockIdx.x * WARPS + warp : (int64_t)blockIdx.x;
    const int64_t sys_stride = (WPS == 1) ? (int64_t)gridDim.x * WARPS : (int64_t)gridDim.x;
    const int64_t M = a.m_dev ? *a.m_dev : a.m;   // systems (a device count for compacted lists)
    for (int64_t i = sys0; i < M; i += sys_stride)
        solve_system<TV, TC, KP, WPS>(a, a.row_map ? a.row_map[i] : i, smem, warp, lane);
}

template <typename TV, typename TC, int KP, int WPS>
static size_t smem_bytes() {
    constexpr int WARPS = (WPS == 1) ? 8 : WPS;
    return sizeof(WarpSmem<TV, TC, KP>) * WARPS;
}

template <typename TV, typename TC, int KP, int WPS>
static cudaError_t set_attr() {
    return cudaFuncSetAttribute(k_row_solve<TV, TC, KP, WPS>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes<TV, TC, KP, WPS>());
}

template <typename TV, typename TC>
static cudaError_t set_attrs_tv() {
    cudaError_t e;
    if ((e = set_attr<TV, TC, 8, 1>()) != cudaSuccess) return e;
    if ((e = set_attr<TV, TC, 16, 1>()) != cudaSuccess) return e;
    if ((e = set_attr<TV, TC, 32, 1>()) != cudaSuccess) return e;
    if ((e = set_attr<TV, TC, 8, 4>()) != cudaSuccess) return e;
    if ((e = set_attr<TV, TC, 16, 4>()) != cudaSuccess) return e;
    return set_attr<TV, TC, 32, 4>();
}

cudaError_t prepare_row_solve() {
    cudaError_t e;
    if ((e = set_attrs_tv<float, float>()) != cudaSuccess) return e;
    if ((e = set_attrs_tv<float, double>()) != cudaSuccess) return e;
    return set_attrs_tv<double, double>();
}

// Observations per system above which a system gets a CTA of 4 warps.
constexpr int64_t LONG_ROW = 96;

// Systems per launch up to which an FP64 factorisation gets a CTA of 4 warps
// per system whatever its row length.
constexpr int64_t SMALL_FP64 = 4 * NUM_SMS_HINT;

template <typename TV, typename TC, int KP>
static cudaError_t launch_kp(const SolveArgs<TV> &a, cudaStream_t st) {
    // The B300's FP64 rate is low enough that one warp's FP64 Gram of a long-ish
    // row is a long chain on one SM sub-partition; in a small FP64 batch each
    // system's Gram is split over 4 warps (the 4 sub-partitions of an SM).
    const bool small_fp64 = sizeof(TC) == 8 && a.m <= SMALL_FP64;
    const bool long_rows = a.nnz >= LONG_ROW * a.m || small_fp64;
    if (long_rows) {
        int64_t blocks = a.m;
        if (blocks > NUM_SMS_HINT * 64) blocks = NUM_SMS_HINT * 64;
        k_row_solve<TV, TC, KP, 4>
            <<<(unsigned)blocks, 128, smem_bytes<TV, TC, KP, 4>(), st>>>(a);
    } else {
        // Small batches are spread over the SMs, fewer warps per CTA: 64 systems
        // in 8-warp CTAs would load 8 SMs and leave the rest idle.
        int wpc = 8;
        const int64_t per_sm = (a.m + NUM_SMS_HINT - 1) / NUM_SMS_HINT;
        if (per_sm < 8) wpc = (int)(per_sm < 1 ? 1 : per_sm);
        int64_t blocks = (a.m + wpc - 1) / wpc;
        if (blocks > NUM_SMS_HINT * 32) blocks = NUM_SMS_HINT * 32;
        k_row_solve<TV, TC, KP, 1><<<(unsigned)blocks, 32 * wpc,
                                     sizeof(WarpSmem<TV, TC, KP>) * wpc, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename TV, typename TC>
cudaError_t launch_row_solve(const SolveArgs<TV> &a, int KP, cudaStream_t st) {
    if (a.m <= 0) return cudaSuccess;
    switch (KP) {
        case 8: return launch_kp<TV, TC, 8>(a, st);
        case 16: return launch_kp<TV, TC, 16>(a, st);
        case 32: return launch_kp<TV, TC, 32>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_row_solve<float, float>(const SolveArgs<float> &, int, cudaStream_t);
template cudaError_t launch_row_solve<float, double>(const SolveArgs<float> &, int, cudaStream_t);
template cudaError_t launch_row_solve<double, double>(const SolveArgs<double> &, int,
                                                      cudaStream_t);

}  // namespace ocf
