// Algorithm 1 (phase-transition detection, Sec. "Online Performance
// Prediction") over many monitored power traces at once.
//
// The algorithm keeps the last N = W / delta GPU power readings in a circular
// buffer and reports a transition on the reading that fills the buffer with N
// values none of which is below P_th (the five 1-second intervals it checks
// cover the buffer, so the interval split does not change the answer).  That
// is: the first reading s that ends a run of N consecutive readings that are
// not below P_th.  Per trace, one warp scans the readings 32 at a time:
// __ballot_sync marks the readings below P_th, the run length ending at each
// lane follows from the highest such mark at or before it (or from the run
// carried in from the previous 32), and the first lane whose run reaches N is
// the answer.  A reading that is not a number is not below P_th, as in the
// algorithm's comparison.  Reads are coalesced 128-byte rows, sixteen of
// them in flight per warp; a warp stops reading its trace at the first report.
#include "common.cuh"
#include "kernels.h"

namespace ocf {

namespace {

constexpr int PH_WARPS = 8;
constexpr int PH_UNROLL = 16;

__global__ void __launch_bounds__(PH_WARPS * 32)
k_phase_detect(const float *__restrict__ power, int64_t n_traces, int64_t len, int64_t ld,
               float p_th, int32_t N, int64_t *__restrict__ first) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * PH_WARPS + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * PH_WARPS;
    const uint32_t le_mask = 0xFFFFFFFFu >> (31 - lane);   // lanes 0 .. lane
    for (int64_t t = w0; t < n_traces; t += nw) {
        const float *pw = power + t * ld;
        int64_t run = 0;   // readings not below p_th ending just before this block
        int64_t found = -1;
        for (int64_t c0 = 0; c0 < len && found < 0; c0 += 32 * PH_UNROLL) {
            float p[PH_UNROLL];
#pragma unroll
            for (int u = 0; u < PH_UNROLL; ++u) {
                const int64_t s = c0 + 32 * u + lane;
                p[u] = s < len ? __ldg(pw + s) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < PH_UNROLL; ++u) {
                const int64_t s0 = c0 + 32 * u;
                if (found >= 0 || s0 >= len) break;   // warp-uniform
                const int64_t s = s0 + lane;
                const bool below = !(s < len) || p[u] < p_th;
                const uint32_t fails = __ballot_sync(FULL, below);
                const uint32_t f_le = fails & le_mask;
                const int64_t run_l = f_le ? (int64_t)(lane - (31 - __clz(f_le))) : run + lane + 1;
                const uint32_t hit = __ballot_sync(FULL, run_l >= (int64_t)N);
                if (hit) {
                    found = s0 + (__ffs(hit) - 1);
                } else {
                    run = fails ? (int64_t)(31 - (31 - __clz(fails))) : run + 32;
                }
            }
        }
        if (lane == 0) first[t] = found;
    }
}

}  // namespace

cudaError_t launch_phase_detect(const float *power, int64_t n_traces, int64_t len, int64_t ld,
                                float p_th, int32_t window, int64_t *first, cudaStream_t st) {
    if (n_traces <= 0) return cudaSuccess;
    int64_t blocks = (n_traces + PH_WARPS - 1) / PH_WARPS;
    if (blocks > NUM_SMS_HINT * 8) blocks = NUM_SMS_HINT * 8;
    k_phase_detect<<<(unsigned)blocks, PH_WARPS * 32, 0, st>>>(power, n_traces, len, ld, p_th,
                                                               window, first);
    return cudaGetLastError();
}

}  // namespace ocf
