// Algorithm 1 (phase-transition detection, Sec. "Online Performance
// Prediction") over many monitored power traces at once.
//
// The algorithm keeps the last N = W / delta GPU power readings in a circular
// buffer and reports a transition on the reading that fills the buffer with N
// values none of which is below P_th (the five 1-second intervals it checks
// cover the buffer, so the interval split does not change the answer).  That
// is: the first reading s that ends a run of N consecutive readings that are
// not below P_th.
//
// Work layout.  One warp per trace and CTAs of two warps, so the hardware
// block scheduler hands out traces as warps free up: read lengths differ by
// up to 3000 readings between traces (a trace is read only up to its report),
// and a static split of traces over resident warps left a long tail.  A warp
// takes its trace 256 readings at a time, lane l holding the 8 consecutive
// readings 8 l .. 8 l + 7 of the chunk (two 16-byte loads; the next chunk's
// loads are issued before the current chunk is scanned, so at most one chunk
// past the report is read).  Per chunk:
//   - each lane forms an 8-bit mask of its readings below P_th (a reading
//     past the end of the trace counts as below, so no run reaches into it;
//     a reading that is not a number is not below, as in the algorithm's
//     comparison);
//   - the run entering lane l is the trailing not-below count of the nearest
//     lower lane with a below reading plus 8 per all-clear lane between them,
//     or the run carried in from the previous chunk plus 8 l (one ballot, one
//     shuffle);
//   - with N >= 8 a run that starts inside a lane's 8 readings is too short
//     to reach N, so only the entering run extended through the lane's
//     leading not-below readings can: its first hit is N - 1 - run_in when
//     that lies before the lane's first below reading; with N < 8 the lane
//     walks its 8 readings;
//   - the report is the first hit of the lowest lane with one (a ballot).
// Run lengths are kept below N + 264 (a run that reaches N ends the scan), so
// 32-bit arithmetic holds them for any N.
#include "common.cuh"
#include "kernels.h"

namespace ocf {

namespace {

constexpr int PH_WARPS = 2;
constexpr int PH_CH = 256;   // readings per chunk: 32 lanes x 8

__device__ __forceinline__ uint32_t below_bits(const float4 &a, const float4 &b, float th) {
    return (uint32_t)(a.x < th) | (uint32_t)(a.y < th) << 1 | (uint32_t)(a.z < th) << 2 |
           (uint32_t)(a.w < th) << 3 | (uint32_t)(b.x < th) << 4 | (uint32_t)(b.y < th) << 5 |
           (uint32_t)(b.z < th) << 6 | (uint32_t)(b.w < th) << 7;
}

__global__ void __launch_bounds__(PH_WARPS * 32)
k_phase_detect(const float *__restrict__ power, int64_t n_traces, int64_t len, int64_t ld,
               float p_th, int32_t N, int64_t *__restrict__ first) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;   // lanes below this one
    const uint32_t n_win = (uint32_t)N;
    for (int64_t t = (int64_t)blockIdx.x * PH_WARPS + (threadIdx.x >> 5); t < n_traces;
         t += (int64_t)gridDim.x * PH_WARPS) {
        const float *pw = power + t * ld;
        // 16-byte loads when the trace starts on a 16-byte boundary (warp-uniform)
        const bool vec = (reinterpret_cast<uintptr_t>(pw) & 15) == 0;
        uint32_t carry = 0;   // not-below readings ending just before the chunk (< N)
        int64_t found = -1;
        float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb = na;
        if (vec && len >= PH_CH) {
            na = __ldg(reinterpret_cast<const float4 *>(pw + 8 * lane));
            nb = __ldg(reinterpret_cast<const float4 *>(pw + 8 * lane + 4));
        }
        for (int64_t c0 = 0; c0 < len; c0 += PH_CH) {
            uint32_t m;
            if (vec && c0 + PH_CH <= len) {
                const float4 a = na, b = nb;
                if (c0 + 2 * PH_CH <= len) {   // the next chunk, in flight during this scan
                    na = __ldg(reinterpret_cast<const float4 *>(pw + c0 + PH_CH + 8 * lane));
                    nb = __ldg(reinterpret_cast<const float4 *>(pw + c0 + PH_CH + 8 * lane + 4));
                }
                m = below_bits(a, b, p_th);
            } else {   // the ragged end of a trace, or a trace off the 16-byte grid
                m = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int64_t s = c0 + 8 * lane + i;
                    const bool below = s >= len || __ldg(pw + s) < p_th;
                    m |= (uint32_t)below << i;
                }
            }
            const uint32_t with_below = __ballot_sync(FULL, m != 0);
            const uint32_t tail = m ? (uint32_t)(__clz(m) - 24) : 8u;   // trailing not-below
            const uint32_t lower = with_below & lt_mask;
            const int hb = 31 - __clz(lower);   // nearest lower lane with a below (-1: none)
            const uint32_t tail_hb = __shfl_sync(FULL, tail, hb & 31);
            const uint32_t run_in =
                lower ? tail_hb + 8u * (uint32_t)(lane - 1 - hb) : carry + 8u * (uint32_t)lane;
            uint32_t f = 8;   // first reading of this lane whose run reaches N (8: none)
            if (n_win >= 8) {
                const uint32_t lead = m ? (uint32_t)(__ffs(m) - 1) : 8u;   // leading not-below
                const uint32_t p = run_in + 1 >= n_win ? 0u : n_win - 1 - run_in;
                if (p < lead) f = p;
            } else {
                uint32_t r = run_in;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    r = ((m >> i) & 1u) ? 0u : r + 1;
                    if (f == 8 && r >= n_win) f = (uint32_t)i;
                }
            }
            const uint32_t hits = __ballot_sync(FULL, f < 8);
            if (hits) {
                const int l = __ffs(hits) - 1;
                found = c0 + 8 * l + (int64_t)__shfl_sync(FULL, f, l);
                break;
            }
            carry = __shfl_sync(FULL, m ? tail : run_in + 8, 31);
        }
        if (lane == 0) first[t] = found;
    }
}

}  // namespace

cudaError_t launch_phase_detect(const float *power, int64_t n_traces, int64_t len, int64_t ld,
                                float p_th, int32_t window, int64_t *first, cudaStream_t st) {
    if (n_traces <= 0) return cudaSuccess;
    int64_t blocks = (n_traces + PH_WARPS - 1) / PH_WARPS;
    if (blocks > 0x7FFFFFFF) blocks = 0x7FFFFFFF;   // the trace loop strides past the grid
    k_phase_detect<<<(unsigned)blocks, PH_WARPS * 32, 0, st>>>(power, n_traces, len, ld, p_th,
                                                               window, first);
    return cudaGetLastError();
}

}  // namespace ocf
