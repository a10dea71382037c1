// Algorithm 2 (energy-efficient power-cap selection, Sec. "Optimal Power
// setting Selection") evaluated in FP32 with correctly rounded operations in
// the order p_j = t_b / t_j, loss = 1 - p_j, E_j = (c_j + g_j) / p_j,
// saving_j = (E_base - E_j) / E_base; shared by the reconstruction kernels.
#pragma once
#include <stdint.h>

namespace ocf {

struct Cand {
    float sv;    // saving
    float cg;    // c + g
    int32_t j;   // setting (-1: none)
    float Ethr;  // screening threshold derived from this candidate's exact energy
};

// a better than b?  (saving desc, c+g asc, index asc; j < 0 means none)
__device__ __forceinline__ bool better(const Cand &a, const Cand &b) {
    if (a.j < 0) return false;
    if (b.j < 0) return true;
    if (a.sv != b.sv) return a.sv > b.sv;
    if (a.cg != b.cg) return a.cg < b.cg;
    return a.j < b.j;
}

// Per-row constants of the selection.  loss(t) = 1 - t_b / t is evaluated as
// fl(1 - fl(t_b / t)), which is non-decreasing in t (correctly rounded
// division and subtraction are monotone), so "loss <= gamma" holds exactly for
// 0 < t <= tstar, the largest float that passes; tstar is found by bisection
// over float bit patterns.  tstar = -1 when the baseline runtime is not > 0.
struct RowCtx {
    float tb, tstar, rtb;
};

__device__ __forceinline__ RowCtx alg2_row(float tb, float gamma) {
    RowCtx r{tb, -1.0f, 0.0f};
    if (!(tb > 0.0f)) return r;
    r.rtb = __frcp_rn(tb);
    auto ok = [&](uint32_t bits) {
        const float t = __uint_as_float(bits);
        return __fsub_rn(1.0f, __fdiv_rn(tb, t)) <= gamma;
    };
    uint32_t lo = 0u, hi = 0x7f7fffffu;   // ok(tiny t) always; bisect up to FLT_MAX
    if (ok(hi)) {
        r.tstar = __uint_as_float(0x7f800000u);   // every finite t > 0 is valid
        return r;
    }
    // In real numbers the bound is t_b / (1 - gamma); the rounded comparison
    // moves it by a few units in the last place, so a short walk from there
    // usually finds the transition (ok(t*) and not ok(next float)).  ok is
    // monotone, so that transition is the one the bisection finds; a walk that
    // does not end within 8 steps falls through to the bisection.
    const float g1 = __fsub_rn(1.0f, gamma);
    if (g1 > 0.0f) {
        uint32_t b = __float_as_uint(__fdiv_rn(tb, g1));
        if (b > 0u && b < hi) {
            if (ok(b)) {
                int s = 0;
                while (s < 8 && ok(b + 1u)) { ++b; ++s; }
                if (s < 8) { r.tstar = __uint_as_float(b); return r; }
            } else {
                int s = 0;
                while (s < 8 && b > 1u && !ok(b - 1u)) { --b; ++s; }
                if (s < 8 && b > 1u) { r.tstar = __uint_as_float(b - 1u); return r; }
            }
        }
    }
    while (hi - lo > 1u) {
        const uint32_t mid = lo + (hi - lo) / 2u;
        if (ok(mid)) lo = mid; else hi = mid;
    }
    r.tstar = __uint_as_float(lo);
    return r;
}

// Exact FP32 evaluation (the order the oracle fixes), reached only by
// candidates the screen cannot exclude.  The screen: E ~ cg * t / t_b from two
// multiplies is within 2^-20 of the exact E = fl(cg / fl(t_b / t)); a candidate
// whose estimate exceeds best.Ethr = (E_best + 2^-16 (E_base + E_best)) (1 + 2^-19)
// has an exact energy so far above the best's that its saving is strictly
// smaller, so it can neither win nor tie.
__device__ __forceinline__ void alg2_consider(Cand &best, const RowCtx &r, float t, float cg,
                                              float Eb, int32_t j) {
    if (!(t > 0.0f) || !(t <= r.tstar)) return;
    if (best.j >= 0 && __fmul_rn(__fmul_rn(cg, t), r.rtb) > best.Ethr) return;
    const float p = __fdiv_rn(r.tb, t);
    const float E = __fdiv_rn(cg, p);
    const float sv = __fdiv_rn(__fsub_rn(Eb, E), Eb);
    const float thr = __fmul_rn(__fadd_rn(E, __fmul_rn(1.52587890625e-05f, __fadd_rn(Eb, E))),
                                1.0000019073486328f);
    Cand c{sv, cg, j, thr};
    if (better(c, best)) best = c;
}

// Cheap energy estimate cg * t / t_b of a valid element; NaN when invalid, so
// fminf ignores it and every comparison with a bound is false.
__device__ __forceinline__ float alg2_estimate(const RowCtx &r, float t, float cg) {
    if (!(t > 0.0f) || !(t <= r.tstar)) return __int_as_float(0x7fffffff);
    return __fmul_rn(__fmul_rn(cg, t), r.rtb);
}

// Screening bound from an estimate: an element whose estimate exceeds
// bound(Emin) has an exact energy beyond E(argmin) + 2^-16 (E_base + E), so it
// can neither win nor tie against the element that produced Emin.
__device__ __forceinline__ float alg2_bound(float Emin, float Eb) {
    const float hi = __fmul_rn(Emin, 1.0000038146972656f);   // estimate error 2^-20, twice
    return __fmul_rn(__fadd_rn(hi, __fmul_rn(1.52587890625e-05f, __fadd_rn(Eb, hi))),
                     1.0000019073486328f);
}

// Exact evaluation of an element that survived the screen (t valid).
__device__ __forceinline__ void alg2_exact(Cand &best, const RowCtx &r, float t, float cg,
                                           float Eb, int32_t j) {
    const float p = __fdiv_rn(r.tb, t);
    const float E = __fdiv_rn(cg, p);
    const float sv = __fdiv_rn(__fsub_rn(Eb, E), Eb);
    const float thr = __fmul_rn(__fadd_rn(E, __fmul_rn(1.52587890625e-05f, __fadd_rn(Eb, E))),
                                1.0000019073486328f);
    Cand c{sv, cg, j, thr};
    if (better(c, best)) best = c;
}

}  // namespace ocf
