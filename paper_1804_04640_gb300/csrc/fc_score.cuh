// fc_score.cuh -- device helpers for the score reductions of Sec. 3.1:
// compensated FP32 sums and the per-cell mutual-information term.
#pragma once

#include <cuda_runtime.h>

namespace fc {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kInvLn2 = 1.4426950408889634f;

struct Kahan {
    float s, c;
};

__device__ __forceinline__ void kahan_add(Kahan &k, float x)
{
    const float y = __fsub_rn(x, k.c);
    const float t = __fadd_rn(k.s, y);
    k.c = __fsub_rn(__fsub_rn(t, k.s), y);
    k.s = t;
}

__device__ __forceinline__ void kahan_merge(Kahan &a, const Kahan &b)
{
    kahan_add(a, b.s);
    kahan_add(a, -b.c);
}

// (1 + x) ln(1 + x) - x, the non-negative per-cell term of the mutual
// information written around the independence point (x = 0).  Near x = 0 the
// direct form cancels, so the Taylor series sum_{n>=2} (-1)^n x^n / (n (n-1))
// is used for |x| < 0.1 (truncation below 4e-8 relative there).
__device__ __forceinline__ float mi_term(float x)
{
    if (x <= -1.0f) return 1.0f;
    if (fabsf(x) < 0.1f) {
        const float x2 = x * x;
        return x2 * (0.5f + x * (-1.0f / 6.0f + x * (1.0f / 12.0f + x * (-1.0f / 20.0f +
                     x * (1.0f / 30.0f + x * (-1.0f / 42.0f))))));
    }
    return (1.0f + x) * log1pf(x) - x;
}

}  // namespace fc
