// Device helpers of the second-eye synthesis kernels (sm_103a).
//
// Every floating-point step is written with an explicit round-to-nearest intrinsic
// (__fadd_rn, __fmul_rn, __fdiv_rn, ...), which the compiler never contracts into an
// FMA, so the kernels compute exactly the binary32 sequence the method defines.
// Denormals are kept (no -ftz): the remaining weight of the fill reaches them.
#pragma once

#include <cstdint>

namespace yoro {

constexpr unsigned long long kEmptyKey = ~0ull;

// Alg. 1 with Eq. 5 in closed form (parallel-axis pinhole pair, baseline ipd along
// +x, left eye as source):  zc = clamp(z, near, far) with non-positive or non-finite
// depth treated as far;  target column floor((x + 0.5) - k / zc) with k = fx * ipd.
// Returns the target column (any int; the caller drops it outside [0, w)) and
// writes the clamped depth.
__device__ __forceinline__ int disparity_target(float z, int x, float k, float near_, float far_,
                                                float& zc)
{
    if (!(z > 0.0f) || fabsf(z) == __int_as_float(0x7f800000)) z = far_;
    zc = fminf(fmaxf(z, near_), far_);
    const float disp = __fdiv_rn(k, zc);
    const float t = __fsub_rn(__fadd_rn((float)x, 0.5f), disp);
    const float f = floorf(t);
    // |f| beyond the int range can only be off-frame; clamp before converting.
    if (f < -1.0f) return -1;
    if (f > 2147483520.0f) return 0x7fffff80;
    return (int)f;
}

// 64-bit z-buffer key of Alg. 2's "keep the nearest": clamped depth bits above the
// source column.  For positive floats the bit order is the value order, so the
// smallest key is the nearest source and, on equal depth, the lowest column (the
// first writer of the paper's left-to-right scan).
__device__ __forceinline__ unsigned long long zkey(float zc, int x)
{
    return ((unsigned long long)__float_as_uint(zc) << 32) | (unsigned)x;
}

// Accumulator of the Patcher (Alg. 3) for one hole pixel.
struct FillAcc {
    float acc[4];
    float wrem;
    float t;
    __device__ __forceinline__ void init(float t_)
    {
        acc[0] = acc[1] = acc[2] = acc[3] = 0.0f;
        wrem = 1.0f;
        t = t_;
    }
    // One contributing candidate of color `rgba`.  Eq. 6: wgt = wrem/2 + 0.3 wrem t,
    // evaluated (wrem * 0.5) + ((0.3 * wrem) * t).  Returns false once wgt == 0: from
    // then on wgt stays 0 and acc/wrem are unchanged (acc + c*0 == acc, wrem - 0 ==
    // wrem), so the remaining candidates cannot change the result.
    __device__ __forceinline__ bool add(uint32_t rgba)
    {
        const float a = __fmul_rn(wrem, 0.5f);
        const float b = __fmul_rn(__fmul_rn(0.3f, wrem), t);
        const float wgt = __fadd_rn(a, b);
        if (wgt == 0.0f) return false;
        acc[0] = __fadd_rn(acc[0], __fmul_rn(__uint2float_rn(rgba & 255u), wgt));
        acc[1] = __fadd_rn(acc[1], __fmul_rn(__uint2float_rn((rgba >> 8) & 255u), wgt));
        acc[2] = __fadd_rn(acc[2], __fmul_rn(__uint2float_rn((rgba >> 16) & 255u), wgt));
        acc[3] = __fadd_rn(acc[3], __fmul_rn(__uint2float_rn(rgba >> 24), wgt));
        wrem = __fsub_rn(wrem, wgt);
        return true;
    }
    __device__ __forceinline__ bool any() const { return wrem != 1.0f; }
    // acc / (1 - wrem) per channel, rounded half to even, clamped to [0, 255].
    __device__ __forceinline__ uint32_t result() const
    {
        const float den = __fsub_rn(1.0f, wrem);
        uint32_t out = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float r = rintf(__fdiv_rn(acc[c], den));
            r = fminf(fmaxf(r, 0.0f), 255.0f);
            out |= (uint32_t)r << (8 * c);
        }
        return out;
    }
};

}  // namespace yoro
