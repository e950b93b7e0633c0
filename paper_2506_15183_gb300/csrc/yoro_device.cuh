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

// rcp.approx.ftz: one MUFU op, within 1 ulp of 1/x for normal x (a denormal
// input flushes to a zero divisor and gives +inf).  Every use below tolerates that
// error and the flush through a checked margin.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The exact fallbacks.  exact_target is inlined into the scatter loop (an out-of-line
// call there cost more, in the caller's registers, than the rare branch it serves);
// exact_rint_quotient stays out of line in the fill.
static __device__ __forceinline__ int exact_target(float xc, float k, float zc)
{
    // cvt.rmi gives floor; out-of-range values saturate to INT_MIN / INT_MAX, which
    // the caller drops like any off-frame column.
    return __float2int_rd(__fsub_rn(xc, __fdiv_rn(k, zc)));
}

static __device__ __noinline__ float exact_rint_quotient(float a, float b) { return rintf(__fdiv_rn(a, b)); }

// Bits of zc = clamp(z, near, far), with a depth that is not a positive finite number
// taken as far (Alg. 1's clamp to the camera planes).  Positive binary32 values order
// like their bit patterns, so the clamp is an unsigned min and max on the bits;
// subtracting 1 first moves +0 (bits 0) to the top of the unsigned range, where the
// negative numbers, -0, the infinities and the NaNs already are, and all of them
// clamp to far.  near_m1 / far_m1 are the bits of near / far minus 1.
__device__ __forceinline__ uint32_t clamped_depth_bits(float z, uint32_t near_m1, uint32_t far_m1)
{
    return max(min(__float_as_uint(z) - 1u, far_m1), near_m1) + 1u;
}

// Alg. 1 with Eq. 5 in closed form (parallel-axis pinhole pair, baseline ipd along
// +x, left eye as source):  zc = clamp(z, near, far) with non-positive or non-finite
// depth treated as far;  target column floor((x + 0.5) - RN(k / zc)) with k = fx * ipd.
// Returns the target column (any int; the caller drops it outside [0, w)) and
// writes the bits of the clamped depth.  `xc` is the pixel centre x + 0.5.
//
// Only the floor is needed, so the IEEE quotient is computed only when a cheaper
// estimate cannot decide it.  With Q = k/zc and r = rcp(zc) (|r - 1/zc| <= 2^-23 / zc),
// the estimate t' = RN(xc - k * r), one fused multiply-add, is within
// 2^-23 Q + 2^-24 (xc + Q) (1 + 2^-23) of xc - Q, and t = RN(xc - RN(Q)) within
// 2^-24 Q + 2^-24 (xc + Q) (1 + 2^-24); so |t' - t| < 2^-21 (xc + Q).  `half_m` is
// 0.5 - M with M = 2^-20 (w + 1.5 + k/near) * (1 + 2^-10) >= twice that distance plus
// an absolute 2^-20 (which also covers flushed denormals), bounded on the host per
// frame.  If frac(t') lies in (M, 1 - M), floor(t) == floor(t').
__device__ __forceinline__ int disparity_target(float z, float xc, float k, uint32_t near_m1, uint32_t far_m1,
                                                float half_m, uint32_t& zbits)
{
    zbits = clamped_depth_bits(z, near_m1, far_m1);
    const float zc = __uint_as_float(zbits);
    const float tp = __fmaf_rn(-k, rcp_approx(zc), xc);
    const float fl = floorf(tp);
    if (fabsf(__fsub_rn(__fsub_rn(tp, fl), 0.5f)) < half_m) return (int)fl;
    return exact_target(xc, k, zc);
}

// 64-bit z-buffer key of Alg. 2's "keep the nearest": clamped depth bits above the
// source column.  For positive floats the bit order is the value order, so the
// smallest key is the nearest source and, on equal depth, the lowest column (the
// first writer of the paper's left-to-right scan).
__device__ __forceinline__ unsigned long long zkey(uint32_t zbits, int x)
{
    return ((unsigned long long)zbits << 32) | (unsigned)x;
}

// A channel byte of an RGBA8 word as a float: the byte is put under the exponent of
// 2^23 (the float 2^23 + byte, exactly) and 2^23 is subtracted, which is exact; equal
// to __uint2float_rn of the byte, without the conversion unit.
__device__ __forceinline__ float channel(uint32_t rgba, uint32_t sel)
{
    return __fsub_rn(__uint_as_float(__byte_perm(rgba, 0x4B00u, sel)), 8388608.0f);
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
    // Each channel sum += channel * wgt (multiply, then add: never fused), wrem -= wgt.
    __device__ __forceinline__ void step(uint32_t rgba, float wgt)
    {
        acc[0] = __fadd_rn(acc[0], __fmul_rn(channel(rgba, 0x5440u), wgt));
        acc[1] = __fadd_rn(acc[1], __fmul_rn(channel(rgba, 0x5441u), wgt));
        acc[2] = __fadd_rn(acc[2], __fmul_rn(channel(rgba, 0x5442u), wgt));
        acc[3] = __fadd_rn(acc[3], __fmul_rn(channel(rgba, 0x5443u), wgt));
        wrem = __fsub_rn(wrem, wgt);
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
        step(rgba, wgt);
        return true;
    }
    // add(rgba) when `take`, else nothing: a weight of exactly 0 leaves acc (acc + c*0)
    // and wrem (wrem - 0) unchanged, so skipping and adding 0 are the same.
    __device__ __forceinline__ void add_if(bool take, uint32_t rgba)
    {
        const float a = __fmul_rn(wrem, 0.5f);
        const float b = __fmul_rn(__fmul_rn(0.3f, wrem), t);
        step(rgba, take ? __fadd_rn(a, b) : 0.0f);
    }
    __device__ __forceinline__ bool any() const { return wrem != 1.0f; }

    // Exact early exit.  Every later step only grows acc and shrinks wrem: the updates
    // wrem -= wgt are exact (wrem/2 <= wgt <= wrem, Sterbenz; exact anyway among
    // denormals), so the remaining weights sum to at most the current wrem, and since
    // wrem at least halves per step at most 150 later steps carry a non-zero weight.
    // A later step adds y = RN(c * wgt) <= 255 wgt (1 + 2^-24) + 2^-150, and RN(acc + y)
    // lies in [acc, acc + y + min(y, ulp/2)] (acc itself is a float no farther from
    // acc + y than y, and acc < 256 keeps ulp/2 <= 2^-17).  With E = 255 (1 + 2^-24) wrem
    // the final acc is therefore at most acc + E + min(E, 150 * 2^-17) + 300 * 2^-150, and the
    // final denominator RN(1 - wrem_N) is at least RN(1 - wrem).  So the final quotient
    // lies in [acc, (acc + E + min(E, 0.00115) + 1e-42) / RN(1 - wrem)] (the lower end
    // when every later color is 0).  The upper end is evaluated with upward rounding; if
    // for every channel it stays below rint(acc) + 0.5, the rounded result is rint(acc)
    // whatever the remaining candidates hold.  The slack vanishes with wrem, so every
    // pixel settles a few contributions after its acc is within reach of its result.
    __device__ __forceinline__ bool settled(uint32_t& out) const
    {
        const float den = __fsub_rn(1.0f, wrem);
        // rcp.approx is within 1 ulp of 1/den, so rcp * (1 + 2^-22) rounded up bounds it
        const float inv = __fmul_ru(rcp_approx(den), 1.0000002384185791f);
        const float e1 = __fmul_ru(255.0000152587890625f, wrem);  // 255 + 2^-16 >= 255 (1 + 2^-24)
        const float e = __fadd_ru(__fadd_ru(e1, fminf(e1, 0.00115f)), 1.0e-42f);
        uint32_t o = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float r = rintf(acc[c]);
            if (r < 255.0f) {  // r >= 255: the clamped result is 255 whatever follows
                const float hi = __fmul_ru(__fadd_ru(acc[c], e), inv);
                if (!(hi < __fadd_rn(r, 0.5f))) return false;
            }
            o |= (uint32_t)fminf(r, 255.0f) << (8 * c);
        }
        out = o;
        return true;
    }
    // acc / (1 - wrem) per channel, rounded half to even, clamped to [0, 255].  As for
    // the disparity, the IEEE quotient is only computed when an estimate cannot decide
    // the rounding: den = RN(1 - wrem) is in [0.5, 1] after a contribution, and
    // q' = RN(acc * rcp(den)) is within 2.01 * 2^-23 * q' of RN(acc / den); if no
    // half-integer lies within 2^-20 (q' + 1) of q', rint(q') is the result.
    __device__ __forceinline__ uint32_t result() const
    {
        const float den = __fsub_rn(1.0f, wrem);
        const float inv = rcp_approx(den);
        uint32_t out = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float qp = __fmul_rn(acc[c], inv);
            const float m = __fmul_rn(__fadd_rn(qp, 1.0f), 9.5367431640625e-07f);
            float r = rintf(__fsub_rn(qp, m));
            if (r != rintf(__fadd_rn(qp, m))) r = exact_rint_quotient(acc[c], den);
            r = fminf(fmaxf(r, 0.0f), 255.0f);
            out |= (uint32_t)r << (8 * c);
        }
        return out;
    }
};

}  // namespace yoro
