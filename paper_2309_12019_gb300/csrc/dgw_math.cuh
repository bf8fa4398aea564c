// Device math helpers shared by the kernels.
#pragma once

namespace dgw {

// sin and cos of x in float.  Cody-Waite reduction (Cody & Waite, "Software Manual for
// the Elementary Functions", 1980) of x by 2 pi with a two-term split C1 + C2 of 2 pi
// (C1 = 2 pi rounded to float, C2 = 2 pi - C1), k = rint(x / 2 pi); the product k*C1
// is exact while |k| < 2^15.  The reduced argument lies in [-pi, pi], where the
// hardware approximations __sincosf have an absolute error below 2^-21.
__device__ __forceinline__ void fast_sincos(float x, float* s, float* c)
{
    const float k = rintf(x * 0.159154943091895336f);
    float r = fmaf(-k, 6.28318548202514648f, x);
    r = fmaf(-k, -1.74845553146951715e-7f, r);
    __sincosf(r, s, c);
}

// fast_sincos of both lanes of x, with the reduction on the packed FP32 pipe: rint of
// t = x / 2 pi through the shift by 1.5 * 2^23 (exact round-to-nearest-even for
// |t| < 2^22), then the same two-term Cody-Waite steps.  Each lane's result is bitwise
// that of fast_sincos.
__device__ __forceinline__ void fast_sincos2(float2 x, float2* s, float2* c)
{
    const float2 t = __fmul2_rn(x, make_float2(0.159154943091895336f, 0.159154943091895336f));
    const float2 k = __fadd2_rn(__fadd2_rn(t, make_float2(12582912.0f, 12582912.0f)),
                                make_float2(-12582912.0f, -12582912.0f));
    float2 r = __ffma2_rn(k, make_float2(-6.28318548202514648f, -6.28318548202514648f), x);
    r = __ffma2_rn(k, make_float2(1.74845553146951715e-7f, 1.74845553146951715e-7f), r);
    __sincosf(r.x, &s->x, &c->x);
    __sincosf(r.y, &s->y, &c->y);
}

}  // namespace dgw
