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

}  // namespace dgw
