// Generated by gen_series_constants.py; do not edit.
#pragma once
#define TTR_LN2_HI 0x1.62e42fee00000p-1
#define TTR_LN2_LO 0x1.a39ef35793c76p-33
#define TTR_SQRT_HALF 0x1.6a09e667f3bcdp-1
#define TTR_TWO_PI_HI 0x1.921fb54442d18p+2
#define TTR_TWO_PI_LO 0x1.1a62633145c07p-52
// 1/(2t+1), t = 0..13 (atanh series)
__device__ __constant__ double kTtrAtanh[14] = {0x1.0000000000000p+0, 0x1.5555555555555p-2, 0x1.999999999999ap-3, 0x1.2492492492492p-3, 0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4, 0x1.3b13b13b13b14p-4, 0x1.1111111111111p-4, 0x1.e1e1e1e1e1e1ep-5, 0x1.af286bca1af28p-5, 0x1.8618618618618p-5, 0x1.642c8590b2164p-5, 0x1.47ae147ae147bp-5, 0x1.2f684bda12f68p-5};
// (-1)^k/(2k)!, k = 0..10 (cos series)
__device__ __constant__ double kTtrCos[11] = {0x1.0000000000000p+0, -0x1.0000000000000p-1, 0x1.5555555555555p-5, -0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-16, -0x1.27e4fb7789f5cp-22, 0x1.1eed8eff8d898p-29, -0x1.93974a8c07c9dp-37, 0x1.ae7f3e733b81fp-45, -0x1.6827863b97d97p-53, 0x1.e542ba4020225p-62};
// (-1)^k/(2k+1)!, k = 0..10 (sin series)
__device__ __constant__ double kTtrSin[11] = {0x1.0000000000000p+0, -0x1.5555555555555p-3, 0x1.1111111111111p-7, -0x1.a01a01a01a01ap-13, 0x1.71de3a556c734p-19, -0x1.ae64567f544e4p-26, 0x1.6124613a86d09p-33, -0x1.ae7f3e733b81fp-41, 0x1.952c77030ad4ap-49, -0x1.2f49b46814157p-57, 0x1.71b8ef6dcf572p-66};
