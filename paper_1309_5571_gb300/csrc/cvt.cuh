// FP64 <-> FP32 conversions with integer operations only.  On this part the hardware
// conversions (cvt between f64 and f32) execute on the FP64 pipe, which runs at about
// 1/64 of the FP32 rate; kernels that convert every element they stream use these instead.
#pragma once

// float64 -> float32 with integer operations only (conversions through the FP64 units
// are slow on this part): the significand is truncated to 24 bits (relative error below
// 2^-23); magnitudes below 2^-126 become zero, magnitudes of 2^128 and above (and NaN)
// become an infinity of the same sign.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
  const unsigned int e = (hi >> 20) & 0x7ffu;
  const unsigned int sign = hi & 0x80000000u;
  // exponent re-biased in place (1023 -> 127), then the 8-bit exponent and 23
  // significand bits shifted into position (3 of them from the low word)
  const unsigned int h = hi - (896u << 20);
  unsigned int f = sign | (__funnelshift_l(lo, h, 3) & 0x7fffffffu);
  f = e >= 1151u ? (sign | 0x7f800000u) : f;
  f = e <= 896u ? 0u : f;
  return __uint_as_float(f);
}

// float32 -> float64, exact for normal numbers, integer operations only; zero and
// subnormals give 0, infinities and NaN keep their class.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int e = (b >> 23) & 0xffu;
  const unsigned int e64 = e == 255u ? 2047u : e + 896u;
  unsigned int hi = (b & 0x80000000u) | (e64 << 20) | ((b & 0x7fffffu) >> 3);
  unsigned int lo = b << 29;
  hi = e == 0u ? 0u : hi;
  lo = e == 0u ? 0u : lo;
  return __hiloint2double((int)hi, (int)lo);
}

// float64 -> float32 rounded to nearest (ties to even), integer operations only; the same
// range handling as f64_to_f32 (magnitudes below 2^-126 give zero: no FP32 subnormals).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
  const unsigned int e = (hi >> 20) & 0x7ffu;
  const unsigned int sign = hi & 0x80000000u;
  const unsigned int h = hi - (896u << 20);
  unsigned int mag = __funnelshift_l(lo, h, 3) & 0x7fffffffu;
  const unsigned int rest = lo & 0x1fffffffu;  // the 29 discarded significand bits
  mag += (rest > 0x10000000u || (rest == 0x10000000u && (mag & 1u))) ? 1u : 0u;
  unsigned int f = sign | (mag >= 0x7f800000u ? 0x7f800000u : mag);
  f = e >= 1151u ? (sign | 0x7f800000u) : f;
  f = e <= 896u ? 0u : f;
  return __uint_as_float(f);
}
