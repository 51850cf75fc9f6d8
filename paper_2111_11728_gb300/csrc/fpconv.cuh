// Conversions between FP64 and FP32 on the integer pipe.
//
// On this part the FP64 unit is small (2 FP64 operations per clock per SM), and
// FP64 <-> FP32 conversions share it: kernels that only move and convert data
// (the gathers and scatters of the reduced-precision operator) become bound by
// it.  These helpers do the same conversions with integer operations on the
// IEEE-754 bit fields.
//   f64_to_f32_rn: round to nearest, ties to even (as cvt.rn.f32.f64) for
//                  inputs of magnitude >= 2^-126 (the smallest normal FP32);
//                  smaller inputs flush to a signed zero, results above the
//                  largest FP32 round to a signed infinity; NaN stays NaN.
//   f32_to_f64:    exact for every finite FP32 value (subnormals included),
//                  infinities and NaN preserved.
// The header also compiles as plain C++ (host), which the CPU tests use.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define FETI_HD __host__ __device__ __forceinline__
#else
#define FETI_HD inline
#endif

namespace feti {

FETI_HD uint64_t fpc_bits64(double x) {
#if defined(__CUDA_ARCH__)
  return static_cast<uint64_t>(__double_as_longlong(x));
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

FETI_HD double fpc_from64(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double(static_cast<long long>(b));
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

FETI_HD uint32_t fpc_bits32(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

FETI_HD float fpc_from32(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

FETI_HD int fpc_clz32(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return __clz(static_cast<int>(v));
#else
  return v ? __builtin_clz(v) : 32;
#endif
}

FETI_HD float f64_to_f32_rn(double x) {
  // Branch-free for FP32-normal results: bits 30..0 of the FP32 pattern are the
  // FP64 pattern shifted right by 29 (the low 8 exponent bits and the top 23
  // mantissa bits) with the exponent's top bit flipped (e - 896 = E for the
  // exponents 897..1150 of the FP32 normals); the 29 dropped mantissa bits round
  // to nearest, ties to even, a carry moving into the exponent (and to the
  // infinity pattern past the largest FP32).
  const uint64_t b = fpc_bits64(x);
  const uint32_t hi = static_cast<uint32_t>(b >> 32);
  const uint32_t sign = hi & 0x80000000u;
  const uint32_t e = (hi >> 20) & 0x7FFu;
  uint32_t r = (static_cast<uint32_t>(b >> 29) ^ 0x40000000u) & 0x7FFFFFFFu;
  const uint32_t rem = static_cast<uint32_t>(b) & 0x1FFFFFFFu;
  r += (rem + 0x0FFFFFFFu + (r & 1u)) >> 29;
  if (e - 897u > 253u) {                            // outside the FP32 normal exponents
    if (e < 897u) r = 0u;                                          // below FP32 normals: signed zero
    else r = (e == 0x7FFu && (b & 0xFFFFFFFFFFFFFull)) ? 0x7FC00000u : 0x7F800000u;   // NaN; infinity
  }
  return fpc_from32(sign | r);
}

FETI_HD double f32_to_f64(float x) {
  const uint32_t b = fpc_bits32(x);
  const uint64_t sign = static_cast<uint64_t>(b & 0x80000000u) << 32;
  const int e = static_cast<int>((b >> 23) & 0xFF);
  uint32_t m = b & 0x7FFFFFu;
  if (e == 0xFF) return fpc_from64(sign | 0x7FF0000000000000ull | (static_cast<uint64_t>(m) << 29));
  if (e == 0) {
    if (m == 0) return fpc_from64(sign);
    const int shift = fpc_clz32(m) - 8;                            // leading one to bit 23
    m = (m << shift) & 0x7FFFFFu;
    const uint64_t ed = static_cast<uint64_t>(1 - 127 - shift + 1023);
    return fpc_from64(sign | (ed << 52) | (static_cast<uint64_t>(m) << 29));
  }
  const uint64_t ed = static_cast<uint64_t>(e - 127 + 1023);
  return fpc_from64(sign | (ed << 52) | (static_cast<uint64_t>(m) << 29));
}

}  // namespace feti
