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
  const uint64_t b = fpc_bits64(x);
  const uint32_t sign = static_cast<uint32_t>(b >> 32) & 0x80000000u;
  const int e = static_cast<int>((b >> 52) & 0x7FF);
  const uint64_t mant = b & 0xFFFFFFFFFFFFFull;
  if (e == 0x7FF) return fpc_from32(sign | 0x7F800000u | (mant ? 0x400000u : 0u));
  int ef = e - 1023 + 127;
  if (ef <= 0) return fpc_from32(sign);                          // below FP32 normals: signed zero
  uint32_t m = static_cast<uint32_t>(mant >> 29);
  const uint32_t rem = static_cast<uint32_t>(mant & 0x1FFFFFFFull);
  if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) {
    if (++m == 0x800000u) {
      m = 0;
      ++ef;
    }
  }
  if (ef >= 255) return fpc_from32(sign | 0x7F800000u);           // overflow: signed infinity
  return fpc_from32(sign | (static_cast<uint32_t>(ef) << 23) | m);
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
