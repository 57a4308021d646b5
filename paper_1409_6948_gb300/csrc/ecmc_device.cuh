// ecmc_device.cuh -- device helpers: counter-based random numbers and the
// periodic wraps used by the sweep kernels.
#pragma once
#include <cstdint>

namespace ecmc {

// Philox4x64 with ten rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
// multiplies counter words 0 and 2 by fixed odd constants into 128-bit
// products, permutes the words and mixes in the key, and the key advances by
// a Weyl sequence (golden ratio and sqrt(3)-1) between rounds.
struct U64x4 {
  uint64_t v[4];
};

__device__ __forceinline__ U64x4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                        uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0_lo = M0 * c0, p0_hi = __umul64hi(M0, c0);
    const uint64_t p1_lo = M1 * c2, p1_hi = __umul64hi(M1, c2);
    const uint64_t n0 = p1_hi ^ c1 ^ k0;
    const uint64_t n2 = p0_hi ^ c3 ^ k1;
    c0 = n0;
    c1 = p1_lo;
    c2 = n2;
    c3 = p0_lo;
    k0 += W0;
    k1 += W1;
  }
  U64x4 r;
  r.v[0] = c0;
  r.v[1] = c1;
  r.v[2] = c2;
  r.v[3] = c3;
  return r;
}

// uniform integer in [0, n): the high word of v * n
__device__ __forceinline__ uint64_t below_n(uint64_t v, uint64_t n) { return __umul64hi(v, n); }

// uniform double in [0, 1) from the 53 high bits
__device__ __forceinline__ double unit_double(uint64_t v) {
  return (double)(v >> 11) * 0x1.0p-53;
}

// periodic wrap into [-L/2, L/2) for |v| < 3L/2
__device__ __forceinline__ double wrap_half(double v, double L) {
  if (v >= 0.5 * L) return v - L;
  if (v < -0.5 * L) return v + L;
  return v;
}

// periodic wrap into [0, L) for v in (-L, 2L)
__device__ __forceinline__ double wrap_box0(double v, double L) {
  if (v < 0.0) v += L;
  if (v >= L) v -= L;
  return v;
}

// cell index along one axis: u = v - shift wrapped into [0, L), then
// floor(u * inv_w) clamped to [0, cells-1]
__device__ __forceinline__ int cell_1d(double v, double shift, double L, double inv_w,
                                       int cells) {
  double u = v - shift;
  if (u < 0.0) u += L;
  int c = (int)(u * inv_w);
  if (c >= cells) c = cells - 1;
  if (c < 0) c = 0;
  return c;
}

}  // namespace ecmc

namespace ecmc {

// ---- FP64 comparisons and conversions on the integer pipes ---------------
// For doubles that are >= +0 (or +inf), the order of the bit patterns read
// as signed 64-bit integers is the numeric order; negative values (and -0.0)
// read as negative integers.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ bool le_nn(double a, double b) { return dbits(a) <= dbits(b); }
__device__ __forceinline__ bool lt_nn(double a, double b) { return dbits(a) < dbits(b); }
__device__ __forceinline__ double min_nn(double a, double b) { return lt_nn(b, a) ? b : a; }
// max(v, +0.0), mapping -0.0 to +0.0 (no result downstream distinguishes them)
__device__ __forceinline__ double clamp0(double v) { return dbits(v) < 0 ? 0.0 : v; }
// v with its sign flipped when neg is set (exact)
__device__ __forceinline__ double flip_if(double v, bool neg) {
  return __longlong_as_double(dbits(v) ^ (neg ? (long long)0x8000000000000000ull : 0ll));
}

// Double to float rounding toward zero: |v - f| < 2^-23 |v| for
// 2^-126 <= |v| < 2^127; smaller magnitudes give +-0.
__device__ __forceinline__ float to_float_trunc(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ff);
  if (e < 1023 - 126) return __int_as_float((int)sign);
  const unsigned fe = (unsigned)(e - 1023 + 127);
  const unsigned fm = (unsigned)((u >> 29) & 0x7fffffu);
  return __int_as_float((int)(sign | (fe << 23) | fm));
}

// Non-negative double (or +inf) to the smallest float >= v.
__device__ __forceinline__ float to_float_up_nn(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  if (u >= 0x7ff0000000000000ull) return __int_as_float(0x7f800000);
  const int e = (int)(u >> 52);
  if (e < 1023 - 126) return u == 0 ? 0.0f : __int_as_float(0x00800000);
  if (e > 1023 + 127) return __int_as_float(0x7f800000);
  const unsigned fe = (unsigned)(e - 1023 + 127);
  unsigned bits = (fe << 23) | (unsigned)((u >> 29) & 0x7fffffu);
  if (u & 0x1fffffffull) bits += 1u;  // a carry into the exponent is still the next float up
  return __int_as_float((int)bits);
}

}  // namespace ecmc

namespace ecmc {

// Signed comparisons of doubles on the integer pipes.  Valid for finite
// values; -0.0 and +0.0 compare equal, as in IEEE arithmetic.
__device__ __forceinline__ long long dkey(double v) {
  // monotone map of the bit pattern: negative values are reflected so that
  // the signed-integer order is the numeric order
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : (long long)0x8000000000000000ull - b;
}
__device__ __forceinline__ bool dlt(double a, double b) { return dkey(a) < dkey(b); }
__device__ __forceinline__ bool dle(double a, double b) { return dkey(a) <= dkey(b); }

// periodic wrap into [-L/2, L/2) for |v| < 3L/2 (hL = L/2), comparisons on
// the integer pipes; the additions are the same as in wrap_half
__device__ __forceinline__ double wrap_half_i(double v, double L, double hL) {
  if (!dlt(v, hL)) return v - L;
  if (dlt(v, -hL)) return v + L;
  return v;
}

}  // namespace ecmc
