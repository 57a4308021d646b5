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

// periodic wrap into [-L/2, L/2) for |v| < 3L/2 (hL = L/2), the result of
// wrap_half: comparisons on the integer pipes and one FP64 addition whatever
// the branch (v - L is by definition v + (-L), rounded alike)
__device__ __forceinline__ double wrap_half_i(double v, double L, double hL) {
  const bool up = !dlt(v, hL), down = dlt(v, -hL);
  const double r = v + (up ? -L : L);
  return (up || down) ? r : v;
}

// v + (+0.0) without the FP64 pipe: -0.0 becomes +0.0, every other finite
// value is unchanged
__device__ __forceinline__ double plus_zero(double v) {
  return __double_as_longlong(v) == (long long)0x8000000000000000ull ? 0.0 : v;
}

}  // namespace ecmc

namespace ecmc {

// ---- correctly rounded FP64 square root on the integer pipes --------------
// The hit distance of Sec. 3.2 needs sqrt(sigma^2 - c^2) rounded to nearest
// as IEEE 754 defines it.  For a positive normal double x write
// x = t 2^E with t = M 2^-52 in [1, 4) and E even (M = the significand,
// doubled when the unbiased exponent is odd).  Then
//   sqrt(x) = sqrt(N) 2^(E/2 - 52),   N = M 2^52 in [2^104, 2^106),
// and sqrt(N) lies in [2^52, 2^53).  Starting from S0 = M Y 2^-31, where
// Y ~ 2^31 / sqrt(t) is an estimate with relative error below 2^-20, two
// Newton steps S <- S + (N - S^2) Y 2^-84 (the residual exact in 128 bits,
// truncated before the product) leave |S - sqrt(N)| < 1.02 (the bound:
// 2^33 after the estimate, 2^14.1 after the first step).  The exact
// remainder N - S^2, which then fits 64 bits, moves S to floor(sqrt(N))
// and decides the rounding: (S + 1/2)^2 = S^2 + S + 1/4 is never an integer,
// so the nearest value is S + 1 exactly when N - S^2 > S, and there are no
// ties.  A result S + 1 = 2^53 carries into the exponent by the addition.
__host__ __device__ __forceinline__ uint64_t mulhi_u64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Bit pattern of the float t (truncated to 24 bits): the input of the
// reciprocal-square-root estimate.  u is the bit pattern of x.
__host__ __device__ __forceinline__ uint32_t sqrt_seed_bits(uint64_t u) {
  const uint32_t odd = ((uint32_t)(u >> 52) & 1u) ^ 1u;  // unbiased exponent odd
  return ((127u + odd) << 23) | (uint32_t)((u >> 29) & 0x7fffffu);
}

// round(y 2^31) of a float y in [2^-2, 2) given by its bit pattern (exact:
// y has 24 significant bits)
__host__ __device__ __forceinline__ uint32_t fixed31_of(uint32_t yb) {
  return (0x800000u | (yb & 0x7fffffu)) << ((yb >> 23) - 119u);
}

__host__ __device__ __forceinline__ double sqrt_rn_with(uint64_t u, uint32_t Y) {
  const int e = (int)(u >> 52);
  const int odd = (e & 1) ^ 1;
  const uint64_t M = ((u & 0xfffffffffffffull) | 0x10000000000000ull) << odd;
  const uint64_t Nhi = M >> 12, Nlo = M << 52;
  uint64_t S = ((M >> 22) * (uint64_t)Y) >> 9;
  {  // |N - S^2| < 2^87: use (N - S^2) >> 56
    const uint64_t lo = S * S, hi = mulhi_u64(S, S);
    const uint64_t dlo = Nlo - lo, dhi = Nhi - hi - (Nlo < lo ? 1u : 0u);
    const int64_t D = (int64_t)((dhi << 8) | (dlo >> 56));
    S += (uint64_t)((D * (int64_t)Y) >> 28);
  }
  {  // |N - S^2| < 2^68.1: use (N - S^2) >> 38
    const uint64_t lo = S * S, hi = mulhi_u64(S, S);
    const uint64_t dlo = Nlo - lo, dhi = Nhi - hi - (Nlo < lo ? 1u : 0u);
    const int64_t D = (int64_t)((dhi << 26) | (dlo >> 38));
    S += (uint64_t)((D * (int64_t)Y) >> 46);
  }
  // |N - S^2| < 2^55.1: the remainder modulo 2^64 is the remainder
  int64_t rem = (int64_t)(Nlo - S * S);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool down = rem < 0;
    S -= down ? 1u : 0u;
    rem += down ? (int64_t)(2 * S + 1) : 0;
  }
  {
    const bool up = rem > (int64_t)(2 * S);
    rem -= up ? (int64_t)(2 * S + 1) : 0;
    S += up ? 1u : 0u;
  }
  S += rem > (int64_t)S ? 1u : 0u;
  const int64_t half = (int64_t)(e - 1023) >> 1;  // floor(E / 2)
  const uint64_t bits = ((uint64_t)(half + 1022) << 52) + S;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double r;
  __builtin_memcpy(&r, &bits, sizeof r);
  return r;
#endif
}

#ifdef __CUDACC__
// The estimate Y from the SFU's reciprocal square root (relative error of
// a few units in the last place of a float, far inside 2^-20).
__device__ __forceinline__ double sqrt_rn(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__uint_as_float(sqrt_seed_bits(u))));
  return sqrt_rn_with(u, fixed31_of(__float_as_uint(y)));
}
#endif

}  // namespace ecmc
