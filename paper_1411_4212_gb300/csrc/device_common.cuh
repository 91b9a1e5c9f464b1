// device_common.cuh -- device helpers shared by the REWL kernels: counter-based random numbers,
// the FP64 exp of the trajectory mode and the exchange test, bcc geometry, fixed-point scales.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rewl_types.h"

namespace rewl {

constexpr unsigned kFullMask = 0xffffffffu;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each multiplies counter words 0
// and 2 by the round constants, keeps both halves of the 64-bit products and permutes/xors them
// with the other words and the round key; the key advances by the Weyl increments.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    const uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
    const uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// 53-bit uniform in [0,1) from the top 27 bits of a and the top 26 bits of b.
__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
  const unsigned long long m = ((unsigned long long)(a >> 5) << 26) | (unsigned long long)(b >> 6);
  return __dmul_rn(__ull2double_rn(m), 0x1.0p-53);
}

// exp(x) in FP64 with one rounding per operation (no contraction), identical on every device and
// reproducible by any IEEE host: x = k ln2 + r (Cody-Waite, ln2 = head + tail with a 29-bit head),
// exp(r) = sum_{n<=13} r^n / n! by Horner, times 2^k.  0 below -708.
__device__ __forceinline__ double exp_fp64(double x, const ExpCoeffs& c) {
  if (x != x) return x;
  if (x < -708.0) return 0.0;
  if (x > 709.0) return __longlong_as_double(0x7ff0000000000000LL);
  const double head = 0x1.62e42ff000000p-1;
  const double tail = -0x1.718432a1b0e26p-35;
  const double inv_ln2 = 0x1.71547652b82fep+0;
  const double kf = floor(__dadd_rn(__dmul_rn(x, inv_ln2), 0.5));
  const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(kf, head)), __dmul_rn(kf, tail));
  double p = c.inv_fact[13];
#pragma unroll
  for (int n = 12; n >= 0; --n) p = __dadd_rn(__dmul_rn(p, r), c.inv_fact[n]);
  const int k = (int)kf;
  const double two_k = __longlong_as_double((long long)(k + 1023) << 52);
  return __dmul_rn(p, two_k);
}

// Half-unit coordinates (X, Y, Z) of bcc site i = 2 (x + L (y + L z)) + s: (2x+s, 2y+s, 2z+s).
// Division by L via the multiplier ceil(2^32 / L), exact for cell indices below 2^32 / L.
__device__ __forceinline__ void bcc_coords(int i, int L, uint32_t divL, int& X, int& Y, int& Z) {
  const int s = i & 1;
  const uint32_t c = (uint32_t)i >> 1;
  const uint32_t q1 = __umulhi(c, divL);
  const uint32_t q2 = __umulhi(q1, divL);
  X = 2 * (int)(c - q1 * (uint32_t)L) + s;
  Y = 2 * (int)(q1 - q2 * (uint32_t)L) + s;
  Z = 2 * (int)q2 + s;
}

// Site index at half-unit offset (dx, dy, dz) from (X, Y, Z), periodic in [0, 2L).
__device__ __forceinline__ int bcc_offset_site(int X, int Y, int Z, int dx, int dy, int dz, int L) {
  const int twoL = 2 * L;
  int x = X + dx, y = Y + dy, z = Z + dz;
  x += (x < 0) ? twoL : 0;
  x -= (x >= twoL) ? twoL : 0;
  y += (y < 0) ? twoL : 0;
  y -= (y >= twoL) ? twoL : 0;
  z += (z < 0) ? twoL : 0;
  z -= (z >= twoL) ? twoL : 0;
  return ((((z >> 1) * L + (y >> 1)) * L + (x >> 1)) << 1) + (x & 1);
}

// Offsets are packed as three biased bytes and the shell: (dx + 8) | (dy + 8) << 8 | (dz + 8) << 16 |
// shell << 24.
__device__ __forceinline__ void unpack_offset(uint32_t p, int& dx, int& dy, int& dz) {
  dx = (int)(p & 0xffu) - 8;
  dy = (int)((p >> 8) & 0xffu) - 8;
  dz = (int)((p >> 16) & 0xffu) - 8;
}

// Production spins are stored as two FP32 octahedral coordinates, 8 bytes per site.  A unit vector s
// is projected to p = s / (|x| + |y| + |z|) on the octahedron |x| + |y| + |z| = 1.  Its upper half
// (z >= 0) is kept as (u, v) = (p_x, p_y); its lower half is folded over the square's edges,
// (u, v) = ((1 - |p_y|) sign p_x, (1 - |p_x|) sign p_y).  Decoding undoes the fold
// (z = 1 - |u| - |v|; for z < 0 x and y move towards 0 by -z) and normalises.  The grid is about
// 1e-7 rad fine everywhere (FP32 spacing of u and v), the resolution of FP32 components.
// Every proposed spin goes through encode and decode before its energy change is taken, and the code
// is what the lattice stores, so the lattice always holds exactly the spin the energy saw.
__device__ __forceinline__ float2 oct_encode(float x, float y, float z) {
  const float s = __fdiv_rn(1.0f, fabsf(x) + fabsf(y) + fabsf(z));
  float u = x * s, v = y * s;
  if (z < 0.0f) {
    const float fu = copysignf(1.0f - fabsf(v), u);
    const float fv = copysignf(1.0f - fabsf(u), v);
    u = fu;
    v = fv;
  }
  return make_float2(u, v);
}

__device__ __forceinline__ void oct_decode(float2 c, float& x, float& y, float& z) {
  z = 1.0f - fabsf(c.x) - fabsf(c.y);
  const float t = fmaxf(-z, 0.0f);
  x = c.x >= 0.0f ? c.x - t : c.x + t;
  y = c.y >= 0.0f ? c.y - t : c.y + t;
  const float r = rsqrtf(fmaf(x, x, fmaf(y, y, z * z)));
  x *= r;
  y *= r;
  z *= r;
}

// Fixed-point scales of the production mode.
//  energy: int64 in units of 2^-32 bins above e_min, so the bin index is the high 32-bit word;
//  ln g, ln f, ln u: int64 in units of 2^-40.
constexpr double kLngScale = 1099511627776.0;        // 2^40
constexpr double kLngUnit = 1.0 / 1099511627776.0;   // 2^-40
constexpr double kEnergyScale = 4294967296.0;        // 2^32 per bin

__device__ __forceinline__ int fx_bin(long long efx) { return (int)(efx >> 32); }

}  // namespace rewl
