// walker_common.cuh -- device pieces shared by the walker kernels: the local field and energy
// change of a trial move, FP64 binning, the trial-move draws of both modes, and the full energy.
#pragma once

#include <type_traits>

#include "device_common.cuh"
#include "walker.h"

namespace rewl {

template <bool kTraj>
struct Mode;
template <>
struct Mode<true> {
  using Real = double;
  using Lng = double;
};
template <>
struct Mode<false> {
  using Real = float;
  using Lng = long long;
};

// Spins of one configuration.
// SpinPlanes: three FP64 arrays x[N], y[N], z[N] -- trajectory lattices, in global memory ([R][3][N])
//   and in shared memory.
// SpinCodes: one float2 octahedral code per site -- production lattices in global memory ([R][N]): a
//   neighbour's spin is one 8-byte load, and eight sites share a 64-byte DRAM access.
// CodePlanes: the same codes as two FP32 arrays u[N], v[N] -- production lattices in shared memory.
// get() returns the spin (decoded in production); trajectory lattices are written with set(x, y, z),
// production lattices with set_code(code).
template <typename Real>
struct SpinPlanes {
  using Value = Real;
  Real *x, *y, *z;
  __device__ __forceinline__ SpinPlanes() : x(nullptr), y(nullptr), z(nullptr) {}
  __device__ __forceinline__ SpinPlanes(Real* p, int N) : x(p), y(p + N), z(p + 2 * (size_t)N) {}
  __device__ __forceinline__ void get(int i, Real& vx, Real& vy, Real& vz) const {
    vx = x[i];
    vy = y[i];
    vz = z[i];
  }
  __device__ __forceinline__ void set(int i, Real vx, Real vy, Real vz) const {
    x[i] = vx;
    y[i] = vy;
    z[i] = vz;
  }
};

struct SpinCodes {
  using Value = float;
  float2* c;
  __device__ __forceinline__ void get(int i, float& vx, float& vy, float& vz) const { oct_decode(c[i], vx, vy, vz); }
  __device__ __forceinline__ float2 get_code(int i) const { return c[i]; }
  __device__ __forceinline__ void set_code(int i, float2 v) const { c[i] = v; }
};

struct CodePlanes {
  using Value = float;
  float *u, *v;
  __device__ __forceinline__ CodePlanes() : u(nullptr), v(nullptr) {}
  __device__ __forceinline__ CodePlanes(float* p, int N) : u(p), v(p + N) {}
  __device__ __forceinline__ void get(int i, float& vx, float& vy, float& vz) const {
    oct_decode(make_float2(u[i], v[i]), vx, vy, vz);
  }
  __device__ __forceinline__ float2 get_code(int i) const { return make_float2(u[i], v[i]); }
  __device__ __forceinline__ void set_code(int i, float2 w) const {
    u[i] = w.x;
    v[i] = w.y;
  }
};

// The global-memory lattice of configuration r: FP64 planes (trajectory) or codes (production).
template <bool kTraj>
struct GlobalLattice {
  using T = SpinPlanes<double>;
  static __device__ __forceinline__ T of(void* spins, int r, int N) {
    return T(reinterpret_cast<double*>(spins) + (size_t)r * 3 * N, N);
  }
};
template <>
struct GlobalLattice<false> {
  using T = SpinCodes;
  static __device__ __forceinline__ T of(void* spins, int r, int N) {
    return SpinCodes{reinterpret_cast<float2*>(spins) + (size_t)r * N};
  }
};

// The lattice a walker reads: its mode's shared-memory layout, else its global layout.
template <bool kTraj, bool kSmem>
struct WalkLattice {
  using T = SpinPlanes<double>;
};
template <>
struct WalkLattice<false, true> {
  using T = CodePlanes;
};
template <bool kTraj>
struct WalkLattice<kTraj, false> {
  using T = typename GlobalLattice<kTraj>::T;
};

// Bytes per site of a lattice in shared memory.
__host__ __device__ constexpr size_t smem_site_bytes(bool traj) { return traj ? 3 * sizeof(double) : 2 * sizeof(float); }

// Copy N spins between a global and a shared-memory lattice by the nt threads t of a group (production
// copies the codes, so a spin never changes on the way).
__device__ __forceinline__ void copy_lattice(const SpinPlanes<double>& d, const SpinPlanes<double>& s, int N, int t,
                                             int nt) {
  for (int i = t; i < N; i += nt) {
    double vx, vy, vz;
    s.get(i, vx, vy, vz);
    d.set(i, vx, vy, vz);
  }
}
template <class Dst, class Src>
__device__ __forceinline__ void copy_lattice(const Dst& d, const Src& s, int N, int t, int nt) {
  for (int i = t; i < N; i += nt) d.set_code(i, s.get_code(i));
}

// Write spin (x, y, z) with production code c at site i (trajectory lattices take the components,
// production lattices the code).
template <class Lat, typename Real>
__device__ __forceinline__ void put_spin(const Lat& lat, int i, Real x, Real y, Real z, float2 c) {
  if constexpr (std::is_same<Lat, SpinPlanes<double>>::value)
    lat.set(i, x, y, z);
  else
    lat.set_code(i, c);
}

__device__ __forceinline__ long long shfl_ll(long long v, int src) {
  return (long long)__shfl_sync(kFullMask, (unsigned long long)v, src);
}

// Energy change of moving spin `site` to (nx, ny, nz), evaluated by the G lanes of one group.
// Summation order: lane `sub` sums slots sub, sub+G, ... in order; then xor butterfly G/2..1.
template <bool kTraj, class Lat>
__device__ __forceinline__ typename Mode<kTraj>::Real delta_energy(
    const WalkerArgs& a, const uint32_t* off_s, const typename Mode<kTraj>::Real* J_s, const Lat& lat,
    int site, int X, int Y, int Z,
    typename Mode<kTraj>::Real nx, typename Mode<kTraj>::Real ny, typename Mode<kTraj>::Real nz,
    int sub, int G, unsigned mask) {
  using Real = typename Mode<kTraj>::Real;
  const int z = a.geo.z, N = a.geo.N, L = a.geo.L;
  Real hx = Real(0), hy = Real(0), hz = Real(0);
  if (a.geo.kind == 0) {
    // production: spins summed per coupling shell (slots are shell-major), each shell sum
    // multiplied by its coupling once -- aligned spins then see no rounding at all
    Real tx = Real(0), ty = Real(0), tz = Real(0), Jcur = Real(0);
    uint32_t shc = 0xffffffffu;
    for (int j = sub; j < z; j += G) {
      int dx, dy, dz;
      const uint32_t o = off_s[j];
      unpack_offset(o, dx, dy, dz);
      const int n = bcc_offset_site(X, Y, Z, dx, dy, dz, L);
      const Real J = J_s[j];
      Real vx, vy, vz;
      lat.get(n, vx, vy, vz);
      if (kTraj) {
        hx = __dadd_rn(hx, __dmul_rn(J, vx));
        hy = __dadd_rn(hy, __dmul_rn(J, vy));
        hz = __dadd_rn(hz, __dmul_rn(J, vz));
      } else {
        const uint32_t sh = o >> 24;
        if (sh != shc) {
          hx = fmaf(Jcur, tx, hx);
          hy = fmaf(Jcur, ty, hy);
          hz = fmaf(Jcur, tz, hz);
          tx = ty = tz = Real(0);
          shc = sh;
          Jcur = J;
        }
        tx += vx;
        ty += vy;
        tz += vz;
      }
    }
    if (!kTraj) {
      hx = fmaf(Jcur, tx, hx);
      hy = fmaf(Jcur, ty, hy);
      hz = fmaf(Jcur, tz, hz);
    }
  } else {
    for (int j = sub; j < z; j += G) {
      const int n = __ldg(a.geo.tab_nbr + (size_t)j * N + site);
      Real vx, vy, vz;
      lat.get(n, vx, vy, vz);
      if (kTraj) {
        const double J = __ldg(a.geo.tab_Jd + (size_t)j * N + site);
        hx = __dadd_rn(hx, __dmul_rn(J, vx));
        hy = __dadd_rn(hy, __dmul_rn(J, vy));
        hz = __dadd_rn(hz, __dmul_rn(J, vz));
      } else {
        const float J = __ldg(a.geo.tab_Jf + (size_t)j * N + site);
        hx = fmaf(J, vx, hx);
        hy = fmaf(J, vy, hy);
        hz = fmaf(J, vz, hz);
      }
    }
  }
  for (int o = G >> 1; o > 0; o >>= 1) {
    const Real px = __shfl_xor_sync(mask, hx, o);
    const Real py = __shfl_xor_sync(mask, hy, o);
    const Real pz = __shfl_xor_sync(mask, hz, o);
    if (kTraj) {
      hx = __dadd_rn(hx, px);
      hy = __dadd_rn(hy, py);
      hz = __dadd_rn(hz, pz);
    } else {
      hx += px;
      hy += py;
      hz += pz;
    }
  }
  Real ox, oy, oz;
  lat.get(site, ox, oy, oz);
  if (kTraj) {
    const double dx = __dsub_rn(nx, ox), dy = __dsub_rn(ny, oy), dz = __dsub_rn(nz, oz);
    return -__dadd_rn(__dadd_rn(__dmul_rn(dx, hx), __dmul_rn(dy, hy)), __dmul_rn(dz, hz));
  } else {
    const float dx = nx - ox, dy = ny - oy, dz = nz - oz;
    return -fmaf(dz, hz, fmaf(dy, hy, dx * hx));
  }
}

// Global bin of an FP64 energy: floor((E - e_min) / dE), clamped to +-2^30.
__device__ __forceinline__ int bin_fp64(double E, const Windows& w) {
  double q = __ddiv_rn(__dsub_rn(E, w.e_min), w.dE);
  if (q != q) return -(1 << 30);
  q = fmin(fmax(q, -1073741824.0), 1073741824.0);
  return (int)floor(q);
}

// Trial-move draws.  Trajectory mode: site and u = u53(x1, x2) from counter (t, p_site, 0);
// direction attempts k = 1.. from (t, p_dir, k), a = 2 u53(x0,x1) - 1, b = 2 u53(x2,x3) - 1,
// accepted when 0 < a^2 + b^2 < 1 (Marsaglia 1972); 64 failures give (0, 0, 1).
__device__ __forceinline__ void draw_traj(uint2 key, unsigned long long t, bool init, int N, int& site,
                                          double& u, double& nx, double& ny, double& nz) {
  const uint32_t lo = (uint32_t)t, hi = (uint32_t)(t >> 32);
  const uint4 x = philox10(make_uint4(lo, hi, init ? 2u : 0u, 0u), key);
  site = (int)__umulhi(x.x, (uint32_t)N);
  u = uniform53(x.y, x.z);
  nx = 0.0;
  ny = 0.0;
  nz = 1.0;
  const uint32_t pdir = init ? 2u : 1u;
  for (uint32_t k = 1; k <= 64; ++k) {
    const uint4 y = philox10(make_uint4(lo, hi, pdir, k), key);
    const double ua = uniform53(y.x, y.y), ub = uniform53(y.z, y.w);
    const double a = __dsub_rn(__dmul_rn(2.0, ua), 1.0);
    const double b = __dsub_rn(__dmul_rn(2.0, ub), 1.0);
    const double q = __dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b));
    if (q < 1.0 && q > 0.0) {
      const double w = __dsqrt_rn(__dsub_rn(1.0, q));
      nx = __dmul_rn(__dmul_rn(2.0, a), w);
      ny = __dmul_rn(__dmul_rn(2.0, b), w);
      nz = __dsub_rn(1.0, __dmul_rn(2.0, q));
      break;
    }
  }
}

// Production draws: one Philox block gives the site (x0), ln u (x1, 2^-40 units) and the first
// direction attempt (x2, x3); further attempts use counter (t, p_dir, k), two per block.  The
// direction uses 24-bit uniforms a = (2m + 1 - 2^24) / 2^24 (never 0) and FP32 arithmetic.
__device__ __forceinline__ float u24_sym(uint32_t x) {
  return (float)((int)((x >> 8) * 2u + 1u) - (1 << 24)) * 0x1.0p-24f;
}

__device__ __forceinline__ void draw_prod(uint2 key, unsigned long long t, bool init, int N, int& site,
                                          long long& lu, float& nx, float& ny, float& nz) {
  const uint32_t lo = (uint32_t)t, hi = (uint32_t)(t >> 32);
  const uint4 x = philox10(make_uint4(lo, hi, init ? 2u : 0u, 0u), key);
  site = (int)__umulhi(x.x, (uint32_t)N);
  const float uf = fmaf(__uint2float_rn(x.y), 0x1.0p-32f, 0x1.0p-33f);   // (0, 1]
  lu = __float2ll_rn(logf(uf) * 0x1.0p40f);
  float a = u24_sym(x.z), b = u24_sym(x.w);
  float q = fmaf(a, a, b * b);
  uint32_t k = 0;
  const uint32_t pdir = init ? 2u : 1u;
  while (!(q < 1.0f) && k < 32) {
    ++k;
    const uint4 y = philox10(make_uint4(lo, hi, pdir, k), key);
    a = u24_sym(y.x);
    b = u24_sym(y.y);
    q = fmaf(a, a, b * b);
    if (q < 1.0f) break;
    a = u24_sym(y.z);
    b = u24_sym(y.w);
    q = fmaf(a, a, b * b);
  }
  if (q < 1.0f) {
    const float w = sqrtf(1.0f - q);
    nx = 2.0f * a * w;
    ny = 2.0f * b * w;
    nz = fmaf(-2.0f, q, 1.0f);
  } else {
    nx = 0.0f;
    ny = 0.0f;
    nz = 1.0f;
  }
}

// Error-free transformations in FP32 (Knuth's two-sum; the product error from a fused multiply-add):
// (hi, lo) pairs carry about 48 significant bits.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

__device__ __forceinline__ void ff_add(float& hi, float& lo, float x, float xe) {
  const float s = hi + x;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += err + xe;
}

// Barrier over the nt threads of a group (id 0 with nt = blockDim.x is __syncthreads()).
__device__ __forceinline__ void group_sync(int id, int nt) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nt) : "memory");
}

// Sum over the nt threads t = 0..nt-1 of a group (warp-aligned), valid in thread t = 0.
__device__ __forceinline__ double block_sum_double(double v, double* red, int t, int nt, int bar) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
  const int w = t >> 5;
  if ((t & 31) == 0) red[w] = v;
  group_sync(bar, nt);
  double s = 0.0;
  if (t == 0)
    for (int i = 0; i < (nt >> 5); ++i) s += red[i];
  group_sync(bar, nt);
  return s;
}

// Full energy of a configuration, E = -w sum_i sum_{energy slots} J S_i.S_n, by the nt threads
// t = 0..nt-1 of a group that synchronises on barrier bar; valid in thread t = 0.
template <bool kTraj, class Lat>
__device__ double full_energy(const WalkerArgs& a, const uint32_t* off_s, const Lat& lat, double* red, int t,
                              int nt, int bar) {
  using Real = typename Mode<kTraj>::Real;
  const int N = a.geo.N;
  const bool bcc = a.geo.kind == 0;
  double part = 0.0;
  float hi = 0.0f, lo = 0.0f;
  for (int i = t; i < N; i += nt) {
    int X = 0, Y = 0, Z = 0;
    if (bcc) bcc_coords(i, a.geo.L, a.geo.divL, X, Y, Z);
    if (kTraj) {
      double hx = 0.0, hy = 0.0, hz = 0.0;
      for (int e = 0; e < a.geo.n_energy_slots; ++e) {
        const int j = a.geo.energy_slot[e];
        int n;
        double J;
        if (bcc) {
          int dx, dy, dz;
          unpack_offset(off_s[j], dx, dy, dz);
          n = bcc_offset_site(X, Y, Z, dx, dy, dz, a.geo.L);
          J = a.geo.Jd[j];
        } else {
          n = a.geo.tab_nbr[(size_t)j * N + i];
          J = a.geo.tab_Jd[(size_t)j * N + i];
        }
        Real vx, vy, vz;
        lat.get(n, vx, vy, vz);
        hx += J * vx;
        hy += J * vy;
        hz += J * vz;
      }
      Real six, siy, siz;
      lat.get(i, six, siy, siz);
      part += six * hx + siy * hy + siz * hz;
    } else {
      // float-float throughout: with nearly parallel spins every site has nearly the same field,
      // so plain FP32 rounding errors would add up coherently over N sites
      float hxh = 0.f, hxl = 0.f, hyh = 0.f, hyl = 0.f, hzh = 0.f, hzl = 0.f;
      for (int e = 0; e < a.geo.n_energy_slots; ++e) {
        const int j = a.geo.energy_slot[e];
        int n;
        float J;
        if (bcc) {
          int dx, dy, dz;
          unpack_offset(off_s[j], dx, dy, dz);
          n = bcc_offset_site(X, Y, Z, dx, dy, dz, a.geo.L);
          J = a.geo.Jf[j];
        } else {
          n = a.geo.tab_nbr[(size_t)j * N + i];
          J = a.geo.tab_Jf[(size_t)j * N + i];
        }
        Real vx, vy, vz;
        lat.get(n, vx, vy, vz);
        float p, pe;
        two_prod(J, (float)vx, p, pe);
        ff_add(hxh, hxl, p, pe);
        two_prod(J, (float)vy, p, pe);
        ff_add(hyh, hyl, p, pe);
        two_prod(J, (float)vz, p, pe);
        ff_add(hzh, hzl, p, pe);
      }
      float p, pe;
      Real rx, ry, rz;
      lat.get(i, rx, ry, rz);
      const float six = (float)rx, siy = (float)ry, siz = (float)rz;
      two_prod(six, hxh, p, pe);
      ff_add(hi, lo, p, fmaf(six, hxl, pe));
      two_prod(siy, hyh, p, pe);
      ff_add(hi, lo, p, fmaf(siy, hyl, pe));
      two_prod(siz, hzh, p, pe);
      ff_add(hi, lo, p, fmaf(siz, hzl, pe));
    }
  }
  if (!kTraj) part = (double)hi + (double)lo;
  const double tot = block_sum_double(part, red, t, nt, bar);
  return -(double)a.geo.energy_weight * tot;
}


}  // namespace rewl
