// walker_pipe.cu -- warp-specialised Wang-Landau walker for bcc lattices, one lane per trial move
// (Sec. 4.2, Eq. 4; trial move Sec. 4.4).
//
// One CTA per walker slot.  Warp 1 (producer) prepares batch b+1 of 32 trial moves while warp 0
// (resolver) resolves batch b strictly in order, so the walk is the sequential Markov chain:
//   producer: Philox draws, the local field h_i = sum_j J_ij S_j over the coupling shells (bcc
//     offsets known at compile time, the neighbour loads in one unrolled loop), dE = -(S'-S).h, and
//     two conflict masks read from a shared-memory owner table -- the moves of batch b (still being
//     resolved while batch b+1 reads the lattice) and the earlier moves of batch b+1 that sit on the
//     same site or a neighbouring one;
//   resolver: a move whose mask meets a move accepted since the lattice was read is corrected
//     exactly (production: from the move records; trajectory: re-evaluated on the current lattice);
//     then accept with min[1, g(E)/g(E')] (reject outside the window) and add ln f to ln g and 1 to
//     H at the resulting state.
// The owner table may alias sites (hashed): an alias names a move that cannot change the field, so
// its correction changes nothing, and the production walker over a global lattice drops it before
// it becomes an event.  Two record buffers alternate; named barriers READY(b mod 2) and DONE(b mod 2)
// order the hand-over, so the producer reads the lattice only after every move of batch b-1 has been
// written.
#include <cstring>

#include "walker_common.cuh"

namespace rewl {

struct ShellTable {
  int dx[kMaxSlotsPerSite], dy[kMaxSlotsPerSite], dz[kMaxSlotsPerSite], sh[kMaxSlotsPerSite];
  int z;
};

// Canonical bcc slot order: shell by shell (squared half-unit lengths 3, 4, 8, 11), lexicographic
// (dx, dy, dz) inside a shell.
constexpr ShellTable make_shells(int nsh) {
  ShellTable t{};
  constexpr int r2s[4] = {3, 4, 8, 11};
  int z = 0;
  for (int s = 0; s < nsh; ++s)
    for (int a = -3; a <= 3; ++a)
      for (int b = -3; b <= 3; ++b)
        for (int c = -3; c <= 3; ++c) {
          if (((a ^ b) & 1) != 0 || ((b ^ c) & 1) != 0) continue;
          if (a * a + b * b + c * c != r2s[s]) continue;
          t.dx[z] = a;
          t.dy[z] = b;
          t.dz[z] = c;
          t.sh[z] = s;
          ++z;
        }
  t.z = z;
  return t;
}

constexpr int kPairThreads = 64;   // resolver warp + producer warp
constexpr int kWorkerThreads = 64;     // batched walker: threads per worker (one pair)

__host__ __device__ constexpr size_t align16(size_t n) { return (n + 15) & ~(size_t)15; }

__device__ __forceinline__ void named_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kPairThreads) : "memory");
}
__device__ __forceinline__ void named_arrive(int id) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(kPairThreads) : "memory");
}

template <bool kTraj>
struct alignas(16) Rec;
template <>
struct alignas(16) Rec<false> {
  long long dq;          // energy increment, 2^-32 bins (a 2^-24-bin integer shifted left by 8)
  int lu;                // ln u, 2^-20 units
  uint32_t cprev;        // batch b-1 moves touching this move's neighbourhood
  uint32_t ccur;         // earlier moves of this batch touching it
  int site;
  float nx, ny, nz;      // proposed spin
  float ox, oy, oz;      // spin at the site before the move (snapshot, corrected by the resolver)
  float hx, hy, hz;      // local field (snapshot, corrected by the resolver)
  float dsx, dsy, dsz;   // new - old spin: the move's change to the lattice if accepted
  float cu, cv;          // octahedral code of the proposed spin (what the lattice stores)
};
template <>
struct alignas(16) Rec<true> {
  double dE;
  double u;
  uint32_t cprev, ccur;
  int site, pad;
  double nx, ny, nz, pad2;
};

// Local field of (X, Y, Z) by one lane over all slots in canonical order, with the owner-table
// words of the site's neighbours OR-ed into own0 / own1 (kOwn).
template <bool kTraj, int NSH, bool kOwn = true, class Lat>
__device__ __forceinline__ void field_one_lane(const Lat& lat, int X, int Y, int Z, int L, const typename Mode<kTraj>::Real (&Jsh)[4],
                                               typename Mode<kTraj>::Real& hx, typename Mode<kTraj>::Real& hy,
                                               typename Mode<kTraj>::Real& hz, const uint2* own, uint32_t omask,
                                               uint32_t& own0, uint32_t& own1) {
  using Real = typename Mode<kTraj>::Real;
  constexpr ShellTable T = make_shells(NSH);
  const int twoL = 2 * L, LL = L * L;
  int xw[7], yw[7], zw[7];
#pragma unroll
  for (int d = -3; d <= 3; ++d) {
    int x = X + d, y = Y + d, z = Z + d;
    x += (x < 0) ? twoL : 0;
    x -= (x >= twoL) ? twoL : 0;
    y += (y < 0) ? twoL : 0;
    y -= (y >= twoL) ? twoL : 0;
    z += (z < 0) ? twoL : 0;
    z -= (z >= twoL) ? twoL : 0;
    xw[d + 3] = x;
    yw[d + 3] = L * y;
    zw[d + 3] = LL * z;
  }
  // site = x' + L y' + L^2 z' - s' (L + L^2), s' the neighbour's sublattice
  const int s = X & 1;
  const int par_same = s * (L + LL), par_flip = (s ^ 1) * (L + LL);
  hx = Real(0);
  hy = Real(0);
  hz = Real(0);
  // production: per-shell spin sums first, then one coupling per shell -- fewer roundings, and
  // none at all for aligned spins (whose dE would otherwise carry the same rounding every move)
  Real tx[4] = {Real(0), Real(0), Real(0), Real(0)}, ty[4] = {Real(0), Real(0), Real(0), Real(0)},
       tz[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
  for (int j = 0; j < T.z; ++j) {
    const int n = xw[T.dx[j] + 3] + yw[T.dy[j] + 3] + zw[T.dz[j] + 3] - ((T.dx[j] & 1) ? par_flip : par_same);
    Real vx, vy, vz;
    lat.get(n, vx, vy, vz);
    if constexpr (kTraj) {
      const Real J = Jsh[T.sh[j]];
      hx = __dadd_rn(hx, __dmul_rn(J, vx));
      hy = __dadd_rn(hy, __dmul_rn(J, vy));
      hz = __dadd_rn(hz, __dmul_rn(J, vz));
    } else {
      tx[T.sh[j]] += vx;
      ty[T.sh[j]] += vy;
      tz[T.sh[j]] += vz;
    }
    if constexpr (kOwn) {
      const uint2 o = own[n & omask];
      own0 |= o.x;
      own1 |= o.y;
    }
  }
  if constexpr (!kTraj) {
#pragma unroll
    for (int s2 = 0; s2 < NSH; ++s2) {
      hx = fmaf(Jsh[s2], tx[s2], hx);
      hy = fmaf(Jsh[s2], ty[s2], hy);
      hz = fmaf(Jsh[s2], tz[s2], hz);
    }
  }
}

// Uniform in [1, 2) from the top 23 bits of a word (no integer-to-float conversion).
__device__ __forceinline__ float one_to_two(uint32_t x) { return __uint_as_float(0x3f800000u | (x >> 9)); }

// dE (FP32) -> int32 in 2^-24 bins: dE * (hi + lo) with the product of the head exact (fmaf).
__device__ __forceinline__ int dq24_of(float dE, const Windows& w) {
  const float p = dE * w.dq24_hi;
  const float e = fmaf(dE, w.dq24_hi, -p) + dE * w.dq24_lo;
  return __float2int_rn(p) + __float2int_rn(e);
}

// One exchange interval of walker slot `slot` by a group of nt threads (tid = 0..nt-1, nt a multiple
// of 32, at least 64): warp 0 resolves, warp 1 produces, every warp loads and stores.  smem_raw is
// the group's shared-memory arena (walker_pipe_smem_bytes), red holds nt/32 doubles.  Barrier
// bar_sync spans the group; bar_pair .. bar_pair+3 are READY(0), READY(1), DONE(0), DONE(1) of the
// resolver/producer pair.
template <bool kTraj, bool kSmem, int NSH>
__device__ __forceinline__ void pipe_walk_slot(const WalkerArgs& a, const int slot, const long long moves,
                                               const int recompute, unsigned char* smem_raw, double* red,
                                               const int tid, const int nt, const int bar_sync,
                                               const int bar_pair) {
  using Real = typename Mode<kTraj>::Real;
  using Lng = typename Mode<kTraj>::Lng;
  const int kBarReady = bar_pair, kBarDone = bar_pair + 2;
  const int warp = tid >> 5, lane = tid & 31;
  const int N = a.geo.N, W = a.win.W, L = a.geo.L;
  const int wlo = a.win.starts[global_slot(a.st, slot) / a.win.m];
  const int rep = a.st.perm[slot];
  const uint32_t omask = (uint32_t)a.own_mask;

  // shared layout: ln g | H | offsets | J per slot | records[2][32] | packed records[2][32] | owner
  // table | lattice (in shared memory only); every section starts on a 16-byte boundary
  unsigned char* p = smem_raw;
  Lng* lng_s = reinterpret_cast<Lng*>(p);
  p += align16(sizeof(Lng) * (size_t)W);
  uint32_t* H_s = reinterpret_cast<uint32_t*>(p);
  p += align16((size_t)W * 4);
  uint32_t* off_s = reinterpret_cast<uint32_t*>(p);
  p += 4 * kMaxSlotsPerSite;
  Real* J_s = reinterpret_cast<Real*>(p);
  p += sizeof(Real) * kMaxSlotsPerSite;
  Rec<kTraj>* rec = reinterpret_cast<Rec<kTraj>*>(p);
  p += sizeof(Rec<kTraj>) * 64;
  int4* pk = reinterpret_cast<int4*>(p);          // production: {dq lo, dq hi, ccur, ln u} per move
  p += sizeof(int4) * 64;
  uint2* own = reinterpret_cast<uint2*>(p);
  p += sizeof(uint2) * ((size_t)omask + 1);
  Real* spin_s = reinterpret_cast<Real*>(p);

  const auto glat = GlobalLattice<kTraj>::of(a.st.spins, rep, N);
  typename WalkLattice<kTraj, kSmem>::T lat;
  if constexpr (kSmem)
    lat = typename WalkLattice<kTraj, true>::T(spin_s, N);
  else
    lat = glat;

  const size_t lbase = (size_t)slot * W;
  for (int w = tid; w < W; w += nt) {
    if constexpr (kTraj)
      lng_s[w] = (Lng)a.st.lng[lbase + w];
    else
      lng_s[w] = (Lng)a.st.lng_fx[lbase + w];
    H_s[w] = a.st.H[lbase + w];
  }
  for (int j = tid; j < kMaxSlotsPerSite; j += nt) {
    off_s[j] = a.geo.off[j];
    J_s[j] = kTraj ? (Real)a.geo.Jd[j] : (Real)a.geo.Jf[j];
  }
  for (uint32_t i = tid; i <= omask; i += nt) own[i] = make_uint2(0u, 0u);
  if constexpr (kSmem) copy_lattice(lat, glat, N, tid, nt);
  group_sync(bar_sync, nt);

  const int nb = (int)((moves + 31) / 32);
  const long long t0 = a.st.steps[slot];
  const uint2 key = make_uint2((uint32_t)global_slot(a.st, slot), a.key1);

  if (warp == 1) {
    // ------------------------------- producer -------------------------------
    Real Jsh[4];
#pragma unroll
    for (int s2 = 0; s2 < 4; ++s2) Jsh[s2] = kTraj ? (Real)a.geo.Jsh_d[s2] : (Real)a.geo.Jsh_f[s2];
    int site_prev = 0;
    bool valid_prev = false;
    for (int b = 0; b < nb; ++b) {
      const int cur = b & 1;
      const bool valid = (long long)b * 32 + lane < moves;
      const unsigned long long t = (unsigned long long)(t0 + (long long)b * 32 + lane);
      int site;
      Real nx, ny, nz;
      double u = 0.0;
      int lu = 0;
      float2 code = make_float2(0.0f, 0.0f);
      if constexpr (kTraj) {
        double dnx, dny, dnz;
        draw_traj(key, t, false, N, site, u, dnx, dny, dnz);
        nx = (Real)dnx;
        ny = (Real)dny;
        nz = (Real)dnz;
      } else {
        const uint4 x = philox10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), 0u, 0u), key);
        site = (int)__umulhi(x.x, (uint32_t)N);
        const float uf = (one_to_two(x.y) - 1.0f) + 0x1.0p-24f;                // (0, 1)
        lu = __float2int_rn(__logf(uf) * 1048576.0f);
        const float zc = (2.0f * one_to_two(x.z) - 3.0f) + 0x1.0p-23f;          // (-1, 1), cos(theta)
        float sn, cs;
        __sincosf((one_to_two(x.w) - 1.5f) * 6.28318530717958648f, &sn, &cs);  // azimuth in [-pi, pi)
        const float q = fmaxf(fmaf(-zc, zc, 1.0f), 0x1.0p-46f);
        const float r = q * rsqrtf(q);                                          // sin(theta)
        // the proposal is the spin its code decodes to
        code = oct_encode(r * cs, r * sn, zc);
        float fx, fy, fz;
        oct_decode(code, fx, fy, fz);
        nx = (Real)fx;
        ny = (Real)fy;
        nz = (Real)fz;
      }
      int X, Y, Z;
      bcc_coords(site, L, a.geo.divL, X, Y, Z);
      uint32_t* own32 = reinterpret_cast<uint32_t*>(own);
      if (valid) atomicOr(own32 + 2 * (site & omask) + cur, 1u << lane);
      __syncwarp();
      uint32_t o0 = 0, o1 = 0;
      Real hx, hy, hz;
      // the draws and the owner-table insert above do not touch the lattice, so they overlap the
      // resolver's publication of batch b-2; the lattice holds every batch up to b-2 after DONE
      if (b >= 2) named_sync(kBarDone + (b & 1));
      field_one_lane<kTraj, NSH>(lat, X, Y, Z, L, Jsh, hx, hy, hz, own, omask, o0, o1);
      const uint2 oself = own[site & omask];
      o0 |= oself.x;
      o1 |= oself.y;
      const uint32_t ocur = cur ? o1 : o0, oprev = cur ? o0 : o1;
      Real ox, oy, oz;
      lat.get(site, ox, oy, oz);
      Rec<kTraj>& r = rec[cur * 32 + lane];
      if constexpr (kTraj) {
        const double dx = __dsub_rn(nx, ox), dy = __dsub_rn(ny, oy), dz = __dsub_rn(nz, oz);
        r.dE = -__dadd_rn(__dadd_rn(__dmul_rn(dx, hx), __dmul_rn(dy, hy)), __dmul_rn(dz, hz));
        r.u = u;
      } else {
        const float dx = nx - ox, dy = ny - oy, dz = nz - oz;
        const float dE = -fmaf(dz, hz, fmaf(dy, hy, dx * hx));
        r.dq = (long long)dq24_of(dE, a.win) << 8;
        r.lu = lu;
        r.ox = ox;
        r.oy = oy;
        r.oz = oz;
        r.hx = hx;
        r.hy = hy;
        r.hz = hz;
        r.dsx = dx;
        r.dsy = dy;
        r.dsz = dz;
        r.cu = code.x;
        r.cv = code.y;
      }
      r.cprev = b > 0 ? oprev : 0u;
      r.ccur = ocur & ((1u << lane) - 1u);
      if constexpr (!kTraj) {
        const unsigned long long dqu = (unsigned long long)r.dq;
        pk[cur * 32 + lane] = make_int4((int)(uint32_t)dqu, (int)(uint32_t)(dqu >> 32), (int)r.ccur, r.lu);
      }
      r.site = site;
      r.nx = nx;
      r.ny = ny;
      r.nz = nz;
      __syncwarp();
      named_arrive(kBarReady + cur);
      // batch b+1 inserts into the other slot, which still holds batch b-1's bits
      if (valid_prev) own32[2 * (site_prev & omask) + (cur ^ 1)] = 0u;
      __syncwarp();   // every clear lands before any lane inserts batch b+1
      site_prev = site;
      valid_prev = valid;
    }
    for (int b = nb - 2 > 0 ? nb - 2 : 0; b < nb; ++b) named_sync(kBarDone + (b & 1));
  } else if (warp == 0) {
   if constexpr (kTraj) {
    // ------------------------ resolver (trajectory mode) ------------------------
    double E = 0.0;
    long long Efx = 0;
    int bcur;
    if constexpr (kTraj) {
      E = a.st.E[slot];
      bcur = a.st.bin[slot];
    } else {
      Efx = a.st.efx[slot];
      bcur = fx_bin(Efx);
    }
    double lnf = 0.0;
    long long lnf_fx = 0;
    bool frozen;
    if constexpr (kTraj) {
      lnf = a.st.lnf[slot];
      frozen = !(lnf >= a.lnf_final);
    } else {
      lnf_fx = a.st.lnf_fx[slot];
      frozen = !((double)lnf_fx * kLngUnit >= a.lnf_final);
    }
    const bool bad = (unsigned)(bcur - wlo) >= (unsigned)W;
    if (bad && lane == 0) atomicExch(a.st.ctrl + 0, kErrOutOfWindow);
    Lng lng_cur = bad ? Lng(0) : lng_s[bcur - wlo];
    uint32_t h_cur = bad ? 0u : H_s[bcur - wlo];
    // ln g of the bins next to the current one, kept in registers (production)
    long long lng_m = 0, lng_p = 0;
    if constexpr (!kTraj) {
      if (!bad) {
        lng_m = bcur - 1 >= wlo ? (long long)lng_s[bcur - 1 - wlo] : 0;
        lng_p = bcur + 1 < wlo + W ? (long long)lng_s[bcur + 1 - wlo] : 0;
      }
    }
    constexpr int kWords = (int)(sizeof(Rec<kTraj>) / sizeof(int4));
    uint32_t acc_prev = 0;
    long long n_acc = 0, n_rec = 0;
    for (int b = 0; b < nb; ++b) {
      const int cur = b & 1;
      named_sync(kBarReady + cur);
      const int nvalid = bad ? 0 : (int)(moves - (long long)b * 32 < 32 ? moves - (long long)b * 32 : 32);
      uint32_t acc_cur = 0;
      const int4* R4 = reinterpret_cast<const int4*>(rec + cur * 32);
      // records are read one move ahead, before the stores of the current move
      int4 nxt[kWords];
      if (nvalid > 0) {
#pragma unroll
        for (int q = 0; q < kWords; ++q) nxt[q] = R4[q];
      }
      for (int k = 0; k < nvalid; ++k) {
        Rec<kTraj> r;
        memcpy(&r, nxt, sizeof r);
        if (k + 1 < nvalid) {
#pragma unroll
          for (int q = 0; q < kWords; ++q) nxt[q] = R4[(k + 1) * kWords + q];
        }
        const uint32_t need = (r.cprev & acc_prev) | (r.ccur & acc_cur);
        const int site = r.site;
        bool acc;
        if constexpr (kTraj) {
          double dE = r.dE;
          if (need) {
            __syncwarp();
            int X, Y, Z;
            bcc_coords(site, L, a.geo.divL, X, Y, Z);
            double dn = 0.0;
            if (lane == 0)
              dn = (double)delta_energy<true>(a, off_s, J_s, lat, site, X, Y, Z, r.nx, r.ny, r.nz, 0, 1, 1u);
            dE = __shfl_sync(kFullMask, dn, 0);
            ++n_rec;
          }
          const double Ep = __dadd_rn(E, dE);
          const int bp = bin_fp64(Ep, a.win);
          const int rel = bp - wlo;
          acc = false;
          if ((unsigned)rel < (unsigned)W) {
            const double lngp = (bp == bcur) ? (double)lng_cur : (double)lng_s[rel];
            const double d = __dsub_rn((double)lng_cur, lngp);
            acc = (d >= 0.0) || (r.u < exp_fp64(d, a.ex));
            if (acc) {
              if (bp != bcur) {
                lng_s[bcur - wlo] = lng_cur;
                H_s[bcur - wlo] = h_cur;
                lng_cur = (Lng)lngp;
                h_cur = H_s[rel];
                bcur = bp;
              }
              E = Ep;
            }
          }
        } else {
          int dq = r.dq;
          if (need) {
            __syncwarp();
            int X, Y, Z;
            bcc_coords(site, L, a.geo.divL, X, Y, Z);
            const float dEn = (float)delta_energy<false>(a, off_s, J_s, lat, site, X, Y, Z, r.nx, r.ny, r.nz,
                                                         lane, 32, kFullMask);
            dq = dq24_of(dEn, a.win);
            ++n_rec;
          }
          const long long Ep = Efx + ((long long)dq << 8);
          const int bp = fx_bin(Ep);
          const int db = bp - bcur;
          if (db == 0) {
            acc = true;                      // same bin: ln g ratio 1
          } else {
            const int rel = bp - wlo;
            acc = false;
            if ((unsigned)rel < (unsigned)W) {
              const long long lngp = db == 1 ? lng_p : (db == -1 ? lng_m : (long long)lng_s[rel]);
              const long long d = (long long)lng_cur - lngp;
              const int d20 = d < -(1LL << 51) ? (int)0x80000000 : (int)(d >> 20);
              acc = d >= 0 || r.lu < d20;
              if (acc) {
                lng_s[bcur - wlo] = lng_cur;
                H_s[bcur - wlo] = h_cur;
                if (db == 1) {
                  lng_m = (long long)lng_cur;
                } else if (db == -1) {
                  lng_p = (long long)lng_cur;
                }
                lng_cur = (Lng)lngp;
                h_cur = H_s[rel];
                bcur = bp;
                if (db != -1) lng_p = bcur + 1 < wlo + W ? (long long)lng_s[bcur + 1 - wlo] : 0;
                if (db != 1) lng_m = bcur - 1 >= wlo ? (long long)lng_s[bcur - 1 - wlo] : 0;
              }
            }
          }
          if (acc) Efx = Ep;
        }
        if (acc) {
          acc_cur |= 1u << k;
          ++n_acc;
          if (lane == 0) lat.set(site, r.nx, r.ny, r.nz);
        }
        if (!frozen) {
          if constexpr (kTraj)
            lng_cur = (Lng)__dadd_rn((double)lng_cur, lnf);
          else
            lng_cur = (Lng)((long long)lng_cur + lnf_fx);
          ++h_cur;
        }
      }
      acc_prev = acc_cur;
      __syncwarp();
      named_arrive(kBarDone + cur);
    }
    if (lane == 0 && !bad) {
      if constexpr (kTraj) {
        a.st.E[slot] = E;
        a.st.bin[slot] = bcur;
      } else {
        a.st.efx[slot] = Efx;
      }
      lng_s[bcur - wlo] = lng_cur;
      H_s[bcur - wlo] = h_cur;
      a.st.steps[slot] = t0 + moves;
      a.st.accepts[slot] += n_acc;
      a.st.recomputes[slot] += n_rec;
    }
   } else {
    // ------------------------ resolver (production mode) ------------------------
    // The lattice holds every batch up to b-2 while batch b is resolved: batch b-1's accepted spins
    // are written at the start of batch b, after the producer has read the lattice for batch b.  A
    // move's energy change then follows exactly from the producer's snapshot (field h, old spin o)
    // and the accepted moves of batch b-1 and of batch b before it that touch its neighbourhood:
    // each adds J (S' - S) to h, or replaces o when it sits on the move's own site.  Corrections
    // from batch b-1 are applied by every lane at the start of the batch; those from batch b are
    // out-of-line events of the sequential part.
    // Current bin: its ln g and H stay in registers and are written back only when the walker
    // leaves the bin; ln g of the two neighbouring bins is cached (lng_m, lng_p).
    long long Efx = a.st.efx[slot];
    int bcur = fx_bin(Efx);
    // shell couplings as four scalars: an indexed read of the parameter array would be a
    // constant-memory load whose lanes take different indexes, serialised lane by lane
    const float J0 = a.geo.Jsh_f[0], J1 = NSH > 1 ? a.geo.Jsh_f[1] : 0.0f, J2 = NSH > 2 ? a.geo.Jsh_f[2] : 0.0f,
                J3 = NSH > 3 ? a.geo.Jsh_f[3] : 0.0f;
    const long long lnf_fx = a.st.lnf_fx[slot];
    const bool frozen = !((double)lnf_fx * kLngUnit >= a.lnf_final);
    const long long lnf_eff = frozen ? 0 : lnf_fx;
    const uint32_t hinc = frozen ? 0u : 1u;
    const bool bad = (unsigned)(bcur - wlo) >= (unsigned)W;
    if (bad && lane == 0) atomicExch(a.st.ctrl + 0, kErrOutOfWindow);
    long long lng_in = bad ? 0 : (long long)lng_s[bcur - wlo];
    uint32_t h_in = bad ? 0u : H_s[bcur - wlo];
    long long lng_m = 0, lng_p = 0;
    if (!bad) {
      lng_m = bcur - 1 >= wlo ? (long long)lng_s[bcur - 1 - wlo] : 0;
      lng_p = bcur + 1 < wlo + W ? (long long)lng_s[bcur + 1 - wlo] : 0;
    }
    // coupling between sites p and q: J of q's shell around p, 0 if q is not a neighbour (every
    // offset component is below L half-units, so the wrapped displacement is the offset itself)
    auto coupling = [&](int p, int q) -> float {
      int Xp, Yp, Zp, Xq, Yq, Zq;
      bcc_coords(p, L, a.geo.divL, Xp, Yp, Zp);
      bcc_coords(q, L, a.geo.divL, Xq, Yq, Zq);
      int dx = Xq - Xp, dy = Yq - Yp, dz = Zq - Zp;
      dx += dx < -L ? 2 * L : 0;
      dx -= dx >= L ? 2 * L : 0;
      dy += dy < -L ? 2 * L : 0;
      dy -= dy >= L ? 2 * L : 0;
      dz += dz < -L ? 2 * L : 0;
      dz -= dz >= L ? 2 * L : 0;
      // squared half-unit distances 3, 4, 8, 11 are the shells 1..4
      const int r2 = dx * dx + dy * dy + dz * dz;
      return r2 == 3 ? J0 : (r2 == 4 ? J1 : (r2 == 8 ? J2 : (r2 == 11 ? J3 : 0.0f)));
    };
    // field and old spin of a move at site p after the accepted moves m of record block R, in order;
    // returns the moves among m that sit on site p (a later accepted move supersedes them)
    auto correct = [&](const Rec<false>* R, uint32_t m, int p, float& hx, float& hy, float& hz, float& ox, float& oy,
                       float& oz) -> uint32_t {
      uint32_t same = 0u;
      while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1u;
        const Rec<false>& rj = R[j];
        const int q = rj.site;
        if (q == p) {
          ox = rj.nx;
          oy = rj.ny;
          oz = rj.nz;
          same |= 1u << j;
        } else {
          const float J = coupling(p, q);
          hx = fmaf(J, rj.dsx, hx);
          hy = fmaf(J, rj.dsy, hy);
          hz = fmaf(J, rj.dsz, hz);
        }
      }
      return same;
    };
    // write the accepted spins of record block R: acc minus the moves superseded on their site
    auto publish = [&](const Rec<false>* R, uint32_t acc) {
      if ((acc >> lane) & 1u) {
        const Rec<false>& rp = R[lane];
        lat.set_code(rp.site, make_float2(rp.cu, rp.cv));
      }
      __syncwarp();
    };
    // segment state: the walker entered bcur (or the batch began) at move k_seg with ln g = lng_seg
    // and histogram h_seg; after j more moves there, ln g = lng_seg + j ln f
    long long lng_seg = lng_in;
    uint32_t h_seg = h_in;
    uint32_t acc_prev = 0, pub_prev = 0;
    int n_rec = 0;
    long long n_acc = 0;
    // Three ways through a batch, all with the same decisions; each batch takes the cheapest for
    // the counts of the batch before it: n_rej moves that left the bin to a neighbour and were
    // rejected, n_ev moves resolved out of line (accepted bin changes, jumps of two or more bins,
    // corrections).
    //   scan       -- one warp scan, one ballot round per event: few events (high-energy windows);
    //   blocks     -- branch-free blocks of 8 moves absorb rejected exits: many of those, few others
    //                 (low-energy windows);
    //   sequential -- one move at a time: many full resolutions (bins as narrow as the temperature).
    enum { kScan = 0, kBlocks = 1, kSequential = 2 };
    // several sites share an owner entry (lattices in global memory; a shared-memory lattice keeps
    // its walker's code as it is, which measured faster at bcc L = 16 where its table has an entry
    // per site)
    const bool aliased = !kSmem && (long long)omask + 1 < (long long)N;
    const int forced = a.resolver - 1;      // -1: per-batch choice
    int path = forced >= 0 ? forced : kBlocks;
    int n_scan = 0, n_blocks = 0, n_seq = 0;   // batches per path
    for (int b = 0; b < nb; ++b) {
      const int cur = b & 1;
      named_sync(kBarReady + cur);
      const int nvalid = bad ? 0 : (int)(moves - (long long)b * 32 < 32 ? moves - (long long)b * 32 : 32);
      int k_seg = 0;
      uint32_t acc_cur = 0, sup = 0;
      int n_rej = 0, n_ev = 0;
      Rec<false>* Rc = rec + cur * 32;
      const Rec<false>* Rp = rec + (cur ^ 1) * 32;
      // ---- parallel part: lane = move index ----
      Rec<false>& mine = Rc[lane];
      {
        // An owner table smaller than the lattice is hashed, so a conflict bit may name a move whose
        // site is neither this move's site nor one of its neighbours: such a move cannot change this
        // move's field or old spin.  Drop those bits once here -- from batch b-1 (accepted moves)
        // and from this batch (before any is resolved) -- so that only real conflicts become events
        // below.  (At bcc L = 32 with 2048 entries, 92 % of the flagged moves were such aliases.)
        uint32_t m = lane < nvalid ? (mine.cprev & acc_prev) : 0u;
        const uint32_t cc = (lane < nvalid && aliased) ? mine.ccur : 0u;
        if (aliased && (m | cc)) {
          const int p0 = mine.site;
          uint32_t real_prev = 0u, real_cur = 0u;
          for (uint32_t t = m; t; t &= t - 1u) {
            const int j = __ffs(t) - 1;
            const int q = Rp[j].site;
            if (q == p0 || coupling(p0, q) != 0.0f) real_prev |= 1u << j;
          }
          for (uint32_t t = cc; t; t &= t - 1u) {
            const int j = __ffs(t) - 1;
            const int q = Rc[j].site;
            if (q == p0 || coupling(p0, q) != 0.0f) real_cur |= 1u << j;
          }
          m = real_prev;
          if (real_cur != cc) pk[cur * 32 + lane].z = (int)real_cur;
        }
        // accepted moves of batch b-1 around this move: correct h and o, then dE
        if (m) {
          float hx = mine.hx, hy = mine.hy, hz = mine.hz, ox = mine.ox, oy = mine.oy, oz = mine.oz;
          correct(Rp, m, mine.site, hx, hy, hz, ox, oy, oz);
          const float dx = mine.nx - ox, dy = mine.ny - oy, dz = mine.nz - oz;
          const float dE = -fmaf(dz, hz, fmaf(dy, hy, dx * hx));
          const long long dq = (long long)dq24_of(dE, a.win) << 8;
          mine.dq = dq;
          mine.hx = hx;
          mine.hy = hy;
          mine.hz = hz;
          mine.ox = ox;
          mine.oy = oy;
          mine.oz = oz;
          mine.dsx = dx;
          mine.dsy = dy;
          mine.dsz = dz;
          const unsigned long long dqu = (unsigned long long)dq;
          pk[cur * 32 + lane].x = (int)(uint32_t)dqu;
          pk[cur * 32 + lane].y = (int)(uint32_t)(dqu >> 32);
        }
        n_rec += __popc(__ballot_sync(kFullMask, m != 0u));
      }
      // batch b-1's spins go to the lattice now that the producer has read it for batch b
      if (b > 0) {
        publish(Rp, pub_prev);
        named_arrive(kBarDone + (cur ^ 1));
      } else {
        __syncwarp();
      }
      const int my_lu = mine.lu;
      // would a step to bcur + 1 / bcur - 1 be accepted at this move, given no change of bin since
      // k_seg (lane = move; ln g at move k is lng_seg + (k - k_seg) ln f)
      auto pass_masks = [&](uint32_t& up, uint32_t& down) {
        const long long ln = lng_seg + (long long)(lane - k_seg) * lnf_eff;
        const long long du = ln - lng_p, dd = ln - lng_m;
        const int u20 = du < -(1LL << 51) ? (int)0x80000000 : (int)(du >> 20);
        const int l20 = dd < -(1LL << 51) ? (int)0x80000000 : (int)(dd >> 20);
        const bool pu = bcur + 1 < wlo + W && (du >= 0 || my_lu < u20);
        const bool pd = bcur - 1 >= wlo && (dd >= 0 || my_lu < l20);
        up = __ballot_sync(kFullMask, pu);
        down = __ballot_sync(kFullMask, pd);
      };
      // One move kk with increment dq (corrected first if it meets an accepted move of this batch):
      // Metropolis step on ln g, bin bookkeeping; every lane computes the same values.  Returns
      // whether the walker changed bin.
      auto resolve = [&](const int kk, long long dq, const uint32_t ccur_w, const int lu) -> bool {
        const uint32_t m = ccur_w & acc_cur;
        uint32_t same = 0u;
        if (m) {
          Rec<false>& rk = Rc[kk];
          float hx = rk.hx, hy = rk.hy, hz = rk.hz, ox = rk.ox, oy = rk.oy, oz = rk.oz;
          same = correct(Rc, m, rk.site, hx, hy, hz, ox, oy, oz);
          const float dx = rk.nx - ox, dy = rk.ny - oy, dz = rk.nz - oz;
          const float dEn = -fmaf(dz, hz, fmaf(dy, hy, dx * hx));
          dq = (long long)dq24_of(dEn, a.win) << 8;
          __syncwarp();
          if (lane == 0) {
            rk.dsx = dx;
            rk.dsy = dy;
            rk.dsz = dz;
          }
          __syncwarp();
          ++n_rec;
        }
        const long long Ep = Efx + dq;
        const int db = fx_bin(Ep) - bcur;
        bool acc = true, moved = false;
        if (db != 0) {
          const int bp = bcur + db;
          const int rel = bp - wlo;
          acc = false;
          if ((unsigned)rel < (unsigned)W) {
            const long long lng_now = lng_seg + (long long)(kk - k_seg) * lnf_eff;
            const long long lngp = db == 1 ? lng_p : (db == -1 ? lng_m : (long long)lng_s[rel]);
            const long long d = lng_now - lngp;
            const int e20 = d < -(1LL << 51) ? (int)0x80000000 : (int)(d >> 20);
            acc = d >= 0 || lu < e20;
            moved = acc;
            if (acc) {
              // leave bcur: write it back, shift the neighbour cache, start a new segment
              lng_s[bcur - wlo] = (Lng)lng_now;
              H_s[bcur - wlo] = h_seg + hinc * (uint32_t)(kk - k_seg);
              if (db == 1) lng_m = lng_now;
              if (db == -1) lng_p = lng_now;
              lng_seg = lngp;
              h_seg = H_s[rel];
              k_seg = kk;
              bcur = bp;
              if (db != -1) lng_p = bcur + 1 < wlo + W ? (long long)lng_s[bcur + 1 - wlo] : 0;
              if (db != 1) lng_m = bcur - 1 >= wlo ? (long long)lng_s[bcur - 1 - wlo] : 0;
            }
          }
        }
        if (acc) {
          Efx = Ep;
          acc_cur |= 1u << kk;
          sup |= same;   // earlier accepted moves on this site are no longer the site's spin
        }
        const bool neighbour_reject = !acc && (db == 1 || db == -1) && !m;
        n_rej += neighbour_reject ? 1 : 0;
        n_ev += (db != 0 && !neighbour_reject) || m ? 1 : 0;
        return moved;
      };
      // ---- sequential part as a scan ----
      // A move that stays in the current bin is accepted (ln g ratio 1), so between events the
      // energy is a running sum: with P_k the inclusive prefix sum of the batch's increments and
      // segment base B (fraction before move s minus the prefix before s), move k >= s lands at
      // fraction B + P_k.  The first move that leaves [0, 2^32) -- or meets an accepted move of this
      // batch -- ends the segment: the moves before it stand.  A step to a neighbouring bin whose
      // pass bit is clear is rejected on the spot (the base drops its increment); anything else is
      // resolved on its own.  One scan per batch, one round of ballots per such move.
      const int4* P4 = pk + cur * 32;
      uint32_t up_mask = 0, down_mask = 0;
      if (path == kScan && nvalid > 0) {
        const int4 wk = P4[lane];
        const long long dqk = lane < nvalid ? (long long)(((unsigned long long)(uint32_t)wk.y << 32) | (uint32_t)wk.x)
                                            : 0LL;
        long long P = dqk;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long t = __shfl_up_sync(kFullMask, P, o);
          if (lane >= o) P += t;
        }
        const uint32_t cck = (uint32_t)wk.z;
        const uint32_t below = (1u << lane) - 1u;          // moves before this one
        const uint32_t upto = nvalid >= 32 ? 0xffffffffu : ((1u << nvalid) - 1u);
        pass_masks(up_mask, down_mask);
        long long B = (long long)(uint32_t)Efx;
        int s0 = 0;
        while (true) {
          const uint32_t from_s = ~((1u << s0) - 1u);      // moves s0 .. 31
          const long long pos = B + P;
          const bool live = lane >= s0 && lane < nvalid;
          const uint32_t outs = __ballot_sync(kFullMask, live && (unsigned long long)pos >= (1ull << 32));
          const uint32_t needs = __ballot_sync(kFullMask, live && (cck & (acc_cur | (below & from_s))) != 0u);
          const uint32_t ev = outs | needs;
          if (ev == 0u) {
            // the rest of the batch stays in the bin
            acc_cur |= upto & from_s;
            const long long Pl = __shfl_sync(kFullMask, P, nvalid - 1);
            Efx = ((long long)bcur << 32) | (long long)(uint32_t)(B + Pl);
            break;
          }
          const int e = __ffs(ev) - 1;
          const uint32_t bit = 1u << e;
          acc_cur |= (bit - 1u) & from_s;
          const long long pe = __shfl_sync(kFullMask, pos, e);
          const long long de = __shfl_sync(kFullMask, dqk, e);
          if (!(needs & bit)) {
            // leaves the bin: one bin up or down with the pass bit clear is rejected here
            const bool one_up = pe >= (1LL << 32) && pe < (2LL << 32);
            const bool one_down = pe < 0 && pe >= -(1LL << 32);
            if ((one_up && !(up_mask & bit)) || (one_down && !(down_mask & bit))) {
              ++n_rej;
              B -= de;
              s0 = e + 1;
              if (s0 >= nvalid) {
                Efx = ((long long)bcur << 32) | (long long)(uint32_t)(pe - de);
                break;
              }
              continue;
            }
          }
          Efx = ((long long)bcur << 32) | (long long)(uint32_t)(pe - de);
          const int4 we = P4[e];
          const long long dq = (long long)(((unsigned long long)(uint32_t)we.y << 32) | (uint32_t)we.x);
          if (resolve(e, dq, (uint32_t)we.z, we.w)) pass_masks(up_mask, down_mask);
          s0 = e + 1;
          if (s0 >= nvalid) break;
          B = (long long)(uint32_t)Efx - (pe - B);
        }
      } else if (path == kSequential) {
        // ---- sequential part, one move at a time ----
        int4 w = P4[0];
        for (int kk = 0; kk < nvalid; ++kk) {
          const int4 wn = P4[(kk + 1) & 31];
          const long long dq = (long long)(((unsigned long long)(uint32_t)w.y << 32) | (uint32_t)w.x);
          resolve(kk, dq, (uint32_t)w.z, w.w);
          w = wn;
        }
      } else {
        // ---- sequential part, in branch-free blocks of 8 moves ----
        // Within a bin the state is frac = Efx - (bcur << 32) in [0, 2^32).  A move in the same bin
        // is accepted (frac += dq); a step to a neighbouring bin is accepted iff its pass bit is
        // set, an event handled out of line, like moves that meet an accepted move of this batch
        // and jumps of two or more bins.  The common path uses no compare-and-select: masks come
        // from sign bits.
        pass_masks(up_mask, down_mask);
        uint32_t frac = (uint32_t)Efx;
        int k = 0;
        while (k < nvalid) {
          const uint32_t acc0 = acc_cur;
          uint32_t exc = 0, outb = 0;
          uint32_t fh[8];   // fraction before each move of the block, for the restart
          int4 q[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) q[u] = P4[(k + u) & 31];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int kk = k + u;
            fh[u] = frac;
            const uint32_t lo = (uint32_t)q[u].x;
            const int hi = q[u].y;
            const uint32_t cc = (uint32_t)q[u].z;
            const uint32_t vmask = (uint32_t)((kk - nvalid) >> 31);          // all ones while kk < nvalid
            const uint32_t bit = (1u << (kk & 31)) & vmask;
            const uint32_t t_lo = frac + lo;
            const uint32_t carry = ((frac & lo) | ((frac | lo) & ~t_lo)) >> 31;
            const int th = hi + (int)carry;                                     // high word of frac + dq: bins moved
            const uint32_t nz = (uint32_t)((th | -th) >> 31);                   // all ones iff th != 0
            const uint32_t stay = ~nz & vmask;
            frac = (t_lo & stay) | (frac & ~stay);
            acc_cur |= bit & stay;
            outb |= bit & nz;
            const uint32_t up = (uint32_t)(((th - 1) | (1 - th)) >> 31);       // all ones iff th != 1
            const uint32_t dn = (uint32_t)(((th + 1) | (-1 - th)) >> 31);      // all ones iff th != -1
            const uint32_t far = nz & up & dn;                                  // |th| >= 2
            const uint32_t need = cc & acc_cur & ~bit;
            exc |= bit & (((~up) & up_mask) | ((~dn) & down_mask) | far | (need ? 0xffffffffu : 0u));
          }
          if (exc == 0u) {
            n_rej += __popc(outb);
            k += 8;
            continue;
          }
          n_rej += __popc(outb & ((exc & (0u - exc)) - 1u));
          // first exceptional move: the block's moves before it stand; restore the state there
          const int kx = __ffs(exc) - 1;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (k + u == kx) frac = fh[u];
          acc_cur = acc0 | (acc_cur & ((1u << kx) - 1u));
          Efx = ((long long)bcur << 32) | frac;
          const int4 wx = P4[kx];
          const long long dq = (long long)(((unsigned long long)(uint32_t)wx.y << 32) | (uint32_t)wx.x);
          if (resolve(kx, dq, (uint32_t)wx.z, wx.w)) pass_masks(up_mask, down_mask);
          frac = (uint32_t)Efx;
          k = kx + 1;
        }
        Efx = ((long long)bcur << 32) | frac;
      }
      // measured: blocks cost about 90 cycles per move whatever the rejected exits; the scan about
      // 200 per batch plus 260 per event, so it wins below about 10 events per batch
      if (nvalid > 0) {
        n_scan += path == kScan ? 1 : 0;
        n_blocks += path == kBlocks ? 1 : 0;
        n_seq += path == kSequential ? 1 : 0;
      }
      path = forced >= 0 ? forced : ((n_rej + n_ev <= 10) ? kScan : (n_ev >= 6 ? kSequential : kBlocks));
      // the batch's moves at the current bin
      lng_seg += (long long)(nvalid - k_seg) * lnf_eff;
      h_seg += hinc * (uint32_t)(nvalid - k_seg);
      n_acc += __popc(acc_cur);
      acc_prev = acc_cur;
      pub_prev = acc_cur & ~sup;
    }
    // the last batch's spins
    if (nb > 0) {
      publish(rec + ((nb - 1) & 1) * 32, pub_prev);
      named_arrive(kBarDone + ((nb - 1) & 1));
    }
    if (lane == 0 && !bad) {
      a.st.efx[slot] = Efx;
      lng_s[bcur - wlo] = (Lng)lng_seg;
      H_s[bcur - wlo] = h_seg;
      a.st.steps[slot] = t0 + moves;
      a.st.accepts[slot] += n_acc;
      a.st.recomputes[slot] += n_rec;
      a.st.path_batches[3 * (size_t)slot + 0] += n_scan;
      a.st.path_batches[3 * (size_t)slot + 1] += n_blocks;
      a.st.path_batches[3 * (size_t)slot + 2] += n_seq;
    }
   }
  }
  group_sync(bar_sync, nt);

  if constexpr (kSmem) copy_lattice(glat, lat, N, tid, nt);
  for (int w = tid; w < W; w += nt) {
    if constexpr (kTraj)
      a.st.lng[lbase + w] = (double)lng_s[w];
    else
      a.st.lng_fx[lbase + w] = (long long)lng_s[w];
    a.st.H[lbase + w] = H_s[w];
  }
  if (recompute) {
    const double Ef = full_energy<kTraj>(a, off_s, lat, red, tid, nt, bar_sync);
    if (tid == 0) {
      if constexpr (kTraj) {
        const double d = fabs(Ef - a.st.E[slot]);
        if (d > a.st.drift[slot]) a.st.drift[slot] = d;
      } else {
        const long long efx = a.st.efx[slot];
        const double Er = a.win.e_min + a.win.dE * ((double)efx / kEnergyScale);
        const double d = fabs(Ef - Er);
        if (d > a.st.drift[slot]) a.st.drift[slot] = d;
        long long nf = __double2ll_rn((Ef - a.win.e_min) / a.win.dE * kEnergyScale);
        const long long lo_fx = (long long)wlo << 32;
        const long long hi_fx = ((long long)(wlo + W) << 32) - 1;
        nf = nf < lo_fx ? lo_fx : (nf > hi_fx ? hi_fx : nf);
        a.st.efx[slot] = nf;
      }
    }
  }
}

// One CTA per slot; barrier 0 spans the CTA, 1..4 serve the pair.  Lattice in shared memory,
// arguments as kernel parameters.  The arena holds the lattice, so at bcc L = 16 one CTA fills an
// SM's shared memory; the register budget is left open (minimum one block per SM), which measured
// about 1 % faster on GB300 than the default budget.  (Small lattices fit 4 CTAs per SM by
// registers at this budget.)
template <bool kTraj, int NSH>
__global__ void __launch_bounds__(kWalkerThreads, 1) walker_pipe_kernel(const WalkerArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kWalkerThreads / 32];
  pipe_walk_slot<kTraj, true, NSH>(a, blockIdx.x, a.moves, a.recompute, smem_raw, red, threadIdx.x, blockDim.x, 0, 1);
}

// The same over a lattice in global memory, with the arguments read from a device copy (through
// L1) and the per-launch moves and recompute flag as parameters.  On GB300 the bcc L = 32
// four-shell walker ran 25 % faster this way than with parameter arguments, while the
// shared-memory walker ran 3 % slower, so each keeps its own form.  Register budget: four blocks
// per SM (128 registers), the residency that runs 512 walkers in one wave at 2048-entry tables;
// 4 % faster than the default budget (96 registers).
template <bool kTraj, int NSH>
__global__ void __launch_bounds__(kWalkerThreads, 4)
    walker_pipe_global_kernel(const WalkerArgs* __restrict__ ap, long long moves, int recompute) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kWalkerThreads / 32];
  pipe_walk_slot<kTraj, false, NSH>(*ap, blockIdx.x, moves, recompute, smem_raw, red, threadIdx.x, blockDim.x, 0, 1);
}

// Persistent walker over many jobs: every 64-thread worker (resolver warp + producer warp) takes
// (job, slot) items from the work list until it is exhausted; a CTA holds `workers` workers, each
// with its own shared-memory arena and barriers (1 + 5w .. 5 + 5w).  A job's lattice sits in the
// arena or stays in global memory (L2) as its smem_lattice flag says.
// Register budget: at least two blocks of the largest shape per SM (at most 170 registers per
// thread).  The tunings the autotuner picks are limited by shared memory, not registers; on GB300
// the 64-job batch ran 7 % faster at this budget (168 registers, no spills) than at the default
// (96 registers and a spill) and 3 % faster than with the budget fully open.
template <bool kTraj, int NSH>
__global__ void __launch_bounds__(kBatchMaxWorkers * kWorkerThreads, 2)
    walker_batch_kernel(const WalkerArgs* __restrict__ jobs, const int2* __restrict__ items, int n_items, int* head,
                        long long moves, int recompute, unsigned arena) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kBatchMaxWorkers][kWorkerThreads / 32];
  __shared__ int next[kBatchMaxWorkers];
  const int w = threadIdx.x / kWorkerThreads, wt = threadIdx.x % kWorkerThreads;
  const int bar_sync = 1 + 5 * w, bar_pair = 2 + 5 * w;
  unsigned char* mine = smem_raw + (size_t)w * arena;
  for (;;) {
    // every thread has read next[w] before the first barrier inside the walk, so the next write
    // cannot overtake a read
    if (wt == 0) next[w] = atomicAdd(head, 1);
    group_sync(bar_sync, kWorkerThreads);
    const int it = next[w];
    if (it >= n_items) break;
    const int2 js = items[it];
    const WalkerArgs& a = jobs[js.x];
    if (a.smem_lattice)
      pipe_walk_slot<kTraj, true, NSH>(a, js.y, moves, recompute, mine, red[w], wt, kWorkerThreads, bar_sync,
                                       bar_pair);
    else
      pipe_walk_slot<kTraj, false, NSH>(a, js.y, moves, recompute, mine, red[w], wt, kWorkerThreads, bar_sync,
                                        bar_pair);
  }
}

template <bool kTraj, int NSH>
static cudaError_t batch_kernel_setup(int workers, size_t arena, int* blocks_per_sm) {
  const size_t smem = (size_t)workers * arena;
  cudaError_t e = cudaFuncSetAttribute(walker_batch_kernel<kTraj, NSH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, walker_batch_kernel<kTraj, NSH>,
                                                       workers * kWorkerThreads, smem);
}

cudaError_t setup_walkers_batch(bool traj, int n_shells, int workers, size_t arena, int* blocks_per_sm) {
  if (workers < 1 || workers > kBatchMaxWorkers) return cudaErrorInvalidValue;
  switch (n_shells * 2 + (traj ? 1 : 0)) {
    case 2: return batch_kernel_setup<false, 1>(workers, arena, blocks_per_sm);
    case 3: return batch_kernel_setup<true, 1>(workers, arena, blocks_per_sm);
    case 4: return batch_kernel_setup<false, 2>(workers, arena, blocks_per_sm);
    case 5: return batch_kernel_setup<true, 2>(workers, arena, blocks_per_sm);
    case 6: return batch_kernel_setup<false, 3>(workers, arena, blocks_per_sm);
    case 7: return batch_kernel_setup<true, 3>(workers, arena, blocks_per_sm);
    case 8: return batch_kernel_setup<false, 4>(workers, arena, blocks_per_sm);
    case 9: return batch_kernel_setup<true, 4>(workers, arena, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_walkers_batch(const BatchLaunch& b, cudaStream_t stream) {
  if (b.workers < 1 || b.workers > kBatchMaxWorkers || b.grid < 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(b.head, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  const dim3 grid(b.grid), block(b.workers * kWorkerThreads);
  const size_t smem = (size_t)b.workers * b.arena;
  const unsigned arena = (unsigned)b.arena;
#define REWL_BATCH_LAUNCH(T, S) \
  walker_batch_kernel<T, S><<<grid, block, smem, stream>>>(b.jobs, b.items, b.n_items, b.head, b.moves, b.recompute, arena)
  switch (b.n_shells * 2 + (b.traj ? 1 : 0)) {
    case 2: REWL_BATCH_LAUNCH(false, 1); break;
    case 3: REWL_BATCH_LAUNCH(true, 1); break;
    case 4: REWL_BATCH_LAUNCH(false, 2); break;
    case 5: REWL_BATCH_LAUNCH(true, 2); break;
    case 6: REWL_BATCH_LAUNCH(false, 3); break;
    case 7: REWL_BATCH_LAUNCH(true, 3); break;
    case 8: REWL_BATCH_LAUNCH(false, 4); break;
    case 9: REWL_BATCH_LAUNCH(true, 4); break;
    default: return cudaErrorInvalidValue;
  }
#undef REWL_BATCH_LAUNCH
  return cudaGetLastError();
}

size_t walker_pipe_smem_bytes(bool traj, bool smem_lattice, int N, int W, int own_entries) {
  const size_t lng = align16((traj ? sizeof(double) : sizeof(long long)) * (size_t)W);
  const size_t h = align16((size_t)W * 4);
  const size_t real = traj ? sizeof(double) : sizeof(float);
  const size_t recs = (traj ? sizeof(Rec<true>) : sizeof(Rec<false>)) * 64 + sizeof(int4) * 64;
  size_t bytes = lng + h + 4 * kMaxSlotsPerSite + real * kMaxSlotsPerSite + recs + 8 * (size_t)own_entries;
  if (smem_lattice) bytes += smem_site_bytes(traj) * (size_t)N;
  return bytes;
}

template <bool kTraj, int NSH>
static cudaError_t launch_pipe_t(const WalkerArgs& a, const WalkerArgs* d_args, int n_slots, size_t smem,
                                 cudaStream_t stream) {
  if (d_args) {
    cudaError_t e = cudaFuncSetAttribute(walker_pipe_global_kernel<kTraj, NSH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    walker_pipe_global_kernel<kTraj, NSH><<<n_slots, kWalkerThreads, smem, stream>>>(d_args, a.moves, a.recompute);
  } else {
    cudaError_t e = cudaFuncSetAttribute(walker_pipe_kernel<kTraj, NSH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    walker_pipe_kernel<kTraj, NSH><<<n_slots, kWalkerThreads, smem, stream>>>(a);
  }
  return cudaGetLastError();
}

template <bool kTraj>
static cudaError_t launch_pipe_shells(const WalkerArgs& a, const WalkerArgs* d_args, int n_slots, size_t smem,
                                      cudaStream_t stream) {
  switch (a.geo.n_shells) {
    case 1: return launch_pipe_t<kTraj, 1>(a, d_args, n_slots, smem, stream);
    case 2: return launch_pipe_t<kTraj, 2>(a, d_args, n_slots, smem, stream);
    case 3: return launch_pipe_t<kTraj, 3>(a, d_args, n_slots, smem, stream);
    case 4: return launch_pipe_t<kTraj, 4>(a, d_args, n_slots, smem, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_walkers_pipe(const WalkerArgs& a, const WalkerArgs* d_args, int n_slots, bool traj, size_t smem,
                                cudaStream_t stream) {
  if (a.smem_lattice == (d_args != nullptr)) return cudaErrorInvalidValue;
  return traj ? launch_pipe_shells<true>(a, d_args, n_slots, smem, stream)
              : launch_pipe_shells<false>(a, d_args, n_slots, smem, stream);
}

}  // namespace rewl
