// walker.cu -- the persistent Wang-Landau walker kernel (Sec. 4.2, Eq. 4; trial move Sec. 4.4).
//
// One CTA per walker slot (window k, walker a).  The CTA stages the slot's ln g / H tables and,
// when it fits, the whole spin lattice of its configuration in shared memory; warp 0 then runs
// `moves` trial moves.  The walk is a strict Markov chain, so it is advanced in speculative
// batches of K = 32 / G moves:
//   phase A (parallel, one group of G lanes per move): Philox draws (site, acceptance variate,
//     new direction), the local field h_i = sum_j J_ij S_j as a G-lane reduction, dE = -(S'-S).h,
//     and a bitmask of the earlier moves in the batch whose site is the same site or one of its
//     neighbours;
//   phase B (sequential, warp-uniform): for k = 0..K-1 the move is re-evaluated if an earlier
//     accepted move in the batch touched its neighbourhood, then accepted with
//     min[1, g(E)/g(E')] (reject outside the window), and ln g += ln f, H += 1 at the resulting
//     state.  The current bin's ln g and H live in registers until the walker leaves the bin.
// The result is the sequential walk exactly: in trajectory mode (FP64, no contraction) it
// reproduces the FP64 reference walk bit for bit.
//
// Production mode keeps FP64 out of the per-move chain (FP64 has a 64-cycle latency on this
// GPU): spins and dE in FP32; the energy as int64 in 2^-32 bin units (bin = high word); ln g,
// ln f and ln u as int64 in 2^-40 units, so ln g accumulates ln f increments exactly.
#include <cstdio>

#include "walker_common.cuh"

namespace rewl {

// Warp 0: the walk.  All state below is warp-uniform unless named per-lane.
template <bool kTraj, class Lat>
__device__ void walk(const WalkerArgs& a, int slot, int wlo, typename Mode<kTraj>::Lng* lng_s,
                     uint32_t* H_s, const uint32_t* off_s, const typename Mode<kTraj>::Real* J_s, const Lat& lat) {
  using Real = typename Mode<kTraj>::Real;
  using Lng = typename Mode<kTraj>::Lng;
  const int lane = threadIdx.x & 31;
  const int G = a.G, K = 32 / G;
  const int g = lane / G, sub = lane % G;
  const unsigned gmask = (G == 32) ? kFullMask : (((1u << G) - 1u) << (g * G));
  const int N = a.geo.N, W = a.win.W;
  const bool bcc = a.geo.kind == 0;
  const bool init = a.init != 0;
  const uint2 key = make_uint2((uint32_t)global_slot(a.st, slot), a.key1);

  // ---- uniform walker state ----
  double E = 0.0;
  long long Efx = 0;
  int bcur;
  if (kTraj) {
    E = a.st.E[slot];
    bcur = a.st.bin[slot];
  } else {
    Efx = a.st.efx[slot];
    bcur = fx_bin(Efx);
  }
  double lnf = 0.0;
  long long lnf_fx = 0;
  bool frozen;
  if (kTraj) {
    lnf = a.st.lnf[slot];
    frozen = !(lnf >= a.lnf_final);
  } else {
    lnf_fx = a.st.lnf_fx[slot];
    frozen = !((double)lnf_fx * kLngUnit >= a.lnf_final);
  }
  if (!init && (unsigned)(bcur - wlo) >= (unsigned)W) {
    if (lane == 0) atomicExch(a.st.ctrl + 0, kErrOutOfWindow);
    return;
  }
  // initial drive: target = window centre
  const double c_traj = kTraj ? __dadd_rn(a.win.e_min, __dmul_rn(__dadd_rn((double)wlo, __dmul_rn((double)W, 0.5)), a.win.dE)) : 0.0;
  const long long c_fx = ((long long)(2 * wlo + W)) << 31;

  Lng lng_cur = Lng(0);
  uint32_t h_cur = 0;
  if (!init) {
    lng_cur = lng_s[bcur - wlo];
    h_cur = H_s[bcur - wlo];
  }
  long long t = init ? 0 : a.st.steps[slot];
  long long remaining = init ? a.init_cap : a.moves;
  long long n_acc = 0, n_rec = 0;
  bool done = false;

  while (remaining > 0 && !done) {
    const int nvalid = (int)(remaining < (long long)K ? remaining : (long long)K);

    // ---------------- phase A: K moves in parallel ----------------
    int site, X = 0, Y = 0, Z = 0;
    Real nx, ny, nz;
    double u = 0.0;
    long long lu = 0;
    float2 code = make_float2(0.0f, 0.0f);
    const unsigned long long tk = (unsigned long long)(t + g);
    if (kTraj) {
      double dnx, dny, dnz;
      draw_traj(key, tk, init, N, site, u, dnx, dny, dnz);
      nx = (Real)dnx;
      ny = (Real)dny;
      nz = (Real)dnz;
    } else {
      float fnx, fny, fnz;
      draw_prod(key, tk, init, N, site, lu, fnx, fny, fnz);
      code = oct_encode(fnx, fny, fnz);        // the proposal is the spin its code decodes to
      oct_decode(code, fnx, fny, fnz);
      nx = (Real)fnx;
      ny = (Real)fny;
      nz = (Real)fnz;
    }
    if (bcc) bcc_coords(site, a.geo.L, a.geo.divL, X, Y, Z);
    const Real dE = delta_energy<kTraj>(a, off_s, J_s, lat, site, X, Y, Z, nx, ny, nz, sub, G, kFullMask);
    long long dq = 0;
    if (!kTraj) dq = __double2ll_rn((double)dE * a.win.dq_scale64);

    // conflicts with earlier moves of the batch: same site or a neighbour of it
    uint32_t conf = 0;
    if (bcc) {
      const uint32_t packed = (uint32_t)X | ((uint32_t)Y << 10) | ((uint32_t)Z << 20);
      const int L = a.geo.L, twoL = 2 * a.geo.L;
      for (int j = 0; j + 1 < K; ++j) {
        const uint32_t pj = __shfl_sync(kFullMask, packed, j * G);
        if (j < g) {
          int ex = X - (int)(pj & 1023u), ey = Y - (int)((pj >> 10) & 1023u), ez = Z - (int)(pj >> 20);
          ex -= (ex > L) ? twoL : 0;
          ex += (ex <= -L) ? twoL : 0;
          ey -= (ey > L) ? twoL : 0;
          ey += (ey <= -L) ? twoL : 0;
          ez -= (ez > L) ? twoL : 0;
          ez += (ez <= -L) ? twoL : 0;
          if (ex * ex + ey * ey + ez * ez <= a.geo.r2max) conf |= 1u << j;
        }
      }
    } else {
      const int z = a.geo.z;
      for (int j = 0; j + 1 < K; ++j) {
        const int sj = __shfl_sync(kFullMask, site, j * G);
        bool hit = false;
        if (j < g) {
          if (sj == site) hit = true;
          for (int s = sub; s < z; s += G)
            if (__ldg(a.geo.tab_nbr + (size_t)s * N + site) == sj) hit = true;
        }
        const uint32_t bal = __ballot_sync(kFullMask, hit);
        if (j < g && (bal & gmask)) conf |= 1u << j;
      }
    }

    // ---------------- phase B: resolve in order ----------------
    uint32_t acc_mask = 0;
    int k = 0;
    for (; k < nvalid; ++k) {
      if (init && (unsigned)(bcur - wlo) < (unsigned)W) {
        done = true;
        break;
      }
      const int src = k * G;
      const uint32_t cm = __shfl_sync(kFullMask, conf, src);
      bool acc;
      if (kTraj) {
        double dE_k = __shfl_sync(kFullMask, (double)dE, src);
        const double u_k = __shfl_sync(kFullMask, u, src);
        if (cm & acc_mask) {
          double dn = 0.0;
          if (g == k) dn = (double)delta_energy<kTraj>(a, off_s, J_s, lat, site, X, Y, Z, nx, ny, nz, sub, G, gmask);
          dE_k = __shfl_sync(kFullMask, dn, src);
          ++n_rec;
        }
        const double Ep = __dadd_rn(E, dE_k);
        if (init) {
          acc = fabs(__dsub_rn(Ep, c_traj)) <= fabs(__dsub_rn(E, c_traj));
          if (acc) {
            E = Ep;
            bcur = bin_fp64(E, a.win);
          }
        } else {
          const int bp = bin_fp64(Ep, a.win);
          const int rel = bp - wlo;
          const bool inw = (unsigned)rel < (unsigned)W;
          acc = false;
          if (inw) {
            const double lngp = (bp == bcur) ? (double)lng_cur : (double)lng_s[rel];
            const double d = __dsub_rn((double)lng_cur, lngp);
            acc = (d >= 0.0) || (u_k < exp_fp64(d, a.ex));
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
        }
      } else {
        long long dq_k = shfl_ll(dq, src);
        const long long lu_k = shfl_ll(lu, src);
        if (cm & acc_mask) {
          long long dn = 0;
          if (g == k) {
            const float dEn = (float)delta_energy<kTraj>(a, off_s, J_s, lat, site, X, Y, Z, nx, ny, nz, sub, G, gmask);
            dn = __double2ll_rn((double)dEn * a.win.dq_scale64);
          }
          dq_k = shfl_ll(dn, src);
          ++n_rec;
        }
        const long long Ep = Efx + dq_k;
        if (init) {
          const long long d0 = Efx - c_fx, d1 = Ep - c_fx;
          acc = (d1 < 0 ? -d1 : d1) <= (d0 < 0 ? -d0 : d0);
          if (acc) {
            Efx = Ep;
            bcur = fx_bin(Efx);
          }
        } else {
          const int bp = fx_bin(Ep);
          const int rel = bp - wlo;
          const bool inw = (unsigned)rel < (unsigned)W;
          long long lngp = (long long)lng_cur;
          if (bp != bcur && inw) lngp = (long long)lng_s[rel];
          const long long d = (long long)lng_cur - lngp;
          acc = inw && (d >= 0 || lu_k < d);
          if (acc) {
            if (bp != bcur) {
              lng_s[bcur - wlo] = lng_cur;
              H_s[bcur - wlo] = h_cur;
              lng_cur = (Lng)lngp;
              h_cur = H_s[rel];
              bcur = bp;
            }
            Efx = Ep;
          }
        }
      }
      if (acc) {
        acc_mask |= 1u << k;
        ++n_acc;
        if (lane == src) put_spin(lat, site, nx, ny, nz, code);
        __syncwarp();
      }
      if (!init && !frozen) {
        if (kTraj)
          lng_cur = (Lng)__dadd_rn((double)lng_cur, lnf);
        else
          lng_cur = (Lng)((long long)lng_cur + lnf_fx);
        ++h_cur;
      }
    }
    t += k;
    remaining -= k;
    __syncwarp();
  }
  if (init && !done && (unsigned)(bcur - wlo) < (unsigned)W) done = true;

  if (lane == 0) {
    if (kTraj) {
      a.st.E[slot] = E;
      a.st.bin[slot] = bcur;
    } else {
      a.st.efx[slot] = Efx;
    }
    if (init) {
      a.st.init_moves[slot] = t;
      if (!done) atomicExch(a.st.ctrl + 0, kErrInitCap);
    } else {
      lng_s[bcur - wlo] = lng_cur;
      H_s[bcur - wlo] = h_cur;
      a.st.steps[slot] = t;
      a.st.accepts[slot] += n_acc;
      a.st.recomputes[slot] += n_rec;
    }
  }
  __syncwarp();
}

template <bool kTraj, bool kSmem>
__global__ void __launch_bounds__(kWalkerThreads) walker_kernel(const WalkerArgs a) {
  using Real = typename Mode<kTraj>::Real;
  using Lng = typename Mode<kTraj>::Lng;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kWalkerThreads / 32];

  const int slot = blockIdx.x;
  const int tid = threadIdx.x;
  const int N = a.geo.N, W = a.win.W;
  const int wlo = a.win.starts[global_slot(a.st, slot) / a.win.m];
  const int rep = a.st.perm[slot];

  Lng* lng_s = reinterpret_cast<Lng*>(smem_raw);
  uint32_t* H_s = reinterpret_cast<uint32_t*>(smem_raw + sizeof(Lng) * (size_t)W);
  uint32_t* off_s = reinterpret_cast<uint32_t*>(smem_raw + sizeof(Lng) * (size_t)W + (((size_t)W * 4 + 15) & ~(size_t)15));
  Real* J_s = reinterpret_cast<Real*>(off_s + kMaxSlotsPerSite);
  Real* spin_s = J_s + kMaxSlotsPerSite;

  const auto glat = GlobalLattice<kTraj>::of(a.st.spins, rep, N);
  typename WalkLattice<kTraj, kSmem>::T lat;
  if constexpr (kSmem)
    lat = typename WalkLattice<kTraj, true>::T(spin_s, N);
  else
    lat = glat;

  // stage tables and lattice
  const size_t lbase = (size_t)slot * W;
  if (!a.init) {
    for (int w = tid; w < W; w += blockDim.x) {
      if (kTraj)
        lng_s[w] = (Lng)a.st.lng[lbase + w];
      else
        lng_s[w] = (Lng)a.st.lng_fx[lbase + w];
      H_s[w] = a.st.H[lbase + w];
    }
  }
  for (int j = tid; j < kMaxSlotsPerSite; j += blockDim.x) {
    off_s[j] = a.geo.off[j];
    J_s[j] = kTraj ? (Real)a.geo.Jd[j] : (Real)a.geo.Jf[j];
  }
  if constexpr (kSmem) copy_lattice(lat, glat, N, tid, blockDim.x);
  __syncthreads();

  if (tid < 32) walk<kTraj>(a, slot, wlo, lng_s, H_s, off_s, J_s, lat);
  __syncthreads();

  if constexpr (kSmem) copy_lattice(glat, lat, N, tid, blockDim.x);
  if (!a.init) {
    for (int w = tid; w < W; w += blockDim.x) {
      if (kTraj)
        a.st.lng[lbase + w] = (double)lng_s[w];
      else
        a.st.lng_fx[lbase + w] = (long long)lng_s[w];
      a.st.H[lbase + w] = H_s[w];
    }
  }
  if (a.recompute && !a.init) {
    const double Ef = full_energy<kTraj>(a, off_s, lat, red, threadIdx.x, blockDim.x, 0);
    if (tid == 0) {
      if (kTraj) {
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

// FP64 energy of every configuration (one CTA each), spins read from global memory.
template <bool kTraj>
__global__ void __launch_bounds__(kWalkerThreads) energies_kernel(const WalkerArgs a, double* out) {
  __shared__ double red[kWalkerThreads / 32];
  __shared__ uint32_t off_s[kMaxSlotsPerSite];
  for (int j = threadIdx.x; j < kMaxSlotsPerSite; j += blockDim.x) off_s[j] = a.geo.off[j];
  __syncthreads();
  const int N = a.geo.N;
  const auto lat = GlobalLattice<kTraj>::of(a.st.spins, blockIdx.x, N);
  const double e = full_energy<kTraj>(a, off_s, lat, red, threadIdx.x, blockDim.x, 0);
  if (threadIdx.x == 0) out[blockIdx.x] = e;
}

cudaError_t launch_energies(const WalkerArgs& a, int n_replicas, bool traj, double* out, cudaStream_t stream) {
  if (traj)
    energies_kernel<true><<<n_replicas, kWalkerThreads, 0, stream>>>(a, out);
  else
    energies_kernel<false><<<n_replicas, kWalkerThreads, 0, stream>>>(a, out);
  return cudaGetLastError();
}

// The neighbour table exactly as the walker kernel computes it: [z][N] indices and couplings.
__global__ void neighbour_dump_kernel(const Geometry g, int32_t* nbr, double* J) {
  const long long total = (long long)g.z * g.N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / g.N), i = (int)(t % g.N);
    if (g.kind == 0) {
      int X, Y, Z, dx, dy, dz;
      bcc_coords(i, g.L, g.divL, X, Y, Z);
      unpack_offset(g.off[j], dx, dy, dz);
      nbr[t] = bcc_offset_site(X, Y, Z, dx, dy, dz, g.L);
      J[t] = g.Jd[j];
    } else {
      nbr[t] = g.tab_nbr[t];
      J[t] = g.tab_Jd[t];
    }
  }
}

cudaError_t launch_neighbour_dump(const Geometry& g, int32_t* nbr, double* J, cudaStream_t stream) {
  neighbour_dump_kernel<<<256, 256, 0, stream>>>(g, nbr, J);
  return cudaGetLastError();
}

size_t walker_smem_bytes(bool traj, bool smem_lattice, int N, int W) {
  const size_t lng = (traj ? sizeof(double) : sizeof(long long)) * (size_t)W;
  const size_t h = ((size_t)W * 4 + 15) & ~(size_t)15;
  const size_t real = traj ? sizeof(double) : sizeof(float);
  size_t bytes = lng + h + 4 * kMaxSlotsPerSite + real * kMaxSlotsPerSite;
  if (smem_lattice) bytes += smem_site_bytes(traj) * (size_t)N;
  return bytes;
}

cudaError_t launch_walkers(const WalkerArgs& a, int n_slots, bool traj, bool smem_lattice, size_t smem,
                           cudaStream_t stream) {
  cudaError_t e = cudaSuccess;
  if (traj && smem_lattice) {
    e = cudaFuncSetAttribute(walker_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) walker_kernel<true, true><<<n_slots, kWalkerThreads, smem, stream>>>(a);
  } else if (traj) {
    e = cudaFuncSetAttribute(walker_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) walker_kernel<true, false><<<n_slots, kWalkerThreads, smem, stream>>>(a);
  } else if (smem_lattice) {
    e = cudaFuncSetAttribute(walker_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) walker_kernel<false, true><<<n_slots, kWalkerThreads, smem, stream>>>(a);
  } else {
    e = cudaFuncSetAttribute(walker_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) walker_kernel<false, false><<<n_slots, kWalkerThreads, smem, stream>>>(a);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace rewl
