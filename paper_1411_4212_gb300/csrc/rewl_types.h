// rewl_types.h -- plain structs passed by value to the REWL kernels (host and device side).
#pragma once

#include <cstdint>

namespace rewl {

constexpr int kMaxSlotsPerSite = 64;   // neighbour slots z
constexpr int kWalkerThreads = 128;    // threads per walker CTA (warp 0 walks; all load/store)

struct ExpCoeffs {
  double inv_fact[14];                 // 1/n!, n = 0..13, each c[n] = c[n-1] / n in IEEE FP64
};

struct Geometry {
  int kind;                            // 0 bcc (arithmetic neighbours), 1 table
  int N, z, L;
  uint32_t divL;                       // ceil(2^32 / L) for bcc
  int r2max;                           // bcc: largest squared half-unit offset of the shells
  uint32_t off[kMaxSlotsPerSite];      // bcc: packed offsets and shell (see unpack_offset)
  float Jf[kMaxSlotsPerSite];          // bcc: coupling per slot
  double Jd[kMaxSlotsPerSite];
  int n_shells;                        // bcc: 1..4
  float Jsh_f[4];                      // bcc: coupling per shell
  double Jsh_d[4];
  int n_energy_slots;                  // slots summed by the energy recomputation
  float energy_weight;                 // 1 (bcc, forward half of every shell) or 0.5 (table, all)
  uint8_t energy_slot[kMaxSlotsPerSite];
  const int32_t* tab_nbr;              // table: [z][N]
  const float* tab_Jf;                 // table: [z][N]
  const double* tab_Jd;                // table: [z][N]
};

struct Windows {
  int B, h, m, W;
  const int32_t* starts;               // [h]
  double e_min, dE;                    // bin b covers [e_min + b dE, e_min + (b+1) dE)
  float dq_scale;                      // 2^32 / dE (FP32 copy, unused by the walk)
  double dq_scale64;                   // 2^32 / dE: production energy increment dq = rint(dE * scale)
  float dq24_hi, dq24_lo;              // 2^24 / dE split into two floats (hi + lo, ~48 bits)
};

struct WalkerState {
  void* spins;                         // [R][N] float2 octahedral codes (production) or [R][3][N] double (trajectory)
  int32_t* perm;                       // [S] configuration held by slot s
  uint32_t* H;                         // [S][W]
  long long* lng_fx;                   // production [S][W], 2^-40 units
  long long* efx;                      // production [S], 2^-32 bins above e_min
  long long* lnf_fx;                   // production [S]
  double* lng;                         // trajectory [S][W]
  double* E;                           // trajectory [S]
  int32_t* bin;                        // trajectory [S]
  double* lnf;                         // [S] (production keeps it equal to lnf_fx * 2^-40)
  int32_t* stage;                      // [S]
  long long* steps;                    // [S] Wang-Landau trial moves done
  long long* accepts;                  // [S]
  long long* recomputes;               // [S]
  long long* path_batches;             // [S][3] production pipelined walker: batches resolved by the
                                       // warp scan, 8-move blocks, one move at a time
  long long* init_moves;               // [S]
  double* drift;                       // [S] largest |running E - recomputed E|
  int32_t* ctrl;                       // [0] error code, [1] halved counter, [2] done counter
  long long* ex_index;                 // replica-exchange rounds done (device counter)
  int32_t* rt_last;                    // [S] per configuration: extreme window seen last (-1, 0 lowest, 1 highest)
  long long* rt_count;                 // [S] per configuration: round trips completed
  unsigned long long* ex_att;          // [h-1]
  unsigned long long* ex_acc;          // [h-1]
  // partitioned simulations (one handle per GPU, together one REWL run): the handle's S positions
  // host global slots; a configuration stays at its position, slot states move between handles
  const int32_t* gid;                  // [S] global slot hosted at each position (Philox key, window);
                                       // null: position = global slot
  const int32_t* pos_of;               // [S_global] position hosting a global slot, -1 elsewhere
  int S_global;                        // slots of the whole run (h m); S for a plain handle
};

// Global slot (window k = slot / m, walker a = slot % m) hosted at position p.
__host__ __device__ __forceinline__ int global_slot(const WalkerState& st, int p) { return st.gid ? st.gid[p] : p; }

struct WalkerArgs {
  Geometry geo;
  Windows win;
  WalkerState st;
  ExpCoeffs ex;
  long long moves;                     // trial moves per walker in this launch
  long long init_cap;                  // cap of the initial drive
  uint32_t key1;                       // seed_lo ^ seed_hi
  int G;                               // lanes per trial move
  int init;                            // 1: initial drive into the windows
  int recompute;                       // 1: energy recomputation at the end of the launch
  int own_mask;                        // pipelined walker: owner-table size - 1 (power of two)
  int smem_lattice;                    // batched pipelined walker: 1 = lattice copied into shared memory
  int resolver;                        // production pipelined walker: 0 per-batch choice, 1 scan,
                                       // 2 blocks, 3 one move at a time (same decisions)
  double lnf_final;
};

// error codes written to ctrl[0]
enum : int32_t { kErrNone = 0, kErrInitCap = 1, kErrOutOfWindow = 2 };

}  // namespace rewl
