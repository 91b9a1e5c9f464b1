/*
 * rewl_oracle.c -- the FP64 single-threaded REWL oracle.  TEST INFRASTRUCTURE ONLY: loaded by the
 * test suite, the smoke entry point and the benchmark's CPU-baseline leg, never by the library.
 *
 * Everything here is written for a reader checking it against the paper:
 *   Sec. 3, Eq. 1    Heisenberg energy on the bcc lattice (N = 2 L^3, two spins per cubic cell)
 *   Sec. 4.2, Eq. 4  Wang-Landau walk, histogram, flatness, f -> sqrt(f)
 *   Sec. 4.3, Eq. 5  energy windows, m walkers per window, replica exchange
 *   Sec. 4.3         joining of fragments where the slopes of ln g coincide
 *   Sec. 4.4         trial move: random spin, uniformly random new direction
 *   Sec. 4.1, Eq. 2-3 partition function, <E>, C_V
 * Points the paper leaves open are fixed by the readings listed in the design notes (window
 * edges, out-of-window moves, initial state, exchange pairing, stitch rule, per-walker ln f).
 *
 * Arithmetic: IEEE FP64, one rounding per operation, no contraction (-ffp-contract=off).
 * Sums whose order matters for bit-exact comparison follow the canonical orders written next to
 * them.  No blocking, fusion or reordering beyond that.
 */
#include "rewl_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------- */
/* Philox4x32-10, Salmon et al. SC'11: 10 rounds of two 32x32->64 multiplications (S-box) and a  */
/* word permutation (P-box); the key is bumped by the Weyl constants between rounds.           */
/* ------------------------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void ro_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform in [0, 1): 27 high bits of a, 26 high bits of b. */
double ro_u53(uint32_t a, uint32_t b) {
  uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
  return (double)m * 0x1.0p-53;
}

/* ------------------------------------------------------------------------------------------- */
/* exp(x): Cody-Waite reduction x = k ln2 + r with ln 2 split into a 29-bit head (so k*head is   */
/* exact for |k| < 2^24) and a tail; exp(r) by its Taylor series to degree 13 (truncation error */
/* < 5e-18 for |r| <= ln2/2), evaluated by Horner; the result is scaled by 2^k.                */
/* The head is ln 2 rounded to a multiple of 2^-32, the tail is ln 2 - head rounded to double. */
/* Defined as 0 below -708 (the result would be subnormal).                                   */
/* ------------------------------------------------------------------------------------------- */
static const double kLn2Head = 0x1.62e42ff000000p-1;
static const double kLn2Tail = -0x1.718432a1b0e26p-35;
static const double kInvLn2 = 0x1.71547652b82fep+0;
static double g_inv_fact[14];
static int g_inv_fact_ready = 0;

static void init_inv_fact(void) {
  if (g_inv_fact_ready) return;
  g_inv_fact[0] = 1.0;
  for (int n = 1; n < 14; ++n) g_inv_fact[n] = g_inv_fact[n - 1] / (double)n;
  g_inv_fact_ready = 1;
}

double ro_exp(double x) {
  init_inv_fact();
  if (x != x) return x;
  if (x < -708.0) return 0.0;
  if (x > 709.0) return INFINITY;
  double kf = floor(x * kInvLn2 + 0.5);
  double r = (x - kf * kLn2Head) - kf * kLn2Tail;
  double p = g_inv_fact[13];
  for (int n = 12; n >= 0; --n) p = p * r + g_inv_fact[n];
  int k = (int)kf;
  /* 2^k for normal k: exponent field k + 1023 */
  uint64_t bits = (uint64_t)(k + 1023) << 52;
  double two_k;
  memcpy(&two_k, &bits, sizeof two_k);
  return p * two_k;
}

/* ------------------------------------------------------------------------------------------- */
/* bcc geometry (Sec. 3).  Positions in half lattice units: a bcc site has all three            */
/* coordinates even (corner sublattice 0) or all odd (body centre, sublattice 1).  Site index   */
/* = 2 (x + L (y + L z)) + s for cell (x, y, z) and sublattice s.  Shell n collects the offsets  */
/* of squared length 3, 4, 8, 11 (quarter a^2 units), i.e. r^2 = 3/4, 1, 2, 11/4 a^2 with 8, 6,  */
/* 12, 24 members.  Canonical slot order: shell by shell, lexicographic (dx, dy, dz) inside.     */
/* ------------------------------------------------------------------------------------------- */
static const int kShellR2[4] = {3, 4, 8, 11};

int ro_bcc_offsets(int n_shells, int32_t* dx, int32_t* dy, int32_t* dz, int32_t* shell) {
  if (n_shells < 1 || n_shells > 4) return -1;
  int z = 0;
  for (int sh = 0; sh < n_shells; ++sh) {
    for (int a = -3; a <= 3; ++a)
      for (int b = -3; b <= 3; ++b)
        for (int c = -3; c <= 3; ++c) {
          int pa = a & 1, pb = b & 1, pc = c & 1;
          if (pa != pb || pb != pc) continue;      /* not a bcc lattice vector */
          if (a * a + b * b + c * c != kShellR2[sh]) continue;
          if (dx) { dx[z] = a; dy[z] = b; dz[z] = c; }
          if (shell) shell[z] = sh;
          ++z;
        }
  }
  return z;
}

static int pmod(int a, int m) {
  int r = a % m;
  return r < 0 ? r + m : r;
}

static int bcc_index(int L, int X, int Y, int Z) {
  /* X, Y, Z half-unit coordinates already reduced to [0, 2L) and of equal parity */
  int s = X & 1;
  int cx = X >> 1, cy = Y >> 1, cz = Z >> 1;
  return 2 * (cx + L * (cy + L * cz)) + s;
}

/* Luttinger-Tisza: E_gs = -(N/2) max_q J(q), J(q) = sum_r J(r) cos(q.r), with q running over a  */
/* grid that contains every wave vector allowed by the periodic box.  In half units            */
/* q.r = pi (n.d) / L for n in [0, 2L)^3.  Exact for a Bravais lattice such as bcc.            */
double ro_bcc_ground_state(int L, int n_shells, const double* J) {
  int32_t dx[64], dy[64], dz[64], sh[64];
  int z = ro_bcc_offsets(n_shells, dx, dy, dz, sh);
  if (z < 0) return NAN;
  const double pi = 3.14159265358979323846;
  double best = -INFINITY;
  for (int n1 = 0; n1 < 2 * L; ++n1)
    for (int n2 = 0; n2 < 2 * L; ++n2)
      for (int n3 = 0; n3 < 2 * L; ++n3) {
        double jq = 0.0;
        for (int j = 0; j < z; ++j) {
          int dot = n1 * dx[j] + n2 * dy[j] + n3 * dz[j];
          jq = jq + J[sh[j]] * cos(pi * (double)dot / (double)L);
        }
        if (jq > best) best = jq;
      }
  double N = 2.0 * (double)L * (double)L * (double)L;
  return -0.5 * N * best;
}

/* ------------------------------------------------------------------------------------------- */
/* Windows (Sec. 4.3): h windows of W bins each over B global bins, adjacent windows overlapping */
/* by the fraction o: B = W (1 + (h - 1)(1 - o)) solved for W and rounded up; window k starts at */
/* bin round(k (B - W) / (h - 1)) (round half up).                                               */
/* ------------------------------------------------------------------------------------------- */
int ro_window_layout(int n_bins, int n_windows, double overlap, int32_t* starts) {
  if (n_bins < 2 || n_windows < 1 || n_windows > n_bins || !(overlap >= 0.0 && overlap < 1.0)) return -1;
  double denom = 1.0 + (double)(n_windows - 1) * (1.0 - overlap);
  int W = (int)ceil((double)n_bins / denom);
  if (W > n_bins) W = n_bins;
  for (int k = 0; k < n_windows; ++k) {
    if (n_windows == 1) {
      starts[k] = 0;
    } else {
      double pos = (double)k * (double)(n_bins - W) / (double)(n_windows - 1);
      starts[k] = (int32_t)floor(pos + 0.5);
    }
  }
  return W;
}

/* Canonical 32-lane reduction: lane l accumulates x[l], x[l+32], x[l+64], ... in index order;  */
/* then lanes combine pairwise with partners l^16, l^8, l^4, l^2, l^1; the result is lane 0.     */
double ro_sum32(const double* x, int n) {
  double p[32], q[32];
  for (int l = 0; l < 32; ++l) {
    p[l] = 0.0;
    for (int i = l; i < n; i += 32) p[l] = p[l] + x[i];
  }
  for (int off = 16; off >= 1; off >>= 1) {
    for (int l = 0; l < 32; ++l) q[l] = p[l] + p[l ^ off];
    memcpy(p, q, sizeof p);
  }
  return p[0];
}

/* ------------------------------------------------------------------------------------------- */
/* Simulation state                                                                             */
/* ------------------------------------------------------------------------------------------- */
struct ro_sim {
  ro_params p;
  int N, z, G;
  int32_t* nbr;    /* [z][N] */
  double* Jt;      /* [z][N] */
  double e_min, e_max, dE;
  int B, h, m, W, S;
  int32_t* starts; /* [h] */
  /* replicas: spins [R][3][N] */
  double* spins;
  /* slots s = k*m + a */
  double* lng;     /* [S][W] */
  uint32_t* H;     /* [S][W] */
  double* E;       /* [S] energy of the replica attached to slot s */
  int32_t* bin;    /* [S] global bin of E */
  int32_t* perm;   /* [S] replica attached to slot s */
  double* lnf;     /* [S] */
  int32_t* stage;  /* [S] number of ln f reductions */
  int64_t* accepts;
  int64_t* steps;
  int64_t* init_moves;
  int32_t* rt_last; /* [S] per replica: extreme window seen last (-1 none, 0 lowest, 1 highest) */
  int64_t* rt_count;/* [S] per replica: round trips completed */
  int64_t* ex_att;  /* [h-1] */
  int64_t* ex_acc;
  int64_t ex_index;
  double max_drift;
  double E0;
  uint32_t key1;
};

static void set_err(char* err, int len, const char* msg) {
  if (err && len > 0) {
    strncpy(err, msg, (size_t)len - 1);
    err[len - 1] = 0;
  }
}

static int bin_of(const ro_sim* s, double E) {
  double q = (E - s->e_min) / s->dE;
  if (q != q) return -(1 << 30);
  if (q < -1073741824.0) q = -1073741824.0;
  if (q > 1073741824.0) q = 1073741824.0;
  return (int)floor(q);
}

static int in_window(const ro_sim* s, int k, int b) {
  return b >= s->starts[k] && b < s->starts[k] + s->W;
}

int ro_create(const ro_params* p, ro_sim** out, char* err, int errlen) {
  *out = NULL;
  init_inv_fact();
  ro_sim* s = (ro_sim*)calloc(1, sizeof(ro_sim));
  if (!s) { set_err(err, errlen, "out of memory"); return -1; }
  s->p = *p;
  s->p.nbr = NULL;
  s->p.Jt = NULL;
  int G = p->group_size;
  if (G != 1 && G != 2 && G != 4 && G != 8 && G != 16 && G != 32) {
    set_err(err, errlen, "group_size must be 1, 2, 4, 8, 16 or 32"); free(s); return -1;
  }
  s->G = G;
  if (p->iteration != 0 && p->iteration != 1) {
    set_err(err, errlen, "iteration must be 0 (per walker) or 1 (per window)"); free(s); return -1;
  }

  /* lattice and neighbour table */
  if (p->kind == RO_BCC) {
    int32_t dx[64], dy[64], dz[64], sh[64];
    int z = ro_bcc_offsets(p->n_shells, dx, dy, dz, sh);
    if (z < 0) { set_err(err, errlen, "n_shells must be 1..4"); free(s); return -1; }
    int maxd = 0;
    for (int j = 0; j < z; ++j) {
      int a = abs(dx[j]), b = abs(dy[j]), c = abs(dz[j]);
      if (a > maxd) maxd = a;
      if (b > maxd) maxd = b;
      if (c > maxd) maxd = c;
    }
    if (p->L < 2 || maxd >= p->L) { set_err(err, errlen, "L too small for the coupling shells"); free(s); return -1; }
    int L = p->L;
    s->N = 2 * L * L * L;
    s->z = z;
    s->nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)z * s->N);
    s->Jt = (double*)malloc(sizeof(double) * (size_t)z * s->N);
    for (int i = 0; i < s->N; ++i) {
      int sub = i & 1, c = i >> 1;
      int cx = c % L, cy = (c / L) % L, cz = c / (L * L);
      int X = 2 * cx + sub, Y = 2 * cy + sub, Z = 2 * cz + sub;
      for (int j = 0; j < z; ++j) {
        int Xn = pmod(X + dx[j], 2 * L), Yn = pmod(Y + dy[j], 2 * L), Zn = pmod(Z + dz[j], 2 * L);
        s->nbr[(size_t)j * s->N + i] = bcc_index(L, Xn, Yn, Zn);
        s->Jt[(size_t)j * s->N + i] = p->J[sh[j]];
      }
    }
  } else if (p->kind == RO_CHAIN) {
    if (p->L < 2) { set_err(err, errlen, "chain needs at least 2 spins"); free(s); return -1; }
    s->N = p->L;
    s->z = 2;
    s->nbr = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)s->N);
    s->Jt = (double*)malloc(sizeof(double) * 2 * (size_t)s->N);
    for (int i = 0; i < s->N; ++i) {
      /* slot 0: left neighbour, slot 1: right neighbour; an open end points at the site itself
         with coupling 0 */
      s->nbr[i] = i > 0 ? i - 1 : i;
      s->Jt[i] = i > 0 ? p->J[0] : 0.0;
      s->nbr[s->N + i] = i + 1 < s->N ? i + 1 : i;
      s->Jt[s->N + i] = i + 1 < s->N ? p->J[0] : 0.0;
    }
  } else if (p->kind == RO_TABLE) {
    if (p->n_sites < 1 || p->z < 1 || !p->nbr || !p->Jt) { set_err(err, errlen, "bad table lattice"); free(s); return -1; }
    s->N = p->n_sites;
    s->z = p->z;
    s->nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)s->z * s->N);
    s->Jt = (double*)malloc(sizeof(double) * (size_t)s->z * s->N);
    memcpy(s->nbr, p->nbr, sizeof(int32_t) * (size_t)s->z * s->N);
    memcpy(s->Jt, p->Jt, sizeof(double) * (size_t)s->z * s->N);
    for (size_t t = 0; t < (size_t)s->z * s->N; ++t)
      if (s->nbr[t] < 0 || s->nbr[t] >= s->N) { set_err(err, errlen, "neighbour index out of range"); ro_destroy(s); return -1; }
  } else {
    set_err(err, errlen, "unknown lattice kind"); free(s); return -1;
  }

  /* energy range */
  double emin = p->e_min, emax = p->e_max;
  if (emin != emin || emax != emax) {
    if (p->kind == RO_BCC) {
      emin = ro_bcc_ground_state(p->L, p->n_shells, p->J);
      emax = 0.0;
    } else if (p->kind == RO_CHAIN) {
      double a = fabs(p->J[0]) * (double)(s->N - 1);
      emin = -a;
      emax = a;
    } else {
      set_err(err, errlen, "table lattices need an explicit energy range"); ro_destroy(s); return -1;
    }
  }
  if (!(emax > emin)) { set_err(err, errlen, "empty energy range"); ro_destroy(s); return -1; }
  s->e_min = emin;
  s->e_max = emax;
  s->B = p->n_bins;
  s->dE = (emax - emin) / (double)s->B;
  s->h = p->n_windows;
  s->m = p->walkers_per_window;
  if (s->m < 1) { set_err(err, errlen, "walkers_per_window must be >= 1"); ro_destroy(s); return -1; }
  if (!(p->flatness > 0.0 && p->flatness < 1.0)) { set_err(err, errlen, "flatness must be in (0,1)"); ro_destroy(s); return -1; }
  if (!(p->lnf_final > 0.0)) { set_err(err, errlen, "lnf_final must be > 0"); ro_destroy(s); return -1; }
  if (p->exchange_interval < 1) { set_err(err, errlen, "exchange_interval must be >= 1"); ro_destroy(s); return -1; }
  s->starts = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->h > 0 ? s->h : 1));
  int W = ro_window_layout(s->B, s->h, p->overlap, s->starts);
  if (W < 2) { set_err(err, errlen, "invalid window layout"); ro_destroy(s); return -1; }
  s->W = W;
  for (int k = 0; k + 1 < s->h; ++k) {
    if (s->starts[k] + W - s->starts[k + 1] < 2) { set_err(err, errlen, "adjacent windows overlap by fewer than 2 bins"); ro_destroy(s); return -1; }
  }
  s->S = s->h * s->m;

  size_t S = (size_t)s->S, N = (size_t)s->N;
  s->spins = (double*)malloc(sizeof(double) * S * 3 * N);
  s->lng = (double*)calloc(S * (size_t)W, sizeof(double));
  s->H = (uint32_t*)calloc(S * (size_t)W, sizeof(uint32_t));
  s->E = (double*)malloc(sizeof(double) * S);
  s->bin = (int32_t*)malloc(sizeof(int32_t) * S);
  s->perm = (int32_t*)malloc(sizeof(int32_t) * S);
  s->lnf = (double*)malloc(sizeof(double) * S);
  s->stage = (int32_t*)calloc(S, sizeof(int32_t));
  s->accepts = (int64_t*)calloc(S, sizeof(int64_t));
  s->steps = (int64_t*)calloc(S, sizeof(int64_t));
  s->init_moves = (int64_t*)calloc(S, sizeof(int64_t));
  s->rt_last = (int32_t*)malloc(sizeof(int32_t) * S);
  s->rt_count = (int64_t*)calloc(S, sizeof(int64_t));
  if (s->rt_last) for (size_t r = 0; r < S; ++r) s->rt_last[r] = -1;
  s->ex_att = (int64_t*)calloc((size_t)(s->h > 1 ? s->h - 1 : 1), sizeof(int64_t));
  s->ex_acc = (int64_t*)calloc((size_t)(s->h > 1 ? s->h - 1 : 1), sizeof(int64_t));
  if (!s->spins || !s->lng || !s->H || !s->E || !s->bin || !s->perm || !s->lnf || !s->rt_last || !s->rt_count) {
    set_err(err, errlen, "out of memory"); ro_destroy(s); return -1;
  }

  /* Initial state (reading: "an arbitrary initial configuration", Sec. 4.2): every replica fully
     aligned along +z.  Its energy is -1/2 sum_i sum_j J_ij, summed site by site in slot order. */
  double acc = 0.0;
  for (int i = 0; i < s->N; ++i) {
    double row = 0.0;
    for (int j = 0; j < s->z; ++j) row = row + s->Jt[(size_t)j * N + i];
    acc = acc + row;
  }
  s->E0 = -0.5 * acc;
  for (size_t r = 0; r < S; ++r) {
    double* sp = s->spins + r * 3 * N;
    for (size_t i = 0; i < N; ++i) {
      sp[i] = 0.0;
      sp[N + i] = 0.0;
      sp[2 * N + i] = 1.0;
    }
    s->E[r] = s->E0;
    s->bin[r] = bin_of(s, s->E0);
    s->perm[r] = (int32_t)r;
    s->lnf[r] = p->lnf_initial > 0.0 ? p->lnf_initial : 1.0; /* f0 = e (Sec. 4.2) */
  }
  s->key1 = (uint32_t)p->seed ^ (uint32_t)(p->seed >> 32);
  s->max_drift = 0.0;
  s->ex_index = 0;
  *out = s;
  return 0;
}

void ro_destroy(ro_sim* s) {
  if (!s) return;
  free(s->nbr); free(s->Jt); free(s->starts); free(s->spins); free(s->lng); free(s->H);
  free(s->E); free(s->bin); free(s->perm); free(s->lnf); free(s->stage); free(s->accepts);
  free(s->steps); free(s->init_moves); free(s->ex_att); free(s->ex_acc); free(s->rt_last); free(s->rt_count);
  free(s);
}

/* ------------------------------------------------------------------------------------------- */
/* Trial move (Sec. 4.4): pick a spin uniformly, give it a direction uniform on the sphere.      */
/* Random words: Philox key (slot, key1); counter (step lo, step hi, purpose, attempt).          */
/*   site  = floor(x0 * N / 2^32) from counter (t, purpose_site, 0)                             */
/*   u     = u53(x1, x2) from the same block (acceptance uniform)                               */
/*   direction: Marsaglia (1972): attempts k = 1, 2, ... with counter (t, purpose_dir, k):      */
/*     a = 2 u53(x0,x1) - 1, b = 2 u53(x2,x3) - 1, s = a^2 + b^2, accepted when 0 < s < 1;      */
/*     S' = (2a sqrt(1-s), 2b sqrt(1-s), 1 - 2s).  After 64 failed attempts S' = (0,0,1).      */
/* Purposes: WL move site 0, WL move direction 1, initial drive 2 (site k = 0, direction k>=1). */
/* ------------------------------------------------------------------------------------------- */
static void draw_direction(uint32_t key0, uint32_t key1, uint64_t t, uint32_t purpose, double S[3]) {
  uint32_t key[2] = {key0, key1};
  for (uint32_t k = 1; k <= 64; ++k) {
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), purpose, k};
    uint32_t x[4];
    ro_philox4x32_10(ctr, key, x);
    double a = 2.0 * ro_u53(x[0], x[1]) - 1.0;
    double b = 2.0 * ro_u53(x[2], x[3]) - 1.0;
    double q = a * a + b * b;
    if (q < 1.0 && q > 0.0) {
      double w = sqrt(1.0 - q);
      S[0] = (2.0 * a) * w;
      S[1] = (2.0 * b) * w;
      S[2] = 1.0 - 2.0 * q;
      return;
    }
  }
  S[0] = 0.0; S[1] = 0.0; S[2] = 1.0;
}

static void draw_site(const ro_sim* s, uint32_t key0, uint64_t t, uint32_t purpose, int* site, double* u) {
  uint32_t key[2] = {key0, s->key1};
  uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), purpose, 0u};
  uint32_t x[4];
  ro_philox4x32_10(ctr, key, x);
  *site = (int)(((uint64_t)x[0] * (uint64_t)s->N) >> 32);
  *u = ro_u53(x[1], x[2]);
}

/* Energy change of S_i -> S' (Eq. 1): dE = -(S' - S_i) . h_i with the local field
   h_i = sum_j J_ij S_j.  Canonical order with group size G: partial l (0 <= l < G) sums slots
   l, l+G, l+2G, ... in order (x, y, z separately); partials combine pairwise with partners
   l^(G/2), ..., l^1; h is partial 0.  dE = -((dx hx + dy hy) + dz hz). */
static double delta_e(const ro_sim* s, const double* sp, int i, const double Sn[3]) {
  const size_t N = (size_t)s->N;
  const double* x = sp;
  const double* y = sp + N;
  const double* zc = sp + 2 * N;
  double px[32], py[32], pz[32];
  int G = s->G;
  for (int l = 0; l < G; ++l) {
    px[l] = 0.0; py[l] = 0.0; pz[l] = 0.0;
    for (int j = l; j < s->z; j += G) {
      int n = s->nbr[(size_t)j * N + i];
      double J = s->Jt[(size_t)j * N + i];
      px[l] = px[l] + J * x[n];
      py[l] = py[l] + J * y[n];
      pz[l] = pz[l] + J * zc[n];
    }
  }
  for (int off = G / 2; off >= 1; off >>= 1) {
    double qx[32], qy[32], qz[32];
    for (int l = 0; l < G; ++l) {
      qx[l] = px[l] + px[l ^ off];
      qy[l] = py[l] + py[l ^ off];
      qz[l] = pz[l] + pz[l ^ off];
    }
    for (int l = 0; l < G; ++l) { px[l] = qx[l]; py[l] = qy[l]; pz[l] = qz[l]; }
  }
  double dx = Sn[0] - x[i];
  double dy = Sn[1] - y[i];
  double dz = Sn[2] - zc[i];
  return -((dx * px[0] + dy * py[0]) + dz * pz[0]);
}

static void set_spin(const ro_sim* s, double* sp, int i, const double Sn[3]) {
  const size_t N = (size_t)s->N;
  sp[i] = Sn[0];
  sp[N + i] = Sn[1];
  sp[2 * N + i] = Sn[2];
}

/* Full energy of one replica: E = -1/2 sum_i sum_j J_ij S_i.S_j (site order, slot order). */
double ro_replica_energy(const ro_sim* s, int r) {
  const size_t N = (size_t)s->N;
  const double* sp = s->spins + (size_t)r * 3 * N;
  double acc = 0.0;
  for (size_t i = 0; i < N; ++i) {
    double row = 0.0;
    for (int j = 0; j < s->z; ++j) {
      int n = s->nbr[(size_t)j * N + i];
      double dot = (sp[i] * sp[n] + sp[N + i] * sp[N + n]) + sp[2 * N + i] * sp[2 * N + n];
      row = row + s->Jt[(size_t)j * N + i] * dot;
    }
    acc = acc + row;
  }
  return -0.5 * acc;
}

/* ------------------------------------------------------------------------------------------- */
/* Initial drive (reading of "arbitrary initial configuration", Sec. 4.2): from the aligned     */
/* state, propose ordinary trial moves (purpose 2) and accept one iff it does not increase      */
/* |E - E_c|, E_c the energy at the centre of the slot's window; no ln g / H updates; stop as   */
/* soon as E lies in the window.                                                                */
/* ------------------------------------------------------------------------------------------- */
int ro_init_walkers(ro_sim* s) {
  const size_t N = (size_t)s->N;
  for (int slot = 0; slot < s->S; ++slot) {
    int k = slot / s->m;
    int r = s->perm[slot];
    double* sp = s->spins + (size_t)r * 3 * N;
    double c = s->e_min + ((double)s->starts[k] + (double)s->W * 0.5) * s->dE;
    double E = s->E[slot];
    int b = s->bin[slot];
    int64_t t = 0;
    while (!in_window(s, k, b)) {
      if (t >= s->p.init_max_moves) return -1;
      int i;
      double u, Sn[3];
      draw_site(s, (uint32_t)slot, (uint64_t)t, 2u, &i, &u);
      draw_direction((uint32_t)slot, s->key1, (uint64_t)t, 2u, Sn);
      double dE = delta_e(s, sp, i, Sn);
      double Ep = E + dE;
      if (fabs(Ep - c) <= fabs(E - c)) {
        E = Ep;
        set_spin(s, sp, i, Sn);
        b = bin_of(s, E);
      }
      ++t;
    }
    s->E[slot] = E;
    s->bin[slot] = b;
    s->init_moves[slot] = t;
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------- */
/* Wang-Landau moves of one slot (Sec. 4.2, Eq. 4).  A trial state outside the slot's window is  */
/* rejected (reading).  Accept A -> B with min[1, g(E_A)/g(E_B)]: d = ln g(E_A) - ln g(E_B);    */
/* accept if d >= 0, else if u < exp(d).  Then, at the resulting state, ln g += ln f and        */
/* H += 1.  A walker whose ln f fell below ln f_final keeps walking with ln g frozen and no     */
/* histogram updates (reading).                                                                 */
/* ------------------------------------------------------------------------------------------- */
static void wl_moves(ro_sim* s, int slot, int64_t n) {
  const size_t N = (size_t)s->N;
  int k = slot / s->m;
  int lo = s->starts[k];
  int r = s->perm[slot];
  double* sp = s->spins + (size_t)r * 3 * N;
  double* lng = s->lng + (size_t)slot * s->W;
  uint32_t* H = s->H + (size_t)slot * s->W;
  double E = s->E[slot];
  int b = s->bin[slot];
  double lnf = s->lnf[slot];
  int frozen = !(lnf >= s->p.lnf_final);
  int64_t t = s->steps[slot];
  int64_t acc_count = s->accepts[slot];
  for (int64_t it = 0; it < n; ++it, ++t) {
    int i;
    double u, Sn[3];
    draw_site(s, (uint32_t)slot, (uint64_t)t, 0u, &i, &u);
    draw_direction((uint32_t)slot, s->key1, (uint64_t)t, 1u, Sn);
    double dE = delta_e(s, sp, i, Sn);
    double Ep = E + dE;
    int bp = bin_of(s, Ep);
    int accept = 0;
    if (in_window(s, k, bp)) {
      double d = lng[b - lo] - lng[bp - lo];
      if (d >= 0.0) accept = 1;
      else accept = u < ro_exp(d);
    }
    if (accept) {
      E = Ep;
      b = bp;
      set_spin(s, sp, i, Sn);
      ++acc_count;
    }
    if (!frozen) {
      lng[b - lo] = lng[b - lo] + lnf;
      H[b - lo] += 1u;
    }
  }
  s->E[slot] = E;
  s->bin[slot] = b;
  s->steps[slot] = t;
  s->accepts[slot] = acc_count;
}

int ro_run_moves_only(ro_sim* s, int64_t moves_per_walker) {
  for (int slot = 0; slot < s->S; ++slot) wl_moves(s, slot, moves_per_walker);
  return 0;
}

/* ------------------------------------------------------------------------------------------- */
/* Replica exchange (Sec. 4.3, Eq. 5).  Round t pairs windows (k, k+1) for k = t mod 2, t mod 2  */
/* + 2, ...; walker a of window k meets walker (a + floor(t/2)) mod m of window k+1.  Slot i of */
/* window k holds configuration A (energy E_A), slot j of window k+1 holds B.  The swap needs    */
/* E_A in window k+1 and E_B in window k; then                                                 */
/*   D = ((ln g_i(E_A) - ln g_i(E_B)) + ln g_j(E_B)) - ln g_j(E_A),                            */
/* accepted if D >= 0 or u < exp(D), u = u53(x0, x1) from Philox key (k, key1 ^ 0x5eed5eed),  */
/* counter (t lo, t hi, 3, a).  On acceptance the slots swap configurations (replica index and  */
/* energy); ln g and H stay with the slots.                                                    */
/* ------------------------------------------------------------------------------------------- */
/* Replica round trips (Sec. 5, Fig. 1): a replica completes one when it is found in the lowest
   window after having been found in the highest.  The replicas of both extreme windows are looked
   at before and after every exchange round (looking twice at the same state changes nothing). */
static void observe_extremes(ro_sim* s) {
  if (s->h < 2) return;
  for (int a = 0; a < s->m; ++a) {
    int r = s->perm[a];
    if (s->rt_last[r] == 1) s->rt_count[r] += 1;
    s->rt_last[r] = 0;
    s->rt_last[s->perm[(s->h - 1) * s->m + a]] = 1;
  }
}

int ro_exchange(ro_sim* s) {
  observe_extremes(s);
  uint64_t t = (uint64_t)s->ex_index;
  int m = s->m;
  int shift = (int)((t / 2u) % (uint64_t)m);
  for (int k = (int)(t & 1u); k + 1 < s->h; k += 2) {
    for (int a = 0; a < m; ++a) {
      int i = k * m + a;
      int j = (k + 1) * m + (a + shift) % m;
      int bA = s->bin[i], bB = s->bin[j];
      s->ex_att[k] += 1;
      if (!in_window(s, k + 1, bA) || !in_window(s, k, bB)) continue;
      const double* Li = s->lng + (size_t)i * s->W;
      const double* Lj = s->lng + (size_t)j * s->W;
      int loi = s->starts[k], loj = s->starts[k + 1];
      double D = ((Li[bA - loi] - Li[bB - loi]) + Lj[bB - loj]) - Lj[bA - loj];
      int accept;
      if (D >= 0.0) {
        accept = 1;
      } else {
        uint32_t key[2] = {(uint32_t)k, s->key1 ^ 0x5eed5eedu};
        uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), 3u, (uint32_t)a};
        uint32_t x[4];
        ro_philox4x32_10(ctr, key, x);
        accept = ro_u53(x[0], x[1]) < ro_exp(D);
      }
      if (accept) {
        int32_t tp = s->perm[i]; s->perm[i] = s->perm[j]; s->perm[j] = tp;
        double te = s->E[i]; s->E[i] = s->E[j]; s->E[j] = te;
        int32_t tb = s->bin[i]; s->bin[i] = s->bin[j]; s->bin[j] = tb;
        s->ex_acc[k] += 1;
      }
    }
  }
  observe_extremes(s);
  s->ex_index += 1;
  return 0;
}

/* ------------------------------------------------------------------------------------------- */
/* Flatness (Sec. 4.2): the histogram of a walker is flat when min_E H(E) >= p * mean_E H(E)     */
/* over all W bins of its window; then ln f -> ln f / 2 (f -> sqrt f) and H -> 0, ln g kept.     */
/* Each walker proceeds independently (Sec. 4.3).                                              */
/* ------------------------------------------------------------------------------------------- */
static int walker_flat(const ro_sim* s, int slot) {
  const uint32_t* H = s->H + (size_t)slot * s->W;
  uint32_t mn = H[0];
  uint64_t sum = 0;
  for (int w = 0; w < s->W; ++w) {
    if (H[w] < mn) mn = H[w];
    sum += H[w];
  }
  double mean = (double)sum / (double)s->W;
  return sum > 0 && (double)mn >= s->p.flatness * mean;
}

/* Window-synchronous reading (the walkers of a window move on together): when every walker of a
   still-active window is flat, each bin's ln g becomes the mean over the window's walkers (summed
   in walker order), then ln f halves and H clears for all of them. */
static int flatness_by_window(ro_sim* s) {
  int halved = 0;
  const int m = s->m;
  for (int k = 0; k < s->h; ++k) {
    const int s0 = k * m;
    if (!(s->lnf[s0] >= s->p.lnf_final)) continue;
    int all = 1;
    for (int a = 0; a < m && all; ++a) all = walker_flat(s, s0 + a);
    if (!all) continue;
    for (int w = 0; w < s->W; ++w) {
      double t = 0.0;
      for (int a = 0; a < m; ++a) t = t + s->lng[(size_t)(s0 + a) * s->W + w];
      const double avg = t / (double)m;
      for (int a = 0; a < m; ++a) s->lng[(size_t)(s0 + a) * s->W + w] = avg;
    }
    for (int a = 0; a < m; ++a) {
      s->lnf[s0 + a] = s->lnf[s0 + a] * 0.5;
      memset(s->H + (size_t)(s0 + a) * s->W, 0, sizeof(uint32_t) * (size_t)s->W);
      s->stage[s0 + a] += 1;
      ++halved;
    }
  }
  return halved;
}

int ro_flatness(ro_sim* s) {
  if (s->p.iteration == 1) return flatness_by_window(s);
  int halved = 0;
  for (int slot = 0; slot < s->S; ++slot) {
    if (!(s->lnf[slot] >= s->p.lnf_final)) continue;
    uint32_t* H = s->H + (size_t)slot * s->W;
    uint32_t mn = H[0];
    uint64_t sum = 0;
    for (int w = 0; w < s->W; ++w) {
      if (H[w] < mn) mn = H[w];
      sum += H[w];
    }
    double mean = (double)sum / (double)s->W;
    if (sum > 0 && (double)mn >= s->p.flatness * mean) {
      s->lnf[slot] = s->lnf[slot] * 0.5;
      memset(H, 0, sizeof(uint32_t) * (size_t)s->W);
      s->stage[slot] += 1;
      ++halved;
    }
  }
  return halved;
}

/* One exchange interval for every walker: WL moves, energy check (the running energy is kept;  */
/* the deviation from a full recomputation is recorded), replica exchange, flatness.            */
int ro_run_intervals(ro_sim* s, int n) {
  for (int it = 0; it < n; ++it) {
    for (int slot = 0; slot < s->S; ++slot) wl_moves(s, slot, s->p.exchange_interval);
    for (int slot = 0; slot < s->S; ++slot) {
      double Ef = ro_replica_energy(s, s->perm[slot]);
      double dr = fabs(Ef - s->E[slot]);
      if (dr > s->max_drift) s->max_drift = dr;
    }
    ro_exchange(s);
    ro_flatness(s);
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------- */
/* Joining the fragments (Sec. 4.3).                                                            */
/*  (1) per window: average of the m walkers' ln g, each taken relative to its own mean          */
/*      (mean by the canonical 32-lane sum): A_k[w] = (sum_a (g_a[w] - mean_a)) / m;           */
/*  (2) per adjacent pair (k, k+1): over the interior of the overlap (global bins b with        */
/*      b-1 and b+1 in both windows) the central differences s(b) = A[b+1] - A[b-1] of both    */
/*      fragments; b* = argmin |s_k(b) - s_{k+1}(b)|, lowest b on ties;                        */
/*  (3) window k+1 is shifted by A_k(b*) - A_{k+1}(b*) (accumulated from window 0); window k    */
/*      supplies bins b*_{k-1} <= b < b*_k;                                                     */
/*  (4) the result has its mean (canonical 32-lane sum over B bins) subtracted.                */
/* ------------------------------------------------------------------------------------------- */
int ro_merge_fragments(const double* frag, const int32_t* starts, int h, int m, int W, int B,
                       double* out, int32_t* bstar_out) {
  double* A = (double*)malloc(sizeof(double) * (size_t)h * W);
  double* mean = (double*)malloc(sizeof(double) * (size_t)m);
  double* shift = (double*)malloc(sizeof(double) * (size_t)h);
  int32_t* bstar = (int32_t*)malloc(sizeof(int32_t) * (size_t)(h > 1 ? h - 1 : 1));
  if (!A || !mean || !shift || !bstar) { free(A); free(mean); free(shift); free(bstar); return -1; }
  for (int k = 0; k < h; ++k) {
    for (int a = 0; a < m; ++a) mean[a] = ro_sum32(frag + ((size_t)k * m + a) * W, W) / (double)W;
    for (int w = 0; w < W; ++w) {
      double t = 0.0;
      for (int a = 0; a < m; ++a) t = t + (frag[((size_t)k * m + a) * W + w] - mean[a]);
      A[(size_t)k * W + w] = t / (double)m;
    }
  }
  int rc = 0;
  for (int k = 0; k + 1 < h; ++k) {
    const double* Ak = A + (size_t)k * W;
    const double* An = A + (size_t)(k + 1) * W;
    int lo = starts[k + 1] + 1;             /* b-1 >= start_{k+1} */
    int hi = starts[k] + W - 2;             /* b+1 <= start_k + W - 1 */
    int best = -1;
    double bestv = INFINITY;
    for (int b = lo; b <= hi; ++b) {
      double sk = Ak[b + 1 - starts[k]] - Ak[b - 1 - starts[k]];
      double sn = An[b + 1 - starts[k + 1]] - An[b - 1 - starts[k + 1]];
      double v = fabs(sk - sn);
      if (v < bestv) { bestv = v; best = b; }
    }
    if (best < 0) { best = starts[k + 1]; rc = -2; }   /* overlap too small: join at its start */
    bstar[k] = best;
  }
  shift[0] = 0.0;
  for (int k = 0; k + 1 < h; ++k) {
    int b = bstar[k];
    shift[k + 1] = shift[k] + (A[(size_t)k * W + (b - starts[k])] - A[(size_t)(k + 1) * W + (b - starts[k + 1])]);
  }
  int k = 0;
  for (int b = 0; b < B; ++b) {
    while (k + 1 < h && b >= bstar[k]) ++k;
    out[b] = A[(size_t)k * W + (b - starts[k])] + shift[k];
  }
  double mu = ro_sum32(out, B) / (double)B;
  for (int b = 0; b < B; ++b) out[b] = out[b] - mu;
  if (bstar_out) memcpy(bstar_out, bstar, sizeof(int32_t) * (size_t)(h > 1 ? h - 1 : 0));
  free(A); free(mean); free(shift); free(bstar);
  return rc;
}

int ro_merge(const ro_sim* s, double* out, double* centres) {
  int rc = ro_merge_fragments(s->lng, s->starts, s->h, s->m, s->W, s->B, out, NULL);
  if (centres)
    for (int b = 0; b < s->B; ++b) centres[b] = s->e_min + ((double)b + 0.5) * s->dE;
  return rc;
}

/* ------------------------------------------------------------------------------------------- */
/* Thermodynamics (Sec. 4.1, Eq. 2-3), k_B = 1: weights w_b = exp(ln g_b - E_b/T - max),         */
/* Z = sum w_b, <E> = sum w_b E_b / Z, var = sum w_b (E_b - <E>)^2 / Z (two-pass),            */
/* C_V = var / T^2, specific heat C_V / N.  ln Z includes the subtracted maximum.              */
/* ------------------------------------------------------------------------------------------- */
void ro_thermo(const double* lng, const double* E, int B, double n_spins, const double* T, int nT,
               double* U, double* C, double* lnZ) {
  double* x = (double*)malloc(sizeof(double) * (size_t)B);
  for (int it = 0; it < nT; ++it) {
    double beta = 1.0 / T[it];
    double mx = -INFINITY;
    for (int b = 0; b < B; ++b) {
      x[b] = lng[b] - E[b] * beta;
      if (x[b] > mx) mx = x[b];
    }
    double z = 0.0, e1 = 0.0;
    for (int b = 0; b < B; ++b) {
      double w = exp(x[b] - mx);
      z += w;
      e1 += w * E[b];
    }
    double u = e1 / z;
    double v = 0.0;
    for (int b = 0; b < B; ++b) {
      double w = exp(x[b] - mx);
      double d = E[b] - u;
      v += w * d * d;
    }
    v /= z;
    if (U) U[it] = u;
    if (C) C[it] = v * beta * beta / n_spins;
    if (lnZ) lnZ[it] = mx + log(z);
  }
  free(x);
}

double ro_peak(const double* T, const double* C, int nT) {
  int best = 0;
  for (int i = 1; i < nT; ++i)
    if (C[i] > C[best]) best = i;
  if (best == 0 || best == nT - 1) return T[best];
  double c0 = C[best - 1], c1 = C[best], c2 = C[best + 1];
  double den = c0 - 2.0 * c1 + c2;
  if (den == 0.0) return T[best];
  double dT = T[best + 1] - T[best];
  return T[best] + 0.5 * dT * (c0 - c2) / den;
}

/* ------------------------------------------------------------------------------------------- */
/* getters                                                                                      */
/* ------------------------------------------------------------------------------------------- */
void ro_sizes(const ro_sim* s, int32_t* N, int32_t* z, int32_t* n_slots, int32_t* W, int32_t* B,
              int32_t* h, int32_t* m) {
  if (N) *N = s->N;
  if (z) *z = s->z;
  if (n_slots) *n_slots = s->S;
  if (W) *W = s->W;
  if (B) *B = s->B;
  if (h) *h = s->h;
  if (m) *m = s->m;
}

void ro_energy_grid(const ro_sim* s, double* e_min, double* e_max, double* dE) {
  if (e_min) *e_min = s->e_min;
  if (e_max) *e_max = s->e_max;
  if (dE) *dE = s->dE;
}

void ro_window_starts(const ro_sim* s, int32_t* starts) { memcpy(starts, s->starts, sizeof(int32_t) * (size_t)s->h); }

void ro_neighbours(const ro_sim* s, int32_t* nbr, double* J) {
  if (nbr) memcpy(nbr, s->nbr, sizeof(int32_t) * (size_t)s->z * s->N);
  if (J) memcpy(J, s->Jt, sizeof(double) * (size_t)s->z * s->N);
}

double ro_initial_energy(const ro_sim* s) { return s->E0; }

void ro_get_walkers(const ro_sim* s, double* lng, uint32_t* H, double* E, int32_t* bin, double* lnf,
                    int32_t* replica, int64_t* accepts, int32_t* stage, int64_t* steps, int64_t* init_moves) {
  size_t S = (size_t)s->S, W = (size_t)s->W;
  if (lng) memcpy(lng, s->lng, sizeof(double) * S * W);
  if (H) memcpy(H, s->H, sizeof(uint32_t) * S * W);
  if (E) memcpy(E, s->E, sizeof(double) * S);
  if (bin) memcpy(bin, s->bin, sizeof(int32_t) * S);
  if (lnf) memcpy(lnf, s->lnf, sizeof(double) * S);
  if (replica) memcpy(replica, s->perm, sizeof(int32_t) * S);
  if (accepts) memcpy(accepts, s->accepts, sizeof(int64_t) * S);
  if (stage) memcpy(stage, s->stage, sizeof(int32_t) * S);
  if (steps) memcpy(steps, s->steps, sizeof(int64_t) * S);
  if (init_moves) memcpy(init_moves, s->init_moves, sizeof(int64_t) * S);
}

void ro_get_spins(const ro_sim* s, double* spins) {
  memcpy(spins, s->spins, sizeof(double) * (size_t)s->S * 3 * s->N);
}

void ro_get_exchange_counts(const ro_sim* s, int64_t* attempts, int64_t* accepts) {
  int n = s->h - 1;
  if (n <= 0) return;
  if (attempts) memcpy(attempts, s->ex_att, sizeof(int64_t) * (size_t)n);
  if (accepts) memcpy(accepts, s->ex_acc, sizeof(int64_t) * (size_t)n);
}

void ro_get_round_trips(const ro_sim* s, int64_t* counts, int32_t* last) {
  if (counts) memcpy(counts, s->rt_count, sizeof(int64_t) * (size_t)s->S);
  if (last) memcpy(last, s->rt_last, sizeof(int32_t) * (size_t)s->S);
}

double ro_max_drift(const ro_sim* s) { return s->max_drift; }
int64_t ro_exchange_index(const ro_sim* s) { return s->ex_index; }

void ro_set_lng(ro_sim* s, const double* lng0, double lnf0) {
  for (int slot = 0; slot < s->S; ++slot) {
    int k = slot / s->m;
    for (int w = 0; w < s->W; ++w) s->lng[(size_t)slot * s->W + w] = lng0[s->starts[k] + w];
    s->lnf[slot] = lnf0;
  }
}

/* ------------------------------------------------------------------------------------------- */
/* test hooks                                                                                   */
/* ------------------------------------------------------------------------------------------- */
void ro_draw_direction(uint32_t slot, uint32_t key1, uint64_t t, uint32_t purpose, double S[3]) {
  draw_direction(slot, key1, t, purpose, S);
}

void ro_draw_site(const ro_sim* s, uint32_t slot, uint64_t t, uint32_t purpose, int32_t* site, double* u) {
  int i;
  draw_site(s, slot, t, purpose, &i, u);
  *site = i;
}

void ro_set_slot(ro_sim* s, int slot, const double* lng, const uint32_t* H, double E) {
  if (lng) memcpy(s->lng + (size_t)slot * s->W, lng, sizeof(double) * (size_t)s->W);
  if (H) memcpy(s->H + (size_t)slot * s->W, H, sizeof(uint32_t) * (size_t)s->W);
  if (E == E) {
    s->E[slot] = E;
    s->bin[slot] = bin_of(s, E);
  }
}
