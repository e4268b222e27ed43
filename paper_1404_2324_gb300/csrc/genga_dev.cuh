// genga_dev.cuh -- device data layout and arithmetic shared by the sm_103a kernels.
//
// FP64 on this part is issued at two lanes per clock per SM (a warp instruction holds its
// sub-partition for 64 cycles, whatever its active mask), and FP64 compares and conversions use
// the same pipe. The helpers below therefore keep every decision that does not need FP64 on the
// integer pipe (comparisons of non-negative doubles by their bit patterns), and seed reciprocal
// and square-root estimates from the single-precision special-function unit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace genga {

typedef unsigned long long u64;

constexpr int TILE = 32;          // bodies per kick tile (one per lane)
constexpr int NMAX = 2048;        // main mode: up to 2048 massive bodies (Sect. 3)
constexpr int BS_LEVELS = 8;      // Bulirsch-Stoer levels, substep sequence n_k = 2k
constexpr int BS_GMAX = 32;       // largest group of the 256-thread BS kernel and the cluster kernel
constexpr int BS_THREADS = 256;
constexpr int BS_HEAVY = 2;      // batched: groups with a member that needed >= 2 BS_HEAVY substeps last time go first
constexpr int BS_SMALL = 4;      // batched: groups of 3 .. BS_SMALL members run on 128-thread CTAs
constexpr int BS_SEQCAP = 256;   // accepted BS substeps one group may record per substep
constexpr int NCOUNTERS = 8;
constexpr int CCAP = 32;          // candidate-list slots per body (more: the bitmap row is scanned)
constexpr double PARK = 1.0e8;    // ghosts are parked this far out (AU) so no pair ever sees them

// status bits (mirrors genga.h)
constexpr int ST_KEPLER_FALLBACK = 1;
constexpr int ST_BS_FAILED = 2;
constexpr int ST_REUSE_FULLKICK = 4;
constexpr int ST_GROUP_TOO_LARGE = 8;
constexpr int ST_UNION_ROUNDS = 16;
constexpr int ST_RECORD_OVERFLOW = 32;  // a recording buffer of the adjoint engine was too small
constexpr int ST_EJECT_OVERFLOW = 64;   // more ejections than EJ_CAP records, or than EJ_STEP in one step
constexpr int ST_GRID_TIMEOUT = 128;    // the grid-wide BS kernel gave up waiting at a grid barrier
constexpr int ST_COLL_OVERFLOW = 256;   // more collision reports than CREC_CAP (later ones dropped)
constexpr int CREC = 24;                // doubles per collision report
constexpr int CREC_CAP = 4096;          // collision reports kept
constexpr int EJ_CAP = 4096;            // ejection records kept (8 doubles each)
constexpr int EJ_STEP = 1024;           // bodies one step can remove in the single-system modes

// counters (mirrors genga_status detail[])
enum { C_STEPS = 0, C_CAND, C_ENC, C_GROUPS, C_BSSTEPS, C_KFALL, C_MERGE, C_FULLKICK };

struct DevParams {
  double G, m0, Gm0, inv_m0, mu2, inv_mu;  // mu = G m0; mu2 = 2 mu
  double n1, n2, pc;
  double bs_eps;
  int bs_kmax, bs_max_halvings, kepler_maxit, kmode, collisions;
  double rcut2, rcut_sun2;  // Sect. 3.2, Ejections: squared limits on |x|; 0: that test is off
  int nmin;                 // batched: a system left with fewer live bodies is stopped; 0: off
};

// Scratch of the grid-wide Bulirsch-Stoer kernel (bs_grid.cu) for one large group at a time; member
// arrays hold up to npad members, chain arrays are [level][member][component].
struct BsGridBuf {
  double *pos;             // [2][BS_LEVELS][npad][3] midpoint positions, double-buffered by round
  double *za, *zb;         // [BS_LEVELS][npad][6] the two newest states of each level's midpoint chain
  double *t1;              // [BS_LEVELS][npad][6] T_{L,1}: level L's modified-midpoint result
  double *prev;            // [npad][6][BS_LEVELS] the newest Neville row of each (member, component)
  double *y;               // [2][npad][6] state at the attempt start / the newest diagonal T_{L,L}
  double *isc;             // [npad][2] 1/|x|, 1/|v| at the attempt start (error scales)
  int *idx, *alive;        // [npad] member -> body, live flag
  double *gm, *m, *R, *A;  // [npad]
  u64 *rcsq;               // [npad]
  u64 *err;                // [2][BS_LEVELS] per-level error maxima, by attempt parity
  unsigned *bar;           // grid barrier: arrivals, generation, abort flag
  int *cont, *ncont;       // contact pairs of an accepted substep (key a * npad + b), their count
};
constexpr int GR_CONTACT_CAP = 4096;

// All per-body arrays are SoA with leading dimension npad (a multiple of 32); vectors are stored
// component-major: x[c * npad + i].
struct Sim {
  int n, npad, nt, W;            // bodies, padded count, tiles, 32-bit words per bitmap row
  double *x, *v, *x0, *v0;       // [3 npad]
  double *m, *gm, *R, *hill;     // [npad]; gm = G m; hill = (m/(3 m0))^(1/3)
  int *alive;                    // [npad]
  double *rc, *A;                // [npad]; A = 1/(0.9 rc)
  u64 *T, *rcsq;                 // [npad]; bits of (pc rc)^2 and rc^2
  double *afar;                  // [3 npad] far-field accelerations of the last kick
  double *part;                  // [nt * nt * 2 * 3 * 32] kick partial sums
  double *pkick, *pfin;          // [nt * 3] per-tile momentum partials
  unsigned *cbm, *rowany;        // candidate bitmap [npad * W], row-nonempty bits [W]
  int *ccnt, *clist;             // per-body candidate count [npad] and partners [npad * CCAP]
  unsigned *ebm;                 // encounter bitmaps [nsub * npad * W] (upper triangle)
  int *edges, *nedges;           // edge list [2 * cap] and its count
  int *fail, *nfail;             // Kepler-fallback bodies [npad] and count
  int *gstart, *gmem, *ngroups;  // groups
  int *big, *nbig;               // groups with gbig or more members (the cluster kernel's work list)
  int *items, nitems, nwarps;    // kick work list
  // batched mode (independent systems; null in the single-system mode)
  int nsys;
  int *sys_of, *sys_start;       // system of each body [npad]; body range of each system [nsys+1]
  double *sys_m0, *sys_ppre, *sys_ppost;  // central masses [nsys], momenta [3 nsys]
  int *sys_flag;                 // per system: opening kick must be recomputed in full
  u64 *bmask, *emask;            // per body: candidate / encounter partners (bit = index in system)
  int *kjobs, nkjobs;            // warp work items of the symmetric kick: [2k] first system, [2k + 1]
                                 // lane-segment width << 8 | systems (width 64: one system of 33..64)
  int *gsize;                    // batched groups: member count per group (gstart = first member)
  int *gtotal;                   // batched groups: members placed so far
  unsigned *bsq;                 // batched groups: next group of queue 0 (1-2 members, pair kernel), queue 1
                                 // (3 .. BS_SMALL members), queue 2 (up to BS_GMAX) and queue 3 (larger)
  int *gorder, *norder;          // batched groups: queue qi is region qi of gorder (npad entries): norder[2 qi]
                                 // groups expected to need many substeps from its front, norder[2 qi + 1]
                                 // from its back
  unsigned char *bsn;            // batched bodies: substeps of the body's last BS group, halved every substep
  // recording of the BS decisions for the adjoint engine (null otherwise): the accepted
  // (H, level) of every substep of group g go to seq_pool[seq_off[g] .. + seq_len[g]]
  double2 *seq_pool;
  int *seq_count, seq_cap;
  int *seq_off, *seq_len;
  // ... and the state after each accepted substep but the last: members x 6 doubles per substep
  // at y_pool[y_off[g] ..], staged in y_scratch [gridDim.x][BS_SEQCAP][BS_GMAX][6] meanwhile
  double *y_pool, *y_scratch;
  long long *y_count, y_cap;
  long long *y_off;
  int *flags;                    // [0] full opening kick needed
  int *status;                   // status bits
  long long *counters;           // [NCOUNTERS]
  double *U;                     // internal energy of mergers and ejections
  double *ejrec;                 // ejection records [EJ_CAP * 8]: index, step, heliocentric x, v
  int *nej;                      // ejections so far (may exceed EJ_CAP: records past it are dropped)
  BsGridBuf gb;                  // grid-wide BS of the largest groups (single-system modes; null otherwise)
  double *spin;                  // spin angular momentum [3 npad] (Sect. 3.2, Collisions; null: not tracked)
  double *crec;                  // collision reports [CREC_CAP * CREC] (null: none kept)
  int *ncrec;                    // mergers so far (may exceed CREC_CAP: reports past it are dropped)
};

// Test particles (massless, perturbed by the massive bodies of a Sim; Sect. 3.3). SoA with
// leading dimension npad; planet quantities are indexed by the planet's body index (< 32).
struct TPSet {
  int n, npad;
  double *x, *v, *x0, *v0;       // [3 npad]
  double *R, *rc, *A, *afar;     // [npad] (afar [3 npad])
  u64 *T, *rcsq;                 // [npad]
  int *alive, *full, *fail;      // [npad]
  unsigned *cmask, *emask;       // candidate / encountered planets per TP
  int *bslist, *nbs;             // TPs that need Bulirsch-Stoer this substep: nbs[0] from the front of
                                 // bslist (deep encounters), nbs[1] from its back (the rest)
  unsigned *bsnext;              // [0] next list entry a BS warp takes, [1] next block of closing kicks,
                                 // [2] encounter blocks done, [3] BS-pass warps done, [4 + 4 b + q]
                                 // warps of BS-pass block b on sub-partition q done with their BS entries
  unsigned *pairs, *npairs;      // candidate (TP, planet) pairs of the last closing kick: i * 32 + j
  double *ptab;                  // planets' Kepler paths at the BS midpoint times [TP_MAXPL * TP_TAB * 6]
  double *ppoly;                 // planets' paths over the substep, polynomials in s = 2t/tau - 1 [TP_MAXPL * 6 * TP_CHEB]
  int *pcok;                     // 1: planet j's series is exact to rounding; 0: solve Kepler instead
  long long *counters;           // candidates, encounters, BS steps, removed, ejected
};
constexpr int TP_MAXPL = 32;     // planets in test-particle mode
constexpr int TP_BS_MAXBLOCKS = 1024;  // blocks of the TP BS pass (one per SM)
constexpr int TP_TAB = 80;       // sum over BS levels k = 1..8 of the 2k + 1 midpoint times
constexpr int TP_CHEB = 16;      // Chebyshev nodes per planet path

// ---------------------------------------------------------------------------------------------
// Integer-pipe helpers
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ u64 dbits(double x) { return (u64)__double_as_longlong(x); }
__device__ __forceinline__ u64 absbits(double x) { return dbits(x) & 0x7fffffffffffffffULL; }
__device__ __forceinline__ u64 umax64(u64 a, u64 b) { return a > b ? a : b; }
__device__ __forceinline__ u64 umin64(u64 a, u64 b) { return a < b ? a : b; }
// max/min of non-negative doubles through their bit patterns
__device__ __forceinline__ double pmax(double a, double b) { return __longlong_as_double((long long)umax64(dbits(a), dbits(b))); }
__device__ __forceinline__ double pmin(double a, double b) { return __longlong_as_double((long long)umin64(dbits(a), dbits(b))); }
__device__ __forceinline__ bool is_neg_or_zero(double x) { return (long long)dbits(x) <= 0 || (dbits(x) >> 63); }

// double -> float by truncating the significand with integer operations (|x| must lie within the
// normal float range), and the exact float -> double widening, both off the FP64 pipe.
__device__ __forceinline__ float d2f_trunc(double x) {
  u64 b = dbits(x);
  unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  unsigned sgn = hi & 0x80000000u;
  unsigned fb = (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
  return __uint_as_float(fb | sgn);
}
// Checked variant for any finite or infinite double: flushes |x| < 2^-126 to a signed zero and
// saturates |x| >= 2^128 to a signed infinity.
__device__ __forceinline__ float d2f_safe(double x) {
  u64 b = dbits(x);
  unsigned hi = (unsigned)(b >> 32);
  unsigned sgn = hi & 0x80000000u;
  unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex < 897u) return __uint_as_float(sgn);
  if (ex > 1150u) return __uint_as_float(sgn | 0x7f800000u);
  return d2f_trunc(x);
}
__device__ __forceinline__ double f2d_exact(float f) {
  unsigned fb = __float_as_uint(f);
  unsigned sgn = fb & 0x80000000u, mag = fb & 0x7fffffffu;
  unsigned hi = ((mag >> 3) + (896u << 20)) | sgn;
  unsigned lo = mag << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// ---------------------------------------------------------------------------------------------
// Refined reciprocal and inverse square roots (Householder iterations of order 3, i.e. the
// Taylor series of (1 - e)^p in the residual e of a single-precision seed). The seed has a
// relative error below 2^-21, so the truncated series leaves ~1e-19 and the result is within
// about one ulp. Valid for positive normal arguments inside the float exponent range.
// The seeds are the single-instruction approximations of the PTX ISA (rsqrt.approx.ftz.f32,
// rcp.approx.ftz.f32: relative error about 2^-23); the refinement supplies the accuracy.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float rsqrt_seed(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_seed(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double rsqrt_refined(double x) {  // x^(-1/2): 5 FP64 operations
  double y = f2d_exact(rsqrt_seed(d2f_trunc(x)));
  double e = fma(-x, y * y, 1.0);   // y*y is exact (24-bit significand squared)
  double p = fma(e, 0.375, 0.5);
  return fma(y * e, p, y);
}
__device__ __forceinline__ double rcube_refined(double x) {  // x^(-3/2): 6 FP64 operations
  double y = f2d_exact(rsqrt_seed(d2f_trunc(x)));
  double y2 = y * y;
  double e = fma(-x, y2, 1.0);
  double y3 = y2 * y;
  double p = fma(e, 1.875, 1.5);
  return fma(y3, e * p, y3);
}
__device__ __forceinline__ double rcp_refined(double x) {  // 1/x, either sign: 3 FP64 operations
  double y = f2d_exact(rcp_seed(d2f_trunc(x)));
  double e = fma(-x, y, 1.0);
  double t = fma(e, e, e);
  return fma(y, t, y);
}

// ---------------------------------------------------------------------------------------------
// Row Lc of the Neville tableau of the Bulirsch-Stoer extrapolation (polynomial in h^2, Sect. 3.2):
// T_{Lc,1} = t1, T_{Lc,j+1} = T_{Lc,j} + (T_{Lc,j} - T_{Lc-1,j}) fac(j), with the previous row in
// prev[] (overwritten by this one). The loops are unrolled with a uniform exit, so both rows stay
// in registers. Returns T_{Lc,Lc}; *before receives T_{Lc,Lc-1} (Lc >= 2).
// ---------------------------------------------------------------------------------------------
template <class Fac>
__device__ __forceinline__ double neville_row(double t1, int Lc, Fac fac, double (&prev)[BS_LEVELS], double &before) {
  double cur[BS_LEVELS];
  cur[0] = t1;
  double last = t1;
  before = 0.0;
#pragma unroll
  for (int j = 1; j < BS_LEVELS; ++j) {
    if (j >= Lc) break;
    cur[j] = fma(cur[j - 1] - prev[j - 1], fac(j), cur[j - 1]);
    before = last;
    last = cur[j];
  }
#pragma unroll
  for (int j = 0; j < BS_LEVELS; ++j) {
    if (j >= Lc) break;
    prev[j] = cur[j];
  }
  return last;
}

// ---------------------------------------------------------------------------------------------
// Changeover weights (Sect. 2.1). For a pair inside its critical radius, y = r A - 1/9 with
// A = 1/(0.9 rc). W_B is the weight of the Newtonian pair force in the kick, W_A = 1 - W_B the
// weight in the Bulirsch-Stoer part. kmode 0: W_B = K; kmode 1: W_B = K - r dK/dr.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void changeover_w(double r, double A, int kmode, double &wB, double &wA) {
  double y = fma(r, A, -1.0 / 9.0);
  if (is_neg_or_zero(y)) { wB = 0.0; wA = 1.0; return; }
  if (dbits(y) >= dbits(1.0)) { wB = 1.0; wA = 0.0; return; }
  double omy = 1.0 - y;
  double y2 = y * y, o2 = omy * omy;
  double iD = rcp_refined(y2 + o2);  // 1/(2y^2 - 2y + 1)
  wB = y2 * iD;
  wA = o2 * iD;
  if (kmode == 1) {  // r K' = (y + 1/9) 2 y (1 - y) / D^2
    double t = (y + 1.0 / 9.0) * (2.0 * y * omy) * (iD * iD);
    wB -= t;
    wA += t;
  }
}

// W_A = 1 - W_B of a pair at distance r, A = 1/(0.9 rc), without branches: y is clamped to [0, 1]
// on the integer pipe, where the formula itself gives exactly 1 (y = 0) and 0 (y = 1), so the value
// equals the branched changeover_w everywhere.
__device__ __forceinline__ double changeover_wA_clamped(double r, double A, int kmode) {
  double y = fma(r, A, -1.0 / 9.0);
  y = is_neg_or_zero(y) ? 0.0 : (dbits(y) >= dbits(1.0) ? 1.0 : y);
  const double omy = 1.0 - y, y2 = y * y, o2 = omy * omy;
  const double iD = rcp_refined(y2 + o2);  // 1/(2y^2 - 2y + 1)
  double wA = o2 * iD;
  if (kmode == 1) wA += (y + 1.0 / 9.0) * (2.0 * y * omy) * (iD * iD);
  return wA;
}

// ---------------------------------------------------------------------------------------------
// Canonical decision quantities, evaluated exactly as the CPU oracle does (no contraction):
// |d|^2 = fma(dz, dz, fma(dy, dy, dx*dx)), a.b likewise.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double r2_exact(double dx, double dy, double dz) {
  return __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
}
__device__ __forceinline__ double dot_exact(double ax, double ay, double az, double bx, double by, double bz) {
  return __fma_rn(az, bz, __fma_rn(ay, by, __dmul_rn(ax, bx)));
}

__device__ __forceinline__ double hermite_eval_exact(double t, double tau, double P0, double P1, double Pd0, double Pd1) {
  double s = __dsub_rn(1.0, t);
  double ss = __dmul_rn(s, s), tt = __dmul_rn(t, t);
  double h00 = __dmul_rn(ss, __dadd_rn(1.0, __dmul_rn(2.0, t)));
  double h01 = __dmul_rn(tt, __dsub_rn(3.0, __dmul_rn(2.0, t)));
  double h10 = __dmul_rn(__dmul_rn(t, ss), tau);
  double h11 = __dmul_rn(__dmul_rn(tt, s), tau);
  return __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(h00, P0), __dmul_rn(h01, P1)), __dmul_rn(h10, Pd0)), __dmul_rn(h11, Pd1));
}

// Minimum over t in [0, 1] of the cubic Hermite interpolant of the squared separation
// (Sect. 2.2, Eqs. teqn and polydelta): P(0), P(1) from the relative positions before and after
// a drift of length tau, dP/dt = 2 dx.dv, dP/d(t) = a t^2 + b t + c with
// a = 6(P0 - P1) + 3 tau (Pd0 + Pd1), b = 6(P1 - P0) - 2 tau (2 Pd0 + Pd1), c = tau Pd0.
// Operation order matches the CPU oracle so that decisions are bit-identical.
static __device__ double hermite_min_exact(double dx0, double dy0, double dz0, double dvx0, double dvy0, double dvz0,
                                    double dx1, double dy1, double dz1, double dvx1, double dvy1, double dvz1,
                                    double tau) {
  double P0 = r2_exact(dx0, dy0, dz0);
  double P1 = r2_exact(dx1, dy1, dz1);
  double Pd0 = __dmul_rn(2.0, dot_exact(dx0, dy0, dz0, dvx0, dvy0, dvz0));
  double Pd1 = __dmul_rn(2.0, dot_exact(dx1, dy1, dz1, dvx1, dvy1, dvz1));
  double a = __dadd_rn(__dmul_rn(6.0, __dsub_rn(P0, P1)), __dmul_rn(__dmul_rn(3.0, tau), __dadd_rn(Pd0, Pd1)));
  double b = __dsub_rn(__dmul_rn(6.0, __dsub_rn(P1, P0)), __dmul_rn(__dmul_rn(2.0, tau), __dadd_rn(__dmul_rn(2.0, Pd0), Pd1)));
  double c = __dmul_rn(tau, Pd0);
  double dmin = P0 < P1 ? P0 : P1;
  double disc = __dsub_rn(__dmul_rn(b, b), __dmul_rn(__dmul_rn(4.0, a), c));
  if (disc >= 0.0) {
    double sq = __dsqrt_rn(disc);
    double q = __dmul_rn(-0.5, __dadd_rn(b, copysign(sq, b)));
    if (a != 0.0) {
      double t = __ddiv_rn(q, a);
      if (t > 0.0 && t < 1.0) {
        double d = hermite_eval_exact(t, tau, P0, P1, Pd0, Pd1);
        if (d < dmin) dmin = d;
      }
    }
    if (q != 0.0) {
      double t = __ddiv_rn(c, q);
      if (t > 0.0 && t < 1.0) {
        double d = hermite_eval_exact(t, tau, P0, P1, Pd0, Pd1);
        if (d < dmin) dmin = d;
      }
    }
  }
  return dmin;
}

// hermite_min_exact where the minimum can fall below thr, else +infinity: the same decision for
// every test "minimum < thr" at a fraction of the cost when the pair stays far apart. Over t in
// [0, 1] the interpolant is h00 P0 + h01 P1 + tau (h10 Pd0 + h11 Pd1) with h00 + h01 = 1, h00, h01 >= 0
// and |h10|, |h11| <= 4/27, so it is at least min(P0, P1) - (4/27) |tau| (|Pd0| + |Pd1|). A bound that
// clears thr by 1e-12 of the terms' size (thousands of times the rounding of either evaluation)
// proves that the full minimum, rounding included, is not below thr; NaN takes the full path.
static __device__ double hermite_min_capped(double dx0, double dy0, double dz0, double dvx0, double dvy0, double dvz0,
                                            double dx1, double dy1, double dz1, double dvx1, double dvy1, double dvz1,
                                            double tau, double thr) {
  const double P0 = r2_exact(dx0, dy0, dz0);
  const double P1 = r2_exact(dx1, dy1, dz1);
  const double Pd0 = __dmul_rn(2.0, dot_exact(dx0, dy0, dz0, dvx0, dvy0, dvz0));
  const double Pd1 = __dmul_rn(2.0, dot_exact(dx1, dy1, dz1, dvx1, dvy1, dvz1));
  const double spread = (4.0 / 27.0) * fabs(tau) * (fabs(Pd0) + fabs(Pd1));
  const double lb = (P0 < P1 ? P0 : P1) - spread;
  if (lb - 1e-12 * (P0 + P1 + spread) > thr) return __longlong_as_double(0x7ff0000000000000LL);
  return hermite_min_exact(dx0, dy0, dz0, dvx0, dvy0, dvz0, dx1, dy1, dz1, dvx1, dvy1, dvz1, tau);
}

// ---------------------------------------------------------------------------------------------
// Stumpff functions (Danby 1988): c_k(z), reduced by quartering z until |z| <= 0.1, Taylor series
// of c2 and c3, then the quadrupling identities c0(4z) = 2c0^2 - 1, c1(4z) = c0 c1,
// c2(4z) = c1^2/2, c3(4z) = (c2 + c0 c3)/4.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void stumpff_f(float z, float &c0, float &c1, float &c2, float &c3) {
  int nred = 0;
  while (fabsf(z) > 0.1f && nred < 40) { z *= 0.25f; nred++; }
  c2 = fmaf(fmaf(fmaf(z, -1.0f / 3628800.0f, 1.0f / 40320.0f), -z, 1.0f / 720.0f), z, -1.0f / 24.0f);
  c2 = fmaf(c2, z, 0.5f);
  c3 = fmaf(fmaf(fmaf(z, -1.0f / 39916800.0f, 1.0f / 362880.0f), -z, 1.0f / 5040.0f), z, -1.0f / 120.0f);
  c3 = fmaf(c3, z, 1.0f / 6.0f);
  c1 = fmaf(-z, c3, 1.0f);
  c0 = fmaf(-z, c2, 1.0f);
  for (; nred > 0; nred--) {
    c3 = fmaf(c0, c3, c2) * 0.25f;
    c2 = 0.5f * c1 * c1;
    c1 = c0 * c1;
    c0 = fmaf(2.0f * c0, c0, -1.0f);
  }
}

__device__ __forceinline__ void stumpff_d(double z, double &c0, double &c1, double &c2, double &c3) {
  int nred = 0;
  float zf = fabsf(d2f_safe(z));
  while (zf > 0.1f && nred < 64) { zf *= 0.25f; nred++; }
  if (nred) z = z * __hiloint2double((1023 - 2 * nred) << 20, 0);  // exact 4^-nred
  // c2 = sum_k (-z)^k/(2k+2)!, c3 = sum_k (-z)^k/(2k+3)!, k = 0..6 (|z| <= 0.1: truncation < 1e-20)
  c2 = fma(z, 1.0 / 87178291200.0, -1.0 / 479001600.0);
  c2 = fma(c2, z, 1.0 / 3628800.0);
  c2 = fma(c2, z, -1.0 / 40320.0);
  c2 = fma(c2, z, 1.0 / 720.0);
  c2 = fma(c2, z, -1.0 / 24.0);
  c2 = fma(c2, z, 0.5);
  c3 = fma(z, 1.0 / 1307674368000.0, -1.0 / 6227020800.0);
  c3 = fma(c3, z, 1.0 / 39916800.0);
  c3 = fma(c3, z, -1.0 / 362880.0);
  c3 = fma(c3, z, 1.0 / 5040.0);
  c3 = fma(c3, z, -1.0 / 120.0);
  c3 = fma(c3, z, 1.0 / 6.0);
  c1 = fma(-z, c3, 1.0);
  c0 = fma(-z, c2, 1.0);
  for (; nred > 0; nred--) {
    c3 = fma(c0, c3, c2) * 0.25;
    c2 = (0.5 * c1) * c1;
    c1 = c0 * c1;
    c0 = fma(2.0 * c0, c0, -1.0);
  }
}

// Kepler drift about mu for dt with Gauss' f and g functions in universal variables (Eq. fg).
// The universal Kepler equation F(s) = r0 s c1 + u s^2 c2 + mu s^3 c3 - dt = 0 (z = beta s^2,
// beta = 2 mu/r0 - v^2, u = x.v) is first solved in single precision, then refined in double
// precision with one Halley step and Newton steps until |ds| <= 4 ulp |s| or a tiny step stops
// shrinking (rounding floor). Returns 0 on success, 1 when no convergence (state untouched).
static __device__ int kepler_drift_dev(double mu, double mu2, double &x, double &y, double &z, double &vx,
                                double &vy, double &vz, double dt, int maxit, int *iters_out,
                                double *s_out = nullptr) {
  double r0sq = fma(z, z, fma(y, y, x * x));
  double ir0 = rsqrt_refined(r0sq);
  double r0 = r0sq * ir0;
  double v2 = fma(vz, vz, fma(vy, vy, vx * vx));
  double u = fma(z, vz, fma(y, vy, x * vx));
  double beta = fma(mu2, ir0, -v2);
  // single-precision pre-solve
  float fr0 = d2f_safe(r0), fmu = d2f_safe(mu), fdt = d2f_safe(dt), fu = d2f_safe(u), fb = d2f_safe(beta);
  float s = fdt / fr0;
  bool fok = false;
  for (int it = 0; it < 12; ++it) {
    float c0, c1, c2, c3;
    stumpff_f(fb * s * s, c0, c1, c2, c3);
    float s2 = s * s;
    float F = fmaf(fr0 * s, c1, fmaf(fu * s2, c2, fmaf(fmu * s2 * s, c3, -fdt)));
    float Fp = fmaf(fr0, c0, fmaf(fu * s, c1, fmu * s2 * c2));
    float ds = F / Fp;
    s -= ds;
    if (!(fabsf(s) < 3.0e38f)) break;
    if (fabsf(ds) <= 2.0e-6f * fabsf(s)) { fok = true; break; }
  }
  double sd = (fok && s != 0.0f) ? f2d_exact(s) : dt * ir0;
  // double-precision refinement: one Halley step from the float root, then Newton
  double c0, c1, c2, c3;
  double s_eval = sd;
  float ds_prev = 3.0e38f;
  int ok = 0, it;
  bool halley = fok;
  for (it = 1; it <= maxit; ++it) {
    stumpff_d(beta * sd * sd, c0, c1, c2, c3);
    double s2 = sd * sd;
    double mus2 = mu * s2;
    double F = fma(r0 * sd, c1, fma(u * s2, c2, fma(mus2 * sd, c3, -dt)));
    double Fp = fma(r0, c0, fma(u * sd, c1, mus2 * c2));
    double ds;
    if (halley) {  // ds = 2 F F' / (2 F'^2 - F F''), F'' = (mu - beta r0) s c1 + u c0
      double Fpp = fma(fma(-beta, r0, mu) * sd, c1, u * c0);
      ds = (2.0 * F * Fp) * rcp_refined(fma(2.0 * Fp, Fp, -F * Fpp));
      halley = false;
    } else {
      ds = F * rcp_refined(Fp);
    }
    s_eval = sd;
    double snew = sd - ds;
    if (((dbits(snew) >> 52) & 0x7ffu) == 0x7ffu) break;  // not finite
    if (absbits(ds) <= absbits(8.881784197001252e-16 * snew)) { ok = 1; break; }  // |ds| <= 4 ulp |s|
    float fa = fabsf(d2f_safe(ds)), fs = fabsf(d2f_safe(snew));
    if (fa <= 1e-10f * fs && fa >= 0.5f * ds_prev) { ok = 1; break; }  // rounding floor reached
    ds_prev = fa;
    sd = snew;
  }
  if (iters_out) *iters_out = it;
  if (!ok) return 1;
  if (s_out) *s_out = s_eval;
  // f, g and their derivatives at s_eval (the last point where the c_k were evaluated)
  double s2 = s_eval * s_eval;
  double mus2 = mu * s2;
  double r = fma(r0, c0, fma(u * s_eval, c1, mus2 * c2));
  double ir = rcp_refined(r);
  double f = fma(-(mu * ir0) * s2, c2, 1.0);
  double g = fma(-mus2 * s_eval, c3, dt);
  double fd = -(mu * s_eval) * c1 * ir * ir0;
  double gd = fma(-mus2 * c2, ir, 1.0);
  double xn = fma(f, x, g * vx), yn = fma(f, y, g * vy), zn = fma(f, z, g * vz);
  double vxn = fma(fd, x, gd * vx), vyn = fma(fd, y, gd * vy), vzn = fma(fd, z, gd * vz);
  x = xn; y = yn; z = zn;
  vx = vxn; vy = vyn; vz = vzn;
  return 0;
}

// ---------------------------------------------------------------------------------------------
// Merger bookkeeping of the BS kernels (Sect. 3.2, Collisions), called by the one thread that applies
// a merger of bodies ia < ib, before the survivor's state is replaced: the report of both bodies'
// positions, velocities and spins at the last time before the contact (ya, yb: the start of the BS
// substep in which it was found, t its time within the composition substep), then the survivor's
// spin from angular-momentum conservation: both spins plus mu (x_b - x_a) x (v_b - v_a) of the
// states yna, ynb after the substep, mu = m_a m_b / (m_a + m_b); the ghost's spin is cleared.
// Report layout: step (1-based), substep, t, ia, ib, x_a, v_a, spin_a, x_b, v_b, spin_b, survivor.
// step_no, substep < 0: the values the step graph keeps in the counters and flags.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void merger_report(const Sim &S, int ia, int ib, const double *ya, const double *yb,
                                              const double *yna, const double *ynb, double ma, double mb,
                                              bool keep_a, double t, int step_no = -1, int substep = -1) {
  const int np = S.npad;
  if (S.crec) {
    const int slot = atomicAdd(S.ncrec, 1);
    if (slot < CREC_CAP) {
      double *r = S.crec + (size_t)slot * CREC;
      r[0] = step_no >= 0 ? (double)step_no : (double)*(volatile long long *)&S.counters[C_STEPS];
      r[1] = substep >= 0 ? (double)substep : (double)*(volatile int *)&S.flags[2];
      r[2] = t;
      r[3] = (double)ia;
      r[4] = (double)ib;
      for (int c = 0; c < 3; ++c) {
        r[5 + c] = ya[c]; r[8 + c] = ya[3 + c]; r[11 + c] = S.spin ? S.spin[c * np + ia] : 0.0;
        r[14 + c] = yb[c]; r[17 + c] = yb[3 + c]; r[20 + c] = S.spin ? S.spin[c * np + ib] : 0.0;
      }
      r[23] = (double)(keep_a ? ia : ib);
    } else {
      atomicOr(S.status, ST_COLL_OVERFLOW);
    }
  }
  if (S.spin) {
    const double mu = ma * mb / (ma + mb);
    const double dx = ynb[0] - yna[0], dy = ynb[1] - yna[1], dz = ynb[2] - yna[2];
    const double dvx = ynb[3] - yna[3], dvy = ynb[4] - yna[4], dvz = ynb[5] - yna[5];
    const double L[3] = {mu * (dy * dvz - dz * dvy), mu * (dz * dvx - dx * dvz), mu * (dx * dvy - dy * dvx)};
    const int sv = keep_a ? ia : ib, dd = keep_a ? ib : ia;
    double nsp[3];
    for (int c = 0; c < 3; ++c) nsp[c] = S.spin[c * np + ia] + S.spin[c * np + ib] + L[c];
    for (int c = 0; c < 3; ++c) { S.spin[c * np + sv] = nsp[c]; S.spin[c * np + dd] = 0.0; }
  }
}

// Largest v over the warp into *dst (shared memory; one atomic per warp instead of one per thread,
// which serialised on the single address). All 32 lanes call it; v = 0 adds nothing.
__device__ __forceinline__ void warp_max_to(u64 *dst, u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const u64 t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  if ((threadIdx.x & 31) == 0 && v) atomicMax((unsigned long long *)dst, (unsigned long long)v);
}

// Warp reductions (butterfly), fixed order -> deterministic
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace genga
