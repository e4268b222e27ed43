// adjoint.cu -- differentiable engine: B independent systems of N bodies each advanced by the hybrid
// step (Sect. 2.2-2.3, perfect merging off), and the hand-written reverse-mode derivative (adjoint)
// of the whole step with every discrete decision frozen from the forward pass: the branch of K, the
// candidate and encounter pairs, the groups, each group's accepted Bulirsch-Stoer sequence and the
// Kepler solves. The paper has no adjoint; this is its step, differentiated.
//
// Layout: body g = b * Np + i of system b (Np = N rounded up to 32), SoA component-major with
// leading dimension NB = B * Np. Padding bodies are not alive and sit far out.
//
// Forward of one substep of signed length tau, h = tau/2 (Eq. z1):
//   v1 = v + h a(x)                     opening kick (K-weighted, critical radii of the step)
//   x1 = x + h P(v1)/m0                 Sun drift
//   (x2, v2) = Kepler(x1, v1; tau)      or, for the members of an encounter group, BS of H_A
//   x3 = x2 + h P(v2)/m0                Sun drift
//   v3 = v2 + h a(x3)                   closing kick (+ prechecker for the next substep)
// The reverse pass runs the same chain backwards with vector-Jacobian products (VJPs). Long runs
// keep a checkpoint every K steps; the backward pass recomputes one K-step segment at a time from
// its checkpoint, recording the intermediate states and decisions, then differentiates it.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/genga.h"
#include "genga_launch.h"

namespace genga {

constexpr int AD_MAXN = 1024;  // bodies per system

// Neville weights: T_kk = sum_l c_lambda[k][l] T_l1 for the sequence n_l = 2l
__constant__ double c_lambda[BS_LEVELS + 1][BS_LEVELS + 1];

struct AdjDev {
  int B, N, Np, NB;
  double G, dt;
  const double *m0;       // [B]
  int *cand, *ccount;     // candidate pairs (i << 16 | j) per system [B * cap], counts [B]
  int ccap;
  double *P;              // per-system momentum [3 B]
  int *fail;              // Kepler non-convergence flag [NB]
  int *ingrp;             // member of an encounter group in the substep being differentiated [NB]
  double *xb, *vb, *mb, *rcb;  // adjoints [3 NB], [3 NB], [NB], [NB]
};

// Records of one substep (each [3 NB] except s [NB]); null when not recording.
struct SubRec {
  double *x, *v1, *x1, *v2, *x3, *s;
  int *gstart, *gsize, *gmem, *ngroups, *seq_off, *seq_len;
  long long *y_off;
};

__device__ __forceinline__ int sys_of_body(const AdjDev &D, int g) { return g / D.Np; }

// ---------------------------------------------------------------------------------------------
// Setup and conversion
// ---------------------------------------------------------------------------------------------
// AoS user input [B][N][3] (heliocentric) -> SoA democratic state; masses, G m, Hill factor.
__global__ void k_ad_setup(Sim S, AdjDev D, const double *xh, const double *vh, const double *m) {
  __shared__ double red[4][128];
  const int b = blockIdx.x, tid = threadIdx.x, NB = D.NB;
  const double m0 = D.m0[b];
  double pm[3] = {0.0, 0.0, 0.0}, msum = 0.0;
  for (int i = tid; i < D.N; i += blockDim.x) {
    const double mi = m[b * D.N + i];
    msum += mi;
    for (int c = 0; c < 3; ++c) pm[c] = fma(mi, vh[(b * D.N + i) * 3 + c], pm[c]);
  }
  red[0][tid] = pm[0]; red[1][tid] = pm[1]; red[2][tid] = pm[2]; red[3][tid] = msum;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (tid < o)
      for (int c = 0; c < 4; ++c) red[c][tid] += red[c][tid + o];
    __syncthreads();
  }
  const double M = m0 + red[3][0];
  const double vcm[3] = {red[0][0] / M, red[1][0] / M, red[2][0] / M};
  for (int i = tid; i < D.Np; i += blockDim.x) {
    const int g = b * D.Np + i;
    if (i < D.N) {
      const double mi = m[b * D.N + i];
      for (int c = 0; c < 3; ++c) {
        S.x[c * NB + g] = xh[(b * D.N + i) * 3 + c];
        S.v[c * NB + g] = vh[(b * D.N + i) * 3 + c] - vcm[c];
      }
      S.m[g] = mi; S.gm[g] = D.G * mi; S.hill[g] = cbrt(mi / (3.0 * m0)); S.alive[g] = 1;
    } else {
      S.x[g] = PARK + 1.0e4 * g; S.x[NB + g] = 0.0; S.x[2 * NB + g] = 0.0;
      for (int c = 0; c < 3; ++c) S.v[c * NB + g] = 0.0;
      S.m[g] = 0.0; S.gm[g] = 0.0; S.hill[g] = 0.0; S.alive[g] = 0;
    }
    S.R[g] = 0.0;
    D.fail[g] = 0;
  }
}

// SoA democratic state -> AoS heliocentric output: v_h = v_b + P/m0.
__global__ void k_ad_output(Sim S, AdjDev D, double *xh, double *vh) {
  __shared__ double red[3][128];
  const int b = blockIdx.x, tid = threadIdx.x, NB = D.NB;
  double pm[3] = {0.0, 0.0, 0.0};
  for (int i = tid; i < D.N; i += blockDim.x) {
    const int g = b * D.Np + i;
    for (int c = 0; c < 3; ++c) pm[c] = fma(S.m[g], S.v[c * NB + g], pm[c]);
  }
  for (int c = 0; c < 3; ++c) red[c][tid] = pm[c];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (tid < o)
      for (int c = 0; c < 3; ++c) red[c][tid] += red[c][tid + o];
    __syncthreads();
  }
  const double im0 = 1.0 / D.m0[b];
  for (int i = tid; i < D.N; i += blockDim.x) {
    const int g = b * D.Np + i;
    for (int c = 0; c < 3; ++c) {
      xh[(b * D.N + i) * 3 + c] = S.x[c * NB + g];
      vh[(b * D.N + i) * 3 + c] = fma(red[c][0], im0, S.v[c * NB + g]);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Critical radii (Eq. rcrit), per system central mass. With rc_in set, the radii are taken from
// it (restart from a checkpoint) and only the derived quantities are filled in.
// ---------------------------------------------------------------------------------------------
__global__ void k_ad_rcrit(Sim S, AdjDev D, DevParams P, double tau_abs, const double *rc_in, double *rec_rc,
                           double *rec_v) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= D.NB) return;
  const int NB = D.NB;
  if (rec_v) for (int c = 0; c < 3; ++c) rec_v[c * NB + g] = S.v[c * NB + g];
  if (!S.alive[g]) { S.rc[g] = 0.0; S.A[g] = 0.0; S.T[g] = 0ULL; S.rcsq[g] = 0ULL; if (rec_rc) rec_rc[g] = 0.0; return; }
  double rc;
  if (rc_in) {
    rc = rc_in[g];
  } else {
    const double inv_mu = 1.0 / (D.G * D.m0[sys_of_body(D, g)]);
    const double x = S.x[g], y = S.x[NB + g], z = S.x[2 * NB + g];
    const double vx = S.v[g], vy = S.v[NB + g], vz = S.v[2 * NB + g];
    const double r2 = fma(z, z, fma(y, y, x * x));
    const double ir = rsqrt_refined(r2);
    const double v2 = fma(vz, vz, fma(vy, vy, vx * vx));
    const double inva = fma(2.0, ir, -v2 * inv_mu);
    const double asemi = is_neg_or_zero(inva) ? r2 * ir : rcp_refined(inva);
    const double rh = asemi * S.hill[g];
    const double vabs = (dbits(v2) == 0ULL) ? 0.0 : v2 * rsqrt_refined(v2);
    rc = pmax(P.n1 * rh, (P.n2 * tau_abs) * vabs);
  }
  S.rc[g] = rc;
  if (rec_rc) rec_rc[g] = rc;
  const double t = __dmul_rn(P.pc, rc);
  S.T[g] = dbits(__dmul_rn(t, t));
  S.rcsq[g] = dbits(__dmul_rn(rc, rc));
  S.A[g] = (dbits(rc) == 0ULL) ? 0.0 : rcp_refined(0.9 * rc);
}

// ---------------------------------------------------------------------------------------------
// Kick (Eq. Hb weighted by K), every unordered pair once (Newton's third law): one warp per pair of
// 32-body tiles (I <= J) of one system; lane l holds body I*32 + l, the bodies of tile J and their
// accumulators rotate through the lanes by warp shuffles. Partial sums per (tile, partner tile)
// are added by k_ad_kick_fin in a fixed order (deterministic).
// MODE 0: opening kick; 1: closing kick + prechecker; 2: prechecker only (no sums).
// ---------------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(128) k_ad_kick_sym(Sim S, AdjDev D, double *part) {
  const int T = D.Np >> 5, npair = T * (T + 1) / 2, NB = D.NB;
  const int lane = threadIdx.x & 31;
  const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (item >= D.B * npair) return;  // uniform within the warp
  const int b = item / npair;
  int k = item % npair, I = 0;
  while (k >= T - I) { k -= T - I; ++I; }
  const int J = I + k;
  const int base = b * D.Np;
  const int gi = base + I * 32 + lane;
  const double xi = S.x[gi], yi = S.x[NB + gi], zi = S.x[2 * NB + gi], gmi = S.gm[gi], Ai = S.A[gi];
  const u64 Ti = S.T[gi], Qi = S.rcsq[gi];
  const bool ali = S.alive[gi] != 0;
  const int gj0 = base + J * 32 + lane;
  double xj = S.x[gj0], yj = S.x[NB + gj0], zj = S.x[2 * NB + gj0], gmj = S.gm[gj0], Aj = S.A[gj0];
  u64 Tj = S.T[gj0], Qj = S.rcsq[gj0];
  int alj = S.alive[gj0];
  double aix = 0.0, aiy = 0.0, aiz = 0.0, ajx = 0.0, ajy = 0.0, ajz = 0.0;
  const int src = (lane + 1) & 31;
  const bool diag = I == J;
  auto rotate = [&]() {
    xj = __shfl_sync(0xffffffffu, xj, src); yj = __shfl_sync(0xffffffffu, yj, src);
    zj = __shfl_sync(0xffffffffu, zj, src); gmj = __shfl_sync(0xffffffffu, gmj, src);
    Aj = __shfl_sync(0xffffffffu, Aj, src); Tj = __shfl_sync(0xffffffffu, Tj, src);
    Qj = __shfl_sync(0xffffffffu, Qj, src); alj = __shfl_sync(0xffffffffu, alj, src);
    ajx = __shfl_sync(0xffffffffu, ajx, src); ajy = __shfl_sync(0xffffffffu, ajy, src);
    ajz = __shfl_sync(0xffffffffu, ajz, src);
  };
  const int nsteps = diag ? 16 : 32;
  for (int st = 0; st < nsteps; ++st) {
    if (diag) rotate();  // diagonal tile: lane l meets l + st + 1
    const int jl = diag ? ((lane + st + 1) & 31) : ((lane + st) & 31);
    const bool act = (!diag || st < 15 || lane < 16) && ali && alj;
    const double dx = xj - xi, dy = yj - yi, dz = zj - zi;
    const double r2 = r2_exact(dx, dy, dz);
    const u64 rb = dbits(r2);
    if (MODE >= 1 && act && rb < umax64(Ti, Tj)) {
      const int i = I * 32 + lane, j = J * 32 + jl;
      const int lo = i < j ? i : j, hi = i < j ? j : i;
      const int kk = atomicAdd(&D.ccount[b], 1);
      if (kk < D.ccap) D.cand[(size_t)b * D.ccap + kk] = (lo << 16) | hi;
      else atomicOr(S.status, ST_RECORD_OVERFLOW);
    }
    if (MODE != 2) {
      const double yr = rsqrt_refined(r2);
      double w3 = act ? yr * yr * yr : 0.0;
      if (act && rb < umax64(Qi, Qj)) {
        double wB, wA;
        changeover_w(r2 * yr, pmin(Ai, Aj), 0, wB, wA);
        w3 *= wB;
      }
      const double fi = gmj * w3, fj = gmi * w3;
      aix = fma(fi, dx, aix); aiy = fma(fi, dy, aiy); aiz = fma(fi, dz, aiz);
      ajx = fma(-fj, dx, ajx); ajy = fma(-fj, dy, ajy); ajz = fma(-fj, dz, ajz);
    }
    if (!diag) rotate();  // after 32 rotations every j value and sum is back on its owning lane
  }
  if (MODE == 2) return;
  double *pb = part + (size_t)b * T * T * 96;
  if (diag) {  // the j sums return to the lane that owns body I*32 + lane
    const int home = (lane + 16) & 31;
    ajx = __shfl_sync(0xffffffffu, ajx, home);
    ajy = __shfl_sync(0xffffffffu, ajy, home);
    ajz = __shfl_sync(0xffffffffu, ajz, home);
    double *p = pb + ((size_t)I * T + I) * 96 + lane;
    p[0] = aix + ajx; p[32] = aiy + ajy; p[64] = aiz + ajz;
  } else {
    double *p = pb + ((size_t)I * T + J) * 96 + lane;
    p[0] = aix; p[32] = aiy; p[64] = aiz;
    double *q = pb + ((size_t)J * T + I) * 96 + lane;
    q[0] = ajx; q[32] = ajy; q[64] = ajz;
  }
}

// v += h a with a the sum of body g's tile partials over the partner tiles in ascending order;
// records the positions the kick saw when asked.
__global__ void k_ad_kick_fin(Sim S, AdjDev D, double h, const double *part, double *rec_x) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= D.NB || !S.alive[g]) return;
  const int NB = D.NB, T = D.Np >> 5, b = g / D.Np, i = g % D.Np, I = i >> 5, lane = i & 31;
  const double *p = part + ((size_t)b * T * T + (size_t)I * T) * 96 + lane;
  for (int c = 0; c < 3; ++c) {
    double a = 0.0;
    for (int J = 0; J < T; ++J) a += p[(size_t)J * 96 + 32 * c];
    S.v[c * NB + g] = fma(h, a, S.v[c * NB + g]);
    if (rec_x) rec_x[c * NB + g] = S.x[c * NB + g];
  }
}

// Per-system momentum P = sum m v (fixed-order tree) and the Sun drift x += (h/m0) P.
// Records v (the velocities the drift saw) and the drifted x when asked.
__global__ void __launch_bounds__(256) k_ad_sundrift(Sim S, AdjDev D, double h, double *rec_v, double *rec_x) {
  __shared__ double red[3][256];
  const int b = blockIdx.x, tid = threadIdx.x, NB = D.NB;
  double pm[3] = {0.0, 0.0, 0.0};
  for (int i = tid; i < D.Np; i += 256) {
    const int g = b * D.Np + i;
    if (!S.alive[g]) continue;
    for (int c = 0; c < 3; ++c) pm[c] = fma(S.m[g], S.v[c * NB + g], pm[c]);
  }
  for (int c = 0; c < 3; ++c) red[c][tid] = pm[c];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o)
      for (int c = 0; c < 3; ++c) red[c][tid] += red[c][tid + o];
    __syncthreads();
  }
  const double f = h / D.m0[b];
  for (int i = tid; i < D.Np; i += 256) {
    const int g = b * D.Np + i;
    if (rec_v) for (int c = 0; c < 3; ++c) rec_v[c * NB + g] = S.v[c * NB + g];
    if (S.alive[g])
      for (int c = 0; c < 3; ++c) S.x[c * NB + g] = fma(f, red[c][0], S.x[c * NB + g]);
    if (rec_x) for (int c = 0; c < 3; ++c) rec_x[c * NB + g] = S.x[c * NB + g];
  }
}

// Keep the pre-drift state, Kepler drift (Eq. fg) about G m0 of the body's system.
__global__ void k_ad_kepler(Sim S, AdjDev D, DevParams P, double tau, double *rec_s) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= D.NB) return;
  const int NB = D.NB;
  D.fail[g] = 0;
  double x = S.x[g], y = S.x[NB + g], z = S.x[2 * NB + g];
  double vx = S.v[g], vy = S.v[NB + g], vz = S.v[2 * NB + g];
  S.x0[g] = x; S.x0[NB + g] = y; S.x0[2 * NB + g] = z;
  S.v0[g] = vx; S.v0[NB + g] = vy; S.v0[2 * NB + g] = vz;
  if (!S.alive[g]) return;
  const double mu = D.G * D.m0[sys_of_body(D, g)];
  double s = 0.0;
  if (kepler_drift_dev(mu, 2.0 * mu, x, y, z, vx, vy, vz, tau, P.kepler_maxit, nullptr, &s)) {
    D.fail[g] = 1;
    atomicOr(S.status, ST_KEPLER_FALLBACK);
  }
  if (rec_s) rec_s[g] = s;
  S.x[g] = x; S.x[NB + g] = y; S.x[2 * NB + g] = z;
  S.v[g] = vx; S.v[NB + g] = vy; S.v[2 * NB + g] = vz;
}

// Encounter search and grouping of one system per CTA: the Hermite test (Eqs. teqn, polydelta)
// on the candidates of the last prechecker, union-find, then groups of >= 2 members (and every
// body whose Kepler solve failed, alone) in ascending member order, appended to the group list.
// Everything the serial parts touch is staged in shared memory first.
__global__ void __launch_bounds__(256) k_ad_group(Sim S, AdjDev D, double tau) {
  __shared__ int par[AD_MAXN];
  __shared__ int root[AD_MAXN];
  __shared__ unsigned char fl[AD_MAXN];
  __shared__ int edges[2 * 1024];
  __shared__ int ne;
  const int b = blockIdx.x, tid = threadIdx.x, Np = D.Np, NB = D.NB, base = b * Np;
  const int nc = min(D.ccount[b], D.ccap);
  if (tid == 0) ne = 0;
  int anyfail = 0;
  for (int i = tid; i < Np; i += blockDim.x) {
    par[i] = i;
    fl[i] = (unsigned char)(i < D.N && D.fail[base + i]);
    anyfail |= fl[i];
  }
  __syncthreads();
  for (int k = tid; k < nc; k += blockDim.x) {
    const int pr = D.cand[(size_t)b * D.ccap + k];
    const int i = pr >> 16, j = pr & 0xffff, gi = base + i, gj = base + j;
    const double rcij = pmax(S.rc[gi], S.rc[gj]);
    const double thr = __dmul_rn(rcij, rcij);
    const double dmin = hermite_min_capped(
        __dsub_rn(S.x0[gj], S.x0[gi]), __dsub_rn(S.x0[NB + gj], S.x0[NB + gi]), __dsub_rn(S.x0[2 * NB + gj], S.x0[2 * NB + gi]),
        __dsub_rn(S.v0[gj], S.v0[gi]), __dsub_rn(S.v0[NB + gj], S.v0[NB + gi]), __dsub_rn(S.v0[2 * NB + gj], S.v0[2 * NB + gi]),
        __dsub_rn(S.x[gj], S.x[gi]), __dsub_rn(S.x[NB + gj], S.x[NB + gi]), __dsub_rn(S.x[2 * NB + gj], S.x[2 * NB + gi]),
        __dsub_rn(S.v[gj], S.v[gi]), __dsub_rn(S.v[NB + gj], S.v[NB + gi]), __dsub_rn(S.v[2 * NB + gj], S.v[2 * NB + gi]), tau, thr);
    if (dmin < thr) {
      const int e = atomicAdd(&ne, 1);
      if (e < 1024) { edges[2 * e] = i; edges[2 * e + 1] = j; }
    }
  }
  anyfail = __syncthreads_or(anyfail);
  if (tid == 0) D.ccount[b] = 0;  // consumed; the closing kick refills it
  if (ne == 0 && !anyfail) return;  // uniform: nothing to integrate by BS in this system
  if (tid == 0) {
    if (ne > 1024) { atomicOr(S.status, ST_RECORD_OVERFLOW); ne = 1024; }
    for (int e = 0; e < ne; ++e) {  // union by smaller root
      int a = edges[2 * e], c = edges[2 * e + 1];
      while (par[a] != a) a = par[a];
      while (par[c] != c) c = par[c];
      if (a != c) { if (a < c) par[c] = a; else par[a] = c; }
    }
  }
  __syncthreads();
  for (int i = tid; i < Np; i += blockDim.x) {
    int r = i;
    while (par[r] != r) r = par[r];
    root[i] = r;  // group id = smallest member
  }
  __syncthreads();
  for (int i = tid; i < Np; i += blockDim.x) par[i] = 0;
  __syncthreads();
  for (int i = tid; i < D.N; i += blockDim.x) atomicAdd(&par[root[i]], 1);  // sizes by root
  __syncthreads();
  if (tid == 0) {  // groups (size >= 2, or a failed Kepler solve alone), ascending root and member
    int g = 0, m = 0;
    for (int i = 0; i < D.N; ++i)
      if (root[i] == i && (par[i] >= 2 || fl[i])) { g++; m += par[i]; }
    const int gbase = g ? atomicAdd(S.ngroups, g) : 0;
    const int mbase = m ? atomicAdd(S.gtotal, m) : 0;
    int gk = gbase, pos = mbase;
    for (int i = 0; i < D.N; ++i) {  // first pass: starts; par[] becomes the fill cursor
      if (root[i] == i && (par[i] >= 2 || fl[i])) {
        S.gstart[gk] = pos;
        S.gsize[gk] = par[i];
        gk++;
        const int sz = par[i];
        par[i] = -(pos + 1);  // negative: start position of this root's group
        pos += sz;
      } else if (root[i] == i) {
        par[i] = 0;
      }
    }
    for (int i = 0; i < D.N; ++i) {  // second pass: members in ascending order
      const int r = root[i];
      if (par[r] < 0) {
        const int at = -par[r] - 1;
        S.gmem[at] = base + i;
        par[r] = -(at + 2);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// VJPs
// ---------------------------------------------------------------------------------------------
// Changeover K(y) and dK/dy for kmode 0 (the force weight W = K).
__device__ __forceinline__ void k_and_dk(double r, double A, double &K, double &dK) {
  const double y = fma(r, A, -1.0 / 9.0);
  if (is_neg_or_zero(y)) { K = 0.0; dK = 0.0; return; }
  if (dbits(y) >= dbits(1.0)) { K = 1.0; dK = 0.0; return; }
  const double omy = 1.0 - y, y2 = y * y, o2 = omy * omy, Dn = y2 + o2;
  K = y2 / Dn;
  dK = 2.0 * y * omy / (Dn * Dn);
}

// Adjoint of one pair term of an acceleration field: the pair (i, j) adds m_j g(d) to a_i and
// -m_i g(d) to a_j, g(d) = G W(r) d/r^3, d = x_j - x_i, W = K (kick, SIGN = +1) or 1 - K (BS,
// SIGN = -1, only inside rc). Given u_i, u_j (adjoints of a_i, a_j), returns the contribution to
// xbar_i (xbar_j gets the negative), to mbar_i (from a_j), and to rcbar of the pair.
template <int SIGN>
__device__ __forceinline__ void pair_vjp(double dx, double dy, double dz, double gmi, double gmj, double G,
                                         const double *ui, const double *uj, double Apair, double rcpair,
                                         bool inside, double *xb, double &mb, double &rcb) {
  const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  const double yr = rsqrt_refined(r2), yr2 = yr * yr, yr3 = yr2 * yr;
  double W, Wr = 0.0, Wrc = 0.0;
  if (inside) {
    const double r = r2 * yr;
    double K, dK;
    k_and_dk(r, Apair, K, dK);
    if (SIGN > 0) { W = K; Wr = dK * Apair; Wrc = -dK * (r * Apair) / rcpair; }
    else { W = 1.0 - K; Wr = -dK * Apair; Wrc = dK * (r * Apair) / rcpair; }
  } else {
    W = SIGN > 0 ? 1.0 : 0.0;
  }
  if (dbits(W) == 0ULL && dbits(Wr) == 0ULL) return;
  const double w0 = gmj * ui[0] - gmi * uj[0], w1 = gmj * ui[1] - gmi * uj[1], w2 = gmj * ui[2] - gmi * uj[2];
  const double dw = fma(dz, w2, fma(dy, w1, dx * w0));
  const double c1 = W * yr3, c2 = dw * (Wr * yr2 * yr2 - 3.0 * W * yr3 * yr2);
  xb[0] -= fma(c1, w0, c2 * dx); xb[1] -= fma(c1, w1, c2 * dy); xb[2] -= fma(c1, w2, c2 * dz);
  mb -= G * c1 * fma(dz, uj[2], fma(dy, uj[1], dx * uj[0]));
  rcb += Wrc * yr3 * dw;
}

// Both sides of one changeover-zone pair of the kick (weight W = K): Jw (xbar_i -= Jw, xbar_j += Jw),
// the mbar contributions of i (from a_j) and of j (from a_i), and the pair's rcbar.
__device__ __forceinline__ void pair_vjp_zone(double dx, double dy, double dz, double gmi, double gmj, double G,
                                              const double *ui, const double *uj, double Apair, double rcpair,
                                              double *Jw, double &mbi, double &mbj, double &rcbp) {
  const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  const double yr = rsqrt_refined(r2), yr2 = yr * yr, yr3 = yr2 * yr;
  const double r = r2 * yr;
  double K, dK;
  k_and_dk(r, Apair, K, dK);
  const double W = K, Wr = dK * Apair, Wrc = -dK * (r * Apair) / rcpair;
  const double w0 = gmj * ui[0] - gmi * uj[0], w1 = gmj * ui[1] - gmi * uj[1], w2 = gmj * ui[2] - gmi * uj[2];
  const double dw = fma(dz, w2, fma(dy, w1, dx * w0));
  const double c1 = W * yr3, c2 = dw * (Wr * yr2 * yr2 - 3.0 * W * yr3 * yr2);
  Jw[0] = fma(c1, w0, c2 * dx); Jw[1] = fma(c1, w1, c2 * dy); Jw[2] = fma(c1, w2, c2 * dz);
  mbi = -G * c1 * fma(dz, uj[2], fma(dy, uj[1], dx * uj[0]));
  mbj = G * c1 * fma(dz, ui[2], fma(dy, ui[1], dx * ui[0]));
  rcbp = Wrc * yr3 * dw;
}

// Kick VJP, Newton's third law: every unordered pair once, on 32x32 tile pairs of one system with a
// warp-shuffle ring (lane l holds body i = I*32 + l, the j data and j-side sums rotate), as in the
// forward kick. Outside the changeover zone a body's sums are S1 = sum Gm_p/r^3, V = sum u_p/r^3,
// Wd = 3 sum (d.w)/r^5 d (d pointing from the body to its partner) and Mb = sum (d.u_p)/r^3, and
// xbar = -u S1 + Gm V + Wd, mbar = -G Mb: the exact regrouping of sum_p -J w, w = Gm_p u - Gm u_p,
// J = (I - 3 d d^T / r^2)/r^3, d.w = Gm_p (d.u) - Gm (d.u_p). Work item k of system
// b is the tile pair (I, J), I <= J; its sums for tile I go to part[b][I][J], those for tile J to
// part[b][J][I] (5 values x 32 lanes each), reduced per body in a fixed order afterwards.
struct VjpBody {
  double x, y, z, gm, u0, u1, u2, rc, A;
  u64 Q;
  int al;
};

__device__ __forceinline__ void vjp_shfl(VjpBody &B, int src) {
  B.x = __shfl_sync(0xffffffffu, B.x, src); B.y = __shfl_sync(0xffffffffu, B.y, src);
  B.z = __shfl_sync(0xffffffffu, B.z, src); B.gm = __shfl_sync(0xffffffffu, B.gm, src);
  B.u0 = __shfl_sync(0xffffffffu, B.u0, src); B.u1 = __shfl_sync(0xffffffffu, B.u1, src);
  B.u2 = __shfl_sync(0xffffffffu, B.u2, src); B.rc = __shfl_sync(0xffffffffu, B.rc, src);
  B.A = __shfl_sync(0xffffffffu, B.A, src); B.Q = __shfl_sync(0xffffffffu, B.Q, src);
  B.al = __shfl_sync(0xffffffffu, B.al, src);
}

struct VjpAcc {
  double S1, V0, V1, V2, W0, W1, W2, Mb, e0, e1, e2, me, rcb;
};

__device__ __forceinline__ void vjp_acc_zero(VjpAcc &a) {
  a.S1 = a.V0 = a.V1 = a.V2 = a.W0 = a.W1 = a.W2 = a.Mb = a.e0 = a.e1 = a.e2 = a.me = a.rcb = 0.0;
}

__device__ __forceinline__ void vjp_acc_shfl(VjpAcc &a, int src) {
  a.S1 = __shfl_sync(0xffffffffu, a.S1, src); a.V0 = __shfl_sync(0xffffffffu, a.V0, src);
  a.V1 = __shfl_sync(0xffffffffu, a.V1, src); a.V2 = __shfl_sync(0xffffffffu, a.V2, src);
  a.W0 = __shfl_sync(0xffffffffu, a.W0, src); a.W1 = __shfl_sync(0xffffffffu, a.W1, src);
  a.W2 = __shfl_sync(0xffffffffu, a.W2, src); a.Mb = __shfl_sync(0xffffffffu, a.Mb, src);
  a.e0 = __shfl_sync(0xffffffffu, a.e0, src); a.e1 = __shfl_sync(0xffffffffu, a.e1, src);
  a.e2 = __shfl_sync(0xffffffffu, a.e2, src); a.me = __shfl_sync(0xffffffffu, a.me, src);
  a.rcb = __shfl_sync(0xffffffffu, a.rcb, src);
}

// The pair (a, b) with d = x_b - x_a, both sides.
__device__ __forceinline__ void vjp_pair(const VjpBody &Pa, const VjpBody &Pb, int ia, int ib, double G, bool act,
                                         VjpAcc &aa, VjpAcc &ab) {
  if (!act || !Pa.al || !Pb.al) return;
  const double dx = Pb.x - Pa.x, dy = Pb.y - Pa.y, dz = Pb.z - Pa.z;
  const double r2 = r2_exact(dx, dy, dz);
  const double ua[3] = {Pa.u0, Pa.u1, Pa.u2}, ub[3] = {Pb.u0, Pb.u1, Pb.u2};
  if (dbits(r2) < umax64(Pa.Q, Pb.Q)) {  // changeover zone (rare): general form
    double Jw[3], mba, mbb, rcbp;
    pair_vjp_zone(dx, dy, dz, Pa.gm, Pb.gm, G, ua, ub, pmin(Pa.A, Pb.A), pmax(Pa.rc, Pb.rc), Jw, mba, mbb, rcbp);
    aa.e0 -= Jw[0]; aa.e1 -= Jw[1]; aa.e2 -= Jw[2]; aa.me += mba;
    ab.e0 += Jw[0]; ab.e1 += Jw[1]; ab.e2 += Jw[2]; ab.me += mbb;
    const bool own_a = dbits(Pa.rc) > dbits(Pb.rc) || (dbits(Pa.rc) == dbits(Pb.rc) && ia < ib);
    if (own_a) aa.rcb += rcbp; else ab.rcb += rcbp;
    return;
  }
  const double yr = rsqrt_refined(r2), yr2 = yr * yr, yr3 = yr2 * yr;
  const double dua = fma(dz, ua[2], fma(dy, ua[1], dx * ua[0]));
  const double dub = fma(dz, ub[2], fma(dy, ub[1], dx * ub[0]));
  const double dw = fma(Pb.gm, dua, -Pa.gm * dub);  // d.w with w = Gm_b u_a - Gm_a u_b
  const double cc = yr3 * yr2 * dw;                 // the factor 3 of Wd is applied to the sums
  aa.S1 = fma(Pb.gm, yr3, aa.S1);
  aa.V0 = fma(yr3, ub[0], aa.V0); aa.V1 = fma(yr3, ub[1], aa.V1); aa.V2 = fma(yr3, ub[2], aa.V2);
  aa.W0 = fma(cc, dx, aa.W0); aa.W1 = fma(cc, dy, aa.W1); aa.W2 = fma(cc, dz, aa.W2);
  aa.Mb = fma(yr3, dub, aa.Mb);
  ab.S1 = fma(Pa.gm, yr3, ab.S1);
  ab.V0 = fma(yr3, ua[0], ab.V0); ab.V1 = fma(yr3, ua[1], ab.V1); ab.V2 = fma(yr3, ua[2], ab.V2);
  ab.W0 = fma(-cc, dx, ab.W0); ab.W1 = fma(-cc, dy, ab.W1); ab.W2 = fma(-cc, dz, ab.W2);
  ab.Mb = fma(-yr3, dua, ab.Mb);
}

// The five per-body outputs of a set of sums.
__device__ __forceinline__ void vjp_store(double *p, const VjpAcc &a, const VjpBody &B, double G) {
  p[0] = a.e0 + fma(-B.u0, a.S1, fma(B.gm, a.V0, 3.0 * a.W0));
  p[32] = a.e1 + fma(-B.u1, a.S1, fma(B.gm, a.V1, 3.0 * a.W1));
  p[64] = a.e2 + fma(-B.u2, a.S1, fma(B.gm, a.V2, 3.0 * a.W2));
  p[96] = fma(-G, a.Mb, a.me);
  p[128] = a.rcb;
}

__global__ void __launch_bounds__(128) k_ad_kick_vjp_sym(Sim S, AdjDev D, double h, const double *xk, double *part) {
  const int T = D.Np >> 5, npair = T * (T + 1) / 2, NB = D.NB;
  const int lane = threadIdx.x & 31;
  const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (item >= D.B * npair) return;
  const int b = item / npair;
  int k = item % npair, I = 0;
  while (k >= T - I) { k -= T - I; ++I; }
  const int J = I + k;
  const int base = b * D.Np;
  auto load = [&](int g, VjpBody &B) {
    B.x = xk[g]; B.y = xk[NB + g]; B.z = xk[2 * NB + g];
    B.gm = S.gm[g]; B.rc = S.rc[g]; B.A = S.A[g]; B.Q = S.rcsq[g]; B.al = S.alive[g];
    B.u0 = h * D.vb[g]; B.u1 = h * D.vb[NB + g]; B.u2 = h * D.vb[2 * NB + g];
  };
  VjpBody Pi, Pj;
  load(base + I * 32 + lane, Pi);
  VjpAcc ai, aj;
  vjp_acc_zero(ai);
  vjp_acc_zero(aj);
  const int src = (lane + 1) & 31;
  double *pbase = part + (size_t)b * T * T * 160;
  if (I == J) {  // diagonal tile: lane l pairs with l + s + 1, s = 0..15 (the last step for half the lanes)
    Pj = Pi;
    for (int s = 0; s < 16; ++s) {
      vjp_shfl(Pj, src);
      vjp_acc_shfl(aj, src);
      const int jl = (lane + s + 1) & 31;
      vjp_pair(Pi, Pj, I * 32 + lane, I * 32 + jl, D.G, s < 15 || lane < 16, ai, aj);
    }
    const int home = (lane + 16) & 31;  // the j sums return to the lane that owns body I*32 + lane
    vjp_acc_shfl(aj, home);
    Pj = Pi;
    VjpAcc t = ai;
    t.S1 += aj.S1; t.V0 += aj.V0; t.V1 += aj.V1; t.V2 += aj.V2; t.W0 += aj.W0; t.W1 += aj.W1; t.W2 += aj.W2;
    t.Mb += aj.Mb; t.e0 += aj.e0; t.e1 += aj.e1; t.e2 += aj.e2; t.me += aj.me; t.rcb += aj.rcb;
    vjp_store(pbase + ((size_t)I * T + I) * 160 + lane, t, Pi, D.G);
  } else {  // off-diagonal: lane l meets body J*32 + (l + s) mod 32 at step s
    load(base + J * 32 + lane, Pj);
    for (int s = 0; s < 32; ++s) {
      const int jl = (lane + s) & 31;
      vjp_pair(Pi, Pj, I * 32 + lane, J * 32 + jl, D.G, true, ai, aj);
      vjp_shfl(Pj, src);
      vjp_acc_shfl(aj, src);
    }
    // after 32 rotations every j value and j sum is back on its owning lane
    vjp_store(pbase + ((size_t)I * T + J) * 160 + lane, ai, Pi, D.G);
    vjp_store(pbase + ((size_t)J * T + I) * 160 + lane, aj, Pj, D.G);
  }
}

// Sum of the tile partials of each body, in a fixed order, into xbar, mbar, rcbar.
__global__ void k_ad_kick_vjp_reduce(Sim S, AdjDev D, const double *part) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= D.NB || !S.alive[g]) return;
  const int T = D.Np >> 5, b = g / D.Np, i = g % D.Np, I = i >> 5, lane = i & 31;
  const double *p = part + ((size_t)b * T * T + (size_t)I * T) * 160 + lane;
  double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int J = 0; J < T; ++J)
    for (int c = 0; c < 5; ++c) t[c] += p[(size_t)J * 160 + 32 * c];
  const int NB = D.NB;
  for (int c = 0; c < 3; ++c) D.xb[c * NB + g] += t[c];
  D.mb[g] += t[3];
  D.rcb[g] += t[4];
}

// Sun-drift VJP: x' = x + (h/m0) sum_k m_k v_k -> vbar_i += (h/m0) m_i Xs, mbar_i += (h/m0) v_i . Xs,
// Xs = sum_k xbar_k over the system (fixed-order tree). v = the velocities the drift saw.
__global__ void __launch_bounds__(256) k_ad_sundrift_vjp(Sim S, AdjDev D, double h, const double *vrec) {
  __shared__ double red[3][256];
  const int b = blockIdx.x, tid = threadIdx.x, NB = D.NB;
  double s[3] = {0.0, 0.0, 0.0};
  for (int i = tid; i < D.Np; i += 256) {
    const int g = b * D.Np + i;
    if (!S.alive[g]) continue;
    for (int c = 0; c < 3; ++c) s[c] += D.xb[c * NB + g];
  }
  for (int c = 0; c < 3; ++c) red[c][tid] = s[c];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o)
      for (int c = 0; c < 3; ++c) red[c][tid] += red[c][tid + o];
    __syncthreads();
  }
  const double f = h / D.m0[b];
  const double X[3] = {red[0][0], red[1][0], red[2][0]};
  for (int i = tid; i < D.Np; i += 256) {
    const int g = b * D.Np + i;
    if (!S.alive[g]) continue;
    const double mi = S.m[g];
    double dm = 0.0;
    for (int c = 0; c < 3; ++c) {
      D.vb[c * NB + g] = fma(f * mi, X[c], D.vb[c * NB + g]);
      dm = fma(vrec[c * NB + g], X[c], dm);
    }
    D.mb[g] = fma(f, dm, D.mb[g]);
  }
}

// c_dst[k][m] = (m+1) / (2m+2+k)!: coefficients of c_k'(z) = -sum_m c_dst[k][m] (-z)^m
constexpr int DST_TERMS = 14;
__constant__ double c_dst[4][DST_TERMS];

// Derivatives of the Stumpff functions, c_k'(z): series for |z| <= 1 (14 terms: the tail is below
// 1e-22), identities beyond (c0' = -c1/2, c_k' = (c_{k-1} - k c_k)/(2z)).
__device__ __forceinline__ void dstumpff(double z, const double c[4], double dc[4]) {
  if (fabs(z) <= 1.0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double acc = c_dst[k][DST_TERMS - 1];
#pragma unroll
      for (int m = DST_TERMS - 2; m >= 0; --m) acc = fma(acc, -z, c_dst[k][m]);
      dc[k] = -acc;
    }
  } else {
    dc[0] = -0.5 * c[1];
    dc[1] = (c[0] - c[1]) / (2.0 * z);
    dc[2] = (c[1] - 2.0 * c[2]) / (2.0 * z);
    dc[3] = (c[2] - 3.0 * c[3]) / (2.0 * z);
  }
}

// Kepler-drift VJP (Eq. fg) of the bodies outside encounter groups: implicit differentiation of
// the universal Kepler equation at the recorded solution s.
__global__ void k_ad_kepler_vjp(Sim S, AdjDev D, double tau, const double *x1, const double *v1, const double *srec) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= D.NB || !S.alive[g] || D.ingrp[g]) return;
  const int NB = D.NB;
  const double mu = D.G * D.m0[sys_of_body(D, g)];
  const double x[3] = {x1[g], x1[NB + g], x1[2 * NB + g]}, v[3] = {v1[g], v1[NB + g], v1[2 * NB + g]};
  const double s = srec[g];
  const double r0 = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  const double u = x[0] * v[0] + x[1] * v[1] + x[2] * v[2];
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const double beta = 2.0 * mu / r0 - v2;
  const double z = beta * s * s;
  double c[4], dc[4];
  stumpff_d(z, c[0], c[1], c[2], c[3]);
  dstumpff(z, c, dc);
  const double s2 = s * s, s3 = s2 * s;
  const double G0 = c[0], G1 = s * c[1], G2 = s2 * c[2], G3 = s3 * c[3];
  const double r = r0 * G0 + u * G1 + mu * G2;
  const double f = 1.0 - (mu / r0) * G2, gg = tau - mu * G3;
  const double fd = -mu * G1 / (r * r0), gd = 1.0 - (mu / r) * G2;
  const double xb[3] = {D.xb[g], D.xb[NB + g], D.xb[2 * NB + g]};
  const double vb[3] = {D.vb[g], D.vb[NB + g], D.vb[2 * NB + g]};
  const double fb = xb[0] * x[0] + xb[1] * x[1] + xb[2] * x[2];
  const double gb = xb[0] * v[0] + xb[1] * v[1] + xb[2] * v[2];
  const double fdb = vb[0] * x[0] + vb[1] * x[1] + vb[2] * x[2];
  const double gdb = vb[0] * v[0] + vb[1] * v[1] + vb[2] * v[2];
  double r0b = 0.0, ub = 0.0, v2b = 0.0, rb = 0.0, G0b = 0.0, G1b = 0.0, G2b = 0.0, G3b = 0.0;
  // f = 1 - mu G2 / r0
  r0b += fb * mu * G2 / (r0 * r0); G2b -= fb * mu / r0;
  // g = tau - mu G3
  G3b -= gb * mu;
  // fd = -mu G1 / (r r0)
  G1b -= fdb * mu / (r * r0); rb += fdb * mu * G1 / (r * r * r0); r0b += fdb * mu * G1 / (r * r0 * r0);
  // gd = 1 - mu G2 / r
  G2b -= gdb * mu / r; rb += gdb * mu * G2 / (r * r);
  // r = r0 G0 + u G1 + mu G2
  r0b += rb * G0; ub += rb * G1; G0b += rb * r0; G1b += rb * u; G2b += rb * mu;
  // G_k(s, beta): dG0/ds = -beta G1, dG_k/ds = G_{k-1}; dG_k/dbeta = s^(k+2) c_k'(z)
  double sb = G0b * (-beta * G1) + G1b * G0 + G2b * G1 + G3b * G2;
  const double dG1b = s3 * dc[1], dG2b = s2 * s2 * dc[2], dG3b = s2 * s3 * dc[3];
  double betab = G0b * s2 * dc[0] + G1b * dG1b + G2b * dG2b + G3b * dG3b;
  // s from F(s) = r0 G1 + u G2 + mu G3 - tau = 0, F_s = r
  const double Fbeta = r0 * dG1b + u * dG2b + mu * dG3b;
  r0b -= sb * G1 / r; ub -= sb * G2 / r; betab -= sb * Fbeta / r;
  // beta = 2 mu / r0 - v2
  r0b -= betab * 2.0 * mu / (r0 * r0); v2b -= betab;
  double nx[3], nv[3];
  for (int k = 0; k < 3; ++k) {
    nx[k] = f * xb[k] + fd * vb[k] + r0b * x[k] / r0 + ub * v[k];
    nv[k] = gg * xb[k] + gd * vb[k] + ub * x[k] + 2.0 * v2b * v[k];
  }
  for (int k = 0; k < 3; ++k) { D.xb[k * NB + g] = nx[k]; D.vb[k * NB + g] = nv[k]; }
}

__global__ void k_ad_mark(AdjDev D, const int *gstart, const int *gsize, const int *gmem, const int *ngroups) {
  const int ng = *ngroups;
  for (int gi = blockIdx.x; gi < ng; gi += gridDim.x)
    for (int q = threadIdx.x; q < gsize[gi]; q += blockDim.x) D.ingrp[gmem[gstart[gi] + q]] = 1;
}

// BS VJP: one CTA per group, warp w = BS level w + 1 (the levels of a substep are independent
// given its start state). The accepted substeps are recomputed from the group's pre-drift state
// with the recorded (H, level) sequence, then differentiated backwards: Neville weights (linear),
// then each level's modified-midpoint chain (Gragg), recomputed with its positions kept in shared
// memory. Lane q is member q (at most 32).
struct GrpShared {  // per group
  double gm[BS_GMAX], A[BS_GMAX], rc[BS_GMAX];
  u64 rcsq[BS_GMAX];
};
struct LevShared {  // per level (warp)
  double pos[2 * BS_LEVELS + 1][BS_GMAX][3];  // chain positions z_0..z_n
  double cur[BS_GMAX][3];                     // positions for an acceleration evaluation
  double fv[BS_GMAX][3];                      // adjoints of the members' accelerations
  double out[BS_GMAX][6];                     // the level's result (forward) or z0 adjoint (reverse)
  double mb[BS_GMAX], rcb[BS_GMAX];           // the level's mbar / rcbar contributions
};

__device__ void grp_accel(const GrpShared &G, const double (*cur)[3], int g, int q, double Gm0, double *a) {
  a[0] = a[1] = a[2] = 0.0;
  if (q >= g) return;
  const double xq = cur[q][0], yq = cur[q][1], zq = cur[q][2];
  const double r2 = fma(zq, zq, fma(yq, yq, xq * xq));
  const double f = -Gm0 * rcube_refined(r2);
  a[0] = f * xq; a[1] = f * yq; a[2] = f * zq;
  for (int p = 0; p < g; ++p) {
    if (p == q) continue;
    const double dx = cur[p][0] - xq, dy = cur[p][1] - yq, dz = cur[p][2] - zq;
    const double pr2 = fma(dz, dz, fma(dy, dy, dx * dx));
    if (dbits(pr2) >= umax64(G.rcsq[q], G.rcsq[p])) continue;
    const double yr = rsqrt_refined(pr2);
    double wB, wA;
    changeover_w(pr2 * yr, pmin(G.A[q], G.A[p]), 0, wB, wA);
    const double ff = G.gm[p] * wA * (yr * yr * yr);
    a[0] = fma(ff, dx, a[0]); a[1] = fma(ff, dy, a[1]); a[2] = fma(ff, dz, a[2]);
  }
}

// x-adjoint of the group acceleration field at cur, given fv (adjoints of the accelerations):
// central term and (1 - K) pair terms; also mbar, rcbar of member q.
__device__ void grp_accel_vjp(const GrpShared &G, const double (*cur)[3], const double (*fv)[3], int g, int q,
                              double Gm0, double Gc, double *xb, double &mb, double &rcb) {
  xb[0] = xb[1] = xb[2] = 0.0;
  if (q >= g) return;
  const double xq = cur[q][0], yq = cur[q][1], zq = cur[q][2];
  const double uq[3] = {fv[q][0], fv[q][1], fv[q][2]};
  {  // central: a = -G m0 x / |x|^3, J = -G m0 (I/r^3 - 3 x x^T / r^5)
    const double r2 = fma(zq, zq, fma(yq, yq, xq * xq));
    const double yr = rsqrt_refined(r2), yr3 = yr * yr * yr, yr5 = yr3 * yr * yr;
    const double xu = fma(zq, uq[2], fma(yq, uq[1], xq * uq[0]));
    xb[0] -= Gm0 * (uq[0] * yr3 - 3.0 * xq * xu * yr5);
    xb[1] -= Gm0 * (uq[1] * yr3 - 3.0 * yq * xu * yr5);
    xb[2] -= Gm0 * (uq[2] * yr3 - 3.0 * zq * xu * yr5);
  }
  for (int p = 0; p < g; ++p) {
    if (p == q) continue;
    const double dx = cur[p][0] - xq, dy = cur[p][1] - yq, dz = cur[p][2] - zq;
    const double pr2 = fma(dz, dz, fma(dy, dy, dx * dx));
    if (dbits(pr2) >= umax64(G.rcsq[q], G.rcsq[p])) continue;
    const double up[3] = {fv[p][0], fv[p][1], fv[p][2]};
    double rcb_pair = 0.0;
    pair_vjp<-1>(dx, dy, dz, G.gm[q], G.gm[p], Gc, uq, up, pmin(G.A[q], G.A[p]), pmax(G.rc[q], G.rc[p]), true, xb,
                 mb, rcb_pair);
    const bool own = dbits(G.rc[q]) > dbits(G.rc[p]) || (dbits(G.rc[q]) == dbits(G.rc[p]) && q < p);
    if (own) rcb += rcb_pair;
  }
}

// The level-l chain of one BS substep of length H from y (lane-held): result into L.out, the chain
// positions into L.pos (when keep).
__device__ void grp_chain(const GrpShared &G, LevShared &L, int g, int q, double Gm0, double H, int l, const double *y,
                          bool keep) {
  const int n = 2 * l;
  const double h = H / n, h2 = 2.0 * h;
  double za[6], zb[6], a[3];
  for (int c = 0; c < 6; ++c) za[c] = y[c];
  if (q < g) for (int c = 0; c < 3; ++c) { L.cur[q][c] = za[c]; if (keep) L.pos[0][q][c] = za[c]; }
  __syncwarp();
  grp_accel(G, L.cur, g, q, Gm0, a);
  __syncwarp();
  for (int c = 0; c < 3; ++c) { zb[c] = fma(h, za[3 + c], za[c]); zb[3 + c] = fma(h, a[c], za[3 + c]); }
  for (int m = 1; m <= n; ++m) {
    if (q < g) for (int c = 0; c < 3; ++c) { L.cur[q][c] = zb[c]; if (keep) L.pos[m][q][c] = zb[c]; }
    __syncwarp();
    grp_accel(G, L.cur, g, q, Gm0, a);
    __syncwarp();
    if (m < n) {
      double zn[6];
      for (int c = 0; c < 3; ++c) { zn[c] = fma(h2, zb[3 + c], za[c]); zn[3 + c] = fma(h2, a[c], za[3 + c]); }
      for (int c = 0; c < 6; ++c) { za[c] = zb[c]; zb[c] = zn[c]; }
    } else if (q < g) {
      for (int c = 0; c < 3; ++c) {
        L.out[q][c] = 0.5 * fma(h, zb[3 + c], zb[c] + za[c]);
        L.out[q][3 + c] = 0.5 * fma(h, a[c], zb[3 + c] + za[3 + c]);
      }
    }
  }
}

constexpr int BSV_WARPS = BS_LEVELS;

// Groups of at most four members (nearly all of them): the whole group on one warp, lane = (level
// (lane >> 2) + 1, member lane & 3), so one warp instruction serves all levels; an FP64 warp
// instruction costs the same whatever its active lanes. Every level's lanes run the same arithmetic
// as in the level-per-warp kernel below, stepping through the evaluations in lock step (a level
// takes part while the index lies within its chain), so the results are that kernel's.
constexpr int BSV4_GROUPS = 4;  // groups (warps) per CTA
struct LevShared4 {
  double pos[2 * BS_LEVELS + 1][4][3];
  double cur[4][3], fv[4][3], out[4][6];
  double mb[4], rcb[4];
};
struct GrpVjp4 {
  GrpShared G;
  LevShared4 L[BS_LEVELS];
};

__global__ void __launch_bounds__(32 * BSV4_GROUPS) k_ad_bs_vjp4(Sim S, AdjDev D, SubRec R, const double *x1,
                                                                 const double *v1) {
  extern __shared__ double smraw4[];
  GrpVjp4 &W = ((GrpVjp4 *)smraw4)[threadIdx.x >> 5];
  GrpShared &G = W.G;
  const int lane = threadIdx.x & 31, l = (lane >> 2) + 1, q = lane & 3, NB = D.NB;
  LevShared4 &L = W.L[l - 1];
  const int ng = *R.ngroups;
  for (int gi = blockIdx.x * BSV4_GROUPS + (threadIdx.x >> 5); gi < ng; gi += gridDim.x * BSV4_GROUPS) {
    const int g = R.gsize[gi], g0 = R.gstart[gi];
    if (g > 4) continue;  // uniform within the warp: the level-per-warp kernel takes it
    const int body = q < g ? R.gmem[g0 + q] : 0;
    const double Gm0 = D.G * D.m0[sys_of_body(D, R.gmem[g0])];
    if (l == 1 && q < g) {
      G.gm[q] = S.gm[body]; G.A[q] = S.A[body]; G.rc[q] = S.rc[body]; G.rcsq[q] = S.rcsq[body];
    }
    double y[6], yb[6];
    for (int c = 0; c < 3; ++c) {
      y[c] = q < g ? x1[c * NB + body] : 0.0;
      y[3 + c] = q < g ? v1[c * NB + body] : 0.0;
      yb[c] = q < g ? D.xb[c * NB + body] : 0.0;
      yb[3 + c] = q < g ? D.vb[c * NB + body] : 0.0;
    }
    L.mb[q] = 0.0; L.rcb[q] = 0.0;
    __syncwarp();
    const int nseq = R.seq_len[gi], soff = R.seq_off[gi];
    const long long yoff = R.y_off[gi];
    for (int s = nseq - 1; s >= 0; --s) {
      const double2 hk = S.seq_pool[soff + s];
      const double H = hk.x;
      const int k = (int)hk.y;
      const bool lvl = l <= k;  // this lane's level enters the accepted extrapolation
      const int n = 2 * l;
      const double h = H / n, h2 = 2.0 * h;
      const double lam = lvl ? c_lambda[k][l] : 0.0;
      double y0[6];  // start state of accepted substep s: the pre-drift state, or recorded by k_bs
      for (int c = 0; c < 6; ++c)
        y0[c] = s == 0 ? y[c] : (q < g ? S.y_pool[yoff + ((long long)(s - 1) * g + q) * 6 + c] : 0.0);
      // the level's modified-midpoint chain again, positions kept
      double za[6], zb[6], a[3] = {0.0, 0.0, 0.0};
      for (int c = 0; c < 6; ++c) za[c] = y0[c];
      if (lvl && q < g) for (int c = 0; c < 3; ++c) { L.cur[q][c] = za[c]; L.pos[0][q][c] = za[c]; }
      __syncwarp();
      if (lvl) grp_accel(G, L.cur, g, q, Gm0, a);
      __syncwarp();
      for (int c = 0; c < 3; ++c) { zb[c] = fma(h, za[3 + c], za[c]); zb[3 + c] = fma(h, a[c], za[3 + c]); }
      for (int m = 1; m <= 2 * k; ++m) {
        const bool on = lvl && m <= n;
        if (on && q < g) for (int c = 0; c < 3; ++c) { L.cur[q][c] = zb[c]; L.pos[m][q][c] = zb[c]; }
        __syncwarp();
        if (on) grp_accel(G, L.cur, g, q, Gm0, a);
        __syncwarp();
        if (on && m < n) {
          double zn[6];
          for (int c = 0; c < 3; ++c) { zn[c] = fma(h2, zb[3 + c], za[c]); zn[3 + c] = fma(h2, a[c], za[3 + c]); }
          for (int c = 0; c < 6; ++c) { za[c] = zb[c]; zb[c] = zn[c]; }
        }
      }
      // backwards through the chain, scaled by the Neville weight lam: t = n is the reverse of
      // out = (z_n + z_{n-1} + h F(z_n)) / 2, t = n-1 .. 1 of z_{t+1} = z_{t-1} + 2h F(z_t), t = 0 of
      // z_1 = z_0 + h F(z_0); zbn holds zbar_{t+1}, zbn1 the partial zbar_t
      double zbn[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, zbn1[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, carry[6], xbq[3];
      double mbq = L.mb[q], rcbq = L.rcb[q];
      for (int t = 2 * k; t >= 0; --t) {
        const bool on = lvl && t <= n;
        if (on) {
          if (t == n) {
            for (int c = 0; c < 6; ++c) { zbn[c] = 0.5 * lam * yb[c]; zbn1[c] = 0.5 * lam * yb[c]; }
            if (q < g) for (int c = 0; c < 3; ++c) { L.cur[q][c] = L.pos[n][q][c]; L.fv[q][c] = 0.5 * h * lam * yb[3 + c]; }
          } else if (t >= 1) {
            for (int c = 0; c < 6; ++c) carry[c] = zbn[c];  // z_{t-1} gets zbar_{t+1}
            if (q < g) for (int c = 0; c < 3; ++c) { L.cur[q][c] = L.pos[t][q][c]; L.fv[q][c] = h2 * zbn[3 + c]; }
          } else {
            if (q < g) for (int c = 0; c < 3; ++c) { L.cur[q][c] = L.pos[0][q][c]; L.fv[q][c] = h * zbn[3 + c]; }
          }
        }
        __syncwarp();
        if (on) grp_accel_vjp(G, L.cur, L.fv, g, q, Gm0, D.G, xbq, mbq, rcbq);
        __syncwarp();
        if (on) {
          if (t == n) {
            for (int c = 0; c < 3; ++c) { zbn[c] += xbq[c]; zbn[3 + c] += 0.5 * h * lam * yb[c]; }
          } else if (t >= 1) {
            for (int c = 0; c < 3; ++c) { zbn1[c] += xbq[c]; zbn1[3 + c] += h2 * zbn[c]; }
            for (int c = 0; c < 6; ++c) { zbn[c] = zbn1[c]; zbn1[c] = carry[c]; }
          } else {
            for (int c = 0; c < 3; ++c) {
              L.out[q][c] = zbn1[c] + zbn[c] + xbq[c];
              L.out[q][3 + c] = zbn1[3 + c] + zbn[3 + c] + h * zbn[c];
            }
          }
        }
      }
      if (lvl) { L.mb[q] = mbq; L.rcb[q] = rcbq; }
      __syncwarp();
      for (int c = 0; c < 6; ++c) {  // ybar of the substep's start: sum over levels in order
        double acc = 0.0;
        for (int ll = 1; ll <= k; ++ll) acc += W.L[ll - 1].out[q][c];
        yb[c] = acc;
      }
      __syncwarp();
    }
    if (l == 1 && q < g) {
      double mb = 0.0, rcb = 0.0;
      for (int ll = 0; ll < BS_LEVELS; ++ll) { mb += W.L[ll].mb[q]; rcb += W.L[ll].rcb[q]; }
      for (int c = 0; c < 3; ++c) { D.xb[c * NB + body] = yb[c]; D.vb[c * NB + body] = yb[3 + c]; }
      D.mb[body] += mb;
      D.rcb[body] += rcb;
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32 * BSV_WARPS) k_ad_bs_vjp(Sim S, AdjDev D, SubRec R, const double *x1,
                                                              const double *v1) {
  extern __shared__ double smraw[];
  __shared__ GrpShared G;
  LevShared *LS = (LevShared *)smraw;
  const int q = threadIdx.x & 31, w = threadIdx.x >> 5, l = w + 1, NB = D.NB;
  LevShared &L = LS[w];
  const int ng = *R.ngroups;
  for (int gi = blockIdx.x; gi < ng; gi += gridDim.x) {
    const int g = R.gsize[gi], g0 = R.gstart[gi];
    if (g <= 4 || g > BS_GMAX) continue;  // uniform: groups of up to four members go to k_ad_bs_vjp4
    const int body = q < g ? R.gmem[g0 + q] : 0;
    const double Gm0 = D.G * D.m0[sys_of_body(D, R.gmem[g0])];
    if (w == 0 && q < g) {
      G.gm[q] = S.gm[body]; G.A[q] = S.A[body]; G.rc[q] = S.rc[body]; G.rcsq[q] = S.rcsq[body];
    }
    double y[6];
    for (int c = 0; c < 3; ++c) {
      y[c] = q < g ? x1[c * NB + body] : 0.0;
      y[3 + c] = q < g ? v1[c * NB + body] : 0.0;
    }
    L.mb[q] = 0.0; L.rcb[q] = 0.0;
    __syncthreads();
    const int nseq = R.seq_len[gi], soff = R.seq_off[gi];
    const long long yoff = R.y_off[gi];
    double yb[6];
    for (int c = 0; c < 3; ++c) {
      yb[c] = q < g ? D.xb[c * NB + body] : 0.0;
      yb[3 + c] = q < g ? D.vb[c * NB + body] : 0.0;
    }
    // backward over the substeps; level l's chain on warp l - 1
    for (int s = nseq - 1; s >= 0; --s) {
      const double2 hk = S.seq_pool[soff + s];
      const double H = hk.x;
      const int k = (int)hk.y;
      double y0[6];  // start state of accepted substep s: the pre-drift state, or recorded by k_bs
      for (int c = 0; c < 6; ++c)
        y0[c] = s == 0 ? y[c] : (q < g ? S.y_pool[yoff + ((long long)(s - 1) * g + q) * 6 + c] : 0.0);
      if (l <= k) {
        const double lam = c_lambda[k][l];
        const int n = 2 * l;
        const double h = H / n, h2 = 2.0 * h;
        grp_chain(G, L, g, q, Gm0, H, l, y0, true);
        // reverse of out = (z_n + z_{n-1} + h F(z_n)) / 2, scaled by lam
        double zbn[6], zbn1[6], xbq[3];
        double mbq = L.mb[q], rcbq = L.rcb[q];
        for (int c = 0; c < 6; ++c) { zbn[c] = 0.5 * lam * yb[c]; zbn1[c] = 0.5 * lam * yb[c]; }
        if (q < g) for (int c = 0; c < 3; ++c) { L.cur[q][c] = L.pos[n][q][c]; L.fv[q][c] = 0.5 * h * lam * yb[3 + c]; }
        __syncwarp();
        grp_accel_vjp(G, L.cur, L.fv, g, q, Gm0, D.G, xbq, mbq, rcbq);
        __syncwarp();
        for (int c = 0; c < 3; ++c) { zbn[c] += xbq[c]; zbn[3 + c] += 0.5 * h * lam * yb[c]; }
        // z_{m+1} = z_{m-1} + 2h F(z_m), m = n-1 .. 1; zbn holds zbar_{m+1}, zbn1 the partial zbar_m
        for (int m = n - 1; m >= 1; --m) {
          double carry[6];
          for (int c = 0; c < 6; ++c) carry[c] = zbn[c];  // z_{m-1} gets zbar_{m+1}
          if (q < g) for (int c = 0; c < 3; ++c) { L.cur[q][c] = L.pos[m][q][c]; L.fv[q][c] = h2 * zbn[3 + c]; }
          __syncwarp();
          grp_accel_vjp(G, L.cur, L.fv, g, q, Gm0, D.G, xbq, mbq, rcbq);
          __syncwarp();
          for (int c = 0; c < 3; ++c) { zbn1[c] += xbq[c]; zbn1[3 + c] += h2 * zbn[c]; }
          for (int c = 0; c < 6; ++c) { zbn[c] = zbn1[c]; zbn1[c] = carry[c]; }
        }
        // z_1 = z_0 + h F(z_0)
        if (q < g) for (int c = 0; c < 3; ++c) { L.cur[q][c] = L.pos[0][q][c]; L.fv[q][c] = h * zbn[3 + c]; }
        __syncwarp();
        grp_accel_vjp(G, L.cur, L.fv, g, q, Gm0, D.G, xbq, mbq, rcbq);
        __syncwarp();
        for (int c = 0; c < 3; ++c) {
          L.out[q][c] = zbn1[c] + zbn[c] + xbq[c];
          L.out[q][3 + c] = zbn1[3 + c] + zbn[3 + c] + h * zbn[c];
        }
        L.mb[q] = mbq; L.rcb[q] = rcbq;
      }
      __syncthreads();
      for (int c = 0; c < 6; ++c) {  // ybar of the substep's start: sum over levels in order
        double acc = 0.0;
        for (int ll = 1; ll <= k; ++ll) acc += LS[ll - 1].out[q][c];
        yb[c] = acc;
      }
      __syncthreads();
    }
    if (w == 0 && q < g) {
      double mb = 0.0, rcb = 0.0;
      for (int ll = 0; ll < BSV_WARPS; ++ll) { mb += LS[ll].mb[q]; rcb += LS[ll].rcb[q]; }
      for (int c = 0; c < 3; ++c) { D.xb[c * NB + body] = yb[c]; D.vb[c * NB + body] = yb[3 + c]; }
      D.mb[body] += mb;
      D.rcb[body] += rcb;
    }
    __syncthreads();
  }
}

// Critical-radius VJP at the state of the step's start (x, v recorded): rc = max(n1 a h, n2 tau |v|).
__global__ void k_ad_rcrit_vjp(Sim S, AdjDev D, DevParams P, double tau_abs, const double *xr, const double *vr) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= D.NB || !S.alive[g]) return;
  const int NB = D.NB;
  const double rcb = D.rcb[g];
  D.rcb[g] = 0.0;
  if (dbits(rcb) == 0ULL) return;
  const double mu = D.G * D.m0[sys_of_body(D, g)];
  const double x[3] = {xr[g], xr[NB + g], xr[2 * NB + g]}, v[3] = {vr[g], vr[NB + g], vr[2 * NB + g]};
  const double r2 = fma(x[2], x[2], fma(x[1], x[1], x[0] * x[0]));
  const double r = sqrt(r2);
  const double v2 = fma(v[2], v[2], fma(v[1], v[1], v[0] * v[0]));
  const double inva = 2.0 / r - v2 / mu;
  const bool bound = inva > 0.0;
  const double a = bound ? 1.0 / inva : r;
  const double hl = S.hill[g];
  const double a1 = P.n1 * a * hl, vabs = sqrt(v2), a2 = P.n2 * tau_abs * vabs;
  if (a1 > a2) {  // Hill branch
    const double ab = rcb * P.n1 * hl;
    const double mi = S.m[g];
    if (mi > 0.0) D.mb[g] += rcb * a1 / (3.0 * mi);
    for (int c = 0; c < 3; ++c) {
      if (bound) {
        D.xb[c * NB + g] += ab * 2.0 * a * a * x[c] / (r2 * r);
        D.vb[c * NB + g] += ab * 2.0 * a * a * v[c] / mu;
      } else {
        D.xb[c * NB + g] += ab * x[c] / r;
      }
    }
  } else if (vabs > 0.0) {
    for (int c = 0; c < 3; ++c) D.vb[c * NB + g] += rcb * P.n2 * tau_abs * v[c] / vabs;
  }
}

// Output conversion VJP (v_h = v_b + P/m0) and input conversion VJP (v_b = v_h - sum m v_h / M)
// with the AoS user layout.
__global__ void k_ad_out_vjp(Sim S, AdjDev D, const double *xbar, const double *vbar) {
  __shared__ double red[3][128];
  const int b = blockIdx.x, tid = threadIdx.x, NB = D.NB;
  double s[3] = {0.0, 0.0, 0.0};
  for (int i = tid; i < D.N; i += blockDim.x)
    for (int c = 0; c < 3; ++c) s[c] += vbar[(b * D.N + i) * 3 + c];
  for (int c = 0; c < 3; ++c) red[c][tid] = s[c];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (tid < o)
      for (int c = 0; c < 3; ++c) red[c][tid] += red[c][tid + o];
    __syncthreads();
  }
  const double im0 = 1.0 / D.m0[b];
  for (int i = tid; i < D.Np; i += blockDim.x) {
    const int g = b * D.Np + i;
    double dm = 0.0;
    for (int c = 0; c < 3; ++c) {
      if (i < D.N) {
        D.xb[c * NB + g] = xbar[(b * D.N + i) * 3 + c];
        D.vb[c * NB + g] = fma(S.m[g] * im0, red[c][0], vbar[(b * D.N + i) * 3 + c]);
        dm = fma(S.v[c * NB + g], red[c][0], dm);
      } else {
        D.xb[c * NB + g] = 0.0; D.vb[c * NB + g] = 0.0;
      }
    }
    D.mb[g] = i < D.N ? dm * im0 : 0.0;
    D.rcb[g] = 0.0;
  }
}

__global__ void k_ad_in_vjp(AdjDev D, const double *m, const double *vh, double *gx, double *gv, double *gm) {
  __shared__ double red[7][128];
  const int b = blockIdx.x, tid = threadIdx.x, NB = D.NB;
  double s[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = tid; i < D.N; i += blockDim.x) {
    const int g = b * D.Np + i;
    const double mi = m[b * D.N + i];
    for (int c = 0; c < 3; ++c) {
      s[c] += D.vb[c * NB + g];
      s[3 + c] = fma(mi, vh[(b * D.N + i) * 3 + c], s[3 + c]);
    }
    s[6] += mi;
  }
  for (int c = 0; c < 7; ++c) red[c][tid] = s[c];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (tid < o)
      for (int c = 0; c < 7; ++c) red[c][tid] += red[c][tid + o];
    __syncthreads();
  }
  const double M = D.m0[b] + red[6][0];
  const double Sb[3] = {red[0][0], red[1][0], red[2][0]};
  const double vcm[3] = {red[3][0] / M, red[4][0] / M, red[5][0] / M};
  for (int i = tid; i < D.N; i += blockDim.x) {
    const int g = b * D.Np + i, u = b * D.N + i;
    const double mi = m[u];
    double dm = 0.0;
    for (int c = 0; c < 3; ++c) {
      gx[u * 3 + c] = D.xb[c * NB + g];
      gv[u * 3 + c] = D.vb[c * NB + g] - (mi / M) * Sb[c];
      dm -= Sb[c] * (vh[u * 3 + c] - vcm[c]) / M;
    }
    gm[u] = D.mb[g] + dm;
  }
}

int num_sms_adj() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

void init_dstumpff() {
  double t[4][DST_TERMS];
  for (int k = 0; k < 4; ++k)
    for (int m = 0; m < DST_TERMS; ++m) {
      long double fact = 1.0L;
      for (int q = 2; q <= 2 * m + 2 + k; ++q) fact *= (long double)q;
      t[k][m] = (double)((long double)(m + 1) / fact);
    }
  cudaMemcpyToSymbol(c_dst, t, sizeof(t));
}

void init_lambda() {
  double lam[BS_LEVELS + 1][BS_LEVELS + 1] = {};
  for (int k = 1; k <= BS_LEVELS; ++k)
    for (int l = 1; l <= k; ++l) {  // tableau on the unit vector e_l
      double T[BS_LEVELS + 1][BS_LEVELS + 1] = {};
      T[l][1] = 1.0;
      for (int kk = 2; kk <= k; ++kk)
        for (int j = 1; j < kk; ++j) {
          const double ratio = (double)kk / (double)(kk - j);
          T[kk][j + 1] = T[kk][j] + (T[kk][j] - T[kk - 1][j]) / (ratio * ratio - 1.0);
        }
      lam[k][l] = T[k][k];
    }
  cudaMemcpyToSymbol(c_lambda, lam, sizeof(lam));
}

}  // namespace genga

using namespace genga;

// ---------------------------------------------------------------------------------------------
// Context and C ABI
// ---------------------------------------------------------------------------------------------
struct genga_adj {
  int B, N, Np, NB, order, nsub, K;
  double G, dt, w[7];
  genga_params prm;
  DevParams P;
  Sim S;
  AdjDev D;
  std::vector<void *> allocs;
  cudaStream_t stream = nullptr;
  double *m0 = nullptr, *rc_prev = nullptr;
  // inputs of the last forward
  double *in_x = nullptr, *in_v = nullptr, *in_m = nullptr;
  int nsteps = 0, nck_alloc = 0;
  double *ck = nullptr;  // checkpoints: [nck][7 NB] = x, v, rc_prev
  // recording of one segment: per substep SubRec, per step rc and step-start v
  double *rec = nullptr, *rec_step = nullptr;
  int *grec = nullptr;
  double2 *seq_pool = nullptr;
  int *seq_count = nullptr, seq_cap = 0;
  double *y_pool = nullptr, *y_scratch = nullptr;
  long long *y_count = nullptr, *yoff_rec = nullptr;
  int bs_blocks = 0, bs_fwd_grid = 0;
  double *kv_part = nullptr;  // kick tile partials: VJP [B][T][T][5][32], forward [B][T][T][3][32]
  // the reverse sweep's branches: the Kepler-drift VJP and the large-group BS VJP beside the
  // small-group BS VJP (they touch disjoint bodies)
  cudaStream_t side = nullptr, side2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
};

namespace {

template <class T>
T *dalloc(genga_adj *c, size_t n, cudaError_t &err) {
  void *p = nullptr;
  if (err == cudaSuccess) err = cudaMalloc(&p, (n ? n : 1) * sizeof(T));
  if (err == cudaSuccess) { c->allocs.push_back(p); cudaMemset(p, 0, (n ? n : 1) * sizeof(T)); }
  return (T *)p;
}

SubRec subrec(genga_adj *c, int slot) {
  const size_t NB = c->NB;
  double *r = c->rec + (size_t)slot * 16 * NB;
  int *gi = c->grec + (size_t)slot * (4 * NB + 2);
  SubRec R;
  R.x = r; R.v1 = r + 3 * NB; R.x1 = r + 6 * NB; R.v2 = r + 9 * NB; R.x3 = r + 12 * NB; R.s = r + 15 * NB;
  R.gstart = gi; R.gsize = gi + NB; R.gmem = gi + 2 * NB; R.seq_off = gi + 3 * NB;
  R.ngroups = gi + 4 * NB; R.seq_len = nullptr;
  R.y_off = c->yoff_rec + (size_t)slot * NB;
  return R;
}

// seq_len lives after the group record block of each substep
int *seq_len_of(genga_adj *c, int slot) { return c->grec + (size_t)c->K * c->nsub * (4 * c->NB + 2) + (size_t)slot * c->NB; }

void launch_kick(genga_adj *c, int mode, double h, double *rec_x) {
  const int T = c->Np / 32, items = c->B * T * (T + 1) / 2;
  const int grid = (items * 32 + 127) / 128;
  if (mode == 2) { k_ad_kick_sym<2><<<grid, 128, 0, c->stream>>>(c->S, c->D, c->kv_part); return; }
  if (mode == 0) k_ad_kick_sym<0><<<grid, 128, 0, c->stream>>>(c->S, c->D, c->kv_part);
  else k_ad_kick_sym<1><<<grid, 128, 0, c->stream>>>(c->S, c->D, c->kv_part);
  k_ad_kick_fin<<<(c->NB + 127) / 128, 128, 0, c->stream>>>(c->S, c->D, h, c->kv_part, rec_x);
}

void launch_kick_vjp(genga_adj *c, double h, const double *xk) {
  const int T = c->Np / 32, items = c->B * T * (T + 1) / 2;
  k_ad_kick_vjp_sym<<<(items * 32 + 127) / 128, 128, 0, c->stream>>>(c->S, c->D, h, xk, c->kv_part);
  k_ad_kick_vjp_reduce<<<(c->NB + 127) / 128, 128, 0, c->stream>>>(c->S, c->D, c->kv_part);
}

// One full step t. With slot >= 0 the step is recorded into segment slot `slot`.
int run_step(genga_adj *c, int slot) {
  cudaStream_t st = c->stream;
  const int NB = c->NB;
  const double tau_abs = std::fabs(c->dt);
  double *rrc = slot >= 0 ? c->rec_step + (size_t)slot * 4 * NB : nullptr;
  double *rv = slot >= 0 ? rrc + NB : nullptr;
  k_ad_rcrit<<<(NB + 127) / 128, 128, 0, st>>>(c->S, c->D, c->P, tau_abs, nullptr, rrc, rv);
  for (int j = 0; j < c->nsub; ++j) {
    const double tau = c->w[j] * c->dt, h = 0.5 * tau;
    SubRec R{};
    Sim S = c->S;
    if (slot >= 0) {
      const int sl = slot * c->nsub + j;
      R = subrec(c, sl);
      R.seq_len = seq_len_of(c, sl);
      S.gstart = R.gstart; S.gsize = R.gsize; S.gmem = R.gmem; S.ngroups = R.ngroups;
      S.seq_off = R.seq_off; S.seq_len = R.seq_len; S.y_off = R.y_off;
    }
    if (cudaMemsetAsync(S.ngroups, 0, sizeof(int), st) != cudaSuccess) return GENGA_ECUDA;
    if (cudaMemsetAsync(S.gtotal, 0, sizeof(int), st) != cudaSuccess) return GENGA_ECUDA;
    launch_kick(c, 0, h, R.x);
    k_ad_sundrift<<<c->B, 256, 0, st>>>(S, c->D, h, R.v1, R.x1);
    k_ad_kepler<<<(NB + 127) / 128, 128, 0, st>>>(S, c->D, c->P, tau, R.s);
    k_ad_group<<<c->B, 256, 0, st>>>(S, c->D, tau);
    launch_bs(S, c->P, tau, c->bs_fwd_grid, st);
    k_ad_sundrift<<<c->B, 256, 0, st>>>(S, c->D, h, R.v2, R.x3);
    launch_kick(c, 1, h, nullptr);
  }
  return cudaGetLastError() == cudaSuccess ? GENGA_OK : GENGA_ECUDA;
}

// Restore checkpoint ck (x, v, rc_prev) and rebuild the candidate lists with rc_prev.
void restore(genga_adj *c, int ck) {
  const size_t NB = c->NB;
  const double *src = c->ck + (size_t)ck * 7 * NB;
  cudaMemcpyAsync(c->S.x, src, 3 * NB * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(c->S.v, src + 3 * NB, 3 * NB * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemsetAsync(c->D.ccount, 0, c->B * sizeof(int), c->stream);
  k_ad_rcrit<<<(c->NB + 127) / 128, 128, 0, c->stream>>>(c->S, c->D, c->P, std::fabs(c->dt), src + 6 * NB, nullptr,
                                                          nullptr);
  launch_kick(c, 2, 0.0, nullptr);
}

void save_ck(genga_adj *c, int ck, const double *rcp) {
  const size_t NB = c->NB;
  double *dst = c->ck + (size_t)ck * 7 * NB;
  cudaMemcpyAsync(dst, c->S.x, 3 * NB * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(dst + 3 * NB, c->S.v, 3 * NB * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(dst + 6 * NB, rcp, NB * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
}

int substep_w(int order, double *w) {
  if (order == 4) {
    const double cb = cbrt(2.0);
    w[0] = w[2] = 1.0 / (2.0 - cb);
    w[1] = -cb / (2.0 - cb);
    return 3;
  }
  if (order == 6) {
    const double w1 = -1.17767998417887, w2 = 0.235573213359357, w3 = 0.784513610477560;
    const double w0 = 1.0 - 2.0 * (w1 + w2 + w3);
    const double s[7] = {w3, w2, w1, w0, w1, w2, w3};
    for (int k = 0; k < 7; ++k) w[k] = s[k];
    return 7;
  }
  w[0] = 1.0;
  return 1;
}

}  // namespace

extern "C" {

int genga_adj_init(genga_adj **out, int n_sys, int n, const double *m0, double G, double dt, int order,
                   int ckpt_every) {
  if (!out) return GENGA_EINVAL;
  *out = nullptr;
  if (n_sys < 1 || n < 1 || n > AD_MAXN || !m0 || !(G > 0.0) || !std::isfinite(dt) || dt == 0.0 ||
      (order != 2 && order != 4 && order != 6) || ckpt_every < 1)
    return GENGA_EINVAL;
  for (int b = 0; b < n_sys; ++b)
    if (!(m0[b] > 0.0) || !std::isfinite(m0[b])) return GENGA_EINVAL;
  genga_adj *c = new genga_adj();
  c->B = n_sys; c->N = n; c->Np = ((n + 31) / 32) * 32; c->NB = c->B * c->Np;
  c->order = order; c->nsub = substep_w(order, c->w); c->K = ckpt_every;
  c->G = G; c->dt = dt;
  genga_default_params(&c->prm);
  c->prm.collisions = 0;
  c->prm.kmode = 0;
  memset(&c->P, 0, sizeof(c->P));
  c->P.G = G; c->P.m0 = 1.0; c->P.Gm0 = G; c->P.inv_m0 = 1.0; c->P.mu2 = 2.0 * G; c->P.inv_mu = 1.0 / G;
  c->P.n1 = c->prm.n1; c->P.n2 = c->prm.n2; c->P.pc = c->prm.pc; c->P.bs_eps = c->prm.bs_eps;
  c->P.bs_kmax = c->prm.bs_kmax; c->P.bs_max_halvings = c->prm.bs_max_halvings;
  c->P.kepler_maxit = c->prm.kepler_maxit; c->P.kmode = 0; c->P.collisions = 0;
  c->stream = nullptr;  // the CUDA default stream until genga_adj_set_stream
  cudaError_t err = cudaSuccess;
  const size_t NB = c->NB;
  Sim &S = c->S;
  memset(&S, 0, sizeof(S));
  S.n = (int)NB; S.npad = (int)NB;
  S.x = dalloc<double>(c, 3 * NB, err); S.v = dalloc<double>(c, 3 * NB, err);
  S.x0 = dalloc<double>(c, 3 * NB, err); S.v0 = dalloc<double>(c, 3 * NB, err);
  S.m = dalloc<double>(c, NB, err); S.gm = dalloc<double>(c, NB, err); S.R = dalloc<double>(c, NB, err);
  S.hill = dalloc<double>(c, NB, err); S.alive = dalloc<int>(c, NB, err);
  S.rc = dalloc<double>(c, NB, err); S.A = dalloc<double>(c, NB, err);
  S.T = dalloc<u64>(c, NB, err); S.rcsq = dalloc<u64>(c, NB, err);
  S.gstart = dalloc<int>(c, NB, err); S.gsize = dalloc<int>(c, NB, err); S.gmem = dalloc<int>(c, NB, err);
  S.ngroups = dalloc<int>(c, 1, err); S.gtotal = dalloc<int>(c, 1, err);
  S.sys_of = dalloc<int>(c, NB, err); S.sys_m0 = dalloc<double>(c, c->B, err);
  S.status = dalloc<int>(c, 1, err); S.counters = dalloc<long long>(c, NCOUNTERS, err); S.U = dalloc<double>(c, 1, err);
  S.nsys = c->B;
  AdjDev &D = c->D;
  D.B = c->B; D.N = n; D.Np = c->Np; D.NB = (int)NB; D.G = G; D.dt = dt;
  D.m0 = S.sys_m0;
  D.ccap = n * (n - 1) / 2 + 1;
  D.cand = dalloc<int>(c, (size_t)c->B * D.ccap, err); D.ccount = dalloc<int>(c, c->B, err);
  D.P = dalloc<double>(c, 3 * c->B, err);
  D.fail = dalloc<int>(c, NB, err); D.ingrp = dalloc<int>(c, NB, err);
  D.xb = dalloc<double>(c, 3 * NB, err); D.vb = dalloc<double>(c, 3 * NB, err);
  D.mb = dalloc<double>(c, NB, err); D.rcb = dalloc<double>(c, NB, err);
  c->rc_prev = dalloc<double>(c, NB, err);
  c->in_x = dalloc<double>(c, 3 * (size_t)c->B * n, err); c->in_v = dalloc<double>(c, 3 * (size_t)c->B * n, err);
  c->in_m = dalloc<double>(c, (size_t)c->B * n, err);
  // segment recording
  const size_t nslot = (size_t)c->K * c->nsub;
  c->rec = dalloc<double>(c, nslot * 16 * NB, err);
  c->rec_step = dalloc<double>(c, (size_t)c->K * 4 * NB, err);
  c->grec = dalloc<int>(c, nslot * (4 * NB + 2) + nslot * NB, err);
  c->seq_cap = (int)std::min<size_t>(nslot * NB * 8 + 1024, (size_t)1 << 26);
  c->seq_pool = dalloc<double2>(c, c->seq_cap, err);
  c->seq_count = dalloc<int>(c, 1, err);
  c->kv_part = dalloc<double>(c, (size_t)c->B * (c->Np / 32) * (c->Np / 32) * 160, err);
  c->bs_blocks = num_sms_adj();
  c->bs_fwd_grid = 2 * c->B > 64 ? 2 * c->B : 64;
  c->y_scratch = dalloc<double>(c, (size_t)c->bs_fwd_grid * BS_SEQCAP * BS_GMAX * 6, err);
  c->y_pool = dalloc<double>(c, (size_t)1 << 24, err);
  c->y_count = dalloc<long long>(c, 1, err);
  c->yoff_rec = dalloc<long long>(c, nslot * NB, err);
  if (err != cudaSuccess) { genga_adj_free(c); return GENGA_ENOMEM; }
  S.seq_pool = c->seq_pool; S.seq_count = c->seq_count; S.seq_cap = c->seq_cap;
  S.y_pool = c->y_pool; S.y_scratch = c->y_scratch; S.y_count = c->y_count; S.y_cap = (long long)1 << 24;
  std::vector<int> sys(NB);
  for (size_t g = 0; g < NB; ++g) sys[g] = (int)(g / c->Np);
  cudaMemcpy(S.sys_of, sys.data(), NB * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(S.sys_m0, m0, c->B * sizeof(double), cudaMemcpyHostToDevice);
  cudaFuncSetAttribute(k_ad_bs_vjp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(BSV_WARPS * sizeof(LevShared)));
  cudaFuncSetAttribute(k_ad_bs_vjp4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(BSV4_GROUPS * sizeof(GrpVjp4)));
  bs_init_constants();
  init_lambda();
  init_dstumpff();
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming) != cudaSuccess) {
    genga_adj_free(c);
    return GENGA_ECUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) { genga_adj_free(c); return GENGA_ECUDA; }
  *out = c;
  return GENGA_OK;
}

int genga_adj_set_stream(genga_adj *c, void *stream) {
  if (!c) return GENGA_EINVAL;
  c->stream = (cudaStream_t)stream;  // NULL: the CUDA default stream
  return GENGA_OK;
}

int genga_adj_forward(genga_adj *c, int n_steps, const double *x, const double *v, const double *m, double *x_out,
                      double *v_out) {
  if (!c || n_steps < 0 || !x || !v || !m || !x_out || !v_out) return GENGA_EINVAL;
  cudaStream_t st = c->stream;
  const size_t NB = c->NB, nin = (size_t)c->B * c->N;
  const int nck = n_steps / c->K + 1;
  if (nck > c->nck_alloc) {
    cudaError_t err = cudaSuccess;
    c->ck = dalloc<double>(c, (size_t)nck * 7 * NB, err);
    if (err != cudaSuccess) return GENGA_ENOMEM;
    c->nck_alloc = nck;
  }
  if (cudaMemcpyAsync(c->in_x, x, 3 * nin * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->in_v, v, 3 * nin * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->in_m, m, nin * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return GENGA_ECUDA;
  cudaMemsetAsync(c->S.status, 0, sizeof(int), st);
  k_ad_setup<<<c->B, 128, 0, st>>>(c->S, c->D, c->in_x, c->in_v, c->in_m);
  // first prechecker: radii of the initial state
  cudaMemsetAsync(c->D.ccount, 0, c->B * sizeof(int), st);
  k_ad_rcrit<<<(NB + 127) / 128, 128, 0, st>>>(c->S, c->D, c->P, std::fabs(c->dt), nullptr, c->rc_prev, nullptr);
  launch_kick(c, 2, 0.0, nullptr);
  c->nsteps = n_steps;
  for (int t = 0; t < n_steps; ++t) {
    if (t % c->K == 0) save_ck(c, t / c->K, c->rc_prev);
    const int rc = run_step(c, -1);
    if (rc != GENGA_OK) return rc;
    cudaMemcpyAsync(c->rc_prev, c->S.rc, NB * sizeof(double), cudaMemcpyDeviceToDevice, st);
  }
  k_ad_output<<<c->B, 128, 0, st>>>(c->S, c->D, x_out, v_out);
  return cudaGetLastError() == cudaSuccess ? GENGA_OK : GENGA_ECUDA;
}

int genga_adj_backward(genga_adj *c, const double *xbar, const double *vbar, double *gx, double *gv, double *gm) {
  if (!c || !xbar || !vbar || !gx || !gv || !gm) return GENGA_EINVAL;
  cudaStream_t st = c->stream;
  const size_t NB = c->NB;
  const double tau_abs = std::fabs(c->dt);
  // the state still holds the forward's final state: output conversion VJP
  k_ad_out_vjp<<<c->B, 128, 0, st>>>(c->S, c->D, xbar, vbar);
  const int nseg = (c->nsteps + c->K - 1) / c->K;
  for (int sgm = nseg - 1; sgm >= 0; --sgm) {
    const int t0 = sgm * c->K, t1 = std::min(t0 + c->K, c->nsteps);
    restore(c, sgm);
    cudaMemsetAsync(c->seq_count, 0, sizeof(int), st);
    cudaMemsetAsync(c->y_count, 0, sizeof(long long), st);
    for (int t = t0; t < t1; ++t) {
      const int rc = run_step(c, t - t0);
      if (rc != GENGA_OK) return rc;
    }
    for (int t = t1 - 1; t >= t0; --t) {
      const int slot = t - t0;
      for (int j = c->nsub - 1; j >= 0; --j) {
        const double tau = c->w[j] * c->dt, h = 0.5 * tau;
        const int sl = slot * c->nsub + j;
        SubRec R = subrec(c, sl);
        R.seq_len = seq_len_of(c, sl);
        // the step's critical radii (and derived A, rcsq) are needed by the kick and BS VJPs
        if (j == c->nsub - 1)
          k_ad_rcrit<<<(NB + 127) / 128, 128, 0, st>>>(c->S, c->D, c->P, tau_abs, c->rec_step + (size_t)slot * 4 * NB,
                                                        nullptr, nullptr);
        launch_kick_vjp(c, h, R.x3);
        k_ad_sundrift_vjp<<<c->B, 256, 0, st>>>(c->S, c->D, h, R.v2);
        // fork: the small-group BS VJP (the longest) here, the Kepler-drift VJP of the bodies outside
        // groups and the large-group BS VJP beside it; join
        cudaEventRecord(c->ev_fork, st);
        cudaStreamWaitEvent(c->side, c->ev_fork, 0);
        cudaStreamWaitEvent(c->side2, c->ev_fork, 0);
        k_ad_bs_vjp4<<<2 * c->bs_blocks, 32 * BSV4_GROUPS, BSV4_GROUPS * sizeof(GrpVjp4), st>>>(c->S, c->D, R, R.x1,
                                                                                               R.v1);
        cudaMemsetAsync(c->D.ingrp, 0, NB * sizeof(int), c->side);
        k_ad_mark<<<c->bs_blocks, 32, 0, c->side>>>(c->D, R.gstart, R.gsize, R.gmem, R.ngroups);
        k_ad_kepler_vjp<<<(NB + 127) / 128, 128, 0, c->side>>>(c->S, c->D, tau, R.x1, R.v1, R.s);
        k_ad_bs_vjp<<<c->bs_blocks, 32 * BSV_WARPS, BSV_WARPS * sizeof(LevShared), c->side2>>>(c->S, c->D, R, R.x1,
                                                                                               R.v1);
        cudaEventRecord(c->ev_join, c->side);
        cudaEventRecord(c->ev_join2, c->side2);
        cudaStreamWaitEvent(st, c->ev_join, 0);
        cudaStreamWaitEvent(st, c->ev_join2, 0);
        k_ad_sundrift_vjp<<<c->B, 256, 0, st>>>(c->S, c->D, h, R.v1);
        launch_kick_vjp(c, h, R.x);
      }
      const double *rstep = c->rec_step + (size_t)slot * 4 * NB;
      const SubRec R0 = subrec(c, slot * c->nsub);
      k_ad_rcrit_vjp<<<(NB + 127) / 128, 128, 0, st>>>(c->S, c->D, c->P, tau_abs, R0.x, rstep + NB);
    }
  }
  k_ad_in_vjp<<<c->B, 128, 0, st>>>(c->D, c->in_m, c->in_v, gx, gv, gm);
  return cudaGetLastError() == cudaSuccess ? GENGA_OK : GENGA_ECUDA;
}

int genga_adj_status(genga_adj *c, int *code) {
  if (!c || !code) return GENGA_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return GENGA_ECUDA;
  if (cudaMemcpy(code, c->S.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GENGA_ECUDA;
  return GENGA_OK;
}

int genga_adj_sync(genga_adj *c) {
  if (!c) return GENGA_EINVAL;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? GENGA_OK : GENGA_ECUDA;
}

void genga_adj_free(genga_adj *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_join2) cudaEventDestroy(c->ev_join2);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->side2) cudaStreamDestroy(c->side2);
  for (void *p : c->allocs) cudaFree(p);
  delete c;
}

}  // extern "C"
