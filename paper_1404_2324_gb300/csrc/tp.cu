// tp.cu -- test-particle mode (Sect. 3.3): up to 32 massive bodies (integrated by the
// single-system kernels) plus massless test particles (TPs) that they perturb.
//
// One thread per TP for the kick (K-weighted, prechecker against every planet, planets staged in
// shared memory), the Sun drift with the massive momentum and the Kepler drift; one lane per
// candidate (TP, planet) pair for the Hermite test. A TP with a confirmed planet encounter (or a
// failed Kepler solve) is integrated alone by Bulirsch-Stoer on one warp (levels on lanes 0..7,
// the tableau on lanes 8..13) in the field of m0 and the (1 - K) pull of the encountered planets,
// which move on their Kepler paths from the pre-drift state (Sect. 3.3: only the test particle is
// updated). The planets' positions at every midpoint time of a full-length BS attempt come from a
// table computed once per substep; shorter attempts evaluate the polynomial through 16 Kepler
// solutions at the Chebyshev nodes of each planet's path (or solve Kepler's equation where that
// polynomial is not admitted) and attempt H/2 on lanes 16..29 beside H. Particles in the deepest
// encounters are integrated first, each alone on its SM sub-partition. A TP whose BS substep
// reaches a planet's surface is removed.
#include <cmath>
#include <cstring>

#include "genga_launch.h"

namespace genga {

__device__ __forceinline__ int tab_index(int k, int m) { return k * k - 1 + m; }  // level k >= 1, m = 0..2k

// Critical radii of the TPs (Eq. rcrit with m = 0: n2 |tau| |v|) and the per-TP reuse test.
__global__ void k_tp_rcrit(TPSet T, DevParams P, double tau_abs, int check_reuse) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T.n) return;
  if (!T.alive[i]) { T.rc[i] = 0.0; T.A[i] = 0.0; T.T[i] = 0ULL; T.rcsq[i] = 0ULL; return; }
  const int np = T.npad;
  const double vx = T.v[i], vy = T.v[np + i], vz = T.v[2 * np + i];
  const double v2 = fma(vz, vz, fma(vy, vy, vx * vx));
  const double vabs = (dbits(v2) == 0ULL) ? 0.0 : v2 * rsqrt_refined(v2);
  const double rc = (P.n2 * tau_abs) * vabs;
  T.full[i] = check_reuse && dbits(rc) > dbits(P.pc * T.rc[i]);
  T.rc[i] = rc;
  const double t = __dmul_rn(P.pc, rc);
  T.T[i] = dbits(__dmul_rn(t, t));
  T.rcsq[i] = dbits(__dmul_rn(rc, rc));
  T.A[i] = (dbits(rc) == 0ULL) ? 0.0 : rcp_refined(0.9 * rc);
}

struct PlanetSm {
  double x[TP_MAXPL], y[TP_MAXPL], z[TP_MAXPL], gm[TP_MAXPL], A[TP_MAXPL];
  u64 T[TP_MAXPL], Q[TP_MAXPL];
  int alive[TP_MAXPL];
};

__device__ void load_planets(const Sim &S, PlanetSm &ps) {
  const int np = S.npad;
  for (int j = threadIdx.x; j < TP_MAXPL; j += blockDim.x) {
    const bool ok = j < S.n && S.alive[j];
    ps.alive[j] = ok;
    ps.x[j] = ok ? S.x[j] : 0.0; ps.y[j] = ok ? S.x[np + j] : 0.0; ps.z[j] = ok ? S.x[2 * np + j] : 0.0;
    ps.gm[j] = ok ? S.gm[j] : 0.0; ps.A[j] = ok ? S.A[j] : 0.0;
    ps.T[j] = ok ? S.T[j] : 0ULL; ps.Q[j] = ok ? S.rcsq[j] : 0ULL;
  }
  __syncthreads();
}

// The closing (or first) kick's forces on K TPs at once (independent FP64 chains for the pipe), TP
// i[k] at x[k], every planet in order, prechecked: pairs outside the precheck threshold add to the
// far field, candidates (with the changeover weight inside rc) to the near field. For each active TP
// stores the far field and the candidate mask for the next step's opening kick; returns the masks
// in cm, the total accelerations in acc.
template <int K>
__device__ __forceinline__ void tp_close_forces_k(const TPSet &T, const DevParams &P, const PlanetSm &ps, int npl,
                                                  const int (&i)[K], const bool (&act)[K], const double (&x)[K][3],
                                                  double (&acc)[K][3], unsigned (&cm)[K]) {
  const int np = T.npad;
  u64 Ti[K], Qi[K];
  double Ai[K], f[K][3], n[K][3];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    Ti[k] = act[k] ? T.T[i[k]] : 0ULL;
    Qi[k] = act[k] ? T.rcsq[i[k]] : 0ULL;
    Ai[k] = act[k] ? T.A[i[k]] : 0.0;
    cm[k] = 0u;
    for (int c = 0; c < 3; ++c) f[k][c] = n[k][c] = 0.0;
  }
  for (int j = 0; j < npl; ++j) {
    if (!ps.alive[j]) continue;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double dx = ps.x[j] - x[k][0], dy = ps.y[j] - x[k][1], dz = ps.z[j] - x[k][2];
      const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
      const u64 rb = dbits(r2);
      double g = ps.gm[j] * rcube_refined(r2);
      if (rb < umax64(Ti[k], ps.T[j])) {
        if (rb < umax64(Qi[k], ps.Q[j])) {  // inside the changeover zone (rare): the weight needs r
          double wB, wA;
          changeover_w(r2 * rsqrt_refined(r2), pmin(Ai[k], ps.A[j]), P.kmode, wB, wA);
          g *= wB;
        }
        cm[k] |= 1u << j;
        n[k][0] = fma(g, dx, n[k][0]); n[k][1] = fma(g, dy, n[k][1]); n[k][2] = fma(g, dz, n[k][2]);
      } else {
        f[k][0] = fma(g, dx, f[k][0]); f[k][1] = fma(g, dy, f[k][1]); f[k][2] = fma(g, dz, f[k][2]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!act[k]) { cm[k] = 0u; continue; }
    T.afar[i[k]] = f[k][0]; T.afar[np + i[k]] = f[k][1]; T.afar[2 * np + i[k]] = f[k][2];
    T.cmask[i[k]] = cm[k];
    for (int c = 0; c < 3; ++c) acc[k][c] = f[k][c] + n[k][c];
  }
}

// One TP (see tp_close_forces_k); returns its mask, the acceleration in (ax, ay, az).
__device__ __forceinline__ unsigned tp_close_forces(const TPSet &T, const DevParams &P, const PlanetSm &ps, int npl,
                                                    int i, double xi, double yi, double zi, double &ax, double &ay,
                                                    double &az) {
  const int ii[1] = {i};
  const bool act[1] = {true};
  const double x[1][3] = {{xi, yi, zi}};
  double acc[1][3];
  unsigned cm[1];
  tp_close_forces_k<1>(T, P, ps, npl, ii, act, x, acc, cm);
  ax = acc[0][0]; ay = acc[0][1]; az = acc[0][2];
  return cm[0];
}

// v += (h1 + h2) a as two kicks (the closing kick of this substep and the opening kick of the next);
// after the step's last substep also the last Sun drift, x += shc (the shift moves every body
// alike, so the kick does not see it).
__device__ __forceinline__ void tp_close_update(const TPSet &T, int i, double xi, double yi, double zi, double ax,
                                                double ay, double az, double h1, double h2, const double *shc) {
  const int np = T.npad;
  double vx = fma(h1, ax, T.v[i]), vy = fma(h1, ay, T.v[np + i]), vz = fma(h1, az, T.v[2 * np + i]);
  if (h2 != 0.0) { vx = fma(h2, ax, vx); vy = fma(h2, ay, vy); vz = fma(h2, az, vz); }
  T.v[i] = vx; T.v[np + i] = vy; T.v[2 * np + i] = vz;
  if (shc) { T.x[i] = xi + shc[0]; T.x[np + i] = yi + shc[1]; T.x[2 * np + i] = zi + shc[2]; }
}

// Appends the candidate (TP, planet) pairs of the warp's lanes (lane's TP i, mask cm) to the pair
// list of the next encounter test with one atomic; counts them when the kick closes a substep.
__device__ __forceinline__ void tp_append_pairs(const TPSet &T, int i, unsigned cm, bool count) {
  const int lane = threadIdx.x & 31;
  const unsigned cnt = __popc(cm);
  unsigned incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned base = 0u;
  if (lane == 31 && total) {
    base = atomicAdd(T.npairs, total);
    if (count) atomicAdd((unsigned long long *)&T.counters[0], (unsigned long long)total);
  }
  base = __shfl_sync(0xffffffffu, base, 31);
  unsigned pos = base + incl - cnt;
  while (cm) {
    const int j = __ffs(cm) - 1;
    cm &= cm - 1;
    T.pairs[pos++] = ((unsigned)i << 5) | (unsigned)j;
  }
}

// The planets (as load_planets) and the step's last Sun drift's shift, hcm_last times the massive
// momentum before the closing kick (the per-tile partials of the massive kick), by one warp for
// itself: no block barrier.
__device__ __forceinline__ void warp_load_planets(const Sim &S, double hcm_last, PlanetSm &ps, double *shc) {
  const int lane = threadIdx.x & 31, np = S.npad;
  const bool ok = lane < S.n && S.alive[lane];
  ps.alive[lane] = ok;
  ps.x[lane] = ok ? S.x[lane] : 0.0; ps.y[lane] = ok ? S.x[np + lane] : 0.0; ps.z[lane] = ok ? S.x[2 * np + lane] : 0.0;
  ps.gm[lane] = ok ? S.gm[lane] : 0.0; ps.A[lane] = ok ? S.A[lane] : 0.0;
  ps.T[lane] = ok ? S.T[lane] : 0ULL; ps.Q[lane] = ok ? S.rcsq[lane] : 0ULL;
  if (hcm_last != 0.0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double a = 0.0;
      for (int t = lane; t < S.nt; t += 32) a += S.pkick[t * 3 + c];
      a = warp_sum(a);
      if (lane == 0) shc[c] = hcm_last * a;
    }
  }
  __syncwarp();
}

// The first kick after a new state: forces, far field and candidates of every TP (no velocity
// change). Also empties the BS list of the coming substep.
__global__ void __launch_bounds__(128) k_tp_kick(Sim S, TPSet T, DevParams P) {
  __shared__ PlanetSm ps;
  load_planets(S, ps);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) { T.nbs[0] = 0; T.nbs[1] = 0; }
  unsigned cm = 0u;
  if (i < T.n && T.alive[i]) {
    double ax, ay, az;
    cm = tp_close_forces(T, P, ps, S.n, i, T.x[i], T.x[T.npad + i], T.x[2 * T.npad + i], ax, ay, az);
  }
  tp_append_pairs(T, i, cm, false);
}

// Sun drifts with the massive momentum (the same partials the massive drift reads), keep the
// pre-drift state, Kepler drift. Clears the encounter masks; a failed solve lists the TP for BS.
__global__ void k_tp_drift(Sim S, TPSet T, DevParams P, double tau, double hcm1, double hcm2) {
  __shared__ double sh[3];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double a = 0.0, b = 0.0;
      for (int t = lane; t < S.nt; t += 32) {
        a += S.pfin[t * 3 + c];
        if (hcm2 != 0.0) b += S.pkick[t * 3 + c];
      }
      a = warp_sum(a);
      double v = hcm1 * a;
      if (hcm2 != 0.0) v = fma(hcm2, warp_sum(b), v);
      if (lane == 0) sh[c] = v;
    }
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T.n) return;
  T.fail[i] = 0;
  T.emask[i] = 0u;
  if (!T.alive[i]) return;
  const int np = T.npad;
  double x = T.x[i] + sh[0], y = T.x[np + i] + sh[1], z = T.x[2 * np + i] + sh[2];
  double vx = T.v[i], vy = T.v[np + i], vz = T.v[2 * np + i];
  T.x0[i] = x; T.x0[np + i] = y; T.x0[2 * np + i] = z;
  T.v0[i] = vx; T.v0[np + i] = vy; T.v0[2 * np + i] = vz;
  int it = 0;
  if (kepler_drift_dev(P.G * P.m0, P.mu2, x, y, z, vx, vy, vz, tau, P.kepler_maxit, &it)) {
    T.fail[i] = 1;
    atomicOr(S.status, ST_KEPLER_FALLBACK);
    T.bslist[T.npad - 1 - atomicAdd(&T.nbs[1], 1)] = i;  // BS in the field of m0 alone (unless it meets a planet)
  }
  T.x[i] = x; T.x[np + i] = y; T.x[2 * np + i] = z;
  T.v[i] = vx; T.v[np + i] = vy; T.v[2 * np + i] = vz;
}

// The start of a full step for the TPs in one pass (the operations of k_tp_rcrit with the reuse
// test, the opening kick and k_tp_drift of the first substep, in that order and arithmetic): the
// critical radius from the velocity, the opening kick (stored far field + candidates with the new
// radii, or every planet when the TP or any planet failed the reuse test), the first Sun drift with
// the momentum after the massive opening kick, the Kepler drift keeping the pre-drift state. The BS
// list is empty on entry (the last warp of the previous substep's BS pass, or the first kick,
// emptied it), so a failed solve appends to it.
__global__ void __launch_bounds__(128) k_tp_open_drift(Sim S, TPSet T, DevParams P, double tau_abs, double h1,
                                                       double tau, double hcm1) {
  __shared__ PlanetSm ps;
  __shared__ double sh[3];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double a = 0.0;
      for (int t = lane; t < S.nt; t += 32) a += S.pfin[t * 3 + c];
      a = warp_sum(a);
      if (lane == 0) sh[c] = hcm1 * a;
    }
  }
  load_planets(S, ps);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T.n) return;
  T.fail[i] = 0;
  T.emask[i] = 0u;
  if (!T.alive[i]) { T.rc[i] = 0.0; T.A[i] = 0.0; T.T[i] = 0ULL; T.rcsq[i] = 0ULL; return; }
  const int np = T.npad, npl = S.n;
  double vx = T.v[i], vy = T.v[np + i], vz = T.v[2 * np + i];
  // critical radius (Eq. rcrit, m = 0) and the reuse test
  const double v2 = fma(vz, vz, fma(vy, vy, vx * vx));
  const double vabs = (dbits(v2) == 0ULL) ? 0.0 : v2 * rsqrt_refined(v2);
  const double rc = (P.n2 * tau_abs) * vabs;
  const bool tfull = dbits(rc) > dbits(P.pc * T.rc[i]);
  const double tq = __dmul_rn(P.pc, rc);
  const u64 Qi = dbits(__dmul_rn(rc, rc));
  const double Ai = (dbits(rc) == 0ULL) ? 0.0 : rcp_refined(0.9 * rc);
  T.rc[i] = rc; T.T[i] = dbits(__dmul_rn(tq, tq)); T.rcsq[i] = Qi; T.A[i] = Ai;
  // opening kick
  double x = T.x[i], y = T.x[np + i], z = T.x[2 * np + i];
  const bool full = tfull || S.flags[0];
  double nx = 0, ny = 0, nz = 0;
  const unsigned scan = full ? 0xffffffffu : T.cmask[i];
  for (int j = 0; j < npl; ++j) {
    if (!ps.alive[j] || !((scan >> j) & 1u)) continue;
    const double dx = ps.x[j] - x, dy = ps.y[j] - y, dz = ps.z[j] - z;
    const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
    const double yr = rsqrt_refined(r2);
    double g = ps.gm[j] * (yr * yr * yr);
    if (dbits(r2) < umax64(Qi, ps.Q[j])) {
      double wB, wA;
      changeover_w(r2 * yr, pmin(Ai, ps.A[j]), P.kmode, wB, wA);
      g *= wB;
    }
    nx = fma(g, dx, nx); ny = fma(g, dy, ny); nz = fma(g, dz, nz);
  }
  double ax, ay, az;
  if (full) { ax = nx; ay = ny; az = nz; }
  else { ax = T.afar[i] + nx; ay = T.afar[np + i] + ny; az = T.afar[2 * np + i] + nz; }
  vx = fma(h1, ax, vx); vy = fma(h1, ay, vy); vz = fma(h1, az, vz);
  // Sun drift, pre-drift state, Kepler drift
  x += sh[0]; y += sh[1]; z += sh[2];
  T.x0[i] = x; T.x0[np + i] = y; T.x0[2 * np + i] = z;
  T.v0[i] = vx; T.v0[np + i] = vy; T.v0[2 * np + i] = vz;
  int it = 0;
  if (kepler_drift_dev(P.G * P.m0, P.mu2, x, y, z, vx, vy, vz, tau, P.kepler_maxit, &it)) {
    T.fail[i] = 1;
    atomicOr(S.status, ST_KEPLER_FALLBACK);
    T.bslist[T.npad - 1 - atomicAdd(&T.nbs[1], 1)] = i;  // BS in the field of m0 alone (unless it meets a planet)
  }
  T.x[i] = x; T.x[np + i] = y; T.x[2 * np + i] = z;
  T.v[i] = vx; T.v[np + i] = vy; T.v[2 * np + i] = vz;
}

// Planet paths for the TP Bulirsch-Stoer, one block per planet, from the pre-drift state:
//  * the Kepler solution at every midpoint time of a full-length attempt (t = m tau/2k, and t = tau
//    at m = 2k), also the drift result itself;
//  * a Chebyshev series in s = 2t/tau - 1 of position and velocity through TP_CHEB Kepler solutions
//    at the Chebyshev nodes, used for the times of shorter attempts. Computed coefficients carry
//    rounding noise of about 1e-16 |x| (16-term sums of values of size |x|), so no coefficient can
//    be told from zero below that floor. The series stands in for the Kepler solve (pcok = 1) when
//    coefficients 12 and 13 are within 2^-49 of |x| (resp. |v|) and the last two within 2^-48:
//    a smooth path's coefficients fall geometrically, so the truncated ones are then far below a
//    rounding, and the series reproduces the Kepler solutions to the nodes' own rounding (a few
//    1e-15 of |x|). Otherwise those times solve Kepler's equation. The polynomial is stored in
//    powers of s (Horner takes one FMA a term, Clenshaw two); pcok also asks that the power
//    coefficients' magnitudes sum to at most 2|x| (2|v|), which bounds Horner's rounding error
//    by a few roundings of the position.
__constant__ double c_cheb_pow[TP_CHEB][TP_CHEB];  // [k][q]: coefficient of s^q in T_k(s)
__device__ double d_cheb_cos[TP_CHEB][TP_CHEB];     // [k][q]: cos(pi k (2q + 1) / 2 TP_CHEB), T_k at node q

__global__ void __launch_bounds__(128) k_planet_table(Sim S, TPSet T, DevParams P, double tau) {
  __shared__ double node[TP_CHEB][6];
  __shared__ double coef[6][TP_CHEB];
  __shared__ double mono[6][TP_CHEB];
  const int j = blockIdx.x, e = threadIdx.x;
  const int np = S.npad;
  const double x0 = S.x0[j], y0 = S.x0[np + j], z0 = S.x0[2 * np + j];
  const double u0 = S.v0[j], v0 = S.v0[np + j], w0 = S.v0[2 * np + j];
  if (e < TP_TAB) {
    int k = 1;
    while (tab_index(k + 1, 0) <= e) k++;
    const int m = e - tab_index(k, 0), nk = 2 * k;
    const double t = (m == nk) ? tau : (double)m * __ddiv_rn(tau, (double)nk);
    double x = x0, y = y0, z = z0, vx = u0, vy = v0, vz = w0;
    if (m > 0) kepler_drift_dev(P.G * P.m0, P.mu2, x, y, z, vx, vy, vz, t, P.kepler_maxit, nullptr);
    double *o = T.ptab + ((size_t)j * TP_TAB + e) * 6;
    o[0] = x; o[1] = y; o[2] = z; o[3] = vx; o[4] = vy; o[5] = vz;
  } else if (e < TP_TAB + TP_CHEB) {
    const int q = e - TP_TAB;
    const double sq = cospi((double)(2 * q + 1) / (double)(2 * TP_CHEB));
    const double t = 0.5 * tau * (sq + 1.0);
    double x = x0, y = y0, z = z0, vx = u0, vy = v0, vz = w0;
    int bad = kepler_drift_dev(P.G * P.m0, P.mu2, x, y, z, vx, vy, vz, t, P.kepler_maxit, nullptr);
    node[q][0] = x; node[q][1] = y; node[q][2] = z;
    node[q][3] = bad ? __longlong_as_double(0x7ff8000000000000LL) : vx; node[q][4] = vy; node[q][5] = vz;
  }
  __syncthreads();
  if (e < 6 * TP_CHEB) {
    const int c = e / TP_CHEB, k = e % TP_CHEB;
    double acc = 0.0;
    for (int q = 0; q < TP_CHEB; ++q) acc = fma(node[q][c], d_cheb_cos[k][q], acc);
    acc *= 2.0 / TP_CHEB;
    coef[c][k] = acc;
  }
  __syncthreads();
  if (e < 6 * TP_CHEB) {  // c_0 / 2 + sum_k c_k T_k(s) in powers of s, the small terms summed first
    const int c = e / TP_CHEB, q = e % TP_CHEB;
    double a = 0.0;
    for (int k = TP_CHEB - 1; k >= q; --k) a = fma(k == 0 ? 0.5 * coef[c][0] : coef[c][k], c_cheb_pow[k][q], a);
    mono[c][q] = a;
    T.ppoly[((size_t)j * 6 + c) * TP_CHEB + q] = a;
  }
  __syncthreads();
  int ok = 1;
  if (e < 6) {  // one component per thread
    const int c = e;
    const double r = sqrt(fma(z0, z0, fma(y0, y0, x0 * x0))), v = sqrt(fma(w0, w0, fma(v0, v0, u0 * u0)));
    const double lim = 1.7763568394002505e-15;  // 2^-49
    const double decay = pmax(fabs(coef[c][TP_CHEB - 4]), fabs(coef[c][TP_CHEB - 3]));
    const double tail = fabs(coef[c][TP_CHEB - 1]) + fabs(coef[c][TP_CHEB - 2]);
    double sum = 0.0;
    for (int q = 0; q < TP_CHEB; ++q) sum += fabs(mono[c][q]);
    const double scale = c < 3 ? r : v;
    // NaN (a failed node) fails every comparison
    if (!(decay <= lim * scale) || !(tail <= 2.0 * lim * scale) || !(sum <= 2.0 * scale)) ok = 0;
  }
  ok = __syncthreads_and(ok);
  if (e == 0) T.pcok[j] = ok;
}

// Hermite test of each candidate (TP, planet) pair of the last closing kick over the drift,
// one pair per thread (bit-exact with the oracle). A TP's first encounter lists it for BS, unless
// its failed Kepler solve listed it already.
__global__ void __launch_bounds__(256) k_tp_encounter(Sim S, TPSet T, double tau) {
  __shared__ int s_last;
  const unsigned npairs = *T.npairs;
  const int np = T.npad, pp = S.npad;
  if (blockIdx.x == 0 && threadIdx.x == 0) { T.bsnext[0] = 0u; T.bsnext[1] = 0u; }  // the BS pass starts at the heads
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += gridDim.x * blockDim.x) {
    const unsigned pr = T.pairs[q];
    const int i = (int)(pr >> 5), j = (int)(pr & 31u);
    if (!T.alive[i] || !S.alive[j]) continue;
    const double *pf = T.ptab + ((size_t)j * TP_TAB + tab_index(1, 2)) * 6;  // t = tau
    const double rcij = pmax(T.rc[i], S.rc[j]);
    const double thr = __dmul_rn(rcij, rcij);
    const double dmin = hermite_min_capped(
        __dsub_rn(S.x0[j], T.x0[i]), __dsub_rn(S.x0[pp + j], T.x0[np + i]), __dsub_rn(S.x0[2 * pp + j], T.x0[2 * np + i]),
        __dsub_rn(S.v0[j], T.v0[i]), __dsub_rn(S.v0[pp + j], T.v0[np + i]), __dsub_rn(S.v0[2 * pp + j], T.v0[2 * np + i]),
        __dsub_rn(pf[0], T.x[i]), __dsub_rn(pf[1], T.x[np + i]), __dsub_rn(pf[2], T.x[2 * np + i]),
        __dsub_rn(pf[3], T.v[i]), __dsub_rn(pf[4], T.v[np + i]), __dsub_rn(pf[5], T.v[2 * np + i]), tau, thr);
    if (dmin < thr) {
      const unsigned old = atomicOr(&T.emask[i], 1u << j);
      atomicAdd((unsigned long long *)&T.counters[1], 1ULL);
      // a pass inside a tenth of the critical radius (the planet's pull entirely in BS) needs the
      // most substeps: such particles go to the front of the list, so they start first
      if (old == 0u && !T.fail[i]) {
        if (dmin < 0.01 * __dmul_rn(rcij, rcij)) T.bslist[atomicAdd(&T.nbs[0], 1)] = i;
        else T.bslist[T.npad - 1 - atomicAdd(&T.nbs[1], 1)] = i;
      }
    }
  }
  // the last block to finish empties the pair list for the closing kicks of the BS pass (every block
  // read its length on entry)
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&T.bsnext[2], 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last && threadIdx.x == 0) { *T.npairs = 0u; T.bsnext[2] = 0u; }
}

// A planet's path polynomial (components c0 .. c0 + 2, powers of s) at s in [-1, 1] (Horner).
__device__ __forceinline__ void poly3(const double *cf, double s, double &a, double &b, double &c) {
  a = cf[TP_CHEB - 1]; b = cf[2 * TP_CHEB - 1]; c = cf[3 * TP_CHEB - 1];
#pragma unroll
  for (int k = TP_CHEB - 2; k >= 0; --k) {
    a = fma(a, s, cf[k]); b = fma(b, s, cf[TP_CHEB + k]); c = fma(c, s, cf[2 * TP_CHEB + k]);
  }
}
__device__ __forceinline__ double poly1(const double *cf, double s) {
  double a = cf[TP_CHEB - 1];
#pragma unroll
  for (int k = TP_CHEB - 2; k >= 0; --k) a = fma(a, s, cf[k]);
  return a;
}

// Planet j's state on its Kepler path at time t of the substep: the table for full-length
// attempts, otherwise the path polynomial (or, where it was not admitted, a Kepler solve).
__device__ __forceinline__ void planet_at(const Sim &S, const TPSet &T, const DevParams &P, int j, bool table,
                                          int k, int m, double t, double i2tau, double &px, double &py, double &pz) {
  if (table) {
    const double *o = T.ptab + ((size_t)j * TP_TAB + tab_index(k, m)) * 6;
    px = o[0]; py = o[1]; pz = o[2];
    return;
  }
  if (T.pcok[j]) {
    poly3(T.ppoly + (size_t)j * 6 * TP_CHEB, fma(t, i2tau, -1.0), px, py, pz);
    return;
  }
  const int pp = S.npad;
  double x = S.x0[j], y = S.x0[pp + j], z = S.x0[2 * pp + j];
  double vx = S.v0[j], vy = S.v0[pp + j], vz = S.v0[2 * pp + j];
  if (dbits(t) != 0ULL) kepler_drift_dev(P.G * P.m0, P.mu2, x, y, z, vx, vy, vz, t, P.kepler_maxit, nullptr);
  px = x; py = y; pz = z;
}

// Planet j's position and velocity at time t (series or Kepler solve), for the contact test.
__device__ __forceinline__ void planet_state_at(const Sim &S, const TPSet &T, const DevParams &P, int j, double t,
                                                double i2tau, double *o) {
  if (T.pcok[j]) {
    const double s = fma(t, i2tau, -1.0);
    const double *cf = T.ppoly + (size_t)j * 6 * TP_CHEB;
    poly3(cf, s, o[0], o[1], o[2]);
    poly3(cf + 3 * TP_CHEB, s, o[3], o[4], o[5]);
    return;
  }
  const int pp = S.npad;
  double x = S.x0[j], y = S.x0[pp + j], z = S.x0[2 * pp + j];
  double vx = S.v0[j], vy = S.v0[pp + j], vz = S.v0[2 * pp + j];
  if (dbits(t) != 0ULL) kepler_drift_dev(P.G * P.m0, P.mu2, x, y, z, vx, vy, vz, t, P.kepler_maxit, nullptr);
  o[0] = x; o[1] = y; o[2] = z; o[3] = vx; o[4] = vy; o[5] = vz;
}

constexpr int TP_PRE = 2;  // encountered planets whose positions a BS attempt evaluates up front

__constant__ double c_tp_facinv[BS_LEVELS + 1][BS_LEVELS];  // 1 / ((L / (L - j))^2 - 1)

// Acceleration of a TP at state y (level k, midpoint m of an attempt of length H from t0): the
// Sun, and each encountered planet weighted by 1 - W_B inside the pair's critical radius. Lanes
// pair up: level lane l (l16 < 8) evaluates the Sun's pull at its own state while lane l + 8
// evaluates the first planet's at the same state (passed over) with the same instructions, and
// hands back g and the separation; further planets follow on the upper lane. The level lane
// accumulates Sun, planet 1, planet 2, ... exactly as a serial evaluation would. `act` holds the
// participating lanes (whole pairs); planet positions come from the prepared list (wpos) for the
// first TP_PRE planets of a shorter attempt, otherwise from the table or the path polynomial.
__device__ __forceinline__ void tp_force(const Sim &S, const TPSet &T, const DevParams &P, int i, unsigned em, bool table,
                                         int k, int m, double t0, double h, double H, double i2tau, const double *wpos,
                                         const double *y, double &ax, double &ay, double &az, unsigned act) {
  const int lane = threadIdx.x & 31;
  const bool up = (lane & 8) != 0;
  const double sx = __shfl_sync(act, y[0], lane & ~8), sy = __shfl_sync(act, y[1], lane & ~8),
               sz = __shfl_sync(act, y[2], lane & ~8);
  unsigned bits = em;
  for (int p = 0;; ++p) {
    // this lane's body: the Sun (level lane, first round) or planet p (upper lane)
    double bx = 0.0, by = 0.0, bz = 0.0, gm = P.Gm0, A = 0.0;
    u64 cut = ~0ULL;
    const bool body = up && bits;
    if (body) {
      const int j = __ffs(bits) - 1;
      if (!table && p < TP_PRE) {
        const double *q = wpos + (p * TP_TAB + tab_index(k, m)) * 3;
        bx = q[0]; by = q[1]; bz = q[2];
      } else {
        const double t = (m == 2 * k) ? t0 + H : t0 + m * h;
        planet_at(S, T, P, j, table, k, m, t, i2tau, bx, by, bz);
      }
      gm = S.gm[j];
      A = pmin(T.A[i], S.A[j]);
      cut = umax64(T.rcsq[i], S.rcsq[j]);
    }
    double g = 0.0, dx = 0.0, dy = 0.0, dz = 0.0;
    if (body || (!up && p == 0)) {
      dx = bx - sx; dy = by - sy; dz = bz - sz;
      const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      const double yr = rsqrt_refined(r2);
      const double r3 = up ? yr * yr * yr : rcube_refined(r2);
      double wB, wA;
      changeover_w(r2 * yr, A, P.kmode, wB, wA);  // 1 for the Sun (A = 0)
      g = dbits(r2) >= cut ? 0.0 : gm * wA * r3;
    }
    if (p == 0 && !up) { ax = g * dx; ay = g * dy; az = g * dz; }  // the Sun: -G m0 y / |y|^3
    const double gp = __shfl_xor_sync(act, g, 8), px = __shfl_xor_sync(act, dx, 8),
                 py = __shfl_xor_sync(act, dy, 8), pz = __shfl_xor_sync(act, dz, 8);
    if (!bits) break;
    if (!up) { ax = fma(gp, px, ax); ay = fma(gp, py, ay); az = fma(gp, pz, az); }
    bits &= bits - 1;
    if (!bits) break;
  }
}

// BS of one listed TP per warp; lane L-1 runs level L (n_L = 2L midpoint substeps) and lanes
// 8..13 hold the tableau rows. One block of TPB_WARPS warps per SM (the register budget allows
// twelve warps per SM); warp w issues on sub-partition w % 4.
//
// Placement. The launch lasts as long as its slowest particle (one deep inside a planet's Hill
// sphere takes 10-30 sequential attempts), and an FP64 warp instruction holds its sub-partition's
// pipe whatever the other warps there do, so a particle sharing its sub-partition with two busy
// warps advances at a third of its own rate. Warp 0 of block b < min(front entries, blocks) takes
// front entry b (the front entries pass inside a tenth of the critical radius) and the other warps of its
// sub-partition leave, so that particle has the pipe to itself; everything else is taken from a
// shared counter, so long encounters do not hold up the rest.
//
// Speculation. After a failed full-length attempt the step control alternates a failed attempt at
// 2H with an accepted one at H. From the second attempt on (from the first for a front entry, whose
// full-length attempt fails), lanes 16..29 mirror lanes 0..13 with H/2 from the same state; their result is used exactly when the serial algorithm's next attempt
// would be that one (the H attempt failed), so results and decisions are the serial algorithm's.
// The mirror lanes cost no FP64 issue: a warp instruction costs the same whatever its active lanes.
// Distinct midpoint times of a shorter attempt pair. Entry (hf, k, m) of half hf (attempt length
// He = H / 2^hf) is at t0 + m h_k with h_k = He / 2k rounded, or t0 + He at m = 2k. Write 2k = o 2^e
// and m = mo 2^a (o, mo odd): h_k is round(H / o) 2^-(e + hf) exactly (a division by a power of
// two only moves the exponent), so m h_k = round(mo round(H / o)) 2^(a - e - hf) depends on
// (o, mo, a - e - hf) alone, and entries with equal keys have bit-identical times: the 160 entries
// of the two attempts fall into 76 classes. The host builds the classes (and checks them on its
// own arithmetic); each class is evaluated once and written to all its slots.
constexpr int TP_PREP_MAX = 96;
__device__ int d_prep_n;
__device__ unsigned short d_prep_rep[TP_PREP_MAX];     // a member: hf << 12 | k << 8 | m
__device__ unsigned char d_prep_first[TP_PREP_MAX + 1];  // class u owns slots [first[u], first[u + 1])
__device__ unsigned char d_prep_slot[2 * TP_TAB];        // hf * TP_TAB + tab_index(k, m)

constexpr int TPB_WARPS = 12;
constexpr int TP_WAIT_MAX = 500;  // naps of about 2 us
constexpr int TPB_WPOS = TP_PRE * TP_TAB * 3;
constexpr size_t TPB_SMEM = (size_t)TPB_WARPS * (2 * TPB_WPOS + 2 * 16) * sizeof(double);

// A warp of the BS pass is done; the last of all empties the BS list for the next substep (every
// warp read its length on entry).
__device__ __forceinline__ void tp_bs_warp_done(const TPSet &T) {
  if ((threadIdx.x & 31) == 0 && atomicAdd(&T.bsnext[3], 1u) == gridDim.x * TPB_WARPS - 1) {
    T.nbs[0] = 0; T.nbs[1] = 0; T.bsnext[3] = 0u;
    for (unsigned k = 0; k < 4 * gridDim.x; ++k) T.bsnext[4 + k] = 0u;  // the sub-partition counts
  }
}

// The closing kick of a TP after its BS substep (kept out of line: the BS loop holds the registers).
__device__ __noinline__ unsigned tp_bs_close(const TPSet &T, const DevParams &P, const PlanetSm &ps, int npl, int i,
                                             double xi, double yi, double zi, double h1, double h2, const double *shc) {
  double ax, ay, az;
  const unsigned cm = tp_close_forces(T, P, ps, npl, i, xi, yi, zi, ax, ay, az);
  tp_close_update(T, i, xi, yi, zi, ax, ay, az, h1, h2, shc);
  return cm;
}

// The BS pass of a substep and the closing kick of every TP. Warps take the listed TPs first (the
// front entries first, each alone on its sub-partition), integrate each over the substep and give
// it its closing kick; then they take the other TPs, 32 at a time, for their closing kick. The
// closing kick has the arithmetic of the first kick and reads the planets at the end of the
// substep; h1 + h2 as in tp_close_update, hcm_last != 0 adds the step's last Sun drift.
__global__ void __launch_bounds__(32 * TPB_WARPS, 1) k_tp_bs(Sim S, TPSet T, DevParams P, double tau, double h1,
                                                           double h2, double hcm_last) {
  constexpr int WPOS = TPB_WPOS;
  extern __shared__ double tpb_smem[];  // per warp: planet positions of both attempts, then s_zt
  __shared__ PlanetSm s_ps[TPB_WARPS];  // per warp: the planets at the end of the substep, for the
  __shared__ double s_shc[TPB_WARPS][3];  // closing kicks, and the last Sun drift's shift
  const int lane = threadIdx.x & 31, half = lane >> 4, l16 = lane & 15, warp = threadIdx.x >> 5;
  double *wpos0 = tpb_smem + warp * 2 * WPOS;
  double (*s_zt)[16] = reinterpret_cast<double (*)[16]>(tpb_smem + TPB_WARPS * 2 * WPOS + warp * 32);
  const int nfront = T.nbs[0], nlist = nfront + T.nbs[1], nprep = d_prep_n;
  const int np = T.npad;
  const double i2tau = 2.0 / tau;
  const int niso = nfront < (int)gridDim.x ? nfront : (int)gridDim.x;  // front entries placed alone
  const bool iso = (int)blockIdx.x < niso;
  if (iso && warp != 0 && (warp & 3) == 0) {  // sub-partition 0 belongs to warp 0's entry
    tp_bs_warp_done(T);
    return;
  }
  warp_load_planets(S, hcm_last, s_ps[warp], s_shc[warp]);
  for (bool first = true;; first = false) {
    int w = 0;
    if (iso && warp == 0 && first) w = blockIdx.x;
    else {
      if (lane == 0) w = niso + (int)atomicAdd(&T.bsnext[0], 1u);
      w = __shfl_sync(0xffffffffu, w, 0);
    }
    if (w >= nlist) break;
    const int i = T.bslist[w < nfront ? w : T.npad - 1 - (w - nfront)];
    const unsigned em = T.emask[i];
    static_assert(BS_LEVELS == 8, "lanes l16 and l16 + 8 pair up on level (l16 & 7) + 1");
    const int L = (l16 & 7) + 1, nk = 2 * L;
    double y[6];
    for (int c = 0; c < 3; ++c) { y[c] = T.x0[c * np + i]; y[3 + c] = T.v0[c * np + i]; }
    double t0 = 0.0, rem = tau, H = tau;
    int halvings = 0, steps = 0, attempts = 0;
    bool removed = false, failed = false;
    while (absbits(rem) != 0ULL && ++attempts < 100000) {
      if (absbits(H) > absbits(rem)) H = rem;
      const bool table = dbits(t0) == 0ULL && dbits(H) == dbits(tau);
      // the mirror lanes attempt H/2; on the full-length attempt only for a front entry, which
      // fails it (a pass inside a tenth of rc needs shorter substeps)
      const bool spec = !table || w < nfront;
      const bool use_tab = table && !(spec && half);  // this lane's positions come from the table
      const double Hl = (spec && half) ? 0.5 * H : H;  // this lane's attempt length
      const double h = __ddiv_rn(Hl, (double)nk), h2 = 2.0 * h;
      double *wpos = wpos0 + (spec ? half * WPOS : 0);
      if (spec && em) {  // positions of the first TP_PRE planets at all midpoint times of both attempts
        __syncwarp();
        unsigned bits = em;
        for (int p = 0; p < TP_PRE && bits; ++p) {
          const int j = __ffs(bits) - 1;
          bits &= bits - 1;
          for (int u0 = 0; u0 < nprep; u0 += 32) {  // one time class per lane
            const int u = u0 + lane;
            const unsigned rp = d_prep_rep[u < nprep ? u : 0];
            const int hf = rp >> 12, k = (rp >> 8) & 15, m = rp & 255;
            const double hk = __shfl_sync(0xffffffffu, h, hf * 16 + k - 1);  // He / 2k: level k's lane of half hf
            if (u < nprep) {
              const double He = hf ? 0.5 * H : H;
              const double t = (m == 2 * k) ? t0 + He : t0 + m * hk;
              double px, py, pz;
              planet_at(S, T, P, j, false, k, m, t, i2tau, px, py, pz);
              for (int q = d_prep_first[u]; q < d_prep_first[u + 1]; ++q) {
                const int sl = d_prep_slot[q], sh = sl >= TP_TAB ? 1 : 0;
                double *o = wpos0 + sh * WPOS + (p * TP_TAB + sl - sh * TP_TAB) * 3;
                o[0] = px; o[1] = py; o[2] = pz;
              }
            }
          }
        }
        __syncwarp();
      }
      double za[6], zb[6], ax, ay, az;
      for (int c = 0; c < 6; ++c) za[c] = y[c];
      tp_force(S, T, P, i, em, use_tab, L, 0, t0, h, Hl, i2tau, wpos, y, ax, ay, az, 0xffffffffu);
      zb[0] = fma(h, y[3], y[0]); zb[1] = fma(h, y[4], y[1]); zb[2] = fma(h, y[5], y[2]);
      zb[3] = fma(h, ax, y[3]); zb[4] = fma(h, ay, y[4]); zb[5] = fma(h, az, y[5]);
      // Level L (lane L - 1 of each half) finishes at evaluation 2L; the half's lanes 8..13 then
      // extend its tableau by that row, component c on lane 8 + c (polynomial extrapolation in h^2,
      // Neville), and the first converged level ends that half's attempt: the same decision as
      // building the whole tableau first.
      const int cc = l16 - BS_LEVELS;            // component of the tableau lanes
      const bool tabl = cc >= 0 && cc < 6;
      double sc = 0.0;                           // 1/|x| or 1/|v| at the start of the attempt
      if (tabl) {
        const double *yy = y + (cc < 3 ? 0 : 3);
        const double s2 = fma(yy[2], yy[2], fma(yy[1], yy[1], yy[0] * yy[0]));
        sc = dbits(s2) == 0ULL ? 4.49423283715579e307 : rsqrt_refined(s2);
      }
      const int lmax = P.bs_kmax < BS_LEVELS ? P.bs_kmax : BS_LEVELS;
      double prev[BS_LEVELS], tlast = 0.0;  // previous tableau row; T_{Lc,Lc} of the current one
      double tfix = 0.0;                    // the mirror half's accepted value (its tableau lanes)
      int acc = 0, accB = 0;
      for (int m = 1; m <= 2 * lmax; ++m) {
        const unsigned act = __ballot_sync(0xffffffffu, m <= nk);
        if (m <= nk) {
          tp_force(S, T, P, i, em, use_tab, L, m, t0, h, Hl, i2tau, wpos, zb, ax, ay, az, act);
          if (m < nk) {
            double zn[6];
            zn[0] = fma(h2, zb[3], za[0]); zn[1] = fma(h2, zb[4], za[1]); zn[2] = fma(h2, zb[5], za[2]);
            zn[3] = fma(h2, ax, za[3]); zn[4] = fma(h2, ay, za[4]); zn[5] = fma(h2, az, za[5]);
            for (int c = 0; c < 6; ++c) { za[c] = zb[c]; zb[c] = zn[c]; }
          }
        }
        if (m & 1) continue;
        const int Lc = m >> 1;
        // level Lc's lane hands its last midpoint state to the tableau lanes, which form
        // T_{Lc,1} = (z_{n-1} + z_n + h z'_n) / 2 one component each
        double *zt = s_zt[half];
        if (l16 == Lc - 1) {
          for (int c = 0; c < 6; ++c) { zt[c] = za[c]; zt[6 + c] = zb[c]; }
          zt[12] = ax; zt[13] = ay; zt[14] = az; zt[15] = h;
        }
        __syncwarp();
        double t1 = 0.0;
        if (tabl) {
          const double dz = cc < 3 ? zt[9 + cc] : zt[12 + cc - 3];
          t1 = 0.5 * fma(zt[15], dz, zt[6 + cc] + zt[cc]);
        }
        __syncwarp();
        bool ok = false;
        if (tabl) {
          double before;
          tlast = neville_row(t1, Lc, [&](int j) { return c_tp_facinv[Lc][j]; }, prev, before);
          ok = Lc >= 2 && absbits((tlast - before) * sc) <= dbits(P.bs_eps);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (spec && !accB && ((bal >> (16 + BS_LEVELS)) & 0x3fu) == 0x3fu) {  // the H/2 attempt converged
          accB = Lc;
          tfix = tlast;
        }
        if (((bal >> BS_LEVELS) & 0x3fu) == 0x3fu) { acc = Lc; break; }  // all six components converged
      }
      int use = 0;
      if (!acc) {  // the serial algorithm halves H and tries again: the mirror lanes' attempt
        H *= 0.5;
        if (++halvings > P.bs_max_halvings) { failed = true; break; }
        if (!spec) continue;
        ++attempts;
        if (!accB) {
          H *= 0.5;
          if (++halvings > P.bs_max_halvings) { failed = true; break; }
          continue;
        }
        use = 1;
      }
      double yn[6];
      const double mine = half ? tfix : tlast;
      for (int c = 0; c < 6; ++c) yn[c] = __shfl_sync(0xffffffffu, tabl ? mine : 0.0, 16 * use + BS_LEVELS + c);
      halvings = 0;
      steps++;
      if (P.collisions) {  // contact with an encountered planet during the substep removes the TP
        bool hit = false;
        unsigned bits = em;
        while (bits && !hit) {
          const int j = __ffs(bits) - 1;
          bits &= bits - 1;
          double pa[6], pb[6];
          if (T.pcok[j]) {  // lane q < 12 evaluates component q % 6 at t0 (q < 6) or t0 + H
            double pv = 0.0;
            if (lane < 12)
              pv = poly1(T.ppoly + ((size_t)j * 6 + lane % 6) * TP_CHEB, fma(lane < 6 ? t0 : t0 + H, i2tau, -1.0));
            for (int c = 0; c < 6; ++c) {
              pa[c] = __shfl_sync(0xffffffffu, pv, c);
              pb[c] = __shfl_sync(0xffffffffu, pv, 6 + c);
            }
          } else {
            planet_state_at(S, T, P, j, t0, i2tau, pa);
            planet_state_at(S, T, P, j, t0 + H, i2tau, pb);
          }
          const double rr = T.R[i] + S.R[j];
          const double dmin = hermite_min_capped(
              __dsub_rn(pa[0], y[0]), __dsub_rn(pa[1], y[1]), __dsub_rn(pa[2], y[2]),
              __dsub_rn(pa[3], y[3]), __dsub_rn(pa[4], y[4]), __dsub_rn(pa[5], y[5]),
              __dsub_rn(pb[0], yn[0]), __dsub_rn(pb[1], yn[1]), __dsub_rn(pb[2], yn[2]),
              __dsub_rn(pb[3], yn[3]), __dsub_rn(pb[4], yn[4]), __dsub_rn(pb[5], yn[5]), H, rr * rr);
          hit = dmin < rr * rr;
        }
        if (hit) { for (int c = 0; c < 6; ++c) y[c] = yn[c]; removed = true; break; }
      }
      for (int c = 0; c < 6; ++c) y[c] = yn[c];
      t0 += H;
      rem -= H;
      H *= 2.0;
    }
    unsigned cm = 0u;
    if (lane == 0) {
      for (int c = 0; c < 3; ++c) { T.x[c * np + i] = y[c]; T.v[c * np + i] = y[3 + c]; }
      if (removed) { T.alive[i] = 0; atomicAdd((unsigned long long *)&T.counters[3], 1ULL); }
      if (failed) atomicOr(S.status, ST_BS_FAILED);
      atomicAdd((unsigned long long *)&T.counters[2], (unsigned long long)steps);
      if (!removed)
        cm = tp_bs_close(T, P, s_ps[threadIdx.x >> 5], S.n, i, y[0], y[1], y[2], h1, h2,
                         hcm_last != 0.0 ? s_shc[threadIdx.x >> 5] : nullptr);
    }
    tp_append_pairs(T, i, cm, true);
  }
  // A warp on a sub-partition where another warp of the block still integrates a TP waits (up to
  // TP_WAIT_MAX naps) until that one is done or the closing kicks are all taken: a kick warp beside
  // it would take two thirds of the sub-partition's FP64 issue from a BS chain that may be the last
  // of the pass.
  unsigned *sp_done = T.bsnext + 4 + 4 * blockIdx.x + (warp & 3);
  if (lane == 0) atomicAdd(sp_done, 1u);
  for (int nap = 0; !iso && nap < TP_WAIT_MAX; ++nap) {
    unsigned ok = 0u;
    if (lane == 0) ok = __ldcg(sp_done) >= TPB_WARPS / 4 || (long long)__ldcg(&T.bsnext[1]) * 64 >= (long long)T.n;
    if (__shfl_sync(0xffffffffu, ok, 0)) break;
    __nanosleep(2000);
  }
  // the closing kick of the TPs outside the BS list (no encounter, no failed solve), 64 a warp: two
  // a lane side by side
  while (!iso) {
    unsigned c = 0u;
    if (lane == 0) c = atomicAdd(&T.bsnext[1], 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    if ((long long)c * 64 >= (long long)T.n) break;
    int ii[2];
    bool act[2];
    double x[2][3], acc[2][3];
    unsigned cm[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int i = (int)c * 64 + 32 * k + lane;
      ii[k] = i;
      act[k] = i < T.n && T.alive[i] && T.emask[i] == 0u && !T.fail[i];
      for (int q = 0; q < 3; ++q) x[k][q] = act[k] ? T.x[q * np + i] : 0.0;
    }
    tp_close_forces_k<2>(T, P, s_ps[warp], S.n, ii, act, x, acc, cm);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (act[k])
        tp_close_update(T, ii[k], x[k][0], x[k][1], x[k][2], acc[k][0], acc[k][1], acc[k][2], h1, h2,
                        hcm_last != 0.0 ? s_shc[warp] : nullptr);
      tp_append_pairs(T, ii[k], cm[k], true);
    }
  }
  tp_bs_warp_done(T);
}

// TP input (heliocentric AoS) -> democratic SoA: v_b = v_h - sum m v_h / (m0 + sum m) with the
// massive bodies' heliocentric input (staged as AoS with the central mass in row 0).
__global__ void k_tp_from_helio(TPSet T, int nmass, const double *mh, const double *vmh, const double *xh,
                                const double *vh, const double *Rh, int keep) {
  __shared__ double vcm[3];
  if (threadIdx.x == 0) {
    double M = mh[0], p[3] = {0.0, 0.0, 0.0};
    for (int j = 1; j < nmass; ++j) {
      M += mh[j];
      for (int c = 0; c < 3; ++c) p[c] += mh[j] * vmh[3 * j + c];
    }
    for (int c = 0; c < 3; ++c) vcm[c] = p[c] / M;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T.npad) return;
  const int np = T.npad;
  if (i >= T.n) {  // padding: never alive
    T.alive[i] = 0;
    return;
  }
  if (keep && !T.alive[i]) return;
  for (int c = 0; c < 3; ++c) { T.x[c * np + i] = xh[3 * i + c]; T.v[c * np + i] = vh[3 * i + c] - vcm[c]; }
  if (!keep) { T.R[i] = Rh ? Rh[i] : 0.0; T.alive[i] = 1; }
}

// TPs back to heliocentric AoS: v_h = v_b + P/m0 with the massive momentum P.
__global__ void k_tp_to_helio(Sim S, TPSet T, DevParams P, double *xh, double *vh, int *alive) {
  __shared__ double pm[3];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x, np = S.npad;
    for (int c = 0; c < 3; ++c) {
      double a = 0.0;
      for (int j = lane; j < S.n; j += 32)
        if (S.alive[j]) a = fma(S.m[j], S.v[c * np + j], a);
      a = warp_sum(a);
      if (lane == 0) pm[c] = a;
    }
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T.n) return;
  const int np = T.npad;
  for (int c = 0; c < 3; ++c) {
    if (xh) xh[3 * i + c] = T.x[c * np + i];
    if (vh) vh[3 * i + c] = fma(pm[c], P.inv_m0, T.v[c * np + i]);
  }
  if (alive) alive[i] = T.alive[i];
}

// ---------------------------------------------------------------------------------------------
static int grid_of(int n, int b) { return (n + b - 1) / b; }

// Classes of bit-identical midpoint times (see d_prep_rep), checked by evaluating every member's
// time for several attempt lengths and start times: a class whose members differ is an error.
static int build_prep_classes() {
  struct Key { int o, mo, ex; };
  Key keys[2 * TP_TAB];
  int cls[2 * TP_TAB], nu = 0;
  unsigned short rep[TP_PREP_MAX];
  for (int hf = 0; hf < 2; ++hf)
    for (int k = 1; k <= BS_LEVELS; ++k)
      for (int m = 0; m <= 2 * k; ++m) {
        Key key{0, 0, 0};  // m = 0: t0
        if (m == 2 * k) key = Key{1, 1, -hf};  // t0 + He
        else if (m > 0) {
          int o = 2 * k, e = 0, mo = m, a = 0;
          while (o % 2 == 0) { o /= 2; ++e; }
          while (mo % 2 == 0) { mo /= 2; ++a; }
          key = Key{o, mo, a - e - hf};
        }
        const int sl = hf * TP_TAB + k * k - 1 + m;
        int c = 0;
        while (c < nu && !(keys[c].o == key.o && keys[c].mo == key.mo && keys[c].ex == key.ex)) ++c;
        if (c == nu) {
          if (nu == TP_PREP_MAX) return -1;
          keys[nu] = key;
          rep[nu] = (unsigned short)(hf << 12 | k << 8 | m);
          ++nu;
        }
        cls[sl] = c;
      }
  unsigned char first[TP_PREP_MAX + 1], slot[2 * TP_TAB];
  int n = 0;
  for (int c = 0; c < nu; ++c) {
    first[c] = (unsigned char)n;
    for (int sl = 0; sl < 2 * TP_TAB; ++sl)
      if (cls[sl] == c) slot[n++] = (unsigned char)sl;
  }
  first[nu] = (unsigned char)n;
  const double Hs[] = {6.0, 3.0, 0.75, 2.2206093, -6.0, -1.7320508075688772, 4.1e-3};
  const double t0s[] = {0.0, 1.5, 2.9137, -3.3};
  for (double H : Hs)
    for (double t0 : t0s)
      for (int c = 0; c < nu; ++c) {
        double tc = 0.0;
        for (int q = first[c]; q < first[c + 1]; ++q) {
          const int sl = slot[q], hf = sl >= TP_TAB ? 1 : 0, e = sl - hf * TP_TAB;
          int k = 1;
          while ((k + 1) * (k + 1) - 1 <= e) ++k;
          const int m = e - (k * k - 1);
          const double He = hf ? 0.5 * H : H, hk = He / (double)(2 * k);
          const double t = (m == 2 * k) ? t0 + He : t0 + m * hk;
          if (q == first[c]) tc = t;
          else if (memcmp(&t, &tc, sizeof(double)) != 0) return -1;
        }
      }
  if (cudaMemcpyToSymbol(d_prep_n, &nu, sizeof(int)) != cudaSuccess ||
      cudaMemcpyToSymbol(d_prep_rep, rep, sizeof(rep)) != cudaSuccess ||
      cudaMemcpyToSymbol(d_prep_first, first, sizeof(first)) != cudaSuccess ||
      cudaMemcpyToSymbol(d_prep_slot, slot, sizeof(slot)) != cudaSuccess)
    return -1;
  return 0;
}

int tp_init_constants() {
  if (build_prep_classes() != 0) return -1;
  double f[BS_LEVELS + 1][BS_LEVELS] = {};
  for (int L = 2; L <= BS_LEVELS; ++L)
    for (int j = 1; j < L; ++j) {
      const double ratio = (double)L / (double)(L - j);
      f[L][j] = 1.0 / (ratio * ratio - 1.0);
    }
  if (cudaFuncSetAttribute(k_tp_bs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TPB_SMEM) != cudaSuccess) return -1;
  double tk[TP_CHEB][TP_CHEB] = {};  // T_0 = 1, T_1 = s, T_{k+1} = 2 s T_k - T_{k-1} (integers)
  tk[0][0] = 1.0;
  tk[1][1] = 1.0;
  for (int k = 1; k + 1 < TP_CHEB; ++k)
    for (int q = 0; q < TP_CHEB; ++q) tk[k + 1][q] = (q > 0 ? 2.0 * tk[k][q - 1] : 0.0) - tk[k - 1][q];
  if (cudaMemcpyToSymbol(c_cheb_pow, tk, sizeof(tk)) != cudaSuccess) return -1;
  double cs[TP_CHEB][TP_CHEB];  // T_k at the Chebyshev nodes, from the host's cos
  for (int k = 0; k < TP_CHEB; ++k)
    for (int q = 0; q < TP_CHEB; ++q) cs[k][q] = cos(M_PI * (double)(k * (2 * q + 1)) / (double)(2 * TP_CHEB));
  if (cudaMemcpyToSymbol(d_cheb_cos, cs, sizeof(cs)) != cudaSuccess) return -1;
  return cudaMemcpyToSymbol(c_tp_facinv, f, sizeof(f)) == cudaSuccess ? 0 : -1;
}

void launch_tp_from_helio(const TPSet &T, int nmass, const double *mh, const double *vmh, const double *xh,
                          const double *vh, const double *Rh, int keep, cudaStream_t st) {
  k_tp_from_helio<<<grid_of(T.npad, 256), 256, 0, st>>>(T, nmass, mh, vmh, xh, vh, Rh, keep);
}
void launch_tp_to_helio(const Sim &S, const TPSet &T, const DevParams &P, double *xh, double *vh, int *alive,
                        cudaStream_t st) {
  k_tp_to_helio<<<grid_of(T.n, 256), 256, 0, st>>>(S, T, P, xh, vh, alive);
}

void launch_tp_rcrit(const TPSet &T, const DevParams &P, double tau_abs, int check, cudaStream_t st) {
  k_tp_rcrit<<<grid_of(T.n, 256), 256, 0, st>>>(T, P, tau_abs, check);
}
void launch_tp_kick(const Sim &S, const TPSet &T, const DevParams &P, cudaStream_t st) {
  k_tp_kick<<<grid_of(T.n, 128), 128, 0, st>>>(S, T, P);
}
void launch_tp_open_drift(const Sim &S, const TPSet &T, const DevParams &P, double tau_abs, double h1, double tau,
                          double hcm1, cudaStream_t st) {
  k_tp_open_drift<<<grid_of(T.n, 128), 128, 0, st>>>(S, T, P, tau_abs, h1, tau, hcm1);
}
void launch_tp_drift(const Sim &S, const TPSet &T, const DevParams &P, double tau, double hcm1, double hcm2, cudaStream_t st) {
  k_tp_drift<<<grid_of(T.n, 128), 128, 0, st>>>(S, T, P, tau, hcm1, hcm2);
}
void launch_planet_table(const Sim &S, const TPSet &T, const DevParams &P, double tau, cudaStream_t st) {
  k_planet_table<<<S.n, 128, 0, st>>>(S, T, P, tau);
}
void launch_tp_encounter(const Sim &S, const TPSet &T, double tau, int blocks, cudaStream_t st) {
  k_tp_encounter<<<blocks, 256, 0, st>>>(S, T, tau);
}
void launch_tp_bs(const Sim &S, const TPSet &T, const DevParams &P, double tau, double h1, double h2, double hcm_last,
                  int blocks, cudaStream_t st) {
  if (blocks > TP_BS_MAXBLOCKS) blocks = TP_BS_MAXBLOCKS;
  k_tp_bs<<<blocks, 32 * TPB_WARPS, TPB_SMEM, st>>>(S, T, P, tau, h1, h2, hcm_last);
}

}  // namespace genga
