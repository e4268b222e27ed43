// batch.cu -- many independent planetary systems advanced together (Sect. 3.4, multi-simulation
// mode), each system with its own central mass and up to 64 orbiting bodies.
//
// Bodies of one system are contiguous and systems are ordered by size, so neighbouring lanes
// loop over partner sets of similar length (the paper masks "false interactions" of a thread
// that runs past its system; here no lane ever reads another system). The kick is autotuned at
// init between one thread (or SPLIT threads) per body summing its whole acceleration, and a
// Newton's-third-law kernel that visits every pair of a system once on one warp; neither needs
// partial-sum buffers or atomics. Candidate and encounter partners are per-body 64-bit masks (bit = index
// within the system). Groups are found by one warp per system and integrated by the
// Bulirsch-Stoer kernel of the single-system mode, which reads the group's central mass.
#include "genga_launch.h"

namespace genga {

__device__ __forceinline__ double sys_inv(double m0) { return rcp_refined(m0); }

// Critical radii with the body's own central mass; the kick-reuse test is per system.
__global__ void k_b_rcrit(Sim S, DevParams P, double tau_abs, int check_reuse) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (check_reuse && i == 0) atomicAdd((unsigned long long *)&S.counters[C_STEPS], 1ULL);
  if (i >= S.npad) return;
  const int np = S.npad;
  if (!S.alive[i]) {
    S.rc[i] = 0.0; S.A[i] = 0.0; S.T[i] = 0ULL; S.rcsq[i] = 0ULL;
    return;
  }
  const int s = S.sys_of[i];
  const double mu = P.G * S.sys_m0[s];
  const double x = S.x[i], y = S.x[np + i], z = S.x[2 * np + i];
  const double vx = S.v[i], vy = S.v[np + i], vz = S.v[2 * np + i];
  const double r2 = fma(z, z, fma(y, y, x * x));
  const double ir = rsqrt_refined(r2);
  const double v2 = fma(vz, vz, fma(vy, vy, vx * vx));
  const double inva = fma(2.0, ir, -v2 * sys_inv(mu));
  const double asemi = is_neg_or_zero(inva) ? r2 * ir : rcp_refined(inva);
  const double rh = asemi * S.hill[i];
  const double vabs = (dbits(v2) == 0ULL) ? 0.0 : v2 * rsqrt_refined(v2);
  const double rc = pmax(P.n1 * rh, (P.n2 * tau_abs) * vabs);
  if (check_reuse && dbits(rc) > dbits(P.pc * S.rc[i])) {
    S.sys_flag[s] = 1;
    atomicOr(S.status, ST_REUSE_FULLKICK);
    atomicAdd((unsigned long long *)&S.counters[C_FULLKICK], 1ULL);
  }
  S.rc[i] = rc;
  const double t = __dmul_rn(P.pc, rc);
  S.T[i] = dbits(__dmul_rn(t, t));
  S.rcsq[i] = dbits(__dmul_rn(rc, rc));
  S.A[i] = (dbits(rc) == 0ULL) ? 0.0 : rcp_refined(0.9 * rc);
}

// Kick with the prechecker. CLOSE: far pairs + candidates (recorded) with the current critical
// radii, v += h1 a (+ h2 a). OPEN: stored far field + candidates with the new radii (or every
// pair when the system failed the reuse test). INIT: far field and candidates only.
template <int MODE, int SPLIT>
__global__ void k_b_kick(Sim S, DevParams P, double h1, double h2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / SPLIT, sub = t % SPLIT;
  const int np = S.npad;
  const bool live = i < np && S.alive[i];
  double fx = 0, fy = 0, fz = 0, nx = 0, ny = 0, nz = 0;
  u64 mask = 0ULL;
  bool full = false;
  if (live) {
    const int s = S.sys_of[i], st = S.sys_start[s], en = S.sys_start[s + 1];
    full = (MODE == FIN_OPEN) && S.sys_flag[s] != 0;
    const double xi = S.x[i], yi = S.x[np + i], zi = S.x[2 * np + i];
    const u64 Ti = S.T[i], Qi = S.rcsq[i];
    const double Ai = S.A[i];
    if (MODE != FIN_OPEN || full) {
      for (int j = st + sub; j < en; j += SPLIT) {
        if (j == i || !S.alive[j]) continue;
        const double dx = S.x[j] - xi, dy = S.x[np + j] - yi, dz = S.x[2 * np + j] - zi;
        const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
        const double w3 = rcube_refined(r2);
        const u64 rb = dbits(r2);
        const bool cand = (MODE != FIN_OPEN) && rb < umax64(Ti, S.T[j]);
        double g = S.gm[j] * w3;
        if (cand || full) {
          if (rb < umax64(Qi, S.rcsq[j])) {
            double wB, wA;
            changeover_w(r2 * rsqrt_refined(r2), pmin(Ai, S.A[j]), P.kmode, wB, wA);
            g *= wB;
          }
          if (cand) mask |= 1ULL << (j - st);
          nx = fma(g, dx, nx); ny = fma(g, dy, ny); nz = fma(g, dz, nz);
        } else {
          fx = fma(g, dx, fx); fy = fma(g, dy, fy); fz = fma(g, dz, fz);
        }
      }
    } else {  // KickA: recompute only the candidates with the new critical radii
      u64 bits = S.bmask[i];
      int k = 0;
      while (bits) {
        const int b = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        if ((k++ % SPLIT) != sub) continue;
        const int j = st + b;
        const double dx = S.x[j] - xi, dy = S.x[np + j] - yi, dz = S.x[2 * np + j] - zi;
        const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
        const double yr = rsqrt_refined(r2);
        double g = S.gm[j] * (yr * yr * yr);
        if (dbits(r2) < umax64(Qi, S.rcsq[j])) {
          double wB, wA;
          changeover_w(r2 * yr, pmin(Ai, S.A[j]), P.kmode, wB, wA);
          g *= wB;
        }
        nx = fma(g, dx, nx); ny = fma(g, dy, ny); nz = fma(g, dz, nz);
      }
    }
  }
#pragma unroll
  for (int o = SPLIT >> 1; o > 0; o >>= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o); fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o); nx += __shfl_xor_sync(0xffffffffu, nx, o);
    ny += __shfl_xor_sync(0xffffffffu, ny, o); nz += __shfl_xor_sync(0xffffffffu, nz, o);
    mask |= __shfl_xor_sync(0xffffffffu, mask, o);
  }
  if (!live || sub != 0) return;
  double ax, ay, az;
  if (MODE == FIN_OPEN) {
    if (full) { ax = nx; ay = ny; az = nz; }
    else { ax = S.afar[i] + nx; ay = S.afar[np + i] + ny; az = S.afar[2 * np + i] + nz; }
  } else {
    S.afar[i] = fx; S.afar[np + i] = fy; S.afar[2 * np + i] = fz;
    S.bmask[i] = mask;
    if (mask) atomicAdd((unsigned long long *)&S.counters[C_CAND], (unsigned long long)__popcll(mask));
    ax = fx + nx; ay = fy + ny; az = fz + nz;
  }
  if (MODE == FIN_INIT) return;
  double vx = fma(h1, ax, S.v[i]), vy = fma(h1, ay, S.v[np + i]), vz = fma(h1, az, S.v[2 * np + i]);
  if (h2 != 0.0) { vx = fma(h2, ax, vx); vy = fma(h2, ay, vy); vz = fma(h2, az, vz); }
  S.v[i] = vx; S.v[np + i] = vy; S.v[2 * np + i] = vz;
}

// ---------------------------------------------------------------------------------------------
// Kick with Newton's third law (CLOSE / INIT): every unordered pair of a system once, on one warp,
// the same terms as k_b_kick (the pull on each side is the partner's Gm r^-3, times the changeover
// weight inside rc). Systems of up to 32 bodies sit in lane segments of width W (the next power of
// two), 32 / W systems a warp; a segment of n bodies runs a ring: at step s = 1 .. floor(n/2) lane
// u meets body (u + s) mod n, whose data and pair sums rotate one lane a step (the last step of an
// even n takes half the lanes). A system of 33..64 bodies takes a warp: the ring of bodies 0..31,
// the ring of bodies 32..n-1, and their cross pairs, for which the second block (padded to P, a
// power of two) is replicated 32 / P times around the warp, so that P one-lane rotations meet every
// cross pair once; the replicas' sums are then added by a butterfly. Each body's far field, near
// field and candidate mask are summed in a fixed order, so results do not depend on the schedule.
// Work item k (one warp): kjobs[2k] = first system, kjobs[2k + 1] = W << 8 | systems (W = 64: one
// system of 33..64 bodies).
// ---------------------------------------------------------------------------------------------
struct BkBody {
  double x, y, z, gm, A;
  u64 T, Q;
  int al;
};
struct BkAcc {
  double f0, f1, f2, n0, n1, n2;  // far field, near field (candidates)
  u64 mask;                       // candidate partners (bit = index in the system)
};

__device__ __forceinline__ void bk_load(const Sim &S, int i, BkBody &B) {  // i < 0: no body
  const int np = S.npad;
  const bool ok = i >= 0 && S.alive[i];
  B.al = ok;
  B.x = ok ? S.x[i] : 0.0; B.y = ok ? S.x[np + i] : 0.0; B.z = ok ? S.x[2 * np + i] : 0.0;
  B.gm = ok ? S.gm[i] : 0.0; B.A = ok ? S.A[i] : 0.0;
  B.T = ok ? S.T[i] : 0ULL; B.Q = ok ? S.rcsq[i] : 0ULL;
}
__device__ __forceinline__ void bk_shfl(BkBody &B, int src) {
  B.x = __shfl_sync(0xffffffffu, B.x, src); B.y = __shfl_sync(0xffffffffu, B.y, src);
  B.z = __shfl_sync(0xffffffffu, B.z, src); B.gm = __shfl_sync(0xffffffffu, B.gm, src);
  B.A = __shfl_sync(0xffffffffu, B.A, src); B.T = __shfl_sync(0xffffffffu, B.T, src);
  B.Q = __shfl_sync(0xffffffffu, B.Q, src); B.al = __shfl_sync(0xffffffffu, B.al, src);
}
__device__ __forceinline__ void bk_zero(BkAcc &a) { a.f0 = a.f1 = a.f2 = a.n0 = a.n1 = a.n2 = 0.0; a.mask = 0ULL; }
__device__ __forceinline__ void bk_acc_shfl(BkAcc &a, int src) {
  a.f0 = __shfl_sync(0xffffffffu, a.f0, src); a.f1 = __shfl_sync(0xffffffffu, a.f1, src);
  a.f2 = __shfl_sync(0xffffffffu, a.f2, src); a.n0 = __shfl_sync(0xffffffffu, a.n0, src);
  a.n1 = __shfl_sync(0xffffffffu, a.n1, src); a.n2 = __shfl_sync(0xffffffffu, a.n2, src);
  a.mask = __shfl_sync(0xffffffffu, a.mask, src);
}
__device__ __forceinline__ void bk_acc_add(BkAcc &a, const BkAcc &b) {
  a.f0 += b.f0; a.f1 += b.f1; a.f2 += b.f2; a.n0 += b.n0; a.n1 += b.n1; a.n2 += b.n2; a.mask |= b.mask;
}

// The pair (i, j), d = x_j - x_i; ui, uj: their indices in the system (mask bits).
__device__ __forceinline__ void bk_pair(const DevParams &P, const BkBody &Bi, const BkBody &Bj, int ui, int uj,
                                        bool act, BkAcc &ai, BkAcc &aj) {
  if (!act || !Bi.al || !Bj.al) return;
  const double dx = Bj.x - Bi.x, dy = Bj.y - Bi.y, dz = Bj.z - Bi.z;
  const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
  const double w3 = rcube_refined(r2);
  const u64 rb = dbits(r2);
  double gi = Bj.gm * w3, gj = Bi.gm * w3;  // the pull on i (along d) and on j (against d)
  if (rb < umax64(Bi.T, Bj.T)) {            // precheck candidate: near field, recorded
    if (rb < umax64(Bi.Q, Bj.Q)) {          // inside the changeover zone (rare): the weight needs r
      double wB, wA;
      changeover_w(r2 * rsqrt_refined(r2), pmin(Bi.A, Bj.A), P.kmode, wB, wA);
      gi *= wB; gj *= wB;
    }
    ai.mask |= 1ULL << uj; aj.mask |= 1ULL << ui;
    ai.n0 = fma(gi, dx, ai.n0); ai.n1 = fma(gi, dy, ai.n1); ai.n2 = fma(gi, dz, ai.n2);
    aj.n0 = fma(-gj, dx, aj.n0); aj.n1 = fma(-gj, dy, aj.n1); aj.n2 = fma(-gj, dz, aj.n2);
  } else {
    ai.f0 = fma(gi, dx, ai.f0); ai.f1 = fma(gi, dy, ai.f1); ai.f2 = fma(gi, dz, ai.f2);
    aj.f0 = fma(-gj, dx, aj.f0); aj.f1 = fma(-gj, dy, aj.f1); aj.f2 = fma(-gj, dz, aj.f2);
  }
}

// Body i's far field, candidates and (CLOSE) velocity from its sums.
template <int MODE>
__device__ __forceinline__ void bk_finish(const Sim &S, int i, const BkAcc &a, double h1, double h2) {
  const int np = S.npad;
  S.afar[i] = a.f0; S.afar[np + i] = a.f1; S.afar[2 * np + i] = a.f2;
  S.bmask[i] = a.mask;
  if (a.mask) atomicAdd((unsigned long long *)&S.counters[C_CAND], (unsigned long long)__popcll(a.mask));
  if (MODE == FIN_INIT) return;
  const double ax = a.f0 + a.n0, ay = a.f1 + a.n1, az = a.f2 + a.n2;
  double vx = fma(h1, ax, S.v[i]), vy = fma(h1, ay, S.v[np + i]), vz = fma(h1, az, S.v[2 * np + i]);
  if (h2 != 0.0) { vx = fma(h2, ax, vx); vy = fma(h2, ay, vy); vz = fma(h2, az, vz); }
  S.v[i] = vx; S.v[np + i] = vy; S.v[2 * np + i] = vz;
}

// The ring of a segment of n bodies (lanes base .. base + n - 1 hold them in Bi; the first is body
// off of its system) over R steps (R >= floor(n/2); the steps past floor(n/2) only rotate): the
// i-side sums in ai, the j-side sums returned to their owners and added.
__device__ __forceinline__ void bk_ring(const DevParams &P, const BkBody &Bi, int base, int n, int off, int R,
                                        BkAcc &ai) {
  const int lane = threadIdx.x & 31, u = lane - base;
  const bool own = u >= 0 && u < n;
  const int src = own ? base + (u + 1 == n ? 0 : u + 1) : lane;
  BkBody Bj = Bi;
  BkAcc aj;
  bk_zero(aj);
  int jb = own ? u : 0;
  for (int s = 1; s <= R; ++s) {
    bk_shfl(Bj, src);
    bk_acc_shfl(aj, src);
    jb = (jb + 1 == n) ? 0 : jb + 1;  // lane u now holds body (u + s) mod n
    const bool act = own && (2 * s < n || (2 * s == n && u < s));
    bk_pair(P, Bi, Bj, off + u, off + jb, act, ai, aj);
  }
  const int back = own ? base + (u + n - R % n) % n : lane;  // body u's j sums are R lanes on
  bk_acc_shfl(aj, back);
  if (own) bk_acc_add(ai, aj);
}

template <int MODE>
__global__ void k_b_kick_sym(Sim S, DevParams P, double h1, double h2) {
  const int lane = threadIdx.x & 31;
  const int nwarp = (gridDim.x * blockDim.x) >> 5;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < S.nkjobs; k += nwarp) {
    const int s0 = S.kjobs[2 * k], code = S.kjobs[2 * k + 1], W = code >> 8, cnt = code & 255;
    if (W <= 32) {  // segments of W lanes, one system each
      const int seg = lane / W, base = seg * W;
      int st = 0, n = 0;
      if (seg < cnt) { st = S.sys_start[s0 + seg]; n = S.sys_start[s0 + seg + 1] - st; }
      const int u = lane - base;
      const bool own = u < n;
      BkBody Bi;
      bk_load(S, own ? st + u : -1, Bi);
      BkAcc ai;
      bk_zero(ai);
      const int R = (S.sys_start[s0 + 1] - S.sys_start[s0]) >> 1;  // the pack's first system is its largest
      bk_ring(P, Bi, base, n, 0, R, ai);
      if (own && Bi.al) bk_finish<MODE>(S, st + u, ai, h1, h2);
    } else {  // one system of 33..64 bodies: blocks A = 0..31, B = 32..n-1
      const int st = S.sys_start[s0], nB = S.sys_start[s0 + 1] - st - 32;
      BkBody Ba, Bb;
      bk_load(S, st + lane, Ba);
      bk_load(S, lane < nB ? st + 32 + lane : -1, Bb);
      BkAcc aa, ab;
      bk_zero(aa);
      bk_zero(ab);
      bk_ring(P, Ba, 0, 32, 0, 16, aa);
      bk_ring(P, Bb, 0, nB, 32, nB >> 1, ab);
      // cross pairs: lane l starts with B body l mod Pp and meets B body (l + s) mod Pp at step s
      int Pp = 1;
      while (Pp < nB) Pp <<= 1;
      BkBody Bj = Bb;
      bk_shfl(Bj, lane & (Pp - 1));
      BkAcc aj;
      bk_zero(aj);
      const int src = (lane + 1) & 31;
      for (int s = 0; s < Pp; ++s) {
        const int b = (lane + s) & (Pp - 1);
        bk_pair(P, Ba, Bj, lane, 32 + b, b < nB, aa, aj);
        bk_shfl(Bj, src);
        bk_acc_shfl(aj, src);
      }
      // lane l holds one replica of B body l mod Pp's sums: add the 32 / Pp replicas
      for (int o = Pp; o < 32; o <<= 1) {
        BkAcc t = aj;
        bk_acc_shfl(t, lane ^ o);
        bk_acc_add(aj, t);
      }
      if (lane < nB) bk_acc_add(ab, aj);
      if (Ba.al) bk_finish<MODE>(S, st + lane, aa, h1, h2);
      if (lane < nB && Bb.al) bk_finish<MODE>(S, st + 32 + lane, ab, h1, h2);
    }
  }
}

// Momentum of every system (one warp per system, fixed order).
__global__ void k_b_momentum(Sim S, double *out) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= S.nsys) return;
  const int st = S.sys_start[s], en = S.sys_start[s + 1], np = S.npad;
  double p[3] = {0.0, 0.0, 0.0};
  for (int j = st + lane; j < en; j += 32)
    if (S.alive[j]) for (int c = 0; c < 3; ++c) p[c] = fma(S.m[j], S.v[c * np + j], p[c]);
  for (int c = 0; c < 3; ++c) {
    const double q = warp_sum(p[c]);
    if (lane == 0) out[3 * s + c] = q;
  }
}

// Sun drifts (this substep's first with the momentum after the opening kick, and the previous
// substep's second with the momentum before its closing kick), then the Kepler drift.
__global__ void k_b_drift(Sim S, DevParams P, double tau, double h1, double h2, int substep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int first = substep == 0;
  if (i == 0) { *S.ngroups = 0; *S.gtotal = 0; S.flags[2] = substep; }
  if (i < 4) S.bsq[i] = 0u;
  if (i < 8) S.norder[i] = 0;
  if (i < S.npad) S.bsn[i] >>= 1;  // the substep history fades
  if (i >= S.npad) return;
  const int np = S.npad;
  const int s = S.sys_of[i];
  if (first && S.alive[i] && i == S.sys_start[s]) S.sys_flag[s] = 0;  // the opening kick used it
  S.fail[i] = 0;
  if (!S.alive[i]) return;
  const double m0 = S.sys_m0[s], im0 = sys_inv(m0), mu = P.G * m0;
  double sh[3];
  for (int c = 0; c < 3; ++c) {
    double a = h1 * S.sys_ppost[3 * s + c];
    if (h2 != 0.0) a = fma(h2, S.sys_ppre[3 * s + c], a);
    sh[c] = a * im0;
  }
  double x = S.x[i] + sh[0], y = S.x[np + i] + sh[1], z = S.x[2 * np + i] + sh[2];
  double vx = S.v[i], vy = S.v[np + i], vz = S.v[2 * np + i];
  S.x0[i] = x; S.x0[np + i] = y; S.x0[2 * np + i] = z;
  S.v0[i] = vx; S.v0[np + i] = vy; S.v0[2 * np + i] = vz;
  int it = 0;
  if (kepler_drift_dev(mu, 2.0 * mu, x, y, z, vx, vy, vz, tau, P.kepler_maxit, &it)) {
    atomicOr(S.status, ST_KEPLER_FALLBACK);
    atomicAdd((unsigned long long *)&S.counters[C_KFALL], 1ULL);
    S.fail[i] = 1;
  }
  S.x[i] = x; S.x[np + i] = y; S.x[2 * np + i] = z;
  S.v[i] = vx; S.v[np + i] = vy; S.v[2 * np + i] = vz;
}

// Encounter search over each body's candidates with a larger index (Hermite, bit-exact).
// Encounter test of the candidate pairs (i, j > i within a system): each CTA gathers the pairs of
// its 128 bodies in shared memory and tests one per thread (a thread per body would issue the FP64
// Hermite test for the few lanes that have a candidate); the same arithmetic, so the same masks.
constexpr int BENC_THREADS = 128;
constexpr int BENC_CAP = 1024;  // gathered pairs per CTA; further pairs are tested where found
__global__ void __launch_bounds__(BENC_THREADS) k_b_encounter(Sim S, double tau) {
  __shared__ u64 s_em[BENC_THREADS];
  __shared__ int s_i[BENC_CAP];
  __shared__ unsigned char s_b[BENC_CAP];
  __shared__ int s_n, s_cnt;
  const int tid = threadIdx.x, i0 = blockIdx.x * BENC_THREADS, np = S.npad;
  s_em[tid] = 0ULL;
  if (tid == 0) { s_n = 0; s_cnt = 0; }
  __syncthreads();
  auto test = [&](int i, int b) {  // pair (i, system index b > i's): sets the bit in i's mask
    const int j = S.sys_start[S.sys_of[i]] + b;
    if (!S.alive[j]) return;
    const double rcij = pmax(S.rc[i], S.rc[j]);
    const double thr = __dmul_rn(rcij, rcij);
    const double dmin = hermite_min_capped(
        __dsub_rn(S.x0[j], S.x0[i]), __dsub_rn(S.x0[np + j], S.x0[np + i]), __dsub_rn(S.x0[2 * np + j], S.x0[2 * np + i]),
        __dsub_rn(S.v0[j], S.v0[i]), __dsub_rn(S.v0[np + j], S.v0[np + i]), __dsub_rn(S.v0[2 * np + j], S.v0[2 * np + i]),
        __dsub_rn(S.x[j], S.x[i]), __dsub_rn(S.x[np + j], S.x[np + i]), __dsub_rn(S.x[2 * np + j], S.x[2 * np + i]),
        __dsub_rn(S.v[j], S.v[i]), __dsub_rn(S.v[np + j], S.v[np + i]), __dsub_rn(S.v[2 * np + j], S.v[2 * np + i]), tau, thr);
    if (dmin < thr) atomicOr(&s_em[i - i0], 1ULL << b);
  };
  const int i = i0 + tid;
  if (i < np && S.alive[i]) {
    const int li = i - S.sys_start[S.sys_of[i]];
    u64 bits = S.bmask[i] & (li >= 63 ? 0ULL : (~0ULL << (li + 1)));
    while (bits) {
      const int b = __ffsll((long long)bits) - 1;
      bits &= bits - 1;
      const int p = atomicAdd(&s_n, 1);
      if (p < BENC_CAP) { s_i[p] = i; s_b[p] = (unsigned char)b; }
      else test(i, b);
    }
  }
  __syncthreads();
  const int n = s_n < BENC_CAP ? s_n : BENC_CAP;
  for (int p = tid; p < n; p += BENC_THREADS) test(s_i[p], s_b[p]);
  __syncthreads();
  if (i < np) {
    const u64 em = s_em[tid];
    S.emask[i] = em;
    if (em) atomicAdd(&s_cnt, __popcll(em));
  }
  __syncthreads();
  if (tid == 0 && s_cnt) atomicAdd((unsigned long long *)&S.counters[C_ENC], (unsigned long long)s_cnt);
}

// Groups of one system per warp: union of encounter pairs by atomicMin on local links, then
// each root becomes a group (members ascending) appended to the global group list.
constexpr int BG_WARPS = 4;
__global__ void __launch_bounds__(32 * BG_WARPS) k_b_group(Sim S) {
  __shared__ int link_s[BG_WARPS][64];
  __shared__ int cnt_s[BG_WARPS][64];
  __shared__ int pos_s[BG_WARPS][64];
  __shared__ unsigned char part_s[BG_WARPS][64];
  __shared__ int hist_s[BG_WARPS][64];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * BG_WARPS + w;
  if (s >= S.nsys) return;  // warp-uniform
  int *link = link_s[w], *cnt = cnt_s[w], *pos = pos_s[w];
  unsigned char *part = part_s[w];
  const int st = S.sys_start[s], n = S.sys_start[s + 1] - st;
  int *hist = hist_s[w];
  for (int k = lane; k < 64; k += 32) { link[k] = k; cnt[k] = 0; part[k] = 0; hist[k] = 0; }
  __syncwarp();
  for (int k = lane; k < n; k += 32) {
    const u64 em = S.emask[st + k];
    if (em || S.fail[st + k]) part[k] = 1;
    u64 bits = em;
    while (bits) { const int b = __ffsll((long long)bits) - 1; bits &= bits - 1; part[b] = 1; }
  }
  __syncwarp();
  bool any = false;
  for (int k = lane; k < n; k += 32) any |= part[k] != 0;
  if (!__any_sync(0xffffffffu, any)) return;
  for (int round = 0; round < 64; ++round) {
    bool ch = false;
    for (int k = lane; k < n; k += 32) {
      u64 bits = S.emask[st + k];
      while (bits) {
        const int b = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        int ru = k, rv = b;
        for (int q = 0; q < 66 && link[ru] != ru; ++q) ru = link[ru];
        for (int q = 0; q < 66 && link[rv] != rv; ++q) rv = link[rv];
        if (ru != rv) { atomicMin(&link[ru > rv ? ru : rv], ru < rv ? ru : rv); ch = true; }
      }
    }
    __syncwarp();
    for (int k = lane; k < n; k += 32) {
      int r = k;
      for (int q = 0; q < 66 && link[r] != r; ++q) r = link[r];
      link[k] = r;
    }
    __syncwarp();
    if (!__any_sync(0xffffffffu, ch)) break;
  }
  for (int k = lane; k < n; k += 32)
    if (part[k]) {
      atomicAdd(&cnt[link[k]], 1);
      atomicMax(&hist[link[k]], (int)S.bsn[st + k]);
    }
  __syncwarp();
  if (lane == 0) {
    int ng = 0;
    for (int r = 0; r < n; ++r)
      if (part[r] && link[r] == r) {
        const int g = atomicAdd(S.ngroups, 1);
        const int p = atomicAdd(S.gtotal, cnt[r]);
        S.gstart[g] = p;
        S.gsize[g] = cnt[r];
        // the queue of the kernel that integrates the group; groups whose members needed many
        // substeps last time start first (they set the BS time)
        const int qi = cnt[r] <= 2 ? 0 : (cnt[r] <= BS_SMALL ? 1 : (cnt[r] <= BS_GMAX ? 2 : 3));
        int *qo = S.gorder + (size_t)qi * S.npad;
        if (hist[r] >= BS_HEAVY) qo[atomicAdd(&S.norder[2 * qi], 1)] = g;
        else qo[S.npad - 1 - atomicAdd(&S.norder[2 * qi + 1], 1)] = g;
        pos[r] = p;
        ng++;
      }
    if (ng) atomicAdd((unsigned long long *)&S.counters[C_GROUPS], (unsigned long long)ng);
  }
  __syncwarp();
  for (int k = lane; k < n; k += 32) {
    if (!part[k]) continue;
    const int r = link[k];
    int rank = 0;
    for (int q = 0; q < k; ++q) rank += (part[q] && link[q] == r) ? 1 : 0;
    S.gmem[pos[r] + rank] = st + k;
  }
}

// Second Sun drift of the last substep.
__global__ void k_b_hc(Sim S, double h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.npad || !S.alive[i]) return;
  const int s = S.sys_of[i], np = S.npad;
  const double im0 = sys_inv(S.sys_m0[s]);
  for (int c = 0; c < 3; ++c) S.x[c * np + i] = fma(h * S.sys_ppre[3 * s + c], im0, S.x[c * np + i]);
}

// State conversions (user order <-> internal order, heliocentric <-> democratic), one warp per
// system. perm[internal body] = user body, sys_user[internal system] = user system.
__global__ void k_b_from_helio(Sim S, DevParams P, const int *perm, const double *xh, const double *vh,
                               const double *m_in, const double *R_in, int keep) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= S.nsys) return;
  const int st = S.sys_start[s], en = S.sys_start[s + 1], np = S.npad;
  const double m0 = S.sys_m0[s];
  double p[3] = {0.0, 0.0, 0.0}, mt = 0.0;
  for (int j = st + lane; j < en; j += 32) {
    const int u = perm[j];
    const double mj = keep ? (S.alive[j] ? S.m[j] : 0.0) : m_in[u];
    mt += mj;
    for (int c = 0; c < 3; ++c) p[c] = fma(mj, vh[3 * u + c], p[c]);
  }
  mt = warp_sum(mt);
  for (int c = 0; c < 3; ++c) p[c] = warp_sum(p[c]) / (m0 + mt);
  for (int j = st + lane; j < en; j += 32) {
    const int u = perm[j];
    if (keep && !S.alive[j]) continue;
    for (int c = 0; c < 3; ++c) {
      S.x[c * np + j] = xh[3 * u + c];
      S.v[c * np + j] = vh[3 * u + c] - p[c];
    }
    if (!keep) {
      const double mj = m_in[u];
      S.m[j] = mj; S.gm[j] = P.G * mj; S.R[j] = R_in[u];
      S.hill[j] = cbrt(mj / (3.0 * m0));
      S.alive[j] = 1;
    }
  }
}

__global__ void k_b_to_helio(Sim S, const int *perm, double *xh, double *vh, double *m_out, double *R_out,
                             int *alive_out) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= S.nsys) return;
  const int st = S.sys_start[s], en = S.sys_start[s + 1], np = S.npad;
  const double im0 = 1.0 / S.sys_m0[s];
  double p[3] = {0.0, 0.0, 0.0};
  for (int j = st + lane; j < en; j += 32)
    if (S.alive[j]) for (int c = 0; c < 3; ++c) p[c] = fma(S.m[j], S.v[c * np + j], p[c]);
  for (int c = 0; c < 3; ++c) p[c] = warp_sum(p[c]);
  for (int j = st + lane; j < en; j += 32) {
    const int u = perm[j];
    for (int c = 0; c < 3; ++c) {
      if (xh) xh[3 * u + c] = S.x[c * np + j];
      if (vh) vh[3 * u + c] = fma(p[c], im0, S.v[c * np + j]);
    }
    if (m_out) m_out[u] = S.m[j];
    if (R_out) R_out[u] = S.R[j];
    if (alive_out) alive_out[u] = S.alive[j];
  }
}

// Energy of each system in democratic coordinates (one warp per system, fixed order).
__global__ void k_b_energy(Sim S, DevParams P, const int *sys_user, double *E) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= S.nsys) return;
  const int st = S.sys_start[s], en = S.sys_start[s + 1], n = en - st, np = S.npad;
  const double m0 = S.sys_m0[s];
  double e = 0.0, p[3] = {0.0, 0.0, 0.0};
  for (int j = st + lane; j < en; j += 32) {
    if (!S.alive[j]) continue;
    const double x = S.x[j], y = S.x[np + j], z = S.x[2 * np + j];
    const double vx = S.v[j], vy = S.v[np + j], vz = S.v[2 * np + j];
    e += 0.5 * S.m[j] * (vx * vx + vy * vy + vz * vz) - P.G * m0 * S.m[j] / sqrt(x * x + y * y + z * z);
    p[0] = fma(S.m[j], vx, p[0]); p[1] = fma(S.m[j], vy, p[1]); p[2] = fma(S.m[j], vz, p[2]);
  }
  for (int k = lane; k < n * n; k += 32) {
    const int a = k / n, b = k % n;
    if (b <= a) continue;
    const int ja = st + a, jb = st + b;
    if (!S.alive[ja] || !S.alive[jb]) continue;
    const double dx = S.x[jb] - S.x[ja], dy = S.x[np + jb] - S.x[np + ja], dz = S.x[2 * np + jb] - S.x[2 * np + ja];
    e -= P.G * S.m[ja] * S.m[jb] / sqrt(dx * dx + dy * dy + dz * dz);
  }
  e = warp_sum(e);
  for (int c = 0; c < 3; ++c) p[c] = warp_sum(p[c]);
  if (lane == 0) E[sys_user[s]] = e + (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) / (2.0 * m0);
}

// ---------------------------------------------------------------------------------------------
void launch_b_rcrit(const Sim &S, const DevParams &P, double tau_abs, int check, cudaStream_t st) {
  k_b_rcrit<<<(S.npad + 127) / 128, 128, 0, st>>>(S, P, tau_abs, check);
}

template <int MODE>
static void b_kick_split(const Sim &S, const DevParams &P, double h1, double h2, int split, int block, cudaStream_t st) {
  if (split == 0) {  // Newton's third law, one warp per work item (CLOSE / INIT; OPEN takes split 1)
    if constexpr (MODE != FIN_OPEN) {
      const int grid = (int)(((long)S.nkjobs * 32 + block - 1) / block);
      k_b_kick_sym<MODE><<<grid > 0 ? grid : 1, block, 0, st>>>(S, P, h1, h2);
      return;
    }
    split = 1;
  }
  const long threads = (long)S.npad * split;
  const int grid = (int)((threads + block - 1) / block);
  if (split == 1) k_b_kick<MODE, 1><<<grid, block, 0, st>>>(S, P, h1, h2);
  else if (split == 2) k_b_kick<MODE, 2><<<grid, block, 0, st>>>(S, P, h1, h2);
  else k_b_kick<MODE, 4><<<grid, block, 0, st>>>(S, P, h1, h2);
}

void launch_b_kick(const Sim &S, const DevParams &P, FinMode mode, double h1, double h2, int split, int block,
                   cudaStream_t st) {
  if (mode == FIN_CLOSE) b_kick_split<FIN_CLOSE>(S, P, h1, h2, split, block, st);
  else if (mode == FIN_OPEN) b_kick_split<FIN_OPEN>(S, P, h1, h2, split, block, st);
  else b_kick_split<FIN_INIT>(S, P, h1, h2, split, block, st);
}

void launch_b_momentum(const Sim &S, double *out, cudaStream_t st) {
  k_b_momentum<<<(S.nsys * 32 + 127) / 128, 128, 0, st>>>(S, out);
}
void launch_b_drift(const Sim &S, const DevParams &P, double tau, double h1, double h2, int substep, cudaStream_t st) {
  k_b_drift<<<(S.npad + 127) / 128, 128, 0, st>>>(S, P, tau, h1, h2, substep);
}
void launch_b_encounter(const Sim &S, double tau, cudaStream_t st) {
  k_b_encounter<<<(S.npad + BENC_THREADS - 1) / BENC_THREADS, BENC_THREADS, 0, st>>>(S, tau);
}
void launch_b_group(const Sim &S, cudaStream_t st) {
  k_b_group<<<(S.nsys + BG_WARPS - 1) / BG_WARPS, 32 * BG_WARPS, 0, st>>>(S);
}
void launch_b_hc(const Sim &S, double h, cudaStream_t st) { k_b_hc<<<(S.npad + 127) / 128, 128, 0, st>>>(S, h); }
void launch_b_from_helio(const Sim &S, const DevParams &P, const int *perm, const double *xh, const double *vh,
                         const double *m_in, const double *R_in, int keep, cudaStream_t st) {
  k_b_from_helio<<<(S.nsys * 32 + 127) / 128, 128, 0, st>>>(S, P, perm, xh, vh, m_in, R_in, keep);
}
void launch_b_to_helio(const Sim &S, const int *perm, double *xh, double *vh, double *m_out, double *R_out,
                       int *alive_out, cudaStream_t st) {
  k_b_to_helio<<<(S.nsys * 32 + 127) / 128, 128, 0, st>>>(S, perm, xh, vh, m_out, R_out, alive_out);
}
void launch_b_energy(const Sim &S, const DevParams &P, const int *sys_user, double *E, cudaStream_t st) {
  k_b_energy<<<(S.nsys * 32 + 127) / 128, 128, 0, st>>>(S, P, sys_user, E);
}

}  // namespace genga
