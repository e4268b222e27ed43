// bs.cu -- Bulirsch-Stoer integration of the encounter groups (Sect. 3.2) with perfect merging
// on contact (Sect. 3.2, Collisions).
//
// k_bs: one CTA per group. The modified-midpoint integrations of all extrapolation levels
// (n_k = 2k, k = 1..8) run at once: thread (level, member, term) evaluates one term of the
// member's acceleration (the central mass or one partner). Level L completes after 2L force
// evaluations; its tableau row is built and tested right away, and the attempt stops at the first
// converged level -- exactly the decision of the serial algorithm, at 2L + 1 evaluations instead
// of the serial scheme's 72. Batched groups come from work queues ordered by expected cost: groups
// of 3..BS_SMALL members from queue 1 on 128-thread CTAs, larger ones from queue 2 on 256 threads.
// k_bs_pair: groups of one or two members, one warp per attempt, the attempt at H/2 run beside the
// attempt at H (see there).
#include "bs_core.cuh"

namespace genga {

// Batched mode: the q-th group of BS queue qi (the expected long ones first); past its end: done.
__device__ __forceinline__ int batch_group(const Sim &S, int qi, int q) {
  const int nfront = S.norder[2 * qi], n = nfront + S.norder[2 * qi + 1];
  if (q >= n) return 0x7fffffff;
  const int *qo = S.gorder + (size_t)qi * S.npad;
  return qo[q < nfront ? q : S.npad - 1 - (q - nfront)];
}

// NT threads: 256, or 128 for the batched queue of groups of 3 .. BS_SMALL members (BS_LEVELS x g
// slots of four threads fill 128), so that two CTAs fit where one of 256 would, or 512 for groups
// of BS_GMAX + 1 .. BS_GWIDE members (one thread a slot; the state, GM = BS_GWIDE, in dynamic
// shared memory). The kernel integrates the groups of gmin .. gsplit - 1 members that it meets and
// reports larger ones than GM; it takes its groups from batched queue qi, else from the
// large-group list (from_big), else every group with a fixed stride.
template <int NT, int GM>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : 512 / NT)
    k_bs(Sim S, DevParams P, double tau, int gmin, int gsplit, int qi, int from_big) {
  __shared__ __align__(16) unsigned char bs_static[GM <= BS_GMAX ? sizeof(BsSharedT<GM>) : 16];
  extern __shared__ __align__(16) unsigned char bs_dyn[];
  BsSharedT<GM> &sh = *reinterpret_cast<BsSharedT<GM> *>(GM <= BS_GMAX ? bs_static : bs_dyn);
  const int tid = threadIdx.x;
  const int ngroups = *S.ngroups;
  for (int it = 0;; ++it) {
    // next group: from the queue when there is one (batched mode), else a fixed stride
    if (tid == 0) {
      int nx = blockIdx.x + it * gridDim.x;
      if (S.bsq) nx = batch_group(S, qi, (int)atomicAdd(&S.bsq[qi], 1u));
      else if (from_big) nx = nx < *S.nbig ? S.big[nx] : 0x7fffffff;
      sh.next = nx;
    }
    __syncthreads();
    const int gidx = sh.next;
    __syncthreads();
    if (gidx >= ngroups) break;  // uniform
    const int g0 = S.gstart[gidx], g = S.gsize ? S.gsize[gidx] : S.gstart[gidx + 1] - g0;
    // central mass of the group's system (batched mode) or of the single system
    const double m0 = S.sys_of ? S.sys_m0[S.sys_of[S.gmem[g0]]] : P.m0;
    if (g < gmin || g >= gsplit) continue;  // uniform: the pair, cluster or wide kernel's
    if (g > GM || (GM > BS_GMAX && S.seq_len)) {  // the adjoint's recording holds BS_GMAX members
      if (tid == 0) atomicOr(S.status, ST_GROUP_TOO_LARGE);
      continue;  // uniform across the CTA
    }
    bs_group<NT, GM>(sh, S, P, tau, gidx, g0, g, m0, -1, -1, blockIdx.x);
  }
}

static_assert(BS_WIDE_THREADS == BS_LEVELS * BS_GWIDE, "one thread per (level, member) slot");

void bs_init_constants() {
  cudaFuncSetAttribute(k_bs<BS_WIDE_THREADS, BS_GWIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(BsSharedT<BS_GWIDE>));
  bs_core_set_factors();
}

void launch_bs(const Sim &S, const DevParams &P, double tau, int max_groups, cudaStream_t st, int gsplit, int gmin) {
  const int grid = max_groups < 1 ? 1 : max_groups;
  k_bs<BS_THREADS, BS_GMAX><<<grid, BS_THREADS, 0, st>>>(S, P, tau, gmin, gsplit, 2, 0);
}
void launch_bs_small(const Sim &S, const DevParams &P, double tau, int blocks, cudaStream_t st) {
  k_bs<128, BS_GMAX><<<blocks < 1 ? 1 : blocks, 128, 0, st>>>(S, P, tau, 3, BS_SMALL + 1, 1, 0);
}
void launch_bs_wide(const Sim &S, const DevParams &P, double tau, int blocks, cudaStream_t st) {
  k_bs<BS_WIDE_THREADS, BS_GWIDE><<<blocks < 1 ? 1 : blocks, BS_WIDE_THREADS, sizeof(BsSharedT<BS_GWIDE>), st>>>(
      S, P, tau, BS_GMAX + 1, 0x7fffffff, 3, 1);
}

// ---------------------------------------------------------------------------------------------
// Groups of one or two members (the common case in systems with many bodies): one unit of two warps
// per group, four groups per CTA. Lane l of a warp: level l/4 + 1, member (l/2) % 2, term l % 2 (the
// central mass or the partner); the same arithmetic and decisions as k_bs.
//
// Speculation. The step control halves H on failure and doubles it on acceptance, so a long
// integration alternates a failed attempt at 2H with an accepted one at H. The unit's first warp
// attempts H while the second attempts H/2 from the same state; the second result is used exactly
// when the serial algorithm's next attempt would be that one (the first failed), so every result
// and decision equals the serial algorithm's, and a fail/accept pair costs one attempt's time.
// ---------------------------------------------------------------------------------------------
constexpr int BSP_UNITS = 4;

struct BsPairShared {
  int idx[2], alive[2];
  double gm[2], m[2], R[2], A[2];
  u64 rcsq[2];
  double y[2][6];                     // state at the start of the round
  double yn[2][2][6];                 // [warp] result of the warp's attempt
  double pos[2][2][BS_LEVELS][2][3];  // [warp][buffer][level][member]
  double zt[2][BS_LEVELS][2][16];     // [warp] a level's last midpoint state: z_{n-1}, z_n, a(z_n), h
  u64 err[2][BS_LEVELS];              // [warp]
  int acc[2];
  int gidx;
  double U;
};

// the two warps of a unit (named barrier 1 + unit, 64 threads)
__device__ __forceinline__ void unit_sync(int bar) { asm volatile("bar.sync %0, 64;" ::"r"(bar) : "memory"); }

// One lane's term (the central mass if p == q, else partner p) with what stays fixed over an
// attempt: the source's G m, the smaller A = 1/(0.9 rc), the larger rc^2 (bits) and the partner's
// live flag; only the positions change between evaluations.
struct PairTerm {
  double pref, Amin;
  u64 thr;
  bool cen, palive, has;
};

__device__ __forceinline__ PairTerm pair_term(const BsPairShared &sh, double Gm0, int g, int q, int p) {
  PairTerm t;
  t.has = p < g;
  const int pp = t.has ? p : q;
  t.cen = p == q;
  t.pref = t.cen ? Gm0 : sh.gm[pp];
  t.Amin = pmin(sh.A[q], sh.A[pp]);
  t.thr = umax64(sh.rcsq[q], sh.rcsq[pp]);
  t.palive = sh.alive[pp] != 0;
  return t;
}

__device__ __forceinline__ void pair_terms(const PairTerm &t, const DevParams &P, int q, int p, const double (*pos)[3],
                                           bool q_alive, double &ax, double &ay, double &az) {
  ax = ay = az = 0.0;
  if (q_alive && t.has) {
    const double xq = pos[q][0], yq = pos[q][1], zq = pos[q][2];
    const bool cen = t.cen;
    const double dx = (cen ? 0.0 : pos[p][0]) - xq, dy = (cen ? 0.0 : pos[p][1]) - yq, dz = (cen ? 0.0 : pos[p][2]) - zq;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const double yr = rsqrt_refined(r2);
    const bool inside = t.palive && dbits(r2) < t.thr;
    const double wA = changeover_wA_clamped(r2 * yr, t.Amin, P.kmode);
    const double w = cen ? 1.0 : (inside ? wA : 0.0);
    const double f = t.pref * w * (yr * yr * yr);
    ax = f * dx; ay = f * dy; az = f * dz;
  }
  ax += __shfl_xor_sync(0xffffffffu, ax, 1);
  ay += __shfl_xor_sync(0xffffffffu, ay, 1);
  az += __shfl_xor_sync(0xffffffffu, az, 1);
}

// One attempt of length H from sh.y by one warp, with the warp's own buffers (index w). Returns the
// accepted level (0: no level converged) and leaves the extrapolated state in sh.yn[w].
__device__ int pair_attempt(BsPairShared &sh, int w, const DevParams &P, double Gm0, int g, double H, int lane) {
  const int slot = lane >> 1, sub = lane & 1;
  const int lev = slot >> 1, q = slot & 1, L = lev + 1, nk = 2 * L;
  const bool act = q < g;
  const double h = __ddiv_rn(H, (double)nk), h2 = 2.0 * h;
  const bool qa = act && sh.alive[q];
  double zA[6], zB[6];
  for (int c = 0; c < 6; ++c) zA[c] = act ? sh.y[q][c] : 0.0;
  if (act && sub == 0) for (int c = 0; c < 3; ++c) sh.pos[w][0][lev][q][c] = zA[c];
  const int qc = lane / 6, cc = lane % 6;
  const bool rowth = qc < g;
  double scale = 0.0;
  if (rowth) {
    const double *yq = sh.y[qc] + (cc < 3 ? 0 : 3);
    const double s2 = fma(yq[2], yq[2], fma(yq[1], yq[1], yq[0] * yq[0]));
    scale = dbits(s2) == 0ULL ? 4.49423283715579e307 : rsqrt_refined(s2);
  }
  if (lane < BS_LEVELS) sh.err[w][lane] = 0ULL;
  __syncwarp();
  const int qq = act ? q : 0;
  const PairTerm term = pair_term(sh, Gm0, g, qq, sub);
  double ax, ay, az;
  pair_terms(term, P, qq, sub, sh.pos[w][0][lev], qa, ax, ay, az);
  if (qa) {
    zB[0] = fma(h, zA[3], zA[0]); zB[1] = fma(h, zA[4], zA[1]); zB[2] = fma(h, zA[5], zA[2]);
    zB[3] = fma(h, ax, zA[3]); zB[4] = fma(h, ay, zA[4]); zB[5] = fma(h, az, zA[5]);
  } else {
    for (int c = 0; c < 6; ++c) zB[c] = zA[c];
  }
  const int lmax = P.bs_kmax < BS_LEVELS ? P.bs_kmax : BS_LEVELS;
  const u64 eps = dbits(P.bs_eps);
  double prev[BS_LEVELS], tlast = 0.0;  // previous tableau row; T_{Lc,Lc} of the current one
  int acc = 0, b = 1;
  for (int e = 1; e <= 2 * lmax; ++e) {
    const bool lv = act && e <= nk;
    if (lv && sub == 0) for (int c = 0; c < 3; ++c) sh.pos[w][b][lev][q][c] = zB[c];
    __syncwarp();
    pair_terms(term, P, qq, sub, sh.pos[w][b][lev], qa && e <= nk, ax, ay, az);
    if (lv) {
      if (qa && e < nk) {
        double zn[6];
        zn[0] = fma(h2, zB[3], zA[0]); zn[1] = fma(h2, zB[4], zA[1]); zn[2] = fma(h2, zB[5], zA[2]);
        zn[3] = fma(h2, ax, zA[3]); zn[4] = fma(h2, ay, zA[4]); zn[5] = fma(h2, az, zA[5]);
        for (int c = 0; c < 6; ++c) { zA[c] = zB[c]; zB[c] = zn[c]; }
      }
      // the level's chain is done: its tableau lanes form T_{L,1} = (z_{n-1} + z_n + h z'_n) / 2,
      // one component each, so the warp issues that arithmetic once instead of per level lane
      if (e == nk && sub == 0) {
        double *z = sh.zt[w][lev][q];
        for (int c = 0; c < 6; ++c) { z[c] = zA[c]; z[6 + c] = zB[c]; }
        z[12] = ax; z[13] = ay; z[14] = az; z[15] = h;
      }
    }
    b ^= 1;
    if (e & 1) continue;
    const int Lc = e >> 1;  // level Lc is complete: its tableau row (Neville, in h^2)
    __syncwarp();
    if (rowth) {
      const double *z = sh.zt[w][Lc - 1][qc];
      const double dz = cc < 3 ? z[9 + cc] : z[12 + cc - 3];  // derivative of component cc at z_n
      const double t1 = sh.alive[qc] ? 0.5 * fma(z[15], dz, z[6 + cc] + z[cc]) : z[cc];
      double before;
      tlast = neville_row(t1, Lc, [&](int j) { return c_facinv[Lc][j]; }, prev, before);
      if (Lc >= 2 && sh.alive[qc]) atomicMax(&sh.err[w][Lc - 1], absbits((tlast - before) * scale));
    }
    __syncwarp();
    if (Lc >= 2 && sh.err[w][Lc - 1] <= eps) { acc = Lc; break; }
  }
  if (acc && rowth) sh.yn[w][qc][cc] = tlast;  // the accepted row is the last one built
  __syncwarp();
  return acc;
}

__global__ void __launch_bounds__(64 * BSP_UNITS, 2) k_bs_pair(Sim S, DevParams P, double tau) {
  __shared__ BsPairShared shu[BSP_UNITS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, unit = wid >> 1, spec = wid & 1;
  const int bar = 1 + unit;
  BsPairShared &sh = shu[unit];
  auto usync = [&]() { unit_sync(bar); };
  const int np = S.npad;
  const int ngroups = *S.ngroups;
  for (int it = 0;; ++it) {
    // next group: from the queue when there is one, else a fixed stride
    if (spec == 0 && lane == 0)
      sh.gidx = S.bsq ? batch_group(S, 0, (int)atomicAdd(&S.bsq[0], 1u)) : (blockIdx.x + it * gridDim.x) * BSP_UNITS + unit;
    usync();
    const int gidx = sh.gidx;
    if (gidx >= ngroups) break;  // uniform within the unit
    const int g0 = S.gstart[gidx], g = S.gsize ? S.gsize[gidx] : S.gstart[gidx + 1] - g0;
    if (g > 2) { usync(); continue; }  // uniform within the unit
    const double m0 = S.sys_of ? S.sys_m0[S.sys_of[S.gmem[g0]]] : P.m0;
    const double Gm0 = P.G * m0;
    if (spec == 0) {
      if (lane < g) {
        const int i = S.gmem[g0 + lane];
        sh.idx[lane] = i;
        sh.alive[lane] = S.alive[i];
        sh.gm[lane] = S.gm[i]; sh.m[lane] = S.m[i]; sh.R[lane] = S.R[i]; sh.A[lane] = S.A[i];
        sh.rcsq[lane] = S.rcsq[i];
        for (int c = 0; c < 3; ++c) { sh.y[lane][c] = S.x0[c * np + i]; sh.y[lane][3 + c] = S.v0[c * np + i]; }
      }
      if (lane == 0) sh.U = 0.0;
    }
    usync();
    // both warps keep identical copies of the step control
    double H = tau, rem = tau;
    int halvings = 0, attempts = 0, steps = 0;
    bool failed = false;
    while (absbits(rem) != 0ULL) {
      if (absbits(H) > absbits(rem)) H = rem;
      if (++attempts > 200000) { failed = true; break; }
      const int a = pair_attempt(sh, spec, P, Gm0, g, spec ? 0.5 * H : H, lane);
      if (lane == 0) sh.acc[spec] = a;
      usync();
      const int a0 = sh.acc[0], a1 = sh.acc[1];
      int use = 0;
      if (!a0) {  // the serial algorithm halves H and tries again: the second warp's attempt
        H *= 0.5;
        if (++halvings > P.bs_max_halvings) { failed = true; break; }
        if (++attempts > 200000) { failed = true; break; }
        if (!a1) {
          H *= 0.5;
          if (++halvings > P.bs_max_halvings) { failed = true; break; }
          usync();  // both warps have read acc[] before the next round writes it
          continue;
        }
        use = 1;
      }
      // accepted: substep H from sh.y to sh.yn[use]
      if (spec == 0 && P.collisions && g == 2 && lane == 0 && sh.alive[0] && sh.alive[1]) {  // contact over the substep
        double (*yn)[6] = sh.yn[use];
        const double rr = sh.R[0] + sh.R[1];
        const double dmin = hermite_min_capped(
            __dsub_rn(sh.y[1][0], sh.y[0][0]), __dsub_rn(sh.y[1][1], sh.y[0][1]), __dsub_rn(sh.y[1][2], sh.y[0][2]),
            __dsub_rn(sh.y[1][3], sh.y[0][3]), __dsub_rn(sh.y[1][4], sh.y[0][4]), __dsub_rn(sh.y[1][5], sh.y[0][5]),
            __dsub_rn(yn[1][0], yn[0][0]), __dsub_rn(yn[1][1], yn[0][1]), __dsub_rn(yn[1][2], yn[0][2]),
            __dsub_rn(yn[1][3], yn[0][3]), __dsub_rn(yn[1][4], yn[0][4]), __dsub_rn(yn[1][5], yn[0][5]), H, rr * rr);
        if (dmin < rr * rr) {  // perfect merger (Sect. 3.2, Collisions), as in k_bs
          const int ia = sh.idx[0], ib = sh.idx[1];
          const double ma = sh.m[0], mb = sh.m[1], M = ma + mb;
          const double dx = yn[1][0] - yn[0][0], dy = yn[1][1] - yn[0][1], dz = yn[1][2] - yn[0][2];
          const double dvx = yn[1][3] - yn[0][3], dvy = yn[1][4] - yn[0][4], dvz = yn[1][5] - yn[0][5];
          const double r = sqrt(dx * dx + dy * dy + dz * dz);
          const double v2 = dvx * dvx + dvy * dvy + dvz * dvz;
          sh.U += 0.5 * ma * mb / M * v2 - P.G * ma * mb / r;
          const bool keep_a = ma > mb || (ma == mb && ia < ib);
          merger_report(S, ia, ib, sh.y[0], sh.y[1], yn[0], yn[1], ma, mb, keep_a, tau - rem);
          const int sv = keep_a ? 0 : 1, d = keep_a ? 1 : 0;
          for (int c = 0; c < 6; ++c) yn[sv][c] = (ma * yn[0][c] + mb * yn[1][c]) / M;
          const double Ra = sh.R[0], Rb = sh.R[1];
          sh.R[sv] = cbrt(Ra * Ra * Ra + Rb * Rb * Rb);
          sh.m[sv] = M; sh.gm[sv] = P.G * M;
          sh.m[d] = 0.0; sh.gm[d] = 0.0; sh.R[d] = 0.0; sh.alive[d] = 0;
          const int is = sh.idx[sv], idd = sh.idx[d];
          S.m[is] = M; S.gm[is] = P.G * M; S.R[is] = sh.R[sv]; S.hill[is] = cbrt(M / (3.0 * m0));
          S.m[idd] = 0.0; S.gm[idd] = 0.0; S.R[idd] = 0.0; S.hill[idd] = 0.0; S.alive[idd] = 0;
          S.T[idd] = 0ULL; S.rcsq[idd] = 0ULL;
          atomicAdd((unsigned long long *)&S.counters[C_MERGE], 1ULL);
        }
      }
      __syncwarp();
      if (spec == 0 && lane < g) for (int c = 0; c < 6; ++c) sh.y[lane][c] = sh.yn[use][lane][c];
      usync();
      rem -= H;
      H *= 2.0;
      halvings = 0;
      steps++;
    }
    if (spec == 0) {
      if (lane < g && S.bsn) S.bsn[sh.idx[lane]] = (unsigned char)(steps < 255 ? steps : 255);
      if (lane < g) {
        const int i = sh.idx[lane];
        if (sh.alive[lane]) {
          for (int c = 0; c < 3; ++c) { S.x[c * np + i] = sh.y[lane][c]; S.v[c * np + i] = sh.y[lane][3 + c]; }
        } else {
          S.x[i] = PARK + 1.0e4 * i; S.x[np + i] = 0.0; S.x[2 * np + i] = 0.0;
          for (int c = 0; c < 3; ++c) S.v[c * np + i] = 0.0;
        }
      }
      if (lane == 0) {
        if (failed) atomicOr(S.status, ST_BS_FAILED);
        atomicAdd((unsigned long long *)&S.counters[C_BSSTEPS], (unsigned long long)steps);
        if (dbits(sh.U) != 0ULL) atomicAdd(S.U, sh.U);
      }
    }
    usync();  // the group's shared state is free for the next one
  }
}

void launch_bs_pair(const Sim &S, const DevParams &P, double tau, int blocks, cudaStream_t st) {
  k_bs_pair<<<blocks, 64 * BSP_UNITS, 0, st>>>(S, P, tau);
}

}  // namespace genga
