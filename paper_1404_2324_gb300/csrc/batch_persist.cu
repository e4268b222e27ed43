// batch_persist.cu -- the many-systems mode (Sect. 3.4) as one persistent launch.
//
// The step graph of batch.cu advances all systems phase by phase: every step waits for the slowest
// Bulirsch-Stoer group of any system (a tight pair that needs many substeps) before the next phase
// starts anywhere. Here every CTA takes a system from a queue (largest first), holds its state in
// shared memory and advances it through all the steps of the launch on its own: rcrit, the opening
// kick (KickA or a full recompute), per substep the Sun and Kepler drifts, the Hermite encounter
// test, grouping, Bulirsch-Stoer of its groups and the closing kick with the prechecker. A system
// whose groups take long holds only its own CTA; the other CTAs go on with other systems. Each system
// follows exactly the single-system step (the same operations in the same order); only the sums run
// in a different fixed order than in the step graph.
//
// Groups of up to BS_GMAX members use the one-CTA level-parallel BS (bs_core.cuh). Groups of
// BS_GMAX + 1 .. 64 members (rare) take bp_big_group: the same algorithm with the levels run one
// after another, every member's force evaluated by four threads.
#include "bs_core.cuh"

namespace genga {

constexpr int BP_THREADS = 256;
constexpr int BP_N = 64;                        // bodies per system
constexpr int BP_PAIRS = BP_N * (BP_N - 1) / 2;
constexpr int BP_SPLIT = BP_THREADS / BP_N;     // threads per body in the kick (4)

struct BpSys {
  double x[3][BP_N], v[3][BP_N], x0[3][BP_N], v0[3][BP_N], af[3][BP_N];
  double m[BP_N], gm[BP_N], hill[BP_N], rc[BP_N], A[BP_N];
  u64 T[BP_N], rq[BP_N], cm[BP_N], em[BP_N];    // precheck threshold, rc^2, candidate / encounter masks
  int alive[BP_N], fail[BP_N], link[BP_N], cnt[BP_N], gmem[BP_N], gst[BP_N + 1];
  unsigned char pa[BP_PAIRS], pb[BP_PAIRS];    // candidate pairs (a < b) of the encounter test
  double red[BP_THREADS / 32][3];
  double P[3], Ppre[3];
  int flag, npairs, ngroups, sys, nenc, ncand;
};

// groups of BS_GMAX + 1 .. BP_N members
struct BpBig {
  int idx[BP_N], alive[BP_N];
  double gm[BP_N], m[BP_N], R[BP_N], A[BP_N];
  u64 rcsq[BP_N];
  double y[BP_N][6], yn[BP_N][6], za[BP_N][6], zb[BP_N][6], a[BP_N][3], a0[BP_N][3], isc[BP_N][2];
  unsigned char cont[BP_PAIRS];
  u64 err;
  int acc;
};

union BpBs {
  BsSharedT<BS_GMAX> small;
  BpBig big;
};

struct BpArgs {
  double dt;
  double w[7];
  int nsub, nsteps;
  int *step_base;  // steps before this launch (advanced by k_bp_advance after it)
  int *queue;      // next system to take (reset to 0 before every launch)
};

constexpr size_t BP_SYS_BYTES = (sizeof(BpSys) + 15) / 16 * 16;  // the BS area starts 16-byte aligned
constexpr size_t BP_SMEM = BP_SYS_BYTES + sizeof(BpBs);

// H_A acceleration of member q of a big group from positions z[p][0..2] (stride 6): the central
// mass plus the (1 - K)-weighted pull of every live partner, as bs_terms; four threads per member.
__device__ __forceinline__ void bp_big_force(BpBig &sh, const DevParams &P, double Gm0, int g, const double (*z)[6],
                                             double (*out)[3]) {
  const int tid = threadIdx.x, q = tid >> 2, sub = tid & 3;
  const bool act = q < g;
  double ax = 0.0, ay = 0.0, az = 0.0;
  if (act && sh.alive[q]) {
    const double xq = z[q][0], yq = z[q][1], zq = z[q][2];
    for (int p = sub; p < g; p += 4) {
      const bool cen = p == q;
      const double dx = (cen ? 0.0 : z[p][0]) - xq, dy = (cen ? 0.0 : z[p][1]) - yq, dz = (cen ? 0.0 : z[p][2]) - zq;
      const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      const double yr = rsqrt_refined(r2);
      const bool inside = sh.alive[p] && dbits(r2) < umax64(sh.rcsq[q], sh.rcsq[p]);
      const double wA = changeover_wA_clamped(r2 * yr, pmin(sh.A[q], sh.A[p]), P.kmode);
      const double w = cen ? 1.0 : (inside ? wA : 0.0);
      const double f = (cen ? Gm0 : sh.gm[p]) * w * (yr * yr * yr);
      ax = fma(f, dx, ax); ay = fma(f, dy, ay); az = fma(f, dz, az);
    }
  }
#pragma unroll
  for (int o = 2; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
  }
  if (act && sub == 0) { out[q][0] = ax; out[q][1] = ay; out[q][2] = az; }
}

// Bulirsch-Stoer of one group of BS_GMAX + 1 .. BP_N members (members S.gmem[g0 ..], ascending) with
// the CTA: the extrapolation levels one after another (n_k = 2k), the error of each level's tableau
// row tested as it completes, the first converged level accepted; the step control, contact test
// and mergers as in bs_group.
__device__ void bp_big_group(BpBig &sh, const Sim &S, const DevParams &P, double tau, int g0, int g, double m0,
                             int step_no, int substep) {
  const int tid = threadIdx.x, np = S.npad;
  const double Gm0 = P.G * m0;
  if (tid < g) {
    const int i = S.gmem[g0 + tid];
    sh.idx[tid] = i;
    sh.alive[tid] = S.alive[i];
    sh.gm[tid] = S.gm[i]; sh.m[tid] = S.m[i]; sh.R[tid] = S.R[i]; sh.A[tid] = S.A[i];
    sh.rcsq[tid] = S.rcsq[i];
    for (int c = 0; c < 3; ++c) { sh.y[tid][c] = S.x0[c * np + i]; sh.y[tid][3 + c] = S.v0[c * np + i]; }
  }
  __syncthreads();
  const int lmax = P.bs_kmax < BS_LEVELS ? P.bs_kmax : BS_LEVELS;
  const u64 eps = dbits(P.bs_eps);
  const int ne = 6 * g;  // tableau elements (member, component); thread tid owns tid and tid + BP_THREADS
  double H = tau, rem = tau, U = 0.0;
  int halvings = 0, attempts = 0, steps = 0;
  while (absbits(rem) != 0ULL) {
    if (absbits(H) > absbits(rem)) H = rem;
    if (++attempts > 200000) { if (tid == 0) atomicOr(S.status, ST_BS_FAILED); break; }
    if (tid < g) {
      const double *yq = sh.y[tid];
      const double sx2 = fma(yq[2], yq[2], fma(yq[1], yq[1], yq[0] * yq[0]));
      const double sv2 = fma(yq[5], yq[5], fma(yq[4], yq[4], yq[3] * yq[3]));
      sh.isc[tid][0] = dbits(sx2) == 0ULL ? 4.49423283715579e307 : rsqrt_refined(sx2);
      sh.isc[tid][1] = dbits(sv2) == 0ULL ? 4.49423283715579e307 : rsqrt_refined(sv2);
    }
    bp_big_force(sh, P, Gm0, g, sh.y, sh.a0);
    __syncthreads();
    double prev[2][BS_LEVELS], tl[2] = {0.0, 0.0};
    int acc = 0;
    for (int k = 1; k <= lmax; ++k) {
      const int nk = 2 * k;
      const double h = __ddiv_rn(H, (double)nk), h2 = 2.0 * h;
      if (tid == 0) sh.err = 0ULL;
      for (int e = tid; e < ne; e += BP_THREADS) {
        const int q = e / 6, c = e % 6;
        const double y0 = sh.y[q][c];
        sh.za[q][c] = y0;
        sh.zb[q][c] = sh.alive[q] ? fma(h, c < 3 ? sh.y[q][c + 3] : sh.a0[q][c - 3], y0) : y0;
      }
      __syncthreads();
      for (int mm = 1; mm < nk; ++mm) {
        bp_big_force(sh, P, Gm0, g, sh.zb, sh.a);
        __syncthreads();
        double zn[2];
        for (int u = 0; u < 2; ++u) {
          const int e = tid + u * BP_THREADS;
          if (e >= ne) continue;
          const int q = e / 6, c = e % 6;
          zn[u] = sh.alive[q] ? fma(h2, c < 3 ? sh.zb[q][c + 3] : sh.a[q][c - 3], sh.za[q][c]) : sh.zb[q][c];
        }
        __syncthreads();
        for (int u = 0; u < 2; ++u) {
          const int e = tid + u * BP_THREADS;
          if (e >= ne) continue;
          const int q = e / 6, c = e % 6;
          sh.za[q][c] = sh.zb[q][c];
          sh.zb[q][c] = zn[u];
        }
        __syncthreads();
      }
      bp_big_force(sh, P, Gm0, g, sh.zb, sh.a);
      __syncthreads();
      for (int u = 0; u < 2; ++u) {  // T_{k,1} and row k of the Neville tableau (extrapolation in h^2)
        const int e = tid + u * BP_THREADS;
        if (e >= ne) continue;
        const int q = e / 6, c = e % 6;
        const double t1 = sh.alive[q] ? 0.5 * fma(h, c < 3 ? sh.zb[q][c + 3] : sh.a[q][c - 3], sh.zb[q][c] + sh.za[q][c])
                                      : sh.za[q][c];
        double before;
        tl[u] = neville_row(t1, k, [&](int j) { return c_facinv[k][j]; }, prev[u], before);
        if (k >= 2 && sh.alive[q]) atomicMax(&sh.err, absbits((tl[u] - before) * sh.isc[q][c < 3 ? 0 : 1]));
      }
      __syncthreads();
      if (k >= 2 && sh.err <= eps) acc = k;  // the same value for every thread
      __syncthreads();
      if (acc) break;
    }
    if (!acc) {
      H *= 0.5;
      if (++halvings > P.bs_max_halvings) { if (tid == 0) atomicOr(S.status, ST_BS_FAILED); break; }
      continue;
    }
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * BP_THREADS;
      if (e < ne) sh.yn[e / 6][e % 6] = tl[u];
    }
    __syncthreads();
    if (P.collisions) {  // contact over the substep (Hermite, threshold (R_a + R_b)^2), pre-merge states
      const int npair = g * (g - 1) / 2;
      int anyhit = 0;
      for (int pi = tid; pi < npair; pi += BP_THREADS) {
        int a = 0, rest = pi;
        while (rest >= g - 1 - a) { rest -= g - 1 - a; a++; }
        const int b = a + 1 + rest;
        unsigned char hit = 0;
        if (sh.alive[a] && sh.alive[b]) {
          const double rr = sh.R[a] + sh.R[b];
          const double dmin = hermite_min_capped(
              __dsub_rn(sh.y[b][0], sh.y[a][0]), __dsub_rn(sh.y[b][1], sh.y[a][1]), __dsub_rn(sh.y[b][2], sh.y[a][2]),
              __dsub_rn(sh.y[b][3], sh.y[a][3]), __dsub_rn(sh.y[b][4], sh.y[a][4]), __dsub_rn(sh.y[b][5], sh.y[a][5]),
              __dsub_rn(sh.yn[b][0], sh.yn[a][0]), __dsub_rn(sh.yn[b][1], sh.yn[a][1]), __dsub_rn(sh.yn[b][2], sh.yn[a][2]),
              __dsub_rn(sh.yn[b][3], sh.yn[a][3]), __dsub_rn(sh.yn[b][4], sh.yn[a][4]), __dsub_rn(sh.yn[b][5], sh.yn[a][5]), H, rr * rr);
          hit = dmin < rr * rr;
        }
        sh.cont[pi] = hit;
        anyhit |= hit;
      }
      if (__syncthreads_or(anyhit) && tid == 0) {  // mergers in ascending pair order, post-substep states (none without contact)
        int pi = 0;
        for (int a = 0; a < g; ++a)
          for (int b = a + 1; b < g; ++b, ++pi) {
            if (!sh.cont[pi] || !sh.alive[a] || !sh.alive[b]) continue;
            const int ia = sh.idx[a], ib = sh.idx[b];
            const double ma = sh.m[a], mb = sh.m[b], M = ma + mb;
            const double dx = sh.yn[b][0] - sh.yn[a][0], dy = sh.yn[b][1] - sh.yn[a][1], dz = sh.yn[b][2] - sh.yn[a][2];
            const double dvx = sh.yn[b][3] - sh.yn[a][3], dvy = sh.yn[b][4] - sh.yn[a][4], dvz = sh.yn[b][5] - sh.yn[a][5];
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            const double v2 = dvx * dvx + dvy * dvy + dvz * dvz;
            U += 0.5 * ma * mb / M * v2 - P.G * ma * mb / r;
            const bool keep_a = ma > mb || (ma == mb && ia < ib);
            merger_report(S, ia, ib, sh.y[a], sh.y[b], sh.yn[a], sh.yn[b], ma, mb, keep_a, tau - rem, step_no, substep);
            const int sv = keep_a ? a : b, d = keep_a ? b : a;
            for (int c = 0; c < 6; ++c) sh.yn[sv][c] = (ma * sh.yn[a][c] + mb * sh.yn[b][c]) / M;
            const double Ra = sh.R[a], Rb = sh.R[b];
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
      __syncthreads();
    }
    for (int e = tid; e < ne; e += BP_THREADS) sh.y[e / 6][e % 6] = sh.yn[e / 6][e % 6];
    __syncthreads();
    rem -= H;
    H *= 2.0;
    halvings = 0;
    steps++;
  }
  if (tid < g) {
    const int i = sh.idx[tid];
    if (sh.alive[tid]) {
      for (int c = 0; c < 3; ++c) { S.x[c * np + i] = sh.y[tid][c]; S.v[c * np + i] = sh.y[tid][3 + c]; }
    } else {
      S.x[i] = PARK + 1.0e4 * i; S.x[np + i] = 0.0; S.x[2 * np + i] = 0.0;
      for (int c = 0; c < 3; ++c) S.v[c * np + i] = 0.0;
    }
  }
  if (tid == 0) {
    atomicAdd((unsigned long long *)&S.counters[C_BSSTEPS], (unsigned long long)steps);
    if (dbits(U) != 0ULL) atomicAdd(S.U, U);
  }
  __syncthreads();
}

// Momentum of the system's live bodies into out[3] (fixed order: warps, then the warp partials).
__device__ __forceinline__ void bp_momentum(BpSys &sy, int n, double *out) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double p[3] = {0.0, 0.0, 0.0};
  if (tid < n && sy.alive[tid])
    for (int c = 0; c < 3; ++c) p[c] = sy.m[tid] * sy.v[c][tid];
  for (int c = 0; c < 3; ++c) {
    const double t = warp_sum(p[c]);
    if (lane == 0) sy.red[wid][c] = t;
  }
  __syncthreads();
  if (tid < 3) {
    double t = 0.0;
    for (int w = 0; w < (n + 31) / 32; ++w) t += sy.red[w][tid];
    out[tid] = t;
  }
  __syncthreads();
}

// The kick of Eq. Hb with the prechecker for the system in shared memory (BP_SPLIT threads per body),
// the arithmetic of k_b_kick. CLOSE: far pairs + candidates (recorded) with the step's critical
// radii, v += h1 a (+ h2 a). OPEN: stored far field + candidates with the new radii, or every pair
// when the system failed the reuse test.
template <int MODE>
__device__ __forceinline__ void bp_kick(BpSys &sy, const DevParams &P, int n, double h1, double h2, int *ncand) {
  const int tid = threadIdx.x, k = tid / BP_SPLIT, sub = tid % BP_SPLIT;
  const bool live = k < n && sy.alive[k];
  const bool full = (MODE == FIN_OPEN) && sy.flag != 0;
  double fx = 0, fy = 0, fz = 0, nx = 0, ny = 0, nz = 0;
  u64 mask = 0ULL;
  if (live) {
    const double xi = sy.x[0][k], yi = sy.x[1][k], zi = sy.x[2][k];
    const u64 Ti = sy.T[k], Qi = sy.rq[k];
    const double Ai = sy.A[k];
    if (MODE != FIN_OPEN || full) {
      for (int j = sub; j < n; j += BP_SPLIT) {
        if (j == k || !sy.alive[j]) continue;
        const double dx = sy.x[0][j] - xi, dy = sy.x[1][j] - yi, dz = sy.x[2][j] - zi;
        const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
        const double w3 = rcube_refined(r2);
        const u64 rb = dbits(r2);
        const bool cand = (MODE != FIN_OPEN) && rb < umax64(Ti, sy.T[j]);
        double gg = sy.gm[j] * w3;
        if (cand || full) {
          if (rb < umax64(Qi, sy.rq[j])) {
            double wB, wA;
            changeover_w(r2 * rsqrt_refined(r2), pmin(Ai, sy.A[j]), P.kmode, wB, wA);
            gg *= wB;
          }
          if (cand) mask |= 1ULL << j;
          nx = fma(gg, dx, nx); ny = fma(gg, dy, ny); nz = fma(gg, dz, nz);
        } else {
          fx = fma(gg, dx, fx); fy = fma(gg, dy, fy); fz = fma(gg, dz, fz);
        }
      }
    } else {  // KickA: only the candidates, with the new critical radii
      u64 bits = sy.cm[k];
      int c = 0;
      while (bits) {
        const int j = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        if ((c++ % BP_SPLIT) != sub) continue;
        const double dx = sy.x[0][j] - xi, dy = sy.x[1][j] - yi, dz = sy.x[2][j] - zi;
        const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
        const double yr = rsqrt_refined(r2);
        double gg = sy.gm[j] * (yr * yr * yr);
        if (dbits(r2) < umax64(Qi, sy.rq[j])) {
          double wB, wA;
          changeover_w(r2 * yr, pmin(Ai, sy.A[j]), P.kmode, wB, wA);
          gg *= wB;
        }
        nx = fma(gg, dx, nx); ny = fma(gg, dy, ny); nz = fma(gg, dz, nz);
      }
    }
  }
#pragma unroll
  for (int o = BP_SPLIT >> 1; o > 0; o >>= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o); fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o); nx += __shfl_xor_sync(0xffffffffu, nx, o);
    ny += __shfl_xor_sync(0xffffffffu, ny, o); nz += __shfl_xor_sync(0xffffffffu, nz, o);
    mask |= __shfl_xor_sync(0xffffffffu, mask, o);
  }
  __syncthreads();  // every thread has read the masks and positions it needs
  if (!live || sub != 0) return;
  double ax, ay, az;
  if (MODE == FIN_OPEN) {
    if (full) { ax = nx; ay = ny; az = nz; }
    else { ax = sy.af[0][k] + nx; ay = sy.af[1][k] + ny; az = sy.af[2][k] + nz; }
  } else {
    sy.af[0][k] = fx; sy.af[1][k] = fy; sy.af[2][k] = fz;
    sy.cm[k] = mask;
    if (mask) atomicAdd(ncand, __popcll(mask));
    ax = fx + nx; ay = fy + ny; az = fz + nz;
  }
  double vx = fma(h1, ax, sy.v[0][k]), vy = fma(h1, ay, sy.v[1][k]), vz = fma(h1, az, sy.v[2][k]);
  if (h2 != 0.0) { vx = fma(h2, ax, vx); vy = fma(h2, ay, vy); vz = fma(h2, az, vz); }
  sy.v[0][k] = vx; sy.v[1][k] = vy; sy.v[2][k] = vz;
}

__global__ void __launch_bounds__(BP_THREADS, 2) k_b_persist(Sim S, DevParams P, BpArgs args) {
  extern __shared__ __align__(16) unsigned char bp_smem[];
  BpSys &sy = *reinterpret_cast<BpSys *>(bp_smem);
  BpBs &bb = *reinterpret_cast<BpBs *>(bp_smem + BP_SYS_BYTES);
  const int tid = threadIdx.x, lane = tid & 31;
  const int np = S.npad;
  const int base = *args.step_base;
  for (;;) {
    if (tid == 0) sy.sys = atomicAdd(args.queue, 1);
    __syncthreads();
    const int s = sy.sys;
    if (s >= S.nsys) break;  // uniform
    const int st = S.sys_start[s], n = S.sys_start[s + 1] - st;
    const double m0 = S.sys_m0[s], im0 = rcp_refined(m0), mu = P.G * m0;
    for (int k = tid; k < n; k += BP_THREADS) {
      const int i = st + k;
      for (int c = 0; c < 3; ++c) { sy.x[c][k] = S.x[c * np + i]; sy.v[c][k] = S.v[c * np + i]; sy.af[c][k] = S.afar[c * np + i]; }
      sy.m[k] = S.m[i]; sy.gm[k] = S.gm[i]; sy.hill[k] = S.hill[i]; sy.rc[k] = S.rc[i]; sy.A[k] = S.A[i];
      sy.T[k] = S.T[i]; sy.rq[k] = S.rcsq[i]; sy.cm[k] = S.bmask[i]; sy.alive[k] = S.alive[i];
    }
    if (tid == 0) { sy.nenc = 0; sy.ncand = 0; }
    __syncthreads();
    for (int step = 0; step < args.nsteps; ++step) {
      const int step_no = base + step + 1;
      if (s == 0 && tid == 0) atomicAdd((unsigned long long *)&S.counters[C_STEPS], 1ULL);
      // critical radii (Eq. rcrit) with the reuse test of the opening kick
      if (tid == 0) sy.flag = 0;
      __syncthreads();
      const double tau_abs = fabs(args.dt);
      if (tid < n) {
        const int k = tid, i = st + k;
        if (!sy.alive[k]) {
          sy.rc[k] = 0.0; sy.A[k] = 0.0; sy.T[k] = 0ULL; sy.rq[k] = 0ULL;
        } else {
          const double x = sy.x[0][k], y = sy.x[1][k], z = sy.x[2][k];
          const double vx = sy.v[0][k], vy = sy.v[1][k], vz = sy.v[2][k];
          const double r2 = fma(z, z, fma(y, y, x * x));
          const double ir = rsqrt_refined(r2);
          const double v2 = fma(vz, vz, fma(vy, vy, vx * vx));
          const double inva = fma(2.0, ir, -v2 * rcp_refined(mu));
          const double asemi = is_neg_or_zero(inva) ? r2 * ir : rcp_refined(inva);
          const double rh = asemi * sy.hill[k];
          const double vabs = (dbits(v2) == 0ULL) ? 0.0 : v2 * rsqrt_refined(v2);
          const double rc = pmax(P.n1 * rh, (P.n2 * tau_abs) * vabs);
          if (dbits(rc) > dbits(P.pc * sy.rc[k])) {
            atomicOr(&sy.flag, 1);
            atomicOr(S.status, ST_REUSE_FULLKICK);
            atomicAdd((unsigned long long *)&S.counters[C_FULLKICK], 1ULL);
          }
          sy.rc[k] = rc;
          const double t = __dmul_rn(P.pc, rc);
          sy.T[k] = dbits(__dmul_rn(t, t));
          sy.rq[k] = dbits(__dmul_rn(rc, rc));
          sy.A[k] = (dbits(rc) == 0ULL) ? 0.0 : rcp_refined(0.9 * rc);
        }
        S.rc[i] = sy.rc[k]; S.A[i] = sy.A[k]; S.T[i] = sy.T[k]; S.rcsq[i] = sy.rq[k];  // for the BS kernels
      }
      __syncthreads();
      bp_kick<FIN_OPEN>(sy, P, n, 0.5 * args.w[0] * args.dt, 0.0, &sy.ncand);
      __syncthreads();
      for (int j = 0; j < args.nsub; ++j) {
        const double tau = args.w[j] * args.dt;
        bp_momentum(sy, n, sy.P);
        // Sun drifts (this substep's first with the momentum after the kick, the previous
        // substep's second with the momentum before its closing kick), then the Kepler drift
        if (tid < n) {
          const int k = tid, i = st + k;
          sy.em[k] = 0ULL;
          sy.fail[k] = 0;
          if (sy.alive[k]) {
            const double h1 = 0.5 * tau, h2 = j > 0 ? 0.5 * args.w[j - 1] * args.dt : 0.0;
            double sh[3];
            for (int c = 0; c < 3; ++c) {
              double a = h1 * sy.P[c];
              if (h2 != 0.0) a = fma(h2, sy.Ppre[c], a);
              sh[c] = a * im0;
            }
            double x = sy.x[0][k] + sh[0], y = sy.x[1][k] + sh[1], z = sy.x[2][k] + sh[2];
            double vx = sy.v[0][k], vy = sy.v[1][k], vz = sy.v[2][k];
            sy.x0[0][k] = x; sy.x0[1][k] = y; sy.x0[2][k] = z;
            sy.v0[0][k] = vx; sy.v0[1][k] = vy; sy.v0[2][k] = vz;
            S.x0[i] = x; S.x0[np + i] = y; S.x0[2 * np + i] = z;
            S.v0[i] = vx; S.v0[np + i] = vy; S.v0[2 * np + i] = vz;
            int it = 0;
            if (kepler_drift_dev(mu, 2.0 * mu, x, y, z, vx, vy, vz, tau, P.kepler_maxit, &it)) {
              atomicOr(S.status, ST_KEPLER_FALLBACK);
              atomicAdd((unsigned long long *)&S.counters[C_KFALL], 1ULL);
              sy.fail[k] = 1;
            }
            sy.x[0][k] = x; sy.x[1][k] = y; sy.x[2][k] = z;
            sy.v[0][k] = vx; sy.v[1][k] = vy; sy.v[2][k] = vz;
          }
        }
        if (tid == 0) { sy.npairs = 0; sy.ngroups = 0; }
        __syncthreads();
        // encounter search: the candidate pairs (k, b > k) of the last closing kick, one per thread
        if (tid < n && sy.alive[tid]) {
          u64 bits = sy.cm[tid] & (tid >= 63 ? 0ULL : (~0ULL << (tid + 1)));
          while (bits) {
            const int b = __ffsll((long long)bits) - 1;
            bits &= bits - 1;
            const int p = atomicAdd(&sy.npairs, 1);
            sy.pa[p] = (unsigned char)tid;
            sy.pb[p] = (unsigned char)b;
          }
        }
        __syncthreads();
        for (int p = tid; p < sy.npairs; p += BP_THREADS) {
          const int a = sy.pa[p], b = sy.pb[p];
          if (!sy.alive[b]) continue;
          const double rcij = pmax(sy.rc[a], sy.rc[b]);
          const double thr = __dmul_rn(rcij, rcij);
          const double dmin = hermite_min_capped(
              __dsub_rn(sy.x0[0][b], sy.x0[0][a]), __dsub_rn(sy.x0[1][b], sy.x0[1][a]), __dsub_rn(sy.x0[2][b], sy.x0[2][a]),
              __dsub_rn(sy.v0[0][b], sy.v0[0][a]), __dsub_rn(sy.v0[1][b], sy.v0[1][a]), __dsub_rn(sy.v0[2][b], sy.v0[2][a]),
              __dsub_rn(sy.x[0][b], sy.x[0][a]), __dsub_rn(sy.x[1][b], sy.x[1][a]), __dsub_rn(sy.x[2][b], sy.x[2][a]),
              __dsub_rn(sy.v[0][b], sy.v[0][a]), __dsub_rn(sy.v[1][b], sy.v[1][a]), __dsub_rn(sy.v[2][b], sy.v[2][a]), tau, thr);
          if (dmin < thr) {
            atomicOr(&sy.em[a], 1ULL << b);
            atomicAdd(&sy.nenc, 1);
          }
        }
        __syncthreads();
        if (tid < n) S.emask[st + tid] = sy.em[tid];  // the substep's pairs, as the step graph leaves them
        // groups: connected components of the encounter pairs (and failed Kepler solves) by the
        // first warp; group g = the g-th root in ascending order, members ascending
        if (tid < 32) {
          for (int k = lane; k < BP_N; k += 32) { sy.link[k] = k; sy.cnt[k] = 0; }
          __syncwarp();
          for (int round = 0; round < 64; ++round) {
            bool ch = false;
            for (int k = lane; k < n; k += 32) {
              u64 bits = sy.em[k];
              while (bits) {
                const int b = __ffsll((long long)bits) - 1;
                bits &= bits - 1;
                int ru = k, rv = b;
                for (int q = 0; q < 66 && sy.link[ru] != ru; ++q) ru = sy.link[ru];
                for (int q = 0; q < 66 && sy.link[rv] != rv; ++q) rv = sy.link[rv];
                if (ru != rv) { atomicMin(&sy.link[ru > rv ? ru : rv], ru < rv ? ru : rv); ch = true; }
              }
            }
            __syncwarp();
            for (int k = lane; k < n; k += 32) {
              int r = k;
              for (int q = 0; q < 66 && sy.link[r] != r; ++q) r = sy.link[r];
              sy.link[k] = r;
            }
            __syncwarp();
            if (!__any_sync(0xffffffffu, ch)) break;
          }
          // participants: an encounter pair's bodies and the failed Kepler solves
          u64 part = 0ULL;
          for (int k = lane; k < n; k += 32)
            if (sy.em[k] || sy.fail[k]) part |= (1ULL << k) | sy.em[k];
          for (int o = 16; o > 0; o >>= 1) part |= __shfl_xor_sync(0xffffffffu, part, o);
          for (int k = lane; k < n; k += 32)
            if ((part >> k) & 1ULL) atomicAdd(&sy.cnt[sy.link[k]], 1);
          __syncwarp();
          if (lane == 0) {
            int ng = 0, off = 0;
            for (int r = 0; r < n; ++r)
              if (((part >> r) & 1ULL) && sy.link[r] == r) {
                sy.gst[ng] = off;
                off += sy.cnt[r];
                sy.cnt[r] = ng++;  // the root's group index
              }
            sy.gst[ng] = off;
            sy.ngroups = ng;
            if (ng) atomicAdd((unsigned long long *)&S.counters[C_GROUPS], (unsigned long long)ng);
          }
          __syncwarp();
          for (int k = lane; k < n; k += 32) {
            if (!((part >> k) & 1ULL)) continue;
            const int gk = sy.cnt[sy.link[k]];
            int rank = 0;
            for (int q = 0; q < k; ++q) rank += (((part >> q) & 1ULL) && sy.link[q] == sy.link[k]) ? 1 : 0;
            sy.gmem[sy.gst[gk] + rank] = k;
          }
        }
        __syncthreads();
        // the system's groups in its own slice of the global group arrays, for the BS code
        const int ng = sy.ngroups;
        for (int q = tid; q < sy.gst[ng]; q += BP_THREADS) S.gmem[st + q] = st + sy.gmem[q];
        for (int g = tid; g < ng; g += BP_THREADS) { S.gstart[st + g] = st + sy.gst[g]; S.gsize[st + g] = sy.gst[g + 1] - sy.gst[g]; }
        __syncthreads();
        for (int g = 0; g < ng; ++g) {
          const int g0 = st + sy.gst[g], gsz = sy.gst[g + 1] - sy.gst[g];
          if (gsz <= BS_GMAX) bs_group<BP_THREADS, BS_GMAX>(bb.small, S, P, tau, st + g, g0, gsz, m0, step_no, j, blockIdx.x);
          else bp_big_group(bb.big, S, P, tau, g0, gsz, m0, step_no, j);
          for (int q = tid; q < gsz; q += BP_THREADS) {  // the members' new state (and merged masses)
            const int k = sy.gmem[sy.gst[g] + q], i = st + k;
            for (int c = 0; c < 3; ++c) { sy.x[c][k] = S.x[c * np + i]; sy.v[c][k] = S.v[c * np + i]; }
            sy.m[k] = S.m[i]; sy.gm[k] = S.gm[i]; sy.hill[k] = S.hill[i]; sy.alive[k] = S.alive[i];
            sy.T[k] = S.T[i]; sy.rq[k] = S.rcsq[i];
          }
          __syncthreads();
        }
        bp_momentum(sy, n, sy.Ppre);
        const double h2 = (j + 1 < args.nsub) ? 0.5 * args.w[j + 1] * args.dt : 0.0;
        bp_kick<FIN_CLOSE>(sy, P, n, 0.5 * tau, h2, &sy.ncand);
        __syncthreads();
      }
      // second Sun drift of the last substep
      if (tid < n && sy.alive[tid]) {
        const double h = 0.5 * args.w[args.nsub - 1] * args.dt;
        for (int c = 0; c < 3; ++c) sy.x[c][tid] = fma(h * sy.Ppre[c], im0, sy.x[c][tid]);
      }
      __syncthreads();
    }
    for (int k = tid; k < n; k += BP_THREADS) {
      const int i = st + k;
      for (int c = 0; c < 3; ++c) { S.x[c * np + i] = sy.x[c][k]; S.v[c * np + i] = sy.v[c][k]; S.afar[c * np + i] = sy.af[c][k]; }
      S.rc[i] = sy.rc[k]; S.A[i] = sy.A[k]; S.T[i] = sy.T[k]; S.rcsq[i] = sy.rq[k]; S.bmask[i] = sy.cm[k];
    }
    if (tid == 0) {
      if (sy.nenc) atomicAdd((unsigned long long *)&S.counters[C_ENC], (unsigned long long)sy.nenc);
      if (sy.ncand) atomicAdd((unsigned long long *)&S.counters[C_CAND], (unsigned long long)sy.ncand);
    }
    __syncthreads();
  }
}

// Per-device set-up (outside any capture): the Neville factors and the shared-memory size.
int b_persist_init() {
  bs_core_set_factors();
  if (cudaFuncSetAttribute(k_b_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BP_SMEM) != cudaSuccess)
    return -1;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_b_persist, BP_THREADS, BP_SMEM) != cudaSuccess) per = 1;
  cudaGetLastError();
  return per < 1 ? 1 : per;
}

__global__ void k_bp_advance(int *step_base, int nsteps) { *step_base += nsteps; }

void launch_b_persist(const Sim &S, const DevParams &P, double dt, const double *w, int nsub, int nsteps,
                      int *step_base, int *queue, int blocks, cudaStream_t st) {
  BpArgs a;
  a.dt = dt;
  for (int k = 0; k < 7; ++k) a.w[k] = k < nsub ? w[k] : 0.0;
  a.nsub = nsub;
  a.nsteps = nsteps;
  a.step_base = step_base;
  a.queue = queue;
  cudaMemsetAsync(queue, 0, sizeof(int), st);
  k_b_persist<<<blocks < 1 ? 1 : blocks, BP_THREADS, BP_SMEM, st>>>(S, P, a);
  k_bp_advance<<<1, 1, 0, st>>>(step_base, nsteps);
}

}  // namespace genga
