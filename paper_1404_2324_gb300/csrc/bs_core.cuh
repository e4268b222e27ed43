// bs_core.cuh -- the Bulirsch-Stoer of one encounter group by one CTA (Sect. 3.2), shared by the
// kernels of bs.cu and the persistent batched kernel (batch_persist.cu). Every translation unit
// that includes it holds its own copy of the Neville factors (bs_core_set_factors fills it).
#pragma once
#include "genga_launch.h"

namespace genga {

// 1/((L/(L-j))^2 - 1) for the Neville extrapolation in h^2 with n_k = 2k
static __constant__ double c_facinv[BS_LEVELS + 1][BS_LEVELS];


// Fills this translation unit's c_facinv (host; once per device, before any capture).
static inline void bs_core_set_factors() {
  double h[BS_LEVELS + 1][BS_LEVELS] = {};
  for (int L = 2; L <= BS_LEVELS; ++L)
    for (int j = 1; j < L; ++j) {
      const double ratio = (double)L / (double)(L - j);
      h[L][j] = 1.0 / (ratio * ratio - 1.0);
    }
  cudaMemcpyToSymbol(c_facinv, h, sizeof(h));
}

// A group's state in shared memory, for groups of up to GM members.
template <int GM>
struct BsSharedT {
  int idx[GM], alive[GM];
  double gm[GM], m[GM], R[GM], A[GM];
  u64 rcsq[GM];
  double y[GM][6], yn[GM][6];
  double pos[2][BS_LEVELS][GM][3];
  double tab[BS_LEVELS][GM][6];
  u64 err[BS_LEVELS], err2[BS_LEVELS];  // per level: the attempt at H, the speculative one at H/2
  unsigned char cont[GM * (GM - 1) / 2];
  double H, rem, U;
  int accept, next;
  int nseq, seq_base;          // recorded accepted substeps (adjoint engine only)
  long long y_base;
  double seqH[BS_SEQCAP];
  unsigned char seqk[BS_SEQCAP];
};
using BsShared = BsSharedT<BS_GMAX>;

// Acceleration terms of member q assigned to this thread: term p == q is the central mass, any
// other p the (1 - K)-weighted pull of partner p (H_A, Eq. Ha). Summed over the slot's threads.
// Every lane runs the same straight-line code (the central mass is a partner at the origin with
// G m0 and weight 1; a partner outside rc gets weight 0): lanes of one warp that took different
// branches would each pay for both, and an FP64 warp instruction costs its sub-partition 64
// cycles whatever its active lanes.
template <class SH>
__device__ __forceinline__ void bs_terms(const SH &sh, const DevParams &P, double Gm0, int g, int q, int sub,
                                         int tps, const double (*pos)[3], bool q_alive, double &ax, double &ay,
                                         double &az) {
  ax = ay = az = 0.0;
  const double xq = pos[q][0], yq = pos[q][1], zq = pos[q][2];
  if (q_alive) {
    for (int p = sub; p < g; p += tps) {
      const bool cen = p == q;
      const double dx = (cen ? 0.0 : pos[p][0]) - xq, dy = (cen ? 0.0 : pos[p][1]) - yq,
                   dz = (cen ? 0.0 : pos[p][2]) - zq;
      const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      const double yr = rsqrt_refined(r2);
      const bool inside = sh.alive[p] && dbits(r2) < umax64(sh.rcsq[q], sh.rcsq[p]);
      const double wA = changeover_wA_clamped(r2 * yr, pmin(sh.A[q], sh.A[p]), P.kmode);
      const double w = cen ? 1.0 : (inside ? wA : 0.0);
      const double f = (cen ? Gm0 : sh.gm[p]) * w * (yr * yr * yr);
      ax = fma(f, dx, ax); ay = fma(f, dy, ay); az = fma(f, dz, az);
    }
  }
  for (int o = tps >> 1; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
  }
}

// Bulirsch-Stoer of one group (members S.gmem[g0 .. g0 + g - 1], ascending; central mass m0) over
// tau by the NT threads of the calling CTA: every level's modified-midpoint chain at once, each
// level's tableau row built and tested as soon as the level completes, the first converged level
// accepted (Sect. 3.2); contacts and mergers after every accepted substep; the result written back
// to S. step_no and substep label the collision reports (< 0: the counters of the step graph);
// rec_slot is the CTA's slot in the adjoint engine's recording scratch.
template <int NT, int GM>
__device__ void bs_group(BsSharedT<GM> &sh, const Sim &S, const DevParams &P, double tau, int gidx, int g0, int g,
                         double m0, int step_no, int substep, int rec_slot) {
  const int tid = threadIdx.x;
  const int np = S.npad;
  const double Gm0 = P.G * m0;
  const int tps = g <= 8 ? 4 : (g <= 16 ? 2 : 1);  // threads per (level, member) slot
  if (BS_LEVELS * g * tps > NT) {  // uniform; the queues route larger groups elsewhere
    if (tid == 0) atomicOr(S.status, ST_GROUP_TOO_LARGE);
    return;
  }
  const int slot = tid / tps, sub = tid % tps;
  const bool act = slot < BS_LEVELS * g;
  const int lev = act ? slot / g : 0;  // level k = lev + 1, n_k = 2k substeps
  const int q = act ? slot % g : 0;
  const int L = lev + 1, nk = 2 * L;
  // Speculation (groups of one or two members, whose slots leave two of their four threads idle):
  // threads 2, 3 of a slot run the attempt at H/2 from the same state, with the same arithmetic, in
  // the same warp instructions; its members sit at index 16 + q of the position and tableau arrays,
  // its tableau rows on threads 64 + (member, component). Its result is taken exactly when the
  // serial step control's next attempt would be that one (the attempt at H failed), so results and
  // decisions are the serial algorithm's, and a failed attempt no longer costs a round of its own.
  const bool spec = g <= 2 && tps == 4 && NT >= 128 && GM >= 18;  // uniform
  const int half = spec ? (sub >> 1) : 0, tsub = spec ? (sub & 1) : sub, ttps = spec ? 2 : tps;
  const int qm = q + 16 * half;  // this thread's member in its attempt's position and tableau arrays
  const int trow = (spec && tid >= 64) ? tid - 64 : tid;  // tableau thread of attempt (spec && tid >= 64)
  const int thalf = (spec && tid >= 64) ? 1 : 0;
  if (tid < g) {
    const int i = S.gmem[g0 + tid];
    sh.idx[tid] = i;
    sh.alive[tid] = S.alive[i];
    sh.gm[tid] = S.gm[i]; sh.m[tid] = S.m[i]; sh.R[tid] = S.R[i]; sh.A[tid] = S.A[i];
    sh.rcsq[tid] = S.rcsq[i];
    for (int c = 0; c < 3; ++c) { sh.y[tid][c] = S.x0[c * np + i]; sh.y[tid][3 + c] = S.v0[c * np + i]; }
  }
  if (tid == 0) { sh.H = tau; sh.rem = tau; sh.U = 0.0; sh.nseq = 0; }
  __syncthreads();
  int halvings = 0, attempts = 0, steps = 0;
  while (true) {
    const double rem = sh.rem;
    double H = sh.H;
    if (absbits(rem) == 0ULL) break;
    if (absbits(H) > absbits(rem)) H = rem;
    if (++attempts > 200000) { if (tid == 0) atomicOr(S.status, ST_BS_FAILED); break; }
    // ---- one attempt of length H: all levels' modified-midpoint integrations at once ----
    // Level L finishes its chain at evaluation 2L; its tableau row and error are then computed
    // right away (thread (qc, cc) holds member qc's component cc of the previous row), and the
    // attempt stops at the first converged level: the same decision as building the whole
    // tableau first, but attempts that converge at level 4-6 (almost all) skip the deeper chains.
    const double h = __ddiv_rn(half ? 0.5 * H : H, (double)nk), h2 = 2.0 * h;
    const bool qa = act && sh.alive[q];
    double zA[6], zB[6], out[6];
    for (int c = 0; c < 6; ++c) zA[c] = sh.y[q][c];
    if (act && tsub == 0) for (int c = 0; c < 3; ++c) sh.pos[0][lev][qm][c] = zA[c];
    const int qc = trow / 6, cc = trow % 6;
    const bool rowth = qc < g;
    double scale = 0.0;  // error scale of (qc, cc): 1/|x| or 1/|v| at the start of the attempt
    if (rowth) {
      const double *yq = sh.y[qc] + (cc < 3 ? 0 : 3);
      const double s2 = fma(yq[2], yq[2], fma(yq[1], yq[1], yq[0] * yq[0]));
      scale = dbits(s2) == 0ULL ? 4.49423283715579e307 : rsqrt_refined(s2);
    }
    if (tid < BS_LEVELS) { sh.err[tid] = 0ULL; sh.err2[tid] = 0ULL; }
    __syncthreads();
    double ax = 0.0, ay = 0.0, az = 0.0;
    // every lane of a warp that holds any active slot takes part (the term sums shuffle across
    // lanes); warps without active slots stay off the FP64 pipe
    if (__any_sync(0xffffffffu, act)) bs_terms(sh, P, Gm0, g, q, tsub, ttps, sh.pos[0][lev] + 16 * half, qa, ax, ay, az);
    if (qa) {
      zB[0] = fma(h, zA[3], zA[0]); zB[1] = fma(h, zA[4], zA[1]); zB[2] = fma(h, zA[5], zA[2]);
      zB[3] = fma(h, ax, zA[3]); zB[4] = fma(h, ay, zA[4]); zB[5] = fma(h, az, zA[5]);
    } else {
      for (int c = 0; c < 6; ++c) zB[c] = zA[c];
    }
    const int lmax = P.bs_kmax < BS_LEVELS ? P.bs_kmax : BS_LEVELS;
    const u64 eps = dbits(P.bs_eps);
    double prev[BS_LEVELS], tlast = 0.0;  // previous tableau row; T_{Lc,Lc} of the current one
    int acc = 0, accB = 0;
    int b = 1;
    for (int e = 1; e <= 2 * lmax; ++e) {
      const bool lv = act && e <= nk;
      if (lv && tsub == 0) for (int c = 0; c < 3; ++c) sh.pos[b][lev][qm][c] = zB[c];
      __syncthreads();
      if (__any_sync(0xffffffffu, lv)) bs_terms(sh, P, Gm0, g, q, tsub, ttps, sh.pos[b][lev] + 16 * half, qa, ax, ay, az);
      if (lv) {
        if (qa) {
          if (e < nk) {
            double zn[6];
            zn[0] = fma(h2, zB[3], zA[0]); zn[1] = fma(h2, zB[4], zA[1]); zn[2] = fma(h2, zB[5], zA[2]);
            zn[3] = fma(h2, ax, zA[3]); zn[4] = fma(h2, ay, zA[4]); zn[5] = fma(h2, az, zA[5]);
            for (int c = 0; c < 6; ++c) { zA[c] = zB[c]; zB[c] = zn[c]; }
          } else {
            out[0] = 0.5 * fma(h, zB[3], zB[0] + zA[0]);
            out[1] = 0.5 * fma(h, zB[4], zB[1] + zA[1]);
            out[2] = 0.5 * fma(h, zB[5], zB[2] + zA[2]);
            out[3] = 0.5 * fma(h, ax, zB[3] + zA[3]);
            out[4] = 0.5 * fma(h, ay, zB[4] + zA[4]);
            out[5] = 0.5 * fma(h, az, zB[5] + zA[5]);
          }
        } else if (e == nk) {
          for (int c = 0; c < 6; ++c) out[c] = zA[c];
        }
        if (e == nk && tsub == 0) for (int c = 0; c < 6; ++c) sh.tab[lev][qm][c] = out[c];  // T_{L,1}
      }
      b ^= 1;
      if (e & 1) continue;
      // level Lc = e/2 is complete: its tableau row (polynomial extrapolation in h^2, Neville)
      const int Lc = e >> 1;
      __syncthreads();
      u64 ev = 0ULL;
      if (rowth) {
        double before;
        tlast = neville_row(sh.tab[Lc - 1][qc + 16 * thalf][cc], Lc, [&](int j) { return c_facinv[Lc][j]; }, prev, before);
        if (Lc >= 2 && sh.alive[qc]) ev = absbits((tlast - before) * scale);
      }
      if (Lc >= 2) warp_max_to(thalf ? &sh.err2[Lc - 1] : &sh.err[Lc - 1], ev);  // thalf is uniform per warp
      __syncthreads();
      if (spec && !accB && Lc >= 2 && sh.err2[Lc - 1] <= eps) {  // the attempt at H/2 converged (uniform)
        accB = Lc;
        if (thalf && rowth) sh.yn[qc + 16][cc] = tlast;
      }
      if (Lc >= 2 && sh.err[Lc - 1] <= eps) { acc = Lc; break; }  // uniform: every thread reads the same error
    }
    if (acc && rowth && !thalf) sh.yn[qc][cc] = tlast;  // the accepted row is the last one built
    double Hs = H;  // length of the accepted substep
    if (!acc && spec) {  // the serial control halves H; its next attempt is the one at H/2
      if (++halvings > P.bs_max_halvings) {
        if (tid == 0) atomicOr(S.status, ST_BS_FAILED);
        __syncthreads();
        break;
      }
      ++attempts;
      if (accB) {
        acc = accB;
        Hs = 0.5 * H;
        __syncthreads();
        if (tid < 6 * g) sh.yn[tid / 6][tid % 6] = sh.yn[tid / 6 + 16][tid % 6];
      } else {  // that attempt failed too: the serial control halves again
        if (tid == 0) sh.H = 0.25 * H;
        if (++halvings > P.bs_max_halvings) {
          if (tid == 0) atomicOr(S.status, ST_BS_FAILED);
          __syncthreads();
          break;
        }
        __syncthreads();
        continue;
      }
    }
    if (acc) {
      __syncthreads();
      if (P.collisions) {  // contact test over the accepted substep (Hermite, threshold (R_a + R_b)^2)
        const int npair = g * (g - 1) / 2;
        int anyhit = 0;
        for (int pi = tid; pi < npair; pi += NT) {
          int a = 0, rest = pi;
          while (rest >= g - 1 - a) { rest -= g - 1 - a; a++; }
          const int bq = a + 1 + rest;
          unsigned char hit = 0;
          if (sh.alive[a] && sh.alive[bq]) {
            const double rr = sh.R[a] + sh.R[bq];
            const double dmin = hermite_min_capped(
                __dsub_rn(sh.y[bq][0], sh.y[a][0]), __dsub_rn(sh.y[bq][1], sh.y[a][1]), __dsub_rn(sh.y[bq][2], sh.y[a][2]),
                __dsub_rn(sh.y[bq][3], sh.y[a][3]), __dsub_rn(sh.y[bq][4], sh.y[a][4]), __dsub_rn(sh.y[bq][5], sh.y[a][5]),
                __dsub_rn(sh.yn[bq][0], sh.yn[a][0]), __dsub_rn(sh.yn[bq][1], sh.yn[a][1]), __dsub_rn(sh.yn[bq][2], sh.yn[a][2]),
                __dsub_rn(sh.yn[bq][3], sh.yn[a][3]), __dsub_rn(sh.yn[bq][4], sh.yn[a][4]), __dsub_rn(sh.yn[bq][5], sh.yn[a][5]), Hs, rr * rr);
            hit = dmin < rr * rr;
          }
          sh.cont[pi] = hit;
          anyhit |= hit;
        }
        if (__syncthreads_or(anyhit) && tid == 0) {  // mergers in ascending pair order, post-substep states (none without contact)
          int pi = 0;
          for (int a = 0; a < g; ++a)
            for (int bq = a + 1; bq < g; ++bq, ++pi) {
              if (!sh.cont[pi] || !sh.alive[a] || !sh.alive[bq]) continue;
              const int ia = sh.idx[a], ib = sh.idx[bq];
              const double ma = sh.m[a], mb = sh.m[bq], M = ma + mb;
              const double dx = sh.yn[bq][0] - sh.yn[a][0], dy = sh.yn[bq][1] - sh.yn[a][1], dz = sh.yn[bq][2] - sh.yn[a][2];
              const double dvx = sh.yn[bq][3] - sh.yn[a][3], dvy = sh.yn[bq][4] - sh.yn[a][4], dvz = sh.yn[bq][5] - sh.yn[a][5];
              const double r = sqrt(dx * dx + dy * dy + dz * dz);
              const double v2 = dvx * dvx + dvy * dvy + dvz * dvz;
              sh.U += 0.5 * ma * mb / M * v2 - P.G * ma * mb / r;
              const bool keep_a = ma > mb || (ma == mb && ia < ib);
              merger_report(S, ia, ib, sh.y[a], sh.y[bq], sh.yn[a], sh.yn[bq], ma, mb, keep_a, tau - rem, step_no, substep);
              const int s = keep_a ? a : bq, d = keep_a ? bq : a;
              for (int c = 0; c < 6; ++c) sh.yn[s][c] = (ma * sh.yn[a][c] + mb * sh.yn[bq][c]) / M;
              const double Ra = sh.R[a], Rb = sh.R[bq];
              sh.R[s] = cbrt(Ra * Ra * Ra + Rb * Rb * Rb);
              sh.m[s] = M; sh.gm[s] = P.G * M;
              sh.m[d] = 0.0; sh.gm[d] = 0.0; sh.R[d] = 0.0; sh.alive[d] = 0;
              const int is = sh.idx[s], idd = sh.idx[d];
              S.m[is] = M; S.gm[is] = P.G * M; S.R[is] = sh.R[s]; S.hill[is] = cbrt(M / (3.0 * m0));
              S.m[idd] = 0.0; S.gm[idd] = 0.0; S.R[idd] = 0.0; S.hill[idd] = 0.0; S.alive[idd] = 0;
              S.T[idd] = 0ULL; S.rcsq[idd] = 0ULL;
              atomicAdd((unsigned long long *)&S.counters[C_MERGE], 1ULL);
            }
        }
        __syncthreads();
      }
      if (tid < g) for (int c = 0; c < 6; ++c) sh.y[tid][c] = sh.yn[tid][c];
      if (S.seq_len && tid < g && steps < BS_SEQCAP)  // adjoint engine: the state after this substep
        for (int c = 0; c < 6; ++c)
          S.y_scratch[(((size_t)rec_slot * BS_SEQCAP + steps) * BS_GMAX + tid) * 6 + c] = sh.yn[tid][c];
      if (tid == 0) {
        sh.rem = rem - Hs; sh.H = 2.0 * Hs;
        if (sh.nseq < BS_SEQCAP) { sh.seqH[sh.nseq] = Hs; sh.seqk[sh.nseq] = (unsigned char)acc; }
        sh.nseq++;
      }
      halvings = 0;
      steps++;
    } else {
      if (tid == 0) sh.H = 0.5 * H;
      if (++halvings > P.bs_max_halvings) {
        if (tid == 0) atomicOr(S.status, ST_BS_FAILED);
        __syncthreads();
        break;
      }
    }
    __syncthreads();
  }
  // write back: live members take the integrated state, ghosts are parked far out
  if (tid < g && S.bsn) S.bsn[sh.idx[tid]] = (unsigned char)(steps < 255 ? steps : 255);
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
    if (dbits(sh.U) != 0ULL) atomicAdd(S.U, sh.U);
    if (S.seq_len) {  // the adjoint engine records the accepted sequence
      int n = sh.nseq, base = -1;
      if (n <= BS_SEQCAP) {
        base = atomicAdd(S.seq_count, n);
        if (base + n > S.seq_cap) base = -1;
      }
      long long ybase = 0;
      if (base >= 0 && n > 1) {  // states after substeps 1 .. n-1 (the last one is the result)
        ybase = atomicAdd((unsigned long long *)S.y_count, (unsigned long long)((n - 1) * g * 6));
        if (ybase + (long long)(n - 1) * g * 6 > S.y_cap) base = -1;
      }
      if (base < 0) { atomicOr(S.status, ST_RECORD_OVERFLOW); n = 0; base = 0; ybase = 0; }
      S.seq_off[gidx] = base;
      S.seq_len[gidx] = n;
      S.y_off[gidx] = ybase;
      sh.seq_base = base;
      sh.y_base = ybase;
      sh.nseq = n;
    }
  }
  __syncthreads();
  if (S.seq_len) {
    for (int k = tid; k < sh.nseq; k += NT) S.seq_pool[sh.seq_base + k] = make_double2(sh.seqH[k], (double)sh.seqk[k]);
    const int ny = (sh.nseq > 1 ? sh.nseq - 1 : 0) * g * 6;
    for (int k = tid; k < ny; k += NT) {
      const int s = k / (g * 6), r = k % (g * 6);
      S.y_pool[sh.y_base + k] = S.y_scratch[(((size_t)rec_slot * BS_SEQCAP + s) * BS_GMAX + r / 6) * 6 + r % 6];
    }
  }
  __syncthreads();
}

}  // namespace genga
