// bs_grid.cu -- Bulirsch-Stoer of the largest encounter groups (Sect. 3.2) on the whole GPU.
//
// The paper integrates groups of up to 128 members in one block per group and, above that, splits
// the method into separate acceleration, error-estimation and acceptance kernels whose sequence the
// host controls. Here one launch takes the large groups one after another and spreads each over
// every SM, and the step control stays on the device: all CTAs hold the same control state (H, the
// remaining time, the halving count) and take the same decisions from the same data, with a grid
// barrier between the phases.
//
// One attempt of length H integrates all extrapolation levels L = 1..8 (n_L = 2L midpoint substeps)
// at once, as the one-CTA and cluster kernels do:
//   round 0      f(y) once per member, the error scales, every level's first substep
//   round r      every level with 2L >= r takes its r-th force evaluation; the work unit is
//                (level, 8 members), one warp per member summing the member's terms over all
//                partners (partner positions staged through shared memory in chunks); level L
//                writes T_{L,1} in round 2L
//   round 2Lc+1  besides the force work: row Lc of the Neville tableau for every (member,
//                component), its error into a per-level maximum; after the round's barrier every CTA
//                reads that maximum and the attempt ends at the first converged level
// An accepted substep is followed by the contact test of all member pairs (Hermite, as in the
// encounter search) and the mergers, applied by one thread in ascending pair order.
//
// Barrier: one launch, at most two CTAs per SM (13 KB of shared memory, 128 registers), so all CTAs
// become resident once the kernels beside it on other graph branches finish, none of which waits on
// this one. Every wait is bounded: after GR_SPIN_LIMIT polls a CTA sets the abort flag and the
// status bit ST_GRID_TIMEOUT, and every CTA leaves.
#include "genga_launch.h"

namespace genga {

// 1/((L/(L-j))^2 - 1), the Neville factors of the extrapolation in h^2 with n_k = 2k
__constant__ double c_facinv_gr[BS_LEVELS + 1][BS_LEVELS];

constexpr int GR_THREADS = 256;
constexpr int GR_WARPS = GR_THREADS / 32;   // members per work unit, one warp each
constexpr int GR_CHUNK = 256;               // partners staged in shared memory at a time
constexpr unsigned GR_SPIN_LIMIT = 1u << 21;  // polls of a barrier wait (about a second with back-off)

// Grid barrier. bar[0] counts arrivals, bar[1] is the generation, bar[2] the abort flag. gen (thread
// 0's copy) is the generation this CTA last passed. Returns false (uniformly in the CTA) when the
// wait was abandoned.
__device__ bool grid_sync(unsigned *bar, unsigned &gen, int *status, int *s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = gen + 1;
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], target);
    } else {
      volatile unsigned *vb = bar;
      unsigned spins = 0;
      while (vb[1] != target) {
        if (vb[2]) { ok = 0; break; }
        if (++spins > GR_SPIN_LIMIT) {
          atomicExch(&bar[2], 1u);
          atomicOr(status, ST_GRID_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    gen = target;
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

struct GrShared {
  double pos[GR_CHUNK][3];
  double gm[GR_CHUNK], A[GR_CHUNK];
  u64 rq[GR_CHUNK];
  int al[GR_CHUNK];
  int ok;
};

// H_A acceleration of member q (the central mass plus the (1 - K)-weighted pull of every live
// partner, as bs_terms in bs.cu) from the positions pl[p * stride + c] of the group's g members.
// Called by whole CTAs (it stages partner chunks with __syncthreads); warp w handles its member q
// (valid = false: the warp only helps staging). Every lane returns the sums.
__device__ void gr_accel(GrShared &sh, const BsGridBuf &B, const DevParams &P, double Gm0, const double *pl,
                         int stride, int g, int q, bool valid, double &ax, double &ay, double &az) {
  const int tid = threadIdx.x, lane = tid & 31;
  double xq = 0.0, yq = 0.0, zq = 0.0, Aq = 0.0;
  u64 rqq = 0ULL;
  bool qa = false;
  if (valid) {
    xq = __ldcg(pl + (size_t)q * stride); yq = __ldcg(pl + (size_t)q * stride + 1); zq = __ldcg(pl + (size_t)q * stride + 2);
    Aq = __ldcg(B.A + q); rqq = __ldcg(B.rcsq + q); qa = __ldcg(B.alive + q) != 0;
  }
  ax = ay = az = 0.0;
  for (int c0 = 0; c0 < g; c0 += GR_CHUNK) {
    const int n = g - c0 < GR_CHUNK ? g - c0 : GR_CHUNK;
    __syncthreads();
    for (int t = tid; t < n; t += GR_THREADS) {
      const int p = c0 + t;
      sh.pos[t][0] = __ldcg(pl + (size_t)p * stride);
      sh.pos[t][1] = __ldcg(pl + (size_t)p * stride + 1);
      sh.pos[t][2] = __ldcg(pl + (size_t)p * stride + 2);
      sh.gm[t] = __ldcg(B.gm + p); sh.A[t] = __ldcg(B.A + p); sh.rq[t] = __ldcg(B.rcsq + p); sh.al[t] = __ldcg(B.alive + p);
    }
    __syncthreads();
    if (qa) {
      for (int t = lane; t < n; t += 32) {
        const bool cen = c0 + t == q;
        const double dx = (cen ? 0.0 : sh.pos[t][0]) - xq, dy = (cen ? 0.0 : sh.pos[t][1]) - yq,
                     dz = (cen ? 0.0 : sh.pos[t][2]) - zq;
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double yr = rsqrt_refined(r2);
        const bool inside = sh.al[t] && dbits(r2) < umax64(rqq, sh.rq[t]);
        const double wA = changeover_wA_clamped(r2 * yr, pmin(Aq, sh.A[t]), P.kmode);
        const double w = cen ? 1.0 : (inside ? wA : 0.0);
        const double f = (cen ? Gm0 : sh.gm[t]) * w * (yr * yr * yr);
        ax = fma(f, dx, ax); ay = fma(f, dy, ay); az = fma(f, dz, az);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
  }
}

__global__ void __launch_bounds__(GR_THREADS, 2) k_bs_grid(Sim S, DevParams P, double tau, int gmin) {
  __shared__ GrShared sh;
  const BsGridBuf B = S.gb;
  const int gcap = S.npad, np = S.npad;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int gthreads = gridDim.x * GR_THREADS, gtid = blockIdx.x * GR_THREADS + tid;
  const int gwarps = gridDim.x * GR_WARPS, gwid = blockIdx.x * GR_WARPS + wid;
  unsigned gen = 0;
  if (tid == 0) gen = *(volatile unsigned *)&B.bar[1];
  const int nbig = *S.nbig;
  const int lmax = P.bs_kmax < BS_LEVELS ? P.bs_kmax : BS_LEVELS;
  const u64 eps = dbits(P.bs_eps);
  const double Gm0 = P.G * P.m0;
  for (int k = 0; k < nbig; ++k) {
    const int gidx = S.big[k];
    const int g0 = S.gstart[gidx], g = S.gstart[gidx + 1] - g0;
    if (g < gmin || g > gcap) continue;  // uniform: a smaller group belongs to the cluster kernel
    for (int q = gtid; q < g; q += gthreads) {
      const int i = S.gmem[g0 + q];
      B.idx[q] = i;
      B.alive[q] = S.alive[i];
      B.gm[q] = S.gm[i]; B.m[q] = S.m[i]; B.R[q] = S.R[i]; B.A[q] = S.A[i]; B.rcsq[q] = S.rcsq[i];
      for (int c = 0; c < 3; ++c) { B.y[q * 6 + c] = S.x0[c * np + i]; B.y[q * 6 + 3 + c] = S.v0[c * np + i]; }
    }
    if (gtid < 2 * BS_LEVELS) B.err[gtid] = 0ULL;
    if (gtid == 0) *B.ncont = 0;
    if (!grid_sync(B.bar, gen, S.status, &sh.ok)) return;
    const int nblk = (g + GR_WARPS - 1) / GR_WARPS;
    double H = tau, rem = tau, U = 0.0;
    int halvings = 0, attempts = 0, steps = 0, cur = 0, par = 0;
    while (true) {
      if (absbits(rem) == 0ULL) break;
      if (absbits(H) > absbits(rem)) H = rem;
      if (++attempts > 200000) { if (gtid == 0) atomicOr(S.status, ST_BS_FAILED); break; }
      const double *yc = B.y + (size_t)cur * gcap * 6;
      double *yn = B.y + (size_t)(cur ^ 1) * gcap * 6;
      u64 *err = B.err + par * BS_LEVELS;
      // ---- round 0: f(y) per member, error scales, the first substep of every level ----
      for (int u = blockIdx.x; u < nblk; u += gridDim.x) {
        const int q = u * GR_WARPS + wid;
        const bool valid = q < g;
        double ax, ay, az;
        gr_accel(sh, B, P, Gm0, yc, 6, g, q, valid, ax, ay, az);
        if (valid) {
          const bool qa = __ldcg(B.alive + q) != 0;
          double z[6];
          for (int c = 0; c < 6; ++c) z[c] = __ldcg(yc + (size_t)q * 6 + c);
          if (lane < lmax) {  // level L = lane + 1
            const int L = lane + 1;
            const double h = __ddiv_rn(H, (double)(2 * L));
            double zb[6];
            if (qa) {
              zb[0] = fma(h, z[3], z[0]); zb[1] = fma(h, z[4], z[1]); zb[2] = fma(h, z[5], z[2]);
              zb[3] = fma(h, ax, z[3]); zb[4] = fma(h, ay, z[4]); zb[5] = fma(h, az, z[5]);
            } else {
              for (int c = 0; c < 6; ++c) zb[c] = z[c];
            }
            const size_t zi = ((size_t)(L - 1) * gcap + q) * 6;
            for (int c = 0; c < 6; ++c) { B.za[zi + c] = z[c]; B.zb[zi + c] = zb[c]; }
            double *pw = B.pos + ((size_t)(BS_LEVELS + L - 1) * gcap + q) * 3;  // buffer 1
            pw[0] = zb[0]; pw[1] = zb[1]; pw[2] = zb[2];
          } else if (lane == 8 || lane == 9) {  // error scale 1/|x| (lane 8) or 1/|v| (lane 9)
            const double *w = z + (lane == 8 ? 0 : 3);
            const double s2 = fma(w[2], w[2], fma(w[1], w[1], w[0] * w[0]));
            B.isc[q * 2 + lane - 8] = dbits(s2) == 0ULL ? 4.49423283715579e307 : rsqrt_refined(s2);
          }
        }
      }
      if (!grid_sync(B.bar, gen, S.status, &sh.ok)) return;
      // ---- rounds 1 .. 2 lmax + 1 ----
      int acc = 0;
      for (int r = 1; r <= 2 * lmax + 1; ++r) {
        if (r == 1 && gtid < BS_LEVELS) B.err[(par ^ 1) * BS_LEVELS + gtid] = 0ULL;  // the next attempt's maxima
        if ((r & 1) && r >= 3) {  // row Lc of the tableau: level Lc completed in round r - 1
          const int Lc = (r - 1) >> 1;
          for (int e = gtid; e < 6 * g; e += gthreads) {
            const int q = e / 6, c = e % 6;
            double *pr = B.prev + (size_t)e * BS_LEVELS;
            double prevr[BS_LEVELS];
#pragma unroll
            for (int j = 0; j < BS_LEVELS; ++j) prevr[j] = (j < Lc - 1) ? __ldcg(pr + j) : 0.0;
            double before;
            const double t1 = __ldcg(B.t1 + ((size_t)(Lc - 1) * gcap + q) * 6 + c);
            const double last = neville_row(t1, Lc, [&](int j) { return c_facinv_gr[Lc][j]; }, prevr, before);
#pragma unroll
            for (int j = 0; j < BS_LEVELS; ++j)
              if (j < Lc) pr[j] = prevr[j];
            yn[e] = last;  // T_{Lc,Lc}: the new state if level Lc is accepted
            if (Lc >= 2 && __ldcg(B.alive + q)) {
              const double scale = __ldcg(B.isc + q * 2 + (c < 3 ? 0 : 1));
              atomicMax(&err[Lc - 1], absbits((last - before) * scale));
            }
          }
        }
        if (r <= 2 * lmax) {  // force evaluation r of every level with 2L >= r
          const int Lmin = (r + 1) >> 1;
          const int nunits = (lmax - Lmin + 1) * nblk;
          const int rb = r & 1, wb = rb ^ 1;
          for (int uu = blockIdx.x; uu < nunits; uu += gridDim.x) {
            const int L = Lmin + uu / nblk, u = uu % nblk, nk = 2 * L;
            const int q = u * GR_WARPS + wid;
            const bool valid = q < g;
            const double *pl = B.pos + (size_t)(rb * BS_LEVELS + L - 1) * gcap * 3;
            double ax, ay, az;
            gr_accel(sh, B, P, Gm0, pl, 3, g, q, valid, ax, ay, az);
            if (valid && lane < 6) {
              const int c = lane;
              const bool qa = __ldcg(B.alive + q) != 0;
              const size_t zi = ((size_t)(L - 1) * gcap + q) * 6;
              const double zAc = __ldcg(B.za + zi + c), zBc = __ldcg(B.zb + zi + c);
              const double drv = c < 3 ? __ldcg(B.zb + zi + c + 3) : (c == 3 ? ax : (c == 4 ? ay : az));
              const double h = __ddiv_rn(H, (double)nk), h2 = 2.0 * h;
              if (r < nk) {
                const double zn = qa ? fma(h2, drv, zAc) : zBc;
                B.za[zi + c] = zBc;
                B.zb[zi + c] = zn;
                if (c < 3) B.pos[((size_t)(wb * BS_LEVELS + L - 1) * gcap + q) * 3 + c] = zn;
              } else {  // r == nk: the level's modified-midpoint result T_{L,1}
                B.t1[zi + c] = qa ? 0.5 * fma(h, drv, zBc + zAc) : zAc;
              }
            }
          }
        }
        if (!grid_sync(B.bar, gen, S.status, &sh.ok)) return;
        if ((r & 1) && r >= 5) {
          const int Lc = (r - 1) >> 1;
          if (*(volatile u64 *)&err[Lc - 1] <= eps) { acc = Lc; break; }  // the same value in every CTA
        }
      }
      par ^= 1;
      if (!acc) {
        H = 0.5 * H;
        if (++halvings > P.bs_max_halvings) {
          if (gtid == 0) atomicOr(S.status, ST_BS_FAILED);
          break;
        }
        continue;
      }
      halvings = 0;
      steps++;
      if (P.collisions) {  // contact test over the substep (Hermite, threshold (R_a + R_b)^2), pre-merge states
        for (int a = gwid; a < g; a += gwarps) {
          if (!__ldcg(B.alive + a)) continue;  // uniform in the warp
          const double Ra = __ldcg(B.R + a);
          double ya[6], yna[6];
          for (int c = 0; c < 6; ++c) { ya[c] = __ldcg(yc + (size_t)a * 6 + c); yna[c] = __ldcg(yn + (size_t)a * 6 + c); }
          for (int b = a + 1 + lane; b < g; b += 32) {
            if (!__ldcg(B.alive + b)) continue;
            double yb[6], ynb[6];
            for (int c = 0; c < 6; ++c) { yb[c] = __ldcg(yc + (size_t)b * 6 + c); ynb[c] = __ldcg(yn + (size_t)b * 6 + c); }
            const double rr = Ra + __ldcg(B.R + b);
            const double dmin = hermite_min_capped(
                __dsub_rn(yb[0], ya[0]), __dsub_rn(yb[1], ya[1]), __dsub_rn(yb[2], ya[2]),
                __dsub_rn(yb[3], ya[3]), __dsub_rn(yb[4], ya[4]), __dsub_rn(yb[5], ya[5]),
                __dsub_rn(ynb[0], yna[0]), __dsub_rn(ynb[1], yna[1]), __dsub_rn(ynb[2], yna[2]),
                __dsub_rn(ynb[3], yna[3]), __dsub_rn(ynb[4], yna[4]), __dsub_rn(ynb[5], yna[5]), H, rr * rr);
            if (dmin < rr * rr) {
              const int s = atomicAdd(B.ncont, 1);
              if (s < GR_CONTACT_CAP) B.cont[s] = a * gcap + b;
            }
          }
        }
        if (!grid_sync(B.bar, gen, S.status, &sh.ok)) return;
        if (gtid == 0) {  // mergers in ascending pair order on the post-substep states
          // (every read bypasses L1: these arrays are written by other CTAs within the launch)
          int nc = __ldcg(B.ncont);
          if (nc > GR_CONTACT_CAP) { atomicOr(S.status, ST_BS_FAILED); nc = GR_CONTACT_CAP; }
          for (int s = 1; s < nc; ++s) {  // insertion sort of the (few) contact keys
            const int key = __ldcg(B.cont + s);
            int t = s - 1;
            while (t >= 0 && __ldcg(B.cont + t) > key) { B.cont[t + 1] = __ldcg(B.cont + t); --t; }
            B.cont[t + 1] = key;
          }
          for (int s = 0; s < nc; ++s) {
            const int key = __ldcg(B.cont + s);
            const int a = key / gcap, bq = key % gcap;
            if (!__ldcg(B.alive + a) || !__ldcg(B.alive + bq)) continue;
            double *ya = yn + (size_t)a * 6, *yb = yn + (size_t)bq * 6;
            double va[6], vb[6];
            for (int c = 0; c < 6; ++c) { va[c] = __ldcg(ya + c); vb[c] = __ldcg(yb + c); }
            const int ia = __ldcg(B.idx + a), ib = __ldcg(B.idx + bq);
            const double ma = __ldcg(B.m + a), mb = __ldcg(B.m + bq), M = ma + mb;
            const double dx = vb[0] - va[0], dy = vb[1] - va[1], dz = vb[2] - va[2];
            const double dvx = vb[3] - va[3], dvy = vb[4] - va[4], dvz = vb[5] - va[5];
            const double rr = sqrt(dx * dx + dy * dy + dz * dz);
            const double v2 = dvx * dvx + dvy * dvy + dvz * dvz;
            U += 0.5 * ma * mb / M * v2 - P.G * ma * mb / rr;
            const bool keep_a = ma > mb || (ma == mb && ia < ib);
            {
              double ya0[6], yb0[6];  // the pair's states at the start of the substep
              for (int c = 0; c < 6; ++c) { ya0[c] = __ldcg(yc + (size_t)a * 6 + c); yb0[c] = __ldcg(yc + (size_t)bq * 6 + c); }
              merger_report(S, ia, ib, ya0, yb0, va, vb, ma, mb, keep_a, tau - rem);
            }
            const int sv = keep_a ? a : bq, dd = keep_a ? bq : a;
            double *ys = yn + (size_t)sv * 6;
            for (int c = 0; c < 6; ++c) ys[c] = (ma * va[c] + mb * vb[c]) / M;
            const double Ra = __ldcg(B.R + a), Rb = __ldcg(B.R + bq);
            const double Rs = cbrt(Ra * Ra * Ra + Rb * Rb * Rb);
            B.R[sv] = Rs;
            B.m[sv] = M; B.gm[sv] = P.G * M;
            B.m[dd] = 0.0; B.gm[dd] = 0.0; B.R[dd] = 0.0; B.alive[dd] = 0;
            const int is = keep_a ? ia : ib, idd = keep_a ? ib : ia;
            S.m[is] = M; S.gm[is] = P.G * M; S.R[is] = Rs; S.hill[is] = cbrt(M / (3.0 * P.m0));
            S.m[idd] = 0.0; S.gm[idd] = 0.0; S.R[idd] = 0.0; S.hill[idd] = 0.0; S.alive[idd] = 0;
            S.T[idd] = 0ULL; S.rcsq[idd] = 0ULL;
            atomicAdd((unsigned long long *)&S.counters[C_MERGE], 1ULL);
          }
          *B.ncont = 0;
        }
        if (!grid_sync(B.bar, gen, S.status, &sh.ok)) return;
      }
      cur ^= 1;
      rem = rem - H;
      H = 2.0 * H;
    }
    // write back: live members take the integrated state, ghosts are parked far out
    const double *yf = B.y + (size_t)cur * gcap * 6;
    for (int q = gtid; q < g; q += gthreads) {
      const int i = __ldcg(B.idx + q);
      if (__ldcg(B.alive + q)) {
        for (int c = 0; c < 3; ++c) { S.x[c * np + i] = __ldcg(yf + (size_t)q * 6 + c); S.v[c * np + i] = __ldcg(yf + (size_t)q * 6 + 3 + c); }
      } else {
        S.x[i] = PARK + 1.0e4 * i; S.x[np + i] = 0.0; S.x[2 * np + i] = 0.0;
        for (int c = 0; c < 3; ++c) S.v[c * np + i] = 0.0;
      }
    }
    if (gtid == 0) {
      atomicAdd((unsigned long long *)&S.counters[C_BSSTEPS], (unsigned long long)steps);
      if (dbits(U) != 0ULL) atomicAdd(S.U, U);
    }
    if (!grid_sync(B.bar, gen, S.status, &sh.ok)) return;  // the next group reuses the buffers
  }
}

void bs_grid_init_constants() {
  double h[BS_LEVELS + 1][BS_LEVELS] = {};
  for (int Lv = 2; Lv <= BS_LEVELS; ++Lv)
    for (int j = 1; j < Lv; ++j) {
      const double ratio = (double)Lv / (double)(Lv - j);
      h[Lv][j] = 1.0 / (ratio * ratio - 1.0);
    }
  cudaMemcpyToSymbol(c_facinv_gr, h, sizeof(h));
}

// Two CTAs per SM (or what the occupancy query allows), never more than can be resident at once.
int bs_grid_blocks() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bs_grid, GR_THREADS, 0) != cudaSuccess || per < 1) per = 1;
  cudaGetLastError();
  if (per > 2) per = 2;
  return (sms > 0 ? sms : 1) * per;
}

void launch_bs_grid(const Sim &S, const DevParams &P, double tau, int gmin, int blocks, cudaStream_t st) {
  cudaMemsetAsync(S.gb.bar, 0, 4 * sizeof(unsigned), st);
  k_bs_grid<<<blocks < 1 ? 1 : blocks, GR_THREADS, 0, st>>>(S, P, tau, gmin);
}

}  // namespace genga
