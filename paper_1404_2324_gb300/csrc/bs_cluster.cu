// bs_cluster.cu -- Bulirsch-Stoer of the larger encounter groups (Sect. 3.2) on a thread-block
// cluster of 8 CTAs: CTA r integrates extrapolation level r + 1 (n = 2(r + 1) midpoint substeps).
//
// A group of g members costs 8 levels x g members x g terms per force evaluation; on one SM (the
// one-CTA kernel in bs.cu) that saturates the FP64 pipes once g reaches a handful. Here each level
// has an SM of its own. After every second evaluation the CTAs meet at a cluster barrier; level Lc
// is then complete in CTA Lc - 1, every CTA reads its T_{Lc,1} from that CTA's shared memory
// (distributed shared memory), extends its own copy of the Neville tableau and tests level Lc, with
// the same arithmetic and order in every CTA. Groups of more than 8 members evaluate each pair
// once (Newton's third law), so that up to 15 members take one FP64 round per SM sub-partition per
// force evaluation. All CTAs therefore take the same decision
// and follow the same control flow: every cluster barrier is reached by all 8 CTAs the same number
// of times. Level results are double-buffered by attempt parity. Cluster k takes the k-th entry of
// the large-group list that the grouping kernel writes.
#include <cooperative_groups.h>

#include "genga_launch.h"

namespace cg = cooperative_groups;

namespace genga {

constexpr int CL_SIZE = BS_LEVELS;  // CTAs per cluster, one per level
constexpr int CL_THREADS = 256;
constexpr int CL_TPS = CL_THREADS / BS_GMAX;  // lanes per member (8)
constexpr int CL_PAIRS = BS_GMAX * (BS_GMAX - 1) / 2;
constexpr int CL_ITEMS = BS_GMAX + CL_PAIRS;  // a force evaluation's terms: one per member, one per pair
// the first level whose convergence is tested: groups of five or more members converge at level 5
// or later in practice, and a level below it that converges is still found (its row is kept), at
// the cost of the evaluations up to this level
constexpr int CL_FIRST_CHECK = 4;

// 1/((L/(L-j))^2 - 1), the Neville factors (same values as the one-CTA kernel's table)
__constant__ double c_facinv_cl[BS_LEVELS + 1][BS_LEVELS];

struct BsClShared {
  int idx[BS_GMAX], alive[BS_GMAX];
  double gm[BS_GMAX], m[BS_GMAX], R[BS_GMAX], A[BS_GMAX];
  u64 rcsq[BS_GMAX];
  double y[BS_GMAX][6], yn[BS_GMAX][6];
  double isc[BS_GMAX][2];                // 1/|x|, 1/|v| at the start of the attempt
  double pos[2][BS_GMAX][3];             // chain positions, double-buffered by evaluation
  double term[CL_ITEMS][3];              // this evaluation's terms: central pulls, then pair factors
  double acc[BS_GMAX][3];                // this evaluation's accelerations
  unsigned char pa[CL_PAIRS], pb[CL_PAIRS];  // pair k = (pa[k], pb[k]), pa < pb, row by row
  double T1[2][BS_GMAX][6];              // this level's result, double-buffered by attempt
  u64 err[BS_LEVELS];
  unsigned char cont[BS_GMAX * (BS_GMAX - 1) / 2];
  double H, rem, U;
  int accept, nseq;
  long long y_base;
  int seq_base;
  double seqH[BS_SEQCAP];
  unsigned char seqk[BS_SEQCAP];
};

// Groups of up to CL_TPS members: the terms of member q over partners p = sub, sub + CL_TPS, ...
// (p == q: the central mass; one term per lane), summed over the member's lanes by a butterfly;
// the same straight-line code on every lane (see bs.cu).
__device__ __forceinline__ void cl_terms(const BsClShared &sh, const DevParams &P, double Gm0, int g, int q, int sub,
                                         const double (*pos)[3], bool q_alive, double &ax, double &ay, double &az) {
  ax = ay = az = 0.0;
  const double xq = pos[q][0], yq = pos[q][1], zq = pos[q][2];
  if (q_alive) {
    for (int p = sub; p < g; p += CL_TPS) {
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
#pragma unroll
  for (int o = CL_TPS >> 1; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
  }
}

// Groups of more than CL_TPS members: one force evaluation at positions pos, by all threads of the
// CTA, into sh.acc.
// Every unordered pair is evaluated once (Newton's third law), beside the central mass's pull on
// each member: term t < g is member t's central pull G m0 d / r^3 (d from the member to the central
// mass; zero for a ghost), term g + k the factor w d / r^3 of pair k = (a, b), d = x_b - x_a, w the
// (1 - K) weight inside the pair's critical radius and 0 outside or for a ghost. Then member a sums,
// one component per thread group, its central pull and G m_b times its pair factors (with the sign
// of d) over the partners b in a fixed order. Item after item, every lane runs the same
// straight-line code; a group of up to 15 members needs one FP64 round per SM sub-partition, where
// a thread per (member, partner slot) needs two.
__device__ __forceinline__ void cl_eval(BsClShared &sh, const DevParams &P, double Gm0, int g, const double (*pos)[3]) {
  const int tid = threadIdx.x;
  const int nitems = g + g * (g - 1) / 2;
  for (int t = tid; t < nitems; t += CL_THREADS) {
    const bool cen = t < g;
    const int a = cen ? t : sh.pa[t - g], b = cen ? t : sh.pb[t - g];
    const double dx = (cen ? 0.0 : pos[b][0]) - pos[a][0], dy = (cen ? 0.0 : pos[b][1]) - pos[a][1],
                 dz = (cen ? 0.0 : pos[b][2]) - pos[a][2];
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const double yr = rsqrt_refined(r2);
    const bool inside = sh.alive[a] && sh.alive[b] && dbits(r2) < umax64(sh.rcsq[a], sh.rcsq[b]);
    const double wA = changeover_wA_clamped(r2 * yr, pmin(sh.A[a], sh.A[b]), P.kmode);
    const double w = cen ? (sh.alive[a] ? Gm0 : 0.0) : (inside ? wA : 0.0);
    const double f = w * (yr * yr * yr);
    sh.term[t][0] = f * dx; sh.term[t][1] = f * dy; sh.term[t][2] = f * dz;
  }
  __syncthreads();
  // member a, component c: ns threads, thread s takes the partners b = s, s + ns, ... (s = 0 also
  // the central pull), partial sums combined by a butterfly over the ns lanes
  const int ns = 24 * g <= CL_THREADS ? 8 : (12 * g <= CL_THREADS ? 4 : 2);
  const int a = tid / (3 * ns), c = (tid / ns) % 3, sl = tid % ns;
  double v = 0.0;
  if (a < g) {
    if (sl == 0) v = sh.term[a][c];
    const int rowa = g + a * (g - 1) - a * (a - 1) / 2 - a - 1;  // term of pair (a, b > a): rowa + b
    for (int bq = sl; bq < g; bq += ns) {
      if (bq == a) continue;
      if (bq > a) v = fma(sh.gm[bq], sh.term[rowa + bq][c], v);
      else v = fma(-sh.gm[bq], sh.term[g + bq * (g - 1) - bq * (bq - 1) / 2 + a - bq - 1][c], v);
    }
  }
  for (int o = ns >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (a < g && sl == 0) sh.acc[a][c] = v;
  __syncthreads();
}

__global__ void __cluster_dims__(CL_SIZE, 1, 1) __launch_bounds__(CL_THREADS, 2)
    k_bs_cluster(Sim S, DevParams P, double tau, int gmin) {
  __shared__ BsClShared sh;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int L = rank + 1, nk = 2 * L;
  const int tid = threadIdx.x, q = tid / CL_TPS, sub = tid % CL_TPS;
  const int np = S.npad;
  const int ngroups = *S.ngroups;
  const int ncl = gridDim.x / CL_SIZE, cid = blockIdx.x / CL_SIZE;
  // the groups listed by size (one per cluster while there are no more than clusters), else all
  const int nwork = S.big ? *S.nbig : ngroups;
  for (int k = cid; k < nwork; k += ncl) {
    const int gidx = S.big ? S.big[k] : k;
    const int g0 = S.gstart[gidx], g = S.gsize ? S.gsize[gidx] : S.gstart[gidx + 1] - g0;
    if (g < gmin || g > BS_GMAX) continue;  // the same for all CTAs of the cluster (g < gmin: one-CTA kernel)
    const double m0 = S.sys_of ? S.sys_m0[S.sys_of[S.gmem[g0]]] : P.m0;
    const double Gm0 = P.G * m0;
    const bool act = q < g;
    if (tid < g) {
      const int i = S.gmem[g0 + tid];
      sh.idx[tid] = i;
      sh.alive[tid] = S.alive[i];
      sh.gm[tid] = S.gm[i]; sh.m[tid] = S.m[i]; sh.R[tid] = S.R[i]; sh.A[tid] = S.A[i];
      sh.rcsq[tid] = S.rcsq[i];
      for (int c = 0; c < 3; ++c) { sh.y[tid][c] = S.x0[c * np + i]; sh.y[tid][3 + c] = S.v0[c * np + i]; }
    }
    if (tid == 0) { sh.H = tau; sh.rem = tau; sh.U = 0.0; sh.nseq = 0; }
    for (int k = tid; k < g * (g - 1) / 2; k += CL_THREADS) {
      int pa = 0, rest = k;
      while (rest >= g - 1 - pa) { rest -= g - 1 - pa; pa++; }
      sh.pa[k] = (unsigned char)pa;
      sh.pb[k] = (unsigned char)(pa + 1 + rest);
    }
    __syncthreads();
    int halvings = 0, attempts = 0, steps = 0, buf = 0;
    while (true) {
      const double rem = sh.rem;
      double H = sh.H;
      if (absbits(rem) == 0ULL) break;
      if (absbits(H) > absbits(rem)) H = rem;
      if (++attempts > 200000) { if (tid == 0 && rank == 0) atomicOr(S.status, ST_BS_FAILED); break; }
      const double h = __ddiv_rn(H, (double)nk), h2 = 2.0 * h;
      const bool qa = act && sh.alive[q];
      if (tid < g) {  // error scales at the start of the attempt
        const double *yq = sh.y[tid];
        const double sx2 = fma(yq[2], yq[2], fma(yq[1], yq[1], yq[0] * yq[0]));
        const double sv2 = fma(yq[5], yq[5], fma(yq[4], yq[4], yq[3] * yq[3]));
        sh.isc[tid][0] = dbits(sx2) == 0ULL ? 4.49423283715579e307 : rsqrt_refined(sx2);
        sh.isc[tid][1] = dbits(sv2) == 0ULL ? 4.49423283715579e307 : rsqrt_refined(sv2);
      }
      // ---- this level's modified-midpoint integration; levels checked as they complete ----
      // Level Lc finishes at evaluation 2 Lc. At every even evaluation all CTAs meet at a cluster
      // barrier, read T_{Lc,1} from its CTA, extend their tableau rows (thread (qc, cc): member
      // qc, component cc) and test level Lc; the first converged level ends the attempt in every
      // CTA at once (the same data, the same arithmetic, so the same decision).
      double zA[6], zB[6], out[6];
      for (int c = 0; c < 6; ++c) zA[c] = act ? sh.y[q][c] : 0.0;
      if (act && sub == 0) for (int c = 0; c < 3; ++c) sh.pos[0][q][c] = zA[c];
      const int qc = tid / 6, cc = tid % 6;
      const bool rowth = qc < g;
      if (tid < BS_LEVELS) sh.err[tid] = 0ULL;
      __syncthreads();
      double ax = 0.0, ay = 0.0, az = 0.0;
      if (g > CL_TPS) {
        cl_eval(sh, P, Gm0, g, sh.pos[0]);
        if (act) { ax = sh.acc[q][0]; ay = sh.acc[q][1]; az = sh.acc[q][2]; }
      } else if (__any_sync(0xffffffffu, act)) {
        cl_terms(sh, P, Gm0, g, act ? q : 0, sub, sh.pos[0], qa, ax, ay, az);
      }
      if (qa) {
        zB[0] = fma(h, zA[3], zA[0]); zB[1] = fma(h, zA[4], zA[1]); zB[2] = fma(h, zA[5], zA[2]);
        zB[3] = fma(h, ax, zA[3]); zB[4] = fma(h, ay, zA[4]); zB[5] = fma(h, az, zA[5]);
      } else {
        for (int c = 0; c < 6; ++c) zB[c] = zA[c];
      }
      const int lmax = P.bs_kmax < BS_LEVELS ? P.bs_kmax : BS_LEVELS;
      const u64 eps = dbits(P.bs_eps);
      const double scale = rowth ? sh.isc[qc][cc < 3 ? 0 : 1] : 0.0;
      double prev[BS_LEVELS], tlast = 0.0;  // previous tableau row; T_{Lc,Lc} of the current one
      int acc = 0;
      int b = 1;
      for (int e = 1; e <= 2 * lmax; ++e) {
        const bool lv = e <= nk;  // this CTA's level is still integrating
        if (lv) {
          if (act && sub == 0) for (int c = 0; c < 3; ++c) sh.pos[b][q][c] = zB[c];
          __syncthreads();
          if (g > CL_TPS) {
            cl_eval(sh, P, Gm0, g, sh.pos[b]);
            if (act) { ax = sh.acc[q][0]; ay = sh.acc[q][1]; az = sh.acc[q][2]; }
          } else if (__any_sync(0xffffffffu, act)) {
            cl_terms(sh, P, Gm0, g, act ? q : 0, sub, sh.pos[b], qa, ax, ay, az);
          }
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
          } else if (act && e == nk) {
            for (int c = 0; c < 6; ++c) out[c] = zA[c];
          }
          if (e == nk && act && sub == 0) for (int c = 0; c < 6; ++c) sh.T1[buf][q][c] = out[c];
          b ^= 1;
        }
        if (e & 1) continue;
        const int Lc = e >> 1;
        // the rows of the levels below the first check are built with it: the same rows and the same
        // first converged level as a check per level, one cluster barrier instead of CL_FIRST_CHECK
        const int fc = lmax < CL_FIRST_CHECK ? lmax : CL_FIRST_CHECK;
        if (Lc < fc) continue;
        cluster.sync();  // T_{r,1} is complete in CTA r - 1 for every r <= Lc
        const int r0 = Lc == fc ? 1 : Lc;
        double tk[CL_FIRST_CHECK + 1];  // T_{r,r} of the rows built at the first check
#pragma unroll
        for (int r = 1; r <= BS_LEVELS; ++r) {
          if (r < r0 || r > Lc) continue;  // uniform
          u64 ev = 0ULL;
          if (rowth) {
            const double *rt = cluster.map_shared_rank(&sh.T1[buf][0][0], (unsigned)(r - 1));
            double before;
            tlast = neville_row(rt[qc * 6 + cc], r, [&](int j) { return c_facinv_cl[r][j]; }, prev, before);
            if (r >= 2 && sh.alive[qc]) ev = absbits((tlast - before) * scale);
            if (r <= CL_FIRST_CHECK) tk[r] = tlast;
          }
          if (r >= 2) warp_max_to(&sh.err[r - 1], ev);
        }
        __syncthreads();
        for (int r = r0 < 2 ? 2 : r0; r <= Lc; ++r)  // uniform: every thread reads the same errors
          if (sh.err[r - 1] <= eps) { acc = r; break; }
        if (acc) {
          if (acc < Lc && rowth) tlast = tk[acc];
          break;
        }
      }
      if (acc && rowth) sh.yn[qc][cc] = tlast;  // the accepted row is the last one built
      buf ^= 1;
      if (acc) {
        __syncthreads();
        if (P.collisions) {  // contact test and mergers, redundantly in every CTA; globals by rank 0
          const int npair = g * (g - 1) / 2;
          int anyhit = 0;
          for (int pi = tid; pi < npair; pi += CL_THREADS) {
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
                  __dsub_rn(sh.yn[bq][3], sh.yn[a][3]), __dsub_rn(sh.yn[bq][4], sh.yn[a][4]), __dsub_rn(sh.yn[bq][5], sh.yn[a][5]), H, rr * rr);
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
                if (rank == 0) merger_report(S, ia, ib, sh.y[a], sh.y[bq], sh.yn[a], sh.yn[bq], ma, mb, keep_a, tau - rem);
                const int s = keep_a ? a : bq, d = keep_a ? bq : a;
                for (int c = 0; c < 6; ++c) sh.yn[s][c] = (ma * sh.yn[a][c] + mb * sh.yn[bq][c]) / M;
                const double Ra = sh.R[a], Rb = sh.R[bq];
                sh.R[s] = cbrt(Ra * Ra * Ra + Rb * Rb * Rb);
                sh.m[s] = M; sh.gm[s] = P.G * M;
                sh.m[d] = 0.0; sh.gm[d] = 0.0; sh.R[d] = 0.0; sh.alive[d] = 0;
                if (rank == 0) {
                  const int is = sh.idx[s], idd = sh.idx[d];
                  S.m[is] = M; S.gm[is] = P.G * M; S.R[is] = sh.R[s]; S.hill[is] = cbrt(M / (3.0 * m0));
                  S.m[idd] = 0.0; S.gm[idd] = 0.0; S.R[idd] = 0.0; S.hill[idd] = 0.0; S.alive[idd] = 0;
                  S.T[idd] = 0ULL; S.rcsq[idd] = 0ULL;
                  atomicAdd((unsigned long long *)&S.counters[C_MERGE], 1ULL);
                }
              }
          }
          __syncthreads();
        }
        if (tid < g) for (int c = 0; c < 6; ++c) sh.y[tid][c] = sh.yn[tid][c];
        if (rank == 0 && S.seq_len && tid < g && steps < BS_SEQCAP)  // adjoint engine: state after this substep
          for (int c = 0; c < 6; ++c)
            S.y_scratch[(((size_t)cid * BS_SEQCAP + steps) * BS_GMAX + tid) * 6 + c] = sh.yn[tid][c];
        if (tid == 0) {
          sh.rem = rem - H; sh.H = 2.0 * H;
          if (sh.nseq < BS_SEQCAP) { sh.seqH[sh.nseq] = H; sh.seqk[sh.nseq] = (unsigned char)acc; }
          sh.nseq++;
        }
        halvings = 0;
        steps++;
      } else {
        if (tid == 0) sh.H = 0.5 * H;
        if (++halvings > P.bs_max_halvings) {
          if (tid == 0 && rank == 0) atomicOr(S.status, ST_BS_FAILED);
          __syncthreads();
          break;
        }
      }
      __syncthreads();
    }
    // write-back, counters and the adjoint recording by rank 0
    if (rank == 0) {
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
        if (S.seq_len) {
          int n = sh.nseq, base = -1;
          if (n <= BS_SEQCAP) {
            base = atomicAdd(S.seq_count, n);
            if (base + n > S.seq_cap) base = -1;
          }
          long long ybase = 0;
          if (base >= 0 && n > 1) {
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
        for (int k = tid; k < sh.nseq; k += CL_THREADS) S.seq_pool[sh.seq_base + k] = make_double2(sh.seqH[k], (double)sh.seqk[k]);
        const int ny = (sh.nseq > 1 ? sh.nseq - 1 : 0) * g * 6;
        for (int k = tid; k < ny; k += CL_THREADS) {
          const int s = k / (g * 6), r = k % (g * 6);
          S.y_pool[sh.y_base + k] = S.y_scratch[(((size_t)cid * BS_SEQCAP + s) * BS_GMAX + r / 6) * 6 + r % 6];
        }
      }
    }
    cluster.sync();  // no CTA starts the next group while another may still read its results
  }
}

void bs_cluster_init_constants() {
  double h[BS_LEVELS + 1][BS_LEVELS] = {};
  for (int Lv = 2; Lv <= BS_LEVELS; ++Lv)
    for (int j = 1; j < Lv; ++j) {
      const double ratio = (double)Lv / (double)(Lv - j);
      h[Lv][j] = 1.0 / (ratio * ratio - 1.0);
    }
  cudaMemcpyToSymbol(c_facinv_cl, h, sizeof(h));
}

// As many clusters as can be resident at once (the scheduler's answer for this kernel's resources);
// one cluster per 8 SMs if the query fails.
int bs_cluster_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int clusters = sms > CL_SIZE ? sms / CL_SIZE : 1;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = CL_SIZE; attr.val.clusterDim.y = 1; attr.val.clusterDim.z = 1;
  cfg.gridDim = dim3(CL_SIZE * clusters, 1, 1);
  cfg.blockDim = dim3(CL_THREADS, 1, 1);
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int active = 0;
  if (cudaOccupancyMaxActiveClusters(&active, k_bs_cluster, &cfg) == cudaSuccess && active > 0) clusters = active;
  cudaGetLastError();
  return clusters * CL_SIZE;
}

void launch_bs_cluster(const Sim &S, const DevParams &P, double tau, int gmin, int grid, cudaStream_t st) {
  k_bs_cluster<<<grid, CL_THREADS, 0, st>>>(S, P, tau, gmin);
}

}  // namespace genga
