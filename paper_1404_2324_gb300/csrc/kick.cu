// kick.cu -- critical radii (Eq. rcrit), the K-weighted pairwise kick with the prechecker
// (Eq. Hb, Sect. 2.2 and 3.2 "Kick"), and its per-body finalisation (KickA/KickB reuse).
//
// The pair kernel evaluates every unordered pair once (Newton's third law) on 32x32 body tiles:
// each lane holds one body i of tile I, the 32 bodies of tile J rotate through the lanes by warp
// shuffles, and the j-side accumulators rotate with them. A work item is half of a tile pair
// (16 ring steps), which balances ~6.7 items per sub-partition at N = 2048. Partial sums go to a
// per-(tile, partner tile, half) buffer that the finalisation sums in a fixed order, so results
// are bitwise reproducible. Per unordered pair the kernel issues 20 FP64 instructions.
#include "genga_launch.h"

namespace genga {

// ---------------------------------------------------------------------------------------------
// Critical radii, precheck thresholds and the kick-reuse test (once per full step)
// ---------------------------------------------------------------------------------------------
__global__ void k_rcrit(Sim S, DevParams P, double tau_abs, int check_reuse) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (check_reuse && i == 0) atomicAdd((unsigned long long *)&S.counters[C_STEPS], 1ULL);
  if (i >= S.npad) return;
  const int np = S.npad;
  if (!S.alive[i]) {
    S.rc[i] = 0.0; S.A[i] = 0.0; S.T[i] = 0ULL; S.rcsq[i] = 0ULL;
    return;
  }
  double x = S.x[i], y = S.x[np + i], z = S.x[2 * np + i];
  double vx = S.v[i], vy = S.v[np + i], vz = S.v[2 * np + i];
  double r2 = fma(z, z, fma(y, y, x * x));
  double ir = rsqrt_refined(r2);
  double v2 = fma(vz, vz, fma(vy, vy, vx * vx));
  double inva = fma(2.0, ir, -v2 * P.inv_mu);  // 1/a = 2/r - v^2/(G m0)
  double asemi = is_neg_or_zero(inva) ? r2 * ir : rcp_refined(inva);
  double rh = asemi * S.hill[i];               // Hill radius a (m/(3 m0))^(1/3)
  double vabs = (dbits(v2) == 0ULL) ? 0.0 : v2 * rsqrt_refined(v2);
  double rc = pmax(P.n1 * rh, (P.n2 * tau_abs) * vabs);
  if (check_reuse) {
    // reusing the last kick for non-candidate pairs is exact while rc_new <= pc * rc_old
    double lim = P.pc * S.rc[i];
    if (dbits(rc) > dbits(lim)) {
      S.flags[0] = 1;
      atomicOr(S.status, ST_REUSE_FULLKICK);
      atomicAdd((unsigned long long *)&S.counters[C_FULLKICK], 1ULL);
    }
  }
  S.rc[i] = rc;
  double t = __dmul_rn(P.pc, rc);
  S.T[i] = dbits(__dmul_rn(t, t));
  S.rcsq[i] = dbits(__dmul_rn(rc, rc));
  S.A[i] = (dbits(rc) == 0ULL) ? 0.0 : rcp_refined(0.9 * rc);
}

// ---------------------------------------------------------------------------------------------
// Pair kernel. FULL: all pairs with inline changeover weights (used only when the critical
// radii grew too much for reuse); otherwise far pairs only, candidates recorded in the bitmap.
// ---------------------------------------------------------------------------------------------
template <bool FULL, bool PRECISE>
__global__ void __launch_bounds__(128) k_kick(Sim S, DevParams P, int force) {
  if (FULL && !force && S.flags[0] == 0) return;
  // a full opening kick after a new state also records the precheck candidates (flag 3)
  const bool record = FULL && !force && S.flags[3] != 0;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int np = S.npad, nt = S.nt, W = S.W;
  const double *__restrict__ X = S.x;
  if ((!FULL || force) && warp < nt) {  // per-tile momentum before the closing kick (second Sun drift)
    int i = warp * 32 + lane;
    double mi = S.m[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double p = warp_sum(mi * S.v[c * np + i]);
      if (lane == 0) S.pkick[warp * 3 + c] = p;
    }
  }
  if (warp >= S.nwarps) return;
  const long it0 = (long)warp * S.nitems / S.nwarps, it1 = (long)(warp + 1) * S.nitems / S.nwarps;
  int curI = -1;
  double xi = 0, yi = 0, zi = 0, gmi = 0, Ai = 0;
  u64 Ti = 0, Qi = 0;
  for (long it = it0; it < it1; ++it) {
    const int code = S.items[it];
    const int I = code & 1023, J = (code >> 10) & 1023, h = code >> 20;
    const int i = I * 32 + lane;
    if (I != curI) {
      curI = I;
      xi = X[i]; yi = X[np + i]; zi = X[2 * np + i];
      gmi = S.gm[i]; Ti = S.T[i];
      if (FULL) { Qi = S.rcsq[i]; Ai = S.A[i]; }
    }
    const bool diag = (I == J);
    const int jl0 = diag ? lane : ((lane + 16 * h) & 31);
    const int j0 = J * 32 + jl0;
    double xj = X[j0], yj = X[np + j0], zj = X[2 * np + j0], gmj = S.gm[j0];
    u64 Tj = S.T[j0], Qj = 0;
    double Aj = 0;
    if (FULL) { Qj = S.rcsq[j0]; Aj = S.A[j0]; }
    double aix = 0, aiy = 0, aiz = 0, ajx = 0, ajy = 0, ajz = 0;
    const int src = (lane + 1) & 31;
#pragma unroll 4
    for (int s = 0; s < 16; ++s) {
      if (diag) {  // diagonal tile: rotate first, pair lane with lane + s + 1
        xj = __shfl_sync(0xffffffffu, xj, src); yj = __shfl_sync(0xffffffffu, yj, src);
        zj = __shfl_sync(0xffffffffu, zj, src); gmj = __shfl_sync(0xffffffffu, gmj, src);
        Tj = __shfl_sync(0xffffffffu, Tj, src);
        ajx = __shfl_sync(0xffffffffu, ajx, src); ajy = __shfl_sync(0xffffffffu, ajy, src);
        ajz = __shfl_sync(0xffffffffu, ajz, src);
        if (FULL) { Qj = __shfl_sync(0xffffffffu, Qj, src); Aj = __shfl_sync(0xffffffffu, Aj, src); }
      }
      const int jl = diag ? ((lane + s + 1) & 31) : ((lane + 16 * h + s) & 31);
      const bool act = !diag || s < 15 || lane < 16;
      const double dx = xj - xi, dy = yj - yi, dz = zj - zi;
      const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
      double w3;
      if (PRECISE) w3 = 1.0 / (r2 * sqrt(r2));
      else w3 = rcube_refined(r2);
      double gj = act ? gmj : 0.0, gi = act ? gmi : 0.0;
      const u64 rb = dbits(r2);
      if (FULL) {
        if (rb < umax64(Qi, Qj)) {  // inside the changeover zone: weight K (rare)
          double r = r2 * rsqrt_refined(r2), wB, wA;
          changeover_w(r, pmin(Ai, Aj), P.kmode, wB, wA);
          gj *= wB; gi *= wB;
        }
      }
      if ((!FULL || record) && act && rb < umax64(Ti, Tj)) {  // precheck candidate
        if (!FULL) { gj = 0.0; gi = 0.0; }  // handled by the near pass
        const int j = J * 32 + jl;
        atomicOr(&S.cbm[(size_t)i * W + (j >> 5)], 1u << (j & 31));
        atomicOr(&S.cbm[(size_t)j * W + (i >> 5)], 1u << (i & 31));
        atomicOr(&S.rowany[i >> 5], 1u << (i & 31));
        atomicOr(&S.rowany[j >> 5], 1u << (j & 31));
        const int ki = atomicAdd(&S.ccnt[i], 1), kj = atomicAdd(&S.ccnt[j], 1);
        if (ki < CCAP) S.clist[i * CCAP + ki] = j;
        if (kj < CCAP) S.clist[j * CCAP + kj] = i;
        atomicAdd((unsigned long long *)&S.counters[C_CAND], 1ULL);
      }
      const double fi = gj * w3, fj = gi * w3;
      aix = fma(fi, dx, aix); aiy = fma(fi, dy, aiy); aiz = fma(fi, dz, aiz);
      ajx = fma(-fj, dx, ajx); ajy = fma(-fj, dy, ajy); ajz = fma(-fj, dz, ajz);
      if (!diag && s < 15) {
        xj = __shfl_sync(0xffffffffu, xj, src); yj = __shfl_sync(0xffffffffu, yj, src);
        zj = __shfl_sync(0xffffffffu, zj, src); gmj = __shfl_sync(0xffffffffu, gmj, src);
        Tj = __shfl_sync(0xffffffffu, Tj, src);
        ajx = __shfl_sync(0xffffffffu, ajx, src); ajy = __shfl_sync(0xffffffffu, ajy, src);
        ajz = __shfl_sync(0xffffffffu, ajz, src);
        if (FULL) { Qj = __shfl_sync(0xffffffffu, Qj, src); Aj = __shfl_sync(0xffffffffu, Aj, src); }
      }
    }
    // return the j accumulators to the lane that owns body J*32 + lane
    const int home = diag ? ((lane + 16) & 31) : ((lane - 16 * h - 15) & 31);
    ajx = __shfl_sync(0xffffffffu, ajx, home);
    ajy = __shfl_sync(0xffffffffu, ajy, home);
    ajz = __shfl_sync(0xffffffffu, ajz, home);
    double *pi = S.part + ((size_t)(I * nt + J) * 2 + h) * 96 + lane;
    if (diag) {
      pi[0] = aix + ajx; pi[32] = aiy + ajy; pi[64] = aiz + ajz;
      pi[96] = 0.0; pi[128] = 0.0; pi[160] = 0.0;  // half 1 of a diagonal tile is empty
    } else {
      pi[0] = aix; pi[32] = aiy; pi[64] = aiz;
      double *pj = S.part + ((size_t)(J * nt + I) * 2 + h) * 96 + lane;
      pj[0] = ajx; pj[32] = ajy; pj[64] = ajz;
    }
  }
}

// Component c of the near-pair acceleration of body i: the precheck candidates recorded in row i
// of the bitmap, with the changeover weight of the current critical radii (IEEE sqrt/division).
__device__ double near_accel(const Sim &S, const DevParams &P, int i, int c) {
  const int np = S.npad;
  const unsigned *row = S.cbm + (size_t)i * S.W;
  const double xi = S.x[i], yi = S.x[np + i], zi = S.x[2 * np + i];
  const u64 Qi = S.rcsq[i];
  const double Ai = S.A[i];
  double acc = 0.0;
  for (int w = 0; w < S.W; ++w) {
    unsigned bits = row[w];
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      const int j = w * 32 + b;
      const double dx = S.x[j] - xi, dy = S.x[np + j] - yi, dz = S.x[2 * np + j] - zi;
      const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
      const double r = sqrt(r2);
      double wB = 1.0, wA;
      if (dbits(r2) < umax64(Qi, S.rcsq[j])) changeover_w(r, pmin(Ai, S.A[j]), P.kmode, wB, wA);
      const double f = S.gm[j] * wB / (r2 * r);
      acc = fma(f, c == 0 ? dx : (c == 1 ? dy : dz), acc);
    }
  }
  return acc;
}

// Component c of the near-pair pull of partner j on body i with the current critical radii
// (refined inverse square root; the changeover weight as in the kick).
__device__ __forceinline__ double near_term(const Sim &S, const DevParams &P, int i, int j, int c) {
  const int np = S.npad;
  const double dx = S.x[j] - S.x[i], dy = S.x[np + j] - S.x[np + i], dz = S.x[2 * np + j] - S.x[2 * np + i];
  const double r2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
  const double yr = rsqrt_refined(r2);
  double wB = 1.0, wA;
  if (dbits(r2) < umax64(S.rcsq[i], S.rcsq[j])) changeover_w(r2 * yr, pmin(S.A[i], S.A[j]), P.kmode, wB, wA);
  return S.gm[j] * wB * (yr * yr * yr) * (c == 0 ? dx : (c == 1 ? dy : dz));
}

// ---------------------------------------------------------------------------------------------
// Finalisation, one CTA per (body tile, component):
//   CLOSE: a = sum of the pair partials (far field, stored for reuse) + near pairs;
//          v += h1 a (+ h2 a for the next substep's opening kick). The second Sun drift of the
//          substep (which the kick does not see: it shifts every body alike) is applied by the
//          next drift kernel, or by k_hc after the last substep, from the momentum the kick
//          kernel recorded before the velocities changed.
//   OPEN : first kick of a full step with the new critical radii: a = stored far field + near
//          pairs recomputed (KickA; KickB when there are none), or the full recompute's partials.
//   INIT : the very first kick: store the far field (and a = far + near into aout if given).
// The near pairs of the tile's 32 bodies are gathered from the candidate lists (one coalesced pass
// into shared memory), put in ascending partner order per body (each entry goes to its rank),
// evaluated one per thread across the CTA and summed per body in partner order.
// Also writes the per-tile momentum of the new velocities for the next Sun drift.
// ---------------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(128) k_fin(Sim S, DevParams P, double h1, double h2, double *aout) {
  constexpr bool ALL = MODE == FIN_CLOSE_ALL;  // the pair kernel weighed every pair: no near pass
  const int B = blockIdx.x, c = blockIdx.y, wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int np = S.npad, nt = S.nt, i = B * 32 + lane;
  __shared__ double red[4][32];
  __shared__ int ent[32 * CCAP], raw[32 * CCAP];
  __shared__ double contrib[32 * CCAP];
  __shared__ int off[33], s_cnt[32];
  const bool use_part = (MODE != FIN_OPEN) || (S.flags[0] != 0);
  const bool full_open = (MODE == FIN_OPEN) && (S.flags[0] != 0);
  // the loads of the final update first (warp 0), so that their latency passes under the sums
  double a_far = 0.0, v_old = 0.0, m_i = 0.0;
  bool alive = false;
  if (wi == 0) {
    if (!use_part) a_far = S.afar[c * np + i];
    if (MODE != FIN_INIT) { v_old = S.v[c * np + i]; m_i = S.m[i]; alive = S.alive[i] != 0; }
  }
  // this tile's candidate partners: counts and offsets (warp 0), then the lists (all threads)
  bool overflow = false;
  if (wi == 0) {
    const bool any = !ALL && !full_open && ((S.rowany[i >> 5] >> (i & 31)) & 1u);
    int cnt = any ? S.ccnt[i] : 0;
    overflow = cnt > CCAP;
    if (overflow) cnt = 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    off[lane + 1] = incl;
    s_cnt[lane] = cnt;
    if (lane == 0) off[0] = 0;
  }
  if (use_part) {  // far-field partial sums: each warp a quarter of the slots, two chains of alternate slots
    const int nslot = 2 * nt, s0 = wi * nslot / 4, s1 = (wi + 1) * nslot / 4;
    const double *base = S.part + (size_t)B * nt * 2 * 96 + c * 32 + lane;
    double acc0 = 0.0, acc1 = 0.0;
    int s = s0;
    for (; s + 1 < s1; s += 2) { acc0 += base[(size_t)s * 96]; acc1 += base[(size_t)(s + 1) * 96]; }
    if (s < s1) acc0 += base[(size_t)s * 96];
    red[wi][lane] = acc0 + acc1;
  }
  __syncthreads();
  const int M = off[32];
  for (int e = threadIdx.x; e < 32 * CCAP; e += 128) {
    const int b = e / CCAP, k = e % CCAP;
    if (k < s_cnt[b]) raw[off[b] + k] = S.clist[(B * 32 + b) * CCAP + k];
  }
  __syncthreads();
  auto owner = [&](int k) {  // the last body whose offset is <= k
    int b = 0;
    for (int s = 16; s > 0; s >>= 1)
      if (b + s <= 32 && off[b + s] <= k) b += s;
    return b;
  };
  for (int k = threadIdx.x; k < M; k += 128) {  // ascending partner order: each entry to its rank
    const int b = owner(k), o = off[b], n = off[b + 1] - o;
    const int j = raw[k];
    int r = 0;
    for (int q = 0; q < n; ++q) r += raw[o + q] < j;
    ent[o + r] = j;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < M; k += 128) contrib[k] = near_term(S, P, B * 32 + owner(k), ent[k], c);
  __syncthreads();
  if (wi != 0) return;
  double a = use_part ? (red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane]) : a_far;
  if (MODE != FIN_OPEN && !ALL) S.afar[c * np + i] = a;
  for (int k = off[lane]; k < off[lane + 1]; ++k) a += contrib[k];
  if (overflow) a += near_accel(S, P, i, c);
  if (aout) aout[c * np + i] = a;
  if (MODE == FIN_INIT) return;
  double v = v_old;
  if (alive) {
    v = fma(h1, a, v);
    if (h2 != 0.0) v = fma(h2, a, v);
    S.v[c * np + i] = v;
  }
  const double pm = warp_sum(m_i * v);
  if (lane == 0) S.pfin[B * 3 + c] = pm;
}

// ---------------------------------------------------------------------------------------------
int kick_grid(const Sim &S) {
  int warps = S.nwarps > S.nt ? S.nwarps : S.nt;
  return (warps * 32 + 127) / 128;
}

void launch_rcrit(const Sim &S, const DevParams &P, double tau_abs, int check_reuse, cudaStream_t st) {
  k_rcrit<<<(S.npad + 127) / 128, 128, 0, st>>>(S, P, tau_abs, check_reuse);
}

void launch_kick(const Sim &S, const DevParams &P, bool full, bool precise, cudaStream_t st, bool force) {
  const int grid = kick_grid(S);
  const int f = force ? 1 : 0;
  if (full) {
    if (precise) k_kick<true, true><<<grid, 128, 0, st>>>(S, P, f);
    else k_kick<true, false><<<grid, 128, 0, st>>>(S, P, f);
  } else {
    if (precise) k_kick<false, true><<<grid, 128, 0, st>>>(S, P, 0);
    else k_kick<false, false><<<grid, 128, 0, st>>>(S, P, 0);
  }
}

void launch_fin(const Sim &S, const DevParams &P, FinMode mode, double h1, double h2, double *aout,
                cudaStream_t st) {
  dim3 grid(S.nt, 3);
  if (mode == FIN_CLOSE) k_fin<FIN_CLOSE><<<grid, 128, 0, st>>>(S, P, h1, h2, aout);
  else if (mode == FIN_CLOSE_ALL) k_fin<FIN_CLOSE_ALL><<<grid, 128, 0, st>>>(S, P, h1, h2, aout);
  else if (mode == FIN_OPEN) k_fin<FIN_OPEN><<<grid, 128, 0, st>>>(S, P, h1, h2, aout);
  else k_fin<FIN_INIT><<<grid, 128, 0, st>>>(S, P, h1, h2, aout);
}

// Second Sun drift after the last substep: x += hcm * P, P the momentum before the closing kick.
__global__ void k_hc(Sim S, double hcm) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double p[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double a = 0.0;
    for (int t = lane; t < S.nt; t += 32) a += S.pkick[t * 3 + c];
    p[c] = warp_sum(a);
  }
  if (i >= S.npad || !S.alive[i]) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) S.x[c * S.npad + i] = fma(hcm, p[c], S.x[c * S.npad + i]);
}

void launch_hc(const Sim &S, double hcm, cudaStream_t st) {
  k_hc<<<(S.npad + 63) / 64, 64, 0, st>>>(S, hcm);
}

}  // namespace genga
