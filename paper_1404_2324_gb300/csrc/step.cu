// step.cu -- the per-substep kernels between two kicks: Sun drift + Kepler drift (Eqs. Hc, fg),
// the close-encounter search (Eqs. teqn, polydelta) and the grouping of encounter pairs
// (Sect. 3.2 and Appendix), plus the list/bitmap conversions used by the phase entry points.
#include "genga_launch.h"

namespace genga {

// ---------------------------------------------------------------------------------------------
// Drift: x += hcm2 P_pre + hcm1 P_post (the previous substep's second Sun drift, if any, and this
// substep's first), keep (x0, v0), then the Kepler drift for tau. One warp per 32 bodies; every
// warp sums the per-tile momentum partials itself (no extra launch).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(32) k_drift(Sim S, DevParams P, double tau, double hcm1, double hcm2, int substep) {
  const int lane = threadIdx.x;
  const int i = blockIdx.x * 32 + lane;
  const int np = S.npad, nt = S.nt;
  if (i == 0) {
    if (substep == 0) { S.flags[0] = 0; S.flags[3] = 0; }  // the opening kick of this step has consumed the flags
    S.flags[2] = substep;              // for the collision reports of this substep's BS
  }
  double shift[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double a = 0.0, b = 0.0;
    for (int t = lane; t < nt; t += 32) {
      a += S.pfin[t * 3 + c];
      if (hcm2 != 0.0) b += S.pkick[t * 3 + c];
    }
    a = warp_sum(a);
    shift[c] = hcm1 * a;
    if (hcm2 != 0.0) shift[c] = fma(hcm2, warp_sum(b), shift[c]);
  }
  if (!S.alive[i]) return;
  double x = S.x[i] + shift[0], y = S.x[np + i] + shift[1], z = S.x[2 * np + i] + shift[2];
  double vx = S.v[i], vy = S.v[np + i], vz = S.v[2 * np + i];
  S.x0[i] = x; S.x0[np + i] = y; S.x0[2 * np + i] = z;
  S.v0[i] = vx; S.v0[np + i] = vy; S.v0[2 * np + i] = vz;
  int it = 0;
  if (kepler_drift_dev(P.G * P.m0, P.mu2, x, y, z, vx, vy, vz, tau, P.kepler_maxit, &it)) {
    atomicOr(S.status, ST_KEPLER_FALLBACK);
    atomicAdd((unsigned long long *)&S.counters[C_KFALL], 1ULL);
    S.fail[atomicAdd(S.nfail, 1)] = i;  // integrated by BS as a group of its own
  }
  S.x[i] = x; S.x[np + i] = y; S.x[2 * np + i] = z;
  S.v[i] = vx; S.v[np + i] = vy; S.v[2 * np + i] = vz;
}

__global__ void k_kepler_phase(int n, double mu, double dt, int maxit, const int *alive, double *X,
                               double *V, int *fail) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  fail[i] = 0;
  if (!alive[i]) return;
  double x = X[i], y = X[n + i], z = X[2 * n + i], vx = V[i], vy = V[n + i], vz = V[2 * n + i];
  int it = 0;
  if (kepler_drift_dev(mu, 2.0 * mu, x, y, z, vx, vy, vz, dt, maxit, &it)) { fail[i] = 1; return; }
  X[i] = x; X[n + i] = y; X[2 * n + i] = z;
  V[i] = vx; V[n + i] = vy; V[2 * n + i] = vz;
}

// ---------------------------------------------------------------------------------------------
// Encounter search: one CTA per 32 bodies. Its warps gather the candidate pairs (i, j > i) of those
// bodies from the candidate lists (or the bitmap row when a list overflowed) into shared memory,
// clearing the candidate rows for the next kick; then every thread tests one pair with the
// Hermite minimum over the drift, and confirmed pairs go into this substep's encounter bitmap and
// the edge list. One pair per lane: a warp per body would issue the whole FP64 test for one or two
// active lanes, and an FP64 warp instruction costs its sub-partition the same whatever its lanes.
// ---------------------------------------------------------------------------------------------
constexpr int ENC_BODIES = 32;   // bodies per CTA (one word of the row-nonempty bits)
constexpr int ENC_THREADS = 256;
constexpr int ENC_CAP = 1024;    // gathered pairs per CTA; further pairs are tested where found

__device__ __forceinline__ bool encounter_test(const Sim &S, double tau, int i, int j) {
  const int np = S.npad;
  if (!S.alive[i] || !S.alive[j]) return false;
  const double rcij = pmax(S.rc[i], S.rc[j]);
  const double thr = __dmul_rn(rcij, rcij);
  const double dmin = hermite_min_capped(
      __dsub_rn(S.x0[j], S.x0[i]), __dsub_rn(S.x0[np + j], S.x0[np + i]), __dsub_rn(S.x0[2 * np + j], S.x0[2 * np + i]),
      __dsub_rn(S.v0[j], S.v0[i]), __dsub_rn(S.v0[np + j], S.v0[np + i]), __dsub_rn(S.v0[2 * np + j], S.v0[2 * np + i]),
      __dsub_rn(S.x[j], S.x[i]), __dsub_rn(S.x[np + j], S.x[np + i]), __dsub_rn(S.x[2 * np + j], S.x[2 * np + i]),
      __dsub_rn(S.v[j], S.v[i]), __dsub_rn(S.v[np + j], S.v[np + i]), __dsub_rn(S.v[2 * np + j], S.v[2 * np + i]), tau, thr);
  return dmin < thr;
}

// The encounter test of the NBOD bodies of this CTA (NT threads; the gathered pairs in s_i, s_j of CAP).
template <int NT, int NBOD, int CAP>
__device__ void encounter_body(const Sim &S, double tau, unsigned *ebm, int keep, int *s_i, int *s_j, int &s_n,
                               int &s_found) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int np = S.npad, W = S.W;
  const int i0 = blockIdx.x * NBOD;
  if (tid == 0) { s_n = 0; s_found = 0; }
  for (int k = tid; k < NBOD * W; k += NT) {  // this substep's rows start empty
    const int i = i0 + k / W;
    if (i < np) ebm[(size_t)i * W + k % W] = 0u;
  }
  __syncthreads();
  int found = 0;
  auto hit = [&](int i, int j) {
    atomicOr(&ebm[(size_t)i * W + (j >> 5)], 1u << (j & 31));
    const int e = atomicAdd(S.nedges, 1);
    S.edges[2 * e] = i;
    S.edges[2 * e + 1] = j;
    found++;
  };
  auto add = [&](int i, int j) {  // gather, or test at once if the shared list is full
    const int p = atomicAdd(&s_n, 1);
    if (p < CAP) { s_i[p] = i; s_j[p] = j; }
    else if (encounter_test(S, tau, i, j)) hit(i, j);
  };
  for (int b = wid; b < NBOD; b += NT / 32) {
    const int i = i0 + b;
    if (i >= np || !((S.rowany[i >> 5] >> (i & 31)) & 1u)) continue;  // uniform within the warp
    unsigned *crow = S.cbm + (size_t)i * W;
    const int cnt = S.ccnt[i];
    if (cnt <= CCAP) {  // partners from the list
      for (int k = lane; k < cnt; k += 32) {
        const int j = S.clist[i * CCAP + k];
        if (j > i) add(i, j);
      }
      if (!keep) for (int w = lane; w < W; w += 32) crow[w] = 0u;
    } else {  // list overflowed: scan the bitmap row
      for (int w = lane; w < W; w += 32) {
        unsigned bits = crow[w];
        if (!keep) crow[w] = 0u;
        const int lo = w * 32;
        if (lo + 31 <= i) bits = 0u;
        else if (lo <= i) bits &= (i - lo + 1 >= 32) ? 0u : (0xffffffffu << (i - lo + 1));
        while (bits) {
          const int bb = __ffs(bits) - 1;
          bits &= bits - 1;
          add(i, lo + bb);
        }
      }
    }
    if (lane == 0 && !keep) S.ccnt[i] = 0;
  }
  __syncthreads();
  if (tid < NBOD / 32 && i0 + 32 * tid < np && !keep) S.rowany[(i0 >> 5) + tid] = 0u;  // the CTA's rows are clear
  const int n = s_n < CAP ? s_n : CAP;
  for (int p = tid; p < n; p += NT)
    if (encounter_test(S, tau, s_i[p], s_j[p])) hit(s_i[p], s_j[p]);
  if (found) atomicAdd(&s_found, found);
  __syncthreads();
  if (tid == 0 && s_found) atomicAdd((unsigned long long *)&S.counters[C_ENC], (unsigned long long)s_found);
}

__global__ void __launch_bounds__(ENC_THREADS) k_encounter(Sim S, double tau, unsigned *ebm, int keep) {
  __shared__ int s_i[ENC_CAP], s_j[ENC_CAP];
  __shared__ int s_n, s_found;
  encounter_body<ENC_THREADS, ENC_BODIES, ENC_CAP>(S, tau, ebm, keep, s_i, s_j, s_n, s_found);
}

// ---------------------------------------------------------------------------------------------
// Grouping (Appendix): one CTA. LINK[i] = i; every edge hooks the larger root onto the smaller
// with atomicMin; pointer jumping compresses the links; repeat until no edge joins two roots.
// Then the members (bodies in an edge or in the Kepler-fallback list) are placed by root with a
// counting placement, which yields groups ordered by smallest member and members ascending -- the
// same lists as a breadth-first search.
// ---------------------------------------------------------------------------------------------
constexpr int GROUP_THREADS = 1024;
constexpr int GROUP_MAX_ROUNDS = 64;

// Ordered compaction over [0, n) by one CTA of GROUP_THREADS threads: emit(i, k) is called for the
// k-th index (in ascending order) with pred(i) true. Returns the count (uniform across the CTA).
template <class Pred, class Emit>
__device__ int block_compact(int n, Pred pred, Emit emit, int *wtot, int *s_base) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) *s_base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += GROUP_THREADS) {
    const int i = c0 + tid;
    const bool f = i < n && pred(i);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wtot[wid] = __popc(bal);
    __syncthreads();
    if (wid == 0) {
      const int v = wtot[lane];
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      wtot[lane] = incl - v;  // exclusive offsets of the warps
    }
    __syncthreads();
    if (f) emit(i, *s_base + wtot[wid] + __popc(bal & ((1u << lane) - 1u)));
    __syncthreads();
    if (tid == GROUP_THREADS - 1) *s_base += wtot[wid] + __popc(bal);
    __syncthreads();
  }
  return *s_base;
}

// In-place exclusive scan of v[0, n) by one CTA of GROUP_THREADS threads (ordered, exact).
__device__ void block_scan_excl(int *v, int n, int *wtot, int *s_base) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) *s_base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += GROUP_THREADS) {
    const int i = c0 + tid;
    const int x = i < n ? v[i] : 0;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const int w = wtot[lane];
      int winc = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, winc, o);
        if (lane >= o) winc += t;
      }
      wtot[lane] = winc - w;  // exclusive offsets of the warps
    }
    __syncthreads();
    const int base = *s_base;
    if (i < n) v[i] = base + wtot[wid] + incl - x;
    __syncthreads();
    if (tid == GROUP_THREADS - 1) *s_base = base + wtot[wid] + incl;
    __syncthreads();
  }
}

__device__ __forceinline__ int find_root(const int *link, int r) {
  for (int k = 0; k < NMAX + 2; ++k) {
    const int l = link[r];
    if (l == r) break;
    r = l;
  }
  return r;
}

struct GroupShared {
  int link[NMAX], key[NMAX], gcnt[NMAX], gst[NMAX + 1];
  unsigned char part[NMAX];
  int wtot[GROUP_THREADS / 32];
  int s_changed, s_base, s_ng;
};

// The grouping by one CTA of GROUP_THREADS threads. The edge list is read past L1 (the fused
// encounter kernel's other CTAs wrote it in the same launch), or from the shared-memory copy
// (ei[e], ej[e]) when the caller made one.
__device__ void group_body(const Sim &S, int gbig, GroupShared &sm, const int *ei = nullptr, const int *ej = nullptr) {
  int *link = sm.link, *key = sm.key, *gcnt = sm.gcnt, *gst = sm.gst, *wtot = sm.wtot;
  unsigned char *part = sm.part;
  int &s_changed = sm.s_changed, &s_base = sm.s_base, &s_ng = sm.s_ng;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int np = S.npad;
  const int ne = __ldcg(S.nedges), nf = __ldcg(S.nfail);
  auto eu = [&](int e) { return ei ? ei[e] : __ldcg(S.edges + 2 * e); };
  auto ev = [&](int e) { return ej ? ej[e] : __ldcg(S.edges + 2 * e + 1); };
  for (int i = tid; i < np; i += GROUP_THREADS) { link[i] = i; part[i] = 0; }
  __syncthreads();
  for (int e = tid; e < ne; e += GROUP_THREADS) { part[eu(e)] = 1; part[ev(e)] = 1; }
  for (int f = tid; f < nf; f += GROUP_THREADS) part[__ldcg(S.fail + f)] = 1;
  int round = 0;
  for (; round < GROUP_MAX_ROUNDS; ++round) {
    if (tid == 0) s_changed = 0;
    __syncthreads();
    for (int e = tid; e < ne; e += GROUP_THREADS) {
      const int ru = find_root(link, eu(e)), rv = find_root(link, ev(e));
      if (ru != rv) {
        atomicMin(&link[ru > rv ? ru : rv], ru < rv ? ru : rv);
        s_changed = 1;
      }
    }
    __syncthreads();
    for (int i = tid; i < np; i += GROUP_THREADS) link[i] = find_root(link, link[i]);
    __syncthreads();
    if (!s_changed) break;
  }
  if (round >= GROUP_MAX_ROUNDS && tid == 0) atomicOr(S.status, ST_UNION_ROUNDS);
  // Groups by root (the smallest member: links only ever point to smaller indices), members
  // ascending. The participants in ascending order; members counted per root; the roots among
  // the participants, ascending, are the groups in order: each group's size goes to gst and an
  // ordered scan makes it the group's first position; one warp then walks the participants in
  // order and puts each at its root's next free position (lanes with the same root take
  // consecutive ones). Only participants are touched after the union rounds.
  const int cnt = block_compact(np, [&](int i) { return part[i] != 0; }, [&](int i, int pos) { key[pos] = i; },
                                wtot, &s_base);
  for (int k = tid; k < cnt; k += GROUP_THREADS) gcnt[key[k]] = 0;
  __syncthreads();
  for (int k = tid; k < cnt; k += GROUP_THREADS) atomicAdd(&gcnt[link[key[k]]], 1);
  __syncthreads();
  s_ng = block_compact(cnt, [&](int k) { const int i = key[k]; return link[i] == i; },
                       [&](int k, int g) { const int r = key[k]; gst[g] = gcnt[r]; gcnt[r] = g; }, wtot, &s_base);
  __syncthreads();  // every thread has read the count in s_base before the scan resets it
  block_scan_excl(gst, s_ng, wtot, &s_base);  // gst[g]: the first position of group g
  for (int k = tid; k < cnt; k += GROUP_THREADS) {
    const int i = key[k];
    if (link[i] == i) gcnt[i] = gst[gcnt[i]];  // root i: its group's first position
  }
  for (int g = tid; g < s_ng; g += GROUP_THREADS) S.gstart[g] = gst[g];
  if (tid == 0) gst[s_ng] = cnt;
  __syncthreads();
  if (wid == 0) {
    for (int c0 = 0; c0 < cnt; c0 += 32) {
      const int k = c0 + lane;
      const bool ok = k < cnt;
      const int i = ok ? key[k] : 0, r = ok ? link[i] : -1 - lane;  // idle lanes: roots of their own
      const unsigned m = __match_any_sync(0xffffffffu, r);
      const int pos = ok ? gcnt[r] + __popc(m & ((1u << lane) - 1u)) : 0;
      __syncwarp();
      if (ok) {
        S.gmem[pos] = i;
        if (lane == __ffs(m) - 1) gcnt[r] += __popc(m);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (tid == 0) {
    S.gstart[s_ng] = cnt;
    *S.ngroups = s_ng;
    if (s_ng) atomicAdd((unsigned long long *)&S.counters[C_GROUPS], (unsigned long long)s_ng);
    *S.nedges = 0;
    *S.nfail = 0;
  }
  if (S.big) {  // the groups of gbig or more members, in group order
    __syncthreads();
    const int nb = block_compact(s_ng, [&](int g) { return gst[g + 1] - gst[g] >= gbig; },
                                 [&](int g, int pos) { S.big[pos] = g; }, wtot, &s_base);
    if (tid == 0) *S.nbig = nb;
  }
}

__global__ void __launch_bounds__(GROUP_THREADS) k_group(Sim S, int gbig) {
  __shared__ GroupShared sm;
  group_body(S, gbig, sm);
}

// The encounter test and the grouping in one launch: CTAs of GROUP_THREADS threads test the pairs
// of EG_BODIES bodies each; the last CTA to finish (a device-wide counter, fenced) groups the edges
// of all of them. Saves the launch between the two and the grouping kernel's ramp-up.
constexpr int EG_BODIES = 32;
constexpr int EG_CAP = 1024;
__global__ void __launch_bounds__(GROUP_THREADS) k_encounter_group(Sim S, double tau, unsigned *ebm, int keep, int gbig) {
  __shared__ int s_i[EG_CAP], s_j[EG_CAP];
  __shared__ int s_n, s_found, s_last;
  __shared__ GroupShared sm;
  encounter_body<GROUP_THREADS, EG_BODIES, EG_CAP>(S, tau, ebm, keep, s_i, s_j, s_n, s_found);
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's edges before its count
    s_last = atomicAdd(&S.flags[1], 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;  // uniform
  __threadfence();
  if (threadIdx.x == 0) S.flags[1] = 0;  // the counter of the next launch
  // the edges into shared memory once (the encounter's pair buffers are free now): the union
  // rounds then read them there instead of from L2 every round
  const int ne = __ldcg(S.nedges);
  if (ne <= EG_CAP) {
    for (int e = threadIdx.x; e < ne; e += blockDim.x) { s_i[e] = __ldcg(S.edges + 2 * e); s_j[e] = __ldcg(S.edges + 2 * e + 1); }
    __syncthreads();
    group_body(S, gbig, sm, s_i, s_j);
  } else {
    group_body(S, gbig, sm);
  }
}

// ---------------------------------------------------------------------------------------------
// List <-> bitmap helpers for the phase entry points and genga_encounters
// ---------------------------------------------------------------------------------------------
__global__ void k_pairs_to_bitmap(Sim S, const int *pairs, int npairs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npairs) return;
  const int i = pairs[2 * k], j = pairs[2 * k + 1];
  atomicOr(&S.cbm[(size_t)i * S.W + (j >> 5)], 1u << (j & 31));
  atomicOr(&S.cbm[(size_t)j * S.W + (i >> 5)], 1u << (i & 31));
  atomicOr(&S.rowany[i >> 5], 1u << (i & 31));
  atomicOr(&S.rowany[j >> 5], 1u << (j & 31));
  const int ki = atomicAdd(&S.ccnt[i], 1), kj = atomicAdd(&S.ccnt[j], 1);
  if (ki < CCAP) S.clist[i * CCAP + ki] = j;
  if (kj < CCAP) S.clist[j * CCAP + kj] = i;
}

// Pairs (i < j) of a bitmap, ascending, into out[2*cap]; *count receives the total.
__global__ void __launch_bounds__(1024) k_bitmap_pairs(const unsigned *bm, int npad, int W, int *out, int cap, int *count) {
  __shared__ int wtot[32];
  __shared__ int s_base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_base = 0;
  __syncthreads();
  for (int r0 = 0; r0 < npad; r0 += 1024) {
    const int i = r0 + tid;
    int c = 0;
    if (i < npad) {
      for (int w = 0; w < W; ++w) {
        unsigned bits = bm[(size_t)i * W + w];
        const int lo = w * 32;
        if (lo + 31 <= i) bits = 0u;
        else if (lo <= i) bits &= (i - lo + 1 >= 32) ? 0u : (0xffffffffu << (i - lo + 1));
        c += __popc(bits);
      }
    }
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int v = wtot[lane], in2 = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, in2, o);
        if (lane >= o) in2 += t;
      }
      wtot[lane] = in2 - v;
    }
    __syncthreads();
    int pos = s_base + wtot[wid] + incl - c;
    if (i < npad && c) {
      for (int w = 0; w < W; ++w) {
        unsigned bits = bm[(size_t)i * W + w];
        const int lo = w * 32;
        if (lo + 31 <= i) bits = 0u;
        else if (lo <= i) bits &= (i - lo + 1 >= 32) ? 0u : (0xffffffffu << (i - lo + 1));
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1;
          if (pos < cap) { out[2 * pos] = i; out[2 * pos + 1] = lo + b; }
          pos++;
        }
      }
    }
    __syncthreads();
    if (tid == 1023) s_base = pos;  // end of the last thread's run = total so far
    __syncthreads();
  }
  if (tid == 0) *count = s_base;
}

__global__ void k_single_to_fail(Sim S, const int *single) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  if (single[i]) S.fail[atomicAdd(S.nfail, 1)] = i;
}

__global__ void k_copy_edges(Sim S, const int *pairs, int npairs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) *S.nedges = npairs;
  if (k >= npairs) return;
  S.edges[2 * k] = pairs[2 * k];
  S.edges[2 * k + 1] = pairs[2 * k + 1];
}

// ---------------------------------------------------------------------------------------------
void launch_drift(const Sim &S, const DevParams &P, double tau, double hcm1, double hcm2,
                  int substep, cudaStream_t st) {
  k_drift<<<S.npad / 32, 32, 0, st>>>(S, P, tau, hcm1, hcm2, substep);
}
void launch_encounter(const Sim &S, double tau, unsigned *ebm, cudaStream_t st, bool keep) {
  k_encounter<<<(S.npad + ENC_BODIES - 1) / ENC_BODIES, ENC_THREADS, 0, st>>>(S, tau, ebm, keep ? 1 : 0);
}
void launch_group(const Sim &S, cudaStream_t st, int gbig) { k_group<<<1, GROUP_THREADS, 0, st>>>(S, gbig); }
void launch_encounter_group(const Sim &S, double tau, unsigned *ebm, cudaStream_t st, bool keep, int gbig) {
  k_encounter_group<<<(S.npad + EG_BODIES - 1) / EG_BODIES, GROUP_THREADS, 0, st>>>(S, tau, ebm, keep ? 1 : 0, gbig);
}
void launch_kepler_phase(int n, double mu, double dt, int maxit, const int *alive, double *x, double *v,
                         int *fail, cudaStream_t st) {
  k_kepler_phase<<<(n + 31) / 32, 32, 0, st>>>(n, mu, dt, maxit, alive, x, v, fail);
}
void launch_pairs_to_bitmap(const Sim &S, const int *pairs, int npairs, cudaStream_t st) {
  if (npairs > 0) k_pairs_to_bitmap<<<(npairs + 127) / 128, 128, 0, st>>>(S, pairs, npairs);
}
void launch_bitmap_pairs(const unsigned *bm, int npad, int W, int *out, int cap, int *count, cudaStream_t st) {
  k_bitmap_pairs<<<1, 1024, 0, st>>>(bm, npad, W, out, cap, count);
}
void launch_single_to_fail(const Sim &S, const int *single, cudaStream_t st) {
  k_single_to_fail<<<(S.n + 127) / 128, 128, 0, st>>>(S, single);
}
void launch_copy_edges(const Sim &S, const int *pairs, int npairs, cudaStream_t st) {
  k_copy_edges<<<(npairs + 128) / 128, 128, 0, st>>>(S, pairs, npairs);
}

}  // namespace genga
