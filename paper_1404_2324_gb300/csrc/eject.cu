// eject.cu -- ejections (Sect. 3.2, Ejections) and the multi-simulation stop (Sect. 3.4, the Remove
// and Stop kernel), at the end of a step on the heliocentric positions.
//
// A live body farther than rcut from its central mass, or closer than rcut_sun, is removed: it
// becomes a ghost as after a merger (zero mass, parked far out) and its heliocentric position and
// velocity are recorded. The energy it takes away is booked into U (U += E before - E after), the
// change written out term by term for the removed set X:
//   E_after - E_before = - sum_{k in X} (m_k |v_k|^2 / 2 - G m0 m_k / |x_k|)
//                        + sum_{k in X; j live, j not in X or j > k} G m_k m_j / |x_j - x_k|
//                        + (|P - P_X|^2 - |P|^2) / (2 m0),
// with P the momentum of the live bodies (barycentric velocities) and P_X that of X. The stored
// far field of the closing kick still holds the removed bodies' pull, so the next opening kick
// recomputes every pair (the flag that the reuse test raises). In the batched mode a system left
// with fewer than nmin live bodies is stopped: all its bodies are removed the same way (recorded
// only if ejected). The paper compacts each system's memory and recomputes the offsets on the
// CPU; here the ghosts stay in place and every kernel skips them.
#include "genga_launch.h"

namespace genga {

// |x|^2 rounded as (x x + y y) + z z, products and sums rounded separately
__device__ __forceinline__ double r2_plain(double x, double y, double z) {
  return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}
__device__ __forceinline__ bool ejected(const DevParams &P, double r2) {
  return (P.rcut2 > 0.0 && r2 > P.rcut2) || (P.rcut_sun2 > 0.0 && r2 < P.rcut_sun2);
}

// body i becomes a ghost, as a merger's partner does
__device__ void make_ghost(const Sim &S, int i) {
  const int np = S.npad;
  S.alive[i] = 0;
  S.m[i] = 0.0; S.gm[i] = 0.0; S.R[i] = 0.0; S.hill[i] = 0.0;
  S.T[i] = 0ULL; S.rcsq[i] = 0ULL; S.rc[i] = 0.0; S.A[i] = 0.0;
  S.x[i] = PARK + 1.0e4 * i; S.x[np + i] = 0.0; S.x[2 * np + i] = 0.0;
  for (int c = 0; c < 3; ++c) S.v[c * np + i] = 0.0;
}

// record of body i (internal index) at the end of step `step`: heliocentric x and v = v_b + P/m0
__device__ void write_record(const Sim &S, int slot, int i, double step, double px, double py, double pz,
                             double inv_m0) {
  if (slot >= EJ_CAP) { atomicOr(S.status, ST_EJECT_OVERFLOW); return; }
  const int np = S.npad;
  double *r = S.ejrec + 8 * (size_t)slot;
  r[0] = (double)i;
  r[1] = step;
  for (int c = 0; c < 3; ++c) r[2 + c] = S.x[c * np + i];
  r[5] = fma(px, inv_m0, S.v[i]);
  r[6] = fma(py, inv_m0, S.v[np + i]);
  r[7] = fma(pz, inv_m0, S.v[2 * np + i]);
}

// ---------------------------------------------------------------------------------------------
// Single system (N <= 2048, the massive bodies of the main and test-particle modes): one block.
constexpr int EJ_THREADS = 1024;
static_assert(NMAX <= 64 * 32, "the removal bitmap of k_eject covers NMAX bodies");

__global__ void __launch_bounds__(EJ_THREADS) k_eject(Sim S, DevParams P) {
  __shared__ int s_n, s_base;
  __shared__ int s_idx[EJ_STEP], s_ord[EJ_STEP];
  __shared__ unsigned s_out[64];  // removal bitmap over N <= 2048 bodies
  __shared__ double s_red[EJ_THREADS / 32][8];
  __shared__ double s_P[3];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int np = S.npad, n = S.n;
  if (tid == 0) s_n = 0;
  if (tid < 64) s_out[tid] = 0u;
  __syncthreads();
  for (int i = tid; i < n; i += EJ_THREADS) {
    if (!S.alive[i] || !ejected(P, r2_plain(S.x[i], S.x[np + i], S.x[2 * np + i]))) continue;
    const int k = atomicAdd(&s_n, 1);
    if (k < EJ_STEP) {
      s_idx[k] = i;
      atomicOr(&s_out[i >> 5], 1u << (i & 31));
    }
  }
  __syncthreads();
  const int ne = s_n < EJ_STEP ? s_n : EJ_STEP;
  if (ne == 0) return;  // uniform
  if (tid == 0 && s_n > EJ_STEP) atomicOr(S.status, ST_EJECT_OVERFLOW);  // the rest go next step
  for (int t = tid; t < ne; t += EJ_THREADS) {  // ascending index: the records' order
    int r = 0;
    for (int q = 0; q < ne; ++q) r += s_idx[q] < s_idx[t];
    s_ord[r] = s_idx[t];
  }
  auto removed = [&](int j) { return ((s_out[j >> 5] >> (j & 31)) & 1u) != 0u; };
  // P, P_X and the removed bodies' own terms
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = tid; i < n; i += EJ_THREADS) {
    if (!S.alive[i]) continue;
    const double mi = S.m[i], vx = S.v[i], vy = S.v[np + i], vz = S.v[2 * np + i];
    acc[0] = fma(mi, vx, acc[0]); acc[1] = fma(mi, vy, acc[1]); acc[2] = fma(mi, vz, acc[2]);
    if (removed(i)) {
      acc[3] = fma(mi, vx, acc[3]); acc[4] = fma(mi, vy, acc[4]); acc[5] = fma(mi, vz, acc[5]);
      const double r = sqrt(r2_plain(S.x[i], S.x[np + i], S.x[2 * np + i]));
      acc[6] += 0.5 * mi * r2_plain(vx, vy, vz) - P.G * P.m0 * mi / r;
    }
  }
  __syncthreads();  // s_ord complete
  // pairs of a removed body with every live body (two removed bodies counted once)
  for (int q = 0; q < ne; ++q) {
    const int k = s_ord[q];
    const double xk = S.x[k], yk = S.x[np + k], zk = S.x[2 * np + k], gmk = P.G * S.m[k];
    for (int j = tid; j < n; j += EJ_THREADS) {
      if (j == k || !S.alive[j] || (removed(j) && j < k)) continue;
      const double dx = S.x[j] - xk, dy = S.x[np + j] - yk, dz = S.x[2 * np + j] - zk;
      acc[7] += gmk * S.m[j] / sqrt(r2_plain(dx, dy, dz));
    }
  }
  for (int c = 0; c < 8; ++c) {
    const double s = warp_sum(acc[c]);
    if (lane == 0) s_red[wid][c] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double t[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < EJ_THREADS / 32; ++w)
      for (int c = 0; c < 8; ++c) t[c] += s_red[w][c];
    const double qx = t[0] - t[3], qy = t[1] - t[4], qz = t[2] - t[5];
    const double dP = (r2_plain(qx, qy, qz) - r2_plain(t[0], t[1], t[2])) / (2.0 * P.m0);
    const double dE = -t[6] + t[7] + dP;  // E after - E before
    *S.U -= dE;
    s_P[0] = t[0]; s_P[1] = t[1]; s_P[2] = t[2];
    s_base = atomicAdd(S.nej, ne);
    S.flags[0] = 1;  // the next opening kick recomputes every pair
  }
  __syncthreads();
  const double step = (double)S.counters[C_STEPS];
  for (int q = tid; q < ne; q += EJ_THREADS) {
    const int k = s_ord[q];
    write_record(S, s_base + q, k, step, s_P[0], s_P[1], s_P[2], P.inv_m0);
    make_ghost(S, k);
  }
}

// ---------------------------------------------------------------------------------------------
// Batched systems (up to 64 bodies each, their own central masses): one warp per system.
constexpr int BEJ_THREADS = 128;

__device__ __forceinline__ u64 warp_or64(u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(BEJ_THREADS) k_b_eject(Sim S, DevParams P) {
  const int s = (blockIdx.x * BEJ_THREADS + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= S.nsys) return;  // warp-uniform
  const int st = S.sys_start[s], n = S.sys_start[s + 1] - st, np = S.npad;
  const double m0 = S.sys_m0[s];
  u64 live = 0ULL, out = 0ULL;  // bit q: body st + q
  for (int q = lane; q < n; q += 32) {
    const int i = st + q;
    if (!S.alive[i]) continue;
    live |= 1ULL << q;
    if (ejected(P, r2_plain(S.x[i], S.x[np + i], S.x[2 * np + i]))) out |= 1ULL << q;
  }
  live = warp_or64(live);
  out = warp_or64(out);
  const int nlive = __popcll(live), nout = __popcll(out);
  const bool stop = P.nmin > 0 && nlive > 0 && nlive - nout < P.nmin;
  const u64 rem = stop ? live : out;
  if (rem == 0ULL) return;  // uniform
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int q = lane; q < n; q += 32) {
    if (!((live >> q) & 1ULL)) continue;
    const int i = st + q;
    const double mi = S.m[i], vx = S.v[i], vy = S.v[np + i], vz = S.v[2 * np + i];
    acc[0] = fma(mi, vx, acc[0]); acc[1] = fma(mi, vy, acc[1]); acc[2] = fma(mi, vz, acc[2]);
    if ((rem >> q) & 1ULL) {
      acc[3] = fma(mi, vx, acc[3]); acc[4] = fma(mi, vy, acc[4]); acc[5] = fma(mi, vz, acc[5]);
      const double r = sqrt(r2_plain(S.x[i], S.x[np + i], S.x[2 * np + i]));
      acc[6] += 0.5 * mi * r2_plain(vx, vy, vz) - P.G * m0 * mi / r;
    }
  }
  u64 bits = rem;
  while (bits) {
    const int qk = __ffsll((long long)bits) - 1;
    bits &= bits - 1;
    const int k = st + qk;
    const double xk = S.x[k], yk = S.x[np + k], zk = S.x[2 * np + k], gmk = P.G * S.m[k];
    for (int q = lane; q < n; q += 32) {
      if (q == qk || !((live >> q) & 1ULL) || (((rem >> q) & 1ULL) && q < qk)) continue;
      const int j = st + q;
      const double dx = S.x[j] - xk, dy = S.x[np + j] - yk, dz = S.x[2 * np + j] - zk;
      acc[7] += gmk * S.m[j] / sqrt(r2_plain(dx, dy, dz));
    }
  }
  for (int c = 0; c < 8; ++c) acc[c] = warp_sum(acc[c]);
  int base = 0;
  if (lane == 0) {
    const double qx = acc[0] - acc[3], qy = acc[1] - acc[4], qz = acc[2] - acc[5];
    const double dP = (r2_plain(qx, qy, qz) - r2_plain(acc[0], acc[1], acc[2])) / (2.0 * m0);
    atomicAdd(S.U, -(-acc[6] + acc[7] + dP));
    S.sys_flag[s] = 1;  // the system's next opening kick recomputes every pair
    if (nout) base = atomicAdd(S.nej, nout);
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  const double step = (double)S.counters[C_STEPS];
  for (int q = lane; q < n; q += 32) {
    if (!((rem >> q) & 1ULL)) continue;
    if ((out >> q) & 1ULL)  // rank among the ejected bodies of this system: ascending index
      write_record(S, base + __popcll(out & ((1ULL << q) - 1ULL)), st + q, step, acc[0], acc[1], acc[2], 1.0 / m0);
    make_ghost(S, st + q);
  }
}

// ---------------------------------------------------------------------------------------------
// Test particles: removed by the same limits (they carry no energy); counted in counters[4].
__global__ void k_tp_eject(TPSet T, DevParams P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T.n || !T.alive[i]) return;
  const int np = T.npad;
  if (!ejected(P, r2_plain(T.x[i], T.x[np + i], T.x[2 * np + i]))) return;
  T.alive[i] = 0;
  atomicAdd((unsigned long long *)&T.counters[4], 1ULL);
}

void launch_eject(const Sim &S, const DevParams &P, cudaStream_t st) { k_eject<<<1, EJ_THREADS, 0, st>>>(S, P); }
void launch_b_eject(const Sim &S, const DevParams &P, cudaStream_t st) {
  k_b_eject<<<(S.nsys * 32 + BEJ_THREADS - 1) / BEJ_THREADS, BEJ_THREADS, 0, st>>>(S, P);
}
void launch_tp_eject(const TPSet &T, const DevParams &P, cudaStream_t st) {
  k_tp_eject<<<(T.n + 255) / 256, 256, 0, st>>>(T, P);
}

}  // namespace genga
