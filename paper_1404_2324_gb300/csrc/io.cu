// io.cu -- coordinate conversions between the caller's heliocentric AoS arrays and the internal
// democratic SoA state (Sect. 2.1: heliocentric positions, barycentric velocities), the total
// energy (Sect. 4.1), and a self-check of the device arithmetic helpers.
#include "genga_launch.h"

namespace genga {

constexpr int IO_THREADS = 1024;

// Block-wide sum of three doubles in a fixed order (one CTA of IO_THREADS threads).
__device__ void block_sum3(double v[3], double (*sh)[3]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = warp_sum(v[c]);
  if (lane == 0) for (int c = 0; c < 3; ++c) sh[wid][c] = v[c];
  __syncthreads();
  if (wid == 0) {
    for (int c = 0; c < 3; ++c) {
      double a = lane < IO_THREADS / 32 ? sh[lane][c] : 0.0;
      v[c] = warp_sum(a);
    }
    if (lane == 0) for (int c = 0; c < 3; ++c) sh[0][c] = v[c];
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) v[c] = sh[0][c];
  __syncthreads();
}

// xh, vh: [3 (n+1)] AoS with the central mass in row 0; m_in, R_in: [n+1]. With m_in == nullptr
// the bodies keep their masses, radii and live flags, and only live bodies take the new state.
__global__ void __launch_bounds__(IO_THREADS) k_from_helio(Sim S, DevParams P, const double *xh, const double *vh,
                                                           const double *m_in, const double *R_in) {
  const bool keep = (m_in == nullptr);
  __shared__ double sh[IO_THREADS / 32][3];
  __shared__ double smass[IO_THREADS / 32];
  const int np = S.npad, n = S.n, tid = threadIdx.x;
  double pm[3] = {0.0, 0.0, 0.0}, mt = 0.0;
  for (int i = tid; i < n; i += IO_THREADS) {
    const double mi = keep ? (S.alive[i] ? S.m[i] : 0.0) : m_in[i + 1];
    mt += mi;
    for (int c = 0; c < 3; ++c) pm[c] = fma(mi, vh[3 * (i + 1) + c], pm[c]);
  }
  block_sum3(pm, sh);
  mt = warp_sum(mt);
  if ((tid & 31) == 0) smass[tid >> 5] = mt;
  __syncthreads();
  if (tid < 32) {
    double a = smass[tid];
    a = warp_sum(a);
    if (tid == 0) smass[0] = a;
  }
  __syncthreads();
  const double Mtot = P.m0 + smass[0];
  double vcm[3];
  for (int c = 0; c < 3; ++c) vcm[c] = pm[c] / Mtot;  // v_b = v_h - sum m v_h / (m0 + sum m)
  for (int i = tid; i < np; i += IO_THREADS) {
    if (keep) {
      if (i < n && S.alive[i])
        for (int c = 0; c < 3; ++c) {
          S.x[c * np + i] = xh[3 * (i + 1) + c];
          S.v[c * np + i] = vh[3 * (i + 1) + c] - vcm[c];
        }
    } else if (i < n) {
      const double mi = m_in[i + 1];
      for (int c = 0; c < 3; ++c) {
        S.x[c * np + i] = xh[3 * (i + 1) + c];
        S.v[c * np + i] = vh[3 * (i + 1) + c] - vcm[c];
      }
      S.m[i] = mi; S.gm[i] = P.G * mi; S.R[i] = R_in[i + 1];
      S.hill[i] = cbrt(mi / (3.0 * P.m0));
      S.alive[i] = 1;
    } else {  // padding: massless, parked far out, never alive
      S.x[i] = PARK + 1.0e4 * i; S.x[np + i] = 0.0; S.x[2 * np + i] = 0.0;
      for (int c = 0; c < 3; ++c) S.v[c * np + i] = 0.0;
      S.m[i] = 0.0; S.gm[i] = 0.0; S.R[i] = 0.0; S.hill[i] = 0.0; S.alive[i] = 0;
    }
  }
}

// Back to heliocentric AoS with the central mass in row 0: v_h = v_b + P/m0 (Sect. 2.1).
__global__ void __launch_bounds__(IO_THREADS) k_to_helio(Sim S, DevParams P, double *xh, double *vh, double *m_out,
                                                         double *R_out, int *alive_out) {
  __shared__ double sh[IO_THREADS / 32][3];
  const int np = S.npad, n = S.n, tid = threadIdx.x;
  double pm[3] = {0.0, 0.0, 0.0};
  for (int i = tid; i < n; i += IO_THREADS)
    if (S.alive[i]) for (int c = 0; c < 3; ++c) pm[c] = fma(S.m[i], S.v[c * np + i], pm[c]);
  block_sum3(pm, sh);
  if (tid == 0) {
    for (int c = 0; c < 3; ++c) { if (xh) xh[c] = 0.0; if (vh) vh[c] = 0.0; }
    if (m_out) m_out[0] = P.m0;
    if (R_out) R_out[0] = 0.0;
    if (alive_out) alive_out[0] = 1;
  }
  for (int i = tid; i < n; i += IO_THREADS) {
    for (int c = 0; c < 3; ++c) {
      if (xh) xh[3 * (i + 1) + c] = S.x[c * np + i];
      if (vh) vh[3 * (i + 1) + c] = fma(pm[c], P.inv_m0, S.v[c * np + i]);
    }
    if (m_out) m_out[i + 1] = S.m[i];
    if (R_out) R_out[i + 1] = S.R[i];
    if (alive_out) alive_out[i + 1] = S.alive[i];
  }
}

// Energy: block (I, J), J >= I, sums the pair potentials of tile I against tile J (and, on the
// diagonal, the kinetic and central terms of tile I) into scratch[I*nt + J].
__global__ void __launch_bounds__(32) k_energy_part(Sim S, DevParams P, double *scratch) {
  const int I = blockIdx.x, J = blockIdx.y, lane = threadIdx.x, np = S.npad, nt = S.nt;
  if (J < I) { if (lane == 0) scratch[I * nt + J] = 0.0; return; }
  const int i = I * 32 + lane;
  double e = 0.0;
  if (S.alive[i]) {
    const double xi = S.x[i], yi = S.x[np + i], zi = S.x[2 * np + i], mi = S.m[i];
    if (I == J) {
      const double vx = S.v[i], vy = S.v[np + i], vz = S.v[2 * np + i];
      e += 0.5 * mi * (vx * vx + vy * vy + vz * vz) - P.G * P.m0 * mi / sqrt(xi * xi + yi * yi + zi * zi);
    }
    for (int jl = 0; jl < 32; ++jl) {
      const int j = J * 32 + jl;
      if (j <= i || !S.alive[j]) continue;
      const double dx = S.x[j] - xi, dy = S.x[np + j] - yi, dz = S.x[2 * np + j] - zi;
      e -= P.G * mi * S.m[j] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  }
  e = warp_sum(e);
  if (lane == 0) scratch[I * nt + J] = e;
}

__global__ void k_energy_sum(Sim S, DevParams P, const double *scratch, double *E) {
  const int lane = threadIdx.x, np = S.npad, nt = S.nt;
  double e = 0.0, p[3] = {0.0, 0.0, 0.0};
  for (int k = lane; k < nt * nt; k += 32) e += scratch[k];
  for (int i = lane; i < np; i += 32)
    if (S.alive[i]) for (int c = 0; c < 3; ++c) p[c] = fma(S.m[i], S.v[c * np + i], p[c]);
  e = warp_sum(e);
  for (int c = 0; c < 3; ++c) p[c] = warp_sum(p[c]);
  if (lane == 0) *E = e + (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) / (2.0 * P.m0);
}

__global__ void k_mathcheck(int n, int which, const double *in, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = in[i];
  out[i] = which == 0 ? rsqrt_refined(x) : (which == 1 ? rcube_refined(x) : rcp_refined(x));
}

// FP64 throughput probe: every thread advances 8 independent FMA chains x -> x b + c (b = 1 - 2^-40,
// so the chains stay near c / (1 - b) and never overflow); 2 flops per FMA. The sum is written only
// when it takes an impossible value, so the chains are not optimised away and nothing is stored.
constexpr int PROBE_CHAINS = 8;
__global__ void __launch_bounds__(256) k_fp64_probe(int iters, double seed, double *out) {
  double a[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = seed + 1e-3 * k + 1e-9 * threadIdx.x;
  const double b = 1.0 - 9.094947017729282e-13, c = 1e-12;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
  if (s == -1.0) out[0] = s;
}

// Phase entry points: load caller SoA arrays of n bodies into a Sim of padded size.
__global__ void k_soa_setup(Sim S, DevParams P, const double *m, const int *alive, const double *x,
                            const double *v, const double *rc, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int np = S.npad;
  if (i >= np) return;
  const bool in = i < n && (alive == nullptr || alive[i]);
  for (int c = 0; c < 3; ++c) {
    S.x[c * np + i] = in ? x[c * n + i] : (c == 0 ? PARK + 1.0e4 * i : 0.0);
    S.v[c * np + i] = (in && v) ? v[c * n + i] : 0.0;
  }
  const double mi = in && m ? m[i] : 0.0;
  S.m[i] = mi; S.gm[i] = P.G * mi; S.R[i] = 0.0;
  S.hill[i] = in ? cbrt(mi / (3.0 * P.m0)) : 0.0;
  S.alive[i] = in ? 1 : 0;
  double r = (in && rc) ? rc[i] : 0.0;
  S.rc[i] = r;
  const double t = __dmul_rn(P.pc, r);
  S.T[i] = in ? dbits(__dmul_rn(t, t)) : 0ULL;
  S.rcsq[i] = in ? dbits(__dmul_rn(r, r)) : 0ULL;
  S.A[i] = (in && dbits(r) != 0ULL) ? rcp_refined(0.9 * r) : 0.0;
}

__global__ void k_soa_out(Sim S, double *x, double *v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int c = 0; c < 3; ++c) {
    if (x) x[c * n + i] = S.x[c * S.npad + i];
    if (v) v[c * n + i] = S.v[c * S.npad + i];
  }
}

void launch_from_helio(const Sim &S, const DevParams &P, const double *xh, const double *vh,
                       const double *m_in, const double *R_in, cudaStream_t st) {
  k_from_helio<<<1, IO_THREADS, 0, st>>>(S, P, xh, vh, m_in, R_in);
}
void launch_to_helio(const Sim &S, const DevParams &P, double *xh, double *vh, double *m_out,
                     double *R_out, int *alive_out, cudaStream_t st) {
  k_to_helio<<<1, IO_THREADS, 0, st>>>(S, P, xh, vh, m_out, R_out, alive_out);
}
void launch_energy(const Sim &S, const DevParams &P, double *scratch, double *E, cudaStream_t st) {
  k_energy_part<<<dim3(S.nt, S.nt), 32, 0, st>>>(S, P, scratch);
  k_energy_sum<<<1, 32, 0, st>>>(S, P, scratch, E);
}
double fp64_probe_flops(int iters, int blocks, float *ms, cudaStream_t st, double *scratch) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fp64_probe<<<blocks, 256, 0, st>>>(iters / 8 > 0 ? iters / 8 : 1, 1.0, scratch);  // warm-up
  cudaEventRecord(e0, st);
  k_fp64_probe<<<blocks, 256, 0, st>>>(iters, 1.0, scratch);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float t = 0.0f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ms) *ms = t;
  return 2.0 * PROBE_CHAINS * (double)iters * (double)blocks * 256.0 / (t * 1e-3);
}

void launch_mathcheck(int n, int which, const double *in, double *out, cudaStream_t st) {
  k_mathcheck<<<(n + 127) / 128, 128, 0, st>>>(n, which, in, out);
}
void launch_soa_setup(const Sim &S, const DevParams &P, const double *m, const int *alive,
                      const double *x, const double *v, const double *rc, int n, cudaStream_t st) {
  k_soa_setup<<<(S.npad + 127) / 128, 128, 0, st>>>(S, P, m, alive, x, v, rc, n);
}
void launch_soa_out(const Sim &S, double *x, double *v, int n, cudaStream_t st) {
  k_soa_out<<<(n + 127) / 128, 128, 0, st>>>(S, x, v, n);
}

}  // namespace genga
