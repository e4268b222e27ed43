// noalloc.cu -- genga_kick_noalloc: the kick phase (accelerations + precheck candidates) for
// callers that must not allocate device memory.
//
// cudaMalloc can block on the driver's allocator and cudaFree synchronises the whole device, so
// code that runs inside a latency-critical loop, or that lives in a process whose device memory
// is owned by another allocator (a framework's caching allocator, an embedding application with
// a fixed memory budget), cannot call entry points that allocate. This variant keeps all of its
// scratch in one file-scope __device__ array instead: every GPU that loads the library holds it
// (about 2 MB) until the process exits. The caller still provides the inputs and outputs.
#include <atomic>
#include <cstring>

#include "../../include/genga.h"
#include "genga_launch.h"

using namespace genga;

namespace {

constexpr int NA_NMAX = 1024;              // largest n accepted by genga_kick_noalloc
constexpr int NA_NT = NA_NMAX / 32;        // tiles
constexpr int NA_W = NA_NMAX / 32;         // bitmap words per row
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// byte offsets of the sub-arrays inside the scratch array
constexpr size_t O_X = 0;
constexpr size_t O_V = O_X + align256(3 * NA_NMAX * sizeof(double));
constexpr size_t O_M = O_V + align256(3 * NA_NMAX * sizeof(double));
constexpr size_t O_GM = O_M + align256(NA_NMAX * sizeof(double));
constexpr size_t O_R = O_GM + align256(NA_NMAX * sizeof(double));
constexpr size_t O_HILL = O_R + align256(NA_NMAX * sizeof(double));
constexpr size_t O_RC = O_HILL + align256(NA_NMAX * sizeof(double));
constexpr size_t O_A = O_RC + align256(NA_NMAX * sizeof(double));
constexpr size_t O_ALIVE = O_A + align256(NA_NMAX * sizeof(double));
constexpr size_t O_T = O_ALIVE + align256(NA_NMAX * sizeof(int));
constexpr size_t O_RCSQ = O_T + align256(NA_NMAX * sizeof(u64));
constexpr size_t O_AFAR = O_RCSQ + align256(NA_NMAX * sizeof(u64));
constexpr size_t O_AOUT = O_AFAR + align256(3 * NA_NMAX * sizeof(double));
constexpr size_t O_PART = O_AOUT + align256(3 * NA_NMAX * sizeof(double));
constexpr size_t O_PKICK = O_PART + align256((size_t)NA_NT * NA_NT * 2 * 96 * sizeof(double));
constexpr size_t O_PFIN = O_PKICK + align256(NA_NT * 3 * sizeof(double));
constexpr size_t O_CBM = O_PFIN + align256(NA_NT * 3 * sizeof(double));
constexpr size_t O_ROWANY = O_CBM + align256((size_t)NA_NMAX * NA_W * sizeof(unsigned));
constexpr size_t O_CCNT = O_ROWANY + align256(NA_W * sizeof(unsigned));
constexpr size_t O_CLIST = O_CCNT + align256(NA_NMAX * sizeof(int));
constexpr size_t O_ITEMS = O_CLIST + align256((size_t)NA_NMAX * CCAP * sizeof(int));
constexpr size_t O_FLAGS = O_ITEMS + align256((size_t)NA_NT * NA_NT * sizeof(int));
constexpr size_t O_STATUS = O_FLAGS + align256(4 * sizeof(int));
constexpr size_t O_COUNTERS = O_STATUS + align256(sizeof(int));
constexpr size_t NA_BYTES = O_COUNTERS + align256(NCOUNTERS * sizeof(long long));

}  // namespace

// The scratch shared by every call. In host code this name is only a stand-in for the device
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_kick_scratch[NA_BYTES];

namespace {

constexpr int NA_MAXDEV = 64;
std::atomic<unsigned char *> g_scratch_ptr[NA_MAXDEV] = {};  // device address of g_kick_scratch, per device

// Set-up, once per device, with that device current. Threads that get here first at the same time
// look the address up alike and store the same value.
int scratch_address(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAXDEV) return GENGA_ECUDA;
  unsigned char *p = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    void *q = nullptr;
    if (cudaGetSymbolAddress(&q, g_kick_scratch) != cudaSuccess || !q) return GENGA_ECUDA;
    p = (unsigned char *)q;
    g_scratch_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return GENGA_OK;
}

// kick work list: for tile I the diagonal item, then both halves of every J > I
__global__ void k_items(int *items, int nt) {
  const int I = threadIdx.x;
  if (I >= nt) return;
  int k = I * (2 * nt - I);
  items[k++] = I | (I << 10);
  for (int J = I + 1; J < nt; ++J) {
    items[k++] = I | (J << 10);
    items[k++] = I | (J << 10) | (1 << 20);
  }
}

}  // namespace

extern "C" int genga_kick_noalloc(int n, double G, double pc, int kmode, int precise_div, const double *m,
                                  const int *alive, const double *x, const double *rc, double *a, int *cand,
                                  int cap, int *ncand, void *stream) {
  if (n > NA_NMAX) return GENGA_ESIZE;
  if (n < 1 || !m || !alive || !x || !rc || !a || !ncand || cap < 0 || (cap > 0 && !cand) || !(G > 0.0) ||
      !(pc >= 1.0) || (kmode != 0 && kmode != 1))
    return GENGA_EINVAL;
  unsigned char *base = nullptr;
  int rc0 = scratch_address(&base);
  if (rc0 != GENGA_OK) return rc0;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GENGA_ECUDA;

  Sim S;
  memset(&S, 0, sizeof(S));
  S.n = n;
  S.npad = ((n + 31) / 32) * 32;
  S.nt = S.npad / 32;
  S.W = S.npad / 32;
  S.x = (double *)(base + O_X); S.v = (double *)(base + O_V);
  S.m = (double *)(base + O_M); S.gm = (double *)(base + O_GM); S.R = (double *)(base + O_R);
  S.hill = (double *)(base + O_HILL); S.rc = (double *)(base + O_RC); S.A = (double *)(base + O_A);
  S.alive = (int *)(base + O_ALIVE); S.T = (u64 *)(base + O_T); S.rcsq = (u64 *)(base + O_RCSQ);
  S.afar = (double *)(base + O_AFAR); S.part = (double *)(base + O_PART);
  S.pkick = (double *)(base + O_PKICK); S.pfin = (double *)(base + O_PFIN);
  S.cbm = (unsigned *)(base + O_CBM); S.rowany = (unsigned *)(base + O_ROWANY);
  S.ccnt = (int *)(base + O_CCNT); S.clist = (int *)(base + O_CLIST);
  S.items = (int *)(base + O_ITEMS);
  S.nitems = S.nt * S.nt;
  S.nwarps = S.nitems < 8 * sms ? S.nitems : 8 * sms;  // the allocating kick's configuration
  S.flags = (int *)(base + O_FLAGS); S.status = (int *)(base + O_STATUS);
  S.counters = (long long *)(base + O_COUNTERS);
  double *aout = (double *)(base + O_AOUT);

  genga_params prm;
  genga_default_params(&prm);
  prm.pc = pc;
  prm.kmode = kmode;
  DevParams P;
  memset(&P, 0, sizeof(P));
  P.G = G; P.m0 = 1.0; P.Gm0 = G; P.inv_m0 = 1.0; P.mu2 = 2.0 * G; P.inv_mu = 1.0 / G;
  P.n1 = prm.n1; P.n2 = prm.n2; P.pc = prm.pc; P.bs_eps = prm.bs_eps; P.bs_kmax = prm.bs_kmax;
  P.bs_max_halvings = prm.bs_max_halvings; P.kepler_maxit = prm.kepler_maxit; P.kmode = kmode;
  P.collisions = prm.collisions;

  // the array keeps the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(S.cbm, 0, (size_t)S.npad * S.W * sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(S.rowany, 0, (size_t)S.W * sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(S.ccnt, 0, (size_t)S.npad * sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(S.flags, 0, 4 * sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(S.status, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(S.counters, 0, NCOUNTERS * sizeof(long long), st) != cudaSuccess)
    return GENGA_ECUDA;
  k_items<<<1, 32, 0, st>>>(S.items, S.nt);
  launch_soa_setup(S, P, m, alive, x, nullptr, rc, n, st);
  launch_kick(S, P, false, precise_div != 0, st);
  launch_fin(S, P, FIN_INIT, 0.0, 0.0, aout, st);
  if (cudaMemcpy2DAsync(a, n * sizeof(double), aout, S.npad * sizeof(double), n * sizeof(double), 3,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return GENGA_ECUDA;
  launch_bitmap_pairs(S.cbm, S.npad, S.W, cand, cap, ncand, st);
  return cudaGetLastError() == cudaSuccess ? GENGA_OK : GENGA_ECUDA;
}
