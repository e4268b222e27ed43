// api.cu -- the C ABI (include/genga.h): context, device memory, the host step driver (one full
// step captured once into a CUDA graph and replayed; every branch is decided on the device),
// state I/O and the phase entry points.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/genga.h"
#include "genga_launch.h"

using namespace genga;

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return GENGA_ECUDA;     \
  } while (0)

namespace {

struct DevMem {
  std::vector<void *> ptrs;
  cudaError_t err = cudaSuccess;
  template <class T>
  T *get(size_t count) {
    void *p = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&p, (count ? count : 1) * sizeof(T));
    if (err == cudaSuccess) { ptrs.push_back(p); cudaMemset(p, 0, (count ? count : 1) * sizeof(T)); }
    return (T *)p;
  }
  void release() {
    for (void *p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Allocates a Sim for n orbiting bodies with room for nsub encounter bitmaps.
bool alloc_sim(Sim &S, DevMem &mem, int n, int nsub) {
  memset(&S, 0, sizeof(S));
  S.n = n;
  S.npad = ((n + 31) / 32) * 32;
  if (S.npad < 32) S.npad = 32;
  S.nt = S.npad / 32;
  S.W = S.npad / 32;
  const size_t np = S.npad, nt = S.nt, W = S.W;
  S.x = mem.get<double>(3 * np); S.v = mem.get<double>(3 * np);
  S.x0 = mem.get<double>(3 * np); S.v0 = mem.get<double>(3 * np);
  S.m = mem.get<double>(np); S.gm = mem.get<double>(np); S.R = mem.get<double>(np); S.hill = mem.get<double>(np);
  S.alive = mem.get<int>(np);
  S.rc = mem.get<double>(np); S.A = mem.get<double>(np);
  S.T = mem.get<u64>(np); S.rcsq = mem.get<u64>(np);
  S.afar = mem.get<double>(3 * np);
  S.part = mem.get<double>(nt * nt * 2 * 96);
  S.pkick = mem.get<double>(nt * 3); S.pfin = mem.get<double>(nt * 3);
  S.cbm = mem.get<unsigned>(np * W); S.rowany = mem.get<unsigned>(W);
  S.ccnt = mem.get<int>(np); S.clist = mem.get<int>(np * CCAP);
  S.ebm = mem.get<unsigned>((size_t)nsub * np * W);
  const size_t ecap = np * (np - 1) / 2 + 1;
  S.edges = mem.get<int>(2 * ecap); S.nedges = mem.get<int>(1);
  S.fail = mem.get<int>(np); S.nfail = mem.get<int>(1);
  S.gstart = mem.get<int>(np + 1); S.gmem = mem.get<int>(np); S.ngroups = mem.get<int>(1);
  S.big = mem.get<int>(np); S.nbig = mem.get<int>(1);
  // kick work list: for each tile I, the diagonal tile, then both halves of every J > I
  std::vector<int> items;
  for (int I = 0; I < S.nt; ++I) {
    items.push_back(I | (I << 10));
    for (int J = I + 1; J < S.nt; ++J) {
      items.push_back(I | (J << 10));
      items.push_back(I | (J << 10) | (1 << 20));
    }
  }
  S.nitems = (int)items.size();
  S.items = mem.get<int>(items.size());
  // two warps per sub-partition: the second hides the first's FP64 dependency waits (measured at
  // N = 2048: one warp 102.6 us, two 88.3 us, three 89.8 us, four 90.2 us per kick)
  const int target = 8 * num_sms();
  S.nwarps = S.nitems < target ? S.nitems : target;
  S.flags = mem.get<int>(4); S.status = mem.get<int>(1);
  S.counters = mem.get<long long>(NCOUNTERS); S.U = mem.get<double>(1);
  S.ejrec = mem.get<double>(8 * (size_t)EJ_CAP); S.nej = mem.get<int>(1);
  // grid-wide BS of one large group at a time (up to npad members)
  BsGridBuf &B = S.gb;
  B.pos = mem.get<double>(2 * BS_LEVELS * np * 3);
  B.za = mem.get<double>(BS_LEVELS * np * 6); B.zb = mem.get<double>(BS_LEVELS * np * 6);
  B.t1 = mem.get<double>(BS_LEVELS * np * 6); B.prev = mem.get<double>(np * 6 * BS_LEVELS);
  B.y = mem.get<double>(2 * np * 6); B.isc = mem.get<double>(np * 2);
  B.idx = mem.get<int>(np); B.alive = mem.get<int>(np);
  B.gm = mem.get<double>(np); B.m = mem.get<double>(np); B.R = mem.get<double>(np); B.A = mem.get<double>(np);
  B.rcsq = mem.get<u64>(np); B.err = mem.get<u64>(2 * BS_LEVELS); B.bar = mem.get<unsigned>(4);
  B.cont = mem.get<int>(GR_CONTACT_CAP); B.ncont = mem.get<int>(1);
  S.spin = mem.get<double>(3 * np);
  S.crec = mem.get<double>((size_t)CREC_CAP * CREC); S.ncrec = mem.get<int>(1);
  if (mem.err != cudaSuccess) return false;
  cudaMemcpy(S.items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice);
  return cudaGetLastError() == cudaSuccess;
}

DevParams make_params(double G, double m0, const genga_params &p) {
  DevParams P;
  memset(&P, 0, sizeof(P));
  P.G = G; P.m0 = m0; P.Gm0 = G * m0; P.inv_m0 = 1.0 / m0;
  P.mu2 = 2.0 * G * m0; P.inv_mu = 1.0 / (G * m0);
  P.n1 = p.n1; P.n2 = p.n2; P.pc = p.pc; P.bs_eps = p.bs_eps;
  P.bs_kmax = p.bs_kmax; P.bs_max_halvings = p.bs_max_halvings; P.kepler_maxit = p.kepler_maxit;
  P.kmode = p.kmode; P.collisions = p.collisions;
  P.rcut2 = p.rcut > 0.0 ? p.rcut * p.rcut : 0.0;
  P.rcut_sun2 = p.rcut_sun > 0.0 ? p.rcut_sun * p.rcut_sun : 0.0;
  P.nmin = p.nmin;
  return P;
}

int substep_weights(int order, double *w) {
  if (order == 4) {  // Yoshida (1990): w1 = 1/(2 - 2^(1/3)), w0 = -2^(1/3)/(2 - 2^(1/3))
    const double c = cbrt(2.0);
    w[0] = w[2] = 1.0 / (2.0 - c);
    w[1] = -c / (2.0 - c);
    return 3;
  }
  if (order == 6) {  // Yoshida (1990) Table 1, solution A
    const double w1 = -1.17767998417887, w2 = 0.235573213359357, w3 = 0.784513610477560;
    const double w0 = 1.0 - 2.0 * (w1 + w2 + w3);
    const double s[7] = {w3, w2, w1, w0, w1, w2, w3};
    for (int k = 0; k < 7; ++k) w[k] = s[k];
    return 7;
  }
  w[0] = 1.0;
  return 1;
}

bool finite_all(const double *a, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(a[k])) return false;
  return true;
}

}  // namespace

struct genga_ctx {
  int n;  // orbiting bodies
  double G, m0, dt;
  int order, nsub;
  double w[7];
  genga_params prm;
  DevParams P;
  Sim S;
  DevMem mem;
  cudaStream_t own = nullptr, stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int bs_grid = 1;
  int tp_grid = 1;  // blocks of the test-particle encounter and BS kernels
  // main mode: groups of gsplit or more members go to the cluster BS kernel, on a side branch of
  // the step graph that runs beside the one-CTA BS kernel
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int gsplit = BS_GMAX + 1, cl_grid = 0, pair_grid = 0;
  // a further branch: groups above BS_GMAX members (main mode; the larger batched groups too)
  cudaStream_t side2 = nullptr;
  cudaEvent_t ev_join2 = nullptr;
  // test-particle mode: the planets' path table on a branch of its own
  cudaStream_t side3 = nullptr;
  cudaEvent_t ev_tab = nullptr, ev_tabj = nullptr;
  int small_grid = 0;
  int wide_grid = 8;  // CTAs of the wide BS kernel (batched groups of BS_GMAX + 1 .. BS_GWIDE members: rare)
  int grid_blocks = 1;  // CTAs of the grid-wide BS kernel (main mode: groups above BS_GMAX members)
  bool profiling = false;
  // batched mode
  bool batched = false;
  int nsys = 0, b_split = 1, b_block = 128, steps_per_launch = 1;
  // batched mode as one persistent launch (batch_persist.cu), chosen at init when faster
  bool persist = false;
  int persist_blocks = 0, persist_per_sm = 0;
  int *bp_queue = nullptr, *bp_base = nullptr;
  float tune_ms_graph = 0.0f, tune_ms_persist = 0.0f;
  int *perm = nullptr, *sys_user = nullptr;  // device: internal body -> user body, internal system -> user system
  std::vector<int> perm_h;                    // host copy of perm (ejection records)
  std::vector<int> start_h;                   // host copy of the internal systems' first bodies
  double *sysE = nullptr;
  // a large batch in parts: sub-contexts over consecutive runs of the caller's systems, each on its
  // own stream, forked from and joined to this context's stream, so that one part's BS tail runs
  // beside the other parts' kicks and drifts (this context then holds no state of its own)
  std::vector<genga_ctx *> parts;
  std::vector<int> part_body0, part_sys0;  // first caller body and system of each part
  std::vector<cudaEvent_t> part_ev;        // per part: the end of its work, for the join
  // test-particle mode
  bool tpmode = false;
  TPSet T{};
  double *stx = nullptr, *stv = nullptr;
  int *stalive = nullptr;
  cudaGraphExec_t gexec1 = nullptr;  // one-step graph for remainders
  cudaGraph_t graph1 = nullptr;
  cudaEvent_t kev[2 * 7] = {};
  int nkev = 0;
  // staging
  double *sx = nullptr, *sv = nullptr, *sm = nullptr, *sR = nullptr, *scratch = nullptr, *sE = nullptr;
  int *salive = nullptr, *spairs = nullptr, *scount = nullptr;
  size_t pair_cap = 0;
};

namespace {

void drop_graph(genga_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->gexec1) cudaGraphExecDestroy(c->gexec1);
  if (c->graph1) cudaGraphDestroy(c->graph1);
  c->gexec = nullptr;
  c->graph = nullptr;
  c->gexec1 = nullptr;
  c->graph1 = nullptr;
}

// The first kick (Sect. 2.2): critical radii, far-field accelerations and candidates of the
// current state, with no velocity change. Also run after set_state / set_params.
int first_kick(genga_ctx *c) {
  Sim &S = c->S;
  cudaStream_t st = c->stream;
  CK(cudaMemsetAsync(S.cbm, 0, (size_t)S.npad * S.W * sizeof(unsigned), st));
  CK(cudaMemsetAsync(S.rowany, 0, (size_t)S.W * sizeof(unsigned), st));
  CK(cudaMemsetAsync(S.ccnt, 0, (size_t)S.npad * sizeof(int), st));
  CK(cudaMemsetAsync(S.flags, 0, 4 * sizeof(int), st));
  CK(cudaMemsetAsync(S.nedges, 0, sizeof(int), st));
  CK(cudaMemsetAsync(S.nfail, 0, sizeof(int), st));
  launch_rcrit(S, c->P, std::fabs(c->dt), 0, st);
  if (!c->tpmode) {
    // the main mode's next step opens with the full pair kick (the plain definition of the opening
    // kick), which also records the precheck candidates of its first substep: flags 0 and 3, which
    // that step's drift clears; a separate first kick would compute the same sums once more
    CK(cudaMemsetAsync(S.flags, 1, sizeof(int), st));
    CK(cudaMemsetAsync(S.flags + 3, 1, sizeof(int), st));
    CK(cudaGetLastError());
    return GENGA_OK;
  }
  launch_kick(S, c->P, false, c->prm.precise_div != 0, st);
  launch_fin(S, c->P, FIN_INIT, 0.0, 0.0, nullptr, st);
  if (c->tpmode) {
    CK(cudaMemsetAsync(c->T.npairs, 0, sizeof(unsigned), st));
    CK(cudaMemsetAsync(c->T.bsnext, 0, (4 + 4 * TP_BS_MAXBLOCKS) * sizeof(unsigned), st));
    launch_tp_rcrit(c->T, c->P, std::fabs(c->dt), 0, st);
    launch_tp_kick(S, c->T, c->P, st);
  }
  CK(cudaGetLastError());
  return GENGA_OK;
}

// Batched mode: first kick of every system (critical radii, far field, candidates).
int first_kick_batch(genga_ctx *c) {
  Sim &S = c->S;
  cudaStream_t st = c->stream;
  CK(cudaMemsetAsync(S.sys_flag, 0, (size_t)c->nsys * sizeof(int), st));
  launch_b_rcrit(S, c->P, std::fabs(c->dt), 0, st);
  launch_b_kick(S, c->P, FIN_INIT, 0.0, 0.0, c->b_split, c->b_block, st);
  CK(cudaGetLastError());
  return GENGA_OK;
}

// Batched mode: one full step of every system (the same sequence as the single system, with
// per-system momenta and central masses).
void enqueue_step_batch(genga_ctx *c, cudaStream_t st) {
  const Sim &S = c->S;
  const DevParams &P = c->P;
  const double dt = c->dt;
  launch_b_rcrit(S, P, std::fabs(dt), 1, st);
  launch_b_kick(S, P, FIN_OPEN, 0.5 * c->w[0] * dt, 0.0, c->b_split, c->b_block, st);
  for (int j = 0; j < c->nsub; ++j) {
    const double tau = c->w[j] * dt;
    launch_b_momentum(S, S.sys_ppost, st);
    launch_b_drift(S, P, tau, 0.5 * tau, j > 0 ? 0.5 * c->w[j - 1] * dt : 0.0, j, st);
    launch_b_encounter(S, tau, st);
    launch_b_group(S, st);
    if (c->side) {  // fork: pairs (two warps each), groups of 3..BS_SMALL (128-thread CTAs) and the
                    // larger ones (256-thread CTAs) on three branches, each from its own queue; join
      cudaEventRecord(c->ev_fork, st);
      cudaStreamWaitEvent(c->side, c->ev_fork, 0);
      cudaStreamWaitEvent(c->side2, c->ev_fork, 0);
      launch_bs_pair(S, P, tau, c->pair_grid, c->side);
      launch_bs(S, P, tau, c->bs_grid, c->side2, BS_GMAX + 1, BS_SMALL + 1);
      launch_bs_wide(S, P, tau, c->wide_grid, c->side2);  // queue 3: groups above BS_GMAX members
      launch_bs_small(S, P, tau, c->small_grid, st);
      cudaEventRecord(c->ev_join, c->side);
      cudaEventRecord(c->ev_join2, c->side2);
      cudaStreamWaitEvent(st, c->ev_join, 0);
      cudaStreamWaitEvent(st, c->ev_join2, 0);
    } else {
      launch_bs(S, P, tau, c->bs_grid, st);
    }
    launch_b_momentum(S, S.sys_ppre, st);
    const double h2 = (j + 1 < c->nsub) ? 0.5 * c->w[j + 1] * dt : 0.0;
    launch_b_kick(S, P, FIN_CLOSE, 0.5 * tau, h2, c->b_split, c->b_block, st);
  }
  launch_b_hc(S, 0.5 * c->w[c->nsub - 1] * dt, st);
  if (P.rcut2 > 0.0 || P.rcut_sun2 > 0.0 || P.nmin > 0) launch_b_eject(S, P, st);
}

// One full step (Sect. 2.2 second list, composed per Sect. 2.3).
void enqueue_step(genga_ctx *c, cudaStream_t st) {
  const Sim &S = c->S;
  const DevParams &P = c->P;
  const bool precise = c->prm.precise_div != 0;
  const double dt = c->dt, inv_m0 = 1.0 / c->m0;
  const bool tp = c->tpmode;
  const TPSet &T = c->T;
  launch_rcrit(S, P, std::fabs(dt), 1, st);
  launch_kick(S, P, true, precise, st);  // runs only if the critical radii grew too much
  launch_fin(S, P, FIN_OPEN, 0.5 * c->w[0] * dt, 0.0, nullptr, st);
  for (int j = 0; j < c->nsub; ++j) {
    const double tau = c->w[j] * dt;
    const double hcm2 = j > 0 ? 0.5 * c->w[j - 1] * dt * inv_m0 : 0.0;
    // the particles' drift runs before the massive drift (which clears the reuse flag the opening
    // kick reads); at the first substep it carries their critical radii and opening kick as well
    if (tp && j == 0) launch_tp_open_drift(S, T, P, std::fabs(dt), 0.5 * c->w[0] * dt, tau, 0.5 * tau * inv_m0, st);
    else if (tp) launch_tp_drift(S, T, P, tau, 0.5 * tau * inv_m0, hcm2, st);
    launch_drift(S, P, tau, 0.5 * tau * inv_m0, hcm2, j, st);             // clears the reuse flag
    if (tp) {  // the planets' paths for the particles, on a branch beside the planets' encounters and BS
      cudaEventRecord(c->ev_tab, st);
      cudaStreamWaitEvent(c->side3, c->ev_tab, 0);
      launch_planet_table(S, T, P, tau, c->side3);
      cudaEventRecord(c->ev_tabj, c->side3);
    }
    // the paper's literal higher-order variant: the step-start candidates serve every substep, and
    // the closing kicks between substeps weigh every pair without prechecking
    const bool inner = c->prm.precheck_substeps == 0 && j + 1 < c->nsub;
    launch_encounter_group(S, tau, S.ebm + (size_t)j * S.npad * S.W, st, inner, c->side ? c->gsplit : BS_GMAX + 1);
    if (c->side) {  // fork: cluster kernel for the groups of gsplit .. BS_GMAX members, one-CTA
                    // kernel for the smaller ones and the grid-wide kernel for groups above BS_GMAX
                    // members (its CTAs leave at once when the large-group list holds none); join
      cudaEventRecord(c->ev_fork, st);
      cudaStreamWaitEvent(c->side, c->ev_fork, 0);
      cudaStreamWaitEvent(c->side2, c->ev_fork, 0);
      launch_bs_cluster(S, P, tau, c->gsplit, c->cl_grid, c->side);
      launch_bs_grid(S, P, tau, BS_GMAX + 1, c->grid_blocks, c->side2);
      launch_bs(S, P, tau, c->bs_grid, st, c->gsplit);
      cudaEventRecord(c->ev_join, c->side);
      cudaEventRecord(c->ev_join2, c->side2);
      cudaStreamWaitEvent(st, c->ev_join, 0);
      cudaStreamWaitEvent(st, c->ev_join2, 0);
    } else {
      launch_bs(S, P, tau, c->bs_grid, st);
    }
    if (tp) {  // the particles' encounter test beside the massive closing kick
      cudaEventRecord(c->ev_fork, st);
      cudaStreamWaitEvent(c->side, c->ev_fork, 0);
      cudaStreamWaitEvent(c->side, c->ev_tabj, 0);  // and the planets' path table
      launch_tp_encounter(S, T, tau, c->tp_grid, c->side);
      cudaEventRecord(c->ev_join, c->side);
    }
    if (c->profiling) cudaEventRecordWithFlags(c->kev[2 * j], st, cudaEventRecordExternal);
    launch_kick(S, P, inner, precise, st, inner);
    if (c->profiling) cudaEventRecordWithFlags(c->kev[2 * j + 1], st, cudaEventRecordExternal);
    const double h2 = (j + 1 < c->nsub) ? 0.5 * c->w[j + 1] * dt : 0.0;
    launch_fin(S, P, inner ? FIN_CLOSE_ALL : FIN_CLOSE, 0.5 * tau, h2, nullptr, st);
    if (tp) {  // join; the particles' BS and every particle's closing kick (after the last substep
               // with their last Sun drift, from the massive momentum before the closing kick)
      cudaStreamWaitEvent(st, c->ev_join, 0);
      launch_tp_bs(S, T, P, tau, 0.5 * tau, h2, j + 1 == c->nsub ? 0.5 * tau * inv_m0 : 0.0, num_sms(), st);
    }
  }
  launch_hc(S, 0.5 * c->w[c->nsub - 1] * dt * inv_m0, st);
  if (P.rcut2 > 0.0 || P.rcut_sun2 > 0.0) {  // ejections at the end of the step (Sect. 3.2)
    if (tp) launch_tp_eject(T, P, st);
    launch_eject(S, P, st);
  }
}

// The persistent batched launch runs the step without the end-of-step ejection limits (Rcut,
// RcutSun, Nmin); with any of them set the step graph runs instead.
bool use_persistent(const genga_ctx *c) {
  return c->persist && !(c->P.rcut2 > 0.0) && !(c->P.rcut_sun2 > 0.0) && c->P.nmin <= 0;
}

// Batched mode: the state of genga_init_batch again (from the staging copies of the input), with every
// counter, record and the step count cleared -- after the autotuner's trial steps.
int reset_batch(genga_ctx *c) {
  Sim &S = c->S;
  cudaStream_t st = c->stream;
  const size_t np = S.npad;
  CK(cudaMemsetAsync(S.counters, 0, NCOUNTERS * sizeof(long long), st));
  CK(cudaMemsetAsync(S.status, 0, sizeof(int), st));
  CK(cudaMemsetAsync(S.U, 0, sizeof(double), st));
  CK(cudaMemsetAsync(S.nej, 0, sizeof(int), st));
  CK(cudaMemsetAsync(S.ncrec, 0, sizeof(int), st));
  CK(cudaMemsetAsync(S.spin, 0, 3 * np * sizeof(double), st));
  CK(cudaMemsetAsync(S.bsn, 0, np, st));
  CK(cudaMemsetAsync(S.alive, 0, np * sizeof(int), st));
  CK(cudaMemsetAsync(c->bp_base, 0, sizeof(int), st));
  launch_b_from_helio(S, c->P, c->perm, c->sx, c->sv, c->sm, c->sR, 0, st);
  CK(cudaGetLastError());
  return first_kick_batch(c);
}

// Captured on the context's own stream (the caller's stream may be the legacy default stream,
// which cannot be captured); the executable graph is then launched on whichever stream is set.
int build_graph(genga_ctx *c) {
  drop_graph(c);
  if (c->stream != c->own) {  // the capture must see everything the caller enqueued so far
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, c->stream));
    CK(cudaStreamWaitEvent(c->own, ev, 0));
    CK(cudaEventDestroy(ev));
  }
  for (int pass = 0; pass < (c->batched && c->steps_per_launch > 1 ? 2 : 1); ++pass) {
    const int nst = pass == 0 ? c->steps_per_launch : 1;
    CK(cudaStreamBeginCapture(c->own, cudaStreamCaptureModeThreadLocal));
    if (c->batched && use_persistent(c)) {
      launch_b_persist(c->S, c->P, c->dt, c->w, c->nsub, nst, c->bp_base, c->bp_queue, c->persist_blocks, c->own);
    } else {
      for (int k = 0; k < nst; ++k) {
        if (c->batched) enqueue_step_batch(c, c->own);
        else enqueue_step(c, c->own);
      }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->own, &g);
    if (e != cudaSuccess || !g) return GENGA_ECUDA;
    if (pass == 0) {
      c->graph = g;
      CK(cudaGraphInstantiate(&c->gexec, c->graph, 0));
    } else {
      c->graph1 = g;
      CK(cudaGraphInstantiate(&c->gexec1, c->graph1, 0));
    }
  }
  return GENGA_OK;
}

}  // namespace

extern "C" {

int genga_default_params(genga_params *p) {
  if (!p) return GENGA_EINVAL;
  p->n1 = 3.0;
  p->n2 = 0.4;
  p->pc = 3.0;
  p->bs_eps = 1e-12;
  p->bs_kmax = 8;
  p->bs_max_halvings = 30;
  p->kepler_maxit = 30;
  p->kmode = 0;
  p->collisions = 1;
  p->precise_div = 0;
  p->rcut = 0.0;
  p->rcut_sun = 0.0;
  p->nmin = 0;
  p->precheck_substeps = 1;
  return GENGA_OK;
}

int genga_init(genga_ctx **out, int n, const double *masses, const double *radii, const double *x,
               const double *v, double G, double dt, int order, int mode) {
  if (!out) return GENGA_EINVAL;
  *out = nullptr;
  if (n < 2 || n > NMAX + 1 || !masses || !radii || !x || !v) return GENGA_EINVAL;
  if (!(G > 0.0) || !std::isfinite(G) || !std::isfinite(dt) || dt == 0.0) return GENGA_EINVAL;
  if (order != 2 && order != 4 && order != 6) return GENGA_EINVAL;
  if (mode != GENGA_MODE_MASSIVE) return GENGA_EINVAL;
  if (!(masses[0] > 0.0) || !finite_all(masses, n) || !finite_all(radii, n) ||
      !finite_all(x, 3 * (size_t)n) || !finite_all(v, 3 * (size_t)n))
    return GENGA_EINVAL;
  for (int i = 1; i < n; ++i)
    if (masses[i] < 0.0 || radii[i] < 0.0) return GENGA_EINVAL;
  genga_ctx *c = new genga_ctx();
  c->n = n - 1;
  c->G = G; c->m0 = masses[0]; c->dt = dt; c->order = order;
  c->nsub = substep_weights(order, c->w);
  genga_default_params(&c->prm);
  c->P = make_params(G, c->m0, c->prm);
  if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) { delete c; return GENGA_ECUDA; }
  c->stream = c->own;
  if (!alloc_sim(c->S, c->mem, c->n, c->nsub)) { c->mem.release(); cudaStreamDestroy(c->own); delete c; return GENGA_ENOMEM; }
  const size_t nn = (size_t)n;
  c->sx = c->mem.get<double>(3 * nn); c->sv = c->mem.get<double>(3 * nn);
  c->sm = c->mem.get<double>(nn); c->sR = c->mem.get<double>(nn);
  c->salive = c->mem.get<int>(nn);
  c->scratch = c->mem.get<double>((size_t)c->S.nt * c->S.nt); c->sE = c->mem.get<double>(1);
  c->pair_cap = (size_t)c->S.npad * (c->S.npad - 1) / 2 + 1;
  c->spairs = c->mem.get<int>(2 * c->pair_cap); c->scount = c->mem.get<int>(1);
  if (c->mem.err != cudaSuccess) { genga_free(c); return GENGA_ENOMEM; }
  c->bs_grid = 2 * num_sms();
  if (c->bs_grid > c->S.npad) c->bs_grid = c->S.npad;
  bs_init_constants();
  bs_cluster_init_constants();
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming) != cudaSuccess) {
    genga_free(c);
    return GENGA_ECUDA;
  }
  c->gsplit = 5;  // measured: from 5 members on, a cluster per group beats one CTA per group
  c->cl_grid = bs_cluster_grid();
  bs_grid_init_constants();
  c->grid_blocks = bs_grid_blocks();
  cudaStream_t st = c->stream;
  if (cudaMemcpyAsync(c->sx, x, 3 * nn * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->sv, v, 3 * nn * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->sm, masses, nn * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->sR, radii, nn * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    genga_free(c);
    return GENGA_ECUDA;
  }
  launch_from_helio(c->S, c->P, c->sx, c->sv, c->sm, c->sR, st);
  int rc = first_kick(c);
  if (rc == GENGA_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GENGA_ECUDA;
  if (rc != GENGA_OK) { genga_free(c); return rc; }
  *out = c;
  return GENGA_OK;
}

int genga_init_tp(genga_ctx **out, int n, const double *masses, const double *radii, const double *x,
                  const double *v, double G, double dt, int order, int n_tp, const double *xt, const double *vt,
                  const double *Rt) {
  if (!out) return GENGA_EINVAL;
  *out = nullptr;
  if (n < 2 || n > 33 || n_tp < 1 || n_tp > (1 << 26) || !xt || !vt) return GENGA_EINVAL;
  if (!finite_all(xt, 3 * (size_t)n_tp) || !finite_all(vt, 3 * (size_t)n_tp) || (Rt && !finite_all(Rt, n_tp)))
    return GENGA_EINVAL;
  genga_ctx *c = nullptr;
  int rc = genga_init(&c, n, masses, radii, x, v, G, dt, order, GENGA_MODE_MASSIVE);
  if (rc != GENGA_OK) return rc;
  TPSet &T = c->T;
  DevMem &mem = c->mem;
  T.n = n_tp;
  T.npad = ((n_tp + 31) / 32) * 32;
  const size_t np = T.npad;
  T.x = mem.get<double>(3 * np); T.v = mem.get<double>(3 * np);
  T.x0 = mem.get<double>(3 * np); T.v0 = mem.get<double>(3 * np);
  T.R = mem.get<double>(np); T.rc = mem.get<double>(np); T.A = mem.get<double>(np);
  T.afar = mem.get<double>(3 * np);
  T.T = mem.get<u64>(np); T.rcsq = mem.get<u64>(np);
  T.alive = mem.get<int>(np); T.full = mem.get<int>(np); T.fail = mem.get<int>(np);
  T.cmask = mem.get<unsigned>(np); T.emask = mem.get<unsigned>(np);
  T.bslist = mem.get<int>(np); T.nbs = mem.get<int>(2); T.bsnext = mem.get<unsigned>(4 + 4 * TP_BS_MAXBLOCKS);
  T.pairs = mem.get<unsigned>(np * (size_t)(n - 1)); T.npairs = mem.get<unsigned>(1);
  T.ptab = mem.get<double>(TP_MAXPL * TP_TAB * 6);
  T.ppoly = mem.get<double>(TP_MAXPL * 6 * TP_CHEB); T.pcok = mem.get<int>(TP_MAXPL);
  T.counters = mem.get<long long>(8);
  c->stx = mem.get<double>(3 * (size_t)n_tp); c->stv = mem.get<double>(3 * (size_t)n_tp);
  c->stalive = mem.get<int>(n_tp);
  double *sR = mem.get<double>(n_tp);
  if (mem.err != cudaSuccess) { genga_free(c); return GENGA_ENOMEM; }
  cudaStream_t st = c->stream;
  if (cudaMemcpyAsync(c->stx, xt, 3 * (size_t)n_tp * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->stv, vt, 3 * (size_t)n_tp * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (Rt && cudaMemcpyAsync(sR, Rt, (size_t)n_tp * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)) {
    genga_free(c);
    return GENGA_ECUDA;
  }
  // the staging arrays still hold the massive heliocentric input of genga_init
  launch_tp_from_helio(T, n, c->sm, c->sv, c->stx, c->stv, Rt ? sR : nullptr, 0, st);
  c->tpmode = true;
  c->tp_grid = 4 * num_sms();
  if (cudaStreamCreateWithFlags(&c->side3, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_tab, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_tabj, cudaEventDisableTiming) != cudaSuccess) {
    genga_free(c);
    return GENGA_ECUDA;
  }
  if (tp_init_constants() != 0) { genga_free(c); return GENGA_ECUDA; }
  rc = first_kick(c);
  if (rc == GENGA_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GENGA_ECUDA;
  if (rc != GENGA_OK) { genga_free(c); return rc; }
  *out = c;
  return GENGA_OK;
}

int genga_get_state_tp(genga_ctx *c, double *xt, double *vt, int *tp_alive) {
  if (!c || !c->tpmode) return GENGA_EINVAL;
  const size_t n = (size_t)c->T.n;
  cudaStream_t st = c->stream;
  launch_tp_to_helio(c->S, c->T, c->P, xt ? c->stx : nullptr, vt ? c->stv : nullptr, tp_alive ? c->stalive : nullptr, st);
  CK(cudaGetLastError());
  if (xt) CK(cudaMemcpyAsync(xt, c->stx, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (vt) CK(cudaMemcpyAsync(vt, c->stv, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (tp_alive) CK(cudaMemcpyAsync(tp_alive, c->stalive, n * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return GENGA_OK;
}

int genga_tp_status(genga_ctx *c, long long *detail) {
  if (!c || !c->tpmode || !detail) return GENGA_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(detail, c->T.counters, 5 * sizeof(long long), cudaMemcpyDeviceToHost));
  return GENGA_OK;
}

static int init_batch_one(genga_ctx **out, int n_sys, const int *offsets, const double *m0, const double *masses,
                          const double *radii, const double *x, const double *v, double G, double dt, int order,
                          int steps_per_launch) {
  if (!out) return GENGA_EINVAL;
  *out = nullptr;
  if (n_sys < 1 || !offsets || !m0 || !masses || !radii || !x || !v || steps_per_launch < 1) return GENGA_EINVAL;
  if (!(G > 0.0) || !std::isfinite(G) || !std::isfinite(dt) || dt == 0.0) return GENGA_EINVAL;
  if (order != 2 && order != 4 && order != 6) return GENGA_EINVAL;
  if (offsets[0] != 0) return GENGA_EINVAL;
  for (int s = 0; s < n_sys; ++s) {
    const int ns = offsets[s + 1] - offsets[s];
    if (ns < 1 || ns > 64 || !(m0[s] > 0.0) || !std::isfinite(m0[s])) return GENGA_EINVAL;
  }
  const int n = offsets[n_sys];
  if (n > (1 << 26)) return GENGA_EINVAL;
  if (!finite_all(masses, n) || !finite_all(radii, n) || !finite_all(x, 3 * (size_t)n) || !finite_all(v, 3 * (size_t)n))
    return GENGA_EINVAL;
  for (int i = 0; i < n; ++i)
    if (masses[i] < 0.0 || radii[i] < 0.0) return GENGA_EINVAL;
  genga_ctx *c = new genga_ctx();
  c->batched = true;
  c->n = n;
  c->nsys = n_sys;
  c->steps_per_launch = steps_per_launch;
  c->G = G; c->m0 = 1.0; c->dt = dt; c->order = order;
  c->nsub = substep_weights(order, c->w);
  genga_default_params(&c->prm);
  c->P = make_params(G, 1.0, c->prm);
  if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) { delete c; return GENGA_ECUDA; }
  c->stream = c->own;
  // internal order: systems by size (largest first), bodies of a system contiguous
  std::vector<int> order_s(n_sys);
  for (int s = 0; s < n_sys; ++s) order_s[s] = s;
  std::stable_sort(order_s.begin(), order_s.end(), [&](int a, int b) {
    return offsets[a + 1] - offsets[a] > offsets[b + 1] - offsets[b];
  });
  std::vector<int> start(n_sys + 1), sys_of, perm, sys_user(n_sys);
  std::vector<double> sm0(n_sys);
  start[0] = 0;
  for (int k = 0; k < n_sys; ++k) {
    const int s = order_s[k], ns = offsets[s + 1] - offsets[s];
    start[k + 1] = start[k] + ns;
    sys_user[k] = s;
    sm0[k] = m0[s];
    for (int q = 0; q < ns; ++q) { perm.push_back(offsets[s] + q); sys_of.push_back(k); }
  }
  c->perm_h = perm;
  c->start_h = start;
  Sim &S = c->S;
  DevMem &mem = c->mem;
  memset(&S, 0, sizeof(S));
  S.n = n;
  S.npad = ((n + 31) / 32) * 32;
  S.nt = S.npad / 32;
  S.W = 0;
  const size_t np = S.npad;
  S.x = mem.get<double>(3 * np); S.v = mem.get<double>(3 * np);
  S.x0 = mem.get<double>(3 * np); S.v0 = mem.get<double>(3 * np);
  S.m = mem.get<double>(np); S.gm = mem.get<double>(np); S.R = mem.get<double>(np); S.hill = mem.get<double>(np);
  S.alive = mem.get<int>(np);
  S.rc = mem.get<double>(np); S.A = mem.get<double>(np);
  S.T = mem.get<u64>(np); S.rcsq = mem.get<u64>(np);
  S.afar = mem.get<double>(3 * np);
  S.fail = mem.get<int>(np); S.nfail = mem.get<int>(1);
  S.gstart = mem.get<int>(np + 1); S.gmem = mem.get<int>(np); S.ngroups = mem.get<int>(1);
  S.gsize = mem.get<int>(np + 1); S.gtotal = mem.get<int>(1); S.bsq = mem.get<unsigned>(4);
  S.gorder = mem.get<int>(4 * (size_t)np); S.norder = mem.get<int>(8); S.bsn = mem.get<unsigned char>(np);
  S.flags = mem.get<int>(4); S.status = mem.get<int>(1);
  S.counters = mem.get<long long>(NCOUNTERS); S.U = mem.get<double>(1);
  S.ejrec = mem.get<double>(8 * (size_t)EJ_CAP); S.nej = mem.get<int>(1);
  S.nsys = n_sys;
  S.sys_of = mem.get<int>(np); S.sys_start = mem.get<int>(n_sys + 1);
  S.sys_m0 = mem.get<double>(n_sys); S.sys_ppre = mem.get<double>(3 * (size_t)n_sys);
  S.sys_ppost = mem.get<double>(3 * (size_t)n_sys); S.sys_flag = mem.get<int>(n_sys);
  S.bmask = mem.get<u64>(np); S.emask = mem.get<u64>(np);
  // the symmetric kick's warp work items: a system of 33..64 bodies alone, smaller ones packed in
  // lane segments of the next power of two of their size (systems are ordered by size, largest first)
  std::vector<int> kjobs;
  for (int k = 0; k < n_sys;) {
    const int ns = start[k + 1] - start[k];
    if (ns > 32) { kjobs.push_back(k); kjobs.push_back(64 << 8 | 1); ++k; continue; }
    int w = 1;
    while (w < ns) w <<= 1;
    const int k0 = k;
    int cnt = 0;
    while (k < n_sys && cnt < 32 / w) {
      const int m = start[k + 1] - start[k];
      int wm = 1;
      while (wm < m) wm <<= 1;
      if (m > 32 || wm != w) break;
      ++cnt;
      ++k;
    }
    kjobs.push_back(k0); kjobs.push_back(w << 8 | cnt);
  }
  S.nkjobs = (int)kjobs.size() / 2;
  S.kjobs = mem.get<int>(kjobs.size());
  S.spin = mem.get<double>(3 * np);
  S.crec = mem.get<double>((size_t)CREC_CAP * CREC); S.ncrec = mem.get<int>(1);
  c->perm = mem.get<int>(n); c->sys_user = mem.get<int>(n_sys); c->sysE = mem.get<double>(n_sys);
  c->sx = mem.get<double>(3 * (size_t)n); c->sv = mem.get<double>(3 * (size_t)n);
  c->sm = mem.get<double>(n); c->sR = mem.get<double>(n); c->salive = mem.get<int>(n);
  if (mem.err != cudaSuccess) { genga_free(c); return GENGA_ENOMEM; }
  // the pair kernel (4 groups per CTA) takes one CTA per SM, which leaves the other register half of
  // every SM to k_bs from the start: at two per SM it held the whole GPU and k_bs, the longer branch,
  // began 0.5 ms later (measured: 3.06M -> 3.15M system-steps/s)
  c->pair_grid = num_sms();
  // groups of 3..BS_SMALL members (most of those above pairs) on 128-thread CTAs: two fit beside a
  // pair CTA in the register file where one 256-thread CTA did; the few larger groups take a half grid
  c->small_grid = 4 * num_sms();
  c->bs_grid = num_sms() / 2;
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming) != cudaSuccess) {
    genga_free(c);
    return GENGA_ECUDA;
  }
  sys_of.resize(np, 0);  // padding bodies: never alive
  cudaStream_t st = c->stream;
  if (cudaMemcpy(S.sys_of, sys_of.data(), np * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(S.sys_start, start.data(), (n_sys + 1) * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(S.kjobs, kjobs.data(), kjobs.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(S.sys_m0, sm0.data(), n_sys * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->perm, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->sys_user, sys_user.data(), n_sys * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpyAsync(c->sx, x, 3 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->sv, v, 3 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->sm, masses, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->sR, radii, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    genga_free(c);
    return GENGA_ECUDA;
  }
  bs_init_constants();
  launch_b_from_helio(S, c->P, c->perm, c->sx, c->sv, c->sm, c->sR, 0, st);
  // autotune the kick's shape on the first kick: threads per body x block size, or (split 0) the
  // Newton's-third-law kernel (one warp per work item) x block size
  launch_b_rcrit(S, c->P, std::fabs(dt), 0, st);
  {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    const int splits[4] = {0, 1, 2, 4}, blocks[3] = {64, 128, 256};
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 3; ++b) {
        launch_b_kick(S, c->P, FIN_INIT, 0.0, 0.0, splits[a], blocks[b], st);  // warm
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) launch_b_kick(S, c->P, FIN_INIT, 0.0, 0.0, splits[a], blocks[b], st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; c->b_split = splits[a]; c->b_block = blocks[b]; }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  int rc = first_kick_batch(c);
  if (rc == GENGA_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GENGA_ECUDA;
  if (rc != GENGA_OK) { genga_free(c); return rc; }
  // the schedule: the step graph (phase by phase over all systems) against one persistent launch (a
  // CTA per system at a time) at one and at two CTAs per SM, each timed on two steps of this batch;
  // the state is then put back as it was
  c->bp_queue = mem.get<int>(1);
  c->bp_base = mem.get<int>(1);
  c->persist_per_sm = mem.err == cudaSuccess ? b_persist_init() : 0;
  if (c->persist_per_sm > 0) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int tsteps = 2;
    float best = 1e30f;
    cudaEventRecord(e0, st);
    for (int k = 0; k < tsteps; ++k) enqueue_step_batch(c, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&c->tune_ms_graph, e0, e1);
    c->tune_ms_graph /= tsteps;
    for (int per = 1; per <= (c->persist_per_sm < 2 ? c->persist_per_sm : 2); ++per) {
      if (reset_batch(c) != GENGA_OK) break;
      const int blocks = per * num_sms();
      cudaEventRecord(e0, st);
      launch_b_persist(S, c->P, dt, c->w, c->nsub, tsteps, c->bp_base, c->bp_queue, blocks, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= tsteps;
      if (ms < best) { best = ms; c->persist_blocks = blocks; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tune_ms_persist = best;
    // the graph's trial issues its kernels one by one, launch gaps the step graph itself does not
    // pay (8192 systems: trial 2.7-2.8 ms a step, 2.13 ms in the graph; persistent 2.85 ms either
    // way), so the persistent launch is taken only when it is clearly faster
    c->persist = c->persist_blocks > 0 && best < 0.85f * c->tune_ms_graph;
    rc = reset_batch(c);
    if (rc == GENGA_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GENGA_ECUDA;
    if (rc != GENGA_OK) { genga_free(c); return rc; }
  }
  *out = c;
  return GENGA_OK;
}

// Parts: this context's stream forks to every part's stream before its work, and waits for all of
// them after it.
static int parts_fork(genga_ctx *c) {
  CK(cudaEventRecord(c->ev_fork, c->stream));
  for (genga_ctx *p : c->parts) CK(cudaStreamWaitEvent(p->stream, c->ev_fork, 0));
  return GENGA_OK;
}
static int parts_join(genga_ctx *c) {
  for (size_t k = 0; k < c->parts.size(); ++k) {
    CK(cudaEventRecord(c->part_ev[k], c->parts[k]->stream));
    CK(cudaStreamWaitEvent(c->stream, c->part_ev[k], 0));
  }
  return GENGA_OK;
}

// Batches of 1024 systems and more run in parts of about 256 systems (at most 32), consecutive in
// the caller's order: measured on 8192 systems, 3.68 M system-steps/s in one step graph, 4.18 M in
// two parts, 4.35 M in three, 4.44 M in eight (each part with the kick shape it chose alone); with
// one Newton's-third-law kick shape for all, 4.83 M in 8 parts and 5.07 M in 16; with the BS grids
// shared out as below, 5.15 M in 16, 5.20 M in 24, 5.21-5.23 M in 32. Every part runs the step
// graph, all with one kick shape, timed over all parts at once.
int genga_init_batch(genga_ctx **out, int n_sys, const int *offsets, const double *m0, const double *masses,
                     const double *radii, const double *x, const double *v, double G, double dt, int order,
                     int steps_per_launch) {
  if (!out) return GENGA_EINVAL;
  *out = nullptr;
  const int K = n_sys >= 1024 ? std::min(32, n_sys / 256) : 1;
  if (K <= 1 || !offsets || !m0 || !masses || !radii || !x || !v)
    return init_batch_one(out, n_sys, offsets, m0, masses, radii, x, v, G, dt, order, steps_per_launch);
  if (offsets[0] != 0) return GENGA_EINVAL;
  genga_ctx *c = new genga_ctx();
  c->batched = true;
  c->n = offsets[n_sys];
  c->nsys = n_sys;
  c->G = G; c->dt = dt; c->order = order;
  c->steps_per_launch = steps_per_launch;
  if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) { delete c; return GENGA_ECUDA; }
  c->stream = c->own;
  if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) { genga_free(c); return GENGA_ECUDA; }
  std::vector<int> sub;
  for (int k = 0; k < K; ++k) {
    const int s0 = (int)((long)n_sys * k / K), s1 = (int)((long)n_sys * (k + 1) / K);
    const int b0 = offsets[s0];
    sub.assign(offsets + s0, offsets + s1 + 1);
    for (int &o : sub) o -= b0;
    genga_ctx *p = nullptr;
    int rc = init_batch_one(&p, s1 - s0, sub.data(), m0 + s0, masses + b0, radii + b0, x + 3 * (size_t)b0,
                            v + 3 * (size_t)b0, G, dt, order, steps_per_launch);
    cudaEvent_t ev = nullptr;
    if (rc == GENGA_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) rc = GENGA_ECUDA;
    if (rc != GENGA_OK) {
      genga_free(p);
      genga_free(c);
      return rc;
    }
    c->parts.push_back(p);
    c->part_ev.push_back(ev);
    c->part_body0.push_back(b0);
    c->part_sys0.push_back(s0);
  }
  // the kick shape, timed with every part's kick at once (a part timed alone prefers other shapes:
  // 8192 systems in 8 parts, 4.44 M system-steps/s with the shape the first part chose alone, 5.09 M
  // with the best one timed together)
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess ? GENGA_OK : GENGA_ECUDA;
  float best = 1e30f;
  int bsplit = 1, bblock = 128;
  const int splits[4] = {0, 1, 2, 4}, blocks[3] = {64, 128, 256};
  for (int a = 0; a < 4 && rc == GENGA_OK; ++a)
    for (int q = 0; q < 3 && rc == GENGA_OK; ++q) {
      float ms = 0.0f;
      for (int r = 0; r < 4 && rc == GENGA_OK; ++r) {  // a warm-up round, then three timed
        if (r == 1) rc = cudaEventRecord(e0, c->stream) == cudaSuccess ? GENGA_OK : GENGA_ECUDA;
        if (rc == GENGA_OK) rc = parts_fork(c);
        for (genga_ctx *p : c->parts) launch_b_kick(p->S, p->P, FIN_INIT, 0.0, 0.0, splits[a], blocks[q], p->stream);
        if (rc == GENGA_OK) rc = parts_join(c);
      }
      if (rc == GENGA_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = GENGA_ECUDA;
      if (rc == GENGA_OK && ms < best) { best = ms; bsplit = splits[a]; bblock = blocks[q]; }
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (genga_ctx *p : c->parts) {
    // the parts' BS kernels run side by side: each part a share of the grids one batch would use
    p->pair_grid = std::max(8, 2 * p->pair_grid / K);
    p->small_grid = std::max(16, 2 * p->small_grid / K);
    p->bs_grid = std::max(4, 2 * p->bs_grid / K);
    if (rc == GENGA_OK) rc = genga_batch_set_schedule(p, 0);
    if (rc == GENGA_OK) rc = genga_batch_set_kick(p, bsplit, bblock);
    // the counters as a batch of one part leaves them after init; then the first kick in this shape
    if (rc == GENGA_OK && cudaMemsetAsync(p->S.counters, 0, NCOUNTERS * sizeof(long long), p->stream) != cudaSuccess)
      rc = GENGA_ECUDA;
    if (rc == GENGA_OK) rc = first_kick_batch(p);
  }
  if (rc == GENGA_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = GENGA_ECUDA;
  for (genga_ctx *p : c->parts)
    if (rc == GENGA_OK && cudaStreamSynchronize(p->stream) != cudaSuccess) rc = GENGA_ECUDA;
  if (rc != GENGA_OK) { genga_free(c); return rc; }
  *out = c;
  return GENGA_OK;
}

int genga_batch_schedule(genga_ctx *c, int *persistent, int *ctas, float *ms_graph, float *ms_persistent) {
  if (!c || !c->batched) return GENGA_EINVAL;
  if (!c->parts.empty()) return genga_batch_schedule(c->parts[0], persistent, ctas, ms_graph, ms_persistent);
  if (persistent) *persistent = use_persistent(c) ? 1 : 0;
  if (ctas) *ctas = c->persist_blocks;
  if (ms_graph) *ms_graph = c->tune_ms_graph;
  if (ms_persistent) *ms_persistent = c->tune_ms_persist;
  return GENGA_OK;
}

int genga_batch_set_schedule(genga_ctx *c, int persistent) {
  if (c && !c->parts.empty()) {
    for (genga_ctx *p : c->parts) {
      const int rc = genga_batch_set_schedule(p, persistent);
      if (rc != GENGA_OK) return rc;
    }
    return GENGA_OK;
  }
  if (!c || !c->batched || (persistent != 0 && persistent != 1) || (persistent && c->persist_blocks < 1))
    return GENGA_EINVAL;
  c->persist = persistent != 0;
  drop_graph(c);
  return GENGA_OK;
}

int genga_batch_set_kick(genga_ctx *c, int split, int block) {
  if (c && !c->parts.empty()) {
    for (genga_ctx *p : c->parts) {
      const int rc = genga_batch_set_kick(p, split, block);
      if (rc != GENGA_OK) return rc;
    }
    return GENGA_OK;
  }
  if (!c || !c->batched || (split != 0 && split != 1 && split != 2 && split != 4) ||
      (block != 64 && block != 128 && block != 256))
    return GENGA_EINVAL;
  c->b_split = split;
  c->b_block = block;
  drop_graph(c);
  return GENGA_OK;
}

int genga_batch_info(genga_ctx *c, int *split, int *block, int *steps_per_launch) {
  if (!c || !c->batched) return GENGA_EINVAL;
  if (!c->parts.empty()) return genga_batch_info(c->parts[0], split, block, steps_per_launch);
  if (split) *split = c->b_split;
  if (block) *block = c->b_block;
  if (steps_per_launch) *steps_per_launch = c->steps_per_launch;
  return GENGA_OK;
}

int genga_get_state_batch(genga_ctx *c, double *x, double *v, double *m, double *R, int *alive) {
  if (!c || !c->batched) return GENGA_EINVAL;
  if (!c->parts.empty()) {
    int rc = parts_fork(c);
    for (size_t k = 0; k < c->parts.size() && rc == GENGA_OK; ++k) {
      const size_t b0 = c->part_body0[k];
      rc = genga_get_state_batch(c->parts[k], x ? x + 3 * b0 : nullptr, v ? v + 3 * b0 : nullptr, m ? m + b0 : nullptr,
                                 R ? R + b0 : nullptr, alive ? alive + b0 : nullptr);
    }
    return rc;
  }
  const size_t n = (size_t)c->n;
  cudaStream_t st = c->stream;
  launch_b_to_helio(c->S, c->perm, x ? c->sx : nullptr, v ? c->sv : nullptr, m ? c->sm : nullptr,
                    R ? c->sR : nullptr, alive ? c->salive : nullptr, st);
  CK(cudaGetLastError());
  if (x) CK(cudaMemcpyAsync(x, c->sx, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (v) CK(cudaMemcpyAsync(v, c->sv, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (m) CK(cudaMemcpyAsync(m, c->sm, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (R) CK(cudaMemcpyAsync(R, c->sR, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (alive) CK(cudaMemcpyAsync(alive, c->salive, n * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return GENGA_OK;
}

int genga_set_state_batch(genga_ctx *c, const double *x, const double *v) {
  if (!c || !c->batched || !x || !v) return GENGA_EINVAL;
  if (!c->parts.empty()) {
    int rc = parts_fork(c);
    for (size_t k = 0; k < c->parts.size() && rc == GENGA_OK; ++k)
      rc = genga_set_state_batch(c->parts[k], x + 3 * (size_t)c->part_body0[k], v + 3 * (size_t)c->part_body0[k]);
    return rc == GENGA_OK ? parts_join(c) : rc;
  }
  const size_t n = (size_t)c->n;
  cudaStream_t st = c->stream;
  CK(cudaMemcpyAsync(c->sx, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(c->sv, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
  launch_b_from_helio(c->S, c->P, c->perm, c->sx, c->sv, nullptr, nullptr, 1, st);
  CK(cudaGetLastError());
  return first_kick_batch(c);
}

int genga_energy_batch(genga_ctx *c, double *E, double *U) {
  if (!c || !c->batched || !E) return GENGA_EINVAL;
  if (!c->parts.empty()) {
    int rc = parts_fork(c);
    double tot = 0.0;
    for (size_t k = 0; k < c->parts.size() && rc == GENGA_OK; ++k) {
      double u = 0.0;
      rc = genga_energy_batch(c->parts[k], E + c->part_sys0[k], &u);
      tot += u;
    }
    if (U) *U = tot;
    return rc;
  }
  cudaStream_t st = c->stream;
  launch_b_energy(c->S, c->P, c->sys_user, c->sysE, st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(E, c->sysE, (size_t)c->nsys * sizeof(double), cudaMemcpyDeviceToHost, st));
  double u = 0.0;
  CK(cudaMemcpyAsync(&u, c->S.U, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (U) *U = u;
  return GENGA_OK;
}

int genga_set_params(genga_ctx *c, const genga_params *p) {
  if (!c || !p) return GENGA_EINVAL;
  if (!(p->n1 >= 0.0) || !(p->n2 >= 0.0) || !(p->pc >= 1.0) || !(p->bs_eps > 0.0) || p->bs_kmax < 2 ||
      p->bs_kmax > BS_LEVELS || p->bs_max_halvings < 0 || p->kepler_maxit < 1 || (p->kmode != 0 && p->kmode != 1))
    return GENGA_EINVAL;
  if (!(p->rcut >= 0.0) || !(p->rcut_sun >= 0.0) || p->nmin < 0 || (p->rcut > 0.0 && !(p->rcut > p->rcut_sun)))
    return GENGA_EINVAL;
  if ((p->precheck_substeps != 0 && p->precheck_substeps != 1) || (!p->precheck_substeps && (c->batched || c->tpmode)))
    return GENGA_EINVAL;
  if (!c->parts.empty()) {
    int rc = parts_fork(c);
    for (size_t k = 0; k < c->parts.size() && rc == GENGA_OK; ++k) rc = genga_set_params(c->parts[k], p);
    if (rc == GENGA_OK) c->prm = *p;
    return rc == GENGA_OK ? parts_join(c) : rc;
  }
  c->prm = *p;
  c->P = make_params(c->G, c->m0, c->prm);
  drop_graph(c);
  return c->batched ? first_kick_batch(c) : first_kick(c);
}

int genga_ejections(genga_ctx *c, double *rec, int cap, int *n) {
  if (!c || cap < 0 || (cap > 0 && !rec)) return GENGA_EINVAL;
  if (!c->parts.empty()) {  // the parts' records in part order, with the caller's body indices
    std::vector<double> all;
    int tot = 0;
    for (size_t k = 0; k < c->parts.size(); ++k) {
      int cnt = 0;
      int rc = genga_ejections(c->parts[k], nullptr, 0, &cnt);
      if (rc != GENGA_OK) return rc;
      tot += cnt;
      const int kept = cnt < EJ_CAP ? cnt : EJ_CAP;
      std::vector<double> r((size_t)kept * 8);
      if (kept > 0 && (rc = genga_ejections(c->parts[k], r.data(), kept, &cnt)) != GENGA_OK) return rc;
      for (int q = 0; q < kept; ++q) r[8 * (size_t)q] += c->part_body0[k];
      all.insert(all.end(), r.begin(), r.end());
    }
    if (n) *n = tot;
    const size_t w = std::min(all.size() / 8, (size_t)cap);
    if (w) memcpy(rec, all.data(), w * 8 * sizeof(double));
    return GENGA_OK;
  }
  CK(cudaStreamSynchronize(c->stream));
  int cnt = 0;
  CK(cudaMemcpy(&cnt, c->S.nej, sizeof(int), cudaMemcpyDeviceToHost));
  if (n) *n = cnt;
  int k = cnt < EJ_CAP ? cnt : EJ_CAP;
  if (k > cap) k = cap;
  if (k > 0) {
    CK(cudaMemcpy(rec, c->S.ejrec, 8 * (size_t)k * sizeof(double), cudaMemcpyDeviceToHost));
    for (int q = 0; q < k; ++q) {  // internal index -> the caller's
      const int i = (int)rec[8 * q];
      rec[8 * q] = (double)(c->batched ? c->perm_h[i] : i + 1);
    }
  }
  return GENGA_OK;
}

int genga_collisions(genga_ctx *c, double *rec, int cap, int *n) {
  if (!c || cap < 0 || (cap > 0 && !rec)) return GENGA_EINVAL;
  if (!c->parts.empty()) {  // the parts' reports with the caller's body indices, in the one order
    std::vector<double> all;
    int tot = 0;
    for (size_t k = 0; k < c->parts.size(); ++k) {
      int cnt = 0;
      int rc = genga_collisions(c->parts[k], nullptr, 0, &cnt);
      if (rc != GENGA_OK) return rc;
      tot += cnt;
      const int kept = cnt < CREC_CAP ? cnt : CREC_CAP;
      std::vector<double> r((size_t)kept * CREC);
      if (kept > 0 && (rc = genga_collisions(c->parts[k], r.data(), kept, &cnt)) != GENGA_OK) return rc;
      for (int q = 0; q < kept; ++q)
        for (int f : {3, 4, 23}) r[(size_t)q * CREC + f] += c->part_body0[k];
      all.insert(all.end(), r.begin(), r.end());
    }
    if (n) *n = tot;
    const int k = (int)(all.size() / CREC);
    std::vector<int> ord(k);
    for (int q = 0; q < k; ++q) ord[q] = q;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      const double *ra = all.data() + (size_t)a * CREC, *rb = all.data() + (size_t)b * CREC;
      for (int f : {0, 1, 2, 3, 4})
        if (ra[f] != rb[f]) return ra[f] < rb[f];
      return false;
    });
    const int w = k < cap ? k : cap;
    for (int q = 0; q < w; ++q) memcpy(rec + (size_t)q * CREC, all.data() + (size_t)ord[q] * CREC, CREC * sizeof(double));
    return GENGA_OK;
  }
  CK(cudaStreamSynchronize(c->stream));
  int cnt = 0;
  CK(cudaMemcpy(&cnt, c->S.ncrec, sizeof(int), cudaMemcpyDeviceToHost));
  if (n) *n = cnt;
  const int k = cnt < CREC_CAP ? cnt : CREC_CAP;
  if (k > 0 && cap > 0) {
    std::vector<double> all((size_t)k * CREC);
    CK(cudaMemcpy(all.data(), c->S.crec, all.size() * sizeof(double), cudaMemcpyDeviceToHost));
    auto user = [&](double i) { return (double)(c->batched ? c->perm_h[(int)i] : (int)i + 1); };
    for (int q = 0; q < k; ++q) {  // internal indices -> the caller's
      double *r = all.data() + (size_t)q * CREC;
      r[3] = user(r[3]); r[4] = user(r[4]); r[23] = user(r[23]);
    }
    // groups merge concurrently on the device: order the reports by (step, substep, time, i, j)
    std::vector<int> ord(k);
    for (int q = 0; q < k; ++q) ord[q] = q;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      const double *ra = all.data() + (size_t)a * CREC, *rb = all.data() + (size_t)b * CREC;
      for (int f : {0, 1, 2, 3, 4})
        if (ra[f] != rb[f]) return ra[f] < rb[f];
      return false;
    });
    const int w = k < cap ? k : cap;
    for (int q = 0; q < w; ++q) memcpy(rec + (size_t)q * CREC, all.data() + (size_t)ord[q] * CREC, CREC * sizeof(double));
  }
  return GENGA_OK;
}

// Spins: internal SoA [3][npad] <-> the caller's layout ([3n] with the central mass at row 0 in the
// single-system modes, [3N] flat in the batched mode).
int genga_set_spin(genga_ctx *c, const double *spin) {
  if (!c || !spin) return GENGA_EINVAL;
  if (!c->parts.empty()) {
    if (!finite_all(spin, 3 * (size_t)c->n)) return GENGA_EINVAL;
    int rc = parts_fork(c);
    for (size_t k = 0; k < c->parts.size() && rc == GENGA_OK; ++k)
      rc = genga_set_spin(c->parts[k], spin + 3 * (size_t)c->part_body0[k]);
    return rc;
  }
  const size_t np = c->S.npad;
  if (!finite_all(spin, 3 * (size_t)(c->batched ? c->n : c->n + 1))) return GENGA_EINVAL;
  std::vector<double> h(3 * np, 0.0);
  for (int i = 0; i < c->n; ++i) {
    const int u = c->batched ? c->perm_h[i] : i + 1;
    for (int k = 0; k < 3; ++k) h[k * np + i] = spin[3 * (size_t)u + k];
  }
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(c->S.spin, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  return GENGA_OK;
}

int genga_get_spin(genga_ctx *c, double *spin) {
  if (!c || !spin) return GENGA_EINVAL;
  if (!c->parts.empty()) {
    int rc = parts_fork(c);
    for (size_t k = 0; k < c->parts.size() && rc == GENGA_OK; ++k)
      rc = genga_get_spin(c->parts[k], spin + 3 * (size_t)c->part_body0[k]);
    return rc;
  }
  const size_t np = c->S.npad;
  std::vector<double> h(3 * np);
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(h.data(), c->S.spin, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
  if (!c->batched) for (int k = 0; k < 3; ++k) spin[k] = 0.0;
  for (int i = 0; i < c->n; ++i) {
    const int u = c->batched ? c->perm_h[i] : i + 1;
    for (int k = 0; k < 3; ++k) spin[3 * (size_t)u + k] = h[k * np + i];
  }
  return GENGA_OK;
}

int genga_set_stream(genga_ctx *c, void *stream) {
  if (!c) return GENGA_EINVAL;
  c->stream = stream ? (cudaStream_t)stream : c->own;
  drop_graph(c);
  return GENGA_OK;
}

int genga_step(genga_ctx *c, int n_steps) {
  if (!c || n_steps < 0) return GENGA_EINVAL;
  if (n_steps == 0) return GENGA_OK;
  if (!c->parts.empty()) {
    int rc = parts_fork(c);
    for (size_t k = 0; k < c->parts.size() && rc == GENGA_OK; ++k) rc = genga_step(c->parts[k], n_steps);
    return rc == GENGA_OK ? parts_join(c) : rc;
  }
  if (!c->gexec) {
    int rc = build_graph(c);
    if (rc != GENGA_OK) return rc;
  }
  if (c->batched && c->steps_per_launch > 1) {
    for (int k = 0; k < n_steps / c->steps_per_launch; ++k) CK(cudaGraphLaunch(c->gexec, c->stream));
    for (int k = 0; k < n_steps % c->steps_per_launch; ++k) CK(cudaGraphLaunch(c->gexec1, c->stream));
    return GENGA_OK;
  }
  for (int k = 0; k < n_steps; ++k) CK(cudaGraphLaunch(c->gexec, c->stream));
  return GENGA_OK;
}

int genga_sync(genga_ctx *c) {
  if (!c) return GENGA_EINVAL;
  if (!c->parts.empty()) {
    int st = 0;
    CK(cudaStreamSynchronize(c->stream));
    for (genga_ctx *p : c->parts) {
      const int r = genga_sync(p);
      if (r < 0) return r;
      st |= r;
    }
    return st;
  }
  CK(cudaStreamSynchronize(c->stream));
  int st = 0;
  CK(cudaMemcpy(&st, c->S.status, sizeof(int), cudaMemcpyDeviceToHost));
  return st;
}

int genga_set_state(genga_ctx *c, const double *x, const double *v) {
  if (!c || !x || !v) return GENGA_EINVAL;
  if (c->batched || c->tpmode) return GENGA_EINVAL;
  const size_t nn = (size_t)c->n + 1;
  cudaStream_t st = c->stream;
  CK(cudaMemcpyAsync(c->sx, x, 3 * nn * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(c->sv, v, 3 * nn * sizeof(double), cudaMemcpyHostToDevice, st));
  // masses, radii and live flags stay as they are on the device
  launch_from_helio(c->S, c->P, c->sx, c->sv, nullptr, nullptr, st);
  CK(cudaGetLastError());
  return first_kick(c);
}

int genga_get_state(genga_ctx *c, double *x, double *v, double *m, double *R, int *alive) {
  if (!c) return GENGA_EINVAL;
  if (c->batched) return GENGA_EINVAL;
  const size_t nn = (size_t)c->n + 1;
  cudaStream_t st = c->stream;
  launch_to_helio(c->S, c->P, x ? c->sx : nullptr, v ? c->sv : nullptr, m ? c->sm : nullptr,
                  R ? c->sR : nullptr, alive ? c->salive : nullptr, st);
  CK(cudaGetLastError());
  if (x) CK(cudaMemcpyAsync(x, c->sx, 3 * nn * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (v) CK(cudaMemcpyAsync(v, c->sv, 3 * nn * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (m) CK(cudaMemcpyAsync(m, c->sm, nn * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (R) CK(cudaMemcpyAsync(R, c->sR, nn * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (alive) CK(cudaMemcpyAsync(alive, c->salive, nn * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return GENGA_OK;
}

int genga_energy(genga_ctx *c, double *E, double *U) {
  if (!c) return GENGA_EINVAL;
  if (c->batched) return GENGA_EINVAL;
  cudaStream_t st = c->stream;
  launch_energy(c->S, c->P, c->scratch, c->sE, st);
  CK(cudaGetLastError());
  double e = 0.0, u = 0.0;
  CK(cudaMemcpyAsync(&e, c->sE, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&u, c->S.U, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (E) *E = e;
  if (U) *U = u;
  return GENGA_OK;
}

int genga_encounters(genga_ctx *c, int substep, int *pairs, int cap, int *n_pairs) {
  if (!c || cap < 0 || c->batched) return GENGA_EINVAL;
  if (substep < 0) substep = c->nsub - 1;
  if (substep >= c->nsub) return GENGA_EINVAL;
  cudaStream_t st = c->stream;
  launch_bitmap_pairs(c->S.ebm + (size_t)substep * c->S.npad * c->S.W, c->S.npad, c->S.W, c->spairs,
                      (int)c->pair_cap, c->scount, st);
  CK(cudaGetLastError());
  int cnt = 0;
  CK(cudaMemcpyAsync(&cnt, c->scount, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (n_pairs) *n_pairs = cnt;
  const int ncopy = cnt < cap ? cnt : cap;
  if (pairs && ncopy > 0) {
    CK(cudaMemcpy(pairs, c->spairs, 2 * (size_t)ncopy * sizeof(int), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 2 * ncopy; ++k) pairs[k] += 1;  // the central mass is body 0
  }
  return cnt > cap ? GENGA_ECAP : GENGA_OK;
}

int genga_tp_encounters(genga_ctx *c, int *pairs, int cap, int *n_pairs) {
  if (!c || !c->tpmode || cap < 0 || (cap > 0 && !pairs)) return GENGA_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  std::vector<unsigned> em(c->T.n);
  CK(cudaMemcpy(em.data(), c->T.emask, em.size() * sizeof(unsigned), cudaMemcpyDeviceToHost));
  int cnt = 0;
  for (int i = 0; i < c->T.n; ++i)
    for (unsigned bits = em[i]; bits; bits &= bits - 1) {
      const int j = __builtin_ctz(bits);
      if (cnt < cap) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j + 1; }  // the central mass is body 0
      cnt++;
    }
  if (n_pairs) *n_pairs = cnt;
  return cnt > cap ? GENGA_ECAP : GENGA_OK;
}

int genga_batch_encounters(genga_ctx *c, int *pairs, int cap, int *n_pairs) {
  if (!c || !c->batched || cap < 0 || (cap > 0 && !pairs)) return GENGA_EINVAL;
  if (!c->parts.empty()) {  // part by part: the parts' body ranges ascend, so the list stays sorted
    int tot = 0;
    for (size_t k = 0; k < c->parts.size(); ++k) {
      int cnt = 0;
      int rc = genga_batch_encounters(c->parts[k], nullptr, 0, &cnt);
      if (rc != GENGA_OK && rc != GENGA_ECAP) return rc;
      std::vector<int> pr(2 * (size_t)cnt);
      if (cnt > 0 && (rc = genga_batch_encounters(c->parts[k], pr.data(), cnt, &cnt)) != GENGA_OK) return rc;
      for (int q = 0; q < cnt; ++q, ++tot)
        if (tot < cap) {
          pairs[2 * tot] = pr[2 * q] + c->part_body0[k];
          pairs[2 * tot + 1] = pr[2 * q + 1] + c->part_body0[k];
        }
    }
    if (n_pairs) *n_pairs = tot;
    return tot > cap ? GENGA_ECAP : GENGA_OK;
  }
  CK(cudaStreamSynchronize(c->stream));
  std::vector<unsigned long long> em(c->n);
  CK(cudaMemcpy(em.data(), c->S.emask, em.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  std::vector<std::pair<int, int>> out;
  for (int k = 0; k < c->nsys; ++k)
    for (int i = c->start_h[k]; i < c->start_h[k + 1]; ++i)
      for (unsigned long long bits = em[i]; bits; bits &= bits - 1) {
        const int j = c->start_h[k] + __builtin_ctzll(bits);
        const int a = c->perm_h[i], b = c->perm_h[j];
        out.emplace_back(a < b ? a : b, a < b ? b : a);
      }
  std::sort(out.begin(), out.end());
  const int cnt = (int)out.size();
  for (int q = 0; q < cnt && q < cap; ++q) { pairs[2 * q] = out[q].first; pairs[2 * q + 1] = out[q].second; }
  if (n_pairs) *n_pairs = cnt;
  return cnt > cap ? GENGA_ECAP : GENGA_OK;
}

int genga_status(genga_ctx *c, int *code, long long *detail) {
  if (!c) return GENGA_EINVAL;
  if (!c->parts.empty()) {  // status bits of any part; counters summed, the step count once
    int st = 0;
    long long sum[NCOUNTERS] = {};
    for (genga_ctx *p : c->parts) {
      int cp = 0;
      long long d[NCOUNTERS];
      const int rc = genga_status(p, &cp, d);
      if (rc != GENGA_OK) return rc;
      st |= cp;
      for (int q = 0; q < NCOUNTERS; ++q) sum[q] = q == C_STEPS ? std::max(sum[q], d[q]) : sum[q] + d[q];
    }
    if (code) *code = st;
    if (detail) memcpy(detail, sum, sizeof(sum));
    return GENGA_OK;
  }
  CK(cudaStreamSynchronize(c->stream));
  int st = 0;
  CK(cudaMemcpy(&st, c->S.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (code) *code = st;
  if (detail) CK(cudaMemcpy(detail, c->S.counters, NCOUNTERS * sizeof(long long), cudaMemcpyDeviceToHost));
  return GENGA_OK;
}

int genga_set_profiling(genga_ctx *c, int on) {
  if (!c || c->batched || c->tpmode) return GENGA_EINVAL;
  if (on && !c->nkev) {
    for (int k = 0; k < 2 * c->nsub; ++k) CK(cudaEventCreate(&c->kev[k]));
    c->nkev = 2 * c->nsub;
  }
  c->profiling = on != 0;
  drop_graph(c);
  return GENGA_OK;
}

int genga_kick_time(genga_ctx *c, float *ms, int *launches) {
  if (!c || !ms || !c->profiling || !c->nkev) return GENGA_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  float tot = 0.0f;
  for (int j = 0; j < c->nsub; ++j) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, c->kev[2 * j], c->kev[2 * j + 1]));
    tot += t;
  }
  *ms = tot;
  if (launches) *launches = c->nsub;
  return GENGA_OK;
}

int genga_launch_count(genga_ctx *c, int *kernels_per_step) {
  if (!c || !kernels_per_step) return GENGA_EINVAL;
  if (!c->parts.empty()) {  // the parts' graphs together
    int tot = 0;
    for (genga_ctx *p : c->parts) {
      int k = 0;
      const int rc = genga_launch_count(p, &k);
      if (rc != GENGA_OK) return rc;
      tot += k;
    }
    *kernels_per_step = tot;
    return GENGA_OK;
  }
  if (!c->gexec) {
    int rc = build_graph(c);
    if (rc != GENGA_OK) return rc;
  }
  size_t nn = 0;
  CK(cudaGraphGetNodes(c->graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CK(cudaGraphGetNodes(c->graph, nodes.data(), &nn));
  int k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) k++;
  }
  *kernels_per_step = k;  // batched mode: per launch of steps_per_launch steps
  return GENGA_OK;
}

void genga_free(genga_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (genga_ctx *p : c->parts) genga_free(p);
  for (cudaEvent_t e : c->part_ev) cudaEventDestroy(e);
  drop_graph(c);
  for (int k = 0; k < c->nkev; ++k) cudaEventDestroy(c->kev[k]);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_join2) cudaEventDestroy(c->ev_join2);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->side2) cudaStreamDestroy(c->side2);
  if (c->ev_tab) cudaEventDestroy(c->ev_tab);
  if (c->ev_tabj) cudaEventDestroy(c->ev_tabj);
  if (c->side3) cudaStreamDestroy(c->side3);
  c->mem.release();
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
}

// ------------------------------------------------------------------------------------------
// Phase entry points
// ------------------------------------------------------------------------------------------
static int phase_sim(Sim &S, DevMem &mem, int n) {
  if (n < 1 || n > NMAX) return GENGA_EINVAL;
  if (!alloc_sim(S, mem, n, 1)) { mem.release(); return GENGA_ENOMEM; }
  return GENGA_OK;
}

static int phase_finish(DevMem &mem, cudaStream_t st, int rc) {
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == GENGA_OK) rc = GENGA_ECUDA;
  if (cudaGetLastError() != cudaSuccess && rc == GENGA_OK) rc = GENGA_ECUDA;
  mem.release();
  return rc;
}

// copy a [3 n] SoA array into a [3 npad] SoA array (or back)
static cudaError_t soa_copy(double *dst, size_t dpitch, const double *src, size_t spitch, int n, cudaStream_t st) {
  return cudaMemcpy2DAsync(dst, dpitch * sizeof(double), src, spitch * sizeof(double), n * sizeof(double), 3,
                           cudaMemcpyDeviceToDevice, st);
}

int genga_phase_rcrit(int n, double G, double m0, double n1, double n2, double tau_abs, const double *m,
                      const int *alive, const double *x, const double *v, double *rc, void *stream) {
  if (!m || !alive || !x || !v || !rc || !(G > 0.0) || !(m0 > 0.0)) return GENGA_EINVAL;
  Sim S; DevMem mem;
  int r = phase_sim(S, mem, n);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  genga_params prm; genga_default_params(&prm); prm.n1 = n1; prm.n2 = n2;
  DevParams P = make_params(G, m0, prm);
  launch_soa_setup(S, P, m, alive, x, v, nullptr, n, st);
  launch_rcrit(S, P, tau_abs, 0, st);
  cudaMemcpyAsync(rc, S.rc, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  return phase_finish(mem, st, GENGA_OK);
}

int genga_phase_kick(int n, double G, double pc, int kmode, int precise_div, const double *m, const int *alive,
                     const double *x, const double *rc, double *a, int *cand, int cap, int *ncand, void *stream) {
  if (!m || !alive || !x || !rc || !a || !ncand || cap < 0 || !(G > 0.0) || !(pc >= 1.0)) return GENGA_EINVAL;
  Sim S; DevMem mem;
  int r = phase_sim(S, mem, n);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  genga_params prm; genga_default_params(&prm); prm.pc = pc; prm.kmode = kmode;
  DevParams P = make_params(G, 1.0, prm);
  double *aout = mem.get<double>(3 * (size_t)S.npad);
  int *dcnt = mem.get<int>(1);
  int *tmp = mem.get<int>(2 * ((size_t)S.npad * (S.npad - 1) / 2 + 1));
  if (mem.err != cudaSuccess) { mem.release(); return GENGA_ENOMEM; }
  launch_soa_setup(S, P, m, alive, x, nullptr, rc, n, st);
  launch_kick(S, P, false, precise_div != 0, st);
  launch_fin(S, P, FIN_INIT, 0.0, 0.0, aout, st);
  soa_copy(a, n, aout, S.npad, n, st);
  launch_bitmap_pairs(S.cbm, S.npad, S.W, tmp, S.npad * (S.npad - 1) / 2 + 1, dcnt, st);
  int cnt = 0;
  cudaMemcpyAsync(&cnt, dcnt, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  *ncand = cnt;
  const int ncopy = cnt < cap ? cnt : cap;
  if (cand && ncopy > 0) cudaMemcpyAsync(cand, tmp, 2 * (size_t)ncopy * sizeof(int), cudaMemcpyDeviceToDevice, st);
  return phase_finish(mem, st, cnt > cap ? GENGA_ECAP : GENGA_OK);
}

int genga_phase_kepler(int n, double mu, double dt, int maxit, const int *alive, double *x, double *v, int *fail,
                       void *stream) {
  if (n < 1 || !alive || !x || !v || !fail || !(mu > 0.0) || maxit < 1) return GENGA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  launch_kepler_phase(n, mu, dt, maxit, alive, x, v, fail, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return GENGA_OK;
}

int genga_phase_encounters(int n, const int *alive, const double *x0, const double *v0, const double *x1,
                           const double *v1, const double *rc, const int *cand, int ncand, double tau, int *out,
                           int cap, int *nout, void *stream) {
  if (!alive || !x0 || !v0 || !x1 || !v1 || !rc || (ncand > 0 && !cand) || ncand < 0 || !nout || cap < 0)
    return GENGA_EINVAL;
  Sim S; DevMem mem;
  int r = phase_sim(S, mem, n);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  genga_params prm; genga_default_params(&prm);
  DevParams P = make_params(1.0, 1.0, prm);
  int *dcnt = mem.get<int>(1);
  int *tmp = mem.get<int>(2 * ((size_t)S.npad * (S.npad - 1) / 2 + 1));
  if (mem.err != cudaSuccess) { mem.release(); return GENGA_ENOMEM; }
  launch_soa_setup(S, P, nullptr, alive, x1, v1, rc, n, st);
  soa_copy(S.x0, S.npad, x0, n, n, st);
  soa_copy(S.v0, S.npad, v0, n, n, st);
  launch_pairs_to_bitmap(S, cand, ncand, st);
  launch_encounter(S, tau, S.ebm, st);
  launch_bitmap_pairs(S.ebm, S.npad, S.W, tmp, S.npad * (S.npad - 1) / 2 + 1, dcnt, st);
  int cnt = 0;
  cudaMemcpyAsync(&cnt, dcnt, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  *nout = cnt;
  const int ncopy = cnt < cap ? cnt : cap;
  if (out && ncopy > 0) cudaMemcpyAsync(out, tmp, 2 * (size_t)ncopy * sizeof(int), cudaMemcpyDeviceToDevice, st);
  return phase_finish(mem, st, cnt > cap ? GENGA_ECAP : GENGA_OK);
}

int genga_phase_groups(int n, const int *pairs, int npairs, const int *single, int *group_start, int *members,
                       int *ngroups, void *stream) {
  if (npairs < 0 || (npairs > 0 && !pairs) || !group_start || !members || !ngroups) return GENGA_EINVAL;
  Sim S; DevMem mem;
  int r = phase_sim(S, mem, n);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if ((size_t)npairs > (size_t)S.npad * (S.npad - 1) / 2 + 1) { mem.release(); return GENGA_EINVAL; }
  launch_copy_edges(S, pairs, npairs, st);
  if (single) launch_single_to_fail(S, single, st);
  launch_group(S, st);
  int ng = 0;
  cudaMemcpyAsync(&ng, S.ngroups, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  *ngroups = ng;
  int nm = 0;
  cudaMemcpyAsync(&nm, S.gstart + ng, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  cudaMemcpyAsync(group_start, S.gstart, (ng + 1) * sizeof(int), cudaMemcpyDeviceToDevice, st);
  if (nm > 0) cudaMemcpyAsync(members, S.gmem, nm * sizeof(int), cudaMemcpyDeviceToDevice, st);
  return phase_finish(mem, st, GENGA_OK);
}

int genga_phase_bs(int n, double G, double m0, double tau, double bs_eps, int bs_kmax, int bs_max_halvings,
                   int kmode, int collisions, int ngroups, const int *group_start, const int *members,
                   const double *rc, double *m, double *R, int *alive, double *x, double *v, double *U, void *stream) {
  if (ngroups < 0 || (ngroups > 0 && (!group_start || !members)) || !rc || !m || !R || !alive || !x || !v || !U ||
      !(G > 0.0) || !(m0 > 0.0) || bs_kmax < 2 || bs_kmax > BS_LEVELS)
    return GENGA_EINVAL;
  Sim S; DevMem mem;
  int r = phase_sim(S, mem, n);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  genga_params prm; genga_default_params(&prm);
  prm.bs_eps = bs_eps; prm.bs_kmax = bs_kmax; prm.bs_max_halvings = bs_max_halvings; prm.kmode = kmode;
  prm.collisions = collisions;
  DevParams P = make_params(G, m0, prm);
  bs_init_constants();
  launch_soa_setup(S, P, m, alive, x, v, rc, n, st);
  cudaMemcpyAsync(S.R, R, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  soa_copy(S.x0, S.npad, x, n, n, st);
  soa_copy(S.v0, S.npad, v, n, n, st);
  cudaMemcpyAsync(S.ngroups, &ngroups, sizeof(int), cudaMemcpyHostToDevice, st);
  // the main mode's routing by size: one CTA per group below 5 members, a cluster per group of 5 to
  // BS_GMAX members, the grid-wide kernel above
  std::vector<int> gs(ngroups + 1, 0), big;
  if (ngroups > 0) {
    cudaMemcpyAsync(gs.data(), group_start, (ngroups + 1) * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    const int nm = gs[ngroups];
    if (nm < 0 || nm > n) { mem.release(); return GENGA_EINVAL; }
    cudaMemcpyAsync(S.gstart, group_start, (ngroups + 1) * sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (nm > 0) cudaMemcpyAsync(S.gmem, members, nm * sizeof(int), cudaMemcpyDeviceToDevice, st);
    for (int k = 0; k < ngroups; ++k)
      if (gs[k + 1] - gs[k] >= 5) big.push_back(k);
  }
  const int nbig = (int)big.size();
  cudaMemcpyAsync(S.nbig, &nbig, sizeof(int), cudaMemcpyHostToDevice, st);
  if (nbig > 0) cudaMemcpyAsync(S.big, big.data(), nbig * sizeof(int), cudaMemcpyHostToDevice, st);
  bs_cluster_init_constants();
  bs_grid_init_constants();
  launch_bs(S, P, tau, 2 * num_sms(), st, 5);
  launch_bs_cluster(S, P, tau, 5, bs_cluster_grid(), st);
  launch_bs_grid(S, P, tau, BS_GMAX + 1, bs_grid_blocks(), st);
  cudaStreamSynchronize(st);  // the host vectors above outlive the copies
  soa_copy(x, n, S.x, S.npad, n, st);
  soa_copy(v, n, S.v, S.npad, n, st);
  cudaMemcpyAsync(m, S.m, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(R, S.R, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(alive, S.alive, n * sizeof(int), cudaMemcpyDeviceToDevice, st);
  int status = 0;
  cudaMemcpyAsync(U, S.U, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&status, S.status, sizeof(int), cudaMemcpyDeviceToHost, st);
  int rc2 = phase_finish(mem, st, GENGA_OK);
  return rc2 != GENGA_OK ? rc2 : status;
}

int genga_phase_energy(int n, double G, double m0, const double *m, const int *alive, const double *x,
                       const double *v, double *E, void *stream) {
  if (!m || !alive || !x || !v || !E || !(G > 0.0) || !(m0 > 0.0)) return GENGA_EINVAL;
  Sim S; DevMem mem;
  int r = phase_sim(S, mem, n);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  genga_params prm; genga_default_params(&prm);
  DevParams P = make_params(G, m0, prm);
  double *scratch = mem.get<double>((size_t)S.nt * S.nt), *dE = mem.get<double>(1);
  if (mem.err != cudaSuccess) { mem.release(); return GENGA_ENOMEM; }
  launch_soa_setup(S, P, m, alive, x, v, nullptr, n, st);
  launch_energy(S, P, scratch, dE, st);
  cudaMemcpyAsync(E, dE, sizeof(double), cudaMemcpyDeviceToHost, st);
  return phase_finish(mem, st, GENGA_OK);
}

int genga_fp64_probe(int iters, double *tflops, float *ms, void *stream) {
  if (iters < 1 || !tflops) return GENGA_EINVAL;
  double *scratch = nullptr;
  CK(cudaMalloc(&scratch, sizeof(double)));
  const double f = fp64_probe_flops(iters, 4 * num_sms(), ms, (cudaStream_t)stream, scratch);
  cudaError_t e = cudaGetLastError();
  cudaFree(scratch);
  if (e != cudaSuccess) return GENGA_ECUDA;
  *tflops = f / 1e12;
  return GENGA_OK;
}

int genga_phase_mathcheck(int n, int which, const double *in, double *out, void *stream) {
  if (n < 0 || !in || !out || which < 0 || which > 2) return GENGA_EINVAL;
  if (n == 0) return GENGA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  launch_mathcheck(n, which, in, out, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return GENGA_OK;
}

}  // extern "C"
