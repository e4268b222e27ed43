// genga_launch.h -- host-side launchers of the sm_103a kernels (one per kernel family).
#pragma once
#include <cuda_runtime.h>

#include "genga_dev.cuh"

namespace genga {

// FIN_CLOSE_ALL: a closing kick whose pair kernel weighed every pair (no near pairs, far field kept)
enum FinMode { FIN_CLOSE = 0, FIN_OPEN = 1, FIN_INIT = 2, FIN_CLOSE_ALL = 3 };

// kick.cu
void launch_rcrit(const Sim &S, const DevParams &P, double tau_abs, int check_reuse, cudaStream_t st);
// full: every pair with its changeover weight, no candidates recorded; runs only when the opening
// kick must be recomputed, unless force (then always, also recording the momentum for the Sun drift)
void launch_kick(const Sim &S, const DevParams &P, bool full, bool precise, cudaStream_t st, bool force = false);
void launch_fin(const Sim &S, const DevParams &P, FinMode mode, double h1, double h2, double *aout,
                cudaStream_t st);
void launch_hc(const Sim &S, double hcm, cudaStream_t st);
int kick_grid(const Sim &S);

// step.cu
void launch_drift(const Sim &S, const DevParams &P, double tau, double hcm1, double hcm2,
                  int substep, cudaStream_t st);
// keep: leave the candidate set in place for the next substep (literal higher-order prechecker)
void launch_encounter(const Sim &S, double tau, unsigned *ebm, cudaStream_t st, bool keep = false);
void launch_group(const Sim &S, cudaStream_t st, int gbig = BS_GMAX + 1);  // gbig: size threshold of S.big
// the two in one launch (the last CTA of the encounter test groups the edges of all)
void launch_encounter_group(const Sim &S, double tau, unsigned *ebm, cudaStream_t st, bool keep, int gbig);
void launch_kepler_phase(int n, double mu, double dt, int maxit, const int *alive, double *x, double *v,
                         int *fail, cudaStream_t st);
void launch_pairs_to_bitmap(const Sim &S, const int *pairs, int npairs, cudaStream_t st);
void launch_bitmap_pairs(const unsigned *bm, int npad, int W, int *out, int cap, int *count, cudaStream_t st);
void launch_single_to_fail(const Sim &S, const int *single, cudaStream_t st);
void launch_copy_edges(const Sim &S, const int *pairs, int npairs, cudaStream_t st);

// eject.cu: ejections (and the batched stop below nmin) at the end of a step
void launch_eject(const Sim &S, const DevParams &P, cudaStream_t st);
void launch_b_eject(const Sim &S, const DevParams &P, cudaStream_t st);
void launch_tp_eject(const TPSet &T, const DevParams &P, cudaStream_t st);
// bs.cu
void bs_init_constants();  // once per device, before any capture
// Groups of at least gsplit members are skipped (left to the cluster or the wide kernel); without
// gsplit every group above BS_GMAX members is reported (GROUP_TOO_LARGE).
void launch_bs(const Sim &S, const DevParams &P, double tau, int max_groups, cudaStream_t st,
               int gsplit = 0x7fffffff, int gmin = 1);
// groups of BS_GMAX + 1 .. BS_GWIDE members, one 512-thread CTA each (larger ones reported): batched
// queue 3, else the large-group list of the grouping kernel
constexpr int BS_GWIDE = 64;
constexpr int BS_WIDE_THREADS = 512;
void launch_bs_wide(const Sim &S, const DevParams &P, double tau, int blocks, cudaStream_t st);
// batched mode: groups of 3 .. BS_SMALL members from BS queue 1, 128-thread CTAs (launch_bs takes
// queue 2 there)
void launch_bs_small(const Sim &S, const DevParams &P, double tau, int blocks, cudaStream_t st);
// groups of one or two members, one warp each (no adjoint recording)
void launch_bs_pair(const Sim &S, const DevParams &P, double tau, int blocks, cudaStream_t st);
// bs_grid.cu: the groups of the large-group list with gmin or more members, one after another on
// the whole GPU (single-system modes; needs Sim::gb)
void bs_grid_init_constants();  // once per device, before any capture
int bs_grid_blocks();
void launch_bs_grid(const Sim &S, const DevParams &P, double tau, int gmin, int blocks, cudaStream_t st);
// bs_cluster.cu: groups of gmin .. BS_GMAX members, one cluster of 8 CTAs (one per level) each
void bs_cluster_init_constants();  // once per device, before any capture
int bs_cluster_grid();
void launch_bs_cluster(const Sim &S, const DevParams &P, double tau, int gmin, int grid, cudaStream_t st);

// batch_persist.cu: the batched step as one persistent launch (a CTA per system at a time); the
// step number of the reports is read from step_base (a device int the launch advances by nsteps)
int b_persist_init();  // once per device, before any capture; returns CTAs per SM that fit
void launch_b_persist(const Sim &S, const DevParams &P, double dt, const double *w, int nsub, int nsteps,
                      int *step_base, int *queue, int blocks, cudaStream_t st);

// batch.cu
void launch_b_rcrit(const Sim &S, const DevParams &P, double tau_abs, int check, cudaStream_t st);
void launch_b_kick(const Sim &S, const DevParams &P, FinMode mode, double h1, double h2, int split, int block,
                   cudaStream_t st);
void launch_b_momentum(const Sim &S, double *out, cudaStream_t st);
void launch_b_drift(const Sim &S, const DevParams &P, double tau, double h1, double h2, int substep, cudaStream_t st);
void launch_b_encounter(const Sim &S, double tau, cudaStream_t st);
void launch_b_group(const Sim &S, cudaStream_t st);
void launch_b_hc(const Sim &S, double h, cudaStream_t st);
void launch_b_from_helio(const Sim &S, const DevParams &P, const int *perm, const double *xh, const double *vh,
                         const double *m_in, const double *R_in, int keep, cudaStream_t st);
void launch_b_to_helio(const Sim &S, const int *perm, double *xh, double *vh, double *m_out, double *R_out,
                       int *alive_out, cudaStream_t st);
void launch_b_energy(const Sim &S, const DevParams &P, const int *sys_user, double *E, cudaStream_t st);

// tp.cu
int tp_init_constants();  // Neville factors of the TP Bulirsch-Stoer (call outside stream capture)
void launch_tp_rcrit(const TPSet &T, const DevParams &P, double tau_abs, int check, cudaStream_t st);
// the first kick after a new state: far field and candidates of every TP, no velocity change
void launch_tp_kick(const Sim &S, const TPSet &T, const DevParams &P, cudaStream_t st);
// the step's start for the TPs in one pass: rcrit (reuse test), opening kick, first Sun drift, Kepler drift
void launch_tp_open_drift(const Sim &S, const TPSet &T, const DevParams &P, double tau_abs, double h1, double tau,
                          double hcm1, cudaStream_t st);
void launch_tp_drift(const Sim &S, const TPSet &T, const DevParams &P, double tau, double hcm1, double hcm2, cudaStream_t st);
void launch_planet_table(const Sim &S, const TPSet &T, const DevParams &P, double tau, cudaStream_t st);
void launch_tp_encounter(const Sim &S, const TPSet &T, double tau, int blocks, cudaStream_t st);
// the BS pass of a substep and the closing kick of every TP (v += (h1 + h2) a; hcm_last != 0: the
// step's last Sun drift)
void launch_tp_bs(const Sim &S, const TPSet &T, const DevParams &P, double tau, double h1, double h2, double hcm_last,
                  int blocks, cudaStream_t st);
void launch_tp_from_helio(const TPSet &T, int nmass, const double *mh, const double *vmh, const double *xh,
                          const double *vh, const double *Rh, int keep, cudaStream_t st);
void launch_tp_to_helio(const Sim &S, const TPSet &T, const DevParams &P, double *xh, double *vh, int *alive,
                        cudaStream_t st);

// io.cu
void launch_from_helio(const Sim &S, const DevParams &P, const double *xh, const double *vh,
                       const double *m_in, const double *R_in, cudaStream_t st);
void launch_to_helio(const Sim &S, const DevParams &P, double *xh, double *vh, double *m_out,
                     double *R_out, int *alive_out, cudaStream_t st);
void launch_energy(const Sim &S, const DevParams &P, double *scratch, double *E, cudaStream_t st);
void launch_mathcheck(int n, int which, const double *in, double *out, cudaStream_t st);
// FP64 FMA throughput of the device (flop/s; FMA = 2), timed with events around one launch
double fp64_probe_flops(int iters, int blocks, float *ms, cudaStream_t st, double *scratch);
void launch_soa_setup(const Sim &S, const DevParams &P, const double *m, const int *alive,
                      const double *x, const double *v, const double *rc, int n, cudaStream_t st);
void launch_soa_out(const Sim &S, double *x, double *v, int n, cudaStream_t st);

}  // namespace genga
