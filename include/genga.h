/*
 * genga.h -- C ABI of the GB300 (sm_103a) FP64 implementation of the hybrid symplectic N-body
 * step of Grimm & Stadel, "The GENGA Code" (arXiv:1404.2324).
 *
 * The library integrates N bodies around a central mass m0 with the splitting H = H_A + H_B + H_C
 * in democratic coordinates (Sect. 2.1, Eqs. Ha, Hb, Hc): a kick weighted by the changeover
 * function K(r_ij) (Eq. Hb) with the prechecker, the Sun drift (Eq. Hc), the Kepler drift with
 * Gauss' f and g functions (Eq. fg) in universal variables, the close-encounter search with the
 * cubic Hermite interpolant (Eqs. teqn, polydelta), encounter grouping (Appendix), and
 * Bulirsch-Stoer integration of the groups with perfect merging (Sect. 3.2), composed to 2nd order
 * (Eq. z1) or Yoshida's 4th/6th order (Sect. 2.3).
 *
 * Conventions
 *   - All floating point is IEEE binary64 (double).
 *   - Bodies: index 0 of every host array passed to genga_init / genga_get_state is the central
 *     mass (its position and velocity are ignored on input and returned as zero); bodies 1..n-1
 *     orbit it. Positions are heliocentric, velocities heliocentric on input and output (the
 *     library converts to barycentric "democratic" velocities internally, Sect. 2.1).
 *   - Host arrays are AoS row-major: x[3*i + c]. The caller owns every host buffer it passes; the
 *     context owns all device memory it allocates and frees it in genga_free.
 *   - "Phase" entry points (genga_phase_*) take DEVICE pointers in SoA layout (component-major:
 *     x[c*n + i]) and a cudaStream_t passed as void*; they exist so that each step of the method can
 *     be checked on its own. They allocate their own temporary device memory.
 *   - Return codes: 0 success; negative = invalid argument or CUDA failure, detected on the host
 *     before anything is launched (or reported by the CUDA runtime); positive = numerical status
 *     raised by the kernels (see GENGA_ST_*), read back by genga_status / genga_sync. Kernels
 *     never trap: every device loop is bounded and reports through the status word.
 */
#ifndef GENGA_H
#define GENGA_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error and status codes ---- */
#define GENGA_OK 0
#define GENGA_EINVAL (-1)      /* bad argument (NULL, n out of range, dt = 0, order not 2/4/6, NaN) */
#define GENGA_ECUDA (-2)       /* a CUDA runtime call failed */
#define GENGA_ENOMEM (-3)      /* device allocation failed */
#define GENGA_ECAP (-4)        /* output capacity too small */
#define GENGA_ESIZE (-5)       /* n above the fixed maximum of genga_kick_noalloc (1024) */

/* status bits accumulated on the device (genga_status); none of them stops the integration */
#define GENGA_ST_KEPLER_FALLBACK 1   /* a Kepler solve did not converge; that body went to BS */
#define GENGA_ST_BS_FAILED 2         /* a BS group exceeded its step-halving cap (state kept) */
#define GENGA_ST_REUSE_FULLKICK 4    /* rcrit grew past pc*rcrit_old: the opening kick was recomputed */
#define GENGA_ST_GROUP_TOO_LARGE 8   /* a group above the size its mode integrates (64 members in the batched
                                        mode and the differentiable engine; its state kept, not integrated) */
#define GENGA_ST_UNION_ROUNDS 16     /* grouping did not reach its fixpoint within its round cap */
#define GENGA_ST_RECORD_OVERFLOW 32  /* adjoint engine: a recording buffer was too small (gradient invalid) */
#define GENGA_ST_EJECT_OVERFLOW 64   /* more than 4096 ejection records (later ones dropped), or more than
                                        1024 bodies out of bounds in one step (the rest leave next step) */
#define GENGA_ST_GRID_TIMEOUT 128    /* the grid-wide BS of a group above 32 members gave up waiting at one of
                                        its grid barriers (its group keeps the state it had) */
#define GENGA_ST_COLL_OVERFLOW 256   /* more than 4096 collision reports (later ones dropped; mergers still happen) */

/* modes of genga_init (Sect. 3): main mode with up to 2048 massive bodies */
#define GENGA_MODE_MASSIVE 0

typedef struct genga_ctx genga_ctx;

/* Method parameters (Sect. 2.1 Eq. rcrit, Sect. 2.2 prechecker, Sect. 3.2 BS). */
typedef struct genga_params {
  double n1;            /* Hill-radius factor of Eq. rcrit (paper default 3) */
  double n2;            /* velocity factor of Eq. rcrit (paper default 0.4) */
  double pc;            /* precheck factor: candidate if r < pc * rcrit (paper: 3) */
  double bs_eps;        /* BS relative tolerance (1e-12) */
  int bs_kmax;          /* deepest BS extrapolation level, sequence n_k = 2k (8, at most 8) */
  int bs_max_halvings;  /* consecutive BS step halvings before a group is declared failed (30) */
  int kepler_maxit;     /* iteration cap of the universal Kepler solve (30) */
  int kmode;            /* 0: K multiplies the Newtonian pair force; 1: exact gradient of H_B */
  int collisions;       /* 1: perfect merging on contact (Sect. 3.2, Collisions) */
  int precise_div;      /* 1: kick uses IEEE sqrt and division; 0: refined reciprocal square root */
  /* Ejections (Sect. 3.2): at the end of every step a body farther than rcut from its central mass
   * or closer than rcut_sun is removed (a ghost, as after a merger), its heliocentric state
   * recorded (genga_ejections) and the energy it takes away booked into U; test particles are
   * removed by the same limits. 0 switches a limit off (the default); rcut > rcut_sun when both. */
  double rcut;
  double rcut_sun;
  /* Batched mode (Sect. 3.4, Nmin): a system left with fewer than nmin live bodies at the end of a
   * step is stopped, all its bodies removed (energy booked into U). 0: off (the default). */
  int nmin;
  /* Higher orders (Sect. 2.3). 1 (the default): the closing kick of every substep prechecks and its
   * candidates feed the next substep's encounter search. 0: as the paper states it, the substeps
   * run the full scheme "but not the prechecker": only the closing kick of a full step prechecks and
   * its candidates serve every substep of the next step (main mode only; EINVAL elsewhere). */
  int precheck_substeps;
} genga_params;

/* Fills *p with the paper's defaults (n1 = 3, n2 = 0.4, pc = 3) and the library's BS/Kepler caps. */
int genga_default_params(genga_params *p);

/* Creates a context on the current CUDA device and uploads the initial state (Sect. 3, main mode).
 *   n        bodies including the central mass at index 0; 2 <= n <= 2049 (2048 orbiting bodies)
 *   masses   [n] masses (masses[0] = m0 > 0; orbiting masses >= 0)
 *   radii    [n] physical radii used for collisions (radii[0] ignored)
 *   x, v     [3n] heliocentric positions and velocities (row 0 ignored)
 *   G        gravitational constant; dt the step tau (sign gives the direction of time)
 *   order    2 (Eq. z1), 4 or 6 (Yoshida compositions, Sect. 2.3); mode GENGA_MODE_MASSIVE
 * The first step opens with the full pair kick (no stored far field yet), which also records the
 * precheck candidates of its first substep (Sect. 2.2). The host buffers are not retained. Returns 0
 * or a negative code; *ctx is NULL on failure. */
int genga_init(genga_ctx **ctx, int n, const double *masses, const double *radii, const double *x,
               const double *v, double G, double dt, int order, int mode);

/* Replaces the method parameters; the next genga_step opens with the full pair kick, as after
 * genga_init. */
int genga_set_params(genga_ctx *ctx, const genga_params *p);

/* Makes the context launch on the given cudaStream_t (NULL: the context's own stream). */
int genga_set_stream(genga_ctx *ctx, void *stream);

/* Enqueues n_steps full steps on the context's stream and returns without waiting. All branching
 * (kick reuse, encounters, groups, BS, mergers) is decided on the device. */
int genga_step(genga_ctx *ctx, int n_steps);

/* Waits for the context's stream; returns 0, a negative CUDA code, or the status bits. */
int genga_sync(genga_ctx *ctx);

/* Replaces positions and velocities (heliocentric, host, [3n] with row 0 ignored) of all bodies;
 * masses and radii stay. The next step opens with the full pair kick, as after genga_init. */
int genga_set_state(genga_ctx *ctx, const double *x, const double *v);

/* Copies the state back (waits for the stream). Any pointer may be NULL. x, v [3n] heliocentric;
 * m, R [n]; alive [n] (1 live, 0 ghost left by a merger; the central mass counts as live). */
int genga_get_state(genga_ctx *ctx, double *x, double *v, double *m, double *R, int *alive);

/* Total energy E of the live bodies in democratic coordinates (Sect. 4.1) and the internal
 * energy U booked by mergers (Sect. 3.2); E + U is the conserved quantity. Waits for the stream. */
int genga_energy(genga_ctx *ctx, double *E, double *U);

/* Confirmed close-encounter pairs (i < j, body indices with the central mass at 0, ascending) found
 * in a substep of the last step (substep -1: the last substep). *n_pairs receives the count;
 * returns GENGA_ECAP if cap < count (the first cap pairs are written). */
int genga_encounters(genga_ctx *ctx, int substep, int *pairs, int cap, int *n_pairs);

/* Ejections since the context was created (Sect. 3.2): *n receives their number; the first
 * min(*n, cap, 4096) records are written to rec [8 cap], each: body index (the caller's: central
 * mass at 0 in the single-system modes, the index into the concatenated bodies in the batched
 * mode), the step (1-based) at whose end it left, heliocentric x[3] and v[3] at that moment, in
 * ascending index within a step. Waits for the stream. */
int genga_ejections(genga_ctx *ctx, double *rec, int cap, int *n);

/* Collision reports since the context was created (Sect. 3.2, Collisions: positions, velocities and
 * spins of both bodies at the last time before the contact). *n receives the number of mergers; the
 * first min(*n, cap, 4096) reports are written to rec [24 cap], ordered by step, substep, time and
 * pair, each: [0] step (1-based), [1] substep of the composition (0-based), [2] time from that
 * substep's start to the start of the BS substep in which the contact was found, [3] body i, [4] body
 * j (i < j; the caller's indices as in genga_ejections), [5..7] x_i, [8..10] v_i, [11..13] spin_i,
 * [14..16] x_j, [17..19] v_j, [20..22] spin_j at that time (heliocentric positions, barycentric
 * velocities), [23] the body that survives (the heavier; equal masses: the smaller index). Waits
 * for the stream. */
int genga_collisions(genga_ctx *ctx, double *rec, int cap, int *n);

/* Spin angular momentum of every body (zero at creation). A merger gives the survivor the sum of
 * both spins and the pair's orbital angular momentum about its centre of mass, so orbital plus spin
 * angular momentum is conserved (Sect. 3.2, Collisions). Layout as the state: [3n] with the central
 * mass at row 0 (ignored on input, zero on output) in the single-system modes, [3N] flat in the
 * caller's order in the batched mode. Both wait for the stream. */
int genga_set_spin(genga_ctx *ctx, const double *spin);
int genga_get_spin(genga_ctx *ctx, double *spin);

/* Device status word: bits GENGA_ST_*; *detail receives counters (may be NULL): detail[0] steps,
 * [1] candidates, [2] encounters, [3] groups, [4] BS steps, [5] Kepler fallbacks, [6] mergers,
 * [7] full-kick recomputes (8 entries). Waits for the stream. */
int genga_status(genga_ctx *ctx, int *code, long long *detail);

/* Enables (1) or disables (0) CUDA-event timing of the pairwise kick kernels inside the captured
 * step graph (event-record nodes around each kick launch; the next genga_step recaptures). */
int genga_set_profiling(genga_ctx *ctx, int on);

/* Waits for the stream, then returns in *ms the summed device time of the pairwise kick launches
 * of the most recent step and in *launches their number (profiling must be on). */
int genga_kick_time(genga_ctx *ctx, float *ms, int *launches);

/* Number of kernel launches one step enqueues (kernel nodes of the captured step graph; captures
 * it if needed). Batched mode: the kernels of one launch of the batch's steps_per_launch steps
 * (the step graph of that many steps, or the persistent kernel and its step counter). */
int genga_launch_count(genga_ctx *ctx, int *kernels_per_step);

/* Frees the context and every device buffer it owns. */
void genga_free(genga_ctx *ctx);

/* ------------------------------------------------------------------------------------------ */
/* Test-particle mode (Sect. 3.3)                                                                */
/* ------------------------------------------------------------------------------------------ */

/* Creates a context with up to 32 massive bodies (arguments as genga_init, 2 <= n <= 33 including
 * the central mass) plus n_tp massless test particles: xt, vt [3 n_tp] heliocentric, Rt [n_tp]
 * physical radii (NULL: 0). Test particles feel the massive bodies (K-weighted kick with the
 * prechecker, the massive bodies' Sun drift, Kepler drift); a test particle with a confirmed planet
 * encounter is integrated alone by Bulirsch-Stoer in the field of m0 and the (1 - K) pull of the
 * planets it meets, which keep their Kepler paths; one that reaches a planet's surface is removed.
 * The massive bodies evolve exactly as without test particles (genga_get_state, genga_energy). */
int genga_init_tp(genga_ctx **ctx, int n, const double *masses, const double *radii, const double *x,
                  const double *v, double G, double dt, int order, int n_tp, const double *xt,
                  const double *vt, const double *Rt);

/* Test-particle state (heliocentric, host): xt, vt [3 n_tp], tp_alive [n_tp]; any may be NULL. */
int genga_get_state_tp(genga_ctx *ctx, double *xt, double *vt, int *tp_alive);

/* Confirmed (test particle, planet) encounter pairs of the last substep of the last step (Sect. 3.3):
 * pairs[2k] the particle's index, pairs[2k+1] the planet's body index (central mass at 0), ascending.
 * *n_pairs receives the count; returns GENGA_ECAP if cap < count (the first cap pairs written). */
int genga_tp_encounters(genga_ctx *ctx, int *pairs, int cap, int *n_pairs);

/* Test-particle counters since genga_init_tp (5 entries): detail[0] (TP, planet) candidate pairs
 * recorded by the closing kicks, [1] confirmed encounter pairs, [2] accepted BS substeps,
 * [3] particles removed on contact, [4] particles ejected (rcut, rcut_sun). */
int genga_tp_status(genga_ctx *ctx, long long *detail);

/* ------------------------------------------------------------------------------------------ */
/* Batched many-systems mode (Sect. 3.4, multi-simulation mode)                                  */
/* ------------------------------------------------------------------------------------------ */

/* Creates a context that advances n_sys independent planetary systems together. System s owns the
 * orbiting bodies offsets[s] .. offsets[s+1]-1 of the flat host arrays (offsets[0] = 0, 1 to 64
 * bodies per system; the central masses are NOT in the flat arrays) and has central mass m0[s].
 *   masses, radii [N], x, v [3N] heliocentric (N = offsets[n_sys]); G, dt, order as genga_init.
 *   steps_per_launch: steps captured in one CUDA-graph launch (genga_step runs whole launches,
 *   then single steps for the remainder).
 * Each system follows exactly the single-system step of genga_init (same parameters for all
 * systems except m0, Sect. 3.4). The kick's tile shape is autotuned here on the first kick
 * (genga_batch_info reports it). From 1024 systems on, the batch runs in parts of about 256
 * consecutive systems (at most 32), each with its own step graph on its own stream, forked from the
 * context's stream at every call and joined back; the parts all run the step graph and one kick
 * shape, timed with all parts at once. Every call of this section behaves the same either way
 * (arrays in the caller's order; counters summed over the parts, the step count once).
 * Returns 0 or a negative code; *ctx is NULL on failure. */
int genga_init_batch(genga_ctx **ctx, int n_sys, const int *offsets, const double *m0, const double *masses,
                     const double *radii, const double *x, const double *v, double G, double dt, int order,
                     int steps_per_launch);

/* Autotuned kick shape and steps per graph launch: *split = threads per body (1, 2, 4) of the
 * one-body-per-thread kick, or 0 for the Newton's-third-law kick (every pair of a system once, one
 * warp per system of 33..64 bodies or per pack of smaller systems; the opening kick's candidate
 * recomputation keeps one thread per body); *block = threads per CTA. */
int genga_batch_info(genga_ctx *ctx, int *split, int *block, int *steps_per_launch);

/* Overrides the autotuned kick shape: split 0 (Newton's third law), 1, 2 or 4 threads per body;
 * block 64, 128 or 256 threads per CTA. Results agree to rounding (the sums' order differs).
 * Takes effect from the next step. Returns GENGA_EINVAL for other values or a non-batched ctx. */
int genga_batch_set_kick(genga_ctx *ctx, int split, int block);

/* The schedule genga_init_batch chose by timing two steps of the batch each way: the step graph
 * (every phase over all systems, then the next phase) or one persistent launch in which each CTA
 * takes a system at a time and advances it through all the steps of the launch (*persistent = 1;
 * *ctas CTAs, one or two per SM). ms_graph, ms_persistent: the measured time per step of each
 * (any pointer may be NULL). The graph's trial issues its kernels one by one, which the step graph
 * does not, so the persistent launch is chosen only when its time is below 0.85 of the graph's. A
 * batch in parts runs the step graph in every part (the values reported are the first part's). The
 * persistent launch is not used while Rcut, RcutSun or Nmin is set. */
int genga_batch_schedule(genga_ctx *ctx, int *persistent, int *ctas, float *ms_graph, float *ms_persistent);

/* Overrides that choice: 1 persistent launch, 0 step graph (EINVAL if the persistent launch is not
 * available on this device). Both give each system the single-system step; the sums run in
 * different fixed orders, so results agree to rounding, not bit for bit. */
int genga_batch_set_schedule(genga_ctx *ctx, int persistent);

/* Flat heliocentric state in the caller's body order (waits for the stream); pointers may be NULL.
 * x, v [3N]; m, R [N]; alive [N] (0 for a ghost left by a merger). */
int genga_get_state_batch(genga_ctx *ctx, double *x, double *v, double *m, double *R, int *alive);

/* Replaces positions and velocities of the live bodies (flat, heliocentric, caller order); the next
 * step recomputes the first kick. */
int genga_set_state_batch(genga_ctx *ctx, const double *x, const double *v);

/* Confirmed close-encounter pairs of every system in the last substep of the last step (Sect. 3.4):
 * indices into the flat body arrays of genga_init_batch, i < j within one system, ascending. *n_pairs
 * receives the count; returns GENGA_ECAP if cap < count (the first cap pairs written). */
int genga_batch_encounters(genga_ctx *ctx, int *pairs, int cap, int *n_pairs);

/* Energy of every system (E [n_sys], caller order, democratic coordinates, Sect. 4.1) and the
 * internal energy U of all mergers so far. Waits for the stream. */
int genga_energy_batch(genga_ctx *ctx, double *E, double *U);

/* ------------------------------------------------------------------------------------------ */
/* Phase entry points: one step of the method on caller-provided device arrays (SoA layout).     */
/* n counts orbiting bodies only (no central mass); 1 <= n <= 2048. alive: int [n] (0 = ghost).  */
/* ------------------------------------------------------------------------------------------ */

/* Eq. rcrit: rc[i] = max(n1 a_i (m_i/(3 m0))^(1/3), n2 |tau| |v_i|), a_i from the democratic
 * state (1/a = 2/|x| - |v|^2/(G m0); |x| if unbound). x, v [3n]; m, rc [n]. */
int genga_phase_rcrit(int n, double G, double m0, double n1, double n2, double tau_abs,
                      const double *m, const int *alive, const double *x, const double *v,
                      double *rc, void *stream);

/* Eq. Hb kick accelerations a[3n] = sum_j G m_j W(r_ij) (x_j - x_i)/r_ij^3 over live j != i with
 * W = K (kmode 0) or K - rK' (kmode 1) and pair radius max(rc_i, rc_j), plus the prechecker
 * (Sect. 2.2): pairs (i < j) with r_ij^2 < max((pc rc_i)^2, (pc rc_j)^2), written ascending to
 * cand[2*cap] (device) with the count in *ncand (host). Returns GENGA_ECAP if cap is too small. */
int genga_phase_kick(int n, double G, double pc, int kmode, int precise_div, const double *m,
                     const int *alive, const double *x, const double *rc, double *a, int *cand,
                     int cap, int *ncand, void *stream);

/* Eq. fg Kepler drift of every live body about mu for dt, in place on x, v [3n]; fail[n] (device)
 * receives 1 where the solve did not converge within maxit (state untouched there). */
int genga_phase_kepler(int n, double mu, double dt, int maxit, const int *alive, double *x,
                       double *v, int *fail, void *stream);

/* Eqs. teqn/polydelta: candidates cand[2*ncand] (device, i < j) whose Hermite minimum separation
 * over the drift from (x0, v0) to (x1, v1) of length tau is below max(rc_i, rc_j); out[2*cap]
 * (device) receives them ascending, *nout (host) the count. Bit-exact with the CPU oracle. */
int genga_phase_encounters(int n, const int *alive, const double *x0, const double *v0,
                           const double *x1, const double *v1, const double *rc, const int *cand,
                           int ncand, double tau, int *out, int cap, int *nout, void *stream);

/* Appendix: connected components of the pair graph pairs[2*npairs] (device) plus the bodies with
 * single[i] != 0 as groups of their own. group_start[n+1] and members[n] (device) receive the
 * groups ordered by smallest member, members ascending; *ngroups (host) the count. */
int genga_phase_groups(int n, const int *pairs, int npairs, const int *single, int *group_start,
                       int *members, int *ngroups, void *stream);

/* Sect. 3.2: Bulirsch-Stoer integration of H_A for each group (group_start/members as produced by
 * genga_phase_groups, device) over tau, in place on x, v [3n]; with collisions on, mergers update
 * m, R, alive and add their internal energy to *U (host). Returns 0 or positive status bits. */
int genga_phase_bs(int n, double G, double m0, double tau, double bs_eps, int bs_kmax,
                   int bs_max_halvings, int kmode, int collisions, int ngroups,
                   const int *group_start, const int *members, const double *rc, double *m,
                   double *R, int *alive, double *x, double *v, double *U, void *stream);

/* Energy of the live bodies in democratic coordinates (x heliocentric, v barycentric), (Sect. 4.1). */
int genga_phase_energy(int n, double G, double m0, const double *m, const int *alive,
                       const double *x, const double *v, double *E, void *stream);

/* Kick phase that allocates no device memory (the paper has no counterpart: this is a service for
 * callers that cannot allocate). cudaMalloc may block on the driver's allocator and cudaFree
 * synchronises the whole device, so code in a latency-critical loop, or in a process whose device
 * memory belongs to another allocator or to a fixed budget, cannot use the entry points above,
 * which allocate temporaries. This one computes exactly what genga_phase_kick computes (same
 * kernels) but keeps its scratch in one file-scope device array of about 2 MB, which every GPU
 * that loads the library holds until the process exits.
 *   n <= 1024 (GENGA_ESIZE otherwise); m, alive, x, rc, a, cand as in genga_phase_kick (device);
 *   ncand is a DEVICE int that receives the full candidate count (nothing is copied to the host).
 *   Unlike genga_phase_kick this call cannot return GENGA_ECAP, since the count stays on the
 *   device: when *ncand exceeds cap, only the first cap pairs were written, and the caller must
 *   compare *ncand with cap itself.
 * Only cudaMemsetAsync, kernel launches and a device-to-device copy are enqueued on stream. The
 * first call on a device looks up the scratch array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture. The address is kept for the
 * life of the process: after a reset of the device (cudaDeviceReset) it is stale, so do not call
 * this entry point again in that process. All calls share the one array, which keeps the last
 * call's contents: calls that overlap on the GPU (different streams without ordering between them)
 * race on it. */
int genga_kick_noalloc(int n, double G, double pc, int kmode, int precise_div, const double *m,
                       const int *alive, const double *x, const double *rc, double *a, int *cand,
                       int cap, int *ncand, void *stream);

/* ------------------------------------------------------------------------------------------ */
/* Differentiable engine and its adjoint (reverse-mode derivative of the hybrid step)            */
/* ------------------------------------------------------------------------------------------ */
/* The paper has no adjoint; this is its hybrid step (Sect. 2.2-2.3: kicks weighted by K, Sun drifts,
 * universal-variable Kepler drifts, the Hermite encounter test, groups, Bulirsch-Stoer of H_A, the
 * Yoshida compositions) differentiated by hand, with perfect merging switched off (a merger changes
 * the number of bodies; the engine integrates through close passes instead). Every discrete
 * decision is frozen from the forward pass: the branch of K, the candidate and encounter pairs, the
 * groups, each group's accepted BS substeps and levels, and the Kepler solves (differentiated
 * implicitly at the converged universal anomaly). The critical radii depend on the state at the
 * start of each step, and that dependence is differentiated too.
 *
 * The engine advances n_sys independent systems of n bodies each (n <= 1024), central mass m0[b]
 * for system b, G, time step dt, order 2, 4 or 6, all with the default parameters of
 * genga_default_params (kmode 0) and collisions off.
 *
 * Memory: a checkpoint (state and critical radii) every ckpt_every steps, kept by
 * genga_adj_forward; genga_adj_backward recomputes one segment of ckpt_every steps at a time from
 * its checkpoint, recording every intermediate state and decision, then runs the vector-Jacobian
 * products backwards through it. The recording holds about 16 doubles per body per substep of a
 * segment, so ckpt_every trades device memory against nothing but that memory: the recomputation
 * is one forward pass in any case. */
typedef struct genga_adj genga_adj;

/* m0: host [n_sys]. Allocates all device memory of the engine (checkpoints grow on demand). */
int genga_adj_init(genga_adj **ctx, int n_sys, int n, const double *m0, double G, double dt, int order,
                   int ckpt_every);

/* Work is enqueued on this stream (cudaStream_t as void*; NULL = the CUDA default stream, which is
 * also the stream until this is called). The engine captures no graphs. */
int genga_adj_set_stream(genga_adj *ctx, void *stream);

/* n_steps hybrid steps from (x, v, m). DEVICE pointers, AoS: x, v, x_out, v_out [n_sys][n][3]
 * heliocentric, m [n_sys][n]. The inputs are copied; the engine keeps what the backward pass needs.
 * Asynchronous on the stream; status bits through genga_adj_status. */
int genga_adj_forward(genga_adj *ctx, int n_steps, const double *x, const double *v, const double *m,
                      double *x_out, double *v_out);

/* Gradients of <xbar, x_out> + <vbar, v_out> of the last genga_adj_forward with respect to its
 * inputs: gx, gv [n_sys][n][3], gm [n_sys][n]. DEVICE pointers, asynchronous on the stream. Must
 * follow the forward call it differentiates (the engine's state is that call's final state). */
int genga_adj_backward(genga_adj *ctx, const double *xbar, const double *vbar, double *gx, double *gv,
                       double *gm);

/* Waits for the stream, then returns the status bits (GENGA_ST_*) raised since the last forward. */
int genga_adj_status(genga_adj *ctx, int *code);
int genga_adj_sync(genga_adj *ctx);
void genga_adj_free(genga_adj *ctx);

/* Measurement aid (the paper has none): the device's FP64 throughput, from one launch of 4 CTAs of 256
 * threads per SM in which every thread runs 8 independent chains of iters fused multiply-adds (2 flop
 * each), timed with CUDA events on stream. *tflops receives TFLOP/s, *ms (may be NULL) the launch
 * time. Synchronises the stream; allocates 8 bytes of device memory for the duration of the call. */
int genga_fp64_probe(int iters, double *tflops, float *ms, void *stream);

/* Self-test of the device arithmetic helpers: out[i] = f(in[i]) for which = 0: x^(-1/2),
 * 1: x^(-3/2), 2: 1/x (the refined estimates used by the kernels). Device arrays. */
int genga_phase_mathcheck(int n, int which, const double *in, double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif
