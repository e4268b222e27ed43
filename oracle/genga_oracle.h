/*
 * genga_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU restatement of the hybrid symplectic N-body step of Grimm & Stadel,
 * "The GENGA Code" (Sect. 2.1-2.3, Sect. 3.2). It exists to check the CUDA path: only the
 * tests, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may load it. It shares
 * no code, header, table or helper with the CUDA library.
 *
 * Conventions (all arrays are caller-owned):
 *   n      number of orbiting bodies; the central mass m0 sits at the origin and is not stored.
 *   x[3n]  heliocentric positions, v[3n] barycentric ("democratic") velocities (Sect. 2.1).
 *   alive  1 for a live body, 0 for a ghost left by a merger (Sect. 3.2, Collisions).
 *   pairs  int pairs (i, j) with i < j, stored as pairs[2k], pairs[2k+1], ascending in (i, j).
 */
#ifndef GENGA_ORACLE_H
#define GENGA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
  double G;          /* gravitational constant */
  double m0;         /* central mass */
  double dt;         /* full time step tau */
  int order;         /* 2, 4 or 6: Eq. z1 and its Yoshida compositions (Sect. 2.3) */
  int kmode;         /* 0: K multiplies the Newtonian pair force; 1: exact gradient of H_B */
  double n1, n2;     /* critical-radius parameters of Eq. rcrit */
  double pc;         /* precheck factor: candidate if r < pc * rcrit (Sect. 2.2) */
  double bs_eps;     /* Bulirsch-Stoer relative tolerance */
  int bs_kmax;       /* deepest extrapolation level (sequence n_k = 2k) */
  int bs_max_halvings; /* consecutive step halvings before a group is declared failed */
  int kepler_maxit;  /* Newton iteration cap of the universal Kepler solve */
  int collisions;    /* 1: perfect merging on contact (Sect. 3.2, Collisions) */
  double rcut;       /* Sect. 3.2, Ejections: a body farther than rcut from m0 is removed (0: off) */
  double rcut_sun;   /* ... and one closer than rcut_sun (0: off) */
  int precheck_substeps; /* 1: the closing kick of every substep prechecks (its candidates feed the next
                            substep's encounter search); 0: only the closing kick of a full step does,
                            and its candidates serve all substeps of the next step (Sect. 2.3 as printed) */
} orc_params;

/* Status bits returned by orc_step and the phase routines. */
#define ORC_ST_KEPLER_FALLBACK 1   /* a Kepler solve failed and the body went to BS (not an error) */
#define ORC_ST_BS_FAILED       2   /* a BS group exceeded its halving cap */
#define ORC_ST_REUSE_VIOLATION 4   /* a non-candidate pair had K(r; new rcrit) != 1 */
#define ORC_ST_CAPACITY        8   /* a pair list exceeded its capacity */

void orc_default_params(orc_params *p);

/* ---- Sect. 2.1: changeover function and critical radius ---- */
double orc_changeover(double r, double rc);          /* K(r) */
double orc_changeover_dr(double r, double rc);       /* dK/dr */
double orc_weight_B(double r2, double rc, int kmode); /* factor on G m_j (x_j-x_i)/r^3 in the kick */
void orc_rcrit(int n, const orc_params *p, double tau_abs, const double *m, const int *alive,
               const double *x, const double *v, double *rc);

/* ---- Sect. 2.2: operators ---- */
void orc_accel_B(int n, const orc_params *p, const double *m, const int *alive, const double *x,
                 const double *rc, double *a);
int orc_precheck(int n, const orc_params *p, const int *alive, const double *x, const double *rc,
                 int *pairs, int cap);
void orc_momentum(int n, const double *m, const int *alive, const double *v, double P[3]);
void orc_sun_drift(int n, const orc_params *p, const int *alive, double *x, const double P[3],
                   double h);
void orc_stumpff(double z, double c[4]);
int orc_kepler_drift(double mu, double x[3], double v[3], double dt, int maxit, int *iters);
double orc_hermite_min(const double dx0[3], const double dv0[3], const double dx1[3],
                       const double dv1[3], double tau);
int orc_encounters(int n, const int *alive, const double *x0, const double *v0, const double *x1,
                   const double *v1, const double *rc, const int *cand, int ncand, double tau,
                   int *pairs, int cap);
int orc_groups(int n, const int *pairs, int npairs, const int *single, int *group_start,
               int *members);
double orc_energy(int n, const orc_params *p, const double *m, const int *alive, const double *x,
                  const double *v);

/* BS integration of one group over tau from (x, v) in place (Sect. 3.2, Bulirsch-Stoer). The
 * group's members are idx[0..g-1] (ascending); x, v, m, R, alive, rc are full-system arrays.
 * With collisions on, merges update m, R, alive, x, v and add to *U. Returns 0 or ORC_ST_BS_FAILED. */
int orc_bs_group(int n, const orc_params *p, int g, const int *idx, double tau, double *m,
                 double *R, int *alive, double *x, double *v, const double *rc, double *U,
                 int *ncoll, int *coll_pairs, int coll_cap, int *bs_steps);

/* Collision reports (Sect. 3.2, Collisions): ORC_CREC doubles per merger --
 *   [0] step (1-based), [1] substep of the composition (0-based), [2] time from the substep's start
 *   to the start of the BS substep in which the contact was found, [3] body i, [4] body j (i < j),
 *   [5..7] x_i, [8..10] v_i, [11..13] spin_i, [14..16] x_j, [17..19] v_j, [20..22] spin_j at that
 *   time (heliocentric positions, barycentric velocities), [23] the surviving body.
 * orc_bs_group_rec is orc_bs_group that also tracks spins (spin [3n], may be NULL) and writes the
 * reports of its mergers (entries 0 and 1 set to -1: the caller knows the step). */
#define ORC_CREC 24
int orc_bs_group_rec(int n, const orc_params *p, int g, const int *idx, double tau, double *m,
                     double *R, int *alive, double *x, double *v, const double *rc, double *U,
                     int *ncoll, int *coll_pairs, int coll_cap, int *bs_steps, double *spin,
                     double *crec, int crec_cap, int *ncrec);

/* Sect. 2.3: substep weights w[0..k-1] of the composition of order 2 (k = 1, Eq. z1), 4 (k = 3) or
 * 6 (k = 7, Yoshida's solution A); substep j has the signed length w[j] * tau. Returns k. */
int orc_substep_weights(int order, double *w);

/* ---- whole simulation (main mode) ---- */
typedef struct orc_sim orc_sim;
orc_sim *orc_create(int n, const orc_params *p, const double *m, const double *R, const double *xh,
                    const double *vh);
void orc_free(orc_sim *s);
int orc_step(orc_sim *s, int nsteps);
void orc_get_state(const orc_sim *s, double *xh, double *vh, double *m, double *R, int *alive);
void orc_get_internal(const orc_sim *s, double *x, double *v, double *a, double *rc);
double orc_get_energy(const orc_sim *s, double *U);
int orc_get_candidates(const orc_sim *s, int *pairs, int cap);
int orc_get_encounters(const orc_sim *s, int substep, int *pairs, int cap);
int orc_get_groups(const orc_sim *s, int substep, int *group_start, int *members, int cap);
void orc_get_stats(const orc_sim *s, long long *stats, int nstats);
int orc_get_collisions(const orc_sim *s, int *pairs, int cap);
/* All collision reports so far (at most cap written; returns the count), ORC_CREC doubles each. */
int orc_get_collision_records(const orc_sim *s, double *rec, int cap);
/* Spin angular momentum of every body [3n] (zero at orc_create; a merger gives the survivor the sum
 * of both spins and the pair's orbital angular momentum about its centre of mass). */
void orc_set_spin(orc_sim *s, const double *spin);
void orc_get_spin(const orc_sim *s, double *spin);
/* Ejections so far (all of them; at most cap records written): record k = rec[8k .. 8k+7] =
 * body index, step (1-based, the step at whose end it was removed), heliocentric x[3] and v[3]. */
int orc_get_ejections(const orc_sim *s, double *rec, int cap);

/* ---- test-particle mode (Sect. 3.3): massive bodies as above plus massless test particles ---- */
typedef struct orc_tpsim orc_tpsim;
orc_tpsim *orc_tp_create(int n, const orc_params *p, const double *m, const double *R, const double *xh,
                         const double *vh, int ntp, const double *xt, const double *vt, const double *Rt);
void orc_tp_free(orc_tpsim *t);
int orc_tp_step(orc_tpsim *t, int nsteps);
void orc_tp_get_state(const orc_tpsim *t, double *xh, double *vh, double *m, int *alive, double *xt,
                      double *vt, int *tp_alive);
void orc_tp_get_stats(const orc_tpsim *t, long long *stats, int nstats);
int orc_tp_get_encounters(const orc_tpsim *t, int substep, int *pairs, int cap);
int orc_tp_get_ejections(const orc_tpsim *t, double *rec, int cap);  /* the planets' (orc_get_ejections) */

#ifdef __cplusplus
}
#endif
#endif
