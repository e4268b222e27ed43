/*
 * genga_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-ordered FP64 CPU restatement of the hybrid symplectic step of
 * Grimm & Stadel, "The GENGA Code" (arXiv:1404.2324). It is the reference the CUDA library is
 * checked against; the product path never loads it. It shares no code with the CUDA sources.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fno-fast-math -fPIC -shared (no FMA contraction:
 * every a*b+c is two roundings unless it is written fma(); the few fma() calls define the
 * canonical evaluation of the decision quantities r^2 and x.v, see pair_r2 / pair_dot).
 *
 * Each routine cites the passage of the paper it restates. Readings where the paper is silent
 * or garbled follow the project's design notes and are repeated in the comments.
 */
#include "genga_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* Small helpers                                                                              */
/* ------------------------------------------------------------------------------------------ */

/* Canonical evaluation of |d|^2 and a.b: dx*dx rounded, then two fused multiply-adds.
 * Decisions (precheck, encounter test) compare these values, so both implementations must
 * evaluate them in exactly this order. */
static double pair_r2(double dx, double dy, double dz) { return fma(dz, dz, fma(dy, dy, dx * dx)); }
static double pair_dot(const double a[3], const double b[3]) {
  return fma(a[2], b[2], fma(a[1], b[1], a[0] * b[0]));
}

static void *xcalloc(size_t n, size_t sz) {
  void *p = calloc(n ? n : 1, sz);
  if (!p) abort();
  return p;
}

void orc_default_params(orc_params *p) {
  memset(p, 0, sizeof(*p));
  p->G = 2.959122082855911e-4; /* k^2, Gaussian gravitational constant, AU^3 Msun^-1 day^-2 */
  p->m0 = 1.0;
  p->dt = 6.0;
  p->order = 2;
  p->kmode = 0;
  p->n1 = 3.0;   /* Sect. 2.1: "usually set to n1 = 3 and n2 = 0.4" */
  p->n2 = 0.4;
  p->pc = 3.0;   /* Sect. 2.2: critical radius increased by a factor of three */
  p->bs_eps = 1e-12;
  p->bs_kmax = 8;
  p->bs_max_halvings = 30;
  p->kepler_maxit = 30;
  p->collisions = 1;
  p->rcut = 0.0;     /* no ejections unless asked for */
  p->rcut_sun = 0.0;
  p->precheck_substeps = 1;
}

/* ------------------------------------------------------------------------------------------ */
/* Sect. 2.1: changeover function K(r), Eq. for K and y                                        */
/* ------------------------------------------------------------------------------------------ */

/* K = 0 for y <= 0, y^2/(2y^2-2y+1) for 0 < y < 1, 1 for y >= 1, with
 * y = (r - 0.1 rc)/(0.9 rc). (The paper's "0.9 r_rcrit" is read as 0.9 rc; the formula is
 * continuous at y = 0 and y = 1, so the end points take the limit values.) */
double orc_changeover(double r, double rc) {
  double y = (r - 0.1 * rc) / (0.9 * rc);
  if (y <= 0.0) return 0.0;
  if (y >= 1.0) return 1.0;
  return y * y / (2.0 * y * y - 2.0 * y + 1.0);
}

/* dK/dr = [2y(1-y)/(2y^2-2y+1)^2] / (0.9 rc) inside the transition, 0 outside. */
double orc_changeover_dr(double r, double rc) {
  double y = (r - 0.1 * rc) / (0.9 * rc);
  if (y <= 0.0 || y >= 1.0) return 0.0;
  double d = 2.0 * y * y - 2.0 * y + 1.0;
  return 2.0 * y * (1.0 - y) / (d * d) / (0.9 * rc);
}

/* Weight of the Newtonian pair force G m_j (x_j - x_i)/r^3 in the kick (Eq. Hb).
 * kmode 0: K(r) (the kick is "weighted by K"); kmode 1: K - r K'(r), the exact -grad H_B.
 * r^2 >= rc^2 is the K = 1 region (y >= 1). */
double orc_weight_B(double r2, double rc, int kmode) {
  double rcsq = rc * rc;
  if (r2 >= rcsq) return 1.0;
  double r = sqrt(r2);
  double w = orc_changeover(r, rc);
  if (kmode == 1) w -= r * orc_changeover_dr(r, rc);
  return w;
}

/* Eq. rcrit: rc_i = max(n1 R_H,i, n2 tau |v_i|). The Hill radius is R_H = a (m/(3 m0))^(1/3)
 * with a from the democratic state, 1/a = 2/|x| - |v|^2/(G m0); an unbound body (1/a <= 0)
 * uses |x| for a. |v| is the barycentric speed at the start of the step. */
void orc_rcrit(int n, const orc_params *p, double tau_abs, const double *m, const int *alive,
               const double *x, const double *v, double *rc) {
  double mu = p->G * p->m0;
  for (int i = 0; i < n; i++) {
    if (!alive[i]) { rc[i] = 0.0; continue; }
    const double *xi = x + 3 * i, *vi = v + 3 * i;
    double r = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    double v2 = vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2];
    double inva = 2.0 / r - v2 / mu;
    double asemi = inva > 0.0 ? 1.0 / inva : r;
    double rh = asemi * cbrt(m[i] / (3.0 * p->m0));
    double a1 = p->n1 * rh;
    double a2 = p->n2 * tau_abs * sqrt(v2);
    rc[i] = a1 > a2 ? a1 : a2;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Sect. 2.2: kick (B), precheck, Sun drift (C)                                                */
/* ------------------------------------------------------------------------------------------ */

/* a_i = sum_{j != i, alive} G m_j W_B(r_ij) (x_j - x_i)/r_ij^3, j ascending; the pair critical
 * radius is max(rc_i, rc_j) (Sect. 2.1). */
void orc_accel_B(int n, const orc_params *p, const double *m, const int *alive, const double *x,
                 const double *rc, double *a) {
  /* bodies are independent (each sum runs over j ascending); a multi-threaded build splits them */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int i = 0; i < n; i++) {
    double ax = 0.0, ay = 0.0, az = 0.0;
    if (alive[i]) {
      for (int j = 0; j < n; j++) {
        if (j == i || !alive[j]) continue;
        double dx = x[3 * j] - x[3 * i], dy = x[3 * j + 1] - x[3 * i + 1], dz = x[3 * j + 2] - x[3 * i + 2];
        double r2 = pair_r2(dx, dy, dz);
        double rcij = rc[i] > rc[j] ? rc[i] : rc[j];
        double w = orc_weight_B(r2, rcij, p->kmode);
        double r = sqrt(r2);
        double f = p->G * m[j] * w / (r2 * r);
        ax += f * dx;
        ay += f * dy;
        az += f * dz;
      }
    }
    a[3 * i] = ax;
    a[3 * i + 1] = ay;
    a[3 * i + 2] = az;
  }
}

/* Sect. 2.2 prechecker: pair (i < j) is a candidate if r_ij < pc * max(rc_i, rc_j), evaluated as
 * r^2 < max((pc rc_i)^2, (pc rc_j)^2) on the positions the kick sees. Output ascending. */
int orc_precheck(int n, const orc_params *p, const int *alive, const double *x, const double *rc,
                 int *pairs, int cap) {
  int cnt = 0;
  for (int i = 0; i < n; i++) {
    if (!alive[i]) continue;
    double ti = p->pc * rc[i];
    double Ti = ti * ti;
    for (int j = i + 1; j < n; j++) {
      if (!alive[j]) continue;
      double tj = p->pc * rc[j];
      double Tj = tj * tj;
      double T = Ti > Tj ? Ti : Tj;
      double dx = x[3 * j] - x[3 * i], dy = x[3 * j + 1] - x[3 * i + 1], dz = x[3 * j + 2] - x[3 * i + 2];
      if (pair_r2(dx, dy, dz) < T) {
        if (cnt < cap) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j; }
        cnt++;
      }
    }
  }
  return cnt;
}

/* Eq. Hc: P = sum of the barycentric momenta of the live bodies, ascending. */
void orc_momentum(int n, const double *m, const int *alive, const double *v, double P[3]) {
  P[0] = P[1] = P[2] = 0.0;
  for (int i = 0; i < n; i++) {
    if (!alive[i]) continue;
    P[0] += m[i] * v[3 * i];
    P[1] += m[i] * v[3 * i + 1];
    P[2] += m[i] * v[3 * i + 2];
  }
}

/* Flow of H_C for time h: every position moves by h P / m0; momenta are unchanged. */
void orc_sun_drift(int n, const orc_params *p, const int *alive, double *x, const double P[3],
                   double h) {
  double f = h / p->m0;
  for (int i = 0; i < n; i++) {
    if (!alive[i]) continue;
    x[3 * i] += f * P[0];
    x[3 * i + 1] += f * P[1];
    x[3 * i + 2] += f * P[2];
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Eq. fg: Kepler drift with Gauss' f and g functions in universal variables (Danby 1988)       */
/* ------------------------------------------------------------------------------------------ */

/* Stumpff functions c_k(z), k = 0..3. For |z| > 0.1 the argument is divided by 4 until it is
 * small, the series of c2 and c3 are summed, c0 = 1 - z c2, c1 = 1 - z c3, and the quadrupling
 * identities c0(4z) = 2c0^2-1, c1(4z) = c0 c1, c2(4z) = c1^2/2, c3(4z) = (c2 + c0 c3)/4 undo the
 * reduction. */
void orc_stumpff(double z, double c[4]) {
  int nred = 0;
  while (fabs(z) > 0.1 && nred < 200) {
    z *= 0.25;
    nred++;
  }
  double t2 = 0.5, s2 = 0.5; /* c2 = sum_k (-z)^k / (2k+2)! */
  double t3 = 1.0 / 6.0, s3 = 1.0 / 6.0; /* c3 = sum_k (-z)^k / (2k+3)! */
  for (int k = 1; k <= 12; k++) {
    t2 *= -z / ((2.0 * k + 1.0) * (2.0 * k + 2.0));
    s2 += t2;
    t3 *= -z / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
    s3 += t3;
  }
  double c2 = s2, c3 = s3;
  double c1 = 1.0 - z * c3, c0 = 1.0 - z * c2;
  for (; nred > 0; nred--) {
    c3 = (c2 + c0 * c3) * 0.25;
    c2 = 0.5 * c1 * c1;
    c1 = c0 * c1;
    c0 = 2.0 * c0 * c0 - 1.0;
  }
  c[0] = c0; c[1] = c1; c[2] = c2; c[3] = c3;
}

/* Two-body drift about mu = G m0 (not G(m0+m_i): democratic coordinates, Sect. 2.2).
 * Universal Kepler equation F(s) = r0 s c1 + u s^2 c2 + mu s^3 c3 - dt = 0, z = beta s^2,
 * beta = 2 mu/r0 - v0^2, u = x0.v0; Newton from s = dt/r0 until |ds| <= 4 ulp |s|, or until a
 * tiny step (|ds| <= 1e-10 |s|) stops shrinking (at least halving) -- the rounding floor of F,
 * where Newton can cycle between neighbours a few ulp apart -- at most maxit iterations. Then f = 1 - (mu/r0) s^2 c2, g = dt - mu s^3 c3, r = r0 c0 + u s c1 + mu s^2 c2,
 * fdot = -mu s c1/(r r0), gdot = 1 - (mu/r) s^2 c2, and x = f x0 + g v0, v = fdot x0 + gdot v0.
 * Returns 0, or 1 (x, v untouched) if Newton did not converge. */
int orc_kepler_drift(double mu, double x[3], double v[3], double dt, int maxit, int *iters) {
  double r0 = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double u = x[0] * v[0] + x[1] * v[1] + x[2] * v[2];
  double beta = 2.0 * mu / r0 - v2;
  double s = dt / r0;
  double c[4];
  double ds_prev = HUGE_VAL;
  int ok = 0, it;
  for (it = 1; it <= maxit; it++) {
    orc_stumpff(beta * s * s, c);
    double F = r0 * s * c[1] + u * s * s * c[2] + mu * s * s * s * c[3] - dt;
    double Fp = r0 * c[0] + u * s * c[1] + mu * s * s * c[2];
    double ds = F / Fp;
    s -= ds;
    if (!isfinite(s)) break;
    if (fabs(ds) <= 4.0 * DBL_EPSILON * fabs(s)) { ok = 1; break; }
    /* rounding floor: the step is already tiny and no longer shrinks (a 2-cycle of a few ulp) */
    if (fabs(ds) <= 1e-10 * fabs(s) && fabs(ds) >= 0.5 * ds_prev) { ok = 1; break; }
    ds_prev = fabs(ds);
  }
  if (iters) *iters = it;
  if (!ok) return 1;
  orc_stumpff(beta * s * s, c);
  double r = r0 * c[0] + u * s * c[1] + mu * s * s * c[2];
  double f = 1.0 - (mu / r0) * s * s * c[2];
  double g = dt - mu * s * s * s * c[3];
  double fd = -(mu / (r * r0)) * s * c[1];
  double gd = 1.0 - (mu / r) * s * s * c[2];
  double xn[3], vn[3];
  for (int k = 0; k < 3; k++) {
    xn[k] = f * x[k] + g * v[k];
    vn[k] = fd * x[k] + gd * v[k];
  }
  if (!isfinite(xn[0] + xn[1] + xn[2] + vn[0] + vn[1] + vn[2])) return 1;
  for (int k = 0; k < 3; k++) { x[k] = xn[k]; v[k] = vn[k]; }
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Sect. 2.2: close-encounter search with the cubic Hermite interpolant (Eqs. teqn, polydelta)  */
/* ------------------------------------------------------------------------------------------ */

static double hermite_eval(double t, double tau, double P0, double P1, double Pd0, double Pd1) {
  double s = 1.0 - t;
  double h00 = (s * s) * (1.0 + 2.0 * t);
  double h01 = (t * t) * (3.0 - 2.0 * t);
  double h10 = (t * (s * s)) * tau;
  double h11 = ((t * t) * s) * tau;
  return ((h00 * P0 + h01 * P1) + h10 * Pd0) - h11 * Pd1;
}

/* Minimum over t in [0, 1] of the Hermite cubic P(t) of the squared separation. P(0), P(1) are
 * |dx|^2 before and after the drift, Pd = dP/dt in physical time = 2 dx.dv (the paper's "square
 * of the difference ... of velocities" is read as this derivative), tau the drift duration.
 * dP/d(t) = a t^2 + b t + c with a = 6(P0-P1) + 3 tau (Pd0 + Pd1) (the sign inside the second
 * term is fixed by differentiating the printed polynomial), b = 6(P1-P0) - 2 tau (2 Pd0 + Pd1),
 * c = tau Pd0. Real roots in (0, 1) come from the cancellation-free quadratic formula. */
double orc_hermite_min(const double dx0[3], const double dv0[3], const double dx1[3],
                       const double dv1[3], double tau) {
  double P0 = pair_r2(dx0[0], dx0[1], dx0[2]);
  double P1 = pair_r2(dx1[0], dx1[1], dx1[2]);
  double Pd0 = 2.0 * pair_dot(dx0, dv0);
  double Pd1 = 2.0 * pair_dot(dx1, dv1);
  double a = 6.0 * (P0 - P1) + (3.0 * tau) * (Pd0 + Pd1);
  double b = 6.0 * (P1 - P0) - (2.0 * tau) * (2.0 * Pd0 + Pd1);
  double c = tau * Pd0;
  double dmin = P0 < P1 ? P0 : P1;
  double disc = b * b - 4.0 * a * c;
  if (disc >= 0.0) {
    double sq = sqrt(disc);
    double q = -0.5 * (b + copysign(sq, b));
    if (a != 0.0) {
      double t = q / a;
      if (t > 0.0 && t < 1.0) {
        double d = hermite_eval(t, tau, P0, P1, Pd0, Pd1);
        if (d < dmin) dmin = d;
      }
    }
    if (q != 0.0) {
      double t = c / q;
      if (t > 0.0 && t < 1.0) {
        double d = hermite_eval(t, tau, P0, P1, Pd0, Pd1);
        if (d < dmin) dmin = d;
      }
    }
  }
  return dmin;
}

/* Confirmed close encounters among the candidates: Delta_min < max(rc_i, rc_j)^2, with the states
 * right before (x0, v0) and right after (x1, v1) the Kepler drift of duration tau. The output keeps
 * the candidates' ascending order. */
int orc_encounters(int n, const int *alive, const double *x0, const double *v0, const double *x1,
                   const double *v1, const double *rc, const int *cand, int ncand, double tau,
                   int *pairs, int cap) {
  (void)n;
  int cnt = 0;
  for (int k = 0; k < ncand; k++) {
    int i = cand[2 * k], j = cand[2 * k + 1];
    if (!alive[i] || !alive[j]) continue;
    double dx0[3], dv0[3], dx1[3], dv1[3];
    for (int c = 0; c < 3; c++) {
      dx0[c] = x0[3 * j + c] - x0[3 * i + c];
      dv0[c] = v0[3 * j + c] - v0[3 * i + c];
      dx1[c] = x1[3 * j + c] - x1[3 * i + c];
      dv1[c] = v1[3 * j + c] - v1[3 * i + c];
    }
    double dmin = orc_hermite_min(dx0, dv0, dx1, dv1, tau);
    double rcij = rc[i] > rc[j] ? rc[i] : rc[j];
    if (dmin < rcij * rcij) {
      if (cnt < cap) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j; }
      cnt++;
    }
  }
  return cnt;
}

/* ------------------------------------------------------------------------------------------ */
/* Sect. 3.2 + Appendix: encounter groups = connected components of the pair graph              */
/* ------------------------------------------------------------------------------------------ */

/* Breadth-first search from each body in ascending order; a group is the set reachable through
 * encounter pairs, plus bodies flagged in single[] (failed Kepler solves) as groups of their own.
 * Groups come out ordered by their smallest index, members ascending. Returns the group count;
 * group_start has ngroups+1 entries, members holds at most n entries. */
int orc_groups(int n, const int *pairs, int npairs, const int *single, int *group_start,
               int *members) {
  int *deg = (int *)xcalloc((size_t)n + 1, sizeof(int));
  for (int k = 0; k < npairs; k++) { deg[pairs[2 * k] + 1]++; deg[pairs[2 * k + 1] + 1]++; }
  for (int i = 0; i < n; i++) deg[i + 1] += deg[i];
  int *adj = (int *)xcalloc((size_t)2 * npairs, sizeof(int));
  int *fill = (int *)xcalloc((size_t)n, sizeof(int));
  for (int k = 0; k < npairs; k++) {
    int i = pairs[2 * k], j = pairs[2 * k + 1];
    adj[deg[i] + fill[i]++] = j;
    adj[deg[j] + fill[j]++] = i;
  }
  int *seen = (int *)xcalloc((size_t)n, sizeof(int));
  int *queue = (int *)xcalloc((size_t)n, sizeof(int));
  int ng = 0, nm = 0;
  group_start[0] = 0;
  for (int s = 0; s < n; s++) {
    int has_edge = deg[s + 1] > deg[s];
    int want = has_edge || (single && single[s]);
    if (!want || seen[s]) continue;
    int qh = 0, qt = 0;
    queue[qt++] = s;
    seen[s] = 1;
    while (qh < qt) {
      int u = queue[qh++];
      for (int e = deg[u]; e < deg[u + 1]; e++) {
        int w = adj[e];
        if (!seen[w]) { seen[w] = 1; queue[qt++] = w; }
      }
    }
    /* members ascending: insertion sort of the (small) component */
    for (int a = 1; a < qt; a++) {
      int key = queue[a], b = a - 1;
      while (b >= 0 && queue[b] > key) { queue[b + 1] = queue[b]; b--; }
      queue[b + 1] = key;
    }
    for (int a = 0; a < qt; a++) members[nm++] = queue[a];
    ng++;
    group_start[ng] = nm;
  }
  free(deg); free(adj); free(fill); free(seen); free(queue);
  return ng;
}

/* ------------------------------------------------------------------------------------------ */
/* Sect. 3.2: Bulirsch-Stoer integration of H_A for one encounter group, with merging           */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  const orc_params *p;
  int g;
  const int *idx;   /* global indices of the members */
  const double *m;  /* full-system masses */
  const int *alive; /* full-system live flags */
  const double *rc; /* full-system critical radii of this step */
} bs_ctx;

/* Right-hand side of H_A restricted to the group: dx/dt = v,
 * dv_q/dt = -G m0 x_q/|x_q|^3 + sum_{p in group, p != q} G m_p W_A(r_qp) (x_p - x_q)/r_qp^3 with
 * W_A = 1 - W_B (the central mass stays at the origin during the step). Dead members are frozen. */
static void bs_deriv(const bs_ctx *c, const double *y, double *dy) {
  const orc_params *p = c->p;
  for (int q = 0; q < c->g; q++) {
    int iq = c->idx[q];
    double *d = dy + 6 * q;
    const double *yq = y + 6 * q;
    if (!c->alive[iq]) { for (int k = 0; k < 6; k++) d[k] = 0.0; continue; }
    d[0] = yq[3]; d[1] = yq[4]; d[2] = yq[5];
    double r2 = yq[0] * yq[0] + yq[1] * yq[1] + yq[2] * yq[2];
    double r = sqrt(r2);
    double f = p->G * p->m0 / (r2 * r);
    double ax = -f * yq[0], ay = -f * yq[1], az = -f * yq[2];
    for (int s = 0; s < c->g; s++) {
      int is = c->idx[s];
      if (s == q || !c->alive[is]) continue;
      const double *ys = y + 6 * s;
      double dx = ys[0] - yq[0], dyy = ys[1] - yq[1], dz = ys[2] - yq[2];
      double pr2 = pair_r2(dx, dyy, dz);
      double rcij = c->rc[iq] > c->rc[is] ? c->rc[iq] : c->rc[is];
      double wa = 1.0 - orc_weight_B(pr2, rcij, p->kmode);
      if (wa == 0.0) continue;
      double pr = sqrt(pr2);
      double fp = p->G * c->m[is] * wa / (pr2 * pr);
      ax += fp * dx;
      ay += fp * dyy;
      az += fp * dz;
    }
    d[3] = ax; d[4] = ay; d[5] = az;
  }
}

/* Modified midpoint rule with nsub substeps over H (Gragg): z0 = y, z1 = z0 + h f(z0),
 * z_{m+1} = z_{m-1} + 2h f(z_m), result = (z_n + z_{n-1} + h f(z_n))/2. */
static void bs_mmid(const bs_ctx *c, const double *y, const double *dy0, double H, int nsub,
                    double *out, double *za, double *zb, double *f) {
  int d = 6 * c->g;
  double h = H / nsub;
  for (int k = 0; k < d; k++) { za[k] = y[k]; zb[k] = y[k] + h * dy0[k]; }
  for (int m = 1; m < nsub; m++) {
    bs_deriv(c, zb, f);
    for (int k = 0; k < d; k++) {
      double t = za[k] + 2.0 * h * f[k];
      za[k] = zb[k];
      zb[k] = t;
    }
  }
  bs_deriv(c, zb, f);
  for (int k = 0; k < d; k++) out[k] = 0.5 * (zb[k] + za[k] + h * f[k]);
}

/* One Bulirsch-Stoer attempt of length H: midpoint sequence n_k = 2k, k = 1..kmax, polynomial
 * (Neville) extrapolation in h^2, T[k][j+1] = T[k][j] + (T[k][j] - T[k-1][j]) / ((n_k/n_{k-j})^2-1).
 * From k = 2 on, the error is max over live members and components of |T[k][k] - T[k][k-1]|
 * divided by |x_q| (position components) or |v_q| (velocity components) at the start of the
 * attempt; the first k with error <= eps is accepted. Returns the accepted level or 0. */
static int bs_attempt(const bs_ctx *c, const double *y, double H, double *out, double *T,
                      double *work) {
  const orc_params *p = c->p;
  int d = 6 * c->g, kmax = p->bs_kmax;
  double *dy0 = work, *za = work + d, *zb = work + 2 * d, *f = work + 3 * d;
  double *sc = work + 4 * d;
  bs_deriv(c, y, dy0);
  for (int q = 0; q < c->g; q++) {
    const double *yq = y + 6 * q;
    double sx = sqrt(yq[0] * yq[0] + yq[1] * yq[1] + yq[2] * yq[2]);
    double sv = sqrt(yq[3] * yq[3] + yq[4] * yq[4] + yq[5] * yq[5]);
    if (!(sx > 0.0)) sx = DBL_MIN;
    if (!(sv > 0.0)) sv = DBL_MIN;
    for (int k = 0; k < 3; k++) { sc[6 * q + k] = sx; sc[6 * q + 3 + k] = sv; }
  }
  /* T is (kmax+1) x (kmax+1) x d, T[k][j] at (k*(kmax+1) + j)*d, 1-based k and j */
#define TT(k, j) (T + ((size_t)(k) * (kmax + 1) + (j)) * d)
  for (int k = 1; k <= kmax; k++) {
    int nk = 2 * k;
    bs_mmid(c, y, dy0, H, nk, TT(k, 1), za, zb, f);
    for (int j = 1; j < k; j++) {
      double ratio = (double)k / (double)(k - j); /* n_k / n_{k-j} */
      double fac = ratio * ratio - 1.0;
      double *tkj = TT(k, j), *tk1j = TT(k - 1, j), *tkj1 = TT(k, j + 1);
      for (int e = 0; e < d; e++) tkj1[e] = tkj[e] + (tkj[e] - tk1j[e]) / fac;
    }
    if (k >= 2) {
      double err = 0.0;
      double *a = TT(k, k), *b = TT(k, k - 1);
      for (int q = 0; q < c->g; q++) {
        if (!c->alive[c->idx[q]]) continue;
        for (int e = 6 * q; e < 6 * q + 6; e++) {
          double ee = fabs(a[e] - b[e]) / sc[e];
          if (!(ee <= err)) err = ee; /* NaN propagates as "not converged" */
        }
      }
      if (err <= p->bs_eps) {
        memcpy(out, a, sizeof(double) * d);
        return k;
      }
    }
  }
#undef TT
  return 0;
}

/* Perfect merger of bodies i and j (Sect. 3.2, Collisions): the heavier survives (equal masses:
 * the smaller index), mass and linear momentum are conserved, R = (R_i^3 + R_j^3)^(1/3), and
 * U += m_i m_j/(2(m_i+m_j)) |v_ij|^2 - G m_i m_j/r_ij is booked. The other body becomes a ghost.
 * The new body's spin follows from angular-momentum conservation: the spins of both bodies plus the
 * orbital angular momentum of the pair about its centre of mass, mu (x_j - x_i) x (v_j - v_i) with
 * mu = m_i m_j / (m_i + m_j) (spin may be NULL: not tracked). */
static void merge_bodies(const orc_params *p, int gi, int gj, double *yi, double *yj, double *m,
                         double *R, int *alive, double *U, double *spin) {
  double mi = m[gi], mj = m[gj], M = mi + mj;
  double dx = yj[0] - yi[0], dy = yj[1] - yi[1], dz = yj[2] - yi[2];
  double dvx = yj[3] - yi[3], dvy = yj[4] - yi[4], dvz = yj[5] - yi[5];
  double r = sqrt(dx * dx + dy * dy + dz * dz);
  double v2 = dvx * dvx + dvy * dvy + dvz * dvz;
  *U += 0.5 * mi * mj / M * v2 - p->G * mi * mj / r;
  int surv, ghost;
  double *ys, *yg;
  if (mi > mj || (mi == mj && gi < gj)) { surv = gi; ghost = gj; ys = yi; yg = yj; }
  else { surv = gj; ghost = gi; ys = yj; yg = yi; }
  if (spin) {
    double mu = mi * mj / M;
    double L[3] = {mu * (dy * dvz - dz * dvy), mu * (dz * dvx - dx * dvz), mu * (dx * dvy - dy * dvx)};
    for (int k = 0; k < 3; k++) spin[3 * surv + k] = spin[3 * gi + k] + spin[3 * gj + k] + L[k];
    for (int k = 0; k < 3; k++) spin[3 * ghost + k] = 0.0;
  }
  double cm[6];
  for (int k = 0; k < 6; k++) cm[k] = (mi * yi[k] + mj * yj[k]) / M;
  for (int k = 0; k < 6; k++) ys[k] = cm[k];
  (void)yg;
  double Ri = R[gi], Rj = R[gj];
  R[surv] = cbrt(Ri * Ri * Ri + Rj * Rj * Rj);
  m[surv] = M;
  m[ghost] = 0.0;
  R[ghost] = 0.0;
  alive[ghost] = 0;
}

int orc_bs_group(int n, const orc_params *p, int g, const int *idx, double tau, double *m,
                 double *R, int *alive, double *x, double *v, const double *rc, double *U,
                 int *ncoll, int *coll_pairs, int coll_cap, int *bs_steps) {
  return orc_bs_group_rec(n, p, g, idx, tau, m, R, alive, x, v, rc, U, ncoll, coll_pairs, coll_cap, bs_steps,
                          NULL, NULL, 0, NULL);
}

int orc_bs_group_rec(int n, const orc_params *p, int g, const int *idx, double tau, double *m,
                     double *R, int *alive, double *x, double *v, const double *rc, double *U,
                     int *ncoll, int *coll_pairs, int coll_cap, int *bs_steps, double *spin,
                     double *crec, int crec_cap, int *ncrec) {
  (void)n;
  int d = 6 * g, kmax = p->bs_kmax;
  double *y = (double *)xcalloc((size_t)d, sizeof(double));
  double *yn = (double *)xcalloc((size_t)d, sizeof(double));
  double *T = (double *)xcalloc((size_t)(kmax + 1) * (kmax + 1) * d, sizeof(double));
  double *work = (double *)xcalloc((size_t)5 * d, sizeof(double));
  for (int q = 0; q < g; q++)
    for (int k = 0; k < 3; k++) { y[6 * q + k] = x[3 * idx[q] + k]; y[6 * q + 3 + k] = v[3 * idx[q] + k]; }
  bs_ctx c = {p, g, idx, m, alive, rc};
  double remaining = tau, H = tau;
  int halvings = 0, status = 0, steps = 0;
  while (remaining != 0.0) {
    if (fabs(H) > fabs(remaining)) H = remaining;
    int k = bs_attempt(&c, y, H, yn, T, work);
    if (k == 0) {
      H *= 0.5;
      if (++halvings > p->bs_max_halvings) { status = ORC_ST_BS_FAILED; break; }
      continue;
    }
    halvings = 0;
    steps++;
    if (p->collisions) {
      /* contact test over the accepted substep: the encounter test with threshold (R_i+R_j)^2,
       * all pairs tested on the pre-merge states, then merged in ascending pair order */
      int nc = 0;
      int *cp = (int *)xcalloc((size_t)g * g, sizeof(int));
      for (int a = 0; a < g; a++) {
        if (!alive[idx[a]]) continue;
        for (int b = a + 1; b < g; b++) {
          if (!alive[idx[b]]) continue;
          double dx0[3], dv0[3], dx1[3], dv1[3];
          for (int e = 0; e < 3; e++) {
            dx0[e] = y[6 * b + e] - y[6 * a + e];
            dv0[e] = y[6 * b + 3 + e] - y[6 * a + 3 + e];
            dx1[e] = yn[6 * b + e] - yn[6 * a + e];
            dv1[e] = yn[6 * b + 3 + e] - yn[6 * a + 3 + e];
          }
          double rr = R[idx[a]] + R[idx[b]];
          if (orc_hermite_min(dx0, dv0, dx1, dv1, H) < rr * rr) { cp[2 * nc] = a; cp[2 * nc + 1] = b; nc++; }
        }
      }
      for (int e = 0; e < nc; e++) {
        int a = cp[2 * e], b = cp[2 * e + 1];
        if (!alive[idx[a]] || !alive[idx[b]]) continue;
        if (*ncoll < coll_cap) { coll_pairs[2 * *ncoll] = idx[a]; coll_pairs[2 * *ncoll + 1] = idx[b]; }
        (*ncoll)++;
        if (crec && ncrec) {
          /* the report (Sect. 3.2): both bodies' positions, velocities and spins at the last time
           * before the contact, i.e. at the start of this BS substep; step and substep are filled in
           * by the caller */
          if (*ncrec < crec_cap) {
            double *r = crec + ORC_CREC * (size_t)*ncrec;
            int ia = idx[a], ib = idx[b];
            int surv = (m[ia] > m[ib] || (m[ia] == m[ib] && ia < ib)) ? ia : ib;
            r[0] = -1.0; r[1] = -1.0;
            r[2] = tau - remaining;
            r[3] = (double)ia; r[4] = (double)ib;
            for (int k = 0; k < 3; k++) {
              r[5 + k] = y[6 * a + k]; r[8 + k] = y[6 * a + 3 + k]; r[11 + k] = spin ? spin[3 * ia + k] : 0.0;
              r[14 + k] = y[6 * b + k]; r[17 + k] = y[6 * b + 3 + k]; r[20 + k] = spin ? spin[3 * ib + k] : 0.0;
            }
            r[23] = (double)surv;
          }
          (*ncrec)++;
        }
        merge_bodies(p, idx[a], idx[b], yn + 6 * a, yn + 6 * b, m, R, alive, U, spin);
      }
      free(cp);
    }
    memcpy(y, yn, sizeof(double) * d);
    remaining -= H;
    H *= 2.0;
  }
  for (int q = 0; q < g; q++)
    for (int k = 0; k < 3; k++) { x[3 * idx[q] + k] = y[6 * q + k]; v[3 * idx[q] + k] = y[6 * q + 3 + k]; }
  if (bs_steps) *bs_steps += steps;
  free(y); free(yn); free(T); free(work);
  return status;
}

/* ------------------------------------------------------------------------------------------ */
/* Energy (Sect. 4.1): E = sum m v^2/2 + |P|^2/(2 m0) - sum G m0 m/|x| - sum_{i<j} G m_i m_j/r_ij  */
/* ------------------------------------------------------------------------------------------ */

double orc_energy(int n, const orc_params *p, const double *m, const int *alive, const double *x,
                  const double *v) {
  double E = 0.0, P[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < n; i++) {
    if (!alive[i]) continue;
    const double *xi = x + 3 * i, *vi = v + 3 * i;
    double v2 = vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2];
    double r = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    E += 0.5 * m[i] * v2 - p->G * p->m0 * m[i] / r;
    for (int k = 0; k < 3; k++) P[k] += m[i] * vi[k];
  }
  E += (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / (2.0 * p->m0);
  for (int i = 0; i < n; i++) {
    if (!alive[i]) continue;
    for (int j = i + 1; j < n; j++) {
      if (!alive[j]) continue;
      double dx = x[3 * j] - x[3 * i], dy = x[3 * j + 1] - x[3 * i + 1], dz = x[3 * j + 2] - x[3 * i + 2];
      E -= p->G * m[i] * m[j] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  }
  return E;
}

/* ------------------------------------------------------------------------------------------ */
/* Whole step (Sect. 2.2 lists, Eq. z1) and Yoshida compositions (Sect. 2.3)                    */
/* ------------------------------------------------------------------------------------------ */

#define ORC_MAXSUB 7
#define ORC_NSTATS 12

struct orc_sim {
  int n;
  orc_params p;
  double *m, *R, *x, *v, *a, *rc, *x0, *v0;
  int *alive, *fail;
  int *cand, ncand, cand_cap;
  int *enc[ORC_MAXSUB], nenc[ORC_MAXSUB];
  int *gstart[ORC_MAXSUB], *gmem[ORC_MAXSUB], ngroups[ORC_MAXSUB];
  int nsub_last;
  int *coll, ncoll, coll_cap;
  double *spin;                  /* spin angular momentum per body [3n] (Sect. 3.2, Collisions) */
  double *crec;                  /* collision reports, ORC_CREC doubles each (orc_get_collision_records) */
  int ncrec, crec_cap;
  double *ej;                    /* ejection records, 8 doubles each (orc_get_ejections) */
  int nej, ej_cap;
  unsigned char *is_cand;
  double U;
  long long stats[ORC_NSTATS];
};

/* Substep weights: 2nd order is Eq. z1 itself; 4th order is S(w1 t) S(w0 t) S(w1 t) with
 * w1 = 1/(2 - 2^(1/3)), w0 = -2^(1/3)/(2 - 2^(1/3)); 6th order is Yoshida's (1990) solution A. */
int orc_substep_weights(int order, double *w) {
  if (order == 4) {
    double c = cbrt(2.0);
    w[0] = w[2] = 1.0 / (2.0 - c);
    w[1] = -c / (2.0 - c);
    return 3;
  }
  if (order == 6) {
    double w1 = -1.17767998417887, w2 = 0.235573213359357, w3 = 0.784513610477560;
    double w0 = 1.0 - 2.0 * (w1 + w2 + w3);
    w[0] = w3; w[1] = w2; w[2] = w1; w[3] = w0; w[4] = w1; w[5] = w2; w[6] = w3;
    return 7;
  }
  w[0] = 1.0;
  return 1;
}

orc_sim *orc_create(int n, const orc_params *p, const double *m, const double *R, const double *xh,
                    const double *vh) {
  orc_sim *s = (orc_sim *)xcalloc(1, sizeof(orc_sim));
  s->n = n;
  s->p = *p;
  s->m = (double *)xcalloc((size_t)n, sizeof(double));
  s->R = (double *)xcalloc((size_t)n, sizeof(double));
  s->x = (double *)xcalloc((size_t)3 * n, sizeof(double));
  s->v = (double *)xcalloc((size_t)3 * n, sizeof(double));
  s->a = (double *)xcalloc((size_t)3 * n, sizeof(double));
  s->x0 = (double *)xcalloc((size_t)3 * n, sizeof(double));
  s->v0 = (double *)xcalloc((size_t)3 * n, sizeof(double));
  s->rc = (double *)xcalloc((size_t)n, sizeof(double));
  s->alive = (int *)xcalloc((size_t)n, sizeof(int));
  s->fail = (int *)xcalloc((size_t)n, sizeof(int));
  s->is_cand = (unsigned char *)xcalloc((size_t)n * n, 1);
  s->cand_cap = n > 1 ? n * (n - 1) / 2 : 1;
  s->cand = (int *)xcalloc((size_t)2 * s->cand_cap, sizeof(int));
  for (int k = 0; k < ORC_MAXSUB; k++) {
    s->enc[k] = (int *)xcalloc((size_t)2 * s->cand_cap, sizeof(int));
    s->gstart[k] = (int *)xcalloc((size_t)n + 1, sizeof(int));
    s->gmem[k] = (int *)xcalloc((size_t)n, sizeof(int));
  }
  s->coll_cap = n;
  s->coll = (int *)xcalloc((size_t)2 * s->coll_cap, sizeof(int));
  s->spin = (double *)xcalloc((size_t)3 * n, sizeof(double));
  s->crec_cap = n;
  s->crec = (double *)xcalloc((size_t)ORC_CREC * s->crec_cap, sizeof(double));
  s->ej_cap = n + 1;
  s->ej = (double *)xcalloc((size_t)8 * s->ej_cap, sizeof(double));
  /* heliocentric input -> democratic (heliocentric x, barycentric v): v_b = v_h - V_cm,
   * V_cm = sum m_i v_h,i / (m0 + sum m_i) (Sect. 2.1) */
  double M = p->m0, Pm[3] = {0, 0, 0};
  for (int i = 0; i < n; i++) {
    s->m[i] = m[i];
    s->R[i] = R[i];
    s->alive[i] = 1;
    M += m[i];
    for (int k = 0; k < 3; k++) Pm[k] += m[i] * vh[3 * i + k];
  }
  for (int i = 0; i < n; i++)
    for (int k = 0; k < 3; k++) {
      s->x[3 * i + k] = xh[3 * i + k];
      s->v[3 * i + k] = vh[3 * i + k] - Pm[k] / M;
    }
  /* the very first kick is computed on its own (Sect. 2.2): accelerations and candidates */
  orc_rcrit(n, &s->p, fabs(p->dt), s->m, s->alive, s->x, s->v, s->rc);
  orc_accel_B(n, &s->p, s->m, s->alive, s->x, s->rc, s->a);
  s->ncand = orc_precheck(n, &s->p, s->alive, s->x, s->rc, s->cand, s->cand_cap);
  return s;
}

void orc_free(orc_sim *s) {
  if (!s) return;
  free(s->m); free(s->R); free(s->x); free(s->v); free(s->a); free(s->x0); free(s->v0);
  free(s->rc); free(s->alive); free(s->fail); free(s->is_cand); free(s->cand); free(s->coll); free(s->ej);
  free(s->spin); free(s->crec);
  for (int k = 0; k < ORC_MAXSUB; k++) { free(s->enc[k]); free(s->gstart[k]); free(s->gmem[k]); }
  free(s);
}

/* One 2nd-order substep of signed length tau (Sect. 2.2, second list), entered after the
 * opening kick's accelerations s->a are known; leaves the closing kick's accelerations and the
 * new candidate list behind (with precheck_substeps = 0 only the last substep of a step, last = 1,
 * replaces the candidate list: Sect. 2.3 applies the full scheme to each substep "but not the
 * prechecker"). */
static int substep(orc_sim *s, int js, double tau, int last) {
  int n = s->n, st = 0;
  orc_params *p = &s->p;
  double h = 0.5 * tau, P[3];
  /* opening kick tau/2 */
  for (int k = 0; k < 3 * n; k++) s->v[k] += h * s->a[k];
  /* Sun drift tau/2 */
  orc_momentum(n, s->m, s->alive, s->v, P);
  orc_sun_drift(n, p, s->alive, s->x, P, h);
  /* Kepler drift tau, keeping the pre-drift state */
  memcpy(s->x0, s->x, sizeof(double) * 3 * n);
  memcpy(s->v0, s->v, sizeof(double) * 3 * n);
  double mu = p->G * p->m0;
  for (int i = 0; i < n; i++) {
    s->fail[i] = 0;
    if (!s->alive[i]) continue;
    int it = 0;
    if (orc_kepler_drift(mu, s->x + 3 * i, s->v + 3 * i, tau, p->kepler_maxit, &it)) {
      s->fail[i] = 1;
      s->stats[6]++;
      st |= ORC_ST_KEPLER_FALLBACK;
    }
    s->stats[9] += it;
  }
  /* close-encounter search over the candidates of the previous closing kick */
  int ne = orc_encounters(n, s->alive, s->x0, s->v0, s->x, s->v, s->rc, s->cand, s->ncand, tau,
                          s->enc[js], s->cand_cap);
  s->nenc[js] = ne;
  s->stats[3] += ne;
  /* groups, then Bulirsch-Stoer from the pre-drift state over tau; collisions inside */
  int ng = orc_groups(n, s->enc[js], ne, s->fail, s->gstart[js], s->gmem[js]);
  s->ngroups[js] = ng;
  s->stats[4] += ng;
  for (int gk = 0; gk < ng; gk++) {
    int g0 = s->gstart[js][gk], g = s->gstart[js][gk + 1] - g0;
    const int *idx = s->gmem[js] + g0;
    for (int q = 0; q < g; q++)
      for (int c = 0; c < 3; c++) {
        s->x[3 * idx[q] + c] = s->x0[3 * idx[q] + c];
        s->v[3 * idx[q] + c] = s->v0[3 * idx[q] + c];
      }
    int bs_steps = 0, nc0 = s->ncoll, nr0 = s->ncrec;
    st |= orc_bs_group_rec(n, p, g, idx, tau, s->m, s->R, s->alive, s->x, s->v, s->rc, &s->U,
                           &s->ncoll, s->coll, s->coll_cap, &bs_steps, s->spin, s->crec, s->crec_cap,
                           &s->ncrec);
    for (int r = nr0; r < s->ncrec && r < s->crec_cap; r++) {
      s->crec[ORC_CREC * (size_t)r] = (double)(s->stats[0] + 1);
      s->crec[ORC_CREC * (size_t)r + 1] = (double)js;
    }
    s->stats[5] += bs_steps;
    s->stats[7] += s->ncoll - nc0;
  }
  /* Sun drift tau/2 */
  orc_momentum(n, s->m, s->alive, s->v, P);
  orc_sun_drift(n, p, s->alive, s->x, P, h);
  /* closing kick tau/2 with new accelerations and the precheck */
  orc_accel_B(n, p, s->m, s->alive, s->x, s->rc, s->a);
  for (int k = 0; k < 3 * n; k++) s->v[k] += h * s->a[k];
  if (p->precheck_substeps || last) {
    s->ncand = orc_precheck(n, p, s->alive, s->x, s->rc, s->cand, s->cand_cap);
    if (s->ncand > s->cand_cap) st |= ORC_ST_CAPACITY;
    s->stats[2] += s->ncand;
  }
  s->stats[1]++;
  return st;
}

/* Ejections (Sect. 3.2): at the end of a step a body farther than rcut from the central mass, or
 * closer than rcut_sun, is removed -- a ghost, as after a merger -- and its position and
 * heliocentric velocity are recorded. The energy it takes away is booked into U (U += E before the
 * removals - E after them), as for a merger, so that E + U does not jump. */
static int eject(orc_sim *s) {
  const orc_params *p = &s->p;
  if (!(p->rcut > 0.0) && !(p->rcut_sun > 0.0)) return 0;
  int n = s->n, nout = 0;
  double E0 = 0.0, P[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < n; i++) {
    if (!s->alive[i]) continue;
    const double *x = s->x + 3 * i;
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    int out = (p->rcut > 0.0 && r2 > p->rcut * p->rcut) || (p->rcut_sun > 0.0 && r2 < p->rcut_sun * p->rcut_sun);
    if (!out) continue;
    if (nout == 0) {  /* the state before any removal */
      E0 = orc_energy(n, p, s->m, s->alive, s->x, s->v);
      orc_momentum(n, s->m, s->alive, s->v, P);
    }
    if (s->nej < s->ej_cap) {
      double *rec = s->ej + 8 * s->nej;
      rec[0] = (double)i;
      rec[1] = (double)s->stats[0];
      for (int k = 0; k < 3; k++) { rec[2 + k] = x[k]; rec[5 + k] = s->v[3 * i + k] + P[k] / p->m0; }
    }
    s->nej++;
    nout++;
  }
  if (!nout) return 0;
  /* remove after the scan: every test above saw the state at the end of the step */
  for (int q = s->nej - nout; q < s->nej && q < s->ej_cap; q++) {
    int i = (int)s->ej[8 * q];
    s->alive[i] = 0;
    s->m[i] = 0.0;
    s->R[i] = 0.0;
  }
  s->U += E0 - orc_energy(n, p, s->m, s->alive, s->x, s->v);
  s->stats[11] += nout;
  return nout;
}

int orc_get_ejections(const orc_sim *s, double *rec, int cap) {
  int k = s->nej < s->ej_cap ? s->nej : s->ej_cap;
  if (rec) memcpy(rec, s->ej, sizeof(double) * 8 * (size_t)(k < cap ? k : cap));
  return s->nej;
}

int orc_step(orc_sim *s, int nsteps) {
  int n = s->n, st = 0;
  double w[ORC_MAXSUB];
  int nsub = orc_substep_weights(s->p.order, w);
  for (int it = 0; it < nsteps; it++) {
    /* critical radii once per full step, from the state at its start */
    orc_rcrit(n, &s->p, fabs(s->p.dt), s->m, s->alive, s->x, s->v, s->rc);
    /* record whether reusing the last closing kick for non-candidate pairs is exact, i.e.
     * K(r; new rcrit) = 1 for every pair the prechecker did not flag */
    memset(s->is_cand, 0, (size_t)n * n);
    for (int k = 0; k < s->ncand && k < s->cand_cap; k++)
      s->is_cand[(size_t)s->cand[2 * k] * n + s->cand[2 * k + 1]] = 1;
    long long viol = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : viol)
#endif
    for (int i = 0; i < n; i++) {
      if (!s->alive[i]) continue;
      for (int j = i + 1; j < n; j++) {
        if (!s->alive[j] || s->is_cand[(size_t)i * n + j]) continue;
        double dx = s->x[3 * j] - s->x[3 * i], dy = s->x[3 * j + 1] - s->x[3 * i + 1],
               dz = s->x[3 * j + 2] - s->x[3 * i + 2];
        double rcij = s->rc[i] > s->rc[j] ? s->rc[i] : s->rc[j];
        if (orc_weight_B(pair_r2(dx, dy, dz), rcij, s->p.kmode) != 1.0) viol++;
      }
    }
    s->stats[8] += viol;
    if (viol) st |= ORC_ST_REUSE_VIOLATION;
    /* opening kick of the step: plain definition, all pairs with the new critical radii */
    orc_accel_B(n, &s->p, s->m, s->alive, s->x, s->rc, s->a);
    for (int js = 0; js < nsub; js++) st |= substep(s, js, w[js] * s->p.dt, js == nsub - 1);
    s->nsub_last = nsub;
    s->stats[0]++;
    eject(s);
  }
  s->stats[10] |= st;
  return st;
}

void orc_get_state(const orc_sim *s, double *xh, double *vh, double *m, double *R, int *alive) {
  double P[3];
  orc_momentum(s->n, s->m, s->alive, s->v, P);
  for (int i = 0; i < s->n; i++) {
    for (int k = 0; k < 3; k++) {
      if (xh) xh[3 * i + k] = s->x[3 * i + k];
      if (vh) vh[3 * i + k] = s->v[3 * i + k] + P[k] / s->p.m0; /* v_h = v_b + P/m0 */
    }
    if (m) m[i] = s->m[i];
    if (R) R[i] = s->R[i];
    if (alive) alive[i] = s->alive[i];
  }
}

void orc_get_internal(const orc_sim *s, double *x, double *v, double *a, double *rc) {
  size_t n = (size_t)s->n;
  if (x) memcpy(x, s->x, sizeof(double) * 3 * n);
  if (v) memcpy(v, s->v, sizeof(double) * 3 * n);
  if (a) memcpy(a, s->a, sizeof(double) * 3 * n);
  if (rc) memcpy(rc, s->rc, sizeof(double) * n);
}

double orc_get_energy(const orc_sim *s, double *U) {
  if (U) *U = s->U;
  return orc_energy(s->n, &s->p, s->m, s->alive, s->x, s->v);
}

int orc_get_candidates(const orc_sim *s, int *pairs, int cap) {
  int c = s->ncand < cap ? s->ncand : cap;
  if (pairs) memcpy(pairs, s->cand, sizeof(int) * 2 * (size_t)c);
  return s->ncand;
}

int orc_get_encounters(const orc_sim *s, int substep_idx, int *pairs, int cap) {
  if (substep_idx < 0) substep_idx = s->nsub_last - 1;
  if (substep_idx < 0 || substep_idx >= s->nsub_last) return 0;
  int ne = s->nenc[substep_idx];
  int c = ne < cap ? ne : cap;
  if (pairs) memcpy(pairs, s->enc[substep_idx], sizeof(int) * 2 * (size_t)c);
  return ne;
}

int orc_get_groups(const orc_sim *s, int substep_idx, int *group_start, int *members, int cap) {
  if (substep_idx < 0) substep_idx = s->nsub_last - 1;
  if (substep_idx < 0 || substep_idx >= s->nsub_last) return 0;
  int ng = s->ngroups[substep_idx];
  if (group_start) memcpy(group_start, s->gstart[substep_idx], sizeof(int) * (size_t)(ng + 1));
  int nm = s->gstart[substep_idx][ng];
  if (members) memcpy(members, s->gmem[substep_idx], sizeof(int) * (size_t)(nm < cap ? nm : cap));
  return ng;
}

void orc_get_stats(const orc_sim *s, long long *stats, int nstats) {
  for (int k = 0; k < nstats && k < ORC_NSTATS; k++) stats[k] = s->stats[k];
}

int orc_get_collisions(const orc_sim *s, int *pairs, int cap) {
  int c = s->ncoll < cap ? s->ncoll : cap;
  if (pairs) memcpy(pairs, s->coll, sizeof(int) * 2 * (size_t)c);
  return s->ncoll;
}

int orc_get_collision_records(const orc_sim *s, double *rec, int cap) {
  int k = s->ncrec < s->crec_cap ? s->ncrec : s->crec_cap;
  if (rec) memcpy(rec, s->crec, sizeof(double) * ORC_CREC * (size_t)(k < cap ? k : cap));
  return s->ncrec;
}

void orc_set_spin(orc_sim *s, const double *spin) { memcpy(s->spin, spin, sizeof(double) * 3 * (size_t)s->n); }

void orc_get_spin(const orc_sim *s, double *spin) { memcpy(spin, s->spin, sizeof(double) * 3 * (size_t)s->n); }

/* ------------------------------------------------------------------------------------------ */
/* Sect. 3.3: test-particle mode                                                               */
/* ------------------------------------------------------------------------------------------ */
/*
 * Massless test particles (TPs) are perturbed by the massive bodies and never by each other; the
 * massive bodies evolve exactly as without TPs. Each TP takes the same operators as a massive body
 * (K-weighted kick with the prechecker, Sun drift with the momentum of the massive bodies, Kepler
 * drift). A TP whose Hermite test confirms an encounter with a planet is integrated by BS alone,
 * from its pre-drift state, in the field of m0 and the (1 - W_B)-weighted pull of the planets it
 * encounters; those planets keep their Kepler-drift ("FG") path, evaluated at the BS times by a
 * Kepler drift from their pre-drift state (Sect. 3.3: only the TP is updated, the planetesimal
 * keeps the coordinates from the FG kernel). A TP whose BS substep brings it within R_tp + R_p of
 * an encountered planet (Hermite contact test) is removed. The TP critical radius has no Hill term
 * (m = 0): rc_tp = n2 |tau| |v_tp|; a TP-planet pair uses max(rc_tp, rc_p).
 */
#define ORC_TP_NSTATS 8
#define ORC_TP_MAXPL 32

static void tp_rcrit(orc_tpsim *T);
static void tp_accel(const orc_sim *s, const double *x, double rct, double *a);
static unsigned tp_precheck(const orc_sim *s, const double *x, double rct);

struct orc_tpsim {
  orc_sim *s;
  int nt;
  double *x, *v, *x0, *v0, *R, *rc, *a;
  int *alive;
  unsigned *cmask;               /* per TP: planets flagged by the last closing kick's precheck */
  double *xp0, *vp0, *xpf, *vpf; /* planets: pre-drift state, Kepler-drift result */
  int *enc[ORC_MAXSUB], nenc[ORC_MAXSUB];
  long long stats[ORC_TP_NSTATS]; /* candidates, encounters, BS steps, removed, BS failures, ejected */
};

orc_tpsim *orc_tp_create(int n, const orc_params *p, const double *m, const double *R, const double *xh,
                         const double *vh, int ntp, const double *xt, const double *vt, const double *Rt) {
  if (n > ORC_TP_MAXPL) return NULL;
  orc_tpsim *t = (orc_tpsim *)xcalloc(1, sizeof(orc_tpsim));
  t->s = orc_create(n, p, m, R, xh, vh);
  t->nt = ntp;
  t->x = (double *)xcalloc((size_t)3 * ntp, sizeof(double));
  t->v = (double *)xcalloc((size_t)3 * ntp, sizeof(double));
  t->x0 = (double *)xcalloc((size_t)3 * ntp, sizeof(double));
  t->v0 = (double *)xcalloc((size_t)3 * ntp, sizeof(double));
  t->a = (double *)xcalloc((size_t)3 * ntp, sizeof(double));
  t->R = (double *)xcalloc((size_t)ntp, sizeof(double));
  t->rc = (double *)xcalloc((size_t)ntp, sizeof(double));
  t->alive = (int *)xcalloc((size_t)ntp, sizeof(int));
  t->cmask = (unsigned *)xcalloc((size_t)ntp + 1, sizeof(unsigned));
  t->xp0 = (double *)xcalloc((size_t)3 * n + 3, sizeof(double));
  t->vp0 = (double *)xcalloc((size_t)3 * n + 3, sizeof(double));
  t->xpf = (double *)xcalloc((size_t)3 * n + 3, sizeof(double));
  t->vpf = (double *)xcalloc((size_t)3 * n + 3, sizeof(double));
  for (int k = 0; k < ORC_MAXSUB; k++) t->enc[k] = (int *)xcalloc((size_t)2 * ntp * (n > 0 ? n : 1) + 2, sizeof(int));
  /* the TPs' velocities become barycentric with the same shift as the massive bodies (Sect. 2.1):
   * v_b = v_h - sum m v_h / (m0 + sum m) over the massive bodies */
  double M = p->m0, Pm[3] = {0, 0, 0};
  for (int i = 0; i < n; i++) {
    M += m[i];
    for (int k = 0; k < 3; k++) Pm[k] += m[i] * vh[3 * i + k];
  }
  for (int i = 0; i < ntp; i++) {
    t->alive[i] = 1;
    t->R[i] = Rt ? Rt[i] : 0.0;
    for (int k = 0; k < 3; k++) { t->x[3 * i + k] = xt[3 * i + k]; t->v[3 * i + k] = vt[3 * i + k] - Pm[k] / M; }
  }
  /* the very first TP kick: accelerations and candidates with the initial critical radii */
  tp_rcrit(t);
  for (int i = 0; i < ntp; i++) {
    tp_accel(t->s, t->x + 3 * i, t->rc[i], t->a + 3 * i);
    t->cmask[i] = tp_precheck(t->s, t->x + 3 * i, t->rc[i]);
  }
  return t;
}

void orc_tp_free(orc_tpsim *t) {
  if (!t) return;
  orc_free(t->s);
  free(t->x); free(t->v); free(t->x0); free(t->v0); free(t->a); free(t->R); free(t->rc); free(t->alive);
  free(t->cmask);
  free(t->xp0); free(t->vp0); free(t->xpf); free(t->vpf);
  for (int k = 0; k < ORC_MAXSUB; k++) free(t->enc[k]);
  free(t);
}

/* TP precheck (Sect. 2.2): planet j is a candidate if r^2 < max((pc rc_tp)^2, (pc rc_j)^2). */
static unsigned tp_precheck(const orc_sim *s, const double *x, double rct) {
  unsigned mask = 0;
  double t = s->p.pc * rct, Tt = t * t;
  for (int j = 0; j < s->n; j++) {
    if (!s->alive[j]) continue;
    double tj = s->p.pc * s->rc[j], Tj = tj * tj;
    double T = Tt > Tj ? Tt : Tj;
    double dx = s->x[3 * j] - x[0], dy = s->x[3 * j + 1] - x[1], dz = s->x[3 * j + 2] - x[2];
    if (pair_r2(dx, dy, dz) < T) mask |= 1u << j;
  }
  return mask;
}

/* TP acceleration: a = sum_p G m_p W_B(r, max(rc_tp, rc_p)) (x_p - x)/r^3 over the live planets. */
static void tp_accel(const orc_sim *s, const double *x, double rct, double *a) {
  const orc_params *p = &s->p;
  a[0] = a[1] = a[2] = 0.0;
  for (int j = 0; j < s->n; j++) {
    if (!s->alive[j]) continue;
    double dx = s->x[3 * j] - x[0], dy = s->x[3 * j + 1] - x[1], dz = s->x[3 * j + 2] - x[2];
    double r2 = pair_r2(dx, dy, dz);
    double rcij = rct > s->rc[j] ? rct : s->rc[j];
    double w = orc_weight_B(r2, rcij, p->kmode);
    double r = sqrt(r2);
    double f = p->G * s->m[j] * w / (r2 * r);
    a[0] += f * dx; a[1] += f * dy; a[2] += f * dz;
  }
}

/* Right-hand side of a TP in BS at time t within the substep: central mass plus the (1 - W_B) pull
 * of the encountered planets (mask) on their Kepler paths from the pre-drift state. */
static void tp_bs_deriv(const orc_tpsim *T, unsigned mask, double rct, double t, const double *y, double *dy) {
  const orc_sim *s = T->s;
  const orc_params *p = &s->p;
  dy[0] = y[3]; dy[1] = y[4]; dy[2] = y[5];
  double r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
  double r = sqrt(r2);
  double f = p->G * p->m0 / (r2 * r);
  double ax = -f * y[0], ay = -f * y[1], az = -f * y[2];
  for (int j = 0; j < s->n; j++) {
    if (!(mask & (1u << j))) continue;
    double xp[3] = {T->xp0[3 * j], T->xp0[3 * j + 1], T->xp0[3 * j + 2]};
    double vp[3] = {T->vp0[3 * j], T->vp0[3 * j + 1], T->vp0[3 * j + 2]};
    orc_kepler_drift(p->G * p->m0, xp, vp, t, p->kepler_maxit, NULL);
    double dx = xp[0] - y[0], dyy = xp[1] - y[1], dz = xp[2] - y[2];
    double pr2 = pair_r2(dx, dyy, dz);
    double rcij = rct > s->rc[j] ? rct : s->rc[j];
    double wa = 1.0 - orc_weight_B(pr2, rcij, p->kmode);
    if (wa == 0.0) continue;
    double pr = sqrt(pr2);
    double fp = p->G * s->m[j] * wa / (pr2 * pr);
    ax += fp * dx; ay += fp * dyy; az += fp * dz;
  }
  dy[3] = ax; dy[4] = ay; dy[5] = az;
}

/* BS of one TP over tau from (x, v): the same controller as orc_bs_group (n_k = 2k, Neville in
 * h^2, error |dx|/|x| and |dv|/|v| <= eps, halving on failure, doubling after acceptance), then the
 * contact test against the encountered planets after every accepted substep. Returns 0, 1 (removed
 * by a collision) or ORC_ST_BS_FAILED. */
static int tp_bs(orc_tpsim *T, int it, unsigned mask, double tau, int *steps) {
  const orc_sim *s = T->s;
  const orc_params *p = &s->p;
  const int kmax = p->bs_kmax;
  double y[6], yn[6], dy0[6], za[6], zb[6], f[6], sc[6];
  double Tt[9][9][6];
  for (int k = 0; k < 3; k++) { y[k] = T->x0[3 * it + k]; y[3 + k] = T->v0[3 * it + k]; }
  double rct = T->rc[it], t0 = 0.0, remaining = tau, H = tau;
  int halvings = 0;
  while (remaining != 0.0) {
    if (fabs(H) > fabs(remaining)) H = remaining;
    tp_bs_deriv(T, mask, rct, t0, y, dy0);
    double sx = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]), sv = sqrt(y[3] * y[3] + y[4] * y[4] + y[5] * y[5]);
    if (!(sx > 0.0)) sx = DBL_MIN;
    if (!(sv > 0.0)) sv = DBL_MIN;
    for (int k = 0; k < 3; k++) { sc[k] = sx; sc[3 + k] = sv; }
    int acc = 0;
    for (int k = 1; k <= kmax && !acc; k++) {
      int nk = 2 * k;
      double h = H / nk;
      for (int e = 0; e < 6; e++) { za[e] = y[e]; zb[e] = y[e] + h * dy0[e]; }
      for (int m = 1; m < nk; m++) {
        tp_bs_deriv(T, mask, rct, t0 + m * h, zb, f);
        for (int e = 0; e < 6; e++) { double tt = za[e] + 2.0 * h * f[e]; za[e] = zb[e]; zb[e] = tt; }
      }
      tp_bs_deriv(T, mask, rct, t0 + H, zb, f);
      for (int e = 0; e < 6; e++) Tt[k][1][e] = 0.5 * (zb[e] + za[e] + h * f[e]);
      for (int j = 1; j < k; j++) {
        double ratio = (double)k / (double)(k - j), fac = ratio * ratio - 1.0;
        for (int e = 0; e < 6; e++) Tt[k][j + 1][e] = Tt[k][j][e] + (Tt[k][j][e] - Tt[k - 1][j][e]) / fac;
      }
      if (k >= 2) {
        double err = 0.0;
        for (int e = 0; e < 6; e++) {
          double ee = fabs(Tt[k][k][e] - Tt[k][k - 1][e]) / sc[e];
          if (!(ee <= err)) err = ee;
        }
        if (err <= p->bs_eps) { memcpy(yn, Tt[k][k], sizeof yn); acc = 1; }
      }
    }
    if (!acc) {
      H *= 0.5;
      if (++halvings > p->bs_max_halvings) {
        for (int k = 0; k < 3; k++) { T->x[3 * it + k] = y[k]; T->v[3 * it + k] = y[3 + k]; }
        return ORC_ST_BS_FAILED;
      }
      continue;
    }
    halvings = 0;
    (*steps)++;
    if (p->collisions) { /* contact with an encountered planet during the substep: the TP is removed */
      for (int j = 0; j < s->n; j++) {
        if (!(mask & (1u << j))) continue;
        double xa[3] = {T->xp0[3 * j], T->xp0[3 * j + 1], T->xp0[3 * j + 2]}, va[3] = {T->vp0[3 * j], T->vp0[3 * j + 1], T->vp0[3 * j + 2]};
        double xb[3] = {xa[0], xa[1], xa[2]}, vb[3] = {va[0], va[1], va[2]};
        orc_kepler_drift(p->G * p->m0, xa, va, t0, p->kepler_maxit, NULL);
        orc_kepler_drift(p->G * p->m0, xb, vb, t0 + H, p->kepler_maxit, NULL);
        double dx0[3], dv0[3], dx1[3], dv1[3];
        for (int e = 0; e < 3; e++) {
          dx0[e] = xa[e] - y[e]; dv0[e] = va[e] - y[3 + e];
          dx1[e] = xb[e] - yn[e]; dv1[e] = vb[e] - yn[3 + e];
        }
        double rr = T->R[it] + s->R[j];
        if (orc_hermite_min(dx0, dv0, dx1, dv1, H) < rr * rr) {
          T->alive[it] = 0;
          for (int k = 0; k < 3; k++) { T->x[3 * it + k] = yn[k]; T->v[3 * it + k] = yn[3 + k]; }
          return 1;
        }
      }
    }
    memcpy(y, yn, sizeof y);
    t0 += H;
    remaining -= H;
    H *= 2.0;
  }
  for (int k = 0; k < 3; k++) { T->x[3 * it + k] = y[k]; T->v[3 * it + k] = y[3 + k]; }
  return 0;
}

/* One 2nd-order substep of the massive bodies (as in substep()) with the TPs interleaved. */
static int tp_substep(orc_tpsim *T, int js, double tau) {
  orc_sim *s = T->s;
  orc_params *p = &s->p;
  int n = s->n, st = 0;
  double h = 0.5 * tau, P[3];
  /* opening kicks */
  for (int k = 0; k < 3 * n; k++) s->v[k] += h * s->a[k];
  for (int k = 0; k < 3 * T->nt; k++) T->v[k] += h * T->a[k];
  /* Sun drift with the massive momentum */
  orc_momentum(n, s->m, s->alive, s->v, P);
  orc_sun_drift(n, p, s->alive, s->x, P, h);
  orc_sun_drift(T->nt, p, T->alive, T->x, P, h);
  /* Kepler drifts, keeping the pre-drift states */
  memcpy(s->x0, s->x, sizeof(double) * 3 * n);
  memcpy(s->v0, s->v, sizeof(double) * 3 * n);
  memcpy(T->x0, T->x, sizeof(double) * 3 * T->nt);
  memcpy(T->v0, T->v, sizeof(double) * 3 * T->nt);
  double mu = p->G * p->m0;
  for (int i = 0; i < n; i++) {
    s->fail[i] = 0;
    if (!s->alive[i]) continue;
    int it = 0;
    if (orc_kepler_drift(mu, s->x + 3 * i, s->v + 3 * i, tau, p->kepler_maxit, &it)) { s->fail[i] = 1; st |= ORC_ST_KEPLER_FALLBACK; }
  }
  memcpy(T->xp0, s->x0, sizeof(double) * 3 * n);
  memcpy(T->vp0, s->v0, sizeof(double) * 3 * n);
  memcpy(T->xpf, s->x, sizeof(double) * 3 * n);
  memcpy(T->vpf, s->v, sizeof(double) * 3 * n);
  int *tfail = (int *)xcalloc((size_t)T->nt + 1, sizeof(int));
  for (int i = 0; i < T->nt; i++) {
    if (!T->alive[i]) continue;
    if (orc_kepler_drift(mu, T->x + 3 * i, T->v + 3 * i, tau, p->kepler_maxit, NULL)) { tfail[i] = 1; st |= ORC_ST_KEPLER_FALLBACK; }
  }
  /* massive encounters, groups, BS (as in substep()) */
  int ne = orc_encounters(n, s->alive, s->x0, s->v0, s->x, s->v, s->rc, s->cand, s->ncand, tau, s->enc[js], s->cand_cap);
  s->nenc[js] = ne;
  int ng = orc_groups(n, s->enc[js], ne, s->fail, s->gstart[js], s->gmem[js]);
  s->ngroups[js] = ng;
  for (int gk = 0; gk < ng; gk++) {
    int g0 = s->gstart[js][gk], g = s->gstart[js][gk + 1] - g0;
    const int *idx = s->gmem[js] + g0;
    for (int q = 0; q < g; q++)
      for (int c = 0; c < 3; c++) { s->x[3 * idx[q] + c] = s->x0[3 * idx[q] + c]; s->v[3 * idx[q] + c] = s->v0[3 * idx[q] + c]; }
    int bs_steps = 0, nr0 = s->ncrec;
    st |= orc_bs_group_rec(n, p, g, idx, tau, s->m, s->R, s->alive, s->x, s->v, s->rc, &s->U, &s->ncoll, s->coll,
                           s->coll_cap, &bs_steps, s->spin, s->crec, s->crec_cap, &s->ncrec);
    for (int r = nr0; r < s->ncrec && r < s->crec_cap; r++) {
      s->crec[ORC_CREC * (size_t)r] = (double)(s->stats[0] + 1);
      s->crec[ORC_CREC * (size_t)r + 1] = (double)js;
    }
  }
  /* TP encounters with planets (candidates from the previous closing TP kick), then BS of every
   * TP with an encounter (or a failed Kepler solve) */
  int nte = 0;
  for (int i = 0; i < T->nt; i++) {
    if (!T->alive[i]) continue;
    unsigned emask = 0;
    for (int j = 0; j < n; j++) {
      if (!(T->cmask[i] & (1u << j)) || !s->alive[j]) continue;
      double dx0[3], dv0[3], dx1[3], dv1[3];
      for (int c = 0; c < 3; c++) {
        dx0[c] = T->xp0[3 * j + c] - T->x0[3 * i + c];
        dv0[c] = T->vp0[3 * j + c] - T->v0[3 * i + c];
        dx1[c] = T->xpf[3 * j + c] - T->x[3 * i + c];
        dv1[c] = T->vpf[3 * j + c] - T->v[3 * i + c];
      }
      double dmin = orc_hermite_min(dx0, dv0, dx1, dv1, tau);
      double rcij = T->rc[i] > s->rc[j] ? T->rc[i] : s->rc[j];
      if (dmin < rcij * rcij) {
        emask |= 1u << j;
        T->enc[js][2 * nte] = i;
        T->enc[js][2 * nte + 1] = j;
        nte++;
      }
    }
    if (emask || tfail[i]) {
      int steps = 0;
      int r = tp_bs(T, i, emask, tau, &steps);
      T->stats[2] += steps;
      if (r == 1) T->stats[3]++;
      else if (r) { st |= r; T->stats[4]++; }
    }
  }
  T->nenc[js] = nte;
  T->stats[1] += nte;
  free(tfail);
  /* Sun drift tau/2 */
  orc_momentum(n, s->m, s->alive, s->v, P);
  orc_sun_drift(n, p, s->alive, s->x, P, h);
  orc_sun_drift(T->nt, p, T->alive, T->x, P, h);
  /* closing kicks */
  orc_accel_B(n, p, s->m, s->alive, s->x, s->rc, s->a);
  for (int k = 0; k < 3 * n; k++) s->v[k] += h * s->a[k];
  s->ncand = orc_precheck(n, p, s->alive, s->x, s->rc, s->cand, s->cand_cap);
  for (int i = 0; i < T->nt; i++) {
    T->cmask[i] = 0;
    if (!T->alive[i]) { T->a[3 * i] = T->a[3 * i + 1] = T->a[3 * i + 2] = 0.0; continue; }
    tp_accel(s, T->x + 3 * i, T->rc[i], T->a + 3 * i);
    for (int k = 0; k < 3; k++) T->v[3 * i + k] += h * T->a[3 * i + k];
    T->cmask[i] = tp_precheck(s, T->x + 3 * i, T->rc[i]);
    T->stats[0] += __builtin_popcount(T->cmask[i]);
  }
  return st;
}

/* TP critical radii: Eq. rcrit with m = 0 (no Hill term): n2 |tau| |v|. */
static void tp_rcrit(orc_tpsim *T) {
  orc_sim *s = T->s;
  double *m0s = (double *)xcalloc((size_t)T->nt + 1, sizeof(double));
  orc_rcrit(T->nt, &s->p, fabs(s->p.dt), m0s, T->alive, T->x, T->v, T->rc);
  free(m0s);
}

int orc_tp_step(orc_tpsim *T, int nsteps) {
  orc_sim *s = T->s;
  int n = s->n, st = 0;
  double w[ORC_MAXSUB];
  int nsub = orc_substep_weights(s->p.order, w);
  for (int it = 0; it < nsteps; it++) {
    orc_rcrit(n, &s->p, fabs(s->p.dt), s->m, s->alive, s->x, s->v, s->rc);
    tp_rcrit(T);
    /* opening kicks of the step: plain definition, all pairs with the new critical radii */
    orc_accel_B(n, &s->p, s->m, s->alive, s->x, s->rc, s->a);
    for (int i = 0; i < T->nt; i++) {
      if (T->alive[i]) tp_accel(s, T->x + 3 * i, T->rc[i], T->a + 3 * i);
      else T->a[3 * i] = T->a[3 * i + 1] = T->a[3 * i + 2] = 0.0;
    }
    for (int js = 0; js < nsub; js++) st |= tp_substep(T, js, w[js] * s->p.dt);
    s->nsub_last = nsub;
    s->stats[0]++;
    /* ejections at the end of the step: test particles by the same rule (they carry no energy),
     * tested on the positions before any planet is removed, then the planets */
    const orc_params *p = &s->p;
    if (p->rcut > 0.0 || p->rcut_sun > 0.0)
      for (int i = 0; i < T->nt; i++) {
        if (!T->alive[i]) continue;
        const double *x = T->x + 3 * i;
        double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        if ((p->rcut > 0.0 && r2 > p->rcut * p->rcut) || (p->rcut_sun > 0.0 && r2 < p->rcut_sun * p->rcut_sun)) {
          T->alive[i] = 0;
          T->stats[5]++;
        }
      }
    eject(s);
  }
  return st;
}

void orc_tp_get_state(const orc_tpsim *T, double *xh, double *vh, double *m, int *alive, double *xt,
                      double *vt, int *tp_alive) {
  const orc_sim *s = T->s;
  orc_get_state(s, xh, vh, m, NULL, alive);
  double P[3];
  orc_momentum(s->n, s->m, s->alive, s->v, P);
  for (int i = 0; i < T->nt; i++) {
    for (int k = 0; k < 3; k++) {
      if (xt) xt[3 * i + k] = T->x[3 * i + k];
      if (vt) vt[3 * i + k] = T->v[3 * i + k] + P[k] / s->p.m0;
    }
    if (tp_alive) tp_alive[i] = T->alive[i];
  }
}

void orc_tp_get_stats(const orc_tpsim *T, long long *stats, int nstats) {
  for (int k = 0; k < nstats && k < ORC_TP_NSTATS; k++) stats[k] = T->stats[k];
}

int orc_tp_get_ejections(const orc_tpsim *T, double *rec, int cap) { return orc_get_ejections(T->s, rec, cap); }

int orc_tp_get_encounters(const orc_tpsim *T, int substep_idx, int *pairs, int cap) {
  if (substep_idx < 0) substep_idx = T->s->nsub_last - 1;
  if (substep_idx < 0 || substep_idx >= T->s->nsub_last) return 0;
  int ne = T->nenc[substep_idx];
  int c = ne < cap ? ne : cap;
  if (pairs) memcpy(pairs, T->enc[substep_idx], sizeof(int) * 2 * (size_t)c);
  return ne;
}
