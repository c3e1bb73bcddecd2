/*
 * oracle.c -- plain, slow FP64 CPU oracle of the per-timestep force
 * evaluation and time update of the minimal dense-suspension model of
 * Li, Royer & Ness, "Minimal model for dense colloidal suspensions"
 * (arXiv 2307.13802).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the bench's CPU
 * baseline leg call this file; the product library never links or calls it,
 * and it shares no code, header, table or constant generator with the CUDA
 * path.  Everything is double precision, evaluated in the written order
 * (compiled with -ffp-contract=off so no multiply-add is fused).
 *
 * Scope, with the passage each part follows:
 *   - equations of motion, Eq. 1 (lang_force) and Eq. 2 (lang_torque), Sec. II,
 *     advanced by Velocity-Verlet (Sec. II, the paragraph after Eq. 2);
 *   - contact force and torque, Eq. 3 (force_contact), Eq. 4 (torque_contact),
 *     with the Coulomb cap |k_t xi| <= mu k_n delta, Sec. II.A;
 *   - one-body Stokes drag, Eq. 5 (force_drag), Eq. 6 (torque_drag), Sec. II.B;
 *   - pairwise lubrication, Eq. 8 (force_lub), Eqs. 13-14 (torque_lub1/2) with
 *     the scalar resistances Eqs. 9-12 and 15-18, the regularisation
 *     xi_eff = 1e-3 for xi < 1e-3 and the cutoff xi > 0.05, Sec. II.B;
 *   - one-body Brownian force/torque, Eqs. 20-21, and pairwise Brownian
 *     force/torques, Eqs. 22-24, Sec. II.C;
 *   - pair stresses -F (x) r for contact, lubrication and Brownian terms
 *     (Sec. II.A, II.B, II.D) and the drag stresslet (20/3) pi eta a^3 E (Sec. II.B);
 *   - the tilted (Lees-Edwards) box with the strain flip 0.5 -> -0.5, Sec. II.E.
 *
 * Readings taken where the paper is silent or inconsistent (all listed in the
 * design notes of the repository):
 *   - forces are applied as "force on i by j" with i the lower tag and n the
 *     unit vector from i to j; the contact force on i is -k_n delta n + k_t xi_t
 *     (Eq. 3 read as the force on j) and the stress is
 *     sigma = (1/V) sum_pairs F_{i<-j} (x) r_ij (tension positive);
 *   - the chi term of T_ji in Eq. 24 carries the sign `torque_sign`
 *     (default -1, the sign for which the pair noise covariance equals
 *     (2kT/dt) times the pair resistance, Eq. 19);
 *   - xi_eff = max(xi, 1e-3) enters both 1/xi and ln(1/xi), also for
 *     overlapping pairs; lubrication and pair noise act for xi <= 0.05;
 *   - tangential history: projected onto the current tangent plane keeping
 *     its length, incremented by the tangential relative surface velocity
 *     times dt, rescaled to the Coulomb cap, erased when the contact opens;
 *     it is not incremented by an evaluation that does not advance time;
 *   - velocity-dependent forces are evaluated with the half-step velocities
 *     of Velocity-Verlet; U_inf = rate (y - Ly/2) x, Omega_inf = -(rate/2) z;
 *   - noise: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) with
 *     counter (k_lo, tag_i, tag_j, 2 k_hi + block), key = seed; uniforms
 *     (w + 0.5) 2^-32 and Box-Muller.
 *
 * Parity pins (tests/test_oracle_*.py): textbook equal-sphere limits of the
 * resistances, rigid-rotation identities at contact, symmetry and positive
 * semi-definiteness of the pair resistance, the fluctuation-dissipation
 * identity B B^T = R built from the pair noise, Newton's third law, Philox
 * known-answer vectors, the isolated-particle mean-square displacement
 * (Eq. 31), exact discrete equipartition of the Velocity-Verlet/Langevin map,
 * the Einstein limit of the drag stresslet, the Coulomb cap, image and flip
 * invariance, and the Pe definition against Table 1.  The tangential history
 * and contact torque (Eqs. 3-4) are pinned by closed forms built from the
 * rigid-body velocities of the two contact points: a history growing as the
 * tangential slip times t with F = k_t xi and torques a n x F at each contact
 * point, no history for spheres rolling on each other, a capped force of
 * magnitude mu k_n delta against the slip, a history that turns with the
 * contact normal at constant length when nothing slips, and the energy of a
 * frictional collision conserved as dt -> 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_PI 3.14159265358979323846
#define O_TWO_PI 6.28318530717958647692

/* ------------------------------------------------------------------ */
/* parameters                                                          */
/* ------------------------------------------------------------------ */
typedef struct {
  double eta;        /* liquid viscosity */
  double rho;        /* particle density */
  double kn;         /* normal contact stiffness */
  double kt;         /* tangential contact stiffness */
  double mu;         /* static friction coefficient (0: frictionless) */
  double xi_min;     /* regularisation xi_eff (1e-3) */
  double xi_max;     /* lubrication cutoff on xi (0.05) */
  double skin;       /* neighbour-list skin, length units */
  double shear_rate; /* imposed xy shear rate */
  double kT;         /* thermal energy */
  double dt;         /* timestep */
  double torque_sign;/* sign of the chi term of T_ji, Eq. 24 */
  int64_t seed;      /* Philox key */
  int64_t noise;     /* 1: Brownian terms on */
  int64_t lubrication; /* 1: lubrication + pair noise on */
  int64_t onebody;   /* 1: one-body drag + noise on */
  int64_t contact;   /* 1: contact forces on */
  int64_t freeze;    /* 1: positions are not advanced (test mode) */
  int64_t rebuild_every_step; /* 1: rebuild the Verlet list at every step */
  double rep_A;      /* repulsion force scale A of Eq. 34 (0: off) */
  double rep_cut;    /* repulsion acts for h <= rep_cut kappa, kappa = 0.01 (a_i + a_j) */
  double shell;      /* structural Brownian shell Delta / a_i of Eq. 26 */
  int64_t structural;/* 1: structural Brownian stress (Eq. 26) on */
} o_params;

typedef struct {
  int32_t i, j;      /* i < j (tags) */
  int32_t in_contact;
  double hist[3];    /* tangential history xi_t */
} o_entry;

typedef struct {
  int32_t N;
  o_params p;
  double L[3];
  double strain;     /* gamma, in (-flip, flip] */
  double tilt;       /* gamma * Ly */
  int64_t k;         /* evaluation index of the forces held in F, T */
  double *a, *m, *I;
  uint32_t *tag;     /* noise-counter tag of each sphere (default: its index) */
  double *x, *U, *W, *F, *T;
  /* Verlet list */
  o_entry* list;
  int64_t nlist, cap;
  int32_t have_list;
  double disp_bound; /* D: accumulated peculiar displacement bound */
  double t_since_build;
  int64_t nbuilds;
  int32_t forces_valid;
  /* per-evaluation stresses: [0]=contact [1]=lubrication [2]=Brownian pair
   * [3]=repulsion [4]=structural Brownian (Eq. 26) */
  double sigma[5][9];
  double kin[2][9];  /* kinetic tensors (translational, rotational) of full-step velocities */
  double sum_sigma[5][9];
  double sum_kin[2][9];
  int64_t nsamples;
  /* diagnostics of the last evaluation */
  int64_t ncontacts, nlub;
  double max_overlap;
} o_sys;

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
/* out = Nmat v with Nmat = n n^T */
static void normal_op(const double n[3], const double v[3], double out[3]) {
  double s = dot3(n, v);
  out[0] = n[0] * s;
  out[1] = n[1] * s;
  out[2] = n[2] * s;
}
/* out = Tmat v with Tmat = I - n n^T */
static void tangent_op(const double n[3], const double v[3], double out[3]) {
  double s = dot3(n, v);
  out[0] = v[0] - n[0] * s;
  out[1] = v[1] - n[1] * s;
  out[2] = v[2] - n[2] * s;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of   */
/* the 4-word S-box with multipliers 0xD2511F53, 0xCD9E8D57 and a key  */
/* schedule bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85.       */
/* ------------------------------------------------------------------ */
void o_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                     uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double o_uniform(uint32_t w) {
  /* (w + 1/2) 2^-32, strictly inside (0, 1) */
  return ((double)w + 0.5) * (1.0 / 4294967296.0);
}

/* Box-Muller on two words -> two standard normal deviates */
static void o_box_muller(uint32_t wa, uint32_t wb, double* g1, double* g2) {
  double ua = o_uniform(wa), ub = o_uniform(wb);
  double r = sqrt(-2.0 * log(ua));
  double ang = O_TWO_PI * ub;
  *g1 = r * cos(ang);
  *g2 = r * sin(ang);
}

/* Six Gaussians for counter (k, t1, t2): pair (t1 < t2) -> theta, chi;
 * one-body (t1 == t2) -> psi, phi.  Block 0 gives g0..g3, block 1 g4, g5. */
void o_gaussians6(int64_t seed, int64_t k, uint32_t t1, uint32_t t2,
                  double g[6]) {
  uint32_t key[2] = {(uint32_t)((uint64_t)seed & 0xffffffffu),
                     (uint32_t)((uint64_t)seed >> 32)};
  uint32_t khi = (uint32_t)((uint64_t)k >> 32);
  uint32_t ctr0[4] = {(uint32_t)((uint64_t)k & 0xffffffffu), t1, t2, 2u * khi + 0u};
  uint32_t ctr1[4] = {(uint32_t)((uint64_t)k & 0xffffffffu), t1, t2, 2u * khi + 1u};
  uint32_t w0[4], w1[4];
  o_philox4x32_10(ctr0, key, w0);
  o_philox4x32_10(ctr1, key, w1);
  o_box_muller(w0[0], w0[1], &g[0], &g[1]);
  o_box_muller(w0[2], w0[3], &g[2], &g[3]);
  o_box_muller(w1[0], w1[1], &g[4], &g[5]);
}

/* ------------------------------------------------------------------ */
/* scalar resistances, Eqs. 9-12 and 15-18 (Sec. II.B)                 */
/* out = {XA11, YA11, YB11, YB21, YC11, YC12, YC21, YC22}              */
/* xi_e is the already regularised dimensionless gap.                  */
/* ------------------------------------------------------------------ */
void o_resistances(double eta, double ai, double aj, double xi_e,
                   double out[8]) {
  double beta = aj / ai;
  double ibeta = 1.0 / beta;
  double opb = 1.0 + beta;
  double opib = 1.0 + ibeta;
  double lg = log(1.0 / xi_e);
  /* Eq. 9 */
  double XA11 = 6.0 * O_PI * eta * ai *
                (2.0 * beta * beta / (opb * opb * opb) * (1.0 / xi_e) +
                 beta * (1.0 + 7.0 * beta + beta * beta) /
                     (5.0 * (opb * opb * opb)) * lg);
  /* Eq. 10 */
  double YA11 = 6.0 * O_PI * eta * ai *
                (4.0 * beta * (2.0 + beta + 2.0 * beta * beta) /
                 (15.0 * (opb * opb * opb)) * lg);
  /* Eq. 11 */
  double YB11 = -4.0 * O_PI * eta * ai * ai *
                (beta * (4.0 + beta) / (5.0 * (opb * opb)) * lg);
  /* Eq. 12 */
  double YB21 = -4.0 * O_PI * eta * aj * aj *
                (ibeta * (4.0 + ibeta) / (5.0 * (opib * opib)) * lg);
  /* Eq. 15 */
  double YC11 = 8.0 * O_PI * eta * ai * ai * ai *
                (2.0 * beta / (5.0 * opb) * lg);
  /* Eq. 16 */
  double YC12 = 8.0 * O_PI * eta * ai * ai * ai *
                (beta * beta / (10.0 * opb) * lg);
  /* Eq. 17 */
  double YC22 = 8.0 * O_PI * eta * aj * aj * aj *
                (2.0 * ibeta / (5.0 * opib) * lg);
  /* Eq. 18 */
  double YC21 = 8.0 * O_PI * eta * aj * aj * aj *
                (ibeta * ibeta / (10.0 * opib) * lg);
  out[0] = XA11; out[1] = YA11; out[2] = YB11; out[3] = YB21;
  out[4] = YC11; out[5] = YC12; out[6] = YC21; out[7] = YC22;
}

/* Lubrication force on i and torques on i, j, Eqs. 8, 13, 14.
 * n points from i to j; dU = U_j - U_i (with the image velocity shift). */
void o_lubrication(const double R[8], const double n[3], const double dU[3],
                   const double Wi[3], const double Wj[3], double Fi[3],
                   double Ti[3], double Tj[3]) {
  double XA11 = R[0], YA11 = R[1], YB11 = R[2], YB21 = R[3];
  double YC11 = R[4], YC12 = R[5], YC21 = R[6], YC22 = R[7];
  double Nd[3], Td[3], wi_n[3], wj_n[3], dU_n[3];
  normal_op(n, dU, Nd);
  tangent_op(n, dU, Td);
  cross3(Wi, n, wi_n);
  cross3(Wj, n, wj_n);
  cross3(dU, n, dU_n);
  double ci[3], cj[3];
  for (int c = 0; c < 3; ++c) {
    ci[c] = YC11 * Wi[c] + YC12 * Wj[c];
    cj[c] = YC21 * Wi[c] + YC22 * Wj[c];
  }
  double Tci[3], Tcj[3];
  tangent_op(n, ci, Tci);
  tangent_op(n, cj, Tcj);
  for (int c = 0; c < 3; ++c) {
    Fi[c] = XA11 * Nd[c] + YA11 * Td[c] + YB11 * wi_n[c] + YB21 * wj_n[c];
    Ti[c] = YB11 * dU_n[c] - Tci[c];
    Tj[c] = YB21 * dU_n[c] - Tcj[c];
  }
}

/* Pairwise Brownian force on i and torques on i, j, Eqs. 22-24, for given
 * standard normal vectors theta, chi and amplitude c = sqrt(2 kT / dt). */
void o_pair_brownian(const double R[8], const double n[3], const double th[3],
                     const double chi[3], double c, double torque_sign,
                     double Fi[3], double Ti[3], double Tj[3]) {
  double XA11 = R[0], YA11 = R[1], YB11 = R[2], YB21 = R[3];
  double YC11 = R[4], YC22 = R[7];
  double sXA = sqrt(XA11), sYA = sqrt(YA11);
  double Nth[3], Tth[3], th_n[3], Tchi[3];
  normal_op(n, th, Nth);
  tangent_op(n, th, Tth);
  cross3(th, n, th_n);
  tangent_op(n, chi, Tchi);
  double bi = YB11 / sYA;
  double bj = YB21 / sYA;
  double si = sqrt(YC11 - YB11 * YB11 / YA11);
  double sj = sqrt(YC22 - YB21 * YB21 / YA11);
  for (int q = 0; q < 3; ++q) {
    Fi[q] = c * (sXA * Nth[q] + sYA * Tth[q]);
    Ti[q] = c * (bi * th_n[q] + si * Tchi[q]);
    Tj[q] = c * (bj * th_n[q] + torque_sign * sj * Tchi[q]);
  }
}

/* ------------------------------------------------------------------ */
/* box: sliding-brick form of the tilted periodic box (Sec. II.E)      */
/* ------------------------------------------------------------------ */
/* Minimum-image separation r = x_j - x_i and the y image count sy. */
static void min_image(const o_sys* s, const double* xi, const double* xj,
                      double r[3], double* sy_out) {
  double dx = xj[0] - xi[0];
  double dy = xj[1] - xi[1];
  double dz = xj[2] - xi[2];
  double sy = rint(dy / s->L[1]);
  dy = dy - sy * s->L[1];
  dx = dx - sy * s->tilt;
  double sx = rint(dx / s->L[0]);
  dx = dx - sx * s->L[0];
  double sz = rint(dz / s->L[2]);
  dz = dz - sz * s->L[2];
  r[0] = dx; r[1] = dy; r[2] = dz;
  *sy_out = sy;
}

/* Wrap particle i into [0,L): a y crossing shifts x by the tilt and U_x by
 * rate * Ly so that U - U_inf stays continuous (Lees-Edwards). */
static void wrap_particle(o_sys* s, int i) {
  double* x = s->x + 3 * i;
  double* U = s->U + 3 * i;
  double Ly = s->L[1];
  double dUx = s->p.shear_rate * Ly;
  if (!isfinite(x[0] + x[1] + x[2])) return;
  /* a sphere moves far less than a box edge per step; the loops stop after
   * 64 images so that a run that has blown up ends instead of spinning */
  int g = 0;
  while (x[1] >= Ly && g < 64) { x[1] = x[1] - Ly; x[0] = x[0] - s->tilt; U[0] = U[0] - dUx; ++g; }
  while (x[1] < 0.0 && g < 64) { x[1] = x[1] + Ly; x[0] = x[0] + s->tilt; U[0] = U[0] + dUx; ++g; }
  while (x[0] >= s->L[0] && g < 64) { x[0] = x[0] - s->L[0]; ++g; }
  while (x[0] < 0.0 && g < 64) { x[0] = x[0] + s->L[0]; ++g; }
  while (x[2] >= s->L[2] && g < 64) { x[2] = x[2] - s->L[2]; ++g; }
  while (x[2] < 0.0 && g < 64) { x[2] = x[2] + s->L[2]; ++g; }
}

/* ------------------------------------------------------------------ */
/* Verlet list: brute force O(N^2), pairs with d^2 < r_list^2,          */
/* r_list = r_int + skin; history carried by (i,j).  r_int is the       */
/* largest centre distance at which a pair interacts: the lubrication   */
/* cutoff (a_i + a_j)(1 + xi_max/2), with repulsion on also             */
/* (a_i + a_j)(1 + 0.01 rep_cut), with the structural stress on also    */
/* a_i + a_j + shell max(a_i, a_j).                                      */
/* ------------------------------------------------------------------ */
static double interaction_cut(const o_sys* s, double ai, double aj) {
  double r = (ai + aj) * (1.0 + 0.5 * s->p.xi_max);
  if (s->p.rep_A > 0.0) {
    double rr = (ai + aj) * (1.0 + 0.01 * s->p.rep_cut);
    if (rr > r) r = rr;
  }
  if (s->p.structural) {
    double rs = (ai + aj) + s->p.shell * (ai > aj ? ai : aj);
    if (rs > r) r = rs;
  }
  return r;
}

static double list_cut(const o_sys* s, double ai, double aj) {
  return interaction_cut(s, ai, aj) + s->p.skin;
}

static int entry_cmp(const o_entry* e, int32_t i, int32_t j) {
  if (e->i != i) return e->i < i ? -1 : 1;
  if (e->j != j) return e->j < j ? -1 : 1;
  return 0;
}

static const o_entry* find_entry(const o_entry* list, int64_t n, int32_t i,
                                 int32_t j) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    int c = entry_cmp(&list[mid], i, j);
    if (c == 0) return &list[mid];
    if (c < 0) lo = mid + 1; else hi = mid - 1;
  }
  return NULL;
}

static int build_list(o_sys* s) {
  int64_t n = 0, cap = s->cap > 0 ? s->cap : 1024;
  o_entry* nl = (o_entry*)malloc((size_t)cap * sizeof(o_entry));
  if (!nl) return -1;
  for (int32_t i = 0; i < s->N; ++i) {
    for (int32_t j = i + 1; j < s->N; ++j) {
      double r[3], sy;
      min_image(s, s->x + 3 * i, s->x + 3 * j, r, &sy);
      double d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      double rc = list_cut(s, s->a[i], s->a[j]);
      if (!(d2 < rc * rc)) continue;
      if (n == cap) {
        cap *= 2;
        o_entry* t = (o_entry*)realloc(nl, (size_t)cap * sizeof(o_entry));
        if (!t) { free(nl); return -1; }
        nl = t;
      }
      o_entry e;
      e.i = i; e.j = j; e.in_contact = 0;
      e.hist[0] = e.hist[1] = e.hist[2] = 0.0;
      const o_entry* old = s->have_list ? find_entry(s->list, s->nlist, i, j) : NULL;
      if (old && old->in_contact) {
        e.in_contact = 1;
        e.hist[0] = old->hist[0]; e.hist[1] = old->hist[1]; e.hist[2] = old->hist[2];
      }
      nl[n++] = e;
    }
  }
  free(s->list);
  s->list = nl;
  s->nlist = n;
  s->cap = cap;
  s->have_list = 1;
  s->disp_bound = 0.0;
  s->t_since_build = 0.0;
  s->nbuilds += 1;
  return 0;
}

/* ------------------------------------------------------------------ */
/* force evaluation at the current state (Eqs. 1-2 right-hand sides)    */
/* `advance` = 1 when time has advanced since the previous evaluation   */
/* (the tangential history is then incremented).                        */
/* ------------------------------------------------------------------ */
static void evaluate(o_sys* s, int advance) {
  const o_params* p = &s->p;
  int32_t N = s->N;
  double rate = p->shear_rate;
  double yc = 0.5 * s->L[1];
  double c = sqrt(2.0 * p->kT / p->dt);
  double Winf[3] = {0.0, 0.0, -0.5 * rate};
  double V = s->L[0] * s->L[1] * s->L[2];
  memset(s->F, 0, sizeof(double) * 3 * (size_t)N);
  memset(s->T, 0, sizeof(double) * 3 * (size_t)N);
  memset(s->sigma, 0, sizeof(s->sigma));
  s->ncontacts = 0; s->nlub = 0; s->max_overlap = 0.0;

  /* one-body drag (Eqs. 5-6) and one-body Brownian terms (Eqs. 20-21) */
  if (p->onebody) {
    for (int32_t i = 0; i < N; ++i) {
      const double* x = s->x + 3 * i;
      const double* U = s->U + 3 * i;
      const double* W = s->W + 3 * i;
      double a = s->a[i];
      double gt = 6.0 * O_PI * p->eta * a;
      double gr = 8.0 * O_PI * p->eta * a * a * a;
      double Uinf[3] = {rate * (x[1] - yc), 0.0, 0.0};
      double g[6] = {0, 0, 0, 0, 0, 0};
      if (p->noise) o_gaussians6(p->seed, s->k, s->tag[i], s->tag[i], g);
      double ct = c * sqrt(gt), cr = c * sqrt(gr);
      for (int q = 0; q < 3; ++q) {
        s->F[3 * i + q] += gt * (Uinf[q] - U[q]) + (p->noise ? ct * g[q] : 0.0);
        s->T[3 * i + q] += gr * (Winf[q] - W[q]) + (p->noise ? cr * g[3 + q] : 0.0);
      }
    }
  }

  /* pair terms, list entries visited in lexicographic (i, j) order */
  for (int64_t e = 0; e < s->nlist; ++e) {
    o_entry* en = &s->list[e];
    int32_t i = en->i, j = en->j;
    double r[3], sy;
    min_image(s, s->x + 3 * i, s->x + 3 * j, r, &sy);
    double d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double d = sqrt(d2);
    double S = s->a[i] + s->a[j];
    double h = d - S;               /* surface gap */
    double xi = 2.0 * h / S;        /* dimensionless gap, Sec. II.B */
    double kappa = 0.01 * S;        /* repulsion length, Eq. 34 */
    int lub = xi <= p->xi_max;
    int rep = p->rep_A > 0.0 && h <= p->rep_cut * kappa;
    int shell_i = p->structural && h <= p->shell * s->a[i];
    int shell_j = p->structural && h <= p->shell * s->a[j];
    if (!lub) {                     /* outside lubrication range: no contact */
      en->in_contact = 0;
      en->hist[0] = en->hist[1] = en->hist[2] = 0.0;
    }
    if (!lub && !rep && !shell_i && !shell_j) continue;
    double n[3] = {r[0] / d, r[1] / d, r[2] / d};
    if (shell_i || shell_j) {
      /* Eq. 26: each sphere i counts the neighbours j in its shell
       * h <= Delta = shell a_i with weight a_i / Delta = 1 / shell; the pair
       * enters once from each side whose shell holds it */
      double w = (shell_i ? 1.0 / p->shell : 0.0) + (shell_j ? 1.0 / p->shell : 0.0);
      for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be)
          s->sigma[4][3 * al + be] += -p->kT * w * n[al] * n[be];
    }
    double FR[3] = {0, 0, 0};
    if (rep) {
      /* Eq. 34 read as the force on j, (A/kappa) exp((S - d)/kappa) n_ij:
       * on i it is the opposite */
      double f = p->rep_A / kappa * exp(-h / kappa);
      for (int q = 0; q < 3; ++q) FR[q] = -f * n[q];
      for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) s->sigma[3][3 * al + be] += FR[al] * r[be];
    }
    if (!lub) {
      for (int q = 0; q < 3; ++q) {
        s->F[3 * i + q] += FR[q];
        s->F[3 * j + q] -= FR[q];
      }
      continue;
    }
    const double* Ui = s->U + 3 * i;
    const double* Uj = s->U + 3 * j;
    const double* Wi = s->W + 3 * i;
    const double* Wj = s->W + 3 * j;
    /* velocity of the image of j minus velocity of i */
    double dU[3] = {Uj[0] - sy * rate * s->L[1] - Ui[0], Uj[1] - Ui[1], Uj[2] - Ui[2]};
    double FL[3] = {0, 0, 0}, TLi[3] = {0, 0, 0}, TLj[3] = {0, 0, 0};
    double FB[3] = {0, 0, 0}, TBi[3] = {0, 0, 0}, TBj[3] = {0, 0, 0};
    double FC[3] = {0, 0, 0}, TCi[3] = {0, 0, 0}, TCj[3] = {0, 0, 0};
    if (p->lubrication) {
      double xi_e = xi < p->xi_min ? p->xi_min : xi;
      double R[8];
      o_resistances(p->eta, s->a[i], s->a[j], xi_e, R);
      o_lubrication(R, n, dU, Wi, Wj, FL, TLi, TLj);
      if (p->noise) {
        double g[6];
        o_gaussians6(p->seed, s->k, s->tag[i], s->tag[j], g);
        double th[3] = {g[0], g[1], g[2]};
        double chi[3] = {g[3], g[4], g[5]};
        o_pair_brownian(R, n, th, chi, c, p->torque_sign, FB, TBi, TBj);
      }
      s->nlub += 1;
    }
    if (h < 0.0 && p->contact) {
      double delta = -h;            /* overlap, Sec. II.A */
      if (delta > s->max_overlap) s->max_overlap = delta;
      s->ncontacts += 1;
      double Ft[3] = {0.0, 0.0, 0.0};
      if (p->mu > 0.0) {
        double* xt = en->hist;
        if (!en->in_contact) { xt[0] = xt[1] = xt[2] = 0.0; }
        if (advance) {
          /* tangential relative velocity of the contact points */
          double ww[3] = {s->a[i] * Wi[0] + s->a[j] * Wj[0],
                          s->a[i] * Wi[1] + s->a[j] * Wj[1],
                          s->a[i] * Wi[2] + s->a[j] * Wj[2]};
          double wxn[3];
          cross3(ww, n, wxn);
          double v[3] = {dU[0] - wxn[0], dU[1] - wxn[1], dU[2] - wxn[2]};
          double vt[3];
          tangent_op(n, v, vt);
          /* rotate the stored displacement into the current tangent plane */
          double len0 = sqrt(dot3(xt, xt));
          double pr[3];
          tangent_op(n, xt, pr);
          double len1 = sqrt(dot3(pr, pr));
          if (len1 > 0.0) {
            double sc = len0 / len1;
            xt[0] = pr[0] * sc; xt[1] = pr[1] * sc; xt[2] = pr[2] * sc;
          } else {
            xt[0] = xt[1] = xt[2] = 0.0;
          }
          xt[0] = xt[0] + vt[0] * p->dt;
          xt[1] = xt[1] + vt[1] * p->dt;
          xt[2] = xt[2] + vt[2] * p->dt;
          /* Coulomb cap |k_t xi| <= mu k_n delta */
          double ft = p->kt * sqrt(dot3(xt, xt));
          double fmax = p->mu * p->kn * delta;
          if (ft > fmax) {
            double sc = fmax / ft;
            xt[0] = xt[0] * sc; xt[1] = xt[1] * sc; xt[2] = xt[2] * sc;
          }
        }
        en->in_contact = 1;
        Ft[0] = p->kt * xt[0]; Ft[1] = p->kt * xt[1]; Ft[2] = p->kt * xt[2];
      }
      /* contact force on i, Eq. 3 read as the force on j */
      for (int q = 0; q < 3; ++q) FC[q] = -p->kn * delta * n[q] + Ft[q];
      /* contact torques, Eq. 4, on i and on j */
      double nxF[3];
      cross3(n, Ft, nxF);
      for (int q = 0; q < 3; ++q) {
        TCi[q] = s->a[i] * nxF[q];
        TCj[q] = s->a[j] * nxF[q];
      }
    } else {
      en->in_contact = 0;
      en->hist[0] = en->hist[1] = en->hist[2] = 0.0;
    }
    for (int q = 0; q < 3; ++q) {
      double Fi = FC[q] + FL[q] + FB[q] + FR[q];
      s->F[3 * i + q] += Fi;
      s->F[3 * j + q] -= Fi;
      s->T[3 * i + q] += TCi[q] + TLi[q] + TBi[q];
      s->T[3 * j + q] += TCj[q] + TLj[q] + TBj[q];
    }
    for (int al = 0; al < 3; ++al)
      for (int be = 0; be < 3; ++be) {
        s->sigma[0][3 * al + be] += FC[al] * r[be];
        s->sigma[1][3 * al + be] += FL[al] * r[be];
        s->sigma[2][3 * al + be] += FB[al] * r[be];
      }
  }
  for (int comp = 0; comp < 5; ++comp)
    for (int q = 0; q < 9; ++q) s->sigma[comp][q] = s->sigma[comp][q] / V;
  s->forces_valid = 1;
}

static void kinetic(o_sys* s) {
  double rate = s->p.shear_rate, yc = 0.5 * s->L[1];
  double V = s->L[0] * s->L[1] * s->L[2];
  memset(s->kin, 0, sizeof(s->kin));
  for (int32_t i = 0; i < s->N; ++i) {
    const double* x = s->x + 3 * i;
    double u[3] = {s->U[3 * i] - rate * (x[1] - yc), s->U[3 * i + 1], s->U[3 * i + 2]};
    double w[3] = {s->W[3 * i], s->W[3 * i + 1], s->W[3 * i + 2] + 0.5 * rate};
    for (int al = 0; al < 3; ++al)
      for (int be = 0; be < 3; ++be) {
        s->kin[0][3 * al + be] += s->m[i] * u[al] * u[be];
        s->kin[1][3 * al + be] += s->I[i] * w[al] * w[be];
      }
  }
  for (int q = 0; q < 9; ++q) { s->kin[0][q] /= V; s->kin[1][q] /= V; }
}

/* ------------------------------------------------------------------ */
/* public entry points (ctypes)                                         */
/* ------------------------------------------------------------------ */
o_sys* o_create(int32_t N, const double* radii, const double box[3],
                const o_params* p) {
  if (N <= 0 || !radii || !box || !p) return NULL;
  o_sys* s = (o_sys*)calloc(1, sizeof(o_sys));
  if (!s) return NULL;
  s->N = N;
  s->p = *p;
  s->L[0] = box[0]; s->L[1] = box[1]; s->L[2] = box[2];
  size_t n3 = 3 * (size_t)N;
  s->a = (double*)malloc(sizeof(double) * (size_t)N);
  s->m = (double*)malloc(sizeof(double) * (size_t)N);
  s->I = (double*)malloc(sizeof(double) * (size_t)N);
  s->x = (double*)calloc(n3, sizeof(double));
  s->U = (double*)calloc(n3, sizeof(double));
  s->W = (double*)calloc(n3, sizeof(double));
  s->F = (double*)calloc(n3, sizeof(double));
  s->T = (double*)calloc(n3, sizeof(double));
  s->tag = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  for (int32_t i = 0; i < N; ++i) s->tag[i] = (uint32_t)i;
  /* m = (4/3) pi rho a^3 (Sec. III.B), I = (2/5) m a^2 (Eq. 2) */
  double cm = 4.0 / 3.0 * O_PI * p->rho;
  for (int32_t i = 0; i < N; ++i) {
    double a = radii[i];
    s->a[i] = a;
    s->m[i] = cm * a * a * a;
    s->I[i] = 0.4 * s->m[i] * a * a;
  }
  return s;
}

void o_destroy(o_sys* s) {
  if (!s) return;
  free(s->a); free(s->m); free(s->I); free(s->x); free(s->U); free(s->W);
  free(s->F); free(s->T); free(s->list); free(s->tag);
  free(s);
}

void o_set_state(o_sys* s, const double* x, const double* U, const double* W) {
  size_t n3 = 3 * (size_t)s->N;
  memcpy(s->x, x, sizeof(double) * n3);
  if (U) memcpy(s->U, U, sizeof(double) * n3); else memset(s->U, 0, sizeof(double) * n3);
  if (W) memcpy(s->W, W, sizeof(double) * n3); else memset(s->W, 0, sizeof(double) * n3);
  for (int32_t i = 0; i < s->N; ++i) wrap_particle(s, i);
  s->have_list = 0;
  s->nlist = 0;
  s->forces_valid = 0;
}

/* Replaces velocities and angular velocities (N x 3 each) and keeps the
 * positions, the Verlet list and the tangential history. */
void o_set_velocities(o_sys* s, const double* U, const double* W) {
  size_t n3 = 3 * (size_t)s->N;
  memcpy(s->U, U, sizeof(double) * n3);
  memcpy(s->W, W, sizeof(double) * n3);
  s->forces_valid = 0;
}

void o_set_strain(o_sys* s, double strain) {
  s->strain = strain;
  s->tilt = strain * s->L[1];
  s->forces_valid = 0;
}

void o_set_k(o_sys* s, int64_t k) { s->k = k; s->forces_valid = 0; }

/* Noise-counter tags (Sec. II.C counters use the spheres' tags): lets a
 * small system stand for spheres of a larger one.  Pairs are still
 * oriented by index, so tags must increase with the index. */
int o_set_tags(o_sys* s, const uint32_t* tags) {
  for (int32_t i = 1; i < s->N; ++i)
    if (!(tags[i] > tags[i - 1])) return -1;
  memcpy(s->tag, tags, sizeof(uint32_t) * (size_t)s->N);
  s->forces_valid = 0;
  return 0;
}

/* Force evaluation at the current state without advancing time. */
int o_evaluate(o_sys* s) {
  if (!s->have_list) { if (build_list(s)) return -1; }
  evaluate(s, 0);
  return 0;
}

int o_build(o_sys* s) { return build_list(s); }

static double max_list_cut(const o_sys* s) {
  double amax = 0.0;
  for (int32_t i = 0; i < s->N; ++i) if (s->a[i] > amax) amax = s->a[i];
  return interaction_cut(s, amax, amax);
}

/* Advance n Velocity-Verlet steps. */
int o_step(o_sys* s, int64_t nsteps) {
  const o_params* p = &s->p;
  int32_t N = s->N;
  double hdt = 0.5 * p->dt;
  double rate = p->shear_rate;
  double rate_dt = rate * p->dt;
  double flip_at = 0.5 * s->L[0] / s->L[1];
  double flip_by = s->L[0] / s->L[1];
  double rcmax = max_list_cut(s);
  if (!s->forces_valid) {
    if (!s->have_list && build_list(s)) return -1;
    evaluate(s, 0);
  }
  for (int64_t n = 0; n < nsteps; ++n) {
    /* first half kick with F(t) */
    for (int32_t i = 0; i < N; ++i)
      for (int q = 0; q < 3; ++q) {
        s->U[3 * i + q] = s->U[3 * i + q] + hdt * s->F[3 * i + q] / s->m[i];
        s->W[3 * i + q] = s->W[3 * i + q] + hdt * s->T[3 * i + q] / s->I[i];
      }
    /* drift, box deformation and flip, wrap */
    if (!p->freeze)
      for (int32_t i = 0; i < N; ++i)
        for (int q = 0; q < 3; ++q)
          s->x[3 * i + q] = s->x[3 * i + q] + p->dt * s->U[3 * i + q];
    s->strain = s->strain + rate_dt;
    if (s->strain > flip_at) s->strain = s->strain - flip_by;
    s->tilt = s->strain * s->L[1];
    double vmax = 0.0;
    if (!p->freeze) {
      double yc = 0.5 * s->L[1];
      for (int32_t i = 0; i < N; ++i) {
        wrap_particle(s, i);
        double ux = s->U[3 * i] - rate * (s->x[3 * i + 1] - yc);
        double uy = s->U[3 * i + 1], uz = s->U[3 * i + 2];
        double v = sqrt(ux * ux + uy * uy + uz * uz);
        if (v > vmax) vmax = v;
      }
    }
    s->k += 1;
    /* list validity: 2D + rate * t (r_c + 2D) < skin */
    s->disp_bound += p->dt * vmax;
    s->t_since_build += p->dt;
    double drift = 2.0 * s->disp_bound +
                   fabs(rate) * s->t_since_build * (rcmax + 2.0 * s->disp_bound);
    if (p->rebuild_every_step || drift >= p->skin) {
      if (build_list(s)) return -1;
    }
    evaluate(s, 1);
    /* second half kick with F(t + dt) */
    for (int32_t i = 0; i < N; ++i)
      for (int q = 0; q < 3; ++q) {
        s->U[3 * i + q] = s->U[3 * i + q] + hdt * s->F[3 * i + q] / s->m[i];
        s->W[3 * i + q] = s->W[3 * i + q] + hdt * s->T[3 * i + q] / s->I[i];
      }
    kinetic(s);
    for (int comp = 0; comp < 5; ++comp)
      for (int q = 0; q < 9; ++q) s->sum_sigma[comp][q] += s->sigma[comp][q];
    for (int comp = 0; comp < 2; ++comp)
      for (int q = 0; q < 9; ++q) s->sum_kin[comp][q] += s->kin[comp][q];
    s->nsamples += 1;
  }
  return 0;
}

void o_get_state(const o_sys* s, double* x, double* U, double* W) {
  size_t n3 = 3 * (size_t)s->N;
  if (x) memcpy(x, s->x, sizeof(double) * n3);
  if (U) memcpy(U, s->U, sizeof(double) * n3);
  if (W) memcpy(W, s->W, sizeof(double) * n3);
}

void o_get_forces(const o_sys* s, double* F, double* T) {
  size_t n3 = 3 * (size_t)s->N;
  if (F) memcpy(F, s->F, sizeof(double) * n3);
  if (T) memcpy(T, s->T, sizeof(double) * n3);
}

/* out: [5][9] pair stresses of the last evaluation (contact, lubrication,
 * Brownian pair, repulsion, structural Brownian), then [2][9] kinetic */
void o_get_stress(const o_sys* s, double* out) {
  memcpy(out, s->sigma, sizeof(s->sigma));
  memcpy(out + 45, s->kin, sizeof(s->kin));
}

/* out: time sums since the last reset: [5][9] pair stresses, [2][9] kinetic;
 * returns the number of samples and resets. */
int64_t o_take_stress_sums(o_sys* s, double* out) {
  memcpy(out, s->sum_sigma, sizeof(s->sum_sigma));
  memcpy(out + 45, s->sum_kin, sizeof(s->sum_kin));
  int64_t n = s->nsamples;
  memset(s->sum_sigma, 0, sizeof(s->sum_sigma));
  memset(s->sum_kin, 0, sizeof(s->sum_kin));
  s->nsamples = 0;
  return n;
}

/* info: strain, tilt, k, nlist, nbuilds, ncontacts, nlub, max_overlap */
void o_get_info(const o_sys* s, double* info) {
  info[0] = s->strain; info[1] = s->tilt; info[2] = (double)s->k;
  info[3] = (double)s->nlist; info[4] = (double)s->nbuilds;
  info[5] = (double)s->ncontacts; info[6] = (double)s->nlub;
  info[7] = s->max_overlap;
}

/* Current Verlet list: pairs (i, j) and their tangential history. */
int64_t o_list_size(const o_sys* s) { return s->nlist; }
void o_get_list(const o_sys* s, int32_t* ij, double* hist, int32_t* contact) {
  for (int64_t e = 0; e < s->nlist; ++e) {
    if (ij) { ij[2 * e] = s->list[e].i; ij[2 * e + 1] = s->list[e].j; }
    if (hist) for (int q = 0; q < 3; ++q) hist[3 * e + q] = s->list[e].hist[q];
    if (contact) contact[e] = s->list[e].in_contact;
  }
}

/* Brute-force pair set at the current state: all i < j with d^2 < r_list^2.
 * Writes at most cap pairs; returns the count. */
int64_t o_brute_pairs(const o_sys* s, int32_t* ij, int64_t cap) {
  int64_t n = 0;
  for (int32_t i = 0; i < s->N; ++i)
    for (int32_t j = i + 1; j < s->N; ++j) {
      double r[3], sy;
      min_image(s, s->x + 3 * i, s->x + 3 * j, r, &sy);
      double d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      double rc = list_cut(s, s->a[i], s->a[j]);
      if (d2 < rc * rc) {
        if (n < cap) { ij[2 * n] = i; ij[2 * n + 1] = j; }
        n++;
      }
    }
  return n;
}

/* Drag stresslet (20/3) pi eta sum_i a_i^3 E / V, Sec. II.B, xy component
 * of E = rate/2 (x y + y x). */
double o_drag_stress_xy(int32_t N, const double* radii, const double box[3],
                        double eta, double rate) {
  double s3 = 0.0;
  for (int32_t i = 0; i < N; ++i) s3 += radii[i] * radii[i] * radii[i];
  double V = box[0] * box[1] * box[2];
  return 20.0 / 3.0 * O_PI * eta * s3 * (0.5 * rate) / V;
}

/* Timescales of Sec. II.F, Eqs. 27-30, and the Peclet number. */
void o_timescales(double a, double rho, double kn, double eta, double kT,
                  double rate, double out[5]) {
  out[0] = sqrt(rho * a * a * a / kn);          /* tau_C */
  out[1] = rho * a * a / eta;                   /* tau_I */
  out[2] = eta * a * a * a / kT;                /* tau_B */
  out[3] = 1.0 / rate;                          /* tau_S */
  out[4] = 6.0 * O_PI * eta * a * a * a * rate / kT; /* Pe = 6 pi tau_B / tau_S */
}

/* ------------------------------------------------------------------ */
/* Green-Kubo Brownian viscosity, Eq. 33 (Sec. III.D)                   */
/* ------------------------------------------------------------------ */
/* C(tau) = <x(t + tau) x(t)> for tau = 0 .. max_lag - 1 sample steps,   */
/* the average over the n - tau available origins.                      */
void o_autocorr(const double* x, int64_t n, int64_t max_lag, double* C) {
  for (int64_t tau = 0; tau < max_lag; ++tau) {
    double acc = 0.0;
    int64_t cnt = n - tau;
    for (int64_t t = 0; t < cnt; ++t) acc = acc + x[t + tau] * x[t];
    C[tau] = cnt > 0 ? acc / (double)cnt : 0.0;
  }
}

/* eta(t_m) = V / kT * integral_0^{t_m} C dt' with the trapezoid rule on
 * the sample spacing dt: eta[0] = 0, eta[m] = eta[m-1] + dt (C[m-1] + C[m]) / 2. */
void o_green_kubo(const double* x, int64_t n, int64_t max_lag, double dt, double V,
                  double kT, double* C, double* eta) {
  o_autocorr(x, n, max_lag, C);
  double pref = V / kT;
  if (max_lag > 0) eta[0] = 0.0;
  for (int64_t m = 1; m < max_lag; ++m)
    eta[m] = eta[m - 1] + pref * dt * 0.5 * (C[m - 1] + C[m]);
}

/* Fit eta(t) ~ eta_phi (1 - exp(-t / tau_phi)) (Sec. III.D): for each tau
 * on the grid tau_g = dt * (10 M)^(g / (G - 1)), g = 0 .. G-1, the least-
 * squares eta_phi(tau) = sum eta f / sum f^2 with f = 1 - exp(-t_m / tau);
 * the grid point of smallest residual wins.  out = {eta_phi, tau_phi}. */
void o_gk_fit(const double* eta, int64_t M, double dt, int64_t G, double* out) {
  double best = -1.0, best_eta = 0.0, best_tau = 0.0;
  for (int64_t g = 0; g < G; ++g) {
    double tau = dt * pow(10.0 * (double)M, (double)g / (double)(G - 1));
    double sff = 0.0, sef = 0.0;
    for (int64_t m = 0; m < M; ++m) {
      double f = 1.0 - exp(-(double)m * dt / tau);
      sff = sff + f * f;
      sef = sef + eta[m] * f;
    }
    double e = sff > 0.0 ? sef / sff : 0.0;
    double res = 0.0;
    for (int64_t m = 0; m < M; ++m) {
      double f = 1.0 - exp(-(double)m * dt / tau);
      double d = eta[m] - e * f;
      res = res + d * d;
    }
    if (best < 0.0 || res < best) { best = res; best_eta = e; best_tau = tau; }
  }
  out[0] = best_eta;
  out[1] = best_tau;
}
