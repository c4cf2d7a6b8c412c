/*
 * oracle.c -- plain FP64 CPU restatement of the dsDNA model of
 * arXiv:1608.03722 (Fosado et al.).
 *
 * TEST INFRASTRUCTURE ONLY: the independent checker for the CUDA library.  It
 * shares no code with that library and only the tests, the smoke check and
 * bench.py's cpu_baseline leg may load it.  See oracle.h for conventions.
 *
 * Parity status per function (what pins it; see tests/test_oracle_*.py):
 *   or_philox4x32_10  published known-answer vectors of Philox4x32-10
 *   or_ideal_helix    geometry fixed by Sec. 2 / Fig. 1 (0.34 nm rise, 0.46 nm
 *                     bead spacing, 36 deg per bp, 2 nm thickness, 90 deg
 *                     planarity)
 *   or_forces         central finite differences of its own energy, closed
 *                     forms of each potential (App. A Eqs. 9-15), zero net
 *                     force and torque, rotation/translation invariance,
 *                     brute-force pair set
 *   or_forces_cells   equal to or_forces (brute force) on small systems
 *   or_run            NVE energy conservation with dt^2 scaling, Langevin
 *                     equipartition (App. A Eq. 8)
 *   or_observables    ideal-helix twist (36 deg / bp), rise, denatured
 *                     fraction limits; Lk of a Hopf link and of torus links
 *                     against a crossing count
 *   rings (ring[m])   planar ring wound lk times: Lk = Tw = lk, Wr = 0,
 *                     bending energy 2N K6 (1 - cos(2 pi/N)); energy and twist
 *                     equal to sums over the N linear cuts (each step term
 *                     missing once, each bend and twist increment twice);
 *                     invariance under cyclic relabelling; finite differences
 *                     across the junction; Lk conserved by dynamics
 *   Sec. 5 rules      closed-form H-bond depths per pair type, bubble energy
 *                     removal, finite differences with the rule on
 * Parity unpinned: absolute dynamical time scales (masses, friction) which
 * the paper does not measure.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

/* ---------------------------------------------------------------- vectors */
static inline void v_sub(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline double v_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void v_cross(const double* a, const double* b, double* o) {
  double x = a[1] * b[2] - a[2] * b[1], y = a[2] * b[0] - a[0] * b[2], z = a[0] * b[1] - a[1] * b[0];
  o[0] = x; o[1] = y; o[2] = z;
}
static inline double v_norm(const double* a) { return sqrt(v_dot(a, a)); }

void or_default_params(or_params* p) {
  memset(p, 0, sizeof(*p));
  /* Table 1 */
  p->K1 = 30.0; p->R0 = 0.6825; p->eps_bb = 1.0; p->sigma_bb = 0.4430;
  p->K2 = 6.0; p->r0_hb = 0.0; p->rc_hb = 0.3;
  p->eps_ev = 1.0; p->sigma_ss = 1.0; p->sigma_cross = 0.5;   /* Sec. 2: ghosts see the other strand at 0.5 */
  p->K3 = 50.0; p->d_dih = -144.0 * PI / 180.0;
  p->K4 = 30.0; p->lambda_m = 8.0; p->r0_m = 0.34;
  p->K5 = 200.0; p->alpha0 = 90.0 * PI / 180.0;
  p->K6 = 52.0;
  /* Sec. 2: patch 0.5 nm from the bead centre */
  p->mass = 1.0; p->ell = 0.5;
  /* App. A: kT = 1, gamma = 1 in simulation units, dt = 0.005 tau_Br (Eq. 16) */
  p->kT = 1.0; p->gamma = 1.0; p->dt = 0.005;
  p->seed = 0; p->noise = 1; p->steric_phase = 0;
  p->bubble_rule = 0; p->K2_gc = 0.0; p->gc = NULL; p->ring = NULL; p->removed = NULL;
  p->sigma_cross_steric = 1.0;   /* reading A1: two steric beads at sigma = 1 on either strand */
  p->box[0] = p->box[1] = p->box[2] = 0.0;
}

/* ---------------------------------------------------------------- Philox */
/* Philox4x32-10 as published by Salmon, Moraes, Dror, Shaw (SC'11): ten
 * rounds of two 32x32->64 multiplications with the round constants
 * 0xD2511F53 / 0xCD9E8D57 and a Weyl key schedule 0x9E3779B9 / 0xBB67AE85. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ---------------------------------------------------------------- topology */
typedef struct {
  int n_mol;
  const int* n_bp;
  const signed char* ring;   /* per molecule, 1 = circular (may be NULL) */
  int64_t* off;     /* bp offset of each molecule */
  int64_t n_nt;
} topo_t;

static int topo_init(topo_t* t, const or_params* p, int n_mol, const int* n_bp) {
  t->n_mol = n_mol; t->n_bp = n_bp; t->ring = p->ring;
  t->off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_mol + 1));
  if (!t->off) return OR_EINVAL;
  int64_t o = 0;
  for (int m = 0; m < n_mol; ++m) {
    t->off[m] = o;
    if (n_bp[m] < 1 || (t->ring && t->ring[m] && n_bp[m] < 6)) { free(t->off); return OR_EINVAL; }
    o += n_bp[m];
  }
  t->off[n_mol] = o;
  t->n_nt = 2 * o;
  return OR_OK;
}
static void topo_free(topo_t* t) { free(t->off); }

static int mol_of(const topo_t* t, int64_t g) {
  int64_t bp = g / 2;
  int lo = 0, hi = t->n_mol - 1;
  while (lo < hi) { int mid = (lo + hi + 1) / 2; if (t->off[mid] <= bp) lo = mid; else hi = mid - 1; }
  return lo;
}
static int is_ring(const topo_t* t, int m) { return t->ring && t->ring[m]; }
/* nucleotide on strand (g & 1) of base pair k of molecule m, k taken modulo
 * N on a ring; -1 past the end of a linear molecule */
static int64_t nt_at(const topo_t* t, int m, int64_t k, int64_t g) {
  const int N = t->n_bp[m];
  if (is_ring(t, m)) k = ((k % N) + N) % N;
  else if (k < 0 || k >= N) return -1;
  return 2 * (t->off[m] + k) + (g & 1);
}
/* next / previous nucleotide along the same strand in 5'->3' order (Sec. 2):
 * strand A (even slots) runs to increasing k, strand B to decreasing k; on a
 * ring the last nucleotide of a strand is followed by its first. */
static int64_t next_nt(const topo_t* t, int64_t g) {
  int m = mol_of(t, g); int64_t k = g / 2 - t->off[m];
  return nt_at(t, m, (g & 1) == 0 ? k + 1 : k - 1, g);
}
static int64_t prev_nt(const topo_t* t, int64_t g) {
  int m = mol_of(t, g); int64_t k = g / 2 - t->off[m];
  return nt_at(t, m, (g & 1) == 0 ? k - 1 : k + 1, g);
}
/* Sec. 2 / Fig. 1d: along each strand one sterically interacting bead is
 * followed by two ghost beads; the index q is counted 5'->3'.  On a ring
 * whose length is not a multiple of 3 the last steric bead before the
 * junction would sit fewer than 3 nucleotides from the first one after it
 * (gap N - q + phase): it is a ghost instead, leaving one gap of 4 or 5. */
static int is_steric(const or_params* p, const topo_t* t, int64_t g) {
  int m = mol_of(t, g); int64_t k = g / 2 - t->off[m]; int N = t->n_bp[m];
  int64_t q = ((g & 1) == 0) ? k : (N - 1 - k);
  if ((int)(q % 3) != p->steric_phase) return 0;
  return !(is_ring(t, m) && q > N + p->steric_phase - 3);
}

/* site position: site 0 = bead, 1 = patch (Sec. 2) */
static void site_pos(const or_params* p, const double* X, const double* u, int64_t g, int site, double* r) {
  double s = (site == 0 ? -0.5 : 0.5) * p->ell;
  for (int c = 0; c < 3; ++c) r[c] = X[3 * g + c] + s * u[3 * g + c];
}
/* displacement b - a with the minimum image in periodic directions */
static void disp(const or_params* p, const double* a, const double* b, double* d) {
  for (int c = 0; c < 3; ++c) {
    double x = b[c] - a[c];
    if (p->box[c] > 0.0) x -= p->box[c] * nearbyint(x / p->box[c]);
    d[c] = x;
  }
}

/* ---------------------------------------------------------------- terms */
/* Each term gets the displacements of its sites from its first site and
 * returns the force on every site. */

/* App. A Eq. 9 plus the Table 1 backbone WCA (sigma_bb) between consecutive
 * beads of one strand.  d = b_next - b_this; f = force on b_next. */
static int term_fene(const or_params* p, const double* d, double* e_fene, double* e_wca, double* f, double* mag) {
  double r2 = v_dot(d, d), R02 = p->R0 * p->R0;
  if (r2 >= R02) return OR_EFENE;               /* U = infinity for r >= R0 */
  *e_fene = -0.5 * p->K1 * R02 * log(1.0 - r2 / R02);
  double fr = -p->K1 / (1.0 - r2 / R02);        /* -(dU/dr)/r */
  double fw = 0.0;
  *e_wca = 0.0;
  double rc = pow(2.0, 1.0 / 6.0) * p->sigma_bb;
  if (r2 < rc * rc) {
    double s2 = p->sigma_bb * p->sigma_bb / r2, s6 = s2 * s2 * s2, s12 = s6 * s6;
    *e_wca = 4.0 * p->eps_bb * (s12 - s6 + 0.25);
    fw = 24.0 * p->eps_bb * (2.0 * s12 - s6) / r2;
  }
  for (int c = 0; c < 3; ++c) f[c] = (fr + fw) * d[c];
  *mag = (fabs(fr) + fabs(fw)) * sqrt(r2);       /* the two terms separately, for the force scale */
  return OR_OK;
}

/* App. A Eq. 13: Morse stacking between consecutive patches. */
static void term_morse(const or_params* p, const double* d, double* e, double* f) {
  double r = v_norm(d);
  double x = exp(-p->lambda_m * (r - p->r0_m));
  *e = p->K4 * (1.0 - x) * (1.0 - x);
  double dUdr = 2.0 * p->K4 * p->lambda_m * x * (1.0 - x);
  double fr = (r > 0.0) ? -dUdr / r : 0.0;
  for (int c = 0; c < 3; ++c) f[c] = fr * d[c];
}

/* App. A Eq. 10: truncated harmonic hydrogen bond between paired patches;
 * zero (broken) beyond rc, tested on r^2 <= rc^2. */
static void term_hbond(const or_params* p, double K2, const double* d, double* e, double* f) {
  double r2 = v_dot(d, d);
  f[0] = f[1] = f[2] = 0.0; *e = 0.0;
  if (r2 > p->rc_hb * p->rc_hb) return;
  double r = sqrt(r2);
  double w = p->r0_hb - p->rc_hb;
  double k = K2 / (2.0 * w * w);
  *e = k * ((r - p->r0_hb) * (r - p->r0_hb) - (p->rc_hb - p->r0_hb) * (p->rc_hb - p->r0_hb));
  /* -(dU/dr)/r = -2k (r - r0)/r = -2k (1 - r0/r) */
  double fr = (p->r0_hb == 0.0) ? -2.0 * k : ((r > 0.0) ? -2.0 * k * (r - p->r0_hb) / r : 0.0);
  for (int c = 0; c < 3; ++c) f[c] = fr * d[c];
}

/* App. A Eq. 11: WCA (truncated, shifted LJ) of diameter sigma. */
static void term_wca(const or_params* p, const double* d, double sigma, double* e, double* f) {
  double r2 = v_dot(d, d);
  double rc = pow(2.0, 1.0 / 6.0) * sigma;
  f[0] = f[1] = f[2] = 0.0; *e = 0.0;
  if (r2 >= rc * rc) return;
  double s2 = sigma * sigma / r2, s6 = s2 * s2 * s2, s12 = s6 * s6;
  *e = 4.0 * p->eps_ev * (s12 - s6 + 0.25);
  double fr = 24.0 * p->eps_ev * (2.0 * s12 - s6) / r2;
  for (int c = 0; c < 3; ++c) f[c] = fr * d[c];
}

/* App. A Eq. 12: dihedral K3 [1 + cos(phi - d)] on the quadruplet A-E-F-B
 * (bead i, patch i, patch i+1, bead i+1; Sec. 2).  rE, rF, rB are relative to
 * A.  phi follows the IUPAC sign: phi = atan2(|b2| b1.(b2 x b3), (b1 x b2).(b2 x b3)).
 * Gradient of phi from Blondel & Karplus, J. Comput. Chem. 17 (1996) 1132. */
static void term_dihedral(const or_params* p, const double* rE, const double* rF, const double* rB,
                          double* e, double* fA, double* fE, double* fF, double* fB, double* phi_out) {
  double b1[3] = {rE[0], rE[1], rE[2]};
  double b2[3], b3[3];
  v_sub(rF, rE, b2); v_sub(rB, rF, b3);
  double n1[3], n2[3];
  v_cross(b1, b2, n1); v_cross(b2, b3, n2);
  double lb2 = v_norm(b2);
  double n1s = v_dot(n1, n1), n2s = v_dot(n2, n2);
  double y = lb2 * v_dot(b1, n2), x = v_dot(n1, n2);
  double phi = atan2(y, x);
  if (phi_out) *phi_out = phi;
  *e = p->K3 * (1.0 + cos(phi - p->d_dih));
  double dUdphi = -p->K3 * sin(phi - p->d_dih);
  if (n1s <= 0.0 || n2s <= 0.0 || lb2 <= 0.0) {
    for (int c = 0; c < 3; ++c) fA[c] = fE[c] = fF[c] = fB[c] = 0.0;
    return;
  }
  double b1b2 = v_dot(b1, b2), b3b2 = v_dot(b3, b2);
  for (int c = 0; c < 3; ++c) {
    double gA = -lb2 / n1s * n1[c];
    double gB = lb2 / n2s * n2[c];
    double gE = (lb2 / n1s + b1b2 / (n1s * lb2)) * n1[c] + b3b2 / (n2s * lb2) * n2[c];
    double gF = -b1b2 / (n1s * lb2) * n1[c] - (b3b2 / (n2s * lb2) + lb2 / n2s) * n2[c];
    fA[c] = -dUdphi * gA; fE[c] = -dUdphi * gE; fF[c] = -dUdphi * gF; fB[c] = -dUdphi * gB;
  }
}

/* gradient of cos(angle) between v1 and v2 with respect to v1 */
static void dcos_dv1(const double* v1, const double* v2, double l1, double l2, double cs, double* g) {
  for (int c = 0; c < 3; ++c) g[c] = v2[c] / (l1 * l2) - cs * v1[c] / (l1 * l1);
}

/* App. A Eq. 14: planarity (K5/2)(alpha - alpha0)^2, alpha the angle E-F-B
 * with its vertex at patch F (patch i+1) between patch E (patch i) and bead B
 * (bead i+1).  v1 = E - F, v2 = B - F.  Returns forces on E, F, B. */
static void term_planar(const or_params* p, const double* v1, const double* v2,
                        double* e, double* fE, double* fF, double* fB, double* alpha_out) {
  double l1 = v_norm(v1), l2 = v_norm(v2);
  double cs = v_dot(v1, v2) / (l1 * l2);
  if (cs > 1.0) cs = 1.0;
  if (cs < -1.0) cs = -1.0;
  double a = acos(cs);
  if (alpha_out) *alpha_out = a;
  *e = 0.5 * p->K5 * (a - p->alpha0) * (a - p->alpha0);
  double dUda = p->K5 * (a - p->alpha0);
  double sn = sqrt(1.0 - cs * cs);
  if (sn < 1e-12) sn = 1e-12;
  /* F = -dU/da * da/dr, da/dcos = -1/sin */
  double coef = dUda / sn;
  double g1[3], g2[3];
  dcos_dv1(v1, v2, l1, l2, cs, g1);
  dcos_dv1(v2, v1, l2, l1, cs, g2);
  for (int c = 0; c < 3; ++c) {
    fE[c] = coef * g1[c];
    fB[c] = coef * g2[c];
    fF[c] = -(fE[c] + fB[c]);
  }
}

/* App. A Eq. 15: Kratky-Porod K6 [1 + cos(theta)], theta the angle at patch
 * i between patches i-1 and i+1.  v1 = p_{i-1} - p_i, v2 = p_{i+1} - p_i. */
static void term_bend(const or_params* p, const double* v1, const double* v2,
                      double* e, double* f1, double* fv, double* f2) {
  double l1 = v_norm(v1), l2 = v_norm(v2);
  double cs = v_dot(v1, v2) / (l1 * l2);
  *e = p->K6 * (1.0 + cs);
  double g1[3], g2[3];
  dcos_dv1(v1, v2, l1, l2, cs, g1);
  dcos_dv1(v2, v1, l2, l1, cs, g2);
  for (int c = 0; c < 3; ++c) {
    f1[c] = -p->K6 * g1[c];
    f2[c] = -p->K6 * g2[c];
    fv[c] = -(f1[c] + f2[c]);
  }
}

/* ------------------------------------------------------- term collection */
typedef struct { int64_t slot; int site; double f[3]; double mag; } contrib_t;
typedef struct {
  contrib_t c[16]; int n;
  double e[OR_NTERMS];
  double vir[6];
} tout_t;

static void tout_add(tout_t* o, int64_t slot, int site, const double* f, const double* rel) {
  contrib_t* c = &o->c[o->n++];
  c->slot = slot; c->site = site; c->f[0] = f[0]; c->f[1] = f[1]; c->f[2] = f[2];
  c->mag = v_norm(f);
  /* site virial sum_s (r_s - r_ref) (x) F_s, xx yy zz xy xz yz */
  o->vir[0] += rel[0] * f[0]; o->vir[1] += rel[1] * f[1]; o->vir[2] += rel[2] * f[2];
  o->vir[3] += rel[0] * f[1]; o->vir[4] += rel[0] * f[2]; o->vir[5] += rel[1] * f[2];
}

/* Sec. 5: a base pair is open (denatured) when its hydrogen bond is broken,
 * r^2 > rc^2 between the paired patches; a base pair outside molecule m
 * counts as closed (on a ring the index is taken modulo its length). */
static int bp_open(const or_params* p, const topo_t* t, const double* X, const double* u, int m, int64_t bp) {
  const int64_t g = nt_at(t, m, bp - t->off[m], 0);
  if (g < 0) return 0;
  bp = g / 2;
  double pa[3], pb[3], d[3];
  site_pos(p, X, u, 2 * bp, 1, pa);
  site_pos(p, X, u, 2 * bp + 1, 1, pb);
  disp(p, pa, pb, d);
  return v_dot(d, d) > p->rc_hb * p->rc_hb;
}

/* Hydrogen-bond stiffness of base pair bp (Sec. 5: K2(AT) < K2(CG)). */
static double pair_K2(const or_params* p, int64_t bp) {
  if (p->gc && p->gc[bp] && p->K2_gc > 0.0) return p->K2_gc;
  return p->K2;
}

/* All bonded terms owned by nucleotide g (everything that starts at g along
 * its strand in 5'->3' order, plus the bending term centred on g).  With the
 * bubble rule of Sec. 5 the dihedral of the step g -> n is left out when both
 * base pairs lie in a run of at least three consecutive open base pairs, and
 * the bending at g when its three base pairs are all open.  Rule 2 also
 * leaves out what the mask p->removed marks, and records in upd[g] (when not
 * NULL) what this evaluation left out. */
static int owner_terms(const or_params* p, const topo_t* t, const double* X, const double* u, int64_t g, tout_t* o,
                       unsigned char* upd) {
  const unsigned rm0 = (p->bubble_rule == 2 && p->removed) ? p->removed[g] : 0u;
  unsigned rm1 = rm0;
  static const double zero[3] = {0, 0, 0};
  int64_t n = next_nt(t, g), pv = prev_nt(t, g);
  const int m = mol_of(t, g);
  double bg[3], pg[3];
  site_pos(p, X, u, g, 0, bg);
  site_pos(p, X, u, g, 1, pg);
  if (n >= 0) {
    double bn[3], pn[3], d[3], f[3], mf[3], e1, e2;
    site_pos(p, X, u, n, 0, bn);
    site_pos(p, X, u, n, 1, pn);
    /* FENE + backbone WCA: b_g -> b_n */
    disp(p, bg, bn, d);
    double mag;
    if (term_fene(p, d, &e1, &e2, f, &mag) != OR_OK) return OR_EFENE;
    o->e[OR_E_FENE] += e1; o->e[OR_E_BONDWCA] += e2;
    mf[0] = -f[0]; mf[1] = -f[1]; mf[2] = -f[2];
    tout_add(o, g, 0, mf, zero); tout_add(o, n, 0, f, d);
    o->c[o->n - 2].mag = mag; o->c[o->n - 1].mag = mag;
    /* Morse: p_g -> p_n */
    disp(p, pg, pn, d);
    term_morse(p, d, &e1, f);
    o->e[OR_E_MORSE] += e1;
    mf[0] = -f[0]; mf[1] = -f[1]; mf[2] = -f[2];
    tout_add(o, g, 1, mf, zero); tout_add(o, n, 1, f, d);
    /* dihedral A-E-F-B = b_g, p_g, p_n, b_n; positions relative to A */
    double rE[3], rF[3], rB[3], fA[3], fE[3], fF[3], fB[3];
    int in_bubble = 0;
    if (p->bubble_rule) {
      /* pairs kg -> kg + s of the step (s = +1 strand A, -1 strand B) and
       * the pairs that flank it, kg - s and kg + 2s */
      const int64_t kg = g / 2, s = (g & 1) == 0 ? 1 : -1;
      in_bubble = bp_open(p, t, X, u, m, kg) && bp_open(p, t, X, u, m, kg + s) &&
                  (bp_open(p, t, X, u, m, kg - s) || bp_open(p, t, X, u, m, kg + 2 * s));
    }
    if (in_bubble) rm1 |= 1u;
    if (!(rm1 & 1u)) {
      disp(p, bg, pg, rE); disp(p, bg, pn, rF); disp(p, bg, bn, rB);
      term_dihedral(p, rE, rF, rB, &e1, fA, fE, fF, fB, NULL);
      o->e[OR_E_DIHEDRAL] += e1;
      tout_add(o, g, 0, fA, zero); tout_add(o, g, 1, fE, rE); tout_add(o, n, 1, fF, rF); tout_add(o, n, 0, fB, rB);
    }
    /* planarity: angle at p_n between p_g and b_n; positions relative to p_g */
    double v1[3], v2[3], rpn[3], rbn[3];
    disp(p, pn, pg, v1); disp(p, pn, bn, v2);
    term_planar(p, v1, v2, &e1, fE, fF, fB, NULL);
    o->e[OR_E_PLANAR] += e1;
    disp(p, pg, pn, rpn); disp(p, pg, bn, rbn);
    tout_add(o, g, 1, fE, zero); tout_add(o, n, 1, fF, rpn); tout_add(o, n, 0, fB, rbn);
  }
  if (n >= 0 && pv >= 0 && p->bubble_rule && bp_open(p, t, X, u, m, pv / 2) && bp_open(p, t, X, u, m, g / 2) &&
      bp_open(p, t, X, u, m, n / 2))
    rm1 |= 2u;
  if (upd && p->bubble_rule == 2) upd[g] = (unsigned char)rm1;
  if (n >= 0 && pv >= 0 && !(rm1 & 2u)) {
    double pp[3], pn[3], v1[3], v2[3], f1[3], fv[3], f2[3], e1, r1[3], r2[3];
    site_pos(p, X, u, pv, 1, pp);
    site_pos(p, X, u, n, 1, pn);
    disp(p, pg, pp, v1); disp(p, pg, pn, v2);
    term_bend(p, v1, v2, &e1, f1, fv, f2);
    o->e[OR_E_BEND] += e1;
    disp(p, pp, pg, r1); disp(p, pp, pn, r2);
    tout_add(o, pv, 1, f1, zero); tout_add(o, g, 1, fv, r1); tout_add(o, n, 1, f2, r2);
  }
  return OR_OK;
}

/* hydrogen bond of base pair whose strand-A nucleotide is g (even slot) */
static void hbond_terms(const or_params* p, const double* X, const double* u, int64_t g, tout_t* o) {
  static const double zero[3] = {0, 0, 0};
  double pa[3], pb[3], d[3], f[3], mf[3], e;
  site_pos(p, X, u, g, 1, pa);
  site_pos(p, X, u, g + 1, 1, pb);
  disp(p, pa, pb, d);
  term_hbond(p, pair_K2(p, g / 2), d, &e, f);
  o->e[OR_E_HBOND] += e;
  mf[0] = -f[0]; mf[1] = -f[1]; mf[2] = -f[2];
  tout_add(o, g, 1, mf, zero); tout_add(o, g + 1, 1, f, d);
}

/* Typed WCA rule between two beads of the same molecule (Sec. 2, reading
 * A1): two steric beads of one strand use sigma_ss, two steric beads of
 * opposite strands sigma_cross_steric (1 by default, the steric size; <= 0:
 * sigma_cross, the other reading), any other pair of opposite strands
 * sigma_cross (ghosts see the other strand at 0.5); a ghost never interacts
 * with its own strand.  Returns sigma or 0 for no interaction. */
static double pair_sigma(const or_params* p, const topo_t* t, int64_t i, int64_t j) {
  if ((i & 1) != (j & 1)) {
    if (p->sigma_cross_steric > 0.0 && is_steric(p, t, i) && is_steric(p, t, j)) return p->sigma_cross_steric;
    return p->sigma_cross;
  }
  if (is_steric(p, t, i) && is_steric(p, t, j)) return p->sigma_ss;
  return 0.0;
}

/* ------------------------------------------------------- accumulation */
typedef struct {
  double *Fb, *Fp;      /* site forces, may be NULL */
  double *energy, *virial;
  double *Sb, *Sp;      /* sum over terms of |force| per site, may be NULL */
} sink_t;

static void sink_tout(sink_t* s, const tout_t* o, int mol) {
  for (int i = 0; i < o->n; ++i) {
    const contrib_t* c = &o->c[i];
    double* F = (c->site == 0) ? s->Fb : s->Fp;
    if (F) for (int k = 0; k < 3; ++k) F[3 * c->slot + k] += c->f[k];
    double* S = (c->site == 0) ? s->Sb : s->Sp;
    if (S) S[c->slot] += c->mag;
  }
  if (s->energy) for (int k = 0; k < OR_NTERMS; ++k) s->energy[OR_NTERMS * mol + k] += o->e[k];
  if (s->virial) for (int k = 0; k < 6; ++k) s->virial[6 * mol + k] += o->vir[k];
}

static void pair_eval(const or_params* p, const topo_t* t, const double* X, const double* u,
                      int64_t i, int64_t j, int mol, sink_t* s) {
  double sig = pair_sigma(p, t, i, j);
  if (sig <= 0.0) return;
  double bi[3], bj[3], d[3], f[3], e;
  site_pos(p, X, u, i, 0, bi);
  site_pos(p, X, u, j, 0, bj);
  disp(p, bi, bj, d);
  term_wca(p, d, sig, &e, f);
  if (e == 0.0 && f[0] == 0.0 && f[1] == 0.0 && f[2] == 0.0) return;
  if (s->Fb) for (int k = 0; k < 3; ++k) { s->Fb[3 * i + k] -= f[k]; s->Fb[3 * j + k] += f[k]; }
  if (s->Sb) { s->Sb[i] += v_norm(f); s->Sb[j] += v_norm(f); }
  if (s->energy) s->energy[OR_NTERMS * mol + OR_E_WCA] += e;
  if (s->virial) {
    double* v = s->virial + 6 * mol;
    v[0] += d[0] * f[0]; v[1] += d[1] * f[1]; v[2] += d[2] * f[2];
    v[3] += d[0] * f[1]; v[4] += d[0] * f[2]; v[5] += d[1] * f[2];
  }
}

/* External load (Sec. 4.1 / 4.2, Figs. 5 and 7): a force f split equally over
 * the two nucleotides of the last base pair, and a torque T applied as a pure
 * couple on their centres: F_s = T x rho_s / sum |rho|^2, rho_s the offset of
 * centre s from the pair centre projected normal to T.  Forces act at the
 * centre of mass, i.e. half on each site. */
static void external_load(const or_params* p, const topo_t* t, const double* X, int m,
                          const double* ef, const double* et, sink_t* s) {
  int64_t gA = 2 * (t->off[m] + t->n_bp[m] - 1), gB = gA + 1;
  double F[2][3] = {{0, 0, 0}, {0, 0, 0}};
  if (ef) for (int c = 0; c < 3; ++c) { F[0][c] += 0.5 * ef[3 * m + c]; F[1][c] += 0.5 * ef[3 * m + c]; }
  if (et) {
    const double* T = et + 3 * m;
    double Tn = v_norm(T);
    if (Tn > 0.0) {
      double th[3] = {T[0] / Tn, T[1] / Tn, T[2] / Tn};
      double dAB[3];
      disp(p, X + 3 * gA, X + 3 * gB, dAB);
      double rho[2][3];
      for (int c = 0; c < 3; ++c) { rho[0][c] = -0.5 * dAB[c]; rho[1][c] = 0.5 * dAB[c]; }
      double S = 0.0;
      for (int k = 0; k < 2; ++k) {
        double a = v_dot(rho[k], th);
        for (int c = 0; c < 3; ++c) rho[k][c] -= a * th[c];
        S += v_dot(rho[k], rho[k]);
      }
      if (S > 1e-12) {
        for (int k = 0; k < 2; ++k) {
          double tc[3];
          v_cross(T, rho[k], tc);
          for (int c = 0; c < 3; ++c) F[k][c] += tc[c] / S;
        }
      }
    }
  }
  for (int k = 0; k < 2; ++k) {
    int64_t g = gA + k;
    for (int c = 0; c < 3; ++c) {
      if (s->Fb) s->Fb[3 * g + c] += 0.5 * F[k][c];
      if (s->Fp) s->Fp[3 * g + c] += 0.5 * F[k][c];
    }
    if (s->Sb) s->Sb[g] += 0.5 * v_norm(F[k]);
    if (s->Sp) s->Sp[g] += 0.5 * v_norm(F[k]);
  }
}

/* ------------------------------------------------------- cell hash (oracle's own) */
typedef struct { int64_t key; int64_t g; } cell_ent_t;
static int cmp_ent(const void* a, const void* b) {
  const cell_ent_t* x = (const cell_ent_t*)a; const cell_ent_t* y = (const cell_ent_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->g < y->g ? -1 : (x->g > y->g ? 1 : 0);
}
static int64_t cell_key(int mol, const int64_t* c) {
  const int64_t B = (int64_t)1 << 16;
  return ((((int64_t)mol * 2 * B + (c[0] + B)) * 2 * B + (c[1] + B)) * 2 * B) + (c[2] + B);
}

/* Visit every interacting bead pair (i<j) of the system once, either brute
 * force or through a uniform grid of edge >= the largest WCA cutoff. */
static void all_pairs(const or_params* p, const topo_t* t, const double* X, const double* u, int use_cells, sink_t* s) {
  if (!use_cells) {
    for (int m = 0; m < t->n_mol; ++m) {
      int64_t g0 = 2 * t->off[m], g1 = 2 * t->off[m + 1];
      for (int64_t i = g0; i < g1; ++i)
        for (int64_t j = i + 1; j < g1; ++j) pair_eval(p, t, X, u, i, j, m, s);
    }
    return;
  }
  double smax = p->sigma_ss > p->sigma_cross ? p->sigma_ss : p->sigma_cross;
  if (p->sigma_cross_steric > smax) smax = p->sigma_cross_steric;
  double rc = pow(2.0, 1.0 / 6.0) * smax;
  double h[3]; int64_t nc[3];
  for (int c = 0; c < 3; ++c) {
    if (p->box[c] > 0.0) { nc[c] = (int64_t)floor(p->box[c] / rc); if (nc[c] < 1) nc[c] = 1; h[c] = p->box[c] / (double)nc[c]; }
    else { nc[c] = 0; h[c] = rc; }
  }
  int64_t n = t->n_nt;
  cell_ent_t* ent = (cell_ent_t*)malloc(sizeof(cell_ent_t) * (size_t)n);
  int64_t (*cc)[3] = malloc(sizeof(int64_t[3]) * (size_t)n);
  for (int64_t g = 0; g < n; ++g) {
    double b[3]; site_pos(p, X, u, g, 0, b);
    for (int c = 0; c < 3; ++c) {
      double x = b[c];
      if (nc[c] > 0) { x -= p->box[c] * floor(x / p->box[c]); }
      int64_t ci = (int64_t)floor(x / h[c]);
      if (nc[c] > 0) { if (ci >= nc[c]) ci = nc[c] - 1; if (ci < 0) ci = 0; }
      cc[g][c] = ci;
    }
    ent[g].key = cell_key(mol_of(t, g), cc[g]);
    ent[g].g = g;
  }
  qsort(ent, (size_t)n, sizeof(cell_ent_t), cmp_ent);
  for (int64_t i = 0; i < n; ++i) {
    int m = mol_of(t, i);
    int64_t seen[27]; int ns = 0;
    for (int dx = -1; dx <= 1; ++dx) for (int dy = -1; dy <= 1; ++dy) for (int dz = -1; dz <= 1; ++dz) {
      int64_t c[3] = {cc[i][0] + dx, cc[i][1] + dy, cc[i][2] + dz};
      for (int k = 0; k < 3; ++k) if (nc[k] > 0) c[k] = ((c[k] % nc[k]) + nc[k]) % nc[k];
      int64_t key = cell_key(m, c);
      int dup = 0;
      for (int q = 0; q < ns; ++q) if (seen[q] == key) dup = 1;
      if (dup) continue;
      seen[ns++] = key;
      /* lower bound of key */
      int64_t lo = 0, hi = n;
      while (lo < hi) { int64_t mid = (lo + hi) / 2; if (ent[mid].key < key) lo = mid + 1; else hi = mid; }
      for (int64_t q = lo; q < n && ent[q].key == key; ++q) {
        int64_t j = ent[q].g;
        if (j > i) pair_eval(p, t, X, u, i, j, m, s);
      }
    }
  }
  free(ent); free(cc);
}

static int forces_impl(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                       const double* ef, const double* et, double* Fb, double* Fp, double* Fbody, double* Tbody,
                       double* energy, double* virial, int use_cells, double* Sb, double* Sp, unsigned char* upd) {
  topo_t t;
  if (topo_init(&t, p, n_mol, n_bp) != OR_OK) return OR_EINVAL;
  int64_t n = t.n_nt;
  double* fb = Fb ? Fb : (double*)calloc((size_t)(3 * n), sizeof(double));
  double* fp = Fp ? Fp : (double*)calloc((size_t)(3 * n), sizeof(double));
  memset(fb, 0, sizeof(double) * (size_t)(3 * n));
  memset(fp, 0, sizeof(double) * (size_t)(3 * n));
  if (energy) memset(energy, 0, sizeof(double) * (size_t)(OR_NTERMS * n_mol));
  if (virial) memset(virial, 0, sizeof(double) * (size_t)(6 * n_mol));
  if (Sb) memset(Sb, 0, sizeof(double) * (size_t)n);
  if (Sp) memset(Sp, 0, sizeof(double) * (size_t)n);
  sink_t s = {fb, fp, energy, virial, Sb, Sp};
  int rc = OR_OK;
  for (int64_t g = 0; g < n && rc == OR_OK; ++g) {
    tout_t o; memset(&o, 0, sizeof(o));
    int m = mol_of(&t, g);
    if (owner_terms(p, &t, X, u, g, &o, upd) != OR_OK) { rc = OR_EFENE; break; }
    if ((g & 1) == 0) hbond_terms(p, X, u, g, &o);
    sink_tout(&s, &o, m);
  }
  if (rc == OR_OK) {
    all_pairs(p, &t, X, u, use_cells, &s);
    for (int m = 0; m < n_mol; ++m) external_load(p, &t, X, m, ef, et, &s);
    for (int64_t g = 0; g < n; ++g) {
      const double* ug = u + 3 * g;
      double dF[3] = {fp[3 * g] - fb[3 * g], fp[3 * g + 1] - fb[3 * g + 1], fp[3 * g + 2] - fb[3 * g + 2]};
      double tq[3];
      v_cross(ug, dF, tq);
      for (int c = 0; c < 3; ++c) {
        if (Fbody) Fbody[3 * g + c] = fb[3 * g + c] + fp[3 * g + c];
        if (Tbody) Tbody[3 * g + c] = 0.5 * p->ell * tq[c];   /* (ell/2) u x (F_p - F_b) */
      }
    }
  }
  if (!Fb) free(fb);
  if (!Fp) free(fp);
  topo_free(&t);
  return rc;
}

int or_forces(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
              const double* ef, const double* et, double* Fb, double* Fp, double* Fbody, double* Tbody,
              double* energy, double* virial) {
  return forces_impl(p, n_mol, n_bp, X, u, ef, et, Fb, Fp, Fbody, Tbody, energy, virial, 0, NULL, NULL, NULL);
}
int or_force_scale(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                   const double* ef, const double* et, double* Sb, double* Sp) {
  return forces_impl(p, n_mol, n_bp, X, u, ef, et, NULL, NULL, NULL, NULL, NULL, NULL, 1, Sb, Sp, NULL);
}
int or_forces_cells(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                    const double* ef, const double* et, double* Fb, double* Fp, double* Fbody, double* Tbody,
                    double* energy, double* virial) {
  return forces_impl(p, n_mol, n_bp, X, u, ef, et, Fb, Fp, Fbody, Tbody, energy, virial, 1, NULL, NULL, NULL);
}

int or_forces_sampled(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                      const double* ef, const double* et, int ns, const int64_t* idx, double* Fb, double* Fp,
                      double* Sb, double* Sp) {
  topo_t t;
  if (topo_init(&t, p, n_mol, n_bp) != OR_OK) return OR_EINVAL;
  int rc = OR_OK;
  for (int q = 0; q < ns && rc == OR_OK; ++q) {
    int64_t g = idx[q];
    int m = mol_of(&t, g);
    double fb[3] = {0, 0, 0}, fp[3] = {0, 0, 0}, sb = 0.0, sp = 0.0;
    int64_t owners[3] = {prev_nt(&t, g), g, next_nt(&t, g)};
    for (int k = 0; k < 3; ++k) {
      if (owners[k] < 0) continue;
      tout_t o; memset(&o, 0, sizeof(o));
      if (owner_terms(p, &t, X, u, owners[k], &o, NULL) != OR_OK) { rc = OR_EFENE; break; }
      for (int i = 0; i < o.n; ++i) if (o.c[i].slot == g) {
        double* F = o.c[i].site == 0 ? fb : fp;
        for (int c = 0; c < 3; ++c) F[c] += o.c[i].f[c];
        *(o.c[i].site == 0 ? &sb : &sp) += o.c[i].mag;
      }
    }
    {
      tout_t o; memset(&o, 0, sizeof(o));
      hbond_terms(p, X, u, g & ~(int64_t)1, &o);
      for (int i = 0; i < o.n; ++i) if (o.c[i].slot == g) {
        for (int c = 0; c < 3; ++c) fp[c] += o.c[i].f[c];
        sp += o.c[i].mag;
      }
    }
    /* pairs with every other bead of the molecule */
    int64_t g0 = 2 * t.off[m], g1 = 2 * t.off[m + 1];
    double bi[3]; site_pos(p, X, u, g, 0, bi);
    for (int64_t j = g0; j < g1; ++j) {
      if (j == g) continue;
      double sig = pair_sigma(p, &t, g, j);
      if (sig <= 0.0) continue;
      double bj[3], d[3], f[3], e;
      site_pos(p, X, u, j, 0, bj);
      disp(p, bi, bj, d);
      term_wca(p, d, sig, &e, f);
      for (int c = 0; c < 3; ++c) fb[c] -= f[c];
      sb += v_norm(f);
    }
    /* external load */
    if (g / 2 == t.off[m] + n_bp[m] - 1) {
      double* tmpb = (double*)calloc((size_t)(3 * t.n_nt), sizeof(double));
      double* tmpp = (double*)calloc((size_t)(3 * t.n_nt), sizeof(double));
      sink_t s = {tmpb, tmpp, NULL, NULL, NULL, NULL};
      external_load(p, &t, X, m, ef, et, &s);
      for (int c = 0; c < 3; ++c) { fb[c] += tmpb[3 * g + c]; fp[c] += tmpp[3 * g + c]; }
      sb += v_norm(tmpb + 3 * g); sp += v_norm(tmpp + 3 * g);
      free(tmpb); free(tmpp);
    }
    for (int c = 0; c < 3; ++c) { Fb[3 * q + c] = fb[c]; Fp[3 * q + c] = fp[c]; }
    if (Sb) Sb[q] = sb;
    if (Sp) Sp[q] = sp;
  }
  topo_free(&t);
  return rc;
}

int64_t or_pairs(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                 double extra, int64_t cap, int64_t* pi, int64_t* pj) {
  topo_t t;
  if (topo_init(&t, p, n_mol, n_bp) != OR_OK) return -1;
  int64_t cnt = 0;
  for (int m = 0; m < n_mol; ++m) {
    int64_t g0 = 2 * t.off[m], g1 = 2 * t.off[m + 1];
    for (int64_t i = g0; i < g1; ++i) {
      double bi[3]; site_pos(p, X, u, i, 0, bi);
      for (int64_t j = i + 1; j < g1; ++j) {
        double sig = pair_sigma(p, &t, i, j);
        if (sig <= 0.0) continue;
        double bj[3], d[3];
        site_pos(p, X, u, j, 0, bj);
        disp(p, bi, bj, d);
        double rl = pow(2.0, 1.0 / 6.0) * sig + extra;
        if (v_dot(d, d) < rl * rl) {
          if (cnt < cap) { pi[cnt] = i; pj[cnt] = j; }
          ++cnt;
        }
      }
    }
  }
  topo_free(&t);
  return cnt;
}

/* ------------------------------------------------------- helix and velocities */
/* Ideal relaxed helix (Sec. 2, Fig. 1b-c): both patches of base pair k sit on
 * the axis at height rise*k (the hydrogen bond rest length r0 is zero, Table
 * 1); the bead of A_k is a distance ell from its patch at azimuth k*twist, the
 * bead of B_k on the opposite side (reading A3).  rise = Morse r0 (0.34 nm),
 * twist = dihedral minimum (d + 180 deg = 36 deg). */
void or_ideal_helix(const or_params* p, int n_bp, const double o[3], double* X, double* u) {
  double twist = p->d_dih + PI;
  for (int k = 0; k < n_bp; ++k) {
    double pz = o[2] + p->r0_m * k;
    for (int s = 0; s < 2; ++s) {
      double ang = twist * k + (s ? PI : 0.0);
      double dir[3] = {cos(ang), sin(ang), 0.0};
      double patch[3] = {o[0], o[1], pz};
      double bead[3] = {o[0] + p->ell * dir[0], o[1] + p->ell * dir[1], pz};
      int64_t g = 2 * (int64_t)k + s;
      for (int c = 0; c < 3; ++c) {
        X[3 * g + c] = 0.5 * (bead[c] + patch[c]);
        u[3 * g + c] = -dir[c];          /* unit vector bead -> patch */
      }
    }
  }
}

static double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* Maxwell-Boltzmann velocities: Box-Muller normals from the Philox stream
 * with counter (local nucleotide, 0xFFFFFFFF, 0xFFFFFFFF, 2*mol + block) and
 * key (seed low, seed high); angular velocity normal to u. */
void or_mb_velocities(const or_params* p, int mol, int n_bp, const double* u, int tether, double* V, double* Om) {
  double M = 2.0 * p->mass, I = 0.5 * p->mass * p->ell * p->ell;
  uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
  int64_t n = 2 * (int64_t)n_bp;
  for (int64_t l = 0; l < n; ++l) {
    double z[8];
    for (int b = 0; b < 2; ++b) {
      uint32_t ctr[4] = {(uint32_t)l, 0xFFFFFFFFu, 0xFFFFFFFFu, (uint32_t)(2 * mol + b)}, r[4];
      or_philox4x32_10(ctr, key, r);
      for (int q = 0; q < 2; ++q) {
        double a = u01(r[2 * q]), c = u01(r[2 * q + 1]);
        double rad = sqrt(-2.0 * log(a));
        z[4 * b + 2 * q] = rad * cos(2.0 * PI * c);
        z[4 * b + 2 * q + 1] = rad * sin(2.0 * PI * c);
      }
    }
    const double* ul = u + 3 * l;
    double ax[3] = {0, 0, 1};
    if (fabs(ul[2]) > 0.9) { ax[0] = 1; ax[2] = 0; }
    double e1[3], e2[3];
    v_cross(ul, ax, e1);
    double ln = v_norm(e1);
    for (int c = 0; c < 3; ++c) e1[c] /= ln;
    v_cross(ul, e1, e2);
    double sv = sqrt(p->kT / M), sw = sqrt(p->kT / I);
    for (int c = 0; c < 3; ++c) {
      V[3 * l + c] = sv * z[c];
      Om[3 * l + c] = sw * (z[3] * e1[c] + z[4] * e2[c]);
    }
  }
  /* remove net momentum of the mobile nucleotides, freeze the anchor */
  int64_t first = tether ? 2 : 0;
  double mean[3] = {0, 0, 0};
  for (int64_t l = first; l < n; ++l) for (int c = 0; c < 3; ++c) mean[c] += V[3 * l + c];
  if (n > first) for (int c = 0; c < 3; ++c) mean[c] /= (double)(n - first);
  for (int64_t l = first; l < n; ++l) for (int c = 0; c < 3; ++c) V[3 * l + c] -= mean[c];
  for (int64_t l = 0; l < first; ++l) for (int c = 0; c < 3; ++c) { V[3 * l + c] = 0.0; Om[3 * l + c] = 0.0; }
}

/* ------------------------------------------------------- Langevin dynamics */
/* Noise of both sites of one nucleotide from one Philox4x32-10 draw with
 * counter (local nucleotide, step low, step high, mol) and key (seed low,
 * seed high).  The four output words x, y, z, w give six 21-bit integers:
 * the top 21 bits of x, y, z (bead x, y, z) and of w (patch x); the low 11
 * bits of x with bits 0-9 of y above them (patch y); the same of z and w
 * (patch z).  U = (k + 1/2) 2^-21.  Uniform mode draws the variance matched
 * uniform sqrt(24 gamma kT / dt) (U - 1/2); Gaussian mode takes Box-Muller
 * pairs (U0, U1), (U2, U3), (U4, U5) with standard deviation sqrt(2 gamma kT / dt). */
static void nucleotide_noise(const or_params* p, int mol, int64_t local, int64_t step, double* eb, double* ep) {
  double e[6] = {0, 0, 0, 0, 0, 0};
  if (p->noise != 0) {
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)local, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)mol}, r[4];
    or_philox4x32_10(ctr, key, r);
    uint32_t k[6] = {r[0] >> 11, r[1] >> 11, r[2] >> 11, r[3] >> 11,
                     (r[0] & 0x7FFu) | ((r[1] & 0x3FFu) << 11), (r[2] & 0x7FFu) | ((r[3] & 0x3FFu) << 11)};
    if (p->noise == 1) {
      double c = ldexp(sqrt(24.0 * p->gamma * p->kT / p->dt), -21);
      for (int q = 0; q < 6; ++q) e[q] = ((double)k[q] - 1048575.5) * c;
    } else {
      double a = sqrt(2.0 * p->gamma * p->kT / p->dt);
      for (int q = 0; q < 6; q += 2) {
        double u0 = ldexp((double)k[q] + 0.5, -21), u1 = ldexp((double)k[q + 1] + 0.5, -21);
        double rad = sqrt(-2.0 * log(u0));
        e[q] = a * rad * cos(2.0 * PI * u1);
        e[q + 1] = a * rad * sin(2.0 * PI * u1);
      }
    }
  }
  for (int c = 0; c < 3; ++c) { eb[c] = e[c]; ep[c] = e[3 + c]; }
}

/* Total (conservative + external + friction + noise) force and torque on a
 * mobile nucleotide (App. A Eq. 8 applied to each site: friction -gamma v_s,
 * noise eta_s; summed over the rigid dumbbell: -2 gamma V and
 * -gamma (ell^2/2) Omega). */
static void total_force(const or_params* p, int mol, int64_t local, int64_t step, const double* F, const double* T,
                        const double* V, const double* Om, const double* u, double* Ft, double* Tt) {
  double eb[3], ep[3];
  nucleotide_noise(p, mol, local, step, eb, ep);
  double de[3] = {ep[0] - eb[0], ep[1] - eb[1], ep[2] - eb[2]}, tn[3];
  v_cross(u, de, tn);
  double gr = p->gamma * 0.5 * p->ell * p->ell;
  for (int c = 0; c < 3; ++c) {
    Ft[c] = F[c] - 2.0 * p->gamma * V[c] + eb[c] + ep[c];
    Tt[c] = T[c] - gr * Om[c] + 0.5 * p->ell * tn[c];
  }
}

int or_run(const or_params* p, int n_mol, const int* n_bp, double* X, double* V, double* u, double* Om,
           const double* ef, const double* et, const int* tether, int64_t step0, int64_t nsteps, int use_cells) {
  topo_t t;
  if (topo_init(&t, p, n_mol, n_bp) != OR_OK) return OR_EINVAL;
  int64_t n = t.n_nt;
  double* F = (double*)malloc(sizeof(double) * (size_t)(3 * n));
  double* T = (double*)malloc(sizeof(double) * (size_t)(3 * n));
  double M = 2.0 * p->mass, I = 0.5 * p->mass * p->ell * p->ell;
  /* rule 2: the mask carries across steps; each force evaluation reads it and
   * adds what it left out */
  or_params q = *p;
  unsigned char* own = NULL;
  if (q.bubble_rule == 2 && !q.removed) q.removed = own = (unsigned char*)calloc((size_t)n, 1);
  int rc = OR_OK;
  for (int64_t s = step0; s < step0 + nsteps; ++s) {
    rc = forces_impl(&q, n_mol, n_bp, X, u, ef, et, NULL, NULL, F, T, NULL, NULL, use_cells, NULL, NULL,
                     q.bubble_rule == 2 ? q.removed : NULL);
    if (rc != OR_OK) break;
    for (int64_t g = 0; g < n; ++g) {
      int m = mol_of(&t, g);
      int64_t local = g - 2 * t.off[m];
      double* Xg = X + 3 * g; double* Vg = V + 3 * g; double* ug = u + 3 * g; double* Og = Om + 3 * g;
      if (tether && tether[m] && local < 2) {      /* anchored base pair (Sec. 4.1) */
        for (int c = 0; c < 3; ++c) { Vg[c] = 0.0; Og[c] = 0.0; }
        continue;
      }
      double Ft[3], Tt[3];
      total_force(p, m, local, s, F + 3 * g, T + 3 * g, Vg, Og, ug, Ft, Tt);
      /* kick: V_{n+1/2} = V_{n-1/2} + dt/M F_n, same for Omega, kept normal to u_n */
      for (int c = 0; c < 3; ++c) { Vg[c] += p->dt / M * Ft[c]; Og[c] += p->dt / I * Tt[c]; }
      double a = v_dot(Og, ug);
      for (int c = 0; c < 3; ++c) Og[c] -= a * ug[c];
      /* drift: X_{n+1} = X_n + dt V_{n+1/2}; u rotated about Omega by |Omega| dt */
      for (int c = 0; c < 3; ++c) Xg[c] += p->dt * Vg[c];
      double w = v_norm(Og);
      if (w > 0.0) {
        double ph = w * p->dt, cs = cos(ph), sn = sin(ph);
        double ax[3] = {Og[0] / w, Og[1] / w, Og[2] / w}, xu[3];
        v_cross(ax, ug, xu);
        double nu[3];
        for (int c = 0; c < 3; ++c) nu[c] = ug[c] * cs + xu[c] * sn;
        double l = v_norm(nu);
        for (int c = 0; c < 3; ++c) ug[c] = nu[c] / l;
      }
    }
  }
  free(F); free(T); free(own);
  topo_free(&t);
  return rc;
}

int or_energy(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* V,
              const double* u, const double* Om, const double* ef, const double* et,
              const int* tether, int64_t step, double* energy, double* virial) {
  topo_t t;
  if (topo_init(&t, p, n_mol, n_bp) != OR_OK) return OR_EINVAL;
  int64_t n = t.n_nt;
  double* F = (double*)malloc(sizeof(double) * (size_t)(3 * n));
  double* T = (double*)malloc(sizeof(double) * (size_t)(3 * n));
  int rc = forces_impl(p, n_mol, n_bp, X, u, ef, et, NULL, NULL, F, T, energy, virial, 0, NULL, NULL, NULL);
  double M = 2.0 * p->mass, I = 0.5 * p->mass * p->ell * p->ell;
  if (rc == OR_OK && energy) {
    for (int64_t g = 0; g < n; ++g) {
      int m = mol_of(&t, g);
      int64_t local = g - 2 * t.off[m];
      if (tether && tether[m] && local < 2) continue;
      double Ft[3], Tt[3], Vf[3], Of[3];
      total_force(p, m, local, step, F + 3 * g, T + 3 * g, V + 3 * g, Om + 3 * g, u + 3 * g, Ft, Tt);
      /* full-step velocities V_n = V_{n-1/2} + dt/(2M) F_n */
      for (int c = 0; c < 3; ++c) { Vf[c] = V[3 * g + c] + 0.5 * p->dt / M * Ft[c]; Of[c] = Om[3 * g + c] + 0.5 * p->dt / I * Tt[c]; }
      double a = v_dot(Of, u + 3 * g);
      for (int c = 0; c < 3; ++c) Of[c] -= a * u[3 * g + c];
      energy[OR_NTERMS * m + OR_E_KIN_T] += 0.5 * M * v_dot(Vf, Vf);
      energy[OR_NTERMS * m + OR_E_KIN_R] += 0.5 * I * v_dot(Of, Of);
    }
  }
  free(F); free(T);
  topo_free(&t);
  return rc;
}

/* ------------------------------------------------------- observables */
/* Gauss linking integral (App. C Eq. 17, read with the vector r_R - r_B in
 * the numerator) of two closed polygons, evaluated exactly for every pair of
 * straight segments as the signed solid angle of the quadrilateral they span
 * (Klenin & Langowski, Biopolymers 54 (2000) 307). */
static double seg_pair_lk(const double* r1, const double* r2, const double* r3, const double* r4) {
  double r13[3], r14[3], r23[3], r24[3], r12[3], r34[3];
  v_sub(r3, r1, r13); v_sub(r4, r1, r14); v_sub(r3, r2, r23); v_sub(r4, r2, r24);
  v_sub(r2, r1, r12); v_sub(r4, r3, r34);
  double n[4][3];
  v_cross(r13, r14, n[0]); v_cross(r14, r24, n[1]); v_cross(r24, r23, n[2]); v_cross(r23, r13, n[3]);
  for (int k = 0; k < 4; ++k) {
    double l = v_norm(n[k]);
    if (l < 1e-300) return 0.0;
    for (int c = 0; c < 3; ++c) n[k][c] /= l;
  }
  double om = 0.0;
  for (int k = 0; k < 4; ++k) {
    double x = v_dot(n[k], n[(k + 1) % 4]);
    if (x > 1.0) x = 1.0;
    if (x < -1.0) x = -1.0;
    om += asin(x);
  }
  double c[3];
  v_cross(r34, r12, c);
  double sg = v_dot(c, r13);
  if (sg > 0) return om / (4.0 * PI);
  if (sg < 0) return -om / (4.0 * PI);
  return 0.0;
}

double or_linking_number(int na, const double* a, int nb, const double* b) {
  double lk = 0.0;
  for (int i = 0; i < na; ++i) {
    const double* r1 = a + 3 * i; const double* r2 = a + 3 * ((i + 1) % na);
    for (int j = 0; j < nb; ++j) {
      const double* r3 = b + 3 * j; const double* r4 = b + 3 * ((j + 1) % nb);
      lk += seg_pair_lk(r1, r2, r3, r4);
    }
  }
  return lk;
}

/* Closure of the two open strands (App. C, Fig. 12): each bead curve (ordered
 * by base-pair index) is extended from both ends along the end-to-end axis e
 * by a distance D, both extensions are moved out by a distance F along a fixed
 * direction normal to e, and the curve is closed there.  D and F exceed the
 * molecule's extent so the closing path stays clear of it. */
static void close_curve(const double* c, int N, const double* e, const double* eperp, double D, double F, double* out) {
  for (int k = 0; k < N; ++k) for (int q = 0; q < 3; ++q) out[3 * k + q] = c[3 * k + q];
  const double* c0 = c; const double* c1 = c + 3 * (N - 1);
  for (int q = 0; q < 3; ++q) {
    out[3 * N + q] = c1[q] + D * e[q];
    out[3 * (N + 1) + q] = c1[q] + D * e[q] + F * eperp[q];
    out[3 * (N + 2) + q] = c0[q] - D * e[q] + F * eperp[q];
    out[3 * (N + 3) + q] = c0[q] - D * e[q];
  }
}

int or_observables(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                   int mol, int with_lk, double* out) {
  topo_t t;
  if (topo_init(&t, p, n_mol, n_bp) != OR_OK || mol < 0 || mol >= n_mol) return OR_EINVAL;
  int N = n_bp[mol];
  int64_t g0 = 2 * t.off[mol];
  double* mid = (double*)malloc(sizeof(double) * 3 * (size_t)N);
  double* bA = (double*)malloc(sizeof(double) * 3 * (size_t)N);
  double* bB = (double*)malloc(sizeof(double) * 3 * (size_t)N);
  int denat = 0;
  for (int k = 0; k < N; ++k) {
    double pa[3], pb[3], d[3];
    site_pos(p, X, u, g0 + 2 * k, 1, pa);
    site_pos(p, X, u, g0 + 2 * k + 1, 1, pb);
    disp(p, pa, pb, d);
    if (v_dot(d, d) > p->rc_hb * p->rc_hb) ++denat;       /* broken bond (Sec. 2, Sec. 5) */
    for (int c = 0; c < 3; ++c) mid[3 * k + c] = pa[c] + 0.5 * d[c];
    double ba[3], bb[3], db[3];
    site_pos(p, X, u, g0 + 2 * k, 0, ba);
    site_pos(p, X, u, g0 + 2 * k + 1, 0, bb);
    disp(p, ba, bb, db);
    for (int c = 0; c < 3; ++c) { bA[3 * k + c] = ba[c]; bB[3 * k + c] = ba[c] + db[c]; }
  }
  /* Sec. 4.1: R_z = [r(L) - r(0)] . e_z, r the base-pair centre (patch midpoint) */
  out[0] = mid[3 * (N - 1) + 2] - mid[2];
  out[1] = (double)denat / (double)N;
  /* Sec. 3.2 / App. B: frames (f, v, t) per base-pair step; twist increment
   * alpha + gamma of the ZYZ Euler rotation between consecutive frames.  A
   * ring has N steps (the last one closes it) and N increments, a linear
   * molecule N - 1 steps and N - 2 increments. */
  const int ring = is_ring(&t, mol);
  const int nfr = ring ? N : N - 1, ninc = ring ? N : N - 2;
  double tw = 0.0;
  if (N >= 3) {
    double (*fr)[3][3] = malloc(sizeof(double[3][3]) * (size_t)nfr);
    for (int k = 0; k < nfr; ++k) {
      double tv[3], w[3];
      v_sub(mid + 3 * ((k + 1) % N), mid + 3 * k, tv);
      double l = v_norm(tv);
      for (int c = 0; c < 3; ++c) tv[c] /= l;
      v_sub(bB + 3 * k, bA + 3 * k, w);
      double a = v_dot(w, tv);
      for (int c = 0; c < 3; ++c) w[c] -= a * tv[c];
      l = v_norm(w);
      for (int c = 0; c < 3; ++c) w[c] /= l;
      double vv[3];
      v_cross(tv, w, vv);
      for (int c = 0; c < 3; ++c) { fr[k][0][c] = w[c]; fr[k][1][c] = vv[c]; fr[k][2][c] = tv[c]; }
    }
    for (int k = 0; k < ninc; ++k) {
      double R[3][3];
      for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) R[i][j] = v_dot(fr[k][i], fr[(k + 1) % nfr][j]);
      tw += atan2(R[1][0] - R[0][1], R[0][0] + R[1][1]);
    }
    free(fr);
    tw /= 2.0 * PI;
  }
  out[2] = tw;
  out[3] = (N >= 3) ? (double)ninc * (p->d_dih + PI) / (2.0 * PI) : 0.0;
  out[4] = out[5] = 0.0;
  if (with_lk && ring) {
    /* App. C Eq. 17 on the two closed bead curves of a ring: no closure */
    out[4] = or_linking_number(N, bA, N, bB);
    out[5] = out[4] - out[2];
  } else if (with_lk && N >= 2) {
    double e[3];
    v_sub(mid + 3 * (N - 1), mid, e);
    double le = v_norm(e);
    if (le < 1e-12) { e[0] = 0; e[1] = 0; e[2] = 1; le = 1; }
    for (int c = 0; c < 3; ++c) e[c] /= le;
    double ax[3] = {1, 0, 0};
    if (fabs(e[0]) > 0.9) { ax[0] = 0; ax[1] = 1; }
    double ep[3];
    v_cross(e, ax, ep);
    double lp = v_norm(ep);
    for (int c = 0; c < 3; ++c) ep[c] /= lp;
    double ext = 0.0;
    for (int k = 0; k < N; ++k) {
      double d1[3], d2[3];
      v_sub(bA + 3 * k, mid, d1); v_sub(bB + 3 * k, mid, d2);
      double a1 = v_norm(d1), a2 = v_norm(d2);
      if (a1 > ext) ext = a1;
      if (a2 > ext) ext = a2;
    }
    double D = ext + 5.0, F = 2.0 * ext + 10.0;
    double* ca = (double*)malloc(sizeof(double) * 3 * (size_t)(N + 4));
    double* cb = (double*)malloc(sizeof(double) * 3 * (size_t)(N + 4));
    close_curve(bA, N, e, ep, D, F, ca);
    close_curve(bB, N, e, ep, D, F, cb);
    out[4] = or_linking_number(N + 4, ca, N + 4, cb);
    out[5] = out[4] - out[2];
    free(ca); free(cb);
  }
  free(mid); free(bA); free(bB);
  topo_free(&t);
  return OR_OK;
}
