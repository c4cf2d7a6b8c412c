/*
 * oracle.h -- plain FP64 CPU restatement of the single-nucleotide dsDNA model
 * of Fosado et al., "A single nucleotide resolution model for large-scale
 * simulations of double stranded DNA" (arXiv:1608.03722).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the independent checker for the
 * CUDA library.  It shares no source, header, table or helper with the CUDA
 * path and is never called by it.  Only the test-suite, the smoke check in
 * __graft_entry__.py and the cpu_baseline leg of bench.py may load it.
 *
 * Everything is double precision, written for clarity, not speed: every
 * interaction is evaluated from its formula, pairs are found by brute force
 * (or by a plain cell hash whose pair set is tested against brute force).
 *
 * Conventions (shared with the CUDA library only through the paper and the
 * written readings, not through code):
 *   - A molecule of N base pairs holds 2N nucleotides.  Global slot
 *     g = 2*(bp_offset + k) + s, s = 0 for strand A nucleotide k, s = 1 for
 *     strand B nucleotide k (the partner of A_k).  Strand A runs 5'->3' with
 *     increasing k, strand B with decreasing k (antiparallel, Sec. 2).
 *   - Host arrays are AoS: X[3*g + c].
 *   - A nucleotide is a rigid body of a backbone bead and a base patch a
 *     distance ell apart (Sec. 2, Fig. 1a), each of mass m: bead
 *     b = X - (ell/2) u, patch p = X + (ell/2) u.
 *   - Velocities carried in the state are half-step (leapfrog) values.
 */
#ifndef DSDNA_ORACLE_H
#define DSDNA_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define OR_NTERMS 10
enum {
  OR_E_FENE = 0,   /* App. A Eq. 9 */
  OR_E_BONDWCA,    /* Table 1 backbone WCA, sigma = 0.443 */
  OR_E_HBOND,      /* App. A Eq. 10 */
  OR_E_WCA,        /* App. A Eq. 11, typed (Sec. 2) */
  OR_E_DIHEDRAL,   /* App. A Eq. 12 */
  OR_E_MORSE,      /* App. A Eq. 13 */
  OR_E_PLANAR,     /* App. A Eq. 14 */
  OR_E_BEND,       /* App. A Eq. 15 */
  OR_E_KIN_T,      /* translational kinetic energy (full-step velocities) */
  OR_E_KIN_R       /* rotational kinetic energy (full-step velocities) */
};

enum { OR_OK = 0, OR_EINVAL = -1, OR_EFENE = -4 };

typedef struct {
  /* Table 1 */
  double K1, R0, eps_bb, sigma_bb;     /* FENE + backbone WCA */
  double K2, r0_hb, rc_hb;             /* hydrogen bond */
  double eps_ev, sigma_ss, sigma_cross;/* steric WCA: two steric beads / cross-strand pair with a ghost */
  double K3, d_dih;                    /* dihedral, d in radians */
  double K4, lambda_m, r0_m;           /* Morse stacking */
  double K5, alpha0;                   /* planarity, alpha0 in radians */
  double K6;                           /* Kratky-Porod bending */
  /* rigid nucleotide (Sec. 2) */
  double mass;                         /* per site */
  double ell;                          /* bead-patch distance */
  /* Langevin (App. A Eq. 8, Eq. 16) */
  double kT, gamma, dt;
  uint64_t seed;
  int noise;                           /* 0 off, 1 uniform (variance matched), 2 Gaussian */
  int steric_phase;                    /* steric iff (index along strand) % 3 == phase */
  double box[3];                       /* > 0: periodic edge; <= 0: open */
  /* Sec. 5 denaturation */
  int bubble_rule;                     /* no dihedral / bending inside bubbles of > 2 open base pairs:
                                          0 off, 1 while the bubble lasts, 2 for good once inside one */
  double K2_gc;                        /* hydrogen-bond stiffness of G.C pairs (<= 0: K2) */
  const signed char* gc;               /* per base pair over all molecules: 1 = G.C, 0 = A.T (NULL: all K2) */
  /* Sec. 6 supercoiled rings: per molecule, 1 = circular (each strand's last
   * nucleotide bonded to its first; at least 6 bp), 0 = linear (NULL: all linear) */
  const signed char* ring;
  /* bubble_rule 2: per nucleotide slot, bit 0 = dihedral of the step to the
   * next nucleotide removed, bit 1 = bending centred on it removed.  Read by
   * every force evaluation, extended by or_run (NULL: nothing removed yet; or_run
   * then keeps its own mask for the run). */
  unsigned char* removed;
  /* Sec. 2, reading A1: sigma of a pair of steric beads on opposite strands
   * (default 1, the steric size); <= 0 gives such pairs sigma_cross like any
   * other cross-strand pair (the other reading). */
  double sigma_cross_steric;
} or_params;

void or_default_params(or_params* p);

/* Philox4x32-10 (Salmon et al., SC'11), counter ctr[4], key key[2]. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Ideal relaxed helix of n_bp base pairs along +z starting at origin o. */
void or_ideal_helix(const or_params* p, int n_bp, const double o[3], double* X, double* u);

/* Maxwell-Boltzmann velocities from the Philox init stream of molecule mol. */
void or_mb_velocities(const or_params* p, int mol, int n_bp, const double* u, int tether,
                      double* V, double* Om);

/* Conservative site forces on every nucleotide of every molecule.
 * Fb, Fp: bead / patch forces [3*n_nt] (may be NULL); Fbody, Tbody: body force
 * and torque [3*n_nt] (may be NULL); energy: [OR_NTERMS*n_mol] potential terms
 * (kinetic slots zero) (may be NULL); virial [6*n_mol] xx yy zz xy xz yz (may
 * be NULL).  ext_f / ext_t: [3*n_mol] applied end force / torque (may be NULL).
 * Pairs by brute force.  Returns OR_OK or OR_EFENE. */
int or_forces(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
              const double* ext_f, const double* ext_t,
              double* Fb, double* Fp, double* Fbody, double* Tbody, double* energy, double* virial);

/* Same, using the oracle's own plain cell hash for the pair search (for large N). */
int or_forces_cells(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                    const double* ext_f, const double* ext_t,
                    double* Fb, double* Fp, double* Fbody, double* Tbody, double* energy, double* virial);

/* Site forces on a sample of nucleotides only (global slots idx[0..ns-1]);
 * pairs by brute force over the sample's molecule.  Fb/Fp are [3*ns];
 * Sb/Sp (may be NULL) receive the sum over contributing terms of |force|. */
int or_forces_sampled(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                      const double* ext_f, const double* ext_t, int ns, const int64_t* idx,
                      double* Fb, double* Fp, double* Sb, double* Sp);

/* Condition scale of the site forces: for every site the sum over all terms
 * acting on it of the magnitude of that term's force [n_nt] each.  A
 * floating-point evaluation of the total force has an error bounded by a
 * small multiple of the unit round-off times this sum. */
int or_force_scale(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                   const double* ext_f, const double* ext_t, double* Sb, double* Sp);

/* All interacting bead pairs (i<j, global slots) with |d| < r_cut(type) + extra, brute force.
 * Writes at most cap pairs into pi/pj, returns the total count. */
int64_t or_pairs(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                 double extra, int64_t cap, int64_t* pi, int64_t* pj);

/* nsteps of Langevin dynamics starting at step counter step0 (state in place).
 * tether[n_mol]: 1 freezes base pair 0 of that molecule.  use_cells selects the
 * cell-hash pair search.  Returns OR_OK or OR_EFENE. */
int or_run(const or_params* p, int n_mol, const int* n_bp, double* X, double* V, double* u, double* Om,
           const double* ext_f, const double* ext_t, const int* tether, int64_t step0, int64_t nsteps,
           int use_cells);

/* Total energy terms including kinetic energy from full-step velocities at step n. */
int or_energy(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* V,
              const double* u, const double* Om, const double* ext_f, const double* ext_t,
              const int* tether, int64_t step, double* energy, double* virial);

/* Observables of molecule mol: out[0] = R_z, out[1] = denatured fraction,
 * out[2] = Tw, out[3] = Tw of the ideal helix of the same length, out[4] = Lk,
 * out[5] = Wr = Lk - Tw.  Lk/Wr only when with_lk != 0. */
int or_observables(const or_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                   int mol, int with_lk, double* out);

/* Gauss linking number of two closed polygons (exact per segment pair). */
double or_linking_number(int na, const double* a, int nb, const double* b);

#ifdef __cplusplus
}
#endif
#endif
