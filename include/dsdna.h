/*
 * dsdna.h -- C ABI of the GB300 (sm_103a) engine for the single-nucleotide
 * double-stranded DNA model of Fosado, Michieletto, Allan, Brackley, Henrich
 * and Marenduzzo, "A single nucleotide resolution model for large-scale
 * simulations of double stranded DNA" (arXiv:1608.03722).
 *
 * What the engine computes (paper references are to that article):
 *   - Each nucleotide is a rigid body: a backbone bead with excluded volume
 *     and a base patch a distance ell = 0.5 from it (Sec. 2, Fig. 1a).
 *   - Interactions (App. A, Eqs. 9-15, Table 1): FENE + WCA backbone bond
 *     between consecutive beads of a strand, breakable harmonic hydrogen bond
 *     between paired patches, typed WCA excluded volume between beads (steric
 *     beads every third nucleotide, ghosts interacting only with the other
 *     strand at sigma = 0.5 and steric beads see each other at sigma = 1
 *     on either strand, Sec. 2 / Fig. 1d), dihedral A-E-F-B, Morse
 *     stacking between consecutive patches, planarity angle E-F-B and
 *     Kratky-Porod bending of three consecutive patches.
 *   - Langevin dynamics (App. A Eq. 8) with the velocity-Verlet step of
 *     App. A Eq. 16, applied per site and summed over the rigid body.
 *   - Loads of the single-molecule experiments (Sec. 4.1, 4.2): base pair 0
 *     anchored, a force and a torque on the last base pair.
 *   - Observables: extension R_z (Sec. 4.1), twist from base-pair frames
 *     (Sec. 3.2, App. B), linking number by the Gauss integral of the closed
 *     strands (App. C Eq. 17), denatured fraction (Sec. 5).
 *   - Denaturation (Sec. 5): per-pair hydrogen-bond stiffness (A.T / G.C) and
 *     the bubble rule that drops dihedral and bending terms inside runs of
 *     more than two open base pairs (dsdna_params.bubble_rule, K2_gc).
 *   - Circular molecules (Sec. 6, Fig. 10): each strand closed on itself, so
 *     the linking number is fixed by the initial state (dsdna_system.circular).
 *   - Many independent molecules in one context (batched engine), stepped by
 *     one persistent kernel per CUDA-graph chunk of steps.
 *
 * Layout of host arrays: AoS, X[3*g + c], with nucleotide slot
 * g = 2*(bp_offset(mol) + k) + s; s = 0 is strand A nucleotide k, s = 1 its
 * partner on strand B.  Strand A runs 5'->3' with increasing k, strand B with
 * decreasing k.  X is the centre of mass of the nucleotide (midpoint of bead
 * and patch), u the unit vector from bead to patch; V and Om are the
 * half-step (leapfrog) centre and angular velocities, Om normal to u.
 * Positions must be unwrapped along each strand (no jump of a box length
 * between consecutive nucleotides), also in a periodic box.
 *
 * Units are the paper's simulation units (Table 2): sigma = 1 nm,
 * epsilon = kT, tau_Br.
 *
 * Ownership: the context owns every device buffer it allocates through the
 * caller's allocator (or cudaMalloc when none is given) and frees them in
 * dsdna_destroy.  Host arrays passed in or out belong to the caller and are
 * only accessed during the call.  A context is bound to the CUDA device that
 * was current at dsdna_create and to one stream; it is not thread-safe.
 *
 * Errors: every call returns DSDNA_OK (0) or a negative dsdna_status.  Work
 * on the device is asynchronous: a device-side error (broken FENE bond,
 * non-finite force, list overflow, barrier timeout) is reported by the next
 * call that synchronises (dsdna_synchronize, get_state, energy_virial,
 * observables, compute_forces).  After any error the context is poisoned:
 * every call except get_state, set_state, last_error and destroy returns
 * DSDNA_ESTATE until dsdna_set_state installs a new state.  get_state on a
 * poisoned context returns the state at the step that raised the error.
 * The device never traps.
 */
#ifndef DSDNA_H
#define DSDNA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DSDNA_NTERMS 10
/* energy[] slots of dsdna_energy_virial */
enum {
  DSDNA_E_FENE = 0,  /* App. A Eq. 9 */
  DSDNA_E_BONDWCA,   /* Table 1 backbone WCA (sigma = 0.443) */
  DSDNA_E_HBOND,     /* App. A Eq. 10 */
  DSDNA_E_WCA,       /* App. A Eq. 11, typed per Sec. 2 */
  DSDNA_E_DIHEDRAL,  /* App. A Eq. 12 */
  DSDNA_E_MORSE,     /* App. A Eq. 13 */
  DSDNA_E_PLANAR,    /* App. A Eq. 14 */
  DSDNA_E_BEND,      /* App. A Eq. 15 */
  DSDNA_E_KIN_T,     /* translational kinetic energy, full-step velocity */
  DSDNA_E_KIN_R      /* rotational kinetic energy, full-step velocity */
};

typedef enum dsdna_status {
  DSDNA_OK = 0,
  DSDNA_EINVAL = -1,    /* bad argument */
  DSDNA_ENOMEM = -2,    /* allocation failed */
  DSDNA_ECUDA = -3,     /* CUDA runtime error */
  DSDNA_EFENE = -4,     /* a backbone bond reached R0 (App. A Eq. 9: U = infinity) */
  DSDNA_ENAN = -5,      /* non-finite force or velocity */
  DSDNA_EOVERFLOW = -6, /* neighbour list capacity or image range exceeded */
  DSDNA_ETIMEOUT = -7,  /* bounded device barrier gave up */
  DSDNA_ESTATE = -8     /* context poisoned by an earlier error */
} dsdna_status;

enum { DSDNA_PREC_MIXED = 0, DSDNA_PREC_FP64 = 1 };
enum { DSDNA_NOISE_OFF = 0, DSDNA_NOISE_UNIFORM = 1, DSDNA_NOISE_GAUSSIAN = 2 };

/* Model, integrator and engine parameters.  dsdna_default_params fills the
 * values of Table 1 (force field), Sec. 2 (geometry), App. A (kT = 1,
 * gamma = 1, dt = 0.005 tau_Br, Eq. 16). */
/* rebuild_mode 0 rebuilds inside the step kernel up to this many nucleotides */
#define DSDNA_FUSED_REBUILD_MAX_NT 262144
/* Chain-window list build: radius (nm) of the widest 16-slot segment (8 base
 * pairs; about 1.3 nm in the relaxed helix) that enters the segment grid whole. */
#define DSDNA_SEG_RCAP 1.8

typedef struct dsdna_params {
  double K1, R0, eps_bb, sigma_bb;       /* FENE + backbone WCA */
  double K2, r0_hb, rc_hb;               /* hydrogen bond */
  double eps_ev, sigma_ss, sigma_cross;  /* steric WCA: two steric beads / a pair across strands with a ghost */
  double K3, d_dih;                      /* dihedral, d in radians (-144 deg) */
  double K4, lambda_m, r0_m;             /* Morse stacking */
  double K5, alpha0;                     /* planarity (K5/2)(alpha - alpha0)^2, alpha0 in radians */
  double K6;                             /* Kratky-Porod bending */
  double mass;                           /* mass of each site (bead and patch) */
  double ell;                            /* bead-patch distance */
  double kT, gamma, dt;                  /* Langevin temperature, friction per site, time step */
  uint64_t seed;                         /* Philox key */
  int noise;                             /* DSDNA_NOISE_* */
  int steric_phase;                      /* steric iff (index along strand from its 5' end) % 3 == phase (0, 1 or 2) */
  double box[3];                         /* > 0: periodic edge in that direction; <= 0: open */
  double skin;                           /* neighbour-list skin, at most 1 nm (0: default 0.3) */
  int precision;                         /* DSDNA_PREC_MIXED (FP32 forces, FP64 X/V) or DSDNA_PREC_FP64 */
  int max_neighbors;                     /* neighbour capacity per bead (0: default 32; at most 32) */
  int block_threads;                     /* threads per CTA of the step kernel, a multiple of 32 in 64..1024
                                            (FP64 path 64..256); 0: 1024 in mixed precision when the system has
                                            at least 32 tiles of 32 nucleotides per SM, else 256 */
  int blocks_per_sm;                     /* persistent CTAs per SM (0: as many as fit) */
  int steps_per_graph;                   /* steps per captured CUDA graph launch (0: default 50) */
  /* Sec. 5 denaturation.  A base pair is open when its hydrogen bond is
   * broken (patch distance > rc_hb).  With the bubble rule the dihedral of a
   * strand step is left out when both of its base pairs lie in a run of at
   * least three consecutive open base pairs, and the bending angle at a
   * nucleotide when the base pairs of it and of its two strand neighbours are
   * all open.  bubble_rule = 1: only while that holds (the terms return when
   * the bubble closes; a returning dihedral can carry tens of kT, which makes
   * runs at low K2 unstable); 2: for good, recorded in a per-nucleotide mask
   * (dsdna_get_bubble_mask) that each step extends.  K2_gc is the
   * hydrogen-bond stiffness of base pairs flagged G.C in dsdna_system.gc
   * (<= 0: K2 for every pair). */
  int bubble_rule;                       /* 0 off, 1 while in a bubble, 2 for good */
  double K2_gc;
  /* Neighbour-list rebuild: 1 separate kernels between step launches, 2
   * inside the persistent step kernel (grid barriers between its phases; one
   * launch runs a whole graph chunk of steps), 0 chooses 2 for systems of at
   * most DSDNA_FUSED_REBUILD_MAX_NT nucleotides without a Morton cell table. */
  int rebuild_mode;
  /* Sec. 2 gives sigma = 1 for steric beads and has ghosts see the other
   * strand at sigma = 0.5, without saying what two steric beads of opposite
   * strands use.  sigma_cross_steric is that sigma: 1 by default (the steric
   * size, the reading whose torsional persistence length matches Sec. 3.2);
   * <= 0 gives such pairs sigma_cross like every other cross-strand pair. */
  double sigma_cross_steric;
  /* Mixed precision, list rebuilt by separate kernels (rebuild_mode 1, or 0
   * above DSDNA_FUSED_REBUILD_MAX_NT): 1 evaluates a list pair whose two
   * nucleotides share a 32-slot tile of the step kernel once and gives the
   * other nucleotide its negative (Newton's third law); 0 evaluates every
   * list pair from both sides.  The pair force is antisymmetric bit for bit,
   * so both give the same forces and trajectories bit for bit. */
  int pair_halving;
  /* Neighbour-list build in the separate rebuild kernels and the force and
   * energy passes (the rebuild inside the step kernel, rebuild_mode 2, walks
   * cells).  0: chain-window build: every pair of beads whose 16-slot
   * segments (8 base pairs) are equal or adjacent is tested directly from
   * shared memory, and the other pairs are found through a grid of segment
   * bounding spheres (Sec. 6 lists, arranged for a chain whose list partners
   * are nearly all a few slots away); a periodic box uses it when that grid
   * has at least 3 cells per edge and its cell table is linear, an open box
   * always.  1: the cell walk (one lane per bead over its 27 neighbour
   * cells).  Both give the same pairs (up to pairs within FP32 rounding of
   * the list radius, which lie beyond every cutoff) in the same order. */
  int list_build;
} dsdna_params;

/* Molecules and (optional) initial state.  NULL X/u builds ideal relaxed
 * helices along +z from the origin (Sec. 2); NULL V/Om draws Maxwell-Boltzmann
 * velocities from the Philox stream of the seed.  tether[m] != 0 anchors base
 * pair 0 of molecule m (Sec. 4.1).  circular[m] != 0 closes molecule m into a
 * ring (the supercoiled rings of Sec. 6 / Fig. 10): on each strand the last
 * nucleotide is bonded to the first with every bonded term of a strand step,
 * so the linking number of the two strands is fixed by the initial X and u
 * (required, at least 6 base pairs).  Molecules never interact with each
 * other. */
typedef struct dsdna_system {
  int n_mol;
  const int* n_bp;       /* [n_mol], each >= 1 */
  const double* X;       /* [3*n_nt] or NULL */
  const double* V;       /* [3*n_nt] or NULL */
  const double* u;       /* [3*n_nt] or NULL (with X) */
  const double* Om;      /* [3*n_nt] or NULL (with V) */
  const int* tether;     /* [n_mol] or NULL */
  const signed char* gc; /* [n_bp total] 1 = G.C pair (stiffness K2_gc), 0 = A.T (K2), or NULL: all A.T */
  const int* circular;   /* [n_mol] or NULL (all linear) */
} dsdna_system;

/* Device allocator used for every buffer of a context.  NULL: cudaMalloc/cudaFree. */
typedef struct dsdna_allocator {
  void* (*alloc)(size_t bytes, void* user);
  void (*release)(void* ptr, void* user);
  void* user;
} dsdna_allocator;

typedef struct dsdna_obs {
  double rz;        /* extension along z of the base-pair centres (Sec. 4.1) */
  double denat;     /* fraction of base pairs with broken hydrogen bond (Sec. 5) */
  double tw;        /* twist in turns, sum of (alpha + gamma) / 2 pi (Sec. 3.2, App. B);
                       N - 2 increments on a linear molecule, N on a ring */
  double tw_ideal;  /* twist of the relaxed helix of the same length: (N-2) (ring: N) x 36 deg */
  double lk;        /* linking number of the closed strands (App. C Eq. 17): a linear
                       molecule's strands closed far away (App. C), a ring's as they are */
  double wr;        /* writhe lk - tw (Sec. 4.2, Eq. 6) */
} dsdna_obs;

enum { DSDNA_OBS_EXT = 1, DSDNA_OBS_DENAT = 2, DSDNA_OBS_TW = 4, DSDNA_OBS_LK = 8 };

typedef struct dsdna_info {
  int64_t n_nt;          /* nucleotides */
  int n_mol;
  int64_t step;          /* step counter */
  int64_t rebuilds;      /* neighbour-list builds so far */
  int grid_blocks;       /* persistent CTAs */
  int block_threads;
  int max_neighbors;
  int precision;
  double skin;
  int64_t cell_table;    /* entries of the cell hash table */
  int64_t device_bytes;  /* bytes allocated on the device */
  int64_t engine_launches; /* persistent step/force/energy kernel launches so far */
  int rebuild_in_step;   /* 1: the step kernel rebuilds the list itself (rebuild_mode) */
  int64_t halved_tiles;  /* 32-slot tiles whose same-tile list pairs the last build set to be evaluated
                            once (pair_halving); 0 when pair halving is off */
  int chain_list;        /* 1: the chain-window list build runs (list_build) */
} dsdna_info;

/* Per-launch timing of dsdna_step_profiled (CUDA events on the context stream). */
typedef struct dsdna_prof {
  int64_t steps;            /* steps advanced */
  int64_t engine_launches;  /* persistent step-kernel launches */
  double engine_ms;         /* summed event time of those launches */
  int64_t rebuild_launches; /* neighbour-list rebuilds (five kernels each) */
  double rebuild_ms;        /* summed event time of the rebuilds */
} dsdna_prof;

typedef struct dsdna_ctx dsdna_ctx;

/* Fill p with the defaults described above. */
void dsdna_default_params(dsdna_params* p);

/* Create a context.  params, sys: read during the call.  alloc: may be NULL.
 * cuda_stream: cudaStream_t all work is queued on (NULL = legacy default).
 * Returns DSDNA_EINVAL for inconsistent input, DSDNA_ENOMEM, DSDNA_ECUDA. */
int dsdna_create(const dsdna_params* params, const dsdna_system* sys, const dsdna_allocator* alloc,
                 void* cuda_stream, dsdna_ctx** out);

/* Set the applied end force f (force on the last base pair, split over its
 * two nucleotides) and torque t (couple on the same pair) of molecule mol;
 * mol = -1 sets every molecule (Sec. 4.1 Fig. 5, Sec. 4.2 Fig. 7). */
int dsdna_set_external_force_torque(dsdna_ctx* ctx, int mol, const double force[3], const double torque[3]);

/* Queue nsteps Langevin steps (App. A Eq. 8, Eq. 16) on the context's stream;
 * returns without waiting.  Neighbour lists are rebuilt on the device when a
 * bead moved more than skin/2 since the last build. */
int dsdna_step(dsdna_ctx* ctx, int64_t nsteps);

/* Wait for queued work; returns the first device-side error, if any. */
int dsdna_synchronize(dsdna_ctx* ctx);

/* Advance nsteps like dsdna_step, but queue every rebuild and step-kernel
 * launch from the host (no graph) and time each with a CUDA event pair on
 * the context stream; the sums go to *out.  Same trajectory as dsdna_step
 * (the kernels and the order of the steps are the same); slower by the host
 * round trip after every launch.  Synchronises; returns device errors. */
int dsdna_step_profiled(dsdna_ctx* ctx, int64_t nsteps, dsdna_prof* out);

/* Energy per term (DSDNA_E_*) and site virial W = sum (r_s - r_ref) (x) F_s
 * (xx yy zz xy xz yz) of molecule mol (-1: sum over all), FP64 reductions.
 * Kinetic terms use the full-step velocities of the current step. */
int dsdna_energy_virial(dsdna_ctx* ctx, int mol, double energy[DSDNA_NTERMS], double virial[6]);

/* Observables of molecule mol selected by flags (DSDNA_OBS_*), FP64
 * reductions on the device.  DSDNA_OBS_LK costs O(N^2) in the molecule length. */
int dsdna_observables(dsdna_ctx* ctx, int mol, unsigned flags, dsdna_obs* out);

/* Per-molecule profiles behind dsdna_observables, for the persistence-length
 * and torsional-persistence correlators of Sec. 3.1-3.2: centre[3*N] the
 * base-pair centres (midpoint of the two patches, the centreline whose
 * tangents Sec. 3.1 correlates), twist[N-2] (a ring: [N]) the twist
 * increment of each pair of consecutive base-pair-step frames in turns
 * (App. B, alpha + gamma / 2 pi).  Caller-owned host arrays, either may be
 * NULL.  Synchronises. */
int dsdna_profiles(dsdna_ctx* ctx, int mol, double* centre, double* twist);

/* Copy the state of molecule mol (-1: all) to caller-owned host arrays
 * [3*n] each (any may be NULL).  Synchronises.  Also allowed on a poisoned
 * context (post-mortem: the state at the step that raised the error). */
int dsdna_get_state(dsdna_ctx* ctx, int mol, double* X, double* V, double* u, double* Om);

/* Install a new state for molecule mol (-1: all) from host arrays (NULL
 * leaves that field unchanged); clears a poisoned context and forces a
 * neighbour-list rebuild. */
int dsdna_set_state(dsdna_ctx* ctx, int mol, const double* X, const double* V, const double* u, const double* Om);

/* Bubble rule 2 mask of molecule mol (-1: all), one byte per nucleotide slot:
 * bit 0 = dihedral of the step to the next nucleotide removed, bit 1 =
 * bending centred on the nucleotide removed (Sec. 5).  get synchronises and
 * copies to a caller-owned host array; set installs one (entries 0..3; NULL
 * clears), e.g. with the state of a checkpoint. */
int dsdna_get_bubble_mask(dsdna_ctx* ctx, int mol, unsigned char* mask);
int dsdna_set_bubble_mask(dsdna_ctx* ctx, int mol, const unsigned char* mask);

/* Conservative site forces (bead, patch) on every nucleotide at the current
 * state, including the applied loads, as FP64 host arrays [3*n_nt] each. */
int dsdna_compute_forces(dsdna_ctx* ctx, double* F_bead, double* F_patch);

/* Build the neighbour list at the current state and return its pairs
 * (i < j, global slots) within r_cut(type) + skin: writes min(count, cap)
 * pairs to pi/pj and the total to *count. */
int dsdna_neighbor_pairs(dsdna_ctx* ctx, int64_t cap, int64_t* pi, int64_t* pj, int64_t* count);

int dsdna_get_info(const dsdna_ctx* ctx, dsdna_info* info);

/* Step counter (number of steps queued so far). */
int64_t dsdna_step_counter(const dsdna_ctx* ctx);

/* Text of the last error of ctx (or of the last failed create when ctx is NULL). */
const char* dsdna_last_error(const dsdna_ctx* ctx);

/* Release every device buffer and the context. */
void dsdna_destroy(dsdna_ctx* ctx);

/* Autotuner for the engine's launch and list parameters (no counterpart in
 * the paper, which ran LAMMPS with hand-set neighbour settings, Sec. 6).
 * Runs trial_steps warm-up steps and trial_steps timed steps of the system
 * sys on temporary contexts for every candidate neighbour skin
 * (0.2, 0.25, 0.3, 0.35, 0.4, 0.5, 0.6 nm), CTA size (128, 256, 1024) and persistent CTAs per SM (and, with
 * rebuild_mode 0 and between a quarter and four times
 * DSDNA_FUSED_REBUILD_MAX_NT nucleotides, both rebuild paths), then the
 * fastest of these with the other list_build, and writes
 * to *best the copy of *base with the fastest choice (ns per
 * nucleotide-step in *best_ns, may be NULL).  The candidates change how
 * often the list is rebuilt and how work is spread, never the computed
 * forces.  Allocates and frees through alloc like dsdna_create; synchronises
 * cuda_stream.  Returns DSDNA_OK, DSDNA_EINVAL or DSDNA_ECUDA. */
int dsdna_autotune(const dsdna_params* base, const dsdna_system* sys, const dsdna_allocator* alloc, void* cuda_stream,
                   int trial_steps, dsdna_params* best, double* best_ns);

/* Force pass that allocates nothing.  The paper has no counterpart: this call
 * exists for callers that cannot call cudaMalloc, such as processes whose
 * device memory is wholly owned by another pool allocator, or tight loops
 * that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 *
 * It computes the same conservative site forces as dsdna_compute_forces
 * (mixed precision, no applied loads, nothing anchored) for the molecules
 * n_bp[0..n_mol-1] at centres X and orientations u, without a context.
 * X, u (inputs) and F_bead, F_patch (outputs) are caller-owned DEVICE arrays
 * of 3*n_nt doubles in the AoS slot layout described above; n_bp is a host
 * array.  Work runs on cuda_stream and the call waits for it.
 *
 * Limits: at most DSDNA_NOALLOC_MAX_NT nucleotides and DSDNA_NOALLOC_MAX_MOL
 * molecules; a periodic box may span at most 32 cells of edge
 * 2^(1/6) max(sigma) + skin per direction; precision must be
 * DSDNA_PREC_MIXED.  Larger inputs return DSDNA_EINVAL, and so do the
 * parameters dsdna_create rejects (skin outside [0, 1] nm, bubble_rule or
 * steric_phase out of range, non-positive ell, R0 or rc_hb, negative K2_gc);
 * skin 0 means the default 0.3 nm, as in dsdna_create.
 *
 * Scratch memory: one fixed device array of about 5 MB (cell table,
 * neighbour list, position mirrors), reserved on every GPU that loads the
 * library until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the device current.  No
 * call can be captured into a CUDA graph: each copies the molecule table
 * from host memory and waits for its stream.  Every call reuses the same
 * array and starts by clearing what must begin at zero; calls that overlap on
 * the GPU (other streams, other host threads) race on it and must be
 * serialised by the caller.  Returns DSDNA_OK or a negative dsdna_status
 * (EFENE for a broken backbone bond, EOVERFLOW for more than 32 neighbours). */
#define DSDNA_NOALLOC_MAX_NT 16384
#define DSDNA_NOALLOC_MAX_MOL 256
int dsdna_forces_noalloc(const dsdna_params* params, int n_mol, const int* n_bp, const double* X, const double* u,
                         double* F_bead, double* F_patch, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Surrogate of the force/torque sweeps: an MLP 4 -> 64 -> 64 -> 3 with GELU
 * activations (the paper has no surrogate; Sec. 4 runs one simulation per
 * load).  Inputs per row: (force along z [kT/nm], end torque about z [kT],
 * length [bp], kT); outputs: (mean extension / contour length, excess twist
 * (Tw - Tw0)/Tw0, denatured-bp fraction).  Weights are FP32 masters with
 * BF16 copies; every contraction runs on the tensor cores with BF16 operands
 * and FP32 accumulation.  Parameters are packed FP32, row-major:
 * W1[64][4] b1[64] W2[64][64] b2[64] W3[3][64] b3[3] (dsdna_mlp_num_params
 * values).  Inputs are normalised inside the kernels with in_mean / in_scale
 * and outputs produced as out_mean + out_scale * (network output).
 * X, Y, T are DEVICE arrays of float ([B][4], [B][3], [B][3]); work runs on
 * the network's stream. */
typedef struct dsdna_mlp dsdna_mlp;

/* Network for batches of up to max_batch rows; parameters start at zero. */
int dsdna_mlp_create(int max_batch, const dsdna_allocator* alloc, void* cuda_stream, dsdna_mlp** out);
int dsdna_mlp_num_params(void);
/* Host arrays; any may be NULL (unchanged).  New parameters reset Adam. */
int dsdna_mlp_set_params(dsdna_mlp* net, const float* params, const float* in_mean, const float* in_scale,
                         const float* out_mean, const float* out_scale);
/* Host copies of the FP32 parameters and of the last gradients (either may be NULL). */
int dsdna_mlp_get_params(dsdna_mlp* net, float* params, float* grads);
/* Y = network(X) for B rows; keeps the activations for dsdna_mlp_backward. */
int dsdna_mlp_forward(dsdna_mlp* net, const float* X, int B, float* Y);
/* Gradients of the mean squared error over the B x 3 normalised outputs of
 * the last forward pass against targets T; writes the loss to *loss_host
 * (may be NULL, then the call does not wait). */
int dsdna_mlp_backward(dsdna_mlp* net, const float* T, int B, float* loss_host);
/* One Adam step (bias-corrected, Kingma & Ba) on the FP32 masters with
 * decoupled weight decay on the three weight matrices (Loshchilov & Hutter):
 * p <- p - lr (m_hat / (sqrt(v_hat) + eps) + weight_decay p); biases are not
 * decayed.  Refreshes the BF16 copies.  weight_decay < 0: DSDNA_EINVAL. */
int dsdna_mlp_adam_step(dsdna_mlp* net, float lr, float beta1, float beta2, float eps, float weight_decay);
void dsdna_mlp_destroy(dsdna_mlp* net);

#ifdef __cplusplus
}
#endif
#endif /* DSDNA_H */
