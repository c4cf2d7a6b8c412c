// engine.cuh -- device side of the dsDNA engine (sm_103a).
//
// One persistent cooperative kernel advances the single-nucleotide dsDNA
// model of Fosado et al. (arXiv:1608.03722): per step every warp walks its
// strip of the chain, evaluates every interaction of App. A (Eqs. 9-15,
// Table 1) on tiles staged in shared memory, adds the typed WCA pairs of a
// full neighbour list, applies the loads of Sec. 4, and integrates App. A
// Eq. 8 with the step of Eq. 16; a bounded grid barrier separates the steps.
// It stops when a bead moved more than skin/2; five ordinary kernels then
// rebuild the cell and neighbour lists before the next launch.
//
// Precision (Real = float, "mixed"): the FP64 centre positions X and
// velocities V are the integrator's accumulators; forces, orientation u and
// angular velocity are FP32.  Displacements between nucleotides come from a
// fixed-point mirror of X: the low 32 bits of round(X S) per axis.  In a
// periodic box 2^32 grid units span L / k (k = max(1, floor(L / 8 nm))), so
// the mirror is the same for every periodic image of a position and the
// wrap-around difference of two mirrors is their minimum-image separation
// (below L / 2k, at least 4 nm), with no image bookkeeping; in an open box
// S = 2^29 / nm (separations below 4 nm).  The grid unit stays at or below
// 3.7e-9 nm.
// Real = double runs every step in FP64.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dsdna {

// ---------------------------------------------------------------- constants
// Topology flags of a slot (bits 0-7; the molecule index sits above bit 8).
// F_GC: G.C base pair (Sec. 5).  F_JUNC: base pair 0, 1, N-2 or N-1 of a
// circular molecule, whose neighbourhood crosses the junction.  Bit 6 is
// used by the step kernel's shared copy of the flags only.
enum : int { F_STERIC = 1, F_PREV = 2, F_NEXT = 4, F_FROZEN = 8, F_TOP = 16, F_GC = 32, F_JUNC = 128 };
// Bits 8-9: terms removed by bubble rule 2 (bit 8 the dihedral of the step to
// the next nucleotide, bit 9 the bending centred on the slot), set by the step
// kernel.  The molecule index starts at bit MOL_SHIFT.
constexpr int RM_SHIFT = 8;
constexpr int MOL_SHIFT = 10;
// Cell table: periodic box with >= 3 cells per edge -> linear index (x fastest;
// the three x-neighbours of a cell are consecutive entries); smaller periodic
// box -> Morton index; open box -> hash of (molecule, cell).
enum : int { TABLE_HASH = 0, TABLE_MORTON = 1, TABLE_LINEAR = 2 };
enum : unsigned {
  B_STALE = 1u, B_EFENE = 2u, B_ENAN = 4u, B_EOVF = 8u, B_ETIMEOUT = 16u, B_EIMG = 32u
};
constexpr unsigned B_ERRMASK = B_EFENE | B_ENAN | B_EOVF | B_ETIMEOUT | B_EIMG;
enum : int { MODE_STEP = 0, MODE_FORCES = 1, MODE_ENERGY = 2 };
constexpr int MODE_EXT = 4;   // launch flag: kernel instance with circular molecules / bubble rule
constexpr int MODE_FUSED = 8; // launch flag (MODE_STEP): instance that rebuilds the list in the kernel
constexpr int NTERMS = 10;
constexpr int EOUT_STRIDE = 16;           // energy terms + 6 virial
constexpr int NBR_J_BITS = 27;   // slot field of a cell-sorted bead word (bit 27: steric flag)
constexpr int EVL_CAP = 96;      // evaluated pairs per tile under pair halving (else the tile's whole list)
constexpr int HALF_NMAX = 8;     // longest list a tile under pair halving may hold

// Neighbour-list entry: partner slot j in the low ENT_J_BITS bits, then the
// minimum-image shift s + 1 in {0, 1, 2} of each axis in a 2-bit field
// (x at bit 26, y at 28, z at 30).  No entry has all bits set (a field never
// holds 3), so -1 marks "no entry".
constexpr int ENT_J_BITS = 26;
constexpr int ENT_JMASK = (1 << ENT_J_BITS) - 1;
__host__ __device__ __forceinline__ int ent_make(int j, int sx, int sy, int sz) {
  return (int)((unsigned)j | ((unsigned)(sx + 1) << 26) | ((unsigned)(sy + 1) << 28) | ((unsigned)(sz + 1) << 30));
}
__host__ __device__ __forceinline__ int ent_shift(int e, int c) { return (int)(((unsigned)e >> (26 + 2 * c)) & 3u) - 1; }

struct GridBar {
  unsigned count;
  unsigned gen;
  unsigned acc[3];
  unsigned pad[3];
};

template <class Real>
struct Coef {
  Real K1, R02, eps_bb, sbb2, rcbb2;
  Real khb, r0hb, rchb2;
  Real eps, sss2, rcss2, scr2, rccr2;
  Real scs2, rccs2;  // steric pair across strands under the other reading of Sec. 2 (0: off)
  Real K3, cosd, sind;
  Real K4, lam, r0m;
  Real K5, alpha0;
  Real K6;
  Real h;            // ell / 2
  Real dtM, dtI;     // dt / M, dt / I
  Real dt;
  Real gam2, gamr;   // 2 gamma, gamma ell^2 / 2
  Real noise_c;      // uniform: sqrt(24 gamma kT/dt) 2^-21; gaussian: sqrt(2 gamma kT/dt)
  Real halfdtM, halfdtI;
  Real M, I;
  float skin_half2;  // (skin/2)^2
  float rl_ss2, rl_cr2, rl_cs2, rl_max2;
  Real khb_gc;       // hydrogen-bond coefficient of G.C pairs (Sec. 5)
  double dt_d;       // FP64 step for the position accumulation
  double noise_cd;   // FP64 copy of noise_c
};

template <class Real>
struct KArgs {
  Coef<Real> c;
  int64_t n;
  int64_t ns;      // row stride of the [component][slot] arrays: n rounded up to a multiple of 32
  int n_mol;
  int bubble;      // no dihedral / bending inside runs of > 2 open base pairs (Sec. 5): 0 off, 1 while, 2 for good
  int64_t nseg;
  int cap;
  int64_t nsteps;
  int noise_mode;
  uint32_t pkey[20];   // Philox round keys: (seed_lo + r W0, seed_hi + r W1) for rounds r = 0 .. 9
  unsigned long long spin_budget;
  // state
  // [k][n] below means k rows of ns entries (slots n .. ns-1 are padding)
  double* X;       // mixed: [3][n]; fp64: [2][3][n]
  double* V;       // [3][n]
  Real* Om;        // [3][n]
  int4* Kw;        // mixed: [2][n] fixed-point mirror (w = packed image)
  float4* U;       // mixed: [2][n] orientation (w unused)
  double* ud;      // fp64: [2][3][n] orientation
  int* topo;       // [n] flags | removed << RM_SHIFT | mol << MOL_SHIFT
  int* img;        // [n] packed image (both modes)
  int* kref;       // [3][n] mirror at the last build
  int* nbr;        // [cap][n] list entries (ent_make)
  int* ncnt;       // [n]
  // pair halving (mixed precision; null: off): per 32-slot tile the pairs it
  // evaluates, and for each list entry where its force is found
  int* evl;        // [nseg][EVL_CAP] partner slot | owner lane << 26
  uint2* psrc;     // [n] byte q (q < 8): the evaluated pair holding list entry q's force; bit 7: negated
  int* tcnt;       // [nseg] evaluated pairs of the tile, or -1: the tile evaluates its list as it stands
  // circular molecules: junction owners (8 per ring)
  int64_t n_junc;
  const int64_t* jslot;  // [n_junc] slot of each junction owner
  const int* jidx;       // [n] junction entry of a F_JUNC slot
  Real* jout;            // [n_junc][16] their forces: sb, sp, nb, np, pp
  // cell hash
  unsigned* cnt;   // [H]
  unsigned* start; // [H + 1]
  unsigned H;
  int table;       // TABLE_LINEAR, TABLE_MORTON or TABLE_HASH (cell_key)
  int morton_bits; // TABLE_MORTON: bits per axis
  int* key;        // [n]
  float4* cent;    // [n] cell-sorted (position, slot)
  float4* wpos;    // [n] wrapped bead position, w = molecule
  unsigned* bsum;  // [grid]
  // chain-window list build (null segc: the cell-walk build).  The cell
  // table above then holds a grid of 16-slot segments (linear in a periodic
  // box, hashed in an open one), cent their bounding spheres and key their
  // slot ranges.
  float4* segc;      // [nseg16] each segment's bounding sphere: wrapped centre, radius (< 0: wide)
  int64_t nseg16;
  int sg_nc[3];      // cells per edge of the segment grid
  float sg_invh[3];  // cells per nm
  unsigned sg_H;     // entries of the segment table scan (whole scan tiles, more than its cells)
  unsigned sg_mask;  // open box: the table is hashed into sg_mask + 1 entries
  float sg_rcap;     // widest segment kept whole in the grid
  float sg_reach;    // largest list radius plus a margin (sphere test)
  int periodic;
  int nc[3];
  float cellh[3];
  float invcellh[3];
  float Lf[3];
  float invLf[3];
  double L[3];
  double fixS[3];   // fixed-point mirror: grid units per nm (2^32 m / L periodic, 2^29 open)
  float fixSf[3];   // the same in FP32
  float fixq[3];    // nm per grid unit
  // molecules
  const int64_t* mol_off;  // [n_mol + 1] base-pair offsets
  const double* ext;       // [n_mol][8]: f xyz, torque xyz
  // control
  GridBar* bar;
  unsigned* err;
  int64_t* step;
  int* rebuild;
  unsigned long long* nrebuild;
  // outputs
  double* fout;    // MODE_FORCES: [n][6]
  double* eout;    // MODE_ENERGY: [n_mol][16]
  // step loop in a CUDA graph (conditional WHILE/IF nodes)
  int64_t* steps_left;              // steps still to run in this graph launch (null: run nsteps)
  int use_cond;
  cudaGraphConditionalHandle h_while;
};

// Philox4x32-10 round keys of a 64-bit seed (Weyl sequence of the key).
template <class Real>
inline void philox_key_schedule(KArgs<Real>& a, uint64_t seed) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    a.pkey[2 * r] = k0;
    a.pkey[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Mirror grid of axis k (a.periodic and a.L set): 2^32 units per L / m with
// m = max(1, floor(L / 8 nm)) in a periodic box, so that 32-bit wrap-around
// differences are minimum-image separations, or 2^29 units per nm in an
// open box.
template <class Real>
inline void mirror_scale(KArgs<Real>& a, int k) {
  const double m = a.periodic ? (a.L[k] >= 16.0 ? (double)(int64_t)(a.L[k] / 8.0) : 1.0) : 1.0;
  const double S = a.periodic ? 4294967296.0 * m / a.L[k] : 536870912.0;
  a.fixS[k] = S;
  a.fixSf[k] = (float)S;
  a.fixq[k] = (float)(1.0 / S);
}

// ---------------------------------------------------------------- small vectors
template <class R>
struct V3 {
  R x, y, z;
};
template <class R> __device__ __forceinline__ V3<R> mk(R x, R y, R z) { return V3<R>{x, y, z}; }
template <class R> __device__ __forceinline__ V3<R> operator+(V3<R> a, V3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class R> __device__ __forceinline__ V3<R> operator-(V3<R> a, V3<R> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class R> __device__ __forceinline__ V3<R> operator-(V3<R> a) { return {-a.x, -a.y, -a.z}; }
template <class R> __device__ __forceinline__ V3<R> operator*(R s, V3<R> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class R> __device__ __forceinline__ void operator+=(V3<R>& a, V3<R> b) { a.x += b.x; a.y += b.y; a.z += b.z; }
template <class R> __device__ __forceinline__ void operator-=(V3<R>& a, V3<R> b) { a.x -= b.x; a.y -= b.y; a.z -= b.z; }
template <class R> __device__ __forceinline__ R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class R> __device__ __forceinline__ V3<R> cross(V3<R> a, V3<R> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float log_(float x) { return logf(x); }
__device__ __forceinline__ double log_(double x) { return log(x); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ float acos_(float x) { return acosf(x); }
__device__ __forceinline__ double acos_(double x) { return acos(x); }
__device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ void sincos_(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincos_(double a, double* s, double* c) { sincos(a, s, c); }

// ---------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon et al. (SC'11): ten rounds, multipliers
// 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85.  The
// key schedule is the same for every counter, so the host computes it once
// (philox_key_schedule) and each round reads its key pair from the kernel
// parameters.
__device__ __forceinline__ uint4 philox10(uint4 c, const uint32_t* key) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a = c.x, b = c.z;
    const uint32_t hi_a = __umulhi(0xD2511F53u, a), lo_a = 0xD2511F53u * a;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, b), lo_b = 0xCD9E8D57u * b;
    c = make_uint4(hi_b ^ c.y ^ key[2 * r], lo_b, hi_a ^ c.w ^ key[2 * r + 1], lo_a);
  }
  return c;
}

// Langevin noise of both sites of one nucleotide (App. A Eq. 8) from one
// Philox draw: counter (local nucleotide, step low, step high, mol), key =
// seed.  The four words give six 21-bit integers k -- the top 21 bits of
// x, y, z (bead) and w (patch x), then the low 11 bits of x with bits 0-9 of
// y above them (patch y) and the same of z and w (patch z) -- and uniform
// variates U = (k + 1/2) 2^-21: variance-matched uniform noise
// sqrt(24 gamma kT / dt) (U - 1/2), or Box-Muller pairs (U0, U1), (U2, U3),
// (U4, U5).  (k - 2^20 + 1/2) is exact in FP32.
template <class Real>
__device__ __forceinline__ void nucleotide_noise(const KArgs<Real>& a, uint32_t local, int64_t step, int mol,
                                                 V3<Real>& eb, V3<Real>& ep) {
  if (a.noise_mode == 0) {
    eb = V3<Real>{0, 0, 0};
    ep = eb;
    return;
  }
  const uint4 r = philox10(make_uint4(local, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)mol), a.pkey);
  const uint32_t k[6] = {r.x >> 11, r.y >> 11, r.z >> 11, r.w >> 11, (r.x & 0x7FFu) | ((r.y & 0x3FFu) << 11),
                         (r.z & 0x7FFu) | ((r.w & 0x3FFu) << 11)};
  Real e[6];
  if (a.noise_mode == 1) {
    const Real cc = sizeof(Real) == 8 ? (Real)a.c.noise_cd : a.c.noise_c;
#pragma unroll
    for (int q = 0; q < 6; ++q) e[q] = ((Real)(int)k[q] - (Real)1048575.5) * cc;
  } else {
    const Real s21 = (Real)(1.0 / 2097152.0);
    const Real cc = a.c.noise_c;
#pragma unroll
    for (int q = 0; q < 6; q += 2) {
      const Real u0 = ((Real)(int)k[q] + (Real)0.5) * s21, u1 = ((Real)(int)k[q + 1] + (Real)0.5) * s21;
      const Real rad = sqrt_((Real)-2 * log_(u0));
      Real sn, cs;
      sincos_((Real)6.283185307179586 * u1, &sn, &cs);
      e[q] = cc * rad * cs;
      e[q + 1] = cc * rad * sn;
    }
  }
  eb = V3<Real>{e[0], e[1], e[2]};
  ep = V3<Real>{e[3], e[4], e[5]};
}

// ---------------------------------------------------------------- positions
// Slot data staged in shared memory.
template <class Real> struct SPos;
template <> struct SPos<float> { int kx, ky, kz; float ux, uy, uz; };
template <> struct SPos<double> { double x, y, z, ux, uy, uz; };

// Separation b - o of two staged slots: wrap-around difference of the mirrors
// times the grid unit q (per axis); FP64 slots subtract their positions.
__device__ __forceinline__ V3<float> rel(const SPos<float>& o, const SPos<float>& b, const float* q) {
  return V3<float>{(float)(int)((unsigned)b.kx - (unsigned)o.kx) * q[0],
                   (float)(int)((unsigned)b.ky - (unsigned)o.ky) * q[1],
                   (float)(int)((unsigned)b.kz - (unsigned)o.kz) * q[2]};
}
__device__ __forceinline__ V3<double> rel(const SPos<double>& o, const SPos<double>& b, const float* /*q*/) {
  return V3<double>{b.x - o.x, b.y - o.y, b.z - o.z};
}
template <class Real> __device__ __forceinline__ V3<Real> uvec(const SPos<Real>& s) { return V3<Real>{s.ux, s.uy, s.uz}; }

// Mirror coordinate: low 32 bits of round(x S) (ties away from zero).  One
// FP64 multiply, then the rounding by integer operations on the bits of the
// product (the FP64 pipe of GB300 runs at a small fraction of the integer
// rate); exact for any |x S| below 2^63.
__device__ __forceinline__ int fixs(double x, double S) {
  const long long b = __double_as_longlong(x * S);
  const int sh = 1075 - (int)((b >> 52) & 0x7FF);          // right shift of the 53-bit significand
  if (sh > 53) return 0;                                    // |x S| < 1/2 rounds to zero
  if (sh < -40) return 0;                                   // an integer multiple of 2^32
  const unsigned long long m = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const unsigned long long r = sh > 0 ? (m + (1ull << (sh - 1))) >> sh : m << (-sh);
  const unsigned lo = (unsigned)r;
  return b < 0 ? (int)(0u - lo) : (int)lo;
}

// FP64 -> FP32 (round to nearest even) and FP32 -> FP64 (exact) by integer
// operations on the bit patterns, for the FP32 arithmetic around the FP64
// accumulators.  Magnitudes below the smallest normal FP32 flush to zero;
// the callers' values (velocities, their increments) stay far inside the
// normal range.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  if (a < 0x3810000000000000ull) return __uint_as_float(sign);
  const unsigned long long t = a - 0x3800000000000000ull;  // rebias the exponent 1023 -> 127
  const unsigned long long r = (t + 0x0FFFFFFFull + ((t >> 29) & 1ull)) >> 29;
  return __uint_as_float((unsigned)r | sign);
}
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7FFFFFFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (a < 0x00800000u) return __longlong_as_double((long long)sign);
  return __longlong_as_double((long long)((((unsigned long long)a << 29) + 0x3800000000000000ull) | sign));
}

// bead offset -h u on the fixed-point grid (rebuild trigger only); Sf: grid units per nm
__device__ __forceinline__ int bead_off(float hu, float Sf) { return __float2int_rn(-hu * Sf); }

template <class Real>
__device__ __forceinline__ void load_slot(const KArgs<Real>& a, int cur, int64_t g, SPos<Real>& s) {
  if constexpr (sizeof(Real) == 4) {
    const unsigned i = (unsigned)cur * (unsigned)a.ns + (unsigned)g;   // below 2^27
    const int4 k = a.Kw[i];
    const float4 u = a.U[i];
    s.kx = k.x; s.ky = k.y; s.kz = k.z;
    s.ux = u.x; s.uy = u.y; s.uz = u.z;
  } else {
    const double* X = a.X + (size_t)cur * 3 * a.ns;
    const double* u = a.ud + (size_t)cur * 3 * a.ns;
    s.x = X[g]; s.y = X[a.ns + g]; s.z = X[2 * a.ns + g];
    s.ux = u[g]; s.uy = u[a.ns + g]; s.uz = u[2 * a.ns + g];
  }
}

__device__ __forceinline__ int img_comp(int packed, int c) {
  return ((int)((unsigned)packed << (22 - 10 * c))) >> 22;   // signed 10-bit field c (bits 30, 31 ignored)
}
constexpr int IMG_STERIC_SHIFT = 30;   // steric flag of the bead in its image word

// ---------------------------------------------------------------- interaction terms
// Each returns the force on the second site (first gets the opposite) or the
// forces on all sites, and the energy when E != nullptr.

// App. A Eq. 9 + Table 1 backbone WCA: d = b_next - b_this.
template <class Real>
__device__ __forceinline__ V3<Real> t_fene(const Coef<Real>& c, V3<Real> d, unsigned& fl, Real* E) {
  Real r2 = dot(d, d);
  if (r2 >= c.R02) { fl |= B_EFENE; r2 = (Real)0.98 * c.R02; }
  const Real q = (Real)1 - r2 / c.R02;
  Real fr = -c.K1 / q;
  Real e = (Real)0, ew = (Real)0;
  if (E) e = (Real)-0.5 * c.K1 * c.R02 * log_(q);
  if (r2 < c.rcbb2) {
    const Real s2 = c.sbb2 / r2, s6 = s2 * s2 * s2;
    fr += (Real)24 * c.eps_bb * s6 * ((Real)2 * s6 - (Real)1) / r2;
    if (E) ew = (Real)4 * c.eps_bb * (s6 * s6 - s6 + (Real)0.25);
  }
  if (E) { E[0] += e; E[1] += ew; }
  return fr * d;
}

// App. A Eq. 13: d = p_next - p_this.
template <class Real>
__device__ __forceinline__ V3<Real> t_morse(const Coef<Real>& c, V3<Real> d, Real* E) {
  const Real r = sqrt_(dot(d, d));
  const Real x = exp_(-c.lam * (r - c.r0m));
  if (E) E[5] += c.K4 * ((Real)1 - x) * ((Real)1 - x);
  // force on the second site: -dU/dr * d / r
  return ((Real)-2 * c.K4 * c.lam * x * ((Real)1 - x) / r) * d;
}

// App. A Eq. 12 on A-E-F-B (positions relative to anything).  phi with the
// IUPAC sign; forces written with p = b1.b2/|b2|^2, q = b3.b2/|b2|^2.
template <class Real>
__device__ __forceinline__ void t_dihedral(const Coef<Real>& c, V3<Real> A, V3<Real> Ep, V3<Real> Fp, V3<Real> B,
                                           V3<Real>& fA, V3<Real>& fE, V3<Real>& fF, V3<Real>& fB, Real* E) {
  const V3<Real> b1 = Ep - A, b2 = Fp - Ep, b3 = B - Fp;
  const V3<Real> n1 = cross(b1, b2), n2 = cross(b2, b3);
  const Real n1s = dot(n1, n1), n2s = dot(n2, n2), b2s = dot(b2, b2);
  const Real lb2 = sqrt_(b2s);
  const Real y = lb2 * dot(b1, n2), x = dot(n1, n2);
  // sin(phi - d) and cos(phi - d) from (x, y) without the angle itself
  const Real inv = rsqrt_(x * x + y * y);
  const Real cp = x * inv, sp = y * inv;
  const Real s_pd = sp * c.cosd - cp * c.sind;   // sin(phi - d)
  if (E) E[4] += c.K3 * ((Real)1 + (cp * c.cosd + sp * c.sind));
  const Real dU = -c.K3 * s_pd;                  // dU/dphi
  fA = (dU * lb2 / n1s) * n1;                    // -dU * (-|b2|/|n1|^2 n1)
  fB = (-dU * lb2 / n2s) * n2;                   // -dU * (|b2|/|n2|^2 n2)
  const Real p = dot(b1, b2) / b2s, q = dot(b3, b2) / b2s;
  fE = ((Real)-1 - p) * fA + q * fB;
  fF = p * fA - ((Real)1 + q) * fB;
}

// App. A Eq. 14: angle at vertex V between ends P (= E, patch i) and Q (= B, bead i+1).
template <class Real>
__device__ __forceinline__ void t_planar(const Coef<Real>& c, V3<Real> v1, V3<Real> v2, V3<Real>& f1, V3<Real>& f2,
                                         Real* E) {
  const Real i1 = rsqrt_(dot(v1, v1)), i2 = rsqrt_(dot(v2, v2));
  const V3<Real> e1 = i1 * v1, e2 = i2 * v2;
  Real cs = dot(e1, e2);
  cs = cs > (Real)1 ? (Real)1 : (cs < (Real)-1 ? (Real)-1 : cs);
  const Real al = acos_(cs);
  Real sn = sqrt_((Real)1 - cs * cs);
  if (sn < (Real)1e-6) sn = (Real)1e-6;
  if (E) E[6] += (Real)0.5 * c.K5 * (al - c.alpha0) * (al - c.alpha0);
  const Real k = c.K5 * (al - c.alpha0) / sn;    // dU/dalpha / sin(alpha)
  f1 = (k * i1) * (e2 - cs * e1);
  f2 = (k * i2) * (e1 - cs * e2);
}

// App. A Eq. 15 at vertex patch i between patches i-1 (v1) and i+1 (v2).
template <class Real>
__device__ __forceinline__ void t_bend(const Coef<Real>& c, V3<Real> v1, V3<Real> v2, V3<Real>& f1, V3<Real>& f2,
                                       Real* E) {
  const Real i1 = rsqrt_(dot(v1, v1)), i2 = rsqrt_(dot(v2, v2));
  const V3<Real> e1 = i1 * v1, e2 = i2 * v2;
  const Real cs = dot(e1, e2);
  if (E) E[7] += c.K6 * ((Real)1 + cs);
  f1 = (-c.K6 * i1) * (e2 - cs * e1);
  f2 = (-c.K6 * i2) * (e1 - cs * e2);
}

// App. A Eq. 11, typed WCA; d = b_other - b_own, returns force on b_own.
template <class Real>
__device__ __forceinline__ V3<Real> t_wca(const Coef<Real>& c, V3<Real> d, Real s2sig, Real rc2, Real* e) {
  const Real r2 = dot(d, d);
  if (r2 >= rc2) { *e = (Real)0; return V3<Real>{0, 0, 0}; }
  const Real s2 = s2sig / r2, s6 = s2 * s2 * s2;
  *e = (Real)4 * c.eps * (s6 * s6 - s6 + (Real)0.25);
  return ((Real)-24 * c.eps * s6 * ((Real)2 * s6 - (Real)1) / r2) * d;
}

template <class Real>
__device__ __forceinline__ void vir_add(Real* W, V3<Real> r, V3<Real> f) {
  W[0] += r.x * f.x; W[1] += r.y * f.y; W[2] += r.z * f.z;
  W[3] += r.x * f.y; W[4] += r.x * f.z; W[5] += r.y * f.z;
}

// ---------------------------------------------------------------- grid barrier
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch that also ORs every block's flag
// word.  The wait is bounded by a clock budget; on expiry the block reports
// B_ETIMEOUT and the caller leaves the kernel.
__device__ __forceinline__ unsigned grid_sync(GridBar* bar, unsigned nblocks,
                                              unsigned local, unsigned long long budget, unsigned* s_word) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = ld_acquire(&bar->gen);
    atomicOr(&bar->acc[g % 3], local);
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    unsigned res = 0;
    if (arrived == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      atomicExch(&bar->acc[(g + 1) % 3], 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = clock64();
      unsigned ns = 32;
      while (ld_acquire(&bar->gen) == g) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        if ((unsigned long long)(clock64() - t0) > budget) { res = B_ETIMEOUT; break; }
      }
    }
    __threadfence();
    res |= ld_acquire(&bar->acc[g % 3]);   // final once gen moved on; a load, not a serialised atomic
    *s_word = res;
  }
  __syncthreads();
  return *s_word;
}

}  // namespace dsdna
