// engine_kernels.cuh -- persistent step kernel of the dsDNA engine: the fused
// force + Langevin strip pass and the step loop with its grid barrier (the
// list rebuild is in rebuild.cuh; small systems run it inside this kernel).
// Included by kern_mixed.cu (Real = float) and kern_fp64.cu (Real = double).
#pragma once
#include "engine.cuh"
#include "rebuild.cuh"

namespace dsdna {

// ---------------------------------------------------------------- shared memory
// Each warp walks a contiguous strip of slots in tiles of SEG = 32 and keeps
// the positions it staged and the owner terms it computed in rings of RING
// entries indexed by slot (mod RING), so a tile stages 32 new slots and
// computes 32 new owners; the warp synchronises with __syncwarp only.
constexpr int SEG = 32;
constexpr int RING = 64;

template <class Real>
struct SegSmem {
  SPos<Real>* pos;   // [RING] staged slots
  int* flg;          // [RING] topology words of the staged slots
  Real* cs;          // [6][RING] forces of owner terms on the owner (bead xyz, patch xyz)
  Real* cn;          // [6][RING] ... on the owner's next nucleotide
  Real* cp;          // [3][RING] ... on the owner's previous patch (bending)
  int* pst;          // [SEG] first pair index of each nucleotide of the tile (warp_pairs)
  Real* pf;          // [EVL_CAP][3] pair forces of a round of warp_pairs (64), or of a halved tile
};

template <class Real>
__host__ __device__ constexpr size_t seg_warp_bytes() {
  size_t b = sizeof(SPos<Real>) * RING + sizeof(int) * RING;
  b = (b + 15) & ~(size_t)15;
  b += sizeof(Real) * (size_t)RING * 15;
  b += sizeof(int) * 32 + sizeof(Real) * EVL_CAP * 3;
  return (b + 15) & ~(size_t)15;
}

template <class Real>
__host__ __device__ inline size_t seg_smem_bytes(int T) {
  return seg_warp_bytes<Real>() * (size_t)(T / 32) + 64;
}

template <class Real>
__device__ __forceinline__ SegSmem<Real> carve(unsigned char* raw, int /*T*/) {
  unsigned char* w = raw + seg_warp_bytes<Real>() * (threadIdx.x >> 5);
  SegSmem<Real> s;
  s.pos = reinterpret_cast<SPos<Real>*>(w);
  s.flg = reinterpret_cast<int*>(w + sizeof(SPos<Real>) * RING);
  size_t off = sizeof(SPos<Real>) * RING + sizeof(int) * RING;
  off = (off + 15) & ~(size_t)15;
  s.cs = reinterpret_cast<Real*>(w + off);
  s.cn = s.cs + (size_t)RING * 6;
  s.cp = s.cn + (size_t)RING * 6;
  s.pf = s.cp + (size_t)RING * 3;
  s.pst = reinterpret_cast<int*>(s.pf + EVL_CAP * 3);
  return s;
}

// ---------------------------------------------------------------- strip pass
__device__ __forceinline__ int ring(int64_t g) { return (int)(g & (RING - 1)); }

// Sec. 5: base pair k is open when the hydrogen bond between its patches is
// broken (distance beyond rc).  mark_open tests the pair whose strand-A slot
// g = 2k was just staged (with its partner g + 1) and sets F_OPEN on the
// ring copy of its flags; bp_open reads that bit back.  A pair outside
// molecule mol (or outside [0, n): flags 0) counts as closed.
constexpr int F_OPEN = 64;   // ring flags only, never in the topology array
template <class Real>
__device__ __forceinline__ void mark_open(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t g) {
  const int ra = ring(g), rb = ring(g + 1);
  const int fa = sm.flg[ra];
  if (fa == 0) return;
  const SPos<Real> pa = sm.pos[ra], pb = sm.pos[rb];
  const V3<Real> d = rel(pa, pb, a.fixq) + a.c.h * (uvec(pb) - uvec(pa));
  if (dot(d, d) > a.c.rchb2) sm.flg[ra] = fa | F_OPEN;
}
__device__ __forceinline__ bool bp_open(const int* flg, int64_t k, int mol) {
  const int fa = flg[ring(2 * k)];
  return (fa & F_OPEN) && (fa >> MOL_SHIFT) == mol;
}

// Forces of the terms one owner evaluates: on the owner's bead and patch
// (sb, sp), on its next nucleotide (nb, np) and on its previous patch (pp).
template <class Real>
struct OwnerOut {
  V3<Real> sb, sp, nb, np, pp;
};

// Where an owner's neighbourhood comes from.  RingSrc: the warp's shared
// ring (every owner whose base pairs o/2 - 2 .. o/2 + 2 are consecutive slots
// of its molecule).  GlobalSrc: global memory with the indices of a circular
// molecule taken modulo its length (owners next to the junction of a ring,
// and the far owners a junction nucleotide re-evaluates).
template <class Real>
struct RingSrc {
  const SPos<Real>* spos;
  const int* flg;
  __device__ __forceinline__ SPos<Real> pos(int64_t g) const { return spos[ring(g)]; }
  __device__ __forceinline__ int64_t step(int64_t g, int d) const { return g + d; }
  __device__ __forceinline__ bool open(int64_t k, int mol) const { return bp_open(flg, k, mol); }
};
template <class Real>
struct GlobalSrc {
  const KArgs<Real>& a;   // the kernel's __grid_constant__ parameters
  int cur;
  int64_t off, N;   // base-pair offset and length of the owner's molecule
  __device__ __forceinline__ int64_t wrap(int64_t k) const {
    int64_t r = (k - off) % N;
    return off + (r < 0 ? r + N : r);
  }
  __device__ __forceinline__ SPos<Real> pos(int64_t g) const {
    SPos<Real> s;
    load_slot(a, cur, g, s);
    return s;
  }
  __device__ __forceinline__ int64_t step(int64_t g, int d) const { return 2 * wrap((g >> 1) + d / 2) + (g & 1); }
  __device__ __forceinline__ bool open(int64_t k, int /*mol*/) const {
    k = wrap(k);
    const SPos<Real> pa = pos(2 * k), pb = pos(2 * k + 1);
    const V3<Real> d = rel(pa, pb, a.fixq) + a.c.h * (uvec(pb) - uvec(pa));
    return dot(d, d) > a.c.rchb2;
  }
};

// Bonded terms owned by slot o with flags f: the step o -> next along its
// strand (FENE + WCA, Morse, dihedral, planarity) and the bending angle at o,
// each evaluated once.  Bubble rule (Sec. 5): the dihedral is left out when
// both base pairs of the step lie in a run of three or more open pairs, and
// the bending when the pairs of o and of both its strand neighbours are open;
// rule 2 also leaves out what the slot's removed bits (RM_SHIFT) mark and,
// when `persist`, adds what it left out to them.
// Terms of owner o that the bubble rule leaves out: bit 0 the dihedral, bit 1
// the bending.  Out of line: it runs only with the rule on, and the step
// kernel's common path keeps its registers.
template <class Real, class Src>
__device__ __noinline__ unsigned bubble_bits(const KArgs<Real>& a, const Src src, int64_t o, int f, bool persist) {
  const unsigned r0 = (unsigned)(f >> RM_SHIFT) & 3u;   // set by rule 2 only
  const int mol = f >> MOL_SHIFT, st = (o & 1) ? -1 : 1;
  const int64_t ko = o >> 1;
  unsigned r1 = r0;
  if (src.open(ko, mol) && src.open(ko + st, mol)) {
    const bool before = src.open(ko - st, mol);
    if (before || src.open(ko + 2 * st, mol)) r1 |= 1u;
    if ((f & F_PREV) && before) r1 |= 2u;
  }
  if (persist && r1 != r0) atomicOr(a.topo + o, (int)(r1 << RM_SHIFT));
  return r1;
}

template <class Real, bool EXT, class Src>
__device__ __forceinline__ void owner_eval(const KArgs<Real>& a, const Src& src, int64_t o, int f, bool persist,
                                           unsigned& fl, Real* E, Real* W, OwnerOut<Real>& out) {
  const int dir = (o & 1) ? -2 : 2;   // strand A (even slot) runs up, strand B down
  unsigned rm = 0u;
  if constexpr (EXT) rm = a.bubble ? bubble_bits(a, src, o, f, persist) : 0u;
  const bool skip_dih = (rm & 1u) != 0, skip_bend = (rm & 2u) != 0;
  const SPos<Real> so = src.pos(o);
  const SPos<Real> sq = src.pos(src.step(o, dir));
  const Real h = a.c.h;
  const V3<Real> uo = uvec(so), uq = uvec(sq);
  const V3<Real> Rq = rel(so, sq, a.fixq);
  const V3<Real> bo = -h * uo, po = h * uo, bq = Rq - h * uq, pq = Rq + h * uq;
  // FENE + WCA, Morse
  V3<Real> fb = t_fene(a.c, bq - bo, fl, E);
  out.nb += fb; out.sb -= fb;
  V3<Real> fm = t_morse(a.c, pq - po, E);
  out.np += fm; out.sp -= fm;
  if (W) { vir_add(W, bq - bo, fb); vir_add(W, pq - po, fm); }
  // dihedral A-E-F-B = bead o, patch o, patch q, bead q
  if (!skip_dih) {
    V3<Real> fA, fE, fF, fB;
    t_dihedral(a.c, bo, po, pq, bq, fA, fE, fF, fB, E);
    out.sb += fA; out.sp += fE; out.np += fF; out.nb += fB;
    if (W) { vir_add(W, bo, fA); vir_add(W, po, fE); vir_add(W, pq, fF); vir_add(W, bq, fB); }
  }
  // planarity: vertex patch q between patch o and bead q
  V3<Real> f1, f2;
  t_planar(a.c, po - pq, bq - pq, f1, f2, E);
  out.sp += f1; out.nb += f2; out.np -= (f1 + f2);
  if (W) { vir_add(W, po, f1); vir_add(W, bq, f2); vir_add(W, pq, -(f1 + f2)); }
  if ((f & F_PREV) && !skip_bend) {
    const SPos<Real> sr = src.pos(src.step(o, -dir));
    const V3<Real> pr = rel(so, sr, a.fixq) + h * uvec(sr);
    V3<Real> g1, g2;
    t_bend(a.c, pr - po, pq - po, g1, g2, E);
    out.pp += g1; out.np += g2; out.sp -= (g1 + g2);
    if (W) { vir_add(W, pr, g1); vir_add(W, pq, g2); vir_add(W, po, -(g1 + g2)); }
  }
}

template <class Real>
__device__ __forceinline__ void store_owner(const SegSmem<Real>& sm, int ri, const OwnerOut<Real>& out) {
  sm.cs[0 * RING + ri] = out.sb.x; sm.cs[1 * RING + ri] = out.sb.y; sm.cs[2 * RING + ri] = out.sb.z;
  sm.cs[3 * RING + ri] = out.sp.x; sm.cs[4 * RING + ri] = out.sp.y; sm.cs[5 * RING + ri] = out.sp.z;
  sm.cn[0 * RING + ri] = out.nb.x; sm.cn[1 * RING + ri] = out.nb.y; sm.cn[2 * RING + ri] = out.nb.z;
  sm.cn[3 * RING + ri] = out.np.x; sm.cn[4 * RING + ri] = out.np.y; sm.cn[5 * RING + ri] = out.np.z;
  sm.cp[0 * RING + ri] = out.pp.x; sm.cp[1 * RING + ri] = out.pp.y; sm.cp[2 * RING + ri] = out.pp.z;
}

// Junction owners of circular molecules (base pairs 0, 1, N-2, N-1, both
// strands; entry t = 8 r + 2 p + strand for ring r and position p), all
// evaluated from global memory at the start of a step, before a grid
// barrier: their forces go to a.jout ([16] per entry: sb, sp, nb, np, pp),
// which the strip pass reads for these owners and for the two nucleotides of
// each strand whose neighbour owner lies across the junction.  MODE_ENERGY
// adds their energies here; MODE_STEP records removed terms (rule 2).
template <class Real, int MODE>
__device__ unsigned junction_pass(const KArgs<Real>& a, int cur) {
  unsigned fl = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_junc; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = a.jslot[t];
    const int f = a.topo[o] | F_PREV | F_NEXT;   // both neighbours exist on a ring
    const int mol = f >> MOL_SHIFT;
    const int64_t off = a.mol_off[mol];
    const GlobalSrc<Real> src{a, cur, off, a.mol_off[mol + 1] - off};
    OwnerOut<Real> out{{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if constexpr (MODE == MODE_ENERGY) {
      Real E[NTERMS], W[6];
      for (int k = 0; k < NTERMS; ++k) E[k] = 0;
      for (int k = 0; k < 6; ++k) W[k] = 0;
      owner_eval<Real, true>(a, src, o, f, false, fl, E, W, out);
      flush_energy(a, mol, E, W);
    } else {
      owner_eval<Real, true>(a, src, o, f, MODE == MODE_STEP, fl, (Real*)nullptr, (Real*)nullptr, out);
    }
    Real* j = a.jout + 16 * t;
    const V3<Real> v[5] = {out.sb, out.sp, out.nb, out.np, out.pp};
    for (int q = 0; q < 5; ++q) { j[3 * q] = v[q].x; j[3 * q + 1] = v[q].y; j[3 * q + 2] = v[q].z; }
  }
  return fl;
}

template <class Real>
__device__ __forceinline__ V3<Real> jvec(const KArgs<Real>& a, int t, int q) {
  const Real* j = a.jout + 16 * (int64_t)t + 3 * q;
  return V3<Real>{j[0], j[1], j[2]};
}

// A junction owner's forces from a.jout into its ring entries.  Nucleotide o
// is the first (position 0 on strand A, 3 on strand B) or last of its strand
// in slot order: the owner across the junction (entry ta) is its previous
// one, whose next-nucleotide forces it takes, or its next one, whose
// previous-patch force it takes.  Its slot flags have that neighbour's
// F_PREV / F_NEXT cleared, so the ring gather of nucleotide_pass skips it.
// Out of line: rings are rare.
template <class Real>
__device__ __noinline__ void junction_copy(const KArgs<Real>& a, Real* cs, Real* cn, Real* cp, int64_t o) {
  const int t = a.jidx[o], pos = (t >> 1) & 3, ta = (t & ~7) | ((3 - pos) << 1) | (t & 1);
  OwnerOut<Real> out{jvec(a, t, 0), jvec(a, t, 1), jvec(a, t, 2), jvec(a, t, 3), jvec(a, t, 4)};
  const bool first = (o & 1) ? pos == 3 : pos == 0, last = (o & 1) ? pos == 0 : pos == 3;
  if (first) { out.sb += jvec(a, ta, 2); out.sp += jvec(a, ta, 3); }
  if (last) out.sp += jvec(a, ta, 4);
  const int ri = ring(o);
  cs[0 * RING + ri] = out.sb.x; cs[1 * RING + ri] = out.sb.y; cs[2 * RING + ri] = out.sb.z;
  cs[3 * RING + ri] = out.sp.x; cs[4 * RING + ri] = out.sp.y; cs[5 * RING + ri] = out.sp.z;
  cn[0 * RING + ri] = out.nb.x; cn[1 * RING + ri] = out.nb.y; cn[2 * RING + ri] = out.nb.z;
  cn[3 * RING + ri] = out.np.x; cn[4 * RING + ri] = out.np.y; cn[5 * RING + ri] = out.np.z;
  cp[0 * RING + ri] = out.pp.x; cp[1 * RING + ri] = out.pp.y; cp[2 * RING + ri] = out.pp.z;
}

// Owner o's terms into the ring entries of o (cs, cn, cp).  EXT: the kernel
// instance for systems with circular molecules or the bubble rule.
template <class Real, bool EXT>
__device__ __forceinline__ void owner_terms(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t o, int cur,
                                            bool persist, unsigned& fl, Real* E, Real* W) {
  const int ri = ring(o);
  const int f = sm.flg[ri];
  if constexpr (EXT) {
    if (f & F_JUNC) {   // evaluated by junction_pass
      junction_copy(a, sm.cs, sm.cn, sm.cp, o);
      return;
    }
  }
  OwnerOut<Real> out{{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  if (f & F_NEXT) owner_eval<Real, EXT>(a, RingSrc<Real>{sm.pos, sm.flg}, o, f, persist, fl, E, W, out);
  store_owner(sm, ri, out);
}

// MODE_ENERGY: per-term energies and virial of one owner or nucleotide, added
// in FP64 to its molecule.
template <class Real>
__device__ __forceinline__ void flush_energy(const KArgs<Real>& a, int mol, Real* E, Real* W) {
  double* dst = a.eout + EOUT_STRIDE * mol;
  for (int k = 0; k < NTERMS; ++k) if (E[k] != (Real)0) atomicAdd(dst + k, (double)E[k]);
  for (int k = 0; k < 6; ++k) if (W[k] != (Real)0) atomicAdd(dst + NTERMS + k, (double)W[k]);
}

// Stage slot g into its ring entry (f = 0 for a slot outside [0, n)).  Two
// ways of loading ahead were measured slower: the next tile's slots in
// registers (64 registers spill; at 80 registers three CTAs per SM hide less
// latency than four), and cp.async copies of each lane's list data and of its
// first two partners into shared memory one tile ahead (the 3 KB per warp of
// buffers cut residency from 32 to 24 warps per SM: 159 against 136 us per
// step at 1 Mbp).
template <class Real>
__device__ __forceinline__ void stage_slot(const KArgs<Real>& a, const SegSmem<Real>& sm, int cur, int64_t g) {
  const int ri = ring(g);
  if (g >= 0 && g < a.n) {
    load_slot(a, cur, g, sm.pos[ri]);
    sm.flg[ri] = a.topo[(unsigned)g];
  } else {
    sm.flg[ri] = 0;
  }
}

// Owner o's terms.  `home`: o's slot belongs to this strip (the strip before
// it evaluates o again for its last nucleotides); MODE_ENERGY then adds the
// energies to the molecule, MODE_STEP records removed terms (rule 2).
template <class Real, int MODE, bool EXT>
__device__ __forceinline__ void owner_pass(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t o, int cur,
                                           bool home, unsigned& fl) {
  if constexpr (MODE == MODE_ENERGY) {
    Real E[NTERMS], W[6];
    for (int k = 0; k < NTERMS; ++k) E[k] = 0;
    for (int k = 0; k < 6; ++k) W[k] = 0;
    owner_terms<Real, EXT>(a, sm, o, cur, false, fl, home ? E : nullptr, home ? W : nullptr);
    if (home) flush_energy(a, sm.flg[ring(o)] >> MOL_SHIFT, E, W);
  } else {
    owner_terms<Real, EXT>(a, sm, o, cur, MODE == MODE_STEP && home, fl, nullptr, nullptr);
  }
}

template <class Real>
__device__ __forceinline__ void store_state(const KArgs<Real>& a, int nxt, int64_t g, int k0, int k1, int k2,
                                            const double* X, V3<Real> u, int packed) {
  const unsigned ns = (unsigned)a.ns, gu = (unsigned)g;   // slot indices stay below 2^26
  if constexpr (sizeof(Real) == 4) {
    a.Kw[(unsigned)nxt * ns + gu] = make_int4(k0, k1, k2, packed);
    a.U[(unsigned)nxt * ns + gu] = make_float4(u.x, u.y, u.z, 0.0f);
  } else {
    double* Xo = a.X + (size_t)nxt * 3 * a.ns;
    double* uo = a.ud + (size_t)nxt * 3 * a.ns;
    Xo[gu] = X[0]; Xo[ns + gu] = X[1]; Xo[2 * ns + gu] = X[2];
    uo[gu] = u.x; uo[ns + gu] = u.y; uo[2 * ns + gu] = u.z;
  }
}

// Own periodic image word of slot gu (image fields and steric flag) in the
// FP64 path; the mixed path's mirror needs no image.
template <class Real>
__device__ __forceinline__ int own_image(const KArgs<Real>& a, int cur, unsigned gu) {
  if constexpr (sizeof(Real) == 4) return 0;
  else return a.img[gu];
}

// Typed WCA force (App. A Eq. 11) on the bead of slot gu (staged record me,
// orientation um, flags f, image word img_me) from its list entry ent; the
// bead separation and the pair energy go to *dout, *eout when given.
template <class Real>
__device__ __forceinline__ V3<Real> pair_force(const KArgs<Real>& a, int cur, unsigned gu, const SPos<Real>& me,
                                               V3<Real> um, int f, int img_me, int ent, V3<Real>* dout, Real* eout) {
  const unsigned ns = (unsigned)a.ns;
  const Real h = a.c.h;
  const int j = ent & ENT_JMASK;
  V3<Real> R;
  V3<Real> uj;
  int wj;   // the partner's image word (periodic image, steric flag)
  if constexpr (sizeof(Real) == 4) {
    const int4 kj = a.Kw[(unsigned)cur * ns + (unsigned)j];
    const float4 u4 = a.U[(unsigned)cur * ns + (unsigned)j];
    wj = kj.w;
    uj = V3<float>{u4.x, u4.y, u4.z};
    // the mirrors' wrap-around difference is the minimum-image separation
    R = V3<float>{(float)(int)((unsigned)kj.x - (unsigned)me.kx) * a.fixq[0],
                  (float)(int)((unsigned)kj.y - (unsigned)me.ky) * a.fixq[1],
                  (float)(int)((unsigned)kj.z - (unsigned)me.kz) * a.fixq[2]};
  } else {
    const double* X = a.X + (size_t)cur * 3 * a.ns;
    const double* ud = a.ud + (size_t)cur * 3 * a.ns;
    uj = V3<double>{ud[(unsigned)j], ud[ns + (unsigned)j], ud[2 * ns + (unsigned)j]};
    R = V3<double>{X[(unsigned)j] - me.x, X[ns + (unsigned)j] - me.y, X[2 * ns + (unsigned)j] - me.z};
    wj = a.img[j];
    if (a.periodic) {
      R.x += (double)(img_comp(img_me, 0) - img_comp(wj, 0) + ent_shift(ent, 0)) * a.L[0];
      R.y += (double)(img_comp(img_me, 1) - img_comp(wj, 1) + ent_shift(ent, 1)) * a.L[1];
      R.z += (double)(img_comp(img_me, 2) - img_comp(wj, 2) + ent_shift(ent, 2)) * a.L[2];
    }
  }
  // bead_j - bead_me; in FP32 formed as fma(h, u_me - u_j, R), which is
  // antisymmetric bit for bit (the pair force from the partner's side is
  // exactly its negative), as pair halving needs
  V3<Real> d;
  if constexpr (sizeof(Real) == 4) {
    d = V3<Real>{fmaf(h, um.x - uj.x, R.x), fmaf(h, um.y - uj.y, R.y), fmaf(h, um.z - uj.z, R.z)};
  } else {
    d = R - h * uj + h * um;
  }
  const bool cross_strand = ((gu ^ (unsigned)j) & 1u) != 0;
  // typed sigma (Sec. 2, reading A1): two steric beads (either strand) at
  // sigma_ss, or at sigma_cross_steric across strands when that is set; any
  // other pair across strands at sigma_cross.  The partner's steric flag is
  // bit 30 of its image word.
  const bool st2 = (f & F_STERIC) && ((wj >> IMG_STERIC_SHIFT) & 1);
  Real s2 = a.c.sss2, rc2 = a.c.rcss2;
  if (cross_strand) {
    const bool cs = st2 && a.c.scs2 > (Real)0;
    s2 = cs ? a.c.scs2 : a.c.scr2;
    rc2 = cs ? a.c.rccs2 : a.c.rccr2;
  }
  Real e;
  const V3<Real> fw = t_wca(a.c, d, s2, rc2, &e);
  if (dout) *dout = d;
  if (eout) *eout = e;
  return fw;
}

// The list pairs of the tile's nucleotides B .. B+31 spread evenly over the
// warp's lanes (warp-collective; `act` false for a lane past the strip): the
// pairs are numbered nucleotide by nucleotide (an exclusive scan of the list
// counts), each lane evaluates pairs lane, lane + 32, ... in rounds of 64
// into the shared buffer, and each nucleotide's lane then adds its own pair
// forces to Fb in list order.  The warp iterates as often as the tile has
// pairs / 32, not as often as its fullest list; steric beads hold most
// pairs (about five against none for a ghost in the relaxed helix).
template <class Real>
__device__ __forceinline__ void warp_pairs(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t g, bool act, int cur,
                                           V3<Real>& Fb) {
  const int lane = threadIdx.x & 31;
  const int64_t B = g - lane;
  const unsigned ns = (unsigned)a.ns;
  if constexpr (sizeof(Real) == 4) {
    // pair halving: the tile's pairs evaluated once each (k_rebuild_pack),
    // 32 at a time, then every nucleotide adds its list entries' forces in
    // list order, negating those its partner evaluated
    const int tc = a.evl ? a.tcnt[(unsigned)(B >> 5)] : -1;
    if (tc >= 0) {
      // the list count and entry codes first, so that their latency overlaps the evaluation
      const int nn = act ? a.ncnt[(unsigned)g] : 0;
      const uint2 cw = act ? a.psrc[(unsigned)g] : make_uint2(0u, 0u);
      const int* ev = a.evl + (size_t)(B >> 5) * EVL_CAP;
#pragma unroll
      for (int k = 0; k < EVL_CAP / SEG; ++k) {
        const int p = k * SEG + lane;
        if (p < tc) {
          const int e = ev[p];
          const int L = (e >> 26) & 31;
          const int rL = ring(B + L);
          const SPos<Real>& mL = sm.pos[rL];
          const V3<Real> fw = pair_force(a, cur, (unsigned)(B + L), mL, uvec(mL), sm.flg[rL], 0, e & ENT_JMASK,
                                         (V3<Real>*)nullptr, (Real*)nullptr);
          Real* o = sm.pf + 3 * p;
          o[0] = fw.x; o[1] = fw.y; o[2] = fw.z;
        }
      }
      __syncwarp();
      for (int q = 0; q < nn; ++q) {
        const unsigned c = ((q < 4 ? cw.x : cw.y) >> (8 * (q & 3))) & 255u;
        const Real* o = sm.pf + 3 * (c & 127u);
        const unsigned sg = (c & 128u) << 24;   // sign bit of a negated force
        Fb += V3<Real>{__uint_as_float(__float_as_uint(o[0]) ^ sg), __uint_as_float(__float_as_uint(o[1]) ^ sg),
                       __uint_as_float(__float_as_uint(o[2]) ^ sg)};
      }
      __syncwarp();
      return;
    }
  }
  const int nn = act ? a.ncnt[(unsigned)g] : 0;
  int incl = nn;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (total == 0) return;
  const int excl = incl - nn;
  sm.pst[lane] = excl;
  __syncwarp();
  for (int c0 = 0; c0 < total; c0 += 2 * SEG) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int p = c0 + k * SEG + lane;
      if (p < total) {
        int L = 0;   // the nucleotide (lane) the pair belongs to: last first-index <= p
#pragma unroll
        for (int st = 16; st > 0; st >>= 1)
          if (sm.pst[L + st] <= p) L += st;
        const unsigned gL = (unsigned)(B + L);
        const int rL = ring(B + L);
        const int fL = sm.flg[rL];
        const SPos<Real>& mL = sm.pos[rL];
        const int img = (sizeof(Real) == 8 && a.periodic) ? own_image(a, cur, gL) : 0;
        const int ent = a.nbr[(unsigned)(p - sm.pst[L]) * ns + gL];
        const V3<Real> fw = pair_force(a, cur, gL, mL, uvec(mL), fL, img, ent, (V3<Real>*)nullptr, (Real*)nullptr);
        Real* o = sm.pf + 3 * (k * SEG + lane);
        o[0] = fw.x; o[1] = fw.y; o[2] = fw.z;
      }
    }
    __syncwarp();
    if (nn) {
      const int p0 = excl > c0 ? excl : c0, p1 = excl + nn < c0 + 2 * SEG ? excl + nn : c0 + 2 * SEG;
      for (int p = p0; p < p1; ++p) {
        const Real* o = sm.pf + 3 * (p - c0);
        Fb += V3<Real>{o[0], o[1], o[2]};
      }
    }
    __syncwarp();
  }
}

// Forces on nucleotide g from the owner rings, its H-bond and its list
// pairs, then (MODE_STEP) its Langevin update; MODE_FORCES writes the site
// forces, MODE_ENERGY adds its per-nucleotide energies.
template <class Real, int MODE, bool EXT>
__device__ __forceinline__ void nucleotide_pass(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t g, bool act,
                                                int cur, int64_t step, unsigned& fl) {
  const int nxt = cur ^ 1;
  const unsigned ns = (unsigned)a.ns, gu = (unsigned)g;   // slot indices stay below 2^26: 32-bit index arithmetic
  Real Eb[NTERMS];
  Real Wb[6];
  if constexpr (MODE == MODE_ENERGY) {
    for (int k = 0; k < NTERMS; ++k) Eb[k] = 0;
    for (int k = 0; k < 6; ++k) Wb[k] = 0;
  }
  {
    const int ri = ring(g);
    const int f = act ? sm.flg[ri] : 0;
    const SPos<Real>& me = sm.pos[ri];
    const Real h = a.c.h;
    const V3<Real> um = uvec(me);
    V3<Real> Fb{0, 0, 0}, Fp{0, 0, 0};
    if (act) {
    Fb = V3<Real>{sm.cs[0 * RING + ri], sm.cs[1 * RING + ri], sm.cs[2 * RING + ri]};
    Fp = V3<Real>{sm.cs[3 * RING + ri], sm.cs[4 * RING + ri], sm.cs[5 * RING + ri]};
    const int dir = (g & 1) ? -2 : 2;
    // (a neighbour across a ring's junction has its flag cleared here: its
    // owner's forces arrive through cs, see owner_terms)
    if (f & F_PREV) {
      const int op = ring(g - dir);
      Fb += V3<Real>{sm.cn[0 * RING + op], sm.cn[1 * RING + op], sm.cn[2 * RING + op]};
      Fp += V3<Real>{sm.cn[3 * RING + op], sm.cn[4 * RING + op], sm.cn[5 * RING + op]};
    }
    if (f & F_NEXT) {
      const int on = ring(g + dir);
      Fp += V3<Real>{sm.cp[0 * RING + on], sm.cp[1 * RING + on], sm.cp[2 * RING + on]};
    }
    // hydrogen bond with the partner (App. A Eq. 10), broken beyond rc
    {
      const SPos<Real>& q = sm.pos[ring(g ^ 1)];
      const V3<Real> d = rel(me, q, a.fixq) + h * uvec(q) - h * um;   // patch_q - patch_me
      const Real r2 = dot(d, d);
      if (r2 <= a.c.rchb2) {
        const Real khb = (f & F_GC) ? a.c.khb_gc : a.c.khb;   // Sec. 5: A.T / G.C stiffness
        Real k2 = (Real)2 * khb;
        if (a.c.r0hb != (Real)0) k2 *= (Real)1 - a.c.r0hb * rsqrt_(r2);
        Fp += k2 * d;
        if constexpr (MODE == MODE_ENERGY) {
          if ((g & 1) == 0) {
            const Real r = sqrt_(r2);
            const Real rc = sqrt_(a.c.rchb2);
            Eb[2] += khb * ((r - a.c.r0hb) * (r - a.c.r0hb) - (rc - a.c.r0hb) * (rc - a.c.r0hb));
            vir_add(Wb, d, -(k2 * d));   // force on the partner patch
          }
        }
      }
    }
    }
    // typed WCA pairs (App. A Eq. 11) from the neighbour list: spread over the
    // warp's lanes (warp_pairs), or one lane per nucleotide with energies
    if constexpr (MODE == MODE_ENERGY) {
      if (act) {
        const int nn = a.ncnt[gu];
        const int img_me = (sizeof(Real) == 8 && a.periodic) ? own_image(a, cur, gu) : 0;
        for (int q = 0; q < nn; ++q) {
          V3<Real> d;
          Real e;
          const V3<Real> fw = pair_force(a, cur, gu, me, um, f, img_me, a.nbr[(unsigned)q * ns + gu], &d, &e);
          Fb += fw;
          Eb[3] += (Real)0.5 * e;
          vir_add(Wb, d, (Real)-0.5 * fw);
        }
      }
    } else {
      warp_pairs(a, sm, g, act, cur, Fb);
    }
    if (!act) return;
    // applied load on the last base pair (Sec. 4.1, 4.2): f/2 at each centre,
    // torque as a couple normal to its axis; half on each site
    if (f & F_TOP) {
      const int mol = f >> MOL_SHIFT;
      const double* ex = a.ext + 8 * mol;
      V3<Real> Fe{(Real)(0.5 * ex[0]), (Real)(0.5 * ex[1]), (Real)(0.5 * ex[2])};
      const V3<Real> Tq{(Real)ex[3], (Real)ex[4], (Real)ex[5]};
      const Real tn2 = dot(Tq, Tq);
      if (tn2 > (Real)0) {
        const V3<Real> th = rsqrt_(tn2) * Tq;
        V3<Real> rho = (Real)-0.5 * rel(me, sm.pos[ring(g ^ 1)], a.fixq);   // centre offset from the pair centre
        rho -= dot(rho, th) * th;
        const Real S = (Real)2 * dot(rho, rho);
        if (S > (Real)1e-12) Fe += ((Real)1 / S) * cross(Tq, rho);
      }
      Fb += (Real)0.5 * Fe;
      Fp += (Real)0.5 * Fe;
    }
    if constexpr (MODE == MODE_FORCES) {
      double* o = a.fout + 6 * g;
      o[0] = Fb.x; o[1] = Fb.y; o[2] = Fb.z; o[3] = Fp.x; o[4] = Fp.y; o[5] = Fp.z;
    } else {
      // rigid body (Sec. 2): force and torque about the centre
      const V3<Real> F = Fb + Fp;
      const V3<Real> Tc = h * cross(um, Fp - Fb);
      const int mol = f >> MOL_SHIFT;
      const uint32_t local = (uint32_t)(g - 2 * a.mol_off[mol]);
      double Xd[3], Vd[3];
      if constexpr (sizeof(Real) == 4) {
        Xd[0] = a.X[gu]; Xd[1] = a.X[ns + gu]; Xd[2] = a.X[2 * ns + gu];
      } else {
        Xd[0] = me.x; Xd[1] = me.y; Xd[2] = me.z;
      }
      Vd[0] = a.V[gu]; Vd[1] = a.V[ns + gu]; Vd[2] = a.V[2 * ns + gu];
      V3<Real> Om{a.Om[gu], a.Om[ns + gu], a.Om[2 * ns + gu]};
      // the rebuild reference and the image word, loaded with the state and
      // ahead of its stores (which the compiler cannot move them across)
      int kr[3] = {0, 0, 0}, packed = 0;
      if constexpr (MODE == MODE_STEP) {
        kr[0] = a.kref[gu]; kr[1] = a.kref[ns + gu]; kr[2] = a.kref[2 * ns + gu];
        if constexpr (sizeof(Real) == 4) packed = a.Kw[(unsigned)cur * ns + gu].w;   // image and steric flag carried
      }
      const bool frozen = (f & F_FROZEN) != 0;
      V3<Real> Ft{0, 0, 0}, Tt{0, 0, 0};
      if (!frozen) {
        // App. A Eq. 8 per site: friction -gamma v_s and noise eta_s, summed over the dumbbell
        V3<Real> eb, ep;
        nucleotide_noise(a, local, step, mol, eb, ep);
        V3<Real> Vh;
        if constexpr (sizeof(Real) == 4) {
          Vh = V3<Real>{d2f_bits(Vd[0]), d2f_bits(Vd[1]), d2f_bits(Vd[2])};
        } else {
          Vh = V3<Real>{Vd[0], Vd[1], Vd[2]};
        }
        Ft = F - a.c.gam2 * Vh + eb + ep;
        Tt = Tc - a.c.gamr * Om + h * cross(um, ep - eb);
      }
      if constexpr (MODE == MODE_ENERGY) {
        if (!frozen) {
          V3<Real> Vf{(Real)Vd[0], (Real)Vd[1], (Real)Vd[2]};
          Vf += a.c.halfdtM * Ft;
          V3<Real> Of = Om + a.c.halfdtI * Tt;
          Of -= dot(Of, um) * um;
          Eb[8] += (Real)0.5 * a.c.M * dot(Vf, Vf);
          Eb[9] += (Real)0.5 * a.c.I * dot(Of, Of);
        }
      } else {
        // MODE_STEP: leapfrog kick and drift (Eq. 16), FP64 accumulation of V and X
        V3<Real> un = um;
        if (!frozen) {
          const V3<Real> dv = a.c.dtM * Ft;
          if constexpr (sizeof(Real) == 4) {
            Vd[0] += f2d_bits(dv.x); Vd[1] += f2d_bits(dv.y); Vd[2] += f2d_bits(dv.z);
          } else {
            Vd[0] += dv.x; Vd[1] += dv.y; Vd[2] += dv.z;
          }
          Om += a.c.dtI * Tt;
          Om -= dot(Om, um) * um;
          Xd[0] = fma(a.c.dt_d, Vd[0], Xd[0]);
          Xd[1] = fma(a.c.dt_d, Vd[1], Xd[1]);
          Xd[2] = fma(a.c.dt_d, Vd[2], Xd[2]);
          const Real w2 = dot(Om, Om);
          if (w2 > (Real)0) {
            const Real w = sqrt_(w2);
            Real sn, cs;
            sincos_(w * a.c.dt, &sn, &cs);
            const V3<Real> ax = ((Real)1 / w) * Om;
            un = cs * um + sn * cross(ax, um);
            un = rsqrt_(dot(un, un)) * un;
          }
          // a NaN or infinity in any component makes the sum non-finite
          if (!isfinite((Ft.x + Ft.y) + (Ft.z + Om.x) + (Om.y + Om.z))) fl |= B_ENAN;
          a.V[gu] = Vd[0]; a.V[ns + gu] = Vd[1]; a.V[2 * ns + gu] = Vd[2];
          a.Om[gu] = Om.x; a.Om[ns + gu] = Om.y; a.Om[2 * ns + gu] = Om.z;
          if constexpr (sizeof(Real) == 4) {
            a.X[gu] = Xd[0]; a.X[ns + gu] = Xd[1]; a.X[2 * ns + gu] = Xd[2];
          }
        }
        // the new position's mirror (in the FP64 path it serves the rebuild trigger only)
        const int k0 = fixs(Xd[0], a.fixS[0]), k1 = fixs(Xd[1], a.fixS[1]), k2 = fixs(Xd[2], a.fixS[2]);
        store_state(a, nxt, g, k0, k1, k2, Xd, un, packed);
        // rebuild trigger: a bead moved more than skin/2 since the last build
        const float hf = (float)h;
        const float ddx = (float)(int)((unsigned)(k0 + bead_off(hf * (float)un.x, a.fixSf[0])) - (unsigned)kr[0]) * a.fixq[0];
        const float ddy = (float)(int)((unsigned)(k1 + bead_off(hf * (float)un.y, a.fixSf[1])) - (unsigned)kr[1]) * a.fixq[1];
        const float ddz = (float)(int)((unsigned)(k2 + bead_off(hf * (float)un.z, a.fixSf[2])) - (unsigned)kr[2]) * a.fixq[2];
        if (ddx * ddx + ddy * ddy + ddz * ddz > a.c.skin_half2) fl |= B_STALE;
      }
    }
  }
  if constexpr (MODE == MODE_ENERGY) flush_energy(a, sm.flg[ring(g)] >> MOL_SHIFT, Eb, Wb);   // act here
}

// One warp's strip: tiles [t0, t1) of SEG slots.  The prologue stages slots
// s0-8 .. s0+7 and computes owners s0-2 .. s0+1; every tile at base B then
// stages slots B+8 .. B+39 (the ring holds B-24 .. B+39), computes owners
// B+2 .. B+33 (one per lane; with their base-pair neighbourhoods they read
// slots B-2 .. B+37) and finishes nucleotides B .. B+31, whose terms come
// from owners B-2 .. B+33.  An owner's energy is counted by the strip that
// holds its slot.
template <class Real, int MODE, bool EXT>
__device__ void strip_pass(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t t0, int64_t t1, int cur,
                           int64_t step, unsigned& fl) {
  if (t0 >= t1) return;
  const int lane = threadIdx.x & 31;
  const int64_t s0 = t0 * SEG;
  const int64_t s1 = t1 * SEG < a.n ? t1 * SEG : a.n;
  if (lane < 16) stage_slot(a, sm, cur, s0 - 8 + lane);
  __syncwarp();
  if (EXT && a.bubble) {
    if (lane < 16 && !(lane & 1)) mark_open(a, sm, s0 - 8 + lane);
    __syncwarp();
  }
  if (lane < 4) owner_pass<Real, MODE, EXT>(a, sm, s0 - 2 + lane, cur, lane >= 2 && s0 - 2 + lane < s1, fl);
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t B = t * SEG;
    __syncwarp();
    stage_slot(a, sm, cur, B + 8 + lane);
    __syncwarp();
    if (EXT && a.bubble) {
      if (!(lane & 1)) mark_open(a, sm, B + 8 + lane);
      __syncwarp();
    }
    owner_pass<Real, MODE, EXT>(a, sm, B + 2 + lane, cur, B + 2 + lane < s1, fl);
    __syncwarp();
    nucleotide_pass<Real, MODE, EXT>(a, sm, B + lane, B + lane < s1, cur, step, fl);   // warp-collective
  }
  __syncwarp();
}

// ---------------------------------------------------------------- list rebuild in the step kernel
// The five phases of the rebuild kernels (bin, block sums, scan, scatter,
// list), each over the whole persistent grid with a bounded grid barrier
// after it, for systems small enough that kernel boundaries cost more than
// the barriers.  The list phase keeps each lane's buffer in the warp's
// shared ring, which the next step restages.  Linear and hashed tables.
template <class Real>
__device__ unsigned fused_rebuild(const KArgs<Real>& a, const SegSmem<Real>& sm, int cur, unsigned* s_word,
                                  unsigned* s_red) {
  static_assert(seg_warp_bytes<Real>() >= sizeof(int) * 32 * LIST_CAP, "list buffers must fit in a warp's ring");
  unsigned fl = 0;
  rebuild_bin(a, cur, fl);
  unsigned r = grid_sync(a.bar, gridDim.x, fl, a.spin_budget, s_word);
  if (r & B_ERRMASK) return r;
  rebuild_scan_a(a, s_red);
  r = grid_sync(a.bar, gridDim.x, 0u, a.spin_budget, s_word);
  if (r & B_ERRMASK) return r;
  rebuild_scan_b(a, s_red);
  r = grid_sync(a.bar, gridDim.x, 0u, a.spin_budget, s_word);
  if (r & B_ERRMASK) return r;
  rebuild_scatter(a);
  r = grid_sync(a.bar, gridDim.x, 0u, a.spin_budget, s_word);
  if (r & B_ERRMASK) return r;
  fl = 0;
  int* list = reinterpret_cast<int*>(sm.pos) + (threadIdx.x & 31) * LIST_CAP;
  if (a.table == TABLE_LINEAR) rebuild_list_lanes<Real>(a, fl, list);
  else rebuild_list_lanes_hash<Real>(a, fl, list);
  r = grid_sync(a.bar, gridDim.x, fl, a.spin_budget, s_word);
  if (blockIdx.x == 0 && threadIdx.x == 0 && !(r & B_ERRMASK)) *a.nrebuild += 1;
  return r;
}

// ---------------------------------------------------------------- persistent kernel
// MODE_STEP: advance up to *steps_left steps (all of them when steps_left is
// null: nsteps), one bounded grid barrier per step; stop early when a bead
// moved more than skin/2 (the rebuild kernels run next) or on an error.
// MODE_FORCES / MODE_ENERGY: one pass with the current list.
// EXT: the instance for systems with circular molecules, the bubble rule or
// steric pairs across strands (junction pass, open-pair marks, removed
// terms, the partner's steric flag); the other instance compiles none of it.
// FUSED (MODE_STEP): a stale list is rebuilt inside the kernel
// (fused_rebuild) and the steps go on, instead of returning so that the
// rebuild kernels run.
// Mixed precision runs CTAs of up to 1024 threads at 64 registers (one CTA
// of 32 warps per SM, or four of 8); FP64 CTAs of up to 256 threads.
template <class Real>
__host__ __device__ constexpr int engine_max_threads() { return sizeof(Real) == 4 ? 1024 : 256; }

template <class Real, int MODE, int CAPMAX, bool EXT, bool FUSED = false>
__global__ void __launch_bounds__(engine_max_threads<Real>(), 1) engine_kernel(const __grid_constant__ KArgs<Real> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned s_word;
  __shared__ unsigned s_fl;
  const SegSmem<Real> sm = carve<Real>(smem_raw, blockDim.x);
  const int64_t step0 = *a.step;
  int64_t budget = (MODE == MODE_STEP) ? (a.steps_left ? *a.steps_left : a.nsteps) : 1;
  if (MODE == MODE_STEP && (*a.err & B_ERRMASK)) budget = 0;
  int need = 0;
  int64_t done = 0;
  unsigned errbits = 0;
  for (int64_t it = 0; it < budget; ++it) {
    const int64_t step = step0 + it;
    const int cur = (int)(step & 1);
    if (threadIdx.x == 0) s_fl = 0;
    __syncthreads();
    unsigned fl = 0;
    if (EXT && a.n_junc) {   // circular molecules: junction owners first, then a grid barrier
      const unsigned r = grid_sync(a.bar, gridDim.x, junction_pass<Real, MODE>(a, cur), a.spin_budget, &s_word);
      if (r & B_ERRMASK) { errbits = r; break; }
    }
    const int64_t wpb = blockDim.x >> 5;
    const int64_t nw = gridDim.x * wpb, w = blockIdx.x * wpb + (threadIdx.x >> 5);
    strip_pass<Real, MODE, EXT>(a, sm, w * a.nseg / nw, (w + 1) * a.nseg / nw, cur, step, fl);
    if (fl) atomicOr(&s_fl, fl);
    __syncthreads();
    if (MODE != MODE_STEP) {
      errbits = s_fl;
      break;
    }
    const unsigned r = grid_sync(a.bar, gridDim.x, s_fl, a.spin_budget, &s_word);
    if (r & B_ERRMASK) { errbits = r; break; }
    ++done;
    if (r & B_STALE) {
      if constexpr (FUSED) {
        __shared__ unsigned s_red[32];
        const unsigned rr = fused_rebuild(a, sm, (int)((step + 1) & 1), &s_word, s_red);
        if (rr & B_ERRMASK) { errbits = rr; break; }
        continue;
      } else {
        need = 1;
        break;
      }
    }
  }
  if (threadIdx.x == 0) {
    if (errbits & B_ERRMASK) atomicOr(a.err, errbits & B_ERRMASK);
    if (blockIdx.x == 0 && MODE == MODE_STEP) {
      *a.step = step0 + done;
      if (need) *a.rebuild = 1;
      const int64_t left = budget - done;
      if (a.steps_left) *a.steps_left = left;
      if (a.use_cond) {
        const bool more = left > 0 && done > 0 && (errbits & B_ERRMASK) == 0;
        cudaGraphSetConditional(a.h_while, more ? 1u : 0u);
      }
    }
  }
}

}  // namespace dsdna
