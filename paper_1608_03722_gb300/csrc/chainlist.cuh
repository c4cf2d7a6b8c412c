// chainlist.cuh -- chain-window neighbour-list build of the dsDNA engine
// (periodic box with at least 3 grid cells per edge, or open box).  Included
// by kern_launch.cuh after rebuild.cuh.
//
// A nucleotide's list partners are of two kinds.  Almost all of them sit a
// few slots away along the chain: the steric beads three nucleotides along
// its own strand and the nearest beads of the partner strand (Sec. 2); in a
// confined 1 Mbp chain 99.7% lie within 8 slots.  The rest are contacts
// between distant stretches of the chain.  The build splits the slot array
// into segments of SEG_W = 16 consecutive slots (8 base pairs) and finds
//  * every pair whose two segments are equal or adjacent by testing all of
//    them: the 48 slots of a bead's segment and its two neighbours, staged
//    in shared memory, with no cell table at all;
//  * every other pair through a grid of segment bounding spheres: a segment
//    of radius R <= sg_rcap sits in the cell of its centre, cells are at
//    least 2 sg_rcap + the largest list radius wide, so a segment's partners
//    lie in segments of its 27 neighbour cells, and the bead pairs of two
//    segments are tested only when their spheres come within list range.
// A segment wider than sg_rcap (a stretched or broken chain, or one that
// spans two molecules) enters the grid bead by bead and queries bead by bead.
// Lists come out sorted by partner slot, as the force sum order requires,
// and the pair-halving pack of each 32-slot tile runs in the same warp.
#pragma once
#include <climits>

#include "rebuild.cuh"

namespace dsdna {

constexpr int SEG_W = 16;          // slots per segment (8 base pairs)
constexpr int CL_WARPS = 8;        // warps per CTA of the list kernel
constexpr int CL_WIN = 64;         // staged slots per 32-slot tile: 16 below it, its own 32, 16 above
constexpr float CL_FAR = 1.0e18f;  // staged position of a slot outside the system (never within reach)
// staged record word: bit 0 steric, bits 1-6 the unwrap shift + 1 of each
// axis (fast path), bit 7 a slot of the system, bits 8.. the molecule (slow path)
constexpr int CL_VALID = 0x80;

// Cell of the segment grid holding position (x, y, z) (periodic box: clamped
// into the box).
template <class Real>
__device__ __forceinline__ void seg_cell(const KArgs<Real>& a, float x, float y, float z, int* ci) {
  const float p[3] = {x, y, z};
  for (int c = 0; c < 3; ++c) {
    const int k = (int)floorf(p[c] * a.sg_invh[c]);
    ci[c] = !a.periodic ? k : (k >= a.sg_nc[c] ? a.sg_nc[c] - 1 : (k < 0 ? 0 : k));
  }
}

// Table entry of neighbour q (0..26; 13 is the cell itself) of cell ci: the
// linear index of the wrapped cell in a periodic box, else a hash of the
// molecule and the cell (different molecules never interact; distinct cells
// may share an entry).
template <class Real>
__device__ __forceinline__ unsigned seg_key(const KArgs<Real>& a, int mol, const int* ci, int q) {
  int cc[3] = {ci[0] + q % 3 - 1, ci[1] + (q / 3) % 3 - 1, ci[2] + q / 9 - 1};
  if (!a.periodic) return hash_block(mol, cc[0], cc[1], cc[2]) & a.sg_mask;
  for (int c = 0; c < 3; ++c) cc[c] = cc[c] < 0 ? cc[c] + a.sg_nc[c] : (cc[c] >= a.sg_nc[c] ? cc[c] - a.sg_nc[c] : cc[c]);
  return (unsigned)cc[0] + (unsigned)a.sg_nc[0] * ((unsigned)cc[1] + (unsigned)a.sg_nc[1] * (unsigned)cc[2]);
}

// S1: bin every bead as the cell-walk build does (wrapped position, image
// word, rebuild reference), then the bounding sphere of each 16-slot segment
// (a 16-lane group of the warp; positions relative to the segment's first
// bead by minimum image) and its count in the segment grid.
template <class Real>
__global__ void k_rebuild_segbin(const KArgs<Real> a) {
  unsigned fl = 0;
  const int cur = (int)(*a.step & 1);
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // whole warps: ns is a multiple of 32, and so is the stride
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.ns; g += stride) {
    const bool in = g < a.n;
    float pw[3] = {0.0f, 0.0f, 0.0f};
    int mol = 0;
    if (in) mol = bin_bead(a, cur, g, fl, pw);
    float r0[3], d[3];
    for (int c = 0; c < 3; ++c) {
      r0[c] = __shfl_sync(0xffffffffu, pw[c], 0, 16);
      float x = pw[c] - r0[c];
      x = fmaf(-rintf(x * a.invLf[c]), a.Lf[c], x);
      d[c] = in ? x : 0.0f;
    }
    const int nin = __popc(__ballot_sync(0xffffffffu, in) & (0xffffu << (lane & 16)));
    float m[3];
    for (int c = 0; c < 3; ++c) {
      float s = d[c];
      for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, 16);
      m[c] = nin > 0 ? s / (float)nin : 0.0f;
    }
    float r2 = 0.0f;
    if (in) {
      const float ex = d[0] - m[0], ey = d[1] - m[1], ez = d[2] - m[2];
      r2 = ex * ex + ey * ey + ez * ez;
    }
    int mlo = in ? mol : INT_MAX, mhi = in ? mol : INT_MIN;
    for (int o = 8; o > 0; o >>= 1) {
      r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o, 16));
      mlo = min(mlo, __shfl_xor_sync(0xffffffffu, mlo, o, 16));
      mhi = max(mhi, __shfl_xor_sync(0xffffffffu, mhi, o, 16));
    }
    const float R = sqrtf(r2) * 1.0001f + 1e-4f;   // rounded up past the FP32 error of the centre
    const bool wide = !(R <= a.sg_rcap) || mlo != mhi;
    int ci[3];
    if (nin > 0 && (lane & 15) == 0) {
      float c3[3];
      for (int c = 0; c < 3; ++c) {
        const float x = r0[c] + m[c];
        c3[c] = fmaf(-floorf(x * a.invLf[c]), a.Lf[c], x);
      }
      a.segc[g >> 4] = make_float4(c3[0], c3[1], c3[2], wide ? -1.0f : R);
      if (!wide) {
        seg_cell(a, c3[0], c3[1], c3[2], ci);
        atomicAdd(&a.cnt[seg_key(a, mol, ci, 13)], 1u);
      }
    }
    if (in && wide) {
      seg_cell(a, pw[0], pw[1], pw[2], ci);
      atomicAdd(&a.cnt[seg_key(a, mol, ci, 13)], 1u);
    }
  }
  if (fl) atomicOr(a.err, fl & B_ERRMASK);
}

// S2: the grid items in cell order: a segment's sphere (cent) and slot range
// (key: first slot | (beads - 1) << ENT_J_BITS), or the beads of a wide
// segment one by one with radius 0.  The count table returns to zero.
template <class Real>
__global__ void k_rebuild_segscatter(const KArgs<Real> a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.nseg16; s += stride) {
    const float4 sc = a.segc[s];
    const int64_t g0 = s * SEG_W;
    const int nb = (int)min((int64_t)SEG_W, a.n - g0);
    int ci[3];
    if (sc.w >= 0.0f) {
      seg_cell(a, sc.x, sc.y, sc.z, ci);
      const unsigned k = seg_key(a, __float_as_int(a.wpos[g0].w), ci, 13);
      const unsigned e = a.start[k] + atomicSub(&a.cnt[k], 1u) - 1u;
      a.cent[e] = sc;
      a.key[e] = (int)g0 | ((nb - 1) << ENT_J_BITS);
    } else {
      for (int b = 0; b < nb; ++b) {
        const float4 p = a.wpos[g0 + b];
        seg_cell(a, p.x, p.y, p.z, ci);
        const unsigned k = seg_key(a, __float_as_int(p.w), ci, 13);
        const unsigned e = a.start[k] + atomicSub(&a.cnt[k], 1u) - 1u;
        a.cent[e] = make_float4(p.x, p.y, p.z, 0.0f);
        a.key[e] = (int)(g0 + b);
      }
    }
  }
}

// Entry ent into a lane's list, kept sorted by partner slot.
__device__ __forceinline__ void cl_append(int* list, int& cnt, int& total, int cap, int ent) {
  ++total;
  if (cnt < cap) {
    const int j = ent & ENT_JMASK;
    int q = cnt++;
    while (q > 0 && (list[q - 1] & ENT_JMASK) > j) { list[q] = list[q - 1]; --q; }
    list[q] = ent;
  }
}

// Do spheres q and it (centre, radius) of the periodic box come within list range?
template <class Real>
__device__ __forceinline__ bool cl_spheres_meet(const KArgs<Real>& a, float4 q, float4 it) {
  const float d0[3] = {it.x - q.x, it.y - q.y, it.z - q.z};
  float r2 = 0.0f;
  for (int c = 0; c < 3; ++c) {
    const float d = fmaf(-rintf(d0[c] * a.invLf[c]), a.Lf[c], d0[c]);
    r2 = fmaf(d, d, r2);
  }
  const float reach = q.w + it.w + a.sg_reach;
  return r2 < reach * reach;
}

// Typed pairs of bead g (wrapped position p, steric flag, molecule) with the
// beads of one grid item, each at its minimum image.
template <class Real>
__device__ __forceinline__ void cl_item_pairs(const KArgs<Real>& a, int g, float4 p, bool st_g, int ir, int* list,
                                              int& cnt, int& total) {
  const int j0 = ir & ENT_JMASK, nb = (int)((unsigned)ir >> ENT_J_BITS) + 1;
  for (int b = 0; b < nb; ++b) {
    const int j = j0 + b;
    const float4 o = a.wpos[j];
    float d[3] = {o.x - p.x, o.y - p.y, o.z - p.z};
    int sc[3];
    for (int c = 0; c < 3; ++c) {
      const float s = -rintf(d[c] * a.invLf[c]);
      d[c] = fmaf(s, a.Lf[c], d[c]);
      sc[c] = (int)s;
    }
    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const float rl2 = list_r2(a.c, ((g ^ j) & 1) != 0, st_g && (a.topo[j] & F_STERIC) != 0);
    if (r2 < rl2 && __float_as_int(o.w) == __float_as_int(p.w))
      cl_append(list, cnt, total, a.cap, ent_make(j, sc[0], sc[1], sc[2]));
  }
}

// S3: one warp per 32-slot tile (segments 2t and 2t + 1), one lane per bead.
// The grid query is a chain of dependent loads (sphere -> table bounds ->
// items), so both segments' loads are issued together and ahead of the window
// test, whose arithmetic covers their latency: a lane per neighbour cell of
// either segment for the bounds, then the items of all 54 ranges spread over
// the lanes.
constexpr unsigned CL_NONE = 0xffffffffu;
template <class Real>
__global__ void __launch_bounds__(CL_WARPS * 32, 4) k_rebuild_list_chain(const KArgs<Real> a) {
  __shared__ float4 s_win[CL_WARPS][CL_WIN + CL_WIN / 16];
  __shared__ int s_list[CL_WARPS][32][LIST_CAP];
  __shared__ unsigned s_tm[CL_WARPS][32];
  __shared__ int s_base[CL_WARPS][32];
  __shared__ unsigned s_rb[CL_WARPS][54], s_ro[CL_WARPS][54];   // first item and flattened offset of each range
  __shared__ int s_gi[CL_WARPS][4];                              // accepted grid items being tested
  __shared__ float4 s_gc[CL_WARPS][4];                           // and their spheres
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned fl = 0;
  int* list = s_list[w][lane];
  float4* win = s_win[w];   // staged slot k at win[k + k / 16]: the half-warps' candidates in other banks
  for (int64_t t = (int64_t)blockIdx.x * CL_WARPS + w; t < a.nseg; t += (int64_t)gridDim.x * CL_WARPS) {
    const int64_t g0 = t * 32;
    const int g = (int)(g0 + lane);
    const bool in = g < a.n;
    // stage slots g0 - 16 .. g0 + 47; unwrapped around the middle slot
    // g0 + 16 when every slot of the window belongs to its molecule and lies
    // within a quarter box of it, so that every difference is the minimum
    // image (fast path); else stored as wrapped, each pair taking its own
    // minimum image
    float4 raw[2];
    int word[2];
    bool val[2];
    for (int h = 0; h < 2; ++h) {
      const int64_t j = g0 - 16 + lane + 32 * h;
      val[h] = j >= 0 && j < a.n;
      raw[h] = val[h] ? a.wpos[j] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      word[h] = val[h] ? ((a.topo[j] & F_STERIC) | CL_VALID) : 0;
    }
    // the two segments' spheres and this lane's own wrapped position
    const int64_t sA = 2 * t;
    const bool hasB = sA + 1 < a.nseg16;
    const float4 sc[2] = {a.segc[sA], hasB ? a.segc[sA + 1] : make_float4(0.0f, 0.0f, 0.0f, -1.0f)};
    const float4 mp = in ? a.wpos[g] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    // molecule of each segment (its first slot: staged slots 16 and 32) and its slot range
    const int qmol[2] = {__shfl_sync(0xffffffffu, __float_as_int(raw[0].w), 16),
                         __shfl_sync(0xffffffffu, __float_as_int(raw[1].w), 0)};
    int64_t slo[2] = {0, 0}, shi[2] = {a.n, a.n};
    if (a.n_mol > 1) {
      for (int h = 0; h < 2; ++h)
        if (h == 0 || hasB) {
          slo[h] = 2 * a.mol_off[qmol[h]];
          shi[h] = 2 * a.mol_off[qmol[h] + 1];
        }
    }
    // table bounds of the 27 neighbour cells of each whole segment (a hashed
    // entry that a lower lane of the same segment also reads is dropped)
    unsigned key[2] = {CL_NONE, CL_NONE};
    for (int h = 0; h < 2; ++h) {
      if (lane < 27 && sc[h].w >= 0.0f) {
        int ci[3];
        seg_cell(a, sc[h].x, sc[h].y, sc[h].z, ci);
        key[h] = seg_key(a, qmol[h], ci, lane);
      }
      if (!a.periodic) {
        for (int o = 0; o < 27; ++o) {
          const unsigned ko = __shfl_sync(0xffffffffu, key[h], o);
          if (o < lane && ko == key[h]) key[h] = CL_NONE;
        }
      }
    }
    unsigned rb[2] = {0u, 0u}, re[2] = {0u, 0u};
    for (int h = 0; h < 2; ++h)
      if (key[h] != CL_NONE) {
        rb[h] = a.start[key[h]];
        re[h] = a.start[key[h] + 1];
      }

    const float ref[3] = {__shfl_sync(0xffffffffu, raw[1].x, 0), __shfl_sync(0xffffffffu, raw[1].y, 0),
                          __shfl_sync(0xffffffffu, raw[1].z, 0)};
    const int rmol = __shfl_sync(0xffffffffu, val[1] ? __float_as_int(raw[1].w) : -1, 0);
    bool ok = true;
    float4 un[2];
    for (int h = 0; h < 2; ++h) {
      un[h] = make_float4(CL_FAR, CL_FAR, CL_FAR, __int_as_float(0));
      if (!val[h]) continue;
      float p[3] = {raw[h].x, raw[h].y, raw[h].z};
      int code = word[h];
      for (int c = 0; c < 3; ++c) {
        const float tq = rintf((ref[c] - p[c]) * a.invLf[c]);
        p[c] = fmaf(tq, a.Lf[c], p[c]);
        code |= ((int)tq + 1) << (1 + 2 * c);
        ok = ok && (!a.periodic || fabsf(p[c] - ref[c]) <= 0.24f * a.Lf[c]);
      }
      ok = ok && __float_as_int(raw[h].w) == rmol;
      un[h] = make_float4(p[0], p[1], p[2], __int_as_float(code));
    }
    const bool fast = __all_sync(0xffffffffu, ok);
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h;
      win[k + (k >> 4)] = fast ? un[h]
                               : make_float4(raw[h].x, raw[h].y, raw[h].z,
                                             __int_as_float(word[h] | (__float_as_int(raw[h].w) << 8)));
    }
    __syncwarp();

    int cnt = 0, total = 0;
    const int kb = lane & 16;   // lanes 0-15 (segment 2t) test staged slots 0..47, lanes 16-31 slots 16..63
    const float4* wb = win + kb + (kb >> 4);
    const float4 me = win[lane + 16 + ((lane + 16) >> 4)];
    const int mew = __float_as_int(me.w);
    const bool st_g = (mew & 1) != 0;
    if (in) {
      if (fast) {
        // candidate c is slot g0 - 16 + kb + c: across strands iff c and lane differ in parity
        const float rs_st = st_g ? a.c.rl_ss2 : -1.0f, rc_st = st_g ? a.c.rl_cs2 : a.c.rl_cr2;
        const bool odd = lane & 1;
        const float rE_st = odd ? rc_st : rs_st, rE_gh = odd ? a.c.rl_cr2 : -1.0f;
        const float rO_st = odd ? rs_st : rc_st, rO_gh = odd ? -1.0f : a.c.rl_cr2;
        // hits as a bit mask first (no branch in the loop; three blocks of 16
        // candidates), then appended in slot order to the still empty list
        unsigned long long hits = 0ull;
        for (int c0 = 0; c0 < 48; c0 += 16) {
          const float4* wc = wb + c0 + (c0 >> 4);
          unsigned m16 = 0u;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float4 o = wc[k];
            const float dx = o.x - me.x, dy = o.y - me.y, dz = o.z - me.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const bool stj = (__float_as_int(o.w) & 1) != 0;
            const float rl2 = (k & 1) ? (stj ? rO_st : rO_gh) : (stj ? rE_st : rE_gh);
            if (r2 < rl2) m16 |= 1u << k;
          }
          hits |= (unsigned long long)m16 << c0;
        }
        hits &= ~(1ull << (lane + 16 - kb));   // the bead itself
        total = __popcll(hits);
        for (; hits && cnt < a.cap; hits &= hits - 1ull) {
          const int c = __ffsll((long long)hits) - 1;
          int ent = ent_make((int)g0 - 16 + kb + c, 0, 0, 0);
          if constexpr (sizeof(Real) == 8) {
            const int ow = __float_as_int(wb[c + (c >> 4)].w);
            ent = ent_make((int)g0 - 16 + kb + c, ((ow >> 1) & 3) - ((mew >> 1) & 3), ((ow >> 3) & 3) - ((mew >> 3) & 3),
                           ((ow >> 5) & 3) - ((mew >> 5) & 3));
          }
          list[cnt++] = ent;
        }
      } else {
        for (int c = 0; c < 48; ++c) {
          const float4 o = wb[c + (c >> 4)];
          const int ow = __float_as_int(o.w);
          const int j = (int)g0 - 16 + kb + c;
          if (!(ow & CL_VALID) || j == g || (ow >> 8) != (mew >> 8)) continue;
          float d[3] = {o.x - me.x, o.y - me.y, o.z - me.z};
          int sc3[3];
          for (int q = 0; q < 3; ++q) {
            const float s = -rintf(d[q] * a.invLf[q]);
            d[q] = fmaf(s, a.Lf[q], d[q]);
            sc3[q] = (int)s;
          }
          const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          const float rl2 = list_r2(a.c, ((g ^ j) & 1) != 0, st_g && (ow & 1));
          if (r2 < rl2) cl_append(list, cnt, total, a.cap, ent_make(j, sc3[0], sc3[1], sc3[2]));
        }
      }
    }

    // partners in segments two or more away, through the segment grid: the
    // 54 ranges flattened over the lanes (range q < 27: cell q of segment 2t,
    // else cell q - 27 of segment 2t + 1); grid items of other molecules (a
    // shared hash entry, or a periodic box of several molecules) are skipped
    // by their first slot
    {
      unsigned len[2] = {re[0] - rb[0], re[1] - rb[1]}, off[2], tot[2];
      for (int h = 0; h < 2; ++h) {
        unsigned incl = len[h];
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        tot[h] = __shfl_sync(0xffffffffu, incl, 31);
        off[h] = incl - len[h];
      }
      if (lane < 27) {
        s_rb[w][lane] = rb[0];
        s_ro[w][lane] = off[0];
        s_rb[w][27 + lane] = rb[1];
        s_ro[w][27 + lane] = tot[0] + off[1];
      }
      __syncwarp();
      const unsigned M = tot[0] + tot[1];
      for (unsigned m0 = 0; m0 < M; m0 += 32) {
        const unsigned m = m0 + lane;
        bool acc = false;
        int ir = 0, hq = 0;
        float4 it = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (m < M) {
          int lo = 0, hi = 53;   // the last range whose flattened offset is at or before m
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_ro[w][mid] <= m) lo = mid; else hi = mid - 1;
          }
          const unsigned e = s_rb[w][lo] + (m - s_ro[w][lo]);
          hq = lo >= 27;
          ir = a.key[e];
          it = a.cent[e];
          const int64_t j0 = ir & ENT_JMASK, js = j0 / SEG_W, s = sA + hq;
          const int64_t lo_h = hq ? slo[1] : slo[0], hi_h = hq ? shi[1] : shi[0];
          if (j0 >= lo_h && j0 < hi_h && (js > s + 1 || js < s - 1)) acc = cl_spheres_meet(a, hq ? sc[1] : sc[0], it);
        }
        // up to two accepted items of each segment at a time (item slot
        // 2h + k: the k-th of segment 2t + h): their beads are staged in the
        // window buffer, one load each and all in flight together, unwrapped
        // around the segment's centre; only the beads within the segment's
        // radius + reach of its centre are kept (compacted), and only the
        // lanes whose bead lies within the item's radius + reach of the
        // item's centre test them, both halves at once.  Any pair within list
        // range passes both filters, and both unwrapped positions lie within
        // 3 radii + 2 reaches of the centre, far below half the box.
        unsigned bal[2] = {__ballot_sync(0xffffffffu, acc && hq == 0), __ballot_sync(0xffffffffu, acc && hq == 1)};
        while (bal[0] | bal[1]) {
          int nh[2];
          for (int h = 0; h < 2; ++h) {
            const int rank = __popc(bal[h] & ((1u << lane) - 1u));
            if (((bal[h] >> lane) & 1u) && rank < 2) {
              s_gi[w][2 * h + rank] = ir;
              s_gc[w][2 * h + rank] = it;
            }
            unsigned rest = bal[h];
            for (int q = 0; q < 2 && rest; ++q) rest &= rest - 1u;
            nh[h] = __popc(bal[h]) - __popc(rest);
            bal[h] = rest;
          }
          __syncwarp();
          unsigned keep[2];
          for (int r = 0; r < 2; ++r) {   // staging round r holds item slots 2r (lanes 0-15) and 2r + 1
            const int q = 2 * r + (lane >> 4), b = lane & 15;
            const float4 c = sc[r];        // item slots 2r, 2r + 1 belong to segment 2t + r
            bool pass = false;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if ((q & 1) < nh[r]) {
              const int gq = s_gi[w][q];
              const int j = (gq & ENT_JMASK) + b;
              if (b <= (int)((unsigned)gq >> ENT_J_BITS)) {
                const float4 pj = a.wpos[j];
                float pp[3] = {pj.x, pj.y, pj.z};
                const float cc[3] = {c.x, c.y, c.z};
                int code = (a.topo[j] & F_STERIC) ? 1 : 0;
                float r2 = 0.0f;
                for (int k = 0; k < 3; ++k) {
                  const float tq = rintf((cc[k] - pp[k]) * a.invLf[k]);
                  pp[k] = fmaf(tq, a.Lf[k], pp[k]);
                  code |= ((int)tq + 1) << (1 + 2 * k);
                  r2 = fmaf(pp[k] - cc[k], pp[k] - cc[k], r2);
                }
                const float reach = c.w + a.sg_reach;
                pass = r2 < reach * reach;
                v = make_float4(pp[0], pp[1], pp[2], __int_as_float(code | (b << 8)));
              }
            }
            keep[r] = __ballot_sync(0xffffffffu, pass);
            const unsigned mine16 = (keep[r] >> (lane & 16)) & 0xffffu;
            if (pass) win[16 * q + __popc(mine16 & ((1u << b) - 1u))] = v;
          }
          __syncwarp();
          const int hme = lane >> 4, nme = hme ? nh[1] : nh[0];
          const float4 cme = hme ? sc[1] : sc[0];
          float pi[3] = {mp.x, mp.y, mp.z};
          int ti[3];
          {
            const float cc[3] = {cme.x, cme.y, cme.z};
            for (int k = 0; k < 3; ++k) {
              const float tq = rintf((cc[k] - pi[k]) * a.invLf[k]);
              pi[k] = fmaf(tq, a.Lf[k], pi[k]);
              ti[k] = (int)tq;
            }
          }
          for (int k = 0; k < 2; ++k) {
            if (!in || k >= nme) continue;
            const int q = 2 * hme + k;
            const unsigned kq = (keep[hme] >> (16 * k)) & 0xffffu;   // round hme, half k
            const float4 cj = s_gc[w][q];
            float r2c = 0.0f;
            {
              const float cc[3] = {cj.x, cj.y, cj.z};
              for (int k3 = 0; k3 < 3; ++k3) {
                float d = cc[k3] - pi[k3];
                d = fmaf(-rintf(d * a.invLf[k3]), a.Lf[k3], d);
                r2c = fmaf(d, d, r2c);
              }
            }
            const float reach = cj.w + a.sg_reach;
            if (!(r2c < reach * reach)) continue;
            const int j0 = s_gi[w][q] & ENT_JMASK, nk = __popc(kq);
            for (int b = 0; b < nk; ++b) {
              const float4 o = win[16 * q + b];
              const int ow = __float_as_int(o.w);
              const int j = j0 + (ow >> 8);
              const float dx = o.x - pi[0], dy = o.y - pi[1], dz = o.z - pi[2];
              const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
              const float rl2 = list_r2(a.c, ((g ^ j) & 1) != 0, st_g && (ow & 1));
              if (r2 < rl2) {
                int ent = ent_make(j, 0, 0, 0);
                if constexpr (sizeof(Real) == 8)
                  ent = ent_make(j, ((ow >> 1) & 3) - 1 - ti[0], ((ow >> 3) & 3) - 1 - ti[1], ((ow >> 5) & 3) - 1 - ti[2]);
                cl_append(list, cnt, total, a.cap, ent);
              }
            }
          }
          __syncwarp();
        }
      }
    }
    // a wide segment: each of its beads queries its own 27 cells
    for (int h = 0; h < 2; ++h) {
      if (!(in && (lane >> 4) == h && (h == 0 || hasB) && sc[h].w < 0.0f)) continue;
      const int64_t s = sA + h;
      int ci[3];
      seg_cell(a, mp.x, mp.y, mp.z, ci);
      const int pmol = __float_as_int(mp.w);
      const int64_t plo = a.n_mol > 1 ? 2 * a.mol_off[pmol] : 0, phi = a.n_mol > 1 ? 2 * a.mol_off[pmol + 1] : a.n;
      const float4 pt = make_float4(mp.x, mp.y, mp.z, 0.0f);
      for (int q = 0; q < 27; ++q) {
        const unsigned k = seg_key(a, pmol, ci, q);
        bool dup = false;
        if (!a.periodic)
          for (int o = 0; o < q; ++o) dup = dup || seg_key(a, pmol, ci, o) == k;
        if (dup) continue;
        const unsigned e1 = a.start[k + 1];
        for (unsigned e = a.start[k]; e < e1; ++e) {
          const int ir = a.key[e];
          const int64_t j0 = ir & ENT_JMASK, js = j0 / SEG_W;
          if (j0 < plo || j0 >= phi || (js <= s + 1 && js >= s - 1)) continue;
          if (cl_spheres_meet(a, pt, a.cent[e])) cl_item_pairs(a, g, mp, st_g, ir, list, cnt, total);
        }
      }
    }

    if (in) {
      if (total > a.cap) fl |= B_EOVF;
      for (int q = 0; q < cnt; ++q) a.nbr[(size_t)q * a.ns + g] = list[q];
      a.ncnt[g] = cnt;
    }
    if (a.evl) {   // pair halving of this tile (mixed precision)
      int e8[HALF_NMAX];
#pragma unroll
      for (int q = 0; q < HALF_NMAX; ++q) e8[q] = q < cnt ? list[q] : 0;
      pack_tile(a, t, lane, in ? cnt : 0, e8, s_tm[w], s_base[w]);
    }
    __syncwarp();   // the window and the range table are rewritten for the next tile
  }
  if (fl) atomicOr(a.err, fl & B_ERRMASK);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.rebuild = 0;
    *a.nrebuild += 1;
  }
}

}  // namespace dsdna
