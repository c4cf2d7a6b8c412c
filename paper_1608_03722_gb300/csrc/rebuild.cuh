// rebuild.cuh -- cell table and neighbour-list rebuild of the dsDNA engine:
// binning, block scan, scatter to cell order and the typed list build, run as
// five ordinary kernels between persistent step launches.  Included by
// kern_mixed.cu (Real = float) and kern_fp64.cu (Real = double).
#pragma once
#include "engine.cuh"

namespace dsdna {

// ---------------------------------------------------------------- cell hash
__device__ __forceinline__ unsigned compact3(unsigned v) {  // every third bit -> 10 bits
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030C30C3u;
  v = (v | (v >> 4)) & 0x0300F00Fu;
  v = (v | (v >> 8)) & 0x030000FFu;
  v = (v | (v >> 16)) & 0x000003FFu;
  return v;
}

__device__ __forceinline__ unsigned spread3(unsigned v) {   // 10 bits -> every third bit
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ unsigned hash_block(int mol, int bx, int cy, int cz) {
  unsigned h = (unsigned)bx * 0x8da6b343u ^ (unsigned)cy * 0xd8163841u ^ (unsigned)cz * 0xcb1ab31fu ^
               (unsigned)mol * 0x9E3779B1u;
  h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
  return h;
}

// The x-blocks of the hashed table start at cell 4 (mod 8): a molecule held
// along an axis through the origin (the anchored single-molecule set-ups of
// Sec. 4) spans x-cells -1 and 0 and so stays inside one block, whose rows
// are then one range each.
constexpr int HASH_X_OFF = 4;

// Squared list radius of a bead pair by type (Sec. 2, reading A1): two steric
// beads (either strand) at the steric radius, any other pair across strands
// at the cross-strand radius, a ghost and a bead of its own strand not at all
// (negative).  With the cross-strand steric reading off, rl_cs2 = rl_cr2.
template <class Real>
__device__ __forceinline__ float list_r2(const Coef<Real>& c, bool cross, bool both_steric) {
  return cross ? (both_steric ? c.rl_cs2 : c.rl_cr2) : (both_steric ? c.rl_ss2 : -1.0f);
}

template <class Real>
__device__ __forceinline__ unsigned cell_key(const KArgs<Real>& a, int mol, int cx, int cy, int cz) {
  if (a.table == TABLE_LINEAR) return (unsigned)cx + (unsigned)a.nc[0] * ((unsigned)cy + (unsigned)a.nc[1] * (unsigned)cz);
  if (a.table == TABLE_MORTON) {   // small periodic box: Morton index of the wrapped cell (no collisions)
    return (spread3((unsigned)cx) | (spread3((unsigned)cy) << 1) | (spread3((unsigned)cz) << 2)) & (a.H - 1u);
  }
  // open box: (molecule, y, z, x / 8) hashed to a bucket of 8 table entries
  // holding the 8 x-consecutive cells of that block, so a row of three
  // x-neighbour cells is one range of the sorted beads (two across a block
  // edge).  Distinct blocks may share a bucket; the list build skips a range
  // it has already walked.
  const int xs = cx + HASH_X_OFF;
  return (hash_block(mol, xs >> 3, cy, cz) & ((a.H >> 3) - 1u)) << 3 | (unsigned)(xs & 7);
}

template <class Real>
__device__ __forceinline__ void bead_position_f(const KArgs<Real>& a, int cur, int64_t g, float* b) {
  const float h = (float)a.c.h;
  if constexpr (sizeof(Real) == 4) {
    const float4 u = a.U[(size_t)cur * a.ns + g];
    b[0] = d2f_bits(a.X[g]) - h * u.x;
    b[1] = d2f_bits(a.X[a.ns + g]) - h * u.y;
    b[2] = d2f_bits(a.X[2 * a.ns + g]) - h * u.z;
  } else {
    const double* X = a.X + (size_t)cur * 3 * a.ns;
    const double* u = a.ud + (size_t)cur * 3 * a.ns;
    for (int c = 0; c < 3; ++c) b[c] = (float)(X[c * a.ns + g] - (double)h * u[c * a.ns + g]);
  }
}

template <class Real>
__device__ __forceinline__ void bead_position(const KArgs<Real>& a, int cur, int64_t g, double* b) {
  const double h = (double)a.c.h;
  if constexpr (sizeof(Real) == 4) {
    const float4 u = a.U[(size_t)cur * a.ns + g];
    b[0] = a.X[g] - h * (double)u.x;
    b[1] = a.X[a.ns + g] - h * (double)u.y;
    b[2] = a.X[2 * a.ns + g] - h * (double)u.z;
  } else {
    const double* X = a.X + (size_t)cur * 3 * a.ns;
    const double* u = a.ud + (size_t)cur * 3 * a.ns;
    for (int c = 0; c < 3; ++c) b[c] = X[c * a.ns + g] - h * u[c * a.ns + g];
  }
}

// Per-bead part of R1: the wrapped FP32 bead position (to wpos, with the
// molecule), the periodic image word and the build-time mirror of the
// rebuild trigger.  Returns the wrapped position in pw and the molecule.
template <class Real>
__device__ __forceinline__ int bin_bead(const KArgs<Real>& a, int cur, int64_t g, unsigned& fl, float* pw) {
  // Binning in FP32: any integer image w with pw = b - w L is exact for the
  // force path (it only uses integer image differences), so rounding here
  // moves a bead by at most a few 1e-5 nm inside the 0.01 nm list margin.
  float b[3];
  bead_position_f(a, cur, g, b);
  int w[3] = {0, 0, 0};
  for (int c = 0; c < 3; ++c) {
    float x = b[c];
    if (a.periodic) {
      const float q = floorf(x * a.invLf[c]);
      w[c] = (int)q;
      x = fmaf(-q, a.Lf[c], x);
      if (w[c] > 511 || w[c] < -512) fl |= B_EIMG;
    }
    pw[c] = x;
  }
  // the image word (three signed 10-bit fields) also carries the bead's steric
  // flag in bit 30, for the pair typing of the force loop
  const int tp = a.topo[g];
  const int packed = (w[0] & 0x3ff) | ((w[1] & 0x3ff) << 10) | ((w[2] & 0x3ff) << 20) | ((tp & F_STERIC) << IMG_STERIC_SHIFT);
  const int mol = tp >> MOL_SHIFT;
  a.wpos[g] = make_float4(pw[0], pw[1], pw[2], __int_as_float(mol));
  if constexpr (sizeof(Real) == 8) a.img[g] = packed;   // mixed precision keeps it in Kw.w
  // build-time bead position on the fixed-point grid, for the rebuild trigger
  const float h = (float)a.c.h;
  if constexpr (sizeof(Real) == 4) {
    int4 kw = a.Kw[(size_t)cur * a.ns + g];
    const float4 u = a.U[(size_t)cur * a.ns + g];
    a.kref[g] = kw.x + bead_off(h * u.x, a.fixSf[0]);
    a.kref[a.ns + g] = kw.y + bead_off(h * u.y, a.fixSf[1]);
    a.kref[2 * a.ns + g] = kw.z + bead_off(h * u.z, a.fixSf[2]);
    kw.w = packed;
    a.Kw[(size_t)cur * a.ns + g] = kw;
  } else {
    const double* X = a.X + (size_t)cur * 3 * a.ns;
    const double* u = a.ud + (size_t)cur * 3 * a.ns;
    for (int c = 0; c < 3; ++c)
      a.kref[c * a.ns + g] = fixs(X[c * a.ns + g], a.fixS[c]) + bead_off(h * (float)u[c * a.ns + g], a.fixSf[c]);
  }
  return mol;
}

// R1: bin beads, record images and the build-time mirror.
template <class Real>
__device__ void rebuild_bin(const KArgs<Real>& a, int cur, unsigned& fl) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.n; g += stride) {
    float pw[3];
    const int mol = bin_bead(a, cur, g, fl, pw);
    int ci[3];
    for (int c = 0; c < 3; ++c) {
      const int k = (int)floorf(pw[c] * a.invcellh[c]);
      ci[c] = a.periodic ? (k >= a.nc[c] ? a.nc[c] - 1 : (k < 0 ? 0 : k)) : k;
    }
    const unsigned k = cell_key(a, mol, ci[0], ci[1], ci[2]);
    a.key[g] = (int)k;
    atomicAdd(&a.cnt[k], 1u);
  }
}

// block-wide exclusive scan of one value per thread (blockDim multiple of 32)
__device__ __forceinline__ unsigned block_exscan(unsigned v, unsigned* s_warp, unsigned* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned t = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) s_warp[lane] = t;
  }
  __syncthreads();
  const unsigned before = (wid > 0 ? s_warp[wid - 1] : 0u) + x - v;
  *total = s_warp[nw - 1];
  __syncthreads();
  return before;
}

// R2a: per-block sums of the count table.  The table is split into chunks
// of whole 2048-entry tiles (256 threads x 8 entries, two 16-byte loads each).
constexpr unsigned SCAN_ITEMS = 8;

__device__ __forceinline__ void scan_chunk(unsigned H, unsigned* lo, unsigned* hi) {
  const unsigned tile = blockDim.x * SCAN_ITEMS;
  const unsigned ntile = (H + tile - 1) / tile;
  const unsigned per = (ntile + gridDim.x - 1) / gridDim.x;
  *lo = min(H, blockIdx.x * per * tile);
  *hi = min(H, (blockIdx.x + 1) * per * tile);
}

template <class Real>
__device__ void rebuild_scan_a(const KArgs<Real>& a, unsigned* s_red) {
  unsigned lo, hi;
  scan_chunk(a.H, &lo, &hi);
  unsigned s = 0;
  for (unsigned i = lo + threadIdx.x * SCAN_ITEMS; i < hi; i += blockDim.x * SCAN_ITEMS) {
    const uint4 x = *reinterpret_cast<const uint4*>(a.cnt + i);
    const uint4 y = *reinterpret_cast<const uint4*>(a.cnt + i + 4);
    s += x.x + x.y + x.z + x.w + y.x + y.y + y.z + y.w;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    a.bsum[blockIdx.x] = t;
  }
  __syncthreads();
}

// R2b: exclusive scan -> start[]
template <class Real>
__device__ void rebuild_scan_b(const KArgs<Real>& a, unsigned* s_red) {
  unsigned lo, hi;
  scan_chunk(a.H, &lo, &hi);
  unsigned pre = 0;
  for (unsigned b = threadIdx.x; b < blockIdx.x; b += blockDim.x) pre += a.bsum[b];
  for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = pre;
  __syncthreads();
  unsigned carry = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) carry += s_red[w];
  __syncthreads();
  for (unsigned base = lo; base < hi; base += blockDim.x * SCAN_ITEMS) {
    const unsigned i = base + threadIdx.x * SCAN_ITEMS;
    uint4 x = make_uint4(0, 0, 0, 0), y = make_uint4(0, 0, 0, 0);
    if (i < hi) {
      x = *reinterpret_cast<const uint4*>(a.cnt + i);
      y = *reinterpret_cast<const uint4*>(a.cnt + i + 4);
    }
    const unsigned v = x.x + x.y + x.z + x.w + y.x + y.y + y.z + y.w;
    unsigned tot;
    unsigned r = carry + block_exscan(v, s_red, &tot);
    if (i < hi) {
      uint4 o1, o2;
      o1.x = r; r += x.x; o1.y = r; r += x.y; o1.z = r; r += x.z; o1.w = r; r += x.w;
      o2.x = r; r += y.x; o2.y = r; r += y.y; o2.z = r; r += y.z; o2.w = r;
      *reinterpret_cast<uint4*>(a.start + i) = o1;
      *reinterpret_cast<uint4*>(a.start + i + 4) = o2;
    }
    carry += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) a.start[a.H] = (unsigned)a.n;
}

// R3: scatter beads into cell order (Morton order for a periodic box);
// the count table returns to zero.
template <class Real>
__device__ void rebuild_scatter(const KArgs<Real>& a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.n; g += stride) {
    const unsigned k = (unsigned)a.key[g];
    const unsigned slot = a.start[k] + atomicSub(&a.cnt[k], 1u) - 1u;
    const float4 w = a.wpos[g];
    const int st = (a.topo[g] & F_STERIC) ? (1 << NBR_J_BITS) : 0;
    a.cent[slot] = make_float4(w.x, w.y, w.z, __int_as_float((int)g | st));
  }
}

// R4: typed full neighbour list of every bead, sorted by partner slot.
// Pairs (Sec. 2, reading A1): opposite strands always (sigma_cross); same
// strand only steric-steric (sigma_ss); same molecule only.  Beads are taken
// in cell order (Morton order in a periodic box).  The 27 neighbour cells are
// read one 3x3 layer at a time so that nine range loads are in flight at once.
template <class Real, int CAPMAX>
__device__ void list_one_bead(const KArgs<Real>& a, int64_t t, unsigned& fl) {
  const int JMASK = (1 << NBR_J_BITS) - 1;
  const bool dedupe = a.table != TABLE_LINEAR;
  {
    const float4 me = a.cent[t];
    const int gw = __float_as_int(me.w);
    const int g = gw & JMASK;
    const bool st_g = (gw >> NBR_J_BITS) & 1;
    const int mol = a.n_mol > 1 ? __float_as_int(a.wpos[g].w) : 0;
    int ci[3];
    const float p[3] = {me.x, me.y, me.z};
    for (int c = 0; c < 3; ++c) {
      int k = (int)floorf(p[c] * a.invcellh[c]);
      if (a.periodic) k = k >= a.nc[c] ? a.nc[c] - 1 : (k < 0 ? 0 : k);
      ci[c] = k;
    }
    int list[CAPMAX];
    int cnt = 0, total = 0;
    unsigned seen[27];
    int nseen = 0;
    for (int dz = -1; dz <= 1; ++dz) {
      unsigned kk[9], b0[9], b1[9];
      bool use[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        int c3[3] = {ci[0] + (q % 3) - 1, ci[1] + (q / 3) - 1, ci[2] + dz};
        if (a.periodic)
          for (int c = 0; c < 3; ++c) c3[c] = c3[c] < 0 ? c3[c] + a.nc[c] : (c3[c] >= a.nc[c] ? c3[c] - a.nc[c] : c3[c]);
        kk[q] = cell_key(a, mol, c3[0], c3[1], c3[2]);
        use[q] = true;
        if (dedupe) {
          for (int r = 0; r < nseen; ++r) use[q] = use[q] && (seen[r] != kk[q]);
          if (use[q]) seen[nseen++] = kk[q];
        }
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        b0[q] = use[q] ? a.start[kk[q]] : 0u;
        b1[q] = use[q] ? a.start[kk[q] + 1] : 0u;
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        for (unsigned e = b0[q]; e < b1[q]; ++e) {
          const float4 o = a.cent[e];
          const int jw = __float_as_int(o.w);
          const int j = jw & JMASK;
          if (j == g) continue;
          float d[3] = {o.x - p[0], o.y - p[1], o.z - p[2]};
          int sc[3] = {0, 0, 0};
          if (a.periodic)
            for (int c = 0; c < 3; ++c) {
              const float s = -rintf(d[c] * a.invLf[c]);
              d[c] = fmaf(s, a.Lf[c], d[c]);
              sc[c] = (int)s;
            }
          const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          const float rl2 = list_r2(a.c, ((g ^ j) & 1) != 0, st_g && ((jw >> NBR_J_BITS) & 1));
          if (r2 >= rl2) continue;
          if (a.n_mol > 1 && __float_as_int(a.wpos[j].w) != mol) continue;
          const int ent = ent_make(j, sc[0], sc[1], sc[2]);
          ++total;
          if (cnt < a.cap) {   // insertion by partner slot keeps the force sum order fixed
            int qq = cnt++;
            while (qq > 0 && (list[qq - 1] & ENT_JMASK) > j) { list[qq] = list[qq - 1]; --qq; }
            list[qq] = ent;
          }
        }
      }
    }
    if (total > a.cap) fl |= B_EOVF;
    for (int q = 0; q < cnt; ++q) a.nbr[(size_t)q * a.ns + g] = list[q];
    a.ncnt[g] = cnt;
  }
}

// Typed pair test of bead (p, g) against candidate o; appends to the sorted list.
template <class Real, int CAPMAX>
__device__ __forceinline__ void consider(const KArgs<Real>& a, const float* p, int g, bool st_g, int mol, float4 o,
                                         int* list, int& cnt, int& total) {
  const int JMASK = (1 << NBR_J_BITS) - 1;
  const int jw = __float_as_int(o.w);
  const int j = jw & JMASK;
  if (j == g) return;
  float d[3] = {o.x - p[0], o.y - p[1], o.z - p[2]};
  int sc[3] = {0, 0, 0};
  if (a.periodic)
    for (int c = 0; c < 3; ++c) {
      const float s = -rintf(d[c] * a.invLf[c]);
      d[c] = fmaf(s, a.Lf[c], d[c]);
      sc[c] = (int)s;
    }
  const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const float rl2 = list_r2(a.c, ((g ^ j) & 1) != 0, st_g && ((jw >> NBR_J_BITS) & 1));
  if (r2 >= rl2) return;
  if (a.n_mol > 1 && __float_as_int(a.wpos[j].w) != mol) return;
  const int ent = ent_make(j, sc[0], sc[1], sc[2]);
  ++total;
  if (cnt < a.cap) {   // insertion by partner slot keeps the force sum order fixed
    int q = cnt++;
    while (q > 0 && (list[q - 1] & ENT_JMASK) > j) { list[q] = list[q - 1]; --q; }
    list[q] = ent;
  }
}

// R4 (warp per table entry): the beads of one cell share one neighbourhood.
// Lanes 0..26 read the ranges of the 27 neighbour cells at once, the warp
// stages their beads in shared memory in tiles of LIST_TILE, and all 32 lanes
// share the (bead, candidate) pair tests of the cell against the tile.  Hits
// go to per-bead shared buffers; a cell holds about three beads, so the warp
// buffers the beads of consecutive cells and, once LIST_NB are waiting, one
// lane per bead sorts its entries by partner slot and writes its list.
// Entries whose beads belong to several cells (hash collisions) take the
// per-bead path.
constexpr int LIST_TILE = 128;
constexpr int LIST_WARPS = 4;    // warps per CTA of the list kernel (static shared memory < 48 KB)
constexpr int LIST_NB = 32;      // beads buffered per warp before their lists are sorted and written
constexpr int LIST_CAP = 32;

// typed pair test; returns the list entry (ent_make), or -1
template <class Real>
__device__ __forceinline__ int pair_entry(const KArgs<Real>& a, float4 me, float4 o, int mol) {
  const int JMASK = (1 << NBR_J_BITS) - 1;
  const int gw = __float_as_int(me.w), jw = __float_as_int(o.w);
  const int g = gw & JMASK, j = jw & JMASK;
  if (j == g) return -1;
  const float rl2 = list_r2(a.c, ((g ^ j) & 1) != 0, ((gw & jw) >> NBR_J_BITS) & 1);
  if (rl2 < 0.0f) return -1;
  float d[3] = {o.x - me.x, o.y - me.y, o.z - me.z};
  int sc[3] = {0, 0, 0};
  if (a.periodic) {
    for (int c = 0; c < 3; ++c) {
      const float s = -rintf(d[c] * a.invLf[c]);
      d[c] = fmaf(s, a.Lf[c], d[c]);
      sc[c] = (int)s;
    }
  }
  if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] >= rl2) return -1;
  if (a.n_mol > 1 && __float_as_int(a.wpos[j].w) != mol) return -1;
  return ent_make(j, sc[0], sc[1], sc[2]);
}

template <class Real, int CAPMAX>
__device__ void rebuild_list_warps(const KArgs<Real>& a, unsigned& fl) {
  __shared__ float4 tile[LIST_WARPS][LIST_TILE];
  __shared__ float4 cpos[LIST_WARPS][LIST_NB];     // buffered beads (cell-sorted positions)
  __shared__ int scount[LIST_WARPS][LIST_NB];
  __shared__ int sent[LIST_WARPS][LIST_NB][LIST_CAP];
  __shared__ unsigned rb[LIST_WARPS][28], roff[LIST_WARPS][28];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int JMASK = (1 << NBR_J_BITS) - 1;
  const bool dedupe = true;   // hash or small Morton table: a key may repeat among the 27
  const unsigned nwarps = gridDim.x * (blockDim.x >> 5);
  const unsigned wid = blockIdx.x * (blockDim.x >> 5) + w;
  int nb = 0;   // beads buffered by this warp (warp-uniform)
  // one lane per buffered bead: order its entries by partner slot (the force
  // sum order is then fixed) and write its list
  auto flush = [&]() {
    __syncwarp();
    if (lane < nb) {
      const int g = __float_as_int(cpos[w][lane].w) & JMASK;
      const int total = scount[w][lane];
      const int cnt = min(total, a.cap);
      if (total > a.cap) fl |= B_EOVF;
      int* e = sent[w][lane];
      for (int x = 1; x < cnt; ++x) {
        const int v = e[x];
        int y = x;
        while (y > 0 && (e[y - 1] & ENT_JMASK) > (v & ENT_JMASK)) { e[y] = e[y - 1]; --y; }
        e[y] = v;
      }
      for (int q = 0; q < cnt; ++q) a.nbr[(size_t)q * a.ns + g] = e[q];
      a.ncnt[g] = cnt;
    }
    nb = 0;
    __syncwarp();
  };
  for (unsigned kb = wid * 32u; kb < a.H; kb += nwarps * 32u) {
    const unsigned k0 = kb + lane;
    const unsigned s0 = k0 < a.H ? a.start[k0] : 0u, s1 = k0 < a.H ? a.start[k0 + 1] : 0u;
    unsigned busy = __ballot_sync(0xffffffffu, s1 > s0);
    while (busy) {
      const int src = __ffs(busy) - 1;
      busy &= busy - 1;
      const unsigned beg = __shfl_sync(0xffffffffu, s0, src), end = __shfl_sync(0xffffffffu, s1, src);
      int c0[3];
      int mol0 = 0;
      bool same = true;
      if (a.table == TABLE_MORTON && a.n_mol == 1) {
        // one molecule in a periodic box: the table entry is exactly one cell
        const unsigned kc = kb + (unsigned)src;
        c0[0] = (int)compact3(kc); c0[1] = (int)compact3(kc >> 1); c0[2] = (int)compact3(kc >> 2);
      } else {
      // the cell of the entry's first bead; all beads must share it
      const float4 f0 = a.cent[beg];
      for (int c = 0; c < 3; ++c) {
        const float q = c == 0 ? f0.x : (c == 1 ? f0.y : f0.z);
        int kk = (int)floorf(q * a.invcellh[c]);
        if (a.periodic) kk = kk >= a.nc[c] ? a.nc[c] - 1 : (kk < 0 ? 0 : kk);
        c0[c] = kk;
      }
      mol0 = a.n_mol > 1 ? __float_as_int(a.wpos[__float_as_int(f0.w) & JMASK].w) : 0;
      for (unsigned t = beg + lane; t < end; t += 32) {
        const float4 f = a.cent[t];
        for (int c = 0; c < 3; ++c) {
          const float q = c == 0 ? f.x : (c == 1 ? f.y : f.z);
          int kk = (int)floorf(q * a.invcellh[c]);
          if (a.periodic) kk = kk >= a.nc[c] ? a.nc[c] - 1 : (kk < 0 ? 0 : kk);
          same = same && kk == c0[c];
        }
        if (a.n_mol > 1) same = same && __float_as_int(a.wpos[__float_as_int(f.w) & JMASK].w) == mol0;
      }
      }
      if (!__all_sync(0xffffffffu, same)) {
        for (unsigned t = beg + lane; t < end; t += 32) list_one_bead<Real, CAPMAX>(a, (int64_t)t, fl);
        continue;
      }
      // ranges of the 27 neighbour cells, one per lane, duplicates (hash) dropped
      unsigned rbeg = 0, rlen = 0, key = 0xffffffffu;
      if (lane < 27) {
        int c3[3] = {c0[0] + (lane % 3) - 1, c0[1] + (lane / 3) % 3 - 1, c0[2] + lane / 9 - 1};
        if (a.periodic)
          for (int c = 0; c < 3; ++c) c3[c] = c3[c] < 0 ? c3[c] + a.nc[c] : (c3[c] >= a.nc[c] ? c3[c] - a.nc[c] : c3[c]);
        key = cell_key(a, mol0, c3[0], c3[1], c3[2]);
      }
      if (dedupe) {
        for (int o = 0; o < 27; ++o) {
          const unsigned ko = __shfl_sync(0xffffffffu, key, o);
          if (o < lane && ko == key) key = 0xffffffffu;
        }
      }
      if (lane < 27 && key != 0xffffffffu) {
        rbeg = a.start[key];
        rlen = a.start[key + 1] - rbeg;
      }
      unsigned incl = rlen;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned M = __shfl_sync(0xffffffffu, incl, 31);
      if (lane < 27) { rb[w][lane] = rbeg; roff[w][lane] = incl - rlen; }
      __syncwarp();
      for (unsigned cb = beg; cb < end;) {
        const int mc = (int)min((unsigned)LIST_NB, end - cb);
        if (nb + mc > LIST_NB) flush();
        if (lane < mc) { cpos[w][nb + lane] = a.cent[cb + lane]; scount[w][nb + lane] = 0; }
        for (unsigned m0 = 0; m0 < M; m0 += LIST_TILE) {
          const unsigned mn = min((unsigned)LIST_TILE, M - m0);
          __syncwarp();
          for (unsigned i = lane; i < mn; i += 32) {
            const unsigned gi = m0 + i;
            int lo = 0, hi = 26;   // last neighbour cell whose staged range starts at or before gi
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (roff[w][mid] <= gi) lo = mid; else hi = mid - 1;
            }
            tile[w][i] = a.cent[rb[w][lo] + (gi - roff[w][lo])];
          }
          __syncwarp();
          // (bead, candidate) pairs of this tile spread over the lanes
          const unsigned P = (unsigned)mc * mn;
          unsigned b = lane / mn, i = lane % mn;
          const unsigned qb = 32u / mn, qi = 32u % mn;
          for (unsigned pp = lane; pp < P; pp += 32) {
            const int ent = pair_entry(a, cpos[w][nb + b], tile[w][i], mol0);
            if (ent != -1) {
              const int q = atomicAdd(&scount[w][nb + b], 1);
              if (q < LIST_CAP) sent[w][nb + b][q] = ent;
            }
            i += qi; b += qb;
            if (i >= mn) { i -= mn; ++b; }
          }
        }
        nb += mc;
        cb += mc;
      }
    }
  }
  flush();
}

// R4 for the linear table (periodic box, >= 3 cells per edge): one lane per
// bead in cell order, so neighbouring lanes share most neighbour cells and
// read them through L1.  A row of three x-consecutive cells is one range of
// the sorted beads (two where the row wraps in x), so each bead walks at most
// 18 (typically 9) ranges, one after the other with the next range's bounds
// loading meanwhile (one merged candidate stream diverged more: 0.37 against
// 0.31 ms per rebuild at 1 Mbp); every candidate of a range takes the range's
// image, the minimum image within the list radius because every edge has >= 3
// cells of at least that radius.  Hits are inserted in partner-slot order
// into the lane's buffer and then written.
// `list`: this lane's LIST_CAP-entry buffer in shared memory.
template <class Real>
__device__ void rebuild_list_lanes(const KArgs<Real>& a, unsigned& fl, int* list) {
  const int JMASK = (1 << NBR_J_BITS) - 1;
  const int nx = a.nc[0], ny = a.nc[1], nz = a.nc[2];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.n; t += stride) {
    const float4 me = a.cent[t];
    const int gw = __float_as_int(me.w), g = gw & JMASK;
    const bool st_g = (gw >> NBR_J_BITS) & 1;
    const int mol = a.n_mol > 1 ? __float_as_int(a.wpos[g].w) : 0;
    // the bead's cell, computed as the binning did from the same wrapped position
    const int kx = (int)floorf(me.x * a.invcellh[0]), ky = (int)floorf(me.y * a.invcellh[1]),
              kz = (int)floorf(me.z * a.invcellh[2]);
    const int cx = kx >= nx ? nx - 1 : (kx < 0 ? 0 : kx);
    const int cy = ky >= ny ? ny - 1 : (ky < 0 ? 0 : ky);
    const int cz = kz >= nz ? nz - 1 : (kz < 0 ? 0 : kz);
    // candidate ranges: 9 rows (dy, dz) of three x-consecutive cells, a row
    // that wraps in x split in two; range i holds the cells [k0, k1) and its
    // image as ent_make(0, sx, sy, sz)
    const int nparts = (cx == 0 || cx == nx - 1) ? 2 : 1;
    const int nr = 9 * nparts;
    auto range = [&](int i, unsigned& k0, unsigned& k1, int& code) {
      const int row = nparts == 2 ? (i >> 1) : i, part = nparts == 2 ? (i & 1) : 0;
      int y = cy + row % 3 - 1, z = cz + row / 3 - 1;
      const int sy = y < 0 ? -1 : (y >= ny ? 1 : 0);
      const int sz = z < 0 ? -1 : (z >= nz ? 1 : 0);
      y -= sy * ny;
      z -= sz * nz;
      const unsigned rb = (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z);
      int sx = 0;
      if (cx == 0) {                 // cells nx-1 (image -1), then 0 and 1
        k0 = part == 0 ? rb + nx - 1 : rb;
        k1 = part == 0 ? rb + nx : rb + 2;
        sx = part == 0 ? -1 : 0;
      } else if (cx == nx - 1) {     // cells nx-2 and nx-1, then 0 (image +1)
        k0 = part == 0 ? rb + nx - 2 : rb;
        k1 = part == 0 ? rb + nx : rb + 1;
        sx = part == 0 ? 0 : 1;
      } else {
        k0 = rb + cx - 1;
        k1 = rb + cx + 2;
      }
      code = ent_make(0, sx, sy, sz);
    };
    int cnt = 0, total = 0;
    unsigned k0, k1, nu0, ne0;
    int ncode;
    range(0, k0, k1, ncode);
    nu0 = a.start[k0];
    ne0 = a.start[k1];
    for (int i = 0; i < nr; ++i) {
      const unsigned u0 = nu0, e0 = ne0;
      const int code = ncode;
      if (i + 1 < nr) {   // the next range's bounds load while this one is walked
        range(i + 1, k0, k1, ncode);
        nu0 = a.start[k0];
        ne0 = a.start[k1];
      }
      // the bead moved by minus the range's image: candidates are compared as stored
      const float px = me.x - (float)ent_shift(code, 0) * a.Lf[0];
      const float py = me.y - (float)ent_shift(code, 1) * a.Lf[1];
      const float pz = me.z - (float)ent_shift(code, 2) * a.Lf[2];
      for (unsigned u = u0; u < e0; ++u) {
        const float4 o = a.cent[u];
        const int jw = __float_as_int(o.w), j = jw & JMASK;
        const float dx = o.x - px, dy = o.y - py, dz = o.z - pz;
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float rl2 = list_r2(a.c, ((g ^ j) & 1) != 0, st_g && ((jw >> NBR_J_BITS) & 1));
        if (r2 < rl2 && j != g && (a.n_mol == 1 || __float_as_int(a.wpos[j].w) == mol)) {
          ++total;
          if (cnt < a.cap) {   // insertion by partner slot keeps the force sum order fixed
            int q = cnt++;
            while (q > 0 && (list[q - 1] & ENT_JMASK) > j) { list[q] = list[q - 1]; --q; }
            list[q] = j | code;
          }
        }
      }
    }
    if (total > a.cap) fl |= B_EOVF;
    for (int q = 0; q < cnt; ++q) a.nbr[(size_t)q * a.ns + g] = list[q];
    a.ncnt[g] = cnt;
  }
}

// R4 for the hashed table (open box): one lane per bead in table order.  The
// 9 rows (dy, dz) of the bead's neighbourhood are each one range of the
// sorted beads, two where x-1 .. x+1 crosses a block edge.  When two rows of
// the same bead land in the same bucket (two blocks hashed together) the
// later row's range is the same range and is skipped, so no pair is listed
// twice; beads of another block or molecule sharing a bucket fail the
// distance or molecule test.
template <class Real>
__device__ void rebuild_list_lanes_hash(const KArgs<Real>& a, unsigned& fl, int* list) {
  const int JMASK = (1 << NBR_J_BITS) - 1;
  const unsigned bmask = (a.H >> 3) - 1u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // beads in slot (chain) order: neighbouring lanes are neighbours in space,
  // so they share rows and candidates in cache and have similar work (the
  // table order of a hashed table scatters them)
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.n; g += stride) {
    const float4 me = a.wpos[g];
    const bool st_g = (a.topo[g] & F_STERIC) != 0;
    const int mol = __float_as_int(me.w);
    const int cx = (int)floorf(me.x * a.invcellh[0]);
    const int cy = (int)floorf(me.y * a.invcellh[1]);
    const int cz = (int)floorf(me.z * a.invcellh[2]);
    const int lo = cx - 1 + HASH_X_OFF, hi = cx + 1 + HASH_X_OFF;   // block coordinates, as cell_key
    const bool split = (lo >> 3) != (hi >> 3);
    // part 0: cells lo .. (split ? block end : hi) of block lo/8; part 1 (split): cells hi/8*8 .. hi
    const unsigned a0 = (unsigned)(lo & 7), b0 = split ? 7u : (unsigned)(hi & 7), b1 = (unsigned)(hi & 7);
    int cnt = 0, total = 0;
    // every row's bucket first, then all range bounds in flight at once, then
    // the walks (a row whose bucket an earlier row of this bead has is empty)
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      if (part == 1 && !split) break;
      const int bx = part == 0 ? (lo >> 3) : (hi >> 3);
      const unsigned c0 = part == 0 ? a0 : 0u, c1 = part == 0 ? b0 : b1;
      unsigned bk[9], u0[9], u1[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        const unsigned b = hash_block(mol, bx, cy + r % 3 - 1, cz + r / 3 - 1) & bmask;
        bool dup = false;
#pragma unroll
        for (int q = 0; q < r; ++q) dup = dup || bk[q] == b;
        bk[r] = b;
        u0[r] = dup ? 0u : a.start[(b << 3) | c0];
        u1[r] = dup ? 0u : a.start[((b << 3) | c1) + 1u];
      }
      // the 9 ranges as one stream of candidates: a warp runs as many
      // iterations as its busiest lane has candidates (plus 9 range switches),
      // not the sum over rows of each row's longest range
      int r = 0;
      unsigned u = u0[0], e = u1[0];
      for (;;) {
        if (u >= e) {
          if (++r == 9) break;
#pragma unroll
          for (int q = 1; q < 9; ++q)
            if (q == r) { u = u0[q]; e = u1[q]; }
          continue;
        }
        {
          const float4 o = a.cent[u++];
          const int jw = __float_as_int(o.w), j = jw & JMASK;
          const float dx = o.x - me.x, dy = o.y - me.y, dz = o.z - me.z;
          const float r2 = dx * dx + dy * dy + dz * dz;
          const float rl2 = list_r2(a.c, ((g ^ j) & 1) != 0, st_g && ((jw >> NBR_J_BITS) & 1));
          if (r2 < rl2 && j != g && (a.n_mol == 1 || __float_as_int(a.wpos[j].w) == mol)) {
            ++total;
            if (cnt < a.cap) {   // insertion by partner slot keeps the force sum order fixed
              int q = cnt++;
              while (q > 0 && (list[q - 1] & ENT_JMASK) > j) { list[q] = list[q - 1]; --q; }
              list[q] = ent_make(j, 0, 0, 0);
            }
          }
        }
      }
    }
    if (total > a.cap) fl |= B_EOVF;
    for (int q = 0; q < cnt; ++q) a.nbr[(size_t)q * a.ns + g] = list[q];
    a.ncnt[g] = cnt;
  }
}

// ---------------------------------------------------------------- rebuild kernels
// The neighbour-list rebuild runs as five ordinary kernels (full occupancy,
// their own register budgets) between persistent step launches: bin + count,
// block sums, scan, scatter to cell order, list build.
template <class Real>
__global__ void k_rebuild_bin(const KArgs<Real> a) {
  unsigned fl = 0;
  rebuild_bin(a, (int)(*a.step & 1), fl);
  if (fl) atomicOr(a.err, fl & B_ERRMASK);
}
template <class Real>
__global__ void k_rebuild_scan_a(const KArgs<Real> a) {
  __shared__ unsigned s_red[32];
  rebuild_scan_a(a, s_red);
}
template <class Real>
__global__ void k_rebuild_scan_b(const KArgs<Real> a) {
  __shared__ unsigned s_red[32];
  rebuild_scan_b(a, s_red);
}
template <class Real>
__global__ void k_rebuild_scatter(const KArgs<Real> a) { rebuild_scatter(a); }
template <class Real, int CAPMAX>
__global__ void __launch_bounds__(LIST_WARPS * 32) k_rebuild_list(const KArgs<Real> a) {
  unsigned fl = 0;
  rebuild_list_warps<Real, CAPMAX>(a, fl);
  if (fl) atomicOr(a.err, fl & B_ERRMASK);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.rebuild = 0;
    *a.nrebuild += 1;
  }
}

// R5 (mixed precision, pair halving): Newton's third law within a tile.  A
// list pair whose nucleotides lie in the same 32-slot tile of the step
// kernel is evaluated once, by its lower slot, and the other nucleotide
// takes its force negated; a pair across tiles is evaluated by both of its
// nucleotides, each for itself.  Per tile (one warp, one lane per slot): the
// evaluated pairs in order (partner slot | owner lane << 26, lane by lane in
// list order) and, for every list entry, the index of the evaluated pair
// that holds its force (bit 7: negated), eight one-byte codes per slot.  An
// entry is a mirror only when the partner's list holds the pair too (a list
// built from the two sides can disagree at the list radius).  A tile with a
// list longer than HALF_NMAX or more than EVL_CAP evaluated pairs is marked
// -1 and evaluates its list as it stands.  The pair force is antisymmetric
// bit for bit, so both ways give the same force sums.
// Lists are sorted by partner slot, so a list holds its partners below the
// tile, then its partners in the tile (ascending lane), then those above;
// with the in-tile partners as a lane bitmask the position of any in-tile
// pair in either list is a population count.
constexpr int PACK_WARPS = 8;

// Pair halving of tile t by one warp (lane = slot t * 32 + lane): nn list
// entries of this lane, the first HALF_NMAX of them in e8; s_tm and s_base
// are the warp's 32-entry shared scratch.  Every lane of the warp calls it.
template <class Real>
__device__ __forceinline__ void pack_tile(const KArgs<Real>& a, int64_t t, int lane, int nn, const int* e8,
                                          unsigned* s_tm, int* s_base) {
  const int64_t g = t * 32 + lane;
  const bool in = g < a.n;
  const unsigned below = (1u << lane) - 1u;
  if (__any_sync(0xffffffffu, nn > HALF_NMAX)) {
    if (lane == 0) a.tcnt[t] = -1;
    return;
  }
  const int t0 = (int)(t * 32);
  int lo = 0;        // partners below the tile
  unsigned tm = 0;   // partners in the tile
#pragma unroll
  for (int q = 0; q < HALF_NMAX; ++q) {
    const int j = e8[q] & ENT_JMASK;
    if (q < nn) {
      if (j < t0) ++lo;
      else if (j < t0 + 32) tm |= 1u << (j - t0);
    }
  }
  s_tm[lane] = tm;
  __syncwarp();
  // mirrors: in-tile partners below this lane whose list holds this lane too
  unsigned mm = 0;
  for (unsigned c = tm & below; c; c &= c - 1u) {
    const int k = __ffs(c) - 1;
    if ((s_tm[k] >> lane) & 1u) mm |= 1u << k;
  }
  const int ne = nn - __popc(mm);
  int incl = ne;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31), excl = incl - ne;
  if (total > EVL_CAP) {
    if (lane == 0) a.tcnt[t] = -1;
    __syncwarp();
    return;
  }
  // the pair (this lane, partner lane l > this lane) sits at list position
  // lo + popc(tm below l), after every mirror of this lane
  s_base[lane] = excl + lo - __popc(mm);
  __syncwarp();
  unsigned code[2] = {0u, 0u};
  int r = 0;
#pragma unroll
  for (int q = 0; q < HALF_NMAX; ++q) {
    if (q < nn) {
      const int j = e8[q] & ENT_JMASK;
      const int k = j - t0;
      unsigned c;
      if (k >= 0 && k < 32 && ((mm >> k) & 1u)) {   // the partner evaluates it: negated
        c = 0x80u | (unsigned)(s_base[k] + __popc(s_tm[k] & below));
      } else {
        a.evl[t * EVL_CAP + excl + r] = j | (lane << 26);
        c = (unsigned)(excl + r);
        ++r;
      }
      code[q >> 2] |= c << (8 * (q & 3));
    }
  }
  if (in) a.psrc[g] = make_uint2(code[0], code[1]);
  if (lane == 0) a.tcnt[t] = total;
  __syncwarp();
}

template <class Real>
__global__ void __launch_bounds__(PACK_WARPS * 32) k_rebuild_pack(const KArgs<Real> a) {
  __shared__ unsigned s_tm[PACK_WARPS][32];   // in-tile partners of each lane (bit = lane)
  __shared__ int s_base[PACK_WARPS][32];      // first evaluated-pair index + partners below the tile - mirrors
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned ns = (unsigned)a.ns;
  for (int64_t t = (int64_t)blockIdx.x * PACK_WARPS + w; t < a.nseg; t += (int64_t)gridDim.x * PACK_WARPS) {
    const int64_t g = t * 32 + lane;
    const int nn = g < a.n ? a.ncnt[g] : 0;
    int e8[HALF_NMAX];   // the entries, all loads in flight at once
#pragma unroll
    for (int q = 0; q < HALF_NMAX; ++q) e8[q] = q < nn ? a.nbr[(unsigned)q * ns + (unsigned)g] : 0;
    pack_tile(a, t, lane, nn, e8, s_tm[w], s_base[w]);
  }
}

template <class Real>
__global__ void __launch_bounds__(LIST_WARPS * 32) k_rebuild_list_lanes_hash(const KArgs<Real> a) {
  __shared__ int sent[LIST_WARPS][32][LIST_CAP];
  unsigned fl = 0;
  rebuild_list_lanes_hash<Real>(a, fl, sent[threadIdx.x >> 5][threadIdx.x & 31]);
  if (fl) atomicOr(a.err, fl & B_ERRMASK);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.rebuild = 0;
    *a.nrebuild += 1;
  }
}

template <class Real>
__global__ void __launch_bounds__(LIST_WARPS * 32) k_rebuild_list_lanes(const KArgs<Real> a) {
  __shared__ int sent[LIST_WARPS][32][LIST_CAP];
  unsigned fl = 0;
  rebuild_list_lanes<Real>(a, fl, sent[threadIdx.x >> 5][threadIdx.x & 31]);
  if (fl) atomicOr(a.err, fl & B_ERRMASK);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.rebuild = 0;
    *a.nrebuild += 1;
  }
}

}  // namespace dsdna
