// engine_kernels.cuh -- persistent kernel of the dsDNA engine: neighbour-list
// rebuild phases and the fused force + Langevin strip pass.  Included by
// kern_mixed.cu (Real = float) and kern_fp64.cu (Real = double).
#pragma once
#include "engine.cuh"

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
};

template <class Real>
__host__ __device__ inline size_t seg_warp_bytes() {
  size_t b = sizeof(SPos<Real>) * RING + sizeof(int) * RING;
  b = (b + 15) & ~(size_t)15;
  b += sizeof(Real) * (size_t)RING * 15;
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
  return s;
}

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

template <class Real>
__device__ __forceinline__ unsigned cell_key(const KArgs<Real>& a, int mol, int cx, int cy, int cz) {
  if (a.table == TABLE_LINEAR) return (unsigned)cx + (unsigned)a.nc[0] * ((unsigned)cy + (unsigned)a.nc[1] * (unsigned)cz);
  if (a.table == TABLE_MORTON) {   // small periodic box: Morton index of the wrapped cell (no collisions)
    return (spread3((unsigned)cx) | (spread3((unsigned)cy) << 1) | (spread3((unsigned)cz) << 2)) & (a.H - 1u);
  }
  unsigned h = (unsigned)cx * 0x8da6b343u ^ (unsigned)cy * 0xd8163841u ^ (unsigned)cz * 0xcb1ab31fu ^
               (unsigned)mol * 0x9E3779B1u;
  h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
  return h & (a.H - 1u);
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

// R1: bin beads, record images and the build-time mirror.
template <class Real>
__device__ void rebuild_bin(const KArgs<Real>& a, int cur, unsigned& fl) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.n; g += stride) {
    // Binning in FP32: any integer image w with pw = b - w L is exact for the
    // force path (it only uses integer image differences), so rounding here
    // moves a bead by at most a few 1e-5 nm inside the 0.01 nm list margin.
    float b[3];
    bead_position_f(a, cur, g, b);
    int w[3] = {0, 0, 0}, ci[3];
    float pw[3];
    for (int c = 0; c < 3; ++c) {
      float x = b[c];
      if (a.periodic) {
        const float q = floorf(x * a.invLf[c]);
        w[c] = (int)q;
        x = fmaf(-q, a.Lf[c], x);
        pw[c] = x;
        int k = (int)floorf(x * a.invcellh[c]);
        ci[c] = k >= a.nc[c] ? a.nc[c] - 1 : (k < 0 ? 0 : k);
        if (w[c] > 511 || w[c] < -512) fl |= B_EIMG;
      } else {
        pw[c] = x;
        ci[c] = (int)floorf(x * a.invcellh[c]);
      }
    }
    const int packed = (w[0] & 0x3ff) | ((w[1] & 0x3ff) << 10) | ((w[2] & 0x3ff) << 20);
    const int mol = a.topo[g] >> 8;
    const unsigned k = cell_key(a, mol, ci[0], ci[1], ci[2]);
    a.key[g] = (int)k;
    a.wpos[g] = make_float4(pw[0], pw[1], pw[2], __int_as_float(mol));
    a.img[g] = packed;
    atomicAdd(&a.cnt[k], 1u);
    // build-time bead position on the fixed-point grid, for the rebuild trigger
    const float h = (float)a.c.h;
    if constexpr (sizeof(Real) == 4) {
      int4 kw = a.Kw[(size_t)cur * a.ns + g];
      const float4 u = a.U[(size_t)cur * a.ns + g];
      a.kref[g] = kw.x + bead_off(h * u.x);
      a.kref[a.ns + g] = kw.y + bead_off(h * u.y);
      a.kref[2 * a.ns + g] = kw.z + bead_off(h * u.z);
      kw.w = packed;
      a.Kw[(size_t)cur * a.ns + g] = kw;
    } else {
      const double* X = a.X + (size_t)cur * 3 * a.ns;
      const double* u = a.ud + (size_t)cur * 3 * a.ns;
      for (int c = 0; c < 3; ++c) a.kref[c * a.ns + g] = fix32(X[c * a.ns + g]) + bead_off(h * (float)u[c * a.ns + g]);
    }
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
          float rl2;
          if ((g ^ j) & 1) rl2 = a.c.rl_cr2;
          else if (st_g && ((jw >> NBR_J_BITS) & 1)) rl2 = a.c.rl_ss2;
          else continue;
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
  float rl2;
  if ((g ^ j) & 1) rl2 = a.c.rl_cr2;
  else if (st_g && ((jw >> NBR_J_BITS) & 1)) rl2 = a.c.rl_ss2;
  else return;
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
  float rl2;
  if ((g ^ j) & 1) rl2 = a.c.rl_cr2;
  else if (((gw & jw) >> NBR_J_BITS) & 1) rl2 = a.c.rl_ss2;
  else return -1;
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
// 18 (typically 9) ranges as one stream of candidates; every candidate of a
// range takes the range's image, the minimum image within the list radius
// because every edge has >= 3 cells of at least that radius.  Hits are
// inserted in partner-slot order into the lane's buffer and then written.
template <class Real>
__device__ void rebuild_list_lanes(const KArgs<Real>& a, unsigned& fl) {
  __shared__ int sent[LIST_WARPS][32][LIST_CAP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int JMASK = (1 << NBR_J_BITS) - 1;
  int* list = sent[w][lane];
  const int nx = a.nc[0], ny = a.nc[1], nz = a.nc[2];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.n; t += stride) {
    const float4 me = a.cent[t];
    const int gw = __float_as_int(me.w), g = gw & JMASK;
    const bool st_g = (gw >> NBR_J_BITS) & 1;
    const int mol = a.n_mol > 1 ? __float_as_int(a.wpos[g].w) : 0;
    const unsigned key = (unsigned)a.key[g];
    const int cx = (int)(key % (unsigned)nx), cyz = (int)(key / (unsigned)nx);
    const int cy = cyz % ny, cz = cyz / ny;
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
    unsigned k0, k1;
    int code, ncode = 0;
    range(0, k0, k1, code);
    unsigned u = a.start[k0], e = a.start[k1], nu = 0, ne = 0;
    int i = 1;
    if (i < nr) {   // the next range's bounds load while this range is walked
      range(i, k0, k1, ncode);
      nu = a.start[k0];
      ne = a.start[k1];
    }
    // the bead moved by minus the range's image: candidates are compared as stored
    float px = me.x - (float)ent_shift(code, 0) * a.Lf[0];
    float py = me.y - (float)ent_shift(code, 1) * a.Lf[1];
    float pz = me.z - (float)ent_shift(code, 2) * a.Lf[2];
    for (;;) {
      if (u == e) {
        if (i >= nr) break;
        u = nu; e = ne; code = ncode;
        if (++i < nr) {
          range(i, k0, k1, ncode);
          nu = a.start[k0];
          ne = a.start[k1];
        }
        px = me.x - (float)ent_shift(code, 0) * a.Lf[0];
        py = me.y - (float)ent_shift(code, 1) * a.Lf[1];
        pz = me.z - (float)ent_shift(code, 2) * a.Lf[2];
        continue;
      }
      const float4 o = a.cent[u++];
      const int jw = __float_as_int(o.w), j = jw & JMASK;
      const float dx = o.x - px, dy = o.y - py, dz = o.z - pz;
      const float r2 = dx * dx + dy * dy + dz * dz;
      const float rl2 = ((g ^ j) & 1) ? a.c.rl_cr2 : ((st_g && ((jw >> NBR_J_BITS) & 1)) ? a.c.rl_ss2 : -1.0f);
      if (r2 < rl2 && j != g && (a.n_mol == 1 || __float_as_int(a.wpos[j].w) == mol)) {
        ++total;
        if (cnt < a.cap) {   // insertion by partner slot keeps the force sum order fixed
          int q = cnt++;
          while (q > 0 && (list[q - 1] & ENT_JMASK) > j) { list[q] = list[q - 1]; --q; }
          list[q] = j | code;
        }
      }
    }
    if (total > a.cap) fl |= B_EOVF;
    for (int q = 0; q < cnt; ++q) a.nbr[(size_t)q * a.ns + g] = list[q];
    a.ncnt[g] = cnt;
  }
}

// ---------------------------------------------------------------- strip pass
__device__ __forceinline__ int ring(int64_t g) { return (int)(g & (RING - 1)); }

// Bonded terms owned by slot o (ring index ri): the step o -> next along its
// strand (FENE + WCA, Morse, dihedral, planarity) and the bending angle at o.
// Forces go to the owner (cs), its next nucleotide (cn) and the previous
// patch (cp), so each term is evaluated once.
template <class Real>
__device__ __forceinline__ void owner_terms(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t o, unsigned& fl,
                                            Real* E, Real* W) {
  const int ri = ring(o);
  const int f = sm.flg[ri];
  V3<Real> sb{0, 0, 0}, sp{0, 0, 0}, nb{0, 0, 0}, np{0, 0, 0}, pp{0, 0, 0};
  if (f & F_NEXT) {
    const int dir = (o & 1) ? -2 : 2;   // strand A (even slot) runs up, strand B down
    const SPos<Real> so = sm.pos[ri];
    const SPos<Real> sq = sm.pos[ring(o + dir)];
    const Real h = a.c.h;
    const V3<Real> uo = uvec(so), uq = uvec(sq);
    const V3<Real> Rq = rel(so, sq);
    const V3<Real> bo = -h * uo, po = h * uo, bq = Rq - h * uq, pq = Rq + h * uq;
    // FENE + WCA, Morse
    V3<Real> fb = t_fene(a.c, bq - bo, fl, E);
    nb += fb; sb -= fb;
    V3<Real> fm = t_morse(a.c, pq - po, E);
    np += fm; sp -= fm;
    if (W) { vir_add(W, bq - bo, fb); vir_add(W, pq - po, fm); }
    // dihedral A-E-F-B = bead o, patch o, patch q, bead q
    V3<Real> fA, fE, fF, fB;
    t_dihedral(a.c, bo, po, pq, bq, fA, fE, fF, fB, E);
    sb += fA; sp += fE; np += fF; nb += fB;
    if (W) { vir_add(W, bo, fA); vir_add(W, po, fE); vir_add(W, pq, fF); vir_add(W, bq, fB); }
    // planarity: vertex patch q between patch o and bead q
    V3<Real> f1, f2;
    t_planar(a.c, po - pq, bq - pq, f1, f2, E);
    sp += f1; nb += f2; np -= (f1 + f2);
    if (W) { vir_add(W, po, f1); vir_add(W, bq, f2); vir_add(W, pq, -(f1 + f2)); }
    if (f & F_PREV) {
      const SPos<Real> sr = sm.pos[ring(o - dir)];
      const V3<Real> pr = rel(so, sr) + h * uvec(sr);
      V3<Real> g1, g2;
      t_bend(a.c, pr - po, pq - po, g1, g2, E);
      pp += g1; np += g2; sp -= (g1 + g2);
      if (W) { vir_add(W, pr, g1); vir_add(W, pq, g2); vir_add(W, po, -(g1 + g2)); }
    }
  }
  sm.cs[0 * RING + ri] = sb.x; sm.cs[1 * RING + ri] = sb.y; sm.cs[2 * RING + ri] = sb.z;
  sm.cs[3 * RING + ri] = sp.x; sm.cs[4 * RING + ri] = sp.y; sm.cs[5 * RING + ri] = sp.z;
  sm.cn[0 * RING + ri] = nb.x; sm.cn[1 * RING + ri] = nb.y; sm.cn[2 * RING + ri] = nb.z;
  sm.cn[3 * RING + ri] = np.x; sm.cn[4 * RING + ri] = np.y; sm.cn[5 * RING + ri] = np.z;
  sm.cp[0 * RING + ri] = pp.x; sm.cp[1 * RING + ri] = pp.y; sm.cp[2 * RING + ri] = pp.z;
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
    sm.flg[ri] = a.topo[g];
  } else {
    sm.flg[ri] = 0;
  }
}

// Owner o's terms; MODE_ENERGY adds them to its molecule when `count`.
template <class Real, int MODE>
__device__ __forceinline__ void owner_pass(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t o, bool count,
                                           unsigned& fl) {
  if constexpr (MODE == MODE_ENERGY) {
    Real E[NTERMS], W[6];
    for (int k = 0; k < NTERMS; ++k) E[k] = 0;
    for (int k = 0; k < 6; ++k) W[k] = 0;
    owner_terms(a, sm, o, fl, count ? E : nullptr, count ? W : nullptr);
    if (count) flush_energy(a, sm.flg[ring(o)] >> 8, E, W);
  } else {
    owner_terms<Real>(a, sm, o, fl, nullptr, nullptr);
  }
}

template <class Real>
__device__ __forceinline__ void store_state(const KArgs<Real>& a, int nxt, int64_t g, int k0, int k1, int k2,
                                            const double* X, V3<Real> u, int packed) {
  if constexpr (sizeof(Real) == 4) {
    a.Kw[(size_t)nxt * a.ns + g] = make_int4(k0, k1, k2, packed);
    a.U[(size_t)nxt * a.ns + g] = make_float4(u.x, u.y, u.z, 0.0f);
  } else {
    double* Xo = a.X + (size_t)nxt * 3 * a.ns;
    double* uo = a.ud + (size_t)nxt * 3 * a.ns;
    Xo[g] = X[0]; Xo[a.ns + g] = X[1]; Xo[2 * a.ns + g] = X[2];
    uo[g] = u.x; uo[a.ns + g] = u.y; uo[2 * a.ns + g] = u.z;
  }
}

// Forces on nucleotide g from the owner rings, its H-bond and its list
// pairs, then (MODE_STEP) its Langevin update; MODE_FORCES writes the site
// forces, MODE_ENERGY adds its per-nucleotide energies.
template <class Real, int MODE>
__device__ __forceinline__ void nucleotide_pass(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t g, int cur,
                                                int64_t step, unsigned& fl) {
  const int nxt = cur ^ 1;
  Real Eb[NTERMS];
  Real Wb[6];
  if constexpr (MODE == MODE_ENERGY) {
    for (int k = 0; k < NTERMS; ++k) Eb[k] = 0;
    for (int k = 0; k < 6; ++k) Wb[k] = 0;
  }
  {
    const int ri = ring(g);
    const int f = sm.flg[ri];
    const SPos<Real>& me = sm.pos[ri];
    const Real h = a.c.h;
    const V3<Real> um = uvec(me);
    V3<Real> Fb{sm.cs[0 * RING + ri], sm.cs[1 * RING + ri], sm.cs[2 * RING + ri]};
    V3<Real> Fp{sm.cs[3 * RING + ri], sm.cs[4 * RING + ri], sm.cs[5 * RING + ri]};
    const int dir = (g & 1) ? -2 : 2;
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
      const V3<Real> d = rel(me, q) + h * uvec(q) - h * um;   // patch_q - patch_me
      const Real r2 = dot(d, d);
      if (r2 <= a.c.rchb2) {
        Real k2 = (Real)2 * a.c.khb;
        if (a.c.r0hb != (Real)0) k2 *= (Real)1 - a.c.r0hb * rsqrt_(r2);
        Fp += k2 * d;
        if constexpr (MODE == MODE_ENERGY) {
          if ((g & 1) == 0) {
            const Real r = sqrt_(r2);
            const Real rc = sqrt_(a.c.rchb2);
            Eb[2] += a.c.khb * ((r - a.c.r0hb) * (r - a.c.r0hb) - (rc - a.c.r0hb) * (rc - a.c.r0hb));
            vir_add(Wb, d, -(k2 * d));   // force on the partner patch
          }
        }
      }
    }
    // typed WCA pairs (App. A Eq. 11) from the neighbour list
    {
      const int nn = a.ncnt[g];
      const int img_me = a.periodic ? a.img[g] : 0;
      for (int q = 0; q < nn; ++q) {
        const int ent = a.nbr[(size_t)q * a.ns + g];
        const int j = ent & ENT_JMASK;
        V3<Real> R;
        V3<Real> uj;
        if constexpr (sizeof(Real) == 4) {
          const int4 kj = a.Kw[(size_t)cur * a.ns + j];
          const float4 u4 = a.U[(size_t)cur * a.ns + j];
          uj = V3<float>{u4.x, u4.y, u4.z};
          unsigned dx = (unsigned)kj.x - (unsigned)me.kx, dy = (unsigned)kj.y - (unsigned)me.ky,
                   dz = (unsigned)kj.z - (unsigned)me.kz;
          if (a.periodic) {
            const int mx = img_comp(img_me, 0) - img_comp(kj.w, 0) + ent_shift(ent, 0);
            const int my = img_comp(img_me, 1) - img_comp(kj.w, 1) + ent_shift(ent, 1);
            const int mz = img_comp(img_me, 2) - img_comp(kj.w, 2) + ent_shift(ent, 2);
            dx += (unsigned)mx * a.Lfix[0]; dy += (unsigned)my * a.Lfix[1]; dz += (unsigned)mz * a.Lfix[2];
          }
          R = V3<float>{(float)(int)dx * FIX_SCALE_F, (float)(int)dy * FIX_SCALE_F, (float)(int)dz * FIX_SCALE_F};
        } else {
          const double* X = a.X + (size_t)cur * 3 * a.ns;
          const double* ud = a.ud + (size_t)cur * 3 * a.ns;
          uj = V3<double>{ud[j], ud[a.ns + j], ud[2 * a.ns + j]};
          R = V3<double>{X[j] - me.x, X[a.ns + j] - me.y, X[2 * a.ns + j] - me.z};
          if (a.periodic) {
            const int ij = a.img[j];
            R.x += (double)(img_comp(img_me, 0) - img_comp(ij, 0) + ent_shift(ent, 0)) * a.L[0];
            R.y += (double)(img_comp(img_me, 1) - img_comp(ij, 1) + ent_shift(ent, 1)) * a.L[1];
            R.z += (double)(img_comp(img_me, 2) - img_comp(ij, 2) + ent_shift(ent, 2)) * a.L[2];
          }
        }
        const V3<Real> d = R - h * uj + h * um;   // bead_j - bead_me
        const bool cross_strand = ((g ^ j) & 1) != 0;
        Real e;
        const V3<Real> fw = t_wca(a.c, d, cross_strand ? a.c.scr2 : a.c.sss2, cross_strand ? a.c.rccr2 : a.c.rcss2, &e);
        Fb += fw;
        if constexpr (MODE == MODE_ENERGY) {
          Eb[3] += (Real)0.5 * e;
          vir_add(Wb, d, (Real)-0.5 * fw);
        }
      }
    }
    // applied load on the last base pair (Sec. 4.1, 4.2): f/2 at each centre,
    // torque as a couple normal to its axis; half on each site
    if (f & F_TOP) {
      const int mol = f >> 8;
      const double* ex = a.ext + 8 * mol;
      V3<Real> Fe{(Real)(0.5 * ex[0]), (Real)(0.5 * ex[1]), (Real)(0.5 * ex[2])};
      const V3<Real> Tq{(Real)ex[3], (Real)ex[4], (Real)ex[5]};
      const Real tn2 = dot(Tq, Tq);
      if (tn2 > (Real)0) {
        const V3<Real> th = rsqrt_(tn2) * Tq;
        V3<Real> rho = (Real)-0.5 * rel(me, sm.pos[ring(g ^ 1)]);   // centre offset from the pair centre
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
      const int mol = f >> 8;
      const uint32_t local = (uint32_t)(g - 2 * a.mol_off[mol]);
      double Xd[3], Vd[3];
      if constexpr (sizeof(Real) == 4) {
        Xd[0] = a.X[g]; Xd[1] = a.X[a.ns + g]; Xd[2] = a.X[2 * a.ns + g];
      } else {
        Xd[0] = me.x; Xd[1] = me.y; Xd[2] = me.z;
      }
      Vd[0] = a.V[g]; Vd[1] = a.V[a.ns + g]; Vd[2] = a.V[2 * a.ns + g];
      V3<Real> Om{a.Om[g], a.Om[a.ns + g], a.Om[2 * a.ns + g]};
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
          if (!(isfinite(Ft.x) && isfinite(Ft.y) && isfinite(Ft.z) && isfinite(Om.x) && isfinite(Om.y) &&
                isfinite(Om.z)))
            fl |= B_ENAN;
          a.V[g] = Vd[0]; a.V[a.ns + g] = Vd[1]; a.V[2 * a.ns + g] = Vd[2];
          a.Om[g] = Om.x; a.Om[a.ns + g] = Om.y; a.Om[2 * a.ns + g] = Om.z;
          if constexpr (sizeof(Real) == 4) {
            a.X[g] = Xd[0]; a.X[a.ns + g] = Xd[1]; a.X[2 * a.ns + g] = Xd[2];
          }
        }
        int packed = 0;
        if constexpr (sizeof(Real) == 4) packed = a.Kw[(size_t)cur * a.ns + g].w;
        const int k0 = fix32(Xd[0]), k1 = fix32(Xd[1]), k2 = fix32(Xd[2]);
        store_state(a, nxt, g, k0, k1, k2, Xd, un, packed);
        // rebuild trigger: a bead moved more than skin/2 since the last build
        const float hf = (float)h;
        const float ddx = fixdiff(a.kref[g], k0 + bead_off(hf * (float)un.x));
        const float ddy = fixdiff(a.kref[a.ns + g], k1 + bead_off(hf * (float)un.y));
        const float ddz = fixdiff(a.kref[2 * a.ns + g], k2 + bead_off(hf * (float)un.z));
        if (ddx * ddx + ddy * ddy + ddz * ddz > a.c.skin_half2) fl |= B_STALE;
      }
    }
  }
  if constexpr (MODE == MODE_ENERGY) flush_energy(a, sm.flg[ring(g)] >> 8, Eb, Wb);
}

// One warp's strip: tiles [t0, t1) of SEG slots.  The prologue stages slots
// s0-4 .. s0+3 and computes owners s0-2 .. s0+1; every tile at base B then
// stages slots B+4 .. B+35, computes owners B+2 .. B+33 (one per lane) and
// finishes nucleotides B .. B+31, whose terms come from owners B-2 .. B+33.
// An owner's energy is counted by the strip that holds its slot.
template <class Real, int MODE>
__device__ void strip_pass(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t t0, int64_t t1, int cur,
                           int64_t step, unsigned& fl) {
  if (t0 >= t1) return;
  const int lane = threadIdx.x & 31;
  const int64_t s0 = t0 * SEG;
  const int64_t s1 = t1 * SEG < a.n ? t1 * SEG : a.n;
  if (lane < 8) stage_slot(a, sm, cur, s0 - 4 + lane);
  __syncwarp();
  if (lane < 4) owner_pass<Real, MODE>(a, sm, s0 - 2 + lane, lane >= 2 && s0 - 2 + lane < s1, fl);
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t B = t * SEG;
    __syncwarp();
    stage_slot(a, sm, cur, B + 4 + lane);
    __syncwarp();
    owner_pass<Real, MODE>(a, sm, B + 2 + lane, B + 2 + lane < s1, fl);
    __syncwarp();
    if (B + lane < s1) nucleotide_pass<Real, MODE>(a, sm, B + lane, cur, step, fl);
  }
  __syncwarp();
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

template <class Real>
__global__ void __launch_bounds__(LIST_WARPS * 32) k_rebuild_list_lanes(const KArgs<Real> a) {
  unsigned fl = 0;
  rebuild_list_lanes<Real>(a, fl);
  if (fl) atomicOr(a.err, fl & B_ERRMASK);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.rebuild = 0;
    *a.nrebuild += 1;
  }
}

// ---------------------------------------------------------------- persistent kernel
// MODE_STEP: advance up to *steps_left steps (all of them when steps_left is
// null: nsteps), one bounded grid barrier per step; stop early when a bead
// moved more than skin/2 (the rebuild kernels run next) or on an error.
// MODE_FORCES / MODE_ENERGY: one pass with the current list.
template <class Real, int MODE, int CAPMAX>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 4 : 1) engine_kernel(const KArgs<Real> a) {
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
    const int64_t wpb = blockDim.x >> 5;
    const int64_t nw = gridDim.x * wpb, w = blockIdx.x * wpb + (threadIdx.x >> 5);
    strip_pass<Real, MODE>(a, sm, w * a.nseg / nw, (w + 1) * a.nseg / nw, cur, step, fl);
    if (fl) atomicOr(&s_fl, fl);
    __syncthreads();
    if (MODE != MODE_STEP) {
      errbits = s_fl;
      break;
    }
    const unsigned r = grid_sync(a.bar, gridDim.x, s_fl, a.spin_budget, &s_word);
    if (r & B_ERRMASK) { errbits = r; break; }
    ++done;
    if (r & B_STALE) { need = 1; break; }
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
