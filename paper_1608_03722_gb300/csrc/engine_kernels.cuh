// engine_kernels.cuh -- persistent kernel of the dsDNA engine: neighbour-list
// rebuild phases and the fused force + Langevin segment pass.  Included by
// kern_mixed.cu (Real = float) and kern_fp64.cu (Real = double).
#pragma once
#include "engine.cuh"

namespace dsdna {

// ---------------------------------------------------------------- shared memory
template <class Real>
struct SegSmem {
  SPos<Real>* pos;   // [T + 8]  slots base-4 .. base+T+3
  int* flg;          // [T + 8]
  Real* cs;          // [T + 4][6] forces of owner terms on the owner (bead xyz, patch xyz)
  Real* cn;          // [T + 4][6] ... on the owner's next nucleotide
  Real* cp;          // [T + 4][3] ... on the owner's previous patch (bending)
};

template <class Real>
__host__ __device__ inline size_t seg_smem_bytes(int T) {
  size_t b = sizeof(SPos<Real>) * (T + 8) + sizeof(int) * (T + 8);
  b = (b + 15) & ~(size_t)15;
  b += sizeof(Real) * (size_t)(T + 4) * 15;
  return b + 64;
}

template <class Real>
__device__ __forceinline__ SegSmem<Real> carve(unsigned char* raw, int T) {
  SegSmem<Real> s;
  s.pos = reinterpret_cast<SPos<Real>*>(raw);
  s.flg = reinterpret_cast<int*>(raw + sizeof(SPos<Real>) * (T + 8));
  size_t off = sizeof(SPos<Real>) * (T + 8) + sizeof(int) * (T + 8);
  off = (off + 15) & ~(size_t)15;
  s.cs = reinterpret_cast<Real*>(raw + off);
  s.cn = s.cs + (size_t)(T + 4) * 6;
  s.cp = s.cn + (size_t)(T + 4) * 6;
  return s;
}

// ---------------------------------------------------------------- cell hash
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
  if (a.morton_bits > 0) {   // periodic box: Morton index of the wrapped cell (no collisions)
    return (spread3((unsigned)cx) | (spread3((unsigned)cy) << 1) | (spread3((unsigned)cz) << 2)) & (a.H - 1u);
  }
  unsigned h = (unsigned)cx * 0x8da6b343u ^ (unsigned)cy * 0xd8163841u ^ (unsigned)cz * 0xcb1ab31fu ^
               (unsigned)mol * 0x9E3779B1u;
  h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
  return h & (a.H - 1u);
}

template <class Real>
__device__ __forceinline__ void bead_position(const KArgs<Real>& a, int cur, int64_t g, double* b) {
  const double h = (double)a.c.h;
  if constexpr (sizeof(Real) == 4) {
    const float4 u = a.U[(size_t)cur * a.n + g];
    b[0] = a.X[g] - h * (double)u.x;
    b[1] = a.X[a.n + g] - h * (double)u.y;
    b[2] = a.X[2 * a.n + g] - h * (double)u.z;
  } else {
    const double* X = a.X + (size_t)cur * 3 * a.n;
    const double* u = a.ud + (size_t)cur * 3 * a.n;
    for (int c = 0; c < 3; ++c) b[c] = X[c * a.n + g] - h * u[c * a.n + g];
  }
}

// R1: bin beads, record images and the build-time mirror.
template <class Real>
__device__ void rebuild_bin(const KArgs<Real>& a, int cur, unsigned& fl) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.n; g += stride) {
    double b[3];
    bead_position(a, cur, g, b);
    int w[3] = {0, 0, 0}, ci[3];
    float pw[3];
    for (int c = 0; c < 3; ++c) {
      double x = b[c];
      if (a.periodic && a.L[c] > 0.0) {
        const double q = floor(x / a.L[c]);
        w[c] = (int)q;
        x -= q * a.L[c];
        float xf = (float)x;
        if (xf >= a.Lf[c]) xf = 0.0f;
        if (xf < 0.0f) xf = 0.0f;
        pw[c] = xf;
        int k = (int)(xf / a.cellh[c]);
        ci[c] = k >= a.nc[c] ? a.nc[c] - 1 : k;
        if (w[c] > 511 || w[c] < -512) fl |= B_EIMG;
      } else {
        pw[c] = (float)x;
        ci[c] = (int)floorf(pw[c] / a.cellh[c]);
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
      int4 kw = a.Kw[(size_t)cur * a.n + g];
      const float4 u = a.U[(size_t)cur * a.n + g];
      a.kref[g] = kw.x + bead_off(h * u.x);
      a.kref[a.n + g] = kw.y + bead_off(h * u.y);
      a.kref[2 * a.n + g] = kw.z + bead_off(h * u.z);
      kw.w = packed;
      a.Kw[(size_t)cur * a.n + g] = kw;
    } else {
      const double* X = a.X + (size_t)cur * 3 * a.n;
      const double* u = a.ud + (size_t)cur * 3 * a.n;
      for (int c = 0; c < 3; ++c) a.kref[c * a.n + g] = fix32(X[c * a.n + g]) + bead_off(h * (float)u[c * a.n + g]);
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

// R2a: per-block sums of the count table
template <class Real>
__device__ void rebuild_scan_a(const KArgs<Real>& a, unsigned* s_red) {
  const unsigned chunk = (a.H + gridDim.x - 1) / gridDim.x;
  const unsigned lo = blockIdx.x * chunk, hi = min(a.H, lo + chunk);
  unsigned s = 0;
  for (unsigned i = lo + threadIdx.x; i < hi; i += blockDim.x) s += a.cnt[i];
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
  const unsigned chunk = (a.H + gridDim.x - 1) / gridDim.x;
  const unsigned lo = blockIdx.x * chunk, hi = min(a.H, lo + chunk);
  unsigned pre = 0;
  for (unsigned b = threadIdx.x; b < blockIdx.x; b += blockDim.x) pre += a.bsum[b];
  for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = pre;
  __syncthreads();
  unsigned carry = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) carry += s_red[w];
  __syncthreads();
  for (unsigned base = lo; base < hi; base += blockDim.x) {
    const unsigned i = base + threadIdx.x;
    const unsigned v = i < hi ? a.cnt[i] : 0u;
    unsigned tot;
    const unsigned ex = block_exscan(v, s_red, &tot);
    if (i < hi) a.start[i] = carry + ex;
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
    a.cent[slot] = make_float4(w.x, w.y, w.z, __int_as_float((int)g));
  }
}

// R4: typed full neighbour list of every bead, sorted by partner slot.
// Pairs (Sec. 2, reading A1): opposite strands always (sigma_cross); same
// strand only steric-steric (sigma_ss); same molecule only.
template <class Real, int CAPMAX>
__device__ void rebuild_list(const KArgs<Real>& a, unsigned& fl) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.n; t += stride) {
    const float4 me = a.cent[t];
    const int g = __float_as_int(me.w);
    const int mol = __float_as_int(a.wpos[g].w);
    const bool st_g = (a.topo[g] & F_STERIC) != 0;
    int ci[3];
    const float p[3] = {me.x, me.y, me.z};
    for (int c = 0; c < 3; ++c) {
      int k = (int)floorf(p[c] / a.cellh[c]);
      if (a.periodic && a.L[c] > 0.0 && k >= a.nc[c]) k = a.nc[c] - 1;
      ci[c] = k;
    }
    int list[CAPMAX];
    int cnt = 0, total = 0;
    unsigned seen[27];
    int nseen = 0;
    const bool dedupe = !(a.morton_bits > 0 && a.nc[0] >= 3 && a.nc[1] >= 3 && a.nc[2] >= 3);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int c3[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
          if (a.periodic)
            for (int c = 0; c < 3; ++c)
              if (a.L[c] > 0.0) c3[c] = (c3[c] % a.nc[c] + a.nc[c]) % a.nc[c];
          const unsigned k = cell_key(a, mol, c3[0], c3[1], c3[2]);
          if (dedupe) {
            bool dup = false;
            for (int q = 0; q < nseen; ++q) dup |= (seen[q] == k);
            if (dup) continue;
            seen[nseen++] = k;
          }
          const unsigned e1 = a.start[k + 1];
          for (unsigned e = a.start[k]; e < e1; ++e) {
            const float4 o = a.cent[e];
            const int j = __float_as_int(o.w);
            if (j == g) continue;
            float d[3] = {o.x - p[0], o.y - p[1], o.z - p[2]};
            int sc[3] = {0, 0, 0};
            if (a.periodic)
              for (int c = 0; c < 3; ++c)
                if (a.L[c] > 0.0) {
                  const float s = -rintf(d[c] / a.Lf[c]);
                  d[c] += s * a.Lf[c];
                  sc[c] = (int)s;
                }
            const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= a.c.rl_max2) continue;
            if (__float_as_int(a.wpos[j].w) != mol) continue;
            float rl2;
            if ((g ^ j) & 1) rl2 = a.c.rl_cr2;
            else if (st_g && (a.topo[j] & F_STERIC)) rl2 = a.c.rl_ss2;
            else continue;
            if (r2 >= rl2) continue;
            const int code = (sc[0] + 1) + 3 * (sc[1] + 1) + 9 * (sc[2] + 1);
            const int ent = j | (code << NBR_J_BITS);
            ++total;
            if (cnt < a.cap) {   // insertion by partner slot keeps the force sum order fixed
              int q = cnt++;
              while (q > 0 && (list[q - 1] & ((1 << NBR_J_BITS) - 1)) > j) { list[q] = list[q - 1]; --q; }
              list[q] = ent;
            }
          }
        }
    if (total > a.cap) fl |= B_EOVF;
    for (int q = 0; q < cnt; ++q) a.nbr[(size_t)q * a.n + g] = list[q];
    a.ncnt[g] = cnt;
  }
}

// ---------------------------------------------------------------- segment pass
template <class Real>
__device__ __forceinline__ void owner_terms(const KArgs<Real>& a, const SegSmem<Real>& sm, int oi, unsigned& fl,
                                            Real* E, Real* W) {
  const int pi = oi + 2;                // position index of the owner
  const int f = sm.flg[pi];
  Real* cs = sm.cs + 6 * oi;
  Real* cn = sm.cn + 6 * oi;
  Real* cp = sm.cp + 3 * oi;
  V3<Real> sb{0, 0, 0}, sp{0, 0, 0}, nb{0, 0, 0}, np{0, 0, 0}, pp{0, 0, 0};
  if (f & F_NEXT) {
    const int dir = (pi & 1) ? -2 : 2;  // strand A (even slot) runs up, strand B down
    const SPos<Real>& o = sm.pos[pi];
    const SPos<Real>& q = sm.pos[pi + dir];
    const Real h = a.c.h;
    const V3<Real> uo = uvec(o), uq = uvec(q);
    const V3<Real> Rq = rel(o, q);
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
      const SPos<Real>& r = sm.pos[pi - dir];
      const V3<Real> pr = rel(o, r) + h * uvec(r);
      V3<Real> g1, g2;
      t_bend(a.c, pr - po, pq - po, g1, g2, E);
      pp += g1; np += g2; sp -= (g1 + g2);
      if (W) { vir_add(W, pr, g1); vir_add(W, pq, g2); vir_add(W, po, -(g1 + g2)); }
    }
  }
  cs[0] = sb.x; cs[1] = sb.y; cs[2] = sb.z; cs[3] = sp.x; cs[4] = sp.y; cs[5] = sp.z;
  cn[0] = nb.x; cn[1] = nb.y; cn[2] = nb.z; cn[3] = np.x; cn[4] = np.y; cn[5] = np.z;
  cp[0] = pp.x; cp[1] = pp.y; cp[2] = pp.z;
}

template <class Real>
__device__ __forceinline__ void store_state(const KArgs<Real>& a, int nxt, int64_t g, int k0, int k1, int k2,
                                            const double* X, V3<Real> u, int packed) {
  if constexpr (sizeof(Real) == 4) {
    a.Kw[(size_t)nxt * a.n + g] = make_int4(k0, k1, k2, packed);
    a.U[(size_t)nxt * a.n + g] = make_float4(u.x, u.y, u.z, 0.0f);
  } else {
    double* Xo = a.X + (size_t)nxt * 3 * a.n;
    double* uo = a.ud + (size_t)nxt * 3 * a.n;
    Xo[g] = X[0]; Xo[a.n + g] = X[1]; Xo[2 * a.n + g] = X[2];
    uo[g] = u.x; uo[a.n + g] = u.y; uo[2 * a.n + g] = u.z;
  }
}

template <class Real, int MODE>
__device__ void segment_pass(const KArgs<Real>& a, const SegSmem<Real>& sm, int64_t base, int cur, int64_t step,
                             unsigned& fl, double* eacc) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int nxt = cur ^ 1;
  // 1. stage slots base-4 .. base+T+3
  for (int s = tid; s < T + 8; s += T) {
    const int64_t g = base - 4 + s;
    if (g >= 0 && g < a.n) {
      load_slot(a, cur, g, sm.pos[s]);
      sm.flg[s] = a.topo[g];
    } else {
      sm.flg[s] = 0;
    }
  }
  __syncthreads();
  // 2. bonded terms of owners base-2 .. base+T+1
  Real Eb[NTERMS];
  Real Wb[6];
  if constexpr (MODE == MODE_ENERGY) {
    for (int k = 0; k < NTERMS; ++k) Eb[k] = 0;
    for (int k = 0; k < 6; ++k) Wb[k] = 0;
  }
  for (int oi = tid; oi < T + 4; oi += T) {
    const bool own = (oi >= 2 && oi < T + 2);   // energy of a term goes to its owner only once
    if constexpr (MODE == MODE_ENERGY) {
      owner_terms(a, sm, oi, fl, own ? Eb : nullptr, own ? Wb : nullptr);
    } else {
      owner_terms<Real>(a, sm, oi, fl, nullptr, nullptr);
    }
  }
  __syncthreads();
  // 3. own nucleotide
  const int64_t g = base + tid;
  if (g < a.n) {
    const int pi = tid + 4, oi = tid + 2;
    const int f = sm.flg[pi];
    const SPos<Real>& me = sm.pos[pi];
    const Real h = a.c.h;
    const V3<Real> um = uvec(me);
    V3<Real> Fb{sm.cs[6 * oi + 0], sm.cs[6 * oi + 1], sm.cs[6 * oi + 2]};
    V3<Real> Fp{sm.cs[6 * oi + 3], sm.cs[6 * oi + 4], sm.cs[6 * oi + 5]};
    const int dir = (pi & 1) ? -2 : 2;
    if (f & F_PREV) {
      const int op = oi - dir;
      Fb += V3<Real>{sm.cn[6 * op + 0], sm.cn[6 * op + 1], sm.cn[6 * op + 2]};
      Fp += V3<Real>{sm.cn[6 * op + 3], sm.cn[6 * op + 4], sm.cn[6 * op + 5]};
    }
    if (f & F_NEXT) {
      const int on = oi + dir;
      Fp += V3<Real>{sm.cp[3 * on + 0], sm.cp[3 * on + 1], sm.cp[3 * on + 2]};
    }
    // hydrogen bond with the partner (App. A Eq. 10), broken beyond rc
    {
      const SPos<Real>& q = sm.pos[pi ^ 1];
      const V3<Real> d = rel(me, q) + h * uvec(q) - h * um;   // patch_q - patch_me
      const Real r2 = dot(d, d);
      if (r2 <= a.c.rchb2) {
        Real k2 = (Real)2 * a.c.khb;
        if (a.c.r0hb != (Real)0) k2 *= (Real)1 - a.c.r0hb * rsqrt_(r2);
        Fp += k2 * d;
        if constexpr (MODE == MODE_ENERGY) {
          if ((pi & 1) == 0) {
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
        const int ent = a.nbr[(size_t)q * a.n + g];
        const int j = ent & ((1 << NBR_J_BITS) - 1);
        const int code = (unsigned)ent >> NBR_J_BITS;
        V3<Real> R;
        V3<Real> uj;
        if constexpr (sizeof(Real) == 4) {
          const int4 kj = a.Kw[(size_t)cur * a.n + j];
          const float4 u4 = a.U[(size_t)cur * a.n + j];
          uj = V3<float>{u4.x, u4.y, u4.z};
          unsigned dx = (unsigned)kj.x - (unsigned)me.kx, dy = (unsigned)kj.y - (unsigned)me.ky,
                   dz = (unsigned)kj.z - (unsigned)me.kz;
          if (a.periodic) {
            const int mx = img_comp(img_me, 0) - img_comp(kj.w, 0) + (code % 3) - 1;
            const int my = img_comp(img_me, 1) - img_comp(kj.w, 1) + (code / 3) % 3 - 1;
            const int mz = img_comp(img_me, 2) - img_comp(kj.w, 2) + code / 9 - 1;
            dx += (unsigned)mx * a.Lfix[0]; dy += (unsigned)my * a.Lfix[1]; dz += (unsigned)mz * a.Lfix[2];
          }
          R = V3<float>{(float)(int)dx * FIX_SCALE_F, (float)(int)dy * FIX_SCALE_F, (float)(int)dz * FIX_SCALE_F};
        } else {
          const double* X = a.X + (size_t)cur * 3 * a.n;
          const double* ud = a.ud + (size_t)cur * 3 * a.n;
          uj = V3<double>{ud[j], ud[a.n + j], ud[2 * a.n + j]};
          R = V3<double>{X[j] - me.x, X[a.n + j] - me.y, X[2 * a.n + j] - me.z};
          if (a.periodic) {
            const int ij = a.img[j];
            R.x += (double)(img_comp(img_me, 0) - img_comp(ij, 0) + (code % 3) - 1) * a.L[0];
            R.y += (double)(img_comp(img_me, 1) - img_comp(ij, 1) + (code / 3) % 3 - 1) * a.L[1];
            R.z += (double)(img_comp(img_me, 2) - img_comp(ij, 2) + code / 9 - 1) * a.L[2];
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
        V3<Real> rho = (Real)-0.5 * rel(me, sm.pos[pi ^ 1]);   // centre offset from the pair centre
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
        Xd[0] = a.X[g]; Xd[1] = a.X[a.n + g]; Xd[2] = a.X[2 * a.n + g];
      } else {
        Xd[0] = me.x; Xd[1] = me.y; Xd[2] = me.z;
      }
      Vd[0] = a.V[g]; Vd[1] = a.V[a.n + g]; Vd[2] = a.V[2 * a.n + g];
      V3<Real> Om{a.Om[g], a.Om[a.n + g], a.Om[2 * a.n + g]};
      const bool frozen = (f & F_FROZEN) != 0;
      V3<Real> Ft{0, 0, 0}, Tt{0, 0, 0};
      if (!frozen) {
        // App. A Eq. 8 per site: friction -gamma v_s and noise eta_s, summed over the dumbbell
        const V3<Real> eb = site_noise(a, local, step, mol, 0);
        const V3<Real> ep = site_noise(a, local, step, mol, 1);
        const V3<Real> Vh{(Real)Vd[0], (Real)Vd[1], (Real)Vd[2]};
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
          Vd[0] += (double)dv.x; Vd[1] += (double)dv.y; Vd[2] += (double)dv.z;
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
          if (!(isfinite(Vd[0]) && isfinite(Vd[1]) && isfinite(Vd[2]) && isfinite(Om.x) && isfinite(Om.y) &&
                isfinite(Om.z)))
            fl |= B_ENAN;
          a.V[g] = Vd[0]; a.V[a.n + g] = Vd[1]; a.V[2 * a.n + g] = Vd[2];
          a.Om[g] = Om.x; a.Om[a.n + g] = Om.y; a.Om[2 * a.n + g] = Om.z;
          if constexpr (sizeof(Real) == 4) {
            a.X[g] = Xd[0]; a.X[a.n + g] = Xd[1]; a.X[2 * a.n + g] = Xd[2];
          }
        }
        int packed = 0;
        if constexpr (sizeof(Real) == 4) packed = a.Kw[(size_t)cur * a.n + g].w;
        const int k0 = fix32(Xd[0]), k1 = fix32(Xd[1]), k2 = fix32(Xd[2]);
        store_state(a, nxt, g, k0, k1, k2, Xd, un, packed);
        // rebuild trigger: a bead moved more than skin/2 since the last build
        const float hf = (float)h;
        const float ddx = fixdiff(a.kref[g], k0 + bead_off(hf * (float)un.x));
        const float ddy = fixdiff(a.kref[a.n + g], k1 + bead_off(hf * (float)un.y));
        const float ddz = fixdiff(a.kref[2 * a.n + g], k2 + bead_off(hf * (float)un.z));
        if (ddx * ddx + ddy * ddy + ddz * ddz > a.c.skin_half2) fl |= B_STALE;
      }
    }
  }
  if constexpr (MODE == MODE_ENERGY) {
    // per-thread FP64 accumulation by molecule of the owner
    if (g < a.n) {
      const int mol = sm.flg[tid + 4] >> 8;
      double* dst = a.eout + EOUT_STRIDE * mol;
      for (int k = 0; k < NTERMS; ++k) if (Eb[k] != (Real)0) atomicAdd(dst + k, (double)Eb[k]);
      for (int k = 0; k < 6; ++k) if (Wb[k] != (Real)0) atomicAdd(dst + NTERMS + k, (double)Wb[k]);
    }
  }
  (void)eacc;
  __syncthreads();
}

// ---------------------------------------------------------------- persistent kernel
template <class Real, int CAPMAX>
__device__ bool do_rebuild(const KArgs<Real>& a, int cur, unsigned* s_word, unsigned* s_red) {
  unsigned fl = 0;
  rebuild_bin(a, cur, fl);
  unsigned r = grid_sync(a.bar, gridDim.x, fl, a.spin_budget, s_word);
  if (r & B_ERRMASK) return false;
  rebuild_scan_a(a, s_red);
  r = grid_sync(a.bar, gridDim.x, 0u, a.spin_budget, s_word);
  if (r & B_ERRMASK) return false;
  rebuild_scan_b(a, s_red);
  r = grid_sync(a.bar, gridDim.x, 0u, a.spin_budget, s_word);
  if (r & B_ERRMASK) return false;
  rebuild_scatter(a);
  r = grid_sync(a.bar, gridDim.x, 0u, a.spin_budget, s_word);
  if (r & B_ERRMASK) return false;
  fl = 0;
  rebuild_list<Real, CAPMAX>(a, fl);
  r = grid_sync(a.bar, gridDim.x, fl, a.spin_budget, s_word);
  if (r & B_ERRMASK) return false;
  return true;
}

template <class Real, int MODE, int CAPMAX>
__global__ void engine_kernel(const KArgs<Real> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned s_word;
  __shared__ unsigned s_red[32];
  __shared__ unsigned s_fl;
  const SegSmem<Real> sm = carve<Real>(smem_raw, blockDim.x);
  const int64_t step0 = *a.step;
  int need = *a.rebuild;
  int64_t done = 0;
  unsigned long long builds = 0;
  unsigned errbits = 0;
  const int64_t nsteps = (MODE == MODE_STEP) ? a.nsteps : 1;
  for (int64_t it = 0; it < nsteps; ++it) {
    const int64_t step = step0 + it;
    const int cur = (int)(step & 1);
    if (need) {
      if (!do_rebuild<Real, CAPMAX>(a, cur, &s_word, s_red)) { errbits = s_word; break; }
      need = 0;
      ++builds;
    }
    if (threadIdx.x == 0) s_fl = 0;
    __syncthreads();
    unsigned fl = 0;
    for (int64_t seg = blockIdx.x; seg < a.nseg; seg += gridDim.x)
      segment_pass<Real, MODE>(a, sm, seg * (int64_t)blockDim.x, cur, step, fl, nullptr);
    if (fl) atomicOr(&s_fl, fl);
    __syncthreads();
    if (MODE != MODE_STEP) {
      errbits = s_fl;
      if (errbits) atomicOr(a.err, errbits & B_ERRMASK);
      break;
    }
    const unsigned r = grid_sync(a.bar, gridDim.x, s_fl, a.spin_budget, &s_word);
    if (r & B_ERRMASK) { errbits = r; break; }
    need = (r & B_STALE) ? 1 : 0;
    ++done;
  }
  if (threadIdx.x == 0) {
    if (errbits & B_ERRMASK) atomicOr(a.err, errbits & B_ERRMASK);
    if (blockIdx.x == 0) {
      if (MODE == MODE_STEP) {
        *a.step = step0 + done;
        *a.rebuild = need;
      } else {
        *a.rebuild = 0;
      }
      *a.nrebuild += builds;
    }
  }
}

}  // namespace dsdna
