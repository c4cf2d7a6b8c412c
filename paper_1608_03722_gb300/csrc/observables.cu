// observables.cu -- FP64 reductions for the observables of one molecule:
// extension R_z (Sec. 4.1), denatured fraction (Sec. 5), twist from base-pair
// frames (Sec. 3.2, App. B) and the linking number of the closed strands by
// the Gauss integral (App. C Eq. 17, read with the vector r_R - r_B).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "obs.h"

namespace dsdna {

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 d3(double x, double y, double z) { return D3{x, y, z}; }
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ D3 add(D3 a, D3 b) { return d3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ D3 scl(double s, D3 a) { return d3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dt3(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cr3(D3 a, D3 b) { return d3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ D3 unit(D3 a) { return scl(1.0 / sqrt(dt3(a, a)), a); }

__device__ __forceinline__ D3 site(const ObsArgs& a, int64_t g, double sgn) {
  D3 X = d3(a.X[g], a.X[a.n + g], a.X[2 * a.n + g]);
  D3 u;
  if (a.uf) {
    const float4 v = a.uf[g];
    u = d3(v.x, v.y, v.z);
  } else {
    u = d3(a.ud[g], a.ud[a.n + g], a.ud[2 * a.n + g]);
  }
  return add(X, scl(sgn * a.h, u));
}

__device__ __forceinline__ void block_add(double v, double* dst) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(dst, t);
  }
  __syncthreads();
}

// per base pair: patch midpoint, both bead positions (curves of App. C), broken bond count
__global__ void obs_bp_kernel(ObsArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double broken = 0.0;
  if (k < a.N) {
    const int64_t gA = a.g0 + 2 * (int64_t)k, gB = gA + 1;
    const D3 pA = site(a, gA, 1.0), pB = site(a, gB, 1.0);
    const D3 bA = site(a, gA, -1.0), bB = site(a, gB, -1.0);
    const D3 d = sub(pB, pA);
    if (dt3(d, d) > a.rc2) broken = 1.0;
    const D3 m = add(pA, scl(0.5, d));
    a.mid[3 * k] = m.x; a.mid[3 * k + 1] = m.y; a.mid[3 * k + 2] = m.z;
    a.ca[3 * k] = bA.x; a.ca[3 * k + 1] = bA.y; a.ca[3 * k + 2] = bA.z;
    a.cb[3 * k] = bB.x; a.cb[3 * k + 1] = bB.y; a.cb[3 * k + 2] = bB.z;
  }
  block_add(broken, a.out + 1);
}

__device__ __forceinline__ D3 ld3(const double* p, int k) { return d3(p[3 * k], p[3 * k + 1], p[3 * k + 2]); }

// frame (f, v, t) of base-pair step k: t along the axis, f the bead-bead
// vector of base pair k projected normal to t (on a ring step N - 1 closes it)
__device__ __forceinline__ void frame(const ObsArgs& a, int k, D3* f, D3* v, D3* t) {
  *t = unit(sub(ld3(a.mid, (k + 1) % a.N), ld3(a.mid, k)));
  D3 w = sub(ld3(a.cb, k), ld3(a.ca, k));
  w = sub(w, scl(dt3(w, *t), *t));
  *f = unit(w);
  *v = cr3(*t, *f);
}

// twist increment alpha + gamma between frames k and k+1 (ZYZ Euler angles):
// N - 2 increments on a linear molecule, N on a ring
__global__ void obs_twist_kernel(ObsArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double inc = 0.0;
  if (a.ring ? k < a.N : k + 2 < a.N) {
    D3 f0, v0, t0, f1, v1, t1;
    frame(a, k, &f0, &v0, &t0);
    frame(a, (k + 1) % a.N, &f1, &v1, &t1);
    // R_ij = e_i(k) . e_j(k+1) with e = (f, v, t)
    const double R11 = dt3(f0, f1), R12 = dt3(f0, v1), R21 = dt3(v0, f1), R22 = dt3(v0, v1);
    inc = atan2(R21 - R12, R11 + R22);
    if (a.inc) a.inc[k] = inc / (2.0 * 3.14159265358979323846);
  }
  block_add(inc / (2.0 * 3.14159265358979323846), a.out + 2);
  if (k == 0) a.out[0] = a.mid[3 * (a.N - 1) + 2] - a.mid[2];
}

// closure of both curves (App. C): extensions along the end-to-end axis and a
// far return path, shared by the two strands
__global__ void obs_close_kernel(ObsArgs a) {
  __shared__ double red[32];
  const D3 m0 = ld3(a.mid, 0);
  double ext = 0.0;
  for (int k = threadIdx.x; k < a.N; k += blockDim.x) {
    const D3 d1 = sub(ld3(a.ca, k), m0), d2 = sub(ld3(a.cb, k), m0);
    ext = fmax(ext, fmax(sqrt(dt3(d1, d1)), sqrt(dt3(d2, d2))));
  }
  for (int o = 16; o > 0; o >>= 1) ext = fmax(ext, __shfl_xor_sync(0xffffffffu, ext, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ext;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) ext = fmax(ext, red[w]);
  D3 e = sub(ld3(a.mid, a.N - 1), m0);
  const double le = sqrt(dt3(e, e));
  e = le < 1e-12 ? d3(0, 0, 1) : scl(1.0 / le, e);
  const D3 ax = fabs(e.x) > 0.9 ? d3(0, 1, 0) : d3(1, 0, 0);
  const D3 ep = unit(cr3(e, ax));
  const double D = ext + 5.0, F = 2.0 * ext + 10.0;
  double* curves[2] = {a.ca, a.cb};
  for (int c = 0; c < 2; ++c) {
    double* p = curves[c];
    const D3 c0 = ld3(p, 0), c1 = ld3(p, a.N - 1);
    const D3 q[4] = {add(c1, scl(D, e)), add(add(c1, scl(D, e)), scl(F, ep)), add(sub(c0, scl(D, e)), scl(F, ep)),
                     sub(c0, scl(D, e))};
    for (int j = 0; j < 4; ++j) {
      p[3 * (a.N + j)] = q[j].x; p[3 * (a.N + j) + 1] = q[j].y; p[3 * (a.N + j) + 2] = q[j].z;
    }
  }
}

// signed solid angle of the quadrilateral spanned by segments (r1,r2) and (r3,r4) / 4 pi
__device__ __forceinline__ double seg_lk(D3 r1, D3 r2, D3 r3, D3 r4) {
  const D3 r13 = sub(r3, r1), r14 = sub(r4, r1), r23 = sub(r3, r2), r24 = sub(r4, r2);
  D3 n[4] = {cr3(r13, r14), cr3(r14, r24), cr3(r24, r23), cr3(r23, r13)};
  for (int k = 0; k < 4; ++k) {
    const double l = sqrt(dt3(n[k], n[k]));
    if (l < 1e-300) return 0.0;
    n[k] = scl(1.0 / l, n[k]);
  }
  double om = 0.0;
  for (int k = 0; k < 4; ++k) om += asin(fmin(1.0, fmax(-1.0, dt3(n[k], n[(k + 1) & 3]))));
  const double sg = dt3(cr3(sub(r4, r3), sub(r2, r1)), r13);
  return sg > 0.0 ? om : (sg < 0.0 ? -om : 0.0);
}

// Gauss double sum over all segment pairs of the closed curves (the bead
// curves of a ring are closed already; a linear molecule's carry the four
// closure points); curve B is staged through shared memory in tiles
__global__ void obs_lk_kernel(ObsArgs a) {
  __shared__ double tb[2 * 128 * 3];
  const int M = a.ring ? a.N : a.N + 4;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  D3 r1 = d3(0, 0, 0), r2 = d3(0, 0, 0);
  if (i < M) { r1 = ld3(a.ca, i); r2 = ld3(a.ca, (i + 1) % M); }
  double acc = 0.0;
  for (int j0 = 0; j0 < M; j0 += 128) {
    __syncthreads();
    for (int t = threadIdx.x; t < 129 * 3 && t < 2 * 128 * 3; t += blockDim.x) {
      const int j = j0 + t / 3;
      tb[t] = a.cb[3 * (j % M) + t % 3];
    }
    __syncthreads();
    if (i < M) {
      const int jn = min(128, M - j0);
      for (int j = 0; j < jn; ++j) {
        const D3 r3 = d3(tb[3 * j], tb[3 * j + 1], tb[3 * j + 2]);
        const D3 r4 = d3(tb[3 * j + 3], tb[3 * j + 4], tb[3 * j + 5]);
        acc += seg_lk(r1, r2, r3, r4);
      }
    }
  }
  block_add(acc / (4.0 * 3.14159265358979323846), a.out + 4);
}

cudaError_t obs_launch(const ObsArgs& a, unsigned flags, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.out, 0, 8 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int T = 256;
  const int nb = (a.N + T - 1) / T;
  obs_bp_kernel<<<nb, T, 0, st>>>(a);
  if (a.N >= 2) obs_twist_kernel<<<nb, T, 0, st>>>(a);
  if ((flags & 8u) && a.N >= 2) {
    if (!a.ring) obs_close_kernel<<<1, 256, 0, st>>>(a);
    const int M = a.ring ? a.N : a.N + 4;
    obs_lk_kernel<<<(M + 127) / 128, 128, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace dsdna
