// capi.cu -- host engine behind the C ABI of include/dsdna.h.
//
// Owns the device buffers of a context, builds the topology flags of the
// dsDNA model (Sec. 2: strands, partners, steric / ghost beads, anchored and
// loaded base pairs of Sec. 4), converts states between the caller's AoS
// host arrays and the engine's SoA device layout, and queues the persistent
// engine kernel (engine_kernels.cuh) as captured CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dsdna.h"
#include "engine.cuh"
#include "obs.h"

namespace dsdna {
template <class Real> cudaError_t engine_occupancy(int mode, int T, int* blocks_per_sm, size_t* smem);
template <class Real> cudaError_t engine_launch(int mode, const KArgs<Real>& a, int grid, int T, size_t smem, cudaStream_t st);
template <class Real> cudaError_t rebuild_launch(const KArgs<Real>& a, int scan_grid, cudaStream_t st);
template <class Real> cudaError_t rebuild_prepare();
}  // namespace dsdna

using namespace dsdna;

static constexpr int64_t SEG_SLOTS = 32;   // slots per tile of the engine kernel (a warp walks a strip of tiles)

static thread_local std::string g_create_error;

struct dsdna_ctx {
  dsdna_params p{};
  int device = 0;
  cudaStream_t st = nullptr;
  dsdna_allocator alloc{};
  bool have_alloc = false;
  int n_mol = 0;
  std::vector<int> n_bp;
  std::vector<int64_t> off;      // bp offsets [n_mol + 1]
  std::vector<int> tether;
  std::vector<int> circular;     // per molecule: 1 = ring
  std::vector<double> ext;       // [n_mol][8]
  int64_t n = 0;
  int64_t ns = 0;                // row stride of the [component][slot] arrays (n rounded up to 32)
  int maxN = 0;
  std::vector<void*> bufs;
  int64_t bytes = 0;
  // device buffers
  double* X = nullptr; double* V = nullptr; void* Om = nullptr;
  int4* Kw = nullptr; float4* U = nullptr; double* ud = nullptr;
  int* topo = nullptr; int* img = nullptr; int* kref = nullptr; int* nbr = nullptr; int* ncnt = nullptr;
  int* evl = nullptr; uint2* psrc = nullptr; int* tcnt = nullptr;   // pair halving (mixed precision)
  int64_t n_junc = 0;            // junction owners of circular molecules (8 per ring)
  bool fused = false;            // list rebuilt inside the step kernel
  // kernel instance: with circular molecules or the bubble rule, MODE_EXT;
  // steps with the rebuild inside, MODE_FUSED
  int kernel_flags(int mode) const {
    return ((n_junc > 0 || p.bubble_rule > 0) ? MODE_EXT : 0) | ((fused && mode == MODE_STEP) ? MODE_FUSED : 0);
  }
  int64_t* jslot = nullptr; int* jidx = nullptr; void* jout = nullptr;
  unsigned* cnt = nullptr; unsigned* start = nullptr; int* key = nullptr;
  float4* cent = nullptr; float4* wpos = nullptr; unsigned* bsum = nullptr;
  int64_t* mol_off = nullptr; double* ext_d = nullptr;
  GridBar* bar = nullptr; unsigned* err = nullptr; int64_t* step_d = nullptr; int* rebuild = nullptr;
  unsigned long long* nrebuild = nullptr;
  double* fout = nullptr; double* eout = nullptr; double* stage = nullptr;
  double* obs_scratch = nullptr; double* obs_out = nullptr;
  int64_t* steps_left = nullptr; unsigned* iters = nullptr;
  unsigned long long* nlaunch = nullptr;   // engine launches made by step graphs
  int64_t host_launches = 0;               // engine launches queued directly by the host
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  unsigned H = 0;
  int table = TABLE_HASH;
  int morton_bits = 0;
  int nc[3] = {0, 0, 0};
  double cellh = 0;
  // chain-window list build (periodic box with a linear table, or open box):
  // the separate rebuild kernels and the force and energy passes; the
  // in-kernel rebuild keeps the cell walk
  bool chain = false;
  float4* segc = nullptr;
  int sg_nc[3] = {0, 0, 0};
  double sg_edge = 0;
  unsigned sg_H = 0, sg_mask = 0;
  unsigned H_alloc = 0;          // entries of cnt (start: one more), for either table
  // launch
  int T = 256;
  int64_t nseg = 0;
  int grid[3] = {0, 0, 0};
  size_t smem[3] = {0, 0, 0};
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // step graphs for steps_per_graph and for a remainder
  int64_t gsteps[2] = {0, 0};
  bool graph_failed = false;
  int scan_grid = 0;
  int64_t step = 0;
  bool poisoned = false;
  std::string errmsg;
  KArgs<float> kf{};
  KArgs<double> kd{};
  bool fp64() const { return p.precision == DSDNA_PREC_FP64; }
};

// ---------------------------------------------------------------- helpers
static int fail(dsdna_ctx* c, int code, const std::string& msg) {
  if (c) c->errmsg = msg; else g_create_error = msg;
  return code;
}
static int cuda_fail(dsdna_ctx* c, cudaError_t e, const char* what) {
  if (c) c->poisoned = true;
  return fail(c, DSDNA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

static void* dalloc(dsdna_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (c->have_alloc) {
    p = c->alloc.alloc(bytes, c->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) { c->bufs.push_back(p); c->bytes += (int64_t)bytes; }
  return p;
}

static void free_all(dsdna_ctx* c) {
  for (auto& g : c->gexec)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  for (void* p : c->bufs) {
    if (c->have_alloc) c->alloc.release(p, c->alloc.user);
    else cudaFree(p);
  }
  c->bufs.clear();
}

// Philox4x32-10 (Salmon et al., SC'11) for the host-side initial velocities.
static void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t m0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t m1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t x0 = (uint32_t)(m1 >> 32) ^ c[1] ^ k0;
    const uint32_t x2 = (uint32_t)(m0 >> 32) ^ c[3] ^ k1;
    c[1] = (uint32_t)m1;
    c[3] = (uint32_t)m0;
    c[0] = x0;
    c[2] = x2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Relaxed helix of Sec. 2: patches of base pair k on the z axis at rise*k,
// beads ell off the axis at azimuth k*(d+180 deg), partner on the opposite side.
static void host_helix(const dsdna_params& p, int N, double* X, double* u) {
  const double tw = p.d_dih + M_PI;
  for (int k = 0; k < N; ++k)
    for (int s = 0; s < 2; ++s) {
      const double a = tw * k + (s ? M_PI : 0.0);
      const double cx = std::cos(a), cy = std::sin(a);
      const int64_t g = 2 * (int64_t)k + s;
      X[3 * g + 0] = 0.5 * p.ell * cx;
      X[3 * g + 1] = 0.5 * p.ell * cy;
      X[3 * g + 2] = p.r0_m * k;
      u[3 * g + 0] = -cx;
      u[3 * g + 1] = -cy;
      u[3 * g + 2] = 0.0;
    }
}

// Maxwell-Boltzmann draw: Box-Muller normals of the Philox stream with
// counter (local nucleotide, 2^32-1, 2^32-1, 2*mol + block), angular
// velocity normal to u, net momentum of the mobile nucleotides removed.
static void host_maxwell(const dsdna_params& p, int mol, int N, const double* u, int tether, double* V, double* Om) {
  const double M = 2.0 * p.mass, I = 0.5 * p.mass * p.ell * p.ell;
  const int64_t n = 2 * (int64_t)N;
  const double sv = std::sqrt(p.kT / M), sw = std::sqrt(p.kT / I);
  for (int64_t l = 0; l < n; ++l) {
    double z[8];
    for (int b = 0; b < 2; ++b) {
      uint32_t c[4] = {(uint32_t)l, 0xFFFFFFFFu, 0xFFFFFFFFu, (uint32_t)(2 * mol + b)};
      philox_host(c, (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
      for (int q = 0; q < 2; ++q) {
        const double ua = ((double)c[2 * q] + 0.5) / 4294967296.0;
        const double ub = ((double)c[2 * q + 1] + 0.5) / 4294967296.0;
        const double rad = std::sqrt(-2.0 * std::log(ua));
        z[4 * b + 2 * q] = rad * std::cos(2.0 * M_PI * ub);
        z[4 * b + 2 * q + 1] = rad * std::sin(2.0 * M_PI * ub);
      }
    }
    const double* ul = u + 3 * l;
    double ax[3] = {0, 0, 1};
    if (std::fabs(ul[2]) > 0.9) { ax[0] = 1; ax[2] = 0; }
    double e1[3] = {ul[1] * ax[2] - ul[2] * ax[1], ul[2] * ax[0] - ul[0] * ax[2], ul[0] * ax[1] - ul[1] * ax[0]};
    const double le = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (double& x : e1) x /= le;
    const double e2[3] = {ul[1] * e1[2] - ul[2] * e1[1], ul[2] * e1[0] - ul[0] * e1[2], ul[0] * e1[1] - ul[1] * e1[0]};
    for (int q = 0; q < 3; ++q) {
      V[3 * l + q] = sv * z[q];
      Om[3 * l + q] = sw * (z[3] * e1[q] + z[4] * e2[q]);
    }
  }
  const int64_t first = tether ? 2 : 0;
  double mean[3] = {0, 0, 0};
  for (int64_t l = first; l < n; ++l) for (int q = 0; q < 3; ++q) mean[q] += V[3 * l + q];
  if (n > first) for (double& m : mean) m /= (double)(n - first);
  for (int64_t l = first; l < n; ++l) for (int q = 0; q < 3; ++q) V[3 * l + q] -= mean[q];
  for (int64_t l = 0; l < first; ++l) for (int q = 0; q < 3; ++q) { V[3 * l + q] = 0.0; Om[3 * l + q] = 0.0; }
}

// ---------------------------------------------------------------- state transfer kernels
// staging layout: four [cnt][3] FP64 regions X, V, u, Om -- the callers' own
// layout, so each array moves in one copy
__global__ void k_scatter_state(const double* stage, int64_t g0, int64_t cnt, unsigned mask, int fp64, int cur, int64_t n,
                                double* X, double* V, void* Om, int4* Kw, float4* U, double* ud, const int* topo,
                                double S0, double S1, double S2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  const int64_t g = g0 + i;
  double s[12];
  for (int r = 0; r < 4; ++r)
    for (int q = 0; q < 3; ++q) s[3 * r + q] = stage[3 * (r * cnt + i) + q];
  double* Xc = fp64 ? X + (size_t)cur * 3 * n : X;
  const bool frozen = (topo[g] & F_FROZEN) != 0;
  if (mask & 1) for (int c = 0; c < 3; ++c) Xc[c * n + g] = s[c];
  if (mask & 2) for (int c = 0; c < 3; ++c) V[c * n + g] = frozen ? 0.0 : s[3 + c];
  if (mask & 4) {
    double uu[3] = {s[6], s[7], s[8]};
    const double l2 = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
    if (fabs(l2 - 1.0) > 1e-6) {   // renormalise only inputs that are not unit already (keeps resumes exact)
      const double l = sqrt(l2);
      for (double& x : uu) x /= l;
    }
    if (fp64) {
      double* u = ud + (size_t)cur * 3 * n;
      for (int c = 0; c < 3; ++c) u[c * n + g] = uu[c];
    } else {
      U[(size_t)cur * n + g] = make_float4((float)uu[0], (float)uu[1], (float)uu[2], 0.0f);
    }
  }
  if (mask & 8) {
    for (int c = 0; c < 3; ++c) {
      const double w = frozen ? 0.0 : s[9 + c];
      if (fp64) ((double*)Om)[c * n + g] = w;
      else ((float*)Om)[c * n + g] = (float)w;
    }
  }
  if (!fp64 && (mask & 1)) {
    int4 k = Kw[(size_t)cur * n + g];
    k.x = fixs(Xc[g], S0); k.y = fixs(Xc[n + g], S1); k.z = fixs(Xc[2 * n + g], S2);
    Kw[(size_t)cur * n + g] = k;
  }
}

__global__ void k_gather_state(double* stage, int64_t g0, int64_t cnt, int fp64, int cur, int64_t n, const double* X,
                               const double* V, const void* Om, const float4* U, const double* ud) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  const int64_t g = g0 + i;
  double s[12];
  const double* Xc = fp64 ? X + (size_t)cur * 3 * n : X;
  for (int c = 0; c < 3; ++c) { s[c] = Xc[c * n + g]; s[3 + c] = V[c * n + g]; }
  if (fp64) {
    const double* u = ud + (size_t)cur * 3 * n;
    for (int c = 0; c < 3; ++c) { s[6 + c] = u[c * n + g]; s[9 + c] = ((const double*)Om)[c * n + g]; }
  } else {
    const float4 u = U[(size_t)cur * n + g];
    s[6] = u.x; s[7] = u.y; s[8] = u.z;
    for (int c = 0; c < 3; ++c) s[9 + c] = ((const float*)Om)[c * n + g];
  }
  for (int r = 0; r < 4; ++r)
    for (int q = 0; q < 3; ++q) stage[3 * (r * cnt + i) + q] = s[3 * r + q];
}

// ---------------------------------------------------------------- setup
template <class Real>
static void fill_coef(const dsdna_params& p, Coef<Real>& c) {
  const double rc6 = std::pow(2.0, 1.0 / 6.0);
  const double M = 2.0 * p.mass, I = 0.5 * p.mass * p.ell * p.ell;
  c.K1 = (Real)p.K1; c.R02 = (Real)(p.R0 * p.R0); c.eps_bb = (Real)p.eps_bb;
  c.sbb2 = (Real)(p.sigma_bb * p.sigma_bb); c.rcbb2 = (Real)(rc6 * rc6 * p.sigma_bb * p.sigma_bb);
  c.khb = (Real)(p.K2 / (2.0 * (p.r0_hb - p.rc_hb) * (p.r0_hb - p.rc_hb)));
  c.khb_gc = (Real)((p.K2_gc > 0.0 ? p.K2_gc : p.K2) / (2.0 * (p.r0_hb - p.rc_hb) * (p.r0_hb - p.rc_hb)));
  c.r0hb = (Real)p.r0_hb; c.rchb2 = (Real)(p.rc_hb * p.rc_hb);
  c.eps = (Real)p.eps_ev;
  c.sss2 = (Real)(p.sigma_ss * p.sigma_ss); c.rcss2 = (Real)(rc6 * rc6 * p.sigma_ss * p.sigma_ss);
  c.scr2 = (Real)(p.sigma_cross * p.sigma_cross); c.rccr2 = (Real)(rc6 * rc6 * p.sigma_cross * p.sigma_cross);
  const double scs = p.sigma_cross_steric > 0.0 ? p.sigma_cross_steric : 0.0;
  c.scs2 = (Real)(scs * scs); c.rccs2 = (Real)(rc6 * rc6 * scs * scs);
  c.K3 = (Real)p.K3; c.cosd = (Real)std::cos(p.d_dih); c.sind = (Real)std::sin(p.d_dih);
  c.K4 = (Real)p.K4; c.lam = (Real)p.lambda_m; c.r0m = (Real)p.r0_m;
  c.K5 = (Real)p.K5; c.alpha0 = (Real)p.alpha0;
  c.K6 = (Real)p.K6;
  c.h = (Real)(0.5 * p.ell);
  c.dtM = (Real)(p.dt / M); c.dtI = (Real)(p.dt / I);
  c.halfdtM = (Real)(0.5 * p.dt / M); c.halfdtI = (Real)(0.5 * p.dt / I);
  c.M = (Real)M; c.I = (Real)I;
  c.dt = (Real)p.dt; c.dt_d = p.dt;
  c.gam2 = (Real)(2.0 * p.gamma); c.gamr = (Real)(p.gamma * 0.5 * p.ell * p.ell);
  if (p.noise == DSDNA_NOISE_GAUSSIAN) {
    c.noise_cd = std::sqrt(2.0 * p.gamma * p.kT / p.dt);
  } else {
    c.noise_cd = std::ldexp(std::sqrt(24.0 * p.gamma * p.kT / p.dt), -21);
  }
  c.noise_c = (Real)c.noise_cd;
  const double margin = 0.01;   // absorbs FP32 rounding of the wrapped build positions
  const double rss = rc6 * p.sigma_ss + p.skin + margin, rcr = rc6 * p.sigma_cross + p.skin + margin;
  c.skin_half2 = (float)(0.25 * p.skin * p.skin);
  const double rcs = scs > 0.0 ? rc6 * scs + p.skin + margin : rcr;   // steric pairs across strands
  c.rl_ss2 = (float)(rss * rss); c.rl_cr2 = (float)(rcr * rcr); c.rl_cs2 = (float)(rcs * rcs);
  const double rmx = std::max({rss, rcr, rcs});
  c.rl_max2 = (float)(rmx * rmx);
}

namespace dsdna {
// coefficient block of the mixed-precision kernels, for the no-allocation entry point
__attribute__((visibility("hidden"))) void fill_coef_mixed(const dsdna_params& p, Coef<float>& c) { fill_coef(p, c); }
}  // namespace dsdna

template <class Real>
static void fill_args(dsdna_ctx* c, KArgs<Real>& a) {
  fill_coef(c->p, a.c);
  a.n = c->n; a.ns = c->ns; a.n_mol = c->n_mol; a.nseg = (c->n + SEG_SLOTS - 1) / SEG_SLOTS; a.cap = c->p.max_neighbors;
  a.nsteps = 0; a.noise_mode = c->p.noise;
  a.bubble = c->p.bubble_rule;
  a.n_junc = c->n_junc; a.jslot = c->jslot; a.jidx = c->jidx; a.jout = (Real*)c->jout;
  philox_key_schedule(a, c->p.seed);
  a.spin_budget = 4000000000ull;
  a.X = c->X; a.V = c->V; a.Om = (Real*)c->Om; a.Kw = c->Kw; a.U = c->U; a.ud = c->ud;
  a.topo = c->topo; a.img = c->img; a.kref = c->kref; a.nbr = c->nbr; a.ncnt = c->ncnt;
  a.evl = sizeof(Real) == 4 ? c->evl : nullptr; a.psrc = c->psrc; a.tcnt = c->tcnt;
  a.cnt = c->cnt; a.start = c->start; a.H = c->H; a.table = c->table; a.morton_bits = c->morton_bits; a.key = c->key;
  a.cent = c->cent; a.wpos = c->wpos; a.bsum = c->bsum;
  a.segc = c->chain ? c->segc : nullptr;
  a.nseg16 = (c->n + 15) / 16;
  a.sg_H = c->sg_H;
  a.sg_mask = c->sg_mask;
  a.sg_rcap = (float)DSDNA_SEG_RCAP;
  a.sg_reach = std::sqrt(a.c.rl_max2) + 0.002f;   // margin over the FP32 rounding of centres and radii
  for (int k = 0; k < 3; ++k) {
    a.sg_nc[k] = c->sg_nc[k];
    a.sg_invh[k] = !c->chain ? 0.0f : (float)(c->p.box[0] > 0.0 ? c->sg_nc[k] / c->p.box[k] : 1.0 / c->sg_edge);
  }
  a.periodic = c->p.box[0] > 0.0 ? 1 : 0;
  for (int k = 0; k < 3; ++k) {
    a.nc[k] = c->nc[k];
    a.L[k] = a.periodic ? c->p.box[k] : 0.0;
    a.Lf[k] = (float)a.L[k];
    a.cellh[k] = (float)(a.periodic ? c->p.box[k] / c->nc[k] : c->cellh);
    a.invcellh[k] = 1.0f / a.cellh[k];
    a.invLf[k] = a.periodic ? (float)(1.0 / a.L[k]) : 0.0f;
    mirror_scale(a, k);
  }
  a.mol_off = c->mol_off; a.ext = c->ext_d;
  a.bar = c->bar; a.err = c->err; a.step = c->step_d; a.rebuild = c->rebuild; a.nrebuild = c->nrebuild;
  a.fout = c->fout; a.eout = c->eout;
  a.steps_left = nullptr; a.use_cond = 0; a.h_while = 0;
}

static int validate(const dsdna_params* p, const dsdna_system* s) {
  if (!p || !s || s->n_mol < 1 || !s->n_bp) return fail(nullptr, DSDNA_EINVAL, "params/system missing or n_mol < 1");
  if (s->n_mol >= (1 << (31 - MOL_SHIFT))) return fail(nullptr, DSDNA_EINVAL, "too many molecules (at most 2^21)");
  int64_t tot = 0;
  for (int m = 0; m < s->n_mol; ++m) {
    if (s->n_bp[m] < 1) return fail(nullptr, DSDNA_EINVAL, "molecule with fewer than one base pair");
    tot += s->n_bp[m];
  }
  if (2 * tot >= ((int64_t)1 << ENT_J_BITS)) return fail(nullptr, DSDNA_EINVAL, "more than 2^26 nucleotides");
  const bool per = p->box[0] > 0.0;
  for (int k = 0; k < 3; ++k)
    if ((p->box[k] > 0.0) != per) return fail(nullptr, DSDNA_EINVAL, "box must be periodic in all or no directions");
  if (!(p->dt > 0.0) || !(p->mass > 0.0) || !(p->ell > 0.0) || !(p->R0 > 0.0) || !(p->rc_hb > 0.0) || p->gamma < 0.0 || p->kT < 0.0)
    return fail(nullptr, DSDNA_EINVAL, "non-positive dt/mass/ell/R0/rc or negative gamma/kT");
  if (p->precision != DSDNA_PREC_MIXED && p->precision != DSDNA_PREC_FP64) return fail(nullptr, DSDNA_EINVAL, "precision");
  if (p->bubble_rule < 0 || p->bubble_rule > 2) return fail(nullptr, DSDNA_EINVAL, "bubble_rule must be 0, 1 or 2");
  if (p->rebuild_mode < 0 || p->rebuild_mode > 2) return fail(nullptr, DSDNA_EINVAL, "rebuild_mode must be 0, 1 or 2");
  if (p->pair_halving < 0 || p->pair_halving > 1) return fail(nullptr, DSDNA_EINVAL, "pair_halving must be 0 or 1");
  if (p->list_build < 0 || p->list_build > 1) return fail(nullptr, DSDNA_EINVAL, "list_build must be 0 or 1");
  if (p->K2_gc < 0.0) return fail(nullptr, DSDNA_EINVAL, "K2_gc must be >= 0");
  if (p->noise < 0 || p->noise > 2) return fail(nullptr, DSDNA_EINVAL, "noise mode");
  if (p->steric_phase < 0 || p->steric_phase > 2) return fail(nullptr, DSDNA_EINVAL, "steric_phase must be 0, 1 or 2");
  if (p->skin < 0.0 || p->skin > 1.0) return fail(nullptr, DSDNA_EINVAL, "skin must be in [0, 1] nm");
  if (p->max_neighbors < 0 || p->max_neighbors > 32) return fail(nullptr, DSDNA_EINVAL, "max_neighbors must be <= 32");
  if (p->block_threads && (p->block_threads < 64 || p->block_threads > 1024 || p->block_threads % 32))
    return fail(nullptr, DSDNA_EINVAL, "block_threads must be a multiple of 32 in [64, 1024]");
  if (p->precision == DSDNA_PREC_FP64 && p->block_threads > 256)
    return fail(nullptr, DSDNA_EINVAL, "block_threads of the FP64 path must be at most 256");
  if ((s->X == nullptr) != (s->u == nullptr)) return fail(nullptr, DSDNA_EINVAL, "X and u must be given together");
  if (s->circular)
    for (int m = 0; m < s->n_mol; ++m)
      if (s->circular[m]) {
        if (s->n_bp[m] < 6) return fail(nullptr, DSDNA_EINVAL, "a circular molecule needs at least 6 base pairs");
        if (!s->X) return fail(nullptr, DSDNA_EINVAL, "circular molecules need an initial X and u");
      }
  if ((s->V == nullptr) != (s->Om == nullptr)) return fail(nullptr, DSDNA_EINVAL, "V and Om must be given together");
  return DSDNA_OK;
}

static int upload_state(dsdna_ctx* c, int64_t g0, int64_t cnt, const double* X, const double* V, const double* u,
                        const double* Om) {
  unsigned mask = (X ? 1u : 0u) | (V ? 2u : 0u) | (u ? 4u : 0u) | (Om ? 8u : 0u);
  if (!mask || cnt == 0) return DSDNA_OK;
  const double* src[4] = {X, V, u, Om};
  for (int r = 0; r < 4; ++r)
    if (src[r])
      CK(cudaMemcpyAsync(c->stage + 3 * r * cnt, src[r], sizeof(double) * 3 * cnt, cudaMemcpyHostToDevice, c->st),
         "upload state");
  const int cur = (int)(c->step & 1);
  k_scatter_state<<<(unsigned)((cnt + 255) / 256), 256, 0, c->st>>>(c->stage, g0, cnt, mask, c->fp64(), cur, c->ns, c->X,
                                                                     c->V, c->Om, c->Kw, c->U, c->ud, c->topo,
                                                                     c->kf.fixS[0], c->kf.fixS[1], c->kf.fixS[2]);
  CK(cudaGetLastError(), "scatter state");
  CK(cudaStreamSynchronize(c->st), "upload state sync");
  return DSDNA_OK;
}

extern "C" void dsdna_default_params(dsdna_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->K1 = 30.0; p->R0 = 0.6825; p->eps_bb = 1.0; p->sigma_bb = 0.4430;   // Table 1 backbone
  p->K2 = 6.0; p->r0_hb = 0.0; p->rc_hb = 0.3;                            // Table 1 hydrogen bond
  p->eps_ev = 1.0; p->sigma_ss = 1.0; p->sigma_cross = 0.5;               // Table 1 steric; Sec. 2 ghosts
  p->K3 = 50.0; p->d_dih = -144.0 * M_PI / 180.0;                         // Table 1 dihedral
  p->K4 = 30.0; p->lambda_m = 8.0; p->r0_m = 0.34;                        // Table 1 Morse
  p->K5 = 200.0; p->alpha0 = 0.5 * M_PI;                                  // Table 1 planarity
  p->K6 = 52.0;                                                           // Table 1 bending
  p->mass = 1.0; p->ell = 0.5;                                            // Sec. 2
  p->kT = 1.0; p->gamma = 1.0; p->dt = 0.005;                             // App. A, Eq. 16
  p->seed = 0; p->noise = DSDNA_NOISE_UNIFORM; p->steric_phase = 0;
  p->skin = 0.3; p->precision = DSDNA_PREC_MIXED;
  p->sigma_cross_steric = 1.0;   // Sec. 2, reading A1: two steric beads at sigma = 1 on either strand
  p->pair_halving = 1;
}

extern "C" int dsdna_create(const dsdna_params* params, const dsdna_system* sys, const dsdna_allocator* alloc,
                            void* cuda_stream, dsdna_ctx** out) {
  if (!out) return fail(nullptr, DSDNA_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(params, sys);
  if (rc) return rc;
  dsdna_ctx* c = new dsdna_ctx();
  c->p = *params;
  if (c->p.skin == 0.0) c->p.skin = 0.3;
  if (c->p.max_neighbors == 0) c->p.max_neighbors = 32;
  if (c->p.steps_per_graph <= 0) c->p.steps_per_graph = 50;
  c->st = (cudaStream_t)cuda_stream;
  if (alloc && alloc->alloc && alloc->release) { c->alloc = *alloc; c->have_alloc = true; }
  auto bad = [&](int code) { g_create_error = c->errmsg; free_all(c); delete c; return code; };
  if (cudaGetDevice(&c->device) != cudaSuccess) return bad(fail(c, DSDNA_ECUDA, "no CUDA device"));
  if (c->p.block_threads == 0) {
    // mixed precision with at least one tile per warp at one CTA of 32 warps per
    // SM: one 1024-thread CTA per SM.  With four 256-thread CTAs per SM the CTAs
    // launched later finish each step up to 18% later than the first (measured
    // per warp at 1 Mbp), and the grid barrier waits for the last; otherwise 256.
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    int64_t nt = 0;
    for (int m = 0; m < sys->n_mol; ++m) nt += 2 * (int64_t)sys->n_bp[m];
    const bool big = nsm > 0 && (nt + SEG_SLOTS - 1) / SEG_SLOTS >= 32 * (int64_t)nsm;
    c->p.block_threads = (c->p.precision == DSDNA_PREC_MIXED && big) ? 1024 : 256;
  }
  c->T = c->p.block_threads;
  c->n_mol = sys->n_mol;
  c->n_bp.assign(sys->n_bp, sys->n_bp + sys->n_mol);
  c->off.assign(c->n_mol + 1, 0);
  for (int m = 0; m < c->n_mol; ++m) { c->off[m + 1] = c->off[m] + c->n_bp[m]; c->maxN = std::max(c->maxN, c->n_bp[m]); }
  c->n = 2 * c->off[c->n_mol];
  c->tether.assign(c->n_mol, 0);
  if (sys->tether) for (int m = 0; m < c->n_mol; ++m) c->tether[m] = sys->tether[m] ? 1 : 0;
  c->circular.assign(c->n_mol, 0);
  if (sys->circular) for (int m = 0; m < c->n_mol; ++m) c->circular[m] = sys->circular[m] ? 1 : 0;
  c->ext.assign((size_t)c->n_mol * 8, 0.0);
  const int64_t n = c->n;
  c->nseg = (n + c->T - 1) / c->T;

  // cell table: linear index of the wrapped cell in a periodic box with >= 3
  // cells per edge (padded to whole 2048-entry scan tiles), Morton index in a
  // smaller periodic box, hash of (molecule, cell) otherwise
  const double rc6 = std::pow(2.0, 1.0 / 6.0);
  const double rmax = rc6 * std::max({c->p.sigma_ss, c->p.sigma_cross, c->p.sigma_cross_steric}) + c->p.skin + 0.01;
  c->cellh = rmax * 1.0001;
  if (c->p.box[0] > 0.0) {
    int bits = 1;
    for (int k = 0; k < 3; ++k) {
      c->nc[k] = (int)std::floor(c->p.box[k] / c->cellh);
      if (c->nc[k] < 1) return bad(fail(c, DSDNA_EINVAL, "periodic box smaller than the interaction range"));
      if (c->nc[k] > 1024) return bad(fail(c, DSDNA_EINVAL, "periodic box wider than 1024 cells"));
      while ((1 << bits) < c->nc[k]) ++bits;
    }
    if (c->nc[0] >= 3 && c->nc[1] >= 3 && c->nc[2] >= 3) {
      const uint64_t cells = (uint64_t)c->nc[0] * c->nc[1] * c->nc[2];
      c->H = (unsigned)((cells + 2047) / 2048 * 2048);
      c->table = TABLE_LINEAR;
      c->morton_bits = 0;
    } else {
      c->H = 1u << (3 * bits);    // one table entry per cell, in Morton order
      c->table = TABLE_MORTON;
      c->morton_bits = bits;
    }
  } else {
    unsigned H = 1024;
    while ((int64_t)H < 2 * n) H <<= 1;
    c->H = H;
    c->table = TABLE_HASH;
    c->morton_bits = 0;
  }
  // rebuild inside the step kernel: small systems, linear or hashed table
  c->fused = c->table != TABLE_MORTON &&
             (c->p.rebuild_mode == 2 || (c->p.rebuild_mode == 0 && n <= DSDNA_FUSED_REBUILD_MAX_NT));
  // chain-window list build: a grid of 16-slot segments whose cells span two
  // of the widest segments kept whole plus the list radius; in a periodic box
  // at least 3 cells per edge, in an open box hashed (at most half full with
  // whole segments)
  c->sg_edge = (2.0 * DSDNA_SEG_RCAP + rmax) * 1.001 + 0.01;
  if (c->table == TABLE_LINEAR && c->p.list_build == 0) {
    bool fits = true;
    uint64_t cells = 1;
    for (int k = 0; k < 3; ++k) {
      c->sg_nc[k] = (int)std::floor(c->p.box[k] / c->sg_edge);
      fits = fits && c->sg_nc[k] >= 3;
      cells *= (uint64_t)std::max(1, c->sg_nc[k]);
    }
    if (fits) {
      c->chain = true;
      c->sg_H = (unsigned)((cells + 1 + 2047) / 2048 * 2048);   // start[cells] is a scanned entry
    }
  } else if (c->table == TABLE_HASH && c->p.list_build == 0) {
    unsigned Hs = 2048;
    while ((int64_t)Hs < n / 8) Hs <<= 1;
    c->chain = true;
    c->sg_mask = Hs - 1;
    c->sg_H = Hs + 2048;   // a last tile of empty entries: start[Hs] is a scanned entry
  }
  c->H_alloc = std::max(c->H, c->sg_H);

  // allocations
  const bool f64 = c->fp64();
  const size_t nn = (size_t)n;
  c->ns = (n + 31) / 32 * 32;
  const size_t ns = (size_t)c->ns;
#define ALLOC(ptr, type, count)                                                              \
  do {                                                                                       \
    c->ptr = (type*)dalloc(c, sizeof(type) * (size_t)(count));                               \
    if (!c->ptr) return bad(fail(c, DSDNA_ENOMEM, "device allocation failed: " #ptr));       \
  } while (0)
  ALLOC(X, double, (f64 ? 6 : 3) * ns);
  ALLOC(V, double, 3 * ns);
  c->Om = dalloc(c, (f64 ? 8 : 4) * 3 * ns);
  if (!c->Om) return bad(fail(c, DSDNA_ENOMEM, "device allocation failed: Om"));
  if (f64) { ALLOC(ud, double, 6 * ns); } else { ALLOC(Kw, int4, 2 * ns); ALLOC(U, float4, 2 * ns); }
  ALLOC(topo, int, ns); ALLOC(img, int, ns); ALLOC(kref, int, 3 * ns);
  for (int m = 0; m < c->n_mol; ++m) c->n_junc += c->circular[m] ? 8 : 0;
  if (c->n_junc) {
    ALLOC(jslot, int64_t, c->n_junc); ALLOC(jidx, int, ns);
    c->jout = dalloc(c, (f64 ? 8 : 4) * 16 * (size_t)c->n_junc);
    if (!c->jout) return bad(fail(c, DSDNA_ENOMEM, "device allocation failed: jout"));
  }
  ALLOC(nbr, int, (size_t)c->p.max_neighbors * ns); ALLOC(ncnt, int, ns);
  // pair halving: mixed precision with the list rebuilt by the separate kernels
  if (!f64 && c->p.pair_halving && !c->fused) {
    const size_t nt = (nn + SEG_SLOTS - 1) / SEG_SLOTS;
    ALLOC(evl, int, nt * EVL_CAP); ALLOC(psrc, uint2, ns); ALLOC(tcnt, int, nt);
  }
  ALLOC(cnt, unsigned, c->H_alloc); ALLOC(start, unsigned, (size_t)c->H_alloc + 1); ALLOC(key, int, nn);
  ALLOC(cent, float4, nn); ALLOC(wpos, float4, nn);
  if (c->chain) ALLOC(segc, float4, (nn + 15) / 16 + 1);
  ALLOC(mol_off, int64_t, c->n_mol + 1); ALLOC(ext_d, double, (size_t)c->n_mol * 8);
  ALLOC(bar, GridBar, 1); ALLOC(err, unsigned, 4); ALLOC(step_d, int64_t, 1); ALLOC(rebuild, int, 4);
  ALLOC(nrebuild, unsigned long long, 1);
  ALLOC(fout, double, 6 * nn); ALLOC(eout, double, (size_t)c->n_mol * EOUT_STRIDE);
  ALLOC(stage, double, 12 * nn);
  ALLOC(obs_scratch, double, 3 * (size_t)(3 * (c->maxN + 4)) + (size_t)c->maxN + 4);   // curves + twist increments
  ALLOC(obs_out, double, 8);
  ALLOC(steps_left, int64_t, 1);
  ALLOC(iters, unsigned, 4);
  ALLOC(nlaunch, unsigned long long, 1);
#undef ALLOC
  // launch shape per mode (cooperative: every CTA resident)
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  for (int mode = 0; mode < 3; ++mode) {
    int bps = 0;
    const int m = mode | c->kernel_flags(mode);
    cudaError_t e = f64 ? engine_occupancy<double>(m, c->T, &bps, &c->smem[mode])
                        : engine_occupancy<float>(m, c->T, &bps, &c->smem[mode]);
    if (e != cudaSuccess || bps < 1) return bad(fail(c, DSDNA_ECUDA, std::string("occupancy: ") + cudaGetErrorString(e)));
    if (c->p.blocks_per_sm > 0) bps = std::min(bps, c->p.blocks_per_sm);
    c->grid[mode] = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)bps * nsm, c->nseg));
  }
  if (c->chain) {
    const cudaError_t e = f64 ? rebuild_prepare<double>() : rebuild_prepare<float>();
    if (e != cudaSuccess) return bad(fail(c, DSDNA_ECUDA, std::string("rebuild kernel attributes: ") + cudaGetErrorString(e)));
  }
  c->scan_grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * 8, ((int64_t)c->H + 2047) / 2048));
  // block sums: one per CTA of the scan kernels, or of the step kernel when it rebuilds
  c->bsum = (unsigned*)dalloc(c, sizeof(unsigned) * (size_t)std::max(c->scan_grid, c->grid[MODE_STEP]));
  if (!c->bsum) return bad(fail(c, DSDNA_ENOMEM, "device allocation failed: bsum"));

  // topology flags (Sec. 2; anchored and loaded base pairs of Sec. 4)
  std::vector<int> topo(ns, 0);   // padding slots: no flags
  for (int m = 0; m < c->n_mol; ++m) {
    const int N = c->n_bp[m];
    for (int k = 0; k < N; ++k)
      for (int s = 0; s < 2; ++s) {
        const int64_t g = 2 * (c->off[m] + k) + s;
        const int q = s == 0 ? k : N - 1 - k;     // index along the strand from its 5' end
        const bool ring = c->circular[m] != 0;     // Sec. 6 rings: the last nucleotide bonds to the first
        const int ph = c->p.steric_phase;
        int f = 0;
        // on a ring the last steric bead before the junction turns ghost when it
        // would sit fewer than 3 nucleotides from the first one after it
        if (q % 3 == ph && !(ring && q > N + ph - 3)) f |= F_STERIC;
        // a ring's neighbour across the junction is reached through the
        // junction table, not the slot-order ring of the step kernel: its
        // F_PREV / F_NEXT stays clear
        if (q > 0) f |= F_PREV;
        if (q < N - 1) f |= F_NEXT;
        if (ring && (k < 2 || k > N - 3)) f |= F_JUNC;
        if (c->tether[m] && k == 0) f |= F_FROZEN;
        if (k == N - 1) f |= F_TOP;
        if (sys->gc && sys->gc[c->off[m] + k]) f |= F_GC;   // Sec. 5: G.C pair, stiffer hydrogen bond
        topo[g] = f | (m << MOL_SHIFT);
      }
  }
  auto cpy = [&](void* dst, const void* src, size_t b) { return cudaMemcpy(dst, src, b, cudaMemcpyHostToDevice); };
  if (c->n_junc) {
    // junction owners of ring r: base pairs 0, 1, N-2, N-1 (position p), both strands: entry 8 r + 2 p + s
    std::vector<int64_t> js((size_t)c->n_junc);
    std::vector<int> ji(ns, -1);
    int64_t t = 0;
    for (int m = 0; m < c->n_mol; ++m) {
      if (!c->circular[m]) continue;
      const int N = c->n_bp[m];
      const int ks[4] = {0, 1, N - 2, N - 1};
      for (int p4 = 0; p4 < 4; ++p4)
        for (int s = 0; s < 2; ++s, ++t) {
          const int64_t g = 2 * (c->off[m] + ks[p4]) + s;
          js[(size_t)t] = g;
          ji[(size_t)g] = (int)t;
        }
    }
    if (cpy(c->jslot, js.data(), sizeof(int64_t) * js.size()) != cudaSuccess ||
        cpy(c->jidx, ji.data(), sizeof(int) * ns) != cudaSuccess)
      return bad(fail(c, DSDNA_ECUDA, "junction table upload"));
  }
  if (cpy(c->topo, topo.data(), sizeof(int) * ns) != cudaSuccess ||
      cpy(c->mol_off, c->off.data(), sizeof(int64_t) * (c->n_mol + 1)) != cudaSuccess ||
      cpy(c->ext_d, c->ext.data(), sizeof(double) * c->ext.size()) != cudaSuccess)
    return bad(fail(c, DSDNA_ECUDA, "topology upload"));
  if (cudaMemset(c->cnt, 0, sizeof(unsigned) * c->H_alloc) != cudaSuccess || cudaMemset(c->err, 0, 16) != cudaSuccess ||
      cudaMemset(c->step_d, 0, 8) != cudaSuccess || cudaMemset(c->nrebuild, 0, 8) != cudaSuccess ||
      cudaMemset(c->nlaunch, 0, 8) != cudaSuccess ||
      cudaMemset(c->bar, 0, sizeof(GridBar)) != cudaSuccess || cudaMemset(c->ncnt, 0, sizeof(int) * ns) != cudaSuccess ||
      cudaMemset(c->Om, 0, (f64 ? 8 : 4) * 3 * ns) != cudaSuccess || cudaMemset(c->V, 0, 24 * ns) != cudaSuccess ||
      cudaMemset(c->X, 0, (f64 ? 48 : 24) * ns) != cudaSuccess || cudaMemset(c->kref, 0, 12 * ns) != cudaSuccess ||
      cudaMemset(c->img, 0, 4 * ns) != cudaSuccess)
    return bad(fail(c, DSDNA_ECUDA, "initialisation"));
  if (!f64 && (cudaMemset(c->Kw, 0, sizeof(int4) * 2 * ns) != cudaSuccess ||
               cudaMemset(c->U, 0, sizeof(float4) * 2 * ns) != cudaSuccess))
    return bad(fail(c, DSDNA_ECUDA, "initialisation"));
  if (f64 && cudaMemset(c->ud, 0, 48 * ns) != cudaSuccess) return bad(fail(c, DSDNA_ECUDA, "initialisation"));
  const int one = 1;
  if (cpy(c->rebuild, &one, sizeof(int)) != cudaSuccess) return bad(fail(c, DSDNA_ECUDA, "initialisation"));
  fill_args(c, c->kf);
  fill_args(c, c->kd);

  // initial state
  std::vector<double> Xh, uh, Vh, Oh;
  const double *X0 = sys->X, *u0 = sys->u, *V0 = sys->V, *O0 = sys->Om;
  if (!X0) {
    Xh.resize(3 * nn); uh.resize(3 * nn);
    for (int m = 0; m < c->n_mol; ++m) host_helix(c->p, c->n_bp[m], &Xh[6 * c->off[m]], &uh[6 * c->off[m]]);
    X0 = Xh.data(); u0 = uh.data();
  }
  if (!V0) {
    Vh.resize(3 * nn); Oh.resize(3 * nn);
    for (int m = 0; m < c->n_mol; ++m)
      host_maxwell(c->p, m, c->n_bp[m], u0 + 6 * c->off[m], c->tether[m], &Vh[6 * c->off[m]], &Oh[6 * c->off[m]]);
    V0 = Vh.data(); O0 = Oh.data();
  }
  rc = upload_state(c, 0, n, X0, V0, u0, O0);
  if (rc) return bad(rc);
  *out = c;
  return DSDNA_OK;
}

// ---------------------------------------------------------------- launches
// Step loop of one graph launch: a WHILE node repeats [head -> IF(rebuild
// requested) {five rebuild kernels} -> persistent step kernel] until the
// step kernel reports that the launch's steps are done.
__global__ void k_loop_init(int64_t* steps_left, int64_t nsteps, unsigned* iters, cudaGraphConditionalHandle h_while) {
  *steps_left = nsteps;
  *iters = 0u;
  cudaGraphSetConditional(h_while, nsteps > 0 ? 1u : 0u);
}

// The loop continues only if the step kernel of this iteration says so (a
// step kernel that never runs ends it); more iterations than steps means no
// progress and ends the loop with a timeout error.
__global__ void k_loop_head(const int* rebuild, unsigned* iters, unsigned max_iters, unsigned* err, int64_t* steps_left,
                            unsigned long long* nlaunch, cudaGraphConditionalHandle h_while,
                            cudaGraphConditionalHandle h_if) {
  const unsigned it = ++*iters;
  ++*nlaunch;                       // every iteration runs one step kernel
  cudaGraphSetConditional(h_while, 0u);
  bool ok = (*err & B_ERRMASK) == 0;
  if (it > max_iters) {
    *steps_left = 0;
    atomicOr(err, (unsigned)B_ETIMEOUT);
    ok = false;
  }
  cudaGraphSetConditional(h_if, (ok && *rebuild != 0) ? 1u : 0u);
}

static cudaError_t launch_rebuild(dsdna_ctx* c) {
  return c->fp64() ? rebuild_launch<double>(c->kd, c->scan_grid, c->st) : rebuild_launch<float>(c->kf, c->scan_grid, c->st);
}

static cudaError_t launch_engine(dsdna_ctx* c, int mode, int64_t nsteps, int64_t* steps_left, int use_cond,
                                 cudaGraphConditionalHandle hw, cudaEvent_t ev_start = nullptr) {
  cudaError_t e = cudaMemsetAsync(c->bar, 0, sizeof(GridBar), c->st);
  if (e != cudaSuccess) return e;
  if (ev_start && (e = cudaEventRecord(ev_start, c->st)) != cudaSuccess) return e;
  if (!use_cond) ++c->host_launches;
  if (c->fp64()) {
    KArgs<double> a = c->kd;
    a.nsteps = nsteps; a.steps_left = steps_left; a.use_cond = use_cond; a.h_while = hw;
    return engine_launch<double>(mode | c->kernel_flags(mode), a, c->grid[mode], c->T, c->smem[mode], c->st);
  }
  KArgs<float> a = c->kf;
  a.nsteps = nsteps; a.steps_left = steps_left; a.use_cond = use_cond; a.h_while = hw;
  return engine_launch<float>(mode | c->kernel_flags(mode), a, c->grid[mode], c->T, c->smem[mode], c->st);
}

// force / energy pass on a fresh list
static int launch(dsdna_ctx* c, int mode, int64_t nsteps) {
  CK(launch_rebuild(c), "rebuild launch");
  CK(launch_engine(c, mode, nsteps, nullptr, 0, 0), "engine launch");
  return DSDNA_OK;
}

static cudaError_t build_step_graph(dsdna_ctx* c, int64_t K, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  auto done = [&](cudaError_t err) {
    if (g) cudaGraphDestroy(g);
    return err;
  };
  cudaGraphConditionalHandle hw = 0, hi = 0;
  if ((e = cudaGraphConditionalHandleCreate(&hw, g, 0, 0)) != cudaSuccess) return done(e);
  if ((e = cudaGraphConditionalHandleCreate(&hi, g, 0, 0)) != cudaSuccess) return done(e);
  cudaGraphNode_t init = nullptr, head = nullptr, wn = nullptr, ifn = nullptr;
  {
    int64_t* sl = c->steps_left;
    unsigned* it = c->iters;
    int64_t k = K;
    void* args[] = {&sl, &k, &it, &hw};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)k_loop_init;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    if ((e = cudaGraphAddKernelNode(&init, g, nullptr, 0, &kp)) != cudaSuccess) return done(e);
  }
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  if ((e = cudaGraphAddNode(&wn, g, &init, nullptr, 1, &wp)) != cudaSuccess) return done(e);
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  {
    int* rb = c->rebuild;
    unsigned* it = c->iters;
    unsigned maxit = (unsigned)(K + 2);
    unsigned* er = c->err;
    int64_t* sl = c->steps_left;
    unsigned long long* nl = c->nlaunch;
    void* args[] = {&rb, &it, &maxit, &er, &sl, &nl, &hw, &hi};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)k_loop_head;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    if ((e = cudaGraphAddKernelNode(&head, body, nullptr, 0, &kp)) != cudaSuccess) return done(e);
  }
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hi;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  if ((e = cudaGraphAddNode(&ifn, body, &head, nullptr, 1, &ip)) != cudaSuccess) return done(e);
  cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(c->st, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return done(e);
  cudaError_t e1 = launch_rebuild(c);
  cudaError_t e2 = cudaStreamEndCapture(c->st, &ifbody);
  if (e1 != cudaSuccess) return done(e1);
  if (e2 != cudaSuccess) return done(e2);
  if ((e = cudaStreamBeginCaptureToGraph(c->st, body, &ifn, nullptr, 1, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return done(e);
  e1 = launch_engine(c, MODE_STEP, K, c->steps_left, 1, hw);
  e2 = cudaStreamEndCapture(c->st, &body);
  if (e1 != cudaSuccess) return done(e1);
  if (e2 != cudaSuccess) return done(e2);
  e = cudaGraphInstantiate(out, g, 0);
  return done(e);
}

// Fallback without conditional graph nodes: the host waits after every
// persistent launch and queues the rebuild itself.
static int step_host_loop(dsdna_ctx* c, int64_t nsteps) {
  int64_t dstep = 0;
  CK(cudaStreamSynchronize(c->st), "step sync");
  CK(cudaMemcpy(&dstep, c->step_d, sizeof(dstep), cudaMemcpyDeviceToHost), "read step");
  const int64_t target = dstep + nsteps;
  for (int guard = 0; guard < nsteps + 2; ++guard) {
    int rb = 0;
    unsigned er = 0;
    CK(cudaMemcpy(&dstep, c->step_d, sizeof(dstep), cudaMemcpyDeviceToHost), "read step");
    CK(cudaMemcpy(&rb, c->rebuild, sizeof(rb), cudaMemcpyDeviceToHost), "read rebuild flag");
    CK(cudaMemcpy(&er, c->err, sizeof(er), cudaMemcpyDeviceToHost), "read error word");
    if (er || dstep >= target) break;
    if (rb) CK(launch_rebuild(c), "rebuild launch");
    CK(launch_engine(c, MODE_STEP, target - dstep, nullptr, 0, 0), "engine launch");
    CK(cudaStreamSynchronize(c->st), "step sync");
  }
  return DSDNA_OK;
}

static int map_err(dsdna_ctx* c, unsigned bits) {
  if (!bits) return DSDNA_OK;
  c->poisoned = true;
  if (bits & B_EFENE) return fail(c, DSDNA_EFENE, "backbone bond reached R0 (FENE diverges)");
  if (bits & B_ENAN) return fail(c, DSDNA_ENAN, "non-finite velocity");
  if (bits & B_EOVF) return fail(c, DSDNA_EOVERFLOW, "neighbour list capacity exceeded");
  if (bits & B_EIMG) return fail(c, DSDNA_EOVERFLOW, "periodic image index out of range");
  if (bits & B_ETIMEOUT) return fail(c, DSDNA_ETIMEOUT, "device barrier timed out");
  return fail(c, DSDNA_ECUDA, "unknown device error");
}

static int sync_check(dsdna_ctx* c) {
  CK(cudaStreamSynchronize(c->st), "synchronize");
  unsigned bits = 0;
  CK(cudaMemcpy(&bits, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read error word");
  return map_err(c, bits);
}

extern "C" int dsdna_set_external_force_torque(dsdna_ctx* c, int mol, const double f[3], const double t[3]) {
  if (!c) return DSDNA_EINVAL;
  if (c->poisoned) return fail(c, DSDNA_ESTATE, "context poisoned by an earlier error");
  if (mol < -1 || mol >= c->n_mol) return fail(c, DSDNA_EINVAL, "molecule index out of range");
  const int m0 = mol < 0 ? 0 : mol, m1 = mol < 0 ? c->n_mol : mol + 1;
  for (int m = m0; m < m1; ++m)
    for (int q = 0; q < 3; ++q) {
      c->ext[8 * m + q] = f ? f[q] : 0.0;
      c->ext[8 * m + 3 + q] = t ? t[q] : 0.0;
    }
  CK(cudaMemcpyAsync(c->ext_d + 8 * m0, c->ext.data() + 8 * m0, sizeof(double) * 8 * (m1 - m0), cudaMemcpyHostToDevice,
                     c->st), "upload load");
  CK(cudaStreamSynchronize(c->st), "upload load sync");
  return DSDNA_OK;
}

extern "C" int dsdna_step(dsdna_ctx* c, int64_t nsteps) {
  if (!c) return DSDNA_EINVAL;
  if (c->poisoned) return fail(c, DSDNA_ESTATE, "context poisoned by an earlier error");
  if (nsteps < 0) return fail(c, DSDNA_EINVAL, "negative step count");
  const int64_t K = c->p.steps_per_graph;
  while (nsteps > 0) {
    const int64_t chunk = std::min(nsteps, K);
    if (!c->graph_failed) {
      const int slot = chunk == K ? 0 : 1;
      if (!c->gexec[slot] || c->gsteps[slot] != chunk) {
        if (c->gexec[slot]) { cudaGraphExecDestroy(c->gexec[slot]); c->gexec[slot] = nullptr; }
        if (build_step_graph(c, chunk, &c->gexec[slot]) == cudaSuccess) {
          c->gsteps[slot] = chunk;
        } else {
          c->gexec[slot] = nullptr;
          c->graph_failed = true;
          cudaGetLastError();
        }
      }
      if (c->gexec[slot]) {
        CK(cudaGraphLaunch(c->gexec[slot], c->st), "graph launch");
        c->step += chunk;
        nsteps -= chunk;
        continue;
      }
    }
    int rc = step_host_loop(c, chunk);
    if (rc) return rc;
    c->step += chunk;
    nsteps -= chunk;
  }
  return DSDNA_OK;
}

// Host-driven steps with a CUDA event pair around every rebuild and every
// step-kernel launch on the context stream.
extern "C" int dsdna_step_profiled(dsdna_ctx* c, int64_t nsteps, dsdna_prof* out) {
  if (!c || !out) return DSDNA_EINVAL;
  if (c->poisoned) return fail(c, DSDNA_ESTATE, "context poisoned by an earlier error");
  if (nsteps < 0) return fail(c, DSDNA_EINVAL, "negative step count");
  std::memset(out, 0, sizeof(*out));
  for (int k = 0; k < 4; ++k)
    if (!c->ev[k]) CK(cudaEventCreate(&c->ev[k]), "event create");
  int64_t dstep = 0;
  CK(cudaStreamSynchronize(c->st), "step sync");
  CK(cudaMemcpy(&dstep, c->step_d, sizeof(dstep), cudaMemcpyDeviceToHost), "read step");
  const int64_t first = dstep, target = dstep + nsteps;
  for (int64_t guard = 0; guard < nsteps + 2 && dstep < target; ++guard) {
    int rb = 0;
    unsigned er = 0;
    CK(cudaMemcpy(&rb, c->rebuild, sizeof(rb), cudaMemcpyDeviceToHost), "read rebuild flag");
    CK(cudaMemcpy(&er, c->err, sizeof(er), cudaMemcpyDeviceToHost), "read error word");
    if (er) break;
    if (rb) {
      CK(cudaEventRecord(c->ev[0], c->st), "event record");
      CK(launch_rebuild(c), "rebuild launch");
      CK(cudaEventRecord(c->ev[1], c->st), "event record");
    }
    CK(launch_engine(c, MODE_STEP, target - dstep, nullptr, 0, 0, c->ev[2]), "engine launch");
    CK(cudaEventRecord(c->ev[3], c->st), "event record");
    CK(cudaStreamSynchronize(c->st), "step sync");
    float ms = 0.f;
    if (rb) {
      CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]), "event time");
      out->rebuild_ms += ms;
      ++out->rebuild_launches;
    }
    CK(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]), "event time");
    out->engine_ms += ms;
    ++out->engine_launches;
    CK(cudaMemcpy(&dstep, c->step_d, sizeof(dstep), cudaMemcpyDeviceToHost), "read step");
  }
  out->steps = dstep - first;
  c->step += out->steps;
  return sync_check(c);
}

extern "C" int dsdna_synchronize(dsdna_ctx* c) {
  if (!c) return DSDNA_EINVAL;
  if (c->poisoned) return fail(c, DSDNA_ESTATE, "context poisoned by an earlier error");
  return sync_check(c);
}

extern "C" int dsdna_energy_virial(dsdna_ctx* c, int mol, double energy[DSDNA_NTERMS], double virial[6]) {
  if (!c) return DSDNA_EINVAL;
  if (c->poisoned) return fail(c, DSDNA_ESTATE, "context poisoned by an earlier error");
  if (mol < -1 || mol >= c->n_mol) return fail(c, DSDNA_EINVAL, "molecule index out of range");
  CK(cudaMemsetAsync(c->eout, 0, sizeof(double) * EOUT_STRIDE * c->n_mol, c->st), "clear energies");
  int rc = launch(c, MODE_ENERGY, 0);
  if (rc) return rc;
  rc = sync_check(c);
  if (rc) return rc;
  std::vector<double> e((size_t)c->n_mol * EOUT_STRIDE);
  CK(cudaMemcpy(e.data(), c->eout, sizeof(double) * e.size(), cudaMemcpyDeviceToHost), "read energies");
  const int m0 = mol < 0 ? 0 : mol, m1 = mol < 0 ? c->n_mol : mol + 1;
  for (int k = 0; k < DSDNA_NTERMS; ++k) if (energy) energy[k] = 0.0;
  for (int k = 0; k < 6; ++k) if (virial) virial[k] = 0.0;
  for (int m = m0; m < m1; ++m) {
    for (int k = 0; k < DSDNA_NTERMS; ++k) if (energy) energy[k] += e[(size_t)m * EOUT_STRIDE + k];
    for (int k = 0; k < 6; ++k) if (virial) virial[k] += e[(size_t)m * EOUT_STRIDE + NTERMS + k];
  }
  return DSDNA_OK;
}

extern "C" int dsdna_observables(dsdna_ctx* c, int mol, unsigned flags, dsdna_obs* out) {
  if (!c || !out) return DSDNA_EINVAL;
  if (c->poisoned) return fail(c, DSDNA_ESTATE, "context poisoned by an earlier error");
  if (mol < 0 || mol >= c->n_mol) return fail(c, DSDNA_EINVAL, "molecule index out of range");
  int rc = sync_check(c);
  if (rc) return rc;
  const int cur = (int)(c->step & 1);
  ObsArgs a{};
  a.n = c->ns;   // row stride of the [3][n] arrays
  a.X = c->fp64() ? c->X + (size_t)cur * 3 * c->ns : c->X;
  a.uf = c->fp64() ? nullptr : c->U + (size_t)cur * c->ns;
  a.ud = c->fp64() ? c->ud + (size_t)cur * 3 * c->ns : nullptr;
  a.g0 = 2 * c->off[mol];
  a.N = c->n_bp[mol];
  a.ring = c->circular[mol];
  a.h = 0.5 * c->p.ell;
  a.rc2 = c->p.rc_hb * c->p.rc_hb;
  a.mid = c->obs_scratch;
  a.ca = a.mid + 3 * (size_t)(c->maxN + 4);
  a.cb = a.ca + 3 * (size_t)(c->maxN + 4);
  a.out = c->obs_out;
  CK(obs_launch(a, flags, c->st), "observables");
  double o[8];
  CK(cudaMemcpyAsync(o, c->obs_out, sizeof(o), cudaMemcpyDeviceToHost, c->st), "read observables");
  CK(cudaStreamSynchronize(c->st), "observables sync");
  out->rz = o[0];
  out->denat = o[1] / (double)a.N;
  out->tw = o[2];
  // twist increments: N on a ring (the last step closes it), N - 2 on a linear molecule
  const int ninc = a.ring ? a.N : a.N - 2;
  out->tw_ideal = a.N >= 3 ? (double)ninc * (c->p.d_dih + M_PI) / (2.0 * M_PI) : 0.0;
  out->lk = (flags & DSDNA_OBS_LK) ? o[4] : 0.0;
  out->wr = (flags & DSDNA_OBS_LK) ? o[4] - o[2] : 0.0;
  return DSDNA_OK;
}

// Per-base-pair centreline (patch midpoints, Sec. 3.1) and per-step twist
// increments (App. B) of one molecule, from the same device reductions as
// dsdna_observables; the FP64 arrays go to caller-owned host memory.
extern "C" int dsdna_profiles(dsdna_ctx* c, int mol, double* centre, double* twist) {
  if (!c) return DSDNA_EINVAL;
  if (c->poisoned) return fail(c, DSDNA_ESTATE, "context poisoned by an earlier error");
  if (mol < 0 || mol >= c->n_mol) return fail(c, DSDNA_EINVAL, "molecule index out of range");
  int rc = sync_check(c);
  if (rc) return rc;
  const int N = c->n_bp[mol];
  const int ninc = c->circular[mol] ? N : std::max(0, N - 2);
  const int cur = (int)(c->step & 1);
  ObsArgs a{};
  a.n = c->ns;
  a.X = c->fp64() ? c->X + (size_t)cur * 3 * c->ns : c->X;
  a.uf = c->fp64() ? nullptr : c->U + (size_t)cur * c->ns;
  a.ud = c->fp64() ? c->ud + (size_t)cur * 3 * c->ns : nullptr;
  a.g0 = 2 * c->off[mol];
  a.N = N;
  a.ring = c->circular[mol];
  a.h = 0.5 * c->p.ell;
  a.rc2 = c->p.rc_hb * c->p.rc_hb;
  a.mid = c->obs_scratch;
  a.ca = a.mid + 3 * (size_t)(c->maxN + 4);
  a.cb = a.ca + 3 * (size_t)(c->maxN + 4);
  a.out = c->obs_out;
  a.inc = c->obs_scratch + 9 * (size_t)(c->maxN + 4);   // beyond the three curves
  CK(obs_launch(a, DSDNA_OBS_TW, c->st), "profiles");
  if (centre) CK(cudaMemcpyAsync(centre, a.mid, sizeof(double) * 3 * (size_t)N, cudaMemcpyDeviceToHost, c->st), "read centre");
  if (twist && ninc) CK(cudaMemcpyAsync(twist, a.inc, sizeof(double) * (size_t)ninc, cudaMemcpyDeviceToHost, c->st), "read twist");
  CK(cudaStreamSynchronize(c->st), "profiles sync");
  return DSDNA_OK;
}

extern "C" int dsdna_get_state(dsdna_ctx* c, int mol, double* X, double* V, double* u, double* Om) {
  if (!c) return DSDNA_EINVAL;
  if (mol < -1 || mol >= c->n_mol) return fail(c, DSDNA_EINVAL, "molecule index out of range");
  if (c->poisoned) {
    // Post-mortem read: the engine stopped at the step that raised the error,
    // so the state shows it; the error itself stays in last_error.
    CK(cudaStreamSynchronize(c->st), "synchronize");
  } else {
    int rc = sync_check(c);
    if (rc) return rc;
  }
  const int64_t g0 = mol < 0 ? 0 : 2 * c->off[mol];
  const int64_t cnt = mol < 0 ? c->n : 2 * (int64_t)c->n_bp[mol];
  const int cur = (int)(c->step & 1);
  k_gather_state<<<(unsigned)((cnt + 255) / 256), 256, 0, c->st>>>(c->stage, g0, cnt, c->fp64(), cur, c->ns, c->X, c->V,
                                                                    c->Om, c->U, c->ud);
  CK(cudaGetLastError(), "gather state");
  double* dst[4] = {X, V, u, Om};
  for (int r = 0; r < 4; ++r)
    if (dst[r])
      CK(cudaMemcpyAsync(dst[r], c->stage + 3 * r * cnt, sizeof(double) * 3 * cnt, cudaMemcpyDeviceToHost, c->st),
         "download state");
  CK(cudaStreamSynchronize(c->st), "download sync");
  return DSDNA_OK;
}

extern "C" int dsdna_set_state(dsdna_ctx* c, int mol, const double* X, const double* V, const double* u, const double* Om) {
  if (!c) return DSDNA_EINVAL;
  if (mol < -1 || mol >= c->n_mol) return fail(c, DSDNA_EINVAL, "molecule index out of range");
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_state sync");
  c->poisoned = false;
  c->errmsg.clear();
  CK(cudaMemsetAsync(c->err, 0, 16, c->st), "clear errors");
  const int one = 1;
  CK(cudaMemcpyAsync(c->rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, c->st), "request rebuild");
  const int64_t g0 = mol < 0 ? 0 : 2 * c->off[mol];
  const int64_t cnt = mol < 0 ? c->n : 2 * (int64_t)c->n_bp[mol];
  return upload_state(c, g0, cnt, X, V, u, Om);
}

// The rule 2 mask lives in bits RM_SHIFT.. of the device topology words.
extern "C" int dsdna_get_bubble_mask(dsdna_ctx* c, int mol, unsigned char* mask) {
  if (!c || !mask) return DSDNA_EINVAL;
  if (mol < -1 || mol >= c->n_mol) return fail(c, DSDNA_EINVAL, "molecule index out of range");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  const int64_t g0 = mol < 0 ? 0 : 2 * c->off[mol];
  const int64_t cnt = mol < 0 ? c->n : 2 * (int64_t)c->n_bp[mol];
  std::vector<int> t((size_t)cnt);
  CK(cudaMemcpy(t.data(), c->topo + g0, sizeof(int) * (size_t)cnt, cudaMemcpyDeviceToHost), "read bubble mask");
  for (int64_t i = 0; i < cnt; ++i) mask[i] = (unsigned char)((t[(size_t)i] >> RM_SHIFT) & 3);
  return DSDNA_OK;
}

extern "C" int dsdna_set_bubble_mask(dsdna_ctx* c, int mol, const unsigned char* mask) {
  if (!c) return DSDNA_EINVAL;
  if (mol < -1 || mol >= c->n_mol) return fail(c, DSDNA_EINVAL, "molecule index out of range");
  const int64_t g0 = mol < 0 ? 0 : 2 * c->off[mol];
  const int64_t cnt = mol < 0 ? c->n : 2 * (int64_t)c->n_bp[mol];
  if (mask)
    for (int64_t i = 0; i < cnt; ++i)
      if (mask[i] > 3) return fail(c, DSDNA_EINVAL, "bubble mask entries must be in 0..3");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  std::vector<int> t((size_t)cnt);
  CK(cudaMemcpy(t.data(), c->topo + g0, sizeof(int) * (size_t)cnt, cudaMemcpyDeviceToHost), "read topology");
  for (int64_t i = 0; i < cnt; ++i)
    t[(size_t)i] = (t[(size_t)i] & ~(3 << RM_SHIFT)) | ((mask ? (int)mask[i] : 0) << RM_SHIFT);
  CK(cudaMemcpy(c->topo + g0, t.data(), sizeof(int) * (size_t)cnt, cudaMemcpyHostToDevice), "write bubble mask");
  return DSDNA_OK;
}

extern "C" int dsdna_compute_forces(dsdna_ctx* c, double* Fb, double* Fp) {
  if (!c) return DSDNA_EINVAL;
  if (c->poisoned) return fail(c, DSDNA_ESTATE, "context poisoned by an earlier error");
  int rc = launch(c, MODE_FORCES, 0);
  if (rc) return rc;
  rc = sync_check(c);
  if (rc) return rc;
  std::vector<double> h((size_t)c->n * 6);
  CK(cudaMemcpy(h.data(), c->fout, sizeof(double) * h.size(), cudaMemcpyDeviceToHost), "read forces");
  for (int64_t i = 0; i < c->n; ++i)
    for (int q = 0; q < 3; ++q) {
      if (Fb) Fb[3 * i + q] = h[6 * i + q];
      if (Fp) Fp[3 * i + q] = h[6 * i + 3 + q];
    }
  return DSDNA_OK;
}

extern "C" int dsdna_neighbor_pairs(dsdna_ctx* c, int64_t cap, int64_t* pi, int64_t* pj, int64_t* count) {
  if (!c || !count) return DSDNA_EINVAL;
  if (c->poisoned) return fail(c, DSDNA_ESTATE, "context poisoned by an earlier error");
  int rc = launch(c, MODE_FORCES, 0);
  if (rc) return rc;
  rc = sync_check(c);
  if (rc) return rc;
  const size_t nn = (size_t)c->n, ns = (size_t)c->ns;
  std::vector<int> nb((size_t)c->p.max_neighbors * ns), nc(nn);
  CK(cudaMemcpy(nb.data(), c->nbr, sizeof(int) * nb.size(), cudaMemcpyDeviceToHost), "read list");
  CK(cudaMemcpy(nc.data(), c->ncnt, sizeof(int) * nc.size(), cudaMemcpyDeviceToHost), "read counts");
  int64_t k = 0;
  for (size_t i = 0; i < nn; ++i)
    for (int q = 0; q < nc[i]; ++q) {
      const int64_t j = nb[(size_t)q * ns + i] & ENT_JMASK;
      if ((int64_t)i < j) {
        if (k < cap) { pi[k] = (int64_t)i; pj[k] = j; }
        ++k;
      }
    }
  *count = k;
  return DSDNA_OK;
}

extern "C" int dsdna_get_info(const dsdna_ctx* c, dsdna_info* info) {
  if (!c || !info) return DSDNA_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->n_nt = c->n;
  info->n_mol = c->n_mol;
  info->step = c->step;
  unsigned long long nb = 0;
  cudaStreamSynchronize(c->st);
  cudaMemcpy(&nb, c->nrebuild, sizeof(nb), cudaMemcpyDeviceToHost);
  info->rebuilds = (int64_t)nb;
  cudaMemcpy(&nb, c->nlaunch, sizeof(nb), cudaMemcpyDeviceToHost);
  info->engine_launches = (int64_t)nb + c->host_launches;
  info->rebuild_in_step = c->fused ? 1 : 0;
  info->chain_list = c->chain ? 1 : 0;
  info->grid_blocks = c->grid[MODE_STEP];
  info->block_threads = c->T;
  info->max_neighbors = c->p.max_neighbors;
  info->precision = c->p.precision;
  info->skin = c->p.skin;
  info->cell_table = c->H;
  info->device_bytes = c->bytes;
  if (c->tcnt && info->rebuilds > 0) {
    std::vector<int> tc((size_t)((c->n + SEG_SLOTS - 1) / SEG_SLOTS));
    if (cudaMemcpy(tc.data(), c->tcnt, sizeof(int) * tc.size(), cudaMemcpyDeviceToHost) == cudaSuccess)
      for (int v : tc) info->halved_tiles += v >= 0 ? 1 : 0;
  }
  return DSDNA_OK;
}

extern "C" int64_t dsdna_step_counter(const dsdna_ctx* c) { return c ? c->step : -1; }

extern "C" const char* dsdna_last_error(const dsdna_ctx* c) {
  return c ? c->errmsg.c_str() : g_create_error.c_str();
}

// Autotuner: time short runs of each candidate (neighbour skin x CTA size x
// persistent CTAs per SM) on temporary contexts of the same system and keep
// the fastest.  Candidates never change the physics: the skin only sets how
// often the list is rebuilt, the launch shape only how work is spread.
extern "C" int dsdna_autotune(const dsdna_params* base, const dsdna_system* sys, const dsdna_allocator* alloc,
                              void* cuda_stream, int trial_steps, dsdna_params* best, double* best_ns) {
  if (!base || !sys || !best || trial_steps < 1) return fail(nullptr, DSDNA_EINVAL, "autotune: bad arguments");
  const double skins[] = {0.2, 0.25, 0.3, 0.35, 0.4, 0.5, 0.6};
  const int blocks[] = {128, 256, 1024};
  const int per_sm[] = {0, 2};
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(nullptr, DSDNA_ECUDA, "autotune: event creation failed");
  double best_t = 1e300;
  dsdna_params winner = *base;
  int tried = 0;
  std::string why;
  // where the automatic choice of rebuild path is close (a quarter to four
  // times its threshold), both paths are tried
  int64_t n_nt = 0;
  for (int m = 0; m < sys->n_mol; ++m) n_nt += 2 * (int64_t)std::max(0, sys->n_bp[m]);
  std::vector<int> modes{base->rebuild_mode};
  if (base->rebuild_mode == 0 && n_nt >= DSDNA_FUSED_REBUILD_MAX_NT / 4 && n_nt <= 4 * (int64_t)DSDNA_FUSED_REBUILD_MAX_NT)
    modes = {1, 2};
  // one timed trial of candidate p (ns per nucleotide-step), keeping the fastest
  auto trial = [&](const dsdna_params& p) {
    dsdna_ctx* c = nullptr;
    if (dsdna_create(&p, sys, alloc, cuda_stream, &c) != DSDNA_OK) { why = g_create_error; return; }
    float ms = 0.f;
    bool ok = dsdna_step(c, trial_steps) == DSDNA_OK && dsdna_synchronize(c) == DSDNA_OK;   // warm-up + first build
    if (ok) {
      ok = cudaEventRecord(e0, st) == cudaSuccess && dsdna_step(c, trial_steps) == DSDNA_OK &&
           cudaEventRecord(e1, st) == cudaSuccess && dsdna_synchronize(c) == DSDNA_OK &&
           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    }
    const double t = 1e6 * (double)ms / ((double)trial_steps * (double)c->n);   // ns per nucleotide-step
    if (!ok) why = c->errmsg.empty() ? std::string("event timing failed") : c->errmsg;
    dsdna_destroy(c);
    if (!ok) return;
    ++tried;
    if (t < best_t) { best_t = t; winner = p; }
  };
  for (int rm : modes)
  for (double sk : skins)
    for (int T : blocks)
      for (int ps : per_sm) {
        if (T > 256 && ps > 1) continue;   // one CTA of this size per SM at most
        dsdna_params p = *base;
        p.rebuild_mode = rm;
        p.skin = sk;
        p.block_threads = T;
        p.blocks_per_sm = ps;
        trial(p);
      }
  // the winner with the other neighbour-list build (the cell walk for the
  // chain window, or the reverse), in case this system favours it
  if (tried) {
    dsdna_params p = winner;
    p.list_build = winner.list_build == 0 ? 1 : 0;
    trial(p);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!tried) return fail(nullptr, DSDNA_ECUDA, "autotune: no candidate ran (last: " + why + ")");
  *best = winner;
  if (best_ns) *best_ns = best_t;
  return DSDNA_OK;
}

extern "C" void dsdna_destroy(dsdna_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  for (cudaEvent_t& e : c->ev)
    if (e) { cudaEventDestroy(e); e = nullptr; }
  free_all(c);
  delete c;
}
