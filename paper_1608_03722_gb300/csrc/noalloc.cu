// noalloc.cu -- conservative forces of the dsDNA model for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: processes whose device memory is
// entirely reserved by another pool allocator, and tight loops that cannot
// afford the device-wide synchronisation that cudaMalloc/cudaFree imply.
// dsdna_forces_noalloc gives them the force pass of the engine (the same
// persistent kernel in its forces mode: cell hash, neighbour list, bonded and
// pair forces) with all of its scratch memory in one file-scope device array
// of fixed size.  That array is reserved on every GPU that loads the library
// and stays there until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/dsdna.h"
#include "engine.cuh"

namespace dsdna {
template <class Real> cudaError_t engine_occupancy(int mode, int T, int* blocks_per_sm, size_t* smem);
template <class Real> cudaError_t engine_launch(int mode, const KArgs<Real>& a, int grid, int T, size_t smem, cudaStream_t st);
template <class Real> cudaError_t rebuild_launch(const KArgs<Real>& a, int scan_grid, cudaStream_t st);
__attribute__((visibility("hidden"))) void fill_coef_mixed(const dsdna_params& p, Coef<float>& c);
}  // namespace dsdna

using namespace dsdna;

namespace {

constexpr int64_t NA_MAX_NT = DSDNA_NOALLOC_MAX_NT;   // nucleotides
constexpr int NA_MAX_MOL = DSDNA_NOALLOC_MAX_MOL;     // molecules
constexpr unsigned NA_MAX_H = 32768u;                 // cell-table entries
constexpr int NA_CAP = 32;                            // neighbours per bead
constexpr int NA_T = 256;                             // threads per CTA
constexpr int NA_MAX_GRID = 4096;

constexpr size_t al(size_t b) { return (b + 255) & ~(size_t)255; }
// byte offsets of the pieces of the scratch array
constexpr size_t O_X = 0;
constexpr size_t O_KW = O_X + al(3 * NA_MAX_NT * sizeof(double));
constexpr size_t O_U = O_KW + al(NA_MAX_NT * sizeof(int4));
constexpr size_t O_TOPO = O_U + al(NA_MAX_NT * sizeof(float4));
constexpr size_t O_IMG = O_TOPO + al(NA_MAX_NT * sizeof(int));
constexpr size_t O_KREF = O_IMG + al(NA_MAX_NT * sizeof(int));
constexpr size_t O_NBR = O_KREF + al(3 * NA_MAX_NT * sizeof(int));
constexpr size_t O_NCNT = O_NBR + al((size_t)NA_CAP * NA_MAX_NT * sizeof(int));
constexpr size_t O_KEY = O_NCNT + al(NA_MAX_NT * sizeof(int));
constexpr size_t O_CENT = O_KEY + al(NA_MAX_NT * sizeof(int));
constexpr size_t O_WPOS = O_CENT + al(NA_MAX_NT * sizeof(float4));
constexpr size_t O_FOUT = O_WPOS + al(NA_MAX_NT * sizeof(float4));
constexpr size_t O_CNT = O_FOUT + al(6 * NA_MAX_NT * sizeof(double));
constexpr size_t O_START = O_CNT + al(NA_MAX_H * sizeof(unsigned));
constexpr size_t O_BSUM = O_START + al((NA_MAX_H + 1) * sizeof(unsigned));
constexpr size_t O_MOLOFF = O_BSUM + al(NA_MAX_GRID * sizeof(unsigned));
constexpr size_t O_EXT = O_MOLOFF + al((NA_MAX_MOL + 1) * sizeof(int64_t));
constexpr size_t O_BAR = O_EXT + al((size_t)NA_MAX_MOL * 8 * sizeof(double));
constexpr size_t O_CTRL = O_BAR + al(sizeof(GridBar));   // err (16 B), step (8 B), rebuild (4 B), nrebuild (8 B)
constexpr size_t NA_BYTES = O_CTRL + 256;

}  // namespace

// The scratch memory itself.  In host code this name is only a host-side
// stand-in: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {

struct DeviceSetup {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch on this device
  int grid = 0;
  size_t smem = 0;
};
constexpr int NA_MAX_DEV = 64;
DeviceSetup g_setup[NA_MAX_DEV];
std::mutex g_setup_mutex;

// error codes only: this entry point keeps no message state
inline int na_fail(int code, const char* /*why*/) { return code; }

// Once per device, with that device current: device address of the scratch
// array and the co-resident grid of the force kernel.
int setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return na_fail(DSDNA_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
    int bps = 0, nsm = 0;
    e = engine_occupancy<float>(MODE_FORCES, NA_T, &bps, &s.smem);
    if (e != cudaSuccess || bps < 1) return na_fail(DSDNA_ECUDA, "occupancy query of the force kernel failed");
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return na_fail(DSDNA_ECUDA, "device attribute query failed");
    s.grid = std::min(bps * nsm, NA_MAX_GRID);
    s.base = static_cast<unsigned char*>(p);
    s.ready = true;
  }
  *out = &s;
  return DSDNA_OK;
}

// Stage the caller's configuration into the scratch array: topology flags of
// Sec. 2 (no anchored or loaded base pairs), SoA centres, fixed-point mirror,
// FP32 orientation; zero the cell counts' companions and the control words.
__global__ void k_noalloc_prep(const double* X, const double* u, int64_t n, int64_t ns, int n_mol, const int64_t* mol_off,
                               int steric_phase, double* Xs, int4* Kw, float4* U, int* topo, unsigned* ctrl, double S0,
                               double S1, double S2) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) {
    ctrl[0] = 0u;                                   // error word
    *reinterpret_cast<int64_t*>(ctrl + 4) = 0;      // step counter
    ctrl[6] = 1u;                                   // rebuild request
    *reinterpret_cast<unsigned long long*>(ctrl + 8) = 0ull;
  }
  if (g >= n) return;
  const int64_t bp = g / 2;
  int lo = 0, hi = n_mol - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (mol_off[mid] <= bp) lo = mid; else hi = mid - 1;
  }
  const int m = lo;
  const int N = (int)(mol_off[m + 1] - mol_off[m]);
  const int k = (int)(bp - mol_off[m]);
  const int s = (int)(g & 1);
  const int q = s == 0 ? k : N - 1 - k;
  int f = 0;
  if (q % 3 == steric_phase) f |= F_STERIC;
  if (q > 0) f |= F_PREV;
  if (q < N - 1) f |= F_NEXT;
  topo[g] = f | (m << MOL_SHIFT);
  const double x0 = X[3 * g], x1 = X[3 * g + 1], x2 = X[3 * g + 2];
  Xs[g] = x0; Xs[ns + g] = x1; Xs[2 * ns + g] = x2;
  Kw[g] = make_int4(fixs(x0, S0), fixs(x1, S1), fixs(x2, S2), 0);
  double u0 = u[3 * g], u1 = u[3 * g + 1], u2 = u[3 * g + 2];
  const double l2 = u0 * u0 + u1 * u1 + u2 * u2;
  if (fabs(l2 - 1.0) > 1e-6) { const double l = sqrt(l2); u0 /= l; u1 /= l; u2 /= l; }
  U[g] = make_float4((float)u0, (float)u1, (float)u2, 0.0f);
}

__global__ void k_noalloc_split(const double* fout, int64_t n, double* Fb, double* Fp) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  for (int c = 0; c < 3; ++c) {
    Fb[3 * g + c] = fout[6 * g + c];
    Fp[3 * g + c] = fout[6 * g + 3 + c];
  }
}

}  // namespace

extern "C" int dsdna_forces_noalloc(const dsdna_params* p, int n_mol, const int* n_bp, const double* X, const double* u,
                                    double* F_bead, double* F_patch, void* cuda_stream) {
  if (!p || !n_bp || !X || !u || !F_bead || !F_patch) return na_fail(DSDNA_EINVAL, "null argument");
  if (n_mol < 1 || n_mol > NA_MAX_MOL) return na_fail(DSDNA_EINVAL, "n_mol must be in [1, DSDNA_NOALLOC_MAX_MOL]");
  if (p->precision != DSDNA_PREC_MIXED) return na_fail(DSDNA_EINVAL, "only the mixed-precision force pass has a no-alloc variant");
  // the checks dsdna_create makes on the parameters this call uses
  if (p->skin < 0.0 || p->skin > 1.0) return na_fail(DSDNA_EINVAL, "skin must be in [0, 1] nm");
  if (p->bubble_rule < 0 || p->bubble_rule > 2) return na_fail(DSDNA_EINVAL, "bubble_rule must be 0, 1 or 2");
  if (p->steric_phase < 0 || p->steric_phase > 2) return na_fail(DSDNA_EINVAL, "steric_phase must be 0, 1 or 2");
  if (!(p->ell > 0.0) || !(p->R0 > 0.0) || !(p->rc_hb > 0.0)) return na_fail(DSDNA_EINVAL, "non-positive ell/R0/rc");
  if (p->K2_gc < 0.0) return na_fail(DSDNA_EINVAL, "K2_gc must be >= 0");
  int64_t mol_off[NA_MAX_MOL + 1];
  mol_off[0] = 0;
  for (int m = 0; m < n_mol; ++m) {
    if (n_bp[m] < 1) return na_fail(DSDNA_EINVAL, "molecule with fewer than one base pair");
    mol_off[m + 1] = mol_off[m] + n_bp[m];
  }
  const int64_t n = 2 * mol_off[n_mol];
  if (n > NA_MAX_NT) return na_fail(DSDNA_EINVAL, "more nucleotides than DSDNA_NOALLOC_MAX_NT");
  dsdna_params q = *p;          // skin 0 means the default, as in dsdna_create
  if (q.skin == 0.0) q.skin = 0.3;
  const double skin = q.skin;
  const double rc6 = std::pow(2.0, 1.0 / 6.0);
  const double cellh = (rc6 * std::max({p->sigma_ss, p->sigma_cross, p->sigma_cross_steric}) + skin + 0.01) * 1.0001;
  const bool periodic = p->box[0] > 0.0;
  int nc[3] = {0, 0, 0};
  unsigned H = 1024;
  int morton_bits = 0, table = TABLE_HASH;
  if (periodic) {
    int bits = 1;
    for (int k = 0; k < 3; ++k) {
      if (!(p->box[k] > 0.0)) return na_fail(DSDNA_EINVAL, "box must be periodic in all or no directions");
      nc[k] = (int)std::floor(p->box[k] / cellh);
      if (nc[k] < 1) return na_fail(DSDNA_EINVAL, "periodic box smaller than the interaction range");
      while ((1 << bits) < nc[k]) ++bits;
    }
    if (3 * bits > 15) return na_fail(DSDNA_EINVAL, "periodic box too wide for the fixed cell table (32 cells per edge)");
    if (nc[0] >= 3 && nc[1] >= 3 && nc[2] >= 3) {
      table = TABLE_LINEAR;
      H = (unsigned)(((unsigned)nc[0] * nc[1] * nc[2] + 2047u) / 2048u * 2048u);
    } else {
      table = TABLE_MORTON;
      morton_bits = bits;
      H = 1u << (3 * bits);
    }
  } else {
    while ((int64_t)H < 2 * n) H <<= 1;
  }
  if (H > NA_MAX_H) return na_fail(DSDNA_EINVAL, "cell table exceeds the fixed scratch");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return na_fail(DSDNA_ECUDA, "no current CUDA device");
  DeviceSetup* s = nullptr;
  int rc = setup_device(dev, &s);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned char* b = s->base;

  KArgs<float> a{};
  fill_coef_mixed(q, a.c);   // list radius from the same skin as the cell edge
  a.n = n; a.ns = NA_MAX_NT; a.n_mol = n_mol; a.nseg = (n + 31) / 32; a.cap = NA_CAP;
  a.nsteps = 0; a.noise_mode = 0;
  philox_key_schedule(a, 0);
  a.bubble = p->bubble_rule ? 1 : 0;   // one evaluation without history: rule 2 removes what rule 1 does
  const bool ext = a.bubble != 0;
  a.n_junc = 0; a.jslot = nullptr; a.jidx = nullptr; a.jout = nullptr;   // linear molecules only
  a.spin_budget = 4000000000ull;
  a.X = reinterpret_cast<double*>(b + O_X);
  a.V = nullptr; a.Om = nullptr;
  a.Kw = reinterpret_cast<int4*>(b + O_KW);
  a.U = reinterpret_cast<float4*>(b + O_U);
  a.ud = nullptr;
  a.topo = reinterpret_cast<int*>(b + O_TOPO);
  a.img = reinterpret_cast<int*>(b + O_IMG);
  a.kref = reinterpret_cast<int*>(b + O_KREF);
  a.nbr = reinterpret_cast<int*>(b + O_NBR);
  a.ncnt = reinterpret_cast<int*>(b + O_NCNT);
  a.cnt = reinterpret_cast<unsigned*>(b + O_CNT);
  a.start = reinterpret_cast<unsigned*>(b + O_START);
  a.H = H; a.table = table; a.morton_bits = morton_bits;
  a.key = reinterpret_cast<int*>(b + O_KEY);
  a.cent = reinterpret_cast<float4*>(b + O_CENT);
  a.wpos = reinterpret_cast<float4*>(b + O_WPOS);
  a.bsum = reinterpret_cast<unsigned*>(b + O_BSUM);
  a.periodic = periodic ? 1 : 0;
  for (int k = 0; k < 3; ++k) {
    a.nc[k] = nc[k];
    a.L[k] = periodic ? p->box[k] : 0.0;
    a.Lf[k] = (float)a.L[k];
    a.cellh[k] = (float)(periodic ? p->box[k] / nc[k] : cellh);
    a.invcellh[k] = 1.0f / a.cellh[k];
    a.invLf[k] = periodic ? (float)(1.0 / a.L[k]) : 0.0f;
    mirror_scale(a, k);
  }
  a.mol_off = reinterpret_cast<int64_t*>(b + O_MOLOFF);
  a.ext = reinterpret_cast<double*>(b + O_EXT);
  a.bar = reinterpret_cast<GridBar*>(b + O_BAR);
  unsigned* ctrl = reinterpret_cast<unsigned*>(b + O_CTRL);
  a.err = ctrl;
  a.step = reinterpret_cast<int64_t*>(ctrl + 4);
  a.rebuild = reinterpret_cast<int*>(ctrl + 6);
  a.nrebuild = reinterpret_cast<unsigned long long*>(ctrl + 8);
  a.fout = reinterpret_cast<double*>(b + O_FOUT);
  a.eout = nullptr;
  a.steps_left = nullptr; a.use_cond = 0; a.h_while = 0;

  // the scratch keeps the previous call's contents: clear what must start at zero
  cudaError_t e = cudaMemcpyAsync(b + O_MOLOFF, mol_off, sizeof(int64_t) * (n_mol + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.cnt, 0, sizeof(unsigned) * H, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.bar, 0, sizeof(GridBar), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.ncnt, 0, sizeof(int) * n, st);
  if (e != cudaSuccess) return na_fail(DSDNA_ECUDA, cudaGetErrorString(e));
  k_noalloc_prep<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, u, n, NA_MAX_NT, n_mol, a.mol_off, p->steric_phase, a.X, a.Kw, a.U,
                                                               a.topo, ctrl, a.fixS[0], a.fixS[1], a.fixS[2]);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(DSDNA_ECUDA, cudaGetErrorString(e));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(s->grid, (n + NA_T - 1) / NA_T));
  const int scan_grid = (int)std::min<int64_t>(NA_MAX_GRID, std::max<int64_t>(1, ((int64_t)H + 2047) / 2048));
  e = rebuild_launch<float>(a, scan_grid, st);
  // the bubble rule runs in the kernel instance that has it (same launch bounds, so the same grid fits)
  if (e == cudaSuccess) e = engine_launch<float>(MODE_FORCES | (ext ? MODE_EXT : 0), a, grid, NA_T, s->smem, st);
  if (e != cudaSuccess) return na_fail(DSDNA_ECUDA, cudaGetErrorString(e));
  k_noalloc_split<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.fout, n, F_bead, F_patch);
  e = cudaGetLastError();
  unsigned bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, ctrl, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(DSDNA_ECUDA, cudaGetErrorString(e));
  if (bits & B_EFENE) return na_fail(DSDNA_EFENE, "backbone bond reached R0 (FENE diverges)");
  if (bits & B_ENAN) return na_fail(DSDNA_ENAN, "non-finite force");
  if (bits & (B_EOVF | B_EIMG)) return na_fail(DSDNA_EOVERFLOW, "neighbour list capacity or image range exceeded");
  if (bits & B_ETIMEOUT) return na_fail(DSDNA_ETIMEOUT, "device barrier timed out");
  return DSDNA_OK;
}
