// kern_launch.cuh -- host-side launch of the persistent engine kernel for one
// precision; included once per precision by kern_mixed.cu / kern_fp64.cu.
#pragma once
#include <algorithm>

#include "engine_kernels.cuh"
#include "rebuild.cuh"
#include "chainlist.cuh"

namespace dsdna {

constexpr int CAPMAX = 64;

// mode | MODE_EXT selects the instance with circular molecules and the bubble
// rule, MODE_STEP | MODE_FUSED the one that rebuilds the list in the kernel.
template <class Real, bool EXT>
static const void* engine_fn_ext(int mode) {
  switch (mode & 3) {
    case MODE_STEP:
      return (mode & MODE_FUSED) ? (const void*)engine_kernel<Real, MODE_STEP, CAPMAX, EXT, true>
                                 : (const void*)engine_kernel<Real, MODE_STEP, CAPMAX, EXT, false>;
    case MODE_FORCES: return (const void*)engine_kernel<Real, MODE_FORCES, CAPMAX, EXT>;
    default: return (const void*)engine_kernel<Real, MODE_ENERGY, CAPMAX, EXT>;
  }
}
template <class Real>
static const void* engine_fn(int mode) {
  return (mode & MODE_EXT) ? engine_fn_ext<Real, true>(mode) : engine_fn_ext<Real, false>(mode);
}

// Largest co-resident grid for the cooperative launch of `mode` with T threads
// (T above engine_max_threads<Real>() has no resident CTA: 0).
template <class Real>
cudaError_t engine_occupancy(int mode, int T, int* blocks_per_sm, size_t* smem) {
  if (T > engine_max_threads<Real>()) {
    *blocks_per_sm = 0;
    return cudaSuccess;
  }
  *smem = seg_smem_bytes<Real>(T);
  const void* fn = engine_fn<Real>(mode);
  // the attribute is per kernel, shared by every context: allow the largest CTA any context may use
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)seg_smem_bytes<Real>(engine_max_threads<Real>()));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, T, *smem);
}

template <class Real>
cudaError_t engine_launch(int mode, const KArgs<Real>& a, int grid, int T, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)T);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // the instance chosen by mode, launched with its parameter block
  void* args[] = {const_cast<KArgs<Real>*>(&a)};
  return cudaLaunchKernelExC(&cfg, engine_fn<Real>(mode), args);
}

// Kernel attributes of the rebuild kernels for the current device, set when a
// context is created: the chain-window list build asks for the largest
// shared-memory carveout, so that four of its CTAs (47 KB of shared memory
// each) are resident per SM.
template <class Real>
cudaError_t rebuild_prepare() {
  return cudaFuncSetAttribute(k_rebuild_list_chain<Real>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

// The rebuild kernels on stream st (grid-stride; the scan pair shares one grid):
// five for the chain-window build, five or six (pair halving) for the cell walks.
template <class Real>
cudaError_t rebuild_launch(const KArgs<Real>& a, int scan_grid, cudaStream_t st) {
  const int T = 256;
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (a.n + T - 1) / T;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * 16));
  if (a.segc) {
    // chain-window build (periodic box): segment grid (bin, scan, scatter),
    // then one warp per 32-slot tile builds its lists and their pair halving
    KArgs<Real> as = a;
    as.H = a.sg_H;
    const int sgrid = std::max(1, std::min(scan_grid, (int)((a.sg_H + 2047u) / 2048u)));
    k_rebuild_segbin<Real><<<grid, T, 0, st>>>(a);
    k_rebuild_scan_a<Real><<<sgrid, T, 0, st>>>(as);
    k_rebuild_scan_b<Real><<<sgrid, T, 0, st>>>(as);
    const int64_t swant = (a.nseg16 + T - 1) / T;
    k_rebuild_segscatter<Real><<<(int)std::max<int64_t>(1, std::min<int64_t>(swant, (int64_t)nsm * 16)), T, 0, st>>>(a);
    int cbps = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cbps, k_rebuild_list_chain<Real>, CL_WARPS * 32, 0);
    const int cgrid = (int)std::max<int64_t>(
        1, std::min<int64_t>((a.nseg + CL_WARPS - 1) / CL_WARPS, (int64_t)nsm * std::max(1, cbps)));
    k_rebuild_list_chain<Real><<<cgrid, CL_WARPS * 32, 0, st>>>(a);
    return cudaGetLastError();
  }
  k_rebuild_bin<Real><<<grid, T, 0, st>>>(a);
  k_rebuild_scan_a<Real><<<scan_grid, T, 0, st>>>(a);
  k_rebuild_scan_b<Real><<<scan_grid, T, 0, st>>>(a);
  k_rebuild_scatter<Real><<<grid, T, 0, st>>>(a);
  const int LT = LIST_WARPS * 32;
  int lbps = 1;
  if (a.table == TABLE_LINEAR) {
    // one lane per bead
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lbps, k_rebuild_list_lanes<Real>, LT, 0);
    const int lgrid = (int)std::max<int64_t>(1, std::min<int64_t>((a.n + LT - 1) / LT, (int64_t)nsm * std::max(1, lbps)));
    k_rebuild_list_lanes<Real><<<lgrid, LT, 0, st>>>(a);
  } else if (a.table == TABLE_HASH) {
    // open box: one lane per bead over the row ranges of the hashed blocks
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lbps, k_rebuild_list_lanes_hash<Real>, LT, 0);
    const int lgrid = (int)std::max<int64_t>(1, std::min<int64_t>((a.n + LT - 1) / LT, (int64_t)nsm * std::max(1, lbps)));
    k_rebuild_list_lanes_hash<Real><<<lgrid, LT, 0, st>>>(a);
  } else {
    // one warp per 32 table entries at a time: enough CTAs for every chunk of
    // a small table, at most a full wave for a large one
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lbps, k_rebuild_list<Real, CAPMAX>, LT, 0);
    const int lgrid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)a.H + 32 * LIST_WARPS - 1) / (32 * LIST_WARPS),
                                                                  (int64_t)nsm * std::max(1, lbps)));
    k_rebuild_list<Real, CAPMAX><<<lgrid, LT, 0, st>>>(a);
  }
  if (a.evl) {   // pair halving: the tiles' evaluated pairs, one resident wave of warps
    int pbps = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pbps, k_rebuild_pack<Real>, PACK_WARPS * 32, 0);
    const int pgrid = (int)std::max<int64_t>(
        1, std::min<int64_t>((a.nseg + PACK_WARPS - 1) / PACK_WARPS, (int64_t)nsm * std::max(1, pbps)));
    k_rebuild_pack<Real><<<pgrid, PACK_WARPS * 32, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace dsdna
