// kern_launch.cuh -- host-side launch of the persistent engine kernel for one
// precision; included once per precision by kern_mixed.cu / kern_fp64.cu.
#pragma once
#include "engine_kernels.cuh"

namespace dsdna {

constexpr int CAPMAX = 64;

template <class Real>
static const void* engine_fn(int mode) {
  switch (mode) {
    case MODE_STEP: return (const void*)engine_kernel<Real, MODE_STEP, CAPMAX>;
    case MODE_FORCES: return (const void*)engine_kernel<Real, MODE_FORCES, CAPMAX>;
    default: return (const void*)engine_kernel<Real, MODE_ENERGY, CAPMAX>;
  }
}

// Largest co-resident grid for the cooperative launch of `mode` with T threads.
template <class Real>
cudaError_t engine_occupancy(int mode, int T, int* blocks_per_sm, size_t* smem) {
  *smem = seg_smem_bytes<Real>(T);
  const void* fn = engine_fn<Real>(mode);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
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
  switch (mode) {
    case MODE_STEP: return cudaLaunchKernelEx(&cfg, engine_kernel<Real, MODE_STEP, CAPMAX>, a);
    case MODE_FORCES: return cudaLaunchKernelEx(&cfg, engine_kernel<Real, MODE_FORCES, CAPMAX>, a);
    default: return cudaLaunchKernelEx(&cfg, engine_kernel<Real, MODE_ENERGY, CAPMAX>, a);
  }
}

}  // namespace dsdna
