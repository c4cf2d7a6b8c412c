// obs.h -- arguments of the observable reductions (observables.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dsdna {

struct ObsArgs {
  const double* X;    // [3][n] centres (FP64)
  const float4* uf;   // [n] orientation (mixed precision) or nullptr
  const double* ud;   // [3][n] orientation (FP64) when uf == nullptr
  int64_t n;          // row stride of the [3][n] arrays (nucleotides rounded up to 32)
  int64_t g0;         // first slot of the molecule
  int N;              // base pairs of the molecule
  int ring;           // 1: circular molecule (closed strands, no closure path)
  double h;           // ell / 2
  double rc2;         // hydrogen-bond break distance squared
  double* mid;        // [3*N] scratch
  double* ca;         // [3*(N+4)] scratch: closed curve of strand A
  double* cb;         // [3*(N+4)] scratch: closed curve of strand B
  double* out;        // [8]: rz, broken count, tw, -, lk
  double* inc;        // [N-2] (ring: [N]) twist increments in turns, or nullptr
};

cudaError_t obs_launch(const ObsArgs& a, unsigned flags, cudaStream_t st);

}  // namespace dsdna
