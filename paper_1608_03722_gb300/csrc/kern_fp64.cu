// kern_fp64.cu -- engine kernels with every quantity in FP64 (reference precision on the GPU).
#include "kern_launch.cuh"
namespace dsdna {
template cudaError_t engine_occupancy<double>(int, int, int*, size_t*);
template cudaError_t engine_launch<double>(int, const KArgs<double>&, int, int, size_t, cudaStream_t);
template cudaError_t rebuild_launch<double>(const KArgs<double>&, int, cudaStream_t);
template cudaError_t rebuild_prepare<double>();
}  // namespace dsdna
