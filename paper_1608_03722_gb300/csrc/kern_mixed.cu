// kern_mixed.cu -- engine kernels with FP32 forces and FP64 position/velocity accumulation.
#include "kern_launch.cuh"
namespace dsdna {
template cudaError_t engine_occupancy<float>(int, int, int*, size_t*);
template cudaError_t engine_launch<float>(int, const KArgs<float>&, int, int, size_t, cudaStream_t);
template cudaError_t rebuild_launch<float>(const KArgs<float>&, int, cudaStream_t);
template cudaError_t rebuild_prepare<float>();
}  // namespace dsdna
