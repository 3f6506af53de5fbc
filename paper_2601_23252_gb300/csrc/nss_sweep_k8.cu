// nss_sweep_k8.cu -- the HRSS sweep kernels for at most 8 mixture components.
#include "nss_sweep_chain.cuh"

namespace nss {

template cudaError_t launch_sweep_kc<8>(int, const Dev&, const WorkItem*, int, int*, int, cudaStream_t);
template int sweep_blocks_per_sm_kc<8>(int);

}  // namespace nss
