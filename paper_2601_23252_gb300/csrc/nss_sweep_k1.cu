// nss_sweep_k1.cu -- the HRSS sweep kernels for at most 1 mixture component.
#include "nss_sweep_chain.cuh"

namespace nss {

template cudaError_t launch_sweep_kc<1>(int, const Dev&, const WorkItem*, int, int*, int, cudaStream_t);
template int sweep_blocks_per_sm_kc<1>(int);

}  // namespace nss
