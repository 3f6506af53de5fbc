// nss_sweep_k4.cu -- the HRSS sweep kernels for at most 4 mixture components.
#include "nss_sweep_chain.cuh"

namespace nss {

template cudaError_t launch_sweep_kc<4>(int, const Dev&, const WorkItem*, int, int*, int, cudaStream_t);
template int sweep_blocks_per_sm_kc<4>(int);

}  // namespace nss
