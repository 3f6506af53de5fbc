// nss_kernels.h -- host-side launchers of the Nested Slice Sampling kernels.
#pragma once
#include <cuda_runtime.h>

#include "nss_internal.h"

namespace nss {

struct VolLaunch {
  const int2* tiles;
  const int* vbase;
  int n_tiles, R;
  double *tsum, *toff, *tmax, *tacc;
};

cudaError_t launch_init(int cfg, const Dev& D, const WorkItem* items, int n, cudaStream_t s);
cudaError_t launch_prologue(const Dev& D, int n_runs, size_t smem, cudaStream_t s);
cudaError_t launch_sweep(int cfg, const Dev& D, const WorkItem* items, int n, int* queue, int grid,
                         cudaStream_t s);
cudaError_t launch_terminate(const Dev& D, int n_runs, cudaStream_t s);
cudaError_t launch_final_sort(const Dev& D, int n_runs, size_t smem, cudaStream_t s);
cudaError_t launch_volsim(const Dev& D, const VolLaunch& V, int n_runs, cudaStream_t s);
int sweep_blocks_per_sm(int cfg);
int cfg_g(int cfg);
int cfg_dpl(int cfg);

}  // namespace nss
