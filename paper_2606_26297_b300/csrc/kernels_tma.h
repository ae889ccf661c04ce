// Launchers of the TMA-pipelined persistent layer-pass kernels.
#pragma once

#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "qaoa_internal.h"

namespace qaoa {

// grid: number of persistent CTAs (one per SM); status: device word set to a
// non-zero value if a bounded wait timed out.
cudaError_t launch_fwd_tma(int type, bool epi, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);
cudaError_t launch_rev_tma(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);

// Final forward pass writing the interleaved (psi, lambda) buffer a.pl, and the
// reverse pass on that buffer (kernels_rev2.cu).
cudaError_t launch_epi_pl(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);
cudaError_t launch_rev_pl(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);

// 512-thread variants (kernels_v3.cu): forward pass, final forward pass of a
// gradient evaluation (writes a.pl), reverse pass on a.pl.
cudaError_t launch_fwd3(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);
cudaError_t launch_epi3(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);
cudaError_t launch_rev3(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);

// Tensor map of the 5-D high-group block view (see kernels_tma.cu).
cudaError_t make_block_map(CUtensorMap *map, const void *base, int n, int lo, int esize);

}  // namespace qaoa
