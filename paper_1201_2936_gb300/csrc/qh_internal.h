// Host-side helpers shared by the translation units of libqh.
#pragma once

#include <cuda_runtime.h>

#include "qh.h"

namespace qh {

// Grid size of a persistent (cooperative) launch of `func` with `block`
// threads: SMs x resident CTAs per SM (capped by blocks_per_sm when > 0).
// Returns 0 on a CUDA error.
int persistent_grid(const void *func, int block, int blocks_per_sm);
// The same for a kernel launched with `dsmem` bytes of dynamic shared memory.
int persistent_grid_smem(const void *func, int block, int blocks_per_sm, size_t dsmem);
// Streaming multiprocessors of the current device (cached per device; 1 on
// a CUDA error, so that grid sizes stay valid).
int sm_count();
// Workspace of the persistent k-th element selection (qh_select).
size_t select_workspace_bytes(long long n, int nseg);

}  // namespace qh
