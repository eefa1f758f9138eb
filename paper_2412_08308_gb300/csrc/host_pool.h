// Host-side allocation helper shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

namespace swgb {

// Stream-ordered allocation from the library's memory pool of the current
// device (freed blocks stay reserved up to 1 GiB, so that the next
// allocation maps no fresh memory, where the process's default pool returns
// its memory at every synchronisation); free with cudaFreeAsync.
cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t s);

}  // namespace swgb
