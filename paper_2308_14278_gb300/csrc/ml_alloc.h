// Device memory of the library.
#pragma once

#include <cuda_runtime.h>

#include <stddef.h>

namespace ml {

// Stream-ordered allocations from a pool per device that the library owns
// (ml_api.cu) and that keeps freed memory for later allocations, instead of
// handing it back to the driver at every synchronisation: a field's create
// re-allocates its node and map buffers, and mapping them anew each time
// showed in its host time.  Freed with cudaFreeAsync or cudaFree like any
// stream-ordered allocation.
cudaError_t ml_malloc_async(void **p, size_t bytes, cudaStream_t s);

}  // namespace ml
