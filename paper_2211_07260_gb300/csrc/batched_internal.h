// Internal interface of the batched kernel for other units of the library.
#pragma once

#include <cuda_runtime.h>

#include "../../include/convtune.h"
#include "batched.cuh"

namespace convtune {

// Fill one table entry from a caller's item (device in/out, taps pointer
// `it.filt` must already point at k rows of round_up(k, 4) device floats);
// grows *smem to the entry's shared-memory need.
int batch_image_from_item(const ct_batch_item& it, const ct_batch_tiles* tiles, BatchImage* im,
                          size_t* smem);

// Launch the persistent batched kernel over a device table (counter must be
// zero), occupancy-sized grid.
int launch_batched_kernel(const BatchArgs& a, size_t smem, int sms, cudaStream_t s);

}  // namespace convtune
