// Internal runtime of libconvtune: problem / configuration validation, the
// launch plan of one correlation, and per-device scratch.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <string>

#include "../../include/convtune.h"
#include "conv2d_launch.h"

namespace convtune {

// Everything needed to launch one correlation, resolved from (problem,
// config) by plan_conv().
struct ConvPlan {
  ConvLaunch L{};
  bool specialised = false;  // square odd filter <= 17
  bool empty = false;        // out_h == 0 or out_w == 0: nothing to launch
  const void* fn = nullptr;  // kernel function
  dim3 grid, block;
  CUtensorMap tmap;          // filled when staging == TMA
};

// Validate and resolve; returns CT_OK / CT_EINVAL / CT_ECONFIG / CT_ENOTSUP /
// CT_ECUDA.  `why` receives a reason when not OK.  device_checks = false
// skips the checks that need a CUDA device (register and shared-memory
// limits), for simulated measurement.
int plan_conv(const ct_problem& p, const ct_config& c, ConvPlan* plan, std::string* why,
              bool device_checks = true);

// cuTensorMapEncodeTiled from the driver (null if unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// Launch a resolved plan on a stream.
int launch_plan(ConvPlan& plan, cudaStream_t s);

// Load the specialised K x K kernel variant of configuration c and raise its
// shared-memory cap now, ahead of its first launch: kernel code is loaded on
// first use, which otherwise stalls that launch's caller for milliseconds.
int prime_conv_kernel(int k, const ct_config& c);

// Device status word of the current device (allocated on first use).
unsigned* device_status_word(int* err);

// Map a CUDA error to a status code (and remember its text for ct_strerror
// callers that want detail).
int cuda_status(cudaError_t e);

// Record a message for ct_last_error() (argument errors worth explaining).
void set_last_error(const char* msg);

// Useful work of one correlation: 2 * fh * fw * out_h * out_w FLOP.
double conv_flop(const ct_problem& p);
// Algorithmic bytes of one correlation: padded input read once, output
// written once, taps once.
double conv_bytes(const ct_problem& p);

}  // namespace convtune
