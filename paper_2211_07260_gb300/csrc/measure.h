// Measurement of one point: a CUDA graph of back-to-back launches replayed
// under an energy-counter window (or, with a simulation table installed, the
// table's run_launches hook).
#pragma once

#include <cuda_runtime.h>

#include <functional>

#include "../../include/convtune.h"
#include "platform.h"

namespace convtune {

// What is measured: one launch of a unit, enqueued on a stream.
struct MeasureUnit {
  int kind = CT_UNIT_CONV;
  const ct_config* cfg = nullptr;          // for CT_UNIT_CONV
  double work = 0.0;                       // useful FLOP (or bytes) per launch
  std::function<int(cudaStream_t)> launch; // enqueue one launch
  bool eager = false;                      // replay by calling launch() (no graph)
};

// Defaults filled in for unset (<= 0) options.
ct_measure_options resolve_options(const ct_measure_options* opt);

// Measure a unit; `clock_req` is recorded as requested clock (0: default).
// On CT_OK the record holds time, energy, power, clocks and flags.
int measure_unit(const MeasureUnit& u, const ct_measure_options& opt, const ct_platform_ops& ops,
                 cudaStream_t order_after, int clock_req, ct_record* out);

}  // namespace convtune
