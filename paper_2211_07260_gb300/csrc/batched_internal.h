// Internal interface of the batched kernel for other units of the library.
#pragma once

#include <cuda_runtime.h>

#include "../../include/convtune.h"
#include <vector>

#include "batched.cuh"

namespace convtune {

// Fill one table entry from a caller's item (device in/out; im->filt is left
// null for the caller to point at k rows of round_up(k, 4) device floats):
// tile from `tiles` (or the default), staging geometry, and the TMA tensor
// map of the input when it is 16-byte aligned (else cp.async staging).
// first_item and tap_off are the caller's / the plan's to set.  Host only;
// allocates nothing.
int batch_image_from_item(const ct_batch_item& it, const ct_batch_tiles* tiles, BatchImage* im);

// Launch plan of a host copy of a batch table, which must be ordered by
// filter-side class (batch_class_of, ascending).  Each class's contiguous run
// of images gets a persistent kernel with that run's shared memory and an
// occupancy-sized grid; the 13..17 class is cut into runs whose taps
// (host_taps[q]: k x k row-major, host) fit one launch's parameter block.
// The plan sets each entry's tap_off, so copy the table to the device after
// planning.  host_taps may be NULL (taps then come from shared memory).  The
// first call per device raises the class kernels' shared-memory caps (make
// it before any stream capture).
struct BatchClassLaunch {
  int cls = 0;                // filter-side class
  int lo = 0, hi = 0, n = 0;  // run of the table
  long long items = 0;        // work items of the run
  long long item_base = 0;    // first_item of its first image
  size_t smem = 0;            // dynamic shared memory per CTA
  int buf_floats = 0;         // floats of each staging buffer (largest of the run)
  int threads = 0;            // CTA size (the class's)
  int claim = 1;              // work items per claim (the class's)
  int stages = 2;             // staging buffers
  int grid = 0;               // persistent CTAs
  std::vector<float> taps;    // the run's parameter-block taps (KP-padded rows)
};
struct BatchPlan {
  std::vector<BatchClassLaunch> launches;
  int total_grid = 0;
  size_t max_smem = 0;
};
int plan_batch(BatchImage* table, int n, const float* const* host_taps, BatchPlan* plan);

// Enqueue a planned batch over the device copy of the same table: zeroes one
// work counter per launch at `counters` (kBatchCounterBytes of device
// memory), then launches the kernels one after another on `s` or, with
// n_branches branch streams and n_branches + 1 events, launch l on branch
// l % n_branches, the branches forked from and joined back into `s`.
int enqueue_batch_plan(const BatchPlan& plan, const BatchImage* d_table, unsigned* counters,
                       unsigned* status, cudaStream_t s, const cudaStream_t* branches = nullptr,
                       const cudaEvent_t* events = nullptr, int n_branches = 0);

}  // namespace convtune
