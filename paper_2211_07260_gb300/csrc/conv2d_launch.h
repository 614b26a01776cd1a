// Host-side launch description shared by the runtime and the per-filter-size
// instantiation units (one translation unit per specialised filter side K,
// compiled in parallel).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace convtune {

// Kernel status bits written to the library's device status word.
enum : unsigned {
  kStatusTmaTimeout = 1u << 0,   // mbarrier wait for the TMA tile gave up
  kStatusQueueTimeout = 1u << 1, // persistent kernel: bounded wait gave up
  kStatusBadItem = 1u << 2,      // persistent kernel: work item out of range
};

constexpr int kMaxK = 17;              // largest specialised odd filter side
constexpr int kGenericMaxTaps = 1024;  // generic kernel: fh * fw limit
constexpr int kStageDirect = 0, kStageSmem = 1, kStageTma = 2;
// CTAs of at least this many threads take the ring form with its left-over
// filter rows first (RingSchedule::kRemFirst), smaller ones with them last
constexpr int kRingRemFirstThreads = 256;
constexpr unsigned kMbarSpinLimit = 1u << 22;

struct ConvLaunch {
  const float* in;
  float* out;
  unsigned* status;
  long long in_pitch, out_pitch;
  int in_h, in_w, out_h, out_w;
  int fh, fw;
  const float* taps;       // host copy, fh * fw floats
  int bx, by, tx, ty;
  int staging, filt_smem, vw;
  int smem_pitch, tile_w, tile_h;
  // staged tile as boxes side by side in shared memory: threads [q*group_x,
  // (q+1)*group_x) in x read box q, group_stride floats after box q-1 (one
  // box of the whole tile: group_x = bx, group_stride = 0)
  int group_x, group_stride, groups;
  size_t smem_bytes;
  const CUtensorMap* tmap; // valid when staging == TMA
};

// Kernel function of one specialised variant (nullptr if not compiled).
using KernelPicker = const void* (*)(int tx, int ty, bool staged, bool filt_smem);
// Fill the variant's arguments and launch it.
using KernelLauncher = cudaError_t (*)(const ConvLaunch& L, cudaStream_t s);

#define CT_DECLARE_K(K)                                                   \
  const void* pick_k##K(int tx, int ty, bool staged, bool filt_smem, bool big_cta); \
  cudaError_t launch_k##K(const ConvLaunch& L, cudaStream_t s);

CT_DECLARE_K(1)
CT_DECLARE_K(3)
CT_DECLARE_K(5)
CT_DECLARE_K(7)
CT_DECLARE_K(9)
CT_DECLARE_K(11)
CT_DECLARE_K(13)
CT_DECLARE_K(15)
CT_DECLARE_K(17)
#undef CT_DECLARE_K

const void* pick_generic();
cudaError_t launch_generic(const ConvLaunch& L, cudaStream_t s);

}  // namespace convtune
