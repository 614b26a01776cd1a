// Persistent batched correlation: many images of uneven sizes and odd
// filter sides in one launch.  CTAs (256 threads, persistent: occupancy x
// SM count) take work items -- one output tile of one image -- from a global
// atomic counter; the image table is sorted by filter side so that CTAs run
// the same unrolled body at the same time.  Each tile runs the same tap
// order as the plain kernel, so batched outputs are bitwise identical to
// plain launches.
#pragma once

#include "conv2d_kernels.cuh"

namespace convtune {

constexpr int kBatchThreads = 256;
constexpr int kBatchTileX = 4;
// Filter sides up to this one may also take 8-row tiles (their bodies are
// small and latency-bound; 8-row tiles for 5 x 5 and 7 x 7 measured no
// faster, and their registers would cost the class kernel a resident CTA).
constexpr int kBatchMaxK8 = 3;

// One image of the batch (device table entry).
struct alignas(16) BatchImage {
  const float* in;       // padded input (device)
  float* out;            // output (device)
  const float* filt;     // taps, k rows of KP = round_up(k, 4) floats (device)
  long long in_pitch, out_pitch;
  long long first_item;  // index of this image's first work item
  int in_h, in_w, out_h, out_w;
  int k, bx, ty, vw;     // filter side; block_x (block_y = 256 / block_x); tile_y; load width
  int tiles_x, tiles_y;
  int tap_off;           // >= 0: the taps (K rows of KP floats) start at w[tap_off] of the
                         // launch's parameter block; -1: read from `filt`
};

// Floats of taps a launch carries in its parameter block (kernel parameters
// live in a constant bank: up to 32,764 bytes per launch on this GPU).  Tiles
// read their image's taps from there, as the single-image kernel does from
// its own parameters, instead of from a shared-memory copy (GB300, 256-image
// batch: filter sides 5..15 5-9 % faster); a launch holds the images whose
// taps fit, and taps in shared memory remain for images beyond the launches
// a batch may have.
constexpr int kBatchParamTaps = 8000;

struct BatchArgs {
  const BatchImage* images;  // this launch's images (a contiguous run of the table)
  int n_images;
  long long n_items;         // work items of these images
  long long item_base;       // first_item of images[0]: item w is table item item_base + w
  unsigned* counter;         // work counter, zero at launch
  unsigned* status;          // device status word
  alignas(16) float w[kBatchParamTaps];  // taps of the images with tap_off >= 0
};
static_assert(sizeof(BatchArgs) <= 32764, "kernel parameter block too large");

// Work counters (one per launch of a batch) live in a 1 KB region.
constexpr int kBatchCounterBytes = 1024;
constexpr int kBatchMaxLaunches = kBatchCounterBytes / 4 - 1;  // one word left for a status

// Filter sides are split into classes, one persistent kernel each: a kernel's
// register allocation is that of its largest body, and the small-filter
// bodies (latency-bound) need far fewer registers than the 13..17 ones, so
// separate kernels keep more of their CTAs resident (GB300: 64, 80 and 124
// registers -> 4, 3 and 2 CTAs of 256 threads per SM).
constexpr int kBatchClasses = 3;
__host__ __device__ constexpr int batch_class_of(int k) { return k <= 7 ? 0 : (k <= 11 ? 1 : 2); }

// Vertically adjacent tiles per work item: the 13..17 class stages one block
// for two tiles (half the stage / barrier cycles per output, and the K-1
// halo rows shared between the two) and computes them one after the other.
__host__ __device__ constexpr int batch_subtiles(int k) { return batch_class_of(k) == 2 ? 2 : 1; }

// Output rows one work item covers.
__host__ __device__ constexpr int batch_item_rows(int k, int bx, int ty) {
  return batch_subtiles(k) * (kBatchThreads / bx) * ty;
}

// Fields stage_tile_cp_async() reads.
struct BatchStage {
  const float* in;
  long long in_pitch;
  int in_h, in_w, vw, tile_w, tile_h, smem_pitch;
};

template <int K, int TY>
__device__ __forceinline__ void batch_tile(const BatchArgs& a, const BatchImage& im, int t,
                                           float* smem) {
  constexpr int TX = kBatchTileX;
  constexpr int KP = (K + 3) / 4 * 4;
  constexpr int kFilt = (K * KP + 31) / 32 * 32;
  const int bx = im.bx, by = kBatchThreads / bx;
  const int tid = threadIdx.x;
  const int lx = tid % bx, ly = tid / bx;
  const int ti = t % im.tiles_x, tj = t / im.tiles_x;
  constexpr int SUB = batch_subtiles(K);
  const int gx0 = ti * bx * TX, gy0 = tj * SUB * by * TY;
  float* sfilt = smem;
  float* tile = smem + kFilt;
  BatchStage st;
  st.in = im.in;
  st.in_pitch = im.in_pitch;
  st.in_h = im.in_h;
  st.in_w = im.in_w;
  st.vw = im.vw;
  st.tile_w = (bx * TX + K - 1 + 3) / 4 * 4;
  st.tile_h = SUB * by * TY + K - 1;
  st.smem_pitch = st.tile_w;
  const bool param_taps = im.tap_off >= 0;  // CTA-uniform
  if (!param_taps)
    for (int q = tid; q < K * KP; q += kBatchThreads) sfilt[q] = im.filt[q];
  stage_tile_cp_async(st, tile, gx0, gy0);
  __syncthreads();

  // the item's SUB tiles, one after the other, from the one staged block
#pragma unroll 1
  for (int sub = 0; sub < SUB; ++sub) {
    float acc[TY][TX];
    const float* sbase = tile + (sub * by * TY + ly * TY) * st.smem_pitch + lx * TX;
    // large bodies take the ring form, as in the single-image kernel (this
    // kernel holds one body per filter side and tile height, so its code size
    // matters even more); the loop keeps its bounds tests here (the peeled
    // form measured slower with parameter taps, and needs 128 registers and a
    // stack frame with shared-memory taps)
    if constexpr (uses_ring(K, TX, TY)) {
      if (param_taps) {
        // taps from the parameter block (constant bank), as in the single-image
        // kernel's ring
        const float* wrow = a.w + im.tap_off;
        accumulate_tile_ring<K, TX, TY, RingSchedule::kTested>(
            acc, [&](int r) { return sbase + r * st.smem_pitch; },
            [&](int j, float(&w)[KP]) {
#pragma unroll
              for (int i = 0; i < K; ++i) w[i] = wrow[j * KP + i];
            });
      } else {
        accumulate_tile_ring<K, TX, TY, RingSchedule::kTested>(
            acc, [&](int r) { return sbase + r * st.smem_pitch; },
            [&](int j, float(&w)[KP]) {
#pragma unroll
              for (int i = 0; i < KP; i += 4) {
                const float4 q = *reinterpret_cast<const float4*>(sfilt + j * KP + i);
                w[i] = q.x;
                w[i + 1] = q.y;
                w[i + 2] = q.z;
                w[i + 3] = q.w;
              }
            });
      }
    } else if (param_taps) {
      const float* wp = a.w + im.tap_off;
      accumulate_tile<K, TX, TY>(
          acc,
          [&](int r, float(&rowv)[TX + K - 1]) { fetch_row_smem<K, TX>(rowv, sbase + r * st.smem_pitch); },
          [&](int j, int i) -> float { return wp[j * KP + i]; });
    } else {
      accumulate_tile<K, TX, TY>(
          acc,
          [&](int r, float(&rowv)[TX + K - 1]) { fetch_row_smem<K, TX>(rowv, sbase + r * st.smem_pitch); },
          [&](int j, int i) -> float { return sfilt[j * KP + i]; });
    }
    const int x0 = gx0 + lx * TX, y0 = gy0 + sub * by * TY + ly * TY;
#pragma unroll
    for (int r = 0; r < TY; ++r) {
      const int y = y0 + r;
      if (y < im.out_h) store_run<TX>(im.out + (long long)y * im.out_pitch, x0, im.out_w, im.vw, acc[r]);
    }
  }
  __syncthreads();  // the next item reuses the shared memory
}

}  // namespace convtune
