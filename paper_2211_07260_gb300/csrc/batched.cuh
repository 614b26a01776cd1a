// Persistent batched correlation: many images of uneven sizes and odd
// filter sides in one launch.  CTAs (256 threads, persistent: occupancy x
// SM count) take work items -- one output tile of one image -- from a global
// atomic counter, two ahead: while one item is computed, the next item's
// taps and halo tile are being copied into the second staging area.  The
// image table is sorted by filter side so that CTAs run the same unrolled
// body at the same time.  Each tile runs the same tap order as the plain
// kernel, so batched outputs are bitwise identical to plain launches.
#pragma once

#include "conv2d_kernels.cuh"

namespace convtune {

constexpr int kBatchThreads = 256;
constexpr int kBatchTileX = 4;

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
};

struct BatchArgs {
  const BatchImage* images;
  int n_images;
  long long n_items;
  unsigned* counter;     // work counter, zero at launch
  unsigned* status;      // device status word
  int stage_stride;      // floats per staging area (two areas: double buffering)
};

// Fields issue_tile_cp_async() reads.
struct BatchStage {
  const float* in;
  long long in_pitch;
  int in_h, in_w, vw, tile_w, tile_h, smem_pitch;
};

// Floats of the tap area at the start of a staging area for filter side K.
template <int K>
__host__ __device__ constexpr int batch_tap_floats() {
  return (K * ((K + 3) / 4 * 4) + 31) / 32 * 32;
}

// Start the asynchronous copies of one work item (taps, halo tile) into a
// staging area; completion is awaited by the caller (cp.async groups).
template <int K, int TY>
__device__ __forceinline__ void batch_stage(const BatchImage& im, int t, float* area) {
  constexpr int TX = kBatchTileX;
  constexpr int KP = (K + 3) / 4 * 4;
  const int bx = im.bx, by = kBatchThreads / bx;
  const int ti = t % im.tiles_x, tj = t / im.tiles_x;
  // taps: K rows of KP floats, 16-byte chunks
  for (int q = threadIdx.x; q < K * KP / 4; q += kBatchThreads)
    cp_async_bytes(area + 4 * q, im.filt + 4 * q, 16, 16);
  BatchStage st;
  st.in = im.in;
  st.in_pitch = im.in_pitch;
  st.in_h = im.in_h;
  st.in_w = im.in_w;
  st.vw = im.vw;
  st.tile_w = (bx * TX + K - 1 + 3) / 4 * 4;
  st.tile_h = by * TY + K - 1;
  st.smem_pitch = st.tile_w;
  issue_tile_cp_async(st, area + batch_tap_floats<K>(), ti * bx * TX, tj * by * TY);
}

// Compute and store one work item from its landed staging area.
template <int K, int TY>
__device__ __forceinline__ void batch_compute(const BatchImage& im, int t, const float* area) {
  constexpr int TX = kBatchTileX;
  constexpr int KP = (K + 3) / 4 * 4;
  const int bx = im.bx, by = kBatchThreads / bx;
  const int lx = threadIdx.x % bx, ly = threadIdx.x / bx;
  const int ti = t % im.tiles_x, tj = t / im.tiles_x;
  const int pitch = (bx * TX + K - 1 + 3) / 4 * 4;
  const float* sfilt = area;
  const float* sbase = area + batch_tap_floats<K>() + (ly * TY) * pitch + lx * TX;
  float acc[TY][TX];
  accumulate_tile<K, TX, TY>(
      acc, [&](int r, float(&rowv)[TX + K - 1]) { fetch_row_smem<K, TX>(rowv, sbase + r * pitch); },
      [&](int j, int i) -> float { return sfilt[j * KP + i]; });
  const int x0 = ti * bx * TX + lx * TX, y0 = tj * by * TY + ly * TY;
#pragma unroll
  for (int r = 0; r < TY; ++r) {
    const int y = y0 + r;
    if (y < im.out_h) store_run<TX>(im.out + (long long)y * im.out_pitch, x0, im.out_w, im.vw, acc[r]);
  }
}

}  // namespace convtune
