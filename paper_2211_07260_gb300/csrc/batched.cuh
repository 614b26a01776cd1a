// Persistent batched correlation: many images of uneven sizes and odd
// filter sides in one launch.  CTAs (256 threads, persistent: occupancy x
// SM count) take work items -- one output tile of one image (two vertically
// adjacent ones for the 13..17 class) -- from a global atomic counter; the
// image table is sorted by filter side so that CTAs run the same unrolled
// body at the same time.  Each tile runs the same tap order as the plain
// kernel, so batched outputs are bitwise identical to plain launches.
//
// Staging is double-buffered: while the CTA computes item i from one shared-
// memory buffer, the TMA unit fills the other with item i+1's input block,
// started by one thread (no registers or issue slots of the computing warps
// are spent on the copy).  The block is staged as one 2-D TMA box per group
// of 32 threads in x (box width 32 x 4 + K - 1 floats, so every box stays
// within the 256-element limit however wide the CTA is); each thread's input
// rows lie inside its group's box.  Images whose input is not 16-byte aligned
// stage the same layout with cp.async instead.
#pragma once

#include "conv2d_kernels.cuh"

namespace convtune {

// CTA size of a class launch: 64, 128 or 256 threads (per class, from the
// caller's tiles; 256 by default); the kernels are compiled for up to 256.
constexpr int kBatchThreads = 256;
// Work items one claim (one increment of a launch's counter) hands a CTA:
// consecutive tiles, so one image lookup and table-entry copy serve several
// items and the counter sees fewer atomics; larger chunks leave a longer
// tail at the end of the launch.  Per class, from the caller's tiles (1..8);
// by default 2 for sides 1-7 and 1 for the others (GB300, 256-image batch,
// each class alone: sides 1-7 177 -> 165 us with 2, 9-11 and 13-17 fastest
// with 1).
__host__ __device__ constexpr int batch_default_claim(int cls) { return cls == 0 ? 2 : 1; }
// Staging buffers of a class kernel (copies run stages - 1 items ahead).
// Two for every class: three for sides 1-7 (short items against their
// copies) measured 148 -> 175 us on GB300, the third buffer of their 8-row
// 3 x 3 tiles costing a resident CTA.
constexpr int kBatchMaxStages = 3;
__host__ __device__ constexpr int batch_class_stages(int /*cls*/) { return 2; }
__host__ __device__ constexpr bool batch_valid_threads(int t) { return t == 64 || t == 128 || t == 256; }
constexpr int kBatchTileX = 4;
// Filter sides up to this one may also take 8-row tiles (their bodies are
// small and latency-bound; 8-row tiles for 5 x 5 and 7 x 7 measured no
// faster, and their registers would cost the class kernel a resident CTA).
constexpr int kBatchMaxK8 = 3;
// Threads in x that share one staged box (one warp's width).
constexpr int kBatchGroupX = 32;
// FFMAs above which a batched body takes the ring form (the single-image
// kernel's threshold is 2500; GB300, 256-image batch: sides 9-11 273 -> 238
// us with 1200, which rings their 4-row tiles; 700 also rings sides 5-7 and
// slowed them 148 -> 159 us)
constexpr int kBatchRingFfma = 1200;

// Geometry of one work item's staged input block.
struct BatchStageGeom {
  int box_w;         // floats per box row (multiple of 4)
  int tile_h;        // rows per box
  int groups;        // boxes side by side: max(1, bx / 32)
  int group_stride;  // floats from one box to the next (multiple of 32: 128 B)
  int buf_floats;    // floats of one staging buffer (multiple of 32)
};

// One image of the batch (device table entry).  128-byte aligned (the tensor
// map's own alignment): the TMA unit reads the map straight from the table
// in global memory.
struct alignas(128) BatchImage {
  CUtensorMap tmap;      // padded input, box (box_w, tile_h); valid when use_tma
  const float* in;       // padded input (device)
  float* out;            // output (device)
  const float* filt;     // taps, k rows of KP = round_up(k, 4) floats (device)
  long long in_pitch, out_pitch;
  long long first_item;  // index of this image's first work item
  int in_h, in_w, out_h, out_w;
  int k, bx, ty, vw;     // filter side; block_x (block_y = threads / block_x); tile_y; load width
  int threads;           // CTA size of the image's class launch
  int claim;             // work items per claim of the image's class launch
  int tiles_x, tiles_y;
  int tap_off;           // >= 0: the taps (K rows of KP floats) start at w[tap_off] of the
                         // launch's parameter block; -1: read from `filt`
  int use_tma;           // 1: TMA staging; 0: cp.async (input not 16-byte aligned)
  BatchStageGeom g;
};
static_assert(sizeof(BatchImage) == 256, "table entries: 256 B (tensor maps aligned, one "
              "8-byte word per lane when a warp copies an entry)");

// Vertically adjacent tiles per work item: the 13..17 class stages one block
// for two tiles (half the stage cycles per output, and the K-1 halo rows
// shared between the two) and computes them one after the other.
constexpr int kBatchClasses = 3;
__host__ __device__ constexpr int batch_class_of(int k) { return k <= 7 ? 0 : (k <= 11 ? 1 : 2); }
__host__ __device__ constexpr int batch_subtiles(int k) { return batch_class_of(k) == 2 ? 2 : 1; }

// Output rows one work item covers.
__host__ __device__ constexpr int batch_item_rows(int k, int bx, int ty, int threads) {
  return batch_subtiles(k) * (threads / bx) * ty;
}

__host__ __device__ inline BatchStageGeom batch_stage_geom(int k, int bx, int ty, int threads) {
  BatchStageGeom g;
  const int gx = bx < kBatchGroupX ? bx : kBatchGroupX;
  g.box_w = (gx * kBatchTileX + k - 1 + 3) / 4 * 4;
  g.tile_h = batch_item_rows(k, bx, ty, threads) + k - 1;
  g.groups = bx / gx;
  g.group_stride = (g.box_w * g.tile_h + 31) / 32 * 32;
  g.buf_floats = g.groups * g.group_stride;
  return g;
}

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
  int buf_floats;            // floats of each staging buffer
  unsigned claim_items;      // consecutive work items each counter increment hands out
  alignas(16) float w[kBatchParamTaps];  // taps of the images with tap_off >= 0
};
static_assert(sizeof(BatchArgs) <= 32764, "kernel parameter block too large");

// Work counters (one per launch of a batch) live in a 1 KB region.
constexpr int kBatchCounterBytes = 1024;
constexpr int kBatchMaxLaunches = kBatchCounterBytes / 4 - 1;  // one word left for a status

// Dynamic shared memory of a class kernel: [taps (shared-memory fallback),
// K x KP padded to 32 floats] [staging buffer 0] [staging buffer 1].
__host__ __device__ constexpr int batch_filt_floats(int k) {
  return (k * ((k + 3) / 4 * 4) + 31) / 32 * 32;
}

// Tile origin (input == output coordinates) of tile t of an image.
__device__ __forceinline__ void batch_tile_origin(const BatchImage& im, int t, int* gx0,
                                                  int* gy0) {
  const int ti = t % im.tiles_x, tj = t / im.tiles_x;
  *gx0 = ti * im.bx * kBatchTileX;
  *gy0 = tj * batch_item_rows(im.k, im.bx, im.ty, im.threads);
}

// One thread: arm the buffer's mbarrier for the block's bytes and start one
// TMA box per 32-thread group (x offsets 128 floats apart: 16-byte aligned).
// `im` is any copy of the image's entry; the tensor map is read by the TMA
// unit from the table itself (`gim`, global memory).
__device__ __forceinline__ void batch_issue_tma(const BatchImage* im, const BatchImage* gim, int t,
                                                float* buf, uint64_t* mbar) {
  int gx0, gy0;
  batch_tile_origin(*im, t, &gx0, &gy0);
  const BatchStageGeom g = im->g;
  const unsigned bar = smem_u32(mbar);
  const unsigned bytes = static_cast<unsigned>(g.groups * g.box_w * g.tile_h * 4);
  // the buffer's previous contents were read through the generic proxy
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
  for (int q = 0; q < g.groups; ++q) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(buf + q * g.group_stride)),
        "l"(reinterpret_cast<uint64_t>(&gim->tmap)), "r"(gx0 + q * kBatchGroupX * kBatchTileX),
        "r"(gy0), "r"(bar)
        : "memory");
  }
}

// All threads: the same block with cp.async (zero-filled outside the input).
__device__ __forceinline__ void batch_stage_cp_async(const BatchImage& im, int t, float* buf) {
  int gx0, gy0;
  batch_tile_origin(im, t, &gx0, &gy0);
  const BatchStageGeom g = im.g;
  const int vw = im.vw;
  const int chunks_per_row = g.box_w / vw;
  const int per_group = chunks_per_row * g.tile_h;
  for (int c = threadIdx.x; c < per_group * g.groups; c += blockDim.x) {
    const int q = c / per_group;
    const int rem = c - q * per_group;
    const int r = rem / chunks_per_row;
    const int col = (rem - r * chunks_per_row) * vw;
    const int gy = gy0 + r, gx = gx0 + q * kBatchGroupX * kBatchTileX + col;
    int avail = 0;
    if (gy < im.in_h && gx < im.in_w) avail = min(vw, im.in_w - gx);
    const float* src = avail > 0 ? im.in + (long long)gy * im.in_pitch + gx : im.in;
    cp_async_bytes(buf + q * g.group_stride + r * g.box_w + col, src, vw * 4, avail * 4);
  }
  cp_async_wait_all();
}

// Bodies the batched kernels run in the ring form: the class kernels hold
// the bodies of several filter sides and tile heights at once, so their code
// competes for the instruction caches sooner than the single-image kernel's.
__host__ __device__ constexpr bool batch_uses_ring(int k, int tx, int ty) {
  return k * k * tx * ty > kBatchRingFfma;
}

// Compute (and store) the item's SUB tiles from its staged block.
template <int K, int TY>
__device__ __forceinline__ void batch_tile(const BatchArgs& a, const BatchImage& im, int t,
                                           const float* buf, const float* sfilt) {
  constexpr int TX = kBatchTileX;
  constexpr int KP = (K + 3) / 4 * 4;
  constexpr int SUB = batch_subtiles(K);
  const int bx = im.bx, by = im.threads / bx;
  const int tid = threadIdx.x;
  const int lx = tid % bx, ly = tid / bx;
  const int grp = lx / kBatchGroupX, lg = lx % kBatchGroupX;
  const BatchStageGeom g = im.g;
  int gx0, gy0;
  batch_tile_origin(im, t, &gx0, &gy0);
  const bool param_taps = im.tap_off >= 0;  // CTA-uniform

  // the item's SUB tiles, one after the other, from the one staged block
#pragma unroll 1
  for (int sub = 0; sub < SUB; ++sub) {
    // threads whose outputs all lie below or right of the image (the ragged
    // last tiles) skip the taps: nothing of theirs is stored, and nothing
    // in the accumulation waits on other threads
    const int x0 = gx0 + lx * TX, y0 = gy0 + sub * by * TY + ly * TY;
    if (y0 >= im.out_h || x0 >= im.out_w) continue;
    float acc[TY][TX];
    const float* sbase = buf + grp * g.group_stride + (sub * by * TY + ly * TY) * g.box_w + lg * TX;
    const int pitch = g.box_w;
    // large bodies take the ring form, as in the single-image kernel (this
    // kernel holds one body per filter side and tile height, so its code size
    // matters even more); the loop keeps its bounds tests here (the peeled
    // form measured slower with parameter taps, and needs 128 registers and a
    // stack frame with shared-memory taps)
    if constexpr (batch_uses_ring(K, TX, TY)) {
      if (param_taps) {
        // taps from the parameter block (constant bank), as in the single-image
        // kernel's ring
        const float4* wrow = reinterpret_cast<const float4*>(a.w + im.tap_off);
        accumulate_tile_ring<K, TX, TY, RingSchedule::kTested>(
            acc, [&](int r) { return sbase + r * pitch; },
            [&](int j, float(&w)[KP]) {
#pragma unroll
              for (int i = 0; i < KP; i += 4) {
                const float4 q = wrow[(j * KP + i) / 4];
                w[i] = q.x;
                w[i + 1] = q.y;
                w[i + 2] = q.z;
                w[i + 3] = q.w;
              }
            });
      } else {
        accumulate_tile_ring<K, TX, TY, RingSchedule::kTested>(
            acc, [&](int r) { return sbase + r * pitch; },
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
          acc, [&](int r, float(&rowv)[TX + K - 1]) { fetch_row_smem<K, TX>(rowv, sbase + r * pitch); },
          [&](int j, int i) -> float { return wp[j * KP + i]; });
    } else {
      accumulate_tile<K, TX, TY>(
          acc, [&](int r, float(&rowv)[TX + K - 1]) { fetch_row_smem<K, TX>(rowv, sbase + r * pitch); },
          [&](int j, int i) -> float { return sfilt[j * KP + i]; });
    }
#pragma unroll
    for (int r = 0; r < TY; ++r) {
      const int y = y0 + r;
      if (y < im.out_h) store_run<TX>(im.out + (long long)y * im.out_pitch, x0, im.out_w, im.vw, acc[r]);
    }
  }
}

}  // namespace convtune
