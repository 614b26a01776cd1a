// Tunable FP32 2-D cross-correlation kernels for sm_103a.
//
//   out[y][x] = sum_{j<fh} sum_{i<fw} in[y+j][x+i] * filt[j][i]
//
// (the workload's "zero-padded input" convolution, computed as a correlation:
// no filter flip).  Every variant accumulates each output in one FP32 register
// with an fmaf chain over the taps in the same order -- j ascending, then i
// ascending -- so all tuning configurations give bitwise-identical results.
//
// Tunable parameters (the tuner's search space):
//   block_x, block_y  threads per CTA in x / y (runtime: blockDim)
//   TX, TY            outputs per thread in x / y (compile time: register tile)
//   staging           DIRECT: each thread reads its rows straight from global
//                     memory (vector loads through L1), the horizontal halo of
//                     a row comes from neighbouring lanes by warp shuffles;
//                     SMEM: the CTA's halo tile is copied to shared memory
//                     (one bulk copy per row with 16-byte loads, else
//                     cp.async chunks); TMA: the same tile arrives by 2-D
//                     cp.async.bulk.tensor copies completing on an mbarrier.
//                     One output tile per CTA in every mode.
//   filter memory     CONST: taps are read from the kernel's parameter space
//                     (constant bank, an immediate FFMA operand once the tap
//                     loops are unrolled); SHARED: taps are copied to shared
//                     memory first and read with LDS
//   vec_width         width (floats) of global loads and stores
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "conv2d_launch.h"


namespace convtune {

// Launch arguments.  The filter travels by value in the parameter space, i.e.
// in the constant bank.
template <int NTAPS>
struct alignas(128) ConvArgs {  // (the tensor map needs 128-byte alignment)
  CUtensorMap tmap;          // TMA descriptor of the padded input (TMA staging)
  const float* in;           // padded input, in_h rows of in_pitch floats
  float* out;                // output, out_h rows of out_pitch floats
  unsigned* status;          // device status word (error bits), may be null
  long long in_pitch, out_pitch;
  int in_h, in_w, out_h, out_w;
  int fh, fw;                // used by the generic kernel only
  int vw;                    // global load width 1, 2 or 4
  int staging;               // kStageDirect / kStageSmem / kStageTma
  int smem_pitch;            // floats per shared-memory tile row
  int tile_w, tile_h;        // staged box (floats); tile_w % 4 == 0
  int group_x, group_stride, groups;  // boxes of the staged tile (see ConvLaunch)
  // taps: the specialised kernels keep K rows of KP = round_up(K, 4) floats
  // (zero padded; a tap row is whole 16-byte words), the generic kernel
  // fh rows of fw floats
  alignas(16) float w[NTAPS];
};

// Floats per tap row of the specialised K x K kernels.
__host__ __device__ constexpr int tap_row_pad(int k) { return (k + 3) / 4 * 4; }

// Bodies of more than ~2500 FFMAs (K*K*TX*TY) no longer fit the instruction
// caches unrolled; they take the ring form (accumulate_tile_ring).
__host__ __device__ constexpr bool uses_ring(int k, int tx, int ty) { return tx * ty * k * k > 2500; }

// Order of the ring form's filter rows around its loop over whole blocks of
// TY rows.  All three give the same fmaf chain per output (bitwise the same
// result); they differ in scheduling only.  Measured on GB300 (17 x 17,
// 4 x 4 tiles, TMA staging, constant-bank taps): CTAs of 1-4 warps ran 2-5 %
// faster with the K % TY left-over rows after the loop, CTAs of 8 warps 2 %
// faster with them before it; taps from shared memory keep the bounds-tested
// loop, which takes fewer registers there.
enum class RingSchedule { kTested, kRemLast, kRemFirst };

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// ----------------------------------------------------------------------------
// Global loads of n (= 1, 2, 4) consecutive floats starting at column c of a
// row.  Columns >= in_w read as zero (they feed only outputs that are never
// stored); rows outside [0, in_h) read as zero.
// ----------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void load_run(float (&v)[N], const float* row, int c, int in_w,
                                         bool row_ok, int vw) {
#pragma unroll
  for (int q = 0; q < N; ++q) v[q] = 0.0f;
  if (!row_ok) return;
  if (c + N <= in_w) {
    if constexpr (N == 4) {
      if (vw >= 4) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(row + c));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        return;
      }
    }
    if constexpr (N % 2 == 0) {
      if (vw >= 2) {
#pragma unroll
        for (int q = 0; q < N; q += 2) {
          const float2 t = __ldg(reinterpret_cast<const float2*>(row + c + q));
          v[q] = t.x; v[q + 1] = t.y;
        }
        return;
      }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = __ldg(row + c + q);
    return;
  }
#pragma unroll
  for (int q = 0; q < N; ++q)
    if (c + q < in_w) v[q] = __ldg(row + c + q);
}

// ----------------------------------------------------------------------------
// Halo tile staging: rows [gy0, gy0 + tile_h) x columns [gx0, gx0 + tile_w)
// of the padded input into shared memory (pitch sp floats).  Outside the input
// the tile holds zeros.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_bytes(float* dst, const float* src, int cp_bytes,
                                               int src_bytes) {
  const unsigned d = smem_u32(dst);
  if (cp_bytes == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(src_bytes));
  } else if (cp_bytes == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
                 "r"(src_bytes));
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(src_bytes));
  }
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <class Args>
__device__ __forceinline__ void issue_tile_cp_async(const Args& a, float* tile, int gx0, int gy0) {
  const int vw = a.vw;
  const int chunks_per_row = a.tile_w / vw;
  const int total = chunks_per_row * a.tile_h;
  const int nthr = blockDim.x * blockDim.y;
  for (int c = threadIdx.y * blockDim.x + threadIdx.x; c < total; c += nthr) {
    const int r = c / chunks_per_row;
    const int col = (c - r * chunks_per_row) * vw;
    const int gy = gy0 + r, gx = gx0 + col;
    int avail = 0;
    if (gy < a.in_h && gx < a.in_w) avail = min(vw, a.in_w - gx);
    const float* src = avail > 0 ? a.in + (long long)gy * a.in_pitch + gx : a.in;
    cp_async_bytes(tile + r * a.smem_pitch + col, src, vw * 4, avail * 4);
  }
}

template <class Args>
__device__ __forceinline__ void stage_tile_cp_async(const Args& a, float* tile, int gx0, int gy0) {
  issue_tile_cp_async(a, tile, gx0, gy0);
  cp_async_wait_all();
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Leader thread: arm the mbarrier for the tile's bytes and start one 2-D TMA
// copy per box of the tile.  A box is at most 256 x 256 floats, so a tile
// wider than that is staged as several boxes side by side, one per group of
// group_x threads in x, each with its own K-1 halo columns (x offsets
// group_x * TX floats apart: multiples of 4, 16-byte aligned).
template <class Args>
__device__ __forceinline__ void issue_tile_tma(const Args& a, float* tile, uint64_t* mbar, int gx0,
                                               int gy0, int tx) {
  const unsigned bar = smem_u32(mbar);
  const unsigned bytes = static_cast<unsigned>(a.groups * a.tile_w * a.tile_h * 4);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
  for (int q = 0; q < a.groups; ++q) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(tile + q * a.group_stride)),
        "l"(reinterpret_cast<uint64_t>(&a.tmap)), "r"(gx0 + q * a.group_x * tx), "r"(gy0),
        "r"(bar)
        : "memory");
  }
}

// Programmatic dependent launch.  A launch made with programmatic stream
// serialization may start while the previous kernel on its stream still
// runs: pdl_launch_dependents() lets the next launch begin once every CTA
// of this grid has called it (or exited); pdl_wait() blocks until the
// previous grid has completed and its memory is visible.  Both are no-ops
// for a launch made without the attribute.  The correlation kernels wait
// right before their first global-memory access and trigger right after
// it: the next launch and its prologue (shared-memory taps, barrier set-up)
// overlap this grid's run, correct whatever the two kernels share, and at
// most one grid waits ahead (a trigger before the wait let every queued
// launch of a CUDA graph start at once: their waiting CTAs crowded the SMs,
// 1024^2 / 7 x 7 graph replay 4.9 -> 13 us per launch).
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Bounded wait for completion of the mbarrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, unsigned parity) {
  const unsigned bar = smem_u32(mbar);
  for (unsigned it = 0; it < kMbarSpinLimit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Shared-memory staging with 16-byte loads (vec_width 4, so the input and its
// row stride are 16-byte aligned): one bulk copy (cp.async.bulk) per tile
// row, issued by the first warp and completing on an mbarrier, instead of a
// 16-byte cp.async per thread and chunk -- a few dozen requests per CTA
// instead of thousands (1024^2 / 7 x 7: the per-chunk form cost ~1.5 us of
// every launch).  Rows below the input and the columns past the end of a
// row's allocation (pitch) are zero-filled in shared memory; a row copy
// never reads past its row's pitch.  All threads call this; returns false
// if the bounded wait for the copies gave up.
template <class Args>
__device__ __forceinline__ bool stage_tile_bulk_rows(const Args& a, float* tile, uint64_t* mbar,
                                                     int gx0, int gy0) {
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int rows_in = max(0, min(a.tile_h, a.in_h - gy0));
  const long long avail = a.in_pitch - gx0;  // floats to the end of the row's pitch (> 0)
  const int cols = (int)(avail < a.tile_w ? avail : a.tile_w);  // a multiple of 4
  // zero-fill what no copy writes: whole rows below the input, and the
  // columns past `cols` of the copied rows
  const int tail = a.tile_w - cols;
  for (int q = tid; q < rows_in * tail; q += nthr)
    tile[(q / tail) * a.smem_pitch + cols + q % tail] = 0.0f;
  for (int q = tid; q < (a.tile_h - rows_in) * a.tile_w; q += nthr)
    tile[(rows_in + q / a.tile_w) * a.smem_pitch + q % a.tile_w] = 0.0f;
  if (rows_in > 0) {
    const int lanes = nthr < 32 ? nthr : 32;  // the first warp (CTAs of 16 threads: half of one)
    if (tid < lanes) {
      const unsigned bar = smem_u32(mbar);
      const unsigned row_bytes = static_cast<unsigned>(cols * 4);
      if (tid == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                     "r"(row_bytes * static_cast<unsigned>(rows_in))
                     : "memory");
      __syncwarp(lanes == 32 ? 0xffffffffu : (1u << lanes) - 1u);
      for (int r = tid; r < rows_in; r += lanes) {
        const float* src = a.in + (long long)(gy0 + r) * a.in_pitch + gx0;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1], %2, [%3];\n" ::"r"(smem_u32(tile + r * a.smem_pitch)),
            "l"(src), "r"(row_bytes), "r"(bar)
            : "memory");
      }
    }
    if (!mbar_wait(mbar, 0u)) return false;
  }
  return true;
}

// ----------------------------------------------------------------------------
// Row fetch for the direct (register) path: the thread's TX + K - 1 input
// values of one row.  Each lane loads its own TX values; the halo to its right
// comes from the next lanes of its x-segment by shuffles (the last lanes take
// it from the first lanes' second load, one segment further right).
// ----------------------------------------------------------------------------
template <int K, int TX>
__device__ __forceinline__ void fetch_row_direct(float (&rowv)[TX + K - 1], const float* row,
                                                 bool row_ok, int x0, int xs_next, int lane,
                                                 int seg, unsigned mask, int in_w, int vw) {
  float A[TX];
  load_run<TX>(A, row, x0, in_w, row_ok, vw);
  constexpr int NB = (TX + K - 2) / TX;  // lanes whose second load is used
  float B[TX];
#pragma unroll
  for (int q = 0; q < TX; ++q) B[q] = 0.0f;
  if (K > 1 && lane < NB) load_run<TX>(B, row, xs_next + lane * TX, in_w, row_ok, vw);
#pragma unroll
  for (int q = 0; q < TX; ++q) rowv[q] = A[q];
#pragma unroll
  for (int m = TX; m < TX + K - 1; ++m) {
    const int d = m / TX, q = m % TX;
    const float send = lane < d ? B[q] : A[q];
    rowv[m] = __shfl_sync(mask, send, (lane + d) & (seg - 1), seg);
  }
}

// Row fetch from the staged shared-memory tile with the widest aligned LDS.
template <int K, int TX>
__device__ __forceinline__ void fetch_row_smem(float (&rowv)[TX + K - 1], const float* srow) {
  constexpr int N = TX + K - 1;
  if constexpr (TX % 4 == 0) {
#pragma unroll
    for (int m = 0; m < N; m += 4) {
      const float4 t = *reinterpret_cast<const float4*>(srow + m);
      rowv[m] = t.x;
      if (m + 1 < N) rowv[m + 1] = t.y;
      if (m + 2 < N) rowv[m + 2] = t.z;
      if (m + 3 < N) rowv[m + 3] = t.w;
    }
  } else if constexpr (TX % 2 == 0) {
#pragma unroll
    for (int m = 0; m < N; m += 2) {
      const float2 t = *reinterpret_cast<const float2*>(srow + m);
      rowv[m] = t.x;
      if (m + 1 < N) rowv[m + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) rowv[m] = srow[m];
  }
}

// Store one thread row of TX outputs (vector width min(vw, TX) when the run
// is fully inside the output, else element by element).
template <int TX>
__device__ __forceinline__ void store_run(float* orow, int x0, int out_w, int vw,
                                          const float (&v)[TX]) {
  if (x0 + TX <= out_w) {
    if constexpr (TX == 4) {
      if (vw >= 4) {
        *reinterpret_cast<float4*>(orow + x0) = make_float4(v[0], v[1], v[2], v[3]);
        return;
      }
    }
    if constexpr (TX % 2 == 0) {
      if (vw >= 2) {
#pragma unroll
        for (int q = 0; q < TX; q += 2)
          *reinterpret_cast<float2*>(orow + x0 + q) = make_float2(v[q], v[q + 1]);
        return;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < TX; ++q)
    if (x0 + q < out_w) orow[x0 + q] = v[q];
}

// ----------------------------------------------------------------------------
// The tap accumulation of one thread: TY x TX outputs whose top-left output is
// (y0, x0).  Input rows r = 0 .. TY+K-2 (relative to y0) are fetched once
// each; row r feeds output row t with filter row j = r - t.  For a fixed
// output the taps therefore arrive in (j, i) lexicographic order.
// FROW(r, rowv) fills rowv with the row's TX+K-1 values; TAP(j, i) returns the
// tap.
// ----------------------------------------------------------------------------
template <int K, int TX, int TY, class FetchRow, class Tap>
__device__ __forceinline__ void accumulate_tile(float (&acc)[TY][TX], FetchRow&& frow, Tap&& tap) {
#pragma unroll
  for (int t = 0; t < TY; ++t)
#pragma unroll
    for (int x = 0; x < TX; ++x) acc[t][x] = 0.0f;
#pragma unroll
  for (int r = 0; r < TY + K - 1; ++r) {
    float rowv[TX + K - 1];
    frow(r, rowv);
#pragma unroll
    for (int t = 0; t < TY; ++t) {
      const int j = r - t;
      if (j >= 0 && j < K) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
          const float w = tap(j, i);
#pragma unroll
          for (int x = 0; x < TX; ++x) acc[t][x] = fmaf(rowv[x + i], w, acc[t][x]);
        }
      }
    }
  }
}

// ----------------------------------------------------------------------------
// The same tap accumulation with the filter-row loop outermost: the TY input
// rows that filter row j needs (rows j .. j+TY-1 relative to y0) live in a
// ring of registers; after row j's taps, the ring slot of the row that is no
// longer needed takes the next input row.  The j loop is a real loop over
// blocks of TY rows (ring positions are then compile-time), so the code is
// about K / TY times shorter than the fully unrolled form.  For a fixed output
// the taps still arrive in (j, i) lexicographic order: bitwise the same
// result.  ROWP(r) points at input row r (shared memory, 16-byte aligned);
// TAPROW(j, w) fills w[0 .. K-1] with filter row j.
// ----------------------------------------------------------------------------
template <int K, int TX, int TY, RingSchedule SCHED, class RowPtr, class TapRow>
__device__ __forceinline__ void accumulate_tile_ring(float (&acc)[TY][TX], RowPtr&& rowp,
                                                     TapRow&& taprow) {
  constexpr int N = TX + K - 1;
  constexpr int KP = (K + 3) / 4 * 4;
  float ring[TY][N];
#pragma unroll
  for (int t = 0; t < TY; ++t) {
#pragma unroll
    for (int x = 0; x < TX; ++x) acc[t][x] = 0.0f;
    fetch_row_smem<K, TX>(ring[t], rowp(t));
  }
  // one filter row j (jj = j % TY, a compile-time ring position): output
  // row t reads input row j + t, held in slot (t + jj) % TY
  auto row_taps = [&](int jj, const float(&w)[KP]) {
#pragma unroll
    for (int t = 0; t < TY; ++t)
#pragma unroll
      for (int i = 0; i < K; ++i)
#pragma unroll
        for (int x = 0; x < TX; ++x)
          acc[t][x] = fmaf(ring[(t + jj) % TY][x + i], w[i], acc[t][x]);
  };
  constexpr int NBF = K / TY, REM = K % TY;
  if constexpr (SCHED == RingSchedule::kRemLast) {
    // K / TY whole blocks of TY filter rows in a loop, the K % TY rows left
    // after it unrolled (no per-row bounds tests in the loop)
#pragma unroll 1
    for (int jb = 0; jb < NBF; ++jb) {
      // no loads move across blocks (prefetched taps would hold registers
      // throughout the loop)
      asm volatile("" ::: "memory");
#pragma unroll
      for (int jj = 0; jj < TY; ++jj) {
        const int j = jb * TY + jj;
        float w[KP];
        taprow(j, w);
        row_taps(jj, w);
        // slot jj held input row j (needed by output row 0 only); it now
        // takes row j + TY, needed from filter row j + 1 on
        if (jj + 1 < TY || REM > 0 || jb + 1 < NBF) fetch_row_smem<K, TX>(ring[jj], rowp(TY + j));
      }
    }
#pragma unroll
    for (int jj = 0; jj < REM; ++jj) {
      const int j = NBF * TY + jj;
      float w[KP];
      taprow(j, w);
      row_taps(jj, w);
      if (jj + 1 < REM) fetch_row_smem<K, TX>(ring[jj], rowp(TY + j));
    }
  } else if constexpr (SCHED == RingSchedule::kRemFirst) {
    // the K % TY first filter rows unrolled, then K / TY whole blocks in a
    // loop; filter row j = REM + jb * TY + jj sits at ring position
    // (REM + jj) % TY
#pragma unroll
    for (int j = 0; j < REM; ++j) {
      float w[KP];
      taprow(j, w);
      row_taps(j, w);
      fetch_row_smem<K, TX>(ring[j], rowp(TY + j));
    }
#pragma unroll 1
    for (int jb = 0; jb < NBF; ++jb) {
      asm volatile("" ::: "memory");
#pragma unroll
      for (int jj = 0; jj < TY; ++jj) {
        const int j = REM + jb * TY + jj;
        float w[KP];
        taprow(j, w);
        row_taps((REM + jj) % TY, w);
        if (jj + 1 < TY || jb + 1 < NBF)
          fetch_row_smem<K, TX>(ring[(REM + jj) % TY], rowp(TY + j));
      }
    }
  } else {
    // ceil(K / TY) blocks, rows past K skipped (for taps read from shared
    // memory: the peeled forms above take more registers there)
    constexpr int NB = (K + TY - 1) / TY;
#pragma unroll 1
    for (int jb = 0; jb < NB; ++jb) {
#pragma unroll
      for (int jj = 0; jj < TY; ++jj) {
        const int j = jb * TY + jj;
        if (j < K) {
          float w[KP];
          taprow(j, w);
          row_taps(jj, w);
          if (j + 1 < K) fetch_row_smem<K, TX>(ring[jj], rowp(TY + j));
        }
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Specialised kernel: square odd filter K x K.
//   STAGED    = false: DIRECT staging; true: SMEM or TMA (args.staging)
//   FILT_SMEM = false: taps from the parameter (constant) space
// Dynamic shared memory: [filter K x KP (if FILT_SMEM), padded to 32 floats]
//                        [staged tile tile_h x smem_pitch (if STAGED)]
// ----------------------------------------------------------------------------
template <int K, int TX, int TY, bool STAGED, bool FILT_SMEM, bool REM_FIRST = false>
__device__ __forceinline__ void conv2d_body(const ConvArgs<K * tap_row_pad(K)>& a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // tap rows padded to a multiple of 4 floats (in the parameters and in
  // shared memory): 4 taps per 16-byte load
  constexpr int KP = tap_row_pad(K);
  constexpr int kFiltFloats = FILT_SMEM ? ((K * KP + 31) / 32) * 32 : 0;
  float* sfilt = reinterpret_cast<float*>(smem_raw);
  const int bx = blockDim.x, by = blockDim.y;

  if constexpr (FILT_SMEM) {
    for (int k = threadIdx.y * bx + threadIdx.x; k < K * KP; k += bx * by) sfilt[k] = a.w[k];
  }
  auto tap = [&](int j, int i) -> float {
    if constexpr (FILT_SMEM) return sfilt[j * KP + i];
    else return a.w[j * KP + i];
  };
  float acc[TY][TX];

  if constexpr (STAGED) {
    // One tile per CTA: the halo tile is copied to shared memory (cp.async,
    // or one 2-D TMA box completing on an mbarrier), then computed.
    __shared__ __align__(8) uint64_t full;  // TMA completion barrier
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    const int gx0 = blockIdx.x * bx * TX, gy0 = blockIdx.y * by * TY;
    float* const tile = sfilt + kFiltFloats;
    if (a.staging == kStageTma) {
      if (leader) {
        mbar_init(&full);
        mbar_init_fence();
      }
      __syncthreads();
      pdl_wait();
      pdl_launch_dependents();
      if (leader) issue_tile_tma(a, tile, &full, gx0, gy0, TX);
      const bool ok = mbar_wait(&full, 0u);
      // every thread takes the same decision, so no thread is left at a
      // barrier; the copy gets one more bounded wait to land before the
      // CTA leaves
      if (__syncthreads_or(!ok)) {
        if (leader) {
          if (a.status) atomicOr(a.status, kStatusTmaTimeout);
          mbar_wait(&full, 0u);
        }
        return;
      }
    } else if (a.vw == 4) {
      if (leader) {
        mbar_init(&full);
        mbar_init_fence();
      }
      __syncthreads();
      pdl_wait();
      pdl_launch_dependents();
      const bool ok = stage_tile_bulk_rows(a, tile, &full, gx0, gy0);
      if (__syncthreads_or(!ok)) {
        if (leader) {
          if (a.status) atomicOr(a.status, kStatusTmaTimeout);
          mbar_wait(&full, 0u);
        }
        return;
      }
    } else {
      pdl_wait();
      pdl_launch_dependents();
      issue_tile_cp_async(a, tile, gx0, gy0);
      cp_async_wait_all();
      __syncthreads();
    }
    const int x0 = gx0 + threadIdx.x * TX;
    const int y0 = gy0 + threadIdx.y * TY;
    const int grp = threadIdx.x / a.group_x;  // (group_x: a power of two)
    const float* sbase = tile + grp * a.group_stride + (threadIdx.y * TY) * a.smem_pitch +
                         (threadIdx.x - grp * a.group_x) * TX;
    // The fully unrolled form runs K*K*TX*TY FFMAs straight through; above
    // ~2500 of them (4 x 4 tiles, K >= 13) its code no longer fits the
    // instruction caches and warps stall on instruction fetch, so those
    // variants take the ring form (measured on GB300: 17 x 17, 4 x 4 tiles,
    // 54 -> 63 TFLOP/s; smaller bodies are faster unrolled).
    if constexpr (uses_ring(K, TX, TY)) {
      constexpr RingSchedule kSched = FILT_SMEM ? RingSchedule::kTested
                                      : REM_FIRST ? RingSchedule::kRemFirst
                                                  : RingSchedule::kRemLast;
      accumulate_tile_ring<K, TX, TY, kSched>(
          acc, [&](int r) { return sbase + r * a.smem_pitch; },
          [&](int j, float(&w)[KP]) {
            if constexpr (FILT_SMEM) {
#pragma unroll
              for (int i = 0; i < KP; i += 4) {
                const float4 q = *reinterpret_cast<const float4*>(sfilt + j * KP + i);
                w[i] = q.x;
                w[i + 1] = q.y;
                w[i + 2] = q.z;
                w[i + 3] = q.w;
              }
            } else {
#pragma unroll
              for (int i = 0; i < K; ++i) w[i] = a.w[j * KP + i];
            }
          });
    } else {
      accumulate_tile<K, TX, TY>(
          acc, [&](int r, float(&rowv)[TX + K - 1]) {
            fetch_row_smem<K, TX>(rowv, sbase + r * a.smem_pitch);
          },
          tap);
    }
#pragma unroll
    for (int r = 0; r < TY; ++r) {
      const int y = y0 + r;
      if (y < a.out_h) store_run<TX>(a.out + (long long)y * a.out_pitch, x0, a.out_w, a.vw, acc[r]);
    }
  } else {
    if constexpr (FILT_SMEM) __syncthreads();
    pdl_wait();
    pdl_launch_dependents();
    const int gx0 = blockIdx.x * bx * TX;  // tile origin (input == output coords)
    const int gy0 = blockIdx.y * by * TY;
    const int x0 = gx0 + threadIdx.x * TX;
    const int y0 = gy0 + threadIdx.y * TY;
    const int nthr = bx * by;
    const unsigned mask = nthr >= 32 ? 0xffffffffu : ((1u << nthr) - 1u);
    const int seg = bx < 32 ? bx : 32;  // lanes sharing one contiguous x run
    const int lane = threadIdx.x & (seg - 1);
    const int xs = gx0 + (threadIdx.x - lane) * TX;
    const int xs_next = xs + seg * TX;
    accumulate_tile<K, TX, TY>(
        acc, [&](int r, float(&rowv)[TX + K - 1]) {
          const int gy = y0 + r;
          const bool ok = gy < a.in_h;
          const float* row = a.in + (long long)(ok ? gy : 0) * a.in_pitch;
          fetch_row_direct<K, TX>(rowv, row, ok, x0, xs_next, lane, seg, mask, a.in_w, a.vw);
        },
        tap);
#pragma unroll
    for (int t = 0; t < TY; ++t) {
      const int y = y0 + t;
      if (y < a.out_h) store_run<TX>(a.out + (long long)y * a.out_pitch, x0, a.out_w, a.vw, acc[t]);
    }
  }
}

template <int K, int TX, int TY, bool STAGED, bool FILT_SMEM, bool REM_FIRST = false>
__global__ void conv2d_kernel(const __grid_constant__ ConvArgs<K * tap_row_pad(K)> a) {
  conv2d_body<K, TX, TY, STAGED, FILT_SMEM, REM_FIRST>(a);
}

// The same variant held to 96 registers.  Used for the 17 x 17 body with
// 4 x 4 tiles, staged, taps in the parameter space and the left-over filter
// rows last (CTAs of up to 4 warps): five CTAs of 128 threads then fit on an
// SM instead of four (108 registers uncapped, 28 bytes spilled capped; GB300,
// 4096^2: 150.8 -> 146.0 us per launch at 16 x 8 threads, 150.1 -> 145.6 us
// at 32 x 4, 32 x 1 unchanged).  Same instructions per output, so the same
// bits.
template <int K, int TX, int TY, bool STAGED, bool FILT_SMEM, bool REM_FIRST = false>
__global__ void __maxnreg__(96)
    conv2d_kernel_r96(const __grid_constant__ ConvArgs<K * tap_row_pad(K)> a) {
  conv2d_body<K, TX, TY, STAGED, FILT_SMEM, REM_FIRST>(a);
}

}  // namespace convtune
