// Instantiation unit for one specialised filter side; compiled once per odd
// K in 1..17 with -DCT_K=K.  Holds the 36 kernel variants
// (tile_x, tile_y in {1,2,4} x staged / direct x filter shared / constant)
// and the launcher that fills their parameter block.
#include <string.h>

#include "conv2d_kernels.cuh"
#include "conv2d_launch.h"

#ifndef CT_K
#error "compile with -DCT_K=<odd filter side>"
#endif

#define CT_CAT2(a, b) a##b
#define CT_CAT(a, b) CT_CAT2(a, b)

namespace convtune {

namespace {
constexpr int K = CT_K;

template <int TX, int TY>
const void* pick_tile(bool staged, bool filt_smem, bool big_cta) {
  if (staged) {
    if (filt_smem) return (const void*)conv2d_kernel<K, TX, TY, true, true>;
    if constexpr (uses_ring(K, TX, TY))
      if (big_cta) return (const void*)conv2d_kernel<K, TX, TY, true, false, true>;
    if constexpr (K == 17 && TX == 4 && TY == 4)
      return (const void*)conv2d_kernel_r96<K, TX, TY, true, false>;
    return (const void*)conv2d_kernel<K, TX, TY, true, false>;
  }
  return filt_smem ? (const void*)conv2d_kernel<K, TX, TY, false, true>
                   : (const void*)conv2d_kernel<K, TX, TY, false, false>;
}

template <int TX>
const void* pick_ty(int ty, bool staged, bool filt_smem, bool big_cta) {
  switch (ty) {
    case 1: return pick_tile<TX, 1>(staged, filt_smem, big_cta);
    case 2: return pick_tile<TX, 2>(staged, filt_smem, big_cta);
    case 4: return pick_tile<TX, 4>(staged, filt_smem, big_cta);
    default: return nullptr;
  }
}
}  // namespace

const void* CT_CAT(pick_k, CT_K)(int tx, int ty, bool staged, bool filt_smem, bool big_cta) {
  switch (tx) {
    case 1: return pick_ty<1>(ty, staged, filt_smem, big_cta);
    case 2: return pick_ty<2>(ty, staged, filt_smem, big_cta);
    case 4: return pick_ty<4>(ty, staged, filt_smem, big_cta);
    default: return nullptr;
  }
}

cudaError_t CT_CAT(launch_k, CT_K)(const ConvLaunch& L, cudaStream_t s) {
  const void* fn = CT_CAT(pick_k, CT_K)(L.tx, L.ty, L.staging != kStageDirect, L.filt_smem != 0,
                                        L.bx * L.by >= kRingRemFirstThreads);
  if (!fn) return cudaErrorInvalidValue;
  constexpr int KP = tap_row_pad(K);
  ConvArgs<K * KP> a;
  memset(&a, 0, sizeof(a));
  if (L.tmap) a.tmap = *L.tmap;
  a.in = L.in;
  a.out = L.out;
  a.status = L.status;
  a.in_pitch = L.in_pitch;
  a.out_pitch = L.out_pitch;
  a.in_h = L.in_h;
  a.in_w = L.in_w;
  a.out_h = L.out_h;
  a.out_w = L.out_w;
  a.fh = L.fh;
  a.fw = L.fw;
  a.vw = L.vw;
  a.staging = L.staging;
  a.smem_pitch = L.smem_pitch;
  a.tile_w = L.tile_w;
  a.tile_h = L.tile_h;
  a.group_x = L.group_x;
  a.group_stride = L.group_stride;
  a.groups = L.groups;
  for (int j = 0; j < K; ++j) memcpy(a.w + j * KP, L.taps + j * K, sizeof(float) * K);
  const dim3 block(L.bx, L.by);
  const dim3 grid((L.out_w + L.bx * L.tx - 1) / (L.bx * L.tx),
                  (L.out_h + L.by * L.ty - 1) / (L.by * L.ty));
  void* args[] = {&a};
  // programmatic stream serialization: the launch and prologue may overlap
  // the previous kernel on the stream (the kernel waits before touching
  // global memory)
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = L.smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace convtune
