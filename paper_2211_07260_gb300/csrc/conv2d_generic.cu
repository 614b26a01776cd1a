// Instantiation unit of the generic correlation kernel (any filter shape up
// to fh * fw <= 1024; one output per thread; taps in shared memory).
#include <string.h>

#include "conv2d_kernels.cuh"
#include "conv2d_launch.h"

namespace convtune {

// Generic kernel: any fh x fw with fh * fw <= kGenericMaxTaps, one output per
// thread, taps from shared memory, loops not unrolled.  Same fmaf order.
__global__ void conv2d_generic_kernel(const __grid_constant__ ConvArgs<kGenericMaxTaps> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* sfilt = reinterpret_cast<float*>(smem_raw);
  const int ntaps = a.fh * a.fw;
  for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < ntaps; k += blockDim.x * blockDim.y)
    sfilt[k] = a.w[k];
  __syncthreads();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= a.out_w || y >= a.out_h) return;
  float acc = 0.0f;
  for (int j = 0; j < a.fh; ++j) {
    const float* row = a.in + (long long)(y + j) * a.in_pitch + x;
    for (int i = 0; i < a.fw; ++i) acc = fmaf(__ldg(row + i), sfilt[j * a.fw + i], acc);
  }
  a.out[(long long)y * a.out_pitch + x] = acc;
}

const void* pick_generic() { return (const void*)conv2d_generic_kernel; }

cudaError_t launch_generic(const ConvLaunch& L, cudaStream_t s) {
  if (L.fh * L.fw > kGenericMaxTaps) return cudaErrorInvalidValue;
  // The parameter block (4 KB of taps) lives on this host frame;
  // cudaLaunchKernel copies it into the launch.
  ConvArgs<kGenericMaxTaps> a;
  memset(&a, 0, sizeof(a));
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
  a.vw = 1;
  a.staging = kStageDirect;
  memcpy(a.w, L.taps, sizeof(float) * L.fh * L.fw);
  const dim3 block(L.bx, L.by);
  const dim3 grid((L.out_w + L.bx - 1) / L.bx, (L.out_h + L.by - 1) / L.by);
  void* args[] = {&a};
  return cudaLaunchKernel((const void*)conv2d_generic_kernel, grid, block, args,
                          sizeof(float) * L.fh * L.fw, s);
}

}  // namespace convtune
