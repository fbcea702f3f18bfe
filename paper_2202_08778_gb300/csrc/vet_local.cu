// vet_local.cu -- the local closures the paper compares the VET closure with
// (Sec. 4.1): Eddington, T = I / 3, and M1,
//   T = (1 - chi)/2 I + (3 chi - 1)/2 n n,  n = F / |F|,
//   chi(f) = (3 + 4 f^2) / (5 + 2 sqrt(4 - 3 f^2)),  f = |F| / E (c = 1),
// from the moments of each cell.  f is clipped to [0, 1]; F = 0 leaves
// chi = 1/3 (the n n term vanishes); E <= 0 gives I / 3.
//
// Memory-bound: per cell 16 bytes read (E, Fx, Fy, Fz of M [10][cells]) and
// 24 bytes written (T [6][cells]).  Each thread takes 4 consecutive cells
// with 16-byte loads and stores where the layout allows (cells a multiple of
// 4, 16-byte aligned rows), scalar accesses otherwise; a grid-stride loop
// over a grid sized to the SMs.
#include <cstdint>

#include <cuda_runtime.h>

#include "vet.h"

namespace {

__device__ __forceinline__ void m1_cell(float E, float Fx, float Fy, float Fz, float t[6]) {
  if (!(E > 0.f)) {
    t[0] = t[1] = t[2] = 1.f / 3.f;
    t[3] = t[4] = t[5] = 0.f;
    return;
  }
  const float F2 = fmaf(Fx, Fx, fmaf(Fy, Fy, Fz * Fz));
  const float Fn = sqrtf(F2);
  const float f = fminf(Fn / E, 1.f);
  const float f2 = f * f;
  const float chi = (3.f + 4.f * f2) / (5.f + 2.f * sqrtf(4.f - 3.f * f2));
  const float a = 0.5f * (1.f - chi), b = 0.5f * (3.f * chi - 1.f);
  const float inv = Fn > 0.f ? 1.f / Fn : 0.f;  // b = 0 where F = 0
  const float nx = Fx * inv, ny = Fy * inv, nz = Fz * inv;
  t[0] = fmaf(b, nx * nx, a);
  t[1] = fmaf(b, ny * ny, a);
  t[2] = fmaf(b, nz * nz, a);
  t[3] = b * nx * ny;
  t[4] = b * nx * nz;
  t[5] = b * ny * nz;
}

template <bool VEC>
__global__ void __launch_bounds__(256) m1_kernel(long long ncell, const float *__restrict__ M, float *__restrict__ T) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  if constexpr (VEC) {
    const long long n4 = ncell / 4;
    const float4 *E4 = reinterpret_cast<const float4 *>(M);
    const float4 *X4 = reinterpret_cast<const float4 *>(M + ncell);
    const float4 *Y4 = reinterpret_cast<const float4 *>(M + 2 * ncell);
    const float4 *Z4 = reinterpret_cast<const float4 *>(M + 3 * ncell);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 e = E4[i], x = X4[i], y = Y4[i], z = Z4[i];
      float t0[6], t1[6], t2[6], t3[6];
      m1_cell(e.x, x.x, y.x, z.x, t0);
      m1_cell(e.y, x.y, y.y, z.y, t1);
      m1_cell(e.z, x.z, y.z, z.z, t2);
      m1_cell(e.w, x.w, y.w, z.w, t3);
#pragma unroll
      for (int m = 0; m < 6; ++m)
        reinterpret_cast<float4 *>(T + m * ncell)[i] = make_float4(t0[m], t1[m], t2[m], t3[m]);
    }
  } else {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += stride) {
      float t[6];
      m1_cell(M[c], M[ncell + c], M[2 * ncell + c], M[3 * ncell + c], t);
#pragma unroll
      for (int m = 0; m < 6; ++m) T[m * ncell + c] = t[m];
    }
  }
}

__global__ void __launch_bounds__(256) eddington_kernel(long long ncell, float *__restrict__ T) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 6 * ncell; i += stride)
    T[i] = i < 3 * ncell ? 1.f / 3.f : 0.f;
}

bool is_device(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) vet_status vet_local_closure(int kind, long long ncell,
                                                                                 const float *M, float *T_out,
                                                                                 void *stream) {
  if (ncell < 0 || !T_out || (kind != VET_CLOSURE_EDDINGTON && kind != VET_CLOSURE_M1)) return VET_EINVAL;
  if (kind == VET_CLOSURE_M1 && !M) return VET_EINVAL;
  if (ncell == 0) return VET_OK;
  if (!is_device(T_out) || (M && kind == VET_CLOSURE_M1 && !is_device(M))) return VET_EINVAL;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) {
    cudaGetLastError();
    return VET_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = 8 * sms;  // 8 CTAs of 256 threads per SM, grid-stride
  if (kind == VET_CLOSURE_EDDINGTON) {
    eddington_kernel<<<grid, 256, 0, st>>>(ncell, T_out);
  } else {
    const bool vec = ncell % 4 == 0 && ((uintptr_t)M % 16) == 0 && ((uintptr_t)T_out % 16) == 0;
    if (vec)
      m1_kernel<true><<<grid, 256, 0, st>>>(ncell, M, T_out);
    else
      m1_kernel<false><<<grid, 256, 0, st>>>(ncell, M, T_out);
  }
  return cudaGetLastError() == cudaSuccess ? VET_OK : VET_ECUDA;
}
