// peaks.cu -- per-SM issue rates of the units the closure's kernels lean on,
// measured on the GPU itself: MUFU ex2 (the exponential of every segment),
// FP32 FMA, packed f32x2 FMA, shared-memory loads of 8 and 16 bytes, and the
// cell pass's paired segment step on its own.
//
// One CTA of 1024 threads per SM runs independent dependency chains long
// enough that only the unit's throughput limits them; the CTA reads clock64
// around its loop, so a rate is results (or bytes) per SM clock, whatever
// the clock the GPU ran at.  Prints one JSON object.  Every loop is a fixed
// count: nothing waits on anything but its own arithmetic.
#include <cstdint>
#include <cstdio>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 1024;
constexpr int kChains = 8;

__device__ __forceinline__ void record(long long t0, long long t1, long long *cycles, float sink, float *out) {
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
  if (sink == 1234.5f) out[blockIdx.x] = sink;  // keeps the chains live
}

__global__ void __launch_bounds__(kThreads, 1) ex2_kernel(int iters, long long *cycles, float *out) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = -1.0f - 1e-3f * (threadIdx.x + j);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[j]));
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  record(t0, t1, cycles, s, out);
}

__global__ void __launch_bounds__(kThreads, 1) ffma_kernel(int iters, long long *cycles, float *out) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1e-3f * (threadIdx.x + j);
  const float m = 0.999f, c = 1e-4f;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[j]) : "f"(m), "f"(c));
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  record(t0, t1, cycles, s, out);
}

__global__ void __launch_bounds__(kThreads, 1) ffma2_kernel(int iters, long long *cycles, float *out) {
  uint64_t a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    const float v = 1e-3f * (threadIdx.x + j);
    a[j] = (uint64_t)__float_as_uint(v) | ((uint64_t)__float_as_uint(v + 1.f) << 32);
  }
  const uint64_t m = (uint64_t)__float_as_uint(0.999f) | ((uint64_t)__float_as_uint(0.999f) << 32);
  const uint64_t c = (uint64_t)__float_as_uint(1e-4f) | ((uint64_t)__float_as_uint(1e-4f) << 32);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(m), "l"(c));
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += __uint_as_float((uint32_t)a[j]) + __uint_as_float((uint32_t)(a[j] >> 32));
  record(t0, t1, cycles, s, out);
}

// Shared-memory loads of W bytes per thread: each warp reads consecutive
// W-byte words (conflict free), at an index that depends on the previous
// load so the loads form chains.
template <int W>
__global__ void __launch_bounds__(kThreads, 1) lds_kernel(int iters, long long *cycles, float *out) {
  constexpr int kWords = 8192;  // 64 or 128 KB of W-byte words
  using V = typename std::conditional<W == 8, uint2, uint4>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  V *buf = reinterpret_cast<V *>(smem);
  for (int i = threadIdx.x; i < kWords; i += blockDim.x) {
    V v;
    v.x = 0u;
    v.y = 0u;
    if constexpr (W == 16) {
      v.z = 0u;
      v.w = 0u;
    }
    buf[i] = v;
  }
  __syncthreads();
  unsigned idx[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) idx[j] = (threadIdx.x + 1024u * j) % kWords;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      const V v = buf[idx[j]];
      idx[j] = (idx[j] + v.x + 32u) % kWords;  // the words hold 0: consecutive, warp-contiguous
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += (float)idx[j];
  record(t0, t1, cycles, s, out);
}

// The cell pass's paired segment step in isolation: a 16-byte load of a
// (kappa, kappa', S, S') tile entry at an event's offset, the scaled optical
// depths (f32x2), two ex2, the thin-segment cubic (f32x2), and one f32x2 FMA
// on per-lane selected operands, per thread one ray pair marching through a
// synthetic tile with an event list in shared memory.  Reports the clocks one
// SM sub-partition spends per warp step (a ceiling on the march's rate).
__global__ void __launch_bounds__(kThreads, 1) step_kernel(int iters, long long *cycles, float *out) {
  extern __shared__ __align__(16) float4 tile[];  // 2048 entries, then 64 events
  float2 *ev = reinterpret_cast<float2 *>(tile + 2048);
  for (int i = threadIdx.x; i < 2048; i += blockDim.x)
    tile[i] = make_float4(0.1f + 0.3f * (i & 7), 0.2f + 0.4f * (i % 5), 1.f + (i & 3), 2.f);
  for (int i = threadIdx.x; i < 64; i += blockDim.x)
    ev[i] = make_float2(-0.5f - 0.01f * i, __int_as_float(((i * 37) % 61 - 30) * 16));
  __syncthreads();
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(tile) + 16u * (1024u + (threadIdx.x & 255u));
  float2 I = make_float2(0.f, 1.f);
  const float q3 = 8.70478970381660493e-03f, q2 = 5.53004379372010468e-02f, q1 = 2.40211763951330648e-01f,
              q0 = 6.93147011611337405e-01f, thr = -0.36067376022224085f;
  const long long t0 = clock64();
  for (int s = 0; s < iters; s += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 v = ev[(s + u) & 63];
      float4 q;
      asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(q.x), "=f"(q.y), "=f"(q.z), "=f"(q.w)
                   : "r"(base + (uint32_t)__float_as_int(v.y)));
      const float2 Y = __fmul2_rn(make_float2(q.x, q.y), make_float2(v.x, v.x));
      float e1, e2;
      asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(Y.x));
      asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e2) : "f"(Y.y));
      float2 p = __ffma2_rn(make_float2(q3, q3), Y, make_float2(q2, q2));
      p = __ffma2_rn(p, Y, make_float2(q1, q1));
      p = __ffma2_rn(p, Y, make_float2(q0, q0));
      const float2 n = __fmul2_rn(p, Y);
      const bool t1 = Y.x > thr, t2 = Y.y > thr;
      I = __ffma2_rn(__fadd2_rn(I, make_float2(-q.z, -q.w)), make_float2(t1 ? n.x : e1, t2 ? n.y : e2),
                     make_float2(t1 ? I.x : q.z, t2 ? I.y : q.w));
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  record(t0, t1, cycles, I.x + I.y, out);
}

template <typename K>
double per_sm_rate(K kernel, int nsm, int iters, size_t smem, double units_per_thread_iter) {
  long long *d_cycles = nullptr;
  float *d_out = nullptr;
  if (cudaMalloc(&d_cycles, sizeof(long long) * nsm) || cudaMalloc(&d_out, sizeof(float) * nsm)) return -1.0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1.0;
  kernel<<<nsm, kThreads, smem>>>(iters / 10, d_cycles, d_out);  // warm-up
  kernel<<<nsm, kThreads, smem>>>(iters, d_cycles, d_out);
  std::vector<long long> cyc(nsm);
  const bool ok = cudaDeviceSynchronize() == cudaSuccess &&
                  cudaMemcpy(cyc.data(), d_cycles, sizeof(long long) * nsm, cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(d_cycles);
  cudaFree(d_out);
  if (!ok) return -1.0;
  double mean = 0.0;
  for (long long c : cyc) mean += (double)c / nsm;
  return units_per_thread_iter * kThreads * (double)iters / mean;
}

}  // namespace

int main() {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) {
    std::printf("{\"error\": \"no CUDA device\"}\n");
    return 1;
  }
  // every launch asks for 128 KB of shared memory, so one CTA fits an SM and
  // each CTA's clock64 interval is its SM's alone
  const int nsm = p.multiProcessorCount, iters = 4096;
  const size_t one_per_sm = 128 << 10;
  const double ex2 = per_sm_rate(ex2_kernel, nsm, iters, one_per_sm, kChains);
  const double ffma = per_sm_rate(ffma_kernel, nsm, iters, one_per_sm, kChains);
  const double ffma2 = per_sm_rate(ffma2_kernel, nsm, iters, one_per_sm, 2.0 * kChains);
  const double lds8 = per_sm_rate(lds_kernel<8>, nsm, iters, one_per_sm, 8.0 * kChains);
  const double lds16 = per_sm_rate(lds_kernel<16>, nsm, iters, one_per_sm, 16.0 * kChains);
  // warp steps per SM clock -> SM sub-partition clocks per warp step
  const double steps = per_sm_rate(step_kernel, nsm, iters, one_per_sm, 1.0 / 32.0);
  const double step_clk = steps > 0 ? 4.0 / steps : -1.0;
  std::printf(
      "{\"device\": \"%s\", \"sms\": %d, \"ex2_per_clk_per_sm\": %.2f, \"ffma_lanes_per_clk_per_sm\": %.2f, "
      "\"ffma2_lanes_per_clk_per_sm\": %.2f, \"lds64_bytes_per_clk_per_sm\": %.2f, "
      "\"lds128_bytes_per_clk_per_sm\": %.2f, \"march_step_clk_per_smsp\": %.2f}\n",
      p.name, nsm, ex2, ffma, ffma2, lds8, lds16, step_clk);
  return (ex2 > 0 && ffma > 0 && ffma2 > 0 && lds8 > 0 && lds16 > 0 && step_clk > 0) ? 0 : 1;
}
