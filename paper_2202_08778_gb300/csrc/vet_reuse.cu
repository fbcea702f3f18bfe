// vet_reuse.cu -- the change gate behind reusing the Eddington tensor across
// time steps (paper Sec. 4.2, the suggestion of recomputing f only every few
// steps).  Per block of B^3 cells and over the grid it finds
//   dtrans = max |a - b| / ((1 + a/2) (1 + b/2)),  a = kappa h, b = kappa_ref h,
//            a bound on the change |e^{-a} - e^{-b}| of the cell's
//            transmission (e^t >= (1 + t/2)^2), which is what moves the
//            intensity leaving the cell under Eq. 14;
//   dS     = max |S - S_ref|,   Sref = max |S_ref|,
// in FP32 with every operation an explicitly rounded IEEE one (no
// contraction), so the result is exact for the given inputs and a maximum
// does not depend on the reduction order; a NaN counts as +inf.  With the
// snapshot flag the same pass also writes kappa_ref <- kappa and
// S_ref <- S, each thread after its own reads.
//
// Memory-bound: 16 bytes read per cell (8 more written with the snapshot).
// One CTA per block; each thread takes 16-byte runs along x where the block
// edge is a multiple of 4 and the fields are 16-byte aligned (scalar cells
// otherwise), keeps its three maxima in registers, and the CTA reduces them
// with warp shuffles and one shared-memory step.  The grid's maxima are
// folded in with integer atomicMax on the float bits, which orders
// non-negative floats (and +inf) correctly.
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "vet.h"

namespace {

struct GateArgs {
  int nx, ny, nz, B;
  int nbx, nby;
  float h;
  int snapshot;
};

__device__ __forceinline__ float nan_to_inf(float x) { return x != x ? INFINITY : x; }

__device__ __forceinline__ void gate_cell(float k, float s, float kr, float sr, float h, float m[3]) {
  const float a = __fmul_rn(k, h), b = __fmul_rn(kr, h);
  const float den = __fmul_rn(__fadd_rn(1.f, __fmul_rn(0.5f, a)), __fadd_rn(1.f, __fmul_rn(0.5f, b)));
  m[0] = fmaxf(m[0], nan_to_inf(__fdiv_rn(fabsf(__fsub_rn(a, b)), den)));
  m[1] = fmaxf(m[1], nan_to_inf(fabsf(__fsub_rn(s, sr))));
  m[2] = fmaxf(m[2], nan_to_inf(fabsf(sr)));
}

template <bool VEC>
__global__ void __launch_bounds__(256, 4) gate_kernel(GateArgs a, const float *__restrict__ kappa,
                                                   const float *__restrict__ S, float *__restrict__ kappa_ref,
                                                   float *__restrict__ S_ref, float *__restrict__ out) {
  const int b = blockIdx.x;
  const int bi = b % a.nbx, bj = (b / a.nbx) % a.nby, bk = b / (a.nbx * a.nby);
  const int B = a.B;
  const long long x0 = (long long)bi * B, y0 = (long long)bj * B, z0 = (long long)bk * B;
  float m[3] = {0.f, 0.f, 0.f};
  if (VEC) {
    const int q = B / 4;  // 16-byte runs per row
    const int nq = B * B * q;
    // two runs per thread per trip, all eight loads issued before any use
    for (int u0 = threadIdx.x; u0 < nq; u0 += 2 * blockDim.x) {
      float4 k[2], s[2], kr[2], sr[2];
      long long c[2];
      bool ok[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int u = u0 + r * blockDim.x;
        ok[r] = u < nq;
        const int uu = ok[r] ? u : u0;
        const int row = uu / q, xq = uu - row * q;
        const int y = row % B, z = row / B;
        c[r] = ((z0 + z) * a.ny + y0 + y) * a.nx + x0 + 4 * xq;
        k[r] = *reinterpret_cast<const float4 *>(kappa + c[r]);
        s[r] = *reinterpret_cast<const float4 *>(S + c[r]);
        kr[r] = *reinterpret_cast<const float4 *>(kappa_ref + c[r]);
        sr[r] = *reinterpret_cast<const float4 *>(S_ref + c[r]);
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!ok[r]) continue;
        gate_cell(k[r].x, s[r].x, kr[r].x, sr[r].x, a.h, m);
        gate_cell(k[r].y, s[r].y, kr[r].y, sr[r].y, a.h, m);
        gate_cell(k[r].z, s[r].z, kr[r].z, sr[r].z, a.h, m);
        gate_cell(k[r].w, s[r].w, kr[r].w, sr[r].w, a.h, m);
        if (a.snapshot) {
          *reinterpret_cast<float4 *>(kappa_ref + c[r]) = k[r];
          *reinterpret_cast<float4 *>(S_ref + c[r]) = s[r];
        }
      }
    }
  } else {
    const int n = B * B * B;
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
      const int x = u % B, y = (u / B) % B, z = u / (B * B);
      const long long c = ((z0 + z) * a.ny + y0 + y) * a.nx + x0 + x;
      const float k = kappa[c], s = S[c], kr = kappa_ref[c], sr = S_ref[c];
      gate_cell(k, s, kr, sr, a.h, m);
      if (a.snapshot) {
        kappa_ref[c] = k;
        S_ref[c] = s;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int t = 0; t < 3; ++t) m[t] = fmaxf(m[t], __shfl_xor_sync(0xffffffffu, m[t], o));
  __shared__ float red[8][3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int t = 0; t < 3; ++t) red[warp][t] = m[t];
  __syncthreads();
  if (threadIdx.x < 3) {
    float v = red[0][threadIdx.x];
    for (int w = 1; w < nw; ++w) v = fmaxf(v, red[w][threadIdx.x]);
    out[3 + 3 * (long long)b + threadIdx.x] = v;
    atomicMax(reinterpret_cast<int *>(out) + threadIdx.x, __float_as_int(v));
  }
}

bool on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" __attribute__((visibility("default"))) vet_status vet_field_change(const vet_grid *grid, const float *kappa,
                                                                                const float *S, float *kappa_ref,
                                                                                float *S_ref, int snapshot, float *out,
                                                                                void *stream) {
  if (!grid || !kappa || !S || !kappa_ref || !S_ref || !out) return VET_EINVAL;
  const int B = grid->block;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || B < 2 || B > 32 || grid->nx % B || grid->ny % B ||
      grid->nz % B || !(grid->h > 0.0) || !std::isfinite(grid->h))
    return VET_EINVAL;
  if (!on_device(kappa) || !on_device(S) || !on_device(kappa_ref) || !on_device(S_ref) || !on_device(out))
    return VET_EINVAL;
  GateArgs a;
  a.nx = grid->nx;
  a.ny = grid->ny;
  a.nz = grid->nz;
  a.B = B;
  a.nbx = grid->nx / B;
  a.nby = grid->ny / B;
  a.h = (float)grid->h;
  a.snapshot = snapshot != 0;
  const long long nb = (long long)a.nbx * a.nby * (grid->nz / B);
  if (nb > 0x7fffffffLL) return VET_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(out, 0, 3 * sizeof(float), st) != cudaSuccess) {
    cudaGetLastError();
    return VET_ECUDA;
  }
  const bool vec = B % 4 == 0 && aligned16(kappa) && aligned16(S) && aligned16(kappa_ref) && aligned16(S_ref);
  const int work = vec ? B * B * B / 4 : B * B * B;
  const int threads = work >= 256 ? 256 : ((work + 31) / 32) * 32;
  if (vec)
    gate_kernel<true><<<(unsigned)nb, threads, 0, st>>>(a, kappa, S, kappa_ref, S_ref, out);
  else
    gate_kernel<false><<<(unsigned)nb, threads, 0, st>>>(a, kappa, S, kappa_ref, S_ref, out);
  return cudaGetLastError() == cudaSuccess ? VET_OK : VET_ECUDA;
}

// The decision the gate serves (Sec. 4.2 reading): recompute on the first
// step, once the stored f is max_age steps old, when a change is not finite,
// or when the grid's transmission bound or source change exceeds its
// tolerance (the source's relative to its scale).  Host arithmetic in double
// on the FP32 triple, exactly as the oracle takes it.
extern "C" __attribute__((visibility("default"))) vet_status vet_reuse_decision(const float *change, int age, int first, double tol_tau, double tol_S,
                                      int max_age, int *recompute) {
  if (!change || !recompute || max_age < 1 || age < 0 || !(tol_tau >= 0.0) || !(tol_S >= 0.0)) return VET_EINVAL;
  const double dtau = change[0], dS = change[1], sref = change[2];
  if (first || age >= max_age || !std::isfinite(dtau) || !std::isfinite(dS))
    *recompute = 1;
  else
    *recompute = (dtau > tol_tau || dS > tol_S * sref) ? 1 : 0;
  return VET_OK;
}
