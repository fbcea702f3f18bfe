// vet_hlle.cu -- the HLLE face wavespeed with the optical-depth correction
// (Sec. 2.2.3, App. A), the first consumer of the Eddington tensor:
//   C = sqrt(f_aa) c sqrt((1 - e^-tau_c) / tau_c),
//   tau_c = (10 h kappa_R)^2 / (2 f_aa) per cell, averaged over the two
// cells of a face (one refinement level); the free-streaming factor of a face
// is the larger of the two cells' sqrt(f_aa); a domain-boundary face takes
// its one cell's values; f_aa <= 0 gives tau = inf (factor 0), kappa_R = 0
// gives tau = 0 (correction 1).
//
// Memory-bound: per face two cells' f_aa and kappa_R read (each cell is read
// by its two faces along the axis; the second read hits in cache) and one
// speed written.
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "vet.h"
#include "vet_internal.h"

namespace {

struct HlleArgs {
  int nx, ny, nz;  // cells
  int fx, fy;      // face grid extents along x and y (fz follows from the count)
  int axis;        // 0, 1, 2: faces normal to x, y, z
  long long ncell, nface;
  float tenh;      // 10 h
  float c;
};

// tau_c of one cell (inf where f_aa <= 0).
__device__ __forceinline__ float cell_tau(float faa, float kap, float tenh) {
  const float a = tenh * kap;
  return faa > 0.f ? __fdividef(0.5f * a * a, faa) : __int_as_float(0x7f800000);
}

// The square of the correction, (1 - e^-tau) / tau: 1 at tau = 0, 0 at
// tau = inf.  Below tau = 1/4 the ratio is log2(e) q(y), y = -tau log2(e),
// with q the thin-segment cubic of the ray march (relative error 3.4e-7: no
// cancellation); above, (1 - e^-tau) / tau with the MUFU exponential and a
// fast quotient (a few ulp; 1 / inf = 0 at tau = inf).
__device__ __forceinline__ float correction_sq(float tau) {
  const float y = -1.4426950408889634f * tau;
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(y));
  const float q = fmaf(fmaf(fmaf(vet::kThinQ3, y, vet::kThinQ2), y, vet::kThinQ1), y, vet::kThinQ0);
  return y > vet::kThinY ? 1.4426950408889634f * q : __fdividef(1.f - e, tau);
}

// sqrt(max(f_L, f_R)) c sqrt(corr) as one square root of the product, by
// the MUFU square root (relative error of order 2^-23)
__device__ __forceinline__ float face_speed(float fL, float tL, float fR, float tR, float c) {
  const float x = fmaxf(fmaxf(fL, fR), 0.f) * correction_sq(0.5f * (tL + tR));
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return c * r;
}

// n / d for n < 2^31 and a divisor d >= 2 fixed per launch: m = ceil(2^32
// / d), the high word of n m is n / d or one more (d = 1: m = 0, n itself).
struct Div {
  unsigned d, m;
};
__device__ __forceinline__ unsigned div_q(unsigned n, Div v) {
  if (v.m == 0) return n;
  const unsigned q = __umulhi(n, v.m);
  return q * v.d > n ? q - 1 : q;
}

// Each thread takes kFaces consecutive faces of a row of the face grid
// (threads numbered along x first: a warp's loads are contiguous runs), forms
// each cell's tau once (a cell serves two faces along x) and issues all its
// loads before any arithmetic; row and position come from two divisions by
// launch constants (multiply-high), a grid-stride loop beyond the first wave.
constexpr int kFaces = 4;
__global__ void __launch_bounds__(128) hlle_kernel(HlleArgs a, Div per_row_div, Div fy_div, const float *__restrict__ faa,
                                                   const float *__restrict__ kap, float *__restrict__ C) {
  const long long along = a.axis == 0 ? 1 : (a.axis == 1 ? a.nx : (long long)a.nx * a.ny);
  const int n_along = a.axis == 0 ? a.nx : (a.axis == 1 ? a.ny : a.nz);
  const unsigned items = (unsigned)(a.nface / a.fx) * per_row_div.d;
  for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
    const unsigned r = div_q(it, per_row_div);
    const int x0 = (int)(it - r * per_row_div.d) * kFaces;
    const unsigned z = div_q(r, fy_div);
    const int y = (int)(r - z * fy_div.d);
    const long long row_cell = ((long long)z * a.ny + y) * a.nx;
    float out[kFaces];
    if (a.axis == 0) {
      // cells x0 - 1 .. x0 + kFaces - 1 of the row (clamped to the row)
      float f[kFaces + 1], t[kFaces + 1];
#pragma unroll
      for (int j = 0; j <= kFaces; ++j) {
        const int cx = min(max(x0 - 1 + j, 0), a.nx - 1);
        f[j] = faa[row_cell + cx];
        t[j] = kap[row_cell + cx];
      }
#pragma unroll
      for (int j = 0; j <= kFaces; ++j) t[j] = cell_tau(f[j], t[j], a.tenh);
#pragma unroll
      for (int j = 0; j < kFaces; ++j) out[j] = face_speed(f[j], t[j], f[j + 1], t[j + 1], a.c);
    } else {
      // the face's two cells are one row apart along y or z
      const int tt = a.axis == 1 ? y : (int)z;
      const long long hi = row_cell, lo = tt > 0 ? hi - along : hi;
      const long long h2 = tt < n_along ? hi : lo;
      float fl[kFaces], tl[kFaces], fh[kFaces], th[kFaces];
#pragma unroll
      for (int j = 0; j < kFaces; ++j) {
        const int cx = min(x0 + j, a.nx - 1);
        fl[j] = faa[lo + cx];
        tl[j] = kap[lo + cx];
        fh[j] = faa[h2 + cx];
        th[j] = kap[h2 + cx];
      }
#pragma unroll
      for (int j = 0; j < kFaces; ++j)
        out[j] = face_speed(fl[j], cell_tau(fl[j], tl[j], a.tenh), fh[j], cell_tau(fh[j], th[j], a.tenh), a.c);
    }
    float *Crow = C + (long long)r * a.fx;
#pragma unroll
    for (int j = 0; j < kFaces; ++j)
      if (x0 + j < a.fx) Crow[x0 + j] = out[j];
  }
}

Div make_div(unsigned d) { return {d, d < 2 ? 0u : (unsigned)((((unsigned long long)1 << 32) + d - 1) / d)}; }

bool on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) vet_status vet_hlle_wavespeed(const vet_grid *grid, const float *f,
                                                                             const float *kappa_R, double c, int axis,
                                                                             float *C_out, void *stream) {
  if (!grid || !f || !kappa_R || !C_out || axis < 0 || axis > 2 || !(c > 0.0) || !std::isfinite(c)) return VET_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->h > 0.0) || !std::isfinite(grid->h)) return VET_EINVAL;
  if (!on_device(f) || !on_device(kappa_R) || !on_device(C_out)) return VET_EINVAL;
  HlleArgs a;
  a.nx = grid->nx;
  a.ny = grid->ny;
  a.nz = grid->nz;
  a.axis = axis;
  a.fx = grid->nx + (axis == 0);
  a.fy = grid->ny + (axis == 1);
  const int fz = grid->nz + (axis == 2);
  a.ncell = (long long)grid->nx * grid->ny * grid->nz;
  a.nface = (long long)a.fx * a.fy * fz;
  a.tenh = (float)(10.0 * grid->h);
  a.c = (float)c;
  const long long rows = (long long)a.fy * fz;
  if (rows > 0x7fffffffLL) return VET_EINVAL;
  const long long per_row = (a.fx + kFaces - 1) / kFaces;
  const long long items = rows * per_row;
  if (items > 0x7fffffffLL) return VET_EINVAL;
  long long blocks = (items + 127) / 128;
  if (blocks > 152LL * 16) blocks = 152LL * 16;  // grid-stride beyond
  hlle_kernel<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(a, make_div((unsigned)per_row), make_div((unsigned)a.fy),
                                                                  f + (long long)axis * a.ncell, kappa_R, C_out);
  return cudaGetLastError() == cudaSuccess ? VET_OK : VET_ECUDA;
}
