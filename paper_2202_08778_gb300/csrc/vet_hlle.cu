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

constexpr float kLog2e = 1.4426950408889634f;

// What a face needs of one of its cells: fc = max(f_aa, 0) and
// ty = -log2(e) tau_c / 2, so that a face's y = ty_L + ty_R is -log2(e)
// times the mean of its cells' tau_c = (10 h kappa_R)^2 / (2 f_aa); ty = -inf
// where f_aa <= 0 (tau_c = inf).  kt = -log2(e) (10 h)^2 / 4, per launch.
struct CellV {
  float fc, ty;
};
__device__ __forceinline__ CellV cell_prep(float faa, float kap, float kt) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(faa));
  return {fmaxf(faa, 0.f), faa > 0.f ? kt * kap * kap * r : __int_as_float(0xff800000)};
}

// C = c sqrt(max(fc_L, fc_R) (1 - e^-tau) / tau), tau the cells' mean tau_c.
// Below tau = 1/4 (y = -tau log2(e) above the thin threshold) the ratio is
// log2(e) q(y), q the thin-segment cubic of the ray march (relative error
// 3.4e-7: no cancellation); above, (e^-tau - 1) log2(e) / y with the MUFU
// exponential and reciprocal (y = -inf: 0).  One MUFU square root.
__device__ __forceinline__ float face_speed(CellV L, CellV R, float c) {
  constexpr float q3 = vet::kThinQ3 * kLog2e, q2 = vet::kThinQ2 * kLog2e, q1 = vet::kThinQ1 * kLog2e,
                  q0 = vet::kThinQ0 * kLog2e;
  const float y = L.ty + R.ty;
  float e, ry;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(y));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(y));
  const float k = kLog2e * ry;
  const float corr = y > vet::kThinY ? fmaf(fmaf(fmaf(q3, y, q2), y, q1), y, q0) : fmaf(e, k, -k);
  const float x = fmaxf(L.fc, R.fc) * corr;
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
// (threads numbered along x first: a warp's loads are contiguous runs),
// prepares each cell once (a cell serves two faces along x) and issues all
// its loads before any arithmetic; row and position come from two
// divisions by launch constants (multiply-high), a grid-stride loop beyond
// the first wave.  AXIS is the faces' normal; I the index type (32-bit
// where the cells and faces allow); VEC where nx is a multiple of 4 and the
// arrays are 16-byte aligned: a thread's cells along x are one 16-byte load
// (x-normal faces: plus the cell to the left), and its four y- or z-normal
// faces one 16-byte store.
constexpr int kFaces = 4;
template <int AXIS, typename I, bool VEC>
__global__ void __launch_bounds__(128) hlle_kernel(HlleArgs a, Div per_row_div, Div fy_div, const float *__restrict__ faa,
                                                   const float *__restrict__ kap, float *__restrict__ C) {
  const I along = AXIS == 0 ? 1 : (AXIS == 1 ? (I)a.nx : (I)a.nx * a.ny);
  const int n_along = AXIS == 0 ? a.nx : (AXIS == 1 ? a.ny : a.nz);
  const float kt = (-0.25f * kLog2e) * a.tenh * a.tenh;
  const unsigned items = (unsigned)(a.nface / a.fx) * per_row_div.d;
  for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
    const unsigned r = div_q(it, per_row_div);
    const int x0 = (int)(it - r * per_row_div.d) * kFaces;
    const unsigned z = div_q(r, fy_div);
    const int y = (int)(r - z * fy_div.d);
    const I row_cell = ((I)z * a.ny + y) * a.nx;
    float out[kFaces];
    if (AXIS == 0 && VEC) {
      // cells x0 - 1 (clamped) and x0 .. x0 + 3; the row's last item
      // (x0 = nx) holds only the face at the row's end, whose cells are both
      // nx - 1 (its 16-byte load stays in the row and goes unused)
      const I q = row_cell + min(x0, a.nx - 4), l = row_cell + max(x0 - 1, 0);
      const float4 f4 = *reinterpret_cast<const float4 *>(faa + q);
      const float4 k4 = *reinterpret_cast<const float4 *>(kap + q);
      const float fl = faa[l], kl = kap[l];
      CellV v[kFaces + 1];
      v[0] = cell_prep(fl, kl, kt);
      v[1] = cell_prep(f4.x, k4.x, kt);
      v[2] = cell_prep(f4.y, k4.y, kt);
      v[3] = cell_prep(f4.z, k4.z, kt);
      v[4] = cell_prep(f4.w, k4.w, kt);
      if (x0 >= a.nx) v[1] = v[0];
#pragma unroll
      for (int j = 0; j < kFaces; ++j) out[j] = face_speed(v[j], v[j + 1], a.c);
    } else if (AXIS == 0) {
      // cells x0 - 1 .. x0 + kFaces - 1 of the row (clamped to the row)
      float f[kFaces + 1], t[kFaces + 1];
#pragma unroll
      for (int j = 0; j <= kFaces; ++j) {
        const int cx = min(max(x0 - 1 + j, 0), a.nx - 1);
        f[j] = faa[row_cell + cx];
        t[j] = kap[row_cell + cx];
      }
      CellV v[kFaces + 1];
#pragma unroll
      for (int j = 0; j <= kFaces; ++j) v[j] = cell_prep(f[j], t[j], kt);
#pragma unroll
      for (int j = 0; j < kFaces; ++j) out[j] = face_speed(v[j], v[j + 1], a.c);
    } else {
      // the face's two cells are one row apart along y or z
      const int tt = AXIS == 1 ? y : (int)z;
      const I hi = row_cell, lo = tt > 0 ? hi - along : hi;
      const I h2 = tt < n_along ? hi : lo;
      float fl[kFaces], tl[kFaces], fh[kFaces], th[kFaces];
      if (VEC) {
        const float4 a4 = *reinterpret_cast<const float4 *>(faa + lo + x0);
        const float4 b4 = *reinterpret_cast<const float4 *>(kap + lo + x0);
        const float4 c4 = *reinterpret_cast<const float4 *>(faa + h2 + x0);
        const float4 d4 = *reinterpret_cast<const float4 *>(kap + h2 + x0);
        fl[0] = a4.x, fl[1] = a4.y, fl[2] = a4.z, fl[3] = a4.w;
        tl[0] = b4.x, tl[1] = b4.y, tl[2] = b4.z, tl[3] = b4.w;
        fh[0] = c4.x, fh[1] = c4.y, fh[2] = c4.z, fh[3] = c4.w;
        th[0] = d4.x, th[1] = d4.y, th[2] = d4.z, th[3] = d4.w;
      } else {
#pragma unroll
        for (int j = 0; j < kFaces; ++j) {
          const int cx = min(x0 + j, a.nx - 1);
          fl[j] = faa[lo + cx];
          tl[j] = kap[lo + cx];
          fh[j] = faa[h2 + cx];
          th[j] = kap[h2 + cx];
        }
      }
#pragma unroll
      for (int j = 0; j < kFaces; ++j)
        out[j] = face_speed(cell_prep(fl[j], tl[j], kt), cell_prep(fh[j], th[j], kt), a.c);
    }
    float *Crow = C + (I)r * a.fx;
    if (AXIS != 0 && VEC) {
      *reinterpret_cast<float4 *>(Crow + x0) = make_float4(out[0], out[1], out[2], out[3]);
    } else {
#pragma unroll
      for (int j = 0; j < kFaces; ++j)
        if (x0 + j < a.fx) Crow[x0 + j] = out[j];
    }
  }
}

template <int AXIS, typename I>
void launch_vec(bool vec, dim3 g, cudaStream_t st, const HlleArgs &a, Div d1, Div d2, const float *fa, const float *k,
                float *C) {
  if (vec) hlle_kernel<AXIS, I, true><<<g, 128, 0, st>>>(a, d1, d2, fa, k, C);
  else hlle_kernel<AXIS, I, false><<<g, 128, 0, st>>>(a, d1, d2, fa, k, C);
}
template <int AXIS>
void launch_index(bool narrow, bool vec, dim3 g, cudaStream_t st, const HlleArgs &a, Div d1, Div d2, const float *fa,
                  const float *k, float *C) {
  if (narrow) launch_vec<AXIS, int>(vec, g, st, a, d1, d2, fa, k, C);
  else launch_vec<AXIS, long long>(vec, g, st, a, d1, d2, fa, k, C);
}
void launch_axis(int axis, bool narrow, bool vec, dim3 g, cudaStream_t st, const HlleArgs &a, Div d1, Div d2,
                 const float *fa, const float *k, float *C) {
  if (axis == 0) launch_index<0>(narrow, vec, g, st, a, d1, d2, fa, k, C);
  else if (axis == 1) launch_index<1>(narrow, vec, g, st, a, d1, d2, fa, k, C);
  else launch_index<2>(narrow, vec, g, st, a, d1, d2, fa, k, C);
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
  const Div d1 = make_div((unsigned)per_row), d2 = make_div((unsigned)a.fy);
  const float *fa = f + (long long)axis * a.ncell;
  const dim3 gdim((unsigned)blocks);
  cudaStream_t st = (cudaStream_t)stream;
  // 32-bit indices where every cell and face index fits; 16-byte cell runs
  // where rows are whole 16-byte runs
  const bool narrow = a.ncell < 0x7fffffffLL && a.nface < 0x7fffffffLL;
  const bool vec = a.nx % 4 == 0 && ((reinterpret_cast<uintptr_t>(fa) | reinterpret_cast<uintptr_t>(kappa_R) |
                                       reinterpret_cast<uintptr_t>(C_out)) & 15) == 0;
  launch_axis(axis, narrow, vec, gdim, st, a, d1, d2, fa, kappa_R, C_out);
  return cudaGetLastError() == cudaSuccess ? VET_OK : VET_ECUDA;
}
