// vet_point.cu -- direct radiation of a point source (paper Sec. 2.2.6):
// the energy and momentum a source of luminosity L at x_s deposits in every
// cell, from the optical depth along the straight ray from x_s through the
// cell centre (long characteristics, the limit of the paper's hybrid
// tracer):
//   tau_*    sum kappa * length over the cells the ray crosses from x_s to
//            where it enters cell c (0 if the source lies in c),
//   dr       the ray's length inside c (from its entry, or from x_s),
//   Edot     L e^{-tau_*} (1 - e^{-kappa_c dr}) / (4 pi r^2 dr), r = |x_c - x_s|,
//            with 1 - e^{-x} = -expm1(-x): the small-tau Taylor form needs
//            no switch,
//   pdot     Edot (x_c - x_s) / r (c = 1).
// A ray point on a cell face lies in the cell the ray enters next; a cell
// whose centre is the source gets zeros.
//
// One thread per cell (grid-stride, x fastest): the rays of a warp start at
// the same point and stay close, so their kappa reads are near one another
// in the caches; each thread walks four steps ahead of its sum of tau, so
// that four reads are in flight.  Geometry in cell units (planes at integers); every plane
// crossing is computed from the source position, not accumulated, so a
// crossing's error is a few ulp of its own distance.  The walk crosses at
// most |di| + |dj| + |dk| + 1 cells and is capped at nx + ny + nz + 3 steps.
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "vet.h"

namespace {

struct PointArgs {
  int nx, ny, nz;
  float h;
  float xs[3];  // source, cell units
  float L;
};

__global__ void __launch_bounds__(256) point_kernel(PointArgs a, const float *__restrict__ kappa,
                                                   float *__restrict__ Edot, float *__restrict__ pdot) {
  const long long ncell = (long long)a.nx * a.ny * a.nz;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int cap = a.nx + a.ny + a.nz + 3;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += stride) {
    const int i = (int)(c % a.nx), j = (int)((c / a.nx) % a.ny), k = (int)(c / ((long long)a.nx * a.ny));
    const float xc[3] = {i + 0.5f, j + 0.5f, k + 0.5f};
    float v[3] = {xc[0] - a.xs[0], xc[1] - a.xs[1], xc[2] - a.xs[2]};
    const float r = sqrtf(fmaf(v[0], v[0], fmaf(v[1], v[1], v[2] * v[2])));
    if (!(r > 0.f)) {
      Edot[c] = 0.f;
      if (pdot) pdot[c] = pdot[ncell + c] = pdot[2 * ncell + c] = 0.f;
      continue;
    }
    float d[3], inv[3];
    for (int q = 0; q < 3; ++q) {
      d[q] = v[q] / r;
      inv[q] = d[q] != 0.f ? 1.f / d[q] : INFINITY;
    }
    // the target cell's parameter interval (slabs)
    const int cc[3] = {i, j, k};
    float t_in = 0.f, t_out = INFINITY;
    for (int q = 0; q < 3; ++q)
      if (d[q] != 0.f) {
        const float t1 = (cc[q] - a.xs[q]) * inv[q], t2 = (cc[q] + 1 - a.xs[q]) * inv[q];
        t_in = fmaxf(t_in, fminf(t1, t2));
        t_out = fminf(t_out, fmaxf(t1, t2));
      }
    const float dr = t_out - t_in;
    // walk from the source cell to the entry of the target cell: the next
    // crossing of each axis is kept, and only the axis just crossed has its
    // next crossing recomputed (from the source position, not accumulated).
    // The per-axis state is kept in scalars updated by selects (an array
    // indexed by the crossed axis would live in local memory), and the walk,
    // which does not depend on kappa, runs four steps ahead of the sum of
    // tau: their four kappa loads are in flight together, and tau takes them
    // in order (a step past the end or outside the grid adds 0 times 0).
    int c0 = (int)floorf(a.xs[0]), c1 = (int)floorf(a.xs[1]), c2 = (int)floorf(a.xs[2]);
    const int s0 = d[0] > 0.f ? 1 : -1, s1 = d[1] > 0.f ? 1 : -1, s2 = d[2] > 0.f ? 1 : -1;
    const int o0 = d[0] > 0.f ? 1 : 0, o1 = d[1] > 0.f ? 1 : 0, o2 = d[2] > 0.f ? 1 : 0;
    const long long plane = (long long)a.nx * a.ny;
    const long long e0 = s0, e1 = s1 > 0 ? (long long)a.nx : -(long long)a.nx, e2 = s2 > 0 ? plane : -plane;
    float tm0 = d[0] != 0.f ? (c0 + o0 - a.xs[0]) * inv[0] : INFINITY;
    float tm1 = d[1] != 0.f ? (c1 + o1 - a.xs[1]) * inv[1] : INFINITY;
    float tm2 = d[2] != 0.f ? (c2 + o2 - a.xs[2]) * inv[2] : INFINITY;
    long long idx = ((long long)c2 * a.ny + c1) * a.nx + c0;
    float t = 0.f, tau = 0.f;
    for (int s = 0; s < cap && t < t_in - 1e-5f;) {
      float kv[4], len[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool live = s < cap && t < t_in - 1e-5f;
        const int ax = tm0 <= tm1 ? (tm0 <= tm2 ? 0 : 2) : (tm1 <= tm2 ? 1 : 2);
        const float tn = fminf(ax == 0 ? tm0 : (ax == 1 ? tm1 : tm2), t_in);
        const bool in = live && (unsigned)c0 < (unsigned)a.nx && (unsigned)c1 < (unsigned)a.ny &&
                        (unsigned)c2 < (unsigned)a.nz;
        kv[u] = in ? __ldg(kappa + idx) : 0.f;
        len[u] = in ? tn - t : 0.f;
        if (live) {
          t = tn;
          c0 += ax == 0 ? s0 : 0;
          c1 += ax == 1 ? s1 : 0;
          c2 += ax == 2 ? s2 : 0;
          idx += ax == 0 ? e0 : (ax == 1 ? e1 : e2);
          if (ax == 0) tm0 = (c0 + o0 - a.xs[0]) * inv[0];
          if (ax == 1) tm1 = (c1 + o1 - a.xs[1]) * inv[1];
          if (ax == 2) tm2 = (c2 + o2 - a.xs[2]) * inv[2];
          ++s;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) tau = fmaf(kv[u], len[u], tau);
    }
    const float taus = tau * a.h, drl = dr * a.h, rl = r * a.h;
    const float tc = kappa[c] * drl;
    const float E = a.L * expf(-taus) * (-expm1f(-tc)) / (4.f * 3.14159265358979f * rl * rl * drl);
    Edot[c] = E;
    if (pdot) {
      pdot[c] = E * d[0];
      pdot[ncell + c] = E * d[1];
      pdot[2 * ncell + c] = E * d[2];
    }
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

}  // namespace

extern "C" __attribute__((visibility("default"))) vet_status vet_point_source(const vet_grid *grid, const double xs[3],
                                                                                double L, const float *kappa,
                                                                                float *Edot_out, float *pdot_out,
                                                                                void *stream) {
  if (!grid || !xs || !kappa || !Edot_out) return VET_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->h > 0.0) || !std::isfinite(L)) return VET_EINVAL;
  const int n[3] = {grid->nx, grid->ny, grid->nz};
  PointArgs a;
  a.nx = n[0];
  a.ny = n[1];
  a.nz = n[2];
  a.h = (float)grid->h;
  a.L = (float)L;
  for (int q = 0; q < 3; ++q) {
    const double u = xs[q] / grid->h;
    if (!(u >= 0.0 && u < n[q])) return VET_EINVAL;  // the source must lie in the grid
    a.xs[q] = (float)u;
  }
  if (!on_device(kappa) || !on_device(Edot_out) || (pdot_out && !on_device(pdot_out))) return VET_EINVAL;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) {
    cudaGetLastError();
    return VET_ECUDA;
  }
  point_kernel<<<8 * sms, 256, 0, (cudaStream_t)stream>>>(a, kappa, Edot_out, pdot_out);
  return cudaGetLastError() == cudaSuccess ? VET_OK : VET_ECUDA;
}
