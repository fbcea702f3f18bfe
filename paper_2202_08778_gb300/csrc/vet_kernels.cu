// vet_kernels.cu -- sm_103a kernels of the VET closure (VETTAM Sec. 2.2.5).
//
// Two passes replace the paper's on-the-fly ray sweep:
//   face pass  -- block wavefront (one launch per wavefront level): for every
//                 block and direction, the intensity at the (B+1)^2 lattice
//                 points of each of the block's three downwind faces, from
//                 long characteristics back to the block's upwind faces where
//                 the upwind neighbours' face nodes are bilinearly
//                 interpolated (hybrid characteristics);
//   cell pass  -- fully parallel: every cell-centre ray of a block for every
//                 direction, with the quadratures E, F, P (Eqs. 6-8)
//                 accumulated in registers across all directions and
//                 f = P/E (Eq. 9) in the epilogue, so that I is never stored.
// Both passes stage the block's kappa/S tile, the direction's ray template and
// the three incoming faces in shared memory.
#include <cstdint>

#include "vet_internal.h"

namespace vet {

namespace {

template <typename R> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };
template <typename R> using vec2_t = typename Vec2<R>::T;

// exp(-x) and 1 - exp(-x) for the optical depth x >= 0 of one segment, given
// y = -x log2(e) (segment lengths are stored pre-scaled by -h log2(e)).
//   FP32: below x = 1/2 both come from the Taylor series of 1 - exp(-x) cut
//   after x^8 (remainder below x^9/9!, i.e. < 1.4e-8 of the value at 1/2),
//   which is accurate to rounding where 1 - e would cancel and more accurate
//   than the MUFU; above it e comes from the MUFU (ex2.approx) and 1 - e is
//   well conditioned.
//   FP64: the CUDA math library's exp2 and expm1.
__device__ __forceinline__ void attenuation(float y, float &e, float &om) {
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(y));
  const float x = y * -0.6931471805599453f;
  float p = -2.48015873015873e-05f;             // -1/8!
  p = fmaf(p, x, 1.984126984126984e-04f);       //  1/7!
  p = fmaf(p, x, -1.388888888888889e-03f);      // -1/6!
  p = fmaf(p, x, 8.333333333333333e-03f);       //  1/5!
  p = fmaf(p, x, -4.166666666666667e-02f);      // -1/4!
  p = fmaf(p, x, 1.666666666666667e-01f);       //  1/3!
  p = fmaf(p, x, -0.5f);                        // -1/2!
  p = fmaf(p, x, 1.0f);
  p *= x;
  const bool thin = x < 0.5f;
  om = thin ? p : 1.0f - e;
  e = thin ? 1.0f - p : e;
}

__device__ __forceinline__ void attenuation(double y, double &e, double &om) {
  e = exp2(y);
  om = -expm1(y * 0.6931471805599453094);
}

// Exact update over piecewise-constant cells, marching backward from the
// ray's start: after the loop, I(start) = acc + T * I(entry point).
template <typename R>
__device__ __forceinline__ void march(const vec2_t<R> *__restrict__ tile, int idx, int last,
                                      const R *__restrict__ len, const int16_t *__restrict__ delta, R &acc,
                                      R &T) {
  acc = R(0);
  T = R(1);
  for (int e = 0; e <= last; ++e) {
    const vec2_t<R> ks = tile[idx];
    R ex, om;
    attenuation(ks.x * len[e], ex, om);
    acc = fma(ks.y * om, T, acc);
    T *= ex;
    idx += delta[e];
  }
}

// Typed view of one direction's template blob.
template <typename R>
struct Tpl {
  const TplHead<R> *h;
  const R *clen, *nlen;
  const int16_t *cdlt, *ndlt, *cpos, *npos, *ck, *nk;
  const vec2_t<R> *cw, *nw;
  __device__ __forceinline__ Tpl(const unsigned char *base, const TplLayout &L)
      : h(reinterpret_cast<const TplHead<R> *>(base)),
        clen(reinterpret_cast<const R *>(base + L.clen)),
        nlen(reinterpret_cast<const R *>(base + L.nlen)),
        cdlt(reinterpret_cast<const int16_t *>(base + L.cdlt)),
        ndlt(reinterpret_cast<const int16_t *>(base + L.ndlt)),
        cpos(reinterpret_cast<const int16_t *>(base + L.cpos)),
        npos(reinterpret_cast<const int16_t *>(base + L.npos)),
        ck(reinterpret_cast<const int16_t *>(base + L.ck)),
        nk(reinterpret_cast<const int16_t *>(base + L.nk)),
        cw(reinterpret_cast<const vec2_t<R> *>(base + L.cw)),
        nw(reinterpret_cast<const vec2_t<R> *>(base + L.nw)) {}
};

// Memory-frame face-node indices and weights along one in-plane axis, from
// the upwind-frame lower node iup and its weights (f on iup + 1, g = 1 - f on
// iup).  Exact ties may put the exit point a rounding error outside the face;
// it is then clamped onto the face edge.
template <typename R>
__device__ __forceinline__ void axis_nodes(int iup, R f, R g, int sgn, int B, int &m0, int &m1, R &w0, R &w1) {
  if (iup < 0) {
    iup = 0; f = R(0); g = R(1);
  } else if (iup > B - 1) {
    iup = B - 1; f = R(1); g = R(0);
  }
  m0 = sgn > 0 ? iup : B - iup;
  m1 = sgn > 0 ? iup + 1 : B - iup - 1;
  w0 = g;
  w1 = f;
}

// Bilinear interpolation on incoming face ae (Sec. 2.2.5 reading: short
// characteristics between blocks).  l[] are the ray's upwind-frame
// coordinates, k/w its exit-table rows for the two in-plane axes.
template <typename R>
__device__ __forceinline__ R face_value(const R *__restrict__ fin, int nnode, int B, int ae, const int *sgn,
                                        int lb, int lc, int kb, int kc, vec2_t<R> wb, vec2_t<R> wc) {
  const int b = ae == 0 ? 1 : 0, c = ae == 2 ? 1 : 2;
  int ub0, ub1, vc0, vc1;
  R gb0, gb1, gc0, gc1;
  axis_nodes<R>(lb + kb, wb.x, wb.y, sgn[b], B, ub0, ub1, gb0, gb1);
  axis_nodes<R>(lc + kc, wc.x, wc.y, sgn[c], B, vc0, vc1, gc0, gc1);
  const R *F = fin + ae * nnode;
  const int W = B + 1;
  return gb0 * gc0 * F[ub0 * W + vc0] + gb1 * gc0 * F[ub1 * W + vc0] + gb0 * gc1 * F[ub0 * W + vc1] +
         gb1 * gc1 * F[ub1 * W + vc1];
}

// Copy a direction template into shared memory (16-byte words).
__device__ __forceinline__ void load_template(unsigned char *dst, const unsigned char *src, int bytes) {
  const int4 *s = reinterpret_cast<const int4 *>(src);
  int4 *d = reinterpret_cast<int4 *>(dst);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
}

// The three faces entering block (bx, by, bz) for internal direction d:
// upwind neighbours' outgoing face nodes, or the constant boundary value.
template <typename R>
__device__ __forceinline__ void load_incoming(R *fin, const GridDims &g, int bx, int by, int bz, int d,
                                              const TplHead<R> *__restrict__ hd, const R *__restrict__ faces,
                                              const R *__restrict__ Ib) {
  const int nblk = g.nbx * g.nby * g.nbz;
  const int b3[3] = {bx, by, bz};
  const int nb3[3] = {g.nbx, g.nby, g.nbz};
  const int ext = hd->ext;
  for (int a = 0; a < 3; ++a) {
    const int s = hd->sgn[a];
    int nb[3] = {b3[0], b3[1], b3[2]};
    nb[a] -= s;
    R *dst = fin + a * g.nnode;
    if (nb[a] < 0 || nb[a] >= nb3[a]) {
      const int face = 2 * a + (s > 0 ? 0 : 1);
      const R v = Ib ? Ib[(long long)face * g.ndir + ext] : R(0);
      for (int i = threadIdx.x; i < g.nnode; i += blockDim.x) dst[i] = v;
    } else {
      const long long nid = ((long long)nb[2] * g.nby + nb[1]) * g.nbx + nb[0];
      const R *src = faces + (((long long)d * nblk + nid) * 3 + a) * g.nnode;
      for (int i = threadIdx.x; i < g.nnode; i += blockDim.x) dst[i] = src[i];
    }
  }
}

template <typename R>
__device__ __forceinline__ void load_tile(vec2_t<R> *tile, const GridDims &g, int bx, int by, int bz,
                                          const R *__restrict__ kappa, const R *__restrict__ S) {
  const int B = g.B, B2 = B * B, B3 = B2 * B;
  for (int i = threadIdx.x; i < B3; i += blockDim.x) {
    const int x = i % B, y = (i / B) % B, z = i / B2;
    const long long gi = ((long long)(bz * B + z) * g.ny + (by * B + y)) * g.nx + (bx * B + x);
    vec2_t<R> v;
    v.x = kappa[gi];
    v.y = S[gi];
    tile[i] = v;
  }
}

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename R>
__host__ __device__ inline size_t smem_bytes(int B, int nnode) {
  return align16(sizeof(vec2_t<R>) * (size_t)B * B * B) + align16(sizeof(R) * 3 * (size_t)nnode) +
         (size_t)tpl_layout<R>(B).bytes;
}

// ---------------------------------------------------------------- face pass
template <typename R>
__global__ void __launch_bounds__(256) face_pass_kernel(GridDims g, const R *__restrict__ kappa,
                                                        const R *__restrict__ S, const R *__restrict__ Ib,
                                                        const unsigned char *__restrict__ tpl_g,
                                                        const FaceItem *__restrict__ items, R *__restrict__ faces) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int B = g.B;
  const TplLayout TL = tpl_layout<R>(B);
  vec2_t<R> *tile = reinterpret_cast<vec2_t<R> *>(smem);
  R *fin = reinterpret_cast<R *>(smem + align16(sizeof(vec2_t<R>) * (size_t)B * B * B));
  unsigned char *tb = reinterpret_cast<unsigned char *>(fin) + align16(sizeof(R) * 3 * (size_t)g.nnode);
  const Tpl<R> T(tb, TL);
  const FaceItem it = items[blockIdx.x];
  const int bx = it.block % g.nbx, by = (it.block / g.nbx) % g.nby, bz = it.block / (g.nbx * g.nby);
  const int nblk = g.nbx * g.nby * g.nbz;
  load_tile<R>(tile, g, bx, by, bz, kappa, S);
  const int nn3 = 3 * g.nnode;
  for (int d = it.dir_begin; d < it.dir_begin + it.dir_count; ++d) {
    __syncthreads();
    load_template(tb, tpl_g + (size_t)d * TL.bytes, TL.bytes);
    load_incoming<R>(fin, g, bx, by, bz, d, reinterpret_cast<const TplHead<R> *>(tpl_g + (size_t)d * TL.bytes),
                     faces, Ib);
    __syncthreads();
    const int sgn[3] = {T.h->sgn[0], T.h->sgn[1], T.h->sgn[2]};
    R *out = faces + ((long long)d * nblk + it.block) * 3 * g.nnode;
    for (int j = threadIdx.x; j < nn3; j += blockDim.x) {
      const int a = j / g.nnode, r = j - a * g.nnode;
      const int u = r / (B + 1), v = r - u * (B + 1);
      const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
      int P[3];
      P[a] = sgn[a] > 0 ? B : 0;  // memory-frame node position
      P[b] = u;
      P[c] = v;
      int L[3], cell[3];
      for (int q = 0; q < 3; ++q) {
        L[q] = sgn[q] > 0 ? P[q] : B - P[q];        // upwind-frame position
        cell[q] = sgn[q] > 0 ? L[q] - 1 : B - L[q];  // memory-frame start cell
      }
      int last = T.npos[L[0]], ae = 0;
      if (T.npos[(B + 1) + L[1]] < last) { last = T.npos[(B + 1) + L[1]]; ae = 1; }
      if (T.npos[2 * (B + 1) + L[2]] < last) { last = T.npos[2 * (B + 1) + L[2]]; ae = 2; }
      R acc = R(0), Tr = R(1);
      if (last >= 0) march<R>(tile, cell[0] + B * (cell[1] + B * cell[2]), last, T.nlen, T.ndlt, acc, Tr);
      const int eb = ae == 0 ? 1 : 0, ec = ae == 2 ? 1 : 2;
      const int row = (ae * 2) * (B + 1) + L[ae];
      const R Iin = face_value<R>(fin, g.nnode, B, ae, sgn, L[eb], L[ec], T.nk[row], T.nk[row + (B + 1)],
                                  T.nw[row], T.nw[row + (B + 1)]);
      out[j] = fma(Tr, Iin, acc);
    }
  }
}

// ---------------------------------------------------------------- cell pass
constexpr int kCPT = 2;  // cells per thread

__device__ __forceinline__ void atomic_max_nonneg(void *p, float v) {
  atomicMax(reinterpret_cast<unsigned int *>(p), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(void *p, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double_as_longlong(v));
}

template <typename R, int MODE>
__global__ void __launch_bounds__(512) cell_pass_kernel(GridDims g, int parts, const R *__restrict__ kappa,
                                                        const R *__restrict__ S, const R *__restrict__ Ib,
                                                        const unsigned char *__restrict__ tpl_g,
                                                        const R *__restrict__ faces, R *__restrict__ I_out,
                                                        R *__restrict__ M_out, R *__restrict__ E_out,
                                                        R *__restrict__ f_out, void *emax_bits) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int B = g.B, B2 = B * B, B3 = B2 * B;
  const TplLayout TL = tpl_layout<R>(B);
  vec2_t<R> *tile = reinterpret_cast<vec2_t<R> *>(smem);
  R *fin = reinterpret_cast<R *>(smem + align16(sizeof(vec2_t<R>) * (size_t)B3));
  unsigned char *tb = reinterpret_cast<unsigned char *>(fin) + align16(sizeof(R) * 3 * (size_t)g.nnode);
  const Tpl<R> T(tb, TL);
  const int blk = blockIdx.x / parts, part = blockIdx.x - blk * parts;
  const int bx = blk % g.nbx, by = (blk / g.nbx) % g.nby, bz = blk / (g.nbx * g.nby);
  const int cpc = B3 / parts;  // cells of this CTA
  load_tile<R>(tile, g, bx, by, bz, kappa, S);

  int lc[kCPT];        // local cell index in the block, or -1
  long long gc[kCPT];  // global cell index
  for (int i = 0; i < kCPT; ++i) {
    const int k = threadIdx.x + i * blockDim.x;
    lc[i] = k < cpc ? part * cpc + k : -1;
    const int c = lc[i] < 0 ? 0 : lc[i];
    const int x = c % B, y = (c / B) % B, z = c / B2;
    gc[i] = ((long long)(bz * B + z) * g.ny + (by * B + y)) * g.nx + (bx * B + x);
  }
  // Moments accumulated over all directions.  E, Pxx, Pyy and Pzz (sums of
  // positive terms that f_ii = P_ii / E depends on) carry a Kahan
  // compensation term: plain sequential FP32 sums of N terms lose about
  // N/2 ulp, which would dominate the error of f.
  R mom[MODE == 0 ? kCPT : 1][10];
  R cmp[MODE == 0 ? kCPT : 1][4];
  if (MODE == 0) {
    for (int i = 0; i < kCPT; ++i) {
      for (int m = 0; m < 10; ++m) mom[i][m] = R(0);
      for (int m = 0; m < 4; ++m) cmp[i][m] = R(0);
    }
  }

  for (int d = 0; d < g.ndir; ++d) {
    __syncthreads();
    load_template(tb, tpl_g + (size_t)d * TL.bytes, TL.bytes);
    load_incoming<R>(fin, g, bx, by, bz, d, reinterpret_cast<const TplHead<R> *>(tpl_g + (size_t)d * TL.bytes),
                     faces, Ib);
    __syncthreads();
    const int sgn[3] = {T.h->sgn[0], T.h->sgn[1], T.h->sgn[2]};
    R coef[10];  // w (1, n, n n) of this direction
    {
      const R w = T.h->w, nx = T.h->n[0], ny = T.h->n[1], nz = T.h->n[2];
      coef[0] = w; coef[1] = w * nx; coef[2] = w * ny; coef[3] = w * nz;
      coef[4] = coef[1] * nx; coef[5] = coef[2] * ny; coef[6] = coef[3] * nz;
      coef[7] = coef[1] * ny; coef[8] = coef[1] * nz; coef[9] = coef[2] * nz;
    }
#pragma unroll
    for (int i = 0; i < kCPT; ++i) {
      if (lc[i] < 0) continue;
      const int c = lc[i];
      const int x = c % B, y = (c / B) % B, z = c / B2;
      int l[3];
      l[0] = sgn[0] > 0 ? x : B - 1 - x;
      l[1] = sgn[1] > 0 ? y : B - 1 - y;
      l[2] = sgn[2] > 0 ? z : B - 1 - z;
      int last = T.cpos[l[0]], ae = 0;
      if (T.cpos[B + l[1]] < last) { last = T.cpos[B + l[1]]; ae = 1; }
      if (T.cpos[2 * B + l[2]] < last) { last = T.cpos[2 * B + l[2]]; ae = 2; }
      R acc, Tr;
      march<R>(tile, c, last, T.clen, T.cdlt, acc, Tr);
      const int eb = ae == 0 ? 1 : 0, ec = ae == 2 ? 1 : 2;
      const int row = (ae * 2) * B + l[ae];
      const R Iin = face_value<R>(fin, g.nnode, B, ae, sgn, l[eb], l[ec], T.ck[row], T.ck[row + B], T.cw[row],
                                  T.cw[row + B]);
      const R I = fma(Tr, Iin, acc);
      if (MODE == 1) {
        I_out[(long long)T.h->ext * g.ncell + gc[i]] = I;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // E, Pxx, Pyy, Pzz: compensated
          const int m = q == 0 ? 0 : 3 + q;
          const R y = I * coef[m] - cmp[i][q];
          const R t = mom[i][m] + y;
          cmp[i][q] = (t - mom[i][m]) - y;
          mom[i][m] = t;
        }
        mom[i][1] = fma(I, coef[1], mom[i][1]);
        mom[i][2] = fma(I, coef[2], mom[i][2]);
        mom[i][3] = fma(I, coef[3], mom[i][3]);
        mom[i][7] = fma(I, coef[7], mom[i][7]);
        mom[i][8] = fma(I, coef[8], mom[i][8]);
        mom[i][9] = fma(I, coef[9], mom[i][9]);
      }
    }
  }
  if (MODE == 0) {
    R emax = R(0);
    for (int i = 0; i < kCPT; ++i) {
      if (lc[i] < 0) continue;
      const long long c = gc[i];
      const R E = mom[i][0];
      if (M_out) {
        for (int m = 0; m < 10; ++m) M_out[m * g.ncell + c] = mom[i][m];
      } else {
        E_out[c] = E;
      }
      if (E > R(0)) {
        const R inv = R(1) / E;
        for (int m = 0; m < 6; ++m) f_out[m * g.ncell + c] = mom[i][4 + m] * inv;
      } else {
        for (int m = 0; m < 6; ++m) f_out[m * g.ncell + c] = m < 3 ? R(1) / R(3) : R(0);
      }
      emax = E > emax ? E : emax;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const R v = __shfl_xor_sync(0xffffffffu, emax, o);
      emax = v > emax ? v : emax;
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(emax_bits, emax);
  }
}

template <typename R> __device__ __forceinline__ R load_max(const void *p);
template <> __device__ __forceinline__ float load_max<float>(const void *p) {
  return __uint_as_float(*reinterpret_cast<const unsigned int *>(p));
}
template <> __device__ __forceinline__ double load_max<double>(const void *p) {
  return __longlong_as_double((long long)*reinterpret_cast<const unsigned long long *>(p));
}

// Cells whose E does not exceed floor_rel * max E get f = I/3.
template <typename R>
__global__ void floor_fix_kernel(long long ncell, const R *__restrict__ E, const void *__restrict__ emax_bits,
                                 double floor_rel, R *__restrict__ f) {
  const R floor = R(floor_rel) * load_max<R>(emax_bits);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    if (!(E[c] > floor)) {
      for (int m = 0; m < 6; ++m) f[m * ncell + c] = m < 3 ? R(1) / R(3) : R(0);
    }
  }
}

// M[m][c] = sum_k I[k][c] coef[k][m] with coef[k] = w_k (1, n, n n).
template <typename R>
__global__ void __launch_bounds__(256) moments_kernel(long long ncell, int ndir, const R *__restrict__ I,
                                                      const R *__restrict__ coef, R *__restrict__ M) {
  __shared__ R cs[64][10];
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  R acc[10];
  for (int m = 0; m < 10; ++m) acc[m] = R(0);
  for (int k0 = 0; k0 < ndir; k0 += 64) {
    const int nk = min(64, ndir - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < nk * 10; i += blockDim.x) cs[i / 10][i % 10] = coef[(long long)k0 * 10 + i];
    __syncthreads();
    if (c < ncell) {
      for (int k = 0; k < nk; ++k) {
        const R v = I[(long long)(k0 + k) * ncell + c];
        for (int m = 0; m < 10; ++m) acc[m] = fma(v, cs[k][m], acc[m]);
      }
    }
  }
  if (c < ncell)
    for (int m = 0; m < 10; ++m) M[m * ncell + c] = acc[m];
}

}  // namespace

static int cell_parts(int B) {
  const int B3 = B * B * B;
  int parts = (B3 + 1023) / 1024;
  while (B3 % parts) ++parts;
  return parts;
}

template <typename R>
cudaError_t launch_face_level(const GridDims &g, const R *kappa, const R *S, const R *Ib,
                              const unsigned char *tpl, const FaceItem *items, int nitems, R *faces,
                              cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const size_t sm = smem_bytes<R>(g.B, g.nnode);
  face_pass_kernel<R><<<nitems, 256, sm, st>>>(g, kappa, S, Ib, tpl, items, faces);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cell_pass(const GridDims &g, int mode, const R *kappa, const R *S, const R *Ib,
                             const unsigned char *tpl, const R *faces, R *I_out, R *M_out, R *E_out,
                             R *f_out, void *emax_bits, cudaStream_t st) {
  const int parts = cell_parts(g.B);
  const int cpc = g.B * g.B * g.B / parts;
  int threads = (cpc + kCPT - 1) / kCPT;
  threads = (threads + 31) / 32 * 32;
  const int nblk = g.nbx * g.nby * g.nbz;
  const size_t sm = smem_bytes<R>(g.B, g.nnode);
  if (mode == 0) {
    cell_pass_kernel<R, 0><<<nblk * parts, threads, sm, st>>>(g, parts, kappa, S, Ib, tpl, faces, I_out, M_out,
                                                               E_out, f_out, emax_bits);
  } else {
    cell_pass_kernel<R, 1><<<nblk * parts, threads, sm, st>>>(g, parts, kappa, S, Ib, tpl, faces, I_out, M_out,
                                                               E_out, f_out, emax_bits);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_floor_fix(long long ncell, const R *E, long long, const void *emax_bits, double floor_rel,
                             R *f_out, cudaStream_t st) {
  const int threads = 256;
  long long blocks = (ncell + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  floor_fix_kernel<R><<<(int)blocks, threads, 0, st>>>(ncell, E, emax_bits, floor_rel, f_out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_moments(long long ncell, int ndir, const R *I, const R *coef, R *M_out, cudaStream_t st) {
  const int threads = 256;
  const long long blocks = (ncell + threads - 1) / threads;
  if (blocks < 1) return cudaSuccess;
  moments_kernel<R><<<(unsigned)blocks, threads, 0, st>>>(ncell, ndir, I, coef, M_out);
  return cudaGetLastError();
}

size_t pass_smem_bytes(int B, int nnode, bool fp64) {
  return fp64 ? smem_bytes<double>(B, nnode) : smem_bytes<float>(B, nnode);
}

// Opt the shared-memory-heavy kernels in to the full 227 KB per CTA on the
// current device (the attribute is per device and function).
cudaError_t prepare_kernels() {
  const int lim = 232448;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(face_pass_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(face_pass_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(cell_pass_kernel<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(cell_pass_kernel<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(cell_pass_kernel<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(cell_pass_kernel<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

#define VET_INSTANTIATE(R)                                                                                      \
  template cudaError_t launch_face_level<R>(const GridDims &, const R *, const R *, const R *,                \
                                            const unsigned char *, const FaceItem *, int, R *, cudaStream_t); \
  template cudaError_t launch_cell_pass<R>(const GridDims &, int, const R *, const R *, const R *,            \
                                           const unsigned char *, const R *, R *, R *, R *, R *, void *,        \
                                           cudaStream_t);                                                       \
  template cudaError_t launch_floor_fix<R>(long long, const R *, long long, const void *, double, R *,        \
                                           cudaStream_t);                                                       \
  template cudaError_t launch_moments<R>(long long, int, const R *, const R *, R *, cudaStream_t);

VET_INSTANTIATE(float)
VET_INSTANTIATE(double)

}  // namespace vet
