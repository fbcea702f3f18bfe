// vet_cnn.cu -- kernels of the learned closure (not in the VETTAM paper: a
// 3D convolutional network predicting the Eddington tensor from local
// features, with the exact ray tracer as fallback): features, the weight
// gradient of the convolutions, head and loss, AdamW, indicator and block
// list.  The convolutions themselves (forward and data gradient) run on the
// tcgen05 tensor cores (vet_cnn_tc.cu).
//
// Activations are stored cells-major, channels-minor ([volume][z][y][x][C],
// BF16, C a multiple of 16).  The weight gradient is, per tap, a GEMM with
// M = output channels, N = input channels and K = the 256 cells of an
// 8 x 8 x 4 tile, on BF16 mma.sync (m16n8k16, FP32 accumulate) with
// ldmatrix.trans operands from shared memory whose rows are XOR-swizzled in
// 16-byte chunks (every ldmatrix phase touches 8 distinct bank groups).
#include <cstdint>

#include <cuda_bf16.h>

#include "vet_cnn.h"

namespace vet {
namespace cnn {
namespace {

constexpr int TX = 8, TY = 8, TZ = 4;      // output tile
constexpr int HX = 10, HY = 10, HZ = 6;    // input halo
constexpr int HN = HX * HY * HZ;           // 600 halo cells
constexpr int TN = TX * TY * TZ;           // 256 tile cells
constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of 16-byte chunk c of row `row` in a swizzled array whose rows
// hold `nch` chunks (C/8 BF16 values each).
__device__ __forceinline__ int swz_off(int row, int c, int nch) {
  const int s = nch == 4 ? (c ^ ((row >> 1) & 3)) : (nch == 2 ? (c ^ ((row >> 2) & 1)) : c);
  return row * nch * 16 + s * 16;
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}


struct TileIdx {
  int v, tz, ty, tx;
};

__device__ __forceinline__ TileIdx tile_of(long long t, const Vol &V) {
  const int ntx = (V.nx + TX - 1) / TX, nty = (V.ny + TY - 1) / TY, ntz = (V.nz + TZ - 1) / TZ;
  TileIdx r;
  r.tx = (int)(t % ntx);
  t /= ntx;
  r.ty = (int)(t % nty);
  t /= nty;
  r.tz = (int)(t % ntz);
  r.v = (int)(t / ntz);
  return r;
}

__device__ __forceinline__ long long ntiles_of(const Vol &V) {
  return (long long)V.n * ((V.nz + TZ - 1) / TZ) * ((V.ny + TY - 1) / TY) * ((V.nx + TX - 1) / TX);
}

// Stage the 10 x 10 x 6 halo of tile `ti` of x (C channels) into smem;
// cells outside the volume are zero (zero padding).
template <int C>
__device__ __forceinline__ void load_halo(unsigned char *sm, const __nv_bfloat16 *__restrict__ x, const Vol &V,
                                          const TileIdx &ti) {
  constexpr int NCH = C / 8;
  const long long vol = (long long)V.nz * V.ny * V.nx;
  for (int h = threadIdx.x; h < HN * NCH; h += blockDim.x) {
    const int hc = h / NCH, c = h - hc * NCH;
    const int hz = hc / (HX * HY), hy = (hc / HX) % HY, hx = hc % HX;
    const int z = ti.tz * TZ + hz - 1, y = ti.ty * TY + hy - 1, xx = ti.tx * TX + hx - 1;
    int4 val = make_int4(0, 0, 0, 0);
    if (z >= 0 && z < V.nz && y >= 0 && y < V.ny && xx >= 0 && xx < V.nx) {
      const long long cell = (long long)ti.v * vol + ((long long)z * V.ny + y) * V.nx + xx;
      val = reinterpret_cast<const int4 *>(x + cell * C)[c];
    }
    *reinterpret_cast<int4 *>(sm + swz_off(hc, c, NCH)) = val;
  }
}

// ---------------------------------------------------------- weight gradient
// gW[tap][co][ci] += sum_cells gpre[cell][co] * x[cell + tap][ci];
// gb[co] += sum_cells gpre[cell][co].  A GEMM per tap with M = C_OUT,
// N = C_IN and K = the 256 cells of a tile; warp w owns taps w, w + 8, ...
// and folds each tile's products into a shared FP32 accumulator (no other
// warp writes those rows), flushed to global memory with atomics once per
// CTA.  Accumulator rows are float2 pairs of input channels, the pair index
// XOR-swizzled by the output channel so that a warp's fold is 2-way at most.
template <int C_IN>
__device__ __forceinline__ int acc_pair(int co, int p) {
  return C_IN == 32 ? (p ^ ((co & 3) << 2)) : (p ^ (((co >> 1) & 1) << 2));
}

template <int C_IN, int C_OUT>
__global__ void __launch_bounds__(kThreads, 1)
    wgrad_kernel(const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ gpre, Vol V,
                 float *__restrict__ gW, float *__restrict__ gb) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NCI = C_IN / 8, NCO = C_OUT / 8, MT = C_OUT / 16, NT = C_IN / 8, NP = C_IN / 2;
  float2 *sAcc = reinterpret_cast<float2 *>(smem);             // [27][C_OUT][NP]
  unsigned char *sX = smem + 27 * C_OUT * C_IN * 4;             // 600 halo rows of C_IN
  unsigned char *sG = sX + HN * C_IN * 2;                       // 256 tile rows of C_OUT
  for (int i = threadIdx.x; i < 27 * C_OUT * NP; i += blockDim.x) sAcc[i] = make_float2(0.f, 0.f);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t4 = lane & 3, q = lane >> 3, r8 = lane & 7;
  constexpr int BSL = kThreads / C_OUT;  // bias: thread owns channel tid % C_OUT, cells tid / C_OUT + BSL j
  const int bco = threadIdx.x % C_OUT, bks = threadIdx.x / C_OUT;
  float bacc = 0.f;
  const long long vol = (long long)V.nz * V.ny * V.nx;
  const long long nt = ntiles_of(V);
  for (long long tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const TileIdx ti = tile_of(tile, V);
    __syncthreads();
    load_halo<C_IN>(sX, x, V, ti);
    for (int h = threadIdx.x; h < TN * NCO; h += blockDim.x) {
      const int k = h / NCO, c = h - k * NCO;
      const int z = ti.tz * TZ + (k >> 6), y = ti.ty * TY + ((k >> 3) & 7), xx = ti.tx * TX + (k & 7);
      int4 val = make_int4(0, 0, 0, 0);
      if (z < V.nz && y < V.ny && xx < V.nx) {
        const long long cell = (long long)ti.v * vol + ((long long)z * V.ny + y) * V.nx + xx;
        val = reinterpret_cast<const int4 *>(gpre + cell * C_OUT)[c];
      }
      *reinterpret_cast<int4 *>(sG + swz_off(k, c, NCO)) = val;
    }
    __syncthreads();
    for (int k = bks; k < TN; k += BSL)
      bacc += __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(sG + swz_off(k, bco >> 3, NCO) + (bco & 7) * 2));
    for (int tap = warp; tap < 27; tap += kThreads / 32) {
      const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
      float acc[MT][NT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[mt][j][e] = 0.f;
      for (int ks = 0; ks < TN / 16; ++ks) {
        uint32_t a[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          // A = gpre^T: rows co, k = cells; stored [cell][co] -> transposed load
          const int k = 16 * ks + r8 + 8 * (q >> 1);
          ldsm_x4_t(smem_u32(sG + swz_off(k, 2 * mt + (q & 1), NCO)), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
        }
#pragma unroll
        for (int j = 0; j < NT; j += 2) {
          // B = shifted input: k = cells, n = ci; stored [halo cell][ci]
          const int k = 16 * ks + r8 + 8 * (q & 1);
          const int hc = ((k >> 6) + 1 + dz) * (HX * HY) + (((k >> 3) & 7) + 1 + dy) * HX + ((k & 7) + 1 + dx);
          uint32_t b0, b1, b2, b3;
          ldsm_x4_t(smem_u32(sX + swz_off(hc, j + (q >> 1), NCI)), b0, b1, b2, b3);
#pragma unroll
          for (int mt = 0; mt < MT; ++mt) {
            mma_bf16(acc[mt][j], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
            mma_bf16(acc[mt][j + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
          }
        }
      }
      float2 *row = sAcc + (size_t)tap * C_OUT * NP;
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int co = 16 * mt + g + 8 * half, p = 4 * j + t4;
            float2 &s = row[co * NP + acc_pair<C_IN>(co, p)];
            s.x += acc[mt][j][2 * half];
            s.y += acc[mt][j][2 * half + 1];
          }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 27 * C_OUT * NP; i += blockDim.x) {
    const int tap = i / (C_OUT * NP), rem = i - tap * C_OUT * NP, co = rem / NP, p = rem - co * NP;
    const float2 s = sAcc[(size_t)tap * C_OUT * NP + co * NP + acc_pair<C_IN>(co, p)];
    float *dst = gW + ((long long)tap * C_OUT + co) * C_IN + 2 * p;
    atomicAdd(dst, s.x);
    atomicAdd(dst + 1, s.y);
  }
  atomicAdd(gb + bco, bacc);
}

// ---------------------------------------------------------------- features
// Per (volume, block) CTA: mean and standard deviation (population) of
// tau = log10(kappa h) over the block, and the volume sums of log10 S and
// log10 E (FP64 atomics).
constexpr float kTiny = 1e-30f;

__device__ __forceinline__ double block_sum_d(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(256) feat_stats_kernel(const float *__restrict__ kappa, const float *__restrict__ S,
                                                         const float *__restrict__ E, Vol V, int B, float h,
                                                         double *__restrict__ sums, float *__restrict__ bstat) {
  __shared__ double red[8];
  const int nbx = V.nx / B, nby = V.ny / B, nbz = V.nz / B;
  const int blk = blockIdx.x, v = blockIdx.y;
  const int bx = blk % nbx, by = (blk / nbx) % nby, bz = blk / (nbx * nby);
  const long long vol = (long long)V.nz * V.ny * V.nx;
  const int B3 = B * B * B;
  double st = 0.0, st2 = 0.0, ss = 0.0, se = 0.0;
  for (int i = threadIdx.x; i < B3; i += blockDim.x) {
    const int x = bx * B + i % B, y = by * B + (i / B) % B, z = bz * B + i / (B * B);
    const long long c = (long long)v * vol + ((long long)z * V.ny + y) * V.nx + x;
    const double tau = log10f(fmaxf(kappa[c] * h, kTiny));
    st += tau;
    st2 += tau * tau;
    ss += log10f(fmaxf(S[c], kTiny));
    se += log10f(fmaxf(E[c], kTiny));
  }
  st = block_sum_d(st, red);
  st2 = block_sum_d(st2, red);
  ss = block_sum_d(ss, red);
  se = block_sum_d(se, red);
  if (threadIdx.x == 0) {
    const double mean = st / B3, var = fmax(st2 / B3 - mean * mean, 0.0);
    bstat[((long long)v * nbx * nby * nbz + blk) * 2] = (float)mean;
    bstat[((long long)v * nbx * nby * nbz + blk) * 2 + 1] = (float)sqrt(var);
    atomicAdd(sums + 2 * v, ss);
    atomicAdd(sums + 2 * v + 1, se);
  }
}

__global__ void __launch_bounds__(256) feat_pack_kernel(const float *__restrict__ kappa, const float *__restrict__ S,
                                                        const float *__restrict__ E, Vol V, int B, float h,
                                                        const double *__restrict__ sums,
                                                        const float *__restrict__ bstat, __nv_bfloat16 *__restrict__ x0,
                                                        float *__restrict__ feat_out) {
  const long long vol = (long long)V.nz * V.ny * V.nx, n = vol * V.n;
  const int nbx = V.nx / B, nby = V.ny / B, nbz = V.nz / B;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(c / vol);
    const long long l = c - v * vol;
    const int x = (int)(l % V.nx), y = (int)((l / V.nx) % V.ny), z = (int)(l / ((long long)V.nx * V.ny));
    const int blk = (x / B) + nbx * ((y / B) + nby * (z / B));
    const float *bs = bstat + ((long long)v * nbx * nby * nbz + blk) * 2;
    float f[kIn];
    f[0] = 1.f;
    f[1] = log10f(fmaxf(kappa[c] * h, kTiny));
    f[2] = (float)((double)log10f(fmaxf(S[c], kTiny)) - sums[2 * v] / vol);
    f[3] = (float)((double)log10f(fmaxf(E[c], kTiny)) - sums[2 * v + 1] / vol);
    f[4] = bs[0];
    f[5] = bs[1];
    __align__(16) __nv_bfloat162 row[kInPad / 2];
#pragma unroll
    for (int i = 0; i < kInPad / 2; ++i) row[i] = __floats2bfloat162_rn(0.f, 0.f);
    row[0] = __floats2bfloat162_rn(f[0], f[1]);
    row[1] = __floats2bfloat162_rn(f[2], f[3]);
    row[2] = __floats2bfloat162_rn(f[4], f[5]);
    int4 *dst = reinterpret_cast<int4 *>(x0 + c * kInPad);
    dst[0] = reinterpret_cast<const int4 *>(row)[0];
    dst[1] = reinterpret_cast<const int4 *>(row)[1];
    if (feat_out)
      for (int i = 0; i < kIn; ++i) feat_out[((long long)v * kIn + i) * vol + l] = f[i];
  }
}

// ------------------------------------------------------------- head / loss
// f_ii = 1/3 + D_ii - tr(D)/3, f_ij = D_ij; the error target
// log(max |f - f_ref| + 1e-4) is a constant of the gradient.
constexpr float kErrEps = 1e-4f;

__device__ __forceinline__ void head_f(const float *o, float *f) {
  const float tr = (o[0] + o[1] + o[2]) * (1.f / 3.f);
  f[0] = 1.f / 3.f + o[0] - tr;
  f[1] = 1.f / 3.f + o[1] - tr;
  f[2] = 1.f / 3.f + o[2] - tr;
  f[3] = o[3];
  f[4] = o[4];
  f[5] = o[5];
}

__global__ void __launch_bounds__(256) count_kernel(const unsigned char *__restrict__ mask, long long n,
                                                    unsigned long long *count) {
  unsigned long long k = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    k += mask ? (mask[c] != 0) : 1;
  for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  if ((threadIdx.x & 31) == 0 && k) atomicAdd(count, k);
}

__global__ void __launch_bounds__(256) head_loss_kernel(const float *__restrict__ o, const float *__restrict__ f_ref,
                                                        const unsigned char *__restrict__ mask, Vol V, float lam,
                                                        const unsigned long long *__restrict__ count,
                                                        double *__restrict__ loss, __nv_bfloat16 *__restrict__ go) {
  __shared__ double red[8];
  const long long vol = (long long)V.nz * V.ny * V.nx, n = vol * V.n;
  const unsigned long long cnt = *count;
  const float inv_n = cnt ? (float)(1.0 / (double)cnt) : 0.f;
  double part = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(c / vol);
    const long long l = c - v * vol;
    float ov[8];
    const float4 *src = reinterpret_cast<const float4 *>(o + c * kOutPad);
    const float4 a = src[0], b = src[1];
    ov[0] = a.x; ov[1] = a.y; ov[2] = a.z; ov[3] = a.w;
    ov[4] = b.x; ov[5] = b.y; ov[6] = b.z; ov[7] = b.w;
    float f[6], d[6];
    head_f(ov, f);
    float mx = 0.f, sq = 0.f;
    for (int i = 0; i < 6; ++i) {
      d[i] = f[i] - f_ref[((long long)v * 6 + i) * vol + l];
      mx = fmaxf(mx, fabsf(d[i]));
      sq += d[i] * d[i];
    }
    const float m = (!mask || mask[c]) ? 1.f : 0.f;
    const float r = ov[6] - logf(mx + kErrEps);
    part += (double)(m * (sq * (1.f / 6.f) + lam * r * r));
    float gf[6];
    for (int i = 0; i < 6; ++i) gf[i] = m * 2.f * d[i] * (1.f / 6.f) * inv_n;
    const float tg = (gf[0] + gf[1] + gf[2]) * (1.f / 3.f);
    __align__(16) __nv_bfloat162 row[kOutPad / 2];
    row[0] = __floats2bfloat162_rn(gf[0] - tg, gf[1] - tg);
    row[1] = __floats2bfloat162_rn(gf[2] - tg, gf[3]);
    row[2] = __floats2bfloat162_rn(gf[4], gf[5]);
    row[3] = __floats2bfloat162_rn(m * lam * 2.f * r * inv_n, 0.f);
#pragma unroll
    for (int i = 4; i < kOutPad / 2; ++i) row[i] = __floats2bfloat162_rn(0.f, 0.f);
    int4 *dst = reinterpret_cast<int4 *>(go + c * kOutPad);
    dst[0] = reinterpret_cast<const int4 *>(row)[0];
    dst[1] = reinterpret_cast<const int4 *>(row)[1];
  }
  part = block_sum_d(part, red);
  if (threadIdx.x == 0) atomicAdd(loss, part * (double)inv_n);
}

// -------------------------------------------------------------------- AdamW
// Loshchilov & Hutter (2019): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
// p <- p - lr (m/bc1 / (sqrt(v/bc2) + eps) + wd p), bc = 1 - beta^step.
__global__ void __launch_bounds__(256) adamw_kernel(NetMeta M, float *__restrict__ p, const float *__restrict__ g,
                                                    float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                                                    float b2, float eps, float wd, float bc1, float bc2, int update) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M.total;
       i += (long long)gridDim.x * blockDim.x) {
    float pi = p[i];
    if (update) {
      const float gi = g[i];
      const float mi = b1 * m[i] + (1.f - b1) * gi;
      const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
      m[i] = mi;
      v[i] = vi;
      pi -= lr * ((mi / bc1) / (sqrtf(vi / bc2) + eps) + wd * pi);
      p[i] = pi;
    }
    for (int l = 0; l < 4; ++l) {
      const LayerMeta &L = M.L[l];
      const long long k = i - L.w_off;
      if (k < 0 || k >= 27LL * L.cout * L.cin) continue;
      const int tap = (int)(k / ((long long)L.cout * L.cin));
      const int rem = (int)(k - (long long)tap * L.cout * L.cin), co = rem / L.cin, ci = rem - co * L.cin;
      const __nv_bfloat16 w = __float2bfloat16_rn(pi);
      L.wb[k] = w;
      L.wt[((long long)(26 - tap) * L.cin + ci) * L.cout + co] = w;
    }
  }
}

// --------------------------------------------------------------- indicator
// Eigenvalues of the symmetric 3 x 3 tensor f by the trigonometric closed form
// (O. K. Smith, Comm. ACM 4 (1961) 168): with q = tr f / 3 and
// p = sqrt(|f - q I|_F^2 / 6), the eigenvalues are q + 2 p cos(phi + 2 pi k/3),
// phi = acos(det((f - q I)/p) / 2) / 3.
__device__ __forceinline__ void sym3_eig_minmax(const float *f, float &lmin, float &lmax) {
  const float q = (f[0] + f[1] + f[2]) * (1.f / 3.f);
  const float p1 = f[3] * f[3] + f[4] * f[4] + f[5] * f[5];
  const float a = f[0] - q, b = f[1] - q, c = f[2] - q;
  const float p2 = a * a + b * b + c * c + 2.f * p1;
  if (!(p2 > 0.f)) {
    lmin = lmax = q;
    return;
  }
  const float p = sqrtf(p2 * (1.f / 6.f)), ip = 1.f / p;
  const float A = a * ip, Bv = b * ip, C = c * ip, xy = f[3] * ip, xz = f[4] * ip, yz = f[5] * ip;
  const float det = A * (Bv * C - yz * yz) - xy * (xy * C - yz * xz) + xz * (xy * yz - Bv * xz);
  const float r = fminf(fmaxf(0.5f * det, -1.f), 1.f);
  const float phi = acosf(r) * (1.f / 3.f);
  lmax = q + 2.f * p * cosf(phi);
  lmin = q + 2.f * p * cosf(phi + 2.0943951023931953f);
}

__global__ void __launch_bounds__(256) indicator_kernel(const float *__restrict__ o, Vol V, int B, float thr,
                                                        float *__restrict__ f_out, float *__restrict__ r_out,
                                                        unsigned int *__restrict__ flags) {
  const long long n = (long long)V.nz * V.ny * V.nx;
  const int nbx = V.nx / B, nby = V.ny / B;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const float4 *src = reinterpret_cast<const float4 *>(o + c * kOutPad);
    const float4 a = src[0], b = src[1];
    const float ov[7] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z};
    float f[6];
    head_f(ov, f);
    for (int i = 0; i < 6; ++i) f_out[i * n + c] = f[i];
    float lmin, lmax;
    sym3_eig_minmax(f, lmin, lmax);
    float r = fmaxf(fmaxf(fmaxf(0.f, -lmin), fmaxf(0.f, lmax - 1.f)), expf(ov[6]));
    // fmaxf drops NaN: a non-finite output must still send its block to the
    // exact closure
    float chk = 0.f;
    for (int i = 0; i < 7; ++i) chk += ov[i] * 0.f;
    if (chk != 0.f) r = INFINITY;
    if (r_out) r_out[c] = r;
    if (r > thr) {
      const int x = (int)(c % V.nx), y = (int)((c / V.nx) % V.ny), z = (int)(c / ((long long)V.nx * V.ny));
      flags[(x / B) + nbx * ((y / B) + nby * (z / B))] = 1u;
    }
  }
}

__global__ void __launch_bounds__(1024) compact_kernel(const unsigned int *__restrict__ flags, int n,
                                                       int *__restrict__ list, int *__restrict__ count) {
  __shared__ int wsum[32];
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per, e = min(n, b + per);
  int k = 0;
  for (int i = b; i < e; ++i) k += flags[i] != 0;
  // block exclusive scan of k
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = k;
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    int s = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    wsum[lane] = s;
  }
  __syncthreads();
  int pos = incl - k + (w ? wsum[w - 1] : 0);
  for (int i = b; i < e; ++i)
    if (flags[i]) list[pos++] = i;
  if (threadIdx.x == blockDim.x - 1) *count = pos;
}

__global__ void __launch_bounds__(256) unpack_kernel(const float *__restrict__ o, Vol V, float *__restrict__ out) {
  const long long vol = (long long)V.nz * V.ny * V.nx, n = vol * V.n;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(c / vol);
    const long long l = c - v * vol;
    for (int i = 0; i < kOut; ++i) out[((long long)v * kOut + i) * vol + l] = o[c * kOutPad + i];
  }
}

int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

size_t wgrad_smem_bytes(int cin, int cout) {
  return (size_t)27 * cout * cin * 4 + (size_t)HN * cin * 2 + (size_t)TN * cout * 2;
}
long long tiles(const Vol &V) {
  return (long long)V.n * ((V.nz + TZ - 1) / TZ) * ((V.ny + TY - 1) / TY) * ((V.nx + TX - 1) / TX);
}

namespace {
// Persistent grid: resident CTAs per SM x SMs, capped by the tile count and
// by `cap` when positive.
int persistent_grid(const void *fn, size_t smem, long long nt, int cap) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, smem) != cudaSuccess || per < 1) per = 1;
  long long g = (long long)per * sms;
  if (cap > 0 && g > cap) g = cap;
  if (g > nt) g = nt;
  return (int)g;
}
}  // namespace

template <int C_IN, int C_OUT>
cudaError_t wgrad(const __nv_bfloat16 *x, const __nv_bfloat16 *gpre, const Vol &V, float *gW, float *gb, int grid,
                  cudaStream_t st) {
  const size_t sm = wgrad_smem_bytes(C_IN, C_OUT);
  const void *fn = (const void *)wgrad_kernel<C_IN, C_OUT>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int g = persistent_grid(fn, sm, tiles(V), grid);
  if (g < 1) return cudaSuccess;
  wgrad_kernel<C_IN, C_OUT><<<g, kThreads, sm, st>>>(x, gpre, V, gW, gb);
  return cudaGetLastError();
}

cudaError_t features(const float *kappa, const float *S, const float *E, const Vol &V, int B, double h, double *sums,
                     float *bstat, __nv_bfloat16 *x0, float *feat_out, cudaStream_t st) {
  if (V.n < 1) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * 2 * V.n, st);
  if (e != cudaSuccess) return e;
  const int nblk = (V.nx / B) * (V.ny / B) * (V.nz / B);
  feat_stats_kernel<<<dim3(nblk, V.n), 256, 0, st>>>(kappa, S, E, V, B, (float)h, sums, bstat);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long n = (long long)V.n * V.nz * V.ny * V.nx;
  feat_pack_kernel<<<grid_for(n, 256), 256, 0, st>>>(kappa, S, E, V, B, (float)h, sums, bstat, x0, feat_out);
  return cudaGetLastError();
}

cudaError_t head_loss(const float *o, const float *f_ref, const unsigned char *mask, const Vol &V, float lam,
                      unsigned long long *count, double *loss, __nv_bfloat16 *go, cudaStream_t st) {
  const long long n = (long long)V.n * V.nz * V.ny * V.nx;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  count_kernel<<<grid_for(n, 256), 256, 0, st>>>(mask, n, count);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  head_loss_kernel<<<grid_for(n, 256), 256, 0, st>>>(o, f_ref, mask, V, lam, count, loss, go);
  return cudaGetLastError();
}

cudaError_t adamw(const NetMeta &M, float *p, const float *g, float *m, float *v, float lr, float b1, float b2,
                  float eps, float wd, float bc1, float bc2, int update, cudaStream_t st) {
  adamw_kernel<<<grid_for(M.total, 256), 256, 0, st>>>(M, p, g, m, v, lr, b1, b2, eps, wd, bc1, bc2, update);
  return cudaGetLastError();
}

cudaError_t indicator(const float *o, const Vol &V, int B, float thr, float *f_out, float *r_out, unsigned int *flags,
                      cudaStream_t st) {
  const int nblk = (V.nx / B) * (V.ny / B) * (V.nz / B);
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned int) * nblk, st);
  if (e != cudaSuccess) return e;
  const long long n = (long long)V.nz * V.ny * V.nx;
  indicator_kernel<<<grid_for(n, 256), 256, 0, st>>>(o, V, B, thr, f_out, r_out, flags);
  return cudaGetLastError();
}

cudaError_t compact_flags(const unsigned int *flags, int n, int *list, int *count, cudaStream_t st) {
  compact_kernel<<<1, 1024, 0, st>>>(flags, n, list, count);
  return cudaGetLastError();
}

cudaError_t unpack_outputs(const float *o, const Vol &V, float *o_out, cudaStream_t st) {
  const long long n = (long long)V.n * V.nz * V.ny * V.nx;
  unpack_kernel<<<grid_for(n, 256), 256, 0, st>>>(o, V, o_out);
  return cudaGetLastError();
}

template cudaError_t wgrad<16, 32>(const __nv_bfloat16 *, const __nv_bfloat16 *, const Vol &, float *, float *, int,
                                   cudaStream_t);
template cudaError_t wgrad<32, 32>(const __nv_bfloat16 *, const __nv_bfloat16 *, const Vol &, float *, float *, int,
                                   cudaStream_t);
template cudaError_t wgrad<32, 16>(const __nv_bfloat16 *, const __nv_bfloat16 *, const Vol &, float *, float *, int,
                                   cudaStream_t);

}  // namespace cnn
}  // namespace vet
