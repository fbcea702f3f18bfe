// vet_cnn_tc.cu -- the learned closure's 3x3x3 convolutions on the 5th
// generation tensor cores (tcgen05, accumulators in tensor memory).
//
// Implicit GEMM per output tile of 8 x 16 x 2 cells (x, y, z): for each of
// the 27 taps and each 16-channel step of the input, one
// tcgen05.mma.kind::f16 (BF16 x BF16 -> FP32) per z-slice with M = 128 cells
// (8 x 16, one z), N = C_out, K = 16.  Both operands sit in shared memory in
// the canonical K-major layout without swizzle: "core matrices" of 8 rows x
// 16 bytes stored contiguously, addressed by a descriptor (start, leading
// byte offset LBO between core matrices along K, stride byte offset SBO
// between 8-row groups along M or N).
//   A (activations): the tile's 10 x 18 x 4 input halo stored as
//     [16-byte channel chunk][halo cell][16 B], so that 8 cells consecutive
//     in x form one core matrix at every tap shift: start = the tap's first
//     halo cell, LBO = one chunk plane (720 x 16 B), SBO = one halo row in y
//     (10 x 16 B).
//   B (weights): [tap][channel chunk][C_out][16 B], LBO = C_out x 16 B,
//     SBO = 8 x 16 B.
// One thread issues the 54 (C_in = 32) or 27 (C_in = 16) x 2 MMAs of a tile
// and commits them to an mbarrier; the other warps wait (bounded) and then
// read the accumulators back with tcgen05.ld (warp w reads tensor-memory
// lanes 32 (w % 4).. of z-slice w / 4), apply the epilogue and store.
// Tensor memory (2 x C_out columns) is allocated once per CTA and released
// before the CTA exits, also when a wait gave up.
#include <cstdint>

#include <cuda_bf16.h>

#include "vet_cnn.h"

namespace vet {
namespace cnn {
namespace {

constexpr int TX = 8, TY = 16, TZ = 2;     // output tile (x, y, z)
constexpr int HX = 10, HY = 18, HZ = 4;    // input halo
constexpr int HN = HX * HY * HZ;           // 720 halo cells
constexpr long long kWaitPolls = 1LL << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = __fdividef(1.0f, 1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// Shared-memory matrix descriptor (tcgen05): start address, LBO and SBO in
// 16-byte units, descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// 32 (or 16) consecutive FP32 columns of this thread's tensor-memory lane.
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[N]);
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct Tile {
  int v, tz, ty, tx;
};

__device__ __forceinline__ Tile tile_of(long long t, const Vol &V) {
  const int ntx = (V.nx + TX - 1) / TX, nty = (V.ny + TY - 1) / TY, ntz = (V.nz + TZ - 1) / TZ;
  Tile r;
  r.tx = (int)(t % ntx);
  t /= ntx;
  r.ty = (int)(t % nty);
  t /= nty;
  r.tz = (int)(t % ntz);
  r.v = (int)(t / ntz);
  return r;
}

// Columns of tensor memory: 2 accumulator sets x 2 z-slices x C_OUT, a
// power of two >= 32 as tcgen05.alloc requires.
template <int C_OUT>
__host__ __device__ constexpr uint32_t tmem_cols() {
  return 4 * C_OUT <= 32 ? 32 : (4 * C_OUT <= 64 ? 64 : 128);
}

template <int C_IN>
__host__ __device__ constexpr size_t halo_bytes() {
  return (size_t)C_IN / 8 * HN * 16;
}

// Halo of tile ti into one buffer (cp.async, zero outside the volume), by
// the `nthreads` threads 0 .. nthreads - 1 of the CTA.
template <int C_IN>
__device__ __forceinline__ void load_halo(uint32_t dst, const __nv_bfloat16 *__restrict__ x, const Vol &V,
                                          const Tile &ti, int nthreads) {
  constexpr int NCI = C_IN / 8;
  const long long vol = (long long)V.nz * V.ny * V.nx;
  for (int h = threadIdx.x; h < HN * NCI; h += nthreads) {
    const int hc = h / NCI, c = h - hc * NCI;
    const int hz = hc / (HX * HY), hy = (hc / HX) % HY, hx = hc % HX;
    const int z = ti.tz * TZ + hz - 1, y = ti.ty * TY + hy - 1, xx = ti.tx * TX + hx - 1;
    const bool in = z >= 0 && z < V.nz && y >= 0 && y < V.ny && xx >= 0 && xx < V.nx;
    const long long cell = in ? (long long)ti.v * vol + ((long long)z * V.ny + y) * V.nx + xx : 0;
    cp_async16(dst + (uint32_t)((c * HN + hc) * 16), x + cell * C_IN + c * 8, in ? 16u : 0u);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// The 27 x (C_IN / 16) x 2 MMAs of one tile (one thread).  Descriptor start
// addresses are 16-byte units in their low 14 bits, so moving an operand by
// b bytes adds b / 16 to the descriptor (no carry: shared memory < 256 KB).
template <int C_IN, int C_OUT>
__device__ __forceinline__ void issue_tile(uint32_t tmem_acc, uint64_t a0, uint64_t b0) {
  constexpr int NCI = C_IN / 8;
  constexpr uint32_t IDESC = idesc_bf16(128, C_OUT);
#pragma unroll
  for (int tap = 0; tap < 27; ++tap) {
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
#pragma unroll
    for (int ks = 0; ks < NCI / 2; ++ks) {
      const uint64_t bd = b0 + (uint64_t)((tap * NCI + 2 * ks) * C_OUT);
#pragma unroll
      for (int z = 0; z < TZ; ++z) {
        const int h0 = (z + dz + 1) * (HX * HY) + (dy + 1) * HX + (dx + 1);
        mma_bf16(tmem_acc + z * C_OUT, a0 + (uint64_t)(2 * ks * HN + h0), bd, IDESC, (tap | ks) ? 1u : 0u);
      }
    }
  }
}

template <int C_OUT, int EPI>
__device__ __forceinline__ void epilogue(uint32_t taddr, const Tile &ti, const Vol &V, const float *__restrict__ sBias,
                                         __nv_bfloat16 *__restrict__ pre_out, const __nv_bfloat16 *__restrict__ pre_in,
                                         void *__restrict__ out, int r, int zs) {
  float acc[C_OUT];
  tmem_ld<C_OUT>(taddr, acc);
  const long long vol = (long long)V.nz * V.ny * V.nx;
  const int xx = ti.tx * TX + (r & 7), y = ti.ty * TY + (r >> 3), z = ti.tz * TZ + zs;
  if (xx >= V.nx || y >= V.ny || z >= V.nz) return;
  const long long cell = (long long)ti.v * vol + ((long long)z * V.ny + y) * V.nx + xx;
  if (EPI == EPI_F32) {
    float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(out) + cell * C_OUT);
#pragma unroll
    for (int i = 0; i < C_OUT / 4; ++i)
      dst[i] = make_float4(acc[4 * i] + sBias[4 * i], acc[4 * i + 1] + sBias[4 * i + 1],
                           acc[4 * i + 2] + sBias[4 * i + 2], acc[4 * i + 3] + sBias[4 * i + 3]);
    return;
  }
  __align__(16) __nv_bfloat162 o2[C_OUT / 2];
  __align__(16) __nv_bfloat162 p2[C_OUT / 2];
  if (EPI == EPI_SILU) {
#pragma unroll
    for (int i = 0; i < C_OUT / 2; ++i) {
      const float z0 = acc[2 * i] + sBias[2 * i], z1 = acc[2 * i + 1] + sBias[2 * i + 1];
      p2[i] = __floats2bfloat162_rn(z0, z1);
      o2[i] = __floats2bfloat162_rn(silu(z0), silu(z1));
    }
    if (pre_out) {
      int4 *pd = reinterpret_cast<int4 *>(pre_out + cell * C_OUT);
#pragma unroll
      for (int i = 0; i < C_OUT / 8; ++i) pd[i] = reinterpret_cast<const int4 *>(p2)[i];
    }
  } else {  // EPI_SILU_BWD
    const int4 *ps = reinterpret_cast<const int4 *>(pre_in + cell * C_OUT);
#pragma unroll
    for (int i = 0; i < C_OUT / 8; ++i) reinterpret_cast<int4 *>(p2)[i] = ps[i];
#pragma unroll
    for (int i = 0; i < C_OUT / 2; ++i)
      o2[i] = __floats2bfloat162_rn(acc[2 * i] * silu_grad(__bfloat162float(p2[i].x)),
                                    acc[2 * i + 1] * silu_grad(__bfloat162float(p2[i].y)));
  }
  int4 *od = reinterpret_cast<int4 *>(reinterpret_cast<__nv_bfloat16 *>(out) + cell * C_OUT);
#pragma unroll
  for (int i = 0; i < C_OUT / 8; ++i) od[i] = reinterpret_cast<const int4 *>(o2)[i];
}

// Bounded wait on an mbarrier phase by a whole warp, giving up early when
// another role has aborted (*abort set).
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort) {
  bool done = false;
  for (long long i = 0; i < kWaitPolls; ++i) {
    if (!done) done = mbar_try(bar, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    if ((i & 1023) == 1023 && __any_sync(0xffffffffu, *abort != 0)) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

constexpr int kWorkers = 256;             // warps 0-7: halo loads and epilogue
constexpr int kTcThreads = kWorkers + 32; // warp 8: issues the MMAs

// Warp-specialised pipeline.  Tile i of this CTA uses halo buffer and
// accumulator set s = i % 2.
//   MMA warp (one lane): wait full[s] (halo of tile i landed) and, from
//     i >= 2, empty[s] (tile i - 2's accumulators read); issue tile i's MMAs;
//     commit them to done[s].
//   Workers: wait done[s] (tile i's MMAs finished: buffer s is free, its
//     accumulators ready); start the cp.async loads of tile i + 2 into buffer
//     s; read and store tile i's outputs; arrive on empty[s]; complete the
//     loads, fence them to the async proxy and arrive on full[s].
// The tensor cores run tile i + 1 while the workers drain tile i and load
// tile i + 2.  Every wait is bounded; a role that gives up sets `abort`,
// which ends the other role's waits too.
template <int C_IN, int C_OUT, int EPI>
__global__ void __launch_bounds__(kTcThreads, 1)
    conv3d_tc_kernel(const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ W,
                     const float *__restrict__ b, Vol V, __nv_bfloat16 *__restrict__ pre_out,
                     const __nv_bfloat16 *__restrict__ pre_in, void *__restrict__ out, int *status) {
  constexpr int NCI = C_IN / 8;
  constexpr uint32_t A_LBO = HN * 16, A_SBO = HX * 16;
  constexpr uint32_t B_LBO = C_OUT * 16, B_SBO = 8 * 16;
  constexpr uint32_t TCOLS = tmem_cols<C_OUT>();
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *sA = smem;                                   // 2 x [NCI][HN][16 B]
  unsigned char *sB = smem + 2 * halo_bytes<C_IN>();          // [27][NCI][C_OUT][16 B]
  __shared__ __align__(8) uint64_t full[2], done[2], empty[2];
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int abort_flag;
  __shared__ int n_committed[2];  // MMA batches committed per accumulator set
  __shared__ float sBias[C_OUT];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int h = threadIdx.x; h < 27 * C_OUT * NCI; h += blockDim.x) {
    const int c = h % NCI, co = (h / NCI) % C_OUT, tap = h / (NCI * C_OUT);
    const int4 val = reinterpret_cast<const int4 *>(W + ((size_t)tap * C_OUT + co) * C_IN)[c];
    *reinterpret_cast<int4 *>(sB + (((size_t)tap * NCI + c) * C_OUT + co) * 16) = val;
  }
  if (threadIdx.x < C_OUT) sBias[threadIdx.x] = b ? b[threadIdx.x] : 0.f;
  if (threadIdx.x == 0) {
    for (int k = 0; k < 2; ++k) {
      mbar_init(&full[k], kWorkers);
      mbar_init(&done[k], 1);
      mbar_init(&empty[k], kWorkers);
      n_committed[k] = 0;
    }
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base_slot;
  const long long nt = (long long)V.n * ((V.nz + TZ - 1) / TZ) * ((V.ny + TY - 1) / TY) * ((V.nx + TX - 1) / TX);
  const int ntile = blockIdx.x < nt ? (int)((nt - 1 - blockIdx.x) / gridDim.x + 1) : 0;  // tiles of this CTA
  const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);

  if (warp == kWorkers / 32) {
    // ---- MMA issuer
    const uint64_t a_desc0 = smem_desc(a_base, A_LBO, A_SBO);
    const uint64_t a_desc1 = smem_desc(a_base + (uint32_t)halo_bytes<C_IN>(), A_LBO, A_SBO);
    const uint64_t b_desc = smem_desc(b_base, B_LBO, B_SBO);
    for (int i = 0; i < ntile; ++i) {
      const int s = i & 1;
      const uint32_t use = (uint32_t)(i >> 1);  // this is use number `use` of buffer / accumulator set s
      bool ok = wait_or_abort(&full[s], use & 1u, &abort_flag);
      if (ok && i >= 2) ok = wait_or_abort(&empty[s], (use - 1) & 1u, &abort_flag);
      if (!ok) {
        if (lane == 0) {
          atomicOr(status, 16);
          abort_flag = 1;
        }
        break;
      }
      fence_after_sync();
      if (lane == 0) {
        issue_tile<C_IN, C_OUT>(tmem + (uint32_t)(s * 2 * C_OUT), s ? a_desc1 : a_desc0, b_desc);
        mma_commit(&done[s]);
        ++n_committed[s];
      }
      __syncwarp();
    }
  }
  int n_waited0 = 0, n_waited1 = 0;  // batches this worker saw complete, per set
  if (warp != kWorkers / 32) {
    // ---- workers
    const int sp = warp & 3, zs = warp >> 2;  // TMEM lane quarter and z-slice of this warp
    const int r = 32 * sp + lane;              // this thread's row of the 128-cell slice
    // prologue: halos of tiles 0 and 1
    for (int k = 0; k < 2 && k < ntile; ++k) {
      load_halo<C_IN>(a_base + (uint32_t)(k * halo_bytes<C_IN>()), x, V,
                      tile_of(blockIdx.x + (long long)k * gridDim.x, V), kWorkers);
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      fence_proxy_async();
      mbar_arrive(&full[k]);
    }
    for (int i = 0; i < ntile; ++i) {
      const int s = i & 1;
      const uint32_t use = (uint32_t)(i >> 1);
      if (!wait_or_abort(&done[s], use & 1u, &abort_flag)) {
        if (lane == 0) {
          atomicOr(status, 16);
          abort_flag = 1;
        }
        break;
      }
      if (s) ++n_waited1; else ++n_waited0;
      fence_after_sync();
      const bool more = i + 2 < ntile;
      if (more)
        load_halo<C_IN>(a_base + (uint32_t)(s * halo_bytes<C_IN>()), x, V,
                        tile_of(blockIdx.x + (long long)(i + 2) * gridDim.x, V), kWorkers);
      epilogue<C_OUT, EPI>(tmem + ((uint32_t)(32 * sp) << 16) + (uint32_t)(s * 2 * C_OUT + zs * C_OUT),
                           tile_of(blockIdx.x + (long long)i * gridDim.x, V), V, sBias, pre_out, pre_in, out, r, zs);
      fence_before_sync();
      mbar_arrive(&empty[s]);
      if (more) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        fence_proxy_async();
        mbar_arrive(&full[s]);
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
  fence_before_sync();
  __syncthreads();
  if (abort_flag && threadIdx.x == 0) {
    // committed MMAs may still run: wait (bounded) for every batch committed
    // but not yet seen complete before tensor and shared memory are released
    for (int k = 0; k < 2; ++k)
      for (int ph = k ? n_waited1 : n_waited0; ph < n_committed[k]; ++ph)
        for (long long n = 0; n < kWaitPolls && !mbar_try(&done[k], (uint32_t)ph & 1u); ++n) {
        }
  }
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
  }
}

}  // namespace

size_t conv_tc_smem_bytes(int cin, int cout) { return 2 * (size_t)cin / 8 * HN * 16 + (size_t)27 * cout * cin * 2; }

template <int C_IN, int C_OUT, int EPI>
cudaError_t conv3d_tc(const __nv_bfloat16 *x, const __nv_bfloat16 *W, const float *b, const Vol &V,
                      __nv_bfloat16 *pre_out, const __nv_bfloat16 *pre_in, void *out, int *status, cudaStream_t st) {
  const size_t sm = conv_tc_smem_bytes(C_IN, C_OUT);
  const void *fn = (const void *)conv3d_tc_kernel<C_IN, C_OUT, EPI>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long nt = (long long)V.n * ((V.nz + TZ - 1) / TZ) * ((V.ny + TY - 1) / TY) * ((V.nx + TX - 1) / TX);
  if (nt < 1) return cudaSuccess;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kTcThreads, sm) != cudaSuccess || per < 1) per = 1;
  // tensor memory: at most 4 CTAs of <= 128 columns share an SM's 512
  if (per > 4) per = 4;
  long long g = (long long)per * sms;
  if (g > nt) g = nt;
  conv3d_tc_kernel<C_IN, C_OUT, EPI><<<(int)g, kTcThreads, sm, st>>>(x, W, b, V, pre_out, pre_in, out, status);
  return cudaGetLastError();
}

#define VET_TC_INST(CI, CO, EPI)                                                                                  \
  template cudaError_t conv3d_tc<CI, CO, EPI>(const __nv_bfloat16 *, const __nv_bfloat16 *, const float *,       \
                                              const Vol &, __nv_bfloat16 *, const __nv_bfloat16 *, void *, int *, \
                                              cudaStream_t);
VET_TC_INST(16, 32, EPI_SILU)
VET_TC_INST(32, 32, EPI_SILU)
VET_TC_INST(32, 16, EPI_F32)
VET_TC_INST(16, 32, EPI_SILU_BWD)
VET_TC_INST(32, 32, EPI_SILU_BWD)

}  // namespace cnn
}  // namespace vet
