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
//                 direction, with the quadratures E, F, P (Eqs. 10-12)
//                 accumulated in registers across all directions and
//                 f = P/E (Eq. 13) in the epilogue, so that I is never stored.
// Both passes stage the block's kappa/S tile, the directions' ray templates
// and the incoming faces in shared memory.  Faces are stored by the face pass
// already in the consumer's upwind frame and padded, so staging is a plain
// 16-byte copy.  Kernels are compiled for the block edges 8 and 16 (index
// arithmetic folds to shifts) and for a runtime edge.
#include <cstdint>

#include "vet_internal.h"

namespace vet {

namespace {

template <typename R> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };
template <typename R> using vec2_t = typename Vec2<R>::T;

// One segment of optical depth x >= 0, given y = -x log2(e) (segment lengths
// are stored pre-scaled by -h log2(e)), updates I exactly over a cell of
// source S: I <- I - (I - S)(1 - e^-x) = S + (I - S) e^-x.  Each form is
// evaluated where it cannot cancel, as I' = fma(I - S, w, base):
//   thin (x < 1/2): base = I, w = -(1 - e^-x) = y q(y) with q of degree 4
//     fitted for relative error by Lawson's iteratively reweighted least
//     squares (7.7e-8 in exact arithmetic, the level of FP32 rounding): the
//     other form would round S to its ulp before subtracting almost all of
//     it when S >> I, and 1 - e would cancel;
//   thick (x >= 1/2): base = S, w = e^-x from the MUFU (ex2.approx); here
//     the first form would cancel when I >> S.
// Thin segments never use the MUFU, whose 1.5e-7 error is not zero-mean and
// would compound along long thin paths.  FP64: expm1 and exp2 of the CUDA
// math library in the same two forms.
__device__ __forceinline__ float seg_weight(float y, bool &thin) {
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(y));
  float q = 1.0833843353054956e-03f;
  q = fmaf(q, y, 9.4645342235962007e-03f);
  q = fmaf(q, y, 5.5464640186780434e-02f);
  q = fmaf(q, y, 2.4022290282685121e-01f);
  q = fmaf(q, y, 6.9314712699664371e-01f);
  thin = y > -0.7213475204444817f;  // x < 1/2
  return thin ? q * y : e;
}

__device__ __forceinline__ double seg_weight(double y, bool &thin) {
  thin = y > -0.7213475204444817;
  return thin ? expm1(y * 0.6931471805599453094) : exp2(y);
}

// tb: byte address of the ray's start cell in the tile; ev.off is the byte
// offset of the segment's cell from it.
template <typename R>
__device__ __forceinline__ void segment(const unsigned char *__restrict__ tb, const TplEvent<R> &ev, R &I) {
  const vec2_t<R> ks = *reinterpret_cast<const vec2_t<R> *>(tb + ev.off);
  bool thin;
  const R w = seg_weight(ks.x * ev.len, thin);
  I = fma(I - ks.y, w, thin ? I : ks.y);
}

// Intensity at a ray's start point: entering with I at the upwind end of
// segment `last`, the segments last, last-1, ..., 0 are crossed downwind.
// last = -1 (a start point on the upwind face) returns I unchanged.
template <typename R>
__device__ __forceinline__ R march(const vec2_t<R> *__restrict__ tile, int idx0, int last,
                                   const TplEvent<R> *__restrict__ ev, R I) {
  const unsigned char *tb = reinterpret_cast<const unsigned char *>(tile + idx0);
  int e = last;
  for (; e > 0; e -= 2) {  // two segments per trip
    const TplEvent<R> e0 = ev[e], e1 = ev[e - 1];
    segment<R>(tb, e0, I);
    segment<R>(tb, e1, I);
  }
  if (e == 0) segment<R>(tb, ev[0], I);
  return I;
}

// march() with the event index shared by the lanes of a warp: from wl (the
// warp's largest `last`) down to 0, a lane with e > last crosses an identity
// segment (length 0, offset 0: the thin form returns I exactly).  Every event
// index read is below the template's event capacity (3B).
template <typename R>
__device__ __forceinline__ R march_aligned(const vec2_t<R> *__restrict__ tile, int idx0, int last, int wl,
                                           const TplEvent<R> *__restrict__ ev, R I) {
  const unsigned char *tb = reinterpret_cast<const unsigned char *>(tile + idx0);
  int e = wl;
  for (; e > 0; e -= 2) {  // two segments per trip
    TplEvent<R> e0 = ev[e], e1 = ev[e - 1];
    if (e > last) { e0.len = R(0); e0.off = 0; }
    if (e - 1 > last) { e1.len = R(0); e1.off = 0; }
    segment<R>(tb, e0, I);
    segment<R>(tb, e1, I);
  }
  if (e == 0 && last >= 0) segment<R>(tb, ev[0], I);
  return I;
}

// Typed view of one direction's template blob.
template <typename R>
struct Tpl {
  const TplHead<R> *h;
  const TplEvent<R> *cev, *nev;
  const int16_t *cpos, *npos, *ck, *nk;
  const vec2_t<R> *cw, *nw;
  __device__ __forceinline__ Tpl(const unsigned char *base, const TplLayout &L)
      : h(reinterpret_cast<const TplHead<R> *>(base)),
        cev(reinterpret_cast<const TplEvent<R> *>(base + L.cev)),
        nev(reinterpret_cast<const TplEvent<R> *>(base + L.nev)),
        cpos(reinterpret_cast<const int16_t *>(base + L.cpos)),
        npos(reinterpret_cast<const int16_t *>(base + L.npos)),
        ck(reinterpret_cast<const int16_t *>(base + L.ck)),
        nk(reinterpret_cast<const int16_t *>(base + L.nk)),
        cw(reinterpret_cast<const vec2_t<R> *>(base + L.cw)),
        nw(reinterpret_cast<const vec2_t<R> *>(base + L.nw)) {}
};

// Bilinear interpolation on incoming face ae (Sec. 2.2.5 reading: short
// characteristics between blocks).  The face is staged in the upwind frame
// with row stride B + 2 (node B + 1 is zero padding, reached only with weight
// 0).  lb, lc are the ray's upwind-frame coordinates along the two in-plane
// axes, kb/kc and wb/wc its exit-table entries (floor and (f, 1-f)).
template <typename R>
__device__ __forceinline__ R face_value(const R *__restrict__ fin, int fstride, int B, int ae, int lb, int lc,
                                        int kb, int kc, vec2_t<R> wb, vec2_t<R> wc) {
  const int W = B + 2;
  const int ib = max(lb + kb, 0), ic = max(lc + kc, 0);
  const R *F = fin + ae * fstride + ib * W + ic;
  return wb.y * (wc.y * F[0] + wc.x * F[1]) + wb.x * (wc.y * F[W] + wc.x * F[W + 1]);
}

// ------------------------------------------------ TMA bulk copies + mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Producer arrival that also announces `bytes` of incoming bulk copies.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for the completion of phase `parity`: gives up after
// `limit` polls, records `code` in the device status word and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit, int *status, int code) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  atomicOr(status, code);
  return false;
}

// The same wait taken by a whole warp (all 32 lanes converged): every lane
// polls, but the warp stops only on a warp-wide decision, so either all lanes
// see the phase complete or all give up together.  A per-lane decision could
// let one lane leave a loop whose other lanes then wait forever at the next
// warp-synchronous instruction.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, long long limit, int *status,
                                               int code) {
  const uint32_t a = smem_u32(bar);
  bool done = false;
  for (long long i = 0; i < limit; ++i) {
    if (!done) {
      uint32_t d;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(d)
          : "r"(a), "r"(parity)
          : "memory");
      done = d != 0;
    }
    if (__all_sync(0xffffffffu, done)) return true;
  }
  if ((threadIdx.x & 31) == 0) atomicOr(status, code);
  return false;
}

// Polls granted to the final wait for copies still in flight after another
// wait gave up (status bit 8 if even that one gives up).
constexpr long long kDrainPolls = 1LL << 22;

// One bulk copy global -> shared (16-byte aligned addresses and size),
// completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// A staged direction ("slot") in shared memory: its template blob followed
// by its three incoming faces.  Called by one thread: issues the four bulk
// copies of internal direction d for block (bx, by, bz); the faces come from
// the upwind neighbours' stored downwind faces or from the materialised
// boundary faces bnd[face][d].
// tpl_bytes: the leading part of the template staged (TL.bytes for the cell
// passes, TL.node_bytes for the face pass; 0 stages the faces alone); the
// faces follow it in the slot.
template <typename R>
__device__ __forceinline__ void issue_slot(unsigned char *slot, const GridDims &g, const TplLayout &TL, int bx,
                                           int by, int bz, int d, const unsigned char *__restrict__ tpl_g,
                                           const R *__restrict__ faces, const R *__restrict__ bnd, uint64_t *bar,
                                           int tpl_bytes, int sgn_bits = -1) {
  const unsigned char *src = tpl_g + (size_t)d * TL.bytes;
  if (tpl_bytes > 0) bulk_g2s(slot, src, (uint32_t)tpl_bytes, bar);
  const TplHead<R> *hd = reinterpret_cast<const TplHead<R> *>(src);
  const int nblk = g.nbx * g.nby * g.nbz;
  const uint32_t fb = (uint32_t)(g.fstride * sizeof(R));
  const int b3[3] = {bx, by, bz};
  const int nb3[3] = {g.nbx, g.nby, g.nbz};
  for (int a = 0; a < 3; ++a) {
    const int s = sgn_bits >= 0 ? ((sgn_bits >> a) & 1 ? -1 : 1) : hd->sgn[a];
    int nb[3] = {b3[0], b3[1], b3[2]};
    nb[a] -= s;
    const R *fsrc;
    if (nb[a] < 0 || nb[a] >= nb3[a]) {
      const int face = 2 * a + (s > 0 ? 0 : 1);
      fsrc = bnd + ((long long)face * g.ndir + d) * g.fstride;
    } else {
      const long long nid = ((long long)nb[2] * g.nby + nb[1]) * g.nbx + nb[0];
      fsrc = faces + (((long long)d * nblk + nid) * 3 + a) * g.fstride;
    }
    bulk_g2s(slot + tpl_bytes + a * fb, fsrc, fb, bar);
  }
}

// Cell-pass order entries: the internal direction index, optionally with the
// direction's signs (bit 16 + a set: component a negative; bit 19: signs
// present), so that staging needs no read of the template head.
__device__ __forceinline__ int order_dir(int v) { return v & 0xffff; }
__device__ __forceinline__ int order_sgn(int v) { return (v >> 19) & 1 ? (v >> 16) & 7 : -1; }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor in the stream drains; it
// runs its independent prologue, then griddep_wait() blocks the calling
// thread until the predecessor has completed and its writes are visible
// (a no-op for an ordinary launch).  griddep_launch_dependents() lets the
// successor start once every CTA of this grid has called it or exited.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

// Bytes of the three staged incoming faces of one direction.
template <typename R>
__host__ __device__ inline size_t faces_bytes(int B) {
  return sizeof(R) * 3 * (size_t)face_stride_elems<R>(B);
}
// One staged direction of the cell passes (whole template and faces) and of
// the face pass (head and node-ray parts, faces).
template <typename R>
__host__ __device__ inline size_t slot_bytes(int B) {
  return (size_t)tpl_layout<R>(B).bytes + faces_bytes<R>(B);
}
template <typename R>
__host__ __device__ inline size_t face_slot_bytes_t(int B) {
  return (size_t)tpl_layout<R>(B).node_bytes + faces_bytes<R>(B);
}

// Tile loaders.  With the block edge and the CTA's thread count known at
// compile time (NT != 0) every thread issues all its global loads before its
// first shared-memory store, so they are in flight together.
template <typename R, int BC, int NT = 0>
__device__ __forceinline__ void load_tile(vec2_t<R> *tile, TileShape ts, const GridDims &g, int bx, int by, int bz,
                                          const R *__restrict__ kappa, const R *__restrict__ S) {
  if constexpr (BC != 0 && NT != 0) {
    constexpr int B = BC, B2 = B * B, K = B2 * B / NT;
    static_assert(B2 * B % NT == 0, "tile cells must divide evenly over the threads");
    vec2_t<R> v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = (int)threadIdx.x + k * NT, x = i % B, y = (i / B) % B, z = i / B2;
      const long long gi = ((long long)(bz * B + z) * g.ny + (by * B + y)) * g.nx + (bx * B + x);
      v[k].x = kappa[gi];
      v[k].y = S[gi];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = (int)threadIdx.x + k * NT, x = i % B, y = (i / B) % B, z = i / B2;
      tile[x + ts.sy * y + ts.sz * z] = v[k];
    }
    return;
  }
  const int B = BC ? BC : g.B;
  const int B2 = B * B, B3 = B2 * B;
  for (int i = threadIdx.x; i < B3; i += blockDim.x) {
    const int x = i % B, y = (i / B) % B, z = i / B2;
    const long long gi = ((long long)(bz * B + z) * g.ny + (by * B + y)) * g.nx + (bx * B + x);
    vec2_t<R> v;
    v.x = kappa[gi];
    v.y = S[gi];
    tile[x + ts.sy * y + ts.sz * z] = v;
  }
}

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Dynamic shared memory of a cell-pass CTA holding `nslots` staged directions.
template <typename R>
__host__ __device__ inline size_t smem_bytes(int B, int nslots) {
  return align16(sizeof(vec2_t<R>) * (size_t)cell_tile(B).elems) + (size_t)nslots * slot_bytes<R>(B);
}
// ... and of an unpaired face-pass CTA.
template <typename R>
__host__ __device__ inline size_t face_smem_bytes(int B, int nslots) {
  return align16(sizeof(vec2_t<R>) * (size_t)node_tile(B).elems) + (size_t)nslots * face_slot_bytes_t<R>(B);
}

// ... and of a paired cell-pass CTA (16-byte tile entries).
__host__ __device__ inline size_t pair_smem_bytes(int B, int nslots) {
  return align16(sizeof(float4) * (size_t)cell_tile(B).elems) + (size_t)nslots * slot_bytes<float>(B);
}

constexpr int kDirTile = 4;   // directions per cell-pass tile (two tiles in flight)
constexpr size_t kSmemMax = 232448 - 64;  // opt-in limit less the static mbarriers

template <typename R>
int cell_dir_tile(int B, int want) {
  int dt = want > 0 ? want : kDirTile;
  while (dt > 1 && smem_bytes<R>(B, 2 * dt) > kSmemMax) --dt;
  return dt;
}

// ---------------------------------------------------------------- face pass
constexpr int kFaceThreads = 512;

// Directions per tile of the paired cell pass: an even number (whole pairs)
// whose two buffers fit, at most the tuned tile rounded up to even.
inline int pair_dir_tile(int B, int want) {
  int dt = want > 0 ? want : kDirTile;
  dt = (dt + 1) & ~1;
  if (dt > kMaxTune) dt = kMaxTune;
  while (dt > 2 && pair_smem_bytes(B, 2 * dt) > kSmemMax - 4096) dt -= 2;  // 4 KB: the staged order
  return dt;
}

// Face pass: one CTA per item (a block and up to kFaceGroup directions of one
// octant at the same wavefront level).  The CTA loads the block's kappa/S
// tile; the lanes of warp 0 then issue the TMA bulk copies of the item's
// template parts and incoming faces, one slot each, all in flight at once
// (once the previous level has completed: each level is a programmatic
// dependent launch of the one before); then the (direction, node) rays are
// spread over the threads.
template <typename R, int BC>
__global__ void __launch_bounds__(kFaceThreads, 3)
    face_pass_kernel(GridDims g, const R *__restrict__ kappa, const R *__restrict__ S,
                     const unsigned char *__restrict__ tpl_g, const FaceItem *__restrict__ items,
                     R *__restrict__ faces, const R *__restrict__ bnd, long long spin_limit, int *status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full;
  const int B = BC ? BC : g.B;
  const int W = B + 2, N1 = B + 1, NN = N1 * N1;
  const TileShape ts = node_tile(B);
  const TplLayout TL = tpl_layout<R>(B);
  const size_t sb = face_slot_bytes_t<R>(B);
  const FaceItem it = items[blockIdx.x];
  vec2_t<R> *tile = reinterpret_cast<vec2_t<R> *>(smem);
  unsigned char *slots = smem + align16(sizeof(vec2_t<R>) * (size_t)ts.elems);
  const int bx = it.block % g.nbx, by = (it.block / g.nbx) % g.nby, bz = it.block / (g.nbx * g.nby);
  const int nblk = g.nbx * g.nby * g.nbz;
  griddep_launch_dependents();  // as in face_pair_kernel
  load_tile<R, BC, kFaceThreads>(tile, ts, g, bx, by, bz, kappa, S);
  if (threadIdx.x < 32) {  // warp 0: one lane per staged direction
    griddep_wait();        // the incoming faces are the previous level's output
    if (threadIdx.x == 0) {
      mbar_init(&full, 1);
      mbar_fence_init();
      mbar_expect_tx(&full, (uint32_t)(sb * it.dir_count));
    }
    __syncwarp();
    const int j = threadIdx.x;
    if (j < it.dir_count)
      issue_slot<R>(slots + sb * j, g, TL, bx, by, bz, it.dir_begin + j, tpl_g, faces, bnd, &full, TL.node_bytes,
                    it.octant);
  }
  __syncthreads();
  if (!mbar_wait_warp(&full, 0, spin_limit, status, 1)) {
    // the copies this CTA issued must land before its shared memory is
    // released: thread 0 waits for them once more (bounded) and all return
    if (threadIdx.x == 0) mbar_wait(&full, 0, kDrainPolls, status, 8);
    return;
  }
  // Downwind faces on the domain boundary are read by no block: only the
  // axes whose downwind neighbour exists are computed (the directions of an
  // item share one octant, hence one set of axes).
  int live = 0, nlive = 0;  // live: the computed axes, 2 bits each
  {
    const TplHead<R> *h0 = reinterpret_cast<const TplHead<R> *>(slots);
    const int bb[3] = {bx, by, bz}, nbb[3] = {g.nbx, g.nby, g.nbz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int nb = bb[a] + h0->sgn[a];
      if (nb >= 0 && nb < nbb[a]) live |= a << (2 * nlive++);
    }
  }
  const int NNL = nlive * NN, total = it.dir_count * NNL;
  // warp-uniform trips: lanes past the end redo the last node and store nothing
  for (int w0 = (int)threadIdx.x & ~31; w0 < total; w0 += blockDim.x) {
    const int wr = w0 + ((int)threadIdx.x & 31);
    const bool act = wr < total;
    const int w = act ? wr : total - 1;
    // w = (j * nlive + ai) * NN + r; NN is a compile-time constant for a
    // templated block edge, and q / nlive (q < 3 * kMaxTune, nlive <= 3) is
    // a multiply-shift instead of a runtime division
    const int q = w / NN, r = w - q * NN;
    const int j = nlive == 1 ? q : (nlive == 2 ? q >> 1 : (q * 21846) >> 16);
    const int ai = q - j * nlive;
    const Tpl<R> T(slots + sb * j, TL);
    const R *fin = reinterpret_cast<const R *>(slots + sb * j + TL.node_bytes);
    const int a = (live >> (2 * ai)) & 3;
    const int ub = r / N1, uc = r - ub * N1;  // upwind-frame node on the downwind face of axis a
    // upwind-frame node coordinates (L0, L1, L2): B along the face's axis
    const int L0 = a == 0 ? B : ub;
    const int L1 = a == 1 ? B : (a == 0 ? ub : uc);
    const int L2 = a == 2 ? B : uc;
    const int p0 = T.npos[L0], p1 = T.npos[N1 + L1], p2 = T.npos[2 * N1 + L2];
    int last = p0, ae = 0, la = L0, lb = L1, lc = L2;
    if (p1 < last) { last = p1; ae = 1; la = L1; lb = L0; }
    if (p2 < last) { last = p2; ae = 2; la = L2; lb = L0; lc = L1; }
    const int row = (ae * 2) * N1 + la;
    R I = face_value<R>(fin, g.fstride, B, ae, lb, lc, T.nk[row], T.nk[row + N1], T.nw[row], T.nw[row + N1]);
    if (!act) last = -1;
    // The lanes march in lockstep aligned at the downwind end: the warp runs
    // from its largest `last` down to event 0, and a lane whose own ray is
    // shorter crosses zero-length segments at its start cell (offset 0,
    // length 0: the update returns I unchanged) until the event index
    // reaches its `last`.  Lanes on one template then cross the same event
    // at the same step, so their tile addresses are one common offset from
    // neighbouring start cells (few shared-memory bank conflicts).
    const int wl = __reduce_max_sync(0xffffffffu, last);
    if (wl >= 0) {
      // where last >= 0, every L >= 1 and the start cell is inside the block
      const int c0 = T.h->sgn[0] > 0 ? L0 - 1 : B - L0;
      const int c1 = T.h->sgn[1] > 0 ? L1 - 1 : B - L1;
      const int c2 = T.h->sgn[2] > 0 ? L2 - 1 : B - L2;
      const int idx0 = last >= 0 ? c0 + ts.sy * c1 + ts.sz * c2 : 0;
      I = march_aligned<R>(tile, idx0, last, wl, T.nev, I);
    }
    if (act) faces[(((long long)(it.dir_begin + j) * nblk + it.block) * 3 + a) * g.fstride + ub * W + uc] = I;
  }
}

// ---------------------------------------------------------------- cell pass
__device__ __forceinline__ void atomic_max_nonneg(void *p, float v) {
  atomicMax(reinterpret_cast<unsigned int *>(p), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(void *p, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double_as_longlong(v));
}

constexpr int kCellThreads = 512;  // one cell per thread

// Cell pass: one CTA per (block, slab of 512 of the block's cells), one cell
// per thread.  Directions are visited in tiles of `dt` (octants interleaved)
// through two shared-memory buffers: thread 0 issues the TMA bulk copies of
// tile t + 2 as soon as every warp has released the buffer of tile t, so the
// loads run behind the ray work; warps wait only on the "full" barrier of the
// tile they start.  For block edges that are multiples of 4, each warp holds a
// 4 x 4 x 2 brick of cells, whose rays have similar lengths.
template <typename R, int MODE, int BC>
__global__ void __launch_bounds__(kCellThreads, 2)
    cell_pass_kernel(GridDims g, int parts, int dt, const R *__restrict__ kappa, const R *__restrict__ S,
                     const unsigned char *__restrict__ tpl_g, const int *__restrict__ order,
                     const R *__restrict__ faces, const R *__restrict__ bnd, R *__restrict__ I_out,
                     R *__restrict__ M_out, R *__restrict__ E_out, R *__restrict__ f_out, void *emax_bits,
                     long long spin_limit, int *status, const int *__restrict__ block_list) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[2], empty[2];
  const int B = BC ? BC : g.B;
  const int B2 = B * B, B3 = B2 * B;
  const TileShape ts = cell_tile(B);
  const TplLayout TL = tpl_layout<R>(B);
  const int fstride = g.fstride;
  const size_t sb = slot_bytes<R>(B);
  vec2_t<R> *tile = reinterpret_cast<vec2_t<R> *>(smem);
  unsigned char *buf0 = smem + align16(sizeof(vec2_t<R>) * (size_t)ts.elems);
  const int item = blockIdx.x / parts, part = blockIdx.x - item * parts;
  const int blk = block_list ? block_list[item] : item;
  const int bx = blk % g.nbx, by = (blk / g.nbx) % g.nby, bz = blk / (g.nbx * g.nby);
  const int cpc = B3 / parts;  // cells of this CTA
  const int nwarps = blockDim.x >> 5;
  const int ntiles = (g.ndir + dt - 1) / dt;
  int issued = 0, consumed = 0;   // thread 0's count of tiles issued / waited for
  auto issue_tile = [&](int t) {  // thread 0 only
    issued = t + 1;
    const int b = t & 1, d0 = t * dt, nd = min(dt, g.ndir - d0);
    unsigned char *buf = buf0 + (size_t)b * dt * sb;
    mbar_expect_tx(&full[b], (uint32_t)(sb * nd));
    for (int j = 0; j < nd; ++j)
      issue_slot<R>(buf + sb * j, g, TL, bx, by, bz, order_dir(order[d0 + j]), tpl_g, faces, bnd, &full[b], TL.bytes,
                    order_sgn(order[d0 + j]));
  };
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], nwarps);
    mbar_init(&empty[1], nwarps);
    mbar_fence_init();
    issue_tile(0);
    if (ntiles > 1) issue_tile(1);
  }
  load_tile<R, BC>(tile, ts, g, bx, by, bz, kappa, S);
  __syncthreads();

  const bool active = (int)threadIdx.x < cpc;
  int cx, cy, cz;
  if (BC != 0 && BC % 4 == 0 && cpc == kCellThreads) {
    // slab of B x B x (512 / B^2) cells; warp w holds brick w of 4 x 4 x 2
    const int nbx4 = B / 4;
    const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    cx = 4 * (w % nbx4) + (ln & 3);
    cy = 4 * ((w / nbx4) % nbx4) + ((ln >> 2) & 3);
    cz = 2 * (w / (nbx4 * nbx4)) + (ln >> 4) + part * (kCellThreads / B2);
  } else {
    const int lc = part * cpc + (active ? (int)threadIdx.x : 0);
    cx = lc % B;
    cy = (lc / B) % B;
    cz = lc / B2;
  }
  const int tc = cx + ts.sy * cy + ts.sz * cz;  // tile index
  const long long gc = ((long long)(bz * B + cz) * g.ny + (by * B + cy)) * g.nx + (bx * B + cx);
  // Moments over all directions: a plain partial sum over the directions of
  // one tile, folded into the totals once per tile.  The fold of E, Pxx, Pyy
  // and Pzz (positive sums that f_ii = P_ii / E depends on) is Kahan
  // compensated: plain sequential FP32 sums of N terms lose about N/2 ulp,
  // which would dominate the error of f.  F is summed only when the caller
  // asks for the moments (MODE 0).
  constexpr bool kWantF = MODE == 0;
  R mom[10], cmp[4];
  for (int m = 0; m < 10; ++m) mom[m] = R(0);
  for (int m = 0; m < 4; ++m) cmp[m] = R(0);

  bool ok = true;
  for (int t = 0; t < ntiles && ok; ++t) {
    const int b = t & 1;
    const uint32_t ph = (uint32_t)((t >> 1) & 1);
    if (!mbar_wait_warp(&full[b], ph, spin_limit, status, 2)) { ok = false; break; }
    consumed = t + 1;
    const int nd = min(dt, g.ndir - t * dt);
    const unsigned char *buf = buf0 + (size_t)b * dt * sb;
    if (active) {
      R part[10];
      for (int m = 0; m < 10; ++m) part[m] = R(0);
      for (int j = 0; j < nd; ++j) {
        const Tpl<R> T(buf + sb * j, TL);
        const R *fin = reinterpret_cast<const R *>(buf + sb * j + TL.bytes);
        // upwind-frame coordinates; the exit axis ae is the one whose plane
        // event comes first, (lb, lc) the other two in increasing axis order
        const int l0 = T.h->sgn[0] > 0 ? cx : B - 1 - cx;
        const int l1 = T.h->sgn[1] > 0 ? cy : B - 1 - cy;
        const int l2 = T.h->sgn[2] > 0 ? cz : B - 1 - cz;
        const int p0 = T.cpos[l0], p1 = T.cpos[B + l1], p2 = T.cpos[2 * B + l2];
        int last = p0, ae = 0, la = l0, lb = l1, lc = l2;
        if (p1 < last) { last = p1; ae = 1; la = l1; lb = l0; }
        if (p2 < last) { last = p2; ae = 2; la = l2; lb = l0; lc = l1; }
        const int row = (ae * 2) * B + la;
        const R Iin = face_value<R>(fin, fstride, B, ae, lb, lc, T.ck[row], T.ck[row + B], T.cw[row], T.cw[row + B]);
        const R I = march<R>(tile, tc, last, T.cev, Iin);
        if (MODE == 1) {
          I_out[(long long)T.h->ext * g.ncell + gc] = I;
        } else {
          const R *c = T.h->c;  // w (1, n, nn), the same for every lane
#pragma unroll
          for (int m = 0; m < 10; ++m)
            if (kWantF || m == 0 || m >= 4) part[m] = fma(I, c[m], part[m]);
        }
      }
      if (MODE != 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // E, Pxx, Pyy, Pzz: compensated fold
          const int m = q == 0 ? 0 : 3 + q;
          const R y = part[m] - cmp[q];
          const R tt = mom[m] + y;
          cmp[q] = (tt - mom[m]) - y;
          mom[m] = tt;
        }
        if (kWantF) {
          mom[1] += part[1];
          mom[2] += part[2];
          mom[3] += part[3];
        }
        mom[7] += part[7];
        mom[8] += part[8];
        mom[9] += part[9];
      }
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[b]);
    bool prod_ok = true;
    if (threadIdx.x == 0 && t + 2 < ntiles) {
      prod_ok = mbar_wait(&empty[b], ph, spin_limit, status, 4);
      if (prod_ok) issue_tile(t + 2);
    }
    // warp 0 leaves together when its producer lane gave up
    if (!__shfl_sync(0xffffffffu, prod_ok ? 1 : 0, 0)) { ok = false; break; }
  }
  if (threadIdx.x == 0) {
    // after a wait gave up, tiles may still be in flight into this CTA's
    // shared memory: wait (bounded) for every tile issued but not consumed
    for (int t = consumed; t < issued; ++t) mbar_wait(&full[t & 1], (uint32_t)((t >> 1) & 1), kDrainPolls, status, 8);
  }
  if (MODE != 1) {
    R emax = R(0);
    if (active && ok) {
      const R E = mom[0];
      if (kWantF) {
        for (int m = 0; m < 10; ++m) M_out[m * g.ncell + gc] = mom[m];
      } else {
        E_out[gc] = E;
      }
      if (E > R(0)) {
        // f = P / E correctly rounded (IEEE division; for FP32 operands the
        // same value as the FP64 quotient rounded to FP32)
        for (int m = 0; m < 6; ++m) f_out[m * g.ncell + gc] = mom[4 + m] / E;
      } else {
        for (int m = 0; m < 6; ++m) f_out[m * g.ncell + gc] = m < 3 ? R(1) / R(3) : R(0);
      }
      emax = E;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const R v = __shfl_xor_sync(0xffffffffu, emax, o);
      emax = v > emax ? v : emax;
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(emax_bits, emax);
  }
}

// --------------------------------------------- cell pass, mirrored ray pairs
// FP32 cell pass for block edges 8 and 16 and direction sets closed under
// negation (HEALPix sets are, rotated or not).  The ray from cell c in
// direction d and the ray from the point-mirrored cell c' = (B-1-x, B-1-y,
// B-1-z) in direction -d are mirror images (and so are (c, -d) and (c', d)):
// in their own upwind frames both
// start at the same coordinates along every axis the direction crosses, leave
// through the same event with the same exit-table entries, and cross segments
// of the same lengths whose tile offsets are negatives of each other.  So one
// thread marches both in lockstep from one event list and one 16-byte load
// of the paired tile per step, with the two exponentials' arithmetic on
// packed FP32 pairs (f32x2); only the in-plane face coordinates (which may
// differ along an axis the direction does not cross) and the staged faces
// are per ray.  The lanes of a warp march aligned at the downwind end, as in
// the face pass, so that at each step they read one event and a brick of
// neighbouring entries.  The cell order lists the pairs (d, -d)
// consecutively; a staged tile holds dt / 2 pairs.
// one lower-half cell and its mirror per thread; 512 threads (two CTAs per SM)
// for 16^3 blocks, where three 256-thread CTAs would hold fewer warps
__host__ __device__ constexpr int pair_threads(int B) { return B == 16 ? 512 : 256; }

__device__ __forceinline__ uint64_t pk2(float a, float b) {
  return (uint64_t)__float_as_uint(a) | ((uint64_t)__float_as_uint(b) << 32);
}
__device__ __forceinline__ void upk2(uint64_t r, float &a, float &b) {
  a = __uint_as_float((uint32_t)r);
  b = __uint_as_float((uint32_t)(r >> 32));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// The paired tiles of both mirrored passes hold 16-byte entries (kappa(p),
// kappa(p'), S(p), S(p')): p' is the cell where the mirror ray stands when
// the primary ray stands at p.  Template offsets are for 8-byte entries,
// hence 2 * off below.

// One ray on a paired tile, on a template of its own (a pair whose templates
// are not exact mirrors): march() reading the ray's own (kappa, S) = (.x, .z).
__device__ __forceinline__ float march4(const unsigned char *__restrict__ tb, int last,
                                       const TplEvent<float> *__restrict__ ev, float I) {
  for (int e = last; e >= 0; --e) {
    const TplEvent<float> E = ev[e];
    const float4 q = *reinterpret_cast<const float4 *>(tb + 2 * E.off);
    bool thin;
    const float w = seg_weight(q.x * E.len, thin);
    I = fmaf(I - q.z, w, thin ? I : q.z);
  }
  return I;
}

// One cell ray on its own template (upwind-frame coordinates l0..l2, start
// entry at byte address tb of the paired tile): exit lookup, entry value,
// march.
__device__ __forceinline__ float cell_ray4(const Tpl<float> &T, const float *fin, int fstride, int B, int l0, int l1,
                                           int l2, const unsigned char *tb) {
  const int p0 = T.cpos[l0], p1 = T.cpos[B + l1], p2 = T.cpos[2 * B + l2];
  int last = p0, ae = 0, la = l0, lb = l1, lc = l2;
  if (p1 < last) { last = p1; ae = 1; la = l1; lb = l0; }
  if (p2 < last) { last = p2; ae = 2; la = l2; lb = l0; lc = l1; }
  const int row = (ae * 2) * B + la;
  const float Iin = face_value<float>(fin, fstride, B, ae, lb, lc, T.ck[row], T.ck[row + B], T.cw[row], T.cw[row + B]);
  return march4(tb, last, T.cev, Iin);
}

// Paired tile of the cell pass: p' is the point-mirrored cell of the same
// block.  (Issuing all loads before the stores, as the face passes do, made
// this kernel slower.)
template <int BC>
__device__ __forceinline__ void load_tile_pair(float4 *tile, TileShape ts, const GridDims &g, int bx, int by, int bz,
                                               const float *__restrict__ kappa, const float *__restrict__ S) {
  constexpr int B = BC, B2 = B * B, B3 = B2 * B;
  for (int i = threadIdx.x; i < B3; i += blockDim.x) {
    const int x = i % B, y = (i / B) % B, z = i / B2;
    const long long gi = ((long long)(bz * B + z) * g.ny + (by * B + y)) * g.nx + (bx * B + x);
    const long long gm = ((long long)(bz * B + B - 1 - z) * g.ny + (by * B + B - 1 - y)) * g.nx + (bx * B + B - 1 - x);
    tile[x + ts.sy * y + ts.sz * z] = make_float4(kappa[gi], kappa[gm], S[gi], S[gm]);
  }
}

// One segment of both rays of a mirrored pair on a paired tile (tb: the
// primary ray's start entry): the update and the two forms of segment() on
// packed FP32 pairs.
__device__ __forceinline__ void segment_pair_tile(const unsigned char *__restrict__ tb, const TplEvent<float> &ev,
                                                  uint64_t &I) {
  const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(tb + 2 * ev.off);  // (k, k'), (S, S')
  const uint64_t Y = mul2(q.x, pk2(ev.len, ev.len));
  float y1, y2;
  upk2(Y, y1, y2);
  float e1, e2;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(y1));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e2) : "f"(y2));
  uint64_t p = pk2(1.0833843353054956e-03f, 1.0833843353054956e-03f);
  p = fma2(p, Y, pk2(9.4645342235962007e-03f, 9.4645342235962007e-03f));
  p = fma2(p, Y, pk2(5.5464640186780434e-02f, 5.5464640186780434e-02f));
  p = fma2(p, Y, pk2(2.4022290282685121e-01f, 2.4022290282685121e-01f));
  p = fma2(p, Y, pk2(6.9314712699664371e-01f, 6.9314712699664371e-01f));
  float n1, n2;  // -(1 - e^-x) of the thin form
  upk2(mul2(p, Y), n1, n2);
  const bool thin1 = y1 > -0.7213475204444817f, thin2 = y2 > -0.7213475204444817f;
  float i1, i2, s1, s2;
  upk2(I, i1, i2);
  upk2(q.y, s1, s2);
  I = fma2(sub2(I, q.y), pk2(thin1 ? n1 : e1, thin2 ? n2 : e2), pk2(thin1 ? i1 : s1, thin2 ? i2 : s2));
}

template <int MODE, int BC>
__global__ void __launch_bounds__(pair_threads(BC), BC == 16 ? 2 : 3)
    cell_pair_kernel(GridDims g, int parts, int dt, const float *__restrict__ kappa, const float *__restrict__ S,
                     const unsigned char *__restrict__ tpl_g, const int *__restrict__ order,
                     const float *__restrict__ faces, const float *__restrict__ bnd, float *__restrict__ I_out,
                     float *__restrict__ M_out, float *__restrict__ E_out, float *__restrict__ f_out, void *emax_bits,
                     long long spin_limit, int *status, const int *__restrict__ block_list) {
  constexpr int B = BC, B2 = B * B;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[2], empty[2];
  constexpr int kOrdMax = 1024;  // direction sets up to nside = 8 keep their order in shared memory
  __shared__ int s_ord[kOrdMax];
  const bool ord_smem = g.ndir <= kOrdMax;
  const TileShape ts = cell_tile(B);
  const TplLayout TL = tpl_layout<float>(B);
  const int fstride = g.fstride;
  const size_t sb = slot_bytes<float>(B);
  float4 *tile = reinterpret_cast<float4 *>(smem);
  unsigned char *buf0 = smem + align16(sizeof(float4) * (size_t)ts.elems);
  const int item = blockIdx.x / parts, part = blockIdx.x - item * parts;
  const int blk = block_list ? block_list[item] : item;
  const int bx = blk % g.nbx, by = (blk / g.nbx) % g.nby, bz = blk / (g.nbx * g.nby);
  const int nwarps = blockDim.x >> 5;
  const int ntiles = (g.ndir + dt - 1) / dt;
  int issued = 0, consumed = 0;
  auto issue_tile = [&](int t) {  // thread 0 only
    issued = t + 1;
    const int b = t & 1, d0 = t * dt, nd = min(dt, g.ndir - d0);
    unsigned char *buf = buf0 + (size_t)b * dt * sb;
    mbar_expect_tx(&full[b], (uint32_t)(sb * nd));
    for (int j = 0; j < nd; ++j) {
      const int v = (ord_smem && t >= 2) ? s_ord[d0 + j] : order[d0 + j];
      issue_slot<float>(buf + sb * j, g, TL, bx, by, bz, order_dir(v), tpl_g, faces, bnd, &full[b], TL.bytes,
                        order_sgn(v));
    }
  };
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], nwarps);
    mbar_init(&empty[1], nwarps);
    mbar_fence_init();
    griddep_wait();  // the faces are the face pass's output
    issue_tile(0);
    if (ntiles > 1) issue_tile(1);
  }
  if (ord_smem)
    for (int i = threadIdx.x; i < g.ndir; i += blockDim.x) s_ord[i] = order[i];
  load_tile_pair<BC>(tile, ts, g, bx, by, bz, kappa, S);
  __syncthreads();

  // this thread's lower-half cell (z < B/2): 4 x 4 x 2 bricks, warp-major
  const int q = part * pair_threads(BC) + (int)threadIdx.x;
  const int qb = q >> 5, ln = q & 31;
  const int cx = 4 * (qb % (B / 4)) + (ln & 3);
  const int cy = 4 * ((qb / (B / 4)) % (B / 4)) + ((ln >> 2) & 3);
  const int cz = 2 * (qb / (B2 / 16)) + (ln >> 4);
  const int mx = B - 1 - cx, my = B - 1 - cy, mz = B - 1 - cz;  // the mirror cell
  const unsigned char *t1 = reinterpret_cast<const unsigned char *>(tile + (cx + ts.sy * cy + ts.sz * cz));
  const unsigned char *t2 = reinterpret_cast<const unsigned char *>(tile + (mx + ts.sy * my + ts.sz * mz));
  const long long gc1 = ((long long)(bz * B + cz) * g.ny + (by * B + cy)) * g.nx + (bx * B + cx);
  const long long gc2 = ((long long)(bz * B + mz) * g.ny + (by * B + my)) * g.nx + (bx * B + mx);
  constexpr bool kWantF = MODE == 0;
  float mom[2][10], cmp[2][4];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int m = 0; m < 10; ++m) mom[r][m] = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) cmp[r][m] = 0.f;
  }

  // plain FP32 partial sums over four tiles, folded into the compensated
  // sums after the fourth (or the last) tile
  float part_[2][10];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int m = 0; m < 10; ++m) part_[r][m] = 0.f;
  bool ok = true;
  for (int t = 0; t < ntiles && ok; ++t) {
    const int b = t & 1;
    const uint32_t ph = (uint32_t)((t >> 1) & 1);
    if (!mbar_wait_warp(&full[b], ph, spin_limit, status, 2)) { ok = false; break; }
    consumed = t + 1;
    const int nd = min(dt, g.ndir - t * dt);
    const unsigned char *buf = buf0 + (size_t)b * dt * sb;
    // every cell needs both members of a pair: (c, d) with (c', -d), then
    // (c, -d) with (c', d), the primary direction's template driving each
    for (int jj = 0; jj < nd; ++jj) {
      const int j = (jj >> 1) << 1, j1 = j + (jj & 1), j2 = j + 1 - (jj & 1);
      const Tpl<float> T(buf + sb * j1, TL);  // primary: events and tables
      const TplHead<float> *H2 = reinterpret_cast<const TplHead<float> *>(buf + sb * j2);  // its antipode
      const float *fin1 = reinterpret_cast<const float *>(buf + sb * j1 + TL.bytes);
      const float *fin2 = reinterpret_cast<const float *>(buf + sb * j2 + TL.bytes);
      // upwind-frame coordinates of the cell in d; on a mirrored pair (every
      // sign flips) the mirror cell in -d has the same ones, since each
      // coordinate c becomes B - 1 - c, so both rays share them, their exit
      // and their face index
      const int l0 = T.h->sgn[0] > 0 ? cx : B - 1 - cx;
      const int l1 = T.h->sgn[1] > 0 ? cy : B - 1 - cy;
      const int l2 = T.h->sgn[2] > 0 ? cz : B - 1 - cz;
      float I1, I2;
      if (T.h->mirror) {
        const int p0 = T.cpos[l0], p1 = T.cpos[B + l1], p2 = T.cpos[2 * B + l2];
        int last = p0, ae = 0, la = l0, lb = l1, lc = l2;
        if (p1 < last) { last = p1; ae = 1; la = l1; lb = l0; }
        if (p2 < last) { last = p2; ae = 2; la = l2; lb = l0; lc = l1; }
        const int row = (ae * 2) * B + la;
        const int kb = T.ck[row], kc = T.ck[row + B];
        const float2 wb = T.cw[row], wc = T.cw[row + B];
        const float Iin1 = face_value<float>(fin1, fstride, B, ae, lb, lc, kb, kc, wb, wc);
        const float Iin2 = face_value<float>(fin2, fstride, B, ae, lb, lc, kb, kc, wb, wc);
        uint64_t I = pk2(Iin1, Iin2);
        // aligned at the downwind end; once the event index reaches the
        // warp's smallest `last` every lane marches and the identity
        // selects are dropped (the face passes, whose warps more often mix
        // templates and upwind-face nodes, measured slower with this split)
        int e = __reduce_max_sync(0xffffffffu, last);
        const int wmin = __reduce_min_sync(0xffffffffu, last);
        for (; e - 1 > wmin; e -= 2) {  // some lanes not yet started
          TplEvent<float> e0 = T.cev[e], e1 = T.cev[e - 1];
          if (e > last) { e0.len = 0.f; e0.off = 0; }
          if (e - 1 > last) { e1.len = 0.f; e1.off = 0; }
          segment_pair_tile(t1, e0, I);
          segment_pair_tile(t1, e1, I);
        }
        if (e > wmin) {
          TplEvent<float> e0 = T.cev[e];
          if (e > last) { e0.len = 0.f; e0.off = 0; }
          segment_pair_tile(t1, e0, I);
          --e;
        }
        for (; e > 0; e -= 2) {  // every lane marching
          segment_pair_tile(t1, T.cev[e], I);
          segment_pair_tile(t1, T.cev[e - 1], I);
        }
        if (e == 0) segment_pair_tile(t1, T.cev[0], I);
        upk2(I, I1, I2);
      } else {
        // the pair's templates differ (near-tied plane crossings ordered
        // differently): each ray follows its own direction's template
        const Tpl<float> T2(buf + sb * j2, TL);
        I1 = cell_ray4(T, fin1, fstride, B, l0, l1, l2, t1);
        const int m0 = H2->sgn[0] > 0 ? mx : B - 1 - mx;
        const int m1 = H2->sgn[1] > 0 ? my : B - 1 - my;
        const int m2 = H2->sgn[2] > 0 ? mz : B - 1 - mz;
        I2 = cell_ray4(T2, fin2, fstride, B, m0, m1, m2, t2);
      }
      if (MODE == 1) {
        I_out[(long long)T.h->ext * g.ncell + gc1] = I1;
        I_out[(long long)H2->ext * g.ncell + gc2] = I2;
      } else {
        const float *c1 = T.h->c, *c2 = H2->c;
#pragma unroll
        for (int m = 0; m < 10; ++m)
          if (kWantF || m == 0 || m >= 4) {
            part_[0][m] = fmaf(I1, c1[m], part_[0][m]);
            part_[1][m] = fmaf(I2, c2[m], part_[1][m]);
          }
      }
    }
    if (MODE != 1 && ((t & 3) == 3 || t + 1 == ntiles)) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {  // E, Pxx, Pyy, Pzz: compensated fold
          const int m = qq == 0 ? 0 : 3 + qq;
          const float y = part_[r][m] - cmp[r][qq];
          const float tt = mom[r][m] + y;
          cmp[r][qq] = (tt - mom[r][m]) - y;
          mom[r][m] = tt;
        }
        if (kWantF) {
          mom[r][1] += part_[r][1];
          mom[r][2] += part_[r][2];
          mom[r][3] += part_[r][3];
        }
        mom[r][7] += part_[r][7];
        mom[r][8] += part_[r][8];
        mom[r][9] += part_[r][9];
#pragma unroll
        for (int m = 0; m < 10; ++m) part_[r][m] = 0.f;
      }
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[b]);
    bool prod_ok = true;
    if (threadIdx.x == 0 && t + 2 < ntiles) {
      prod_ok = mbar_wait(&empty[b], ph, spin_limit, status, 4);
      if (prod_ok) issue_tile(t + 2);
    }
    if (!__shfl_sync(0xffffffffu, prod_ok ? 1 : 0, 0)) { ok = false; break; }
  }
  if (threadIdx.x == 0) {
    for (int t = consumed; t < issued; ++t) mbar_wait(&full[t & 1], (uint32_t)((t >> 1) & 1), kDrainPolls, status, 8);
  }
  if (MODE != 1) {
    float emax = 0.f;
    if (ok) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const long long gc = r ? gc2 : gc1;
        const float E = mom[r][0];
        if (kWantF) {
          for (int m = 0; m < 10; ++m) M_out[m * g.ncell + gc] = mom[r][m];
        } else {
          E_out[gc] = E;
        }
        if (E > 0.f) {
          // correctly rounded, as in cell_pass_kernel
          for (int m = 0; m < 6; ++m) f_out[m * g.ncell + gc] = mom[r][4 + m] / E;
        } else {
          for (int m = 0; m < 6; ++m) f_out[m * g.ncell + gc] = m < 3 ? 1.f / 3.f : 0.f;
        }
        emax = fmaxf(emax, E);
      }
    }
    for (int o = 16; o > 0; o >>= 1) emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(emax_bits, emax);
  }
}

// ------------------------------------------- face pass, mirrored block pairs
// FP32 face pass for block edges 8 and 16 and direction sets closed under
// negation with no zero component.  The node ray of block b in direction d
// from upwind-frame node coordinates L and the node ray of the point-mirrored
// block b' (nb - 1 - b per axis) in direction -d from the same L are mirror
// images: same exit event and exit-table entries, equal segment lengths, tile
// offsets negated, and b' sits at the same wavefront level.  One CTA takes an
// item (b, directions of one octant) together with (b', their antipodes); its
// tile holds, per cell p of b, (kappa_b(p), kappa_b'(p'), S_b(p), S_b'(p'))
// with p' the mirrored cell, so each step of a ray pair is one 16-byte load
// already packed for the f32x2 arithmetic.  Only the staged incoming faces
// differ between the two rays of a pair.

// Paired tile of the face pass: p' is the point-mirrored cell of block
// (mx, my, mz) (NT threads, all loads in flight before the stores).
template <int BC, int NT>
__device__ __forceinline__ void load_tile_mirrored(float4 *tile, TileShape ts, const GridDims &g, int bx, int by,
                                                   int bz, int mx, int my, int mz, const float *__restrict__ kappa,
                                                   const float *__restrict__ S) {
  constexpr int B = BC, B2 = B * B, K = B2 * B / NT;
  static_assert(B2 * B % NT == 0, "tile cells must divide evenly over the threads");
  float4 v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = (int)threadIdx.x + k * NT, x = i % B, y = (i / B) % B, z = i / B2;
    const long long gi = ((long long)(bz * B + z) * g.ny + (by * B + y)) * g.nx + (bx * B + x);
    const long long gm =
        ((long long)(mz * B + B - 1 - z) * g.ny + (my * B + B - 1 - y)) * g.nx + (mx * B + B - 1 - x);
    v[k] = make_float4(kappa[gi], kappa[gm], S[gi], S[gm]);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = (int)threadIdx.x + k * NT, x = i % B, y = (i / B) % B, z = i / B2;
    tile[x + ts.sy * y + ts.sz * z] = v[k];
  }
}

// Dynamic shared memory of a paired face-pass CTA for `dirs` direction pairs.
__host__ __device__ inline size_t face_pair_smem_bytes(int B, int dirs) {
  return align16(sizeof(float4) * (size_t)node_tile(B).elems) +
         (size_t)dirs * (face_slot_bytes_t<float>(B) + faces_bytes<float>(B));
}

template <int BC>
__global__ void __launch_bounds__(kFaceThreads, 2)
    face_pair_kernel(GridDims g, const float *__restrict__ kappa, const float *__restrict__ S,
                     const unsigned char *__restrict__ tpl_g, const FaceItem *__restrict__ items,
                     float *__restrict__ faces, const float *__restrict__ bnd, long long spin_limit, int *status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full;
  constexpr int B = BC, W = B + 2, N1 = B + 1, NN = N1 * N1;
  const TileShape ts = node_tile(B);
  const TplLayout TL = tpl_layout<float>(B);
  const size_t sb = face_slot_bytes_t<float>(B), fb3 = faces_bytes<float>(B);
  const FaceItem it = items[blockIdx.x];
  float4 *tile = reinterpret_cast<float4 *>(smem);
  // slots: the item's directions for b (node template parts and faces), then
  // the incoming faces of b' for their antipodes (whose node rays follow the
  // primary templates)
  unsigned char *slots = smem + align16(sizeof(float4) * (size_t)ts.elems);
  const int bx = it.block % g.nbx, by = (it.block / g.nbx) % g.nby, bz = it.block / (g.nbx * g.nby);
  const int mx = g.nbx - 1 - bx, my = g.nby - 1 - by, mz = g.nbz - 1 - bz;
  const int mblock = (mz * g.nby + my) * g.nbx + mx;
  const int nblk = g.nbx * g.nby * g.nbz;
  const int cnt = it.dir_count;
  griddep_launch_dependents();  // the next level may start its prologue
  // kappa and S are the call's inputs: loaded before the previous level ends
  load_tile_mirrored<BC, kFaceThreads>(tile, ts, g, bx, by, bz, mx, my, mz, kappa, S);
  if (threadIdx.x < 32) {  // warp 0: one lane per staged slot
    griddep_wait();        // the incoming faces are the previous level's output
    if (threadIdx.x == 0) {
      mbar_init(&full, 1);
      mbar_fence_init();
      mbar_expect_tx(&full, (uint32_t)((sb + fb3) * cnt));
    }
    __syncwarp();
    const int j = threadIdx.x;
    if (j < cnt)  // the octant's signs: no read of the template head before the copies
      issue_slot<float>(slots + sb * j, g, TL, bx, by, bz, it.dir_begin + j, tpl_g, faces, bnd, &full,
                        TL.node_bytes, it.octant);
    else if (j < 2 * cnt)  // antipodes: the opposite octant
      issue_slot<float>(slots + sb * cnt + fb3 * (j - cnt), g, TL, mx, my, mz, it.mirror_begin + (j - cnt), tpl_g,
                        faces, bnd, &full, 0, 7 - it.octant);
  }
  __syncthreads();
  if (!mbar_wait_warp(&full, 0, spin_limit, status, 1)) {
    if (threadIdx.x == 0) mbar_wait(&full, 0, kDrainPolls, status, 8);
    return;
  }
  // live axes (downwind neighbour exists): the same for b in d and b' in -d
  int live = 0, nlive = 0;
  {
    const TplHead<float> *h0 = reinterpret_cast<const TplHead<float> *>(slots);
    const int bb[3] = {bx, by, bz}, nbb[3] = {g.nbx, g.nby, g.nbz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int nb = bb[a] + h0->sgn[a];
      if (nb >= 0 && nb < nbb[a]) live |= a << (2 * nlive++);
    }
  }
  const int total = cnt * nlive * NN;
  for (int w0 = (int)threadIdx.x & ~31; w0 < total; w0 += blockDim.x) {
    const int wr = w0 + ((int)threadIdx.x & 31);
    const bool act = wr < total;
    const int w = act ? wr : total - 1;
    const int q = w / NN, r = w - q * NN;
    const int j = nlive == 1 ? q : (nlive == 2 ? q >> 1 : (q * 21846) >> 16);
    const int ai = q - j * nlive;
    const Tpl<float> T(slots + sb * j, TL);
    const float *fin1 = reinterpret_cast<const float *>(slots + sb * j + TL.node_bytes);
    const float *fin2 = reinterpret_cast<const float *>(slots + sb * cnt + fb3 * j);
    const int a = (live >> (2 * ai)) & 3;
    const int ub = r / N1, uc = r - ub * N1;
    const int L0 = a == 0 ? B : ub;
    const int L1 = a == 1 ? B : (a == 0 ? ub : uc);
    const int L2 = a == 2 ? B : uc;
    const int p0 = T.npos[L0], p1 = T.npos[N1 + L1], p2 = T.npos[2 * N1 + L2];
    int last = p0, ae = 0, la = L0, lb = L1, lc = L2;
    if (p1 < last) { last = p1; ae = 1; la = L1; lb = L0; }
    if (p2 < last) { last = p2; ae = 2; la = L2; lb = L0; lc = L1; }
    const int row = (ae * 2) * N1 + la;
    const int kb = T.nk[row], kc = T.nk[row + N1];
    const float2 wb = T.nw[row], wc = T.nw[row + N1];
    uint64_t I = pk2(face_value<float>(fin1, g.fstride, B, ae, lb, lc, kb, kc, wb, wc),
                     face_value<float>(fin2, g.fstride, B, ae, lb, lc, kb, kc, wb, wc));
    if (!act) last = -1;
    // lockstep aligned at the downwind end, as in the unpaired face pass
    const int wl = __reduce_max_sync(0xffffffffu, last);
    if (wl >= 0) {
      const int c0 = T.h->sgn[0] > 0 ? L0 - 1 : B - L0;
      const int c1 = T.h->sgn[1] > 0 ? L1 - 1 : B - L1;
      const int c2 = T.h->sgn[2] > 0 ? L2 - 1 : B - L2;
      const int idx0 = last >= 0 ? c0 + ts.sy * c1 + ts.sz * c2 : 0;
      const unsigned char *tb = reinterpret_cast<const unsigned char *>(tile + idx0);
      int e = wl;
      for (; e > 0; e -= 2) {
        TplEvent<float> e0 = T.nev[e], e1 = T.nev[e - 1];
        if (e > last) { e0.len = 0.f; e0.off = 0; }
        if (e - 1 > last) { e1.len = 0.f; e1.off = 0; }
        segment_pair_tile(tb, e0, I);
        segment_pair_tile(tb, e1, I);
      }
      if (e == 0 && last >= 0) segment_pair_tile(tb, T.nev[0], I);
    }
    if (act) {
      float I1, I2;
      upk2(I, I1, I2);
      const int node = ub * W + uc;
      faces[(((long long)(it.dir_begin + j) * nblk + it.block) * 3 + a) * g.fstride + node] = I1;
      faces[(((long long)(it.mirror_begin + j) * nblk + mblock) * 3 + a) * g.fstride + node] = I2;
    }
  }
}

// Boundary faces of every direction, materialised so that staging is a
// plain bulk copy: bnd[face][d][i] = Ib[face][ext(d)] (0 for vacuum).
template <typename R>
__global__ void fill_boundary_kernel(const GridDims g, const unsigned char *__restrict__ tpl_g, int tpl_bytes,
                                     const R *__restrict__ Ib, R *__restrict__ bnd) {
  const int face = blockIdx.y, d = blockIdx.x;
  const int ext = reinterpret_cast<const TplHead<R> *>(tpl_g + (size_t)d * tpl_bytes)->ext;
  const R v = Ib ? Ib[(long long)face * g.ndir + ext] : R(0);
  R *dst = bnd + ((long long)face * g.ndir + d) * g.fstride;
  for (int i = threadIdx.x; i < g.fstride; i += blockDim.x) dst[i] = v;
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
// The same rule on the cells of the listed blocks only.
template <typename R>
__global__ void floor_fix_blocks_kernel(const GridDims g, const int *__restrict__ block_list, const R *__restrict__ E,
                                        const void *__restrict__ emax_bits, double floor_rel, R *__restrict__ f) {
  const R floor = R(floor_rel) * load_max<R>(emax_bits);
  const int B = g.B, blk = block_list[blockIdx.x];
  const int bx = blk % g.nbx, by = (blk / g.nbx) % g.nby, bz = blk / (g.nbx * g.nby);
  for (int i = threadIdx.x; i < B * B * B; i += blockDim.x) {
    const long long c = ((long long)(bz * B + i / (B * B)) * g.ny + (by * B + (i / B) % B)) * g.nx + (bx * B + i % B);
    if (!(E[c] > floor)) {
      for (int m = 0; m < 6; ++m) f[m * g.ncell + c] = m < 3 ? R(1) / R(3) : R(0);
    }
  }
}

// Quadratures of stored intensities (Eqs. 10-12, c = 1): M[m][c] =
// sum_k coef[k][m] I[k][c].  HBM-bound (4 bytes of I per 10 FMAs): one thread
// per V consecutive cells with V-wide loads, directions unrolled by 4 so that
// several loads are in flight, coefficients of a chunk of 64 directions in
// shared memory.  The FP32 version keeps pairs of cells in packed f32x2
// accumulators against (c, c) coefficient pairs.
template <typename R, int V>
__global__ void __launch_bounds__(256, 4) moments_kernel(long long ncell, int ndir, const R *__restrict__ I,
                                                      const R *__restrict__ coef, R *__restrict__ M) {
  __shared__ R cs[64][10];
  const long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * V;
  R acc[V][10];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int m = 0; m < 10; ++m) acc[v][m] = R(0);
  for (int k0 = 0; k0 < ndir; k0 += 64) {
    const int nk = min(64, ndir - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < nk * 10; i += blockDim.x) cs[i / 10][i % 10] = coef[(long long)k0 * 10 + i];
    __syncthreads();
    if (c < ncell) {
#pragma unroll 4
      for (int k = 0; k < nk; ++k) {
        R v[V];
        const R *src = I + (long long)(k0 + k) * ncell + c;
        if (V == 4) {
          const float4 q = *reinterpret_cast<const float4 *>(src);
          v[0] = q.x; v[1] = q.y; v[V > 2 ? 2 : 0] = q.z; v[V > 3 ? 3 : 0] = q.w;
        } else if (V == 2) {
          const double2 q = *reinterpret_cast<const double2 *>(src);
          v[0] = q.x; v[V > 1 ? 1 : 0] = q.y;
        } else {
          v[0] = src[0];
        }
#pragma unroll
        for (int m = 0; m < 10; ++m) {
          const R cm = cs[k][m];
#pragma unroll
          for (int j = 0; j < V; ++j) acc[j][m] = fma(v[j], cm, acc[j][m]);
        }
      }
    }
  }
  if (c >= ncell) return;
#pragma unroll
  for (int m = 0; m < 10; ++m) {
    R *dst = M + m * ncell + c;
    if (V == 4) {
      *reinterpret_cast<float4 *>(dst) = make_float4(acc[0][m], acc[V > 1 ? 1 : 0][m], acc[V > 2 ? 2 : 0][m],
                                                     acc[V > 3 ? 3 : 0][m]);
    } else if (V == 2) {
      *reinterpret_cast<double2 *>(dst) = make_double2(acc[0][m], acc[V > 1 ? 1 : 0][m]);
    } else {
      dst[0] = acc[0][m];
    }
  }
}

int cell_parts(int B) {
  const int B3 = B * B * B;
  int parts = (B3 + kCellThreads - 1) / kCellThreads;
  while (B3 % parts) ++parts;
  return parts;
}

template <typename R, int BC>
void face_launch(const GridDims &g, const R *kappa, const R *S, const unsigned char *tpl, const FaceItem *items,
                 int nitems, int max_dirs, R *faces, const R *bnd, long long spin, int *status, cudaStream_t st) {
  if constexpr (sizeof(R) == sizeof(float) && BC != 0) {
    if (g.face_paired) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.gridDim = dim3(nitems);
      cfg.blockDim = dim3(kFaceThreads);
      cfg.dynamicSmemBytes = face_pair_smem_bytes(BC, max_dirs);
      cfg.stream = st;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, face_pair_kernel<BC>, g, kappa, S, tpl, items, faces, bnd, spin, status);
      return;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3(nitems);
  cfg.blockDim = dim3(kFaceThreads);
  cfg.dynamicSmemBytes = face_smem_bytes<R>(g.B, max_dirs);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, face_pass_kernel<R, BC>, g, kappa, S, tpl, items, faces, bnd, spin, status);
}

template <typename R, int MODE, int BC>
void cell_launch(const GridDims &g, const R *kappa, const R *S, const unsigned char *tpl, const int *order,
                 const R *faces, const R *bnd, R *I_out, R *M_out, R *E_out, R *f_out, void *emax_bits,
                 long long spin, int *status, const int *block_list, int nlist, cudaStream_t st) {
  const int parts = cell_parts(g.B);
  const int cpc = g.B * g.B * g.B / parts;
  const int threads = (cpc + 31) / 32 * 32;
  const int nblk = block_list ? nlist : g.nbx * g.nby * g.nbz;
  const int dt = cell_dir_tile<R>(g.B, g.dir_tile);
  cell_pass_kernel<R, MODE, BC><<<nblk * parts, threads, smem_bytes<R>(g.B, 2 * dt), st>>>(
      g, parts, dt, kappa, S, tpl, order, faces, bnd, I_out, M_out, E_out, f_out, emax_bits, spin, status,
      block_list);
}

template <int MODE, int BC>
void pair_launch(const GridDims &g, const float *kappa, const float *S, const unsigned char *tpl, const int *order,
                 const float *faces, const float *bnd, float *I_out, float *M_out, float *E_out, float *f_out,
                 void *emax_bits, long long spin, int *status, const int *block_list, int nlist, cudaStream_t st) {
  const int parts = BC * BC * BC / 2 / pair_threads(BC);
  const int nblk = block_list ? nlist : g.nbx * g.nby * g.nbz;
  const int dt = pair_dir_tile(BC, g.dir_tile);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // prologue overlaps the face pass's end
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3(nblk * parts);
  cfg.blockDim = dim3(pair_threads(BC));
  cfg.dynamicSmemBytes = pair_smem_bytes(BC, 2 * dt);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, cell_pair_kernel<MODE, BC>, g, parts, dt, kappa, S, tpl, order, faces, bnd, I_out, M_out,
                     E_out, f_out, emax_bits, spin, status, block_list);
}

template <typename R>
cudaError_t set_smem_attrs() {
  const int lim = (int)kSmemMax;
  const void *fns[] = {(const void *)face_pass_kernel<R, 8>,       (const void *)face_pass_kernel<R, 16>,
                       (const void *)face_pass_kernel<R, 0>,       (const void *)cell_pass_kernel<R, 0, 8>,
                       (const void *)cell_pass_kernel<R, 0, 16>,   (const void *)cell_pass_kernel<R, 0, 0>,
                       (const void *)cell_pass_kernel<R, 1, 8>,    (const void *)cell_pass_kernel<R, 1, 16>,
                       (const void *)cell_pass_kernel<R, 1, 0>,    (const void *)cell_pass_kernel<R, 2, 8>,
                       (const void *)cell_pass_kernel<R, 2, 16>,   (const void *)cell_pass_kernel<R, 2, 0>};
  for (const void *f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
  }
  const void *pfns[] = {(const void *)cell_pair_kernel<0, 8>,  (const void *)cell_pair_kernel<0, 16>,
                        (const void *)cell_pair_kernel<1, 8>,  (const void *)cell_pair_kernel<1, 16>,
                        (const void *)cell_pair_kernel<2, 8>,  (const void *)cell_pair_kernel<2, 16>,
                        (const void *)face_pair_kernel<8>,     (const void *)face_pair_kernel<16>};
  for (const void *f : pfns) {  // less their static shared memory
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448 - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

template <typename R>
cudaError_t launch_face_level(const GridDims &g, const R *kappa, const R *S, const unsigned char *tpl,
                              const FaceItem *items, int nitems, int max_dirs, R *faces, const R *bnd,
                              long long spin, int *status, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  if (g.B == 16) face_launch<R, 16>(g, kappa, S, tpl, items, nitems, max_dirs, faces, bnd, spin, status, st);
  else if (g.B == 8) face_launch<R, 8>(g, kappa, S, tpl, items, nitems, max_dirs, faces, bnd, spin, status, st);
  else face_launch<R, 0>(g, kappa, S, tpl, items, nitems, max_dirs, faces, bnd, spin, status, st);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cell_pass(const GridDims &g, int mode, const R *kappa, const R *S, const unsigned char *tpl,
                             const int *order, const R *faces, const R *bnd, R *I_out, R *M_out, R *E_out,
                             R *f_out, void *emax_bits, long long spin, int *status, cudaStream_t st,
                             const int *block_list, int nlist) {
  if (block_list && nlist <= 0) return cudaSuccess;
  if constexpr (sizeof(R) == sizeof(float)) {
    if (g.paired && (g.B == 16 || g.B == 8)) {
      const float *k = reinterpret_cast<const float *>(kappa), *s = reinterpret_cast<const float *>(S);
      const float *fc = reinterpret_cast<const float *>(faces), *bd = reinterpret_cast<const float *>(bnd);
      float *Io = reinterpret_cast<float *>(I_out), *Mo = reinterpret_cast<float *>(M_out);
      float *Eo = reinterpret_cast<float *>(E_out), *fo = reinterpret_cast<float *>(f_out);
      const int mode2 = mode == 0 ? (M_out ? 0 : 2) : 1;
#define VET_PAIR(MODE, BC) \
  pair_launch<MODE, BC>(g, k, s, tpl, order, fc, bd, Io, Mo, Eo, fo, emax_bits, spin, status, block_list, nlist, st)
      if (g.B == 16) {
        if (mode2 == 0) VET_PAIR(0, 16);
        else if (mode2 == 2) VET_PAIR(2, 16);
        else VET_PAIR(1, 16);
      } else {
        if (mode2 == 0) VET_PAIR(0, 8);
        else if (mode2 == 2) VET_PAIR(2, 8);
        else VET_PAIR(1, 8);
      }
#undef VET_PAIR
      return cudaGetLastError();
    }
  }
#define VET_CELL(MODE, BC)                                                                                  \
  cell_launch<R, MODE, BC>(g, kappa, S, tpl, order, faces, bnd, I_out, M_out, E_out, f_out, emax_bits, spin, \
                           status, block_list, nlist, st)
  if (mode == 0 && M_out) {
    if (g.B == 16) VET_CELL(0, 16);
    else if (g.B == 8) VET_CELL(0, 8);
    else VET_CELL(0, 0);
  } else if (mode == 0) {
    if (g.B == 16) VET_CELL(2, 16);
    else if (g.B == 8) VET_CELL(2, 8);
    else VET_CELL(2, 0);
  } else {
    if (g.B == 16) VET_CELL(1, 16);
    else if (g.B == 8) VET_CELL(1, 8);
    else VET_CELL(1, 0);
  }
#undef VET_CELL
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fill_boundary(const GridDims &g, const unsigned char *tpl, const R *Ib, R *bnd, cudaStream_t st) {
  fill_boundary_kernel<R><<<dim3(g.ndir, 6), 128, 0, st>>>(g, tpl, tpl_layout<R>(g.B).bytes, Ib, bnd);
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
cudaError_t launch_floor_fix_blocks(const GridDims &g, const int *block_list, int nlist, const R *E,
                                    const void *emax_bits, double floor_rel, R *f_out, cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  floor_fix_blocks_kernel<R><<<nlist, 256, 0, st>>>(g, block_list, E, emax_bits, floor_rel, f_out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_moments(long long ncell, int ndir, const R *I, const R *coef, R *M_out, cudaStream_t st) {
  const int threads = 256;
  // vector loads need every direction's row to start 16-byte aligned
  constexpr int VW = 16 / (int)sizeof(R);
  const bool vec = ncell % VW == 0 && (reinterpret_cast<uintptr_t>(I) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(M_out) & 15) == 0;
  const long long per = vec ? VW : 1;
  const long long blocks = ((ncell + per - 1) / per + threads - 1) / threads;
  if (blocks < 1) return cudaSuccess;
  if (vec)
    moments_kernel<R, VW><<<(unsigned)blocks, threads, 0, st>>>(ncell, ndir, I, coef, M_out);
  else
    moments_kernel<R, 1><<<(unsigned)blocks, threads, 0, st>>>(ncell, ndir, I, coef, M_out);
  return cudaGetLastError();
}

size_t pass_smem_bytes(int B, int dirs, bool fp64) {
  return fp64 ? face_smem_bytes<double>(B, dirs) : face_smem_bytes<float>(B, dirs);
}

int cell_tile_fit(int B, int want, bool fp64) {
  return fp64 ? cell_dir_tile<double>(B, want) : cell_dir_tile<float>(B, want);
}

size_t cell_smem_bytes(int B, int nslots, bool fp64) {
  return fp64 ? smem_bytes<double>(B, nslots) : smem_bytes<float>(B, nslots);
}

// Opt the shared-memory-heavy kernels in to the full 227 KB per CTA on the
// current device (the attribute is per device and function).
cudaError_t prepare_kernels() {
  cudaError_t e = set_smem_attrs<float>();
  if (e != cudaSuccess) return e;
  return set_smem_attrs<double>();
}

#define VET_INSTANTIATE(R)                                                                                   \
  template cudaError_t launch_face_level<R>(const GridDims &, const R *, const R *, const unsigned char *,   \
                                            const FaceItem *, int, int, R *, const R *, long long, int *,   \
                                            cudaStream_t);                                                   \
  template cudaError_t launch_cell_pass<R>(const GridDims &, int, const R *, const R *, const unsigned char *, \
                                           const int *, const R *, const R *, R *, R *, R *, R *, void *,    \
                                           long long, int *, cudaStream_t, const int *, int);                \
  template cudaError_t launch_floor_fix_blocks<R>(const GridDims &, const int *, int, const R *, const void *, \
                                                  double, R *, cudaStream_t);                                \
  template cudaError_t launch_fill_boundary<R>(const GridDims &, const unsigned char *, const R *, R *,      \
                                               cudaStream_t);                                                \
  template cudaError_t launch_floor_fix<R>(long long, const R *, long long, const void *, double, R *,     \
                                           cudaStream_t);                                                    \
  template cudaError_t launch_moments<R>(long long, int, const R *, const R *, R *, cudaStream_t);

VET_INSTANTIATE(float)
VET_INSTANTIATE(double)

}  // namespace vet
