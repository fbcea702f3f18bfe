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
#include <algorithm>
#include <cstddef>
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
//   thin (FP32: x < 1/4): base = I, w = -(1 - e^-x) = y q(y) with q of
//     degree 3 fitted for relative error by Lawson's iteratively reweighted
//     least squares (2.4e-7 in exact arithmetic, 3.4e-7 evaluated in FP32):
//     the other form would round S to its ulp before subtracting almost all
//     of it when S >> I, and 1 - e would cancel;
//   thick: base = S, w = e^-x from the MUFU (ex2.approx); here the first
//     form would cancel when I >> S.  Where S >> I the thick form's result
//     is about S (1 - e^-x), so the MUFU's relative error (1.5e-7, not
//     zero-mean) grows by e^-x / (1 - e^-x) <= 3.5 at x >= 1/4.
// The FMA pipe bounds the FP32 ray march, so the thin range is set to 1/4,
// where a cubic suffices (a quartic on x < 1/2 costs one more fused
// multiply-add per segment: 8% of the cell pass).  FP64: expm1 and exp2 of
// the CUDA math library in the same two forms, thin for x < 1/2.
constexpr float kQ3 = kThinQ3, kQ2 = kThinQ2, kQ1 = kThinQ1, kQ0 = kThinQ0;  // vet_internal.h
__device__ __forceinline__ float seg_weight(float y, bool &thin) {
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(y));
  float q = kQ3;
  q = fmaf(q, y, kQ2);
  q = fmaf(q, y, kQ1);
  q = fmaf(q, y, kQ0);
  thin = y > kThinY;
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
    const int q = w / NN, k = w - q * NN;
    const int j = nlive == 1 ? q : (nlive == 2 ? q >> 1 : (q * 21846) >> 16);
    const int ai = q - j * nlive;
    const Tpl<R> T(slots + sb * j, TL);
    const R *fin = reinterpret_cast<const R *>(slots + sb * j + TL.node_bytes);
    // the k-th node ray by length, as in the paired face pass
    int a = (live >> (2 * ai)) & 3, r = k;
    if (g.node_order) {
      const uint16_t *no = g.node_order + (size_t)(it.dir_begin + j) * (6 * NN);
      if (nlive == 3) {
        const int k3 = w - j * (3 * NN);
        const int code = __ldg(no + 3 * NN + ((j & 1) ? 3 * NN - 1 - k3 : k3));
        a = code / NN;
        r = code - a * NN;
      } else {
        r = __ldg(no + a * NN + ((q & 1) ? NN - 1 - k : k));
      }
    }
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
// in their own upwind frames both start at the same coordinates along every
// axis the direction crosses, leave through the same event with the same
// exit-table entries, and cross segments of the same lengths whose tile
// offsets are negatives of each other.  So one thread marches both in
// lockstep from one event list and one 16-byte load of the paired tile per
// step, with the two exponentials' arithmetic on packed FP32 pairs (f32x2);
// only the staged faces (and, along an axis the direction does not cross,
// the in-plane face coordinates) are per ray.  The lanes of a warp march
// aligned at the downwind end, as in the face pass, so that at each step they
// read one event and a brick of neighbouring entries.  The cell order lists
// the pairs (d, -d) consecutively; every staged tile holds whole pairs.
//
// Each thread owns one cell of the block's lower half and its mirror: for
// 16^3 blocks 1024 threads (one CTA per SM, whose 32 warps share one kappa/S
// tile and a deep ring of staged directions), for 8^3 blocks 256.  All
// shared-memory addressing is 32-bit (the state of a march is a handful of
// registers: the pair's intensities, the tile address of the start entries
// and the event index, which is the same for the whole warp).
__host__ __device__ constexpr int pair_threads(int B) { return B == 16 ? 1024 : 256; }
__host__ __device__ constexpr int pair_min_ctas(int B) { return B == 16 ? 1 : 4; }
constexpr int kPairStagesMax = 16;  // staging ring depth limit of the paired cell pass

// Shared-memory loads at 32-bit shared-window addresses.  volatile keeps
// them after the mbarrier waits that publish the staged data.
__device__ __forceinline__ uint4 lds_4x32(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ uint2 lds_2x32(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ float lds_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int lds_s16(uint32_t a) {
  int v;
  asm volatile("ld.shared.s16 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}


__device__ __forceinline__ float4 lds_f4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

// One segment of both rays of a mirrored pair (the update of segment() on
// packed FP32 pairs, f32x2).  ta: shared address of the paired tile entry
// (kappa, kappa', S, S') the primary ray crosses; len: the segment's scaled
// length.  Both forms are formed and each lane keeps the one that cannot
// cancel: thin  I + (I - S) * (-(1 - e^-x)),  thick  S + (I - S) e^-x.
__device__ __forceinline__ float2 step_pair(uint32_t ta, float len, float2 I) {
  const float4 q = lds_f4(ta);
  const float2 Y = __fmul2_rn(make_float2(q.x, q.y), make_float2(len, len));
  float e1, e2;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(Y.x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e2) : "f"(Y.y));
  float2 p = __ffma2_rn(make_float2(kQ3, kQ3), Y, make_float2(kQ2, kQ2));
  p = __ffma2_rn(p, Y, make_float2(kQ1, kQ1));
  p = __ffma2_rn(p, Y, make_float2(kQ0, kQ0));
  const float2 n = __fmul2_rn(p, Y);
  const bool t1 = Y.x > kThinY, t2 = Y.y > kThinY;
  // one FFMA2 on per-lane selected operands: the FMA pipe, not issue, bounds
  // this step (an FFMA2 of each form and a select of the results measured
  // 13% slower)
  return __ffma2_rn(__fadd2_rn(I, neg2(make_float2(q.z, q.w))), make_float2(t1 ? n.x : e1, t2 ? n.y : e2),
                    make_float2(t1 ? I.x : q.z, t2 ? I.y : q.w));
}

// The step of a lane that may be idle: an idle lane loads nothing and
// steps on zeros (kappa = 0: the thin form returns I exactly), so that a
// quarter-warp with no active lane issues no shared-memory wavefront.
__device__ __forceinline__ float2 step_pair_g(bool act, uint32_t ta, float len, float2 I) {
  float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
  asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n @p ld.shared.v4.f32 {%0, %1, %2, %3}, [%5];\n}\n"
               : "+f"(q.x), "+f"(q.y), "+f"(q.z), "+f"(q.w)
               : "r"((uint32_t)act), "r"(ta));
  const float2 Y = __fmul2_rn(make_float2(q.x, q.y), make_float2(len, len));
  float e1, e2;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(Y.x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e2) : "f"(Y.y));
  float2 p = __ffma2_rn(make_float2(kQ3, kQ3), Y, make_float2(kQ2, kQ2));
  p = __ffma2_rn(p, Y, make_float2(kQ1, kQ1));
  p = __ffma2_rn(p, Y, make_float2(kQ0, kQ0));
  const float2 n = __fmul2_rn(p, Y);
  const bool t1 = Y.x > kThinY, t2 = Y.y > kThinY;
  return __ffma2_rn(__fadd2_rn(I, neg2(make_float2(q.z, q.w))), make_float2(t1 ? n.x : e1, t2 ? n.y : e2),
                    make_float2(t1 ? I.x : q.z, t2 ? I.y : q.w));
}

// March of a mirrored ray pair: events at shared address ev (8 bytes each:
// scaled length, byte offset for 8-byte tile entries), primary start entry
// at t1.  The warp runs from its largest `last` down to event 0; a lane
// whose own ray is shorter reads the identity entry id (kappa = 0: the thin
// form returns I exactly) until the index reaches its `last`; below the
// warp's smallest `last` every lane marches.  After one step to an odd
// index, events are read in 16-byte pairs, four steps a trip, in both
// phases (the guarded phase while four or more of its steps remain).
__device__ __forceinline__ float2 march_pair(uint32_t t1, uint32_t id, uint32_t ev, int last, float2 I) {
  int e = __reduce_max_sync(0xffffffffu, last);
  const int wmin = __reduce_min_sync(0xffffffffu, last);
  if (e - wmin >= 4) {  // guarded steps four at a time on 16-byte event pairs
    if (!(e & 1)) {
      const float2 v = lds_f2(ev + 8 * e);
      I = step_pair(e <= last ? t1 + 2 * (int)__float_as_uint(v.y) : id, v.x, I);
      --e;
    }
    for (; e - wmin >= 4; e -= 4) {  // e - 3 > wmin >= 0
      const float4 a = lds_f4(ev + 8 * (e - 1));
      const float4 b = lds_f4(ev + 8 * (e - 3));
      I = step_pair(e <= last ? t1 + 2 * (int)__float_as_uint(a.w) : id, a.z, I);
      I = step_pair(e - 1 <= last ? t1 + 2 * (int)__float_as_uint(a.y) : id, a.x, I);
      I = step_pair(e - 2 <= last ? t1 + 2 * (int)__float_as_uint(b.w) : id, b.z, I);
      I = step_pair(e - 3 <= last ? t1 + 2 * (int)__float_as_uint(b.y) : id, b.x, I);
    }
  }
  for (; e > wmin; --e) {
    const float2 v = lds_f2(ev + 8 * e);
    I = step_pair(e <= last ? t1 + 2 * (int)__float_as_uint(v.y) : id, v.x, I);
  }
  if (e >= 0 && !(e & 1)) {  // to an odd index: event pairs (e - 1, e) are 16-byte aligned
    const float2 v = lds_f2(ev + 8 * e);
    I = step_pair(t1 + 2 * (int)__float_as_uint(v.y), v.x, I);
    --e;
  }
  for (; e >= 3; e -= 4) {
    const float4 a = lds_f4(ev + 8 * (e - 1));
    const float4 b = lds_f4(ev + 8 * (e - 3));
    I = step_pair(t1 + 2 * (int)__float_as_uint(a.w), a.z, I);
    I = step_pair(t1 + 2 * (int)__float_as_uint(a.y), a.x, I);
    I = step_pair(t1 + 2 * (int)__float_as_uint(b.w), b.z, I);
    I = step_pair(t1 + 2 * (int)__float_as_uint(b.y), b.x, I);
  }
  if (e == 1) {
    const float4 a = lds_f4(ev);
    I = step_pair(t1 + 2 * (int)__float_as_uint(a.w), a.z, I);
    I = step_pair(t1 + 2 * (int)__float_as_uint(a.y), a.x, I);
  }
  return I;
}

// One ray on its own template (a pair whose templates are not exact
// mirrors), reading its own (kappa, S) = (.x, .z) of the paired entries.
__device__ __forceinline__ float march_one(uint32_t t, uint32_t ev, int last, float I) {
  for (int e = last; e >= 0; --e) {
    const uint2 v = lds_2x32(ev + 8 * e);
    const uint4 q = lds_4x32(t + 2 * (int)v.y);
    const float y = __uint_as_float(q.x) * __uint_as_float(v.x);
    float ex;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex) : "f"(y));
    float p = kQ3;
    p = fmaf(p, y, kQ2);
    p = fmaf(p, y, kQ1);
    p = fmaf(p, y, kQ0);
    const float s = __uint_as_float(q.z), D = I - s;
    I = y > kThinY ? fmaf(D, p * y, I) : fmaf(D, ex, s);
  }
  return I;
}

// Paired-cell-pass slot: the template head, the template's cell-ray parts,
// then the three incoming faces (offsets in bytes from the slot's start).
struct CellSlot {
  int cev, cpos, ck, cw, faces, bytes;
};
__host__ __device__ inline CellSlot cell_slot(int B) {
  const TplLayout L = tpl_layout<float>(B);
  const int shift = L.cev - L.nev;  // the node-ray parts are not staged
  CellSlot s;
  s.cev = L.cev - shift;
  s.cpos = L.cpos - shift;
  s.ck = L.ck - shift;
  s.cw = L.cw - shift;
  s.faces = L.bytes - shift;
  s.bytes = s.faces + (int)faces_bytes<float>(B);
  return s;
}

// Issues the bulk copies of one paired-cell-pass slot (thread 0): the
// head, the cell-ray parts and the three incoming faces of direction d.
__device__ __forceinline__ void issue_cell_slot(unsigned char *slot, const GridDims &g, const TplLayout &TL,
                                                const CellSlot &CS, int bx, int by, int bz, int d, int sgn_bits,
                                                const unsigned char *__restrict__ tpl_g, const float *__restrict__ faces,
                                                const float *__restrict__ bnd, uint64_t *bar) {
  const unsigned char *src = tpl_g + (size_t)d * TL.bytes;
  bulk_g2s(slot, src, (uint32_t)TL.nev, bar);
  bulk_g2s(slot + CS.cev, src + TL.cev, (uint32_t)(TL.bytes - TL.cev), bar);
  const int nblk = g.nbx * g.nby * g.nbz;
  const uint32_t fb = (uint32_t)(g.fstride * sizeof(float));
  const int b3[3] = {bx, by, bz};
  const int nb3[3] = {g.nbx, g.nby, g.nbz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int s = (sgn_bits >> a) & 1 ? -1 : 1;
    int nb[3] = {b3[0], b3[1], b3[2]};
    nb[a] -= s;
    const float *fsrc;
    if (nb[a] < 0 || nb[a] >= nb3[a]) {
      fsrc = bnd + ((long long)(2 * a + (s > 0 ? 0 : 1)) * g.ndir + d) * g.fstride;
    } else {
      const long long nid = ((long long)nb[2] * g.nby + nb[1]) * g.nbx + nb[0];
      fsrc = faces + (((long long)d * nblk + nid) * 3 + a) * g.fstride;
    }
    bulk_g2s(slot + CS.faces + a * fb, fsrc, fb, bar);
  }
}

// Non-blocking test of a phase (no suspension).
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  return done != 0;
}

// One potentially blocking poll: the hardware may suspend the thread for a
// short while when the phase is not complete.
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait of one thread: a test, then up to limit - 1 blocking polls,
// four per trip of a 32-bit counter, so that a waiting warp spends few issue
// slots on the loop itself (a loop of 64-bit counters, a sleep schedule and
// single polls took a third of the cell pass's issued instructions).
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t a, uint32_t parity, long long limit) {
  if (limit < 1) return false;
  if (mbar_test(a, parity)) return true;
  int n = limit - 1 > 0x7ffffff0LL ? 0x7ffffff0 : (int)(limit - 1);
  for (; n >= 4; n -= 4)
    if (mbar_try(a, parity) || mbar_try(a, parity) || mbar_try(a, parity) || mbar_try(a, parity)) return true;
  for (; n > 0; --n)
    if (mbar_try(a, parity)) return true;
  return false;
}

// The same wait taken by every lane of a converged warp, with a warp-wide
// verdict (the warp proceeds only if every lane saw the phase complete).
__device__ __forceinline__ bool mbar_wait_sleep_warp(uint32_t a, uint32_t parity, long long limit, int *status,
                                                     int code) {
  const bool done = mbar_wait_sleep(a, parity, limit);
  if (__all_sync(0xffffffffu, done)) return true;
  if ((threadIdx.x & 31) == 0) atomicOr(status, code);
  return false;
}

// Dynamic shared memory of a paired cell-pass CTA: the paired tile and
// `nslots` staged directions.
__host__ __device__ inline size_t pair_smem_bytes(int B, int nslots) {
  return align16(sizeof(float4) * (size_t)cell_tile(B).elems) + (size_t)nslots * cell_slot(B).bytes;
}

// Paired tile of the cell pass: entry p holds (kappa(p), kappa(p'), S(p),
// S(p')), p' the point-mirrored cell of the same block; every thread issues
// its global loads before its stores.
template <int BC, int NT>
__device__ __forceinline__ void load_tile_pair(float4 *tile, TileShape ts, const GridDims &g, int bx, int by, int bz,
                                               const float *__restrict__ kappa, const float *__restrict__ S) {
  constexpr int B = BC, B2 = B * B, K = B2 * B / NT;
  static_assert(B2 * B % NT == 0, "tile cells must divide evenly over the threads");
  float4 v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = (int)threadIdx.x + k * NT, x = i % B, y = (i / B) % B, z = i / B2;
    const long long gi = ((long long)(bz * B + z) * g.ny + (by * B + y)) * g.nx + (bx * B + x);
    const long long gm = ((long long)(bz * B + B - 1 - z) * g.ny + (by * B + B - 1 - y)) * g.nx + (bx * B + B - 1 - x);
    v[k] = make_float4(kappa[gi], kappa[gm], S[gi], S[gm]);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = (int)threadIdx.x + k * NT, x = i % B, y = (i / B) % B, z = i / B2;
    tile[x + ts.sy * y + ts.sz * z] = v[k];
  }
}

// Compensated (Kahan) accumulation of t = c * x into s on packed pairs; nc
// holds the negated compensation.
__device__ __forceinline__ void kahan2(float2 &s, float2 &nc, float2 c, float2 x) {
  const float2 y = __ffma2_rn(c, x, nc);
  const float2 t = __fadd2_rn(s, y);
  nc = __fadd2_rn(y, neg2(__fadd2_rn(t, neg2(s))));
  s = t;
}

// the head fields the paired cell pass reads at fixed offsets
static_assert(offsetof(TplHead<float>, sgn) == 16 && offsetof(TplHead<float>, ext) == 28 &&
                  offsetof(TplHead<float>, mirror) == 32 && offsetof(TplHead<float>, cp) % 16 == 0,
              "TplHead<float> layout");

template <int MODE, int BC, bool MERGED>
__global__ void __launch_bounds__(pair_threads(BC), pair_min_ctas(BC))
    cell_pair_kernel(GridDims g_arg, int parts, int dt, int nstage, const float *__restrict__ kappa_arg,
                     const float *__restrict__ S_arg, const unsigned char *__restrict__ tpl_arg,
                     const int *__restrict__ order_arg, const float *__restrict__ faces_arg,
                     const float *__restrict__ bnd_arg, float *__restrict__ I_out, float *__restrict__ M_arg,
                     float *__restrict__ E_arg, float *__restrict__ f_arg, void *emax_arg, long long spin_limit,
                     int *status_arg, const int *__restrict__ block_list, int nfull, int ksplit,
                     float *__restrict__ split_part, int *__restrict__ split_count,
                     const CellGrid *__restrict__ grids, const int2 *__restrict__ items) {
  constexpr int B = BC, B2 = B * B, NT = pair_threads(BC);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kPairStagesMax], empty[kPairStagesMax];
  constexpr int kOrdMax = 1024;  // direction sets up to nside = 8 keep their order in shared memory
  __shared__ int s_ord[kOrdMax];
  // a merged launch (several grids of one block edge) takes its grid from the
  // work item's entry of `grids`; a single grid's launch from the arguments
  const CellGrid *gd = nullptr;
  if constexpr (MERGED) gd = grids + items[(int)blockIdx.x / parts].x;
  const GridDims g = MERGED ? gd->g : g_arg;
  const float *__restrict__ kappa = MERGED ? gd->kappa : kappa_arg;
  const float *__restrict__ S = MERGED ? gd->S : S_arg;
  const unsigned char *__restrict__ tpl_g = MERGED ? gd->tpl : tpl_arg;
  const int *__restrict__ order = MERGED ? gd->order : order_arg;
  const float *__restrict__ faces = MERGED ? gd->faces : faces_arg;
  const float *__restrict__ bnd = MERGED ? gd->bnd : bnd_arg;
  float *__restrict__ M_out = MERGED ? gd->M_out : M_arg;
  float *__restrict__ E_out = MERGED ? gd->E_out : E_arg;
  float *__restrict__ f_out = MERGED ? gd->f_out : f_arg;
  void *emax_bits = MERGED ? gd->emax_bits : emax_arg;
  int *status = MERGED ? gd->status : status_arg;
  const bool ord_smem = g.ndir <= kOrdMax;
  const TileShape ts = cell_tile(B);
  const TplLayout TL = tpl_layout<float>(B);
  const CellSlot CS = cell_slot(B);
  const int fstride = g.fstride;
  float4 *tile = reinterpret_cast<float4 *>(smem);
  unsigned char *ring = smem + align16(sizeof(float4) * (size_t)ts.elems);
  const uint32_t ring_s = smem_u32(ring);
  const size_t stage_bytes = (size_t)dt * CS.bytes;
  // the parts of a block are neighbours in launch order, so that the second
  // finds the block's staged faces still in L2 (running every block's part 1
  // before any part 0 read them from DRAM twice: 736 instead of 361 MB)
  // past nfull, ksplit consecutive CTAs share one work item (slot), each a
  // contiguous run of its direction tiles (the tail split)
  int cta = (int)blockIdx.x, share = 0, slot = -1;
  if (ksplit > 1 && cta >= nfull) {
    slot = (cta - nfull) / ksplit;
    share = cta - nfull - slot * ksplit;
    cta = nfull + slot;
  }
  const int item = cta / parts, part = parts - 1 - (cta - item * parts);
  const int blk = MERGED ? items[item].y : (block_list ? block_list[item] : item);
  const int bx = blk % g.nbx, by = (blk / g.nbx) % g.nby, bz = blk / (g.nbx * g.nby);
  constexpr int nwarps = NT / 32;
  const int ntiles_all = (g.ndir + dt - 1) / dt, nshares = slot >= 0 ? ksplit : 1;
  const int tile0 = share * ntiles_all / nshares, ntiles = (share + 1) * ntiles_all / nshares - tile0;
  // producer state, meaningful in thread 0 only; tiles counted from tile0
  int issued = 0, consumed = 0;
  auto issue_tile = [&](int t) {
    const int s = t % nstage, d0 = (tile0 + t) * dt, nd = min(dt, g.ndir - d0);
    unsigned char *buf = ring + (size_t)s * stage_bytes;
    mbar_expect_tx(&full[s], (uint32_t)(CS.bytes * nd));
    for (int j = 0; j < nd; ++j) {
      const int v = (ord_smem && t >= nstage) ? s_ord[d0 + j] : order[d0 + j];
      issue_cell_slot(buf + (size_t)CS.bytes * j, g, TL, CS, bx, by, bz, order_dir(v), (v >> 16) & 7, tpl_g, faces,
                      bnd, &full[s]);
    }
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstage; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], nwarps);
    }
    mbar_fence_init();
    griddep_wait();  // the faces are the face pass's output
    while (issued < ntiles && issued < nstage) issue_tile(issued++);
  }
  if (ord_smem)
    for (int i = threadIdx.x; i < g.ndir; i += NT) s_ord[i] = order[i];
  load_tile_pair<BC, NT>(tile, ts, g, bx, by, bz, kappa, S);
  if (threadIdx.x == 0) tile[B] = make_float4(0.f, 0.f, 0.f, 0.f);  // identity entry (padding, x = B)
  __syncthreads();

  // this thread's lower-half cell (z < B/2): 4 x 4 x 2 bricks, warp-major
  const int q = part * NT + (int)threadIdx.x;
  const int qb = q >> 5, ln = q & 31;
  const int cx = 4 * (qb % (B / 4)) + (ln & 3);
  const int cy = 4 * ((qb / (B / 4)) % (B / 4)) + ((ln >> 2) & 3);
  // layer pair lp holds z = 2 lp, 2 lp + 1 of the lower half; with two parts
  // of a 16^3 block, part 0 takes layer pairs 0 and 3 and part 1 takes 1 and
  // 2 (85e3 and 89e3 warp steps over 192 directions, where z-order parts
  // differ by 15%), so that the CTAs of a wave carry about equal work
  int lp = qb / (B2 / 16);
  if (B == 16 && parts == 2) lp = (0x2130 >> (4 * lp)) & 15;
  const int cz = 2 * lp + (ln >> 4);
  const int mx = B - 1 - cx, my = B - 1 - cy, mz = B - 1 - cz;  // the mirror cell
  const uint32_t tile_s = smem_u32(tile);
  const uint32_t t1 = tile_s + 16u * (uint32_t)(cx + ts.sy * cy + ts.sz * cz);
  const uint32_t t2 = tile_s + 16u * (uint32_t)(mx + ts.sy * my + ts.sz * mz);
  const long long gc1 = ((long long)(bz * B + cz) * g.ny + (by * B + cy)) * g.nx + (bx * B + cx);
  const long long gc2 = ((long long)(bz * B + mz) * g.ny + (by * B + my)) * g.nx + (bx * B + mx);
  constexpr bool kWantF = MODE == 0;
  // moments of (c, c') as packed pairs: E, Fx, Fy, Fz, Pxx, Pyy, Pzz, Pxy,
  // Pxz, Pyz; compensated E and Pii (nc: their negated compensations), which
  // a staged tile's pairs add into plain partial sums pk first, folded into
  // the compensated sums once per tile (fewer f32x2 operations and fewer
  // register moves than a compensated addition per pair)
  float2 mom[10], nc[4];
#pragma unroll
  for (int m = 0; m < 10; ++m) mom[m] = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < 4; ++m) nc[m] = make_float2(0.f, 0.f);
  float2 pk[4];  // plain partial sums of the compensated moments over one tile
#pragma unroll
  for (int m = 0; m < 4; ++m) pk[m] = make_float2(0.f, 0.f);
  // a tile padding entry (x = B) set to zero: the identity segment
  const uint32_t id_s = tile_s + 16u * (uint32_t)B;
  constexpr int W = B + 2;
  const uint32_t fW = 4u * W;

  // Exit lookup and entry value of the ray(s) of one march: primary slot ps
  // (its template), upwind-frame coordinates l0..l2; returns the pair of
  // entry intensities from faces f1 (primary) and f2 (the pair's second ray).
  auto entry = [&](uint32_t ps, int l0, int l1, int l2, uint32_t f1, uint32_t f2, int &last) -> float2 {
    const int p0 = lds_s16(ps + CS.cpos + 2 * l0), p1 = lds_s16(ps + CS.cpos + 2 * (B + l1)),
              p2 = lds_s16(ps + CS.cpos + 2 * (2 * B + l2));
    int ae = 0, la = l0, lb = l1, lc = l2;
    last = p0;
    if (p1 < last) { last = p1; ae = 1; la = l1; lb = l0; }
    if (p2 < last) { last = p2; ae = 2; la = l2; lb = l0; lc = l1; }
    const int row = (ae * 2) * B + la;
    const int kb = lds_s16(ps + CS.ck + 2 * row), kc = lds_s16(ps + CS.ck + 2 * (row + B));
    const uint2 ub = lds_2x32(ps + CS.cw + 8 * row), uc = lds_2x32(ps + CS.cw + 8 * (row + B));
    const float wbx = __uint_as_float(ub.x), wby = __uint_as_float(ub.y);
    const float wcx = __uint_as_float(uc.x), wcy = __uint_as_float(uc.y);
    const int ib = max(lb + kb, 0), ic = max(lc + kc, 0);
    const uint32_t fo = 4u * (uint32_t)(ae * fstride + ib * W + ic);
    const uint32_t a1 = f1 + fo, a2 = f2 + fo;
    const float I1 = wby * (wcy * lds_f32(a1) + wcx * lds_f32(a1 + 4)) +
                     wbx * (wcy * lds_f32(a1 + fW) + wcx * lds_f32(a1 + fW + 4));
    const float I2 = wby * (wcy * lds_f32(a2) + wcx * lds_f32(a2 + 4)) +
                     wbx * (wcy * lds_f32(a2 + fW) + wcx * lds_f32(a2 + fW + 4));
    return make_float2(I1, I2);
  };
  // one ray of a pair that is not an exact mirror image: its own template
  // (slot ps, signs sg), start cell (x, y, z), entry face f
  auto single = [&](uint32_t ps, uint4 hd, int x, int y, int z, uint32_t tstart) -> float {
    const int l0 = (int)hd.x > 0 ? x : B - 1 - x;
    const int l1 = (int)hd.y > 0 ? y : B - 1 - y;
    const int l2 = (int)hd.z > 0 ? z : B - 1 - z;
    int last;
    const float2 Iin = entry(ps, l0, l1, l2, ps + CS.faces, ps + CS.faces, last);
    return march_one(tstart, ps + CS.cev, last, Iin.x);
  };

  bool ok = true;
  const uint32_t full_s = smem_u32(full), empty_s = smem_u32(empty);
  for (int t = 0; t < ntiles && ok; ++t) {
    const int st = t % nstage;
    const uint32_t ph = (uint32_t)((t / nstage) & 1);
    if (threadIdx.x < 32) {  // warp 0: thread 0 makes sure tile t is in flight
      int pok = 1;
      if (threadIdx.x == 0) {
        // its stage must have been released by every warp for tile t - nstage
        while (pok && issued <= t) {
          pok = mbar_wait_sleep(empty_s + 8 * (issued % nstage), (uint32_t)(((issued / nstage) - 1) & 1),
                                spin_limit);
          if (pok) issue_tile(issued++);
          else atomicOr(status, 4);
        }
      }
      if (!__shfl_sync(0xffffffffu, pok, 0)) { ok = false; break; }
    }
    if (!mbar_wait_sleep_warp(full_s + 8 * st, ph, spin_limit, status, 2)) { ok = false; break; }
    if (threadIdx.x == 0) consumed = t + 1;
    const int nd = min(dt, g.ndir - (tile0 + t) * dt);
    const uint32_t buf = ring_s + (uint32_t)(st * stage_bytes);
    for (int j = 0; j < nd; j += 2) {  // the antipodal pair (j, j + 1)
      const uint32_t sa = buf + (uint32_t)(CS.bytes * j), sb = sa + (uint32_t)CS.bytes;
      const uint4 ha = lds_4x32(sa + 16), hb = lds_4x32(sb + 16);  // (sgn0, sgn1, sgn2, ext)
      const int mirror = (int)lds_2x32(sa + 32).x;
      float2 m1, m2;  // m1 = (I(c, d), I(c', -d)), m2 = (I(c, -d), I(c', d))
      if (mirror) {
        // upwind-frame coordinates of c in the primary direction; the mirror
        // cell in the antipode has the same ones (each flips to B - 1 - c)
        int last;
        {
          const int l0 = (int)ha.x > 0 ? cx : mx, l1 = (int)ha.y > 0 ? cy : my, l2 = (int)ha.z > 0 ? cz : mz;
          const float2 Iin = entry(sa, l0, l1, l2, sa + CS.faces, sb + CS.faces, last);
          m1 = march_pair(t1, id_s, sa + CS.cev, last, Iin);
        }
        {
          const int l0 = (int)hb.x > 0 ? cx : mx, l1 = (int)hb.y > 0 ? cy : my, l2 = (int)hb.z > 0 ? cz : mz;
          const float2 Iin = entry(sb, l0, l1, l2, sb + CS.faces, sa + CS.faces, last);
          m2 = march_pair(t1, id_s, sb + CS.cev, last, Iin);
        }
      } else {
        // the pair's templates differ (near-tied plane crossings ordered
        // differently): each ray follows its own direction's template
        m1 = make_float2(single(sa, ha, cx, cy, cz, t1), single(sb, hb, mx, my, mz, t2));
        m2 = make_float2(single(sb, hb, cx, cy, cz, t1), single(sa, ha, mx, my, mz, t2));
      }
      if (MODE == 1) {
        I_out[(long long)ha.w * g.ncell + gc1] = m1.x;
        I_out[(long long)hb.w * g.ncell + gc2] = m1.y;
        I_out[(long long)hb.w * g.ncell + gc1] = m2.x;
        I_out[(long long)ha.w * g.ncell + gc2] = m2.y;
      } else {
        // E and P take I(d) + I(-d), F takes I(d) - I(-d), with the primary
        // direction's coefficient pairs
        const float2 sum = __fadd2_rn(m1, m2), dif = __fadd2_rn(m1, neg2(m2));
        const uint32_t cpa = sa + (uint32_t)offsetof(TplHead<float>, cp);
        const float4 c01 = lds_f4(cpa), c23 = lds_f4(cpa + 16), c45 = lds_f4(cpa + 32), c67 = lds_f4(cpa + 48),
                     c89 = lds_f4(cpa + 64);
        pk[0] = __ffma2_rn(make_float2(c01.x, c01.y), sum, pk[0]);
        if (kWantF) {
          mom[1] = __ffma2_rn(make_float2(c01.z, c01.w), dif, mom[1]);
          mom[2] = __ffma2_rn(make_float2(c23.x, c23.y), dif, mom[2]);
          mom[3] = __ffma2_rn(make_float2(c23.z, c23.w), dif, mom[3]);
        }
        pk[1] = __ffma2_rn(make_float2(c45.x, c45.y), sum, pk[1]);
        pk[2] = __ffma2_rn(make_float2(c45.z, c45.w), sum, pk[2]);
        pk[3] = __ffma2_rn(make_float2(c67.x, c67.y), sum, pk[3]);
        mom[7] = __ffma2_rn(make_float2(c67.z, c67.w), sum, mom[7]);
        mom[8] = __ffma2_rn(make_float2(c89.x, c89.y), sum, mom[8]);
        mom[9] = __ffma2_rn(make_float2(c89.z, c89.w), sum, mom[9]);
      }
    }
    if (MODE != 1) {  // the tile's plain partial sums into the compensated ones
      const float2 one = make_float2(1.f, 1.f);
      kahan2(mom[0], nc[0], one, pk[0]);
      kahan2(mom[4], nc[1], one, pk[1]);
      kahan2(mom[5], nc[2], one, pk[2]);
      kahan2(mom[6], nc[3], one, pk[3]);
#pragma unroll
      for (int m = 0; m < 4; ++m) pk[m] = make_float2(0.f, 0.f);
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[st]);
    if (threadIdx.x == 0) {
      // refill every stage the other warps have released, without waiting
      while (issued < ntiles && issued <= t + nstage &&
             mbar_test(empty_s + 8 * (issued % nstage), (uint32_t)(((issued / nstage) - 1) & 1)))
        issue_tile(issued++);
    }
  }
  if (threadIdx.x == 0) {
    for (int t = consumed; t < issued; ++t)
      if (!mbar_wait_sleep(full_s + 8 * (t % nstage), (uint32_t)((t / nstage) & 1), kDrainPolls)) atomicOr(status, 8);
  }
  if (MODE != 1 && slot >= 0) {
    // one share of a split work item: its partial sums go to the slot's
    // scratch, and the share that finishes last adds the others' (the
    // compensated sums as compensated sums) and writes the outputs
    constexpr int kVals = 28;
    __shared__ int s_last;
    float *mine = split_part + ((size_t)slot * ksplit + share) * kVals * NT + threadIdx.x;
#pragma unroll
    for (int m = 0; m < 10; ++m) {
      mine[(2 * m) * NT] = mom[m].x;
      mine[(2 * m + 1) * NT] = mom[m].y;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      mine[(20 + 2 * m) * NT] = nc[m].x;
      mine[(21 + 2 * m) * NT] = nc[m].y;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(split_count + slot, 1) == ksplit - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const float2 one = make_float2(1.f, 1.f);
    for (int r = 0; r < ksplit; ++r) {
      if (r == share) continue;
      const float *other = split_part + ((size_t)slot * ksplit + r) * kVals * NT + threadIdx.x;
      float2 pm[10], pn[4];
#pragma unroll
      for (int m = 0; m < 10; ++m) pm[m] = make_float2(__ldcg(other + (2 * m) * NT), __ldcg(other + (2 * m + 1) * NT));
#pragma unroll
      for (int m = 0; m < 4; ++m) pn[m] = make_float2(__ldcg(other + (20 + 2 * m) * NT), __ldcg(other + (21 + 2 * m) * NT));
      nc[0] = __fadd2_rn(nc[0], pn[0]);
      kahan2(mom[0], nc[0], one, pm[0]);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        nc[1 + m] = __fadd2_rn(nc[1 + m], pn[1 + m]);
        kahan2(mom[4 + m], nc[1 + m], one, pm[4 + m]);
      }
#pragma unroll
      for (int m = 1; m < 4; ++m) mom[m] = __fadd2_rn(mom[m], pm[m]);
#pragma unroll
      for (int m = 7; m < 10; ++m) mom[m] = __fadd2_rn(mom[m], pm[m]);
    }
    if (threadIdx.x == 0) split_count[slot] = 0;  // ready for the next call
  }
  if (MODE != 1) {
    // Outputs: staged in the (now idle) staging ring as [value][z slot][y][x]
    // over the CTA's 2L layers, then written row by row, so that every
    // warp writes runs of B consecutive cells of a component (a host-mapped
    // output then crosses the host link in whole runs, not 16-byte pieces)
    constexpr int L = NT / B2, CELLS = 2 * NT, NV = kWantF ? 16 : 7, NM = kWantF ? 10 : 1;
    const bool staged = (size_t)nstage * stage_bytes >= sizeof(float) * NV * CELLS;
    float emax = 0.f;
    if (__syncthreads_and(ok)) {  // also: every warp is done with the ring
      float Ms[2][10];
#pragma unroll
      for (int m = 0; m < 10; ++m) {
        Ms[0][m] = mom[m].x;
        Ms[1][m] = mom[m].y;
      }
      float *st = reinterpret_cast<float *>(ring);
      const int zs = 2 * (qb / (B2 / 16) - part * (L / 2)) + (ln >> 4);  // the lower cell's z slot
      const int li[2] = {(zs * B + cy) * B + cx, ((L + zs) * B + my) * B + mx};
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const long long gc = r ? gc2 : gc1;
        const float E = Ms[r][0];
        float v[NV];
        if (kWantF) {
#pragma unroll
          for (int m = 0; m < 10; ++m) v[m] = Ms[r][m];
        } else {
          v[0] = E;
        }
#pragma unroll
        for (int m = 0; m < 6; ++m)  // correctly rounded, as in cell_pass_kernel
          v[NM + m] = E > 0.f ? Ms[r][4 + m] / E : (m < 3 ? 1.f / 3.f : 0.f);
        if (staged) {
#pragma unroll
          for (int m = 0; m < NV; ++m) st[m * CELLS + li[r]] = v[m];
        } else {
#pragma unroll
          for (int m = 0; m < NV; ++m) {
            float *dst = m < NM ? (kWantF ? M_out + m * g.ncell : E_out) : f_out + (m - NM) * g.ncell;
            dst[gc] = v[m];
          }
        }
        emax = fmaxf(emax, E);
      }
      if (staged) {
        __syncthreads();
        for (int i = threadIdx.x; i < CELLS; i += NT) {
          const int zsl = i / B2, y = (i / B) % B, x = i % B, zl = zsl < L ? zsl : zsl - L;
          int lp = part * (L / 2) + (zl >> 1);
          if (B == 16 && parts == 2) lp = (0x2130 >> (4 * lp)) & 15;
          const int z = zsl < L ? 2 * lp + (zl & 1) : B - 1 - (2 * lp + (zl & 1));
          const long long gi = ((long long)(bz * B + z) * g.ny + (by * B + y)) * g.nx + (bx * B + x);
#pragma unroll
          for (int m = 0; m < NV; ++m) {
            float *dst = m < NM ? (kWantF ? M_out + m * g.ncell : E_out) : f_out + (m - NM) * g.ncell;
            dst[gi] = st[m * CELLS + i];
          }
        }
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
  if (threadIdx.x == 0) tile[B] = make_float4(0.f, 0.f, 0.f, 0.f);  // identity entry (padding, x = B)
  __syncthreads();
  if (!mbar_wait_sleep_warp(smem_u32(&full), 0, spin_limit, status, 1)) {
    if (threadIdx.x == 0 && !mbar_wait_sleep(smem_u32(&full), 0, kDrainPolls)) atomicOr(status, 8);
    return;
  }
  const uint32_t tile_s = smem_u32(tile), id_s = tile_s + 16u * (uint32_t)B;
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
  const uint32_t slots_s = smem_u32(slots);
  for (int w0 = (int)threadIdx.x & ~31; w0 < total; w0 += blockDim.x) {
    const int wr = w0 + ((int)threadIdx.x & 31);
    const bool act = wr < total;
    const int w = act ? wr : total - 1;
    const int q = w / NN, k = w - q * NN;
    const int j = nlive == 1 ? q : (nlive == 2 ? q >> 1 : (q * 21846) >> 16);
    const int ai = q - j * nlive;
    // 32-bit shared addresses of the slot's template parts and both rays'
    // incoming faces
    const uint32_t ps = slots_s + (uint32_t)(sb * j);
    const uint32_t f1 = ps + (uint32_t)TL.node_bytes, f2 = slots_s + (uint32_t)(sb * cnt + fb3 * j);
    // the k-th node ray by length: of the face, or where all three faces
    // are computed, of the three merged; every other face (or direction)
    // of the item taken from its longest ray down, so that a warp that
    // straddles two joins rays of similar length too
    int a = (live >> (2 * ai)) & 3, r = k;
    if (g.node_order) {
      const uint16_t *no = g.node_order + (size_t)(it.dir_begin + j) * (6 * NN);
      if (nlive == 3) {
        const int k3 = w - j * (3 * NN);
        const int code = __ldg(no + 3 * NN + ((j & 1) ? 3 * NN - 1 - k3 : k3));
        a = code / NN;
        r = code - a * NN;
      } else {
        r = __ldg(no + a * NN + ((q & 1) ? NN - 1 - k : k));
      }
    }
    const int ub = r / N1, uc = r - ub * N1;
    const int L0 = a == 0 ? B : ub;
    const int L1 = a == 1 ? B : (a == 0 ? ub : uc);
    const int L2 = a == 2 ? B : uc;
    const uint32_t pp = ps + (uint32_t)TL.npos;
    const int p0 = lds_s16(pp + 2 * L0), p1 = lds_s16(pp + 2 * (N1 + L1)), p2 = lds_s16(pp + 2 * (2 * N1 + L2));
    int last = p0, ae = 0, la = L0, lb = L1, lc = L2;
    if (p1 < last) { last = p1; ae = 1; la = L1; lb = L0; }
    if (p2 < last) { last = p2; ae = 2; la = L2; lb = L0; lc = L1; }
    const int row = (ae * 2) * N1 + la;
    const int kb = lds_s16(ps + TL.nk + 2 * row), kc = lds_s16(ps + TL.nk + 2 * (row + N1));
    const uint2 wbu = lds_2x32(ps + TL.nw + 8 * row), wcu = lds_2x32(ps + TL.nw + 8 * (row + N1));
    const float wbx = __uint_as_float(wbu.x), wby = __uint_as_float(wbu.y);
    const float wcx = __uint_as_float(wcu.x), wcy = __uint_as_float(wcu.y);
    const int ib = max(lb + kb, 0), ic = max(lc + kc, 0);
    const uint32_t fo = 4u * (uint32_t)(ae * g.fstride + ib * W + ic);
    const uint32_t a1 = f1 + fo, a2 = f2 + fo;
    float2 I = make_float2(wby * (wcy * lds_f32(a1) + wcx * lds_f32(a1 + 4)) +
                               wbx * (wcy * lds_f32(a1 + 4 * W) + wcx * lds_f32(a1 + 4 * W + 4)),
                           wby * (wcy * lds_f32(a2) + wcx * lds_f32(a2 + 4)) +
                               wbx * (wcy * lds_f32(a2 + 4 * W) + wcx * lds_f32(a2 + 4 * W + 4)));
    if (!act) last = -1;
    // lockstep aligned at the downwind end, as in the unpaired face pass; a
    // lane whose own ray is shorter steps on zeros without a load (a
    // quarter-warp of such lanes costs no shared-memory wavefront); events
    // four at a time in 16-byte pairs
    const int wl = __reduce_max_sync(0xffffffffu, last);
    if (wl >= 0) {
      const uint4 hd = lds_4x32(ps + 16);  // (sgn0, sgn1, sgn2, ext)
      const int c0 = (int)hd.x > 0 ? L0 - 1 : B - L0;
      const int c1 = (int)hd.y > 0 ? L1 - 1 : B - L1;
      const int c2 = (int)hd.z > 0 ? L2 - 1 : B - L2;
      const uint32_t tb = last >= 0 ? tile_s + 16u * (uint32_t)(c0 + ts.sy * c1 + ts.sz * c2) : id_s;
      const uint32_t ev = ps + (uint32_t)TL.nev;
      int e = wl;
      if (!(e & 1)) {  // to an odd index: event pairs (e - 1, e) are 16-byte aligned
        const float2 v = lds_f2(ev + 8 * e);
        I = step_pair_g(e <= last, tb + 2 * (int)__float_as_uint(v.y), v.x, I);
        --e;
      }
      for (; e >= 3; e -= 4) {
        const float4 v = lds_f4(ev + 8 * (e - 1));
        const float4 u = lds_f4(ev + 8 * (e - 3));
        I = step_pair_g(e <= last, tb + 2 * (int)__float_as_uint(v.w), v.z, I);
        I = step_pair_g(e - 1 <= last, tb + 2 * (int)__float_as_uint(v.y), v.x, I);
        I = step_pair_g(e - 2 <= last, tb + 2 * (int)__float_as_uint(u.w), u.z, I);
        I = step_pair_g(e - 3 <= last, tb + 2 * (int)__float_as_uint(u.y), u.x, I);
      }
      if (e == 1) {
        const float4 v = lds_f4(ev);
        I = step_pair_g(1 <= last, tb + 2 * (int)__float_as_uint(v.w), v.z, I);
        I = step_pair_g(0 <= last, tb + 2 * (int)__float_as_uint(v.y), v.x, I);
      }
    }
    if (act) {
      const float I1 = I.x, I2 = I.y;
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
template <typename R, int V, bool WITH_E64>
__global__ void __launch_bounds__(256, 4) moments_kernel(long long ncell, int ndir, const R *__restrict__ I,
                                                      const R *__restrict__ coef, R *__restrict__ M,
                                                      double *__restrict__ E64, double w64) {
  __shared__ R cs[64][10];
  const long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * V;
  R acc[V][10];
  double e64[V];  // E in FP64: the weights are equal, so the sum of I times w
#pragma unroll
  for (int v = 0; v < V; ++v) {
    e64[v] = 0.0;
#pragma unroll
    for (int m = 0; m < 10; ++m) acc[v][m] = R(0);
  }
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
        if constexpr (WITH_E64) {
#pragma unroll
          for (int j = 0; j < V; ++j) e64[j] += (double)v[j];
        }
      }
    }
  }
  if (c >= ncell) return;
  if constexpr (WITH_E64) {
#pragma unroll
    for (int j = 0; j < V; ++j)
      if (c + j < ncell) E64[c + j] = w64 * e64[j];
  }
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

// Staging of the paired cell pass: directions per tile (whole antipodal
// pairs: the tuned tile rounded up to even) and ring depth, the most stages
// (at most kPairStagesMax) that fit the shared memory of one of the
// pair_min_ctas(B) CTAs an SM holds beside the paired tile.
inline void pair_staging(int B, int want, int &dt, int &nstage) {
  constexpr long long kSmemPerSM = 233472, kReservedPerCta = 1024;
  constexpr long long kStatic = 1024 * 4 + 2 * kPairStagesMax * 8 + 64;  // order, barriers, margin
  const long long per_cta = std::min<long long>(232448, kSmemPerSM / pair_min_ctas(B) - kReservedPerCta) - kStatic;
  dt = want > 0 ? want : 8;  // untuned: the tile the autotuner picks on the 128^3 workload
  dt = (dt + 1) & ~1;
  if (dt > kMaxTune) dt = kMaxTune;
  for (;;) {
    const long long ring = per_cta - (long long)pair_smem_bytes(B, 0);
    nstage = (int)std::min<long long>(kPairStagesMax, ring / ((long long)dt * cell_slot(B).bytes));
    if (nstage >= 2 || dt <= 2) break;
    dt -= 2;
  }
}

}  // namespace

TailPlan plan_tail_split(int B, int nblk, int nsm, int ntiles) {
  TailPlan p;
  if (B != 8 && B != 16) return p;
  const int parts = B * B * B / 2 / pair_threads(B), total = nblk * parts;
  p.nfull = total;
  const int wave = nsm * pair_min_ctas(B);
  if (nsm <= 0 || total < wave) return p;
  const int r = total % wave;
  if (r == 0) return p;
  // tail time in CTA times, with each share's own start (tile load, first
  // staging) counted as 3% of a CTA; split only for a gain above 5%
  double best = 1.0;
  for (int k : {2, 3, 4, 6, 8}) {
    if (k > ntiles) break;
    const double cost = (double)((k * r + wave - 1) / wave) / k + 0.03 * k;
    if (cost < best - 0.05) {
      best = cost;
      p.k = k;
    }
  }
  if (p.k == 1) return p;
  p.nfull = total - r;
  p.slots = r;
  p.part_bytes = (size_t)r * p.k * 28 * pair_threads(B) * sizeof(float);
  return p;
}

namespace {

template <int MODE, int BC>
void pair_launch(const GridDims &g, const float *kappa, const float *S, const unsigned char *tpl, const int *order,
                 const float *faces, const float *bnd, float *I_out, float *M_out, float *E_out, float *f_out,
                 void *emax_bits, long long spin, int *status, const int *block_list, int nlist, cudaStream_t st,
                 const TailSplit *split) {
  const int parts = BC * BC * BC / 2 / pair_threads(BC);
  const int nblk = block_list ? nlist : g.nbx * g.nby * g.nbz;
  int dt, nstage;
  pair_staging(BC, g.dir_tile, dt, nstage);
  // the tail split: whole grids only; the moment passes need its scratch
  TailPlan tp;
  tp.nfull = nblk * parts;
  if (split && !block_list) {
    const TailPlan q = plan_tail_split(BC, nblk, split->nsm, (g.ndir + dt - 1) / dt);
    const bool room = MODE == 1 || (split->part && split->count && q.part_bytes <= split->part_bytes &&
                                    q.slots <= split->slots);
    if (q.k > 1 && room) tp = q;
  }
  const int grid = tp.nfull + (nblk * parts - tp.nfull) * tp.k;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // prologue overlaps the face pass's end
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(pair_threads(BC));
  cfg.dynamicSmemBytes = pair_smem_bytes(BC, nstage * dt);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, cell_pair_kernel<MODE, BC, false>, g, parts, dt, nstage, kappa, S, tpl, order, faces, bnd, I_out,
                     M_out, E_out, f_out, emax_bits, spin, status, block_list, tp.nfull, tp.k,
                     split ? split->part : nullptr, split ? split->count : nullptr, nullptr, nullptr);
}

// One launch of the paired cell pass over the blocks of several grids of
// block edge BC: items[i] = (grid, block), grids as the single-grid
// launches' arguments.
template <int MODE, int BC>
void pair_launch_merged(int dir_tile, const CellGrid *grids, const int2 *items, int nitems, long long spin,
                        cudaStream_t st) {
  const int parts = BC * BC * BC / 2 / pair_threads(BC);
  int dt, nstage;
  pair_staging(BC, dir_tile, dt, nstage);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nitems * parts);
  cfg.blockDim = dim3(pair_threads(BC));
  cfg.dynamicSmemBytes = pair_smem_bytes(BC, nstage * dt);
  cfg.stream = st;
  const int total = nitems * parts;
  cudaLaunchKernelEx(&cfg, cell_pair_kernel<MODE, BC, true>, GridDims{}, parts, dt, nstage, (const float *)nullptr,
                     (const float *)nullptr, (const unsigned char *)nullptr, (const int *)nullptr,
                     (const float *)nullptr, (const float *)nullptr, (float *)nullptr, (float *)nullptr,
                     (float *)nullptr, (float *)nullptr, (void *)nullptr, spin, (int *)nullptr, (const int *)nullptr,
                     total, 1, (float *)nullptr, (int *)nullptr, grids, items);
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
  const void *pfns[] = {(const void *)cell_pair_kernel<0, 8, false>,  (const void *)cell_pair_kernel<0, 16, false>,
                        (const void *)cell_pair_kernel<1, 8, false>,  (const void *)cell_pair_kernel<1, 16, false>,
                        (const void *)cell_pair_kernel<2, 8, false>,  (const void *)cell_pair_kernel<2, 16, false>,
                        (const void *)cell_pair_kernel<0, 8, true>,   (const void *)cell_pair_kernel<0, 16, true>,
                        (const void *)cell_pair_kernel<2, 8, true>,   (const void *)cell_pair_kernel<2, 16, true>,
                        (const void *)face_pair_kernel<8>,            (const void *)face_pair_kernel<16>};
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

cudaError_t launch_cell_pass_merged(int B, bool with_M, int dir_tile, const CellGrid *grids, const int2 *items,
                                   int nitems, long long spin, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  if (B == 16) {
    if (with_M) pair_launch_merged<0, 16>(dir_tile, grids, items, nitems, spin, st);
    else pair_launch_merged<2, 16>(dir_tile, grids, items, nitems, spin, st);
  } else if (B == 8) {
    if (with_M) pair_launch_merged<0, 8>(dir_tile, grids, items, nitems, spin, st);
    else pair_launch_merged<2, 8>(dir_tile, grids, items, nitems, spin, st);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cell_pass(const GridDims &g, int mode, const R *kappa, const R *S, const unsigned char *tpl,
                             const int *order, const R *faces, const R *bnd, R *I_out, R *M_out, R *E_out,
                             R *f_out, void *emax_bits, long long spin, int *status, cudaStream_t st,
                             const int *block_list, int nlist, const TailSplit *split) {
  if (block_list && nlist <= 0) return cudaSuccess;
  if constexpr (sizeof(R) == sizeof(float)) {
    if (g.paired && (g.B == 16 || g.B == 8)) {
      const float *k = reinterpret_cast<const float *>(kappa), *s = reinterpret_cast<const float *>(S);
      const float *fc = reinterpret_cast<const float *>(faces), *bd = reinterpret_cast<const float *>(bnd);
      float *Io = reinterpret_cast<float *>(I_out), *Mo = reinterpret_cast<float *>(M_out);
      float *Eo = reinterpret_cast<float *>(E_out), *fo = reinterpret_cast<float *>(f_out);
      const int mode2 = mode == 0 ? (M_out ? 0 : 2) : 1;
#define VET_PAIR(MODE, BC) \
  pair_launch<MODE, BC>(g, k, s, tpl, order, fc, bd, Io, Mo, Eo, fo, emax_bits, spin, status, block_list, nlist, st, \
                        split)
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
cudaError_t launch_moments(long long ncell, int ndir, const R *I, const R *coef, R *M_out, cudaStream_t st,
                           double *E64, double w64) {
  const int threads = 256;
  // vector loads need every direction's row to start 16-byte aligned
  constexpr int VW = 16 / (int)sizeof(R);
  const bool vec = ncell % VW == 0 && (reinterpret_cast<uintptr_t>(I) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(M_out) & 15) == 0;
  const long long per = vec ? VW : 1;
  const long long blocks = ((ncell + per - 1) / per + threads - 1) / threads;
  if (blocks < 1) return cudaSuccess;
  if (E64) {
    if (vec)
      moments_kernel<R, VW, true><<<(unsigned)blocks, threads, 0, st>>>(ncell, ndir, I, coef, M_out, E64, w64);
    else
      moments_kernel<R, 1, true><<<(unsigned)blocks, threads, 0, st>>>(ncell, ndir, I, coef, M_out, E64, w64);
  } else if (vec) {
    moments_kernel<R, VW, false><<<(unsigned)blocks, threads, 0, st>>>(ncell, ndir, I, coef, M_out, E64, w64);
  } else {
    moments_kernel<R, 1, false><<<(unsigned)blocks, threads, 0, st>>>(ncell, ndir, I, coef, M_out, E64, w64);
  }
  return cudaGetLastError();
}

size_t pass_smem_bytes(int B, int dirs, bool fp64) {
  return fp64 ? face_smem_bytes<double>(B, dirs) : face_smem_bytes<float>(B, dirs);
}

int cell_tile_fit(int B, int want, bool fp64) {
  return fp64 ? cell_dir_tile<double>(B, want) : cell_dir_tile<float>(B, want);
}

int pair_tile_fit(int B, int want) {
  int dt, nstage;
  pair_staging(B, want, dt, nstage);
  return dt;
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
                                           long long, int *, cudaStream_t, const int *, int,                 \
                                           const TailSplit *);                                               \
  template cudaError_t launch_floor_fix_blocks<R>(const GridDims &, const int *, int, const R *, const void *, \
                                                  double, R *, cudaStream_t);                                \
  template cudaError_t launch_fill_boundary<R>(const GridDims &, const unsigned char *, const R *, R *,      \
                                               cudaStream_t);                                                \
  template cudaError_t launch_floor_fix<R>(long long, const R *, long long, const void *, double, R *,     \
                                           cudaStream_t);                                                    \
  template cudaError_t launch_moments<R>(long long, int, const R *, const R *, R *, cudaStream_t, double *, double);

VET_INSTANTIATE(float)
VET_INSTANTIATE(double)

}  // namespace vet
