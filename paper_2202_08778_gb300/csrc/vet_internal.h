// vet_internal.h -- data shared by the host side and the kernels of libvet.
//
// Geometry is in cell units inside one block: memory-frame coordinates run
// from 0 to B along each axis of the block; the "upwind frame" of a direction
// flips every axis whose direction component is negative, so that backward
// rays always move towards lower upwind-frame coordinates and a block's
// upwind faces sit at upwind-frame coordinate 0.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace vet {

constexpr int kMaxBlock = 32;             // largest block edge B

// The thin-segment cubic: -(1 - e^-x) = y q(y), y = -x log2(e), for x < 1/4
// (q fitted for relative error by Lawson's iteratively reweighted least
// squares: 2.4e-7 in exact arithmetic, 3.4e-7 evaluated in FP32), and the
// threshold on y.
constexpr float kThinQ3 = 8.70478970381660493e-03f, kThinQ2 = 5.53004379372010468e-02f,
                kThinQ1 = 2.40211763951330648e-01f, kThinQ0 = 6.93147011611337405e-01f;
constexpr float kThinY = -0.36067376022224085f;  // x < 1/4
constexpr int kNever = 0x3fff;            // event index of an axis the ray never exits by

// Per-direction ray templates (Sec. 2.2.5 reading: long characteristics in a
// block).  A backward ray from a cell centre crosses the block's cell planes
// at parameters t = (m + 1/2)/|n_a| (m = 0, 1, ...) on axis a, independently
// of which cell it starts from; merging the three sequences gives one event
// list per direction.  A ray from a cell whose upwind-frame coordinate along
// axis a is l_a leaves the block at the event (a, m = l_a), whichever of the
// three comes first in the merged order (ties: lowest axis).  Face-node rays
// start on lattice points and cross planes at t = m/|n_a| (m = 1, 2, ...).
//
// The exit point of a ray leaving through axis a after depth l (cells:
// l + 1/2, nodes: l) has, along another axis b, the upwind-frame coordinate
// l_b + d with d = (1/2 or 0) - depth |n_b|/|n_a|; d depends on the direction
// and l only.  The host evaluates it in FP64 and stores k = floor(d) and the
// interpolation weights (f, 1 - f), f = d - k, so that the device never forms
// a position by cancellation.
//
// One direction's template is a byte blob laid out by TplLayout for the
// block edge B: a TplHead followed by the arrays below (16-byte aligned).
template <typename R>
struct TplHead {
  R n[3];     // direction
  R w;        // quadrature weight 4 pi / N
  int sgn[3]; // +1 if n_a >= 0 (a zero component counts as positive) else -1
  int ext;    // index of this direction in the documented HEALPix order
  int mirror; // 1: this template and its antipode's are exact mirror images
              // and every sign flips (no zero component)
              // (same event lengths, negated offsets, same exit tables)
  // quadrature coefficients w (1, nx, ny, nz, nx nx, ny ny, nz nz, nx ny,
  // nx nz, ny nz) of E, F and P (Eqs. 10-12, c = 1), rounded once from FP64;
  // two unused entries keep the array a multiple of 16 bytes
  alignas(16) R c[12];
  // the same ten coefficients as pairs (c_m, +-c_m) for a cell and its mirror
  // cell: the paired cell pass adds I(c, d) + I(c, -d) into E and P and
  // I(c, d) - I(c, -d) into F, and the mirror cell c' sees -d where c sees d,
  // so its F pair member is negated
  alignas(16) R cp[20];
};

// One event of a ray template: the length of the segment that ends at it,
// scaled by -h log2(e), and the byte offset in the shared-memory tile, from
// the ray's start cell, of the cell that segment crosses (0 for the first
// segment).  Rays are marched downwind, from their last event back to the
// start.
template <typename R>
struct alignas(2 * sizeof(R)) TplEvent {
  R len;
  int off;
};

// The head and the node-ray parts come first, so that the face pass stages
// only [0, node_bytes) of a template.
struct TplLayout {
  int nev;         // TplEvent<R>[3B]  node-ray events
  int npos;        // int16[3][B+1] merged index of node event (a, m); [a][0] = -1
  int nk;          // int16[3][2][B+1] floor(d) of node exits
  int nw;          // R[3][2][B+1][2]  (f, 1-f) of node exits
  int node_bytes;  // head and node-ray parts, a multiple of 16
  int cev;         // TplEvent<R>[3B]  cell-ray events
  int cpos;        // int16[3][B]  merged index of cell event (a, m)
  int ck;          // int16[3][2][B]   floor(d) of cell exits
  int cw;          // R[3][2][B][2]    (f, 1-f) of cell exits
  int bytes;       // total, a multiple of 16
};

__host__ __device__ inline int tpl_align16(int x) { return (x + 15) & ~15; }

template <typename R>
__host__ __device__ inline TplLayout tpl_layout(int B) {
  TplLayout L;
  int o = tpl_align16((int)sizeof(TplHead<R>));
  L.nev = o;  o = tpl_align16(o + 3 * B * (int)sizeof(TplEvent<R>));
  L.npos = o; o = tpl_align16(o + 3 * (B + 1) * 2);
  L.nk = o;   o = tpl_align16(o + 6 * (B + 1) * 2);
  L.nw = o;   o = tpl_align16(o + 6 * (B + 1) * 2 * (int)sizeof(R));
  L.node_bytes = o;
  L.cev = o;  o = tpl_align16(o + 3 * B * (int)sizeof(TplEvent<R>));
  L.cpos = o; o = tpl_align16(o + 3 * B * 2);
  L.ck = o;   o = tpl_align16(o + 6 * B * 2);
  L.cw = o;   o = tpl_align16(o + 6 * B * 2 * (int)sizeof(R));
  L.bytes = o;
  return L;
}

// Fixed sizes of one launch.
struct GridDims {
  int nx, ny, nz;     // cells
  int B;              // block edge
  int nbx, nby, nbz;  // blocks
  int nnode;          // (B+1)^2 face nodes per face
  int fstride;        // elements per stored face: (B+2)^2 rounded up to 16 bytes
  int ndir;           // directions
  long long ncell;    // nx*ny*nz
  int dir_tile;       // directions per cell-pass tile (0: default)
  int paired;         // 1: the cell order lists antipodal pairs (d, -d), see the paired cell pass
  int face_paired;    // 1: face-pass items are mirrored block pairs, see the paired face pass
  // face passes: per template (internal order), the (B+1)^2 face nodes of
  // each face axis by ascending node-ray length, then the node codes of all
  // three faces merged the same way, [N][6][(B+1)^2] (geom::node_order;
  // null: row order)
  const uint16_t *node_order;
};

// Shared-memory kappa/S tiles of a block, in entries of 8 bytes (kappa, S) or,
// for the FP32 mirrored passes, 16 bytes (kappa, kappa', S, S').  Face pass:
// cell (x, y, z) at x + (B+1) y + (B+1)^2 z; the three strides are odd, so a
// warp walking a row, column or pillar of a face (and any uniform shift of
// it) touches distinct banks.  Cell pass: x + (B+4) y + (B+4) B z; with B a
// multiple of 8 the y stride is 4 or 12 mod 16 entries of 8 bytes (a 4 x 4
// layer of a warp's 4 x 4 x 2 cell brick is conflict free) and 4 mod 8
// entries of 16 bytes (each quarter warp, 4 x 2 cells, covers the 32 banks
// once).
struct TileShape {
  int sy, sz, elems;
};
__host__ __device__ inline TileShape node_tile(int B) { return {B + 1, (B + 1) * (B + 1), (B + 1) * (B + 1) * B}; }
__host__ __device__ inline TileShape cell_tile(int B) { return {B + 4, (B + 4) * B, (B + 4) * B * B}; }

// Stored faces: node (ub, uc) of a face, in the upwind frame of the direction
// (the in-plane axes flipped where the direction component is negative), at
// ub * (B + 2) + uc; row and column B + 1 are zero padding.
template <typename R>
__host__ __device__ inline int face_stride_elems(int B) {
  const int per = 16 / (int)sizeof(R);
  return ((B + 2) * (B + 2) + per - 1) / per * per;
}

// One work item of the face pass: a block and a run of directions of one
// octant, all at the same wavefront level.
struct FaceItem {
  int block;
  int dir_begin;     // internal direction index
  int dir_count;
  int mirror_begin;  // paired face pass: internal index of the antipode of dir_begin
  int octant;        // the directions' octant: bit a set where component a is negative
};

// Launchers (vet_kernels.cu).  All return the cudaGetLastError() of the
// launch.  R = float or double.  `bnd` holds the boundary faces materialised
// by launch_fill_boundary; `spin` bounds every device-side wait (polls of an
// mbarrier); a wait that gives up ORs a code into *status and the kernel
// returns early with its outputs incomplete.
//   status bits: 1 face-pass staging, 2 cell-pass staging, 4 cell-pass buffer
//   release, 8 the final wait for copies still in flight.

// Face pass of one wavefront level: nitems items of at most max_dirs
// directions each.
template <typename R>
cudaError_t launch_face_level(const GridDims &g, const R *kappa, const R *S, const unsigned char *tpl,
                              const FaceItem *items, int nitems, int max_dirs, R *faces, const R *bnd,
                              long long spin, int *status, cudaStream_t st);

// Split of the paired cell pass's last partial wave.  With `total` CTAs and
// room for `wave` of them at once (SMs x CTAs per SM) the last wave holds
// r = total mod wave CTAs and leaves the other slots idle for a whole CTA's
// time; the last r CTAs' work is then cut into k shares of their direction
// tiles (k CTAs each), so that the tail takes about ceil(k r / wave) / k of
// a CTA's time.  The shares' partial moments meet in `part`
// ([slot][share][28][threads] floats) and the last share of a slot to
// finish (counted in `count`, which it resets) adds the others' and writes
// the outputs.
struct TailPlan {
  int nfull = 0;          // CTAs that run whole (total - r)
  int k = 1;              // shares per split work item (1: no split)
  int slots = 0;          // r
  size_t part_bytes = 0;  // scratch the moments of the shares need
};
TailPlan plan_tail_split(int B, int nblk, int nsm, int ntiles);

// One grid of a merged launch of the paired FP32 cell pass (the batched
// closure): what a single grid's launch passes as arguments.  M_out null:
// E goes to E_out (the floor rule's input) and only f is written.
struct CellGrid {
  GridDims g;
  const float *kappa, *S;
  const unsigned char *tpl;
  const int *order;
  const float *faces, *bnd;
  float *M_out, *E_out, *f_out;
  void *emax_bits;
  int *status;
};

// The paired FP32 cell pass (moments and f) over the blocks of several grids
// of block edge B (8 or 16) in one launch: items[i] = (grid index, block
// index), both device arrays; with_M: every grid writes M (else none does);
// one direction tile for all (0: untuned).
cudaError_t launch_cell_pass_merged(int B, bool with_M, int dir_tile, const CellGrid *grids, const int2 *items,
                                   int nitems, long long spin, cudaStream_t st);

// What the caller provides for the split: the SM count and the scratch
// (part: part_bytes, count: slots zeroed ints).  part == nullptr: no split
// of the moment passes (the trace needs no scratch).
struct TailSplit {
  int nsm = 0;
  float *part = nullptr;
  size_t part_bytes = 0;
  int *count = nullptr;
  int slots = 0;
};

// mode 0: moments + f (+ E for the floor rule); mode 1: write I_out.  The
// directions are visited in cell_order.  With a block_list (device, nlist
// block indices) only the cells of those blocks are computed.  `split`
// (paired FP32 pass only; null: none) cuts the last partial wave, see
// TailSplit; its part/count must hold the plan's slots.
template <typename R>
cudaError_t launch_cell_pass(const GridDims &g, int mode, const R *kappa, const R *S, const unsigned char *tpl,
                             const int *cell_order, const R *faces, const R *bnd, R *I_out, R *M_out, R *E_out,
                             R *f_out, void *emax_bits, long long spin, int *status, cudaStream_t st,
                             const int *block_list = nullptr, int nlist = 0, const TailSplit *split = nullptr);

// The floor rule on the cells of the listed blocks.
template <typename R>
cudaError_t launch_floor_fix_blocks(const GridDims &g, const int *block_list, int nlist, const R *E,
                                    const void *emax_bits, double floor_rel, R *f_out, cudaStream_t st);

// bnd[face][d] <- constant Ib[face][ext(d)] (or 0 when Ib is NULL).
template <typename R>
cudaError_t launch_fill_boundary(const GridDims &g, const unsigned char *tpl, const R *Ib, R *bnd, cudaStream_t st);

template <typename R>
cudaError_t launch_floor_fix(long long ncell, const R *E, long long E_stride, const void *emax_bits,
                             double floor_rel, R *f_out, cudaStream_t st);

// E64 (optional, device): E of every cell summed in FP64, w64 times the sum
// of I over the directions (the weights are all equal to w64).
template <typename R>
cudaError_t launch_moments(long long ncell, int ndir, const R *I, const R *coef, R *M_out,
                           cudaStream_t st, double *E64 = nullptr, double w64 = 0.0);

// Dynamic shared memory of an unpaired face-pass CTA staging `dirs` directions.
size_t pass_smem_bytes(int B, int dirs, bool fp64);

// Largest cell-pass direction tile (<= want) whose two buffers fit.
int cell_tile_fit(int B, int want, bool fp64);

// The direction tile the paired FP32 cell pass runs with for a requested
// tile (0: untuned), after its staging ring is fitted to shared memory.
int pair_tile_fit(int B, int want);

// Dynamic shared memory of an unpaired cell-pass CTA with `nslots` staged
// directions.
size_t cell_smem_bytes(int B, int nslots, bool fp64);

// Directions per face-pass item (default; a context may be tuned to 1..8).
constexpr int kFaceGroup = 4;
constexpr int kMaxTune = 8;

// Per-device kernel attributes; call with the context's device current.
cudaError_t prepare_kernels();

// Sets the calling thread's message returned by vet_last_error(NULL).
void set_thread_error(const char *msg);

}  // namespace vet
