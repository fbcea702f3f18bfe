// vet_host.cu -- host side of libvet: argument checks, the HEALPix direction
// set, per-direction ray templates, the wavefront schedule of the face pass,
// workspace, and the exported C ABI declared in include/vet.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "vet.h"
#include "vet_bridge.h"
#include "vet_geometry.h"
#include "vet_internal.h"

#define VET_API extern "C" __attribute__((visibility("default")))

using vet::FaceItem;
using vet::GridDims;

struct vet_ctx {
  vet_grid grid{};
  vet_config cfg{};
  GridDims dims{};
  int N = 0;
  int nblk = 0;
  int nlevels = 0;
  bool fp64 = false;
  std::vector<double> dirs_ext;  // [N][4] in HEALPix order
  std::vector<int> level_off;    // face items of level L: [level_off[L], level_off[L+1])
  std::vector<int> level_group;  // directions per face item on level L
  void *d_tpl = nullptr;         // N template blobs, internal (octant-sorted) order
  FaceItem *d_items = nullptr;
  int *d_cell_order = nullptr;   // cell-pass visiting order of internal directions
  uint16_t *d_node_order = nullptr;  // paired face pass: face nodes by ray length (dims.node_order)
  void *d_faces = nullptr;       // [N][blocks][3][fstride], upwind frame, padded
  void *d_emax = nullptr;        // 8 bytes: bit pattern of max E (nonnegative)
  void *d_E = nullptr;           // [cells] E when the caller does not want M
  void *d_coef = nullptr;        // [N][10] w (1, n, nn), HEALPix order
  void *d_bnd = nullptr;         // [6][N][fstride] boundary faces of the current call
  int *d_status = nullptr;       // device error bits (bounded waits that gave up)
  long long spin = 0;            // polls per device-side wait
  void *d_stage = nullptr;       // staging of host-pointer arguments
  size_t stage_bytes = 0;
  vet::TailSplit split;          // scratch of the cell pass's tail split (none: split.nsm = 0)
  long long cell_segs = 0, face_segs = 0;
  int ob[9] = {0};                // octant ranges of the internal direction order
  int face_group = vet::kFaceGroup;  // directions per face-pass item (tunable)
  unsigned long long tuning_gen = 0;  // bumped whenever the launches change (schedule, tiles)
  cudaStream_t last_stream = nullptr;
  bool timing = false;
  bool timed = false;            // events of the last call were recorded
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::string err;
};

namespace {

thread_local std::string g_create_err;

vet_status set_err(vet_ctx *c, vet_status st, const std::string &msg) {
  if (c) c->err = msg;
  else g_create_err = msg;
  return st;
}

vet_status cuda_err(vet_ctx *c, cudaError_t e, const char *what) {
  return set_err(c, e == cudaErrorMemoryAllocation ? VET_ENOMEM : VET_ECUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

// Switches to the context's device for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void free_ctx(vet_ctx *c) {
  if (!c) return;
  for (auto &e : c->ev)
    if (e) cudaEventDestroy(e);
  cudaFree(c->d_tpl);
  cudaFree(c->d_items);
  cudaFree(c->d_cell_order);
  cudaFree(c->d_node_order);
  cudaFree(c->d_faces);
  cudaFree(c->d_emax);
  cudaFree(c->d_E);
  cudaFree(c->d_coef);
  cudaFree(c->d_bnd);
  cudaFree(c->d_status);
  cudaFree(c->d_stage);
  cudaFree(c->split.part);
  cudaFree(c->split.count);
  delete c;
}

// Face-pass schedule for `group` directions per item (uploaded; replaces the
// previous one).  A level whose items would not fill the GPU's face-pass
// CTA slots once (three per SM, two for the paired face pass) gets smaller
// items (group halved, down to one direction): the first and last wavefront
// levels hold few blocks, and shorter CTAs end them sooner.
vet_status build_schedule(vet_ctx *c, int group) {
  const int nb[3] = {c->dims.nbx, c->dims.nby, c->dims.nbz};
  c->nlevels = nb[0] + nb[1] + nb[2] - 2;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->cfg.device) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 1;
  }
  const bool paired = c->dims.face_paired != 0;
  const long long slots = (paired ? 2LL : 3LL) * sms;
  std::vector<int> lg(c->nlevels, group), off(c->nlevels + 1, 0);
  for (int g = group / 2; g >= 1; g /= 2) {  // items per level at g directions per item
    std::vector<int> prev(c->nlevels + 1, 0);
    vet::geom::build_schedule(nb, c->ob, g * 2, nullptr, 1LL << 40, prev.data(), nullptr, paired);
    for (int L = 0; L < c->nlevels; ++L)
      if (lg[L] == g * 2 && prev[L + 1] - prev[L] < slots) lg[L] = g;  // 2g left the level under one wave
  }
  const long long nitems =
      vet::geom::build_schedule(nb, c->ob, group, nullptr, 1LL << 40, off.data(), lg.data(), paired);
  std::vector<FaceItem> built((size_t)std::max<long long>(1, nitems));
  vet::geom::build_schedule(nb, c->ob, group, built.data(), nitems, off.data(), lg.data(), paired);
  // A level of at least one wave whose last partial wave is at most half a
  // wave ends with its last r items cut in two (halves of their direction
  // runs): the 2r shorter CTAs then finish in one round, sooner than the r
  // whole ones.
  std::vector<FaceItem> items;
  items.reserve(built.size() + slots);
  std::vector<int> noff(c->nlevels + 1, 0);
  for (int L = 0; L < c->nlevels; ++L) {
    noff[L] = (int)items.size();
    const int n = off[L + 1] - off[L], r = (int)(n % slots);
    const bool cut = n >= slots && r > 0 && 2LL * r <= slots && lg[L] >= 2;
    for (int i = off[L]; i < off[L + 1]; ++i) {
      const FaceItem it = built[i];
      if (cut && i >= off[L + 1] - r && it.dir_count >= 2) {
        const int h = it.dir_count / 2;
        items.push_back({it.block, it.dir_begin, h, it.mirror_begin, it.octant});
        items.push_back({it.block, it.dir_begin + h, it.dir_count - h, paired ? it.mirror_begin + h : 0, it.octant});
      } else {
        items.push_back(it);
      }
    }
  }
  noff[c->nlevels] = (int)items.size();
  if (items.empty()) items.push_back(FaceItem{});
  off = noff;
  FaceItem *d = nullptr;
  cudaError_t e = cudaMalloc((void **)&d, sizeof(FaceItem) * items.size());
  if (e) return cuda_err(c, e, "cudaMalloc(schedule)");
  if ((e = cudaMemcpy(d, items.data(), sizeof(FaceItem) * items.size(), cudaMemcpyHostToDevice))) {
    cudaFree(d);
    return cuda_err(c, e, "upload schedule");
  }
  cudaFree(c->d_items);
  c->d_items = d;
  c->level_off = off;
  c->level_group = lg;
  c->face_group = group;
  ++c->tuning_gen;  // a batch graph captured with the old schedule must not replay
  return VET_OK;
}

// Scratch of the paired cell pass's tail split for the whole grid (the
// largest plan over the direction tiles the tuning can pick); the split is
// left off when the pass is not paired or the plan does not split.
vet_status enable_tail_split(vet_ctx *c) {
  if (!c->dims.paired || c->split.part) return VET_OK;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->cfg.device) != cudaSuccess) {
    cudaGetLastError();
    return VET_OK;
  }
  vet::TailPlan best;
  for (int dt = 2; dt <= vet::kMaxTune; dt += 2) {
    const vet::TailPlan p = vet::plan_tail_split(c->grid.block, c->nblk, nsm, (c->N + dt - 1) / dt);
    if (p.part_bytes > best.part_bytes) best = p;
  }
  c->split.nsm = nsm;
  if (best.k <= 1) return VET_OK;  // trace-mode splits need no scratch
  cudaError_t e;
  if ((e = cudaMalloc((void **)&c->split.part, best.part_bytes))) return cuda_err(c, e, "cudaMalloc(tail split)");
  if ((e = cudaMalloc((void **)&c->split.count, sizeof(int) * best.slots)))
    return cuda_err(c, e, "cudaMalloc(tail split counts)");
  if ((e = cudaMemset(c->split.count, 0, sizeof(int) * best.slots))) return cuda_err(c, e, "cudaMemset(tail split)");
  c->split.part_bytes = best.part_bytes;
  c->split.slots = best.slots;
  return VET_OK;
}

// Off for grids of a batch, whose closures share the GPU: a lone grid's last
// wave leaves SMs idle, a batch's does not.
void disable_tail_split(vet_ctx *c) {
  cudaFree(c->split.part);
  cudaFree(c->split.count);
  c->split = vet::TailSplit();
}

template <typename R>
vet_status build_context(vet_ctx *c) {
  const int B = c->grid.block, N = c->N;
  std::vector<int> order(N);
  int ob[9];
  vet::geom::internal_order(N, c->dirs_ext.data(), order.data(), ob);
  // FP32 face pass on mirrored block pairs: antipodes at equal positions of
  // opposite octants (block edges 8 and 16, no zero direction component)
  const bool mirror_order =
      !c->fp64 && (B == 8 || B == 16) && vet::geom::mirror_octant_order(N, c->dirs_ext.data(), order.data(), ob);
  const int tbytes = vet::tpl_layout<R>(B).bytes;
  std::vector<unsigned char> tpl((size_t)tbytes * N);
  long long cs_tot = 0, ns_tot = 0;
  for (int i = 0; i < N; ++i) {
    long long cs, ns[3];
    vet::geom::build_template<R>(&c->dirs_ext[4 * order[i]], order[i], B, c->grid.h, tpl.data() + (size_t)i * tbytes,
                                 cs, ns);
    cs_tot += cs;
    ns_tot += ns[0] + ns[1] + ns[2];
  }
  // the method's work: every block's three downwind faces (the face pass
  // skips those on the domain boundary, which no block reads)
  c->cell_segs = cs_tot * c->nblk;
  c->face_segs = ns_tot * c->nblk;
  std::memcpy(c->ob, ob, sizeof ob);
  std::vector<int> cell_order(N);
  vet::geom::interleaved_order(ob, cell_order.data());
  // FP32 cell pass on mirrored ray pairs where the set is closed under
  // negation (block edges 8 and 16)
  c->dims.paired = 0;
  if (!c->fp64 && (B == 8 || B == 16) && vet::geom::antipodal_order(N, c->dirs_ext.data(), order.data(),
                                                                     cell_order.data())) {
    c->dims.paired = 1;
    // pairs whose templates are not exact mirrors, or with a zero direction
    // component (whose sign the antipode need not flip), are marched ray by ray
    for (int k = 0; k < N; k += 2) {
      unsigned char *ta = tpl.data() + (size_t)cell_order[k] * tbytes;
      unsigned char *tb = tpl.data() + (size_t)cell_order[k + 1] * tbytes;
      const int m = vet::geom::mirrored_cell_pair<R>(ta, tb, B) ? 1 : 0;
      reinterpret_cast<vet::TplHead<R> *>(ta)->mirror = m;
      reinterpret_cast<vet::TplHead<R> *>(tb)->mirror = m;
    }
  }
  // the face pass pairs (b, d) with (b', -d) only if every pair's node rays
  // are exact mirror images (near-tied plane crossings can break this)
  c->dims.face_paired = 0;
  if (mirror_order) {
    bool all = true;
    for (int o = 0; o < 8 && all; o += 2)
      for (int k = 0; k < ob[o + 1] - ob[o] && all; ++k)
        all = vet::geom::mirror_node_templates<R>(tpl.data() + (size_t)(ob[o] + k) * tbytes,
                                                  tpl.data() + (size_t)(ob[7 - o] + k) * tbytes, B);
    c->dims.face_paired = all ? 1 : 0;
  }
  // moment coefficients in HEALPix order
  std::vector<R> coef((size_t)N * 10);
  for (int k = 0; k < N; ++k) {
    const double *d = &c->dirs_ext[4 * k];
    const double w = d[3], x = d[0], y = d[1], z = d[2];
    const double v[10] = {w, w * x, w * y, w * z, w * x * x, w * y * y, w * z * z, w * x * y, w * x * z, w * y * z};
    for (int m = 0; m < 10; ++m) coef[(size_t)k * 10 + m] = R(v[m]);
  }
  cudaError_t e;
  c->dims.fstride = vet::face_stride_elems<R>(B);
  const size_t face_elems = (size_t)N * c->nblk * 3 * c->dims.fstride;
  if ((e = cudaMalloc(&c->d_tpl, tpl.size()))) return cuda_err(c, e, "cudaMalloc(templates)");
  if ((e = cudaMalloc(&c->d_faces, sizeof(R) * face_elems))) return cuda_err(c, e, "cudaMalloc(face intensities)");
  // the padding row and column of every stored face stay zero for good
  if ((e = cudaMemset(c->d_faces, 0, sizeof(R) * face_elems))) return cuda_err(c, e, "cudaMemset(face intensities)");
  if ((e = cudaMalloc(&c->d_emax, 8))) return cuda_err(c, e, "cudaMalloc(emax)");
  if ((e = cudaMalloc(&c->d_E, sizeof(R) * c->dims.ncell))) return cuda_err(c, e, "cudaMalloc(E)");
  if ((e = cudaMalloc(&c->d_coef, sizeof(R) * coef.size()))) return cuda_err(c, e, "cudaMalloc(coef)");
  if ((e = cudaMalloc(&c->d_bnd, sizeof(R) * 6 * (size_t)N * c->dims.fstride)))
    return cuda_err(c, e, "cudaMalloc(boundary faces)");
  if ((e = cudaMalloc((void **)&c->d_status, sizeof(int)))) return cuda_err(c, e, "cudaMalloc(status)");
  if ((e = cudaMemset(c->d_status, 0, sizeof(int)))) return cuda_err(c, e, "cudaMemset(status)");
  if ((e = cudaMemcpy(c->d_tpl, tpl.data(), tpl.size(), cudaMemcpyHostToDevice)))
    return cuda_err(c, e, "upload templates");
  vet_status st = build_schedule(c, c->face_group);
  if (st != VET_OK) return st;
  // the cell passes stage by this order: each entry also carries the
  // direction's signs (bits 16-18, flag bit 19)
  for (int k = 0; k < N; ++k) {
    const auto *hd = reinterpret_cast<const vet::TplHead<R> *>(tpl.data() + (size_t)cell_order[k] * tbytes);
    int bits = 0;
    for (int a = 0; a < 3; ++a) bits |= (hd->sgn[a] < 0 ? 1 : 0) << a;
    cell_order[k] |= (1 << 19) | (bits << 16);
  }
  if ((e = cudaMalloc((void **)&c->d_cell_order, sizeof(int) * N))) return cuda_err(c, e, "cudaMalloc(order)");
  if ((e = cudaMemcpy(c->d_cell_order, cell_order.data(), sizeof(int) * N, cudaMemcpyHostToDevice)))
    return cuda_err(c, e, "upload order");
  {  // both face passes hand their node rays to the lanes by ray length
    const int NN = (B + 1) * (B + 1);
    std::vector<uint16_t> nord((size_t)N * 6 * NN);
    for (int i = 0; i < N; ++i)
      vet::geom::node_order<R>(tpl.data() + (size_t)i * tbytes, B, nord.data() + (size_t)i * 6 * NN);
    if ((e = cudaMalloc((void **)&c->d_node_order, sizeof(uint16_t) * nord.size())))
      return cuda_err(c, e, "cudaMalloc(node order)");
    if ((e = cudaMemcpy(c->d_node_order, nord.data(), sizeof(uint16_t) * nord.size(), cudaMemcpyHostToDevice)))
      return cuda_err(c, e, "upload node order");
    c->dims.node_order = c->d_node_order;
  }
  if ((e = cudaMemcpy(c->d_coef, coef.data(), sizeof(R) * coef.size(), cudaMemcpyHostToDevice)))
    return cuda_err(c, e, "upload coefficients");
  if ((e = vet::prepare_kernels())) return cuda_err(c, e, "cudaFuncSetAttribute");
  return enable_tail_split(c);
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of pinned, mapped host memory (page-locked by
// cudaHostAlloc or cudaHostRegister; under unified addressing such memory is
// mapped), or nullptr for device or pageable memory.
void *mapped_host_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Device views of the caller's arguments; host arguments are staged.
struct Staging {
  vet_ctx *c;
  size_t used = 0;
  bool any_host = false;
  std::vector<std::pair<void *, const void *>> d2h;  // (host dst, device src)
  std::vector<size_t> d2h_bytes;
};

vet_status reserve_stage(vet_ctx *c, size_t bytes) {
  if (bytes <= c->stage_bytes) return VET_OK;
  cudaFree(c->d_stage);
  c->d_stage = nullptr;
  c->stage_bytes = 0;
  cudaError_t e = cudaMalloc(&c->d_stage, bytes);
  if (e) return cuda_err(c, e, "cudaMalloc(staging)");
  c->stage_bytes = bytes;
  return VET_OK;
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename R>
vet_status check_ctx(vet_ctx *c, bool want_fp64) {
  if (!c) return VET_EINVAL;
  if (c->fp64 != want_fp64)
    return set_err(c, VET_EINVAL, want_fp64 ? "FP64 entry point on an FP32 context" : "FP32 entry point on an FP64 context");
  return VET_OK;
}

// Prepares device pointers for a call.  ins: inputs (ptr, elements, may be
// null); outs: outputs.  Host inputs are copied to the staging buffer on
// `st`.  Host outputs in pinned (mapped) memory are written by the kernels
// directly, through their device address: the results cross the host link
// as the kernels write them (each output element is written once), with no
// separate copy afterwards; pageable host outputs are staged and copied
// back.
template <typename R>
vet_status stage_args(vet_ctx *c, cudaStream_t st, std::vector<std::pair<const R *, size_t>> ins,
                      std::vector<std::pair<R *, size_t>> outs, std::vector<const R *> &din,
                      std::vector<R *> &dout, std::vector<std::pair<R *, R *>> &copy_back,
                      std::vector<size_t> &copy_bytes, bool &any_host) {
  size_t need = 0;
  std::vector<bool> in_host(ins.size()), out_host(outs.size());
  for (size_t i = 0; i < ins.size(); ++i) {
    in_host[i] = ins[i].first && !is_device_ptr(ins[i].first);
    if (in_host[i]) need += round256(ins[i].second * sizeof(R));
  }
  std::vector<void *> out_mapped(outs.size(), nullptr);
  for (size_t i = 0; i < outs.size(); ++i) {
    out_host[i] = outs[i].first && !is_device_ptr(outs[i].first);
    if (out_host[i]) out_mapped[i] = mapped_host_ptr(outs[i].first);
    if (out_host[i] && !out_mapped[i]) need += round256(outs[i].second * sizeof(R));
  }
  any_host = false;  // then the call returns only once its results are in place
  for (bool h : in_host) any_host = any_host || h;
  for (bool h : out_host) any_host = any_host || h;
  if (need) {
    vet_status s = reserve_stage(c, need);
    if (s != VET_OK) return s;
  }
  char *base = (char *)c->d_stage;
  size_t off = 0;
  din.clear();
  dout.clear();
  for (size_t i = 0; i < ins.size(); ++i) {
    if (!in_host[i]) {
      din.push_back(ins[i].first);
      continue;
    }
    R *d = (R *)(base + off);
    off += round256(ins[i].second * sizeof(R));
    cudaError_t e = cudaMemcpyAsync(d, ins[i].first, ins[i].second * sizeof(R), cudaMemcpyHostToDevice, st);
    if (e) return cuda_err(c, e, "host-to-device copy");
    din.push_back(d);
  }
  for (size_t i = 0; i < outs.size(); ++i) {
    if (!out_host[i]) {
      dout.push_back(outs[i].first);
      continue;
    }
    if (out_mapped[i]) {  // written in place; the call still synchronises
      dout.push_back((R *)out_mapped[i]);
      continue;
    }
    R *d = (R *)(base + off);
    off += round256(outs[i].second * sizeof(R));
    dout.push_back(d);
    copy_back.push_back({outs[i].first, d});
    copy_bytes.push_back(outs[i].second * sizeof(R));
  }
  return VET_OK;
}

// Reads and clears the device status word (the stream must be idle).
vet_status check_status(vet_ctx *c) {
  int st = 0;
  cudaError_t e = cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e) return cuda_err(c, e, "status read");
  if (st) {
    cudaMemset(c->d_status, 0, sizeof(int));
    // a share that gave up may not have counted itself
    if (c->split.count) cudaMemset(c->split.count, 0, sizeof(int) * c->split.slots);
    return set_err(c, VET_ETIMEOUT,
                   "a device-side wait gave up (status bits " + std::to_string(st) + "); outputs are incomplete");
  }
  return VET_OK;
}

template <typename R>
vet_status finish_args(vet_ctx *c, cudaStream_t st, const std::vector<std::pair<R *, R *>> &copy_back,
                       const std::vector<size_t> &bytes, bool had_host) {
  for (size_t i = 0; i < copy_back.size(); ++i) {
    cudaError_t e = cudaMemcpyAsync(copy_back[i].first, copy_back[i].second, bytes[i], cudaMemcpyDeviceToHost, st);
    if (e) return cuda_err(c, e, "device-to-host copy");
  }
  if (had_host) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e) return cuda_err(c, e, "stream synchronize");
    return check_status(c);
  }
  return VET_OK;
}

// Records timing event i on st when timing is enabled.
vet_status mark(vet_ctx *c, int i, cudaStream_t st) {
  if (!c->timing) return VET_OK;
  cudaError_t e = cudaEventRecord(c->ev[i], st);
  if (e) return cuda_err(c, e, "cudaEventRecord");
  if (i == 3) c->timed = true;
  return VET_OK;
}

template <typename R>
vet_status run_face_pass(vet_ctx *c, const R *kappa, const R *S, const R *Ib, cudaStream_t st) {
  cudaError_t e = vet::launch_fill_boundary<R>(c->dims, (const unsigned char *)c->d_tpl, Ib, (R *)c->d_bnd, st);
  if (e) return cuda_err(c, e, "boundary fill launch");
  for (int L = 0; L < c->nlevels; ++L) {
    const int n = c->level_off[L + 1] - c->level_off[L];
    e = vet::launch_face_level<R>(c->dims, kappa, S, (const unsigned char *)c->d_tpl, c->d_items + c->level_off[L], n,
                                  c->level_group[L], (R *)c->d_faces, (const R *)c->d_bnd, c->spin, c->d_status, st);
    if (e) return cuda_err(c, e, "face pass launch");
  }
  return VET_OK;
}

template <typename R>
vet_status do_trace(vet_ctx *c, const R *kappa, const R *S, const R *Ib, R *I_out, void *stream, bool fp64) {
  vet_status s = check_ctx<R>(c, fp64);
  if (s) return s;
  if (!kappa || !S || !I_out) return set_err(c, VET_EINVAL, "kappa, S and I_out are required");
  DeviceGuard dg(c->cfg.device);
  if (!dg.ok) return set_err(c, VET_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nc = (size_t)c->dims.ncell;
  std::vector<const R *> din;
  std::vector<R *> dout;
  std::vector<std::pair<R *, R *>> back;
  std::vector<size_t> bytes;
  bool had_host = false;
  s = stage_args<R>(c, st, {{kappa, nc}, {S, nc}, {Ib, Ib ? (size_t)6 * c->N : 0}}, {{I_out, (size_t)c->N * nc}},
                    din, dout, back, bytes, had_host);
  if (s) return s;
  c->timed = false;
  if ((s = mark(c, 0, st))) return s;
  if ((s = run_face_pass<R>(c, din[0], din[1], din[2], st))) return s;
  if ((s = mark(c, 1, st))) return s;
  cudaError_t e = vet::launch_cell_pass<R>(c->dims, 1, din[0], din[1], (const unsigned char *)c->d_tpl,
                                           c->d_cell_order, (const R *)c->d_faces, (const R *)c->d_bnd, dout[0],
                                           nullptr, nullptr, nullptr, nullptr, c->spin, c->d_status, st, nullptr, 0,
                                           c->split.nsm ? &c->split : nullptr);
  if (e) return cuda_err(c, e, "cell pass launch");
  if ((s = mark(c, 2, st)) || (s = mark(c, 3, st))) return s;
  c->last_stream = st;
  return finish_args<R>(c, st, back, bytes, had_host);
}

template <typename R>
vet_status do_moments(vet_ctx *c, const R *I, R *M_out, void *stream, bool fp64, double *E64_out = nullptr) {
  vet_status s = check_ctx<R>(c, fp64);
  if (s) return s;
  if (!I || !M_out) return set_err(c, VET_EINVAL, "I and M_out are required");
  if (E64_out && !is_device_ptr(E64_out)) return set_err(c, VET_EINVAL, "E64_out must be device memory");
  DeviceGuard dg(c->cfg.device);
  if (!dg.ok) return set_err(c, VET_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nc = (size_t)c->dims.ncell;
  std::vector<const R *> din;
  std::vector<R *> dout;
  std::vector<std::pair<R *, R *>> back;
  std::vector<size_t> bytes;
  bool had_host = false;
  s = stage_args<R>(c, st, {{I, (size_t)c->N * nc}}, {{M_out, 10 * nc}}, din, dout, back, bytes, had_host);
  if (s) return s;
  cudaError_t e = vet::launch_moments<R>(c->dims.ncell, c->N, din[0], (const R *)c->d_coef, dout[0], st, E64_out,
                                         c->dirs_ext[3]);
  if (e) return cuda_err(c, e, "moments launch");
  c->last_stream = st;
  return finish_args<R>(c, st, back, bytes, had_host);
}

template <typename R>
vet_status do_closure(vet_ctx *c, const R *kappa, const R *S, const R *Ib, R *f_out, R *M_out, void *stream,
                      bool fp64) {
  vet_status s = check_ctx<R>(c, fp64);
  if (s) return s;
  if (!kappa || !S || !f_out) return set_err(c, VET_EINVAL, "kappa, S and f_out are required");
  DeviceGuard dg(c->cfg.device);
  if (!dg.ok) return set_err(c, VET_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nc = (size_t)c->dims.ncell;
  std::vector<const R *> din;
  std::vector<R *> dout;
  std::vector<std::pair<R *, R *>> back;
  std::vector<size_t> bytes;
  bool had_host = false;
  s = stage_args<R>(c, st, {{kappa, nc}, {S, nc}, {Ib, Ib ? (size_t)6 * c->N : 0}},
                    {{f_out, 6 * nc}, {M_out, M_out ? 10 * nc : 0}}, din, dout, back, bytes, had_host);
  if (s) return s;
  c->timed = false;
  if ((s = mark(c, 0, st))) return s;
  cudaError_t e = cudaMemsetAsync(c->d_emax, 0, 8, st);
  if (e) return cuda_err(c, e, "cudaMemsetAsync");
  if ((s = run_face_pass<R>(c, din[0], din[1], din[2], st))) return s;
  if ((s = mark(c, 1, st))) return s;
  R *Mdev = dout[1];
  e = vet::launch_cell_pass<R>(c->dims, 0, din[0], din[1], (const unsigned char *)c->d_tpl, c->d_cell_order,
                               (const R *)c->d_faces, (const R *)c->d_bnd, nullptr, Mdev, (R *)c->d_E, dout[0],
                               c->d_emax, c->spin, c->d_status, st, nullptr, 0, c->split.nsm ? &c->split : nullptr);
  if (e) return cuda_err(c, e, "cell pass launch");
  if ((s = mark(c, 2, st))) return s;
  const R *E = Mdev ? Mdev : (const R *)c->d_E;
  e = vet::launch_floor_fix<R>(c->dims.ncell, E, 1, c->d_emax, 1e-30, dout[0], st);
  if (e) return cuda_err(c, e, "floor launch");
  if ((s = mark(c, 3, st))) return s;
  c->last_stream = st;
  return finish_args<R>(c, st, back, bytes, had_host);
}

}  // namespace

void vet::set_thread_error(const char *msg) { g_create_err = msg; }

vet::CtxInfo vet::ctx_info(const vet_ctx *c) {
  CtxInfo i{};
  i.grid = c->grid;
  i.ndir = c->N;
  i.nblk = c->nblk;
  i.fp64 = c->fp64;
  i.device = c->cfg.device;
  return i;
}

vet_status vet::ctx_fail(vet_ctx *c, vet_status st, const char *msg) { return set_err(c, st, msg); }

vet_status vet::exact_on_blocks(vet_ctx *c, const float *kappa, const float *S, const float *Ib, const int *d_list,
                                int nlist, float *f_out, cudaStream_t st) {
  if (!c || c->fp64) return set_err(c, VET_EINVAL, "the learned closure needs an FP32 context");
  if (nlist <= 0) return VET_OK;
  cudaError_t e = cudaMemsetAsync(c->d_emax, 0, 8, st);
  if (e) return cuda_err(c, e, "cudaMemsetAsync");
  vet_status s = run_face_pass<float>(c, kappa, S, Ib, st);
  if (s) return s;
  e = vet::launch_cell_pass<float>(c->dims, 0, kappa, S, (const unsigned char *)c->d_tpl, c->d_cell_order,
                                   (const float *)c->d_faces, (const float *)c->d_bnd, nullptr, nullptr,
                                   (float *)c->d_E, f_out, c->d_emax, c->spin, c->d_status, st, d_list, nlist);
  if (e) return cuda_err(c, e, "cell pass launch");
  e = vet::launch_floor_fix_blocks<float>(c->dims, d_list, nlist, (const float *)c->d_E, c->d_emax, 1e-30, f_out, st);
  if (e) return cuda_err(c, e, "floor launch");
  c->last_stream = st;
  return VET_OK;
}

VET_API vet_status vet_create(vet_ctx **out, const vet_grid *grid, const vet_config *cfg) {
  if (!out) return set_err(nullptr, VET_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grid || !cfg) return set_err(nullptr, VET_EINVAL, "grid and cfg are required");
  const vet_grid g = *grid;
  if (g.block < 2 || g.block > vet::kMaxBlock) return set_err(nullptr, VET_EINVAL, "block edge must be in 2..32");
  if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nx % g.block || g.ny % g.block || g.nz % g.block)
    return set_err(nullptr, VET_EINVAL, "grid extents must be positive multiples of the block edge");
  if (!(g.h > 0.0) || !std::isfinite(g.h)) return set_err(nullptr, VET_EINVAL, "cell edge h must be positive");
  if (cfg->nside < 1 || cfg->nside > 16 || (cfg->nside & (cfg->nside - 1)))
    return set_err(nullptr, VET_EINVAL, "nside must be a power of two in 1..16");
  if (cfg->precision != VET_FP32 && cfg->precision != VET_FP64)
    return set_err(nullptr, VET_EINVAL, "precision must be VET_FP32 or VET_FP64");
  const double qn = std::sqrt(cfg->rot_q[0] * cfg->rot_q[0] + cfg->rot_q[1] * cfg->rot_q[1] +
                              cfg->rot_q[2] * cfg->rot_q[2] + cfg->rot_q[3] * cfg->rot_q[3]);
  if (!(qn > 1e-12) || !std::isfinite(qn)) return set_err(nullptr, VET_EINVAL, "rotation quaternion is zero or not finite");
  const bool fp64 = cfg->precision == VET_FP64;
  const int nnode = (g.block + 1) * (g.block + 1);
  if (vet::pass_smem_bytes(g.block, vet::kFaceGroup, fp64) > 232448 - 64 ||
      vet::cell_smem_bytes(g.block, 2, fp64) > 232448 - 64)
    return set_err(nullptr, VET_EUNSUPPORTED, "block edge too large for one CTA's shared memory at this precision");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return set_err(nullptr, VET_ECUDA, "no CUDA device");
  }
  if (cfg->device < 0 || cfg->device >= ndev) return set_err(nullptr, VET_EINVAL, "device ordinal out of range");
  vet_ctx *c = new (std::nothrow) vet_ctx;
  if (!c) return set_err(nullptr, VET_ENOMEM, "host allocation failed");
  c->grid = g;
  c->cfg = *cfg;
  c->spin = cfg->spin_limit > 0 ? cfg->spin_limit : (1LL << 22);
  c->fp64 = fp64;
  c->N = 12 * cfg->nside * cfg->nside;
  c->dims.nx = g.nx;
  c->dims.ny = g.ny;
  c->dims.nz = g.nz;
  c->dims.B = g.block;
  c->dims.nbx = g.nx / g.block;
  c->dims.nby = g.ny / g.block;
  c->dims.nbz = g.nz / g.block;
  c->dims.nnode = nnode;
  c->dims.ndir = c->N;
  c->dims.ncell = (long long)g.nx * g.ny * g.nz;
  c->nblk = c->dims.nbx * c->dims.nby * c->dims.nbz;
  c->dirs_ext.assign((size_t)c->N * 4, 0.0);
  vet::geom::healpix_directions(cfg->nside, cfg->rot_q, c->dirs_ext.data());
  vet_status s;
  {
    DeviceGuard dg(cfg->device);
    if (!dg.ok) {
      delete c;
      return set_err(nullptr, VET_ECUDA, "cudaSetDevice failed");
    }
    s = fp64 ? build_context<double>(c) : build_context<float>(c);
  }
  if (s != VET_OK) {
    g_create_err = c->err;
    free_ctx(c);
    return s;
  }
  *out = c;
  return VET_OK;
}

VET_API vet_status vet_destroy(vet_ctx *ctx) {
  if (!ctx) return VET_OK;
  DeviceGuard dg(ctx->cfg.device);
  free_ctx(ctx);
  return VET_OK;
}

VET_API int vet_num_directions(const vet_ctx *ctx) { return ctx ? ctx->N : -1; }

VET_API vet_status vet_directions(const vet_ctx *ctx, double *dirs_out) {
  if (!ctx || !dirs_out) return VET_EINVAL;
  std::memcpy(dirs_out, ctx->dirs_ext.data(), sizeof(double) * ctx->dirs_ext.size());
  return VET_OK;
}

VET_API vet_status vet_trace(vet_ctx *ctx, const float *kappa, const float *S, const float *Ib, float *I_out,
                             void *stream) {
  return do_trace<float>(ctx, kappa, S, Ib, I_out, stream, false);
}

VET_API vet_status vet_moments(vet_ctx *ctx, const float *I, float *M_out, double *E64_out, void *stream) {
  return do_moments<float>(ctx, I, M_out, stream, false, E64_out);
}

VET_API vet_status vet_closure(vet_ctx *ctx, const float *kappa, const float *S, const float *Ib, float *f_out,
                               float *M_out, void *stream) {
  return do_closure<float>(ctx, kappa, S, Ib, f_out, M_out, stream, false);
}

VET_API vet_status vet_trace_f64(vet_ctx *ctx, const double *kappa, const double *S, const double *Ib,
                                 double *I_out, void *stream) {
  return do_trace<double>(ctx, kappa, S, Ib, I_out, stream, true);
}

VET_API vet_status vet_moments_f64(vet_ctx *ctx, const double *I, double *M_out, void *stream) {
  return do_moments<double>(ctx, I, M_out, stream, true);
}

VET_API vet_status vet_closure_f64(vet_ctx *ctx, const double *kappa, const double *S, const double *Ib,
                                   double *f_out, double *M_out, void *stream) {
  return do_closure<double>(ctx, kappa, S, Ib, f_out, M_out, stream, true);
}

VET_API vet_status vet_sync(vet_ctx *ctx) {
  if (!ctx) return VET_EINVAL;
  DeviceGuard dg(ctx->cfg.device);
  cudaError_t e = cudaStreamSynchronize(ctx->last_stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e) return cuda_err(ctx, e, "device work failed");
  return check_status(ctx);
}

VET_API vet_status vet_work_counts(const vet_ctx *ctx, long long *cell_segments, long long *face_segments) {
  if (!ctx || !cell_segments || !face_segments) return VET_EINVAL;
  *cell_segments = ctx->cell_segs;
  *face_segments = ctx->face_segs;
  return VET_OK;
}

VET_API vet_status vet_set_timing(vet_ctx *ctx, int enable) {
  if (!ctx) return VET_EINVAL;
  DeviceGuard dg(ctx->cfg.device);
  if (enable && !ctx->ev[0]) {
    for (auto &e : ctx->ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r) return cuda_err(ctx, r, "cudaEventCreate");
    }
  }
  ctx->timing = enable != 0;
  ctx->timed = false;
  return VET_OK;
}

VET_API vet_status vet_last_timing(vet_ctx *ctx, float ms[4]) {
  if (!ctx || !ms) return VET_EINVAL;
  if (!ctx->timed) return set_err(ctx, VET_EINVAL, "no timed call since timing was enabled");
  DeviceGuard dg(ctx->cfg.device);
  cudaError_t e = cudaEventSynchronize(ctx->ev[3]);
  if (e) return cuda_err(ctx, e, "cudaEventSynchronize");
  const int from[4] = {0, 1, 2, 0}, to[4] = {1, 2, 3, 3};
  for (int i = 0; i < 4; ++i) {
    e = cudaEventElapsedTime(&ms[i], ctx->ev[from[i]], ctx->ev[to[i]]);
    if (e) return cuda_err(ctx, e, "cudaEventElapsedTime");
  }
  return VET_OK;
}

VET_API int vet_launches_per_closure(const vet_ctx *ctx) {
  if (!ctx) return -1;
  int n = 0;
  for (int L = 0; L < ctx->nlevels; ++L) n += ctx->level_off[L + 1] > ctx->level_off[L];
  return n + 3;  // + boundary fill, cell pass, floor fix
}

VET_API vet_status vet_set_tuning(vet_ctx *ctx, int face_group, int dir_tile) {
  if (!ctx) return VET_EINVAL;
  if (face_group < 0 || face_group > vet::kMaxTune || dir_tile < 0 || dir_tile > vet::kMaxTune)
    return set_err(ctx, VET_EINVAL, "face_group and dir_tile must be in 0..8 (0 keeps the current value)");
  DeviceGuard dg(ctx->cfg.device);
  if (face_group > 0 && face_group != ctx->face_group) {
    if (vet::pass_smem_bytes(ctx->grid.block, face_group, ctx->fp64) > 232448 - 64)
      return set_err(ctx, VET_EUNSUPPORTED, "face_group too large for this block edge's shared memory");
    vet_status st = build_schedule(ctx, face_group);
    if (st != VET_OK) return st;
  }
  if (dir_tile > 0) {
    const int dt = ctx->dims.paired ? vet::pair_tile_fit(ctx->grid.block, dir_tile)
                                    : vet::cell_tile_fit(ctx->grid.block, dir_tile, ctx->fp64);
    if (dt != ctx->dims.dir_tile) ++ctx->tuning_gen;
    ctx->dims.dir_tile = dt;
  }
  return VET_OK;
}

VET_API vet_status vet_get_tuning(const vet_ctx *ctx, int *face_group, int *dir_tile) {
  if (!ctx || !face_group || !dir_tile) return VET_EINVAL;
  *face_group = ctx->face_group;
  // the tile the cell pass actually runs with (the paired pass has its own
  // default and ring fitting)
  *dir_tile = ctx->dims.paired ? vet::pair_tile_fit(ctx->grid.block, ctx->dims.dir_tile)
                               : vet::cell_tile_fit(ctx->grid.block, ctx->dims.dir_tile > 0 ? ctx->dims.dir_tile : 4,
                                                    ctx->fp64);
  return VET_OK;
}

VET_API vet_status vet_autotune(vet_ctx *ctx, const float *kappa, const float *S, const float *Ib, int *face_group,
                                int *dir_tile, void *stream) {
  vet_status s = check_ctx<float>(ctx, false);
  if (s) return s;
  if (!kappa || !S) return set_err(ctx, VET_EINVAL, "kappa and S are required");
  DeviceGuard dg(ctx->cfg.device);
  cudaStream_t st = (cudaStream_t)stream;
  float *f = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaMalloc((void **)&f, sizeof(float) * 6 * (size_t)ctx->dims.ncell);
  if (e) return cuda_err(ctx, e, "cudaMalloc(autotune output)");
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int old_fg = ctx->face_group, old_dt = ctx->dims.dir_tile;
  const bool old_timing = ctx->timing;
  ctx->timing = false;
  float best = 1e30f;
  int best_fg = old_fg, best_dt = old_dt;
  const int cand[3] = {2, 4, 8};
  for (int i = 0; i < 3 && s == VET_OK; ++i) {
    for (int j = 0; j < 3 && s == VET_OK; ++j) {
      if (vet_set_tuning(ctx, cand[i], cand[j]) != VET_OK) continue;
      if (ctx->dims.dir_tile != cand[j]) continue;  // did not fit
      float t = 1e30f;
      for (int rep = 0; rep < 3 && s == VET_OK; ++rep) {  // first run warms up
        cudaEventRecord(a, st);
        s = do_closure<float>(ctx, kappa, S, Ib, f, nullptr, st, false);
        cudaEventRecord(b, st);
        if (s == VET_OK && (e = cudaEventSynchronize(b))) s = cuda_err(ctx, e, "autotune run");
        float ms = 0.f;
        if (s == VET_OK && rep > 0 && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) t = std::min(t, ms);
      }
      if (s == VET_OK && t < best) {
        best = t;
        best_fg = cand[i];
        best_dt = cand[j];
      }
    }
  }
  ctx->timing = old_timing;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(f);
  if (s != VET_OK) {
    vet_set_tuning(ctx, old_fg, old_dt > 0 ? old_dt : 4);
    return s;
  }
  s = vet_set_tuning(ctx, best_fg, best_dt);
  if (s == VET_OK && face_group) *face_group = best_fg;
  if (s == VET_OK && dir_tile) *dir_tile = best_dt;
  return s;
}

// ------------------------------------------------------------- batches
struct vet_batch {
  int n = 0;
  int device = 0;
  std::vector<vet_ctx *> ctx;
  std::vector<cudaStream_t> branch;   // one capture stream per grid
  std::vector<cudaEvent_t> joined;
  cudaStream_t origin = nullptr;
  cudaEvent_t forked = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void *> key;      // pointers the graph was captured with
  // merged cell passes: the grids' descriptors and (grid, block) work items
  // in device memory, grouped by block edge (16 first), each group's grids
  // largest first
  vet::CellGrid *d_grids = nullptr;
  int2 *d_items = nullptr;
  size_t items_cap = 0;
  std::vector<cudaEvent_t> group_done;  // one per (block edge, direction tile) group
  bool merged = true;  // one cell-pass launch per block edge (else one per grid)
  std::string err;
};

namespace {

vet_status batch_err(vet_batch *b, vet_status st, const std::string &msg) {
  b->err = msg;
  return st;
}

void free_batch(vet_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto s : b->branch) cudaStreamDestroy(s);
  for (auto e : b->joined) cudaEventDestroy(e);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->forked) cudaEventDestroy(b->forked);
  for (auto e : b->group_done)
    if (e) cudaEventDestroy(e);
  b->group_done.clear();
  cudaFree(b->d_grids);
  cudaFree(b->d_items);
  for (auto c : b->ctx) free_ctx(c);
  delete b;
}


// Whether a batch's cell passes can run merged: FP32 grids whose paired
// cell pass runs (block edges 8 and 16), M wanted by all grids or by none.
bool can_merge(const vet_batch *b, float *const *M_out) {
  if (!b->merged) return false;
  int with_M = 0;
  for (int i = 0; i < b->n; ++i) {
    const vet_ctx *c = b->ctx[i];
    if (c->fp64 || !c->dims.paired || (c->grid.block != 8 && c->grid.block != 16)) return false;
    with_M += (M_out && M_out[i]) ? 1 : 0;
  }
  return with_M == 0 || with_M == b->n;
}

// One merged cell-pass launch: the grids of one block edge and one
// direction tile (so that each grid computes exactly what its own closure
// at its tuning computes).
struct MergedGroup {
  int B, dt, first, nitems, lead;  // lead: the grid on whose branch the launch goes
  std::vector<int> members;
};

// Descriptors and work items of the merged cell passes, uploaded before
// capture: groups of one block edge and direction tile, edge 16 first; each
// group's grids with more blocks first (the long ones start first, the
// small ones fill in).
vet_status upload_merged(vet_batch *b, const float *const *kappa, const float *const *S, float *const *f_out,
                         float *const *M_out, std::vector<MergedGroup> &groups) {
  std::vector<vet::CellGrid> grids(b->n);
  for (int i = 0; i < b->n; ++i) {
    vet_ctx *c = b->ctx[i];
    vet::CellGrid &g = grids[i];
    g.g = c->dims;
    g.kappa = kappa[i];
    g.S = S[i];
    g.tpl = (const unsigned char *)c->d_tpl;
    g.order = c->d_cell_order;
    g.faces = (const float *)c->d_faces;
    g.bnd = (const float *)c->d_bnd;
    g.M_out = M_out ? M_out[i] : nullptr;
    g.E_out = (float *)c->d_E;
    g.f_out = f_out[i];
    g.emax_bits = c->d_emax;
    g.status = c->d_status;
  }
  groups.clear();
  for (int B : {16, 8})
    for (int i = 0; i < b->n; ++i) {
      const vet_ctx *c = b->ctx[i];
      if (c->grid.block != B) continue;
      const int dt = vet::pair_tile_fit(B, c->dims.dir_tile);
      auto it = std::find_if(groups.begin(), groups.end(), [&](const MergedGroup &m) { return m.B == B && m.dt == dt; });
      if (it == groups.end()) {
        groups.push_back(MergedGroup{B, dt, 0, 0, i, {}});
        it = groups.end() - 1;
      }
      it->members.push_back(i);
    }
  std::vector<int2> items;
  for (auto &m : groups) {
    std::stable_sort(m.members.begin(), m.members.end(),
                     [&](int x, int y) { return b->ctx[x]->nblk > b->ctx[y]->nblk; });
    m.lead = m.members[0];
    m.first = (int)items.size();
    for (int i : m.members)
      for (int blk = 0; blk < b->ctx[i]->nblk; ++blk) items.push_back(make_int2(i, blk));
    m.nitems = (int)items.size() - m.first;
  }
  cudaError_t e = cudaSuccess;
  if (!b->d_grids && (e = cudaMalloc((void **)&b->d_grids, sizeof(vet::CellGrid) * b->n)))
    return batch_err(b, VET_ENOMEM, std::string("cudaMalloc(batch grids): ") + cudaGetErrorString(e));
  if (items.size() > b->items_cap) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    if ((e = cudaMalloc((void **)&b->d_items, sizeof(int2) * items.size())))
      return batch_err(b, VET_ENOMEM, std::string("cudaMalloc(batch items): ") + cudaGetErrorString(e));
    b->items_cap = items.size();
  }
  if ((e = cudaMemcpy(b->d_grids, grids.data(), sizeof(vet::CellGrid) * b->n, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice)))
    return batch_err(b, VET_ECUDA, std::string("upload batch items: ") + cudaGetErrorString(e));
  while (b->group_done.size() < groups.size()) {
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)))
      return batch_err(b, VET_ECUDA, std::string("event: ") + cudaGetErrorString(e));
    b->group_done.push_back(ev);
  }
  return VET_OK;
}

// The captured work of a merged batch: each grid's face pass on its own
// branch; per group, once its grids' face passes are done, one cell pass
// over all their blocks on the lead grid's branch; then each grid's floor
// rule on its branch.
vet_status capture_merged(vet_batch *b, const float *const *kappa, const float *const *S, const float *const *Ib,
                          float *const *f_out, float *const *M_out, const std::vector<MergedGroup> &groups,
                          cudaError_t &e) {
  const bool with_M = M_out && M_out[0];
  for (int i = 0; i < b->n && !e; ++i) {
    vet_ctx *c = b->ctx[i];
    if ((e = cudaStreamWaitEvent(b->branch[i], b->forked, 0))) break;
    if ((e = cudaMemsetAsync(c->d_emax, 0, 8, b->branch[i]))) break;
    vet_status st = run_face_pass<float>(c, kappa[i], S[i], Ib ? Ib[i] : nullptr, b->branch[i]);
    if (st != VET_OK) {
      b->err = "grid " + std::to_string(i) + ": " + c->err;
      return st;
    }
    e = cudaEventRecord(b->joined[i], b->branch[i]);
  }
  std::vector<int> group_of(b->n, -1);
  for (size_t k = 0; k < groups.size() && !e; ++k) {
    const MergedGroup &m = groups[k];
    cudaStream_t gs = b->branch[m.lead];
    for (int i : m.members) {
      group_of[i] = (int)k;
      if (!e && i != m.lead) e = cudaStreamWaitEvent(gs, b->joined[i], 0);
    }
    if (!e)
      e = vet::launch_cell_pass_merged(m.B, with_M, m.dt, b->d_grids, b->d_items + m.first, m.nitems,
                                       b->ctx[m.lead]->spin, gs);
    if (!e) e = cudaEventRecord(b->group_done[k], gs);
  }
  for (int i = 0; i < b->n && !e; ++i) {
    vet_ctx *c = b->ctx[i];
    const MergedGroup &m = groups[group_of[i]];
    if (i != m.lead && (e = cudaStreamWaitEvent(b->branch[i], b->group_done[group_of[i]], 0))) break;
    const float *E = with_M ? M_out[i] : (const float *)c->d_E;
    if ((e = vet::launch_floor_fix<float>(c->dims.ncell, E, 1, c->d_emax, 1e-30, f_out[i], b->branch[i]))) break;
    if ((e = cudaEventRecord(b->joined[i], b->branch[i]))) break;
    e = cudaStreamWaitEvent(b->origin, b->joined[i], 0);
  }
  return VET_OK;
}
}  // namespace

VET_API vet_status vet_batch_create(vet_batch **out, int n, const vet_grid *grids, const vet_config *cfgs) {
  if (!out) return set_err(nullptr, VET_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !grids || !cfgs) return set_err(nullptr, VET_EINVAL, "n >= 1 grids and configs are required");
  vet_batch *b = new (std::nothrow) vet_batch;
  if (!b) return set_err(nullptr, VET_ENOMEM, "host allocation failed");
  b->n = n;
  b->device = cfgs[0].device;
  for (int i = 0; i < n; ++i) {
    if (cfgs[i].precision != VET_FP32 || cfgs[i].device != b->device) {
      free_batch(b);
      return set_err(nullptr, VET_EINVAL, "a batch holds FP32 grids on one device");
    }
    vet_ctx *c = nullptr;
    vet_status st = vet_create(&c, &grids[i], &cfgs[i]);
    if (st != VET_OK) {
      g_create_err = "grid " + std::to_string(i) + ": " + g_create_err;
      free_batch(b);
      return st;
    }
    disable_tail_split(c);
    b->ctx.push_back(c);
  }
  DeviceGuard dg(b->device);
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (!e) e = cudaEventCreateWithFlags(&b->forked, cudaEventDisableTiming);
  for (int i = 0; i < n && !e; ++i) {
    cudaStream_t s;
    cudaEvent_t ev;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking))) break;
    b->branch.push_back(s);
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) break;
    b->joined.push_back(ev);
  }
  if (e) {
    free_batch(b);
    return set_err(nullptr, VET_ECUDA, std::string("batch streams: ") + cudaGetErrorString(e));
  }
  *out = b;
  return VET_OK;
}

VET_API vet_status vet_batch_destroy(vet_batch *b) {
  if (!b) return VET_OK;
  DeviceGuard dg(b->device);
  free_batch(b);
  return VET_OK;
}

VET_API vet_ctx *vet_batch_context(vet_batch *b, int i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->ctx[i];
}

VET_API vet_status vet_batch_closure(vet_batch *b, const float *const *kappa, const float *const *S,
                                     const float *const *Ib, float *const *f_out, float *const *M_out, void *stream) {
  if (!b || !kappa || !S || !f_out) return VET_EINVAL;
  std::vector<const void *> key;
  for (int i = 0; i < b->n; ++i) {
    if (!kappa[i] || !S[i] || !f_out[i]) return batch_err(b, VET_EINVAL, "missing field pointer");
    if (!is_device_ptr(kappa[i]) || !is_device_ptr(S[i]) || !is_device_ptr(f_out[i]) ||
        (Ib && Ib[i] && !is_device_ptr(Ib[i])) || (M_out && M_out[i] && !is_device_ptr(M_out[i])))
      return batch_err(b, VET_EINVAL, "batch field pointers must be device memory");
    key.insert(key.end(), {kappa[i], S[i], Ib ? Ib[i] : nullptr, f_out[i], M_out ? M_out[i] : nullptr});
    // a member retuned through vet_batch_context (new schedule or tiles)
    // invalidates the captured launches
    key.push_back(reinterpret_cast<const void *>(static_cast<uintptr_t>(b->ctx[i]->tuning_gen)));
  }
  DeviceGuard dg(b->device);
  if (!b->exec || key != b->key) {
    // capture one closure per grid, each on its own branch of the graph (the
    // cell passes of grids of one block edge merged into one launch where
    // they can be)
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    const bool merged = can_merge(b, M_out);
    std::vector<MergedGroup> groups;
    if (merged) {
      vet_status su = upload_merged(b, kappa, S, f_out, M_out, groups);
      if (su != VET_OK) return su;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
    if (e) return batch_err(b, VET_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    vet_status st = VET_OK;
    e = cudaEventRecord(b->forked, b->origin);
    if (merged && !e) st = capture_merged(b, kappa, S, Ib, f_out, M_out, groups, e);
    for (int i = 0; !merged && i < b->n && !e && st == VET_OK; ++i) {
      if ((e = cudaStreamWaitEvent(b->branch[i], b->forked, 0))) break;
      vet_ctx *c = b->ctx[i];
      const bool timing = c->timing;
      c->timing = false;
      st = do_closure<float>(c, kappa[i], S[i], Ib ? Ib[i] : nullptr, f_out[i], M_out ? M_out[i] : nullptr,
                             b->branch[i], false);
      c->timing = timing;
      if (st != VET_OK) b->err = "grid " + std::to_string(i) + ": " + c->err;
      if (!e) e = cudaEventRecord(b->joined[i], b->branch[i]);
      if (!e) e = cudaStreamWaitEvent(b->origin, b->joined[i], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->origin, &graph);
    if (st != VET_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e || e2) {
      if (graph) cudaGraphDestroy(graph);
      return batch_err(b, VET_ECUDA, std::string("capture: ") + cudaGetErrorString(e ? e : e2));
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e) {
      b->exec = nullptr;
      return batch_err(b, VET_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    b->key = key;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e) return batch_err(b, VET_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  for (auto c : b->ctx) c->last_stream = (cudaStream_t)stream;
  return VET_OK;
}

VET_API vet_status vet_batch_sync(vet_batch *b) {
  if (!b) return VET_EINVAL;
  for (int i = 0; i < b->n; ++i) {
    vet_status st = vet_sync(b->ctx[i]);
    if (st != VET_OK) return batch_err(b, st, "grid " + std::to_string(i) + ": " + b->ctx[i]->err);
  }
  return VET_OK;
}

VET_API vet_status vet_batch_autotune(vet_batch *b, const float *const *kappa, const float *const *S,
                                      const float *const *Ib, void *stream) {
  if (!b || !kappa || !S) return VET_EINVAL;
  // one tuning per distinct grid shape, applied to every grid of that shape
  for (int i = 0; i < b->n; ++i) {
    const vet_ctx *ci = b->ctx[i];
    int j = 0;
    for (; j < i; ++j) {
      const vet_ctx *cj = b->ctx[j];
      if (cj->grid.nx == ci->grid.nx && cj->grid.ny == ci->grid.ny && cj->grid.nz == ci->grid.nz &&
          cj->grid.block == ci->grid.block && cj->N == ci->N)
        break;
    }
    vet_status st;
    if (j < i) {
      st = vet_set_tuning(b->ctx[i], b->ctx[j]->face_group, b->ctx[j]->dims.dir_tile);
    } else {
      st = vet_autotune(b->ctx[i], kappa[i], S[i], Ib ? Ib[i] : nullptr, nullptr, nullptr, stream);
    }
    if (st != VET_OK) return batch_err(b, st, "grid " + std::to_string(i) + ": " + b->ctx[i]->err);
  }
  if (b->exec) {  // tunings changed the launches: capture again on the next call
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return VET_OK;
}

VET_API const char *vet_batch_last_error(const vet_batch *b) { return b ? b->err.c_str() : ""; }

VET_API const char *vet_last_error(const vet_ctx *ctx) {
  if (!ctx) return g_create_err.c_str();
  return ctx->err.c_str();
}
