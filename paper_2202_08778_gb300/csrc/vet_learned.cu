// vet_learned.cu -- host side of the learned closure: model parameters and
// optimiser state, activation workspace, the training entry points and
// vet_closure_learned (network + indicator + exact fallback on flagged
// blocks).  Kernels are in vet_cnn.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "vet.h"
#include "vet_bridge.h"
#include "vet_cnn.h"

#define VET_API extern "C" __attribute__((visibility("default")))

namespace cnn = vet::cnn;
using bf16 = __nv_bfloat16;

struct vet_model {
  int device = 0;
  int channels = cnn::kHidden;
  cnn::NetMeta meta{};
  long long host_params = 0;  // parameters in the host layout
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // flat FP32 (padded layout)
  bf16 *wb = nullptr, *wt = nullptr;                              // BF16 copies, all layers
  long long step = 0;
  // workspace
  long long cap_cells = 0;
  bool cap_train = false;
  bf16 *x0 = nullptr, *act[3] = {nullptr, nullptr, nullptr}, *pre[3] = {nullptr, nullptr, nullptr};
  bf16 *go = nullptr, *g1 = nullptr, *g2 = nullptr;
  float *o = nullptr, *r = nullptr;
  long long cap_vols = 0, cap_blocks = 0;
  double *sums = nullptr;
  float *bstat = nullptr;
  unsigned long long *count = nullptr;
  double *loss = nullptr;
  unsigned int *flags = nullptr;
  int *list = nullptr, *nlist = nullptr;
  int *h_nlist = nullptr;  // pinned
  int *status = nullptr;   // device: bounded waits of the tensor-core kernels that gave up
  // state of the current batch
  cnn::Vol V{0, 0, 0, 0};
  bool have_features = false, have_forward = false, have_backward = false;
  long long last_r_cells = 0;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool timed = false;
  std::string err;
};

namespace {

thread_local std::string g_model_err;

vet_status fail(vet_model *m, vet_status st, const std::string &msg) {
  if (m) m->err = msg;
  else g_model_err = msg;
  return st;
}

vet_status cuda_fail(vet_model *m, cudaError_t e, const char *what) {
  return fail(m, e == cudaErrorMemoryAllocation ? VET_ENOMEM : VET_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DevGuard {
  int prev = -1;
  bool ok = true;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool on_device(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_workspace(vet_model *m) {
  cudaFree(m->x0);
  for (int i = 0; i < 3; ++i) {
    cudaFree(m->act[i]);
    cudaFree(m->pre[i]);
    m->act[i] = m->pre[i] = nullptr;
  }
  cudaFree(m->go);
  cudaFree(m->g1);
  cudaFree(m->g2);
  cudaFree(m->o);
  cudaFree(m->r);
  m->x0 = m->go = m->g1 = m->g2 = nullptr;
  m->o = m->r = nullptr;
  m->cap_cells = 0;
  m->cap_train = false;
}

void free_model(vet_model *m) {
  if (!m) return;
  free_workspace(m);
  for (auto &e : m->ev)
    if (e) cudaEventDestroy(e);
  cudaFree(m->p);
  cudaFree(m->g);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->wb);
  cudaFree(m->wt);
  cudaFree(m->sums);
  cudaFree(m->bstat);
  cudaFree(m->count);
  cudaFree(m->loss);
  cudaFree(m->flags);
  cudaFree(m->list);
  cudaFree(m->nlist);
  cudaFree(m->status);
  cudaFreeHost(m->h_nlist);
  delete m;
}

// Activation workspace for `cells` cells; `train` adds what the backward pass
// needs (pre-activations, the third activation, gradient buffers).
// A request the current buffers cannot serve reallocates them for exactly
// that request.
vet_status ensure_cells(vet_model *m, long long cells, bool train) {
  if (cells <= m->cap_cells && (!train || m->cap_train)) return VET_OK;
  const bool want_train = train;
  const long long n = cells;
  cudaDeviceSynchronize();  // the old buffers may still be in use by enqueued work
  free_workspace(m);
  const size_t h16 = sizeof(bf16) * cnn::kInPad, h32 = sizeof(bf16) * cnn::kHidden;
  cudaError_t e = cudaMalloc((void **)&m->x0, n * h16);
  if (!e) e = cudaMalloc((void **)&m->act[0], n * h32);
  if (!e) e = cudaMalloc((void **)&m->act[1], n * h32);
  if (!e) e = cudaMalloc((void **)&m->o, n * sizeof(float) * cnn::kOutPad);
  if (!e) e = cudaMalloc((void **)&m->r, n * sizeof(float));
  if (!e && want_train) {
    e = cudaMalloc((void **)&m->act[2], n * h32);
    for (int i = 0; i < 3 && !e; ++i) e = cudaMalloc((void **)&m->pre[i], n * h32);
    if (!e) e = cudaMalloc((void **)&m->go, n * sizeof(bf16) * cnn::kOutPad);
    if (!e) e = cudaMalloc((void **)&m->g1, n * h32);
    if (!e) e = cudaMalloc((void **)&m->g2, n * h32);
  }
  if (e) {
    free_workspace(m);
    return cuda_fail(m, e, "cudaMalloc(activations)");
  }
  m->cap_cells = n;
  m->cap_train = want_train;
  return VET_OK;
}

vet_status ensure_small(vet_model *m, long long vols, long long blocks) {
  cudaError_t e = cudaSuccess;
  if (vols > m->cap_vols) {
    cudaDeviceSynchronize();
    cudaFree(m->sums);
    m->sums = nullptr;
    if ((e = cudaMalloc((void **)&m->sums, sizeof(double) * 2 * vols))) return cuda_fail(m, e, "cudaMalloc(sums)");
    m->cap_vols = vols;
  }
  if (blocks > m->cap_blocks) {
    cudaDeviceSynchronize();
    cudaFree(m->bstat);
    cudaFree(m->flags);
    cudaFree(m->list);
    m->bstat = nullptr;
    m->flags = nullptr;
    m->list = nullptr;
    e = cudaMalloc((void **)&m->bstat, sizeof(float) * 2 * blocks);
    if (!e) e = cudaMalloc((void **)&m->flags, sizeof(unsigned int) * blocks);
    if (!e) e = cudaMalloc((void **)&m->list, sizeof(int) * blocks);
    if (e) return cuda_fail(m, e, "cudaMalloc(block tables)");
    m->cap_blocks = blocks;
  }
  return VET_OK;
}

// Host layout <-> padded device layout.
void host_to_padded(const vet_model *m, const float *src, std::vector<float> &dst) {
  dst.assign((size_t)m->meta.total, 0.f);
  long long k = 0;
  for (int l = 0; l < 4; ++l) {
    const cnn::LayerMeta &L = m->meta.L[l];
    for (int t = 0; t < 27; ++t)
      for (int co = 0; co < L.cout_real; ++co)
        for (int ci = 0; ci < L.cin_real; ++ci) dst[L.w_off + ((long long)t * L.cout + co) * L.cin + ci] = src[k++];
    for (int co = 0; co < L.cout_real; ++co) dst[L.b_off + co] = src[k++];
  }
}

void padded_to_host(const vet_model *m, const std::vector<float> &src, float *dst) {
  long long k = 0;
  for (int l = 0; l < 4; ++l) {
    const cnn::LayerMeta &L = m->meta.L[l];
    for (int t = 0; t < 27; ++t)
      for (int co = 0; co < L.cout_real; ++co)
        for (int ci = 0; ci < L.cin_real; ++ci) dst[k++] = src[L.w_off + ((long long)t * L.cout + co) * L.cin + ci];
    for (int co = 0; co < L.cout_real; ++co) dst[k++] = src[L.b_off + co];
  }
}

const bf16 *W(const vet_model *m, int l) { return m->meta.L[l].wb; }
const bf16 *Wt(const vet_model *m, int l) { return m->meta.L[l].wt; }
const float *bias(const vet_model *m, int l) { return m->p + m->meta.L[l].b_off; }
float *gW(const vet_model *m, int l) { return m->g + m->meta.L[l].w_off; }
float *gb(const vet_model *m, int l) { return m->g + m->meta.L[l].b_off; }

// The four convolutions; with `train` the pre-activations and all three
// hidden activations are kept, otherwise two buffers alternate.
cudaError_t run_forward(vet_model *m, const cnn::Vol &V, bool train, cudaStream_t st) {
  using namespace cnn;
  cudaError_t e;
  bf16 *a0 = m->act[0], *a1 = m->act[1], *a2 = train ? m->act[2] : m->act[0];
  int *sts = m->status;
  e = conv3d_tc<kInPad, kHidden, EPI_SILU>(m->x0, W(m, 0), bias(m, 0), V, train ? m->pre[0] : nullptr, nullptr, a0,
                                          sts, st);
  if (!e)
    e = conv3d_tc<kHidden, kHidden, EPI_SILU>(a0, W(m, 1), bias(m, 1), V, train ? m->pre[1] : nullptr, nullptr, a1,
                                              sts, st);
  if (!e)
    e = conv3d_tc<kHidden, kHidden, EPI_SILU>(a1, W(m, 2), bias(m, 2), V, train ? m->pre[2] : nullptr, nullptr, a2,
                                              sts, st);
  if (!e) e = conv3d_tc<kHidden, kOutPad, EPI_F32>(a2, W(m, 3), bias(m, 3), V, nullptr, nullptr, m->o, sts, st);
  return e;
}

}  // namespace

VET_API vet_status vet_model_create(vet_model **out, int channels, int device) {
  if (!out) return fail(nullptr, VET_EINVAL, "out is NULL");
  *out = nullptr;
  if (channels != cnn::kHidden) return fail(nullptr, VET_EUNSUPPORTED, "only 32 hidden channels are supported");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(nullptr, VET_ECUDA, "no CUDA device");
  }
  if (device < 0 || device >= ndev) return fail(nullptr, VET_EINVAL, "device ordinal out of range");
  vet_model *m = new (std::nothrow) vet_model;
  if (!m) return fail(nullptr, VET_ENOMEM, "host allocation failed");
  m->device = device;
  m->channels = channels;
  const int cin_p[4] = {cnn::kInPad, cnn::kHidden, cnn::kHidden, cnn::kHidden};
  const int cout_p[4] = {cnn::kHidden, cnn::kHidden, cnn::kHidden, cnn::kOutPad};
  const int cin_r[4] = {cnn::kIn, channels, channels, channels};
  const int cout_r[4] = {channels, channels, channels, cnn::kOut};
  long long off = 0, woff = 0, hp = 0;
  long long wofs[4];
  for (int l = 0; l < 4; ++l) {
    cnn::LayerMeta &L = m->meta.L[l];
    L.cin = cin_p[l];
    L.cout = cout_p[l];
    L.cin_real = cin_r[l];
    L.cout_real = cout_r[l];
    L.w_off = off;
    off += 27LL * L.cout * L.cin;
    L.b_off = off;
    off += L.cout;
    wofs[l] = woff;
    woff += 27LL * L.cout * L.cin;
    hp += 27LL * cout_r[l] * cin_r[l] + cout_r[l];
  }
  m->meta.total = off;
  m->host_params = hp;
  DevGuard dg(device);
  if (!dg.ok) {
    delete m;
    return fail(nullptr, VET_ECUDA, "cudaSetDevice failed");
  }
  cudaError_t e = cudaSuccess;
  for (float **ptr : {&m->p, &m->g, &m->m, &m->v})
    if (!e) e = cudaMalloc((void **)ptr, sizeof(float) * off);
  if (!e) e = cudaMalloc((void **)&m->wb, sizeof(bf16) * woff);
  if (!e) e = cudaMalloc((void **)&m->wt, sizeof(bf16) * woff);
  if (!e) e = cudaMalloc((void **)&m->count, sizeof(unsigned long long));
  if (!e) e = cudaMalloc((void **)&m->loss, sizeof(double));
  if (!e) e = cudaMalloc((void **)&m->nlist, sizeof(int));
  if (!e) e = cudaMalloc((void **)&m->status, sizeof(int));
  if (!e) e = cudaMemset(m->status, 0, sizeof(int));
  if (!e) e = cudaMallocHost((void **)&m->h_nlist, sizeof(int));
  for (int i = 0; i < 5 && !e; ++i) e = cudaEventCreate(&m->ev[i]);
  for (float *ptr : {m->p, m->g, m->m, m->v})
    if (!e) e = cudaMemset(ptr, 0, sizeof(float) * off);
  if (!e) e = cudaMemset(m->wb, 0, sizeof(bf16) * woff);
  if (!e) e = cudaMemset(m->wt, 0, sizeof(bf16) * woff);
  if (e) {
    g_model_err = std::string("model allocation: ") + cudaGetErrorString(e);
    free_model(m);
    return e == cudaErrorMemoryAllocation ? VET_ENOMEM : VET_ECUDA;
  }
  for (int l = 0; l < 4; ++l) {
    m->meta.L[l].wb = m->wb + wofs[l];
    m->meta.L[l].wt = m->wt + wofs[l];
  }
  *out = m;
  return VET_OK;
}

VET_API vet_status vet_model_destroy(vet_model *model) {
  if (!model) return VET_OK;
  DevGuard dg(model->device);
  free_model(model);
  return VET_OK;
}

VET_API long long vet_model_num_params(const vet_model *model) { return model ? model->host_params : -1; }

VET_API vet_status vet_model_set_params(vet_model *m, const float *params) {
  if (!m || !params) return fail(m, VET_EINVAL, "model and params are required");
  DevGuard dg(m->device);
  std::vector<float> pad;
  host_to_padded(m, params, pad);
  cudaError_t e = cudaMemcpy(m->p, pad.data(), sizeof(float) * pad.size(), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemset(m->m, 0, sizeof(float) * m->meta.total);
  if (!e) e = cudaMemset(m->v, 0, sizeof(float) * m->meta.total);
  if (!e) e = cnn::adamw(m->meta, m->p, m->g, m->m, m->v, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, 0, nullptr);
  if (!e) e = cudaDeviceSynchronize();
  if (e) return cuda_fail(m, e, "set_params");
  m->step = 0;
  return VET_OK;
}

// Reads and clears the device status word (after a synchronisation).
static vet_status check_status(vet_model *m) {
  int sts = 0;
  cudaError_t e = cudaMemcpy(&sts, m->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e) return cuda_fail(m, e, "status read");
  if (sts) {
    cudaMemset(m->status, 0, sizeof(int));
    return fail(m, VET_ETIMEOUT, "a tensor-core wait gave up (status " + std::to_string(sts) + "); outputs are incomplete");
  }
  return VET_OK;
}

static vet_status copy_flat(vet_model *m, const float *src, float *dst) {
  DevGuard dg(m->device);
  std::vector<float> pad((size_t)m->meta.total);
  cudaError_t e = cudaDeviceSynchronize();
  if (!e) e = cudaMemcpy(pad.data(), src, sizeof(float) * pad.size(), cudaMemcpyDeviceToHost);
  if (e) return cuda_fail(m, e, "parameter read");
  vet_status s = check_status(m);
  if (s) return s;
  padded_to_host(m, pad, dst);
  return VET_OK;
}

VET_API vet_status vet_model_get_params(vet_model *m, float *params) {
  if (!m || !params) return fail(m, VET_EINVAL, "model and params are required");
  return copy_flat(m, m->p, params);
}

VET_API vet_status vet_model_get_grads(vet_model *m, float *grads) {
  if (!m || !grads) return fail(m, VET_EINVAL, "model and grads are required");
  if (!m->have_backward) return fail(m, VET_EINVAL, "no backward pass has run");
  return copy_flat(m, m->g, grads);
}

// Model files: the 8-byte tag "VETMODL1", int32 hidden channels, int32 0,
// int64 parameter count, int64 AdamW step count, then three FP32 arrays in
// the host parameter layout: the parameters and AdamW's first and second
// moments.  Little-endian, as both host architectures store them.
namespace {
constexpr char kModelTag[8] = {'V', 'E', 'T', 'M', 'O', 'D', 'L', '1'};
struct ModelFileHead {
  char tag[8];
  int32_t channels, zero;
  int64_t nparams, step;
};
static_assert(sizeof(ModelFileHead) == 32, "model file head");
}  // namespace

VET_API vet_status vet_model_save(vet_model *m, const char *path) {
  if (!m || !path) return fail(m, VET_EINVAL, "model and path are required");
  const size_t n = (size_t)m->host_params;
  std::vector<float> buf(3 * n);
  vet_status s = copy_flat(m, m->p, buf.data());
  if (!s) s = copy_flat(m, m->m, buf.data() + n);
  if (!s) s = copy_flat(m, m->v, buf.data() + 2 * n);
  if (s) return s;
  ModelFileHead h{};
  std::memcpy(h.tag, kModelTag, sizeof h.tag);
  h.channels = m->channels;
  h.nparams = (int64_t)n;
  h.step = (int64_t)m->step;
  FILE *f = std::fopen(path, "wb");
  if (!f) return fail(m, VET_EINVAL, std::string("cannot open ") + path + " for writing");
  const bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 && std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) return fail(m, VET_EINVAL, std::string("write to ") + path + " failed");
  return VET_OK;
}

VET_API vet_status vet_model_load(vet_model *m, const char *path) {
  if (!m || !path) return fail(m, VET_EINVAL, "model and path are required");
  FILE *f = std::fopen(path, "rb");
  if (!f) return fail(m, VET_EINVAL, std::string("cannot open ") + path);
  ModelFileHead h{};
  const size_t n = (size_t)m->host_params;
  std::vector<float> buf(3 * n);
  bool ok = std::fread(&h, sizeof h, 1, f) == 1;
  std::string why;
  if (!ok || std::memcmp(h.tag, kModelTag, sizeof h.tag) != 0) why = "not a libvet model file";
  else if (h.channels != m->channels) why = "file has " + std::to_string(h.channels) + " hidden channels, model has " + std::to_string(m->channels);
  else if (h.nparams != (int64_t)n || h.step < 0) why = "parameter count does not match";
  else if (std::fread(buf.data(), sizeof(float), buf.size(), f) != buf.size()) why = "file is truncated";
  std::fclose(f);
  if (!why.empty()) return fail(m, VET_EINVAL, std::string(path) + ": " + why);
  vet_status s = vet_model_set_params(m, buf.data());  // also refreshes the BF16 copies
  if (s) return s;
  DevGuard dg(m->device);
  std::vector<float> pad;
  host_to_padded(m, buf.data() + n, pad);
  cudaError_t e = cudaMemcpy(m->m, pad.data(), sizeof(float) * pad.size(), cudaMemcpyHostToDevice);
  if (!e) {
    host_to_padded(m, buf.data() + 2 * n, pad);
    e = cudaMemcpy(m->v, pad.data(), sizeof(float) * pad.size(), cudaMemcpyHostToDevice);
  }
  if (e) return cuda_fail(m, e, "optimiser state upload");
  m->step = (long long)h.step;
  return VET_OK;
}

VET_API vet_status vet_model_features(vet_model *m, const vet_grid *grid, int nvol, const float *kappa,
                                      const float *S, const float *E, float *feat_out, void *stream) {
  if (!m || !grid) return fail(m, VET_EINVAL, "model and grid are required");
  const vet_grid g = *grid;
  if (nvol < 1 || g.block < 1 || g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nx % g.block || g.ny % g.block ||
      g.nz % g.block)
    return fail(m, VET_EINVAL, "extents must be positive multiples of the block edge, nvol >= 1");
  if (!(g.h > 0.0) || !std::isfinite(g.h)) return fail(m, VET_EINVAL, "cell edge h must be positive");
  DevGuard dg(m->device);
  if (!on_device(kappa) || !on_device(S) || !on_device(E) || (feat_out && !on_device(feat_out)))
    return fail(m, VET_EINVAL, "kappa, S, E (and feat_out) must be device pointers");
  const cnn::Vol V{nvol, g.nz, g.ny, g.nx};
  const long long cells = (long long)nvol * g.nx * g.ny * g.nz;
  const long long blocks = (long long)nvol * (g.nx / g.block) * (g.ny / g.block) * (g.nz / g.block);
  vet_status s = ensure_cells(m, cells, true);
  if (!s) s = ensure_small(m, nvol, blocks);
  if (s) return s;
  cudaError_t e = cnn::features(kappa, S, E, V, g.block, g.h, m->sums, m->bstat, m->x0, feat_out, (cudaStream_t)stream);
  if (e) return cuda_fail(m, e, "features launch");
  m->V = V;
  m->have_features = true;
  m->have_forward = m->have_backward = false;
  return VET_OK;
}

VET_API vet_status vet_model_forward(vet_model *m, float *o_out, void *stream) {
  if (!m) return VET_EINVAL;
  if (!m->have_features) return fail(m, VET_EINVAL, "no features: call vet_model_features first");
  DevGuard dg(m->device);
  if (o_out && !on_device(o_out)) return fail(m, VET_EINVAL, "o_out must be a device pointer");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = run_forward(m, m->V, true, st);
  if (!e && o_out) e = cnn::unpack_outputs(m->o, m->V, o_out, st);
  if (e) return cuda_fail(m, e, "forward launch");
  m->have_forward = true;
  return VET_OK;
}

VET_API vet_status vet_model_backward(vet_model *m, const float *f_ref, const uint8_t *mask, float lam,
                                      double *loss_out, void *stream) {
  using namespace cnn;
  if (!m || !f_ref) return fail(m, VET_EINVAL, "model and f_ref are required");
  if (!m->have_forward) return fail(m, VET_EINVAL, "no forward pass: call vet_model_forward first");
  if (!(lam >= 0.f) || !std::isfinite(lam)) return fail(m, VET_EINVAL, "lam must be finite and >= 0");
  DevGuard dg(m->device);
  if (!on_device(f_ref) || (mask && !on_device(mask)) || (loss_out && !on_device(loss_out)))
    return fail(m, VET_EINVAL, "f_ref, mask and loss_out must be device pointers");
  cudaStream_t st = (cudaStream_t)stream;
  const Vol &V = m->V;
  cudaError_t e = cudaMemsetAsync(m->g, 0, sizeof(float) * m->meta.total, st);
  if (!e) e = head_loss(m->o, f_ref, mask, V, lam, m->count, m->loss, m->go, st);
  // layer 4: gradient of its output is go
  if (!e) e = wgrad<kHidden, kOutPad>(m->act[2], m->go, V, gW(m, 3), gb(m, 3), 0, st);
  if (!e) e = conv3d_tc<kOutPad, kHidden, EPI_SILU_BWD>(m->go, Wt(m, 3), nullptr, V, nullptr, m->pre[2], m->g1, m->status, st);
  // layer 3
  if (!e) e = wgrad<kHidden, kHidden>(m->act[1], m->g1, V, gW(m, 2), gb(m, 2), 0, st);
  if (!e) e = conv3d_tc<kHidden, kHidden, EPI_SILU_BWD>(m->g1, Wt(m, 2), nullptr, V, nullptr, m->pre[1], m->g2, m->status, st);
  // layer 2
  if (!e) e = wgrad<kHidden, kHidden>(m->act[0], m->g2, V, gW(m, 1), gb(m, 1), 0, st);
  if (!e) e = conv3d_tc<kHidden, kHidden, EPI_SILU_BWD>(m->g2, Wt(m, 1), nullptr, V, nullptr, m->pre[0], m->g1, m->status, st);
  // layer 1 (its input gradient is not needed)
  if (!e) e = wgrad<kInPad, kHidden>(m->x0, m->g1, V, gW(m, 0), gb(m, 0), 0, st);
  if (!e && loss_out) e = cudaMemcpyAsync(loss_out, m->loss, sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e) return cuda_fail(m, e, "backward launch");
  m->have_backward = true;
  return VET_OK;
}

VET_API vet_status vet_model_step(vet_model *m, float lr, float beta1, float beta2, float eps, float weight_decay,
                                  void *stream) {
  if (!m) return VET_EINVAL;
  if (!m->have_backward) return fail(m, VET_EINVAL, "no gradients: call vet_model_backward first");
  if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) ||
      !(weight_decay >= 0.f))
    return fail(m, VET_EINVAL, "need lr >= 0, 0 <= beta < 1, eps > 0, weight_decay >= 0");
  DevGuard dg(m->device);
  m->step += 1;
  const float bc1 = (float)(1.0 - std::pow((double)beta1, (double)m->step));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, (double)m->step));
  cudaError_t e = cnn::adamw(m->meta, m->p, m->g, m->m, m->v, lr, beta1, beta2, eps, weight_decay, bc1, bc2, 1,
                             (cudaStream_t)stream);
  if (e) return cuda_fail(m, e, "adamw launch");
  return VET_OK;
}

VET_API vet_status vet_closure_learned(vet_ctx *ctx, vet_model *m, const float *kappa, const float *S,
                                       const float *E, const float *Ib, float threshold, float *f_out,
                                       uint32_t *block_flags_out, int *n_fallback_out, void *stream) {
  if (!ctx || !m) return fail(m, VET_EINVAL, "ctx and model are required");
  const vet::CtxInfo ci = vet::ctx_info(ctx);
  if (ci.fp64) return fail(m, VET_EINVAL, "the learned closure needs an FP32 context");
  if (ci.device != m->device) return fail(m, VET_EINVAL, "context and model are on different devices");
  if (!kappa || !S || !E || !f_out) return fail(m, VET_EINVAL, "kappa, S, E and f_out are required");
  if (!(threshold >= 0.f)) return fail(m, VET_EINVAL, "threshold must be >= 0");
  DevGuard dg(m->device);
  if (!on_device(kappa) || !on_device(S) || !on_device(E) || !on_device(f_out) || (Ib && !on_device(Ib)) ||
      (block_flags_out && !on_device(block_flags_out)))
    return fail(m, VET_EINVAL, "field pointers must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  const vet_grid g = ci.grid;
  const cnn::Vol V{1, g.nz, g.ny, g.nx};
  const long long cells = (long long)g.nx * g.ny * g.nz;
  vet_status s = ensure_cells(m, cells, false);
  if (!s) s = ensure_small(m, 1, ci.nblk);
  if (s) return s;
  m->timed = false;
  cudaError_t e = cudaEventRecord(m->ev[0], st);
  if (!e) e = cnn::features(kappa, S, E, V, g.block, g.h, m->sums, m->bstat, m->x0, nullptr, st);
  if (!e) e = cudaEventRecord(m->ev[3], st);
  if (!e) e = run_forward(m, V, false, st);
  if (!e) e = cudaEventRecord(m->ev[4], st);
  if (!e) e = cnn::indicator(m->o, V, g.block, threshold, f_out, m->r, m->flags, st);
  if (!e) e = cnn::compact_flags(m->flags, ci.nblk, m->list, m->nlist, st);
  if (!e && block_flags_out)
    e = cudaMemcpyAsync(block_flags_out, m->flags, sizeof(unsigned int) * ci.nblk, cudaMemcpyDeviceToDevice, st);
  if (!e) e = cudaMemcpyAsync(m->h_nlist, m->nlist, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaEventRecord(m->ev[1], st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return cuda_fail(m, e, "learned closure");
  vet_status s2 = check_status(m);
  if (s2) return s2;
  // the features, activations and flags of this call replace the training batch's
  m->have_features = m->have_forward = m->have_backward = false;
  m->last_r_cells = cells;
  const int nfb = *m->h_nlist;
  if (n_fallback_out) *n_fallback_out = nfb;
  if (nfb > 0) {
    s = vet::exact_on_blocks(ctx, kappa, S, Ib, m->list, nfb, f_out, st);
    if (s) return fail(m, s, std::string("fallback: ") + vet_last_error(ctx));
  }
  e = cudaEventRecord(m->ev[2], st);
  if (e) return cuda_fail(m, e, "cudaEventRecord");
  m->timed = true;
  return VET_OK;
}

VET_API vet_status vet_model_last_timing(vet_model *m, float ms[4]) {
  if (!m || !ms) return VET_EINVAL;
  if (!m->timed) return fail(m, VET_EINVAL, "no timed learned closure");
  DevGuard dg(m->device);
  cudaError_t e = cudaEventSynchronize(m->ev[2]);
  if (!e) e = cudaEventElapsedTime(&ms[0], m->ev[0], m->ev[1]);
  if (!e) e = cudaEventElapsedTime(&ms[1], m->ev[1], m->ev[2]);
  if (!e) e = cudaEventElapsedTime(&ms[2], m->ev[0], m->ev[2]);
  if (!e) e = cudaEventElapsedTime(&ms[3], m->ev[3], m->ev[4]);
  if (e) return cuda_fail(m, e, "event timing");
  return VET_OK;
}

VET_API vet_status vet_model_last_indicator(vet_model *m, float *r_out, void *stream) {
  if (!m || !r_out) return fail(m, VET_EINVAL, "model and r_out are required");
  if (!m->last_r_cells) return fail(m, VET_EINVAL, "no learned closure has run");
  DevGuard dg(m->device);
  if (!on_device(r_out)) return fail(m, VET_EINVAL, "r_out must be a device pointer");
  cudaError_t e = cudaMemcpyAsync(r_out, m->r, sizeof(float) * m->last_r_cells, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream);
  if (e) return cuda_fail(m, e, "indicator copy");
  return VET_OK;
}

VET_API const char *vet_model_last_error(const vet_model *m) {
  if (!m) return g_model_err.c_str();
  return m->err.c_str();
}
