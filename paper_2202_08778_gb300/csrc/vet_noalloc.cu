// vet_noalloc.cu -- vet_closure_noalloc: the fused FP32 closure of
// vet_closure for callers that cannot allocate memory.
//
// Who needs it: code that runs while another framework's caching allocator
// holds nearly all device memory (cudaMalloc would fail), real-time loops that
// must not block on cudaMalloc / cudaFree (both can synchronise the device),
// and plug-ins whose host application forbids allocations outside its own
// pool.  Such callers own their input and output buffers but cannot give the
// library a workspace.
//
// How: every piece of workspace (direction templates, face-pass schedule,
// boundary and face intensities, E, the max-E word, the status word) lives in
// one file-scope device array of VET_NOALLOC_SCRATCH_BYTES that every GPU
// loading the library holds until the process exits; the host-side geometry
// is built in fixed static host arrays.  The array's device address is looked
// up once per device, on the first call made with that device selected.
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "vet.h"
#include "vet_geometry.h"
#include "vet_internal.h"

#define VET_API extern "C" __attribute__((visibility("default")))

namespace {

static __device__ __align__(256) unsigned char g_scratch[VET_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr int kMaxDirs = 192;            // nside <= 4
constexpr int kMaxEdge = 16;             // block edge <= 16
constexpr int kTplMax = 4096;            // bytes of one FP32 template at B <= 16
constexpr long long kMaxItems = 1 << 17; // face-pass items
constexpr int kMaxLevels = 4096;

std::mutex g_mutex;                     // one host thread stages at a time
void *g_addr[kMaxDevices];              // device address of g_scratch per device

// fixed host staging (no heap)
alignas(16) unsigned char h_tpl[kMaxDirs * kTplMax];
double h_dirs[kMaxDirs * 4];
int h_order[kMaxDirs], h_cell_order[kMaxDirs];
vet::FaceItem h_items[kMaxItems];
int h_level_off[kMaxLevels + 1];

vet_status fail(vet_status st, const std::string &msg) {
  vet::set_thread_error(("vet_closure_noalloc: " + msg).c_str());  // read by vet_last_error(NULL)
  return st;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

bool on_device(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Marks f as invalid (NaN) when a bounded device-side wait gave up: the call
// returns before its GPU work runs and has no context to report it later.
__global__ void poison_on_failure(const int *__restrict__ status, long long n, float *__restrict__ f) {
  if (*status == 0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    f[i] = __int_as_float(0x7fc00000);
}

}  // namespace

VET_API vet_status vet_closure_noalloc(const vet_grid *grid, const vet_config *cfg, const float *kappa,
                                       const float *S, const float *Ib, float *f_out, float *M_out, void *stream) {
  if (!grid || !cfg || !kappa || !S || !f_out) return fail(VET_EINVAL, "grid, cfg, kappa, S and f_out are required");
  const vet_grid g = *grid;
  if (cfg->precision != VET_FP32) return fail(VET_EINVAL, "only VET_FP32 is supported");
  if (g.block < 2 || g.block > kMaxEdge) return fail(VET_EINVAL, "block edge must be in 2..16");
  if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nx % g.block || g.ny % g.block || g.nz % g.block)
    return fail(VET_EINVAL, "grid extents must be positive multiples of the block edge");
  if (!(g.h > 0.0) || !std::isfinite(g.h)) return fail(VET_EINVAL, "cell edge h must be positive");
  if (cfg->nside < 1 || cfg->nside > 4 || (cfg->nside & (cfg->nside - 1)))
    return fail(VET_EINVAL, "nside must be 1, 2 or 4");
  const double qn = std::sqrt(cfg->rot_q[0] * cfg->rot_q[0] + cfg->rot_q[1] * cfg->rot_q[1] +
                              cfg->rot_q[2] * cfg->rot_q[2] + cfg->rot_q[3] * cfg->rot_q[3]);
  if (!(qn > 1e-12) || !std::isfinite(qn)) return fail(VET_EINVAL, "rotation quaternion is zero or not finite");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(VET_ECUDA, "no CUDA device");
  }
  if (cfg->device < 0 || cfg->device >= ndev || cfg->device >= kMaxDevices)
    return fail(VET_EINVAL, "device ordinal out of range");

  const int B = g.block, N = 12 * cfg->nside * cfg->nside;
  vet::GridDims dims{};
  dims.nx = g.nx;
  dims.ny = g.ny;
  dims.nz = g.nz;
  dims.B = B;
  dims.nbx = g.nx / B;
  dims.nby = g.ny / B;
  dims.nbz = g.nz / B;
  dims.nnode = (B + 1) * (B + 1);
  dims.fstride = vet::face_stride_elems<float>(B);
  dims.ndir = N;
  dims.ncell = (long long)g.nx * g.ny * g.nz;
  const long long nblk = (long long)dims.nbx * dims.nby * dims.nbz;
  const int nb[3] = {dims.nbx, dims.nby, dims.nbz};
  const int nlevels = nb[0] + nb[1] + nb[2] - 2;
  if (nlevels > kMaxLevels) return fail(VET_EINVAL, "too many blocks along the grid axes");
  const int tbytes = vet::tpl_layout<float>(B).bytes;
  if (tbytes > kTplMax) return fail(VET_EINVAL, "direction template larger than the static host staging slot");

  std::lock_guard<std::mutex> lock(g_mutex);

  // geometry, on the host, into the static arrays
  vet::geom::healpix_directions(cfg->nside, cfg->rot_q, h_dirs);
  int ob[9];
  vet::geom::internal_order(N, h_dirs, h_order, ob);
  for (int i = 0; i < N; ++i) {
    long long cs, ns[3];
    vet::geom::build_template<float>(h_dirs + 4 * h_order[i], h_order[i], B, g.h, h_tpl + (size_t)i * tbytes, cs,
                                     ns);
  }
  vet::geom::interleaved_order(ob, h_cell_order);
  const long long nitems = vet::geom::build_schedule(nb, ob, vet::kFaceGroup, h_items, kMaxItems, h_level_off);
  if (nitems < 0) return fail(VET_EINVAL, "grid has too many blocks for the static face-pass schedule");

  // workspace layout inside the static device array
  size_t off = 0;
  const size_t o_tpl = off;
  off = up256(off + (size_t)N * tbytes);
  const size_t o_items = off;
  off = up256(off + sizeof(vet::FaceItem) * (size_t)nitems);
  const size_t o_order = off;
  off = up256(off + sizeof(int) * N);
  const size_t o_bnd = off;
  off = up256(off + sizeof(float) * 6 * (size_t)N * dims.fstride);
  const size_t o_faces = off;
  const size_t faces_bytes = sizeof(float) * (size_t)N * nblk * 3 * dims.fstride;
  off = up256(off + faces_bytes);
  const size_t o_E = off;
  off = up256(off + (M_out ? 0 : sizeof(float) * (size_t)dims.ncell));
  const size_t o_emax = off;
  off = up256(off + 8);
  const size_t o_status = off;
  off = up256(off + sizeof(int));
  if (off > (size_t)VET_NOALLOC_SCRATCH_BYTES)
    return fail(VET_EINVAL, "problem needs " + std::to_string(off) + " bytes of workspace, more than the " +
                                std::to_string((size_t)VET_NOALLOC_SCRATCH_BYTES) +
                                " compiled into the library (use vet_create / vet_closure)");
  if (!on_device(kappa) || !on_device(S) || !on_device(f_out) || (Ib && !on_device(Ib)) ||
      (M_out && !on_device(M_out)))
    return fail(VET_EINVAL, "all field pointers must be device memory");

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return fail(VET_ECUDA, "cudaGetDevice failed");
  if (prev != cfg->device && cudaSetDevice(cfg->device) != cudaSuccess)
    return fail(VET_ECUDA, "cudaSetDevice failed");
  vet_status result = VET_OK;
  cudaError_t e = cudaSuccess;
  do {
    if (!g_addr[cfg->device]) {  // first call on this device: find the array
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) { result = fail(VET_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)); break; }
      e = vet::prepare_kernels();
      if (e != cudaSuccess) { result = fail(VET_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e)); break; }
      g_addr[cfg->device] = p;
    }
    unsigned char *base = static_cast<unsigned char *>(g_addr[cfg->device]);
    cudaStream_t st = (cudaStream_t)stream;
    auto *d_tpl = base + o_tpl;
    auto *d_items = reinterpret_cast<vet::FaceItem *>(base + o_items);
    auto *d_order = reinterpret_cast<int *>(base + o_order);
    auto *d_bnd = reinterpret_cast<float *>(base + o_bnd);
    auto *d_faces = reinterpret_cast<float *>(base + o_faces);
    auto *d_E = reinterpret_cast<float *>(base + o_E);
    void *d_emax = base + o_emax;
    auto *d_status = reinterpret_cast<int *>(base + o_status);
    // inputs of this call; the array keeps the previous call's contents, so
    // the face padding, max-E and status words are cleared explicitly
    if ((e = cudaMemcpyAsync(d_tpl, h_tpl, (size_t)N * tbytes, cudaMemcpyHostToDevice, st))) break;
    if ((e = cudaMemcpyAsync(d_items, h_items, sizeof(vet::FaceItem) * (size_t)nitems, cudaMemcpyHostToDevice, st)))
      break;
    if ((e = cudaMemcpyAsync(d_order, h_cell_order, sizeof(int) * N, cudaMemcpyHostToDevice, st))) break;
    if ((e = cudaMemsetAsync(d_faces, 0, faces_bytes, st))) break;
    if ((e = cudaMemsetAsync(d_emax, 0, 8, st))) break;
    if ((e = cudaMemsetAsync(d_status, 0, sizeof(int), st))) break;
    const long long spin = cfg->spin_limit > 0 ? cfg->spin_limit : (1LL << 22);
    if ((e = vet::launch_fill_boundary<float>(dims, d_tpl, Ib, d_bnd, st))) break;
    for (int L = 0; L < nlevels && !e; ++L)
      e = vet::launch_face_level<float>(dims, kappa, S, d_tpl, d_items + h_level_off[L],
                                        h_level_off[L + 1] - h_level_off[L], vet::kFaceGroup, d_faces, d_bnd, spin,
                                        d_status, st);
    if (e) break;
    if ((e = vet::launch_cell_pass<float>(dims, 0, kappa, S, d_tpl, d_order, d_faces, d_bnd, nullptr, M_out, d_E,
                                          f_out, d_emax, spin, d_status, st)))
      break;
    if ((e = vet::launch_floor_fix<float>(dims.ncell, M_out ? M_out : d_E, 1, d_emax, 1e-30, f_out, st))) break;
    poison_on_failure<<<152, 256, 0, st>>>(d_status, 6 * dims.ncell, f_out);
    e = cudaGetLastError();
  } while (false);
  if (result == VET_OK && e != cudaSuccess)
    result = fail(e == cudaErrorMemoryAllocation ? VET_ENOMEM : VET_ECUDA, cudaGetErrorString(e));
  if (prev >= 0 && prev != cfg->device) cudaSetDevice(prev);
  return result;
}
