// vet_cnn.h -- launchers of the learned-closure kernels (vet_cnn.cu).
//
// Activation layout: cells-major, channels-minor, [volume][z][y][x][C] with
// C a multiple of 16 (BF16 rows of 32 or 64 bytes).  Network outputs are FP32
// rows of 16 (7 used).  Weights of a layer: [27][C_out][C_in] with
// tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); the data-gradient pass uses
// the flipped transpose Wt[tap][C_in][C_out] = W[26 - tap][C_out][C_in].
#pragma once

#include <cstddef>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace vet {
namespace cnn {

constexpr int kIn = 6;      // real input features
constexpr int kOut = 7;     // real outputs: D (6) and log error
constexpr int kInPad = 16;  // stored input channels
constexpr int kOutPad = 16; // stored output channels
constexpr int kHidden = 32; // hidden channels

// n volumes of nz x ny x nx cells.
struct Vol {
  int n, nz, ny, nx;
};

enum { EPI_SILU = 0, EPI_F32 = 1, EPI_SILU_BWD = 2 };

size_t wgrad_smem_bytes(int cin, int cout);
long long tiles(const Vol &V);

// out = epi(conv3d(x, W) + b) on the tcgen05 tensor cores (vet_cnn_tc.cu):
// tiles of 8 x 16 x 2 cells, accumulators in tensor memory.  Epilogues:
//   EPI_SILU:     pre = acc + b (stored BF16 if pre_out), out = SiLU(pre) BF16
//   EPI_F32:      out = acc + b, FP32
//   EPI_SILU_BWD: out = acc * SiLU'(pre_in) BF16 (data gradient through the
//                 previous layer's activation), no bias
// A bounded wait that gives up ORs 16 into *status (device) and the kernel
// returns early.
size_t conv_tc_smem_bytes(int cin, int cout);
template <int C_IN, int C_OUT, int EPI>
cudaError_t conv3d_tc(const __nv_bfloat16 *x, const __nv_bfloat16 *W, const float *b, const Vol &V,
                      __nv_bfloat16 *pre_out, const __nv_bfloat16 *pre_in, void *out, int *status, cudaStream_t st);

// gW[tap][co][ci] += sum_cells gpre[cell][co] x[cell + tap][ci], gb[co] +=
// sum_cells gpre[cell][co] (FP32, accumulated into the given arrays).
template <int C_IN, int C_OUT>
cudaError_t wgrad(const __nv_bfloat16 *x, const __nv_bfloat16 *gpre, const Vol &V, float *gW, float *gb, int grid,
                  cudaStream_t st);

// Features of the learned closure into x0 [cells][16] BF16; sums [n][2]
// (FP64, zeroed here) and bstat [n][blocks][2] are scratch.  feat_out
// (optional, [n][6][cells] FP32) receives the unrounded values.
cudaError_t features(const float *kappa, const float *S, const float *E, const Vol &V, int B, double h,
                     double *sums, float *bstat, __nv_bfloat16 *x0, float *feat_out, cudaStream_t st);

// Loss of the head against f_ref [n][6][cells] and its gradient go
// [cells][16] BF16.  mask (optional, [cells] u8) selects the cells that
// count; count (device) receives their number.  loss (device FP64) is
// overwritten.
cudaError_t head_loss(const float *o, const float *f_ref, const unsigned char *mask, const Vol &V, float lam,
                      unsigned long long *count, double *loss, __nv_bfloat16 *go, cudaStream_t st);

// One network layer's parameters inside the flat FP32 arrays, and its BF16
// copies for the forward (wb) and data-gradient (wt) passes.
struct LayerMeta {
  int cin, cout;          // stored (padded) channels
  int cin_real, cout_real;
  long long w_off, b_off; // offsets into the flat arrays
  __nv_bfloat16 *wb, *wt;
};
struct NetMeta {
  LayerMeta L[4];
  long long total;
};

// AdamW on every parameter (update != 0) and refresh of the BF16 copies.
cudaError_t adamw(const NetMeta &M, float *p, const float *g, float *m, float *v, float lr, float b1, float b2,
                  float eps, float wd, float bc1, float bc2, int update, cudaStream_t st);

// f = head(o) into f_out [6][cells] (one volume), indicator r into r_out
// (optional), flags[block] = 1 where some cell has r > thr.
cudaError_t indicator(const float *o, const Vol &V, int B, float thr, float *f_out, float *r_out,
                      unsigned int *flags, cudaStream_t st);

// list <- indices of the nonzero flags in increasing order, *count <- their
// number (one CTA).
cudaError_t compact_flags(const unsigned int *flags, int n, int *list, int *count, cudaStream_t st);

// Output rows [cells][16] FP32 -> [n][7][cells] FP32.
cudaError_t unpack_outputs(const float *o, const Vol &V, float *o_out, cudaStream_t st);

}  // namespace cnn
}  // namespace vet
