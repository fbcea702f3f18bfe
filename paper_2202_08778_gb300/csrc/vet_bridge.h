// vet_bridge.h -- what the learned closure (vet_learned.cu) uses of a closure
// context (vet_host.cu), whose layout stays private to vet_host.cu.
#pragma once

#include <cuda_runtime.h>

#include "vet.h"

namespace vet {

struct CtxInfo {
  vet_grid grid;
  int ndir;
  int nblk;
  bool fp64;
  int device;
};

CtxInfo ctx_info(const vet_ctx *c);

// Sets the context's error message and returns st.
vet_status ctx_fail(vet_ctx *c, vet_status st, const char *msg);

// The exact closure on the listed blocks of an FP32 context: the face pass
// over the whole grid (every block's upwind faces are needed), then the cell
// pass and the floor rule on the cells of the nlist blocks in d_list (device).
// f_out rows of those cells are overwritten; the others are left alone.  All
// pointers are device pointers; Ib may be NULL (vacuum).  Asynchronous on st;
// device-side timeouts are latched and reported by vet_sync.
vet_status exact_on_blocks(vet_ctx *c, const float *kappa, const float *S, const float *Ib, const int *d_list,
                           int nlist, float *f_out, cudaStream_t st);

}  // namespace vet
