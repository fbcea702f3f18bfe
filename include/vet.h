/*
 * vet.h -- C ABI of libvet, a GB300 (sm_103a) implementation of the
 * non-local Variable Eddington Tensor (VET) closure of VETTAM
 * (Menon, Federrath, Krumholz, Kuiper, Wibking & Jung 2022, MNRAS;
 * arXiv 2202.08778).
 *
 * The closure is the paper's Sec. 2.2.5 ("Computing the Eddington Tensor"):
 *   1. solve the time-independent gray transfer equation
 *        dI/ds = kappa (S - I)                                  (Eq. 14)
 *      along a HEALPix set of N = 12 nside^2 directions (Sec. 2.2.5, App. B)
 *      with hybrid characteristics (long characteristics inside cubic blocks,
 *      bilinear interpolation of face intensities between blocks);
 *   2. take the angular quadratures (Eqs. 10-12 and the discrete sums of
 *      Sec. 2.2.5, with c = 1)
 *        E = sum_k w_k I_k,  F_i = sum_k w_k I_k n_ik,
 *        P_ij = sum_k w_k I_k n_ik n_jk,   w_k = 4 pi / N;
 *   3. form the Eddington tensor f_ij = P_ij / E                (Eq. 13).
 *
 * Conventions shared by every entry point
 *   - kappa is the absorption coefficient per unit length (the paper's
 *     rho kappa_P); h (cell edge) is in the same length unit.
 *   - Cell fields are [nz][ny][nx] row-major, x fastest.
 *   - Boundary intensities Ib are [6][N]: one constant per domain face and
 *     direction, faces ordered x-low, x-high, y-low, y-high, z-low, z-high.
 *     NULL means vacuum (Ib = 0).
 *   - Direction k is the k-th HEALPix ring-scheme pixel centre (ring by ring
 *     from the north pole, increasing azimuth), rotated by the configured
 *     quaternion.  vet_directions() returns the table.
 *   - Moments are [10][cells]: E, Fx, Fy, Fz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz.
 *   - The tensor f is [6][cells]: xx, yy, zz, xy, xz, yz.  Where E does not
 *     exceed 1e-30 times the grid's largest E (no radiation arrives, or it
 *     underflowed), f is the isotropic tensor I/3.
 *   - Field pointers may be device memory or host memory (pageable or
 *     pinned); the library detects which with cudaPointerGetAttributes and
 *     stages host data through its own device buffers.  The caller owns all
 *     field memory; the context owns its workspace.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous for device pointers.  Calls given host
 *     pointers synchronise the stream before returning.
 *   - Argument errors are returned at once and nothing is enqueued.  A
 *     failure of an enqueued kernel is reported by the next call or by
 *     vet_sync().  vet_last_error() gives a message for the last failure on
 *     the context.
 *   - A context is not thread-safe: calls on one context must not overlap.
 */
#ifndef VET_H
#define VET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VET_OK = 0,
  VET_EINVAL = 1,       /* bad argument (null pointer, size, precision) */
  VET_ENOMEM = 2,       /* device or host allocation failed */
  VET_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  VET_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
  VET_EUNSUPPORTED = 5  /* valid request the library cannot serve */
} vet_status;

#define VET_FP32 0 /* float fields, FP32 ray march and moments */
#define VET_FP64 1 /* double fields, FP64 everywhere */

/* Uniform grid of nx x ny x nz cells of edge h, cut into cubic blocks of
 * `block` cells per edge; block must divide nx, ny and nz.  Hybrid
 * characteristics run long characteristics inside each block
 * (Sec. 2.2.5, via Buntemeyer et al. 2016). */
typedef struct {
  int nx, ny, nz;
  int block; /* 2..32 */
  double h;  /* > 0 */
} vet_grid;

/* Direction set and arithmetic.  nside is the HEALPix resolution (a power of
 * two, 1..16; N = 12 nside^2).  rot_q is a quaternion (w, x, y, z) applied to
 * every direction, the paper's random rotation of the HEALPix set
 * (Sec. 2.2.5); it is normalised internally, (1,0,0,0) means no rotation. */
typedef struct {
  int nside;
  double rot_q[4];
  int precision;        /* VET_FP32 or VET_FP64 */
  int device;           /* CUDA device ordinal the context works on */
  long long spin_limit; /* polls per device-side wait before it gives up and
                           the call reports VET_ETIMEOUT; 0 = default (2^22) */
} vet_config;

typedef struct vet_ctx vet_ctx;

/* Create a context: validates grid and config, builds the direction set and
 * the per-direction ray templates, allocates the face-intensity workspace
 * (N x blocks x 3 x about (block+2)^2 values).  *out is NULL on failure. */
vet_status vet_create(vet_ctx **out, const vet_grid *grid, const vet_config *cfg);

/* Release the context and all its device memory.  NULL is accepted. */
vet_status vet_destroy(vet_ctx *ctx);

/* Number of directions N, or -1 for a NULL context. */
int vet_num_directions(const vet_ctx *ctx);

/* Copy the direction table to host memory dirs_out[N][4] = (nx, ny, nz, w),
 * FP64, in the documented HEALPix order. */
vet_status vet_directions(const vet_ctx *ctx, double *dirs_out);

/* Formal solution of Eq. 14 for all N directions (Sec. 2.2.5):
 * I_out[N][cells] = cell-centre intensities.  FP32 context only. */
vet_status vet_trace(vet_ctx *ctx, const float *kappa, const float *S, const float *Ib, float *I_out,
                     void *stream);

/* Angular quadratures of given intensities (Eqs. 10-12, c = 1):
 * I[N][cells] -> M_out[10][cells].  E64_out (optional, NULL to skip; DEVICE
 * memory, [cells]) also receives E summed in FP64 (the weights are all
 * 4 pi / N, so E64 = (4 pi / N) sum_k I_k accumulated in double), for callers
 * that guard f where E is far below its neighbours.  FP32 context only;
 * VET_EINVAL if E64_out is not device memory. */
vet_status vet_moments(vet_ctx *ctx, const float *I, float *M_out, double *E64_out, void *stream);

/* Whole closure, fused: trace + quadratures + f = P/E (Eq. 13) without
 * storing I.  f_out[6][cells] required; M_out[10][cells] optional (NULL).
 * FP32 context only. */
vet_status vet_closure(vet_ctx *ctx, const float *kappa, const float *S, const float *Ib, float *f_out,
                       float *M_out, void *stream);

/* The same three operations on double fields, FP64 context only. */
vet_status vet_trace_f64(vet_ctx *ctx, const double *kappa, const double *S, const double *Ib,
                         double *I_out, void *stream);
vet_status vet_moments_f64(vet_ctx *ctx, const double *I, double *M_out, void *stream);
vet_status vet_closure_f64(vet_ctx *ctx, const double *kappa, const double *S, const double *Ib,
                           double *f_out, double *M_out, void *stream);

/* Wait for the context's last enqueued work and report any device error:
 * VET_ECUDA for a CUDA fault, VET_ETIMEOUT when a bounded device-side wait
 * (a kernel waiting for its staged data) gave up; the outputs of that call are
 * then incomplete.  The context stays usable either way. */
vet_status vet_sync(vet_ctx *ctx);

/* Work measure of one closure, from the ray templates: the number of
 * cell-ray segments and face-node-ray segments (one exponential each)
 * summed over all cells, face nodes (three downwind faces per block) and
 * directions.  The face pass skips the downwind faces that lie on the
 * domain boundary (no block reads them), so it executes a little less. */
vet_status vet_work_counts(const vet_ctx *ctx, long long *cell_segments, long long *face_segments);

/* Per-phase device timing.  After vet_set_timing(ctx, 1), every vet_trace /
 * vet_closure call records CUDA events on its stream around its phases;
 * vet_last_timing() waits for the last call's events and writes, in
 * milliseconds: ms[0] the face pass (all wavefront levels), ms[1] the cell
 * pass (rays, quadratures and f), ms[2] the closing step (floor rule), ms[3]
 * the whole call.  Timing is off by default. */
vet_status vet_set_timing(vet_ctx *ctx, int enable);
vet_status vet_last_timing(vet_ctx *ctx, float ms[4]);

/* Kernel launches one vet_closure call makes (its work is split into this
 * many kernels: the boundary fill, one per wavefront level of the face pass,
 * the cell pass and the closing step). */
int vet_launches_per_closure(const vet_ctx *ctx);

/* Performance tunables of the two passes (autotuned; the paper has no
 * counterpart -- its tracer runs on CPUs):
 *   face_group -- directions of one octant per face-pass work item, 1..8;
 *   dir_tile   -- directions per cell-pass staging tile, 1..8 (clamped to
 *                 what fits twice in shared memory).
 * 0 keeps the current value.  Results change only at rounding level (the
 * order of the partial sums over directions). */
vet_status vet_set_tuning(vet_ctx *ctx, int face_group, int dir_tile);
vet_status vet_get_tuning(const vet_ctx *ctx, int *face_group, int *dir_tile);

/* Time vet_closure on the given device inputs for the candidate tunings
 * {2,4,8} x {2,4,8}, keep the fastest and report it (either out pointer may
 * be NULL).  Allocates one f-sized scratch buffer for the duration of the
 * call.  FP32 contexts. */
vet_status vet_autotune(vet_ctx *ctx, const float *kappa, const float *S, const float *Ib, int *face_group,
                        int *dir_tile, void *stream);

/* ------------------------------------------------------------------------
 * Batches of independent grids (ragged sizes, block edges and direction
 * sets).  Each grid gets its own context (vet_create); vet_batch_closure
 * runs one closure per grid, each on its own branch of one CUDA graph that is
 * captured on the first call and replayed while the field pointers and the
 * members' tunings stay the same (retuning a member through
 * vet_batch_context makes the next call capture again), so the grids'
 * kernels run concurrently and the whole batch costs one graph launch.  FP32,
 * one device, device pointers only.
 * ---------------------------------------------------------------------- */
typedef struct vet_batch vet_batch;

vet_status vet_batch_create(vet_batch **out, int n, const vet_grid *grids, const vet_config *cfgs);
vet_status vet_batch_destroy(vet_batch *batch);

/* The context of grid i (directions, work counts, tuning), owned by the
 * batch; NULL when i is out of range. */
vet_ctx *vet_batch_context(vet_batch *batch, int i);

/* Arrays of n pointers, one per grid; Ib and M_out may be NULL (or hold NULL
 * entries).  Enqueued on `stream`; errors of the device work are reported by
 * vet_batch_sync. */
vet_status vet_batch_closure(vet_batch *batch, const float *const *kappa, const float *const *S,
                             const float *const *Ib, float *const *f_out, float *const *M_out, void *stream);
vet_status vet_batch_sync(vet_batch *batch);

/* vet_autotune for the first grid of every distinct shape (cells, block edge,
 * directions), applied to all grids of that shape. */
vet_status vet_batch_autotune(vet_batch *batch, const float *const *kappa, const float *const *S,
                              const float *const *Ib, void *stream);

/* Message for the last failure on the batch.  Never NULL. */
const char *vet_batch_last_error(const vet_batch *batch);

/* ------------------------------------------------------------------------
 * Learned closure (not in the paper, whose closures are the exact VET, M1
 * and Eddington, Sec. 2.2.5 and App. A): a small 3D convolutional network
 * predicts f from local features; the exact ray tracer above is its fallback
 * and the reference for its error.
 *
 * Features per cell (6): 1 (validity; the zero padding at the domain edge
 * reads 0), log10(kappa h), log10 S and log10 E each minus its mean over the
 * volume (f does not change when S, and with it I and E, is scaled), and the
 * mean and population standard deviation of log10(kappa h) over the cell's
 * block.  Arguments of log10 are clamped below at 1e-30.
 * Network: four 3x3x3 convolutions with zero padding, 6 -> C -> C -> C -> 7
 * channels (C = 32), SiLU z/(1+exp(-z)) after the first three; BF16 weights
 * and activations, FP32 accumulation, FP32 master weights.  Outputs 0..5 are
 * a correction D (xx, yy, zz, xy, xz, yz) to I/3 with the trace projected
 * out: f_ii = 1/3 + D_ii - tr(D)/3, f_ij = D_ij.  Output 6 is the log of the
 * predicted max_ij |f - f_exact|.
 * Loss: mean over cells and components of (f - f_ref)^2 plus
 * lam * mean over cells of (o6 - log(max_ij |f - f_ref| + 1e-4))^2, the
 * target of o6 held constant.
 * Indicator: r = max(-lambda_min(f), lambda_max(f) - 1, exp(o6), 0); blocks
 * holding a cell with r > threshold are recomputed by the exact closure.
 *
 * Parameters cross the ABI as one FP32 host array: for each layer in order,
 * W[27][C_out][C_in] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1), the input cell at
 * offset (dx, dy, dz)) then b[C_out], with the real channel counts above.
 * All field pointers of the model calls are device memory; work is enqueued
 * on `stream`.  A model is not thread-safe.
 * ---------------------------------------------------------------------- */
typedef struct vet_model vet_model;

/* Create a model on `device` with `channels` hidden channels (32 is the
 * only value the library supports).  Weights start at zero: call
 * vet_model_set_params. */
vet_status vet_model_create(vet_model **out, int channels, int device);
vet_status vet_model_destroy(vet_model *model);

/* Number of parameters in the host layout (66631 for 32 channels), or -1. */
long long vet_model_num_params(const vet_model *model);

/* Host FP32 parameters in / out.  set_params also resets the optimiser
 * (moments and step count) and synchronises the device. */
vet_status vet_model_set_params(vet_model *model, const float *params);
vet_status vet_model_get_params(vet_model *model, float *params);

/* Host FP32 copy of the gradients of the last vet_model_backward (same
 * layout as the parameters). */
vet_status vet_model_get_grads(vet_model *model, float *grads);

/* Checkpoint of a model to a file and back: the parameters, AdamW's two
 * moment estimates and its step count, so that training resumes where it
 * stopped.  Format: the 8 bytes "VETMODL1", int32 hidden channels, int32 0,
 * int64 parameter count, int64 step count, then three FP32 arrays in the host
 * parameter layout above (parameters, first moments, second moments),
 * little-endian.  load checks the tag, the hidden width and the parameter
 * count (VET_EINVAL on a mismatch, an unreadable or truncated file; the model
 * is then unchanged) and synchronises the device.  Not in the paper. */
vet_status vet_model_save(vet_model *model, const char *path);
vet_status vet_model_load(vet_model *model, const char *path);

/* Features of `nvol` volumes of the grid (each [nz][ny][nx], stacked) into
 * the model's workspace: kappa, S, E are [nvol][nz][ny][nx]; grid->block is
 * the block of the block statistics and must divide every extent.
 * feat_out (optional, [nvol][6][cells]) receives the FP32 features before
 * their rounding to BF16. */
vet_status vet_model_features(vet_model *model, const vet_grid *grid, int nvol, const float *kappa,
                              const float *S, const float *E, float *feat_out, void *stream);

/* Network forward pass on the current features, keeping what the backward
 * pass needs.  o_out (optional, [nvol][7][cells] FP32) receives the raw
 * outputs. */
vet_status vet_model_forward(vet_model *model, float *o_out, void *stream);

/* Loss of the last forward pass against f_ref [nvol][6][cells] and the
 * gradients of all parameters.  mask (optional, [nvol][cells] bytes) selects
 * the cells that count (nonzero).  loss_out (optional) is a DEVICE double. */
vet_status vet_model_backward(vet_model *model, const float *f_ref, const uint8_t *mask, float lam,
                              double *loss_out, void *stream);

/* One AdamW step (decoupled weight decay, applied to every parameter) with
 * the gradients of the last backward pass. */
vet_status vet_model_step(vet_model *model, float lr, float beta1, float beta2, float eps, float weight_decay,
                          void *stream);

/* Learned closure of one grid with the exact closure as fallback: features
 * from (kappa, S, E) (E is the caller's radiation energy density, e.g. from
 * its moment solve), network, indicator, then vet_closure's computation on
 * every block whose indicator exceeds `threshold`.  ctx (FP32) supplies the
 * grid, directions and tracer; f_out [6][cells].  block_flags_out (optional,
 * device [blocks] uint32, blocks x-fastest) receives 1 for the recomputed
 * blocks; *n_fallback_out (optional, host) their number.  The call
 * synchronises `stream` once (to size the fallback); device-side timeouts of
 * the fallback are reported by vet_sync(ctx). */
vet_status vet_closure_learned(vet_ctx *ctx, vet_model *model, const float *kappa, const float *S,
                               const float *E, const float *Ib, float threshold, float *f_out,
                               uint32_t *block_flags_out, int *n_fallback_out, void *stream);

/* Device time of the last vet_closure_learned, in milliseconds: ms[0] the
 * network (features, convolutions, indicator and block list), ms[1] the
 * fallback (exact closure on the flagged blocks), ms[2] the whole call,
 * ms[3] the four convolutions alone (part of ms[0]). */
vet_status vet_model_last_timing(vet_model *model, float ms[4]);

/* Individual indicator values of the last vet_closure_learned call's grid:
 * r_out [cells] FP32, device.  For inspection. */
vet_status vet_model_last_indicator(vet_model *model, float *r_out, void *stream);

/* Message for the last failure on the model.  Never NULL. */
const char *vet_model_last_error(const vet_model *model);

/* Message for the last failure on ctx (or, when ctx is NULL, for the last
 * failure of vet_create or vet_closure_noalloc in this thread).  Never NULL. */
const char *vet_last_error(const vet_ctx *ctx);

/* ------------------------------------------------------------------------
 * Local closures (paper Sec. 4.1, the comparison with FLD and M1): the
 * Eddington tensor of each cell from that cell's moments alone.
 *   VET_CLOSURE_EDDINGTON: T = I / 3 (M may be NULL).
 *   VET_CLOSURE_M1:        T = (1 - chi)/2 I + (3 chi - 1)/2 n n with
 *                          n = F / |F| and the Levermore factor
 *                          chi(f) = (3 + 4 f^2) / (5 + 2 sqrt(4 - 3 f^2)),
 *                          f = |F| / E (c = 1).
 * Readings: f is clipped to [0, 1]; F = 0 gives chi = 1/3 (T = I / 3); E <= 0
 * gives T = I / 3.
 * M: [10][ncell] moments in vet_moments' layout (only E, Fx, Fy, Fz are
 * read); T_out: [6][ncell] (xx, yy, zz, xy, xz, yz).  Both device memory,
 * caller-owned; work is enqueued on `stream` and the call returns before it
 * runs.  VET_EINVAL for a bad kind, a negative ncell, a missing or host
 * pointer; VET_ECUDA for a failed launch.  Needs no context.
 * ---------------------------------------------------------------------- */
enum { VET_CLOSURE_EDDINGTON = 0, VET_CLOSURE_M1 = 1 };
vet_status vet_local_closure(int kind, long long ncell, const float *M, float *T_out, void *stream);

/* ------------------------------------------------------------------------
 * Direct radiation of a point source (paper Sec. 2.2.6, "Point Sources
 * Contribution"): the energy and momentum deposition rates of a source of
 * luminosity L at xs in every cell of the grid, from the optical depth
 * along the straight ray from the source through the cell centre:
 *   Edot = L e^{-tau_*} (1 - e^{-tau_cell}) / (4 pi r^2 dr),  pdot = Edot r_hat
 * with tau_* the optical depth from the source to where the ray enters the
 * cell (0 in the source's own cell), dr the ray's length inside the cell,
 * tau_cell = kappa dr, r the distance to the cell centre and c = 1; 1 -
 * e^{-tau_cell} is evaluated as -expm1(-tau_cell) (the paper's small-tau
 * Taylor form without a switch).  A cell whose centre is the source gets 0.
 * grid: cells and h (block is ignored); xs: host, length units, inside the
 * grid [0, n h) per axis; kappa: [nz][ny][nx] opacity to the direct
 * radiation per unit length; Edot_out: [cells]; pdot_out: [3][cells] or
 * NULL.  Field pointers are device memory; work is enqueued on `stream`.
 * VET_EINVAL for a bad grid, a source outside it or a missing or host
 * pointer; VET_ECUDA for a failed launch.  Needs no context.
 * ---------------------------------------------------------------------- */
vet_status vet_point_source(const vet_grid *grid, const double xs[3], double L, const float *kappa, float *Edot_out,
                            float *pdot_out, void *stream);

/* ------------------------------------------------------------------------
 * Change gate for reusing the Eddington tensor across time steps (paper
 * Sec. 4.2, "Performance": f may be recomputed only every few time steps).
 * Measures how far the closure's inputs moved since a snapshot, per block of
 * grid->block^3 cells and over the grid:
 *   dtrans = max |a - b| / ((1 + a/2) (1 + b/2)),  a = kappa h, b = kappa_ref h
 *            (a bound on the change |e^{-a} - e^{-b}| of a cell's
 *            transmission, which moves the intensity leaving the cell:
 *            ~ |a - b| for thin cells, small for thick ones)
 *   dS     = max |S - S_ref|    (largest change of the source)
 *   Sref   = max |S_ref|        (scale of the source)
 * computed in FP32, each operation one IEEE rounding (h as (float)h) and a
 * maximum exact, so the result is the same for any reduction order.  A NaN
 * (in a difference, the quotient or S_ref) counts as +inf.
 * out: device float [3 + 3 * blocks]: out[0..2] the grid's (dtrans, dS, Sref),
 * then each block's triple, blocks x-fastest (b = (bk * nby + bj) * nbx + bi).
 * With snapshot != 0 the same pass also copies kappa into kappa_ref and S
 * into S_ref; out then describes the change before the copy.
 * dtrans bounds the change of the transmission across one cell EDGE (optical
 * depth kappa h); a ray crossing a cell diagonally travels up to sqrt(3) h,
 * so its transmission may change by up to about sqrt(3) times dtrans: a
 * tolerance on dtrans is a tolerance per cell edge.
 * grid: cells, block edge (2..32, dividing every extent) and h; kappa, S,
 * kappa_ref, S_ref: [nz][ny][nx] device memory, caller-owned, the two
 * snapshot arrays not overlapping the others.  Work is enqueued on `stream`
 * (out[0..2] is cleared on the stream first).  VET_EINVAL for a bad grid or a
 * missing or host pointer; VET_ECUDA for a failed launch.  Needs no context.
 * ---------------------------------------------------------------------- */
vet_status vet_field_change(const vet_grid *grid, const float *kappa, const float *S, float *kappa_ref, float *S_ref,
                            int snapshot, float *out, void *stream);

/* The reuse decision for one time step (paper Sec. 4.2, which suggests
 * recomputing f only every few steps and gives no criterion; this is the
 * library's reading): *recompute = 1 on the first step (first != 0), once
 * the stored f is max_age steps old (age >= max_age), when dtrans or dS is
 * not finite, or when dtrans > tol_tau or dS > tol_S * Sref; else 0.
 * change: HOST float[3], the grid triple (dtrans, dS, Sref) of
 * vet_field_change copied back; the comparisons are made in double on those
 * FP32 values.  Host only, no GPU work.  VET_EINVAL for a NULL pointer,
 * max_age < 1, age < 0 or a negative or NaN tolerance. */
vet_status vet_reuse_decision(const float *change, int age, int first, double tol_tau, double tol_S, int max_age,
                              int *recompute);

/* ------------------------------------------------------------------------
 * HLLE face wavespeed with the optical-depth correction (paper Sec. 2.2.3,
 * "Implicit Hyperbolic Transport of Radiation", and App. A): the first
 * consumer of the Eddington tensor in the implicit moment update.  For the
 * faces normal to axis a (0 = x, 1 = y, 2 = z),
 *   C = sqrt(f_aa) c sqrt((1 - e^-tau_c) / tau_c),
 *   tau_c = (10 h kappa_R)^2 / (2 f_aa),
 * tau_c formed per cell with that cell's f_aa and kappa_R and averaged over
 * the face's two cells (the paper's rule between cells of one refinement
 * level; the grid is uniform).  Readings: the face's free-streaming factor
 * is the larger of its two cells' sqrt(f_aa) (left- and right-going speeds
 * are -C and +C); a face on the domain boundary takes its one cell's values;
 * f_aa <= 0 gives tau_c = inf and C's cell factor 0, kappa_R = 0 gives
 * tau_c = 0 and the correction 1.  FP32: below tau_c = 1/4 the correction
 * comes from the ray march's thin-segment cubic (no cancellation), above it
 * from the hardware exponential; quotients use the hardware reciprocal (a
 * few ulp), so the result is within a few 1e-7 relative of the exact
 * formula.
 * grid: cells and h (block is ignored); f: [6][nz][ny][nx] as vet_closure
 * writes it (only component a is read); kappa_R: [nz][ny][nx], rho kappa_R
 * per unit length; c > 0; C_out: [nz][ny][nx+1] for a = 0, [nz][ny+1][nx]
 * for a = 1, [nz+1][ny][nx] for a = 2 (face (x, y, z) lies on the low side
 * of cell (x, y, z)).  All device memory, caller-owned; work is enqueued on
 * `stream`.  VET_EINVAL for a bad grid, axis or c, or a missing or host
 * pointer; VET_ECUDA for a failed launch.  Needs no context.
 * ---------------------------------------------------------------------- */
vet_status vet_hlle_wavespeed(const vet_grid *grid, const float *f, const float *kappa_R, double c, int axis,
                              float *C_out, void *stream);

/* ------------------------------------------------------------------------
 * An entry point that allocates nothing (the paper has no counterpart; it
 * exists for callers of this library, not for the method).
 *
 * Some callers cannot call cudaMalloc: code running while another framework's
 * caching allocator holds nearly all device memory (the allocation would
 * fail), real-time loops that must not block on cudaMalloc / cudaFree (both
 * can synchronise the whole device), and plug-ins whose host application
 * forbids allocations outside its own pool.  They still own their inputs and
 * outputs; what they cannot provide is the library's workspace.
 *
 * vet_closure_noalloc computes exactly what vet_create + vet_closure (FP32)
 * compute, without a context: every piece of workspace lives in one static
 * device array of VET_NOALLOC_SCRATCH_BYTES compiled into libvet, which every
 * GPU that loads the library holds until the process exits, and the host-side
 * geometry uses fixed static host arrays.  It calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *   - Limits: FP32 only; nside 1, 2 or 4; block edge 2..16; and the problem's
 *     workspace (about 12 * N * blocks * (block+2)^2 bytes for the face
 *     intensities plus templates and schedule) must fit the array, e.g.
 *     64^3 cells in 16^3 blocks with 192 directions, or 32^3 cells in 8^3
 *     blocks with 48.  Larger problems return VET_EINVAL with a message
 *     (vet_last_error(NULL)).
 *   - Field pointers must be device memory.  Work is enqueued on `stream`
 *     and the call returns before it runs.
 *   - The first call made for a device (cfg->device) looks up the array's
 *     device address with that device selected; make that first call before
 *     any stream capture.
 *   - Every call shares the one array and overwrites what the previous call
 *     left there.  Calls whose GPU work overlaps (different streams, or
 *     different host threads with no ordering between them) race on it and
 *     give wrong results: order them.
 *   - If a bounded device-side wait gives up (see vet_sync), f_out is filled
 *     with NaN: there is no context to report it through.
 * ---------------------------------------------------------------------- */
#define VET_NOALLOC_SCRATCH_BYTES (64u << 20)

vet_status vet_closure_noalloc(const vet_grid *grid, const vet_config *cfg, const float *kappa, const float *S,
                               const float *Ib, float *f_out, float *M_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VET_H */
