/*
 * opm.h - C ABI of the GB300 (sm_103a) oblique-plane deskew library.
 *
 * The library implements the data-parallel hot path of live OPM viewing
 * (Lamb, Ward & Kaminski, arXiv 2211.00645): the shear deskew of a raw stack
 * of tilted camera frames onto the real-space (z, y', x) grid and the
 * widefield-like maximum projection of the deskewed stack, plus the adjoint
 * of the deskew and the backward pass of the z-MIP.
 *
 * Geometry (lab frame, Eq. 1 with the sheet angle alpha = theta):
 *   raw      R[n][r][x]    n in [0, nscan) scan plane, r in [0, nrows) camera
 *                          row, x in [0, ncols) column; C order, x fastest.
 *   output   V[k][j][x]    k in [0, nz = nrows), j in [0, ny), x in [0, nx = ncols).
 *   n_f(j,k) = ((j - J0)*pixel - k*pixel*cos(theta)) / step
 *   LINEAR   V = (1-w) R~[n0] + w R~[n0+1],  n0 = floor(n_f), w = n_f - n0
 *   NEAREST  V = R~[floor(n_f + 1/2)]
 *   R~[n] = R[n] for 0 <= n < nscan and 0 otherwise (zero-padded tent).
 *   J0 = ceil(step/pixel) - 1,
 *   ny = ceil(J0 + nscan*(step/pixel) + (nrows-1)*cos(theta) - 1e-9).
 * cos(theta) is exactly 0 at 90 degrees and exactly 1/2 at 60 degrees.
 *
 * Conventions shared by every call below:
 *   - Array pointers are DEVICE pointers to C-contiguous arrays owned by the
 *     caller; the library never keeps them after the call returns.
 *   - Compute calls are asynchronous on `cuda_stream` (a cudaStream_t; NULL is
 *     the legacy default stream).  They neither allocate nor synchronise.
 *   - A plan is immutable after creation and may be shared by threads and
 *     streams.  Compute calls must run on the device the plan was created on.
 *   - Every call returns an opm_status; on failure opm_last_error() gives a
 *     description, valid in the calling thread until its next library call.
 *     Output buffers are left untouched when a call fails its argument checks.
 */
#ifndef OPM_H
#define OPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct opm_plan opm_plan; /* opaque; owns only its small geometry tables */

typedef enum {
  OPM_OK = 0,
  OPM_ERR_INVALID_ARG = 1,   /* a parameter is out of its documented domain  */
  OPM_ERR_UNSUPPORTED = 2,   /* valid but not handled (dtype pair, size)     */
  OPM_ERR_CUDA = 3,          /* a CUDA runtime/driver call failed            */
  OPM_ERR_OUT_OF_MEMORY = 4, /* plan tables could not be allocated           */
  OPM_ERR_INTERNAL = 5       /* a device-side consistency check tripped      */
} opm_status;

typedef enum { OPM_INTERP_LINEAR = 0, OPM_INTERP_NEAREST = 1 } opm_interp;

typedef enum {
  OPM_U16 = 0, /* uint16 camera counts                                      */
  OPM_F32 = 1, /* float                                                     */
  OPM_F64 = 2  /* double (gradient checks only)                             */
} opm_dtype;

/*
 * opm_plan_create - geometry of one acquisition (Eq. 1; Fig. 2c remap).
 *   nscan >= 2 scan planes, nrows >= 1 camera rows, ncols >= 1 columns,
 *   theta_deg in (0, 90] sheet angle to the scan axis, step > 0 scan step,
 *   pixel > 0 sample-plane pixel size (step and pixel in the same unit),
 *   interp LINEAR or NEAREST.  On success *out receives a new plan.
 * Derives nz, ny, J0 in FP64 and splits the per-column term (j-J0)*pixel/step
 * and the per-row term k*cos(theta)*pixel/step into an integer and an FP32
 * fraction, uploaded to the current CUDA device (the plan's device) when one
 * is present.  A plan made without a device answers opm_plan_shape but its
 * compute calls return OPM_ERR_CUDA.
 * Errors: OPM_ERR_INVALID_ARG (domain, NULL out), OPM_ERR_UNSUPPORTED (a
 * dimension of the output grid above 2^31 - 1 or more than 2^40 voxels),
 * OPM_ERR_OUT_OF_MEMORY, OPM_ERR_CUDA.
 */
opm_status opm_plan_create(int64_t nscan, int64_t nrows, int64_t ncols,
                           double theta_deg, double step, double pixel,
                           opm_interp interp, opm_plan** out);

/* Output grid of a plan: nz = nrows, ny, nx = ncols, and J0.  Any output
 * pointer may be NULL.  Errors: OPM_ERR_INVALID_ARG for a NULL plan. */
opm_status opm_plan_shape(const opm_plan* plan, int64_t* nz, int64_t* ny,
                          int64_t* nx, int64_t* j0);

/*
 * opm_plan_path - which live-view kernel opm_project runs for this plan with
 * uint16 input, z-MIP and/or y-MIP outputs and no z-sum or arg-max (the
 * serving outputs).  A diagnostic of the plan; it computes nothing.
 *   *path = OPM_PATH_PERIODIC: the periodic kernel for pixel/step = p/q,
 *           chosen when every 32-column tile row steps through its planes as
 *           floor((t p + ph) / q) (Eq. 1 with a rational scan-to-pixel ratio;
 *           checked with the kernels' own arithmetic); *fam_p, *fam_q = p, q.
 *   *path = OPM_PATH_FAST: the fast kernel (pixel <= step, ny >= 32).
 *   *path = OPM_PATH_GENERAL: the general kernel (any plan; also every call
 *           with z-sum or arg-max output, or FP32 input).
 * Any output pointer may be NULL.  Errors: OPM_ERR_INVALID_ARG (plan NULL).
 * The raw stack's alignment is not known here; opm_project takes the plain
 * kernels when a row is not a multiple of 16 bytes or raw is misaligned.
 */
typedef enum { OPM_PATH_GENERAL = 0, OPM_PATH_FAST = 1, OPM_PATH_PERIODIC = 2 } opm_path;
opm_status opm_plan_path(const opm_plan* plan, int* path, int* fam_p, int* fam_q);

/*
 * opm_plan_schedule - the live-view schedule of the fast and periodic kernels
 * (the live view of opm_project, Fig. 2d).  The work is cut into units of
 * *chunk_rows camera rows of one 32-column j-tile at one 128-column x-tile,
 * placed longest-first on *nlists lists, one per persistent CTA.  The plan
 * takes the largest of 256, 128, 64, 32 and 16 rows that gives at least 1.1
 * units per list, so that narrow stacks (an x-shard of one) still fill the
 * GPU.  All three are 0 for a plan without that schedule (the general
 * kernel's plans, and plans made with no CUDA device).  Any output pointer
 * may be NULL.  Errors: OPM_ERR_INVALID_ARG (plan NULL).
 */
opm_status opm_plan_schedule(const opm_plan* plan, int64_t* nunits, int* nlists, int* chunk_rows);

/* Frees a plan and its device tables.  NULL is accepted.  The caller must not
 * destroy a plan while work that uses it is still queued on a stream. */
opm_status opm_plan_destroy(opm_plan* plan);

/*
 * opm_deskew - materialise the deskewed volume (Fig. 2c).
 *   raw  [nscan][nrows][ncols] of in_t;  vol [nz][ny][nx] of out_t.
 *   Supported (in_t -> out_t): U16->F32, U16->U16, F32->F32, F32->U16,
 *   F64->F64.  A U16 output is the value rounded half to even and clamped to
 *   [0, 65535].
 * Errors: OPM_ERR_INVALID_ARG (NULL plan or pointers), OPM_ERR_UNSUPPORTED
 * (dtype pair), OPM_ERR_CUDA (launch failure, wrong device).
 */
opm_status opm_deskew(const opm_plan* plan, const void* raw, opm_dtype in_t,
                      void* vol, opm_dtype out_t, void* cuda_stream);

/*
 * opm_deskew_dual - the deskew of opm_deskew (Fig. 2c) written twice in one pass over
 * the raw stack: as FP32 into vol_f32 and rounded to nearest (ties to even,
 * clamped to [0, 65535]) into vol_u16, both [nz][ny][nx] device arrays owned
 * by the caller.  Each uint16 voxel is the rounding of the FP32 voxel beside
 * it.  in_t: OPM_U16 or OPM_F32.  Asynchronous on cuda_stream; allocates
 * nothing.  Errors: OPM_ERR_INVALID_ARG (NULL plan or pointer),
 * OPM_ERR_UNSUPPORTED (input type, launch limits), OPM_ERR_CUDA.
 */
opm_status opm_deskew_dual(const opm_plan* plan, const void* raw, opm_dtype in_t, float* vol_f32,
                           uint16_t* vol_u16, void* cuda_stream);

/*
 * opm_deskew_mip - the volume and the live view in one call (the paper's
 * remap followed by its maximum projection, Fig. 2c-d): vol_f32 and/or
 * vol_u16 [nz][ny][nx] as opm_deskew / opm_deskew_dual write them, zmip
 * [ny][nx] and ymip [nz][nx] as opm_project writes them (either may be
 * NULL), all bit-identical to those calls.
 * By default the projection runs on the plan's own high-priority stream
 * beside the volume on cuda_stream: it is forked from cuda_stream (an event
 * recorded there) and joined back into it before the call returns, so work
 * queued on cuda_stream afterwards sees every output; the pair is
 * capturable into a CUDA graph.  The projection's persistent kernel then
 * takes one CTA per SM, which leaves room on each SM for the write-bound
 * volume kernel.  Calls on one plan are serialised on a host mutex for the
 * fork and join.  A plan created with the environment variable
 * OPM_ONE_PASS_FUSED=1 instead runs uint16 input through one fused kernel
 * that stores every voxel as it folds it into the projections (raw read
 * once), and FP32 input through the separate kernels on cuda_stream.
 * Asynchronous; allocates nothing.
 * Errors: OPM_ERR_INVALID_ARG (NULL plan or raw, no volume), OPM_ERR_UNSUPPORTED
 * (input type, launch limits), OPM_ERR_CUDA.
 */
opm_status opm_deskew_mip(const opm_plan* plan, const void* raw, opm_dtype in_t, float* vol_f32, uint16_t* vol_u16,
                          float* zmip, float* ymip, void* cuda_stream);

/*
 * opm_project - widefield-like live view, fused with the deskew (Fig. 2d):
 * the volume is never written to memory.
 *   raw  [nscan][nrows][ncols] of in_t (U16 or F32)
 *   zmip [ny][nx] float  max over k of V          (the widefield-like view)
 *   zsum [ny][nx] float  sum over k of V
 *   ymip [nz][nx] float  max over j of V          (side view)
 *   argz [ny][nx] int32  smallest k attaining zmip (needed by opm_mip_backward)
 * Any of the four outputs may be NULL, but not all of them.  The maxima run
 * over the whole output grid, zero-padded voxels included.
 * Errors: OPM_ERR_INVALID_ARG (NULL plan/raw, all outputs NULL),
 * OPM_ERR_UNSUPPORTED (in_t F64), OPM_ERR_CUDA.
 */
opm_status opm_project(const opm_plan* plan, const void* raw, opm_dtype in_t,
                       float* zmip, float* zsum, float* ymip, int32_t* argz,
                       void* cuda_stream);

/*
 * The paper's own live view (sheet frame).  Every raw frame n is remapped
 * into a larger image shifted along the camera-row axis by its accumulated
 * lateral offset, n * shear rows, where Eq. (1) gives shear =
 * step * cos(alpha) / pixel (Fig. 2c); the view is the brightest value over
 * the frames at each pixel (Fig. 2d).  A sub-row shift interpolates linearly
 * between the two neighbouring camera rows (zero outside the frame).  A
 * smaller shear followed by opm_warp_rows changes the viewing angle
 * (shear-warp, Fig. 3).
 *
 * opm_sheet_rows - rows of the remapped image: nrows + ceil((nscan - 1) *
 * shear) (shear >= 0, finite; nscan, nrows >= 1).
 * Errors: OPM_ERR_INVALID_ARG, OPM_ERR_UNSUPPORTED (over 2^31 rows).
 *
 * opm_sheet_project - out[Y][x] = max_n S[n][Y][x] for raw [nscan][nrows]
 * [ncols] (in_t U16 or F32, device) into out [out_rows][ncols] FP32
 * (device, caller-owned); out_rows must equal opm_sheet_rows.  Frames that
 * do not reach a row contribute 0 to its maximum.  Asynchronous; allocates
 * nothing.  Errors: OPM_ERR_INVALID_ARG (NULL, sizes, out_rows),
 * OPM_ERR_UNSUPPORTED (type, more planes than the shared-memory shift
 * table holds, sizes past 2^31), OPM_ERR_CUDA.
 */
opm_status opm_sheet_rows(int64_t nscan, int64_t nrows, double shear, int64_t* rows);
opm_status opm_sheet_project(const void* raw, opm_dtype in_t, int64_t nscan, int64_t nrows, int64_t ncols,
                             double shear, float* out, int64_t out_rows, void* cuda_stream);

/*
 * opm_sheet_check - uint16 stacks whose rows are a multiple of 8 columns
 * (at least 128 columns, 33 rows, 16-byte aligned base) take a TMA kernel
 * that stages each frame's rows through a ring with bounded waits; the
 * others take a plain kernel.  A wait that gives up sets an error word on
 * the device.  This call reads and clears the word of the current device:
 * OPM_ERR_INTERNAL when a wait gave up since the last check (that view is
 * incomplete), OPM_ERR_CUDA on a failed copy, else OPM_OK.  Synchronous
 * (a blocking copy on the legacy default stream); not for the hot path.
 */
opm_status opm_sheet_check(void);

/*
 * opm_warp_rows - the warp of the shear-warp view (Fig. 3): out[Y'][x] =
 * in at row a * Y' + b, linear between rows, zero outside [0, in_rows).
 * in [in_rows][ncols], out [out_rows][ncols], FP32 device arrays.
 * Asynchronous; allocates nothing.  Errors: OPM_ERR_INVALID_ARG (NULL,
 * sizes, non-finite a or b), OPM_ERR_UNSUPPORTED (sizes), OPM_ERR_CUDA.
 */
opm_status opm_warp_rows(const float* in, int64_t in_rows, int64_t ncols, float* out, int64_t out_rows, double a,
                         double b, void* cuda_stream);

/*
 * Plane-by-plane live view (the rolling update of Fig. 4a: the maximum
 * projection is refreshed after every camera exposure).  A stack's z-MIP,
 * z-sum and y-MIP are accumulated one scan-plane pair at a time, with only
 * two camera frames on the device.
 *
 * opm_stream_begin - zeroes the outputs (zmip, zsum [ny][nx], ymip [nz][nx]
 * FP32 device arrays; any may be NULL, not all) for a new stack.
 *
 * opm_stream_pair - folds into the outputs every voxel whose lower
 * interpolation plane is n: V = (1 - w) R~[n] + w R~[n + 1] (zero-padded
 * tent, LINEAR; R~[n] alone for NEAREST).  plane_lo is frame n and plane_hi
 * frame n + 1, each [nrows][ncols] uint16 on the device; plane_lo is NULL
 * exactly when n == -1 and plane_hi exactly when n == nscan - 1.  n lies in
 * [-1, nscan - 1].  After the calls for n = -1, 0, ..., nscan - 1 (any
 * order) the z-MIP and y-MIP equal opm_project's on the whole stack bit for
 * bit; the z-sum equals it up to FP32 summation order.  Calls that update
 * the same outputs must be ordered on one stream.  Asynchronous; allocates
 * nothing.  A column search that runs past its bound records an error bit
 * (see opm_plan_check).
 * Errors: OPM_ERR_INVALID_ARG (NULL plan, no output, n out of range, plane
 * pointers not matching n), OPM_ERR_UNSUPPORTED (more than 65535 rows),
 * OPM_ERR_CUDA.
 */
opm_status opm_stream_begin(const opm_plan* plan, float* zmip, float* zsum, float* ymip, void* cuda_stream);

/*
 * opm_max_combine - out[i] = max(a[i], b[i]) for i < n, FP32 device arrays
 * (out may be a or b).  The maximum over frames is associative and exact, so
 * the projections of disjoint sets of plane pairs (each accumulated by
 * opm_stream_pair from zeroed outputs) combine to the projection of their
 * union bit for bit; the sliding view of a camera stream (Fig. 4a, a full
 * stack of the newest frames) keeps such partial maxima and combines them
 * per frame.  Asynchronous on cuda_stream; allocates nothing.
 * Errors: OPM_ERR_INVALID_ARG (NULL array, n < 0), OPM_ERR_CUDA.
 */
opm_status opm_max_combine(float* out, const float* a, const float* b, int64_t n, void* cuda_stream);

/*
 * opm_sliding_push - the sliding live view (Fig. 4a refreshed after every
 * frame, always spanning a full stack of the newest frames): call it after
 * writing frame m (0 <= m < nscan) of the current stack into stack[m]
 * ([nscan][nrows][ncols] uint16, device), on the stream that wrote it.
 * Frames 0..m are then the current stack's and m+1..nscan-1 the previous
 * stack's (all zero before the first).  Each projection buffer is an FP32
 * z-MIP [ny][nx] followed by a y-MIP [nz][nx] (P = ny nx + nz nx floats):
 *   run   [P]         maximum over the current stack's complete plane pairs;
 *   slots [nscan][P]  slot q: the previous stack's maximum over its pairs
 *                     q..nscan-1, until the current stack's pair q replaces
 *                     it (slot 0 is not used);
 *   view  [P]         the published projections.
 * All three must be zero before the first push and are owned by the caller.
 * After the call, view equals opm_project of the stack buffer bit for bit
 * (z-MIP and y-MIP).  A call costs two opm_stream_pair passes, one zeroing
 * and two maxima over P; the call for m = nscan - 1 also builds the next
 * suffixes (nscan - 2 maxima).  Asynchronous; allocates nothing.
 * Errors: OPM_ERR_INVALID_ARG (NULL, m out of range), OPM_ERR_UNSUPPORTED
 * (more than 65535 rows), OPM_ERR_CUDA.
 */
opm_status opm_sliding_push(const opm_plan* plan, const uint16_t* stack, int64_t m, float* run, float* slots,
                            float* view, void* cuda_stream);
opm_status opm_stream_pair(const opm_plan* plan, const uint16_t* plane_lo, const uint16_t* plane_hi, int64_t n,
                           float* zmip, float* zsum, float* ymip, void* cuda_stream);

/*
 * opm_skew_adjoint - transpose of the LINEAR deskew map:
 *   raw_out[n][k][x] = sum_j vol[k][j][x] * t(n_f(j,k) - n),  t(u) = max(0, 1-|u|).
 *   vol [nz][ny][nx] and raw_out [nscan][nrows][ncols], both of type t (F32 or
 *   F64).  Each output element is a gather over j in ascending order: no
 *   atomics, bitwise reproducible.  Plans made with NEAREST use the matching
 *   0/1 weights.
 * Errors: OPM_ERR_INVALID_ARG, OPM_ERR_UNSUPPORTED (t = U16), OPM_ERR_CUDA.
 */
opm_status opm_skew_adjoint(const opm_plan* plan, const void* vol,
                            void* raw_out, opm_dtype t, void* cuda_stream);

/*
 * opm_mip_backward - gradient of sum(g_zmip * zmip) with respect to the raw
 * stack, routed through the voxel that attained each maximum:
 *   g_raw[n][k][x] = sum_j [argz[j][x] == k] g_zmip[j][x] t(n_f(j,k) - n).
 *   g_zmip [ny][nx] float, argz [ny][nx] int32 (from opm_project),
 *   g_raw [nscan][nrows][ncols] float (fully overwritten).
 * Errors: OPM_ERR_INVALID_ARG, OPM_ERR_CUDA.
 */
opm_status opm_mip_backward(const opm_plan* plan, const float* g_zmip,
                            const int32_t* argz, float* g_raw,
                            void* cuda_stream);

/*
 * Batched live view: persistent launches compute the projections (as
 * opm_project with U16 input) of many stacks, channels and ROIs of uneven
 * sizes.  Multi-colour acquisitions split every camera frame into channels,
 * each deskewed on its own (the paper's channel split in the section "Methods
 * for the fast processing and visualisation of lightsheet data"); here a
 * channel is an item whose raw pointer and pitches select its ROI of a
 * shared frame stack.
 *
 * Items whose plan the fast kernels take (opm_plan_path: FAST or PERIODIC)
 * and that ask for z-MIP and/or y-MIP only run in one persistent launch of
 * the fast (or periodic) kernel over row chunks.  All other items (pixel >
 * step, ny < 32, or a z-sum or arg-max output) run in a second persistent
 * launch of the general kernel, one unit per tile and whole row band.
 * Results equal opm_project's for the same plan and outputs.
 */
typedef struct opm_batch opm_batch; /* opaque; owns device + pinned work lists */

typedef struct {
  const opm_plan* plan; /* geometry of the item: nscan x nrows x ncols     */
  const uint16_t* raw;  /* device pointer to sample (n=0, r=0, x=0)        */
  int64_t row_pitch;    /* elements between camera rows (0: ncols)         */
  int64_t plane_pitch;  /* elements between scan planes (0: nrows*row_pitch) */
  float* zmip;          /* [ny][nx] device output, or NULL                 */
  float* ymip;          /* [nz][nx] device output, or NULL                 */
  float* zsum;          /* [ny][nx] device output, or NULL                 */
  int32_t* argz;        /* [ny][nx] device output (first arg-max), or NULL */
} opm_batch_item;

/*
 * opm_batch_create - work lists for up to max_items items and max_units
 * (<= 2^26) work units (a unit is one 32-column j-tile x 128-column x-tile x
 * row chunk of one item, or a whole row band for items of the general
 * kernel; 32 bytes of work list each).  Allocates device memory and pinned
 * host memory once; the other batch calls allocate nothing except the CUDA
 * graph of opm_batch_launch_graph.
 * Errors: OPM_ERR_INVALID_ARG, OPM_ERR_OUT_OF_MEMORY, OPM_ERR_CUDA.
 */
opm_status opm_batch_create(int max_items, int64_t max_units, opm_batch** out);

/*
 * Kernel shapes of the batch (results are bit for bit the same for every
 * shape; only the speed differs, see the autotuner).  The shape applies to
 * the items the fast kernels may take; the others always run in the general
 * kernel.  The periodic shapes need every such item to share one periodic
 * plan family (opm_plan_path: PERIODIC with the same p/q), else they fall
 * back to OPM_SHAPE_FAST_J8X4.
 */
typedef enum {
  OPM_SHAPE_AUTO = 0,      /* periodic 32 x 2 for one shared family, else fast 8 x 4     */
  OPM_SHAPE_FAST_J8X4 = 1, /* fast kernel: 8 columns j per warp x 4 columns x per lane,  */
                           /* two rows per stage                                          */
  OPM_SHAPE_PER_J32X2 = 2, /* periodic kernel: 32 columns j per warp x 2 x per lane      */
  OPM_SHAPE_PER_J16X2 = 3, /* periodic kernel: 16 columns j per warp x 2 x per lane      */
                           /* (family 1/3; other families run as PER_J32X2)              */
  OPM_SHAPE_GEN_J8X4 = 4   /* general kernel for every item: 8 j x 4 x, whole row band   */
                           /* per unit, one row per stage                                 */
} opm_shape;

/*
 * opm_batch_set - host-side preparation of the work list (TMA descriptors of
 * every item, unit lists sorted by decreasing length).  kchunk = rows per
 * unit of the fast kernels (0: the largest of 256, 128, 64, 32 and 16 that
 * gives at least 1.1 units per CTA list within max_units, as
 * opm_plan_schedule describes); shape = an opm_shape (the one used is
 * reported by opm_batch_info).  Waits until the previous
 * opm_batch_upload of this batch has completed before overwriting its pinned
 * staging.  Every item's plan must live on the batch's device and stage at
 * most 256 planes per row (opm_project's TMA path); raw pointers must be
 * 16-byte aligned and pitches multiples of 8 elements.
 * Errors: OPM_ERR_INVALID_ARG (NULL, counts, pitches), OPM_ERR_UNSUPPORTED
 * (slab depth, alignment, capacity exceeded), OPM_ERR_CUDA.
 */
opm_status opm_batch_set(opm_batch* b, const opm_batch_item* items, int n_items, int kchunk, int shape);

/* opm_batch_upload - asynchronous copy of the prepared work list (only its
 * used bytes: a 256-byte header, 256 bytes per item, 32 per output and 32 per
 * unit) to the device on cuda_stream.
 * Errors: OPM_ERR_INVALID_ARG, OPM_ERR_CUDA. */
opm_status opm_batch_upload(opm_batch* b, void* cuda_stream);

/*
 * opm_batch_launch - zeroes the outputs combined by atomic max and runs the
 * persistent projections over all units on cuda_stream (ctas_per_sm in
 * 1..4, 0: 4; the general kernel runs at most 2 CTAs per SM).  The kernels
 * take the unit and output counts from the device copy of the work list, so
 * the launches may be captured in a CUDA graph by the caller and replayed
 * after later set + upload calls of any content with the same slab depths
 * (plans of the same theta, step and pixel), the same kinds of items (fast
 * kernels, general kernel) and the same grid.
 * Errors: OPM_ERR_INVALID_ARG, OPM_ERR_UNSUPPORTED, OPM_ERR_CUDA.
 */
opm_status opm_batch_launch(opm_batch* b, int ctas_per_sm, void* cuda_stream);

/*
 * opm_batch_launch_graph - as opm_batch_launch, through CUDA graphs the
 * batch owns, one per launch shape (kernel shape, periodic family, slab
 * depths, kinds of items and grids; the 4 most recently used are kept):
 * captured on first use of a launch shape (on a private stream, so
 * cuda_stream may be the legacy default stream) and launched on
 * cuda_stream.  The graph always runs
 * persistent grids (ctas_per_sm x SM CTAs of the fast kernels, up to 2 x SM
 * of the general kernel, for the kinds of items present); CTAs without
 * units return at once.
 * Errors: OPM_ERR_INVALID_ARG, OPM_ERR_UNSUPPORTED, OPM_ERR_CUDA.
 */
opm_status opm_batch_launch_graph(opm_batch* b, int ctas_per_sm, void* cuda_stream);

/* Items, work units (of both kernels), the larger of the two kernels'
 * shared-memory bytes per CTA and the opm_shape used for the prepared batch,
 * and how many graphs opm_batch_launch_graph has captured (any pointer may
 * be NULL).  Errors: OPM_ERR_INVALID_ARG. */
opm_status opm_batch_info(const opm_batch* b, int* n_items, int64_t* n_units, int* smem_bytes,
                          int* graph_captures, int* shape);

/* Synchronising diagnostic, as opm_plan_check for the batch's launches. */
opm_status opm_batch_check(const opm_batch* b);

/* Frees a batch (NULL accepted).  No work using it may still be queued. */
opm_status opm_batch_destroy(opm_batch* b);

/*
 * opm_batch_project_static - the batched live view (opm_batch_set, upload
 * and launch in one call, same kernels and results) with nothing allocated:
 * the work list is built in a fixed host array and copied into a fixed
 * device array reserved when the library is loaded (about 2.1 MB per
 * device).  The paper has no counterpart to this call.
 *
 * Why: cudaMalloc and cudaFree can synchronise the whole device and take
 * milliseconds, which stalls the copy and compute streams of a live
 * acquisition; a caller with a hard per-frame deadline, or one that accounts
 * for every device byte before it starts (a fixed memory plan), cannot
 * create an opm_batch on the fly.  This call gives it a fixed footprint.
 *
 * Limits: at most 64 items and 65536 work units per call (a unit is one
 * 32-column j-tile x 128-column x-tile x kchunk rows of one item); larger
 * requests fail with OPM_ERR_UNSUPPORTED and launch nothing.  Item rules as
 * for opm_batch_set.  kchunk: rows per unit (0: as opm_batch_set);
 * ctas_per_sm: 1..4 (0: 4).
 * check != 0 synchronises cuda_stream afterwards and reports a failed
 * device consistency check as OPM_ERR_INTERNAL (a diagnostic, not for the
 * hot path).
 *
 * The first call on each device does set-up (looks up the device array's
 * address with that device current, sets the kernel's shared-memory limit).
 * The work list is built in one host array shared by the whole process and
 * copied with a pageable cudaMemcpyAsync; the call holds a process-wide lock
 * from building the list until that copy returns (once its source is
 * staged), so threads driving different devices may call it at once.  The
 * call must never be captured in a CUDA graph: on a capturing stream it
 * returns OPM_ERR_UNSUPPORTED and launches nothing.  There is one device
 * array per device: calls whose kernels overlap on one device (several
 * streams, or several threads on one device) race on it and corrupt each
 * other's work lists; serialise them (consecutive calls on one stream are
 * safe).
 * Errors: OPM_ERR_INVALID_ARG, OPM_ERR_UNSUPPORTED, OPM_ERR_CUDA,
 * OPM_ERR_INTERNAL (check only).
 */
opm_status opm_batch_project_static(const opm_batch_item* items, int n_items, int kchunk, int ctas_per_sm,
                                    int check, void* cuda_stream);

/*
 * opm_plan_check - synchronising diagnostic (not for the hot path): waits for
 * the plan's device, then reports OPM_ERR_INTERNAL if any kernel launched with
 * this plan recorded a failed internal consistency check (and clears the
 * record), OPM_OK otherwise.
 */
opm_status opm_plan_check(const opm_plan* plan);

/* Description of the last failure in the calling thread ("" if none). */
const char* opm_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int opm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OPM_H */
