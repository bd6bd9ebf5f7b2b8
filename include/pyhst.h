/*
 * pyhst.h — C ABI of the B300 (sm_103a) parallel-beam reconstruction library.
 *
 * The calls follow the problem statement of the PyHST2 paper (Mirone et al.):
 * raw radiographies with flat ("beam profile") and dark ("detector noise")
 * fields and a per-projection rotation-axis position and angle (Sec. 2.1),
 * dark/flat correction and rearrangement into one sinogram per detector row
 * (Sec. 2.3), filtered back-projection (Sec. 2.3), the forward projector used
 * by the iterative methods (Sec. 2.3, last paragraph), and the TV-penalised
 * least-squares problem of Eq. 3 solved by ISTA/FISTA (Sec. 3.1).
 *
 * Conventions shared by every call
 *   - Images are row-major [ny][nx] float32; pixel (row i, column j).
 *   - Sinograms are row-major [n_angles][n_bins] float32 (one row per angle).
 *   - Detector coordinate of pixel (i, j) at angle index a, in bin units:
 *         t = (j - cx) cos(angles[a]) + (i - cy) sin(angles[a]) + axis[a]
 *     and bin b is centred at t = b.  Linear interpolation between bins,
 *     zero outside [0, n_bins).
 *   - Every pointer passed to a call is DEVICE memory unless stated, owned by
 *     the caller; the library allocates nothing on these paths.  Scratch
 *     memory is the caller's `workspace` of `ws_bytes` bytes, sized with
 *     pyhst_workspace_size(); it must be 256-byte aligned.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) and returns a status; nothing synchronises the
 *     host.  Calls sharing a workspace must be ordered on one stream.
 *   - Errors: a negative status; pyhst_last_error() gives a message (per host
 *     thread).  Argument errors are detected before anything is launched.
 */
#ifndef PYHST_H
#define PYHST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pyhst_stream_t; /* same type as cudaStream_t */

/* Status codes. */
enum {
    PYHST_OK = 0,
    PYHST_ERR_INVALID_ARG = -1,  /* sizes <= 0, NULL pointers, bad enums, unsupported pad */
    PYHST_ERR_CUDA = -2,         /* a CUDA launch or runtime call failed (message has it) */
    PYHST_ERR_WORKSPACE = -3,    /* workspace NULL, too small or misaligned */
    PYHST_ERR_TIMEOUT = -4,      /* a bounded device-side wait gave up */
    PYHST_ERR_NUMERIC = -5       /* non-finite energy / step size */
};

/* Geometry of a stack of n_slices slices that share angles and axis
 * (Sec. 2.1: rotation axis displacement and angle given per projection).
 *   angles [n_angles]  DEVICE float32, radians (any order, any values)
 *   axis   [n_angles]  DEVICE float32, detector position of the rotation axis
 *                      at each projection, in bin units
 *   cx, cy            image centre in pixel-index units ((nx-1)/2, (ny-1)/2
 *                      for a centred grid)
 *   pixel_size        s: detector bin = pixel = s in physical units
 * Limits: 1 <= n_angles <= 65535, 1 <= n_bins <= 16384, 1 <= nx, ny <= 16384. */
typedef struct {
    int32_t n_angles;
    int32_t n_bins;
    int32_t nx;
    int32_t ny;
    int32_t n_slices;
    const float *angles;
    const float *axis;
    float cx;
    float cy;
    float pixel_size;
} pyhst_geometry;

/* Input data kinds of pyhst_fbp. */
typedef enum {
    PYHST_U16_RAW = 0,   /* uint16 counts; normalised with flat and dark     */
    PYHST_F32_RAW = 1,   /* float32 counts; normalised with flat and dark    */
    PYHST_F32_SINO = 2,  /* float32 -ln(I/I0) already normalised             */
    PYHST_F16_SINO = 3,  /* IEEE half sinogram, converted to float32 on load */
    PYHST_BF16_SINO = 4  /* bfloat16 sinogram, converted to float32 on load  */
} pyhst_input_t;

/* Ramp filters, as spatial kernels h(n) (tau = 1 bin) applied by linear
 * convolution along detector rows:
 *   PYHST_RAMLAK       h(0) = 1/4, h(odd n) = -1/(pi n)^2, h(even n) = 0
 *   PYHST_SHEPP_LOGAN  h(n) = -2 / (pi^2 (4 n^2 - 1))
 *   PYHST_HANN         Ram-Lak smoothed by (1/4, 1/2, 1/4) (its spectrum times
 *                      (1 + cos w) / 2)
 * The paper does not name its filter; Ram-Lak is the default. */
typedef enum { PYHST_RAMLAK = 0, PYHST_SHEPP_LOGAN = 1, PYHST_HANN = 2 } pyhst_filter_t;

/* Operation selectors of pyhst_workspace_size(). */
enum { PYHST_OP_FBP = 0, PYHST_OP_BACKPROJECT = 1, PYHST_OP_PROJECT = 2, PYHST_OP_TV_SOLVE = 3 };

/* Workspace bytes one call of operation `op` needs for geometry `g` (host
 * pointer; the angle and axis pointers are not read).  For PYHST_OP_FBP the
 * size is for the default padding and min(n_slices, 4) slices per pass
 * (pyhst_fbp_workspace_size gives other choices); pyhst_fbp uses as many
 * slices per pass as the workspace holds, down to one.
 * Returns 0 for invalid arguments. */
size_t pyhst_workspace_size(const pyhst_geometry *g, int op);

/* Workspace bytes of pyhst_fbp with padding pad_len (0: the default) that
 * filters `slices_per_pass` slices per pass (clamped to [1, n_slices]).
 * Returns 0 for invalid arguments. */
size_t pyhst_fbp_workspace_size(const pyhst_geometry *g, int32_t pad_len, int32_t slices_per_pass);

/* Filtered back-projection of n_slices slices (Sec. 2.3).
 * For each slice z, angle a and bin b the input value is
 *     data[z * slice_stride + a * angle_stride + b]      (strides in elements)
 * so a raw radiography stack [n_angles][n_slices][n_bins] is read in place
 * with slice_stride = n_bins, angle_stride = n_slices * n_bins (the sinogram
 * of a detector row is a strided view; Sec. 2.3, rearrangement into
 * sinograms).  For *_RAW kinds, flat and dark are [n_slices][n_bins] float32
 * (averaged fields, Sec. 2.3) and p = -ln((I - D) / (F - D)) with p = 0 where
 * F - D <= 0 and the ratio clamped below at 1e-6; for *_SINO kinds flat and
 * dark are ignored (may be NULL).  Each row is Ram-Lak filtered (linear
 * convolution with h(0) = 1/4, h(odd n) = -1/(pi n)^2, h(even n) = 0,
 * computed as an FFT of length pad_len; pad_len = 0 picks the smallest power
 * of two >= 2 n_bins; otherwise pad_len must be a power of two in
 * [2 n_bins, 16384]), then back-projected with weight pi / (n_angles *
 * pixel_size).  out: [n_slices][ny][nx] float32, overwritten. */
int pyhst_fbp(const pyhst_geometry *g, int input_type, const void *data,
              int64_t slice_stride, int64_t angle_stride,
              const float *flat, const float *dark, int filter, int32_t pad_len,
              float *out, void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* Normalisation and ramp filter only (the first two steps of pyhst_fbp):
 * same inputs as pyhst_fbp, output q [n_slices][n_angles][n_bins] float32,
 * the filtered sinograms (no angular weight).  Workspace:
 * pyhst_filter_workspace_size (the FFT tables). */
size_t pyhst_filter_workspace_size(const pyhst_geometry *g, int32_t pad_len);
int pyhst_filter(const pyhst_geometry *g, int input_type, const void *data,
                 int64_t slice_stride, int64_t angle_stride,
                 const float *flat, const float *dark, int filter, int32_t pad_len,
                 float *q, void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* pyhst_fbp with HOST input and output: host_data (strides as in pyhst_fbp),
 * host_flat/host_dark [n_slices][n_bins] and host_out [n_slices][ny][nx] are
 * host memory (page-locked for the copies to overlap compute).  Chunks of at
 * most slices_per_chunk slices are copied to the device on an internal stream,
 * reconstructed on `stream` and copied back on a second internal stream, with
 * two buffers of each so that copies overlap compute; the chunks grow from one
 * slice (1, 4, 16, ...) at the start and shrink back to one at the end, so
 * that only one slice's copy in and one slice's copy back are not overlapped.
 * Each slice's result does not depend on the chunking.  The internal streams
 * start after the work already queued on `stream`, and the call's completion
 * is ordered on `stream` (synchronise it before reading host_out).  The
 * workspace (pyhst_fbp_host_workspace_size) holds the FBP scratch and the
 * double-buffered chunks. */
size_t pyhst_fbp_host_workspace_size(const pyhst_geometry *g, int input_type, int32_t pad_len,
                                     int32_t slices_per_chunk);
int pyhst_fbp_host(const pyhst_geometry *g, int input_type, const void *host_data,
                   int64_t slice_stride, int64_t angle_stride,
                   const float *host_flat, const float *host_dark, int filter, int32_t pad_len,
                   float *host_out, int32_t slices_per_chunk, void *workspace, size_t ws_bytes,
                   pyhst_stream_t stream);

/* pyhst_fbp without a workspace, for callers that cannot allocate device
 * memory (for example code inside a host framework that owns all device
 * allocations and exposes none to plug-ins, or an acquisition loop that may
 * not call cudaMalloc once it runs).  The paper has no counterpart: this is
 * an interface of this library only.  Arguments and results are those of
 * pyhst_fbp; the scratch is one fixed device array of
 * pyhst_fbp_static_max_bytes() bytes (32 MiB) inside the library, which every
 * GPU that loads the library holds until the process exits.  A geometry whose
 * angle table, FFT tables and one slice of filtered rows do not fit
 * (n_angles * n_bins * 4 bytes plus about 16 * pad_len bytes) is rejected with
 * PYHST_ERR_INVALID_ARG before anything runs.  The first call on a device
 * looks up the array's address on that device (make it before any stream
 * capture).  All calls share the array: calls that overlap on the GPU race on
 * it, so order them on one stream.  Nothing in it needs clearing between
 * calls; it allocates nothing. */
size_t pyhst_fbp_static_max_bytes(void);
int pyhst_fbp_static(const pyhst_geometry *g, int input_type, const void *data,
                     int64_t slice_stride, int64_t angle_stride,
                     const float *flat, const float *dark, int filter, int32_t pad_len,
                     float *out, pyhst_stream_t stream);

/* Preprocessing variants of Sec. 2.3 for pyhst_fbp_pre. */
typedef struct {
    int32_t n_flats;          /* >= 1 flats acquired at different times                     */
    const float *flats;       /* DEVICE [n_flats][n_slices][n_bins]                         */
    const float *flat_pos;    /* DEVICE [n_angles]: position of each projection between the
                                 flats (0 .. n_flats-1, clamped); the flat is the linear
                                 interpolation there; NULL when n_flats == 1               */
    float hotspot_threshold;  /* > 0: hot-spot median filter on r = (I - D) / (F - D): a pixel
                                 whose neighbours' median (up to 8 pixels around it in the
                                 (slice, bin) plane of its projection; mean of the two middle
                                 values for an even count) is below r - threshold takes that
                                 median.  0: off                                            */
    int32_t ring_window;      /* odd >= 3: ring filter, subtracting from each sinogram the
                                 high-pass part of its mean over angles (mean minus its
                                 moving average over this many bins).  0: off               */
} pyhst_preproc;

/* pyhst_fbp with the preprocessing of Sec. 2.3, in the paper's order
 * (dark/flat with flats interpolated in time, hot spots, -ln, sinograms, ring
 * filter, then the Ram-Lak filter and back-projection).  Raw kinds only; data
 * strides as in pyhst_fbp; dark [n_slices][n_bins]; the hot-spot filter reads
 * the neighbouring detector rows of the stack (slices 0 .. n_slices-1 are the
 * whole detector).  Workspace: pyhst_fbp_pre_workspace_size (slices_per_pass
 * slices of filtered and of preprocessed rows). */
size_t pyhst_fbp_pre_workspace_size(const pyhst_geometry *g, int32_t pad_len, int32_t slices_per_pass);
int pyhst_fbp_pre(const pyhst_geometry *g, int input_type, const void *data,
                  int64_t slice_stride, int64_t angle_stride, const float *dark,
                  const pyhst_preproc *pre, int filter, int32_t pad_len, float *out,
                  void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* Back-projection (Sec. 2.3) of n_slices sinograms [n_slices][n_angles][n_bins]
 * into images [n_slices][ny][nx]:
 *     img[i][j] = weight * sum_a L(sino_a, t_a(i, j))
 * (weight = pi / (n_angles * pixel_size) for FBP, pixel_size for the adjoint
 * of pyhst_project).  img is overwritten. */
int pyhst_backproject(const pyhst_geometry *g, const float *sino, float *img, float weight,
                      void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* Forward projection, the exact transpose of the unweighted back-projector
 * scaled by pixel_size (line integrals in physical units; the projector the
 * iterative methods use, Sec. 2.3 and Eq. 1):
 *     sino[a][b] = pixel_size * sum_{i,j} img[i][j] * max(0, 1 - |t_a(i,j) - b|)
 * img [n_slices][ny][nx] -> sino [n_slices][n_angles][n_bins], overwritten. */
int pyhst_project(const pyhst_geometry *g, const float *img, float *sino,
                  void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* Options of the TV-penalised solve (Eq. 3, Sec. 3.1). */
typedef struct {
    float beta;          /* weight of TV(x) in Eq. 3 (>= 0)                         */
    int32_t n_iter;      /* outer ISTA/FISTA iterations (>= 1)                      */
    int32_t n_inner;     /* Chambolle dual steps of each TV prox (>= 1)             */
    float tau;           /* Chambolle step (0 < tau <= 1/4; 1/8 is the safe bound)  */
    int32_t use_fista;   /* 1: FISTA momentum; 0: ISTA                              */
    int32_t warm_start;  /* 1: x holds the start iterate; 0: start from zeros       */
    double lipschitz;    /* L >= ||P||^2; 0: estimate 1.01 * lambda_max(P^T P)       */
    int32_t n_power_iter;/* power iterations of the estimate (from the all-ones image) */
    int32_t warm_dual;   /* 1: each TV prox after the first starts its Chambolle steps
                          * from the previous prox's final dual field (its input z
                          * moves little between outer iterations); 0: from a zero
                          * field, as the prox is defined (Sec. 3.1).  Changes the
                          * iterates; ignored by the learned prox. */
} pyhst_tv_opts;

/* Solve x = argmin 1/2 ||sino - P x||^2 + beta TV(x) (Eq. 3) for each of the
 * n_slices slices of g, with P = pyhst_project's operator and TV the
 * isotropic total variation of Eq. 2 (forward differences, Neumann
 * boundary).  Each outer iteration takes a gradient step of length 1/L and
 * the prox of (beta/L) TV by n_inner Chambolle steps from a zero dual field
 * (from the previous prox's field with warm_dual).
 *   sino   [n_slices][n_angles][n_bins]
 *   x      [n_slices][ny][nx]  in: start (if warm_start), out: last iterate
 *   energy [n_slices][n_iter] float64 DEVICE or NULL: Eq. 3 at every iterate
 *   gap    [n_slices][n_iter] float64 DEVICE or NULL: the duality gap of each
 *          iteration's TV prox (see pyhst_tv_prox; 0 when beta = 0), a measure
 *          of how far n_inner Chambolle steps leave the prox from its optimum
 *   lipschitz_out  DEVICE float64 [n_slices] or NULL: the L that was used. */
int pyhst_tv_solve(const pyhst_geometry *g, const float *sino, const pyhst_tv_opts *opts,
                   float *x, double *energy, double *gap, double *lipschitz_out,
                   void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* Workspace bytes of pyhst_tv_solve for a given option set (n_inner does not
 * matter; n_iter does not matter). */
size_t pyhst_tv_workspace_size(const pyhst_geometry *g, const pyhst_tv_opts *opts);

/* Proximal map of lam * TV (Eq. 2) for each of n_slices images [ny][nx]:
 *     x = argmin_x 1/2 ||x - z||^2 + lam TV(x)
 * by n_inner steps of Chambolle's dual fixed point from a zero dual field
 * (the TV prox inside pyhst_tv_solve; on its own it is the denoising case of
 * the paper's functional, where the projection operator is the identity,
 * Sec. 3.2.1).  z, x: [n_slices][ny][nx] float32; x must not overlap z
 * (PYHST_ERR_INVALID_ARG).  lam = 0 copies z.
 * gap [n_slices] float64 DEVICE or NULL: the ROF duality gap of the result,
 * primal 1/2 ||x - z||^2 + lam TV(x) minus dual 1/2 ||z||^2 - 1/2 ||z - lam div p||^2
 * for the final dual field p (|p| <= 1, x = z - lam div p); it is >= 0 and
 * bounds the primal suboptimality of x.  Evaluated as
 * lam * sum over pixels of (|grad x| + p . grad x), the same value written
 * as a sum of non-negative terms (float32 terms, float64 sums). */
size_t pyhst_tv_prox_workspace_size(int32_t nx, int32_t ny, int32_t n_slices);
int pyhst_tv_prox(const float *z, int32_t nx, int32_t ny, int32_t n_slices, float lam, int32_t n_inner,
                  float tau, float *x, double *gap, void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* Estimators of beta without ground truth (Sec. 4).  Reconstructs one slice
 * (geometry g, n_slices ignored) for each of the n_beta values betas (HOST
 * array; the first should be a very small beta, the paper's "0+") in one
 * batched solve with options opts, leaving out the projection at angle index
 * held_out (-1: use all projections), then returns, per beta:
 *   x     [n_beta][ny][nx]  the reconstructions;
 *   cv    [n_beta] float64 (DEVICE, or NULL; needs held_out >= 0): the
 *         cross-validation error || P_k x - y_k ||^2 at the held-out angle k;
 *   ecohe [n_beta] float64 (DEVICE, or NULL): Eq. 11,
 *         Cos(I(beta) - I(betas[0]), I(beta)) (NaN for a zero difference).
 * Workspace: pyhst_beta_scan_workspace_size. */
size_t pyhst_beta_scan_workspace_size(const pyhst_geometry *g, int32_t n_beta, int32_t held_out,
                                      const pyhst_tv_opts *opts);
int pyhst_beta_scan(const pyhst_geometry *g, const float *sino, const float *betas, int32_t n_beta,
                    int32_t held_out, const pyhst_tv_opts *opts, float *x, double *cv, double *ecohe,
                    void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* Opt-in per-kernel timing for measurement: while enabled (per host thread),
 * every launch of the back-projection, filter, projection and fused Chambolle
 * kernels is bracketed by CUDA events on its launch stream (event-record nodes
 * when the stream is being captured into a CUDA graph, as in
 * pyhst_tv_solve_batch).  pyhst_profile_read waits for the recorded launches
 * of one kernel ("backproject", "filter", "project" or "chambolle"), returns
 * their summed duration (ms) and count, and forgets them. */
int pyhst_profile_enable(int on);
int pyhst_profile_read(const char *kernel, double *total_ms, int64_t *launches);

/* Measurement support: microbenchmarks of the on-chip rates that bound the
 * back-projector and the projector (shared memory, FP32) and the Chambolle
 * steps (MUFU), the denominators of their rooflines.
 *   kind 0: shared-memory reads, 8-byte loads with no bank conflicts (256
 *           bytes per warp instruction, two wavefronts); *units = bytes read;
 *   kind 1: FP32 fma chains, scalar;        *units = flops (an fma is two);
 *   kind 2: FP32 fma chains, paired f32x2;  *units = flops;
 *   kind 3: approximate reciprocal and square-root chains (the XU pipe's
 *           MUFU operations);               *units = MUFU operations.
 * One launch of 4 CTAs x 256 threads per SM, iters loop iterations, on the
 * stream (asynchronous; time it with events around the call).  sink: DEVICE
 * float buffer of pyhst_microbench_sink_floats() floats that receives the
 * loops' results (values without meaning).  PYHST_ERR_INVALID_ARG for another
 * kind, iters < 1 or NULL pointers. */
size_t pyhst_microbench_sink_floats(void);
int pyhst_microbench(int32_t kind, int32_t iters, float *sink, double *units, pyhst_stream_t stream);

/* One slice of a mixed-size batch: its own geometry (n_slices is ignored),
 * sinogram [n_angles][n_bins], iterate x [ny][nx] (in: start if warm_start,
 * out: result), energy [n_iter] and prox duality gaps [n_iter] float64
 * (DEVICE, or NULL; as in pyhst_tv_solve) and its own beta (>= 0; a negative
 * value takes the options' beta). */
typedef struct {
    pyhst_geometry geom;
    const float *sino;
    float *x;
    double *energy;
    double *gap;
    float beta;
} pyhst_tv_item;

/* Autotuning of the TV prox.  The Chambolle steps run fused, several per
 * launch on shared-memory tiles; the number fused per launch (2, 3, 4, 5, 6
 * or 8) trades halo recomputation against launches and gives bit-identical
 * results.  pyhst_autotune_tv_prox times every choice on the caller's z
 * [n_slices][ny][nx] (DEVICE; workspace: pyhst_tv_prox_workspace_size),
 * synchronizing `stream`, and records the fastest for images of ny x nx on
 * the current device; pyhst_tv_prox, pyhst_tv_solve, pyhst_pnp_solve,
 * pyhst_beta_scan and pyhst_tv_solve_batch (for its largest slice size) then
 * use it.  pyhst_set_tv_prox_steps records a choice directly (0 clears it;
 * the default is 5). */
int pyhst_autotune_tv_prox(const float *z, int32_t nx, int32_t ny, int32_t n_slices, float lam, int32_t n_inner,
                           float tau, void *workspace, size_t ws_bytes, int32_t *best_steps, pyhst_stream_t stream);
int pyhst_set_tv_prox_steps(int32_t nx, int32_t ny, int32_t steps);

/* Autotuning of the back-projector.  Each CTA stages the filtered rows of a
 * block of angles at a time; the block size (8, 16 or 24 angles) trades
 * barriers and set-up per angle against the padding slots of a last, partial
 * block, and gives identical results (every pixel sums its angles in the same
 * order).  pyhst_autotune_backproject times every choice on the caller's
 * sinograms sino [n_slices][n_angles][n_bins] (DEVICE; img receives the
 * back-projection, workspace as pyhst_backproject's), synchronizing `stream`,
 * and records the fastest for (nx, ny, n_angles) on the current device;
 * pyhst_backproject, the FBP entry points, the TV solvers and
 * pyhst_tv_solve_batch (for its geometry with the most updates) then use it.
 * pyhst_set_backproject_block records a choice directly (0 clears it; the
 * default is 16). */
int pyhst_autotune_backproject(const pyhst_geometry *g, const float *sino, float *img, void *workspace,
                               size_t ws_bytes, int32_t *best, pyhst_stream_t stream);
int pyhst_set_backproject_block(int32_t nx, int32_t ny, int32_t n_angles, int32_t angles_per_block);

/* Autotuning of the projector.  A CTA stages, per 16 image rows, the band of
 * columns its rays cross, in a buffer of 256, 384 or 512 columns (a band that
 * does not fit is walked in smaller angle subsets); the width trades shared
 * memory and staging work against those extra walks, and gives identical
 * results (every ray is walked with the same fixed-point positions, in the
 * same row order).  pyhst_autotune_project times every width on the caller's images
 * img [n_slices][ny][nx] (DEVICE; sino receives the projection, workspace as
 * pyhst_project's), synchronizing `stream`, and records the fastest for
 * (nx, ny, n_angles) on the current device; pyhst_project, the TV solvers and
 * pyhst_tv_solve_batch (per slice geometry) then use it.
 * pyhst_set_project_staging records a choice directly (0 clears it; the
 * default is 512 when max(nx, ny) > 2 n_angles, else 256). */
int pyhst_autotune_project(const pyhst_geometry *g, const float *img, float *sino, void *workspace, size_t ws_bytes,
                           int32_t *best, pyhst_stream_t stream);
int pyhst_set_project_staging(int32_t nx, int32_t ny, int32_t n_angles, int32_t width);

/* pyhst_tv_solve for many slices of different sizes and angle sets at once
 * (same options for all): every stage of an iteration is one launch over the
 * whole batch, and the n_iter iterations are captured in one CUDA graph on
 * `stream` (when `stream` is not already capturing and is not the legacy
 * NULL stream, where the launches are issued directly).  The step size is
 * estimated once per distinct geometry (same angle and axis pointers, sizes,
 * centre and pixel size).  items is a HOST array of n_items entries whose
 * pointers are device memory; lipschitz_out: DEVICE float64 [n_items] or
 * NULL.  The call copies small tables from host memory into the workspace
 * (pyhst_tv_batch_workspace_size) before launching. */
size_t pyhst_tv_batch_workspace_size(const pyhst_tv_item *items, int32_t n_items, const pyhst_tv_opts *opts);
int pyhst_tv_solve_batch(const pyhst_tv_item *items, int32_t n_items, const pyhst_tv_opts *opts,
                         double *lipschitz_out, void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* ------------------------------------------------------------------------
 * Learned proximal denoiser: a residual CNN that can replace the TV prox in
 * the FISTA loop (Sec. 3.2 introduces learned priors with the patch
 * dictionary; the network is a convolutional learned prior).
 *
 *   a_0 = z;  a_l = ReLU(conv3x3(a_{l-1}; W_l) + b_l), l = 1..7;
 *   out = z + conv3x3(a_7; W_8) + b_8
 *
 * Channel widths 1, 32 x 7, 1; conv3x3 is cross-correlation with zero
 * padding.  Weights and the hidden activations a_1..a_7 are bfloat16 (round
 * to nearest even), sums float32 (the 32 -> 32 layers on the tensor cores),
 * z, the biases and out float32.
 *
 * params: DEVICE float32 [pyhst_cnn_param_count()] in the order W_1, b_1,
 * ..., W_8, b_8 with W_l [C_out][C_in][3][3] row-major (float32 master
 * values; the call rounds the weights to bfloat16).
 * ------------------------------------------------------------------------ */
int64_t pyhst_cnn_param_count(void);

/* Workspace of pyhst_cnn_forward for n_images of ny x nx:
 * two bfloat16 activation buffers (64 bytes per pixel each) + packed
 * weights.  0 for invalid sizes. */
size_t pyhst_cnn_workspace_size(int32_t n_images, int32_t ny, int32_t nx);

/* out [n_images][ny][nx] = network(z [n_images][ny][nx]), all DEVICE
 * float32; out may equal z.  1 <= n_images <= 65535, 1 <= ny, nx <= 16384. */
int pyhst_cnn_forward(const float *params, const float *z, float *out, int32_t n_images, int32_t ny, int32_t nx,
                      void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* Training.  Workspace of pyhst_cnn_grad for n_images of ny x nx (all seven
 * hidden activations are kept: ~9 x 64 bytes per pixel). */
size_t pyhst_cnn_train_workspace_size(int32_t n_images, int32_t ny, int32_t nx);

/* Loss = mean over every pixel of the batch of (network(z) - target)^2 and
 * its gradient grad [pyhst_cnn_param_count()] (DEVICE float32, same layout
 * as params), by the chain rule through the bf16 network (the rounding of
 * stored values is differentiated as the identity; gradients of the hidden
 * pre-activations are stored as bf16).  Weight gradients are summed over
 * pixels in a fixed order (deterministic).  loss: DEVICE float64 or NULL. */
int pyhst_cnn_grad(const float *params, const float *z, const float *target, int32_t n_images, int32_t ny,
                   int32_t nx, float *grad, double *loss, void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* One Adam step (Kingma & Ba 2015) on count DEVICE float32 values:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).  step >= 1. */
int pyhst_cnn_adam(float *params, const float *grad, float *m, float *v, int64_t count, int32_t step, float lr,
                   float beta1, float beta2, float eps, pyhst_stream_t stream);

/* FISTA/ISTA with the learned prox (plug-and-play): pyhst_tv_solve's
 * iteration with x_k = network(z_k) in place of the TV prox of z_k, for the
 * n_slices slices of g.  opts: n_iter, use_fista, warm_start, lipschitz and
 * n_power_iter are used; beta, n_inner and tau are ignored.  energy [n_slices][n_iter]
 * (DEVICE float64, or NULL) records the data term
 * 1/2 ||sino - P x_k||^2.  Workspace: pyhst_pnp_workspace_size. */
size_t pyhst_pnp_workspace_size(const pyhst_geometry *g);
int pyhst_pnp_solve(const pyhst_geometry *g, const float *sino, const float *params, const pyhst_tv_opts *opts,
                    float *x, double *energy, double *lipschitz_out, void *workspace, size_t ws_bytes,
                    pyhst_stream_t stream);

/* pyhst_tv_solve (without energies) that also copies the prox input
 * z_k = y_k - (1/L) P^T (P y_k - sino) of iterations capture_iters[c]
 * (HOST array, 1-based, each in [1, n_iter]) into capture + c n_slices ny nx
 * (DEVICE float32).  Same workspace as pyhst_tv_solve. */
int pyhst_tv_solve_capture(const pyhst_geometry *g, const float *sino, const pyhst_tv_opts *opts, float *x,
                           int32_t n_capture, const int32_t *capture_iters, float *capture, void *workspace,
                           size_t ws_bytes, pyhst_stream_t stream);

/* ------------------------------------------------------------------------
 * Overlapping-patch prior (Sec. 3.2.1).  m x m patches on a grid of step
 * `stride` (1 <= stride <= m <= 16): along an axis of n pixels patch k starts
 * at min(k stride, n - m), k = 0 .. K-1, K = ceil((n - m) / stride) + 1, so
 * the patches cover the image (Eq. 4).  The core of a pixel (Eqs. 5-6) is the
 * patch with the nearest centre start + (m-1)/2 along each axis (ties to the
 * lower index).  Coefficients W [N][n_atoms] (N = K_rows K_cols, patch index
 * k_row K_cols + k_col), dictionary D [n_atoms][m m] (patch pixels
 * row-major); patches P = W D; the image takes each pixel from its core
 * patch (Eq. 7):  x_j = P[core(j)][j - r_core(j)].
 *   f(W) = ||y - Pi x||^2 + rho sum_p sum_{i in p} (x_{r_p + i} - P_{p,i})^2   (Eq. 8)
 *   F(W) = f(W) + beta ||W||_1
 * Pi is the projector of `g` (pyhst_project's operator, one slice) or, with
 * g = NULL, the identity (denoising; y is then an ny x nx image).
 * All arrays are DEVICE float32 unless stated.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t ny, nx;        /* image size                                      */
    int32_t m, stride;     /* patch size and grid step                         */
    int32_t n_atoms;       /* dictionary size (n_atoms x m^2 <= 65536)         */
    const float *dict;     /* DEVICE [n_atoms][m*m]                            */
    float rho;             /* weight of the patch-agreement term (>= 0)        */
} pyhst_patch_problem;

/* Patches per axis (host, no GPU work); PYHST_ERR_INVALID_ARG for bad sizes. */
int pyhst_patch_grid(int32_t ny, int32_t nx, int32_t m, int32_t stride, int32_t *k_rows, int32_t *k_cols);

/* Workspace of the calls below (g: NULL for denoising). */
size_t pyhst_patch_workspace_size(const pyhst_patch_problem *pp, const pyhst_geometry *g);

/* x [ny][nx] = the image of the coefficients W (Eq. 7). */
int pyhst_patch_image(const pyhst_patch_problem *pp, const float *W, float *x, void *workspace, size_t ws_bytes,
                      pyhst_stream_t stream);

/* G [N][n_atoms] = gradient of f at W (Eq. 9), computed with the steps of
 * Algorithm 1 (P = W D, the image from the cores, R = Pi^T (Pi x - y), the
 * patch sum S and cover count, the auxiliary patches P', G = 2 P' D^T).
 * f_out: DEVICE float64 [1] or NULL, receives f(W) (Eq. 8).  The two
 * dictionary products run on the tensor cores with both operands split into
 * three bf16 terms (float32 accuracy) when the padded dictionary side fits
 * (<= 256 columns); a completion wait there that gives up sets bit 1 of
 * pyhst_device_status. */
int pyhst_patch_gradient(const pyhst_patch_problem *pp, const pyhst_geometry *g, const float *W, const float *y,
                         float *G, double *f_out, void *workspace, size_t ws_bytes, pyhst_stream_t stream);

/* ISTA / FISTA on F(W) (Sec. 3.2.2): a gradient step of length 1/L on f,
 * then the L1 shrinkage sign(v) max(|v| - beta/L, 0), FISTA momentum of
 * Beck-Teboulle.  lipschitz > 0: L; 0: L = 1.01 x the largest eigenvalue of
 * f's (constant) Hessian by n_power_iter power iterations from W = 1.
 * W [N][n_atoms] in: start, out: last iterate; x (or NULL) receives its
 * image; energy: DEVICE float64 [n_iter] or NULL, F at every iterate;
 * lipschitz_out: DEVICE float64 [1] or NULL. */
int pyhst_patch_solve(const pyhst_patch_problem *pp, const pyhst_geometry *g, const float *y, float beta,
                      double lipschitz, int32_t n_power_iter, int32_t n_iter, int32_t use_fista, float *W, float *x,
                      double *energy, double *lipschitz_out, void *workspace, size_t ws_bytes,
                      pyhst_stream_t stream);

/* Error bits recorded on the current device by kernels whose bounded waits
 * gave up (1: a tensor-core completion wait), since the last clear.  Reads
 * the word synchronously; clear != 0 resets it.  A kernel whose wait gave up
 * stops issuing work, waits (with the default limit) for the tensor-core
 * operations it already issued, frees its tensor memory and returns; its
 * output is then incomplete. */
int pyhst_device_status(uint32_t *flags, int32_t clear);

/* Failure detection (the paper has no counterpart): number of polls after
 * which the pipeline waits of the tensor-core kernels (CNN convolutions,
 * patch products) give up; a negative value restores the default (2^22
 * polls, far longer than any healthy wait), 0 makes every such wait give up
 * without polling, so that tests can exercise the give-up path and
 * pyhst_device_status without a GPU fault.  Process-wide; takes effect at the
 * next launch.  PYHST_ERR_INVALID_ARG above 2^32 - 1. */
int pyhst_set_wait_limit(int64_t polls);

/* Message of the last failed call on this host thread ("" if none). */
const char *pyhst_last_error(void);

/* Library version string. */
const char *pyhst_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PYHST_H */
