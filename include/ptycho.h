/*
 * libptycho: multislice ptychography loss and image gradient on one GB300 GPU.
 *
 * The library evaluates the amplitude cost of Eq. 1 (Sec. II-B),
 *     F = sum_i sum_k ( sqrt(I_i[k]) - |G(P, O)_i[k]| )^2,
 * where G is the multislice model of Sec. II-B (each slice transmits the
 * wave, which is then Fourier transformed, multiplied by the Fresnel
 * propagator and inverse transformed before the next slice; the exit wave is
 * Fourier transformed to the detector), together with its exact gradient,
 * which by Eq. 2 (Sec. III) is the sum of per-position gradients, each
 * supported on its own probe window.
 *
 * Conventions (fixed, not options):
 *   - complex numbers are interleaved float pairs (re, im), i.e. complex64;
 *   - 2-D FFTs are orthonormal with forward kernel exp(-2 pi i k.n / M); the
 *     far field and the measurements are in FFT order (DC at [0][0]);
 *   - the Fresnel propagator between consecutive slices is
 *     h(ky, kx) = exp(-i pi lambda dz (ky^2 + kx^2)), k = fftfreq(M, pixel)
 *     in 1/Angstrom, applied S-1 times for S slices;
 *   - one probe P [M][M] is shared by all positions; position i is the
 *     integer top-left corner (y_i, x_i) of its M x M window in the object,
 *     with 0 <= y_i <= H-M and 0 <= x_i <= W-M (no wrap-around);
 *   - gradients are g = dF/dRe + i dF/dIm (PyTorch's convention), written
 *     (overwritten, never accumulated) into caller-owned buffers;
 *   - where |Psi| = 0 the amplitude's subgradient Psi/|Psi| is taken as 0.
 *
 * Memory: every array argument is caller-owned and must be CUDA device
 * memory (cudaMalloc / PyTorch), except where an argument says a host
 * pointer is accepted.  The plan owns only its tables and its workspace;
 * nothing is freed across this interface.
 *
 * Streams: work is enqueued on the stream given to each call (NULL = the
 * legacy default stream) and runs asynchronously unless stated otherwise;
 * outputs are valid once that stream has been synchronised.  A plan's
 * workspace serves one call at a time: calls on one plan must be ordered
 * (the same stream, or streams the caller orders); different plans are
 * independent.  Inside a gradient call the library may fork part of the
 * work onto a stream of its own and join it back into the call's stream
 * with events, so the call stays ordered on that stream and can be captured
 * in a CUDA graph.
 *
 * Errors: every entry point returns PTYCHO_OK (0) or a negative code and
 * records a message retrievable with ptycho_last_error() (per host thread).
 */
#ifndef PTYCHO_H_
#define PTYCHO_H_

#include <stdint.h>

#if defined(__GNUC__)
#define PTYCHO_API __attribute__((visibility("default")))
#else
#define PTYCHO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define PTYCHO_OK              0
#define PTYCHO_ERR_ARG        -1  /* null pointer, bad shape or parameter */
#define PTYCHO_ERR_POSITION   -2  /* a probe window lies outside the object */
#define PTYCHO_ERR_CUDA       -3  /* a CUDA runtime call failed */
#define PTYCHO_ERR_NOMEM      -4  /* workspace allocation failed */
#define PTYCHO_ERR_TIMEOUT    -5  /* a bounded device-side wait gave up (reported
                                     by ptycho_plan_status after the stream syncs) */
#define PTYCHO_ERR_UNSUPPORTED -6 /* probe window size not supported */

#define PTYCHO_FP32    0   /* all bulk complex arithmetic in FP32 */
#define PTYCHO_BF16X3  1   /* the 2-D transforms as DFT-matrix products on the
                              tensor cores: operands split into BF16 hi + lo,
                              three products per real product (hi*hi, hi*lo,
                              lo*hi), FP32 accumulation; pointwise work FP32,
                              loss FP64.  M = 128 only. */
#define PTYCHO_FP16X3  2   /* the same with IEEE half hi + lo (22 significant
                              bits instead of 16, same tensor rate); wave
                              values must stay below 60000 in magnitude, else
                              ptycho_plan_status reports PTYCHO_ERR_UNSUPPORTED. */

/* Flags for ptycho_params.flags */
#define PTYCHO_FLAG_ASYNC_CHECK 1  /* do not synchronise to validate positions
                                      on the host; out-of-range windows are
                                      skipped on the device and reported by
                                      ptycho_plan_status() */
#define PTYCHO_FLAG_TIMING      2  /* record CUDA events around every kernel
                                      family on the call's stream; read them
                                      with ptycho_plan_timing() */
#define PTYCHO_FLAG_SELFTEST_TIMEOUT 4 /* diagnostic, split precisions only: the
                                      kernel issues no tensor-core work and
                                      waits for it anyway, so its bounded wait
                                      (about 1 s) expires, it releases tensor
                                      memory and ptycho_plan_status reports
                                      PTYCHO_ERR_TIMEOUT.  Exercises that path
                                      without a GPU fault; results are
                                      meaningless. */

typedef struct {
  float re, im;
} ptycho_c64;

/* Problem description (Sec. II-B, Eq. 1).  Windows: M = 64 and 128 run the
 * register-resident kernels; with PTYCHO_FP32 any other M = 2^a 3^b in
 * [8, 4096] runs the generic line-pass path; the split precisions take
 * M = 128 only.  Other windows give PTYCHO_ERR_UNSUPPORTED. */
typedef struct {
  int32_t M;          /* probe window / detector side, pixels */
  int32_t S;          /* number of object slices */
  int32_t H, W;       /* object height and width, pixels */
  int32_t N;          /* number of probe positions per call */
  double lambda_A;    /* wavelength, Angstrom */
  double dz_A;        /* slice spacing, Angstrom */
  double pixel_A;     /* real-space pixel, Angstrom */
  int32_t precision;  /* PTYCHO_FP32, PTYCHO_BF16X3 or PTYCHO_FP16X3 */
  int32_t flags;      /* PTYCHO_FLAG_* */
  int64_t workspace_bytes; /* cap on the plan's workspace; 0 = 8 GiB.  Positions
                              are processed in chunks that fit the cap, so the
                              memory used does not grow with N. */
  int32_t tile_h, tile_w;  /* object-gradient accumulation tile (pixels);
                              0 = 32 x 32.  tile_h * tile_w <= 8192. */
  int32_t ckpt_every; /* 0: keep every slice's wave for the adjoint (fastest).
                         L >= 1: per-slice recomputation.  Keep the waves
                         entering every L-th slice (checkpoints), and during
                         the adjoint rebuild one segment of L slices at a
                         time from its checkpoint; each segment's gradient
                         patches are summed into grad_obj before the next
                         segment is rebuilt.  With K = ceil(S / L) segments
                         the workspace per position holds K + L wave-sized
                         buffers (K - 2 checkpoints, one segment, the parked
                         adjoint state, the probe gradient) instead of 2S
                         (the generic-window path: K + 2L + 1, the segment's
                         exit-wave gradients and the chunk's wave buffer
                         besides), for (K - 1)(L - 1) extra propagations.
                         L = 0 is
                         used when L >= S.  PTYCHO_CKPT_AUTO: K =
                         ceil(sqrt(S)), L = ceil(S / K): about 2 sqrt(S)
                         buffers.  Applies to the FP32 path (every window);
                         the split precisions keep every wave. */
} ptycho_params;

#define PTYCHO_CKPT_AUTO (-1)  /* ptycho_params.ckpt_every: ceil(sqrt(S)) checkpoints */

typedef struct ptycho_plan_s* ptycho_plan;

/* Create a plan: validates *params, computes the FFT twiddles and the
 * Fresnel propagator in FP64 on the host, uploads them as FP32 tables and
 * allocates the workspace.  The caller's current CUDA device is used.
 * Returns PTYCHO_ERR_ARG / _UNSUPPORTED / _NOMEM / _CUDA on failure, in which
 * case *plan is set to NULL. */
PTYCHO_API int ptycho_plan_create(ptycho_plan* plan, const ptycho_params* params);

/* Release the plan's tables and workspace (synchronises the device). */
PTYCHO_API int ptycho_plan_destroy(ptycho_plan plan);

/* Number of positions processed per chunk and workspace bytes held. */
PTYCHO_API int ptycho_plan_info(ptycho_plan plan, int32_t* chunk_positions, int64_t* workspace_bytes);

/* Device-side status of the calls on this plan since the last read (after
 * the stream has been synchronised), and clears it: PTYCHO_OK,
 * PTYCHO_ERR_POSITION (a window outside the object was skipped),
 * PTYCHO_ERR_TIMEOUT (a bounded tensor-core wait gave up) or
 * PTYCHO_ERR_UNSUPPORTED (a wave value left the FP16 range). */
PTYCHO_API int ptycho_plan_status(ptycho_plan plan);

/* Forward model G (Sec. II-B) for all N positions.
 *   pos_yx     int32 [N][2]   device, (y, x) window corners
 *   probe      c64   [M][M]   device
 *   obj        c64   [S][H][W] device, slice transmissions O_s
 *   psi_out    c64   [N][M][M] device or NULL: orthonormal far field, FFT order
 *   intens_out f32   [N][M][M] device or NULL: |psi_out|^2
 * At least one output must be non-NULL. */
PTYCHO_API int ptycho_forward(ptycho_plan plan, const int32_t* pos_yx, const ptycho_c64* probe,
                   const ptycho_c64* obj, ptycho_c64* psi_out, float* intens_out,
                   void* stream);

/* Cost of Eq. 1 and its gradients (Eq. 2).
 *   meas_I     f32 [N][M][M] device, measured intensities (>= 0), FFT order
 *   loss_out   double[1], device or host pointer: F, accumulated in FP64.
 *              For a host pointer the call synchronises the stream.
 *   grad_obj   c64 [S][H][W] device or NULL: dF/dO (overwritten; zero outside
 *              every window)
 *   grad_probe c64 [M][M] device or NULL: dF/dP (overwritten)
 * Deterministic: the same inputs give bit-identical outputs (fixed-order
 * reductions, no atomics). */
PTYCHO_API int ptycho_loss_grad(ptycho_plan plan, const int32_t* pos_yx, const ptycho_c64* probe,
                     const ptycho_c64* obj, const float* meas_I, double* loss_out,
                     ptycho_c64* grad_obj, ptycho_c64* grad_probe, void* stream);

/* ptycho_loss_grad with every array in HOST memory, for callers whose data
 * live on the host.  Same operation (Eq. 1, Eq. 2), arguments, layouts and
 * results bit for bit; the call is synchronous: it returns when loss_out,
 * grad_obj and grad_probe hold the results.
 *   pos_yx, probe, obj, meas_I   host inputs (layouts as above).  Pinned
 *       memory (cudaHostAlloc, or PyTorch's pin_memory) lets the uploads
 *       run beside the kernels; pageable memory works with plain copies.
 *   loss_out   double[1] host (required)
 *   grad_obj, grad_probe   host outputs, or NULL
 * The plan keeps device copies of the inputs and gradients (allocated on the
 * first call: (N M^2 4 + 2 S H W 8 + 2 M^2 8 + N 8) bytes) and a copy
 * stream.  Positions are checked on the host before any upload.  The object
 * and the first chain wave's intensities go up on `stream`; the other
 * intensities go up on the copy stream while that wave runs, and the chain of
 * the later positions waits for them.  Errors as for ptycho_loss_grad, and
 * PTYCHO_ERR_ARG when an array is a device pointer.  A device-side error
 * (a bounded wait that gave up, the FP16 range) is returned by this call
 * itself, as ptycho_plan_status would return it, and the results are then
 * undefined.  The paper has no counterpart: it is a packaging of the same
 * kernels. */
PTYCHO_API int ptycho_loss_grad_host(ptycho_plan plan, const int32_t* pos_yx, const ptycho_c64* probe,
                     const ptycho_c64* obj, const float* meas_I, double* loss_out,
                     ptycho_c64* grad_obj, ptycho_c64* grad_probe, void* stream);

/* One full-batch gradient-descent step (Sec. II-B update rule, applied to the
 * position sum of Eq. 2): O <- O - t alpha_obj dF/dO, P <- P - t alpha_probe dF/dP,
 * in place.  line_search = 0: t = 1.  line_search = 1: Armijo backtracking,
 * t = 1, 1/2, ... (at most 20 halvings) until
 *   F(new) <= F(old) - 1e-4 t (alpha_obj |dF/dO|^2 + alpha_probe |dF/dP|^2),
 * else t = 0 (inputs unchanged).  The scalars are FP64; the line search reads
 * them on the host and therefore synchronises the stream.
 *   loss_out   double[1] device or host, or NULL: F before the step
 *   t_out      double[1] host, or NULL: the accepted t */
PTYCHO_API int ptycho_step(ptycho_plan plan, const int32_t* pos_yx, ptycho_c64* probe, ptycho_c64* obj,
                const float* meas_I, double alpha_obj, double alpha_probe,
                int32_t line_search, double* loss_out, double* t_out, void* stream);

/* Algorithm 1's per-location update with its delayed accumulation, for the
 * positions of this call (one position per call for Algorithm 1 itself):
 * the update of ptycho_step without line search, O <- O - alpha_obj dF/dO,
 * P <- P - alpha_probe dF/dP, and the accumulated-gradient buffer
 * acc <- acc + dF/dO.  With flush != 0 (the caller's counter of locations
 * reached a multiple of the period T) it then applies the buffer as the
 * second update, O <- O - alpha_obj acc, and clears it.  On one GPU the
 * whole object is one tile, so the passes that would add the neighbouring
 * tiles' buffers before the second update have nothing to add.
 *   acc        c64 [S][H][W] device, caller-owned, updated in place; it must
 *              not overlap obj or probe
 *   loss_out   double[1] device or host, or NULL: F (these positions) before the update
 * The paper updates only V; pass alpha_probe = 0 to keep the probe fixed. */
PTYCHO_API int ptycho_step_accumulate(ptycho_plan plan, const int32_t* pos_yx, ptycho_c64* probe,
                                      ptycho_c64* obj, const float* meas_I, double alpha_obj,
                                      double alpha_probe, ptycho_c64* acc, int32_t flush, double* loss_out,
                                      void* stream);

/* Several independent reconstructions in one call (the batched workload:
 * problems of different windows, slice counts and sizes).  Each problem has
 * its own plan and arrays, as for the single-problem calls; two entries may
 * not share a plan, and problems must not share output arrays.  The
 * problems' work is enqueued on `stream`, so one call can be captured in one
 * CUDA graph when every plan uses PTYCHO_FLAG_ASYNC_CHECK: first, in order,
 * the problems the register-resident kernels do not take; then the FP32
 * problems with M = 64 or 128 that keep every wave, grouped by window, whose
 * chains of chunk r run in one launch per group (up to 16 problems per
 * launch), each followed by that problem's reductions of the chunk.  The
 * call never synchronises (unless a plan lacks PTYCHO_FLAG_ASYNC_CHECK):
 * loss_out must be a device pointer or NULL.  Results are bit-identical to
 * the single-problem calls.  On an error the message names the problem; the
 * work enqueued before it stays enqueued.  The paper has no counterpart: it
 * reconstructs one dataset at a time. */
typedef struct {
  ptycho_plan plan;
  const int32_t* pos_yx;   /* [N][2] device */
  ptycho_c64* probe;       /* [M][M] device (updated in place by ptycho_multi_step) */
  ptycho_c64* obj;         /* [S][H][W] device (updated in place by ptycho_multi_step) */
  const float* meas_I;     /* [N][M][M] device */
  double* loss_out;        /* device, or NULL: F (before the step) */
  ptycho_c64* grad_obj;    /* ptycho_multi_loss_grad: [S][H][W] device or NULL */
  ptycho_c64* grad_probe;  /* ptycho_multi_loss_grad: [M][M] device or NULL */
} ptycho_problem;

/* ptycho_loss_grad for every problem. */
PTYCHO_API int ptycho_multi_loss_grad(const ptycho_problem* problems, int32_t n, void* stream);

/* ptycho_step with a fixed step (t = 1, no line search) for every problem,
 * with the same alpha_obj, alpha_probe. */
PTYCHO_API int ptycho_multi_step(const ptycho_problem* problems, int32_t n, double alpha_obj,
                                 double alpha_probe, void* stream);

/* Per-kernel-family device time and launch counts accumulated since the
 * last reset.  Times are filled only for plans created with
 * PTYCHO_FLAG_TIMING (CUDA events on the call's stream); launch counts are
 * always kept.  Synchronises on the recorded events.  reset != 0 clears. */
typedef struct {
  double chain_ms;        /* per-position slice-chain kernels (forward/adjoint) */
  double accum_ms;        /* object-gradient tiled accumulation */
  double probe_ms;        /* probe-gradient reduction */
  double other_ms;        /* loss reduction, checks, step vector kernels */
  int64_t chain_launches;
  int64_t accum_launches;
  int64_t launches;       /* all kernels this library launched */
  int64_t chain_positions; /* positions processed by the chain kernels */
} ptycho_timing;

PTYCHO_API int ptycho_plan_timing(ptycho_plan plan, ptycho_timing* out, int32_t reset);

/* Loss and gradients exactly as ptycho_loss_grad, for callers that cannot
 * allocate device memory: code that runs inside a custom device allocator or
 * a memory-pool callback (where calling cudaMalloc would re-enter it), or a
 * process whose device allocations are fixed after start-up.  It allocates
 * nothing -- no plan, no cudaMalloc/cudaFree, no allocating library call.
 * The paper has no counterpart: this is the same kernels, differently fed.
 *
 * Limits: M = 64 or 128 only (other windows: PTYCHO_ERR_UNSUPPORTED),
 * PTYCHO_FP32 only, and every wave is kept (no recompute mode:
 * params->ckpt_every is ignored).
 *
 * Scratch: one static device array of 64 MiB, held by every GPU that loads
 * the library until the process exits.  A fixed part (the twiddle and
 * propagator tables, among them the M * M * 8-byte full propagator,
 * 4 * M * M * 8 bytes of probe-gradient partials and a few words; about
 * 0.63 MiB at M = 128) comes first; positions then run in chunks
 * that fit in the rest, each position needing
 *     (2S - 1) * M * M * 8 + M * M * 8 + 8 bytes
 * (S = 253 is the deepest chain at M = 128, S = 1021 at M = 64).  A problem whose
 * single position does not fit returns PTYCHO_ERR_UNSUPPORTED.
 * The first call on a device looks up the array's device address (and sets
 * the kernels' shared-memory limit); make that first call before any stream
 * capture.  Every call shares the array and keeps the previous call's
 * contents (what must start at zero is cleared by each call): calls that
 * overlap on the GPU -- two streams, two host threads, two devices sharing
 * nothing else are fine only if they do not run at the same time on the same
 * device -- race on it.
 *   params     problem description (tile_h/tile_w as for plans; flags,
 *              workspace_bytes and ckpt_every are ignored)
 *   pos_yx, probe, obj, meas_I, grad_obj, grad_probe: as ptycho_loss_grad,
 *              device pointers, 8-byte aligned (else PTYCHO_ERR_ARG, checked
 *              before anything is launched)
 *   loss_out   double[1], device or host (required)
 * Positions are checked on the device; the call then synchronises the stream
 * and returns PTYCHO_ERR_POSITION if a window lay outside the object (that
 * window contributes nothing; the loss and gradients of the others are still
 * written).  Errors are reported by the return code only (ptycho_last_error()
 * is not updated). */
PTYCHO_API int ptycho_loss_grad_noalloc(const ptycho_params* params, const int32_t* pos_yx,
                                        const ptycho_c64* probe, const ptycho_c64* obj,
                                        const float* meas_I, double* loss_out, ptycho_c64* grad_obj,
                                        ptycho_c64* grad_probe, void* stream);

/* Potential parameterisation.  The paper's unknown is the real scattering
 * potential V (Sec. II-B, Eq. 1); the slices transmit O = exp(i sigma V).
 * ptycho_potential_to_transmission: obj[k] = exp(i sigma V[k]), k < n.
 * ptycho_potential_grad: grad_V[k] = sigma * Im(conj(obj[k]) * grad_obj[k]),
 * the chain rule of dF/dO through O = exp(i sigma V) (with the gradient
 * convention above), so that gradient descent can update V directly.
 *   V, grad_V   float [n] device;  obj, grad_obj  c64 [n] device (e.g. [S][H][W]) */
PTYCHO_API int ptycho_potential_to_transmission(const float* V, ptycho_c64* obj, int64_t n, double sigma,
                                                void* stream);
PTYCHO_API int ptycho_potential_grad(const ptycho_c64* obj, const ptycho_c64* grad_obj, float* grad_V, int64_t n,
                                     double sigma, void* stream);

/* Text of the last error on the calling host thread ("" if none). */
PTYCHO_API const char* ptycho_last_error(void);

/* Library version string. */
PTYCHO_API const char* ptycho_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PTYCHO_H_ */
