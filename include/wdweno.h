/*
 * wdweno.h -- C ABI of the GB300 (sm_103a) WD WENO 2x image zoom.
 *
 * The method is the two-phase "Weighted Direction" WENO interpolation of
 * B. Crnkovic, J. Skific, T. Bosner, "WENO based adaptive image zooming
 * algorithm" (arXiv 2312.00229), Sec. 3:
 *   phase 1 (Sec. 3.1, Algorithm 1) fills the "x" points of the doubled grid
 *   from four diagonal quadratic interpolants (Eq. p), weighted by
 *   neighbour-smoothed smoothness indicators (Eqs. 2Dsmoothness,
 *   2DsmoothnessFinal, alpha, IzrazOmega2d, 2dKombinacija);
 *   phase 2 (Sec. 3.2, Algorithm 2) fills the "+" points the same way along
 *   the axes, using the input samples and the phase-1 values (Eqs. tezine,
 *   IzrazOmega2dRavno, 2dKombinacijaRavno).
 * Each channel is processed independently.
 *
 * Conventions for every entry point
 *   - All data pointers are DEVICE pointers owned by the caller.  The library
 *     never allocates or frees device or host memory.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and runs asynchronously; the call returns once it is enqueued.
 *   - Sizes and strides are in ELEMENTS, not bytes; strides may be any
 *     positive values (channel, row, column), so planar [C][H][W],
 *     interleaved [H][W][C] and cropped views are all accepted.  The fastest
 *     path is a unit column stride on the output with 4-element aligned rows.
 *   - Arguments are validated on the host before anything is launched; a
 *     failed check returns a negative WENO_E* code and enqueues nothing.
 *     No device-side traps are used.
 *   - Input and output must not overlap.
 *   - The boundary rule (not given in the paper) is clamp-to-edge: the method
 *     is evaluated on the edge-replicated extension of the image and cropped.
 */
#ifndef WDWENO_H
#define WDWENO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define WENO_OK 0
#define WENO_EINVAL -1     /* null pointer, bad size, stride, shape or overlap */
#define WENO_EDTYPE -2     /* unsupported storage type combination */
#define WENO_EWORKSPACE -3 /* workspace missing or too small */
#define WENO_ECUDA -4      /* a CUDA call failed (launch or attribute query) */
#define WENO_ERANGE -5     /* a size exceeds a documented maximum */

/* Storage types.  Arithmetic is always FP32.  uint8 values are decoded as
 * v / 255 and encoded as round-half-even(saturate(u) * 255). */
typedef enum { WENO_U8 = 0, WENO_F16 = 1, WENO_BF16 = 2, WENO_F32 = 3 } weno_dtype;

/* Output grid.  WENO_OUT_2N: 2n x 2m (every coarse cell owns a 2x2 quad;
 * the last fine row/column is the scheme evaluated half a pixel past the
 * edge, the domain of Theorem 1).  WENO_OUT_2N_MINUS_1: the (2n-1) x (2m-1)
 * grid of Sec. 3, Fig. inputdata. */
typedef enum { WENO_OUT_2N = 0, WENO_OUT_2N_MINUS_1 = 1 } weno_out_mode;

/* Length scale of the smoothness indicator, Eq. (2Dsmoothness).
 * NORMALIZED: the stencil's own node spacing in both phases, i.e. the 1-D
 * indicator of Sec. 2 on each line: SI = g^2 + 13/12 s^2 with
 * g = N1 - N0, s = N0 - 2 N1 + N2.  LITERAL_SQRT2H: sqrt(2) h as printed;
 * on the axes of phase 2 this gives sqrt(2) (g^2 + 25/12 s^2). */
typedef enum { WENO_SI_NORMALIZED = 0, WENO_SI_LITERAL_SQRT2H = 1 } weno_si_scale;

typedef struct {
  float beta;      /* exponent of Eq. (alpha); default 2 (Sec. 4); >= 0 */
  float k_eps;     /* eps_h = k_eps * h^2 (Sec. 2); default 1e-8; >= 0 */
  float h;         /* coarse grid spacing; default 1 (pixel units); > 0 */
  int si_scale;    /* weno_si_scale; default WENO_SI_NORMALIZED */
  int out_mode;    /* weno_out_mode; default WENO_OUT_2N */
  int clamp_float; /* 1: saturate float outputs to [0, 1]; default 0.
                      uint8 outputs always saturate. */
  float data_bound; /* 0 (default): unknown.  Otherwise the caller guarantees
                       |input value| <= data_bound (after decoding; uint8 is
                       v / 255).  This changes no result beyond rounding: it
                       lets the library take the beta = 2 weights of Eq.
                       (alpha) as 1 / D^2 directly for any storage type, where
                       it proves that every weight stays in the FP32 range (as
                       it does from the type alone for uint8 and FP16).  A
                       bound that the data exceed can overflow the weights
                       (inf / NaN outputs).  Must be >= 0 and finite. */
  float nbr_c;     /* neighbour weight of the smoothed indicator D is
                      nbr_c * h^2 in both phases (Eqs. 2DsmoothnessFinal and
                      tezine print h^2/4; the proof of Theorem 1, Eq.
                      DDiffOrder, uses h^2/8, which reproduces the paper's
                      Table 1).  Default 0.125 (h^2/8); >= 0 and finite. */
} weno_params;

/* One image: `channels` planes of height x width. */
typedef struct {
  void* data; /* device pointer, caller-owned */
  int64_t height, width, channels;
  int64_t stride_c, stride_h, stride_w; /* element strides, all > 0 */
} weno_image;

/* Defaults: beta 2, k_eps 1e-8, h 1, normalized SI, 2n x 2m, no clamp,
 * data_bound 0 (unknown), nbr_c 0.125.  Start from these and change fields:
 * a zeroed struct is not the default. */
weno_params weno_params_default(void);

/* Human-readable text of a status code (static storage). */
const char* weno_status_string(int status);

/* Forward 2x zoom, Sec. 3 (Algorithms 1 and 2).
 *   in   : n x m x C image of type in_t (n, m, C >= 1)
 *   out  : (2n x 2m or (2n-1) x (2m-1), per p->out_mode) x C, type out_t
 *   p    : parameters (NULL = defaults)
 * Any in_t/out_t pair from weno_dtype is accepted.
 * Returns WENO_OK, WENO_EINVAL, WENO_EDTYPE or WENO_ECUDA. */
int weno_zoom2x_fwd(const weno_image* in, weno_dtype in_t, const weno_image* out,
                    weno_dtype out_t, const weno_params* p, void* stream);

/* Adjoint (vector-Jacobian product) of weno_zoom2x_fwd with respect to its
 * input, for FP32 data: grad_in = (d out / d in)^T grad_out, differentiating
 * through the nonlinear weights (Eqs. alpha, IzrazOmega2d, IzrazOmega2dRavno),
 * the neighbour-smoothed indicators (Eqs. 2DsmoothnessFinal, tezine), the
 * indicators themselves (Eq. 2Dsmoothness), the interpolants (Eq. p), the
 * phase-1 values that phase 2 reads, and the clamp-to-edge extension.
 *   x         : the forward input (FP32, n x m x C)
 *   grad_out  : FP32, shaped like the forward output for p->out_mode
 *   grad_in   : FP32, shaped like x; overwritten (not accumulated)
 *   workspace : device scratch of >= weno_zoom2x_bwd_workspace_bytes(x)
 *               bytes, 16-byte aligned; no initialisation needed; it carries
 *               the adjoints of the phase-1 values and the partial adjoint
 *               of the input samples from the phase-2 sweep to the phase-1
 *               sweep (two fused kernels, everything else stays on chip)
 * Returns WENO_OK, WENO_EINVAL, WENO_EWORKSPACE or WENO_ECUDA. */
int weno_zoom2x_bwd(const weno_image* x, const weno_image* grad_out,
                    const weno_image* grad_in, const weno_params* p, void* workspace,
                    size_t workspace_bytes, void* stream);

/* Scratch bytes weno_zoom2x_bwd needs for an input shaped like `x`
 * (2 FP32 values per cell of the image extended by 2 cells per side, per
 * channel).  Returns 0 for a malformed descriptor. */
size_t weno_zoom2x_bwd_workspace_bytes(const weno_image* x);

/* Workspace needed by weno_zoom2x_batched for `count` images (bytes). */
size_t weno_zoom2x_batched_workspace_bytes(int count);

/* Forward 2x zoom of `count` images of independent sizes in ONE persistent
 * launch fed by a device-side tile queue.
 *   d_in, d_out : DEVICE arrays of `count` weno_image descriptors (the
 *                 descriptors, not just the pixels, live on the device, so
 *                 the call can be captured into a CUDA graph and replayed)
 *   workspace   : device buffer of >= weno_zoom2x_batched_workspace_bytes
 *                 bytes; contents need no initialisation and are scratch
 *   rows_per_tile, tile_width : tile shape (0 = library default: 128-row
 *                 bands, 247-column strips); tile_width takes the values of
 *                 weno_zoom2x_fwd_tiled (247, 119, 246, 118); narrower
 *                 strips leave a smaller part of each image's last strip
 *                 idle, which pays for narrow images; the autotuner chooses
 *                 both per size class
 * Shapes follow weno_zoom2x_fwd per image; descriptors are read on the
 * device, so a malformed descriptor is skipped (its output is left
 * untouched) rather than reported.
 * Returns WENO_OK, WENO_EINVAL, WENO_EDTYPE, WENO_EWORKSPACE or WENO_ECUDA. */
int weno_zoom2x_batched(int count, const weno_image* d_in, weno_dtype in_t,
                        const weno_image* d_out, weno_dtype out_t, const weno_params* p,
                        void* workspace, size_t workspace_bytes, int rows_per_tile,
                        int tile_width, void* stream);

/* weno_zoom2x_fwd with an explicit tile shape, for the autotuner.
 *   rows_per_tile : coarse rows per CTA band, 1..4096 (0 = the default:
 *                   the band count that best balances the last wave of CTAs
 *                   on this GPU against the per-band pipeline fill)
 *   tile_width    : coarse output columns per CTA, which also fixes the
 *                   coarse columns each thread owns: 247 (256 threads of one
 *                   column, 9 columns covering the dependency halo), 119
 *                   (128 threads of one column), 246 (128 threads of two
 *                   adjacent columns, 10 halo columns), 118 (64 threads of
 *                   two), or 0 = the library's choice for the image width
 *                   (the shape that spends the fewest column-steps across
 *                   it).  Every shape gives bit-identical outputs.
 * Returns as weno_zoom2x_fwd, or WENO_EINVAL for an unsupported shape and
 * WENO_ERANGE when the band count exceeds 65535. */
int weno_zoom2x_fwd_tiled(const weno_image* in, weno_dtype in_t, const weno_image* out,
                          weno_dtype out_t, const weno_params* p, int rows_per_tile,
                          int tile_width, void* stream);

/* Number of bounded waits in the forward kernels that gave up on the current
 * device since the library was loaded or the count was last reset.  The
 * waits are those of the fused cascade (weno_zoom2x_cascade), where a tile
 * of one level waits for the tiles of the previous level it reads, with a
 * time limit of one second; a wait that runs out marks the outputs of that
 * call as invalid and lets the kernel finish instead of hanging.  Expected
 * to stay 0.  Synchronises the device.
 *   count : receives the count (host pointer)
 *   reset : nonzero resets the count to 0 after reading
 * Returns WENO_OK, WENO_EINVAL (null count) or WENO_ECUDA. */
int weno_wait_timeouts(unsigned int* count, int reset);

/* Tensor-product WENO resampling to an arbitrary size (Sec. 3.3, Eq.
 * tensor): each output sample is the 1-D WENO interpolant of Sec. 2 (Eqs.
 * TezinskiPolinom1d, IzrazOmega, with the linear weights that recover the
 * cubic, Eq. PolinomZaVelikiStencil) across the columns of four 1-D
 * interpolants down the rows.  The output grids are endpoint-aligned:
 * output row r samples input row r (n-1)/(n_out-1) (0 when n_out = 1), and
 * likewise for columns; samples outside the image are clamped to the edge.
 *   in  : n x m x C, type in_t;  out : any n_out x m_out x C, type out_t
 *   p   : beta, k_eps and h (eps_h = k_eps h^2, h = the input grid spacing;
 *         eps_h is floored at 1e-30); si_scale and out_mode are ignored;
 *         clamp_float as for the zoom
 * Output sizes down to half the input's per axis use a separable tiled
 * kernel; larger reductions fall back to one thread per output sample.
 * Values are expected below ~1e18 in magnitude (squared differences must
 * stay finite in FP32).
 * The second stage of the arbitrary-scale zoom: k doublings on the
 * (2n-1) grid (Eq. zoomfactor) followed by this resampling.
 * Returns WENO_OK, WENO_EINVAL, WENO_EDTYPE, WENO_ERANGE (more than 524280
 * output rows) or WENO_ECUDA. */
int weno_resample(const weno_image* in, weno_dtype in_t, const weno_image* out,
                  weno_dtype out_t, const weno_params* p, void* stream);

/* 2^levels zoom by `levels` successive 2x zooms (Sec. 3.3, Eq. zoomfactor)
 * in ONE persistent launch (plus a small setup kernel).  Level L zooms the
 * image of level L-1 with h = p->h / 2^L (its coarse grid is the previous
 * level's fine grid) and p->out_mode at every level; the intermediate images
 * are FP32 planes in the workspace, and only the last level encodes to out_t.
 * The result equals `levels` weno_zoom2x_fwd calls with FP32 intermediates.
 * The input type's bound (uint8, FP16) or p->data_bound is carried to the
 * later levels at 1.5625x per level, as weno_params.data_bound describes.
 *   in, in_t   : n x m x C image
 *   out, out_t : the last level's image: 2^L n x 2^L m in WENO_OUT_2N mode,
 *                (2^L (n-1) + 1) x (2^L (m-1) + 1) in WENO_OUT_2N_MINUS_1
 *   levels     : 1 .. WENO_CASCADE_MAX_LEVELS
 *   workspace  : device scratch of >= weno_zoom2x_cascade_workspace_bytes
 *                bytes, 256-byte aligned, overlapping neither image; no
 *                initialisation needed; calls that share it must not overlap
 * A tile of a later level waits (bounded, one second) for the bands of the
 * previous level it reads; a wait that gives up is counted by
 * weno_wait_timeouts.
 * Returns WENO_OK, WENO_EINVAL (shapes, overlap, levels, parameters),
 * WENO_EDTYPE, WENO_EWORKSPACE, WENO_ERANGE (more than 65535 bands in a
 * level) or WENO_ECUDA. */
#define WENO_CASCADE_MAX_LEVELS 6
int weno_zoom2x_cascade(const weno_image* in, weno_dtype in_t, const weno_image* out,
                        weno_dtype out_t, int levels, const weno_params* p, void* workspace,
                        size_t workspace_bytes, void* stream);

/* Scratch bytes of weno_zoom2x_cascade for `in`, `levels` and p's out_mode
 * on the current device (the band heights follow its SM count); 0 for a
 * malformed request. */
size_t weno_zoom2x_cascade_workspace_bytes(const weno_image* in, int levels,
                                           const weno_params* p);

/* weno_zoom2x_batched without a workspace, for callers that cannot allocate
 * device memory (for example code inside another application's real-time
 * video pipeline, where cudaMalloc may synchronise the device and stall every
 * other stream, or a plugin that is given image pointers but no allocator).
 * The paper has no counterpart: this is a deployment variant of the batched
 * call, with the same arguments minus the workspace.
 *   - The tile queue lives in a fixed array inside the library's own device
 *     memory (WENO_NOALLOC_SCRATCH_BYTES bytes, held on every GPU that loads
 *     the library until the process exits); at most WENO_NOALLOC_MAX_IMAGES
 *     images per call, larger counts return WENO_ERANGE.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (that device must be current); make that first
 *     call before any stream capture.  The address is kept for the life of
 *     the process: after cudaDeviceReset on that device it is stale, so do
 *     not call this entry point again in a process that reset the device.
 *   - The call allocates nothing (no cudaMalloc, cudaFree or allocating
 *     library routine).  Every call shares the one array and resets what it
 *     uses, so calls that overlap on the GPU (e.g. on two streams at once)
 *     race and must be serialised by the caller.
 * Returns as weno_zoom2x_batched, plus WENO_ERANGE. */
#define WENO_NOALLOC_MAX_IMAGES 4096
#define WENO_NOALLOC_SCRATCH_BYTES 32800
int weno_zoom2x_batched_noalloc(int count, const weno_image* d_in, weno_dtype in_t,
                                const weno_image* d_out, weno_dtype out_t, const weno_params* p,
                                int rows_per_tile, int tile_width, void* stream);

/* Calibration of the FP32 pipe (measurement support, not part of the
 * method): launches `blocks` CTAs of 256 threads, each thread running
 * `iters` x 128 FP32 fused multiply-adds in 16 independent chains, and
 * writes one float per thread to `out` (device buffer of >= blocks x 256
 * floats, caller-owned).  Timing the launch on `stream` gives the measured
 * FP32 operation rate beside the nominal one (SMs x 128 lanes x clock).
 * Returns WENO_OK, WENO_EINVAL (blocks or iters outside 1 .. 2^23, null
 * out) or WENO_ECUDA. */
int weno_fp32_probe(int blocks, int iters, float* out, void* stream);

/* FP32 operations (one per fused multiply-add) one weno_fp32_probe launch
 * performs; -1 for arguments weno_fp32_probe rejects. */
long long weno_fp32_probe_ops(int blocks, int iters);

#ifdef __cplusplus
}
#endif

#endif /* WDWENO_H */
