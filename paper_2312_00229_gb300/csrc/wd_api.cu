// C ABI of the WD WENO library (declarations and contracts: include/wdweno.h).
// Host-side argument validation, folding of the method's constants, and
// kernel dispatch.  Nothing here allocates memory.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "wd_bwd.h"
#include "wd_batched.h"
#include "wd_cascade.h"
#include "wd_common.cuh"
#include "wd_fwd.h"
#include "wd_resample.h"
#include "wdweno.h"

using namespace wdweno;

namespace {

constexpr int64_t kDefaultRowsPerBand = 64;
// Persistent batched launches: 128-row bands measured best on 256 FP16 images
// of sides 64..1024 (77.2 Gpix/s at 64 rows, 78.7 at 128, 76.7 at 192); the
// queue still holds some 10,000 tiles for 304 CTA slots.
constexpr int64_t kBatchedRowsPerBand = 128;
constexpr int kFwdCtasPerSm = 2;  // 256-thread CTAs x 128 registers (twice as many at 128)

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!cached[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      cached[dev] = v;
  }
  return cached[dev];
}

// CTA shape for a requested tile width (output columns per CTA): 247 -> 256
// threads of one column, 119 -> 128 threads of one column, 246 -> 128
// threads of two columns, 118 -> 64 threads of two columns; false for any
// other width.
bool shape_for_width(int tile_width, int* threads, int* cols) {
  *cols = 1;
  if (tile_width == tile_width_fwd()) { *threads = threads_fwd(); return true; }
  if (tile_width == tile_width_fwd() - (threads_fwd() - 128)) { *threads = 128; return true; }
  *cols = 2;
  if (tile_width == 2 * 128 - 10) { *threads = 128; return true; }
  if (tile_width == 2 * 64 - 10) { *threads = 64; return true; }
  return false;
}

// Band height for a one-launch forward: choose the number of bands B that
// minimises (waves of CTAs) x (rows per band + pipeline fill), i.e. balance
// the tail of the last wave against the fixed per-band cost.  `cols` coarse
// columns per thread: one-column CTAs of 256 (128) threads keep 2 (4)
// resident per SM, two-column CTAs of 128 (64) threads 3 (6).
int64_t default_rows_per_band(int64_t n, int64_t m, int64_t planes, int threads, int cols = 1) {
  const int sms = sm_count();
  if (sms <= 0) return kDefaultRowsPerBand;
  const int64_t per_sm = cols == 2 ? 3 * 128 / threads : kFwdCtasPerSm * (threads_fwd() / threads);
  const int64_t slots = (int64_t)sms * per_sm;
  const int64_t tw = cols == 2 ? 2 * threads - 10 : threads - 9;
  const int64_t strips = (m + tw - 1) / tw;
  const int64_t base = strips * planes;
  const int64_t fill = 7;  // extra steps per band: 4 + 5 halo rows + 2 pipeline steps
  int64_t best_rpb = n, best_cost = -1;
  for (int64_t bands = 1; bands <= 4096; ++bands) {
    const int64_t rpb = (n + bands - 1) / bands;
    if (rpb < 16 && bands > 1) break;
    if (bands > 1 && (n + rpb - 1) / rpb != bands) continue;  // same rpb as a smaller count
    const int64_t waves = (base * bands + slots - 1) / slots;
    const int64_t cost = waves * (rpb + fill);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best_rpb = rpb;
    }
  }
  return best_rpb < 1 ? 1 : best_rpb;
}

int64_t dtype_size(int dt) {
  switch (dt) {
    case WENO_U8: return 1;
    case WENO_F16: return 2;
    case WENO_BF16: return 2;
    case WENO_F32: return 4;
    default: return 0;
  }
}

bool image_ok(const weno_image* im) {
  return im && im->data && im->height >= 1 && im->width >= 1 && im->channels >= 1 &&
         im->stride_c >= 1 && im->stride_h >= 1 && im->stride_w >= 1 &&
         im->height < (int64_t(1) << 31) && im->width < (int64_t(1) << 31) &&
         im->channels < 65536;
}

// Byte range [lo, hi) touched by an image view.
void byte_extent(const weno_image* im, int64_t esz, uintptr_t* lo, uintptr_t* hi) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(im->data);
  const int64_t last = (im->channels - 1) * im->stride_c + (im->height - 1) * im->stride_h +
                       (im->width - 1) * im->stride_w;
  *lo = base;
  *hi = base + static_cast<uintptr_t>((last + 1) * esz);
}

bool overlaps(const weno_image* a, int64_t ea, const weno_image* b, int64_t eb) {
  uintptr_t alo, ahi, blo, bhi;
  byte_extent(a, ea, &alo, &ahi);
  byte_extent(b, eb, &blo, &bhi);
  return alo < bhi && blo < ahi;
}

// Fold Eq. (alpha)'s eps_h and the neighbour weight of Eqs.
// (2DsmoothnessFinal)/(tezine) into per-SI constants (see MethodConsts).
bool fold_consts(const weno_params& p, MethodConsts* k, int* bmode) {
  if (!(p.beta >= 0.f) || !(p.k_eps >= 0.f) || !(p.h > 0.f) || !std::isfinite(p.beta) ||
      !std::isfinite(p.k_eps) || !std::isfinite(p.h) || !(p.data_bound >= 0.f) ||
      !std::isfinite(p.data_bound) || !(p.nbr_c >= 0.f) || !std::isfinite(p.nbr_c))
    return false;
  if (p.si_scale != WENO_SI_NORMALIZED && p.si_scale != WENO_SI_LITERAL_SQRT2H) return false;
  const double h = p.h;
  const double w = double(p.nbr_c) * h * h;
  const double eps_h = double(p.k_eps) * h * h;
  const double spread = 1.0 + 4.0 * w;
  k->w = float(w);
  k->kappa1 = float(std::sqrt(13.0 / 12.0));
  k->eps1 = float(eps_h / spread);
  if (p.si_scale == WENO_SI_NORMALIZED) {
    k->kappa2 = float(std::sqrt(13.0 / 12.0));
    k->eps2 = float(eps_h / spread);
  } else {
    // sqrt(2) (g^2 + 25/12 s^2): the common sqrt(2) cancels in the weights
    // once eps_h is divided by it.
    k->kappa2 = float(std::sqrt(25.0 / 12.0));
    k->eps2 = float(eps_h / (std::sqrt(2.0) * spread));
  }
  k->beta = p.beta;
  k->clamp_float = p.clamp_float ? 1 : 0;
  if (p.beta == 0.f) {
    *bmode = B0;
  } else if (p.beta == 2.f) {
    *bmode = B2;
  } else {
    *bmode = BGEN;
  }
  return true;
}

// Whether the forward kernels may take the beta = 2 weights of Eq. (alpha)
// as 1 / D^2 directly (B2R) instead of the scale-free (D_min / D)^2.  That
// needs every D inside [lo, hi] with 1/hi^2 and 1/lo^2 normal FP32 numbers,
// and the weight sum and the blend numerator finite.  The storage type
// bounds the data (uint8 decodes to [0, 1]; FP16 <= 65504), or the caller
// does through weno_params::data_bound: |input| <= v0.
// Every node of an interpolant is an input or a phase-1 value, a convex
// combination of quadratic interpolants (|p| <= 1.25 max |node|), so
// |node| <= v = 1.25 v0; then |g| <= 2v, |s| <= 4v and
//   SI <= 4 v^2 + (25/12) 16 v^2 + eps_h,  D <= (1 + 4w) SI_max,
//   D >= eps_h / sqrt(2) (phase 2 of the literal SI scaling; eps_h otherwise).
// The weights are at most 1/lo^2 each, the numerator at most 16 v times their
// largest value.  BFloat16 and FP32 data without a caller's bound keep B2.
// Bound on |input| from the storage type (uint8, FP16) or from the caller's
// weno_params::data_bound, the smaller when both hold; 0 when neither does.
double input_bound(const weno_params& p, int in_t) {
  double v0 = in_t == WENO_U8 ? 1.0 : (in_t == WENO_F16 ? 65504.0 : 0.0);
  if (p.data_bound > 0.f && (v0 == 0.0 || double(p.data_bound) < v0)) v0 = p.data_bound;
  return v0;
}

bool direct_b2_ok(const weno_params& p, int in_t) {
  const double v0 = input_bound(p, in_t);
  if (!(v0 > 0.0)) return false;
  const double h = p.h, w = double(p.nbr_c) * h * h, eps_h = double(p.k_eps) * h * h;
  const double v = 1.25 * v0 * (1.0 + 1e-3);  // slack for the approximate reciprocals
  const double si_max = 4.0 * v * v + 25.0 / 12.0 * 16.0 * v * v + eps_h;
  const double hi = (1.0 + 4.0 * w) * si_max;
  const double lo = eps_h / 2.0;
  if (!(lo >= 1e-18) || !(hi <= 1e18)) return false;
  const double a_max = 1.0 / (lo * lo);
  return 8.0 * a_max <= 1e37 && 16.0 * v * a_max <= 1e37;
}

// The same choice for the 1-D WENO weights of the tensor resampling: with
// indicators e = g^2 + 13/12 s^2 + eps, alpha_0 : alpha_1 = C_0 eR^2 : C_1 eL^2
// as written needs eps^2 normal and (e_max)^2 times the largest |s| finite.
// The nodes are inputs or first-pass values, quadratic interpolants on
// [0, 1] of inputs (|p| <= 1.25 max|node|).
bool resample_direct_ok(const weno_params& p, int in_t, double eps) {
  const double v0 = input_bound(p, in_t);
  if (!(v0 > 0.0)) return false;
  const double v = 1.25 * v0 * (1.0 + 1e-3);
  const double e_hi = 4.0 * v * v + 13.0 / 12.0 * 16.0 * v * v + eps;
  return eps >= 1e-18 && e_hi <= 1e18 && e_hi * e_hi * 4.0 * v <= 1e37;
}

int check_pair(const weno_image* in, int in_t, const weno_image* out, int out_t,
               const weno_params& p, int64_t* orows, int64_t* ocols) {
  if (!image_ok(in) || !image_ok(out)) return WENO_EINVAL;
  if (dtype_size(in_t) == 0 || dtype_size(out_t) == 0) return WENO_EDTYPE;
  if (p.out_mode != WENO_OUT_2N && p.out_mode != WENO_OUT_2N_MINUS_1) return WENO_EINVAL;
  const bool m1 = p.out_mode == WENO_OUT_2N_MINUS_1;
  *orows = 2 * in->height - (m1 ? 1 : 0);
  *ocols = 2 * in->width - (m1 ? 1 : 0);
  if (out->height != *orows || out->width != *ocols || out->channels != in->channels)
    return WENO_EINVAL;
  if (overlaps(in, dtype_size(in_t), out, dtype_size(out_t))) return WENO_EINVAL;
  return WENO_OK;
}

FwdArgs make_fwd_args(const weno_image* in, int in_t, const weno_image* out, int out_t,
                      int64_t orows, int64_t ocols, int64_t rows_per_band) {
  FwdArgs a;
  a.threads = threads_fwd();
  a.in = in->data;
  a.out = out->data;
  a.in_dtype = in_t;
  a.out_dtype = out_t;
  a.n = in->height;
  a.m = in->width;
  a.planes = in->channels;
  a.in_sc = in->stride_c;
  a.in_sh = in->stride_h;
  a.in_sw = in->stride_w;
  a.out_sc = out->stride_c;
  a.out_sh = out->stride_h;
  a.out_sw = out->stride_w;
  a.orows = orows;
  a.ocols = ocols;
  a.rows_per_band = rows_per_band;
  const int64_t esz = dtype_size(out_t);
  const uintptr_t base = reinterpret_cast<uintptr_t>(out->data);
  a.out_vec = (out->stride_w == 1) && (out->stride_h % 2 == 0) && (out->stride_c % 2 == 0) &&
              (base % uintptr_t(2 * esz) == 0);
  a.out_vec4 = (out->stride_w == 1) && (out->stride_h % 4 == 0) && (out->stride_c % 4 == 0) &&
               (base % uintptr_t(4 * esz) == 0);
  a.cols = 1;
  return a;
}

// Fused 2^k cascade (Sec. 3.3, Eq. zoomfactor).
static_assert(CASCADE_MAX_LEVELS == WENO_CASCADE_MAX_LEVELS, "cascade level limit");
// Shapes, band heights and workspace layout of a cascade; false when the
// request is malformed.  Level L zooms image L (image 0 = the input, image
// `levels` = the output); images 1 .. levels-1 are FP32 planes in the
// workspace, then come the queue head and the finished-strip counters.
struct CascadePlan {
  int levels;
  int64_t n[CASCADE_MAX_LEVELS + 1], m[CASCADE_MAX_LEVELS + 1];
  int64_t rpb[CASCADE_MAX_LEVELS];
  size_t img_off[CASCADE_MAX_LEVELS + 1];  // byte offset of FP32 image L (1 .. levels-1)
  size_t head_off, done_off, bytes;
  int64_t done_count;
};

bool cascade_plan(const weno_image* in, int levels, const weno_params& p, CascadePlan* c) {
  if (!image_ok(in) || levels < 1 || levels > CASCADE_MAX_LEVELS) return false;
  if (p.out_mode != WENO_OUT_2N && p.out_mode != WENO_OUT_2N_MINUS_1) return false;
  const int64_t d = p.out_mode == WENO_OUT_2N_MINUS_1 ? 1 : 0;
  c->levels = levels;
  c->n[0] = in->height;
  c->m[0] = in->width;
  size_t off = 0;
  for (int L = 0; L < levels; ++L) {
    c->n[L + 1] = 2 * c->n[L] - d;
    c->m[L + 1] = 2 * c->m[L] - d;
    if (c->n[L + 1] < 1 || c->m[L + 1] < 1 || c->n[L + 1] >= (int64_t(1) << 31) ||
        c->m[L + 1] >= (int64_t(1) << 31))
      return false;
    c->rpb[L] = default_rows_per_band(c->n[L], c->m[L], in->channels, CASCADE_THREADS);
  }
  c->done_count = 0;
  for (int L = 0; L < levels; ++L) {
    c->img_off[L + 1] = off;
    if (L + 1 < levels)
      off += ((size_t)(c->n[L + 1] * c->m[L + 1] * in->channels) * 4 + 255) & ~size_t(255);
    c->done_count += ((c->n[L] + c->rpb[L] - 1) / c->rpb[L]) * in->channels;
  }
  c->head_off = off;
  c->done_off = off + 16;
  c->bytes = (c->done_off + 4 * (size_t)c->done_count + 255) & ~size_t(255);
  return true;
}

}  // namespace

extern "C" {

weno_params weno_params_default(void) {
  weno_params p;
  p.beta = 2.0f;
  p.k_eps = 1e-8f;
  p.h = 1.0f;
  p.si_scale = WENO_SI_NORMALIZED;
  p.out_mode = WENO_OUT_2N;
  p.clamp_float = 0;
  p.data_bound = 0.f;
  p.nbr_c = 0.125f;
  return p;
}

const char* weno_status_string(int status) {
  switch (status) {
    case WENO_OK: return "ok";
    case WENO_EINVAL: return "invalid argument (pointer, size, stride, shape or overlap)";
    case WENO_EDTYPE: return "unsupported storage type";
    case WENO_EWORKSPACE: return "workspace missing or too small";
    case WENO_ECUDA: return "CUDA launch or runtime error";
    case WENO_ERANGE: return "size exceeds the documented maximum";
    default: return "unknown status";
  }
}

int weno_zoom2x_fwd_tiled(const weno_image* in, weno_dtype in_t, const weno_image* out,
                          weno_dtype out_t, const weno_params* pp, int rows_per_tile,
                          int tile_width, void* stream) {
  const weno_params p = pp ? *pp : weno_params_default();
  int64_t orows, ocols;
  int rc = check_pair(in, in_t, out, out_t, p, &orows, &ocols);
  if (rc != WENO_OK) return rc;
  if (rows_per_tile < 0 || rows_per_tile > 4096) return WENO_EINVAL;
  int threads = 0, cols = 1;
  if (tile_width == 0) {
    fwd_shape_for(in->width, &threads, &cols);
  } else if (!shape_for_width(tile_width, &threads, &cols)) {
    return WENO_EINVAL;
  }
  MethodConsts k;
  int bmode;
  if (!fold_consts(p, &k, &bmode)) return WENO_EINVAL;
  const int64_t rpb = rows_per_tile > 0 ? rows_per_tile
                                        : default_rows_per_band(in->height, in->width,
                                                                in->channels, threads, cols);
  if (bmode == B2 && direct_b2_ok(p, in_t)) bmode = B2R;
  FwdArgs a = make_fwd_args(in, in_t, out, out_t, orows, ocols, rpb);
  a.threads = threads;
  a.cols = cols;
  if ((a.n + rpb - 1) / rpb > 65535) return WENO_ERANGE;
  cudaError_t e = launch_zoom2x_fwd(a, k, bmode, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? WENO_OK : WENO_ECUDA;
}

int weno_zoom2x_fwd(const weno_image* in, weno_dtype in_t, const weno_image* out,
                    weno_dtype out_t, const weno_params* p, void* stream) {
  return weno_zoom2x_fwd_tiled(in, in_t, out, out_t, p, 0, 0, stream);
}

size_t weno_zoom2x_bwd_workspace_bytes(const weno_image* x) {
  if (!x || x->height < 1 || x->width < 1 || x->channels < 1) return 0;
  return bwd_workspace_bytes(x->height, x->width, x->channels);
}

int weno_zoom2x_bwd(const weno_image* x, const weno_image* grad_out, const weno_image* grad_in,
                    const weno_params* pp, void* workspace, size_t workspace_bytes,
                    void* stream) {
  const weno_params p = pp ? *pp : weno_params_default();
  int64_t orows, ocols;
  int rc = check_pair(x, WENO_F32, grad_out, WENO_F32, p, &orows, &ocols);
  if (rc != WENO_OK) return rc;
  if (!image_ok(grad_in) || grad_in->height != x->height || grad_in->width != x->width ||
      grad_in->channels != x->channels)
    return WENO_EINVAL;
  if (overlaps(grad_in, 4, x, 4) || overlaps(grad_in, 4, grad_out, 4)) return WENO_EINVAL;
  if (!workspace || workspace_bytes < bwd_workspace_bytes(x->height, x->width, x->channels) ||
      reinterpret_cast<uintptr_t>(workspace) % 16 != 0)
    return WENO_EWORKSPACE;
  // (image_ok bounds the output's sides below 2^31, so the kernels' 32-bit
  // rows and columns and the one grid layer of CTAs per channel fit)
  MethodConsts k;
  int bmode;
  if (!fold_consts(p, &k, &bmode)) return WENO_EINVAL;
  BwdArgs a;
  a.x = static_cast<const float*>(x->data);
  a.gout = static_cast<const float*>(grad_out->data);
  a.gin = static_cast<float*>(grad_in->data);
  a.n = x->height;
  a.m = x->width;
  a.planes = x->channels;
  a.x_sc = x->stride_c; a.x_sh = x->stride_h; a.x_sw = x->stride_w;
  a.g_sc = grad_out->stride_c; a.g_sh = grad_out->stride_h; a.g_sw = grad_out->stride_w;
  a.gi_sc = grad_in->stride_c; a.gi_sh = grad_in->stride_h; a.gi_sw = grad_in->stride_w;
  a.orows = orows;
  a.ocols = ocols;
  a.ws = static_cast<float*>(workspace);
  cudaError_t e = launch_zoom2x_bwd(a, k, bmode, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? WENO_OK : WENO_ECUDA;
}

size_t weno_zoom2x_batched_workspace_bytes(int count) {
  if (count < 0) return 0;
  return batched_workspace_bytes(count);
}

int weno_zoom2x_batched(int count, const weno_image* d_in, weno_dtype in_t,
                        const weno_image* d_out, weno_dtype out_t, const weno_params* pp,
                        void* workspace, size_t workspace_bytes, int rows_per_tile,
                        int tile_width, void* stream) {
  const weno_params p = pp ? *pp : weno_params_default();
  if (count < 0 || count > (1 << 24)) return WENO_EINVAL;
  if (count == 0) return WENO_OK;
  if (!d_in || !d_out) return WENO_EINVAL;
  if (dtype_size(in_t) == 0 || dtype_size(out_t) == 0) return WENO_EDTYPE;
  if (p.out_mode != WENO_OUT_2N && p.out_mode != WENO_OUT_2N_MINUS_1) return WENO_EINVAL;
  if (!workspace || workspace_bytes < batched_workspace_bytes(count)) return WENO_EWORKSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % 16 != 0) return WENO_EWORKSPACE;
  if (rows_per_tile < 0 || rows_per_tile > 4096) return WENO_EINVAL;
  int threads = threads_fwd(), cols = 1;
  if (tile_width != 0 && !shape_for_width(tile_width, &threads, &cols)) return WENO_EINVAL;
  MethodConsts k;
  int bmode;
  if (!fold_consts(p, &k, &bmode)) return WENO_EINVAL;
  if (bmode == B2 && direct_b2_ok(p, in_t)) bmode = B2R;
  BatchedArgs a;
  a.threads = threads;
  a.cols = cols;
  a.count = count;
  a.in = d_in;
  a.out = d_out;
  a.in_dtype = in_t;
  a.out_dtype = out_t;
  a.out_mode = p.out_mode;
  a.rows_per_band = rows_per_tile > 0 ? rows_per_tile : kBatchedRowsPerBand;
  a.workspace = workspace;
  cudaError_t e = launch_zoom2x_batched(a, k, bmode, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? WENO_OK : WENO_ECUDA;
}

size_t weno_zoom2x_cascade_workspace_bytes(const weno_image* in, int levels,
                                           const weno_params* pp) {
  const weno_params p = pp ? *pp : weno_params_default();
  CascadePlan c;
  return cascade_plan(in, levels, p, &c) ? c.bytes : 0;
}

int weno_zoom2x_cascade(const weno_image* in, weno_dtype in_t, const weno_image* out,
                        weno_dtype out_t, int levels, const weno_params* pp, void* workspace,
                        size_t workspace_bytes, void* stream) {
  const weno_params p = pp ? *pp : weno_params_default();
  if (!image_ok(in) || !image_ok(out)) return WENO_EINVAL;
  if (dtype_size(in_t) == 0 || dtype_size(out_t) == 0) return WENO_EDTYPE;
  CascadePlan c;
  if (!cascade_plan(in, levels, p, &c)) return WENO_EINVAL;
  if (out->height != c.n[levels] || out->width != c.m[levels] || out->channels != in->channels)
    return WENO_EINVAL;
  if (overlaps(in, dtype_size(in_t), out, dtype_size(out_t))) return WENO_EINVAL;
  if (!workspace || workspace_bytes < c.bytes || reinterpret_cast<uintptr_t>(workspace) % 256)
    return WENO_EWORKSPACE;
  {  // the workspace overlaps neither image
    weno_image w{workspace, 1, (int64_t)c.bytes, 1, (int64_t)c.bytes, (int64_t)c.bytes, 1};
    if (overlaps(&w, 1, in, dtype_size(in_t)) || overlaps(&w, 1, out, dtype_size(out_t)))
      return WENO_EINVAL;
  }
  for (int L = 0; L < levels; ++L)
    if ((c.n[L] + c.rpb[L] - 1) / c.rpb[L] > 65535) return WENO_ERANGE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  CascadeArgs a;
  std::memset(&a, 0, sizeof(a));
  a.levels = levels;
  // one weight form for every level: the direct one when the input's bound,
  // carried at 1.5625x (x values are convex combinations of interpolants with
  // |p| <= 1.25 max|node|, "+" values take x values as nodes) with slack for
  // the weights' rounding, proves the range at every level
  int bmode = B2;
  bool all_direct = true;
  double bound = input_bound(p, in_t);
  int64_t first = 0, done = 0;
  for (int L = 0; L < levels; ++L) {
    weno_params pl = p;
    pl.h = float(double(p.h) / double(int64_t(1) << L));
    pl.data_bound = float(bound);
    int bm;
    if (!fold_consts(pl, &a.k[L], &bm)) return WENO_EINVAL;
    bmode = bm;
    if (!(bound > 0.0) || !direct_b2_ok(pl, L == 0 ? int(in_t) : int(WENO_F32)))
      all_direct = false;
    bound *= 1.5625 * (1.0 + 1e-3);
    weno_image src = *in, dst = *out;
    if (L > 0) {
      src = weno_image{ws + c.img_off[L], c.n[L], c.m[L], in->channels, c.n[L] * c.m[L], c.m[L], 1};
    }
    if (L + 1 < levels) {
      dst = weno_image{ws + c.img_off[L + 1], c.n[L + 1], c.m[L + 1], in->channels,
                       c.n[L + 1] * c.m[L + 1], c.m[L + 1], 1};
    }
    const int st = L == 0 ? int(in_t) : int(WENO_F32);
    const int dt = L + 1 == levels ? int(out_t) : int(WENO_F32);
    a.f[L] = make_fwd_args(&src, st, &dst, dt, c.n[L + 1], c.m[L + 1], c.rpb[L]);
    a.strips[L] = (c.m[L] + CASCADE_THREADS - 9 - 1) / (CASCADE_THREADS - 9);
    a.bands[L] = (c.n[L] + c.rpb[L] - 1) / c.rpb[L];
    a.first[L] = first;
    first += a.strips[L] * a.bands[L] * in->channels;
    a.done_off[L] = done;
    done += a.bands[L] * in->channels;
  }
  a.first[levels] = first;
  if (bmode == B2 && all_direct) bmode = B2R;
  a.head = reinterpret_cast<unsigned long long*>(ws + c.head_off);
  a.done = reinterpret_cast<unsigned int*>(ws + c.done_off);
  a.done_count = c.done_count;
  cudaError_t e = launch_zoom2x_cascade(a, bmode, in_t, out_t, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? WENO_OK : WENO_ECUDA;
}

int weno_wait_timeouts(unsigned int* count, int reset) {
  if (!count) return WENO_EINVAL;
  return fwd_wait_timeouts(count, reset != 0) == cudaSuccess ? WENO_OK : WENO_ECUDA;
}

int weno_resample(const weno_image* in, weno_dtype in_t, const weno_image* out,
                  weno_dtype out_t, const weno_params* pp, void* stream) {
  const weno_params p = pp ? *pp : weno_params_default();
  if (!image_ok(in) || !image_ok(out)) return WENO_EINVAL;
  if (dtype_size(in_t) == 0 || dtype_size(out_t) == 0) return WENO_EDTYPE;
  if (out->channels != in->channels) return WENO_EINVAL;
  if (overlaps(in, dtype_size(in_t), out, dtype_size(out_t))) return WENO_EINVAL;
  if ((out->height + 7) / 8 > 65535) return WENO_ERANGE;
  MethodConsts k;
  int bmode;
  if (!fold_consts(p, &k, &bmode)) return WENO_EINVAL;
  ResampleArgs a;
  a.in = in->data;
  a.out = out->data;
  a.in_dtype = in_t;
  a.out_dtype = out_t;
  a.n = in->height; a.m = in->width; a.planes = in->channels;
  a.n_out = out->height; a.m_out = out->width;
  a.in_sc = in->stride_c; a.in_sh = in->stride_h; a.in_sw = in->stride_w;
  a.out_sc = out->stride_c; a.out_sh = out->stride_h; a.out_sw = out->stride_w;
  a.clamp_float = p.clamp_float ? 1 : 0;
  a.out_vec4 = out->stride_w == 1 && out->stride_h % 4 == 0 && out->stride_c % 4 == 0 &&
               reinterpret_cast<uintptr_t>(out->data) % uintptr_t(4 * dtype_size(out_t)) == 0;
  a.win_rows = 0;
  // a floor of 1e-30 keeps the larger indicator a normal FP32 number
  const float eps = std::max(float(double(p.k_eps) * double(p.h) * double(p.h)), 1e-30f);
  if (bmode == B2 && resample_direct_ok(p, in_t, eps)) bmode = B2R;
  cudaError_t e = launch_resample(a, eps, p.beta, bmode, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? WENO_OK : WENO_ECUDA;
}

}  // extern "C"
