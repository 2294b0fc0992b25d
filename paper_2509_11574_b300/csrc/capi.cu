// extern "C" entry points of libgps: argument checks, workspace layout and
// the order of kernel launches.  No call synchronises the stream except
// gps_query_status.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>

#include "gps_common.cuh"

namespace gps {
cudaError_t launch_fuse(const GpsTsdf&, const float*, const float*, const Cam&, cudaStream_t);
cudaError_t launch_mark_bricks(const GpsTsdf&, cudaStream_t);
cudaError_t launch_raycast(const GpsTsdf&, const Cam&, float, float, void*, int, float*, float*,
                           cudaStream_t);
cudaError_t launch_project(const GpsGaussians&, float, const ViewBatch&, int, cudaStream_t);
cudaError_t launch_project_backward(const GpsGaussians&, float, const ViewBatch&,
                                    const GpsGaussians&, bool, const float*, cudaStream_t);
cudaError_t launch_bin_histogram(int, const ViewBatch&, int, cudaStream_t);
cudaError_t launch_scan_super(const ViewBatch&, int*, cudaStream_t);
cudaError_t launch_emit_super(int, const ViewBatch&, int, cudaStream_t);
cudaError_t launch_block_prefix(int, const ViewBatch&, int, cudaStream_t);
cudaError_t launch_sort_split(const ViewBatch&, int, int, int, cudaStream_t);
cudaError_t launch_composite_fwd(const ViewBatch&, int, int, float, int, int, int, int, cudaStream_t);
cudaError_t launch_composite_bwd_per_gaussian(const ViewBatch&, int, float, float, const float*,
                                              int, cudaStream_t);
cudaError_t launch_composite_bwd(const ViewBatch&, int, int, float, float, const float*, int, int,
                                 int, int, cudaStream_t);
cudaError_t launch_finalize_loss(const ViewBatch&, float, float*, int, cudaStream_t);
cudaError_t launch_gather_pair_grads(const ViewBatch&, int, cudaStream_t);
cudaError_t launch_upstream_max(const ViewBatch&, float, float, const float*, cudaStream_t);
cudaError_t launch_fixed_to_grad2d(const ViewBatch&, int, const float*, cudaStream_t);
cudaError_t launch_pair_base(const ViewBatch&, int, const int*, cudaStream_t);
cudaError_t launch_adam(const GpsGaussians&, const GpsGaussians&, const GpsGaussians&,
                        const GpsGaussians&, const GpsAdamHyper&, int, int*, cudaStream_t);
cudaError_t launch_project_backward_adam(const GpsGaussians&, float, const ViewBatch&,
                                         const GpsGaussians&, const GpsGaussians&,
                                         const GpsAdamHyper&, int, int*, bool, const float*,
                                         cudaStream_t);
}  // namespace gps

using namespace gps;

namespace {

thread_local std::string g_err;

int32_t fail(int32_t code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int32_t fail(int32_t code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int32_t cuda_fail(cudaError_t e, const char* where) {
  return fail(GPS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

struct TileCfg {
  int tw, th;
};

bool tile_cfg(const GpsRenderSettings* s, TileCfg& c) {
  c.tw = s->tile_w;
  c.th = s->tile_h;
  if (c.tw == 0 && c.th == 0) {  // the default: fastest on the 640x480 room workload
    c.tw = 16;
    c.th = 8;
  }
  return (c.tw == 16 && c.th == 16) || (c.tw == 16 && c.th == 8) || (c.tw == 8 && c.th == 8) ||
         (c.tw == 32 && c.th == 8);
}

long long pair_cap(const GpsRenderSettings* s, int M) {
  return s->pair_capacity > 0 ? s->pair_capacity : 16LL * (M > 0 ? M : 1);
}

constexpr int kSuperMax = 16384;  // the bin histogram lives in shared memory
// fixed-order emission: 8 warps' 16-bit offsets per bin beside the bin bases
// in shared memory (20 B per bin: 120 KB at this size)
constexpr int kFixedBinsMax = 6144;

long long view_tiles(const GpsView& vw, const TileCfg& tc) {
  return (long long)((vw.K.width + tc.tw - 1) / tc.tw) * ((vw.K.height + tc.th - 1) / tc.th);
}

// The binning of each view is decided from the settings and that view's
// own tile grid alone, so that a view renders bit for bit the same whether
// it is batched with other views or not.
//
// Deterministic mode with the order-independent blend needs one fixed list
// order, not a depth sort: a view's lists go straight into its tile bins in
// ascending Gaussian index, their places computed from counts (block bases
// by a prefix over the binning blocks, warp offsets inside a block), where
// its tile grid fits the emission's shared memory.
bool view_fixed_order(const GpsView& vw, const GpsRenderSettings& s, const TileCfg& tc) {
  return s.deterministic && s.blend_mode == GPS_BLEND_OIT && s.schedule == GPS_SCHEDULE_TILES &&
         view_tiles(vw, tc) <= kFixedBinsMax;
}

// Are a view's tile lists sorted by (depth, index)?  The "with sort" blend
// needs front-to-back order, and deterministic mode needs one fixed order for
// the forward's sums and the pair-slot gather: with the OIT blend that is the
// fixed-order emission where the tile grid allows it (no sort), else the
// depth sort.  The OIT blend of Eq. 1-4 is order-independent, so by default
// it skips the sort (the paper's sort-free pass): its lists keep emission
// order, which varies with the order in which the binning's atomics ran, so
// its FP32 sums may differ run to run in the last bits.  The per-Gaussian
// schedule never sorts.
bool view_sorted(const GpsView& vw, const GpsRenderSettings& s, const TileCfg& tc) {
  return s.schedule == GPS_SCHEDULE_TILES &&
         (s.blend_mode == GPS_BLEND_ALPHA || (s.deterministic && !view_fixed_order(vw, s, tc)));
}

// Bins of a view's binning pass.  Lists that stay unsorted are binned
// straight into tiles (one pass: histogram, scan, emission) when the view's
// tile grid fits the shared-memory histogram; otherwise its Gaussians go into
// square super-tiles, whose segments are sorted (where an order is wanted)
// and split into their tiles.
bool view_tile_bins(const GpsView& vw, const GpsRenderSettings& s, const TileCfg& tc) {
  return !view_sorted(vw, s, tc) && view_tiles(vw, tc) <= kSuperMax;
}

// Workspace: [status 256 B] then per view, in order, its regions.
// Deterministic mode sums the OIT blend's 2D gradients in fixed point (any
// order of the carry-over backward's additions gives the same bits).
bool fixed_point_grads(const GpsRenderSettings& s) {
  return s.deterministic && s.blend_mode == GPS_BLEND_OIT && s.schedule == GPS_SCHEDULE_TILES;
}

// A backward call that runs both the composite and the projection adjoint
// of deterministic OIT lets the projection adjoint convert the fixed-point
// sums as it reads them (grad2d is then not written).
bool folds_fixed_sums(const GpsRenderSettings& s, int stages) {
  return fixed_point_grads(s) && (stages & GPS_STAGE_COMPOSITE_BWD) &&
         (stages & GPS_STAGE_PROJECT_BWD);
}

int32_t layout(int32_t M, const GpsView* views, int32_t n_views, const GpsRenderSettings* s,
               int32_t want, GpsWorkspaceLayout* out, size_t* total) {
  if (M < 0 || n_views <= 0 || !views || !s) return fail(GPS_ERR_INVALID_ARG, "bad layout arguments");
  TileCfg tc;
  if (!tile_cfg(s, tc)) return fail(GPS_ERR_INVALID_ARG, "unsupported tile size %dx%d", s->tile_w, s->tile_h);
  const long long cap = pair_cap(s, M);
  const int sh = super_shift_for(tc.tw), sp = 1 << sh;
  const int per_super = (sp / tc.tw) * (sp / tc.th);
  if (cap <= 0 || cap * per_super > 0xFFFFFFF0LL)
    return fail(GPS_ERR_INVALID_ARG, "pair_capacity out of range");
  const size_t nblocks = (size_t)bin_blocks(M);
  for (int v = 0; v < n_views; ++v)
    if (views[v].K.width <= 0 || views[v].K.height <= 0)
      return fail(GPS_ERR_INVALID_ARG, "view %d has size %dx%d", v, views[v].K.width,
                  views[v].K.height);
  size_t off = 256;
  for (int v = 0; v < n_views; ++v) {
    const bool by_tile = view_tile_bins(views[v], *s, tc);
    const int W = views[v].K.width, H = views[v].K.height;
    const int tx = (W + tc.tw - 1) / tc.tw, ty = (H + tc.th - 1) / tc.th;
    const int sx = by_tile ? tx : (W + sp - 1) / sp, sy = by_tile ? ty : (H + sp - 1) / sp;
    if ((long long)sx * sy > kSuperMax)
      return fail(GPS_ERR_INVALID_ARG, "view %d: image too large (%d super-tiles)", v, sx * sy);
    const size_t ntiles = (size_t)tx * ty, npx = (size_t)W * H, nbins = (size_t)sx * sy;
    GpsWorkspaceLayout L{};
    L.status = 0;
    L.records = off; off = align256(off + (size_t)M * 64);
    L.super_counts = off; off = align256(off + nbins * 4);
    L.block_base = off; off = align256(off + nblocks * nbins * 4);
    L.super_ranges = off; off = align256(off + nbins * 8);
    if (by_tile) {
      // the emission writes the tile lists themselves (room for per_super *
      // cap entries, as the split's output); no segments, no sort scratch
      L.super_keys = off; off = align256(off + (size_t)cap * per_super * 8);
      L.super_scratch = L.super_keys;
      L.tile_ranges = L.super_ranges;
      L.pair_keys = L.super_keys;
    } else {
      L.super_keys = off; off = align256(off + (size_t)cap * 8);
      L.super_scratch = off; off = align256(off + (size_t)cap * 8);
    }
    // with one tile per super-tile the tile lists are the sorted segments
    // themselves: tile ranges and pair keys alias the super-tile regions
    if (!by_tile && per_super == 1) {
      L.tile_ranges = L.super_ranges;
      L.pair_keys = L.super_keys;
    } else if (!by_tile) {
      L.tile_ranges = off; off = align256(off + ntiles * 8);
      L.pair_keys = off; off = align256(off + (size_t)cap * per_super * 8);
    }
    L.pix_state = off; off = align256(off + npx * 32);
    L.tile_partials = off; off = align256(off + ntiles * 16);
    L.view_scalars = off; off = align256(off + 64);
    L.grad2d = off; off = align256(off + (size_t)M * 48);
    // deterministic mode: fixed-point sums (OIT, tile schedule) or one slot
    // per (tile, Gaussian) pair (the front-to-back variant)
    const bool fixed = fixed_point_grads(*s);
    L.pair_grads = off;
    off = align256(off + (s->deterministic && !fixed ? (size_t)cap * per_super * 48 : 0));
    L.pix_grad = off;
    off = align256(off + (s->schedule == GPS_SCHEDULE_PER_GAUSSIAN ? npx * 32 : 0));
    L.pair_base = off;
    off = align256(off + (s->deterministic && !fixed ? (size_t)M * 4 : 0));
    L.tile_order = off;
    off = align256(off + ntiles * 4);
    L.grad_fixed = off;
    off = align256(off + (fixed ? (size_t)M * 80 : 0));
    L.tiles_x = tx;
    L.tiles_y = ty;
    L.tile_w = tc.tw;
    L.tile_h = tc.th;
    L.super_x = sx;
    L.super_y = sy;
    L.super_px = by_tile ? 0 : sp;
    L.tile_bins = by_tile ? 1 : 0;
    L.pair_capacity = cap;
    if (v == want && out) *out = L;
  }
  if (out) out->total_bytes = off;
  if (total) *total = off;
  return GPS_OK;
}

// Does any view of the batch have depth-sorted lists?  (The super-tile views
// of one call are all sorted or all unsorted: sorting follows the blend and
// deterministic mode, and deterministic OIT views sort only as super-tiles.)
int batch_sorted(const ViewBatch& vb) {
  for (int j = 0; j < vb.n; ++j)
    if (vb.v[j].sorted) return 1;
  return 0;
}

bool finite_cam(const GpsIntrinsics& K, const GpsPose& P) {
  bool ok = std::isfinite(K.fx) && std::isfinite(K.fy) && std::isfinite(K.cx) &&
            std::isfinite(K.cy) && K.fx > 0 && K.fy > 0 && K.width > 0 && K.height > 0;
  for (int k = 0; k < 9; ++k) ok = ok && std::isfinite(P.R[k]);
  for (int k = 0; k < 3; ++k) ok = ok && std::isfinite(P.t[k]);
  return ok;
}

int32_t check_gaussians(const GpsGaussians* g, const char* what) {
  if (!g) return fail(GPS_ERR_INVALID_ARG, "%s is NULL", what);
  if (g->M < 0) return fail(GPS_ERR_INVALID_ARG, "%s.M < 0", what);
  if (g->sh_degree < 0 || g->sh_degree > 3)
    return fail(GPS_ERR_INVALID_ARG, "%s.sh_degree must be 0..3", what);
  if (g->M == 0) return GPS_OK;
  if (g->sh_degree > 0 && (!g->sh_rest || !aligned(g->sh_rest, 4)))
    return fail(GPS_ERR_INVALID_ARG, "%s.sh_rest must be a 4-byte aligned array", what);
  if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->rgb)
    return fail(GPS_ERR_INVALID_ARG, "%s has a NULL array", what);
  if (!aligned(g->means, 4) || !aligned(g->log_scales, 4) || !aligned(g->quats, 16) ||
      !aligned(g->opacity_logits, 4) || !aligned(g->rgb, 4))
    return fail(GPS_ERR_INVALID_ARG, "%s arrays must be 4-byte aligned (quats 16-byte)", what);
  return GPS_OK;
}

ViewDev make_view(const GpsView& vw, char* ws, const GpsWorkspaceLayout& L, int prec, int M,
                  bool fixed, bool fixed_order, bool sorted) {
  ViewDev v{};
  v.cam = make_cam(vw.K, vw.T_wc);
  v.Ct = vw.sdf_rgb;
  v.Dt = vw.sdf_depth;
  v.Ctgt = vw.target_rgb;
  v.Dtgt = vw.target_depth;
  v.out_rgb = vw.out_rgb;
  v.out_depth = vw.out_depth;
  v.out_weight = vw.out_weight;
  v.g_rgb = vw.grad_rgb;
  v.g_depth = vw.grad_depth;
  v.fused = (vw.grad_rgb || vw.grad_depth) ? 0 : 1;
  v.prec = prec;
  v.rec = reinterpret_cast<float4*>(ws + L.records);
  v.sup_count = reinterpret_cast<uint32_t*>(ws + L.super_counts);
  v.block_base = reinterpret_cast<uint32_t*>(ws + L.block_base);
  v.sup_ranges = reinterpret_cast<uint2*>(ws + L.super_ranges);
  v.sup_keys = reinterpret_cast<unsigned long long*>(ws + L.super_keys);
  v.sup_tmp = reinterpret_cast<unsigned long long*>(ws + L.super_scratch);
  v.tile_ranges = reinterpret_cast<uint2*>(ws + L.tile_ranges);
  v.keys = reinterpret_cast<unsigned long long*>(ws + L.pair_keys);
  const size_t npx = (size_t)vw.K.width * vw.K.height;
  v.pix_a = reinterpret_cast<float4*>(ws + L.pix_state);
  v.pix_b = v.pix_a + npx;
  v.tile_partials = reinterpret_cast<float4*>(ws + L.tile_partials);
  v.scalars = reinterpret_cast<float*>(ws + L.view_scalars);
  v.grad2d = reinterpret_cast<float4*>(ws + L.grad2d);
  v.pair_grads = reinterpret_cast<float4*>(ws + L.pair_grads);
  v.pix_g = reinterpret_cast<float4*>(ws + L.pix_grad);
  v.pair_base = reinterpret_cast<uint32_t*>(ws + L.pair_base);
  v.tile_order = reinterpret_cast<int*>(ws + L.tile_order);
  v.fixed_order = fixed_order && L.tile_bins ? 1 : 0;
  v.tile_bin = L.tile_bins;
  v.sorted = sorted ? 1 : 0;
  v.grad_fixed = fixed ? reinterpret_cast<long long*>(ws + L.grad_fixed) : nullptr;
  {
    const int sp = 1 << super_shift_for(L.tile_w);
    v.pair_slots = L.pair_capacity * ((sp / L.tile_w) * (sp / L.tile_h));
  }
  v.tiles_x = L.tiles_x;
  v.tiles_y = L.tiles_y;
  v.tw = L.tile_w;
  v.th = L.tile_h;
  v.sup_x = L.super_x;
  v.sup_y = L.super_y;
  if (L.tile_bins) {
    v.bin_sx = L.tile_w == 32 ? 5 : L.tile_w == 16 ? 4 : 3;
    v.bin_sy = L.tile_h == 16 ? 4 : 3;
    v.cap = L.pair_capacity * (((1 << super_shift_for(L.tile_w)) / L.tile_w) *
                               ((1 << super_shift_for(L.tile_w)) / L.tile_h));
  } else {
    v.bin_sx = v.bin_sy = L.super_px == 32 ? 5 : 4;
    v.cap = L.pair_capacity;
  }
  return v;
}

// Views [b0, b0 + kMaxBatch) of a call as one batch: device descriptors,
// work items ordered largest view first, and the largest super-tile count.
void make_batch(int M, const GpsView* views, int32_t n_views, const GpsRenderSettings* s,
                char* base, int b0, ViewBatch& vb, int& max_nsup) {
  std::memset(&vb, 0, sizeof(vb));
  vb.n = std::min(kMaxBatch, n_views - b0);
  max_nsup = 0;
  int tiles[kMaxBatch];
  TileCfg tc;
  tile_cfg(s, tc);
  for (int j = 0; j < vb.n; ++j) {
    GpsWorkspaceLayout L;
    layout(M, views, n_views, s, b0 + j, &L, nullptr);
    const GpsView& vw = views[b0 + j];
    vb.v[j] = make_view(vw, base, L, s->precision, M, fixed_point_grads(*s),
                        view_fixed_order(vw, *s, tc), view_sorted(vw, *s, tc));
    max_nsup = std::max(max_nsup, vb.v[j].sup_x * vb.v[j].sup_y);
    tiles[j] = vb.v[j].tiles_x * vb.v[j].tiles_y;
    vb.order[j] = j;
  }
  std::stable_sort(vb.order, vb.order + vb.n, [&](int a, int b) { return tiles[a] > tiles[b]; });
  for (int k = 0; k < vb.n; ++k) {
    const ViewDev& v = vb.v[vb.order[k]];
    vb.tile_start[k + 1] = vb.tile_start[k] + v.tiles_x * v.tiles_y;
    vb.sup_start[k + 1] = vb.sup_start[k] + v.sup_x * v.sup_y;
  }
}

int32_t check_render_args(const GpsGaussians* g, const GpsView* views, int32_t n_views,
                          const GpsRenderSettings* s, void* ws, size_t ws_bytes) {
  if (int32_t e = check_gaussians(g, "gaussians")) return e;
  if (!views || n_views <= 0) return fail(GPS_ERR_INVALID_ARG, "no views");
  if (!s) return fail(GPS_ERR_INVALID_ARG, "settings is NULL");
  if (!std::isfinite(s->eps_depth) || !std::isfinite(s->lambda_depth) || !std::isfinite(s->near_plane))
    return fail(GPS_ERR_INVALID_ARG, "non-finite settings");
  if (s->blend_mode != GPS_BLEND_OIT && s->blend_mode != GPS_BLEND_ALPHA)
    return fail(GPS_ERR_INVALID_ARG, "unknown blend_mode %d", s->blend_mode);
  if (s->precision != GPS_PREC_FP32 && s->precision != GPS_PREC_FP16 && s->precision != GPS_PREC_BF16)
    return fail(GPS_ERR_INVALID_ARG, "unknown precision %d", s->precision);
  if (s->schedule != GPS_SCHEDULE_TILES && s->schedule != GPS_SCHEDULE_PER_GAUSSIAN)
    return fail(GPS_ERR_INVALID_ARG, "unknown schedule %d", s->schedule);
  if (s->schedule == GPS_SCHEDULE_PER_GAUSSIAN && s->blend_mode != GPS_BLEND_OIT)
    return fail(GPS_ERR_INVALID_ARG, "the per-Gaussian schedule is order-independent (OIT) only");
  if (!ws || !aligned(ws, 256)) return fail(GPS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  for (int v = 0; v < n_views; ++v) {
    if (!finite_cam(views[v].K, views[v].T_wc))
      return fail(GPS_ERR_INVALID_ARG, "view %d: bad intrinsics or pose", v);
    if (!views[v].sdf_rgb || !views[v].sdf_depth)
      return fail(GPS_ERR_INVALID_ARG, "view %d: sdf_rgb / sdf_depth are required", v);
  }
  size_t need = 0;
  if (int32_t e = layout(g->M, views, n_views, s, -1, nullptr, &need)) return e;
  if (ws_bytes < need)
    return fail(GPS_ERR_WORKSPACE_TOO_SMALL, "workspace has %zu bytes, needs %zu", ws_bytes, need);
  return GPS_OK;
}

// The composite adjoint of one batch of views, into the views' grad2d.
// Deterministic mode first places each Gaussian's pair slots (pair_base),
// writes every pair's gradient into its slot and sums each Gaussian's slots
// in order; with the OIT blend it sums into fixed-point integers instead,
// left unconverted when `fold` (the projection adjoint of the same call
// reads them).
cudaError_t composite_backward(const ViewBatch& vb, int M, const GpsRenderSettings* s, int stages,
                               const float* dloss, const int* status, bool fold,
                               cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if ((stages & GPS_STAGE_COMPOSITE_BWD) && s->schedule == GPS_SCHEDULE_PER_GAUSSIAN) {
    e = launch_composite_bwd_per_gaussian(vb, M, s->eps_depth, s->lambda_depth, dloss,
                                          s->instrument ? 1 : 0, st);
  } else if ((stages & GPS_STAGE_COMPOSITE_BWD) && fixed_point_grads(*s)) {
    // deterministic, OIT: the carry-over walk with fixed-point sums.  The
    // quanta need bounds on the upstream terms: the forward's loss left them
    // for views with the fused loss; the others take the maxima of their
    // upstream images.
    bool any_explicit = false;
    for (int j = 0; j < vb.n && e == cudaSuccess; ++j) {
      e = cudaMemsetAsync(vb.v[j].grad_fixed, 0, (size_t)M * 80, st);
      if (e == cudaSuccess && !vb.v[j].fused) {
        e = cudaMemsetAsync(vb.v[j].scalars + 6, 0, 2 * sizeof(float), st);
        any_explicit = true;
      }
    }
    if (e == cudaSuccess && any_explicit)
      e = launch_upstream_max(vb, s->eps_depth, s->lambda_depth, dloss, st);
    if (e == cudaSuccess)
      e = launch_composite_bwd(vb, vb.v[0].tw, vb.v[0].th, s->eps_depth, s->lambda_depth, dloss,
                               s->blend_mode, 1, s->instrument ? 1 : 0, batch_sorted(vb), st);
    if (e == cudaSuccess && M > 0 && !fold) e = launch_fixed_to_grad2d(vb, M, dloss, st);
  } else if (stages & GPS_STAGE_COMPOSITE_BWD) {
    for (int j = 0; j < vb.n && e == cudaSuccess; ++j)
      e = s->deterministic ? cudaMemsetAsync(vb.v[j].scalars + 5, 0, sizeof(float), st)
                           : cudaMemsetAsync(vb.v[j].grad2d, 0, (size_t)M * 48, st);
    if (e == cudaSuccess && s->deterministic && M > 0) e = launch_pair_base(vb, M, status, st);
    if (e == cudaSuccess)
      e = launch_composite_bwd(vb, vb.v[0].tw, vb.v[0].th, s->eps_depth, s->lambda_depth, dloss,
                               s->blend_mode, s->deterministic ? 1 : 0, s->instrument ? 1 : 0,
                               batch_sorted(vb), st);
    if (e == cudaSuccess && s->deterministic && M > 0) e = launch_gather_pair_grads(vb, M, st);
  }
  return e;
}

int32_t check_backward_views(const GpsView* views, int32_t n_views) {
  for (int vi = 0; vi < n_views; ++vi) {
    const GpsView& vw = views[vi];
    if (!vw.grad_rgb && !vw.grad_depth && (!vw.target_rgb || !vw.target_depth))
      return fail(GPS_ERR_INVALID_ARG, "view %d: no upstream gradients and no targets", vi);
  }
  return GPS_OK;
}

int32_t check_adam(const GpsGaussians* params, const GpsGaussians* m, const GpsGaussians* v,
                   const GpsAdamHyper* hyper, int32_t step, const int32_t* device_step) {
  if (int32_t e = check_gaussians(m, "m")) return e;
  if (int32_t e = check_gaussians(v, "v")) return e;
  if (m->M != params->M || v->M != params->M) return fail(GPS_ERR_INVALID_ARG, "group sizes differ");
  if (m->sh_degree != params->sh_degree || v->sh_degree != params->sh_degree)
    return fail(GPS_ERR_INVALID_ARG, "SH degrees differ");
  if (!hyper) return fail(GPS_ERR_INVALID_ARG, "hyper is NULL");
  if (step <= 0 && !device_step) return fail(GPS_ERR_INVALID_ARG, "step <= 0 needs device_step");
  if (!(hyper->beta1 >= 0 && hyper->beta1 < 1 && hyper->beta2 >= 0 && hyper->beta2 < 1 &&
        hyper->eps >= 0))
    return fail(GPS_ERR_INVALID_ARG, "bad Adam hyper-parameters");
  return GPS_OK;
}

}  // namespace

namespace gps {
void set_error(const char* msg) { g_err = msg; }
}  // namespace gps

extern "C" {

const char* gps_last_error(void) { return g_err.c_str(); }

const char* gps_version(void) { return "gps-b300 0.1 (sm_103a)"; }

int32_t gps_workspace_size(int32_t M, const GpsView* views, int32_t n_views,
                           const GpsRenderSettings* settings, size_t* bytes) {
  if (!bytes) return fail(GPS_ERR_INVALID_ARG, "bytes is NULL");
  return layout(M, views, n_views, settings, -1, nullptr, bytes);
}

int32_t gps_workspace_layout(int32_t M, const GpsView* views, int32_t n_views,
                             const GpsRenderSettings* settings, int32_t view,
                             GpsWorkspaceLayout* out) {
  if (!out || view < 0 || view >= n_views) return fail(GPS_ERR_INVALID_ARG, "bad view / out");
  return layout(M, views, n_views, settings, view, out, nullptr);
}

int32_t gps_query_status(const void* ws, size_t ws_bytes, int32_t* status, void* stream) {
  if (!ws || !status || ws_bytes < 256) return fail(GPS_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(status, ws, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "gps_query_status");
  return GPS_OK;
}

int32_t fuse_frame(GpsTsdf* vol, const float* depth, const float* rgb, const GpsIntrinsics* K,
                   const GpsPose* T_wc, void* stream) {
  if (!vol || !depth || !rgb || !K || !T_wc) return fail(GPS_ERR_INVALID_ARG, "NULL argument");
  if (vol->nx <= 0 || vol->ny <= 0 || vol->nz <= 0 || vol->nx % 8 || vol->ny % 8 || vol->nz % 8)
    return fail(GPS_ERR_INVALID_ARG, "volume dims must be positive multiples of 8");
  if ((vol->ny >> 3) > 65535 || (vol->nz >> 3) > 65535)
    return fail(GPS_ERR_INVALID_ARG, "ny and nz must be at most 8 * 65535");
  if (!vol->sdf || !vol->weight || !vol->rgbw || !aligned(vol->rgbw, 16))
    return fail(GPS_ERR_INVALID_ARG, "volume arrays missing or rgbw not 16-byte aligned");
  if (!(vol->voxel > 0) || !(vol->trunc > 0) || !(vol->max_weight > 0))
    return fail(GPS_ERR_INVALID_ARG, "voxel, trunc and max_weight must be positive");
  if (!finite_cam(*K, *T_wc)) return fail(GPS_ERR_INVALID_ARG, "bad intrinsics or pose");
  cudaError_t e = launch_fuse(*vol, depth, rgb, make_cam(*K, *T_wc), static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GPS_OK : cuda_fail(e, "fuse_frame");
}

int32_t tsdf_mark_bricks(GpsTsdf* vol, void* stream) {
  if (!vol || !vol->sdf || !vol->brick_flags) return fail(GPS_ERR_INVALID_ARG, "NULL volume or flags");
  if (vol->nx < 8 || vol->ny < 8 || vol->nz < 8 || vol->nx % 8 || vol->ny % 8 || vol->nz % 8)
    return fail(GPS_ERR_INVALID_ARG, "volume dims must be positive multiples of 8");
  const cudaError_t e = launch_mark_bricks(*vol, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GPS_OK : cuda_fail(e, "tsdf_mark_bricks");
}

int32_t raycast_sdf(const GpsTsdf* vol, const GpsIntrinsics* K, const GpsPose* T_wc,
                    float near_plane, float far_plane, void* out_rgb, int32_t rgb_precision,
                    float* out_depth, float* out_vertex, void* stream) {
  if (!vol || !K || !T_wc || !out_rgb || !out_depth) return fail(GPS_ERR_INVALID_ARG, "NULL argument");
  if (rgb_precision != GPS_PREC_FP32 && rgb_precision != GPS_PREC_FP16 && rgb_precision != GPS_PREC_BF16)
    return fail(GPS_ERR_INVALID_ARG, "unknown rgb precision %d", rgb_precision);
  if (vol->nx < 8 || vol->ny < 8 || vol->nz < 8 || vol->nx % 8 || vol->ny % 8 || vol->nz % 8)
    return fail(GPS_ERR_INVALID_ARG, "volume dims must be positive multiples of 8");
  if (!vol->sdf || !vol->rgbw || !aligned(vol->rgbw, 16))
    return fail(GPS_ERR_INVALID_ARG, "volume arrays missing or rgbw not 16-byte aligned");
  if (!(vol->voxel > 0) || !(vol->trunc > 0) || !std::isfinite(near_plane) || !std::isfinite(far_plane))
    return fail(GPS_ERR_INVALID_ARG, "bad voxel / trunc / near / far");
  if (!finite_cam(*K, *T_wc)) return fail(GPS_ERR_INVALID_ARG, "bad intrinsics or pose");
  cudaError_t e = launch_raycast(*vol, make_cam(*K, *T_wc), near_plane, far_plane, out_rgb,
                                 rgb_precision, out_depth, out_vertex,
                                 static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GPS_OK : cuda_fail(e, "raycast_sdf");
}

int32_t render_forward(const GpsGaussians* g, const GpsView* views, int32_t n_views,
                       const GpsRenderSettings* s, void* ws, size_t ws_bytes, float* loss,
                       void* stream) {
  if (int32_t e = check_render_args(g, views, n_views, s, ws, ws_bytes)) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int stages = s->stages ? s->stages : 0x1f;
  bool has_tgt = true;
  for (int v = 0; v < n_views; ++v) has_tgt = has_tgt && views[v].target_rgb && views[v].target_depth;
  char* base = static_cast<char*>(ws);
  int* status = reinterpret_cast<int*>(base);
  cudaError_t e = cudaSuccess;
  if (stages & GPS_STAGE_PROJECT) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  // one launch per stage for up to kMaxBatch views
  for (int b0 = 0; b0 < n_views && e == cudaSuccess; b0 += kMaxBatch) {
    ViewBatch vb;
    int max_nsup = 0;
    make_batch(g->M, views, n_views, s, base, b0, vb, max_nsup);
    const ViewDev& v0 = vb.v[0];
    if (stages & (GPS_STAGE_PROJECT | GPS_STAGE_BIN)) {
      for (int j = 0; j < vb.n && e == cudaSuccess; ++j)
        e = cudaMemsetAsync(vb.v[j].sup_count, 0, (size_t)vb.v[j].sup_x * vb.v[j].sup_y * 4, st);
      if (e == cudaSuccess && g->M > 0)
        e = (stages & GPS_STAGE_PROJECT) ? launch_project(*g, s->near_plane, vb, max_nsup, st)
                                         : launch_bin_histogram(g->M, vb, max_nsup, st);
    }
    if (e == cudaSuccess && (stages & GPS_STAGE_BIN)) {
      // fixed order: the histogram wrote per-block counts; turn them into
      // bases in block order and the bins' totals (the views with other
      // bins return at once)
      bool any_fixed = false, any_super = false;
      for (int j = 0; j < vb.n; ++j) {
        any_fixed = any_fixed || vb.v[j].fixed_order;
        any_super = any_super || !vb.v[j].tile_bin;
      }
      if (any_fixed && g->M > 0) e = launch_block_prefix(g->M, vb, max_nsup, st);
      if (e == cudaSuccess) e = launch_scan_super(vb, status, st);
      if (e == cudaSuccess && g->M > 0) e = launch_emit_super(g->M, vb, max_nsup, st);
      // super-tile bins: split each segment into its tiles' lists, sorted by
      // depth where the settings ask for an order (see view_sorted); views
      // binned straight into tiles return at once
      if (e == cudaSuccess && any_super)
        e = launch_sort_split(vb, v0.tw, v0.th, batch_sorted(vb), st);
    }
    if (e == cudaSuccess && (stages & GPS_STAGE_COMPOSITE)) {
      for (int j = 0; j < vb.n && e == cudaSuccess && s->instrument; ++j)
        e = cudaMemsetAsync(vb.v[j].scalars + 8, 0, 32, st);
      if (e == cudaSuccess)
        e = launch_composite_fwd(vb, v0.tw, v0.th, s->eps_depth, s->blend_mode, has_tgt ? 1 : 0,
                                 s->instrument ? 1 : 0, batch_sorted(vb), st);
      if (e == cudaSuccess && has_tgt)
        e = launch_finalize_loss(vb, s->lambda_depth, loss, b0 == 0 ? 1 : 0, st);
    }
  }
  if (e == cudaSuccess && !has_tgt && loss) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  return e == cudaSuccess ? GPS_OK : cuda_fail(e, "render_forward");
}

int32_t render_backward(const GpsGaussians* g, const GpsView* views, int32_t n_views,
                        const GpsRenderSettings* s, void* ws, size_t ws_bytes, const float* dloss,
                        GpsGaussians* grads, void* stream) {
  if (int32_t e = check_render_args(g, views, n_views, s, ws, ws_bytes)) return e;
  if (int32_t e = check_gaussians(grads, "grads")) return e;
  if (grads->M != g->M) return fail(GPS_ERR_INVALID_ARG, "grads.M != gaussians.M");
  if (grads->sh_degree != g->sh_degree)
    return fail(GPS_ERR_INVALID_ARG, "grads.sh_degree != gaussians.sh_degree");
  if (int32_t e = check_backward_views(views, n_views)) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int stages = s->stages ? s->stages : 0x1f;
  char* base = static_cast<char*>(ws);
  cudaError_t e = cudaSuccess;
  for (int b0 = 0; b0 < n_views && e == cudaSuccess; b0 += kMaxBatch) {
    ViewBatch vb;
    int max_nsup = 0;
    make_batch(g->M, views, n_views, s, base, b0, vb, max_nsup);
    const bool fold = folds_fixed_sums(*s, stages);
    e = composite_backward(vb, g->M, s, stages, dloss, reinterpret_cast<const int*>(base), fold,
                           st);
    if (e == cudaSuccess && (stages & GPS_STAGE_PROJECT_BWD) && g->M > 0)
      e = launch_project_backward(*g, s->near_plane, vb, *grads, fold, dloss, st);
  }
  return e == cudaSuccess ? GPS_OK : cuda_fail(e, "render_backward");
}

int32_t render_backward_adam(GpsGaussians* g, const GpsView* views, int32_t n_views,
                             const GpsRenderSettings* s, void* ws, size_t ws_bytes,
                             const float* dloss, GpsGaussians* m, GpsGaussians* v,
                             const GpsAdamHyper* hyper, int32_t step, int32_t* device_step,
                             void* stream) {
  if (int32_t e = check_render_args(g, views, n_views, s, ws, ws_bytes)) return e;
  if (n_views > kMaxBatch)
    return fail(GPS_ERR_INVALID_ARG, "render_backward_adam takes at most %d views", kMaxBatch);
  const int stages = s->stages ? s->stages : 0x1f;
  if (!(stages & GPS_STAGE_PROJECT_BWD))
    return fail(GPS_ERR_INVALID_ARG, "render_backward_adam needs the GPS_STAGE_PROJECT_BWD stage");
  if (int32_t e = check_backward_views(views, n_views)) return e;
  if (int32_t e = check_adam(g, m, v, hyper, step, device_step)) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ViewBatch vb;
  int max_nsup = 0;
  make_batch(g->M, views, n_views, s, static_cast<char*>(ws), 0, vb, max_nsup);
  const bool fold = folds_fixed_sums(*s, stages);
  cudaError_t e =
      composite_backward(vb, g->M, s, stages, dloss, static_cast<const int*>(ws), fold, st);
  if (e == cudaSuccess && g->M > 0)
    e = launch_project_backward_adam(*g, s->near_plane, vb, *m, *v, *hyper, step, device_step,
                                     fold, dloss, st);
  return e == cudaSuccess ? GPS_OK : cuda_fail(e, "render_backward_adam");
}

int32_t adam_step(GpsGaussians* params, GpsGaussians* grads, GpsGaussians* m, GpsGaussians* v,
                  const GpsAdamHyper* hyper, int32_t step, int32_t* device_step, void* stream) {
  if (int32_t e = check_gaussians(params, "params")) return e;
  if (int32_t e = check_gaussians(grads, "grads")) return e;
  if (grads->M != params->M) return fail(GPS_ERR_INVALID_ARG, "group sizes differ");
  if (grads->sh_degree != params->sh_degree) return fail(GPS_ERR_INVALID_ARG, "SH degrees differ");
  if (int32_t e = check_adam(params, m, v, hyper, step, device_step)) return e;
  cudaError_t e = launch_adam(*params, *grads, *m, *v, *hyper, step, device_step,
                              static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GPS_OK : cuda_fail(e, "adam_step");
}

}  // extern "C"
