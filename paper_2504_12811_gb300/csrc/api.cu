// C ABI of libaaag: workspace management, argument checks, host-side frame
// setup and the entry points declared in include/aaag.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>

#include "aaag_internal.cuh"

namespace aaag {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

aaag_status check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return AAAG_ERR_CUDA;
  }
  return AAAG_OK;
}

const LaunchConfig& launch_config() {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static LaunchConfig cfg[kMaxDevices];
  static bool ready[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (!ready[dev]) {
    LaunchConfig c;
    std::memset(&c, 0, sizeof(c));
    if (cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c.sms < 1) c.sms = 1;
    configure_preprocess(c);
    configure_cull(c);
    configure_sort(c);
    configure_render(c);
    configure_backward(c);
    cfg[dev] = c;
    ready[dev] = true;
  }
  return cfg[dev];
}

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
  size_t records, aux, cand, counts, offsets, owner, mask, cull_lb, keys0, keys1, vals0, vals1, hist, counters,
      lookback, ranges, order, final_T, n_blended, stats, grad, fc, total;
};

int tiles_of(int size) { return (size + kTile - 1) / kTile; }

// Work items of the tile culling: every visible Gaussian has at least one
// chunk of 32 candidate tiles; the pair capacity bounds the rest.
int64_t chunk_capacity_of(int64_t n, int64_t cap) { return n + cap / 4 + 1024; }

Layout layout_of(int64_t n, int w, int h, int64_t cap) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + (bytes ? bytes : 1));
    return at;
  };
  const int64_t ccap = chunk_capacity_of(n, cap);
  const int64_t nst = sort_max_tiles(cap) + 1;
  const size_t ntiles = (size_t)tiles_of(w) * tiles_of(h);
  L.records = take((size_t)n * sizeof(Record));
  L.aux = take((size_t)n * 16);
  L.cand = take((size_t)n * 4);
  L.counts = take((size_t)n * 4);
  L.offsets = take((size_t)n * 4);
  L.owner = take((size_t)ccap * 4);
  L.mask = take((size_t)ccap * 4);
  L.cull_lb = take((size_t)cull_lookback_words(n, ccap) * 8);
  L.keys0 = take((size_t)cap * 4);
  L.keys1 = take((size_t)cap * 4);
  L.vals0 = take((size_t)cap * 4);
  L.vals1 = take((size_t)cap * 4);
  L.hist = take(4 * 256 * 4);
  L.counters = take(4 * 4);
  L.lookback = take((size_t)nst * 256 * 8);
  L.ranges = take(ntiles * sizeof(uint2));
  L.order = take(ntiles * sizeof(uint32_t));
  L.final_T = take((size_t)w * h * 4);
  L.n_blended = take((size_t)w * h * 4);
  L.stats = take(kStatCount * 8);
  L.grad = take((size_t)n * 64);
  L.fc = take(sizeof(FrameConst));
  L.total = off;
  return L;
}

bool finite_camera(const aaag_camera* c) {
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(c->viewmat[i])) return false;
  const float v[] = {c->fx, c->fy, c->cx, c->cy, c->znear, c->bg[0], c->bg[1], c->bg[2]};
  for (float x : v)
    if (!std::isfinite(x)) return false;
  return c->fx > 0 && c->fy > 0 && c->znear > 0;
}

// Frame constants in double precision: exact inverse of the view rotation for
// the camera origin, tile and key geometry.
aaag_status make_frame(const aaag_camera* cam, const aaag_params* prm, int sh_degree,
                       const aaag_workspace* ws, FrameConst* fc) {
  const float* V = cam->viewmat;
  double R[9], t[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) R[3 * r + c] = V[4 * r + c];
    t[r] = V[4 * r + 3];
  }
  const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                     R[2] * (R[3] * R[7] - R[4] * R[6]);
  if (!(std::fabs(det) > 1e-12)) {
    set_error("view matrix rotation is singular");
    return AAAG_ERR_INVALID_ARG;
  }
  double Ri[9];
  Ri[0] = (R[4] * R[8] - R[5] * R[7]) / det;
  Ri[1] = (R[2] * R[7] - R[1] * R[8]) / det;
  Ri[2] = (R[1] * R[5] - R[2] * R[4]) / det;
  Ri[3] = (R[5] * R[6] - R[3] * R[8]) / det;
  Ri[4] = (R[0] * R[8] - R[2] * R[6]) / det;
  Ri[5] = (R[2] * R[3] - R[0] * R[5]) / det;
  Ri[6] = (R[3] * R[7] - R[4] * R[6]) / det;
  Ri[7] = (R[1] * R[6] - R[0] * R[7]) / det;
  Ri[8] = (R[0] * R[4] - R[1] * R[3]) / det;
  for (int i = 0; i < 9; ++i) fc->Rv[i] = (float)R[i];
  for (int i = 0; i < 3; ++i) {
    fc->tv[i] = (float)t[i];
    fc->o[i] = (float)-(Ri[3 * i] * t[0] + Ri[3 * i + 1] * t[1] + Ri[3 * i + 2] * t[2]);
    fc->bg[i] = cam->bg[i];
  }
  fc->fx = cam->fx;
  fc->fy = cam->fy;
  fc->cx = cam->cx;
  fc->cy = cam->cy;
  fc->W = cam->width;
  fc->H = cam->height;
  {
    // pixel x >= 0, x <= W, y >= 0, y <= H as half-spaces through the camera
    const double W = cam->width, H = cam->height;
    const double n[4][3] = {{cam->fx, 0.0, cam->cx},
                            {-cam->fx, 0.0, W - cam->cx},
                            {0.0, cam->fy, cam->cy},
                            {0.0, -cam->fy, H - cam->cy}};
    for (int j = 0; j < 4; ++j) {
      const double len = std::sqrt(n[j][0] * n[j][0] + n[j][1] * n[j][1] + n[j][2] * n[j][2]);
      for (int c = 0; c < 3; ++c) fc->side[j][c] = (float)(n[j][c] / len);
    }
  }
  fc->tiles_x = ws->tiles_x;
  fc->tiles_y = ws->tiles_y;
  fc->znear = cam->znear;
  fc->k = prm ? prm->k : 0.3f;
  fc->eps = prm ? prm->eps : 1e-3f;
  fc->flags = prm ? prm->flags : 0u;
  int bits = 1;
  while ((1 << bits) < ws->n_tiles) ++bits;
  // key = tile id above the depth key: 24 bits (three radix passes) while at
  // least 16 depth bits remain, else 32.  Coarser depth keys put more pairs of
  // a tile under one key, where they arrive in index order: with 11 depth bits
  // at 1080p the per-pixel queue overflowed 20-45% more often.  (The no-re-sort
  // and bounded-buffer ablations, whose blend order follows the pair order,
  // keep the full 32.)
  const int key_bits = (bits + kMinDepthBits <= 24 && !(fc->flags & kFullKeyFlags)) ? 24 : 32;
  fc->tile_bits = bits;
  fc->depth_bits = key_bits - bits;
  // (bits(z) - bits(znear)) spans 2^27 for z/znear up to 2^16; larger depths
  // clamp to the largest key, which stays a lower bound
  fc->depth_shift = fc->depth_bits >= 27 ? 0 : 27 - fc->depth_bits;
  uint32_t zb;
  std::memcpy(&zb, &cam->znear, 4);
  fc->znear_bits = zb;
  fc->sh_degree = sh_degree;
  return AAAG_OK;
}

__global__ void set_u32_kernel(uint32_t* p, uint32_t v) { *p = v; }

// Frame constants are a kernel parameter here and device memory for every
// other kernel of the frame: a captured frame graph is re-aimed at a new
// camera by updating this one node.
// Frame constants to device memory, and the per-frame statistics reset (the
// words below kStatFrameReset; the sort epoch and the others stay).  The frame
// epoch tags this frame's cull look-back words with its low 24 bits.  When
// those wrap to zero every word is cleared (an unpublished word), so that a
// word left from 2^24 frames earlier can never pass for one of this frame.
__global__ void set_frame_kernel(FrameConst* dst, FrameConst v, unsigned long long* stats,
                                 unsigned long long* cull_lb, long long lb_words) {
  pdl_begin();
  __shared__ unsigned long long e;
  if (threadIdx.x < kStatFrameReset) stats[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    *dst = v;
    e = stats[kStatFrameEpoch] + 1ull;
    stats[kStatFrameEpoch] = e;
  }
  __syncthreads();
  if ((e & 0xffffffull) == 0ull)
    for (long long i = threadIdx.x; i < lb_words; i += blockDim.x) cull_lb[i] = 0ull;
}

SceneDev scene_dev(const aaag_scene* scene) {
  SceneDev s;
  s.n = scene->n;
  s.sh_degree = scene->sh_degree;
  s.means = scene->means;
  s.log_scales = scene->log_scales;
  s.quats = scene->quats;
  s.opacity_logits = scene->opacity_logits;
  s.sh = scene->sh;
  s.vhat_train = scene->vhat_train;
  return s;
}

aaag_status check_scene(const aaag_scene* scene, const aaag_workspace* ws, const char* who, bool same_frame) {
  if (same_frame && scene->n != ws->n) {
    set_error("%s: scene has %lld Gaussians, the workspace %lld", who, (long long)scene->n, (long long)ws->n);
    return AAAG_ERR_INVALID_ARG;
  }
  if (scene->sh_degree < 0 || scene->sh_degree > kMaxShDegree) {
    set_error("%s: sh_degree %d not in 0..3", who, scene->sh_degree);
    return AAAG_ERR_UNSUPPORTED;
  }
  if (scene->n > 0 && (!scene->means || !scene->log_scales || !scene->quats || !scene->opacity_logits ||
                       !scene->sh || !scene->vhat_train)) {
    set_error("%s: null scene array", who);
    return AAAG_ERR_INVALID_ARG;
  }
  if (((uintptr_t)scene->quats) % 16 || ((uintptr_t)scene->sh) % 16) {
    set_error("%s: quats and sh must be 16-byte aligned", who);
    return AAAG_ERR_INVALID_ARG;
  }
  return AAAG_OK;
}

}  // namespace
}  // namespace aaag

using namespace aaag;

extern "C" {

const char* aaag_last_error(void) { return g_err; }

size_t aaag_workspace_bytes(int64_t n, int32_t width, int32_t height, int64_t pair_capacity) {
  if (n < 0 || width <= 0 || height <= 0 || pair_capacity < 0) return 0;
  return layout_of(n, width, height, pair_capacity).total;
}

aaag_status aaag_workspace_init(void* dev_mem, size_t bytes, int64_t n, int32_t width, int32_t height,
                                int64_t pair_capacity, aaag_workspace** ws) {
  if (!dev_mem || !ws || n < 0 || n >= (1ll << 32) || width <= 0 || height <= 0 || pair_capacity < 0) {
    set_error("aaag_workspace_init: invalid argument");
    return AAAG_ERR_INVALID_ARG;
  }
  if (((uintptr_t)dev_mem) % kAlign) {
    set_error("aaag_workspace_init: device memory must be %zu-byte aligned", kAlign);
    return AAAG_ERR_INVALID_ARG;
  }
  const int tx = tiles_of(width), ty = tiles_of(height);
  if ((int64_t)tx * ty > (1 << kMaxTileBits) || pair_capacity >= (1ll << 30)) {
    set_error("aaag_workspace_init: at most 65536 tiles and 2^30 pairs");
    return AAAG_ERR_UNSUPPORTED;
  }
  const Layout L = layout_of(n, width, height, pair_capacity);
  if (bytes < L.total) {
    set_error("aaag_workspace_init: %zu bytes given, %zu needed", bytes, L.total);
    return AAAG_ERR_CAPACITY;
  }
  auto* w = static_cast<aaag_workspace*>(std::calloc(1, sizeof(aaag_workspace)));
  if (!w) {
    set_error("aaag_workspace_init: out of host memory");
    return AAAG_ERR_CAPACITY;
  }
  char* b = static_cast<char*>(dev_mem);
  w->n_max = n;
  w->width_max = width;
  w->height_max = height;
  w->n_tiles_max = tx * ty;
  w->n = n;
  w->width = width;
  w->height = height;
  w->tiles_x = tx;
  w->tiles_y = ty;
  w->n_tiles = tx * ty;
  w->capacity = pair_capacity;
  w->bytes = bytes;
  w->base = b;
  w->records = reinterpret_cast<Record*>(b + L.records);
  w->aux = reinterpret_cast<uint4*>(b + L.aux);
  w->candidates = reinterpret_cast<uint32_t*>(b + L.cand);
  w->counts = reinterpret_cast<uint32_t*>(b + L.counts);
  w->offsets = reinterpret_cast<uint32_t*>(b + L.offsets);
  w->cull_lookback = reinterpret_cast<unsigned long long*>(b + L.cull_lb);
  w->chunk_mask = reinterpret_cast<uint32_t*>(b + L.mask);
  w->chunk_capacity = chunk_capacity_of(n, pair_capacity);
  w->chunk_owner = reinterpret_cast<uint32_t*>(b + L.owner);
  w->keys[0] = reinterpret_cast<uint32_t*>(b + L.keys0);
  w->keys[1] = reinterpret_cast<uint32_t*>(b + L.keys1);
  w->vals[0] = reinterpret_cast<uint32_t*>(b + L.vals0);
  w->vals[1] = reinterpret_cast<uint32_t*>(b + L.vals1);
  w->sort_hist = reinterpret_cast<uint32_t*>(b + L.hist);
  w->sort_counters = reinterpret_cast<uint32_t*>(b + L.counters);
  w->sort_lookback = reinterpret_cast<unsigned long long*>(b + L.lookback);
  w->ranges = reinterpret_cast<uint2*>(b + L.ranges);
  w->tile_order = reinterpret_cast<uint32_t*>(b + L.order);
  w->final_T = reinterpret_cast<float*>(b + L.final_T);
  w->n_blended = reinterpret_cast<uint32_t*>(b + L.n_blended);
  w->stats = reinterpret_cast<unsigned long long*>(b + L.stats);
  w->grad_acc = reinterpret_cast<float4*>(b + L.grad);
  w->fc_dev = reinterpret_cast<FrameConst*>(b + L.fc);
  w->n_sort_tiles = sort_max_tiles(pair_capacity);
  w->n_cull_words = cull_lookback_words(n, w->chunk_capacity);
  // the look-back epoch lives in the stats block and must start defined; the
  // look-back words are cleared once so that no stale word can match an epoch
  if (cudaMemset(w->stats, 0, kStatCount * 8) != cudaSuccess ||
      cudaMemset(w->sort_lookback, 0, (size_t)(w->n_sort_tiles + 1) * 256 * 8) != cudaSuccess ||
      cudaMemset(w->cull_lookback, 0, (size_t)w->n_cull_words * 8) != cudaSuccess) {
    std::free(w);
    return check_launch("workspace_init memset");
  }
  // function attributes and occupancy queries of this device, outside any
  // stream capture
  launch_config();
  *ws = w;
  return AAAG_OK;
}

void aaag_workspace_destroy(aaag_workspace* ws) { std::free(ws); }

aaag_status aaag_workspace_get_view(const aaag_workspace* ws, aaag_workspace_view* out) {
  if (!ws || !out) {
    set_error("aaag_workspace_get_view: null argument");
    return AAAG_ERR_INVALID_ARG;
  }
  std::memset(out, 0, sizeof(*out));
  out->records = reinterpret_cast<float*>(ws->records);
  out->aux = reinterpret_cast<uint32_t*>(ws->aux);
  out->counts = ws->counts;
  out->offsets = ws->offsets;
  out->keys_unsorted = ws->keys[0];
  out->vals_unsorted = ws->vals[0];
  out->keys_sorted = ws->keys[ws->sorted_in_alt];
  out->vals_sorted = ws->vals[ws->sorted_in_alt];
  out->tile_ranges = reinterpret_cast<uint32_t*>(ws->ranges);
  out->final_T = ws->final_T;
  out->n_blended = ws->n_blended;
  out->tiles_x = ws->tiles_x;
  out->tiles_y = ws->tiles_y;
  out->tile_bits = ws->have_frame ? ws->fc.tile_bits : 0;
  out->depth_shift = ws->have_frame ? ws->fc.depth_shift : 0;
  out->depth_bits = ws->have_frame ? ws->fc.depth_bits : 0;
  return AAAG_OK;
}

aaag_status aaag_preprocess(const aaag_scene* scene, const aaag_camera* camera, const aaag_params* params,
                            aaag_workspace* ws, cudaStream_t stream) {
  if (!scene || !camera || !ws) {
    set_error("aaag_preprocess: null argument");
    return AAAG_ERR_INVALID_ARG;
  }
  if (scene->n < 0 || scene->n > ws->n_max || camera->width <= 0 || camera->height <= 0 ||
      camera->width > ws->width_max || camera->height > ws->height_max) {
    set_error("aaag_preprocess: scene/camera size (%lld, %dx%d) exceeds the workspace (%lld, %dx%d)",
              (long long)scene->n, camera->width, camera->height, (long long)ws->n_max, ws->width_max,
              ws->height_max);
    return AAAG_ERR_INVALID_ARG;
  }
  {
    const aaag_status e = check_scene(scene, ws, "aaag_preprocess", false);
    if (e != AAAG_OK) return e;
  }
  if (!finite_camera(camera)) {
    set_error("aaag_preprocess: camera has non-finite or non-positive fields");
    return AAAG_ERR_INVALID_ARG;
  }
  if (params && (!(params->k >= 0.0f) || !(params->eps > 0.0f) || !(params->eps < 1.0f))) {
    set_error("aaag_preprocess: params out of range");
    return AAAG_ERR_INVALID_ARG;
  }
  // frame dimensions (at most the workspace's)
  ws->n = scene->n;
  ws->width = camera->width;
  ws->height = camera->height;
  ws->tiles_x = tiles_of(camera->width);
  ws->tiles_y = tiles_of(camera->height);
  ws->n_tiles = ws->tiles_x * ws->tiles_y;
  FrameConst fc;
  std::memset(&fc, 0, sizeof(fc));
  aaag_status e = make_frame(camera, params, scene->sh_degree, ws, &fc);
  if (e != AAAG_OK) return e;
  ws->fc = fc;
  ws->have_frame = true;
  ws->pairs_unsorted = false;
  ws->sorted_in_alt = 0;
  set_frame_kernel<<<1, 256, 0, stream>>>(ws->fc_dev, fc, ws->stats, ws->cull_lookback,
                                          (long long)ws->n_cull_words);
  e = check_launch("set_frame");
  if (e != AAAG_OK) return e;
  return launch_preprocess(scene_dev(scene), ws, stream);
}

aaag_status aaag_cull(aaag_workspace* ws, cudaStream_t stream) {
  if (!ws || !ws->have_frame) {
    set_error("aaag_cull: workspace without a preprocessed frame");
    return AAAG_ERR_INVALID_ARG;
  }
  const aaag_status e = launch_cull(ws, stream);
  ws->pairs_unsorted = e == AAAG_OK;
  return e;
}

aaag_status aaag_sort(aaag_workspace* ws, cudaStream_t stream) {
  if (!ws || !ws->have_frame) {
    set_error("aaag_sort: workspace without a preprocessed frame");
    return AAAG_ERR_INVALID_ARG;
  }
  if (!ws->pairs_unsorted) {
    // the digit histograms and tile counters of the sort are prepared by the cull
    set_error("aaag_sort: no culled pairs to sort (one aaag_sort per aaag_cull)");
    return AAAG_ERR_INVALID_ARG;
  }
  ws->pairs_unsorted = false;
  return launch_sort_pairs(ws, stream);
}

aaag_status aaag_render(aaag_workspace* ws, float* rgb, float* alpha, cudaStream_t stream) {
  if (!ws || !ws->have_frame || !rgb || !alpha) {
    set_error("aaag_render: null argument or no preprocessed frame");
    return AAAG_ERR_INVALID_ARG;
  }
  return launch_render(ws, rgb, alpha, stream);
}

aaag_status aaag_render_frame(const aaag_scene* scene, const aaag_camera* camera, const aaag_params* params,
                              aaag_workspace* ws, float* rgb, float* alpha, cudaStream_t stream) {
  aaag_status e = aaag_preprocess(scene, camera, params, ws, stream);
  if (e == AAAG_OK) e = aaag_cull(ws, stream);
  if (e == AAAG_OK) e = aaag_sort(ws, stream);
  if (e == AAAG_OK) e = aaag_render(ws, rgb, alpha, stream);
  return e;
}

aaag_status aaag_render_backward(const aaag_scene* scene, aaag_workspace* ws, const float* rgb,
                                 const float* dL_drgb, const float* dL_dalpha, const aaag_grads* grads,
                                 cudaStream_t stream) {
  if (!scene || !ws || !ws->have_frame || !rgb || !dL_drgb || !grads) {
    set_error("aaag_render_backward: null argument or no rendered frame");
    return AAAG_ERR_INVALID_ARG;
  }
  aaag_status e = check_scene(scene, ws, "aaag_render_backward", true);
  if (e != AAAG_OK) return e;
  if (scene->sh_degree != ws->fc.sh_degree) {
    set_error("aaag_render_backward: scene differs from the preprocessed one");
    return AAAG_ERR_INVALID_ARG;
  }
  if (scene->n > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits ||
                       !grads->sh)) {
    set_error("aaag_render_backward: null gradient array");
    return AAAG_ERR_INVALID_ARG;
  }
  if (ws->fc.flags & AAAG_FLAG_EVAL_2D) {
    set_error("aaag_render_backward: the 2D-evaluation ablation is forward only");
    return AAAG_ERR_UNSUPPORTED;
  }
  if (cudaMemsetAsync(ws->stats + kStatReplayMismatch, 0, 8, stream) != cudaSuccess)
    return check_launch("backward memset");
  return launch_render_backward(scene_dev(scene), ws, rgb, dL_drgb, dL_dalpha, grads, stream);
}

size_t aaag_radix_sort_scratch_bytes(int64_t n) { return n < 0 ? 0 : radix_sort_scratch(n); }

aaag_status aaag_radix_sort(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int64_t n,
                            int32_t key_bits, void* scratch, size_t scratch_bytes, int32_t* result_in_alt,
                            cudaStream_t stream) {
  if (n < 0 || n >= (1ll << 30) || key_bits < 1 || key_bits > 32 || !result_in_alt) {
    set_error("aaag_radix_sort: invalid argument");
    return AAAG_ERR_INVALID_ARG;
  }
  if (n > 0 && (!keys || !vals || !keys_alt || !vals_alt || !scratch)) {
    set_error("aaag_radix_sort: null pointer");
    return AAAG_ERR_INVALID_ARG;
  }
  if (n == 0) {
    *result_in_alt = 0;
    return AAAG_OK;
  }
  if (scratch_bytes < radix_sort_scratch(n) || ((uintptr_t)scratch) % 16) {
    set_error("aaag_radix_sort: scratch too small or unaligned (%zu < %zu)", scratch_bytes,
              radix_sort_scratch(n));
    return AAAG_ERR_CAPACITY;
  }
  // scratch layout: hist | counters | epoch | timeout | n | lookback
  char* b = static_cast<char*>(scratch);
  uint32_t* hist = reinterpret_cast<uint32_t*>(b);
  uint32_t* counters = reinterpret_cast<uint32_t*>(b + 4096);
  unsigned long long* epoch = reinterpret_cast<unsigned long long*>(b + 4096 + 64);
  unsigned long long* timeout = epoch + 1;
  uint32_t* n_dev = reinterpret_cast<uint32_t*>(epoch + 2);
  unsigned long long* lookback = reinterpret_cast<unsigned long long*>(b + 4096 + 256);
  set_u32_kernel<<<1, 1, 0, stream>>>(n_dev, (uint32_t)n);
  int alt = 0;
  const int64_t lb_words = std::max<int64_t>(sort_max_tiles(n), 1) * 256;
  const aaag_status e = radix_sort_device_n(keys, vals, keys_alt, vals_alt, n_dev, n, key_bits, hist, counters,
                                            lookback, lb_words, epoch, timeout, &alt, stream, false, true);
  *result_in_alt = alt;
  return e;
}

aaag_status aaag_get_stats(aaag_workspace* ws, aaag_stats* out, cudaStream_t stream) {
  if (!ws || !out) {
    set_error("aaag_get_stats: null argument");
    return AAAG_ERR_INVALID_ARG;
  }
  unsigned long long h[kStatCount];
  if (cudaMemcpyAsync(h, ws->stats, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return check_launch("get_stats");
  std::memset(out, 0, sizeof(*out));
  out->n_gaussians = (uint64_t)ws->n;
  out->n_visible = h[kStatVisible];
  out->n_pairs = h[kStatPairs];
  out->pair_capacity = (uint64_t)ws->capacity;
  out->tiles_tested = h[kStatTilesTested];
  out->evaluations = h[kStatEvaluations];
  out->blended = h[kStatBlended];
  out->misorders = h[kStatMisorders];
  out->extra_passes = h[kStatExtraPasses];
  out->capacity_overflow = (uint32_t)h[kStatOverflow];
  out->timeout = (uint32_t)h[kStatTimeout];
  out->replay_mismatch = h[kStatReplayMismatch];
  if (out->capacity_overflow) {
    set_error("pair capacity %lld exceeded: %llu pairs", (long long)ws->capacity, (unsigned long long)h[kStatPairs]);
    return AAAG_ERR_CAPACITY;
  }
  if (out->timeout) {
    set_error("a bounded device wait gave up");
    return AAAG_ERR_TIMEOUT;
  }
  return AAAG_OK;
}

aaag_status aaag_render_batch(aaag_workspace* const* ws, float* const* rgb, float* const* alpha, int32_t n,
                              cudaStream_t stream) {
  if (!ws || !rgb || !alpha || n < 1 || n > kMaxRenderBatch) {
    set_error("aaag_render_batch: need 1..%d frames", kMaxRenderBatch);
    return AAAG_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i) {
    if (!ws[i] || !ws[i]->have_frame || !rgb[i] || !alpha[i]) {
      set_error("aaag_render_batch: frame %d has no workspace, no sorted pairs or no output", i);
      return AAAG_ERR_INVALID_ARG;
    }
  }
  return launch_render_batch(ws, rgb, alpha, n, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// frame graphs
// ---------------------------------------------------------------------------

struct aaag_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaGraphNode_t frame_node;
  cudaKernelNodeParams frame_params;
  aaag_workspace* ws;
  aaag_params params;
  bool has_params;
  int sh_degree, width, height, stages;
  int64_t n;
  int sorted_in_alt;     // buffer of the sorted pairs after a launch
  bool pairs_unsorted;   // culled but not sorted by the captured stages
};

extern "C" {

aaag_status aaag_graph_create(const aaag_scene* scene, const aaag_camera* camera, const aaag_params* params,
                              aaag_workspace* ws, int32_t stages, float* rgb, float* alpha, cudaStream_t stream,
                              aaag_graph** out) {
  if (!scene || !camera || !ws || !out || !(stages & AAAG_STAGE_PREPROCESS) || (stages & ~15) ||
      ((stages & AAAG_STAGE_RENDER) && (!rgb || !alpha))) {
    set_error("aaag_graph_create: invalid argument");
    return AAAG_ERR_INVALID_ARG;
  }
  if (!stream) {
    set_error("aaag_graph_create: capture needs a non-default stream");
    return AAAG_ERR_INVALID_ARG;
  }
  if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return check_launch("aaag_graph_create begin capture");
  aaag_status e = aaag_preprocess(scene, camera, params, ws, stream);
  if (e == AAAG_OK && (stages & AAAG_STAGE_CULL)) e = aaag_cull(ws, stream);
  if (e == AAAG_OK && (stages & AAAG_STAGE_SORT)) e = aaag_sort(ws, stream);
  if (e == AAAG_OK && (stages & AAAG_STAGE_RENDER)) e = aaag_render(ws, rgb, alpha, stream);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(stream, &graph);
  if (e != AAAG_OK || ce != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    if (e == AAAG_OK) {
      set_error("aaag_graph_create: capture failed: %s", cudaGetErrorString(ce));
      e = AAAG_ERR_CUDA;
    }
    cudaGetLastError();
    return e;
  }
  // the frame-constant node
  size_t count = 0;
  cudaGraphGetNodes(graph, nullptr, &count);
  cudaGraphNode_t* nodes = static_cast<cudaGraphNode_t*>(std::calloc(count ? count : 1, sizeof(cudaGraphNode_t)));
  cudaGraphGetNodes(graph, nodes, &count);
  cudaGraphNode_t frame_node = nullptr;
  cudaKernelNodeParams fp;
  std::memset(&fp, 0, sizeof(fp));
  for (size_t i = 0; i < count && !frame_node; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams p;
    if (cudaGraphKernelNodeGetParams(nodes[i], &p) == cudaSuccess &&
        p.func == reinterpret_cast<void*>(set_frame_kernel)) {
      frame_node = nodes[i];
      fp = p;
    }
  }
  std::free(nodes);
  cudaGraphExec_t exec = nullptr;
  if (!frame_node || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    set_error("aaag_graph_create: %s", frame_node ? "instantiation failed" : "frame node not found");
    cudaGetLastError();
    return AAAG_ERR_CUDA;
  }
  auto* g = static_cast<aaag_graph*>(std::calloc(1, sizeof(aaag_graph)));
  if (!g) {
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    set_error("aaag_graph_create: out of host memory");
    return AAAG_ERR_CAPACITY;
  }
  g->graph = graph;
  g->exec = exec;
  g->frame_node = frame_node;
  g->frame_params = fp;
  g->ws = ws;
  g->has_params = params != nullptr;
  if (params) g->params = *params;
  g->sh_degree = scene->sh_degree;
  g->n = scene->n;
  g->width = camera->width;
  g->height = camera->height;
  g->stages = stages;
  g->sorted_in_alt = ws->sorted_in_alt;
  g->pairs_unsorted = ws->pairs_unsorted;
  *out = g;
  return AAAG_OK;
}

aaag_status aaag_graph_launch(aaag_graph* g, const aaag_camera* camera, cudaStream_t stream) {
  if (!g || !camera) {
    set_error("aaag_graph_launch: null argument");
    return AAAG_ERR_INVALID_ARG;
  }
  if (camera->width != g->width || camera->height != g->height || !finite_camera(camera)) {
    set_error("aaag_graph_launch: camera must be finite and %dx%d like the captured frame", g->width, g->height);
    return AAAG_ERR_INVALID_ARG;
  }
  aaag_workspace* ws = g->ws;
  // the workspace dimensions are those of the captured frame
  ws->n = g->n;
  ws->width = g->width;
  ws->height = g->height;
  ws->tiles_x = tiles_of(g->width);
  ws->tiles_y = tiles_of(g->height);
  ws->n_tiles = ws->tiles_x * ws->tiles_y;
  FrameConst fc;
  std::memset(&fc, 0, sizeof(fc));
  aaag_status e = make_frame(camera, g->has_params ? &g->params : nullptr, g->sh_degree, ws, &fc);
  if (e != AAAG_OK) return e;
  FrameConst* dst = ws->fc_dev;
  unsigned long long* stats = ws->stats;
  unsigned long long* cull_lb = ws->cull_lookback;
  long long lb_words = (long long)ws->n_cull_words;
  void* args[5] = {&dst, &fc, &stats, &cull_lb, &lb_words};
  cudaKernelNodeParams p = g->frame_params;
  p.kernelParams = args;
  p.extra = nullptr;
  if (cudaGraphExecKernelNodeSetParams(g->exec, g->frame_node, &p) != cudaSuccess)
    return check_launch("aaag_graph_launch update");
  if (cudaGraphLaunch(g->exec, stream) != cudaSuccess) return check_launch("aaag_graph_launch");
  ws->fc = fc;
  ws->have_frame = true;
  ws->sorted_in_alt = g->sorted_in_alt;
  ws->pairs_unsorted = g->pairs_unsorted;
  return AAAG_OK;
}

aaag_status aaag_selftest_wait_timeout(aaag_workspace* ws, int32_t which, cudaStream_t stream) {
  if (which == 2) return static_sort_wait_selftest(stream);
  if (!ws || which < 0 || which > 1) {
    set_error("aaag_selftest_wait_timeout: invalid argument");
    return AAAG_ERR_INVALID_ARG;
  }
  if (cudaMemsetAsync(ws->stats + kStatTimeout, 0, sizeof(unsigned long long), stream) != cudaSuccess)
    return check_launch("aaag_selftest_wait_timeout memset");
  return which == 0 ? launch_cull_wait_selftest(ws, stream)
                    : launch_sort_wait_selftest(ws->sort_lookback, ws->stats + kStatTimeout, stream);
}

void aaag_graph_destroy(aaag_graph* g) {
  if (!g) return;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  std::free(g);
}

}  // extern "C"
