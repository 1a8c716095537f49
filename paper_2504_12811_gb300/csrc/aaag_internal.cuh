// Internal definitions shared by the CUDA translation units of libaaag.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "aaag.h"

namespace aaag {

constexpr int kTile = 16;                 // 16x16 pixel tiles
constexpr int kMinDepthBits = 16;         // depth-key bits below which pair keys grow to 32 bits
constexpr int kTilePixels = kTile * kTile;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;
constexpr int kMaxShDegree = 3;
constexpr int kSortItems = 8;             // keys per thread in a sort pass
constexpr int kSortThreads = 256;
constexpr int kSortTileKeys = kSortItems * kSortThreads;   // 2048: the largest sort tile
// Sorts of at least kSortWideKeys / 2 keys use 8 keys per thread, smaller ones
// 4, so that small sorts still spread over every SM (16 measured slower at
// every size: fewer blocks per SM hide less of the memory latency).
constexpr int64_t kSortWideKeys = 1 << 20;
// Most look-back tiles that a sort of up to n keys uses.
__host__ __device__ constexpr int64_t sort_max_tiles(int64_t n) {
  return ((n < kSortWideKeys / 2 ? n : kSortWideKeys / 2) + 1023) / 1024 > (n + 2047) / 2048
             ? ((n < kSortWideKeys / 2 ? n : kSortWideKeys / 2) + 1023) / 1024
             : (n + 2047) / 2048;
}
constexpr int kMaxTileBits = 16;          // at most 65536 tiles per image
// Ablations whose pairs are keyed by the view depth of the mean instead of a
// lower bound of t*, and those of them that keep every key bit (their blend
// order follows the pair order).
constexpr uint32_t kMeanDepthKeyFlags = AAAG_FLAG_NO_RESORT | AAAG_FLAG_EVAL_2D | AAAG_FLAG_KBUFFER;
constexpr uint32_t kFullKeyFlags = AAAG_FLAG_NO_RESORT | AAAG_FLAG_KBUFFER;

// Frame constants, prepared on the host in double precision and rounded once.
struct FrameConst {
  float Rv[9];          // world -> view rotation (row-major)
  float tv[3];          // world -> view translation
  float o[3];           // camera origin in world space: -Rv^-1 tv
  float fx, fy, cx, cy;
  float side[4][3];     // inward unit normals of the image frustum's side planes (view space)
  int W, H, tiles_x, tiles_y;
  float znear;
  float bg[3];
  float k;              // filter size
  float eps;            // angle clamp epsilon
  uint32_t flags;
  int tile_bits;        // bits of the tile id in a pair key
  int depth_bits;       // key_bits - tile_bits (key_bits 24 or 32)
  int depth_shift;      // depth key = (bits(z) - bits(znear)) >> depth_shift
  uint32_t znear_bits;
  int sh_degree;
};

struct SceneDev {
  int64_t n;
  int sh_degree;
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const float* sh;
  const float* vhat_train;
};

// Per-Gaussian record (64 B): rows of T_view = V T (Gaussian space -> view
// space, T = [R S' mu; 0 1], S' = diag(sqrt(s_hat))) and (r, g, b, o_hat).
struct __align__(16) Record {
  float4 t1, t2, t3;
  float4 rgba;
};

// Stats slots in the workspace (uint64 each).
enum StatSlot : int {
  kStatVisible = 0,
  kStatPairs = 1,
  kStatTilesTested = 2,
  kStatEvaluations = 3,
  kStatBlended = 4,
  kStatMisorders = 5,
  kStatOverflow = 6,
  kStatTimeout = 7,
  kStatCandidates = 8,     // uint32: Gaussians that passed the early preprocessing test (work
                           // items taken, in the fused preprocessing of a large scene)
  kStatCullTileA = 9,      // uint32 tile counters of the cull's look-back kernels
  kStatCullTileB = 10,
  kStatChunks = 11,        // chunks of 32 candidate tiles (K2 work items)
  kStatChunksClipped = 12, // uint32: chunk count clipped to the chunk capacity
  kStatPairsClipped = 13,  // uint32: pair count clipped to the pair capacity
  kStatExtraPasses = 14,   // depth-peeling passes beyond each pixel's first
  kStatFrameReset = 15,    // slots below this one are cleared at the start of every frame
  kStatReplayMismatch = 15,// pixels whose backward replay blended a different count
  kStatBatchCounter = 16,  // uint32 work-item counter of the batched render
  kStatSortEpoch = 17,
  kStatFrameEpoch = 18,    // bumped by every frame's constants: tags the cull look-back words
  kStatRenderCounter = 19, // uint32 tile counter of the persistent render
  kStatBackwardCounter = 20, // uint32 tile counter of the persistent backward
  kStatCount = 21
};


}  // namespace aaag

// Host-side workspace descriptor.
struct aaag_workspace {
  // capacity fixed at init
  int64_t n_max;
  int width_max, height_max, n_tiles_max;
  // current frame (set by aaag_preprocess)
  int64_t n;
  int width, height, tiles_x, tiles_y, n_tiles;
  int64_t capacity;
  size_t bytes;
  char* base;
  aaag::Record* records;
  uint4* aux;
  uint32_t* candidates;          // [n] Gaussians that passed the early preprocessing test
  uint32_t* counts;              // [n] chunks of 32 candidate tiles per Gaussian
  uint32_t* offsets;             // [n] exclusive prefix of counts
  int64_t chunk_capacity;
  uint32_t* chunk_owner;         // [chunk_capacity] Gaussian of each chunk
  uint32_t* chunk_mask;          // [chunk_capacity] needed-tile ballot of each chunk
  unsigned long long* cull_lookback;   // look-back words of the cull's scans
  int64_t n_cull_words;
  uint32_t* keys[2];
  uint32_t* vals[2];
  uint32_t* sort_hist;           // [4][256]
  uint32_t* sort_counters;       // [4] tile counters per pass
  unsigned long long* sort_lookback;   // [max sort tiles][256]
  uint2* ranges;                 // [n_tiles]
  uint32_t* tile_order;          // [n_tiles] render order (longest tiles first)
  float* final_T;                // [H*W]
  uint32_t* n_blended;           // [H*W]
  unsigned long long* stats;     // [kStatCount]
  float4* grad_acc;              // [n][4] backward accumulators (dt1, dt2, dt3, colour + o_hat)
  aaag::FrameConst fc;            // host copy of the current frame constants
  aaag::FrameConst* fc_dev;       // device copy read by the kernels
  bool have_frame;
  bool pairs_unsorted;           // aaag_cull emitted pairs that aaag_sort has not consumed
  int sorted_in_alt;             // which buffer holds the sorted pairs
  int64_t n_sort_tiles;
};

namespace aaag {

// ---------------------------------------------------------------------------
// host helpers (api.cu)
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
aaag_status check_launch(const char* what);

// Programmatic dependent launch along the frame's chain of kernels: each is
// launched with programmatic stream serialisation, so the next kernel's grid
// is set up while the previous one drains; its blocks start with pdl_begin,
// which waits until the previous grid has completed and its writes are
// visible (exactly the ordering of a plain launch) and then lets the next
// grid launch.  Without a programmatic dependency the wait returns at once.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                           Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// kernel launchers (one per translation unit)
aaag_status launch_preprocess(const SceneDev& s, aaag_workspace* ws, cudaStream_t st);
aaag_status launch_cull(aaag_workspace* ws, cudaStream_t st);
aaag_status launch_cull_wait_selftest(aaag_workspace* ws, cudaStream_t st);
aaag_status launch_sort_wait_selftest(unsigned long long* lookback, unsigned long long* timeout_flag,
                                      cudaStream_t st);
aaag_status static_sort_wait_selftest(cudaStream_t st);
int64_t cull_lookback_words(int64_t n, int64_t chunk_cap);
aaag_status launch_sort_pairs(aaag_workspace* ws, cudaStream_t st);
aaag_status launch_render(aaag_workspace* ws, float* rgb, float* alpha, cudaStream_t st);
// tiles of the frame in descending order of their pair counts into
// ws->tile_order; resets the work counter of the persistent kernel that uses it
aaag_status launch_tile_order(aaag_workspace* ws, uint32_t* counter, cudaStream_t st);
aaag_status launch_render_batch(aaag_workspace* const* ws, float* const* rgb, float* const* alpha, int n,
                                cudaStream_t st);
// Launch shapes that depend on the device: its SM count and the occupancy of
// the persistent kernels, queried once per device with that device current
// (thread-safe; every launcher reads the current device's entry).
struct LaunchConfig {
  int sms;
  int pre_per_sm;        // preprocess_kernel blocks per SM
  int pre_fused_per_sm;  // preprocess_fused_kernel
  int cull_a_per_sm;     // chunk_offsets_kernel
  int cull_b_per_sm;     // cull_emit_kernel
  int sort_pass_per_sm;  // sort_pass_kernel
  int sort_wide_per_sm;  // sort_pass_kernel, 12 keys per thread
  int sort_xwide_per_sm; // sort_pass_kernel_x16, 16 keys per thread
  int serve_per_sm;      // serve_render_kernel
  int backward_per_sm;   // render_backward_kernel
};
const LaunchConfig& launch_config();
// per translation unit: function attributes and occupancy of its kernels
void configure_preprocess(LaunchConfig& c);
void configure_cull(LaunchConfig& c);
void configure_sort(LaunchConfig& c);
void configure_render(LaunchConfig& c);
void configure_backward(LaunchConfig& c);
constexpr int kMaxRenderBatch = 64;
aaag_status launch_render_backward(const SceneDev& s, aaag_workspace* ws, const float* rgb, const float* drgb,
                                   const float* dalpha, const aaag_grads* out, cudaStream_t st);
aaag_status radix_sort_device_n(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                                uint32_t* vals_alt, const uint32_t* n_dev, int64_t n_max,
                                int key_bits, uint32_t* hist, uint32_t* counters,
                                unsigned long long* lookback, int64_t lookback_words,
                                unsigned long long* epoch, unsigned long long* timeout_flag,
                                int* result_in_alt, cudaStream_t st, bool prepared = false,
                                bool n_exact = false);
size_t radix_sort_scratch(int64_t n_max);

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }

}  // namespace aaag
