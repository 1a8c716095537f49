/*
 * aaag.h -- C ABI of a GB300 (sm_103a) renderer for 3D-evaluated Gaussians
 * with an adaptive 3D smoothing filter, view-space bounds, 3D frustum tile
 * culling, per-pixel depth ordering and front-to-back compositing
 * (AAA-Gaussians, arXiv 2504.12811).
 *
 * Conventions shared by every call
 * --------------------------------
 * - All array pointers are DEVICE pointers owned by the caller unless a
 *   comment says "host".  Arrays are dense, C-contiguous float32 / uint32.
 * - Nothing here allocates device memory.  Per-frame storage lives in a
 *   caller-provided workspace buffer (aaag_workspace_bytes / _init).
 * - Calls are asynchronous and ordered on the given stream.  Host-side
 *   argument errors return a status immediately and launch nothing.  Errors
 *   only the device can see (pair capacity exceeded, a bounded wait that gave
 *   up) set flags in the workspace that aaag_get_stats reports; the frame is
 *   then invalid and no call traps, asserts or hangs.
 * - A workspace is used by one stream at a time.
 * - Images are planar: rgb[3][height][width], alpha[height][width]; pixel
 *   (px, py) is sampled at its centre (px + 0.5, py + 0.5).
 * - View space: x right, y down, z forward.  Pinhole cameras only (the
 *   bounding is tied to the pinhole model, paper Sec. 5).
 */
#ifndef AAAG_H_
#define AAAG_H_

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AAAG_OK = 0,
  AAAG_ERR_INVALID_ARG = 1,  /* null pointer, bad size, non-finite camera     */
  AAAG_ERR_CAPACITY = 2,     /* workspace too small (host check) or pair
                                capacity exceeded on the device              */
  AAAG_ERR_CUDA = 3,         /* a CUDA launch or copy failed                 */
  AAAG_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up           */
  AAAG_ERR_UNSUPPORTED = 5   /* e.g. SH degree > 3, image too large          */
} aaag_status;

/* Scene (paper Sec. 3.1: mean mu, scale s, rotation quaternion q, opacity;
 * view-dependent colour as real spherical harmonics; Sec. 3.2: the training
 * sampling frequency v_hat_train of the 3D smoothing filter).  Device
 * pointers, caller-owned, read only:
 *   means          [n][3]  world space
 *   log_scales     [n][3]  s = exp(log_scales)
 *   quats          [n][4]  (w, x, y, z), normalised inside
 *   opacity_logits [n]     opacity = sigmoid(logit)
 *   sh             [n][(sh_degree+1)^2][3]  coefficients, (l,m) order
 *                  (0,0),(1,-1),(1,0),(1,1),(2,-2)...; real orthonormal SH
 *                  with Condon-Shortley phase; colour = max(0, sum + 0.5)
 *   vhat_train     [n]     pixels per world unit seen in training; +inf = none
 */
typedef struct {
  int64_t n;
  int32_t sh_degree;              /* 0..3 */
  int32_t reserved;
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const float* sh;
  const float* vhat_train;
} aaag_scene;

/* Pinhole camera (paper Sec. 3.1 Eq. 4: view matrix V, projection P,
 * viewport M_vp).  Host struct, copied at call time. */
typedef struct {
  float viewmat[16];   /* world -> view, row-major 4x4, last row (0,0,0,1)  */
  float fx, fy;        /* focal lengths in pixels                           */
  float cx, cy;        /* principal point in pixels                         */
  int32_t width, height;
  float znear;         /* near plane (Sec. 3.3); e.g. 0.2                   */
  float bg[3];         /* background colour blended behind the last layer   */
} aaag_camera;

/* Method parameters. */
#define AAAG_FLAG_NO_FILTER 1u  /* ablation: no 3D smoothing filter (phi=1)  */
#define AAAG_FLAG_NO_CULL   2u  /* ablation: keep every tile of the bounds   */
/* ablation of the blending sort order (Sec. 3.1 'Blending Sort Order', the
 * sort ablation of Sec. 5): pairs are keyed by the view depth of the mean
 * (clamped to z_near) and contributors are blended in pair order, with no
 * per-pixel re-sort */
#define AAAG_FLAG_NO_RESORT 4u
/* bounded-buffer approximate re-sort (the per-ray sorting the paper retains
 * from hierarchical rasterisation): pairs are keyed by the view depth of the
 * mean (clamped to z_near), so contributors arrive in that order (ties by
 * Gaussian index); they wait in the 16-entry per-pixel buffer, ordered by
 * (t*, arrival); an arrival that finds it full blends the nearest of the
 * buffer and itself (the older on a tie), and the rest is blended nearest
 * first at the end; no release by key and no further pass, so the order is
 * exact only while the buffer never fills */
#define AAAG_FLAG_KBUFFER   8u
/* ablation without 3D evaluation (Sec. 5, 'w/o 3D'): each Gaussian is
 * splatted in 2D, its filtered covariance projected with the Jacobian of the
 * perspective map at the mean (EWA, no extra screen-space dilation); alpha =
 * min(0.99, o_hat exp(-rho^2/2)) with rho^2 the 2D Mahalanobis distance, the
 * depth of every contribution is the mean's view depth, the camera-inside
 * rule is not applied.  Forward only: aaag_render_backward returns
 * AAAG_ERR_UNSUPPORTED for a frame rendered with it. */
#define AAAG_FLAG_EVAL_2D   16u
typedef struct {
  float k;             /* filter size, Sec. 4: k = 0.3                       */
  float eps;           /* angle clamp epsilon of Sec. 3.3 Eq. 17, e.g. 1e-3  */
  uint32_t flags;      /* AAAG_FLAG_*                                        */
  int32_t reserved;
} aaag_params;

typedef struct aaag_workspace aaag_workspace;

/* Device-side frame statistics (aaag_get_stats). */
typedef struct {
  uint64_t n_gaussians;    /* n of the last preprocess                      */
  uint64_t n_visible;      /* survived discard + whole-frustum cull         */
  uint64_t n_pairs;        /* (tile, Gaussian) pairs kept by tile culling   */
  uint64_t pair_capacity;
  uint64_t tiles_tested;   /* tiles inside the bounds that were culled/kept */
  uint64_t evaluations;    /* pixel x Gaussian evaluations in aaag_render   */
  uint64_t blended;        /* contributors blended                          */
  uint64_t misorders;      /* early releases of the per-pixel buffer in the
                              bounded-buffer ablation (AAAG_FLAG_KBUFFER);
                              0 otherwise: the default order is exact       */
  uint64_t extra_passes;   /* depth-peeling passes beyond the first, summed
                              over pixels (a pixel whose buffer filled
                              defers its farthest contributors to another
                              pass over its tile)                           */
  uint64_t replay_mismatch;/* pixels whose backward replay blended a count
                              different from the forward pass (expected 0)  */
  uint32_t capacity_overflow;  /* 1 when n_pairs > pair_capacity            */
  uint32_t timeout;            /* 1 when a bounded device wait gave up       */
} aaag_stats;

/* Gradients, same layout as aaag_scene (device pointers, caller-owned,
 * overwritten). */
typedef struct {
  float* means;
  float* log_scales;
  float* quats;
  float* opacity_logits;
  float* sh;
} aaag_grads;

/* Internal arrays of a workspace, for inspection by tests and tools.  Device
 * pointers into the workspace buffer; valid until the next call that writes
 * them. */
typedef struct {
  float* records;        /* [n][16]: rows t1,t2,t3 of T_view = V T (Gaussian
                            space -> view space; t_i = (A_i0,A_i1,A_i2,mu_v,i)),
                            then (r, g, b, o_hat)                            */
  uint32_t* aux;         /* [n][4], written for visible Gaussians only:
                            inclusive pixel ranges whose centres can see the
                            Gaussian (x0 | y0<<16, x1 | y1<<16; its tiles are
                            those holding them), tau_rho float bits (negated
                            when the ellipsoid reaches znear), depth-key bits */
  uint32_t* counts;      /* [n] chunks of 32 candidate tiles per Gaussian;
                            0 = not visible                                  */
  uint32_t* offsets;     /* [n] exclusive prefix sum of counts               */
  uint32_t* keys_unsorted;   /* [capacity] pair keys as emitted              */
  uint32_t* vals_unsorted;   /* [capacity] Gaussian index per pair           */
  uint32_t* keys_sorted;     /* [capacity] after aaag_sort                   */
  uint32_t* vals_sorted;
  uint32_t* tile_ranges; /* [tiles][2] start, end of each tile's pairs       */
  float* final_T;        /* [height][width] transmittance after the last blend */
  uint32_t* n_blended;   /* [height][width] contributors blended             */
  int32_t tiles_x, tiles_y;
  int32_t tile_bits;     /* key = tile << depth_bits | depth key             */
  int32_t depth_shift;   /* depth key = (bits(z) - bits(znear)) >> shift,
                            clamped to the largest depth key                 */
  int32_t depth_bits;    /* tile_bits + depth_bits = 24 when that leaves at
                            least 16 depth bits (three radix passes), else 32 */
} aaag_workspace_view;

/* --------------------------------------------------------------------------
 * Workspace.  Bytes needed for up to n Gaussians, images up to width x height
 * and up to pair_capacity (tile, Gaussian) pairs; any smaller scene or image
 * can be rendered with it.  The caller allocates that many bytes
 * of device memory (256-byte aligned) and keeps them alive while the
 * workspace is used; _init writes a small host-side descriptor to *ws
 * (malloc'd; release with _destroy, which never frees dev_mem).
 * Errors: INVALID_ARG (null, n < 0, size <= 0), CAPACITY (bytes too small),
 * UNSUPPORTED (more than 2^16 tiles or pair_capacity >= 2^30).
 * ------------------------------------------------------------------------ */
size_t aaag_workspace_bytes(int64_t n, int32_t width, int32_t height,
                            int64_t pair_capacity);
aaag_status aaag_workspace_init(void* dev_mem, size_t bytes, int64_t n,
                                int32_t width, int32_t height,
                                int64_t pair_capacity, aaag_workspace** ws);
void aaag_workspace_destroy(aaag_workspace* ws);
aaag_status aaag_workspace_get_view(const aaag_workspace* ws,
                                    aaag_workspace_view* out /* host */);

/* --------------------------------------------------------------------------
 * aaag_preprocess -- per-Gaussian preparation for one view (Sec. 3.2, 3.3,
 * 3.4 last paragraph):
 *   s = exp(log s), R(q/|q|), o = sigmoid(logit); view mean mu_v = V mu;
 *   v_hat = fx / max(z_v, znear) (Eq. 6), v_hat' = min(v_hat_train, v_hat)
 *   (Eq. 13); s_hat_i = s_i^2 + k / v_hat'^2; amplitude factor of Eq. 12;
 *   o_hat = o * factor; tau_rho = 2 ln(255 o_hat) (alpha >= 1/255 inside);
 *   discard when o_hat <= 1/255 or the camera is inside the tau-ellipsoid;
 *   view-space angular bounds of Eq. 14-17 (for a Gaussian reaching in
 *   front of znear, intersected with the bounds of its part beyond znear)
 *   -> tile rectangle; cull against
 *   the whole image frustum truncated at znear (Eq. 18 over the image);
 *   SH colour; depth key: a lower bound of the depth t* of the maximum on
 *   every ray the Gaussian contributes to (never below the front of its
 *   tau-ellipsoid), quantised and rounded down.
 * Reads scene arrays; writes the workspace records.  scene->n, width and
 * height may be anything up to the workspace's maxima.  The frame constants
 * (camera, tiling, key layout) go to device memory through one single-thread
 * kernel, the first launch of the frame.  Resets the frame statistics.
 * Errors: INVALID_ARG, UNSUPPORTED (sh_degree > 3), CUDA.
 * ------------------------------------------------------------------------ */
aaag_status aaag_preprocess(const aaag_scene* scene /* host struct */,
                            const aaag_camera* camera /* host */,
                            const aaag_params* params /* host; NULL = defaults */,
                            aaag_workspace* ws, cudaStream_t stream);

/* --------------------------------------------------------------------------
 * aaag_cull -- 3D frustum tile culling (Sec. 3.4, Eq. 18, and the near-plane
 * tile rule of Sec. 3.3): for every tile of a visible Gaussian's rectangle,
 * keep the tile iff min over the tile's frustum (planes through the tile
 * borders) of rho^2 is below tau_rho; for a Gaussian whose tau-ellipsoid
 * reaches in front of znear, iff some point of the tile has rho^2 <= tau_rho
 * with the ray's maximum at t* >= znear (the per-pixel near-plane rule over
 * the tile's area).  Emits one (key, Gaussian index) pair per kept tile,
 * key = tile id (high bits) and the quantised depth bound (low bits; the
 * layout is in aaag_workspace_view): the larger of the Gaussian's own lower
 * bound of t* and the smallest t* over the tile's pixel centres (attained
 * at a corner), lowered by a rounding allowance and rounded down.  Also
 * empties the tile ranges that aaag_sort fills.  Pairs beyond the capacity
 * are dropped and flagged (aaag_get_stats -> capacity_overflow); a
 * look-back wait that gives up sets the timeout flag.
 * Errors: INVALID_ARG, CUDA.
 * ------------------------------------------------------------------------ */
aaag_status aaag_cull(aaag_workspace* ws, cudaStream_t stream);

/* --------------------------------------------------------------------------
 * aaag_sort -- global depth sort of the pairs (Sec. 3.1 'Blending Sort
 * Order': tile-major, front depth minor) by a stable LSD radix sort with
 * 8-bit digits and decoupled look-back (one pass per digit), then the
 * [start, end) range of each tile.  The pair count is read on the device.
 * Its counters and look-back epoch are prepared by aaag_cull, so each
 * aaag_cull allows exactly one aaag_sort.
 * Errors: INVALID_ARG (no preceding aaag_cull, or a second sort of the same
 * pairs), CUDA; a look-back wait that gives up sets the timeout flag.
 * ------------------------------------------------------------------------ */
aaag_status aaag_sort(aaag_workspace* ws, cudaStream_t stream);

/* --------------------------------------------------------------------------
 * aaag_render -- per-pixel 3D evaluation and compositing (Sec. 3.1 'Evaluation
 * in 3D'): for each pixel and each pair of its tile, the Gaussian's maximum
 * along the pixel ray rho^2 = |h1 n2 - h2 n1|^2 / |n1 x n2|^2 from the planes
 * pi' = T'^T pi_x, T'^T pi_y (Eq. 4-5) and the depth t* of that maximum;
 * alpha = min(0.99, o_hat exp(-rho^2/2)); contributors with alpha >= 1/255
 * and t* >= znear are re-sorted per pixel by t* in a 16-entry buffer that
 * releases an entry once every later pair of the tile is known to lie behind
 * it (per-ray sorting, Sec. 4 'Implementation Details'); when the buffer is
 * full the farthest contributors are deferred to another pass over the tile
 * (depth peeling), so every pixel blends in exact (t*, pair order) order;
 * front-to-back blending stops before transmittance would fall below 1e-4.
 * Writes rgb[3][H][W] = C + T * bg and alpha[H][W] = 1 - T (device,
 * caller-owned), plus final T and blended counts in the workspace.
 * Errors: INVALID_ARG (null outputs), CUDA.
 * ------------------------------------------------------------------------ */
aaag_status aaag_render(aaag_workspace* ws, float* rgb, float* alpha,
                        cudaStream_t stream);

/* --------------------------------------------------------------------------
 * aaag_render_backward -- gradients of a scalar loss L with respect to the
 * scene parameters, given dL/drgb [3][H][W] and optionally dL/dalpha [H][W]
 * (NULL = 0) for the frame last rendered with this workspace (the workspace
 * must be untouched since aaag_render).  `rgb` is that frame's output.  The
 * pass replays each pixel's blend sequence and differentiates front-to-back
 * compositing using the stored final transmittance (S_i = rgb - C_{<=i}), the
 * maximum response of Sec. 3.1 through the planes of Eq. 4-5, the filtered
 * opacity of Eq. 12-13, the activations, and the SH colour.  Discrete
 * decisions (discards, bounds, culling, the alpha and colour clamps, early
 * termination) are held fixed.  Writes every entry of *grads (device arrays,
 * caller-owned, layout of aaag_scene; zero for Gaussians not visible).
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 * ------------------------------------------------------------------------ */
aaag_status aaag_render_backward(const aaag_scene* scene /* host struct */,
                                 aaag_workspace* ws, const float* rgb,
                                 const float* dL_drgb, const float* dL_dalpha,
                                 const aaag_grads* grads /* host struct */,
                                 cudaStream_t stream);

/* Convenience: preprocess + cull + sort + render in one call. */
aaag_status aaag_render_frame(const aaag_scene* scene, const aaag_camera* camera,
                              const aaag_params* params, aaag_workspace* ws,
                              float* rgb, float* alpha, cudaStream_t stream);

/* --------------------------------------------------------------------------
 * aaag_render_batch -- the render of aaag_render for n frames (1..64) at once,
 * as one persistent launch whose blocks take (frame, tile) work items from a
 * shared counter (a serving form of Sec. 3.1 rendering: tiles of small and
 * large frames interleave on the GPU).  Each workspace must hold a sorted
 * frame (aaag_sort, possibly issued on other streams: order them before this
 * call, e.g. with events).  rgb[i], alpha[i] are device outputs of frame i
 * (layout of aaag_render).  Host arrays of n pointers.  Per-frame results are
 * identical to aaag_render's.  Errors: INVALID_ARG, CUDA.
 * ------------------------------------------------------------------------ */
aaag_status aaag_render_batch(aaag_workspace* const* ws, float* const* rgb,
                              float* const* alpha, int32_t n, cudaStream_t stream);

/* --------------------------------------------------------------------------
 * Frame graphs.  aaag_graph_create captures the listed stages of one frame
 * (AAAG_STAGE_PREPROCESS must be among them) for a fixed scene, workspace,
 * image size and parameters into a CUDA graph on `stream` (a non-default
 * stream; the stages are recorded, not run).  aaag_graph_launch runs it for
 * any camera of the same image size: only the first node, the one that writes
 * the frame constants to device memory, is re-parameterised.  The workspace
 * then holds that frame as if the stages had been called one by one.  A graph
 * is host memory (release with aaag_graph_destroy); device memory is still only
 * the caller's.  Errors: INVALID_ARG, CUDA (capture or instantiation failed).
 * ------------------------------------------------------------------------ */
#define AAAG_STAGE_PREPROCESS 1
#define AAAG_STAGE_CULL       2
#define AAAG_STAGE_SORT       4
#define AAAG_STAGE_RENDER     8
typedef struct aaag_graph aaag_graph;
aaag_status aaag_graph_create(const aaag_scene* scene, const aaag_camera* camera,
                              const aaag_params* params, aaag_workspace* ws,
                              int32_t stages, float* rgb, float* alpha,
                              cudaStream_t stream, aaag_graph** out);
aaag_status aaag_graph_launch(aaag_graph* g, const aaag_camera* camera,
                              cudaStream_t stream);
void aaag_graph_destroy(aaag_graph* g);

/* --------------------------------------------------------------------------
 * aaag_selftest_wait_timeout -- failure detection without a fault: runs one
 * of the library's bounded device-side waits against a predecessor that
 * never publishes (which = 0: the warp look-back of aaag_cull's scans;
 * which = 1: the per-digit look-back of the radix sort), on the workspace's
 * own look-back words (their first entries are cleared; later frames carry
 * new epochs and ignore them).  The wait gives up after about one second,
 * raises the workspace's timeout flag and returns, so the context stays
 * usable: aaag_get_stats then reports TIMEOUT until the next
 * aaag_preprocess resets the frame statistics.  which = 2 runs the sort's
 * wait on the fixed array of aaag_radix_sort_static instead (ws may be
 * NULL); aaag_radix_sort_static_status then reports TIMEOUT until the next
 * aaag_radix_sort_static.  Asynchronous on stream.
 * Errors: INVALID_ARG (null ws for which 0 or 1, which not 0, 1 or 2), CUDA.
 * ------------------------------------------------------------------------ */
aaag_status aaag_selftest_wait_timeout(aaag_workspace* ws, int32_t which,
                                       cudaStream_t stream);

/* --------------------------------------------------------------------------
 * aaag_radix_sort -- the stable LSD radix sort used by aaag_sort, on caller
 * arrays: sorts keys[0..n) (low `key_bits` bits significant, 1..32) and
 * carries vals along.  keys_alt / vals_alt are ping-pong buffers of n
 * elements; scratch is aaag_radix_sort_scratch_bytes(n) bytes (16-byte
 * aligned), zeroed by the caller before its first use and then kept as the
 * calls leave it (it holds the look-back words and their epoch).  The result
 * ends in (keys, vals) when the number of 8-bit passes is even, else in
 * (keys_alt, vals_alt); *result_in_alt (host) says which.  n is a host
 * value here.  Errors: INVALID_ARG, CAPACITY (scratch too small), CUDA.
 * ------------------------------------------------------------------------ */
size_t aaag_radix_sort_scratch_bytes(int64_t n);
aaag_status aaag_radix_sort(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                            uint32_t* vals_alt, int64_t n, int32_t key_bits,
                            void* scratch, size_t scratch_bytes,
                            int32_t* result_in_alt, cudaStream_t stream);

/* --------------------------------------------------------------------------
 * aaag_radix_sort_static -- the same stable radix sort for callers that
 * cannot allocate device memory: a plug-in inside a host application that
 * owns every device allocation, or a real-time loop that must not wait on the
 * allocator or fragment its pool.  (This entry point has no counterpart in
 * the paper; it is an interface convenience.)  It sorts keys[0..n) in place
 * (low `key_bits` bits significant, 1..32) and carries vals along; the caller
 * passes only these two device arrays.  Every other buffer (ping-pong copies,
 * histograms, look-back words) lives in one fixed device array inside the
 * library, sized for aaag_radix_sort_static_capacity() = 2^20 keys (about
 * 9 MB, held by every GPU that loads the library until the process exits).
 * Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 * The first call on a device resolves that array's address (once per
 * device, with the device current), so make the first call before any stream
 * capture.  All calls share the array: two calls that overlap on the GPU
 * (different streams, or different threads without ordering) race and give
 * wrong results; order them on one stream.  A look-back wait that gives up
 * leaves the output unspecified (no trap, no hang) and raises a flag in the
 * array that aaag_radix_sort_static_status reports.
 * Errors: INVALID_ARG (n < 0, key_bits out of range, null arrays),
 * CAPACITY (n > capacity), CUDA.
 * ------------------------------------------------------------------------ */
int64_t aaag_radix_sort_static_capacity(void);
aaag_status aaag_radix_sort_static(uint32_t* keys, uint32_t* vals, int64_t n,
                                   int32_t key_bits, cudaStream_t stream);
/* Outcome of the last aaag_radix_sort_static on the current device: reads the
 * timeout flag of its bounded look-back waits from the fixed array (a
 * synchronous device-to-host copy of 8 bytes; nothing is allocated).  Call it
 * after synchronising the stream of that sort.  Returns OK, TIMEOUT (a wait
 * gave up and that call's output is unspecified) or CUDA.  Each
 * aaag_radix_sort_static clears the flag when it starts. */
aaag_status aaag_radix_sort_static_status(void);

/* --------------------------------------------------------------------------
 * aaag_vhat_train -- the training sampling frequency of every Gaussian (Sec.
 * 3.2, Eq. 5): v_train = max over the training cameras of f / d, f the
 * camera's focal length in pixels (fx) and d the view depth of the mean.
 * Reading: a camera counts when the mean lies beyond its near plane and
 * projects inside its image (0 <= u <= width, 0 <= v <= height); a Gaussian
 * that no camera sees gets +inf (no clamp of the filter).
 *   means   device [n][3] float32 (the scene's means)
 *   cams    host array of n_cams cameras (copied into the launches)
 *   out     device [n] float32, written (the scene's vhat_train input)
 * Asynchronous on `stream`; n = 0 or n_cams = 0 (all +inf) are allowed.
 * Errors: INVALID_ARG (n < 0, n_cams < 0, null pointers, a non-finite or
 * degenerate camera), CUDA.
 * ------------------------------------------------------------------------ */
aaag_status aaag_vhat_train(const float* means, int64_t n, const aaag_camera* cams, int32_t n_cams,
                            float* out, cudaStream_t stream);

/* --------------------------------------------------------------------------
 * aaag_get_stats -- synchronises `stream` and copies the frame statistics to
 * *out (host).  Returns CAPACITY if the pair capacity overflowed, TIMEOUT if a
 * bounded device wait gave up, else OK.
 * ------------------------------------------------------------------------ */
aaag_status aaag_get_stats(aaag_workspace* ws, aaag_stats* out, cudaStream_t stream);

/* Text of the last host-side error on this thread (static storage). */
const char* aaag_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AAAG_H_ */
