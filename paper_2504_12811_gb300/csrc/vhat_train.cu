// Training sampling frequency of every Gaussian (Sec. 3.2, Eq. 5):
// v_train = max over the training cameras of f / d, d the view depth of the
// mean.  A camera counts when the mean lies beyond its near plane and projects
// inside its image; a Gaussian no camera sees gets +inf.  One thread per
// Gaussian; the cameras travel by value in the launch, up to kCamsPerLaunch
// per launch, and later launches fold their maximum into the earlier ones.
#include <algorithm>
#include <cmath>

#include "aaag_internal.cuh"

namespace aaag {
namespace {

constexpr int kCamsPerLaunch = 64;

struct TrainCam {
  float R[9], t[3];
  float fx, fy, cx, cy, w, h, znear;
};
struct TrainCams {
  TrainCam c[kCamsPerLaunch];
  int n;
  int first;   // first batch: initialise instead of folding
  int last;    // last batch: no camera seen -> +inf
};

__global__ void __launch_bounds__(256)
vhat_train_kernel(const float* __restrict__ means, int64_t n, const __grid_constant__ TrainCams cams,
                  float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
  float best = cams.first ? -INFINITY : out[i];   // -inf: no camera yet (+inf only after the last batch)
  for (int j = 0; j < cams.n; ++j) {
    const TrainCam& c = cams.c[j];
    const float x = fmaf(c.R[2], mz, fmaf(c.R[1], my, c.R[0] * mx)) + c.t[0];
    const float y = fmaf(c.R[5], mz, fmaf(c.R[4], my, c.R[3] * mx)) + c.t[1];
    const float z = fmaf(c.R[8], mz, fmaf(c.R[7], my, c.R[6] * mx)) + c.t[2];
    if (!(z > c.znear)) continue;
    const float u = fmaf(c.fx, x / z, c.cx), v = fmaf(c.fy, y / z, c.cy);
    if (u >= 0.0f && u <= c.w && v >= 0.0f && v <= c.h) best = fmaxf(best, c.fx / z);
  }
  out[i] = (cams.last && best == -INFINITY) ? INFINITY : best;
}

bool usable(const aaag_camera& c) {
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(c.viewmat[i])) return false;
  return std::isfinite(c.fx) && std::isfinite(c.fy) && std::isfinite(c.cx) && std::isfinite(c.cy) &&
         std::isfinite(c.znear) && c.fx > 0 && c.fy > 0 && c.znear > 0 && c.width > 0 && c.height > 0;
}

}  // namespace
}  // namespace aaag

using namespace aaag;

extern "C" aaag_status aaag_vhat_train(const float* means, int64_t n, const aaag_camera* cams, int32_t n_cams,
                                       float* out, cudaStream_t stream) {
  if (n < 0 || n_cams < 0 || (n > 0 && (!means || !out)) || (n_cams > 0 && !cams)) {
    set_error("aaag_vhat_train: negative size or null pointer");
    return AAAG_ERR_INVALID_ARG;
  }
  for (int j = 0; j < n_cams; ++j)
    if (!usable(cams[j])) {
      set_error("aaag_vhat_train: non-finite or degenerate camera");
      return AAAG_ERR_INVALID_ARG;
    }
  if (n == 0) return AAAG_OK;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  int done = 0;
  do {
    TrainCams b;
    b.n = std::min(kCamsPerLaunch, n_cams - done);
    b.first = done == 0;
    b.last = done + b.n >= n_cams;
    for (int j = 0; j < b.n; ++j) {
      const aaag_camera& c = cams[done + j];
      TrainCam& t = b.c[j];
      for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) t.R[3 * r + q] = c.viewmat[4 * r + q];
        t.t[r] = c.viewmat[4 * r + 3];
      }
      t.fx = c.fx;
      t.fy = c.fy;
      t.cx = c.cx;
      t.cy = c.cy;
      t.w = (float)c.width;
      t.h = (float)c.height;
      t.znear = c.znear;
    }
    vhat_train_kernel<<<blocks, 256, 0, stream>>>(means, n, b, out);
    const aaag_status e = check_launch("vhat_train");
    if (e != AAAG_OK) return e;
    done += b.n;
  } while (done < n_cams);
  return AAAG_OK;
}
