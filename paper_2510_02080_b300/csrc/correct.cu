// Point correction (Sec. III-C "Point Correction"): once the submap transforms
// are estimated, the global coordinates of a submap's points are regarded as
// accurate, and every point of the tracker's local sparse map that corresponds
// to a submap pixel takes that pixel's global coordinates.
//
//   k_correct   one thread per sparse point: gather the referenced submap
//               point and confidence, transform it by its submap's pose (FP32
//               from the FP32-rounded pose, the fusion's FMA order, so a
//               corrected point equals the fused point of the same pixel),
//               write it; warp-aggregated count of corrected points.
//
// Bytes per sparse point: 8 (reference) + 12 + 4 gathered + 12 read and
// written: latency-bound gathers.
#include <cfloat>

#include "common.cuh"

namespace ec3r {
namespace correct {

constexpr int THREADS = 256;

__device__ __forceinline__ bool finf(float x) { return fabsf(x) <= FLT_MAX; }

__global__ void __launch_bounds__(THREADS) k_correct(
    int64_t n_points, float* __restrict__ points, const int64_t* __restrict__ refs,
    int n_submaps, int64_t pts_per_submap, const float* __restrict__ xyz,
    const float* __restrict__ conf, const ec3r_sim3* __restrict__ poses, float thr,
    unsigned long long* __restrict__ n_corrected, unsigned* flags) {
  const int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x;
  int done = 0;
  if (i < n_points) {
    const int64_t g = refs[i];
    const int64_t total = (int64_t)n_submaps * pts_per_submap;
    if (g < -1 || g >= total) {
      atomicOr(flags, FLAG_BAD_INDEX);
    } else if (g >= 0) {
      const float c = conf[g];
      const float x0 = xyz[3 * g], x1 = xyz[3 * g + 1], x2 = xyz[3 * g + 2];
      if (c > thr && finf(x0) && finf(x1) && finf(x2)) {
        const ec3r_sim3& P = poses[g / pts_per_submap];
        float a[12];
        for (int r = 0; r < 3; ++r) {
          for (int col = 0; col < 3; ++col) a[4 * r + col] = (float)(P.s * P.R[3 * r + col]);
          a[4 * r + 3] = (float)P.t[r];
        }
        points[3 * i + 0] = fmaf(a[0], x0, fmaf(a[1], x1, fmaf(a[2], x2, a[3])));
        points[3 * i + 1] = fmaf(a[4], x0, fmaf(a[5], x1, fmaf(a[6], x2, a[7])));
        points[3 * i + 2] = fmaf(a[8], x0, fmaf(a[9], x1, fmaf(a[10], x2, a[11])));
        done = 1;
      }
    }
  }
  const unsigned cnt = __reduce_add_sync(0xffffffffu, (unsigned)done);
  if (n_corrected && (threadIdx.x & 31) == 0 && cnt) atomicAdd(n_corrected, cnt);
}

}  // namespace correct
}  // namespace ec3r

using namespace ec3r;
using namespace ec3r::correct;

extern "C" ec3r_status ec3r_correct_points(ec3r_ctx* ctx, int64_t n_points, float* d_points,
                                           const int64_t* d_refs, int n_submaps,
                                           int64_t pts_per_submap, const float* d_xyz,
                                           const float* d_conf, const ec3r_sim3* d_poses,
                                           float conf_threshold, int64_t* d_n_corrected,
                                           void* stream) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  if (n_points < 0 || n_submaps < 0 || pts_per_submap < 0)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "bad sizes");
  if (n_points == 0) return EC3R_OK;
  if (!d_points || !d_refs || (n_submaps > 0 && pts_per_submap > 0 &&
                               (!d_xyz || !d_conf || !d_poses)))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "a required pointer is NULL");
  if (conf_threshold != conf_threshold)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "conf_threshold is NaN");
  if (n_submaps > 0 && pts_per_submap > ((int64_t)1 << 62) / n_submaps)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "problem too large");
  if (n_points > ((int64_t)1 << 40))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "too many points for one call");
  EC3R_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t blocks = (n_points + THREADS - 1) / THREADS;
  traced(ctx, s, "correct_points", [&] {
    k_correct<<<(unsigned)blocks, THREADS, 0, s>>>(
        n_points, d_points, d_refs, n_submaps, pts_per_submap, d_xyz, d_conf, d_poses,
        conf_threshold, reinterpret_cast<unsigned long long*>(d_n_corrected), ctx->d_flags);
  });
  EC3R_CUDA_TRY(ctx, cudaGetLastError());
  return EC3R_OK;
}
