// Global loop retrieval over keyframe embeddings (Sec. III-D "Loop Retrieval
// and Verification"): similarities between every N-th keyframe, thresholded at
// tau_global; the neighbourhoods of the similar pairs, thresholded at
// tau_local, give the loop candidates (verified by a homography outside this
// path).
//
//   k_loop_prep     one warp per keyframe: 1 / |e_k| in FP32; the sampled
//                   keyframes' normalised embeddings rounded to BF16 (rows
//                   padded with zeros to a multiple of 128)
//   k_sim_tc        one CTA (4 warps) per 128 x 256 tile reaching the upper
//                   triangle of S = A A^T, two CTAs per SM: the BF16
//                   contraction on the 5th-generation tensor cores
//                   (tcgen05.mma M128 N256 K16, FP32 accumulators in 256
//                   columns of tensor memory), K in chunks of 64 through a
//                   2-stage ring of 128-byte-swizzled tiles that one thread
//                   fills by TMA (full/empty mbarriers) and another consumes
//                   by MMAs; epilogue: tcgen05.ld of the accumulators, a
//                   maximum pre-test per 32 columns, threshold and gap test,
//                   compaction of the coarse pairs (and optionally the tile of
//                   S); the other CTA of the SM multiplies meanwhile
//   k_loop_expand   one warp per coarse pair: FP32 cosines of its
//                   (2r+1) x (2r+1) neighbourhood (for r <= 3 from one read
//                   of the 2 (2r+1) rows, all products accumulated in
//                   registers), best pair, tau_local
//
// Waits on mbarriers are bounded; a wait that runs out sets FLAG_TIMEOUT, the
// CTA stops issuing, waits (bounded) for what it issued, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cfloat>

#include "common.cuh"

namespace ec3r {
namespace loops {

constexpr int TM = 128;           // tile rows (MMA M)
constexpr int TN = 256;           // tile columns (MMA N)
constexpr int TK = 64;            // K per stage: one 128-byte swizzle row, 4 MMAs of K = 16
constexpr int STAGES = 2;         // shared-memory ring (97 KB: two CTAs per SM)
constexpr int SIM_THREADS = 128;  // 4 warps: the 128 accumulator lanes
constexpr int A_BYTES = TM * TK * 2;                       // 16 KB
constexpr int B_BYTES = TN * TK * 2;                       // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;    // + alignment of the ring
constexpr long long WAIT_LIMIT = 1ll << 22;          // polls of an mbarrier

// ---------------------------------------------------------------------------
// PTX wrappers (tcgen05, mbarrier, proxy fences)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

// true when the barrier completed the phase of parity `parity` within the
// limits: WAIT_LIMIT polls and `limit` SM cycles
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit) {
  const unsigned a = smem_addr(bar);
  const long long t0 = clock64();
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) break;
  }
  return false;
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major.
constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TN >> 3) << 17) |
                           ((unsigned)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, uint64_t a, uint64_t b, unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// preparation
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_loop_prep(const float* __restrict__ E, int n, int d,
                                                   int stride, int m, int m_pad,
                                                   float* __restrict__ inv_norm,
                                                   __nv_bfloat16* __restrict__ A) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp < n) {
    const float* e = E + (int64_t)warp * d;
    float s = 0.f;
    for (int k = lane; k < d; k += 32) s = fmaf(e[k], e[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float inv = s > 0.f ? 1.f / sqrtf(s) : 0.f;
    if (lane == 0) inv_norm[warp] = inv;
    if (warp % stride == 0) {
      __nv_bfloat16* a = A + (int64_t)(warp / stride) * d;
      for (int k = lane; k < d; k += 32) a[k] = __float2bfloat16_rn(e[k] * inv);
    }
  }
  // zero rows past the samples (rows m .. m_pad - 1)
  const int pad = warp - n;
  if (pad >= 0 && pad < m_pad - m) {
    __nv_bfloat16* a = A + (int64_t)(m + pad) * d;
    for (int k = lane; k < d; k += 32) a[k] = __float2bfloat16_rn(0.f);
  }
}

// ---------------------------------------------------------------------------
// coarse similarities on the tensor cores
// ---------------------------------------------------------------------------
struct Coarse {
  int a, b;
  float s;
};

// Tests the 32 accumulator values of one thread (row a, columns b0 .. b0+31)
// and compacts the coarse pairs; the slice's maximum is tested first, so the
// per-element work only runs where a value passes tau.
__device__ __forceinline__ void emit_slice(const unsigned* r, int a, int b0, int m, int stride,
                                           int gap, float tau, Coarse* out, int64_t capacity,
                                           unsigned long long* count, float* S_out) {
  const int lane = threadIdx.x & 31;
  float mx = -FLT_MAX;
#pragma unroll
  for (int j = 0; j < 32; ++j) mx = fmaxf(mx, __uint_as_float(r[j]));
  if (S_out && a < m) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (a <= b0 + j && b0 + j < m) S_out[(int64_t)a * m + b0 + j] = __uint_as_float(r[j]);
  }
  if (!__any_sync(0xffffffffu, mx > tau)) return;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int b = b0 + j;
    const float v = __uint_as_float(r[j]);
    const bool hit = a < m && b < m && a < b && (int64_t)(b - a) * stride >= gap && v > tau;
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (!mask) continue;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (hit) {
      const unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
      if ((int64_t)slot < capacity) out[slot] = Coarse{a, b, v};
    }
  }
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle:
// rows of 64 BF16 (128 bytes), 8-row atoms 1024 bytes apart (the leading
// offset is unused in this layout); the start moves by 32 bytes per K = 16.
__device__ __forceinline__ uint64_t sw128_desc(unsigned addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

// One 128 x 256 tile of S: tiles arrive by cp.async.bulk.tensor in the
// 128-byte-swizzled K-major layout; thread 0 is the producer (one 128-row box
// of A and two of B per chunk, completing on full[s]), thread 32 issues the
// MMAs (waiting on full[s], committing to empty[s], which the producer waits on
// before refilling the stage), and all four warps read the accumulators.
__global__ void __launch_bounds__(SIM_THREADS, 2) k_sim_tc(
    const __grid_constant__ CUtensorMap tmap, int m, int d, int stride, int gap, float tau,
    int side_m, int side_n, Coarse* __restrict__ out, int64_t capacity,
    unsigned long long* __restrict__ count, float* __restrict__ S_out, unsigned* flags,
    long long limit, int no_copy) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ unsigned tmem_base;
  __shared__ int bad;  // a wait of this CTA ran out
  // tile (bm, bn) of linear index blockIdx.x: row blocks of 128, column blocks
  // of 256, only those reaching the upper triangle (bn >= bm / 2)
  int bm = 0, t = (int)blockIdx.x;
  while (t >= side_n - bm / 2) {
    t -= side_n - bm / 2;
    ++bm;
  }
  const int bn = bm / 2 + t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;
  // 1024-byte alignment of every stage (the swizzle atoms)
  const unsigned s0 = (smem_addr(smem) + 1023u) & ~1023u;
  const int nk = d / TK;
  const uint64_t tmap_addr = reinterpret_cast<uint64_t>(&tmap);
  int issued = 0;  // chunks whose copies the producer started
  if (threadIdx.x == 0) {  // producer (with no_copy, a test injection, it starts nothing)
    for (int kc = 0; kc < (no_copy ? 0 : nk); ++kc) {
      const int st = kc % STAGES;
      if (kc >= STAGES && !mbar_wait(&empty[st], (unsigned)((kc / STAGES - 1) & 1), limit)) {
        atomicOr(flags, FLAG_TIMEOUT);
        bad = 1;
        break;
      }
      const unsigned dst = s0 + st * STAGE_BYTES;
      const unsigned fb = smem_addr(&full[st]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                   "r"(STAGE_BYTES)
                   : "memory");
      const int k0 = kc * TK;
      const int rows[3] = {bm * TM, bn * TN, bn * TN + 128};
      const unsigned dsts[3] = {dst, dst + A_BYTES, dst + A_BYTES + A_BYTES};
      for (int q = 0; q < 3; ++q)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
            "[%0], [%1, {%2, %3}], [%4];" ::"r"(dsts[q]),
            "l"(tmap_addr), "r"(k0), "r"(rows[q]), "r"(fb)
            : "memory");
      issued = kc + 1;
    }
  } else if (threadIdx.x == 32) {  // MMA issuer
    bool ok = true;
    for (int kc = 0; kc < nk && ok; ++kc) {
      const int st = kc % STAGES;
      if (!mbar_wait(&full[st], (unsigned)((kc / STAGES) & 1), limit)) {
        atomicOr(flags, FLAG_TIMEOUT);
        bad = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a0 = s0 + st * STAGE_BYTES, b0 = a0 + A_BYTES;
      for (int kk = 0; kk < TK / 16; ++kk)  // K = 16: 32 bytes along the swizzled row
        mma_bf16(tmem, sw128_desc(a0 + 32 * kk), sw128_desc(b0 + 32 * kk),
                 (kc > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[st]);
    }
    mma_commit(&done);  // completion of every MMA issued
  }
  __syncwarp();
  if (!mbar_wait(&done, 0, limit)) {
    if (threadIdx.x == 0) atomicOr(flags, FLAG_TIMEOUT);
    bad = 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (bad && threadIdx.x == 0)  // the copies still in flight land before the CTA exits
    for (int kc = max(issued - STAGES, 0); kc < issued; ++kc)
      mbar_wait(&full[kc % STAGES], (unsigned)((kc / STAGES) & 1), limit);
  if (!bad) {
    const int a = bm * TM + 32 * warp + lane;
    for (int c0 = 0; c0 < TN; c0 += 32) {
      unsigned r[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
          "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
          "%26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
            "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
            "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
            "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
            "=r"(r[30]), "=r"(r[31])
          : "r"(tmem + ((unsigned)(32 * warp) << 16) + (unsigned)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      emit_slice(r, a, bn * TN + c0, m, stride, gap, tau, out, capacity, count, S_out);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN)
                 : "memory");
}

// 2-D tensor map of A (BF16 [rows][d]) with 64 x 128 boxes and the 128-byte
// swizzle, or false when the driver cannot encode it.
static bool encode_tmap(CUtensorMap* map, const void* A, int rows, int d) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      return false;
    }
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)d * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TK, 128};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(A), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// neighbourhood of each coarse pair
// ---------------------------------------------------------------------------
// R >= 0: the radius is R; each lane reads float4 slices of the 2R+1 rows
// around a*stride and the 2R+1 rows around b*stride once and accumulates all
// (2R+1)^2 products (rows past the end read as zeros and are never chosen).
// R < 0: any radius, one pair of rows at a time.
template <int R>
__global__ void __launch_bounds__(256) k_loop_expand(
    const float* __restrict__ E, const float* __restrict__ inv_norm, int n, int d, int stride,
    int radius, int gap, float tau, const Coarse* __restrict__ coarse,
    const unsigned long long* __restrict__ n_coarse, int64_t coarse_cap,
    ec3r_loop* __restrict__ loops, int64_t capacity, unsigned long long* __restrict__ count,
    unsigned* flags) {
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nc = (int64_t)*n_coarse;
  if (w0 == 0 && lane == 0 && nc > coarse_cap) atomicOr(flags, FLAG_CAPACITY);
  for (int64_t w = w0; w < (nc < coarse_cap ? nc : coarse_cap); w += nw) {
    const Coarse c = coarse[w];
    const int ka = c.a * stride, kb = c.b * stride;
    float best = -FLT_MAX;
    int bi = -1, bj = -1;
    if constexpr (R >= 0) {
      constexpr int NR = 2 * R + 1;
      const int i0 = max(ka - R, 0), j0 = max(kb - R, 0);
      const int ni = min(ka + R, n - 1) - i0 + 1, nj = min(kb + R, n - 1) - j0 + 1;
      float acc[NR][NR];
#pragma unroll
      for (int p = 0; p < NR; ++p)
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[p][q] = 0.f;
      for (int k = 4 * lane; k < d; k += 128) {
        float4 x[NR], y[NR];
#pragma unroll
        for (int p = 0; p < NR; ++p) {
          x[p] = p < ni ? __ldg(reinterpret_cast<const float4*>(E + (int64_t)(i0 + p) * d + k))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
          y[p] = p < nj ? __ldg(reinterpret_cast<const float4*>(E + (int64_t)(j0 + p) * d + k))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int p = 0; p < NR; ++p)
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            float t = acc[p][q];
            t = fmaf(x[p].x, y[q].x, t);
            t = fmaf(x[p].y, y[q].y, t);
            t = fmaf(x[p].z, y[q].z, t);
            acc[p][q] = fmaf(x[p].w, y[q].w, t);
          }
      }
#pragma unroll
      for (int p = 0; p < NR; ++p)
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          float t = acc[p][q];
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          const int i = i0 + p, j = j0 + q;
          if (p < ni && q < nj && j - i >= gap) {
            t *= inv_norm[i] * inv_norm[j];
            if (t > best) {  // first (smallest i, then j) of equal values stays
              best = t;
              bi = i;
              bj = j;
            }
          }
        }
    } else {
      for (int i = max(ka - radius, 0); i <= min(ka + radius, n - 1); ++i) {
        for (int j = max(kb - radius, 0); j <= min(kb + radius, n - 1); ++j) {
          if (j - i < gap) continue;
          const float* ei = E + (int64_t)i * d;
          const float* ej = E + (int64_t)j * d;
          float t = 0.f;
          for (int k = lane; k < d; k += 32) t = fmaf(ei[k], ej[k], t);
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          t *= inv_norm[i] * inv_norm[j];
          if (t > best) {
            best = t;
            bi = i;
            bj = j;
          }
        }
      }
    }
    if (lane == 0 && bi >= 0 && best > tau) {
      const unsigned long long slot = atomicAdd(count, 1ull);
      if ((int64_t)slot < capacity) loops[slot] = ec3r_loop{c.a, c.b, bi, bj, c.s, best};
      else atomicOr(flags, FLAG_CAPACITY);
    }
  }
}

}  // namespace loops
}  // namespace ec3r

using namespace ec3r;
using namespace ec3r::loops;

extern "C" ec3r_status ec3r_loop_candidates(ec3r_ctx* ctx, const float* d_emb, int n, int d,
                                            const ec3r_loop_opts* opts, ec3r_loop* d_loops,
                                            int64_t capacity, int64_t* d_counts,
                                            float* d_sim, void* stream) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  if (!opts || !d_emb || !d_counts || (capacity > 0 && !d_loops))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "a required pointer is NULL");
  if (n < 0 || d <= 0 || d % TK != 0 || capacity < 0 || (int64_t)n * d >= ((int64_t)1 << 40))
    return set_error(ctx, EC3R_ERR_INVALID_ARG,
                     "bad sizes (n %d, d %d: d must be a positive multiple of %d)", n, d, TK);
  const ec3r_loop_opts o = *opts;
  if (o.stride < 1 || o.radius < 0 || o.gap < 1 || !(o.tau_global == o.tau_global) ||
      !(o.tau_local == o.tau_local))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "bad ec3r_loop_opts");
  EC3R_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  EC3R_CUDA_TRY(ctx, cudaMemsetAsync(d_counts, 0, 2 * sizeof(int64_t), s));
  if (n == 0) return EC3R_OK;
  const int m = (n + o.stride - 1) / o.stride;
  const int side_n = (m + TN - 1) / TN;  // column blocks of 256
  const int side_m = 2 * side_n;         // row blocks of 128
  const int m_pad = side_n * TN;
  int64_t n_tiles = 0;                   // row block bm meets column blocks bm / 2 ..
  for (int bm = 0; bm < side_m; ++bm) n_tiles += side_n - bm / 2;
  if (n_tiles >= ((int64_t)1 << 31))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "too many keyframes for one call");
  // coarse-pair buffer: grows with the problem, at least 1 M entries
  const int64_t coarse_cap = std::max<int64_t>((int64_t)1 << 20, 64 * (int64_t)m);
  void *p_a, *p_inv, *p_c;
  ec3r_status st;
  if ((st = ensure_buf(ctx, "loops.a", sizeof(__nv_bfloat16) * (size_t)m_pad * d, s, &p_a)))
    return st;
  if ((st = ensure_buf(ctx, "loops.inv", sizeof(float) * (size_t)n, s, &p_inv))) return st;
  if ((st = ensure_buf(ctx, "loops.coarse", sizeof(Coarse) * (size_t)coarse_cap, s, &p_c)))
    return st;
  __nv_bfloat16* A = (__nv_bfloat16*)ctx->bufs["loops.a"].ptr;
  float* inv = (float*)ctx->bufs["loops.inv"].ptr;
  Coarse* coarse = (Coarse*)ctx->bufs["loops.coarse"].ptr;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(d_counts);
  static bool attr_set[64] = {};
  if (ctx->device < 64 && !attr_set[ctx->device]) {
    EC3R_CUDA_TRY(ctx, cudaFuncSetAttribute(k_sim_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            SMEM_BYTES));
    attr_set[ctx->device] = true;
  }
  CUtensorMap tmap;
  if (!encode_tmap(&tmap, A, m_pad, d))
    return set_error(ctx, EC3R_ERR_CUDA, "cuTensorMapEncodeTiled failed for the %d x %d matrix",
                     m_pad, d);
  const int64_t prep_warps = (int64_t)n + (m_pad - m);
  traced(ctx, s, "loop_prep", [&] {
    k_loop_prep<<<(unsigned)((prep_warps * 32 + 255) / 256), 256, 0, s>>>(
        d_emb, n, d, o.stride, m, m_pad, inv, A);
  });
  traced(ctx, s, "loop_sim_tc", [&] {
    k_sim_tc<<<(unsigned)n_tiles, SIM_THREADS, SMEM_BYTES, s>>>(
        tmap, m, d, o.stride, o.gap, o.tau_global, side_m, side_n, coarse, coarse_cap, cnt, d_sim,
        ctx->d_flags, wait_limit_cycles(ctx), (ctx->inject & EC3R_INJECT_LOOPS_NO_COPY) ? 1 : 0);
  });
  // the number of coarse pairs is on the device: a fixed grid of warps
  // strides over them
  traced(ctx, s, "loop_expand", [&] {
    const bool vec = ((uintptr_t)d_emb & 15) == 0;
    const unsigned g = (unsigned)(ctx->sm_count * 8);
#define EC3R_EXPAND(R)                                                                      \
  k_loop_expand<R><<<g, 256, 0, s>>>(d_emb, inv, n, d, o.stride, o.radius, o.gap,           \
                                     o.tau_local, coarse, cnt, coarse_cap, d_loops, capacity, \
                                     cnt + 1, ctx->d_flags)
    if (vec && o.radius == 0) EC3R_EXPAND(0);
    else if (vec && o.radius == 1) EC3R_EXPAND(1);
    else if (vec && o.radius == 2) EC3R_EXPAND(2);
    else if (vec && o.radius == 3) EC3R_EXPAND(3);
    else EC3R_EXPAND(-1);
#undef EC3R_EXPAND
  });
  EC3R_CUDA_TRY(ctx, cudaGetLastError());
  return EC3R_OK;
}
