// Global loop retrieval over keyframe embeddings (Sec. III-D "Loop Retrieval
// and Verification"): similarities between every N-th keyframe, thresholded at
// tau_global; the neighbourhoods of the similar pairs, thresholded at
// tau_local, give the loop candidates (verified by a homography outside this
// path).
//
//   k_loop_prep     one warp per keyframe: 1 / |e_k| in FP32; the sampled
//                   keyframes' normalised embeddings rounded to BF16 (rows
//                   padded with zeros to a multiple of 128)
//   k_sim_tc        one CTA (4 warps) per 128 x 128 tile of the upper triangle
//                   of S = A A^T: the BF16 contraction on the 5th-generation
//                   tensor cores (tcgen05.mma, FP32 accumulators in tensor
//                   memory), K in chunks of 64 through a two-stage shared-memory
//                   ring whose MMAs complete on mbarriers; epilogue: tcgen05.ld
//                   of the accumulators, threshold and gap test, compaction of
//                   the coarse pairs (and optionally the tile of S)
//   k_loop_expand   one warp per coarse pair: FP32 cosines of its
//                   (2r+1) x (2r+1) neighbourhood, best pair, tau_local
//
// Waits on mbarriers are bounded; a wait that runs out sets FLAG_TIMEOUT, the
// CTA stops issuing, waits (bounded) for what it issued, frees its tensor
// memory and returns.
#include <cuda_bf16.h>

#include <cfloat>

#include "common.cuh"

namespace ec3r {
namespace loops {

constexpr int TM = 128;          // tile rows (MMA M)
constexpr int TN = 128;          // tile columns (MMA N)
constexpr int TK = 64;           // K per stage (4 MMAs of K = 16)
constexpr int STAGES = 2;
constexpr int SIM_THREADS = 128;  // 4 warps: the 128 accumulator lanes
constexpr int TILE_BYTES = TM * TK * 2;              // one operand tile, BF16
constexpr int SMEM_BYTES = STAGES * 2 * TILE_BYTES;  // 64 KB
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

// true when the barrier completed the phase of parity `parity` within the limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = smem_addr(bar);
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
  }
  return false;
}

// Shared-memory matrix descriptor: no swizzle, K-major core matrices of 8 rows
// x 16 bytes; lbo = byte step between core matrices along K, sbo = along M/N.
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
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

// Copies rows r0 .. r0 + 127, columns k0 .. k0 + 63 of A (row-major, d columns)
// into the no-swizzle K-major core-matrix layout: the 16-byte chunk (row r,
// k-chunk j) goes to ((r / 8) * 8 + j) * 128 + (r % 8) * 16.
__device__ __forceinline__ void load_tile(unsigned char* dst, const __nv_bfloat16* A, int d,
                                          int r0, int k0) {
  for (int c = threadIdx.x; c < TM * (TK / 8); c += SIM_THREADS) {
    const int r = c >> 3, j = c & 7;
    const uint4 v = *reinterpret_cast<const uint4*>(A + (int64_t)(r0 + r) * d + k0 + 8 * j);
    *reinterpret_cast<uint4*>(dst + ((r >> 3) * 8 + j) * 128 + (r & 7) * 16) = v;
  }
}

__global__ void __launch_bounds__(SIM_THREADS, 1) k_sim_tc(
    const __nv_bfloat16* __restrict__ A, int m, int d, int stride, int gap, float tau,
    int n_tiles_side, Coarse* __restrict__ out, int64_t capacity,
    unsigned long long* __restrict__ count, float* __restrict__ S_out, unsigned* flags) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[STAGES + 1];  // per-stage MMA completion, final
  __shared__ unsigned tmem_base;
  __shared__ int timed_out;
  // upper-triangle tile (bm <= bn) of linear index blockIdx.x, row-major
  int bm = 0, t = (int)blockIdx.x;
  while (t >= n_tiles_side - bm) {
    t -= n_tiles_side - bm;
    ++bm;
  }
  const int bn = bm + t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i <= STAGES; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    timed_out = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;
  const int nk = d / TK;
  bool ok = true;
  for (int kc = 0; kc < nk && ok; ++kc) {
    const int s = kc % STAGES;
    if (kc >= STAGES && !mbar_wait(&bar[s], (unsigned)((kc / STAGES - 1) & 1))) {
      if (threadIdx.x == 0) atomicOr(flags, FLAG_TIMEOUT);
      timed_out = 1;
    }
    __syncthreads();
    if (timed_out) {
      ok = false;
      break;
    }
    unsigned char* sa = smem + s * 2 * TILE_BYTES;
    unsigned char* sb = sa + TILE_BYTES;
    load_tile(sa, A, d, bm * TM, kc * TK);
    load_tile(sb, A, d, bn * TN, kc * TK);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a0 = smem_addr(sa), b0 = smem_addr(sb);
      for (int kk = 0; kk < TK / 16; ++kk) {
        // K = 16 is two core matrices along K: 256 bytes further per step
        mma_bf16(tmem, smem_desc(a0 + 256 * kk, 128, 1024), smem_desc(b0 + 256 * kk, 128, 1024),
                 (kc > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&bar[s]);
    }
  }
  // completion of everything this CTA issued
  if (threadIdx.x == 0) mma_commit(&bar[STAGES]);
  __syncthreads();
  if (!mbar_wait(&bar[STAGES], 0)) {
    if (threadIdx.x == 0) atomicOr(flags, FLAG_TIMEOUT);
    ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && !timed_out) {
    // epilogue: warp w reads accumulator lanes (rows) 32w .. 32w + 31
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
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int b = bn * TN + c0 + j;
        const float v = __uint_as_float(r[j]);
        if (S_out && a <= b && b < m) S_out[(int64_t)a * m + b] = v;
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
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN)
                 : "memory");
}

// ---------------------------------------------------------------------------
// neighbourhood of each coarse pair
// ---------------------------------------------------------------------------
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
  for (int i = max(ka - radius, 0); i <= min(ka + radius, n - 1); ++i) {
    for (int j = max(kb - radius, 0); j <= min(kb + radius, n - 1); ++j) {
      if (j - i < gap) continue;
      const float* ei = E + (int64_t)i * d;
      const float* ej = E + (int64_t)j * d;
      float s = 0.f;
      for (int k = lane; k < d; k += 32) s = fmaf(ei[k], ej[k], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      s *= inv_norm[i] * inv_norm[j];
      if (s > best) {  // first (smallest i, then j) of equal values stays
        best = s;
        bi = i;
        bj = j;
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
  const int side = (m + TM - 1) / TM;
  const int m_pad = side * TM;
  const int64_t n_tiles = (int64_t)side * (side + 1) / 2;
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
  const int64_t prep_warps = (int64_t)n + (m_pad - m);
  traced(ctx, s, "loop_prep", [&] {
    k_loop_prep<<<(unsigned)((prep_warps * 32 + 255) / 256), 256, 0, s>>>(
        d_emb, n, d, o.stride, m, m_pad, inv, A);
  });
  traced(ctx, s, "loop_sim_tc", [&] {
    k_sim_tc<<<(unsigned)n_tiles, SIM_THREADS, SMEM_BYTES, s>>>(
        A, m, d, o.stride, o.gap, o.tau_global, side, coarse, coarse_cap, cnt, d_sim,
        ctx->d_flags);
  });
  // the number of coarse pairs is on the device: a fixed grid of warps
  // strides over them
  traced(ctx, s, "loop_expand", [&] {
    k_loop_expand<<<(unsigned)(ctx->sm_count * 8), 256, 0, s>>>(
        d_emb, inv, n, d, o.stride, o.radius, o.gap, o.tau_local, coarse, cnt, coarse_cap,
        d_loops, capacity, cnt + 1, ctx->d_flags);
  });
  EC3R_CUDA_TRY(ctx, cudaGetLastError());
  return EC3R_OK;
}
