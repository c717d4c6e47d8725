// Complex64 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// C = alpha op(A) op(B) + beta C, batched, op in {N, C}; complex64 in and out.
// Each complex product is formed as four real products (Cr += Ar Br - Ai Bi,
// Ci += Ar Bi + Ai Br; the minus comes from the MMA's negate bit) and each
// real product in split TF32 ("3xTF32": x = x_hi + x_lo with x_hi = tf32(x),
// x_lo = tf32(x - x_hi); a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi), which keeps
// float32-level accuracy with float32 accumulation in tensor memory.
//
// CTA tile: 128 rows x 128 complex columns; K in chunks of 16 complex, three
// shared-memory stages of 64 KB (planes re/im x hi/lo for A and B, K-major,
// canonical no-swizzle core-matrix layout).  Warps 0-3 load, split and store
// the operands (any op, ragged edges zero-filled), warp 4 lane 0 issues the
// MMAs (kind::tf32, M = 128, N = 128, K = 8) into two 128-column TMEM
// accumulators and commits stage releases to mbarriers; warps 4-7 drain TMEM
// (tcgen05.ld 32x32b) into shared memory and write C row-wise with alpha/beta.  Every mbarrier wait is bounded:
// on expiry the kernel records an error code and leaves after freeing TMEM.
#include <atomic>

#include "kernels.cuh"

namespace nne {

namespace tc {

constexpr int BM = 128, BN = 128, BKC = 8;        // tile rows, complex columns, complex K per chunk (one MMA K)
constexpr int STAGES = 3;                         // split-operand stages read by the MMAs
constexpr int PLANE = BM * BKC * 4;               // bytes of one 128 x 8 tf32 plane (4 KB)
constexpr int STAGE_BYTES = 8 * PLANE;            // A: ar_hi ai_hi ar_lo ai_lo, B: br_hi bi_hi br_lo bi_lo
// raw complex64 operand stages filled by cp.async: a 128 x 8 block either row-major with rows
// padded to 10 elements (80 B: 16-byte reads of 8 consecutive rows hit distinct banks) or
// k-major 8 x 128
constexpr int RAW_STAGES = 4;
constexpr int RAW_LD = BKC + 2;
constexpr int RAW_OP_BYTES = BM * RAW_LD * 8;     // 10 KB (>= the 8 KB k-major form)
constexpr int RAW_STAGE_BYTES = 2 * RAW_OP_BYTES;
constexpr int RAW_OFFSET = STAGES * STAGE_BYTES;
constexpr int SMEM_BYTES = RAW_OFFSET + RAW_STAGES * RAW_STAGE_BYTES + 1024;
constexpr long long SPIN_LIMIT = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Canonical K-major layout, no swizzle: core matrices of 8 rows x 16 bytes;
// row groups SBO = 256 B apart (8 tf32 of K per row group), K groups LBO = 128 B apart.
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128 >> 4) & 0x3FFF) << 16;   // leading byte offset (K direction)
  d |= (uint64_t)((256 >> 4) & 0x3FFF) << 32;   // stride byte offset (8-row groups)
  d |= (uint64_t)1 << 46;                       // descriptor version for tcgen05
  return d;                                     // base offset 0, no swizzle
}

// kind::tf32 instruction descriptor: D f32, A/B tf32, both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t idesc(bool negate_a) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((negate_a ? 1u : 0u) << 13) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for phase `parity`; returns false when the limit expires.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8-byte asynchronous copy global -> shared; bytes beyond src_bytes (0 or 8) are zero-filled.
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Barrier 2 over the 128 producer threads that also returns the OR of `flag` over them, so every
// producer takes the same branch afterwards.
__device__ __forceinline__ bool producers_sync_or(bool flag) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 2, 128, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)flag)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void cp_async_wait_stages() {
  asm volatile("cp.async.wait_group %0;" ::"n"(RAW_STAGES - 2) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Split four values (consecutive k of one row) into hi/lo planes, one 16-byte store each.
__device__ __forceinline__ void put4(unsigned char* st, int plane_re, int plane_im, uint32_t off, const float2* z) {
  float rh[4], rl[4], ih[4], il[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    rh[i] = tf32_rna(z[i].x);
    rl[i] = tf32_rna(z[i].x - rh[i]);
    ih[i] = tf32_rna(z[i].y);
    il[i] = tf32_rna(z[i].y - ih[i]);
  }
  *reinterpret_cast<float4*>(st + plane_re * PLANE + off) = make_float4(rh[0], rh[1], rh[2], rh[3]);
  *reinterpret_cast<float4*>(st + plane_im * PLANE + off) = make_float4(ih[0], ih[1], ih[2], ih[3]);
  *reinterpret_cast<float4*>(st + (plane_re + 2) * PLANE + off) = make_float4(rl[0], rl[1], rl[2], rl[3]);
  *reinterpret_cast<float4*>(st + (plane_im + 2) * PLANE + off) = make_float4(il[0], il[1], il[2], il[3]);
}

}  // namespace tc

template <int OPA, int OPB>
__global__ void __launch_bounds__(256, 1) cgemm_tc_kernel(int M, int N, int K, float2 alpha, const float2* __restrict__ A,
                                                          long long sA, int lda, const float2* __restrict__ B,
                                                          long long sB, int ldb, float2 beta, float2* __restrict__ C,
                                                          long long sC, int ldc, int ksplit, int kc, int* err) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grid z = matrix x K-slice; slice s covers k in [kbeg, kend) and writes its own C block
  const int zz = blockIdx.z, z = zz / ksplit, slice = zz % ksplit;
  const int kbeg = slice * kc, kend = min(K, kbeg + kc);
  A += z * sA;
  B += z * sB;
  C += zz * sC;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  const int nchunks = kend > kbeg ? (kend - kbeg + BKC - 1) / BKC : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 128);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;

  if (warp < 4) {
    // ---------------- producers (128 threads).  Raw complex64 operands of chunk c + RAW_STAGES - 1
    // are copied asynchronously while chunk c is split into hi/lo tf32 planes (thread t: tile
    // row t of A and tile column t of B); the split stages feed the MMAs through mbarriers.
    const int t = threadIdx.x;
    unsigned char* raw0 = smem + RAW_OFFSET;
    // A is "row-major" in the raw stage when its rows hold K (op N), B when its columns do (op C)
    constexpr bool A_RM = OPA == OP_N, B_RM = OPB == OP_C;
    auto issue = [&](int c) {
      if (c < nchunks) {
        const int k0 = kbeg + c * BKC;
        unsigned char* ra = raw0 + (c % RAW_STAGES) * RAW_STAGE_BYTES;
        unsigned char* rb = ra + RAW_OP_BYTES;
#pragma unroll
        for (int q8 = 0; q8 < BKC; ++q8) {
          const int q = t + 128 * q8;
          // A
          {
            int i, kk;
            if (A_RM) { i = q / BKC; kk = q % BKC; } else { kk = q / BM; i = q % BM; }
            const int gi = row0 + i, gk = k0 + kk;
            const bool ok = gi < M && gk < kend;
            const float2* src = ok ? (A_RM ? A + (long long)gi * lda + gk : A + (long long)gk * lda + gi) : A;
            const int off = A_RM ? (i * RAW_LD + kk) : (kk * BM + i);
            cp_async8(smem_u32(ra + off * 8), src, ok ? 8u : 0u);
          }
          // B
          {
            int j, kk;
            if (B_RM) { j = q / BKC; kk = q % BKC; } else { kk = q / BN; j = q % BN; }
            const int gj = col0 + j, gk = k0 + kk;
            const bool ok = gj < N && gk < kend;
            const float2* src = ok ? (B_RM ? B + (long long)gj * ldb + gk : B + (long long)gk * ldb + gj) : B;
            const int off = B_RM ? (j * RAW_LD + kk) : (kk * BN + j);
            cp_async8(smem_u32(rb + off * 8), src, ok ? 8u : 0u);
          }
        }
      }
      cp_async_commit();   // possibly empty: keeps the group count uniform
    };
    for (int c = 0; c < RAW_STAGES - 1; ++c) issue(c);
    for (int c = 0; c < nchunks; ++c) {
      cp_async_wait_stages();                           // this thread's copies of chunk c landed
      // everyone's copies landed and everyone is done reading chunk c-1; all agree on aborting
      if (producers_sync_or(*(volatile int*)&abort_flag != 0)) break;
      issue(c + RAW_STAGES - 1);                        // into the stage chunk c-1 used
      const int s = c % STAGES;
      if (c >= STAGES) {
        // one thread waits (bounded) for the MMAs to release the stage; the vote spreads the outcome
        bool ok = true;
        if (t == 0) ok = mbar_wait(&empty_bar[s], ((c / STAGES) - 1) & 1);
        if (producers_sync_or(!ok)) {
          if (t == 0) atomicExch(&abort_flag, 1);
          break;
        }
      }
      const unsigned char* ra = raw0 + (c % RAW_STAGES) * RAW_STAGE_BYTES;
      const unsigned char* rb = ra + RAW_OP_BYTES;
      float2 va[BKC], vb[BKC];
      if (A_RM) {
        const float4* r4 = reinterpret_cast<const float4*>(ra + t * RAW_LD * 8);
#pragma unroll
        for (int h = 0; h < BKC / 2; ++h) {
          const float4 x = r4[h];
          va[2 * h] = make_float2(x.x, x.y);
          va[2 * h + 1] = make_float2(x.z, x.w);
        }
      } else {
        const float2* r2 = reinterpret_cast<const float2*>(ra);
#pragma unroll
        for (int kk = 0; kk < BKC; ++kk) {
          float2 v = r2[kk * BM + t];
          v.y = -v.y;                                   // op C: conjugate
          va[kk] = v;
        }
      }
      if (B_RM) {
        const float4* r4 = reinterpret_cast<const float4*>(rb + t * RAW_LD * 8);
#pragma unroll
        for (int h = 0; h < BKC / 2; ++h) {
          const float4 x = r4[h];
          vb[2 * h] = make_float2(x.x, -x.y);           // op C: conjugate
          vb[2 * h + 1] = make_float2(x.z, -x.w);
        }
      } else {
        const float2* r2 = reinterpret_cast<const float2*>(rb);
#pragma unroll
        for (int kk = 0; kk < BKC; ++kk) vb[kk] = r2[kk * BN + t];
      }
      unsigned char* st = smem + s * STAGE_BYTES;
#pragma unroll
      for (int q = 0; q < BKC / 4; ++q) put4(st, 0, 1, core_off(t, 4 * q), &va[4 * q]);
#pragma unroll
      for (int q = 0; q < BKC / 4; ++q) put4(st + 4 * PLANE, 0, 1, core_off(t, 4 * q), &vb[4 * q]);
      fence_async_smem();
      mbar_arrive(&full_bar[s]);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == 4) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t id_pos = idesc(false), id_neg = idesc(true);
      const uint32_t d_re = tbase, d_im = tbase + BN;
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int s = c % STAGES;
        if (!mbar_wait(&full_bar[s], (c / STAGES) & 1)) {
          ok = false;
          atomicExch(&abort_flag, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
        // planes: A 0 ar_hi, 1 ai_hi, 2 ar_lo, 3 ai_lo; B 4 br_hi, 5 bi_hi, 6 br_lo, 7 bi_lo
#pragma unroll
        for (int ks = 0; ks < BKC / 8; ++ks) {
          const uint32_t ko = ks * 128 * 8;
          const uint64_t arh = smem_desc(base + 0 * PLANE + ko), aih = smem_desc(base + 1 * PLANE + ko);
          const uint64_t arl = smem_desc(base + 2 * PLANE + ko), ail = smem_desc(base + 3 * PLANE + ko);
          const uint64_t brh = smem_desc(base + 4 * PLANE + ko), bih = smem_desc(base + 5 * PLANE + ko);
          const uint64_t brl = smem_desc(base + 6 * PLANE + ko), bil = smem_desc(base + 7 * PLANE + ko);
          const uint32_t first = (c == 0 && ks == 0) ? 0u : 1u;
          // real part: Ar Br - Ai Bi
          mma_tf32(d_re, arh, brh, id_pos, first);
          mma_tf32(d_re, arh, brl, id_pos, 1u);
          mma_tf32(d_re, arl, brh, id_pos, 1u);
          mma_tf32(d_re, aih, bih, id_neg, 1u);
          mma_tf32(d_re, aih, bil, id_neg, 1u);
          mma_tf32(d_re, ail, bih, id_neg, 1u);
          // imaginary part: Ar Bi + Ai Br
          mma_tf32(d_im, arh, bih, id_pos, first);
          mma_tf32(d_im, arh, bil, id_pos, 1u);
          mma_tf32(d_im, arl, bih, id_pos, 1u);
          mma_tf32(d_im, aih, brh, id_pos, 1u);
          mma_tf32(d_im, aih, brl, id_pos, 1u);
          mma_tf32(d_im, ail, brh, id_pos, 1u);
        }
        mma_commit(&empty_bar[s]);
      }
      mma_commit(&done_bar);
    }
    __syncwarp();
  }

  if (warp >= 4) {
    // ---------------- epilogue: warp 4+e drains TMEM lanes 32e .. 32e+31 into a
    // shared-memory tile (the pipeline buffers are free once every MMA is done),
    // then the four warps write rows of C with coalesced accesses.
    const int e = warp - 4;
    if (!mbar_wait(&done_bar, 0)) atomicExch(&abort_flag, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("bar.sync 1, 128;" ::: "memory");     // every epilogue warp sees the same abort_flag
    const bool aborted = *(volatile int*)&abort_flag != 0;
    if (aborted) {
      if (threadIdx.x == 128) atomicExch(err, NNE_ERR_TIMEOUT);
    }
    {
      constexpr int LDS = BN + 1;                       // padded row stride (float2)
      float2* tile = reinterpret_cast<float2*>(smem);   // BM x LDS float2 = 132 KB
      const int r = 32 * e + lane;
      const uint32_t lane_off = (uint32_t)(32 * e) << 16;
      for (int cc = 0; cc < BN / 16 && !aborted; ++cc) {
        float re[16], im[16];
        tmem_ld16(tbase + lane_off + cc * 16, re);
        tmem_ld16(tbase + lane_off + BN + cc * 16, im);
#pragma unroll
        for (int q = 0; q < 16; ++q) tile[r * LDS + cc * 16 + q] = make_float2(re[q], im[q]);
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const bool use_beta = (beta.x != 0.f || beta.y != 0.f);
      for (int rr = e; rr < BM && !aborted; rr += 4) {
        const int i = row0 + rr;
        if (i >= M) break;
        float2* crow = C + (long long)i * ldc + col0;
        for (int q = lane; q < BN; q += 32) {
          if (col0 + q >= N) break;
          const float2 a = tile[rr * LDS + q];
          float2 v = make_float2(alpha.x * a.x - alpha.y * a.y, alpha.x * a.y + alpha.y * a.x);
          if (use_beta) {
            const float2 o = crow[q];
            v.x += beta.x * o.x - beta.y * o.y;
            v.y += beta.x * o.y + beta.y * o.x;
          }
          crow[q] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 4) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tbase));
  }
}

static int g_tc_enabled = 1;
static __device__ int g_tc_error = 0;

static int g_tma_enabled = 1;

void set_tensor_cores(int on) { g_tc_enabled = on ? 1 : 0; }
int tensor_cores_enabled() { return g_tc_enabled; }
void set_gemm_tma(int on) { g_tma_enabled = on ? 1 : 0; }
int gemm_tma_enabled() { return g_tma_enabled; }

// Device address of the tensor-core kernels' error word (per device, looked up once).
int* tc_error_ptr() {
  static std::atomic<int*> ptrs[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tc_error) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs[dev] = reinterpret_cast<int*>(p);
  }
  return ptrs[dev];
}

// C[z] = alpha sum_s P[z * S + s] + beta C[z]: the K-slices of a split GEMM added in slice order.
__global__ void __launch_bounds__(256) cgemm_split_reduce_kernel(int M, int N, int S, const float2* __restrict__ P,
                                                                 float2 alpha, float2 beta, float2* __restrict__ C,
                                                                 long long sC, int ldc) {
  const int z = blockIdx.y;
  const long long mn = (long long)M * N;
  const bool use_beta = (beta.x != 0.f || beta.y != 0.f);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < mn;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    float2 a = make_float2(0.f, 0.f);
    for (int s = 0; s < S; ++s) {
      const float2 p = P[((long long)z * S + s) * mn + idx];
      a.x += p.x;
      a.y += p.y;
    }
    float2 v = make_float2(alpha.x * a.x - alpha.y * a.y, alpha.x * a.y + alpha.y * a.x);
    float2* c = C + z * sC + (long long)i * ldc + j;
    if (use_beta) {
      const float2 o = *c;
      v.x += beta.x * o.x - beta.y * o.y;
      v.y += beta.x * o.y + beta.y * o.x;
    }
    *c = v;
  }
}

cudaError_t cgemm_split_reduce(cudaStream_t st, int M, int N, int S, const float2* P, float2 alpha, float2 beta,
                               float2* C, long long sC, int ldc, int batch) {
  const long long mn = (long long)M * N;
  const int blocks = (int)std::min<long long>((mn + 255) / 256, 2048);
  cgemm_split_reduce_kernel<<<dim3(blocks, batch), 256, 0, st>>>(M, N, S, P, alpha, beta, C, sC, ldc);
  return cudaGetLastError();
}

template <int OPA, int OPB>
static cudaError_t launch_tc(cudaStream_t st, int M, int N, int K, float2 alpha, const float2* A, long long sA, int lda,
                             const float2* B, long long sB, int ldb, float2 beta, float2* C, long long sC, int ldc,
                             int batch, int* err) {
  cudaError_t e0 = ensure_kernel_smem((const void*)cgemm_tc_kernel<OPA, OPB>, tc::SMEM_BYTES, false);
  if (e0 != cudaSuccess) return e0;
  const int tiles = ((N + tc::BN - 1) / tc::BN) * ((M + tc::BM - 1) / tc::BM) * batch;
  // split K when the tiles leave most of the 152 SMs idle and K is long: about two CTAs per SM,
  // slices of at least 256 complex K
  int S = 1;
  if (tiles < 152 && K >= 512) S = std::min(16, std::min((2 * 152 + tiles - 1) / tiles, K / 256));
  int kc = (K + S - 1) / S;
  kc = (kc + tc::BKC - 1) / tc::BKC * tc::BKC;
  S = std::max(1, (K + kc - 1) / kc);
  if (S == 1) {
    dim3 grid((N + tc::BN - 1) / tc::BN, (M + tc::BM - 1) / tc::BM, batch);
    cgemm_tc_kernel<OPA, OPB><<<grid, 256, tc::SMEM_BYTES, st>>>(M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC,
                                                                  ldc, 1, K, err);
    return cudaGetLastError();
  }
  float2* P = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&P, sizeof(float2) * (size_t)M * N * S * batch, st);
  if (e != cudaSuccess) return e;
  dim3 grid((N + tc::BN - 1) / tc::BN, (M + tc::BM - 1) / tc::BM, batch * S);
  cgemm_tc_kernel<OPA, OPB><<<grid, 256, tc::SMEM_BYTES, st>>>(M, N, K, make_float2(1.f, 0.f), A, sA, lda, B, sB,
                                                                ldb, make_float2(0.f, 0.f), P, (long long)M * N, N, S,
                                                                kc, err);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    const long long mn = (long long)M * N;
    const int blocks = (int)std::min<long long>((mn + 255) / 256, 2048);
    cgemm_split_reduce_kernel<<<dim3(blocks, batch), 256, 0, st>>>(M, N, S, P, alpha, beta, reinterpret_cast<float2*>(C),
                                                                   sC, ldc);
    e = cudaGetLastError();
  }
  cudaFreeAsync(P, st);
  return e;
}

cudaError_t cgemm_tc(cudaStream_t st, int opA, int opB, int M, int N, int K, cx<float> alpha, const cx<float>* A,
                     long long sA, int lda, const cx<float>* B, long long sB, int ldb, cx<float> beta, cx<float>* C,
                     long long sC, int ldc, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  int* err = tc_error_ptr();
  if (!err) return cudaErrorInvalidSymbol;
  ProfScope ps(st, K_GEMM_TC, 1, 8.0 * M * N * (double)K * batch);
  const float2 al = make_float2(alpha.re, alpha.im), be = make_float2(beta.re, beta.im);
  const float2* a = reinterpret_cast<const float2*>(A);
  const float2* b = reinterpret_cast<const float2*>(B);
  float2* c = reinterpret_cast<float2*>(C);
  if (opA == OP_N && opB == OP_N) return launch_tc<OP_N, OP_N>(st, M, N, K, al, a, sA, lda, b, sB, ldb, be, c, sC, ldc, batch, err);
  if (opA == OP_N && opB == OP_C) return launch_tc<OP_N, OP_C>(st, M, N, K, al, a, sA, lda, b, sB, ldb, be, c, sC, ldc, batch, err);
  if (opA == OP_C && opB == OP_N) return launch_tc<OP_C, OP_N>(st, M, N, K, al, a, sA, lda, b, sB, ldb, be, c, sC, ldc, batch, err);
  return launch_tc<OP_C, OP_C>(st, M, N, K, al, a, sA, lda, b, sB, ldb, be, c, sC, ldc, batch, err);
}

}  // namespace nne
