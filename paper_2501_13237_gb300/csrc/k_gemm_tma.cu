// Complex64 GEMM on the 5th-generation tensor cores, operands fed by TMA
// (tcgen05 + cp.async.bulk.tensor, sm_103a).
//
// C = alpha op(A) op(B) + beta C, batched, op in {N, C}, complex64 in and out.
//
// Complex product as one real GEMM.  With a(i,k) = op(A)[i][k] and b(k,j) =
// op(B)[k][j], the real matrices
//   A'[i][2k] = Re a(i,k),  A'[i][2k+1] = Im a(i,k)                 (M x 2K)
//   B'[2j][2k] = Re b,  B'[2j][2k+1] = -Im b,
//   B'[2j+1][2k] = Im b, B'[2j+1][2k+1] = Re b   (b = b(k,j))       (2N x 2K)
// give C'[i][2j] + i C'[i][2j+1] = sum_k a(i,k) b(k,j) for C' = A' B'^T, which
// is C itself in interleaved complex64 storage.  Both are stored K-major, each
// as two TF32 planes (x = x_hi + x_lo, x_hi = tf32(x), x_lo = tf32(x - x_hi)),
// written once per operand by split kernels; the product takes the three
// terms hi.hi + hi.lo + lo.hi ("3xTF32"), float32-level accuracy with float32
// accumulation in tensor memory.
//
// Tile: 128 rows x 256 real columns (128 complex), K in stages of 32 floats
// (one 128-byte swizzle row).  Warp 0 lane 0 issues the TMA loads of a stage
// (A hi/lo 128 x 32, B hi/lo 256 x 32, 128-byte swizzle) against an
// mbarrier's transaction count; warp 1 lane 0 issues 12 MMAs per stage
// (kind::tf32, M = 128, N = 256, K = 8) into a 256-column TMEM accumulator and
// commits the stage back to the producer; warps 2-5 drain TMEM through shared
// memory to coalesced rows of C with alpha and beta.  Every mbarrier wait is
// bounded: on expiry the kernel records NNE_ERR_TIMEOUT, waits (bounded) for
// the copies it issued, frees TMEM and returns.  The tensor maps cover this
// GPU's own memory only; there is no multicast.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace nne {

namespace tg {

constexpr int BM = 128, BN = 256;
constexpr int THREADS = 192;
constexpr int TMEM_COLS = BN;
constexpr int EPI_LD = BN + 4;                       // floats per epilogue row in shared memory
constexpr long long SPIN_LIMIT = 1LL << 26;

// Pipeline shapes: SWZ-byte swizzled rows of BK = SWZ / 4 floats per stage;
// 128-byte rows in 2 stages of 96 KB, or 64-byte rows in 4 stages of 48 KB.
template <int SWZ>
struct Pipe {
  static constexpr int BK = SWZ / 4;
  static constexpr int STAGES = SWZ == 128 ? 2 : 4;
  static constexpr int A_PLANE = BM * BK * 4;
  static constexpr int B_PLANE = BN * BK * 4;
  static constexpr int STAGE = 2 * A_PLANE + 2 * B_PLANE;
  static constexpr int SMEM = STAGES * STAGE + 1024;
  static_assert(BM * EPI_LD * 4 <= STAGES * STAGE, "epilogue tile reuses the pipeline buffers");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major operand in SWZ-byte-swizzled rows (8-row atoms of 8 SWZ bytes):
// start address, leading offset unused (1), stride between 8-row groups
// 8 SWZ bytes, descriptor version 1, layout type 2 (128-byte swizzle) or 4
// (64-byte swizzle).
template <int SWZ>
__device__ __forceinline__ uint64_t desc_sw(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((8 * SWZ) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(SWZ == 128 ? 2 : 4) << 61;
  return d;
}

// kind::tf32: D f32, A/B tf32, both K-major, M = 128, N = 256.
__host__ __device__ constexpr uint32_t idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = SPIN_LIMIT) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
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

// 3-D tiled TMA load (x = K float, y = row, z = plane) into shared memory,
// completing bytes on the mbarrier.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
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

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tg

// ---------------------------------------------------------------- operand splits
// Planes buffer of one operand: [z][plane hi, lo][row][ldp] floats.

// A' rows i < M from op(A) (M x K complex): A' (i, 2k..2k+1) = (Re, Im) a(i, k).
// 32 x 32 complex tiles through shared memory (op C reads A transposed).
template <int OP>
__global__ void __launch_bounds__(256) split_a_kernel(const float2* __restrict__ A, long long sA, int lda, int M, int K,
                                                      float* __restrict__ P, int ldp) {
  __shared__ float2 t[32][33];
  const int z = blockIdx.z;
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  A += z * sA;
  float* Phi = P + (long long)z * 2 * M * ldp;
  float* Plo = Phi + (long long)M * ldp;
  if (OP == OP_N) {
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r, k = k0 + tx;
      if (i < M && k < K) {
        const float2 a = A[(long long)i * lda + k];
        const float rh = tg::tf32_rna(a.x), ih = tg::tf32_rna(a.y);
        *reinterpret_cast<float2*>(Phi + (long long)i * ldp + 2 * k) = make_float2(rh, ih);
        *reinterpret_cast<float2*>(Plo + (long long)i * ldp + 2 * k) =
            make_float2(tg::tf32_rna(a.x - rh), tg::tf32_rna(a.y - ih));
      }
    }
  } else {
    // a(i, k) = conj(A[k][i])
    for (int r = ty; r < 32; r += 8) {
      const int k = k0 + r, i = i0 + tx;
      t[r][tx] = (k < K && i < M) ? A[(long long)k * lda + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r, k = k0 + tx;
      if (i < M && k < K) {
        const float2 v = t[tx][r];
        const float re = v.x, im = -v.y;
        const float rh = tg::tf32_rna(re), ih = tg::tf32_rna(im);
        *reinterpret_cast<float2*>(Phi + (long long)i * ldp + 2 * k) = make_float2(rh, ih);
        *reinterpret_cast<float2*>(Plo + (long long)i * ldp + 2 * k) =
            make_float2(tg::tf32_rna(re - rh), tg::tf32_rna(im - ih));
      }
    }
  }
}

// B' rows 2j, 2j+1 (j < N) from op(B) (K x N complex):
//   B'(2j, 2k..2k+1) = (Re b, -Im b),  B'(2j+1, 2k..2k+1) = (Im b, Re b),  b = b(k, j).
// op N reads B transposed through shared memory.
template <int OP>
__global__ void __launch_bounds__(256) split_b_kernel(const float2* __restrict__ B, long long sB, int ldb, int K, int N,
                                                      float* __restrict__ P, int ldp) {
  __shared__ float2 t[32][33];
  const int z = blockIdx.z;
  const int j0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  B += z * sB;
  const long long rows = 2LL * N;
  float* Phi = P + (long long)z * 2 * rows * ldp;
  float* Plo = Phi + rows * ldp;
  auto put = [&](int j, int k, float re, float im) {
    const float rh = tg::tf32_rna(re), ih = tg::tf32_rna(im);
    const float rl = tg::tf32_rna(re - rh), il = tg::tf32_rna(im - ih);
    const long long o0 = (2LL * j) * ldp + 2 * k, o1 = o0 + ldp;
    // -Im b is exactly -(Im b)_hi - (Im b)_lo: tf32 rounding is symmetric
    *reinterpret_cast<float2*>(Phi + o0) = make_float2(rh, -ih);
    *reinterpret_cast<float2*>(Plo + o0) = make_float2(rl, -il);
    *reinterpret_cast<float2*>(Phi + o1) = make_float2(ih, rh);
    *reinterpret_cast<float2*>(Plo + o1) = make_float2(il, rl);
  };
  if (OP == OP_C) {
    // b(k, j) = conj(B[j][k]): rows of B run along k
    for (int r = ty; r < 32; r += 8) {
      const int j = j0 + r, k = k0 + tx;
      if (j < N && k < K) {
        const float2 v = B[(long long)j * ldb + k];
        put(j, k, v.x, -v.y);
      }
    }
  } else {
    for (int r = ty; r < 32; r += 8) {
      const int k = k0 + r, j = j0 + tx;
      t[r][tx] = (k < K && j < N) ? B[(long long)k * ldb + j] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int j = j0 + r, k = k0 + tx;
      if (j < N && k < K) {
        const float2 v = t[tx][r];
        put(j, k, v.x, v.y);
      }
    }
  }
}

// ---------------------------------------------------------------- the GEMM
// grid (ceil(2N / BN), ceil(M / BM), batch * ksplit); slice s of K covers the
// real range [s kc, (s + 1) kc) and writes its own C block (zz = z ksplit + s).
template <int SWZ>
__global__ void __launch_bounds__(tg::THREADS, 1)
    cgemm_tma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N2,
                     int Kp, int ksplit, int kc, float2 alpha, float2 beta, float2* __restrict__ C, long long sC,
                     int ldc, int* err, long long wait_limit) {
  using namespace tg;
  constexpr int BK = Pipe<SWZ>::BK, STAGES = Pipe<SWZ>::STAGES, A_PLANE = Pipe<SWZ>::A_PLANE,
                B_PLANE = Pipe<SWZ>::B_PLANE, STAGE = Pipe<SWZ>::STAGE;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, issued_s, consumed_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int zz = blockIdx.z, z = zz / ksplit, slice = zz % ksplit;
  const int kbeg = slice * kc, kend = min(Kp, kbeg + kc);
  const int nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  C += zz * sC;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    issued_s = 0;
    consumed_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int issued = 0;
      for (int c = 0; c < nk; ++c) {
        const int s = c % STAGES;
        if (c >= STAGES && !mbar_wait(&empty_bar[s], ((c / STAGES) - 1) & 1, wait_limit)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int*)&abort_flag) break;
        unsigned char* st = smem + s * STAGE;
        const int k0 = kbeg + c * BK;
        mbar_expect_tx(&full_bar[s], STAGE);
        tma_load_3d(smem_u32(st), &tmA, k0, row0, 2 * z, &full_bar[s]);
        tma_load_3d(smem_u32(st + A_PLANE), &tmA, k0, row0, 2 * z + 1, &full_bar[s]);
        tma_load_3d(smem_u32(st + 2 * A_PLANE), &tmB, k0, col0, 2 * z, &full_bar[s]);
        tma_load_3d(smem_u32(st + 2 * A_PLANE + B_PLANE), &tmB, k0, col0, 2 * z + 1, &full_bar[s]);
        issued = c + 1;
      }
      issued_s = issued;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issue
      const uint32_t id = idesc_tf32();
      int consumed = 0;
      for (int c = 0; c < nk; ++c) {
        const int s = c % STAGES;
        if (!mbar_wait(&full_bar[s], (c / STAGES) & 1, wait_limit)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        consumed = c + 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_u32(smem + s * STAGE);
        const uint32_t a_hi = base, a_lo = base + A_PLANE, b_hi = base + 2 * A_PLANE, b_lo = b_hi + B_PLANE;
#pragma unroll
        for (int kk = 0; kk < BK / 8; ++kk) {
          const uint32_t ko = kk * 32;   // 8 tf32 = 32 bytes along the swizzled row
          const uint32_t first = (c == 0 && kk == 0) ? 0u : 1u;
          mma_tf32(tbase, desc_sw<SWZ>(a_hi + ko), desc_sw<SWZ>(b_hi + ko), id, first);
          mma_tf32(tbase, desc_sw<SWZ>(a_hi + ko), desc_sw<SWZ>(b_lo + ko), id, 1u);
          mma_tf32(tbase, desc_sw<SWZ>(a_lo + ko), desc_sw<SWZ>(b_hi + ko), id, 1u);
        }
        mma_commit(&empty_bar[s]);
      }
      consumed_s = consumed;
      mma_commit(&done_bar);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 2-5): TMEM lanes 32 (warp % 4) .. + 31
    const int q = warp & 3;
    const bool ok = nk == 0 || mbar_wait(&done_bar, 0, wait_limit);
    if (!ok) atomicExch(&abort_flag, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const bool aborted = *(volatile int*)&abort_flag != 0;
    if (aborted && threadIdx.x == 64) atomicExch(err, NNE_ERR_TIMEOUT);
    float* tile = reinterpret_cast<float*>(smem);
    const int r = 32 * q + lane;
    if (!aborted) {
      const uint32_t lane_off = (uint32_t)(32 * q) << 16;
      for (int cc = 0; cc < BN / 16; ++cc) {
        float v[16];
        if (nk > 0) tmem_ld16(tbase + lane_off + cc * 16, v);
        else
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 16; i += 4)
          *reinterpret_cast<float4*>(tile + r * EPI_LD + cc * 16 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
      }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (!aborted) {
      const bool use_beta = (beta.x != 0.f || beta.y != 0.f);
      const int e = threadIdx.x - 64;        // 0 .. 127
      const int cw = BN / 2;                 // complex columns of the tile
      const int ccol0 = col0 / 2, ncol = N2 / 2;
      for (int rr = e / 32; rr < BM; rr += 4) {
        const int i = row0 + rr;
        if (i >= M) break;
        float2* crow = C + (long long)i * ldc + ccol0;
        for (int jj = lane; jj < cw; jj += 32) {
          if (ccol0 + jj >= ncol) break;
          const float2 a = *reinterpret_cast<const float2*>(tile + rr * EPI_LD + 2 * jj);
          float2 v = make_float2(alpha.x * a.x - alpha.y * a.y, alpha.x * a.y + alpha.y * a.x);
          if (use_beta) {
            const float2 o = crow[jj];
            v.x += beta.x * o.x - beta.y * o.y;
            v.y += beta.x * o.y + beta.y * o.x;
          }
          crow[jj] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *(volatile int*)&abort_flag) {
    // after an expired wait: copies issued but never consumed still land in
    // shared memory, and issued MMAs still use tensor memory; wait for both
    // (with the full bound) before leaving
    for (int c = consumed_s; c < issued_s; ++c) mbar_wait(&full_bar[c % STAGES], (c / STAGES) & 1);
    if (nk > 0) mbar_wait(&done_bar, 0);
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(TMEM_COLS));
  }
}

// ---------------------------------------------------------------- host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of a planes buffer: x = real K (kdim valid floats, row pitch ldp),
// y = rows, z = 2 x batch planes; box (swz / 4) x box_rows x 1 with a swz-byte
// swizzle, zero fill outside (rows >= rows_valid or x >= kdim).
cudaError_t make_map(CUtensorMap* map, float* base, int kdim, int ldp, int rows, int planes, int box_rows, int swz) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)kdim, (cuuint64_t)rows, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)ldp * 4, (cuuint64_t)ldp * 4 * (cuuint64_t)rows};
  const cuuint32_t box[3] = {(cuuint32_t)(swz / 4), (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

// Pipeline variant of the TMA kernel: 1 = 128-byte rows, 2 stages; 2 = 64-byte rows, 4 stages
// (the default: about 10 % faster on the gate step's shapes).
static int g_tma_variant = 2;
void set_tma_variant(int v) { g_tma_variant = v == 2 ? 2 : 1; }

// Bound of the pipeline's mbarrier waits (test hook): > 0 polls, 0 the default
// 2^26 polls, < 0 expire without polling (deterministic, for tests).
static long long g_wait_limit = 0;
void set_tc_wait_limit(long long polls) { g_wait_limit = polls; }

bool cgemm_tma_available() { return encode_fn() != nullptr; }

// A operands split ahead of their GEMMs (tma_hold_a), per host thread: a
// matrix that several GEMMs read unchanged (the two-site matrix X in the
// subspace iteration) is split once instead of once per product.
namespace {
struct HeldPlanes {
  const void* A;
  int op, M, K, lda, batch;
  long long sA;
  cudaStream_t st;
  float* planes;
};
thread_local std::vector<HeldPlanes> g_held;

int plane_pitch(int K) { return (2 * K + 3) / 4 * 4; }   // real K, row pitch a 16-byte multiple

cudaError_t split_a(cudaStream_t st, int opA, int M, int K, const float2* a, long long sA, int lda, int batch,
                    float* PA) {
  ProfScope pss(st, K_ELEMWISE);
  dim3 ga((K + 31) / 32, (M + 31) / 32, batch);
  if (opA == OP_N) split_a_kernel<OP_N><<<ga, 256, 0, st>>>(a, sA, lda, M, K, PA, plane_pitch(K));
  else split_a_kernel<OP_C><<<ga, 256, 0, st>>>(a, sA, lda, M, K, PA, plane_pitch(K));
  return cudaGetLastError();
}
}  // namespace

cudaError_t tma_hold_a(cudaStream_t st, int opA, int M, int K, const cx<float>* A, long long sA, int lda, int batch) {
  float* p = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&p, sizeof(float) * (size_t)2 * M * plane_pitch(K) * batch, st);
  if (e != cudaSuccess) return e;
  e = split_a(st, opA, M, K, reinterpret_cast<const float2*>(A), sA, lda, batch, p);
  if (e != cudaSuccess) {
    cudaFreeAsync(p, st);
    return e;
  }
  g_held.push_back(HeldPlanes{A, opA, M, K, lda, batch, sA, st, p});
  return cudaSuccess;
}

void tma_release(cudaStream_t st) {
  for (size_t i = 0; i < g_held.size();) {
    if (g_held[i].st == st) {
      cudaFreeAsync(g_held[i].planes, st);
      g_held.erase(g_held.begin() + i);
    } else {
      ++i;
    }
  }
}

cudaError_t cgemm_tma(cudaStream_t st, int opA, int opB, int M, int N, int K, cx<float> alpha, const cx<float>* A,
                      long long sA, int lda, const cx<float>* B, long long sB, int ldb, cx<float> beta, cx<float>* C,
                      long long sC, int ldc, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  int* err = tc_error_ptr();
  if (!err) return cudaErrorInvalidSymbol;
  const int swz = g_tma_variant == 2 ? 64 : 128;
  const void* kern = swz == 128 ? (const void*)cgemm_tma_kernel<128> : (const void*)cgemm_tma_kernel<64>;
  const int smem = swz == 128 ? tg::Pipe<128>::SMEM : tg::Pipe<64>::SMEM;
  const int BK = swz / 4;
  cudaError_t e = ensure_kernel_smem(kern, smem, false);
  if (e != cudaSuccess) return e;
  const int Kr = 2 * K;                             // real K
  const int ldp = plane_pitch(K);
  const int N2 = 2 * N;
  float* held = nullptr;
  for (const HeldPlanes& h : g_held)
    if (h.A == A && h.op == opA && h.M == M && h.K == K && h.lda == lda && h.sA == sA && h.batch == batch && h.st == st)
      held = h.planes;
  const size_t a_floats = held ? 0 : (size_t)2 * M * ldp * batch, b_floats = (size_t)2 * N2 * ldp * batch;
  float* planes = nullptr;
  if ((e = cudaMallocAsync((void**)&planes, sizeof(float) * (a_floats + b_floats) + 1024, st)) != cudaSuccess) return e;
  float* PA = held ? held : planes;
  float* PB = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(planes + a_floats) + 255) & ~uintptr_t(255));
  // (pad columns of the pitch lie outside the tensor maps' extent: the loads fill zeros there)
  const float2* b = reinterpret_cast<const float2*>(B);
  if (!held) e = split_a(st, opA, M, K, reinterpret_cast<const float2*>(A), sA, lda, batch, PA);
  if (e == cudaSuccess) {
    ProfScope pss(st, K_ELEMWISE);
    dim3 gb((K + 31) / 32, (N + 31) / 32, batch);
    if (opB == OP_N) split_b_kernel<OP_N><<<gb, 256, 0, st>>>(b, sB, ldb, K, N, PB, ldp);
    else split_b_kernel<OP_C><<<gb, 256, 0, st>>>(b, sB, ldb, K, N, PB, ldp);
    e = cudaGetLastError();
  }
  CUtensorMap mA, mB;
  if (e == cudaSuccess) e = make_map(&mA, PA, Kr, ldp, M, 2 * batch, tg::BM, swz);
  if (e == cudaSuccess) e = make_map(&mB, PB, Kr, ldp, N2, 2 * batch, tg::BN, swz);
  if (e == cudaSuccess) {
    ProfScope ps(st, K_GEMM_TC, 1, 8.0 * M * N * (double)K * batch);
    const int tiles = ((N2 + tg::BN - 1) / tg::BN) * ((M + tg::BM - 1) / tg::BM) * batch;
    // split K when the tiles leave most of the 152 SMs idle and K is long
    int S = 1;
    if (tiles < 152 && Kr >= 1024) S = std::min(16, std::min((2 * 152 + tiles - 1) / tiles, Kr / 512));
    int kc = (Kr + S - 1) / S;
    kc = (kc + BK - 1) / BK * BK;
    S = std::max(1, (Kr + kc - 1) / kc);
    const float2 al = make_float2(alpha.re, alpha.im), be = make_float2(beta.re, beta.im);
    const long long wl = g_wait_limit > 0 ? g_wait_limit : (g_wait_limit < 0 ? 0 : tg::SPIN_LIMIT);
    dim3 grid((N2 + tg::BN - 1) / tg::BN, (M + tg::BM - 1) / tg::BM, batch * S);
    auto launch = [&](int ks, int kcl, float2 a, float2 bt, float2* out, long long so, int ldo) {
      if (swz == 128)
        cgemm_tma_kernel<128><<<grid, tg::THREADS, smem, st>>>(mA, mB, M, N2, Kr, ks, kcl, a, bt, out, so, ldo, err, wl);
      else
        cgemm_tma_kernel<64><<<grid, tg::THREADS, smem, st>>>(mA, mB, M, N2, Kr, ks, kcl, a, bt, out, so, ldo, err, wl);
      return cudaGetLastError();
    };
    if (S == 1) {
      e = launch(1, Kr, al, be, reinterpret_cast<float2*>(C), sC, ldc);
    } else {
      float2* P = nullptr;
      e = cudaMallocAsync((void**)&P, sizeof(float2) * (size_t)M * N * S * batch, st);
      if (e == cudaSuccess) {
        e = launch(S, kc, make_float2(1.f, 0.f), make_float2(0.f, 0.f), P, (long long)M * N, N);
        if (e == cudaSuccess) e = cgemm_split_reduce(st, M, N, S, P, al, be, reinterpret_cast<float2*>(C), sC, ldc, batch);
        cudaFreeAsync(P, st);
      }
    }
  }
  cudaFreeAsync(planes, st);
  return e;
}

}  // namespace nne
