// Complex FP32 GEMM on the 5th-generation tensor cores (sm_103a): tcgen05.mma
// kind::tf32 with operands staged in shared memory by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) and the accumulators in TMEM.
//
// C = alpha op(A) op(B) + beta C for one complex M x N x K product is computed
// as a real product on interleaved data: A' (M x 2K) holds (re, im) of A
// along K, and the K-major B' (2N x 2K) holds, for complex column n, the rows
// 2n = (Re b, -Im b) and 2n+1 = (Im b, Re b) along K, so that
// (A' B'^T)[m, 2n] = Re c and [m, 2n+1] = Im c. Each real operand is split
// x = hi + lo with hi = tf32(x), lo = tf32(x - hi) by the preparation
// kernels; the CTA accumulates hi*hi in one TMEM accumulator and
// hi*lo + lo*hi in a second one (the tensor core aligns the addends of one
// MMA to the largest, so the small corrections keep their bits only when
// accumulated apart), and the epilogue adds them: FP32-level accuracy.
//
// One CTA of 128 threads per 128 x 128 real output tile: thread 0 issues the
// TMA loads of a 3-stage ring, thread 32 issues the MMAs (M 128, N 128, K 8
// per instruction, four per 32-wide K tile and accumulator pass), and all
// four warps read the accumulators back with tcgen05.ld (warp w owns TMEM
// lanes 32w..32w+31, i.e. output rows). Every mbarrier wait is bounded: on
// expiry the kernel records an error code, waits (bounded) for its own
// copies in flight, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qtt {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3;
constexpr int TILE_A = BM * BK * 4;                   // 16 KB
constexpr int TILE_B = BN * BK * 4;                   // 16 KB
constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;  // Ah, Al, Bh, Bl
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr unsigned WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// Wait for the phase of the given parity; false when the bounded spin ran out.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (unsigned i = 0; i < WAIT_LIMIT; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, unsigned bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
// Shared-memory operand descriptor: K-major tile with 128-byte swizzle (rows
// of 128 B, 8-row groups 1024 B apart), start address and offsets in 16-byte
// units, descriptor version 1, layout code 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(unsigned addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__device__ __forceinline__ void mma_tf32(unsigned tmem, uint64_t a, uint64_t b, unsigned idesc,
                                         unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(unsigned bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void split_tf32x2(float x, float& hi, float& lo) {
  unsigned h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  const float hf = __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hf));
  hi = hf;
  lo = __uint_as_float(l);
}

// A' split: row m, columns (2k, 2k+1) = (re, im) of op(A)[m, k]; columns
// 2K..Kp-1 are zero. Ah, Al: M x Kp, row-major.
__global__ void tc_prep_a_kernel(const Cx<float>* __restrict__ A, long long a_rs, long long a_cs,
                                 int conjA, int M, int K, int Kp, float* __restrict__ Ah,
                                 float* __restrict__ Al) {
  const long long total = (long long)M * (Kp / 2);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(e / (Kp / 2)), k = (int)(e % (Kp / 2));
    float re = 0.f, im = 0.f;
    if (k < K) {
      const Cx<float> v = A[(long long)m * a_rs + (long long)k * a_cs];
      re = v.x;
      im = conjA ? -v.y : v.y;
    }
    float h0, l0, h1, l1;
    split_tf32x2(re, h0, l0);
    split_tf32x2(im, h1, l1);
    const long long o = (long long)m * Kp + 2 * k;
    Ah[o] = h0;
    Ah[o + 1] = h1;
    Al[o] = l0;
    Al[o + 1] = l1;
  }
}

// B' split (K-major): for complex column n of op(B), row 2n = (Re b, -Im b)
// and row 2n+1 = (Im b, Re b) at columns (2k, 2k+1). Bh, Bl: 2N x Kp.
__global__ void tc_prep_b_kernel(const Cx<float>* __restrict__ B, long long b_rs, long long b_cs,
                                 int conjB, int N, int K, int Kp, float* __restrict__ Bh,
                                 float* __restrict__ Bl) {
  const long long total = (long long)N * (Kp / 2);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e / (Kp / 2)), k = (int)(e % (Kp / 2));
    float re = 0.f, im = 0.f;
    if (k < K) {
      const Cx<float> v = B[(long long)k * b_rs + (long long)n * b_cs];
      re = v.x;
      im = conjB ? -v.y : v.y;
    }
    float hr, lr, hi_, li, hn, ln;
    split_tf32x2(re, hr, lr);
    split_tf32x2(im, hi_, li);
    split_tf32x2(-im, hn, ln);
    const long long o0 = (long long)(2 * n) * Kp + 2 * k, o1 = o0 + Kp;
    Bh[o0] = hr;
    Bh[o0 + 1] = hn;
    Bl[o0] = lr;
    Bl[o0 + 1] = ln;
    Bh[o1] = hi_;
    Bh[o1 + 1] = hr;
    Bl[o1] = li;
    Bl[o1 + 1] = lr;
  }
}

struct TcEpilogue {
  Cx<float>* C;
  long long c_rs, c_cs;
  int M, N;  // complex output size
  float alpha_re, alpha_im, beta_re, beta_im;
  int use_beta;
  int* err;  // 0 on success; 1, 2, 3: a bounded wait ran out (producer, MMA, epilogue)
};

__global__ void __launch_bounds__(128, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
               const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
               int Kp, TcEpilogue ep) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);  // full[S], empty[S], done
  unsigned* tmem_slot = (unsigned*)(bars + 2 * STAGES + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;  // n0: real column
  const int ktiles = Kp / BK;
  const unsigned full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                 done = smem_u32(bars + 2 * STAGES);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // 256 TMEM columns: two 128-column FP32 accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
        smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned tmem = *tmem_slot;
  if (warp == 0 && lane == 0) {
    int issued = 0;
    bool ok = true;
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % STAGES;
      if (kt >= STAGES && !mbar_wait(empty0 + 8 * s, ((kt / STAGES) - 1) & 1)) {
        ok = false;
        break;
      }
      unsigned char* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
      tma_load_2d(smem_u32(st), &mAh, full0 + 8 * s, kt * BK, m0);
      tma_load_2d(smem_u32(st + TILE_A), &mAl, full0 + 8 * s, kt * BK, m0);
      tma_load_2d(smem_u32(st + 2 * TILE_A), &mBh, full0 + 8 * s, kt * BK, n0);
      tma_load_2d(smem_u32(st + 2 * TILE_A + TILE_B), &mBl, full0 + 8 * s, kt * BK, n0);
      issued = kt + 1;
    }
    if (!ok) {
      atomicExch(ep.err, 1);
      // the copies issued into the last stages land before the CTA exits
      for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
        mbar_wait(full0 + 8 * (kt % STAGES), (kt / STAGES) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // M 128, N 128, D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2),
    // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
    const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(BN >> 3) << 17) |
                           ((unsigned)(BM >> 4) << 24);
    bool ok = true;
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % STAGES;
      if (!mbar_wait(full0 + 8 * s, (kt / STAGES) & 1)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      unsigned char* st = smem + s * STAGE_BYTES;
      const unsigned ah = smem_u32(st), al = smem_u32(st + TILE_A);
      const unsigned bh = smem_u32(st + 2 * TILE_A), bl = smem_u32(st + 2 * TILE_A + TILE_B);
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
        const unsigned off = kk * 32;  // 8 TF32 values per MMA along K
        const unsigned acc = (kt > 0 || kk > 0) ? 1u : 0u;
        mma_tf32(tmem, smem_desc(ah + off), smem_desc(bh + off), idesc, acc);
        mma_tf32(tmem + 128, smem_desc(ah + off), smem_desc(bl + off), idesc, acc);
        mma_tf32(tmem + 128, smem_desc(al + off), smem_desc(bh + off), idesc, 1u);
      }
      mma_commit(empty0 + 8 * s);  // the stage is free once these MMAs have read it
    }
    if (!ok) atomicExch(ep.err, 2);
    mma_commit(done);  // arrives when every MMA issued above has completed
  }
  __syncwarp();
  // warp-uniform outcome, and the warp reconverged, before the .sync.aligned loads
  const bool dok = __all_sync(0xffffffffu, mbar_wait(done, 0));
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (dok) {
    const int m = m0 + warp * 32 + lane;
    const Cx<float> alpha = mk<float>(ep.alpha_re, ep.alpha_im);
    const Cx<float> beta = mk<float>(ep.beta_re, ep.beta_im);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      unsigned r0[32], r1[32];
      const unsigned ta = tmem + ((unsigned)(warp * 32) << 16) + c0;
      tmem_ld32(ta, r0);
      tmem_ld32(ta + 128, r1);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (m < ep.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = (n0 + c0) / 2 + j;
          if (n < ep.N) {
            const Cx<float> v = mk<float>(__uint_as_float(r0[2 * j]) + __uint_as_float(r1[2 * j]),
                                          __uint_as_float(r0[2 * j + 1]) +
                                              __uint_as_float(r1[2 * j + 1]));
            Cx<float>* p = ep.C + (long long)m * ep.c_rs + (long long)n * ep.c_cs;
            Cx<float> o = cmul(alpha, v);
            if (ep.use_beta) o = cadd(o, cmul(beta, *p));
            *p = o;
          }
        }
      }
    }
  } else if (threadIdx.x == 64) {
    atomicExch(ep.err, 3);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

}  // namespace tc
}  // namespace qtt
