// Device kernels of the QTT homogenisation library (sm_103a).
//
// Complex numbers are interleaved (re, im) pairs of R = double (FP64 mode) or
// float (FP32 mode). Matrices are addressed through (row stride, column
// stride) pairs so that one GEMM kernel serves every contraction of the
// tensor-train sweeps without explicit transposes.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qtt {

template <typename R>
struct alignas(2 * sizeof(R)) Cx {
  R x, y;
};

template <typename R>
__host__ __device__ __forceinline__ Cx<R> mk(R a, R b) {
  Cx<R> c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename R>
__device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename R>
__device__ __forceinline__ Cx<R> csub(Cx<R> a, Cx<R> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename R>
__device__ __forceinline__ Cx<R> cmulc(Cx<R> a, Cx<R> b) {
  return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename R>
__device__ __forceinline__ Cx<R> cconj(Cx<R> a) { return mk(a.x, -a.y); }
template <typename R>
__device__ __forceinline__ R cabs2(Cx<R> a) { return a.x * a.x + a.y * a.y; }
template <typename R>
__device__ __forceinline__ Cx<R> cscale(Cx<R> a, R s) { return mk(a.x * s, a.y * s); }

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename R>
__device__ __forceinline__ Cx<R> warp_sum(Cx<R> v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}

// ------------------------------------------------------------------ GEMM
// C[b] = alpha * op(A)[b] * op(B)[b] + beta * C[b] for a 3-level batch
// (b1, b2, b3) and an optional split of K over `ksplit` CTAs (then beta must
// be 0, C must be zeroed by the caller and partial sums are added atomically).
struct GemmArgs {
  int M, N, K;
  const void* A;
  long long a_rs, a_cs, a_b1, a_b2, a_b3;
  const void* B;
  long long b_rs, b_cs, b_b1, b_b2, b_b3;
  void* C;
  long long c_rs, c_cs, c_b1, c_b2, c_b3;
  int nb1, nb2, nb3, ksplit;
  int conjA, conjB;
  double alpha_re, alpha_im, beta_re, beta_im;
  // split-K without atomics: with ksplit > 1 and part != nullptr each split
  // writes alpha * (its partial product) to part[((ks * nbatch + b) * M + m) * N
  // + n] and splitk_reduce_kernel sums the splits in a fixed order.
  void* part;
};

template <typename R, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_kernel(GemmArgs g) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ Cx<R> As[BK][BM + 1];
  __shared__ Cx<R> Bs[BK][BN + 1];
  int z = blockIdx.z;
  const int ks = z % g.ksplit;
  z /= g.ksplit;
  const int b3 = z % g.nb3;
  z /= g.nb3;
  const int b2 = z % g.nb2;
  const int b1 = z / g.nb2;
  const Cx<R>* A = (const Cx<R>*)g.A + b1 * g.a_b1 + b2 * g.a_b2 + b3 * g.a_b3;
  const Cx<R>* B = (const Cx<R>*)g.B + b1 * g.b_b1 + b2 * g.b_b2 + b3 * g.b_b3;
  Cx<R>* C = (Cx<R>*)g.C + b1 * g.c_b1 + b2 * g.c_b2 + b3 * g.c_b3;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  // K range of this split
  const int kchunk = ((g.K + g.ksplit - 1) / g.ksplit + BK - 1) / BK * BK;
  const int kbeg = ks * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const int tid = threadIdx.x;
  const int tr = tid / (BN / TN), tc = tid % (BN / TN);
  Cx<R> acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = mk<R>(0, 0);
  const bool a_mfast = (g.a_rs == 1);
  const bool b_nfast = (g.b_cs == 1);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int e = tid; e < BM * BK; e += NT) {
      int mm, kk;
      if (a_mfast) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      Cx<R> v = mk<R>(0, 0);
      if (gm < g.M && gk < kend) {
        v = A[(long long)gm * g.a_rs + (long long)gk * g.a_cs];
        if (g.conjA) v.y = -v.y;
      }
      As[kk][mm] = v;
    }
    for (int e = tid; e < BK * BN; e += NT) {
      int kk, nn;
      if (b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      const int gk = k0 + kk, gn = n0 + nn;
      Cx<R> v = mk<R>(0, 0);
      if (gk < kend && gn < g.N) {
        v = B[(long long)gk * g.b_rs + (long long)gn * g.b_cs];
        if (g.conjB) v.y = -v.y;
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Cx<R> a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tr + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tc + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
  const Cx<R> alpha = mk<R>((R)g.alpha_re, (R)g.alpha_im);
  const Cx<R> beta = mk<R>((R)g.beta_re, (R)g.beta_im);
  const bool use_beta = (g.beta_re != 0.0 || g.beta_im != 0.0);
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + tr + i * (BM / TM);
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tc + j * (BN / TN);
      if (gn >= g.N) continue;
      Cx<R>* p = C + (long long)gm * g.c_rs + (long long)gn * g.c_cs;
      Cx<R> v = cmul(alpha, acc[i][j]);
      if (g.part) {
        const long long nbat = (long long)g.nb1 * g.nb2 * g.nb3;
        const long long bidx = ((long long)b1 * g.nb2 + b2) * g.nb3 + b3;
        ((Cx<R>*)g.part)[(((long long)ks * nbat + bidx) * g.M + gm) * g.N + gn] = v;
      } else if (g.ksplit > 1) {
        atomicAdd(&p->x, v.x);
        atomicAdd(&p->y, v.y);
      } else {
        if (use_beta) v = cadd(v, cmul(beta, *p));
        *p = v;
      }
    }
  }
}

// ------------------------------------------------------------------ split-TF32 tensor-core GEMM
// Complex FP32 GEMM on the tensor cores (mma.sync m16n8k8, TF32 inputs, FP32
// accumulation) with split precision: each real operand x = hi + lo with
// hi = tf32(x), lo = tf32(x - hi), and each real product taken as
// hi*hi + hi*lo + lo*hi (the dropped lo*lo term is ~2^-22 relative, the
// level of FP32 rounding). The complex product is four real products:
// re = Ar Br - Ai Bi, im = Ar Bi + Ai Br, i.e. 12 MMAs per k-step and tile.
// The hi*hi products and the ~2^-11 smaller correction products go to
// separate accumulators, summed in the epilogue: the tensor core aligns the
// addends of one MMA to the largest before adding, so corrections added into
// the hi*hi accumulator would lose their low bits.
// Same arguments, batching, split-K and epilogue as gemm_kernel<float>.
// Tile 64 x 64 x 8, four warps of 32 x 32 outputs each.
__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = f32_to_tf32(x);
  lo = f32_to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) gemm_tf32x3_kernel(GemmArgs g) {
  constexpr int BM = 64, BN = 64, BK = 8;
  __shared__ float Ar[BK][BM + 4], Ai[BK][BM + 4];
  __shared__ float Br[BK][BN + 4], Bi[BK][BN + 4];
  int z = blockIdx.z;
  const int ks = z % g.ksplit;
  z /= g.ksplit;
  const int b3 = z % g.nb3;
  z /= g.nb3;
  const int b2 = z % g.nb2;
  const int b1 = z / g.nb2;
  const Cx<float>* A = (const Cx<float>*)g.A + b1 * g.a_b1 + b2 * g.a_b2 + b3 * g.a_b3;
  const Cx<float>* B = (const Cx<float>*)g.B + b1 * g.b_b1 + b2 * g.b_b2 + b3 * g.b_b3;
  Cx<float>* C = (Cx<float>*)g.C + b1 * g.c_b1 + b2 * g.c_b2 + b3 * g.c_b3;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kchunk = ((g.K + g.ksplit - 1) / g.ksplit + BK - 1) / BK * BK;
  const int kbeg = ks * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gq = lane >> 2, tq = lane & 3;              // group, thread in group
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // warp tile origin
  float accr[2][4][4], acci[2][4][4];  // hi*hi products
  float corr[2][4][4], cori[2][4][4];  // hi*lo and lo*hi corrections
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) accr[i][j][q] = acci[i][j][q] = corr[i][j][q] = cori[i][j][q] = 0.f;
  const bool a_mfast = (g.a_rs == 1);
  const bool b_nfast = (g.b_cs == 1);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 128) {
      int mm, kk;
      if (a_mfast) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      Cx<float> v = mk<float>(0, 0);
      if (gm < g.M && gk < kend) {
        v = A[(long long)gm * g.a_rs + (long long)gk * g.a_cs];
        if (g.conjA) v.y = -v.y;
      }
      Ar[kk][mm] = v.x;
      Ai[kk][mm] = v.y;
    }
    for (int e = tid; e < BK * BN; e += 128) {
      int kk, nn;
      if (b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      const int gk = k0 + kk, gn = n0 + nn;
      Cx<float> v = mk<float>(0, 0);
      if (gk < kend && gn < g.N) {
        v = B[(long long)gk * g.b_rs + (long long)gn * g.b_cs];
        if (g.conjB) v.y = -v.y;
      }
      Br[kk][nn] = v.x;
      Bi[kk][nn] = v.y;
    }
    __syncthreads();
    // A fragments (16 x 8, row-major): a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4)
    uint32_t arh[2][4], arl[2][4], aih[2][4], ail[2][4], anh[2][4], anl[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = wm + i * 16 + gq;
      const float xr[4] = {Ar[tq][r], Ar[tq][r + 8], Ar[tq + 4][r], Ar[tq + 4][r + 8]};
      const float xi[4] = {Ai[tq][r], Ai[tq][r + 8], Ai[tq + 4][r], Ai[tq + 4][r + 8]};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        split_tf32(xr[q], arh[i][q], arl[i][q]);
        split_tf32(xi[q], aih[i][q], ail[i][q]);
        split_tf32(-xi[q], anh[i][q], anl[i][q]);
      }
    }
    // B fragments (8 x 8, k x n): b0 (k = t, n = g), b1 (k = t+4, n = g)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = wn + j * 8 + gq;
      uint32_t brh[2], brl[2], bih[2], bil[2];
      split_tf32(Br[tq][c], brh[0], brl[0]);
      split_tf32(Br[tq + 4][c], brh[1], brl[1]);
      split_tf32(Bi[tq][c], bih[0], bil[0]);
      split_tf32(Bi[tq + 4][c], bih[1], bil[1]);
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        // re += Ar Br - Ai Bi
        mma_tf32(accr[i][j], arh[i], brh);
        mma_tf32(accr[i][j], anh[i], bih);
        mma_tf32(corr[i][j], arh[i], brl);
        mma_tf32(corr[i][j], arl[i], brh);
        mma_tf32(corr[i][j], anh[i], bil);
        mma_tf32(corr[i][j], anl[i], bih);
        // im += Ar Bi + Ai Br
        mma_tf32(acci[i][j], arh[i], bih);
        mma_tf32(acci[i][j], aih[i], brh);
        mma_tf32(cori[i][j], arh[i], bil);
        mma_tf32(cori[i][j], arl[i], bih);
        mma_tf32(cori[i][j], aih[i], brl);
        mma_tf32(cori[i][j], ail[i], brh);
      }
    }
    __syncthreads();
  }
  const Cx<float> alpha = mk<float>((float)g.alpha_re, (float)g.alpha_im);
  const Cx<float> beta = mk<float>((float)g.beta_re, (float)g.beta_im);
  const bool use_beta = (g.beta_re != 0.0 || g.beta_im != 0.0);
  // accumulator (16 x 8): c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1)
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gm = m0 + wm + i * 16 + gq + (q >= 2 ? 8 : 0);
        const int gn = n0 + wn + j * 8 + 2 * tq + (q & 1);
        if (gm >= g.M || gn >= g.N) continue;
        Cx<float>* p = C + (long long)gm * g.c_rs + (long long)gn * g.c_cs;
        Cx<float> v = cmul(alpha, mk<float>(accr[i][j][q] + corr[i][j][q],
                                            acci[i][j][q] + cori[i][j][q]));
        if (g.part) {
          const long long nbat = (long long)g.nb1 * g.nb2 * g.nb3;
          const long long bidx = ((long long)b1 * g.nb2 + b2) * g.nb3 + b3;
          ((Cx<float>*)g.part)[(((long long)ks * nbat + bidx) * g.M + gm) * g.N + gn] = v;
        } else if (g.ksplit > 1) {
          atomicAdd(&p->x, v.x);
          atomicAdd(&p->y, v.y);
        } else {
          if (use_beta) v = cadd(v, cmul(beta, *p));
          *p = v;
        }
      }
}

// C = sum over the ks splits of part (fixed order) + beta C, for the batch
// and strides of the GEMM that wrote part (layout in GemmArgs::part).
template <typename R>
__global__ void splitk_reduce_kernel(const Cx<R>* __restrict__ part, int ks, long long nbat, int M,
                                     int N, int nb2, int nb3, Cx<R>* C, long long c_rs,
                                     long long c_cs, long long c_b1, long long c_b2,
                                     long long c_b3, double beta_re, double beta_im) {
  const long long per = (long long)M * N, tot = nbat * per;
  const Cx<R> beta = mk<R>((R)beta_re, (R)beta_im);
  const bool use_beta = (beta_re != 0.0 || beta_im != 0.0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    Cx<R> s = part[e];
    for (int k = 1; k < ks; ++k) s = cadd(s, part[e + k * tot]);
    const long long bidx = e / per, r = e - bidx * per;
    const long long gm = r / N, gn = r - gm * N;
    const long long b3 = bidx % nb3, t = bidx / nb3;
    const long long b2 = t % nb2, b1 = t / nb2;
    Cx<R>* p = C + b1 * c_b1 + b2 * c_b2 + b3 * c_b3 + gm * c_rs + gn * c_cs;
    if (use_beta) s = cadd(s, cmul(beta, *p));
    *p = s;
  }
}

// ------------------------------------------------------------------ block reduction helper
template <typename R>
__device__ R block_sum(R v, R* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  R t = (threadIdx.x < nw) ? sh[threadIdx.x] : (R)0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  R r = sh[0];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------ Householder QR
// One CTA factors the m x n matrix A (element (i, j) at A[i*rs + j*cs],
// conjugated when conjA) as A = Q R with k = min(m, n): Q is m x k with
// orthonormal columns (column-major, ld m), R is k x n upper trapezoidal
// (column-major, ld k). Reflectors H = I - h v v^H with v = x - beta e1 and
// beta = -phase(x0) ||x||, applied to the trailing columns column by column;
// Q is accumulated backwards from [I; 0]. W (m x n) is workspace.
template <typename R>
__global__ void qr_kernel(int m, int n, const Cx<R>* __restrict__ A, long long rs, long long cs,
                          int conjA, Cx<R>* Wg, Cx<R>* Q, Cx<R>* Rm, R* hbuf, Cx<R>* vhead,
                          int use_smem) {
  // the working copy lives in dynamic shared memory when it fits
  extern __shared__ __align__(16) unsigned char qr_dyn[];
  Cx<R>* W = use_smem ? (Cx<R>*)qr_dyn : Wg;
  __shared__ R red[32];
  __shared__ Cx<R> s_v0;
  __shared__ R s_h;
  const int tid = threadIdx.x, nt = blockDim.x;
  // lanes per column in the trailing updates: with the matrix in shared
  // memory, the largest power of two <= 32 that gives every column its own
  // group (at least 4 lanes); from global memory, whole warps (more loads in
  // flight per column beat more columns in flight)
  int G = 32;
  if (use_smem)
    while (G > 4 && (nt / G) < n) G >>= 1;
  const int gid = tid / G, gl = tid % G, ngroups = nt / G;
  for (long long e = tid; e < (long long)m * n; e += nt) {
    const int i = (int)(e % m), j = (int)(e / m);
    Cx<R> v = A[(long long)i * rs + (long long)j * cs];
    if (conjA) v.y = -v.y;
    W[e] = v;
  }
  __syncthreads();
  // a column at the rounding-noise floor of the matrix (|x|^2 <= eps^2
  // ||A||_F^2) is treated as zero (R_jj = 0, no reflector): reflecting it
  // would divide by a norm that can underflow single precision
  R f2 = 0;
  for (long long e = tid; e < (long long)m * n; e += nt) f2 += cabs2(W[e]);
  f2 = block_sum(f2, red);
  const double eps_r = sizeof(R) == 8 ? 2.220446049250313e-16 : 1.1920928955078125e-7;
  const double negl = eps_r * eps_r * (double)f2;
  const int k = min(m, n);
  for (int j = 0; j < k; ++j) {
    Cx<R>* col = W + (long long)j * m;
    R s2 = 0;
    for (int i = j + tid; i < m; i += nt) s2 += cabs2(col[i]);
    s2 = block_sum(s2, red);
    const double s2d = (double)s2;
    if (tid == 0) {
      const Cx<R> a = col[j];
      const R s = sqrt(s2);
      if (!(s2d > negl) || s == (R)0) {
        s_h = 0;
        s_v0 = mk<R>(0, 0);
        col[j] = mk<R>(0, 0);
      } else {
        // hypot keeps |phase| = 1 when |a| is tiny (no underflow of |a|^2)
        const R aa = hypot(a.x, a.y);
        const Cx<R> ph = aa > (R)0 ? mk<R>(a.x / aa, a.y / aa) : mk<R>(1, 0);
        const Cx<R> beta = mk<R>(-ph.x * s, -ph.y * s);
        const Cx<R> v0 = csub(a, beta);
        const double vtv = s2d - (double)aa * aa + (double)v0.x * v0.x + (double)v0.y * v0.y;
        const double hd = 2.0 / vtv;
        if (!(hd < (sizeof(R) == 8 ? 1e300 : 1e30))) {  // a matrix at the underflow edge
          s_h = 0;
          s_v0 = mk<R>(0, 0);
          col[j] = mk<R>(0, 0);
        } else {
          s_h = (R)hd;
          s_v0 = v0;
          col[j] = beta;
        }
      }
      hbuf[j] = s_h;
      vhead[j] = s_v0;
    }
    __syncthreads();
    const R h = s_h;
    const Cx<R> v0 = s_v0;
    if (h != (R)0) {
      // one group of G lanes per trailing column (uniform loop: every lane
      // takes part in the shuffles)
      for (int c0 = j + 1; c0 < n; c0 += ngroups) {
        const int c = c0 + gid;
        const bool valid = c < n;
        Cx<R>* a = W + (long long)(valid ? c : j) * m;
        Cx<R> w = mk<R>(0, 0);
        if (valid) {
          if (gl == 0) w = cmulc(v0, a[j]);
          for (int i = j + 1 + gl; i < m; i += G) w = cadd(w, cmulc(col[i], a[i]));
        }
        for (int o = G >> 1; o > 0; o >>= 1) {
          w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
          w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
        }
        if (!valid) continue;
        const Cx<R> hw = cscale(w, h);
        if (gl == 0) a[j] = csub(a[j], cmul(hw, v0));
        for (int i = j + 1 + gl; i < m; i += G) a[i] = csub(a[i], cmul(hw, col[i]));
      }
    }
    __syncthreads();
  }
  // R (k x n)
  for (long long e = tid; e < (long long)k * n; e += nt) {
    const int i = (int)(e % k), j = (int)(e / k);
    Rm[e] = (i <= j) ? W[(long long)j * m + i] : mk<R>(0, 0);
  }
  // Q = H_0 ... H_{k-1} [I; 0]
  for (long long e = tid; e < (long long)m * k; e += nt) {
    const int i = (int)(e % m), j = (int)(e / m);
    Q[e] = mk<R>(i == j ? (R)1 : (R)0, 0);
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const R h = hbuf[j];
    if (h == (R)0) continue;
    const Cx<R> v0 = vhead[j];
    const Cx<R>* col = W + (long long)j * m;
    for (int c0 = j; c0 < k; c0 += ngroups) {
      const int c = c0 + gid;
      const bool valid = c < k;
      Cx<R>* q = Q + (long long)(valid ? c : j) * m;
      Cx<R> w = mk<R>(0, 0);
      if (valid) {
        if (gl == 0) w = cmulc(v0, q[j]);
        for (int i = j + 1 + gl; i < m; i += G) w = cadd(w, cmulc(col[i], q[i]));
      }
      for (int o = G >> 1; o > 0; o >>= 1) {
        w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
        w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
      }
      if (!valid) continue;
      const Cx<R> hw = cscale(w, h);
      if (gl == 0) q[j] = csub(q[j], cmul(hw, v0));
      for (int i = j + 1 + gl; i < m; i += G) q[i] = csub(q[i], cmul(hw, col[i]));
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ one-sided Jacobi SVD
// One CTA orthogonalises the n columns of the m x n (m >= n) column-major
// matrix A in place by complex plane rotations (Hestenes), round-robin
// ordering so that the n/2 pairs of a round are disjoint, with the rotations
// accumulated in V (n x n, column-major). At exit A V_in = U diag(sigma):
// sigma is sorted descending into `sigma`, the columns of A are overwritten
// by U (unit columns, permuted) and V by the permuted V. The truncation rank
// k (smallest k >= 1 with sum_{i >= k} sigma_i^2 <= delta2, then min(k,
// rmax); sigma_i instead of sigma_i^2 when values_are_squares, for the
// eigenvalues of a Gram matrix) is written to trunc[0] and trunc[1] = 1 if the cap cut more than
// delta2 allows. `perm` (n ints) and `snorm` (n reals) are workspace.
// The sweep loop is bounded by max_sweeps; trunc[2] receives the sweeps run.
template <typename R>
__global__ void jacobi_svd_kernel(int m, int n, Cx<R>* A, Cx<R>* V, double* sigma,
                                  int* perm, R* snorm, double delta2, int rmax, int* trunc,
                                  int max_sweeps, R tol, int values_are_squares, int use_smem,
                                  int want_v) {
  // the column data lives in dynamic shared memory when it fits (copied in
  // here, copied back to A before the columns are read out)
  extern __shared__ __align__(16) unsigned char jac_dyn[];
  Cx<R>* const Ag = A;
  if (use_smem) {
    A = (Cx<R>*)jac_dyn;
    for (long long e = threadIdx.x; e < (long long)m * n; e += blockDim.x) A[e] = Ag[e];
    __syncthreads();
  }
  __shared__ int s_rot;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  if (want_v)
    for (long long e = tid; e < (long long)n * n; e += nt) {
      const int i = (int)(e % n), j = (int)(e / n);
      V[e] = mk<R>(i == j ? (R)1 : (R)0, 0);
    }
  __shared__ R s_red[32];
  R f2 = 0;
  for (long long e = tid; e < (long long)m * n; e += nt) f2 += cabs2(A[e]);
  f2 = block_sum(f2, s_red);
  // Columns whose squared norm is below eps^2 ||A||_F^2 are at the rounding
  // noise floor: rotating them cannot orthogonalise them any further, so they
  // are left alone (otherwise the sweep never settles).
  const R eps_r = sizeof(R) == 8 ? (R)2.220446049250313e-16 : (R)1.1920929e-7;
  const R negl = eps_r * eps_r * f2;
  const int np = (n + 1) & ~1;  // players (even)
  const int mp = np - 1;
  // lanes per pair: the largest power of two <= 32 that still gives every
  // pair of a round its own group (at least 4 lanes)
  int G = 32;
  while (G > 4 && (nt / G) < np / 2) G >>= 1;
  const int gid = tid / G, gl = tid % G, ngroups = nt / G;
  int sweep = 0;
  if (tid == 0) s_rot = 1;
  __syncthreads();
  for (sweep = 0; sweep < max_sweeps && np > 1; ++sweep) {
    __syncthreads();
    if (s_rot == 0) break;
    __syncthreads();
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < mp; ++r) {
      // G lanes per column pair (aligned sub-warp groups): all pairs of a
      // round in one wave, short shuffle trees, m/G elements per lane.
      for (int pi0 = 0; pi0 < np / 2; pi0 += ngroups) {  // uniform across the block
        const int pi = pi0 + gid;
        int p = 0, q = 0;
        bool valid = pi < np / 2;
        if (valid) {
          if (pi == 0) {
            p = 0;
            q = (r % mp) + 1;
          } else {
            p = ((r + pi) % mp) + 1;
            q = ((r + mp - pi) % mp) + 1;
          }
          valid = p < n && q < n;
        }
        Cx<R>* ap = A + (long long)p * m;
        Cx<R>* aq = A + (long long)q * m;
        R app = 0, aqq = 0;
        Cx<R> apq = mk<R>(0, 0);
        if (valid)
          for (int i = gl; i < m; i += G) {
            const Cx<R> x = ap[i], y = aq[i];
            app += cabs2(x);
            aqq += cabs2(y);
            apq = cadd(apq, cmulc(x, y));
          }
        for (int o = G >> 1; o > 0; o >>= 1) {  // executed by every lane of the warp
          app += __shfl_xor_sync(0xffffffffu, app, o);
          aqq += __shfl_xor_sync(0xffffffffu, aqq, o);
          apq.x += __shfl_xor_sync(0xffffffffu, apq.x, o);
          apq.y += __shfl_xor_sync(0xffffffffu, apq.y, o);
        }
        if (!valid || app <= negl || aqq <= negl) continue;
        const R g = hypot(apq.x, apq.y);
        if (!(g > tol * sqrt(app) * sqrt(aqq))) continue;
        // reduce to a real symmetric 2x2 problem with phase e^{i phi} = apq/|apq|
        const Cx<R> e = mk<R>(apq.x / g, apq.y / g);
        const R zeta = (aqq - app) / ((R)2 * g);
        const R t = (zeta >= (R)0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt((R)1 + zeta * zeta));
        const R c = (R)1 / sqrt((R)1 + t * t);
        const R s = c * t;
        // a_p' = c a_p - s conj(e) a_q ; a_q' = s a_p + c conj(e) a_q
        const Cx<R> ec = cconj(e);
        for (int i = gl; i < m; i += G) {
          const Cx<R> x = ap[i], y = cmul(ec, aq[i]);
          ap[i] = mk<R>(c * x.x - s * y.x, c * x.y - s * y.y);
          aq[i] = mk<R>(s * x.x + c * y.x, s * x.y + c * y.y);
        }
        if (want_v) {
          Cx<R>* vp = V + (long long)p * n;
          Cx<R>* vq = V + (long long)q * n;
          for (int i = gl; i < n; i += G) {
            const Cx<R> x = vp[i], y = cmul(ec, vq[i]);
            vp[i] = mk<R>(c * x.x - s * y.x, c * x.y - s * y.y);
            vq[i] = mk<R>(s * x.x + c * y.x, s * x.y + c * y.y);
          }
        }
        if (gl == 0) s_rot = 1;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  // column norms
  for (int j = warp; j < n; j += nw) {
    R s2 = 0;
    const Cx<R>* a = A + (long long)j * m;
    for (int i = lane; i < m; i += 32) s2 += cabs2(a[i]);
    s2 = warp_sum(s2);
    // a column at the rounding-noise floor (never rotated, see negl) is not
    // orthogonal to the others: its singular value is zero to working
    // precision, so the truncation drops it
    if (lane == 0) snorm[j] = s2 <= negl ? (R)0 : sqrt(s2);
  }
  __syncthreads();
  // rank of each column in descending order (ties by index); a NaN norm
  // sorts last and raises trunc[4], so the ranks stay a permutation
  for (int j = tid; j < n; j += nt) {
    const R sj = isnan(snorm[j]) ? (R)-1 : snorm[j];
    if (isnan(snorm[j])) trunc[4] = 1;
    int rk = 0;
    for (int i = 0; i < n; ++i) {
      const R si = isnan(snorm[i]) ? (R)-1 : snorm[i];
      rk += (si > sj) || (si == sj && i < j);
    }
    perm[rk] = j;
  }
  __syncthreads();
  if (tid == 0) {
    double tail = 0;
    int k = n;
    // tail[j] = sum_{i >= j} s_i^2 ; smallest j >= 1 with tail[j] <= delta2
    double* tails = sigma;  // reuse sigma as scratch for the tails, fixed below
    for (int j = n - 1; j >= 0; --j) {
      const double s = (double)snorm[perm[j]];
      tail += values_are_squares ? s : s * s;
      tails[j] = tail;
    }
    k = n;
    for (int j = 1; j < n; ++j)
      if (tails[j] <= delta2) {
        k = j;
        break;
      }
    trunc[1] = (k > rmax) ? 1 : 0;
    trunc[0] = k < rmax ? k : rmax;
    trunc[2] = sweep;
  }
  __syncthreads();
  for (int j = tid; j < n; j += nt) {
    const R v = snorm[perm[j]];
    sigma[j] = isnan(v) ? 0.0 : (double)v;
  }
  if (use_smem)
    for (long long e = tid; e < (long long)m * n; e += nt) Ag[e] = A[e];
  __syncthreads();
}

// Multi-CTA one-sided Jacobi for matrices too large for one CTA's shared
// memory (cooperative launch: all CTAs resident). Same rotations and
// round-robin ordering as jacobi_svd_kernel; the n/2 disjoint pairs of a
// round are spread over the warps of the whole grid, grid.sync() separates
// rounds, and flags[sweep] (zeroed by the host, max_sweeps entries) records
// whether any warp rotated in that sweep. Writes the column norms to snorm;
// jacobi_finish_kernel sorts them and picks the truncation rank.
template <typename R>
__global__ void jacobi_grid_kernel(int m, int n, Cx<R>* A, Cx<R>* V, R* snorm, int* flags,
                                   int max_sweeps, R tol, R negl, int* sweeps_out, int want_v) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  if (want_v)
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
      const int i = (int)(e % n), j = (int)(e / n);
      V[e] = mk<R>(i == j ? (R)1 : (R)0, 0);
    }
  grid.sync();
  const int np = (n + 1) & ~1;
  const int mp = np - 1;
  int sweep = 0;
  for (sweep = 0; sweep < max_sweeps && np > 1; ++sweep) {
    for (int r = 0; r < mp; ++r) {
      for (int pi = gw; pi < np / 2; pi += nwarps) {
        int p, q;
        if (pi == 0) {
          p = 0;
          q = (r % mp) + 1;
        } else {
          p = ((r + pi) % mp) + 1;
          q = ((r + mp - pi) % mp) + 1;
        }
        if (p >= n || q >= n) continue;
        Cx<R>* ap = A + (long long)p * m;
        Cx<R>* aq = A + (long long)q * m;
        R app = 0, aqq = 0;
        Cx<R> apq = mk<R>(0, 0);
        for (int i = lane; i < m; i += 32) {
          const Cx<R> x = ap[i], y = aq[i];
          app += cabs2(x);
          aqq += cabs2(y);
          apq = cadd(apq, cmulc(x, y));
        }
        app = warp_sum(app);
        aqq = warp_sum(aqq);
        apq = warp_sum(apq);
        if (app <= negl || aqq <= negl) continue;
        const R g = hypot(apq.x, apq.y);
        if (!(g > tol * sqrt(app) * sqrt(aqq))) continue;
        const Cx<R> e = mk<R>(apq.x / g, apq.y / g);
        const R zeta = (aqq - app) / ((R)2 * g);
        const R t = (zeta >= (R)0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt((R)1 + zeta * zeta));
        const R c = (R)1 / sqrt((R)1 + t * t);
        const R s = c * t;
        const Cx<R> ec = cconj(e);
        for (int i = lane; i < m; i += 32) {
          const Cx<R> x = ap[i], y = cmul(ec, aq[i]);
          ap[i] = mk<R>(c * x.x - s * y.x, c * x.y - s * y.y);
          aq[i] = mk<R>(s * x.x + c * y.x, s * x.y + c * y.y);
        }
        if (want_v) {
          Cx<R>* vp = V + (long long)p * n;
          Cx<R>* vq = V + (long long)q * n;
          for (int i = lane; i < n; i += 32) {
            const Cx<R> x = vp[i], y = cmul(ec, vq[i]);
            vp[i] = mk<R>(c * x.x - s * y.x, c * x.y - s * y.y);
            vq[i] = mk<R>(s * x.x + c * y.x, s * x.y + c * y.y);
          }
        }
        if (lane == 0) atomicExch(&flags[sweep], 1);
      }
      grid.sync();
    }
    if (atomicAdd(&flags[sweep], 0) == 0) break;  // uniform: read after the last grid.sync
  }
  for (int j = gw; j < n; j += nwarps) {
    R s2 = 0;
    const Cx<R>* a = A + (long long)j * m;
    for (int i = lane; i < m; i += 32) s2 += cabs2(a[i]);
    s2 = warp_sum(s2);
    if (lane == 0) snorm[j] = s2 <= negl ? (R)0 : sqrt(s2);  // noise-floor column: zero
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = sweep;
}

// Sort column norms descending (ties by index) into sigma/perm and pick the
// truncation rank (same rule as jacobi_svd_kernel). One CTA.
template <typename R>
__global__ void jacobi_finish_kernel(int n, const R* snorm, double* sigma, int* perm,
                                     double delta2, int rmax, int* trunc,
                                     int values_are_squares, const int* sweeps) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const R sj = isnan(snorm[j]) ? (R)-1 : snorm[j];
    if (isnan(snorm[j])) trunc[4] = 1;
    int rk = 0;
    for (int i = 0; i < n; ++i) {
      const R si = isnan(snorm[i]) ? (R)-1 : snorm[i];
      rk += (si > sj) || (si == sj && i < j);
    }
    perm[rk] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tail = 0;
    for (int j = n - 1; j >= 0; --j) {
      const double s = (double)snorm[perm[j]];
      tail += values_are_squares ? s : s * s;
      sigma[j] = tail;
    }
    int k = n;
    for (int j = 1; j < n; ++j)
      if (sigma[j] <= delta2) {
        k = j;
        break;
      }
    trunc[1] = (k > rmax) ? 1 : 0;
    trunc[0] = k < rmax ? k : rmax;
    trunc[2] = *sweeps;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const R v = snorm[perm[j]];
    sigma[j] = isnan(v) ? 0.0 : (double)v;
  }
}

// Reorders/normalises columns after jacobi_svd_kernel: Uout[:, j] =
// A[:, perm[j]] / sigma_j (0 when sigma_j == 0), Vout[:, j] = V[:, perm[j]].
template <typename R>
__global__ void svd_finish_kernel(int m, int n, const Cx<R>* A, const Cx<R>* V, const double* sigma,
                                  const int* perm, Cx<R>* Uout, Cx<R>* Vout, int* err, int want_v) {
  const long long tot = (long long)m * n + (want_v ? (long long)n * n : 0ll);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int pj = perm[(e < (long long)m * n) ? (int)(e / m) : (int)((e - (long long)m * n) / n)];
    if (pj < 0 || pj >= n) {  // data-dependent index: check, record, skip
      atomicExch(err, 1);
      continue;
    }
    if (e < (long long)m * n) {
      const int i = (int)(e % m), j = (int)(e / m);
      const double s = sigma[j];
      const Cx<R> a = A[(long long)pj * m + i];
      Uout[e] = s > 0 ? mk<R>((R)(a.x / s), (R)(a.y / s)) : mk<R>(0, 0);
    } else {
      const long long f = e - (long long)m * n;
      const int i = (int)(f % n);
      Vout[f] = V[(long long)pj * n + i];
    }
  }
}

// ------------------------------------------------------------------ strided copy / permute
// out[flat] = s * op(in[sum_d idx_d * in_stride_d]) over an up-to-6-D index
// space (sizes[0] slowest), optional conjugation; out is contiguous or has
// its own strides.
struct CopyArgs {
  int nd;
  long long size[6];
  long long in_st[6];
  long long out_st[6];
  int conj;
  double scale;
};

template <typename R>
__global__ void copy_kernel(const Cx<R>* __restrict__ in, Cx<R>* __restrict__ out, CopyArgs a,
                            long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e, io = 0, oo = 0;
    for (int d = a.nd - 1; d >= 0; --d) {
      const long long i = r % a.size[d];
      r /= a.size[d];
      io += i * a.in_st[d];
      oo += i * a.out_st[d];
    }
    if (a.scale == 0.0) {
      out[oo] = mk<R>(0, 0);
      continue;
    }
    Cx<R> v = in[io];
    if (a.conj) v.y = -v.y;
    out[oo] = mk<R>((R)(v.x * a.scale), (R)(v.y * a.scale));
  }
}

template <typename Rin, typename Rout>
__global__ void convert_kernel(const Cx<Rin>* __restrict__ in, Cx<Rout>* __restrict__ out,
                               long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = mk<Rout>((Rout)in[e].x, (Rout)in[e].y);
}

// Scale column j of an m x k column-major matrix by sigma[j].
template <typename R>
__global__ void scale_cols_kernel(Cx<R>* M, int m, int k, const double* sigma) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)m * k;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / m);
    M[e] = cscale(M[e], (R)sigma[j]);
  }
}

// sum |x|^2 in FP64, atomically added to *out.
template <typename R>
__global__ void norm2_kernel(const Cx<R>* __restrict__ x, long long n, double* out) {
  double s = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    s += (double)x[e].x * x[e].x + (double)x[e].y * x[e].y;
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// x /= sqrt(*nrm2) (no-op when the norm is 0): keeps the random sketch
// environments at unit scale; only their range matters downstream.
template <typename R>
__global__ void scale_inv_norm_kernel(Cx<R>* x, long long n, const double* nrm2) {
  const double s2 = *nrm2;
  if (!(s2 > 0.0)) return;
  const R inv = (R)(1.0 / sqrt(s2));
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[e] = cscale(x[e], inv);
}

// ------------------------------------------------------------------ Philox sketches
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32
// multiplications with key schedule increments (Weyl sequence).
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
    k0 += W0;
    k1 += W1;
  }
}

__device__ __forceinline__ double u32_unit(uint32_t w) {
  return ((double)(int32_t)w + 0.5) * 4.656612873077392578125e-10;  // 2^-31
}

// Sketch core entries: entry e uses counter (e >> 1, core, apply_id, tag) and
// key (seed low, seed high); even e takes words (0, 1), odd e words (2, 3) as
// (re, im), each mapped to (int32(w) + 1/2) 2^-31 in (-1, 1).
template <typename R>
__global__ void sketch_kernel(Cx<R>* out, long long count, uint64_t seed, int core, int apply_id) {
  const uint32_t tag = 0x5EC7C0DEu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)(e >> 1), (uint32_t)core, (uint32_t)apply_id, tag};
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const uint32_t wr = (e & 1) ? c[2] : c[0];
    const uint32_t wi = (e & 1) ? c[3] : c[1];
    out[e] = mk<R>((R)u32_unit(wr), (R)u32_unit(wi));
  }
}

// ------------------------------------------------------------------ dense fields (preprocessing)

__device__ __forceinline__ int bitrev(int k, int n) { return (int)(__brev((unsigned)k) >> (32 - n)); }

// Green operator of the Direct scheme (App. A) in the SFFT momentum
// convention: at momentum index (k1, k2, k3) the frequency is xi_a =
// xi(rev k_a), xi(k) = k for k <= N/2 else k - N, and
// Gamma_ijkl = (d_ik n_j n_l + d_il n_j n_k + d_jk n_i n_l + d_jl n_i n_k) / (4 mu0)
//              - (lam0 + mu0) / (mu0 (lam0 + 2 mu0)) n_i n_j n_k n_l,
// Gamma_V[I, J] = w_I w_J Gamma_{i_I j_I k_J l_J}, Gamma(0) = 0; at modes with
// a Nyquist component (|xi_a| = N/2) the value is averaged with the one at xi
// with those components negated (Nyquist symmetrisation, the aliased partner
// -xi mod N). Real-valued, so the conjugation of the convention is the identity.
// Gamma_V is a fixed 36 x 15 matrix (depending on lam0, mu0; built on the
// host) times the 15 degree-4 monomials n_a n_b n_c n_d (a <= b <= c <= d,
// lexicographic order), since n_a n_b = sum_c n_a n_b n_c n_c; the kernels
// below evaluate those monomials (all 0 at xi = 0, Nyquist-averaged).
__device__ void green_monomials_at(const double xi[3], double* m15) {
  const double r2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
  double nn[3] = {0, 0, 0};
  if (r2 > 0) {
    const double r = sqrt(r2);
    for (int a = 0; a < 3; ++a) nn[a] = xi[a] / r;
  }
  int g = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b)
      for (int c = b; c < 3; ++c)
        for (int d = c; d < 3; ++d) m15[g++] = nn[a] * nn[b] * nn[c] * nn[d];
}

// Monomials of v/|v| for the schemes whose divergence operator is a common
// factor times a real vector v (App. A table):
//   scheme 0 (Direct, k = i q): v = xi.
//   scheme 1 (Centered, k = i sin q): v_a = sin(2 pi xi_a / N), 0 at a Nyquist
//     component.
//   scheme 4 (Hex8R, k_j = (i/4) tan(q_j/2) prod_l (1 + e^{i q_l})):
//     v_j = sin(q_j/2) prod_{l != j} cos(q_l/2); cos(q_l/2) = 0 at a Nyquist
//     component and sin(q_j/2) = sign(xi_j) there, so v = 0 where two
//     components sit at the Nyquist frequency.
// At Nyquist modes the value is the average with the aliased partner (the
// Nyquist components negated); the monomials are even in v, so for schemes 1
// and 4 the average is the value itself. plane = 1 evaluates only the plane
// xi_1 = 0: N^2 points (xi_2, xi_3), out[q * N^2 + e].
__global__ void green_monomials_kernel(Cx<double>* out, int n, int scheme, int plane) {
  const long long N = 1ll << n, N3 = plane ? N * N : N * N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N3;
       e += (long long)gridDim.x * blockDim.x) {
    const int ks[3] = {plane ? 0 : (int)(e / (N * N)), (int)((e / N) % N), (int)(e % N)};
    double xi[3], xf[3], hs[3], hc[3];
    bool nyq = false;
    for (int a = 0; a < 3; ++a) {
      const int k = n > 0 ? bitrev(ks[a], n) : 0;
      xi[a] = (k <= N / 2) ? (double)k : (double)(k - N);
      const bool isn = (2 * (long long)fabs(xi[a]) == N);
      nyq |= isn;
      xf[a] = isn ? -xi[a] : xi[a];
      sincospi(xi[a] / (double)N, &hs[a], &hc[a]);
      if (isn) {
        hs[a] = xi[a] > 0 ? 1.0 : -1.0;
        hc[a] = 0.0;
      }
      if (scheme == 1) {
        xi[a] = isn ? 0.0 : sinpi(2.0 * xi[a] / (double)N);
        xf[a] = isn ? 0.0 : xi[a];
      }
    }
    if (scheme == 4) {
      for (int a = 0; a < 3; ++a) {
        xi[a] = hs[a] * hc[(a + 1) % 3] * hc[(a + 2) % 3];
        xf[a] = xi[a];
      }
    }
    double g[15], gf[15];
    green_monomials_at(xi, g);
    if (nyq) {
      green_monomials_at(xf, gf);
      for (int q = 0; q < 15; ++q) g[q] = 0.5 * (g[q] + gf[q]);
    }
    for (int q = 0; q < 15; ++q) out[(long long)q * N3 + e] = mk<double>(g[q], 0.0);
  }
}

__host__ __device__ inline double2 zmul(double2 x, double2 y) {
  return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
}
__host__ __device__ inline double2 zsub(double2 x, double2 y) {
  return make_double2(x.x - y.x, x.y - y.y);
}

// eq. (orig_green_eshelby) in Voigt form for a strain symbol with normal
// components kn and shear components kt (eps_aa = kn_a u_a, 2 eps_ab =
// kt_b u_a + kt_a u_b, Voigt order 11 22 33 23 13 12): with B the 6 x 3
// symbol, Gamma_V = B (B^H C0_V B)^-1 B^H for the isotropic C0 of Lame
// parameters (lam0, mu0). The symbols must not all vanish and should be
// scaled to |k| ~ 1 (Gamma is homogeneous of degree 0 in k). The 3 x 3 inverse
// is the adjugate over the determinant. g[I * 6 + J] = conj(Gamma_V[I][J]).
__host__ __device__ inline void green_symbol_voigt_conj(const double2 kn[3], const double2 kt[3],
                                                        double lam0, double mu0, double2 g[36]) {
  const int vi[3] = {1, 0, 0}, vj[3] = {2, 2, 1};  // Voigt 3, 4, 5 = (23), (13), (12)
  double2 B[6][3];
  for (int I = 0; I < 6; ++I)
    for (int m = 0; m < 3; ++m) B[I][m] = make_double2(0.0, 0.0);
  for (int a = 0; a < 3; ++a) B[a][a] = kn[a];
  for (int t = 0; t < 3; ++t) {
    B[3 + t][vi[t]] = kt[vj[t]];
    B[3 + t][vj[t]] = kt[vi[t]];
  }
  // CB = C0_V B: lam0 tr + 2 mu0 on the normal rows, mu0 on the shear rows
  double2 CB[6][3];
  for (int m = 0; m < 3; ++m) {
    const double trx = B[0][m].x + B[1][m].x + B[2][m].x;
    const double try_ = B[0][m].y + B[1][m].y + B[2][m].y;
    for (int a = 0; a < 3; ++a)
      CB[a][m] = make_double2(lam0 * trx + 2.0 * mu0 * B[a][m].x,
                              lam0 * try_ + 2.0 * mu0 * B[a][m].y);
    for (int t = 3; t < 6; ++t) CB[t][m] = make_double2(mu0 * B[t][m].x, mu0 * B[t][m].y);
  }
  // K = B^H C0_V B (3 x 3 Hermitian)
  double2 K[3][3];
  for (int m = 0; m < 3; ++m)
    for (int p = 0; p < 3; ++p) {
      double re = 0, im = 0;
      for (int I = 0; I < 6; ++I) {
        const double2 u = B[I][m], v = CB[I][p];  // conj(u) v
        re += u.x * v.x + u.y * v.y;
        im += u.x * v.y - u.y * v.x;
      }
      K[m][p] = make_double2(re, im);
    }
  double2 cof[3][3];
  for (int m = 0; m < 3; ++m)
    for (int p = 0; p < 3; ++p) {
      const int m1 = (m + 1) % 3, m2 = (m + 2) % 3, p1 = (p + 1) % 3, p2 = (p + 2) % 3;
      cof[m][p] = zsub(zmul(K[m1][p1], K[m2][p2]), zmul(K[m1][p2], K[m2][p1]));
    }
  double2 det = make_double2(0.0, 0.0);
  for (int p = 0; p < 3; ++p) {
    const double2 t = zmul(K[0][p], cof[0][p]);
    det.x += t.x;
    det.y += t.y;
  }
  const double dd = det.x * det.x + det.y * det.y;
  const double2 rdet = make_double2(det.x / dd, -det.y / dd);
  for (int I = 0; I < 6; ++I) {
    double2 W[3];  // (B K^-1)[I][:], K^-1[p][m] = cof[m][p] / det
    for (int m = 0; m < 3; ++m) {
      double2 acc = make_double2(0.0, 0.0);
      for (int p = 0; p < 3; ++p) {
        const double2 t = zmul(B[I][p], zmul(cof[m][p], rdet));
        acc.x += t.x;
        acc.y += t.y;
      }
      W[m] = acc;
    }
    for (int J = 0; J < 6; ++J) {
      double re = 0, im = 0;
      for (int m = 0; m < 3; ++m) {
        const double2 w = W[m], u = B[J][m];  // w conj(u)
        re += w.x * u.x + w.y * u.y;
        im += w.y * u.x - w.x * u.y;
      }
      g[I * 6 + J] = make_double2(re, -im);
    }
  }
}

// Green field of the schemes with complex divergence operators (App. A table):
// scheme 2 (Forward, k+_a = e^{i q_a} - 1), 3 (Backward, k-_a = 1 - e^{-i q_a})
// and 5 (staggered grid: normal strains with k+, shear strains with k-), from
// green_symbol_voigt_conj; Gamma_V = 0 at xi = 0. The symbols are real and
// equal at +-N/2 for a Nyquist component, so the Nyquist rule leaves these
// operators unchanged. Stored in the SFFT convention (its transform sign is
// opposite to the one the symbols are written for, and Gamma(-xi) =
// conj(Gamma(xi))): out[(I * 6 + J) * N3 + e] = conj(Gamma_V[I][J]) at the
// frequency of bit-reversed index e. plane = 1 evaluates only the plane
// xi_1 = 0 (N3 = N^2 points).
__global__ void green_symbol_field_kernel(Cx<double>* out, int n, double lam0, double mu0,
                                          int scheme, int plane) {
  const long long N = 1ll << n, N3 = plane ? N * N : N * N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N3;
       e += (long long)gridDim.x * blockDim.x) {
    const int ks[3] = {plane ? 0 : (int)(e / (N * N)), (int)((e / N) % N), (int)(e % N)};
    double2 kp[3], km[3];
    double nrm2 = 0;
    for (int a = 0; a < 3; ++a) {
      const int k = n > 0 ? bitrev(ks[a], n) : 0;
      const double x = (k <= N / 2) ? (double)k : (double)(k - N);
      double s, c;
      sincospi(2.0 * x / (double)N, &s, &c);
      if (2 * (long long)fabs(x) == N) {
        s = 0.0;
        c = -1.0;
      }
      kp[a] = make_double2(c - 1.0, s);
      km[a] = make_double2(1.0 - c, s);
      nrm2 += (c - 1.0) * (c - 1.0) + s * s;
    }
    if (nrm2 == 0.0) {
      for (int P = 0; P < 36; ++P) out[(long long)P * N3 + e] = mk<double>(0.0, 0.0);
      continue;
    }
    const double inv = 1.0 / sqrt(nrm2);
    for (int a = 0; a < 3; ++a) {
      kp[a] = make_double2(kp[a].x * inv, kp[a].y * inv);
      km[a] = make_double2(km[a].x * inv, km[a].y * inv);
    }
    double2 g[36];
    green_symbol_voigt_conj(scheme == 3 ? km : kp, scheme == 2 ? kp : km, lam0, mu0, g);
    for (int P = 0; P < 36; ++P) out[(long long)P * N3 + e] = mk<double>(g[P].x, g[P].y);
  }
}

// Voigt-matrix stiffness-difference field from a phase array with broadcast
// axes: out[P * cells + c] = dC[phase(c)][P] where P indexes the 36 Voigt
// pairs (row-major 6x6) and c runs over the non-broadcast cells.
__global__ void stiffness_field_kernel(const uint8_t* phase, long long cells, const double* dC,
                                       int nphase, Cx<double>* out) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    int p = phase[c];
    if (p >= nphase) p = nphase - 1;
    for (int P = 0; P < 36; ++P) out[(long long)P * cells + c] = mk<double>(dC[p * 36 + P], 0.0);
  }
}

// Squared column norms (FP64) of a row-major P x c matrix, accumulated into
// out[c] (zeroed by the caller); each CTA sums a slab of rows in shared memory.
template <typename R>
__global__ void colnorm2_kernel(const Cx<R>* __restrict__ M, long long P, int c, double* out) {
  extern __shared__ double cn_acc[];
  for (int j = threadIdx.x; j < c; j += blockDim.x) cn_acc[j] = 0;
  __syncthreads();
  const long long tot = P * c;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const Cx<R> v = M[e];
    atomicAdd(&cn_acc[e % c], (double)v.x * v.x + (double)v.y * v.y);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < c; j += blockDim.x) atomicAdd(&out[j], cn_acc[j]);
}

// dst[r * k + a] = src[r * c + idx[a]] for a row-major P x c source.
template <typename R>
__global__ void gather_cols_kernel(const Cx<R>* __restrict__ src, long long P, int c,
                                   const int* __restrict__ idx, int k, Cx<R>* __restrict__ dst,
                                   int* err) {
  const long long tot = P * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / k;
    const int a = (int)(e % k);
    const int j = idx[a];
    if (j < 0 || j >= c) {  // data-dependent index: check, record, skip
      atomicExch(err, 1);
      continue;
    }
    dst[e] = src[r * c + j];
  }
}

// Orthonormalising factor of a sketch environment. G (row-major L x L) is
// the Gram matrix P^H P of a matrix P with L columns. One CTA runs a Cholesky
// factorisation with diagonal pivoting (step j takes the largest remaining
// diagonal entry, the first on ties), R^H R = Pi^T G Pi, and stops at the
// first step whose pivot is at or below tau * max_i G_ii; with k steps taken,
// M (row-major L x L) gets M[perm[i]][j] = (R^{-1})[i][j] for i <= j < k and
// zeros elsewhere, so that P M has k orthonormal columns followed by zero
// ones. Pivoting keeps R^{-1} bounded where columns of P are nearly dependent.
// The working matrix (L x L, then R, then R^{-1} in place) and an L-vector
// live in dynamic shared memory when use_smem, else in Wg (L * L + L
// entries). perm: int scratch of L. A non-finite diagonal of G sets *err and
// leaves M zero.
template <typename R>
__global__ void __launch_bounds__(1024)
chol_piv_inv_kernel(int L, const Cx<R>* __restrict__ G, Cx<R>* Wg, Cx<R>* M, int* perm,
                    double tau, int* err, int use_smem) {
  extern __shared__ __align__(16) unsigned char chol_dyn[];
  Cx<R>* const A = use_smem ? (Cx<R>*)chol_dyn : Wg;
  Cx<R>* const tmp = A + (long long)L * L;
  __shared__ R red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_bad, s_p;
  __shared__ R s_d;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nw = (nt + 31) >> 5;
  const long long LL = (long long)L * L;
  for (long long e = tid; e < LL; e += nt) {
    A[e] = G[e];
    M[e] = mk<R>(0, 0);
  }
  for (int i = tid; i < L; i += nt) perm[i] = i;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  R mx = 0;
  for (int i = tid; i < L; i += nt) {
    const R v = G[(long long)i * L + i].x;
    if (!isfinite(v)) s_bad = 1;
    mx = v > mx ? v : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const R w = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = w > mx ? w : mx;
  }
  if (lane == 0) red_v[warp] = mx;
  __syncthreads();
  if (s_bad) {
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  R ref = 0;
  for (int w = 0; w < nw; ++w) ref = red_v[w] > ref ? red_v[w] : ref;
  const R thr = (R)tau * ref;
  __syncthreads();
  int k = L;
  for (int j = 0; j < L; ++j) {
    // pivot: largest remaining diagonal entry, lowest index on ties
    R bv = (R)-1;
    int bi = L;
    for (int i = j + tid; i < L; i += nt) {
      const R v = A[(long long)i * L + i].x;
      if (v > bv) {
        bv = v;
        bi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const R ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_i[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      R v = red_v[0];
      int ix = red_i[0];
      for (int w = 1; w < nw; ++w)
        if (red_v[w] > v || (red_v[w] == v && red_i[w] < ix)) {
          v = red_v[w];
          ix = red_i[w];
        }
      s_d = v;
      s_p = ix;
    }
    __syncthreads();
    if (!(s_d > thr) || s_p >= L) {  // uniform: every thread reads the same values
      k = j;
      break;
    }
    const int p = s_p;
    if (p != j) {
      for (int c = tid; c < L; c += nt) {
        const Cx<R> t = A[(long long)j * L + c];
        A[(long long)j * L + c] = A[(long long)p * L + c];
        A[(long long)p * L + c] = t;
      }
      __syncthreads();
      for (int r = tid; r < L; r += nt) {
        const Cx<R> t = A[(long long)r * L + j];
        A[(long long)r * L + j] = A[(long long)r * L + p];
        A[(long long)r * L + p] = t;
      }
      if (tid == 0) {
        const int t = perm[j];
        perm[j] = perm[p];
        perm[p] = t;
      }
      __syncthreads();
    }
    Cx<R>* rowj = A + (long long)j * L;
    const R d = rowj[j].x;
    const R sd = sqrt(d);
    const R inv = (R)1 / sd;
    __syncthreads();  // every thread has read the pivot before row j changes
    for (int c = j + 1 + tid; c < L; c += nt) rowj[c] = cscale(rowj[c], inv);
    if (tid == 0) rowj[j] = mk<R>(sd, 0);
    __syncthreads();
    const int t = L - j - 1;
    for (long long e = tid; e < (long long)t * t; e += nt) {
      const int r = j + 1 + (int)(e / t), c = j + 1 + (int)(e % t);
      Cx<R>* q = A + (long long)r * L + c;
      *q = csub(*q, cmulc(rowj[r], rowj[c]));
    }
    __syncthreads();
  }
  __syncthreads();
  // R^{-1} of the leading k x k block in place, column by column:
  // Rinv[i][j] = -(sum_{i<=l<j} Rinv[i][l] R[l][j]) / R[j][j] (i < j),
  // Rinv[j][j] = 1 / R[j][j]; columns < j already hold Rinv, column j still R
  for (int j = 0; j < k; ++j) {
    const R rjj = A[(long long)j * L + j].x;
    for (int i = tid; i < j; i += nt) {
      Cx<R> acc = mk<R>(0, 0);
      for (int l = i; l < j; ++l)
        acc = csub(acc, cmul(A[(long long)i * L + l], A[(long long)l * L + j]));
      tmp[i] = acc;
    }
    __syncthreads();
    const R inv = (R)1 / rjj;
    for (int i = tid; i < j; i += nt) A[(long long)i * L + j] = cscale(tmp[i], inv);
    if (tid == 0) A[(long long)j * L + j] = mk<R>(inv, 0);
    __syncthreads();
  }
  for (long long e = tid; e < (long long)k * k; e += nt) {
    const int i = (int)(e / k), j = (int)(e % k);
    if (i <= j) {
      const Cx<R> v = A[(long long)i * L + j];
      if (!isfinite(v.x) || !isfinite(v.y)) atomicExch(err, 2);
      M[(long long)perm[i] * L + j] = v;
    }
  }
}

// Q[:, j] = 0 for every j < k with R[j][j] exactly zero (Q column-major m x k,
// R column-major with leading dimension ldr): a zero column of the factored
// matrix spans nothing, so the reflector's arbitrary direction is removed.
template <typename R>
__global__ void zero_dead_cols_kernel(Cx<R>* Q, int m, int k, const Cx<R>* Rm, int ldr) {
  const long long tot = (long long)m * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / m);
    const Cx<R> d = Rm[j + (long long)j * ldr];
    if (d.x == (R)0 && d.y == (R)0) Q[e] = mk<R>(0, 0);
  }
}

// Tall-skinny Gram matrix G += M^H M (G column-major c x c, zeroed by the
// caller) of a row-major P x c matrix M with c <= kGramMaxCols. A 64 x 64 GEMM
// tile would do (64/c)^2 times the useful work here, and FP64 is slow enough
// on this part for that to dominate the TT-SVD of a dense field. Each CTA
// stages a contiguous slab of rows through shared memory; each thread owns
// entries (a <= b) of the upper triangle and, when there are fewer than 256 of
// them, one of S interleaved row slices. Per-CTA partial sums are reduced over
// the slices in shared memory and added to both triangles of G atomically.
constexpr int kGramMaxCols = 64;
constexpr int kGramChunk = 2048;  // complex elements staged per chunk

template <typename R>
__global__ void __launch_bounds__(256)
gram_skinny_kernel(const Cx<R>* __restrict__ M, long long P, int c, long long rows_per_cta,
                   Cx<R>* G) {
  constexpr int kMaxOwn = (kGramMaxCols * (kGramMaxCols + 1) / 2 + 255) / 256;
  __shared__ Cx<R> sm[kGramChunk];
  __shared__ Cx<R> red[256];
  const int Q = c * (c + 1) / 2;
  const int S = Q >= 256 ? 1 : 256 / Q;
  const int t = threadIdx.x;
  const bool active = S > 1 ? t < S * Q : true;
  const int s = S > 1 ? t / Q : 0;
  int pa[kMaxOwn], pb[kMaxOwn];
  int np = 0;
  if (active) {
    const int step = S > 1 ? Q : 256;
#pragma unroll
    for (int k = 0; k < kMaxOwn; ++k) {
      const int q = (S > 1 ? t % Q : t) + k * step;
      pa[k] = 0;
      pb[k] = 0;
      if (q < Q && (S == 1 || k == 0)) {
        int b = 0;
        while ((b + 1) * (b + 2) / 2 <= q) ++b;
        pa[k] = q - b * (b + 1) / 2;
        pb[k] = b;
        np = k + 1;
      }
    }
  }
  Cx<R> acc[kMaxOwn];
#pragma unroll
  for (int k = 0; k < kMaxOwn; ++k) acc[k] = mk<R>(0, 0);
  const long long r0 = (long long)blockIdx.x * rows_per_cta;
  const long long r1 = r0 + rows_per_cta < P ? r0 + rows_per_cta : P;
  const int ch = kGramChunk / c;
  for (long long rb = r0; rb < r1; rb += ch) {
    const int nr = (int)(r1 - rb < ch ? r1 - rb : ch);
    const Cx<R>* src = M + rb * c;
    __syncthreads();
    for (int i = t; i < nr * c; i += 256) sm[i] = src[i];
    __syncthreads();
    for (int r = s; r < nr; r += S) {
      const Cx<R>* row = sm + r * c;
#pragma unroll
      for (int k = 0; k < kMaxOwn; ++k)
        if (k < np) acc[k] = cadd(acc[k], cmulc(row[pa[k]], row[pb[k]]));
    }
  }
  if (S > 1) {
    __syncthreads();
    red[t] = active ? acc[0] : mk<R>(0, 0);
    __syncthreads();
    if (t < Q) {
      Cx<R> v = red[t];
      for (int j = 1; j < S; ++j) v = cadd(v, red[t + j * Q]);
      acc[0] = v;
      np = 1;
    } else {
      np = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < kMaxOwn; ++k)
    if (k < np) {
      const int a = pa[k], b = pb[k];
      atomicAdd(&G[a + (long long)b * c].x, acc[k].x);
      atomicAdd(&G[a + (long long)b * c].y, acc[k].y);
      if (a != b) {
        atomicAdd(&G[b + (long long)a * c].x, acc[k].x);
        atomicAdd(&G[b + (long long)a * c].y, -acc[k].y);
      }
    }
}

// out = M V for a row-major P x c matrix M and a column-major c x c matrix V,
// c <= kSkinnyMaxCols, written row-major P x c; V sits in shared memory and
// one thread computes one output entry (the threads of a row share its loads).
constexpr int kSkinnyMaxCols = 32;

template <typename R>
__global__ void matmul_skinny_kernel(const Cx<R>* __restrict__ M, long long P, int c,
                                     const Cx<R>* __restrict__ V, Cx<R>* __restrict__ out) {
  __shared__ Cx<R> vs[kSkinnyMaxCols * kSkinnyMaxCols];
  for (int i = threadIdx.x; i < c * c; i += blockDim.x) vs[i] = V[i];
  __syncthreads();
  const long long tot = P * c;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / c;
    const int j = (int)(e - p * c);
    const Cx<R>* row = M + p * c;
    Cx<R> acc = mk<R>(0, 0);
    for (int a = 0; a < c; ++a) acc = cadd(acc, cmul(row[a], vs[a + j * c]));
    out[e] = acc;
  }
}

// out[a * cells + x] = table[phase(x) + a * nphase] for a < k: a field whose
// rows are k complex coefficient vectors indexed by the phase of each cell.
__global__ void phase_table_field_kernel(const uint8_t* __restrict__ phase, long long cells,
                                         const Cx<double>* __restrict__ table, int nphase, int k,
                                         Cx<double>* __restrict__ out) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < cells;
       x += (long long)gridDim.x * blockDim.x) {
    int p = phase[x];
    if (p >= nphase) p = nphase - 1;
    for (int a = 0; a < k; ++a) out[(long long)a * cells + x] = table[p + a * nphase];
  }
}

// SFFT tensor of one axis in core order: out[e], e = sum_b (2 o_b + i_b) 4^(n-1-b),
// = S[k', x] = N^-1/2 exp(2 pi i rev(k') x / N) with k' bits o_b, x bits i_b (MSB first).
__global__ void sfft_tensor_kernel(double* out, int n) {
  const long long N = 1ll << n, tot = N * N;
  const double inv = 1.0 / sqrt((double)N);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    int kp = 0, x = 0;
    for (int b = 0; b < n; ++b) {
      const int digit = (int)((e >> (2 * (n - 1 - b))) & 3);
      kp = (kp << 1) | (digit >> 1);
      x = (x << 1) | (digit & 1);
    }
    const long long k = n > 0 ? bitrev(kp, n) : 0;
    const long long ph = (k * x) % N;  // exact phase index
    double s, c;
    sincospi(2.0 * (double)ph / (double)N, &s, &c);
    out[2 * e] = c * inv;
    out[2 * e + 1] = s * inv;
  }
}

}  // namespace qtt
