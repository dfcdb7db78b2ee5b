// Host engine and C ABI of the QTT homogenisation library (see
// include/qtt_homog.h for the contract of every entry point).
//
// The engine drives sweeps over the tensor-train cores from the host: every
// contraction is a launch of the strided batched complex GEMM, every
// factorisation a one-CTA Householder QR or one-sided Jacobi SVD, and the
// ranks chosen by a truncation are read back before the next core is sized.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <thread>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/qtt_homog.h"
#include "kernels.cuh"
#include "sfft_zipup.h"
#include "tc_gemm.cuh"

using namespace qtt;

namespace {

struct QttError : std::runtime_error {
  int code;
  QttError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define QCHECK(call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw QttError(QTT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)

#define QREQ(cond, msg)                                  \
  do {                                                   \
    if (!(cond)) throw QttError(QTT_EINVAL, (msg));      \
  } while (0)

// ------------------------------------------------------------------ workspace arena
// First-fit allocator over the caller's device buffer, 256-byte granules,
// neighbouring free blocks coalesced on release. Host-side bookkeeping only.
struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0, peak = 0;
  std::mutex mu;  // lanes own separate arenas; the lock guards misuse
  std::map<size_t, size_t> free_;   // offset -> bytes
  std::map<size_t, size_t> taken_;  // offset -> bytes
  void init(void* b, size_t s) {
    base = (char*)b;
    size = s & ~(size_t)255;
    free_.clear();
    taken_.clear();
    free_[0] = size;
    used = peak = 0;
  }
  void* alloc(size_t bytes) {
    std::lock_guard<std::mutex> g(mu);
    bytes = std::max<size_t>(256, (bytes + 255) & ~(size_t)255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rem = it->second - bytes;
        if (off + bytes > size)
          throw QttError(QTT_EINVAL, "workspace allocator state corrupted");
        free_.erase(it);
        if (rem) free_[off + bytes] = rem;
        taken_[off] = bytes;
        used += bytes;
        peak = std::max(peak, used);
        return base + off;
      }
    }
    throw QttError(QTT_ENOMEM, "workspace exhausted: need " + std::to_string(bytes) +
                                   " bytes, " + std::to_string(size - used) + " free");
  }
  // Bytes from p to the end of the allocation holding p, or -1.
  long long extent(const void* p) {
    std::lock_guard<std::mutex> g(mu);
    if (!p || (const char*)p < base || (const char*)p >= base + size) return -1;
    const size_t off = (const char*)p - base;
    auto it = taken_.upper_bound(off);
    if (it == taken_.begin()) return -1;
    --it;
    if (off >= it->first + it->second) return -1;
    return (long long)(it->first + it->second - off);
  }
  void release(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(mu);
    const size_t off = (char*)p - base;
    auto it = taken_.find(off);
    if (it == taken_.end()) return;
    size_t bytes = it->second;
    taken_.erase(it);
    used -= bytes;
    size_t start = off;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && nx->first == off + bytes) {
      bytes += nx->second;
      free_.erase(nx);
    }
    auto pv = free_.lower_bound(off);
    if (pv != free_.begin()) {
      --pv;
      if (pv->first + pv->second == off) {
        start = pv->first;
        bytes += pv->second;
        free_.erase(pv);
      }
    }
    free_[start] = bytes;
  }
};

// Kernel-class timing of one lane (class: 0 gemm, 1 qr, 2 svd): CUDA
// events recorded around launches on the lane's stream, resolved in batches
// by the lane's own host thread, so that lanes never share a lock while they
// launch. The totals are merged into the context when the lanes finish.
struct ProfBuf {
  struct Ev {
    cudaEvent_t a, b;
    int cls;
    double flops;
  };
  std::vector<Ev> evs;
  double ms[3] = {0, 0, 0};
  double flops[3] = {0, 0, 0};
  long long n[3] = {0, 0, 0};
  double sweeps = 0;  // Jacobi sweeps run
  double tc_launches = 0;  // GEMMs run on the tcgen05 kernel
  std::vector<cudaEvent_t> pool;  // resolved events, reused
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void resolve() {
    for (auto& e : evs) {
      float t = 0;
      if (cudaEventSynchronize(e.b) == cudaSuccess && cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) {
        ms[e.cls] += t;
        flops[e.cls] += e.flops;
        n[e.cls] += 1;
      }
      pool.push_back(e.a);
      pool.push_back(e.b);
    }
    evs.clear();
  }
  void release_events() {
    resolve();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
  }
  void merge_into(ProfBuf& o) {
    resolve();
    for (int i = 0; i < 3; ++i) {
      o.ms[i] += ms[i];
      o.flops[i] += flops[i];
      o.n[i] += n[i];
      ms[i] = flops[i] = 0;
      n[i] = 0;
    }
    o.sweeps += sweeps;
    o.tc_launches += tc_launches;
    sweeps = tc_launches = 0;
  }
};

// An execution lane: a stream, the arena its temporaries come from, a
// pinned host buffer for small readbacks and its profile buffer. Work on one
// lane is stream-ordered, so arena memory released on a lane can be reused
// by that lane at once.
struct Lane {
  Arena* arena = nullptr;
  cudaStream_t stream = nullptr;
  void* pinned = nullptr;
  ProfBuf prof;
  // Host waits on the lane use this event, created with blocking
  // synchronisation: the waiting thread sleeps instead of spinning, so many
  // lanes can wait at once on a few host cores.
  cudaEvent_t wait_ev = nullptr;
  cudaError_t wait() {
    if (!wait_ev) {
      const cudaError_t e =
          cudaEventCreateWithFlags(&wait_ev, cudaEventBlockingSync | cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    const cudaError_t e = cudaEventRecord(wait_ev, stream);
    if (e != cudaSuccess) return e;
    return cudaEventSynchronize(wait_ev);
  }
  void destroy_wait() {
    if (wait_ev) cudaEventDestroy(wait_ev);
    wait_ev = nullptr;
  }
};

}  // namespace

struct qtt_tt;
struct qtt_op;

struct qtt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int prec = QTT_FP64;
  uint64_t seed = 0;
  Arena arena;
  Lane lane0;  // the context's own stream and arena
  std::string err;
  std::atomic<uint64_t> launches{0};
  std::mutex prof_mu;  // guards prof (the merged totals) and lane0.prof
  int concurrent_loads = 1;  // load cases of ls_solve_ceff run side by side
  std::atomic<int> active_lanes{1};  // lanes of the running solve queue (split-K sizing)
  int contraction = QTT_CONTRACT_SIMT;  // FP32 mode: SIMT or split-TF32 tensor-core GEMMs
  int factor = QTT_FACTOR_NATIVE;       // FP32 mode: factorisations in FP32 or in FP64
  int svd_precond = 1;                  // FP64 SVDs beyond shared memory: FP32-preconditioned
  int svd_refine_sweeps = 6;            // FP64 Jacobi sweep cap after the FP32 preconditioner
  double gram_threshold = 2e9;     // TT-SVD: 8 P c min(P, c) above this takes the Gram path
  double jacobi_tol_scale = 1.0;   // Jacobi stop: |a_p^H a_q| <= scale sqrt(m) eps |a_p||a_q|
  int jacobi_max_sweeps32 = 40;    // sweep cap in FP32 mode
  void* pinned = nullptr;  // small host readback buffer
  // Optional per-kernel-class timing (see ProfBuf): totals of the finished
  // lanes; lane0 keeps its own buffer.
  int profiling = 0;
  ProfBuf prof;
  std::map<std::pair<int, int>, qtt_op*> sfft_cache;                            // (n, adjoint)
  std::map<std::tuple<int, double, double, int, double, int>, qtt_op*> gamma_cache;
  // Green operators restricted to xi_1 = 0 (identity x1 cores) for stiffness
  // operators broadcast along x1, when green_broadcast is set
  int green_broadcast = 0;
  std::map<std::tuple<int, double, double, int, double, int>, qtt_op*> gamma_plane_cache;
  // TT of the 15 Green monomial fields per (n, eps, rmax), FP64, in the arena
  struct GreenMono {
    std::vector<void*> cores;
    std::vector<int> ranks;
  };
  std::map<std::tuple<int, double, int, int>, GreenMono> green_mono_cache;  // (n, eps, rmax, scheme)
  size_t esize() const { return prec == QTT_FP64 ? 16 : 8; }
};

static void prof_flush(qtt_ctx* c) {
  c->lane0.prof.merge_into(c->prof);
}

struct ProfScope {
  Lane* ln;
  ProfBuf::Ev e{};
  bool on;
  cudaStream_t s;
  ProfScope(qtt_ctx* ctx, Lane* lane, int cls, double flops)
      : ln(lane), on(ctx->profiling != 0), s(lane->stream) {
    if (!on) return;
    e.cls = cls;
    e.flops = flops;
    e.a = ln->prof.take();
    e.b = ln->prof.take();
    cudaEventRecord(e.a, s);
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(e.b, s);
    ln->prof.evs.push_back(e);
    if (ln->prof.evs.size() > 4096) ln->prof.resolve();
  }
};

struct qtt_tt {
  qtt_ctx* ctx = nullptr;
  Arena* arena = nullptr;  // where the cores live
  int L = 0;
  int dims[QTT_MAX_CORES] = {0};
  int ranks[QTT_MAX_CORES + 1] = {0};
  void* core[QTT_MAX_CORES] = {nullptr};
  long long count(int k) const { return (long long)ranks[k] * dims[k] * ranks[k + 1]; }
};

struct qtt_op {
  qtt_ctx* ctx = nullptr;
  int L = 0;
  int dout[QTT_MAX_CORES] = {0};
  int din[QTT_MAX_CORES] = {0};
  int ranks[QTT_MAX_CORES + 1] = {0};
  int diag[QTT_MAX_CORES] = {0};
  void* core[QTT_MAX_CORES] = {nullptr};
  int n = 0;
  int bcast[3] = {0, 0, 0};  // axes carried by identity cores (raised operators of fields)
  int has_c0 = 0;
  double lame0[2] = {0, 0};
  double C0[36] = {0};
  long long count(int k) const {
    return diag[k] ? (long long)ranks[k] * dout[k] * ranks[k + 1]
                   : (long long)ranks[k] * dout[k] * din[k] * ranks[k + 1];
  }
};

namespace {

// ------------------------------------------------------------------ launch helpers

struct Cplx {
  double re, im;
};

struct MatRef {
  const void* p;
  long long rs, cs, b1, b2, b3;
  int conj;
};
inline MatRef mref(const void* p, long long rs, long long cs, long long b1 = 0, long long b2 = 0,
                   long long b3 = 0, int conj = 0) {
  return MatRef{p, rs, cs, b1, b2, b3, conj};
}

constexpr long long kSMs = 152;  // streaming multiprocessors of a GB300

int grid1d(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

template <typename R>
struct Eng {
  qtt_ctx* c;
  Lane* ln;
  explicit Eng(qtt_ctx* ctx, Lane* lane = nullptr) : c(ctx), ln(lane ? lane : &ctx->lane0) {}
  cudaStream_t st() const { return ln->stream; }
  // After every launch: count it and surface launch errors. With the
  // environment variable QTT_SYNC_EACH_LAUNCH=1 the stream is synchronised
  // too, so that an execution fault is reported against the kernel (name and
  // line of the launch) that caused it.
  void post(const char* what = nullptr, int line = 0) {
    ++c->launches;
    QCHECK(cudaGetLastError());
    static const bool sync_each = [] {
      const char* v = getenv("QTT_SYNC_EACH_LAUNCH");
      return v && v[0] == '1';
    }();
    if (sync_each) {
      const cudaError_t e = cudaStreamSynchronize(st());
      if (e != cudaSuccess)
        throw QttError(QTT_ECUDA, std::string("kernel fault after launch ") +
                                      (what ? what : "?") + " (line " + std::to_string(line) +
                                      "): " + cudaGetErrorString(e));
    }
  }
  Cx<R>* alloc(long long count) { return (Cx<R>*)ln->arena->alloc((size_t)count * sizeof(Cx<R>)); }
  // Host-side launch validation: the largest element offset a strided access
  // reaches must lie inside the workspace allocation the pointer belongs to.
  void check_span(const void* p, long long max_off, const char* what) {
    if (max_off < 0) return;
    long long ext = ln->arena->extent(p);
    if (ext < 0 && ln->arena != &c->arena) ext = c->arena.extent(p);  // shared operators
    if (ext < 0 || (max_off + 1) * (long long)sizeof(Cx<R>) > ext)
      throw QttError(QTT_EINVAL, std::string("launch bounds check failed: ") + what +
                                     " needs " + std::to_string((max_off + 1) * sizeof(Cx<R>)) +
                                     " bytes, allocation has " + std::to_string(ext));
  }
  static long long span(long long n0, long long s0, long long n1 = 1, long long s1 = 0,
                        long long n2 = 1, long long s2 = 0, long long n3 = 1, long long s3 = 0,
                        long long n4 = 1, long long s4 = 0) {
    if (n0 <= 0 || n1 <= 0 || n2 <= 0 || n3 <= 0 || n4 <= 0) return -1;
    return (n0 - 1) * s0 + (n1 - 1) * s1 + (n2 - 1) * s2 + (n3 - 1) * s3 + (n4 - 1) * s4;
  }
  void release(void* p) { ln->arena->release(p); }

  // cuTensorMapEncodeTiled from the driver, looked up once.
  typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                    const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                    const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
      void* f = nullptr;
      cudaDriverEntryPointQueryResult q{};
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                           &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess)
        f = nullptr;
      return (EncodeTiledFn)f;
    }();
    return fn;
  }
  // 2-D FP32 tensor map over a rows x cols row-major array (cols a multiple
  // of 32, so rows start on 128-byte boundaries), box 32 x 128, 128-byte
  // swizzle, zero fill outside.
  static void tc_map(CUtensorMap* m, float* p, long long rows, long long cols) {
    EncodeTiledFn enc = encode_fn();
    QREQ(enc, "tensor-core GEMM: cuTensorMapEncodeTiled unavailable");
    QREQ(((uintptr_t)p & 15) == 0 && cols % 32 == 0, "tensor-core GEMM: misaligned operand");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)tc::BM};
    cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      throw QttError(QTT_ECUDA, "tensor-core GEMM: tensor map encoding failed (" +
                                    std::to_string((int)r) + ")");
  }

  // One unbatched complex FP32 GEMM on the tcgen05 tensor cores (see
  // tc_gemm.cuh): operands split into TF32 hi/lo planes by two preparation
  // kernels, then one 128 x 128 tile per CTA.
  void gemm_tc(int M, int N, int K, MatRef A, MatRef B, void* C, long long c_rs, long long c_cs,
               Cplx alpha, Cplx beta) {
    const int Kp = (2 * K + tc::BK - 1) / tc::BK * tc::BK;
    float* Ah = (float*)ln->arena->alloc((size_t)M * Kp * 4);
    float* Al = (float*)ln->arena->alloc((size_t)M * Kp * 4);
    float* Bh = (float*)ln->arena->alloc((size_t)2 * N * Kp * 4);
    float* Bl = (float*)ln->arena->alloc((size_t)2 * N * Kp * 4);
    int* err = (int*)ln->arena->alloc(sizeof(int));
    QCHECK(cudaMemsetAsync(err, 0, sizeof(int), st()));
    tc::tc_prep_a_kernel<<<grid1d((long long)M * (Kp / 2)), 256, 0, st()>>>(
        (const Cx<float>*)A.p, A.rs, A.cs, A.conj, M, K, Kp, Ah, Al);
    post("tc_prep_a_kernel", __LINE__);
    tc::tc_prep_b_kernel<<<grid1d((long long)N * (Kp / 2)), 256, 0, st()>>>(
        (const Cx<float>*)B.p, B.rs, B.cs, B.conj, N, K, Kp, Bh, Bl);
    post("tc_prep_b_kernel", __LINE__);
    CUtensorMap mAh, mAl, mBh, mBl;
    tc_map(&mAh, Ah, M, Kp);
    tc_map(&mAl, Al, M, Kp);
    tc_map(&mBh, Bh, 2ll * N, Kp);
    tc_map(&mBl, Bl, 2ll * N, Kp);
    static const bool attr = [] {
      cudaFuncSetAttribute(tc::tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           tc::SMEM_BYTES);
      return true;
    }();
    (void)attr;
    tc::TcEpilogue ep{};
    ep.C = (Cx<float>*)C;
    ep.c_rs = c_rs;
    ep.c_cs = c_cs;
    ep.M = M;
    ep.N = N;
    ep.alpha_re = (float)alpha.re;
    ep.alpha_im = (float)alpha.im;
    ep.beta_re = (float)beta.re;
    ep.beta_im = (float)beta.im;
    ep.use_beta = (beta.re != 0.0 || beta.im != 0.0);
    ep.err = err;
    const dim3 grid((unsigned)((M + tc::BM - 1) / tc::BM), (unsigned)((2 * N + tc::BN - 1) / tc::BN));
    {
      ProfScope ps(c, ln, 0, 8.0 * M * N * (double)K);
      tc::tc_gemm_kernel<<<grid, 128, tc::SMEM_BYTES, st()>>>(mAh, mAl, mBh, mBl, Kp, ep);
      post("tc_gemm_kernel", __LINE__);
    }
    if (c->profiling) ln->prof.tc_launches += 1;
    int h = 0;
    QCHECK(cudaMemcpyAsync(ln->pinned, err, sizeof(int), cudaMemcpyDeviceToHost, st()));
    QCHECK(ln->wait());
    memcpy(&h, ln->pinned, sizeof(int));
    ln->arena->release(Ah);
    ln->arena->release(Al);
    ln->arena->release(Bh);
    ln->arena->release(Bl);
    ln->arena->release(err);
    if (h) throw QttError(QTT_ETIMEOUT, "tensor-core GEMM: a device wait ran out (code " +
                                            std::to_string(h) + ")");
  }

  // One GEMM launch: SIMT FP32/FP64 tiles, or in FP32 mode with the
  // split-TF32 contraction setting the tensor-core kernel (same tiling and
  // arguments).
  void launch_gemm(dim3 grid, const GemmArgs& a) {
    if (sizeof(R) == 4 && c->contraction == QTT_CONTRACT_TF32X3) {
      gemm_tf32x3_kernel<<<grid, dim3(128), 0, st()>>>(a);
      post("gemm_tf32x3_kernel", __LINE__);
    } else {
      constexpr int BK = sizeof(R) == 8 ? 8 : 16;
      gemm_kernel<R, 64, 64, BK, 4, 4><<<grid, dim3(256), 0, st()>>>(a);
      post("gemm_kernel", __LINE__);
    }
  }

  // C = alpha op(A) op(B) + beta C over a (nb1, nb2, nb3) batch.
  void gemm(int M, int N, int K, MatRef A, MatRef B, void* C, long long c_rs, long long c_cs,
            long long c_b1, long long c_b2, long long c_b3, int nb1, int nb2, int nb3,
            Cplx alpha = {1, 0}, Cplx beta = {0, 0}, int ksplit = 1, bool allow_tc = false) {
    if (M <= 0 || N <= 0 || nb1 <= 0 || nb2 <= 0 || nb3 <= 0) return;
    if (K <= 0) {
      QREQ(beta.re == 0 && beta.im == 0, "gemm: K = 0 with beta != 0");
      // C = 0
      for (int b1 = 0; b1 < nb1; ++b1)
        for (int b2 = 0; b2 < nb2; ++b2)
          for (int b3 = 0; b3 < nb3; ++b3) {
            CopyArgs a{};
            a.nd = 2;
            a.size[0] = M;
            a.size[1] = N;
            a.in_st[0] = 0;
            a.in_st[1] = 0;
            a.out_st[0] = c_rs;
            a.out_st[1] = c_cs;
            a.scale = 0.0;
            Cx<R>* cp = (Cx<R>*)C + b1 * c_b1 + b2 * c_b2 + b3 * c_b3;
            copy_kernel<R><<<grid1d((long long)M * N), 256, 0, st()>>>(cp, cp, a, (long long)M * N);
            post("copy_kernel", __LINE__);
          }
      return;
    }
    if (sizeof(R) == 4 && allow_tc && c->contraction == QTT_CONTRACT_TC && nb1 == 1 && nb2 == 1 &&
        nb3 == 1 && ksplit == 1 && M >= 64 && N >= 32 && K >= 64) {
      check_span(A.p, span(M, A.rs, K, A.cs), "gemm A");
      check_span(B.p, span(K, B.rs, N, B.cs), "gemm B");
      check_span(C, span(M, c_rs, N, c_cs), "gemm C");
      gemm_tc(M, N, K, A, B, C, c_rs, c_cs, alpha, beta);
      return;
    }
    GemmArgs g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = A.p;
    g.a_rs = A.rs;
    g.a_cs = A.cs;
    g.a_b1 = A.b1;
    g.a_b2 = A.b2;
    g.a_b3 = A.b3;
    g.conjA = A.conj;
    g.B = B.p;
    g.b_rs = B.rs;
    g.b_cs = B.cs;
    g.b_b1 = B.b1;
    g.b_b2 = B.b2;
    g.b_b3 = B.b3;
    g.conjB = B.conj;
    g.C = C;
    g.c_rs = c_rs;
    g.c_cs = c_cs;
    g.c_b1 = c_b1;
    g.c_b2 = c_b2;
    g.c_b3 = c_b3;
    g.nb2 = nb2;
    g.nb3 = nb3;
    g.ksplit = std::max(1, ksplit);
    g.alpha_re = alpha.re;
    g.alpha_im = alpha.im;
    g.beta_re = beta.re;
    g.beta_im = beta.im;
    if (g.ksplit > 1) QREQ(beta.re == 0 && beta.im == 0, "split-K gemm needs beta = 0");
    QREQ(A.rs >= 0 && A.cs >= 0 && B.rs >= 0 && B.cs >= 0 && c_rs >= 0 && c_cs >= 0,
         "gemm: negative stride");
    check_span(A.p, span(M, A.rs, K, A.cs, nb1, A.b1, nb2, A.b2, nb3, A.b3), "gemm A");
    check_span(B.p, span(K, B.rs, N, B.cs, nb1, B.b1, nb2, B.b2, nb3, B.b3), "gemm B");
    check_span(C, span(M, c_rs, N, c_cs, nb1, c_b1, nb2, c_b2, nb3, c_b3), "gemm C");
    constexpr int BM = 64, BN = 64;
    {
      // Few output tiles and a long K (the sketched carry T Psi: M = 2 r,
      // N = r + oversampling, K = r x operator rank): split K over enough
      // CTAs to cover the SMs, partial products summed by a second kernel in
      // a fixed order (deterministic, unlike atomics).
      const long long tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN) * (long long)nb1 * nb2 * nb3;
      // with several lanes running, each GEMM aims at its share of the SMs
      const long long target = std::max<long long>(16, 2 * kSMs / std::max(1, c->active_lanes.load()));
      if (g.ksplit == 1 && tiles < target / 2 && K >= 256) {
        long long ks = std::min<long long>((target + tiles - 1) / tiles, K / 128);
        ks = std::min<long long>(ks, 32);
        const long long nbat = (long long)nb1 * nb2 * nb3;
        if (ks >= 2 && ks * nbat <= 65535 && ks * nbat * M * N <= (16ll << 20)) {
          Cx<R>* part = alloc(ks * nbat * M * N);
          g.ksplit = (int)ks;
          g.nb1 = nb1;
          g.part = part;
          const dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN),
                          (unsigned)(nbat * ks));
          {
            ProfScope ps(c, ln, 0, 8.0 * M * N * (double)K * nbat);
            launch_gemm(grid, g);
            splitk_reduce_kernel<R><<<grid1d(nbat * M * N), 256, 0, st()>>>(
                part, (int)ks, nbat, M, N, nb2, nb3, (Cx<R>*)C, c_rs, c_cs, c_b1, c_b2, c_b3,
                beta.re, beta.im);
            post("splitk_reduce_kernel", __LINE__);
          }
          release(part);
          return;
        }
      }
    }
    const long long per_b1 = (long long)nb2 * nb3 * g.ksplit;
    QREQ(per_b1 <= 65535, "gemm batch too large");
    const int chunk = (int)std::max<long long>(1, 65535 / per_b1);
    const dim3 block(256);
    const long long gx = (M + BM - 1) / BM, gy = (N + BN - 1) / BN;
    QREQ(gy <= 65535, "gemm N too large");
    for (int b0 = 0; b0 < nb1; b0 += chunk) {
      const int nb = std::min(chunk, nb1 - b0);
      GemmArgs h = g;
      h.nb1 = nb;
      h.A = (const Cx<R>*)g.A + b0 * g.a_b1;
      h.B = (const Cx<R>*)g.B + b0 * g.b_b1;
      h.C = (Cx<R>*)g.C + b0 * g.c_b1;
      if (g.ksplit > 1) {
        // zero the outputs first (atomic accumulation)
        for (int b1 = 0; b1 < nb; ++b1)
          for (int b2 = 0; b2 < nb2; ++b2)
            for (int b3 = 0; b3 < nb3; ++b3) {
              CopyArgs a{};
              a.nd = 2;
              a.size[0] = M;
              a.size[1] = N;
              a.out_st[0] = c_rs;
              a.out_st[1] = c_cs;
              a.scale = 0.0;
              Cx<R>* cp = (Cx<R>*)h.C + b1 * c_b1 + b2 * c_b2 + b3 * c_b3;
              copy_kernel<R><<<grid1d((long long)M * N), 256, 0, st()>>>(cp, cp, a,
                                                                          (long long)M * N);
              post("copy_kernel", __LINE__);
            }
      }
      const dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)(nb * per_b1));
      ProfScope ps(c, ln, 0, 8.0 * M * N * (double)K * nb * nb2 * nb3);
      launch_gemm(grid, h);
    }
  }

  // Strided copy out = scale * op(in) over an nd-D index space.
  void copy(const void* in, void* out, int nd, const long long* size, const long long* in_st,
            const long long* out_st, int conj = 0, double scale = 1.0) {
    CopyArgs a{};
    a.nd = nd;
    long long tot = 1;
    for (int d = 0; d < nd; ++d) {
      a.size[d] = size[d];
      a.in_st[d] = in_st[d];
      a.out_st[d] = out_st[d];
      tot *= size[d];
    }
    a.conj = conj;
    a.scale = scale;
    if (tot <= 0) return;
    long long mi = 0, mo = 0;
    for (int d = 0; d < nd; ++d) {
      mi += (size[d] - 1) * in_st[d];
      mo += (size[d] - 1) * out_st[d];
    }
    if (scale != 0.0) check_span(in, mi, "copy in");
    check_span(out, mo, "copy out");
    copy_kernel<R><<<grid1d(tot), 256, 0, st()>>>((const Cx<R>*)in, (Cx<R>*)out, a, tot);
    post("copy_kernel", __LINE__);
  }

  void zero(void* p, long long count) {
    if (count > 0) QCHECK(cudaMemsetAsync(p, 0, (size_t)count * sizeof(Cx<R>), st()));
  }

  // Largest dynamic shared-memory allocation a one-CTA factorisation may
  // use on this device (opt-in limit minus the kernels' static needs).
  static size_t smem_cap() {
    static const size_t cap = [] {  // initialised once, thread-safe
      int dev = 0, v = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      const size_t c = v > 2048 ? (size_t)v - 2048 : 0;
      cudaFuncSetAttribute(qr_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c);
      cudaFuncSetAttribute(jacobi_svd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)c);
      cudaFuncSetAttribute(chol_piv_inv_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)c);
      return c;
    }();
    return cap;
  }

  // Householder QR of the strided m x n matrix A: Q (m x k) and Rm (k x n),
  // column-major, k = min(m, n).
  bool rounding = false;  // inside a TT rounding sweep (QR / truncated SVD)
  bool factor64() const {
    return sizeof(R) == 4 && (c->factor == QTT_FACTOR_FP64 ||
                              (c->factor == QTT_FACTOR_FP64_ROUNDING && rounding));
  }

  // FP32 context with FP64 factorisations: the operand is widened to FP64,
  // factorised by the FP64 kernels on the same lane, and the factors are
  // rounded back to FP32.
  Cx<double>* widen(const Cx<R>* p, long long cnt) {
    Cx<double>* w = (Cx<double>*)ln->arena->alloc((size_t)cnt * sizeof(Cx<double>));
    convert_kernel<R, double><<<grid1d(cnt), 256, 0, st()>>>(p, w, cnt);
    post("convert_kernel", __LINE__);
    return w;
  }
  void narrow(const Cx<double>* w, Cx<R>* p, long long cnt) {
    convert_kernel<double, R><<<grid1d(cnt), 256, 0, st()>>>(w, p, cnt);
    post("convert_kernel", __LINE__);
  }

  void qr(int m, int n, const void* A, long long rs, long long cs, int conj, Cx<R>* Q, Cx<R>* Rm) {
    const int k = std::min(m, n);
    if (factor64()) {
      check_span(A, span(m, rs, n, cs), "qr A");
      Cx<R>* Ac = alloc((long long)m * n);  // column-major FP32 copy, then FP64
      const long long sz[2] = {m, n}, ist[2] = {rs, cs}, ost[2] = {1, m};
      copy(A, Ac, 2, sz, ist, ost, conj);
      Cx<double>* A64 = widen(Ac, (long long)m * n);
      release(Ac);
      Eng<double> d(c, ln);
      Cx<double>* Q64 = d.alloc((long long)m * k);
      Cx<double>* R64 = d.alloc((long long)k * n);
      d.qr(m, n, A64, 1, m, 0, Q64, R64);
      narrow(Q64, Q, (long long)m * k);
      narrow(R64, Rm, (long long)k * n);
      d.release(A64);
      d.release(Q64);
      d.release(R64);
      return;
    }
    check_span(A, span(m, rs, n, cs), "qr A");
    check_span(Q, (long long)m * k - 1, "qr Q");
    check_span(Rm, (long long)k * n - 1, "qr R");
    Cx<R>* W = alloc((long long)m * n);
    R* h = (R*)ln->arena->alloc(sizeof(R) * std::max(1, k));
    Cx<R>* v0 = alloc(std::max(1, k));
    {
      // complex Householder QR with explicit Q: 4 x (2 m n^2 - 2 n^3 / 3) real
      // flops for the factor plus as many for forming Q (LAPACK operation counts)
      const double kk = k;
      ProfScope ps(c, ln, 1, 2.0 * 4.0 * (2.0 * m * kk * kk - 2.0 * kk * kk * kk / 3.0));
      const size_t bytes = (size_t)m * n * sizeof(Cx<R>);
      const bool sm = bytes <= smem_cap();
      qr_kernel<R><<<1, 1024, sm ? bytes : 0, st()>>>(m, n, (const Cx<R>*)A, rs, cs, conj, W, Q,
                                                       Rm, h, v0, sm ? 1 : 0);
      post("qr_kernel", __LINE__);
    }
    release(W);
    release(h);
    release(v0);
  }

  // M (row-major L x L, upper) with P M orthonormal-or-zero columns for the
  // row-major m x L matrix P: Gram matrix by GEMM, then one CTA factors it
  // (pivoted Cholesky stopped at dependent columns) and inverts the factor.
  Cx<R>* orth_factor(const Cx<R>* P, long long m, int L, double tau, int* err) {
    if (factor64()) {
      Cx<double>* P64 = widen(P, m * L);
      Eng<double> d(c, ln);
      Cx<double>* M64 = d.orth_factor(P64, m, L, tau, err);
      d.release(P64);
      Cx<R>* M = alloc((long long)L * L);
      narrow(M64, M, (long long)L * L);
      d.release(M64);
      return M;
    }
    Cx<R>* G = alloc((long long)L * L);
    QREQ(m < (1ll << 31), "orth_factor: too many rows");
    gemm(L, L, (int)m, mref(P, 1, L, 0, 0, 0, 1), mref(P, L, 1), G, L, 1, 0, 0, 0, 1, 1, 1);
    const size_t bytes = ((size_t)L * L + L) * sizeof(Cx<R>);
    const bool sm = bytes <= smem_cap();
    Cx<R>* A = sm ? nullptr : alloc((long long)L * L + L);
    Cx<R>* M = alloc((long long)L * L);
    int* perm = (int*)ln->arena->alloc(sizeof(int) * L);
    {
      const double l3 = (double)L * L * L;
      ProfScope ps(c, ln, 1, 8.0 * l3 / 3.0 * 2.0);
      chol_piv_inv_kernel<R><<<1, 1024, sm ? bytes : 0, st()>>>(L, G, A, M, perm, tau, err,
                                                                sm ? 1 : 0);
      post("chol_piv_inv_kernel", __LINE__);
    }
    release(G);
    if (A) release(A);
    ln->arena->release(perm);
    return M;
  }

  // One-sided Jacobi SVD of the column-major m x n (m >= n) matrix in A
  // (destroyed): U (m x n), sigma (n, descending), V (n x n), all
  // column-major; returns the truncation rank for (delta2, rmax).
  // SVD of a tall m x n matrix: Householder QR first, then Jacobi on the
  // n x n triangular factor (which then fits shared memory far more often),
  // U = Q U_R. Same contract as svd_direct.
  // V == nullptr: the right singular vectors are not accumulated (cheaper
  // rotations); the caller forms what it needs from U by a GEMM.
  int svd(int m, int n, Cx<R>* A, Cx<R>* U, double* sigma, Cx<R>* V, double delta2, int rmax,
          int* cap_hit, bool squares = false) {
    if (factor64()) {
      Cx<double>* A64 = widen(A, (long long)m * n);
      Eng<double> d(c, ln);
      Cx<double>* U64 = d.alloc((long long)m * n);
      Cx<double>* V64 = V ? d.alloc((long long)n * n) : nullptr;
      const int k = d.svd(m, n, A64, U64, sigma, V64, delta2, rmax, cap_hit, squares);
      narrow(U64, U, (long long)m * n);
      if (V) narrow(V64, V, (long long)n * n);
      d.release(A64);
      d.release(U64);
      if (V64) d.release(V64);
      return k;
    }
    if (squares || m <= n + n / 4) return svd_direct(m, n, A, U, sigma, V, delta2, rmax, cap_hit, squares);
    Cx<R>* Q = alloc((long long)m * n);
    Cx<R>* Rf = alloc((long long)n * n);
    qr(m, n, A, 1, m, 0, Q, Rf);
    Cx<R>* UR = alloc((long long)n * n);
    const int k = svd_direct(n, n, Rf, UR, sigma, V, delta2, rmax, cap_hit, false);
    gemm(m, n, n, mref(Q, 1, m), mref(UR, 1, n), U, 1, m, 0, 0, 0, 1, 1, 1);
    release(Q);
    release(Rf);
    release(UR);
    return k;
  }

  // FP64 SVD of a matrix too large for one CTA's shared memory, with an FP32
  // preconditioner (mixed-precision one-sided Jacobi): the FP32 Jacobi kernel
  // (shared memory) gives right singular vectors V32 of the rounded matrix;
  // V32 is made orthonormal in FP64 by one Newton-Schulz step
  // V <- V (3 I - V^H V) / 2 (orthogonality error 1e-7 -> ~1e-14); B = A V has
  // nearly orthogonal columns and the same singular values as A, and the FP64
  // one-sided Jacobi on B converges quadratically from there (a few sweeps
  // instead of tens; columns at the FP32 noise floor, which the FP32 pass
  // leaves unrotated, take a few more). Result: U from B, sigma,
  // V = V_orth V_B. Every kernel is one CTA or a small GEMM grid, so many
  // lanes factorise side by side.
  int svd_precond(int m, int n, Cx<R>* A, Cx<R>* U, double* sigma, Cx<R>* V, double delta2,
                  int rmax, int* cap_hit) {
    Eng<float> f(c, ln);
    f.no_grid = true;
    const long long mn = (long long)m * n, nn = (long long)n * n;
    Cx<float>* A32 = f.alloc(mn);
    convert_kernel<R, float><<<grid1d(mn), 256, 0, st()>>>(A, A32, mn);
    post("convert_kernel", __LINE__);
    Cx<float>* U32 = f.alloc(mn);
    Cx<float>* V32 = f.alloc(nn);
    double* s32 = (double*)ln->arena->alloc(sizeof(double) * n);
    int cap32 = 0;
    f.svd_direct(m, n, A32, U32, s32, V32, 0.0, n, &cap32, false);
    f.release(A32);
    f.release(U32);
    ln->arena->release(s32);
    Cx<R>* V0 = alloc(nn);
    convert_kernel<float, R><<<grid1d(nn), 256, 0, st()>>>(V32, V0, nn);
    post("convert_kernel", __LINE__);
    f.release(V32);
    // Newton-Schulz: X = V0^H V0, Vo = 1.5 V0 - 0.5 V0 X
    Cx<R>* X = alloc(nn);
    gemm(n, n, n, mref(V0, n, 1, 0, 0, 0, 1), mref(V0, 1, n), X, 1, n, 0, 0, 0, 1, 1, 1);
    Cx<R>* Vo = alloc(nn);
    {
      const long long sz[1] = {nn}, st1[1] = {1};
      copy(V0, Vo, 1, sz, st1, st1, 0, 1.5);
    }
    gemm(n, n, n, mref(V0, 1, n), mref(X, 1, n), Vo, 1, n, 0, 0, 0, 1, 1, 1, Cplx{-0.5, 0},
         Cplx{1, 0});
    release(X);
    release(V0);
    // B = A Vo (column-major m x n)
    Cx<R>* B = alloc(mn);
    gemm(m, n, n, mref(A, 1, m), mref(Vo, 1, n), B, 1, m, 0, 0, 0, 1, 1, 1);
    Eng<R> d(c, ln);
    d.no_grid = true;
    d.sweeps_override = c->svd_refine_sweeps;
    Cx<R>* VB = V ? alloc(nn) : nullptr;
    const int k = d.svd_direct(m, n, B, U, sigma, VB, delta2, rmax, cap_hit, false);
    release(B);
    if (V) {
      gemm(n, n, n, mref(Vo, 1, n), mref(VB, 1, n), V, 1, n, 0, 0, 0, 1, 1, 1);
      release(VB);
    }
    release(Vo);
    return k;
  }

  bool no_grid = false;     // never the cooperative Jacobi (several lanes factorise at once)
  int sweeps_override = 0;  // Jacobi sweep cap instead of the precision's default

  int svd_direct(int m, int n, Cx<R>* A, Cx<R>* U, double* sigma, Cx<R>* V, double delta2,
                 int rmax, int* cap_hit, bool squares = false) {
    QREQ(m >= n && n >= 1, "svd: needs m >= n >= 1");
    if (sizeof(R) == 8 && !squares && !no_grid && c->svd_precond && n >= 48 &&
        (size_t)m * n * sizeof(Cx<R>) > smem_cap() && (size_t)m * n * 8 <= Eng<float>::smem_cap())
      return svd_precond(m, n, A, U, sigma, V, delta2, rmax, cap_hit);
    QREQ(n <= 4096, "svd: too many columns");
    check_span(A, (long long)m * n - 1, "svd A");
    check_span(U, (long long)m * n - 1, "svd U");
    const bool want_v = V != nullptr;
    if (want_v) check_span(V, (long long)n * n - 1, "svd V");
    Cx<R>* Vw = want_v ? alloc((long long)n * n) : nullptr;
    int* perm = (int*)ln->arena->alloc(sizeof(int) * n);
    R* snorm = (R*)ln->arena->alloc(sizeof(R) * n);
    int* tr = (int*)ln->arena->alloc(sizeof(int) * 8);
    QCHECK(cudaMemsetAsync(tr, 0, sizeof(int) * 8, st()));
    const R eps = sizeof(R) == 8 ? (R)2.220446049250313e-16 : (R)1.1920929e-7;
    const R tol = eps * (R)std::sqrt((double)m) * (R)c->jacobi_tol_scale;
    const int sweeps = sweeps_override ? sweeps_override
                                       : (sizeof(R) == 8 ? 60 : c->jacobi_max_sweeps32);
    {
      // flops counted for the sweeps actually run are not known here; the
      // profile records one sweep's count (n^2/2 pairs x (3 dots + 2
      // rotations of length m + 2 of length n) x 8 real flops) per launch
      ProfScope ps(c, ln, 2, 0.5 * n * (double)n * (5.0 * m + 2.0 * n) * 8.0);
      const size_t bytes = (size_t)m * n * sizeof(Cx<R>);
      const bool sm = bytes <= smem_cap();
      // the cooperative grid only when one lane runs: a grid starts when all
      // its blocks fit at once, which other lanes' kernels keep delaying
      if (sm || n < 64 || no_grid || c->active_lanes.load() > 1) {
        jacobi_svd_kernel<R><<<1, 1024, sm ? bytes : 0, st()>>>(
            m, n, A, Vw, sigma, perm, snorm, delta2, rmax, tr, sweeps, tol, squares ? 1 : 0,
            sm ? 1 : 0, want_v ? 1 : 0);
        post("jacobi_svd_kernel", __LINE__);
      } else {
        // too large for one CTA's shared memory: spread each round's pairs
        // over the whole GPU (cooperative launch, grid-wide barriers)
        int dev = 0, nsm = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int threads = 128;
        QCHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_grid_kernel<R>,
                                                             threads, 0));
        const int want = ((n + 1) / 2 + (threads / 32) - 1) / (threads / 32);
        const int blocks = std::max(1, std::min(want, nsm * std::max(1, per_sm)));
        int* flags = (int*)ln->arena->alloc(sizeof(int) * (sweeps + 1));
        QCHECK(cudaMemsetAsync(flags, 0, sizeof(int) * (sweeps + 1), st()));
        const R eps_r = sizeof(R) == 8 ? (R)2.220446049250313e-16 : (R)1.1920929e-7;
        R f2 = (R)norm2(A, (long long)m * n);
        R negl = eps_r * eps_r * f2;
        int mm = m, nn = n, ms = sweeps;
        R tl = tol;
        int* swp = tr + 3;
        int wv = want_v ? 1 : 0;
        void* args[] = {&mm, &nn, &A, &Vw, &snorm, &flags, &ms, &tl, &negl, &swp, &wv};
        QCHECK(cudaLaunchCooperativeKernel((void*)jacobi_grid_kernel<R>, dim3(blocks),
                                           dim3(threads), args, 0, st()));
        post("jacobi_grid_kernel", __LINE__);
        jacobi_finish_kernel<R><<<1, 256, 0, st()>>>(n, snorm, sigma, perm, delta2, rmax, tr,
                                                     squares ? 1 : 0, swp);
        post("jacobi_finish_kernel", __LINE__);
        ln->arena->release(flags);
      }
    }
    svd_finish_kernel<R><<<grid1d((long long)m * n + (want_v ? (long long)n * n : 0)), 256, 0, st()>>>(
        m, n, A, Vw, sigma, perm, U, V, tr + 5, want_v ? 1 : 0);
    post("svd_finish_kernel", __LINE__);
    int h[8];
    QCHECK(cudaMemcpyAsync(ln->pinned, tr, sizeof(int) * 8, cudaMemcpyDeviceToHost, st()));
    QCHECK(ln->wait());
    memcpy(h, ln->pinned, sizeof(int) * 8);
    if (Vw) release(Vw);
    release(perm);
    release(snorm);
    release(tr);
    if (h[4]) throw QttError(QTT_ENAN, "svd: NaN in the singular values");
    if (h[5]) throw QttError(QTT_EINVAL, "svd: permutation out of range (kernel skipped access)");
    if (cap_hit) *cap_hit = h[1];
    if (c->profiling) {
      // the launch was counted with one sweep; add the further sweeps run
      if (h[2] > 1) ln->prof.flops[2] += (h[2] - 1) * 0.5 * n * (double)n * (5.0 * m + 2.0 * n) * 8.0;
      ln->prof.sweeps += h[2];
    }
    return h[0];
  }

  double norm2(const void* p, long long count) {
    double* d = (double*)ln->arena->alloc(sizeof(double));
    QCHECK(cudaMemsetAsync(d, 0, sizeof(double), st()));
    norm2_kernel<R><<<grid1d(count), 256, 0, st()>>>((const Cx<R>*)p, count, d);
    post("norm2_kernel", __LINE__);
    QCHECK(cudaMemcpyAsync(ln->pinned, d, sizeof(double), cudaMemcpyDeviceToHost, st()));
    QCHECK(ln->wait());
    double v;
    memcpy(&v, ln->pinned, sizeof(double));
    release(d);
    return v;
  }
};

// ------------------------------------------------------------------ TT / op helpers

qtt_tt* new_tt(qtt_ctx* c, Arena* a, int L, const int* dims) {
  QREQ(L >= 1 && L <= QTT_MAX_CORES, "TT core count out of range");
  qtt_tt* t = new qtt_tt();
  t->ctx = c;
  t->arena = a;
  t->L = L;
  for (int k = 0; k < L; ++k) t->dims[k] = dims[k];
  t->ranks[0] = t->ranks[L] = 1;
  return t;
}

void free_tt(qtt_tt* t) {
  if (!t) return;
  for (int k = 0; k < t->L; ++k) t->arena->release(t->core[k]);
  delete t;
}

void free_op(qtt_op* o) {
  if (!o) return;
  for (int k = 0; k < o->L; ++k) o->ctx->arena.release(o->core[k]);
  delete o;
}

void set_core(qtt_tt* t, int k, void* p) {
  t->arena->release(t->core[k]);
  t->core[k] = p;
}

template <typename R>
qtt_tt* clone_tt(Eng<R>& e, const qtt_tt* x) {
  qtt_tt* y = new_tt(e.c, e.ln->arena, x->L, x->dims);
  for (int k = 0; k <= x->L; ++k) y->ranks[k] = x->ranks[k];
  for (int k = 0; k < x->L; ++k) {
    y->core[k] = e.alloc(x->count(k));
    QCHECK(cudaMemcpyAsync(y->core[k], x->core[k], x->count(k) * sizeof(Cx<R>),
                           cudaMemcpyDeviceToDevice, e.st()));
  }
  return y;
}

// ------------------------------------------------------------------ rounding

// Right-to-left truncated-SVD sweep of a left-orthogonal TT (Sec. 3,
// eq. (rounding_condition_tt)); per-bond threshold delta2 = eps^2 ||x||^2 /
// (L - 1) with ||x|| = ||last core||_F. Result is right-orthogonal.
// Marks an engine as inside a rounding sweep for its lifetime.
template <typename R>
struct RoundingScope {
  Eng<R>& e;
  bool prev;
  explicit RoundingScope(Eng<R>& eng) : e(eng), prev(eng.rounding) { e.rounding = true; }
  ~RoundingScope() { e.rounding = prev; }
};

template <typename R>
int round_right_to_left(Eng<R>& e, qtt_tt* x, double eps, int rmax) {
  RoundingScope<R> rs(e);
  const int L = x->L;
  const double nrm2 = e.norm2(x->core[L - 1], x->count(L - 1));
  const double delta2 = L > 1 ? eps * eps * nrm2 / (double)(L - 1) : 0.0;
  int cap_any = 0;
  for (int k = L - 1; k >= 1; --k) {
    const int r0 = x->ranks[k], d = x->dims[k], r1 = x->ranks[k + 1];
    const int m = d * r1;
    Cx<R>* core = (Cx<R>*)x->core[k];
    int kk, cap = 0;
    Cx<R>* newcore;
    Cx<R>* carry;  // r0 x kk, column-major (ld r0)
    if (m >= r0) {
      // A = M^H (m x r0), M = core as r0 x m row-major. A = U S V^H gives
      // M = V S U^H: new core = U[:, :kk]^H and carry = V S = M U[:, :kk],
      // formed by a GEMM (no rotation accumulation of V needed).
      Cx<R>* A = e.alloc((long long)m * r0);
      const long long sz[2] = {r0, m}, ist[2] = {m, 1}, ost[2] = {m, 1};
      e.copy(core, A, 2, sz, ist, ost, 1);  // A[j + c m] = conj(M[c, j])
      Cx<R>* U = e.alloc((long long)m * r0);
      double* sig = (double*)e.ln->arena->alloc(sizeof(double) * r0);
      kk = e.svd(m, r0, A, U, sig, nullptr, delta2, rmax, &cap);
      newcore = e.alloc((long long)kk * m);
      const long long s2[2] = {kk, m}, i2[2] = {m, 1}, o2[2] = {m, 1};
      e.copy(U, newcore, 2, s2, i2, o2, 1);
      carry = e.alloc((long long)r0 * kk);  // column-major r0 x kk
      e.gemm(r0, kk, m, mref(core, m, 1), mref(U, 1, m), carry, 1, r0, 0, 0, 0, 1, 1, 1);
      e.release(A);
      e.release(U);
      e.ln->arena->release(sig);
    } else {
      // M tall (r0 x m): Jacobi on its columns, M = U S V^H.
      Cx<R>* A = e.alloc((long long)r0 * m);
      const long long sz[2] = {m, r0}, ist[2] = {1, m}, ost[2] = {r0, 1};
      e.copy(core, A, 2, sz, ist, ost, 0);  // column-major copy of M
      Cx<R>* U = e.alloc((long long)r0 * m);
      Cx<R>* V = e.alloc((long long)m * m);
      double* sig = (double*)e.ln->arena->alloc(sizeof(double) * m);
      kk = e.svd(r0, m, A, U, sig, V, delta2, rmax, &cap);
      newcore = e.alloc((long long)kk * m);
      const long long s2[2] = {kk, m}, i2[2] = {m, 1}, o2[2] = {m, 1};
      e.copy(V, newcore, 2, s2, i2, o2, 1);  // V^H rows
      carry = U;
      scale_cols_kernel<R><<<grid1d((long long)r0 * kk), 256, 0, e.st()>>>(U, r0, kk, sig);
      e.post("scale_cols_kernel", __LINE__);
      e.release(A);
      e.release(V);
      e.release(sig);
    }
    cap_any |= cap;
    // core_{k-1} (rp, dp, r0) <- core_{k-1} * carry (r0 x kk)
    const int rp = x->ranks[k - 1], dp = x->dims[k - 1];
    Cx<R>* prev = e.alloc((long long)rp * dp * kk);
    e.gemm(rp * dp, kk, r0, mref(x->core[k - 1], r0, 1), mref(carry, 1, r0), prev, kk, 1, 0, 0, 0,
           1, 1, 1);
    e.release(carry);
    set_core(x, k, newcore);
    set_core(x, k - 1, prev);
    x->ranks[k] = kk;
  }
  return cap_any;
}

// Left-to-right Householder QR sweep (orthogonalisation step of rounding).
template <typename R>
void orthogonalize_left(Eng<R>& e, qtt_tt* x) {
  RoundingScope<R> rs(e);
  const int L = x->L;
  for (int k = 0; k < L - 1; ++k) {
    const int r0 = x->ranks[k], d = x->dims[k], r1 = x->ranks[k + 1];
    const int m = r0 * d, kq = std::min(m, r1);
    Cx<R>* Q = e.alloc((long long)m * kq);
    Cx<R>* Rm = e.alloc((long long)kq * r1);
    e.qr(m, r1, x->core[k], r1, 1, 0, Q, Rm);
    Cx<R>* nc = e.alloc((long long)m * kq);
    const long long sz[2] = {m, kq}, ist[2] = {1, m}, ost[2] = {kq, 1};
    e.copy(Q, nc, 2, sz, ist, ost);
    const int d2 = x->dims[k + 1], r2 = x->ranks[k + 2];
    Cx<R>* next = e.alloc((long long)kq * d2 * r2);
    e.gemm(kq, d2 * r2, r1, mref(Rm, 1, kq), mref(x->core[k + 1], d2 * r2, 1), next, d2 * r2, 1,
           0, 0, 0, 1, 1, 1);
    e.release(Q);
    e.release(Rm);
    set_core(x, k, nc);
    set_core(x, k + 1, next);
    x->ranks[k + 1] = kq;
  }
}

template <typename R>
int round_full(Eng<R>& e, qtt_tt* x, double eps, int rmax) {
  orthogonalize_left(e, x);
  return round_right_to_left(e, x, eps, rmax);
}

// ------------------------------------------------------------------ sketched product

long long prod_dims(const int* d, int a, int b) {  // prod d[a..b-1], saturating
  long long p = 1;
  for (int i = a; i < b; ++i) {
    p *= d[i];
    if (p > (1ll << 40)) return 1ll << 40;
  }
  return p;
}

// QTT_CHECK_FINITE=1 in the environment: intermediate results are checked
// for non-finite values and the first one is reported by where it arose.
bool debug_finite() {
  static const bool on = [] {
    const char* v = getenv("QTT_CHECK_FINITE");
    return v && v[0] == '1';
  }();
  return on;
}

// y = A x by successive randomized compression (see the oracle's
// tto_apply_sketched for the statement): right-to-left random sketches Psi,
// then left-to-right QR of the sketched carries. Output left-orthogonal.
template <typename R>
qtt_tt* apply_sketched(Eng<R>& e, const qtt_op* A, const qtt_tt* x, int ell, int apply_id) {
  const int L = x->L;
  QREQ(A->L == L, "operator and TT have different core counts");
  for (int k = 0; k < L; ++k) QREQ(A->din[k] == x->dims[k], "operator input dims mismatch");
  int lr[QTT_MAX_CORES + 1];
  lr[0] = lr[L] = 1;
  for (int b = 1; b < L; ++b) {
    long long v = std::min<long long>(ell, (long long)A->ranks[b] * x->ranks[b]);
    v = std::min(v, prod_dims(A->dout, 0, b));
    v = std::min(v, prod_dims(A->dout, b, L));
    lr[b] = (int)std::max<long long>(1, v);
  }
  // ---- right-to-left sketches: Psi[b] has layout (s, a, l) = (x->ranks[b], A->ranks[b], lr[b])
  std::vector<Cx<R>*> psi(L + 1, nullptr);
  // Mk[k]: Psi_k Mk[k] is an orthonormal basis of range(Psi_k) followed by
  // zero columns (dependent directions). The next sketch is taken of that basis (Mk
  // folded into the next random core) so that the environments' condition
  // number does not compound over the cores (a product of random cores loses
  // ~10x per core, more than single precision can hold after a few cores).
  std::vector<Cx<R>*> Mk(L + 1, nullptr);
  // relative Cholesky pivot below which a sketch direction is dropped: the
  // reach of the Gram matrix's working precision (FP64 factors in an FP32
  // context see FP32 data, whose own rounding sets the floor)
  const double drop_tau = sizeof(R) == 8 ? 1e-11 : (e.factor64() ? 1e-9 : 1e-6);
  int* oerr = (int*)e.ln->arena->alloc(sizeof(int));
  QCHECK(cudaMemsetAsync(oerr, 0, sizeof(int), e.st()));
  psi[L] = e.alloc(1);
  {
    Cx<R> one = mk<R>(1, 0);
    QCHECK(cudaMemcpyAsync(psi[L], &one, sizeof(one), cudaMemcpyHostToDevice, e.st()));
  }
  for (int k = L - 1; k >= 1; --k) {
    const int S0 = x->ranks[k], S1 = x->ranks[k + 1], A0 = A->ranks[k], A1 = A->ranks[k + 1];
    const int L0 = lr[k], L1 = lr[k + 1], Din = A->din[k], Dout = A->dout[k];
    const bool dg = A->diag[k];
    Cx<R>* Om = e.alloc((long long)L0 * Dout * L1);
    sketch_kernel<R><<<grid1d((long long)L0 * Dout * L1), 256, 0, e.st()>>>(
        Om, (long long)L0 * Dout * L1, e.c->seed, k, apply_id);
    e.post("sketch_kernel", __LINE__);
    if (Mk[k + 1]) {
      // sketch of Psi_{k+1} M_{k+1}: Om'[(l0 o), j] = sum_l1 Om[(l0 o), l1] M[j, l1]
      Cx<R>* Om2 = e.alloc((long long)L0 * Dout * L1);
      e.gemm(L0 * Dout, L1, L1, mref(Om, L1, 1), mref(Mk[k + 1], 1, L1), Om2, L1, 1, 0, 0, 0, 1,
             1, 1);
      e.release(Om);
      Om = Om2;
    }
    // S1: XP[i][s0][a1 l1] = sum_s1 X[s0, i, s1] Psi[s1, (a1 l1)]
    Cx<R>* XP = e.alloc((long long)Din * S0 * A1 * L1);
    e.gemm(S0, A1 * L1, S1, mref(x->core[k], (long long)Din * S1, 1, S1), mref(psi[k + 1], (long long)A1 * L1, 1),
           XP, (long long)A1 * L1, 1, (long long)S0 * A1 * L1, 0, 0, Din, 1, 1);
    Cx<R>* Pk = e.alloc((long long)S0 * A0 * L0);
    if (dg) {
      // S2: U[s0][i][a1][l0] = sum_l1 XP[i][s0][a1][l1] Om[l0, i, l1]
      Cx<R>* U = e.alloc((long long)S0 * Din * A1 * L0);
      e.gemm(A1, L0, L1, mref(XP, L1, 1, (long long)A1 * L1, (long long)S0 * A1 * L1),
             mref(Om, 1, (long long)Din * L1, 0, L1), U, L0, 1, (long long)Din * A1 * L0,
             (long long)A1 * L0, 0, S0, Din, 1);
      // S3: Psi_k[s0][a0][l0] = sum_{(i a1)} w[a0, (i a1)] U[s0][(i a1)][l0]
      e.gemm(A0, L0, Din * A1, mref(A->core[k], (long long)Din * A1, 1),
             mref(U, L0, 1, (long long)Din * A1 * L0), Pk, L0, 1, (long long)A0 * L0, 0, 0, S0, 1,
             1);
      e.release(U);
    } else {
      Cx<R>* U = e.alloc((long long)S0 * Dout * Din * A1 * L0);
      e.gemm(A1, L0, L1, mref(XP, L1, 1, (long long)A1 * L1, 0, (long long)S0 * A1 * L1),
             mref(Om, 1, (long long)Dout * L1, 0, L1, 0), U, L0, 1,
             (long long)Dout * Din * A1 * L0, (long long)Din * A1 * L0, (long long)A1 * L0, S0,
             Dout, Din);
      e.gemm(A0, L0, Dout * Din * A1, mref(A->core[k], (long long)Dout * Din * A1, 1),
             mref(U, L0, 1, (long long)Dout * Din * A1 * L0), Pk, L0, 1, (long long)A0 * L0, 0, 0,
             S0, 1, 1);
      e.release(U);
    }
    e.release(XP);
    e.release(Om);
    {
      // Psi_k grows like sqrt(ell) per core (a product of random sketches):
      // rescale it to unit norm on the device. The compression below uses
      // only the range of T Psi, so the result does not change.
      const long long cnt = (long long)S0 * A0 * L0;
      double* nrm = (double*)e.ln->arena->alloc(sizeof(double));
      QCHECK(cudaMemsetAsync(nrm, 0, sizeof(double), e.st()));
      norm2_kernel<R><<<grid1d(cnt), 256, 0, e.st()>>>(Pk, cnt, nrm);
      e.post("norm2_kernel", __LINE__);
      scale_inv_norm_kernel<R><<<grid1d(cnt), 256, 0, e.st()>>>(Pk, cnt, nrm);
      e.post("scale_inv_norm_kernel", __LINE__);
      e.ln->arena->release(nrm);
    }
    psi[k] = Pk;
    Mk[k] = e.orth_factor(Pk, (long long)S0 * A0, L0, drop_tau, oerr);
    if (debug_finite()) {
      const double a = e.norm2(Pk, (long long)S0 * A0 * L0), b = e.norm2(Mk[k], (long long)L0 * L0);
      if (!std::isfinite(a) || !std::isfinite(b))
        throw QttError(QTT_ENAN, "sketched product: non-finite sketch at core " + std::to_string(k) +
                                     " (|Psi|^2 " + std::to_string(a) + ", |M|^2 " +
                                     std::to_string(b) + ")");
    }
  }
  // ---- left-to-right compression
  qtt_tt* y = new_tt(e.c, e.ln->arena, L, A->dout);
  Cx<R>* C = e.alloc(1);  // carry (R, S0, A0)
  {
    Cx<R> one = mk<R>(1, 0);
    QCHECK(cudaMemcpyAsync(C, &one, sizeof(one), cudaMemcpyHostToDevice, e.st()));
  }
  int Rr = 1;
  for (int k = 0; k < L; ++k) {
    const int S0 = x->ranks[k], S1 = x->ranks[k + 1], A0 = A->ranks[k], A1 = A->ranks[k + 1];
    const int Din = A->din[k], Dout = A->dout[k];
    const bool dg = A->diag[k];
    // CW[r, s0, (o, i), a1] = sum_a0 C[r, s0, a0] W[a0, ...]
    const int wcols = dg ? Din * A1 : Dout * Din * A1;
    Cx<R>* CW = e.alloc((long long)Rr * S0 * wcols);
    e.gemm(Rr * S0, wcols, A0, mref(C, A0, 1), mref(A->core[k], wcols, 1), CW, wcols, 1, 0, 0, 0,
           1, 1, 1);
    // T[o][r][s1][a1]
    Cx<R>* T = e.alloc((long long)Dout * Rr * S1 * A1);
    if (dg) {
      // T[i][r] (s1 x a1) = sum_s0 X[s0, i, s1] CW[r, s0, i, a1]
      e.gemm(S1, A1, S0, mref(x->core[k], 1, (long long)Din * S1, S1, 0),
             mref(CW, (long long)Din * A1, 1, A1, (long long)S0 * Din * A1), T, A1, 1,
             (long long)Rr * S1 * A1, (long long)S1 * A1, 0, Din, Rr, 1);
    } else {
      for (int i = 0; i < Din; ++i) {
        // T[o][r] += sum_s0 X[s0, i, s1] CW[r, s0, o, i, a1]
        e.gemm(S1, A1, S0, mref((const Cx<R>*)x->core[k] + (long long)i * S1, 1, (long long)Din * S1),
               mref((const Cx<R>*)CW + (long long)i * A1, (long long)Dout * Din * A1, 1,
                    (long long)Din * A1, (long long)S0 * Dout * Din * A1),
               T, A1, 1, (long long)Rr * S1 * A1, (long long)S1 * A1, 0, Dout, Rr, 1, Cplx{1, 0},
               Cplx{i == 0 ? 0.0 : 1.0, 0});
      }
    }
    e.release(CW);
    e.release(C);
    if (k == L - 1) {
      // Y[r][o][0] = T[o][r]
      Cx<R>* Y = e.alloc((long long)Rr * Dout);
      const long long sz[2] = {Rr, Dout}, ist[2] = {1, Rr}, ost[2] = {Dout, 1};
      e.copy(T, Y, 2, sz, ist, ost);
      y->core[k] = Y;
      y->ranks[k] = Rr;
      e.release(T);
      break;
    }
    const int L1 = lr[k + 1];
    const int mz = Dout * Rr;
    Cx<R>* Z0 = e.alloc((long long)mz * L1);
    e.gemm(mz, L1, S1 * A1, mref(T, (long long)S1 * A1, 1), mref(psi[k + 1], L1, 1), Z0, L1, 1, 0,
           0, 0, 1, 1, 1, Cplx{1, 0}, Cplx{0, 0}, 1, true);
    e.release(psi[k + 1]);
    psi[k + 1] = nullptr;
    // Z = T Psi_{k+1} M_{k+1}: the sketch of T by the orthonormal basis
    Cx<R>* Z = e.alloc((long long)mz * L1);
    e.gemm(mz, L1, L1, mref(Z0, L1, 1), mref(Mk[k + 1], L1, 1), Z, L1, 1, 0, 0, 0, 1, 1, 1);
    e.release(Z0);
    e.release(Mk[k + 1]);
    Mk[k + 1] = nullptr;
    const int kq = std::min(mz, L1);
    Cx<R>* Q = e.alloc((long long)mz * kq);
    Cx<R>* Rm = e.alloc((long long)kq * L1);
    if (debug_finite() && !std::isfinite(e.norm2(Z, (long long)mz * L1)))
      throw QttError(QTT_ENAN, "sketched product: non-finite compression matrix at core " +
                                   std::to_string(k));
    e.qr(mz, L1, Z, L1, 1, 0, Q, Rm);
    if (debug_finite() && !std::isfinite(e.norm2(Q, (long long)mz * kq)))
      throw QttError(QTT_ENAN, "sketched product: non-finite QR factor at core " + std::to_string(k));
    // a dropped sketch direction gives an exactly zero column of Z: its
    // reflector direction is arbitrary, so it is removed from the output
    zero_dead_cols_kernel<R><<<grid1d((long long)mz * kq), 256, 0, e.st()>>>(Q, mz, kq, Rm, kq);
    e.post("zero_dead_cols_kernel", __LINE__);
    e.release(Z);
    e.release(Rm);
    // carry' (kq, S1, A1) = Q^H T
    Cx<R>* Cn = e.alloc((long long)kq * S1 * A1);
    e.gemm(kq, S1 * A1, mz, mref(Q, mz, 1, 0, 0, 0, 1), mref(T, (long long)S1 * A1, 1), Cn,
           (long long)S1 * A1, 1, 0, 0, 0, 1, 1, 1, Cplx{1, 0}, Cplx{0, 0}, 1, true);
    // Y[r][o][m] = Q[(o R + r) + m mz]
    Cx<R>* Y = e.alloc((long long)Rr * Dout * kq);
    const long long sz[3] = {Rr, Dout, kq}, ist[3] = {1, Rr, mz},
                    ost[3] = {(long long)Dout * kq, kq, 1};
    e.copy(Q, Y, 3, sz, ist, ost);
    e.release(Q);
    e.release(T);
    y->core[k] = Y;
    y->ranks[k] = Rr;
    C = Cn;
    Rr = kq;
  }
  y->ranks[0] = 1;
  y->ranks[L] = 1;
  for (int b = 0; b <= L; ++b) {
    if (psi[b]) e.release(psi[b]);
    if (Mk[b]) e.release(Mk[b]);
  }
  int herr = 0;
  QCHECK(cudaMemcpyAsync(e.ln->pinned, oerr, sizeof(int), cudaMemcpyDeviceToHost, e.st()));
  QCHECK(e.ln->wait());
  memcpy(&herr, e.ln->pinned, sizeof(int));
  e.ln->arena->release(oerr);
  if (herr) {
    free_tt(y);
    throw QttError(QTT_ENAN, herr == 2 ? "sketched product: non-finite orthonormalising factor"
                                       : "sketched product: non-finite sketch environment");
  }
  return y;
}

// alpha a + beta b as a TT of rank r(a) + r(b) (Table 2, "x + y").
template <typename R>
qtt_tt* tt_add(Eng<R>& e, const qtt_tt* a, const qtt_tt* b, double alpha, double beta) {
  const int L = a->L;
  QREQ(b->L == L && L >= 2, "tt_add: core counts differ or L < 2");
  for (int k = 0; k < L; ++k) QREQ(a->dims[k] == b->dims[k], "tt_add: dims differ");
  qtt_tt* y = new_tt(e.c, e.ln->arena, L, a->dims);
  for (int k = 1; k < L; ++k) y->ranks[k] = a->ranks[k] + b->ranks[k];
  for (int k = 0; k < L; ++k) {
    const int d = a->dims[k];
    const int ra0 = a->ranks[k], ra1 = a->ranks[k + 1], rb0 = b->ranks[k], rb1 = b->ranks[k + 1];
    const int y0 = y->ranks[k], y1 = y->ranks[k + 1];
    Cx<R>* Y = e.alloc((long long)y0 * d * y1);
    e.zero(Y, (long long)y0 * d * y1);
    // place a at (0, :, 0), b at (row off, :, col off)
    const int boff0 = (k == 0) ? 0 : ra0;
    const int boff1 = (k == L - 1) ? 0 : ra1;
    const double sa = (k == 0) ? alpha : 1.0, sb = (k == 0) ? beta : 1.0;
    {
      const long long sz[3] = {ra0, d, ra1}, ist[3] = {(long long)d * ra1, ra1, 1},
                      ost[3] = {(long long)d * y1, y1, 1};
      e.copy(a->core[k], Y, 3, sz, ist, ost, 0, sa);
    }
    {
      const long long sz[3] = {rb0, d, rb1}, ist[3] = {(long long)d * rb1, rb1, 1},
                      ost[3] = {(long long)d * y1, y1, 1};
      e.copy(b->core[k], Y + (long long)boff0 * d * y1 + boff1, 3, sz, ist, ost, 0, sb);
    }
    y->core[k] = Y;
  }
  return y;
}

// <a, b> with FP64 transfer matrices.
template <typename R>
void tt_dot(Eng<R>& e, const qtt_tt* a, const qtt_tt* b, double* re, double* im) {
  Eng<double> d(e.c, e.ln);  // same lane: stream and arena of the caller
  const int L = a->L;
  QREQ(b->L == L, "dot: core counts differ");
  Cx<double>* E = d.alloc(1);
  {
    Cx<double> one = mk<double>(1, 0);
    QCHECK(cudaMemcpyAsync(E, &one, sizeof(one), cudaMemcpyHostToDevice, e.st()));
  }
  for (int k = 0; k < L; ++k) {
    QREQ(a->dims[k] == b->dims[k], "dot: dims differ");
    const int ra = a->ranks[k], rb = b->ranks[k], pa = a->ranks[k + 1], pb = b->ranks[k + 1],
              D = a->dims[k];
    const Cx<double>* Ak = (const Cx<double>*)a->core[k];
    const Cx<double>* Bk = (const Cx<double>*)b->core[k];
    Cx<double>* tA = nullptr;
    Cx<double>* tB = nullptr;
    if (sizeof(R) != 8) {
      tA = d.alloc(a->count(k));
      tB = d.alloc(b->count(k));
      convert_kernel<R, double><<<grid1d(a->count(k)), 256, 0, e.st()>>>(
          (const Cx<R>*)a->core[k], tA, a->count(k));
      e.post("convert_kernel", __LINE__);
      convert_kernel<R, double><<<grid1d(b->count(k)), 256, 0, e.st()>>>(
          (const Cx<R>*)b->core[k], tB, b->count(k));
      e.post("convert_kernel", __LINE__);
      Ak = tA;
      Bk = tB;
    }
    // EB[ra][i pb] = E (ra x rb) B (rb x (i pb))
    Cx<double>* EB = d.alloc((long long)ra * D * pb);
    d.gemm(ra, D * pb, rb, mref(E, rb, 1), mref(Bk, (long long)D * pb, 1), EB, (long long)D * pb, 1,
           0, 0, 0, 1, 1, 1);
    // F (pa x pb) = A^H ((ra i) x pa)^H EB ((ra i) x pb)
    Cx<double>* F = d.alloc((long long)pa * pb);
    d.gemm(pa, pb, ra * D, mref(Ak, 1, pa, 0, 0, 0, 1), mref(EB, pb, 1), F, pb, 1, 0, 0, 0, 1, 1, 1);
    d.release(EB);
    d.release(E);
    if (tA) d.release(tA);
    if (tB) d.release(tB);
    E = F;
  }
  double h[2];
  QCHECK(cudaMemcpyAsync(e.ln->pinned, E, 16, cudaMemcpyDeviceToHost, e.st()));
  QCHECK(e.ln->wait());
  memcpy(h, e.ln->pinned, 16);
  d.release(E);
  *re = h[0];
  *im = h[1];
}

// Grid mean of (A x): first core full (1, Dout, Din, a1), binary cores raised.
template <typename R>
void op_mean(Eng<R>& e, const qtt_op* A, const qtt_tt* x, std::vector<double>& out) {
  Eng<double> d(e.c, e.ln);  // same lane: stream and arena of the caller
  const int L = x->L;
  QREQ(A->L == L, "mean: core counts differ");
  QREQ(!A->diag[0], "mean: first operator core must be full");
  for (int k = 1; k < L; ++k) QREQ(A->diag[k], "mean: binary operator cores must be raised");
  auto to64 = [&](const void* p, long long cnt) -> Cx<double>* {
    Cx<double>* t = d.alloc(cnt);
    if (sizeof(R) == 8) {
      QCHECK(cudaMemcpyAsync(t, p, cnt * 16, cudaMemcpyDeviceToDevice, e.st()));
    } else {
      convert_kernel<R, double><<<grid1d(cnt), 256, 0, e.st()>>>((const Cx<R>*)p, t, cnt);
      e.post("convert_kernel", __LINE__);
    }
    return t;
  };
  const int Do = A->dout[0], Di = A->din[0], a1 = A->ranks[1], s1 = x->ranks[1];
  Cx<double>* W0 = to64(A->core[0], A->count(0));
  Cx<double>* X0 = to64(x->core[0], x->count(0));
  // V[I][a1][s1] = sum_J W0[I, J, a1] X0[J, s1]
  Cx<double>* V = d.alloc((long long)Do * a1 * s1);
  d.gemm(a1, s1, Di, mref(W0, 1, a1, (long long)Di * a1), mref(X0, s1, 1), V, s1, 1,
         (long long)a1 * s1, 0, 0, Do, 1, 1);
  d.release(W0);
  d.release(X0);
  int Ar = a1, Sr = s1;
  for (int k = 1; k < L; ++k) {
    const int D = x->dims[k], B = A->ranks[k + 1], T = x->ranks[k + 1];
    Cx<double>* Wk = to64(A->core[k], A->count(k));
    Cx<double>* Xk = to64(x->core[k], x->count(k));
    // VX[I][a][i t] = V[I][a][s] X[s, (i t)]
    Cx<double>* VX = d.alloc((long long)Do * Ar * D * T);
    d.gemm(Do * Ar, D * T, Sr, mref(V, Sr, 1), mref(Xk, (long long)D * T, 1), VX, (long long)D * T,
           1, 0, 0, 0, 1, 1, 1);
    // V'[I][b][t] = 1/2 sum_{(a i)} w[(a i), b] VX[I][(a i)][t]
    Cx<double>* Vn = d.alloc((long long)Do * B * T);
    d.gemm(B, T, Ar * D, mref(Wk, 1, B), mref(VX, T, 1, (long long)Ar * D * T), Vn, T, 1,
           (long long)B * T, 0, 0, Do, 1, 1, Cplx{0.5, 0});
    d.release(VX);
    d.release(V);
    d.release(Wk);
    d.release(Xk);
    V = Vn;
    Ar = B;
    Sr = T;
  }
  out.assign(2 * Do, 0.0);
  std::vector<double> h(2 * Do);
  QCHECK(cudaMemcpyAsync(e.ln->pinned, V, 16 * Do, cudaMemcpyDeviceToHost, e.st()));
  QCHECK(e.ln->wait());
  memcpy(h.data(), e.ln->pinned, 16 * Do);
  d.release(V);
  out = h;
}

// Bilinear grid mean of y^T A x (no conjugation) by an FP64 transfer sweep:
// first core full (1, Do, Di, a1), binary cores raised.
template <typename R>
void op_sandwich(Eng<R>& e, const qtt_op* A, const qtt_tt* y, const qtt_tt* x, double* out2) {
  Eng<double> d(e.c, e.ln);
  const int L = x->L;
  QREQ(A->L == L && y->L == L, "sandwich: core counts differ");
  QREQ(!A->diag[0], "sandwich: first operator core must be full");
  for (int k = 1; k < L; ++k) QREQ(A->diag[k], "sandwich: binary operator cores must be raised");
  for (int k = 0; k < L; ++k)
    QREQ(x->dims[k] == A->din[k] && y->dims[k] == A->dout[k], "sandwich: dims differ");
  auto to64 = [&](const void* p, long long cnt) -> Cx<double>* {
    Cx<double>* t = d.alloc(cnt);
    if (sizeof(R) == 8) {
      QCHECK(cudaMemcpyAsync(t, p, cnt * 16, cudaMemcpyDeviceToDevice, e.st()));
    } else {
      convert_kernel<R, double><<<grid1d(cnt), 256, 0, e.st()>>>((const Cx<R>*)p, t, cnt);
      e.post("convert_kernel", __LINE__);
    }
    return t;
  };
  const int Do = A->dout[0], Di = A->din[0], A1 = A->ranks[1], T1 = x->ranks[1], S1 = y->ranks[1];
  Cx<double>* W0 = to64(A->core[0], A->count(0));
  Cx<double>* X0 = to64(x->core[0], x->count(0));
  Cx<double>* Y0 = to64(y->core[0], y->count(0));
  // XW[I][a][t] = sum_J W0[I, J, a] X0[J, t]
  Cx<double>* XW = d.alloc((long long)Do * A1 * T1);
  d.gemm(A1, T1, Di, mref(W0, 1, A1, (long long)Di * A1), mref(X0, T1, 1), XW, T1, 1,
         (long long)A1 * T1, 0, 0, Do, 1, 1);
  // V[s][(a t)] = sum_I Y0[I, s] XW[I][(a t)]
  Cx<double>* V = d.alloc((long long)S1 * A1 * T1);
  d.gemm(S1, A1 * T1, Do, mref(Y0, 1, S1), mref(XW, (long long)A1 * T1, 1), V,
         (long long)A1 * T1, 1, 0, 0, 0, 1, 1, 1);
  d.release(W0);
  d.release(X0);
  d.release(Y0);
  d.release(XW);
  int S = S1, Ar = A1, T = T1;
  for (int k = 1; k < L; ++k) {
    const int D = x->dims[k], Sp = y->ranks[k + 1], B = A->ranks[k + 1], Tp = x->ranks[k + 1];
    Cx<double>* Wk = to64(A->core[k], A->count(k));
    Cx<double>* Xk = to64(x->core[k], x->count(k));
    Cx<double>* Yk = to64(y->core[k], y->count(k));
    // VX[(s a)][(i t')] = V[(s a)][t] X[t][(i t')]
    Cx<double>* VX = d.alloc((long long)S * Ar * D * Tp);
    d.gemm(S * Ar, D * Tp, T, mref(V, T, 1), mref(Xk, (long long)D * Tp, 1), VX, (long long)D * Tp,
           1, 0, 0, 0, 1, 1, 1);
    // VXW[s][i][b][t'] = sum_a w[a, i, b] VX[s][a][i][t']   (batch s, i)
    Cx<double>* VXW = d.alloc((long long)S * D * B * Tp);
    d.gemm(B, Tp, Ar, mref(Wk, 1, (long long)D * B, 0, B),
           mref(VX, (long long)D * Tp, 1, (long long)Ar * D * Tp, Tp), VXW, Tp, 1,
           (long long)D * B * Tp, (long long)B * Tp, 0, S, D, 1);
    // V'[s'][(b t')] = 1/2 sum_{(s i)} Y[(s i), s'] VXW[(s i)][(b t')]
    Cx<double>* Vn = d.alloc((long long)Sp * B * Tp);
    d.gemm(Sp, B * Tp, S * D, mref(Yk, 1, Sp), mref(VXW, (long long)B * Tp, 1), Vn,
           (long long)B * Tp, 1, 0, 0, 0, 1, 1, 1, Cplx{0.5, 0});
    d.release(VX);
    d.release(VXW);
    d.release(V);
    d.release(Wk);
    d.release(Xk);
    d.release(Yk);
    V = Vn;
    S = Sp;
    Ar = B;
    T = Tp;
  }
  QCHECK(cudaMemcpyAsync(e.ln->pinned, V, 16, cudaMemcpyDeviceToHost, e.st()));
  QCHECK(e.ln->wait());
  memcpy(out2, e.ln->pinned, 16);
  d.release(V);
}

// ------------------------------------------------------------------ TT-SVD (preprocessing, FP64)

// TT-SVD of a dense complex tensor T (dims[0..L-1], row-major) right to left:
// at core j the unfolding M (P x c), c = d_j r_{j+1}, gives the Gram matrix
// G = M^H M; its eigenvectors (one-sided Jacobi of G) V and eigenvalues
// lambda = sigma^2 decide the rank by the tail rule, core j = V[:, :k]^H and
// the carry is M V[:, :k]. T is consumed (overwritten).
std::vector<Cx<double>*> tt_svd_device(Eng<double>& e, Cx<double>* T, const std::vector<int>& dims,
                                       double eps, int rmax, std::vector<int>& ranks,
                                       bool consume_T = false) {
  const int L = (int)dims.size();
  std::vector<Cx<double>*> cores(L, nullptr);
  ranks.assign(L + 1, 1);
  Cx<double>* M = T;
  bool own_M = false;
  double delta2 = 0;
  {
    long long tot = 1;
    for (int d : dims) tot *= d;
    delta2 = L > 1 ? eps * eps * e.norm2(T, tot) / (double)(L - 1) : 0.0;
  }
  for (int j = L - 1; j >= 1; --j) {
    const int c = dims[j] * ranks[j + 1];
    const long long P = prod_dims(dims.data(), 0, j);
    QREQ(P < (1ll << 31), "TT-SVD unfolding too large");
    if (8.0 * (double)P * c * std::min<double>(P, c) < e.c->gram_threshold) {
      // Small unfolding: accurate SVD of M itself (QR + one-sided Jacobi; no
      // squared condition number). M = U S V^H, core j = V[:, :kk]^H, carry
      // = U[:, :kk] S (row-major P x kk for the next reshape).
      const int m0 = (int)std::max<long long>(P, c), n0 = (int)std::min<long long>(P, c);
      Cx<double>* A = e.alloc((long long)P * c);
      Cx<double>* Uw = e.alloc((long long)m0 * n0);
      Cx<double>* Vw = e.alloc((long long)n0 * n0);
      double* sg = (double*)e.ln->arena->alloc(sizeof(double) * n0);
      int cap = 0, kk;
      Cx<double>* core;
      Cx<double>* Mn = e.alloc(P * std::min<long long>(P, c));
      if (P >= c) {
        const long long sz[2] = {P, c}, ist[2] = {c, 1}, ost[2] = {1, P};
        e.copy(M, A, 2, sz, ist, ost);  // column-major copy
        kk = e.svd((int)P, c, A, Uw, sg, Vw, delta2, rmax, &cap);
        core = e.alloc((long long)kk * c);
        const long long s2[2] = {kk, c}, i2[2] = {c, 1}, o2[2] = {c, 1};
        e.copy(Vw, core, 2, s2, i2, o2, 1);  // V[:, :kk]^H
        scale_cols_kernel<double><<<grid1d(P * kk), 256, 0, e.st()>>>(Uw, (int)P, kk, sg);
        e.post("scale_cols_kernel", __LINE__);
        const long long s3[2] = {P, kk}, i3[2] = {1, P}, o3[2] = {kk, 1};
        e.copy(Uw, Mn, 2, s3, i3, o3);
      } else {
        // wide: A = M^H (c x P), M^H = U' S V'^H -> M = V' S U'^H
        const long long sz[2] = {P, c}, ist[2] = {c, 1}, ost[2] = {c, 1};
        e.copy(M, A, 2, sz, ist, ost, 1);  // A[jc + p c] = conj(M[p, jc])
        kk = e.svd(c, (int)P, A, Uw, sg, Vw, delta2, rmax, &cap);
        core = e.alloc((long long)kk * c);
        const long long s2[2] = {kk, c}, i2[2] = {c, 1}, o2[2] = {c, 1};
        e.copy(Uw, core, 2, s2, i2, o2, 1);  // U'[:, :kk]^H
        scale_cols_kernel<double><<<grid1d(P * kk), 256, 0, e.st()>>>(Vw, (int)P, kk, sg);
        e.post("scale_cols_kernel", __LINE__);
        const long long s3[2] = {P, kk}, i3[2] = {1, P}, o3[2] = {kk, 1};
        e.copy(Vw, Mn, 2, s3, i3, o3);
      }
      e.release(A);
      e.release(Uw);
      e.release(Vw);
      e.ln->arena->release(sg);
      cores[j] = core;
      ranks[j] = kk;
      if (own_M || consume_T) e.release(M);  // T itself once consumed, if allowed
      M = Mn;
      own_M = true;
      continue;
    }
    if (c > 4096)
      throw QttError(QTT_EINVAL, "TT-SVD: bond " + std::to_string(j) + " of " +
                                     std::to_string(L) + " too wide (c = " + std::to_string(c) +
                                     ", dims[j] = " + std::to_string(dims[j]) +
                                     ", eps = " + std::to_string(eps) + ")");
    // eigenvectors V of the Gram matrix G = M^H M (column-major for the
    // Jacobi kernel)
    Cx<double>* G = e.alloc((long long)c * c);
    if (c <= kGramMaxCols) {
      // tall-skinny: a dedicated kernel (a 64 x 64 GEMM tile wastes (64/c)^2)
      e.zero(G, (long long)c * c);
      const int ch = kGramChunk / c;
      long long rows = std::max<long long>(ch, (P + 152 * 6 - 1) / (152 * 6));
      const long long nb = (P + rows - 1) / rows;
      gram_skinny_kernel<double><<<(unsigned)nb, 256, 0, e.st()>>>(M, P, c, rows, G);
      e.post("gram_skinny_kernel", __LINE__);
    } else {
      const int ks = (int)std::min<long long>(std::max<long long>(1, P / 8192),
                                              4096 / std::max(1, (c / 64 + 1) * (c / 64 + 1)));
      e.gemm(c, c, (int)P, mref(M, 1, c, 0, 0, 0, 1), mref(M, c, 1), G, 1, c, 0, 0, 0, 1, 1, 1,
             Cplx{1, 0}, Cplx{0, 0}, std::max(1, ks));
    }
    Cx<double>* U = e.alloc((long long)c * c);
    Cx<double>* V = e.alloc((long long)c * c);
    double* sig = (double*)e.ln->arena->alloc(sizeof(double) * c);
    int cap = 0;
    e.svd(c, c, G, U, sig, V, 0.0, c, &cap, true);
    e.release(G);
    e.release(U);
    e.release(sig);
    // MV (P x c): its column norms are the singular values to working
    // accuracy (the Gram eigenvalues carry noise ~ c eps lambda_max, which
    // would swamp the tail threshold for wide bonds); they decide the rank.
    Cx<double>* MV = e.alloc(P * c);
    if (c <= kSkinnyMaxCols) {
      matmul_skinny_kernel<double><<<grid1d(P * c), 256, 0, e.st()>>>(M, P, c, V, MV);
      e.post("matmul_skinny_kernel", __LINE__);
    } else {
      e.gemm((int)P, c, c, mref(M, c, 1), mref(V, 1, c), MV, c, 1, 0, 0, 0, 1, 1, 1);
    }
    double* cn = (double*)e.ln->arena->alloc(sizeof(double) * c);
    QCHECK(cudaMemsetAsync(cn, 0, sizeof(double) * c, e.st()));
    colnorm2_kernel<double><<<grid1d(P * c), 256, sizeof(double) * c, e.st()>>>(MV, P, c, cn);
    e.post("colnorm2_kernel", __LINE__);
    std::vector<double> h(c);
    QCHECK(cudaMemcpyAsync(e.ln->pinned, cn, sizeof(double) * c, cudaMemcpyDeviceToHost, e.st()));
    QCHECK(e.ln->wait());
    memcpy(h.data(), e.ln->pinned, sizeof(double) * c);
    e.ln->arena->release(cn);
    std::vector<int> perm(c);
    for (int i = 0; i < c; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return h[a] > h[b]; });
    int kk = c;
    double tail = 0;
    std::vector<double> tails(c + 1, 0.0);
    for (int i = c - 1; i >= 0; --i) tails[i] = (tail += h[perm[i]]);
    for (int i = 1; i < c; ++i)
      if (tails[i] <= delta2) {
        kk = i;
        break;
      }
    kk = std::max(1, std::min(kk, rmax));
    int* didx = (int*)e.ln->arena->alloc(sizeof(int) * kk);
    memcpy(e.ln->pinned, perm.data(), sizeof(int) * kk);  // pinned staging (kk <= 4096)
    QCHECK(cudaMemcpyAsync(didx, e.ln->pinned, sizeof(int) * kk, cudaMemcpyHostToDevice, e.st()));
    // core j = V[:, perm[:kk]]^H (kk x c): gather rows of V^H
    Cx<double>* VH = e.alloc((long long)c * c);
    {
      const long long sz[2] = {c, c}, ist[2] = {c, 1}, ost[2] = {c, 1};
      e.copy(V, VH, 2, sz, ist, ost, 1);  // VH[a][b] = conj(V[b, a]) (row a = column a of V)
    }
    Cx<double>* core = e.alloc((long long)kk * c);
    for (int a = 0; a < kk; ++a)  // rows perm[0..kk) of VH
      QCHECK(cudaMemcpyAsync(core + (long long)a * c, VH + (long long)perm[a] * c,
                             sizeof(Cx<double>) * c, cudaMemcpyDeviceToDevice, e.st()));
    e.release(VH);
    e.release(V);
    cores[j] = core;
    ranks[j] = kk;
    // carry = MV[:, perm[:kk]] (P x kk)
    Cx<double>* Mn = e.alloc(P * kk);
    int* gerr = (int*)e.ln->arena->alloc(sizeof(int));
    QCHECK(cudaMemsetAsync(gerr, 0, sizeof(int), e.st()));
    gather_cols_kernel<double><<<grid1d(P * kk), 256, 0, e.st()>>>(MV, P, c, didx, kk, Mn, gerr);
    e.post("gather_cols_kernel", __LINE__);
    {
      int hg = 0;
      QCHECK(cudaMemcpyAsync(e.ln->pinned, gerr, sizeof(int), cudaMemcpyDeviceToHost, e.st()));
      QCHECK(e.ln->wait());
      memcpy(&hg, e.ln->pinned, sizeof(int));
      e.ln->arena->release(gerr);
      if (hg) throw QttError(QTT_EINVAL, "TT-SVD: column index out of range (kernel skipped access)");
    }
    e.ln->arena->release(didx);
    e.release(MV);
    if (own_M || consume_T) e.release(M);  // T itself once consumed, if allowed
    M = Mn;
    own_M = true;
  }
  if (!own_M) {
    Cx<double>* c0 = e.alloc((long long)dims[0] * ranks[1]);
    QCHECK(cudaMemcpyAsync(c0, M, 16 * (size_t)dims[0] * ranks[1], cudaMemcpyDeviceToDevice,
                           e.st()));
    if (consume_T) e.release(M);
    M = c0;
  }
  cores[0] = M;
  return cores;
}

// Copy FP64 device cores into an op of the context's precision.
template <typename R>
void *to_prec(Eng<R>& e, Cx<double>* p, long long cnt) {
  if (sizeof(R) == 8) return p;
  Cx<R>* q = e.alloc(cnt);
  convert_kernel<double, R><<<grid1d(cnt), 256, 0, e.st()>>>(p, q, cnt);
  e.post("convert_kernel", __LINE__);
  e.release(p);
  return q;
}

// ------------------------------------------------------------------ C0 and stiffness

void lame_of(double E, double nu, double& lam, double& mu) {
  lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  mu = E / (2.0 * (1.0 + nu));
}

void voigt_stiffness(double lam, double mu, double* C) {
  for (int i = 0; i < 36; ++i) C[i] = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i * 6 + j] = lam + (i == j ? 2.0 * mu : 0.0);
  for (int i = 3; i < 6; ++i) C[i * 6 + i] = mu;
}

}  // namespace

// ================================================================== C ABI

#define API_BEGIN(ctx)      \
  qtt_ctx* c_ = (ctx);      \
  try {
#define API_END                                      \
  }                                                  \
  catch (const QttError& ex) {                       \
    if (c_) c_->err = ex.what();                     \
    return ex.code;                                  \
  }                                                  \
  catch (const std::exception& ex) {                 \
    if (c_) c_->err = ex.what();                     \
    return QTT_EINVAL;                               \
  }

#define DISPATCH(ctx, FN, ...)                               \
  ((ctx)->prec == QTT_FP64 ? FN<double>(__VA_ARGS__) : FN<float>(__VA_ARGS__))

namespace {

template <typename R>
qtt_tt* op_apply_impl(qtt_ctx* c, const qtt_op* op, const qtt_tt* in, double eps, int rmax,
                      int oversample, int apply_id, int* cap) {
  Eng<R> e(c);
  qtt_tt* y = apply_sketched<R>(e, op, in, rmax + oversample, apply_id);
  *cap = round_right_to_left<R>(e, y, eps, rmax);
  return y;
}

// Full tensor of a TT by left-to-right contraction of the cores, as
// complex128 on the host (prod(dims) entries, row-major).
template <typename R>
void to_dense_impl(qtt_ctx* c, const qtt_tt* t, double* out) {
  Eng<R> e(c);
  long long rows = t->dims[0];  // running product of the leading dims
  QREQ(t->ranks[0] == 1, "qtt_tt_to_dense: ranks[0] must be 1");
  Cx<R>* cur = e.alloc(t->count(0));
  QCHECK(cudaMemcpyAsync(cur, t->core[0], t->count(0) * sizeof(Cx<R>), cudaMemcpyDeviceToDevice,
                         e.st()));
  for (int k = 1; k < t->L; ++k) {
    const int r0 = t->ranks[k], d = t->dims[k], r1 = t->ranks[k + 1];
    QREQ(rows * d <= (1ll << 30) && rows < (1ll << 31), "qtt_tt_to_dense: tensor too large");
    Cx<R>* nx = e.alloc(rows * d * r1);
    // nx (rows x d r1) = cur (rows x r0) core_k (r0 x d r1)
    e.gemm((int)rows, d * r1, r0, mref(cur, r0, 1), mref(t->core[k], (long long)d * r1, 1), nx,
           (long long)d * r1, 1, 0, 0, 0, 1, 1, 1);
    e.release(cur);
    cur = nx;
    rows *= d;
  }
  std::vector<Cx<R>> h(rows);
  QCHECK(cudaMemcpyAsync(h.data(), cur, rows * sizeof(Cx<R>), cudaMemcpyDeviceToHost, e.st()));
  QCHECK(e.ln->wait());
  e.release(cur);
  for (long long i = 0; i < rows; ++i) {
    out[2 * i] = (double)h[i].x;
    out[2 * i + 1] = (double)h[i].y;
  }
}

template <typename R>
int round_impl(qtt_ctx* c, qtt_tt* x, double eps, int rmax) {
  Eng<R> e(c);
  return round_full<R>(e, x, eps, rmax);
}

template <typename R>
void dot_impl(qtt_ctx* c, const qtt_tt* a, const qtt_tt* b, double* re, double* im) {
  Eng<R> e(c);
  tt_dot<R>(e, a, b, re, im);
}

template <typename R>
void mean_impl(qtt_ctx* c, const qtt_op* op, const qtt_tt* x, std::vector<double>& out) {
  Eng<R> e(c);
  op_mean<R>(e, op, x, out);
}

// Build an operator from FP64 device cores.
template <typename R>
qtt_op* op_from_fp64(qtt_ctx* c, std::vector<Cx<double>*>& cores, const std::vector<int>& ranks,
                     const std::vector<int>& dout, const std::vector<int>& din,
                     const std::vector<int>& diag) {
  Eng<R> e(c);
  qtt_op* o = new qtt_op();
  o->ctx = c;
  o->L = (int)cores.size();
  for (int k = 0; k < o->L; ++k) {
    o->dout[k] = dout[k];
    o->din[k] = din[k];
    o->diag[k] = diag[k];
  }
  for (int k = 0; k <= o->L; ++k) o->ranks[k] = ranks[k];
  for (int k = 0; k < o->L; ++k) o->core[k] = to_prec<R>(e, cores[k], o->count(k));
  return o;
}

qtt_op* build_sfft(qtt_ctx* c, int n, int adjoint, double eps) {
  QREQ(n >= 1 && 3 * n + 1 <= QTT_MAX_CORES, "sfft: n out of range");
  Eng<double> e(c);
  const long long N = 1ll << n;
  Cx<double>* T = e.alloc(N * N);
  sfft_tensor_kernel<<<grid1d(N * N), 256, 0, e.st()>>>((double*)T, n);
  e.post("sfft_tensor_kernel", __LINE__);
  std::vector<int> dims(n, 4), ranks;
  std::vector<Cx<double>*> ax = tt_svd_device(e, T, dims, eps, 1 << 30, ranks, true);
  // assemble: Voigt identity core, then the axis MPO three times
  const int L = 3 * n + 1;
  std::vector<Cx<double>*> cores(L);
  std::vector<int> R(L + 1, 1), dout(L, 2), din(L, 2), diag(L, 0);
  dout[0] = din[0] = 6;
  Cx<double>* I6 = e.alloc(36);
  {
    std::vector<double> h(72, 0.0);
    for (int i = 0; i < 6; ++i) h[2 * (i * 6 + i)] = 1.0;
    QCHECK(cudaMemcpyAsync(I6, h.data(), 72 * 8, cudaMemcpyHostToDevice, e.st()));
    QCHECK(e.ln->wait());
  }
  cores[0] = I6;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < n; ++b) {
      const int k = 1 + a * n + b;
      const long long cnt = (long long)ranks[b] * 4 * ranks[b + 1];
      Cx<double>* p = e.alloc(cnt);
      if (!adjoint) {
        QCHECK(cudaMemcpyAsync(p, ax[b], cnt * 16, cudaMemcpyDeviceToDevice, e.st()));
      } else {
        // W^H core: (f, o, i, f') <- conj(W(f, i, o, f'))
        const long long sz[4] = {ranks[b], 2, 2, ranks[b + 1]};
        const long long ist[4] = {4ll * ranks[b + 1], ranks[b + 1], 2ll * ranks[b + 1], 1};
        const long long ost[4] = {4ll * ranks[b + 1], 2ll * ranks[b + 1], ranks[b + 1], 1};
        e.copy(ax[b], p, 4, sz, ist, ost, 1);
      }
      cores[k] = p;
      R[k] = ranks[b];
      R[k + 1] = ranks[b + 1];
    }
  for (auto p : ax) e.release(p);
  qtt_op* o = c->prec == QTT_FP64 ? op_from_fp64<double>(c, cores, R, dout, din, diag)
                                  : op_from_fp64<float>(c, cores, R, dout, din, diag);
  o->n = n;
  return o;
}

qtt_op* assemble_raised(qtt_ctx* c, Eng<double>& e, std::vector<Cx<double>*>& tc,
                        const std::vector<int>& ranks, int n, const int bcast[3]);

// Raised operator from a dense (36, 2^bits) FP64 complex field with
// broadcast axes (axis a contributes nbits[a] cores from the field or n
// identity cores when broadcast). With `Uleft` (column-major 36 x rows, and
// F holding `rows` rows) the field is Uleft F and Uleft multiplies the first
// core after the TT-SVD.
qtt_op* raised_from_field(qtt_ctx* c, Cx<double>* F, int n, const int bcast[3], double eps,
                          int rmax, int rows = 36, const Cx<double>* Uleft = nullptr) {
  Eng<double> e(c);
  int bits = 0;
  for (int a = 0; a < 3; ++a) bits += bcast[a] ? 0 : n;
  std::vector<int> dims(1 + bits, 2), ranks;
  dims[0] = rows;
  std::vector<Cx<double>*> tc = tt_svd_device(e, F, dims, eps, rmax, ranks, true);
  if (Uleft) {
    Cx<double>* c0 = e.alloc(36ll * ranks[1]);
    e.gemm(36, ranks[1], rows, mref(Uleft, 1, 36), mref(tc[0], ranks[1], 1), c0, ranks[1], 1, 0,
           0, 0, 1, 1, 1);
    e.release(tc[0]);
    tc[0] = c0;
  }
  return assemble_raised(c, e, tc, ranks, n, bcast);
}

// Raised operator from FP64 TT cores of a controlled field (first core
// 36 x r1, then one binary core per non-broadcast bit; ownership of the cores
// passes to the operator), with identity cores for broadcast axes.
qtt_op* assemble_raised(qtt_ctx* c, Eng<double>& e, std::vector<Cx<double>*>& tc,
                        const std::vector<int>& ranks, int n, const int bcast[3]) {
  const int L = 3 * n + 1;
  std::vector<Cx<double>*> cores(L);
  std::vector<int> R(L + 1, 1), dout(L, 2), din(L, 2), diag(L, 1);
  dout[0] = din[0] = 6;
  diag[0] = 0;
  cores[0] = tc[0];
  R[1] = ranks[1];
  int src = 1, k = 1;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < n; ++b, ++k) {
      if (bcast[a]) {
        const int r = R[k];
        Cx<double>* I = e.alloc((long long)r * 2 * r);
        e.zero(I, (long long)r * 2 * r);
        // C[alpha, i, alpha] = 1
        std::vector<double> one = {1.0, 0.0};
        Cx<double>* d1 = e.alloc(1);
        QCHECK(cudaMemcpyAsync(d1, one.data(), 16, cudaMemcpyHostToDevice, e.st()));
        const long long sz[2] = {r, 2}, ist[2] = {0, 0}, ost[2] = {2ll * r + 1, r};
        e.copy(d1, I, 2, sz, ist, ost);
        QCHECK(e.ln->wait());
        e.release(d1);
        cores[k] = I;
        R[k + 1] = r;
      } else {
        cores[k] = tc[src];
        R[k + 1] = ranks[src + 1];
        ++src;
      }
    }
  qtt_op* o = c->prec == QTT_FP64 ? op_from_fp64<double>(c, cores, R, dout, din, diag)
                                  : op_from_fp64<float>(c, cores, R, dout, din, diag);
  for (int a = 0; a < 3; ++a) o->bcast[a] = bcast[a] ? 1 : 0;
  return o;
}

// Raised operator of a phase field whose cells carry one of nphase Voigt
// matrices, D[:, p] = Dh[36 p .. 36 p + 36). The field's 36 Voigt rows lie in
// the column space of D: with the thin SVD D = U S V^H the field is U Y,
// Y[a, x] = s_a conj(V[phase(x), a]). U has orthonormal columns, so it leaves
// the singular values of every unfolding unchanged: the TT-SVD of the k-row
// field Y, with U applied to its first core, is that of the 36-row field up to
// rounding, on k/36 of the data (k <= 2 for isotropic phases).
qtt_op* raised_from_phases(qtt_ctx* ctx, const uint8_t* phase, long long cells, const double* Dh,
                           int nphase, int n, const int bc[3], double eps, int rmax) {
  Eng<double> e(ctx);
  uint8_t* dph = (uint8_t*)ctx->arena.alloc(cells);
  QCHECK(cudaMemcpyAsync(dph, phase, cells, cudaMemcpyHostToDevice, ctx->stream));
  if (nphase > 36) {  // no reduction possible: the 36-row field itself
    double* ddc = (double*)ctx->arena.alloc(sizeof(double) * 36 * nphase);
    QCHECK(cudaMemcpyAsync(ddc, Dh, sizeof(double) * 36 * nphase, cudaMemcpyHostToDevice,
                           ctx->stream));
    Cx<double>* F = e.alloc(36 * cells);
    stiffness_field_kernel<<<grid1d(cells), 256, 0, ctx->stream>>>(dph, cells, ddc, nphase, F);
    e.post("stiffness_field_kernel", __LINE__);
    QCHECK(cudaStreamSynchronize(ctx->stream));
    ctx->arena.release(dph);
    ctx->arena.release(ddc);
    return raised_from_field(ctx, F, n, bc, eps, rmax);  // consumes F
  }
  // D as a complex column-major 36 x nphase matrix (same linear order)
  std::vector<double> hD(2 * 36 * nphase, 0.0);
  double nD2 = 0;
  for (int i = 0; i < 36 * nphase; ++i) {
    hD[2 * i] = Dh[i];
    nD2 += Dh[i] * Dh[i];
  }
  Cx<double>* A = e.alloc(36ll * nphase);
  QCHECK(cudaMemcpyAsync(A, hD.data(), hD.size() * sizeof(double), cudaMemcpyHostToDevice,
                         ctx->stream));
  Cx<double>* U = e.alloc(36ll * nphase);
  Cx<double>* V = e.alloc((long long)nphase * nphase);
  double* sg = (double*)ctx->arena.alloc(sizeof(double) * nphase);
  int cap = 0;
  // directions below 1e-14 of ||D|| are rounding noise of the differences
  const int k = e.svd(36, nphase, A, U, sg, V, 1e-28 * nD2, nphase, &cap);
  // table[p + a nphase] = s_a conj(V[p, a])
  Cx<double>* table = e.alloc((long long)nphase * k);
  {
    const long long sz[1] = {(long long)nphase * k}, st1[1] = {1};
    e.copy(V, table, 1, sz, st1, st1, 1);
  }
  scale_cols_kernel<double><<<grid1d((long long)nphase * k), 256, 0, e.st()>>>(table, nphase, k,
                                                                               sg);
  e.post("scale_cols_kernel", __LINE__);
  Cx<double>* Y = e.alloc((long long)k * cells);
  phase_table_field_kernel<<<grid1d(cells), 256, 0, e.st()>>>(dph, cells, table, nphase, k, Y);
  e.post("phase_table_field_kernel", __LINE__);
  QCHECK(cudaStreamSynchronize(ctx->stream));
  e.release(A);
  e.release(V);
  e.release(table);
  ctx->arena.release(sg);
  ctx->arena.release(dph);
  qtt_op* o = raised_from_field(ctx, Y, n, bc, eps, rmax, k, U);  // consumes Y
  e.release(U);
  return o;
}

// Coefficients of the Direct-scheme Green field in the 15 degree-4 monomials
// of n = xi / |xi| (order of green_monomials_at): Gamma_V[I][J] = w_I w_J
// Gamma_ijkl with Gamma_ijkl = (d_ik n_j n_l + d_il n_j n_k + d_jk n_i n_l +
// d_jl n_i n_k) / (4 mu0) - beta0 n_i n_j n_k n_l (App. A), each quadratic
// n_a n_b written as sum_c n_a n_b n_c n_c. C is 36 x 15 row-major.
int green_monomial_index(int a, int b, int c, int d) {
  int v[4] = {a, b, c, d};
  std::sort(v, v + 4);
  int g = 0;
  for (int p = 0; p < 3; ++p)
    for (int q = p; q < 3; ++q)
      for (int r = q; r < 3; ++r)
        for (int s = r; s < 3; ++s, ++g)
          if (p == v[0] && q == v[1] && r == v[2] && s == v[3]) return g;
  return -1;
}

void green_coeffs(double lam0, double mu0, double* C) {
  static const int vi[6] = {0, 1, 2, 1, 0, 0}, vj[6] = {0, 1, 2, 2, 2, 1};
  const double beta0 = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0));
  for (int q = 0; q < 36 * 15; ++q) C[q] = 0;
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      const int i = vi[I], j = vj[I], k = vi[J], l = vj[J];
      const double w = (I < 3 ? 1.0 : 2.0) * (J < 3 ? 1.0 : 2.0);
      double* row = C + (I * 6 + J) * 15;
      auto add2 = [&](int a, int b) {
        for (int cc = 0; cc < 3; ++cc) row[green_monomial_index(a, b, cc, cc)] += w / (4.0 * mu0);
      };
      if (i == k) add2(j, l);
      if (i == l) add2(j, k);
      if (j == k) add2(i, l);
      if (j == l) add2(i, k);
      row[green_monomial_index(i, j, k, l)] -= w * beta0;
    }
}

// Green operator from its separable form: the TT of the 15 monomial fields
// (TT-SVD at eps, cached per grid: it does not depend on the reference
// medium), then its first core mixed by the 36 x 15 coefficient matrix C of
// (lam0, mu0). The operator's relative error is at most cond(C) eps (C's
// condition number is ~7 for the media of the workloads).
//
// The Forward, Backward and staggered schemes have complex divergence
// operators and no such separable form: their Green field (36 complex
// entries per frequency, green_symbol_field_kernel) is compressed directly
// by TT-SVD, which bounds n by the 2^31-row unfolding (n <= 8) and needs
// 36 x 2^(3n) x 16 bytes of workspace for the field (9.7 GB at n = 8).
qtt_op* build_gamma_symbol(qtt_ctx* c, int n, double lam0, double mu0, int scheme, double eps,
                           int rmax) {
  QREQ(n >= 1 && n <= 8, "gamma: n must be in 1..8 for the Forward, Backward and staggered schemes");
  Eng<double> e(c);
  const long long N3 = 1ll << (3 * n);
  Cx<double>* F = e.alloc(36 * N3);
  green_symbol_field_kernel<<<grid1d(N3), 256, 0, e.st()>>>(F, n, lam0, mu0, scheme, 0);
  e.post("green_symbol_field_kernel", __LINE__);
  const int bc[3] = {0, 0, 0};
  qtt_op* o = raised_from_field(c, F, n, bc, eps, rmax);  // consumes F
  o->n = n;
  o->has_c0 = 1;
  o->lame0[0] = lam0;
  o->lame0[1] = mu0;
  voigt_stiffness(lam0, mu0, o->C0);
  return o;
}

qtt_op* build_gamma(qtt_ctx* c, int n, double lam0, double mu0, int scheme, double eps, int rmax) {
  QREQ(scheme >= QTT_SCHEME_DIRECT && scheme <= QTT_SCHEME_STAGGERED,
       "gamma: scheme must be 0..5 (Direct, Centered, Forward, Backward, Hex8R, staggered)");
  QREQ(mu0 > 0 && lam0 + 2 * mu0 > 0, "gamma: reference medium not positive definite");
  if (scheme == QTT_SCHEME_FORWARD || scheme == QTT_SCHEME_BACKWARD ||
      scheme == QTT_SCHEME_STAGGERED)
    return build_gamma_symbol(c, n, lam0, mu0, scheme, eps, rmax);
  QREQ(n >= 1 && n <= 9, "gamma: n must be in 1..9");
  Eng<double> e(c);
  const double eps_m = eps;
  const auto key = std::make_tuple(n, eps_m, rmax, scheme);
  auto it = c->green_mono_cache.find(key);
  if (it == c->green_mono_cache.end()) {
    const long long N3 = 1ll << (3 * n);
    Cx<double>* F = e.alloc(15 * N3);
    green_monomials_kernel<<<grid1d(N3), 256, 0, e.st()>>>(F, n, scheme, 0);
    e.post("green_monomials_kernel", __LINE__);
    std::vector<int> dims(1 + 3 * n, 2), ranks;
    dims[0] = 15;
    std::vector<Cx<double>*> tc = tt_svd_device(e, F, dims, eps_m, rmax, ranks, true);
    qtt_ctx::GreenMono gm;
    for (auto* p : tc) gm.cores.push_back(p);
    gm.ranks = ranks;
    it = c->green_mono_cache.emplace(key, gm).first;
  }
  const qtt_ctx::GreenMono& gm = it->second;
  const int L = 3 * n + 1, r1 = gm.ranks[1];
  std::vector<double> Ch(36 * 15), hc(2 * 36 * 15, 0.0);
  green_coeffs(lam0, mu0, Ch.data());
  for (int q = 0; q < 36 * 15; ++q) hc[2 * q] = Ch[q];
  Cx<double>* Cd = e.alloc(36 * 15);
  QCHECK(cudaMemcpyAsync(Cd, hc.data(), hc.size() * sizeof(double), cudaMemcpyHostToDevice,
                         e.st()));
  std::vector<Cx<double>*> tc(L);
  tc[0] = e.alloc(36ll * r1);
  e.gemm(36, r1, 15, mref(Cd, 15, 1), mref(gm.cores[0], r1, 1), tc[0], r1, 1, 0, 0, 0, 1, 1, 1);
  for (int k = 1; k < L; ++k) {
    const long long cnt = (long long)gm.ranks[k] * 2 * gm.ranks[k + 1];
    tc[k] = e.alloc(cnt);
    QCHECK(cudaMemcpyAsync(tc[k], gm.cores[k], cnt * sizeof(Cx<double>), cudaMemcpyDeviceToDevice,
                           e.st()));
  }
  QCHECK(e.ln->wait());
  e.release(Cd);
  const int bc[3] = {0, 0, 0};
  qtt_op* o = assemble_raised(c, e, tc, gm.ranks, n, bc);
  o->n = n;
  o->has_c0 = 1;
  o->lame0[0] = lam0;
  o->lame0[1] = mu0;
  voigt_stiffness(lam0, mu0, o->C0);
  return o;
}

// The solver's SFFT MPOs are rounded at 1e-12. The reduced QFT circuit
// (Sec. 4.1-4.2) has ranks 2^min(b, n-b) (at most 11-12 for n = 8 within
// 1e-12), and rounding at 1e-12 reproduces the DFT to ~1e-14. Rounding at
// 1e-14, the level of the SVD's own rounding noise, keeps noise directions
// instead (ranks up to ~127 at n = 8), which only widens every S and S^H
// product.
constexpr double kSfftRoundEps = 1e-12;

qtt_op* cached_sfft(qtt_ctx* c, int n, int adjoint) {
  auto key = std::make_pair(n, adjoint);
  auto it = c->sfft_cache.find(key);
  if (it != c->sfft_cache.end()) return it->second;
  qtt_op* o = build_sfft(c, n, adjoint, kSfftRoundEps);
  c->sfft_cache[key] = o;
  return o;
}

qtt_op* cached_gamma(qtt_ctx* c, int n, double lam0, double mu0, int scheme, double eps, int rmax) {
  auto key = std::make_tuple(n, lam0, mu0, scheme, eps, rmax);
  auto it = c->gamma_cache.find(key);
  if (it != c->gamma_cache.end()) return it->second;
  qtt_op* o = build_gamma(c, n, lam0, mu0, scheme, eps, rmax);
  c->gamma_cache[key] = o;
  return o;
}

// Green operator for stiffness operators broadcast along x1. The strain of
// such a problem is x1-invariant, so after the SFFT its x1 bits hold only the
// frequency xi_1 = 0, where Gamma acts as Gamma(0, xi_2, xi_3); the operator
// Gamma(0, xi_2, xi_3) (x) I on the x1 cores acts on these fields exactly as
// the full operator does (Sec. 4.3 on broadcast axes). It is built from the
// N^2-point plane field instead of the N^3 one: the 15 monomial fields for the
// Direct, Centered and Hex8R schemes (mixed into the 36 Voigt entries through
// the first core), the 36 entries for the others. Its rank through the x1
// cores is that of the first bond. n <= 13 (2^31-row TT-SVD unfoldings).
qtt_op* build_gamma_plane(qtt_ctx* c, int n, double lam0, double mu0, int scheme, double eps,
                          int rmax) {
  QREQ(scheme >= QTT_SCHEME_DIRECT && scheme <= QTT_SCHEME_STAGGERED,
       "gamma (plane): scheme must be 0..5");
  QREQ(n >= 1 && n <= 13, "gamma (plane): n must be in 1..13");
  QREQ(mu0 > 0 && lam0 + 2 * mu0 > 0, "gamma: reference medium not positive definite");
  Eng<double> e(c);
  const long long N2 = 1ll << (2 * n);
  const int bc[3] = {1, 0, 0};
  qtt_op* o = nullptr;
  if (scheme == QTT_SCHEME_FORWARD || scheme == QTT_SCHEME_BACKWARD ||
      scheme == QTT_SCHEME_STAGGERED) {
    Cx<double>* F = e.alloc(36 * N2);
    green_symbol_field_kernel<<<grid1d(N2), 256, 0, e.st()>>>(F, n, lam0, mu0, scheme, 1);
    e.post("green_symbol_field_kernel", __LINE__);
    o = raised_from_field(c, F, n, bc, eps, rmax);  // consumes F
  } else {
    Cx<double>* F = e.alloc(15 * N2);
    green_monomials_kernel<<<grid1d(N2), 256, 0, e.st()>>>(F, n, scheme, 1);
    e.post("green_monomials_kernel", __LINE__);
    std::vector<double> Ch(36 * 15), U(2 * 36 * 15, 0.0);
    green_coeffs(lam0, mu0, Ch.data());
    for (int P = 0; P < 36; ++P)
      for (int g = 0; g < 15; ++g) U[2 * (P + 36 * g)] = Ch[P * 15 + g];  // column-major 36 x 15
    Cx<double>* Ud = e.alloc(36 * 15);
    QCHECK(cudaMemcpyAsync(Ud, U.data(), U.size() * sizeof(double), cudaMemcpyHostToDevice,
                           e.st()));
    QCHECK(e.ln->wait());
    o = raised_from_field(c, F, n, bc, eps, rmax, 15, Ud);  // consumes F
    QCHECK(e.ln->wait());
    e.release(Ud);
  }
  o->n = n;
  o->has_c0 = 1;
  o->lame0[0] = lam0;
  o->lame0[1] = mu0;
  voigt_stiffness(lam0, mu0, o->C0);
  return o;
}

// The Green operator a solve with stiffness operator d uses: the plane form
// when the context asks for it and d is broadcast along x1 only, else the
// full operator.
qtt_op* solve_gamma(qtt_ctx* c, const qtt_op* d, const qtt_solve_params* p) {
  if (c->green_broadcast && d->bcast[0] && !d->bcast[1] && !d->bcast[2]) {
    auto key = std::make_tuple(d->n, d->lame0[0], d->lame0[1], p->scheme, p->eps_tt, 1 << 30);
    auto it = c->gamma_plane_cache.find(key);
    if (it != c->gamma_plane_cache.end()) return it->second;
    qtt_op* o = build_gamma_plane(c, d->n, d->lame0[0], d->lame0[1], p->scheme, p->eps_tt,
                                  1 << 30);
    c->gamma_plane_cache[key] = o;
    return o;
  }
  return cached_gamma(c, d->n, d->lame0[0], d->lame0[1], p->scheme, p->eps_tt, 1 << 30);
}

// E field as a rank-1 controlled QTT: Voigt core E sqrt(2)^(3n), binary
// cores (1, 1)/sqrt(2).
template <typename R>
qtt_tt* e_field(qtt_ctx* c, Lane* ln, int L, const int* dims, const double* Ev) {
  Eng<R> e(c, ln);
  qtt_tt* t = new_tt(c, e.ln->arena, L, dims);
  for (int k = 0; k <= L; ++k) t->ranks[k] = 1;
  double scale = 1.0;
  for (int k = 1; k < L; ++k) scale *= std::sqrt((double)dims[k]);
  for (int k = 0; k < L; ++k) {
    std::vector<Cx<R>> h(dims[k]);
    for (int i = 0; i < dims[k]; ++i)
      h[i] = (k == 0) ? mk<R>((R)(Ev[i] * scale), 0) : mk<R>((R)(1.0 / std::sqrt((double)dims[k])), 0);
    t->core[k] = e.alloc(dims[k]);
    QCHECK(cudaMemcpyAsync(t->core[k], h.data(), sizeof(Cx<R>) * dims[k], cudaMemcpyHostToDevice,
                           e.st()));
    QCHECK(e.ln->wait());
  }
  return t;
}

// QTT_TRACE=1 in the environment: every LS iteration prints its residual
// and the largest rank of each intermediate TT to stderr.
bool trace_on() {
  static const bool on = [] {
    const char* v = getenv("QTT_TRACE");
    return v && v[0] == '1';
  }();
  return on;
}

int trace_load(const double* Ev) {
  for (int i = 0; i < 6; ++i)
    if (Ev[i] != 0.0) return i;
  return -1;
}

template <typename R>
int max_rank(const qtt_tt* t) {
  int m = 1;
  for (int k = 0; k <= t->L; ++k) m = std::max(m, t->ranks[k]);
  return m;
}

// Alg. 2, one load case.
template <typename R>
int solve_impl(qtt_ctx* c, const qtt_op* dC, const qtt_op* S, const qtt_op* Sh, const qtt_op* G,
               const double* C0, const double* Ev, const qtt_solve_params* p, double* sig,
               qtt_solve_info* info, int apply_base, Lane* lane = nullptr,
               qtt_tt** keep = nullptr) {
  Eng<R> e(c, lane);
  const auto t0 = std::chrono::steady_clock::now();
  const int L = dC->L;
  qtt_tt* Ett = e_field<R>(c, e.ln, L, dC->dout, Ev);
  double nE2 = 0;
  for (int i = 0; i < 6; ++i) nE2 += Ev[i] * Ev[i];
  double cells = 1.0;
  for (int k = 1; k < L; ++k) cells *= dC->dout[k];
  const double normE = std::sqrt(nE2 * cells);
  QREQ(normE > 0, "ls_solve: E = 0");
  qtt_tt* x = clone_tt<R>(e, Ett);
  const int ell = p->rmax + p->oversample;
  int cap = 0, maxr = 1, it = 0, status = QTT_OK;
  double rel = 0;
  // With QTT_CHECK_FINITE=1 in the environment every intermediate TT of
  // the iteration is checked (its FP64 norm) and the first non-finite one is
  // reported by step and iteration.
  const bool check_finite = debug_finite();
  auto chk = [&](qtt_tt* t, const char* step) {
    if (!check_finite) return;
    double a, b;
    tt_dot<R>(e, t, t, &a, &b);
    if (!std::isfinite(a))
      throw QttError(QTT_ENAN, std::string("ls_solve: non-finite after ") + step + " in iteration " +
                                   std::to_string(it));
  };
  for (it = 1; it <= p->max_iter; ++it) {
    const int t0id = apply_base + 4 * (it - 1);
    qtt_tt* tau = apply_sketched<R>(e, dC, x, ell, t0id);
    chk(tau, "(C - C0) product");
    cap |= round_right_to_left<R>(e, tau, p->eps_tt, p->rmax);
    chk(tau, "rounding of (C - C0) product");
    qtt_tt* tauh = apply_sketched<R>(e, S, tau, ell, t0id + 1);
    chk(tauh, "SFFT product");
    cap |= round_right_to_left<R>(e, tauh, p->eps_tt, p->rmax);
    chk(tauh, "rounding of SFFT product");
    qtt_tt* epsh = apply_sketched<R>(e, G, tauh, ell, t0id + 2);
    chk(epsh, "Green product");
    cap |= round_right_to_left<R>(e, epsh, p->eps_tt, p->rmax);
    chk(epsh, "rounding of Green product");
    qtt_tt* yv = apply_sketched<R>(e, Sh, epsh, ell, t0id + 3);
    chk(yv, "inverse SFFT product");
    qtt_tt* xn = tt_add<R>(e, Ett, yv, 1.0, -1.0);
    cap |= round_full<R>(e, xn, p->eps_tt, p->rmax);
    chk(xn, "rounding of the new strain");
    maxr = std::max({maxr, max_rank<R>(tau), max_rank<R>(tauh), max_rank<R>(epsh), max_rank<R>(xn)});
    const int rk_tau = max_rank<R>(tau), rk_tauh = max_rank<R>(tauh), rk_epsh = max_rank<R>(epsh),
              rk_x = max_rank<R>(xn);
    // ||xn - x||^2 = ||xn||^2 + ||x||^2 - 2 Re <xn, x>
    double a2r, a2i, b2r, b2i, abr, abi;
    tt_dot<R>(e, xn, xn, &a2r, &a2i);
    tt_dot<R>(e, x, x, &b2r, &b2i);
    tt_dot<R>(e, xn, x, &abr, &abi);
    // ||xn - x||^2 cancels: below ~64 eps (||xn||^2 + ||x||^2) the difference
    // is rounding noise (it can even come out <= 0), so the residual is never
    // reported below that floor and the stop test cannot fire on noise.
    const double floor2 = 64.0 * 2.220446049250313e-16 * (a2r + b2r);
    const double d2 = std::max(floor2, a2r + b2r - 2.0 * abr);
    rel = std::sqrt(d2) / normE;
    if (trace_on())
      fprintf(stderr, "[qtt] load %d iter %d residual %.4e ranks tau %d tauh %d epsh %d eps %d\n",
              trace_load(Ev), it, rel, rk_tau, rk_tauh, rk_epsh, rk_x);
    free_tt(tau);
    free_tt(tauh);
    free_tt(epsh);
    free_tt(yv);
    free_tt(x);
    x = xn;
    if (!std::isfinite(rel)) {
      free_tt(x);
      free_tt(Ett);
      throw QttError(QTT_ENAN, "ls_solve: non-finite residual");
    }
    if (rel < p->tol) break;
  }
  if (it > p->max_iter) {
    it = p->max_iter;
    status = QTT_WNOCONV;
  }
  std::vector<double> m;
  op_mean<R>(e, dC, x, m);
  double leak = 0;
  for (int i = 0; i < 6; ++i) {
    double c0e = 0;
    for (int j = 0; j < 6; ++j) c0e += C0[i * 6 + j] * Ev[j];
    sig[2 * i] = c0e + m[2 * i];
    sig[2 * i + 1] = m[2 * i + 1];
    leak = std::max(leak, std::fabs(m[2 * i + 1]));
  }
  if (keep) {
    // copy of the final strain in the context's own arena (outlives the lane)
    qtt_tt* k = new_tt(c, &c->arena, x->L, x->dims);
    for (int b = 0; b <= x->L; ++b) k->ranks[b] = x->ranks[b];
    for (int b = 0; b < x->L; ++b) {
      k->core[b] = c->arena.alloc((size_t)x->count(b) * sizeof(Cx<R>));
      QCHECK(cudaMemcpyAsync(k->core[b], x->core[b], x->count(b) * sizeof(Cx<R>),
                             cudaMemcpyDeviceToDevice, e.st()));
    }
    QCHECK(e.ln->wait());
    *keep = k;
  }
  free_tt(x);
  free_tt(Ett);
  if (info) {
    info->iters = it;
    info->residual = rel;
    info->max_rank = maxr;
    info->rank_cap_hit = cap;
    info->imag_leak = leak;
    info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status == QTT_OK && cap) status = QTT_WRANKCAP;
  return status;
}

}  // namespace

extern "C" {

int qtt_ctx_create(qtt_ctx_t* out, int device, void* cuda_stream, int precision, void* workspace,
                   size_t workspace_bytes, uint64_t seed) {
  if (!out) return QTT_EINVAL;
  *out = nullptr;
  if (precision != QTT_FP64 && precision != QTT_FP32) return QTT_EINVAL;
  if (!workspace || workspace_bytes < (1u << 20) || ((uintptr_t)workspace & 255)) return QTT_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return QTT_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return QTT_ECUDA;
  qtt_ctx* c = new qtt_ctx();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  c->prec = precision;
  c->seed = seed;
  c->arena.init(workspace, workspace_bytes);
  if (cudaMallocHost(&c->pinned, 1 << 16) != cudaSuccess) {
    delete c;
    return QTT_ECUDA;
  }
  c->lane0.arena = &c->arena;
  c->lane0.stream = c->stream;
  c->lane0.pinned = c->pinned;
  *out = c;
  return QTT_OK;
}

void qtt_ctx_destroy(qtt_ctx_t c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  prof_flush(c);
  for (auto& kv : c->sfft_cache) free_op(kv.second);
  for (auto& kv : c->gamma_cache) free_op(kv.second);
  for (auto& kv : c->gamma_plane_cache) free_op(kv.second);
  for (auto& kv : c->green_mono_cache)
    for (void* p : kv.second.cores) c->arena.release(p);
  if (c->pinned) cudaFreeHost(c->pinned);
  c->lane0.destroy_wait();
  c->lane0.prof.release_events();
  delete c;
}

const char* qtt_last_error(qtt_ctx_t c) { return c ? c->err.c_str() : "null context"; }

int qtt_ctx_set_profiling(qtt_ctx_t c, int on) {
  if (!c) return QTT_EINVAL;
  std::lock_guard<std::mutex> g(c->prof_mu);
  if (!on) prof_flush(c);
  c->profiling = on ? 1 : 0;
  return QTT_OK;
}

int qtt_ctx_profile(qtt_ctx_t c, int reset, double* out) {
  if (!c || !out) return QTT_EINVAL;
  std::lock_guard<std::mutex> g(c->prof_mu);
  prof_flush(c);
  for (int i = 0; i < 3; ++i) {
    out[3 * i] = (double)c->prof.n[i];
    out[3 * i + 1] = c->prof.ms[i];
    out[3 * i + 2] = c->prof.flops[i];
  }
  out[9] = c->prof.sweeps;
  out[10] = c->prof.tc_launches;
  if (reset) c->prof = ProfBuf();
  return QTT_OK;
}
size_t qtt_ctx_bytes_in_use(qtt_ctx_t c) { return c ? c->arena.used : 0; }
size_t qtt_ctx_bytes_peak(qtt_ctx_t c) { return c ? c->arena.peak : 0; }
uint64_t qtt_ctx_launches(qtt_ctx_t c) { return c ? c->launches.load() : 0; }

int qtt_tt_create(qtt_ctx_t ctx, int L, const int* dims, const int* ranks, const double* cores,
                  qtt_tt_t* out) {
  API_BEGIN(ctx)
  QREQ(ctx && out && dims && ranks && cores, "qtt_tt_create: null argument");
  QREQ(ranks[0] == 1 && ranks[L] == 1, "qtt_tt_create: boundary ranks must be 1");
  qtt_tt* t = new_tt(ctx, &ctx->arena, L, dims);
  long long off = 0;
  const size_t es = ctx->esize();
  for (int k = 0; k <= L; ++k) {
    QREQ(ranks[k] >= 1, "qtt_tt_create: ranks must be >= 1");
    t->ranks[k] = ranks[k];
  }
  for (int k = 0; k < L; ++k) {
    QREQ(dims[k] >= 1, "qtt_tt_create: dims must be >= 1");
    const long long cnt = t->count(k);
    t->core[k] = ctx->arena.alloc(cnt * es);
    if (ctx->prec == QTT_FP64) {
      QCHECK(cudaMemcpyAsync(t->core[k], cores + 2 * off, cnt * 16, cudaMemcpyHostToDevice,
                             ctx->stream));
    } else {
      std::vector<float> h(2 * cnt);
      for (long long i = 0; i < 2 * cnt; ++i) h[i] = (float)cores[2 * off + i];
      QCHECK(cudaMemcpyAsync(t->core[k], h.data(), cnt * 8, cudaMemcpyHostToDevice, ctx->stream));
      QCHECK(cudaStreamSynchronize(ctx->stream));
    }
    off += cnt;
  }
  QCHECK(cudaStreamSynchronize(ctx->stream));
  *out = t;
  return QTT_OK;
  API_END
}

int qtt_tt_from_dense(qtt_ctx_t ctx, int L, const int* dims, const double* dense, double eps,
                      int rmax, qtt_tt_t* out) {
  API_BEGIN(ctx)
  QREQ(ctx && dims && dense && out, "qtt_tt_from_dense: null argument");
  QREQ(L >= 1 && L <= QTT_MAX_CORES && eps >= 0 && rmax >= 1, "qtt_tt_from_dense: bad arguments");
  long long tot = 1;
  for (int k = 0; k < L; ++k) {
    QREQ(dims[k] >= 1, "qtt_tt_from_dense: dims must be >= 1");
    tot *= dims[k];
    QREQ(tot < (1ll << 34), "qtt_tt_from_dense: tensor too large");
  }
  Eng<double> e(ctx);
  Cx<double>* T = e.alloc(tot);
  QCHECK(cudaMemcpyAsync(T, dense, (size_t)tot * 16, cudaMemcpyHostToDevice, ctx->stream));
  std::vector<int> dv(dims, dims + L), ranks;
  std::vector<Cx<double>*> cores = tt_svd_device(e, T, dv, eps, rmax, ranks, true);
  qtt_tt* t = new_tt(ctx, &ctx->arena, L, dims);
  for (int k = 0; k <= L; ++k) t->ranks[k] = ranks[k];
  if (ctx->prec == QTT_FP64) {
    for (int k = 0; k < L; ++k) t->core[k] = cores[k];
  } else {
    Eng<float> f(ctx);
    for (int k = 0; k < L; ++k) t->core[k] = to_prec<float>(f, cores[k], t->count(k));
  }
  QCHECK(cudaStreamSynchronize(ctx->stream));
  *out = t;
  return QTT_OK;
  API_END
}

int qtt_tt_shape(qtt_tt_t t, int* L, int* dims, int* ranks) {
  if (!t || !L) return QTT_EINVAL;
  *L = t->L;
  for (int k = 0; k < t->L; ++k)
    if (dims) dims[k] = t->dims[k];
  for (int k = 0; k <= t->L; ++k)
    if (ranks) ranks[k] = t->ranks[k];
  return QTT_OK;
}

int qtt_tt_export(qtt_ctx_t ctx, qtt_tt_t t, double* cores) {
  API_BEGIN(ctx)
  QREQ(ctx && t && cores, "qtt_tt_export: null argument");
  long long off = 0;
  for (int k = 0; k < t->L; ++k) {
    const long long cnt = t->count(k);
    if (ctx->prec == QTT_FP64) {
      QCHECK(cudaMemcpyAsync(cores + 2 * off, t->core[k], cnt * 16, cudaMemcpyDeviceToHost,
                             ctx->stream));
    } else {
      std::vector<float> h(2 * cnt);
      QCHECK(cudaMemcpyAsync(h.data(), t->core[k], cnt * 8, cudaMemcpyDeviceToHost, ctx->stream));
      QCHECK(cudaStreamSynchronize(ctx->stream));
      for (long long i = 0; i < 2 * cnt; ++i) cores[2 * off + i] = h[i];
    }
    off += cnt;
  }
  QCHECK(cudaStreamSynchronize(ctx->stream));
  return QTT_OK;
  API_END
}

int qtt_tt_to_dense(qtt_ctx_t ctx, qtt_tt_t t, double* dense) {
  API_BEGIN(ctx)
  QREQ(ctx && t && dense, "qtt_tt_to_dense: null argument");
  QREQ(t->ctx == ctx, "qtt_tt_to_dense: TT from another context");
  QREQ(t->ranks[t->L] == 1, "qtt_tt_to_dense: ranks[L] must be 1");
  DISPATCH(ctx, to_dense_impl, ctx, t, dense);
  return QTT_OK;
  API_END
}

void qtt_tt_free(qtt_tt_t t) { free_tt(t); }

int qtt_op_create(qtt_ctx_t ctx, int L, const int* d_out, const int* d_in, const int* ranks,
                  const int* diag, const double* cores, qtt_op_t* out) {
  API_BEGIN(ctx)
  QREQ(ctx && out && d_out && d_in && ranks && diag && cores, "qtt_op_create: null argument");
  QREQ(L >= 1 && L <= QTT_MAX_CORES, "qtt_op_create: L out of range");
  QREQ(ranks[0] == 1 && ranks[L] == 1, "qtt_op_create: boundary ranks must be 1");
  qtt_op* o = new qtt_op();
  o->ctx = ctx;
  o->L = L;
  for (int k = 0; k <= L; ++k) o->ranks[k] = ranks[k];
  for (int k = 0; k < L; ++k) {
    o->dout[k] = d_out[k];
    o->din[k] = d_in[k];
    o->diag[k] = diag[k] ? 1 : 0;
    if (o->diag[k] && d_out[k] != d_in[k]) {
      delete o;
      throw QttError(QTT_EINVAL, "qtt_op_create: diagonal core needs d_out == d_in");
    }
  }
  o->n = (L - 1) / 3;
  long long off = 0;
  const size_t es = ctx->esize();
  for (int k = 0; k < L; ++k) {
    const long long cnt = o->count(k);
    o->core[k] = ctx->arena.alloc(cnt * es);
    if (ctx->prec == QTT_FP64) {
      QCHECK(cudaMemcpyAsync(o->core[k], cores + 2 * off, cnt * 16, cudaMemcpyHostToDevice,
                             ctx->stream));
    } else {
      std::vector<float> h(2 * cnt);
      for (long long i = 0; i < 2 * cnt; ++i) h[i] = (float)cores[2 * off + i];
      QCHECK(cudaMemcpyAsync(o->core[k], h.data(), cnt * 8, cudaMemcpyHostToDevice, ctx->stream));
      QCHECK(cudaStreamSynchronize(ctx->stream));
    }
    off += cnt;
  }
  QCHECK(cudaStreamSynchronize(ctx->stream));
  *out = o;
  return QTT_OK;
  API_END
}

int qtt_op_shape(qtt_op_t o, int* L, int* d_out, int* d_in, int* ranks, int* diag) {
  if (!o || !L) return QTT_EINVAL;
  *L = o->L;
  for (int k = 0; k < o->L; ++k) {
    if (d_out) d_out[k] = o->dout[k];
    if (d_in) d_in[k] = o->din[k];
    if (diag) diag[k] = o->diag[k];
  }
  for (int k = 0; k <= o->L; ++k)
    if (ranks) ranks[k] = o->ranks[k];
  return QTT_OK;
}

int qtt_op_export(qtt_ctx_t ctx, qtt_op_t o, double* cores) {
  API_BEGIN(ctx)
  QREQ(ctx && o && cores, "qtt_op_export: null argument");
  long long off = 0;
  for (int k = 0; k < o->L; ++k) {
    const long long cnt = o->count(k);
    if (ctx->prec == QTT_FP64) {
      QCHECK(cudaMemcpyAsync(cores + 2 * off, o->core[k], cnt * 16, cudaMemcpyDeviceToHost,
                             ctx->stream));
    } else {
      std::vector<float> h(2 * cnt);
      QCHECK(cudaMemcpyAsync(h.data(), o->core[k], cnt * 8, cudaMemcpyDeviceToHost, ctx->stream));
      QCHECK(cudaStreamSynchronize(ctx->stream));
      for (long long i = 0; i < 2 * cnt; ++i) cores[2 * off + i] = h[i];
    }
    off += cnt;
  }
  QCHECK(cudaStreamSynchronize(ctx->stream));
  return QTT_OK;
  API_END
}

void qtt_op_free(qtt_op_t o) {
  if (!o) return;
  // cached operators are owned by their context
  for (auto& kv : o->ctx->sfft_cache)
    if (kv.second == o) return;
  for (auto& kv : o->ctx->gamma_cache)
    if (kv.second == o) return;
  free_op(o);
}

int qtt_from_phase_field(qtt_ctx_t ctx, const uint8_t* phase, const int shape[3], int n,
                         int nphase, const double* E, const double* nu, const double* lame0,
                         double eps_tt, int rmax, qtt_op_t* dC) {
  API_BEGIN(ctx)
  QREQ(ctx && phase && shape && E && nu && dC, "qtt_from_phase_field: null argument");
  QREQ(n >= 1 && 3 * n + 1 <= QTT_MAX_CORES, "qtt_from_phase_field: n out of range");
  QREQ(nphase >= 1 && nphase <= 255, "qtt_from_phase_field: nphase out of range");
  const long long N = 1ll << n;
  int bc[3];
  long long cells = 1;
  for (int a = 0; a < 3; ++a) {
    QREQ(shape[a] == 1 || shape[a] == N, "qtt_from_phase_field: extents must be 1 or 2^n");
    bc[a] = shape[a] == 1;
    cells *= shape[a];
  }
  double lam0, mu0;
  if (lame0) {
    lam0 = lame0[0];
    mu0 = lame0[1];
  } else {
    double lmin = 1e300, lmax = -1e300, mmin = 1e300, mmax = -1e300;
    for (int p = 0; p < nphase; ++p) {
      double l, m;
      lame_of(E[p], nu[p], l, m);
      lmin = std::min(lmin, l);
      lmax = std::max(lmax, l);
      mmin = std::min(mmin, m);
      mmax = std::max(mmax, m);
    }
    lam0 = 0.5 * (lmin + lmax);
    mu0 = 0.5 * (mmin + mmax);
  }
  double C0[36];
  voigt_stiffness(lam0, mu0, C0);
  std::vector<double> dCh(36 * nphase);
  for (int p = 0; p < nphase; ++p) {
    double l, m, Cp[36];
    lame_of(E[p], nu[p], l, m);
    voigt_stiffness(l, m, Cp);
    for (int i = 0; i < 36; ++i) dCh[p * 36 + i] = Cp[i] - C0[i];
  }
  qtt_op* o = raised_from_phases(ctx, phase, cells, dCh.data(), nphase, n, bc, eps_tt, rmax);
  o->n = n;
  o->has_c0 = 1;
  o->lame0[0] = lam0;
  o->lame0[1] = mu0;
  memcpy(o->C0, C0, sizeof(C0));
  *dC = o;
  return QTT_OK;
  API_END
}

int qtt_rank_estimate(qtt_ctx_t ctx, const uint8_t* phase_a, const int shape_a[3],
                      const uint8_t* phase_b, const int shape_b[3], int n, int nphase,
                      const double* E, const double* nu, double eps_tt, int n_target,
                      double* out) {
  API_BEGIN(ctx)
  QREQ(ctx && phase_a && phase_b && shape_a && shape_b && E && nu && out,
       "qtt_rank_estimate: null argument");
  QREQ(n_target >= n, "qtt_rank_estimate: n_target below n");
  int ra = 0, rb = 0;
  for (int pass = 0; pass < 2; ++pass) {
    qtt_op_t o = nullptr;
    const int rc = qtt_from_phase_field(ctx, pass ? phase_b : phase_a, pass ? shape_b : shape_a,
                                        n + pass, nphase, E, nu, nullptr, eps_tt, 1 << 30, &o);
    if (rc < 0) throw QttError(rc, ctx->err);
    int r = 1;
    for (int k = 0; k <= o->L; ++k) r = std::max(r, o->ranks[k]);
    free_op(o);
    (pass ? rb : ra) = r;
  }
  const double g = (double)rb / (double)ra;
  out[0] = ra;
  out[1] = rb;
  out[2] = g;
  out[3] = ra * std::pow(g, (double)(n_target - n));
  return QTT_OK;
  API_END
}

int qtt_sfft_operator(qtt_ctx_t ctx, int n, int adjoint, double eps, qtt_op_t* out) {
  API_BEGIN(ctx)
  QREQ(ctx && out, "qtt_sfft_operator: null argument");
  *out = build_sfft(ctx, n, adjoint ? 1 : 0, eps);
  return QTT_OK;
  API_END
}

int qtt_gamma_operator(qtt_ctx_t ctx, int n, double lambda0, double mu0, int scheme,
                       double eps_tt, int rmax, qtt_op_t* out) {
  API_BEGIN(ctx)
  QREQ(ctx && out, "qtt_gamma_operator: null argument");
  *out = build_gamma(ctx, n, lambda0, mu0, scheme, eps_tt, rmax);
  return QTT_OK;
  API_END
}

int qtt_op_apply(qtt_ctx_t ctx, qtt_op_t op, qtt_tt_t in, double eps_tt, int rmax, int oversample,
                 int apply_id, qtt_tt_t* out) {
  API_BEGIN(ctx)
  QREQ(ctx && op && in && out, "qtt_op_apply: null argument");
  QREQ(rmax >= 1 && oversample >= 0 && eps_tt >= 0, "qtt_op_apply: bad tolerance/rank");
  int cap = 0;
  *out = DISPATCH(ctx, op_apply_impl, ctx, op, in, eps_tt, rmax, oversample, apply_id, &cap);
  return cap ? QTT_WRANKCAP : QTT_OK;
  API_END
}

static int cubic_n(const qtt_tt* t) {
  QREQ((t->L - 1) % 3 == 0 && t->L >= 4, "TT is not a controlled QTT of a cubic grid");
  return (t->L - 1) / 3;
}

int sfft_apply(qtt_ctx_t ctx, qtt_tt_t in, double eps_tt, int rmax, qtt_tt_t* out) {
  API_BEGIN(ctx)
  QREQ(ctx && in && out, "sfft_apply: null argument");
  qtt_op* S = cached_sfft(ctx, cubic_n(in), 0);
  int cap = 0;
  *out = DISPATCH(ctx, op_apply_impl, ctx, S, in, eps_tt, rmax, 16, 1, &cap);
  return cap ? QTT_WRANKCAP : QTT_OK;
  API_END
}

int isfft_apply(qtt_ctx_t ctx, qtt_tt_t in, double eps_tt, int rmax, qtt_tt_t* out) {
  API_BEGIN(ctx)
  QREQ(ctx && in && out, "isfft_apply: null argument");
  qtt_op* S = cached_sfft(ctx, cubic_n(in), 1);
  int cap = 0;
  *out = DISPATCH(ctx, op_apply_impl, ctx, S, in, eps_tt, rmax, 16, 3, &cap);
  return cap ? QTT_WRANKCAP : QTT_OK;
  API_END
}

int gamma0_apply(qtt_ctx_t ctx, const int n[3], double lambda0, double mu0, int scheme,
                 qtt_tt_t in, double eps_tt, int rmax, qtt_tt_t* out) {
  API_BEGIN(ctx)
  QREQ(ctx && n && in && out, "gamma0_apply: null argument");
  QREQ(n[0] == n[1] && n[1] == n[2] && n[0] == cubic_n(in), "gamma0_apply: grid mismatch");
  qtt_op* G = cached_gamma(ctx, n[0], lambda0, mu0, scheme, eps_tt, 1 << 30);
  int cap = 0;
  *out = DISPATCH(ctx, op_apply_impl, ctx, G, in, eps_tt, rmax, 16, 2, &cap);
  return cap ? QTT_WRANKCAP : QTT_OK;
  API_END
}

int tt_round(qtt_ctx_t ctx, qtt_tt_t inout, double eps_tt, int rmax) {
  API_BEGIN(ctx)
  QREQ(ctx && inout, "tt_round: null argument");
  QREQ(rmax >= 1 && eps_tt >= 0, "tt_round: bad tolerance/rank");
  const int cap = DISPATCH(ctx, round_impl, ctx, inout, eps_tt, rmax);
  return cap ? QTT_WRANKCAP : QTT_OK;
  API_END
}

int qtt_tt_dot(qtt_ctx_t ctx, qtt_tt_t a, qtt_tt_t b, double* re, double* im) {
  API_BEGIN(ctx)
  QREQ(ctx && a && b && re && im, "qtt_tt_dot: null argument");
  DISPATCH(ctx, dot_impl, ctx, a, b, re, im);
  return QTT_OK;
  API_END
}

int qtt_op_mean_apply(qtt_ctx_t ctx, qtt_op_t op, qtt_tt_t x, double* out) {
  API_BEGIN(ctx)
  QREQ(ctx && op && x && out, "qtt_op_mean_apply: null argument");
  std::vector<double> m;
  DISPATCH(ctx, mean_impl, ctx, op, x, m);
  memcpy(out, m.data(), sizeof(double) * m.size());
  return QTT_OK;
  API_END
}

int ls_solve_ops(qtt_ctx_t ctx, qtt_op_t dC, qtt_op_t S, qtt_op_t Sh, qtt_op_t gamma,
                 const double C0[36], const double E_voigt[6], const qtt_solve_params* p,
                 double sigma_bar[12], qtt_solve_info* info) {
  API_BEGIN(ctx)
  QREQ(ctx && dC && S && Sh && gamma && C0 && E_voigt && p && sigma_bar,
       "ls_solve_ops: null argument");
  QREQ(p->tol > 0 && p->max_iter >= 1 && p->rmax >= 1 && p->eps_tt >= 0 && p->oversample >= 0,
       "ls_solve_ops: bad parameters");
  return DISPATCH(ctx, solve_impl, ctx, dC, S, Sh, gamma, C0, E_voigt, p, sigma_bar, info, 0);
  API_END
}

int ls_solve(qtt_ctx_t ctx, qtt_op_t dC, const double E_voigt[6], const qtt_solve_params* p,
             double sigma_bar[12], qtt_solve_info* info) {
  API_BEGIN(ctx)
  QREQ(ctx && dC && E_voigt && p && sigma_bar, "ls_solve: null argument");
  QREQ(dC->has_c0, "ls_solve: dC must come from qtt_from_phase_field");
  const int n = dC->n;
  qtt_op* S = cached_sfft(ctx, n, 0);
  qtt_op* Sh = cached_sfft(ctx, n, 1);
  qtt_op* G = solve_gamma(ctx, dC, p);
  return DISPATCH(ctx, solve_impl, ctx, dC, S, Sh, G, dC->C0, E_voigt, p, sigma_bar, info, 0);
  API_END
}

}  // extern "C"

namespace {
// One unit-load LS solve of a job queue.
struct SolveJob {
  const qtt_op* dC = nullptr;
  const qtt_op *S = nullptr, *Sh = nullptr, *G = nullptr;
  int load = 0;
  double sig[12] = {0};
  qtt_solve_info inf{};
  int status = QTT_OK;
  std::string err;
  qtt_tt* keep = nullptr;
};

// Runs the jobs in queue order on nl lanes. One lane per concurrently solved
// load: own stream, own slice of the workspace (so that no lane reuses memory
// another lane's kernels still touch), own pinned readback buffer. Operators
// are shared read-only. Errors stay in the jobs.
void run_jobs(qtt_ctx* ctx, std::vector<SolveJob>& jobs, const qtt_solve_params* p, int nl,
              bool keep) {
  const int nj = (int)jobs.size();
  nl = std::max(1, std::min(nl, nj));
  std::vector<Lane> lanes(nl);
  std::vector<Arena> arenas(nl);
  std::vector<void*> blocks(nl, nullptr);
  if (nl > 1) {
    size_t freeb = 0;
    {
      std::lock_guard<std::mutex> g(ctx->arena.mu);
      for (auto& kv : ctx->arena.free_) freeb = std::max(freeb, kv.second);
    }
    // the lanes share 7/8 of the largest free block; the rest stays with the
    // context for what the solves leave behind (kept final strains)
    const size_t share = freeb - freeb / 8;
    const size_t slice = ((share / nl) & ~(size_t)255) - 4096;
    QREQ(share / nl > (64u << 20), "concurrent solves: workspace too small for the lanes");
    for (int l = 0; l < nl; ++l) {
      blocks[l] = ctx->arena.alloc(slice);
      arenas[l].init(blocks[l], slice);
      lanes[l].arena = &arenas[l];
      QCHECK(cudaStreamCreateWithFlags(&lanes[l].stream, cudaStreamNonBlocking));
      QCHECK(cudaMallocHost(&lanes[l].pinned, 1 << 16));
    }
  }
  // one lane: the context's own (its stream, arena and profile buffer)
  auto lane_of = [&](int l) { return nl > 1 ? &lanes[l] : &ctx->lane0; };
  std::atomic<int> next{0};
  struct LaneCount {
    qtt_ctx* c;
    LaneCount(qtt_ctx* ctx, int nl) : c(ctx) { c->active_lanes = nl; }
    ~LaneCount() { c->active_lanes = 1; }
  } lane_count(ctx, nl);
  auto worker = [&](int lane_id) {
    cudaSetDevice(ctx->device);
    for (int j = next++; j < nj; j = next++) {
      SolveJob& J = jobs[j];
      double Ev[6] = {0, 0, 0, 0, 0, 0};
      Ev[J.load] = 1.0;
      try {
        J.status = DISPATCH(ctx, solve_impl, ctx, J.dC, J.S, J.Sh, J.G, J.dC->C0, Ev, p, J.sig,
                            &J.inf, 0, lane_of(lane_id), keep ? &J.keep : nullptr);
      } catch (const QttError& ex) {
        J.status = ex.code;
        J.err = ex.what();
      } catch (const std::exception& ex) {
        J.status = QTT_EINVAL;
        J.err = ex.what();
      }
    }
  };
  if (nl > 1) {
    std::vector<std::thread> th;
    for (int l = 0; l < nl; ++l) th.emplace_back(worker, l);
    for (auto& t : th) t.join();
    for (int l = 0; l < nl; ++l) {
      cudaStreamSynchronize(lanes[l].stream);
      lanes[l].destroy_wait();
      {
        std::lock_guard<std::mutex> g(ctx->prof_mu);
        lanes[l].prof.merge_into(ctx->prof);
      }
      lanes[l].prof.release_events();
      cudaStreamDestroy(lanes[l].stream);
      cudaFreeHost(lanes[l].pinned);
      ctx->arena.release(blocks[l]);
    }
  } else {
    worker(0);
  }
}

// First error of a finished queue (its kept strains freed), else the worst
// warning.
int jobs_status(std::vector<SolveJob>& jobs) {
  int worst = QTT_OK;
  for (auto& J : jobs)
    if (J.status < 0) {
      for (auto& K : jobs) free_tt(K.keep);
      throw QttError(J.status, J.err);
    }
  for (auto& J : jobs) worst = std::max(worst, J.status);
  return worst;
}

int solve_loads(qtt_ctx_t ctx, qtt_op_t dC, const qtt_solve_params* p, const int* loads,
                int nloads, double* Ceff, qtt_solve_info* info, std::vector<qtt_tt*>* keep) {
  QREQ(ctx && dC && p && Ceff, "ls_solve_ceff: null argument");
  QREQ(dC->has_c0, "ls_solve_ceff: dC must come from qtt_from_phase_field");
  int all[6] = {0, 1, 2, 3, 4, 5};
  if (!loads) {
    loads = all;
    nloads = 6;
  }
  QREQ(nloads >= 1 && nloads <= 6, "ls_solve_ceff: nloads out of range");
  for (int l = 0; l < nloads; ++l) QREQ(loads[l] >= 0 && loads[l] < 6, "ls_solve_ceff: bad load");
  for (int i = 0; i < 36; ++i) Ceff[i] = 0;
  const int n = dC->n;
  qtt_op* S = cached_sfft(ctx, n, 0);
  qtt_op* Sh = cached_sfft(ctx, n, 1);
  qtt_op* G = solve_gamma(ctx, dC, p);
  QCHECK(cudaStreamSynchronize(ctx->stream));
  std::vector<SolveJob> jobs(nloads);
  for (int l = 0; l < nloads; ++l) {
    jobs[l].dC = dC;
    jobs[l].S = S;
    jobs[l].Sh = Sh;
    jobs[l].G = G;
    jobs[l].load = loads[l];
  }
  run_jobs(ctx, jobs, p, std::min(ctx->concurrent_loads, 6), keep != nullptr);
  const int worst = jobs_status(jobs);
  if (keep) {
    keep->assign(nloads, nullptr);
    for (int l = 0; l < nloads; ++l) (*keep)[l] = jobs[l].keep;
  }
  for (int l = 0; l < nloads; ++l) {
    for (int i = 0; i < 6; ++i) Ceff[loads[l] * 6 + i] = jobs[l].sig[2 * i];
    if (info) info[l] = jobs[l].inf;
  }
  return worst;
}

// An arbitrary list of (microstructure, unit load) solves through one queue,
// largest grids first; sigma_bar of job j at sig + 12 j.
int solve_jobs(qtt_ctx_t ctx, int njobs, const qtt_op_t* dC, const int* load,
               const qtt_solve_params* p, double* sig, qtt_solve_info* info) {
  QREQ(ctx && dC && load && p && sig && njobs >= 1, "ls_solve_jobs: bad argument");
  std::vector<SolveJob> jobs((size_t)njobs);
  for (int j = 0; j < njobs; ++j) {
    const qtt_op* d = dC[j];
    QREQ(d, "ls_solve_jobs: null operator");
    QREQ(d->has_c0, "ls_solve_jobs: dC must come from qtt_from_phase_field");
    QREQ(load[j] >= 0 && load[j] < 6, "ls_solve_jobs: load out of range");
    SolveJob& J = jobs[(size_t)j];
    J.dC = d;
    J.S = cached_sfft(ctx, d->n, 0);
    J.Sh = cached_sfft(ctx, d->n, 1);
    J.G = solve_gamma(ctx, d, p);
    J.load = load[j];
  }
  QCHECK(cudaStreamSynchronize(ctx->stream));
  std::vector<int> order((size_t)njobs);
  for (int j = 0; j < njobs; ++j) order[(size_t)j] = j;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return jobs[(size_t)a].dC->n > jobs[(size_t)b].dC->n; });
  std::vector<SolveJob> queue((size_t)njobs);
  for (int j = 0; j < njobs; ++j) queue[(size_t)j] = jobs[(size_t)order[(size_t)j]];
  run_jobs(ctx, queue, p, ctx->concurrent_loads, false);
  const int worst = jobs_status(queue);
  for (int j = 0; j < njobs; ++j) {
    const SolveJob& J = queue[(size_t)j];
    const int dst = order[(size_t)j];
    for (int r = 0; r < 12; ++r) sig[(size_t)dst * 12 + r] = J.sig[r];
    if (info) info[dst] = J.inf;
  }
  return worst;
}

// nitems x 6 unit-load solves through one queue, largest grids first.
int solve_batched(qtt_ctx_t ctx, int nitems, const qtt_op_t* dC, const qtt_solve_params* p,
                  double* Ceff, qtt_solve_info* info) {
  QREQ(ctx && dC && p && Ceff && nitems >= 1, "ls_solve_batched: bad argument");
  for (int i = 0; i < nitems; ++i) {
    QREQ(dC[i], "ls_solve_batched: null operator");
    QREQ(dC[i]->has_c0, "ls_solve_batched: dC must come from qtt_from_phase_field");
  }
  std::vector<SolveJob> jobs((size_t)nitems * 6);
  for (int i = 0; i < nitems; ++i) {
    const qtt_op* d = dC[i];
    qtt_op* S = cached_sfft(ctx, d->n, 0);
    qtt_op* Sh = cached_sfft(ctx, d->n, 1);
    qtt_op* G = solve_gamma(ctx, d, p);
    for (int k = 0; k < 6; ++k) {
      SolveJob& J = jobs[(size_t)i * 6 + k];
      J.dC = d;
      J.S = S;
      J.Sh = Sh;
      J.G = G;
      J.load = k;
    }
  }
  QCHECK(cudaStreamSynchronize(ctx->stream));
  // queue order: largest grids first (they take longest), then item, load
  std::vector<int> order(jobs.size());
  for (size_t j = 0; j < order.size(); ++j) order[j] = (int)j;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return jobs[a].dC->n > jobs[b].dC->n; });
  std::vector<SolveJob> queue(jobs.size());
  for (size_t j = 0; j < order.size(); ++j) queue[j] = jobs[order[j]];
  run_jobs(ctx, queue, p, ctx->concurrent_loads, false);
  const int worst = jobs_status(queue);
  for (size_t j = 0; j < order.size(); ++j) {
    const SolveJob& J = queue[j];
    const int item = order[j] / 6, k = J.load;
    for (int r = 0; r < 6; ++r) Ceff[(size_t)item * 36 + k * 6 + r] = J.sig[2 * r];
    if (info) info[(size_t)item * 6 + k] = J.inf;
  }
  return worst;
}

}  // namespace

extern "C" {

int ls_solve_batched(qtt_ctx_t ctx, int nitems, const qtt_op_t* dC, const qtt_solve_params* p,
                     double* Ceff, qtt_solve_info* info) {
  API_BEGIN(ctx)
  return solve_batched(ctx, nitems, dC, p, Ceff, info);
  API_END
}

int ls_solve_jobs(qtt_ctx_t ctx, int njobs, const qtt_op_t* dC, const int* load,
                  const qtt_solve_params* p, double* sigma_bar, qtt_solve_info* info) {
  API_BEGIN(ctx)
  return solve_jobs(ctx, njobs, dC, load, p, sigma_bar, info);
  API_END
}

int ls_solve_ceff(qtt_ctx_t ctx, qtt_op_t dC, const qtt_solve_params* p, const int* loads,
                  int nloads, double* Ceff, qtt_solve_info* info) {
  API_BEGIN(ctx)
  return solve_loads(ctx, dC, p, loads, nloads, Ceff, info, nullptr);
  API_END
}

int qtt_from_phase_matrices(qtt_ctx_t ctx, const uint8_t* phase, const int shape[3], int n,
                            int nphase, const double* mats, double eps_tt, int rmax,
                            qtt_op_t* out) {
  API_BEGIN(ctx)
  QREQ(ctx && phase && shape && mats && out, "qtt_from_phase_matrices: null argument");
  QREQ(n >= 1 && 3 * n + 1 <= QTT_MAX_CORES, "qtt_from_phase_matrices: n out of range");
  QREQ(nphase >= 1 && nphase <= 255, "qtt_from_phase_matrices: nphase out of range");
  const long long N = 1ll << n;
  int bc[3];
  long long cells = 1;
  for (int a = 0; a < 3; ++a) {
    QREQ(shape[a] == 1 || shape[a] == N, "qtt_from_phase_matrices: extents must be 1 or 2^n");
    bc[a] = shape[a] == 1;
    cells *= shape[a];
  }
  qtt_op* o = raised_from_phases(ctx, phase, cells, mats, nphase, n, bc, eps_tt, rmax);
  o->n = n;
  *out = o;
  return QTT_OK;
  API_END
}

int qtt_op_sandwich_mean(qtt_ctx_t ctx, qtt_op_t op, qtt_tt_t y, qtt_tt_t x, double* re,
                         double* im) {
  API_BEGIN(ctx)
  QREQ(ctx && op && y && x && re && im, "qtt_op_sandwich_mean: null argument");
  double v[2];
  if (ctx->prec == QTT_FP64) {
    Eng<double> e(ctx);
    op_sandwich<double>(e, op, y, x, v);
  } else {
    Eng<float> e(ctx);
    op_sandwich<float>(e, op, y, x, v);
  }
  *re = v[0];
  *im = v[1];
  return QTT_OK;
  API_END
}

int ls_solve_ceff_grad(qtt_ctx_t ctx, qtt_op_t dC, const uint8_t* phase, const int shape[3],
                       int nphase, const double* E, const double* nu, int nparams,
                       const int* param_phase, const int* param_kind, const qtt_solve_params* p,
                       double* Ceff, double* dCeff, qtt_solve_info* info) {
  API_BEGIN(ctx)
  QREQ(ctx && dC && phase && shape && E && nu && p && Ceff && (nparams == 0 || dCeff),
       "ls_solve_ceff_grad: null argument");
  QREQ(nparams >= 0 && nparams <= 64 && (nparams == 0 || (param_phase && param_kind)),
       "ls_solve_ceff_grad: bad parameter list");
  for (int q = 0; q < nparams; ++q)
    QREQ(param_phase[q] >= 0 && param_phase[q] < nphase &&
             (param_kind[q] == 0 || param_kind[q] == 1),
         "ls_solve_ceff_grad: bad parameter");
  std::vector<qtt_tt*> eps;
  const int st = solve_loads(ctx, dC, p, nullptr, 6, Ceff, info, &eps);
  struct Guard {
    std::vector<qtt_tt*>& v;
    ~Guard() {
      for (auto* t : v) free_tt(t);
    }
  } guard{eps};
  for (int q = 0; q < nparams; ++q) {
    // dC/dp: derivative of the phase's isotropic stiffness through
    // lambda(E, nu), mu(E, nu); zero in the other phases
    const double e0 = E[param_phase[q]], n0 = nu[param_phase[q]];
    double dlam, dmu;
    if (param_kind[q] == 0) {
      dlam = n0 / ((1.0 + n0) * (1.0 - 2.0 * n0));
      dmu = 1.0 / (2.0 * (1.0 + n0));
    } else {
      const double dd = 1.0 - 2.0 * n0;
      dlam = e0 * (1.0 + 2.0 * n0 * n0) / ((1.0 + n0) * (1.0 + n0) * dd * dd);
      dmu = -e0 / (2.0 * (1.0 + n0) * (1.0 + n0));
    }
    std::vector<double> mats(36 * nphase, 0.0);
    voigt_stiffness(dlam, dmu, &mats[36 * param_phase[q]]);
    qtt_op_t D = nullptr;
    const int rc = qtt_from_phase_matrices(ctx, phase, shape, dC->n, nphase, mats.data(), p->eps_tt,
                                           1 << 30, &D);
    if (rc < 0) return rc;
    for (int k = 0; k < 6; ++k)
      for (int l = k; l < 6; ++l) {
        double v[2];
        if (ctx->prec == QTT_FP64) {
          Eng<double> e(ctx);
          op_sandwich<double>(e, D, eps[l], eps[k], v);
        } else {
          Eng<float> e(ctx);
          op_sandwich<float>(e, D, eps[l], eps[k], v);
        }
        // column-major like Ceff: dCeff[q*36 + k*6 + l] = dC_eff[l][k] / dp
        dCeff[q * 36 + k * 6 + l] = v[0];
        dCeff[q * 36 + l * 6 + k] = v[0];
      }
    free_op(D);
  }
  return st;
  API_END
}

int qtt_ctx_set_jacobi(qtt_ctx_t ctx, double tol_scale, int max_sweeps_fp32) {
  if (!ctx || !(tol_scale > 0) || max_sweeps_fp32 < 1 || max_sweeps_fp32 > 200) return QTT_EINVAL;
  ctx->jacobi_tol_scale = tol_scale;
  ctx->jacobi_max_sweeps32 = max_sweeps_fp32;
  return QTT_OK;
}

int qtt_ctx_set_contraction(qtt_ctx_t ctx, int mode) {
  if (!ctx || (mode != QTT_CONTRACT_SIMT && mode != QTT_CONTRACT_TF32X3 &&
               mode != QTT_CONTRACT_TC))
    return QTT_EINVAL;
  if (mode != QTT_CONTRACT_SIMT && ctx->prec != QTT_FP32) return QTT_EINVAL;
  ctx->contraction = mode;
  return QTT_OK;
}

int qtt_contraction_bench(qtt_ctx_t ctx, int mode, int M, int N, int K, int reps,
                          double* ms_per_launch, double* rel_err) {
  API_BEGIN(ctx)
  QREQ(ctx && ms_per_launch && rel_err && M >= 1 && N >= 1 && K >= 1 && reps >= 1,
       "qtt_contraction_bench: bad argument");
  QREQ(mode == QTT_CONTRACT_SIMT || mode == QTT_CONTRACT_TF32X3 || mode == QTT_CONTRACT_TC,
       "qtt_contraction_bench: unknown mode");
  Eng<float> e(ctx);
  Eng<double> d(ctx);
  const long long na = (long long)M * K, nb = (long long)K * N, nc = (long long)M * N;
  Cx<float>* A = e.alloc(na);
  Cx<float>* B = e.alloc(nb);
  Cx<float>* C = e.alloc(nc);
  sketch_kernel<float><<<grid1d(na), 256, 0, e.st()>>>(A, na, ctx->seed, 1, 0x7C0);
  e.post("sketch_kernel", __LINE__);
  sketch_kernel<float><<<grid1d(nb), 256, 0, e.st()>>>(B, nb, ctx->seed, 2, 0x7C0);
  e.post("sketch_kernel", __LINE__);
  // FP64 product of the same (FP32) operands as the reference
  Cx<double>* A64 = d.alloc(na);
  Cx<double>* B64 = d.alloc(nb);
  Cx<double>* C64 = d.alloc(nc);
  convert_kernel<float, double><<<grid1d(na), 256, 0, e.st()>>>(A, A64, na);
  e.post("convert_kernel", __LINE__);
  convert_kernel<float, double><<<grid1d(nb), 256, 0, e.st()>>>(B, B64, nb);
  e.post("convert_kernel", __LINE__);
  d.gemm(M, N, K, mref(A64, K, 1), mref(B64, N, 1), C64, N, 1, 0, 0, 0, 1, 1, 1);
  const int saved = ctx->contraction;
  ctx->contraction = mode;
  cudaEvent_t e0, e1;
  QCHECK(cudaEventCreate(&e0));
  QCHECK(cudaEventCreate(&e1));
  float ms = 0;
  try {
    e.gemm(M, N, K, mref(A, K, 1), mref(B, N, 1), C, N, 1, 0, 0, 0, 1, 1, 1, Cplx{1, 0},
           Cplx{0, 0}, 1, true);  // warm-up
    QCHECK(cudaEventRecord(e0, e.st()));
    for (int r = 0; r < reps; ++r)
      e.gemm(M, N, K, mref(A, K, 1), mref(B, N, 1), C, N, 1, 0, 0, 0, 1, 1, 1, Cplx{1, 0},
             Cplx{0, 0}, 1, true);
    QCHECK(cudaEventRecord(e1, e.st()));
    QCHECK(cudaEventSynchronize(e1));
    QCHECK(cudaEventElapsedTime(&ms, e0, e1));
  } catch (...) {
    ctx->contraction = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  ctx->contraction = saved;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::vector<Cx<float>> hc(nc);
  std::vector<Cx<double>> hr(nc);
  QCHECK(cudaMemcpyAsync(hc.data(), C, nc * sizeof(Cx<float>), cudaMemcpyDeviceToHost, e.st()));
  QCHECK(cudaMemcpyAsync(hr.data(), C64, nc * sizeof(Cx<double>), cudaMemcpyDeviceToHost, e.st()));
  QCHECK(cudaStreamSynchronize(e.st()));
  double num = 0, den = 0;
  for (long long i = 0; i < nc; ++i) {
    const double dx = hc[i].x - hr[i].x, dy = hc[i].y - hr[i].y;
    num += dx * dx + dy * dy;
    den += hr[i].x * hr[i].x + hr[i].y * hr[i].y;
  }
  *rel_err = den > 0 ? std::sqrt(num / den) : 0.0;
  *ms_per_launch = ms / reps;
  e.release(A);
  e.release(B);
  e.release(C);
  d.release(A64);
  d.release(B64);
  d.release(C64);
  return QTT_OK;
  API_END
}

int qtt_sfft_mpo_zipup(int n, double eps, int* ranks, double* cores, size_t cap,
                       size_t* needed) {
  if (n < 1 || n > 24 || !(eps > 0) || !ranks || !needed) return QTT_EINVAL;
  qtt_zipup::Mpo op;
  try {
    op = qtt_zipup::sfft_mpo(n, eps);
  } catch (const std::bad_alloc&) {
    return QTT_ENOMEM;
  }
  size_t tot = 0;
  for (const auto& c : op) tot += 2 * c.a.size();
  *needed = tot;
  ranks[0] = 1;
  for (int k = 0; k < n; ++k) ranks[k + 1] = op[k].r1;
  if (!cores || cap < tot) return QTT_EINVAL;
  size_t off = 0;
  for (const auto& c : op)
    for (const auto& z : c.a) {
      cores[off++] = z.real();
      cores[off++] = z.imag();
    }
  return QTT_OK;
}

int qtt_ctx_set_green_broadcast(qtt_ctx_t ctx, int on) {
  if (!ctx) return QTT_EINVAL;
  ctx->green_broadcast = on ? 1 : 0;
  return QTT_OK;
}

int qtt_ctx_set_svd(qtt_ctx_t ctx, int precond, int refine_sweeps) {
  if (!ctx || refine_sweeps < 1 || refine_sweeps > 60) return QTT_EINVAL;
  ctx->svd_precond = precond ? 1 : 0;
  ctx->svd_refine_sweeps = refine_sweeps;
  return QTT_OK;
}

int qtt_ctx_set_factorization(qtt_ctx_t ctx, int mode) {
  if (!ctx) return QTT_EINVAL;
  if (mode != QTT_FACTOR_NATIVE && mode != QTT_FACTOR_FP64 && mode != QTT_FACTOR_FP64_ROUNDING) {
    ctx->err = "qtt_ctx_set_factorization: unknown mode";
    return QTT_EINVAL;
  }
  ctx->factor = mode;
  return QTT_OK;
}

int qtt_ctx_set_tt_svd(qtt_ctx_t ctx, double gram_threshold) {
  if (!ctx || !(gram_threshold >= 0)) return QTT_EINVAL;
  ctx->gram_threshold = gram_threshold;
  return QTT_OK;
}

int qtt_ctx_set_concurrency(qtt_ctx_t ctx, int concurrent_loads) {
  if (!ctx || concurrent_loads < 1 || concurrent_loads > 64) return QTT_EINVAL;
  ctx->concurrent_loads = concurrent_loads;
  return QTT_OK;
}

}  // extern "C"

// ================================================================== inner product without allocation
//
// qtt_tt_dot_noalloc computes the same <a, b> as qtt_tt_dot for callers that
// must not allocate while they call it (nothing here touches cudaMalloc,
// cudaFree, the context's workspace arena or any allocating library call):
// every temporary lives in the file-scope device array below, sized for TT
// ranks up to QTT_NOALLOC_MAX_RANK and mode sizes up to QTT_NOALLOC_MAX_DIM.
// Host code cannot pass the array's name to a kernel (on the host it is only
// a stand-in symbol, not a device address): its device address is looked up
// once per device with cudaGetSymbolAddress, on the first call made on that
// device, and cached.

namespace {

constexpr int kNoAllocMaxRank = QTT_NOALLOC_MAX_RANK;
constexpr int kNoAllocMaxDim = QTT_NOALLOC_MAX_DIM;
// Layout (complex128 elements): E (R x R), F (R x R), EB (R x D x R),
// A64 (R x D x R), B64 (R x D x R).
constexpr long long kNoAllocRR = (long long)kNoAllocMaxRank * kNoAllocMaxRank;
constexpr long long kNoAllocRDR = (long long)kNoAllocMaxRank * kNoAllocMaxDim * kNoAllocMaxRank;
constexpr long long kNoAllocElems = 2 * kNoAllocRR + 3 * kNoAllocRDR;

static __device__ __align__(256) Cx<double> g_noalloc_scratch[kNoAllocElems];

std::mutex g_noalloc_mu;
std::map<int, Cx<double>*> g_noalloc_addr;  // device -> device address of the scratch

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
int noalloc_scratch(Cx<double>** out, std::string& err) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    err = "qtt_tt_dot_noalloc: no current CUDA device";
    return QTT_ECUDA;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  auto it = g_noalloc_addr.find(dev);
  if (it != g_noalloc_addr.end()) {
    *out = it->second;
    return QTT_OK;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    err = std::string("qtt_tt_dot_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
    return QTT_ECUDA;
  }
  g_noalloc_addr[dev] = (Cx<double>*)p;
  *out = (Cx<double>*)p;
  return QTT_OK;
}

// One launch of the strided GEMM kernel on caller-checked scratch buffers.
cudaError_t noalloc_gemm(cudaStream_t st, int M, int N, int K, const Cx<double>* A, long long a_rs,
                         long long a_cs, int conjA, const Cx<double>* B, long long b_rs,
                         long long b_cs, Cx<double>* C, long long c_rs, long long c_cs) {
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = A;
  g.a_rs = a_rs;
  g.a_cs = a_cs;
  g.conjA = conjA;
  g.B = B;
  g.b_rs = b_rs;
  g.b_cs = b_cs;
  g.C = C;
  g.c_rs = c_rs;
  g.c_cs = c_cs;
  g.nb1 = g.nb2 = g.nb3 = g.ksplit = 1;
  g.alpha_re = 1.0;
  const dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64), 1);
  gemm_kernel<double, 64, 64, 8, 4, 4><<<grid, 256, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace

extern "C" int qtt_tt_dot_noalloc(qtt_tt_t a, qtt_tt_t b, void* cuda_stream, double* re,
                                  double* im) {
  if (!a || !b || !re || !im) return QTT_EINVAL;
  qtt_ctx* c = a->ctx;
  auto fail = [&](int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
  };
  if (b->ctx != c) return fail(QTT_EINVAL, "qtt_tt_dot_noalloc: TTs from different contexts");
  const int L = a->L;
  if (b->L != L) return fail(QTT_EINVAL, "qtt_tt_dot_noalloc: core counts differ");
  for (int k = 0; k < L; ++k) {
    if (a->dims[k] != b->dims[k]) return fail(QTT_EINVAL, "qtt_tt_dot_noalloc: dims differ");
    if (a->dims[k] > kNoAllocMaxDim)
      return fail(QTT_EINVAL, "qtt_tt_dot_noalloc: mode size " + std::to_string(a->dims[k]) +
                                  " exceeds the maximum " + std::to_string(kNoAllocMaxDim));
  }
  for (int k = 0; k <= L; ++k)
    if (a->ranks[k] > kNoAllocMaxRank || b->ranks[k] > kNoAllocMaxRank)
      return fail(QTT_EINVAL, "qtt_tt_dot_noalloc: TT rank above the maximum " +
                                  std::to_string(kNoAllocMaxRank));
  // the work runs on the context's device; the caller's current device is
  // restored on every return
  int prev_dev = -1;
  if (cudaGetDevice(&prev_dev) != cudaSuccess)
    return fail(QTT_ECUDA, "qtt_tt_dot_noalloc: cudaGetDevice failed");
  struct RestoreDevice {
    int dev;
    ~RestoreDevice() { cudaSetDevice(dev); }
  } restore{prev_dev};
  if (cudaSetDevice(c->device) != cudaSuccess)
    return fail(QTT_ECUDA, "qtt_tt_dot_noalloc: cudaSetDevice failed");
  Cx<double>* base = nullptr;
  std::string err;
  const int rc = noalloc_scratch(&base, err);
  if (rc != QTT_OK) return fail(rc, err);
  // NULL: the context's stream, which is ordered after the work that wrote a and b
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->stream;
  Cx<double>* E = base;
  Cx<double>* F = base + kNoAllocRR;
  Cx<double>* EB = base + 2 * kNoAllocRR;
  Cx<double>* A64 = EB + kNoAllocRDR;
  Cx<double>* B64 = A64 + kNoAllocRDR;
  // E starts as the 1 x 1 matrix [1] (the array keeps the previous call's data)
  const Cx<double> one = mk<double>(1.0, 0.0);
  if (cudaMemcpyAsync(E, &one, sizeof(one), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(QTT_ECUDA, "qtt_tt_dot_noalloc: upload of the start value failed");
  for (int k = 0; k < L; ++k) {
    const int ra = a->ranks[k], rb = b->ranks[k], pa = a->ranks[k + 1], pb = b->ranks[k + 1];
    const int D = a->dims[k];
    const Cx<double>* Ak = (const Cx<double>*)a->core[k];
    const Cx<double>* Bk = (const Cx<double>*)b->core[k];
    if (c->prec != QTT_FP64) {
      convert_kernel<float, double><<<grid1d(a->count(k)), 256, 0, st>>>(
          (const Cx<float>*)a->core[k], A64, a->count(k));
      convert_kernel<float, double><<<grid1d(b->count(k)), 256, 0, st>>>(
          (const Cx<float>*)b->core[k], B64, b->count(k));
      Ak = A64;
      Bk = B64;
    }
    // EB (ra x D pb) = E (ra x rb) B_k (rb x D pb); F (pa x pb) = A_k^H EB
    cudaError_t e1 = noalloc_gemm(st, ra, D * pb, rb, E, rb, 1, 0, Bk, (long long)D * pb, 1, EB,
                                  (long long)D * pb, 1);
    cudaError_t e2 = noalloc_gemm(st, pa, pb, ra * D, Ak, 1, pa, 1, EB, pb, 1, F, pb, 1);
    if (e1 != cudaSuccess || e2 != cudaSuccess)
      return fail(QTT_ECUDA, std::string("qtt_tt_dot_noalloc: launch failed: ") +
                                 cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    std::swap(E, F);
  }
  double h[2];
  if (cudaMemcpyAsync(h, E, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(QTT_ECUDA, "qtt_tt_dot_noalloc: kernel or read-back failed");
  *re = h[0];
  *im = h[1];
  return QTT_OK;
}
