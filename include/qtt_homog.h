/*
 * qtt_homog.h -- C ABI of the GB300 (sm_103a) library for SFFT-based
 * homogenisation: the Moulinec-Suquet basic-scheme Lippmann-Schwinger
 * iteration on quantised tensor trains (arXiv 2412.11566, Alg. 2), ending in
 * the 6x6 effective stiffness C_eff.
 *
 * Data model (Sec. 3 eq. (tt_format), (tto_format); Sec. 4.3):
 *   - A tensor train (TT) with L cores; core k has shape (r_{k-1}, d_k, r_k),
 *     r_0 = r_L = 1, stored row-major (the last index is fastest). Host arrays
 *     hold complex numbers as interleaved (re, im) doubles; the cores of one TT
 *     are concatenated in core order.
 *   - A controlled QTT on a 2^n grid per axis has L = 3n + 1 cores: core 0 is
 *     the Voigt core (d = 6, order 11, 22, 33, 23, 13, 12; strains with
 *     engineering shear), then the n bits of x1, of x2, of x3, most significant
 *     bit first (eq. (binary_discretization)). The field value at voxel
 *     (i1, i2, i3) is the TT entry at (Voigt, bits(i1), bits(i2), bits(i3)).
 *   - An operator (TTO) has cores (a_{k-1}, d_out, d_in, a_k). A core flagged
 *     "diag" is a raised TT core (eq. (tt_to_tto)) stored as (a_{k-1}, d, a_k):
 *     G(a, i, j, b) = C(a, i, b) delta_ij.
 *
 * Ownership: handles are owned by the library until their *_free call. All
 * device memory of a context comes from the single workspace the caller hands
 * to qtt_ctx_create (sub-allocated by the library; the caller keeps it alive
 * until qtt_ctx_destroy). Host arrays are owned by the caller and only read or
 * written during the call. Calls are ordered on the context's CUDA stream;
 * every call that returns host values synchronises that stream first.
 *
 * Errors: 0 = OK; negative = error (no result): QTT_EINVAL bad argument,
 * QTT_ENOMEM workspace exhausted, QTT_ECUDA a CUDA error, QTT_ENAN a NaN/Inf
 * was produced, QTT_ETIMEOUT a device wait ran out. Positive = warning with the
 * result returned: QTT_WRANKCAP the rank cap dropped more than the tolerance
 * allows, QTT_WNOCONV the iteration limit was reached. qtt_last_error gives
 * the message of the last failing call on a context.
 *
 * Precision: QTT_FP64 keeps cores in complex128 and runs every step in FP64.
 * QTT_FP32 keeps cores in complex64 with FP32 contractions (SIMT, or split
 * TF32 on the tensor cores: qtt_ctx_set_contraction) and FP32 or FP64
 * factorisations (qtt_ctx_set_factorization); norms, inner products, the
 * Green operator assembly and the C_eff average stay FP64.
 *
 * Concurrency: the solvers run up to qtt_ctx_set_concurrency solves side by
 * side, each on its own CUDA stream; the GPU maps streams onto
 * CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 unless the environment sets
 * it before CUDA starts; 32 at most), and streams sharing a queue run one
 * after the other.
 */
#ifndef QTT_HOMOG_H
#define QTT_HOMOG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QTT_OK 0
#define QTT_EINVAL (-1)
#define QTT_ENOMEM (-2)
#define QTT_ECUDA (-3)
#define QTT_ENAN (-4)
#define QTT_ETIMEOUT (-5)
#define QTT_WRANKCAP 1
#define QTT_WNOCONV 2

#define QTT_FP64 0
#define QTT_FP32 1
#define QTT_CONTRACT_SIMT 0
#define QTT_CONTRACT_TF32X3 1
#define QTT_CONTRACT_TC 2
#define QTT_SCHEME_DIRECT 0    /* App. A table of divergence operators, in its order */
#define QTT_SCHEME_CENTERED 1
#define QTT_SCHEME_FORWARD 2
#define QTT_SCHEME_BACKWARD 3
#define QTT_SCHEME_HEX8R 4
#define QTT_SCHEME_STAGGERED 5
#define QTT_FACTOR_NATIVE 0
#define QTT_FACTOR_FP64 1
#define QTT_FACTOR_FP64_ROUNDING 2

#define QTT_MAX_CORES 64

typedef struct qtt_ctx* qtt_ctx_t;
typedef struct qtt_tt* qtt_tt_t;
typedef struct qtt_op* qtt_op_t;

/* ---------------------------------------------------------------- context */

/* Handles belong to the context that made them: free them before
 * qtt_ctx_destroy; after it they must not be used or freed. */
/* Create a context on CUDA device `device`, ordering all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * `workspace` is a device buffer of `workspace_bytes` bytes (256-byte
 * aligned) from which every device allocation of the context is carved.
 * `seed` keys the counter-based generator of the random sketches.
 * Returns QTT_EINVAL on a bad precision, device or workspace. */
int qtt_ctx_create(qtt_ctx_t* out, int device, void* cuda_stream, int precision,
                   void* workspace, size_t workspace_bytes, uint64_t seed);
void qtt_ctx_destroy(qtt_ctx_t ctx);
const char* qtt_last_error(qtt_ctx_t ctx);
/* Bytes of the workspace currently allocated, and the high-water mark. */
size_t qtt_ctx_bytes_in_use(qtt_ctx_t ctx);
size_t qtt_ctx_bytes_peak(qtt_ctx_t ctx);
/* Number of kernels this context has launched since creation. */
uint64_t qtt_ctx_launches(qtt_ctx_t ctx);
/* Kernel-class timing: when on, CUDA events on the context stream bracket
 * every GEMM, QR and SVD launch. qtt_ctx_profile writes 9 doubles: for class
 * c in (0 gemm, 1 qr, 2 svd) out[3c] = launches, out[3c+1] = total ms,
 * out[3c+2] = algorithmic real flops (GEMM: 8 M N K per complex product;
 * QR: 8 (2 m n^2 - 2 n^3/3); SVD: one Jacobi sweep's count per launch);
 * out[9] = Jacobi sweeps run over all SVD launches, out[10] = GEMMs run on
 * the tcgen05 tensor-core kernel (11 doubles in all);
 * reset = 1 clears the counters. */
int qtt_ctx_set_profiling(qtt_ctx_t ctx, int on);
int qtt_ctx_profile(qtt_ctx_t ctx, int reset, double* out);

/* ---------------------------------------------------------------- TT handles */

/* Upload a TT: L cores, dims[L], ranks[L+1] (ranks[0] = ranks[L] = 1), host
 * cores as interleaved complex doubles, concatenated row-major. */
int qtt_tt_create(qtt_ctx_t ctx, int L, const int* dims, const int* ranks,
                  const double* cores, qtt_tt_t* out);
/* TT-SVD of a dense host tensor (Sec. 3; App. D): dims[L] (row-major,
 * interleaved complex doubles, prod(dims) entries), compressed on the device
 * with per-bond threshold eps ||T|| / sqrt(L - 1) and rank cap rmax. For
 * tests and small grids (the dense tensor is copied to the workspace). */
int qtt_tt_from_dense(qtt_ctx_t ctx, int L, const int* dims, const double* dense, double eps,
                      int rmax, qtt_tt_t* out);
/* Shape query: writes *L, dims[L], ranks[L+1] (arrays of QTT_MAX_CORES+1). */
int qtt_tt_shape(qtt_tt_t tt, int* L, int* dims, int* ranks);
/* Download the cores (interleaved complex doubles, concatenated). */
int qtt_tt_export(qtt_ctx_t ctx, qtt_tt_t tt, double* cores);
/* The full tensor a TT represents (eq. (tt_format): the entry at (i_1..i_L)
 * is the product of the core slices G_k[:, i_k, :]), contracted on the device
 * left to right and written to `dense` as prod(dims) interleaved complex
 * doubles in row-major order (caller-owned, 2 prod(dims) doubles). For tests
 * and small grids: returns QTT_EINVAL above 2^30 entries, QTT_ENOMEM when
 * the workspace cannot hold the partial products. */
int qtt_tt_to_dense(qtt_ctx_t ctx, qtt_tt_t tt, double* dense);
void qtt_tt_free(qtt_tt_t tt);

/* Upload an operator: L cores with d_out[L], d_in[L], ranks[L+1] and
 * diag[L] (1 = raised diagonal core stored (a, d, a'), requires d_out = d_in;
 * 0 = full core (a, d_out, d_in, a')). */
int qtt_op_create(qtt_ctx_t ctx, int L, const int* d_out, const int* d_in,
                  const int* ranks, const int* diag, const double* cores,
                  qtt_op_t* out);
int qtt_op_shape(qtt_op_t op, int* L, int* d_out, int* d_in, int* ranks, int* diag);
int qtt_op_export(qtt_ctx_t ctx, qtt_op_t op, double* cores);
void qtt_op_free(qtt_op_t op);

/* ---------------------------------------------------------------- operators */

/* (C(x) - C0) as a raised TTO (Sec. 4.3; preprocessing, App. D): the phase
 * field (host uint8, C order, shape[3] each 1 or 2^n; an extent of 1 is a
 * broadcast axis) is mapped to the Voigt-matrix field
 * sum_p (C_p - C0) [phase == p] with isotropic phases (E[p], nu[p]),
 * p < nphase, and compressed by TT-SVD at eps_tt with rank cap rmax. The
 * 36 Voigt rows of that field span at most nphase directions (columns of D =
 * [C_p - C0]); with D = U S V^H the TT-SVD runs on the k-row field S V^H
 * indexed by phase and U multiplies the first core, which gives the same
 * decomposition (U has orthonormal columns). lame0 = (lambda0, mu0) of the
 * reference medium, or NULL for the arithmetic mean of the smallest and
 * largest phase Lame parameters. The handle remembers C0. */
int qtt_from_phase_field(qtt_ctx_t ctx, const uint8_t* phase, const int shape[3], int n,
                         int nphase, const double* E, const double* nu,
                         const double* lame0, double eps_tt, int rmax, qtt_op_t* dC);

/* Raised TTO of the Voigt-matrix field sum_p mats[p] [phase == p]: the same
 * construction as qtt_from_phase_field with arbitrary per-phase 6x6 matrices
 * (mats: nphase row-major 6x6 blocks), e.g. dC/dp for a material parameter. */
int qtt_from_phase_matrices(qtt_ctx_t ctx, const uint8_t* phase, const int shape[3], int n,
                            int nphase, const double* mats, double eps_tt, int rmax,
                            qtt_op_t* out);

/* Applicability estimate (Sec. 5.2: compress the geometry at two
 * discretisation orders to see its rank and how the rank grows): builds the
 * stiffness operator (as qtt_from_phase_field, no rank cap, at eps_tt) of
 * phase_a on a 2^n grid and of phase_b, the same geometry sampled on a
 * 2^(n+1) grid (extents 1 or 2^n, resp. 2^(n+1)), and writes out[0] = its
 * largest TT rank at n, out[1] = at n + 1, out[2] = the growth factor
 * out[1] / out[0] per order, out[3] = out[0] * out[2]^(n_target - n), the
 * rank the geometry would need at 2^n_target if it kept growing that way
 * (about 1 for laminates, about 2 per order for spheres). The operators are
 * freed. */
int qtt_rank_estimate(qtt_ctx_t ctx, const uint8_t* phase_a, const int shape_a[3],
                      const uint8_t* phase_b, const int shape_b[3], int n, int nphase,
                      const double* E, const double* nu, double eps_tt, int n_target,
                      double* out);
/* The SFFT (Sec. 4.1-4.2): S = P_rev F+ per axis, F+[k, x] =
 * N^-1/2 exp(+2 pi i k x / N), P_rev reversing the n output bits, as a TTO
 * with an identity Voigt core; adjoint = 1 gives S^H = S^-1. Built on the
 * device by TT-SVD of the per-axis matrix at accuracy eps. */
int qtt_sfft_operator(qtt_ctx_t ctx, int n, int adjoint, double eps, qtt_op_t* out);
/* The SFFT MPO of one axis built the way Sec. 4.2 builds it, on the host (no
 * context, no GPU): the reduced QFT circuit of Sec. 4.1 (Hadamard and
 * controlled-phase gates, no SWAP network; each controlled phase split into
 * a copy and a phase tensor) applied gate by gate to the identity MPO by
 * zip-up sweeps, then one TT rounding at eps. It is the operator
 * S[k', x] = N^-1/2 exp(2 pi i rev(k') x / N) that qtt_sfft_operator builds
 * by TT-SVD, with the circuit's ranks. Output: ranks[0..n] (n + 1 ints) and
 * the cores (r_k, 2 out, 2 in, r_{k+1}) concatenated in core order, row-major,
 * interleaved complex doubles, into `cores` of capacity `cap` doubles;
 * *needed receives the number of doubles. Each partial product of the gates
 * is rounded at eps / 100, so the ranks stay near the final ones and the
 * cost is milliseconds (0.05 s at n = 12). Returns QTT_EINVAL for n outside
 * 1..24, eps <= 0, null ranks/needed, or cores null or too small (ranks and
 * *needed are filled in then, so a first call with cap = 0 sizes the
 * buffer); QTT_ENOMEM if host memory runs out. */
int qtt_sfft_mpo_zipup(int n, double eps, int* ranks, double* cores, size_t cap,
                       size_t* needed);

/* The Green operator Gamma_hat^0 (App. A, eq. (orig_green_eshelby),
 * isotropic C0 = (lambda0, mu0)) of a discretisation scheme in the SFFT
 * momentum convention (Sec. 4.3: bit-reversed per axis, conjugated), as a
 * raised TTO. scheme (App. A table of divergence operators k(q)):
 *   QTT_SCHEME_DIRECT (k = i q), QTT_SCHEME_CENTERED (k = i sin q) and
 *   QTT_SCHEME_HEX8R (k_j = (i/4) tan(q_j/2) prod_l (1 + e^{i q_l}), the
 *   table's sum over l read as this product) have k = common factor x real
 *   vector v (v = xi, sin q, and sin(q_j/2) prod_{l!=j} cos(q_l/2)), and
 *   Gamma is the Direct closed form at v. It is built from its separable
 *   form: Gamma_V is a 36 x 15 matrix of (lambda0, mu0) times the 15
 *   degree-4 monomials of v/|v|; the monomial fields are compressed by TT-SVD
 *   at eps_tt and rank cap rmax once per (n, eps_tt, rmax, scheme) and
 *   context, and the matrix multiplies their first core (relative error at
 *   most cond(matrix) eps_tt, cond ~7). n in 1..9.
 *   QTT_SCHEME_FORWARD (k+ = e^{iq} - 1), QTT_SCHEME_BACKWARD
 *   (k- = 1 - e^{-iq}) and QTT_SCHEME_STAGGERED (normal strains with k+,
 *   shear strains with k-) are complex: Gamma_V = B (B^H C0 B)^-1 B^H with
 *   B the 6 x 3 strain symbol is evaluated at every frequency and the
 *   36-entry field compressed by TT-SVD at (eps_tt, rmax). n in 1..8; the
 *   field takes 36 x 2^(3n) x 16 bytes of workspace while it is built.
 * At Nyquist modes App. A's symmetrisation applies (it changes only the Direct
 * scheme). Errors: QTT_EINVAL for a scheme outside 0..5, n out of range or
 * a reference medium that is not positive definite; QTT_ENOMEM when the
 * workspace cannot hold the field. */
int qtt_gamma_operator(qtt_ctx_t ctx, int n, double lambda0, double mu0, int scheme,
                       double eps_tt, int rmax, qtt_op_t* out);

/* ---------------------------------------------------------------- TT algebra */

/* y = round(A x): compressed product by randomized sketching with sketch rank
 * rmax + oversample (sketch entries from the context's Philox-4x32-10 stream
 * number apply_id; each right-to-left sketch environment is replaced by an
 * orthonormal basis of its range, from a pivoted Cholesky factor of its Gram
 * matrix, before the next one is formed), then TT rounding at (eps_tt, rmax)
 * (Sec. 3, Table 2). The result is right-orthogonal. */
int qtt_op_apply(qtt_ctx_t ctx, qtt_op_t op, qtt_tt_t in, double eps_tt, int rmax,
                 int oversample, int apply_id, qtt_tt_t* out);
/* SFFT, inverse SFFT and Green products with the context's cached operators
 * (built on first use for the TT's n; Sec. 4.3, Alg. 2's transform and Green steps, App. D
 * lookup table). n[3] must be equal (cubic grids). gamma0_apply's scheme is
 * one of QTT_SCHEME_* (0..5), as for qtt_gamma_operator. */
int sfft_apply(qtt_ctx_t ctx, qtt_tt_t in, double eps_tt, int rmax, qtt_tt_t* out);
int isfft_apply(qtt_ctx_t ctx, qtt_tt_t in, double eps_tt, int rmax, qtt_tt_t* out);
int gamma0_apply(qtt_ctx_t ctx, const int n[3], double lambda0, double mu0, int scheme,
                 qtt_tt_t in, double eps_tt, int rmax, qtt_tt_t* out);
/* TT rounding in place (Sec. 3, eq. (rounding_condition_tt)): QR sweep left
 * to right, then truncated SVDs right to left with per-bond threshold
 * eps_tt ||x|| / sqrt(L - 1) and rank cap rmax. Returns QTT_WRANKCAP when the
 * cap dropped more than the threshold allows. */
int tt_round(qtt_ctx_t ctx, qtt_tt_t inout, double eps_tt, int rmax);
/* <a, b> = sum conj(a) b (Sec. 3, Table 2: the TT inner product as a
 * left-to-right sweep of transfer matrices, O(L d r^3); the stop test of
 * Alg. 2 is formed from three of them). Transfer matrices in FP64 in both
 * precisions; *re, *im are written after the context stream is synchronised. */
int qtt_tt_dot(qtt_ctx_t ctx, qtt_tt_t a, qtt_tt_t b, double* re, double* im);
/* <a, b> for callers that cannot allocate memory during the call -- code
 * that runs while an external framework owns all device memory, a hot loop
 * that must not block in the allocator, or a process that has handed its
 * memory budget out already. No counterpart in the paper: it is the same
 * inner product as qtt_tt_dot (FP64 transfer matrices, same kernels) with
 * every temporary in a fixed device array compiled into the library, so the
 * call neither allocates device or host memory nor uses the context's
 * workspace. Limits: TT ranks <= QTT_NOALLOC_MAX_RANK (64) and mode sizes <=
 * QTT_NOALLOC_MAX_DIM (6); larger inputs return QTT_EINVAL with a message in
 * qtt_last_error of the TTs' context. The array (1.25 MiB) stays resident on
 * every device that loads the library until the process exits. The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it; make that first call before any stream capture. All calls
 * share the one array: calls whose work overlaps on the GPU (other streams or
 * host threads) race and must be serialised by the caller. Work is ordered on
 * `cuda_stream`; NULL means the stream of the TTs' context, which is already
 * ordered after the library work that wrote a and b (another stream must be
 * ordered after that work by the caller). The call synchronises the stream
 * before writing *re, *im, runs on the context's device and leaves the
 * caller's current device as it found it. */
#define QTT_NOALLOC_MAX_RANK 64
#define QTT_NOALLOC_MAX_DIM 6
int qtt_tt_dot_noalloc(qtt_tt_t a, qtt_tt_t b, void* cuda_stream, double* re, double* im);
/* Bilinear grid mean of y^T A x = mean_x sum_{I,J} y_I(x) A[I,J](x) x_J(x)
 * (no conjugation), by an FP64 transfer sweep; A's first core full, binary
 * cores raised. */
int qtt_op_sandwich_mean(qtt_ctx_t ctx, qtt_op_t op, qtt_tt_t y, qtt_tt_t x, double* re,
                         double* im);
/* Grid mean of A x without forming A x (Sec. 2, the C_eff paragraph: the
 * volume average <(C - C0) eps> of the polarisation, which with C0 E gives
 * sigma_bar): every binary core is contracted with the averaging vector
 * (1/2, 1/2) in an FP64 sweep; writes 2 * d_out[0] doubles (interleaved
 * complex, one per component of the first core). */
int qtt_op_mean_apply(qtt_ctx_t ctx, qtt_op_t op, qtt_tt_t x, double* out);

/* ---------------------------------------------------------------- solver */

typedef struct {
  double tol;      /* stop when ||eps_{m+1} - eps_m||_F / ||E||_F < tol; the
                      residual comes from FP64 inner products and is never
                      reported below their cancellation floor
                      sqrt(64 eps (||eps_{m+1}||^2 + ||eps_m||^2)) / ||E||_F
                      (about 2e-7 relative to ||eps||), so a smaller tol runs
                      to max_iter */
  int max_iter;    /* iteration cap (QTT_WNOCONV when reached) */
  double eps_tt;   /* rounding accuracy of every step */
  int rmax;        /* rank cap of every rounding */
  int scheme;      /* Green operator discretisation, QTT_SCHEME_* (0..5) */
  int oversample;  /* sketch rank = rmax + oversample */
} qtt_solve_params;

typedef struct {
  int iters;         /* iterations run */
  double residual;   /* last ||eps_{m+1} - eps_m||_F / ||E||_F */
  int max_rank;      /* largest TT rank met */
  int rank_cap_hit;  /* 1 if some rounding hit the cap */
  double imag_leak;  /* max |Im sigma_bar| */
  double ms;         /* wall time of the solve */
} qtt_solve_info;

/* Alg. 2 for one macro strain E_voigt with explicit operators (dC raised, S,
 * S^H, Gamma raised) and reference stiffness C0 (6x6 row-major): writes
 * sigma_bar = C0 E + mean(dC eps_final) as 6 interleaved complex values. */
int ls_solve_ops(qtt_ctx_t ctx, qtt_op_t dC, qtt_op_t S, qtt_op_t Sh, qtt_op_t gamma,
                 const double C0[36], const double E_voigt[6], const qtt_solve_params* p,
                 double sigma_bar[12], qtt_solve_info* info);
/* Alg. 2 with the context's cached S, S^H and Gamma for dC's grid and C0. */
int ls_solve(qtt_ctx_t ctx, qtt_op_t dC, const double E_voigt[6],
             const qtt_solve_params* p, double sigma_bar[12], qtt_solve_info* info);
/* C_eff column by column (Sec. 2): column k = Re sigma_bar for E = e_k, for
 * the load cases listed in loads[nloads] (NULL = all six). Ceff is 36 doubles,
 * column-major (Ceff[k*6 + i] = C_eff[i][k]); info has nloads entries. Up to
 * qtt_ctx_set_concurrency load cases run side by side, each on its own CUDA
 * stream and host thread with a private slice of the workspace (the
 * operators are shared); the call returns when all are done. */
int ls_solve_ceff(qtt_ctx_t ctx, qtt_op_t dC, const qtt_solve_params* p, const int* loads,
                  int nloads, double* Ceff, qtt_solve_info* info);
/* Jacobi SVD stopping rule: a column pair counts as orthogonal when
 * |a_p^H a_q| <= tol_scale sqrt(m) eps |a_p| |a_q| (eps of the working
 * precision; default tol_scale 1); max_sweeps_fp32 caps the sweeps in FP32
 * mode (default 40; FP64 mode uses 60). */
int qtt_ctx_set_jacobi(qtt_ctx_t ctx, double tol_scale, int max_sweeps_fp32);
/* TT-SVD of a dense field (Alg. 1, used to build the stiffness and Green
 * operators): a P x c unfolding with 8 P c min(P, c) above gram_threshold
 * (default 2e9) takes its right factor from the eigenvectors of the Gram
 * matrix M^H M, with the ranks decided by the column norms of M V; smaller
 * ones take an SVD of M itself (QR + one-sided Jacobi). 0 sends every
 * unfolding through the Gram path. Returns QTT_EINVAL for a negative value. */
int qtt_ctx_set_tt_svd(qtt_ctx_t ctx, double gram_threshold);
/* Contraction precision of an FP32 context (the split-precision pattern of
 * the method's mixed mode; the paper itself states no precision):
 * QTT_CONTRACT_SIMT (default) runs every core contraction as FP32 SIMT
 * GEMMs; QTT_CONTRACT_TF32X3 runs them on the tensor cores with TF32 inputs
 * split as x = hi + lo and products hi*hi + hi*lo + lo*hi accumulated in FP32
 * (FP32-level accuracy); QTT_CONTRACT_TC runs the two large unbatched
 * contractions of each core of a product (the sketched carry T Psi and the
 * next carry Q^H T) when M >= 64, N >= 32, K >= 64 on the 5th-generation
 * tensor cores
 * (tcgen05.mma kind::tf32, TMA-staged operands, TMEM accumulators; the same
 * hi/lo split with the hi*hi products and the corrections in separate
 * accumulators) and the other contractions as FP32 SIMT GEMMs. Factorisations, norms and the C_eff average are unaffected. Returns
 * QTT_EINVAL for an unknown mode or a tensor-core mode on an FP64 context. */
int qtt_ctx_set_contraction(qtt_ctx_t ctx, int mode);
/* Throughput and accuracy of one contraction kernel (measurement of the
 * contraction that every product of Alg. 2 is built from; the paper has no
 * counterpart): C = A B for a random complex M x K by K x N product (Philox
 * entries in the context's FP32 precision, row-major), run once to warm up
 * and `reps` times between CUDA events on the context stream with
 * contraction mode `mode` (QTT_CONTRACT_SIMT, _TF32X3 or _TC; the TC kernel
 * takes the product when M >= 64, N >= 32, K >= 64, else SIMT). Writes the
 * average ms per launch (the TC path includes its two operand-split
 * kernels) and the Frobenius relative error against an FP64 GEMM of the same
 * operands. Uses the workspace; any context precision. */
int qtt_contraction_bench(qtt_ctx_t ctx, int mode, int M, int N, int K, int reps,
                          double* ms_per_launch, double* rel_err);
/* FP64 SVDs whose matrix does not fit one CTA's shared memory: precond = 1
 * (default) takes the FP32-preconditioned path (FP32 one-sided Jacobi for the
 * right singular vectors, one FP64 Newton-Schulz step, then FP64 Jacobi
 * sweeps on A V until a sweep rotates nothing, at most refine_sweeps,
 * default 6); precond = 0 runs the FP64 Jacobi from the start. The FP32
 * preconditioner leaves the columns near the FP32 noise floor unresolved,
 * and the truncation threshold of eps_tt = 1e-6 lies there, so the FP64
 * sweeps must be allowed to converge (with a cap of 2 the e11 solves of the
 * laminate-with-fibres workload stagnated at a residual of 3e-3). Returns
 * QTT_EINVAL for refine_sweeps outside 1..60. */
int qtt_ctx_set_svd(qtt_ctx_t ctx, int precond, int refine_sweeps);
/* Green operator of solves whose stiffness operator is broadcast along x1
 * (a phase field of shape (1, N, N)), Sec. 4.3 on broadcast axes. Such a
 * strain is x1-invariant, so after the SFFT its x1 bits hold only xi_1 = 0;
 * with on = 1 the solves (ls_solve, ls_solve_ceff, ls_solve_batched,
 * ls_solve_jobs and the gradient) use Gamma(0, xi_2, xi_3) (x) I on the x1
 * cores, built from the 2^(2n)-point plane field instead of the 2^(3n)-point
 * one. On these fields it acts as the full operator does, its ranks through
 * the x1 cores are those of its first bond, and it allows n up to 13 (the
 * full build stops at 9, or 8 for the complex schemes). Operators with
 * another broadcast pattern keep the full Green operator. Default 0.
 * Returns QTT_EINVAL for a null context. */
int qtt_ctx_set_green_broadcast(qtt_ctx_t ctx, int on);
/* Factorisation precision of an FP32 context (the mixed mode of the
 * method's precision pattern: bulk contractions in FP32, the QR and SVD
 * steps of TT rounding in FP64; Sec. 3 rounding, whose per-bond threshold
 * eps_tt ||x|| / sqrt(L - 1) is 2e-7 ||x|| at eps_tt 1e-6 on 25 cores, at
 * the FP32 rounding level): QTT_FACTOR_NATIVE (default) factorises in the
 * context's precision; QTT_FACTOR_FP64 widens every QR, SVD and sketch
 * Cholesky operand of an FP32 context to FP64, factorises it with the FP64
 * kernels and rounds the factors back (cores stay complex64);
 * QTT_FACTOR_FP64_ROUNDING does so only for the QR and SVD steps of TT
 * rounding (the sketch Cholesky and the compression QR inside a product stay
 * FP32). An FP64 SVD whose matrix does not fit one CTA's shared memory takes
 * an FP32 Jacobi preconditioner (right singular vectors made orthonormal in
 * FP64 by a Newton-Schulz step) and finishes with a few FP64 Jacobi sweeps
 * on the rotated matrix, in FP64 contexts as well. No effect on an FP64
 * context. Returns QTT_EINVAL for an unknown mode. */
int qtt_ctx_set_factorization(qtt_ctx_t ctx, int mode);
/* C_eff and its derivatives with respect to phase parameters (E or nu of a
 * phase). The LS operator of every scheme (with the Nyquist symmetrisation of
 * App. A for the Direct one) is self-adjoint, so the adjoint solution of load l equals its
 * forward strain and dC_eff[l][k]/dp = mean(eps_l^T (dC/dp) eps_k): the six
 * forward solves are kept and contracted with the raised TTO of dC/dp
 * (qtt_from_phase_matrices of the derivative of the phase stiffness). phase,
 * shape, nphase, E, nu: the inputs dC was built from. param_phase[q],
 * param_kind[q] (0 = E, 1 = nu) for q < nparams. Ceff as in ls_solve_ceff;
 * dCeff: nparams blocks of 36 doubles, same column-major layout; info: 6. */
int ls_solve_ceff_grad(qtt_ctx_t ctx, qtt_op_t dC, const uint8_t* phase, const int shape[3],
                       int nphase, const double* E, const double* nu, int nparams,
                       const int* param_phase, const int* param_kind, const qtt_solve_params* p,
                       double* Ceff, double* dCeff, qtt_solve_info* info);
/* Number of unit-load solves run side by side (1..64, default 1): each on
 * its own CUDA stream and host thread with a private slice of the workspace.
 * ls_solve_ceff uses at most 6 (its loads), ls_solve_batched all of them. */
int qtt_ctx_set_concurrency(qtt_ctx_t ctx, int concurrent_loads);
/* C_eff of many microstructures in one call (Sec. 2 per item; the batched
 * generation of elastic training data the paper motivates). dC[i]: stiffness
 * operator of item i from qtt_from_phase_field; grid sizes n and reference
 * media may differ between items (S, S^H and Gamma are built once per grid
 * and medium and cached). All nitems x 6 unit-load solves go through one
 * queue, largest grids first, served by qtt_ctx_set_concurrency lanes; each
 * solve is exactly the one ls_solve_ceff runs for that item and load (same
 * sketches, same result). Ceff: nitems x 36 doubles, item i at Ceff + 36 i,
 * column-major as in ls_solve_ceff. info: nitems x 6 entries (item i, load k
 * at info[6 i + k]) or NULL. Returns the worst status over all solves; on an
 * error nothing is written. */
int ls_solve_batched(qtt_ctx_t ctx, int nitems, const qtt_op_t* dC, const qtt_solve_params* p,
                     double* Ceff, qtt_solve_info* info);
/* A list of unit-load LS solves (Alg. 2 with E = e_load[j] on dC[j]; Sec. 2
 * C_eff paragraph for sigma_bar) through the same queue and lanes as
 * ls_solve_batched: job j solves load[j] (0..5) on the stiffness operator
 * dC[j] (from qtt_from_phase_field; jobs may share an operator) and writes
 * sigma_bar = C0 e_load + mean(dC eps_final) as 6 interleaved complex values
 * at sigma_bar + 12 j (column load[j] of that microstructure's C_eff is its
 * real part); info: njobs entries or NULL. Each job is exactly the solve
 * ls_solve_ceff runs for that operator and load. Returns the worst status;
 * on an error nothing is written. */
int ls_solve_jobs(qtt_ctx_t ctx, int njobs, const qtt_op_t* dC, const int* load,
                  const qtt_solve_params* p, double* sigma_bar, qtt_solve_info* info);

#ifdef __cplusplus
}
#endif

#endif /* QTT_HOMOG_H */
