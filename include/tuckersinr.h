/*
 * tuckersinr.h -- C ABI of the GB300 (sm_103a) library for SINR evaluation
 * from the groupwise Tucker form of MIMO channel submatrices
 * (Zhang, Zhu, Zhang: "Compressing MIMO Channel Submatrices with Tucker
 * Decomposition", arXiv 2401.09792).
 *
 * System (Section 2.2): J cells, one BS and one UE per cell (the paper's
 * experiments keep one interfering UE per cell, Section 4).  Link (i, k) is
 * the channel from BS k to the UE of cell i; it is stored as ch = i * J + k.
 * Every BS sends L streams to its own UE and interferes with all other UEs.
 *
 * Groupwise Tucker form (eq. 14): X_ik ~ G_ik x_1 A_i x_2 B_k x_3 C_ik with
 * orthonormal A_i (M x m), B_k (N x n), C_ik (P x p) and core G_ik
 * (m x n x p).  For subcarrier kappa with path coefficients c_ik(kappa) in
 * C^P the compressed channel is (eq. 15)
 *     H~_ik(kappa) = G_ik x_3 (c_ik(kappa)* C_ik)   (m x n),
 * and the SINR is evaluated on H~ alone because A and B cancel (Section 3.3).
 *
 * Conventions
 *   - complex numbers are interleaved (re, im) float32 pairs (ts_c64);
 *   - every array is row-major and dense, with the layouts given per call;
 *   - every data pointer is DEVICE memory owned by the caller unless a call
 *     says otherwise; the library allocates nothing and frees nothing;
 *   - calls are asynchronous on the given CUDA stream (a cudaStream_t passed
 *     as void*; NULL = the legacy default stream) and never synchronise;
 *   - return value: TS_OK, or a TS_ERR_* code.  Argument errors are detected
 *     before any launch and leave the outputs untouched.  TS_ERR_CUDA reports
 *     a launch failure (the CUDA error is kept for ts_last_cuda_error()).
 *     Numerical trouble inside a kernel does not fail the call: it sets bits
 *     in the per-result flags array (when given) and the affected SINR values
 *     become NaN.
 *   - the gradient of a real loss l with respect to a complex parameter
 *     z = x + iy is reported as dl/dx + i dl/dy.
 */
#ifndef TUCKERSINR_H
#define TUCKERSINR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  float re, im;
} ts_c64;

/* Sizes of one multi-cell system (notation of the paper, Section 2.1). */
typedef struct {
  int32_t J;          /* cells = base stations = groups                        */
  int32_t M, N, P;    /* UE antennas, BS antennas, submatrices per link         */
  int32_t m, n, p;    /* Tucker ranks: 1 <= m <= M, n <= min(N, 1024),
                         p <= P <= 1024.  SVD-precoded SINR (FP32): m <= 64
                         (m > 16: shared-memory precoder and finalisation,
                         L <= 8), p <= 256 (p > 32 or P p > 8192 runs the
                         wide-core kernel, as the paper's compressed sizes
                         need), n > 512 only with L <= 8 (shared-memory
                         precoder); wideband precoder, adjoints and
                         tensor-core modes: m <= 16, n <= 512, p <= 32 and
                         P p <= 8192.  Dense comparator: M, N, P as m, n, p
                         of the matching compressed call, P <= 1024 (SVD)  */
  int32_t K;          /* OFDM subcarriers, kappa = 0 .. K-1                      */
  int32_t L;          /* streams per UE, 1 <= L <= min(m, n)                     */
  float delta_f_hz;   /* subcarrier spacing (path-form coefficients only)      */
} ts_dims;

/* Path coefficients c_ik(kappa) of eq. (2) / eq. (9). */
enum { TS_COEF_DENSE = 0, TS_COEF_PATHS = 1 };
typedef struct {
  int32_t mode;        /* TS_COEF_DENSE or TS_COEF_PATHS                         */
  const ts_c64* c;     /* DENSE: c[ch][kappa][P]                                 */
  const ts_c64* alpha; /* PATHS: alpha[ch][P]: c_p(kappa) = conj(alpha_p        */
  const float* tau_s;  /* PATHS: tau[ch][P] (s)   * exp(-j 2 pi kappa df tau_p)) */
} ts_coef;

/* Status codes. */
enum {
  TS_OK = 0,
  TS_ERR_DIMS = 1,      /* sizes out of range or inconsistent                 */
  TS_ERR_NULL = 2,      /* a required pointer is NULL                         */
  TS_ERR_ALIGN = 3,     /* a pointer is not 8-byte aligned                    */
  TS_ERR_WORKSPACE = 4, /* workspace too small (see ts_workspace_bytes)       */
  TS_ERR_CUDA = 5,      /* a CUDA launch failed                               */
  TS_ERR_MODE = 6       /* unknown coefficient mode or operation              */
};

/* Per-result flag bits (flags[i][kappa], uint8). */
enum {
  TS_FLAG_NOT_PD = 1,         /* a Cholesky pivot was not positive            */
  TS_FLAG_NONFINITE = 2,      /* a non-finite value reached the solve         */
  TS_FLAG_RANK_DEFICIENT = 4, /* a serving link had a zero singular value
                                 among the top L (SVD precoding)              */
  TS_FLAG_EIG_UNCONVERGED = 8, /* the Jacobi eigensolver hit its sweep cap    */
  TS_FLAG_TIMEOUT = 16,       /* a bounded device wait of the tensor-core pass
                                 gave up; the unit's SINR is NaN             */
  TS_FLAG_REFINED = 32,       /* informational: the SINR comes from the
                                 accurate re-evaluation (R in double-float,
                                 FP64-residual refinement of the solves):
                                 units above the refinement threshold, and
                                 every unit of more than 16 rows            */
  TS_FLAG_PRECODER_REFINED = 64 /* informational (SVD precoders): a serving
                                 link at this subcarrier had two adjacent
                                 squared singular values among its L + 1
                                 largest within 5e-3 of the largest, and its
                                 precoder was recomputed in FP64 (with the
                                 refinement threshold >= 0)                  */
};

/* Operations, for ts_workspace_bytes. */
enum {
  TS_OP_SINR_SVD = 0,
  TS_OP_SINR_MMSE = 1,
  TS_OP_DENSE_SVD = 2,
  TS_OP_DENSE_MMSE = 3,
  TS_OP_SINR_SVD_ADJOINT = 4,
  TS_OP_SINR_MMSE_ADJOINT = 5,
  TS_OP_TUCKER_FIT = 6,
  TS_OP_SINR_SVD_TF32 = 7,    /* ts_sinr_svd_prec with TS_PREC_TF32   */
  TS_OP_SINR_SVD_BF16X2 = 8,  /* ts_sinr_svd_prec with TS_PREC_BF16X2 */
  TS_OP_TUCKER_FIT_SHARED = 9,     /* ts_tucker_fit_model, TS_MODEL_SHARED     */
  TS_OP_TUCKER_FIT_INDIVIDUAL = 10, /* ts_tucker_fit_model, TS_MODEL_INDIVIDUAL */
  TS_OP_RECONSTRUCT = 11,          /* ts_tucker_reconstruct                    */
  TS_OP_SINR_SVD_MULTIUSER = 12,   /* ts_sinr_svd_multiuser (any U)            */
  TS_OP_DENSE_SVD_MULTIUSER = 13,  /* ts_dense_sinr_svd_multiuser (any U)      */
  TS_OP_SINR_SVD_TF32X3 = 14       /* ts_sinr_svd_prec with TS_PREC_TF32X3     */
};

/* The three compression models of Section 3.1: which links share the
 * receive (A) and transmit (B) factors.  Groupwise (eq. 14): A_i for the
 * links into UE i, B_k for the links out of BS k (J of each).  Shared
 * (eq. 12): one A and one B for every link.  Individual (eq. 10): A_ik and
 * B_ik per link (J^2 of each).  C_ik and G_ik are per link in all three. */
enum {
  TS_MODEL_GROUPWISE = 0,
  TS_MODEL_SHARED = 1,
  TS_MODEL_INDIVIDUAL = 2
};

/* Arithmetic of the interfering links' core contraction H~ = G x_3 (c* C)
 * (eq. 15) in ts_sinr_svd_prec.  FP32: FMA pipe, the default of every other
 * call.  TF32: tensor cores, w = c* C and G rounded to TF32 (10-bit
 * mantissa), FP32 accumulation.  BF16X2: tensor cores, w and G split into
 * BF16 high and low parts, products w_hi G_hi + w_hi G_lo + w_lo G_hi, FP32
 * accumulation (about 16 significant bits).  TF32X3: the same three
 * products with TF32 parts (about 22 significant bits, close to FP32).  The
 * projection, the serving links, the precoders, the effective channels,
 * the covariance and the solves stay FP32. */
enum {
  TS_PREC_FP32 = 0,
  TS_PREC_TF32 = 1,
  TS_PREC_BF16X2 = 2,
  TS_PREC_TF32X3 = 3
};

/* Human-readable name of a status code (static storage). */
const char* ts_status_string(int status);

/* The CUDA error (cudaError_t as int) behind the last TS_ERR_CUDA on this
 * host thread, or 0. */
int ts_last_cuda_error(void);

/* Version of this ABI (incremented on any incompatible change). */
int ts_abi_version(void);

/* Profiling hook: caller-created CUDA events (cudaEvent_t as void*) that the
 * following SINR calls on this host thread record on their stream right
 * before and right after their dominant kernel (the per-link rebuild and
 * covariance kernel).  NULL, NULL turns it off.  Not used otherwise. */
void ts_set_timing_events(void* start, void* stop);

/* Profiling hook: a caller-created CUDA event (cudaEvent_t as void*) that
 * the following SVD-precoded SINR calls on this host thread record on their
 * stream once the precoders are in the workspace (after the serving pass,
 * the precoder kernels and the close-pair refinement, before the
 * interfering-link pass): the boundary between the precoder phase and the
 * link phase of one call.  NULL turns it off.  Not used otherwise. */
void ts_set_phase_event(void* event);

/* Mixed-precision re-evaluation of sensitive units (eq. 25-28).  The
 * interference-plus-noise covariance R = sum_{k != i} E_ik E_ik* +
 * sigma^2 I is formed and factored in FP32; a unit whose SINRs are
 * sensitive to that rounding,
 *   s = max_r sqrt(sum_ab |y_ar|^2 |R_ab|^2 |y_br|^2) / (e_r* y_r) > threshold
 * (e_r the serving effective channel's columns, y_r = R^{-1} e_r; the FP32
 * rounding of R moves SINR_r by a few u s, u = 2^-24), is evaluated again by
 * SINR calls on this host thread from R formed in double-float out of the
 * stored effective channels, with the solves refined by FP64 residuals
 * (three steps of R^{-1} E_ii, then the L x L system in FP64); its flags get
 * TS_FLAG_REFINED.  Default threshold 8; 0 re-evaluates every unit, a
 * negative threshold none.  Units of more than 16 rows are always evaluated
 * the accurate way. */
void ts_set_refinement(float threshold);

/* Inner iterations of the fit's eigensolves for factors whose mode dimension
 * exceeds 72 (block subspace iteration with Cholesky-QR, then a
 * Rayleigh-Ritz step): `iterations` per update warm-started from the current
 * factor, three times as many for the initialisation.  Default 40; fewer
 * trade accuracy of each block update of Algorithm 2 for time (the outer
 * sweeps keep refining the factors).  Applies to the fit calls that follow
 * on this host thread; iterations <= 0 restores the default. */
void ts_set_fit_iterations(int iterations);

/* Self-test of the bounded mbarrier wait that the tensor-core kernel uses
 * for its operand copies and MMA completions: one thread waits on an
 * mbarrier phase that nothing completes (arrive = 0) or that it completes
 * first (arrive != 0), for at most `limit` tries (1 .. 2^24), and writes
 * *out (device int) = 1 if the wait gave up, 0 if the phase completed.
 * The context stays usable after a give-up; the SINR kernels turn one into
 * TS_FLAG_TIMEOUT and NaN for the units concerned. */
int ts_selftest_bounded_wait(long long limit, int arrive, int* out, void* stream);

/* Measured throughput of the current device in TFLOP/s: FP32 FMA (chains of
 * independent fmaf on every SM), TF32 tensor-core MMA (tcgen05, M = 128,
 * N = 256, K = 8, FP32 accumulation in TMEM, one CTA per SM) and FP64 FMA.
 * A diagnostics call (the paper has no counterpart): it allocates and frees
 * a small scratch buffer and synchronises on `stream`; it runs a few
 * milliseconds of work.  TS_ERR_CUDA if a tensor-core wait timed out. */
int ts_device_peaks(double* fp32_tflops, double* tf32_tflops, double* fp64_tflops, void* stream);

/* Device workspace, in bytes, that operation `op` needs for sizes `d`.
 * Returns 0 for invalid sizes.  The caller allocates it (256-byte aligned)
 * and passes it to the call; its contents need no initialisation. */
size_t ts_workspace_bytes(const ts_dims* d, int op);

/* a0 -- path coefficients on the subcarrier grid (eq. 2, eq. 9):
 *   c[ch][kappa][p] = conj(alpha[ch][p]) * exp(+j 2 pi kappa df tau[ch][p]).
 * The phase kappa * df * tau is reduced modulo one turn in 64-bit fixed point
 * before the float32 sine/cosine, so its error does not grow with kappa.
 * alpha: [J*J][P]; tau_s: [J*J][P]; c (out): [J*J][K][P]. */
int ts_coefficients(const ts_dims* d, const ts_c64* alpha, const float* tau_s,
                    ts_c64* c, void* stream);

/* Wideband precoder carried into the compressed domain (Section 3.3, with the
 * matrix form A G B^T of the mode products of Section 2.3):
 *   Pt[k] = B_k^T P_k   (n x L).
 * B: [J][N][n]; Pfull: [J][N][L]; Pt (out): [J][n][L]. */
int ts_project_precoder(const ts_dims* d, const ts_c64* B, const ts_c64* Pfull,
                        ts_c64* Pt, void* stream);

/* MMSE SINR with caller-given wideband precoders (eq. 3-6 evaluated on the
 * compressed form, eq. 15 and eq. 24-28):
 *   E_ik(kappa) = H~_ik(kappa) Pt_k,  Q~_i = sum_k E_ik E_ik* + sigma2_i I_m,
 *   SINR_i,r(kappa) = s~_r / (w~_r* Q~_i w~_r - s~_r),  W~ = Q~_i^{-1} E_ii.
 * G: [J*J][p][m][n] (core, mode-3 slabs G_ik[:, :, q], n fastest);
 * C: [J*J][P][p]; coef: see ts_coef; Pt: [J][n][L] (ts_project_precoder);
 * sigma2: [J] noise power per UE; sinr (out): [J][K][L] float;
 * flags (out, may be NULL): [J][K] uint8 TS_FLAG_* bits;
 * ws: workspace of ts_workspace_bytes(d, TS_OP_SINR_MMSE) bytes. */
int ts_sinr_mmse(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                 const ts_c64* C, const ts_c64* Pt, const float* sigma2,
                 float* sinr, uint8_t* flags, void* ws, size_t ws_bytes,
                 void* stream);

/* SVD-precoded SINR (eq. 7 and eq. 23-28): every BS k precodes with the top-L
 * right singular vectors V~_k(kappa) of its compressed serving channel
 * H~_kk(kappa), found from a Jacobi eigensolve of H~_kk H~_kk* (m x m); then
 * the same MMSE SINR as ts_sinr_mmse with E_ik = H~_ik V~_k.  Streams are
 * ordered by decreasing singular value.  Arguments as ts_sinr_mmse; ws holds
 * ts_workspace_bytes(d, TS_OP_SINR_SVD) bytes. */
int ts_sinr_svd(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                const ts_c64* C, const float* sigma2, float* sinr,
                uint8_t* flags, void* ws, size_t ws_bytes, void* stream);

/* The two phases of ts_sinr_svd, for callers that time or reuse them.
 * ts_svd_precoders writes the precoders V~_k(kappa) (eq. 7, eq. 23; and, for
 * path-form coefficients, the per-path phase steps) into ws.
 * ts_sinr_svd_from_precoders then evaluates eq. (24)-(28) from them.  Both
 * calls must receive the same d, coef, G, C and ws, in this order on one
 * stream; ts_sinr_svd issues exactly these two calls. */
int ts_svd_precoders(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                     const ts_c64* C, void* ws, size_t ws_bytes, void* stream);
int ts_sinr_svd_from_precoders(const ts_dims* d, const ts_coef* coef,
                               const ts_c64* G, const ts_c64* C,
                               const float* sigma2, float* sinr,
                               uint8_t* flags, void* ws, size_t ws_bytes,
                               void* stream);

/* ts_sinr_svd with the interfering links' core contraction (eq. 15) in the
 * arithmetic `precision` (TS_PREC_*; TS_PREC_FP32 is ts_sinr_svd).  The
 * precoders stay FP32; the serving links' channels H~_kk that they are
 * computed from are FP32 too, except that TS_PREC_TF32X3 forms them with
 * the same three-product tensor-core contraction when the precoder does not
 * contract the serving core itself (m n p > 8192).  Tensor-core modes need
 * even L <= 8, p <= 32 and m <= 16 (else TS_ERR_MODE); ws holds
 * ts_workspace_bytes(d, TS_OP_SINR_SVD_TF32 / _BF16X2 / _TF32X3) bytes (the
 * ts_sinr_svd workspace, then the core rewritten as a tensor-core operand,
 * the projections and the tiled precoder rows).
 * ts_sinr_svd_from_precoders_prec is its second phase after ts_svd_precoders
 * on the same ws (the serving channels of that sequence are FP32 in every
 * mode). */
int ts_sinr_svd_prec(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                     const ts_c64* C, const float* sigma2, int precision,
                     float* sinr, uint8_t* flags, void* ws, size_t ws_bytes,
                     void* stream);
int ts_sinr_svd_from_precoders_prec(const ts_dims* d, const ts_coef* coef,
                                    const ts_c64* G, const ts_c64* C,
                                    const float* sigma2, int precision,
                                    float* sinr, uint8_t* flags, void* ws,
                                    size_t ws_bytes, void* stream);

/* Subcarrier ranges (the partition of one system across devices): the SINR
 * of subcarriers kappa0 .. kappa0 + count - 1 of the system d (eq. 2, 9:
 * every subcarrier is an independent unit, the precoders of eq. 7 are per
 * subcarrier too), with G, C and the coefficients of the whole system
 * (dense coefficients: c[ch][d->K][P]).  Results and per-result flags of
 * the range only: sinr [J][count][L], flags [J][count]; they equal the same
 * subcarriers of a whole-system call bit for bit (the same arithmetic per
 * unit).  ws: ts_workspace_bytes of d with K = count, for the op of the
 * call (TS_OP_SINR_SVD / _TF32 / _BF16X2 / _TF32X3 by precision, or
 * TS_OP_SINR_MMSE).  TS_ERR_DIMS unless 0 <= kappa0 and
 * kappa0 + count <= d->K. */
int ts_sinr_svd_range(const ts_dims* d, int kappa0, int count, const ts_coef* coef,
                      const ts_c64* G, const ts_c64* C, const float* sigma2,
                      int precision, float* sinr, uint8_t* flags, void* ws,
                      size_t ws_bytes, void* stream);
int ts_sinr_mmse_range(const ts_dims* d, int kappa0, int count, const ts_coef* coef,
                       const ts_c64* G, const ts_c64* C, const ts_c64* Pt,
                       const float* sigma2, float* sinr, uint8_t* flags, void* ws,
                       size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- batches
 * Many independent systems with their own sizes (numbers of cells, antennas,
 * ranks, streams, subcarriers), evaluated by one graph launch.  The paper has
 * no counterpart; it serves callers that evaluate many small systems per
 * scheduling step, where one launch per kernel per system would dominate.
 *
 * ts_instance describes one system: its sizes, the operation
 * (TS_OP_SINR_SVD or TS_OP_SINR_MMSE), the arithmetic of the SVD path's core
 * contraction (TS_PREC_*; TS_PREC_FP32 for MMSE), and the device arrays of
 * ts_sinr_svd / ts_sinr_mmse (Pt: MMSE only, else NULL; flags may be NULL).
 */
typedef struct {
  ts_dims d;
  int op;
  int precision;
  ts_coef coef;
  const ts_c64* G;
  const ts_c64* C;
  const ts_c64* Pt;
  const float* sigma2;
  float* sinr;
  uint8_t* flags;
} ts_instance;

typedef struct ts_batch_plan ts_batch_plan;   /* opaque */

/* Device workspace for the whole batch: four slots, 256-byte aligned, back
 * to back; slot b is as large as the largest ts_workspace_bytes of the
 * instances j with j % 4 == b, which run one after the other on graph
 * branch b and share it.  0 if an instance is invalid. */
size_t ts_batch_workspace_bytes(const ts_instance* inst, int n);

/* Options of ts_batch_plan_create. */
enum {
  TS_BATCH_AUTOTUNE = 1   /* time the launch-shape candidates of every new
                             shape class on its instance and keep the
                             fastest (in the process-wide tuning table) */
};

/* Builds a plan for the n instances of `inst` (host array, copied): checks
 * every instance (sizes, pointers, workspace) before any launch, optionally
 * autotunes, then captures the instances' kernels into one CUDA graph --
 * independent instances on four parallel branches -- and instantiates it.
 * The device arrays must stay valid and in place for the plan's lifetime;
 * their contents may change between launches.  Allocates host memory and
 * CUDA streams, events and a graph (released by ts_batch_plan_destroy); no
 * device memory of its own.  Autotuning runs the instances' kernels on
 * their own data (outputs are overwritten by the next launch). */
int ts_batch_plan_create(const ts_instance* inst, int n, void* ws, size_t ws_bytes, int options,
                         ts_batch_plan** plan);
/* One evaluation of every instance of the plan: one graph launch on
 * `stream`.  Returns TS_ERR_CUDA if the launch fails. */
int ts_batch_launch(ts_batch_plan* plan, void* stream);
void ts_batch_plan_destroy(ts_batch_plan* plan);

/* The process-wide tuning table (shape class -> launch-shape choice) as a
 * text file, one class per line; load merges into the table. */
int ts_autotune_save(const char* path);
int ts_autotune_load(const char* path);

/* SVD-precoded SINR with U UEs per cell, as in the paper's experiments
 * (Section 4): UE u of cell i is served by BS i with the top-L right singular
 * vectors of its own link; only the first UE of every other cell causes
 * inter-cell interference (BS k transmits with its first UE's precoder) and
 * there is no intra-cell interference.  Every array holds U UE groups of the
 * single-UE layout, group u = UE u of every cell: G [U][J*J][p][m][n],
 * C [U][J*J][P][p], coef [U][J*J][K][P] (dense) or alpha, tau [U][J*J][P]
 * (paths), sigma2 [U][J], sinr (out) [U][J][K][L], flags (out, may be NULL)
 * [U][J][K].  U = 1 is ts_sinr_svd.  FP32, sizes as ts_sinr_svd (wide cores
 * included).  ws: at least ts_workspace_bytes(d, TS_OP_SINR_SVD_MULTIUSER)
 * bytes = two single-UE workspaces (the first UEs' precoders stay in the
 * first while the other groups, one after the other, reuse the second).
 * With U single-UE workspaces (U / 2 times that size) the groups after the
 * first run concurrently on up to four library-owned side streams, created
 * on the first such call on a device and kept; `stream` waits for them
 * before the call's work is complete.  Either way the results are the same
 * bit for bit.  To capture such a call in a CUDA graph, make one uncaptured
 * call first (stream creation) and capture in relaxed mode. */
int ts_sinr_svd_multiuser(const ts_dims* d, int U, const ts_coef* coef, const ts_c64* G,
                          const ts_c64* C, const float* sigma2, float* sinr, uint8_t* flags,
                          void* ws, size_t ws_bytes, void* stream);

/* The same on the uncompressed channels X [U][J*J][P][M][N] (the dense
 * comparator; d's M, N, P are used, P <= 1024).
 * ws: ts_workspace_bytes(d, TS_OP_DENSE_SVD_MULTIUSER) bytes. */
int ts_dense_sinr_svd_multiuser(const ts_dims* d, int U, const ts_coef* coef, const ts_c64* X,
                                const float* sigma2, float* sinr, uint8_t* flags, void* ws,
                                size_t ws_bytes, void* stream);

/* Dense-channel comparator: the same SINR computed from the uncompressed
 * channel tensors, rebuilding the full M x N channel of every link and
 * subcarrier, H_ik(kappa) = X_ik x_3 c_ik(kappa)* (eq. 9), and running the
 * precoder, covariance and solves at size (M, N) (eq. 3-7) -- the "original
 * data" side of the paper's speedup R_t (Section 4).
 * X: [J*J][P][M][N] (the submatrices of eq. 2 stacked on mode 3, N fastest).
 * Pfull (mmse): [J][N][L].  d->m, d->n, d->p are ignored; limits: SVD
 * M <= 64, N <= 1024, P <= 1024 (L <= 8 when N > 512); wideband precoder
 * M <= 16, N <= 512, P <= 32.  ws: ts_workspace_bytes(d, TS_OP_DENSE_SVD /
 * _MMSE). */
int ts_dense_sinr_svd(const ts_dims* d, const ts_coef* coef, const ts_c64* X,
                      const float* sigma2, float* sinr, uint8_t* flags, void* ws,
                      size_t ws_bytes, void* stream);
int ts_dense_sinr_mmse(const ts_dims* d, const ts_coef* coef, const ts_c64* X,
                       const ts_c64* Pfull, const float* sigma2, float* sinr,
                       uint8_t* flags, void* ws, size_t ws_bytes, void* stream);

/* Groupwise Tucker compression (Section 3.2, eq. 16-22, Algorithm 2), FP64
 * inside: initialisation from the mode Grams of X (eq. 20-22 with the other
 * factors set to the identity; init = 0) or from the factors given in A, B,
 * C (init = 1, e.g. to resume), then S Gauss-Seidel sweeps -- all A_i
 * (eq. 20), then all B_k (eq. 21), then all C_ik (eq. 22), each the leading
 * eigenvectors of a summed mode Gram -- and the core (eq. 17) once at the
 * end.  Eigensolvers: cyclic Jacobi for Gram dimensions <= 72, block subspace
 * iteration with a Rayleigh-Ritz step above that (blocks beyond 72 columns
 * in global scratch; a block that would span the Gram solves it directly).
 * X: [J*J][P][M][N] (link i*J+k, submatrices of eq. 2 stacked on mode 3);
 * A (out, or in for init = 1): [J][M][m]; B: [J][N][n]; C: [J*J][P][p];
 * G (out): [J*J][p][m][n]; g_hist (device, may be NULL): 3 S + 1 doubles,
 * the objective g of eq. (19) after the initialisation and after every block
 * update.  Ranks up to 256.  ws: ts_workspace_bytes(d, TS_OP_TUCKER_FIT). */
int ts_tucker_fit(const ts_dims* d, const ts_c64* X, int S, int init, ts_c64* A,
                  ts_c64* B, ts_c64* C, ts_c64* G, double* g_hist, void* ws,
                  size_t ws_bytes, void* stream);

/* Algorithm 2 for any of the three models (TS_MODEL_*): the same
 * initialisation and Gauss-Seidel sweeps, each factor fitted from the mode
 * Gram summed over the links that share it.  A: [nA][M][m], B: [nB][N][n]
 * with nA = nB = J (groupwise), 1 (shared) or J^2 (individual, link i*J+k);
 * other arguments as ts_tucker_fit (which is the groupwise model).
 * ws: ts_workspace_bytes(d, TS_OP_TUCKER_FIT / _FIT_SHARED / _FIT_INDIVIDUAL). */
int ts_tucker_fit_model(const ts_dims* d, const ts_c64* X, int S, int init, int model, ts_c64* A,
                        ts_c64* B, ts_c64* C, ts_c64* G, double* g_hist, void* ws, size_t ws_bytes,
                        void* stream);

/* Reconstruction X^_ik = G_ik x_1 A x_2 B x_3 C_ik (eq. 10, 12, 14) with the
 * model's factors, FP32: Xhat (out) [J*J][P][M][N] -- e.g. to evaluate a
 * model whose factors do not cancel (individual) on the dense-channel path.
 * Factor layouts as ts_tucker_fit_model; G: [J*J][p][m][n].  Any ranks up
 * to the dimensions (M, N, P <= 4096, J <= 256).
 * ws: ts_workspace_bytes(d, TS_OP_RECONSTRUCT) bytes. */
int ts_tucker_reconstruct(const ts_dims* d, int model, const ts_c64* A, const ts_c64* B,
                          const ts_c64* C, const ts_c64* G, ts_c64* Xhat, void* ws,
                          size_t ws_bytes, void* stream);

/* Adjoints (vector-Jacobian products) of the compressed SINR.  The paper has
 * no adjoint; these differentiate its compressed SINR (eq. 15, 23-28) for a
 * real loss l whose gradient dl/dSINR is `dsinr` ([J][K][L] float):
 *   ts_sinr_svd_adjoint:  dG = dl/dG ([J*J][p][m][n]), dC = dl/dC ([J*J][P][p])
 *                         through the SVD precoders of eq. (7) as well;
 *   ts_sinr_mmse_adjoint: also dPt = dl/dPt ([J][n][L]) for the wideband
 *                         precoders (ts_project_precoder_adjoint carries it to
 *                         dl/dB).
 * Gradients of complex parameters are dl/dRe + i dl/dIm; outputs are
 * overwritten.  dl/dA is zero: A cancels (eq. 28).  The forward quantities
 * are recomputed from (G, C, coefficients), nothing is kept from a forward
 * call; `sinr` (may be NULL) receives the recomputed forward SINR.
 * Near-degenerate singular values of a serving channel make the SVD adjoint
 * ill-conditioned (1 / (s_r^2 - s_s^2) terms), as they make the SINR itself.
 * ws: ts_workspace_bytes(d, TS_OP_SINR_SVD_ADJOINT / _MMSE_ADJOINT) bytes. */
int ts_sinr_svd_adjoint(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                        const ts_c64* C, const float* sigma2, const float* dsinr,
                        ts_c64* dG, ts_c64* dC, float* sinr, void* ws,
                        size_t ws_bytes, void* stream);
int ts_sinr_mmse_adjoint(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                         const ts_c64* C, const ts_c64* Pt, const float* sigma2,
                         const float* dsinr, ts_c64* dG, ts_c64* dC, ts_c64* dPt,
                         float* sinr, void* ws, size_t ws_bytes, void* stream);
/* dB[k] = conj(Pfull[k]) dPt[k]^T, the adjoint of Pt = B^T Pfull.
 * Pfull: [J][N][L]; dPt: [J][n][L]; dB (out): [J][N][n]. */
int ts_project_precoder_adjoint(const ts_dims* d, const ts_c64* Pfull,
                                const ts_c64* dPt, ts_c64* dB, void* stream);

/* Allocation-free variant of ts_sinr_mmse (the paper has no counterpart: it
 * is a service of this library).  For callers that cannot allocate device
 * memory when they evaluate SINR -- a per-slot scheduler loop with a fixed
 * latency budget, where cudaMalloc/cudaFree may synchronise the device and
 * stall for milliseconds, or a plug-in inside a framework that owns and
 * pre-reserves all device memory.  Same arguments and results as
 * ts_sinr_mmse, without ws/ws_bytes: the scratch is a fixed array of
 * TS_NOALLOC_SCRATCH_BYTES in the library's own device memory, which every
 * GPU that loads the library holds until the process exits.
 *   - Sizes whose ts_workspace_bytes(d, TS_OP_SINR_MMSE) exceeds
 *     TS_NOALLOC_SCRATCH_BYTES are rejected with TS_ERR_WORKSPACE before
 *     any launch (for example J = 8, m = 8, L = 8 fits up to K = 495
 *     subcarriers).
 *   - Every call looks up the array's device address (cudaGetSymbolAddress,
 *     with the calling thread's current device); after the first call on a
 *     device that lookup only reads a host-side table.  The first call on
 *     each device also loads the library's module there, which commits the
 *     array: it may synchronise the device, and it fails with a CUDA error
 *     (TS_ERR_CUDA) if the device has no room left.  Make that first call at
 *     start-up, before a framework reserves the device's memory; later calls
 *     change no allocation.
 *   - Every call shares the one array per device, which keeps the previous
 *     call's contents (nothing needs clearing: each call writes every byte
 *     it reads).  Calls that overlap on the GPU -- on two streams, or from
 *     two host threads on one device -- race on it; serialise them.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library
 *     routine. */
#define TS_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int ts_sinr_mmse_noalloc(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                         const ts_c64* C, const ts_c64* Pt, const float* sigma2,
                         float* sinr, uint8_t* flags, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TUCKERSINR_H */
