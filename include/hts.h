/*
 * hts.h -- C ABI of the GB300 (sm_103a) library for the two-stage reduction of a real
 * matrix pencil (A, B) to Hessenberg-triangular (HT) form, after Steel & Vandebril,
 * "Parallel two-stage reduction to Hessenberg-triangular form".
 *
 * The decomposition (Section 1 of the paper): orthogonal Q, Z, upper Hessenberg H and upper
 * triangular T with (A, B) = Q (H, T) Z^T.  A pencil is in r-Hessenberg-triangular (r-HT)
 * form when T is upper triangular and H(i, j) = 0 for i > j + r.
 *
 * Conventions shared by every entry point
 *  - Matrices are device pointers to column-major FP64 arrays owned by the caller; the
 *    leading dimension must be >= max(1, n).  The library never allocates device memory on
 *    these paths: all scratch lives in the caller's `work` buffer, whose size
 *    hts_workspace_size() reports.  `work` must be 256-byte aligned.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy
 *    default stream).  Argument errors are detected on the host before anything is
 *    enqueued and are returned as HTS_ERR_ARG / HTS_ERR_WORKSPACE / HTS_ERR_UNSUPPORTED.
 *    Errors found on the device are recorded in a status word of the context and reported by
 *    hts_sync_status(): a bounded inter-block wait that ran out (HTS_ERR_TIMEOUT), and a NaN or
 *    infinite entry among the inputs a call reads (HTS_ERR_NONFINITE, info = {0, matrix (0 A,
 *    1 B, 2 Q, 3 Z), row, column}; for the batched call {pencil, matrix, row, column}).  Every
 *    call first scans the entries it reads: A on and above its r-th subdiagonal and the upper
 *    triangle of B for stage 2, all of A and the upper triangle of B for stage 1, all of A and
 *    B for the full reduction, and Q / Z with HTS_COMP_UPDATE.  After a non-finite input the
 *    stage-2 kernels do nothing; stages 0 and 1 of the full reduction may still run, so the
 *    contents of the matrices are then unspecified.
 *  - On exit A holds H and B holds T with exact zeros below the first subdiagonal of H and
 *    below the diagonal of T.
 *  - compq / compz: HTS_COMP_NONE leaves Q / Z untouched (the pointer may be NULL);
 *    HTS_COMP_INIT overwrites it with the stage's own orthogonal factor; HTS_COMP_UPDATE
 *    multiplies it from the right (Q := Q Q_stage), so that A_in = Q H Z^T holds for the
 *    matrices passed in.
 */
#ifndef HTS_H
#define HTS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HTS_OK = 0,
    HTS_ERR_ARG = 1,          /* invalid size, leading dimension, pointer or parameter */
    HTS_ERR_CUDA = 2,         /* a CUDA runtime call failed (launch, stream, device) */
    HTS_ERR_WORKSPACE = 3,    /* work is NULL, misaligned or smaller than required */
    HTS_ERR_TIMEOUT = 4,      /* a bounded wait between thread blocks ran out (device) */
    HTS_ERR_NONFINITE = 5,    /* NaN / Inf among the input entries (device; hts_sync_status) */
    HTS_ERR_UNSUPPORTED = 6   /* valid request this build does not implement */
} hts_status;

typedef enum {
    HTS_COMP_NONE = 0,
    HTS_COMP_INIT = 1,
    HTS_COMP_UPDATE = 2
} hts_comp;

/* Arithmetic of the delayed reflector-block updates (the far-from-diagonal updates of
 * Alg. 4 of the paper).  The near-diagonal chase always runs in native FP64. */
typedef enum {
    HTS_GEMM_FP64 = 0,        /* native FP64 */
    HTS_GEMM_EMU_BF16 = 1     /* FP64 emulated on BF16 tensor cores (split operands) */
} hts_gemm_mode;

/* Tuning parameters; 0 selects the library default.
 *  q          sweeps grouped per generate/apply iteration (Section "Blocked stage two");
 *             1 <= q <= r.  Default: r.
 *  p          stage-1 block height in units of r (Alg. 1); p >= 2 and p*r <= 128 (one
 *             block's RQ runs in shared memory).  Default: min(8, 128/r).
 *  emu_slices number of BF16 digits per FP64 operand in HTS_GEMM_EMU_BF16 mode: 0 or 8 (the
 *             only value this build implements; others give HTS_ERR_UNSUPPORTED).
 *  tile_m     emulated delayed updates of the look-ahead schedule: 0 or 64 selects the
 *             tensor-core kernel on tiles of 64 lines (tcgen05.mma with TMEM accumulators,
 *             the reflector products loaded by TMA; needs r = 16), 32 the warp-level kernel on
 *             tiles of 32 lines (mma.sync); other values give HTS_ERR_UNSUPPORTED.
 *  tile_n     batched calls: persistent blocks per SM of the launch (0, the default, or more
 *             than the SM holds: as many as it holds; < 0: HTS_ERR_ARG).  hts_plan_batched keeps
 *             the value in the context for the planned launches that follow it.  Other calls:
 *             reserved.
 *  flags      bit 0 (HTS_FLAG_NO_CLEAN): skip the final exact zeroing below the band.
 *             bit 1 (HTS_FLAG_SERIAL_UPDATES): run each group's delayed updates after its
 *             chase instead of beside the next group's chase (the look-ahead of Section
 *             "Parallel stage two", the default); same results up to rounding, for comparison.
 *             bit 30 (HTS_FLAG_TEST_STALL): fault injection for tests of the failure path:
 *             the chase block of the first sweep never publishes its progress, so the next
 *             block's bounded wait (2 s) runs out and HTS_ERR_TIMEOUT is reported by
 *             hts_sync_status; every later kernel of the call then returns at once.
 *             bit 29 (HTS_FLAG_TEST_DIRECT_RQ): for tests of the fallback path of the r <= 16
 *             chase: every step takes the direction of its opposite reflector from the RQ
 *             of the B block, as when the elimination's residual check fails (the r > 16
 *             kernel always uses the RQ). */
typedef struct {
    int q;
    int p;
    int emu_slices;
    int tile_m;
    int tile_n;
    int flags;
} hts_params;

#define HTS_FLAG_NO_CLEAN 1
#define HTS_FLAG_SERIAL_UPDATES 2
#define HTS_FLAG_TEST_STALL (1 << 30)
#define HTS_FLAG_TEST_DIRECT_RQ (1 << 29)

typedef struct hts_ctx hts_ctx;

/* Create a context bound to CUDA device `device` (allocates a small device status word).
 * Returns HTS_ERR_ARG for a NULL ctx pointer, HTS_ERR_CUDA if the device is unusable. */
hts_status hts_create(hts_ctx **ctx, int device);

/* Destroy a context created by hts_create (NULL is ignored). */
void hts_destroy(hts_ctx *ctx);

/* Bytes of `work` needed by hts_reduce_stage1 / hts_reduce_stage2 / hts_reduce for an n x n
 * pencil with r subdiagonals and parameters p (NULL = defaults).  The size covers all three
 * entry points and both update modes (HTS_GEMM_EMU_BF16 adds 64 KiB per block of r columns
 * for the digit planes of the reflector products; stages 0 and 1 include 4 MiB that the
 * context's cuBLAS handle uses as its workspace for the block-reflector products). */
hts_status hts_workspace_size(int n, int r, const hts_params *p, size_t *bytes);

/*
 * Stage 1: Alg. 1 of the paper ("Blocked stage 1") with n_b = r.  Requires B upper
 * triangular (its strictly lower part is ignored and zeroed) and 1 <= r < n, r <= 64.  On
 * exit (A, B) is in r-HT form with exact zeros below the r-th subdiagonal of A and below the
 * diagonal of B.  The block reflectors are applied in compact WY form (native FP64);
 * HTS_GEMM_EMU_BF16 returns HTS_ERR_UNSUPPORTED.
 */
hts_status hts_reduce_stage1(hts_ctx *ctx, int n, int r,
                             double *A, int lda, double *B, int ldb,
                             hts_comp compq, double *Q, int ldq,
                             hts_comp compz, double *Z, int ldz,
                             hts_gemm_mode mode, const hts_params *p,
                             void *work, size_t work_bytes, void *stream);

/*
 * Stage 2: reduction of an r-HT pencil to HT form by bulge chasing (Section "Reduction to
 * Hessenberg-triangular form"; Alg. 2 defines the reflectors, Alg. 3 and Alg. 4 the blocked
 * generate / apply schedule this implementation runs).  Requires 1 <= r and n >= 1; entries
 * of A below the r-th subdiagonal and of B below the diagonal are treated as zero.  r = 1
 * (and n <= 2) is a no-op apart from HTS_COMP_INIT.  Reflectors act on rows/columns 2..n
 * only, so Q e_1 and Z e_1 are unchanged.  Each step's opposite reflector is the one the paper
 * forms from an RQ of the B block; its first column is the direction z with (B block) z
 * parallel to e_1.  For r <= 16 the library finds z by column elimination with partial
 * pivoting and checks the entries the reflector zeroes against 2^-44 max|block| max|z|; a
 * step that fails the check (or meets extreme magnitudes) takes z from the RQ.
 * mode selects the arithmetic of the delayed updates (Alg. 4): HTS_GEMM_FP64 applies the
 * reflectors one at a time in native FP64; HTS_GEMM_EMU_BF16 forms each block's reflector
 * product U_k (w x w, w = r + q - 1) and applies it as a product emulated on the BF16 tensor
 * cores (8 base-256 digits per operand, FP32 accumulation of exact integer partial sums,
 * error of each product below 2^-55 of the power of two above the window's largest entry,
 * about 2^-58 typically); it requires r = 16
 * (HTS_ERR_UNSUPPORTED otherwise).  The chase runs in native FP64 in both modes.
 */
hts_status hts_reduce_stage2(hts_ctx *ctx, int n, int r,
                             double *A, int lda, double *B, int ldb,
                             hts_comp compq, double *Q, int ldq,
                             hts_comp compz, double *Z, int ldz,
                             hts_gemm_mode mode, const hts_params *p,
                             void *work, size_t work_bytes, void *stream);

/*
 * Stage 2 without a caller-provided workspace, for callers that cannot allocate device
 * memory when they need the reduction (services that must not allocate once running, code
 * inside a host framework that owns all device memory and lends out only the matrices).
 * The paper has no counterpart: this is a deployment variant of hts_reduce_stage2 with the
 * same arguments minus work / work_bytes and the same results.
 *  - Scratch lives in one fixed 8 MiB array compiled into the library; every GPU that loads
 *    the library holds it until the process exits.  A call whose stage-2 scratch in the chosen
 *    update mode exceeds 8 MiB is rejected with HTS_ERR_WORKSPACE before anything runs (the
 *    check precedes every other argument check).  In native FP64 mode r = 16 fits n up to
 *    6943 and r = 32 up to 5215; the emulated mode's digit planes fit n up to 1119 at r = 16.
 *  - The call allocates nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *    with that device current); make that first call before any stream capture.
 *  - All calls on a device share the array and it keeps the last call's contents (each call
 *    clears what must start at zero).  Calls that overlap on the GPU (other streams, other
 *    threads) race on it: serialise them.
 */
hts_status hts_reduce_stage2_noalloc(hts_ctx *ctx, int n, int r,
                                     double *A, int lda, double *B, int ldb,
                                     hts_comp compq, double *Q, int ldq,
                                     hts_comp compz, double *Z, int ldz,
                                     hts_gemm_mode mode, const hts_params *p, void *stream);

/*
 * Full reduction of a dense pencil: QR of B (stage 0; the paper QR-factorises B first,
 * Section "Experiments"), then stage 1 with n_b = r, then stage 2.  Requires 1 <= r < n and
 * r <= 32.  With HTS_COMP_INIT, Q e_1 = +-B(:,1)/||B(:,1)|| and Z e_1 = e_1.  mode applies to
 * stage 2's delayed updates (stages 0 and 1 run in native FP64).
 */
hts_status hts_reduce(hts_ctx *ctx, int n, int r,
                      double *A, int lda, double *B, int ldb,
                      hts_comp compq, double *Q, int ldq,
                      hts_comp compz, double *Z, int ldz,
                      hts_gemm_mode mode, const hts_params *p,
                      void *work, size_t work_bytes, void *stream);

/*
 * Batched full reduction (QR of B, stage 1 with n_b = r_i, stage 2) of `count` independent
 * pencils of possibly different sizes in one launch.  The array arguments are host arrays
 * of length count (device pointers for the matrices); compq / compz apply to every pencil.
 * Each pencil is reduced by one thread block with its reflectors applied one at a time, so
 * the batch, not a single pencil, supplies the parallelism.  The launch is persistent: as many
 * blocks as the SMs hold at once (or params.tile_n per SM) take pencils from a device queue,
 * largest pencil first.
 * Limits of this path: n_i <= 512, r_i <= 16 and r_i < n_i (or n_i <= 2),
 * p * r_i <= 64 (p defaults to min(8, 64/r_i)).  `work` (256-byte aligned,
 * hts_workspace_size_batched() bytes) holds the pencil descriptors, the order and the queue.
 * The results equal those of hts_reduce up to rounding.  Equivalent to hts_plan_batched
 * followed by hts_reduce_batched_planned.
 */
hts_status hts_workspace_size_batched(int count, const int *n, const int *r, const hts_params *p,
                                      size_t *bytes);
hts_status hts_reduce_batched(hts_ctx *ctx, int count, const int *n, const int *r,
                              double *const *A, const int *lda, double *const *B, const int *ldb,
                              hts_comp compq, double *const *Q, const int *ldq,
                              hts_comp compz, double *const *Z, const int *ldz,
                              hts_gemm_mode mode, const hts_params *p, void *work, size_t work_bytes,
                              void *stream);

/*
 * The batched reduction in two parts, for a batch that is reduced many times with the same
 * matrix pointers (new values each time), and for CUDA graphs:
 *  - hts_plan_batched checks the arguments as hts_reduce_batched does and writes the batch's
 *    descriptors, largest-first order, compq / compz and p into `work` (an asynchronous copy
 *    on `stream`; the host arrays may be released when it returns).  It reads no matrix.
 *  - hts_reduce_batched_planned reduces the planned batch: it resets the queue counter in
 *    `work` and launches the persistent kernel, both on `stream`, using no host data but
 *    `count`.  It may be captured into a CUDA graph and replayed; the plan must stay in
 *    `work`, and work must not be shared by launches that overlap on the GPU.
 * Errors: HTS_ERR_ARG, HTS_ERR_UNSUPPORTED as for hts_reduce_batched; HTS_ERR_WORKSPACE when
 * work is null, not 256-byte aligned or shorter than hts_workspace_size_batched(); HTS_ERR_CUDA.
 * Device errors (HTS_ERR_NONFINITE with the pencil index) through hts_sync_status.
 */
hts_status hts_plan_batched(hts_ctx *ctx, int count, const int *n, const int *r,
                            double *const *A, const int *lda, double *const *B, const int *ldb,
                            hts_comp compq, double *const *Q, const int *ldq,
                            hts_comp compz, double *const *Z, const int *ldz,
                            hts_gemm_mode mode, const hts_params *p, void *work, size_t work_bytes,
                            void *stream);
hts_status hts_reduce_batched_planned(hts_ctx *ctx, int count, void *work, size_t work_bytes, void *stream);

/*
 * Wait for `stream`, then report and clear the context's device status word.
 * info (may be NULL) receives {pencil, group, k, j} of the first device-side error.
 * Returns HTS_OK, HTS_ERR_TIMEOUT, or HTS_ERR_CUDA if the stream itself failed.
 */
hts_status hts_sync_status(hts_ctx *ctx, void *stream, int info[4]);

/* Human-readable name of a status code (static string). */
const char *hts_status_string(hts_status s);

#ifdef __cplusplus
}
#endif

#endif /* HTS_H */
