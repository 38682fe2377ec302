/*
 * dbp.h -- C ABI of the B300 (sm_103a) decentralized baseband processing
 * library libdbp.so.
 *
 * The library runs the per-subcarrier, per-antenna-cluster hot path of
 * decentralized massive MU-MIMO baseband processing (Li, Sharan, Chen,
 * Goldstein, Cavallaro, Studer, "Decentralized Baseband Processing for
 * Massive MU-MIMO Systems"):
 *   - decentralized consensus-ADMM uplink detection   (Alg. 1, Sec. III-B/C)
 *   - decentralized conjugate-gradient uplink detection (Alg. 2, Sec. III-D)
 *   - decentralized ADMM downlink beamforming          (Alg. 3, Sec. IV-B/C)
 * as hand-written CUDA kernels.  There is no CPU fallback: every compute
 * entry point fails with DBP_ERR_CUDA when no usable GPU is present.
 *
 * Shapes (Sec. II): B base-station antennas in C clusters of S = B / C
 * antennas, U single-antenna users, W subcarriers, N OFDM symbols per
 * subcarrier (the channel is constant over the N symbols of a subcarrier).
 *
 * Memory layouts: row-major, complex numbers interleaved (re, im):
 *   H      [W][B][U]  uplink channel; cluster c owns rows c*S .. c*S+S-1
 *                     (row-wise partition of Sec. II-A.2).  The downlink
 *                     uses the same buffer: H^d = (H^u)^T (reciprocity,
 *                     Sec. II-B).
 *   y      [W][N][B]  uplink receive vectors
 *   x_hat  [W][N][U]  equaliser outputs (uplink)
 *   labels [W][N][U]  uint8 Gray bit labels of the sliced symbols: for
 *                     M = L*L points and m = log2 M, label =
 *                     (g(kI) << m/2) | g(kQ), g(k) = k ^ (k >> 1), where the
 *                     PAM index k maps to amplitude (2k-(L-1))*sqrt(3/(2(M-1)))
 *   s      [W][N][U]  downlink transmit symbols
 *   x      [W][N][B]  downlink beamforming vectors
 * Element type by precision: DBP_FP32 -> float complex (8 B),
 * DBP_FP64 -> double complex (16 B), DBP_FP16 / DBP_BF16 -> two 16-bit
 * floats (4 B) for H and y with x_hat as float complex.  All device
 * pointers must be aligned to the element size; 16-byte alignment enables
 * the bulk-copy kernel.
 *
 * Ownership: the caller owns every input and output buffer and keeps it
 * alive until the work enqueued on `stream` has completed.  The library
 * owns its handle, its workspace and its host staging buffers; descriptors
 * are copied at call time.  `stream` is a cudaStream_t (NULL = the legacy
 * default stream).  Compute calls are stream-ordered: DBP_OK means the work
 * was validated and enqueued.  No C++ exception crosses this interface.
 */
#ifndef DBP_H
#define DBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dbp_status {
    DBP_OK = 0,
    DBP_ERR_INVALID_ARG = 1,   /* bad shape, parameter or pointer            */
    DBP_ERR_UNSUPPORTED = 2,   /* valid but outside what the kernels handle  */
    DBP_ERR_NOMEM = 3,         /* device or host allocation failed           */
    DBP_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed       */
    DBP_ERR_TIMEOUT = 5,       /* a bounded wait ran out                     */
    DBP_ERR_UNIMPLEMENTED = 6, /* entry point not provided by this library   */
    DBP_PENDING = 7,           /* submitted work has not completed yet       */
    DBP_ERR_CANCELLED = 8      /* a queued request was cancelled (dbp_cancel)*/
} dbp_status;

typedef enum dbp_precision {
    DBP_FP32 = 0,              /* complex float in, FP32 arithmetic          */
    DBP_FP64 = 1,              /* complex double in, FP64 arithmetic         */
    DBP_FP16 = 2,              /* uplink only: H and y stored as complex
                                  FP16 (4 B); Gram and matched filter on the
                                  tensor cores with FP32 accumulation, FP32
                                  inverse (FP64 retry on a small pivot) and
                                  iterations; x_hat is complex float        */
    DBP_BF16 = 3               /* as DBP_FP16 with BF16 storage             */
} dbp_precision;

/* Regulariser g(s) of the equalisation problem (E0), Sec. III-A, and its
 * proximal step (E2), Lemma 1. */
typedef enum dbp_regularizer {
    DBP_REG_ZF = 0,            /* g = 0                 : s = v              */
    DBP_REG_MMSE = 1,          /* g = N0/(2Es)||s||^2   : (E2-MMSE)          */
    DBP_REG_BOX = 2,           /* g = box indicator     : (E2-BOX), radius r */
    DBP_REG_BPSK = 3           /* g = indicator of the real segment [-r, r]:
                                * s_u = sign(Re v_u) min(|Re v_u|, r), Im s_u = 0
                                * (the BPSK prox of Sec. III-B); qam_order 2
                                * or 0 */
} dbp_regularizer;

/* Descriptor flags. */
#define DBP_FLAG_NORMALIZE 1u  /* downlink: scale x to unit mean per-antenna
                                  power over the frame (one scalar beta)    */

typedef struct dbp_config {
    int32_t device;            /* CUDA device ordinal                        */
    int32_t reserved;
    uint64_t hbm_budget_bytes; /* cap on the device memory the library itself
                                  allocates for this handle (host-variant
                                  staging buffers, the request loop's pool,
                                  the separate operator kernel's buffers, the
                                  normalisation accumulator); an allocation
                                  past it fails with DBP_ERR_NOMEM.  0 = no
                                  limit.  The caller's own buffers do not
                                  count                                      */
} dbp_config;

typedef struct dbp_frame_desc {
    int32_t B, C, U;           /* antennas, clusters (B % C == 0), users     */
    int32_t W, N;              /* subcarriers, OFDM symbols per subcarrier   */
    int32_t qam_order;         /* 4, 16, 64 or 256: slicer alphabet (unit-
                                  energy Gray QAM); 2: BPSK {-1, +1}, label k
                                  for 2k - 1, only with DBP_REG_BPSK; 0 = no
                                  labels                                     */
    int32_t T_max;             /* iterations: ADMM counts the init as the
                                  first (T_max >= 1); CG counts loop trips
                                  (T_max >= 0)                               */
    int32_t regularizer;       /* dbp_regularizer (uplink ADMM; CG uses
                                  rho = N0/Es for MMSE, 0 for ZF)            */
    int32_t precision;         /* dbp_precision                              */
    uint32_t flags;            /* DBP_FLAG_*                                 */
    double rho;                /* ADMM penalty rho > 0 (Alg. 1 and Alg. 3)   */
    double gamma;              /* dual step gamma (the paper uses 1)         */
    double N0;                 /* noise variance per complex entry           */
    double Es;                 /* symbol energy E[|s_u|^2] > 0               */
    double box_r;              /* radius r for DBP_REG_BOX and DBP_REG_BPSK  */
    double eps;                /* downlink: residual-interference bound
                                  epsilon >= 0 of (P0); the consensus step
                                  scales (s - w)/C by max{0, 1 - eps /
                                  ||s - w||} (Lemma 2).  0 = Alg. 3 as
                                  printed; must be 0 for the uplink          */
} dbp_frame_desc;

/* Launch-shape tuning (the autotuner's knobs; results do not depend on them
 * beyond floating-point rounding of the consensus, which is summed in the
 * same cluster order under every shape). */
typedef enum dbp_mapping {
    DBP_MAP_AUTO = 0,          /* CTA mapping when one CTA holds all C warps */
    DBP_MAP_CTA = 1,           /* P whole subcarriers per CTA, shared-memory
                                  consensus                                  */
    DBP_MAP_CLUSTER = 2        /* one subcarrier per thread-block cluster of
                                  cluster_size CTAs, DSMEM consensus         */
} dbp_mapping;

typedef enum dbp_kernel_path {
    DBP_PATH_AUTO = 0,         /* uplink ADMM: DBP_PATH_TC5 (unless the
                                  operator kernel or a resident operator is
                                  asked for), then as uplink CG: DBP_PATH_MMA,
                                  else DBP_PATH_BCAST, else DBP_PATH_TMA;
                                  downlink: DBP_PATH_MMA, else DBP_PATH_TMA;
                                  each where eligible, then
                                  DBP_PATH_GENERIC                           */
    DBP_PATH_GENERIC = 1,      /* per-subcarrier kernel with staged loads:
                                  any shape, FP64, thread-block clusters     */
    DBP_PATH_TMA = 2,          /* persistent kernel fed by cp.async.bulk:
                                  U in {4,8,16,32}, even S <= 64, 16-byte
                                  aligned buffers, CTA mapping               */
    DBP_PATH_MMA = 3,          /* FP32, C <= 16, every dense product (Gram,
                                  matched filter, operator x state, output)
                                  on the tensor cores (three products per
                                  FP32 product: TF32 halves at U = 8, FP16
                                  halves with power-of-two scales at U = 16),
                                  consensus as DBP_PATH_BCAST: uplink ADMM and
                                  CG with U = 8 and even S; downlink ADMM with
                                  U = 16 and S a multiple of 8               */
    DBP_PATH_BCAST = 4         /* uplink ADMM and CG, FP32, U in {4,8,16},
                                  even S, C <= 16: the consensus and the
                                  centralized step (the (E2) prox of Alg. 1;
                                  the e, x, r, p updates of Alg. 2, the first
                                  placement of Sec. III-D) run once per
                                  symbol and s or p is broadcast to the
                                  clusters                                   */,
    DBP_PATH_TC5 = 5           /* uplink ADMM with U = S = 32 (B = 32 C), C
                                  even and <= 8, N <= 16, FP32 / FP16 / BF16
                                  inputs, 16-byte aligned buffers: every
                                  dense product (Gram, matched filter,
                                  B_c^{-1} times the state) on the tcgen05
                                  tensor cores with accumulators in tensor
                                  memory, two clusters per M = 128 MMA; FP32
                                  operands as scaled FP16 hi / lo pairs
                                  (three products, FP32 accumulation);
                                  B_c^{-1} by the 2 x 2 block inverse (two
                                  16-row eliminations, two tensor-core
                                  products per cluster)                      */
} dbp_kernel_path;

typedef enum dbp_prefactor {
    DBP_PREFACTOR_AUTO = 0,    /* off (measured slower on every shape where
                                  it is available); the autotuner times both */
    DBP_PREFACTOR_OFF = 1,     /* the fused kernel forms B_c^{-1} itself     */
    DBP_PREFACTOR_ON = 2       /* where available: B_c^{-1} of every
                                  (subcarrier, cluster) first, by a kernel
                                  with independent warps (many per SM), into
                                  a stream-ordered buffer of W*C*U*U complex
                                  FP32 taken from a pool of the handle; the
                                  fused kernel then loads it.  Available for
                                  ADMM (Alg. 1, Alg. 3) on the persistent
                                  bulk-copy kernel with U in {16, 32} and on
                                  the U = 16 tensor-core downlink kernel,
                                  outside stream capture and the request
                                  loop.  Same results bit for bit            */
} dbp_prefactor;

typedef struct dbp_tuning {
    int32_t mapping;           /* dbp_mapping                                */
    int32_t cluster_size;      /* CTAs per cluster (divides C, <= 16); 0 =
                                  smallest that fits                         */
    int32_t warps_per_cta;     /* CTA mapping: target warps per CTA; 0 = 8   */
    int32_t kernel;            /* dbp_kernel_path                            */
    int32_t prefactor;         /* dbp_prefactor                              */
} dbp_tuning;

typedef struct dbp_context *dbp_handle_t;

/* Create a handle bound to cfg->device (NULL cfg = device 0, no budget).
 * Returns DBP_ERR_CUDA when the device cannot be used. */
dbp_status dbp_create(dbp_handle_t *out, const dbp_config *cfg);

/* Release the handle and its workspace.  Waits for nothing: the caller
 * synchronises its streams first. */
dbp_status dbp_destroy(dbp_handle_t h);

/* Text of the last error on this handle ("" if none).  Valid until the next
 * call on the handle. */
const char *dbp_last_error(dbp_handle_t h);

/* Library version string. */
const char *dbp_version(void);

/* Set the launch-shape knobs used by later calls on this handle.
 * DBP_ERR_INVALID_ARG for out-of-range values; a shape that does not fit a
 * frame is reported by the compute call (DBP_ERR_UNSUPPORTED). */
dbp_status dbp_set_tuning(dbp_handle_t h, const dbp_tuning *t);

/* Wait for all work on the handle's device and report whether any kernel
 * gave up a bounded wait for its input copies since the last check
 * (DBP_ERR_TIMEOUT; the flag is then cleared).  The host-buffer variants
 * check this themselves. */
dbp_status dbp_device_status(dbp_handle_t h);

/* Wait for all work on the handle's device and return in *count how many
 * (subcarrier, cluster) inverses were recomputed in FP64 because a pivot
 * of the FP32 Gauss-Jordan elimination fell below 2^-12 of the largest
 * diagonal entry, since the last call (the counter is then cleared). */
dbp_status dbp_fp64_retries(dbp_handle_t h, uint32_t *count);

/* Decentralized ADMM-based data detection, Alg. 1 (Sec. III-B, III-C):
 * per subcarrier w and symbol n, C clusters each solve (E1) locally with
 * their own H_c, y_c; the consensus w = sum_c (z_c + lambda_c) is formed on
 * chip and every cluster applies the (E2) proximal step of Lemma 1 itself.
 * Inputs H [W][B][U], y [W][N][B] (device).  Outputs x_hat = s^(T_max)
 * [W][N][U] (device) and, if labels != NULL and qam_order > 0, the sliced
 * Gray labels [W][N][U] (device, uint8). */
dbp_status dbp_uplink_admm(dbp_handle_t h, const dbp_frame_desc *d,
                           const void *H, const void *y, void *x_hat,
                           uint8_t *labels, void *stream);

/* Decentralized CG-based data detection, Alg. 2 (Sec. III-D): MRC
 * y = sum_c H_c^H y_c, then T_max CG iterations on (H^H H + rho I) x = y
 * with the Gram product decentralized as sum_c H_c^H H_c p; every cluster
 * keeps its own copy of the CG state.  rho = N0/Es for DBP_REG_MMSE and
 * 0 for DBP_REG_ZF.  Same buffers as dbp_uplink_admm. */
dbp_status dbp_uplink_cg(dbp_handle_t h, const dbp_frame_desc *d,
                         const void *H, const void *y, void *x_hat,
                         uint8_t *labels, void *stream);

/* Decentralized ADMM-based beamforming, Alg. 3 (Sec. IV-B, IV-C) with
 * eps = 0: per subcarrier and symbol, cluster c computes its own part x_c of
 * the beamforming vector from H^d_c = (H^u_c)^T and the consensus
 * w = sum_c (H^d_c x_c - lambda_c).  Inputs H [W][B][U] (uplink layout),
 * s [W][N][U] (device).  Output x [W][N][B] (device).  With
 * DBP_FLAG_NORMALIZE, x is scaled in place by beta = sqrt(B*W*N / sum|x|^2)
 * and, if beta_out != NULL, beta is stored there (device, one double). */
dbp_status dbp_downlink_admm(dbp_handle_t h, const dbp_frame_desc *d,
                             const void *H, const void *s, void *x,
                             double *beta_out, void *stream);

/* Soft outputs (max-log LLRs) of an uplink estimate x_hat [W][N][U]
 * (complex64, e.g. the output of dbp_uplink_admm or dbp_uplink_cg) for the
 * frame whose channel H [W][B][U] (complex64) is given.  With the
 * subcarrier's Gram G = H^H H and A = (G + delta I)^{-1}, the estimate is
 * modelled as x_u = mu_u s_u + e_u:
 *   DBP_REG_MMSE (delta = N0/Es): mu_u = 1 - delta A_uu, E|e_u|^2 = Es mu_u (1 - mu_u)
 *   DBP_REG_ZF   (delta = 0):     mu_u = 1,              E|e_u|^2 = N0 A_uu
 * (the statistics of the estimate the detectors converge to, Sec. III-A).
 * llr [W][N][U][log2 M] (float32) receives, most significant label bit
 * first (labels as in the slicer: Gray I bits over Gray Q bits),
 *   L = (min_{s: bit = 1} |x - mu s|^2 - min_{s: bit = 0} |x - mu s|^2) / E|e|^2,
 * positive when the bit is more likely 0.  Needs qam_order > 0, N0 > 0,
 * Es > 0, precision DBP_FP32 and, for ZF, U <= B.  Stream-ordered. */
dbp_status dbp_uplink_llr(dbp_handle_t h, const dbp_frame_desc *d, const void *H,
                          const void *x_hat, float *llr, void *stream);

/* Host-memory variants (end-to-end path): the same computations with every
 * buffer in host memory.  The call copies the inputs to library-owned
 * device buffers, runs the kernels, copies the outputs back and returns
 * when all of it is done, ordered after the work already on `stream` (and
 * `stream` waits for it).  Frames of 512 subcarriers or more without a
 * whole-frame pass (all but a normalised downlink) run in up to 8 chunks of
 * subcarriers on three library-owned streams, so that input copies, kernels
 * and output copies overlap; the results are those of one launch, bit for
 * bit.  Pinned host memory gives the fastest copies (and the overlap);
 * pageable memory also works. */
dbp_status dbp_uplink_admm_host(dbp_handle_t h, const dbp_frame_desc *d,
                                const void *H, const void *y, void *x_hat,
                                uint8_t *labels, void *stream);
dbp_status dbp_uplink_cg_host(dbp_handle_t h, const dbp_frame_desc *d,
                              const void *H, const void *y, void *x_hat,
                              uint8_t *labels, void *stream);
dbp_status dbp_downlink_admm_host(dbp_handle_t h, const dbp_frame_desc *d,
                                  const void *H, const void *s, void *x,
                                  double *beta_out, void *stream);

/* ------------------------------------------------------------------------
 * Request loop (serving).  Frames arrive with HOST buffers and are admitted
 * as device memory and stream slots free up: a frame is admitted when one
 * of `streams` slots is free and the device pool (hbm_bytes) can hold its
 * staged inputs and outputs; a frame that does not fit yet may be passed by
 * later, smaller frames until it has waited 20 ms.  Admitted frames run
 * concurrently on separate streams (copies in, fused kernel, copies out).
 * Frames that carry the same non-zero channel_key and coherence_epoch share
 * one resident device copy of H and, where the persistent bulk-copy kernel
 * runs, the per-cluster operator (B_c^{-1} or G_c) computed by the
 * first of them: later frames of the coherence block skip the copy of H and
 * the Gram and inverse (the channel is constant over a coherence block,
 * Sec. II and Sec. VI-A).  Resident channels are evicted least recently
 * used when the pool is full.  A frame's result does not depend on what
 * else is in flight.
 * ------------------------------------------------------------------------ */
typedef enum dbp_kind {
    DBP_KIND_UPLINK_ADMM = 0,
    DBP_KIND_UPLINK_CG = 1,
    DBP_KIND_DOWNLINK_ADMM = 2
} dbp_kind;

typedef struct dbp_server_config {
    int32_t streams;           /* concurrent frames (slots); 0 = 4           */
    int32_t reserved;
    uint64_t hbm_bytes;        /* device pool for staged frames and resident
                                  channels; 0 = 2 GiB                        */
} dbp_server_config;

/* dbp_request.flags */
#define DBP_REQ_DEVICE_BUFFERS 1u  /* H, in, out, labels and beta_out are
                                      device pointers (caller-owned, alive
                                      until the ticket finishes): the frame
                                      runs on them in place, with no host
                                      copies; only the resident per-cluster
                                      operator of a coherence block comes
                                      from the pool                          */

typedef struct dbp_request {
    int32_t kind;              /* dbp_kind                                   */
    uint32_t flags;            /* DBP_REQ_*; 0 = host buffers               */
    dbp_frame_desc desc;
    const void *H;             /* host [W][B][U] (device with the flag)      */
    const void *in;            /* host y [W][N][B] (uplink), s [W][N][U]     */
    void *out;                 /* host x_hat [W][N][U] or x [W][N][B]        */
    uint8_t *labels;           /* host [W][N][U] or NULL (uplink)            */
    double *beta_out;          /* host, downlink normalisation, or NULL      */
    uint64_t channel_key;      /* 0 = no reuse                               */
    uint64_t coherence_epoch;  /* a new epoch of a key replaces its channel  */
    uint64_t user_tag;         /* returned in the result                     */
} dbp_request;

typedef struct dbp_result {
    int32_t status;            /* the frame's dbp_status                     */
    int32_t resident_hit;      /* 1 if the resident channel was reused       */
    uint64_t user_tag;
    double submit_us;          /* host monotonic microseconds since
                                  dbp_server_start: submission               */
    double start_us;           /*   admission (work enqueued)                */
    double finish_us;          /*   completion observed (outputs in host
                                    memory)                                  */
} dbp_result;

/* Start the request loop on this handle (one per handle).  Allocates the
 * device pool and the streams; DBP_ERR_NOMEM if the pool cannot be had. */
dbp_status dbp_server_start(dbp_handle_t h, const dbp_server_config *cfg);

/* Stop admitting, let in-flight frames finish (bounded: 30 s), fail the
 * frames still queued with DBP_ERR_TIMEOUT and release the pool. */
dbp_status dbp_server_stop(dbp_handle_t h);

/* Queue one frame.  The descriptor and pointers are copied; the buffers
 * must stay valid until dbp_poll / dbp_wait reports the ticket finished.
 * DBP_ERR_INVALID_ARG for a bad descriptor or unknown flags (checked here);
 * DBP_ERR_NOMEM if the frame's staged inputs and outputs alone are larger
 * than the pool (it could never be admitted). */
dbp_status dbp_submit(dbp_handle_t h, const dbp_request *req, uint64_t *ticket);

/* Cancel a frame that is still queued: DBP_OK (the ticket then finishes
 * with status DBP_ERR_CANCELLED and nothing ran), DBP_PENDING if it has
 * already been admitted (it runs to completion and keeps its ticket),
 * DBP_ERR_INVALID_ARG for an unknown or already finished ticket. */
dbp_status dbp_cancel(dbp_handle_t h, uint64_t ticket);

/* DBP_PENDING while the frame is queued or running; otherwise fills *res,
 * releases the ticket and returns DBP_OK (res->status holds the frame's own
 * status).  DBP_ERR_INVALID_ARG for an unknown ticket. */
dbp_status dbp_poll(dbp_handle_t h, uint64_t ticket, dbp_result *res);

/* As dbp_poll, blocking up to timeout_s seconds; DBP_ERR_TIMEOUT if the
 * frame has not finished by then (the ticket stays valid). */
dbp_status dbp_wait(dbp_handle_t h, uint64_t ticket, double timeout_s, dbp_result *res);

/* ------------------------------------------------------------------------
 * Autotuner.  Launch choices (kernel path, CTA size, thread-block cluster
 * size, separate operator kernel) are timed on a representative frame and the fastest is remembered
 * per frame shape (kind, B, C, U, N, precision) on the handle; calls whose
 * tuning is fully automatic (dbp_set_tuning defaults) then use it for every
 * frame of that shape, whatever W.  Results depend on the choice only
 * through floating-point rounding.
 * ------------------------------------------------------------------------ */

/* Time every launch choice that accepts the frame (device buffers; `out`
 * and `labels` are overwritten) with `reps` runs each (0 = 10) on `stream`,
 * remember the fastest for this shape and return it in *best (may be
 * NULL).  Not to be called while other calls on the handle are in flight.
 * DBP_ERR_INVALID_ARG for a bad descriptor. */
dbp_status dbp_autotune(dbp_handle_t h, int32_t kind, const dbp_frame_desc *d, const void *H,
                        const void *in, void *out, uint8_t *labels, void *stream, int32_t reps,
                        dbp_tuning *best);

/* Forget every tuned shape. */
dbp_status dbp_autotune_clear(dbp_handle_t h);

/* Write / read the tuned shapes as text, one shape per line
 * ("kind B C U N precision mapping cluster_size warps_per_cta kernel prefactor").
 * Loading adds to (and overrides) the handle's table; DBP_ERR_INVALID_ARG
 * for an unreadable file or a malformed line (nothing is loaded then). */
dbp_status dbp_autotune_save(dbp_handle_t h, const char *path);
dbp_status dbp_autotune_load(dbp_handle_t h, const char *path);

/* The launch choice that dbp_uplink_admm / dbp_uplink_cg /
 * dbp_downlink_admm (by `kind`) would make now for this descriptor and these
 * device buffers: the handle's tuning, else the autotuned choice for the
 * frame's shape, else the AUTO rule of dbp_kernel_path, resolved into
 * *chosen (may be NULL): a concrete kernel path (never DBP_PATH_AUTO), the
 * mapping, cluster_size (1 for the CTA mapping), warps_per_cta (the CTA's
 * warps) and prefactor (DBP_PREFACTOR_ON or _OFF).  Launches nothing and
 * reads no buffer: the pointers count only through their alignment (16-byte
 * alignment admits the bulk-copy and tensor-core kernels).  Returns what the
 * call would return for a descriptor or tuning it rejects
 * (DBP_ERR_INVALID_ARG, DBP_ERR_UNSUPPORTED), with dbp_last_error set. */
dbp_status dbp_plan(dbp_handle_t h, int32_t kind, const dbp_frame_desc *d, const void *H, const void *in,
                    const void *out, dbp_tuning *chosen);

/* ------------------------------------------------------------------------
 * Graphs: a batch of frames of any kinds and shapes (device buffers)
 * captured once into one CUDA graph and then run by a single launch.  The
 * frames are spread over `branches` independent branches of the graph, so
 * frames of different shapes run concurrently on the device, each with the
 * kernel its shape selects.  Descriptors and pointers are fixed when the
 * graph is made; every launch recomputes all frames from whatever their
 * input buffers hold at that point of `stream`.  Results equal those of
 * the same frames issued one by one.
 * ------------------------------------------------------------------------ */
typedef struct dbp_graph *dbp_graph_t;

typedef struct dbp_graph_item {
    int32_t kind;              /* dbp_kind                                   */
    int32_t reserved;
    dbp_frame_desc desc;
    const void *H;             /* device [W][B][U]                           */
    const void *in;            /* device y [W][N][B] (uplink), s [W][N][U]   */
    void *out;                 /* device x_hat [W][N][U] or x [W][N][B]      */
    uint8_t *labels;           /* device [W][N][U] or NULL (uplink)          */
    double *beta_out;          /* device, downlink normalisation, or NULL    */
} dbp_graph_item;

/* Capture items[0..n-1] into a graph (branches: 0 = 4, at most 16).
 * Validates every item first (DBP_ERR_INVALID_ARG / UNSUPPORTED name the
 * first bad item in dbp_last_error); DBP_ERR_NOMEM if its scratch cannot be
 * allocated; DBP_ERR_CUDA if capture or instantiation fails.  The graph
 * holds the handle: destroy graphs before the handle. */
dbp_status dbp_graph_create(dbp_handle_t h, const dbp_graph_item *items, int32_t n, int32_t branches,
                            dbp_graph_t *out);

/* Enqueue one run of every frame of the graph on `stream` (NULL: the
 * default stream).  Stream-ordered like the single-frame calls. */
dbp_status dbp_graph_launch(dbp_graph_t g, void *stream);

/* Release the graph (waits for its launches to finish). */
dbp_status dbp_graph_destroy(dbp_graph_t g);

/* ------------------------------------------------------------------------
 * Test hook of the bounded device waits (the paper has no counterpart).
 * Every wait of a kernel on its input copies is bounded: it gives up after a
 * limit, raises a device status bit and the kernel returns normally, and the
 * host reports DBP_ERR_TIMEOUT (dbp_device_status, the host-buffer variants).
 * With DBP_TEST_STARVE_COPY set, later calls on the handle arm every input
 * copy's mbarrier with 16 bytes more than the copy delivers, so the barrier
 * never completes, and use a wait limit of about 1 ms: the waits run out
 * without any fault, the kernels return and their outputs are unspecified.
 * dbp_set_test_faults(h, 0) restores normal operation.
 * ------------------------------------------------------------------------ */
#define DBP_TEST_STARVE_COPY 1u
dbp_status dbp_set_test_faults(dbp_handle_t h, uint32_t flags);

/* Largest subcarrier count W accepted by dbp_downlink_admm_static. */
#define DBP_STATIC_MAX_SUBCARRIERS 16384

/* Downlink beamforming with power normalisation that allocates no device
 * memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- processes whose device memory is
 * entirely reserved by another allocator, and real-time front ends that
 * must not allocate once they are running.  dbp_downlink_admm with
 * DBP_FLAG_NORMALIZE allocates a small accumulator on its first use; this
 * call instead keeps its scratch (one partial energy per subcarrier, plus
 * the frame total and beta) in a fixed library-owned device array of
 * DBP_STATIC_MAX_SUBCARRIERS + 2 doubles that every GPU which loads the
 * library holds until the process exits.  It never runs the separate
 * operator kernel (whose buffer comes from a pool).
 * Same arguments and results as dbp_downlink_admm: x is scaled in place by
 * beta = sqrt(B*W*N / sum|x|^2) when DBP_FLAG_NORMALIZE is set (the sum is
 * taken per subcarrier and then over subcarriers in a fixed order, so beta
 * does not depend on scheduling), and beta is stored at beta_out (device)
 * if non-NULL.  The caller still passes every input and output buffer.
 * Errors: DBP_ERR_UNSUPPORTED when W > DBP_STATIC_MAX_SUBCARRIERS (no work
 * is enqueued); DBP_ERR_CUDA, without enqueueing anything, when a CUDA error
 * from earlier work is still pending; otherwise as dbp_downlink_admm.  Every
 * error leaves its text in dbp_last_error.
 * Set-up: the first call on each device (with that device current) looks
 * up the array's device address (a CUDA runtime query) and keeps it for the
 * life of the process; do not use the entry point after cudaDeviceReset.  Every call reuses the same array: two calls
 * whose work overlaps on the GPU (different streams, or different host
 * threads) race on it and must be serialised by the caller.  Each call
 * overwrites every scratch entry it reads, so nothing has to be cleared
 * between calls. */
dbp_status dbp_downlink_admm_static(dbp_handle_t h, const dbp_frame_desc *d,
                                    const void *H, const void *s, void *x,
                                    double *beta_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DBP_H */
