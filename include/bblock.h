/*
 * bblock.h -- C ABI of the GB300 (sm_103a) stochastic-LapH baryon-block library.
 *
 * What it computes (arXiv:2211.16278, Sec. 2): for each time slice t and each
 * momentum p,
 *
 *   q_i[alpha][x][a][d] = sum_l V[l][x][a] * phi_i[alpha*n_ev + l][d]            (Eq. 2)
 *   B[t][p][d1][d2][d3] = sum_s c_s^{(p)} sum_x e^{-i p.x} eps_{abc}
 *                         q1[alpha_s][x][a][d1] q2[beta_s][x][b][d2] q3[gamma_s][x][c][d3]
 *                                                                                  (Eq. 1/3)
 *
 * with p = 2 pi n / L for integer triples n, sites x = x0 + L*(x1 + L*x2) in
 * [0, L)^3, eps_{012} = +1 and no complex conjugation. The spin sum over
 * (alpha_s, beta_s, gamma_s, c_s) is the caller-supplied baryon operator of
 * Eq. (1); with a single triple and c = 1 the call is the kernel of Eq. (3).
 *
 * Complex numbers are interleaved (re, im) IEEE doubles ("complex128").
 * Arrays are dense, row-major, with the last index fastest:
 *   V      complex128 [n_t][n_ev][L^3][3]            eigenvector l, site x, colour a
 *   phi_i  complex128 [n_t][4*n_ev][nd_i]            row alpha*n_ev + l, column d
 *   B_out  complex128 [n_t][n_mom][nd1][nd2][nd3]
 *   momenta     int32 [n_mom][3]                     host memory, any sign
 *   spin_idx    int32 [n_spin][3]                    host memory, entries in 0..3
 *   spin_coeffs complex128 [n_spin] (coeff_per_mom == 0) or [n_mom][n_spin] (!= 0), host memory
 *
 * Ownership: the caller owns every argument buffer; the library never frees
 * them and keeps no pointer to them after a call returns. A context owns its
 * device workspace (reconstructed fields, phase table, per-slab partial sums)
 * and the host staging buffers of bblock_compute_host; bblock_destroy releases
 * them. A context is not thread-safe; use one context per host thread and
 * stream, or serialise calls.
 *
 * Errors: every int-returning entry point returns BBLOCK_OK (0) or one of the
 * negative codes below and never throws. bblock_last_error() gives a one-line
 * message. Kernel launches are asynchronous: errors the device detects show up
 * in bblock_status(), which synchronises the stream of the last call.
 */
#ifndef BBLOCK_H
#define BBLOCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BBLOCK_OK 0
#define BBLOCK_ERR_INVALID_ARG (-1)  /* bad size, index, pointer kind or alignment */
#define BBLOCK_ERR_UNSUPPORTED (-2)  /* valid request this build does not implement */
#define BBLOCK_ERR_OOM (-3)          /* device or pinned-host allocation failed */
#define BBLOCK_ERR_CUDA (-4)         /* a CUDA runtime call failed */
#define BBLOCK_ERR_TIMEOUT (-5)      /* a bounded device wait gave up */
#define BBLOCK_ERR_DEVICE_FLAG (-6)  /* a kernel flagged an inconsistent job table */
#define BBLOCK_ERR_TOO_LARGE (-7)    /* request exceeds the fixed scratch of bblock_contract_noalloc */

/* Arithmetic of the projection and the contraction. */
typedef enum {
  BBLOCK_FP64 = 0,       /* IEEE double throughout (DFMA); parity target 1e-12 */
  BBLOCK_TF32X3 = 1,     /* contraction on the tensor cores in a TF32 split (hi/lo, 3
                            products), FP32 accumulate; projection in FP32 FMA (or on the
                            tensor cores, BBLOCK_OPT_TC_PROJECTION); parity target 1e-6 */
  BBLOCK_BF16_SPLIT = 2, /* as BBLOCK_TF32X3 with a BF16 split (3, 6 or 9 products);
                            parity target 1e-6 with 6 or 9 products */
  BBLOCK_DF64 = 3,       /* projection and contraction in double-float arithmetic (pairs
                            of FP32, about 48 significant bits) on the FP32 pipe; FP64 only
                            for the input conversion, the phases and the slab reduction;
                            parity target 1e-12 */
  BBLOCK_FP16X3 = 4,     /* contraction on the tensor cores with FP16 operands split in two
                            (hi = rn16(v), lo = rn16(v - hi), about 22 bits), 3 products
                            (hi hi, hi lo, lo hi), FP32 accumulate; the operands are scaled
                            by powers of two chosen per job from the largest field entry of
                            each quark line, so FP16's range never overflows, and the FP64
                            slab reduction removes the scale exactly; projection in FP32 FMA;
                            parity target 1e-6 */
  BBLOCK_OZAKI = 5       /* FP64-accurate contraction on the BF16 tensor cores (Ozaki scheme):
                            the double-float projection's diquark and phase-folded third
                            quark, scaled by powers of two per row and column of each site
                            slab, split into 7 BF16 digits of 8 bits; the 28 digit products
                            down to 2^-56 of the scales are summed exactly (levels 0-3, one
                            FP32 accumulator each, drained every 240 K elements) or to FP32
                            rounding (levels 4-6) into double-float running sums; FP64 slab
                            reduction; parity target 1e-12 */
} bblock_precision;

typedef struct bblock_ctx bblock_ctx;

typedef struct {
  int L;             /* lattice extent; X = L^3 sites per time slice; 1 <= L <= 128 */
  int n_ev;          /* Laplacian eigenvectors; 1 <= n_ev <= 3 L^3 */
  int max_ndil;      /* bound on every nd_i passed later; 1 <= max_ndil <= 256 */
  int precision;     /* a bblock_precision value */
  int bf16_products; /* BBLOCK_BF16_SPLIT: 3, 6 or 9 split products; ignored otherwise */
  int device;        /* CUDA device ordinal the context runs on */
} bblock_config;

/* Create a context for one device. *out is set on success, NULL otherwise.
 * No device memory is reserved until the first compute call. */
int bblock_create(bblock_ctx** out, const bblock_config* cfg);

/* Release the context and everything it owns. Waits for its pending work. NULL is a no-op. */
void bblock_destroy(bblock_ctx* ctx);

/* One-line description of the last error on this context ("" if none). Valid until the next call. */
const char* bblock_last_error(const bblock_ctx* ctx);

/* Synchronise the stream of the last call and report device-side status:
 * BBLOCK_OK, BBLOCK_ERR_CUDA (a launch or kernel failed), BBLOCK_ERR_TIMEOUT (a bounded
 * device wait gave up; the kernel stopped early and its blocks are invalid) or
 * BBLOCK_ERR_DEVICE_FLAG (an inconsistent job table, or an index violation found by the
 * checked kernel variant). The status word is cleared once reported, so the context stays
 * usable for the next call. */
int bblock_status(bblock_ctx* ctx);

/* Baryon blocks of n_t time slices and one noise triple (Eq. 2 then Eq. 1).
 *   V, phi1, phi2, phi3, B_out: DEVICE pointers (cudaMalloc or managed), 16-byte aligned,
 *     layouts as in the file comment; V and phi_i hold n_t consecutive time slices.
 *   nd1, nd2, nd3: dilution sizes, 1..max_ndil.
 *   n_mom >= 0 momenta (n_mom == 0 or n_t == 0 is a no-op); n_spin >= 1 spin triples.
 *   coeff_per_mom: 0 -> spin_coeffs is [n_spin]; 1 -> [n_mom][n_spin] (Eq. 1's c depends on p).
 *   stream: a cudaStream_t (NULL = legacy default stream). Work is enqueued, not awaited.
 * The momentum phases are cached in the context per (L, momentum list). */
int bblock_compute(bblock_ctx* ctx, int n_t, const void* V, const void* phi1, const void* phi2,
                   const void* phi3, int nd1, int nd2, int nd3, const int32_t* momenta,
                   int n_mom, const int32_t* spin_idx, const double* spin_coeffs, int n_spin,
                   int coeff_per_mom, void* B_out, void* stream);

/* Same computation from HOST buffers: copies V and phi_i to context-owned device
 * buffers, computes on `stream`, copies B back into the host buffer B_out and
 * synchronises before returning. The time slices move in up to 8 chunks on a
 * context-owned copy stream, so that the copies of one chunk overlap the
 * computation of another (the slices are independent). Page-locked host memory
 * (cudaHostAlloc / pin_memory) gives full copy bandwidth and overlap; pageable
 * memory works. */
int bblock_compute_host(bblock_ctx* ctx, int n_t, const void* V, const void* phi1,
                        const void* phi2, const void* phi3, int nd1, int nd2, int nd3,
                        const int32_t* momenta, int n_mom, const int32_t* spin_idx,
                        const double* spin_coeffs, int n_spin, int coeff_per_mom, void* B_out,
                        void* stream);

/* One unit of a batched run: one time slice of one noise triple.
 * All pointers are device pointers with the single-slice layouts above
 * (V [n_ev][L^3][3], phi_i [4*n_ev][nd_i], B_out [n_mom][nd1][nd2][nd3]). */
typedef struct {
  const void* V;
  const void* phi1;
  const void* phi2;
  const void* phi3;
  int nd1, nd2, nd3;
  void* B_out;
} bblock_job;

/* Every job of a run (time slices x noise triples, dilution sizes may differ per
 * job) in one pass: one projection launch, one persistent contraction launch
 * and one reduction launch for all jobs, sharing the momenta and spin operator
 * (Sec. 2: the kernel is called for many noise and spin combinations with the
 * same momentum set and eigenvectors). Arguments as in bblock_compute. */
int bblock_compute_batch(bblock_ctx* ctx, const bblock_job* jobs, int n_jobs,
                         const int32_t* momenta, int n_mom, const int32_t* spin_idx,
                         const double* spin_coeffs, int n_spin, int coeff_per_mom, void* stream);

/* ---------------------------------------------------------------- mode-triplet ordering
 * Eq. (3) can be evaluated in two steps through the eigenvector mode triplet of Eq. (4)
 * (Sec. 2): T does not depend on the noise, dilution or spin, so one T per time slice
 * serves every noise triple and spin operator of a run.
 *
 * bblock_mode_triplet: T[t][p][l1][l2][l3] = sum_x e^{-i p.x} eps_abc V[l1][x][a]
 * V[l2][x][b] V[l3][x][c] for every time slice, computed by the context's form (it is the
 * contraction with identity coefficients). V as in bblock_compute (device); T_out device,
 * complex128 [n_t][n_mom][n_ev][n_ev][n_ev], l3 fastest, caller-owned. Requires
 * max_ndil >= n_ev (BBLOCK_ERR_INVALID_ARG otherwise). Asynchronous on `stream`. */
int bblock_mode_triplet(bblock_ctx* ctx, int n_t, const void* V, const int32_t* momenta,
                        int n_mom, void* T_out, void* stream);

/* bblock_from_triplet: B[t][p][d1][d2][d3] = sum_s c_s sum_{l1 l2 l3} T[t][p][l1][l2][l3]
 * phi1[t][alpha_s n_ev + l1][d1] phi2[t][beta_s n_ev + l2][d2] phi3[t][gamma_s n_ev + l3][d3]
 * as three batched complex mode products in FP64 (per time slice and (alpha, beta) pair:
 * T x3 folded phi3, then x2 phi2, then x1 phi1). T as written by bblock_mode_triplet; phi_i,
 * B_out, spins and coefficients as in bblock_compute (device buffers; the momenta
 * themselves are not needed, only their number). Asynchronous on `stream`. */
int bblock_from_triplet(bblock_ctx* ctx, int n_t, const void* T, const void* phi1,
                        const void* phi2, const void* phi3, int nd1, int nd2, int nd3,
                        int n_mom, const int32_t* spin_idx, const double* spin_coeffs,
                        int n_spin, int coeff_per_mom, void* B_out, void* stream);

/* Device bytes the context holds right now (workspace + caches). */
size_t bblock_workspace_bytes(const bblock_ctx* ctx);

/* Number of kernel launches enqueued by the last compute call. */
int bblock_last_launch_count(const bblock_ctx* ctx);

/* Contraction path of the last compute call (for reporting executed work; the blocks do
 * not depend on it beyond rounding): the FP64 or double-float kernels; the tensor-core
 * kernel with N tiles over (p, d3) columns, plain, as clusters sharing the diquark tile, or
 * as CTA pairs sharing the third-quark tile; or the row-factored phase (N tiles over
 * (distinct n0, d3), BBLOCK_OPT_TC_ROWS). -1 before any call or for a NULL context. */
#define BBLOCK_PATH_FP64 0
#define BBLOCK_PATH_TC 1
#define BBLOCK_PATH_TC_CLUSTER 2
#define BBLOCK_PATH_TC_PAIRS 3
#define BBLOCK_PATH_TC_ROWS 4
#define BBLOCK_PATH_TC_ROWS_CLUSTER 5   /* row-factored, clusters of 2 sharing each diquark tile */
#define BBLOCK_PATH_OZAKI 6             /* the BBLOCK_OZAKI contraction */
int bblock_last_path(const bblock_ctx* ctx);

/* Number of waves the last compute call ran its jobs in: jobs are taken in list order, and
 * a wave holds as many as the workspace budget (BBLOCK_OPT_WAVE_MB) allows. 0 for a call
 * with no work or a NULL context. */
int bblock_last_wave_count(const bblock_ctx* ctx);

/* Options of a context (bblock_set_option). The tuning options are the search space of
 * the tile autotuner; 0 means "chosen automatically". */
#define BBLOCK_OPT_GRAPHS 1    /* 1 (default): a call repeated with identical arguments on a
                                  created stream (not the legacy or per-thread default
                                  stream) is captured as a CUDA graph on its second
                                  occurrence and replayed afterwards; 0: plain launches */
#define BBLOCK_OPT_TC_NC 2     /* tensor-core forms: complex columns per tile, 16, 32 or 48;
                                  the FP16 form's CTA pairs also take 64 or 80 */
#define BBLOCK_OPT_TC_CHUNK 3  /* tensor-core forms: stages between accumulator drains, 1..8
                                  (default 2). Longer intervals are faster and less accurate:
                                  the accumulator's rounding drift grows with the MMAs it
                                  collects; the autotuner tries up to 3 (up to 2 in the FP16
                                  form) */
#define BBLOCK_OPT_SLABS 4     /* site slabs per job (split of the site sum), 1..4096 */
#define BBLOCK_OPT_CHECKS 5    /* 1: the tensor-core contraction checks every global index
                                  against its buffer, skips and records violations, and in
                                  every form a 256-byte canary follows each workspace block
                                  (fields, converted inputs, partial blocks), filled before
                                  and verified after each wave; violations and overwritten
                                  canaries are reported by bblock_status
                                  (BBLOCK_ERR_DEVICE_FLAG); 0 (default): no checks */
#define BBLOCK_OPT_WAIT_LIMIT_US 7  /* test hook: limit of the tensor-core contraction's
                                       bounded waits in microseconds (0: the default of about
                                       2 s); a wait that runs out sets the status word, which
                                       bblock_status reports as BBLOCK_ERR_TIMEOUT */
#define BBLOCK_OPT_FAIL_NEXT_ALLOC 8 /* test hook: 1 makes the next device allocation of the
                                       context fail as if the device were out of memory
                                       (BBLOCK_ERR_OOM), once */
#define BBLOCK_OPT_TC_CLUSTER 10  /* BF16 tensor-core forms: CTAs of a thread-block cluster
                                       sharing each 128-pair diquark tile, 2, 4 or 8 (each
                                       builds 1/C of it and takes its own N tile; results are
                                       bitwise those of the plain kernel with the same tiles);
                                       0 (default) or 1: no clusters. FP16 form: 1 runs plain
                                       CTAs with N tiles of up to 48 columns; any other value
                                       (the default) runs CTA pairs that share the third-quark
                                       tile of an N tile of up to 80 columns and take adjacent
                                       128-pair tiles. With the row-factored phase
                                       (BBLOCK_OPT_TC_ROWS): 2, or 0 when every job of a wave
                                       has at least two d3 tiles, runs clusters that share each
                                       diquark tile and take adjacent d3 tiles; 1 plain CTAs.
                                       Index checks and the wait-limit test hook use no
                                       clusters. BBLOCK_OZAKI: 1, 2, 3 or 4 CTAs sharing each
                                       diquark tile across adjacent N tiles (results bitwise
                                       those of 1); 0 (default): 2 unless the ragged last
                                       clusters pad the N tiles by more than 20 %, else 1 */
#define BBLOCK_OPT_CORRUPT_CANARY 9  /* test hook (with BBLOCK_OPT_CHECKS): 1 makes the next
                                       call overwrite its first canary from the host, in
                                       stream order between the fill and the check, once */
#define BBLOCK_OPT_TC_ROWS 13  /* FP16 form: the momentum phase factorised along the lattice,
                                  e^{-i p.x} = w^{n0 x0} w^{n1 x1 + n2 x2} with w = e^{-2 pi i/L}:
                                  the tensor cores sum each lattice row (fixed x1, x2) against
                                  the third quark times w^{n0 x0} for each distinct n0 of the
                                  momenta, and the row's sums are multiplied by
                                  w^{n1 x1 + n2 x2} into one running sum per momentum. 0
                                  (default): where it pays (at least twice as many momenta as
                                  distinct n0) and the running sums fit TMEM; 1: wherever they
                                  fit; 2: never (CTA pairs over all (p, d3) columns). With it,
                                  BBLOCK_OPT_TC_NC sets the d3 columns per tile. Not with
                                  index checks, per-momentum coefficients or the wait-limit
                                  test hook */
#define BBLOCK_OPT_TC_PROJECTION 12  /* mixed forms' projection (Eq. 2): 0 (default) on the
                                       tensor cores from pre-tiled operands (V once per
                                       distinct V of a call's wave, and every field's folded
                                       phi, split into three BF16 pieces exact for FP32 and
                                       written in the MMA's layout; staged by bulk copies;
                                       six piece products, the leading one over four
                                       accumulators): as accurate as FP32 FMA and faster;
                                       1: on the tensor cores with operands built per stage in
                                       the form's own split (the FP16 form then uses 2);
                                       2: FP32 FMA. The index checks use the FP32 projection */
#define BBLOCK_OPT_HOST_CHUNKS 11  /* bblock_compute_host: chunks of time slices whose copies
                                       overlap the computation, 1..64 (0, the default: 8). With
                                       1 the blocks equal those of bblock_compute bit for bit;
                                       with more, a chunk may split its sites into other slabs,
                                       which changes the rounding only */
#define BBLOCK_OPT_WAVE_MB 6   /* workspace budget of one wave of jobs, MiB: a batch whose
                                  fields and partial blocks exceed it runs as several waves
                                  of launches; 0 (default): half the device memory free at
                                  bblock_create, at most 96 GiB */

/* Set an option; BBLOCK_ERR_INVALID_ARG for an unknown option or value. */
int bblock_set_option(bblock_ctx* ctx, int option, int value);

/* Current value of an option (>= 0), or BBLOCK_ERR_INVALID_ARG. */
int bblock_get_option(const bblock_ctx* ctx, int option);

/* Per-step timing: while enabled, every step of the path ("project" is the tiling of V
 * and of the fields plus the projection kernel) is bracketed by two CUDA events recorded
 * on the launching stream. */
typedef struct {
  char name[32];    /* "phase", "project", "contract", "reduce", ... */
  int launches;     /* kernel launches of the steps timed since the last read */
  double total_ms;  /* summed event-to-event durations of those steps */
} bblock_kernel_stat;

/* Turn launch timing on (enable != 0) or off. Off by default. Every kernel launch is
 * bracketed by CUDA events on the launching stream. A call captured into a CUDA graph while
 * timing is on carries those events as event-record nodes, so graph replays are timed per
 * launch as well (each replay's times are read before the next replay starts, which waits
 * for the previous replay to finish). Turning timing on or off changes the call signature:
 * the next two identical calls run plainly and then capture a new graph. */
int bblock_profile_enable(bblock_ctx* ctx, int enable);

/* Synchronise the recorded events, write up to max_entries per-kernel totals to
 * out (one entry per kernel name that launched), set *n_entries, and reset. */
int bblock_profile_read(bblock_ctx* ctx, bblock_kernel_stat* out, int max_entries,
                        int* n_entries);

/* ---------------------------------------------------------------- tile autotuner
 * Not in the paper, whose block sizes are tuned by hand for a CPU cache hierarchy
 * (Sec. 4); here the tile options of a context are chosen by timing candidates on the
 * caller's own inputs. A learned cost model (a small MLP trained on the GPU by this
 * library's own kernels) can rank the candidates so that only the top few are timed. */

#define BBLOCK_TUNE_FEATURES 12

typedef struct bblock_costmodel bblock_costmodel;

typedef struct {
  int nc, chunk, slabs;      /* option values of the candidate (0 = automatic) */
  float features[BBLOCK_TUNE_FEATURES];  /* cost-model input of the candidate */
  float predicted;           /* model prediction of log(ms), 0 without a model */
  double ms;                 /* median time of one compute call, -1 if not timed */
} bblock_tune_entry;

/* Time the tile candidates of the context's precision on one bblock_compute workload
 * (same arguments as bblock_compute; B_out is overwritten) and keep the fastest as the
 * context's options. With a model, all candidates are ranked by predicted time and only
 * the top_k are timed; without one (model == NULL) every candidate is timed. Each timed
 * candidate runs once untimed and `repeats` times timed with CUDA events on `stream`.
 * Up to max_report entries (all candidates, timed or not) go to report; *n_report is set.
 * Synchronises the stream. */
int bblock_autotune(bblock_ctx* ctx, int n_t, const void* V, const void* phi1, const void* phi2,
                    const void* phi3, int nd1, int nd2, int nd3, const int32_t* momenta,
                    int n_mom, const int32_t* spin_idx, const double* spin_coeffs, int n_spin,
                    void* B_out, void* stream, bblock_costmodel* model, int top_k, int repeats,
                    bblock_tune_entry* report, int max_report, int* n_report);

/* Cost model: MLP with two tanh hidden layers of `hidden` units (<= 64), n_features
 * (<= 16) inputs and one output, deterministic initial weights from `seed`. */
int bblock_costmodel_create(bblock_costmodel** out, int n_features, int hidden, uint64_t seed,
                            int device);
void bblock_costmodel_destroy(bblock_costmodel* model);
int bblock_costmodel_num_params(const bblock_costmodel* model);
/* Parameters as FP32, order W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3 (host buffers). */
int bblock_costmodel_get_params(bblock_costmodel* model, float* out, int n);
/* Replace the parameters and reset the optimiser state. */
int bblock_costmodel_set_params(bblock_costmodel* model, const float* in, int n);
/* Mean-squared-error loss and its gradient with respect to the parameters over n samples
 * X [n][F], y [n] (host buffers), computed by the forward and backward kernels on the GPU. */
int bblock_costmodel_gradient(bblock_costmodel* model, const float* X, const float* y, int n,
                              float* loss, float* grad);
/* `epochs` full-batch Adam steps (learning rate lr) on the GPU; *final_loss = last loss. */
int bblock_costmodel_train(bblock_costmodel* model, const float* X, const float* y, int n,
                           int epochs, float lr, float* final_loss);
/* Predictions y [n] for X [n][F] (host buffers). */
int bblock_costmodel_predict(bblock_costmodel* model, const float* X, int n, float* y);

/* ---------------------------------------------------------------- FP64 throughput probe
 * Not in the paper. Measures the two FP64 paths of `device`: scalar fused multiply-adds
 * (DFMA, which the FP64 form's kernels use) and the FP64 tensor-core MMA (mma.sync
 * m8n8k4 f64), each as the best of three timed launches of register-resident loops over
 * every SM, in TFLOP/s (2 flops per FMA). The FP64 form's roofline takes the measured DFMA
 * rate as its peak. Allocates 16 bytes of device memory and two events for the duration of
 * the call; synchronises `stream`. Returns BBLOCK_ERR_INVALID_ARG (bad device or NULL
 * outputs) or BBLOCK_ERR_CUDA. */
int bblock_probe_fp64(int device, double* dfma_tflops, double* dmma_tflops, void* stream);

/* Size of the fixed device scratch used by bblock_contract_noalloc (32 MiB). */
#define BBLOCK_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* Allocation-free contraction. The paper has no counterpart: this entry point exists
 * for callers that must not allocate device memory, such as applications whose memory
 * manager has reserved the device's memory up front (a pooled allocator of a larger
 * code, or solver fields that fill HBM), or hot loops that forbid cudaMalloc/cudaFree
 * because those calls synchronise the whole device.
 *
 * It computes the same blocks as bblock_compute for one time slice, but from fields that
 * are already reconstructed, and needs no context:
 *   q1, q2, q3  complex128 [4][L^3][3][nd_i], device memory of the CURRENT device: the
 *               reconstructed field of quark line i, indexed [spin][site][colour][dilution
 *               index], last index fastest (the fields bblock_compute builds internally
 *               from V and phi_i); spins a caller does not use may hold anything, they are
 *               not read;
 *   B_out       complex128 [n_mom][nd1][nd2][nd3], device memory of the current device;
 *   momenta, spin_idx, spin_coeffs: host arrays as for bblock_compute, with one
 *               coefficient per spin triple (no per-momentum coefficients);
 *   stream      the cudaStream_t the two kernels are enqueued on (not awaited);
 *   err         optional host buffer of err_len bytes for a one-line message.
 * Limits: n_mom <= 8 and n_mom*nd1*nd2*nd3*16 <= BBLOCK_NOALLOC_SCRATCH_BYTES; larger
 * requests return BBLOCK_ERR_TOO_LARGE without launching anything.
 * The per-slab partial sums live in one file-scope device array of
 * BBLOCK_NOALLOC_SCRATCH_BYTES that every device loading the library holds until the
 * process exits. It calls no cudaMalloc, cudaFree or other allocating routine. The
 * first call on a device looks up that array's device address (cudaGetSymbolAddress,
 * with the device current); make that first call before any stream capture. The address
 * is kept per device and CUDA context: after a cudaDeviceReset the next call looks it up
 * again in the new context (make that call, too, before any capture). All calls
 * share the one array and every call overwrites the part it reads, so calls that overlap
 * on the GPU (different streams or host threads without ordering between them) race and
 * must be serialised by the caller. */
int bblock_contract_noalloc(int L, const void* q1, const void* q2, const void* q3, int nd1,
                            int nd2, int nd3, const int32_t* momenta, int n_mom,
                            const int32_t* spin_idx, const double* spin_coeffs, int n_spin,
                            void* B_out, void* stream, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* BBLOCK_H */
