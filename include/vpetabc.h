/*
 * vpetabc — voxelwise ABC rejection for dynamic PET kinetic modelling on one
 * NVIDIA B300 (sm_103a).  C ABI of libvpetabc.so.
 *
 * The library runs the data-parallel hot path of vPET-ABC (Algorithm 1 of the
 * paper): prior draws -> simulated frame-mean TACs -> frame-weighted squared
 * Euclidean discrepancy to every voxel TAC -> the k nearest draws per voxel ->
 * posterior model probabilities and posterior summaries.
 *
 * Conventions shared by every entry point
 *  - Time is in minutes, rate constants in 1/min.
 *  - `_dev` pointers are CUDA device memory owned by the caller; `_host`
 *    pointers (and structs) are host memory read before the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is enqueued on it asynchronously; host pointers are not
 *    retained after return.
 *  - Matrices are row-major with an explicit leading dimension (elements).
 *  - Return value: ABC_OK (0) or a negative ABC_ERR_* code.  On error nothing
 *    is enqueued, and abc_last_error() (thread-local) describes the cause.
 *  - The library never allocates device memory on these paths: scratch comes
 *    from the caller's `workspace`.
 */
#ifndef VPETABC_H
#define VPETABC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ABC_OK 0
#define ABC_ERR_ARG (-1)         /* invalid argument (null, size, alignment, range) */
#define ABC_ERR_CUDA (-2)        /* a CUDA runtime/driver call failed */
#define ABC_ERR_WORKSPACE (-3)   /* workspace too small or misaligned */
#define ABC_ERR_TIMEOUT (-4)     /* a bounded device wait ran out (reported by abc_topk_status) */
#define ABC_ERR_UNSUPPORTED (-5) /* shape outside what the kernels support (e.g. L > 61) */

/* Kinetic models (Sec. II-A).  Parameter order of a draw row (theta):
 *  ABC_2TCM_IRR: K1, k2, k3, Vb            (Eq. 1-2 with k4 = 0)
 *  ABC_2TCM_REV: K1, k2, k3, k4, Vb        (Eq. 1-2)
 *  ABC_MRTM:     R1, k2, BPnd              (Eq. 3 with gamma = 0; k2a = k2/(1+BPnd))
 *  ABC_LPNTPET:  R1, k2, BPnd, gamma, tD, tP - tD, alpha   (Eq. 3-4)
 * 2TCM models take the plasma input C_p (= C_wb for FDG, Sec. II-A); MRTM and
 * lp-ntPET take the reference-region TAC C_r. */
#define ABC_2TCM_IRR 0
#define ABC_2TCM_REV 1
#define ABC_MRTM 2
#define ABC_LPNTPET 3

/* Precision of the tensor-core discrepancy (Sec. II-C distance, Alg. 1 step 4).
 * Every form returns the exact fp32 top-k: the k draws of smallest fp32 re-scored
 * distance, ties to the lower draw index.  They differ in how the tensor cores rank.
 *  ABC_BF16_RESCORE: the fast form.  bf16 operands, fp32 accumulate: the voxel row
 *                    rounded once, the draw row as bf16 hi + lo (two bf16 products
 *                    per term) with its rounding residual folded into the draw's
 *                    norm column, so that a key's error is at most
 *                    2 sqrt(d) (||delta|| + 2^-16 ||x||) plus fp32 accumulation
 *                    (delta = the voxel row's rounding).  The finest pilot pass sets
 *                    each voxel's threshold from that bound and its rank-rk pilot key,
 *                    so the candidate list (the net) holds every draw the certificate
 *                    can need; the net is re-scored exactly in fp32, the k-th
 *                    distance d_k found, and the result certified (no draw outside the
 *                    net can have distance <= d_k).  An uncertified voxel is resolved by
 *                    an exact fp32 scan of all draws (counted by abc_topk_status).
 *  ABC_SPLIT_DRAWS:  the same computation as ABC_BF16_RESCORE (the name of the
 *                    operand layout it uses).
 *  ABC_FP32:         both operands split into bf16 hi + lo pairs (three bf16
 *                    products per term); each voxel keeps its 2k nearest by that
 *                    key, re-scores them exactly in fp32 and certifies from the
 *                    product error bound; an uncertified voxel is resolved by an
 *                    exact fp32 scan. */
#define ABC_FP32 0
#define ABC_BF16_RESCORE 1
#define ABC_SPLIT_DRAWS 2

/* Contiguous or gapped frame schedule: frame l spans [t_start[l], t_end[l]). */
typedef struct {
    int32_t L;
    const double* t_start;
    const double* t_end;
} abc_frames;

/* Input function sum_i (a0[i] + a1[i] t + a2[i] t^2) exp(-c[i] t), c[i] >= 0. */
typedef struct {
    int32_t n_terms;       /* 1 .. 16 */
    const double* c;
    const double* a0;
    const double* a1;
    const double* a2;
} abc_polyexp;

/* Feng's three-exponential plasma input (Sec. III-A):
 * C_a(t) = (beta1 t - beta2 - beta3) e^{-kappa1 t} + beta2 e^{-kappa2 t} + beta3 e^{-kappa3 t},
 * written into three poly-exponential terms (c, a0, a1, a2 each of length 3). */
int abc_feng_input(const double beta[3], const double kappa[3], double c[3], double a0[3], double a1[3],
                   double a2[3]);

/* Prior draws (Algorithm 1, steps 1-2; uniform priors of Sec. III-A).
 * Writes theta_dev[n * ldtheta + p] for n in [0, N), p in [0, P) with
 * theta = fl32(lo[p] + (hi[p] - lo[p]) * u) evaluated in fp64, where u is the
 * top 24 bits of word (p % 4) of Philox4x32-10 at counter
 * (first_index + n [lo 32, hi 32 bits], model, p / 4) and key (seed lo, seed hi).
 * The stream is reproducible from (seed, model, global draw index).
 * lo/hi: host, P entries, lo <= hi.  P in 1..8, ldtheta >= P. */
int abc_sample_prior(uint64_t seed, int32_t model, const double* lo_host, const double* hi_host, int32_t P,
                     int64_t N, int64_t first_index, float* theta_dev, int32_t ldtheta, void* stream);

/* Simulated frame-mean TACs (Algorithm 1, step 3):
 * x_dev[n * ldx + l] = (1 / dt_l) * integral over frame l of C_t(t) for draw n,
 * C_t from Eq. 1-2 (2TCM, closed-form convolution with `input` = C_p),
 * Eq. 3 with gamma = 0 (MRTM, closed form, `input` = C_r), or Eq. 3-4
 * (lp-ntPET: closed form up to t_D, exponential integrator after it).
 * Columns l >= L of each row are left untouched.
 * theta_dev: N x ldtheta fp32 (layout above).  L in 1..64, ldx >= L. */
int abc_simulate(int32_t model, const abc_frames* frames_host, const abc_polyexp* input_host,
                 const float* theta_dev, int64_t N, int32_t ldtheta, float* x_dev, int32_t ldx, void* stream);

/* Bytes of device workspace abc_discrepancy_topk needs for these sizes. */
size_t abc_workspace_size(int64_t J, int64_t N, int32_t L, int32_t k, int32_t precision);

/* Discrepancy and top-k (Algorithm 1, steps 4-5; fixed-budget rejection,
 * Sec. II-C).  For every voxel j in [0, J) finds the k draws n in [0, N)
 * with the smallest d_jn = sum_l w_l (y_jl - x_nl)^2 and writes them sorted
 * ascending by (d, n):
 *   idx_dev[j * k + r]  = n       (global draw index, int32)
 *   dist_dev[j * k + r] = d_jn    (fp32, computed directly from y and x)
 * y_dev: J x ldy fp32 voxel TACs; x_dev: N x ldx fp32 simulated TACs;
 * w_host: L frame weights >= 0 (not all zero); 1 <= k <= min(N, 2048);
 * 1 <= L <= 61; N < 2^31.  ldx and ldy are multiples of 4 and the pointers
 * 16-byte aligned.  workspace: >= abc_workspace_size(...) bytes, 256-byte
 * aligned, device memory; its contents on entry do not matter.
 * The voxel-by-draw distance matrix is never formed in memory. */
int abc_discrepancy_topk(const float* y_dev, int64_t J, int32_t ldy, const float* x_dev, int64_t N, int32_t ldx,
                         int32_t L, const float* w_host, int32_t k, int32_t precision, void* workspace,
                         size_t ws_bytes, int32_t* idx_dev, float* dist_dev, void* stream);

/* Launch choices of the fused tensor-core kernel (picked by the project's
 * autotuner; abc_default_tuning gives the values used when none is passed).
 *  bn:           draws per tile and TMEM accumulator width, 64 or 128;
 *  ctas_per_sm:  persistent CTAs launched per SM (1..4, capped by occupancy);
 *  pilot_stride: draw stride between pilot levels, 8, 16 or 32;
 *  pilot_factor: candidates a pilot threshold aims to admit, as a multiple of
 *                the net size at the next finer level (1.25 .. 4). */
typedef struct {
    int32_t bn;
    int32_t ctas_per_sm;
    int32_t pilot_stride;
    float pilot_factor;
} abc_tuning;

/* The tuning used for `precision` when none is passed: the built-in choice
 * (128-draw tiles and 2 CTAs/SM; pilot stride 8 and factor 2.25 for ABC_FP32,
 * pilot stride 8 and factor 1.5 otherwise, where a single-scan call with
 * k >= 400 uses pilot stride 16) unless abc_set_default_tuning replaced it.
 * This call reports the choice for a batch (no single-scan adjustment). */
int abc_default_tuning(int32_t precision, abc_tuning* out);

/* Replaces the process-wide default tuning for both precisions (NULL restores
 * the built-in ones).  Results never depend on the tuning; only speed does. */
int abc_set_default_tuning(const abc_tuning* tuning);

/* One scan (volume or ROI set) of a batch: its own voxel TACs, simulated
 * draws, frame count and weights, k and outputs; arguments as in
 * abc_discrepancy_topk. */
typedef struct {
    const float* y_dev;
    int64_t J;
    int32_t ldy;
    const float* x_dev;
    int64_t N;
    int32_t ldx;
    int32_t L;
    const float* w_host;
    int32_t k;
    int32_t* idx_dev;
    float* dist_dev;
} abc_scan;

/* Bytes of workspace abc_batch_discrepancy_topk needs (0 for invalid sizes). */
size_t abc_batch_workspace_size(const abc_scan* scans, int32_t n_scans, int32_t precision);

/* Batched discrepancy + top-k (Alg. 1 steps 4-5 for many scans at once): up to
 * 64 scans with uneven voxel counts, frame schedules and draw counts, each with
 * the same result as its own abc_discrepancy_topk.  All scans share one
 * persistent launch of the fused kernel per pass (pilot levels, main pass),
 * whose CTAs take (scan, 128-voxel tile) work items costliest-scan first; one
 * launch re-scores and sorts every voxel of every scan.  Everything is enqueued
 * on `stream` with no host-to-device copies, so the call can be captured in a
 * CUDA graph and replayed while the buffers stay in place.  tuning may be NULL
 * (default tuning).  Status as for abc_discrepancy_topk (abc_topk_status on
 * this workspace covers the whole batch). */
int abc_batch_discrepancy_topk(const abc_scan* scans, int32_t n_scans, int32_t precision, const abc_tuning* tuning,
                               void* workspace, size_t ws_bytes, void* stream);

/* Allocation-free variant of abc_discrepancy_topk.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory themselves (a host framework that owns the whole device-memory
 * budget, a real-time pipeline that forbids allocation once running, a plugin
 * handed only its input and output buffers).  Same computation, arguments and
 * outputs as abc_discrepancy_topk, but the scratch memory is a fixed 64 MiB
 * device array inside this library (held on every GPU that loads the library
 * until the process exits); the call allocates nothing.
 *  - Sizes whose abc_workspace_size() exceeds 64 MiB are rejected with
 *    ABC_ERR_UNSUPPORTED (e.g. 2,048 voxels x 50,000 draws x 22 frames, k = 100,
 *    fits in either precision).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the one array, which keeps the previous call's contents
 *    (the call clears what must start at zero).  Calls that overlap on the GPU
 *    (concurrent streams, or several host threads) race on it: serialise them.
 *  - Its status words (abc_topk_status's) live in that array: read them with
 *    abc_topk_status_noalloc after the call, before trusting idx_dev / dist_dev
 *    (a bounded device wait that ran out leaves them invalid). */
int abc_discrepancy_topk_noalloc(const float* y_dev, int64_t J, int32_t ldy, const float* x_dev, int64_t N,
                                 int32_t ldx, int32_t L, const float* w_host, int32_t k, int32_t precision,
                                 int32_t* idx_dev, float* dist_dev, void* stream);

/* Status of the last abc_discrepancy_topk_noalloc on the current device, in the
 * layout of abc_topk_status (status_host[0] = ABC_OK or ABC_ERR_TIMEOUT, ...).
 * Blocks on `stream`; like the call itself it allocates nothing.  ABC_ERR_ARG
 * when no abc_discrepancy_topk_noalloc has run on this device yet. */
int abc_topk_status_noalloc(int32_t status_host[8], void* stream);

/* Status of the last abc_discrepancy_topk that used this workspace.  Blocks
 * on `stream`.  Writes
 *   status[0] = ABC_OK or ABC_ERR_TIMEOUT (a bounded device wait ran out; the
 *               outputs are then not valid), or ABC_ERR_UNSUPPORTED (an internal
 *               consistency check of the k-d row order failed; outputs not valid);
 *   status[1] = number of voxels resolved by an exact fp32 scan of all draws
 *               (ABC_FP32 voxels whose tensor-core result could not be
 *               certified, or whose candidate list overflowed; exact results);
 *   status[2] = number of voxels with more candidates tied at the k-th
 *               distance than the final sort holds (the ties kept are then
 *               chosen by a selection on their draw indices: still the lowest);
 *   status[3] = ABC_BF16_RESCORE / ABC_SPLIT_DRAWS voxels whose pilot-sized net
 *               could not be certified (resolved by the exact scan, also
 *               counted in status[1]);
 *   status[4..7] = diagnostics: voxels whose candidate list overflowed, voxels
 *               left with fewer than k / fewer than the net size of candidates,
 *               and (voxel, pilot level) pairs left without a pilot threshold. */
int abc_topk_status(const void* workspace, int32_t status_host[8], void* stream);

/* Work done by the last main pass on this workspace: out_host[0] = draw tiles it
 * processed, out_host[1] = draw tiles a pass without skipping would process, in
 * units of 64 draws whatever the tile width, summed over voxel tiles (both 0
 * when no tile was skipped).  The main pass
 * skips a draw tile when a lower bound on every voxel-draw distance of the two
 * tiles, (F_c(y) - F_c(x))^2 / W_c summed over the three consecutive thirds c
 * of the frames (F_c = sum over the third of w_l v_l, W_c = sum of its w_l; a
 * Cauchy-Schwarz bound on Sec. II-C's distance), exceeds the voxel tile's
 * largest threshold.  Synchronises `stream`. */
int abc_topk_work(const void* workspace, int64_t out_host[2], void* stream);

/* Timing hook: when both are non-NULL (cudaEvent_t passed as void*), every
 * later abc_discrepancy_topk records `start_event` on its stream right before
 * the fused tensor-core kernel and `stop_event` right after it, so a caller can
 * time that kernel alone with cudaEventElapsedTime.  NULL, NULL turns it off.
 * Process-wide setting; the events stay owned by the caller. */
int abc_profile_events(void* start_event, void* stop_event);

/* Test hook for the bounded waits of the fused tensor-core kernel.  Every
 * barrier wait of that kernel gives up after a time limit, flags
 * ABC_ERR_TIMEOUT (abc_topk_status), waits (with the same limit) for the copies
 * and MMAs its CTA has in flight, frees its tensor memory and returns, so the
 * CUDA context stays usable.  This hook makes later calls exercise that path:
 * with withheld_tile >= 0 the TMA producer of every CTA skips the load of its
 * draw tile with that sequence number, so the waits behind it run out; wait_ns
 * (1 ms .. 10 s, or 0 for the 2 s default) replaces the limit.  withheld_tile
 * < 0 turns the stall off.  Process-wide; for tests only. */
int abc_debug_inject_stall(int64_t withheld_tile, uint64_t wait_ns);

/* Test hook for the split form's second pass.  mode is a mask: with bit 1, later calls
 * treat every voxel's first net as uncertified, so voxels are queued for the rescue pass
 * (all of them while the queue holds them: every voxel of a scan of at most 16,384
 * voxels, a quarter otherwise; the rest take the exact fp32 scan); with bit 2, every
 * rescue net is treated as uncertified too (those voxels take the exact scan, bounded by
 * their first net's k-th distance); with bit 4, the queue holds at most a quarter of the
 * scan's voxels.  0 turns the hook off.  Results do not change, only the path.
 * Process-wide; for tests only.  ABC_ERR_ARG for a mode outside 0..7. */
int abc_debug_force_rescue(int32_t mode);

/* Test hook for the row order of voxels and draws (which decides only how many draw
 * tiles each pass can skip, never a result).  mode 0: k-d splits for scans of at least
 * 2^36 voxel-draw pairs, the Morton key below; 1: the Morton key always; 2: k-d splits
 * always (scans of at least 256 rows, when the scratch holds them).  Process-wide; for
 * tests only.  ABC_ERR_ARG for a mode outside 0..2. */
int abc_debug_order(int32_t mode);

/* Diagnostics: grid size of the last fused-kernel launch of this process, the
 * CTAs per SM its variant can keep resident (shared memory, registers and TMEM
 * columns), and how many kernels this library has launched in this process
 * (replays of a captured CUDA graph are not counted). */
int abc_launch_info(int64_t* grid, int32_t* resident_per_sm, int64_t* kernel_launches);

/* Test hook: the raw tensor-core ranking keys d' = ||yh||^2-free part of the
 * distance (||xh_n||^2 - 2 yh_j . xh_n, yh = sqrt(w)(y - mu), xh = sqrt(w)(x - mu),
 * mu the voxel-mean TAC held in the workspace at byte offset 256) for every
 * pair, written to dump_dev (row stride ld_dump >= N rounded up to 128; J
 * rounded up to 128 rows), without the top-k.  Same argument rules as
 * abc_discrepancy_topk with k = 1. */
int abc_debug_gemm_keys(const float* y_dev, int64_t J, int32_t ldy, const float* x_dev, int64_t N, int32_t ldx,
                        int32_t L, const float* w_host, int32_t precision, void* workspace, size_t ws_bytes,
                        float* dump_dev, int64_t ld_dump, void* stream);

/* Posterior model probabilities (Sec. II-B Eq. 6; Sec. III-B).  Draws of model
 * m are the global indices [offsets[m], offsets[m+1]).  prob_dev[j*M + m] =
 * (# of the k accepted draws of voxel j from model m) / k; preferred_dev[j] =
 * the model with most accepted draws, ties to the lower model position (with
 * M = 2 a model is preferred with more than 50 % of the draws; an even split
 * goes to the first-listed model).  M in 1..16. */
int abc_model_select(const int32_t* idx_dev, int64_t J, int32_t k, const int64_t* model_offsets_host, int32_t M,
                     float* prob_dev, int8_t* preferred_dev, void* stream);

/* Posterior summaries (Sec. II-D point estimate = posterior mean; 95 %
 * credible intervals; Sec. III-B K_i = K1 k3/(k2 + k3) per accepted sample).
 * For voxel j the summarised set is the accepted draws of model
 * preferred_dev[j] (or all k accepted draws when preferred_dev is NULL, using
 * the parameters common to all models).  Output rows have ncols = Pmax + 1
 * columns, Pmax = max(nparams): columns 0..P_m-1 hold the model's parameters,
 * columns P_m..Pmax-1 are NaN, and column Pmax holds K_i when has_ki[m] (K1,
 * k2, k3 read from theta columns ki_cols[0..2]) else NaN.
 *   mean: arithmetic mean;  sd: standard deviation with ddof = 1 (0 for one
 *   sample), two passes about the mean;  lo / hi: the 0.025 / 0.975 quantiles
 *   by linear interpolation between order statistics (type 7).  Sums are
 *   compensated fp32 (relative error near 2^-24 for any k).
 * Each output is J x ncols fp32, row-major.  k in 1..2048, J <= 2^31 - 1;
 * ABC_ERR_ARG for arguments out of range (nothing launched). */
int abc_summarize(const float* theta_dev, int32_t ldtheta, const int64_t* model_offsets_host, int32_t M,
                  const int32_t* nparams_host, const int32_t* has_ki_host, const int32_t* ki_cols_host,
                  const int32_t* idx_dev, int64_t J, int32_t k, const int8_t* preferred_dev, int32_t ncols,
                  float* mean_dev, float* sd_dev, float* lo_dev, float* hi_dev, void* stream);

/* Top-k by the frame-weighted L1 distance d(y, x) = sum_l w_l |y_l - x_l|, the
 * distance Sec. V recommends (Algorithm 1, steps 4-5 with rho = L1).  Same layouts as
 * abc_discrepancy_topk: y_dev J x ldy, x_dev N x ldx (fp32, row-major, first L
 * columns used), w_host L weights (finite, >= 0, copied at the call); outputs idx_dev /
 * dist_dev J x k, per voxel the k nearest draws sorted by (distance, draw index), ties
 * to the lower draw index.  Distances are exact fp32 sums over the frames in order
 * (d += w_l |y_l - x_l| by fma), within (L + 1) 2^-24 d of the exact value.  No
 * tensor-core form exists for L1: a SIMT scan of shared-memory draw tiles with a
 * running threshold per voxel.  L in 1..64, k in 1..2048, k <= N <= 2^31 - 1, J <=
 * 2^31 - 1.  workspace_dev: at least abc_l1_workspace_size(J, k) bytes (candidate
 * lists of 2k + 512 entries per voxel, up to 16 per voxel when few voxels leave the
 * draws split across blocks, and a counter).  ABC_ERR_ARG for arguments out of
 * range or a short workspace (nothing launched). */
size_t abc_l1_workspace_size(int64_t J, int32_t k);
int abc_discrepancy_topk_l1(const float* y_dev, int64_t J, int32_t ldy, const float* x_dev, int64_t N, int32_t ldx,
                            int32_t L, const float* w_host, int32_t k, int32_t* idx_dev, float* dist_dev,
                            void* workspace_dev, size_t workspace_bytes, void* stream);

/* Diagnostics of the last abc_discrepancy_topk_l1 call that used this workspace
 * (synchronous): the number of voxels at which more candidates tied at a cut's k-th
 * distance than the list holds (the ties with the lowest draw indices were kept). */
int abc_l1_status(const void* workspace_dev, int64_t J, int32_t k, int32_t* tie_overflow_host);

/* Posterior band of the lp-ntPET response function (Sec. II-D and its
 * response-function figure): k2a(t) / k2a = 1 + (gamma / k2a) g(t), k2a =
 * k2 / (1 + BP_ND), g the gamma variate of Eq. 4 normalised to 1 at t_P (0 before
 * t_D; x^alpha e^{alpha (1 - x)}, x = (t - t_D) / (t_P - t_D), after).
 *   theta_dev: draw parameters, row i at theta_dev + i * ldtheta (ldtheta >= 7); the
 *     lp-ntPET draws are the global indices [first, last), their columns R1, k2,
 *     BP_ND, gamma, t_D, t_P - t_D, alpha (the caller keeps last within theta).
 *   idx_dev: J x k accepted global draw indices (e.g. abc_discrepancy_topk's output);
 *     entries outside [first, last) (other models' draws, -1) are skipped.
 *   t_host: T times (minutes; 1 <= T <= 256), copied at the call.
 *   mean_dev / lo_dev / hi_dev: J x T fp32, row-major: the mean (compensated fp32 sum)
 *     and the 0.025 / 0.975 type-7 quantiles of the responses of voxel j's accepted
 *     lp-ntPET draws at time t[m]; NaN where the voxel accepted none.
 * Evaluated in fp32 (responses within a few ulp of the exact value). ABC_ERR_ARG for
 * arguments out of range (nothing launched). */
int abc_response_cri(const float* theta_dev, int32_t ldtheta, const int32_t* idx_dev, int64_t J, int32_t k,
                     int64_t first, int64_t last, const float* t_host, int32_t T, float* mean_dev,
                     float* lo_dev, float* hi_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Learned proposal and importance-weighted local ABC.  A build extra: the paper
 * has no counterpart; it replaces the global scan of Algorithm 1 for the
 * irreversible 2TCM (Eq. 1-2 with k4 = 0) by a few thousand proposals per
 * voxel drawn from a per-voxel truncated Gaussian that a small network
 * predicts from the voxel's TAC.
 *
 * Network: D = L + 1 features -> H -> H -> O = 2P outputs, GELU (exact, erf
 * form) after the two hidden layers.  Parameters are one fp32 array in the
 * order W1 (H x D), b1 (H), W2 (H x H), b2 (H), W3 (O x H), b3 (O), row-major;
 * every weight matrix is used rounded to bf16 (round to nearest even), biases
 * and accumulation are fp32.  Output p pairs (out[2p], out[2p+1]) =
 * (mu_p, log sigma_p) of a normal truncated to [0, 1] over the unit-box
 * coordinate u_p = (theta_p - lo_p) / (hi_p - lo_p); mu is clamped to [-3, 4]
 * and log sigma to [-7, 2] wherever they are used.  All buffers are device
 * memory owned by the caller; calls are asynchronous on `stream`.
 * The network's matrix products run on the tensor cores (bf16 products, fp32
 * accumulation): every fp32 activation or gradient operand is split into three
 * bf16 parts (hi + mid + lo, its full 24 bits) and a weight is its bf16 value,
 * so a product equals the fp32 sum up to accumulation rounding (terms of order
 * 2^-24 relative are dropped where both operands are split).
 * ------------------------------------------------------------------------- */

/* Bounded waits of the network's tensor-core products: *timeout_host = 1 if one of them
 * ran out since the last query (the outputs of that call are then not valid), else 0;
 * the flag is cleared.  Synchronous. */
int abc_mlp_status(int32_t* timeout_host);

/* Number of fp32 parameters of a D -> H -> H -> O network (0 on bad sizes). */
size_t abc_mlp_param_count(int32_t D, int32_t H, int32_t O);

/* Bytes of device workspace abc_mlp_forward / abc_mlp_loss_grad need for a
 * batch of B rows (0 on bad sizes): the activations and their gradients, and
 * a fixed slab area where the weight-gradient GEMMs keep per-slice partial
 * sums that are added in a fixed order (gradients are bitwise reproducible). */
size_t abc_mlp_workspace_size(int32_t D, int32_t H, int32_t O, int64_t B);

/* Weights uniform in +-1/sqrt(fan_in) from Philox4x32-10 (counter = parameter
 * index, key = seed), biases zero.  D, H in 1..4096, O in 1..64. */
int abc_mlp_init(uint64_t seed, int32_t D, int32_t H, int32_t O, float* params_dev, void* stream);

/* Network input of each voxel TAC: feat[j*(L+1) + l] = y_jl / s_j for l < L and
 * feat[j*(L+1) + L] = ln(s_j) / 10, s_j = sqrt(sum_l w_l y_jl^2) (the frame
 * weights of Sec. II-C).  y_dev J x ldy; w_host L weights; L in 1..64. */
int abc_mlp_features(const float* y_dev, int64_t J, int32_t ldy, int32_t L, const float* w_host, float* feat_dev,
                     void* stream);

/* out_dev (B x O) = the network applied to the rows of X_dev (B x D).
 * work_dev: >= abc_mlp_workspace_size(D, H, O, B) bytes (its first 2 B H
 * floats are left holding the two hidden pre-activations). */
int abc_mlp_forward(const float* params_dev, int32_t D, int32_t H, int32_t O, const float* X_dev, int64_t B,
                    float* out_dev, void* work_dev, size_t work_bytes, void* stream);

/* Training loss and gradient: *loss_dev = (1/B) sum_n sum_p -log TN(T_np; mu_np,
 * sigma_np, [0, 1]) for targets T_dev (B x P, unit-box coordinates in [0, 1])
 * with O = 2P outputs, and grad_dev (abc_mlp_param_count entries) = its
 * gradient with respect to the parameters (the bf16-rounded weights are
 * differentiated as if they were the fp32 ones; a clamped output passes no
 * gradient).  P in 1..32. */
int abc_mlp_loss_grad(const float* params_dev, int32_t D, int32_t H, int32_t P, const float* X_dev,
                      const float* T_dev, int64_t B, void* work_dev, size_t work_bytes, float* grad_dev,
                      float* loss_dev, void* stream);

/* Training targets: t_dev[n*P + p] = (theta_np - lo_p) / (hi_p - lo_p) clamped to
 * [0, 1], theta_dev N x ldtheta (the layout of abc_sample_prior); P in 1..8. */
int abc_unit_box(const float* theta_dev, int64_t N, int32_t ldtheta, int32_t P, const double* lo_host,
                 const double* hi_host, float* t_dev, void* stream);

/* One Adam step (Kingma and Ba, 2015) with bias correction at step t >= 1:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps); n entries each. */
int abc_adam_update(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, int64_t n, float lr,
                    float beta1, float beta2, float eps, int32_t t, void* stream);

/* Gaussian decay-weighted noise of Sec. III-A on N simulated TACs:
 * y_nl = x_nl + l_n sigma_nl z_nl, sigma_nl = sqrt(max(x_nl, 0) exp(lambda t_l) / dt_l)
 * (t_l the frame mid-time, lambda = ln 2 / half_life), l_n = q_n ||x_n|| / ||sigma_n||,
 * q_n ~ U(q_lo, q_hi), z ~ N(0, 1) by Box-Muller; the uniforms come from
 * Philox4x32-10 keyed by seed at counters tied to the global row
 * first_index + n, so a chunked run reproduces a single call.  L in 1..64. */
int abc_add_noise(const float* x_dev, int64_t N, int32_t ldx, const abc_frames* frames, double half_life, double q_lo,
                  double q_hi, uint64_t seed, int64_t first_index, float* y_dev, int32_t ldy, void* stream);

/* Shared memory abc_local_abc needs per block (it must stay <= 227 KB). */
size_t abc_local_abc_smem_bytes(int32_t T, int32_t L, int32_t M);

/* The G table in the layout abc_local_abc reads: table_dev[l * T + i] =
 * rows_dev[i * ld + l] for the T rows (one per grid node a_i, L frames each,
 * row stride ld >= L) that abc_simulate writes.  table_dev: L x T floats,
 * caller-owned.  ABC_ERR_ARG on bad sizes or null pointers. */
int abc_local_abc_table(const float* rows_dev, int32_t T, int32_t L, int32_t ld, float* table_dev, void* stream);

/* Importance-weighted local ABC for the irreversible 2TCM, P = 4 parameters
 * (K1, k2, k3, Vb) on the prior box [lo, hi] (host, 4 entries each, lo >= 0).
 * For each voxel j: M proposals u_i ~ TN(mu_jp, sigma_jp) on [0, 1] per
 * parameter, mu and sigma = sigma_scale * exp(log sigma) from prop_dev (J x 8
 * network outputs, clamped as above; sigma_scale in (0, 100] widens the
 * proposal), drawn by inverse CDF of the
 * uniforms ((r_p >> 9) + 1/2) 2^-23, r = Philox4x32-10 at counter
 * (i, j lo, j hi, 0x4C4F43) and key (seed lo, seed hi); theta = lo + (hi - lo) u; the TAC
 * of each proposal from
 *   x_l = Vb cp_l + (1 - Vb) K1 / a (k3 G_l(0) + k2 G_l(a)),  a = k2 + k3,
 * where table_dev (L x T, frame-major: table_dev[l * T + i], see
 * abc_local_abc_table) holds G(a_i) = frame means of e^{-a_i t} (*) C_p at
 * a_i = a_max (i / (T - 1))^2 (column 0 = frame means of 1 (*) C_p) and
 * cp_frames_dev the L frame means of C_p, read by cubic Lagrange interpolation
 * in i; d_ji = sum_l w_l (y_jl - x_l)^2, evaluated as y.y - 2 y.x + x.x from
 * weighted dot products of y, cp, G(0) and the table rows (interpolated alike);
 * the k nearest kept (ties to the lower
 * proposal index; the k-th distance is found exactly, by radix selection over
 * the candidates a pilot sample of the first proposals brackets, or over all
 * M distances when the bracket misses); weights W = (1/q(u)) normalised over the accepted set
 * (uniform prior).  Outputs (J x 5, columns K1, k2, k3, Vb, K_i = K1 k3/(k2+k3)):
 * weighted mean, weighted SD sqrt(sum W (v - m)^2), and weighted 2.5 / 97.5 %
 * quantiles (the smallest accepted value whose cumulative weight reaches the
 * level); per voxel ess = 1 / sum W^2, dmed = the ((k-1)/2)-th smallest
 * distance, ynorm = sum_l w_l y_jl^2.  u_dump_dev (J x M x 4) and d_dump_dev
 * (J x M) receive every proposal and distance when non-NULL.
 * 1 <= k <= 256, k <= M; T >= 8; lo[1] + lo[2] > 0 and hi[1] + hi[2] <= a_max;
 * abc_local_abc_smem_bytes(T, L, M) <= 227 KB. */
int abc_local_abc(const float* y_dev, int64_t J, int32_t ldy, int32_t L, const float* w_host, const float* prop_dev,
                  const float* table_dev, int32_t T, double a_max, const float* cp_frames_dev, const double* lo_host,
                  const double* hi_host, int32_t M, int32_t k, float sigma_scale, uint64_t seed, float* mean_dev,
                  float* sd_dev,
                  float* qlo_dev, float* qhi_dev, float* ess_dev, float* dmed_dev, float* ynorm_dev,
                  float* u_dump_dev, float* d_dump_dev, void* stream);

/* Reliability check of the learned path (a workload extension with no counterpart in the
 * paper): the voxels whose local run is handed to the global path (Algorithm 1).
 * For j < J, voxel j falls back when !(ess_dev[j] >= k / 4) (a NaN ESS included) or, with
 * rel_max > 0, when dmed_dev[j] > rel_max * ynorm_dev[j] (the abc_local_abc outputs;
 * dmed_dev and ynorm_dev may be NULL when rel_max <= 0).  rows_dev (J int32, device)
 * receives the fallback voxels in ascending order, *count_dev (one int32, device) their
 * number; nothing is read back, so the call is one asynchronous enqueue on stream.
 * scratch_dev: abc_fallback_scratch_size(J) bytes of device memory, caller-owned.
 * ABC_ERR_ARG for J outside 1 .. 2^31 - 1, k < 1, a null pointer or a short scratch. */
size_t abc_fallback_scratch_size(int64_t J);
int abc_fallback_rows(const float* ess_dev, const float* dmed_dev, const float* ynorm_dev, int64_t J, int32_t k,
                      float rel_max, int32_t* rows_dev, int32_t* count_dev, void* scratch_dev, size_t scratch_bytes,
                      void* stream);

/* Row moves for the fallback (fp32, device): gather dst[i, 0:width) = src[rows[i], 0:width),
 * scatter dst[rows[i], 0:width) = src[i, 0:width), for i < min(*count_dev, max_rows) (the
 * count is read on the device, so a count from abc_fallback_rows needs no host copy).
 * Row strides ld_src, ld_dst >= width, in floats.  ABC_ERR_ARG on a null pointer or bad
 * sizes. */
int abc_gather_rows(const float* src_dev, int32_t ld_src, const int32_t* rows_dev, const int32_t* count_dev,
                    int64_t max_rows, int32_t width, float* dst_dev, int32_t ld_dst, void* stream);
int abc_scatter_rows(const float* src_dev, int32_t ld_src, const int32_t* rows_dev, const int32_t* count_dev,
                     int64_t max_rows, int32_t width, float* dst_dev, int32_t ld_dst, void* stream);

/* Calibration of the fallback threshold: over voxels j < J, the relative median accepted
 * distance rel_j = dist_dev[j k + (k - 1) / 2] / sum_l w_l y_jl^2 (dist_dev: J x k accepted
 * distances of the global path, ascending per voxel; y_dev: J x L TACs, row stride ldy;
 * w_host: L frame weights), and its q-quantile by linear interpolation between the order
 * statistics floor(h) and floor(h) + 1, h = q (J - 1) (numpy's default), both found exactly
 * by a radix selection on the device; the result goes to *out_host (blocks on stream).
 * scratch_dev: abc_quantile_scratch_size(J) bytes.  ABC_ERR_ARG for J outside
 * 1 .. 2^31 - 1, k < 1, L outside 1 .. 64, ldy < L, q outside [0, 1], a null pointer or a
 * short scratch. */
size_t abc_quantile_scratch_size(int64_t J);
int abc_median_rel_quantile(const float* dist_dev, int64_t J, int32_t k, const float* y_dev, int32_t ldy, int32_t L,
                            const float* w_host, double q, float* out_host, void* scratch_dev, size_t scratch_bytes,
                            void* stream);

/* Description of the last error on this thread ("" if none). */
const char* abc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VPETABC_H */
