/*
 * hologen.h -- C ABI of the GB300 phase-retrieval library (libhologen.so).
 *
 * The paper (section "Algorithm Interface") passes a target image and the algorithm parameters down
 * to a CUDA class (AlgorithmCuda: "stores target, illumination and starting images as well as
 * common algorithm parameters"), whose RunIterations() runs the loop.  This header is that
 * boundary, re-cut as a plan object plus one call per algorithm:
 *
 *   hg_plan_create / hg_plan_destroy   sizes, propagation (Fourier / Fresnel: wavelength, pitch,
 *                                      distances) and quantisation levels; owns tables + workspace
 *   hg_propagate                       bare forward / inverse Fourier or Fresnel transform
 *   hg_gs_run                          Gerchberg-Saxton (section "Algorithm Libraries",
 *                                      HoloGenAlgGSCuda), single- or multi-plane
 *   hg_ospr_run                        One-Step Phase-Retrieval (HoloGenAlgOSPRCuda)
 *   hg_gd_step                         one Adam step of gradient-descent hologram optimisation
 *                                      (no counterpart in the paper)
 *   hg_mraf_run / hg_hio_run           GS variants with a signal window: mixed-region amplitude
 *                                      freedom and hybrid input-output ("other iterative Fourier
 *                                      transform approaches" of HoloGenAlgGSCuda)
 *   hg_dbs_run / hg_sa_run             direct binary search and simulated annealing with the
 *                                      single-pixel replay update (the DS and SA classes,
 *                                      FFTUpdaterCuda)
 *   hg_plan_set_illumination,          SLM illumination profile; multi-amplitude / complex-
 *   hg_plan_set_slm_levels             modulation SLM values (the MultiAmpSLM option)
 *   hg_plan_autotune, graph mode,      strip widths, CUDA-graph replay, per-kernel timing and
 *   timing, hg_gs_run_noalloc          a no-allocation GS call
 *
 * Conventions (every entry point):
 *  - Data pointers are DEVICE pointers owned by the caller (CUDA global memory on the plan's device).
 *    Arrays typed `T* const*` are HOST arrays holding one device pointer per item (n_items entries)
 *    or per item and plane (item-major: [item * n_planes + plane]).
 *  - Fields are complex64 stored as interleaved (re, im) float32, row-major [H][W], FFT order
 *    (DC at [0][0]).  Real images are float32 [H][W] row-major.  Field pointers must be 8-byte
 *    aligned, float pointers 4-byte aligned.
 *  - Calls are asynchronous and stream-ordered on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Only hg_plan_create, hg_plan_destroy and hg_plan_sync synchronise the host.
 *  - Each call returns a status and never throws.  Argument errors leave outputs untouched.  A CUDA
 *    launch error is returned as HG_ERR_CUDA; asynchronous device errors surface on a later call or
 *    in hg_plan_sync.  hg_last_error() gives a thread-local detail string for the last failure.
 *  - Device pointers are checked before launch: a pointer that is not device memory of the plan's
 *    device, or a buffer that does not fit in its allocation, is rejected with HG_ERR_INVALID_ARG.
 *  - A plan is used from one host thread at a time.  Different plans are independent.
 *  - Supported FFT lengths (H and W): every n = 2^a 3^b 5^c with 1 <= n <= 4096 (137 lengths).
 *    8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 12, 15, 30, 60, 120, 720, 864, 1080, 1152,
 *    1200, 1280, 1440, 1536, 1600, 1920, 2160, 2560 and 3840 have compiled kernels (radix plans fixed at build time, the field in registers between
 *    stages); the others run on generic kernels (a run-time radix plan, the tile in shared memory
 *    between stages; slower, same arithmetic).  Other sizes give HG_ERR_UNSUPPORTED_SIZE.
 */
#ifndef HOLOGEN_H
#define HOLOGEN_H

#include <stdint.h>

#if defined(__GNUC__)
#define HG_API __attribute__((visibility("default")))
#else
#define HG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HG_OK = 0,
  HG_ERR_INVALID_ARG = 1,
  HG_ERR_UNSUPPORTED_SIZE = 2,
  HG_ERR_OUT_OF_MEMORY = 3,
  HG_ERR_CUDA = 4,
  HG_ERR_TIMEOUT = 5,
  HG_ERR_INTERNAL = 6
} hg_status;

/* Fourier / Fresnel holograms (paper keywords "Fourier", "Fresnel"). */
typedef enum { HG_FOURIER = 0, HG_FRESNEL = 1 } hg_propagation;

typedef struct hg_plan hg_plan;

typedef struct {
  int32_t n_items;         /* holograms per run, 1..256 */
  const int32_t* heights;  /* H of each item (n_items entries) */
  const int32_t* widths;   /* W of each item */
  int32_t propagation;     /* hg_propagation */
  double wavelength_m;     /* Fresnel: wavelength lambda (> 0) */
  double pitch_m;          /* Fresnel: SLM pixel pitch p (> 0) */
  int32_t n_planes;        /* replay planes P >= 1 (Fourier: must be 1) */
  const double* z_m;       /* Fresnel: P propagation distances (> 0); may be NULL for Fourier */
  int32_t quant_levels;    /* 0 continuous phase; 2 binary {0, pi}; N in 3..256 N-level */
  uint32_t flags;          /* 0, or HG_PLAN_AUTOTUNE and / or HG_TARGET_CENTRED */
} hg_plan_desc;

/* hg_plan_create runs hg_plan_autotune before returning. */
#define HG_PLAN_AUTOTUNE 1u
/* Strip width that selects the whole-run cluster kernel (hg_plan_set_strip_width). */
#define HG_STRIP_CLUSTER (-1)
/* Targets (hg_gs_run, hg_mraf_run, hg_hio_run, hg_ospr_run amplitudes, gradient-descent target
 * intensities) and MRAF / HIO signal masks are given in display order, with the zero frequency at
 * row H/2, column W/2 (integer halves): the plan reads pixel (i, j) of the FFT-ordered replay plane
 * from ((i + H/2) mod H, (j + W/2) mod W) of the caller's array (numpy's ifftshift), in the pass
 * that copies targets into the plan, so the loops run at the same speed.  Holograms, NMSE and
 * gradients stay in the SLM's own pixel order; hg_propagate is not affected. */
#define HG_TARGET_CENTRED 2u

/*
 * Fresnel model (single-FFT, reading of the paper's "Fresnel" keyword): SLM pixel (i, j) at
 * y_i = (i - floor(H/2)) p, x_j = (j - floor(W/2)) p; input chirp
 * c(i, j) = exp(i pi (x_j^2 + y_i^2) / (lambda z)); forward R = F(h c), inverse g = conj(c) F^-1(R).
 * F is the unitary 2D DFT.  The output-plane chirp and constant phase factor are omitted.
 *
 * SLM projection: continuous h = g/|g| (1 where g = 0); N-level: nearest of exp(2 pi i q / N),
 * q = floor(arg(g) N / (2 pi) + 1/2) mod N, arg in [0, 2 pi).
 */

/* Creates a plan on the current CUDA device.  desc (and its arrays) may be freed after the call.
 * Errors: INVALID_ARG (bad field), UNSUPPORTED_SIZE (H or W not a supported length),
 * OUT_OF_MEMORY (workspace), CUDA. */
HG_API hg_status hg_plan_create(const hg_plan_desc* desc, hg_plan** out);

/* Destroys a plan (synchronises its device first).  NULL is accepted. */
HG_API hg_status hg_plan_destroy(hg_plan* plan);

/* Waits for all work issued by the plan and reports any asynchronous device error. */
HG_API hg_status hg_plan_sync(hg_plan* plan);

/*
 * Bare propagation of every item through plane `plane` (0..P-1):
 *   direction +1:  out = F(in * c)          direction -1:  out = conj(c) * F^-1(in)
 * (c = 1 for Fourier).  in[k], out[k]: complex64 [H_k][W_k]; in and out may alias (in place).
 */
HG_API hg_status hg_propagate(hg_plan* plan, int32_t plane, int32_t direction, const void* const* in,
                       void* const* out, void* stream);

/*
 * Gerchberg-Saxton phase retrieval (Gerchberg & Saxton 1972, error-reduction form), n_iter >= 0
 * iterations for every item:
 *   h_0 = P_SLM(exp(i phi_0));  R_k = F(h_k c);  R'_k = A R_k / |R_k|;
 *   h_{k+1} = P_SLM(conj(c) F^-1(R'_k)).
 * With P > 1 planes the SLM update averages the P back-propagated fields (multi-plane GS,
 * averaged projections) before projecting.
 *  target_amp[k*P + p]  float32 [H][W] target amplitude A of item k, plane p (FFT order, >= 0)
 *  init_phase           NULL, or per item NULL / float32 [H][W] starting phase phi_0 (radians);
 *                       a NULL entry draws phi_0 = 2 pi u, u from Philox4x32-10 with counter
 *                       (pixel, 0, 1, 0) and key (seed_lo, seed_hi ^ item)
 *  phase_out            NULL, or per item NULL / float32 [H][W]: phase of h_{n_iter} in [0, 2 pi)
 *  level_out            NULL, or per item NULL / uint8 [H][W]: level index q (quantised plans only)
 *  nmse_out             NULL or device float32 [n_items][n_iter + 1]: NMSE of h_k, k = 0..n_iter,
 *                       NMSE = 1 - (sum I T)^2 / (sum I^2 sum T^2), I = |R|^2, T = A^2 (mean over
 *                       planes when P > 1)
 */
HG_API hg_status hg_gs_run(hg_plan* plan, const float* const* target_amp, const float* const* init_phase,
                    uint64_t seed, int32_t n_iter, float* const* phase_out, uint8_t* const* level_out,
                    float* nmse_out, void* stream);

/*
 * SLM illumination (section "Algorithm Libraries": AlgorithmCuda stores "target, illumination and
 * starting images").  illum_amp: host array of n_items device pointers to float32 [H][W]
 * amplitude profiles (row-major, the SLM plane), or NULL entries for uniform unit illumination; a
 * NULL array clears the setting.  The plan keeps the pointers (the caller keeps the buffers alive
 * and unchanged while runs use them).  hg_gs_run then takes the SLM field as illum * P_SLM(g): the
 * SLM sets the phase only.  Single-plane plans; hg_mraf_run, hg_hio_run, hg_ospr_run and the
 * gradient-descent calls reject a plan that has a profile set (HG_ERR_INVALID_ARG).
 */
HG_API hg_status hg_plan_set_illumination(hg_plan* plan, const float* const* illum_amp);

/*
 * Multi-amplitude / complex-modulation SLM (section "Application": the SLM type option offers a
 * multi-amplitude SLM, MultiAmpSLM).  levels: host array of 2 n_levels floats, the (re, im) pairs
 * of the n_levels (2..256) complex values a pixel can take; copied.  hg_gs_run, hg_mraf_run and
 * hg_hio_run then project the SLM-plane field g onto the nearest of them, h = m_q with
 * q = argmin |g - m_q| (float32 squared distance, the lowest index on a tie), with g in the
 * unitary scale of the loop (the replay target at the energy of a unit-modulus field);
 * level_out[i] receives q and phase_out[i] arg(m_q) in [0, 2 pi).  NULL or n_levels 0 restores the
 * plan's phase-only levels.  Drops captured graphs.  Errors: HG_ERR_INVALID_ARG for a multi-plane
 * or illuminated plan, n_levels outside 2..256 or a non-finite value; direct binary search,
 * annealing and gradient descent reject a plan with a table.
 */
HG_API hg_status hg_plan_set_slm_levels(hg_plan* plan, const float* levels, int32_t n_levels);

/*
 * Mixed-region amplitude freedom (MRAF; Pasienski & DeMarco 2008): the reading taken here of the
 * paper's "other iterative Fourier transform approaches" (section "Algorithm Libraries",
 * HoloGenAlgGSCuda).  Same loop, arguments and outputs as hg_gs_run on a single-plane plan, except
 * in the replay plane: with signal region S (signal_mask[i][px] != 0; a NULL array or entry means
 * the whole plane) and mix m in (0, 1],
 *   R' = m A_s R / |R| on S,   R' = (1 - m) R elsewhere,   A_s = A sqrt(HW / sum_S A^2),
 * and nmse_out[i][k] is the NMSE of h_k over S only.  signal_mask: per item a device uint8 [H][W]
 * (FFT order, like the target); read only.  Errors: HG_ERR_INVALID_ARG for a multi-plane plan or m
 * outside (0, 1], plus those of hg_gs_run.
 */
HG_API hg_status hg_mraf_run(hg_plan* plan, const float* const* target_amp, const uint8_t* const* signal_mask,
                             float mix, const float* const* init_phase, uint64_t seed, int32_t n_iter,
                             float* const* phase_out, uint8_t* const* level_out, float* nmse_out, void* stream);

/*
 * Hybrid input-output (HIO; Fienup 1982) with the replay plane as the constrained domain: a second
 * reading of the paper's "other iterative Fourier transform approaches" (section "Algorithm
 * Libraries").  Arguments and outputs as hg_mraf_run, with feedback beta in (0, 2] in place of mix.
 * The input X is a replay-plane field; h_k = P_SLM(conj(c) F^-1(X_k)), Y_k = F(h_k c) and
 *   X_{k+1} = A_s Y_k / |Y_k| on S,   X_{k+1} = X_k - beta Y_k elsewhere,   X_0 = Y_0,
 * A_s as for MRAF; nmse_out[i][k] is the NMSE of h_k over S.  With S the whole plane it is GS.  The
 * plan allocates an input buffer (8 bytes per pixel) on the first call.  Errors: HG_ERR_INVALID_ARG
 * for a multi-plane plan, a plan with an illumination profile or beta outside (0, 2], plus those
 * of hg_gs_run.
 */
HG_API hg_status hg_hio_run(hg_plan* plan, const float* const* target_amp, const uint8_t* const* signal_mask,
                            float beta, const float* const* init_phase, uint64_t seed, int32_t n_iter,
                            float* const* phase_out, uint8_t* const* level_out, float* nmse_out, void* stream);

/*
 * Direct binary search (section "Algorithm Libraries": the DS algorithm class and the single-pixel
 * replay updater FFTUpdaterCuda; reading: Seldowitz, Allebach & Sweeney 1987) on a binary plan
 * (quant_levels 2, one plane, no illumination profile).  From h_0 = P_2(exp(i phi_0)) (init_phase
 * as in hg_gs_run, or the Philox draw from seed), each of n_sweeps sweeps visits the SLM pixels in
 * row-major order and keeps the flip h_p -> -h_p when it strictly lowers the NMSE of
 * |F(h c)|^2 against A^2 (optimal scale); the replay is updated by the single-pixel change
 * -2 h_p c_p exp(-2 pi i (k m / H + l n / W)) (unnormalised) instead of a new transform.
 *  phase_out / level_out  as in hg_gs_run (phase 0 or pi, level 0 or 1), after the last sweep
 *  nmse_out               NULL or device float32 [n_items][n_sweeps + 1]: NMSE after s sweeps
 * Each item runs in one thread-block cluster of ceil(H W / 4096) CTAs (replay plane in registers,
 * one cluster barrier per trial flip); items of at most 65536 pixels (HG_ERR_UNSUPPORTED_SIZE
 * beyond, or where the device cannot run the cluster).  Errors: HG_ERR_INVALID_ARG for a plan
 * that is not binary, multi-plane or illuminated, n_sweeps outside 0..10000, and bad pointers.
 */
HG_API hg_status hg_dbs_run(hg_plan* plan, const float* const* target_amp, const float* const* init_phase,
                            uint64_t seed, int32_t n_sweeps, float* const* phase_out, uint8_t* const* level_out,
                            float* nmse_out, void* stream);

/*
 * Simulated annealing (section "Algorithm Libraries": the SA algorithm class; reading: Kirkpatrick,
 * Gelatt & Vecchi 1983) over the trial flips of hg_dbs_run, with its arguments, outputs, limits
 * and errors: sweep s runs at temperature T_s = t0 alpha^s (t0 > 0 finite, alpha in (0, 1]); a flip
 * that does not lower the NMSE E is still kept when u < exp(-(E' - E) / T_s), with u = (x >> 8) 2^-24
 * and x word 0 of Philox4x32-10 with counter (pixel, s, 2, 0) and key (seed_lo, seed_hi ^ item).
 */
HG_API hg_status hg_sa_run(hg_plan* plan, const float* const* target_amp, const float* const* init_phase,
                           uint64_t seed, int32_t n_sweeps, double t0, double alpha, float* const* phase_out,
                           uint8_t* const* level_out, float* nmse_out, void* stream);

/*
 * One-Step Phase-Retrieval (Cable, Buckley et al.; section "Algorithm Libraries",
 * HoloGenAlgOSPRCuda): for every item (target t) and subframe s = 0..n_subframes-1
 *   E = A exp(2 pi i u),  u = (x >> 8) 2^-24,  x = word 0 of Philox4x32-10 with counter
 *       (pixel, s, 0, 0) and key (seed_lo, seed_hi ^ t)
 *   h_s = binary(conj(c) F^-1(E))           (+ n_iter binary GS iterations against A)
 *   I_acc += |F(h_s c)|^2,   nmse_out[t][s] = NMSE(I_acc, A^2)
 * Binary projection as in hg_plan_desc (N = 2, h = +1 / -1), whatever the plan's quant_levels.
 *  target_amp[t]  float32 [H][W] amplitude (FFT order).  A real hologram has a point-symmetric
 *                 replay, so only the symmetric part of a target is reachable.
 *  bits_out       NULL, or per item NULL / uint32 [n_subframes][H][ceil(W/32)]: bit (w*32 + i) of
 *                 row word w is pixel w*32 + i, 1 = phase pi.
 *  nmse_out       NULL or device float32 [n_items][n_subframes].
 * The plan allocates an intensity buffer (4 bytes per pixel) on the first call.
 */
HG_API hg_status hg_ospr_run(hg_plan* plan, const float* const* target_amp, int32_t n_subframes, int32_t n_iter,
                             uint64_t seed, uint32_t* const* bits_out, float* nmse_out, void* stream);

/*
 * Gradient-descent hologram optimisation (Wirtinger calculus; no counterpart in the paper, which
 * offers GS, SA, DS and OSPR): one Adam step on the phase phi of every item, for a loss over the
 * plan's P replay planes (Fresnel distances z_m, or one Fourier plane):
 *   U_p = F(exp(i phi) c_p),  I_p = |U_p|^2,  s_p = sum(I_p T_p) / sum(I_p^2),
 *   L_p = sum((s_p I_p - T_p)^2) / sum(T_p^2),  L = (1/P) sum_p L_p,
 *   dL/dphi = 2 Im(g conj(exp(i phi))),  g = sum_p conj(c_p) F^-1((2/P) s_p (s_p I_p - T_p)/sum(T_p^2) U_p)
 * (s_p is optimal, so it is held fixed in the derivative), then Adam (Kingma & Ba):
 *   m = b1 m + (1-b1) grad;  v = b2 v + (1-b2) grad^2;
 *   phi -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 *  phase[k]          float32 [H][W], updated in place (unwrapped)
 *  target_int[k*P+p] float32 [H][W] target intensity T_p (FFT order)
 *  adam_m, adam_v    per item float32 [H][W] moments (zero before step 1), updated in place
 *  step              1-based step count
 *  loss_out          NULL or device float32 [n_items][P + 1]: L_p per plane, then L (before the update)
 *  grad_out          NULL, or per item NULL / float32 [H][W]: dL/dphi at the input phase
 * The plan must be continuous-phase (quant_levels 0).  The per-plane row-FFT fields of the forward
 * transform are kept in the plan workspace as the checkpoint the adjoint pass recomputes U_p from.
 */
HG_API hg_status hg_gd_step(hg_plan* plan, float* const* phase, const float* const* target_int,
                            float* const* adam_m, float* const* adam_v, int32_t step, float lr, float beta1,
                            float beta2, float eps, float* loss_out, float* const* grad_out, void* stream);

/* The two halves of hg_gd_step without the update, for autograd front ends: hg_gd_forward writes
 * loss_out and keeps the checkpoint; hg_gd_backward (after exactly one hg_gd_forward with the same
 * phase and targets) writes grad_out[k] = grad_scale * dL/dphi (grad_scale: NULL = 1, or a device
 * float32 scalar). */
HG_API hg_status hg_gd_forward(hg_plan* plan, float* const* phase, const float* const* target_int,
                               float* loss_out, void* stream);
HG_API hg_status hg_gd_backward(hg_plan* plan, float* const* phase, const float* const* target_int,
                                const float* grad_scale, float* const* grad_out, void* stream);

/*
 * Gerchberg-Saxton for ONE Fourier hologram without allocating device memory.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc -- code running inside a memory
 * arena it does not own, plug-ins whose host forbids allocation after start-up, real-time loops in
 * which an allocation (it may synchronise the device) would break the latency budget -- and so
 * cannot create a plan.
 *
 * Same algorithm, kernels and argument meanings as hg_gs_run with a one-item, one-plane Fourier plan
 * (quant_levels as in hg_plan_desc; target_amp, init_phase, phase_out, level_out are single device
 * pointers; nmse_out is [n_iter + 1]).  Its scratch (field, reduction partials, twiddle and level
 * tables) is a static device array of 8 MiB + 155 KiB that every device which loads this
 * library keeps until the process exits.
 *  - Limits: height * width <= 1048576 pixels, each a supported FFT length; larger sizes return
 *    HG_ERR_UNSUPPORTED_SIZE before anything is launched.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress), so make
 *    that first call before any stream capture.  The address is looked up again whenever the
 *    calling thread's current context is a different one from the last lookup's (for example after
 *    cudaDeviceReset, which unloads the module holding the array).
 *  - Under CUDA's default lazy module loading the driver loads the module that holds the array, and
 *    reserves the array, during the first call on a device, and loads each FFT length's kernels at
 *    their first launch.  Callers that must not allocate after start-up should make one warm-up
 *    call per device and per (height, width) at start-up, or run with CUDA_MODULE_LOADING=EAGER.
 *  - Calls no cudaMalloc / cudaFree or allocating routine.  Every call shares the one array and
 *    leaves its contents behind; each call rewrites the tables and every partial it reads on its own
 *    stream before using them, so nothing has to start at zero.  Any two calls that are not ordered
 *    on one stream race on the array and give wrong results -- calls from other host threads, and
 *    calls from the same thread on two different streams alike: the caller serialises them (one
 *    stream, or an event and a stream wait between them).
 */
HG_API hg_status hg_gs_run_noalloc(int32_t height, int32_t width, int32_t quant_levels, const float* target_amp,
                                   const float* init_phase, uint64_t seed, int32_t n_iter, float* phase_out,
                                   uint8_t* level_out, float* nmse_out, void* stream);

/*
 * Kernel timing (tracing aid; no counterpart in the paper).  While enabled, every kernel the plan
 * launches is bracketed by two CUDA events on its stream and its device time is added to the
 * total of its kind.  hg_plan_kernel_time synchronises the plan's device, folds the pending events
 * in and returns (total milliseconds, launches) for one kind; hg_kernel_kind_name names the kinds
 * (NULL past the last).  hg_plan_launch_count counts every kernel launched by the plan since
 * creation, timed or not.
 */
HG_API hg_status hg_plan_set_timing(hg_plan* plan, int32_t enabled);
HG_API hg_status hg_plan_kernel_time(hg_plan* plan, int32_t kind, double* total_ms, int64_t* launches);
HG_API hg_status hg_plan_reset_timing(hg_plan* plan);
HG_API const char* hg_kernel_kind_name(int32_t kind);
HG_API int64_t hg_plan_launch_count(const hg_plan* plan);

/*
 * Execution options (no counterpart in the paper, whose batch processing is a job table in the user
 * interface).  hg_gs_run runs the size classes of a plan smallest first (each class one batched
 * launch per pass), so small holograms finish early.  With graph mode on, it captures the whole launch
 * sequence into a CUDA graph the first time it sees an argument set, and replays that graph with a
 * single launch while the arguments (pointers, n_iter, seed) stay the same (hg_ospr_run likewise).
 * A plan keeps one graph with timing off and one with timing on; the timed graph records the event
 * pair of every kernel as graph nodes, and the timing totals take its latest replay only.  Outside
 * graphs, GS passes of at most 2048 x 2048 pixels per launch use programmatic dependent launch.
 * hg_plan_item_latency synchronises and returns, for each item, the device time (ms, %globaltimer)
 * from the start of the last hg_gs_run to the end of its size class.
 */
HG_API hg_status hg_plan_set_graph(hg_plan* plan, int32_t enabled);

/*
 * Autotuner (a tuning choice the plan owns; no counterpart in the paper).  GS keeps its field
 * tiled in column strips so that a column pass reads its strip as one contiguous block; the strip
 * width trades the column pass's CTA size against the row pass's access pattern.  The plan starts
 * from a measured default per column length (multi-plane GS: that default where it is 2, 4 or 8
 * columns, else a row-major field; gradient descent always keeps its field row-major).
 * hg_plan_autotune times, for every size class, a 10-iteration GS run (seeded start, zero target
 * in its own scratch; the fastest of five runs) with each width the class allows (2, 4, 8 or 16
 * columns for one plane, 2, 4 or 8 for several, or a row-major field) and each radix plan of the
 * row and column passes (below; single-plane only) and keeps the fastest; choices are cached per process by (device, H, W,
 * items in the class, levels, propagation).  It
 * synchronises `stream` before and after, allocates and frees one scratch target per class, does
 * not count or time its own launches, and drops captured graphs.  Results of later runs do not
 * depend on the width except for the order in which NMSE partial sums are added.
 * hg_plan_strip_width returns the width in use for an item's size class (0: row-major field);
 * hg_plan_set_strip_width sets it by hand (synchronises the device, drops captured graphs;
 * HG_ERR_INVALID_ARG for a width the class does not allow).
 * Width -1 (HG_STRIP_CLUSTER), available for square classes of 64, 128 or 256 pixels on a
 * single-plane plan and the default for such a class of one item: hg_gs_run runs the whole loop of each item in one
 * launch, one thread-block cluster (16 CTAs where the device runs clusters that large, else 8)
 * per item with the field held in the cluster's shared memory; the arithmetic per pixel is that
 * of the two-pass kernels, only the NMSE partial sums are grouped differently.  MRAF, HIO and
 * illuminated runs of such a class use the default strip width; the autotuner includes -1 among
 * the candidates.
 */
HG_API hg_status hg_plan_autotune(hg_plan* plan, void* stream);
HG_API hg_status hg_plan_strip_width(const hg_plan* plan, int32_t item, int32_t* width_out);
HG_API hg_status hg_plan_set_strip_width(hg_plan* plan, int32_t item, int32_t width);

/*
 * Radix plans (part of the same autotuner; no counterpart in the paper, whose FFT handler defers to
 * cuFFT's own planning).  Lengths 864, 1024, 1080, 1536, 1920 and 2048 have their single-plane
 * tiled GS passes compiled with two radix plans: the default (e.g. 2048 = 16 x 16 x 8) and an
 * alternative (2048 = 16 x 8 x 16; 1024 = 4 x 16 x 16; 864 = 9 x 6 x 16; 1080 = 15 x 9 x 8;
 * 1536 = 16 x 6 x 16; 1920 = 15 x 8 x 16).  Row and column passes choose independently: plan 0 the
 * default, 1 the alternative.  hg_plan_autotune times every (strip width, row plan, column plan)
 * the class allows and keeps the fastest; hg_plan_radix_plan returns the choice of an item's size
 * class and hg_plan_set_radix_plan sets it by hand (HG_ERR_INVALID_ARG for 1 on a length without
 * an alternative; synchronises the device and drops captured graphs).  The alternative applies to
 * plain GS runs on a tiled field (not row-major, cluster, MRAF, HIO, illumination or level-table
 * runs, which use the default plan).  Results differ between plans only by float32 rounding.
 */
HG_API hg_status hg_plan_radix_plan(const hg_plan* plan, int32_t item, int32_t* row_plan, int32_t* col_plan);
HG_API hg_status hg_plan_set_radix_plan(hg_plan* plan, int32_t item, int32_t row_plan, int32_t col_plan);
HG_API hg_status hg_plan_item_latency(hg_plan* plan, double* ms_out);

/* Human-readable name of a status code (static string). */
HG_API const char* hg_status_string(hg_status status);

/* Detail message of the last failing call on this host thread ("" if none). */
HG_API const char* hg_last_error(void);

/* 1 if n is a supported FFT length (n = 2^a 3^b 5^c, 1 <= n <= 4096), else 0. */
HG_API int32_t hg_supported_length(int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* HOLOGEN_H */
