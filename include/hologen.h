/*
 * hologen.h -- C ABI of the GB300 iterative Fourier-transform hologram engine.
 *
 * The engine computes 2D Fourier holograms for phase-only spatial light
 * modulators (SLMs) with the iterative Fourier-transform algorithms of
 * HoloGen (Christopher, Kadis, Gordon, Wilkinson, arXiv:2008.12214):
 * Gerchberg-Saxton (GS) and weighted GS (Section 3.2) and one-step phase
 * retrieval (OSPR, Section 3.4).  The far field of the SLM is the unitary 2D
 * DFT of Section 2, eqs. (fouriertrans2d5c) and (fouriertrans2d5d); the SLM
 * keeps only phases on its levels (Section 3, Fig. 1); the error is the MSE of
 * Section 3.1, eq. (mse), plus the intensity MSE described below.
 *
 * Conventions used by every call
 *  - Images are row-major [ny][nx], x fastest, one image per target; a batch
 *    is [batch][ny][nx].  ny and nx must be supported lengths (see
 *    hg_supported_length); otherwise HG_ERR_UNSUPPORTED_SIZE.
 *  - Targets and replay-plane quantities (target amplitude, phases, weights,
 *    intensities) are in REPLAY order: the zero spatial frequency at pixel
 *    (ny/2, nx/2) (integer division), i.e. replay = fftshift(FFT2(slm)).
 *    Holograms are in natural SLM order.
 *  - Pointers may be device pointers or ordinary host pointers.  With device
 *    pointers the call only enqueues work on the plan's stream and returns
 *    (errors detected on the device surface at hg_sync or at the next call
 *    that synchronises); with any host pointer the call copies through
 *    plan-owned device buffers and synchronises the stream before returning.
 *  - The caller owns every buffer it passes; the plan owns its workspace.
 *    No call keeps a caller pointer after it returns.
 *  - No call throws, aborts, or falls back to a CPU path; failures come back
 *    as a status code.  A plan must not be used from two threads at once.
 */
#ifndef HOLOGEN_H
#define HOLOGEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hg_plan_s *hg_plan;

typedef enum {
    HG_OK = 0,
    HG_ERR_INVALID_ARG = 1,      /* bad pointer, size, enum, or target values */
    HG_ERR_UNSUPPORTED_SIZE = 2, /* ny or nx has no compiled transform plan */
    HG_ERR_OOM = 3,              /* device allocation failed */
    HG_ERR_CUDA = 4,             /* a CUDA runtime call failed */
    HG_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up */
    HG_ERR_NUMERIC = 6,          /* target with zero energy */
    HG_ERR_TOO_LARGE = 7         /* hg_run_noalloc: a side above HG_NOALLOC_MAX_SIDE */
} hg_status;

/* SLM modulation (Section 3; Fig. 1).  BINARY: levels {0, pi}, level 0 iff
 * Re h >= 0 for the back-propagated field h.  LLEVEL: `levels` phases
 * 2 pi q / levels over the full circle, q = round-half-away(arg h /
 * (2 pi / levels)) mod levels, 2 <= levels <= 256.  AMPLITUDE (Fig. 1's
 * amplitude modulation; binary amplitude is levels = 2): transmittance
 * q / (levels - 1), q = round-half-away((levels - 1) (1/2 + m / (2 amp_clip)))
 * clamped to [0, levels - 1], where m = Re(h conj E) / |E|^2 is the
 * least-squares real transmittance under the illumination E (0 where E = 0)
 * and h is the unitary field of a target carrying sqrt(N) T; with levels = 2
 * that is q = 1 exactly where Re(h conj E) >= 0.  AMPLITUDE makes the plan
 * modulated (hg_opts.modulated). */
typedef enum { HG_SLM_BINARY = 0, HG_SLM_LLEVEL = 1, HG_SLM_AMPLITUDE = 2 } hg_slm_kind;
typedef struct {
    int kind;   /* hg_slm_kind */
    int levels; /* ignored for BINARY */
} hg_slm;

/* GS: Section 3.2.  WGS: GS whose target amplitude is multiplied by a weight
 * updated every iteration as w <- w T / sqrt(I) on pixels with T > 0, where
 * I is the energy-normalised replay intensity.  OSPR: Section 3.4, binary
 * SLM only, `subframes` independent random-phase subframes per target whose
 * replay intensities are averaged.  ADOSPR: adaptive OSPR (Section 3.4's
 * feedback variant), binary only: the subframes run in order and subframe n
 * (1-based) aims at the intensity deficit sqrt(max(n T^2 - S, 0)), S the sum
 * of the earlier subframes' energy-normalised intensities; same random
 * phases and outputs as OSPR.  LT: Liu-Taghizadeh GS (Section 3.2): only a
 * centred window of the replay field is constrained at first, and the window
 * grows each iteration (hg_opts lt_start, lt_grow): inside it the GS
 * constraint with the target carrying the replay's total energy, outside it
 * the replay field is left free; the first field is the windowed target.
 * DS / SA: the holographic search algorithms of Section 3.3, direct search
 * and simulated annealing, for phase SLMs (binary or L-level).  The initial
 * guess is the quantised back-propagation of the target with the initial
 * phase (GS's first half-step).  Each sweep (`iters` counts sweeps) visits
 * every SLM pixel once in raster order and tries the other binary level, or
 * for L levels level (q + 1 + r1 mod (L - 1)) mod L; the change is kept when
 * it lowers the intensity MSE, and under SA also when u < exp(-dE / tau_s)
 * with tau_s = sa_temp * MSE(initial guess) * sa_cool^s.  (u, r1): Philox
 * words 0 and 1 at counter {y*nx + x, sweep, target index, 2}, u = (word0 >>
 * 8) 2^-24.  The replay field is updated incrementally in shared memory, one
 * CTA per target, so ny * nx is limited to 16384 pixels and the thread
 * layout to nx with lcm(32, nx) <= 1024 (else HG_ERR_UNSUPPORTED_SIZE).
 * mse_out[b][s] is the MSE after sweep s; hg_get_metrics slot 3 holds the
 * number of accepted changes of the sweep instead of sum |R|^2. */
typedef enum { HG_GS = 0, HG_WGS = 1, HG_OSPR = 2, HG_ADOSPR = 3, HG_LT = 4, HG_DS = 5, HG_SA = 6 } hg_algo;

typedef struct {
    void *stream;      /* cudaStream_t to enqueue on; NULL = legacy default stream */
    uint64_t seed;     /* Philox4x32-10 key for drawn phases */
    int subframes;     /* OSPR subframes per target (>= 1); ignored otherwise */
    int precision;     /* 0 (default): FP32 transforms.  1..4: the row pass runs its
                          radix-32 DFT stages as tensor-core GEMMs (tcgen05, FP32
                          accumulation) with 1 FP16 hi+lo split operands, 2 FP16,
                          3 BF16 hi+lo, 4 BF16 (the 16-bit builds of Section 4.5);
                          rows of 1024 or 2048 samples (2048 = a radix-2 step
                          over two 1024-point halves) and ny a multiple of 4
                          (1024) or 2 (2048), else HG_ERR_UNSUPPORTED_SIZE;
                          not OSPR */
    int use_graph;     /* 1 = replay the iteration loop as a CUDA graph (default) */
    int pipeline;      /* -1 auto (default): TMA-fed passes where the size allows;
                          0: generic passes only; 1: require TMA-fed passes */
    int autotune;      /* 1 (default): time the candidate pass variants on the plan's
                          own buffers at creation and keep the fastest (cached per
                          device and shape); 0: first candidate; 2 + k: candidate k
                          for both passes (HG_ERR_UNSUPPORTED_SIZE if absent) */
    float lt_start;    /* LT: window side fraction of the first field, in (0, 1]
                          (default 0.25); constraint k uses min(1, lt_start +
                          (1 - lt_start) k / lt_grow) */
    int lt_grow;       /* LT: constraints over which the window grows to the full
                          field (>= 1, default 10) */
    int modulated;     /* 1: a modulated plan (implied by an AMPLITUDE SLM or a
                          non-zero fresnel).  Its SLM plane is lit by an
                          illumination field E (hg_set_illumination; uniform 1
                          until set) times the Fresnel term, and a region of
                          interest (hg_set_roi; the whole field until set)
                          limits the replay constraint and the metrics.  The
                          target is restricted to the ROI and normalised there;
                          inside the ROI the GS constraint uses sqrt(N) T (the
                          replay energy of a unit-modulus hologram, unitary
                          transforms), outside it the replay field is left free;
                          the first field is sqrt(N) T e^{i phase}.  Metrics
                          scale the replay to the ROI's energy, I = |R|^2 /
                          sum_ROI |R|^2, and average over the ROI; efficiency is
                          the energy on the target's support over all replay
                          energy.  GS only (not precision > 0), no
                          hg_debug_step, else HG_ERR_INVALID_ARG.  TMA-fed
                          row passes without paired rows where the size has them;
                          a TMA-fed column pass where the size has one that
                          stages E in shared memory, else the generic one
                          (pipeline 0: generic passes only; 1: both TMA-fed).
                          Default 0. */
    float fresnel;     /* Fresnel (mid-field) hologram, Section 2: the SLM-plane
                          field gains the quadratic phase fresnel * ((x - nx/2)^2
                          + (y - ny/2)^2) radians (pi dx^2 / (lambda z) for
                          pixel pitch dx at distance z); 0 (default): far field */
    float amp_clip;    /* AMPLITUDE SLM: the transmittance range [0, 1] spans
                          m in [-amp_clip, amp_clip]; > 0, default 2 */
    float sa_temp;     /* SA: initial temperature relative to the initial guess's
                          MSE (> 0, default 1e-3) */
    float sa_cool;     /* SA: temperature factor per sweep, in (0, 1] (default 0.9) */
    int host_chunks;   /* hg_run with host buffers (GS, WGS, LT, modulated): the batch
                          runs in this many even chunks, one chunk's copies
                          overlapping another's iterations, with results identical
                          to a whole-batch run; 0 (default): batches of 2^24 pixels
                          and more run a short lead chunk, about batch * 8 /
                          (iters + 8) targets, whose iterations hide the input copy
                          of one chunk holding the rest, and that call times its
                          copies and iterations; later calls with the same
                          iteration count take the chunk sizes this timing says
                          are fastest (two chunks when host copies are fast, a
                          growing sequence when they are slow); 1 copies the whole
                          batch first; >= 0 */
} hg_opts;

/* sizeof(hg_opts) as this library was built: a binding that lays the
 * structure out itself compares it with its own before the first call (no
 * counterpart in the paper). */
size_t hg_opts_size(void);

/* Fills *opts with the defaults: stream NULL, seed 0, subframes 24, lt_start
 * 0.25, lt_grow 10, modulated 0, fresnel 0, amp_clip 2, sa_temp 1e-3, sa_cool 0.9,
 * precision 0, use_graph 1, pipeline -1, autotune 1, host_chunks 0. */
void hg_opts_default(hg_opts *opts);

/* 1 if a line of n samples (a row of nx or a column of ny) has a compiled
 * transform plan, else 0. */
int hg_supported_length(int n);

/* Creates a plan for `batch` targets of ny x nx pixels on the current CUDA
 * device.  The parameters are those of the problem the paper states: its
 * program summary (two-dimensional Fourier holograms for SLMs with binary or
 * multi-level control, by one of the listed algorithm variants), Section 2
 * (an ny x nx field) and Section 4.7, whose quantiser is constructed from the
 * SLM's level range and level count before it is applied to any field.
 * Allocates the plan's device workspace (the field, the prepared
 * targets, weights, twiddle tables and metric partials).  opts may be NULL
 * (defaults).  Errors: HG_ERR_INVALID_ARG (out NULL, batch < 1, bad slm or
 * algo, OSPR with a non-binary SLM, subframes < 1, precision outside 0..4),
 * HG_ERR_UNSUPPORTED_SIZE, HG_ERR_OOM, HG_ERR_CUDA. */
hg_status hg_plan_create(hg_plan *out, int ny, int nx, int batch, hg_slm slm, hg_algo algo,
                         const hg_opts *opts);

/*
 * Runs the algorithm on a batch (Section 3.2 / 3.4).
 *  target      [batch][ny][nx] float, replay order, >= 0, finite, not all zero
 *              per target.  Normalised inside to sum T^2 = 1.
 *  init_phase  GS/WGS: [batch][ny][nx] float radians, replay order, the
 *              starting replay phase; NULL draws U[0, 2 pi) from Philox with
 *              counter {(y*nx + x) / 4, 0, target index, 1}, replay pixel
 *              y*nx + x taking output word (y*nx + x) mod 4.  OSPR: must be
 *              NULL (subframe n of target t: counter {(y*nx + x) / 4, n, t, 0},
 *              the same word).
 *  iters       GS/WGS iterations, >= 1.  OSPR / ADOSPR: ignored.
 *  holo_out    GS/WGS: [batch][ny][nx] uint8 level indices of the last
 *              iteration's hologram; OSPR: [batch][subframes][ny][nx].  NULL
 *              to skip.
 *  mse_out     GS/WGS: [batch][iters] double, intensity MSE
 *              mean((I - T^2)^2) of iteration k's replay (I = |R|^2 / sum|R|^2,
 *              T normalised); OSPR: [batch] double, the MSE of the
 *              time-averaged replay.  NULL to skip.
 * WGS weights start at 1 unless hg_set_weights was called since the last
 * run.  Errors: HG_ERR_INVALID_ARG (NULL target, iters < 1, OSPR with
 * init_phase, negative / NaN / infinite target values), HG_ERR_NUMERIC
 * (a target with zero energy), HG_ERR_OOM, HG_ERR_CUDA.  Value errors are
 * found on the device: with device pointers they are returned by hg_sync.
 */
hg_status hg_run(hg_plan plan, const float *target, const float *init_phase, int iters,
                 uint8_t *holo_out, double *mse_out);

/* Per-iteration metrics of the last hg_run: [batch][iters][4] double with
 * {intensity MSE, amplitude MSE of eq. (mse) on sqrt(I) vs T, diffraction
 * efficiency sum_{T>0}|R|^2 / sum|R|^2, sum |R|^2}; OSPR: [batch][1][4].
 * `count` is the number of doubles the buffer holds.  Errors:
 * HG_ERR_INVALID_ARG (no run yet, NULL, count too small). */
hg_status hg_get_metrics(hg_plan plan, double *out, size_t count);

/* Normalised replay intensity (sums to 1, replay order) of holograms of level
 * indices, i.e. |fftshift(FFT2(e^{iH}))|^2 / sum, the replay field of
 * Section 2, eq. (fouriertrans2d5c), under the scale freedom of Section 3.1
 * (OSPR plans time-average the subframes' intensities, Section 3.4): holo [batch][ny][nx] (OSPR plans: [batch][subframes][ny][nx],
 * time-averaged per target); intensity_out [batch][ny][nx] float. */
hg_status hg_replay(hg_plan plan, const uint8_t *holo, float *intensity_out);

/* Illumination of the SLM plane of a modulated plan (Section 4: the
 * quantiser is handed the illumination's phases and magnitudes; the paper
 * gives no further rule).  amp and phase: [ny][nx] float, natural SLM order
 * (NULL: 1 and 0).  The light leaving SLM pixel (y, x) is E = amp exp(i
 * (phase + Fresnel term)) times the pixel's modulation; phase SLMs pick the
 * level nearest arg(h conj E) and emit E e^{iH}, the AMPLITUDE SLM emits
 * E q / (levels - 1).  Applies to later runs.  Synchronises the plan's
 * stream.  Errors: HG_ERR_INVALID_ARG (NULL or unmodulated plan, a negative
 * or non-finite amplitude, a non-finite phase), HG_ERR_CUDA. */
hg_status hg_set_illumination(hg_plan plan, const float *amp, const float *phase);

/* Region of interest of a modulated plan (Section 2: many applications use
 * part of the replay field; metrics restricted to it give extra freedom):
 * roi [ny][nx] uint8, replay order, nonzero inside; NULL = the whole field.
 * Applies to later runs and hg_evaluate calls (the target is restricted to
 * the ROI, so a ROI that misses the target gives HG_ERR_NUMERIC at the
 * run).  Synchronises the plan's stream.  Errors: HG_ERR_INVALID_ARG (NULL
 * or unmodulated plan), HG_ERR_CUDA. */
hg_status hg_set_roi(hg_plan plan, const uint8_t *roi);

/* Metrics of given holograms (Section 3.1), on any plan: the replay of holo
 * (layout and SLM as in hg_replay, under the plan's illumination) against
 * target ([batch][ny][nx] float, replay order, >= 0, normalised inside over
 * the plan's region of interest), out [batch][5] double = {intensity MSE,
 * amplitude MSE of eq. (mse), efficiency, SSIM, sum |R|^2 (unitary)}.  The
 * replay intensity is scaled to the ROI's energy (I = |R|^2 / sum_ROI
 * |R|^2) and the means run over the ROI's pixels (the whole field for
 * unmodulated plans); efficiency = energy on the target's support in the
 * ROI over all replay energy.  SSIM is Section 3.1's formula over the whole
 * ROI (means, population variances and covariance; k1 = 0.01, k2 = 0.03,
 * dynamic range 1) of x = T / max T and y = sqrt(I) / max T, i.e. the
 * phase-insensitive (amplitude) variant.  Errors: HG_ERR_INVALID_ARG (NULL,
 * negative / NaN / infinite target values), HG_ERR_NUMERIC (a target with
 * no energy in the region of interest) -- both found on the device, so with
 * device pointers returned by hg_sync -- HG_ERR_OOM, HG_ERR_CUDA. */
hg_status hg_evaluate(hg_plan plan, const uint8_t *holo, const float *target, double *out);

/* Replay phase arg R after the last GS/WGS run (0 where R = 0), replay order,
 * [batch][ny][nx] float radians: the state from which a run resumes.  In
 * Section 3.2's loop this is the phase the replay-plane constraint keeps
 * when it replaces |R| by the target amplitude; the next iteration starts
 * from F = T e^{i arg R}.  Errors: HG_ERR_INVALID_ARG (NULL, no GS/WGS run
 * since the plan was created or since hg_replay / hg_debug_loop_step reused
 * the field, OSPR plans). */
hg_status hg_get_phase(hg_plan plan, float *phase_out);

/* WGS weights, replay order, [batch][ny][nx] float.  hg_set_weights makes the
 * next hg_run start from w instead of 1; hg_get_weights returns the weights
 * after the last run's final update. */
hg_status hg_set_weights(hg_plan plan, const float *w);
hg_status hg_get_weights(hg_plan plan, float *w_out);

/*
 * One GS/WGS iteration with its intermediate fields, for checking:
 *  h_out       [batch][ny][nx] complex64 (re, im) SLM-plane field
 *              IFFT2(ifftshift(w T e^{i phase})) before quantisation
 *  holo_out    [batch][ny][nx] uint8 level indices
 *  replay_out  [batch][ny][nx] complex64 replay field fftshift(FFT2(e^{iH}))
 *  metrics_out [batch][4] double as in hg_get_metrics
 * phase_in is required; WGS uses the weights set by hg_set_weights (else 1).
 * Any output may be NULL.
 */
hg_status hg_debug_step(hg_plan plan, const float *target, const float *phase_in, float *h_out,
                        uint8_t *holo_out, float *replay_out, double *metrics_out);

/*
 * One iteration of the fused LOOP (the row and column passes that hg_run
 * repeats between its first and last iteration, in the variants the plan
 * chose), started from a given hologram H_k, for checking the loop kernels
 * against one step of Section 3.2 (unitary DFT of Section 2, eqs.
 * fouriertrans2d5c/d).  GS, WGS, LT and modulated plans; DEVICE pointers only.
 *  holo_in     [batch][ny][nx] uint8 level indices H_k, natural SLM order.
 *  k           iteration index of H_k (LT: the row pass applies the window
 *              of constraint k + 1; ignored otherwise).
 *  row_out     [batch][ny][nx] complex64: the field the row pass leaves,
 *              G[ky][x] = sum_kx F[ky][kx] exp(+2 pi i kx x / nx) (an
 *              unnormalised inverse row DFT), ky and kx in DFT order, x in
 *              natural order, where F = A w T R / |R| (F = A for R = 0) with
 *              R = FFT2(E e^{iH_k}) unnormalised (E = 1 unless the plan is
 *              modulated), T the normalised target moved to DFT order, w the
 *              updated WGS weight (1 otherwise) and A = 1 (GS, WGS) or N
 *              (LT and modulated plans, where F = R outside the window or the
 *              region of interest).  When the plan runs the binary loop in
 *              Hermitian form (hg_plan_variant(plan, 0) contains "+herm") F
 *              is replaced by F_H(u) = (F(u) + conj F(-u)) / 2 and only rows
 *              ky <= ny/2 are defined.
 *  holo_out    [batch][ny][nx] uint8: H_{k+1}, the column pass's quantisation.
 *  col_out     [batch][ny][nx] complex64: the field the column pass leaves,
 *              sum_y E e^{iH_{k+1}[y][x]} exp(-2 pi i ky y / ny) (unnormalised
 *              forward column DFT); only rows ky <= ny/2 are defined when the
 *              row pass is paired (variant name contains "pair").
 *  metrics_out [batch][4] double: the metrics of iteration k (the replay of
 *              H_k), as in hg_get_metrics.
 * WGS starts from the weights set by hg_set_weights (else 1); the updated
 * weights are returned by hg_get_weights.  Any output may be NULL.  Errors:
 * HG_ERR_INVALID_ARG (NULL plan, target or holo_in, k < 0, OSPR or search
 * plans, a host pointer), HG_ERR_CUDA; device-detected value errors at
 * hg_sync.
 */
hg_status hg_debug_loop_step(hg_plan plan, const float *target, const uint8_t *holo_in, int k, float *row_out,
                             uint8_t *holo_out, float *col_out, double *metrics_out);

/* Waits for the plan's stream and reports errors found on the device since
 * the last run started (invalid or zero-energy targets, CUDA faults). */
hg_status hg_sync(hg_plan plan);

/* Number of kernels the last hg_run / hg_replay / hg_debug_step enqueued. */
int hg_last_launch_count(hg_plan plan);

/* Bit 0: the row pass of the iteration runs the TMA-fed kernel; bit 1: the
 * column pass does (hg_opts.pipeline, sizes and alignment decide). */
int hg_pipelined(hg_plan plan);

/* Name of the variant running the row (pass 0) or column (pass 1) pass of
 * the iteration loop ("generic" or the TMA-fed plan's radix/threads tag).
 * The string is static; NULL plan gives "". */
const char *hg_plan_variant(hg_plan plan, int pass);

/* Per-pass timing (diagnostics; no counterpart in the paper).
 * hg_profile_enable(plan, n) makes the next runs record a CUDA event pair on
 * the plan's stream around each of up to n row and column passes of the
 * iteration loop (the loop is then launched pass by pass, not as a graph);
 * n = 0 switches timing off.  hg_profile_read waits for the stream and
 * stores {row ms, row passes, column ms, column passes} accumulated since the
 * last read into out4[4]. */
hg_status hg_profile_enable(hg_plan plan, int max_passes);
hg_status hg_profile_read(hg_plan plan, double *out4);

/* Failure-injection hook for tests (no counterpart in the paper).  The
 * TMA-fed passes bound every device-side wait by `wait_ns` nanoseconds
 * (default 2 s); when a wait runs out the kernel stops, sets an error bit and
 * the next hg_sync returns HG_ERR_TIMEOUT, with the context still usable.
 * drop_job >= 0 makes the producer of the next runs never issue that job's
 * copy (job = item * panels + panel in the pass's order), so the consumer's
 * wait runs out; -1 restores normal operation.  Errors: HG_ERR_INVALID_ARG. */
hg_status hg_debug_inject(hg_plan plan, int drop_job, uint64_t wait_ns);

void hg_plan_destroy(hg_plan plan);
const char *hg_status_string(hg_status st);

/*
 * Groups: targets of different sizes (each size a plan) run as ONE CUDA graph
 * holding the plans' whole GS/WGS runs, one after another or as concurrent
 * branches (hg_group_set_schedule).
 * This serves mixed batches such as 512^2, 1024^2, 2048^2 and 1080 x 1920
 * targets side by side (Section 2 notes that field size is a free parameter;
 * the batch mix itself has no counterpart in the paper).
 *  hg_group_create  nplans in [1, HG_GROUP_MAX] GS/WGS plans on one device.
 *                   The group keeps the plan handles (not owned; they must
 *                   outlive the group and must not run on their own while a
 *                   group run is in flight).
 *  hg_group_run     per plan i: targets[i], init_phases[i] (array may be NULL,
 *                   entries may be NULL), holo_out[i], mse_out[i] (arrays or
 *                   entries may be NULL) exactly as in hg_run; DEVICE buffers
 *                   only.  WGS weights restart at 1.  The graph is captured on
 *                   the first call and replayed while iters and every buffer
 *                   pointer stay the same.  Enqueued on `stream` (NULL:
 *                   legacy default stream).
 *  hg_group_sync    waits for `stream` and returns the first error any plan's
 *                   device flag reports.
 * Errors: HG_ERR_INVALID_ARG (NULL, counts, host pointers, OSPR plans),
 * HG_ERR_OOM, HG_ERR_CUDA.
 */
#define HG_GROUP_MAX 16
typedef struct hg_group_s *hg_group;
hg_status hg_group_create(hg_group *out, int nplans, const hg_plan *plans);
hg_status hg_group_run(hg_group group, const float *const *targets, const float *const *init_phases,
                       int iters, uint8_t *const *holo_out, double *const *mse_out, void *stream);
hg_status hg_group_sync(hg_group group, void *stream);
int hg_group_launch_count(hg_group group);
/* Order of the plans' runs inside the group's graph: HG_GROUP_SERIAL (the
 * default) runs them one after another, HG_GROUP_CONCURRENT as concurrent
 * branches.  Every pass of a size of 512^2 and up fills the GPU on its own,
 * so concurrent branches only contend for the SMs and the L2; concurrency can
 * pay for many small plans.  The next hg_group_run captures the graph again.
 * Errors: HG_ERR_INVALID_ARG (NULL group, unknown schedule). */
#define HG_GROUP_SERIAL 0
#define HG_GROUP_CONCURRENT 1
hg_status hg_group_set_schedule(hg_group group, int schedule);
void hg_group_destroy(hg_group group);

/*
 * hg_run_noalloc -- one GS or WGS run of ONE target that allocates no
 * device memory.  The paper has no counterpart: it is a deployment variant
 * of hg_run, not part of the method.
 *
 * Who needs it: callers that must not allocate device memory at the moment
 * they compute a hologram.  Examples: a display loop that refreshes an SLM
 * within a fixed frame time (cudaMalloc and cudaFree may synchronise the
 * whole device and take milliseconds, stalling every other stream); an
 * application whose device memory is owned by another framework's pool or
 * capped at a size it may not exceed; code that must not meet an
 * out-of-memory error once it is running.  hg_run cannot serve them because
 * creating a plan allocates its workspace.
 *
 * What it computes: the same as hg_run with the same arguments on a plan of
 * batch 1 created with opts.pipeline = 0 (the generic row and column
 * passes) and opts.seed = 0.  Holograms and mse_out agree with that call.
 *
 * Where the work memory lives: one fixed region of HG_NOALLOC_SCRATCH_BYTES
 * (about 4 MiB) of static device memory inside this library, reserved on
 * each device where the library's kernels are loaded, and reused by every
 * call on that device.  Its size is the limit: ny and nx must each be at
 * most HG_NOALLOC_MAX_SIDE and supported lengths; a larger side returns
 * HG_ERR_TOO_LARGE before any device work (use a plan for such sizes).  Each
 * call clears the region's device error flag itself; nothing else in it has
 * to start at zero.
 *
 *  ny, nx, slm, algo  as hg_plan_create (algo HG_GS or HG_WGS; WGS weights
 *              start at 1 on every call).
 *  target, init_phase, iters, holo_out, mse_out  as hg_run with batch 1, but
 *              every pointer must be a DEVICE pointer (host pointers would
 *              need staging buffers).  init_phase NULL draws the Philox
 *              phases of seed 0.
 *  stream      cudaStream_t to run on (NULL: the legacy default stream).
 * The call waits for its work on `stream` to finish before it returns, so
 * device-detected errors (bad target values, zero energy) are returned by
 * the call itself.
 *
 * One-time setup: the first call on each device looks up the region's
 * address and sets the kernel attributes of every supported length up to
 * HG_NOALLOC_MAX_SIDE.  Make that first call before any stream capture
 * begins on that device.
 *
 * Concurrency: all calls on one device share the one region.  Calls that
 * overlap in time, for example from two host threads, overwrite each other's
 * data and give wrong results: serialise them.  Calls on different devices
 * are independent, and plans are unaffected (they own their memory).
 *
 * Errors: HG_ERR_INVALID_ARG (NULL target, iters < 1, OSPR, bad slm, a host
 * pointer, negative / NaN / infinite target values), HG_ERR_TOO_LARGE,
 * HG_ERR_UNSUPPORTED_SIZE (a length with no compiled plan),
 * HG_ERR_NUMERIC (a target with zero energy), HG_ERR_CUDA.
 */
#define HG_NOALLOC_MAX_SIDE 512
#define HG_NOALLOC_SCRATCH_BYTES 4222208u
hg_status hg_run_noalloc(int ny, int nx, hg_slm slm, hg_algo algo, const float *target,
                         const float *init_phase, int iters, uint8_t *holo_out, double *mse_out,
                         void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HOLOGEN_H */
