/*
 * libfdas — GB300 (sm_103a) Fourier Domain Acceleration Search hot path.
 *
 * The library turns the time series of one dispersion-measure trial into the
 * frequency/frequency-derivative (f-z) power plane and its harmonic-summed peak list,
 * following arXiv:2206.12205 (White et al., "Bits missing: finding exotic pulsars using
 * bfloat16 on NVIDIA GPUs"):
 *
 *   x[N] --(long real FFT, FP32; Sec. 3)--> X[Nb]                          fdas_spectrum
 *        --(overlap-save correlation with K acceleration templates;
 *           Sec. 2.1, Fig. fdas_flow "blue box"; BF16 variant Sec. 3)--> P[K][Nb]   fdas_plane
 *        --(harmonic sum + threshold + local maxima; Sec. 2.1)--> peaks        fdas_peaks
 *   peaks --(gradient ascent on the interpolated power)--> sub-bin (r, z)  fdas_refine
 *
 * fdas_search runs all three.  Every step runs in this library's CUDA kernels.
 *
 * Conventions used by every entry point:
 *   - Nb = N/2 frequency bins (the Nyquist bin is dropped), bin 0 (DC) is set to zero.
 *   - Spectrum normalisation: Xhat = X * sqrt(2/sigma2), sigma2 = mean |X_k|^2 over
 *     k = 1..Nb-1 (or the fixed value in fdas_config.sigma2), so that noise-only plane
 *     cells follow chi^2 with 2 degrees of freedom (Sec. 5.1).  A series with no power
 *     outside DC (all zero or constant: sigma2 = 0) normalises to Xhat = 0, a zero plane
 *     and no candidates.
 *   - Templates: K = zmax + 1 rows at z_i = -zmax + 2i (z = fdot T^2 in bins, Eq. fdotz);
 *     m taps at q = -m/2 .. m/2-1 of the response of a constant-fdot sinusoid
 *     I(q, z) = int_0^1 exp(i pi (z u^2 - 2 q u)) du, scaled to unit norm (Sec. 3.3).
 *   - Plane: P[i][r] = | sum_q Xhat[r+q] conj(T_i(q)) |^2, r = 0..Nb-1, row-major [K][Nb]
 *     (r contiguous); Xhat is zero outside [0, Nb).  Element type is bfloat16 (the upper
 *     16 bits of the float) for FDAS_BF16 and FDAS_BF16_DIRECT, float otherwise.
 *   - The tensor-core DFT precisions (FDAS_BF16, FDAS_BF16_SPLIT, FDAS_FP16_SCALED) run their
 *     overlap-save with 4096-bin segments whatever seg_len says (the plane does not depend
 *     on it) and accept at most 2048 taps.
 *   - All device pointers are CUDA device addresses on the current device; the caller
 *     owns them.  Alignment: series and spectra 8 bytes, plane 16 bytes, workspace 256
 *     bytes, peak list and counts 4 bytes (cudaMalloc'd and torch buffers satisfy all of
 *     these); a misaligned pointer is rejected with FDAS_E_INVALID.  Streams are
 *     cudaStream_t values passed as void* (NULL = default stream).  Calls are asynchronous
 *     unless stated.  Nothing inside fdas_spectrum, fdas_plane, fdas_peaks or fdas_search
 *     allocates memory.
 *   - A workspace serves one call at a time: it holds the call's spectrum, segment spectra,
 *     peak units and counters, so calls that share one must be ordered (one stream).
 *   - Errors are returned as fdas_status; nothing is thrown across the ABI.  Device-side
 *     conditions (peak-list overflow, a wait that ran out) are recorded in a sticky
 *     per-plan status word read by fdas_device_status.
 */
#ifndef FDAS_H
#define FDAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FDAS_OK = 0,
    FDAS_E_INVALID = 1,      /* an argument is out of range or a pointer is NULL          */
    FDAS_E_UNSUPPORTED = 2,  /* a valid request this build does not implement             */
    FDAS_E_NOMEM = 3,        /* a plan-time allocation failed                             */
    FDAS_E_CUDA = 4,         /* a CUDA call or kernel launch failed (fdas_last_error)     */
    FDAS_E_OVERFLOW = 5,     /* more peaks than fdas_config.max_peaks                     */
    FDAS_E_TIMEOUT = 6,      /* a bounded device wait gave up                             */
    FDAS_E_STATE = 7         /* call out of order (e.g. a search before make_templates)   */
} fdas_status;

typedef enum {
    FDAS_FP32 = 0,           /* FP32 plane, FP32 CUDA-core FFTs                           */
    FDAS_BF16 = 1,           /* BF16 spectrum/templates, tensor-core DFT stages with FP32
                                accumulation, BF16 plane (Sec. 3)                          */
    FDAS_BF16_SPLIT = 2,     /* compensated hi+lo BF16 operands (three products per MMA step,
                                about 16 significant bits), FP32 plane                      */
    FDAS_FP16_SCALED = 3,    /* ablation of Sec. 3.2 (FP16 rejected there for its range): FP16
                                operands on the tensor cores with a power-of-two scale per
                                segment (largest component in [0.5, 1)) and the template bank
                                scaled by the segment length, so no operand overflows and small
                                ones stay normal; FP32 accumulation; FP32 plane               */
    FDAS_BF16_DIRECT = 4,    /* direct correlation variant: the spectrum (BF16) times the
                                time-domain taps (BF16) as one tensor-core GEMM per block of
                                bins (the Hankel matrix of the spectrum against all K
                                templates), FP32 accumulation, BF16 plane; no segment FFTs.
                                Needs 2 ceil(K/8) 8 <= 256 and the taps image plus windows in
                                shared memory (K <= 128; taps <= 256 at K = 85), else
                                FDAS_E_UNSUPPORTED                                            */
    FDAS_FP8_DIRECT = 5      /* precision ablation of Sec. 3 below BF16: the direct form with
                                FP8 E4M3 operands (3 mantissa bits), the spectrum scaled by a
                                power of two per 1024-bin tile and each template by its own,
                                so that the largest |Re| or |Im| lands in [224, 448]; FP32
                                accumulation; FP32 plane with the scales divided out.  Needs
                                taps % 16 == 0 and the taps image (ceil(K/32) x 64 rows x 2
                                taps bytes) plus the windows in one CTA's shared memory (taps
                                <= 416 at K = 85), else FDAS_E_UNSUPPORTED                     */
} fdas_precision;

/* Device status bits (fdas_device_status). */
#define FDAS_DEV_PEAK_OVERFLOW 0x1
#define FDAS_DEV_TIMEOUT       0x2

/* Search configuration for one series (one DM trial). */
typedef struct {
    int64_t n_samples;   /* N: power of two, 2^11 .. 2^27                                  */
    int32_t zmax;        /* even, 0 .. 1022; K = zmax + 1 template rows                    */
    int32_t taps;        /* m: even, 2 .. seg_len/2                                        */
    int32_t seg_len;     /* S: overlap-save segment, 1024, 2048, 4096 or 8192 bins; the
                            plane does not depend on it (linear-correlation identity)       */
    int32_t precision;   /* fdas_precision                                                 */
    int32_t max_harm;    /* highest harmonic-sum level: 1, 2, 4, 8 or 16                   */
    float   thr[5];      /* peak thresholds on S_H for H = 1, 2, 4, 8, 16                   */
    int32_t max_peaks;   /* capacity of the caller's peak buffer, >= 0                      */
    double  sigma2;      /* 0: estimate sigma2 from the spectrum; > 0: use this value       */
    int32_t norm_block;  /* 0: one normalisation for the whole spectrum (sigma2 above); a
                            power of two 64 .. 65536: robust local normalisation instead, each
                            block of this many bins scaled by sqrt(2 ln 2 / median |X_k|^2)
                            over the block (k >= 1; exclusive with sigma2 > 0)               */
    int32_t harm_mode;   /* 0: harmonic sums anchored at the fundamental, every term on the
                            grid (S_H(r, z) = sum_h P(h r, h z), H r < Nb, |H z| <= zmax);
                            1: anchored at the highest harmonic with rounding (a variant):
                            the cell (r, z) is harmonic H and harmonic j < H is read at
                            (round(j r / H), the grid z nearest j z / H), halves rounded up,
                            nested so that S_2H = S_H + the odd j of 2H in increasing j;
                            every level covers the whole plane; records give the cell      */
} fdas_config;

/* One peak record, 16 bytes, ordered by (series, harm, zi, r) in the output list. */
typedef struct {
    uint32_t series;     /* series index (0 for single-series calls)                        */
    uint32_t r;          /* frequency bin of the fundamental                                 */
    int16_t  zi;         /* template row; z = -zmax + 2 zi                                   */
    uint8_t  harm;       /* harmonic-sum level H (1, 2, 4, 8, 16)                            */
    uint8_t  pad;        /* 0                                                                */
    float    power;      /* S_H(r, zi): the summed normalised power                          */
} fdas_peak;

/* Sizes derived by fdas_plan. */
typedef struct {
    int64_t nb;              /* N/2 frequency bins                                           */
    int32_t K;               /* template rows                                                */
    int32_t seg_valid;       /* L plane bins kept per segment: S - m + 1 rounded down to a
                                multiple of 32 (FP32) or of 64 (tensor-core DFT paths)          */
    int64_t n_seg;           /* ceil(Nb / L) overlap-save segments                            */
    int32_t plane_elem_bytes;/* 2 for FDAS_BF16 and FDAS_BF16_DIRECT, else 4                  */
    int64_t plane_bytes;     /* K * Nb * plane_elem_bytes                                     */
    size_t  workspace_bytes; /* caller-provided scratch for fdas_search                       */
    int64_t cells;           /* K * Nb                                                        */
} fdas_plan_info;

typedef struct fdas_plan_s *fdas_plan_t;

/*
 * Validate cfg, derive sizes and create a plan (host only: no device work, no device
 * allocation).  On success *plan receives a new plan and *workspace_bytes (nullable) the
 * size of the scratch buffer fdas_search needs.
 * Errors: FDAS_E_INVALID for a NULL pointer or a value outside the ranges above;
 * FDAS_E_UNSUPPORTED for a precision this build does not implement.
 */
fdas_status fdas_plan(const fdas_config *cfg, fdas_plan_t *plan, size_t *workspace_bytes);

/* Copy the derived sizes of a plan into *info.  Host only. */
fdas_status fdas_plan_get_info(fdas_plan_t plan, fdas_plan_info *info);

/*
 * Build the template bank on the current device (Sec. 3.3: templates generated once, then
 * converted to the working precision).  Allocates plan-owned device memory (freed by
 * fdas_destroy): the responses I(q, z_i) are integrated in FP64 (Gauss-Legendre), scaled
 * to unit norm, and their length-S DFTs G_i(k) = (1/S) sum_d T_i(d - m/2) e^{-2 pi i d k/S}
 * stored in FP32 (and in BF16 hi/lo for the BF16 precisions).  Synchronises the stream.
 * Errors: FDAS_E_NOMEM, FDAS_E_CUDA.
 */
fdas_status fdas_make_templates(fdas_plan_t plan, void *stream);

/*
 * Long real FFT [Sec. 3, kept in FP32]: d_series holds N float samples; d_xhat receives
 * Nb complex values (interleaved float re, im) of the normalised spectrum Xhat with
 * Xhat[0] = 0.  d_workspace: fdas_plan's workspace_bytes.  d_sigma2 (nullable, device):
 * receives sigma2 as a double.
 * Errors: FDAS_E_INVALID (NULL pointer), FDAS_E_STATE (no templates yet), FDAS_E_CUDA.
 */
fdas_status fdas_spectrum(fdas_plan_t plan, const float *d_series, void *d_workspace,
                          float *d_xhat, double *d_sigma2, void *stream);

/*
 * The f-z plane from a normalised spectrum [Sec. 2.1 overlap-save; Fig. fdas_flow blue
 * box]: segment FFTs of length S with stride L, per-template complex multiply, inverse
 * FFT, |.|^2 and overlap discard.  d_xhat: Nb interleaved complex floats.  d_plane:
 * K*Nb elements of the plan's plane type.  This is the step the throughput metric times.
 * Errors: FDAS_E_INVALID, FDAS_E_STATE, FDAS_E_CUDA.
 */
fdas_status fdas_plane(fdas_plan_t plan, const float *d_xhat, void *d_workspace,
                       void *d_plane, void *stream);

/*
 * fdas_plane for callers that must not allocate device memory at call time (no counterpart
 * in the paper).  Such callers include code running while a CUDA stream is being captured
 * into a graph, real-time pipelines that reserve all device memory at start-up and forbid
 * allocation later, and hosts whose own allocator owns the device's memory.  The result is
 * the same plane as fdas_plane; the segment spectra live in a library-owned static device
 * array of FDAS_STATIC_SCRATCH_BYTES (reserved on every GPU that loads the library, until the
 * process exits) instead of the workspace.
 *   - Only FDAS_FP32 plans with n_seg * S * 8 <= FDAS_STATIC_SCRATCH_BYTES are accepted
 *     (e.g. S = 8192 up to N = 2^23); larger ones return FDAS_E_UNSUPPORTED with the sizes in
 *     fdas_last_error.
 *   - The first call on a device looks up the array's device address (once per device, with
 *     that device current); make that first call before any stream capture.  The address is
 *     kept for the life of the process: after cudaDeviceReset of that device, do not call
 *     fdas_plane_static again in the same process.
 *   - The plan's device (the one current at fdas_make_templates) must be current, else
 *     FDAS_E_INVALID (with both device numbers in fdas_last_error).
 *   - All calls share the one array: calls whose work overlaps on the GPU (different streams,
 *     or different plans at once) race on it.  Each call overwrites the whole part it reads,
 *     so no clearing is needed between calls.
 *   - Allocates nothing; the plan's templates must exist (fdas_make_templates, which does
 *     allocate, called earlier), else FDAS_E_STATE.
 * Errors: FDAS_E_INVALID, FDAS_E_STATE, FDAS_E_UNSUPPORTED, FDAS_E_CUDA.
 */
#define FDAS_STATIC_SCRATCH_BYTES ((size_t)40 << 20)
fdas_status fdas_plane_static(fdas_plan_t plan, const float *d_xhat, void *d_plane, void *stream);

/*
 * Harmonic sums and peak list of a plane [Sec. 2.1]: for H = 1, 2, 4, .. max_harm,
 * S_H(r, i) = sum_{h=1..H} P(h r, i_h) with z_{i_h} = h z_i (summed in FP32 in the order
 * h = 1..H), defined where |H z_i| <= zmax and H r < Nb.  A cell is a peak when
 * S_H > thr[level] and it beats each defined 3x3 neighbour (strictly for neighbours earlier
 * in row-major (i, r) order, or equal for later ones).  Peaks are written to d_peaks in
 * (harm, zi, r) order, at most max_peaks of them; *d_npeaks (device int32) receives the
 * true count, and a count above max_peaks also sets FDAS_DEV_PEAK_OVERFLOW.
 * The records are written from the list of (level, row, 512-bin chunk) units that hold peaks by
 * one block; when more than 1024 units hold peaks (low thresholds) one block per SM scans every
 * unit's count instead (5.8 million peaks at N = 2^23, 85 templates: about 0.4 ms for the
 * output, beside 8.5 ms for the harmonic sums' local-maximum tests).
 * Errors: FDAS_E_INVALID, FDAS_E_STATE, FDAS_E_CUDA.
 */
fdas_status fdas_peaks(fdas_plan_t plan, const void *d_plane, void *d_workspace,
                       fdas_peak *d_peaks, int32_t *d_npeaks, void *stream);

/*
 * The order in which fdas_peaks searches levels 2..16 over level 2's region (the harmonic sums
 * above; rows with |2 z_i| <= zmax, bins r < Nb/2 rounded up to 512-bin chunks), as blocks of
 * four consecutive chunks of one row: entry k = (row - first row of the region) << 16 | block.
 * Cell (r, z) gathers harmonic h at (h r, h z), on its own ray through the origin, so the blocks
 * are taken by increasing z / (middle bin of the block), ties by row then block, which keeps the
 * reads of each plane sector close together in time.  Host only (computed from the plan; the
 * same table is uploaded by fdas_make_templates).  h_order (host, nullable) receives
 * *n_out entries when capacity >= *n_out.
 * Errors: FDAS_E_INVALID (NULL plan or n_out, capacity too small for a non-NULL h_order);
 * FDAS_E_UNSUPPORTED if the region has 2^16 rows or blocks or more (outside the plan limits).
 */
fdas_status fdas_levels_order(fdas_plan_t plan, uint32_t *h_order, int64_t capacity, int64_t *n_out);

/*
 * Whole path for one series: fdas_spectrum (into the workspace), fdas_plane, fdas_peaks.
 * d_plane must hold plane_bytes.  Same errors as the three steps.
 */
fdas_status fdas_search(fdas_plan_t plan, const float *d_series, void *d_workspace,
                        void *d_plane, fdas_peak *d_peaks, int32_t *d_npeaks, void *stream);

/*
 * Band maxima of a plane (the paper's harmonic-band analysis, Sec. 4.3, Table harm_bounds: with
 * the fundamental f known, band n spans frequencies [(n+0.5) f, (n+1.5) f], the fundamental's
 * [0, 1.5 f], and the highest cell of band n is taken as harmonic n).  Band b covers bins
 * [h_lo[b], h_hi[b]] of every template row (host arrays, clipped to [0, Nb)); d_value[b],
 * d_r[b], d_zi[b] receive the largest value in it and the first cell holding it in row-major
 * (zi, r) order, or -1 in all three for a band with no cell.  d_plane: the plan's plane type.
 * d_scratch: 24 * n_bands bytes, 8-byte aligned (the host bounds are copied into it).
 * Errors: FDAS_E_INVALID (NULL or misaligned pointer, n_bands < 0, lo > hi);
 * FDAS_E_UNSUPPORTED when K * Nb >= 2^32; FDAS_E_CUDA.
 */
fdas_status fdas_band_max(fdas_plan_t plan, const void *d_plane, const int64_t *h_lo,
                          const int64_t *h_hi, int32_t n_bands, void *d_scratch, float *d_value,
                          int64_t *d_r, int32_t *d_zi, void *stream);

/*
 * Copy the frequency-domain template bank G[K][S]/*
 * Copy the frequency-domain template bank G[K][S] (interleaved complex float, FP32) to the
 * device buffer d_out (K*S*8 bytes).  For verification.
 * Errors: FDAS_E_INVALID, FDAS_E_STATE, FDAS_E_CUDA.
 */
fdas_status fdas_get_templates(fdas_plan_t plan, float *d_out, void *stream);

/*
 * Failure-detection self-check of the bounded waits.  Launches one block on the stream whose
 * thread waits on an mbarrier that nothing arrives on, in the bounded form every wait of the
 * plane kernels has, for at most max_cycles SM clock cycles (1 .. 2^36; at 2 GHz 2e9 is about
 * one second).  When the bound runs out the block sets FDAS_DEV_TIMEOUT in the plan's status
 * word and returns, leaving the context usable; read it with fdas_device_status.  Needs
 * fdas_make_templates first (the status word).  Errors: FDAS_E_INVALID, FDAS_E_STATE,
 * FDAS_E_CUDA.
 */
fdas_status fdas_check_timeout(fdas_plan_t plan, int64_t max_cycles, void *stream);

/*
 * Read (and clear when clear != 0) the plan's sticky device status word
 * (FDAS_DEV_* bits).  Synchronises the device.  Errors: FDAS_E_INVALID, FDAS_E_CUDA.
 */
fdas_status fdas_device_status(fdas_plan_t plan, int32_t *bits, int clear);

/* A point of the f-z plane at sub-bin resolution: r is the frequency bin at the start of the
 * observation (the plane's r axis) and z the drift in bins over the observation (Eq. fdotz). */
typedef struct {
    double r;
    double z;
} fdas_cand;

/* Largest step count fdas_refine accepts. */
#define FDAS_REFINE_MAX_STEPS 1000

/*
 * Fourier-interpolated power between the plane's grid points and its gradient (the f-z plane of
 * Sec. 2.1 evaluated at fractional (r, z); the derivatives are the adjoint sums of the same
 * interpolation).  For each point:
 *   A = sum_{k = k0-m/2}^{k0+m/2-1} Xhat_k conj(I(k - r, z)),  P = |A|^2,
 * with the unnormalised response I(q, z) = int_0^1 exp(i pi (z u^2 - 2 q u)) du, the plan's m
 * taps, and Xhat_k = 0 outside [0, Nb).
 *   d_xhat  Nb interleaved complex floats (a normalised spectrum, as from fdas_spectrum).
 *   d_pts   n points; d_k0 (nullable) n window anchors, NULL meaning floor(r + 1/2) per point.
 *   fp64    0: FP32 arithmetic (phases of large argument reduced in FP64); 1: FP64 throughout.
 *   d_out   n x 3 doubles: P, dP/dr, dP/dz.  A non-finite point, |r| >= 2^52, |z| >= 2^20 or an
 *           anchor 2^24 or more bins from r gives NaN in all three.
 * Device pointers 8-byte aligned.  Needs no templates (fdas_make_templates not required).
 * Errors: FDAS_E_INVALID (NULL or misaligned pointer, n < 0, fp64 not 0 or 1), FDAS_E_CUDA.
 */
fdas_status fdas_interp_power(fdas_plan_t plan, const float *d_xhat, const fdas_cand *d_pts,
                              const int64_t *d_k0, int32_t n, int32_t fp64, double *d_out, void *stream);

/*
 * Sub-bin candidate refinement: gradient ascent on the interpolated power of fdas_interp_power,
 * one warp per candidate.  From each seed in d_in, with the window anchored at
 * k0 = floor(r_seed + 1/2) for the whole ascent: up to `steps` FP32 steps, then one FP64 step, of
 *   d = (1/(2 pi^2)) [[48, -90], [-90, 180]] grad P / P
 * (the inverse Hessian of 1 - P/P_peak of an ideal chirp, i.e. a Newton step on a matched
 * response), scaled to |dr| <= 1/4 and |dz| <= 1 and halved up to three times until P does not
 * decrease; a candidate stops early when no such step exists.
 *   d_out    n refined points (may equal d_in).
 *   d_power  (nullable) n x 3 doubles: FP64 P, dP/dr, dP/dz at the refined point.
 *   d_evals  (nullable) n int32: power evaluations spent on each candidate.
 * A seed that fdas_interp_power would reject is copied unchanged with NaN power.
 * Device pointers 8-byte aligned (d_evals 4).  Needs no templates.
 * Errors: FDAS_E_INVALID (NULL or misaligned pointer, n < 0, steps outside
 * 0..FDAS_REFINE_MAX_STEPS), FDAS_E_CUDA.
 */
fdas_status fdas_refine(fdas_plan_t plan, const float *d_xhat, const fdas_cand *d_in, int32_t n,
                        int32_t steps, fdas_cand *d_out, double *d_power, int32_t *d_evals, void *stream);

/*
 * Batched search over many series: dispersion-measure trials of uneven length and zmax, one
 * configuration each (the paper searches every trial of a dedispersed observation; Sec. 2.1).
 * Series with the same (n_samples, zmax, taps, seg_len, precision) share one template bank.
 * All series run in one CUDA graph (captured on a library-owned stream the first time a set of
 * buffers is seen, relaunched on the caller's stream afterwards).  The graph has `lanes`
 * concurrent branches (default 1; fdas_batch_set_lanes, or chosen by fdas_batch_autotune): the
 * series are dealt to the lanes largest first, each to the least loaded, and run back to back
 * inside a lane; each lane reuses one workspace slice and one plane buffer sized for the largest
 * series, so device memory (lanes x that) does not grow with the number of series.
 */
typedef struct fdas_batch_s *fdas_batch_t;

/*
 * Validate and plan n_series configurations (host only).  *workspace_bytes (nullable)
 * receives the scratch fdas_batch_search needs.  Errors: as fdas_plan for any series;
 * FDAS_E_INVALID for n_series <= 0 or NULL pointers.
 */
fdas_status fdas_batch_plan(const fdas_config *cfgs, int32_t n_series, fdas_batch_t *batch,
                            size_t *workspace_bytes);

/*
 * Autotune (optional, before fdas_batch_make_templates; allocates and runs on the current
 * device): for each FP32 group, time the segment lengths S = 1024 .. 8192 (S >= 2 taps) and
 * 1 .. 16 templates per correlation CTA on a zero spectrum, keep the fastest and re-plan the
 * group's series with it (the plane does not depend on S); then build the template banks and
 * time the whole batch on a zero input at 1 .. 4 lanes and keep the fastest (this allocates the
 * packed input's size and four lanes' workspace for the duration of the call).  Choices are read
 * from and written to the JSON file cache_path (nullable: no cache), keyed by the device and the
 * group's or the batch's shape.  The workspace size may change: read it again with
 * fdas_batch_get_info.
 * Errors: FDAS_E_STATE after templates exist; FDAS_E_INVALID when the cache cannot be written;
 * FDAS_E_NOMEM, FDAS_E_CUDA.
 */
fdas_status fdas_batch_autotune(fdas_batch_t batch, const char *cache_path, void *stream);

/*
 * Set the number of concurrent lanes of a batch (1 .. FDAS_BATCH_MAX_LANES; host only, any time
 * before a search; the next fdas_batch_search captures its graph again).  *workspace_bytes
 * (nullable) receives the new workspace size, lanes x (the largest series' scratch + plane).
 * Peak lists do not depend on the lane count.  Errors: FDAS_E_INVALID.
 */
#define FDAS_BATCH_MAX_LANES 8
fdas_status fdas_batch_set_lanes(fdas_batch_t batch, int32_t lanes, size_t *workspace_bytes);

/* Build the template banks (one per group) on the current device.  Synchronises the stream. */
fdas_status fdas_batch_make_templates(fdas_batch_t batch, void *stream);

/*
 * Search every series.  d_series: the series packed back to back (series i starts at element
 * sample_offset(i) = sum of the earlier n_samples, 8-byte aligned).  d_workspace: the batch's
 * workspace_bytes (256-byte aligned).  d_peaks: one region of cfgs[i].max_peaks records per
 * series, region i at record peak_offset(i) = sum of the earlier max_peaks, each record's
 * series field = i; d_npeaks: n_series true counts (overflow as in fdas_peaks).
 * Errors: FDAS_E_INVALID, FDAS_E_STATE (no templates), FDAS_E_CUDA.
 */
fdas_status fdas_batch_search(fdas_batch_t batch, const float *d_series, void *d_workspace,
                              fdas_peak *d_peaks, int32_t *d_npeaks, void *stream);

/* Totals of a batch (each pointer nullable). */
fdas_status fdas_batch_get_info(fdas_batch_t batch, int32_t *n_series, size_t *workspace_bytes,
                                int64_t *total_samples, int64_t *total_peaks, int64_t *total_cells);

/* One series of a batch: its plan sizes, configuration (seg_len as tuned), offsets and group. */
fdas_status fdas_batch_series_info(fdas_batch_t batch, int32_t series, fdas_plan_info *info,
                                   fdas_config *cfg, int64_t *sample_offset, int64_t *peak_offset,
                                   int32_t *group);

/* OR of every series' sticky device status word (synchronises; clears when clear != 0). */
fdas_status fdas_batch_device_status(fdas_batch_t batch, int32_t *bits, int clear);

/* Text of the batch's last error ("" if none). */
const char *fdas_batch_last_error(fdas_batch_t batch);

/* Free a batch, its plans and template banks (NULL is ignored).  Synchronises the device. */
void fdas_batch_destroy(fdas_batch_t batch);

/* Per-stage device times of profiled calls (CUDA events on the caller's stream). */
typedef struct {
    int64_t calls;          /* entry-point calls that launched work since the last reset        */
    int64_t launches;       /* libfdas kernels launched by those calls                          */
    int64_t n_timed[4];     /* timed launch groups per stage: spectrum, segments, correlate, peaks */
    double  ms[4];          /* their summed event times in milliseconds                         */
    int64_t n_timed_peaks[2]; /* inside the peaks stage: level-1 pass, level 2..16 pass          */
    double  ms_peaks[2];    /* their summed event times in milliseconds                         */
    int64_t level1_fused;   /* peak searches whose level-1 pass visited only the 512-bin units
                               that the plane kernel (every precision but FDAS_BF16_SPLIT,
                               inside fdas_search / fdas_batch_search) marked as holding a value
                               above thr[0], instead of reading the whole plane                */
} fdas_profile;

/* Stage indices of fdas_profile.ms / n_timed. */
#define FDAS_STAGE_SPECTRUM  0   /* K1: long real FFT + normalisation                            */
#define FDAS_STAGE_SEGMENTS  1   /* K2: segment FFTs                                              */
#define FDAS_STAGE_CORRELATE 2   /* K3: multiply, inverse FFT, |.|^2, overlap discard            */
#define FDAS_STAGE_PEAKS     3   /* K4: harmonic sums and peak list                               */
/* Indices of fdas_profile.ms_peaks / n_timed_peaks (single kernels inside FDAS_STAGE_PEAKS). */
#define FDAS_PEAKS_LEVEL1    0   /* harmonic level 1 over the whole plane (or its marked units)   */
#define FDAS_PEAKS_LEVELS    1   /* levels 2 .. 16 over level 2's region                          */

/*
 * Turn per-stage timing on (enable != 0) or off.  Enabling creates CUDA events (plan-owned)
 * so that every later stage launch is bracketed by an event pair on its stream; at most
 * 512 launch groups per stage are timed between reads.  Launch counting is always on.
 * Errors: FDAS_E_INVALID, FDAS_E_CUDA.
 */
fdas_status fdas_profile_enable(fdas_plan_t plan, int enable);

/*
 * Synchronise the device, add up the recorded event pairs into *out, and reset the
 * counters when reset != 0.  Errors: FDAS_E_INVALID, FDAS_E_CUDA.
 */
fdas_status fdas_profile_read(fdas_plan_t plan, fdas_profile *out, int reset);

/* Text of the last CUDA error seen by this plan ("" if none).  Host only. */
const char *fdas_last_error(fdas_plan_t plan);

/* Free a plan and its device memory (NULL is ignored).  Synchronises the device. */
void fdas_destroy(fdas_plan_t plan);

/* Static text for a status code. */
const char *fdas_status_string(fdas_status s);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int fdas_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FDAS_H */
