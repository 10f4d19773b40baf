/*
 * qew.h -- C ABI of the GB300 (sm_103a) engine for the explicit-Euler relaxation of the
 * discretised 1D quenched Edwards-Wilkinson equation (Ferrero, Bustingorry, Kolton,
 * arXiv:1211.7275).
 *
 * The method (Sec. II and Sec. III.B of the paper): each chain s is a periodic line of L sites
 * with a continuous displacement u_i, started flat (u_i = 0, Sec. II) and integrated with
 * the explicit Euler method,
 *     u_i <- u_i + dt (u_{i+1} + u_{i-1} - 2 u_i + f + F_p(i, u_i))       (Eq. 1, eta = c = 1)
 * all forces taken from the old state.  The pinning force is built from random numbers drawn
 * at the integer points (i, n) of the (x, u) plane and interpolated in u (Sec. III.B; the cases
 * of Sec. IV.C):
 *     QEW_RF_GAUSS_LINEAR        F_p = (1 - d) R(i, n) + d R(i, n + 1),  R ~ N(0, 1)  (Case 4)
 *     QEW_RB_UNIFORM_CATMULLROM  F_p = -dV/du, V the Catmull-Rom spline through
 *                                V(i, n - 1 .. n + 2),  V ~ U(-1, 1)               (Case 2)
 *     QEW_NONE                   F_p = 0 (disorder-free line)
 *     QEW_RB_GAUSS_LINEAR        F_p = -dV/du, V the linear spline through G(i, n), G(i, n + 1):
 *                                F_p = G(i, n) - G(i, n + 1), constant inside a cell and
 *                                discontinuous at the integers; G ~ N(0, 1)        (Case 3)
 *     QEW_RB_GAUSS_CATMULLROM    F_p = -dV/du, V the Catmull-Rom spline through
 *                                G(i, n - 1 .. n + 2)                              (Case 1)
 * with n = floor(u), d = u - n.  The random numbers come from Philox4x32-10 (Salmon et al.,
 * SC'11) with key (lo32(seed), hi32(seed)) and counter (i, (uint32) n, s, tag), tag 0 for R,
 * 1 for V and 2 for G (the two Gaussian random-bond kinds interpolate the same G), regenerated
 * on the device whenever a site changes cell (the "memory-free" disorder of Sec. IV.D).  Observables (Eqs. 3-5), per chain: v = f + (1/L) sum_i F_p(i, u_i)
 * (the mean velocity, since the periodic Laplacian sums to zero), ubar = (1/L) sum_i u_i and
 * w2 = (1/L) sum_i (u_i - ubar)^2.
 *
 * Conventions for every entry point:
 *  - Return value: QEW_OK (0) or a negative QEW_E* status; no call aborts the process.  After
 *    an error, qew_last_error(h) describes it (for creation errors, qew_last_error(NULL)).
 *  - Pointers named *_out / *_in / steps / L / f / kind are HOST pointers owned by the caller;
 *    the library copies what it needs before returning.  Device memory is owned by the handle
 *    and freed by qew_destroy.
 *  - Calls on one handle must not run concurrently from several host threads; different
 *    handles may be used from different threads at the same time.
 *  - Work is issued on the handle's stream (default: the legacy default stream, or the one set
 *    by qew_set_stream); calls that return host data synchronise that stream.
 *  - Time: after k Euler steps the chains are at t = k dt.  "step" always counts Euler steps
 *    since the flat start (or since the last qew_set_state/qew_reset).
 */
#ifndef QEW_H
#define QEW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qew_ctx* qew_handle;

enum qew_status {
    QEW_OK = 0,
    QEW_EINVAL = -1,     /* invalid argument (message says which) */
    QEW_ENOMEM = -2,     /* device or host allocation failed */
    QEW_ECUDA = -3,      /* a CUDA call failed (message carries cudaGetErrorString) */
    QEW_ETIMEOUT = -4,   /* a bounded device wait (bulk-copy completion) gave up */
    QEW_ENONFINITE = -5, /* an observable came out NaN or infinite */
    QEW_ESTATE = -6      /* call not allowed in the handle's current state */
};

enum qew_disorder {
    QEW_RF_GAUSS_LINEAR = 0,
    QEW_RB_UNIFORM_CATMULLROM = 1,
    QEW_NONE = 2,
    QEW_RB_GAUSS_LINEAR = 3,
    QEW_RB_GAUSS_CATMULLROM = 4
};

enum qew_precision {
    QEW_FP32_SPLIT = 0, /* int32 cell n + FP32 offset d in [0,1); fused, temporally blocked */
    QEW_FP64 = 1        /* plain FP64 state, one launch per Euler step */
};

/*
 * qew_create -- `batch` chains of `L` sites, samples s = 0 .. batch-1, all with drive `f` and
 * disorder `disorder_kind`, time step `dt`, flat start, precision QEW_FP32_SPLIT.
 * Requirements: 1 <= L < 2^31, batch >= 1, L * batch < 2^40, 0 < dt < 0.5, |f| < 2^12 (so that,
 * with neighbouring displacements below 2^12, no Euler step moves a site by 2^15 cells or more).
 * Allocates the state on the current CUDA device (QEW_ENOMEM if it does not fit).
 * On success *out receives the handle; on failure *out is set to NULL.
 */
int qew_create(qew_handle* out, int64_t L, int32_t batch, double f, double dt, int32_t disorder_kind,
               uint64_t seed);

/*
 * qew_create_batch -- `n_chains` chains of uneven lengths L[c], each with its own drive f[c]
 * and disorder kind[c]; chain c uses sample index s = c.  `precision` is a qew_precision.
 * Same limits per chain as qew_create; sum of L[c] < 2^40.
 */
int qew_create_batch(qew_handle* out, int32_t n_chains, const int64_t* L, const double* f,
                     const int32_t* kind, double dt, uint64_t seed, int32_t precision);

/* qew_set_precision -- switch between QEW_FP32_SPLIT and QEW_FP64.  Allowed only before the
 * first Euler step (QEW_ESTATE otherwise); resets the handle to the flat start. */
int qew_set_precision(qew_handle h, int32_t precision);

/* qew_set_stream -- issue all further work on `stream` (a cudaStream_t owned by the caller,
 * e.g. torch.cuda.current_stream().cuda_stream); NULL selects the handle's own non-blocking
 * stream (the default).  Drops any captured CUDA graph. */
int qew_set_stream(qew_handle h, void* stream);

/*
 * qew_set_disorder_period -- make the disorder of every chain periodic in u with period M (the
 * periodic L x M samples of Sec. III.B; the paper notes that the memory-free generator can be
 * forced to be periodic as well): every node index n keys the generator as n mod M, in [0, M).
 * period = 0 (the default) restores the aperiodic disorder of the memory-free runs (Sec. IV.D).
 * The state is reset to the flat start at step 0, since every cache depends on the period.
 * QEW_EINVAL unless 0 <= period < 2^31.  (qew_observe_state_noalloc and qew_disorder_values take
 * node indices as given, i.e. aperiodic.)
 */
int qew_set_disorder_period(qew_handle h, int64_t period);

/*
 * qew_set_samples -- sample index s of each chain (counter word 2 of the generator, so the
 * disorder realisation of the chain; Sec. III.B draws an independent disorder per sample):
 * s[c] for chain c, n_chains entries (host array, copied).  By default chain c uses s = c.  With
 * it a chain can be relaxed on its own, or a set of samples split over several handles or GPUs,
 * on exactly the disorder it has inside a batch.  The state is reset to the flat start at
 * step 0, since every cache depends on s.  QEW_EINVAL if s is NULL.
 */
int qew_set_samples(qew_handle h, const uint32_t* s);

/*
 * qew_set_tuning -- launch shape of the fused FP32-split kernel: `tile_w` sites per warp tile
 * (32 lanes x an odd number of sites: 224, 480, 736, 992 or 1248).  Each disorder kind takes the
 * widest tile it supports up to tile_w: cubic random-bond chains (Cases 1 and 2) at most 480,
 * disorder-free chains at most 992, so in a mixed batch every kind runs its own widest tile.
 * `K` Euler steps per HBM round trip (temporal-block depth, 1 <= K <= w / 4 for the narrowest
 * tile w in use),
 * `tiles_per_cta` warp tiles per thread block (1, 2, 4 or 8).
 * Passing 0 for all three asks for the autotuner: it times candidate shapes (every supported tile
 * width, K in {4, 8, 16, 32} up to the limit above, 1, 2 or 4 tiles per block) on the handle's
 * own chains, without changing their state, as soon as they are at least 1024 Euler steps past
 * the flat start (the best shape changes while the rate of cell crossings decays after the flat
 * start); until then the default shape is used.
 * Results never depend on the shape beyond FP32 rounding order, which is identical: each
 * site's arithmetic is the same for every shape.
 */
int qew_set_tuning(qew_handle h, int32_t tile_w, int32_t K, int32_t tiles_per_cta);

/* qew_get_tuning -- the shape in use (after autotuning, the one it picked); tile_w is the widest
 * tile among the batch's kinds. */
int qew_get_tuning(qew_handle h, int32_t* tile_w, int32_t* K, int32_t* tiles_per_cta);

/* qew_advance -- n_steps >= 0 Euler steps of every chain.  Asynchronous: the work is queued on the
 * handle's stream.  A range violation of the FP32-split state found at its end (see qew_observe)
 * is reported by the next call that reads results (qew_observe, qew_get_state, qew_get_cells). */
int qew_advance(qew_handle h, int64_t n_steps);

/*
 * qew_observe -- advance through the observation steps `steps[0..n_times)` (strictly
 * increasing, steps[0] >= the current step) and record at each the per-chain observables of
 * Eqs. 3-5, fused into the integration: v_out[k * n_chains + c] = v and
 * w2_out[k * n_chains + c] = w2 of chain c at step steps[k].  Either output may be NULL.
 * n_times == 0 is a no-op.  Returns after the results are in host memory.  On return the
 * chains are at step steps[n_times - 1].  QEW_ENONFINITE if an observable is NaN/Inf (the
 * outputs are still written).  QEW_ESTATE if, at the end of the call (or of an earlier
 * qew_advance), neighbouring sites of the FP32-split state differ by 2^12 cells or more: outside
 * that range the fused kernel's cell arithmetic is no longer exact, so the state is reported as
 * invalid instead of silently wrong (the Euler map with dt < 0.5 grows a neighbour difference by
 * at most 2 dt max|F_p| per step, so a line started within the range stays in it for thousands of
 * steps at least; physical lines stay far inside it).  The schedule's launches (fused segments, reductions and the copy
 * to the host) are captured into a CUDA graph the first time and replayed whenever the same
 * schedule is observed again from the same step (e.g. after qew_reset); not while statistics
 * are enabled, and not for schedules needing more than 20000 launches.
 */
int qew_observe(qew_handle h, const int64_t* steps, int32_t n_times, double* v_out, double* w2_out);

/* qew_observe_ex -- as qew_observe, also writing the centre of mass ubar (Eq. 4). */
int qew_observe_ex(qew_handle h, const int64_t* steps, int32_t n_times, double* v_out, double* ubar_out,
                   double* w2_out);

/*
 * qew_get_state -- copy the displacement field to the host as FP64: u_out holds the chains one
 * after another (chain c at offset sum_{c'<c} L[c']); *step_out (if not NULL) receives the
 * current step.  For QEW_FP32_SPLIT the value is (double) n + (double) d, exact.
 */
int qew_get_state(qew_handle h, double* u_out, int64_t* step_out);

/*
 * qew_get_cells -- copy the integer cell index n_i = floor(u_i) of every site (int32, same
 * layout as qew_get_state).  For QEW_FP64 it is floor of the FP64 state.
 */
int qew_get_cells(qew_handle h, int32_t* cells_out);

/*
 * qew_set_state -- replace the displacement field (FP64, layout of qew_get_state) and set the
 * step counter to 0.  Values must be finite with |u| < 2^30, and neighbouring sites (periodic)
 * must differ by less than 2^12 (so that the cells of a warp tile stay exact in FP32).  The
 * disorder caches are regenerated for the new cells.
 */
int qew_set_state(qew_handle h, const double* u_in);

/*
 * qew_structure_factor -- the disorder-averaged structure factor of the current state (Eq. 6,
 * Sec. II):  S_out[k] = (1/n_chains) sum_c |(1/L) sum_x u_c(x) e^{-iqx}|^2  at q = 2 pi (k+1) / L,
 * for k < n_modes.  Modes n and L - n are equal for a real line, so 1 <= n_modes <= L/2 covers
 * the spectrum.  All chains of the handle must have the same length L (QEW_EINVAL otherwise).
 * The line is taken in FP64 (exact for QEW_FP32_SPLIT), transformed by a batched real-to-complex
 * cuFFT and the mode powers are summed over chains in a fixed order: the result is
 * deterministic.  Does not advance the state.  S_out: host array of n_modes doubles, written
 * before the call returns.  The first call makes a cuFFT plan that the handle keeps; every call
 * allocates a work area of about 8 bytes per site and frees it again (QEW_ENOMEM if that fails).
 */
int qew_structure_factor(qew_handle h, int32_t n_modes, double* S_out);

/* qew_reset -- back to the flat start u = 0 at step 0. */
int qew_reset(qew_handle h);

/* qew_num_sites -- total number of sites (sum of the chain lengths). */
int qew_num_sites(qew_handle h, int64_t* n_sites);

/*
 * qew_disorder_values -- the device generator's disorder values, for validation: for each
 * k < count, out[k] = R(s, i[k], n[k]) (kind QEW_RF_GAUSS_LINEAR), V(s, i[k], n[k])
 * (QEW_RB_UNIFORM_CATMULLROM) or G(s, i[k], n[k]) (QEW_RB_GAUSS_LINEAR and
 * QEW_RB_GAUSS_CATMULLROM; QEW_NONE is rejected), computed on the current device in the arithmetic of
 * `precision` (FP32 values are widened to double).  Host pointers; synchronous.
 */
int qew_disorder_values(int32_t kind, int32_t precision, uint64_t seed, uint32_t s, const int64_t* i,
                        const int64_t* n, int64_t count, double* out);

/*
 * qew_philox_words -- the device Philox4x32-10 block function: out[4k..4k+4) = Philox(ctr
 * [4k..4k+4), key [2k..2k+2)) for k < n_blocks, on the current device.  Host pointers.
 */
int qew_philox_words(const uint32_t* ctr, const uint32_t* key, int64_t n_blocks, uint32_t* out);

/*
 * qew_measure_alu_peaks -- measured rates of the lane arithmetic on the current device, the
 * denominators of the relaxation kernels' rooflines (the fused FP32-split kernel is bound by
 * instruction issue, Sec. III.B's Euler scheme being a few operations per site and step):
 *   out[0]  FP32 fused multiply-adds per second, summed over all lanes (independent chains on a
 *           grid filling every SM): the lane-operation peak, nominally SMs x 128 x SM clock;
 *   out[1]  FP64 fused multiply-adds per second (the plain FP64 comparison path);
 *   out[2]  Philox4x32-10 blocks per second with a precomputed key schedule (the generator that
 *           redraws the disorder at each cell crossing, Sec. III.B / IV.D);
 *   out[3]  the SM clock in MHz during the FP32 run (cycle counter against the global timer).
 * Each rate is the best of three event-timed launches after one untimed, on the legacy default
 * stream; the call takes some tens of milliseconds and synchronises the device.  n_out >= 4
 * (host array).  QEW_EINVAL for a NULL or short array; QEW_ECUDA if a CUDA call fails.
 */
int qew_measure_alu_peaks(double* out, int32_t n_out);

/*
 * qew_enable_stats -- with enable != 0, bracket every launch of the fused FP32-split kernel with
 * CUDA events on the handle's stream and count cell crossings; 0 turns this off.  Counters
 * start from zero.
 * qew_get_stats -- synchronise the handle's stream and report, since the last reset: all kernel
 * launches issued by the handle (`launches`), launches of the fused kernel (`fused_launches`),
 * their summed event-timed duration in ms (`fused_ms`, 0 unless stats are enabled), the
 * site-updates they performed (`site_updates`: owned sites x Euler steps) and the cell
 * crossings among them (`crossings`, 0 unless stats are enabled); then reset the counters.
 * Any output pointer may be NULL.
 */
int qew_enable_stats(qew_handle h, int32_t enable);
int qew_get_stats(qew_handle h, int64_t* launches, int64_t* fused_launches, double* fused_ms, int64_t* site_updates,
                  int64_t* crossings);

/*
 * qew_critical_force_rf -- the critical force f_c^s and the critical configuration of one random-field
 * sample periodic in x (L sites) and in u (period M): the largest drive at which a pinned
 * configuration exists, and that configuration (Sec. III.B; the paper computes them with an exact
 * algorithm built on Middleton's theorems, which it cites; Sec. IV.A compares them with the
 * short-time-dynamics threshold).  Host code, FP64, no GPU work.
 *   R         HOST array [L][M], R[i*M + m] = R(i, m): the sample's force values at the integer
 *             points (e.g. from qew_disorder_values, QEW_FP64, with n = 0 .. M-1); the force is
 *             their linear interpolation, periodic in u (Case 4).
 *   dt        Euler step of the avalanches (0 < dt < 0.5); f_start: a drive at which the flat
 *             line pins (the search starts from its pinned configuration).
 *   f_c_out   receives f_c^s; u_c_out (L doubles, or NULL) the critical configuration;
 *   events_out / dyn_steps_out (or NULL): branch events and Euler steps used.
 * Method: with the cells fixed the static equation is a linear (periodic tridiagonal) system, so
 * the pinned configuration is followed exactly while f grows, one cell change at a time; where a
 * branch ends (the system loses positive definiteness) the line avalanches at fixed f, followed
 * with the Euler map until it pins again, and f_c^s is the drive at which an avalanche carries
 * every site a full period M (the motion then repeats forever).
 * Errors: QEW_EINVAL (sizes, NULL, dt), QEW_ESTATE (the flat line does not pin at f_start, or an
 * avalanche does not end within the step limit), QEW_ENOMEM; message via qew_last_error(NULL).
 */
int qew_critical_force_rf(int64_t L, int64_t M, const double* R, double dt, double f_start, double* f_c_out,
                          double* u_c_out, int64_t* events_out, int64_t* dyn_steps_out);

/*
 * qew_observe_state_noalloc -- per-chain observables (Eqs. 3-5: v, ubar, w2) of an FP32-split
 * state that the CALLER holds in device memory, computed without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot let a library
 * call cudaMalloc -- for instance a framework whose caching allocator already owns the GPU's
 * memory, or a time-critical loop that must not pay the device-wide synchronisation that
 * cudaMalloc/cudaFree can cause.  It computes the same quantities as qew_observe_ex does at the
 * current step of a handle.
 *   cell, off  DEVICE pointers, batch * L elements each, chain c at offset c * L: the integer cell
 *              n_i and the FP32 offset d_i in [0, 1) of u_i = n_i + d_i (the layout that
 *              qew_get_cells / qew_get_state describe).  Chain c has sample index s = c.
 *              Cells are summed relative to the first cell of each 256-site tile, in FP32: the
 *              sums keep their accuracy while cells inside a tile differ by less than 2^24.
 *   f, disorder_kind, seed  as in qew_create; the pinning force is regenerated from them.
 *   stream     cudaStream_t to run on (NULL: legacy default stream); synchronised before return.
 *   v_out, ubar_out, w2_out  HOST pointers to `batch` doubles each, or NULL.
 * Scratch: a fixed array of 256-byte-aligned device memory inside the library (about 1.7 MB,
 * held by every GPU that loads the library until the process exits): at most 4096 chains and
 * 65536 tiles of 256 sites (batch * ceil(L / 256) <= 65536, i.e. up to 2^24 sites); larger
 * inputs are rejected with QEW_EINVAL.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress), so the first call should come before any stream
 * capture.  Every call overwrites the part of the array it uses and leaves its contents there;
 * calls whose work overlaps on the GPU (other streams, other host threads) share the array and
 * race -- serialise them.  Errors: QEW_EINVAL (bad sizes or pointers), QEW_ECUDA; message via
 * qew_last_error(NULL).
 */
int qew_observe_state_noalloc(const int32_t* cell, const float* off, int64_t L, int32_t batch, double f,
                              int32_t disorder_kind, uint64_t seed, void* stream, double* v_out,
                              double* ubar_out, double* w2_out);

/*
 * qew_selftest_bounded_wait -- exercise the failure path of the bounded device waits: one warp
 * waits on an mbarrier that nothing completes, gives up after `spin_limit` polls (1 .. 2^22) and
 * raises the handle's device error flag, which this call reports as QEW_ETIMEOUT (and clears).
 * Any other status means the failure path is broken.  The handle stays usable afterwards.
 */
int qew_selftest_bounded_wait(qew_handle h, int32_t spin_limit);

/* qew_last_error -- message of the last failed call on `h` (NULL: of the last failed creation
 * or handle-less call on this thread).  Never NULL; "" if there was no error. */
const char* qew_last_error(qew_handle h);

/* qew_destroy -- free the handle and its device memory; NULL is a no-op. */
void qew_destroy(qew_handle h);

#ifdef __cplusplus
}
#endif

#endif /* QEW_H */
