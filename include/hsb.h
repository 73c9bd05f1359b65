/*
 * hsb.h -- C ABI of the GB300 heated simulated bifurcation library (libhsb.so).
 *
 * Heated simulated bifurcation (HbSB / HdSB) searches for low-energy states of
 * the Ising problem
 *     E = -1/2 sum_i sum_j J_ij s_i s_j,  s_i = +/-1,  J_ij = J_ji,  J_ii = 0
 * (Kanao & Goto, arXiv 2203.08361, Eq. (eq_Ising)) by integrating, for R
 * independent replicas, the equations of motion
 *     dx_i/dt = a0 y_i,
 *     dy_i/dt = -[a0 - a(t)] x_i + c0 f_i + gamma y_i          Eqs. (eq_PosHeat), (eq_MomHeat)
 * with f_i = sum_j J_ij x_j (ballistic, Eq. (eq_fb)) or
 *      f_i = sum_j J_ij sgn(x_j) (discrete, Eq. (eq_fd)),
 * discretised as in the Methods section: symplectic Euler on the terms other
 * than gamma*y (Eqs. (eq_SyEuY), (eq_SyEuX)), perfectly inelastic walls at
 * x = +/-1 (Eqs. (eq_WallX), (eq_WallY)) and an Euler heating step that uses
 * the momentum before the step (Eq. (eq_EuHeat)).  a(t) rises linearly from 0
 * to a0; c0 = c1 / (sqrt(N) sigma_J) (Results, "SB with thermal fluctuation").
 *
 * Conventions shared by every entry point:
 *   - Every call returns an hsb_status and never aborts the process.  On an
 *     error, hsb_last_error() returns a message for the calling thread.
 *   - There is no CPU fallback: without a CUDA device every compute call
 *     returns HSB_E_NODEVICE.
 *   - Arrays are dense and row-major; "spins x replicas" state is stored one
 *     replica per row: element (r, i) of an R x N array is at r*N + i.
 *   - Host pointers are caller-owned and are not retained after the call
 *     returns.  Device pointers (the *_device variants) must stay valid until
 *     the work queued on the handle's stream has completed.
 *   - A handle is not thread-safe: calls on one handle must not overlap.
 *     Distinct handles are independent.
 *
 * Evaluation protocol (Results, K2000 and 700-spin studies): the energy of
 * s = sgn(x(t_k)) is evaluated at t_k for k = m*eval_every (m >= 1, k < steps)
 * and at the final time k = steps; eval_every = 0 evaluates the final time
 * only.  The best (strictly lowest, earliest on ties) energy and its spins are
 * returned per replica.  sgn(x) = +1 for x >= 0 (including -0.0).
 */
#ifndef HSB_H
#define HSB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HSB_API_VERSION 2

#if defined(__GNUC__)
#define HSB_API __attribute__((visibility("default")))
#else
#define HSB_API
#endif

typedef struct hsb_ctx *hsb_handle; /* opaque, library-owned */

typedef enum {
    HSB_OK = 0,
    HSB_E_INVAL = 1,       /* bad argument (size, null pointer, parameter range) */
    HSB_E_ASYM = 2,        /* J is not exactly symmetric */
    HSB_E_DIAG = 3,        /* J has a nonzero diagonal entry */
    HSB_E_NOMEM = 4,       /* device or host allocation failed */
    HSB_E_CUDA = 5,        /* a CUDA runtime call or kernel failed */
    HSB_E_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    HSB_E_UNSUPPORTED = 7, /* precision not valid for these couplings / form */
    HSB_E_NODEVICE = 8     /* no usable CUDA device */
} hsb_status;

typedef enum {
    HSB_BALLISTIC = 0, /* f = J x        (HbSB when gamma > 0), Eq. (eq_fb) */
    HSB_DISCRETE = 1   /* f = J sgn(x)   (HdSB when gamma > 0), Eq. (eq_fd) */
} hsb_form;

typedef enum {
    /* discrete form with J in {-1,0,+1}: FP8; otherwise BF16X3 */
    HSB_PREC_AUTO = 0,
    /* plain FP32 on CUDA cores: force sums are fused multiply-adds over j
       ascending, so trajectories equal the binary32 oracle's bit for bit */
    HSB_PREC_FP32 = 1,
    /* tcgen05 tensor cores, J and sgn(x) in FP8 e4m3, FP32 accumulation.
       Exact (integer forces); discrete form with J in {-1,0,+1} only. */
    HSB_PREC_FP8 = 2,
    /* tcgen05 tensor cores, J = J_hi + J_lo and x = x_hi + x_lo in BF16,
       J_hi x_hi + J_lo x_hi + J_hi x_lo accumulated in FP32 */
    HSB_PREC_BF16X3 = 3,
    /* tcgen05 tensor cores (kind::mxf4, block-scaled with unit UE8M0 scales),
       J and sgn(x) in packed FP4 e2m1 (+1 = 0x2, -1 = 0xA), FP32
       accumulation.  Exact (integer forces), so trajectories equal the FP8
       ones bit for bit.  Discrete form with J in {-1,0,+1} only; the
       persistent kernel or one kernel launch per step (schedule 0, 1 or 2,
       else HSB_E_UNSUPPORTED); never picked by AUTO. */
    HSB_PREC_FP4 = 4
} hsb_prec;

typedef struct {
    int form;               /* hsb_form */
    int prec;               /* hsb_prec */
    double a0;              /* a0 > 0 (paper: 1) */
    double c1;              /* c0 = c1 / (sqrt(N) sigma_J) when c0 <= 0 */
    double c0;              /* interaction scale; > 0 overrides c1 */
    double dt;              /* time step Delta t > 0 */
    double gamma;           /* heating rate >= 0 (0: plain bSB / dSB) */
    double init_half_width; /* x0, y0 uniform in (-L, L); paper L = 1 */
    int eval_every;         /* >= 0; 100 in the K2000 study, 0 = final only */
    int trace_every;        /* >= 0; > 0 records, at t_k for k = m*trace_every < steps,
                               the minimum and mean Ising energy over replicas and
                               the mean instantaneous temperature (1/N) sum y^2
                               (Eq. (eq_TInst)); see hsb_get_trace.  FP32, FP8 and
                               FP4 (persistent or one launch per step; not
                               schedules 3 and 4);
                               BF16X3 returns HSB_E_UNSUPPORTED */
    uint32_t instance;      /* random stream of the instance (x0, y0) */
    int schedule;           /* FP8 / FP4 step loop: 0 = automatic (persistent kernel
                               when its grid fits on the device), 1 = persistent
                               kernel only (HSB_E_UNSUPPORTED if it cannot fit),
                               2 = one kernel launch per step (on CTA pairs,
                               tcgen05 cta_group::2, once N rounded up to 128
                               reaches 1024), 3 = persistent
                               kernel with the CTA's rows of J held on chip for
                               the whole run (N <= 2048, else
                               HSB_E_UNSUPPORTED), 4 = persistent kernel run by
                               CTA pairs, F^T = S^T J (constant heating, no
                               trace, N <= 4096, R rounded up to 128 a multiple
                               of 256 and a grid that fits, else
                               HSB_E_UNSUPPORTED).  Automatic takes 1
                               where its grid fits, then 4 (FP8), then 2.
                               FP4 takes 0, 1 and 2 only. */
    int thermostat;         /* HSB_HEAT_CONSTANT: the constant heating rate gamma of
                               Eq. (eq_MomHeat) (HbSB / HdSB); HSB_HEAT_NOSE_HOOVER:
                               the dynamic xi of Eqs. (eq_NH1), (eq_NH), one per
                               replica, in place of -gamma (gamma is then unused).
                               Nose-Hoover runs on FP32, FP8 and FP4 (persistent or one
                               launch per step; AUTO never picks BF16X3 for it);
                               schedule 3 and hsb_advance* return HSB_E_UNSUPPORTED,
                               hsb_run_batch runs the instances one after another.
                               A momentum |y| >= 256 (an unstable setting: M much
                               below N) makes the run return HSB_E_INVAL.  See
                               hsb_get_xi. */
    int reserved0;          /* must be zero */
    double nh_T;            /* Nose-Hoover temperature T >= 0 */
    double nh_M;            /* Nose-Hoover mass M > 0 */
    double nh_xi0;          /* xi(t_0), finite; negative values heat from the start */
    uint32_t reserved[2];   /* must be zero */
} hsb_params;

typedef enum {
    HSB_HEAT_CONSTANT = 0,
    /* Per step, in binary64 with each operation rounded once: the update uses
       the friction factor g_r = fl32(-xi_r dt) where HbSB uses fl32(gamma dt)
       (the friction -xi y(t_k) in place of the heating term); then
       S_r = sum_i y_i(t_{k+1})^2, xi_r += (dt / M) (S_r - N T).  S_r is
       exact fixed point, independent of summation order: each y_i rounded
       to a multiple of 2^-24, the squares summed as integers, one rounding. */
    HSB_HEAT_NOSE_HOOVER = 1
} hsb_thermostat;

/* Fills *p with the paper's tuned HdSB settings (Fig. 1 caption): discrete
 * form, AUTO precision, a0 = 1, c1 = 0.7, dt = 1.1, gamma = 0.06, L = 1,
 * eval_every = 100. */
HSB_API hsb_status hsb_params_default(hsb_params *p);

/* Library ABI version (HSB_API_VERSION). */
HSB_API int hsb_version(void);

/* Creates a handle for the couplings J (host, float32, N x N, row-major),
 * copying them to the current CUDA device.  J must be exactly symmetric with a
 * zero diagonal (Eq. (eq_Ising)); otherwise HSB_E_ASYM / HSB_E_DIAG (a NaN
 * entry fails the symmetry test).  An infinite entry or an all-zero J gives
 * HSB_E_INVAL.  N >= 2.
 * Work is queued on a private stream of the handle until hsb_set_stream(). */
HSB_API hsb_status hsb_create(const float *J, int N, hsb_handle *out);

/* Destroys the handle and frees its device memory (waits for its stream).
 * NULL is ignored. */
HSB_API void hsb_destroy(hsb_handle h);

/* Sets the CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream())
 * on which the handle queues its work; NULL selects the handle's private
 * stream again.  Work the handle queued on the previous stream is ordered
 * before anything it queues on the new one (the new stream waits on an event;
 * the host does not block), unless either stream is being captured into a
 * CUDA graph, where the capturing caller orders the two.  Errors: HSB_E_INVAL for a NULL handle,
 * HSB_E_CUDA when the event cannot be recorded or waited on (the handle then
 * keeps its previous stream). */
HSB_API hsb_status hsb_set_stream(hsb_handle h, void *cuda_stream);

/* Number of spins N and whether J is in {-1, 0, +1} (the FP8 path applies). */
HSB_API hsb_status hsb_info(hsb_handle h, int *N, int *is_pm1);

/* MAX-CUT front end (Results, Eq. (eq_Cut)): a MAX-CUT problem with weights
 * w_ij = w_ji is the Ising problem with J_ij = -w_ij, and a spin vector with
 * Ising energy E cuts C = -E/2 - (1/4) sum_ij J_ij.  Writes cut[r] for the
 * energies best_energy[r], r = 0..R-1 (e.g. the output of hsb_run); both are
 * caller-owned HOST arrays of R doubles.  sum_ij J_ij is summed row by row in
 * binary64 when the couplings are set, so for integer weights the cut values
 * are exact.  Errors: HSB_E_INVAL for a NULL argument or R < 1. */
HSB_API hsb_status hsb_cut_values(hsb_handle h, int R, const double *best_energy, double *cut);

/* Runs `steps` >= 1 heated SB steps for replicas r = 0..R-1 (R >= 1) from the
 * seeded initial state and returns, per replica, the best evaluated energy
 * best_energy[r] (float64) and its spins best_spins[r*N + i] (+1 / -1).
 * One step is the Methods update, Eqs. (eq_SyEuY), (eq_SyEuX), (eq_WallX),
 * (eq_WallY), (eq_EuHeat), with the force of Eq. (eq_fb) or (eq_fd); the
 * energy of Eq. (eq_Ising) is evaluated every p->eval_every steps and after
 * the last one, and the first strictly lowest is kept.
 * Both outputs are caller-owned HOST buffers; the call blocks until they are
 * written.  Replica r's result depends only on (J, params, steps, seed, r),
 * not on R.  Errors: HSB_E_INVAL (NULL argument, R, steps or a parameter out
 * of range), HSB_E_UNSUPPORTED (a precision, schedule or thermostat the
 * couplings or form do not allow), HSB_E_NOMEM, HSB_E_CUDA, HSB_E_TIMEOUT (a
 * bounded device wait gave up; the handle stays usable). */
HSB_API hsb_status hsb_run(hsb_handle h, const hsb_params *p, int R, int steps, uint64_t seed,
                   int8_t *best_spins, double *best_energy);

/* As hsb_run, but the outputs are DEVICE pointers (best_spins R*N int8,
 * best_energy R float64) and the call only queues the work on the handle's
 * stream and returns. */
HSB_API hsb_status hsb_run_device(hsb_handle h, const hsb_params *p, int R, int steps, uint64_t seed,
                          int8_t *best_spins, double *best_energy);

/* Runs `count` instances (handles hs[0..count-1], each with its own N) with
 * the same parameters, R replicas and steps, and returns each instance's best
 * spins (best_spins[b], host, R x N_b int8) and energies (best_energy[b],
 * host, R float64).  Instance b draws its initial state from the random
 * stream p->instance + b, so its result equals hsb_run on hs[b] with
 * instance = p->instance + b.  For the discrete form with couplings in
 * {-1, 0, +1}, constant heating and no trace, all instances run in one
 * kernel launch that takes them from a queue, largest first, one CTA per
 * instance, where the shape allows: with p->prec AUTO or FP8, R rounded up
 * to 32 at most 256 and (N rounded up to 128) times that at most 128 KiB;
 * with HSB_PREC_FP4 (packed e2m1 operands), R rounded up to 32 at most 224
 * and (N rounded up to 256) / 2 times that at most 128 KiB.  Otherwise the
 * instances run one after another.  All handles must be on one device; the
 * work is queued on hs[0]'s stream.  Blocks. */
HSB_API hsb_status hsb_run_batch(const hsb_handle *hs, int count, const hsb_params *p, int R,
                                 int steps, uint64_t seed, int8_t *const *best_spins,
                                 double *const *best_energy);

/* Copies x(t_steps), y(t_steps) of the last run on this handle (R x N float32
 * each, host) into x and y (either may be NULL).  Blocks. */
HSB_API hsb_status hsb_get_state(hsb_handle h, float *x, float *y);

/* Advances a given state: applies the updates k = k_begin .. k_end-1 of a
 * `steps`-step pump schedule (0 <= k_begin <= k_end <= steps) to x, y (host,
 * R x N float32, read and overwritten).  No energy is evaluated.  Used for
 * one-step accuracy checks and for resuming a run from a saved state: the
 * schedule uses the absolute k, so splitting a run gives the same result. */
HSB_API hsb_status hsb_advance(hsb_handle h, const hsb_params *p, int R, int steps, int k_begin,
                       int k_end, float *x, float *y);

/* Continues the state that the last hsb_run / hsb_run_device /
 * hsb_advance_device left on the device (same R and precision): queues the
 * updates k = k_begin .. k_end-1 of a `steps`-step pump schedule on the
 * handle's stream, without energy evaluation and without host copies.
 * Resuming with k_begin equal to the previous call's end step continues the
 * trajectory exactly; the step loop is graph-captured once per range. */
HSB_API hsb_status hsb_advance_device(hsb_handle h, const hsb_params *p, int R, int steps, int k_begin,
                              int k_end);

/* Copies the trace of the last run (params.trace_every > 0): entry m holds
 * {min_r E_r, mean_r E_r, mean_r T_inst,r} at t_k, k = m*trace_every, as 3
 * doubles, E of s = sgn(x(t_k)) (Eq. (eq_Ising)) and T_inst = (1/N) sum_i
 * y_i(t_k)^2 (Eq. (eq_TInst)).  Writes min(max_entries, length) entries to
 * buf (host, 3 doubles each) and the trace length to *entries (may be NULL).
 * Blocks. */
HSB_API hsb_status hsb_get_trace(hsb_handle h, double *buf, size_t max_entries, size_t *entries);

/* Copies xi_r(t_Ns) of the last run's R replicas (binary64, host buffer of R
 * doubles) after a run with thermostat = HSB_HEAT_NOSE_HOOVER (Eq. (eq_NH)).
 * HSB_E_INVAL when the last run had no Nose-Hoover thermostat or R differs
 * from its replica count.  Blocks. */
HSB_API hsb_status hsb_get_xi(hsb_handle h, int R, double *xi);

/* Failure-detection test hook.  The next FP8 run on the persistent schedule
 * (streamed J) of this handle skips the publication of one tile's sign
 * operand (row block `row_block`, first replica block), so that the bounded
 * device waits of the other tiles expire: the run returns HSB_E_TIMEOUT after
 * the wait budget (about 2 s), the kernel frees its tensor memory, and the
 * handle stays usable (the following run is unaffected).  0 <= row_block <
 * ceil(N / 128), else HSB_E_INVAL. */
HSB_API hsb_status hsb_debug_drop_publication(hsb_handle h, int row_block);

/* Allocation-failure test hook, process-wide.  From this call on, every device
 * allocation the library makes of more than `bytes` bytes fails as the
 * device's allocator does when memory runs out: the call that needed it
 * returns HSB_E_NOMEM and its handle stays usable (what that call allocated
 * before the failure is freed by the next run or by hsb_destroy; a failed
 * hsb_create frees it at once).  0 removes the cap.  Buffers allocated earlier are kept.  Not
 * thread-safe with respect to calls in flight on other threads. */
HSB_API hsb_status hsb_debug_alloc_cap(size_t bytes);

/* Replaces the couplings of the handle by a new instance of the same N (host,
 * float32, N x N, row-major; validated as in hsb_create).  Device buffers and
 * captured step loops are kept, so solving many instances of one size pays
 * the set-up once.  Blocks until the copy is done. */
HSB_API hsb_status hsb_set_couplings(hsb_handle h, const float *J);

/* Number of kernels the last hsb_run / hsb_run_device / hsb_advance_device
 * queued on the device. */
HSB_API hsb_status hsb_run_stats(hsb_handle h, long long *kernel_launches);

/* Plain FP32 heated SB run (as hsb_run with HSB_PREC_FP32) that allocates
 * nothing.  The paper has no counterpart: this entry point serves callers
 * that cannot allocate device memory on demand -- code running under a fixed
 * device-memory budget owned by another allocator (a framework's caching
 * pool, a serving process sized at start-up), or code that must not call
 * cudaMalloc / cudaFree because those calls synchronize the device and stall
 * the work of other streams.
 *   J            DEVICE, float32, N x N row-major couplings (symmetric, zero
 *                diagonal; not validated, the caller owns them)
 *   best_spins   DEVICE, int8, R x N (+1 / -1), written
 *   best_energy  DEVICE, float64, R, written (binary64 Eq. (eq_Ising))
 *   cuda_stream  cudaStream_t on which all work is queued (NULL: legacy
 *                default stream); the call returns once the work is queued.
 * Limits: 2 <= N <= 512 and 1 <= R <= 256; larger sizes return HSB_E_INVAL.
 * p->c0 must be given (> 0): the couplings stay on the device, so the c1
 * normalisation is not applied; p->prec and p->schedule are ignored.
 * Every intermediate buffer lives in one file-scope device array of about
 * 2.6 MB that each GPU loading the library holds until the process exits.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture.  The kept address belongs to the
 * device's context of that time: after cudaDeviceReset, or once the primary
 * context has been destroyed and created again, it no longer names the array,
 * so do not call this entry point on that device again in the process.
 * All calls share the array and it keeps the previous call's contents (the
 * call rewrites every part it reads first): calls whose work overlaps on the
 * GPU -- on different streams, or from different threads -- race and give
 * wrong results, so serialise them. */
HSB_API hsb_status hsb_run_fp32_noalloc(const float *J, int N, const hsb_params *p, int R,
                                        int steps, uint64_t seed, int8_t *best_spins,
                                        double *best_energy, void *cuda_stream);

/* Waits for the work queued on the handle's stream and reports a device-side
 * failure of it (HSB_E_TIMEOUT when a bounded wait inside a kernel gave up). */
HSB_API hsb_status hsb_synchronize(hsb_handle h);

/* Thread-local message of the last failed call on this thread ("" if none). */
HSB_API const char *hsb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HSB_H */
