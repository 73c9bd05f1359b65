// hsb_api.cu -- C ABI and host runtime of libhsb (declared in include/hsb.h).
//
// Host side of the heated SB run (Kanao & Goto, arXiv 2203.08361): argument
// validation, coupling conversion, device buffers, the per-run constants
// (Methods; Results "SB with thermal fluctuation"), and the step loop: one
// persistent launch when its grid fits (FP8, split BF16), otherwise one launch
// per step captured once into a CUDA graph per run shape and replayed; the
// batch of instances with its autotuner; the Nose-Hoover thermostat and the
// per-step trace around either form.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "hsb.h"
#include "hsb_internal.cuh"

using namespace hsb;

namespace {

// Message of the last failed call on this thread (fixed storage, so that
// reporting an error never allocates).
thread_local char g_last_error[512];

hsb_status set_error(hsb_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return s;
}

hsb_status cuda_error(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return set_error(HSB_E_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(HSB_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Allocation-failure test hook (hsb_debug_alloc_cap): a device allocation of
// more than this many bytes fails as the device's own allocator does when it
// is out of memory; 0 = no cap.  Every device allocation of the library goes
// through dev_alloc.
std::atomic<size_t> g_alloc_cap{0};

cudaError_t dev_alloc(void **ptr, size_t bytes)
{
    const size_t cap = g_alloc_cap.load(std::memory_order_relaxed);
    if (cap != 0 && bytes > cap) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

template <typename T>
cudaError_t dev_alloc(T **ptr, size_t bytes)
{
    return dev_alloc(reinterpret_cast<void **>(ptr), bytes);
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess)                           \
            return cuda_error(e_, what);                 \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess)
            ok = true;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

// Everything that determines the captured step loop.
struct GraphKey {
    int prec, form, R, Rp, steps, eval_every, trace_every, pm1, thermo;
    float c0, dt, q, g;
    double a0, nh_h, nh_NT, dt64;
    uint64_t buffers_gen;
    bool operator==(const GraphKey &o) const { return memcmp(this, &o, sizeof *this) == 0; }
};

struct RunCfg {
    int prec, form, R, Rp, steps, eval_every, trace_every, schedule;
    double a0;
    // Nose-Hoover thermostat: h = dt / M, N T and dt in binary64, xi(t_0)
    int thermo;
    double nh_h, nh_NT, nh_xi0, dt64;
    StepConsts c;
    std::vector<float> pk;  // p_k = a0 - a(t_k), k = 0..steps-1, rounded once
};

}  // namespace

struct hsb_ctx {
    int N = 0, Np = 0, device = 0, pm1 = 0;
    double sigma = 0.0;
    double sumJ = 0.0;  // sum_ij J_ij in binary64, row by row (cut values, Eq. (eq_Cut))
    int jscale = 0;     // fixed-point exponent of the final energies: max |J| 2^jscale < 2^40
    cudaStream_t work = nullptr;     // where work is queued (user's or own)
    cudaStream_t own = nullptr;      // private stream (default work stream, capture stream)
    float *J32 = nullptr;            // [Np][Np]
    uint8_t *J8 = nullptr;           // [Np][Np], FP8 e4m3, created on first FP8 run
    uint8_t *J4 = nullptr;           // [Np][Kp/2], packed e2m1, created on first FP4 run
    int Kp = 0;                      // Np rounded up to 256 (FP4 row length in values)
    // run buffers, sized for Rcap padded replicas
    int Rcap = 0;
    float *X[2] = {nullptr, nullptr};
    float *Y = nullptr;
    uint8_t *S8[2] = {nullptr, nullptr};
    uint8_t *S4[2] = {nullptr, nullptr};  // [Rcap][Kp/2] packed e2m1 operand (FP4 runs)
    TcPlan *plan4 = nullptr;              // tensor maps of J4 and S4
    float *Epart = nullptr;
    float *Tpart = nullptr;  // [nblk][Rp] sums of y^2 for the trace
    double *trace = nullptr; // [n_traced][3] {min E, mean E, mean T_inst}
    size_t trace_cap = 0, trace_len = 0;
    double *Ebest = nullptr;
    double *Efinal = nullptr;
    double *Efpart = nullptr;  // partial sums of the binary64 final energies (and trace)
    unsigned *trace_ticket = nullptr;  // block ticket of the trace reduction, kept at zero
    double *xi = nullptr;    // [Rp] Nose-Hoover xi per replica
    float *gvec = nullptr;   // [Rp] friction factor fl32(-xi dt) of the next step
    bool have_xi = false;    // the last run used the Nose-Hoover thermostat
    int debug_drop_mb = -1;  // failure-detection test hook, consumed by the next launch
    int8_t *Sbest = nullptr;
    int *err = nullptr;
    uint64_t buffers_gen = 0;
    TcPlan *plan = nullptr;
    // persistent FP8 schedule: flags, p_k table, per-evaluation partials and
    // spin snapshots
    int *flags = nullptr;  // [2][nblk][nrb] strided: sign tiles, Nose-Hoover sums
    size_t flags_cap = 0;
    unsigned long long *nhpart = nullptr;  // [3][nblk][Rp][2] Nose-Hoover tile sums
    size_t nhpart_cap = 0;
    // per-step trace on the persistent kernel: row-block sums of every traced
    // step, the batched reduction's scratch and its tickets (kept at zero)
    float *trE = nullptr, *trT = nullptr;
    size_t trE_cap = 0, trT_cap = 0;
    double *tr_scratch = nullptr;
    size_t tr_scratch_cap = 0;
    unsigned *tr_tickets = nullptr;
    size_t tr_tickets_cap = 0;
    float *pk_dev = nullptr;
    int pk_cap = 0, pk_steps = -1;
    double pk_a0 = 0.0;
    float *Eeval = nullptr;
    size_t eeval_cap = 0;
    // split-BF16 path: couplings [J_hi | J_lo], operand ping/pong, plan
    void *Jcat = nullptr;
    void *Xcat[2] = {nullptr, nullptr};
    Bf16Plan *bplan = nullptr;
    uint8_t *Snap = nullptr;
    size_t snap_cap = 0;
    // graph cache: the whole run, and the step range of hsb_advance_device
    bool graph_valid = false;
    GraphKey gkey{};
    cudaGraphExec_t gexec = nullptr;
    bool adv_valid = false;
    GraphKey adv_key{};
    int adv_k0 = 0, adv_k1 = 0, adv_par = 0;
    cudaGraphExec_t adv_exec = nullptr;
    // device state left by the last call, for hsb_get_state / hsb_advance_device
    int last_R = 0, last_x = 0;  // which X buffer holds x (FP32 path)
    int state_par = 0;           // ping/pong buffer holding the current state
    bool have_state = false;
    long long launches = 0;      // kernels queued by the last run
};

namespace {

void free_run_buffers(hsb_ctx *h)
{
    if (h->plan) {
        tc_plan_destroy(h->plan);
        h->plan = nullptr;
    }
    if (h->plan4) {
        tc_plan_destroy(h->plan4);
        h->plan4 = nullptr;
    }
    cudaFree(h->S4[0]);
    cudaFree(h->S4[1]);
    h->S4[0] = h->S4[1] = nullptr;
    if (h->bplan) {
        bf16_plan_destroy(h->bplan);
        h->bplan = nullptr;
    }
    cudaFree(h->Xcat[0]);
    cudaFree(h->Xcat[1]);
    h->Xcat[0] = h->Xcat[1] = nullptr;
    cudaFree(h->X[0]);
    cudaFree(h->X[1]);
    cudaFree(h->Y);
    cudaFree(h->S8[0]);
    cudaFree(h->S8[1]);
    cudaFree(h->Epart);
    cudaFree(h->Tpart);
    cudaFree(h->Ebest);
    cudaFree(h->Efinal);
    cudaFree(h->Efpart);
    h->Efpart = nullptr;
    cudaFree(h->trace_ticket);
    h->trace_ticket = nullptr;
    cudaFree(h->xi);
    cudaFree(h->gvec);
    h->xi = nullptr;
    h->gvec = nullptr;
    h->have_xi = false;
    cudaFree(h->Sbest);
    h->X[0] = h->X[1] = h->Y = nullptr;
    h->S8[0] = h->S8[1] = nullptr;
    h->Epart = nullptr;
    h->Tpart = nullptr;
    h->Ebest = h->Efinal = nullptr;
    h->Sbest = nullptr;
    h->Rcap = 0;
    h->have_state = false;
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    h->graph_valid = false;
    if (h->adv_exec) {
        cudaGraphExecDestroy(h->adv_exec);
        h->adv_exec = nullptr;
    }
    h->adv_valid = false;
}

hsb_status ensure_buffers(hsb_ctx *h, int Rp, int R)
{
    // Every buffer is sized for Rcap >= Rp >= R padded replicas.
    (void)R;
    if (Rp <= h->Rcap && h->X[0])
        return HSB_OK;
    free_run_buffers(h);
    const size_t elems = (size_t)Rp * h->Np;
    CK(dev_alloc(&h->X[0], elems * sizeof(float)), "cudaMalloc X");
    CK(dev_alloc(&h->X[1], elems * sizeof(float)), "cudaMalloc X");
    CK(dev_alloc(&h->Y, elems * sizeof(float)), "cudaMalloc Y");
    CK(dev_alloc(&h->S8[0], elems), "cudaMalloc S8");
    CK(dev_alloc(&h->S8[1], elems), "cudaMalloc S8");
    CK(dev_alloc(&h->Epart, (size_t)(h->Np / kTileM) * Rp * sizeof(float)), "cudaMalloc Epart");
    CK(dev_alloc(&h->Tpart, (size_t)(h->Np / kTileM) * Rp * sizeof(float)), "cudaMalloc Tpart");
    CK(dev_alloc(&h->Ebest, (size_t)Rp * sizeof(double)), "cudaMalloc Ebest");
    CK(dev_alloc(&h->Efinal, (size_t)Rp * sizeof(double)), "cudaMalloc Efinal");
    CK(dev_alloc(&h->Efpart, final_energy_part_doubles(Rp) * sizeof(double)),
       "cudaMalloc Efpart");
    CK(dev_alloc(&h->trace_ticket, sizeof(unsigned)), "cudaMalloc trace ticket");
    // on the work stream: the kernels that read it run there (a non-blocking
    // stream is not ordered after the legacy default stream)
    CK(cudaMemsetAsync(h->trace_ticket, 0, sizeof(unsigned), h->work), "cudaMemset trace ticket");
    CK(dev_alloc(&h->xi, (size_t)Rp * sizeof(double)), "cudaMalloc xi");
    CK(dev_alloc(&h->gvec, (size_t)Rp * sizeof(float)), "cudaMalloc gvec");
    CK(dev_alloc(&h->Sbest, (size_t)Rp * h->N), "cudaMalloc Sbest");
    h->Rcap = Rp;
    h->buffers_gen++;
    return HSB_OK;
}

hsb_status ensure_fp8(hsb_ctx *h)
{
    if (!h->J8) {
        CK(dev_alloc(&h->J8, (size_t)h->Np * h->Np), "cudaMalloc J8");
        CK(launch_j_to_fp8(h->work, h->J32, h->Np, h->J8), "j_to_fp8");
    }
    if (!h->plan) {
        CK(tc_fp8_plan_create(&h->plan, h->J8, h->S8[0], h->S8[1], h->Np, h->Rcap),
           "tc_fp8_plan_create");
        // A captured step loop holds the old plan's tensor maps, which may name
        // a J8 that hsb_set_couplings has freed since: such a graph must not
        // be replayed, and the generation is part of its key.
        h->buffers_gen++;
    }
    return HSB_OK;
}

hsb_status ensure_fp4(hsb_ctx *h)
{
    if (!h->J4) {
        CK(dev_alloc(&h->J4, (size_t)h->Np * (h->Kp / 2)), "cudaMalloc J4");
        CK(launch_j_to_fp4(h->work, h->J32, h->Np, h->Kp, h->J4), "j_to_fp4");
    }
    for (int b = 0; b < 2; ++b)
        if (!h->S4[b]) {
            CK(dev_alloc(&h->S4[b], (size_t)h->Rcap * (h->Kp / 2)), "cudaMalloc S4");
            CK(cudaMemsetAsync(h->S4[b], 0, (size_t)h->Rcap * (h->Kp / 2), h->work),
               "memset S4");
        }
    if (!h->plan4) {
        CK(tc_fp4_plan_create(&h->plan4, h->J4, h->S4[0], h->S4[1], h->Np, h->Kp, h->Rcap),
           "tc_fp4_plan_create");
        h->buffers_gen++;  // as for the FP8 plan: captured loops name these maps
    }
    return HSB_OK;
}

hsb_status ensure_bf16(hsb_ctx *h)
{
    const size_t np = (size_t)h->Np;
    if (!h->Jcat) {
        CK(dev_alloc(&h->Jcat, np * 2 * np * 2), "cudaMalloc Jcat");
        CK(launch_split_couplings(h->work, h->J32, h->Np, h->Jcat), "split couplings");
    }
    for (int b = 0; b < 2; ++b)
        if (!h->Xcat[b]) {
            CK(dev_alloc(&h->Xcat[b], (size_t)h->Rcap * 2 * np * 2), "cudaMalloc Xcat");
            CK(cudaMemsetAsync(h->Xcat[b], 0, (size_t)h->Rcap * 2 * np * 2, h->work),
               "memset Xcat");
        }
    if (!h->bplan)
        CK(bf16_plan_create(&h->bplan, h->Jcat, h->Xcat[0], h->Xcat[1], h->Np, h->Rcap),
           "bf16_plan_create");
    return HSB_OK;
}

hsb_status resolve(const hsb_ctx *h, const hsb_params *p, int R, int steps, RunCfg *cfg)
{
    if (!p)
        return set_error(HSB_E_INVAL, "params is NULL");
    if (R < 1)
        return set_error(HSB_E_INVAL, "R must be >= 1 (got %d)", R);
    if (steps < 1)
        return set_error(HSB_E_INVAL, "steps must be >= 1 (got %d)", steps);
    if (p->form != HSB_BALLISTIC && p->form != HSB_DISCRETE)
        return set_error(HSB_E_INVAL, "form must be HSB_BALLISTIC or HSB_DISCRETE");
    if (!(p->a0 > 0.0) || !(p->dt > 0.0) || !(p->gamma >= 0.0) || !(p->init_half_width > 0.0))
        return set_error(HSB_E_INVAL, "need a0 > 0, dt > 0, gamma >= 0, init_half_width > 0");
    if (!(p->c0 > 0.0) && !(p->c1 > 0.0))
        return set_error(HSB_E_INVAL, "need c0 > 0 or c1 > 0");
    if (p->eval_every < 0 || p->trace_every < 0)
        return set_error(HSB_E_INVAL, "eval_every and trace_every must be >= 0");
    if (p->schedule < 0 || p->schedule > 4)
        return set_error(HSB_E_INVAL, "schedule must be 0, 1, 2, 3 or 4");
    if (p->thermostat != HSB_HEAT_CONSTANT && p->thermostat != HSB_HEAT_NOSE_HOOVER)
        return set_error(HSB_E_INVAL, "thermostat must be HSB_HEAT_CONSTANT or "
                                      "HSB_HEAT_NOSE_HOOVER");
    const bool nose_hoover = p->thermostat == HSB_HEAT_NOSE_HOOVER;
    if (nose_hoover && (!(p->nh_M > 0.0) || !(p->nh_T >= 0.0) || !std::isfinite(p->nh_M) ||
                        !std::isfinite(p->nh_T) || !std::isfinite(p->nh_xi0)))
        return set_error(HSB_E_INVAL, "Nose-Hoover needs finite nh_M > 0, nh_T >= 0 and nh_xi0");
    if ((long long)R * h->N > (1LL << 40))
        return set_error(HSB_E_INVAL, "R*N too large");
    int prec = p->prec;
    const int Rp_ = round_up(R, kTileR);
    if (prec == HSB_PREC_AUTO) {
        if (p->form == HSB_DISCRETE && h->pm1)
            prec = HSB_PREC_FP8;
        else
            prec = !nose_hoover && tc_bf16_persistent_fits(h->Np, Rp_) ? HSB_PREC_BF16X3
                                                                       : HSB_PREC_FP32;
    }
    if (prec == HSB_PREC_FP8 && !(p->form == HSB_DISCRETE && h->pm1))
        return set_error(HSB_E_UNSUPPORTED,
                         "FP8 needs the discrete form and couplings in {-1, 0, +1}");
    if (prec == HSB_PREC_FP4 && !(p->form == HSB_DISCRETE && h->pm1))
        return set_error(HSB_E_UNSUPPORTED,
                         "FP4 needs the discrete form and couplings in {-1, 0, +1}");
    if (prec == HSB_PREC_FP4 && p->schedule != 0 && p->schedule != 1 && p->schedule != 2)
        return set_error(HSB_E_UNSUPPORTED,
                         "FP4 runs the persistent kernel or one launch per step (schedule 0, "
                         "1 or 2)");
    if (prec == HSB_PREC_BF16X3 && !tc_bf16_persistent_fits(h->Np, Rp_))
        return set_error(HSB_E_UNSUPPORTED,
                         "BF16X3 runs as one persistent kernel; its %d x %d grid does not fit",
                         h->Np / kTileM, Rp_ / kTileR);
    if (prec != HSB_PREC_FP32 && prec != HSB_PREC_FP8 && prec != HSB_PREC_BF16X3 &&
        prec != HSB_PREC_FP4)
        return set_error(HSB_E_INVAL, "unknown precision %d", p->prec);
    if (p->trace_every > 0 && prec == HSB_PREC_BF16X3)
        return set_error(HSB_E_UNSUPPORTED, "the trace needs the FP32 or FP8 precision");
    if (p->trace_every > 0 && prec == HSB_PREC_FP8 && p->schedule == 3)
        return set_error(HSB_E_UNSUPPORTED, "the trace does not run on the resident-J schedule");
    if (nose_hoover && prec == HSB_PREC_BF16X3)
        return set_error(HSB_E_UNSUPPORTED, "the Nose-Hoover thermostat needs FP32 or FP8");
    if (nose_hoover && prec == HSB_PREC_FP8 && p->schedule == 3)
        return set_error(HSB_E_UNSUPPORTED,
                         "the Nose-Hoover thermostat does not run on the resident-J schedule");
    cfg->prec = prec;
    cfg->form = p->form;
    cfg->R = R;
    cfg->Rp = round_up(R, kTileR);
    cfg->steps = steps;
    cfg->eval_every = p->eval_every;
    cfg->trace_every = p->trace_every;
    cfg->schedule = p->schedule;
    cfg->a0 = p->a0;
    cfg->thermo = nose_hoover ? 1 : 0;
    cfg->nh_h = nose_hoover ? p->dt / p->nh_M : 0.0;
    cfg->nh_NT = nose_hoover ? (double)h->N * p->nh_T : 0.0;
    cfg->nh_xi0 = nose_hoover ? p->nh_xi0 : 0.0;
    cfg->dt64 = p->dt;
    // c0 = c1 / (sqrt(N) sigma_J) (Results; sigma_J = 1 for +/-1 couplings)
    const double c0 = p->c0 > 0.0 ? p->c0 : p->c1 / (sqrt((double)h->N) * h->sigma);
    cfg->c.c0 = (float)c0;
    cfg->c.dt = (float)p->dt;
    cfg->c.q = (float)(p->a0 * p->dt);
    cfg->c.g = (float)(p->gamma * p->dt);
    cfg->c.nz = -0.0f;
    cfg->pk.resize(steps);
    for (int k = 0; k < steps; ++k) {
        // a(t_k) = a0 k / Ns, linear from 0 to a0 (Results); p_k = a0 - a(t_k)
        double t = p->a0 * (double)k;
        t = t / (double)steps;
        cfg->pk[k] = (float)(p->a0 - t);
    }
    return HSB_OK;
}

bool is_eval_step(const RunCfg &c, int k)
{
    return c.eval_every > 0 && k > 0 && k < c.steps && k % c.eval_every == 0;
}

// One step k of the loop (update from t_k to t_{k+1}); evaluates E(t_k) first
// when k is an evaluation step.  `cur` selects the ping/pong buffer holding
// the state at t_k (X for the FP32 path, the FP8 operand S8 otherwise).
hsb_status enqueue_step(hsb_ctx *h, cudaStream_t st, const RunCfg &c, int k, int cur,
                        bool allow_eval)
{
    const bool ev = allow_eval && is_eval_step(c, k);
    // traced time t_k: energy and T_inst of the state before this update
    const bool tr = allow_eval && c.trace_every > 0 && k % c.trace_every == 0;
    const bool en = ev || tr;
    float *tpart = tr ? h->Tpart : nullptr;
    const int nblk = h->Np / kTileM;
    const float *gv = c.thermo ? h->gvec : nullptr;  // Nose-Hoover friction per replica
    if (c.prec == HSB_PREC_FP32) {
        if (en && c.form == HSB_BALLISTIC)
            CK(launch_simt_step(st, 1, true, true, h->J32, h->N, h->Np, c.Rp, h->X[cur], nullptr,
                                h->Y, 0.f, c.c, h->Epart, nullptr),
               "energy kernel");
        CK(launch_simt_step(st, c.form, false, en && c.form == HSB_DISCRETE, h->J32, h->N, h->Np,
                            c.Rp, h->X[cur], h->X[cur ^ 1], h->Y, c.pk[k], c.c, h->Epart, tpart,
                            gv),
           "fp32 step kernel");
        if (ev)
            CK(launch_best_update(st, h->Epart, nblk, h->N, h->Np, c.R, c.Rp, h->X[cur], nullptr,
                                  h->Ebest, h->Sbest),
               "best kernel");
    } else if (c.prec == HSB_PREC_FP4) {  // S4[cur] -> S4[cur^1], X and Y in place
        CK(launch_tc_fp4_step(st, h->plan4, cur, en, false, h->N, c.Rp, h->X[0], h->Y, c.pk[k],
                              c.c, h->Epart, tpart, h->S4[cur ^ 1], h->err, gv),
           "fp4 step kernel");
        if (ev)
            CK(launch_best_update(st, h->Epart, nblk, h->N, h->Np, c.R, c.Rp, nullptr, nullptr,
                                  h->Ebest, h->Sbest, h->S4[cur], h->Kp),
               "best kernel");
    } else {  // FP8: S8[cur] -> S8[cur^1], X and Y in place
        CK(launch_tc_fp8_step(st, h->plan, cur, en, false, h->N, c.Rp, h->X[0], h->Y, c.pk[k],
                              c.c, h->Epart, tpart, h->S8[cur ^ 1], h->err, gv),
           "fp8 step kernel");
        if (ev)
            CK(launch_best_update(st, h->Epart, nblk, h->N, h->Np, c.R, c.Rp, nullptr, h->S8[cur],
                                  h->Ebest, h->Sbest),
               "best kernel");
    }
    if (tr)
        CK(launch_trace_reduce(st, h->Epart, h->Tpart, nblk, h->N, c.R, c.Rp,
                               h->Efpart, h->trace_ticket,
                               h->trace + 3 * (size_t)(k / c.trace_every)),
           "trace kernel");
    if (c.thermo)  // xi_{k+1} from y(t_{k+1}), Eq. (eq_NH)
        CK(launch_nh_update(st, h->Y, h->N, h->Np, c.R, c.nh_h, c.nh_NT, c.dt64, h->xi, h->gvec,
                            h->err),
           "Nose-Hoover kernel");
    return HSB_OK;
}

// Final evaluation at t_steps, best update and (general J) binary64 energies.
hsb_status enqueue_final(hsb_ctx *h, cudaStream_t st, const RunCfg &c)
{
    const int nblk = h->Np / kTileM;
    const int cur = c.steps & 1;
    if (c.prec == HSB_PREC_FP32) {
        CK(launch_simt_step(st, 1, true, true, h->J32, h->N, h->Np, c.Rp, h->X[cur], nullptr,
                            h->Y, 0.f, c.c, h->Epart, nullptr),
           "energy kernel");
        CK(launch_best_update(st, h->Epart, nblk, h->N, h->Np, c.R, c.Rp, h->X[cur], nullptr,
                              h->Ebest, h->Sbest),
           "best kernel");
    } else if (c.prec == HSB_PREC_FP4) {
        CK(launch_tc_fp4_step(st, h->plan4, cur, true, true, h->N, c.Rp, h->X[0], h->Y, 0.f, c.c,
                              h->Epart, nullptr, nullptr, h->err),
           "fp4 energy kernel");
        CK(launch_best_update(st, h->Epart, nblk, h->N, h->Np, c.R, c.Rp, nullptr, nullptr,
                              h->Ebest, h->Sbest, h->S4[cur], h->Kp),
           "best kernel");
    } else {
        CK(launch_tc_fp8_step(st, h->plan, cur, true, true, h->N, c.Rp, h->X[0], h->Y, 0.f, c.c,
                              h->Epart, nullptr, nullptr, h->err),
           "fp8 energy kernel");
        CK(launch_best_update(st, h->Epart, nblk, h->N, h->Np, c.R, c.Rp, nullptr, h->S8[cur],
                              h->Ebest, h->Sbest),
           "best kernel");
    }
    if (!h->pm1)
        CK(launch_final_energy_f64_parts(st, h->J32, h->N, h->Np, c.R, h->Sbest, h->jscale,
                                         h->Efpart, h->Efinal),
           "final energy kernel");
    return HSB_OK;
}

// Kernels one run queues: init, the steps, the energy evaluations of the
// ballistic form, the best updates, the final evaluation and (general J) the
// binary64 energies.
long long count_launches(const hsb_ctx *h, const RunCfg &c)
{
    long long evals = c.eval_every > 0 ? (c.steps - 1) / c.eval_every : 0;
    long long n = 1 + c.steps + evals /* best */ + 2 /* final energy + best */;
    if (c.form == HSB_BALLISTIC && c.prec == HSB_PREC_FP32)
        n += evals;
    if (c.trace_every > 0) {
        const long long traced = (c.steps - 1) / c.trace_every + 1;
        n += traced;  // trace reductions
        if (c.form == HSB_BALLISTIC && c.prec == HSB_PREC_FP32)
            n += traced;  // energy passes at traced times (shared with evaluations)
    }
    if (!h->pm1)
        n += 1;
    if (c.prec == HSB_PREC_FP4)
        n += 1;  // sign of x0 packed into the e2m1 operand
    if (c.thermo)
        n += 1 + c.steps;  // xi init, one xi update per step
    return n;
}

hsb_status build_graph(hsb_ctx *h, const RunCfg &c, const GraphKey &key)
{
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    h->graph_valid = false;
    CK(cudaStreamBeginCapture(h->own, cudaStreamCaptureModeThreadLocal), "begin capture");
    hsb_status s = HSB_OK;
    for (int k = 0; k < c.steps && s == HSB_OK; ++k)
        s = enqueue_step(h, h->own, c, k, k & 1, true);
    if (s == HSB_OK)
        s = enqueue_final(h, h->own, c);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->own, &graph);
    if (s != HSB_OK) {
        if (graph)
            cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess)
        return cuda_error(e, "end capture");
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return cuda_error(e, "graph instantiate");
    h->gkey = key;
    h->graph_valid = true;
    return HSB_OK;
}

hsb_status prepare(hsb_ctx *h, const RunCfg &c)
{
    hsb_status s = ensure_buffers(h, c.Rp, c.R);
    if (s != HSB_OK)
        return s;
    if (c.prec == HSB_PREC_FP8) {
        s = ensure_fp8(h);
        if (s != HSB_OK)
            return s;
    }
    if (c.prec == HSB_PREC_FP4) {
        s = ensure_fp4(h);
        if (s != HSB_OK)
            return s;
    }
    if (c.prec == HSB_PREC_BF16X3) {
        s = ensure_bf16(h);
        if (s != HSB_OK)
            return s;
    }
    return HSB_OK;
}

// Eq. (eq_Ising): J_ij = J_ji and J_ii = 0 (host, row-major N x N).  Also
// reports whether every entry is -1, 0 or +1, and sum_ij J_ij^2 and
// sum_ij J_ij (sigma_J and the cut offset) as the binary64 sums taken row by
// row with j ascending.  Symmetry is checked in 64 x 64 block pairs over the
// upper triangle; for +/-1 couplings every partial sum is an integer below
// 2^53, so integer counts give the same binary64 values.  Row blocks are
// split over a few host threads (interleaved, for balance); every result is
// a boolean or an exact integer, so the split does not change it.  General
// couplings take the sequential binary64 sums afterwards.
struct CouplingScan {
    long long nonzero = 0, signed_sum = 0;
    bool other = false;           // an entry outside {-1, 0, +1}
    int ai = -1, aj = -1;         // first asymmetric pair found (i < j)
};

void scan_row_blocks(const float *J, int N, int first, int stride, CouplingScan *out)
{
    constexpr int kB = 64;
    const size_t n = (size_t)N;
    CouplingScan r;
    for (int ib = first * kB; ib < N && r.ai < 0; ib += stride * kB) {
        const int ie = std::min(ib + kB, N);
        for (int jb = ib; jb < N && r.ai < 0; jb += kB) {
            const int je = std::min(jb + kB, N);
            for (int i = ib; i < ie && r.ai < 0; ++i)
                for (int j = std::max(jb, i + 1); j < je; ++j)
                    if (!(J[(size_t)i * n + j] == J[(size_t)j * n + i])) {
                        r.ai = i;
                        r.aj = j;
                        break;
                    }
        }
        for (int i = ib; i < ie; ++i) {
            // branch-free (random signs would defeat branch prediction)
            const float *row = J + (size_t)i * n;
            int nz = 0, sg = 0, other = 0;
            for (int jj = 0; jj < N; ++jj) {
                const float v = row[jj];
                const int p = v == 1.0f, m = v == -1.0f, z = v == 0.0f;
                nz += p + m;
                sg += p - m;
                other |= (p | m | z) ^ 1;
            }
            r.nonzero += nz;
            r.signed_sum += sg;
            r.other = r.other || other != 0;
        }
    }
    *out = r;
}

hsb_status validate_couplings(const float *J, int N, int *pm1_out, double *sum2_out,
                              double *sumJ_out, double *maxabs_out)
{
    const size_t n = (size_t)N;
    for (int i = 0; i < N; ++i)
        if (J[(size_t)i * n + i] != 0.0f)
            return set_error(HSB_E_DIAG, "J[%d][%d] = %g is not zero", i, i,
                             (double)J[(size_t)i * n + i]);
    const unsigned hw = std::thread::hardware_concurrency();
    int nt = N >= 1024 ? (int)std::min(8u, hw ? hw : 1u) : 1;
    std::vector<CouplingScan> part((size_t)nt);
    std::vector<std::thread> pool;
    try {
        for (int t = 1; t < nt; ++t)
            pool.emplace_back(scan_row_blocks, J, N, t, nt, &part[(size_t)t]);
    } catch (...) {
        // no threads to be had: scan the remaining row blocks here
        for (size_t t = pool.size() + 1; t < (size_t)nt; ++t)
            scan_row_blocks(J, N, (int)t, nt, &part[t]);
    }
    scan_row_blocks(J, N, 0, nt, &part[0]);
    for (std::thread &th : pool)
        th.join();
    long long nonzero = 0, signed_sum = 0;
    bool pm1 = true;
    int ai = -1, aj = -1;
    for (const CouplingScan &r : part) {
        nonzero += r.nonzero;
        signed_sum += r.signed_sum;
        pm1 = pm1 && !r.other;
        if (r.ai >= 0 && (ai < 0 || r.ai < ai || (r.ai == ai && r.aj < aj))) {
            ai = r.ai;
            aj = r.aj;
        }
    }
    if (ai >= 0)
        return set_error(HSB_E_ASYM, "J[%d][%d] != J[%d][%d]", ai, aj, aj, ai);
    double sum2 = 0.0, sumJ = 0.0, maxabs = 1.0;
    if (pm1) {
        sum2 = (double)nonzero;
        sumJ = (double)signed_sum;
    } else {
        // sigma_J^2 = sum_ij J_ij^2 / (N(N-1)), summed row by row in binary64
        maxabs = 0.0;
        for (size_t e = 0; e < n * n; ++e) {
            const double d = (double)J[e];
            sum2 += d * d;
            sumJ += d;
            maxabs = std::max(maxabs, std::fabs(d));
        }
    }
    if (!std::isfinite(sum2))
        return set_error(HSB_E_INVAL, "J has an infinite entry");
    if (!(sum2 > 0.0))
        return set_error(HSB_E_INVAL, "J is all zero");
    *pm1_out = pm1 ? 1 : 0;
    *sum2_out = sum2;
    *sumJ_out = sumJ;
    *maxabs_out = maxabs;
    return HSB_OK;
}

// Exponent s of the fixed-point final energies: max |J| 2^s < 2^40.
int energy_scale_exp(double maxabs)
{
    int e = 0;
    std::frexp(maxabs, &e);  // maxabs = m 2^e, m in [0.5, 1): maxabs < 2^e
    return 40 - e;
}

GraphKey make_key(const hsb_ctx *h, const RunCfg &c);
GraphKey make_key(const hsb_ctx *h, const RunCfg &c);

int num_evals(const RunCfg &c)
{
    return (c.eval_every > 0 ? (c.steps - 1) / c.eval_every : 0) + 1;
}

// Whether the FP8 step loop runs on the CTA-pair kernel: schedule 4, or the
// automatic choice when the one-CTA persistent grid does not fit.  It needs
// constant heating, no per-step trace, N <= 4096, an even number of
// 128-replica blocks and a grid that fits.
bool use_pair(const hsb_ctx *h, const RunCfg &c)
{
    if (c.prec != HSB_PREC_FP8 || (c.schedule != 0 && c.schedule != 4) || c.thermo ||
        c.trace_every > 0)
        return false;
    if (c.schedule == 0 && tc_persistent_fits(h->Np, c.Rp))
        return false;
    return tc_pair_fits(h->Np, c.Rp);
}

// Whether the FP8 (or FP4) step loop runs as one persistent kernel.
hsb_status use_persistent(const hsb_ctx *h, const RunCfg &c, bool *out)
{
    *out = false;
    if (c.prec == HSB_PREC_FP4 && c.schedule != 2) {
        const bool fits = tc_fp4_persistent_fits(h->Np, c.Rp);
        if (!fits && c.schedule == 1)
            return set_error(HSB_E_UNSUPPORTED,
                             "the persistent kernel's %d x %d grid does not fit on the device",
                             h->Np / kTileM, c.Rp / kTileR);
        *out = fits;
        return HSB_OK;
    }
    if (c.prec != HSB_PREC_FP8 || c.schedule == 2)
        return HSB_OK;
    if (c.schedule == 4) {
        if (!use_pair(h, c))
            return set_error(HSB_E_UNSUPPORTED,
                             "the CTA-pair schedule needs constant heating, no trace, N <= 4096 "
                             "and an even number of 128-replica blocks whose grid fits");
        *out = true;
        return HSB_OK;
    }
    if (use_pair(h, c)) {
        *out = true;
        return HSB_OK;
    }
    const bool fits = c.schedule == 3 ? tc_resident_fits(h->Np, c.Rp)
                                      : tc_persistent_fits(h->Np, c.Rp);
    if (!fits && (c.schedule == 1 || c.schedule == 3))
        return set_error(HSB_E_UNSUPPORTED,
                         "the persistent kernel's %d x %d grid does not fit on the device",
                         h->Np / kTileM, c.Rp / kTileR);
    *out = fits;
    return HSB_OK;
}

template <typename T>
hsb_status grow(T **ptr, size_t *cap, size_t n, const char *what)
{
    if (*cap >= n && *ptr)
        return HSB_OK;
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    CK(dev_alloc(ptr, n * sizeof(T)), what);
    *cap = n;
    return HSB_OK;
}

// Device p_k table of the run (uploaded when steps or a0 change).
hsb_status ensure_pk(hsb_ctx *h, const RunCfg &c)
{
    if (h->pk_steps == c.steps && h->pk_a0 == c.a0 && h->pk_dev)
        return HSB_OK;
    if (h->pk_cap < c.steps) {
        cudaFree(h->pk_dev);
        h->pk_dev = nullptr;
        h->pk_cap = 0;
        CK(dev_alloc(&h->pk_dev, (size_t)c.steps * sizeof(float)), "cudaMalloc pk");
        h->pk_cap = c.steps;
    }
    CK(cudaMemcpyAsync(h->pk_dev, c.pk.data(), (size_t)c.steps * sizeof(float),
                       cudaMemcpyHostToDevice, h->work),
       "copy pk");
    CK(cudaStreamSynchronize(h->work), "synchronize");
    h->pk_steps = c.steps;
    h->pk_a0 = c.a0;
    return HSB_OK;
}

// Queues the persistent kernel for updates [k_begin, k_begin + nsteps) of the
// run's schedule, starting from operand buffer par0.
hsb_status enqueue_persistent(hsb_ctx *h, const RunCfg &c, int k_begin, int nsteps,
                              bool evaluate, int par0)
{
    const int nblk = h->Np / kTileM;
    const int nrb = c.Rp / kTileR;
    const int ne = evaluate ? num_evals(c) : 0;
    hsb_status s = ensure_pk(h, c);
    const size_t nflags = (size_t)nblk * nrb * kFlagStride;
    if (s == HSB_OK)
        s = grow(&h->flags, &h->flags_cap, 2 * nflags, "cudaMalloc flags");
    if (s == HSB_OK && c.thermo)
        s = grow(&h->nhpart, &h->nhpart_cap, (size_t)3 * nblk * c.Rp * 2, "cudaMalloc nhpart");
    const bool traced = evaluate && c.trace_every > 0;
    const int ntr = traced ? (c.steps - 1) / c.trace_every + 1 : 0;
    const int nparts = (c.R + 31) / 32;
    if (s == HSB_OK && traced)
        s = grow(&h->trE, &h->trE_cap, (size_t)ntr * nblk * c.Rp, "cudaMalloc trace sums");
    if (s == HSB_OK && traced)
        s = grow(&h->trT, &h->trT_cap, (size_t)ntr * nblk * c.Rp, "cudaMalloc trace sums");
    if (s == HSB_OK && traced)
        s = grow(&h->tr_scratch, &h->tr_scratch_cap, (size_t)3 * nparts * ntr,
                 "cudaMalloc trace scratch");
    if (s == HSB_OK && traced && h->tr_tickets_cap < (size_t)ntr) {
        s = grow(&h->tr_tickets, &h->tr_tickets_cap, (size_t)ntr, "cudaMalloc trace tickets");
        if (s == HSB_OK)
            CK(cudaMemsetAsync(h->tr_tickets, 0, h->tr_tickets_cap * sizeof(unsigned), h->work),
               "memset trace tickets");
    }
    if (s == HSB_OK && evaluate)
        s = grow(&h->Eeval, &h->eeval_cap, (size_t)ne * nblk * c.Rp, "cudaMalloc Eeval");
    if (s == HSB_OK && evaluate)
        s = grow(&h->Snap, &h->snap_cap, (size_t)ne * c.Rp * h->Np, "cudaMalloc snapshots");
    if (s != HSB_OK)
        return s;
    CK(cudaMemsetAsync(h->flags, 0, (c.thermo ? 2 : 1) * nflags * sizeof(int), h->work),
       "memset flags");
    PersistArgs a;
    memset(&a, 0, sizeof a);
    a.N = h->N;
    a.Np = h->Np;
    a.Rp = c.Rp;
    a.nblk = nblk;
    a.nrb = nrb;
    a.k_begin = k_begin;
    a.nsteps = nsteps;
    a.final_pass = evaluate ? 1 : 0;
    a.eval_every = evaluate ? c.eval_every : 0;
    a.steps_total = c.steps;
    a.n_evals = ne;
    a.par0 = par0;
    a.pk = h->pk_dev;
    a.c = c.c;
    a.X = h->X[0];
    a.Y = h->Y;
    a.S8a = h->S8[0];
    a.S8b = h->S8[1];
    a.flags = h->flags;
    a.Epart = h->Eeval;
    a.Snap = h->Snap;
    a.err = h->err;
    if (traced) {
        a.trace_every = c.trace_every;
        a.trE = h->trE;
        a.trT = h->trT;
    }
    a.drop_mb = -1;
    if (c.schedule != 3) {
        a.drop_mb = h->debug_drop_mb;
        h->debug_drop_mb = -1;
    }
    if (c.thermo) {
        // Nose-Hoover: xi (set by launch_nh_init) in and out, tile sums, flags
        a.nh = 1;
        a.nh_h = c.nh_h;
        a.nh_NT = c.nh_NT;
        a.dt64 = c.dt64;
        a.xi = h->xi;
        a.nhpart = h->nhpart;
        a.nhflags = h->flags + nflags;
    }
    // the CTA-pair kernel where it applies; schedule 3: J resident on chip;
    // otherwise J streamed every step
    if (c.prec == HSB_PREC_FP4) {
        a.S8a = h->S4[0];
        a.S8b = h->S4[1];
        a.Kp = h->Kp;
        CK(launch_tc_fp4_persistent(h->work, h->plan4, a), "persistent fp4 kernel");
    } else if (use_pair(h, c))
        CK(launch_tc_fp8_pair(h->work, h->plan, a), "pair fp8 kernel");
    else if (c.schedule == 3)
        CK(launch_tc_fp8_resident(h->work, h->plan, h->J8, a), "resident fp8 kernel");
    else
        CK(launch_tc_fp8_persistent(h->work, h->plan, a), "persistent fp8 kernel");
    if (evaluate)
        CK(launch_select_best(h->work, h->Eeval, h->Snap, ne, nblk, h->N, h->Np, c.R, c.Rp,
                              h->Ebest, h->Sbest),
           "select best kernel");
    if (traced)
        CK(launch_trace_reduce_many(h->work, h->trE, h->trT, nblk, h->N, c.R, c.Rp, ntr,
                                    h->tr_scratch, h->tr_tickets, h->trace),
           "trace kernel");
    return HSB_OK;
}

// Queues the split-BF16 persistent kernel for updates [k_begin, k_begin +
// nsteps) from operand buffer par0 (state in X[0], Y).
hsb_status enqueue_bf16(hsb_ctx *h, const RunCfg &c, int k_begin, int nsteps, int par0)
{
    const int nblk = h->Np / kTileM;
    const int nrb = c.Rp / kTileR;
    hsb_status s = ensure_pk(h, c);
    if (s == HSB_OK)
        s = grow(&h->flags, &h->flags_cap, (size_t)nblk * nrb * kFlagStride, "cudaMalloc flags");
    if (s != HSB_OK)
        return s;
    CK(cudaMemsetAsync(h->flags, 0, (size_t)nblk * nrb * kFlagStride * sizeof(int), h->work),
       "memset flags");
    PersistArgs a;
    memset(&a, 0, sizeof a);
    a.N = h->N;
    a.Np = h->Np;
    a.Rp = c.Rp;
    a.nblk = nblk;
    a.nrb = nrb;
    a.k_begin = k_begin;
    a.nsteps = nsteps;
    a.final_pass = 0;
    a.steps_total = c.steps;
    a.par0 = par0;
    a.pk = h->pk_dev;
    a.c = c.c;
    a.X = h->X[0];
    a.Y = h->Y;
    a.flags = h->flags;
    a.err = h->err;
    CK(launch_tc_bf16x3_persistent(h->work, h->bplan, c.form, a), "persistent bf16x3 kernel");
    return HSB_OK;
}

// Energy of s = sgn(x) for every replica on the split-BF16 tensor-core path:
// one energy-only pass of the discrete kernel over the operand buffer `buf`,
// which holds [sgn x | 0], writes Epart[nblk][Rp].
hsb_status enqueue_bf16_energy(hsb_ctx *h, const RunCfg &c, int buf)
{
    const int nblk = h->Np / kTileM;
    const int nrb = c.Rp / kTileR;
    CK(cudaMemsetAsync(h->flags, 0, (size_t)nblk * nrb * kFlagStride * sizeof(int), h->work),
       "memset flags");
    PersistArgs a;
    memset(&a, 0, sizeof a);
    a.N = h->N;
    a.Np = h->Np;
    a.Rp = c.Rp;
    a.nblk = nblk;
    a.nrb = nrb;
    a.nsteps = 0;
    a.final_pass = 1;
    a.steps_total = c.steps;
    a.par0 = buf;
    a.pk = h->pk_dev;
    a.c = c.c;
    a.X = h->X[0];
    a.Y = h->Y;
    a.flags = h->flags;
    a.Epart = h->Epart;
    a.err = h->err;
    CK(launch_tc_bf16x3_persistent(h->work, h->bplan, 1, a), "bf16x3 energy pass");
    return HSB_OK;
}

// Whole split-BF16 run: the step loop is cut at the evaluation steps; each
// evaluation is an energy-only tensor-core pass over sgn(x) (f = J_hi s +
// J_lo s, FP32 accumulation: the candidate energies) and a best update; the
// returned energies are recomputed in binary64 for the chosen spins.
hsb_status enqueue_run_bf16(hsb_ctx *h, const RunCfg &c, uint64_t seed, const hsb_params *p)
{
    const int nblk = h->Np / kTileM;
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->work), "memset err");
    CK(launch_init(h->work, seed, p->instance, (float)p->init_half_width, h->N, h->Np, c.R, c.Rp,
                   h->X[0], h->Y, nullptr, h->Ebest),
       "init kernel");
    CK(launch_split_state(h->work, h->X[0], h->N, h->Np, c.Rp, c.form, h->Xcat[0]),
       "split state");
    int par = 0, k = 0;
    long long launches = 2;
    while (k < c.steps) {
        int kb = c.steps;
        if (c.eval_every > 0) {
            const int next = (k / c.eval_every + 1) * c.eval_every;
            if (next < c.steps)
                kb = next;
        }
        hsb_status s = enqueue_bf16(h, c, k, kb - k, par);
        if (s != HSB_OK)
            return s;
        par = (par + (kb - k)) & 1;
        k = kb;
        // evaluation of s(t_k): at an evaluation step, and at the end.  The
        // discrete form has just published [sgn x | 0] into buffer par; the
        // ballistic form writes it into the idle buffer.
        int ebuf = par;
        if (c.form == 0) {
            ebuf = par ^ 1;
            CK(launch_split_state(h->work, h->X[0], h->N, h->Np, c.Rp, 1, h->Xcat[ebuf]),
               "sign operand");
            ++launches;
        }
        s = enqueue_bf16_energy(h, c, ebuf);
        if (s != HSB_OK)
            return s;
        CK(launch_best_update(h->work, h->Epart, nblk, h->N, h->Np, c.R, c.Rp, h->X[0], nullptr,
                              h->Ebest, h->Sbest),
           "best kernel");
        launches += 3;
    }
    if (!h->pm1) {
        CK(launch_final_energy_f64_parts(h->work, h->J32, h->N, h->Np, c.R, h->Sbest,
                                         h->jscale, h->Efpart, h->Efinal),
           "final energy kernel");
        launches += 2;
    }
    h->last_R = c.R;
    h->last_x = 0;
    h->state_par = par;
    h->have_state = true;
    h->have_xi = false;
    h->launches = launches;
    h->trace_len = 0;
    return HSB_OK;
}

// Queues a whole run (init, graph of the step loop) on the work stream.
// The trace buffer of a run: 3 doubles per traced time t_k, k = m trace_every
// < steps (sets trace_len; 0 without a trace).
hsb_status ensure_trace(hsb_ctx *h, const RunCfg &c)
{
    if (c.trace_every <= 0) {
        h->trace_len = 0;
        return HSB_OK;
    }
    const size_t need = 3 * (size_t)((c.steps - 1) / c.trace_every + 1);
    if (h->trace_cap < need) {
        cudaFree(h->trace);
        h->trace = nullptr;
        h->trace_cap = 0;
        CK(dev_alloc(&h->trace, need * sizeof(double)), "cudaMalloc trace");
        h->trace_cap = need;
        h->graph_valid = false;  // the captured loop holds the trace pointer
    }
    h->trace_len = need / 3;
    return HSB_OK;
}

hsb_status enqueue_run(hsb_ctx *h, const RunCfg &c, uint64_t seed, const hsb_params *p)
{
    hsb_status s = prepare(h, c);
    if (s != HSB_OK)
        return s;
    if (c.prec == HSB_PREC_BF16X3)
        return enqueue_run_bf16(h, c, seed, p);
    bool persistent = false;
    s = use_persistent(h, c, &persistent);
    if (s != HSB_OK)
        return s;
    if (persistent) {
        s = ensure_trace(h, c);
        if (s != HSB_OK)
            return s;
        CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->work), "memset err");
        CK(launch_init(h->work, seed, p->instance, (float)p->init_half_width, h->N, h->Np, c.R,
                       c.Rp, h->X[0], h->Y, c.prec == HSB_PREC_FP8 ? h->S8[0] : nullptr,
                       h->Ebest),
           "init kernel");
        if (c.prec == HSB_PREC_FP4)
            CK(launch_sign_to_fp4(h->work, h->X[0], h->N, h->Np, h->Kp, c.Rp, h->S4[0]),
               "fp4 sign kernel");
        if (c.thermo)
            CK(launch_nh_init(h->work, c.R, c.Rp, c.nh_xi0, c.dt64, h->xi, h->gvec), "xi init");
        s = enqueue_persistent(h, c, 0, c.steps, true, 0);
        if (s != HSB_OK)
            return s;
        h->last_R = c.R;
        h->last_x = 0;
        h->state_par = c.steps & 1;
        h->have_state = true;
        // init, (xi init), the step loop, best selection, trace entries in
        // launches of at most 65535
        const long long ntr = c.trace_every > 0 ? (c.steps - 1) / c.trace_every + 1 : 0;
        h->launches = 3 + (c.thermo ? 1 : 0) + (c.prec == HSB_PREC_FP4 ? 1 : 0) +
                      (ntr + 65534) / 65535;
        h->have_xi = c.thermo != 0;
        return HSB_OK;
    }
    s = ensure_trace(h, c);
    if (s != HSB_OK)
        return s;
    const GraphKey key = make_key(h, c);
    if (!h->graph_valid || !(h->gkey == key)) {
        s = build_graph(h, c, key);
        if (s != HSB_OK)
            return s;
    }
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->work), "memset err");
    CK(launch_init(h->work, seed, p->instance, (float)p->init_half_width, h->N, h->Np, c.R, c.Rp,
                   h->X[0], h->Y, c.prec == HSB_PREC_FP8 ? h->S8[0] : nullptr, h->Ebest),
       "init kernel");
    if (c.prec == HSB_PREC_FP4)
        CK(launch_sign_to_fp4(h->work, h->X[0], h->N, h->Np, h->Kp, c.Rp, h->S4[0]),
           "fp4 sign kernel");
    if (c.thermo)
        CK(launch_nh_init(h->work, c.R, c.Rp, c.nh_xi0, c.dt64, h->xi, h->gvec), "xi init");
    h->have_xi = c.thermo != 0;
    CK(cudaGraphLaunch(h->gexec, h->work), "graph launch");
    h->last_R = c.R;
    h->last_x = c.prec == HSB_PREC_FP32 ? (c.steps & 1) : 0;
    h->state_par = c.steps & 1;
    h->have_state = true;
    h->launches = count_launches(h, c);
    return HSB_OK;
}

GraphKey make_key(const hsb_ctx *h, const RunCfg &c)
{
    GraphKey key;
    memset(&key, 0, sizeof key);
    key.prec = c.prec;
    key.form = c.form;
    key.R = c.R;
    key.Rp = c.Rp;
    key.steps = c.steps;
    key.eval_every = c.eval_every;
    key.trace_every = c.trace_every;
    key.pm1 = h->pm1;
    key.c0 = c.c.c0;
    key.dt = c.c.dt;
    key.q = c.c.q;
    key.g = c.c.g;
    key.a0 = c.a0;
    key.thermo = c.thermo;
    key.nh_h = c.nh_h;
    key.nh_NT = c.nh_NT;
    key.dt64 = c.dt64;
    key.buffers_gen = h->buffers_gen;
    return key;
}

hsb_status check_device_error(hsb_ctx *h)
{
    int e = 0;
    CK(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->work), "read err");
    CK(cudaStreamSynchronize(h->work), "synchronize");
    if (e == kErrTimeout)
        return set_error(HSB_E_TIMEOUT, "a bounded device-side wait gave up");
    if (e == kErrRange)
        return set_error(HSB_E_INVAL, "a momentum reached |y| >= 256 in the Nose-Hoover sum");
    if (e != 0)
        return set_error(HSB_E_CUDA, "device error code %d", e);
    return HSB_OK;
}

}  // namespace

namespace hsb {
hsb_status report_error(hsb_status s, const char *msg)
{
    return set_error(s, "%s", msg);
}
}  // namespace hsb

// =================================================================== ABI ===

namespace {

// ---- batch autotuner ---------------------------------------------------
// The batched kernel runs one instance per CTA.  How many CTAs run at once
// trades SMs against L2: the FP8 couplings of the instances in flight share
// the L2, and once they exceed it every step re-reads them from HBM.  Whether
// K is split over two MMA warps trades tensor issue rate against accumulator
// room.  Every choice gives the same bits (each instance is computed by one
// CTA, with exact integer forces), so the choice is made by timing: on the
// first batch of a shape (device, instance count, replica width, total FP8
// coupling bytes rounded to a power of two) each candidate runs the whole
// queue for a short prefix of the steps, and the fastest is kept for the
// process.
struct BatchChoice {
    int ctas = 0;
    int split = 1;
};

struct BatchTuneKey {
    int device, count, BN, log2bytes, fp4;
    bool operator<(const BatchTuneKey &o) const
    {
        return std::tie(device, count, BN, log2bytes, fp4) <
               std::tie(o.device, o.count, o.BN, o.log2bytes, o.fp4);
    }
};

std::mutex g_tune_mu;
std::map<BatchTuneKey, BatchChoice> g_tune;

// CTA counts tried: the SM count down to a quarter of it.
std::vector<int> batch_cta_candidates(int sms, int count)
{
    std::vector<int> v;
    for (int num : {8, 7, 6, 5, 4, 3, 2}) {
        int c = std::min(count, std::max(1, sms * num / 8));
        if (std::find(v.begin(), v.end(), c) == v.end())
            v.push_back(c);
    }
    return v;
}

// Times one launch of the queue (queue counter reset before); returns ms or
// a negative value on error.
float time_batch(cudaStream_t st, const BatchInst *d_insts, BatchArgs a, int ctas)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return -1.f;
    float ms = -1.f;
    if (cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), st) == cudaSuccess &&
        cudaEventRecord(e0, st) == cudaSuccess &&
        launch_tc_batch(st, d_insts, a, ctas) == cudaSuccess &&
        cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess)
        cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

BatchChoice tune_batch(const BatchTuneKey &key, cudaStream_t st, const BatchInst *d_insts,
                       const BatchArgs &a, int sms, int count)
{
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end())
            return it->second;
    }
    BatchArgs t = a;
    t.steps = std::min(a.steps, 64);
    t.eval_every = 0;
    BatchChoice best;
    best.ctas = std::min(count, sms);
    float best_ms = -1.f;
    for (int split = 1; split >= 0; --split)
        for (int ctas : batch_cta_candidates(sms, count)) {
            t.allow_split = split;
            const float ms = time_batch(st, d_insts, t, ctas);
            if (ms > 0.f && (best_ms < 0.f || ms < best_ms)) {
                best_ms = ms;
                best.ctas = ctas;
                best.split = split;
            }
        }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    return best;
}

}  // namespace

extern "C" {

int hsb_version(void) { return HSB_API_VERSION; }

const char *hsb_last_error(void) { return g_last_error; }

hsb_status hsb_params_default(hsb_params *p)
{
    if (!p)
        return set_error(HSB_E_INVAL, "params is NULL");
    memset(p, 0, sizeof *p);
    p->form = HSB_DISCRETE;
    p->prec = HSB_PREC_AUTO;
    p->a0 = 1.0;
    p->c1 = 0.7;
    p->c0 = 0.0;
    p->dt = 1.1;
    p->gamma = 0.06;
    p->init_half_width = 1.0;
    p->eval_every = 100;
    p->trace_every = 0;
    p->instance = 0;
    p->thermostat = HSB_HEAT_CONSTANT;
    p->nh_T = 0.0;
    p->nh_M = 1.0;
    p->nh_xi0 = 0.0;
    return HSB_OK;
}

hsb_status hsb_create(const float *J, int N, hsb_handle *out)
{
    if (!out)
        return set_error(HSB_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!J)
        return set_error(HSB_E_INVAL, "J is NULL");
    if (N < 2 || N > (1 << 20))
        return set_error(HSB_E_INVAL, "N must be in [2, 2^20] (got %d)", N);
    int pm1 = 1;
    double sum2 = 0.0, sumJ = 0.0;
    double maxabs = 1.0;
    hsb_status vs = validate_couplings(J, N, &pm1, &sum2, &sumJ, &maxabs);
    if (vs != HSB_OK)
        return vs;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return set_error(HSB_E_NODEVICE, "no CUDA device");
    }
    hsb_ctx *h = new hsb_ctx();
    cudaGetDevice(&h->device);
    h->N = N;
    h->Np = round_up(N, kTileM);
    h->Kp = round_up(h->Np, 256);
    h->pm1 = pm1;
    h->sigma = sqrt(sum2 / ((double)N * (double)(N - 1)));
    h->jscale = energy_scale_exp(maxabs);
    h->sumJ = sumJ;
    hsb_status s = HSB_OK;
    do {
        cudaError_t e = cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            s = cuda_error(e, "stream create");
            break;
        }
        h->work = h->own;
        e = dev_alloc(&h->err, sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemsetAsync(h->err, 0, sizeof(int), h->work);
        if (e != cudaSuccess) {
            s = cuda_error(e, "cudaMalloc err");
            break;
        }
        const size_t np = (size_t)h->Np;
        e = dev_alloc(&h->J32, np * np * sizeof(float));
        if (e != cudaSuccess) {
            s = cuda_error(e, "cudaMalloc J");
            break;
        }
        e = cudaMemsetAsync(h->J32, 0, np * np * sizeof(float), h->work);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(h->J32, np * sizeof(float), J, (size_t)N * sizeof(float),
                                  (size_t)N * sizeof(float), (size_t)N, cudaMemcpyHostToDevice,
                                  h->work);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(h->work);
        if (e != cudaSuccess) {
            s = cuda_error(e, "copy J");
            break;
        }
    } while (0);
    if (s != HSB_OK) {
        hsb_destroy(h);
        return s;
    }
    *out = h;
    return HSB_OK;
}

void hsb_destroy(hsb_handle h)
{
    if (!h)
        return;
    DeviceGuard g(h->device);
    if (h->work)
        cudaStreamSynchronize(h->work);
    free_run_buffers(h);
    cudaFree(h->J32);
    cudaFree(h->J8);
    cudaFree(h->J4);
    cudaFree(h->Jcat);
    cudaFree(h->trace);
    cudaFree(h->err);
    cudaFree(h->trE);
    cudaFree(h->trT);
    cudaFree(h->tr_scratch);
    cudaFree(h->tr_tickets);
    cudaFree(h->nhpart);
    cudaFree(h->flags);
    cudaFree(h->pk_dev);
    cudaFree(h->Eeval);
    cudaFree(h->Snap);
    if (h->own)
        cudaStreamDestroy(h->own);
    delete h;
}

hsb_status hsb_set_stream(hsb_handle h, void *cuda_stream)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    const cudaStream_t next = cuda_stream ? (cudaStream_t)cuda_stream : h->own;
    if (next == h->work)
        return HSB_OK;
    DeviceGuard g(h->device);
    if (!g.ok)
        return set_error(HSB_E_NODEVICE, "cannot select the handle's device");
    // Work already queued on the old stream uses the handle's buffers: the new
    // stream waits for it (without blocking the host).  The event may be
    // destroyed at once; the wait holds and its resources go when it completes.
    // While either stream is being captured into a graph, an event between
    // them would fail (the new stream) or pull the new stream into the capture
    // (the old one); the caller that captures orders the two streams itself.
    cudaStreamCaptureStatus cap_new = cudaStreamCaptureStatusNone;
    cudaStreamCaptureStatus cap_old = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(next, &cap_new), "stream capture status");
    CK(cudaStreamIsCapturing(h->work, &cap_old), "stream capture status");
    if (cap_new != cudaStreamCaptureStatusNone || cap_old != cudaStreamCaptureStatusNone) {
        h->work = next;
        return HSB_OK;
    }
    cudaEvent_t ev = nullptr;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event create");
    cudaError_t e = cudaEventRecord(ev, h->work);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(next, ev, 0);
    cudaEventDestroy(ev);
    CK(e, "order the new stream after the old one");
    h->work = next;
    return HSB_OK;
}

hsb_status hsb_info(hsb_handle h, int *N, int *is_pm1)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    if (N)
        *N = h->N;
    if (is_pm1)
        *is_pm1 = h->pm1;
    return HSB_OK;
}

hsb_status hsb_cut_values(hsb_handle h, int R, const double *best_energy, double *cut)
{
    if (!h || !best_energy || !cut)
        return set_error(HSB_E_INVAL, "hsb_cut_values: null argument");
    if (R < 1)
        return set_error(HSB_E_INVAL, "R must be >= 1 (got %d)", R);
    // Eq. (eq_Cut) with w_ij = -J_ij: C = -E/2 - (1/4) sum_ij J_ij
    for (int r = 0; r < R; ++r)
        cut[r] = -0.5 * best_energy[r] - 0.25 * h->sumJ;
    return HSB_OK;
}

hsb_status hsb_run_device(hsb_handle h, const hsb_params *p, int R, int steps, uint64_t seed,
                          int8_t *best_spins, double *best_energy)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    if (!best_spins || !best_energy)
        return set_error(HSB_E_INVAL, "output pointer is NULL");
    DeviceGuard g(h->device);
    if (!g.ok)
        return set_error(HSB_E_NODEVICE, "cannot select the handle's device");
    RunCfg c;
    hsb_status s = resolve(h, p, R, steps, &c);
    if (s != HSB_OK)
        return s;
    s = enqueue_run(h, c, seed, p);
    if (s != HSB_OK)
        return s;
    CK(cudaMemcpyAsync(best_spins, h->Sbest, (size_t)R * h->N, cudaMemcpyDeviceToDevice, h->work),
       "copy spins");
    CK(cudaMemcpyAsync(best_energy, h->pm1 ? h->Ebest : h->Efinal, (size_t)R * sizeof(double),
                       cudaMemcpyDeviceToDevice, h->work),
       "copy energies");
    return HSB_OK;
}

hsb_status hsb_run(hsb_handle h, const hsb_params *p, int R, int steps, uint64_t seed,
                   int8_t *best_spins, double *best_energy)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    if (!best_spins || !best_energy)
        return set_error(HSB_E_INVAL, "output pointer is NULL");
    DeviceGuard g(h->device);
    if (!g.ok)
        return set_error(HSB_E_NODEVICE, "cannot select the handle's device");
    RunCfg c;
    hsb_status s = resolve(h, p, R, steps, &c);
    if (s != HSB_OK)
        return s;
    s = enqueue_run(h, c, seed, p);
    if (s != HSB_OK)
        return s;
    CK(cudaMemcpyAsync(best_spins, h->Sbest, (size_t)R * h->N, cudaMemcpyDeviceToHost, h->work),
       "copy spins");
    CK(cudaMemcpyAsync(best_energy, h->pm1 ? h->Ebest : h->Efinal, (size_t)R * sizeof(double),
                       cudaMemcpyDeviceToHost, h->work),
       "copy energies");
    return check_device_error(h);
}

hsb_status hsb_get_state(hsb_handle h, float *x, float *y)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    if (!h->have_state)
        return set_error(HSB_E_INVAL, "no run on this handle yet");
    DeviceGuard g(h->device);
    const size_t row = (size_t)h->N * sizeof(float);
    const size_t pitch = (size_t)h->Np * sizeof(float);
    if (x)
        CK(cudaMemcpy2DAsync(x, row, h->X[h->last_x], pitch, row, (size_t)h->last_R,
                             cudaMemcpyDeviceToHost, h->work),
           "copy x");
    if (y)
        CK(cudaMemcpy2DAsync(y, row, h->Y, pitch, row, (size_t)h->last_R, cudaMemcpyDeviceToHost,
                             h->work),
           "copy y");
    CK(cudaStreamSynchronize(h->work), "synchronize");
    return HSB_OK;
}

hsb_status hsb_advance(hsb_handle h, const hsb_params *p, int R, int steps, int k_begin,
                       int k_end, float *x, float *y)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    if (!x || !y)
        return set_error(HSB_E_INVAL, "state pointer is NULL");
    if (p && p->thermostat == HSB_HEAT_NOSE_HOOVER)
        return set_error(HSB_E_UNSUPPORTED, "hsb_advance keeps no Nose-Hoover xi");
    if (k_begin < 0 || k_end < k_begin || k_end > steps)
        return set_error(HSB_E_INVAL, "need 0 <= k_begin <= k_end <= steps");
    DeviceGuard g(h->device);
    if (!g.ok)
        return set_error(HSB_E_NODEVICE, "cannot select the handle's device");
    RunCfg c;
    hsb_status s = resolve(h, p, R, steps, &c);
    if (s != HSB_OK)
        return s;
    s = prepare(h, c);
    if (s != HSB_OK)
        return s;
    const size_t row = (size_t)h->N * sizeof(float);
    const size_t pitch = (size_t)h->Np * sizeof(float);
    const size_t elems = (size_t)c.Rp * h->Np;
    // FP32 path: step k reads X[k & 1]; FP8 path: X[0] in place, S8[k & 1].
    const int xin = c.prec == HSB_PREC_FP32 ? (k_begin & 1) : 0;
    CK(cudaMemsetAsync(h->X[xin], 0, elems * sizeof(float), h->work), "memset x");
    CK(cudaMemsetAsync(h->Y, 0, elems * sizeof(float), h->work), "memset y");
    CK(cudaMemcpy2DAsync(h->X[xin], pitch, x, row, row, (size_t)R, cudaMemcpyHostToDevice,
                         h->work),
       "copy x");
    CK(cudaMemcpy2DAsync(h->Y, pitch, y, row, row, (size_t)R, cudaMemcpyHostToDevice, h->work),
       "copy y");
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->work), "memset err");
    if (c.prec == HSB_PREC_FP8)
        CK(launch_sign_to_fp8(h->work, h->X[0], h->N, h->Np, c.Rp, h->S8[k_begin & 1]),
           "sign kernel");
    if (c.prec == HSB_PREC_FP4)
        CK(launch_sign_to_fp4(h->work, h->X[0], h->N, h->Np, h->Kp, c.Rp, h->S4[k_begin & 1]),
           "fp4 sign kernel");
    if (c.prec == HSB_PREC_BF16X3) {
        CK(launch_split_state(h->work, h->X[0], h->N, h->Np, c.Rp, c.form, h->Xcat[0]),
           "split state");
        if (k_end > k_begin) {
            s = enqueue_bf16(h, c, k_begin, k_end - k_begin, 0);
            if (s != HSB_OK)
                return s;
        }
        CK(cudaMemcpy2DAsync(x, row, h->X[0], pitch, row, (size_t)R, cudaMemcpyDeviceToHost,
                             h->work),
           "copy x back");
        CK(cudaMemcpy2DAsync(y, row, h->Y, pitch, row, (size_t)R, cudaMemcpyDeviceToHost,
                             h->work),
           "copy y back");
        h->have_state = false;
        return check_device_error(h);
    }
    bool persistent = false;
    s = use_persistent(h, c, &persistent);
    if (s != HSB_OK)
        return s;
    if (persistent) {
        if (k_end > k_begin) {
            s = enqueue_persistent(h, c, k_begin, k_end - k_begin, false, k_begin & 1);
            if (s != HSB_OK)
                return s;
        }
    } else {
        for (int k = k_begin; k < k_end; ++k) {
            s = enqueue_step(h, h->work, c, k, k & 1, false);
            if (s != HSB_OK)
                return s;
        }
    }
    const int xout = c.prec == HSB_PREC_FP32 ? (k_end & 1) : 0;
    CK(cudaMemcpy2DAsync(x, row, h->X[xout], pitch, row, (size_t)R, cudaMemcpyDeviceToHost,
                         h->work),
       "copy x back");
    CK(cudaMemcpy2DAsync(y, row, h->Y, pitch, row, (size_t)R, cudaMemcpyDeviceToHost, h->work),
       "copy y back");
    h->have_state = false;
    return check_device_error(h);
}

hsb_status hsb_advance_device(hsb_handle h, const hsb_params *p, int R, int steps, int k_begin,
                              int k_end)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    if (p && p->thermostat == HSB_HEAT_NOSE_HOOVER)
        return set_error(HSB_E_UNSUPPORTED, "hsb_advance_device keeps no Nose-Hoover xi");
    h->have_xi = false;
    if (k_begin < 0 || k_end < k_begin || k_end > steps)
        return set_error(HSB_E_INVAL, "need 0 <= k_begin <= k_end <= steps");
    DeviceGuard g(h->device);
    if (!g.ok)
        return set_error(HSB_E_NODEVICE, "cannot select the handle's device");
    RunCfg c;
    hsb_status s = resolve(h, p, R, steps, &c);
    if (s != HSB_OK)
        return s;
    if (!h->have_state || h->last_R != R || c.Rp > h->Rcap)
        return set_error(HSB_E_INVAL, "no device state of %d replicas on this handle", R);
    s = prepare(h, c);
    if (s != HSB_OK)
        return s;
    const int par = h->state_par;
    if (c.prec == HSB_PREC_BF16X3) {
        if (k_end > k_begin) {
            s = enqueue_bf16(h, c, k_begin, k_end - k_begin, par);
            if (s != HSB_OK)
                return s;
        }
        h->state_par = (par + (k_end - k_begin)) & 1;
        h->launches = k_end > k_begin ? 1 : 0;
        return HSB_OK;
    }
    bool persistent = false;
    s = use_persistent(h, c, &persistent);
    if (s != HSB_OK)
        return s;
    if (persistent) {
        if (k_end > k_begin) {
            s = enqueue_persistent(h, c, k_begin, k_end - k_begin, false, par);
            if (s != HSB_OK)
                return s;
        }
        h->state_par = (par + (k_end - k_begin)) & 1;
        h->launches = k_end > k_begin ? 1 : 0;
        return HSB_OK;
    }
    const GraphKey key = make_key(h, c);
    if (!h->adv_valid || !(h->adv_key == key) || h->adv_k0 != k_begin || h->adv_k1 != k_end ||
        h->adv_par != par) {
        if (h->adv_exec) {
            cudaGraphExecDestroy(h->adv_exec);
            h->adv_exec = nullptr;
        }
        h->adv_valid = false;
        CK(cudaStreamBeginCapture(h->own, cudaStreamCaptureModeThreadLocal), "begin capture");
        for (int k = k_begin; k < k_end && s == HSB_OK; ++k)
            s = enqueue_step(h, h->own, c, k, (par + (k - k_begin)) & 1, false);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->own, &graph);
        if (s != HSB_OK) {
            if (graph)
                cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess)
            return cuda_error(e, "end capture");
        e = cudaGraphInstantiate(&h->adv_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess)
            return cuda_error(e, "graph instantiate");
        h->adv_key = key;
        h->adv_k0 = k_begin;
        h->adv_k1 = k_end;
        h->adv_par = par;
        h->adv_valid = true;
    }
    if (k_end > k_begin)
        CK(cudaGraphLaunch(h->adv_exec, h->work), "graph launch");
    const int n = k_end - k_begin;
    h->state_par = (par + n) & 1;
    if (c.prec == HSB_PREC_FP32)
        h->last_x = h->state_par;
    h->launches = n;
    return HSB_OK;
}

hsb_status hsb_set_couplings(hsb_handle h, const float *J)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    if (!J)
        return set_error(HSB_E_INVAL, "J is NULL");
    const int N = h->N;
    int pm1 = 1;
    double sum2 = 0.0, sumJ = 0.0;
    double maxabs = 1.0;
    hsb_status vs = validate_couplings(J, N, &pm1, &sum2, &sumJ, &maxabs);
    if (vs != HSB_OK)
        return vs;
    DeviceGuard g(h->device);
    if (!g.ok)
        return set_error(HSB_E_NODEVICE, "cannot select the handle's device");
    const size_t np = (size_t)h->Np;
    CK(cudaMemcpy2DAsync(h->J32, np * sizeof(float), J, (size_t)N * sizeof(float),
                         (size_t)N * sizeof(float), (size_t)N, cudaMemcpyHostToDevice, h->work),
       "copy J");
    h->pm1 = pm1;
    h->sigma = sqrt(sum2 / ((double)N * (double)(N - 1)));
    h->jscale = energy_scale_exp(maxabs);
    h->sumJ = sumJ;
    if (h->J8) {
        if (pm1) {
            CK(launch_j_to_fp8(h->work, h->J32, h->Np, h->J8), "j_to_fp8");
        } else {
            if (h->plan) {
                tc_plan_destroy(h->plan);
                h->plan = nullptr;
            }
            cudaFree(h->J8);
            h->J8 = nullptr;
        }
    }
    if (h->J4) {
        if (pm1) {
            CK(launch_j_to_fp4(h->work, h->J32, h->Np, h->Kp, h->J4), "j_to_fp4");
        } else {
            if (h->plan4) {
                tc_plan_destroy(h->plan4);
                h->plan4 = nullptr;
            }
            cudaFree(h->J4);
            h->J4 = nullptr;
        }
    }
    if (h->Jcat)
        CK(launch_split_couplings(h->work, h->J32, h->Np, h->Jcat), "split couplings");
    CK(cudaStreamSynchronize(h->work), "synchronize");
    return HSB_OK;
}

hsb_status hsb_get_trace(hsb_handle h, double *buf, size_t max_entries, size_t *entries)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    const size_t n = h->trace_len < max_entries ? h->trace_len : max_entries;
    if (entries)
        *entries = h->trace_len;
    if (n == 0)
        return HSB_OK;
    if (!buf)
        return set_error(HSB_E_INVAL, "buf is NULL");
    DeviceGuard g(h->device);
    CK(cudaMemcpyAsync(buf, h->trace, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->work),
       "copy trace");
    CK(cudaStreamSynchronize(h->work), "synchronize");
    return HSB_OK;
}

hsb_status hsb_get_xi(hsb_handle h, int R, double *xi)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    if (!xi)
        return set_error(HSB_E_INVAL, "xi is NULL");
    if (!h->have_xi || !h->have_state || R != h->last_R)
        return set_error(HSB_E_INVAL, "the last run had no Nose-Hoover thermostat or %d replicas",
                         R);
    DeviceGuard g(h->device);
    CK(cudaMemcpyAsync(xi, h->xi, (size_t)R * sizeof(double), cudaMemcpyDeviceToHost, h->work),
       "copy xi");
    CK(cudaStreamSynchronize(h->work), "synchronize");
    return HSB_OK;
}

hsb_status hsb_debug_drop_publication(hsb_handle h, int row_block)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    if (row_block < 0 || row_block >= h->Np / kTileM)
        return set_error(HSB_E_INVAL, "row_block must be in [0, %d)", h->Np / kTileM);
    h->debug_drop_mb = row_block;
    return HSB_OK;
}

hsb_status hsb_debug_alloc_cap(size_t bytes)
{
    g_alloc_cap.store(bytes, std::memory_order_relaxed);
    return HSB_OK;
}

hsb_status hsb_run_stats(hsb_handle h, long long *kernel_launches)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    if (kernel_launches)
        *kernel_launches = h->launches;
    return HSB_OK;
}

hsb_status hsb_run_batch(const hsb_handle *hs, int count, const hsb_params *p, int R, int steps,
                         uint64_t seed, int8_t *const *best_spins, double *const *best_energy)
{
    if (!hs || count < 1 || !best_spins || !best_energy)
        return set_error(HSB_E_INVAL, "hsb_run_batch: null argument or count < 1");
    if (!p)
        return set_error(HSB_E_INVAL, "params is NULL");
    for (int b = 0; b < count; ++b) {
        if (!hs[b] || !best_spins[b] || !best_energy[b])
            return set_error(HSB_E_INVAL, "hsb_run_batch: null handle or output %d", b);
        if (hs[b]->device != hs[0]->device)
            return set_error(HSB_E_INVAL, "hsb_run_batch: all handles must share one device");
    }
    // The batched kernel applies to the discrete form with +/-1 couplings in
    // FP8 (AUTO) or FP4; any other case runs the instances one after another.
    const bool fp4 = p->prec == HSB_PREC_FP4;
    bool batched = p->form == HSB_DISCRETE &&
                   (p->prec == HSB_PREC_AUTO || p->prec == HSB_PREC_FP8 || fp4) &&
                   p->trace_every == 0 && p->thermostat == HSB_HEAT_CONSTANT;
    for (int b = 0; b < count && batched; ++b)
        batched = hs[b]->pm1 && batch_shape_ok(hs[b]->Np, R, fp4);
    if (!batched) {
        for (int b = 0; b < count; ++b) {
            hsb_params pb = *p;
            pb.instance = p->instance + (uint32_t)b;
            hsb_status s = hsb_run(hs[b], &pb, R, steps, seed, best_spins[b], best_energy[b]);
            if (s != HSB_OK)
                return s;
        }
        return HSB_OK;
    }
    DeviceGuard g(hs[0]->device);
    if (!g.ok)
        return set_error(HSB_E_NODEVICE, "cannot select the handles' device");
    std::vector<BatchInst> insts((size_t)count);
    RunCfg c0cfg;
    for (int b = 0; b < count; ++b) {
        hsb_ctx *h = hs[b];
        hsb_params pb = *p;
        pb.prec = fp4 ? HSB_PREC_FP4 : HSB_PREC_FP8;
        pb.schedule = 0;
        pb.instance = p->instance + (uint32_t)b;
        RunCfg c;
        hsb_status s = resolve(h, &pb, R, steps, &c);
        if (s != HSB_OK)
            return s;
        s = prepare(h, c);
        if (s != HSB_OK)
            return s;
        if (b == 0)
            c0cfg = c;
        BatchInst &in = insts[(size_t)b];
        memset(&in, 0, sizeof in);
        in.X = h->X[0];
        in.Y = h->Y;
        in.S8a = fp4 ? h->S4[0] : h->S8[0];
        in.S8b = fp4 ? h->S4[1] : h->S8[1];
        in.Ebest = h->Ebest;
        in.Sbest = h->Sbest;
        in.c0 = c.c.c0;
        in.N = h->N;
        in.Np = h->Np;
        in.R = R;
        in.BN = round_up(R, 32);
        in.instance = pb.instance;
        CK(batch_fill_maps(&in, fp4 ? h->J4 : h->J8, in.S8a, in.S8b, h->Np, h->Rcap,
                           fp4 ? h->Kp : 0),
           "batch maps");
    }
    // largest instances first
    std::vector<int> order((size_t)count);
    for (int b = 0; b < count; ++b)
        order[(size_t)b] = b;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return insts[(size_t)x].Np > insts[(size_t)y].Np; });
    std::vector<BatchInst> sorted((size_t)count);
    for (int b = 0; b < count; ++b)
        sorted[(size_t)b] = insts[(size_t)order[(size_t)b]];
    CK(cudaDeviceSynchronize(), "synchronize");  // couplings converted on each handle's stream

    BatchInst *d_insts = nullptr;
    unsigned int *d_queue = nullptr;
    float *d_pk = nullptr;
    cudaStream_t st = hs[0]->work;
    hsb_status status = HSB_OK;
    cudaError_t e = dev_alloc(&d_insts, sizeof(BatchInst) * (size_t)count);
    if (e == cudaSuccess)
        e = dev_alloc(&d_queue, sizeof(unsigned int));
    if (e == cudaSuccess)
        e = dev_alloc(&d_pk, sizeof(float) * (size_t)steps);
    // The set-up is ordered on the stream of the launch: the handles' streams
    // are non-blocking, so they are not ordered after the legacy default
    // stream, and a pageable cudaMemcpy may return before its DMA lands.  The
    // host vectors live until the stream synchronize at the end of the call.
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_insts, sorted.data(), sizeof(BatchInst) * (size_t)count,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_pk, c0cfg.pk.data(), sizeof(float) * (size_t)steps,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_queue, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(hs[0]->err, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        BatchArgs a;
        memset(&a, 0, sizeof a);
        a.count = count;
        a.queue = d_queue;
        a.steps = steps;
        a.eval_every = p->eval_every;
        a.pk = d_pk;
        a.dt = c0cfg.c.dt;
        a.q = c0cfg.c.q;
        a.g = c0cfg.c.g;
        a.nz = -0.0f;
        a.scale = (float)(p->init_half_width / 16777216.0);
        a.seed = seed;
        a.err = hs[0]->err;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, hs[0]->device);
        sms = std::max(sms, 1);
        double bytes = 0.0;
        for (int b = 0; b < count; ++b)
            bytes += (double)insts[(size_t)b].Np * insts[(size_t)b].Np;
        a.fp4 = fp4 ? 1 : 0;
        const BatchTuneKey key{hs[0]->device, count, round_up(R, 32), (int)ceil(log2(bytes)),
                               a.fp4};
        const BatchChoice ch = tune_batch(key, st, d_insts, a, sms, count);
        a.allow_split = ch.split;
        e = cudaMemsetAsync(d_queue, 0, sizeof(unsigned int), st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(hs[0]->err, 0, sizeof(int), st);
        if (e == cudaSuccess)
            e = launch_tc_batch(st, d_insts, a, ch.ctas);
    }
    for (int b = 0; b < count && e == cudaSuccess; ++b) {
        hsb_ctx *h = hs[b];
        e = cudaMemcpyAsync(best_spins[b], h->Sbest, (size_t)R * h->N, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(best_energy[b], h->Ebest, (size_t)R * sizeof(double),
                                cudaMemcpyDeviceToHost, st);
        h->have_state = false;
        h->launches = 1;
    }
    if (e != cudaSuccess)
        status = cuda_error(e, "batched run");
    else
        status = check_device_error(hs[0]);
    cudaStreamSynchronize(st);
    cudaFree(d_insts);
    cudaFree(d_queue);
    cudaFree(d_pk);
    return status;
}

hsb_status hsb_synchronize(hsb_handle h)
{
    if (!h)
        return set_error(HSB_E_INVAL, "handle is NULL");
    DeviceGuard g(h->device);
    return check_device_error(h);
}

}  // extern "C"
