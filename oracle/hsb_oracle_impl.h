/*
 * hsb_oracle_impl.h -- precision-generic body of the CPU oracle.
 * Included twice by hsb_oracle.c with REAL = double and REAL = float.
 * TEST INFRASTRUCTURE ONLY (see hsb_oracle.c for the readings it follows).
 */

/* sgn(x) of Eq. (eq_fd) and of the spin readout s_i = sgn(x_i): +1 for x >= 0
 * (including -0.0), -1 otherwise. */
static REAL SFX(sgn)(REAL x)
{
    return x >= (REAL)0 ? (REAL)1 : (REAL)-1;
}

/* One term of the running force sum.  binary64: acc + J*b with two
 * roundings.  binary32: one fused multiply-add, fmaf(J, b, acc), rounded once
 * (C99 fmaf is correctly rounded); this is the binary32 reading of the sum. */
static REAL SFX(accumulate)(REAL acc, REAL jv, REAL b)
{
    if (sizeof(REAL) == sizeof(float))
        return (REAL)fmaf((float)jv, (float)b, (float)acc);
    {
        REAL t = jv * b;
        return acc + t;
    }
}

/* Force of one replica: f_i = sum_j J_ij b_j with b_j = x_j (Eq. eq_fb) or
 * b_j = sgn(x_j) (Eq. eq_fd), j ascending.  `Jint` (may be NULL) is the int8
 * copy of +/-1/0 couplings; with it the discrete sum is formed exactly in int32. */
static void SFX(force)(const REAL *J, const int8_t *Jint, int N, int form,
                       const REAL *x, REAL *f, int8_t *stmp)
{
    if (form == 1 && Jint) {
        for (int j = 0; j < N; ++j)
            stmp[j] = x[j] >= (REAL)0 ? (int8_t)1 : (int8_t)-1;
        for (int i = 0; i < N; ++i) {
            const int8_t *row = Jint + (size_t)i * N;
            int32_t acc = 0;
            for (int j = 0; j < N; ++j)
                acc += (int32_t)row[j] * (int32_t)stmp[j];
            f[i] = (REAL)acc;
        }
        return;
    }
    for (int i = 0; i < N; ++i) {
        const REAL *row = J + (size_t)i * N;
        REAL acc = (REAL)0;
        for (int j = 0; j < N; ++j) {
            REAL b = form == 1 ? SFX(sgn)(x[j]) : x[j];
            acc = SFX(accumulate)(acc, row[j], b);
        }
        f[i] = acc;
    }
}

/* One spin update from x(t_k), y(t_k) and the force f_i (Methods):
 *   y~  = y + {-(a0 - a(t_k)) x + c0 f} dt          Eq. (eq_SyEuY)
 *   x~  = x + a0 y~ dt                               Eq. (eq_SyEuX)
 *   x'  = g(x~),  y~~ = h(x~, y~)                    Eqs. (eq_WallX, eq_WallY)
 *   y'  = y~~ + gamma y(t_k) dt                      Eq. (eq_EuHeat)
 * in the pinned order with q = a0*dt and g = gamma*dt. */
static void SFX(update)(int N, REAL *x, REAL *y, const REAL *f, REAL c0, REAL pk,
                        REAL dt, REAL q, REAL g)
{
    for (int i = 0; i < N; ++i) {
        REAL x0 = x[i];
        REAL y0 = y[i];
        REAL u = c0 * f[i];
        REAL v = pk * x0;
        REAL w = u - v;
        REAL wd = w * dt;
        REAL yt = y0 + wd;
        REAL qy = q * yt;
        REAL xt = x0 + qy;
        REAL xn, ytt;
        if (xt > (REAL)1) {
            xn = (REAL)1;
            ytt = (REAL)0;
        } else if (xt < (REAL)-1) {
            xn = (REAL)-1;
            ytt = (REAL)0;
        } else {
            xn = xt;
            ytt = yt;
        }
        REAL gy = g * y0;
        x[i] = xn;
        y[i] = ytt + gy;
    }
}

/* S = sum_i y_i^2 of the Nose-Hoover equation (eq_NH), by its definition,
 * for the state of this precision:
 *   binary32 -- every square y_i^2 is exact in binary64 (two 24-bit
 *               significands), the squares are added exactly
 *               (oracle_exact_square_sum_f32) and the total is rounded once
 *               to binary64;
 *   binary64 -- the plain binary64 sum, i ascending, each square and each
 *               addition rounded once. */
double SFX(oracle_kinetic_sum)(const REAL *y, int N)
{
    if (sizeof(REAL) == sizeof(float))
        return oracle_exact_square_sum_f32((const float *)y, N);
    {
        double s = 0.0;
        for (int i = 0; i < N; ++i) {
            const double v = (double)y[i];
            const double sq = v * v;
            s = s + sq;
        }
        return s;
    }
}

/* TEST DOUBLE of the CUDA kernels' kinetic sum (not the paper's quantity):
 * each y_i scaled by 2^24 (exact) and rounded to the nearest integer q_i,
 * ties to even (nearbyint in the default rounding mode); the squares q_i^2
 * (exact in 64 bits for |y_i| < 256) added exactly to a 128-bit unsigned
 * integer; 2^-48 times the total converted once to binary64.  Independent of
 * the order of the terms.  It differs from the plain sum by at most
 * 2^-24 sum_i |y_i| + N 2^-50 before the final rounding.  Runs select it
 * with oracle_params.nh_sum = 1, to check the kernels' trajectories bit for
 * bit; the plain definition above is the oracle proper. */
double SFX(oracle_kinetic_sum_q24)(const REAL *y, int N)
{
    unsigned __int128 acc = 0;
    for (int i = 0; i < N; ++i) {
        const uint64_t q = (uint64_t)fabs(nearbyint((double)y[i] * 0x1p24));
        acc += (unsigned __int128)q * q;
    }
    return (double)acc * 0x1p-48;
}

static REAL *SFX(widen)(const float *J, int N)
{
    REAL *Jr = (REAL *)malloc(sizeof(REAL) * (size_t)N * (size_t)N);
    if (!Jr)
        return NULL;
    for (size_t e = 0; e < (size_t)N * (size_t)N; ++e)
        Jr[e] = (REAL)J[e];
    return Jr;
}

/* One time step for `nrep` replicas, state x, y laid out [nrep][N].  The
 * constants are given already rounded to REAL; p_k = a0 - a(t_k).  f_out
 * (may be NULL) receives the forces [nrep][N]. */
int SFX(oracle_step)(const float *J, int N, int nrep, REAL *x, REAL *y, int form,
                     REAL pk, REAL c0, REAL dt, REAL q, REAL g, REAL *f_out)
{
    if (N < 1 || nrep < 0)
        return -1;
    REAL *Jr = SFX(widen)(J, N);
    REAL *f = (REAL *)malloc(sizeof(REAL) * (size_t)N);
    int8_t *stmp = (int8_t *)malloc((size_t)N);
    if (!Jr || !f || !stmp) {
        free(Jr);
        free(f);
        free(stmp);
        return -2;
    }
    for (int r = 0; r < nrep; ++r) {
        REAL *xr = x + (size_t)r * N;
        REAL *yr = y + (size_t)r * N;
        SFX(force)(Jr, NULL, N, form, xr, f, stmp);
        if (f_out)
            memcpy(f_out + (size_t)r * N, f, sizeof(REAL) * (size_t)N);
        SFX(update)(N, xr, yr, f, c0, pk, dt, q, g);
    }
    free(Jr);
    free(f);
    free(stmp);
    return 0;
}

/* Whole run for the replicas listed in rep_ids (replica r only depends on
 * seed, instance, r and i, so any subset reproduces the full run).
 * Outputs, each [nrep] or [nrep][N]: best_e, best_s (spins at the best
 * evaluation step), x_out / y_out (state after `steps` updates, may be NULL),
 * e_trace (energy at every evaluation step, [nrep][oracle_num_evals], may be
 * NULL), trace_e / trace_t (Ising energy, Eq. (eq_Ising), and instantaneous
 * temperature T_inst = (1/N) sum_i y_i^2, Eq. (eq_TInst), at the traced times
 * t_k, k = m*trace_every < Ns, [nrep][oracle_num_traced]; may be NULL),
 * xi_out (Nose-Hoover xi(t_Ns) per replica, [nrep], may be NULL; xi0 when the
 * heating is constant). */
int SFX(oracle_run)(const float *J, int N, const oracle_params *p, int steps, uint64_t seed,
                    int nrep, const int32_t *rep_ids, int8_t *best_s, double *best_e,
                    REAL *x_out, REAL *y_out, double *e_trace, double *trace_e,
                    double *trace_t, double *xi_out, int nthreads)
{
    if (N < 1 || steps < 1 || nrep < 0 || p->eval_every < 0)
        return -1;
    REAL *Jr = SFX(widen)(J, N);
    REAL *pk = (REAL *)malloc(sizeof(REAL) * (size_t)steps);
    int8_t *Jint = NULL;
    int use_int = p->form == 1 && !p->force_plain_sum && oracle_is_pm1(J, N);
    if (use_int) {
        Jint = (int8_t *)malloc((size_t)N * (size_t)N);
        if (Jint)
            for (size_t e = 0; e < (size_t)N * (size_t)N; ++e)
                Jint[e] = (int8_t)J[e];
    }
    if (!Jr || !pk || (use_int && !Jint)) {
        free(Jr);
        free(pk);
        free(Jint);
        return -2;
    }
    const REAL c0 = (REAL)p->c0;
    const REAL dt = (REAL)p->dt;
    const REAL q = (REAL)(p->a0 * p->dt);
    const REAL g = (REAL)(p->gamma * p->dt);
    /* Nose-Hoover (Eqs. eq_NH1, eq_NH): h = dt/M and N T, binary64 */
    const int nose_hoover = p->thermostat == 1;
    const double nh_h = p->dt / p->nh_M;
    const double nh_NT = (double)N * p->nh_T;
    for (int k = 0; k < steps; ++k)
        pk[k] = (REAL)oracle_pump_factor(p->a0, k, steps);
    const int n_evals = (p->eval_every > 0 ? (steps - 1) / p->eval_every : 0) + 1;
    const int n_traced = oracle_num_traced(steps, p->trace_every);
    int failed = 0;

#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(| : failed)
#else
    (void)nthreads;
#endif
    for (int t = 0; t < nrep; ++t) {
        uint32_t r = (uint32_t)rep_ids[t];
        REAL *x = (REAL *)malloc(sizeof(REAL) * (size_t)N);
        REAL *y = (REAL *)malloc(sizeof(REAL) * (size_t)N);
        REAL *f = (REAL *)malloc(sizeof(REAL) * (size_t)N);
        int8_t *s = (int8_t *)malloc((size_t)N);
        int8_t *stmp = (int8_t *)malloc((size_t)N);
        if (!x || !y || !f || !s || !stmp) {
            failed = 1;
        } else {
            for (int i = 0; i < N; ++i) {
                x[i] = (REAL)oracle_init_value(seed, p->instance, r, (uint32_t)i, 0, p->init_half_width);
                y[i] = (REAL)oracle_init_value(seed, p->instance, r, (uint32_t)i, 1, p->init_half_width);
            }
            double best = INFINITY;
            double xi = p->nh_xi0;
            int ev = 0;
            for (int k = 0; k <= steps; ++k) {
                int is_eval = (k == steps) || (p->eval_every > 0 && k > 0 && k % p->eval_every == 0);
                if (is_eval) {
                    for (int i = 0; i < N; ++i)
                        s[i] = x[i] >= (REAL)0 ? (int8_t)1 : (int8_t)-1;
                    double e = oracle_ising_energy(J, N, s);
                    if (e_trace)
                        e_trace[(size_t)t * n_evals + ev] = e;
                    ++ev;
                    if (e < best) {
                        best = e;
                        memcpy(best_s + (size_t)t * N, s, (size_t)N);
                    }
                }
                if (k == steps)
                    break;
                if (p->trace_every > 0 && k % p->trace_every == 0) {
                    const size_t at = (size_t)t * n_traced + (size_t)(k / p->trace_every);
                    for (int i = 0; i < N; ++i)
                        s[i] = x[i] >= (REAL)0 ? (int8_t)1 : (int8_t)-1;
                    if (trace_e)
                        trace_e[at] = oracle_ising_energy(J, N, s);
                    double t2 = 0.0;
                    for (int i = 0; i < N; ++i)
                        t2 += (double)y[i] * (double)y[i];
                    if (trace_t)
                        trace_t[at] = t2 / (double)N;
                }
                SFX(force)(Jr, Jint, N, p->form, x, f, stmp);
                if (nose_hoover) {
                    /* friction -xi_k y in place of the heating term */
                    const REAL gk = (REAL)(-xi * p->dt);
                    SFX(update)(N, x, y, f, c0, pk[k], dt, q, gk);
                    /* xi_{k+1} from the updated momenta, Eq. (eq_NH) */
                    const double s2 = p->nh_sum == 1 ? SFX(oracle_kinetic_sum_q24)(y, N)
                                                     : SFX(oracle_kinetic_sum)(y, N);
                    xi = xi + nh_h * (s2 - nh_NT);
                } else {
                    SFX(update)(N, x, y, f, c0, pk[k], dt, q, g);
                }
            }
            best_e[t] = best;
            if (xi_out)
                xi_out[t] = xi;
            if (x_out)
                memcpy(x_out + (size_t)t * N, x, sizeof(REAL) * (size_t)N);
            if (y_out)
                memcpy(y_out + (size_t)t * N, y, sizeof(REAL) * (size_t)N);
        }
        free(x);
        free(y);
        free(f);
        free(s);
        free(stmp);
    }
    free(Jr);
    free(pk);
    free(Jint);
    return failed ? -2 : 0;
}
