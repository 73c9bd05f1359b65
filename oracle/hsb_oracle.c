/*
 * hsb_oracle.c -- plain, slow CPU oracle for heated simulated bifurcation
 * (Kanao & Goto, "Simulated bifurcation assisted by thermal fluctuation",
 * arXiv 2203.08361).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers.  It shares no code, header, table or
 * constant generator with the CUDA library; both implement the same written
 * reading of the paper.
 *
 * What it computes (every function cites the passage it follows):
 *   - Ising energy, Eq. (eq_Ising), straight from its definition;
 *   - brute-force ground states for tiny N (exhaustive enumeration);
 *   - the heated SB time step of the Methods section: symplectic Euler on the
 *     terms other than gamma*y (Eqs. eq_SyEuY, eq_SyEuX), the perfectly
 *     inelastic walls g and h (Eqs. eq_WallX, eq_WallY) and the Euler heating
 *     step (Eq. eq_EuHeat), with the force of Eq. (eq_fb) (ballistic) or
 *     Eq. (eq_fd) (discrete);
 *   - the whole run: initial x, y uniform (Results, last paragraph of "SB with
 *     thermal fluctuation"), the linear pump a(t) from 0 to a0, best energy
 *     kept over evaluation steps (K2000 study: evaluated every 100 steps,
 *     best kept; 700-spin study: last step only).
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *   - a(t_k) = a0 * k / Ns, so the factor a0 - a(t_k) is p_k = a0 - (a0*k)/Ns,
 *     evaluated in binary64 and rounded once to the working precision.
 *   - sgn(x) = +1 for x >= 0 (including -0.0), -1 otherwise, for both the
 *     discrete force and the spin readout.
 *   - walls compare strictly: |x~| > 1 clamps, |x~| == 1 keeps x~ and y~.
 *   - the heating step uses y(t_k), the momentum before the step.
 *   - operation order of one spin update, each operation rounded separately
 *     (no fused multiply-add; build with -ffp-contract=off):
 *       u = c0*f; v = p_k*x; w = u - v; yt = y + w*dt; xt = x + q*yt;
 *       walls; y' = ytt + g*y(t_k)         with q = a0*dt and g = gamma*dt.
 *   - the force sum runs over j in ascending order; in binary64 each term is
 *     a product and an add, in binary32 each term is one fused multiply-add
 *     (fmaf, a single rounding).  When every coupling is
 *     -1, 0 or +1 and the form is discrete, the sum is a sum of integers of
 *     magnitude < 2^24 and is formed in int32: the result is the exact sum,
 *     identical to the sequential floating-point sum in either precision.
 *   - initial values come from a counter-based SplitMix64 generator
 *     (Steele, Lea & Flood, OOPSLA 2014), see oracle_init_value().
 *   - evaluation steps are t_k for k = m*eval_every (m >= 1, k < Ns) and
 *     k = Ns; eval_every = 0 evaluates the final step only.  A new best needs
 *     a strictly lower energy, so the earliest step wins ties.
 *   - Nose-Hoover SB (Eqs. eq_NH1, eq_NH; the paper gives no discretisation):
 *     the friction term -xi y_i takes the place of the heating term, so step k
 *     uses g_k = -xi_k dt (binary64, rounded once to the working precision)
 *     in the same update; xi is kept per replica in binary64 and advanced
 *     after the momenta, from the updated ones (the ordering of the
 *     symplectic Euler method applied to (y, xi)):
 *       S = sum_i y_i(t_{k+1})^2
 *       xi_{k+1} = xi_k + (dt/M) (S - N T)  (h = dt/M and N T in binary64,
 *                                            each operation rounded once)
 *     S is the plain sum of squares (oracle_kinetic_sum): for binary32
 *     momenta the exact sum of the exact squares, rounded once to binary64
 *     (it does not depend on the order of the terms); for binary64 momenta
 *     the binary64 sum, i ascending.  The CUDA kernels form S from momenta
 *     rounded to multiples of 2^-24; oracle_kinetic_sum_q24 restates that
 *     as a test double (oracle_params.nh_sum = 1) for bit-exact trajectory
 *     checks, and the kernels are compared with the plain definition within
 *     the bound that quantisation implies.
 *
 * Precision: every routine exists twice, in binary64 ("_f64", the reference
 * for tolerance checks) and in binary32 ("_f32", the paper's own single
 * precision, used for bit-exact checks).  Both take the user's float32
 * couplings; the binary64 variant widens them exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- RNG --- */

/* SplitMix64: the state advances by the odd constant GAMMA and each output is
 * the 64-bit finaliser of the new state, so output number n (n >= 1) of the
 * generator started from state s is mix64(s + n*GAMMA). */
#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t oracle_splitmix64(uint64_t state, uint64_t n)
{
    return sm64_mix(state + n * SM64_GAMMA);
}

/* Initial position (comp = 0) or momentum (comp = 1) of spin i of replica r of
 * instance `instance`.  The paper draws x_i, y_i uniformly from (-1, 1); the
 * half width L is a parameter (1 in the paper).
 *   s_inst = output (instance + 1) of SplitMix64(seed)
 *   u      = output (1 + r*2^32 + 2*i + comp) of SplitMix64(s_inst)
 *   m      = top 24 bits of u
 *   value  = fl32( (2m + 1 - 2^24) * fl32(L * 2^-24) )
 * 2m + 1 - 2^24 is an odd integer of magnitude < 2^24 (exact in binary32), so
 * value lies in the open interval (-L, L) and needs one rounding. */
float oracle_init_value(uint64_t seed, uint32_t instance, uint32_t r, uint32_t i,
                        int comp, double half_width)
{
    uint64_t s_inst = oracle_splitmix64(seed, (uint64_t)instance + 1u);
    uint64_t n = 1u + ((uint64_t)r << 32) + 2u * (uint64_t)i + (uint64_t)(comp & 1);
    uint64_t u = oracle_splitmix64(s_inst, n);
    uint32_t m = (uint32_t)(u >> 40);
    float v = (float)(2.0 * (double)m + 1.0 - 16777216.0);
    float scale = (float)(half_width / 16777216.0);
    return v * scale;
}

/* ------------------------------------------------------------- energy --- */

/* Eq. (eq_Ising): E = -1/2 sum_i sum_j J_ij s_i s_j, summed in binary64 over
 * i then j in ascending order. */
double oracle_ising_energy(const float *J, int N, const int8_t *s)
{
    double acc = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            acc += (double)J[(size_t)i * N + j] * (double)s[i] * (double)s[j];
    return -0.5 * acc;
}

/* Eq. (eq_Cut), first line, with w_ij = -J_ij:
 * C = 1/2 sum_i sum_j w_ij (1 - s_i s_j) / 2. */
double oracle_cut_value(const float *J, int N, const int8_t *s)
{
    double acc = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            acc += -(double)J[(size_t)i * N + j] * (1.0 - (double)s[i] * (double)s[j]) / 2.0;
    return 0.5 * acc;
}

/* Exhaustive search over all 2^N spin states (state index b, spin i = +1 when
 * bit i of b is 0).  Returns the minimum energy and the first state (lowest b)
 * that reaches it.  N <= 24. */
int oracle_brute_force(const float *J, int N, double *e_min, int8_t *s_min)
{
    if (N < 1 || N > 24)
        return -1;
    int8_t *s = (int8_t *)malloc((size_t)N);
    if (!s)
        return -2;
    double best = INFINITY;
    for (uint64_t b = 0; b < (1ULL << N); ++b) {
        for (int i = 0; i < N; ++i)
            s[i] = ((b >> i) & 1u) ? -1 : 1;
        double e = oracle_ising_energy(J, N, s);
        if (e < best) {
            best = e;
            memcpy(s_min, s, (size_t)N);
        }
    }
    *e_min = best;
    free(s);
    return 0;
}

/* Scale of the couplings, sigma_J = sqrt(sum_ij J_ij^2 / (N(N-1))), summed in
 * binary64 row by row.  For +/-1 couplings sigma_J = 1 and c0 = c1/sqrt(N) as
 * in the paper; for other couplings the same normalisation generalises the
 * random-matrix argument. */
double oracle_sigma_j(const float *J, int N)
{
    double acc = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double v = (double)J[(size_t)i * N + j];
            acc += v * v;
        }
    return sqrt(acc / ((double)N * (double)(N - 1)));
}

double oracle_c0(const float *J, int N, double c1)
{
    return c1 / (sqrt((double)N) * oracle_sigma_j(J, N));
}

/* p_k = a0 - a(t_k) with a(t_k) = a0*k/Ns, in binary64. */
double oracle_pump_factor(double a0, int k, int steps)
{
    double t = a0 * (double)k;
    t = t / (double)steps;
    return a0 - t;
}

/* Number of evaluation steps of a run: t_k for k = m*eval_every < Ns, and Ns. */
int oracle_num_evals(int steps, int eval_every)
{
    return (eval_every > 0 ? (steps - 1) / eval_every : 0) + 1;
}

/* 1 when every coupling is -1, 0 or +1 (the exact-integer force applies). */
int oracle_is_pm1(const float *J, int N)
{
    for (size_t e = 0; e < (size_t)N * (size_t)N; ++e)
        if (!(J[e] == 1.0f || J[e] == -1.0f || J[e] == 0.0f))
            return 0;
    return 1;
}

/* Exact sum of the squares of binary32 values, rounded once to binary64
 * (round to nearest, ties to even).  A nonzero binary32 value is
 * v = m 2^(e-24) with an integer m < 2^24 (frexpf: |v| = f 2^e, f in
 * [1/2, 1), m = f 2^24 exactly), so v^2 = m^2 2^(2e-48) is an integer
 * multiple of 2^-298, the square of the least binary32 subnormal 2^-149.  The
 * squares are added as integers in units of 2^-298 in a 640-bit accumulator
 * (a finite binary32 value has e <= 128, so one square stays below 2^554 and
 * 2^24 of them below 2^578).  The total X is rounded once: with its top bit
 * at position t, bits t-52 .. t form the significand, bit t-53 is the
 * rounding bit, any lower set bit is sticky, and the result is the rounded
 * significand times 2^(t-52-298) (X itself when it has at most 53 bits). */
#define SQ_LIMBS 10

/* acc += sq 2^sh for sq < 2^48, sh >= 0 */
static void sq_add(uint64_t acc[SQ_LIMBS], uint64_t sq, int sh)
{
    const int limb = sh / 64, bit = sh % 64;
    const uint64_t part[2] = {sq << bit, bit ? sq >> (64 - bit) : 0};
    uint64_t carry = 0;
    for (int l = limb; l < SQ_LIMBS; ++l) {
        const uint64_t a = l - limb < 2 ? part[l - limb] : 0;
        const uint64_t s1 = acc[l] + a;
        const uint64_t c1 = s1 < a ? 1u : 0u;
        const uint64_t s2 = s1 + carry;
        const uint64_t c2 = s2 < carry ? 1u : 0u;
        acc[l] = s2;
        carry = c1 | c2;
        if (l > limb && !carry)
            break;
    }
}

static int sq_bit(const uint64_t acc[SQ_LIMBS], int b)
{
    return (int)((acc[b / 64] >> (b % 64)) & 1u);
}

double oracle_exact_square_sum_f32(const float *y, int N)
{
    uint64_t acc[SQ_LIMBS];
    memset(acc, 0, sizeof acc);
    for (int i = 0; i < N; ++i) {
        const float v = fabsf(y[i]);
        if (v == 0.0f)
            continue;
        int e = 0;
        const float f = frexpf(v, &e);
        const uint64_t m = (uint64_t)ldexpf(f, 24);
        /* v^2 = m^2 2^(2e + 250) units of 2^-298.  For a subnormal v the
         * shift can be negative; m then ends in enough zero bits that the
         * right shift drops zeros only. */
        uint64_t sq = m * m;
        int sh = 2 * e + 250;
        if (sh < 0) {
            sq >>= -sh;
            sh = 0;
        }
        sq_add(acc, sq, sh);
    }
    int t = -1;
    for (int b = 64 * SQ_LIMBS - 1; b >= 0; --b)
        if (sq_bit(acc, b)) {
            t = b;
            break;
        }
    if (t < 0)
        return 0.0;
    uint64_t sig = 0;
    const int low = t >= 52 ? t - 52 : 0;
    for (int b = t; b >= low; --b)
        sig = (sig << 1) | (uint64_t)sq_bit(acc, b);
    if (t <= 52)
        return ldexp((double)sig, -298);  /* exact */
    int expo = t - 52 - 298;
    const int round = sq_bit(acc, t - 53);
    int sticky = 0;
    for (int b = t - 54; b >= 0 && !sticky; --b)
        sticky = sq_bit(acc, b);
    if (round && (sticky || (sig & 1u))) {
        sig += 1;
        if (sig >> 53) {
            sig >>= 1;
            expo += 1;
        }
    }
    return ldexp((double)sig, expo);
}

/* Run parameters of the whole-trajectory driver. */
typedef struct {
    int form;               /* 0: ballistic, Eq. (eq_fb); 1: discrete, Eq. (eq_fd) */
    int eval_every;         /* evaluate every eval_every steps; 0: final step only */
    double a0;              /* a0 (paper: 1) */
    double c0;              /* interaction scale c0 */
    double dt;              /* time step Delta t */
    double gamma;           /* heating rate gamma (0: plain bSB / dSB) */
    double init_half_width; /* x0, y0 uniform in (-L, L) (paper: L = 1) */
    uint32_t instance;      /* RNG stream of the instance */
    int force_plain_sum;    /* 1: never take the int32 force shortcut */
    int trace_every;        /* > 0: record E(t_k) and T_inst(t_k) for k = m*trace_every < Ns */
    int thermostat;         /* 0: constant heating gamma, Eq. (eq_MomHeat);
                               1: Nose-Hoover xi per replica, Eqs. (eq_NH1), (eq_NH) */
    double nh_T;            /* Nose-Hoover temperature T */
    double nh_M;            /* Nose-Hoover mass M */
    double nh_xi0;          /* xi(t_0) */
    int nh_sum;             /* Nose-Hoover S: 0 the plain definition (oracle_kinetic_sum),
                               1 the CUDA kernels' 2^-24 fixed point (test double,
                               oracle_kinetic_sum_q24) */
} oracle_params;

/* Number of traced times of a run: t_k for k = m*trace_every < Ns. */
int oracle_num_traced(int steps, int trace_every)
{
    return trace_every > 0 ? (steps - 1) / trace_every + 1 : 0;
}

/* ----------------------------------------- precision-generic routines --- */

#define REAL double
#define SFX(name) name##_f64
#include "hsb_oracle_impl.h"
#undef REAL
#undef SFX

#define REAL float
#define SFX(name) name##_f32
#include "hsb_oracle_impl.h"
#undef REAL
#undef SFX
