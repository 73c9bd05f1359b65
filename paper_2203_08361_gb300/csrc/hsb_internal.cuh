// hsb_internal.cuh -- declarations shared by the translation units of libhsb.
//
// Device layout (all buffers padded; Np = N rounded up to 128, Rp = R rounded
// up to 128; padded spins have zero couplings and zero state):
//   J32  [Np][Np] float32    couplings (final energies, FP32 path)
//   J8   [Np][Np] uint8      FP8 e4m3 couplings (+1 = 0x38, -1 = 0xB8, 0 = 0x00)
//   X[b] [Rp][Np] float32    positions, one replica per row (b = ping/pong
//                            buffer for the FP32 path, which reads x of every
//                            spin while it writes the next step)
//   Y    [Rp][Np] float32    momenta (updated in place by the owning thread)
//   S8[b][Rp][Np] uint8      sgn(x) in FP8, the tensor-core B operand
//   Epart[Np/128][Rp] float  per row-block partial sums of s_i f_i
//   Ebest[R] double, Sbest[R][N] int8   best energy / spins so far
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hsb {

constexpr int kTileM = 128;  // spins per row block
constexpr int kTileR = 128;  // replica padding granule

// Scalar constants of one run, each rounded once from binary64 to binary32
// (c0, dt, q = a0*dt, g = gamma*dt).  p_k is passed per step.
struct StepConsts {
    float c0;
    float dt;
    float q;
    float g;
    float nz;  // -0.0f, set at run time (see sb_update2)
};

// Published-step flags of the persistent kernels: one int per (row block,
// replica block) tile, each on its own 128-byte line, so that the 16 CTAs
// polling one tile's flag do not queue behind the polls of other tiles.
constexpr int kFlagStride = 32;
__host__ __device__ constexpr int flag_index(int mb, int rb, int nrb)
{
    return (mb * nrb + rb) * kFlagStride;
}

// Error word written by kernels whose bounded waits gave up.
enum : int { kErrNone = 0, kErrTimeout = 1, kErrBadLaunch = 2, kErrRange = 3 };

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// ---- hsb_simt.cu -------------------------------------------------------
// Initial state (Results: x_i, y_i uniform in (-L, L)); also the FP8 operand
// S8 = sgn(x0) when s8 != nullptr.  Ebest <- +inf.
cudaError_t launch_init(cudaStream_t st, uint64_t seed, uint32_t instance, float half_width,
                        int N, int Np, int R, int Rp, float *X, float *Y, uint8_t *S8,
                        double *Ebest);

// One plain-FP32 step (force by fused multiply-adds over j ascending, then the
// pinned update).  energy != 0 also writes Epart from s(t_k) and f (discrete
// form only).  energy_only computes Epart for s = sgn(Xcur) without updating.
// Tpart (may be NULL): per row block sums of y_i(t_k)^2 for the trace.
cudaError_t launch_simt_step(cudaStream_t st, int form, bool energy_only, bool energy,
                             const float *J32, int N, int Np, int Rp, const float *Xcur,
                             float *Xnext, float *Y, float pk, StepConsts c, float *Epart,
                             float *Tpart, const float *gvec = nullptr);

// Nose-Hoover thermostat (Eqs. eq_NH1, eq_NH), one variable xi_r per replica
// (binary64) and the friction factor g_r = fl32(-xi_r dt) that replaces the
// constant heating factor gamma dt in the next step (gvec of the step kernels).
// init: xi_r = xi0, g_r = fl32(-xi0 dt) for every r < Rp (padding included).
cudaError_t launch_nh_init(cudaStream_t st, int R, int Rp, double xi0, double dt, double *xi,
                           float *gvec);
// update after a step: S_r = sum_{i<N} y_i^2 (y_i rounded to a multiple of
// 2^-24, squares summed exactly, one rounding to binary64), xi_r += h (S_r -
// NT) with h = dt / M and NT = N T given in binary64, then g_r = fl32(-xi_r
// dt).  A momentum with |y| >= 256 (or not finite) sets *err = kErrRange.
cudaError_t launch_nh_update(cudaStream_t st, const float *Y, int N, int Np, int R, double h,
                             double NT, double dt, double *xi, float *gvec, int *err);

// Trace entry {min_r E_r, mean_r E_r, mean_r T_inst,r} from Epart / Tpart.
// One trace entry {min E, mean E, mean T_inst} into out.  scratch (3 ceil(R / 32)
// doubles) and ticket (one unsigned, zero before the first call; the kernel
// leaves it zero) select the many-block reduction; NULL selects one block.
cudaError_t launch_trace_reduce(cudaStream_t st, const float *Epart, const float *Tpart, int nblk,
                                int N, int R, int Rp, double *scratch, unsigned *ticket,
                                double *out);
// `entries` trace entries at once: entry m reads Epart / Tpart + m nblk Rp,
// uses scratch + m 3 ceil(R / 32) and ticket m (zero before, left zero), and
// writes out[3 m .. 3 m + 2].
cudaError_t launch_trace_reduce_many(cudaStream_t st, const float *Epart, const float *Tpart,
                                     int nblk, int N, int R, int Rp, int entries, double *scratch,
                                     unsigned *tickets, double *out);

// Best tracking after an evaluation: E_r = -1/2 sum_blocks Epart; if E_r <
// Ebest[r] store it with the spins sgn(x) read from X (fp32), S8 (fp8) or the
// packed S4 (fp4, rows of Kp/2 bytes).
cudaError_t launch_best_update(cudaStream_t st, const float *Epart, int nblk, int N, int Np,
                               int R, int Rp, const float *X, const uint8_t *S8,
                               double *Ebest, int8_t *Sbest, const uint8_t *S4 = nullptr,
                               int Kp = 0);

// Energy of the final best spins in binary64 (Eq. (eq_Ising)) for general J.
cudaError_t launch_final_energy_f64(cudaStream_t st, const float *J32, int N, int Np, int R,
                                    const int8_t *Sbest, double *Eout);

// The same energies through partial sums part[16][R] (scratch of
// final_energy_part_doubles(R) 8-byte words) in exact fixed point: every
// J_ij is rounded to a multiple of 2^-scale_exp (scale_exp = 40 - e with
// max |J| < 2^e, so |J_ij| 2^scale_exp < 2^40), the upper-triangle sum
// -sum_{i<j} J_ij s_i s_j is formed exactly in 64-bit integers, and the total
// is rounded once to binary64; it does not depend on the summation order.
// N above about 6300 falls back to launch_final_energy_f64.
size_t final_energy_part_doubles(int R);
cudaError_t launch_final_energy_f64_parts(cudaStream_t st, const float *J32, int N, int Np, int R,
                                          const int8_t *Sbest, int scale_exp, double *part,
                                          double *Eout);

// sgn(X) -> FP8 operand (used when a state is loaded from the host).
cudaError_t launch_sign_to_fp8(cudaStream_t st, const float *X, int N, int Np, int Rp,
                               uint8_t *S8);

// float32 couplings -> FP8 e4m3 (+/-1/0 only).
cudaError_t launch_j_to_fp8(cudaStream_t st, const float *J32, int Np, uint8_t *J8);

// ---- hsb_tc.cu -----------------------------------------------------------
// TMA tensor maps of the FP8 operands: J8 [Np][Np] and the two S8 ping/pong
// buffers [Rcap][Np], 128-byte boxes with the 128-byte swizzle.
struct TcPlan {
    CUtensorMap mapA;      // 2-D J8, box 128 B x 128 rows
    CUtensorMap mapB[2];   // 2-D S8a / S8b, box 128 B x 128 rows
    CUtensorMap mapA3;     // 3-D J8 (128 B, rows, K chunks), box 128 x 128 x 2
    CUtensorMap mapB3[2];  // 3-D S8a / S8b, box 128 x 128 x 2
    CUtensorMap mapBw[2];  // 2-D S8a / S8b, box 128 B x 256 rows (per-step kernel)
    CUtensorMap mapJ64;    // 2-D J8, box 128 B x 64 rows (CTA-pair kernel)
    CUtensorMap mapBq[2];  // 2-D S a / b, box 128 B x BN/2 rows (CTA-pair per-step kernel)
    int Np, Rp;            // Rp: replica capacity the maps were encoded for
    int Kp = 0;            // FP4 plans: row length in e2m1 values (Np rounded up to 256)
};

// tcgen05 FP8 step: F = J8 * S8cur^T on the tensor cores (FP32 accumulation
// in tensor memory), fused update; writes S8next, X and Y in place, and Epart
// on evaluation steps.  Requires Np % 128 == 0 and Rp % 128 == 0.  A
// persistent grid (one CTA per SM) walks 128-spin x 256-replica tiles.
cudaError_t tc_fp8_plan_create(TcPlan **out, const uint8_t *J8, const uint8_t *S8a,
                               const uint8_t *S8b, int Np, int Rp);
void tc_plan_destroy(TcPlan *p);
cudaError_t launch_tc_fp8_step(cudaStream_t st, const TcPlan *plan, int parity, bool energy,
                               bool energy_only, int N, int Rp, float *X, float *Y, float pk,
                               StepConsts c, float *Epart, float *Tpart, uint8_t *S8next,
                               int *err, const float *gvec = nullptr);

// The same step with packed FP4 e2m1 operands (tcgen05 kind::mxf4, unit
// block scales): J4 [Np][Kp/2] and S4 [Rcap][Kp/2] bytes, two values per byte
// (+1 = 0x2, -1 = 0xA, 0 = 0x0, the even index in the low nibble), Kp = Np
// rounded up to 256 with zero padding.  Only mapA (J4, box 128 rows) and
// mapBw[2] (S4, box 192 rows) for the per-step kernel and mapA3 / mapB3[2]
// (3-D, two 128-byte slices, 128 rows) for the persistent kernel are encoded
// in an FP4 plan.
cudaError_t tc_fp4_plan_create(TcPlan **out, const uint8_t *J4, const uint8_t *S4a,
                               const uint8_t *S4b, int Np, int Kp, int Rp);
cudaError_t launch_tc_fp4_step(cudaStream_t st, const TcPlan *plan, int parity, bool energy,
                               bool energy_only, int N, int Rp, float *X, float *Y, float pk,
                               StepConsts c, float *Epart, float *Tpart, uint8_t *S4next,
                               int *err, const float *gvec = nullptr);
// float32 couplings (+/-1/0) -> packed e2m1 J4 [Np][Kp/2]; sgn(X) -> packed
// S4 [Rp][Kp/2] (padded spins and the K padding 0).
cudaError_t launch_j_to_fp4(cudaStream_t st, const float *J32, int Np, int Kp, uint8_t *J4);
cudaError_t launch_sign_to_fp4(cudaStream_t st, const float *X, int N, int Np, int Kp, int Rp,
                               uint8_t *S4);

// ---- hsb_persist.cu --------------------------------------------------------
// Arguments of the persistent FP8 kernel: `nsteps` updates starting at global
// step k_begin of a `steps_total`-step schedule, then (final_pass) one
// energy-only pass.  The operand of the first update is in S8a (par0 = 0) or
// S8b (par0 = 1).  Evaluations e = 0..n_evals-1 write Epart[e][nblk][Rp] and
// the spin snapshot Snap[e][Rp][Np].  flags[nblk][nrb] must be zero at launch.
struct PersistArgs {
    int N, Np, Rp, nblk, nrb;
    int k_begin, nsteps, final_pass, eval_every, steps_total, n_evals, par0;
    const float *pk;
    StepConsts c;
    float *X, *Y;
    uint8_t *S8a, *S8b;
    int *flags;
    float *Epart;
    uint8_t *Snap;
    int *err;
    // Nose-Hoover thermostat (Eqs. eq_NH1, eq_NH; persistent kernel only):
    // nh != 0 selects it; h = dt / M, NT = N T and dt in binary64; xi [Rp]
    // holds xi(t_k_begin) on entry and xi after the last update on exit;
    // nhpart [3][nblk][Rp][2] the exact per-tile sums of q^2 (q = 2^24 y,
    // rounded) as (hi, lo) words; nhflags like flags, tile (mb, rb) stores
    // pass + 1 once its sums of that pass are written.
    int nh;
    double nh_h, nh_NT, dt64;
    double *xi;
    unsigned long long *nhpart;
    int *nhflags;
    // failure-detection test: tile (drop_mb, 0) never publishes its signs, so
    // the bounded waits of the launch expire (-1: off)
    int drop_mb;
    // per-step trace (persistent kernel): at t_k, k = m trace_every < steps,
    // each tile stores its row block's sums of s_i f_i and y_i^2 per replica
    // in trE / trT [m][nblk][Rp] (binary32)
    int trace_every;
    float *trE, *trT;
    // FP4 operands (launch_tc_fp4_persistent): S8a / S8b hold packed e2m1
    // rows of Kp / 2 bytes, Kp = Np rounded up to 256
    int Kp;
};

// Resident-J variant (hsb_persist_ar.cu): N <= 2048, same arguments.
bool tc_resident_fits(int Np, int Rp);
cudaError_t launch_tc_fp8_resident(cudaStream_t st, const TcPlan *plan, const uint8_t *J8,
                                   const PersistArgs &a);

// CTA-pair variant (hsb_pair.cu): F^T = S^T J with each pair of CTAs holding
// 256 replicas x 128 spins; N <= 4096, Rp a multiple of 256, no Nose-Hoover,
// no trace; same arguments otherwise.
bool tc_pair_fits(int Np, int Rp);
cudaError_t launch_tc_fp8_pair(cudaStream_t st, const TcPlan *plan, const PersistArgs &a);

// True when the nblk x nrb grid of the persistent kernel can be co-resident.
bool tc_persistent_fits(int Np, int Rp);
cudaError_t launch_tc_fp8_persistent(cudaStream_t st, const TcPlan *plan, const PersistArgs &a);
// The same step loop with packed e2m1 operands (kind::mxf4, unit block
// scales): the FP4 plan's maps, S8a / S8b pointing at the S4 buffers.
bool tc_fp4_persistent_fits(int Np, int Rp);
cudaError_t launch_tc_fp4_persistent(cudaStream_t st, const TcPlan *plan, const PersistArgs &a);
cudaError_t launch_select_best(cudaStream_t st, const float *Epart, const uint8_t *Snap,
                               int n_evals, int nblk, int N, int Np, int R, int Rp,
                               double *Ebest, int8_t *Sbest);

// ---- hsb_persist_bf16.cu ---------------------------------------------------
// Split-BF16 persistent kernel for general couplings (form 0 ballistic, 1
// discrete).  Jcat: [Np][2 Np] BF16 [J_hi | J_lo]; operand buffers Xcat[b]:
// [Rcap][2 Np] BF16 [x_hi | x_lo] (ballistic) or [sgn x | unused] (discrete).
// The kernel runs a.nsteps updates without evaluation (a.final_pass == 0).
struct Bf16Plan;
cudaError_t bf16_plan_create(Bf16Plan **out, const void *Jcat, const void *Xcat0,
                             const void *Xcat1, int Np, int Rp);
void bf16_plan_destroy(Bf16Plan *p);
cudaError_t launch_split_couplings(cudaStream_t st, const float *J32, int Np, void *Jcat);
cudaError_t launch_split_state(cudaStream_t st, const float *X, int N, int Np, int Rp, int form,
                               void *Xcat);
bool tc_bf16_persistent_fits(int Np, int Rp);
cudaError_t launch_tc_bf16x3_persistent(cudaStream_t st, const Bf16Plan *plan, int form,
                                        const PersistArgs &a);

// ---- hsb_batch.cu -----------------------------------------------------------
// One instance of a batched FP8 run (a device array of these is read by the
// kernel; aligned as its tensor maps require).
struct BatchInst {
    CUtensorMap mapA;     // J8 as (128 B, rows, K chunk), box 128 x 128 x 2
    CUtensorMap mapS[2];  // S8a / S8b as (128 B, rows, chunk), box 128 x BN x Np/128
    float *X, *Y;         // [Rcap][Np] state
    uint8_t *S8a, *S8b;   // [Rcap][Np] FP8 (or [Rcap][Kp/2] packed e2m1) operand ping/pong
    double *Ebest;        // [R]
    int8_t *Sbest;        // [R][N]
    float c0;
    int N, Np, R, BN;     // BN = R rounded up to 32
    int Kp;               // FP4: Np rounded up to 256 (operand rows of Kp / 2 bytes); 0 for FP8
    uint32_t instance;    // random stream of the instance
};

struct BatchArgs {
    int count;             // instances in the queue
    unsigned int *queue;   // next instance to take (zero at launch)
    int steps, eval_every;
    const float *pk;       // [steps] p_k = a0 - a(t_k)
    float dt, q, g;        // binary32 constants shared by the batch
    float nz;              // -0.0f (run-time zero addend of the packed products)
    float scale;           // fl32(L * 2^-24) of the initial distribution
    uint64_t seed;
    int *err;
    int allow_split;       // K may be split over the two MMA warps
    int fp4;               // packed e2m1 operands (kind::mxf4) instead of FP8
};

bool batch_shape_ok(int Np, int R, bool fp4);
// Kp = 0: FP8 J8 and operands [rows][Np]; Kp > 0: packed e2m1 J4 and
// operands [rows][Kp/2].
cudaError_t batch_fill_maps(BatchInst *in, const uint8_t *J, const uint8_t *Sa,
                            const uint8_t *Sb, int Np, int Rcap, int Kp);
cudaError_t launch_tc_batch(cudaStream_t st, const BatchInst *d_insts, const BatchArgs &a,
                            int ctas);

}  // namespace hsb
