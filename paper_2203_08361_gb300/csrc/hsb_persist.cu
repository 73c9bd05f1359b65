// hsb_persist.cu -- persistent tcgen05 kernel running the whole heated
// discrete SB step loop (HdSB, couplings in {-1, 0, +1}) on sm_103a.
//
// Kanao & Goto, arXiv 2203.08361: force Eq. (eq_fd); update Methods Eqs.
// (eq_SyEuY), (eq_SyEuX), (eq_WallX), (eq_WallY), (eq_EuHeat); energy Eq.
// (eq_Ising) evaluated every `eval_every` steps and at the end (K2000 study).
//
// Each CTA owns one tile of 128 spins x 128 replicas for the whole run.  The
// tile's positions x and momenta y stay in tensor memory next to the FP32
// accumulator (columns 0-127 accumulator, 128-255 x, 256-383 y; lane = spin),
// so a step moves only J and the FP8 spin operand S = sgn(x) through L2:
//   warp 0      producer: polls the per-tile "published" flags of the step's
//               operand (one flag per 128-spin chunk, all lanes at once),
//               then TMA-loads J (128 x 128 bytes) and S chunks into a ring of
//               shared-memory stages, in the order the chunks become ready
//               (the FP8 products are exact integers, so the summation order
//               does not change the force);
//   warp 1      allocates 512 tensor-memory columns, issues tcgen05.mma
//               (kind::f8f6f4, M = N = 128, K = 32) from one lane;
//   warps 2-9   epilogue, two warps per 32-lane quadrant (64 replicas each):
//               accumulator, x and y from tensor memory, the pinned spin
//               update, x and y back to tensor memory, sgn(x') as FP8 into the
//               other operand buffer, then a gpu-scope release of the tile's
//               flag.  On evaluation steps also the per-replica partial sums
//               of s_i f_i and a snapshot of s = sgn(x(t_k)).
// A final pass after the last update evaluates E(t_Ns).  The best evaluation
// per replica is chosen afterwards by select_best_kernel.
//
// All CTAs must be co-resident (cooperative launch).  Every wait is bounded:
// mbarrier and flag waits give up after a wall-clock budget, raise the CTA's
// abort flag and the error word; epilogue warps decide to leave through a
// barrier reduction, so they never wait at a named barrier for a warp that
// has left.  Tensor memory is freed on every exit path.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hsb_device.cuh"
#include "hsb_internal.cuh"
#include "hsb_ptx.cuh"

namespace hsb {

namespace {

constexpr int kPM = 128;
constexpr int kPN = 128;
constexpr int kPK = 128;
constexpr int kPStages = 6;
constexpr int kPStageA = kPM * kPK;
constexpr int kPStageB = kPN * kPK;
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kPThreads = 64 + kEpiThreads;
constexpr uint32_t kPTmemCols = 512;
constexpr uint32_t kColAcc = 0;
constexpr uint32_t kColX = 128;
constexpr uint32_t kColY = 256;
constexpr uint32_t kIdesc = ptx::idesc_e4m3_f32(kPM, kPN);

struct __align__(8) PShared {
    uint64_t full[kPStages];
    uint64_t empty[kPStages];
    uint64_t accfull;
    uint64_t tmem_empty;
    uint32_t tmem_base;
    int abort;
    float red[4][kPN];
};

constexpr size_t kPSmem = 1024 + (size_t)kPStages * (kPStageA + kPStageB) + sizeof(PShared);

// Barrier among the epilogue warps that also ORs a predicate over them, so
// that a decision to leave the step loop is the same in every epilogue warp.
__device__ __forceinline__ bool epi_bar_or(bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(kEpiThreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void epi_bar() { ptx::named_bar(1, kEpiThreads); }

}  // namespace

__global__ void __launch_bounds__(kPThreads, 1)
tc_fp8_persistent_kernel(const __grid_constant__ CUtensorMap tmapA,
                         const __grid_constant__ CUtensorMap tmapB0,
                         const __grid_constant__ CUtensorMap tmapB1, const PersistArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = base;
    uint8_t *sB = base + (size_t)kPStages * kPStageA;
    PShared *sh = reinterpret_cast<PShared *>(sB + (size_t)kPStages * kPStageB);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int mb = blockIdx.x;
    const int rb = blockIdx.y;
    const int m0 = mb * kPM;
    const int r0 = rb * kPN;
    const int nblk = a.nblk;
    const int passes = a.nsteps + a.final_pass;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPStages; ++s) {
            ptx::mbar_init(&sh->full[s], 1);
            ptx::mbar_init(&sh->empty[s], 1);
        }
        ptx::mbar_init(&sh->accfull, 1);
        ptx::mbar_init(&sh->tmem_empty, 1);
        sh->abort = 0;
        ptx::mbar_init_fence();
    }
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmapA);
        ptx::prefetch_tmap(&tmapB0);
        ptx::prefetch_tmap(&tmapB1);
    }
    if (warp == 1)
        ptx::tmem_alloc(&sh->tmem_base, kPTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        uint32_t g = 0;
        bool fail = false;
        for (int kl = 0; kl < passes && !fail; ++kl) {
            const CUtensorMap *mapB = ((a.par0 + kl) & 1) ? &tmapB1 : &tmapB0;
            uint32_t pending = nblk >= 32 ? 0xFFFFFFFFu : ((1u << nblk) - 1u);
            const unsigned long long t0 = ptx::globaltimer();
            while (pending) {
                bool ready = false;
                if (lane < nblk && ((pending >> lane) & 1u))
                    ready = ptx::ld_acquire_gpu(&a.flags[lane * a.nrb + rb]) >= kl;
                const uint32_t rmask = __ballot_sync(0xFFFFFFFFu, ready);
                __syncwarp();
                if (rmask) {
                    if (lane == 0) {
                        ptx::fence_proxy_async_global();
                        for (int t = 0; t < nblk; ++t) {
                            int kc = mb + t;
                            if (kc >= nblk)
                                kc -= nblk;
                            if (!((rmask >> kc) & 1u))
                                continue;
                            const int s = (int)(g % kPStages);
                            const uint32_t ph = (g / kPStages) & 1u;
                            if (!ptx::mbar_wait(&sh->empty[s], ph ^ 1u, &sh->abort, a.err)) {
                                fail = true;
                                break;
                            }
                            ptx::mbar_expect_tx(&sh->full[s], (uint32_t)(kPStageA + kPStageB));
                            ptx::tma_load_2d(sA + (size_t)s * kPStageA, &tmapA, kc * kPK, m0,
                                             &sh->full[s]);
                            ptx::tma_load_2d(sB + (size_t)s * kPStageB, mapB, kc * kPK, r0,
                                             &sh->full[s]);
                            ++g;
                        }
                    }
                    pending &= ~rmask;
                    fail = __shfl_sync(0xFFFFFFFFu, fail, 0);
                    g = __shfl_sync(0xFFFFFFFFu, g, 0);
                    if (fail)
                        break;
                } else {
                    int give_up = 0;
                    if (lane == 0) {
                        if (*(volatile int *)&sh->abort) {
                            give_up = 1;
                        } else if (ptx::globaltimer() - t0 > ptx::kWaitBudgetNs) {
                            *(volatile int *)&sh->abort = 1;
                            atomicExch(a.err, kErrTimeout);
                            give_up = 1;
                        }
                    }
                    if (__shfl_sync(0xFFFFFFFFu, give_up, 0)) {
                        fail = true;
                        break;
                    }
                    __nanosleep(32);
                }
            }
        }
    } else if (warp == 1) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            uint32_t g = 0;
            for (int kl = 0; kl < passes; ++kl) {
                if (kl > 0) {
                    if (!ptx::mbar_wait(&sh->tmem_empty, (uint32_t)(kl - 1) & 1u, &sh->abort,
                                        a.err))
                        break;
                    ptx::tc_fence_after();
                }
                bool ok = true;
                for (int t = 0; t < nblk; ++t) {
                    const int s = (int)(g % kPStages);
                    const uint32_t ph = (g / kPStages) & 1u;
                    if (!ptx::mbar_wait(&sh->full[s], ph, &sh->abort, a.err)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t a0 = ptx::smem_u32(sA + (size_t)s * kPStageA);
                    const uint32_t b0 = ptx::smem_u32(sB + (size_t)s * kPStageB);
#pragma unroll
                    for (int kk = 0; kk < kPK / 32; ++kk)
                        ptx::mma_fp8(tmem + kColAcc, ptx::sw128_desc(a0 + kk * 32),
                                     ptx::sw128_desc(b0 + kk * 32), kIdesc,
                                     (t | kk) != 0 ? 1u : 0u);
                    ptx::mma_commit(&sh->empty[s]);
                    ++g;
                }
                if (!ok)
                    break;
                ptx::mma_commit(&sh->accfull);
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - 2;            // 0..7
        const int q = warp & 3;             // tensor-memory lane quadrant
        const int c0 = (ew >> 2) * 64;      // first of this warp's 64 replica columns
        const int et = threadIdx.x - 64;    // 0..255
        const int i = m0 + q * 32 + lane;   // spin of this thread
        const bool live = i < a.N;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const size_t plane = (size_t)a.Rp * a.Np;

        // initial state of the tile into tensor memory
#pragma unroll
        for (int cb = 0; cb < 2; ++cb) {
            uint32_t xr[32], yr[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const size_t e = (size_t)(r0 + c0 + cb * 32 + j) * a.Np + i;
                xr[j] = __float_as_uint(a.X[e]);
                yr[j] = __float_as_uint(a.Y[e]);
            }
            ptx::tmem_st32(tmem + lane_off + kColX + c0 + cb * 32, xr);
            ptx::tmem_st32(tmem + lane_off + kColY + c0 + cb * 32, yr);
        }
        ptx::tmem_st_wait();

        bool left = false;
        for (int kl = 0; kl < passes; ++kl) {
            const bool final_pass = kl == a.nsteps;
            const int k = a.k_begin + kl;
            int e = -1;
            if (final_pass)
                e = a.n_evals - 1;
            else if (a.eval_every > 0 && k > 0 && k < a.steps_total && k % a.eval_every == 0)
                e = k / a.eval_every - 1;

            const bool ok = ptx::mbar_wait(&sh->accfull, (uint32_t)kl & 1u, &sh->abort, a.err);
            if (epi_bar_or(!ok)) {
                left = true;
                break;
            }
            ptx::tc_fence_after();
            uint32_t f[2][32];
            ptx::tmem_ld32(tmem + lane_off + kColAcc + c0, f[0]);
            ptx::tmem_ld32(tmem + lane_off + kColAcc + c0 + 32, f[1]);
            ptx::tmem_ld_wait();
            ptx::tc_fence_before();
            epi_bar();
            if (et == 0)
                ptx::mbar_arrive(&sh->tmem_empty);  // the next step's MMA may overwrite

            const float pk = final_pass ? 0.f : a.pk[k];
            uint8_t *Snext = ((a.par0 + kl + 1) & 1) ? a.S8b : a.S8a;
#pragma unroll
            for (int cb = 0; cb < 2; ++cb) {
                uint32_t xr[32], yr[32];
                ptx::tmem_ld32(tmem + lane_off + kColX + c0 + cb * 32, xr);
                ptx::tmem_ld32(tmem + lane_off + kColY + c0 + cb * 32, yr);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = c0 + cb * 32 + j;
                    const size_t eidx = (size_t)(r0 + col) * a.Np + i;
                    const float fj = __uint_as_float(f[cb][j]);
                    const float x0 = __uint_as_float(xr[j]);
                    const float y0 = __uint_as_float(yr[j]);
                    if (e >= 0) {
                        float term = live ? (x0 >= 0.f ? fj : -fj) : 0.f;
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1)
                            term += __shfl_xor_sync(0xFFFFFFFFu, term, off);
                        if (lane == 0)
                            sh->red[q][col] = term;
                        a.Snap[(size_t)e * plane + eidx] = live ? fp8_sign(x0) : (uint8_t)0;
                    }
                    if (!final_pass) {
                        float xn, yn;
                        sb_update(fj, x0, y0, pk, a.c, xn, yn);
                        xr[j] = __float_as_uint(xn);
                        yr[j] = __float_as_uint(yn);
                        Snext[eidx] = live ? fp8_sign(xn) : (uint8_t)0;
                    }
                }
                if (!final_pass) {
                    ptx::tmem_st32(tmem + lane_off + kColX + c0 + cb * 32, xr);
                    ptx::tmem_st32(tmem + lane_off + kColY + c0 + cb * 32, yr);
                }
            }
            if (!final_pass) {
                ptx::tmem_st_wait();
                ptx::fence_proxy_async_global();
            }
            epi_bar();
            if (!final_pass && et == 0) {
                ptx::fence_acq_rel_gpu();
                ptx::st_release_gpu(&a.flags[mb * a.nrb + rb], kl + 1);
            }
            if (e >= 0 && et < kPN) {
                const float s = sh->red[0][et] + sh->red[1][et] + sh->red[2][et] + sh->red[3][et];
                a.Epart[((size_t)e * nblk + mb) * a.Rp + r0 + et] = s;
            }
        }

        // final state back to global memory
        if (!left) {
#pragma unroll
            for (int cb = 0; cb < 2; ++cb) {
                uint32_t xr[32], yr[32];
                ptx::tmem_ld32(tmem + lane_off + kColX + c0 + cb * 32, xr);
                ptx::tmem_ld32(tmem + lane_off + kColY + c0 + cb * 32, yr);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const size_t eidx = (size_t)(r0 + c0 + cb * 32 + j) * a.Np + i;
                    a.X[eidx] = __uint_as_float(xr[j]);
                    a.Y[eidx] = __uint_as_float(yr[j]);
                }
            }
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1)
        ptx::tmem_dealloc(tmem, kPTmemCols);
}

// Best evaluation of each replica: E_e = -1/2 sum_b Epart[e][b][r] (binary64,
// blocks in order); the first strictly lowest wins; its snapshot is copied.
__global__ void select_best_kernel(const float *__restrict__ Epart,
                                   const uint8_t *__restrict__ Snap, int n_evals, int nblk,
                                   int N, int Np, int Rp, double *__restrict__ Ebest,
                                   int8_t *__restrict__ Sbest)
{
    const int r = blockIdx.x;
    __shared__ int best_e;
    if (threadIdx.x == 0) {
        double best = INFINITY;
        int be = 0;
        for (int e = 0; e < n_evals; ++e) {
            double s = 0.0;
            for (int b = 0; b < nblk; ++b)
                s += (double)Epart[((size_t)e * nblk + b) * Rp + r];
            const double E = -0.5 * s;
            if (E < best) {
                best = E;
                be = e;
            }
        }
        Ebest[r] = best;
        best_e = be;
    }
    __syncthreads();
    const uint8_t *src = Snap + ((size_t)best_e * Rp + r) * Np;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        Sbest[(size_t)r * N + i] = src[i] == kFp8PlusOne ? (int8_t)1 : (int8_t)-1;
}

// ------------------------------------------------------------- host side ---

bool tc_persistent_fits(int Np, int Rp)
{
    const int nblk = Np / kPM;
    const int nrb = Rp / kPN;
    if (nblk < 1 || nblk > 32 || nrb < 1)
        return false;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    if (cudaFuncSetAttribute(tc_fp8_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPSmem) != cudaSuccess)
        return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_fp8_persistent_kernel,
                                                      kPThreads, kPSmem) != cudaSuccess)
        return false;
    return (long long)nblk * nrb <= (long long)per_sm * sms;
}

cudaError_t launch_tc_fp8_persistent(cudaStream_t st, const TcPlan *plan, const PersistArgs &a)
{
    if (!plan || a.Np != plan->Np || a.Rp > plan->Rp || a.Rp % kPN != 0 || a.nblk > 32)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc_fp8_persistent_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kPSmem);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nblk, a.nrb, 1);
    cfg.blockDim = dim3(kPThreads, 1, 1);
    cfg.dynamicSmemBytes = kPSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tc_fp8_persistent_kernel, plan->mapA, plan->mapB[0],
                              plan->mapB[1], a);
}

cudaError_t launch_select_best(cudaStream_t st, const float *Epart, const uint8_t *Snap,
                               int n_evals, int nblk, int N, int Np, int R, int Rp,
                               double *Ebest, int8_t *Sbest)
{
    select_best_kernel<<<R, 256, 0, st>>>(Epart, Snap, n_evals, nblk, N, Np, Rp, Ebest, Sbest);
    return cudaGetLastError();
}

}  // namespace hsb
