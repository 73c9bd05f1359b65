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
//               then TMA-loads J and S two K chunks at a time (3-D boxes of
//               128 x 128 x 2 bytes: one 32 KB copy each, which moves data
//               into the SM faster than two 16 KB copies) into a ring of
//               shared-memory stages, in the order the chunk pairs become
//               ready (the FP8 products are exact integers, so the summation
//               order does not change the force);
//   warp 1      allocates 512 tensor-memory columns, issues tcgen05.mma
//               (kind::f8f6f4, M = N = 128, K = 32) from one lane;
//   warps 2-17  epilogue, four warps per 32-lane quadrant (32 replicas each,
//               moved through tensor memory 16 columns at a time):
//               accumulator, x and y from tensor memory, the pinned spin
//               update, x and y back to tensor memory, sgn(x') as FP8 into a shared-memory
//               tile that one TMA store writes to the other operand buffer,
//               then a gpu-scope release of the tile's flag.  On evaluation steps also the per-replica partial sums
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
constexpr int kPChunks = 2;  // K chunks of 128 per stage
constexpr int kPStages = 3;
constexpr int kPStageA = kPChunks * kPM * kPK;
constexpr int kPStageB = kPChunks * kPN * kPK;
constexpr int kPTileS = kPN * kPM;  // FP8 spin tile [replica][spin] for the store
constexpr int kEpiWarps = 16;
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

constexpr size_t kPSmem =
    1024 + (size_t)kPStages * (kPStageA + kPStageB) + kPTileS + sizeof(PShared);
static_assert(kPSmem <= 232448, "shared memory per CTA is limited to 227 KB");

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
                         const __grid_constant__ CUtensorMap tmapB1,
                         const __grid_constant__ CUtensorMap tmapSt0,
                         const __grid_constant__ CUtensorMap tmapSt1, const PersistArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = base;
    uint8_t *sB = base + (size_t)kPStages * kPStageA;
    uint8_t *sS = sB + (size_t)kPStages * kPStageB;
    PShared *sh = reinterpret_cast<PShared *>(sS + kPTileS);

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
        ptx::prefetch_tmap(&tmapSt0);
        ptx::prefetch_tmap(&tmapSt1);
    }
    if (warp == 1)
        ptx::tmem_alloc(&sh->tmem_base, kPTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        // K chunks are fetched in pairs (2p, 2p+1); a chunk past the end reads
        // as zero, so an odd chunk count adds zero products only.
        const int npairs = (nblk + 1) >> 1;
        uint32_t g = 0;
        bool fail = false;
        for (int kl = 0; kl < passes && !fail; ++kl) {
            const CUtensorMap *mapB = ((a.par0 + kl) & 1) ? &tmapB1 : &tmapB0;
            uint32_t pending = nblk >= 32 ? 0xFFFFFFFFu : ((1u << nblk) - 1u);
            uint32_t have = 0;  // chunks seen published, not yet loaded
            const unsigned long long t0 = ptx::globaltimer();
            int idle = 0;
            while (pending) {
                bool ready = false;
                if (lane < nblk && ((pending >> lane) & 1u))
                    ready = ptx::ld_acquire_gpu(&a.flags[flag_index(lane, rb, a.nrb)]) >= kl;
                const uint32_t rmask = __ballot_sync(0xFFFFFFFFu, ready);
                __syncwarp();
                have |= rmask;
                pending &= ~rmask;
                // a pair can be loaded when both of its chunks are published
                uint32_t pmask = 0;
                for (int pp = 0; pp < npairs; ++pp) {
                    const uint32_t need = (2 * pp + 1 < nblk) ? (3u << (2 * pp)) : (1u << (2 * pp));
                    if ((have & need) == need)
                        pmask |= 1u << pp;
                }
                if (pmask) {
                    if (lane == 0) {
                        ptx::fence_proxy_async_global();
                        const int p0 = mb >> 1;
                        for (int t = 0; t < npairs; ++t) {
                            int pp = p0 + t;
                            if (pp >= npairs)
                                pp -= npairs;
                            if (!((pmask >> pp) & 1u))
                                continue;
                            const int s = (int)(g % kPStages);
                            const uint32_t ph = (g / kPStages) & 1u;
                            if (!ptx::mbar_wait(&sh->empty[s], ph ^ 1u, &sh->abort, a.err)) {
                                fail = true;
                                break;
                            }
                            ptx::mbar_expect_tx(&sh->full[s], (uint32_t)(kPStageA + kPStageB));
                            ptx::tma_load_3d(sA + (size_t)s * kPStageA, &tmapA, 0, m0, 2 * pp,
                                             &sh->full[s]);
                            ptx::tma_load_3d(sB + (size_t)s * kPStageB, mapB, 0, r0, 2 * pp,
                                             &sh->full[s]);
                            ++g;
                        }
                    }
                    for (int pp = 0; pp < npairs; ++pp)
                        if ((pmask >> pp) & 1u)
                            have &= ~((2 * pp + 1 < nblk) ? (3u << (2 * pp)) : (1u << (2 * pp)));
                    fail = __shfl_sync(0xFFFFFFFFu, fail, 0);
                    g = __shfl_sync(0xFFFFFFFFu, g, 0);
                    if (fail)
                        break;
                } else {
                    int give_up = 0;
                    if (lane == 0) {
                        // the clock is read every 16th idle poll (a read costs ~0.1 us)
                        if (*(volatile int *)&sh->abort) {
                            give_up = 1;
                        } else if ((++idle & 15) == 0 &&
                                   ptx::globaltimer() - t0 > ptx::kWaitBudgetNs) {
                            *(volatile int *)&sh->abort = 1;
                            atomicExch(a.err, kErrTimeout);
                            give_up = 1;
                        }
                    }
                    if (__shfl_sync(0xFFFFFFFFu, give_up, 0)) {
                        fail = true;
                        break;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            // descriptors of stage 0; a stage or K step further is a plain
            // add on the 14-bit start-address field (addresses < 256 KB)
            const uint64_t adesc0 = ptx::sw128_desc(ptx::smem_u32(sA));
            const uint64_t bdesc0 = ptx::sw128_desc(ptx::smem_u32(sB));
            uint32_t g = 0;
            for (int kl = 0; kl < passes; ++kl) {
                if (kl > 0) {
                    if (!ptx::mbar_wait(&sh->tmem_empty, (uint32_t)(kl - 1) & 1u, &sh->abort,
                                        a.err))
                        break;
                    ptx::tc_fence_after();
                }
                bool ok = true;
                const int npairs = (nblk + 1) >> 1;
                for (int t = 0; t < npairs; ++t) {
                    const int s = (int)(g % kPStages);
                    const uint32_t ph = (g / kPStages) & 1u;
                    if (!ptx::mbar_wait(&sh->full[s], ph, &sh->abort, a.err)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint64_t ad = adesc0 + (uint64_t)((s * kPStageA) >> 4);
                    const uint64_t bd = bdesc0 + (uint64_t)((s * kPStageB) >> 4);
#pragma unroll
                    for (int c = 0; c < kPChunks; ++c) {
#pragma unroll
                        for (int kk = 0; kk < kPK / 32; ++kk)
                            ptx::mma_fp8(tmem + kColAcc,
                                         ad + (uint64_t)((c * kPM * kPK + kk * 32) >> 4),
                                         bd + (uint64_t)((c * kPN * kPK + kk * 32) >> 4), kIdesc,
                                         (t | c | kk) != 0 ? 1u : 0u);
                    }
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
        const int ew = warp - 2;            // 0..15
        const int q = warp & 3;             // tensor-memory lane quadrant
        const int c0 = (ew >> 2) * 32;      // first of this warp's 32 replica columns
        const int et = threadIdx.x - 64;    // 0..511
        const int i = m0 + q * 32 + lane;   // spin of this thread
        const bool live = i < a.N;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const size_t plane = (size_t)a.Rp * a.Np;

        // initial state of the tile into tensor memory
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t xr[16], yr[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const size_t e = (size_t)(r0 + c0 + h * 16 + j) * a.Np + i;
                xr[j] = __float_as_uint(a.X[e]);
                yr[j] = __float_as_uint(a.Y[e]);
            }
            ptx::tmem_st16(tmem + lane_off + kColX + c0 + h * 16, xr);
            ptx::tmem_st16(tmem + lane_off + kColY + c0 + h * 16, yr);
        }
        ptx::tmem_st_wait();

        bool left = false;
        uint8_t *srow = sS + q * 32 + lane;  // this spin's byte in row `col` of the tile
        const StepConsts2 k2 = step_consts2(a.c);
        float pk_next = a.nsteps > 0 ? a.pk[a.k_begin] : 0.f;
        for (int kl = 0; kl < passes; ++kl) {
            const bool final_pass = kl == a.nsteps;
            const int k = a.k_begin + kl;
            int e = -1;
            if (final_pass)
                e = a.n_evals - 1;
            else if (a.eval_every > 0 && k > 0 && k < a.steps_total && k % a.eval_every == 0)
                e = k / a.eval_every - 1;
            const float pk = final_pass ? 0.f : pk_next;
            const uint64_t pk2 = f2_pack(pk, pk);
            if (kl + 1 < a.nsteps)
                pk_next = a.pk[k + 1];  // p_k of the next pass, off the critical path

            // x and y of the first 16 columns: the MMA does not write them
            uint32_t xpre[16], ypre[16];
            ptx::tmem_ld16(tmem + lane_off + kColX + c0, xpre);
            ptx::tmem_ld16(tmem + lane_off + kColY + c0, ypre);
            const bool ok = ptx::mbar_wait(&sh->accfull, (uint32_t)kl & 1u, &sh->abort, a.err);
            ptx::tmem_ld_wait(xpre);
            ptx::tmem_ld_wait(ypre);
            if (epi_bar_or(!ok)) {
                left = true;
                break;
            }
            ptx::tc_fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t col0 = (uint32_t)(c0 + h * 16);
                uint32_t f[16], xr[16], yr[16];
                ptx::tmem_ld16(tmem + lane_off + kColAcc + col0, f);
                if (h == 0) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        xr[j] = xpre[j];
                        yr[j] = ypre[j];
                    }
                } else {
                    ptx::tmem_ld16(tmem + lane_off + kColX + col0, xr);
                    ptx::tmem_ld16(tmem + lane_off + kColY + col0, yr);
                    ptx::tmem_ld_wait(xr);
                    ptx::tmem_ld_wait(yr);
                }
                ptx::tmem_ld_wait(f);
                if (e >= 0) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = col0 + j;
                        const float fj = __uint_as_float(f[j]);
                        const float x0 = __uint_as_float(xr[j]);
                        float term = live ? (x0 >= 0.f ? fj : -fj) : 0.f;
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1)
                            term += __shfl_xor_sync(0xFFFFFFFFu, term, off);
                        if (lane == 0)
                            sh->red[q][col] = term;
                        a.Snap[(size_t)e * plane + (size_t)(r0 + col) * a.Np + i] =
                            live ? fp8_sign(x0) : (uint8_t)0;
                    }
                }
                if (!final_pass) {
                    // two replicas per packed binary32 operation
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        float xn0, xn1;
                        uint64_t yn;
                        sb_update2(f2_pack_bits(f[j], f[j + 1]), f2_pack_bits(xr[j], xr[j + 1]),
                                   f2_pack_bits(yr[j], yr[j + 1]), pk2, k2, xn0, xn1, yn);
                        xr[j] = __float_as_uint(xn0);
                        xr[j + 1] = __float_as_uint(xn1);
                        yr[j] = (uint32_t)yn;
                        yr[j + 1] = (uint32_t)(yn >> 32);
                        srow[(col0 + j) * kPM] = live ? fp8_sign(xn0) : (uint8_t)0;
                        srow[(col0 + j + 1) * kPM] = live ? fp8_sign(xn1) : (uint8_t)0;
                    }
                    ptx::tmem_st16(tmem + lane_off + kColX + col0, xr);
                    ptx::tmem_st16(tmem + lane_off + kColY + col0, yr);
                }
            }
            ptx::tc_fence_before();
            if (!final_pass) {
                ptx::tmem_st_wait();
                ptx::fence_proxy_async_smem();  // tile writes before the TMA store reads them
            }
            epi_bar();
            if (!final_pass && et == 0) {
                // S(t_{k+1}) of this tile: one tile store, then publish the flag
                ptx::tma_store_2d(((a.par0 + kl + 1) & 1) ? &tmapSt1 : &tmapSt0, m0, r0, sS);
                ptx::mbar_arrive(&sh->tmem_empty);  // accumulator read: the next MMA may start
                ptx::bulk_commit();
                ptx::bulk_wait_all();
                ptx::fence_proxy_async_global();
                ptx::st_release_gpu(&a.flags[flag_index(mb, rb, a.nrb)], kl + 1);
            } else if (et == 0) {
                ptx::mbar_arrive(&sh->tmem_empty);
            }
            if (e >= 0 && et < kPN) {
                const float s = sh->red[0][et] + sh->red[1][et] + sh->red[2][et] + sh->red[3][et];
                a.Epart[((size_t)e * nblk + mb) * a.Rp + r0 + et] = s;
            }
        }

        // final state back to global memory
        if (!left) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t xr[16], yr[16];
                ptx::tmem_ld16(tmem + lane_off + kColX + c0 + h * 16, xr);
                ptx::tmem_ld16(tmem + lane_off + kColY + c0 + h * 16, yr);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const size_t eidx = (size_t)(r0 + c0 + h * 16 + j) * a.Np + i;
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
    return cudaLaunchKernelEx(&cfg, tc_fp8_persistent_kernel, plan->mapA3, plan->mapB3[0],
                              plan->mapB3[1], plan->mapSt[0], plan->mapSt[1], a);
}

cudaError_t launch_select_best(cudaStream_t st, const float *Epart, const uint8_t *Snap,
                               int n_evals, int nblk, int N, int Np, int R, int Rp,
                               double *Ebest, int8_t *Sbest)
{
    select_best_kernel<<<R, 256, 0, st>>>(Epart, Snap, n_evals, nblk, N, Np, Rp, Ebest, Sbest);
    return cudaGetLastError();
}

}  // namespace hsb
