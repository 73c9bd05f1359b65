// hsb_persist_ar.cu -- persistent tcgen05 kernel for heated discrete SB with
// couplings in {-1, 0, +1} (FP8) and N <= 2048, with each CTA's row block of
// J resident on chip for the whole run (Kanao & Goto, arXiv 2203.08361:
// force Eq. (eq_fd), Methods update, energy Eq. (eq_Ising)).
//
// Why resident: streaming J and the spin operand S together needs about
// 250 GB/s per SM to keep the MMA busy, beyond what TMA delivers into one SM;
// with J resident only S streams (half the bytes per step).
//
// Placement per CTA (tile = 128 spins x 128 replicas, the whole launch):
//   tensor memory  columns   0-255  J rows of the tile, K chunks 0..7 (FP8,
//                                   4 K elements per 32-bit column, row i in
//                                   lane i): the A operand read from TMEM
//                  columns 256-383  FP32 accumulator
//                  columns 384-511  momenta y
//   shared memory  J rows of the tile, K chunks 8..nblk-1 (up to 128 KB,
//                  128-byte swizzle, loaded once), five 16 KB stages of the
//                  streamed S chunks (one K chunk each, so that five copies
//                  are in flight and the MMA rarely waits for data)
//   registers      positions x (32 per epilogue thread)
// Roles, flags and bounded waits as in hsb_persist.cu: warp 0 polls the
// per-tile published flags and TMA-loads S chunks in the order they are
// ready, recording which chunk each stage holds (the FP8 products are exact
// integers, so order does not matter); warp 1 issues tcgen05.mma with A from
// tensor memory (chunks 0-7) or shared memory (chunks 8-15); warps 2-17 run
// the pinned update and write sgn(x') straight from registers to the other
// operand buffer (32 consecutive spins per store instruction), then one
// thread releases the tile's flag after a barrier and a gpu-scope fence;
// evaluation passes write per-replica partial energies and spin snapshots; a
// final pass evaluates E(t_Ns).
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hsb_device.cuh"
#include "hsb_internal.cuh"
#include "hsb_ptx.cuh"

namespace hsb {

namespace {

constexpr int kRM = 128;
constexpr int kRN = 128;
constexpr int kRTmemChunks = 8;                    // K chunks of J held in tensor memory
constexpr int kRMaxChunks = 16;                    // N <= 2048
constexpr int kRSmemA = (kRMaxChunks - kRTmemChunks) * kRM * 128;  // 128 KB
constexpr int kRStages = 5;
constexpr int kRStageB = kRN * 128;                // one K chunk of S, 16 KB
constexpr int kREpiWarps = 16;
constexpr int kREpiThreads = 32 * kREpiWarps;
constexpr int kRFirstEpi = 4;                      // warps 0-3: poller, 2 issuers, MMA
constexpr int kRThreads = 32 * kRFirstEpi + kREpiThreads;
constexpr int kROrder = 32;                        // ring of chunk ids in load order
constexpr uint32_t kRColA = 0;
constexpr uint32_t kRColAcc = 256;
constexpr uint32_t kRColY = 384;
constexpr uint32_t kRIdesc = ptx::idesc_e4m3_f32(kRM, kRN);

struct __align__(8) RShared {
    uint64_t full[kRStages];
    uint64_t empty[kRStages];
    uint64_t a_full;
    uint64_t accfull;
    uint64_t tmem_empty;
    uint64_t drain;       // arrives once every MMA issued has completed
    int last_use[kRStages];  // last use of each stage a copy was issued for
    uint32_t tmem_base;
    int abort;
    int stage_chunk[kRStages];
    int order[kROrder];   // chunk of load g at order[g % kROrder]
    int avail;            // loads whose chunk is known (monotonic over passes)
    float red[4][kRN];
};

constexpr size_t kRSmem = 1024 + (size_t)kRSmemA + (size_t)kRStages * kRStageB + sizeof(RShared);
static_assert(kRSmem <= 232448, "shared memory per CTA is limited to 227 KB");

__device__ __forceinline__ bool rbar_or(bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(kREpiThreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void rbar() { ptx::named_bar(1, kREpiThreads); }

// tcgen05.mma with the A operand in tensor memory (row i in lane i).
__device__ __forceinline__ void mma_fp8_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc,
                                           uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %3, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %4, p;\n\t}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(accumulate), "r"(kRIdesc)
        : "memory");
}

}  // namespace

__global__ void __launch_bounds__(kRThreads, 1)
tc_fp8_resident_kernel(const __grid_constant__ CUtensorMap tmapA,
                       const __grid_constant__ CUtensorMap tmapB0,
                       const __grid_constant__ CUtensorMap tmapB1, const uint8_t *__restrict__ J8,
                       const PersistArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sAres = base;                               // J chunks 8.. (resident)
    uint8_t *sB = base + kRSmemA;                        // S stages
    RShared *sh = reinterpret_cast<RShared *>(sB + (size_t)kRStages * kRStageB);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int mb = blockIdx.x;
    const int rb = blockIdx.y;
    const int m0 = mb * kRM;
    const int r0 = rb * kRN;
    const int nblk = a.nblk;
    const int ntm = nblk < kRTmemChunks ? nblk : kRTmemChunks;   // chunks in tensor memory
    const int nsm = nblk - ntm;                                  // chunks in shared memory
    const int passes = a.nsteps + a.final_pass;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRStages; ++s) {
            ptx::mbar_init(&sh->full[s], 1);
            ptx::mbar_init(&sh->empty[s], 1);
        }
        ptx::mbar_init(&sh->a_full, 1);
        ptx::mbar_init(&sh->accfull, 1);
        ptx::mbar_init(&sh->tmem_empty, 1);
        ptx::mbar_init(&sh->drain, 1);
        for (int s = 0; s < kRStages; ++s)
            sh->last_use[s] = -1;
        sh->abort = 0;
        sh->avail = 0;
        ptx::mbar_init_fence();
    }
    if (warp == 3)
        ptx::tmem_alloc(&sh->tmem_base, 512);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    // ------------------------------------------------ resident J and state
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmapA);
        ptx::prefetch_tmap(&tmapB0);
        ptx::prefetch_tmap(&tmapB1);
        if (nsm > 0) {
            // chunks ntm .. nblk-1, two per copy (a chunk past the end reads 0)
            const int ncopies = (nsm + 1) >> 1;
            ptx::mbar_expect_tx(&sh->a_full, (uint32_t)(ncopies * 2 * kRM * 128));
            for (int c = 0; c < ncopies; ++c)
                ptx::tma_load_3d(sAres + (size_t)c * 2 * kRM * 128, &tmapA, 0, m0, ntm + 2 * c,
                                 &sh->a_full);
        }
    }
    const int ew = warp - kRFirstEpi;        // epilogue warp 0..15
    const int q = warp & 3;                  // tensor-memory lane quadrant
    const int c0 = (ew >> 2) * 32;           // this warp's 32 replica columns
    const int et = threadIdx.x - 32 * kRFirstEpi;
    const int i = m0 + q * 32 + lane;        // spin of this thread
    const bool live = i < a.N;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    float xs[32];                            // positions of (i, c0 .. c0+31)
    if (warp >= kRFirstEpi) {
        // J row i, K chunk kc = 2 w + h (128 bytes) -> tensor-memory columns
        // [32 kc, 32 kc + 32), w = ew >> 2: 4 K bytes per column in K order
        const int w = ew >> 2;
        const uint4 *src = reinterpret_cast<const uint4 *>(J8 + (size_t)i * a.Np);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kc = 2 * w + h;
            if (kc < ntm) {
                uint32_t cols[32];
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const uint4 u = src[kc * 8 + v];
                    cols[4 * v + 0] = u.x;
                    cols[4 * v + 1] = u.y;
                    cols[4 * v + 2] = u.z;
                    cols[4 * v + 3] = u.w;
                }
                ptx::tmem_st32(tmem + lane_off + kRColA + (uint32_t)(32 * kc), cols);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t yr[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const size_t e = (size_t)(r0 + c0 + h * 16 + j) * a.Np + i;
                xs[h * 16 + j] = a.X[e];
                yr[j] = __float_as_uint(a.Y[e]);
            }
            ptx::tmem_st16(tmem + lane_off + kRColY + c0 + h * 16, yr);
        }
        ptx::tmem_st_wait();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();

    if (warp == 0) {
        // ------------------------------------------------------------ poller
        // Reads the published flags of the pass (one lane per chunk) and
        // appends the chunks in the order they become ready to the order ring.
        int G = 0;
        bool fail = false;
        for (int kl = 0; kl < passes && !fail; ++kl) {
            uint32_t pending = (1u << nblk) - 1u;
            const unsigned long long t0 = ptx::globaltimer();
            while (pending) {
                bool ready = false;
                if (lane < nblk && ((pending >> lane) & 1u))
                    ready = ptx::ld_acquire_gpu(&a.flags[flag_index(lane, rb, a.nrb)]) >= kl;
                const uint32_t rmask = __ballot_sync(0xFFFFFFFFu, ready);
                if (rmask) {
                    if (lane == 0) {
                        // own chunk first, then the following ones cyclically
                        for (int t = 0; t < nblk; ++t) {
                            int kc = mb + t;
                            if (kc >= nblk)
                                kc -= nblk;
                            if ((rmask >> kc) & 1u)
                                sh->order[(G++) % kROrder] = kc;
                        }
                        __threadfence_block();
                        *(volatile int *)&sh->avail = G;
                    }
                    G = __shfl_sync(0xFFFFFFFFu, G, 0);
                    pending &= ~rmask;
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
    } else if (warp <= 2) {
        // ----------------------------------------------------------- issuers
        // Issuer w (1 or 2) takes the loads g with g % 2 == w - 1: it waits
        // until the poller has named the chunk of load g, then for the stage
        // g % kRStages to be free, and TMA-loads the chunk.
        if (lane == 0) {
            const int p = warp - 1;
            bool fail = false;
            for (int kl = 0; kl < passes && !fail; ++kl) {
                const CUtensorMap *mapB = ((a.par0 + kl) & 1) ? &tmapB1 : &tmapB0;
                for (int t = p; t < nblk; t += 2) {
                    const int g = kl * nblk + t;
                    if (*(volatile int *)&sh->avail <= g) {
                        const unsigned long long t0 = ptx::globaltimer();
                        int spins = 0;
                        while (*(volatile int *)&sh->avail <= g) {
                            if (*(volatile int *)&sh->abort) {
                                fail = true;
                                break;
                            }
                            if ((++spins & 63) == 0 && ptx::globaltimer() - t0 > ptx::kWaitBudgetNs) {
                                *(volatile int *)&sh->abort = 1;
                                atomicExch(a.err, kErrTimeout);
                                fail = true;
                                break;
                            }
                            __nanosleep(20);
                        }
                        if (fail)
                            break;
                    }
                    __threadfence_block();
                    const int kc = *(volatile int *)&sh->order[g % kROrder];
                    const int s = g % kRStages;
                    const uint32_t ph = (uint32_t)(g / kRStages) & 1u;
                    if (!ptx::mbar_wait(&sh->empty[s], ph ^ 1u, &sh->abort, a.err)) {
                        fail = true;
                        break;
                    }
                    sh->stage_chunk[s] = kc;
                    ptx::fence_proxy_async_global();
                    atomicMax(&sh->last_use[s], g / kRStages);  // for the drain
                    ptx::mbar_expect_tx(&sh->full[s], (uint32_t)kRStageB);
                    ptx::tma_load_2d(sB + (size_t)s * kRStageB, mapB, kc * 128, r0, &sh->full[s]);
                }
            }
        }
    } else if (warp == 3) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            bool ok = nsm == 0 || ptx::mbar_wait(&sh->a_full, 0u, &sh->abort, a.err);
            ptx::tc_fence_after();
            // descriptors of the first resident chunk and of stage 0; further
            // chunks, stages and K steps are adds on the start-address field
            const uint64_t adesc0 = ptx::sw128_desc(ptx::smem_u32(sAres));
            const uint64_t bdesc0 = ptx::sw128_desc(ptx::smem_u32(sB));
            uint32_t g = 0;
            for (int kl = 0; kl < passes && ok; ++kl) {
                if (kl > 0) {
                    if (!ptx::mbar_wait(&sh->tmem_empty, (uint32_t)(kl - 1) & 1u, &sh->abort,
                                        a.err))
                        break;
                    ptx::tc_fence_after();
                }
                for (int t = 0; t < nblk; ++t) {
                    const int s = (int)(g % kRStages);
                    const uint32_t ph = (g / kRStages) & 1u;
                    if (!ptx::mbar_wait(&sh->full[s], ph, &sh->abort, a.err)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const int kc = *(volatile int *)&sh->stage_chunk[s];
                    const uint64_t bd = bdesc0 + (uint64_t)((s * kRStageB) >> 4);
                    const uint32_t acc0 = t != 0 ? 1u : 0u;
                    if (kc < ntm) {
                        const uint32_t ta = tmem + kRColA + (uint32_t)(kc * 32);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_fp8_ta(tmem + kRColAcc, ta + (uint32_t)(kk * 8),
                                       bd + (uint64_t)(kk * 2), acc0 | (kk != 0 ? 1u : 0u));
                    } else {
                        const uint64_t ad = adesc0 + (uint64_t)(((kc - ntm) * kRM * 128) >> 4);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            ptx::mma_fp8(tmem + kRColAcc, ad + (uint64_t)(kk * 2),
                                         bd + (uint64_t)(kk * 2), kRIdesc,
                                         acc0 | (kk != 0 ? 1u : 0u));
                    }
                    ptx::mma_commit(&sh->empty[s]);
                    ++g;
                }
                if (!ok)
                    break;
                ptx::mma_commit(&sh->accfull);
            }
            ptx::mma_commit(&sh->drain);  // arrives once every MMA issued has completed
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const size_t plane = (size_t)a.Rp * a.Np;
        const StepConsts2 k2 = step_consts2(a.c);
        float pk_next = a.nsteps > 0 ? a.pk[a.k_begin] : 0.f;
        bool left = false;
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
                pk_next = a.pk[k + 1];
            // sgn(x') of (i, r0 + c0 + j) goes to byte j * Np of this pointer
            uint8_t *sdst = (((a.par0 + kl + 1) & 1) ? a.S8b : a.S8a) + (size_t)(r0 + c0) * a.Np + i;

            // momenta of the first 16 columns: the MMA does not write them
            uint32_t ypre[16];
            ptx::tmem_ld16(tmem + lane_off + kRColY + c0, ypre);
            const bool ok = ptx::mbar_wait(&sh->accfull, (uint32_t)kl & 1u, &sh->abort, a.err);
            ptx::tmem_ld_wait(ypre);
            if (rbar_or(!ok)) {
                left = true;
                break;
            }
            ptx::tc_fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t col0 = (uint32_t)(c0 + h * 16);
                uint32_t f[16], yr[16];
                ptx::tmem_ld16(tmem + lane_off + kRColAcc + col0, f);
                if (h == 0) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        yr[j] = ypre[j];
                } else {
                    ptx::tmem_ld16(tmem + lane_off + kRColY + col0, yr);
                    ptx::tmem_ld_wait(yr);
                }
                ptx::tmem_ld_wait(f);
                if (e >= 0) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = col0 + j;
                        const float fj = __uint_as_float(f[j]);
                        const float x0 = xs[h * 16 + j];
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
                        sb_update2(f2_pack_bits(f[j], f[j + 1]),
                                   f2_pack(xs[h * 16 + j], xs[h * 16 + j + 1]),
                                   f2_pack_bits(yr[j], yr[j + 1]), pk2, k2, xn0, xn1, yn);
                        xs[h * 16 + j] = xn0;
                        xs[h * 16 + j + 1] = xn1;
                        yr[j] = (uint32_t)yn;
                        yr[j + 1] = (uint32_t)(yn >> 32);
                        sdst[(size_t)(h * 16 + j) * a.Np] = live ? fp8_sign(xn0) : (uint8_t)0;
                        sdst[(size_t)(h * 16 + j + 1) * a.Np] = live ? fp8_sign(xn1) : (uint8_t)0;
                    }
                    ptx::tmem_st16(tmem + lane_off + kRColY + col0, yr);
                }
            }
            ptx::tc_fence_before();
            if (!final_pass)
                ptx::tmem_st_wait();
            rbar();
            if (et == 0)
                ptx::mbar_arrive(&sh->tmem_empty);
            if (!final_pass && et == 0) {
                // every epilogue thread's S stores precede the barrier; the
                // gpu-scope release (cumulative) publishes them with the flag
                ptx::fence_proxy_async_global();
                ptx::st_release_gpu(&a.flags[flag_index(mb, rb, a.nrb)], kl + 1);
            }
            if (e >= 0 && et < kRN) {
                const float s = sh->red[0][et] + sh->red[1][et] + sh->red[2][et] + sh->red[3][et];
                a.Epart[((size_t)e * nblk + mb) * a.Rp + r0 + et] = s;
            }
        }
        if (!left) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t yr[16];
                ptx::tmem_ld16(tmem + lane_off + kRColY + c0 + h * 16, yr);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const size_t eidx = (size_t)(r0 + c0 + h * 16 + j) * a.Np + i;
                    a.X[eidx] = xs[h * 16 + j];
                    a.Y[eidx] = __uint_as_float(yr[j]);
                }
            }
        }
    }

    // drain before tensor memory and shared memory are given up (every exit
    // path): the resident chunks and the last copy into each stage have
    // landed and every MMA has completed, each wait bounded
    __syncthreads();
    if (threadIdx.x < kRStages) {
        const int u = sh->last_use[threadIdx.x];
        if (u >= 0)
            ptx::mbar_drain(&sh->full[threadIdx.x], (uint32_t)u & 1u, a.err);
    }
    if (threadIdx.x == 32 && nsm > 0)
        ptx::mbar_drain(&sh->a_full, 0u, a.err);
    if (threadIdx.x == 96)
        ptx::mbar_drain(&sh->drain, 0u, a.err);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 3)
        ptx::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------- host side ---

bool tc_resident_fits(int Np, int Rp)
{
    const int nblk = Np / kRM, nrb = Rp / kRN;
    if (nblk < 1 || nblk > kRMaxChunks || nrb < 1)
        return false;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    if (cudaFuncSetAttribute(tc_fp8_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kRSmem) != cudaSuccess)
        return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_fp8_resident_kernel, kRThreads,
                                                      kRSmem) != cudaSuccess)
        return false;
    return (long long)nblk * nrb <= (long long)per_sm * sms;
}

cudaError_t launch_tc_fp8_resident(cudaStream_t st, const TcPlan *plan, const uint8_t *J8,
                                   const PersistArgs &a)
{
    if (!plan || a.Np != plan->Np || a.Rp > plan->Rp || a.Rp % kRN != 0 || a.nblk > kRMaxChunks)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc_fp8_resident_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRSmem);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nblk, a.nrb, 1);
    cfg.blockDim = dim3(kRThreads, 1, 1);
    cfg.dynamicSmemBytes = kRSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tc_fp8_resident_kernel, plan->mapA3, plan->mapB[0],
                              plan->mapB[1], J8, a);
}

}  // namespace hsb
