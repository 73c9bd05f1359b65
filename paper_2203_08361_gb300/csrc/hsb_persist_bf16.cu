// hsb_persist_bf16.cu -- persistent tcgen05 kernel for heated SB with general
// (e.g. Gaussian) couplings: the force J x (ballistic, Eq. (eq_fb)) or
// J sgn(x) (discrete, Eq. (eq_fd)) as split-BF16 products with FP32
// accumulation, fused with the Methods update (Kanao & Goto, arXiv 2203.08361).
//
// Split precision: J = J_hi + J_lo and x = x_hi + x_lo with BF16 parts
// (hi = bf16(v), lo = bf16(v - hi); v - hi is exact in binary32).  The force
//     F = J_hi x_hi + J_lo x_hi + J_hi x_lo
// drops only J_lo x_lo and the rounding of the lo parts, about 3 * 2^-18 of
// |J_ij x_j| per term; accumulation is FP32 in tensor memory.  In the discrete
// form the operand sgn(x) is exact in BF16 and F = J_hi s + J_lo s.
//
// Layout: J and the operand are stored as [hi | lo] planes side by side, a
// [rows][2 * Np] BF16 array, so one 3-D TMA box (64 K elements x 128 rows x
// 2 planes, 128-byte swizzle) fetches both planes of a K chunk in one copy.
//
// One 128 x 128 tile per CTA for the whole launch, x and y in tensor memory,
// per-tile published flags and bounded waits, as in hsb_persist.cu.  K chunks
// are consumed in a fixed order per CTA (own row block first, then ascending
// with wrap-around), because BF16 products are not exact and the sum must not
// depend on timing; there is no evaluation inside the kernel (the host splits
// a run at evaluation steps).  Roles:
//   warp 0     J issuer: TMA-loads both planes of each K chunk of J (one
//              3-D box, 32 KB) into a ring of three stages as soon as a stage
//              is free (J does not change, so the first chunks of a step
//              arrive during the previous epilogue) and posts the stage's
//              expected bytes;
//   warp 1     operand issuer: waits for the row block's flag, then loads the
//              same chunks of [x_hi | x_lo] (or sgn x).
//              Copies from one thread complete one after another, so the two
//              boxes of a stage come from two threads; each issuer takes
//              every load in order, so its parity waits see every phase;
//   warps 2-3  MMA (kind::f16, M = N = 128, K = 16), issued from an elected
//              lane of the converged warp.  One warp issues an MMA of this
//              shape about every 90 cycles, slower than the tensor core runs
//              it, so K is split: loads in stage 1 go to warp 3 and a second
//              accumulator, the others to warp 2 (a fixed assignment per
//              step and chunk, so the FP32 sums do not depend on timing);
//   warps 4-19 epilogue, in two phases.  Phase 1 computes x' (the walls are
//              part of it), writes the next operand ([bf16(x') | bf16(x' -
//              hi)], or sgn x') straight from registers and releases the
//              tile's flag; phase 2 repeats the pinned update in full and
//              stores x' and y' in tensor memory while the flags travel.
// An energy-only launch (discrete form, operand sgn x, a.final_pass = 1 and
// no updates) forms the per-row-block partial sums of s_i f_i of every
// replica (Eq. (eq_Ising)), with f = J_hi s + J_lo s, into Epart[nblk][Rp].
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hsb_device.cuh"
#include "hsb_internal.cuh"
#include "hsb_ptx.cuh"

namespace hsb {

namespace {

constexpr int kQM = 128;        // spins per tile
constexpr int kQN = 128;        // replicas per tile
constexpr int kQKE = 64;        // K elements per chunk (128 bytes of BF16)
constexpr int kQStages = 3;
constexpr int kQPlane = kQM * 128;           // one 128 x 128-byte plane, 16 KB
constexpr int kQStageA = 2 * kQPlane;        // hi + lo
constexpr int kQStageB = 2 * kQPlane;        // hi + lo (discrete form uses one plane)
constexpr int kQFirstEpi = 4;
constexpr int kQEpiWarps = 16;
constexpr int kQEpiThreads = 32 * kQEpiWarps;
constexpr int kQThreads = 32 * kQFirstEpi + kQEpiThreads;
constexpr uint32_t kQTmemCols = 512;
constexpr uint32_t kQColAcc0 = 0;
constexpr uint32_t kQColAcc1 = 128;
constexpr uint32_t kQColX = 256;
constexpr uint32_t kQColY = 384;

// Instruction descriptor, kind::f16 with A = B = BF16 (format 1 at bits 7-9
// and 10-12), D = F32 (bits 4-5 = 1), K-major, N >> 3 at 17-22, M >> 4 at 24-28.
constexpr uint32_t kQIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kQN >> 3) << 17) |
                             ((uint32_t)(kQM >> 4) << 24);

struct __align__(8) QShared {
    uint64_t full[kQStages];
    uint64_t empty[kQStages];
    uint64_t accfull;     // one arrival per accumulator
    uint64_t tmem_empty;  // one arrival per epilogue warp
    uint64_t drain;       // one arrival per MMA warp once its MMAs have completed
    int last_use[kQStages];  // last use of each stage a copy was issued for
    uint32_t tmem_base;
    int abort;
    float red[4][kQN];    // per-quadrant energy partials (energy-only pass)
};

constexpr size_t kQSmem = 1024 + (size_t)kQStages * (kQStageA + kQStageB) + sizeof(QShared);
static_assert(kQSmem <= 232448, "shared memory per CTA is limited to 227 KB");

__device__ __forceinline__ void mma_bf16_elect(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                               uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %3, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(accumulate), "r"(kQIdesc)
        : "memory");
}

__device__ __forceinline__ void commit_elect(uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
            ptx::smem_u32(bar))
        : "memory");
}

// Bounded wait by every lane; false in all lanes if any gave up.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, int *abort, int *err)
{
    const bool ok = ptx::mbar_wait<false>(bar, parity, abort, err);
    return __all_sync(0xFFFFFFFFu, ok);
}

__device__ __forceinline__ bool qbar_or(bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(kQEpiThreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void qbar() { ptx::named_bar(1, kQEpiThreads); }

// Force of 16 replica columns: accumulator 0, plus accumulator 1 when K is
// split (its chunks are disjoint from those of accumulator 0).
__device__ __forceinline__ void load_force(uint32_t tcol, bool split, uint32_t (&f)[16])
{
    ptx::tmem_ld16(tcol + kQColAcc0, f);
    if (split) {
#pragma unroll
        for (int p8 = 0; p8 < 2; ++p8) {
            uint32_t f1[8];
            ptx::tmem_ld8(tcol + kQColAcc1 + p8 * 8, f1);
            ptx::tmem_ld_wait(f1);
            ptx::tmem_ld_wait(f);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                f[p8 * 8 + j] = __float_as_uint(
                    __fadd_rn(__uint_as_float(f[p8 * 8 + j]), __uint_as_float(f1[j])));
        }
    }
    ptx::tmem_ld_wait(f);
}

}  // namespace

template <int FORM>
__global__ void __launch_bounds__(kQThreads, 1)
tc_bf16x3_persistent_kernel(const __grid_constant__ CUtensorMap tmapJ,
                            const __grid_constant__ CUtensorMap tmapB0,
                            const __grid_constant__ CUtensorMap tmapB1,
                            __nv_bfloat16 *__restrict__ Xc0, __nv_bfloat16 *__restrict__ Xc1,
                            const PersistArgs a)
{
    constexpr int kBPlanes = FORM == 0 ? 2 : 1;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = base;
    uint8_t *sB = base + (size_t)kQStages * kQStageA;
    QShared *sh = reinterpret_cast<QShared *>(sB + (size_t)kQStages * kQStageB);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int mb = blockIdx.x;
    const int rb = blockIdx.y;
    const int m0 = mb * kQM;
    const int r0 = rb * kQN;
    const int nblk = a.nblk;
    const int nchunks = a.Np / kQKE;  // two per row block
    // a.final_pass: one pass that only evaluates s_i f_i (discrete form,
    // operand sgn x), no update and no publication
    const int passes = a.nsteps + a.final_pass;
    // K is split when a pass has 3 or more loads: every pass then fills all
    // three stages, so both accumulators take part in every pass
    const bool split = nchunks >= 3;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kQStages; ++s) {
            ptx::mbar_init(&sh->full[s], 1);
            ptx::mbar_init(&sh->empty[s], 1);
        }
        ptx::mbar_init(&sh->accfull, 2);
        ptx::mbar_init(&sh->tmem_empty, kQEpiWarps);
        ptx::mbar_init(&sh->drain, 2);
        for (int s = 0; s < kQStages; ++s)
            sh->last_use[s] = -1;
        sh->abort = 0;
        ptx::mbar_init_fence();
    }
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmapJ);
        ptx::prefetch_tmap(&tmapB0);
        ptx::prefetch_tmap(&tmapB1);
    }
    if (warp == 2)
        ptx::tmem_alloc(&sh->tmem_base, kQTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (warp < 2) {
        // --------------------------------------------------------- issuers
        if (lane == 0) {
            const bool isJ = warp == 0;
            uint32_t g = 0;
            bool fail = false;
            for (int kl = 0; kl < passes && !fail; ++kl) {
                const CUtensorMap *mapB = ((a.par0 + kl) & 1) ? &tmapB1 : &tmapB0;
                const unsigned long long t0 = ptx::globaltimer();
                for (int t = 0; t < nblk && !fail; ++t) {
                    int kb = mb + t;  // fixed order: own row block first
                    if (kb >= nblk)
                        kb -= nblk;
                    // the operand rows of block kb change every pass; J does
                    // not, so the J issuer only waits for a free stage and
                    // fetches the first chunks of a pass during the epilogue
                    unsigned n = 0;
                    while (!isJ && ptx::ld_acquire_gpu(&a.flags[flag_index(kb, rb, a.nrb)]) < kl) {
                        if (*(volatile int *)&sh->abort ||
                            ((++n & 15) == 0 && ptx::globaltimer() - t0 > ptx::kWaitBudgetNs)) {
                            *(volatile int *)&sh->abort = 1;
                            atomicExch(a.err, kErrTimeout);
                            fail = true;
                            break;
                        }
                    }
                    if (fail)
                        break;
                    ptx::fence_proxy_async_global();
                    for (int h = 0; h < 2; ++h) {
                        const int c = 2 * kb + h;
                        const int s = (int)(g % kQStages);
                        const uint32_t ph = (g / kQStages) & 1u;
                        if (!ptx::mbar_wait<false>(&sh->empty[s], ph ^ 1u, &sh->abort, a.err)) {
                            fail = true;
                            break;
                        }
                        atomicMax(&sh->last_use[s], (int)(g / kQStages));  // for the drain
                        if (isJ) {
                            ptx::mbar_expect_tx(&sh->full[s],
                                                (uint32_t)(kQStageA + kBPlanes * kQPlane));
                            ptx::tma_load_3d(sA + (size_t)s * kQStageA, &tmapJ, c * kQKE, m0, 0,
                                             &sh->full[s]);
                        } else {
                            ptx::tma_load_3d(sB + (size_t)s * kQStageB, mapB, c * kQKE, r0, 0,
                                             &sh->full[s]);
                        }
                        ++g;
                    }
                }
            }
        }
    } else if (warp < kQFirstEpi) {
        // --------------------------------------------------------------- MMA
        // warp 2 + part issues the loads of its stages (part 1: stage 1)
        const int part = warp - 2;
        const uint32_t dcol = tmem + (part ? kQColAcc1 : kQColAcc0);
        const uint64_t adesc0 = ptx::sw128_desc(ptx::smem_u32(sA));
        const uint64_t bdesc0 = ptx::sw128_desc(ptx::smem_u32(sB));
        for (int kl = 0; kl < passes; ++kl) {
            if (kl > 0) {
                if (!warp_wait(&sh->tmem_empty, (uint32_t)(kl - 1) & 1u, &sh->abort, a.err))
                    break;
                ptx::tc_fence_after();
            }
            bool ok = true;
            int mine = 0;
            for (int t = 0; t < nchunks; ++t) {
                const int g = kl * nchunks + t;
                const int s = g % kQStages;
                if ((split && s == 1) != (part == 1))
                    continue;
                const uint32_t ph = (uint32_t)(g / kQStages) & 1u;
                if (!warp_wait(&sh->full[s], ph, &sh->abort, a.err)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint64_t ahi = adesc0 + (uint64_t)((s * kQStageA) >> 4);
                const uint64_t alo = ahi + (uint64_t)(kQPlane >> 4);
                const uint64_t bhi = bdesc0 + (uint64_t)((s * kQStageB) >> 4);
                const uint64_t blo = bhi + (uint64_t)(kQPlane >> 4);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t off = (uint64_t)((kk * 32) >> 4);
                    mma_bf16_elect(dcol, ahi + off, bhi + off, (mine | kk) != 0 ? 1u : 0u);
                    mma_bf16_elect(dcol, alo + off, bhi + off, 1u);
                    if (FORM == 0)
                        mma_bf16_elect(dcol, ahi + off, blo + off, 1u);
                }
                commit_elect(&sh->empty[s]);
                ++mine;
            }
            if (!ok)
                break;
            if (mine > 0)
                commit_elect(&sh->accfull);
            else if (lane == 0)
                ptx::mbar_arrive(&sh->accfull);  // no load of this pass for this accumulator
        }
        commit_elect(&sh->drain);  // arrives once this warp's MMAs have completed
    } else {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - kQFirstEpi;
        const int q = warp & 3;
        const int c0 = (ew >> 2) * 32;
        const int et = threadIdx.x - 32 * kQFirstEpi;
        const int i = m0 + q * 32 + lane;
        const bool live = i < a.N;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const size_t row2 = 2 * (size_t)a.Np;  // elements per [hi | lo] row

#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t xr[16], yr[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const size_t e = (size_t)(r0 + c0 + h * 16 + j) * a.Np + i;
                xr[j] = __float_as_uint(a.X[e]);
                yr[j] = __float_as_uint(a.Y[e]);
            }
            ptx::tmem_st16(tmem + lane_off + kQColX + c0 + h * 16, xr);
            ptx::tmem_st16(tmem + lane_off + kQColY + c0 + h * 16, yr);
        }
        ptx::tmem_st_wait();

        bool left = false;
        const StepConsts2 k2 = step_consts2(a.c);
        float pk_next = passes > 0 ? a.pk[a.k_begin] : 0.f;
        for (int kl = 0; kl < passes; ++kl) {
            const bool energy_pass = kl == a.nsteps;
            const int k = a.k_begin + kl;
            const float pk = energy_pass ? 0.f : pk_next;
            const uint64_t pk2 = f2_pack(pk, pk);
            if (kl + 1 < a.nsteps)
                pk_next = a.pk[k + 1];
            __nv_bfloat16 *nxt = (((a.par0 + kl + 1) & 1) ? Xc1 : Xc0) + (size_t)(r0 + c0) * row2 + i;

            // x and y of the first 16 columns: the MMA does not write them
            uint32_t xpre[16], ypre[16];
            ptx::tmem_ld16(tmem + lane_off + kQColX + c0, xpre);
            ptx::tmem_ld16(tmem + lane_off + kQColY + c0, ypre);
            const bool ok = ptx::mbar_wait<false>(&sh->accfull, (uint32_t)kl & 1u, &sh->abort, a.err);
            ptx::tmem_ld_wait(xpre);
            ptx::tmem_ld_wait(ypre);
            if (qbar_or(!ok)) {
                left = true;
                break;
            }
            ptx::tc_fence_after();

            // ---- phase 1: x' and the next operand, published first
#pragma unroll
            for (int h = 0; h < 2 && !energy_pass; ++h) {
                const uint32_t col0 = (uint32_t)(c0 + h * 16);
                uint32_t f[16], xr[16], yr[16];
                load_force(tmem + lane_off + col0, split, f);
                if (h == 0) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        xr[j] = xpre[j];
                        yr[j] = ypre[j];
                    }
                } else {
                    ptx::tmem_ld16(tmem + lane_off + kQColX + col0, xr);
                    ptx::tmem_ld16(tmem + lane_off + kQColY + col0, yr);
                    ptx::tmem_ld_wait(xr);
                    ptx::tmem_ld_wait(yr);
                }
#pragma unroll
                for (int j = 0; j < 16; j += 2) {
                    const uint64_t xt =
                        sb_position2(f2_pack_bits(f[j], f[j + 1]), f2_pack_bits(xr[j], xr[j + 1]),
                                     f2_pack_bits(yr[j], yr[j + 1]), pk2, k2);
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        // walls as in sb_update2: x' = clamp(x~, -1, 1)
                        const float xn = fminf(fmaxf(u ? f2_hi(xt) : f2_lo(xt), -1.f), 1.f);
                        __nv_bfloat16 *dst = nxt + (size_t)(h * 16 + j + u) * row2;
                        if (FORM == 0) {
                            // x' = hi + lo, hi = bf16(x'), lo = bf16(x' - hi)
                            const __nv_bfloat16 hi = __float2bfloat16_rn(xn);
                            const __nv_bfloat16 lo =
                                __float2bfloat16_rn(__fsub_rn(xn, __bfloat162float(hi)));
                            dst[0] = live ? hi : __float2bfloat16_rn(0.f);
                            dst[a.Np] = live ? lo : __float2bfloat16_rn(0.f);
                        } else {
                            dst[0] = __float2bfloat16_rn(live ? (xn >= 0.f ? 1.f : -1.f) : 0.f);
                        }
                    }
                }
            }
            if (!energy_pass)
                qbar();
            if (et == 0 && !energy_pass) {
                // every epilogue thread's operand stores precede the barrier;
                // the gpu-scope release (cumulative) publishes them
                ptx::fence_proxy_async_global();
                ptx::st_release_gpu(&a.flags[flag_index(mb, rb, a.nrb)], kl + 1);
            }

            // ---- phase 2: the full update into tensor memory
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t col0 = (uint32_t)(c0 + h * 16);
                uint32_t f[16], xr[16], yr[16];
                ptx::tmem_ld16(tmem + lane_off + kQColX + col0, xr);
                ptx::tmem_ld16(tmem + lane_off + kQColY + col0, yr);
                load_force(tmem + lane_off + col0, split, f);
                ptx::tmem_ld_wait(xr);
                ptx::tmem_ld_wait(yr);
                if (energy_pass) {
                    // s_i f_i summed over the tile's 32 spins of this quadrant
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float fj = __uint_as_float(f[j]);
                        float term = live ? (__uint_as_float(xr[j]) >= 0.f ? fj : -fj) : 0.f;
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1)
                            term += __shfl_xor_sync(0xFFFFFFFFu, term, off);
                        if (lane == 0)
                            sh->red[q][col0 + j] = term;
                    }
                    continue;
                }
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
                }
                ptx::tmem_st16(tmem + lane_off + kQColX + col0, xr);
                ptx::tmem_st16(tmem + lane_off + kQColY + col0, yr);
            }
            ptx::tc_fence_before();
            ptx::tmem_st_wait();
            __syncwarp();
            if (lane == 0)
                ptx::mbar_arrive(&sh->tmem_empty);  // this warp has read the accumulators
            if (energy_pass) {
                qbar();
                if (et < kQN)
                    a.Epart[(size_t)mb * a.Rp + r0 + et] =
                        sh->red[0][et] + sh->red[1][et] + sh->red[2][et] + sh->red[3][et];
            }
        }
        if (!left && a.nsteps > 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t xr[16], yr[16];
                ptx::tmem_ld16(tmem + lane_off + kQColX + c0 + h * 16, xr);
                ptx::tmem_ld16(tmem + lane_off + kQColY + c0 + h * 16, yr);
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

    // drain before tensor memory and shared memory are given up (every exit
    // path): the last copy into each stage has landed and every MMA has
    // completed, each wait bounded.  A stage whose last use was never armed
    // (the J issuer gave up first) waits out the bound, with the error word set.
    __syncthreads();
    if (threadIdx.x < kQStages) {
        const int u = sh->last_use[threadIdx.x];
        if (u >= 0)
            ptx::mbar_drain(&sh->full[threadIdx.x], (uint32_t)u & 1u, a.err);
    }
    if (warp == 2 || warp == 3)
        ptx::mbar_drain(&sh->drain, 0u, a.err);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 2)
        ptx::tmem_dealloc(tmem, kQTmemCols);
}

// ------------------------------------------------------------- host side ---

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 3-D load map over a [rows][2 * Np] BF16 [hi | lo] array: (K element, row,
// plane) with strides (2, 4 * Np, 2 * Np) bytes; box 64 x 128 x planes.
bool encode_planes(CUtensorMap *m, const void *ptr, uint64_t rows, uint64_t Np, uint32_t planes)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(ptr) & 15u) != 0)
        return false;
    const cuuint64_t dims[3] = {Np, rows, 2};
    const cuuint64_t strides[2] = {4 * Np, 2 * Np};
    const cuuint32_t box[3] = {(cuuint32_t)kQKE, 128, planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// J -> [J_hi | J_lo] BF16 planes, zero padding.
__global__ void split_couplings_kernel(const float *__restrict__ J32, int Np,
                                       __nv_bfloat16 *__restrict__ Jcat)
{
    const size_t total = (size_t)Np * Np;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / Np, c = e % Np;
        const float v = J32[e];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(hi)));
        Jcat[r * 2 * Np + c] = hi;
        Jcat[r * 2 * Np + Np + c] = lo;
    }
}

// Operand of the first step: [x_hi | x_lo] (ballistic) or [sgn x | 0]
// (discrete) from the state X, zero for padded spins.
__global__ void split_state_kernel(const float *__restrict__ X, int N, int Np, int Rp, int form,
                                   __nv_bfloat16 *__restrict__ Xcat)
{
    const size_t total = (size_t)Rp * Np;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / Np, i = e % Np;
        const float x = X[e];
        __nv_bfloat16 hi, lo = __float2bfloat16_rn(0.f);
        if ((int)i >= N) {
            hi = __float2bfloat16_rn(0.f);
        } else if (form == 0) {
            hi = __float2bfloat16_rn(x);
            lo = __float2bfloat16_rn(__fsub_rn(x, __bfloat162float(hi)));
        } else {
            hi = __float2bfloat16_rn(x >= 0.f ? 1.f : -1.f);
        }
        Xcat[r * 2 * Np + i] = hi;
        Xcat[r * 2 * Np + Np + i] = lo;
    }
}

}  // namespace

struct Bf16Plan {
    CUtensorMap mapJ;
    CUtensorMap mapB[2][2];  // [form][buffer]: 2 planes (ballistic) / 1 plane (discrete)
    void *xcat[2];           // the operand buffers the maps describe
    int Np, Rp;
};

cudaError_t bf16_plan_create(Bf16Plan **out, const void *Jcat, const void *Xcat0,
                             const void *Xcat1, int Np, int Rp)
{
    *out = nullptr;
    if (Np % 128 != 0 || Rp % 128 != 0)
        return cudaErrorInvalidValue;
    Bf16Plan *p = new Bf16Plan();
    p->Np = Np;
    p->Rp = Rp;
    const void *xb[2] = {Xcat0, Xcat1};
    p->xcat[0] = const_cast<void *>(Xcat0);
    p->xcat[1] = const_cast<void *>(Xcat1);
    bool ok = encode_planes(&p->mapJ, Jcat, (uint64_t)Np, (uint64_t)Np, 2);
    for (int b = 0; b < 2 && ok; ++b) {
        ok = encode_planes(&p->mapB[0][b], xb[b], (uint64_t)Rp, (uint64_t)Np, 2) &&
             encode_planes(&p->mapB[1][b], xb[b], (uint64_t)Rp, (uint64_t)Np, 1);
    }
    if (!ok) {
        delete p;
        return cudaErrorInvalidValue;
    }
    *out = p;
    return cudaSuccess;
}

void bf16_plan_destroy(Bf16Plan *p) { delete p; }

cudaError_t launch_split_couplings(cudaStream_t st, const float *J32, int Np, void *Jcat)
{
    split_couplings_kernel<<<152 * 8, 256, 0, st>>>(J32, Np,
                                                    static_cast<__nv_bfloat16 *>(Jcat));
    return cudaGetLastError();
}

cudaError_t launch_split_state(cudaStream_t st, const float *X, int N, int Np, int Rp, int form,
                               void *Xcat)
{
    split_state_kernel<<<152 * 8, 256, 0, st>>>(X, N, Np, Rp, form,
                                                static_cast<__nv_bfloat16 *>(Xcat));
    return cudaGetLastError();
}

bool tc_bf16_persistent_fits(int Np, int Rp)
{
    const int nblk = Np / kQM, nrb = Rp / kQN;
    if (nblk < 1 || nrb < 1)
        return false;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    if (cudaFuncSetAttribute(tc_bf16x3_persistent_kernel<0>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQSmem) != cudaSuccess ||
        cudaFuncSetAttribute(tc_bf16x3_persistent_kernel<1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQSmem) != cudaSuccess)
        return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_bf16x3_persistent_kernel<0>,
                                                      kQThreads, kQSmem) != cudaSuccess)
        return false;
    return (long long)nblk * nrb <= (long long)per_sm * sms;
}

cudaError_t launch_tc_bf16x3_persistent(cudaStream_t st, const Bf16Plan *plan, int form,
                                        const PersistArgs &a)
{
    // either nsteps >= 1 updates, or (discrete form) one energy-only pass
    const bool energy_only = a.nsteps == 0 && a.final_pass == 1 && form == 1;
    if (!plan || a.Np != plan->Np || a.Rp > plan->Rp || a.Rp % kQN != 0 ||
        (!energy_only && (a.nsteps < 1 || a.final_pass != 0)) || (form != 0 && form != 1))
        return cudaErrorInvalidValue;
    auto kern = form == 0 ? tc_bf16x3_persistent_kernel<0> : tc_bf16x3_persistent_kernel<1>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQSmem);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nblk, a.nrb, 1);
    cfg.blockDim = dim3(kQThreads, 1, 1);
    cfg.dynamicSmemBytes = kQSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, plan->mapJ, plan->mapB[form][0], plan->mapB[form][1],
                              static_cast<__nv_bfloat16 *>(plan->xcat[0]),
                              static_cast<__nv_bfloat16 *>(plan->xcat[1]), a);
}

}  // namespace hsb
