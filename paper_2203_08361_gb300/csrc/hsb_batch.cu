// hsb_batch.cu -- many heated discrete SB problems (+/-1 couplings, FP8 or
// packed FP4 e2m1 operands) of uneven size in one launch: a work queue of
// instances, one CTA per instance at a time, largest first.
//
// Per instance the whole step loop (Kanao & Goto, arXiv 2203.08361: force
// Eq. (eq_fd), Methods update, evaluations every `eval_every` steps and at the
// end, best kept) runs inside one CTA, so no CTA waits on another:
//   - the spin operand S = sgn(x) of all N spins x BN replicas (FP8, at most
//     128 KB) stays in shared memory for the step; the new signs go to the
//     other global buffer and are fetched back with one TMA copy at the step
//     boundary (the old ones are read by every row block of the step);
//   - J streams through shared memory two 128-wide K chunks per TMA copy
//     (3-D box, 32 KB), three copies in flight;
//   - for each 128-spin row block tcgen05.mma (M = 128, N = BN) accumulates
//     F = J S in tensor memory, double-buffered so that the next block's MMA
//     overlaps the epilogue of this one;
//   - the epilogue (8 warps) applies the pinned update to x, y in global
//     memory, writes sgn(x') as FP8, and on evaluation steps adds s_i f_i into
//     per-replica integer sums; after the step the best energy and spins of
//     each replica are updated in place (exact integers, strict <).
// Roles: warps 0-1 stream J through three stages, warp p filling the stages
// s with s % 2 == p (J does not change, so the next step's first chunks load
// while the epilogue runs); warps 2-3 issue tcgen05.mma from elected lanes,
// warp 2 + (s % 2) consuming stage s into its own accumulator (split K, exact
// integer partial forces) when BN <= 128 and a row block has three or more
// loads, warp 2 alone otherwise; warp 2 also loads
// the resident S of each step; warps 4-11 are the epilogue.  Every stage has one
// producer and one consumer, so each mbarrier phase is awaited in order.
// FP4 (kFP4): J and S packed two e2m1 values per byte (rows of Kp / 2 bytes,
// Kp = Np rounded up to 256), so a 128-byte K slice holds 256 spins and a
// load of two slices 512; kind::mxf4 MMAs (K = 64) with unit UE8M0 block
// scales in tensor memory columns 496-511; the epilogue writes sgn(x') as
// nibble pairs (two lanes, two spins, one byte).
// Every wait is bounded; a wait that gives up raises the error word and the
// CTA stops taking instances.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hsb_device.cuh"
#include "hsb_internal.cuh"
#include "hsb_ptx.cuh"

namespace hsb {

namespace {

constexpr int kTM = 128;                 // spins per row block
constexpr int kMaxBN = 256;              // replica columns per instance
constexpr int kMaxS = 128 * 1024;        // resident spin operand bytes (BN * Np)
constexpr int kGStages = 3;             // stage s is filled by producer s % 2
constexpr int kGStageA = 2 * kTM * 128;  // two K chunks of J, 32 KB
constexpr int kGEpiWarps = 8;
constexpr int kGEpiThreads = 32 * kGEpiWarps;
constexpr int kGFirstEpi = 4;            // 2 J producers, 2 MMA warps
constexpr int kGThreads = 32 * kGFirstEpi + kGEpiThreads;
constexpr uint32_t kGColSF = 496;        // FP4 unit block scales (16 columns)

struct __align__(8) GShared {
    uint64_t full[kGStages];
    uint64_t empty[kGStages];
    uint64_t s_full;        // resident S of the step has arrived
    uint64_t step_done;     // epilogue finished a step (or the initial state)
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t drain;         // one arrival per MMA warp once its MMAs have completed
    int last_use[kGStages]; // last use of each J stage a copy was issued for
    int s_loads;            // copies of the resident S issued
    uint32_t tmem_base;
    int abort;
    int inst;               // current instance index (-1: none left)
    int esum[kMaxBN];       // per-replica sum of s_i f_i of the step (exact)
    uint8_t improved[kMaxBN];
};

constexpr size_t kGSmem = 1024 + (size_t)kMaxS + (size_t)kGStages * kGStageA + sizeof(GShared);
static_assert(kGSmem <= 232448, "shared memory per CTA is limited to 227 KB");

__device__ __forceinline__ void gbar() { ptx::named_bar(1, kGEpiThreads); }

__device__ __forceinline__ bool gbar_or(bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(kGEpiThreads)
        : "memory");
    return r != 0;
}

// tcgen05.mma from an elected lane of the converged warp (warp-uniform
// operands issue faster than from one divergent thread).
__device__ __forceinline__ void mma_fp8_elect(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
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
    const bool ok = ptx::mbar_wait(bar, parity, abort, err);
    return __all_sync(0xFFFFFFFFu, ok);
}

}  // namespace

template <bool kFP4>
__global__ void __launch_bounds__(kGThreads, 1)
tc_batch_kernel(const BatchInst *__restrict__ insts, const BatchArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sS = base;                      // resident operand [chunk][BN][128]
    uint8_t *sA = base + kMaxS;              // J stages
    GShared *sh = reinterpret_cast<GShared *>(sA + (size_t)kGStages * kGStageA);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStages; ++s) {
            ptx::mbar_init(&sh->full[s], 1);
            ptx::mbar_init(&sh->empty[s], 1);
        }
        ptx::mbar_init(&sh->s_full, 1);
        ptx::mbar_init(&sh->step_done, 1);
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&sh->acc_full[b], 2);  // one arrival per MMA warp
            ptx::mbar_init(&sh->acc_empty[b], 1);
        }
        ptx::mbar_init(&sh->drain, 2);
        for (int s = 0; s < kGStages; ++s)
            sh->last_use[s] = -1;
        sh->s_loads = 0;
        sh->abort = 0;
        ptx::mbar_init_fence();
    }
    if (warp == 2)
        ptx::tmem_alloc(&sh->tmem_base, 512);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    if (kFP4) {
        // unit block scales (UE8M0 0x7F = 2^0) in 16 columns of every lane,
        // before the first MMA reads them
        if (warp >= kGFirstEpi && warp < kGFirstEpi + 4) {
            uint32_t one[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
                one[j] = 0x7F7F7F7Fu;
            ptx::tmem_st16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + kGColSF, one);
            ptx::tmem_st_wait();
        }
        ptx::tc_fence_before();
        __syncthreads();
        ptx::tc_fence_after();
    }

    // running counters of each role, continued across instances
    uint32_t g = 0;       // J stages (producer, MMA)
    uint32_t tile = 0;    // accumulator tiles (MMA, epilogue)
    uint32_t sdone = 0;   // step_done phases (producer waits, epilogue arrives)
    uint32_t sfull = 0;   // s_full phases (producer arrives via TMA, MMA waits)

    for (;;) {
        if (threadIdx.x == 0)
            sh->inst = *(volatile int *)&sh->abort ? -1 : (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int idx = sh->inst;
        if (idx < 0 || idx >= a.count)
            break;
        const BatchInst &in = insts[idx];
        const int N = in.N, Np = in.Np, BN = in.BN, R = in.R;
        const int nblk = Np / kTM;
        // 128-byte K slices of an operand row: Np / 128 (FP8), Kp / 256 (FP4)
        const int nslice = kFP4 ? in.Kp / 256 : nblk;
        const int npairs = (nslice + 1) >> 1;  // loads of two slices per row block
        const size_t srow = kFP4 ? (size_t)in.Kp / 2 : (size_t)Np;  // operand row bytes
        const int passes = a.steps + 1;  // updates, then the final evaluation

        // K is split over the two MMA warps (each into its own accumulator,
        // the loads of stage p to warp p) when the accumulators fit and every
        // row block has at least two loads
        // (every kGStages consecutive loads include stages of both parities,
        // so each MMA warp gets at least one load of every row block)
        const bool split = a.allow_split && BN <= (kFP4 ? 96 : 128) && npairs >= kGStages;

        if (warp < 2) {
            // --------------------------------------------------- J producers
            // producer p fills stage p (loads g with g % 2 == p); J does not
            // change, so the next step's first chunks load during the epilogue
            if (lane == 0) {
                const int pw = warp;
                ptx::prefetch_tmap(&in.mapA);
                bool fail = false;
                for (int k = 0; k < passes && !fail; ++k)
                    for (int mb = 0; mb < nblk && !fail; ++mb)
                        for (int p = 0; p < npairs; ++p, ++g) {
                            const int s = (int)(g % kGStages);
                            if ((s & 1) != pw)
                                continue;
                            const uint32_t ph = (g / kGStages) & 1u;
                            if (!ptx::mbar_wait(&sh->empty[s], ph ^ 1u, &sh->abort, a.err)) {
                                fail = true;
                                break;
                            }
                            atomicMax(&sh->last_use[s], (int)(g / kGStages));  // for the drain
                            ptx::mbar_expect_tx(&sh->full[s], (uint32_t)kGStageA);
                            ptx::tma_load_3d(sA + (size_t)s * kGStageA, &in.mapA, 0, mb * kTM,
                                             2 * p, &sh->full[s]);
                        }
            }
        } else if (warp < kGFirstEpi) {
            // ----------------------------------------------------------- MMA
            // warp 2 + pw consumes stage pw (with the split) or every stage
            // (warp 2, without it), always in load order; warp 2 also loads
            // the resident S of each step (its MMAs cannot start before)
            const int pw = warp - 2;
            const uint32_t idesc =
                kFP4 ? ptx::idesc_mxf4_e2m1(kTM, BN) : ptx::idesc_e4m3_f32(kTM, BN);
            const uint64_t sdesc0 = ptx::sw128_desc(ptx::smem_u32(sS));
            const uint64_t adesc0 = ptx::sw128_desc(ptx::smem_u32(sA));
            bool ok = true;
            for (int k = 0; k < passes && ok; ++k) {
                if (pw == 0) {
                    // the operand of step k is complete once the previous
                    // step's epilogue (or the initial state) is done
                    if (!warp_wait(&sh->step_done, sdone & 1u, &sh->abort, a.err))
                        break;
                    ++sdone;
                    if (lane == 0) {
                        ptx::fence_proxy_async_global();
                        ++sh->s_loads;  // for the drain
                        ptx::mbar_expect_tx(&sh->s_full, (uint32_t)(BN * srow));
                        ptx::tma_load_3d(sS, &in.mapS[k & 1], 0, 0, 0, &sh->s_full);
                    }
                    __syncwarp();
                }
                if (!warp_wait(&sh->s_full, sfull & 1u, &sh->abort, a.err))
                    break;
                ++sfull;
                ptx::tc_fence_after();
                for (int mb = 0; mb < nblk && ok; ++mb) {
                    const uint32_t buf = tile & 1u;
                    if (!warp_wait(&sh->acc_empty[buf], ((tile >> 1) & 1u) ^ 1u, &sh->abort,
                                   a.err)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t dcol =
                        tmem + (split ? buf * 2u + (uint32_t)pw : buf) * (uint32_t)BN;
                    int mine = 0;
                    for (int p = 0; p < npairs; ++p, ++g) {
                        const int s = (int)(g % kGStages);
                        if (split ? (s & 1) != pw : pw != 0)
                            continue;
                        const uint32_t ph = (g / kGStages) & 1u;
                        if (!warp_wait(&sh->full[s], ph, &sh->abort, a.err)) {
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        for (int c = 0; c < 2; ++c) {
                            const int kc = 2 * p + c;
                            if (kc >= nslice)
                                break;
                            const uint64_t ad =
                                adesc0 + (uint64_t)(((size_t)s * kGStageA + c * kTM * 128) >> 4);
                            const uint64_t bd = sdesc0 + (uint64_t)((kc * BN * 128) >> 4);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint32_t acc = (mine | c | kk) != 0 ? 1u : 0u;
                                if (kFP4)
                                    ptx::mma_mxf4_elect(dcol, ad + (uint64_t)(kk * 2),
                                                        bd + (uint64_t)(kk * 2), idesc,
                                                        tmem + kGColSF, tmem + kGColSF, acc);
                                else
                                    mma_fp8_elect(dcol, ad + (uint64_t)(kk * 2),
                                                  bd + (uint64_t)(kk * 2), idesc, acc);
                            }
                        }
                        commit_elect(&sh->empty[s]);
                        ++mine;
                    }
                    if (!ok)
                        break;
                    if (mine > 0)
                        commit_elect(&sh->acc_full[buf]);
                    else if (lane == 0)
                        ptx::mbar_arrive(&sh->acc_full[buf]);  // no load of this tile here
                    ++tile;
                }
            }
        } else {
            // ------------------------------------------------------ epilogue
            const int et = threadIdx.x - 32 * kGFirstEpi;  // 0..255
            const int q = warp & 3;                        // lane quadrant
            const int half = (warp - kGFirstEpi) >> 2;     // column half
            const int cw = BN / 2;                     // columns per warp (multiple of 16)
            const int cbase = half * cw;
            const uint32_t lane_off = (uint32_t)(q * 32) << 16;
            const uint64_t s_inst = splitmix64_out(a.seed, (uint64_t)in.instance + 1u);
            // the instance's buffers as local restrict pointers: read through
            // the instance table, they would be reloaded after every store
            float *__restrict__ X = in.X;
            float *__restrict__ Y = in.Y;
            uint8_t *__restrict__ S8a = in.S8a;
            uint8_t *__restrict__ S8b = in.S8b;
            double *__restrict__ Ebest = in.Ebest;
            int8_t *__restrict__ Sbest = in.Sbest;

            // initial state: x, y uniform in (-L, L), S = sgn(x), best = +inf
            for (size_t e = et; e < (size_t)BN * Np; e += kGEpiThreads) {
                const int r = (int)(e / Np), i = (int)(e % Np);
                float x = 0.f, y = 0.f;
                uint8_t sg = 0;
                if (i < N) {
                    x = init_uniform(s_inst, (uint32_t)r, (uint32_t)i, 0, a.scale);
                    y = init_uniform(s_inst, (uint32_t)r, (uint32_t)i, 1, a.scale);
                    sg = fp8_sign(x);
                }
                X[e] = x;
                Y[e] = y;
                if (!kFP4)
                    S8a[e] = sg;
            }
            if (kFP4) {
                // packed e2m1 signs of the stored x (spins 2b and 2b + 1 of
                // byte b; padded spins and the K padding 0)
                gbar();
                for (size_t e = et; e < (size_t)BN * srow; e += kGEpiThreads) {
                    const int r = (int)(e / srow), i = 2 * (int)(e % srow);
                    const uint32_t lo =
                        i < N ? (X[(size_t)r * Np + i] >= 0.f ? kFp4PlusOne : kFp4MinusOne) : 0u;
                    const uint32_t hi = i + 1 < N ? (X[(size_t)r * Np + i + 1] >= 0.f ? kFp4PlusOne
                                                                                      : kFp4MinusOne)
                                                  : 0u;
                    S8a[e] = (uint8_t)(lo | (hi << 4));
                }
            }
            for (int r = et; r < R; r += kGEpiThreads)
                Ebest[r] = INFINITY;
            for (int r = et; r < kMaxBN; r += kGEpiThreads)
                sh->esum[r] = 0;
            ptx::fence_proxy_async_global();
            gbar();
            if (et == 0)
                ptx::mbar_arrive(&sh->step_done);

            StepConsts c;
            c.c0 = in.c0;
            c.dt = a.dt;
            c.q = a.q;
            c.g = a.g;
            c.nz = a.nz;
            const StepConsts2 k2 = step_consts2(c);
            bool left = false;
            for (int k = 0; k < passes && !left; ++k) {
                const bool final_pass = k == a.steps;
                const bool ev = final_pass ||
                                (a.eval_every > 0 && k > 0 && k % a.eval_every == 0);
                const float pk = final_pass ? 0.f : a.pk[k];
                const uint64_t pk2 = f2_pack(pk, pk);
                const uint8_t *Sold = (k & 1) ? S8b : S8a;
                uint8_t *Snew = (k & 1) ? S8a : S8b;
                for (int mb = 0; mb < nblk; ++mb) {
                    const uint32_t buf = tile & 1u;
                    const int i = mb * kTM + q * 32 + lane;
                    const bool live = i < N;
                    // x, y of the first 16 columns are fetched before the
                    // accumulator is ready, so the loads overlap the MMA
                    float xr[16], yr[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const size_t e = (size_t)(cbase + j) * Np + i;
                        xr[j] = X[e];
                        yr[j] = Y[e];
                    }
                    const bool ok = ptx::mbar_wait(&sh->acc_full[buf], (tile >> 1) & 1u,
                                                   &sh->abort, a.err);
                    if (gbar_or(!ok)) {
                        left = true;
                        break;
                    }
                    ++tile;
                    ptx::tc_fence_after();
                    for (int cb = 0; cb < cw; cb += 16) {
                        uint32_t f[16], f1[16];
                        const uint32_t acol = tmem + (split ? buf * 2u : buf) * (uint32_t)BN +
                                              lane_off + (uint32_t)(cbase + cb);
                        ptx::tmem_ld16(acol, f);
                        if (split)
                            ptx::tmem_ld16(acol + (uint32_t)BN, f1);
                        // next chunk's x, y in flight while this chunk computes
                        float xn[16], yn[16];
                        const bool more = cb + 16 < cw;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const size_t e = (size_t)(cbase + cb + 16 + j) * Np + i;
                            xn[j] = more ? X[e] : 0.f;
                            yn[j] = more ? Y[e] : 0.f;
                        }
                        ptx::tmem_ld_wait();
                        if (split) {
                            // partial forces over disjoint K ranges: exact integers
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                f[j] = __float_as_uint(
                                    __fadd_rn(__uint_as_float(f[j]), __uint_as_float(f1[j])));
                        }
                        if (ev) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const int r = cbase + cb + j;
                                const float fj = __uint_as_float(f[j]);
                                int term = live ? (xr[j] >= 0.f ? (int)fj : -(int)fj) : 0;
#pragma unroll
                                for (int off = 16; off > 0; off >>= 1)
                                    term += __shfl_xor_sync(0xFFFFFFFFu, term, off);
                                if (lane == 0)
                                    atomicAdd(&sh->esum[r], term);
                            }
                        }
                        if (!final_pass) {
                            // two replicas per packed binary32 operation
#pragma unroll
                            for (int j = 0; j < 16; j += 2) {
                                const size_t e = (size_t)(cbase + cb + j) * Np + i;
                                float xo0, xo1;
                                uint64_t yo;
                                sb_update2(f2_pack_bits(f[j], f[j + 1]), f2_pack(xr[j], xr[j + 1]),
                                           f2_pack(yr[j], yr[j + 1]), pk2, k2, xo0, xo1, yo);
                                X[e] = xo0;
                                X[e + Np] = xo1;
                                Y[e] = f2_lo(yo);
                                Y[e + Np] = f2_hi(yo);
                                if (kFP4) {
                                    // spins i (even lane) and i + 1 share a byte
                                    const uint32_t n0 =
                                        live ? (xo0 >= 0.f ? kFp4PlusOne : kFp4MinusOne) : 0u;
                                    const uint32_t n1 =
                                        live ? (xo1 >= 0.f ? kFp4PlusOne : kFp4MinusOne) : 0u;
                                    const uint32_t u0 = __shfl_down_sync(0xFFFFFFFFu, n0, 1);
                                    const uint32_t u1 = __shfl_down_sync(0xFFFFFFFFu, n1, 1);
                                    if ((lane & 1) == 0) {
                                        const size_t b = (size_t)(cbase + cb + j) * srow + i / 2;
                                        Snew[b] = (uint8_t)(n0 | (u0 << 4));
                                        Snew[b + srow] = (uint8_t)(n1 | (u1 << 4));
                                    }
                                } else {
                                    Snew[e] = live ? fp8_sign(xo0) : (uint8_t)0;
                                    Snew[e + Np] = live ? fp8_sign(xo1) : (uint8_t)0;
                                }
                            }
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            xr[j] = xn[j];
                            yr[j] = yn[j];
                        }
                    }
                    ptx::tc_fence_before();
                    gbar();
                    if (et == 0)
                        ptx::mbar_arrive(&sh->acc_empty[buf]);
                }
                if (left)
                    break;
                // end of step k: best update from the evaluation of s(t_k)
                if (ev) {
                    for (int r = et; r < R; r += kGEpiThreads) {
                        const double E = -0.5 * (double)sh->esum[r];
                        const int take = E < Ebest[r];
                        if (take)
                            Ebest[r] = E;
                        sh->improved[r] = take;
                    }
                    gbar();
                    const int w = warp - kGFirstEpi;
                    for (int r = w; r < R; r += kGEpiWarps)
                        if (sh->improved[r])
                            for (int i = lane; i < N; i += 32) {
                                const bool plus =
                                    kFP4 ? ((Sold[(size_t)r * srow + i / 2] >> (4 * (i & 1))) &
                                            15u) == kFp4PlusOne
                                         : Sold[(size_t)r * Np + i] == kFp8PlusOne;
                                Sbest[(size_t)r * N + i] = plus ? (int8_t)1 : (int8_t)-1;
                            }
                    for (int r = et; r < kMaxBN; r += kGEpiThreads)
                        sh->esum[r] = 0;
                }
                ptx::fence_proxy_async_global();
                gbar();
                // one arrival per pass the producer waits for: the initial state
                // and steps 0..steps-1 (the final evaluation pass has no successor)
                if (et == 0 && !final_pass)
                    ptx::mbar_arrive(&sh->step_done);
            }
        }
        __syncthreads();
        if (*(volatile int *)&sh->abort)
            break;
    }

    // drain before tensor memory and shared memory are given up (every exit
    // path): the last copy into each J stage and the last resident S have
    // landed and every MMA has completed, each wait bounded
    if (warp == 2 || warp == 3)
        commit_elect(&sh->drain);
    __syncthreads();
    if (threadIdx.x < kGStages) {
        const int u = sh->last_use[threadIdx.x];
        if (u >= 0)
            ptx::mbar_drain(&sh->full[threadIdx.x], (uint32_t)u & 1u, a.err);
    }
    if (threadIdx.x == 32 && sh->s_loads > 0)
        ptx::mbar_drain(&sh->s_full, (uint32_t)(sh->s_loads - 1) & 1u, a.err);
    if (warp == 2 || warp == 3)
        ptx::mbar_drain(&sh->drain, 0u, a.err);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 2)
        ptx::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------- host side ---

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn batch_encode_fn()
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

// 3-D view of a [rows][cols] byte array as (byte in a 128-byte K chunk, row,
// chunk), box 128 x box_rows x box_chunks, 128-byte swizzle.
bool encode_chunks(CUtensorMap *m, const void *ptr, uint64_t rows, uint64_t cols,
                   uint32_t box_rows, uint32_t box_chunks)
{
    EncodeTiledFn fn = batch_encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(ptr) & 15u) != 0 || cols % 128u != 0)
        return false;
    const cuuint64_t dims[3] = {128, rows, cols / 128};
    const cuuint64_t strides[2] = {cols, 128};
    const cuuint32_t box[3] = {128, box_rows, box_chunks};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool batch_shape_ok(int Np, int R, bool fp4)
{
    const int BN = round_up(R, 32);
    const int Kp = round_up(Np, 256);
    if (fp4)  // two accumulators and the block scales in 512 columns
        return R >= 1 && 2 * BN + 16 <= 512 && Np % kTM == 0 && Kp / 256 <= 256 &&
               BN * (Kp / 2) <= kMaxS;
    return R >= 1 && BN <= kMaxBN && Np % kTM == 0 && Np / 128 <= 256 && BN * Np <= kMaxS;
}

cudaError_t batch_fill_maps(BatchInst *in, const uint8_t *J, const uint8_t *Sa,
                            const uint8_t *Sb, int Np, int Rcap, int Kp)
{
    const int BN = in->BN;
    // operand rows: Np bytes (FP8) or Kp / 2 bytes of packed e2m1 (Kp > 0)
    const uint64_t cols = Kp > 0 ? (uint64_t)Kp / 2 : (uint64_t)Np;
    if (!encode_chunks(&in->mapA, J, (uint64_t)Np, cols, kTM, 2) ||
        !encode_chunks(&in->mapS[0], Sa, (uint64_t)Rcap, cols, (uint32_t)BN,
                       (uint32_t)(cols / 128)) ||
        !encode_chunks(&in->mapS[1], Sb, (uint64_t)Rcap, cols, (uint32_t)BN,
                       (uint32_t)(cols / 128)))
        return cudaErrorInvalidValue;
    in->Kp = Kp;
    return cudaSuccess;
}

cudaError_t launch_tc_batch(cudaStream_t st, const BatchInst *d_insts, const BatchArgs &a,
                            int ctas)
{
    auto kern = a.fp4 ? tc_batch_kernel<true> : tc_batch_kernel<false>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem);
    if (e != cudaSuccess)
        return e;
    kern<<<ctas, kGThreads, kGSmem, st>>>(d_insts, a);
    return cudaGetLastError();
}

}  // namespace hsb
