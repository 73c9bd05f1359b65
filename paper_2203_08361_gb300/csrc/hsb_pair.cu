// hsb_pair.cu -- persistent tcgen05 kernel for the heated discrete SB step
// loop (HdSB, couplings in {-1, 0, +1}, N <= 4096) run by CTA pairs.
//
// Kanao & Goto, arXiv 2203.08361: force Eq. (eq_fd); update Methods Eqs.
// (eq_SyEuY), (eq_SyEuX), (eq_WallX), (eq_WallY), (eq_EuHeat); energy Eq.
// (eq_Ising) evaluated every `eval_every` steps and at the end (K2000 study).
//
// The force is formed transposed, F^T = S^T J: the MMA's M dimension is the
// replicas and its N dimension the spins.  A pair of CTAs (a cluster of two,
// tcgen05 cta_group::2) owns 256 replicas x 128 spins: each CTA holds 128
// replicas (M = 256 over the pair) and loads 64 of the 128 spins' rows of J
// (the B operand, split over the pair), so a step moves per CTA 128 x Np
// bytes of the sign operand S = sgn(x) and 64 x Np bytes of J through L2.
// Each CTA's tensor memory holds its 128 replicas x 128 spins: the FP32
// accumulator (columns 0-127), x (128-255) and y (256-383); lane = replica,
// column = spin, so an epilogue thread owns 32 spins of one replica and
// writes their sign bytes as one row segment of S (K-major, the A operand of
// the next step) with no transpose.
//
// Roles (736 threads):
//   warps 0-4   TMA issuers: issuer w owns stages w and w + 5 of the nine
//               24 KB stages (a 16 KB chunk of S, 128 replicas x 128 spins,
//               and the 8 KB of J the pair's MMAs multiply it with).  Lane 1
//               copies the rows of J as soon as the stage is free; lane 0
//               copies the chunk of S once the poller has seen it published.
//               The chunks of a pass are taken in the order 0, 1, ...,
//               the same in every tile (an order that starts from the tile's
//               own chunk chains each tile to its predecessor's publication
//               and the tiles drift apart).  Every copy
//               counts on the even CTA's barrier of the stage (tcgen05 pair
//               form), which the even CTA arms for both CTAs' 48 KB;
//   warp 5      poller: reads the published-step flags of the pass's chunks
//               (one per lane, all at once) and raises each chunk's pass
//               counter in shared memory, so no copy waits for a flag round
//               trip once its pass has started;
//   warp 6      even CTA: the pair's MMAs (M = 256, N = 128, K = 32, issued
//               from an elected lane), committed to both CTAs' barriers;
//   warps 7-22  epilogue, four warps per 32-lane quadrant of tensor memory
//               (one per 32-spin column group), in two phases.  Phase 1
//               computes only the sign of x~ (the walls keep it), writes it as
//               FP8 into the other operand buffer with 16-byte stores, and one
//               thread releases the tile's flag at gpu scope.  Phase 2 repeats
//               the pinned update in full, stores x' and y' in tensor memory
//               and, on evaluation passes, forms the per-replica partial sums
//               of s_i f_i (exact integers) and the snapshot of s.
// A final pass after the last update evaluates E(t_Ns); select_best_kernel
// picks each replica's best evaluation afterwards.
//
// The pair's CTAs must all be co-resident (the launcher checks the number of
// active clusters).  Every wait is bounded (2 s of wall clock); on expiry the
// CTA's abort flag and the error word are raised, epilogue warps decide to
// leave together through an OR-barrier.  Before tensor memory is freed the
// MMA warp waits (bounded) for every MMA it issued and, after a cluster
// barrier, the even CTA waits (bounded) for the last copies of each stage
// from either CTA (both CTAs record their copies in its shared memory); a
// second cluster barrier keeps both CTAs' shared memory alive until then.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsb_device.cuh"
#include "hsb_internal.cuh"
#include "hsb_ptx.cuh"

namespace hsb {

namespace {

constexpr int kQM = 128;                       // replicas per CTA (pair MMA M = 256)
constexpr int kQN = 128;                       // spins per pair tile (MMA N)
constexpr int kQK = 128;                       // spins (K) per S chunk
constexpr int kQStages = 9;
constexpr int kQStageA = kQM * kQK;            // 16 KB of S per stage
constexpr int kQJRows = kQN / 2;               // rows of J loaded by one CTA
constexpr int kQStageJ = kQJRows * kQK;        // 8 KB of J per stage
constexpr int kQStageBytes = 2 * (kQStageA + kQStageJ);  // both CTAs' copies
constexpr int kQMaxChunks = 32;                // Np <= 4096 (one poller lane each)
constexpr int kQIssuers = 5;                   // issuer w owns stages w, w + 5
constexpr int kQPoller = kQIssuers;
constexpr int kQMmaWarp = kQPoller + 1;
constexpr int kQFirstEpi = kQMmaWarp + 1;
constexpr int kQEpiWarps = 16;
constexpr int kQEpiThreads = 32 * kQEpiWarps;
constexpr int kQThreads = 32 * kQFirstEpi + kQEpiThreads;
constexpr uint32_t kQTmemCols = 512;
constexpr uint32_t kQColAcc = 0;
constexpr uint32_t kQColX = 128;
constexpr uint32_t kQColY = 256;
constexpr uint32_t kQIdesc = ptx::idesc_e4m3_f32(2 * kQM, kQN);

struct __align__(8) QShared {
    uint64_t full[kQStages];   // (even CTA) both CTAs' copies of the stage have landed
    uint64_t empty[kQStages];  // the pair's MMAs have read the stage
    uint64_t accfull;          // the accumulator holds the pass's force
    uint64_t tmem_empty;       // (even CTA) both epilogues have read the accumulator
    uint64_t drain;            // (even CTA) every MMA issued has completed
    uint32_t tmem_base;
    int abort;
    int copies[kQStages][2][2];  // (even CTA) uses copied per stage: [stage][CTA][S, J]
    int rdy[kQMaxChunks];        // chunk c is published for passes < rdy[c] (poller)
    int red[4][kQM];             // per column group sums of s_i f_i
};

constexpr size_t kQSmem =
    1024 + (size_t)kQStages * (kQStageA + kQStageJ) + sizeof(QShared);
static_assert(kQSmem <= 232448, "shared memory per CTA is limited to 227 KB");
static_assert(kQThreads <= 1024, "too many threads per CTA");

// Barrier among the epilogue warps that ORs a predicate over them.
__device__ __forceinline__ bool qepi_bar_or(bool pred)
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

__device__ __forceinline__ void qepi_bar() { ptx::named_bar(1, kQEpiThreads); }

// Bounded wait by every lane of a warp; false in all lanes if any gave up.
__device__ __forceinline__ bool warp_wait_cl(uint64_t *bar, uint32_t parity, int *abort, int *err)
{
    const bool ok = ptx::mbar_wait_cluster(bar, parity, abort, err);
    return __all_sync(0xFFFFFFFFu, ok);
}

__device__ __forceinline__ uint32_t pack4(uint8_t b0, uint8_t b1, uint8_t b2, uint8_t b3)
{
    return (uint32_t)b0 | ((uint32_t)b1 << 8) | ((uint32_t)b2 << 16) | ((uint32_t)b3 << 24);
}

}  // namespace

__global__ void __launch_bounds__(kQThreads, 1)
tc_fp8_pair_kernel(const __grid_constant__ CUtensorMap tmapJ,
                   const __grid_constant__ CUtensorMap tmapS0,
                   const __grid_constant__ CUtensorMap tmapS1, const PersistArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = base;                                  // [stage][128 replicas][128 B]
    uint8_t *sJ = base + (size_t)kQStages * kQStageA;    // [stage][64 spins][128 B]
    QShared *sh = reinterpret_cast<QShared *>(sJ + (size_t)kQStages * kQStageJ);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t h = ptx::cluster_ctarank();  // 0: the CTA that issues the pair's MMAs
    const int sg = blockIdx.x >> 1;             // spin block of the pair
    const int rho = 2 * blockIdx.y + (int)h;    // 128-replica block of this CTA
    const int i0 = sg * kQN;
    const int r0 = rho * kQM;
    const int nchunk = a.nblk;                  // Np / 128 K chunks
    const int passes = a.nsteps + a.final_pass;
    const int total = passes * nchunk;          // S loads of the launch

    if (threadIdx.x == 0) {
        for (int s = 0; s < kQStages; ++s) {
            ptx::mbar_init(&sh->full[s], 1);  // armed by the even CTA for both
            ptx::mbar_init(&sh->empty[s], 1);
            sh->copies[s][0][0] = sh->copies[s][0][1] = 0;
            sh->copies[s][1][0] = sh->copies[s][1][1] = 0;
        }
        ptx::mbar_init(&sh->accfull, 1);
        ptx::mbar_init(&sh->tmem_empty, 2 * kQEpiWarps);
        ptx::mbar_init(&sh->drain, 1);
        for (int c = 0; c < kQMaxChunks; ++c)
            sh->rdy[c] = 0;
        sh->abort = 0;
        ptx::mbar_init_fence();
    }
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmapJ);
        ptx::prefetch_tmap(&tmapS0);
        ptx::prefetch_tmap(&tmapS1);
    }
    if (warp == kQMmaWarp)
        ptx::tmem_alloc_pair(&sh->tmem_base, kQTmemCols);
    ptx::tc_fence_before();
    ptx::cluster_sync();  // both CTAs' barriers and tensor memory exist
    ptx::tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (warp < kQIssuers) {
        // ------------------------------------------------------- TMA issuers
        // lane 0: chunks of S, lane 1: rows of J; each copies the loads of
        // the warp's two stages in load order
        if (lane < 2) {
            const bool jl = lane == 1;
            const int st0 = warp, st1 = warp + kQIssuers;  // st1 < kQStages for warps 0-3
            int used0 = 0, used1 = 0;                      // uses copied per owned stage
            int next0 = st0, next1 = st1 < kQStages ? st1 : total;
            while (true) {
                const bool w = next1 < next0;
                const int g = w ? next1 : next0;
                if (g >= total)
                    break;
                const int s = w ? st1 : st0;
                const int u = g / kQStages;
                if (w)
                    next1 = g + kQStages;
                else
                    next0 = g + kQStages;
                const int kl = g / nchunk;
                const int t = g - kl * nchunk;
                const int c = t;  // the same chunk order in every tile
                const uint32_t full_own = ptx::smem_u32(&sh->full[s]);
                const uint32_t full_c = h == 0 ? full_own : ptx::mapa_shared(full_own, 0u);
                if (!ptx::mbar_wait_cluster(&sh->empty[s], (uint32_t)(u & 1) ^ 1u, &sh->abort,
                                            a.err))
                    break;
                if (jl) {
                    // the even CTA arms the stage for both CTAs' copies; a copy
                    // of the odd CTA that lands first takes the transaction
                    // count below zero until then (it cannot belong to the
                    // previous use: that use's MMAs had completed before this
                    // stage was free)
                    if (h == 0)
                        ptx::mbar_expect_tx(&sh->full[s], (uint32_t)kQStageBytes);
                    ptx::tma_load_2d_pair(sJ + (size_t)s * kQStageJ, &tmapJ, c * kQK,
                                          i0 + (int)h * kQJRows, full_c);
                } else {
                    // chunk c of this CTA's replicas for pass kl is published
                    if (!ptx::wait_count(&sh->rdy[c], kl + 1, &sh->abort, a.err))
                        break;
                    ptx::fence_proxy_async_global();
                    const CUtensorMap *mapS = ((a.par0 + kl) & 1) ? &tmapS1 : &tmapS0;
                    ptx::tma_load_2d_pair(sA + (size_t)s * kQStageA, mapS, c * kQK, r0, full_c);
                }
                if (w)
                    used1 = u + 1;
                else
                    used0 = u + 1;
            }
            // the copies made, for the drain (in the even CTA's shared memory)
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                const int s = w ? st1 : st0;
                if (s >= kQStages)
                    continue;
                int *dst = &sh->copies[s][h][jl ? 1 : 0];
                const int n = w ? used1 : used0;
                if (h == 0)
                    *(volatile int *)dst = n;
                else
                    ptx::st_shared_cluster(ptx::mapa_shared(ptx::smem_u32(dst), 0u), n);
            }
        }
    } else if (warp == kQPoller) {
        // ------------------------------------------------------------ poller
        // lane c reads the flag of chunk c (tile (c, rho)) for each pass
        bool fail = false;
        for (int kl = 0; kl < passes && !fail; ++kl) {
            bool pending = lane < nchunk;
            const unsigned long long t0 = ptx::globaltimer();
            int idle = 0;
            while (__any_sync(0xFFFFFFFFu, pending)) {
                bool ready = false;
                if (pending)
                    ready = ptx::ld_acquire_gpu(&a.flags[flag_index(lane, rho, a.nrb)]) >= kl;
                if (ready) {
                    ptx::st_release_cta_shared(&sh->rdy[lane], kl + 1);
                    pending = false;
                }
                if (!__any_sync(0xFFFFFFFFu, ready)) {
                    int give_up = 0;
                    if (lane == 0) {
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
    } else if (warp == kQMmaWarp && h == 0) {
        // --------------------------------------------------- the pair's MMAs
        const uint64_t adesc0 = ptx::sw128_desc(ptx::smem_u32(sA));
        const uint64_t bdesc0 = ptx::sw128_desc(ptx::smem_u32(sJ));
        const uint32_t acc = tmem + kQColAcc;
        bool ok = true;
        for (int kl = 0; ok && kl < passes; ++kl) {
            if (kl > 0) {
                ok = warp_wait_cl(&sh->tmem_empty, (uint32_t)(kl - 1) & 1u, &sh->abort, a.err);
                if (!ok)
                    break;
                ptx::tc_fence_after();
            }
            for (int t = 0; t < nchunk; ++t) {
                const int g = kl * nchunk + t;
                const int s = g % kQStages;
                ok = warp_wait_cl(&sh->full[s], (uint32_t)(g / kQStages) & 1u, &sh->abort, a.err);
                if (!ok)
                    break;
                ptx::tc_fence_after();
                const uint64_t ad = adesc0 + (uint64_t)((s * kQStageA) >> 4);
                const uint64_t bd = bdesc0 + (uint64_t)((s * kQStageJ) >> 4);
#pragma unroll
                for (int kk = 0; kk < kQK / 32; ++kk)
                    ptx::mma_fp8_pair_elect(acc, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2),
                                            kQIdesc, (t | kk) != 0 ? 1u : 0u);
                const uint32_t e_own = ptx::smem_u32(&sh->empty[s]);
                ptx::commit_pair_elect(e_own);
                ptx::commit_pair_elect(ptx::mapa_shared(e_own, 1u));
            }
            if (!ok)
                break;
            const uint32_t a_own = ptx::smem_u32(&sh->accfull);
            ptx::commit_pair_elect(a_own);
            ptx::commit_pair_elect(ptx::mapa_shared(a_own, 1u));
        }
        // drain: every MMA issued by this warp has completed
        ptx::commit_pair_elect(ptx::smem_u32(&sh->drain));
        ptx::mbar_drain(&sh->drain, 0u, a.err);
        __syncwarp();
    } else if (warp >= kQFirstEpi) {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - kQFirstEpi;   // 0..15
        const int q = warp & 3;             // tensor-memory lane quadrant of this warp
        const int cg = ew >> 2;             // spin column group (32 spins)
        const int et = threadIdx.x - 32 * kQFirstEpi;
        const int r = r0 + q * 32 + lane;   // replica of this thread
        const int ib = i0 + cg * 32;        // first of this thread's 32 spins
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const uint32_t col0 = (uint32_t)(cg * 32);
        const uint32_t tmem_empty0 = ptx::mapa_shared(ptx::smem_u32(&sh->tmem_empty), 0u);
        const size_t plane = (size_t)a.Rp * a.Np;
        // live spins of this thread's 32 (padded spins publish a zero byte)
        const uint32_t live = ib + 32 <= a.N ? 0xFFFFFFFFu
                              : ib >= a.N   ? 0u
                                            : ((1u << (a.N - ib)) - 1u);

        // initial state of the tile into tensor memory
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            uint32_t xr[16], yr[16];
            const float4 *xs = reinterpret_cast<const float4 *>(a.X + (size_t)r * a.Np + ib + 16 * hh);
            const float4 *ys = reinterpret_cast<const float4 *>(a.Y + (size_t)r * a.Np + ib + 16 * hh);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float4 xv = xs[v], yv = ys[v];
                xr[4 * v] = __float_as_uint(xv.x);
                xr[4 * v + 1] = __float_as_uint(xv.y);
                xr[4 * v + 2] = __float_as_uint(xv.z);
                xr[4 * v + 3] = __float_as_uint(xv.w);
                yr[4 * v] = __float_as_uint(yv.x);
                yr[4 * v + 1] = __float_as_uint(yv.y);
                yr[4 * v + 2] = __float_as_uint(yv.z);
                yr[4 * v + 3] = __float_as_uint(yv.w);
            }
            ptx::tmem_st16(tmem + lane_off + kQColX + col0 + 16 * hh, xr);
            ptx::tmem_st16(tmem + lane_off + kQColY + col0 + 16 * hh, yr);
        }
        ptx::tmem_st_wait();

        bool left = false;
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
                pk_next = a.pk[k + 1];  // off the critical path

            // x and y of the first 16 spins (the MMA does not write them) and
            // v = p_k x of the update, formed in the MMA's shadow
            uint32_t xpre[16], ypre[16];
            uint64_t vpre[8];
            ptx::tmem_ld16(tmem + lane_off + kQColX + col0, xpre);
            ptx::tmem_ld16(tmem + lane_off + kQColY + col0, ypre);
            ptx::tmem_ld_wait(xpre);
            ptx::tmem_ld_wait(ypre);
#pragma unroll
            for (int j = 0; j < 16; j += 2)
                vpre[j / 2] = f2_fma(pk2, f2_pack_bits(xpre[j], xpre[j + 1]), k2.z);
            const bool ok = ptx::mbar_wait_cluster(&sh->accfull, (uint32_t)kl & 1u, &sh->abort,
                                                   a.err);
            if (qepi_bar_or(!ok)) {
                left = true;
                break;
            }
            ptx::tc_fence_after();

            if (!final_pass) {
                // ---- phase 1: sgn(x') = sgn(x~) of this thread's 32 spins,
                // published before the rest of the update.  The operations are
                // those of the update up to p = q yt; x~ = fl(x + p) is
                // negative exactly when p < -x (a nonzero sum of two binary32
                // values does not round to zero, a zero sum rounds to +0).
                uint8_t *dst = (((a.par0 + kl + 1) & 1) ? a.S8b : a.S8a) + (size_t)r * a.Np + ib;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    uint32_t f[16], xr[16], yr[16];
                    uint64_t v[8];
                    ptx::tmem_ld16(tmem + lane_off + kQColAcc + col0 + 16 * hh, f);
                    if (hh == 0) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            xr[j] = xpre[j];
                            yr[j] = ypre[j];
                        }
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            v[j] = vpre[j];
                    } else {
                        ptx::tmem_ld16(tmem + lane_off + kQColX + col0 + 16, xr);
                        ptx::tmem_ld16(tmem + lane_off + kQColY + col0 + 16, yr);
                        ptx::tmem_ld_wait(xr);
                        ptx::tmem_ld_wait(yr);
#pragma unroll
                        for (int j = 0; j < 16; j += 2)
                            v[j / 2] = f2_fma(pk2, f2_pack_bits(xr[j], xr[j + 1]), k2.z);
                    }
                    ptx::tmem_ld_wait(f);
                    uint32_t neg[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        const uint64_t u = f2_fma(k2.c0, f2_pack_bits(f[j], f[j + 1]), k2.z);
                        const uint64_t w = f2_sub(u, v[j / 2]);
                        const uint64_t wd = f2_fma(w, k2.dt, k2.z);
                        const uint64_t yt = f2_add(f2_pack_bits(yr[j], yr[j + 1]), wd);
                        const uint64_t qy = f2_fma(k2.q, yt, k2.z);
                        const uint32_t n0 = f2_lo(qy) < -__uint_as_float(xr[j]) ? 1u : 0u;
                        const uint32_t n1 = f2_hi(qy) < -__uint_as_float(xr[j + 1]) ? 1u : 0u;
                        neg[j / 4] |= (n0 << (8 * (j & 3) + 7)) | (n1 << (8 * ((j + 1) & 3) + 7));
                    }
                    // +1 = 0x38, -1 = 0xB8 (sign bit); padded spins publish 0
                    uint32_t wv[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        wv[m] = 0x38383838u | neg[m];
                    if (live != 0xFFFFFFFFu) {
#pragma unroll
                        for (int m = 0; m < 4; ++m)
                            wv[m] &= byte_mask4(live >> (16 * hh + 4 * m));
                    }
                    *reinterpret_cast<uint4 *>(dst + 16 * hh) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                }
                qepi_bar();
                if (et == 0 && !(sg == a.drop_mb && rho == 0)) {
                    // every epilogue thread's stores precede the barrier; the
                    // gpu-scope release (cumulative) publishes them with the flag
                    ptx::fence_proxy_async_global();
                    ptx::st_release_gpu(&a.flags[flag_index(sg, rho, a.nrb)], kl + 1);
                }
            }

            // ---- phase 2: energy of s(t_k) on evaluation passes, and the full
            // update of x and y in tensor memory
            int esum = 0;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t f[16], xr[16], yr[16];
                ptx::tmem_ld16(tmem + lane_off + kQColX + col0 + 16 * hh, xr);
                ptx::tmem_ld16(tmem + lane_off + kQColY + col0 + 16 * hh, yr);
                ptx::tmem_ld16(tmem + lane_off + kQColAcc + col0 + 16 * hh, f);
                ptx::tmem_ld_wait(xr);
                ptx::tmem_ld_wait(yr);
                ptx::tmem_ld_wait(f);
                if (e >= 0) {
                    uint8_t sb[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const bool lv = (live >> (16 * hh + j)) & 1u;
                        const float x0 = __uint_as_float(xr[j]);
                        const int fj = (int)__uint_as_float(f[j]);  // exact integer force
                        esum += lv ? (x0 >= 0.f ? fj : -fj) : 0;
                        sb[j] = lv ? fp8_sign(x0) : (uint8_t)0;
                    }
                    uint4 w;
                    w.x = pack4(sb[0], sb[1], sb[2], sb[3]);
                    w.y = pack4(sb[4], sb[5], sb[6], sb[7]);
                    w.z = pack4(sb[8], sb[9], sb[10], sb[11]);
                    w.w = pack4(sb[12], sb[13], sb[14], sb[15]);
                    *reinterpret_cast<uint4 *>(a.Snap + (size_t)e * plane + (size_t)r * a.Np + ib +
                                               16 * hh) = w;
                }
                if (!final_pass) {
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
                    ptx::tmem_st16(tmem + lane_off + kQColX + col0 + 16 * hh, xr);
                    ptx::tmem_st16(tmem + lane_off + kQColY + col0 + 16 * hh, yr);
                }
            }
            ptx::tc_fence_before();
            if (!final_pass)
                ptx::tmem_st_wait();
            __syncwarp();
            if (lane == 0)
                ptx::mbar_arrive_cluster(tmem_empty0);  // this warp has read the accumulator
            if (e >= 0) {
                sh->red[cg][q * 32 + lane] = esum;
                qepi_bar();
                if (et < kQM) {
                    const int s4 = sh->red[0][et] + sh->red[1][et] + sh->red[2][et] + sh->red[3][et];
                    a.Epart[((size_t)e * a.nblk + sg) * a.Rp + r0 + et] = (float)s4;
                }
            }
        }

        // final state back to global memory
        if (!left) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t xr[16], yr[16];
                ptx::tmem_ld16(tmem + lane_off + kQColX + col0 + 16 * hh, xr);
                ptx::tmem_ld16(tmem + lane_off + kQColY + col0 + 16 * hh, yr);
                ptx::tmem_ld_wait(xr);
                ptx::tmem_ld_wait(yr);
                float4 *xd = reinterpret_cast<float4 *>(a.X + (size_t)r * a.Np + ib + 16 * hh);
                float4 *yd = reinterpret_cast<float4 *>(a.Y + (size_t)r * a.Np + ib + 16 * hh);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    xd[v] = make_float4(__uint_as_float(xr[4 * v]), __uint_as_float(xr[4 * v + 1]),
                                        __uint_as_float(xr[4 * v + 2]),
                                        __uint_as_float(xr[4 * v + 3]));
                    yd[v] = make_float4(__uint_as_float(yr[4 * v]), __uint_as_float(yr[4 * v + 1]),
                                        __uint_as_float(yr[4 * v + 2]),
                                        __uint_as_float(yr[4 * v + 3]));
                }
            }
        }
    }

    // every role of both CTAs has left its loop: no issuer copies any more.
    // The even CTA then waits for the last copies of each stage from either
    // CTA; a last use some of whose copies were never made is completed here
    // (copies of use u are made only after the pair's MMAs have read use
    // u - 1, so only the last use of a stage can be incomplete).
    ptx::tc_fence_before();
    ptx::cluster_sync();
    if (h == 0 && threadIdx.x < kQStages) {
        // stage s: the copies of its last use (U - 1) from either CTA
        const int st = threadIdx.x;
        const int sL = sh->copies[st][0][0], jL = sh->copies[st][0][1];
        const int sP = sh->copies[st][1][0], jP = sh->copies[st][1][1];
        int U = sL > jL ? sL : jL;
        U = sP > U ? sP : U;
        U = jP > U ? jP : U;
        if (U > 0) {
            const uint32_t landing = (sL >= U ? kQStageA : 0) + (jL >= U ? kQStageJ : 0) +
                                     (sP >= U ? kQStageA : 0) + (jP >= U ? kQStageJ : 0);
            if (jL >= U) {
                // armed for both CTAs' copies: stand in for the missing ones
                if (landing < (uint32_t)kQStageBytes)
                    ptx::mbar_complete_tx(&sh->full[st], (uint32_t)kQStageBytes - landing);
            } else {
                // never armed: arm it for the copies that were made
                ptx::mbar_expect_tx(&sh->full[st], landing);
            }
            ptx::mbar_drain(&sh->full[st], (uint32_t)(U - 1) & 1u, a.err);
        }
    }
    // both CTAs' copies and MMAs are done with the pair's shared and tensor memory
    ptx::cluster_sync();
    ptx::tc_fence_after();
    if (warp == kQMmaWarp)
        ptx::tmem_dealloc_pair(tmem, kQTmemCols);
}

// ------------------------------------------------------------- host side ---

namespace {

cudaError_t pair_config(cudaLaunchConfig_t *cfg, cudaLaunchAttribute *attr, int nblk, int Rp,
                        cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(tc_fp8_pair_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQSmem);
    if (e != cudaSuccess)
        return e;
    *cfg = cudaLaunchConfig_t{};
    cfg->gridDim = dim3(2 * nblk, Rp / (2 * kQM), 1);
    cfg->blockDim = dim3(kQThreads, 1, 1);
    cfg->dynamicSmemBytes = kQSmem;
    cfg->stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg->attrs = attr;
    cfg->numAttrs = 1;
    return cudaSuccess;
}

}  // namespace

bool tc_pair_fits(int Np, int Rp)
{
    if (Np % kQK != 0 || Np / kQK < 1 || Np / kQK > kQMaxChunks || Rp % (2 * kQM) != 0 ||
        Rp < 2 * kQM)
        return false;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    if (pair_config(&cfg, attr, Np / kQK, Rp, nullptr) != cudaSuccess)
        return false;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, tc_fp8_pair_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (long long)(Np / kQK) * (Rp / (2 * kQM)) <= (long long)clusters;
}

cudaError_t launch_tc_fp8_pair(cudaStream_t st, const TcPlan *plan, const PersistArgs &a)
{
    if (!plan || a.Np != plan->Np || a.Rp > plan->Rp || a.Rp % (2 * kQM) != 0 ||
        a.nblk != a.Np / kQK || a.nblk > kQMaxChunks || a.nrb != a.Rp / kQM || a.nh ||
        a.trace_every > 0)
        return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = pair_config(&cfg, attr, a.nblk, a.Rp, st);
    if (e != cudaSuccess)
        return e;
    return cudaLaunchKernelEx(&cfg, tc_fp8_pair_kernel, plan->mapJ64, plan->mapB[0],
                              plan->mapB[1], a);
}

}  // namespace hsb
